"""GB300-native evaluation of the Boys functions F_m(x), m = 0..n_max, with the
closed-form global approximation of Laikov (arXiv 2504.07637).

The compute path is libboys.so (CUDA for sm_103a) behind a C ABI
(``include/boys.h``); ``api`` wraps it for torch tensors.  Importing this
package does not import torch; the wrappers load it on first use.
"""
from ._capi import BoysError  # noqa: F401

_API = ("boys", "boys_contract", "boys_from_host", "boys_backward", "boys_autograd", "BoysFunction", "RaggedBatch",
        "ragged_variants", "cutoff", "max_n", "top_order_f64", "top_order_f32")


def __getattr__(name):
    if name in _API:
        from . import api

        return getattr(api, name)
    raise AttributeError(name)
