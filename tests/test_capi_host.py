"""The C-ABI library builds, loads and exports every declared symbol; its
host-side argument checks answer before any CUDA call (no GPU needed)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    import shutil

    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2504_07637_gb300 import _capi
    from paper_2504_07637_gb300.build import build_library

    build_library()
    return _capi


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(boys_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(capi):
    lib = capi.load()
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(capi.SIGNATURES) == declared


def test_host_argument_checks(capi):
    f = capi.load().boys_eval_f64
    assert f(8, -1, 8, 8, None) == 2  # count < 0
    assert f(8, 10, -1, 8, None) == 3  # n_max < 0
    assert f(8, 10, capi.load().boys_max_n(53) + 1, 8, None) == 3
    assert f(None, 0, 8, None, None) == 0  # empty is a no-op
    assert f(None, 5, 8, 8, None) == 1  # null input
    assert f(8, 5, 8, None, None) == 1  # null output
    assert f(0x1004, 5, 8, 0x2000, None) == 4  # misaligned double pointer
    assert f(8, 2**62, 8, 8, None) == 2  # row count overflows int64


def test_status_strings(capi):
    for code in range(9):
        assert capi.status_string(code)
    assert capi.status_string(0) == "ok"


def test_table_metadata(capi, oracle_mod):
    lib = capi.load()
    assert lib.boys_max_n(53) == 36
    for n in range(0, 42):
        assert abs(lib.boys_cutoff(n, 53) / oracle_mod.cutoff(n, 53) - 1) < 1e-13
    assert np.isnan(lib.boys_cutoff(99, 53))
    assert [lib.boys_top_order_f64(k) for k in (0, 3, 4, 8, 13, 23, 36, 37)] == [0, 3, 5, 9, 15, 26, 40, -1]


def test_backward_host_argument_checks(capi):
    f = capi.load().boys_eval_backward_f64
    # (x, F, ld_F, g, g_row, g_col, count, n_max, grad, stream)
    assert f(8, 8, 10, 8, 9, 1, -1, 8, 8, None) == 2  # count < 0
    assert f(8, 8, 10, 8, 9, 1, 10, 36, 8, None) == 3  # needs F_{n_max+1}
    assert f(8, 8, 10, 8, -9, 1, 10, 8, 8, None) == 7  # negative stride
    assert f(8, 8, 9, 8, 9, 1, 10, 8, 8, None) == 7  # ld_F < n_max + 2
    assert f(8, 8, 10, None, 9, 1, 10, 8, 8, None) == 1  # no gradient
    assert f(None, None, 0, 8, 9, 1, 10, 8, 8, None) == 1  # neither F nor x
    assert f(8, 8, 10, 8, 9, 1, 0, 8, 8, None) == 0  # empty
    assert f(8, 0x1004, 10, 8, 9, 1, 10, 8, 8, None) == 4  # misaligned F


def test_ragged_host_argument_checks(capi):
    lib = capi.load()
    f = lib.boys_eval_ragged_f64
    need = lib.boys_ragged_workspace_bytes(10)
    assert need == 256 + 8 * 11 + 4 * 10  # counters, the tile prefix (R + 1) and the request order (R)
    # (x, x_size, offsets, n_max, out_offsets, R, out, out_size, ws, ws_bytes, variant, stream)
    assert f(8, 10, 8, 4, 8, -1, 8, 10, 256, need, -1, None) == 2  # R < 0
    assert f(8, 10, 8, 4, 8, 0, 8, 10, 256, need, -1, None) == 0  # empty batch
    assert f(8, 10, 8, 4, 8, 10, 8, 10, 256, need - 8, -1, None) == 5  # workspace too small
    assert f(8, 10, 8, 4, 8, 10, 8, 10, 256, need, 99, None) == 7  # no such variant
    assert f(8, 10, 8, 4, 8, 10, 8, 10, 264, need, -1, None) == 4  # workspace not 256-aligned
    assert f(8, 10, None, 4, 8, 10, 8, 10, 256, need, -1, None) == 1  # missing offsets
    assert lib.boys_ragged_max_n() == 16
    assert lib.boys_ragged_num_variants() >= 2
