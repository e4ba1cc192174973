"""The float path's arithmetic at high orders, run on the CPU.

`csrc/boys_f32_row.cuh` holds the per-argument code of the float path and
compiles for the host too.  `tests/precision/f32_rows_host.cpp` evaluates it
with g++ (correctly rounded sqrt and division, where the GPU uses its
approximations), and the rows are compared with the oracle at the float
arguments.  From n_max = 17 on the closed form carries its rational part in
float-float and the asymptote's chain is a compensated product (Graillat);
these pins fail if either scheme is broken, without a GPU.  The device's own
results are checked by the `-m gpu` parity tests.
"""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2504_07637_gb300", "csrc")
SRC = os.path.join(ROOT, "tests", "precision", "f32_rows_host.cpp")
FLT_MIN = float(np.finfo(np.float32).tiny)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("f32rows")
    exe = str(d / "f32_rows_host")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, SRC, "-o", exe])
    return exe, d


def _cutoff(n_top):
    with open(os.path.join(ROOT, "paper_2504_07637_gb300", "coeffs", "boys_fit_b24_plus1.json")) as fh:
        return {r["n"]: float(r["z"]) for r in json.load(fh)["fits"]}[n_top]


def _rows(harness, n_max, mode, x):
    exe, d = harness
    xf, of = d / f"x{n_max}_{mode}.bin", d / f"o{n_max}_{mode}.bin"
    x.astype(np.float32).tofile(xf)
    subprocess.check_call([exe, str(n_max), str(mode), str(xf), str(of)])
    return np.fromfile(of, dtype=np.float32).reshape(x.size, n_max + 1).astype(np.float64)


def _rel(got, ref):
    ok = ref >= FLT_MIN
    return np.where(ok, np.abs(got - ref) / np.where(ok, ref, 1.0), 0.0).max(axis=0)


@pytest.mark.parametrize("n_max,bound", [(8, 1.0e-6), (16, 1.6e-6), (17, 1.2e-6), (24, 1.2e-6), (36, 1.4e-6)])
def test_closed_form_below_the_cutoff(harness, oracle_mod, n_max, bound):
    z = _cutoff(n_max if n_max <= 8 else n_max + 1)
    rng = np.random.default_rng(n_max)
    x = np.concatenate([np.linspace(0, z, 1 << 15, endpoint=False), rng.uniform(0, z, 1 << 15)]).astype(np.float32)
    rel = _rel(_rows(harness, n_max, 0, x), oracle_mod.boys(x.astype(np.float64), n_max))
    assert rel.max() <= bound, (n_max, rel.max(), int(rel.argmax()))


@pytest.mark.parametrize("n_max", [17, 24, 36])
def test_compensated_chain_above_the_cutoff(harness, oracle_mod, n_max):
    # within about one rounding of the exact chain at every m (the plain chain
    # of two roundings per order reaches 2.5e-6 at m = 36)
    z = _cutoff(n_max + 1)
    rng = np.random.default_rng(100 + n_max)
    x = np.exp(rng.uniform(np.log(z), np.log(2e5), 1 << 16)).astype(np.float32)
    rel = _rel(_rows(harness, n_max, 1, x), oracle_mod.boys(x.astype(np.float64), n_max))
    assert rel.max() <= 4e-7, (n_max, rel.max(), int(rel.argmax()))


def test_plain_chain_grows_where_the_compensated_one_does_not(harness, oracle_mod):
    # n_max = 16 keeps the plain chain; its error grows with m (the reason for
    # the compensated product above 16)
    rng = np.random.default_rng(7)
    x = np.exp(rng.uniform(np.log(_cutoff(17)), np.log(2e5), 1 << 16)).astype(np.float32)
    rel = _rel(_rows(harness, 16, 1, x), oracle_mod.boys(x.astype(np.float64), 16))
    assert rel[16] > 3 * rel[1] and rel[16] > 8e-7, rel
