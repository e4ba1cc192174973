"""Out-of-bounds writes, found without compute-sanitizer: every entry point
writes into a buffer whose padding before and after the output holds a
signalling-NaN canary.  After the call the canaries must be intact and no
element of the output may still hold one (every element written once).

The cases cover both FP64 row layouts (rows kept in registers below
n_max = 12, staged through shared memory from 12 on), both launch shapes
(at most 2^20 arguments and above), the two-point path, the float path, the
fused contractions, both backward modes and every ragged launch variant."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

PAD = 4096  # elements of canary on each side
CANARY64 = np.int64(0x7FF0DEADBEEF0001)  # a signalling NaN
CANARY32 = np.int32(0x7F80DEAD)
SMALL_MAX = 1 << 20  # largest count with the small launch shape


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_07637_gb300 import _capi, workloads
    from paper_2504_07637_gb300.build import build_library

    build_library()
    return torch, _capi, workloads


def _padded(torch, n, f32=False):
    """A canary-filled buffer of n + 2 PAD elements and the address of element PAD."""
    if f32:
        buf = torch.full((n + 2 * PAD,), int(CANARY32), dtype=torch.int32, device="cuda")
        return buf, buf.data_ptr() + PAD * 4
    buf = torch.full((n + 2 * PAD,), int(CANARY64), dtype=torch.int64, device="cuda")
    return buf, buf.data_ptr() + PAD * 8


def _check(torch, buf, n, f32=False):
    torch.cuda.synchronize()
    h = buf.cpu().numpy()
    canary = CANARY32 if f32 else CANARY64
    assert np.all(h[:PAD] == canary), "write before the output"
    assert np.all(h[PAD + n:] == canary), "write after the output"
    assert not np.any(h[PAD:PAD + n] == canary), "output element left unwritten"


def _x(torch, workloads, count, f32=False, seed=3):
    x = workloads.scale(count, seed=seed)
    x[:: 97] = 0.0  # exact zeros among them
    return torch.from_numpy(x.astype(np.float32) if f32 else x).cuda()


COUNTS = [1, 33, 4097, SMALL_MAX, SMALL_MAX + 7]


@pytest.mark.parametrize("n_max", [0, 8, 11, 12, 16, 23, 36])
@pytest.mark.parametrize("count", COUNTS)
def test_rows_f64(env, n_max, count):
    torch, capi, workloads = env
    x = _x(torch, workloads, count)
    n = count * (n_max + 1)
    buf, ptr = _padded(torch, n)
    capi.call("boys_eval_f64", x.data_ptr(), count, n_max, ptr, torch.cuda.current_stream().cuda_stream)
    _check(torch, buf, n)


@pytest.mark.parametrize("n_max", [2, 11, 12, 36])
@pytest.mark.parametrize("count", [33, 4097, SMALL_MAX + 7])
def test_rows_f64_two_point(env, n_max, count):
    torch, capi, workloads = env
    x = _x(torch, workloads, count)
    n = count * (n_max + 1)
    buf, ptr = _padded(torch, n)
    capi.call("boys_eval_f64_two_point", x.data_ptr(), count, n_max, ptr, torch.cuda.current_stream().cuda_stream)
    _check(torch, buf, n)


@pytest.mark.parametrize("n_max", [0, 8, 9, 16, 17, 36])
@pytest.mark.parametrize("count", [1, 33, 1025, 4097, (1 << 22) + 5])
def test_rows_f32(env, n_max, count):
    torch, capi, workloads = env
    x = _x(torch, workloads, count, f32=True)
    n = count * (n_max + 1)
    buf, ptr = _padded(torch, n, f32=True)
    capi.call("boys_eval_f32", x.data_ptr(), count, n_max, ptr, torch.cuda.current_stream().cuda_stream)
    _check(torch, buf, n, f32=True)


@pytest.mark.parametrize("f32", [False, True])
@pytest.mark.parametrize("n_max", [0, 8, 16])
@pytest.mark.parametrize("count", [33, 4097, SMALL_MAX + 7])
def test_contraction(env, f32, n_max, count):
    torch, capi, workloads = env
    x = _x(torch, workloads, count, f32=f32)
    dt = torch.float32 if f32 else torch.float64
    c = torch.linspace(-1.0, 1.0, n_max + 1, dtype=dt, device="cuda")
    buf, ptr = _padded(torch, count, f32=f32)
    fn = "boys_eval_contract_f32" if f32 else "boys_eval_contract_f64"
    capi.call(fn, x.data_ptr(), count, n_max, c.data_ptr(), 0, 1, ptr, torch.cuda.current_stream().cuda_stream)
    _check(torch, buf, count, f32=f32)


@pytest.mark.parametrize("saved", [False, True])
@pytest.mark.parametrize("n_max", [0, 8, 20])
@pytest.mark.parametrize("count", [33, 4097, SMALL_MAX + 7])
def test_backward(env, saved, n_max, count):
    torch, capi, workloads = env
    x = _x(torch, workloads, count)
    g = torch.linspace(-1.0, 1.0, n_max + 1, dtype=torch.float64, device="cuda")
    F, ld = None, 0
    if saved:
        F = torch.empty((count, n_max + 2), dtype=torch.float64, device="cuda")
        capi.call("boys_eval_f64", x.data_ptr(), count, n_max + 1, F.data_ptr(), torch.cuda.current_stream().cuda_stream)
        ld = n_max + 2
    buf, ptr = _padded(torch, count)
    capi.call("boys_eval_backward_f64", x.data_ptr(), F.data_ptr() if saved else 0, ld, g.data_ptr(), 0, 1, count,
              n_max, ptr, torch.cuda.current_stream().cuda_stream)
    _check(torch, buf, count)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_ragged_variants(env, variant):
    torch, capi, workloads = env
    rng = np.random.default_rng(40 + variant)
    R = 300
    counts = np.floor(np.exp(rng.uniform(0, np.log(20000), R))).astype(np.int64)
    counts[:3] = [0, 1, 4097]
    n_max = rng.integers(0, 17, R).astype(np.int32)
    offsets = np.zeros(R + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    out_offsets = np.zeros(R + 1, dtype=np.int64)
    np.cumsum(counts * (n_max.astype(np.int64) + 1), out=out_offsets[1:])
    total = int(out_offsets[-1])
    x = torch.from_numpy(workloads.plain(int(offsets[-1]), 53, seed=variant)).cuda()
    od, nd, ood = (torch.from_numpy(a).cuda() for a in (offsets, n_max, out_offsets))
    lib = capi.load()
    ws_bytes = lib.boys_ragged_workspace_bytes(R)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    buf, ptr = _padded(torch, total)
    capi.call("boys_eval_ragged_f64", x.data_ptr(), x.numel(), od.data_ptr(), nd.data_ptr(), ood.data_ptr(), R, ptr,
              total, ws.data_ptr(), ws_bytes, variant, torch.cuda.current_stream().cuda_stream)
    _check(torch, buf, total)
