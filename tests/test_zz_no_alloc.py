"""The allocation-free selection entry point against the regular one.

panache_topk_row_noalloc serves callers that cannot allocate device memory
(code inside another framework's memory pool, or under a budget that forbids
new allocations): all of its scratch is one fixed array inside the library.
These tests take the profile rows left by a regular panache_pmp call, run the
allocation-free selection on them twice in a row through the C ABI, and
check that both calls report the same motifs as the regular call; that the
calls take nothing from the device's stream-ordered memory pool (the one the
regular path allocates from); that a pool overflow is reported and leaves the
output alone, and that the next call starts from cleared scratch.  They run
last (file name) so that a failure here cannot hide earlier results.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MOTIF_BYTES = 32


@pytest.fixture(scope="module")
def pn():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2607_17481_b300 as pkg
    from paper_2607_17481_b300 import build
    build.build()
    return pkg


def _pool():
    """The device's current stream-ordered memory pool (cuda-bindings)."""
    from cuda.bindings import runtime as cudart
    err, pool = cudart.cudaDeviceGetMemPool(torch.cuda.current_device())
    assert err == cudart.cudaError_t.cudaSuccess
    return cudart, pool


def _pool_marks_reset():
    from cuda.bindings import driver
    cudart, pool = _pool()
    for attr in (cudart.cudaMemPoolAttr.cudaMemPoolAttrUsedMemHigh,
                 cudart.cudaMemPoolAttr.cudaMemPoolAttrReservedMemHigh):
        err, = cudart.cudaMemPoolSetAttribute(pool, attr, driver.cuuint64_t(0))
        assert err == cudart.cudaError_t.cudaSuccess


def _pool_marks():
    cudart, pool = _pool()
    out = []
    for attr in (cudart.cudaMemPoolAttr.cudaMemPoolAttrUsedMemHigh,
                 cudart.cudaMemPoolAttr.cudaMemPoolAttrReservedMemHigh,
                 cudart.cudaMemPoolAttr.cudaMemPoolAttrUsedMemCurrent,
                 cudart.cudaMemPoolAttr.cudaMemPoolAttrReservedMemCurrent):
        err, v = cudart.cudaMemPoolGetAttribute(pool, attr)
        assert err == cudart.cudaError_t.cudaSuccess
        out.append(int(v))
    return out


def _noalloc(pn, x, keys_row, m, k):
    from paper_2607_17481_b300 import native
    x_dev = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    keys_dev = torch.from_numpy(np.ascontiguousarray(keys_row).view(np.int64)).cuda()
    out = torch.zeros(k * MOTIF_BYTES, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    stream.synchronize()
    _pool_marks_reset()
    before = _pool_marks()
    results = []
    for _ in range(2):
        out.zero_()
        cnt.fill_(-99)
        rc = native.topk_row_noalloc(x_dev, keys_dev, m, k, 1e-6, out, cnt, stream.cuda_stream)
        assert rc == 0
        stream.synchronize()
        c = int(cnt.item())
        assert c >= 0
        mot = out.cpu().numpy().view(native.MOTIF_DTYPE)[:c].copy()
        results.append(mot)
    after = _pool_marks()
    # the high-water marks were reset to the current use just before the calls:
    # nothing the calls did raised them
    assert after[0] <= before[2] and after[1] <= before[3], (before, after)
    return results


def _same(a, b):
    assert len(a) == len(b)
    for ra, rb in zip(a, b):
        assert (int(ra["m"]), int(ra["i"]), int(ra["j"])) == (int(rb["m"]), int(rb["i"]), int(rb["j"]))
        assert abs(float(ra["d"]) - float(rb["d"])) <= 1e-9 * float(rb["d"]) + 1e-12


def test_single_length_matches_pmp(pn):
    s = workloads.planted_random_walk()
    n = s.x.shape[0]
    ctx = pn.Context(topk_mode=pn.TOPK_GLOBAL)
    ref = ctx.pmp(s.x, 40, 40, 20, s.excl)
    rows = ctx.profile_rows(0, n, 1)
    first, second = _noalloc(pn, s.x, rows[0], 40, 20)
    _same(first, ref)
    _same(second, ref)


def test_rows_of_per_length_run(pn):
    s = workloads.planted_random_walk()
    n = s.x.shape[0]
    ctx = pn.Context(topk_mode=pn.TOPK_PER_LENGTH)
    ref = ctx.pmp(s.x, s.m_min, s.m_max, s.k, s.excl)
    rows = ctx.profile_rows(0, n, s.m_max - s.m_min + 1)
    for m in (32, 47, 64):
        want = ref[ref["m"] == m]
        first, second = _noalloc(pn, s.x, rows[m - s.m_min], m, s.k)
        _same(first, want)
        _same(second, want)


def test_pool_overflow_reported_then_cleared(pn):
    """A row whose cells all snap to zero (every window repeats 50 samples
    later) overflows the 8192-cell pool: the call reports EPOOL through the
    count and leaves the output untouched; the next call on the same device
    starts from cleared scratch and matches the regular selection."""
    from paper_2607_17481_b300 import native
    n, m, k = 20000, 40, 20
    t = np.arange(n)
    x = np.sin(2 * np.pi * t / 50.0) + 0.3 * np.sin(2 * np.pi * t / 25.0)
    j = np.where(t + 50 <= n - m, t + 50, t - 50).astype(np.int64)
    keys = j.copy()                                     # pack(0.0, j): distance bits zero
    keys[t > n - m] = -1                                # cells past the last window are empty
    x_dev = torch.from_numpy(x).cuda()
    keys_dev = torch.from_numpy(keys).cuda()
    out = torch.full((k * MOTIF_BYTES,), 0xAB, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    assert native.topk_row_noalloc(x_dev, keys_dev, m, k, 1e-6, out, cnt, stream.cuda_stream) == 0
    stream.synchronize()
    assert int(cnt.item()) == native.EPOOL
    assert bool((out == 0xAB).all())
    # the same scratch, next call: a normal row is selected exactly
    s = workloads.planted_random_walk()
    ctx = pn.Context(topk_mode=pn.TOPK_GLOBAL)
    ref = ctx.pmp(s.x, 40, 40, 20, s.excl)
    rows = ctx.profile_rows(0, s.x.shape[0], 1)
    first, second = _noalloc(pn, s.x, rows[0], 40, 20)
    _same(first, ref)
    _same(second, ref)


def test_limit_boundary(pn):
    """k (m + 1) = NOALLOC_NEED_MAX is accepted, one more motif is not."""
    from paper_2607_17481_b300 import native
    n, m = 8192, 125                                     # m + 1 = 126 divides 6300
    k = native.NOALLOC_NEED_MAX // (m + 1)
    assert k * (m + 1) == native.NOALLOC_NEED_MAX
    x = torch.from_numpy(np.random.default_rng(3).standard_normal(n)).cuda()
    keys = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    out = torch.zeros((k + 1) * MOTIF_BYTES, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    assert native.topk_row_noalloc(x, keys, m, k, 1e-6, out, cnt, stream.cuda_stream) == 0
    stream.synchronize()
    assert int(cnt.item()) == 0                         # every cell empty: no motif
    assert native.topk_row_noalloc(x, keys, m, k + 1, 1e-6, out, cnt, stream.cuda_stream) == native.EINVAL


def test_rejects_out_of_range(pn):
    from paper_2607_17481_b300 import native
    x = torch.zeros(1000, dtype=torch.float64, device="cuda")
    keys = torch.full((1000,), -1, dtype=torch.int64, device="cuda")
    out = torch.zeros(64 * MOTIF_BYTES, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert native.topk_row_noalloc(x, keys, 2, 5, 1e-6, out, cnt) == native.EINVAL        # m < 3
    assert native.topk_row_noalloc(x, keys, 500, 64, 1e-6, out, cnt) == native.EINVAL     # pool too small


def test_binding_rejects_bad_buffers(pn):
    """The binding refuses buffers the kernels would overrun, before any launch."""
    from paper_2607_17481_b300 import native
    n = 1000
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    keys = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    out = torch.zeros(5 * MOTIF_BYTES, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    bad = [
        (x.float(), keys, out, cnt),                         # float32 samples
        (x.cpu(), keys, out, cnt),                           # host samples
        (x, keys[:-1], out, cnt),                            # one key short
        (x, keys.int(), out, cnt),                           # 32-bit keys
        (x, keys, out[:-1], cnt),                            # out smaller than k motifs
        (x, keys, out, cnt.long()),                          # 64-bit count
        (torch.zeros(2 * n, dtype=torch.float64, device="cuda")[::2], keys, out, cnt),   # strided
    ]
    for args in bad:
        with pytest.raises(ValueError):
            native.topk_row_noalloc(args[0], args[1], 40, 5, 1e-6, args[2], args[3])
