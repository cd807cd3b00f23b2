"""The allocation-free selection entry point against the regular one.

panache_topk_row_noalloc serves callers that cannot allocate device memory
(code inside another framework's memory pool, or under a budget that forbids
new allocations): all of its scratch is one fixed array inside the library.
This test takes the profile rows left by a regular panache_pmp call, runs the
allocation-free selection on them twice in a row through the C ABI, and
checks that both calls report the same motifs as the regular call.  It runs
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


def _noalloc(pn, x, keys_row, m, k):
    from paper_2607_17481_b300 import native
    x_dev = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    keys_dev = torch.from_numpy(np.ascontiguousarray(keys_row).view(np.int64)).cuda()
    out = torch.zeros(k * MOTIF_BYTES, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
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


def test_rejects_out_of_range(pn):
    from paper_2607_17481_b300 import native
    x = torch.zeros(1000, dtype=torch.float64, device="cuda")
    keys = torch.full((1000,), -1, dtype=torch.int64, device="cuda")
    out = torch.zeros(64 * MOTIF_BYTES, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert native.topk_row_noalloc(x, keys, 2, 5, 1e-6, out, cnt) == native.EINVAL        # m < 3
    assert native.topk_row_noalloc(x, keys, 500, 64, 1e-6, out, cnt) == native.EINVAL     # pool too small
