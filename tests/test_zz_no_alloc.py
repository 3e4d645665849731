"""The allocation-free BFS entry point against the context-based one.

percis_bfs_noalloc serves callers that cannot allocate device memory (a
process whose memory pool owns the whole GPU, or a path that cannot take
cudaMalloc's implicit synchronisation).  Its scratch is a fixed array inside
the library, shared by every call.  This file is collected last so a run that
stops at the first failure has already run every other test; it also passes
when run alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2509_11454_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_11454_gb300 import binding as b, build_lib

    build_lib.build()
    b.load_library()
    return b


def _transpose(g):
    """In-adjacency of a directed CSR (sources ascending), built on the host."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    order = np.lexsort((rows, g.col))
    icol = rows[order].astype(np.int32)
    irp = np.zeros(g.n + 1, dtype=np.int64)
    np.cumsum(np.bincount(g.col, minlength=g.n), out=irp[1:])
    return irp, icol


def _dev(a):
    return torch.as_tensor(a, device="cuda")


@pytest.mark.parametrize("name", ["ba", "rmat"])
def test_noalloc_matches_context_bfs_twice(binding, name):
    if name == "ba":
        g = synth.barabasi_albert(5000, 4, 3)
        irp = icol = None
    else:
        g = synth.rmat(12, 8, 0.57, 0.19, 0.19, 4)
        irp, icol = _transpose(g)
    eng = binding.PercIS(0)
    eng.load_csr(g.row_ptr, g.col, directed=g.directed)
    rp_d, col_d = _dev(g.row_ptr), _dev(g.col)
    irp_d = _dev(irp) if irp is not None else None
    icol_d = _dev(icol) if icol is not None else None
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(0)
    # two calls in a row (different sources and targets) share the scratch array
    for src, tgt in [(int(rng.integers(g.n)), -1), (int(rng.integers(g.n)), int(rng.integers(g.n)))]:
        dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
        sig = torch.empty(g.n, dtype=torch.float64, device="cuda")
        st = binding.percis_bfs_noalloc(g.n, rp_d, col_d, irp_d, icol_d, src, tgt, dist, sig, stream)
        assert st == 0
        rd, rs = eng.bfs(src, tgt)
        torch.cuda.synchronize()
        assert torch.equal(dist, rd)
        # sigma is exact below 2^53 in both
        assert torch.equal(sig, rs)
    eng.close()


def test_noalloc_rejects_oversize_and_bad_vertices(binding):
    g = synth.path_graph(10)
    rp_d, col_d = _dev(g.row_ptr), _dev(g.col)
    dist = torch.empty(10, dtype=torch.int32, device="cuda")
    sig = torch.empty(10, dtype=torch.float64, device="cuda")
    assert binding.percis_bfs_noalloc(1048577, rp_d, col_d, None, None, 0, -1, dist, sig) == 1
    assert binding.percis_bfs_noalloc(10, rp_d, col_d, None, None, 10, -1, dist, sig) == 1
    assert binding.percis_bfs_noalloc(10, rp_d, col_d, None, None, 0, -1, dist, sig) == 0
    torch.cuda.synchronize()
    assert dist.cpu().tolist() == list(range(10))
