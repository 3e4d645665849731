"""The allocation-free BFS entry point against the oracle and the
context-based entry point.

percis_bfs_noalloc serves callers that cannot allocate device memory (a
process whose memory pool owns the whole GPU, or a path that cannot take
cudaMalloc's implicit synchronisation).  Its scratch is a fixed array inside
the library, shared by every call.  This file is collected last so a run that
stops at the first failure has already run every other test; it also passes
when run alone in a fresh process.
"""
import numpy as np
import pytest

import oracle
from paper_2509_11454_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

OK, INVALID, TIMEOUT = 0, 1, 5


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


def _noalloc(binding, g, irp_d, icol_d, src, tgt, timeout_s=0.0):
    rp_d, col_d = _dev(g.row_ptr), _dev(g.col)
    dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
    sig = torch.empty(g.n, dtype=torch.float64, device="cuda")
    ovf = []
    st = binding.percis_bfs_noalloc(g.n, rp_d, col_d, irp_d, icol_d, src, tgt, dist, sig,
                                    torch.cuda.current_stream().cuda_stream, timeout_s, ovf)
    torch.cuda.synchronize()
    return st, dist.cpu().numpy(), sig.cpu().numpy(), ovf[0]


def _check_oracle(og, src, tgt, dist, sig, ovf):
    ret, d_o, s_o, _, _, ovf_o = oracle.bfs(og, src, tgt)
    np.testing.assert_array_equal(dist, d_o)
    exact = s_o < 2.0 ** 53
    np.testing.assert_array_equal(sig[exact], s_o[exact])  # path counts are exact below 2^53
    assert bool(ovf) == ovf_o


@pytest.mark.parametrize("name", ["ba", "rmat"])
def test_noalloc_matches_oracle_and_context_bfs_twice(binding, name):
    if name == "ba":
        g = synth.barabasi_albert(5000, 4, 3)
        irp = icol = None
    else:
        g = synth.rmat(12, 8, 0.57, 0.19, 0.19, 4)
        irp, icol = _transpose(g)
    og = oracle.from_synth(g)
    eng = binding.PercIS(0)
    eng.load_csr(g.row_ptr, g.col, directed=g.directed)
    irp_d = _dev(irp) if irp is not None else None
    icol_d = _dev(icol) if icol is not None else None
    rng = np.random.default_rng(0)
    # calls in a row (full, truncated, target = source) share the scratch array
    s1, s2 = int(rng.integers(g.n)), int(rng.integers(g.n))
    for src, tgt in [(s1, -1), (s2, int(rng.integers(g.n))), (s1, s1)]:
        st, dist, sig, ovf = _noalloc(binding, g, irp_d, icol_d, src, tgt)
        assert st == OK
        _check_oracle(og, src, tgt, dist, sig, ovf)
        rd, rs = eng.bfs(src, tgt)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(dist, rd.cpu().numpy())
        np.testing.assert_array_equal(sig, rs.cpu().numpy())
    eng.close()


def test_noalloc_flags_sigma_overflow(binding):
    """A chain of complete bipartite layers of width 8: sigma = 8^(k-1) at
    layer k passes 2^53 at layer 19; both entry points raise the flag then,
    and not on the chain cut before it."""
    width = 8
    for layers, expect in [(20, True), (17, False)]:
        src, dst = [0] * width, list(range(1, width + 1))
        for k in range(layers - 1):
            a = 1 + k * width
            for i in range(width):
                for j in range(width):
                    src.append(a + i)
                    dst.append(a + width + j)
        g = synth.csr_from_edges(1 + layers * width, np.array(src), np.array(dst), directed=False)
        st, dist, sig, ovf = _noalloc(binding, g, None, None, 0, -1)
        assert st == OK and bool(ovf) == expect
        _check_oracle(oracle.from_synth(g), 0, -1, dist, sig, ovf)
        eng = binding.PercIS(0)
        eng.load_csr(g.row_ptr, g.col, directed=False)
        d_ = torch.empty(g.n, dtype=torch.int32, device="cuda")
        s_ = torch.empty(g.n, dtype=torch.float64, device="cuda")
        assert binding.percis_bfs(eng.ctx, 0, -1, d_, s_) == expect
        eng.close()


def test_noalloc_skips_out_of_range_column(binding):
    """A column index outside [0, n) is skipped and reported as INVALID; the
    outputs hold the traversal of the graph without that entry."""
    g = synth.path_graph(10)
    row = 3
    at = int(g.row_ptr[row + 1])
    col = np.insert(g.col, at, np.int32(1_000_000))
    rp = g.row_ptr.copy()
    rp[row + 1:] += 1
    bad = synth.Graph(n=10, row_ptr=rp, col=col, directed=False)
    st, dist, sig, _ = _noalloc(binding, bad, None, None, 0, -1)
    assert st == INVALID
    _check_oracle(oracle.from_synth(g), 0, -1, dist, sig, False)
    # the next call on the same scratch array is unaffected
    st, dist, sig, ovf = _noalloc(binding, g, None, None, 9, -1)
    assert st == OK
    _check_oracle(oracle.from_synth(g), 9, -1, dist, sig, ovf)


def test_noalloc_wait_budget_runs_out_then_recovers(binding):
    """A 1 ns budget makes the grid-wide waits give up: TIMEOUT, and the next
    call (default budget) on the same scratch array is correct."""
    g = synth.barabasi_albert(3000, 3, 5)
    st, *_ = _noalloc(binding, g, None, None, 1, -1, timeout_s=1e-9)
    assert st == TIMEOUT
    st, dist, sig, ovf = _noalloc(binding, g, None, None, 1, -1)
    assert st == OK
    _check_oracle(oracle.from_synth(g), 1, -1, dist, sig, ovf)


def test_noalloc_refuses_a_capturing_stream(binding):
    g = synth.path_graph(10)
    _noalloc(binding, g, None, None, 0, -1)  # device set-up outside the capture
    rp_d, col_d = _dev(g.row_ptr), _dev(g.col)
    dist = torch.full((10,), 7, dtype=torch.int32, device="cuda")
    sig = torch.empty(10, dtype=torch.float64, device="cuda")
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.graph(graph, stream=side):
        st = binding.percis_bfs_noalloc(10, rp_d, col_d, None, None, 0, -1, dist, sig,
                                        torch.cuda.current_stream().cuda_stream)
    assert st == INVALID
    torch.cuda.synchronize()
    assert dist.cpu().tolist() == [7] * 10  # no work was issued


def test_noalloc_rejects_oversize_and_bad_vertices(binding):
    g = synth.path_graph(10)
    rp_d, col_d = _dev(g.row_ptr), _dev(g.col)
    dist = torch.empty(10, dtype=torch.int32, device="cuda")
    sig = torch.empty(10, dtype=torch.float64, device="cuda")
    assert binding.percis_bfs_noalloc(1048577, rp_d, col_d, None, None, 0, -1, dist, sig) == INVALID
    assert binding.percis_bfs_noalloc(10, rp_d, col_d, None, None, 10, -1, dist, sig) == INVALID
    assert binding.percis_bfs_noalloc(10, rp_d, col_d, None, None, 0, -1, dist, sig) == OK
    torch.cuda.synchronize()
    assert dist.cpu().tolist() == list(range(10))
