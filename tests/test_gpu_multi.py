"""Many independent graphs in one context (block-diagonal CSR): every graph's
estimate, sample-size bound and gradient against the oracle run on that graph
alone with its sample indices starting where the batch numbering puts them."""
import numpy as np
import pytest

import oracle
from paper_2509_11454_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SIZES = [300, 1200, 200, 2500, 800, 150, 600, 3000, 400, 1000, 90, 2000]


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_11454_gb300 import binding as b

    b.load_library()
    return b


@pytest.fixture(scope="module")
def batch():
    graphs = synth.graph_batch(SIZES, 5)
    vptr, rp, col = synth.union_csr(graphs)
    x = synth.states_uniform(int(vptr[-1]), 5)
    return graphs, vptr, rp, col, x


def _engine(binding, batch, **opts):
    graphs, vptr, rp, col, x = batch
    eng = binding.PercIS(0)
    if opts:
        eng.set_options(**opts)
    eng.load_graphs(vptr, rp, col)
    eng.set_states(x)
    return eng


@pytest.mark.parametrize("form", ["batched", "bidir"])
def test_fixed_sample_sizes_match_oracle_per_graph(binding, batch, form):
    graphs, vptr, rp, col, x = batch
    ell1, ell = 500, 1500
    eng = _engine(binding, batch, ell1=ell1, ell=ell, form=form)
    pc, infos = eng.estimate_graphs(0.05, 0.1, seed=3)
    pc = pc.cpu().numpy()
    assert len(infos) == len(graphs)
    gvec = np.random.default_rng(9).standard_normal(int(vptr[-1]))
    gx = eng.backward(torch.as_tensor(gvec, device="cuda")).cpu().numpy()
    for g, G in enumerate(graphs):
        og = oracle.from_synth(G)
        lo, hi = vptr[g], vptr[g + 1]
        xg = x[lo:hi]
        res = oracle.percis(og, xg, 0.05, 0.1, 3, ell1=ell1, ell=ell, offsets=(g * ell1, g * ell),
                            bidir=form == "bidir")
        assert infos[g]["ell"] == ell and infos[g]["vertex_diam"] == res.D
        assert infos[g]["rho_tilde"] == res.rho_tilde
        if res.phase1.overflow or res.phase2.overflow:
            # a path count passed 2^53: FP64 counts on both sides, summed in other
            # orders, so only the flag and the count-free quantities are compared
            assert infos[g]["sigma_overflow"] == 1, g
            continue
        assert np.max(np.abs(pc[lo:hi] - res.pc)) <= 1e-9, g
        prep = oracle.prepare(xg, cv_method="sorted")
        F = prep.lam * res.phase2.cnt / ell
        ref = oracle.vjp_fixed(prep, ell, res.phase2, F, gvec[lo:hi])
        assert np.linalg.norm(gx[lo:hi] - ref) <= 1e-10 * max(np.linalg.norm(ref), 1e-300), g
    eng.close()


def test_sample_size_bound_per_graph(binding, batch):
    """Phase 1 of every graph (indices g * l1 ..) gives the oracle's rho~ and
    max p~, and l from the bound within one sample."""
    graphs, vptr, rp, col, x = batch
    eng = _engine(binding, batch)
    pc, infos = eng.estimate_graphs(0.05, 0.1, seed=4)
    ell1 = infos[0]["ell1"]
    for g, G in enumerate(graphs):
        og = oracle.from_synth(G)
        xg = x[vptr[g]:vptr[g + 1]]
        prep = oracle.prepare(xg)
        D = oracle.vertex_diam_ub(og)
        ph1 = oracle.run_samples(og, prep, 4, 0, 2, g * ell1, ell1, keep_paths=False)
        rh, rt, _ = oracle.rho_hat(ph1.ilen, D, 0.1)
        p1max = float((ph1.acc / ell1).max())
        vh = oracle.v_hat(p1max, prep.dhat, ell1, 0.1)
        ell, _ = oracle.ell_sup(0.05, 0.1, prep.dhat, rh, oracle.x_hat(vh, prep.dhat))
        assert infos[g]["rho_tilde"] == rt
        assert infos[g]["p1_max"] == pytest.approx(p1max, rel=1e-12)
        assert abs(infos[g]["ell"] - ell) <= 1, g
    eng.close()


def test_batch_of_one_equals_single_graph(binding):
    """A batch of one graph is the single-graph method (offsets 0)."""
    g, x, eps, delta = synth.workload("er1000")
    vptr, rp, col = synth.union_csr([g])
    eng = binding.PercIS(0)
    eng.load_graphs(vptr, rp, col)
    eng.set_states(x)
    pc_b, infos = eng.estimate_graphs(eps, delta, seed=5)
    one = binding.PercIS(0)
    one.load_csr(g.row_ptr, g.col)
    one.set_states(x)
    pc_1, info = one.estimate(eps, delta, seed=5)
    assert infos[0]["ell"] == info["ell"]
    assert torch.equal(pc_b, pc_1)
    eng.close()
    one.close()


def test_malformed_batches_are_rejected(binding):
    a = synth.path_graph(4)
    b = synth.path_graph(5)
    vptr, rp, col = synth.union_csr([a, b])
    eng = binding.PercIS(0)
    bad = col.copy()
    bad[0] = 6  # an edge of graph 0 into graph 1
    with pytest.raises(binding.PercisError) as e:
        eng.load_graphs(vptr, rp, bad)
    assert e.value.status == 1
    with pytest.raises(binding.PercisError) as e:
        eng.load_graphs(np.array([0, 1, 9]), rp, col)  # a graph of one vertex
    assert e.value.status == 1
    eng.load_graphs(vptr, rp, col)
    with pytest.raises(binding.PercisError) as e:
        eng.estimate(0.1, 0.1, seed=0, out=torch.empty(9, dtype=torch.float64, device="cuda"))
    assert e.value.status in (1, 8)
    eng.close()


@pytest.mark.slow
def test_full_size_512_uneven_graphs(binding):
    """512 graphs, vertex counts log-uniform in [1,000, 200,000] (Watts-Strogatz,
    Barabasi-Albert, grids with 5% of edges deleted), uniform states,
    eps=0.01: the bound-driven estimate gives every graph the oracle's
    phase-1 statistics and l (checked on sampled graphs); with fixed sample
    sizes the estimates and dPC/dx of sampled graphs equal the oracle's."""
    sizes = synth.uneven_batch_sizes(512, 1000, 200_000, 0)
    graphs = synth.graph_batch(sizes, 0)  # bidirectional form: deep grids need no level-synchronous batches
    vptr, rp, col = synth.union_csr(graphs)
    x = synth.states_uniform(int(vptr[-1]), 0)
    eng = binding.PercIS(0)
    eng.set_options(form="bidir", cuda_graphs=1)
    eng.load_graphs(vptr, rp, col)
    eng.set_states(x)
    pc, infos = eng.estimate_graphs(0.01, 0.1, seed=0)
    assert len(infos) == 512 and all(f["ell"] > 0 for f in infos)
    rng = np.random.default_rng(1)
    small = [g for g in range(512) if graphs[g].n < 12_000]
    picks = [int(v) for v in rng.choice(small, 3, replace=False)]
    ell1 = infos[0]["ell1"]
    for g in picks:
        og = oracle.from_synth(graphs[g])
        xg = x[vptr[g]:vptr[g + 1]]
        prep = oracle.prepare(xg)
        D = oracle.vertex_diam_ub(og)
        ph1 = oracle.run_samples(og, prep, 0, 0, 2, g * ell1, ell1, keep_paths=False, bidir=True)
        rh, rt, _ = oracle.rho_hat(ph1.ilen, D, 0.1)
        p1max = float((ph1.acc / ell1).max())
        vh = oracle.v_hat(p1max, prep.dhat, ell1, 0.1)
        ell, _ = oracle.ell_sup(0.01, 0.1, prep.dhat, rh, oracle.x_hat(vh, prep.dhat))
        assert infos[g]["rho_tilde"] == rt and infos[g]["vertex_diam"] == D
        assert abs(infos[g]["ell"] - ell) <= 1, g
    # fixed sample sizes: deterministic offsets, estimates and gradients per graph
    fixed = 2000
    eng.set_options(ell1=1000, ell=fixed)
    pc, infos = eng.estimate_graphs(0.01, 0.1, seed=2)
    pc = pc.cpu().numpy()
    gvec = np.random.default_rng(3).standard_normal(int(vptr[-1]))
    gx = eng.backward(torch.as_tensor(gvec, device="cuda")).cpu().numpy()
    for g in picks:
        og = oracle.from_synth(graphs[g])
        lo, hi = vptr[g], vptr[g + 1]
        prep = oracle.prepare(x[lo:hi], cv_method="sorted")
        ph2 = oracle.run_samples(og, prep, 2, 1, 3, g * fixed, fixed, keep_paths=True, bidir=True)
        F = prep.lam * ph2.cnt / fixed
        assert np.max(np.abs(pc[lo:hi] - F)) <= 1e-9, g
        ref = oracle.vjp_fixed(prep, fixed, ph2, F, gvec[lo:hi])
        assert np.linalg.norm(gx[lo:hi] - ref) <= 1e-10 * np.linalg.norm(ref), g
    eng.close()


def test_cuda_graph_sampling_matches_eager(binding, batch):
    """Recorded per-graph sampling (replayed with each call's seed from device
    memory) gives bit-identical estimates to the eager launches, call after call."""
    eager = _engine(binding, batch)
    rec = _engine(binding, batch, cuda_graphs=1)
    for seed in (3, 4, 5):
        pa, ia = eager.estimate_graphs(0.05, 0.1, seed=seed)
        pb, ib = rec.estimate_graphs(0.05, 0.1, seed=seed)
        assert torch.equal(pa, pb)
        assert [f["ell"] for f in ia] == [f["ell"] for f in ib]
    eager.close()
    rec.close()
