"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer and index results (sorted order, tables, pairs, distances, sigma,
paths, counts) must be bit-exact; sigma is exact below 2^53 so its FP64
values must match exactly too.  Estimates: 1e-9 absolute.  Gradients: 1e-10
norm-wise relative to the oracle's VJP and 1e-6 to finite differences.
"""
import numpy as np
import pytest

import oracle
from paper_2509_11454_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_11454_gb300 import binding as b

    b.load_library()
    return b


def _engine(binding, g, x=None, **opts):
    eng = binding.PercIS(0)
    if opts:
        eng.set_options(**opts)
    eng.load_csr(g.row_ptr, g.col, directed=g.directed)
    if x is not None:
        eng.set_states(x)
    return eng


def _np(t):
    return t.cpu().numpy()


def _sigma_equal(got, ref):
    """sigma is exact below 2^53; above it both sides carry FP64 roundings."""
    exact = ref < 2.0 ** 53
    return np.array_equal(got[exact], ref[exact]) and np.allclose(got[~exact], ref[~exact], rtol=1e-13, atol=0)


GRAPHS = {
    "er1000": lambda: synth.erdos_renyi(1000, 8.0, 0),
    "ba3000": lambda: synth.barabasi_albert(3000, 3, 1),
    "rmat12": lambda: synth.rmat(12, 8, 0.57, 0.19, 0.19, 2),
    "grid30": lambda: synth.grid_2d(30, 0.05, 3),
}


@pytest.fixture(scope="module", params=list(GRAPHS))
def gcase(request):
    g = GRAPHS[request.param]()
    return request.param, g, oracle.from_synth(g)


def _states(name, n):
    if name == "ba3000":
        return synth.states_outbreak(n, 0.1, 0.5, 1.0, 0)  # 90% ties at 0
    if name == "rmat12":
        return synth.states_beta(n, 0.5, 2.0, 0)
    return synth.states_uniform(n, 0)


def test_prep_bitexact(binding, gcase):
    name, g, og = gcase
    x = _states(name, g.n)
    eng = _engine(binding, g, x)
    got = eng.prep()
    prep = oracle.prepare(x, cv_method="sorted")
    assert np.array_equal(_np(got["perm"]), prep.perm)
    assert np.array_equal(_np(got["xs"]), prep.xs)
    for k in ("w", "ci", "r"):
        assert np.array_equal(_np(got[k]), getattr(prep, k)), k
    assert got["c"] == prep.c
    assert np.array_equal(_np(got["Cv"]), prep.Cv)
    assert np.array_equal(_np(got["lam"]), prep.lam)
    assert got["dhat"] == prep.dhat
    assert got["vertex_diam"] == oracle.vertex_diam_ub(og)
    eng.close()


def _adversarial_states(kind, n, seed):
    """State vectors that stress the exact evaluation of the Algorithm 2 running sums:
    halfway roundings, subnormal and tiny terms, long runs of zero c_i, many binades."""
    rng = np.random.default_rng(seed)
    if kind == "halfway":  # 40-bit significands: once w passes 2^13 every other term is a tie
        return rng.integers(2 ** 39, 2 ** 40, n).astype(np.float64) * 2.0 ** -40
    if kind == "dyadic":  # few significant bits: most sums exact, some halfway
        return rng.integers(1, 4097, n).astype(np.float64) / 4096.0
    if kind == "subnormal":
        pool = np.array([0.0, 5e-324, 7e-322, 1e-310, 2.2250738585072014e-308, 1e-300, 1e-20, 0.5, 1.0])
        return np.where(rng.random(n) < 0.5, pool[rng.integers(0, len(pool), n)], rng.random(n))
    if kind == "equal":  # 90% equal smallest states: c_i = 0 over them, so r starts with a run of +0
        return np.where(rng.random(n) < 0.9, 0.375, 0.5 + 0.5 * rng.random(n))
    if kind == "binades":  # values over ~300 decades: the sums cross many binades
        return rng.random(n) * 10.0 ** (-rng.random(n) * 300.0)
    if kind == "large":  # several chunks of terms
        return rng.random(n)
    raise ValueError(kind)


@pytest.mark.parametrize("kind,n", [("halfway", 30000), ("dyadic", 20000), ("subnormal", 6000),
                                    ("equal", 5000), ("binades", 8000), ("large", 300000)])
def test_tables_bitexact_adversarial(binding, kind, n):
    """w, c_i, r and c equal the sequential FP64 evaluation of Algorithm 2 bit for bit."""
    x = _adversarial_states(kind, n, 5)
    g = synth.barabasi_albert(n, 2, 0)  # the tables do not depend on the graph
    eng = _engine(binding, g, x)
    got = eng.prep()
    prep = oracle.prepare(x, cv_method="sorted")
    assert np.array_equal(_np(got["xs"]), prep.xs)
    for k in ("w", "ci", "r"):
        a, b = _np(got[k]), getattr(prep, k)
        assert np.array_equal(a.view(np.int64), b.view(np.int64)), (k, int(np.sum(a != b)))
    assert got["c"] == prep.c
    assert np.array_equal(_np(got["Cv"]), prep.Cv)
    eng.close()


def test_pairs_bitexact(binding, gcase):
    name, g, og = gcase
    x = _states(name, g.n)
    eng = _engine(binding, g, x)
    prep = oracle.prepare(x)
    for tag, i0, cnt in [(0, 0, 20000), (1, 123457, 5001)]:
        s, t = eng.sample_pairs(seed=77, tag=tag, i0=i0, count=cnt)
        rs, rt, _, _ = oracle.sample_pairs(prep, 77, tag, i0, cnt)
        assert np.array_equal(_np(s), rs)
        assert np.array_equal(_np(t), rt)
    eng.close()


def test_plain_bfs_bitexact(binding, gcase):
    name, g, og = gcase
    eng = _engine(binding, g)
    rng = np.random.default_rng(0)
    for src in rng.integers(0, g.n, 4):
        for tgt in (-1, int(rng.integers(0, g.n)), int(src)):
            dist, sig = eng.bfs(int(src), tgt)
            ret, rd, rsig, _, _, _ = oracle.bfs(og, int(src), tgt)
            if tgt < 0 or tgt == src:  # full traversal, or level 0 alone
                assert np.array_equal(_np(dist), rd)
                assert _sigma_equal(_np(sig), rsig)
            else:
                # truncated: every vertex the oracle settled matches exactly
                m = rd >= 0
                assert np.array_equal(_np(dist)[m], rd[m])
                assert _sigma_equal(_np(sig)[m], rsig[m])
    eng.close()


@pytest.mark.parametrize("direction", [0, 1, 2])
@pytest.mark.parametrize("nsrc", [1, 5, 64, 100, 200, 512])
def test_msbfs_bitexact(binding, gcase, nsrc, direction):
    name, g, og = gcase
    eng = _engine(binding, g, direction=direction)
    rng = np.random.default_rng(nsrc)
    srcs = rng.choice(g.n, size=nsrc, replace=False)
    dist, sig = eng.msbfs(srcs)
    dist, sig = _np(dist), _np(sig)
    check = list(range(nsrc)) if nsrc <= 8 else list(rng.choice(nsrc, 8, replace=False)) + [nsrc - 1]
    for j in check:
        _, rd, rsig, _, _, _ = oracle.bfs(og, int(srcs[j]))
        assert np.array_equal(dist[j], rd), j
        assert _sigma_equal(sig[j], rsig), j
    eng.close()


# bidirectional stores: the default (the direct store when it fits), every
# sample in the direct store, one hashed table per block, small first tables
# that must move to larger ones, and a heavy-level threshold low enough that
# most samples are handed to the 1,024-thread pass
BIDIR_STORES = {"bidir": {}, "bidir_direct": {"bi_table_log": -1},
                "bidir_hashed": {"bi_table_log": 18, "bi_table_max_log": 18},
                "bidir_grow": {"bi_table_log": 10, "bi_table_max_log": 14},
                "bidir_heavy": {"bi_heavy_edges": 64}}


@pytest.mark.parametrize("form,direction", [("batched", 0), ("batched", 1), ("batched", 2), ("plain", 2),
                                            ("bidir", 2), ("bidir_direct", 2), ("bidir_hashed", 2),
                                            ("bidir_grow", 2), ("bidir_heavy", 2)])
def test_phase_bitexact(binding, gcase, form, direction):
    name, g, og = gcase
    x = _states(name, g.n)
    count = 600 if form == "plain" else 3000
    store = BIDIR_STORES.get(form)
    if store is not None:
        form = "bidir"
    eng = _engine(binding, g, x, form=form, direction=direction, **(store or {}))
    prep = oracle.prepare(x)
    got = eng.run_phase(seed=11, phase=1, count=count)
    ph = oracle.run_samples(og, prep, 11, 1, 3, 0, count, keep_paths=True, bidir=form == "bidir")
    assert np.array_equal(_np(got["s"]), ph.s)
    assert np.array_equal(_np(got["t"]), ph.t)
    assert np.array_equal(_np(got["kind"]), ph.kind)
    assert np.array_equal(_np(got["ilen"]), ph.ilen)
    if ph.overflow:
        # path counts past 2^53: FP64 on both sides (rounded in different orders)
        eng.close()
        return
    assert np.array_equal(_np(got["cnt"]), ph.cnt)
    ptr, nodes = eng.get_paths(count)
    assert np.array_equal(_np(ptr), ph.path_ptr)
    assert np.array_equal(_np(nodes), ph.path_nodes)
    eng.close()


@pytest.mark.parametrize("scale", [17, 18])
def test_bidir_directed_large_transpose_bitexact(binding, scale):
    """Directed graphs of more than 2^16 vertices: the in-adjacency sort takes
    three digit passes (the last with one or two bits) over a ragged last tile;
    every in-list must come out in source order, so the bidirectional phase's
    paths (which scan in-lists in that order) equal the oracle's bit for bit."""
    g = synth.rmat(scale, 16, 0.57, 0.19, 0.19, 8)
    og = oracle.from_synth(g)
    x = synth.states_beta(g.n, 0.5, 2.0, 8)
    eng = _engine(binding, g, x, form="bidir")
    prep = oracle.prepare(x)
    got = eng.run_phase(seed=13, phase=1, count=2000)
    ph = oracle.run_samples(og, prep, 13, 1, 3, 0, 2000, keep_paths=True, bidir=True)
    assert np.array_equal(_np(got["kind"]), ph.kind)
    assert np.array_equal(_np(got["ilen"]), ph.ilen)
    ptr, nodes = eng.get_paths(2000)
    assert np.array_equal(_np(ptr), ph.path_ptr)
    assert np.array_equal(_np(nodes), ph.path_nodes)
    eng.close()


def test_estimate_matches_oracle(binding):
    g, x, eps, delta = synth.workload("er1000")
    og = oracle.from_synth(g)
    eng = _engine(binding, g, x)
    pc, info = eng.estimate(eps, delta, seed=5)
    res = oracle.percis(og, x, eps, delta, 5, keep_paths=False)
    assert info["ell1"] == res.ell1
    assert info["vertex_diam"] == res.D
    assert info["rho_tilde"] == res.rho_tilde and info["Lambda"] == res.Lam
    assert abs(info["ell"] - res.ell) <= 1
    if info["ell"] != res.ell:
        res = oracle.percis(og, x, eps, delta, 5, ell=info["ell"], keep_paths=False)
    assert np.max(np.abs(_np(pc) - res.pc)) <= 1e-9
    assert info["rho_hat"] == pytest.approx(res.rho_hat, rel=1e-12)
    assert info["v_hat"] == pytest.approx(res.v_hat, rel=1e-12)
    # same seed, other form, other lane width: identical estimate
    eng2 = _engine(binding, g, x, form="plain")
    pc2, info2 = eng2.estimate(eps, delta, seed=5)
    assert np.array_equal(_np(pc2), _np(pc))
    eng3 = _engine(binding, g, x, lanes=64)
    pc3, _ = eng3.estimate(eps, delta, seed=5)
    assert np.array_equal(_np(pc3), _np(pc))
    for e in (eng, eng2, eng3):
        e.close()


@pytest.mark.parametrize("name", ["er1000", "ba3000", "rmat12", "grid30"])
def test_allpaths_estimate_matches_oracle(binding, name):
    """All-paths form: p(v) = lambda_v sum_i sigma_sv tau_v / sigma_st / l over
    the same sampled pairs; per-sample fractions are exact ratios, the sums
    differ from the oracle's only in rounding order."""
    g = GRAPHS[name]()
    og = oracle.from_synth(g)
    x = _states(name, g.n)
    eng = _engine(binding, g, x, estimator="allpaths", ell1=1500, ell=4000)
    pc, info = eng.estimate(0.05, 0.1, seed=9)
    res = oracle.percis(og, x, 0.05, 0.1, 9, ell1=1500, ell=4000, keep_paths=False, allpaths=True)
    ref = res.pc
    assert info["ell"] == 4000 and info["ell1"] == 1500
    assert info["rho_tilde"] == res.rho_tilde
    assert info["p1_max"] == pytest.approx(res.p1_max, rel=1e-12)
    assert np.allclose(_np(pc), ref, rtol=1e-12, atol=1e-15)
    # same pairs as the one-path form: identical rho~ and sum over v of the
    # unnormalised sums equals sum_i |I(tau_i)| (each sample spreads d-1)
    lam = res.prep.lam
    tot = float(np.sum(_np(pc) / lam)) * 4000
    assert tot == pytest.approx(float(res.phase2.ilen.sum()), rel=1e-10)
    with pytest.raises(binding.PercisError):
        eng.backward(torch.ones(g.n, dtype=torch.float64, device="cuda"))
    eng.close()


@pytest.mark.parametrize("name", ["er1000", "ba3000", "rmat12", "grid30"])
def test_bidir_estimate_matches_oracle(binding, name):
    """The bidirectional form through Algorithm 1: l, rho~ and the estimate
    as the oracle's bidirectional replica computes them; its backward equals
    the oracle's VJP on the same sample."""
    g = GRAPHS[name]()
    og = oracle.from_synth(g)
    x = _states(name, g.n)
    eng = _engine(binding, g, x, form="bidir")
    pc, info = eng.estimate(0.05, 0.1, seed=6)
    res = oracle.percis(og, x, 0.05, 0.1, 6, keep_paths=True, bidir=True)
    assert info["rho_tilde"] == res.rho_tilde
    if res.phase1.overflow or res.phase2.overflow:
        assert info["sigma_overflow"] == 1
        eng.close()
        return
    assert abs(info["ell"] - res.ell) <= 1
    if info["ell"] != res.ell:
        res = oracle.percis(og, x, 0.05, 0.1, 6, ell=info["ell"], keep_paths=True, bidir=True)
    assert np.max(np.abs(_np(pc) - res.pc)) <= 1e-9
    prep = oracle.prepare(x, cv_method="sorted")
    gvec = np.random.default_rng(4).standard_normal(g.n)
    gx = _np(eng.backward(torch.as_tensor(gvec, device="cuda")))
    F = prep.lam * res.phase2.cnt / info["ell"]
    ref = oracle.vjp_fixed(prep, info["ell"], res.phase2, F, gvec)
    assert np.linalg.norm(gx - ref) <= 1e-10 * np.linalg.norm(ref)
    eng.close()


def test_bidir_hand_over_to_direct_store(binding):
    """Samples the hashed tables cannot hold -- more vertices than 3/4 of
    the largest table minus a block's claims in flight (a 60x60 grid with the
    tables capped at 2^10 entries), or more than 4,095 levels on a side (a
    path of 12,000 vertices with states falling along it, so that far pairs
    weigh most) -- are handed to the direct store and give the oracle's paths
    and counts bit for bit.  Both cases ask for hashed tables: the default
    store for graphs this small is the direct one, which has neither limit."""
    cases = [(synth.grid_2d(60, 0.05, 7), None, {"bi_table_log": 10, "bi_table_max_log": 10}),
             (synth.path_graph(12000), "falling", {"bi_table_log": 16, "bi_table_max_log": 16})]
    for g, xs, opts in cases:
        og = oracle.from_synth(g)
        x = 1.0 - np.arange(g.n) / g.n if xs == "falling" else synth.states_uniform(g.n, 3)
        eng = _engine(binding, g, x, form="bidir", instrument=1, ell1=200, ell=600, **opts)
        pc, info = eng.estimate(0.05, 0.1, seed=4)
        assert info["work"][1][4] > 0 and info["work"][0][4] >= 0  # some samples handed over
        prep = oracle.prepare(x)
        ph = oracle.run_samples(og, prep, 4, 1, 3, 0, 600, keep_paths=True, bidir=True)
        assert np.array_equal(_np(pc), prep.lam * ph.cnt / 600) or \
            np.max(np.abs(_np(pc) - prep.lam * ph.cnt / 600)) <= 1e-12
        ptr, nodes = eng.get_paths(600)
        assert np.array_equal(_np(ptr), ph.path_ptr)
        assert np.array_equal(_np(nodes), ph.path_nodes)
        eng.close()


@pytest.mark.parametrize("shuffle", [False, True])
@pytest.mark.parametrize("name", ["rmat14", "ba20000"])
def test_bidir_hub_backtracks_bitexact(binding, name, shuffle):
    """Backtrack steps through hubs (candidate lists longer than a warp's
    share): with strictly sorted rows the kernel may find a small previous
    level's vertices in w's list by bisection; with every row shuffled it must
    scan the list in its stored order, as the oracle does.  Paths and counts
    equal the oracle's either way."""
    g = synth.rmat(14, 16, 0.57, 0.19, 0.19, 5) if name == "rmat14" else synth.barabasi_albert(20000, 3, 5)
    if shuffle:
        rng = np.random.default_rng(9)
        col = g.col.copy()
        for u in range(g.n):
            a, b = g.row_ptr[u], g.row_ptr[u + 1]
            col[a:b] = rng.permutation(col[a:b])
        g = synth.Graph(n=g.n, row_ptr=g.row_ptr, col=col, directed=g.directed)
    og = oracle.from_synth(g)
    x = synth.states_uniform(g.n, 2)
    eng = _engine(binding, g, x, form="bidir")
    got = eng.run_phase(seed=13, phase=1, count=3000)
    prep = oracle.prepare(x)
    ph = oracle.run_samples(og, prep, 13, 1, 3, 0, 3000, keep_paths=True, bidir=True)
    assert np.array_equal(_np(got["kind"]), ph.kind)
    assert np.array_equal(_np(got["cnt"]), ph.cnt)
    ptr, nodes = eng.get_paths(3000)
    assert np.array_equal(_np(ptr), ph.path_ptr)
    assert np.array_equal(_np(nodes), ph.path_nodes)
    eng.close()


@pytest.mark.slow
def test_bidir_full_size_rmat22_sampled(binding):
    """Directed R-MAT scale 22, Beta(0.5, 2) states, eps=0.01 in the
    bidirectional form (hashed tables, the heavy samples in the direct store):
    every phase-2 pair bit-exact, 40 sampled paths (reachable, unreachable and
    long ones) against the oracle's bidirectional replica one by one, and the
    estimate equal to lambda_v cnt_v / l over the returned paths."""
    g, x, eps, delta = synth.workload("rmat22_beta")
    og = oracle.from_synth(g)
    eng = _engine(binding, g, x, form="bidir", instrument=1)
    pc, info = eng.estimate(eps, delta, seed=0)
    ell = info["ell"]
    assert info["ell1"] == 1000 and info["vertex_diam"] == g.n - 2
    prep = oracle.prepare(x)
    s, t = eng.sample_pairs(0, 1, 0, ell)
    rs, rt, _, _ = oracle.sample_pairs(prep, 0, 1, 0, ell)
    assert np.array_equal(_np(s), rs) and np.array_equal(_np(t), rt)
    ptr, nodes = eng.get_paths(ell)
    ptr, nodes = _np(ptr), _np(nodes)
    cnt = np.bincount(nodes, minlength=g.n)
    assert np.max(np.abs(_np(pc) - prep.lam * cnt / ell)) <= 1e-12
    assert info["sum_internal"][1] == int(ptr[-1])
    rng = np.random.default_rng(0)
    long_ = np.flatnonzero(np.diff(ptr) >= 2)
    picks = np.concatenate([rng.choice(ell, 30, replace=False), rng.choice(long_, 10, replace=False)])
    kinds = set()
    for i in picks:
        ph = oracle.run_samples(og, prep, 0, 1, 3, int(i), 1, keep_paths=True, bidir=True)
        kinds.add(int(ph.kind[0]))
        assert np.array_equal(nodes[ptr[i]:ptr[i + 1]], ph.path_nodes), i
    assert {0, 2} <= kinds
    eng.close()


@pytest.mark.slow
def test_bidir_full_size_outbreak_sampled(binding):
    """BA n=100,000 outbreak, eps=0.005, bidirectional form: every phase-2
    pair, sampled paths against the oracle one by one, estimate = lambda cnt / l."""
    g, x, eps, delta = synth.workload("ba100k_outbreak")
    og = oracle.from_synth(g)
    eng = _engine(binding, g, x, form="bidir")
    pc, info = eng.estimate(eps, delta, seed=0)
    ell = info["ell"]
    prep = oracle.prepare(x)
    ptr, nodes = eng.get_paths(ell)
    ptr, nodes = _np(ptr), _np(nodes)
    cnt = np.bincount(nodes, minlength=g.n)
    assert np.max(np.abs(_np(pc) - prep.lam * cnt / ell)) <= 1e-12
    for i in np.random.default_rng(0).choice(ell, 40, replace=False):
        ph = oracle.run_samples(og, prep, 0, 1, 3, int(i), 1, keep_paths=True, bidir=True)
        assert np.array_equal(nodes[ptr[i]:ptr[i + 1]], ph.path_nodes), i
    eng.close()


def test_allpaths_lower_variance(binding):
    """Rao-Blackwellisation: on the same pairs the all-paths estimate is
    closer to the exact value than the one-path estimate (summed squared
    error over vertices, a grid with many shortest paths per pair)."""
    g = synth.grid_2d(24, 0.0, 0)
    x = synth.states_uniform(g.n, 4)
    eng = _engine(binding, g, x)
    exact = eng.exact()
    e1 = e2 = 0.0
    for seed in range(4):
        eng.set_options(estimator="path", ell1=1000, ell=3000)
        p1, _ = eng.estimate(0.05, 0.1, seed=seed)
        eng.set_options(estimator="allpaths")
        p2, _ = eng.estimate(0.05, 0.1, seed=seed)
        e1 += float(torch.sum((p1 - exact) ** 2))
        e2 += float(torch.sum((p2 - exact) ** 2))
    assert e2 < 0.7 * e1
    eng.close()


def test_percis_di_matches_oracle(binding):
    """PercIS-DI: no first phase, rho^ = D, v^ = d^2/4; l and the estimate
    as the oracle computes them."""
    g, x, eps, delta = synth.workload("er1000")
    og = oracle.from_synth(g)
    eng = _engine(binding, g, x, data_independent=1)
    pc, info = eng.estimate(eps, delta, seed=3)
    res = oracle.percis(og, x, eps, delta, 3, keep_paths=False, data_independent=True)
    assert info["ell1"] == 0 and info["batches"][0] == 0
    assert info["rho_hat"] == res.rho_hat and info["v_hat"] == pytest.approx(res.v_hat, rel=1e-15)
    assert abs(info["ell"] - res.ell) <= 1
    if info["ell"] != res.ell:
        res = oracle.percis(og, x, eps, delta, 3, ell=info["ell"], keep_paths=False, data_independent=True)
    assert np.max(np.abs(_np(pc) - res.pc)) <= 1e-9
    eng.close()


@pytest.mark.parametrize("name", ["rmat14", "ba20000"])
def test_autotune_bidir_keeps_results(binding, name):
    """Tuning the bidirectional form (heavy-level threshold, store, blocks per
    SM) keeps the estimate bit-identical to the default options' and to the
    oracle's bidirectional replica; with tune_form the form may change and
    the estimate is then that form's at the same seed."""
    g = synth.rmat(14, 16, 0.57, 0.19, 0.19, 5) if name == "rmat14" else synth.barabasi_albert(20000, 3, 5)
    og = oracle.from_synth(g)
    x = synth.states_uniform(g.n, 6)
    ref_eng = _engine(binding, g, x, form="bidir", ell1=1000, ell=4000)
    ref, _ = ref_eng.estimate(0.05, 0.1, seed=8)
    eng = _engine(binding, g, x, form="bidir", ell1=1000, ell=4000)
    o = eng.autotune(probe_samples=2000, seed=1)
    assert o["form"] == binding.FORM_BIDIR
    assert o["bi_heavy_edges"] in (0, 2048, 4096, 8192, 16384, 65536, -1)
    assert o["bi_table_log"] in (0, 16, 18) and o["bi_blocks_per_sm"] in (0, 2, 3, 4)
    pc, info = eng.estimate(0.05, 0.1, seed=8)
    assert np.array_equal(_np(pc), _np(ref))
    prep = oracle.prepare(x)
    ph = oracle.run_samples(og, prep, 8, 1, 3, 0, 4000, keep_paths=False, bidir=True)
    assert np.max(np.abs(_np(pc) - prep.lam * ph.cnt / 4000)) <= 1e-12
    eng.set_options(tune_form=1)
    o2 = eng.autotune(probe_samples=2000, seed=1)
    assert o2["form"] in (binding.FORM_BIDIR, binding.FORM_BATCHED)
    pc2, _ = eng.estimate(0.05, 0.1, seed=8)
    ph2 = oracle.run_samples(og, prep, 8, 1, 3, 0, 4000, keep_paths=False,
                             bidir=o2["form"] == binding.FORM_BIDIR)
    assert np.max(np.abs(_np(pc2) - prep.lam * ph2.cnt / 4000)) <= 1e-12
    ref_eng.close()
    eng.close()


def test_autotune_keeps_results(binding):
    """The autotuner only picks speed options: the estimate after tuning is
    bit-identical to the default one and to the oracle's."""
    g, x, eps, delta = synth.workload("er1000")
    og = oracle.from_synth(g)
    ref_eng = _engine(binding, g, x)
    ref, _ = ref_eng.estimate(eps, delta, seed=8)
    eng = _engine(binding, g, x)
    o = eng.autotune(probe_samples=3000, seed=1)
    assert o["lanes"] in (0, 64, 128, 256, 512) and o["lane_order"] in (0, 1) and o["direction"] in (0, 1, 2)
    pc, info = eng.estimate(eps, delta, seed=8)
    assert np.array_equal(_np(pc), _np(ref))
    res = oracle.percis(og, x, eps, delta, 8, ell=info["ell"], keep_paths=False)
    assert np.max(np.abs(_np(pc) - res.pc)) <= 1e-9
    ref_eng.close()
    eng.close()


def test_backward_matches_oracle_and_fd(binding):
    g = synth.barabasi_albert(2000, 4, 0)
    og = oracle.from_synth(g)
    x = synth.states_uniform(g.n, 0)
    ell = 4000
    eng = _engine(binding, g, x, ell1=1000, ell=ell)
    pc, info = eng.estimate(0.01, 0.1, seed=9)
    prep = oracle.prepare(x, cv_method="sorted")
    ph = oracle.run_samples(og, prep, 9, 1, 3, 0, ell, keep_paths=True)
    F = prep.lam * ph.cnt / ell
    assert np.max(np.abs(_np(pc) - F)) <= 1e-12
    gvec = np.random.default_rng(2).standard_normal(g.n)
    gx = _np(eng.backward(torch.as_tensor(gvec, device="cuda")))
    ref = oracle.vjp_fixed(prep, ell, ph, F, gvec)
    assert np.linalg.norm(gx - ref) / np.linalg.norm(ref) <= 1e-10
    h = 1e-6
    checked = 0
    for u in np.random.default_rng(3).permutation(g.n)[:200]:
        if np.any(np.abs(np.delete(x, u) - x[u]) < 4 * h):
            continue
        touch = (ph.kind == 0) & ((ph.s == u) | (ph.t == u))
        if np.any(np.abs(x[ph.s[touch]] - x[ph.t[touch]]) <= 1e-3):
            continue
        fd = oracle.fd_fixed(prep, ell, ph, gvec, int(u), h)
        assert gx[u] == pytest.approx(fd, rel=1e-6, abs=1e-12 * np.abs(gx).max())
        checked += 1
        if checked >= 25:
            break
    assert checked >= 10
    eng.close()


@pytest.mark.parametrize("form", ["batched", "bidir"])
def test_gpu_gradient_unbiased_for_exact_gradient_ba2000(binding, form):
    """The fixed-sample gradient (the estimator's adjoint with the sample
    held) is an importance-sampling estimate of the gradient of g . p(x) for
    the exact percolation centrality p: over 48 seeds its mean lies within 6
    standard errors of the oracle's exact VJP at every vertex of BA(2000, 4),
    and the squared distance of the mean to it is within twice its expected
    value sum_u Var/K.  The same checks reject the negated exact gradient."""
    g = synth.barabasi_albert(2000, 4, 0)
    og = oracle.from_synth(g)
    x = synth.states_uniform(g.n, 0)
    gvec = np.random.default_rng(12).standard_normal(g.n)
    exact = oracle.exact_vjp(og, x, gvec)
    eng = _engine(binding, g, x, form=form, ell1=1000, ell=20000)
    K = 48
    gt = torch.as_tensor(gvec, device="cuda")
    gs = np.empty((K, g.n))
    for k in range(K):
        eng.estimate(0.05, 0.1, seed=1000 + k)
        gs[k] = _np(eng.backward(gt))
    eng.close()
    mean = gs.mean(axis=0)
    var = gs.var(axis=0, ddof=1)
    se = np.sqrt(var / K)
    floor = 1e-9 * np.abs(exact).max()
    assert np.all(np.abs(mean - exact) <= 6 * se + floor)
    assert np.sum((mean - exact) ** 2) <= 2 * var.sum() / K
    assert not np.all(np.abs(mean + exact) <= 6 * se + floor)
    assert np.sum((mean + exact) ** 2) > 2 * var.sum() / K


def test_autograd_function(binding):
    g = synth.barabasi_albert(500, 3, 4)
    x = torch.as_tensor(synth.states_uniform(g.n, 4), device="cuda").requires_grad_(True)
    eng = _engine(binding, g, None, ell1=500, ell=1500)
    pc = binding.percolation_centrality(x, eng, 0.05, 0.1, seed=1)
    w = torch.randn(g.n, device="cuda", dtype=torch.float64)
    (pc * w).sum().backward()
    og = oracle.from_synth(g)
    prep = oracle.prepare(x.detach().cpu().numpy(), cv_method="sorted")
    ph = oracle.run_samples(og, prep, 1, 1, 3, 0, 1500, keep_paths=True)
    ref = oracle.vjp_fixed(prep, 1500, ph, prep.lam * ph.cnt / 1500, w.cpu().numpy())
    assert np.linalg.norm(_np(x.grad) - ref) / np.linalg.norm(ref) <= 1e-10
    eng.close()


@pytest.mark.parametrize("name", ["er1000", "rmat12", "grid30"])
def test_exact_small_matches_oracle(binding, name):
    g = GRAPHS[name]() if name != "er1000" else synth.erdos_renyi(1000, 8.0, 0)
    og = oracle.from_synth(g)
    x = _states(name, g.n)
    eng = _engine(binding, g, x)
    pc = _np(eng.exact())
    ref = oracle.exact_pc(og, x, oracle.prepare(x).Cv)
    assert np.max(np.abs(pc - ref)) <= 1e-9
    eng.close()


def test_epsilon_guarantee_gpu(binding):
    g, x, eps, delta = synth.workload("er1000")
    og = oracle.from_synth(g)
    exact = oracle.exact_pc(og, x, oracle.prepare(x).Cv)
    eng = _engine(binding, g, x)
    ok = 0
    for seed in range(20):
        pc, _ = eng.estimate(eps, delta, seed=seed)
        ok += int(np.max(np.abs(_np(pc) - exact)) <= eps)
    assert ok >= 18
    eng.close()


def _state_setting(setting):
    """The four state settings of Section V-A on small synthetic graphs."""
    if setting == "rs":
        g = synth.barabasi_albert(3000, 3, 1)
        return g, synth.states_random_seeds(g.n, 50, 0)
    if setting == "rss":
        g = synth.barabasi_albert(3000, 3, 1)
        return g, synth.states_seeds_spread(g, 0)
    if setting == "ic":
        return synth.isolated_component(synth.barabasi_albert(3000, 3, 1), 0)
    if setting == "ic_directed":
        return synth.isolated_component(synth.rmat(12, 8, 0.57, 0.19, 0.19, 2), 0)
    if setting == "un":
        g = synth.barabasi_albert(3000, 3, 1)
        return g, synth.states_uniform(g.n, 0)
    raise ValueError(setting)


@pytest.mark.parametrize("form", ["batched", "bidir"])
@pytest.mark.parametrize("setting", ["rs", "rss", "ic", "ic_directed", "un"])
def test_state_settings_match_oracle(binding, setting, form):
    """Algorithm 1 on the paper's four state settings (random seeds, seeds spread,
    isolated component, uniform): l and the estimate as the oracle computes them."""
    g, x = _state_setting(setting)
    og = oracle.from_synth(g)
    eng = _engine(binding, g, x, form=form)
    pc, info = eng.estimate(0.02, 0.1, seed=3)
    res = oracle.percis(og, x, 0.02, 0.1, 3, keep_paths=False, bidir=form == "bidir")
    assert info["ell1"] == res.ell1 and info["vertex_diam"] == res.D
    assert info["rho_tilde"] == res.rho_tilde
    assert abs(info["ell"] - res.ell) <= 1
    if info["ell"] != res.ell:
        res = oracle.percis(og, x, 0.02, 0.1, 3, ell=info["ell"], keep_paths=False, bidir=form == "bidir")
    assert np.max(np.abs(_np(pc) - res.pc)) <= 1e-9
    eng.close()


def test_epsilon_guarantee_isolated_component(binding):
    """Section V-A's isolated-component setting (the shape of Proposition 7's
    instance): max |p~ - p| <= eps in at least 18 of 20 runs."""
    g, x = synth.isolated_component(synth.erdos_renyi(1000, 8.0, 0), 0)
    og = oracle.from_synth(g)
    exact = oracle.exact_pc(og, x, oracle.prepare(x).Cv)
    assert exact[:1000].max() == 0.0 and exact[1000:].max() > 0.0  # all of it on the path
    eng = _engine(binding, g, x, form="bidir")
    eps = 0.002  # well below max p (0.0122), so an all-zero estimate fails
    ok = 0
    for seed in range(20):
        pc, _ = eng.estimate(eps, 0.1, seed=seed)
        ok += int(np.max(np.abs(_np(pc) - exact)) <= eps)
    assert ok >= 18
    eng.close()


@pytest.mark.slow
@pytest.mark.parametrize("name", ["ba100k_outbreak", "ba200k_uniform"])
def test_epsilon_guarantee_full_size_gpu_exact(binding, name):
    """Proposition 4 at full size: the exact centrality from the GPU
    (all-sources batched sigma-BFS + the extended Brandes dependencies,
    parity-tested against the oracle on small graphs) as ground truth;
    max_v |p~(v) - p(v)| <= eps in at least 18 of 20 seeds."""
    g, x, eps, delta = synth.workload(name)
    eng = _engine(binding, g, x)
    exact = eng.exact()
    ok = 0
    for seed in range(20):
        pc, _ = eng.estimate(eps, delta, seed=seed)
        ok += int(float(torch.max(torch.abs(pc - exact))) <= eps)
    assert ok >= 18
    eng.close()


def test_full_size_outbreak_sampled(binding):
    """Barabasi-Albert n=100,000 (m=5), 10% outbreak states, eps=0.005: the
    launch configuration the benchmark times.  Pairs, |I| and paths are
    checked on sampled indices against the oracle; counts and estimates via
    properties that hold at any size."""
    g, x, eps, delta = synth.workload("ba100k_outbreak")
    og = oracle.from_synth(g)
    eng = _engine(binding, g, x)
    pc, info = eng.estimate(eps, delta, seed=0)
    ell = info["ell"]
    assert info["ell1"] == 1000 and ell > 10000
    prep = oracle.prepare(x)
    s, t = eng.sample_pairs(0, 1, 0, ell)
    rs, rt, _, _ = oracle.sample_pairs(prep, 0, 1, 0, ell)
    assert np.array_equal(_np(s), rs) and np.array_equal(_np(t), rt)
    ptr, nodes = eng.get_paths(ell)
    ptr, nodes = _np(ptr), _np(nodes)
    cnt = np.bincount(nodes, minlength=g.n)
    assert np.max(np.abs(_np(pc) - prep.lam * cnt / ell)) <= 1e-12
    for i in np.random.default_rng(0).choice(ell, 25, replace=False):
        ph = oracle.run_samples(og, prep, 0, 1, 3, int(i), 1, keep_paths=True)
        assert np.array_equal(nodes[ptr[i]:ptr[i + 1]], ph.path_nodes), i
    eng.close()


@pytest.mark.slow
def test_full_size_rmat22_sampled(binding):
    """Directed R-MAT scale 22 (edge factor 16), Beta(0.5, 2) states,
    eps=0.01: every phase-2 pair bit-exact, sampled paths (reachable and
    unreachable targets) against the oracle one by one, and the estimate
    equal to lambda_v cnt_v / l over the returned paths."""
    g, x, eps, delta = synth.workload("rmat22_beta")
    og = oracle.from_synth(g)
    eng = _engine(binding, g, x)
    pc, info = eng.estimate(eps, delta, seed=0)
    ell = info["ell"]
    assert info["ell1"] == 1000 and info["vertex_diam"] == g.n - 2
    prep = oracle.prepare(x)
    s, t = eng.sample_pairs(0, 1, 0, ell)
    rs, rt, _, _ = oracle.sample_pairs(prep, 0, 1, 0, ell)
    assert np.array_equal(_np(s), rs) and np.array_equal(_np(t), rt)
    ptr, nodes = eng.get_paths(ell)
    ptr, nodes = _np(ptr), _np(nodes)
    cnt = np.bincount(nodes, minlength=g.n)
    assert np.max(np.abs(_np(pc) - prep.lam * cnt / ell)) <= 1e-12
    assert info["sum_internal"][1] == int(ptr[-1])
    rng = np.random.default_rng(0)
    long_ = np.flatnonzero(np.diff(ptr) >= 2)
    picks = np.concatenate([rng.choice(ell, 6, replace=False), rng.choice(long_, 4, replace=False)])
    kinds = set()
    for i in picks:
        ph = oracle.run_samples(og, prep, 0, 1, 3, int(i), 1, keep_paths=True)
        kinds.add(int(ph.kind[0]))
        assert np.array_equal(nodes[ptr[i]:ptr[i + 1]], ph.path_nodes), i
    assert 0 in kinds
    eng.close()


@pytest.mark.slow
def test_full_size_differentiation_ba200k(binding):
    """Barabasi-Albert n=200,000 (m=4), uniform states: the full-size
    forward + backward (l from the bound at eps=0.01) satisfies the two
    invariances of the fixed-sample estimator (F is unchanged by x -> x + c
    and by x -> a x, so sum_u grad_u = 0 and sum_u x_u grad_u = 0); on the
    same graph with l fixed to 2,000 the gradient equals the oracle's VJP
    and central finite differences on sampled coordinates."""
    g, x, eps, delta = synth.workload("ba200k_uniform")
    og = oracle.from_synth(g)
    gvec = np.random.default_rng(2).standard_normal(g.n)
    eng = _engine(binding, g, x)
    pc, info = eng.estimate(eps, delta, seed=0)
    assert info["ell"] > 10000
    gx = _np(eng.backward(torch.as_tensor(gvec, device="cuda")))
    scale = np.sum(np.abs(gx))
    assert abs(np.sum(gx)) <= 1e-10 * scale
    assert abs(np.sum(x * gx)) <= 1e-10 * np.sum(np.abs(x * gx))
    ell = 2000
    eng.set_options(ell1=1000, ell=ell)
    pc, info = eng.estimate(eps, delta, seed=4)
    prep = oracle.prepare(x, cv_method="sorted")
    ph = oracle.run_samples(og, prep, 4, 1, 3, 0, ell, keep_paths=True)
    F = prep.lam * ph.cnt / ell
    assert np.max(np.abs(_np(pc) - F)) <= 1e-12
    gx = _np(eng.backward(torch.as_tensor(gvec, device="cuda")))
    ref = oracle.vjp_fixed(prep, ell, ph, F, gvec)
    assert np.linalg.norm(gx - ref) / np.linalg.norm(ref) <= 1e-10
    h = 1e-6
    checked = 0
    xs = np.sort(x)
    for u in np.random.default_rng(3).permutation(g.n)[:400]:
        k = np.searchsorted(xs, x[u])
        near = xs[max(0, k - 2):k + 3]
        if np.sum(np.abs(near - x[u]) < 4 * h) > 1:
            continue
        touch = (ph.kind == 0) & ((ph.s == u) | (ph.t == u))
        if np.any(np.abs(x[ph.s[touch]] - x[ph.t[touch]]) <= 1e-3):
            continue
        fd = oracle.fd_fixed(prep, ell, ph, gvec, int(u), h)
        assert gx[u] == pytest.approx(fd, rel=1e-6, abs=1e-12 * np.abs(gx).max())
        checked += 1
        if checked >= 12:
            break
    assert checked >= 8
    eng.close()


def test_edge_cases(binding):
    # directed graph with unreachable targets, n = 2, binary states with ties
    gd = synth.csr_from_edges(6, np.array([0, 1, 2, 4]), np.array([1, 2, 3, 5]), directed=True)
    x = np.array([1.0, 0.9, 0.8, 0.0, 0.7, 0.1])
    ogd = oracle.from_synth(gd)
    eng = _engine(binding, gd, x, ell1=50, ell=400)
    got = eng.run_phase(seed=3, phase=1, count=400)
    ph = oracle.run_samples(ogd, oracle.prepare(x), 3, 1, 3, 0, 400, keep_paths=True)
    assert np.array_equal(_np(got["kind"]), ph.kind) and (ph.kind == 2).any()
    assert np.array_equal(_np(got["cnt"]), ph.cnt)
    eng.close()
    # n = 2: every C_v is empty, so p is undefined (Section II-A)
    g2 = synth.path_graph(2)
    eng = _engine(binding, g2)
    with pytest.raises(binding.PercisError) as e:
        eng.set_states(np.array([1.0, 0.0]))
    assert e.value.status == 2
    eng.close()
    # path 0-1-2, x = (1, 1/2, 0): C = 2, C_1 = 1, lambda_1 = 2, p = (0, 1, 0);
    # pair (0,2) has probability 1/2 and always crosses 1
    g3 = synth.path_graph(3)
    eng = _engine(binding, g3, np.array([1.0, 0.5, 0.0]), ell1=1000, ell=4000)
    pc, info = eng.estimate(0.1, 0.1, seed=0)
    pc = _np(pc)
    assert pc[0] == 0.0 and pc[2] == 0.0
    assert pc[1] == 2.0 * info["sum_internal"][1] / 4000
    assert abs(pc[1] - 1.0) < 0.1
    eng.close()


def test_errors_are_reported(binding):
    g = synth.path_graph(5)
    eng = _engine(binding, g)
    with pytest.raises(binding.PercisError) as e:
        eng.set_states(np.array([0.5, 0.5, 0.5, 0.5, 0.5]))
    assert e.value.status == 2  # DEGENERATE
    with pytest.raises(binding.PercisError) as e:
        eng.set_states(np.array([0.5, 1.5, 0.5, 0.5, 0.5]))
    assert e.value.status == 1
    with pytest.raises(binding.PercisError) as e:
        eng.set_states(np.array([0.5, np.nan, 0.5, 0.5, 0.5]))
    assert e.value.status == 1
    eng.set_states(np.array([0.9, 0.5, 0.1, 0.3, 0.7]))
    with pytest.raises(binding.PercisError) as e:
        eng.backward(torch.zeros(5, dtype=torch.float64, device="cuda"))
    assert e.value.status == 7
    bad = binding.PercIS(0)
    with pytest.raises(binding.PercisError) as e:
        bad.load_csr(np.array([0, 2, 1, 3], dtype=np.int64), np.array([1, 2, 0], dtype=np.int32))
    assert e.value.status == 1
    with pytest.raises(binding.PercisError) as e:
        bad.load_csr(np.array([0, 1, 2], dtype=np.int64), np.array([1, 7], dtype=np.int32))
    assert e.value.status == 1
    bad.close()
    eng.close()


def test_device_wait_budget_reports_timeout(binding):
    """A budget too small for any grid barrier makes every bounded wait give
    up; the call returns TIMEOUT and the context stays usable."""
    g = synth.barabasi_albert(2000, 3, 5)
    x = synth.states_uniform(g.n, 5)
    eng = _engine(binding, g, x, ell1=100, ell=200)
    eng.set_options(timeout_s=1e-9)
    with pytest.raises(binding.PercisError) as e:
        eng.estimate(0.05, 0.1, seed=0)
    assert e.value.status == 5
    eng.set_options(timeout_s=10.0)
    pc, info = eng.estimate(0.05, 0.1, seed=0)
    og = oracle.from_synth(g)
    ph = oracle.run_samples(og, oracle.prepare(x), 0, 1, 3, 0, 200, keep_paths=False)
    assert np.array_equal(np.round(_np(pc) * 200 / oracle.prepare(x).lam).astype(np.int64), ph.cnt)
    eng.close()
