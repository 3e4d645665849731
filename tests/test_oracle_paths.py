"""Pins for the oracle's sigma-counting BFS, RandomSP and exact percolation
centrality against library routines, walk counts, brute-force enumeration,
closed forms and the paper's invariants."""
import os
from fractions import Fraction

import networkx as nx
import numpy as np
import pytest
from scipy import stats
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import shortest_path

import oracle
from paper_2509_11454_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_graph(n, m, directed, seed):
    rng = np.random.default_rng(seed)
    return synth.csr_from_edges(n, rng.integers(0, n, m), rng.integers(0, n, m), directed)


def _dense(g):
    a = np.zeros((g.n, g.n), dtype=np.int64)
    for u in range(g.n):
        a[u, g.col[g.row_ptr[u]:g.row_ptr[u + 1]]] = 1
    return a


@pytest.mark.parametrize("directed", [False, True])
def test_bfs_distances_match_scipy(directed):
    g = _rand_graph(300, 700, directed, 1)
    og = oracle.from_synth(g)
    a = csr_matrix((np.ones(g.nnz), g.col, g.row_ptr), shape=(g.n, g.n))
    ref = shortest_path(a, directed=True, unweighted=True)
    for s in range(0, 300, 37):
        _, dist, _, _, _, _ = oracle.bfs(og, s)
        exp = np.where(np.isinf(ref[s]), -1, ref[s]).astype(np.int64)
        assert np.array_equal(dist.astype(np.int64), exp)


@pytest.mark.parametrize("directed", [False, True])
def test_sigma_equals_walk_counts(directed):
    """sigma_st = number of length-d(s,t) walks from s to t: a walk whose
    length equals the distance cannot revisit a vertex, so it is a shortest
    path.  (A^d)_{st} by exact integer matrix powers."""
    g = _rand_graph(60, 160, directed, 2)
    og = oracle.from_synth(g)
    A = _dense(g).astype(object)
    powers = [np.eye(g.n, dtype=object)]
    for _ in range(g.n):
        powers.append(powers[-1].dot(A))
        if len(powers) > 25:
            break
    for s in range(0, 60, 7):
        _, dist, sigma, _, _, _ = oracle.bfs(og, s)
        for t in range(g.n):
            if dist[t] >= 0:
                assert sigma[t] == float(powers[dist[t]][s, t])
            else:
                assert sigma[t] == 0.0


def test_truncated_bfs_settles_target_level():
    g = synth.grid_2d(12, 0.0, 0)
    og = oracle.from_synth(g)
    s, t = 0, 5 * 12 + 7
    ret, dist, sigma, order, edges, _ = oracle.bfs(og, s, t)
    full = oracle.bfs(og, s)
    assert ret == full[1][t] == 12
    # every vertex at distance <= d(t) is discovered with the full sigma;
    # nothing beyond d(t)
    m = full[1] <= ret
    assert np.array_equal(dist[m], full[1][m]) and np.all(dist[~m] == -1)
    assert np.array_equal(sigma[m], full[2][m])
    deg = np.diff(g.row_ptr)
    assert edges == int(deg[full[1] < ret].sum())


def test_randomsp_uniform_over_shortest_paths():
    """RandomSP returns each path of Gamma_st with probability 1/sigma_st."""
    g = synth.grid_2d(5, 0.0, 0)
    og = oracle.from_synth(g)
    s, t = 0, 24  # opposite corners: C(8,4) = 70 shortest paths
    _, dist, sigma, _, _, _ = oracle.bfs(og, s, t)
    assert sigma[t] == 70.0
    counts = {}
    N = 70 * 300
    for i in range(N):
        k, path = oracle.backtrack(og, dist, sigma, s, t, 99, 3, i)
        assert k == 7
        counts[tuple(path)] = counts.get(tuple(path), 0) + 1
    assert len(counts) == 70
    obs = np.array(list(counts.values()))
    assert stats.chisquare(obs).pvalue > 1e-4


def test_backtrack_path_is_a_shortest_path():
    g = synth.barabasi_albert(400, 2, 1)
    og = oracle.from_synth(g)
    adj = _dense(g)
    rng = np.random.default_rng(0)
    for i in range(50):
        s, t = rng.integers(0, 400, 2)
        if s == t:
            continue
        _, dist, sigma, _, _, _ = oracle.bfs(og, s, t)
        k, path = oracle.backtrack(og, dist, sigma, s, t, 5, 2, i)
        full = [t] + list(path) + [s]
        assert k == dist[t] - 1
        for a, b in zip(full[1:], full[:-1]):
            assert adj[a, b] == 1
        assert len(set(full)) == len(full)


@pytest.mark.parametrize("seed", range(6))
def test_exact_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = 8 + seed % 3
    directed = seed % 2 == 1
    g = _rand_graph(n, 2 * n + 2, directed, 100 + seed)
    x = rng.random(n)
    if seed >= 3:
        x = (rng.random(n) > 0.5).astype(float)  # binary states, many ties
        x[0], x[1] = 1.0, 0.0
    og = oracle.from_synth(g)
    pb, _ = oracle.brute_force_pc(n, g.row_ptr, g.col, x)
    _, Cv = oracle.cv_literal(x)
    pe = oracle.exact_pc(og, x, Cv)
    assert np.allclose(pe, pb, rtol=1e-12, atol=1e-14)
    assert np.all(pe >= 0) and np.all(pe <= 1 + 1e-12)


def _prop7(n):
    # a=0, b=1, c=2, H = 3..n-1
    src = [0, 1] + list(range(3, n)) + [3]
    dst = [1, 2] + [3 + (k + 1) % (n - 3) for k in range(n - 3)] + [0]
    if n - 3 == 1:
        src, dst = [0, 1, 3], [1, 2, 0]
    g = synth.csr_from_edges(n, np.array(src), np.array(dst), directed=True)
    x = np.zeros(n)
    x[0], x[2] = 1.0, 0.5
    return g, x


def test_prop7_closed_form():
    rows = []
    with open(os.path.join(GOLDEN, "prop7_instance.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                n, frac = line.split()
                rows.append((int(n), Fraction(frac)))
    for n, pb in rows:
        g, x = _prop7(n)
        og = oracle.from_synth(g)
        pe = oracle.exact_pc(og, x)
        assert pe[1] == pytest.approx(float(pb), rel=1e-13)
        others = np.delete(pe, 1)
        assert np.all(others == 0.0)
        if n <= 6:
            pbf, _ = oracle.brute_force_pc(n, g.row_ptr, g.col, x)
            assert pbf[1] == pytest.approx(float(pb), rel=1e-13)


@pytest.mark.parametrize("directed", [True, False])
def test_binary_states_reduce_to_subset_betweenness(directed):
    """x in {0,1}: p(v) = B_{S1->S0}(v) / (|S1 minus v| |S0 minus v|) with B
    the source-target subset betweenness (networkx, library routine)."""
    g = _rand_graph(40, 120, directed, 7)
    rng = np.random.default_rng(3)
    x = (rng.random(40) < 0.3).astype(float)
    og = oracle.from_synth(g)
    pe = oracle.exact_pc(og, x)
    G = nx.DiGraph() if directed else nx.Graph()
    G.add_nodes_from(range(40))
    for u in range(40):
        for v in g.col[g.row_ptr[u]:g.row_ptr[u + 1]]:
            G.add_edge(u, int(v))
    S1 = [v for v in range(40) if x[v] == 1]
    S0 = [v for v in range(40) if x[v] == 0]
    B = nx.betweenness_centrality_subset(G, S1, S0, normalized=False)
    for v in range(40):
        Cv = (len(S1) - (x[v] == 1)) * (len(S0) - (x[v] == 0))
        b = B[v] * (1.0 if directed else 2.0)  # networkx halves undirected sums
        assert pe[v] == pytest.approx(b / Cv, rel=1e-12, abs=1e-15)


def test_lemma3_and_normalisation():
    """Lemma 3: rho <= sum_v p(v) <= d^ rho, rho = sum_{s,t} |I(tau_st)| kappa~(s,t)."""
    for seed, directed in [(0, False), (1, True), (2, False)]:
        g = _rand_graph(50, 150, directed, 40 + seed)
        x = np.random.default_rng(seed).random(50)
        og = oracle.from_synth(g)
        prep = oracle.prepare(x)
        pe = oracle.exact_pc(og, x, prep.Cv)
        a = csr_matrix((np.ones(g.nnz), g.col, g.row_ptr), shape=(50, 50))
        d = shortest_path(a, directed=True, unweighted=True)
        R = np.maximum(0.0, x[:, None] - x[None, :])
        I = np.where(np.isfinite(d) & (d >= 1), d - 1, 0.0)
        rho = float((I * R).sum() / prep.c)
        assert rho - 1e-12 <= pe.sum() <= prep.dhat * rho + 1e-12
        # sum_{s != v != t} kappa(s,t,v) = 1 for every v (Section II-A)
        for v in range(0, 50, 7):
            m = np.ones(50, bool)
            m[v] = False
            assert R[np.ix_(m, m)].sum() / prep.Cv[v] == pytest.approx(1.0, rel=1e-12)


def test_vertex_diameter_bound():
    rng = np.random.default_rng(1)
    for k in range(4):
        g = _rand_graph(120, 150 + 40 * k, False, 70 + k)  # often disconnected
        og = oracle.from_synth(g)
        D = oracle.vertex_diam_ub(og)
        a = csr_matrix((np.ones(g.nnz), g.col, g.row_ptr), shape=(120, 120))
        d = shortest_path(a, directed=False, unweighted=True)
        true = int(np.max(np.where(np.isfinite(d), d, 0))) - 1
        assert D >= true
    p = synth.path_graph(30)
    assert oracle.vertex_diam_ub(oracle.from_synth(p)) == 2 * 28 - 1
    gd = _rand_graph(30, 60, True, 3)
    assert oracle.vertex_diam_ub(oracle.from_synth(gd)) == 28


def test_allpaths_fractions_match_path_enumeration():
    """f(v) = sigma_sv tau_v / sigma_st equals sigma_st(v)/sigma_st counted by
    enumerating Gamma_st (brute force), and sums to d(s,t) - 1."""
    for seed, directed in [(0, False), (1, True), (2, False)]:
        g = _rand_graph(9, 22, directed, 200 + seed)
        og = oracle.from_synth(g)
        _, paths = oracle.brute_force_pc(g.n, g.row_ptr, g.col, np.random.default_rng(seed).random(g.n))
        for (s, t), G in paths.items():
            _, dist, sigma, _, _, _ = oracle.bfs(og, s, t)
            nodes, frac = oracle.allpaths(og, dist, sigma, s, t)
            ref = {}
            for p in G:
                for v in p[1:-1]:
                    ref[v] = ref.get(v, 0) + 1.0 / len(G)
            assert dict(zip(nodes.tolist(), frac.tolist())) == pytest.approx(ref, rel=1e-12)
            assert frac.sum() == pytest.approx(len(G[0]) - 2, rel=1e-12, abs=1e-12)


def test_allpaths_estimator_unbiased():
    """The all-paths estimator has the same expectation as the path estimator (Lemma 1)."""
    g = synth.barabasi_albert(14, 2, 11)
    og = oracle.from_synth(g)
    x = np.random.default_rng(11).random(14)
    prep = oracle.prepare(x)
    pe = oracle.exact_pc(og, x, prep.Cv)
    ell, reps = 200, 150
    est = np.zeros(14)
    for k in range(reps):
        ph = oracle.run_samples(og, prep, 50 + k, 1, 3, 0, ell, keep_paths=False, allpaths=True)
        est += ph.acc_all / ell
    sd = np.sqrt(np.maximum(pe * (prep.dhat - pe), 1e-30) / (ell * reps))
    assert np.all(np.abs(est / reps - pe) <= 5 * sd + 1e-12)


def test_allpaths_estimator_lower_error():
    """Averaging over all shortest s-t paths (a conditional expectation of the
    one-path estimator given the pair) cannot raise the variance; on a grid,
    where pairs have many shortest paths, the squared error drops well below
    the one-path estimator's on the same pairs."""
    g = synth.grid_2d(24, 0.0, 0)
    x = synth.states_uniform(g.n, 4)
    og = oracle.from_synth(g)
    prep = oracle.prepare(x)
    ex = oracle.exact_pc(og, x, prep.Cv)
    e1 = e2 = 0.0
    for seed in range(4):
        r1 = oracle.percis(og, x, 0.05, 0.1, seed, ell1=1000, ell=3000, keep_paths=False, prep=prep)
        r2 = oracle.percis(og, x, 0.05, 0.1, seed, ell1=1000, ell=3000, keep_paths=False, prep=prep, allpaths=True)
        assert np.array_equal(r1.phase2.s, r2.phase2.s) and np.array_equal(r1.phase2.ilen, r2.phase2.ilen)
        e1 += float(((r1.pc - ex) ** 2).sum())
        e2 += float(((r2.pc - ex) ** 2).sum())
    assert e2 < 0.6 * e1


@pytest.mark.parametrize("directed", [False, True])
def test_bidirectional_distance_and_count_match_bfs(directed):
    """The balanced bidirectional search meets at d(s,t) with sigma_st equal
    to the one-sided BFS count (scipy-pinned distances, walk-pinned counts);
    unreachable targets give -1 on both."""
    g = _rand_graph(200, 420 if directed else 260, directed, 31)
    og = oracle.from_synth(g)
    rng = np.random.default_rng(5)
    seen_unreach = False
    for k in range(120):
        s, t = (int(v) for v in rng.integers(0, g.n, 2))
        if s == t:
            continue
        d, path, sst, _ = oracle.bibfs(og, s, t, 7, 3, k)
        ret, dist, sigma, _, _, _ = oracle.bfs(og, s, t)
        if dist[t] < 0:
            assert d == -1
            seen_unreach = True
            continue
        assert d == dist[t] and sst == sigma[t]
        assert len(path) == d - 1
    assert seen_unreach or not directed


def test_bidirectional_path_is_a_shortest_path():
    g = synth.barabasi_albert(400, 2, 1)
    og = oracle.from_synth(g)
    adj = _dense(g)
    rng = np.random.default_rng(0)
    for i in range(60):
        s, t = (int(v) for v in rng.integers(0, 400, 2))
        if s == t:
            continue
        d, path, _, _ = oracle.bibfs(og, s, t, 5, 2, i)
        ret, dist, _, _, _, _ = oracle.bfs(og, s, t)
        assert d == dist[t]
        # the internal nodes are v, then the s side from v, then the t side from v
        assert len(path) == d - 1 and len(set(path.tolist()) | {s, t}) == d + 1
        ds = {int(v): int(dist[v]) for v in path}
        order = sorted(path.tolist(), key=lambda v: ds[v])
        full = [s] + order + [t]
        for a, b in zip(full[:-1], full[1:]):
            assert adj[a, b] == 1


def test_bidirectional_randomsp_uniform_over_shortest_paths():
    """Each of the 70 corner-to-corner paths of a 5x5 grid with probability 1/70."""
    g = synth.grid_2d(5, 0.0, 0)
    og = oracle.from_synth(g)
    counts = {}
    for i in range(70 * 300):
        d, path, sst, _ = oracle.bibfs(og, 0, 24, 99, 3, i)
        assert d == 8 and sst == 70.0
        key = tuple(sorted(path.tolist()))
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 70
    assert stats.chisquare(np.array(list(counts.values()))).pvalue > 1e-4


def test_bidirectional_estimator_unbiased():
    g = synth.barabasi_albert(14, 2, 11)
    og = oracle.from_synth(g)
    x = np.random.default_rng(11).random(14)
    prep = oracle.prepare(x)
    pe = oracle.exact_pc(og, x, prep.Cv)
    ell, reps = 200, 150
    est = np.zeros(14)
    for k in range(reps):
        ph = oracle.run_samples(og, prep, 50 + k, 1, 3, 0, ell, keep_paths=False, bidir=True)
        est += ph.acc / ell
    sd = np.sqrt(np.maximum(pe * (prep.dhat - pe), 1e-30) / (ell * reps))
    assert np.all(np.abs(est / reps - pe) <= 5 * sd + 1e-12)
