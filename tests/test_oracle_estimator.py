"""Pins for the oracle's estimator, bounds and gradients: Lemma 1
(unbiasedness), Lemma 2 (variance bound), Proposition 4 (the
epsilon-guarantee), library cross-checks of Lambda and of the sup in
Theorem 1, and finite differences of the gradients."""
import math

import numpy as np
import pytest
from scipy import optimize

import oracle
from paper_2509_11454_gb300 import synth


def _small_instance(seed=0, n=12):
    g = synth.barabasi_albert(n, 2, seed)
    x = np.random.default_rng(seed).random(n)
    return g, oracle.from_synth(g), x


def test_estimator_unbiased_lemma1():
    """E_q[p~(v)] = p(v): the mean over many independent seeds converges."""
    g, og, x = _small_instance(1, 14)
    prep = oracle.prepare(x)
    pe = oracle.exact_pc(og, x, prep.Cv)
    ell, reps = 200, 300
    est = np.zeros((reps, g.n))
    for k in range(reps):
        ph = oracle.run_samples(og, prep, 1000 + k, 1, 3, 0, ell, keep_paths=False)
        est[k] = ph.acc / ell
    mean = est.mean(axis=0)
    # Lemma 2: Var[single sample] <= p (d^ - p); 5 sigma band on the mean
    sd = np.sqrt(np.maximum(pe * (prep.dhat - pe), 1e-30) / (ell * reps))
    assert np.all(np.abs(mean - pe) <= 5 * sd + 1e-12)


def test_variance_bound_lemma2():
    g, og, x = _small_instance(2, 12)
    prep = oracle.prepare(x)
    pe = oracle.exact_pc(og, x, prep.Cv)
    N = 20000
    ph = oracle.run_samples(og, prep, 5, 1, 3, 0, N, keep_paths=True)
    # per-sample values kappa/kappa~ 1[v in I]
    vals = np.zeros((N, g.n))
    for i in range(N):
        nodes = ph.path_nodes[ph.path_ptr[i]:ph.path_ptr[i + 1]]
        vals[i, nodes] = prep.lam[nodes]
    var = vals.var(axis=0, ddof=1)
    bound = pe * (prep.dhat - pe)
    assert np.all(var <= bound * 1.1 + 1e-9)


def test_lambda_is_sample_variance():
    rng = np.random.default_rng(0)
    a = rng.integers(0, 9, size=400)
    assert oracle.Lambda_literal(a) == pytest.approx(float(np.var(a, ddof=1)), rel=1e-12)


def test_ell1_default():
    assert oracle.ell1_default(0.05, 0.1) == 1000
    assert oracle.ell1_default(0.0005, 0.1) == math.ceil(math.log(10) / 0.0005)


@pytest.mark.parametrize("eps,dhat,rho,vh", [(0.05, 1.003, 2.7, 0.028), (0.005, 1.0001, 3.45, 0.079),
                                             (0.01, 1.05, 9.0, 0.2), (0.01, 1.0, 2.0, 0.25)])
def test_ell_sup_matches_library_optimizer(eps, dhat, rho, vh):
    """The grid + golden-section sup of Theorem 1's objective agrees with a
    dense log grid refined by scipy's bounded scalar minimiser."""
    delta = 0.1
    xh = oracle.x_hat(vh, dhat)
    ell, best = oracle.ell_sup(eps, delta, dhat, rho, xh)
    f = lambda lx: -oracle.ell_objective(math.exp(lx), eps, delta, dhat, rho)
    grid = np.linspace(math.log(xh) - 12 * math.log(10), math.log(xh), 200001)
    vals = np.array([-f(v) for v in grid[::50]])
    k = int(np.argmax(vals))
    lo = grid[max(0, (k - 1) * 50)]
    hi = grid[min(len(grid) - 1, (k + 1) * 50)]
    r = optimize.minimize_scalar(f, bounds=(lo, hi), method="bounded", options={"xatol": 1e-12})
    ref = max(-r.fun, vals.max())
    assert best == pytest.approx(ref, rel=1e-9)
    assert ell == math.ceil(best)
    # the paper's approximation (Section III-C): (2v^ + 2/3 eps d^)/eps^2 (ln(d^ rho^/v^) + ln(2/delta))
    approx = (2 * vh + 2.0 / 3.0 * eps * dhat) / eps ** 2 * (math.log(dhat * rho / vh) + math.log(2 / delta))
    assert 0.5 * approx <= ell <= 2.0 * approx


def test_xhat_properties():
    assert oracle.x_hat(10.0, 1.0) == pytest.approx(0.5)
    # x^ solves g(x^) = v^ when v^ <= d^2/4
    for vh in (1e-4, 0.01, 0.2):
        xh = oracle.x_hat(vh, 1.0)
        assert xh * (1.0 - xh) == pytest.approx(vh, rel=1e-9)


def test_epsilon_guarantee_er1000():
    """Proposition 4: an eps-approximation with probability >= 1 - delta;
    over 20 seeds at least 18 must meet eps (G(1000, M=4000), eps = 0.05)."""
    g, x, eps, delta = synth.workload("er1000")
    og = oracle.from_synth(g)
    prep = oracle.prepare(x)
    pe = oracle.exact_pc(og, x, prep.Cv)
    ok = 0
    for seed in range(20):
        res = oracle.percis(og, x, eps, delta, seed, prep=prep, keep_paths=False)
        if np.max(np.abs(res.pc - pe)) <= eps:
            ok += 1
        assert np.allclose(res.pc, res.pc_counts, rtol=1e-12, atol=1e-15)
    assert ok >= 18


def test_fixed_sample_vjp_matches_finite_differences():
    g = synth.barabasi_albert(80, 3, 4)
    og = oracle.from_synth(g)
    x = np.random.default_rng(4).random(80)
    prep = oracle.prepare(x)
    ell = 400
    ph = oracle.run_samples(og, prep, 17, 1, 3, 0, ell, keep_paths=True)
    F = ph.acc / ell
    gvec = np.random.default_rng(5).standard_normal(80)
    grad = oracle.vjp_fixed(prep, ell, ph, F, gvec)
    h = 1e-6
    checked = 0
    for u in range(80):
        if np.any(np.abs(np.delete(x, u) - x[u]) < 4 * h):
            continue
        touch = (ph.kind == 0) & ((ph.s == u) | (ph.t == u))
        if np.any(np.abs(x[ph.s[touch]] - x[ph.t[touch]]) <= 1e-3):
            continue
        fd = oracle.fd_fixed(prep, ell, ph, gvec, u, h)
        assert grad[u] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(grad).max())
        checked += 1
    assert checked > 60


def test_exact_vjp_matches_finite_differences():
    g = synth.barabasi_albert(14, 2, 6)
    og = oracle.from_synth(g)
    x = np.random.default_rng(6).random(14)
    gvec = np.random.default_rng(7).standard_normal(14)
    grad = oracle.exact_vjp(og, x, gvec)
    h = 1e-6
    for u in range(14):
        xp, xm = x.copy(), x.copy()
        xp[u] += h
        xm[u] -= h
        # literal C_v keeps the perturbed evaluation independent of the
        # closed forms used elsewhere
        lp = float(np.dot(gvec, oracle.exact_pc(og, xp, oracle.cv_literal(xp)[1])))
        lm = float(np.dot(gvec, oracle.exact_pc(og, xm, oracle.cv_literal(xm)[1])))
        assert grad[u] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-8)


def test_is_gradient_is_unbiased_for_exact_gradient():
    """The fixed-sample gradient is an importance-sampling estimate of the
    exact gradient: its mean over seeds approaches the exact VJP."""
    g = synth.barabasi_albert(12, 2, 8)
    og = oracle.from_synth(g)
    x = np.random.default_rng(8).random(12)
    prep = oracle.prepare(x)
    gvec = np.random.default_rng(9).standard_normal(12)
    exact = oracle.exact_vjp(og, x, gvec, prep.Cv)
    ell, reps = 400, 200
    acc = np.zeros(12)
    sq = np.zeros(12)
    for k in range(reps):
        ph = oracle.run_samples(og, prep, 300 + k, 1, 3, 0, ell, keep_paths=True)
        gr = oracle.vjp_fixed(prep, ell, ph, ph.acc / ell, gvec)
        acc += gr
        sq += gr * gr
    mean = acc / reps
    sd = np.sqrt(np.maximum(sq / reps - mean ** 2, 0) / reps)
    assert np.all(np.abs(mean - exact) <= 5 * sd + 1e-3 * np.abs(exact).max())


def test_fixed_sample_vjp_invariances():
    """R(x_s - x_t) and C_v(x) are unchanged by x -> x + c and scale by a
    under x -> a x, so the fixed-sample estimator F is invariant under both
    and its VJP satisfies sum_u grad_u = 0 and sum_u x_u grad_u = 0 (Euler's
    identity for degree-0 homogeneous functions)."""
    g = synth.barabasi_albert(300, 3, 6)
    og = oracle.from_synth(g)
    x = np.random.default_rng(6).random(300)
    prep = oracle.prepare(x, cv_method="sorted")
    ell = 1500
    ph = oracle.run_samples(og, prep, 21, 1, 3, 0, ell, keep_paths=True)
    F = ph.acc / ell
    gvec = np.random.default_rng(7).standard_normal(300)
    grad = oracle.vjp_fixed(prep, ell, ph, F, gvec)
    assert abs(grad.sum()) <= 1e-11 * np.abs(grad).sum()
    assert abs((x * grad).sum()) <= 1e-11 * np.abs(x * grad).sum()


def test_percis_di_guarantee_and_larger_sample():
    """PercIS-DI (rho^ = D, v^ = d^2/4, no first phase) keeps the eps
    guarantee (>= 18 of 20 seeds on G(1000, M=4000)) and never needs fewer
    samples than the data-dependent bound (Section V: DI is always larger)."""
    g, x, eps, delta = synth.workload("er1000")
    og = oracle.from_synth(g)
    prep = oracle.prepare(x)
    pe = oracle.exact_pc(og, x, prep.Cv)
    D = oracle.vertex_diam_ub(og)
    ok = 0
    for seed in range(20):
        res = oracle.percis(og, x, eps, delta, seed, prep=prep, D=D, keep_paths=False, data_independent=True)
        assert res.ell1 == 0 and res.rho_hat == D and res.x_hat == pytest.approx(prep.dhat / 2, rel=1e-12)
        ok += int(np.max(np.abs(res.pc - pe)) <= eps)
        if seed < 3:
            dd = oracle.percis(og, x, eps, delta, seed, prep=prep, D=D, keep_paths=False)
            assert res.ell >= dd.ell
    assert ok >= 18


def test_state_settings_inputs():
    """The Section V-A state settings as generated: seeds-spread states are
    max_s 4^-d(s, v) over the seeds (x = 1), with d from the oracle's BFS; the
    isolated component is a separate 50-vertex path with 25 states at 1."""
    g = synth.barabasi_albert(2000, 3, 4)
    x = synth.states_seeds_spread(g, 1)
    og = oracle.from_synth(g)
    seeds = np.flatnonzero(x == 1.0)
    assert len(seeds) == int(np.ceil(np.log(g.n)))
    ref = np.zeros(g.n)
    for s in seeds:
        _, dist, _, _, _, _ = oracle.bfs(og, int(s))  # dist -1: unreached
        ref = np.maximum(ref, np.where(dist >= 0, 4.0 ** (-dist.astype(np.float64)), 0.0))
    assert np.array_equal(x, ref)
    h, xi = synth.isolated_component(g, 2)
    assert h.n == g.n + 50 and xi[: g.n].max() == 0.0 and xi[g.n:].sum() == 25.0
    oh = oracle.from_synth(h)
    _, dist, _, _, _, _ = oracle.bfs(oh, g.n)
    assert np.all(dist[: g.n] == -1)  # a component of its own
    assert np.array_equal(dist[g.n:], np.arange(50))  # a path from its first vertex
