"""Pins for the oracle's phase-1 bounds rho^ (Proposition 2) and v^
(Proposition 3) against the guarantees they exist to give.

Algorithm 1 applies both propositions at confidence delta/4 (proof of
Proposition 4), so over independent phase-1 samples
  * rho^ >= rho = sum_{s,t} kappa~(s,t) |I(s,t)| must hold in >= 1 - delta/4
    of them, and
  * v^ >= max_v Var_q[X_v] must hold in >= 1 - delta/4 of them, with
    X_v = kappa(s,t,v)/kappa~(s,t) 1[v in I] = lambda_v 1[v in I], so
    E[X_v] = p(v), E[X_v^2] = lambda_v p(v) and Var_q[X_v] = lambda_v p(v) - p(v)^2.
    The proof of Proposition 3 passes through max_v p(v) <= v^/d^, which is
    checked too (the sharper of the two claims).

The targets come from elsewhere: rho from scipy's all-pairs BFS distances
(|I| = d(s,t) - 1 for reachable pairs, 0 otherwise) and kappa~ = R/C; p(v)
from the exact percolation centrality, itself pinned by brute-force
enumeration of shortest paths.

A coverage rate alone cannot fail for a bound that is merely too loose, so
each test also plants the plausible mistakes on the CPU (a dropped term) and
asserts that the coverage then falls below 1 - delta/4 on an instance chosen
to expose it:
  * the square-root terms bind when l1 is large (WS(100, 4, 0.1), BA(200, 2));
  * the D term of rho^ and the log/(3 l1) term of v^ bind when l1 is small and
    most of the weight sits on adjacent pairs (K_100 plus one pendant vertex),
    where a phase-1 sample often sees no internal vertex at all.
The constant inside the logarithms (8/delta, 4/delta) changes the coverage of
these conservative bounds too little to be seen by sampling; it is pinned by
test_bounds_are_the_propositions_at_delta_over_4, which rebuilds both bounds
from the published inequalities (Maurer and Pontil's empirical Bernstein
bound for [0,1] variables with numpy's sample variance, scaled by D; the
self-bounding bound on max p scaled by d^) at confidence delta/4."""
import math

import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import shortest_path

import oracle
from paper_2509_11454_gb300 import synth

DELTA = 0.1
REPS = 400
NEED = 1.0 - DELTA / 4.0


def _rho_exact(g, x):
    a = csr_matrix((np.ones(g.nnz), g.col, g.row_ptr), shape=(g.n, g.n))
    d = shortest_path(a, directed=g.directed, unweighted=True)
    R = np.maximum(0.0, x[:, None] - x[None, :])
    internal = np.where(np.isfinite(d) & (d >= 1), d - 1.0, 0.0)
    np.fill_diagonal(internal, 0.0)
    return float((R * internal).sum() / R.sum())


def _k_plus_pendant(m):
    iu = np.triu_indices(m, 1)
    src = np.concatenate([iu[0], [0]])
    dst = np.concatenate([iu[1], [m]])
    return synth.csr_from_edges(m + 1, src, dst, directed=False, name=f"K{m}+pendant")


INSTANCES = {
    # name: (graph, states, l1)
    "ws100_l2000": (lambda: synth.watts_strogatz(100, 4, 0.1, 0), 5, 2000),
    "ba200_l500": (lambda: synth.barabasi_albert(200, 2, 0), 5, 500),
    "k100pendant_l50": (lambda: _k_plus_pendant(100), 3, 50),
}


def _draws(name):
    make, xseed, l1 = INSTANCES[name]
    g = make()
    x = synth.states_uniform(g.n, xseed)
    og = oracle.from_synth(g)
    prep = oracle.prepare(x)
    assert np.all(prep.Cv > 0)
    pe = oracle.exact_pc(og, x, prep.Cv)
    D = oracle.vertex_diam_ub(og)
    out = []
    for k in range(REPS):
        ph = oracle.run_samples(og, prep, 7000 + k, 0, 2, 0, l1, keep_paths=False)
        out.append((ph.ilen.copy(), float((ph.acc / l1).max())))
    return g, x, prep, pe, D, l1, out


_CACHE = {}


def draws(name):
    if name not in _CACHE:
        _CACHE[name] = _draws(name)
    return _CACHE[name]


def _rho_parts(ilen, D, l1):
    a = np.asarray(ilen, dtype=np.float64)
    lg = math.log(8.0 / DELTA)
    return (a.mean(), math.sqrt(2.0 * oracle.Lambda_sums(ilen) * lg / l1), 7.0 * D * lg / (3.0 * (l1 - 1)))


def _v_parts(pm, l1):
    lg = math.log(4.0 / DELTA)
    return pm, math.sqrt(2.0 * pm * lg / l1), lg / (3.0 * l1)


@pytest.mark.parametrize("name,dropped", [("ws100_l2000", "sqrt"), ("k100pendant_l50", "D")])
def test_rho_hat_covers_rho(name, dropped):
    """Proposition 2 at delta/4: rho^ >= rho in >= 1 - delta/4 of the phase-1
    samples; without the named term the coverage falls below that."""
    g, x, prep, pe, D, l1, out = draws(name)
    rho = _rho_exact(g, x)
    # Proposition 1's sum: rho <= sum_v p(v) <= d^ rho (Lemma 3) ties rho to the exact PC
    assert rho <= pe.sum() * (1 + 1e-12) and pe.sum() <= prep.dhat * rho * (1 + 1e-12)
    ok = bad = 0
    for ilen, _ in out:
        rh, rt, _lam = oracle.rho_hat(ilen, D, DELTA)
        mean, sq, dterm = _rho_parts(ilen, D, l1)
        assert rt == pytest.approx(mean, rel=1e-15)
        ok += rh >= rho
        bad += (mean + dterm if dropped == "sqrt" else mean + sq) >= rho
    assert ok / REPS >= NEED
    assert bad / REPS < NEED


@pytest.mark.parametrize("name,dropped", [("ba200_l500", "sqrt"), ("ws100_l2000", "sqrt"),
                                          ("k100pendant_l50", "last")])
def test_v_hat_covers_max_variance(name, dropped):
    """Proposition 3 at delta/4: v^ >= max_v Var_q[X_v] and v^/d^ >= max_v p(v)
    in >= 1 - delta/4 of the phase-1 samples; without the named term the
    coverage of the second claim falls below that."""
    g, x, prep, pe, D, l1, out = draws(name)
    var = prep.lam * pe - pe * pe
    # Lemma 2 (the step of Proposition 3's proof): Var <= d^ p(v)
    assert np.all(var <= prep.dhat * pe * (1 + 1e-12))
    ok_var = ok_p = bad = 0
    for _, pm in out:
        vh = oracle.v_hat(pm, prep.dhat, l1, DELTA)
        a, sq, last = _v_parts(pm, l1)
        ok_var += vh >= var.max()
        ok_p += vh / prep.dhat >= pe.max()
        kept = a + last if dropped == "sqrt" else a + sq
        bad += prep.dhat * kept >= pe.max()
    assert ok_var / REPS >= NEED
    assert ok_p / REPS >= NEED
    assert bad / REPS < NEED


def test_bounds_are_the_propositions_at_delta_over_4():
    """The constants: rho^ is Maurer and Pontil's empirical Bernstein bound
    (their Theorem 4: for i.i.d. Z in [0,1], E Z <= mean + sqrt(2 V ln(2/d')/l)
    + 7 ln(2/d')/(3(l-1)) with V the unbiased sample variance) applied to
    Z = |I|/D and rescaled by D; v^ is d^ times the self-bounding bound
    d^ {p~ + sqrt(2 p~ ln(1/d')/l) + ln(1/d')/(3 l)} on max p; both at
    d' = delta/4 (Proposition 4's union bound over four events)."""
    rng = np.random.default_rng(11)
    dp = DELTA / 4.0
    for _ in range(200):
        l1 = int(rng.integers(2, 3000))
        D = int(rng.integers(1, 60))
        ilen = rng.integers(0, D + 1, size=l1)
        z = ilen / D
        mp = z.mean() + math.sqrt(2.0 * np.var(z, ddof=1) * math.log(2.0 / dp) / l1) + \
            7.0 * math.log(2.0 / dp) / (3.0 * (l1 - 1))
        assert oracle.rho_hat(ilen, D, DELTA)[0] == pytest.approx(D * mp, rel=1e-12)
        pm = float(rng.random()) * 1.5
        dh = 1.0 + float(rng.random())
        sb = dh * (pm + math.sqrt(2.0 * pm * math.log(1.0 / dp) / l1) + math.log(1.0 / dp) / (3.0 * l1))
        assert oracle.v_hat(pm, dh, l1, DELTA) == pytest.approx(dh * sb, rel=1e-12)


def test_lambda_sums_equals_pairwise_form():
    """Proposition 2's Lambda: the two-sum form is bit-identical to the
    literal pairwise sum (same integer numerator, one division)."""
    rng = np.random.default_rng(5)
    for L in (2, 3, 17, 400):
        for hi in (1, 9, 1000):
            a = rng.integers(0, hi + 1, size=L)
            assert oracle.Lambda_sums(a) == oracle.Lambda_literal(a)
