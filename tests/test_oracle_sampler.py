"""Pins for the oracle's random numbers, sorted tables and pair sampler
(Algorithm 2).  Each check compares against something other than the oracle:
published known-answer vectors, closed forms written from the paper, exact
rational arithmetic, or a chi-square test against kappa~(s,t)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(v, 16) for v in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = oracle.philox4x32_10(r[0:4], r[4:6])
        assert out.tolist() == r[6:10]


def test_uniforms_open_closed_interval_and_uniform():
    us = np.array([oracle.uniforms(12345, i, 0, 0) for i in range(20000)]).ravel()
    assert us.min() > 0.0 and us.max() <= 1.0
    # Kolmogorov-Smirnov against U(0,1) (library routine)
    assert stats.kstest(us, "uniform").pvalue > 1e-4
    # distinct tags / counters give different streams
    assert oracle.uniforms(1, 0, 0, 0) != oracle.uniforms(1, 0, 1, 0)
    assert oracle.uniforms(1, 0, 0, 0) != oracle.uniforms(1, 0, 0, 1)
    assert oracle.uniforms(1, 0, 0, 0) != oracle.uniforms(2, 0, 0, 0)


def test_sort_states_non_increasing_stable():
    rng = np.random.default_rng(3)
    x = rng.integers(0, 5, size=200) / 4.0  # many ties
    perm, xs = oracle.sort_states(x)
    assert sorted(perm.tolist()) == list(range(200))
    assert np.all(np.diff(xs) <= 0)
    for a, b in zip(perm[:-1], perm[1:]):
        if x[a] == x[b]:
            assert a < b  # ties by ascending node id
    # against numpy's stable lexsort (library routine)
    ref = np.lexsort((np.arange(200), -x))
    assert np.array_equal(perm, ref)


@pytest.mark.parametrize("n,seed", [(7, 0), (25, 1), (60, 2)])
def test_tables_match_closed_forms(n, seed):
    """Closed forms of Algorithm 2's tables (proof of Proposition 1):
    w_i = sum_{j>=i} x_j, c_i = sum_{j>=i} R(x_i - x_j), r_i = sum_{j>=i} c_j,
    c = sum_{u != w} R(x_u - x_w)."""
    rng = np.random.default_rng(seed)
    x = rng.random(n)
    x[: n // 3] = np.round(x[: n // 3], 1)  # some ties
    perm, xs = oracle.sort_states(x)
    w, ci, r, c = oracle.tables(xs)
    R = lambda a: a if a > 0 else 0.0
    for i in range(1, n + 1):
        wi = math.fsum(xs[i - 1:])
        ci_ref = math.fsum(R(xs[i - 1] - xs[j - 1]) for j in range(i, n + 1))
        assert w[i] == pytest.approx(wi, rel=1e-13, abs=1e-13)
        assert ci[i] == pytest.approx(ci_ref, rel=1e-12, abs=1e-12)
    for i in range(1, n + 1):
        assert r[i] == pytest.approx(math.fsum(ci[i:n + 1]), rel=1e-12, abs=1e-12)
    c_ref = math.fsum(R(x[u] - x[v]) for u in range(n) for v in range(n) if u != v)
    assert c == pytest.approx(c_ref, rel=1e-12)
    assert c == r[1]  # same accumulation order, so bit-identical


def _exact_marginals(xs):
    """Exact rational cumulative marginals sum_{i<=x} sum_z kappa~(i,z)
    (proof of Proposition 1) from the doubles xs."""
    fx = [Fraction(v) for v in xs]
    n = len(fx)
    rows = [sum((fx[i] - fx[j] for j in range(n) if fx[i] > fx[j]), Fraction(0)) for i in range(n)]
    tot = sum(rows, Fraction(0))
    cum, acc = [], Fraction(0)
    for v in rows:
        acc += v
        cum.append(acc / tot)
    return rows, cum, tot


def test_first_search_is_inverse_cdf():
    rng = np.random.default_rng(5)
    x = rng.random(40)
    perm, xs = oracle.sort_states(x)
    w, ci, r, c = oracle.tables(xs)
    rows, cum, tot = _exact_marginals(xs)
    # the k evaluated by the first search is (c - r_{x+1})/c: equal to the
    # exact cumulative marginal up to rounding
    for xx in range(1, 41):
        k = (c - r[xx + 1]) / c
        assert abs(k - float(cum[xx - 1])) < 1e-12
    mism = 0
    for _ in range(4000):
        u = float(rng.random()) or 1.0
        s = oracle.lib().orc_search_s(40, oracle._p(r), c, u)
        s_ref = next(i + 1 for i, cv in enumerate(cum) if cv >= Fraction(u))
        if s != s_ref:
            # only allowed where u sits within rounding of a boundary
            assert min(abs(float(cv) - u) for cv in cum) < 1e-12
            mism += 1
    assert mism <= 2


def test_pair_distribution_chisquare():
    """Pairs follow kappa~(s,t) = R(x_s - x_t)/C (Section III-A)."""
    x = np.array([0.9, 0.1, 0.55, 0.3, 0.75, 0.0, 0.42])
    n = len(x)
    prep = oracle.prepare(x)
    N = 200_000
    s, t, sp, tp = oracle.sample_pairs(prep, seed=7, tag=0, i0=0, count=N)
    counts = np.zeros((n, n))
    np.add.at(counts, (s, t), 1)
    R = np.maximum(0.0, x[:, None] - x[None, :])
    p = R / R.sum()
    assert counts[p == 0].sum() == 0  # zero-weight pairs never drawn
    mask = p > 0
    chi = stats.chisquare(counts[mask], N * p[mask])
    assert chi.pvalue > 1e-4
    assert np.all(tp >= sp)


def test_pairs_reproducible_and_index_addressed():
    x = np.random.default_rng(9).random(300)
    prep = oracle.prepare(x)
    s1, t1, _, _ = oracle.sample_pairs(prep, 11, 1, 0, 500)
    s2, t2, _, _ = oracle.sample_pairs(prep, 11, 1, 200, 300)
    assert np.array_equal(s1[200:], s2) and np.array_equal(t1[200:], t2)


def test_cv_forms_agree():
    """C_v three ways: the literal double sum of Definition 1 (O(n^3)), the
    C - sum|x_v - x_u| identity (proof of Proposition 5) and the sorted-prefix
    closed form."""
    rng = np.random.default_rng(4)
    for n in (5, 13, 40):
        x = rng.random(n)
        x[:3] = 0.5
        C1, Cl = oracle.cv_literal(x)
        C2, Cd = oracle.cv_direct(x)
        prep = oracle.prepare(x, cv_method="sorted")
        assert C1 == pytest.approx(C2, rel=1e-14)
        assert np.allclose(Cl, Cd, rtol=1e-12, atol=1e-12)
        assert np.allclose(Cl, prep.Cv, rtol=1e-12, atol=1e-12)


def test_likelihood_ratio_closed_form():
    """d_v = max over pairs with kappa~ > 0 of kappa(s,t,v)/kappa~(s,t)
    (Section III-A) equals C / C_v (proof of Proposition 5)."""
    rng = np.random.default_rng(8)
    n = 9
    x = rng.random(n)
    C, Cv = oracle.cv_literal(x)
    for v in range(n):
        best = 0.0
        for s in range(n):
            for t in range(n):
                R = max(0.0, x[s] - x[t])
                if R <= 0 or s == v or t == v:
                    continue
                best = max(best, (R / Cv[v]) / (R / C))
        assert best == pytest.approx(C / Cv[v], rel=1e-13)
    prep = oracle.prepare(x, cv_method="literal")
    assert prep.dhat == pytest.approx(max(C / Cv), rel=1e-13)
