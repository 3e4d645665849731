"""The reasoning behind the parallel evaluation of Algorithm 2's running sums
(the table kernel), checked on the CPU: inside one binade a non-decreasing FP64
running sum is an integer sum in units of its ulp, halfway roundings resolved by
the parity of the sum before the term (ties to even), and a term whose sum
leaves the binade is added once in plain FP64.  This model processes chunks of
terms the way the kernel does (per-term maps composed left to right, first
crossing found, restart after it) and must reproduce the sequential sum bit for
bit on inputs with halfway cases, subnormal terms, runs of zeros and sums that
cross many binades."""
import struct

import numpy as np
import pytest

TWO53 = 1 << 53


def _bits(x: float) -> int:
    return struct.unpack("<q", struct.pack("<d", x))[0]


def _dbl(b: int) -> float:
    return struct.unpack("<d", struct.pack("<q", b))[0]


def _term(a: float, e: int):
    """(q, kind) of a term against a binade of exponent field e >= 1:
    kind 0 exact or rounded down, 1 up, 2 halfway, 3 leaves the binade alone."""
    ab = _bits(a)
    ea = (ab >> 52) & 0x7FF
    if ea > e:
        return TWO53, 3
    ma = (ab & ((1 << 52) - 1)) | ((1 << 52) if ea else 0)
    sh = e - max(ea, 1)
    if sh == 0:
        return ma, 0
    if sh > 54:
        return 0, 0
    rem, half = ma & ((1 << sh) - 1), 1 << (sh - 1)
    return ma >> sh, (1 if rem > half else 2 if rem == half else 0)


def chunked_running_sum(terms, chunk):
    out, s, pos = [0.0] * len(terms), 0.0, 0
    while pos < len(terms):
        cnt = min(chunk, len(terms) - pos)
        b = _bits(s)
        es = (b >> 52) & 0x7FF
        e = max(es, 1)
        s0 = (b & ((1 << 52) - 1)) | ((1 << 52) if es else 0)
        p, acc, kstar, vals = s0 & 1, 0, cnt, []
        for k in range(cnt):
            q, kind = _term(terms[pos + k], e)
            if kind == 2:
                r = q + ((q ^ p) & 1)
                p = 0
            else:
                r = q + (kind & 1)
                p ^= r & 1
            acc += r
            if kind == 3 or s0 + acc >= TWO53:
                kstar = k
                break
            vals.append(s0 + acc)
        for k in range(kstar):
            out[pos + k] = _dbl(((e - 1) << 52) + vals[k])
        if kstar < cnt:
            prev = _dbl(((e - 1) << 52) + vals[kstar - 1]) if kstar > 0 else s
            s = prev + terms[pos + kstar]  # one plain FP64 add where the sum leaves its binade
            out[pos + kstar] = s
            pos += kstar + 1
        else:
            s = out[pos + cnt - 1]
            pos += cnt
    return out


def _sequential(terms):
    s, out = 0.0, []
    for a in terms:
        s = s + a
        out.append(s)
    return out


def _inputs(kind, n, seed=3):
    rng = np.random.default_rng(seed)
    if kind == "halfway":
        return list(rng.integers(2 ** 39, 2 ** 40, n) * 2.0 ** -40)
    if kind == "dyadic":
        return list(rng.integers(1, 4097, n) / 4096.0)
    if kind == "subnormal":
        pool = [0.0, 5e-324, 7e-322, 1e-310, 2.2250738585072014e-308, 1e-300, 0.5]
        return [pool[i] if rng.random() < 0.6 else float(rng.random()) for i in rng.integers(0, len(pool), n)]
    if kind == "zeros":
        return [0.0] * (n // 2) + list(rng.random(n - n // 2))
    if kind == "binades":
        return sorted(float(v) for v in rng.random(n) * 10.0 ** (-rng.random(n) * 300.0))
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["halfway", "dyadic", "subnormal", "zeros", "binades"])
@pytest.mark.parametrize("chunk", [1, 7, 64, 4096])
def test_chunked_exact_sum_equals_sequential(kind, chunk):
    terms = _inputs(kind, 3000)
    got = chunked_running_sum(terms, chunk)
    ref = _sequential(terms)
    assert [_bits(v) for v in got] == [_bits(v) for v in ref]


def test_halfway_cases_are_exercised():
    """The halfway input really has ties once the sum passes 2^13."""
    terms = _inputs("halfway", 30000)
    s, ties = 0.0, 0
    for a in terms:
        if s > 0:
            e = max((_bits(s) >> 52) & 0x7FF, 1)
            ties += _term(a, e)[1] == 2
        s += a
    assert ties > 1000


# ---------------------------------------------------------------- predicted pass

def _key(v: float) -> int:
    return max((_bits(v) >> 52) & 0x7FF, 1)


def _map(a: float, e: int):
    """(d0, d1, par) of one term against binade key e: the integer added for
    parity 0 / 1 of the sum before it, bit p of par the parity after it."""
    q, kind = _term(a, e)
    if kind == 2:
        return q + (q & 1), q + 1 - (q & 1), 0
    r = q + (kind & 1)
    b = r & 1
    return r, r, b | ((b ^ 1) << 1)


def _then(f, g):
    f0, f1 = f[2] & 1, (f[2] >> 1) & 1
    return (f[0] + (g[1] if f0 else g[0]), f[1] + (g[1] if f1 else g[0]),
            ((g[2] >> f0) & 1) | (((g[2] >> f1) & 1) << 1))


IDENT = (0, 0, 2)


def predicted_running_sum(terms, nthreads, max_segs=256, shift_pred=None):
    """The table kernel's predicted pass: per-thread FP64 sums give every term a
    predicted prefix (another summation order), a change of its binade key
    starts a segment, each segment's run of per-term maps is composed, and the
    binades are walked in order from s = +0 -- first term by a plain add, the
    run below the binade's top -- until a check fails; the terms from there
    on go to the windowed scan.  shift_pred(k, key) may alter a predicted key
    (to exercise the checks)."""
    m = len(terms)
    if m == 0:
        return []
    T = -(-m // nthreads)
    ranges = [(min(m, t * T), min(m, t * T + T)) for t in range(nthreads)]
    # prediction: exclusive prefix of the thread sums, then running adds
    sums = []
    for k0, k1 in ranges:
        s = 0.0
        for k in range(k0, k1):
            s += terms[k]
        sums.append(s)
    pins, acc = [], 0.0
    for s in sums:
        pins.append(acc)
        acc += s
    keys, conflict = [None] * m, False
    last_keys = []
    for (k0, k1), pin in zip(ranges, pins):
        key_in = -1 if k0 == 0 else _key(pin)
        if k0 < k1 and last_keys and key_in != last_keys[-1]:
            conflict = True
        P, before = pin, key_in
        for k in range(k0, k1):
            P += terms[k]
            e = _key(P)
            if shift_pred is not None:
                e = shift_pred(k, e)
            keys[k] = e
            before = e
        last_keys.append(before)
    # segments: starts where the key changes (term 0 always)
    starts = [k for k in range(m) if k == 0 or keys[k] != keys[k - 1]]
    seen = set()
    for k in starts:
        if keys[k] in seen:
            conflict = True
        seen.add(keys[k])
    out = [None] * m
    fail = 0 if conflict or len(starts) > max_segs else m
    S = 0.0
    if fail == m:
        for i, b in enumerate(starts):
            e = keys[b]
            end_k = starts[i + 1] if i + 1 < len(starts) else m
            sc = S + terms[b]
            if _key(sc) != e:
                fail = b
                break
            sb = _bits(sc)
            es = (sb >> 52) & 0x7FF
            s0 = (sb & ((1 << 52) - 1)) | ((1 << 52) if es else 0)
            run, vals = IDENT, []
            for k in range(b + 1, end_k):
                run = _then(run, _map(terms[k], e))
                vals.append(run[1] if s0 & 1 else run[0])
            if s0 + (vals[-1] if vals else 0) >= TWO53:
                fail = b
                break
            out[b] = sc
            for j, d in enumerate(vals):
                out[b + 1 + j] = _dbl(((e - 1) << 52) + s0 + d)
            S = _dbl(((e - 1) << 52) + s0 + (vals[-1] if vals else 0))
    if fail < m:  # the windowed scan from the sum before term `fail`
        rest = chunked_running_sum_from(terms[fail:], 4096, S)
        out[fail:] = rest
    return out


def chunked_running_sum_from(terms, chunk, s0_value):
    """chunked_running_sum started from the running sum s0_value."""
    shifted = chunked_running_sum([s0_value] + list(terms), chunk) if s0_value != 0.0 else \
        chunked_running_sum(list(terms), chunk)
    return shifted[1:] if s0_value != 0.0 else shifted


@pytest.mark.parametrize("kind", ["halfway", "dyadic", "subnormal", "zeros", "binades", "beta"])
@pytest.mark.parametrize("nthreads", [1, 5, 64, 1000])
def test_predicted_pass_equals_sequential(kind, nthreads):
    terms = _inputs(kind, 3000) if kind != "beta" else \
        sorted(np.random.default_rng(9).beta(0.5, 2.0, 3000).tolist())
    assert [_bits(v) for v in predicted_running_sum(terms, nthreads)] == [_bits(v) for v in _sequential(terms)]


def test_predicted_pass_checks_catch_wrong_predictions():
    """Keys shifted one binade early or late at one term are caught (a first
    term off its binade, a run past its top, a binade entered twice) and the
    rest of the sum comes from the windowed scan, still bit for bit."""
    terms = sorted(np.random.default_rng(2).beta(0.5, 2.0, 2000).tolist())
    ref = [_bits(v) for v in _sequential(terms)]
    for at in (0, 1, 37, 500, 1999):
        for delta in (-1, 1):
            got = predicted_running_sum(terms, 16, shift_pred=lambda k, e: e + delta if k == at else e)
            assert [_bits(v) for v in got] == ref
    # more binades than the resolution holds: all from the windowed scan
    assert [_bits(v) for v in predicted_running_sum(terms, 16, max_segs=2)] == ref
