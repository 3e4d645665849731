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
