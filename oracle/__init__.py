"""CPU oracle for PercIS -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library and its Python
binding never import it; the two implementations share no code.

The heavy loops live in ``percis_oracle.c`` (plain C, FP64, one thread,
-ffp-contract=off).  This module builds and loads it and adds the pieces that
are clearest in Python: the brute-force Definition 1 for tiny graphs, the
bound quantities of Algorithm 1 / Theorem 1 / Propositions 2-3, the
two-phase driver of Algorithm 1, and central finite differences of the
fixed-sample estimator in difference form.

Parity status: every function here is pinned by a test in tests/ against
something other than itself (closed forms, brute force, library routines,
published Philox known-answer vectors, statistical properties of the paper's
lemmas).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "percis_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2 -ffp-contract=off)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_LIB_PATH)
            _declare(_lib)
        return _lib


P = ctypes.c_void_p
I64 = ctypes.c_int64
I32 = ctypes.c_int32
U32 = ctypes.c_uint32
U64 = ctypes.c_uint64
F64 = ctypes.c_double


def _declare(L):
    L.orc_philox4x32_10.argtypes = [P, P, P]
    L.orc_uniforms.argtypes = [U64, U64, U32, U32, P]
    L.orc_sort_states.argtypes = [I64, P, P, P]
    L.orc_tables.argtypes = [I64, P, P, P, P]
    L.orc_tables.restype = F64
    L.orc_search_s.argtypes = [I64, P, F64, F64]
    L.orc_search_s.restype = I64
    L.orc_search_t.argtypes = [I64, I64, P, P, P, F64]
    L.orc_search_t.restype = I64
    L.orc_sample_pairs.argtypes = [I64, P, P, P, P, P, F64, U64, U32, I64, I64, P, P, P, P]
    L.orc_transpose.argtypes = [I64, P, P, P, P]
    L.orc_bfs.argtypes = [I64, P, P, P, P, I32, I32, P, P, P, P, P, P]
    L.orc_bfs.restype = I64
    L.orc_backtrack.argtypes = [P, P, P, P, I32, I32, U64, U32, U64, P]
    L.orc_backtrack.restype = I32
    L.orc_run_samples.argtypes = [I64, P, P, P, P, P, P, P, P, P, P, F64, P, U64, U32, U32, I64, I64,
                                  P, P, P, P, P, P, P, P, I64, P, P, P, ctypes.c_int]
    L.orc_bibfs.argtypes = [I64, P, P, P, P, I32, I32, U64, U32, U64, P, P, P, P, P]
    L.orc_bibfs.restype = I32
    L.orc_allpaths.argtypes = [I64, P, P, P, P, I32, I32, P, P]
    L.orc_allpaths.restype = I32
    L.orc_run_samples.restype = ctypes.c_int
    L.orc_cv_literal.argtypes = [I64, P, P]
    L.orc_cv_literal.restype = F64
    L.orc_cv_direct.argtypes = [I64, P, P]
    L.orc_cv_direct.restype = F64
    L.orc_cv_sorted.argtypes = [I64, P, P, P, F64, P]
    L.orc_exact_pc.argtypes = [I64, P, P, P, P, P, P, P]
    L.orc_vertex_diam_ub.argtypes = [I64, P, P, ctypes.c_int]
    L.orc_vertex_diam_ub.restype = I64
    L.orc_vjp_fixed.argtypes = [I64, P, F64, P, I64, I64, P, P, P, P, P, P, P, I64, P, P]
    L.orc_exact_vjp.argtypes = [I64, P, P, P, P, P, P, P, P, P]


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ------------------------------------------------------------------ Philox

def philox4x32_10(ctr, key) -> np.ndarray:
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def uniforms(seed: int, i: int, tag: int, j: int):
    out = np.zeros(2)
    lib().orc_uniforms(seed, i, tag, j, _p(out))
    return float(out[0]), float(out[1])


# ------------------------------------------------------------- graph views

@dataclass
class OGraph:
    """CSR plus in-adjacency (identical to the CSR for undirected graphs)."""
    n: int
    rp: np.ndarray
    col: np.ndarray
    irp: np.ndarray
    icol: np.ndarray
    directed: bool


def graph(n, row_ptr, col, directed) -> OGraph:
    rp = _c(row_ptr, np.int64)
    cl = _c(col, np.int32)
    if directed:
        irp = np.zeros(n + 1, dtype=np.int64)
        icol = np.zeros(cl.shape[0], dtype=np.int32)
        lib().orc_transpose(n, _p(rp), _p(cl), _p(irp), _p(icol))
    else:
        irp, icol = rp, cl
    return OGraph(n, rp, cl, irp, icol, bool(directed))


def from_synth(g) -> OGraph:
    return graph(g.n, g.row_ptr, g.col, g.directed)


# ------------------------------------------------------------ preparation

@dataclass
class Prep:
    n: int
    x: np.ndarray
    perm: np.ndarray
    xs: np.ndarray
    w: np.ndarray
    ci: np.ndarray
    r: np.ndarray
    c: float
    Cv: np.ndarray
    lam: np.ndarray
    dhat: float


def sort_states(x):
    x = _c(x, np.float64)
    n = x.shape[0]
    perm = np.zeros(n, dtype=np.int32)
    xs = np.zeros(n)
    lib().orc_sort_states(n, _p(x), _p(perm), _p(xs))
    return perm, xs


def tables(xs):
    n = xs.shape[0]
    w = np.zeros(n + 2)
    ci = np.zeros(n + 2)
    r = np.zeros(n + 2)
    c = lib().orc_tables(n, _p(_c(xs, np.float64)), _p(w), _p(ci), _p(r))
    return w, ci, r, c


def cv_literal(x):
    x = _c(x, np.float64)
    Cv = np.zeros(x.shape[0])
    C = lib().orc_cv_literal(x.shape[0], _p(x), _p(Cv))
    return C, Cv


def cv_direct(x):
    x = _c(x, np.float64)
    Cv = np.zeros(x.shape[0])
    C = lib().orc_cv_direct(x.shape[0], _p(x), _p(Cv))
    return C, Cv


def prepare(x, cv_method: str = "auto") -> Prep:
    """Sorted states, Algorithm 2 tables, C_v, lambda_v = C / C_v and
    d^ = max_v lambda_v (closed form of d_v, proof of Proposition 5)."""
    x = _c(x, np.float64)
    n = x.shape[0]
    perm, xs = sort_states(x)
    w, ci, r, c = tables(xs)
    if cv_method == "auto":
        cv_method = "direct" if n <= 3000 else "sorted"
    if cv_method == "direct":
        _, Cv = cv_direct(x)
    elif cv_method == "literal":
        _, Cv = cv_literal(x)
    else:
        Cv = np.zeros(n)
        lib().orc_cv_sorted(n, _p(xs), _p(perm), _p(w), c, _p(Cv))
    with np.errstate(divide="ignore"):
        lam = np.where(Cv > 0, c / np.where(Cv > 0, Cv, 1.0), np.inf)
    return Prep(n, x, perm, xs, w, ci, r, c, Cv, lam, float(lam.max()) if n else 0.0)


def sample_pairs(prep: Prep, seed: int, tag: int, i0: int, count: int):
    s = np.zeros(count, dtype=np.int32)
    t = np.zeros(count, dtype=np.int32)
    sp = np.zeros(count, dtype=np.int64)
    tp = np.zeros(count, dtype=np.int64)
    lib().orc_sample_pairs(prep.n, _p(prep.xs), _p(prep.perm), _p(prep.w), _p(prep.ci), _p(prep.r), prep.c,
                           seed, tag, i0, count, _p(s), _p(t), _p(sp), _p(tp))
    return s, t, sp, tp


def bfs(g: OGraph, s: int, t: int = -1):
    """Returns (ret, dist, sigma, order, edges_scanned, overflow)."""
    n = g.n
    dist = np.zeros(n, dtype=np.int32)
    sigma = np.zeros(n)
    order = np.zeros(n, dtype=np.int32)
    no = np.zeros(1, dtype=np.int64)
    edges = np.zeros(1, dtype=np.int64)
    ovf = np.zeros(1, dtype=np.int32)
    ret = lib().orc_bfs(n, _p(g.rp), _p(g.col), _p(g.irp), _p(g.icol), int(s), int(t), _p(dist), _p(sigma),
                        _p(order), _p(no), _p(edges), _p(ovf))
    return int(ret), dist, sigma, order[: int(no[0])], int(edges[0]), bool(ovf[0])


def backtrack(g: OGraph, dist, sigma, s, t, seed, tag, i):
    path = np.zeros(g.n + 1, dtype=np.int32)
    k = lib().orc_backtrack(_p(g.irp), _p(g.icol), _p(_c(dist, np.int32)), _p(_c(sigma, np.float64)), int(s),
                            int(t), seed, tag, i, _p(path))
    return int(k), path[: max(int(k), 0)]


@dataclass
class Phase:
    s: np.ndarray
    t: np.ndarray
    kind: np.ndarray
    ilen: np.ndarray
    cnt: np.ndarray
    acc: np.ndarray
    path_ptr: np.ndarray
    path_nodes: np.ndarray
    edges: np.ndarray
    overflow: bool
    acc_all: np.ndarray | None = None


def run_samples(g: OGraph, prep: Prep, seed: int, tag_pair: int, tag_path: int, i0: int, count: int,
                keep_paths: bool = True, path_cap: int | None = None, allpaths: bool = False,
                bidir: bool = False) -> Phase:
    """One sampling phase: Algorithm 2 pairs, RandomSP paths, estimator sums.
    bidir: RandomSP by the balanced bidirectional BFS (see bibfs); the
    edges then count what both sides scanned."""
    if bidir and allpaths:
        raise ValueError("the all-paths form uses the one-sided BFS")
    n = g.n
    s = np.zeros(count, dtype=np.int32)
    t = np.zeros(count, dtype=np.int32)
    kind = np.zeros(count, dtype=np.int32)
    ilen = np.zeros(count, dtype=np.int32)
    cnt = np.zeros(n, dtype=np.int64)
    acc = np.zeros(n)
    acc_all = np.zeros(n) if allpaths else None
    edges = np.zeros(count, dtype=np.int64)
    ovf = np.zeros(1, dtype=np.int32)
    if keep_paths:
        cap = path_cap if path_cap is not None else max(1, count * 64)
        while True:
            pp = np.zeros(count + 1, dtype=np.int64)
            pn = np.zeros(cap, dtype=np.int32)
            cnt[:] = 0
            acc[:] = 0
            if acc_all is not None:
                acc_all[:] = 0
            rc = lib().orc_run_samples(n, _p(g.rp), _p(g.col), _p(g.irp), _p(g.icol), _p(prep.x), _p(prep.xs),
                                       _p(prep.perm), _p(prep.w), _p(prep.ci), _p(prep.r), prep.c, _p(prep.Cv),
                                       seed, tag_pair, tag_path, i0, count, _p(s), _p(t), _p(kind), _p(ilen),
                                       _p(cnt), _p(acc), _p(pp), _p(pn), cap, _p(edges), _p(ovf), _p(acc_all),
                                       int(bidir))
            if rc == -1:
                cap = int(pp[-1]) + 1
                continue
            break
        pn = pn[: int(pp[-1])]
    else:
        pp = None
        pn = None
        rc = lib().orc_run_samples(n, _p(g.rp), _p(g.col), _p(g.irp), _p(g.icol), _p(prep.x), _p(prep.xs),
                                   _p(prep.perm), _p(prep.w), _p(prep.ci), _p(prep.r), prep.c, _p(prep.Cv),
                                   seed, tag_pair, tag_path, i0, count, _p(s), _p(t), _p(kind), _p(ilen),
                                   _p(cnt), _p(acc), None, None, 0, _p(edges), _p(ovf), _p(acc_all), int(bidir))
    if rc == -2:
        raise RuntimeError("oracle backtrack failed (sigma not exact?)")
    return Phase(s, t, kind, ilen, cnt, acc, pp, pn, edges, bool(ovf[0]), acc_all)


def bibfs(g: OGraph, s: int, t: int, seed: int, tag: int, i: int):
    """Balanced bidirectional RandomSP of sample i: (d(s,t) or -1, internal
    nodes, sigma_st, edges scanned)."""
    path = np.zeros(g.n + 1, dtype=np.int32)
    plen = np.zeros(1, dtype=np.int32)
    sst = np.zeros(1)
    edges = np.zeros(1, dtype=np.int64)
    ovf = np.zeros(1, dtype=np.int32)
    d = lib().orc_bibfs(g.n, _p(g.rp), _p(g.col), _p(g.irp), _p(g.icol), s, t, seed, tag, i, _p(path), _p(plen),
                        _p(sst), _p(edges), _p(ovf))
    if d == -2:
        raise RuntimeError("oracle bidirectional backtrack failed")
    return int(d), path[: int(plen[0])].copy(), float(sst[0]), int(edges[0])


def allpaths(g: OGraph, dist, sigma, s: int, t: int):
    """Internal nodes of all shortest s-t paths and f(v) = sigma_sv tau_v / sigma_st."""
    nodes = np.zeros(g.n, dtype=np.int32)
    frac = np.zeros(g.n)
    k = lib().orc_allpaths(g.n, _p(g.irp), _p(g.icol), _p(_c(dist, np.int32)), _p(_c(sigma, np.float64)), int(s),
                           int(t), _p(nodes), _p(frac))
    return nodes[:max(k, 0)], frac[:max(k, 0)]


def exact_pc(g: OGraph, x, Cv=None):
    x = _c(x, np.float64)
    if Cv is None:
        Cv = prepare(x).Cv
    pc = np.zeros(g.n)
    lib().orc_exact_pc(g.n, _p(g.rp), _p(g.col), _p(g.irp), _p(g.icol), _p(x), _p(_c(Cv, np.float64)), _p(pc))
    return pc


def vertex_diam_ub(g: OGraph) -> int:
    return int(lib().orc_vertex_diam_ub(g.n, _p(g.rp), _p(g.col), int(g.directed)))


def vjp_fixed(prep: Prep, ell: int, ph: Phase, F, gvec, us=None):
    n = prep.n
    us = np.arange(n, dtype=np.int64) if us is None else _c(us, np.int64)
    out = np.zeros(us.shape[0])
    lib().orc_vjp_fixed(n, _p(prep.x), prep.c, _p(prep.Cv), ell, ph.s.shape[0], _p(ph.s), _p(ph.t), _p(ph.kind),
                        _p(ph.path_ptr), _p(ph.path_nodes), _p(_c(F, np.float64)), _p(_c(gvec, np.float64)),
                        us.shape[0], _p(us), _p(out))
    return out


def exact_vjp(g: OGraph, x, gvec, Cv=None, pc=None):
    x = _c(x, np.float64)
    if Cv is None:
        Cv = prepare(x).Cv
    if pc is None:
        pc = exact_pc(g, x, Cv)
    out = np.zeros(g.n)
    lib().orc_exact_vjp(g.n, _p(g.rp), _p(g.col), _p(g.irp), _p(g.icol), _p(x), _p(_c(Cv, np.float64)),
                        _p(_c(pc, np.float64)), _p(_c(gvec, np.float64)), _p(out))
    return out


# ------------------------------------------------------- brute force (tiny)

def brute_force_pc(n, row_ptr, col, x):
    """Definition 1 written out for tiny graphs: enumerate every simple s-t
    path by DFS, keep the shortest ones (Gamma_st), count sigma_st(v), and use
    the literal double-sum denominator of kappa(s,t,v)."""
    adj = [list(col[row_ptr[u]:row_ptr[u + 1]]) for u in range(n)]
    R = lambda a: a if a > 0 else 0.0
    paths = {}

    def dfs(u, t, stack, onpath, out):
        if u == t:
            out.append(list(stack))
            return
        for v in adj[u]:
            if not onpath[v]:
                onpath[v] = True
                stack.append(v)
                dfs(v, t, stack, onpath, out)
                stack.pop()
                onpath[v] = False

    for s in range(n):
        for t in range(n):
            if s == t:
                continue
            out = []
            onpath = [False] * n
            onpath[s] = True
            dfs(s, t, [s], onpath, out)
            if out:
                L = min(len(p) for p in out)
                paths[(s, t)] = [p for p in out if len(p) == L]
    p = np.zeros(n)
    for v in range(n):
        den = sum(R(x[u] - x[w]) for u in range(n) for w in range(n) if u != v and w != v)
        tot = 0.0
        for (s, t), G in paths.items():
            if s == v or t == v:
                continue
            sig = len(G)
            sig_v = sum(1 for q in G if v in q[1:-1])
            if sig_v:
                tot += sig_v / sig * R(x[s] - x[t]) / den
        p[v] = tot
    return p, paths


# ---------------------------------------------------------------- bounds

def ell1_default(eps: float, delta: float) -> int:
    """Section III-B: l1 = max{10^3, ln(1/delta)/eps}."""
    return int(max(1000, math.ceil(math.log(1.0 / delta) / eps)))


def Lambda_literal(ilen) -> float:
    """Proposition 2: Lambda(S) = 1/(l(l-1)) sum_{i<j} (|I_i| - |I_j|)^2."""
    a = [int(v) for v in ilen]
    L = len(a)
    tot = 0
    for i in range(L):
        ai = a[i]
        for j in range(i + 1, L):
            d = ai - a[j]
            tot += d * d
    return tot / (L * (L - 1))


def Lambda_sums(ilen) -> float:
    """Proposition 2's Lambda(S) from two exact integer sums: the pairwise sum
    sum_{i<j} (a_i - a_j)^2 equals l sum a_i^2 - (sum a_i)^2, so the integer
    numerator is the same as Lambda_literal's and one division gives the same
    double."""
    a = [int(v) for v in ilen]
    L = len(a)
    S = sum(a)
    Q = sum(v * v for v in a)
    return (L * Q - S * S) / (L * (L - 1))


def rho_hat(ilen, D: int, delta: float) -> tuple[float, float, float]:
    """Algorithm 1: rho^ = rho~ + sqrt(2 Lambda log(8/delta)/l1) + 7 D log(8/delta)/(3(l1-1)),
    i.e. Proposition 2 (an empirical Bernstein bound on the mean of |I| in
    [0, D]) at confidence delta/4, as the proof of Proposition 4 applies it."""
    l1 = len(ilen)
    rt = float(np.sum(np.asarray(ilen, dtype=np.int64))) / l1
    Lam = Lambda_sums(ilen)
    lg = math.log(8.0 / delta)
    return rt + math.sqrt(2.0 * Lam * lg / l1) + 7.0 * D * lg / (3.0 * (l1 - 1)), rt, Lam


def v_hat(p1_max: float, dhat: float, l1: int, delta: float) -> float:
    """Algorithm 1: v^ = d^2 max_v {p~ + sqrt(2 p~ log(4/delta)/l1) + log(4/delta)/(3 l1)},
    i.e. Proposition 3 at confidence delta/4.  The braced expression increases
    with p~, so the max is at max_v p~(v)."""
    lg = math.log(4.0 / delta)
    return dhat * dhat * (p1_max + math.sqrt(2.0 * p1_max * lg / l1) + lg / (3.0 * l1))


def x_hat(vh: float, dhat: float) -> float:
    """Algorithm 1: x^ = d^/2 - sqrt(d^2/4 - min{d^2/4, v^})."""
    q = dhat * dhat / 4.0
    return dhat / 2.0 - math.sqrt(q - min(q, vh))


def ell_objective(x: float, eps: float, delta: float, dhat: float, rho_h: float) -> float:
    """Theorem 1 / Algorithm 1 objective with g(x) = x(d^-x), h(y) = (1+y)ln(1+y)-y."""
    gx = x * (dhat - x)
    y = eps * dhat / gx
    hy = (1.0 + y) * math.log(1.0 + y) - y
    return dhat * dhat * math.log(4.0 * dhat * rho_h / (x * delta)) / (gx * hy)


ELL_GRID = 4096
ELL_REFINE = 100


def ell_sup(eps: float, delta: float, dhat: float, rho_h: float, xh: float) -> tuple[int, float]:
    """l = sup over x in (0, x^] of the Theorem 1 objective.  Reading (the
    paper gives no method): maximum over x_k = x^ 10^(-12 + 12k/K),
    k = 0..K (K = 4096), then golden-section refinement on the bracket
    [x_{k*-1}, x_{k*+1}] of the best grid point; l = ceil(max)."""
    K = ELL_GRID
    best_k, best = 0, -math.inf
    for k in range(K + 1):
        xk = xh * math.pow(10.0, -12.0 + 12.0 * k / K)
        fv = ell_objective(xk, eps, delta, dhat, rho_h)
        if fv > best:
            best, best_k = fv, k
    lo = xh * math.pow(10.0, -12.0 + 12.0 * max(best_k - 1, 0) / K)
    hi = xh * math.pow(10.0, -12.0 + 12.0 * min(best_k + 1, K) / K)
    gr = (math.sqrt(5.0) - 1.0) / 2.0
    a, b = lo, hi
    c1 = b - gr * (b - a)
    c2 = a + gr * (b - a)
    f1 = ell_objective(c1, eps, delta, dhat, rho_h)
    f2 = ell_objective(c2, eps, delta, dhat, rho_h)
    for _ in range(ELL_REFINE):
        if f1 > best:
            best = f1
        if f2 > best:
            best = f2
        if f1 >= f2:
            b, c2, f2 = c2, c1, f1
            c1 = b - gr * (b - a)
            f1 = ell_objective(c1, eps, delta, dhat, rho_h)
        else:
            a, c1, f1 = c1, c2, f2
            c2 = a + gr * (b - a)
            f2 = ell_objective(c2, eps, delta, dhat, rho_h)
    best = max(best, f1, f2)
    return int(math.ceil(best)), best


# ------------------------------------------------------------- Algorithm 1

@dataclass
class Result:
    pc: np.ndarray
    pc_counts: np.ndarray
    cnt: np.ndarray
    ell1: int
    ell: int
    D: int
    dhat: float
    rho_tilde: float
    Lam: float
    rho_hat: float
    v_hat: float
    x_hat: float
    p1_max: float
    phase1: Phase
    phase2: Phase
    prep: Prep
    extra: dict = field(default_factory=dict)


def percis(g: OGraph, x, eps: float, delta: float, seed: int, ell1: int | None = None, ell: int | None = None,
           D: int | None = None, prep: Prep | None = None, keep_paths: bool = True, allpaths: bool = False,
           data_independent: bool = False, offsets: tuple[int, int] = (0, 0), bidir: bool = False) -> Result:
    """Algorithm 1 (PercIS): D, phase 1 (l1 samples, pair tag 0, path tag 2),
    rho^, v^, x^, l, then phase 2 (l fresh samples, pair tag 1, path tag 3).
    The phase-1 estimate uses 1/l1 (the 1/l printed in that line of
    Algorithm 1 is read as the phase-1 sample size).

    data_independent: PercIS-DI (Section V, sample-size experiment): no first
    phase; rho^ = D and v^ = d^2/4 (its largest possible value).

    offsets: index of the first sample of phase 1 and of phase 2 in the
    Philox counters (a graph of a batch whose samples follow other graphs')."""
    if prep is None:
        prep = prepare(x)
    if not np.all(prep.Cv > 0):
        raise ValueError("degenerate states: some C_v = 0 (p(v) undefined)")
    if D is None:
        D = vertex_diam_ub(g)
    if data_independent:
        l1, ph1, p1_max, rt, Lam = 0, None, 0.0, 0.0, 0.0
        rh, vh = float(D), prep.dhat * prep.dhat / 4.0
    else:
        l1 = ell1 if ell1 is not None else ell1_default(eps, delta)
        ph1 = run_samples(g, prep, seed, 0, 2, offsets[0], l1, keep_paths=False, allpaths=allpaths, bidir=bidir)
        p1 = (ph1.acc_all if allpaths else ph1.acc) / l1
        p1_max = float(p1.max())
        rh, rt, Lam = rho_hat(ph1.ilen, D, delta)
        vh = v_hat(p1_max, prep.dhat, l1, delta)
    xh = x_hat(vh, prep.dhat)
    if ell is None:
        ell, _ = ell_sup(eps, delta, prep.dhat, rh, xh)
    ph2 = run_samples(g, prep, seed, 1, 3, offsets[1], ell, keep_paths=keep_paths, allpaths=allpaths, bidir=bidir)
    pc = (ph2.acc_all if allpaths else ph2.acc) / ell
    pc_counts = prep.lam * ph2.cnt / ell
    return Result(pc, pc_counts, ph2.cnt, l1, ell, D, prep.dhat, rt, Lam, rh, vh, xh, p1_max, ph1, ph2, prep)


# ------------------------------------------------ finite differences of F

def fd_fixed(prep: Prep, ell: int, ph: Phase, gvec, u: int, h: float = 1e-6) -> float:
    """Central difference (L(x + h e_u) - L(x - h e_u)) / 2h of
    L = sum_v g_v F_v with F the fixed-sample estimator, evaluated in
    difference form: the changes of C, C_v and R_i caused by moving x_u are
    summed from the few terms that involve u, so no O(n^2)-sized quantity is
    subtracted from another."""
    x = prep.x
    n = prep.n
    gvec = np.asarray(gvec, dtype=np.float64)
    Cbar = prep.c
    Cv = prep.Cv

    def deltas(hh):
        xu_new = x[u] + hh
        others = np.delete(np.arange(n), u)
        # change of C: pairs (u, w) and (w, u), w != u
        dC = float(np.sum((np.maximum(0.0, xu_new - x[others]) - np.maximum(0.0, x[u] - x[others]))
                          + (np.maximum(0.0, x[others] - xu_new) - np.maximum(0.0, x[others] - x[u]))))
        # change of A_v = sum_w |x_v - x_w|
        dA = np.abs(x - xu_new) - np.abs(x - x[u])
        dA[u] = float(np.sum(np.abs(xu_new - x[others]) - np.abs(x[u] - x[others])))
        return dC - dA  # change of C_v for every v

    dCp = deltas(+h)
    dCm = deltas(-h)
    cnt = np.zeros(n)
    touched_p = np.zeros(n)
    touched_m = np.zeros(n)
    for i in range(ph.s.shape[0]):
        if ph.kind[i] != 0:
            continue
        s, t = int(ph.s[i]), int(ph.t[i])
        nodes = ph.path_nodes[ph.path_ptr[i]:ph.path_ptr[i + 1]]
        if s != u and t != u:
            cnt[nodes] += 1.0
            continue
        Rb = x[s] - x[t]
        dp = (h if s == u else -h)
        # R(x_s - x_t) moves by +-h exactly away from the kink (checked by caller)
        touched_p[nodes] += dp / Rb
        touched_m[nodes] += -dp / Rb
        cnt[nodes] += 1.0
    # F_v(x') - F_v(x'') with x' = x + h e_u, x'' = x - h e_u:
    # (Cbar/l) [ (cnt_v + tp_v)/(Cv+dCp) - (cnt_v + tm_v)/(Cv+dCm) ]
    a = Cv + dCp
    b = Cv + dCm
    diff = (cnt * (dCm - dCp) / (a * b) + touched_p / a - touched_m / b) * (Cbar / ell)
    return float(np.dot(gvec, diff) / (2.0 * h))
