"""Seeded synthetic graphs and percolation states.

This module only builds inputs: CSR adjacency (int64 row offsets, int32
column indices, rows sorted by neighbour id) and FP64 state vectors. It holds
none of the percolation-centrality arithmetic, so both the CUDA path and the
CPU oracle can be fed from it without sharing any of the method's code.

Graph families (all unweighted, simple):
  * Erdos-Renyi G(n, M): M distinct uniform edges, redrawn with sub-seeds
    0, 1, ... until connected.
  * Barabasi-Albert(n, m): an (m+1)-clique, then each new vertex links to m
    distinct existing vertices chosen proportionally to degree.
  * R-MAT(scale, edge_factor, a, b, c): directed, self-loops and duplicate
    edges removed, vertex ids randomly permuted.
  * Watts-Strogatz(n, k, p): ring lattice with k/2 neighbours per side, each
    lattice edge rewired with probability p.
  * 2D grid side x side, 4-neighbour, with a fraction of edges deleted.

States follow the settings the paper evaluates (Section IV-A): uniform
x ~ U[0,1], a seeded outbreak (a random fraction of vertices with
x ~ U[lo, hi], the rest 0), Beta(a, b), and binary random seeds.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Graph:
    n: int
    row_ptr: np.ndarray  # int64[n+1]
    col: np.ndarray  # int32[nnz]
    directed: bool
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])


def csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray, directed: bool, name: str = "") -> Graph:
    """CSR from an edge list; undirected edges are stored in both directions.

    Self-loops and duplicates are removed; each row is sorted by column id.
    """
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if not directed:
        src, dst = np.concatenate([src, dst]), np.concatenate([dst, src])
    keep = src != dst
    src, dst = src[keep], dst[keep]
    key = np.sort(src * n + dst)
    if key.size:
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    rows = key // n
    cols = (key % n).astype(np.int32)
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return Graph(n=n, row_ptr=row_ptr, col=cols, directed=directed, name=name)


def is_connected(g: Graph) -> bool:
    """Weak connectivity (scipy connected components on the CSR)."""
    if g.n == 0:
        return True
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    a = csr_matrix((np.ones(g.nnz, dtype=np.int8), g.col, g.row_ptr), shape=(g.n, g.n))
    ncomp, _ = connected_components(a, directed=True, connection="weak")
    return ncomp == 1


def erdos_renyi(n: int, avg_degree: float, seed: int) -> Graph:
    """Connected G(n, M) with M = n*avg_degree/2; sub-seed k is recorded in name."""
    m_edges = int(round(n * avg_degree / 2))
    for k in range(1000):
        rng = np.random.default_rng([seed, k])
        chosen = set()
        src, dst = [], []
        while len(chosen) < m_edges:
            need = m_edges - len(chosen)
            u = rng.integers(0, n, size=2 * need + 16)
            v = rng.integers(0, n, size=2 * need + 16)
            for a, b in zip(u.tolist(), v.tolist()):
                if a == b:
                    continue
                e = (a, b) if a < b else (b, a)
                if e in chosen:
                    continue
                chosen.add(e)
                src.append(e[0])
                dst.append(e[1])
                if len(chosen) == m_edges:
                    break
        g = csr_from_edges(n, np.array(src), np.array(dst), directed=False, name=f"er_n{n}_deg{avg_degree:g}_s{seed}_k{k}")
        if is_connected(g):
            return g
    raise RuntimeError("could not draw a connected G(n, M)")


def barabasi_albert(n: int, m: int, seed: int) -> Graph:
    rng = np.random.default_rng(seed)
    src, dst = [], []
    pool = np.empty(2 * (m * n + m * (m + 1)), dtype=np.int64)
    plen = 0
    for i in range(m + 1):
        for j in range(i + 1, m + 1):
            src.append(i)
            dst.append(j)
            pool[plen] = i
            pool[plen + 1] = j
            plen += 2
    draws = rng.random(size=int(1.5 * m * n) + 1024)
    di = 0
    for v in range(m + 1, n):
        chosen = []
        while len(chosen) < m:
            if di >= draws.shape[0]:
                draws = rng.random(size=int(0.5 * m * n) + 1024)
                di = 0
            k = int(pool[int(draws[di] * plen)])
            di += 1
            if k not in chosen:
                chosen.append(k)
        for k in chosen:
            src.append(v)
            dst.append(k)
            pool[plen] = v
            pool[plen + 1] = k
            plen += 2
    return csr_from_edges(n, np.array(src), np.array(dst), directed=False, name=f"ba_n{n}_m{m}_s{seed}")


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int,
         chunk: int = 1 << 22) -> Graph:
    n = 1 << scale
    n_edges = edge_factor * n
    rng = np.random.default_rng(seed)
    srcs, dsts = [], []
    # quadrant thresholds on 32-bit uniform integers (probabilities exact to 2^-32)
    ta, tab, tabc = (np.uint32(min(round(p * 2.0 ** 32), 2 ** 32 - 1)) for p in (a, a + b, a + b + c))
    done = 0
    while done < n_edges:
        cnt = min(chunk, n_edges - done)
        u = np.zeros(cnt, dtype=np.int64)
        v = np.zeros(cnt, dtype=np.int64)
        for bit in range(scale):
            r = rng.integers(0, 2 ** 32, size=cnt, dtype=np.uint32)
            ubit = r >= tab  # quadrants c, d
            vbit = ((r >= ta) & (r < tab)) | (r >= tabc)  # quadrants b, d
            u |= ubit.astype(np.int64) << bit
            v |= vbit.astype(np.int64) << bit
        srcs.append(u)
        dsts.append(v)
        done += cnt
    perm = rng.permutation(n)
    src = perm[np.concatenate(srcs)]
    dst = perm[np.concatenate(dsts)]
    return csr_from_edges(n, src, dst, directed=True, name=f"rmat_s{scale}_ef{edge_factor}_s{seed}")


def watts_strogatz(n: int, k: int, p: float, seed: int) -> Graph:
    rng = np.random.default_rng(seed)
    half = k // 2
    u = np.repeat(np.arange(n, dtype=np.int64), half)
    v = (u + np.tile(np.arange(1, half + 1, dtype=np.int64), n)) % n
    rewire = rng.random(u.shape[0]) < p
    new_v = rng.integers(0, n, size=u.shape[0])
    v = np.where(rewire, new_v, v)
    return csr_from_edges(n, u, v, directed=False, name=f"ws_n{n}_k{k}_p{p:g}_s{seed}")


def grid_2d(side: int, delete_frac: float, seed: int) -> Graph:
    rng = np.random.default_rng(seed)
    n = side * side
    idx = np.arange(n, dtype=np.int64).reshape(side, side)
    h = np.stack([idx[:, :-1].ravel(), idx[:, 1:].ravel()], axis=1)
    vv = np.stack([idx[:-1, :].ravel(), idx[1:, :].ravel()], axis=1)
    e = np.concatenate([h, vv])
    keep = rng.random(e.shape[0]) >= delete_frac
    e = e[keep]
    return csr_from_edges(n, e[:, 0], e[:, 1], directed=False, name=f"grid_{side}x{side}_del{delete_frac:g}_s{seed}")


def path_graph(n: int, directed: bool = False) -> Graph:
    s = np.arange(n - 1)
    return csr_from_edges(n, s, s + 1, directed=directed, name=f"path_{n}")


# ---------------------------------------------------------------- states

def states_uniform(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng([seed, 7]).random(n)


def states_outbreak(n: int, frac: float, lo: float, hi: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng([seed, 11])
    x = np.zeros(n)
    k = int(round(frac * n))
    chosen = rng.choice(n, size=k, replace=False)
    x[chosen] = lo + (hi - lo) * rng.random(k)
    return x


def states_beta(n: int, a: float, b: float, seed: int) -> np.ndarray:
    return np.random.default_rng([seed, 13]).beta(a, b, size=n)


def states_random_seeds(n: int, k: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng([seed, 17])
    x = np.zeros(n)
    x[rng.choice(n, size=min(k, n), replace=False)] = 1.0
    return x


def states_seeds_spread(g: Graph, seed: int, k: int | None = None) -> np.ndarray:
    """Random Seeds Spread (Section V-A): k = ceil(ln n) random seeds, and every vertex
    gets x_v = max over seeds s of 4^(-d(s, v)) (0 where no seed reaches v; distances
    along out-edges).  The paper writes "log n" seeds; the natural log is taken here."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import breadth_first_order

    rng = np.random.default_rng([seed, 19])
    n = g.n
    if k is None:
        k = max(1, int(math.ceil(math.log(n)))) if n > 1 else 1
    seeds = rng.choice(n, size=min(k, n), replace=False)
    a = csr_matrix((np.ones(g.nnz, dtype=np.int8), g.col, g.row_ptr), shape=(n, n))
    x = np.zeros(n)
    for s in seeds:
        order, pred = breadth_first_order(a, int(s), directed=True, return_predecessors=True)
        d = np.zeros(n, dtype=np.int64)
        for v in order[1:]:  # BFS order: a predecessor's distance is set before its children
            d[v] = d[pred[v]] + 1
        x[order] = np.maximum(x[order], 4.0 ** (-d[order].astype(np.float64)))
    return x


def isolated_component(g: Graph, seed: int, length: int = 50) -> tuple[Graph, np.ndarray]:
    """Isolated Component (Section V-A): a path P of `length` new vertices is added, both
    directions of each path edge (so P is strongly connected).  Undirected: P is its own
    component.  Directed: one edge from a random vertex of the largest strongly connected
    component of g to the first vertex of P.  Half of P's vertices (a seeded random half)
    get state 1, every other vertex 0."""
    rng = np.random.default_rng([seed, 23])
    n0, n = g.n, g.n + length
    rows = np.repeat(np.arange(n0, dtype=np.int64), np.diff(g.row_ptr))
    src = [rows, np.arange(n0, n - 1), np.arange(n0 + 1, n)]
    dst = [g.col.astype(np.int64), np.arange(n0 + 1, n), np.arange(n0, n - 1)]
    if g.directed:
        from scipy.sparse import csr_matrix
        from scipy.sparse.csgraph import connected_components

        a = csr_matrix((np.ones(g.nnz, dtype=np.int8), g.col, g.row_ptr), shape=(n0, n0))
        _, lab = connected_components(a, directed=True, connection="strong")
        big = np.flatnonzero(lab == np.bincount(lab).argmax())
        src.append(np.array([rng.choice(big)]))
        dst.append(np.array([n0]))
    else:  # undirected: csr_from_edges adds the reverse of every edge, the path's included
        src, dst = src[:2], dst[:2]
    h = csr_from_edges(n, np.concatenate(src), np.concatenate(dst), g.directed, name=f"{g.name}+ic{length}")
    x = np.zeros(n)
    x[n0 + rng.choice(length, size=length // 2, replace=False)] = 1.0
    return h, x


# ---------------------------------------------------------------- named workloads

def workload(name: str, seed: int = 0):
    """Named synthetic workloads: returns (graph, states, eps, delta)."""
    if name == "er1000":
        g = erdos_renyi(1000, 8.0, seed)
        return g, states_uniform(g.n, seed), 0.05, 0.1
    if name == "ba100k_outbreak":
        g = barabasi_albert(100_000, 5, seed)
        return g, states_outbreak(g.n, 0.10, 0.5, 1.0, seed), 0.005, 0.1
    if name == "rmat22_beta":
        g = rmat(22, 16, 0.57, 0.19, 0.19, seed)
        return g, states_beta(g.n, 0.5, 2.0, seed), 0.01, 0.1
    if name == "rmat20_beta":
        g = rmat(20, 16, 0.57, 0.19, 0.19, seed)
        return g, states_beta(g.n, 0.5, 2.0, seed), 0.01, 0.1
    if name == "ba200k_uniform":
        g = barabasi_albert(200_000, 4, seed)
        return g, states_uniform(g.n, seed), 0.01, 0.1
    if name == "ba2000_uniform":
        g = barabasi_albert(2000, 4, seed)
        return g, states_uniform(g.n, seed), 0.01, 0.1
    raise KeyError(name)


def graph_batch(sizes, seed: int) -> list[Graph]:
    """Independent graphs of the given vertex counts, the type taken in turn:
    Watts-Strogatz (k=10, p=0.05), Barabasi-Albert (m=3), square grid with 5%
    of its edges deleted (side round(sqrt(n)), so its size is close to n)."""
    out = []
    for g, n in enumerate(sizes):
        n = int(n)
        sub = seed * 100_003 + g
        if g % 3 == 0:
            out.append(watts_strogatz(n, 10, 0.05, sub))
        elif g % 3 == 1:
            out.append(barabasi_albert(n, 3, sub))
        else:
            out.append(grid_2d(max(2, int(round(math.sqrt(n)))), 0.05, sub))
    return out


def union_csr(graphs) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Block-diagonal CSR of independent graphs: (graph_vptr, row_ptr, col)."""
    vptr = np.zeros(len(graphs) + 1, dtype=np.int64)
    vptr[1:] = np.cumsum([g.n for g in graphs])
    eptr = np.zeros(len(graphs) + 1, dtype=np.int64)
    eptr[1:] = np.cumsum([g.nnz for g in graphs])
    row_ptr = np.zeros(int(vptr[-1]) + 1, dtype=np.int64)
    col = np.zeros(int(eptr[-1]), dtype=np.int32)
    for k, g in enumerate(graphs):
        row_ptr[vptr[k]:vptr[k + 1] + 1] = g.row_ptr + eptr[k]
        col[eptr[k]:eptr[k + 1]] = g.col + np.int32(vptr[k])
    return vptr, row_ptr, col


def uneven_batch_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Vertex counts log-uniform in [lo, hi]."""
    rng = np.random.default_rng([seed, 19])
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=count)).astype(np.int64)
