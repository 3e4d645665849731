"""ctypes binding of libpercis (include/percis.h).

Argument marshalling only: every computation happens in the CUDA library.
The functions below carry the C names; `PercIS` wraps a context for torch
tensors (device memory and the current stream come from torch), and
`PercISFunction` exposes dPC/dx through torch.autograd.

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_2509_11454_gb300.build_lib``); loading fails loudly
otherwise -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpercis.so")

PERCIS_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "DEGENERATE", 3: "OOM", 4: "CUDA", 5: "TIMEOUT", 6: "TOO_LARGE",
                7: "NO_SAMPLE", 8: "STATE"}
FORM_BATCHED = 0
FORM_PLAIN = 1
FORM_BIDIR = 2


class PercisError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"percis {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class percis_options(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int32), ("lanes", ctypes.c_int32), ("ell1", ctypes.c_int64),
                ("ell", ctypes.c_int64), ("vertex_diam", ctypes.c_int64), ("keep_paths", ctypes.c_int32),
                ("data_independent", ctypes.c_int32), ("timeout_s", ctypes.c_double),
                ("instrument", ctypes.c_int32), ("lane_order", ctypes.c_int32),
                ("direction", ctypes.c_int32), ("estimator", ctypes.c_int32), ("push_alpha", ctypes.c_double),
                ("cuda_graphs", ctypes.c_int32), ("bi_table_log", ctypes.c_int32),
                ("bi_table_max_log", ctypes.c_int32), ("bi_scratch_gib", ctypes.c_int32),
                ("bi_blocks_per_sm", ctypes.c_int32), ("tune_form", ctypes.c_int32),
                ("bi_heavy_edges", ctypes.c_int64), ("reserved", ctypes.c_int64)]


class percis_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("ell1", ctypes.c_int64), ("ell", ctypes.c_int64),
                ("vertex_diam", ctypes.c_int64), ("C", ctypes.c_double), ("dhat", ctypes.c_double),
                ("rho_tilde", ctypes.c_double), ("Lambda", ctypes.c_double), ("rho_hat", ctypes.c_double),
                ("v_hat", ctypes.c_double), ("x_hat", ctypes.c_double), ("p1_max", ctypes.c_double),
                ("zero_weight", ctypes.c_int64 * 2), ("unreachable", ctypes.c_int64 * 2),
                ("sum_internal", ctypes.c_int64 * 2), ("sources", ctypes.c_int64 * 2),
                ("batches", ctypes.c_int64 * 2), ("sigma_overflow", ctypes.c_int32), ("lanes", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int64), ("bfs_ms", ctypes.c_double * 2),
                ("bfs_launches", ctypes.c_int64 * 2), ("work", (ctypes.c_int64 * 8) * 2)]

    def as_dict(self) -> dict:
        def conv(v):
            if isinstance(v, ctypes.Array):
                return [conv(e) for e in v]
            return v
        return {name: conv(getattr(self, name)) for name, _ in self._fields_}


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_U32 = ctypes.c_uint32
_U64 = ctypes.c_uint64
_F64 = ctypes.c_double
_ST = ctypes.c_int

# name -> (restype, argtypes); mirrors include/percis.h
SIGNATURES = {
    "percis_create": (_ST, [ctypes.POINTER(_P), ctypes.c_int, _P]),
    "percis_destroy": (None, [_P]),
    "percis_set_stream": (_ST, [_P, _P]),
    "percis_last_error": (ctypes.c_char_p, [_P]),
    "percis_launch_count": (_I64, [_P]),
    "percis_default_options": (None, [ctypes.POINTER(percis_options)]),
    "percis_set_options": (_ST, [_P, ctypes.POINTER(percis_options)]),
    "percis_load_csr": (_ST, [_P, _I64, _I64, _P, _P, ctypes.c_int, ctypes.c_int]),
    "percis_set_states": (_ST, [_P, _P, ctypes.c_int]),
    "percis_estimate": (_ST, [_P, _F64, _F64, _U64, _P, ctypes.c_int, ctypes.POINTER(percis_info)]),
    "percis_exact_small": (_ST, [_P, _P, ctypes.c_int]),
    "percis_backward": (_ST, [_P, _P, _P, ctypes.c_int]),
    "percis_get_prep": (_ST, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "percis_sample_pairs": (_ST, [_P, _U64, _U32, _I64, _I64, _P, _P]),
    "percis_bfs": (_ST, [_P, _I32, _I32, _P, _P, _P]),
    "percis_msbfs": (_ST, [_P, _I32, _P, _P, _P]),
    "percis_run_phase": (_ST, [_P, _U64, ctypes.c_int, _I64, _P, _P, _P, _P, _P]),
    "percis_get_paths": (_ST, [_P, _P, _P, _P]),
    "percis_last_levels": (_I64, [_P, _P, _I64]),
    "percis_sample_trace": (_I64, [_P, _P, _I64]),
    "percis_autotune": (_ST, [_P, _I64, _U64, ctypes.POINTER(percis_options)]),
    "percis_load_graphs": (_ST, [_P, _I32, _P, _I64, _I64, _P, _P, ctypes.c_int]),
    "percis_num_graphs": (_I32, [_P]),
    "percis_estimate_graphs": (_ST, [_P, _F64, _F64, _U64, _P, ctypes.c_int, _P]),
    "percis_bfs_noalloc": (_ST, [_I64, _P, _P, _P, _P, _I32, _I32, _P, _P, _P, _F64, _P]),
}

_lib = None
_lock = threading.Lock()


def load_library() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build(); "
                                   "there is no CPU fallback")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
        return _lib


def _ptr(a) -> int | None:
    """Address of a torch tensor or numpy array (None passes through)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _on_device(a) -> int:
    return 0 if isinstance(a, np.ndarray) else int(a.is_cuda)


def _check(ctx, st: int):
    if st != PERCIS_OK:
        msg = load_library().percis_last_error(ctx)
        raise PercisError(st, msg.decode() if msg else "")


# ------------------------------------------------- C-named thin wrappers

def percis_create(device: int = 0, stream: int | None = None):
    h = _P()
    st = load_library().percis_create(ctypes.byref(h), device, stream)
    if st != PERCIS_OK:
        raise PercisError(st, "percis_create failed")
    return h


def percis_destroy(ctx):
    load_library().percis_destroy(ctx)


def percis_set_stream(ctx, stream: int):
    _check(ctx, load_library().percis_set_stream(ctx, stream))


def percis_last_error(ctx) -> str:
    m = load_library().percis_last_error(ctx)
    return m.decode() if m else ""


def percis_launch_count(ctx) -> int:
    return int(load_library().percis_launch_count(ctx))


def percis_default_options() -> percis_options:
    o = percis_options()
    load_library().percis_default_options(ctypes.byref(o))
    return o


def percis_set_options(ctx, opt: percis_options):
    _check(ctx, load_library().percis_set_options(ctx, ctypes.byref(opt)))


def percis_load_csr(ctx, n: int, nnz: int, row_ptr, col, directed: bool, on_device: int | None = None):
    od = _on_device(row_ptr) if on_device is None else on_device
    _check(ctx, load_library().percis_load_csr(ctx, n, nnz, _ptr(row_ptr), _ptr(col), int(directed), od))


def percis_set_states(ctx, x, on_device: int | None = None):
    od = _on_device(x) if on_device is None else on_device
    _check(ctx, load_library().percis_set_states(ctx, _ptr(x), od))


def percis_estimate(ctx, eps: float, delta: float, seed: int, pc_out, pc_on_device: int | None = None) -> dict:
    info = percis_info()
    od = _on_device(pc_out) if pc_on_device is None else pc_on_device
    _check(ctx, load_library().percis_estimate(ctx, eps, delta, seed, _ptr(pc_out), od, ctypes.byref(info)))
    return info.as_dict()


def percis_exact_small(ctx, pc_out, on_device: int | None = None):
    od = _on_device(pc_out) if on_device is None else on_device
    _check(ctx, load_library().percis_exact_small(ctx, _ptr(pc_out), od))


def percis_backward(ctx, grad_pc, grad_x, on_device: int | None = None):
    od = _on_device(grad_pc) if on_device is None else on_device
    _check(ctx, load_library().percis_backward(ctx, _ptr(grad_pc), _ptr(grad_x), od))


def percis_get_prep(ctx, perm=None, xs=None, w=None, ci=None, r=None, Cv=None, lam=None) -> dict:
    c = ctypes.c_double()
    dh = ctypes.c_double()
    D = ctypes.c_int64()
    _check(ctx, load_library().percis_get_prep(ctx, _ptr(perm), _ptr(xs), _ptr(w), _ptr(ci), _ptr(r), _ptr(Cv),
                                               _ptr(lam), ctypes.byref(c), ctypes.byref(dh), ctypes.byref(D)))
    return {"c": c.value, "dhat": dh.value, "vertex_diam": D.value}


def percis_sample_pairs(ctx, seed: int, tag: int, i0: int, count: int, s, t):
    _check(ctx, load_library().percis_sample_pairs(ctx, seed, tag, i0, count, _ptr(s), _ptr(t)))


def percis_bfs(ctx, source: int, target: int, dist, sigma) -> bool:
    """Single-source sigma BFS into device tensors; returns True when a path
    count reached 2^53 (sigma rounded there)."""
    ovf = ctypes.c_int32(0)
    _check(ctx, load_library().percis_bfs(ctx, source, target, _ptr(dist), _ptr(sigma), ctypes.byref(ovf)))
    return bool(ovf.value)


def percis_msbfs(ctx, nsrc: int, sources, dist, sigma):
    _check(ctx, load_library().percis_msbfs(ctx, nsrc, _ptr(sources), _ptr(dist), _ptr(sigma)))


def percis_run_phase(ctx, seed: int, phase: int, count: int, s=None, t=None, kind=None, ilen=None, cnt=None):
    _check(ctx, load_library().percis_run_phase(ctx, seed, phase, count, _ptr(s), _ptr(t), _ptr(kind), _ptr(ilen),
                                                _ptr(cnt)))


def percis_get_paths(ctx, path_ptr=None, path_nodes=None) -> int:
    tot = ctypes.c_int64()
    _check(ctx, load_library().percis_get_paths(ctx, _ptr(path_ptr), _ptr(path_nodes), ctypes.byref(tot)))
    return tot.value


def percis_bfs_noalloc(n: int, row_ptr, col, in_row_ptr, in_col, source: int, target: int, dist, sigma,
                       stream: int | None = None, timeout_s: float = 0.0, overflow: list | None = None) -> int:
    """Allocation-free single-source sigma BFS (device tensors); returns the
    status code.  If `overflow` is a list, the sigma-overflow flag (0/1) is
    appended to it."""
    ovf = ctypes.c_int32(0)
    st = int(load_library().percis_bfs_noalloc(n, _ptr(row_ptr), _ptr(col), _ptr(in_row_ptr), _ptr(in_col),
                                               source, target, _ptr(dist), _ptr(sigma), stream, float(timeout_s),
                                               ctypes.byref(ovf)))
    if overflow is not None:
        overflow.append(int(ovf.value))
    return st


def percis_load_graphs(ctx, graph_vptr, row_ptr, col, directed: bool = False):
    vp = np.ascontiguousarray(graph_vptr, dtype=np.int64)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    _check(ctx, load_library().percis_load_graphs(ctx, int(vp.shape[0]) - 1, _ptr(vp), int(rp.shape[0]) - 1,
                                                  int(cl.shape[0]), _ptr(rp), _ptr(cl), int(directed)))


def percis_num_graphs(ctx) -> int:
    return int(load_library().percis_num_graphs(ctx))


def percis_estimate_graphs(ctx, eps: float, delta: float, seed: int, pc_out,
                           pc_on_device: int | None = None) -> list[dict]:
    G = percis_num_graphs(ctx)
    infos = (percis_info * max(G, 1))()
    od = _on_device(pc_out) if pc_on_device is None else pc_on_device
    _check(ctx, load_library().percis_estimate_graphs(ctx, eps, delta, seed, _ptr(pc_out), od,
                                                      ctypes.cast(infos, ctypes.c_void_p)))
    return [infos[g].as_dict() for g in range(G)]


def percis_autotune(ctx, probe_samples: int, seed: int) -> percis_options:
    o = percis_options()
    _check(ctx, load_library().percis_autotune(ctx, probe_samples, seed, ctypes.byref(o)))
    return o


def percis_sample_trace(ctx, cap: int) -> np.ndarray:
    """Per-sample trace of the last bidirectional phase (instrument = 2):
    rows {start ns, end ns, edges, levels | store << 32 | block << 33 | heavy << 63,
    levels end ns, meeting choice end ns, failed walk step, failed walk vertex}."""
    out = np.zeros((max(cap, 1), 8), dtype=np.int64)
    k = int(load_library().percis_sample_trace(ctx, out.ctypes.data, cap))
    return out[:k]


def percis_last_levels(ctx, cap: int = 32) -> list[tuple[int, ...]]:
    out = np.zeros(6 * cap, dtype=np.int64)
    k = int(load_library().percis_last_levels(ctx, out.ctypes.data, cap))
    return [tuple(int(v) for v in out[6 * i:6 * i + 6]) for i in range(k)]


# ------------------------------------------------------ torch-facing engine

class PercIS:
    """One library context bound to a CUDA device and torch's current stream."""

    def __init__(self, device: int = 0, **options):
        import torch

        self.torch = torch
        self.device = torch.device("cuda", device)
        stream = torch.cuda.current_stream(self.device).cuda_stream
        self.ctx = percis_create(device, stream)
        self.n = 0
        self.options = percis_default_options()
        if options:
            self.set_options(**options)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            percis_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, **kw):
        for k, v in kw.items():
            if k == "form" and isinstance(v, str):
                v = {"batched": FORM_BATCHED, "plain": FORM_PLAIN, "bidir": FORM_BIDIR}[v]
            if k == "estimator" and isinstance(v, str):
                v = {"path": 0, "allpaths": 1}[v]
            setattr(self.options, k, v)
        percis_set_options(self.ctx, self.options)

    def autotune(self, probe_samples: int = 8192, seed: int = 0) -> dict:
        """Pick the speed options of the form (batched: lane width, lane order,
        direction rule; bidirectional: heavy-level threshold, store, blocks per
        SM; with tune_form=1 also the form) by timing probe phases; returns the
        chosen options."""
        o = percis_autotune(self.ctx, probe_samples, seed)
        self.options = o
        return {name: getattr(o, name) for name, _ in o._fields_}

    def _sync_stream(self):
        percis_set_stream(self.ctx, self.torch.cuda.current_stream(self.device).cuda_stream)

    def load_csr(self, row_ptr, col, directed: bool = False):
        t = self.torch
        rp = row_ptr if isinstance(row_ptr, np.ndarray) else row_ptr.to(t.int64).contiguous()
        cl = col if isinstance(col, np.ndarray) else col.to(t.int32).contiguous()
        if isinstance(rp, np.ndarray):
            rp = np.ascontiguousarray(rp, dtype=np.int64)
            cl = np.ascontiguousarray(cl, dtype=np.int32)
        n = int(rp.shape[0]) - 1
        percis_load_csr(self.ctx, n, int(cl.shape[0]), rp, cl, directed)
        self.n = n

    def set_states(self, x):
        if isinstance(x, np.ndarray):
            x = np.ascontiguousarray(x, dtype=np.float64)
        else:
            x = x.detach().to(self.torch.float64).contiguous()
        percis_set_states(self.ctx, x)

    def estimate(self, eps: float, delta: float, seed: int = 0, out=None):
        t = self.torch
        if out is None:
            out = t.empty(self.n, dtype=t.float64, device=self.device)
        info = percis_estimate(self.ctx, eps, delta, seed, out)
        return out, info

    def load_graphs(self, graph_vptr, row_ptr, col, directed: bool = False):
        """Many independent graphs as one block-diagonal CSR (host arrays)."""
        percis_load_graphs(self.ctx, graph_vptr, row_ptr, col, directed)
        self.n = int(np.asarray(row_ptr).shape[0]) - 1

    def estimate_graphs(self, eps: float, delta: float, seed: int = 0, out=None):
        t = self.torch
        if out is None:
            out = t.empty(self.n, dtype=t.float64, device=self.device)
        return out, percis_estimate_graphs(self.ctx, eps, delta, seed, out)

    def exact(self):
        t = self.torch
        out = t.empty(self.n, dtype=t.float64, device=self.device)
        percis_exact_small(self.ctx, out)
        return out

    def backward(self, grad_pc):
        t = self.torch
        g = grad_pc.detach().to(device=self.device, dtype=t.float64).contiguous()
        out = t.empty(self.n, dtype=t.float64, device=self.device)
        percis_backward(self.ctx, g, out)
        return out

    def prep(self):
        t = self.torch
        n = self.n
        d = dict(perm=t.empty(n, dtype=t.int32, device=self.device), xs=t.empty(n, dtype=t.float64, device=self.device),
                 w=t.empty(n + 2, dtype=t.float64, device=self.device),
                 ci=t.empty(n + 2, dtype=t.float64, device=self.device),
                 r=t.empty(n + 2, dtype=t.float64, device=self.device),
                 Cv=t.empty(n, dtype=t.float64, device=self.device), lam=t.empty(n, dtype=t.float64, device=self.device))
        sc = percis_get_prep(self.ctx, **d)
        d.update(sc)
        return d

    def sample_pairs(self, seed: int, tag: int, i0: int, count: int):
        t = self.torch
        s = t.empty(count, dtype=t.int32, device=self.device)
        tt = t.empty(count, dtype=t.int32, device=self.device)
        percis_sample_pairs(self.ctx, seed, tag, i0, count, s, tt)
        return s, tt

    def bfs(self, source: int, target: int = -1):
        t = self.torch
        dist = t.empty(self.n, dtype=t.int32, device=self.device)
        sig = t.empty(self.n, dtype=t.float64, device=self.device)
        percis_bfs(self.ctx, source, target, dist, sig)
        return dist, sig

    def msbfs(self, sources):
        t = self.torch
        src = t.as_tensor(np.asarray(sources, dtype=np.int32), device=self.device)
        k = int(src.shape[0])
        dist = t.empty(k * self.n, dtype=t.int32, device=self.device)
        sig = t.empty(k * self.n, dtype=t.float64, device=self.device)
        percis_msbfs(self.ctx, k, src, dist, sig)
        return dist.view(k, self.n), sig.view(k, self.n)

    def run_phase(self, seed: int, phase: int, count: int):
        t = self.torch
        d = dict(s=t.empty(count, dtype=t.int32, device=self.device), t=t.empty(count, dtype=t.int32, device=self.device),
                 kind=t.empty(count, dtype=t.int32, device=self.device),
                 ilen=t.empty(count, dtype=t.int32, device=self.device),
                 cnt=t.empty(self.n, dtype=t.int64, device=self.device))
        percis_run_phase(self.ctx, seed, phase, count, **d)
        return d

    def get_paths(self, count: int):
        t = self.torch
        total = percis_get_paths(self.ctx)
        ptr = t.empty(count + 1, dtype=t.int64, device=self.device)
        nodes = t.empty(max(total, 1), dtype=t.int32, device=self.device)
        percis_get_paths(self.ctx, ptr, nodes)
        return ptr, nodes[:total]


def _autograd():
    import torch

    class PercISFunction(torch.autograd.Function):
        """pc = PercIS estimate of x; backward = percis_backward (the VJP of the
        fixed-sample estimator).  The engine keeps only its last sample, so call
        backward before the next forward on the same engine."""

        @staticmethod
        def forward(ctx, x, engine, eps, delta, seed):
            engine.set_states(x)
            pc, info = engine.estimate(eps, delta, seed)
            ctx.engine = engine
            ctx.info = info
            return pc

        @staticmethod
        def backward(ctx, g):
            return ctx.engine.backward(g), None, None, None, None

    return PercISFunction


_fn = None


def percolation_centrality(x, engine: PercIS, eps: float, delta: float, seed: int = 0):
    """Differentiable PercIS estimate of the percolation centrality of every node."""
    global _fn
    if _fn is None:
        _fn = _autograd()
    return _fn.apply(x, engine, eps, delta, seed)
