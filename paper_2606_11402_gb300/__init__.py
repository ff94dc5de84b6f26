"""GB300 GraphGP: Vecchia approximation of a Gaussian process on 3-D points.

Thin Python binding of ``libgraphgp.so`` (C ABI in ``include/graphgp.h``):
argument marshalling only.  Every step of the method runs in the library's
CUDA kernels; there is no CPU or PyTorch fallback.  PyTorch provides device
memory (tensors) and streams.

Python names mirror the C entry points without the ``graphgp_`` prefix:
``build_graph``, ``graph_import``, ``factor``, ``generate``, ``whiten``,
``logdet``, ``nll`` and the ``*_backward`` adjoints.  Vectors are float32
CUDA tensors in graph order (the depth-sorted generation order, Sec. 2.2).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgraphgp.so")

MATERN12, MATERN32, MATERN52, SQEXP = 0, 1, 2, 3

OK = 0
ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NAN, ERR_IO = -1, -2, -3, -4, -5, -6
WARN_NOT_PD = 1


class GraphGPError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


class _Kernel(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("sigma2", ctypes.c_double), ("lengthscale", ctypes.c_double),
                ("nugget", ctypes.c_double), ("rescue_tol", ctypes.c_double)]


class _BuildOpts(ctypes.Structure):
    _fields_ = [("n0", ctypes.c_int32), ("split_rule", ctypes.c_int32),
                ("max_spin", ctypes.c_int64)]


@dataclass(frozen=True)
class Kernel:
    """Stationary covariance kappa(r) of Sec. 2.1 (Matern nu=1/2,3/2,5/2 or SE)."""
    type: int = MATERN32
    sigma2: float = 1.0
    lengthscale: float = 0.1
    nugget: float = 0.0
    # rows whose a-priori FP32 error estimate exceeds this are recomputed in
    # FP64 (0 = library default 2^-7, negative = every row in FP64)
    rescue_tol: float = 0.0

    def _c(self) -> _Kernel:
        return _Kernel(int(self.type), 0, float(self.sigma2), float(self.lengthscale),
                       float(self.nugget), float(self.rescue_tol))


_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int


def load() -> ctypes.CDLL:
    """Load libgraphgp.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                "(nvcc, sm_103a); the GraphGP path has no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "graphgp_build_graph": [_P, _I64, _I, _I, _P, _P, _P],
            "graphgp_graph_import": [_P, _I64, _I, _I, _P, _P, _P, _I, _P, _P],
            "graphgp_graph_info": [_P, _P, _P, _P, _P, _P],
            "graphgp_graph_export": [_P, _P, _P, _P, _P],
            "graphgp_graph_export_tree": [_P, _P, _P, _P, _P, _P, _P],
            "graphgp_graph_save": [_P, ctypes.c_char_p, _P],
            "graphgp_graph_load": [ctypes.c_char_p, _P, _P],
            "graphgp_factor": [_P, _P, _P, _P],
            "graphgp_factor_export": [_P, _P, _P, _P, _P],
            "graphgp_sync_status": [_P, _P, _P, _P],
            "graphgp_generate": [_P, _P, _P, _P, _P],
            "graphgp_whiten": [_P, _P, _P, _P, _P],
            "graphgp_logdet": [_P, _P, _P],
            "graphgp_nll": [_P, _P, _P, _P, _P],
            "graphgp_nll_noalloc": [_P, _P, _P, _P, _P],
            "graphgp_generate_backward": [_P, _P, _P, _P, _P, _P, _P, _P],
            "graphgp_whiten_backward": [_P, _P, _P, _P, _P, ctypes.c_double, _P, _P, _P],
            "graphgp_nll_backward": [_P, _P, _P, ctypes.c_double, _P, _P, _P],
            "graphgp_nll_backward_points": [_P, _P, _P, ctypes.c_double, _P, _P],
            "graphgp_selftest_wait_timeout": [_I64, _P],
            "graphgp_binary_version": [_P],
            "graphgp_factor_rows": [_P, _P, _I64, _I64, _P, _P],
            "graphgp_nll_rows": [_P, _P, _P, _P, _P],
            "graphgp_nll_backward_rows": [_P, _P, _P, ctypes.c_double, _P, _P, _P],
            "graphgp_generate_fused": [_P, _P, _P, _P, _P, _P],
            "graphgp_whiten_fused": [_P, _P, _P, _P, _P, _P, _P],
            "graphgp_nll_fused": [_P, _P, _P, _P, _P, _P],
            "graphgp_nll_grad_fused": [_P, _P, _P, ctypes.c_double, _P, _P, _P, _P, _P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        for name in ("graphgp_graph_destroy", "graphgp_factor_destroy"):
            f = getattr(L, name)
            f.argtypes = [_P]
            f.restype = None
        L.graphgp_status_string.argtypes = [_I]
        L.graphgp_status_string.restype = ctypes.c_char_p
        _lib = L
    return _lib


def lib() -> ctypes.CDLL:
    """The loaded library (alias of load())."""
    if _lib is None:
        load()
    return _lib


def status_string(status: int) -> str:
    return load().graphgp_status_string(status).decode()


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise GraphGPError(rc, what)
    return rc


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t: torch.Tensor, dtype, n=None, what="tensor") -> ctypes.c_void_p:
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{what}: expected a contiguous CUDA {dtype} tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{what}: expected {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


class Graph:
    """Owns a graphgp_graph_t (neighbour graph and depth levels in HBM)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle
        N, k, n0, nl, nb = _I64(), _I(), _I(), _I(), ctypes.c_size_t()
        _check(load().graphgp_graph_info(handle, ctypes.byref(N), ctypes.byref(k),
                                         ctypes.byref(n0), ctypes.byref(nl), ctypes.byref(nb)),
               "graph_info")
        self.N, self.k, self.n0, self.num_levels, self.bytes = N.value, k.value, n0.value, nl.value, nb.value

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.graphgp_graph_destroy(self._h)
            self._h = None

    def export(self, stream=None):
        """(order int32[N], nbr int32[N-n0, k], level_offsets int64[num_levels+1])."""
        dev = torch.device("cuda")
        order = torch.empty(self.N, dtype=torch.int32, device=dev)
        nbr = torch.empty((self.N - self.n0, self.k), dtype=torch.int32, device=dev)
        lo = (ctypes.c_int64 * (self.num_levels + 1))()
        _check(load().graphgp_graph_export(self._h, _dev(order, torch.int32), _dev(nbr, torch.int32),
                                           lo, _stream(stream)), "graph_export")
        return order, nbr, torch.tensor(list(lo), dtype=torch.int64)

    def export_tree(self, stream=None):
        """(tree_point, split_dim, inorder, depth, nbr_tree) indexed by tree index."""
        dev = torch.device("cuda")
        N = self.N
        tp = torch.empty(N, dtype=torch.int32, device=dev)
        sd = torch.empty(N, dtype=torch.uint8, device=dev)
        io = torch.empty(N, dtype=torch.int32, device=dev)
        dp = torch.empty(N, dtype=torch.int32, device=dev)
        nt = torch.empty((N - self.n0, self.k), dtype=torch.int32, device=dev)
        _check(load().graphgp_graph_export_tree(self._h, _dev(tp, torch.int32), _dev(sd, torch.uint8),
                                                _dev(io, torch.int32), _dev(dp, torch.int32),
                                                _dev(nt, torch.int32), _stream(stream)),
               "graph_export_tree")
        return tp, sd, io, dp, nt

    def save(self, path: str, stream=None):
        _check(load().graphgp_graph_save(self._h, path.encode(), _stream(stream)), "graph_save")


class Factor:
    """Owns a graphgp_factor_t (weights b, sigma, dense block) for one kernel."""

    def __init__(self, handle: ctypes.c_void_p, graph: Graph, kernel: Kernel):
        self._h = handle
        self.graph = graph  # keeps the graph alive
        self.kernel = kernel

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.graphgp_factor_destroy(self._h)
            self._h = None

    def export(self, stream=None):
        g = self.graph
        dev = torch.device("cuda")
        b = torch.empty((g.N - g.n0, g.k), dtype=torch.float32, device=dev)
        sigma = torch.empty(g.N, dtype=torch.float32, device=dev)
        L0 = torch.empty((g.n0, g.n0), dtype=torch.float32, device=dev)
        _check(load().graphgp_factor_export(self._h, _dev(b, torch.float32), _dev(sigma, torch.float32),
                                            _dev(L0, torch.float32), _stream(stream)), "factor_export")
        return b, sigma, L0


# --- entry points ------------------------------------------------------------
def build_graph(points: torch.Tensor, k: int, n0: int = 0, split_rule: int = 0,
                max_spin: int = 0, stream=None) -> Graph:
    """graphgp_build_graph: points float32[N, d], d in {1, 2, 3}, on the GPU
    (input order)."""
    if points.dim() != 2 or points.shape[1] not in (1, 2, 3):
        raise ValueError("points must be [N, d] with d in {1, 2, 3}")
    h = ctypes.c_void_p()
    opts = _BuildOpts(int(n0), int(split_rule), int(max_spin))
    _check(load().graphgp_build_graph(_dev(points, torch.float32), points.shape[0],
                                      points.shape[1], int(k),
                                      ctypes.byref(opts), _stream(stream), ctypes.byref(h)),
           "build_graph")
    return Graph(h)


def graph_import(points, k, n0, order, nbr, level_offsets, stream=None) -> Graph:
    """graphgp_graph_import from host (numpy) arrays already in graph order."""
    import numpy as np
    pts = np.ascontiguousarray(points, dtype=np.float32)
    order = np.ascontiguousarray(order, dtype=np.int32)
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    lo = np.ascontiguousarray(level_offsets, dtype=np.int64)
    h = ctypes.c_void_p()
    _check(load().graphgp_graph_import(pts.ctypes.data, pts.shape[0], int(k), int(n0),
                                       order.ctypes.data, nbr.ctypes.data, lo.ctypes.data,
                                       len(lo) - 1, _stream(stream), ctypes.byref(h)),
           "graph_import")
    return Graph(h)


def graph_load(path: str, stream=None) -> Graph:
    h = ctypes.c_void_p()
    _check(load().graphgp_graph_load(path.encode(), _stream(stream), ctypes.byref(h)), "graph_load")
    return Graph(h)


def factor(graph: Graph, kernel: Kernel, stream=None) -> Factor:
    h = ctypes.c_void_p()
    kc = kernel._c()
    _check(load().graphgp_factor(graph.handle, ctypes.byref(kc), _stream(stream), ctypes.byref(h)),
           "factor")
    return Factor(h, graph, kernel)


def factor_rows(graph: Graph, kernel: Kernel, pos_begin: int, pos_end: int, stream=None) -> Factor:
    """graphgp_factor_rows: the conditionals of positions [pos_begin, pos_end)."""
    h = ctypes.c_void_p()
    kc = kernel._c()
    _check(load().graphgp_factor_rows(graph.handle, ctypes.byref(kc), int(pos_begin),
                                      int(pos_end), _stream(stream), ctypes.byref(h)),
           "factor_rows")
    return Factor(h, graph, kernel)


def nll_rows(graph: Graph, fac: Factor, v: torch.Tensor, out: torch.Tensor | None = None,
             stream=None) -> torch.Tensor:
    """graphgp_nll_rows: the own positions' part of the NLL (float64[1])."""
    o = torch.empty(1, dtype=torch.float64, device="cuda") if out is None else out
    _check(load().graphgp_nll_rows(graph.handle, fac.handle, _dev(v, torch.float32, graph.N, "v"),
                                   _dev(o, torch.float64, 1, "out"), _stream(stream)), "nll_rows")
    return o


def nll_backward_rows(graph: Graph, fac: Factor, v: torch.Tensor, vbar: torch.Tensor,
                      thetabar: torch.Tensor, nllbar: float = 1.0, stream=None):
    """graphgp_nll_backward_rows: adds the own positions' gradient part to
    vbar (float32[N]) and thetabar (float64[3])."""
    _check(load().graphgp_nll_backward_rows(graph.handle, fac.handle,
                                            _dev(v, torch.float32, graph.N, "v"), float(nllbar),
                                            _dev(vbar, torch.float32, graph.N, "vbar"),
                                            _dev(thetabar, torch.float64, 3, "thetabar"),
                                            _stream(stream)), "nll_backward_rows")
    return vbar, thetabar


def sync_status(graph=None, fac=None, stream=None):
    """Synchronise and return (status, n_not_pd)."""
    n = ctypes.c_int64(0)
    rc = load().graphgp_sync_status(graph.handle if graph else None, fac.handle if fac else None,
                                    _stream(stream), ctypes.byref(n))
    _check(rc, "sync_status")
    return rc, n.value


def generate(graph: Graph, fac: Factor, xi: torch.Tensor, out: torch.Tensor | None = None,
             stream=None) -> torch.Tensor:
    v = torch.empty_like(xi) if out is None else out
    _check(load().graphgp_generate(graph.handle, fac.handle, _dev(xi, torch.float32, graph.N, "xi"),
                                   _dev(v, torch.float32, graph.N, "v"), _stream(stream)), "generate")
    return v


def whiten(graph: Graph, fac: Factor, v: torch.Tensor, out: torch.Tensor | None = None,
           stream=None) -> torch.Tensor:
    xi = torch.empty_like(v) if out is None else out
    _check(load().graphgp_whiten(graph.handle, fac.handle, _dev(v, torch.float32, graph.N, "v"),
                                 _dev(xi, torch.float32, graph.N, "xi"), _stream(stream)), "whiten")
    return xi


def logdet(fac: Factor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    o = torch.empty(1, dtype=torch.float64, device="cuda") if out is None else out
    _check(load().graphgp_logdet(fac.handle, _dev(o, torch.float64, 1), _stream(stream)), "logdet")
    return o


def nll(graph: Graph, fac: Factor, v: torch.Tensor, out: torch.Tensor | None = None,
        stream=None) -> torch.Tensor:
    o = torch.empty(1, dtype=torch.float64, device="cuda") if out is None else out
    _check(load().graphgp_nll(graph.handle, fac.handle, _dev(v, torch.float32, graph.N, "v"),
                              _dev(o, torch.float64, 1), _stream(stream)), "nll")
    return o


def _opt(t, dtype, n, what):
    return None if t is None else _dev(t, dtype, n, what)


def generate_fused(graph: Graph, kernel: Kernel, xi: torch.Tensor, out: torch.Tensor | None = None,
                   not_pd: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """graphgp_generate_fused: v = L xi with the factors recomputed in the pass
    (k <= 32); not_pd (int64[1], optional) has the floored pivots added."""
    v = torch.empty_like(xi) if out is None else out
    kc = kernel._c()
    _check(load().graphgp_generate_fused(graph.handle, ctypes.byref(kc),
                                         _dev(xi, torch.float32, graph.N, "xi"),
                                         _dev(v, torch.float32, graph.N, "v"),
                                         _opt(not_pd, torch.int64, 1, "not_pd"), _stream(stream)),
           "generate_fused")
    return v


def whiten_fused(graph: Graph, kernel: Kernel, v: torch.Tensor, out: torch.Tensor | None = None,
                 logdet: torch.Tensor | None = None, not_pd: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    """graphgp_whiten_fused: xi = L^-1 v with the factors recomputed in the
    pass; logdet (float64[1], optional) receives log det(L L^T)."""
    xi = torch.empty_like(v) if out is None else out
    kc = kernel._c()
    _check(load().graphgp_whiten_fused(graph.handle, ctypes.byref(kc),
                                       _dev(v, torch.float32, graph.N, "v"),
                                       _dev(xi, torch.float32, graph.N, "xi"),
                                       _opt(logdet, torch.float64, 1, "logdet"),
                                       _opt(not_pd, torch.int64, 1, "not_pd"), _stream(stream)),
           "whiten_fused")
    return xi


def nll_grad_fused(graph: Graph, kernel: Kernel, v: torch.Tensor, nllbar: float = 1.0,
                   out: torch.Tensor | None = None, vbar: torch.Tensor | None = None,
                   thetabar: torch.Tensor | None = None, not_pd: torch.Tensor | None = None,
                   stream=None):
    """graphgp_nll_grad_fused: (nll[1], vbar = nllbar dNLL/dv, thetabar[3] +=
    nllbar dNLL/dtheta) with the factors recomputed in one pass."""
    o = torch.empty(1, dtype=torch.float64, device="cuda") if out is None else out
    vb = torch.empty_like(v) if vbar is None else vbar
    tb = torch.zeros(3, dtype=torch.float64, device="cuda") if thetabar is None else thetabar
    kc = kernel._c()
    _check(load().graphgp_nll_grad_fused(graph.handle, ctypes.byref(kc),
                                         _dev(v, torch.float32, graph.N, "v"), float(nllbar),
                                         _dev(o, torch.float64, 1, "nll"),
                                         _dev(vb, torch.float32, graph.N, "vbar"),
                                         _dev(tb, torch.float64, 3, "thetabar"),
                                         _opt(not_pd, torch.int64, 1, "not_pd"), _stream(stream)),
           "nll_grad_fused")
    return o, vb, tb


def nll_fused(graph: Graph, kernel: Kernel, v: torch.Tensor, out: torch.Tensor | None = None,
              not_pd: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """graphgp_nll_fused: 0.5 xi.xi + 0.5 logdet without a stored factor."""
    o = torch.empty(1, dtype=torch.float64, device="cuda") if out is None else out
    kc = kernel._c()
    _check(load().graphgp_nll_fused(graph.handle, ctypes.byref(kc),
                                    _dev(v, torch.float32, graph.N, "v"),
                                    _dev(o, torch.float64, 1, "nll"),
                                    _opt(not_pd, torch.int64, 1, "not_pd"), _stream(stream)),
           "nll_fused")
    return o


def binary_version() -> int:
    """Compute capability (major * 10 + minor) of the loaded device code."""
    v = ctypes.c_int(0)
    _check(load().graphgp_binary_version(ctypes.byref(v)), "binary_version")
    return v.value


def selftest_wait_timeout(max_spin: int = 20000, stream=None) -> int:
    """Runs the bounded-wait self-test; returns its status (ERR_TIMEOUT when the
    device waits gave up as designed)."""
    return load().graphgp_selftest_wait_timeout(int(max_spin), _stream(stream))


def nll_noalloc(graph: Graph, fac: Factor, v: torch.Tensor, out: torch.Tensor,
                stream=None) -> torch.Tensor:
    """graphgp_nll_noalloc: nll() without any device allocation inside the
    call, for callers that cannot allocate (pass a preallocated `out`)."""
    _check(load().graphgp_nll_noalloc(graph.handle, fac.handle,
                                      _dev(v, torch.float32, graph.N, "v"),
                                      _dev(out, torch.float64, 1), _stream(stream)),
           "nll_noalloc")
    return out


def _theta_arg(thetabar, theta):
    """(tensor or None, pointer): thetabar to accumulate into, or NULL when
    the kernel-parameter gradient is not wanted."""
    if not theta:
        return None, None
    tb = torch.zeros(3, dtype=torch.float64, device="cuda") if thetabar is None else thetabar
    return tb, _dev(tb, torch.float64, 3, "thetabar")


def generate_backward(graph, fac, xi, v, vbar, xibar=None, thetabar=None, stream=None,
                      theta=True):
    """Returns (xibar, thetabar[3] += [dl, dsigma2, dnugget]); with
    theta=False the per-row factor backward is skipped and thetabar is None."""
    xb = torch.empty_like(xi) if xibar is None else xibar
    tb, tbp = _theta_arg(thetabar, theta)
    _check(load().graphgp_generate_backward(graph.handle, fac.handle,
                                            _dev(xi, torch.float32, graph.N, "xi"),
                                            _dev(v, torch.float32, graph.N, "v"),
                                            _dev(vbar, torch.float32, graph.N, "vbar"),
                                            _dev(xb, torch.float32, graph.N, "xibar"),
                                            tbp, _stream(stream)),
           "generate_backward")
    return xb, tb


def whiten_backward(graph, fac, v, xi, xibar, logdetbar=0.0, vbar=None, thetabar=None,
                    stream=None, theta=True):
    """Returns (vbar, thetabar[3] += ...); thetabar is None with theta=False."""
    vb = torch.empty_like(v) if vbar is None else vbar
    tb, tbp = _theta_arg(thetabar, theta)
    _check(load().graphgp_whiten_backward(graph.handle, fac.handle,
                                          _dev(v, torch.float32, graph.N, "v"),
                                          _dev(xi, torch.float32, graph.N, "xi"),
                                          _dev(xibar, torch.float32, graph.N, "xibar"),
                                          float(logdetbar),
                                          _dev(vb, torch.float32, graph.N, "vbar"),
                                          tbp, _stream(stream)),
           "whiten_backward")
    return vb, tb


def nll_backward(graph, fac, v, nllbar=1.0, vbar=None, thetabar=None, stream=None, theta=True):
    """(nllbar dNLL/dv, thetabar[3] += nllbar dNLL/dtheta); thetabar is None
    with theta=False."""
    vb = torch.empty_like(v) if vbar is None else vbar
    tb, tbp = _theta_arg(thetabar, theta)
    _check(load().graphgp_nll_backward(graph.handle, fac.handle,
                                       _dev(v, torch.float32, graph.N, "v"), float(nllbar),
                                       _dev(vb, torch.float32, graph.N, "vbar"),
                                       tbp, _stream(stream)),
           "nll_backward")
    return vb, tb


def nll_backward_points(graph, fac, v, nllbar=1.0, out=None, stream=None):
    """nllbar * dNLL/d(points) with the graph held fixed: float32[N, 3] in
    input order (the layout of the points given to build_graph)."""
    pb = torch.empty((graph.N, 3), dtype=torch.float32, device="cuda") if out is None else out
    _check(load().graphgp_nll_backward_points(graph.handle, fac.handle,
                                              _dev(v, torch.float32, graph.N, "v"), float(nllbar),
                                              _dev(pb, torch.float32, 3 * graph.N, "pbar"),
                                              _stream(stream)),
           "nll_backward_points")
    return pb
