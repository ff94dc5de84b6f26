"""FP64 CPU oracle for the GraphGP Vecchia hot path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this package.  It shares no code with the CUDA
library (``paper_2606_11402_gb300``) and neither imports the other; the two
meet only on the seeded inputs of the ``workloads`` module.

The arithmetic lives in ``graphgp_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module marshals numpy arrays through ctypes and
composes the steps in the paper's order:

* tree build and bit-reversed layout -- Sec. 2.2 "Tree ordering",
  "Bit-reversed ordering";
* preceding k-nearest neighbours -- Sec. 2.1, Sec. 2.2;
* depth and depth-sorted order -- Sec. 2.2 "Batch construction";
* factor -- Sec. 2.1 Eq. 2 (dense block: the dense initial batch of Alg. 1);
* generate / whiten / logdet -- Alg. 1 and Sec. 3;
* adjoints -- Sec. 2.3 (derivatives of the conditioning steps).

Parity pins: every function here is checked in ``tests/test_oracle_*.py``
against closed forms, brute force and textbook routines (never against the
CUDA path).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from collections import namedtuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

MATERN12, MATERN32, MATERN52, SQEXP = 0, 1, 2, 3
Kernel = namedtuple("Kernel", "type sigma2 lengthscale nugget")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no CUDA).  Returns the library path."""
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
             "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_D = ctypes.c_double


def _declare(L):
    sig = {
        "oracle_level": (_I, [_I64]),
        "oracle_left": (_I64, [_I64]),
        "oracle_right": (_I64, [_I64]),
        "oracle_parent": (_I64, [_I64]),
        "oracle_subtree_size": (_I64, [_I64, _I64]),
        "oracle_canonicalise": (_I64, [_P, _I64]),
        "oracle_tree_build": (_I, [_P, _I64, _I, _P, _P, _P]),
        "oracle_d2": (ctypes.c_float, [_P, _P]),
        "oracle_knn_brute": (_I, [_P, _P, _I64, _I, _I64, _P]),
        "oracle_knn_tree": (_I, [_P, _P, _P, _I64, _I, _I64, _P]),
        "oracle_knn_brute_some": (_I, [_P, _P, _P, _I64, _I, _P]),
        "oracle_factor_rows": (_I, [_P, _P, _P, _I64, _I, _I, _D, _D, _D, _P, _P]),
        "oracle_depth": (_I, [_P, _I64, _I, _I64, _P]),
        "oracle_order": (_I, [_P, _P, _I64, ctypes.c_int32, _P, _P, _P]),
        "oracle_relabel": (_I, [_P, _P, _P, _I64, _I, _I64, _P]),
        "oracle_kappa": (_D, [_I, _D, _D, _D]),
        "oracle_dkappa_dell": (_D, [_I, _D, _D, _D]),
        "oracle_factor": (_I, [_P, _P, _I64, _I, _I64, _I, _D, _D, _D, _P, _P, _P, _P, _P]),
        "oracle_generate": (None, [_P, _P, _P, _P, _I64, _I, _I64, _P, _P]),
        "oracle_whiten": (None, [_P, _P, _P, _P, _I64, _I, _I64, _P, _P]),
        "oracle_logdet": (_D, [_P, _I64]),
        "oracle_logdet_f32": (_D, [_P, _I64]),
        "oracle_generate_alg1": (_I, [_P, _P, _I64, _I, _I64, _I, _D, _D, _D, _P, _P]),
        "oracle_dense_rows": (_I, [_P, _I64, _P]),
        "oracle_whiten_vjp": (None, [_P, _P, _P, _P, _I64, _I, _I64, _P, _P, _P, _D, _P, _P, _P, _P]),
        "oracle_generate_vjp": (None, [_P, _P, _P, _P, _I64, _I, _I64, _P, _P, _P, _P, _P, _P, _P]),
        "oracle_factor_backward": (_I, [_P, _P, _I64, _I, _I64, _I, _D, _D, _D, _P, _P, _P, _P]),
        "oracle_kappa_h": (_D, [_I, _D, _D, _D]),
        "oracle_factor_backward_points": (_I, [_P, _P, _I64, _I, _I64, _I, _D, _D, _D, _P, _P, _P,
                                                _P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed ({rc})")


def default_n0(N: int, k: int) -> int:
    """Dense block size when none is given: min(N, max(k, 256))."""
    return min(N, max(k, 256))


# --- tree shape ----------------------------------------------------------------
def level(j): return lib().oracle_level(j)
def left(j): return lib().oracle_left(j)
def right(j): return lib().oracle_right(j)
def parent(j): return lib().oracle_parent(j)
def subtree_size(j, N): return lib().oracle_subtree_size(j, N)


def canonicalise(pts):
    """Copy of float32[N,3] points with -0.0 read as +0.0; raises on NaN/inf."""
    p = np.array(pts, dtype=np.float32, order="C", copy=True)
    bad = lib().oracle_canonicalise(_p(p), p.size)
    if bad:
        raise ValueError(f"{bad} non-finite coordinates")
    return p


def tree_build(pts, rule: int = 0):
    pts = _c(pts, np.float32)
    N = pts.shape[0]
    tp = np.empty(N, np.int32)
    sd = np.empty(N, np.uint8)
    io = np.empty(N, np.int64)
    _check(lib().oracle_tree_build(_p(pts), N, rule, _p(tp), _p(sd), _p(io)), "tree_build")
    return tp, sd, io


def d2(a, b) -> np.float32:
    a = _c(a, np.float32)
    b = _c(b, np.float32)
    return np.float32(lib().oracle_d2(_p(a), _p(b)))


def knn_brute(pts, tree_point, k, n0):
    pts = _c(pts, np.float32)
    tp = _c(tree_point, np.int32)
    N = pts.shape[0]
    out = np.empty((max(N - n0, 0), k), np.int32)
    _check(lib().oracle_knn_brute(_p(pts), _p(tp), N, k, n0, _p(out)), "knn_brute")
    return out


def knn_brute_some(pts, tree_point, js, k):
    """The brute-force definition for the tree indices js only: row r holds
    c(js[r]) nearest first (-1 padding)."""
    pts = _c(pts, np.float32)
    tp = _c(tree_point, np.int32)
    js = _c(js, np.int64)
    out = np.empty((len(js), k), np.int32)
    _check(lib().oracle_knn_brute_some(_p(pts), _p(tp), _p(js), len(js), k, _p(out)),
           "knn_brute_some")
    return out


def knn_tree(pts, tree_point, split_dim, k, n0):
    pts = _c(pts, np.float32)
    tp = _c(tree_point, np.int32)
    sd = _c(split_dim, np.uint8)
    N = pts.shape[0]
    out = np.empty((max(N - n0, 0), k), np.int32)
    _check(lib().oracle_knn_tree(_p(pts), _p(tp), _p(sd), N, k, n0, _p(out)), "knn_tree")
    return out


def depth(nbr_tree, N, k, n0):
    nb = _c(nbr_tree, np.int32)
    out = np.empty(N, np.int32)
    _check(lib().oracle_depth(_p(nb), N, k, n0, _p(out)), "depth")
    return out


def order(depth_arr, inorder):
    dp = _c(depth_arr, np.int32)
    io = _c(inorder, np.int64)
    N = dp.shape[0]
    md = int(dp.max())
    top = np.empty(N, np.int32)
    pot = np.empty(N, np.int32)
    lo = np.empty(md + 2, np.int64)
    _check(lib().oracle_order(_p(dp), _p(io), N, md, _p(top), _p(pot), _p(lo)), "order")
    return top, pot, lo


def relabel(nbr_tree, tree_of_pos, pos_of_tree, k, n0):
    nb = _c(nbr_tree, np.int32)
    top = _c(tree_of_pos, np.int32)
    pot = _c(pos_of_tree, np.int32)
    N = top.shape[0]
    out = np.empty((max(N - n0, 0), k), np.int32)
    _check(lib().oracle_relabel(_p(nb), _p(top), _p(pot), N, k, n0, _p(out)), "relabel")
    return out


def build_graph(pts, k, n0=None, rule=0, knn="brute"):
    """The whole graph construction of Sec. 2.2, step by step."""
    pts = canonicalise(pts)
    N = pts.shape[0]
    if n0 is None:
        n0 = default_n0(N, k)
    tp, sd, io = tree_build(pts, rule)
    if knn == "brute":
        nbt = knn_brute(pts, tp, k, n0)
    else:
        nbt = knn_tree(pts, tp, sd, k, n0)
    dp = depth(nbt, N, k, n0)
    top, pot, lo = order(dp, io)
    nbp = relabel(nbt, top, pot, k, n0)
    order_in = tp[top]  # position -> input index
    return dict(N=N, k=k, n0=n0, pts=pts, tree_point=tp, split_dim=sd, inorder=io,
                nbr_tree=nbt, depth=dp, tree_of_pos=top, pos_of_tree=pot,
                level_offsets=lo, nbr_pos=nbp, order=order_in,
                pts_pos=np.ascontiguousarray(pts[order_in]))


# --- covariance and factor -----------------------------------------------------
def kappa(kern: Kernel, r):
    return lib().oracle_kappa(kern.type, kern.sigma2, kern.lengthscale, float(r))


def dkappa_dell(kern: Kernel, r):
    return lib().oracle_dkappa_dell(kern.type, kern.sigma2, kern.lengthscale, float(r))


def factor(pts_pos, nbr_pos, k, n0, kern: Kernel):
    pp = _c(pts_pos, np.float32)
    nb = _c(nbr_pos, np.int32)
    N = pp.shape[0]
    b = np.zeros((max(N - n0, 0), k), np.float64)
    sigma = np.empty(N, np.float64)
    L0 = np.zeros((n0, n0), np.float64)
    ld = ctypes.c_double(0.0)
    bad = ctypes.c_int64(0)
    _check(lib().oracle_factor(_p(pp), _p(nb), N, k, n0, kern.type, kern.sigma2,
                               kern.lengthscale, kern.nugget, _p(b), _p(sigma), _p(L0),
                               ctypes.byref(ld), ctypes.byref(bad)), "factor")
    return dict(b=b, sigma=sigma, L0=L0, logdet=ld.value, n_not_pd=bad.value)


def factor_rows(pts, idx, nbr, kern: Kernel):
    """Eq. 2 for the points idx of pts (any order) with neighbour lists nbr
    (indices into pts, -1 padding): (b [n, k], sigma [n]) in FP64."""
    pp = _c(pts, np.float32)
    ix = _c(idx, np.int64)
    nb = _c(nbr, np.int32)
    n, k = nb.shape
    b = np.zeros((n, k), np.float64)
    sigma = np.empty(n, np.float64)
    _check(lib().oracle_factor_rows(_p(pp), _p(ix), _p(nb), n, k, kern.type, kern.sigma2,
                                    kern.lengthscale, kern.nugget, _p(b), _p(sigma)), "factor_rows")
    return b, sigma


def generate(fac, nbr_pos, k, n0, xi):
    xi = _c(xi, np.float64)
    N = xi.shape[0]
    v = np.empty(N, np.float64)
    lib().oracle_generate(_p(fac["b"]), _p(fac["sigma"]), _p(fac["L0"]), _p(_c(nbr_pos, np.int32)),
                          N, k, n0, _p(xi), _p(v))
    return v


def whiten(fac, nbr_pos, k, n0, v):
    v = _c(v, np.float64)
    N = v.shape[0]
    xi = np.empty(N, np.float64)
    lib().oracle_whiten(_p(fac["b"]), _p(fac["sigma"]), _p(fac["L0"]), _p(_c(nbr_pos, np.int32)),
                        N, k, n0, _p(v), _p(xi))
    return xi


def logdet(sigma):
    s = _c(sigma, np.float64)
    return lib().oracle_logdet(_p(s), s.shape[0])


def logdet_f32(sigma):
    s = _c(sigma, np.float32)
    return lib().oracle_logdet_f32(_p(s), s.shape[0])


def generate_alg1(pts_pos, nbr_pos, k, n0, kern: Kernel, xi):
    pp = _c(pts_pos, np.float32)
    xi = _c(xi, np.float64)
    N = pp.shape[0]
    v = np.empty(N, np.float64)
    _check(lib().oracle_generate_alg1(_p(pp), _p(_c(nbr_pos, np.int32)), N, k, n0, kern.type,
                                      kern.sigma2, kern.lengthscale, kern.nugget, _p(xi), _p(v)),
           "generate_alg1")
    return v


def nll(fac, nbr_pos, k, n0, v):
    """0.5 xi.xi + 0.5 logdet with xi = whiten(v); no 0.5 N log(2 pi) term."""
    xi = whiten(fac, nbr_pos, k, n0, v)
    return 0.5 * float(xi @ xi) + 0.5 * fac["logdet"]


# --- adjoints ------------------------------------------------------------------
def dense_rows(L0):
    L0 = _c(L0, np.float64)
    n0 = L0.shape[0]
    bd = np.zeros((n0, n0), np.float64)
    _check(lib().oracle_dense_rows(_p(L0), n0, _p(bd)), "dense_rows")
    return bd


def whiten_vjp(fac, nbr_pos, k, n0, v, xi, xibar, logdetbar=0.0):
    v = _c(v, np.float64); xi = _c(xi, np.float64); xibar = _c(xibar, np.float64)
    N = v.shape[0]
    bd = dense_rows(fac["L0"])
    vbar = np.empty(N); bbar = np.zeros((max(N - n0, 0), k)); bdbar = np.zeros((n0, n0))
    sigbar = np.empty(N)
    lib().oracle_whiten_vjp(_p(fac["b"]), _p(bd), _p(fac["sigma"]), _p(_c(nbr_pos, np.int32)),
                            N, k, n0, _p(v), _p(xi), _p(xibar), float(logdetbar),
                            _p(vbar), _p(bbar), _p(bdbar), _p(sigbar))
    return dict(vbar=vbar, bbar=bbar, bdbar=bdbar, sigbar=sigbar)


def generate_vjp(fac, nbr_pos, k, n0, xi, v, vbar):
    v = _c(v, np.float64); xi = _c(xi, np.float64); vbar = _c(vbar, np.float64)
    N = v.shape[0]
    bd = dense_rows(fac["L0"])
    xibar = np.empty(N); bbar = np.zeros((max(N - n0, 0), k)); bdbar = np.zeros((n0, n0))
    sigbar = np.empty(N)
    lib().oracle_generate_vjp(_p(fac["b"]), _p(bd), _p(fac["sigma"]), _p(_c(nbr_pos, np.int32)),
                              N, k, n0, _p(xi), _p(v), _p(vbar), _p(xibar), _p(bbar), _p(bdbar),
                              _p(sigbar))
    return dict(xibar=xibar, bbar=bbar, bdbar=bdbar, sigbar=sigbar)


def factor_backward(pts_pos, nbr_pos, k, n0, kern: Kernel, bbar, bdbar, sigbar):
    pp = _c(pts_pos, np.float32)
    N = pp.shape[0]
    tb = np.zeros(3, np.float64)
    _check(lib().oracle_factor_backward(_p(pp), _p(_c(nbr_pos, np.int32)), N, k, n0, kern.type,
                                        kern.sigma2, kern.lengthscale, kern.nugget,
                                        _p(_c(bbar, np.float64)), _p(_c(bdbar, np.float64)),
                                        _p(_c(sigbar, np.float64)), _p(tb)), "factor_backward")
    return tb  # [d/dlengthscale, d/dsigma2, d/dnugget]


def nll_grad(g, kern: Kernel, v):
    """Gradient of nll(v; theta): returns (vbar, thetabar[3])."""
    k, n0 = g["k"], g["n0"]
    fac = factor(g["pts_pos"], g["nbr_pos"], k, n0, kern)
    xi = whiten(fac, g["nbr_pos"], k, n0, v)
    a = whiten_vjp(fac, g["nbr_pos"], k, n0, v, xi, xi, 0.5)
    tb = factor_backward(g["pts_pos"], g["nbr_pos"], k, n0, kern, a["bbar"], a["bdbar"], a["sigbar"])
    return a["vbar"], tb


def kappa_h(kern: Kernel, r):
    """kappa'(r) / r (0 at r = 0 for Matern-1/2)."""
    return lib().oracle_kappa_h(kern.type, kern.sigma2, kern.lengthscale, float(r))


def nll_grad_points(g, kern: Kernel, v):
    """Gradient of nll(v; points) with respect to the point coordinates, the
    graph (order, neighbour lists, levels) held fixed.  Returns float64[N, 3]
    in INPUT order (the layout of the points given to build_graph)."""
    k, n0 = g["k"], g["n0"]
    fac = factor(g["pts_pos"], g["nbr_pos"], k, n0, kern)
    xi = whiten(fac, g["nbr_pos"], k, n0, v)
    a = whiten_vjp(fac, g["nbr_pos"], k, n0, v, xi, xi, 0.5)
    pp = _c(g["pts_pos"], np.float32)
    N = pp.shape[0]
    xb = np.zeros((N, 3), np.float64)
    _check(lib().oracle_factor_backward_points(
        _p(pp), _p(_c(g["nbr_pos"], np.int32)), N, k, n0, kern.type, kern.sigma2,
        kern.lengthscale, kern.nugget, _p(_c(a["bbar"], np.float64)),
        _p(_c(a["bdbar"], np.float64)), _p(_c(a["sigbar"], np.float64)), _p(xb)),
        "factor_backward_points")
    out = np.empty_like(xb)
    out[np.asarray(g["order"], np.int64)] = xb
    return out
