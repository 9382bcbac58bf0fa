"""Test infrastructure: ctypes front end of the CPU oracle (oracle.cpp).

The oracle is the plain FP64 restatement of the Embedded-IPC contact stage that the CUDA
library is checked against.  Only the tests, the smoke check and the CPU-baseline leg of
the benchmark use it; the library never imports it.  `build()` compiles oracle.cpp with
-ffp-contract=off (no fused multiply-adds, so every operation rounds as written) and
OpenMP, into oracle/_build/.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRCS = ["oracle.cpp", "ad.hpp", "geometry.hpp", "predicates.hpp"]
_lib = None


def compile_so(src_dir: str, out: str) -> None:
    """Compiles oracle.cpp (and the headers beside it) from src_dir into the shared library
    `out`, written under a temporary name first."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           os.path.join(src_dir, "oracle.cpp"), "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    src_time = max(os.path.getmtime(os.path.join(_HERE, s)) for s in _SRCS)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < src_time:
        compile_so(_HERE, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = bind(ctypes.CDLL(_SO))
    return _lib


def bind(L):
    """Declares the argument and result types of every entry point of a loaded oracle."""
    P = ctypes.c_void_p
    i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    L.orc_embed.argtypes = [i64, P, P, P, P, P]
    L.orc_pair_d2.argtypes = [ctypes.c_int, P, P, P]
    L.orc_pair_d2.restype = dbl
    L.orc_barrier.argtypes = [dbl, dbl, P]
    L.orc_f0.argtypes = [dbl, dbl, P]
    L.orc_pair_barrier.argtypes = [ctypes.c_int, P, dbl, dbl, P, P, P, P]
    L.orc_psd_project.argtypes = [ctypes.c_int, P, P]
    L.orc_eigen.argtypes = [ctypes.c_int, P, P, P]
    L.orc_pairs.argtypes = [i64, P, P, i64, P, i64, P, dbl, i64, P, P, P, P]
    L.orc_pairs.restype = i64
    L.orc_pairs_of.argtypes = [i64, P, P, i64, P, i64, P, dbl, ctypes.c_int, i64, P, i64, P, P, P]
    L.orc_pairs_of.restype = i64
    L.orc_friction_lag.argtypes = [i64, P, i64, P, i64, P, i64, P, P, P, dbl, dbl, P, P, P, P, P]
    L.orc_eval.argtypes = [i64, P, i64, P, i64, P, P, P, i64, i64, P, P, P, i64, P, P, P, P, P,
                           dbl, dbl, dbl, dbl, ctypes.c_int]
    L.orc_eval.restype = P
    L.orc_hvp.argtypes = [i64, P, i64, P, i64, P, P, P, i64, i64, P, P, P, i64, P, P, P, P, P,
                          dbl, dbl, dbl, dbl, P, P, P]
    L.orc_dedup.argtypes = [i64, P, i64, P, i64, P, i64, P, P, P, P]
    L.orc_set_mollifier.argtypes = [i64, P, dbl]
    L.orc_pair_barrier_mollified.argtypes = [P, dbl, dbl, dbl, P, P, P]
    L.orc_result_nnzb.argtypes = [P]
    L.orc_result_nnzb.restype = i64
    L.orc_result_copy.argtypes = [P, P, P, P, P, P, P]
    L.orc_result_free.argtypes = [P]
    L.orc_pair_friction.argtypes = [P, P, P, P, dbl, P, dbl, dbl, P, P, P]
    L.orc_ca_pair.argtypes = [ctypes.c_int, P, P, dbl, ctypes.c_int, P, P]
    L.orc_ca_pair.restype = dbl
    L.orc_accd.argtypes = [i64, P, P, P, i64, P, i64, P, dbl, ctypes.c_int, P, P, P]
    L.orc_accd.restype = dbl
    L.orc_accd_list.argtypes = [i64, P, P, P, i64, P, P, i64, P, i64, P, dbl, ctypes.c_int, P]
    L.orc_accd_list.restype = dbl
    L.orc_accd_of.argtypes = [i64, P, P, P, i64, P, i64, P, dbl, ctypes.c_int, ctypes.c_int, i64, P, P, P]
    L.orc_accd_of.restype = dbl
    L.orc_intersection_free.argtypes = [i64, P, i64, P, i64, P]
    L.orc_intersection_free.restype = ctypes.c_int
    L.orc_num_threads.restype = ctypes.c_int
    L.orc_set_threads.argtypes = [ctypes.c_int]
    return L


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


# ---------------------------------------------------------------------------- wrappers

def embed(scene, q: np.ndarray, displacement: bool = False) -> np.ndarray:
    """x = J q (Sec. III-D).  With displacement=True the map is applied to a reduced
    displacement dq: kinematic vertices then do not move (dx = 0)."""
    q = _f64(q)
    x = np.zeros((scene.Nv, 3))
    xk = np.zeros_like(scene.x_kin) if displacement else _f64(scene.x_kin)
    lib().orc_embed(scene.Nv, _p(_i32(scene.cage_idx)), _p(_f64(scene.w)), _p(xk), _p(q), _p(x))
    return x


def pair_d2(ptype: int, x4: np.ndarray):
    x4 = _f64(x4).reshape(12)
    reg = np.zeros(1, np.int32)
    c = np.zeros(4)
    d2 = lib().orc_pair_d2(int(ptype), _p(x4), _p(reg), _p(c))
    return d2, int(reg[0]), c


def barrier(d: float, dhat: float) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_barrier(float(d), float(dhat), _p(out))
    return out


def f0(y: float, eps: float) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_f0(float(y), float(eps), _p(out))
    return out


def pair_barrier(ptype: int, x4: np.ndarray, dhat: float, kappa: float):
    x4 = _f64(x4).reshape(12)
    E = np.zeros(1); g = np.zeros(12); H = np.zeros(144); Hp = np.zeros(144)
    lib().orc_pair_barrier(int(ptype), _p(x4), float(dhat), float(kappa), _p(E), _p(g), _p(H), _p(Hp))
    return float(E[0]), g, H.reshape(12, 12), Hp.reshape(12, 12)


def psd_project(H: np.ndarray) -> np.ndarray:
    H = _f64(H)
    n = H.shape[0]
    out = np.zeros_like(H)
    lib().orc_psd_project(n, _p(H), _p(out))
    return out


def eigen(H: np.ndarray):
    H = _f64(H)
    n = H.shape[0]
    lam = np.zeros(n); V = np.zeros((n, n))
    lib().orc_eigen(n, _p(H), _p(lam), _p(V))
    return lam, V


def _kin(scene) -> np.ndarray:
    return np.ascontiguousarray(scene.kinematic.astype(np.uint8))


def pairs(scene, x: np.ndarray, dhat: Optional[float] = None) -> Dict[str, np.ndarray]:
    """Brute-force contact set, ordered by (type, i, j).  Raises on penetration."""
    dhat = scene.params["dhat"] if dhat is None else dhat
    x = _f64(x)
    cap = 1 << 16
    while True:
        t = np.zeros(cap, np.int32); i = np.zeros(cap, np.int32); j = np.zeros(cap, np.int32); d = np.zeros(cap)
        n = lib().orc_pairs(scene.Nv, _p(x), _p(_kin(scene)), scene.F, _p(_i32(scene.tris)), scene.E,
                            _p(_i32(scene.edges)), float(dhat), cap, _p(t), _p(i), _p(j), _p(d))
        if n < 0:
            raise RuntimeError("penetration: a contact pair has d <= 0")
        if n <= cap:
            return dict(type=t[:n], i=i[:n], j=j[:n], d=d[:n])
        cap = int(n)


def pairs_of(scene, x: np.ndarray, ptype: int, queries: np.ndarray, dhat: Optional[float] = None):
    dhat = scene.params["dhat"] if dhat is None else dhat
    q = _i32(queries)
    cap = 1 << 14
    while True:
        i = np.zeros(cap, np.int32); j = np.zeros(cap, np.int32); d = np.zeros(cap)
        n = lib().orc_pairs_of(scene.Nv, _p(_f64(x)), _p(_kin(scene)), scene.F, _p(_i32(scene.tris)), scene.E,
                               _p(_i32(scene.edges)), float(dhat), int(ptype), len(q), _p(q), cap,
                               _p(i), _p(j), _p(d))
        if n <= cap:
            return dict(i=i[:n], j=j[:n], d=d[:n])
        cap = int(n)


MOLLIFIER_FACTOR = 1e-3


def set_mollifier(scene, x_rest: Optional[np.ndarray], factor: float = MOLLIFIER_FACTOR) -> None:
    """Turn the EE mollifier on (eps_x = factor |e_i|^2 |e_j|^2 at the rest positions
    x_rest) or off (x_rest None).  Applies to every later oracle call."""
    if x_rest is None:
        lib().orc_set_mollifier(0, None, 0.0)
        return
    e = scene.edges
    r2 = np.ascontiguousarray(np.sum((x_rest[e[:, 1]] - x_rest[e[:, 0]]) ** 2, axis=1), np.float64)
    lib().orc_set_mollifier(len(r2), _p(r2), float(factor))


def pair_barrier_mollified(x4: np.ndarray, eps: float, dhat: float, kappa: float):
    E = np.zeros(1); g = np.zeros(12); H = np.zeros(144)
    lib().orc_pair_barrier_mollified(_p(_f64(x4).reshape(12)), float(eps), float(dhat), float(kappa), _p(E), _p(g),
                                     _p(H))
    return float(E[0]), g, H.reshape(12, 12)


def dedup(scene, x: np.ndarray, prs: Dict[str, np.ndarray]) -> Dict[str, np.ndarray]:
    """The deduplicated contact set: pairs realising the same feature pair (face-vertex,
    vertex-edge, vertex-vertex, edge-edge interior) count once, the first in (type, i, j)
    order standing for them."""
    order = np.lexsort((prs["j"], prs["i"], prs["type"]))
    t, i, j = (np.ascontiguousarray(prs[k][order], np.int32) for k in ("type", "i", "j"))
    keep = np.zeros(len(t), np.int32)
    lib().orc_dedup(scene.Nv, _p(_f64(x)), scene.F, _p(_i32(scene.tris)), scene.E, _p(_i32(scene.edges)), len(t),
                    _p(t), _p(i), _p(j), _p(keep))
    sel = keep.astype(bool)
    out = dict(type=t[sel], i=i[sel], j=j[sel])
    if "d" in prs:
        out["d"] = np.asarray(prs["d"])[order][sel]
    return out


def friction_lag(scene, xn: np.ndarray, prs: Dict[str, np.ndarray]) -> Dict[str, np.ndarray]:
    n = len(prs["type"])
    lv = np.zeros((n, 4), np.int32); lg = np.zeros((n, 4)); ln = np.zeros((n, 3)); la = np.zeros((n, 3))
    ll = np.zeros(n)
    p = scene.params
    lib().orc_friction_lag(scene.Nv, _p(_f64(xn)), scene.F, _p(_i32(scene.tris)), scene.E, _p(_i32(scene.edges)),
                           n, _p(_i32(prs["type"])), _p(_i32(prs["i"])), _p(_i32(prs["j"])),
                           float(p["dhat"]), float(p["kappa"]), _p(lv), _p(lg), _p(ln), _p(la), _p(ll))
    return dict(v=lv, gamma=lg, n=ln, anchor=la, lam=ll)


def eval_contact(scene, x: np.ndarray, prs: Dict[str, np.ndarray], lag: Optional[Dict[str, np.ndarray]],
                 project: bool = True, params: Optional[dict] = None):
    """E, g_r [Ns,3] and the reduced Hessian as sorted blocks (I, J, vals[9])."""
    p = dict(scene.params) if params is None else params
    np_ = len(prs["type"])
    if lag is None or p["mu"] == 0.0:
        nfr = 0
        lag = dict(v=np.zeros((0, 4), np.int32), gamma=np.zeros((0, 4)), n=np.zeros((0, 3)),
                   anchor=np.zeros((0, 3)), lam=np.zeros(0))
    else:
        nfr = len(lag["lam"])
    L = lib()
    h = L.orc_eval(scene.Nv, _p(_f64(x)), scene.F, _p(_i32(scene.tris)), scene.E, _p(_i32(scene.edges)),
                   _p(_i32(scene.cage_idx)), _p(_f64(scene.w)), scene.Ns, np_,
                   _p(_i32(prs["type"])), _p(_i32(prs["i"])), _p(_i32(prs["j"])), nfr,
                   _p(_i32(lag["v"])), _p(_f64(lag["gamma"])), _p(_f64(lag["n"])), _p(_f64(lag["anchor"])),
                   _p(_f64(lag["lam"])), float(p["dhat"]), float(p["kappa"]), float(p["mu"]),
                   float(p["eps_v"] * p["h"]), 1 if project else 0)
    try:
        nnzb = L.orc_result_nnzb(h)
        E = np.zeros(1); g = np.zeros((scene.Ns, 3)); I = np.zeros(nnzb, np.int32); J = np.zeros(nnzb, np.int32)
        V = np.zeros((nnzb, 3, 3)); Ek = np.zeros(max(np_, 1))
        L.orc_result_copy(h, _p(E), _p(g), _p(I), _p(J), _p(V), _p(Ek))
    finally:
        L.orc_result_free(h)
    return dict(E=float(E[0]), g=g, I=I, J=J, V=V, Ek=Ek[:np_])


def hvp(scene, x: np.ndarray, prs: Dict[str, np.ndarray], lag: Optional[Dict[str, np.ndarray]], u: np.ndarray,
        params: Optional[dict] = None):
    """Unprojected contact Hessian times a full-space direction u [Nv,3] (kinematic
    vertices included): returns (J^T y [Ns,3], sum of y over kinematic vertices [3])."""
    p = dict(scene.params) if params is None else params
    np_ = len(prs["type"])
    if lag is None or p["mu"] == 0.0:
        nfr = 0
        lag = dict(v=np.zeros((0, 4), np.int32), gamma=np.zeros((0, 4)), n=np.zeros((0, 3)),
                   anchor=np.zeros((0, 3)), lam=np.zeros(0))
    else:
        nfr = len(lag["lam"])
    out_r = np.zeros((scene.Ns, 3))
    out_k = np.zeros(3)
    lib().orc_hvp(scene.Nv, _p(_f64(x)), scene.F, _p(_i32(scene.tris)), scene.E, _p(_i32(scene.edges)),
                  _p(_i32(scene.cage_idx)), _p(_f64(scene.w)), scene.Ns, np_,
                  _p(_i32(prs["type"])), _p(_i32(prs["i"])), _p(_i32(prs["j"])), nfr,
                  _p(_i32(lag["v"])), _p(_f64(lag["gamma"])), _p(_f64(lag["n"])), _p(_f64(lag["anchor"])),
                  _p(_f64(lag["lam"])), float(p["dhat"]), float(p["kappa"]), float(p["mu"]),
                  float(p["eps_v"] * p["h"]), _p(_f64(u)), _p(out_r), _p(out_k))
    return out_r, out_k


def pair_friction(v4, gamma4, n3, anchor3, lam, x4, mu, eps):
    E = np.zeros(1); g = np.zeros(12); H = np.zeros(144)
    lib().orc_pair_friction(_p(_i32(v4)), _p(_f64(gamma4)), _p(_f64(n3)), _p(_f64(anchor3)), float(lam),
                            _p(_f64(x4).reshape(12)), float(mu), float(eps), _p(E), _p(g), _p(H))
    return float(E[0]), g, H.reshape(12, 12)


def ca_pair(ptype, x4, dx4, s=0.1, max_iter=10000):
    it = np.zeros(1, np.int32); cap = np.zeros(1, np.int32)
    t = lib().orc_ca_pair(int(ptype), _p(_f64(x4).reshape(12)), _p(_f64(dx4).reshape(12)), float(s),
                          int(max_iter), _p(it), _p(cap))
    return t, int(it[0]), bool(cap[0])


def accd(scene, x: np.ndarray, dx: np.ndarray, s: Optional[float] = None, max_iter: Optional[int] = None):
    p = scene.params
    s = p["accd_s"] if s is None else s
    max_iter = p["accd_max_iter"] if max_iter is None else max_iter
    nc = np.zeros(1, np.int64); it = np.zeros(1, np.int64); cp = np.zeros(1, np.int32)
    a = lib().orc_accd(scene.Nv, _p(_f64(x)), _p(_f64(dx)), _p(_kin(scene)), scene.F, _p(_i32(scene.tris)),
                       scene.E, _p(_i32(scene.edges)), float(s), int(max_iter), _p(nc), _p(it), _p(cp))
    return dict(alpha=a, n_candidates=int(nc[0]), iters=int(it[0]), capped=bool(cp[0]))


def accd_of(scene, x, dx, ptype: int, queries, s=None, max_iter=None):
    """Step bound over the pairs having one of `queries` (vertices if ptype == 0, edges if
    ptype == 1) as a side: a bounded sample of `accd`."""
    p = scene.params
    s = p["accd_s"] if s is None else s
    max_iter = p["accd_max_iter"] if max_iter is None else max_iter
    q = _i32(queries)
    nc = np.zeros(1, np.int64); it = np.zeros(1, np.int64)
    a = lib().orc_accd_of(scene.Nv, _p(_f64(x)), _p(_f64(dx)), _p(_kin(scene)), scene.F, _p(_i32(scene.tris)),
                          scene.E, _p(_i32(scene.edges)), float(s), int(max_iter), int(ptype), len(q), _p(q),
                          _p(nc), _p(it))
    return dict(alpha=a, n_candidates=int(nc[0]), iters=int(it[0]))


def accd_list(scene, x, dx, cand, s=None, max_iter=None):
    p = scene.params
    s = p["accd_s"] if s is None else s
    max_iter = p["accd_max_iter"] if max_iter is None else max_iter
    it = np.zeros(1, np.int64)
    n = len(cand["type"])
    a = lib().orc_accd_list(n, _p(_i32(cand["type"])), _p(_i32(cand["i"])), _p(_i32(cand["j"])), scene.Nv,
                            _p(_f64(x)), _p(_f64(dx)), scene.F, _p(_i32(scene.tris)), scene.E,
                            _p(_i32(scene.edges)), float(s), int(max_iter), _p(it))
    return dict(alpha=a, iters=int(it[0]))


def intersection_free(scene, x: np.ndarray) -> bool:
    return bool(lib().orc_intersection_free(scene.Nv, _p(_f64(x)), scene.F, _p(_i32(scene.tris)), scene.E,
                                            _p(_i32(scene.edges))))
