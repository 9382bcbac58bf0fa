"""ctypes binding of libembipc.so (include/embipc.h): argument marshalling only.

Device memory comes from torch CUDA tensors and every call is enqueued on torch's current
CUDA stream; all arithmetic runs in the library's kernels.  Importing works without a GPU;
constructing a `ContactScene` requires the compiled library and a CUDA device and raises
otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import build as _build

_lib = None

EIPC_OK = 0
FLAGS = {1: "PENETRATION", 2: "PAIR_OVERFLOW", 4: "CAND_OVERFLOW", 8: "REC_OVERFLOW", 16: "BSR_OVERFLOW",
         32: "NONFINITE", 64: "ACCD_CAP", 128: "LAG_OVERFLOW", 256: "STACK_OVERFLOW", 512: "BAD_INDEX"}
EXPORTS = ["eipc_scene_create", "eipc_scene_destroy", "eipc_embed", "eipc_build_candidates", "eipc_friction_lag",
           "eipc_eval_contact", "eipc_accd_toi", "eipc_status_read", "eipc_version", "eipc_timing_enable",
           "eipc_timing_read", "eipc_kernel_name", "eipc_launch_count", "eipc_set_rebuild_interval",
           "eipc_scene_set_groups", "eipc_group_energy", "eipc_group_alpha", "eipc_set_launch",
           "eipc_contact_hvp", "eipc_scene_set_kinematic", "eipc_scene_set_mollifier", "eipc_bsr_spmv",
           "eipc_work_counts", "eipc_candidates_read", "eipc_fp64_probe", "eipc_fp64_probe_flops",
           "eipc_set_programmatic_launch"]


class Params(ctypes.Structure):
    _fields_ = [("dhat", ctypes.c_double), ("kappa", ctypes.c_double), ("mu", ctypes.c_double),
                ("eps_v", ctypes.c_double), ("h", ctypes.c_double), ("accd_s", ctypes.c_double),
                ("accd_max_iter", ctypes.c_int32), ("flags", ctypes.c_int32)]


class _Pairs(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64), ("type", ctypes.c_void_p), ("i", ctypes.c_void_p),
                ("j", ctypes.c_void_p), ("d", ctypes.c_void_p), ("count", ctypes.c_void_p)]


class _Lag(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64), ("v", ctypes.c_void_p), ("gamma", ctypes.c_void_p),
                ("n", ctypes.c_void_p), ("anchor", ctypes.c_void_p), ("lam", ctypes.c_void_p),
                ("count", ctypes.c_void_p)]


class _Bsr(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                ("val", ctypes.c_void_p), ("nnzb", ctypes.c_void_p)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libembipc.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libembipc.so is not built ({_build.LIB}); run paper_2409_16385_gb300.build.build()")
    L = ctypes.CDLL(_build.LIB)
    P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    L.eipc_scene_create.argtypes = [i64, i64, i64, i64, P, P, P, P, P, i64, i64, ctypes.POINTER(P)]
    L.eipc_scene_create.restype = i32
    L.eipc_scene_destroy.argtypes = [P]
    L.eipc_embed.argtypes = [P, P, P, i32, P]
    L.eipc_embed.restype = i32
    L.eipc_build_candidates.argtypes = [P, P, ctypes.POINTER(Params), ctypes.POINTER(_Pairs), P]
    L.eipc_build_candidates.restype = i32
    L.eipc_friction_lag.argtypes = [P, P, ctypes.POINTER(_Pairs), ctypes.POINTER(Params), ctypes.POINTER(_Lag), P]
    L.eipc_friction_lag.restype = i32
    L.eipc_eval_contact.argtypes = [P, P, ctypes.POINTER(_Pairs), ctypes.POINTER(_Lag), ctypes.POINTER(Params), P, P,
                                    ctypes.POINTER(_Bsr), P]
    L.eipc_eval_contact.restype = i32
    L.eipc_accd_toi.argtypes = [P, P, P, ctypes.POINTER(Params), P, P, P]
    L.eipc_accd_toi.restype = i32
    L.eipc_status_read.argtypes = [P, P, ctypes.POINTER(i32), P, P]
    L.eipc_status_read.restype = i32
    L.eipc_work_counts.argtypes = [P, P, P, i32]
    L.eipc_work_counts.restype = i32
    L.eipc_version.restype = ctypes.c_char_p
    L.eipc_timing_enable.argtypes = [P, ctypes.c_uint32]
    L.eipc_timing_enable.restype = i32
    L.eipc_timing_read.argtypes = [P, P, P, i32]
    L.eipc_timing_read.restype = i32
    L.eipc_kernel_name.argtypes = [i32]
    L.eipc_kernel_name.restype = ctypes.c_char_p
    L.eipc_set_rebuild_interval.argtypes = [P, i32]
    L.eipc_set_rebuild_interval.restype = i32
    L.eipc_launch_count.restype = i64
    L.eipc_set_programmatic_launch.argtypes = [i32]
    L.eipc_set_programmatic_launch.restype = None
    L.eipc_scene_set_groups.argtypes = [P, P, i32]
    L.eipc_scene_set_groups.restype = i32
    L.eipc_group_energy.argtypes = [P, P, P]
    L.eipc_group_energy.restype = i32
    L.eipc_group_alpha.argtypes = [P, P, P]
    L.eipc_group_alpha.restype = i32
    L.eipc_set_launch.argtypes = [P, i32, i32, i32, i32]
    L.eipc_set_launch.restype = i32
    L.eipc_contact_hvp.argtypes = [P, P, ctypes.POINTER(_Pairs), ctypes.POINTER(_Lag), ctypes.POINTER(Params), P, P, P,
                                   P, P]
    L.eipc_contact_hvp.restype = i32
    L.eipc_scene_set_kinematic.argtypes = [P, P, P]
    L.eipc_scene_set_kinematic.restype = i32
    L.eipc_scene_set_mollifier.argtypes = [P, P, ctypes.c_double, P]
    L.eipc_scene_set_mollifier.restype = i32
    L.eipc_bsr_spmv.argtypes = [i64, P, P, P, P, ctypes.c_double, ctypes.c_double, P, P]
    L.eipc_bsr_spmv.restype = i32
    L.eipc_candidates_read.argtypes = [P, P, P, P, i64, P, P]
    L.eipc_candidates_read.restype = i32
    L.eipc_fp64_probe.argtypes = [i64, P, P]
    L.eipc_fp64_probe.restype = i32
    L.eipc_fp64_probe_flops.argtypes = [i64]
    L.eipc_fp64_probe_flops.restype = i64
    _lib = L
    return L


def _check(rc: int, what: str):
    if rc != EIPC_OK:
        raise RuntimeError(f"{what} failed with status {rc}")


def _ptr(t) -> int:
    return t.data_ptr()


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def make_params(p: dict) -> Params:
    return Params(float(p["dhat"]), float(p["kappa"]), float(p.get("mu", 0.0)), float(p.get("eps_v", 1e-3)),
                  float(p.get("h", 1e-2)), float(p.get("accd_s", 0.1)), int(p.get("accd_max_iter", 10000)), 0)


@dataclass
class PairList:
    type: "object"
    i: "object"
    j: "object"
    d: "object"
    count: "object"   # int64[1] device

    def n(self) -> int:
        return int(self.count.item())

    def host(self):
        n = min(self.n(), self.type.shape[0])
        return dict(type=self.type[:n].cpu().numpy(), i=self.i[:n].cpu().numpy(), j=self.j[:n].cpu().numpy(),
                    d=self.d[:n].cpu().numpy())

    def _c(self) -> _Pairs:
        return _Pairs(self.type.shape[0], _ptr(self.type), _ptr(self.i), _ptr(self.j), _ptr(self.d), _ptr(self.count))


@dataclass
class LagState:
    v: "object"
    gamma: "object"
    n: "object"
    anchor: "object"
    lam: "object"
    count: "object"

    def host(self):
        k = min(int(self.count.item()), self.v.shape[0])
        return dict(v=self.v[:k].cpu().numpy(), gamma=self.gamma[:k].cpu().numpy(), n=self.n[:k].cpu().numpy(),
                    anchor=self.anchor[:k].cpu().numpy(), lam=self.lam[:k].cpu().numpy())

    def _c(self) -> _Lag:
        return _Lag(self.v.shape[0], _ptr(self.v), _ptr(self.gamma), _ptr(self.n), _ptr(self.anchor), _ptr(self.lam),
                    _ptr(self.count))


@dataclass
class BSR:
    row_ptr: "object"
    col: "object"
    val: "object"
    nnzb: "object"

    def host(self):
        k = min(int(self.nnzb.item()), self.col.shape[0])
        return dict(row_ptr=self.row_ptr.cpu().numpy(), col=self.col[:k].cpu().numpy(),
                    val=self.val[:k].cpu().numpy().reshape(-1, 3, 3))

    def _c(self) -> _Bsr:
        return _Bsr(self.col.shape[0], _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val), _ptr(self.nnzb))


class ContactScene:
    """One scene on the device: topology + embedding copied at creation, workspace sized
    once.  Methods map 1:1 to the C ABI calls and enqueue on torch's current stream."""

    def __init__(self, scene, pair_capacity: int = 1 << 20, bsr_capacity: int = 1 << 22,
                 cand_capacity: int = 0, rec_capacity: int = 0, device: str = "cuda"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("ContactScene needs a CUDA device: the contact stage has no CPU path")
        self.lib = load()
        self.device = torch.device(device)
        self.scene = scene
        self.params = make_params(scene.params)
        h = ctypes.c_void_p()
        tris = np.ascontiguousarray(scene.tris, np.int32)
        edges = np.ascontiguousarray(scene.edges, np.int32)
        idx = np.ascontiguousarray(scene.cage_idx, np.int32)
        w = np.ascontiguousarray(scene.w, np.float64)
        xk = np.ascontiguousarray(scene.x_kin, np.float64)
        rc = self.lib.eipc_scene_create(scene.Nv, scene.F, scene.E, scene.Ns, tris.ctypes.data, edges.ctypes.data,
                                        idx.ctypes.data, w.ctypes.data, xk.ctypes.data, int(cand_capacity),
                                        int(rec_capacity), ctypes.byref(h))
        _check(rc, "eipc_scene_create")
        self.handle = h
        self.Ns, self.Nv = scene.Ns, scene.Nv
        self.pair_capacity = int(pair_capacity)
        self.bsr_capacity = int(bsr_capacity)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.eipc_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- buffers
    def new_pairs(self, capacity: Optional[int] = None) -> PairList:
        import torch
        c = self.pair_capacity if capacity is None else int(capacity)
        dev = self.device
        return PairList(torch.empty(c, dtype=torch.int32, device=dev), torch.empty(c, dtype=torch.int32, device=dev),
                        torch.empty(c, dtype=torch.int32, device=dev), torch.empty(c, dtype=torch.float64, device=dev),
                        torch.zeros(1, dtype=torch.int64, device=dev))

    def new_lag(self, capacity: Optional[int] = None) -> LagState:
        import torch
        c = self.pair_capacity if capacity is None else int(capacity)
        dev = self.device
        return LagState(torch.empty((c, 4), dtype=torch.int32, device=dev), torch.empty((c, 4), dtype=torch.float64, device=dev),
                        torch.empty((c, 3), dtype=torch.float64, device=dev), torch.empty((c, 3), dtype=torch.float64, device=dev),
                        torch.empty(c, dtype=torch.float64, device=dev), torch.zeros(1, dtype=torch.int64, device=dev))

    def new_bsr(self, capacity: Optional[int] = None) -> BSR:
        import torch
        c = self.bsr_capacity if capacity is None else int(capacity)
        dev = self.device
        return BSR(torch.zeros(self.Ns + 1, dtype=torch.int32, device=dev), torch.empty(c, dtype=torch.int32, device=dev),
                   torch.empty((c, 9), dtype=torch.float64, device=dev), torch.zeros(1, dtype=torch.int64, device=dev))

    # -- calls
    def embed(self, q, out=None, displacement: bool = False):
        import torch
        x = out if out is not None else torch.empty((self.Nv, 3), dtype=torch.float64, device=self.device)
        _check(self.lib.eipc_embed(self.handle, _ptr(q), _ptr(x), 1 if displacement else 0, _stream()), "eipc_embed")
        return x

    def build_candidates(self, q, out: Optional[PairList] = None) -> PairList:
        pr = out if out is not None else self.new_pairs()
        c = pr._c()
        _check(self.lib.eipc_build_candidates(self.handle, _ptr(q), ctypes.byref(self.params), ctypes.byref(c), _stream()),
               "eipc_build_candidates")
        return pr

    def friction_lag(self, q_n, pairs_n: PairList, out: Optional[LagState] = None) -> LagState:
        lag = out if out is not None else self.new_lag()
        pc, lc = pairs_n._c(), lag._c()
        _check(self.lib.eipc_friction_lag(self.handle, _ptr(q_n), ctypes.byref(pc), ctypes.byref(self.params),
                                          ctypes.byref(lc), _stream()), "eipc_friction_lag")
        return lag

    def eval_contact(self, q, pairs: PairList, lag: Optional[LagState] = None, E=None, g_r=None, H: Optional[BSR] = None,
                     project: bool = True):
        """(E, g_r, H_r); project=False returns the exact Hessian instead of the
        projected-Newton one."""
        import torch
        E = E if E is not None else torch.zeros(1, dtype=torch.float64, device=self.device)
        g_r = g_r if g_r is not None else torch.zeros((self.Ns, 3), dtype=torch.float64, device=self.device)
        H = H if H is not None else self.new_bsr()
        pc, hc = pairs._c(), H._c()
        lp = ctypes.byref(lag._c()) if lag is not None else None
        prm = self.params
        if not project:
            prm = Params(*[getattr(self.params, f) for f, _ in Params._fields_])
            prm.flags = self.params.flags | 1
        _check(self.lib.eipc_eval_contact(self.handle, _ptr(q), ctypes.byref(pc), lp, ctypes.byref(prm), _ptr(E),
                                          _ptr(g_r), ctypes.byref(hc), _stream()), "eipc_eval_contact")
        return E, g_r, H

    def contact_hvp(self, q, pairs: PairList, v, lag: Optional[LagState] = None, kin_dir=None, out=None,
                    out_kin=None):
        """Exact (unprojected) contact Hessian applied to the reduced direction v [Ns,3],
        with the kinematic vertices moving along kin_dir (3 floats, or None).  Returns
        (J^T H u [Ns,3], sum of H u over the kinematic vertices [3])."""
        import torch
        out = out if out is not None else torch.empty((self.Ns, 3), dtype=torch.float64, device=self.device)
        out_kin = out_kin if out_kin is not None else torch.empty(3, dtype=torch.float64, device=self.device)
        kd = None
        if kin_dir is not None:
            kd_arr = (ctypes.c_double * 3)(*[float(c) for c in kin_dir])
            kd = ctypes.cast(kd_arr, ctypes.c_void_p)
        pc = pairs._c()
        lp = ctypes.byref(lag._c()) if lag is not None else None
        _check(self.lib.eipc_contact_hvp(self.handle, _ptr(q), ctypes.byref(pc), lp, ctypes.byref(self.params), _ptr(v),
                                         kd, _ptr(out), _ptr(out_kin), _stream()), "eipc_contact_hvp")
        return out, out_kin

    def set_kinematic(self, x_kin):
        """New positions of the kinematic vertices (device f64 [Nv,3]; other rows ignored)."""
        _check(self.lib.eipc_scene_set_kinematic(self.handle, _ptr(x_kin), _stream()), "eipc_scene_set_kinematic")

    def set_mollifier(self, x_rest=None, factor: float = 1e-3):
        """EE mollifier with eps_x = factor |e_i|^2 |e_j|^2 at the rest positions x_rest
        ([Nv,3], moved to the device); x_rest None turns it off."""
        import torch
        if x_rest is None:
            _check(self.lib.eipc_scene_set_mollifier(self.handle, None, 0.0, _stream()), "eipc_scene_set_mollifier")
            return
        xr = torch.as_tensor(x_rest, dtype=torch.float64, device=self.device).contiguous()
        _check(self.lib.eipc_scene_set_mollifier(self.handle, _ptr(xr), float(factor), _stream()),
               "eipc_scene_set_mollifier")

    def candidates(self, capacity: Optional[int] = None):
        """The broad-phase candidate list of the last build_candidates or accd_toi call, as
        device int32 tensors (type, i, j) (eipc_candidates_read; synchronises once to size
        the result)."""
        import torch
        n = torch.zeros(1, dtype=torch.int64, device=self.device)
        _check(self.lib.eipc_candidates_read(self.handle, None, None, None, 0, _ptr(n), _stream()),
               "eipc_candidates_read")
        m = int(n.item()) if capacity is None else int(capacity)
        out = [torch.empty(max(m, 1), dtype=torch.int32, device=self.device) for _ in range(3)]
        _check(self.lib.eipc_candidates_read(self.handle, _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), m, _ptr(n),
                                             _stream()), "eipc_candidates_read")
        k = min(m, int(n.item()))
        return out[0][:k], out[1][:k], out[2][:k]

    def set_dedup(self, on: bool = True):
        """Deduplicated contact sets from build_candidates (EIPC_PARAM_DEDUP)."""
        self.params.flags = (self.params.flags | 2) if on else (self.params.flags & ~2)

    def set_params(self, **kw):
        """Change contact parameters (dhat, kappa, mu, eps_v, h, accd_s, accd_max_iter)."""
        for k, v in kw.items():
            setattr(self.params, k, type(getattr(self.params, k))(v))

    def accd_toi(self, x, dx, alpha=None, n_candidates=None):
        import torch
        alpha = alpha if alpha is not None else torch.zeros(1, dtype=torch.float64, device=self.device)
        nc = _ptr(n_candidates) if n_candidates is not None else None
        _check(self.lib.eipc_accd_toi(self.handle, _ptr(x), _ptr(dx), ctypes.byref(self.params), _ptr(alpha), nc,
                                      _stream()), "eipc_accd_toi")
        return alpha

    def set_rebuild_interval(self, n: int):
        """Full LBVH rebuild every n-th build_candidates call, refit in between."""
        _check(self.lib.eipc_set_rebuild_interval(self.handle, int(n)), "eipc_set_rebuild_interval")

    def set_groups(self, vertex_group, n_groups: int):
        """Split the scene into n_groups independent scenes: vertex_group (host int32 [Nv])
        holds each vertex's scene id.  Pairs never join two groups, and E and alpha are
        reported per group by group_energy / group_alpha."""
        vg = np.ascontiguousarray(vertex_group, np.int32)
        if vg.shape != (self.Nv,):
            raise ValueError("vertex_group must have one entry per vertex")
        _check(self.lib.eipc_scene_set_groups(self.handle, vg.ctypes.data, int(n_groups)), "eipc_scene_set_groups")
        self.n_groups = int(n_groups)

    def group_energy(self, out=None):
        """Per-group energy of the last eval_contact call (device f64 [n_groups])."""
        import torch
        out = out if out is not None else torch.zeros(getattr(self, "n_groups", 1), dtype=torch.float64,
                                                      device=self.device)
        _check(self.lib.eipc_group_energy(self.handle, _ptr(out), _stream()), "eipc_group_energy")
        return out

    def group_alpha(self, out=None):
        """Per-group step bound of the last accd_toi call (device f64 [n_groups])."""
        import torch
        out = out if out is not None else torch.zeros(getattr(self, "n_groups", 1), dtype=torch.float64,
                                                      device=self.device)
        _check(self.lib.eipc_group_alpha(self.handle, _ptr(out), _stream()), "eipc_group_alpha")
        return out

    LAUNCH_KERNELS = {"eval_barrier": 0, "bvh_query": 1, "bvh_refit": 2, "eval_tile": 3, "ccd_tile": 4}

    def set_launch(self, kernel: str, threads: int, blocks_per_sm: int, variant: int = 2):
        """Launch shape of a tunable kernel; results do not depend on it."""
        _check(self.lib.eipc_set_launch(self.handle, self.LAUNCH_KERNELS[kernel], int(threads), int(blocks_per_sm),
                                        int(variant)), "eipc_set_launch")

    N_TIMERS = 14

    def timing_enable(self, names=None):
        """Brackets every launch of the named kernels (all if None, none if []) with CUDA
        events on the launching stream."""
        mask = 0
        for k in range(self.N_TIMERS):
            if names is None or self.lib.eipc_kernel_name(k).decode() in names:
                mask |= 1 << k
        _check(self.lib.eipc_timing_enable(self.handle, mask), "eipc_timing_enable")

    def timing_read(self) -> dict:
        ms = np.zeros(self.N_TIMERS)
        n = np.zeros(self.N_TIMERS, np.int64)
        _check(self.lib.eipc_timing_read(self.handle, ms.ctypes.data, n.ctypes.data, self.N_TIMERS), "eipc_timing_read")
        return {self.lib.eipc_kernel_name(k).decode(): (float(ms[k]), int(n[k])) for k in range(self.N_TIMERS) if n[k]}

    def status(self) -> dict:
        flags = ctypes.c_int32(0)
        need = np.zeros(4, np.int64)
        it = np.zeros(1, np.int64)
        _check(self.lib.eipc_status_read(self.handle, _stream(), ctypes.byref(flags), need.ctypes.data, it.ctypes.data),
               "eipc_status_read")
        names = [n for b, n in FLAGS.items() if flags.value & b]
        return dict(flags=int(flags.value), names=names, needed=need.tolist(), accd_iters=int(it[0]))

    def work_counts(self) -> dict:
        """Work counts of the last calls (eipc_work_counts), by name."""
        out = np.zeros(len(WORK_COUNTS), np.int64)
        _check(self.lib.eipc_work_counts(self.handle, _stream(), out.ctypes.data, len(WORK_COUNTS)), "eipc_work_counts")
        return dict(zip(WORK_COUNTS, out.tolist()))


WORK_COUNTS = ("candidates", "screened", "pairs", "items", "hessian_records", "gradient_records", "hessian_blocks",
               "gradient_nodes", "ccd_advanced")


def fp64_peak(iters: int = 1 << 16, repeats: int = 5) -> dict:
    """Measured FP64 rate of the current device (eipc_fp64_probe): the best of `repeats`
    launches timed with CUDA events on the current stream, in TFLOP/s."""
    import torch
    L = load()
    sink = torch.zeros(152 * 4 * 256, dtype=torch.float64, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    best = None
    _check(L.eipc_fp64_probe(1024, _ptr(sink), _stream()), "eipc_fp64_probe")     # warm-up
    for _ in range(repeats):
        ev[0].record()
        _check(L.eipc_fp64_probe(int(iters), _ptr(sink), _stream()), "eipc_fp64_probe")
        ev[1].record()
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1])
        best = ms if best is None else min(best, ms)
    flops = L.eipc_fp64_probe_flops(int(iters))
    return dict(tflops=flops / (best / 1e3) / 1e12, ms=best, flops=int(flops), iters=int(iters))


def set_programmatic_launch(on: bool = True):
    """Process-wide launch mode of the library's kernels (eipc_set_programmatic_launch):
    programmatic dependent launch (the default) or plain stream order."""
    load().eipc_set_programmatic_launch(1 if on else 0)


def bsr_spmv(row_ptr, col, val, x, out=None, alpha: float = 1.0, beta: float = 0.0):
    """y = alpha A x + beta y for a 3x3-block CSR matrix (device tensors; x, y [n,3])."""
    import torch
    L = load()
    n = row_ptr.shape[0] - 1
    y = out if out is not None else torch.zeros_like(x)
    _check(L.eipc_bsr_spmv(n, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(x), float(alpha), float(beta), _ptr(y), _stream()),
           "eipc_bsr_spmv")
    return y


# -------------------------------------------------------------- functional front end
_scene_cache: dict = {}


def _scene_for(scene) -> ContactScene:
    key = id(scene)
    cs = _scene_cache.get(key)
    if cs is None or cs.scene is not scene:
        cs = ContactScene(scene)
        _scene_cache[key] = cs
    return cs


def build_candidates(scene, q):
    """Contact pairs of `scene` at reduced coordinates q (torch CUDA f64 [Ns,3])."""
    return _scene_for(scene).build_candidates(q)


def eval_contact(q, scene, lag=None, pairs=None):
    """(E, g_r, H_r) at reduced coordinates q.  `scene` carries W (cage_idx, w), the
    surface (tris, edges) and dhat, kappa, mu in scene.params."""
    cs = _scene_for(scene)
    pr = pairs if pairs is not None else cs.build_candidates(q)
    return cs.eval_contact(q, pr, lag)


def accd_toi(scene, x, dx):
    """Step bound alpha for the full-space motion x + t dx (torch CUDA f64 [Nv,3])."""
    return _scene_for(scene).accd_toi(x, dx)
