"""eipc_accd_toi_static -- the CCD step bound for callers that cannot allocate device
memory (code whose device memory is owned by another framework's allocator, or a control
loop that cannot take the synchronisation of an allocation) -- against the scene-based
eipc_accd_toi, through the C ABI.

The static entry point keeps its scratch in a fixed array inside the library, so the
test calls it twice in a row with different motions: each call must start from clean
scratch and agree with the scene-based bound."""
import ctypes

import numpy as np
import pytest

from paper_2409_16385_gb300 import binding, scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

def _small_scene():
    return scenes.sphere_on_pad(seed=3, level=1, pad_cells=8, cage_cubes=2)


def _all_candidates(sc):
    """Every PT and EE pair that shares no vertex and is not all kinematic: a superset of
    the pairs whose swept boxes overlap."""
    kin = sc.kinematic
    tris, edges = sc.tris, sc.edges
    v = np.arange(sc.Nv)[:, None]
    f = np.arange(sc.F)[None, :]
    inc = (tris[None, :, 0] == v) | (tris[None, :, 1] == v) | (tris[None, :, 2] == v)
    allk = kin[:, None] & kin[tris].all(1)[None, :]
    vi, fj = np.nonzero(~inc & ~allk)
    e = np.arange(sc.E)
    a, b = np.meshgrid(e, e, indexing="ij")
    up = a < b
    ea, eb = edges[a], edges[b]
    share = (ea[..., 0] == eb[..., 0]) | (ea[..., 0] == eb[..., 1]) | (ea[..., 1] == eb[..., 0]) | (ea[..., 1] == eb[..., 1])
    ek = kin[edges].all(1)
    allk_e = ek[a] & ek[b]
    ei, ej = np.nonzero(up & ~share & ~allk_e)
    ctype = np.concatenate([np.zeros(len(vi), np.int32), np.ones(len(ei), np.int32)])
    ci = np.concatenate([vi, ei]).astype(np.int32)
    cj = np.concatenate([fj, ej]).astype(np.int32)
    del f
    return ctype, ci, cj


def _static_call(lib, sc, x, dx, tris_d, edges_d, cand, params):
    P = ctypes.c_void_p
    lib.eipc_accd_toi_static.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, P, P, P, P, ctypes.c_int64,
                                         P, P, P, ctypes.POINTER(binding.Params), P, P, P, P]
    lib.eipc_accd_toi_static.restype = ctypes.c_int32
    alpha = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    flags = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    nadv = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    ct, ci, cj = cand
    rc = lib.eipc_accd_toi_static(sc.Nv, sc.F, sc.E, x.data_ptr(), dx.data_ptr(), tris_d.data_ptr(), edges_d.data_ptr(),
                                  ct.shape[0], ct.data_ptr(), ci.data_ptr(), cj.data_ptr(), ctypes.byref(params),
                                  alpha.data_ptr(), flags.data_ptr(), nadv.data_ptr(),
                                  P(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    return alpha.item(), int(flags.item()), int(nadv.item())


def test_static_ccd_matches_scene_ccd_on_two_calls_in_a_row():
    from paper_2409_16385_gb300 import ContactScene
    sc = _small_scene()
    cs = ContactScene(sc, pair_capacity=1 << 12, bsr_capacity=1 << 12)
    lib = binding.load()
    params = binding.make_params(sc.params)
    dev = "cuda"
    q = torch.tensor(sc.iterate(0), dtype=torch.float64, device=dev)
    x = cs.embed(q)
    tris_d = torch.tensor(sc.tris, dtype=torch.int32, device=dev)
    edges_d = torch.tensor(sc.edges, dtype=torch.int32, device=dev)
    cand = tuple(torch.tensor(c, device=dev) for c in _all_candidates(sc))
    results = []
    for scale in (1.0, 0.6):
        dx = cs.embed(torch.tensor(scale * sc.dq(0), dtype=torch.float64, device=dev), displacement=True)
        nc = torch.zeros(1, dtype=torch.int64, device=dev)
        a_scene = cs.accd_toi(x, dx, n_candidates=nc).item()
        st = cs.status()
        assert st["flags"] == 0, st
        a_static, flags, nadv = _static_call(lib, sc, x, dx, tris_d, edges_d, cand, params)
        assert flags == 0
        # same FP64 advancement and the same exact minimum over the same overlapping
        # pairs: the two bounds are the same double, bit for bit
        assert np.float64(a_static).tobytes() == np.float64(a_scene).tobytes(), (scale, a_static, a_scene)
        assert nadv == int(nc.item())
        results.append(a_static)
    assert results[0] < 1.0 and results[0] != results[1]


def test_static_ccd_rejects_too_many_vertices():
    lib = binding.load()
    lib.eipc_accd_static_max_vertices.restype = ctypes.c_int64
    nmax = lib.eipc_accd_static_max_vertices()
    assert nmax == 131072
    params = binding.make_params(scenes.DEFAULT_PARAMS)
    P = ctypes.c_void_p
    lib.eipc_accd_toi_static.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, P, P, P, P, ctypes.c_int64,
                                         P, P, P, ctypes.POINTER(binding.Params), P, P, P, P]
    lib.eipc_accd_toi_static.restype = ctypes.c_int32
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = lib.eipc_accd_toi_static(nmax + 1, 0, 0, dummy.data_ptr(), dummy.data_ptr(), None, None, 0, None, None, None,
                                  ctypes.byref(params), dummy.data_ptr(), None, None, None)
    assert rc == -4
