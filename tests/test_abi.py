"""The C-ABI library loads and exports every entry point include/embipc.h declares (no
GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

from paper_2409_16385_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(eipc_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    d = _declared()
    for n in ("eipc_build_candidates", "eipc_eval_contact", "eipc_accd_toi", "eipc_scene_create",
              "eipc_friction_lag", "eipc_embed", "eipc_status_read"):
        assert n in d


def test_library_loads_and_exports_every_declared_symbol():
    build.build()
    lib = ctypes.CDLL(build.LIB)
    for n in _declared():
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    assert set(binding.EXPORTS) <= set(_declared())


def test_version_string():
    lib = binding.load()
    assert b"embipc" in lib.eipc_version()


def test_scene_create_rejects_bad_input_without_gpu_work():
    """Host-side validation: out-of-range ids are refused before any device call."""
    import numpy as np
    lib = binding.load()
    h = ctypes.c_void_p()
    tris = np.array([[0, 1, 5]], np.int32)          # vertex 5 does not exist
    edges = np.array([[0, 1], [0, 5], [1, 5]], np.int32)
    idx = np.full((3, 4), -1, np.int32)
    w = np.zeros((3, 4)); xk = np.zeros((3, 3))
    rc = lib.eipc_scene_create(3, 1, 3, 0, tris.ctypes.data, edges.ctypes.data, idx.ctypes.data, w.ctypes.data,
                               xk.ctypes.data, 0, 0, ctypes.byref(h))
    assert rc == -1 and not h.value
    rc = lib.eipc_scene_create(0, 0, 0, 0, None, None, None, None, None, 0, 0, ctypes.byref(h))
    assert rc == -1


def test_binding_refuses_to_run_without_cuda():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2409_16385_gb300 import ContactScene, scenes
    with pytest.raises(RuntimeError):
        ContactScene(scenes.make_config(1))


def test_entry_points_reject_misuse_without_gpu_work():
    """Host-detectable misuse returns EIPC_ERR_INVALID before any device call: a null scene,
    a count out of range, a launch shape outside the documented set, non-finite scalars."""
    import numpy as np
    lib = binding.load()
    INVALID = -1
    out = np.zeros(16, np.int64)
    assert lib.eipc_work_counts(None, None, out.ctypes.data, 9) == INVALID
    flags = ctypes.c_int32(0)
    need = np.zeros(4, np.int64)
    it = np.zeros(1, np.int64)
    assert lib.eipc_status_read(None, None, ctypes.byref(flags), need.ctypes.data, it.ctypes.data) == INVALID
    assert lib.eipc_set_launch(None, 0, 128, 8, 2) == INVALID
    assert lib.eipc_set_rebuild_interval(None, 4) == INVALID
    ms = np.zeros(16); n = np.zeros(16, np.int64)
    assert lib.eipc_timing_read(None, ms.ctypes.data, n.ctypes.data, 4) == INVALID
    x = np.zeros(3); y = np.zeros(3)
    rp = np.zeros(2, np.int32)
    assert lib.eipc_bsr_spmv(-1, rp.ctypes.data, None, None, x.ctypes.data, 1.0, 0.0, y.ctypes.data, None) == INVALID
    assert lib.eipc_bsr_spmv(1, rp.ctypes.data, None, None, x.ctypes.data, float("nan"), 0.0, y.ctypes.data,
                             None) == INVALID
    assert lib.eipc_bsr_spmv(1, None, None, None, x.ctypes.data, 1.0, 0.0, y.ctypes.data, None) == INVALID


def test_every_entry_point_is_documented():
    """Each declared entry point (or the group of declarations it belongs to) follows a
    comment that states what it computes and how its arguments are laid out."""
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        lines = open(os.path.join(ROOT, "include", f)).read().splitlines()
        for k, line in enumerate(lines):
            m = re.match(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(eipc_[a-z_0-9]+)\s*\(", line)
            if not m:
                continue
            j = k - 1
            # skip the other declarations of the same group (and their continuation lines)
            while j >= 0 and lines[j].strip() and not lines[j].rstrip().endswith("*/"):
                j -= 1
            assert j >= 0 and lines[j].rstrip().endswith("*/"), f"{m.group(1)} has no comment above it"
            start = j
            while start >= 0 and "/*" not in lines[start]:
                start -= 1
            words = " ".join(lines[start:j + 1]).split()
            assert len(words) >= 6, f"{m.group(1)}: comment too short"
