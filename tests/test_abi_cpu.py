"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports
every function declared in include/*.h, and rejects bad arguments before any
CUDA call (no GPU needed)."""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

import paper_1307_2265_gb300 as ez

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(enzo_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    names = _declared()
    for must in ("enzo_ppm_sweep", "enzo_riemann_solve", "enzo_timestep_cfl", "enzo_step",
                 "enzo_ghost_fill_periodic", "enzo_workspace_size", "enzo_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol():
    path = ez._build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = sorted(n for n in _declared() if n not in exported)
    assert not missing, missing
    L = ez.lib()
    for n in _declared():
        assert hasattr(L, n)


def test_null_and_bad_arguments_rejected_without_gpu():
    L = ez.lib()
    p = ez.Params().c()
    assert L.enzo_ppm_sweep(None, 0, 0.1, 0, ctypes.byref(p)) == -1
    b = ez._Batch()
    b.npatch = -1
    assert L.enzo_ppm_sweep(ctypes.byref(b), 0, 0.1, 0, ctypes.byref(p)) == -1
    b.npatch = 0
    assert L.enzo_ppm_sweep(ctypes.byref(b), 0, 0.1, 0, ctypes.byref(p)) == 0      # empty batch: no-op
    bad = ez.Params(gamma=1.0).c()
    assert L.enzo_ppm_sweep(ctypes.byref(b), 0, 0.1, 0, ctypes.byref(bad)) == -1
    bad = ez.Params(precision=7).c()
    assert L.enzo_ppm_sweep(ctypes.byref(b), 0, 0.1, 0, ctypes.byref(bad)) == -1
    b.npatch = 3
    assert L.enzo_ppm_sweep(ctypes.byref(b), 0, 0.1, 0, ctypes.byref(p)) == -1      # NULL arrays
    assert L.enzo_riemann_solve(None, ctypes.byref(p)) == -1
    assert L.enzo_workspace_size(4000) >= 4 * 4001
    assert ez.strerror(-3) == "patch descriptor out of range, or batch larger than a fixed limit"


def test_validate_patches_ranges():
    L = ez.lib()
    t = ez.patch_table([(8, 9, 10), (1, 1, 1)], [0, 14 * 15 * 16], [0.1, 0.1, 0.1])
    assert t["freg_all"][0] == -1 and t["freg_bnd"][1] == -1
    total = 14 * 15 * 16 + 7 * 7 * 7
    bad = ctypes.c_int32(0)
    assert L.enzo_validate_patches(t.ctypes.data, 2, total, ctypes.byref(bad)) == 0 and bad.value == -1
    assert L.enzo_validate_patches(t.ctypes.data, 2, total - 1, ctypes.byref(bad)) == -3 and bad.value == 1
    for field, val in (("ng", 2), ("n", (0, 4, 4)), ("n", (5000, 1, 1)), ("off", -1)):
        u = t.copy()
        u[field][0] = val
        assert L.enzo_validate_patches(u.ctypes.data, 2, total, ctypes.byref(bad)) == -3 and bad.value == 0
    u = t.copy()
    u["dx"][1] = (0.1, 0.0, 0.1)
    assert L.enzo_validate_patches(u.ctypes.data, 2, total, ctypes.byref(bad)) == -3 and bad.value == 1


def test_patch_struct_layout_matches_header():
    assert ez.PATCH_DTYPE.itemsize == 72
    assert ctypes.sizeof(ez._Batch) == 4 + 4 + 8 + 8 + 40 + 8 + 8 + 8 + 8 + 8 + 8


def test_boundary_conditions_rejected_without_gpu():
    L = ez.lib()
    b = ez._Batch()
    b.npatch = 0
    bad = (ctypes.c_int32 * 3)(0, 7, 0)
    good = (ctypes.c_int32 * 3)(ez.BC_REFLECT, ez.BC_OUTFLOW, ez.BC_PERIODIC)
    assert L.enzo_ghost_fill_boundary(ctypes.byref(b), bad) == -1
    assert L.enzo_ghost_fill_boundary(ctypes.byref(b), None) == -1
    assert L.enzo_ghost_fill_boundary(ctypes.byref(b), good) == 0       # empty batch: no-op
    p = ez.Params().c()
    assert L.enzo_step_boundary(ctypes.byref(b), ctypes.byref(p), 0, None, good) == -1   # no dt


def test_solver_selector_rejected_without_gpu():
    L = ez.lib()
    b = ez._Batch()
    b.npatch = 0
    assert L.enzo_ppm_sweep(ctypes.byref(b), 0, 0.1, 0, ctypes.byref(ez.Params(solver=ez.SOLVER_HLLC).c())) == 0
    assert L.enzo_ppm_sweep(ctypes.byref(b), 0, 0.1, 0, ctypes.byref(ez.Params(solver=5).c())) == -1
    fake_blob = ctypes.c_void_p(4096)          # never dereferenced: rejected before any launch
    p = ez.Params(precision=ez.FP32, guess=ez.GUESS_MLP, mlp=fake_blob.value, solver=ez.SOLVER_HLL).c()
    assert L.enzo_ppm_sweep(ctypes.byref(b), 0, 0.1, 0, ctypes.byref(p)) == -1


def test_reconstruction_options_rejected_without_gpu():
    L = ez.lib()
    b = ez._Batch()
    b.npatch = 0
    ok = ez.Params(options=ez.OPT_STEEPEN | ez.OPT_FLATTEN | ez.OPT_DIFFUSE).c()
    assert L.enzo_ppm_sweep(ctypes.byref(b), 0, 0.1, 0, ctypes.byref(ok)) == 0
    assert L.enzo_ppm_sweep(ctypes.byref(b), 0, 0.1, 0, ctypes.byref(ez.Params(options=16).c())) == -1
    p = ez.Params(precision=ez.FP32, guess=ez.GUESS_MLP, mlp=4096, options=ez.OPT_STEEPEN).c()
    assert L.enzo_ppm_sweep(ctypes.byref(b), 0, 0.1, 0, ctypes.byref(p)) == -1


def test_dual_energy_arguments_rejected_without_gpu():
    """OPT_DUAL needs the two-shock solver and a gas-energy field, and a batch
    with both a gas-energy field and flux registers (six components per face)
    needs OPT_DUAL; each is refused on the host before any launch (the fake
    device pointers below are never dereferenced)."""
    L = ez.lib()
    b = ez._Batch()
    b.npatch = 0
    dual = ez.Params(options=ez.OPT_DUAL)
    assert L.enzo_ppm_sweep(ctypes.byref(b), 0, 0.1, 0, ctypes.byref(dual.c())) == 0
    assert L.enzo_ppm_sweep(ctypes.byref(b), 0, 0.1, 0,
                            ctypes.byref(ez.Params(options=ez.OPT_DUAL, solver=ez.SOLVER_HLLC).c())) == -1
    b.npatch = 1
    b.patches = 4096
    b.field_len = 1000
    for i in range(5):
        b.U[i] = 8192 + 8192 * i
    b.workspace = 65536
    b.ws_bytes = int(L.enzo_workspace_size(1))
    b.status = 131072
    assert L.enzo_ppm_sweep(ctypes.byref(b), 0, 0.1, 0, ctypes.byref(dual.c())) == -1      # ge missing
    assert L.enzo_step(ctypes.byref(b), ctypes.byref(dual.c()), 0, ctypes.c_void_p(262144)) == -1
    b.ge = 524288
    b.freg = 1048576
    plain = ez.Params()
    assert L.enzo_ppm_sweep(ctypes.byref(b), 0, 0.1, 0, ctypes.byref(plain.c())) == -1     # registers, no option
    assert L.enzo_step(ctypes.byref(b), ctypes.byref(plain.c()), 0, ctypes.c_void_p(262144)) == -1
    assert L.enzo_ppm_sweep_noalloc(ctypes.byref(b), 0, 0.1, 0,
                                    ctypes.byref(ez.Params(options=ez.OPT_DUAL, solver=ez.SOLVER_HLL).c())) == -1


def test_fallback_modes_rejected_without_gpu():
    """fallback accepts 0, 1 and 2; mode 2 runs in the option kernels and not
    with the learned guess.  Refused on the host before any launch."""
    L = ez.lib()
    b = ez._Batch()
    b.npatch = 0
    for mode, want in ((0, 0), (1, 0), (2, 0), (3, -1), (-1, -1)):
        assert L.enzo_ppm_sweep(ctypes.byref(b), 0, 0.1, 0, ctypes.byref(ez.Params(fallback=mode).c())) == want
    p = ez.Params(precision=ez.FP32, guess=ez.GUESS_MLP, mlp=4096, fallback=2).c()
    assert L.enzo_ppm_sweep(ctypes.byref(b), 0, 0.1, 0, ctypes.byref(p)) == -1


def _fake_batch(ge):
    """A one-patch batch of fake device pointers (never dereferenced)."""
    b = ez._Batch()
    b.npatch = 1
    b.patches = 4096
    b.field_len = 1000
    for i in range(5):
        b.U[i] = 8192 + 8192 * i
    b.freg = 1048576
    b.ge = 524288 if ge else None
    return b


def test_hierarchy_gas_energy_pairing_rejected_without_gpu():
    """The hierarchy calls carry the gas energy only when every batch involved
    has it: a coarse/fine (or source/destination) pair where one side alone
    has ge, or a ghost fill of a level with ge whose parent's old ge is
    missing, is refused on the host before any launch."""
    from paper_1307_2265_gb300 import hierarchy as gh
    L = gh._lib()
    a, n = _fake_batch(True), _fake_batch(False)
    links, boxes = ctypes.c_void_p(2048), ctypes.c_void_p(3072)
    old = (ctypes.c_void_p * 5)(*[16384 + 8192 * i for i in range(5)])
    for x, y in ((a, n), (n, a)):
        assert L.enzo_flux_correct(ctypes.byref(x), links, ctypes.byref(y), links, boxes, 1, 0.1, 2, 0) == -1
        assert L.enzo_project(ctypes.byref(x), links, ctypes.byref(y), links, 2) == -1
        assert L.enzo_copy_level(ctypes.byref(x), links, ctypes.byref(y), links, boxes, 1) == -1
        assert L.enzo_ghost_fill_level(ctypes.byref(x), links, ctypes.byref(y), links, old, 32768, 0.5,
                                       boxes, 1, None, 0, 0, 2) == -1
    # ge on both levels, but no old ge of the parent for the interpolation
    assert L.enzo_ghost_fill_level(ctypes.byref(a), links, ctypes.byref(a), links, old, None, 0.5,
                                   boxes, 1, None, 0, 0, 2) == -1
    # no ge anywhere, yet an old ge given
    assert L.enzo_ghost_fill_level(ctypes.byref(n), links, ctypes.byref(n), links, old, 32768, 0.5,
                                   boxes, 1, None, 0, 0, 2) == -1


def test_pack_arguments_rejected_without_gpu():
    """enzo_pack_active / enzo_unpack_active refuse NULL packed arrays or
    offsets, and a packed gas energy for a batch without one, before any
    launch; an empty batch is a no-op."""
    L = ez.lib()
    b = _fake_batch(False)
    b.workspace = 65536
    b.ws_bytes = int(L.enzo_workspace_size(1))
    b.status = 131072
    packed = (ctypes.c_void_p * 5)(*[2 ** 20 + 8192 * i for i in range(5)])
    off = ctypes.c_void_p(4096)
    for fn in (L.enzo_pack_active, L.enzo_unpack_active):
        assert fn(ctypes.byref(b), packed, None, None) == -1
        assert fn(ctypes.byref(b), None, None, off) == -1
        assert fn(ctypes.byref(b), packed, ctypes.c_void_p(8192), off) == -1      # ge packed, batch has none
        e = ez._Batch()
        e.npatch = 0
        assert fn(ctypes.byref(e), packed, None, off) == 0
