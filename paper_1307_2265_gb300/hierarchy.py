"""AMR hierarchy on the GPU (paper Sec. 3), run by the library's native driver
(enzo_hierarchy_*, csrc/driver.cu): the level plans, the EvolveLevel W-cycle
and the rebuild of the finer levels from flagged cells (Sec. 3.5, 3.6) are
host C++ in the library, every operation on the fields one of its kernels.
This module marshals arguments, views the levels' device state as tensors,
and exposes the plans and the rebuild's building blocks on their own.

Plans per level (again after a rebuild):
  * links: origin (global index of the first active cell) and parent index;
  * sibling copy boxes: every intersection of a patch's ghost-extended box with
    another patch's active box;
  * interpolated ghost regions: the 26 regions around each patch that no single
    sibling covers (the copies that follow overwrite what siblings do cover);
  * flux-correction face parts: the cells outside each fine face, per coarse
    patch holding them, in waves so that corrections meeting in one coarse
    cell add in a fixed order;
  * flux registers: all-face registers for patches with children, boundary-face
    registers for patches with a parent.
sibling_boxes / interp_boxes / correction_faces are the lattice versions of the
same plans for the tensor-product tilings of synth.hierarchy_layout, kept as an
independent check of the library's general ones.

W-cycle of one root step (EvolveLevel of Sec. 3):
  fill ghosts; dt = min(CFL, t_parent - t); save the old state if the level has
  children; three sweeps (recording fluxes); t += dt; if children: fill ghosts
  at the new time, zero the children's boundary registers, advance the children
  to t, flux correction, projection, and (with a rebuild) new finer levels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import PATCH_DTYPE, STATUS_WORDS, PatchBatch, Params, _Batch, _check, lib

NG = 3
LINK_DTYPE = np.dtype([("origin", "<i4", (3,)), ("parent", "<i4")])
BOX_DTYPE = np.dtype([("dst", "<i4"), ("src", "<i4"), ("lo", "<i4", (3,)), ("hi", "<i4", (3,))])
FACE_DTYPE = np.dtype([("fine", "<i4"), ("dir", "<i4"), ("side", "<i4"), ("target", "<i4"),
                       ("lo", "<i4", (2,)), ("hi", "<i4", (2,))])
FLAG_SLOPE, FLAG_SHOCK, FLAG_MASS = 1, 2, 4


class _FlagParams(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("slope", ctypes.c_double), ("shock_dp", ctypes.c_double),
                ("shock_e", ctypes.c_double), ("mass", ctypes.c_double), ("precision", ctypes.c_int32)]


class _ClusterParams(ctypes.Structure):
    _fields_ = [("efficiency", ctypes.c_double), ("small_cells", ctypes.c_int32), ("buffer", ctypes.c_int32),
                ("margin", ctypes.c_int32)]


class _Box(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int32 * 3), ("hi", ctypes.c_int32 * 3)]


def _lib():
    L = lib()
    if not getattr(L, "_hier_ready", False):
        vp, i32, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
        L.enzo_ghost_fill_level.argtypes = [vp, vp, vp, vp, vp, vp, d, vp, i32, vp, i32, i32, i32]
        L.enzo_flux_correct.argtypes = [vp, vp, vp, vp, vp, i32, d, i32, i32]
        L.enzo_project.argtypes = [vp, vp, vp, vp, i32]
        L.enzo_copy_level.argtypes = [vp, vp, vp, vp, vp, i32]
        L.enzo_flag_cells.argtypes = [vp, vp, vp, vp]
        L.enzo_cluster_flags.argtypes = [vp, vp, vp, vp, i32, vp]
        L.enzo_plan_level.argtypes = [vp, vp, i32, vp, i32, vp, vp, i32, vp]
        L.enzo_plan_correction.argtypes = [vp, vp, i32, vp, vp, i32, vp, vp, i32, vp]
        L.enzo_hierarchy_create.argtypes = [vp, i32, d, i32, vp, vp, vp, vp]
        L.enzo_hierarchy_destroy.argtypes = [vp]
        L.enzo_hierarchy_nlevel.argtypes = [vp]
        L.enzo_hierarchy_level.argtypes = [vp, i32, vp]
        L.enzo_hierarchy_root_step.argtypes = [vp, vp, vp, vp, vp]
        L.enzo_hierarchy_rebuild.argtypes = [vp, i32, vp, vp, i32, vp]
        L.enzo_hierarchy_step_to.argtypes = [vp, d, vp, vp, vp]
        L.enzo_hierarchy_take_log.argtypes = [vp, vp, vp, i32, vp]
        L.enzo_hierarchy_timing.argtypes = [vp, i32, vp, vp]
        for n in ("enzo_ghost_fill_level", "enzo_flux_correct", "enzo_project", "enzo_copy_level",
                  "enzo_flag_cells", "enzo_cluster_flags", "enzo_plan_level", "enzo_plan_correction",
                  "enzo_hierarchy_create", "enzo_hierarchy_destroy", "enzo_hierarchy_nlevel",
                  "enzo_hierarchy_level", "enzo_hierarchy_root_step", "enzo_hierarchy_rebuild",
                  "enzo_hierarchy_take_log", "enzo_hierarchy_timing", "enzo_hierarchy_step_to"):
            getattr(L, n).restype = ctypes.c_int
        L._hier_ready = True
    return L


class _Grid:
    """Patch lookup of a level: patches start at per-axis start positions, and a
    dense table over the start indices maps each start corner to its patch."""

    def __init__(self, n, origin):
        self.n, self.origin = np.asarray(n), np.asarray(origin)
        self.starts = [np.unique(self.origin[:, a]) for a in range(3)]
        k = [np.searchsorted(self.starts[a], self.origin[:, a]) for a in range(3)]
        self.cube = np.full([len(st) for st in self.starts], -1, dtype=np.int64)
        self.cube[k[0], k[1], k[2]] = np.arange(len(self.origin))

    def find_many(self, g):
        """Patch whose active box contains each global cell g[m] (array [M, 3]), or -1."""
        g = np.asarray(g).reshape(-1, 3)
        k = [np.searchsorted(self.starts[a], g[:, a], side="right") - 1 for a in range(3)]
        ok = (k[0] >= 0) & (k[1] >= 0) & (k[2] >= 0)
        i = np.full(len(g), -1, dtype=np.int64)
        i[ok] = self.cube[k[0][ok], k[1][ok], k[2][ok]]
        hit = i >= 0
        lo, hi = self.origin[i[hit]], self.origin[i[hit]] + self.n[i[hit]]
        inside = np.all((lo <= g[hit]) & (g[hit] < hi), axis=1)
        i[np.flatnonzero(hit)[~inside]] = -1
        return i

    def find(self, g):
        """Patch whose active box contains global cell g, or -1."""
        return int(self.find_many(np.asarray(g)[None, :])[0])


_DIRS = np.array([(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                  if (dx, dy, dz) != (0, 0, 0)])


def _probe(lo, hi, d):
    """Cell just outside the active box [lo, hi) in direction d (per patch)."""
    return np.where(d < 0, lo - 1, np.where(d > 0, hi, lo))


def _boxes(dst, src, blo, bhi):
    t = np.zeros(len(dst), dtype=BOX_DTYPE)
    t["dst"], t["src"] = dst, src
    t["lo"], t["hi"] = blo, bhi
    return t


def sibling_boxes(n, origin):
    """Copy boxes (dst, src, lo, hi) of ghost cells lying in siblings' active
    boxes.  Ghost layers (3 cells) are thinner than any patch, so only the 26
    neighbours across faces, edges and corners can meet a patch's ghost region."""
    n, origin = np.asarray(n), np.asarray(origin)
    grid = _Grid(n, origin)
    lo, hi = origin, origin + n
    P = len(n)
    pairs = []
    for d in _DIRS:
        b = grid.find_many(_probe(lo, hi, d))
        a = np.flatnonzero(b >= 0)
        pairs.append(np.stack([a, b[a]], axis=1))
    pairs = np.unique(np.concatenate(pairs), axis=0) if P else np.zeros((0, 2), dtype=np.int64)
    a, b = pairs[:, 0], pairs[:, 1]
    blo = np.maximum(lo[a] - NG, origin[b])
    bhi = np.minimum(hi[a] + NG, origin[b] + n[b])
    keep = np.all(blo < bhi, axis=1)
    return _boxes(a[keep], b[keep], blo[keep], bhi[keep])


def interp_boxes(n, origin):
    """Ghost regions (of the 26 around each patch: faces, edges, corners) that no
    sibling covers; these are interpolated from the parent."""
    n, origin = np.asarray(n), np.asarray(origin)
    grid = _Grid(n, origin)
    lo, hi = origin, origin + n
    out = []
    for d in _DIRS:
        blo = np.where(d < 0, lo - NG, np.where(d > 0, hi, lo))
        bhi = np.where(d < 0, lo, np.where(d > 0, hi + NG, hi))
        touched = grid.find_many(_probe(lo, hi, d)) >= 0
        # a sibling touching a region must cover all of it (tensor-product tiling)
        corner = np.where(d >= 0, bhi - 1, blo)
        if np.any(grid.find_many(corner[touched]) < 0):
            raise ValueError("ghost region partly covered by siblings")
        a = np.flatnonzero(~touched)
        out.append((a, blo[a], bhi[a]))
    a = np.concatenate([o[0] for o in out])
    order = np.argsort(a, kind="stable")
    return _boxes(a[order], a[order], np.concatenate([o[1] for o in out])[order],
                  np.concatenate([o[2] for o in out])[order])


def correction_faces(fine, coarse, r=2):
    """Faces of fine patches whose outside coarse cells are not covered by the
    fine level, with the coarse patch holding those cells."""
    fn, fo = np.asarray(fine["n"]), np.asarray(fine["origin"])
    cn, co = np.asarray(coarse["n"]), np.asarray(coarse["origin"])
    fgrid = _Grid(fn, fo)
    cgrid = _Grid(cn, co)
    cols = []
    for d in range(3):
        for side in (0, 1):
            probe = fo.copy()
            probe[:, d] = fo[:, d] - 1 if side == 0 else fo[:, d] + fn[:, d]
            i = np.flatnonzero(fgrid.find_many(probe) < 0)
            cell = probe[i] // r
            t = cgrid.find_many(cell)
            if np.any(t < 0):
                raise ValueError("coarse cell outside a fine face is not in a coarse patch")
            last = (fo[i] + fn[i]) // r - 1
            last[:, d] = cell[:, d]
            if not np.all((co[t] <= last) & (last < co[t] + cn[t])):
                raise ValueError("a fine face spans more than one coarse patch")
            cols.append(np.stack([i, np.full_like(i, d), np.full_like(i, side), t], axis=1))
    f = np.concatenate(cols) if cols else np.zeros((0, 4), dtype=np.int64)
    f = f[np.lexsort((f[:, 2], f[:, 1], f[:, 0]))]
    t = np.zeros(len(f), dtype=FACE_DTYPE)
    t["fine"], t["dir"], t["side"], t["target"] = f[:, 0], f[:, 1], f[:, 2], f[:, 3]
    a1 = np.where(f[:, 1] == 0, 1, 0)
    a2 = np.where(f[:, 1] == 2, 1, 2)
    t["hi"][:, 0] = fn[f[:, 0], a1] // r
    t["hi"][:, 1] = fn[f[:, 0], a2] // r
    return t


def _layout_arrays(n, origin):
    n = np.ascontiguousarray(np.asarray(n, dtype=np.int32).reshape(-1, 3))
    origin = np.ascontiguousarray(np.asarray(origin, dtype=np.int32).reshape(-1, 3))
    return n, origin


def _level_plans(n, origin):
    """The library's level plans (enzo_plan_level): sibling copy boxes and the
    ghost regions to interpolate."""
    n, origin = _layout_arrays(n, origin)
    ns, ni = ctypes.c_int32(0), ctypes.c_int32(0)
    L = _lib()
    r = L.enzo_plan_level(n.ctypes.data, origin.ctypes.data, len(n), None, 0, ctypes.byref(ns), None, 0,
                          ctypes.byref(ni))
    if r not in (0, -3):
        _check(r, "enzo_plan_level")
    sib = np.zeros(ns.value, dtype=BOX_DTYPE)
    itp = np.zeros(ni.value, dtype=BOX_DTYPE)
    _check(L.enzo_plan_level(n.ctypes.data, origin.ctypes.data, len(n), sib.ctypes.data, len(sib),
                             ctypes.byref(ns), itp.ctypes.data, len(itp), ctypes.byref(ni)), "enzo_plan_level")
    return sib, itp


def sibling_boxes_general(n, origin):
    """sibling_boxes for any disjoint layout: every intersection of a patch's
    ghost-extended box with another patch's active box (the library's plan, the
    one its hierarchy driver uses)."""
    return _level_plans(n, origin)[0]


def interp_boxes_general(n, origin):
    """The 26 ghost regions of every patch, except those lying wholly in one
    sibling's active box; the sibling copies that follow overwrite the parts
    siblings cover (the order of Sec. 3.1).  The library's plan."""
    return _level_plans(n, origin)[1]


def correction_parts(fine, coarse, r=2):
    """Flux-correction face parts for any disjoint layouts, in the order
    (fine patch, axis, side), each part the cells outside one fine face that
    one coarse patch holds; faces whose outside cells the fine level covers
    entirely are left out (projection overwrites those cells).  Returns the
    parts and, for each, a wave: parts in one wave share no coarse cell, and a
    part that shares cells with earlier parts comes in a later wave, so the
    additions happen in the listed order.  The library's plan
    (enzo_plan_correction, refinement factor 2)."""
    if r != 2:
        raise ValueError("the library refines by 2")
    fn, fo = _layout_arrays(fine["n"], fine["origin"])
    cn, co = _layout_arrays(coarse["n"], coarse["origin"])
    L = _lib()
    cnt = ctypes.c_int32(0)
    rc = L.enzo_plan_correction(fn.ctypes.data, fo.ctypes.data, len(fn), cn.ctypes.data, co.ctypes.data, len(cn),
                                None, None, 0, ctypes.byref(cnt))
    if rc not in (0, -3):
        _check(rc, "enzo_plan_correction")
    out = np.zeros(cnt.value, dtype=FACE_DTYPE)
    wave = np.zeros(cnt.value, dtype=np.int32)
    _check(L.enzo_plan_correction(fn.ctypes.data, fo.ctypes.data, len(fn), cn.ctypes.data, co.ctypes.data,
                                  len(cn), out.ctypes.data, wave.ctypes.data, len(out), ctypes.byref(cnt)),
           "enzo_plan_correction")
    return out, wave.astype(np.int64)


def cluster_flags(flags, efficiency=0.3, small_cells=64, buffer=1, margin=0):
    """Boxes ((lo), (hi)) of active-cell indices (x, y, z), half-open, covering
    the flagged cells of one grid (host array (z, y, x), nonzero = flagged),
    grown by `buffer` cells and cleared within `margin` of the grid's edge, by
    the library's Berger-Rigoutsos clustering (Sec. 3.5)."""
    f = np.ascontiguousarray(flags, dtype=np.uint8)
    n = (ctypes.c_int32 * 3)(f.shape[2], f.shape[1], f.shape[0])
    cp = _ClusterParams(efficiency, small_cells, buffer, margin)
    cap = 256
    while True:
        arr = (_Box * cap)()
        nb = ctypes.c_int32(0)
        r = _lib().enzo_cluster_flags(f.ctypes.data, n, ctypes.byref(cp), arr, cap, ctypes.byref(nb))
        if r == -3 and nb.value > cap:          # ENZO_ERR_RANGE: more boxes than room
            cap = nb.value
            continue
        _check(r, "enzo_cluster_flags")
        return [(tuple(arr[i].lo), tuple(arr[i].hi)) for i in range(nb.value)]


_PINNED = {}   # pinned host buffers for the flags, by size (reused across rebuilds)


def flag_cells(batch, gamma, slope=0.3, shock_dp=0.33, shock_e=0.1, mass=0.0, precision=0):
    """Flags (host uint8, one array (z, y, x) per patch) of a batch's active
    cells by the library's flag kernel (Sec. 3.6; ENZO_FLAG_* bits); ghost
    zones must be filled, periodic-flagged patches wrap.  precision: FP64 (the
    ratios as the paper writes them) or FP32 (staged primitives, no division)."""
    import torch
    n = np.asarray(batch.table["n"], dtype=np.int64)
    cells = np.prod(n, axis=1)
    off = np.concatenate([[0], np.cumsum(cells)[:-1]]).astype(np.int64)
    stream = batch.stream if batch.stream is not None else torch.cuda.current_stream(batch.device)
    with torch.cuda.stream(stream):
        flags = torch.zeros(max(int(cells.sum()), 1), dtype=torch.uint8, device=batch.device)
        offd = torch.from_numpy(off).to(batch.device)
        fp = _FlagParams(gamma, slope, shock_dp, shock_e, mass, precision)
        b = batch.c()
        _check(_lib().enzo_flag_cells(ctypes.byref(b), ctypes.byref(fp), flags.data_ptr(), offd.data_ptr()),
               "enzo_flag_cells")
        pinned = _PINNED.get(flags.numel())
        if pinned is None:
            pinned = _PINNED[flags.numel()] = torch.empty(flags.numel(), dtype=torch.uint8, pin_memory=True)
        pinned.copy_(flags, non_blocking=True)
        stream.synchronize()
        host = pinned.numpy().copy()
    return [host[off[i]:off[i] + cells[i]].reshape(int(n[i][2]), int(n[i][1]), int(n[i][0]))
            for i in range(len(cells))]


def register_sizes(n, nc=5):
    """(all-face, boundary-face) register sizes in doubles of patches of sizes n,
    nc components per face (5, or 6 with the dual-energy gas energy)."""
    n = np.asarray(n, dtype=np.int64)
    nx, ny, nz = n[:, 0], n[:, 1], n[:, 2]
    all_f = ((nx + 1) * ny * nz + (ny + 1) * nx * nz + (nz + 1) * nx * ny) * nc
    bnd = 2 * (ny * nz + nx * nz + nx * ny) * nc
    return all_f, bnd


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class _Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("release", _FREE_FN), ("ctx", ctypes.c_void_p)]


class _LevelLayout(ctypes.Structure):
    _fields_ = [("npatch", ctypes.c_int32), ("n", ctypes.c_void_p), ("origin", ctypes.c_void_p),
                ("parent", ctypes.c_void_p)]


class _RebuildParams(ctypes.Structure):
    _fields_ = [("flag", _FlagParams), ("cluster", _ClusterParams), ("root_margin", ctypes.c_int32),
                ("nest", ctypes.c_int32)]


class _LevelInfo(ctypes.Structure):
    _fields_ = [("batch", _Batch), ("links", ctypes.c_void_p), ("table", ctypes.c_void_p),
                ("n", ctypes.c_void_p), ("origin", ctypes.c_void_p), ("parent", ctypes.c_void_p),
                ("dx", ctypes.c_double), ("t", ctypes.c_double), ("cells", ctypes.c_int64),
                ("freg_len", ctypes.c_int64), ("generation", ctypes.c_uint64)]


OPS = ("ghost_fill", "cfl", "save_old", "sweeps", "correct_project", "rebuild")   # ENZO_HOP_* order


class _TorchMemory:
    """Device memory of a hierarchy, taken from PyTorch's allocator on the
    hierarchy's stream, so that tensors can view the levels' state."""

    def __init__(self, device, stream):
        import torch
        self.torch, self.device, self.stream = torch, device, stream
        self.blocks = {}
        self._alloc = _ALLOC_FN(self._alloc_cb)
        self._free = _FREE_FN(self._free_cb)
        self.c = _Allocator(self._alloc, self._free, None)

    def _alloc_cb(self, nbytes, ctx):
        try:
            with self.torch.cuda.stream(self.stream):
                t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
            self.blocks[t.data_ptr()] = t
            return t.data_ptr()
        except Exception:           # the library sees NULL and reports ENZO_ERR_CUDA
            return None

    def _free_cb(self, ptr, ctx):
        self.blocks.pop(ptr, None)

    def view(self, ptr, dtype, count):
        return self.blocks[ptr].view(dtype)[:count]


def _host_array(addr, dtype, count):
    if count == 0 or not addr:
        return np.zeros(0, dtype=dtype)
    nbytes = count * np.dtype(dtype).itemsize
    return np.frombuffer((ctypes.c_char * nbytes).from_address(addr), dtype=dtype).copy()


class _LevelView(dict):
    """One level of a Hierarchy; its time ("t") is read from the driver on each
    access, so a view held across steps stays current."""

    def __init__(self, hier, l, data):
        super().__init__(data)
        self._hier, self._l = hier, l

    def __getitem__(self, key):
        if key == "t":
            return self._hier._time(self._l)
        return super().__getitem__(key)


class Hierarchy:
    """An AMR hierarchy run by the library's native driver (enzo_hierarchy_*:
    level plans, the EvolveLevel W-cycle of Sec. 3, rebuilds of Sec. 3.5, 3.6).
    This class marshals arguments and gives tensor views of the levels' state,
    whose device memory the driver takes from PyTorch's allocator."""

    def __init__(self, layout, fields, root_dx, device="cuda", stream=None, root_bc=None):
        """layout: per level {"n", "origin", "parent"} (synth.hierarchy_layout).
        fields: per level, per patch, the five ghost-zoned fields, or six with
        the gas energy of the dual-energy option (Sec. 4.1.1; every patch then
        carries it, it goes through every hierarchy operation, and the level
        sweeps need OPT_DUAL).  root_bc: external boundaries (bc_x, bc_y, bc_z)
        of the root grid (BC_PERIODIC, BC_REFLECT, BC_OUTFLOW; its ghosts are
        then filled before each step), or None: a periodic root that wraps
        inside its sweeps."""
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.root_dx = root_dx
        self.root_bc = None if root_bc is None else tuple(int(v) for v in root_bc)
        self.nf = len(fields[0][0])
        if self.nf not in (5, 6):
            raise ValueError("a patch has five fields, or six with the gas energy")
        keep, lays = [], []
        for L in layout:
            n = np.ascontiguousarray(np.asarray(L["n"], dtype=np.int32).reshape(-1, 3))
            o = np.ascontiguousarray(np.asarray(L["origin"], dtype=np.int32).reshape(-1, 3))
            par = np.ascontiguousarray(np.asarray(L["parent"], dtype=np.int32).reshape(-1))
            keep += [n, o, par]
            lays.append(_LevelLayout(len(n), n.ctypes.data, o.ctypes.data, par.ctypes.data))
        arr = (_LevelLayout * len(lays))(*lays)
        bc = (ctypes.c_int32 * 3)(*self.root_bc) if self.root_bc is not None else None
        self._mem = _TorchMemory(self.device, self.stream)
        self._h = ctypes.c_void_p()
        self._views = {}
        self._timing = None
        with torch.cuda.device(self.device):
            _check(_lib().enzo_hierarchy_create(arr, len(lays), float(root_dx), self.nf, bc,
                                                self.stream.cuda_stream, ctypes.byref(self._mem.c),
                                                ctypes.byref(self._h)), "enzo_hierarchy_create")
        with torch.cuda.stream(self.stream):
            for l, lev in enumerate(self.levels):
                targets = self._fields(lev["batch"])
                for f, u in enumerate(targets):
                    flat = np.zeros(int(u.numel()))
                    for i, t in enumerate(lev["table"]):
                        blk = np.asarray(fields[l][i][f], dtype=np.float64).ravel()
                        flat[int(t["off"]):int(t["off"]) + blk.size] = blk
                    u.copy_(torch.from_numpy(flat))
        self.stream.synchronize()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                _lib().enzo_hierarchy_destroy(h)
            except Exception:
                pass
            self._h = None

    def _fields(self, batch):
        """The fields a hierarchy operation carries: U, and ge with dual energy."""
        return list(batch.U) + ([batch.ge] if self.nf == 6 else [])

    # -- views of the driver's levels ------------------------------------------
    def _level(self, l):
        torch = self.torch
        info = _LevelInfo()
        _check(_lib().enzo_hierarchy_level(self._h, l, ctypes.byref(info)), "enzo_hierarchy_level")
        b = info.batch
        npatch = int(b.npatch)
        key = (l, int(info.generation), b.U[0])
        batch = self._views.get(key)
        if batch is None:
            m = self._mem
            flen = int(b.field_len)
            table = _host_array(info.table, PATCH_DTYPE, npatch)
            batch = PatchBatch.wrap(
                table, [m.view(b.U[f], torch.float64, flen) for f in range(5)],
                m.view(b.patches, torch.uint8, 72 * npatch), m.view(b.workspace, torch.uint8, int(b.ws_bytes)),
                int(b.ws_bytes), m.view(b.status, torch.int64, STATUS_WORDS), self.stream,
                freg=m.view(b.freg, torch.float64, int(info.freg_len)) if b.freg else None,
                ge=m.view(b.ge, torch.float64, flen) if b.ge else None)
            self._views = {k: v for k, v in self._views.items() if k[0] != l}
            self._views[key] = batch
        n = _host_array(info.n, np.int32, 3 * npatch).reshape(-1, 3).astype(np.int64)
        origin = _host_array(info.origin, np.int32, 3 * npatch).reshape(-1, 3).astype(np.int64)
        parent = _host_array(info.parent, np.int32, npatch).astype(np.int64)
        return _LevelView(self, l, {"batch": batch, "n": n, "origin": origin, "parent": parent, "dx": info.dx,
                                    "table": batch.table, "cells": int(info.cells), "links": info.links})

    def _time(self, l):
        info = _LevelInfo()
        _check(_lib().enzo_hierarchy_level(self._h, l, ctypes.byref(info)), "enzo_hierarchy_level")
        return info.t

    @property
    def levels(self):
        """Per level: its batch (tensor views of the driver's state), layout
        (n, origin, parent), dx, time and descriptor table."""
        return [self._level(l) for l in range(_lib().enzo_hierarchy_nlevel(self._h))]

    # -- the W-cycle, rebuilds, timing -----------------------------------------
    @staticmethod
    def _rebuild_params(gamma, crit, clus, margin=3, nest=1, precision=0):
        crit, clus = dict(crit or {}), dict(clus or {})
        fp = _FlagParams(gamma, crit.get("slope", 0.3), crit.get("shock_dp", 0.33), crit.get("shock_e", 0.1),
                         crit.get("mass", 0.0), precision)
        cp = _ClusterParams(clus.get("efficiency", 0.3), clus.get("small_cells", 64), clus.get("buffer", 1), 0)
        return _RebuildParams(fp, cp, margin, nest)

    def _take_log(self, log):
        L = _lib()
        n = ctypes.c_int32(0)
        cap = 256
        while True:
            lv = (ctypes.c_int32 * cap)()
            dt = (ctypes.c_double * cap)()
            r = L.enzo_hierarchy_take_log(self._h, lv, dt, cap, ctypes.byref(n))
            if r == -3:
                cap = n.value
                continue
            _check(r, "enzo_hierarchy_take_log")
            break
        if log is not None:
            log.extend((int(lv[k]), float(dt[k])) for k in range(n.value))

    def root_step(self, params, cfl_params=None, log=None, rebuild=None):
        """One root step: dt_0 from the root CFL rule, then the W-cycle.
        rebuild: None, or a dict (gamma, crit, clus[, margin, nest]) for a
        rebuild after every step of a level with children (flags in the sweeps'
        precision).  Appends (level, dt) of every level step to log."""
        cfl_params = cfl_params if cfl_params is not None else Params(
            gamma=params.gamma, cfl=params.cfl, precision=params.precision)
        p, c = params.c(), cfl_params.c()
        rb = self._rebuild_params(**rebuild, precision=params.precision) if rebuild is not None else None
        dt0 = ctypes.c_double(0.0)
        with self.torch.cuda.device(self.device):
            r = _lib().enzo_hierarchy_root_step(self._h, ctypes.byref(p), ctypes.byref(c),
                                                ctypes.byref(rb) if rb is not None else None, ctypes.byref(dt0))
        self._take_log(log)
        _check(r, "enzo_hierarchy_root_step")
        return dt0.value

    def evolve_level(self, l, t_parent, params, cfl_params, log=None, rebuild=None):
        """Advance the root (l = 0) and with it every finer level to t_parent in
        one root step (the W-cycle below it as in root_step)."""
        if l != 0:
            raise ValueError("the driver advances the hierarchy from its root")
        p, c = params.c(), cfl_params.c()
        rb = self._rebuild_params(**rebuild, precision=params.precision) if rebuild is not None else None
        with self.torch.cuda.device(self.device):
            r = _lib().enzo_hierarchy_step_to(self._h, float(t_parent), ctypes.byref(p), ctypes.byref(c),
                                              ctypes.byref(rb) if rb is not None else None)
        self._take_log(log)
        _check(r, "enzo_hierarchy_step_to")

    def rebuild(self, l, gamma, crit, clus, margin=3, nest=1, precision=0):
        """Replace levels l+1, l+2, ... by grids covering the flagged cells of the
        level above each (Sec. 3.5, 3.6): level l's ghosts are filled, its cells
        flagged on the GPU and each patch's flags clustered on the host; every
        new patch is interpolated from its parent (SecondOrderA, FP64) and
        overwritten by the old patches of its level where they overlap (a level
        whose boxes come out unchanged is kept as it is).  On the root, flags
        within `margin` cells of the domain boundary are dropped, on deeper
        levels those within `nest` cells of the patch's edge.  `precision`
        picks the flag kernel (FP64 or FP32).  Returns the new boxes of level
        l+1 as (parent, lo, hi) in level-l cells."""
        rb = self._rebuild_params(gamma, crit, clus, margin, nest, precision)
        cap = 1 << 16
        while True:
            boxes = (ctypes.c_int32 * (7 * cap))()
            nb = ctypes.c_int32(0)
            with self.torch.cuda.device(self.device):
                r = _lib().enzo_hierarchy_rebuild(self._h, l, ctypes.byref(rb), boxes, cap, ctypes.byref(nb))
            if r == -3 and nb.value > cap:
                # rebuilt, but the box list was short: level l is unchanged, so
                # flagging it again gives the same grids, which are then kept
                cap = nb.value
                continue
            _check(r, "enzo_hierarchy_rebuild")
            break
        v = np.frombuffer(boxes, dtype=np.int32)[:7 * nb.value].reshape(-1, 7)
        return [(int(e[0]), tuple(int(x) for x in e[1:4]), tuple(int(x) for x in e[4:7])) for e in v]

    @property
    def timing(self):
        return self._timing

    @timing.setter
    def timing(self, value):
        """Set to {} to time each operation kind on the device (CUDA events), None to stop."""
        _check(_lib().enzo_hierarchy_timing(self._h, 0 if value is None else 1, None, None), "enzo_hierarchy_timing")
        self._timing = value

    def timing_ms(self):
        """Milliseconds per operation kind since timing was switched on (synchronises the stream)."""
        ms = (ctypes.c_double * len(OPS))()
        _check(_lib().enzo_hierarchy_timing(self._h, -1, ms, None), "enzo_hierarchy_timing")
        return {name: ms[k] for k, name in enumerate(OPS) if ms[k] > 0.0}

    @property
    def cell_updates(self):
        cu = ctypes.c_int64(0)
        _check(_lib().enzo_hierarchy_timing(self._h, -1, None, ctypes.byref(cu)), "enzo_hierarchy_timing")
        return int(cu.value)

    def patch_fields(self, l, i):
        """Host copies of patch i of level l: the five fields, and the gas
        energy as a sixth with dual energy."""
        self.stream.synchronize()
        b = self.levels[l]["batch"]
        views = b.patch_fields(i) + ([b.patch_ge(i)] if self.nf == 6 else [])
        return [f.cpu().numpy() for f in views]
