"""AMR hierarchy on the GPU: host plans per level, every step of the W-cycle
run by the library's kernels (paper Sec. 3), and an optional rebuild of the
finer levels from flagged cells (Sec. 3.5, 3.6).

A level is one PatchBatch.  Host plans per level (again after a rebuild):
  * links: origin (global index of the first active cell) and parent index;
  * sibling copy boxes: ghost regions of each patch that lie in a sibling's
    active box.  Static levels tile boxes by tensor-product cuts, so a patch's
    ghost region meets at most its 26 neighbours, found by a lattice lookup;
    rebuilt levels are any disjoint boxes, and every pair of patches is
    intersected;
  * flux-correction face parts: the cells outside each fine face, per coarse
    patch holding them, in waves so that corrections meeting in one coarse
    cell add in a fixed order;
  * flux registers: all-face registers for patches with children, boundary-face
    registers for patches with a parent.

W-cycle of one root step (EvolveLevel of Sec. 3):
  fill ghosts; dt = min(CFL, t_parent - t); save the old state if the level has
  children; three sweeps (recording fluxes); t += dt; if children: fill ghosts
  at the new time, zero the children's boundary registers, advance the children
  to t, flux correction, projection, and (with a rebuild) new finer levels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import (GUESS_MLP, PATCH_PERIODIC, PatchBatch, Params, _check, ghost_fill_boundary, lib, patch_table,
               ppm_sweep, timestep_cfl)

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
        for n in ("enzo_ghost_fill_level", "enzo_flux_correct", "enzo_project", "enzo_copy_level",
                  "enzo_flag_cells", "enzo_cluster_flags"):
            getattr(L, n).restype = ctypes.c_int
        L._hier_ready = True
    return L


def _to_dev(arr, device):
    import torch
    raw = np.frombuffer(np.ascontiguousarray(arr).tobytes(), dtype=np.uint8).copy()
    if raw.size == 0:
        raw = np.zeros(16, dtype=np.uint8)
    return torch.from_numpy(raw).to(device)


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


def sibling_boxes_general(n, origin):
    """sibling_boxes for any disjoint layout: every intersection of a patch's
    ghost-extended box with another patch's active box."""
    n, origin = np.asarray(n, dtype=np.int64), np.asarray(origin, dtype=np.int64)
    lo, hi = origin, origin + n
    out = []
    for a in range(len(n)):
        blo = np.maximum(lo[a] - NG, lo)
        bhi = np.minimum(hi[a] + NG, hi)
        keep = np.all(blo < bhi, axis=1)
        keep[a] = False
        b = np.flatnonzero(keep)
        out.append(_boxes(np.full(len(b), a), b, blo[b], bhi[b]))
    return np.concatenate(out) if out else _boxes([], [], np.zeros((0, 3)), np.zeros((0, 3)))


def interp_boxes_general(n, origin):
    """The 26 ghost regions of every patch, except those lying wholly in one
    sibling's active box; the sibling copies that follow overwrite the parts
    siblings cover (the order of Sec. 3.1)."""
    n, origin = np.asarray(n, dtype=np.int64), np.asarray(origin, dtype=np.int64)
    lo, hi = origin, origin + n
    out = []
    for a in range(len(n)):
        for d in _DIRS:
            blo = np.where(d < 0, lo[a] - NG, np.where(d > 0, hi[a], lo[a]))
            bhi = np.where(d < 0, lo[a], np.where(d > 0, hi[a] + NG, hi[a]))
            inside = np.all((lo <= blo) & (bhi <= hi), axis=1)
            if not inside.any():
                out.append((a, blo, bhi))
    if not out:
        return _boxes([], [], np.zeros((0, 3)), np.zeros((0, 3)))
    a = np.array([o[0] for o in out])
    return _boxes(a, a, np.array([o[1] for o in out]), np.array([o[2] for o in out]))


def correction_parts(fine, coarse, r=2):
    """Flux-correction face parts for any disjoint layouts, in the order
    (fine patch, axis, side), each part the cells outside one fine face that
    one coarse patch holds; faces whose outside cells the fine level covers
    entirely are left out (projection overwrites those cells).  Returns the
    parts and, for each, a wave: parts in one wave share no coarse cell, and a
    part that shares cells with earlier parts comes in a later wave, so the
    additions happen in the listed order."""
    fn, fo = np.asarray(fine["n"], dtype=np.int64), np.asarray(fine["origin"], dtype=np.int64)
    cn, co = np.asarray(coarse["n"], dtype=np.int64), np.asarray(coarse["origin"], dtype=np.int64)
    flo, fhi = fo // r, (fo + fn) // r          # coarse footprints of the fine patches
    clo, chi = co, co + cn
    parts, cells = [], []
    for i in range(len(fn)):
        for d in range(3):
            a1 = 1 if d == 0 else 0
            a2 = 1 if d == 2 else 2
            for side in (0, 1):
                X = (fo[i, d] + (fn[i, d] if side else 0)) // r
                olo, ohi = flo[i].copy(), fhi[i].copy()
                olo[d], ohi[d] = (X - 1, X) if side == 0 else (X, X + 1)
                vol = int(np.prod(ohi - olo))
                ilo, ihi = np.maximum(olo, flo), np.minimum(ohi, fhi)
                covered = int(np.prod(np.clip(ihi - ilo, 0, None), axis=1).sum())
                if covered >= vol:
                    continue
                tlo, thi = np.maximum(olo, clo), np.minimum(ohi, chi)
                for t in np.flatnonzero(np.all(tlo < thi, axis=1)):
                    parts.append((i, d, side, t, tlo[t][a1] - flo[i, a1], tlo[t][a2] - flo[i, a2],
                                  thi[t][a1] - flo[i, a1], thi[t][a2] - flo[i, a2]))
                    cells.append((t, tlo[t], thi[t]))
    out = np.zeros(len(parts), dtype=FACE_DTYPE)
    wave = np.zeros(len(parts), dtype=np.int64)
    for k, (i, d, side, t, l1, l2, h1, h2) in enumerate(parts):
        out[k] = (i, d, side, t, (l1, l2), (h1, h2))
        tk, lk, hk = cells[k]
        for q in range(k):
            tq, lq, hq = cells[q]
            if tq == tk and np.all(np.maximum(lk, lq) < np.minimum(hk, hq)):
                wave[k] = max(wave[k], wave[q] + 1)
    return out, wave


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


class Hierarchy:
    """Device state of a hierarchy built from synth.hierarchy_layout (static),
    with an optional rebuild of the finer levels from flagged cells (Sec. 3.5,
    3.6)."""

    def __init__(self, layout, fields, root_dx, device="cuda", stream=None, root_bc=None):
        """fields: per level, per patch, the five ghost-zoned fields, or six with
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
        self.levels = []
        self.nf = len(fields[0][0])
        if self.nf not in (5, 6):
            raise ValueError("a patch has five fields, or six with the gas energy")
        nlev = len(layout)
        if nlev > 1:
            self._check_root_margin(np.asarray(layout[0]["n"][0]), np.asarray(layout[1]["origin"]),
                                    np.asarray(layout[1]["n"]))
        for l, L in enumerate(layout):
            n = np.asarray(L["n"], dtype=np.int64)
            vols = np.prod(n + 2 * NG, axis=1)
            offs = np.concatenate([[0], np.cumsum(vols)[:-1]]).astype(np.int64)
            flat = [np.zeros(int(vols.sum())) for _ in range(self.nf)]
            for i in range(len(n)):
                for f in range(self.nf):
                    blk = np.asarray(fields[l][i][f])
                    flat[f][offs[i]:offs[i] + blk.size] = blk.ravel()
            self.levels.append(self._build_level(l, n, np.asarray(L["origin"]), np.asarray(L["parent"]), flat,
                                                 l + 1 < nlev, general=False))
        for l in range(nlev - 1):
            self._plan_correction(l, general=False)
        # the uploads and zero fills above ran on the current stream; the
        # hierarchy's own stream must not start before they are done
        torch.cuda.synchronize(self.device)
        self.cell_updates = 0
        self.timing = None          # {op: [(start, end) events]} when profiling

    @staticmethod
    def _check_root_margin(root_n, origin, n):
        # the periodic root wraps inside its sweeps and keeps no ghost cells, so
        # the level-1 ghost interpolation (SecondOrderA reaches one root cell
        # beyond the cell under a fine ghost) must find its parent cells inside it
        if len(n) and (np.any(origin // 2 < 3) or np.any((origin + n + 1) // 2 > root_n - 3)):
            raise ValueError("level 1 must stay 3 root cells away from the domain boundary")

    def _build_level(self, l, n, origin, parent, flat, has_children, general, state=None):
        """Device state of level l from its layout; flat: the five (six with
        gas energy) flat host fields, or None for zeros.  state: time
        bookkeeping to keep."""
        torch = self.torch
        n = np.asarray(n, dtype=np.int64).reshape(-1, 3)
        vols = np.prod(n + 2 * NG, axis=1)
        offs = np.concatenate([[0], np.cumsum(vols)[:-1]]).astype(np.int64)
        dx = self.root_dx / 2 ** l
        wrap = l == 0 and self.root_bc is None
        table = patch_table(n, offs, [dx] * 3, flags=PATCH_PERIODIC if wrap else 0, level=l)
        has_parent = l > 0
        a_sz, b_sz = register_sizes(n, self.nf)
        reg = 0
        if has_children:
            table["freg_all"] = np.concatenate([[0], np.cumsum(a_sz)[:-1]]) + reg
            reg += int(a_sz.sum())
        if has_parent:
            table["freg_bnd"] = np.concatenate([[0], np.cumsum(b_sz)[:-1]]) + reg
            reg += int(b_sz.sum())
        if flat is None:
            flat = [torch.zeros(max(int(vols.sum()), 1), dtype=torch.float64, device=self.device)
                    for _ in range(self.nf)]
        with torch.cuda.stream(self.stream):
            batch = PatchBatch(table, flat[:5], device=self.device, stream=self.stream,
                               ge=flat[5] if self.nf == 6 else None)
        if reg:
            batch.freg = torch.zeros(reg, dtype=torch.float64, device=self.device)
        links = np.zeros(len(n), dtype=LINK_DTYPE)
        links["origin"] = np.asarray(origin).reshape(-1, 3)
        links["parent"] = np.asarray(parent).reshape(-1)
        lev = {"batch": batch, "links": _to_dev(links, self.device), "table": table, "n": n,
               "origin": np.asarray(origin).reshape(-1, 3), "parent": np.asarray(parent).reshape(-1), "dx": dx,
               "t": 0.0, "step": 0, "t_old": 0.0, "has_children": has_children, "bnd_sl": None,
               "cells": int(np.prod(n, axis=1).sum()), "general": general}
        if state is not None:
            lev.update(state)
        if has_parent:
            sib = sibling_boxes_general if general else sibling_boxes
            itp = interp_boxes_general if general else interp_boxes
            bx = sib(n, lev["origin"])
            lev["boxes"], lev["nbox"] = _to_dev(bx, self.device), len(bx)
            ib = itp(n, lev["origin"])
            lev["ibox"], lev["nibox"] = _to_dev(ib, self.device), len(ib)
            lo = int(table["freg_bnd"].min()) if len(n) else 0
            lev["bnd_sl"] = (lo, lo + int(b_sz.sum()))
        if has_children:
            lev["old"] = [torch.empty_like(u) for u in self._fields(batch)]
        return lev

    def _fields(self, batch):
        """The fields a hierarchy operation carries: U, and ge with dual energy."""
        return list(batch.U) + ([batch.ge] if self.nf == 6 else [])

    def _plan_correction(self, l, general):
        """Flux-correction parts of level l (coarse) against level l + 1, as
        device arrays per wave."""
        fine = {"n": self.levels[l + 1]["n"], "origin": self.levels[l + 1]["origin"]}
        coarse = {"n": self.levels[l]["n"], "origin": self.levels[l]["origin"]}
        if general:
            fc, wave = correction_parts(fine, coarse)
        else:
            fc = correction_faces(fine, coarse)
            wave = np.zeros(len(fc), dtype=np.int64)
        waves = []
        for w in range(int(wave.max()) + 1 if len(wave) else 0):
            sel = fc[wave == w]
            waves.append((_to_dev(sel, self.device), len(sel)))
        self.levels[l]["waves"] = waves

    def _mark(self, op):
        """Record a CUDA event pair around an operation when timing is on."""
        if self.timing is None:
            return None
        e = self.torch.cuda.Event(enable_timing=True)
        e.record(self.stream)
        self.timing.setdefault(op, []).append([e, None])
        return self.timing[op][-1]

    def _end(self, mark):
        if mark is None:
            return
        e = self.torch.cuda.Event(enable_timing=True)
        e.record(self.stream)
        mark[1] = e

    def timing_ms(self):
        """Milliseconds per operation type (after synchronising the stream)."""
        self.stream.synchronize()
        return {op: sum(a.elapsed_time(b) for a, b in v) for op, v in (self.timing or {}).items()}

    # -- primitive operations -------------------------------------------
    def _fill(self, l, precision):
        lev = self.levels[l]
        if l == 0:
            if self.root_bc is not None:
                ghost_fill_boundary(lev["batch"], self.root_bc)
            return          # a periodic root wraps inside its sweeps
        par = self.levels[l - 1]
        w = (lev["t"] - par["t_old"]) / (par["t"] - par["t_old"])
        b, pb = lev["batch"].c(), par["batch"].c()
        old = (ctypes.c_void_p * 5)(*[u.data_ptr() for u in par["old"][:5]])
        old_ge = par["old"][5].data_ptr() if self.nf == 6 else None
        _check(_lib().enzo_ghost_fill_level(ctypes.byref(b), lev["links"].data_ptr(), ctypes.byref(pb),
                                            par["links"].data_ptr(), old, old_ge, w, lev["ibox"].data_ptr(),
                                            lev["nibox"], lev["boxes"].data_ptr(), lev["nbox"], precision, 2),
               "enzo_ghost_fill_level")

    def _step(self, l, dt, params):
        lev = self.levels[l]
        order = (0, 1, 2) if lev["step"] % 2 == 0 else (2, 1, 0)
        done = 0
        for d in order:
            cover = 7 & ~done & ~(1 << d)
            ppm_sweep(lev["batch"], d, dt, cover, params)
            done |= 1 << d
        lev["step"] += 1
        self.cell_updates += lev["cells"]

    def _correct_and_project(self, l, dt, params):
        c, f = self.levels[l], self.levels[l + 1]
        cb, fb = c["batch"].c(), f["batch"].c()
        for faces, nface in c["waves"]:
            _check(_lib().enzo_flux_correct(ctypes.byref(cb), c["links"].data_ptr(), ctypes.byref(fb),
                                            f["links"].data_ptr(), faces.data_ptr(), nface, dt, 2,
                                            1 if params.precision == 1 else 0),
                   "enzo_flux_correct")
        _check(_lib().enzo_project(ctypes.byref(cb), c["links"].data_ptr(), ctypes.byref(fb),
                                   f["links"].data_ptr(), 2), "enzo_project")

    # -- rebuild (Sec. 3.5, 3.6) ---------------------------------------------
    def rebuild(self, l, gamma, crit, clus, margin=3, nest=1, precision=0):
        """Replace levels l+1, l+2, ... by grids covering the flagged cells of the
        level above each (Sec. 3.5, 3.6): level l's ghosts are filled, its cells
        flagged on the GPU and each patch's flags clustered on the host; every
        new patch is interpolated from its parent (SecondOrderA) and overwritten
        by the old patches of its level where they overlap (a level whose boxes
        come out unchanged is kept as it is).  On the root, flags
        within `margin` cells of the domain boundary are dropped, on deeper
        levels those within `nest` cells of the patch's edge (the coarse cells
        outside every new fine face then lie in the parent).  The fill and
        the interpolation run in FP64 in both precisions (the new grids keep
        their parents' means to FP64 rounding); `precision` picks the flag
        kernel (FP64 or FP32).  Returns the new boxes of level l+1 as (parent,
        lo, hi) in level-l cells."""
        with self.torch.cuda.stream(self.stream):
            self._fill(l, 0)
            first = None
            for m in range(l, len(self.levels) - 1):
                boxes = self._rebuild_one(m, gamma, crit, clus, margin if m == 0 else nest, precision)
                first = boxes if first is None else first
        return first

    def _rebuild_one(self, m, gamma, crit, clus, margin, flag_precision=0):
        precision = 0
        lev = self.levels[m]
        flags = flag_cells(lev["batch"], gamma, precision=flag_precision, **crit)
        boxes = []
        for i, fl in enumerate(flags):
            o = lev["origin"][i]
            for lo, hi in cluster_flags(fl, margin=margin, **clus):
                boxes.append((i, tuple(int(o[a] + lo[a]) for a in range(3)), tuple(int(o[a] + hi[a]) for a in range(3))))
        n = np.array([[2 * (hi[a] - lo[a]) for a in range(3)] for _, lo, hi in boxes], dtype=np.int64).reshape(-1, 3)
        origin = np.array([[2 * lo[a] for a in range(3)] for _, lo, _ in boxes], dtype=np.int64).reshape(-1, 3)
        parent = np.array([b[0] for b in boxes], dtype=np.int64)
        old = self.levels[m + 1]
        same = [(int(p), tuple(int(v) // 2 for v in o), tuple((int(v) + int(w)) // 2 for v, w in zip(o, n_)))
                for p, o, n_ in zip(old["parent"], old["origin"], old["n"])]
        if boxes == same:
            # the same grids: the level stays as it is; the level above may be
            # new, so its correction parts are planned again
            self._plan_correction(m, general=True)
            return boxes
        state = {k: old[k] for k in ("t", "step", "t_old")}
        new = self._build_level(m + 1, n, origin, parent, None, old["has_children"], general=True, state=state)
        if len(n):
            L = _lib()
            full = _boxes(np.arange(len(n)), np.arange(len(n)), origin - NG, origin + n + NG)
            fb = _to_dev(full, self.device)
            nb, pb = new["batch"].c(), lev["batch"].c()
            cur = (ctypes.c_void_p * 5)(*[u.data_ptr() for u in lev["batch"].U])
            cur_ge = lev["batch"].ge.data_ptr() if self.nf == 6 else None
            _check(L.enzo_ghost_fill_level(ctypes.byref(nb), new["links"].data_ptr(), ctypes.byref(pb),
                                           lev["links"].data_ptr(), cur, cur_ge, 0.0, fb.data_ptr(), len(full),
                                           None, 0,
                                           precision, 2), "enzo_ghost_fill_level")
            # cells of the new patches (ghosts included) lying in an old patch
            olo, ohi = old["origin"], old["origin"] + old["n"]
            cps = []
            for a in range(len(n)):
                blo = np.maximum(origin[a] - NG, olo)
                bhi = np.minimum(origin[a] + n[a] + NG, ohi)
                b = np.flatnonzero(np.all(blo < bhi, axis=1))
                cps.append(_boxes(np.full(len(b), a), b, blo[b], bhi[b]))
            cp = np.concatenate(cps)
            if len(cp):
                cb = _to_dev(cp, self.device)
                ob = old["batch"].c()
                _check(L.enzo_copy_level(ctypes.byref(nb), new["links"].data_ptr(), ctypes.byref(ob),
                                         old["links"].data_ptr(), cb.data_ptr(), len(cp)), "enzo_copy_level")
        self.levels[m + 1] = new
        self._plan_correction(m, general=True)
        return boxes

    # -- W-cycle ------------------------------------------------------------
    def evolve_level(self, l, t_parent, params, cfl_params, log=None, rebuild=None):
        """Advance level l to t_parent (W-cycle).  rebuild: None, or a dict
        (gamma, crit, clus) for rebuild() after every step of a level with
        children (after flux correction and projection)."""
        lev = self.levels[l]
        if lev["cells"] == 0:
            lev["t"] = t_parent          # a level without grids has nothing to advance
            return
        with self.torch.cuda.stream(self.stream):
            while lev["t"] < t_parent * (1 - 1e-14):
                m = self._mark("ghost_fill")
                self._fill(l, params.precision)
                self._end(m)
                if l == 0:
                    dt = t_parent - lev["t"]
                else:
                    m = self._mark("cfl")
                    dt = min(timestep_cfl(lev["batch"], cfl_params), t_parent - lev["t"])
                    self._end(m)
                if lev["has_children"]:
                    m = self._mark("save_old")
                    for u, o in zip(self._fields(lev["batch"]), lev["old"]):
                        o.copy_(u)
                    self._end(m)
                    lev["t_old"] = lev["t"]
                m = self._mark("sweeps")
                self._step(l, dt, params)
                self._end(m)
                lev["t"] += dt
                if log is not None:
                    log.append((l, dt))
                if lev["has_children"]:
                    m = self._mark("ghost_fill")
                    self._fill(l, params.precision)
                    self._end(m)
                    child = self.levels[l + 1]
                    if child["batch"].freg is not None:         # None: a level without grids
                        lo, hi = child["bnd_sl"]
                        child["batch"].freg[lo:hi].zero_()
                    self.evolve_level(l + 1, lev["t"], params, cfl_params, log, rebuild)
                    m = self._mark("correct_project")
                    self._correct_and_project(l, dt, params)
                    self._end(m)
                    if rebuild is not None:
                        m = self._mark("rebuild")
                        self.rebuild(l, **rebuild, precision=params.precision)
                        self._end(m)
            # the loop stops within 1e-14 of the parent's time; the level has reached it
            lev["t"] = t_parent

    def root_step(self, params, cfl_params=None, log=None, rebuild=None):
        """One root step: dt_0 from the root CFL rule, then the W-cycle."""
        cfl_params = cfl_params if cfl_params is not None else Params(
            gamma=params.gamma, cfl=params.cfl, precision=params.precision)
        root = self.levels[0]
        with self.torch.cuda.stream(self.stream):
            dt0 = timestep_cfl(root["batch"], cfl_params)
        self.evolve_level(0, root["t"] + dt0, params, cfl_params, log, rebuild)
        return dt0

    def patch_fields(self, l, i):
        """Host copies of patch i of level l: the five fields, and the gas
        energy as a sixth with dual energy."""
        b = self.levels[l]["batch"]
        views = b.patch_fields(i) + ([b.patch_ge(i)] if self.nf == 6 else [])
        return [f.cpu().numpy() for f in views]
