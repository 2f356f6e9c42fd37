"""Static AMR hierarchy on the GPU: plans built on the host once, every step of
the W-cycle run by the library's kernels (paper Sec. 3).

A level is one PatchBatch.  Host plans per level:
  * links: origin (global index of the first active cell) and parent index;
  * sibling copy boxes: ghost regions of each patch that lie in a sibling's
    active box (the patches of a level tile boxes by tensor-product cuts, so a
    patch's ghost region meets at most its 26 neighbours);
  * flux-correction faces: faces of fine patches on the boundary of the refined
    region, with the coarse patch holding the cells outside them;
  * flux registers: all-face registers for patches with children, boundary-face
    registers for patches with a parent.

W-cycle of one root step (EvolveLevel of Sec. 3, as in the reference):
  fill ghosts; dt = min(CFL, t_parent - t); save the old state if the level has
  children; three sweeps (recording fluxes); t += dt; if children: fill ghosts
  at the new time, zero the children's boundary registers, advance the children
  to t, flux correction, projection.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import (GUESS_MLP, PATCH_PERIODIC, PatchBatch, Params, _check, lib, patch_table, ppm_sweep,
               timestep_cfl)

NG = 3
LINK_DTYPE = np.dtype([("origin", "<i4", (3,)), ("parent", "<i4")])
BOX_DTYPE = np.dtype([("dst", "<i4"), ("src", "<i4"), ("lo", "<i4", (3,)), ("hi", "<i4", (3,))])
FACE_DTYPE = np.dtype([("fine", "<i4"), ("dir", "<i4"), ("side", "<i4"), ("target", "<i4")])


def _lib():
    L = lib()
    if not getattr(L, "_hier_ready", False):
        vp, i32, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
        L.enzo_ghost_fill_level.argtypes = [vp, vp, vp, vp, vp, d, vp, i32, vp, i32, i32, i32]
        L.enzo_flux_correct.argtypes = [vp, vp, vp, vp, vp, i32, d, i32, i32]
        L.enzo_project.argtypes = [vp, vp, vp, vp, i32]
        for n in ("enzo_ghost_fill_level", "enzo_flux_correct", "enzo_project"):
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
    return t


def register_sizes(n):
    """(all-face, boundary-face) register sizes in doubles of patches of sizes n."""
    n = np.asarray(n, dtype=np.int64)
    nx, ny, nz = n[:, 0], n[:, 1], n[:, 2]
    all_f = ((nx + 1) * ny * nz + (ny + 1) * nx * nz + (nz + 1) * nx * ny) * 5
    bnd = 2 * (ny * nz + nx * nz + nx * ny) * 5
    return all_f, bnd


class Hierarchy:
    """Device state of a static hierarchy built from synth.hierarchy_layout."""

    def __init__(self, layout, fields, root_dx, device="cuda", stream=None):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.levels = []
        nlev = len(layout)
        if nlev > 1:
            # the periodic root wraps inside its sweeps and keeps no ghost cells, so
            # the level-1 ghost interpolation must find its parent cells inside it
            root_n = np.asarray(layout[0]["n"][0])
            o1 = np.asarray(layout[1]["origin"])
            e1 = o1 + np.asarray(layout[1]["n"])
            if np.any(o1 // 2 < 2) or np.any((e1 + 1) // 2 > root_n - 2):
                raise ValueError("level 1 must stay 2 root cells away from the domain boundary")
        for l, L in enumerate(layout):
            n = np.asarray(L["n"], dtype=np.int64)
            vols = np.prod(n + 2 * NG, axis=1)
            offs = np.concatenate([[0], np.cumsum(vols)[:-1]]).astype(np.int64)
            flat = [np.zeros(int(vols.sum())) for _ in range(5)]
            for i in range(len(n)):
                for f in range(5):
                    blk = np.asarray(fields[l][i][f])
                    flat[f][offs[i]:offs[i] + blk.size] = blk.ravel()
            dx = root_dx / 2 ** l
            table = patch_table(n, offs, [dx] * 3, flags=PATCH_PERIODIC if l == 0 else 0, level=l)
            has_children = l + 1 < nlev
            has_parent = l > 0
            a_sz, b_sz = register_sizes(n)
            reg = 0
            if has_children:
                table["freg_all"] = np.concatenate([[0], np.cumsum(a_sz)[:-1]]) + reg
                reg += int(a_sz.sum())
            if has_parent:
                table["freg_bnd"] = np.concatenate([[0], np.cumsum(b_sz)[:-1]]) + reg
                reg += int(b_sz.sum())
            with torch.cuda.stream(self.stream):
                batch = PatchBatch(table, flat, device=self.device, stream=self.stream)
            if reg:
                batch.freg = torch.zeros(reg, dtype=torch.float64, device=self.device)
            links = np.zeros(len(n), dtype=LINK_DTYPE)
            links["origin"] = np.asarray(L["origin"])
            links["parent"] = np.asarray(L["parent"])
            lev = {"batch": batch, "links": _to_dev(links, self.device), "table": table, "n": n,
                   "origin": np.asarray(L["origin"]), "dx": dx, "t": 0.0, "step": 0, "t_old": 0.0,
                   "has_children": has_children, "bnd_sl": None, "cells": int(np.prod(n, axis=1).sum())}
            if has_parent:
                bx = sibling_boxes(n, np.asarray(L["origin"]))
                lev["boxes"], lev["nbox"] = _to_dev(bx, self.device), len(bx)
                ib = interp_boxes(n, np.asarray(L["origin"]))
                lev["ibox"], lev["nibox"] = _to_dev(ib, self.device), len(ib)
                lo = int(table["freg_bnd"].min())
                lev["bnd_sl"] = (lo, lo + int(b_sz.sum()))
            if has_children:
                lev["old"] = [torch.empty_like(u) for u in batch.U]
            self.levels.append(lev)
        for l in range(nlev - 1):
            fc = correction_faces({"n": self.levels[l + 1]["n"], "origin": self.levels[l + 1]["origin"]},
                                  {"n": self.levels[l]["n"], "origin": self.levels[l]["origin"]})
            self.levels[l]["faces"], self.levels[l]["nface"] = _to_dev(fc, self.device), len(fc)
        self.cell_updates = 0
        self.timing = None          # {op: [(start, end) events]} when profiling

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
            return          # the periodic root wraps inside its sweeps
        par = self.levels[l - 1]
        w = (lev["t"] - par["t_old"]) / (par["t"] - par["t_old"])
        b, pb = lev["batch"].c(), par["batch"].c()
        old = (ctypes.c_void_p * 5)(*[u.data_ptr() for u in par["old"]])
        _check(_lib().enzo_ghost_fill_level(ctypes.byref(b), lev["links"].data_ptr(), ctypes.byref(pb),
                                            par["links"].data_ptr(), old, w, lev["ibox"].data_ptr(),
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
        _check(_lib().enzo_flux_correct(ctypes.byref(cb), c["links"].data_ptr(), ctypes.byref(fb),
                                        f["links"].data_ptr(), c["faces"].data_ptr(), c["nface"], dt, 2,
                                        1 if params.precision == 1 else 0),
               "enzo_flux_correct")
        _check(_lib().enzo_project(ctypes.byref(cb), c["links"].data_ptr(), ctypes.byref(fb),
                                   f["links"].data_ptr(), 2), "enzo_project")

    # -- W-cycle ------------------------------------------------------------
    def evolve_level(self, l, t_parent, params, cfl_params, log=None):
        lev = self.levels[l]
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
                    for u, o in zip(lev["batch"].U, lev["old"]):
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
                    lo, hi = child["bnd_sl"]
                    child["batch"].freg[lo:hi].zero_()
                    self.evolve_level(l + 1, lev["t"], params, cfl_params, log)
                    m = self._mark("correct_project")
                    self._correct_and_project(l, dt, params)
                    self._end(m)

    def root_step(self, params, cfl_params=None, log=None):
        """One root step: dt_0 from the root CFL rule, then the W-cycle."""
        cfl_params = cfl_params if cfl_params is not None else Params(
            gamma=params.gamma, cfl=params.cfl, precision=params.precision)
        root = self.levels[0]
        with self.torch.cuda.stream(self.stream):
            dt0 = timestep_cfl(root["batch"], cfl_params)
        self.evolve_level(0, root["t"] + dt0, params, cfl_params, log)
        return dt0

    def patch_fields(self, l, i):
        return [f.cpu().numpy() for f in self.levels[l]["batch"].patch_fields(i)]
