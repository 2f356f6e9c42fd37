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
    """Patch lookup of a level tiled by the tensor product of per-axis segments."""

    def __init__(self, n, origin):
        self.n, self.origin = np.asarray(n), np.asarray(origin)
        self.starts = [np.unique(self.origin[:, a]) for a in range(3)]
        self.index = {}
        for i, o in enumerate(self.origin):
            self.index[tuple(int(v) for v in o)] = i

    def seg(self, a, x):
        """Index of the segment of axis a containing coordinate x, or -1."""
        k = int(np.searchsorted(self.starts[a], x, side="right")) - 1
        return k

    def find(self, g):
        """Patch whose active box contains global cell g, or -1."""
        key = []
        for a in range(3):
            k = self.seg(a, g[a])
            if k < 0:
                return -1
            key.append(int(self.starts[a][k]))
        i = self.index.get(tuple(key), -1)
        if i < 0:
            return -1
        lo, hi = self.origin[i], self.origin[i] + self.n[i]
        return i if np.all((lo <= g) & (g < hi)) else -1


def sibling_boxes(n, origin):
    """Copy boxes (dst, src, lo, hi) of ghost cells lying in siblings' active
    boxes.  Ghost layers (3 cells) are thinner than any patch, so only the 26
    neighbours across faces, edges and corners can meet a patch's ghost region."""
    n, origin = np.asarray(n), np.asarray(origin)
    grid = _Grid(n, origin)
    boxes = []
    for a in range(len(n)):
        lo, hi = origin[a], origin[a] + n[a]
        glo, ghi = lo - NG, hi + NG
        seen = set()
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if dx == dy == dz == 0:
                        continue
                    probe = np.array([lo[0] - 1 if dx < 0 else (hi[0] if dx > 0 else lo[0]),
                                      lo[1] - 1 if dy < 0 else (hi[1] if dy > 0 else lo[1]),
                                      lo[2] - 1 if dz < 0 else (hi[2] if dz > 0 else lo[2])])
                    b = grid.find(probe)
                    if b < 0 or b in seen:
                        continue
                    seen.add(b)
                    blo = np.maximum(glo, origin[b])
                    bhi = np.minimum(ghi, origin[b] + n[b])
                    if np.all(blo < bhi):
                        boxes.append((a, int(b), *blo.tolist(), *bhi.tolist()))
    t = np.zeros(len(boxes), dtype=BOX_DTYPE)
    for i, bx in enumerate(boxes):
        t[i]["dst"], t[i]["src"] = bx[0], bx[1]
        t[i]["lo"] = bx[2:5]
        t[i]["hi"] = bx[5:8]
    return t


def interp_boxes(n, origin):
    """Ghost regions (of the 26 around each patch: faces, edges, corners) that no
    sibling covers; these are interpolated from the parent."""
    n, origin = np.asarray(n), np.asarray(origin)
    grid = _Grid(n, origin)
    boxes = []
    for a in range(len(n)):
        lo, hi = origin[a], origin[a] + n[a]
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if dx == dy == dz == 0:
                        continue
                    dd = (dx, dy, dz)
                    blo = np.array([lo[t] - NG if dd[t] < 0 else (hi[t] if dd[t] > 0 else lo[t]) for t in range(3)])
                    bhi = np.array([lo[t] if dd[t] < 0 else (hi[t] + NG if dd[t] > 0 else hi[t]) for t in range(3)])
                    probe = np.array([lo[t] - 1 if dd[t] < 0 else (hi[t] if dd[t] > 0 else lo[t]) for t in range(3)])
                    if grid.find(probe) >= 0:
                        # a sibling touches this region; it must then cover all of it
                        corner = np.array([bhi[t] - 1 if dd[t] >= 0 else blo[t] for t in range(3)])
                        if grid.find(corner) < 0:
                            raise ValueError("ghost region partly covered by siblings")
                        continue
                    boxes.append((a, a, *blo.tolist(), *bhi.tolist()))
    t = np.zeros(len(boxes), dtype=BOX_DTYPE)
    for i, bx in enumerate(boxes):
        t[i]["dst"], t[i]["src"] = bx[0], bx[1]
        t[i]["lo"] = bx[2:5]
        t[i]["hi"] = bx[5:8]
    return t


def correction_faces(fine, coarse, r=2):
    """Faces of fine patches whose outside coarse cells are not covered by the
    fine level, with the coarse patch holding those cells."""
    fn, fo = np.asarray(fine["n"]), np.asarray(fine["origin"])
    cn, co = np.asarray(coarse["n"]), np.asarray(coarse["origin"])
    fgrid = _Grid(fn, fo)
    cgrid = _Grid(cn, co)
    faces = []
    for i in range(len(fn)):
        for d in range(3):
            for side in (0, 1):
                probe = fo[i].copy()
                probe[d] = fo[i][d] - 1 if side == 0 else fo[i][d] + fn[i][d]
                if fgrid.find(probe) >= 0:
                    continue
                cell = probe // r
                t = cgrid.find(cell)
                if t < 0:
                    raise ValueError("coarse cell outside a fine face is not in a coarse patch")
                last = cell.copy()
                for a in range(3):
                    if a != d:
                        last[a] = (fo[i][a] + fn[i][a]) // r - 1
                if not np.all((co[t] <= last) & (last < co[t] + cn[t])):
                    raise ValueError("a fine face spans more than one coarse patch")
                faces.append((i, d, side, t))
    t = np.zeros(len(faces), dtype=FACE_DTYPE)
    for k, f in enumerate(faces):
        t[k] = f
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
