"""FP64 reference of the hierarchy rebuild (test infrastructure only: the
library never imports it).

Follows the paper:
  * Sec. 3.6 (refinement criteria), three of its flagging methods:
      slope: (q_{i+1} - q_{i-1}) / (2 q_i) beyond a threshold (typically 0.3)
        for the baryon quantities, along any axis;
      shocks: a pressure jump (p_{i+1} - p_{i-1}) / min(p_{i+1}, p_{i-1}) above
        0.33 with converging flow u_{i-1} - u_{i+1} > 0 and e_i / E_i > 0.1,
        along any axis;
      baryon mass: rho dx^3 above a threshold mass.
  * Sec. 3.5 (hierarchy reconstruction): flagged cells of each grid are
    covered by rectangular regions following Berger & Rigoutsos: the smallest
    region covering the flags is adopted when its efficiency (flagged / total)
    is large enough or it is small enough; otherwise it is cut in two at the
    strongest inflection of the flag signature along the longest axis (ties to
    the cut nearest the centre; then the next-longest axes; with no inflection
    anywhere the longest axis is halved), and each part is treated the same way.
  * New grids are filled from the parent by SecondOrderA (Appendix A) and then
    overwritten by the old grids of the same level where they overlap
    (Sec. 3.1 uses the same interpolate-then-copy order for ghost zones).

Readings where the paper is silent:
  * the slope criterion takes |q_{i+1} - q_{i-1}| / (2 |q_i|) for q = rho and
    E (the conserved densities), the shock criterion the absolute pressure
    jump (shocks moving either way), p = (gamma - 1)(E - KE) and e = E - KE;
    each ratio is formed as the paper writes it, in FP64, and compared with
    its threshold;
  * flags are grown by `buffer` cells (Chebyshev distance, inside the grid)
    before clustering, and cells within `margin` of the grid's edge are then
    cleared (see the last item);
  * an inflection is a sign change of the signature's second difference
    D_i = s_{i-1} - 2 s_i + s_{i+1} between i and i+1; its strength is
    |D_{i+1} - D_i|; the cut goes between them; axes are searched longest
    first (ties: x, y, z); regions are processed depth first, the low part
    before the high part, which fixes the order of the boxes;
  * a region is small enough when it holds at most `small_cells` cells;
  * flags are dropped within 3 cells of the domain boundary on the root (the
    periodic root keeps no ghost cells for the level-1 interpolation) and
    within 1 cell of a patch's edge on deeper levels (proper nesting: the
    coarse cells outside every fine face lie in the parent, so flux correction
    reaches them).
"""
from __future__ import annotations

import numpy as np

from . import hierarchy as H

NG = 3
SLOPE, SHOCK, MASS = 1, 2, 4


def _shifted(a, axis, s):
    """Neighbour values a[i + s] along `axis` (storage (z, y, x) axes 2, 1, 0 for
    x, y, z) of the active cells of a ghost-zoned array."""
    sl = [slice(NG, -NG)] * 3
    t = 2 - axis
    sl[t] = slice(NG + s, a.shape[t] - NG + s)
    return a[tuple(sl)]


def flag_patch(U, dx, gamma, slope=0.3, shock_dp=0.33, shock_e=0.1, mass=0.0):
    """Flags (uint8, active cells (z, y, x)) of one patch whose ghost zones are
    filled: bit 0 slope, bit 1 shock, bit 2 baryon mass.  A criterion with a
    threshold <= 0 is off.  Every quantity is FP64, each ratio formed as
    Sec. 3.6 writes it:
      slope:  |q_{i+1} - q_{i-1}| / (2 |q_i|) > slope,  q = rho, E;
      shock:  |p_{i+1} - p_{i-1}| / min(p_{i+1}, p_{i-1}) > shock_dp,
              u_{i-1} - u_{i+1} > 0 and e_i / E_i > shock_e;
      mass:   rho dx^3 > mass;
    with e = E - |m|^2 / (2 rho), p = (gamma - 1) e and u = m / rho (Sec. 2.1)."""
    rho, m1, m2, m3, E = U
    shape = tuple(s - 2 * NG for s in rho.shape)
    out = np.zeros(shape, dtype=np.uint8)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        ke = 0.5 * ((m1 * m1 + m2 * m2) + m3 * m3) / rho
        e = E - ke
        p = (gamma - 1.0) * e
        mom = (m1, m2, m3)
        for ax in range(3):
            if slope > 0.0:
                for q in (rho, E):
                    qm, q0, qp = _shifted(q, ax, -1), _shifted(q, ax, 0), _shifted(q, ax, 1)
                    hit = np.abs(qp - qm) / (2.0 * np.abs(q0)) > slope
                    out[hit] |= SLOPE
            if shock_dp > 0.0:
                pm, pp = _shifted(p, ax, -1), _shifted(p, ax, 1)
                pmin = np.minimum(pm, pp)
                um = _shifted(mom[ax], ax, -1) / _shifted(rho, ax, -1)
                up = _shifted(mom[ax], ax, 1) / _shifted(rho, ax, 1)
                frac = _shifted(e, ax, 0) / _shifted(E, ax, 0)
                hit = (np.abs(pp - pm) / pmin > shock_dp) & (um - up > 0.0) & (frac > shock_e)
                out[hit] |= SHOCK
        if mass > 0.0:
            hit = _shifted(rho, 0, 0) * (dx * dx * dx) > mass
            out[hit] |= MASS
    return out


def grow(flags, buffer):
    """Flags grown by `buffer` cells in Chebyshev distance, inside the grid
    (a cube neighbourhood is separable: grow along x, then y, then z)."""
    f = flags != 0
    for t in range(3):
        for _ in range(buffer):
            g = f.copy()
            lo = [slice(None)] * 3
            hi = [slice(None)] * 3
            lo[t], hi[t] = slice(0, -1), slice(1, None)
            g[tuple(lo)] |= f[tuple(hi)]
            g[tuple(hi)] |= f[tuple(lo)]
            f = g
    return f


def cluster(flags, efficiency=0.3, small_cells=64, buffer=1, margin=0):
    """Boxes (lo, hi), x-y-z half-open in the grid's active-cell indices, that
    cover the flagged cells of one grid (flags (z, y, x)), after growing them
    by `buffer` cells and clearing those within `margin` cells of the grid's
    edge."""
    F = grow(flags, buffer) if buffer > 0 else flags != 0
    nz, ny, nx = F.shape
    if margin > 0:
        keep = np.zeros(F.shape, dtype=bool)
        keep[margin:nz - margin, margin:ny - margin, margin:nx - margin] = True
        F = F & keep
    out = []
    if not F.any():
        return out

    def count(lo, hi):
        return int(F[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]].sum())

    def shrink(lo, hi):
        sub = F[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        if not sub.any():
            return None
        nlo, nhi = list(lo), list(hi)
        for ax in range(3):
            t = 2 - ax
            other = tuple(u for u in range(3) if u != t)
            prof = sub.any(axis=other)
            idx = np.flatnonzero(prof)
            nlo[ax] = lo[ax] + int(idx[0])
            nhi[ax] = lo[ax] + int(idx[-1]) + 1
        return nlo, nhi

    def best_cut(lo, hi, ax):
        n = hi[ax] - lo[ax]
        if n < 4:
            return None
        t = 2 - ax
        sub = F[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        other = tuple(u for u in range(3) if u != t)
        s = sub.sum(axis=other).astype(np.int64)            # signature along ax
        D = s[:-2] - 2 * s[1:-1] + s[2:]                    # D[j] at index j + 1
        best = None
        for j in range(len(D) - 1):
            if D[j] * D[j + 1] < 0:
                strength = abs(int(D[j + 1]) - int(D[j]))
                c = j + 2                                    # cut between index j + 1 and j + 2
                dist = abs(2 * c - n)                        # twice the distance to the centre
                key = (-strength, dist, c)
                if best is None or key < best:
                    best = key
        return None if best is None else best[2]

    def process(lo, hi):
        r = shrink(lo, hi)
        if r is None:
            return
        lo, hi = r
        vol = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])
        if count(lo, hi) >= efficiency * vol or vol <= small_cells:
            out.append((tuple(lo), tuple(hi)))
            return
        ext = [hi[a] - lo[a] for a in range(3)]
        axes = sorted(range(3), key=lambda a: (-ext[a], a))
        cut_ax, cut = None, None
        for ax in axes:
            c = best_cut(lo, hi, ax)
            if c is not None:
                cut_ax, cut = ax, c
                break
        if cut_ax is None:
            cut_ax = axes[0]
            if ext[cut_ax] < 2:
                out.append((tuple(lo), tuple(hi)))
                return
            cut = ext[cut_ax] // 2
        mid = lo[cut_ax] + cut
        hi1 = list(hi)
        hi1[cut_ax] = mid
        lo2 = list(lo)
        lo2[cut_ax] = mid
        process(list(lo), hi1)
        process(lo2, list(hi))

    process([0, 0, 0], [nx, ny, nz])
    return out


def fill_patch_from_parent(child, parent):
    """Every cell of `child` (active and ghost) from its parent's current state
    by SecondOrderA."""
    nx, ny, nz = child["n"]
    ox, oy, oz = child["origin"]
    px, py, pz = parent["origin"]
    shape = (nz + 2 * NG, ny + 2 * NG, nx + 2 * NG)
    k, j, i = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), np.arange(shape[2]), indexing="ij")
    k, j, i = k.ravel(), j.ravel(), i.ravel()
    g = (oz + k - NG, oy + j - NG, ox + i - NG)
    G = tuple(np.floor_divide(v, H.R) for v in g)
    kk = tuple(g[t] - H.R * G[t] for t in range(3))
    P = (G[0] - pz + NG, G[1] - py + NG, G[2] - px + NG)
    off = np.arange(-1, 2)
    iz = P[0][:, None, None, None] + off[None, :, None, None]
    iy = P[1][:, None, None, None] + off[None, None, :, None]
    ix = P[2][:, None, None, None] + off[None, None, None, :]
    for f in range(len(child["U"])):          # five fields, a sixth with dual energy
        Q = parent["U"][f][iz, iy, ix]
        kids = H.second_order_a(Q, H.R)
        child["U"][f][k, j, i] = kids[np.arange(len(k)), kk[0], kk[1], kk[2]]


def copy_from_old(new, old_level):
    """Cells of `new` (active and ghost) that lie in an old patch's active box
    take that patch's value."""
    nlo, nhi = H._box_of(new)
    glo, ghi = nlo - NG, nhi + NG
    for po in old_level:
        blo, bhi = H._box_of(po)
        lo = np.maximum(glo, blo)
        hi = np.minimum(ghi, bhi)
        if np.any(lo >= hi):
            continue
        dn = [slice(lo[t] - glo[t], hi[t] - glo[t]) for t in (2, 1, 0)]
        do = [slice(lo[t] - blo[t] + NG, hi[t] - blo[t] + NG) for t in (2, 1, 0)]
        for f in range(len(new["U"])):
            new["U"][f][dn[0], dn[1], dn[2]] = po["U"][f][do[0], do[1], do[2]]


def new_boxes(levels, l, gamma, crit, clus, margin=3, nest=1):
    """Boxes of the new level l+1 as (parent index, lo, hi) in level-l cell
    indices (global), from the flags of level l's patches (ghosts filled).
    Flags within `margin` cells of the domain boundary (on the root: level-1
    ghost interpolation stays inside the periodic root) or within `nest` cells
    of the patch's edge (deeper levels: the coarse cells outside every new fine
    face lie in the parent, so flux correction reaches them) are dropped."""
    out = []
    L = levels[l]
    for pi, p in enumerate(L["patches"]):
        fl = flag_patch(p["U"][:5], L["dx"], gamma, **crit)
        for lo, hi in cluster(fl, margin=margin if l == 0 else nest, **clus):
            o = p["origin"]
            out.append((pi, tuple(o[a] + lo[a] for a in range(3)), tuple(o[a] + hi[a] for a in range(3))))
    return out


def rebuild_level(levels, l, gamma, crit, clus, margin=3, nest=1):
    """Replace level l+1 by grids covering the flagged cells of level l: each
    new patch is interpolated from its parent, then overwritten by the old
    level l+1 where they overlap.  When the boxes (and parents) are those of
    the old level, the level is kept as it is.  Level l's ghosts must be
    filled."""
    boxes = new_boxes(levels, l, gamma, crit, clus, margin, nest)
    old = levels[l + 1]["patches"]
    same = [(p["parent"], tuple(o // H.R for o in p["origin"]),
             tuple((o + n) // H.R for o, n in zip(p["origin"], p["n"]))) for p in old]
    if boxes == same:
        return boxes           # the same grids: the level stays as it is
    par = levels[l]["patches"]
    new = []
    for pi, lo, hi in boxes:
        n = tuple(H.R * (hi[a] - lo[a]) for a in range(3))
        origin = tuple(H.R * lo[a] for a in range(3))
        shape = (n[2] + 2 * NG, n[1] + 2 * NG, n[0] + 2 * NG)
        p = {"n": n, "origin": origin, "parent": pi, "U": [np.zeros(shape) for _ in par[pi]["U"]]}
        fill_patch_from_parent(p, par[pi])
        copy_from_old(p, old)
        new.append(p)
    levels[l + 1]["patches"] = new
    return boxes
