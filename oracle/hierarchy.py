"""FP64 reference of the AMR hierarchy operations around the sweep (test
infrastructure only).

Follows the paper:
  * Sec. 3.1: ghost zones of a subgrid are first interpolated from the parent,
    then overwritten by copies from siblings; the root grid is periodic.
  * Appendix A (SecondOrderA): corner values are averages of the 8 parent cells
    around each corner; minmod slopes are taken along the four cell diagonals;
    the 3-D consistency fix-up uses s, chi_n and f; the slopes are converted to
    f_x, f_y, f_z; children get Q0 + sum_axes ((i + (1-r)/2)/r) f_axis.
  * Sec. 3.3 (projection): coarse = r^-3 sum of the covering fine cells.
  * Sec. 3.4 (flux correction): coarse cells next to a fine region get
    dt_c F_coarse replaced by the time- and area-summed fine fluxes.
  * Sec. 3 (W-cycle): a level subcycles until it reaches its parent's time,
    dt_l = min(CFL_l, t_parent - t_l); after the fine level catches up, flux
    correction then projection.

Readings where the paper is silent or garbled:
  * the printed adjustment factor f has the sign that would make the adjusted
    diagonal slopes imply -s' dQ0; the sign that makes them imply s' dQ0 is
    taken: f = (s' dQ0 - sum (1-chi_n) dQ_n) / (sum chi_n dQ_n + eps), eps = 1e-300;
  * 0 <= s <= 1 needs no adjustment; where dQ0 = 0 all slopes are set to zero;
  * the five conserved fields are interpolated independently;
  * parent values are interpolated linearly in time between the parent's state
    at the start and end of its step before the spatial interpolation;
  * the sum of each corner's 8 cells runs z-major, then y, then x, and is
    scaled by 1/8; child values add the x, y, z terms in that order;
  * with dual energy (Sec. 4.1.1) the gas energy rho e is a sixth field that
    is interpolated, copied, projected and flux-corrected like the conserved
    ones; its correction swaps only its advected flux (the -p div v source is a
    zone term, not a face flux), and neither the time step nor the composite
    totals use it.

Data model: a level is a list of patches, each a dict with
  n (nx, ny, nz), origin (global index of the first active cell at this level),
  U (five ghost-zoned arrays, (z, y, x), and the gas energy as a sixth when the
  dual-energy option is on), parent (index into the parent level or -1).
"""
from __future__ import annotations

import numpy as np

import oracle

NG = 3
R = 2
EPS = 1e-300


def minmod(a, b):
    """0 where a b < 0, else min(|a|, |b|) with the sign of a."""
    m = np.where(np.abs(a) < np.abs(b), np.abs(a), np.abs(b))
    out = np.where(a > 0.0, m, np.where(a < 0.0, -m, 0.0))
    return np.where(a * b < 0.0, 0.0, out)


def corners(Q):
    """Corner averages of a (..., 3, 3, 3) neighbourhood; returns dict keyed by
    (sz, sy, sx) in {0, 1} (0 = minus side, 1 = plus side)."""
    out = {}
    for sz in (0, 1):
        for sy in (0, 1):
            for sx in (0, 1):
                acc = np.zeros(Q.shape[:-3])
                for dz in (0, 1):
                    for dy in (0, 1):
                        for dx in (0, 1):
                            acc = acc + Q[..., sz + dz, sy + dy, sx + dx]
                out[(sz, sy, sx)] = acc * 0.125
    return out


# plus corner (sz, sy, sx) of each diagonal; the minus corner is its opposite
DIAG_PLUS = [(1, 1, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1)]


def second_order_a(Q, r=R):
    """Children (..., r, r, r) [kz, ky, kx] of the centre cell of each
    (..., 3, 3, 3) parent neighbourhood Q."""
    Q0 = Q[..., 1, 1, 1]
    C = corners(Q)
    dQ = []
    for (pz, py, px) in DIAG_PLUS:
        plus = C[(pz, py, px)]
        minus = C[(1 - pz, 1 - py, 1 - px)]
        dQ.append(minmod(plus - Q0, Q0 - minus))
    d0, d1, d2, d3 = dQ
    zero0 = d0 == 0.0
    safe0 = np.where(zero0, 1.0, d0)
    s = (d1 + d2 + d3) / safe0
    adjust = ~zero0 & ((s < 0.0) | (s > 1.0))
    sp = np.minimum(np.maximum(s, 0.0), 1.0)
    chi = []
    for dn in (d1, d2, d3):
        ratio = dn / safe0
        chi.append(np.where(s < 0.0, ratio < 0.0, ratio > 0.0).astype(np.float64))
    num = sp * d0 - (((1.0 - chi[0]) * d1 + (1.0 - chi[1]) * d2) + (1.0 - chi[2]) * d3)
    den = ((chi[0] * d1 + chi[1] * d2) + chi[2] * d3) + EPS
    f = num / den
    adj = [np.where(adjust, f * c * dn + (1.0 - c) * dn, dn) for c, dn in zip(chi, (d1, d2, d3))]
    adj = [np.where(zero0, 0.0, a) for a in adj]
    a1, a2, a3 = adj
    fx = a2 + a3
    fy = a1 + a3
    fz = a1 + a2
    out = np.empty(Q.shape[:-3] + (r, r, r))
    for kz in range(r):
        cz = (kz + (1.0 - r) / 2.0) / r
        for ky in range(r):
            cy = (ky + (1.0 - r) / 2.0) / r
            for kx in range(r):
                cx = (kx + (1.0 - r) / 2.0) / r
                out[..., kz, ky, kx] = ((Q0 + cx * fx) + cy * fy) + cz * fz
    return out


def _active(a):
    return a[NG:-NG, NG:-NG, NG:-NG]


def _box_of(p):
    lo = np.array(p["origin"])
    return lo, lo + np.array(p["n"])


def fill_from_parent(child, parent, parent_old, w, r=R):
    """Interpolate every ghost cell of `child` from its parent: parent cells are
    first interpolated in time (weight w between parent_old and parent), then
    SecondOrderA gives the child cell's value."""
    nx, ny, nz = child["n"]
    ox, oy, oz = child["origin"]
    px, py, pz = parent["origin"]
    shape = (nz + 2 * NG, ny + 2 * NG, nx + 2 * NG)
    k, j, i = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), np.arange(shape[2]), indexing="ij")
    a = (k - NG, j - NG, i - NG)
    ghost = ~((a[0] >= 0) & (a[0] < nz) & (a[1] >= 0) & (a[1] < ny) & (a[2] >= 0) & (a[2] < nx))
    k, j, i = k[ghost], j[ghost], i[ghost]
    g = (oz + k - NG, oy + j - NG, ox + i - NG)
    G = tuple(np.floor_divide(v, r) for v in g)
    kk = tuple(g[t] - r * G[t] for t in range(3))
    P = (G[0] - pz + NG, G[1] - py + NG, G[2] - px + NG)
    off = np.arange(-1, 2)
    iz = P[0][:, None, None, None] + off[None, :, None, None]
    iy = P[1][:, None, None, None] + off[None, None, :, None]
    ix = P[2][:, None, None, None] + off[None, None, None, :]
    for f in range(len(child["U"])):          # five fields, a sixth with dual energy
        old = parent_old["U"][f][iz, iy, ix]
        new = parent["U"][f][iz, iy, ix]
        Q = old + w * (new - old)
        kids = second_order_a(Q, r)
        child["U"][f][k, j, i] = kids[np.arange(len(k)), kk[0], kk[1], kk[2]]


def copy_from_siblings(level):
    """Ghost cells lying in a sibling's active box take the sibling's value."""
    for a, pa in enumerate(level):
        alo, ahi = _box_of(pa)
        glo, ghi = alo - NG, ahi + NG
        for b, pb in enumerate(level):
            if a == b:
                continue
            blo, bhi = _box_of(pb)
            lo = np.maximum(glo, blo)
            hi = np.minimum(ghi, bhi)
            if np.any(lo >= hi):
                continue
            # storage slices (z, y, x)
            da = [slice(lo[t] - glo[t], hi[t] - glo[t]) for t in (2, 1, 0)]
            db = [slice(lo[t] - blo[t] + NG, hi[t] - blo[t] + NG) for t in (2, 1, 0)]
            for f in range(len(pa["U"])):
                pa["U"][f][da[0], da[1], da[2]] = pb["U"][f][db[0], db[1], db[2]]


def fill_level(levels, l, parent_old, w):
    """SetBoundaryValues of level l: the root's external boundaries (periodic
    unless the level carries "bc", Sec. 3.1), else parent interpolation then
    sibling copies."""
    if l == 0:
        bc = levels[0].get("bc")
        for p in levels[0]["patches"]:
            if bc is None:
                oracle.fill_periodic(p["U"])
            else:
                oracle.fill_boundary(p["U"], bc)
        return
    parents = levels[l - 1]["patches"]
    for p in levels[l]["patches"]:
        fill_from_parent(p, parents[p["parent"]], parent_old[p["parent"]], w)
    copy_from_siblings(levels[l]["patches"])


def level_rate(levels, l, P):
    dx = levels[l]["dx"]
    return max(oracle.cfl_rate(p["U"][:5], [dx] * 3, P) for p in levels[l]["patches"])


def step_level(levels, l, dt, step_index, P, has_children):
    """Three sweeps with once-per-step ghost coverage; records face fluxes:
    every face of patches with children (coarse register), dt x boundary-face
    fluxes accumulated for patches with a parent (fine register)."""
    dx = levels[l]["dx"]
    order = (0, 1, 2) if step_index % 2 == 0 else (2, 1, 0)
    for p in levels[l]["patches"]:
        n = p["n"]
        N = [n[a] + 2 * NG for a in range(3)]
        done = [False] * 3
        for d in order:
            lo = [NG if done[a] else 0 for a in range(3)]
            hi = [NG + n[a] if done[a] else N[a] for a in range(3)]
            ge = p["U"][5] if len(p["U"]) == 6 else None
            F, _ = oracle.sweep_fluxes(p["U"][:5], [dx] * 3, d, dt, lo, hi, P, ge=ge)
            if has_children:
                p.setdefault("Fc", {})[d] = F
            if p["parent"] >= 0:
                reg = p.setdefault("Ff", {})
                if d not in reg:
                    reg[d] = np.zeros((F.shape[0], F.shape[1], 2, F.shape[3]))
                reg[d][:, :, 0, :] += dt * F[:, :, 0, :]
                reg[d][:, :, 1, :] += dt * F[:, :, -1, :]
            done[d] = True


def _field_of(d, v):
    """Conserved-field index of pencil component v for a sweep along d."""
    a1 = 1 if d == 0 else 0
    a2 = 1 if d == 2 else 2
    return (0, 1 + d, 1 + a1, 1 + a2, 4, 5)[v]


def flux_correct(levels, l, dt_c, r=R):
    """Correct level-l cells that share a face with a level-(l+1) patch."""
    coarse = levels[l]["patches"]
    dxc = levels[l]["dx"]
    for fp in levels[l + 1]["patches"]:
        par = coarse[fp["parent"]]
        fo = np.array(fp["origin"])
        fn = np.array(fp["n"])
        po = np.array(par["origin"])
        for d in range(3):
            a1 = 1 if d == 0 else 0
            a2 = 1 if d == 2 else 2
            Fc = par["Fc"][d]           # [n_a2, n_a1, n_d + 1, 5 or 6] of the parent
            Ff = fp["Ff"][d]            # [fn_a2, fn_a1, 2, 5 or 6]
            for side in (0, 1):
                X = (fo[d] + (fn[d] if side else 0)) // r      # coarse face index (global)
                cell = X - 1 if side == 0 else X                # coarse cell outside the fine patch
                fc = X - po[d]                                  # face index within the parent
                for q2 in range(fn[a2] // r):
                    for q1 in range(fn[a1] // r):
                        c1 = fo[a1] // r + q1
                        c2 = fo[a2] // r + q2
                        fine = (((Ff[r * q2, r * q1, side] + Ff[r * q2, r * q1 + 1, side])
                                 + Ff[r * q2 + 1, r * q1, side]) + Ff[r * q2 + 1, r * q1 + 1, side]) * (1.0 / (r * r))
                        coarse_f = Fc[c2 - po[a2], c1 - po[a1], fc]
                        delta = (dt_c * coarse_f - fine) / dxc
                        # the coarse patch holding the corrected cell
                        g = [0, 0, 0]
                        g[d], g[a1], g[a2] = cell, c1, c2
                        for tp in coarse:
                            lo, hi = _box_of(tp)
                            if all(lo[t] <= g[t] < hi[t] for t in range(3)):
                                s = [g[t] - lo[t] + NG for t in range(3)]
                                for v in range(len(delta)):
                                    f = _field_of(d, v)
                                    if side == 0:
                                        tp["U"][f][s[2], s[1], s[0]] += delta[v]
                                    else:
                                        tp["U"][f][s[2], s[1], s[0]] -= delta[v]
                                break


def project(levels, l, r=R):
    """Coarse cells covered by level l+1 become the mean of their r^3 children."""
    coarse = levels[l]["patches"]
    for fp in levels[l + 1]["patches"]:
        par = coarse[fp["parent"]]
        fo = np.array(fp["origin"])
        po = np.array(par["origin"])
        nx, ny, nz = fp["n"]
        c0 = fo // r - po + NG
        for f in range(len(fp["U"])):
            a = _active(fp["U"][f])
            s = np.zeros((nz // r, ny // r, nx // r))
            for kz in range(r):
                for ky in range(r):
                    for kx in range(r):
                        s = s + a[kz::r, ky::r, kx::r]
            par["U"][f][c0[2]:c0[2] + nz // r, c0[1]:c0[1] + ny // r, c0[0]:c0[0] + nx // r] = s * (1.0 / r ** 3)


def _weight(levels, l):
    """Time weight of level l's current time within its parent's last step."""
    if l == 0:
        return 0.0
    par = levels[l - 1]
    return (levels[l]["t"] - par["t_old"]) / (par["t"] - par["t_old"])


def evolve_level(levels, l, t_parent, P, cfl=0.4, log=None, rebuild=None):
    """Advance level l until it reaches t_parent (W-cycle recursion).  Ghosts
    are set before every step (so sibling copies and coverage keep the fluxes
    of shared faces identical) and again after it, before the finer level
    interpolates from this level's new state.  With `rebuild` (a dict of
    oracle.amr.rebuild_level's gamma, crit, clus), every step of a level with
    children ends, after flux correction and projection, by rebuilding the
    finer levels from flags (Sec. 3, RebuildHierarchy in EvolveLevel)."""
    L = levels[l]
    has_children = l + 1 < len(levels)
    if not L["patches"]:
        L["t"] = t_parent                # a level without grids has nothing to advance
        return
    while L["t"] < t_parent * (1 - 1e-14):
        fill_level(levels, l, levels[l - 1].get("old") if l > 0 else None, _weight(levels, l))
        if l == 0:
            dt = t_parent - L["t"]
        else:
            dt = min(cfl / level_rate(levels, l, P), t_parent - L["t"])
        if has_children:
            L["old"] = [{"U": [f.copy() for f in p["U"]]} for p in L["patches"]]
            L["t_old"] = L["t"]
        step_level(levels, l, dt, L["step"], P, has_children)
        L["t"] += dt
        L["step"] += 1
        if log is not None:
            log.append((l, dt))
        if has_children:
            fill_level(levels, l, levels[l - 1].get("old") if l > 0 else None, _weight(levels, l))
            for fp in levels[l + 1]["patches"]:
                fp.pop("Ff", None)
            evolve_level(levels, l + 1, L["t"], P, cfl, log, rebuild)
            flux_correct(levels, l, dt)
            project(levels, l)
            if rebuild is not None:
                from . import amr
                fill_level(levels, l, levels[l - 1].get("old") if l > 0 else None, _weight(levels, l))
                for m in range(l, len(levels) - 1):
                    amr.rebuild_level(levels, m, **rebuild)
    # the loop stops within 1e-14 of the parent's time; the level has reached it
    L["t"] = t_parent


def root_step(levels, P, cfl=0.4, log=None, rebuild=None):
    """One root step: dt_0 from the root CFL rule, then the W-cycle."""
    rate = level_rate(levels, 0, P)
    dt0 = cfl / rate
    t_end = levels[0]["t"] + dt0
    evolve_level(levels, 0, t_end, P, cfl, log, rebuild)
    return dt0


def composite_totals(levels, r=R):
    """Sum of each conserved field x cell volume over cells not covered by a
    finer level (the conserved totals of the composite grid)."""
    tot = np.zeros(5)
    for l, L in enumerate(levels):
        vol = L["dx"] ** 3
        for pi, p in enumerate(L["patches"]):
            mask = np.ones(tuple(reversed(p["n"])), dtype=bool)
            if l + 1 < len(levels):
                for fp in levels[l + 1]["patches"]:
                    if fp["parent"] != pi:
                        continue
                    fo = np.array(fp["origin"]) // r - np.array(p["origin"])
                    fn = np.array(fp["n"]) // r
                    mask[fo[2]:fo[2] + fn[2], fo[1]:fo[1] + fn[1], fo[0]:fo[0] + fn[0]] = False
            for f in range(5):
                tot[f] += vol * float(np.sum(_active(p["U"][f])[mask]))
    return tot


def make_levels(layout, fields, root_dx, root_bc=None):
    """Level dicts of the oracle's W-cycle driver from a synth.hierarchy_layout and its
    fields (copied); root_bc: external boundaries (bc_x, bc_y, bc_z) of the
    root grid, or None for periodic."""
    levels = []
    for l, L in enumerate(layout):
        patches = []
        for i in range(len(L["n"])):
            patches.append({"n": tuple(int(v) for v in L["n"][i]),
                            "origin": tuple(int(v) for v in L["origin"][i]),
                            "parent": int(L["parent"][i]),
                            "U": [f.copy() for f in fields[l][i]]})
        levels.append({"patches": patches, "dx": root_dx / R ** l, "t": 0.0, "step": 0})
    if root_bc is not None:
        levels[0]["bc"] = tuple(root_bc)
    return levels
