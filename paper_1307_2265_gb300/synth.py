"""Seeded synthetic inputs shared by the tests, the oracle timing leg and the benchmark.

This module draws random initial conditions and lays them out in the patch storage
format; it holds none of the PPM method's arithmetic.  The one formula here is the
definition of total energy density used to build an initial state from primitives,
E = p/(gamma-1) + rho |v|^2 / 2 (Section 2.1, total energy and ideal-gas equation of
state), applied once to the generated input, never inside a step.

Storage of one patch: five float64 arrays (rho, m_x, m_y, m_z, E), each of shape
(n_z + 2 ng, n_y + 2 ng, n_x + 2 ng) in C order, so x is the fastest index.  Ghost
cells are left at zero; the ghost-fill step fills them.

Recipes (all seeds derive from SEED_BASE + 100 * config + patch index):
  * single grid, white noise: rho lognormal exp(sigma g - sigma^2/2) with iid unit
    normal g, p uniform, velocity components iid N(0, (mach c0)^2 / 3) so the rms
    Mach number is `mach` with c0 = sqrt(gamma p / 1).
  * single grid, turbulent: each velocity component a Gaussian random field with
    P(k) ~ k^-4 (FFT filtered white noise), scaled to rms Mach `mach`; rho lognormal
    on an independent k^-4 field with sigma = 1.
  * batched level: per-axis active sizes uniform in {8..64}; each patch its own
    white-noise realisation as above.
  * strong-shock grid: lognormal background clipped to [1e-2, 1e2], p = 1e-3,
    seeded spheres of radius 4..24 cells with p up to 1e3, v = 0.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1307_2265
NG = 3
FIELDS = ("rho", "mx", "my", "mz", "E")


def rng_for(config: int, index: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + 100 * config + index))


def lognormal(g: np.ndarray, sigma: float) -> np.ndarray:
    """Mean-one lognormal field from a unit-variance Gaussian field g."""
    return np.exp(sigma * g - 0.5 * sigma * sigma)


def grf_kpow(rng: np.random.Generator, shape, power: float = -4.0) -> np.ndarray:
    """Zero-mean, unit-variance periodic Gaussian random field with P(k) ~ k^power."""
    white = rng.standard_normal(shape)
    fk = np.fft.rfftn(white)
    ks = [np.fft.fftfreq(s) * s for s in shape[:-1]] + [np.fft.rfftfreq(shape[-1]) * shape[-1]]
    grids = np.meshgrid(*ks, indexing="ij")
    k2 = sum(g * g for g in grids)
    k2[(0,) * len(shape)] = 1.0
    amp = k2 ** (power / 4.0)          # sqrt(P(k)) = k^(power/2)
    amp[(0,) * len(shape)] = 0.0
    f = np.fft.irfftn(fk * amp, s=shape, axes=tuple(range(len(shape))))
    f -= f.mean()
    return f / f.std()


def white_noise_prims(rng, shape, sigma=0.5, mach=1.0, gamma=5.0 / 3.0, p0=1.0):
    """(rho, vx, vy, vz, p) arrays of `shape` (z, y, x) for the white-noise recipe."""
    rho = lognormal(rng.standard_normal(shape), sigma)
    c0 = np.sqrt(gamma * p0 / 1.0)
    sd = mach * c0 / np.sqrt(3.0)
    v = [rng.standard_normal(shape) * sd for _ in range(3)]
    p = np.full(shape, p0)
    return rho, v[0], v[1], v[2], p


def turbulent_prims(rng, shape, mach=3.0, sigma=1.0, gamma=5.0 / 3.0, p0=1.0):
    rho = lognormal(grf_kpow(rng, shape), sigma)
    c0 = np.sqrt(gamma * p0)
    v = [grf_kpow(rng, shape) for _ in range(3)]
    rms = np.sqrt(np.mean(v[0] ** 2 + v[1] ** 2 + v[2] ** 2))
    v = [vi * (mach * c0 / rms) for vi in v]
    p = np.full(shape, p0)
    return rho, v[0], v[1], v[2], p


def blast_prims(rng, shape, nblast=16, p_bg=1e-3, p_max=1e3, r_min=4, r_max=24):
    """Blast spheres on a clipped lognormal background (density contrast 1e4,
    pressure ratio up to p_max / p_bg), at rest.  Sphere centres, radii and
    pressures are seeded; distances are periodic (minimum image, in cell
    indices).  Each sphere touches only the cells of its bounding box."""
    rho = np.clip(lognormal(grf_kpow(rng, shape), 1.0), 1e-2, 1e2)
    p = np.full(shape, p_bg)
    dims = np.array(shape)
    for _ in range(nblast):
        c = rng.uniform(0, 1, 3) * dims
        r = rng.uniform(r_min, r_max)
        pb = p_max * 10.0 ** rng.uniform(-2.0, 0.0)
        idx, dist = [], []
        for a in range(3):
            s = int(dims[a])
            i = np.unique(np.mod(np.arange(int(np.floor(c[a] - r)), int(np.ceil(c[a] + r)) + 1), s))
            d = np.abs(i - c[a])
            idx.append(i)
            dist.append(np.minimum(d, s - d))
        inside = (dist[0][:, None, None] ** 2 + dist[1][None, :, None] ** 2 + dist[2][None, None, :] ** 2) <= r * r
        box = np.ix_(*idx)
        sub = p[box]
        p[box] = np.where(inside, np.maximum(sub, pb), sub)
    zero = np.zeros(shape)
    return rho, zero, zero.copy(), zero.copy(), p


def prims_to_conserved(rho, vx, vy, vz, p, gamma):
    """Initial-state construction: conserved (rho, m, E) from primitives."""
    E = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz)
    return rho.copy(), rho * vx, rho * vy, rho * vz, E


def embed(active: np.ndarray, ng: int = NG) -> np.ndarray:
    """Place an active (z, y, x) block inside zeroed ghost storage."""
    nz, ny, nx = active.shape
    out = np.zeros((nz + 2 * ng, ny + 2 * ng, nx + 2 * ng))
    out[ng:ng + nz, ng:ng + ny, ng:ng + nx] = active
    return out


def single_grid(n, recipe="white", config=1, gamma=5.0 / 3.0, ng=NG, **kw):
    """Five ghost-zoned float64 fields for one periodic grid of n = (nx, ny, nz) cells."""
    nx, ny, nz = n
    rng = rng_for(config)
    shape = (nz, ny, nx)
    if recipe == "white":
        prims = white_noise_prims(rng, shape, gamma=gamma, **kw)
    elif recipe == "turbulent":
        prims = turbulent_prims(rng, shape, gamma=gamma, **kw)
    elif recipe == "blast":
        prims = blast_prims(rng, shape, **kw)
    else:
        raise ValueError(recipe)
    return [embed(f, ng) for f in prims_to_conserved(*prims, gamma)]


def patch_sizes(npatch, config=3, lo=8, hi=64):
    """Per-axis active sizes (nx, ny, nz), uniform integers in [lo, hi]."""
    rng = rng_for(config, 10 ** 6)
    return rng.integers(lo, hi + 1, size=(npatch, 3))


def batched_level(npatch, config=3, gamma=5.0 / 3.0, lo=8, hi=64, ng=NG, sizes=None):
    """A batch of independent white-noise patches.

    Returns (sizes[npatch,3] as (nx,ny,nz), offsets[npatch], five flat float64 arrays)
    with each patch stored contiguously per field at its offset.
    """
    if sizes is None:
        sizes = patch_sizes(npatch, config, lo, hi)
    sizes = np.asarray(sizes, dtype=np.int64)
    vols = np.prod(sizes + 2 * ng, axis=1)
    offsets = np.concatenate([[0], np.cumsum(vols)[:-1]]).astype(np.int64)
    total = int(vols.sum())
    flat = [np.zeros(total) for _ in range(5)]
    for i, (nx, ny, nz) in enumerate(sizes):
        rng = rng_for(config, i)
        prims = white_noise_prims(rng, (int(nz), int(ny), int(nx)), gamma=gamma)
        cons = prims_to_conserved(*prims, gamma)
        for f in range(5):
            blk = embed(cons[f], ng)
            flat[f][offsets[i]:offsets[i] + blk.size] = blk.ravel()
    return sizes, offsets, flat


def patch_view(flat, off, size, ng=NG):
    nx, ny, nz = (int(s) for s in size)
    cnt = (nx + 2 * ng) * (ny + 2 * ng) * (nz + 2 * ng)
    return flat[off:off + cnt].reshape(nz + 2 * ng, ny + 2 * ng, nx + 2 * ng)


def riemann_states(rng, n, log_rho_sd=1.0, mach=1.0, log_p_sd=1.0, gamma=5.0 / 3.0):
    """Random left/right Riemann states (rhoL, uL, pL, rhoR, uR, pR) for solver tests."""
    rl = np.exp(rng.normal(0, log_rho_sd, n))
    rr = np.exp(rng.normal(0, log_rho_sd, n))
    pl = np.exp(rng.normal(0, log_p_sd, n))
    pr = np.exp(rng.normal(0, log_p_sd, n))
    cl = np.sqrt(gamma * pl / rl)
    cr = np.sqrt(gamma * pr / rr)
    ul = rng.normal(0, mach, n) * cl
    ur = rng.normal(0, mach, n) * cr
    return rl, ul, pl, rr, ur, pr


# ---------------------------------------------------------------------------
# static refinement hierarchies (geometry only)
# ---------------------------------------------------------------------------
def _compose(length, sizes, rng):
    """Random split of `length` into parts drawn from `sizes` (all even)."""
    sizes = sorted(sizes)
    parts = []
    left = length
    while left > 0:
        opts = [s for s in sizes if s == left or (left - s) >= sizes[0]]
        opts = [s for s in opts if _composable(left - s, sizes)]
        if not opts:
            raise ValueError(f"cannot split {length} into {sizes}")
        s = int(rng.choice(opts))
        parts.append(s)
        left -= s
    return parts


def _composable(n, sizes):
    ok = [False] * (n + 1)
    ok[0] = True
    for v in range(1, n + 1):
        ok[v] = any(v >= s and ok[v - s] for s in sizes)
    return ok[n]


def hierarchy_layout(root_n, regions, sizes, seed=0, r=2):
    """Static nested refinement: level 0 is one root patch of root_n^3 cells;
    level l >= 1 covers the box [a_l, b_l)^3 of root cells, tiled by the tensor
    product of per-axis cuts with part lengths from `sizes`.  Every level-(l+1)
    patch lies inside one level-l patch (its parent), and patch edges sit on
    parent cell boundaries (all sizes even).

    regions: [(a_1, b_1), (a_2, b_2), ...] in root cells, nested.
    Returns a list of levels, each {"n": int array [P, 3] (nx, ny, nz),
    "origin": int array [P, 3] (global index of the first active cell at that
    level), "parent": int array [P] (-1 for the root), "segs": per-axis segment
    lists}.
    """
    rng = np.random.default_rng(SEED_BASE + 500 + seed)
    levels = [{"n": np.array([[root_n] * 3]), "origin": np.zeros((1, 3), dtype=np.int64),
               "parent": np.array([-1]), "segs": [[(0, root_n)]] * 3}]
    for l, (a, b) in enumerate(regions, start=1):
        scale = r ** l
        lo, hi = a * scale, b * scale
        # breakpoints: the parent level's cut positions inside the region (doubled)
        # and the boundaries of every deeper region at this level
        deeper = [(aa * scale, bb * scale) for (aa, bb) in regions[l:]]
        segs_axes = []
        for ax in range(3):
            parent_cuts = sorted({x * r for seg in levels[l - 1]["segs"][ax] for x in seg})
            bps = {lo, hi} | {x for x in parent_cuts if lo < x < hi}
            for (dl, dh) in deeper:
                bps |= {dl, dh}
            bps = sorted(x for x in bps if lo <= x <= hi)
            segs = []
            for s0, s1 in zip(bps[:-1], bps[1:]):
                x = s0
                for part in _compose(s1 - s0, sizes, rng):
                    segs.append((x, x + part))
                    x += part
            segs_axes.append(segs)
        ns, origins, parents = [], [], []
        prev = levels[l - 1]
        pindex = {tuple(int(v) for v in o): i for i, o in enumerate(prev["origin"])}
        pstarts = [np.array(sorted({sg[0] for sg in prev["segs"][a]})) for a in range(3)]
        for sz in segs_axes[2]:
            for sy in segs_axes[1]:
                for sx in segs_axes[0]:
                    o = np.array([sx[0], sy[0], sz[0]])
                    n = np.array([sx[1] - sx[0], sy[1] - sy[0], sz[1] - sz[0]])
                    # parent: the level-(l-1) patch whose active box contains this one
                    key = tuple(int(pstarts[a][np.searchsorted(pstarts[a], o[a] // r, side="right") - 1])
                                for a in range(3))
                    pi = pindex.get(key, -1)
                    po, pn = prev["origin"][pi], prev["n"][pi]
                    if pi < 0 or not np.all((po * r <= o) & (o + n <= (po + pn) * r)):
                        raise ValueError("patch not enclosed by exactly one parent")
                    ns.append(n)
                    origins.append(o)
                    parents.append(int(pi))
        levels.append({"n": np.array(ns), "origin": np.array(origins, dtype=np.int64),
                       "parent": np.array(parents), "segs": segs_axes})
    return levels


def hierarchy_fields(layout, config=5, gamma=5.0 / 3.0, ng=NG):
    """White-noise initial state on the root (rms Mach 1, lognormal rho); finer
    levels start from their parent's values (each fine cell takes its parent
    cell's conserved state).  Returns per level a list of per-patch field lists."""
    root = single_grid(tuple(int(v) for v in layout[0]["n"][0]), "white", config=config, gamma=gamma, ng=ng)
    out = [[root]]
    for l in range(1, len(layout)):
        L = layout[l]
        prev = layout[l - 1]
        fields = []
        for i in range(len(L["n"])):
            nx, ny, nz = (int(v) for v in L["n"][i])
            o = L["origin"][i]
            p = int(L["parent"][i])
            po = prev["origin"][p]
            PU = out[l - 1][p]
            c0 = o // 2 - po + ng           # first covering parent cell (storage index)
            fl = []
            for f in range(5):
                blk = PU[f][c0[2]:c0[2] + nz // 2, c0[1]:c0[1] + ny // 2, c0[0]:c0[0] + nx // 2]
                act = blk.repeat(2, axis=0).repeat(2, axis=1).repeat(2, axis=2)
                fl.append(embed(act, ng))
            fields.append(fl)
        out.append(fields)
    return out


def cold_contact_fields(layout, root_n, gamma=1.4, eps=2.0, v=(8.0, 6.0, 5.0), ng=NG):
    """A density wave rho = 1 + 0.5 sin(2 pi x) cos(2 pi y) sin(2 pi (z + 0.1))
    at uniform pressure 1 carried by the uniform velocity v (Mach 6.7 to 11.6
    for gamma 1.4: internal energy 2.6% to 7.3% of E), sampled at each patch's
    cell centres on every level of `layout` (root cell size 1 / root_n).  A
    sixth field, the gas energy, is eps * rho.  Per level a list of per-patch
    field lists (ghost zones zero)."""
    out = []
    for l, L in enumerate(layout):
        dx = 1.0 / (root_n * 2 ** l)
        per = []
        for i in range(len(L["n"])):
            nx, ny, nz = (int(c) for c in L["n"][i])
            o = L["origin"][i]
            z, y, x = np.meshgrid((o[2] + np.arange(nz) + 0.5) * dx, (o[1] + np.arange(ny) + 0.5) * dx,
                                  (o[0] + np.arange(nx) + 0.5) * dx, indexing="ij")
            rho = 1.0 + 0.5 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) * np.sin(2 * np.pi * (z + 0.1))
            one = np.ones_like(rho)
            U = [embed(f, ng) for f in prims_to_conserved(rho, v[0] * one, v[1] * one, v[2] * one, one, gamma)]
            U.append(embed(eps * rho, ng))
            per.append(U)
        out.append(per)
    return out
