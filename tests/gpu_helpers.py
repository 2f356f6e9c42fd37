"""Shared helpers of the GPU tests: build patch batches from host fields, run the
oracle on the same inputs, and compare."""
import numpy as np

import oracle
import paper_1307_2265_gb300 as ez
from paper_1307_2265_gb300 import synth

NG = 3


def batch_from_patches(patches, dx, flags=0):
    """patches: list of 5-field lists (ghost-zoned (z,y,x) arrays)."""
    sizes, offs, flat = [], [], [[] for _ in range(5)]
    off = 0
    for U in patches:
        nz, ny, nx = U[0].shape
        sizes.append((nx - 2 * NG, ny - 2 * NG, nz - 2 * NG))
        offs.append(off)
        off += U[0].size
        for f in range(5):
            flat[f].append(U[f].ravel())
    fields = [np.concatenate(f) for f in flat]
    table = ez.patch_table(sizes, offs, dx, flags=flags)
    return ez.PatchBatch(table, fields)


def gpu_patches(batch):
    return [[f.cpu().numpy() for f in batch.patch_fields(i)] for i in range(len(batch.table))]


def active(a):
    return a[NG:-NG, NG:-NG, NG:-NG]


def oracle_evolve_batch(patches, dx, nsteps, P, cfl=0.4, step0=0):
    """Oracle level advance: shared dt = cfl / max over patches of the CFL rate."""
    dts = []
    for s in range(nsteps):
        rate = max(oracle.cfl_rate(U, dx, P) for U in patches)
        dt = cfl / rate
        for U in patches:
            oracle.step_periodic(U, dx, dt, step0 + s, P)
        dts.append(dt)
    return dts


def gpu_evolve(batch, params, nsteps, step0=0):
    dts = []
    for s in range(nsteps):
        ez.timestep_cfl(batch, params, out=batch.dt_dev)
        dts.append(float(batch.dt_dev.item()))
        ez.step(batch, params, step0 + s, batch.dt_dev)
    return dts


def max_rel(gpu, ora, gamma):
    """Largest per-cell relative difference over the five fields (active cells).
    rho and E relative to their own value; each momentum component relative to
    |m| + rho c_s of the cell (components may pass through zero)."""
    g = [active(a) for a in gpu]
    o = [active(a) for a in ora]
    rho = o[0]
    mag = np.sqrt(o[1] ** 2 + o[2] ** 2 + o[3] ** 2)
    p = (gamma - 1.0) * (o[4] - 0.5 * mag ** 2 / rho)
    cs = np.sqrt(gamma * np.maximum(p, 1e-300) / rho)
    worst = 0.0
    for f in range(5):
        den = np.abs(o[f]) if f in (0, 4) else mag + rho * cs
        worst = max(worst, float(np.max(np.abs(g[f] - o[f]) / den)))
    return worst


def l1_rel(gpu, ora):
    """Per-field L1 relative error sum|a-b| / sum|b| over active cells."""
    return [float(np.sum(np.abs(active(a) - active(b))) / np.sum(np.abs(active(b)))) for a, b in zip(gpu, ora)]


def white_patch(n, seed, mach=1.0, sigma=0.5, gamma=5.0 / 3.0):
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    prims = synth.white_noise_prims(rng, (nz, ny, nx), sigma=sigma, mach=mach, gamma=gamma)
    return [synth.embed(f) for f in synth.prims_to_conserved(*prims, gamma)]


def with_registers(batch, nc=5):
    """Give every patch all-face and boundary-face flux registers (the layout
    of a hierarchy level), zeroed."""
    import torch
    from paper_1307_2265_gb300 import hierarchy as gh
    tab = batch.table
    a_sz, b_sz = gh.register_sizes(tab["n"], nc)
    tab["freg_all"] = np.concatenate([[0], np.cumsum(a_sz)[:-1]])
    tab["freg_bnd"] = np.concatenate([[0], np.cumsum(b_sz)[:-1]]) + int(a_sz.sum())
    batch.patches.copy_(torch.from_numpy(np.frombuffer(tab.tobytes(), dtype=np.uint8).copy()).to(batch.device))
    batch.freg = torch.zeros(int(a_sz.sum() + b_sz.sum()), dtype=torch.float64, device=batch.device)
    return batch
