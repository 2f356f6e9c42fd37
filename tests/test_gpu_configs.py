"""Full-size parity of the single-grid workloads against the FP64 oracle.

* Turbulent grid: 256^3 periodic, k^-4 Gaussian random velocity at rms Mach 3,
  lognormal rho (sigma 1), uniform p, gamma 5/3, 20 steps at CFL 0.4.  FP64 path:
  bit-identical to the oracle, timestep for timestep.  FP32 path on the
  oracle's timesteps: per-field L1 relative error <= 1e-4 (the FP32 bound of the
  parity rule); the L1 and max relative errors are printed.
* Blast grid: 512^3 periodic, sixteen blast spheres (p up to 1e3 over 1e-3,
  density contrast 1e4), 2 steps.  FP64 path bit-identical; plain and learned
  FP32 paths within the same L1 bound of the oracle and within 1e-5 of each
  other (the learned guess only moves Newton's start), with no more Newton
  iterations for the gated learned guess than for the plain one (in the
  quiescent background the plain guess is exact, and the gate keeps it).
The oracle runs on the host cores (OpenMP over pencils).
"""
import numpy as np
import pytest

import oracle
import paper_1307_2265_gb300 as ez
from gpu_helpers import oracle_evolve_batch
from paper_1307_2265_gb300 import synth, train_guess

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


def _errors(got, ref):
    """Per-field L1 relative error and largest per-cell relative difference
    (rho, E against their value; momenta against |m| + rho c_s), on the device."""
    import torch
    rho = ref[0]
    mag = torch.sqrt(ref[1] ** 2 + ref[2] ** 2 + ref[3] ** 2)
    p = (G - 1.0) * (ref[4] - 0.5 * mag ** 2 / rho)
    cs = torch.sqrt(G * torch.clamp(p, min=1e-300) / rho)
    l1, worst = [], 0.0
    for f in range(5):
        d = (got[f] - ref[f]).abs()
        l1.append(float(d.sum() / ref[f].abs().sum()))
        worst = max(worst, float((d / (ref[f].abs() if f in (0, 4) else mag + rho * cs)).max()))
    return l1, worst


def _active(batch):
    return [f[3:-3, 3:-3, 3:-3] for f in batch.patch_fields(0)]


def _run(U0, n, params, nsteps, dts=None):
    """nsteps GPU steps of the periodic grid; own device CFL timestep unless the
    host timesteps dts are given.  Returns (batch, timesteps used)."""
    import torch
    table = ez.patch_table([(n, n, n)], [0], [1.0 / n] * 3, flags=ez.PATCH_PERIODIC)
    b = ez.PatchBatch(table, [f.ravel() for f in U0])
    used = []
    for s in range(nsteps):
        if dts is None:
            ez.timestep_cfl(b, params, out=b.dt_dev)
        else:
            b.dt_dev.fill_(dts[s])
        used.append(float(b.dt_dev.item()))
        ez.step(b, params, s, b.dt_dev)
    torch.cuda.synchronize()
    return b, used


def _oracle(U0, n, nsteps):
    import torch
    ora = [[f.copy() for f in U0]]
    dts = oracle_evolve_batch(ora, [1.0 / n] * 3, nsteps, oracle.Params(gamma=G))
    ref = [torch.from_numpy(np.ascontiguousarray(f[3:-3, 3:-3, 3:-3])).cuda() for f in ora[0]]
    return dts, ref


def _bitwise(b, ref):
    import torch
    return all(bool(torch.equal(a, r)) for a, r in zip(_active(b), ref))


def test_turbulent_grid_256_twenty_steps():
    n, nsteps = 256, 20
    U0 = synth.single_grid((n, n, n), "turbulent", config=2, gamma=G)
    dts, ref = _oracle(U0, n, nsteps)
    b64, dts64 = _run(U0, n, ez.Params(gamma=G, precision=ez.FP64), nsteps)
    assert dts64 == dts
    assert _bitwise(b64, ref)
    st = b64.read_status()
    assert st["nan"] == 0 and st["newton_nonconv"] == 0
    del b64
    b32, _ = _run(U0, n, ez.Params(gamma=G, precision=ez.FP32), nsteps, dts)
    l1, worst = _errors(_active(b32), ref)
    print(f"\nturbulent 256^3 x 20, FP32 vs oracle: L1 rel {['%.2e' % e for e in l1]}, max rel {worst:.2e}")
    assert max(l1) <= 1e-4, l1
    assert b32.read_status()["nan"] == 0


@pytest.fixture(scope="module")
def trained():
    states = train_guess.default_training_set(stride=8, cap=2_000_000)
    x, y, _ = train_guess.dataset(states, G)
    net, _ = train_guess.train(x, y, steps=1200)
    return net


def test_blast_grid_512_learned_and_plain(trained):
    n, nsteps = 512, 2
    U0 = synth.single_grid((n, n, n), "blast", config=4, gamma=G)
    dts, ref = _oracle(U0, n, nsteps)
    b64, dts64 = _run(U0, n, ez.Params(gamma=G, precision=ez.FP64), nsteps)
    assert dts64 == dts
    assert _bitwise(b64, ref)
    del b64
    b32, _ = _run(U0, n, ez.Params(gamma=G, precision=ez.FP32), nsteps, dts)
    bml, _ = _run(U0, n, ez.Params(gamma=G, precision=ez.FP32, guess=ez.GUESS_MLP, mlp=trained.blob), nsteps, dts)
    l1_p, w_p = _errors(_active(b32), ref)
    l1_l, w_l = _errors(_active(bml), ref)
    l1_lp, _ = _errors(_active(bml), _active(b32))
    sp, sl = b32.read_status(), bml.read_status()
    print(f"\nblast 512^3 x 2: FP32 plain vs oracle L1 {['%.2e' % e for e in l1_p]} max {w_p:.2e}; "
          f"learned L1 {['%.2e' % e for e in l1_l]} max {w_l:.2e}; Newton iterations per interface "
          f"{sp['newton_iters'] / sp['interfaces']:.3f} plain, {sl['newton_iters'] / sl['interfaces']:.3f} learned; "
          f"restarts {sl['guess_restarts']}, HLL cells {sl['hll_cells']}")
    assert max(l1_p) <= 1e-4 and max(l1_l) <= 1e-4
    assert max(l1_lp) <= 1e-5
    assert sl["interfaces"] == sp["interfaces"] and sl["guess_calls"] < sl["interfaces"]
    assert sl["newton_iters"] <= sp["newton_iters"]
    assert sp["nan"] == 0 and sl["nan"] == 0 and sl["newton_nonconv"] == 0


def test_config3_full_level_sampled_patches_match_the_oracle():
    """The batched level at full size (4000 self-periodic patches of 8..64
    cells per axis, 1.89e8 cells), in the bench's launch configuration: one
    persistent launch per sweep over the whole level, the FP32 + learned steps
    replayed from CUDA graphs.  Sampled patches (the first, the last, the
    largest, the smallest and four seeded ones) are stepped by the oracle one
    by one with the same level dt:
      * one FP64 step (dt from the oracle's CFL rule over every patch, which
        the GPU's FP64 reduction reproduces) is bit-identical;
      * K = 5 FP32 + learned steps, each with the dt the GPU's CFL rule gives
        on its own state, are within the FP32 rule of the other configurations
        over the sampled cells: per-field L1 relative error <= max(4 x floor,
        2e-6) and <= 1e-4, the floor being the L1 spread of two oracle runs
        whose inputs differ by 2^-24 relative noise."""
    import torch
    K = 5
    sizes = synth.patch_sizes(4000, config=3)
    sizes, offsets, flat = synth.batched_level(4000, config=3, sizes=sizes)
    dx = [1.0 / 64] * 3
    table = ez.patch_table(sizes, offsets, dx, flags=ez.PATCH_PERIODIC)
    P = oracle.Params(gamma=G)
    rate = max(oracle.cfl_rate([synth.patch_view(f, offsets[i], sizes[i]) for f in flat], dx, P)
               for i in range(len(sizes)))
    dt = 0.4 / rate
    cells = np.prod(sizes, axis=1)
    rng = np.random.default_rng(77)
    sample = sorted({0, len(sizes) - 1, int(np.argmax(cells)), int(np.argmin(cells)),
                     *rng.choice(len(sizes), 4, replace=False).tolist()})
    init = {i: [synth.patch_view(f, offsets[i], sizes[i]).copy() for f in flat] for i in sample}
    ref = {}
    for i in sample:
        U = [f.copy() for f in init[i]]
        oracle.step_periodic(U, dx, dt, 0, P)
        ref[i] = U
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch = ez.PatchBatch(table, flat, stream=stream)
    host = [torch.from_numpy(f) for f in flat]

    def reset():
        torch.cuda.synchronize()
        for u, h in zip(batch.U, host):
            u.copy_(h)
        torch.cuda.synchronize()

    p64 = ez.Params(gamma=G, precision=ez.FP64)
    with torch.cuda.stream(stream):
        assert ez.timestep_cfl(batch, ez.Params(gamma=G, cfl=0.4, precision=ez.FP64)) == dt
        batch.dt_dev.fill_(dt)
        for d in (0, 1, 2):
            ez.ppm_sweep_dev(batch, d, batch.dt_dev, 0, p64)
    stream.synchronize()
    for i in sample:
        for a, b in zip(batch.patch_fields(i), ref[i]):
            assert np.array_equal(a.cpu().numpy()[3:-3, 3:-3, 3:-3], b[3:-3, 3:-3, 3:-3]), i

    net = ez.MLP(seed=4)
    pml = ez.Params(gamma=G, precision=ez.FP32, guess=ez.GUESS_MLP, mlp=net.blob)
    reset()
    with torch.cuda.stream(stream):                      # warm-up outside the capture
        batch.dt_dev.fill_(dt)
        for d in (0, 1, 2):
            ez.ppm_sweep_dev(batch, d, batch.dt_dev, 0, pml)
    stream.synchronize()
    graphs = []
    for order in ((0, 1, 2), (2, 1, 0)):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for d in order:
                ez.ppm_sweep_dev(batch, d, batch.dt_dev, 0, pml)
        graphs.append(g)
    reset()
    batch.reset_status()
    dts = []
    for s in range(K):
        with torch.cuda.stream(stream):
            dts.append(ez.timestep_cfl(batch, ez.Params(gamma=G, cfl=0.4, precision=ez.FP64)))
            batch.dt_dev.fill_(dts[-1])
            graphs[s % 2].replay()
    stream.synchronize()
    assert batch.read_status()["nan"] == 0

    def evolve(start):
        out = {}
        for i in sample:
            U = [f.copy() for f in start[i]]
            for s, dts_ in enumerate(dts):
                oracle.step_periodic(U, dx, dts_, s, P)
            out[i] = U
        return out

    base = evolve(init)
    noise = np.random.default_rng(78)
    pert = evolve({i: [f * (1.0 + 2.0 ** -24 * noise.standard_normal(f.shape)) for f in init[i]] for i in sample})

    def l1(a_of, b_of):
        num, den = np.zeros(5), np.zeros(5)
        for i in sample:
            for f in range(5):
                A = a_of(i, f)[3:-3, 3:-3, 3:-3]
                B = base[i][f][3:-3, 3:-3, 3:-3]
                num[f] += np.sum(np.abs(A - B))
                den[f] += np.sum(np.abs(B))
        return num / den

    got = {i: [a.cpu().numpy() for a in batch.patch_fields(i)] for i in sample}
    err = l1(lambda i, f: got[i][f], None)
    floor = l1(lambda i, f: pert[i][f], None)
    print(f"config 3, {K} FP32 + learned steps, sampled cells: L1 {err.tolist()}, floor {floor.tolist()}")
    for e, fl in zip(err, floor):
        assert e <= max(4.0 * fl, 2e-6) and e <= 1e-4, (err, floor)
