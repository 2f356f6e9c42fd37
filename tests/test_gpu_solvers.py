"""The approximate interface solvers (Sec. 4.1.2: HLL, HLLC) as the sweep's
flux, on the GPU against the oracle: FP64 bit-identical over several steps of
a config-1 grid and of a ragged batch; FP32 within the FP32 bound; a stationary
contact kept exactly sharp by HLLC and smeared by HLL."""
import numpy as np
import pytest

import oracle
import paper_1307_2265_gb300 as ez
from gpu_helpers import (active, batch_from_patches, gpu_evolve, gpu_patches, l1_rel, oracle_evolve_batch,
                         white_patch)
from paper_1307_2265_gb300 import synth

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


@pytest.mark.parametrize("solver", [ez.SOLVER_HLL, ez.SOLVER_HLLC])
def test_approximate_solvers_match_oracle(solver):
    U = synth.single_grid((32, 24, 16), "white", config=1)
    patches = [U] + [white_patch(n, seed=300 + i, mach=2.0) for i, n in enumerate([(1, 1, 1), (9, 3, 17), (40, 5, 6)])]
    dx = [1.0 / 32] * 3
    P = oracle.Params(solver=solver)
    ora = [[f.copy() for f in V] for V in patches]
    dts_o = oracle_evolve_batch(ora, dx, 6, P)
    for flags in (0, ez.PATCH_PERIODIC):
        b = batch_from_patches(patches, dx, flags=flags)
        assert gpu_evolve(b, ez.Params(precision=ez.FP64, solver=solver), 6) == dts_o
        for g, o in zip(gpu_patches(b), ora):
            for a, c in zip(g, o):
                assert np.array_equal(active(a), active(c))
        st = b.read_status()
        assert st["newton_iters"] == 0 and st["nan"] == 0
    b32 = batch_from_patches(patches, dx, flags=ez.PATCH_PERIODIC)
    gpu_evolve(b32, ez.Params(precision=ez.FP32, solver=solver), 6)
    for g, o in zip(gpu_patches(b32), ora):
        for e in l1_rel(g, o):
            assert e <= 1e-4


def test_stationary_contact_on_the_gpu():
    g = 1.4
    nx = 64
    x = np.arange(nx)
    shape = (2, 3, nx)
    rho = np.broadcast_to(np.where((x >= 16) & (x < 48), 1.0, 0.125), shape).copy()
    z = np.zeros(shape)
    U0 = [synth.embed(f) for f in synth.prims_to_conserved(rho, z, z, z, np.ones(shape), g)]
    out = {}
    for name, solver in (("hllc", ez.SOLVER_HLLC), ("hll", ez.SOLVER_HLL)):
        b = batch_from_patches([[f.copy() for f in U0]], [1.0 / nx, 1.0, 1.0], flags=ez.PATCH_PERIODIC)
        gpu_evolve(b, ez.Params(gamma=g, precision=ez.FP64, solver=solver), 40)
        out[name] = float(np.max(np.abs(active(gpu_patches(b)[0][0]) - active(U0[0]))))
    assert out["hllc"] == 0.0 and out["hll"] > 1e-2, out
