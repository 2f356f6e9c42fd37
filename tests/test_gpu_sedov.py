"""Sedov blast (the blast test of Sec. 11) through the headline path on the
GPU: FP32 arithmetic with the learned Newton guess, and the HLLC solver, on a
96^3 box.  The shock radius follows xi0 (E t^2 / rho)^(1/5) (xi0 integrated from
the self-similar equations) to within one cell at every checkpoint, and mass
and energy stay conserved; an untrained network only moves Newton's start."""
import numpy as np
import pytest

import paper_1307_2265_gb300 as ez
import sedov_similarity
from gpu_helpers import active, batch_from_patches, gpu_patches
from paper_1307_2265_gb300 import synth

pytestmark = pytest.mark.gpu


def _blast(n, g):
    dx = 1.0 / n
    c = (np.arange(n) + 0.5) * dx - 0.5
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    R = np.sqrt(X * X + Y * Y + Z * Z)
    inside = R < 3.01 * dx
    p = np.full((n, n, n), 1e-5)
    p[inside] = (g - 1.0) / (inside.sum() * dx ** 3)
    one, zero = np.ones((n, n, n)), np.zeros((n, n, n))
    return [synth.embed(f) for f in synth.prims_to_conserved(one, zero, zero, zero, p, g)], R


@pytest.mark.parametrize("name", ["fp32_learned", "fp32_hllc"])
def test_sedov_radius_on_the_gpu(name):
    n, g = 96, 5.0 / 3.0
    dx = 1.0 / n
    U, R = _blast(n, g)
    b = batch_from_patches([U], [dx] * 3, flags=ez.PATCH_PERIODIC)
    net = ez.MLP(seed=1)
    params = (ez.Params(gamma=g, precision=ez.FP32, guess=ez.GUESS_MLP, mlp=net.blob) if name == "fp32_learned"
              else ez.Params(gamma=g, precision=ez.FP32, solver=ez.SOLVER_HLLC))
    xi = sedov_similarity.xi0(g)
    bins = np.floor(R / dx).astype(int).ravel()
    counts = np.bincount(bins)
    m0 = float(np.sum(active(U[0])))
    e0 = float(np.sum(active(U[4])))
    t, step = 0.0, 0
    for r_exact in (0.2, 0.25, 0.3, 0.35):
        t_end = (r_exact / xi) ** 2.5
        while t < t_end - 1e-14:
            ez.timestep_cfl(b, params, out=b.dt_dev)
            dt = min(float(b.dt_dev.item()), t_end - t)
            b.dt_dev.fill_(dt)
            ez.step(b, params, step, b.dt_dev)
            t += dt
            step += 1
        rho = active(gpu_patches(b)[0][0])
        prof = np.bincount(bins, rho.ravel()) / counts
        k = int(np.argmax(prof))
        half = 0.5 * (prof[k] + 1.0)
        j = k
        while prof[j + 1] > half:
            j += 1
        r_num = (j + 0.5) * dx + (prof[j] - half) / (prof[j] - prof[j + 1]) * dx
        assert abs(r_num - r_exact) < 1.0 * dx, (name, r_exact, r_num)
    fields = gpu_patches(b)[0]
    assert abs(float(np.sum(active(fields[0]))) - m0) <= 1e-11 * m0
    assert abs(float(np.sum(active(fields[4]))) - e0) <= 1e-8 * e0
    st = b.read_status()
    assert st["nan"] == 0 and st["newton_nonconv"] == 0
