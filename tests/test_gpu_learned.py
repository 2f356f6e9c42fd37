"""GPU tests of the learned-guess sweep (tensor-core MLP inside the FP32 sweep)
and of the interface-state logger that feeds its training.

The learned guess only changes where Newton starts: the converged root is the
plain solver's to its tolerance (residual 1e-6 of the velocity scale), so the
learned and plain FP32 sweeps agree to a per-field L1 relative difference of
1e-5 after several steps.
"""
import numpy as np
import pytest

import oracle
import paper_1307_2265_gb300 as ez
from gpu_helpers import NG, active, batch_from_patches, gpu_evolve, gpu_patches, l1_rel, white_patch
from paper_1307_2265_gb300 import synth, train_guess

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


def test_logger_records_the_traced_states_fp64():
    """Stride 1 logs every interface of one x sweep; as a set the rows equal the
    oracle's traced left/right states of the same pencils (rounded to float32)."""
    import torch
    U = white_patch((9, 4, 3), seed=5, mach=1.5)
    oracle.fill_periodic(U)
    dx = [0.1, 0.1, 0.1]
    dt = 0.4 / oracle.cfl_rate(U, dx, oracle.Params())
    b = batch_from_patches([U], dx)
    log = torch.zeros((4096, 6), dtype=torch.float32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    ez.ppm_sweep_logged(b, 0, dt, 0, ez.Params(precision=ez.FP64), log, cnt, 1)
    n = int(cnt.item())
    assert n == 4 * 3 * (9 + 1)
    got = log[:n].cpu().numpy()
    rows = []
    for k in range(NG, NG + 3):
        for j in range(NG, NG + 4):
            pen = np.stack([U[f][k, j, :] for f in (0, 1, 2, 3, 4)])
            o = oracle.pencil_debug(pen, dt / dx[0], oracle.Params())
            for s in range(NG - 1, NG + 9):
                rows.append([o["sL"][0, s], o["sL"][1, s], o["sL"][2, s],
                             o["sR"][0, s + 1], o["sR"][1, s + 1], o["sR"][2, s + 1]])
    ref = np.asarray(rows, dtype=np.float32)
    key = lambda a: a[np.lexsort(a.T[::-1])]
    assert np.array_equal(key(got), key(ref))


@pytest.fixture(scope="module")
def trained():
    states = train_guess.default_training_set(stride=8, cap=2_000_000)
    x, y, _ = train_guess.dataset(states, G)
    net, info = train_guess.train(x, y, steps=1200)
    return net, info


def test_training_on_logged_states_converges(trained):
    net, info = trained
    assert info["samples"] > 100000
    assert info["test_loss"] < 0.05 * info["first_loss"], info
    assert int(net.status[12].item()) == 0


@pytest.mark.parametrize("flags", [0, ez.PATCH_PERIODIC])
def test_learned_sweep_agrees_with_plain_and_saves_iterations(trained, flags):
    net, _ = trained
    patches = [white_patch(n, seed=700 + i) for i, n in enumerate(
        [(1, 1, 1), (3, 2, 5), (17, 5, 33), (40, 8, 8), (32, 32, 32), (130, 3, 4)])]
    dx = [0.05] * 3
    plain = batch_from_patches([[f.copy() for f in U] for U in patches], dx, flags=flags)
    learn = batch_from_patches([[f.copy() for f in U] for U in patches], dx, flags=flags)
    gpu_evolve(plain, ez.Params(precision=ez.FP32), 6)
    gpu_evolve(learn, ez.Params(precision=ez.FP32, guess=ez.GUESS_MLP, mlp=net.blob, mlp_gate=-1.0), 6)
    for g_p, g_l in zip(gpu_patches(plain), gpu_patches(learn)):
        for e in l1_rel(g_l, g_p):
            assert e <= 1e-5
    sp, sl = plain.read_status(), learn.read_status()
    assert sl["interfaces"] == sp["interfaces"]
    assert sl["guess_calls"] == sl["interfaces"]
    assert sl["nan"] == 0 and sl["newton_nonconv"] == 0
    assert sl["newton_iters"] < sp["newton_iters"], (sl["newton_iters"], sp["newton_iters"])


def test_gate_keeps_the_plain_guess_on_weak_interfaces(trained):
    """Smooth flow (k^-4 velocity, rms Mach 3): most interfaces are weak jumps
    where the plain guess is already within a Newton step.  With the default
    gate the learned guess is taken only at strong jumps, answers still match
    the plain path, and the Newton count does not exceed the plain path's."""
    U = synth.single_grid((48, 40, 32), "turbulent", config=2)
    dx = [1.0 / 48] * 3
    runs = {}
    for name, p in (("plain", ez.Params(precision=ez.FP32)),
                    ("gated", ez.Params(precision=ez.FP32, guess=ez.GUESS_MLP, mlp=trained[0].blob)),
                    ("always", ez.Params(precision=ez.FP32, guess=ez.GUESS_MLP, mlp=trained[0].blob, mlp_gate=-1.0))):
        b = batch_from_patches([[f.copy() for f in U]], dx, flags=ez.PATCH_PERIODIC)
        gpu_evolve(b, p, 4)
        runs[name] = (gpu_patches(b)[0], b.read_status())
    for name in ("gated", "always"):
        for e in l1_rel(runs[name][0], runs["plain"][0]):
            assert e <= 1e-5
    sp, sg, sa = runs["plain"][1], runs["gated"][1], runs["always"][1]
    assert sa["guess_calls"] == sa["interfaces"]
    assert 0 < sg["guess_calls"] < sg["interfaces"]
    assert sg["newton_iters"] <= sp["newton_iters"]
    assert sg["newton_iters"] <= sa["newton_iters"]


def test_learned_guess_with_untrained_net_still_gives_plain_answers():
    """A random network is a bad guess; Newton (with the plain-guess restart)
    still converges to the same roots."""
    net = ez.MLP(seed=3)
    U = synth.single_grid((24, 20, 16), "white", config=1)
    dx = [1.0 / 24] * 3
    plain = batch_from_patches([[f.copy() for f in U]], dx, flags=ez.PATCH_PERIODIC)
    learn = batch_from_patches([[f.copy() for f in U]], dx, flags=ez.PATCH_PERIODIC)
    gpu_evolve(plain, ez.Params(precision=ez.FP32), 4)
    gpu_evolve(learn, ez.Params(precision=ez.FP32, guess=ez.GUESS_MLP, mlp=net.blob, mlp_gate=-1.0), 4)
    for e in l1_rel(gpu_patches(learn)[0], gpu_patches(plain)[0]):
        assert e <= 1e-5
    assert learn.read_status()["nan"] == 0


def test_learned_path_rejected_in_fp64():
    net = ez.MLP(seed=0)
    b = batch_from_patches([white_patch((4, 4, 4), seed=1)], [0.1] * 3)
    with pytest.raises(ez.EnzoError):
        ez.ppm_sweep(b, 0, 1e-3, 0, ez.Params(precision=ez.FP64, guess=ez.GUESS_MLP, mlp=net.blob))
