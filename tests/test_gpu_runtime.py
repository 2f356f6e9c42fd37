"""GPU tests of the level runtime: CUDA-graph replay of whole steps, the tile
shapes the autotuner chooses among, and the autotuner itself."""
import numpy as np
import pytest

import paper_1307_2265_gb300 as ez
from gpu_helpers import active, batch_from_patches, gpu_evolve, gpu_patches, white_patch
from paper_1307_2265_gb300 import tune

pytestmark = pytest.mark.gpu
SIZES = [(8, 9, 10), (17, 5, 33), (40, 8, 8), (64, 12, 20), (3, 2, 5), (30, 30, 30)]


def _patches(seed):
    return [white_patch(n, seed=seed + i) for i, n in enumerate(SIZES)]


@pytest.mark.parametrize("precision", [ez.FP64, ez.FP32])
def test_graph_replay_equals_eager_steps(precision):
    import torch
    pats = _patches(1000)
    dx = [0.05] * 3
    eager = batch_from_patches([[f.copy() for f in U] for U in pats], dx, flags=ez.PATCH_PERIODIC)
    graph = batch_from_patches([[f.copy() for f in U] for U in pats], dx, flags=ez.PATCH_PERIODIC)
    params = ez.Params(precision=precision)
    gpu_evolve(eager, params, 4)
    graph.stream = torch.cuda.Stream()
    # warm the launch caches outside capture, on a scratch copy of the batch
    scratch = batch_from_patches([[f.copy() for f in U] for U in pats], dx, flags=ez.PATCH_PERIODIC)
    gpu_evolve(scratch, params, 1)
    graphs = tune.capture_steps(graph, params)
    with torch.cuda.stream(graph.stream):
        for s in range(4):
            graphs[s % 2].replay()
    graph.stream.synchronize()
    for a, b in zip(gpu_patches(eager), gpu_patches(graph)):
        for x, y in zip(a, b):
            assert np.array_equal(active(x), active(y))


@pytest.mark.parametrize("tile", [64, 256])
def test_tile_shapes_give_the_same_sweep(tile):
    pats = _patches(2000)
    dx = [0.05] * 3
    ref = batch_from_patches([[f.copy() for f in U] for U in pats], dx, flags=ez.PATCH_PERIODIC)
    alt = batch_from_patches([[f.copy() for f in U] for U in pats], dx, flags=ez.PATCH_PERIODIC)
    gpu_evolve(ref, ez.Params(precision=ez.FP32), 3)
    gpu_evolve(alt, ez.Params(precision=ez.FP32, tile=(tile, tile, tile)), 3)
    for a, b in zip(gpu_patches(ref), gpu_patches(alt)):
        for x, y in zip(a, b):
            assert np.max(np.abs(active(x) - active(y))) <= 1e-6 * np.max(np.abs(active(y)))
    assert ref.read_status()["interfaces"] == alt.read_status()["interfaces"]


def test_autotuner_picks_valid_tiles_and_restores_fields():
    pats = _patches(3000)
    b = batch_from_patches([[f.copy() for f in U] for U in pats], [0.05] * 3, flags=ez.PATCH_PERIODIC)
    before = [u.clone() for u in b.U]
    tiles, ms = tune.autotune_tiles(b, ez.Params(precision=ez.FP32))
    assert all(t in tune.CANDIDATES for t in tiles)
    assert all(len(ms[d]) == len(tune.CANDIDATES) for d in range(3))
    for u, v in zip(b.U, before):
        assert bool((u == v).all())


def test_bad_tile_rejected():
    b = batch_from_patches([white_patch((4, 4, 4), seed=1)], [0.1] * 3)
    with pytest.raises(ez.EnzoError):
        ez.ppm_sweep(b, 0, 1e-3, 0, ez.Params(precision=ez.FP32, tile=(96, 0, 0)))
