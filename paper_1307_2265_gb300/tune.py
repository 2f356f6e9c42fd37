"""Autotuner of the sweep's tile shape, and CUDA-graph capture of a step.

The FP32 plain-guess sweep can run 64, 128 or 256 pencils per CTA tile
(enzo_params.tile per axis).  The best choice depends on the batch: patch
sizes set how many pencils each patch has and how full its last tile is.
`autotune_tiles` times each candidate on the batch itself, one sweep per
candidate and direction with CUDA events, and restores the fields afterwards.

`capture_steps` records one level step (device CFL + three sweeps, reading dt
on the device) for each sweep order into CUDA graphs, so a run replays one
graph per step instead of launching nine kernels.
"""
from __future__ import annotations

from . import Params, PatchBatch, ppm_sweep_dev, timestep_cfl

CANDIDATES = (64, 128, 256)


def autotune_tiles(batch: PatchBatch, params: Params, candidates=CANDIDATES, reps=2):
    """Returns (tile per axis, {axis: {tile: ms}})."""
    import torch
    saved = [u.clone() for u in batch.U]
    stream = batch.stream if batch.stream is not None else torch.cuda.current_stream(batch.device)
    timings = {}
    best = []
    with torch.cuda.stream(stream):
        timestep_cfl(batch, params, out=batch.dt_dev)
        for d in range(3):
            timings[d] = {}
            for t in candidates:
                tiles = [0, 0, 0]
                tiles[d] = t
                p = Params(**{**params.__dict__, "tile": tuple(tiles)})
                ppm_sweep_dev(batch, d, batch.dt_dev, 0, p)          # warm the variant
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    ppm_sweep_dev(batch, d, batch.dt_dev, 0, p)
                e1.record(stream)
                e1.synchronize()
                timings[d][t] = e0.elapsed_time(e1) / reps
            best.append(min(timings[d], key=timings[d].get))
    for u, s in zip(batch.U, saved):
        u.copy_(s)
    torch.cuda.synchronize(batch.device)
    batch.reset_status()
    return tuple(best), timings


def capture_steps(batch: PatchBatch, params: Params):
    """Two CUDA graphs: a full step with sweep order x,y,z and one with z,y,x.
    The batch's patches must be periodic (no ghost fill in the step)."""
    import torch
    stream = batch.stream if batch.stream is not None else torch.cuda.Stream(batch.device)
    batch.stream = stream
    graphs = []
    for order in ((0, 1, 2), (2, 1, 0)):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            timestep_cfl(batch, params, out=batch.dt_dev)
            for d in order:
                ppm_sweep_dev(batch, d, batch.dt_dev, 0, params)
        graphs.append(g)
    return graphs
