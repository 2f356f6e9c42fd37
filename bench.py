"""Benchmark of the split PPM hydro step on GB300.

Workload (default): a batched AMR level of 4000 self-periodic patches with
per-axis active sizes uniform in 8..64 (about 1.9e8 cells), 3 ghost layers,
white-noise lognormal density (sigma 0.5), rms Mach 1, gamma 5/3, CFL 0.4.
One step = device CFL timestep + three split PPM sweeps over every patch in
one persistent launch per sweep (the whole hot path), FP32 arithmetic with
FP64 conserved accumulation.  The plain FP64 batched sweep is timed on the
same batch for comparison.  Inputs (about 13 GB) exceed L2 (129 MB).

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NPATCH = 4000
GAMMA = 5.0 / 3.0
CFL = 0.4
METRIC = "Mcell-updates/s on GB300: batched FP32+learned vs plain FP64, at stated L1 err"


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def dist_init(backend=None):
    """Process group of the replicas (RANK / WORLD_SIZE / MASTER_* from the
    environment): NCCL with one GPU per rank, gloo on hosts without CUDA."""
    rank, world = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1)
    if world > 1:
        import torch.distributed as dist
        import torch
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
        dist.init_process_group(backend)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    """Largest value over the ranks (the slowest replica's time)."""
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def build_level(rank, npatch=NPATCH):
    from paper_1307_2265_gb300 import synth
    sizes = synth.patch_sizes(npatch, config=3)
    # each rank advances its own level (weak scaling): seeds offset by rank
    sizes, offsets, flat = synth.batched_level(npatch, config=3 + 1000 * rank, sizes=sizes)
    return sizes, offsets, flat


def _clocks_path():
    """Where this rank's nvidia-smi samples go: $ENZO_BENCH_CLOCKS, else a
    temporary file (ranks other than 0 add their local rank to the name)."""
    import tempfile
    r = _env_int("LOCAL_RANK", 0)
    base = os.environ.get("ENZO_BENCH_CLOCKS") or os.path.join(tempfile.gettempdir(), "bench_clocks.csv")
    return base if r == 0 else f"{base}.rank{r}"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, path):
        self.path, self.proc = path, None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self, gpu_index):
        if not self.proc:
            return None
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        if vis.strip().isdigit():
            gpu_index = int(vis.strip())
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9 or parts[0] != str(gpu_index):
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        except OSError:
            return None
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


class _Range:
    """An NVTX range around a leg of the bench, so a profiler can pick its
    kernels (ncu --nvtx --nvtx-include "name/")."""

    def __init__(self, name):
        self.name = name

    def __enter__(self):
        import torch
        torch.cuda.nvtx.range_push(self.name)

    def __exit__(self, *a):
        import torch
        torch.cuda.nvtx.range_pop()


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def measured_traffic(cells_per_sweep, kernel):
    """DRAM bytes per sweep launch from the committed ncu capture of `kernel`,
    scaled by the cells a launch processes; None when there is no capture of
    that kernel or its source changed since."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        if t.get("kernel") != kernel:
            return None
        with open(os.path.join(ROOT, t["source"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
    except (OSError, KeyError, ValueError):
        return None
    if sha != t["source_sha256_16"]:
        return None
    return float(t["bytes_per_cell_sweep"]) * cells_per_sweep


def issue_bound(value_mcu, sm_mhz, sms=152):
    """The learned sweep's issue bound: warp instructions per cell-sweep from the
    committed ncu capture (null once the kernel source changed), against 4
    schedulers x 1 warp instruction per clock per SM at the sampled SM clock."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        with open(os.path.join(ROOT, t["source"]), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest()[:16] != t["source_sha256_16"]:
                return None
        wi = float(t["warp_instr_per_cell_sweep"])
    except (OSError, KeyError, ValueError):
        return None
    peak = sms * 4 * sm_mhz * 1e6                    # warp instructions per second
    bound = peak / (3 * wi) / 1e6                    # Mcell-updates/s at 100% issue
    return {"warp_instr_per_cell_sweep": wi, "issue_active_ncu": t.get("issue_active"),
            "peak_warp_instr_per_s": peak, "bound_mcell_updates_s": bound, "frac": value_mcu / bound}


def fp64_probe(stream):
    """Measured FP64-pipe throughput on this GPU: the library's probe
    (enzo_probe_fp64, 8 independent chains per thread) for DFMA, DADD, DMUL,
    square root and division, each timed with CUDA events on `stream` after a
    warm-up launch.  Rates in operations per second, and per SM per clock at
    the GPU's maximum SM clock."""
    import torch
    import paper_1307_2265_gb300 as ez
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sms = props.multi_processor_count
    sink = torch.zeros(sms * ez.PROBE_BLOCKS_PER_SM + 1, dtype=torch.float64, device="cuda")
    out = {}
    clk = ClockSampler(_clocks_path() + ".probe")
    with clk:
        # DFMA for about a second (clock samples every 200 ms), the others briefly
        for name, op, n, reps in (("dfma", ez.PROBE_DFMA, 4096, 100), ("dadd", ez.PROBE_DADD, 2048, 1),
                                  ("dmul", ez.PROBE_DMUL, 2048, 1), ("dsqrt", ez.PROBE_DSQRT, 128, 1),
                                  ("ddiv", ez.PROBE_DDIV, 128, 1)):
            with torch.cuda.stream(stream):
                ez.probe_fp64(op, 16, sink, stream)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ops = sum(ez.probe_fp64(op, n, sink, stream) for _ in range(reps))
                e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            out[name] = {"ops_per_s": ops / (ms * 1e-3), "ms": ms, "ops": ops}
    c = clk.summary(_env_int("LOCAL_RANK", 0)) or {}
    mhz = c.get("sm_mhz") or _max_sm_mhz()
    for v in out.values():
        v["per_sm_per_clock"] = v["ops_per_s"] / (sms * mhz * 1e6)
    out["sms"], out["sm_mhz"], out["clocks"] = sms, mhz, c
    return out


def _max_sm_mhz():
    try:
        r = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits", "-i",
                            str(_env_int("LOCAL_RANK", 0))], capture_output=True, text=True, timeout=20)
        return float(r.stdout.strip().splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        return 2070.0


def fp64_alu_roofline(value_mcu, probe):
    """The plain FP64 sweep against GB300's FP64 pipe: its DFMA + DMUL + DADD
    thread instructions per cell-sweep from the committed ncu capture (null
    once the kernel source changed) times the measured cell-sweeps per second,
    against the DFMA rate the probe measured in the same run."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "fp64_alu.json")) as f:
            t = json.load(f)
        with open(os.path.join(ROOT, t["source"]), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest()[:16] != t["source_sha256_16"]:
                return None
        per = float(t["fp64_arith_thread_inst_per_cell_sweep"])
    except (OSError, KeyError, ValueError):
        return None
    peak = probe["dfma"]["ops_per_s"]
    achieved = per * 3 * value_mcu * 1e6
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "FP64 thread-instructions/s",
            "frac": achieved / peak, "fp64_arith_per_cell_sweep": per,
            "fp64_pipe_active_ncu": t.get("fp64_pipe_active"),
            "peak_source": "measured: enzo_probe_fp64 DFMA chains in this run"}


def sweep_bytes(table, flags):
    """Algorithmic HBM bytes of one sweep per direction: each pencil reads its
    cells once and writes its active cells once (5 float64 fields).  Periodic
    patches read only active cells (ghost positions are wrapped images)."""
    n = table["n"].astype(np.int64)
    out = []
    for d in range(3):
        if flags:
            cells = np.prod(n, axis=1)
            out.append(int(np.sum(cells * 80)))
        else:
            raise NotImplementedError
    return out


def run_gpu(args, rank, world):
    import torch
    import paper_1307_2265_gb300 as ez
    from paper_1307_2265_gb300 import train_guess, tune
    dev = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(dev)

    # --- learned Newton guess: trained on this GPU with the library's kernels
    net, train_info = _train_net(args)

    sizes, offsets, flat = build_level(rank, args.npatch)
    table = ez.patch_table(sizes, offsets, [1.0 / 64] * 3, flags=ez.PATCH_PERIODIC)
    cells = int(np.prod(sizes, axis=1).sum())
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch = ez.PatchBatch(table, flat, stream=stream)
    host0 = [torch.from_numpy(f).pin_memory() for f in flat]
    p64 = ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP64)
    p32 = ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP32)
    tiles, tile_ms = tune.autotune_tiles(batch, p32)
    p32 = ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP32, tile=tiles)
    pml = ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP32, guess=ez.GUESS_MLP, mlp=net.blob,
                    mlp_gate=args.mlp_gate)
    bytes_per_sweep = sweep_bytes(table, True)

    def reset():
        torch.cuda.synchronize()          # nothing still writing the fields
        for u, h in zip(batch.U, host0):
            u.copy_(h, non_blocking=True)
        torch.cuda.synchronize()
        batch.reset_status()

    def one_step(params, step_idx, ev=None):
        """CFL timestep on the device, then the three split sweeps (dt read on the
        device).  Periodic patches need no ghost fill: the sweeps wrap."""
        ez.timestep_cfl(batch, params, out=batch.dt_dev)
        order = (0, 1, 2) if step_idx % 2 == 0 else (2, 1, 0)
        for q, d in enumerate(order):
            if ev is not None:
                ev[q][0].record(stream)
            ez.ppm_sweep_dev(batch, d, batch.dt_dev, 0, params)
            if ev is not None:
                ev[q][1].record(stream)

    def timed_graph(params, steps, warmup):
        with torch.cuda.stream(stream):
            for w in range(warmup):
                one_step(params, w)
        stream.synchronize()
        graphs = tune.capture_steps(batch, params)
        reset()
        barrier(world)
        launches0 = ez.launch_count()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            t0.record(stream)
            for s in range(steps):
                graphs[s % 2].replay()
            t1.record(stream)
        t1.synchronize()
        return t0.elapsed_time(t1), graphs

    # --- headline: batched FP32 + learned guess, graph replay
    clk = ClockSampler(_clocks_path())
    with clk, _Range("headline"):
        ms, graphs = timed_graph(pml, args.steps, args.warmup)
    ms = max_over_ranks(ms, world)
    status_ml = batch.read_status()
    launches = 9 * args.steps      # per step: prefix+CFL+finalize, 3 x (prefix+sweep)
    del graphs

    # per-sweep event timing of the dominant kernel (eager, same work)
    reset()
    ksw = max(2, min(args.steps, 4))
    evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(3)] for _ in range(ksw)]
    with torch.cuda.stream(stream), _Range("headline_sweeps"):
        for s in range(ksw):
            one_step(pml, s, evs[s])
    stream.synchronize()
    sweep_avg = float(np.mean([[e[q][0].elapsed_time(e[q][1]) for q in range(3)] for e in evs]))

    # --- plain FP32 (autotuned tiles), graph replay
    reset()
    with _Range("fp32_plain"):
        ms32, graphs = timed_graph(p32, args.steps, 1)
    status_32 = batch.read_status()
    del graphs

    # --- plain FP64 batched sweep on the same level (ALU bound: one step)
    reset()
    with torch.cuda.stream(stream), _Range("fp64_plain"):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_step(p64, 1)
        e1.record(stream)
    e1.synchronize()
    ms64 = e0.elapsed_time(e1)

    # --- end to end through the public API with host buffers.  The level's
    # state lives in pinned host memory as its active cells, packed patch by
    # patch (ghost zones are scratch that the steps derive: these patches wrap).
    # Every step copies the whole state in, scatters it into the ghosted device
    # layout (enzo_unpack_active), takes the step, gathers the active cells
    # (enzo_pack_active) and copies them out.  Several device copies of the
    # level take the steps in turn, each on its own stream, so one step's
    # copy-in, another's sweeps and a third's copy-out overlap.
    reset()
    act_off_h = ez.active_offsets(table)
    act_off = torch.from_numpy(act_off_h).to(dev)
    host_act = []
    for f in flat:
        buf = torch.empty(cells, dtype=torch.float64).pin_memory()
        hv = buf.numpy()
        for i in range(len(sizes)):
            nx, ny, nz = (int(v) for v in sizes[i])
            blk = f[offsets[i]:offsets[i] + (nx + 6) * (ny + 6) * (nz + 6)].reshape(nz + 6, ny + 6, nx + 6)
            hv[act_off_h[i]:act_off_h[i] + nx * ny * nz] = blk[3:-3, 3:-3, 3:-3].ravel()
        host_act.append(buf)
    lanes = [(batch, stream)]
    for _ in range(args.e2e_lanes - 1):
        st2 = torch.cuda.Stream()
        with torch.cuda.stream(st2):
            lanes.append((ez.PatchBatch(table, flat, stream=st2), st2))
    nl = len(lanes)
    dev_act = [[torch.empty(cells, dtype=torch.float64, device=dev) for _ in range(5)] for _ in lanes]
    host_out = [[torch.empty_like(h).pin_memory() for h in host_act] for _ in lanes]
    h2d = sum(h.numel() * 8 for h in host_act)
    ke = args.steps                 # the same K steps as the device-resident timing

    def e2e_step(b, st, s):
        pk = dev_act[s % nl]
        for u, h in zip(pk, host_act):
            u.copy_(h, non_blocking=True)
        ez.unpack_active(b, pk, act_off)
        ez.timestep_cfl(b, pml, out=b.dt_dev)
        order = (0, 1, 2) if s % 2 == 0 else (2, 1, 0)
        for d in order:
            ez.ppm_sweep_dev(b, d, b.dt_dev, 0, pml)
        ez.pack_active(b, pk, act_off)
        for u, h in zip(pk, host_out[s % nl]):
            h.copy_(u, non_blocking=True)

    torch.cuda.synchronize()
    ee0 = torch.cuda.Event(enable_timing=True)
    ee0.record(stream)
    for _, st in lanes[1:]:
        st.wait_event(ee0)
    for s in range(ke):
        b, st = lanes[s % nl]
        with torch.cuda.stream(st):
            e2e_step(b, st, s)
    ends = []
    for _, st in lanes:
        e = torch.cuda.Event(enable_timing=True)
        e.record(st)
        ends.append(e)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(max(ee0.elapsed_time(e) for e in ends) / ke, world)
    # the copy-out of lane 0's last step holds that lane's state: check the
    # first and last patches against the device fields directly
    for i in (0, len(sizes) - 1):
        o, c = int(act_off_h[i]), int(np.prod(sizes[i]))
        for f in range(5):
            got = host_out[0][f][o:o + c].numpy()
            want = lanes[0][0].patch_fields(i)[f][3:-3, 3:-3, 3:-3].cpu().numpy().ravel()
            if not np.array_equal(got, want):
                raise RuntimeError(f"end-to-end copy-out differs from the device state (patch {i}, field {f})")
    # the packing kernels alone (one launch each, on lane 0)
    b0, s0 = lanes[0]
    pk_ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    with torch.cuda.stream(s0):
        pk_ev[0].record(s0)
        ez.unpack_active(b0, dev_act[0], act_off)
        pk_ev[1].record(s0)
        ez.pack_active(b0, dev_act[0], act_off)
        pk_ev[2].record(s0)
    s0.synchronize()
    unpack_ms, pack_ms = pk_ev[0].elapsed_time(pk_ev[1]), pk_ev[1].elapsed_time(pk_ev[2])
    del lanes, host_out, dev_act, host_act, b0
    torch.cuda.empty_cache()

    # --- sampled parity + CPU baseline (rank 0, N=1).  (a) The headline path's
    # error over K steps: the learned FP32 path runs K steps of the full level
    # (eager launches, the device dt of each step read back), and the oracle
    # steps sampled patches with the same dts, beside two oracle runs whose
    # inputs differ by 2^-24 (the chaotic floor).  (b) One learned step of the
    # full batch, which the oracle redoes on the first patches with the same
    # dt while it is timed (the CPU baseline).
    cpu = None
    l1 = None
    kerr = None
    if rank == 0 and world == 1 and not args.no_cpu:
        reset()
        dts = []
        with torch.cuda.stream(stream):
            for s in range(args.steps):
                ez.timestep_cfl(batch, pml, out=batch.dt_dev)
                dts.append(float(batch.dt_dev.item()))
                for d in ((0, 1, 2) if s % 2 == 0 else (2, 1, 0)):
                    ez.ppm_sweep_dev(batch, d, batch.dt_dev, 0, pml)
        stream.synchronize()
        ncell = np.prod(sizes, axis=1)
        rng = np.random.default_rng(77)
        pick = sorted({0, len(sizes) - 1, int(np.argmax(ncell)), int(np.argmin(ncell)),
                       *rng.choice(len(sizes), 4, replace=False).tolist()})
        got = {i: [f.cpu().numpy() for f in batch.patch_fields(i)] for i in pick}
        kerr = oracle_k_step_error(flat, sizes, offsets, pick, dts, got)
        reset()
        with torch.cuda.stream(stream):
            one_step(pml, 0)
        stream.synchronize()
        sample = {"dt": float(batch.dt_dev.item()), "patches": [], "l1_num": [0.0] * 5, "l1_den": [0.0] * 5}
        for i in range(args.sample_patches):
            sample["patches"].append([f.cpu().numpy() for f in batch.patch_fields(i)])
        cpu = cpu_baseline_leg(flat, sizes, offsets, sample, budget_s=args.cpu_budget)
        l1 = [n / d for n, d in zip(sample["l1_num"], sample["l1_den"])]

    peak, peak_kind = measured_peak()
    achieved = float(np.mean(bytes_per_sweep)) / (sweep_avg * 1e-3) / 1e9
    value = cells * world * args.steps / (ms * 1e-3) / 1e6
    it_ml = status_ml["newton_iters"] / max(1, status_ml["interfaces"])
    it_32 = status_32["newton_iters"] / max(1, status_32["interfaces"])
    res = {
        "metric": METRIC, "value": value, "unit": "Mcell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64acc",
        "data": "synthetic",
        "config": {"workload": f"batched AMR level: {args.npatch} self-periodic patches, per-axis 8..64 cells, "
                               f"3 ghost layers, white-noise lognormal rho sigma 0.5, rms Mach 1, gamma 5/3, CFL 0.4",
                   "cells_per_step": cells, "precision": "FP32 arithmetic, FP64 accumulation",
                   "guess": "learned (tcgen05 MLP in the sweep), plain-guess restart",
                   "launch": "one CUDA graph per step (CFL + 3 persistent sweeps)",
                   "l2": "inputs larger than L2 (no flush needed)", "parallelism": f"replicas x{world}"},
        "fp32_plain": {"value": cells / (ms32 * 1e-3 / args.steps) / 1e6, "unit": "Mcell-updates/s",
                       "ms_per_step": ms32 / args.steps, "tiles": list(tiles),
                       "tile_ms": {str(d): {str(t): v for t, v in tile_ms[d].items()} for d in tile_ms}},
        "fp64_plain": {"value": cells / (ms64 * 1e-3) / 1e6, "unit": "Mcell-updates/s", "ms_per_step": ms64},
        "newton_iters_per_interface": {"learned": it_ml, "plain": it_32,
                                       "restarts": status_ml["guess_restarts"],
                                       "learned_calls": status_ml["guess_calls"]},
        "training": train_info,
        "e2e": {"value": cells * world / (ms_e2e * 1e-3) / 1e6, "unit": "Mcell-updates/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d, "steps": ke,
                "overlap": f"{nl} device copies of the level on their own streams: copy-in, sweeps and "
                           "copy-out of consecutive steps overlap",
                "host_layout": "active cells packed per patch (enzo_unpack_active / enzo_pack_active on "
                               "the device each step)",
                "unpack_ms": unpack_ms, "pack_ms": pack_ms},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": measured_traffic(cells, "ppm_sweep_kernel<float, DIR, true>"),
                     "kernel": "ppm_sweep_kernel<float, DIR, LEARNED=true>",
                     "peak_source": peak_kind, "sweep_ms_avg": sweep_avg},
        "gpu_launches": int(launches),
        "status": status_ml,
        "cpu_baseline": cpu,
        "fp32_l1_rel_err_vs_oracle_one_step": l1,
        "fp32_err_vs_oracle_k_steps": kerr,
        "clocks": clk.summary(dev),
    }
    sm = (res["clocks"] or {}).get("sm_mhz") or 2070.0
    res["roofline"]["issue"] = issue_bound(value / world, sm)
    res["fp64_probe"] = fp64_probe(stream)
    res["fp64_plain"]["roofline"] = fp64_alu_roofline(res["fp64_plain"]["value"], res["fp64_probe"])
    if world == 1 and not args.no_extra:
        # the other configurations of the metric, on the same GPU with the same
        # network: the 256^3 Mach-3 grid (config 2) and the static hierarchy
        # (config 5), each path timed as its own workload times it
        del batch, host0
        torch.cuda.empty_cache()
        t0 = time.perf_counter()
        paths, cfg, nsteps, setup, _ = single_grid_paths(net, "turbulence", 0, args.mlp_gate, rank)
        res["config2_turbulence"] = {"config": cfg, "paths": paths, "setup_seconds": setup,
                                     "wall_seconds": time.perf_counter() - t0}
        t0 = time.perf_counter()
        hp, layout, setup = hierarchy_paths(net, args.root, args.mlp_gate, rank,
                                            ("fp32_learned", "fp32_plain", "fp64_plain"), probe=res["fp64_probe"])
        res["config5_hierarchy"] = {"config": {"workload": _hierarchy_workload(args.root, layout),
                                               "patches_per_level": [len(L["n"]) for L in layout]},
                                    "paths": hp, "setup_seconds": setup, "wall_seconds": time.perf_counter() - t0}
    return res


def _internal_energy(A):
    """E - KE of conserved active-cell arrays (rho, m_x, m_y, m_z, E)."""
    return A[4] - 0.5 * ((A[1] * A[1] + A[2] * A[2]) + A[3] * A[3]) / A[0]


def run_hierarchy(args, rank, world):
    """Full hierarchy: 256^3 periodic root and three nested levels refined by 2
    (central 192^3, 128^3 and 64^3 root cells; patches from guillotine cuts with
    per-axis sizes 16..32), white-noise initial state on the root inherited by
    the finer levels.  One root step is the subcycled W-cycle (level l takes
    about 2^l steps), with ghost fill from parents and siblings, flux
    correction and projection.  Times one root step of each path: FP32 with
    the learned guess, FP32 plain, FP32 with dual energy (the gas energy, E - KE
    of the initial state, a sixth field of every hierarchy operation) and FP64
    plain."""
    import torch
    dev = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(dev)
    net, train_info = _train_net(args)
    probe = fp64_probe(torch.cuda.Stream())
    out, layout, setup = hierarchy_paths(net, args.root, args.mlp_gate, rank,
                                         ("fp32_learned", "fp32_plain", "fp32_dual", "fp64_plain"), probe=probe)
    res = {"metric": METRIC, "value": out["fp32_learned"]["value"], "unit": "Mcell-updates/s", "n_gpus": world,
           "steps": 1, "warmup": 0, "ms_per_step": out["fp32_learned"]["ms_per_root_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64acc",
           "data": "synthetic",
           "config": {"workload": _hierarchy_workload(args.root, layout),
                      "patches_per_level": [len(L["n"]) for L in layout],
                      "cells_per_level": [int(np.prod(L["n"], axis=1).sum()) for L in layout]},
           "paths": out, "training": train_info, "setup_seconds": setup, "fp64_probe": probe}
    return res


def _hierarchy_workload(root, layout):
    return (f"static hierarchy: {root}^3 periodic root + 3 levels (r=2) over the central 3/4, 1/2, 1/4 of the "
            f"root per axis, patches 16..32 per axis, {sum(len(L['n']) for L in layout)} patches, one subcycled "
            f"root step")


def hierarchy_paths(net, root, mlp_gate, seed, names, probe=None):
    """One subcycled root step of the config-5 hierarchy per path in `names`
    (fp32_learned, fp32_plain, fp32_dual, fp64_plain), timed with CUDA events
    on the hierarchy's stream.  The sweeps' HBM rate counts 240 algorithmic
    bytes per cell update (80 per cell-sweep, ghost reads excluded)."""
    import torch
    import paper_1307_2265_gb300 as ez
    from paper_1307_2265_gb300 import hierarchy as gh
    from paper_1307_2265_gb300 import synth
    t0 = time.perf_counter()
    layout = synth.hierarchy_layout(root, [(root // 8, 7 * root // 8), (root // 4, 3 * root // 4),
                                           (3 * root // 8, 5 * root // 8)], list(range(16, 33, 2)), seed=seed)
    fields = synth.hierarchy_fields(layout, config=5)
    setup = time.perf_counter() - t0
    peak, peak_kind = measured_peak()
    out = {}
    all_paths = (("fp32_learned", ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP32, guess=ez.GUESS_MLP,
                                            mlp=net.blob, mlp_gate=mlp_gate)),
                 ("fp32_plain", ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP32)),
                 ("fp32_dual", ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP32, options=ez.OPT_DUAL)),
                 ("fp64_plain", ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP64)))
    for name, params in all_paths:
        if name not in names:
            continue
        if name == "fp32_dual":
            # the gas energy as a sixth field of every patch: E - KE of the initial state
            ng = synth.NG
            hf = [[U + [synth.embed(_internal_energy([f[ng:-ng, ng:-ng, ng:-ng] for f in U]))] for U in lev]
                  for lev in fields]
        else:
            hf = fields
        hier = gh.Hierarchy(layout, hf, 1.0 / root)
        del hf
        hier.timing = {}
        cflp = ez.Params(gamma=GAMMA, cfl=CFL, precision=params.precision)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(hier.stream)
        log = []
        hier.root_step(params, cflp, log=log)
        e1.record(hier.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        st = {}
        for lev in hier.levels:
            for k, v in lev["batch"].read_status().items():
                st[k] = st.get(k, 0) + v
        out[name] = {"value": hier.cell_updates / (ms * 1e-3) / 1e6, "unit": "Mcell-updates/s",
                     "ms_per_root_step": ms, "cell_updates_per_root_step": hier.cell_updates,
                     "substeps_per_level": [sum(1 for l, _ in log if l == k) for k in range(len(layout))],
                     "newton_iters_per_interface": st["newton_iters"] / max(1, st["interfaces"]),
                     "nan": st["nan"], "hll_cells": st["hll_cells"],
                     "ms_by_operation": hier.timing_ms()}
        sweep_ms = out[name]["ms_by_operation"].get("sweeps")
        if sweep_ms and params.precision == ez.FP64 and probe is not None:
            # the FP64 path is bound by the FP64 pipe: its arithmetic per cell-sweep
            # (the batched level's capture) over the sweeps' time, against the
            # probe's DFMA rate; ghost-cover pencils are not counted as work
            roof = fp64_alu_roofline(hier.cell_updates / (sweep_ms * 1e-3) / 1e6, probe)
            if roof is not None:
                out[name]["sweep_roofline"] = dict(roof, cell_sweeps="3 per cell update, over the sweeps' time")
        elif sweep_ms:
            ach = 240.0 * hier.cell_updates / (sweep_ms * 1e-3) / 1e9
            out[name]["sweep_roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                           "frac": ach / peak, "peak_source": peak_kind,
                                           "bytes": "240 per cell update (80 per cell-sweep, ghost reads "
                                                    "excluded) over the sweeps' time"}
        del hier
        torch.cuda.empty_cache()
    return out, layout, setup


def run_variants(args, rank, world):
    """The sweep's optional rows on the headline's level (periodic patches of 8..64
    cells per axis): FP32 plain; with the reconstruction options (contact
    steepening, flattening, diffusive flux); with HLLC and with HLL as the
    interface solver; HLLC and the two-shock solver with fallback mode 2 (HLL
    re-flux of cells whose internal energy would go negative); with dual energy
    (gas energy from E - KE of the initial state); FP64 with the options and
    with dual energy.  Each runs the device
    CFL timestep and three sweeps per step, W warm-up steps then K timed steps
    (2 for FP64) bracketed by CUDA events on the launching stream, each sweep
    also timed alone for the roofline: algorithmic bytes 80 per cell-sweep (5
    FP64 fields read and written once), 96 with the gas energy."""
    import torch
    import paper_1307_2265_gb300 as ez
    dev = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(dev)
    sizes, offsets, flat = build_level(rank, args.npatch)
    table = ez.patch_table(sizes, offsets, [1.0 / 64] * 3, flags=ez.PATCH_PERIODIC)
    cells = int(np.prod(sizes, axis=1).sum())
    with np.errstate(divide="ignore", invalid="ignore"):
        ke = 0.5 * ((flat[1] * flat[1] + flat[2] * flat[2]) + flat[3] * flat[3]) / flat[0]
        ge = np.where(flat[0] > 0, flat[4] - ke, 0.0)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch = ez.PatchBatch(table, flat, stream=stream, ge=ge)
    host0 = [torch.from_numpy(f).pin_memory() for f in flat] + [torch.from_numpy(ge).pin_memory()]
    del ge, ke

    def reset():
        # the launching stream is not synchronised with the current one: wait
        # for its steps before the copies overwrite the fields they write
        torch.cuda.synchronize()
        for u, h in zip(batch.U + [batch.ge], host0):
            u.copy_(h, non_blocking=True)
        torch.cuda.synchronize()
        batch.reset_status()

    def one_step(params, s, ev):
        ez.timestep_cfl(batch, params, out=batch.dt_dev)
        order = (0, 1, 2) if s % 2 == 0 else (2, 1, 0)
        for q, d in enumerate(order):
            ev[q][0].record(stream)
            ez.ppm_sweep_dev(batch, d, batch.dt_dev, 0, params)
            ev[q][1].record(stream)

    opts = ez.OPT_STEEPEN | ez.OPT_FLATTEN | ez.OPT_DIFFUSE
    variants = [("fp32_plain", ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP32), 80),
                ("fp32_options", ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP32, options=opts), 80),
                ("fp32_hllc", ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP32, solver=ez.SOLVER_HLLC), 80),
                ("fp32_hll", ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP32, solver=ez.SOLVER_HLL), 80),
                ("fp32_hllc_fallback2", ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP32, solver=ez.SOLVER_HLLC,
                                                  fallback=2), 80),
                ("fp32_fallback2", ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP32, fallback=2), 80),
                ("fp32_dual", ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP32, options=ez.OPT_DUAL), 96),
                ("fp64_options", ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP64, options=opts), 80),
                ("fp64_dual", ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP64, options=ez.OPT_DUAL), 96)]
    peak, peak_kind = measured_peak()
    out = {}
    launches0 = ez.launch_count()
    clk = ClockSampler(_clocks_path())
    with clk:
        for name, params, bpc in variants:
            k = args.steps if params.precision == ez.FP32 else min(args.steps, 2)
            reset()
            ev = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(3)]
                  for _ in range(max(args.warmup, k))]
            with torch.cuda.stream(stream):
                for w in range(args.warmup):
                    one_step(params, w, ev[w])
            reset()
            barrier(world)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                for s in range(k):
                    one_step(params, s, ev[s])
                e1.record(stream)
            e1.synchronize()
            ms = max_over_ranks(e0.elapsed_time(e1), world)
            sweep = float(np.mean([[ev[s][q][0].elapsed_time(ev[s][q][1]) for q in range(3)] for s in range(k)]))
            st = batch.read_status()
            achieved = cells * bpc / (sweep * 1e-3) / 1e9
            out[name] = {"value": cells * world * k / (ms * 1e-3) / 1e6, "unit": "Mcell-updates/s",
                         "ms_per_step": ms / k, "steps": k, "sweep_ms_avg": sweep,
                         "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                      "frac": achieved / peak, "bytes_per_cell_sweep": bpc},
                         "newton_iters_per_interface": st["newton_iters"] / max(1, st["interfaces"]),
                         "hll_cells": st["hll_cells"], "ge_pressure": st["ge_pressure"], "nan": st["nan"],
                         "p_floor_hits": st["p_floor_hits"], "neg_after": st["neg_after"]}
    launches = ez.launch_count() - launches0
    head = out["fp32_options"]
    return {"metric": METRIC, "value": head["value"], "unit": "Mcell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64acc",
            "data": "synthetic",
            "config": {"workload": f"sweep variants on the batched AMR level: {args.npatch} self-periodic patches, "
                                   f"per-axis 8..64 cells, white-noise lognormal rho sigma 0.5, rms Mach 1, "
                                   f"gamma 5/3, CFL 0.4, eager launches (CFL + 3 sweeps per step)",
                       "cells_per_step": cells, "value_is": "fp32_options",
                       "l2": "inputs larger than L2 (no flush needed)", "parallelism": f"replicas x{world}"},
            "variants": out, "roofline": dict(head["roofline"], kernel="ppm_sweep_kernel<float, DIR, EXT=1>",
                                              peak_source=peak_kind, traffic=None),
            "gpu_launches": int(launches), "cpu_baseline": None, "clocks": clk.summary(dev)}


def _blast_hierarchy(R, gamma):
    """Root R^3 at rest (rho 1, p 1e-5) with energy 1 deposited as pressure in
    a sphere of radius 3 root cells at the centre, and one refined patch over
    the central (R/4)^3 root cells whose cells take their parents' values."""
    from paper_1307_2265_gb300 import synth
    x = (np.arange(R) + 0.5) / R - 0.5
    z, y, xx = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt(xx * xx + y * y + z * z)
    inside = r < 3.0 / R
    vol = inside.sum() / R ** 3
    p = np.where(inside, (gamma - 1.0) / vol, 1e-5)
    zero = np.zeros_like(p)
    root = [synth.embed(f) for f in synth.prims_to_conserved(np.ones_like(p), zero, zero, zero, p, gamma)]
    lo, hi = 3 * R // 8, 5 * R // 8
    n1 = 2 * (hi - lo)
    act = [f[3:-3, 3:-3, 3:-3][lo:hi, lo:hi, lo:hi].repeat(2, 0).repeat(2, 1).repeat(2, 2) for f in root]
    layout = [{"n": np.array([(R, R, R)]), "origin": np.zeros((1, 3), int), "parent": np.array([-1])},
              {"n": np.array([(n1, n1, n1)]), "origin": np.array([(2 * lo,) * 3]), "parent": np.array([0])}]
    return layout, [[root], [[synth.embed(a) for a in act]]]


def run_rebuild(args, rank, world):
    """Dynamic hierarchy: a Sedov blast in a periodic root of args.root^3 cells
    with one refined level that is rebuilt after every root step from the slope
    (0.3) and shock (0.33, 0.1) flags of the root (Berger-Rigoutsos, efficiency
    0.3, buffer 1).  W warm-up root steps let the blast grow; K timed root steps
    (the subcycled W-cycle, flux correction, projection and the rebuild) give the
    throughput in cell updates of all levels.  The flag kernel is also timed
    alone on the root for its roofline (41 algorithmic bytes per cell: five
    FP64 fields read, one flag byte written), and the host clustering of the
    root's flags on its own."""
    import ctypes
    import torch
    import paper_1307_2265_gb300 as ez
    from paper_1307_2265_gb300 import hierarchy as gh
    dev = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(dev)
    R = args.root
    layout, fields = _blast_hierarchy(R, GAMMA)
    rb = {"gamma": GAMMA, "crit": {"slope": 0.3, "shock_dp": 0.33, "shock_e": 0.1},
          "clus": {"efficiency": 0.3, "small_cells": 64, "buffer": 1}}
    out = {}
    launches0 = ez.launch_count()
    for name, prec in (("fp32_plain", ez.FP32), ("fp64_plain", ez.FP64)):
        hier = gh.Hierarchy(layout, fields, 1.0 / R)
        params = ez.Params(gamma=GAMMA, cfl=CFL, precision=prec)
        for _ in range(args.warmup):
            hier.root_step(params, rebuild=rb)
        hier.stream.synchronize()
        hier.timing = {}
        c0 = hier.cell_updates
        npatch = []
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(hier.stream)
        t0 = time.perf_counter()
        k = args.steps if prec == ez.FP32 else min(args.steps, 3)
        for _ in range(k):
            hier.root_step(params, rebuild=rb)
            npatch.append(len(hier.levels[1]["n"]))
        e1.record(hier.stream)
        e1.synchronize()
        wall = time.perf_counter() - t0
        ms = e0.elapsed_time(e1)
        ops = hier.timing_ms()
        out[name] = {"value": (hier.cell_updates - c0) / (ms * 1e-3) / 1e6, "unit": "Mcell-updates/s",
                     "ms_per_root_step": ms / k, "wall_ms_per_root_step": wall * 1e3 / k, "root_steps": k,
                     "level1_patches": npatch,
                     "level1_cells": int(np.prod(hier.levels[1]["n"], axis=1).sum()),
                     "rebuild_share": ops.get("rebuild", 0.0) / ms, "ms_by_operation": ops}
        if prec == ez.FP32:
            # flag kernel alone on the root, and the host clustering of its flags
            root = hier.levels[0]["batch"]
            flags = torch.zeros(R ** 3, dtype=torch.uint8, device=root.device)
            off = torch.zeros(1, dtype=torch.int64, device=root.device)
            fp = gh._FlagParams(GAMMA, 0.3, 0.33, 0.1, 0.0, ez.FP32)
            L = gh._lib()
            with torch.cuda.stream(hier.stream):
                b = root.c()
                for _ in range(3):
                    L.enzo_flag_cells(ctypes.byref(b), ctypes.byref(fp), flags.data_ptr(), off.data_ptr())
                f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                nrep = 10
                f0.record(hier.stream)
                for _ in range(nrep):
                    L.enzo_flag_cells(ctypes.byref(b), ctypes.byref(fp), flags.data_ptr(), off.data_ptr())
                f1.record(hier.stream)
            f1.synchronize()
            fms = f0.elapsed_time(f1) / nrep
            host = flags.cpu().numpy().reshape(R, R, R)
            t1 = time.perf_counter()
            boxes = gh.cluster_flags(host, margin=3, **rb["clus"])
            cms = (time.perf_counter() - t1) * 1e3
            peak, peak_kind = measured_peak()
            achieved = R ** 3 * 41 / (fms * 1e-3) / 1e9
            out["flag_kernel"] = {"ms": fms, "cells": R ** 3, "flagged_fraction": float((host != 0).mean()),
                                  "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                               "frac": achieved / peak, "bytes_per_cell": 41,
                                               "peak_source": peak_kind}}
            out["clustering_host"] = {"ms": cms, "boxes": len(boxes)}
        del hier
        torch.cuda.empty_cache()
    launches = ez.launch_count() - launches0
    head = out["fp32_plain"]
    return {"metric": METRIC, "value": head["value"], "unit": "Mcell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_root_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64acc",
            "data": "synthetic",
            "config": {"workload": f"dynamic hierarchy: Sedov blast (E = 1, rho 1, p 1e-5) in a {R}^3 periodic "
                                   f"root, one refined level rebuilt after every root step from slope and shock "
                                   f"flags, gamma 5/3, CFL 0.4", "value_is": "fp32_plain"},
            "paths": out, "roofline": dict(out["flag_kernel"]["roofline"], kernel="flag_kernel", traffic=None),
            "gpu_launches": int(launches), "cpu_baseline": None}


def _train_net(args):
    """The learned Newton guess, trained on this GPU with the library's kernels
    on interface states logged from the white-noise and turbulent recipes."""
    from paper_1307_2265_gb300 import train_guess
    t0 = time.perf_counter()
    if args.train_set == "configs":
        states = train_guess.config_training_set(gamma=GAMMA)
    else:
        states = train_guess.default_training_set(gamma=GAMMA, stride=8, cap=3_000_000)
    x, y, _ = train_guess.dataset(states, GAMMA)
    del states
    net, info = train_guess.train(x, y, steps=args.train_steps, batch=args.train_batch)
    info["wall_seconds"] = time.perf_counter() - t0
    info["set"] = args.train_set
    return net, info


def field_errors(got, ref, gamma):
    """L1 relative error per field (sum |a-b| / sum |b|) and the largest per-cell
    relative difference (rho and E against their own value; momentum components
    against |m| + rho c_s of the cell), on the device."""
    import torch
    rho = ref[0]
    mag = torch.sqrt(ref[1] ** 2 + ref[2] ** 2 + ref[3] ** 2)
    p = (gamma - 1.0) * (ref[4] - 0.5 * mag ** 2 / rho)
    cs = torch.sqrt(gamma * torch.clamp(p, min=1e-300) / rho)
    l1, worst = [], 0.0
    for f in range(5):
        diff = (got[f] - ref[f]).abs()
        l1.append(float(diff.sum() / ref[f].abs().sum()))
        den = ref[f].abs() if f in (0, 4) else mag + rho * cs
        worst = max(worst, float((diff / den).max()))
    return {"l1_rel": l1, "max_rel": worst}


def run_single_grid(args, rank, world):
    """Single periodic grids of the precision and learned-guess studies:
    turbulence: 256^3, k^-4 Gaussian random velocity at rms Mach 3, lognormal
      rho (sigma 1), uniform p, 20 steps;
    blast: 512^3, sixteen blast spheres (radius 4..24 cells, p up to 1e3 over
      p = 1e-3, clipped lognormal rho with contrast 1e4), at rest, 4 steps."""
    import torch
    dev = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(dev)
    net, train_info = _train_net(args)
    paths, cfg, nsteps, setup, launches = single_grid_paths(net, args.workload, args.grid_steps, args.mlp_gate, rank)
    lrn, pln = paths["fp32_learned"], paths["fp32_plain"]
    return {"metric": METRIC, "value": lrn["value"], "unit": "Mcell-updates/s", "n_gpus": world,
            "steps": nsteps, "warmup": 1, "ms_per_step": lrn["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64acc", "data": "synthetic",
            "config": cfg, "paths": paths,
            "newton_iters_saved_per_interface": pln["newton_iters_per_interface"] - lrn["newton_iters_per_interface"],
            "gpu_launches": int(launches), "training": train_info, "setup_seconds": setup}


def single_grid_paths(net, workload, grid_steps, mlp_gate, seed):
    """Each path runs the same steps from the same state: plain FP64 (the
    reference answer; bit-identical to the oracle), plain FP32 and FP32 with
    the learned guess.  Throughput uses each path's own device CFL timestep;
    the errors come from a second FP32 run on the FP64 path's timesteps.  The
    FP32 paths' HBM rate counts 240 algorithmic bytes per cell update."""
    import torch
    import paper_1307_2265_gb300 as ez
    from paper_1307_2265_gb300 import synth
    if workload == "turbulence":
        n, recipe, config, nsteps = 256, "turbulent", 2, grid_steps or 20
    else:
        n, recipe, config, nsteps = 512, "blast", 4, grid_steps or 4
    t0 = time.perf_counter()
    U = synth.single_grid((n, n, n), recipe, config=config + 1000 * seed, gamma=GAMMA)
    setup = time.perf_counter() - t0
    table = ez.patch_table([(n, n, n)], [0], [1.0 / n] * 3, flags=ez.PATCH_PERIODIC)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch = ez.PatchBatch(table, [f.ravel() for f in U], stream=stream)
    del U
    init = [u.clone() for u in batch.U]
    cells = n ** 3
    peak, peak_kind = measured_peak()

    def reset():
        torch.cuda.synchronize()          # nothing still writing the fields
        for u, i in zip(batch.U, init):
            u.copy_(i)
        torch.cuda.synchronize()
        batch.reset_status()

    def run(params, dts=None):
        """nsteps steps; own CFL timestep unless dts (device scalars) are given."""
        reset()
        out_dts = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for s in range(nsteps):
                if dts is None:
                    ez.timestep_cfl(batch, params, out=batch.dt_dev)
                    out_dts.append(batch.dt_dev.clone())
                else:
                    batch.dt_dev.copy_(dts[s])
                ez.step(batch, params, s, batch.dt_dev)
            e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), out_dts, batch.read_status()

    def active():
        return [f[3:-3, 3:-3, 3:-3] for f in batch.patch_fields(0)]

    p64 = ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP64)
    p32 = ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP32)
    pml = ez.Params(gamma=GAMMA, cfl=CFL, precision=ez.FP32, guess=ez.GUESS_MLP, mlp=net.blob, mlp_gate=mlp_gate)
    launches0 = ez.launch_count()
    ms64, dts64, st64 = run(p64)
    ref = [a.clone() for a in active()]
    paths = {"fp64_plain": {"value": cells * nsteps / (ms64 * 1e-3) / 1e6, "ms_per_step": ms64 / nsteps,
                            "status": st64}}
    for name, params in (("fp32_plain", p32), ("fp32_learned", pml)):
        run(params)                                   # warm-up
        ms, _, st = run(params)
        _, _, st_e = run(params, dts64)
        err = field_errors(active(), ref, GAMMA)
        sweeps = 3 * cells * nsteps
        ach = 240.0 * cells * nsteps / (ms * 1e-3) / 1e9
        paths[name] = {"value": cells * nsteps / (ms * 1e-3) / 1e6, "ms_per_step": ms / nsteps,
                       "newton_iters_per_interface": st["newton_iters"] / max(1, st["interfaces"]),
                       "learned_guess_fraction": st["guess_calls"] / max(1, st["interfaces"]),
                       "guess_restart_fraction": st["guess_restarts"] / max(1, st["guess_calls"]),
                       "hll_fallback_fraction": st["hll_cells"] / sweeps,
                       "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                    "frac": ach / peak, "peak_source": peak_kind,
                                    "bytes": "240 per cell update over the whole step (CFL included)"},
                       "error_vs_fp64": err, "status": st_e}
    launches = ez.launch_count() - launches0
    cfg = {"workload": (f"{n}^3 periodic grid, " + (
        "k^-4 Gaussian random velocity at rms Mach 3, lognormal rho sigma 1, uniform p"
        if recipe == "turbulent" else
        "16 blast spheres r 4..24 cells, p up to 1e3 over 1e-3, lognormal rho clipped to [1e-2, 1e2]")
        + f", gamma 5/3, CFL 0.4, {nsteps} steps"),
        "cells": cells, "errors": "FP32 paths run on the FP64 path's timesteps; the FP64 GPU path is "
                                  "bit-identical to the oracle (tested at this size for the turbulent grid)"}
    del batch, init, ref
    torch.cuda.empty_cache()
    return paths, cfg, nsteps, setup, launches


def run_reference(args):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the same level:
    each step advances the first patches of the batch (by index) until about
    `budget` seconds of CPU work, one step each with the level's CFL dt."""
    import oracle
    from paper_1307_2265_gb300 import synth
    sizes, offsets, flat = build_level(0, args.npatch)
    P = oracle.Params(gamma=GAMMA)
    dx = [1.0 / 64] * 3
    npick = 24
    pats = []
    for i in range(npick):
        v = [synth.patch_view(f, offsets[i], sizes[i]).copy() for f in flat]
        pats.append(v)
    cells_each = [int(np.prod(sizes[i])) for i in range(npick)]
    rate = max(oracle.cfl_rate(U, dx, P) for U in pats)
    dt = CFL / rate
    t_all, cells_all = 0.0, 0
    for w in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        done = 0
        for U, c in zip(pats, cells_each):
            oracle.step_periodic(U, dx, dt, w, P)
            done += c
        el = time.perf_counter() - t0
        if w >= args.warmup:
            t_all += el
            cells_all += done
    v = cells_all / t_all / 1e6
    return {"metric": METRIC, "value": v, "unit": "Mcell-updates/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"sample of the batched AMR level: first {npick} of {args.npatch} patches, "
                                   "one oracle step each per timed step"},
            "cpu_baseline": {"value": v, "unit": "Mcell-updates/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": f"{npick} patches, {sum(cells_each)} cells per step"},
            "e2e": {"value": v, "unit": "Mcell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _cell_errors(got, ref, gamma):
    """Per field: sum |a - b| and sum |b| over the active cells, and the largest
    per-cell relative difference (rho and E against their own value; momentum
    components against |m| + rho c_s of the cell)."""
    A = [g[3:-3, 3:-3, 3:-3] for g in got]
    B = [r[3:-3, 3:-3, 3:-3] for r in ref]
    mag = np.sqrt(B[1] ** 2 + B[2] ** 2 + B[3] ** 2)
    p = (gamma - 1.0) * (B[4] - 0.5 * mag ** 2 / B[0])
    cs = np.sqrt(gamma * np.maximum(p, 1e-300) / B[0])
    out = []
    for f in range(5):
        den = np.abs(B[f]) if f in (0, 4) else mag + B[0] * cs
        d = np.abs(A[f] - B[f])
        out.append((float(d.sum()), float(np.abs(B[f]).sum()), float(np.max(d / den))))
    return out


def oracle_k_step_error(flat, sizes, offsets, pick, dts, got):
    """The FP32 path's error after len(dts) steps on the sampled patches `pick`
    (GPU fields `got`), against the oracle stepping each patch with the same
    dts, and the chaotic floor: the same comparison between that oracle run and
    one whose inputs carry 2^-24 relative noise."""
    import oracle
    from paper_1307_2265_gb300 import synth
    P = oracle.Params(gamma=GAMMA)
    dx = [1.0 / 64] * 3
    t0 = time.perf_counter()
    noise = np.random.default_rng(78)
    err = np.zeros((5, 3))
    flo = np.zeros((5, 3))
    cells = 0
    for i in pick:
        U = [synth.patch_view(f, offsets[i], sizes[i]).copy() for f in flat]
        V = [u * (1.0 + 2.0 ** -24 * noise.standard_normal(u.shape)) for u in U]
        for s, dt in enumerate(dts):
            oracle.step_periodic(U, dx, dt, s, P)
            oracle.step_periodic(V, dx, dt, s, P)
        for acc, other in ((err, got[i]), (flo, V)):
            e = np.array(_cell_errors(other, U, GAMMA))
            acc[:, :2] += e[:, :2]
            acc[:, 2] = np.maximum(acc[:, 2], e[:, 2])
        cells += int(np.prod(sizes[i]))
    l1, l1f = err[:, 0] / err[:, 1], flo[:, 0] / flo[:, 1]
    return {"steps": len(dts), "fields": ["rho", "m_x", "m_y", "m_z", "E"],
            "l1_rel": l1.tolist(), "max_rel": err[:, 2].tolist(),
            "floor_l1_rel": l1f.tolist(), "floor_max_rel": flo[:, 2].tolist(),
            "l1_over_floor": (l1 / l1f).tolist(),
            "rule": "L1 <= max(4 x floor, 2e-6) and <= 1e-4 per field",
            "within_rule": bool(np.all((l1 <= np.maximum(4 * l1f, 2e-6)) & (l1 <= 1e-4))),
            "sample": f"patches {pick} ({cells} cells): first, last, largest, smallest, four seeded",
            "oracle_seconds": time.perf_counter() - t0}


def cpu_baseline_leg(flat, sizes, offsets, gpu_fields_after_one_step=None, budget_s=12.0):
    """Oracle timed on the host cores on a bounded sample (first patches of the
    level, one step each), plus the FP32 path's error on that sample when the
    GPU result of the same step is given."""
    import oracle
    from paper_1307_2265_gb300 import synth
    P = oracle.Params(gamma=GAMMA)
    dx = [1.0 / 64] * 3
    t0 = time.perf_counter()
    cells = 0
    i = 0
    while time.perf_counter() - t0 < budget_s and i < len(sizes):
        U = [synth.patch_view(f, offsets[i], sizes[i]).copy() for f in flat]
        oracle.step_periodic(U, dx, gpu_fields_after_one_step["dt"], 0, P)
        cells += int(np.prod(sizes[i]))
        if gpu_fields_after_one_step is not None and i < len(gpu_fields_after_one_step["patches"]):
            g = gpu_fields_after_one_step["patches"][i]
            for f in range(5):
                a = U[f][3:-3, 3:-3, 3:-3]
                b = g[f][3:-3, 3:-3, 3:-3]
                gpu_fields_after_one_step["l1_num"][f] += float(np.sum(np.abs(a - b)))
                gpu_fields_after_one_step["l1_den"][f] += float(np.sum(np.abs(a)))
        i += 1
    el = time.perf_counter() - t0
    cores = oracle.num_threads()
    # the same oracle on one thread, on the first patches, for a fifth of the budget
    oracle.set_num_threads(1)
    t1 = time.perf_counter()
    cells1, j = 0, 0
    while time.perf_counter() - t1 < budget_s / 5 and j < len(sizes):
        U = [synth.patch_view(f, offsets[j], sizes[j]).copy() for f in flat]
        oracle.step_periodic(U, dx, gpu_fields_after_one_step["dt"], 0, P)
        cells1 += int(np.prod(sizes[j]))
        j += 1
    el1 = time.perf_counter() - t1
    oracle.set_num_threads(cores)
    return {"value": cells / el / 1e6, "unit": "Mcell-updates/s", "cores": cores,
            "kind": "oracle", "sample": f"first {i} patches of the level, one step each ({cells} cells, {el:.1f} s)",
            "single_thread": {"value": cells1 / el1 / 1e6, "cores": 1,
                              "sample": f"first {j} patches, one step each ({cells1} cells, {el1:.1f} s)"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--npatch", type=int, default=NPATCH)
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU-baseline leg")
    ap.add_argument("--no-extra", action="store_true", help="skip the config-2 and config-5 keys of the default run")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle work in the CPU leg")
    ap.add_argument("--sample-patches", type=int, default=6)
    ap.add_argument("--train-steps", type=int, default=6000)
    ap.add_argument("--train-batch", type=int, default=16384)
    ap.add_argument("--train-set", default="configs", choices=["small", "configs"],
                    help="small: ~3e6 states from reduced grids (fast); configs: ~1e8 states from the "
                         "full-size 32^3 and 256^3 single-grid recipes")
    ap.add_argument("--workload", default="level",
                    choices=["level", "hierarchy", "turbulence", "blast", "variants", "rebuild"])
    ap.add_argument("--e2e-lanes", type=int, default=3, help="device copies of the level in the end-to-end "
                    "measurement (their copies and sweeps overlap)")
    ap.add_argument("--mlp-gate", type=float, default=0.0, help="jump-strength gate of the learned guess "
                    "(0: library default 0.03, < 0: learned guess at every interface)")
    ap.add_argument("--grid-steps", type=int, default=0, help="steps of the single-grid workloads (0: 20 / 4)")
    ap.add_argument("--root", type=int, default=256, help="root grid size of the hierarchy workload")
    args = ap.parse_args()
    rank, world = dist_init()
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    if args.workload == "hierarchy":
        res = run_hierarchy(args, rank, world)
    elif args.workload == "variants":
        res = run_variants(args, rank, world)
    elif args.workload == "rebuild":
        res = run_rebuild(args, rank, world)
    elif args.workload in ("turbulence", "blast"):
        res = run_single_grid(args, rank, world)
    else:
        res = run_gpu(args, rank, world)
    if rank == 0:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
