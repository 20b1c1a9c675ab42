"""Benchmark: scene frames per second matched (every model x every scene x every offset).

Default workload: the full combined workload -- 100 models (M 16..256) against 16 scenes of 10k-100k
frames at 640x480 with Poisson(80) points per frame, K = 64, w = 3, about 991k scene frames. A step is one
pass of the whole hot path (unary table, candidate selection, recursion, backtrack) over one batch of that
job: every model against one block of each of the 16 scenes, the block owning `hop` consecutive offsets
(their windows lie inside it, so every result is the full scene's). Tiling the scenes with such blocks is
the whole job; a step therefore stands for 16 x hop scene frames, and the job's time is its frames over
the measured rate. The headline `value` is the plain exact FP32 path; the BF16-distance + learned-pruning
forms run on the same batch beside it. Models and blocks are resident in HBM, outputs on the device.

Prints ONE JSON line (rank 0); the roofline object names the dominant kernel, its algorithmic work per
launch, the measured peak it is divided by and its DRAM traffic.
  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]
Workloads: combined (default; --hop offsets per block), batched_exact (10 models x 8 scenes of
300-1500 frames), precision_long (50 models x one 30,000-frame scene, F = 176), batched_small, single_match.
Under torchrun each rank matches its own batch (combined: other blocks of the same scenes; otherwise a
reseeded copy), weak scaling with no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "scene frames/sec matched (all models × offsets), plain exact vs pruned+BF16"
OPS_PER_TRIPLE = 12          # FP32 lane ops per evaluated triple after hoisting the per-(a, b) and per-(b, c) terms
SM_COUNT_FALLBACK = 152
FP32_LANES_PER_SM = 128
L2_NOTE = "flushed (512 MiB write) before every step"
# DRAM bytes of one recursion launch, from an ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of
# a small case, with the sources of the kernel it captured and the capture's argmin-table bytes
# sum n_offsets (M - 2) K^2. Both the tables written and the lists read grow in proportion to that sum,
# so a full launch's traffic is scaled by it; a changed kernel source voids the figure.
RECURSE_NCU = {"sources_sha256": "015ced47a289cc2cc1d45f3754dcef8c424ddc24374815637abff006ea0717e5",
               "bytes": 845_508_608 + 1_285_723_000, "beta_bytes": 1_667_760_128, "case": "combined_small"}
RECURSE_SOURCES = ("k_recurse.cu", "recurse_common.cuh", "f32x2.cuh")


def recurse_traffic(wl, chunks_per_step: int):
    """DRAM bytes per recursion launch scaled from the committed capture, or None if the kernel changed."""
    import hashlib
    h = hashlib.sha256()
    for f in RECURSE_SOURCES:
        with open(os.path.join(ROOT, "paper_1505_00581_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    beta = sum(wl.n_offsets(m, s) * (wl.models[m].n - 2) * wl.K * wl.K
               for m in range(len(wl.models)) for s in range(len(wl.scenes)))
    if h.hexdigest() != RECURSE_NCU["sources_sha256"]:
        return None, beta / chunks_per_step
    return RECURSE_NCU["bytes"] * beta / RECURSE_NCU["beta_bytes"] / chunks_per_step, beta / chunks_per_step


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest value of x over the ranks (the job's wall time is the slowest rank's)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / seconds


def workload(name: str, rank: int, hop: int = 256):
    """(workload, job description) for a named workload; rank r gets its own batch."""
    from paper_1505_00581_gb300 import synth
    if name == "combined":
        cs = synth.CombinedScenes(seed=3)
        wl = cs.step(hop=hop, seed=rank)
        job = {"job_frames": cs.total_frames, "job_scenes": len(cs.n_frames),
               "job_scene_frames": [min(cs.n_frames), max(cs.n_frames)],
               "step": f"all {len(wl.models)} models x one {hop}-offset block of each of the {len(wl.scenes)} "
                       f"scenes (block {hop} + 35 frames: the windows of its offsets lie inside it); the whole "
                       f"job is {cs.total_frames / wl.total_frames:.1f} such steps"}
        return wl, job
    if name == "combined_small":     # 2 blocks of 16 offsets: the profiling case of the combined workload
        cs = synth.CombinedScenes(seed=3)
        wl = cs.step(hop=16, seed=rank)
        wl.scenes, wl.frames_credit, wl.name = wl.scenes[:2], 2 * 16, wl.name + "_2blocks"
        return wl, None
    if name == "batched_exact":
        return synth.batched_exact(seed=1 + 1000 * rank), None
    if name == "batched_small":      # one 300-frame scene: the profiling case (a few hundred MB on the device)
        return synth.batched_exact(seed=1 + 1000 * rank, n_scenes=1, frames_range=(300, 300)), None
    if name == "precision_long":
        return synth.precision_long(seed=2 + 1000 * rank), None
    if name == "single_match":
        return synth.single_match(seed=0 + 1000 * rank), None
    raise SystemExit(f"unknown workload {name}")


def total_units(wl):
    return sum(wl.n_offsets(m, s) for m in range(len(wl.models)) for s in range(len(wl.scenes)))


def config_of(wl, job, args, world):
    """The config dict of the JSON line, the same for both arms."""
    cfg = {"workload": wl.name, "models": len(wl.models), "scenes": len(wl.scenes), "K": wl.K, "window": wl.window,
           "T": wl.T, "frames_per_step_per_rank": wl.total_frames, "units_per_step_per_rank": total_units(wl),
           "form": "plain exact (Eqs. 9-13)", "l2": L2_NOTE, "parallelism": f"replicas x{world}"}
    if job is not None:
        cfg.update(job)
        cfg["hop"] = args.hop
    return cfg


def params_of(hgm, wl, **over):
    kw = dict(K=wl.K, window=wl.window, T=wl.T, lambda1=wl.lambda1, lambda2=wl.lambda2, lambda3=wl.lambda3)
    if wl.offset_lo is not None:
        kw["offset_lo"] = wl.offset_lo
    if wl.offset_hi is not None:
        kw["offset_hi"] = wl.offset_hi
    kw.update(over)
    return hgm.default_params(**kw)


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv", prefix="clocks_")
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- the FP64 oracle on the host cores ----------------------------------------------------------------------
def sample_units(wl, n_units: int, seed: int):
    """n_units seeded (model, scene, offset) units, uniform over the workload's units."""
    rng = np.random.default_rng(seed)
    pairs = [(m, s) for m in range(len(wl.models)) for s in range(len(wl.scenes))]
    weights = np.array([wl.n_offsets(m, s) for m, s in pairs], dtype=np.float64)
    picks = rng.choice(len(pairs), size=n_units, p=weights / weights.sum())
    out = []
    for q in picks:
        m, s = pairs[q]
        lo, _ = wl.offset_range(m, s)
        out.append((m, s, lo + int(rng.integers(wl.n_offsets(m, s)))))
    return out


def _solve_unit(wl, m, s, o):
    """FP64 oracle of unit (m, s, o) on the scene frames its windows reach, shifted to frame 0 (candidate lists
    and energies are the full scene's); returns (energy, caller-order assignment in the scene's indices)."""
    from oracle import Oracle
    mod, sc = wl.models[m], wl.scenes[s]
    f0 = max(0, o + int(mod.t.min()) - wl.window)
    f1 = min(sc.n_frames - 1, o + int(mod.t.max()) + wl.window)
    keep = np.nonzero((sc.t >= f0) & (sc.t <= f1))[0]
    orc = Oracle(mod.xy, mod.t, mod.f, sc.xy[keep], sc.t[keep] - f0, sc.f[keep], f1 - f0 + 1, K=wl.K,
                 window=wl.window, lambda1=wl.lambda1, lambda2=wl.lambda2, lambda3=wl.lambda3, T=wl.T)
    e, z, _ = orc.match(o - f0)
    z = np.asarray(z, dtype=np.int64)
    return e, np.where(z >= 0, keep[np.maximum(z, 0)], z)


def oracle_time(wl, units, threads: int):
    """Seconds the FP64 oracle takes for these units on `threads` host threads; the results per unit."""
    from concurrent.futures import ThreadPoolExecutor
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        out = list(ex.map(lambda u: _solve_unit(wl, *u), units))
    return time.perf_counter() - t0, out


def run_reference(args):
    """--impl reference: the FP64 oracle (as it stands) on the host cores, a bounded sample of the batch's
    units per step; the rate is projected from the sample to the whole batch."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    wl, job = workload(args.workload, 0, args.hop)
    threads = os.cpu_count() or 1
    units = total_units(wl)
    per_step = max(threads, args.ref_units)
    for w in range(args.warmup):
        oracle_time(wl, sample_units(wl, threads, 7 + w), threads)
    measured, projected = [], []
    for k in range(args.steps):
        t, _ = oracle_time(wl, sample_units(wl, per_step, 100 + k), threads)
        measured.append(t)
        projected.append(t / per_step * units)       # seconds for the whole batch at the sample's rate
    value = wl.total_frames / float(np.mean(projected))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(measured)) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(wl, job, args, world),
            "measured_s_per_step": float(np.mean(measured)), "units_per_step_sampled": per_step,
            "projected_s_per_batch": float(np.mean(projected)),
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} seeded units of the batch's {units} per step "
                                       f"({np.mean(measured):.1f} s measured on {threads} threads), projected to "
                                       f"the batch"},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- GPU timing helpers -------------------------------------------------------------------------------------
def _time_plan(torch, hgm, models, scenes, p, energy, assign, steps, warmup, stream, flush):
    """The same batch as one CUDA-graph replay per step (hgm_plan): ms per step, CUDA events on the stream."""
    plan = hgm.Plan(models, scenes, p, energy, assign, stream=stream)
    for _ in range(warmup):
        plan.run(stream)
    plan.check(stream)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        starts[k].record(stream)
        plan.run(stream)
        ends[k].record(stream)
    plan.check(stream)
    plan.close()
    return sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / steps


def _time_form(torch, hgm, models, scenes, p, energy, assign, steps, warmup, stream, flush, profile=False):
    for _ in range(warmup):
        hgm.match_batch(models, scenes, p, energy, assign)
    torch.cuda.synchronize()
    hgm.profile_reset()
    hgm.profile_enable(True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if profile:
        torch.cuda.profiler.start()
    for k in range(steps):
        flush.zero_()
        starts[k].record(stream)
        hgm.match_batch(models, scenes, p, energy, assign)
        ends[k].record(stream)
    torch.cuda.synchronize()
    if profile:
        torch.cuda.profiler.stop()
    hgm.profile_enable(False)
    return sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / steps, hgm.profile_read()


def alu_peak(torch):
    pk, pk_kind = peaks()
    sm_count = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count \
        or SM_COUNT_FALLBACK
    peak_ops = sm_count * FP32_LANES_PER_SM * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    src = f"{sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x sm_max_mhz of MEASURED_PEAKS.json ({pk_kind})"
    return peak_ops, src


def alu_roofline(torch, hgm, run_once, prof, steps, kernel, note):
    """Roofline of a form's recursion kernel, defined as for the main line: the triples its loops evaluate
    (one untimed pass of the kernel's accounting variant) x OPS_PER_TRIPLE, over the kernel's average
    launch time in the timed steps, against the FP32 lane peak."""
    hgm.profile_evaluated(reset=True)
    hgm.profile_enable(2)
    run_once()
    hgm.profile_enable(False)
    evaluated = hgm.profile_evaluated(reset=True)
    rec_ms, rec_n = prof["recurse"]
    per_step = max(1, rec_n // steps)
    avg_ms = rec_ms / max(rec_n, 1)
    eval_launch = evaluated / per_step
    peak_ops, src = alu_peak(torch)
    achieved = eval_launch * OPS_PER_TRIPLE / (avg_ms / 1e3) / 1e12
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak_ops,
            "unit": "Tops/s (FP32 lane ops)", "frac": achieved / peak_ops, "traffic": None, "traffic_source": note,
            "peak_source": src, "evaluated_triples_per_launch": eval_launch, "ops_per_triple": OPS_PER_TRIPLE,
            "avg_launch_ms": avg_ms}


def run_chains(args, torch, hgm, wl, models, scenes, dev, stream, world, flush, dist=None, n_chains=3):
    """The independent-chains variant (Sec. 4, method 2) on the same workload, whose models hold several
    points per frame: every model split into its within-frame-rank chains, all chains of all models run
    as one exact batch, the per-offset energy the mean over a model's chains."""
    p = params_of(hgm, wl)
    _, es, as_ = hgm.batch_layout(models, scenes, p)
    e = torch.empty(int(es[-1]), dtype=torch.float32, device=dev)
    a = torch.empty(int(as_[-1]), dtype=torch.int32, device=dev)
    steps = max(1, min(args.steps, 5))
    for _ in range(min(args.warmup, 3)):
        hgm.match_chains_batch(models, scenes, p, n_chains, e, a)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    hgm.profile_reset()
    hgm.profile_enable(True)
    for k in range(steps):
        flush.zero_()
        starts[k].record(stream)
        hgm.match_chains_batch(models, scenes, p, n_chains, e, a)
        ends[k].record(stream)
    torch.cuda.synchronize()
    hgm.profile_enable(False)
    prof = hgm.profile_read()
    ms = max_over_ranks(sum(x.elapsed_time(y) for x, y in zip(starts, ends)) / steps, dist, dev)
    roofline = alu_roofline(torch, hgm, lambda: hgm.match_chains_batch(models, scenes, p, n_chains, e, a), prof,
                            steps, "recurse_kernel",
                            "the same kernel as the main line; its traffic there is per argmin-table byte")
    covered = total = n_chain_models = 0
    for m in wl.models:
        _, counts = np.unique(m.t, return_counts=True)
        total += m.n
        sizes = [int((counts > c).sum()) for c in range(n_chains)]
        covered += sum(z for z in sizes if z >= 3)
        n_chain_models += sum(1 for z in sizes if z >= 3)
    fin = torch.isfinite(e).sum().item()
    return {"value": job_rate(wl.total_frames, world, ms / 1e3), "unit": "frames/s", "ms_per_step": ms,
            "steps": steps, "n_chains": n_chains, "chain_models": n_chain_models,
            "model_points_covered": covered / max(total, 1), "finite_offsets": int(fin),
            "kernel_ms_per_step": {k: v[0] / steps for k, v in prof.items()},
            "roofline": roofline, "form": "plain exact FP32 per chain, mean over chains"}


def run_blocks(args, torch, hgm, dev, stream, flush):
    """The paper's own formulation (every scene point a candidate, no offsets) in its two scenarios (Sec. 4,
    Table 2): 50 models of 30 points streamed over a one-minute scene as 60-frame blocks every 30 frames
    (latency per block, end to end from host points to host results), and 50 models against a 723-frame
    scene of ~754 points matched whole."""
    from paper_1505_00581_gb300 import synth
    ws = synth.paper_stream()
    p = hgm.default_params(T=ws.T, lambda1=ws.lambda1, lambda2=ws.lambda2, lambda3=ws.lambda3)
    models = [hgm.Model(*(torch.from_numpy(a).to(dev) for a in (m.xy, m.t, m.f))) for m in ws.models]
    sc = ws.scenes[0]
    blocks = [b[1:4] for b in hgm.stream_blocks(sc.xy, sc.t, sc.f, sc.n_frames, 60, 30)]
    cap = max(len(b[1]) for b in blocks)
    st = hgm.Stream(models, p, 60, stream=stream, max_points=cap)
    e = np.zeros(len(models), np.float32)
    a = np.zeros(int(st.starts[-1]), np.int32)
    for b in blocks:             # warm-up over every block
        st.match(*b, energy=e, assign=a, stream=stream)
    lat = []
    reps = max(1, min(args.steps, 3))
    for rep in range(reps):
        for b in blocks:
            t0 = time.perf_counter()
            st.match(*b, energy=e, assign=a, stream=stream)
            lat.append(time.perf_counter() - t0)
    lat_ms = np.array(lat) * 1e3
    per_pass = float(lat_ms.sum()) / reps
    h2d = sum(x.nbytes for b in blocks for x in b) / len(blocks)
    streaming = {"workload": ws.name, "blocks": len(blocks), "block_frames": 60, "hop_frames": 30,
                 "points_per_block": float(np.mean([len(b[1]) for b in blocks])), "max_points": cap,
                 "models": len(models),
                 "latency_ms": {"median": float(np.median(lat_ms)), "p90": float(np.percentile(lat_ms, 90)),
                                "max": float(lat_ms.max())},
                 "value": sc.n_frames / (per_pass / 1e3), "unit": "scene frames/s (overlapping blocks, e2e)",
                 "ms_per_frame": per_pass / sc.n_frames, "h2d_bytes_per_block": int(h2d),
                 "d2h_bytes_per_block": int(e.nbytes + a.nbytes)}
    st.close()
    # Table 2's whole-scene case, device outputs, CUDA events
    ww = synth.paper_whole()
    wm = [hgm.Model(*(torch.from_numpy(a_).to(dev) for a_ in (m.xy, m.t, m.f))) for m in ww.models]
    s0 = ww.scenes[0]
    wsc = [hgm.Scene(*(torch.from_numpy(a_).to(dev) for a_ in (s0.xy, s0.t, s0.f)), s0.n_frames)]
    ed = torch.empty(len(wm), dtype=torch.float32, device=dev)
    ad = torch.empty(int(hgm.block_layout(wm, 1)[-1]), dtype=torch.int32, device=dev)
    for _ in range(max(3, min(args.warmup, 5))):
        hgm.match_block(wm, wsc, p, ed, ad, stream=stream)
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 10))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if args.profile_form == "whole_block":
        torch.cuda.profiler.start()
    for x, y in evs:
        flush.zero_()
        x.record(stream)
        hgm.match_block(wm, wsc, p, ed, ad, stream=stream)
        y.record(stream)
    torch.cuda.synchronize()
    if args.profile_form == "whole_block":
        torch.cuda.profiler.stop()
    ms = sum(x.elapsed_time(y) for x, y in evs) / len(evs)
    whole = {"workload": ww.name, "scene_points": s0.n, "scene_frames": s0.n_frames, "models": len(wm),
             "ms": ms, "value": s0.n_frames / (ms / 1e3), "unit": "scene frames/s (all models, whole scene)",
             "finite": int(torch.isfinite(ed).sum().item())}
    return {"streaming": streaming, "whole_scene": whole}


def run_dummy(args, torch, hgm, wl, models, scenes, dev, stream, world, flush, dist=None, wd=8.0):
    """The exact path with the dummy assignment of Eq. 2 (W^d = 8 descriptor-distance units: a model point
    whose best candidate differs from it by more than about the distance between two descriptor clusters'
    members is left unmatched) on the same workload."""
    p = params_of(hgm, wl, dummy_cost=wd)
    _, es, as_ = hgm.batch_layout(models, scenes, p)
    e = torch.empty(int(es[-1]), dtype=torch.float32, device=dev)
    a = torch.empty(int(as_[-1]), dtype=torch.int32, device=dev)
    steps = max(1, min(args.steps, 3))
    ms, prof = _time_form(torch, hgm, models, scenes, p, e, a, steps, 1, stream, flush, args.profile_form == "dummy")
    ms = max_over_ranks(ms, dist, dev)
    eps_fraction = float((a == -2).float().mean().item())
    finite = int(torch.isfinite(e).sum().item())
    roofline = alu_roofline(torch, hgm, lambda: hgm.match_batch(models, scenes, p, e, a), prof, steps,
                            "dummy_recurse_kernel", "not captured at this size")
    return {"value": job_rate(wl.total_frames, world, ms / 1e3), "unit": "frames/s", "ms_per_step": ms,
            "steps": steps, "dummy_cost": wd, "eps_fraction": eps_fraction, "finite_offsets": finite,
            "kernel_ms_per_step": {k: v[0] / steps for k, v in prof.items()}, "roofline": roofline,
            "form": "exact FP32 with an eps slot per list (own recursion kernel, kept-list branch and bound)"}


def fp64_errors(sampled, wl, first, es, as_, e_h, a_h):
    """Relative energy error of a GPU result (e_h, a_h host arrays in the batch layout) against the FP64
    optimum at the sampled units, and how often the assignment equals the oracle's."""
    errs, same, fin_mismatch = [], 0, 0
    for (m, s, o), (e64, z64) in sampled:
        q = m * len(wl.scenes) + s
        k = o - int(first[q])
        eg = float(e_h[int(es[q]) + k])
        M = wl.models[m].n
        zg = a_h[int(as_[q]) + k * M:int(as_[q]) + (k + 1) * M]
        if np.isfinite(e64) != np.isfinite(eg):
            fin_mismatch += 1
        elif np.isfinite(e64):
            errs.append((eg - e64) / max(abs(e64), 1e-30))
        same += int(np.array_equal(zg, z64) or (not np.isfinite(e64) and not np.isfinite(eg)))
    errs = np.array(errs)
    return {"units": len(sampled), "finite": int(errs.size), "feasibility_mismatch": fin_mismatch,
            "max_abs_rel_err": float(np.abs(errs).max()) if errs.size else None,
            "mean_abs_rel_err": float(np.abs(errs).mean()) if errs.size else None,
            "mean_rel_err": float(errs.mean()) if errs.size else None,
            "assignment_equal": same / max(len(sampled), 1)}


def dump_sample(args, wl, first, es, e_exact, e_bf16):
    """The exact and BF16 forms' energies at a seeded sample of the units, for an FP64 check off the GPU machine
    (tests/fp64_sample_report.py solves the same units with the oracle)."""
    n_s = max(1, int(round(args.fp64_sample_frac * total_units(wl))))
    picks = np.array(sample_units(wl, n_s, 21), dtype=np.int64)
    rows = np.array([int(es[m_ * len(wl.scenes) + s_]) + o_ - int(first[m_ * len(wl.scenes) + s_])
                     for m_, s_, o_ in picks], dtype=np.int64)
    np.savez(args.fp64_dump, workload=args.workload, hop=args.hop, units=picks, e_exact=e_exact[rows],
             e_bf16=e_bf16[rows])
    return {"path": args.fp64_dump, "units": int(n_s), "fraction": args.fp64_sample_frac}


def run_pruned(args, torch, hgm, wl, job_cs, models, scenes, energy, assign, first, es, as_, dev, stream, world,
               flush, sampled, dist=None):
    """The BF16-distance + learned-pruning forms on the same batch: BF16 tensor-core unary table, the
    proposal network keeps `keep` of the 64 candidates per list, recursion on the short lists, exact fallback
    for infeasible units (optionally the `refine` offsets of lowest pruned energy per pair re-solved
    unpruned). Quality is measured against this run's exact results (energy/assign hold them), errors
    against the FP64 oracle at the sampled units."""
    from paper_1505_00581_gb300 import prop_train
    e_ref = energy.cpu().numpy().copy()
    a_ref = assign.cpu().numpy().copy()
    t0 = time.time()
    rank = int(os.environ.get("RANK", "0"))
    if args.no_network:
        prop, info = None, {}
    elif args.checkpoint:
        prop, info = prop_train.load_checkpoint(args.checkpoint), {"checkpoint": args.checkpoint}
    else:
        train_wl = job_cs.training_scenes(101 + 1000 * rank) if job_cs is not None else None
        prop, info = prop_train.train_default(torch, wl, steps=args.train_steps, seed=101 + 1000 * rank,
                                              train_wl=train_wl)
    train_s = time.time() - t0
    steps, warm = max(1, min(args.steps, 5)), min(args.warmup, 3)
    M_rows = []
    for mi, m in enumerate(wl.models):
        for si in range(len(wl.scenes)):
            q = mi * len(wl.scenes) + si
            M_rows.append((int(as_[q]), int(es[q + 1] - es[q]), m.n))
    e_rows = [int(es[q]) for q in range(len(M_rows))]
    masks = prop_train.implant_masks(wl, first, es)
    e2 = torch.empty_like(energy)
    a2 = torch.empty_like(assign)
    pk, pk_kind = peaks()

    def form(p, label, with_graph=False, profile=False):
        hgm.prune_counters(reset=True)
        hgm.refine_counter(reset=True)
        ms, prof = _time_form(torch, hgm, models, scenes, p, e2, a2, steps, warm, stream, flush, profile)
        ms = max_over_ranks(ms, dist, dev)
        n_pruned, n_fb = hgm.prune_counters(reset=True)
        n_ref = hgm.refine_counter(reset=True)
        eh, ah = e2.cpu().numpy(), a2.cpu().numpy()
        out = {"value": job_rate(wl.total_frames, world, ms / 1e3), "unit": "frames/s", "ms_per_step": ms,
               "steps": steps, "form": label, "kernel_ms_per_step": {k: v[0] / steps for k, v in prof.items()},
               **prop_train.compare(e_ref, a_ref, eh, ah, M_rows, e_rows, masks)}
        if n_pruned:
            out["fallback_units_per_step"] = n_fb / (steps + warm)
            out["units_per_step"] = n_pruned / (steps + warm)
        if n_ref:
            out["refined_units_per_step"] = n_ref / (steps + warm)
        if sampled:
            out["fp64"] = fp64_errors(sampled, wl, first, es, as_, eh, ah)
        if with_graph and not args.no_graph:
            g_ms = max_over_ranks(_time_plan(torch, hgm, models, scenes, p, e2, a2, max(1, min(steps, 3)), 1, stream,
                                             flush), dist, dev)
            out["graph"] = {"value": job_rate(wl.total_frames, world, g_ms / 1e3), "unit": "frames/s",
                            "ms_per_step": g_ms}
        return out, prof

    if prop is None:   # the precision form alone (no learned stage)
        out, _ = form(params_of(hgm, wl, precision=1),
                      "BF16 unary + FP32 re-score of the 8 smallest of every list, no pruning", True)
        out["speedup_note"] = "precision form only (--no-network)"
        if args.fp64_dump:
            out["fp64_dump"] = dump_sample(args, wl, first, es, e_ref, e2.cpu().numpy())
        return out
    # keep 8 is the configuration the learned stage is specified with; on the combined workload (models of up
    # to 256 points) most units have no time-ordered chain through 8 candidates per point and fall back to the
    # exact solve, so its main form keeps 16
    keep = args.keep if args.keep is not None else (16 if job_cs is not None else 8)
    pruned, prof = form(params_of(hgm, wl, precision=1, prune=prop, keep=keep),
                        f"BF16 unary + FP32 re-score of the kept candidates, network keeps {keep} of {wl.K}",
                        args.profile_form != "pruned", args.profile_form == "pruned")
    cands = sum(wl.n_offsets(mi, si) * wl.models[mi].n * wl.K
                for mi in range(len(wl.models)) for si in range(len(wl.scenes)))
    prune_ms = prof["prune"][0] / steps
    sc_tflops = cands * 2.0 * 128 * 128 / (prune_ms / 1e3) / 1e12
    pruned["scoring_roofline"] = {"kernel": "prop_score_kernel (+ keep, re-score)", "bound": "tensor",
                                  "achieved": sc_tflops, "peak": pk.get("bf16_tflops", 1900.0), "unit": "TFLOP/s",
                                  "frac": sc_tflops / pk.get("bf16_tflops", 1900.0),
                                  "work": f"{cands} candidate slots x 2 x 128 x 128 (layer 2 on the tensor cores)",
                                  "peak_source": f"bf16_tflops of MEASURED_PEAKS.json ({pk_kind})"}
    pruned["keep"] = keep
    if args.profile_form == "pruned":   # a profiling run: the main pruned form alone
        return pruned
    if keep != 8:
        pruned["keep8"], _ = form(params_of(hgm, wl, precision=1, prune=prop, keep=8),
                                  f"network keeps 8 of {wl.K} (the learned stage as specified)")
    refine = args.refine if args.refine is not None else (8 if job_cs is not None else 32)
    rkeep = 16 if job_cs is not None else 12
    pruned["refined"], _ = form(params_of(hgm, wl, precision=1, prune=prop, keep=rkeep, refine=refine),
                                f"network keeps {rkeep} of {wl.K}, then per (model, scene) pair the {refine} offsets "
                                f"of lowest pruned energy solved unpruned")
    pruned["refined"].update(keep=rkeep, refine=refine)
    pruned["bf16_unpruned"], _ = form(params_of(hgm, wl, precision=1),
                                      "BF16 unary + FP32 re-score of the 8 smallest of every list, no pruning")
    if args.fp64_dump:
        pruned["fp64_dump"] = dump_sample(args, wl, first, es, e_ref, e2.cpu().numpy())
    # the same cut without the network: the 8 smallest unary costs (K = 8 window cap), BF16 + re-score
    pb = params_of(hgm, wl, K=8, precision=1)
    _, es8, as8 = hgm.batch_layout(models, scenes, pb)
    e8 = torch.empty(int(es8[-1]), dtype=torch.float32, device=dev)
    a8 = torch.empty(int(as8[-1]), dtype=torch.int32, device=dev)
    ms8, _ = _time_form(torch, hgm, models, scenes, pb, e8, a8, steps, warm, stream, flush)
    ms8 = max_over_ranks(ms8, dist, dev)
    pruned["top8_by_unary_baseline"] = {
        "value": job_rate(wl.total_frames, world, ms8 / 1e3), "unit": "frames/s", "ms_per_step": ms8,
        **prop_train.compare(e_ref, a_ref, e8.cpu().numpy(), a8.cpu().numpy(), M_rows, e_rows, masks)}
    pruned["training"] = {k: v for k, v in info.items() if k != "loss"}
    pruned["final_loss"] = (info.get("loss") or [[0, None]])[-1][1]
    pruned["train_s"] = train_s
    prop.close()
    return pruned


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="combined")
    ap.add_argument("--hop", type=int, default=256, help="combined workload: offsets owned by each block")
    ap.add_argument("--ref-units", type=int, default=16, help="reference arm: oracle units per step")
    ap.add_argument("--cpu-units", type=int, default=96, help="cpu_baseline: oracle units on all host threads")
    ap.add_argument("--cpu-units-1t", type=int, default=4, help="cpu_baseline: oracle units on one thread")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph replay lines")
    ap.add_argument("--no-pruned", action="store_true", help="skip the pruned+BF16 forms")
    ap.add_argument("--no-blocks", action="store_true", help="skip the whole-block and streaming forms")
    ap.add_argument("--forms", default=None,
                    help="comma list of extra forms: chains,dummy (default: both on batched_exact only)")
    ap.add_argument("--refine", type=int, default=None, help="refined pruned form: offsets re-solved per pair")
    ap.add_argument("--keep", type=int, default=None, help="pruned form: candidates kept per list")
    ap.add_argument("--no-network", action="store_true",
                    help="pruned_bf16 holds only the BF16-distance form (no proposal network is trained)")
    ap.add_argument("--fp64-dump", default=None,
                    help="write the exact and BF16 forms' energies at a seeded sample of units to this .npz")
    ap.add_argument("--fp64-sample-frac", type=float, default=0.01, help="fraction of units in --fp64-dump")
    ap.add_argument("--profile-form", default="exact", choices=["exact", "pruned", "dummy", "whole_block"],
                    help="whose timed steps are bracketed by cudaProfilerStart/Stop (for ncu --profile-from-start "
                         "off); pruned also skips the secondary pruned forms")
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--checkpoint", default=None, help="load the proposal network from <path>.bin/.json")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_1505_00581_gb300 import build as hgm_build
    if rank == 0:
        hgm_build.build()
    if dist:
        dist.barrier()
    from paper_1505_00581_gb300 import hgm
    hgm.load()

    t_gen = time.time()
    wl, job = workload(args.workload, rank, args.hop)
    job_cs = None
    if args.workload.startswith("combined"):
        from paper_1505_00581_gb300 import synth
        job_cs = synth.CombinedScenes(seed=3)
    t_gen = time.time() - t_gen
    dev = torch.device("cuda", local)
    p = params_of(hgm, wl)
    models = [hgm.Model(*(torch.from_numpy(a).to(dev) for a in (m.xy, m.t, m.f))) for m in wl.models]
    scenes = [hgm.Scene(*(torch.from_numpy(a).to(dev) for a in (s.xy, s.t, s.f)), s.n_frames) for s in wl.scenes]
    first, es, as_ = hgm.batch_layout(models, scenes, p)
    n_out, n_assign = int(es[-1]), int(as_[-1])
    energy = torch.empty(n_out, dtype=torch.float32, device=dev)
    assign = torch.empty(n_assign, dtype=torch.int32, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB): evicts between steps

    # algorithmic work: feasible triples of the whole batch (outside the timed region)
    triples = 0
    for mi, m in enumerate(models):
        for si, s in enumerate(scenes):
            q = mi * len(scenes) + si
            n = int(es[q + 1] - es[q])
            if n:
                buf = torch.empty(n, dtype=torch.int64, device=dev)
                hgm.count_triples(m, s, p, int(first[q]), n, buf)
                triples += int(buf.sum().item())

    stream = torch.cuda.current_stream()
    variant, variant_ms = hgm.autotune(models, scenes, p, sample_offsets=16 if job_cs is not None else 128,
                                       use_cache=False)
    for _ in range(args.warmup):
        hgm.match_batch(models, scenes, p, energy, assign)
    torch.cuda.synchronize()
    # evaluations the recursion's triple loop performs (branch and bound skips provably losing z_i):
    # one untimed pass of the accounting variant of the kernel
    hgm.profile_evaluated(reset=True)
    hgm.profile_enable(2)
    hgm.match_batch(models, scenes, p, energy, assign)
    hgm.profile_enable(False)
    evaluated = hgm.profile_evaluated(reset=True)
    hgm.profile_reset()
    hgm.profile_enable(True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if args.profile_form == "exact":
        torch.cuda.profiler.start()     # an ncu run with --profile-from-start off captures only the timed steps
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            hgm.match_batch(models, scenes, p, energy, assign)
            ends[k].record(stream)
        torch.cuda.synchronize()
    if args.profile_form == "exact":
        torch.cuda.profiler.stop()
    if dist:
        dist.barrier()
    hgm.profile_enable(False)
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    prof = hgm.profile_read()
    ms_max = max_over_ranks(ms, dist, dev)
    ms_step = ms_max / args.steps
    value = job_rate(wl.total_frames, world, ms_step / 1e3)
    fin = torch.isfinite(energy).sum().item()

    # end to end: host arrays -> handles -> batch -> host outputs, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        host_m = [tuple(pin(a) for a in (m.xy, m.t, m.f)) for m in wl.models]
        host_s = [tuple(pin(a) for a in (s.xy, s.t, s.f)) for s in wl.scenes]
        host_e = torch.zeros(n_out, dtype=torch.float32).pin_memory()
        host_a = torch.zeros(n_assign, dtype=torch.int32).pin_memory()
        h2d = sum(a.numel() * a.element_size() for arrs in host_m + host_s for a in arrs)
        d2h = host_e.numel() * 4 + host_a.numel() * 4
        e2e_times = []
        for k in range(max(1, min(args.steps, 3)) + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ms_ = [hgm.Model(*arrs) for arrs in host_m]
            ss_ = [hgm.Scene(*arrs, s.n_frames) for arrs, s in zip(host_s, wl.scenes)]
            hgm.match_batch(ms_, ss_, p, host_e, host_a)
            t1 = time.perf_counter()
            for h in ms_ + ss_:
                h.close()
            if k > 0:
                e2e_times.append(t1 - t0)
        e2e_sec = max_over_ranks(float(np.mean(e2e_times)), dist, dev)
        same = bool(torch.equal(host_e, energy.cpu()) and torch.equal(host_a, assign.cpu()))
        e2e = {"value": job_rate(wl.total_frames, world, e2e_sec), "unit": "frames/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "results_equal_device_run": same}

    # the same exact batch replayed as a CUDA graph (hgm_plan)
    graph = None
    if not args.no_graph:
        g_ms = max_over_ranks(_time_plan(torch, hgm, models, scenes, p, energy, assign, max(1, min(args.steps, 3)),
                                         1, stream, flush), dist, dev)
        graph = {"value": job_rate(wl.total_frames, world, g_ms / 1e3), "unit": "frames/s", "ms_per_step": g_ms,
                 "form": "plain exact FP32, one graph launch per step"}

    clk_sum = clk.summary()
    rec_ms, rec_n = prof["recurse"]
    rec_avg_ms = rec_ms / max(rec_n, 1)
    # the recursion handles the step's units in rec_n / steps launches (chunks bounded by the workspace)
    chunks_per_step = max(1, rec_n // args.steps)
    eval_per_launch = evaluated / chunks_per_step
    achieved = eval_per_launch * OPS_PER_TRIPLE / (rec_avg_ms / 1e3) / 1e12
    peak_ops, peak_src = alu_peak(torch)
    traffic, beta_bytes = recurse_traffic(wl, chunks_per_step)
    roofline = {"bound": "alu", "kernel": "recurse_kernel", "achieved": achieved, "peak": peak_ops,
                "unit": "Tops/s (FP32 lane ops)", "frac": achieved / peak_ops, "traffic": traffic,
                "traffic_source": None if traffic is None else
                f"ncu DRAM bytes of the {RECURSE_NCU['case']} capture, scaled by argmin-table bytes "
                f"{beta_bytes:.4g} / {RECURSE_NCU['beta_bytes']:.4g}",
                "argmin_table_bytes_per_launch": beta_bytes, "peak_source": peak_src,
                "evaluated_triples_per_launch": eval_per_launch, "ops_per_triple": OPS_PER_TRIPLE,
                "feasible_triples_per_launch": triples / chunks_per_step,
                "feasible_triples_per_s": triples / chunks_per_step / (rec_avg_ms / 1e3),
                "avg_launch_ms": rec_avg_ms, "launches_per_step": chunks_per_step,
                "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()}}
    # the other kernels of the step against their own bounds
    F_pad = (wl.models[0].F + 3) // 4 * 4
    R_rows = sum(m.n for m in wl.models)
    pairs_u = R_rows * sum(sc_.n for sc_ in wl.scenes)
    un_ms = prof["unary"][0] / args.steps
    sel_ms = prof["select"][0] / args.steps
    lists = sum(wl.n_offsets(mi, si) * wl.models[mi].n for mi in range(len(wl.models)) for si in range(len(wl.scenes)))
    roofline["other_kernels"] = {
        "unary_kernel": {"bound": "alu", "achieved": pairs_u * 2 * F_pad / (un_ms / 1e3) / 1e12, "peak": peak_ops,
                         "unit": "Tops/s (FP32 lane ops)",
                         "frac": pairs_u * 2 * F_pad / (un_ms / 1e3) / 1e12 / peak_ops,
                         "work": f"{pairs_u:.4g} (model point, scene point) pairs x 2 x {F_pad} ops"},
        "select_kernel": {"bound": "latency", "lists_per_s": lists / (sel_ms / 1e3), "ms_per_step": sel_ms,
                          "work": f"{lists} candidate lists (4 radix passes over each window)"}}
    launches = sum(v[1] for v in prof.values())

    # the FP64 oracle on the host cores: all threads and one thread, on seeded units of this batch, which
    # also serve as the FP64 check of every GPU form
    cpu, sampled = None, []
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        units = sample_units(wl, max(threads, args.cpu_units), 11)
        t_all, res = oracle_time(wl, units, threads)
        sampled = list(zip(units, res))
        u1 = sample_units(wl, max(1, args.cpu_units_1t), 12)
        t_one, _ = oracle_time(wl, u1, 1)
        n_batch = total_units(wl)
        cpu = {"value": wl.total_frames / (t_all / len(units) * n_batch), "unit": "frames/s", "cores": threads,
               "kind": "oracle",
               "sample": f"{len(units)} seeded units of the batch's {n_batch} ({t_all:.1f} s on {threads} threads), "
                         f"projected to the batch",
               "single_thread": {"value": wl.total_frames / (t_one / len(u1) * n_batch), "unit": "frames/s",
                                 "sample": f"{len(u1)} seeded units ({t_one:.1f} s on 1 thread)"},
               "fp64_check": fp64_errors(sampled, wl, first, es, as_, energy.cpu().numpy(), assign.cpu().numpy())}

    forms = set((args.forms or ("chains,dummy" if args.workload == "batched_exact" else "")).split(",")) - {""}
    chains = run_chains(args, torch, hgm, wl, models, scenes, dev, stream, world, flush, dist) \
        if "chains" in forms else None
    dummy = run_dummy(args, torch, hgm, wl, models, scenes, dev, stream, world, flush, dist) \
        if "dummy" in forms else None
    blocks = None if args.no_blocks else run_blocks(args, torch, hgm, dev, stream, flush)
    pruned = None
    if not args.no_pruned:
        pruned = run_pruned(args, torch, hgm, wl, job_cs, models, scenes, energy, assign, first, es, as_, dev,
                            stream, world, flush, sampled, dist)
        pruned["speedup_vs_exact"] = pruned["value"] / value
        # the precision path's (BF16 distance + FP32 re-score, unpruned) error on the oracle's units, beside the
        # exact path's
        bf = pruned if args.no_network else pruned.get("bf16_unpruned")
        if cpu is not None and bf and bf.get("fp64"):
            cpu["fp64_check_bf16_rescore"] = bf["fp64"]

    if rank == 0:
        cfg = config_of(wl, job, args, world)
        line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
                "form": "plain exact FP32 (value); pruned_bf16 holds the BF16-distance + learned-pruning forms",
                "recurse_variant": variant, "autotune_ms": variant_ms,
                "feasible_triples_per_step": triples, "evaluated_triples_per_step": evaluated,
                "input_generation_s": t_gen,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "graph": graph, "gpu_launches": launches,
                "clocks": clk_sum, "finite_offsets": int(fin), "pruned_bf16": pruned,
                "chains": chains, "whole_block": blocks, "dummy": dummy}
        if job is not None:
            line["job_seconds_at_value"] = job["job_frames"] / value
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
