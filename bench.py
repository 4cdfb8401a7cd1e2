"""Benchmark: SDP-BSREM ordered-subsets subiterations per second on one GB300.

One step = one whole reconstruction of the clinical-size stacked workload (256 x 256 x 89
planes at 2.7 mm, 288 views x 357 bins, 24 subsets, 20 iterations of SDP-P2(24), with the
objective Phi(f^k) after every iteration): 480 subiterations (subset forward projection +
Poisson ratio, gather backprojection + RDP gradient + nu + preconditioned update + clamp,
the mu reduction when nu is dynamic) plus 21 objective evaluations, on inputs already
resident in HBM.  L2 is flushed (a 256 MiB write) before every timed step and each step is
timed with CUDA events on its stream.  ``value`` = subiterations per second over the job.

``e2e`` repeats the measurement through pet_reconstruct_host from pinned host buffers (counts,
gamma and f^0 copied in, f^T and the objective history copied out inside the timed call).

``--impl reference`` times the FP64 CPU oracle instead (bounded sample of subiterations of the
same workload on the host cores).  Multi-GPU: independent replicas, one scan per rank, no
collective (scans do not exchange data).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2111_07886_gb300 import synth  # noqa: E402

L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="stacked", choices=["stacked", "2d"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer measurement")
    ap.add_argument("--no-kernel-times", action="store_true",
                    help="skip the per-kernel event pass (roofline)")
    ap.add_argument("--ray-chunks", type=int, default=0,
                    help="pin the forward projector's ray chunks instead of autotuning (profiling "
                         "runs: the profiler's per-launch cost distorts the autotuner's timings)")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-scan batched run")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the no-objective and FP32 / FP64 arithmetic measurements")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-loop run")
    ap.add_argument("--serve-requests", type=int, default=500)
    ap.add_argument("--serve-slots", type=int, default=8,
                    help="scans the server keeps resident (1: one at a time, FIFO)")
    ap.add_argument("--serve-rates", default="0.5,0.9,1.5",
                    help="arrival rates as fractions of the sequential plain capacity")
    return ap.parse_args()


def workload(name: str):
    return synth.config_stacked_256x89(seed=0) if name == "stacked" else synth.config_2d_128(seed=0)


def algo_config(p) -> dict:
    """The SDP-BSREM parameters the run uses (the P2 form of Sec. III with the workload's rho,
    delta, a and nu bounds, not Table II's SDP-P2 rows)."""
    names = {0: "BSREM", 1: "SDP-M1", 2: "SDP-M2", 3: "SDP-P1", 4: "SDP-P2"}
    return {"precond": names[p.precond], "rho": p.rho, "delta1": p.delta1, "delta2": p.delta2,
            "a": p.a, "lambda0": p.lambda0, "nu1": p.nu1, "nu2": p.nu2, "J0": p.J0, "J1": p.J1,
            "gamma_r": p.gamma_r, "eps": p.eps, "t": p.t, "U": p.U,
            "params_source": "P2 form (Sec. III) with workload settings; Table II's P2 rows are "
                             "chaotic on these phantoms"}


def workload_config(w) -> dict:
    return {"workload": w.name, "image": [w.nplanes, w.n, w.n], "pixel_mm": w.pixel_mm,
            "views": w.nviews, "bins": w.nbins, "subsets": w.nsubsets,
            "iterations": w.params.iterations, **algo_config(w.params), "beta": w.params.beta,
            "counts": w.counts, "subiters_per_step": w.params.iterations * w.nsubsets,
            "objective_per_iteration": True, "l2": "flushed (256 MiB write) before each step",
            "global_batch": 1, "parallelism": "replicas"}


def replica_seed(base_seed: int, rank: int) -> int:
    """Each replica reconstructs its own scan (weak scaling, no data-path collective)."""
    return base_seed + 1000 * rank


def reduce_max(value: float, world: int, device) -> float:
    """Max over ranks (the job is as slow as its slowest replica)."""
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job units per second: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / (ms_max / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# roofline: algorithmic bytes per launch of each kernel kind
# ------------------------------------------------------------------------------------------
def algorithmic_bytes(w) -> dict:
    q = w.n * w.n * w.nplanes                                  # image elements
    sub_bins = (w.nviews // w.nsubsets) * w.nbins * w.nplanes  # |I_i| (equal subsets here)
    all_bins = w.nviews * w.nbins * w.nplanes
    return {
        # f read, counts + gamma read, ratio w written
        "forward_ratio": 4 * q + 12 * sub_bins,
        # w read, f read, 1/p read (one plane), f written
        "update": 4 * sub_bins + 8 * q + 4 * w.n * w.n,
        "mu_sum": 4 * q,
        # f read, counts + gamma read (all views)
        "obj_forward": 4 * q + 8 * all_bins,
        "rdp_value": 4 * q,
    }


def load_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback"}


def kernel_source_hash() -> str:
    import glob
    import hashlib
    h = hashlib.sha256()
    base = os.path.join(ROOT, "paper_2111_07886_gb300", "csrc")
    for f in sorted(glob.glob(os.path.join(base, "*.cu")) + glob.glob(os.path.join(base, "*.cuh"))):
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary of the same kernel; None when the
    kernel sources changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        if d.get("source_hash") != kernel_source_hash():
            return None
        return d.get(kernel)
    except Exception:
        return None


# ------------------------------------------------------------------------------------------
def run_ours(args, rank, world, local):
    import torch
    from paper_2111_07886_gb300 import pet

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args.workload)
    w.seed = replica_seed(w.seed, rank)
    scan = synth.make_scan(w)
    g = pet.Geometry.from_dict(w.geometry(), scan["sens"])
    if args.ray_chunks > 0:
        g.set_ray_chunks(args.ray_chunks)        # pinned (profiling runs), no autotuning
        tuned_S = args.ray_chunks
    else:
        tuned_S = g.autotune()
    prm = pet.make_params(w.params)
    counts = torch.from_numpy(scan["counts"]).to(dev)
    gamma = torch.from_numpy(scan["gamma"]).to(dev)
    f0 = torch.ones((w.nplanes, w.n, w.n), dtype=torch.float32, device=dev)
    img = torch.empty_like(f0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    subiters = w.params.iterations * w.nsubsets

    def step():
        img.copy_(f0)
        return pet.reconstruct(g, counts, gamma, prm, img, objective=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    n0 = pet.launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    t_wall = time.perf_counter()
    obj = None
    for k in range(args.steps):
        flush.fill_(float(k))
        evs[k][0].record(stream)
        obj = step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    launches = (pet.launch_count() - n0) // args.steps
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    if world > 1:
        torch.distributed.barrier()
    ms_max = reduce_max(ms, world, dev)
    ms_per_step = ms_max / args.steps
    value = job_throughput(subiters, world, ms_per_step)

    line = {
        "metric": "OS subiters/s", "value": round(value, 2), "unit": "subiters/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (Kahan sums) + f64 scalars/objective",
        "data": "synthetic (seeded random-ellipsoid phantom, analytic projections, Poisson counts)",
        "config": {**workload_config(w),
                   ("ray_chunks_pinned" if args.ray_chunks > 0 else "autotuned_ray_chunks"): tuned_S},
        "clocks": clk, "gpu_launches": int(launches),
        "wall_s_timed": round(wall, 3), "objective_final": obj[-1] if obj else None,
    }
    if not args.no_variants:
        line["variants"] = variants_measure(args, w, g, counts, gamma, pet, flush, subiters)
        line["variants"]["tof"] = tof_measure(w, scan, pet, flush, subiters)
    if not args.no_kernel_times:
        line.update(kernel_times(args, w, pet, step, flush))
    if not args.no_e2e:
        line["e2e"] = end_to_end(args, w, scan, g, prm, pet, flush, dev, world, subiters)
    if not args.no_batched:
        line["batched"] = batched_measure(pet, torch)
    if not args.no_serving:
        line["serving"] = serving_measure(args, pet, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, scan, args.cpu_seconds)
    return line


def variants_measure(args, w, g, counts, gamma, pet, flush, subiters) -> dict:
    """Subiterations per second of the same reconstruction (a) without the per-iteration
    objective, which the paper evaluates for reporting only, and (b) in the other arithmetics of
    the precision study: plain FP32 sums and FP64 on the GPU (with the objective, as the main
    line).  CUDA events, L2 flushed before each step."""
    import torch
    stream = torch.cuda.current_stream()
    f0 = torch.ones((w.nplanes, w.n, w.n), dtype=torch.float32, device=counts.device)
    img = torch.empty_like(f0)

    def timed(prm, objective, steps, warm):
        def one():
            img.copy_(f0)
            pet.reconstruct(g, counts, gamma, prm, img, objective=objective)
        for _ in range(warm):
            one()
        ms = 0.0
        for k in range(steps):
            flush.fill_(float(k))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            one()
            b.record(stream)
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
        return round(subiters / (ms / steps / 1e3), 2), round(ms / steps, 3)

    out = {"unit": "subiters/s"}
    v, ms = timed(pet.make_params(w.params), False, max(1, min(args.steps, 3)), 1)
    out["no_objective"] = {"value": v, "ms_per_step": ms, "precision": "fp32+kahan"}
    v, ms = timed(pet.make_params(w.params, synth.PREC_FP32), True, max(1, min(args.steps, 3)), 1)
    out["fp32_plain_sums"] = {"value": v, "ms_per_step": ms, "objective_per_iteration": True}
    v, ms = timed(pet.make_params(w.params, synth.PREC_FP64), True, 1, 1)
    out["fp64_on_gpu"] = {"value": v, "ms_per_step": ms, "objective_per_iteration": True}
    return out


TOF_BINS, TOF_BIN_MM, TOF_FWHM_MM = 13, 60.0, 82.5     # ~550 ps timing resolution


def tof_measure(w, scan, pet, flush, subiters) -> dict:
    """The same reconstruction (with the per-iteration objective) as TOF data: 13 TOF bins of
    60 mm per bin, timing kernel FWHM 82.5 mm (about 550 ps).  The counts are Poisson draws of
    the library's own TOF projection of the phantom sampled at the pixel centres (plus the same
    10 % uniform background); one warm-up and one timed reconstruction, CUDA events."""
    import torch
    dev = torch.device("cuda")
    geo = dict(w.geometry(), tof_bins=TOF_BINS, tof_bin_mm=TOF_BIN_MM, tof_fwhm_mm=TOF_FWHM_MM)
    g = pet.Geometry.from_dict(geo, scan["sens"])
    img = torch.from_numpy(synth.rasterize(scan["planes"], w.n, w.pixel_mm, supersample=1)
                           .astype(np.float32)).to(dev)
    proj = torch.empty((w.nplanes, w.nviews, w.nbins, TOF_BINS), device=dev)
    pet.forward_subset(g, -1, img, proj)
    gam = torch.full_like(proj, float(0.1 * proj.mean()))
    gen = torch.Generator(device=dev)
    gen.manual_seed(w.seed + 31)
    counts = torch.poisson(proj + gam, generator=gen).to(torch.int32)
    f0 = torch.ones((w.nplanes, w.n, w.n), device=dev)
    out_img = torch.empty_like(f0)
    prm = pet.make_params(w.params)
    stream = torch.cuda.current_stream()

    def one():
        out_img.copy_(f0)
        pet.reconstruct(g, counts, gam, prm, out_img, objective=True)

    one()
    flush.fill_(3.0)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    one()
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    g.close()
    return {"value": round(subiters / (ms / 1e3), 2), "ms_per_step": round(ms, 3),
            "tof_bins": TOF_BINS, "tof_bin_mm": TOF_BIN_MM, "tof_fwhm_mm": TOF_FWHM_MM,
            "objective_per_iteration": True}


def kernel_times(args, w, pet, step, flush) -> dict:
    """Per-kernel device time: a second pass with every launch bracketed by CUDA events on
    its stream; the dominant kernel's roofline from its algorithmic bytes per launch."""
    import torch
    pet.profile_reset()
    pet.profile_enable(True)
    for k in range(args.steps):
        flush.fill_(float(k))
        step()
    torch.cuda.synchronize()
    prof = pet.profile_read()
    pet.profile_enable(False)
    byts = algorithmic_bytes(w)
    # with per-kernel timing on, the library runs its side-stream work (mu pass, objective) on
    # the caller's stream, so each event pair brackets one kernel alone, as in an ncu launch list
    tot = sum(v[0] for v in prof.values())
    shares = {k: {"ms": round(v[0] / max(1, args.steps), 4), "launches_per_step": v[1] // max(1, args.steps),
                  "share": round(v[0] / tot, 4) if tot else 0.0} for k, v in prof.items() if v[1]}
    dom = max((k for k in prof if k in byts and prof[k][1]), key=lambda k: prof[k][0])
    avg_ms = prof[dom][0] / prof[dom][1]
    peaks = load_peaks()
    achieved = byts[dom] / (avg_ms / 1e3) / 1e9
    roof = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
            "peak_source": peaks["source"] + " (burst copy)", "unit": "GB/s",
            "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": ncu_traffic(dom),
            "algorithmic_bytes_per_launch": byts[dom], "avg_launch_ms": round(avg_ms, 5)}
    # every kernel kind against the same peak; the projector's fraction is the one the 50 % HBM
    # target names (forward_ratio inside the subiteration, obj_forward for the objective)
    by_kind = {}
    for k in byts:
        if k in prof and prof[k][1]:
            ms_k = prof[k][0] / prof[k][1]
            ach = byts[k] / (ms_k / 1e3) / 1e9
            by_kind[k] = {"achieved": round(ach, 1), "frac": round(ach / peaks["hbm_gbs"], 4),
                          "algorithmic_bytes_per_launch": byts[k], "avg_launch_ms": round(ms_k, 5),
                          "traffic": ncu_traffic(k)}
    proj = by_kind.get("forward_ratio", {}).get("frac")
    roof["by_kernel"] = by_kind
    roof["projector_target"] = {"kernel": "forward_ratio", "frac": proj, "target_frac": 0.5,
                                "met": bool(proj is not None and proj >= 0.5)}
    return {"roofline": roof, "kernels": shares}


def end_to_end(args, w, scan, g, prm, pet, flush, dev, world, subiters) -> dict:
    """Same metric through pet_reconstruct_host from pinned host buffers."""
    import torch
    h_counts = torch.from_numpy(scan["counts"]).pin_memory()
    h_gamma = torch.from_numpy(scan["gamma"]).pin_memory()
    h_img = torch.ones((w.nplanes, w.n, w.n), dtype=torch.float32).pin_memory()
    h_f0 = h_img.clone()
    e2e_steps = max(1, min(args.steps, 3))
    pet.reconstruct_host(g, h_counts.numpy(), h_gamma.numpy(), prm, h_img.numpy(), objective=True)
    e2e_ms = 0.0
    for k in range(e2e_steps):
        h_img.copy_(h_f0)
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pet.reconstruct_host(g, h_counts.numpy(), h_gamma.numpy(), prm, h_img.numpy(), objective=True)
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_ms /= e2e_steps
    e2e_max = reduce_max(e2e_ms, world, dev)
    e2e = {"value": round(job_throughput(subiters, world, e2e_max), 2), "unit": "subiters/s",
           "h2d_bytes_per_step": int(h_counts.numel() * 4 + h_gamma.numel() * 4 + h_img.numel() * 4),
           "d2h_bytes_per_step": int(h_img.numel() * 4 + 8 * (w.params.iterations + 1)),
           "api": "pet_reconstruct_host", "ms_per_step": round(e2e_max, 3)}
    return e2e


def batched_measure(pet, torch) -> dict:
    """64 independent 2-D scans of mixed sizes (N in {128, 200, 256, 400}, 120-360 views,
    12-36 subsets, 10 iterations, objective each iteration): all advanced together by the
    batched, graph-replayed kernels, against the plain path (pet_reconstruct, one scan at a
    time).  Same states, same bits (tests check it); both timed with CUDA events."""
    dev = torch.device("cuda")
    ws = synth.mixed_2d_scans(64, seed=0, iterations=10)
    scans = [synth.make_scan(w) for w in ws]
    stream = torch.cuda.Stream()
    items = []
    for w, sc in zip(ws, scans):
        g = pet.Geometry.from_dict(w.geometry(), sc["sens"])
        c = torch.from_numpy(sc["counts"]).to(dev)
        gm = torch.from_numpy(sc["gamma"]).to(dev)
        f0 = torch.ones((1, w.n, w.n), device=dev)
        st = pet.State(g, c, gm, pet.make_params(w.params), f0)
        items.append((w, g, c, gm, f0, st))
    subiters = sum(w.params.iterations * w.nsubsets for w in ws)
    batch = pet.Batch(64, use_graph=True)

    def batched_run():
        for it in items:
            if it[5] in batch.members:
                batch.remove(it[5])
            it[5].reset(stream=stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for it in items:
            batch.add(it[5], with_objective=True, stream=stream)
        n0 = pet.launch_count()
        ticks = 0
        while batch.step(stream=stream) > 0:
            ticks += 1
        b.record(stream)
        stream.synchronize()
        return a.elapsed_time(b) / 1e3, ticks + 1, pet.launch_count() - n0

    batched_run()                               # warm-up: graph capture, caches
    tb, ticks, launches = batched_run()

    def plain_run():
        t = 0.0
        for w, g, c, gm, f0, st in items:
            img = f0.clone()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            pet.reconstruct(g, c, gm, pet.make_params(w.params), img, objective=True)
            b.record()
            torch.cuda.synchronize()
            t += a.elapsed_time(b) / 1e3
        return t

    plain_run()
    tp = plain_run()
    # the same with every geometry tuned for 64 scans sharing the GPU (pet_autotune_batch)
    tuned = {}
    for w, g, c, gm, f0, st in items:
        tuned[w.name] = g.autotune_batch(len(items), stream=stream)
    stream.synchronize()
    batched_run()
    tbt, ticks_t, launches_t = batched_run()
    plain_run()
    tpt = plain_run()
    for w, g, c, gm, f0, st in items:
        g.set_ray_chunks(0)
    return {"workload": "64 mixed 2-D scans (N 128-400, 120-360 views, 12-36 subsets, 10 it.)",
            "subiters": subiters, "ticks": ticks, "gpu_launches": int(launches),
            "batched_s": round(tb, 4), "plain_s": round(tp, 4),
            "batched_subiters_per_s": round(subiters / tb, 1),
            "plain_subiters_per_s": round(subiters / tp, 1),
            "batched_scans_per_s": round(len(ws) / tb, 2), "plain_scans_per_s": round(len(ws) / tp, 2),
            "speedup_vs_plain": round(tp / tb, 2),
            "tuned": {"tuner": "pet_autotune_batch(g, 64): forward ray chunks S per geometry",
                      "ray_chunks_per_geometry": tuned,
                      "batched_s": round(tbt, 4), "plain_s": round(tpt, 4),
                      "batched_subiters_per_s": round(subiters / tbt, 1),
                      "batched_scans_per_s": round(len(ws) / tbt, 2),
                      "speedup_vs_untuned_plain": round(tp / tbt, 2),
                      "speedup_vs_untuned_batched": round(tb / tbt, 3)}}


def serving_measure(args, pet, torch) -> dict:
    """Serving loop: a Poisson-arrival stream of requests drawn from the 64 mixed 2-D scans plus
    5 % stacked 256 x 256 x 89 jobs, each run to 20 iterations, at rates that are fractions of
    the sequential plain capacity.  Reports scans/s, p50/p99 latency (submit to result) and the
    mean per-request breakdown (queue, prepare, run, readback), next to the same arrival stream
    served by the plain per-scan path one request at a time (FIFO over service times measured on
    the GPU with inputs resident: no host upload, which favours the plain arm)."""
    dev = torch.device("cuda")
    ws = synth.mixed_2d_scans(64, seed=1, iterations=20)
    ws.append(synth.config_stacked_256x89(seed=5))
    scans = [synth.make_scan(w) for w in ws]
    # plain service time of every pool entry (pet_reconstruct, inputs resident, events)
    service = []
    for w, sc in zip(ws, scans):
        g = pet.Geometry.from_dict(w.geometry(), sc["sens"])
        c = torch.from_numpy(sc["counts"]).to(dev)
        gm = torch.from_numpy(sc["gamma"]).to(dev)
        img = torch.ones((w.nplanes, w.n, w.n), device=dev)
        pet.reconstruct(g, c, gm, pet.make_params(w.params), img, objective=True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        img.fill_(1.0)
        a.record()
        pet.reconstruct(g, c, gm, pet.make_params(w.params), img, objective=True)
        b.record()
        torch.cuda.synchronize()
        service.append(a.elapsed_time(b) / 1e3)
        del g, c, gm, img
    rng = np.random.Generator(np.random.PCG64(42))
    n = args.serve_requests
    pick = [len(ws) - 1 if rng.uniform() < 0.05 else int(rng.integers(0, len(ws) - 1)) for _ in range(n)]
    mean_service = float(np.mean([service[k] for k in pick]))
    capacity = 1.0 / mean_service
    slots = args.serve_slots
    out = {"requests": n, "pool": f"{len(ws) - 1} mixed 2-D scans + 1 stacked 256x256x89 (5 %)",
           "stacked_requests": int(sum(1 for k in pick if k == len(ws) - 1)),
           "iterations": 20, "slots": slots, "autotune": f"pet_serve_autotune({slots})",
           "plain_capacity_scans_per_s": round(capacity, 2),
           "plain_arm": "FIFO over measured GPU service times, inputs resident (no upload)",
           "rates": []}
    for rho in [float(x) for x in args.serve_rates.split(",") if x]:
        gaps = rng.exponential(1.0 / (rho * capacity), size=n)
        arrivals = np.cumsum(gaps) - gaps[0]
        server = pet.Server(hbm_budget_bytes=64 << 30, max_slots=slots)
        server.autotune(slots)
        tickets = {}
        t0 = time.perf_counter()
        done = {}
        k = 0
        while len(done) < n:
            now = time.perf_counter() - t0
            while k < n and arrivals[k] <= now:
                w, sc = ws[pick[k]], scans[pick[k]]
                tickets[server.submit(w.geometry(), sc["sens"], sc["counts"], sc["gamma"],
                                      pet.make_params(w.params), with_objective=True)] = k
                k += 1
            for t in list(tickets):
                r = server.poll(t)
                if r is not None:
                    done[tickets.pop(t)] = r[2]
            time.sleep(0.0005)
        st = server.stats()
        server.close()
        lat_s = np.array([done[i] for i in range(n)])
        big = np.array([pick[i] == len(ws) - 1 for i in range(n)])
        # the same arrivals served one at a time by the plain path (FIFO)
        finish, lat = 0.0, []
        for i in range(n):
            start = max(arrivals[i], finish)
            finish = start + service[pick[i]]
            lat.append(finish - arrivals[i])
        lat = np.array(lat)
        span_plain = finish - arrivals[0]
        out["rates"].append({
            "rho": rho, "served_scans_per_s": round(st["scans_per_s"], 2),
            "p50_s": round(st["p50_s"], 4), "p99_s": round(st["p99_s"], 4),
            "failed": int(st["failed"]),
            "breakdown_mean_s": {k: round(st["mean_" + k + "_s"], 5)
                                 for k in ("queue", "prepare", "run", "readback")},
            "tuned_geometries": int(st["tuned_geometries"]),
            "p50_2d_s": round(float(np.percentile(lat_s[~big], 50)), 4),
            "p50_stacked_s": round(float(np.percentile(lat_s[big], 50)), 4) if big.any() else None,
            "plain_scans_per_s": round(n / span_plain, 2),
            "plain_p50_s": round(float(np.percentile(lat, 50)), 4),
            "plain_p99_s": round(float(np.percentile(lat, 99)), 4),
            "plain_p50_2d_s": round(float(np.percentile(lat[~big], 50)), 4),
            "plain_p50_stacked_s": round(float(np.percentile(lat[big], 50)), 4) if big.any() else None})
    return out


def cpu_baseline(w, scan, seconds: float) -> dict:
    """The FP64 oracle, as it stands, on a bounded sample of the same workload: runs
    ora_reconstruct for a growing number of subiterations until ~`seconds` of CPU time."""
    import oracle
    og = oracle.geom_from(w.geometry(), scan["sens"])
    f0 = np.ones((w.nplanes, w.n, w.n))
    n = 2
    while True:
        t0 = time.perf_counter()
        oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params, f0, nsub=n)
        dt = time.perf_counter() - t0
        if dt >= 0.6 * seconds or n >= w.params.iterations * w.nsubsets:
            break
        n = min(w.params.iterations * w.nsubsets, max(n + 1, int(n * seconds / max(dt, 1e-3))))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": round(n / dt, 4), "unit": "subiters/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} subiterations of {w.name} from f0 = 1 (incl. its sensitivity setup), "
                      f"{dt:.1f} s"}


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step is a bounded sample of subiterations."""
    w = workload(args.workload)
    scan = synth.make_scan(w)
    import oracle
    og = oracle.geom_from(w.geometry(), scan["sens"])
    f0 = np.ones((w.nplanes, w.n, w.n))
    # past J0, so that most sampled subiterations compute nu (Eq. nuki) as the timed run does
    nsub = w.params.J0 + 5 if args.workload == "stacked" else 24
    for _ in range(args.warmup):
        oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params, f0, nsub=1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.reconstruct(og, scan["counts"], scan["gamma"], w.params, f0, nsub=nsub)
    dt = time.perf_counter() - t0
    value = args.steps * nsub / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = f"{nsub} subiterations of {w.name} per step from f0 = 1"
    return {"impl": "reference", "metric": "OS subiters/s", "value": round(value, 4),
            "unit": "subiters/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w),
            "cpu_baseline": {"value": round(value, 4), "unit": "subiters/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "subiters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def spawn_ranks(n: int, argv: list[str]) -> int:
    """`--gpus N` without a launcher: start N ranks of this script with torch.distributed.run
    (one process per GPU, rendezvous on 127.0.0.1); rank 0 prints the job's line."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *argv]
    return subprocess.call(cmd)


def main():
    args = parse()
    if args.gpus > 1 and "RANK" not in os.environ:
        sys.exit(spawn_ranks(args.gpus, sys.argv[1:]))
    rank, world, local = dist_env()
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, rank, world, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
