"""Benchmark of the fused thermal emulsion lattice Boltzmann step on GB300.

Workload: the 1024 x 512 concentrated emulsion (350 droplets, phi = 0.8,
Ra = 3.6e4), synthetic and seeded.  One bench step = one lattice update of
the whole lattice by the fused kernel.  Headline: the FP32-shifted storage
form; the FP64 form is measured on the same workload and reported beside it.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the launching stream; before every timed step a 512 MiB buffer is written
and another 512 MiB buffer is read (L2 flush: the FP32 working set, 113 MB,
fits in the 135 MB L2; the read leaves L2 holding clean lines, so the timed
step does not pay for writing back the flush's own data).
MLUPS = nx * ny * K / sum(step times) / 1e6 (all lattice nodes).

Other forms on the same line: the FP32-fluid + FP16-thermal storage form on
the same lattice (180 B per update); the batched 64-replica ensemble
(aggregate MLUPS); the adjoint on the 512 x 256 emulsion (time of one reverse
step and of the whole sqrt(N)-checkpointed gradient against forward steps);
the 4096 x 2048 rough channel (8.4 M nodes, larger than L2); and the droplet
topology analysis (labels, centres, digital Voronoi, Delaunay links) in
milliseconds and in step equivalents.  Every step form picks its tile with
the cold-L2 autotuner before timing.

``--impl reference`` times the FP64 CPU oracle (OpenMP build, all host
cores) on the same workload and metric, each step a full lattice update.

Multi-GPU: the step does not shard in this build; under torchrun each rank
runs an independent replica (no data-path collective) and rank 0 reports
the aggregate over ranks with the max-over-ranks time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM roofline: FP64 vs FP32-shifted vs batched; adjoint/forward cost"
FLUSH_BYTES = 512 << 20
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# FP64 (non-tensor) peak from the unit counts and the clock: 152 SMs x 2 FP64 FMA per clock per SM
# x 2 flops per FMA x the maximum SM clock (MEASURED_PEAKS.json sm_max_mhz, else 2070 MHz).
FP64_SMS, FP64_FMA_PER_CLK_PER_SM = 152, 2
DETAIL_DEFAULT = os.path.join("_build", "bench_detail.json")  # git-ignored


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return PEAKS_FALLBACK["hbm_gbs"], "fallback"


def fp64_peak_tflops():
    """FP64 FMA-pipe peak of the GPU from its unit counts and maximum SM clock."""
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            mhz = float(json.load(fh).get("sm_max_mhz", mhz))
    except Exception:
        pass
    return FP64_SMS * FP64_FMA_PER_CLK_PER_SM * 2 * mhz * 1e6 / 1e12


def rnd(v, digits=5):
    """Round floats (recursively) to `digits` significant digits to keep the JSON line short."""
    if isinstance(v, float):
        return float(f"{v:.{digits}g}") if v == v and abs(v) != float("inf") else v
    if isinstance(v, dict):
        return {k: rnd(x, digits) for k, x in v.items()}
    if isinstance(v, (list, tuple)):
        return [rnd(x, digits) for x in v]
    return v


# sources that define the step kernels (their DRAM counters go stale when one of these changes)
STEP_KERNEL_SOURCES = ("lb_cfg.h", "lb_kernels.cuh", "lb_f32.cu", "lb_f64.cu", "lb_f32h.cu", "lb_df.cuh", "lb_df64.cu")


def _kernel_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2109_12565_gb300", "csrc")
    for fn in STEP_KERNEL_SOURCES:
        with open(os.path.join(csrc, fn), "rb") as fh:
            h.update(fn.encode() + fh.read())
    return h.hexdigest()[:16]


def _profile_counters():
    """Per-launch DRAM traffic of the step kernels from the committed ncu summary, if it was taken
    on the current kernel sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            d = json.load(fh)
    except Exception:
        return {}
    if d.get("kernel_sources_sha256_16") != _kernel_hash():
        return {}
    return d


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of a list of floats over all ranks (one all-reduce), or the list itself
    without a process group.  Every rank must call it, before any rank leaves."""
    if dist is None:
        return [float(v) for v in values]
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def aggregate_mlups(world, nodes, steps, t_ms_max):
    """Whole-job MLUPS: every rank updates `nodes` nodes `steps` times; the job takes the slowest
    rank's time (milliseconds)."""
    return world * nodes * steps / (t_ms_max * 1e3)


def _traffic(prof, form, tile):
    """DRAM bytes per launch of the step kernel of this form and tile candidate, if captured."""
    v = prof.get(f"{form}_step_dram_bytes_by_tile", {}).get(str(tile))
    if v is None and prof.get(f"{form}_step_tile_candidate") == tile:
        v = prof.get(f"{form}_step_dram_bytes_per_launch")
    return v


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap,utilization.gpu")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.5)  # nvidia-smi start-up
            self.n_before = len(self.samples)
        except Exception:
            self.proc = None
        return self

    n_before = 0

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.n_after = len(self.samples)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        # keep the samples taken while the timed loops ran
        self.samples = self.samples[self.n_before:getattr(self, "n_after", len(self.samples))]
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(s[0]) for s in self.samples if num(s[0]) is not None]
        util = [num(s[7]) or 0.0 for s in self.samples]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            for k, n in enumerate(names):
                if s[3 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(self.samples[0][1]),
                "reasons": sorted(reasons), "samples_in_timed_region": len(self.samples),
                "max_util": max(util) if util else None}


def flush_l2(flush):
    """Write one buffer larger than L2, then read another (see the module docstring)."""
    flush[0].fill_(1)
    flush[1].max()  # a reduction that reads the whole buffer (no widened copy)


def time_form(w, precision, steps, warmup, flush, tile=-1):
    """Per-step CUDA-event timing of the fused step on the Lattice's stream, L2 flushed before each step."""
    import torch

    from paper_2109_12565_gb300 import lb

    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, mask=w.mask, precision=precision)
    if tile < 0:
        # the timed steps start with L2 flushed, so the candidates are timed the same way
        tile, cand_ms = g.autotune(launches=30, scratch=flush[0])
    else:
        g.set_tile(tile)
        cand_ms = []
    shape = g.tile_info(tile)
    s = g.stream
    with torch.cuda.stream(s):
        for _ in range(warmup):
            flush_l2(flush)
            g.step(1)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush_l2(flush)
            ev[k][0].record(s)
            g.step(1)
            ev[k][1].record(s)
        torch.cuda.synchronize()
    times = [a.elapsed_time(b) for a, b in ev]
    obs = g.observables()
    g.close()
    return {"ms_total": sum(times), "ms_per_step": sum(times) / steps, "ms_min": min(times),
            "ms_median": statistics.median(times), "obs": obs,
            "tile": {"candidate": tile, "tx": shape["tx"], "ty": shape["ty"], "threads": shape["threads"]},
            "autotune_ms_per_candidate": [round(m, 5) for m in cand_ms]}


def time_batch(reps, steps, warmup, trial_steps=16):
    """The ensemble in one lb_batch: autotune (schedule x tile; those steps are real steps), W warm-up
    steps, then K steps timed with CUDA events on the batch's stream (inputs >> L2, no flush)."""
    import torch

    from paper_2109_12565_gb300 import lb

    b = lb.Batch([w.params for w in reps], [w.rho1 for w in reps], [w.rho2 for w in reps], [w.T0 for w in reps],
                 masks=[w.mask for w in reps], precision=lb.LB_FP32_SHIFTED)
    tune = b.autotune(trial_steps=trial_steps)
    b.step(warmup)
    assert b.sync() == 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.step(steps)
    e1.record(b.stream)
    torch.cuda.synchronize()
    rc = b.sync()
    ms = e0.elapsed_time(e1)
    nodes = sum(w.params["nx"] * w.params["ny"] for w in reps)
    info = b.info()
    obs0 = b.observables(0)
    b.close()
    assert rc == 0
    return {"ms_total": ms, "ms_per_step": ms / steps, "nodes": nodes, "info": info, "tune": tune,
            "Nu_replica0": obs0["Nu"]}


def time_adjoint(w, precision, n_steps, fwd_steps=200):
    """Adjoint cost on workload w: mean forward step (CUDA events, K back-to-back single steps) against
    the reverse-step time and the whole lb_adjoint (forward with Nu, recompute, reverse) per step."""
    import torch

    from paper_2109_12565_gb300 import lb

    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, mask=w.mask, precision=precision)
    g.autotune(launches=5)
    g.step(10)
    s = g.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s):
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(fwd_steps):
            g.step(1)
        e1.record(s)
        torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / fwd_steps
    t0 = time.perf_counter()
    J, gT0, gTd = g.adjoint(n_steps)
    wall = time.perf_counter() - t0
    tm = lb.Lattice.adjoint_timing()
    g.close()
    rev_ms = tm["reverse_ms"] / tm["adjoint_steps"]
    total_ms = tm["forward_ms"] + tm["recompute_ms"] + tm["reverse_ms"]
    return {"forward_step_ms": fwd_ms, "adjoint_step_ms": rev_ms, "adjoint_over_forward": rev_ms / fwd_ms,
            "gradient_total_ms": total_ms, "gradient_wall_s": wall,
            "amortised_over_forward": total_ms / (n_steps * fwd_ms), "n_steps": n_steps,
            "checkpoints": max(1, round(n_steps ** 0.5)), "J": J, "dJ_dTdown": gTd,
            "phases_ms": {k: tm[k] for k in ("forward_ms", "recompute_ms", "reverse_ms")}}


def time_e2e(w, precision, steps, obs_every=500):
    """End to end through the C ABI: lb_init from pinned host fields, `steps` steps (graph replays),
    observables every `obs_every` steps and at the end, fields back to pinned host memory."""
    import numpy as np
    import torch

    from paper_2109_12565_gb300 import lb

    N = w.params["nx"] * w.params["ny"]
    host_in = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory() for a in
               (w.rho1, w.rho2, w.T0)]
    arrays = [t.numpy() for t in host_in]
    out = torch.empty((5, w.params["ny"], w.params["nx"]), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = lb.Lattice(w.params, arrays[0], arrays[1], arrays[2], mask=w.mask, precision=precision)
    done, n_obs = 0, 0
    while done < steps:
        n = min(obs_every, steps - done)
        g.step(n)
        done += n
        g.observables()
        n_obs += 1
    o = out.numpy()
    import ctypes
    dp = [o[k].ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for k in range(5)]
    rc = lb.lib().lb_get_fields(g._h, *dp)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    assert rc == 0
    g.close()
    h2d = 3 * N * 8 + (N if w.mask is not None else 0)
    d2h = n_obs * 16 * 8 + 5 * N * 8
    return {"value": N * steps / (t1 - t0) / 1e6, "unit": "MLUPS", "seconds": t1 - t0,
            "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps, "steps": steps,
            "observables_every": obs_every}


def cpu_baseline(w, seconds=12.0, min_steps=2):
    """The FP64 oracle as it stands (OpenMP build, all host cores) on the same workload."""
    import oracle as O

    cores = O.available_cores()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    o = O.Oracle(w.params, w.rho1, w.rho2, w.T0, mask=w.mask, omp=True)
    o.step(1)
    n, t0 = 0, time.perf_counter()
    while n < min_steps or time.perf_counter() - t0 < seconds:
        o.step(1)
        n += 1
    dt = time.perf_counter() - t0
    N = w.params["nx"] * w.params["ny"]
    # the single-threaded build of the same oracle, a shorter sample
    o1 = O.Oracle(w.params, w.rho1, w.rho2, w.T0, mask=w.mask, omp=False)
    n1, t1 = 0, time.perf_counter()
    while n1 < 1 or time.perf_counter() - t1 < seconds / 4:
        o1.step(1)
        n1 += 1
    dt1 = time.perf_counter() - t1
    return {"value": N * n / dt / 1e6, "unit": "MLUPS", "cores": int(os.environ["OMP_NUM_THREADS"]),
            "kind": "oracle", "sample": f"{n} full steps of the {w.name} lattice after 1 untimed step "
                                        f"({dt:.1f} s, FP64 C oracle, OpenMP over rows)",
            "single_thread": {"value": N * n1 / dt1 / 1e6, "unit": "MLUPS", "cores": 1,
                              "sample": f"{n1} full steps ({dt1:.1f} s, same oracle, single-threaded build)"}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2109_12565_gb300 import inputs as I
    import oracle as O

    w = I.emulsion_1024x512()
    cores = O.available_cores()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    o = O.Oracle(w.params, w.rho1, w.rho2, w.T0, omp=True)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    N = w.params["nx"] * w.params["ny"]
    v = N * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "nx": 1024, "ny": 512, "n_drops": 350,
                                             "phi": 0.8, "Ra": 3.6e4},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": int(os.environ["OMP_NUM_THREADS"]),
                             "kind": "oracle",
                             "sample": f"{args.steps} full steps of {w.name} after {args.warmup} warm-up steps"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def time_droplets(w, I, lb, reps=5):
    """Wall time of one droplet analysis (lb_droplets: labels, centres, digital Voronoi, links; a
    synchronous call) on the 1024 x 512 emulsion and the 4096 x 2048 rough channel, median of reps
    after one warm-up call."""
    import torch

    out = {}
    for name, ww, prec in (("emulsion_1024x512", w, lb.LB_FP32_SHIFTED),
                           ("rough_channel_4096x2048", I.rough_channel_4096x2048(), lb.LB_FP32_SHIFTED)):
        g = lb.Lattice(ww.params, ww.rho1, ww.rho2, ww.T0, mask=ww.mask, precision=prec)
        g.step(20)
        res = g.droplets(0.8, arrays=False)
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = g.droplets(0.8, arrays=False)
            ts.append((time.perf_counter() - t0) * 1e3)
        out[name] = {"ms": statistics.median(ts), "n_drops": res["n"], "n_links": res["n_links"]}
        g.close()
        del res
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=2000)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--forms", default="fp32,fp64,df64,fp16t,batched,adjoint,rough,droplets",
                    help="comma list of fp32, fp64, df64, fp16t, batched, adjoint, rough, droplets")
    ap.add_argument("--rough-steps", type=int, default=200, help="timed steps of the 4096 x 2048 rough channel")
    ap.add_argument("--fp64-steps", type=int, default=0, help="timed FP64 steps (default steps // 4)")
    ap.add_argument("--tile", type=int, default=-1,
                    help="fixed tile candidate (index within the precision's own list) instead of autotuning")
    ap.add_argument("--batch-steps", type=int, default=200, help="timed steps of the 64-replica ensemble")
    ap.add_argument("--adjoint-steps", type=int, default=2000, help="N of the adjoint gradient (512 x 256)")
    ap.add_argument("--detail", default=DETAIL_DEFAULT,
                    help="file for the per-candidate autotuner timings and other detail kept off the JSON line")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_2109_12565_gb300 import build as B
    from paper_2109_12565_gb300 import inputs as I
    from paper_2109_12565_gb300 import lb

    B.build()
    w = I.emulsion_1024x512()
    N = w.params["nx"] * w.params["ny"]
    flush = (torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda"),
             torch.ones(FLUSH_BYTES, dtype=torch.uint8, device="cuda"))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    forms_req = set(args.forms.split(","))
    ens = I.ensemble() if "batched" in forms_req else None
    steps64 = args.fp64_steps or max(3, args.steps // 4)
    r32 = r64 = None
    with ClockSampler(local) as clk:
        if "fp32" in forms_req:
            r32 = time_form(w, lb.LB_FP32_SHIFTED, args.steps, args.warmup, flush, args.tile)
        if "fp64" in forms_req:
            r64 = time_form(w, lb.LB_FP64, steps64, args.warmup, flush, args.tile)
        rdf = time_form(w, lb.LB_DF64, steps64, args.warmup, flush, args.tile) if "df64" in forms_req else None
        r16 = time_form(w, lb.LB_FP32_FP16T, args.steps, args.warmup, flush, args.tile) if "fp16t" in forms_req else None
        rb = time_batch(ens, args.batch_steps, args.warmup) if ens else None
        wr = I.rough_channel_4096x2048() if "rough" in forms_req else None
        rr = time_form(wr, lb.LB_FP32_SHIFTED, args.rough_steps, args.warmup, flush, args.tile) if wr else None
    rdrop = time_droplets(w, I, lb) if "droplets" in forms_req else None
    radj = None
    if "adjoint" in forms_req:
        wa = I.emulsion_512x256()
        radj = {"fp64": time_adjoint(wa, lb.LB_FP64, args.adjoint_steps),
                "fp32_shifted": time_adjoint(wa, lb.LB_FP32_SHIFTED, args.adjoint_steps)}
    torch.cuda.synchronize()
    e2e = time_e2e(w, lb.LB_FP32_SHIFTED, args.e2e_steps) if args.e2e_steps > 0 else None
    # every rank's timed totals, max over ranks, before rank 0 alone goes on to report
    t32, t64, t16, trr, tb, te2e, tdf = max_over_ranks(
        [r32["ms_total"] if r32 else 0.0, r64["ms_total"] if r64 else 0.0, r16["ms_total"] if r16 else 0.0,
         rr["ms_total"] if rr else 0.0, rb["ms_total"] if rb else 0.0, e2e["seconds"] if e2e else 0.0,
         rdf["ms_total"] if rdf else 0.0],
        dist, "cuda")
    mlups32 = aggregate_mlups(world, N, args.steps, t32) if r32 else None
    mlups64 = aggregate_mlups(world, N, steps64, t64) if r64 else None
    if e2e:
        e2e["value"] = aggregate_mlups(world, N, args.e2e_steps, te2e * 1e3)
    if rank != 0:
        dist.destroy_process_group()
        return 0
    peak, peak_kind = _peaks()
    prof = _profile_counters()
    bytes32, bytes64 = 216.0 * N, 432.0 * N  # 27 populations read + written per node
    forms, detail = {}, {}

    def tile_of(r):
        t = r["tile"]
        return f'{t["tx"]}x{t["ty"]}/{t["threads"]}#{t["candidate"]}'

    roof = None
    if r32:
        ach32 = bytes32 / (r32["ms_per_step"] * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach32, "peak": peak, "unit": "GB/s", "frac": ach32 / peak,
                "traffic": _traffic(prof, "fp32", r32["tile"]["candidate"]), "peak_source": peak_kind,
                "kernel": "lb_step_kernel<float, shifted> (fused step)", "algorithmic_bytes_per_launch": bytes32}
        forms["fp32_shifted"] = {"MLUPS": mlups32, "ms_per_step": r32["ms_per_step"], "hbm_frac": ach32 / peak,
                                 "Nu": r32["obs"]["Nu"], "tile": tile_of(r32)}
        detail["fp32_autotune_ms_per_candidate"] = r32["autotune_ms_per_candidate"]
    if r16:
        ach16 = 180.0 * N / (r16["ms_per_step"] * 1e-3) / 1e9  # 18 FP32 + 9 FP16 values read + written
        forms["fp32_fp16_thermal"] = {"MLUPS": aggregate_mlups(world, N, args.steps, t16),
                                      "hbm_frac": ach16 / peak, "bytes_per_update": 180,
                                      "traffic": _traffic(prof, "fp16t", r16["tile"]["candidate"]),
                                      "Nu": r16["obs"]["Nu"], "tile": tile_of(r16)}
        detail["fp16t_autotune_ms_per_candidate"] = r16["autotune_ms_per_candidate"]
    if rr:
        Nr = wr.params["nx"] * wr.params["ny"]
        achr = 216.0 * Nr / (rr["ms_per_step"] * 1e-3) / 1e9
        forms["rough_4096x2048"] = {"MLUPS": aggregate_mlups(world, Nr, args.rough_steps, trr),
                                    "hbm_frac": achr / peak,
                                    "traffic": _traffic(prof, "rough_channel_fp32", rr["tile"]["candidate"]),
                                    "tile": tile_of(rr)}
        detail["rough_autotune_ms_per_candidate"] = rr["autotune_ms_per_candidate"]
    if rb:
        achb = 216.0 * rb["nodes"] / (rb["ms_per_step"] * 1e-3) / 1e9
        forms["batched"] = {"MLUPS": aggregate_mlups(world, rb["nodes"], args.batch_steps, tb), "replicas": len(ens),
                            "nodes": rb["nodes"], "hbm_frac": achb / peak,
                            "schedule": ["per-step graph", "persistent"][rb["info"]["schedule"]],
                            "tile": rb["info"]["tile"]}
        detail["batched"] = {"autotune_ms_per_step": rb["tune"]["ms_per_step"], "info": rb["info"],
                             "Nu_replica0": rb["Nu_replica0"], "ms_per_step": rb["ms_per_step"]}
    if radj:
        forms["adjoint_512x256"] = {k: {"rev_over_fwd": v["adjoint_step_ms"] / v["forward_step_ms"],
                                        "grad_over_fwd_run": v["amortised_over_forward"],
                                        "fwd_step_ms": v["forward_step_ms"]} for k, v in radj.items()}
        detail["adjoint"] = radj
    if rdrop:
        step_ms = r32["ms_per_step"] if r32 else None
        forms["droplets_ms"] = {k: v["ms"] for k, v in rdrop.items()}
        if step_ms:
            forms["droplets_ms"]["fp32_steps_1024x512"] = rdrop["emulsion_1024x512"]["ms"] / step_ms
        detail["droplets"] = rdrop
    if rdf:
        # double-float storage and arithmetic on the FP32 pipe, held to the FP64 tolerance of the oracle
        achdf = bytes64 / (rdf["ms_per_step"] * 1e-3) / 1e9
        forms["df64"] = {"MLUPS": aggregate_mlups(world, N, steps64, tdf), "ms_per_step": rdf["ms_per_step"],
                         "hbm_frac": achdf / peak, "bytes_per_update": 432, "Nu": rdf["obs"]["Nu"],
                         "tile": tile_of(rdf)}
        if r64:
            forms["df64"]["over_fp64"] = forms["df64"]["MLUPS"] / mlups64
        detail["df64_autotune_ms_per_candidate"] = rdf["autotune_ms_per_candidate"]
    if r64:
        # the paper's arithmetic: FP64 storage and FP64 arithmetic; bound by the FP64 pipe, not by HBM
        ach64 = bytes64 / (r64["ms_per_step"] * 1e-3) / 1e9
        f64 = {"MLUPS": mlups64, "ms_per_step": r64["ms_per_step"], "hbm_frac": ach64 / peak,
               "Nu": r64["obs"]["Nu"], "tile": tile_of(r64)}
        dp = prof.get("fp64_dp_flops_per_node")
        pk = fp64_peak_tflops()
        if dp:
            ach_tf = dp * N / (r64["ms_per_step"] * 1e-3) / 1e12
            f64["roofline"] = {"bound": "alu", "achieved": ach_tf, "peak": pk, "unit": "TFLOP/s",
                               "frac": ach_tf / pk, "flops_per_node": dp,
                               "peak_source": "152 SMs x 2 DFMA/clk x 2 flop x sm_max_mhz"}
        else:
            f64["roofline"] = {"bound": "alu", "achieved": None, "peak": pk, "unit": "TFLOP/s", "frac": None,
                               "flops_per_node": None, "note": "no ncu FP64 instruction count for these kernels"}
        f64["hbm"] = {"achieved": ach64, "peak": peak, "unit": "GB/s", "frac": ach64 / peak,
                      "traffic": _traffic(prof, "fp64", r64["tile"]["candidate"])}
        if r32:
            f64["fp32_over_fp64"] = mlups32 / mlups64
        detail["fp64_autotune_ms_per_candidate"] = r64["autotune_ms_per_candidate"]
        forms["fp64"] = f64  # last key of the line: it survives a truncated tail
    head = r32 or r64 or {"ms_per_step": None}
    line = {
        "metric": METRIC, "value": mlups32 if r32 else mlups64, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps if r32 else steps64, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32" if r32 else "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "nx": 1024, "ny": 512, "n_drops": 350, "phi": 0.8, "Ra": 3.6e4,
                   "form": "fp32_shifted" if r32 else "fp64",
                   "l2": "flushed before every timed step (512 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": (args.steps if r32 else 0) + (steps64 if r64 else 0) + (steps64 if rdf else 0) + (
            args.steps if r16 else 0) + (
            args.rough_steps if rr else 0) + (
            (args.batch_steps if rb["info"]["schedule"] == 0 else -(-args.batch_steps // 64)) if rb else 0),
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        cb = cpu_baseline(w, seconds=args.cpu_seconds)
        detail["cpu_single_thread"] = cb.pop("single_thread")
        line["cpu_baseline"] = cb
    line["forms"] = forms
    line = rnd(line)
    if args.detail:
        try:
            os.makedirs(os.path.dirname(os.path.abspath(args.detail)), exist_ok=True)
            with open(args.detail, "w") as fh:
                json.dump(rnd(detail, 6), fh, indent=1)
        except OSError:
            pass
    print(json.dumps(line, separators=(",", ":")), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
