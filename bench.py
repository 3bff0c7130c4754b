"""Benchmark of the particle push on GB300 (one JSON line on rank 0).

Workload (default): the learned-guess curved channel -- 64^3 curved hexahedra
(NGeo = 3) of [0,2pi]x[-1,1]x[0,pi], N = 5 on Gauss nodes, synthetic channel
turbulence, 10^7 particles, Schiller-Naumann drag, dt = 1e-3; FP32 push: FP32
interpolation, drag and RK update, the final Newton iterations in double-float
(FP32 pairs) to |dxi| < 1e-12, FP64 face intersection where FP32 cannot decide
the crossing.
A bench step is one pt_push call advancing every particle by --inner time
steps (one element re-binning, then --inner x 5 RK stages).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs its own particles on its own GPU (weak
scaling, no data-path collective); value = all ranks' particle-steps / max
rank time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s"
# bounded oracle sample (particles, time steps) of the cpu_baseline leg and of
# every step of --impl reference: about 10 s of work on a 16-core host
REF_SAMPLE = (100_000, 2)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--inner", type=int, default=10, help="time steps per pt_push call")
    ap.add_argument("--particles", type=int, default=10_000_000)
    ap.add_argument("--dims", type=int, default=64)
    ap.add_argument("--guess", default="auto", choices=["auto", "trilinear", "mlp"])
    ap.add_argument("--schedule", default="auto", choices=["auto", "resident", "staged"],
                    help="pt_push kernel schedule (results do not depend on it)")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e / fp64 / cpu legs")
    ap.add_argument("--extras", default="trilinear,reference,coupled,e2e,fp64,cpu",
                    help="comma list of extra legs to run (trilinear, reference, coupled, e2e, "
                         "fp64, cpu)")
    ap.add_argument("--config", default="c3", choices=["c1", "c2", "c3", "c4", "c5"],
                    help="c3 (default): the learned-start 64^3 channel; c1: 8^3 TGV box FP64; "
                         "c2: 32^3 NGeo=2 channel FP64; c4: 128 batched boxes FP32; "
                         "c5: 128x64x64 N=7 two-way channel FP32 with deposition")
    ap.add_argument("--shard", action="store_true",
                    help="c4 on several GPUs: split the same 128 boxes over the ranks by cost "
                         "(strong scaling) instead of giving every rank its own 128 (weak)")
    return ap.parse_args()


def reduce_time_ms(ms: float, world: int, device=None) -> float:
    """Max of the per-rank timed-region durations (every rank waits for the slowest)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device=None) -> float:
    """Sum of a per-rank value over all ranks (the particles they advanced)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard_by_cost(costs, world: int):
    """Greedy longest-processing-time split of independent units over ranks:
    units in decreasing cost (lower index first on ties) go to the least
    loaded rank (lowest rank on ties).  Returns one sorted index list per rank;
    the largest load exceeds the smallest by at most one unit's cost."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(o) for o in out]


def throughput(particles_per_rank: int, inner: int, steps: int, world: int, ms: float) -> float:
    """Whole-job particle-steps/s: every rank advances its own particles."""
    return particles_per_rank * inner * steps * world / (ms / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def inputs_vs_l2(P, wl):
    """The particle record and the fluid field against the 129 MB L2."""
    part_b = P * (3 * 8 + 3 * 4 + 4 + 3 * 4)
    field_b = wl.mesh.nelem * 5 * (wl.N + 1) ** 3 * 4
    rel = "larger" if part_b + field_b > 129e6 else "SMALLER"
    return f"inputs {rel} than L2 (particles {part_b / 1e9:.2f} GB, field {field_b / 1e9:.2f} GB)"


def make_workload(args, device, seed, precision):
    from paper_2211_05458_gb300 import workloads as W
    return W.curved_channel((args.dims,) * 3, 3, 5, P=args.particles, nsteps=args.inner,
                            seed=seed, device=device, precision=precision)


# DRAM bytes per particle-stage of the stage kernel k_stage_f32 (learned start),
# from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum of one
# launch on the 32^3, 10^6-particle channel, divided by its 10^6 particles;
# profiles/); the traffic is per particle, so it scales with the particles of
# a launch.  None while the kernel differs from the captured one.
TRAFFIC_BYTES_PER_PARTICLE_STAGE = (235.257088e6 + 48.194816e6) / 1e6


def algorithmic_flops_per_particle_stage(G=4, NP=6, ntri=2, it_full=2.0, it_resid=2.0):
    """Flops of one particle-stage as the method prescribes them (a multiply-add
    is 2 flops whatever precision or emulation carries it out): the trilinear
    start; it_full Newton iterations that evaluate chi and J (the FP32
    iterations of the FP32 mode, every iteration of the FP64 mode) and it_resid
    iterations that need the residual only (the final iterations of the FP32
    mode), each sum-factorised, ntri of the 3 coordinates in 8-corner trilinear
    form; interpolation of 4 variables; drag, RK update and the 6 slab tests.
    The double-float emulation and the learned start are not counted."""
    full = 3 - ntri
    basis_d = 3 * 6 * G                                   # product-form values + derivatives
    basis = 3 * 4 * G
    map_j = full * 2 * (2 * G ** 3 + 3 * G ** 2 + 4 * G) + ntri * 64
    map_v = full * 2 * (G ** 3 + G ** 2 + G) + ntri * 32
    newton_full = basis_d + map_j + 74                    # + 3x3 inverse, product, update
    newton_resid = basis + map_v + 24
    interp = 3 * 5 * NP + 4 * 2 * (NP ** 3 + NP ** 2 + NP)
    misc = 30 + 30 + 24 + 48                              # start, drag, RK, slabs
    return int(round(it_full * newton_full + it_resid * newton_resid + interp + misc))


def fp32_peak_tflops(clk_max_mhz=2070.0, sms=152, lanes=128):
    """FP32 FMA rate from the unit counts and the maximum clock (context only;
    the roofline uses the measured rate)."""
    return sms * lanes * 2 * clk_max_mhz * 1e6 / 1e12


def alu_peaks(stream):
    """Measured FP32 and FP64 FMA throughput (TFLOP/s) of this GPU from libpt's
    probe kernels, with the SM count read from the device."""
    import torch

    from paper_2211_05458_gb300 import pt
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return {"fp32": pt.measure_peak(0, stream), "fp64": pt.measure_peak(1, stream), "sms": sms}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class OracleSample:
    """The oracle (as it stands) on a bounded sample of the same workload;
    threads run disjoint particle chunks on one oracle context (ctypes
    releases the GIL during each call)."""

    def __init__(self, wl, max_threads=None):
        import numpy as np

        from tests import helpers as H
        self.orc = H.make_oracle(wl)
        self.x, self.v = H.np64(wl.x), H.np64(wl.v)
        self.d, self.el = H.np64(wl.d), H.np64(wl.elem).astype(np.int32)
        self.prm = H.oracle_params(wl)
        self.dt = wl.dt
        self.threads = max_threads or (os.cpu_count() or 1)
        self.rng = np.random.default_rng(123)

    def run(self, sample_particles, sample_steps):
        import numpy as np
        idx = np.sort(self.rng.choice(self.x.shape[0], size=sample_particles, replace=False))
        chunks = np.array_split(idx, self.threads)
        args = [(self.x[c], self.v[c], self.d[c], self.el[c]) for c in chunks]
        t0 = time.perf_counter()

        def work(a):
            self.orc.push(self.prm, *a, nsteps=sample_steps, dt=self.dt)
        ths = [threading.Thread(target=work, args=(a,)) for a in args]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        dt = time.perf_counter() - t0
        return sample_particles * sample_steps / dt, self.threads, dt


def fp64_peak_tflops(clk_max_mhz=2070.0, sms=152, dfma_per_clk=2):
    return sms * dfma_per_clk * 2 * clk_max_mhz * 1e6 / 1e12


def config_workloads(cfg, dev, seed, shard=None):
    """The workloads other than the default one (seeded, synthetic).  shard =
    (rank, world): the 128 batched boxes (c4) split over the ranks by cost
    P (N+1)^3, every rank drawing the same boxes."""
    from paper_2211_05458_gb300 import workloads as W
    if cfg == "c4" and shard is not None:
        rank, world = shard
        prm = W.batched_box_params(nbox=128, seed=1)
        mine = shard_by_cost([P * (N + 1) ** 3 for _, N, P in prm], world)[rank]
        return W.batched_boxes(nbox=128, seed=1, device=dev, nsteps=50, select=mine)
    if cfg == "c1":
        return [W.tgv_box(8, 3, P=10_000, nsteps=100, seed=seed, device=dev)]
    if cfg == "c2":
        return [W.curved_channel((32, 32, 32), 2, 5, P=1_000_000, nsteps=200, seed=seed,
                                 device=dev)]
    if cfg == "c4":
        return W.batched_boxes(nbox=128, seed=1 + seed, device=dev, nsteps=50)
    if cfg == "c5":
        return [W.curved_channel((128, 64, 64), 2, 7, P=20_000_000, nsteps=50, seed=seed,
                                 device=dev, mass_loading=0.3)]
    raise ValueError(cfg)


def run_config(args):
    """--config c1|c2|c4|c5: one JSON line for that workload (same schema)."""
    import torch
    import torch.distributed as dist

    from paper_2211_05458_gb300 import pt
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    cfg = args.config
    sharded = cfg == "c4" and args.shard and world > 1
    wls = config_workloads(cfg, dev, rank, shard=(rank, world) if sharded else None)
    f64 = cfg in ("c1", "c2")
    prec = pt.FP64 if f64 else pt.FP32
    dt_ = torch.float64 if f64 else torch.float32
    ctxs, parts = [], []
    sched = {"auto": pt.SCHEDULE_AUTO, "resident": pt.SCHEDULE_RESIDENT,
             "staged": pt.SCHEDULE_STAGED}[args.schedule]
    for wl in wls:
        c = pt.Context(wl.mesh, stream=stream, precision=prec, mu=wl.mu, rho_p=wl.rho_p,
                       drag_law=wl.drag_law, rebin_every=args.inner, schedule=sched)
        c.set_fluid(wl.N, wl.node_type, wl.U.to(dt_).contiguous())
        ctxs.append(c)
        parts.append(pt.ParticleSet.create(wl.x, wl.v, wl.d, wl.elem, prec, dev))
    P = sum(p.n for p in parts)
    dt = wls[0].dt
    inner = 50 if cfg == "c4" else args.inner
    S = None
    if cfg == "c5":
        n3 = (wls[0].N + 1) ** 3
        S = torch.empty((wls[0].mesh.nelem, 4, n3), dtype=torch.float32, device=dev)
    dep_ev = []

    def step():
        if cfg == "c4":
            pt.push_batch(ctxs, parts, inner, dt, stats=False)
        else:
            ctxs[0].push(parts[0], inner, dt, stats=False)
        if S is not None:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctxs[0].deposit(parts[0], pt.DEPOSIT_SEGMENTED, S)
            e1.record(stream)
            dep_ev.append((e0, e1))

    warm = max(args.warmup, 3)  # the batched push tunes, then captures its graph
    for _ in range(warm):
        step()
    torch.cuda.synchronize()
    dep_ev.clear()
    for c in ctxs:
        c.launch_count()  # clear
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ms = reduce_time_ms(ev0.elapsed_time(ev1), world, dev)
    launches = sum(c.launch_count() for c in ctxs)
    peaks_alu = alu_peaks(stream)
    P_all = sum_over_ranks(P, world, dev)  # ranks may hold different particle counts (c4)
    value = P_all * inner * args.steps / (ms / 1e3)
    wl0 = wls[0]
    G, NP = wl0.mesh.ngeo + 1, wl0.N + 1
    # measured Newton iterations per particle-stage, from one more step with counters
    if cfg == "c4":
        sts = pt.push_batch(ctxs, parts, 1, dt, stats=True)
        st = {k: sum(x[k] for x in sts) for k in ("particle_steps", "newton_it_fp32",
                                                    "newton_it_fp64")}
    else:
        st = ctxs[0].push(parts[0], 1, dt, stats=True)
    nps = max(st["particle_steps"], 1) * 5
    it32, it64 = st["newton_it_fp32"] / nps, st["newton_it_fp64"] / nps
    if f64:
        flops = algorithmic_flops_per_particle_stage(G=G, NP=NP, ntri=3 if G == 2 else 2,
                                                     it_full=it64, it_resid=0.0)
    else:
        flops = algorithmic_flops_per_particle_stage(G=G, NP=NP, ntri=3 if G == 2 else 2,
                                                     it_full=it32, it_resid=it64)
    if f64:
        # FP64 mode: the same operation count in FP64, against the FP64 rate
        peak = peaks_alu["fp64"]
        peak_kind = "measured: libpt FP64 FMA probe (pt_measure_peak)"
    else:
        peak = peaks_alu["fp32"]
        peak_kind = "measured: libpt FP32 FMA probe (pt_measure_peak)"
    achieved = flops * 5 * value / world / 1e12
    names = {"c1": "TGV box 8^3 NGeo=1 N=3 Gauss, 10^4 particles, Stokes, FP64",
             "c2": "curved channel 32^3 NGeo=2 N=5 Gauss, 10^6 particles, Schiller-Naumann, FP64",
             "c4": f"128 periodic TGV boxes (sides 8..40, N 3..7, {int(P_all)} particles"
                   + (" split over the GPUs by cost" if sharded else "") + "), FP32, "
                   "graph of 50 steps",
             "c5": "two-way channel 128x64x64 NGeo=2 N=7, 2x10^7 particles, FP32, push of "
                   f"{inner} steps + segmented deposition"}
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": warm, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "strong" if sharded else "weak",
            "vs_baseline": None,
            "dtype": "f64" if f64 else "f32", "data": "synthetic",
            "config": {"workload": names[cfg], "inner_steps_per_call": inner,
                       "schedule": args.schedule,
                       "parallelism": (f"{world} GPU(s), boxes split by cost P (N+1)^3"
                                       if sharded else f"weak, {world} independent GPU(s)")},
            "gpu_launches": launches, "clocks": clk.summary(),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "whole step",
                         "peak_kind": peak_kind, "flops_per_particle_stage": flops,
                         "newton_iterations_per_stage": {"full": it64 if f64 else it32,
                                                         "residual_only": 0.0 if f64 else it64}}}
    if cfg == "c4":
        line["batch_tuning"] = pt.batch_tuning(ctxs[0])
    if dep_ev:
        dep_ms = sum(a.elapsed_time(b) for a, b in dep_ev) / len(dep_ev)
        Sbytes = S.numel() * 4
        line["deposit"] = {"ms": dep_ms, "share_of_step": dep_ms / (ms / args.steps),
                           "S_bytes": Sbytes, "S_write_gbs": Sbytes / (dep_ms / 1e3) / 1e9}
    if rank == 0 and not args.no_extras:
        try:
            samp = {"c1": (2000, 5), "c2": (2000, 2), "c4": (2000, 2), "c5": (2000, 1)}[cfg]
            wl_s = max(wls, key=lambda w: w.x.shape[0]) if cfg == "c4" else wl0
            wl_s.U = wl_s.U.cpu()
            wl_s.x, wl_s.v, wl_s.d, wl_s.elem = (wl_s.x.cpu(), wl_s.v.cpu(), wl_s.d.cpu(),
                                                 wl_s.elem.cpu())
            n_s = min(samp[0], wl_s.x.shape[0])
            rate, threads, _ = OracleSample(wl_s).run(n_s, samp[1])
            rate1, _, _ = OracleSample(wl_s, max_threads=1).run(max(n_s // 8, 1), samp[1])
            line["cpu_baseline"] = {"value": rate, "unit": METRIC, "cores": threads,
                                    "kind": "oracle", "single_thread": rate1,
                                    "sample": f"{n_s} particles x {samp[1]} time steps"
                                              + (" of the largest box" if cfg == "c4" else "")}
        except Exception as e:  # pragma: no cover
            line["cpu_baseline"] = {"unavailable": str(e)[:200]}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, same workload/metric."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import torch
    wl = make_workload(args, "cuda" if torch.cuda.is_available() else "cpu", 0, "fp64")
    wl.U = wl.U.cpu()
    wl.x, wl.v, wl.d, wl.elem = wl.x.cpu(), wl.v.cpu(), wl.d.cpu(), wl.elem.cpu()
    sample, ssteps = REF_SAMPLE
    times = []
    osmp = OracleSample(wl)
    warm = args.warmup
    for i in range(warm + args.steps):
        rate, threads, dt = osmp.run(sample, ssteps)
        if i >= warm:
            times.append(dt)
    tot = sum(times)
    value = sample * ssteps * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"curved channel {args.dims}^3 NGeo=3 N=5, "
                       f"{args.particles} particles, Schiller-Naumann, dt=1e-3",
                       "inputs_vs_l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": threads, "kind": "oracle",
                             "sample": f"{sample} particles x {ssteps} time steps per bench "
                                       "step (the cpu_baseline sample of the default run)"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.config != "c3":
        return run_config(args)
    import torch
    import torch.distributed as dist

    from paper_2211_05458_gb300 import pt
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks, peak_kind = measured_peaks()

    wl = make_workload(args, dev, seed=rank, precision="fp32")
    stream = torch.cuda.current_stream()
    guess = pt.GUESS_TRILINEAR
    sched = {"auto": pt.SCHEDULE_AUTO, "resident": pt.SCHEDULE_RESIDENT,
             "staged": pt.SCHEDULE_STAGED}[args.schedule]
    ctx = pt.Context(wl.mesh, stream=stream, precision=pt.FP32, mu=wl.mu, rho_p=wl.rho_p,
                     drag_law=wl.drag_law, rebin_every=args.inner, schedule=sched)
    mlp_info = None
    if args.guess in ("auto", "mlp"):
        try:
            t0 = time.perf_counter()
            inp, tgt = ctx.mlp_make_pairs(2_000_000, seed=1000 + rank)
            losses = ctx.mlp_train(inp, tgt, epochs=20, batch=4096, lr=1e-3, seed=rank)
            torch.cuda.synchronize()
            mlp_info = {"train_s": time.perf_counter() - t0, "final_loss": losses[-1]}
            guess = pt.GUESS_MLP
            del inp, tgt
        except pt.PtError as e:
            if args.guess == "mlp":
                raise
            mlp_info = {"unavailable": str(e)[:200]}
    ctx.set_config(guess=guess)
    U32 = wl.U.to(torch.float32).contiguous()
    ctx.set_fluid(wl.N, wl.node_type, U32)
    parts = pt.ParticleSet.create(wl.x, wl.v, wl.d, wl.elem, pt.FP32, dev)
    P = parts.n

    def step():
        ctx.push(parts, args.inner, wl.dt, stats=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.profile_read()  # clear
    ctx.launch_count()  # clear
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ms = ev0.elapsed_time(ev1)
    # device time per kernel kind from libpt's own events on its stream:
    # 0 push chunks (the resident kernel, or a staged chunk incl. its copies),
    # 1 stage kernels, 2 learned-start kernels, 3 exact-tracking kernels
    kinds = {k: ctx.profile_read_kind(k) for k in (1, 2, 3)}
    kern_ms, launches = ctx.profile_read()
    gpu_launches = ctx.launch_count()
    ctx.profile(False)
    peaks_alu = alu_peaks(stream)
    ms = reduce_time_ms(ms, world, dev)
    value = throughput(P, args.inner, args.steps, world, ms)
    stats = ctx.push(parts, 1, wl.dt, stats=True)  # one more step with counters
    hist = ctx.histograms()
    staged = kinds[1][1] > 0

    # roofline of the dominant kernel: the stage kernel of the staged schedule
    # (one RK stage of every particle per launch), else the resident push (a
    # whole chunk of steps per launch).  It is bound by FP32 arithmetic and
    # issue latency, not by memory.
    nps = max(stats["particle_steps"], 1) * 5
    it32, it64 = stats["newton_it_fp32"] / nps, stats["newton_it_fp64"] / nps
    # iterations per stage as the stage kernel runs them (the totals also
    # hold the walk's inverse maps after a crossing)
    h_it32 = sum(k * c for k, c in enumerate(hist["newton_fp32"])) / max(sum(hist["newton_fp32"]), 1)
    h_it64 = sum(k * c for k, c in enumerate(hist["newton_final"])) / max(sum(hist["newton_final"]), 1)
    if staged:
        it32, it64 = h_it32, h_it64
    flops_stage = algorithmic_flops_per_particle_stage(G=4, NP=wl.N + 1, ntri=2, it_full=it32,
                                                       it_resid=it64)
    if staged:
        kname = "k_stage_f32<G=4,NP=6,%s>" % ("learned start" if guess else "trilinear start")
        k_ms, k_n = kinds[1]
        flops_launch = flops_stage * P
    else:
        kname = "k_push<4,6,fp32,%s>" % ("learned" if guess else "trilinear")
        k_ms, k_n = kern_ms, launches
        flops_launch = flops_stage * 5 * args.inner * P
    avg_launch_s = (k_ms / 1e3) / max(k_n, 1)
    achieved = flops_launch / avg_launch_s / 1e12
    fp32_peak = peaks_alu["fp32"]
    # DRAM bytes per particle-stage of the stage kernel from one ncu capture
    # of the same kernel on the 32^3, 10^6-particle channel (profiles/)
    traffic = (TRAFFIC_BYTES_PER_PARTICLE_STAGE * P
               if (staged and TRAFFIC_BYTES_PER_PARTICLE_STAGE) else None)
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak,
                "traffic": traffic,
                "kernel": kname,
                "peak_kind": "measured: libpt FP32 FMA probe (pt_measure_peak), "
                             f"{peaks_alu['sms']} SMs; from unit counts: "
                             f"{fp32_peak_tflops(sms=peaks_alu['sms']):.1f}",
                "fp64_peak_measured": peaks_alu["fp64"],
                "flops_per_particle_stage": flops_stage,
                "newton_iterations_per_stage": {"full": it32, "residual_only": it64},
                "launch_ms": avg_launch_s * 1e3,
                "kernel_share_of_step": (k_ms / ms) if ms > 0 else None,
                "hbm_gbs_from_traffic": (traffic / avg_launch_s / 1e9 if traffic else None),
                "hbm_frac_of_measured": (traffic / avg_launch_s / 1e9 /
                                         float(peaks.get("hbm_gbs", 6800.0)) if traffic else None),
                "other_kernels_ms_per_launch": {
                    "learned_start": kinds[2][0] / max(kinds[2][1], 1) if kinds[2][1] else None,
                    "exact_tracking": kinds[3][0] / max(kinds[3][1], 1) if kinds[3][1] else None},
                "share_of_step": {"stage": kinds[1][0] / ms, "learned_start": kinds[2][0] / ms,
                                  "exact_tracking": kinds[3][0] / ms} if staged else None}
    if guess:
        # the learned start's own products run on the tensor cores (BF16, FP32
        # accumulate): 3x64 + 2 x 64x64 + 64x3 multiply-adds per particle-stage
        mlp_flops = 2 * (3 * 64 + 2 * 64 * 64 + 64 * 3)
        if staged and kinds[2][1]:
            t_s = kinds[2][0] / 1e3 / kinds[2][1]
            t_ach = mlp_flops * P / t_s / 1e12
            t_kern = "k_guess_tc (tcgen05, one RK stage of every particle per launch)"
        else:
            t_ach = mlp_flops * 5 * args.inner * P / avg_launch_s / 1e12
            t_kern = "inside k_push (mma.sync)"
        roofline["mlp_tensor"] = {"kernel": t_kern, "flops_per_particle_stage": mlp_flops,
                                  "achieved": t_ach,
                                  "peak": float(peaks.get("bf16_tflops", 1900.0)),
                                  "unit": "TFLOP/s", "peak_kind": peak_kind + " (cuBLAS bf16)",
                                  "frac": t_ach / float(peaks.get("bf16_tflops", 1900.0))}

    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"curved channel {args.dims}^3 NGeo=3 N=5 Gauss, "
                       f"{P} particles/GPU, Schiller-Naumann, dt=1e-3; FP32 interpolation, "
                       "drag and RK; double-float final Newton to |dxi| < 1e-12; FP64 "
                       "intersection where FP32 is ambiguous",
                       "inner_steps_per_call": args.inner, "guess": "mlp" if guess else "trilinear",
                       "schedule": "staged (one kernel per RK stage)" if staged else
                                   "resident (one kernel per call chunk)",
                       "inputs_vs_l2": inputs_vs_l2(P, wl),
                       "parallelism": f"weak, {world} independent GPU(s)"},
            "gpu_launches": gpu_launches, "clocks": clk.summary(), "roofline": roofline,
            "stats_one_step": {k: stats[k] for k in ("particle_steps", "crossings", "wall_hits",
                                                     "newton_it_fp32", "newton_it_fp64",
                                                     "slow_track", "near_face", "near_wall")},
            "histograms_one_step": hist}
    if mlp_info:
        line["mlp"] = mlp_info

    if not args.no_extras and rank == 0:
        # the same FP32 push with the trilinear Newton start (no learned correction)
        legs = set(args.extras.split(","))
        if guess == pt.GUESS_MLP and "trilinear" in legs:
            ctx.set_config(guess=pt.GUESS_TRILINEAR)
            ptri = pt.ParticleSet.create(wl.x, wl.v, wl.d, wl.elem, pt.FP32, dev)
            ctx.push(ptri, args.inner, wl.dt, stats=False)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                ctx.push(ptri, args.inner, wl.dt, stats=False)
            e1.record(stream)
            torch.cuda.synchronize()
            line["fp32_trilinear"] = {"value": P * args.inner * 3 / (e0.elapsed_time(e1) / 1e3),
                                      "unit": METRIC,
                                      "note": "same FP32 push, trilinear Newton start"}
            ctx.set_config(guess=guess)
            del ptri
        if "reference" in legs:
            # reference-space localisation (Sec. 3.2.3): only walls intersected;
            # same start guess as the headline; owners compared with the
            # physical tracking of the same particles after the same steps
            pref = pt.ParticleSet.create(wl.x, wl.v, wl.d, wl.elem, pt.FP32, dev)
            pphy = pt.ParticleSet.create(wl.x, wl.v, wl.d, wl.elem, pt.FP32, dev)
            ctx.push(pphy, args.inner, wl.dt, stats=False)
            ctx.set_config(track=pt.TRACK_REFERENCE)
            ctx.push(pref, args.inner, wl.dt, stats=False)
            torch.cuda.synchronize()
            same = float((pref.elem == pphy.elem).float().mean())
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                ctx.push(pref, args.inner, wl.dt, stats=False)
            e1.record(stream)
            torch.cuda.synchronize()
            line["fp32_reference_tracking"] = {
                "value": P * args.inner * 3 / (e0.elapsed_time(e1) / 1e3), "unit": METRIC,
                "same_owner_as_physical": same,
                "note": "same FP32 push, owners found by inverse map + face walk (walls traced)"}
            ctx.set_config(track=pt.TRACK_PHYSICAL)
            del pref, pphy
    if not args.no_extras and rank == 0 and "coupled" in legs:
        # a coupled solver that updates the fluid state every time step calls
        # pt_push with nsteps = 1: binning, sorted copy and copy back per step
        pc = pt.ParticleSet.create(wl.x, wl.v, wl.d, wl.elem, pt.FP32, dev)
        ctx.push(pc, 1, wl.dt, stats=False)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(10):
            ctx.push(pc, 1, wl.dt, stats=False)
        e1.record(stream)
        torch.cuda.synchronize()
        line["coupled_one_step_calls"] = {
            "value": P * 10 / (e0.elapsed_time(e1) / 1e3), "unit": METRIC,
            "note": "same push, pt_push(nsteps = 1) per time step (fluid state updated by the "
                    "caller between calls); the default run uses 10 steps per call"}
        # a solver that advances fluid and particles stage by stage together
        e0.record(stream)
        for _ in range(10):
            for s_ in range(5):
                ctx.push_stage(pc, s_, wl.dt)
        e1.record(stream)
        torch.cuda.synchronize()
        line["coupled_per_stage_calls"] = {
            "value": P * 10 / (e0.elapsed_time(e1) / 1e3), "unit": METRIC,
            "note": "same push, pt_push_stage(0..4) per time step (fluid state updated by the "
                    "caller between RK stages)"}
        del pc
    if not args.no_extras and rank == 0 and "e2e" in legs:
        # e2e: same metric through pt_push_host with pinned host buffers
        hp = parts.to("cpu", pin=True)
        e2e_steps = max(1, min(3, args.steps))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ctx.push_host(hp, args.inner, wl.dt, stats=False)
        e2e_s = time.perf_counter() - t0
        h2d = P * (24 + 12 + 4 + 12)
        d2h = P * (24 + 12 + 12)
        line["e2e"] = {"value": P * args.inner * e2e_steps / e2e_s, "unit": METRIC,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        del hp
    if not args.no_extras and rank == 0 and "fp64" in legs:
        # plain FP64 Newton (FP64 mode) on the same workload, fewer steps
        ctx64 = pt.Context(wl.mesh, stream=stream, precision=pt.FP64, mu=wl.mu, rho_p=wl.rho_p,
                           drag_law=wl.drag_law, rebin_every=2)
        U64 = wl.U.to(torch.float64).contiguous()
        ctx64.set_fluid(wl.N, wl.node_type, U64)
        p64 = pt.ParticleSet.create(wl.x, wl.v, wl.d, wl.elem, pt.FP64, dev)
        ctx64.push(p64, 1, wl.dt, stats=False)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx64.push(p64, 2, wl.dt, stats=False)
        e1.record(stream)
        torch.cuda.synchronize()
        line["plain_fp64"] = {"value": P * 2 / (e0.elapsed_time(e1) / 1e3), "unit": METRIC,
                              "note": "FP64 mode: FP64 Newton from the trilinear guess, FP64 "
                                      "interpolation, drag and RK"}
        del p64, U64, ctx64
    if not args.no_extras and rank == 0 and "cpu" in legs:
        # oracle on the host cores, bounded sample
        try:
            wl.U = wl.U.cpu()
            wl.x, wl.v, wl.d, wl.elem = wl.x.cpu(), wl.v.cpu(), wl.d.cpu(), wl.elem.cpu()
            osamp = OracleSample(wl)
            rate, threads, dt = osamp.run(REF_SAMPLE[0], REF_SAMPLE[1])
            osamp.threads = 1
            rate1, _, _ = osamp.run(2000, 2)
            line["cpu_baseline"] = {"value": rate, "unit": METRIC, "cores": threads,
                                    "kind": "oracle", "single_thread": rate1,
                                    "sample": f"{REF_SAMPLE[0]} particles x {REF_SAMPLE[1]} time "
                                              "steps of the same workload (single thread: "
                                              "2000 x 2)"}
            # per-result error of the FP32 arithmetic against the FP64 oracle
            # (first-stage terms of 2000 sampled particles with a slip velocity)
            from tests import helpers as H
            err = H.stage_term_errors(wl, ctx, osamp.orc, 2000, seed=0)
            line["precision_split_error"] = {
                "xi_abs": err["xi"], "rho_rhou_rel": err["U"], "accel_rel": err["acc"],
                "dx_rel": err["dx"], "dv_rel": err["dv"],
                "note": "max over 2000 sampled (x, element) of the first RK stage, FP32 mode "
                        "vs the FP64 oracle at its own xi; rel = normwise per component"}
        except Exception as e:  # pragma: no cover
            line["cpu_baseline"] = {"unavailable": str(e)[:200]}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
