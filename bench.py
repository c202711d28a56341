"""Throughput of the OS-MPM hot path on GB300.

Default line (no --workload): one step = one global Schwarz step (Alg. 1) of
every pair of the batched inclusion family (256 instances of uneven size:
inclusion radius, modulus and fine resolution 0.01 / 0.005 from SplitMix64;
coarse grid [0,1]^2 at dx 0.05, fine grid [0.3,0.7]^2, M = 2, top edge
displaced 1e-3 per step) in mixed precision, advanced by
osmpm_schwarz_couple_multi: host threads drive the pairs and one batched
PCG service solves every Newton system.  Beside it, ``fp64_single_instance``
times the FP64 single inclusion (fine dx 0.005, M = 2) with CUDA events.
Metric: particle-substeps/s (fine particles count M per global step,
coarse particles 1; Schwarz re-iterations are overhead).

The batched line is timed on the host clock around each batched step with
the device synchronised on both sides (the pairs run on their own streams);
the single-instance line with CUDA events on its stream, the L2 flushed
(a 256 MiB write) between steps.  End-to-end numbers time the public-API
sequence a user runs per step: upload every domain's particle state from
pinned host memory, the step, download the state.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload default|inclusion|batched|fold3d|fold3d_solve]

``--impl reference`` times the FP64 CPU oracle (the reference arm of this
repository: a plain NumPy/SciPy restatement of the method) on the host cores.
"""
from __future__ import annotations

import os

# The oracle legs are timed single-threaded (BLAS and OpenMP pools pinned to
# one thread before NumPy loads); the CPU baseline reports cores = 1.
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import dataclasses
import json
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2605_09097_gb300 import workloads as W  # noqa: E402

METRIC = "OS-MPM particle-substeps/s at fixed error vs FP64 oracle; % HBM peak"
UNIT = "particle-substeps/s"
DX_S, M_SUB = 0.005, 2
WORKLOAD = "inclusion_osmpm_2d_fp64_dxB0.05_dxS0.005_M2"
# Schwarz iterations of one global step of this workload, averaged over the
# first three global steps of an FP64 oracle run (used to scale the oracle's
# bounded sample, which runs a fixed number of Schwarz iterations).
ORACLE_SCHWARZ_ITERS_PER_STEP = 12.0
ORACLE_SAMPLE_ITERS = 2
L2_FLUSH_BYTES = 256 << 20
AUTOTUNE_THREADS = [8, 12, 16]
# (host threads, DOFs per DOF tile, PCG iterations per graph replay, slot
# tiles per work item of the batched product)
AUTOTUNE_MULTI = [(128, 2048, 16, 1), (128, 2048, 16, 2), (128, 2048, 16, 4)]
# dram__bytes_read.sum + dram__bytes_write.sum of one fine-domain k_pcg
# launch, from the ncu capture of the current kernel (the k_pcg profile
# summary of this workload); None whenever the kernel changes
PCG_TRAFFIC_BYTES = 3.05e6 + 0.06e6
# FP64 flops of one Hessian-vector product per particle: gather G (2 d^2 3^d),
# Y = L G (2 d^4), G:Y (2 d^2), scatter (2 d^2 3^d); an FMA counts 2.
HVP_FLOPS_PER_PARTICLE = {2: 184, 3: 1152}


def workload():
    return W.inclusion(dx_S=DX_S, M=M_SUB)


def units_per_step(cB, cS, M):
    return cB.particles.n + M * cS.particles.n


# ----------------------------------------------------------------------------
# distributed plumbing (independent replicas, one per GPU)
# ----------------------------------------------------------------------------
def dist_init(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if _cuda_ok() else "gloo"
        dist.init_process_group(backend=backend)
    return rank, local, world


def _cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if _cuda_ok() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if _cuda_ok() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.proc = None
        self.path = None
        self.index = index

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        lines = open(self.path).read().splitlines()
        os.unlink(self.path)
        return parse_clock_rows(lines)


def parse_clock_rows(lines):
    """Summary of the sampler's CSV rows (the QUERY fields, no header, no
    units): median and maximum SM clock, and every throttle reason seen
    active during the samples; None without a complete row."""
    rows = []
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) >= 9:
            rows.append(parts)
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    reasons = set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        for k, name in enumerate(names):
            if r[5 + k].lower().startswith("active"):
                reasons.add(name)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(mx) if mx else None,
            "reasons": sorted(reasons), "samples": len(rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def run_ours(args, rank, local, world):
    import torch
    torch.cuda.set_device(local)
    from paper_2605_09097_gb300 import build
    build.build()
    from paper_2605_09097_gb300 import osmpm

    cB, cS, sch, dT = workload()
    cB = dataclasses.replace(cB, launch_mode=args.launch_mode)
    cS = dataclasses.replace(cS, launch_mode=args.launch_mode)
    units = units_per_step(cB, cS, sch.M)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        B = osmpm.Domain(cB, stream=stream.cuda_stream)
        S = osmpm.Domain(cS, stream=stream.cuda_stream)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        for _ in range(args.warmup):
            osmpm.osmpm_schwarz_couple(B, S, dT, sch)
        torch.cuda.synchronize()
        B.set_profiling(True)
        S.set_profiling(True)
        stats = []
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        clocks = ClockSampler(local)
        barrier(world)
        torch.cuda.synchronize()
        launches0 = osmpm.launch_count()
        clocks.start()
        t_wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            stats.append(osmpm.osmpm_schwarz_couple(B, S, dT, sch))
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
        clk = clocks.stop()
        launches = osmpm.launch_count() - launches0 - 0
        barrier(world)
        ms = sum(a.elapsed_time(b) for a, b in ev)
        ms_max = max_over_ranks(ms, world)
        cB_ = B.counters()
        cS_ = S.counters()
        B.set_profiling(False)
        S.set_profiling(False)
        adj = adjoint_cost(osmpm, stream) if rank == 0 else None

        # end to end through the public API with host buffers
        e2e = None
        if args.e2e_steps > 0:
            xs = [d.get_particles() for d in (B, S)]
            pinned = []
            for arrs in xs:
                pa = []
                for a in arrs:
                    t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
                    t.numpy()[...] = a
                    pa.append(t.numpy())
                pinned.append(pa)
            h2d = sum(a.nbytes for pa in pinned for a in pa)
            barrier(world)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.e2e_steps):
                B.set_particles(*pinned[0])
                S.set_particles(*pinned[1])
                osmpm.osmpm_schwarz_couple(B, S, dT, sch)
                for d, pa in zip((B, S), pinned):
                    x, v, Bm, F = d.get_particles()
                    pa[0][...] = x
                    pa[1][...] = v
                    pa[2][...] = Bm
                    pa[3][...] = F
            torch.cuda.synchronize()
            te = max_over_ranks(time.perf_counter() - t0, world)
            e2e = {"value": sum_over_ranks(units * args.e2e_steps, world) / te, "unit": UNIT,
                   "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
                   "steps": args.e2e_steps}

    value = sum_over_ranks(units * args.steps, world) / (ms_max / 1e3)
    # roofline of the dominant kernel, the persistent PCG (one launch per
    # Newton iteration): FP64 ALU bound; algorithmic flops = PCG iterations x
    # particles x HVP flops (the vector updates are not counted)
    pcg_ms = cB_["pcg_ms"] + cS_["pcg_ms"]
    pcg_n = cB_["pcg_launches"] + cS_["pcg_launches"]
    flops = (cB_["pcg_iters"] * cB_["particles"] + cS_["pcg_iters"] * cS_["particles"]) \
        * HVP_FLOPS_PER_PARTICLE[2]
    achieved = flops / (pcg_ms / 1e3) / 1e9 if pcg_ms > 0 else 0.0
    fp64_peak = 1250.0  # GFLOP/s, nominal GB300 FP64 (non-tensor)
    iters = [s["schwarz_iters"] for s in stats]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "particles_coarse": cB.particles.n,
                   "particles_fine": cS.particles.n, "M": sch.M, "dT": dT,
                   "units_per_step": units, "parallelism": f"replicas{world}",
                   "l2": "flushed between steps (256 MiB write, outside the timed events)",
                   "launch": ("CUDA graph per Newton iteration" if args.launch_mode == 0
                              else "plain stream launches"),
                   "schwarz_iters_per_step": iters,
                   "newton_iters_per_step": [s["newton_iters"] for s in stats],
                   "cg_iters_per_step": [s["cg_iters"] for s in stats],
                   "wall_ms_per_step": 1e3 * t_wall / args.steps},
        "gpu_launches": int(launches),
        "roofline": {"kernel": "k_pcg (persistent PCG)", "bound": "alu", "achieved": achieved,
                     "peak": fp64_peak, "unit": "GFLOP/s", "frac": achieved / fp64_peak,
                     "traffic": PCG_TRAFFIC_BYTES,
                     "traffic_source": ("ncu, one fine-domain launch (dram read + write bytes)"
                                        if PCG_TRAFFIC_BYTES is not None
                                        else "not captured for the current kernel"),
                     "peak_source": "nominal FP64 1.25 TFLOP/s (GB300)",
                     "launches": pcg_n, "avg_launch_us": 1e3 * pcg_ms / max(pcg_n, 1),
                     "pcg_iters": cB_["pcg_iters"] + cS_["pcg_iters"],
                     "us_per_pcg_iter": 1e3 * pcg_ms / max(cB_["pcg_iters"] + cS_["pcg_iters"], 1),
                     "flops_per_particle_iter": HVP_FLOPS_PER_PARTICLE[2]},
        "clocks": clk,
        "e2e": e2e,
        "adjoint": adj,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(ORACLE_SAMPLE_ITERS)
    return out


ADJ_STEPS, ADJ_DT = 20, 1e-3


def adjoint_cost(osmpm, stream):
    """Reverse-mode cost per forward step on the single-domain cantilever
    (2560 particles, FP64): CUDA-event times of ADJ_STEPS plain steps, of the
    same steps while recording, and of one osmpm_adjoint over the record
    (J = mean tip deflection)."""
    import torch
    spec = W.cantilever()
    x0 = spec.particles.x
    tip = x0[:, 0] > 0.98
    c = np.zeros_like(x0)
    c[tip, 1] = -1.0 / tip.sum()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b), r

    def steps(dom):
        for _ in range(ADJ_STEPS):
            dom.step(ADJ_DT)

    plain = osmpm.Domain(spec, stream=stream.cuda_stream)
    ms_plain, _ = timed(lambda: steps(plain))
    rec = osmpm.Domain(spec, stream=stream.cuda_stream)
    rec.record(True)
    ms_rec, _ = timed(lambda: steps(rec))
    g = torch.from_numpy(c).cuda()
    ms_adj, (_, _, st) = timed(lambda: rec.adjoint(g))
    rec.record(False)
    return {"workload": f"cantilever_2d_fp64 ({x0.shape[0]} particles), {ADJ_STEPS} steps of "
                        f"{ADJ_DT:g} s, J = mean tip deflection",
            "forward_ms_per_step": ms_plain / ADJ_STEPS,
            "recording_ms_per_step": ms_rec / ADJ_STEPS,
            "adjoint_ms_per_step": ms_adj / ADJ_STEPS,
            "adjoint_over_forward": ms_adj / ms_plain,
            "adjoint_cg_iters": st["cg_iters"]}


# ----------------------------------------------------------------------------
# the oracle on the host cores
# ----------------------------------------------------------------------------
def oracle_sample(n_iters):
    """Times the FP64 oracle on the bench workload: the first ``n_iters``
    Schwarz iterations of global step 1.  Returns (seconds, units), units
    scaled by n_iters / ORACLE_SCHWARZ_ITERS_PER_STEP."""
    from oracle import osmpm_oracle as O
    cB, cS, sch, dT = workload()
    sch = dataclasses.replace(sch, k_max=n_iters - 1)
    B, S = O.DomainState.create(cB), O.DomainState.create(cS)
    t0 = time.perf_counter()
    O.schwarz_step(B, S, dT, sch)
    t = time.perf_counter() - t0
    units = units_per_step(cB, cS, sch.M) * n_iters / ORACLE_SCHWARZ_ITERS_PER_STEP
    return t, units


def _threads():
    return int(os.environ.get("OMP_NUM_THREADS", "1"))


def cpu_baseline(n_iters):
    t, units = oracle_sample(n_iters)
    return {"value": units / t, "unit": UNIT, "cores": _threads(), "kind": "oracle",
            "sample": f"first {n_iters} Schwarz iterations of global step 1 of {WORKLOAD} "
                      f"({t:.1f} s), scaled by {n_iters}/{ORACLE_SCHWARZ_ITERS_PER_STEP:g} "
                      "of a global step's units"}


# Algorithmic bytes of one mixed-precision Hessian-vector product per
# particle (the particle state read once, the gathered
# x_hat and d and the scattered Hd once per node at 1/ppc node per
# particle): 2D x 16 + F^n 16 + V0 4 + mu lam 8 + (16 + 8 + 8)/4 = 52 B,
# 3D x 24 + F^n 36 + V0 4 + mu lam 8 + (24 + 12 + 12)/8 = 78 B
MIXED_HVP_BYTES_PER_PARTICLE = {2: 52.0, 3: 78.0}
# dram__bytes_read.sum + dram__bytes_write.sum of one launch on the
# 3.07M-particle fold band (ncu), per kernel; absent until captured for the
# current kernel
FOLD_HVP_TRAFFIC_BYTES = {"k_cgs_hvp_tile": 347.653e6 + 5.941e6}
# dram__bytes_read.sum + dram__bytes_write.sum per launch of the batched
# Hessian-vector product (k_m_hvp) on the batched family, from ncu; None
# until captured for the current kernel
MULTI_HVP_TRAFFIC_BYTES = None


def run_batched(args, rank, local, world):
    """Aggregate throughput of ``--instances`` independent inclusion pairs of
    the batched family (uneven fine resolutions), each on its own stream,
    advanced together by osmpm_schwarz_couple_multi (mixed precision: one
    batched PCG service for every pair's Newton systems; ``--batch-mode
    multi``) or osmpm_schwarz_couple_batch (each pair launching its own PCG;
    ``--batch-mode threads``).  Host wall clock around each batched step,
    the device synchronised on both sides (the pairs run on many streams)."""
    import torch
    torch.cuda.set_device(local)
    from paper_2605_09097_gb300 import build
    build.build()
    from paper_2605_09097_gb300 import osmpm
    scaled = bool(getattr(args, "scaled", False))
    specs = [W.inclusion_instance(i, scaled=scaled) for i in range(args.instances)]
    prec = 1 if args.precision == "mixed" else 0
    B, S, streams = [], [], []
    for cB, cS, sch, dT in specs:
        st = osmpm.create_stream()  # one stream per pair (torch's streams come from a pool of 32)
        streams.append(st)
        B.append(osmpm.Domain(dataclasses.replace(cB, precision=prec), stream=st))
        S.append(osmpm.Domain(dataclasses.replace(cS, precision=prec), stream=st))
    schs = [s[2] for s in specs]
    dT = specs[0][3]
    units = sum(units_per_step(s[0], s[1], s[2].M) for s in specs)
    threads, tuned = args.threads, None
    multi = args.batch_mode == "multi"
    shape = None
    tune_steps = 0
    if multi:
        if args.threads == 0:
            shape, scores = osmpm.osmpm_autotune_multi(B, S, dT, schs, AUTOTUNE_MULTI)
            tuned = {"x".join(map(str, c)): v for c, v in zip(AUTOTUNE_MULTI, scores)}
            tune_steps = len(AUTOTUNE_MULTI) + 1
        else:
            shape = (args.threads, args.dof_tile, args.chunk, args.slot_tiles)
        threads = shape[0]

        def batched_step():
            return osmpm.osmpm_schwarz_couple_multi(B, S, dT, schs, *shape)[2]
    else:
        if threads == 0:
            threads, tuned = osmpm.osmpm_autotune_batch(B, S, dT, schs, AUTOTUNE_THREADS)
            tune_steps = len(AUTOTUNE_THREADS) + 1

        def batched_step():
            osmpm.osmpm_schwarz_couple_batch(B, S, dT, schs, n_threads=threads)
            return None
    # the autotuner's steps count as warm-up steps
    for _ in range(max(args.warmup - tune_steps, 0)):
        batched_step()
    torch.cuda.synchronize()
    barrier(world)
    launches0 = osmpm.launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.perf_counter()
    service = []
    for _ in range(args.steps):
        service.append(batched_step())
    torch.cuda.synchronize()
    t = max_over_ranks(time.perf_counter() - t0, world)
    clk = clocks.stop()
    value = sum_over_ranks(units * args.steps, world) / t
    launches = int(osmpm.launch_count() - launches0)
    roofline = None
    if multi and service:
        # the dominant kernel of the PCG service: the batched Hessian-vector
        # product k_m_hvp; in every 8th chunk of iterations each launch is
        # bracketed by CUDA events on the service's stream (a sample of the
        # timed region's launches); its algorithmic bytes are the mixed HVP
        # figure per particle and iteration over the systems those launches
        # iterated
        peaks, src = measured_peaks()
        d = specs[0][0].grid.dim
        pit = sum(x["hvp_particle_iterations"] for x in service)
        bytes_ = pit * MIXED_HVP_BYTES_PER_PARTICLE[d]
        hvp_s = sum(x["hvp_ms"] for x in service) / 1e3
        nl = sum(x["hvp_launches"] for x in service)
        achieved = bytes_ / hvp_s / 1e9 if hvp_s > 0 else 0.0
        roofline = {"kernel": "k_m_hvp", "bound": "hbm", "achieved": achieved,
                    "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "traffic": MULTI_HVP_TRAFFIC_BYTES,
                    "peak_source": f"{src} hbm_gbs (MEASURED_PEAKS.json)" if src == "measured"
                    else "fallback 6.8 TB/s",
                    "launches": nl, "avg_launch_us": 1e6 * hvp_s / max(nl, 1),
                    "bytes_per_launch": bytes_ / max(nl, 1),
                    "bytes_per_particle_iteration": MIXED_HVP_BYTES_PER_PARTICLE[d],
                    "particle_iterations_timed": pit,
                    "sampling": "the product launches of every 8th chunk of 16 iterations",
                    "pcg_iterations": sum(x["iterations"] for x in service),
                    "pcg_device_ms": sum(x["device_ms"] for x in service),
                    "hvp_device_ms_timed": 1e3 * hvp_s,
                    "systems_per_composition": sum(x["instances"] for x in service)
                    / max(sum(x["batches"] for x in service), 1)}
    e2e = None
    if args.e2e_steps > 0:
        # end to end through the public API: every pair's particle state
        # uploaded from pinned host memory, the batched step, the state read
        # back, per step
        host = []
        for dd in B + S:
            arrs = []
            for a in dd.get_particles():
                tp = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
                tp.numpy()[...] = a
                arrs.append(tp.numpy())
            host.append(arrs)
        nbytes = sum(a.nbytes for h in host for a in h)
        torch.cuda.synchronize()
        te0 = time.perf_counter()
        service_e2e = []
        for _ in range(args.e2e_steps):
            for dd, h in zip(B + S, host):
                dd.set_particles(*h)
            service_e2e.append(batched_step())
            for dd, h in zip(B + S, host):
                x, v, Bm, F = dd.get_particles()
                h[0][...] = x
                h[1][...] = v
                h[2][...] = Bm
                h[3][...] = F
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - te0, world)
        e2e = {"value": sum_over_ranks(units * args.e2e_steps, world) / te, "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "steps": args.e2e_steps,
               "note": "the global steps after the timed ones (the state continues from them)"}
        if multi:
            e2e["pcg_iterations_per_step"] = [x["iterations"] for x in service_e2e if x]
    for dd in B + S:
        dd.close()
    for st in streams:
        osmpm.destroy_stream(st)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, tune_steps),
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == 0 else "f32/f64",
            "data": "synthetic",
            "config": {"workload": f"batched_inclusion_{args.instances}_"
                                   f"{'scaled' if scaled else 'literal'}_"
                                   f"{'mixed' if prec else 'fp64'}",
                       "instances": args.instances, "host_threads": threads,
                       "batch_mode": args.batch_mode, "launch_shape": shape,
                       "pcg_service": service if multi else None,
                       "pcg_iterations_per_step": [x["iterations"] for x in service] if multi
                       else None,
                       "autotune_us_per_cg_iter": tuned,
                       "particles": sum(s[0].particles.n + s[1].particles.n for s in specs),
                       "units_per_step": units, "precision": args.precision,
                       "timing": "host wall clock around each batched step, device synchronised "
                                 "on both sides (the pairs run on their own streams)",
                       "l2": "not flushed: the instances' resident state (~0.6 KB per particle, "
                             f"{sum(s[0].particles.n + s[1].particles.n for s in specs):,} "
                             "particles) is larger than L2",
                       "parallelism": f"replicas{world}"},
            "gpu_launches": launches, "roofline": roofline, "clocks": clk, "e2e": e2e}


def oracle_instance_sample(i, n_iters=ORACLE_SAMPLE_ITERS):
    """The FP64 oracle on instance i of the batched family: the first
    ``n_iters`` Schwarz iterations of global step 1.  Returns (seconds,
    units), units scaled by n_iters / ORACLE_SCHWARZ_ITERS_PER_STEP of a
    global step's particle-substeps."""
    from oracle import osmpm_oracle as O
    cB, cS, sch, dT = W.inclusion_instance(i)
    sch = dataclasses.replace(sch, k_max=n_iters - 1)
    B, S = O.DomainState.create(cB), O.DomainState.create(cS)
    t0 = time.perf_counter()
    O.schwarz_step(B, S, dT, sch)
    t = time.perf_counter() - t0
    return t, units_per_step(cB, cS, sch.M) * n_iters / ORACLE_SCHWARZ_ITERS_PER_STEP


def cpu_baseline_batched():
    """The oracle on a bounded sample of the batched family: on one core the
    first Schwarz iterations of instances 0 and 1 (one of each fine
    resolution) one after the other; on all host cores one such sample per
    core (instances 0 .. nproc-1) in a spawn-started process pool, counted
    by wall clock.  Rates in particle-substeps/s, reported only."""
    import multiprocessing as mp
    t0, u0 = oracle_instance_sample(0)
    t1, u1 = oracle_instance_sample(1)
    one = (u0 + u1) / (t0 + t1)
    cores = os.cpu_count() or 1
    out = {"value": one, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"first {ORACLE_SAMPLE_ITERS} Schwarz iterations of global step 1 of batched "
                     f"instances 0 and 1 (fine dx 0.01 and 0.005; {t0 + t1:.1f} s), units scaled "
                     f"by {ORACLE_SAMPLE_ITERS}/{ORACLE_SCHWARZ_ITERS_PER_STEP:g} of a global step"}
    try:
        ctx = mp.get_context("spawn")
        tw = time.perf_counter()
        with ctx.Pool(cores) as pool:
            res = pool.map(oracle_instance_sample, range(cores))
        wall = time.perf_counter() - tw
        out["all_cores"] = {"value": sum(u for _, u in res) / wall, "unit": UNIT, "cores": cores,
                            "sample": f"instances 0..{cores - 1}, one process each, wall clock "
                                      f"{wall:.1f} s (process start included)"}
    except Exception as e:  # the one-core figure stands alone
        out["all_cores"] = {"unavailable": str(e)[:200]}
    return out


def run_default(args, rank, local, world):
    """The headline: the batched inclusion family (256 instances of uneven
    size, mixed precision) through the
    batched PCG service, with the plain FP64 single-instance inclusion
    (fine dx 0.005, M = 2) beside it as ``fp64_single_instance``."""
    a = argparse.Namespace(**vars(args))
    a.precision, a.batch_mode, a.instances = "mixed", "multi", 256
    main_line = run_batched(a, rank, local, world)
    b = argparse.Namespace(**vars(args))
    b.steps, b.warmup, b.no_cpu_baseline = max(args.steps, 10), max(args.warmup, 3), True
    single = run_ours(b, rank, local, world)
    main_line["fp64_single_instance"] = {
        k: single[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup", "dtype", "config",
                               "roofline", "e2e", "clocks", "gpu_launches") if k in single}
    main_line["adjoint"] = single.get("adjoint")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        main_line["cpu_baseline"] = cpu_baseline_batched()
    return main_line


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle on the host cores, on the
    workload of ``--workload`` (default: the batched family; each step one
    bounded sample, the first Schwarz iteration of global step 1 of the next
    instance; inclusion: the FP64 single inclusion, same sample)."""
    if rank != 0:
        return None
    batched = args.workload in ("default", "batched")
    k = [0]

    def sample():
        if batched:
            i = k[0] % 2  # instances 0 and 1: one of each fine resolution
            k[0] += 1
            return oracle_instance_sample(i, 1)
        return oracle_sample(1)

    for _ in range(args.warmup):
        sample()
    tot_t, tot_u = 0.0, 0.0
    for _ in range(args.steps):
        t, u = sample()
        tot_t += t
        tot_u += u
    value = tot_u / tot_t
    cores = _threads()
    workload = "batched_inclusion_256_literal_mixed" if batched else WORKLOAD
    what = ("batched instances 0, 1, 0, ... (fine dx 0.01, 0.005)" if batched else WORKLOAD)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload, "parallelism": "cpu"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: the first Schwarz iteration of global step 1 of "
                                       f"{what}, scaled by 1/{ORACLE_SCHWARZ_ITERS_PER_STEP:g} "
                                       "of a global step's units"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_fold(args, rank, local, world):
    """The 3D folding plate (mixed precision): coarse plate at 0.02, fine
    hinge band at 0.005 (128k particles) or, with --scaled, a band [0.2, 0.8]
    at 0.0025 (3.07M particles), M = 4.  Times --steps coupled steps after
    --warmup with CUDA events on the domains' stream; the per-kernel HBM
    fractions of this configuration come from ncu (profiles)."""
    import torch
    torch.cuda.set_device(local)
    from paper_2605_09097_gb300 import build
    build.build()
    from paper_2605_09097_gb300 import osmpm
    kw = dict(dx_f=0.0025, band=(0.2, 0.8)) if args.scaled else {}
    cB, cS, sch, dT = W.fold3d(**kw)
    units = cB.particles.n + sch.M * cS.particles.n
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        B = osmpm.Domain(cB, stream=stream.cuda_stream)
        S = osmpm.Domain(cS, stream=stream.cuda_stream)
        for _ in range(args.warmup):
            osmpm.osmpm_schwarz_couple(B, S, dT, sch)
        torch.cuda.synchronize()
        B.set_profiling(True)
        S.set_profiling(True)
        stats, ms = [], 0.0
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            stats.append(osmpm.osmpm_schwarz_couple(B, S, dT, sch))
            b.record(stream)
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
        cS_ = S.counters()
    return {"metric": METRIC, "value": units * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "mixed",
            "data": "synthetic",
            "config": {"workload": "fold3d_mixed" + ("_scaled" if args.scaled else ""),
                       "particles_coarse": cB.particles.n, "particles_fine": cS.particles.n,
                       "M": sch.M, "dT": dT, "units_per_step": units,
                       "schwarz_iters_per_step": [s["schwarz_iters"] for s in stats],
                       "newton_iters_per_step": [s["newton_iters"] for s in stats],
                       "cg_iters_per_step": [s["cg_iters"] for s in stats],
                       "fine_us_per_pcg_iter": 1e3 * cS_["pcg_ms"] / max(cS_["pcg_iters"], 1)}}


def run_fold_solve(args, rank, local, world):
    """Single-domain implicit steps of the fine band of the scaled 3D fold
    (3.07M particles at dx 0.0025, mixed precision, streaming PCG), folded
    on its own: the nodes of its edge x = 0.2 clamped, those of its edge
    x = 0.8 turned about the fold axis (x = 0.5, z = 0.01, parallel to y) at
    the fold's rate of 90 degrees per 400 steps of 0.01 s, dt = 0.0025.  The
    configuration of the tiled Hessian-vector product.  CUDA events around
    each step on the domain's stream; the library's PCG events give the time
    per PCG iteration."""
    import torch
    torch.cuda.set_device(local)
    from paper_2605_09097_gb300 import build
    build.build()
    from paper_2605_09097_gb300 import osmpm
    cB, cS, sch, dT = W.fold3d(dx_f=0.0025, band=(0.2, 0.8))
    h = cS.grid.dx
    clamp = W.Dirichlet(lo=(-W.BIG, -W.BIG, -W.BIG), hi=(0.2 + 0.5 * h, W.BIG, W.BIG),
                        comp_mask=0b111)
    turn = dataclasses.replace(cB.dirichlet[1], lo=(0.8 - 1.5 * h, -W.BIG, -W.BIG))
    spec = dataclasses.replace(cS, dirichlet=[clamp, turn], hvp_mode=args.hvp_mode)
    dt = dT / sch.M
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        dom = osmpm.Domain(spec, stream=stream.cuda_stream)
        for _ in range(args.warmup):
            dom.step(dt)
        torch.cuda.synchronize()
        dom.set_profiling(True)
        stats, ms = [], 0.0
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            stats.append(dom.step(dt))
            b.record(stream)
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
        c = dom.counters()
    n = spec.particles.n
    peaks, src = measured_peaks()
    # the dominant kernel: the streaming PCG's Hessian-vector product (each
    # launch that iterated bracketed by CUDA events on the domain's stream);
    # algorithmic bytes per launch = particles x the 3D mixed HVP figure
    nl, hvp_s = c["hvp_launches"], c["hvp_ms"] / 1e3
    bpl = n * MIXED_HVP_BYTES_PER_PARTICLE[3]
    achieved = nl * bpl / hvp_s / 1e9 if hvp_s > 0 else 0.0
    kname = "k_cgs_hvp_tile" if args.hvp_mode != 1 else "k_cgs_hvp"
    roofline = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "traffic": FOLD_HVP_TRAFFIC_BYTES.get(kname),
                "peak_source": f"{src} hbm_gbs (MEASURED_PEAKS.json)" if src == "measured"
                else "fallback 6.8 TB/s",
                "launches": nl, "avg_launch_us": 1e6 * hvp_s / max(nl, 1), "bytes_per_launch": bpl}
    return {"metric": METRIC, "value": n * args.steps / (ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "mixed",
            "data": "synthetic",
            "config": {"workload": "fold3d_scaled_fine_band_single_domain_mixed", "particles": n,
                       "hvp_mode": args.hvp_mode, "dt": dt,
                       "newton_iters_per_step": [s["newton_iters"] for s in stats],
                       "cg_iters_per_step": [s["cg_iters"] for s in stats],
                       "us_per_pcg_iter": 1e3 * c["pcg_ms"] / max(c["pcg_iters"], 1)},
            "roofline": roofline}


def hertz_profile(p, xc, F, R=0.5, E1=1e7, E2=1e6, nu=0.3):
    """Contact half-width and peak pressure of a measured pressure profile
    p(x) (bins centred at xc, contact centre x = 2) by a least-squares fit of
    the semi-ellipse p0 sqrt(1 - ((x - 2)/b)^2), beside the Hertz closed form
    for a cylinder on a half-space in plane strain at the measured line load
    F: E* = 1/((1 - nu^2)/E1 + (1 - nu^2)/E2), b = 2 sqrt(F R/(pi E*)),
    p_max = 2F/(pi b)."""
    Es = 1.0 / ((1 - nu ** 2) / E1 + (1 - nu ** 2) / E2)
    b_h = 2.0 * np.sqrt(F * R / (np.pi * Es))
    best = (np.inf, 0.0, 0.0)
    for b in np.linspace(0.3, 3.0, 271) * b_h:
        shape = np.sqrt(np.clip(1.0 - ((xc - 2.0) / b) ** 2, 0.0, None))
        den = float(shape @ shape)
        if den <= 0.0:
            continue
        p0 = float(shape @ p) / den
        res = float(np.sum((p - p0 * shape) ** 2))
        if res < best[0]:
            best = (res, b, p0)
    return {"F_N_per_m": F, "b_fit": best[1], "b_hertz": b_h, "p_max_fit": best[2],
            "p_max_hertz": 2.0 * F / (np.pi * b_h)}


def run_hertz(args, rank, local, world):
    """The elastic Hertz contact configuration (elastic
    cylinder R 0.5, E 1e7, pressed 0.02 into an elastic block E 1e6 over 100
    global steps of 2e-4 s, fine box at dx 1/256, M = 4, mixed precision),
    run whole; every 10 steps the contact pressure on the block's top layer
    of fine particles (their initial y within one cell below the surface),
    from the Cauchy stress of each particle's F, binned at the fine spacing,
    against the Hertz closed form at the measured line load.  A validation
    study, not a throughput line."""
    import torch
    torch.cuda.set_device(local)
    from paper_2605_09097_gb300 import build
    build.build()
    from paper_2605_09097_gb300 import osmpm
    cB, cS, sch, dT = W.hertz()
    B, S = osmpm.Domain(cB), osmpm.Domain(cS)
    dx = cS.grid.dx
    x0 = cS.particles.x
    top = (cS.particles.E < 5e6) & (x0[:, 1] < 2.0) & (x0[:, 1] >= 2.0 - dx)
    E, nu = cS.particles.E[top], cS.particles.nu[top]
    mu, lam = E / (2 * (1 + nu)), E * nu / ((1 + nu) * (1 - 2 * nu))
    edges = np.arange(1.75, 2.25 + 1e-12, dx)
    xc = 0.5 * (edges[1:] + edges[:-1])
    rows, t0 = [], time.perf_counter()
    for k in range(1, 101):
        osmpm.osmpm_schwarz_couple(B, S, dT, sch)
        if k % 10:
            continue
        x, _, _, F = S.get_particles()
        Ft = F[top]
        J = np.linalg.det(Ft)
        FFt = np.einsum("pij,pkj->pik", Ft, Ft)
        sig = (mu[:, None, None] * (FFt - np.eye(2)) +
               (lam * np.log(J))[:, None, None] * np.eye(2)) / J[:, None, None]
        idx = np.digitize(x[top, 0], edges) - 1
        p = np.array([-sig[idx == i, 1, 1].mean() if np.any(idx == i) else 0.0
                      for i in range(len(xc))])
        load = float(np.sum(np.clip(p, 0.0, None)) * dx)
        rows.append({"step": k, **hertz_profile(np.clip(p, 0.0, None), xc, load)})
    wall = time.perf_counter() - t0
    return {"workload": "hertz_contact_cylinder_on_block_mixed", "study": "contact pressure vs Hertz",
            "particles": cB.particles.n + cS.particles.n, "steps": 100, "wall_s": wall,
            "profiles": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--launch-mode", type=int, choices=[0, 1], default=0,
                    help="0: each Newton iteration replays a captured CUDA graph; 1: plain launches")
    ap.add_argument("--hvp-mode", type=int, choices=[0, 1, 2], default=0,
                    help="fold3d_solve: Hessian-vector product of the streaming PCG")
    ap.add_argument("--workload", choices=["default", "inclusion", "batched", "fold3d",
                                           "fold3d_solve", "hertz"],
                    default="default",
                    help="default: the batched family in mixed precision with the FP64 single "
                         "inclusion beside it; inclusion: the FP64 single inclusion alone; batched: "
                         "many instances; fold3d: the 3D folding plate (mixed); fold3d_solve: the "
                         "fold's 3.07M-particle band folded on its own; hertz: the contact "
                         "configuration's pressure against the Hertz closed form (a study)")
    ap.add_argument("--scaled", action="store_true",
                    help="fold3d: the 3.07M-particle band; batched: the scaled family (fine dx "
                         "0.0025 / 0.001, 45k / 283k fine particles per instance)")
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--threads", type=int, default=0,
                    help="host threads of the batched workload; 0: chosen by the autotuner")
    ap.add_argument("--dof-tile", type=int, default=0,
                    help="batched multi with --threads > 0: DOFs per DOF tile (0: default)")
    ap.add_argument("--chunk", type=int, default=0,
                    help="batched multi with --threads > 0: iterations per graph replay")
    ap.add_argument("--slot-tiles", type=int, default=0,
                    help="batched multi with --threads > 0: slot tiles per product work item")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--batch-mode", choices=["threads", "multi"], default="threads",
                    help="batched: per-pair PCG launches from a host thread pool, or the "
                         "batched PCG service (mixed precision)")
    args = ap.parse_args()
    rank, local, world = dist_init(args.gpus)
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.workload == "default":
        out = run_default(args, rank, local, world)
    elif args.workload == "batched":
        out = run_batched(args, rank, local, world)
    elif args.workload == "fold3d":
        out = run_fold(args, rank, local, world)
    elif args.workload == "fold3d_solve":
        out = run_fold_solve(args, rank, local, world)
    elif args.workload == "hertz":
        out = run_hertz(args, rank, local, world)
    else:
        out = run_ours(args, rank, local, world)
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
