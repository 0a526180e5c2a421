#!/usr/bin/env python
"""Throughput of the MLSVD-compressed damped Gauss-Newton CPD on one GB300.

Default workload (one step = one whole CPD through the C ABI): the largest
single-GPU configuration, a 100x100x100x100 FP32 tensor (400 MB) of rank 15
with Gaussian factors and relative noise 1e-5 (synthetic, seeded),
compressed by ST-MLSVD to a <= 15^4 core (the first-mode Gram on BF16 tensor
cores, --gram fp32 for CUDA cores), dGN on the core from the random start
(seed 0; the MLSVD-energy start stalls on this problem in the method itself),
uncompression, FP32 refinement iterations on T, output normalisation.
--workload compressed200 runs the 200^3 rank-10 configuration (collinearity
0.5, noise 1e-4, MLSVD-energy start) instead, and --workload full400 dGN
without compression on a 400^3 rank-10 tensor (256 MB), every iteration one
pass over T.  Metric: CPDs per second, with the fit of every result checked
against the FP64 oracle's (within 1e-6).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU runs (torchrun) give every rank its own CPD (independent problems,
no collective): weak scaling, value = all ranks' CPDs / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "CPDs/sec to fit err <= 1e-6 vs FP64 oracle"
UNIT = "CPD/s"
REFINE_MAXITER = 20


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return dict(hbm=float(d["hbm_gbs"]), bf16=float(d["bf16_tflops"]),
                    bf16_sus=float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                    sm_max_mhz=float(d.get("sm_max_mhz", 2070.0)), src="measured (MEASURED_PEAKS.json)")
    return dict(hbm=6800.0, bf16=1900.0, bf16_sus=1700.0, sm_max_mhz=2070.0, src="fallback")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms (the timed
    region of the default run is ~0.1 s)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.t:
                self.t.join(timeout=2)

    def summary(self):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return dict(sm_mhz=(statistics.median(mhz) if mhz else None), sm_max_mhz=mx,
                    reasons=sorted(reasons), samples=len(mhz))


# single-tensor workloads: generator, solver options, name
WORKLOADS = {
    "order4": dict(gen=synth.c3_order4, opts=dict(init="random", seed=0),
                   name="mlsvd_dgn_100x100x100x100_r15_noise1e-5_random_start"),
    "compressed200": dict(gen=synth.c2_compressed, opts=dict(),
                          name="mlsvd_dgn_200x200x200_r10_rho0.5_noise1e-4"),
    # dGN without compression on a large tensor: every iteration one pass over T
    "full400": dict(gen=lambda: dict(T=synth.planted(7, (400, 400, 400), 10, 0.0, 1e-5, np.float32)[0], R=10),
                    opts=dict(compress=0, init="random", seed=5, gram_precision="fp32", refine_maxiter=0),
                    name="dgn_uncompressed_400x400x400_r10_noise1e-5_random_start_seed5"),
    # the same on the 100^4 rank-15 tensor, a shape the tensor-core pass takes
    "full_order4": dict(gen=synth.c3_order4, opts=dict(compress=0, init="random", seed=0, gram_precision="fp32",
                                                       refine_maxiter=0),
                        name="dgn_uncompressed_100x100x100x100_r15_noise1e-5_random_start"),
}


def workload(name):
    w = WORKLOADS[name]
    c = w["gen"]()
    return c["T"], c["R"], w["opts"], w["name"]


def oracle_options(extra):
    import dataclasses
    import oracle as O
    o = dict(refine_maxiter=REFINE_MAXITER)
    o.update(extra)
    known = {f.name for f in dataclasses.fields(O.Options)}
    return O.Options(**{k: (bool(v) if k == "compress" else v) for k, v in o.items() if k in known})


def solve_options(cpd, args, extra):
    kw = dict(refine_maxiter=REFINE_MAXITER, gram_precision=args.gram)
    kw.update(extra)
    return cpd.cpd_default_options(**kw)


# sources whose kernels a stage times; a DRAM-traffic figure recorded in
# profiles/traffic.json is reported only while these files are unchanged
STAGE_SOURCES = {
    "dgn_core": ["k_dgn.cu", "k_dgn_cluster.cu", "dgn_cta.cuh", "solver.cuh", "common.cuh", "kernels.h"],
    "gram_bf16_tc": ["k_gram_tc.cu", "tc_common.cuh", "kernels.h"],
    "project_T": ["k_project_tc.cu", "tc_common.cuh", "kernels.h"],
    "refine_pass": ["k_refine_tc.cu", "tc_common.cuh", "k_refine_pass3.cu", "k_refine_pass4.cu", "refine_pass.cuh",
                    "solver.cuh", "common.cuh", "kernels.h"],
}


def sources_sha256(stage: str):
    import hashlib
    files = STAGE_SOURCES.get(stage)
    if not files:
        return None
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2110_05997_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(stage: str):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch from the ncu
    capture recorded in profiles/traffic.json, or None when there is none or
    the kernel's sources changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        rec = json.load(fh).get(stage)
    if not rec or rec.get("sources_sha256") != sources_sha256(stage):
        return None
    return rec["dram_bytes_per_launch"]


def algorithmic(stage: str, dims, R: int, info: dict, per_launch_ms: float, pk: dict, clk_mhz,
                gram_bf16: bool = True, sms: int = 152):
    """Roofline entry of a stage: algorithmic bytes or flops per launch over
    its measured average launch time.  The FP32 peak is derived (SM count of
    the device x 128 FMA lanes x 2 flops x the sampled SM clock), not measured."""
    N = int(np.prod(dims))
    I1 = int(dims[0])
    mhz = clk_mhz or pk["sm_max_mhz"]
    fp32_peak_tf = sms * 128 * 2 * mhz * 1e6 / 1e12          # FP32 FMA pipes, all SMs
    if stage == "refine_pass":
        nbytes = 4.0 * N + 4.0 * 2 * R * sum(dims)              # read T, read W, write G
        ach = nbytes / (per_launch_ms * 1e-3) / 1e9
        return dict(bound="hbm", achieved=ach, peak=pk["hbm"], unit="GB/s", frac=ach / pk["hbm"],
                    algorithmic_per_launch=nbytes)
    if stage == "project_T":
        # first-mode projection: read T, write the rank-P1 partial core
        P1 = int(info["core_dims"][0])
        nbytes = 4.0 * N + 4.0 * P1 * (N // I1)
        ach = nbytes / (per_launch_ms * 1e-3) / 1e9
        return dict(bound="hbm", achieved=ach, peak=pk["hbm"], unit="GB/s", frac=ach / pk["hbm"],
                    algorithmic_per_launch=nbytes, flops=2.0 * P1 * N)
    if stage == "project":
        # later-mode projections of the sequentially truncated tensor: read the
        # mode-l input, write its projection, averaged over those launches
        cd = [int(d) for d in info["core_dims"] if d > 0]
        bs = []
        for l in range(1, len(dims)):
            nin = float(np.prod(cd[:l])) * float(np.prod([int(d) for d in dims[l:]]))
            nout = float(np.prod(cd[:l + 1])) * float(np.prod([int(d) for d in dims[l + 1:]]))
            bs.append(4.0 * (nin + nout))
        nbytes = sum(bs) / len(bs)
        ach = nbytes / (per_launch_ms * 1e-3) / 1e9
        return dict(bound="hbm", achieved=ach, peak=pk["hbm"], unit="GB/s", frac=ach / pk["hbm"],
                    algorithmic_per_launch=nbytes)
    if stage == "gram_fp32":
        # the FP32 launches are the Grams of modes 2..L (and of mode 1 when it
        # is not on the tensor cores) on the sequentially truncated tensors
        # (modes < l already projected to their ranks): 2 I_l N_l flops each,
        # averaged over those launches
        cd = [int(d) for d in info["core_dims"] if d > 0]
        fls = []
        for l in range(1 if gram_bf16 else 0, len(dims)):
            Nl = float(np.prod(cd[:l])) * float(np.prod([int(d) for d in dims[l:]]))
            fls.append(2.0 * int(dims[l]) * Nl)
        fl = sum(fls) / len(fls)
        ach = fl / (per_launch_ms * 1e-3) / 1e12
        return dict(bound="alu", achieved=ach, peak=fp32_peak_tf, peak_kind="derived FP32 FMA peak", unit="TFLOP/s",
                    frac=ach / fp32_peak_tf,
                    algorithmic_per_launch=fl)
    if stage in ("gram_fp32", "gram_bf16_tc"):
        # mode-1 Gram G = T_(1) T_(1)^T: I1^2 * (N / I1) multiply-adds (2 flops each)
        fl = 2.0 * I1 * N
        if stage == "gram_bf16_tc":
            nbytes = 4.0 * N
            ach = nbytes / (per_launch_ms * 1e-3) / 1e9
            return dict(bound="hbm", achieved=ach, peak=pk["hbm"], unit="GB/s", frac=ach / pk["hbm"],
                        algorithmic_per_launch=nbytes, flops=fl)
        ach = fl / (per_launch_ms * 1e-3) / 1e12
        return dict(bound="alu", achieved=ach, peak=fp32_peak_tf, peak_kind="derived FP32 FMA peak", unit="TFLOP/s",
                    frac=ach / fp32_peak_tf,
                    algorithmic_per_launch=fl)
    if stage == "dgn_core":
        # per-iteration flop model of Sec. 4.1.3 ("Overall cost of dGN"), with
        # the measured iterations and CG iterations, on the core dims
        cd = [d for d in info["core_dims"] if d > 0]
        L = len(cd)
        Nc = float(np.prod(cd))
        sR = float(sum(cd))
        it = max(1, info["iters"])
        cg = info["cg_total"] + it          # one extra J^T J x per iteration (gain ratio)
        fl = it * ((L * R + L - 1) * Nc + L * R * Nc + R * R * (L + sR) + 3 * R * sR) * 2 \
            + cg * (9 * R + L * R * R) * sR * 2
        ach = fl / (per_launch_ms * 1e-3) / 1e12
        return dict(bound="alu", achieved=ach, peak=fp32_peak_tf, peak_kind="derived FP32 FMA peak", unit="TFLOP/s",
                    frac=ach / fp32_peak_tf,
                    algorithmic_per_launch=fl)
    ach = 0.0
    return dict(bound="latency", achieved=ach, peak=None, unit="-", frac=None)


def cpu_baseline(T, R, extra, name, ours_W=None, ours_lam=None, budget_s: float = 20.0):
    """The FP64 oracle, as it stands, on the same tensor with the same start:
    whole CPDs until the budget is spent (at least one)."""
    import oracle as O
    T64 = T.astype(np.float64)
    opts = oracle_options(extra)
    times, res = [], None
    t_all = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        res = O.cpd(T64, R, opts)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_all > budget_s or len(times) >= 50:
            break
    Wo, lo, io = res
    out = dict(value=len(times) / sum(times), unit=UNIT, cores=os.cpu_count(), kind="oracle",
               sample=f"{len(times)} whole CPDs of {name} (numpy FP64, default BLAS threads)")
    if ours_W is not None:
        fo = O.fit(T64, Wo, lo)
        fg = O.fit(T64, ours_W, ours_lam)
        c = O.compare_cpd(ours_W, ours_lam, Wo, lo)
        out["parity"] = dict(fit_gpu=fg, fit_oracle=fo, abs_diff=abs(fg - fo), ok=abs(fg - fo) <= 1e-6,
                             factor_rel_err=max(c["mode_err"]), lambda_rel_err=c["lam_err"])
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    wl = args.workload if args.workload in WORKLOADS else "order4"
    T, R, extra, name = workload(wl)
    import oracle as O
    T64 = T.astype(np.float64)
    opts = oracle_options(extra)
    for _ in range(args.warmup):
        O.cpd(T64, R, opts)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.cpd(T64, R, opts)
    dt = time.perf_counter() - t0
    v = args.steps / dt
    line = dict(metric=METRIC, value=v, unit=UNIT, n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * dt / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=name, tensor_dims=list(T.shape), rank=R, global_batch=1,
                            parallelism="host"),
                cpu_baseline=dict(kind="oracle", cores=os.cpu_count(), value=v, unit=UNIT,
                                  sample=f"{args.steps} whole CPDs of {name} after {args.warmup} warm-up"),
                e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


def max_over_ranks(ms: float, world: int, device="cpu") -> float:
    """The slowest rank's timed-region milliseconds; every rank calls it after
    its own timed region (a barrier, then an all-reduce MAX)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    dist.barrier()
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank_step: float, steps: int, world: int, ms: float) -> float:
    """Units all ranks processed per second, over the slowest rank's time."""
    return world * units_per_rank_step * steps / (ms * 1e-3)


def start_barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _timed_steps(torch, step, flush, stream, K):
    """K steps, each bracketed by CUDA events on the launching stream, with an
    L2 flush (256 MB write) between steps outside the events."""
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    out = []
    for i in range(K):
        flush.zero_()
        starts[i].record(stream)
        out.append(step())
        ends[i].record(stream)
    torch.cuda.synchronize()
    return sum(s.elapsed_time(e) for s, e in zip(starts, ends)), out


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2110_05997_gb300 import build as bld
    from paper_2110_05997_gb300 import cpd

    bld.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)          # a capturable stream: solves replay CUDA graphs
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    if args.workload == "batch":
        return run_batch_workload(args, rank, world, local_rank, torch, cpd, dev, stream, flush)
    if args.workload == "initnet":
        return run_initnet_workload(args, rank, world, local_rank, torch, cpd, dev, stream, flush)
    T, R, extra, wname = workload(args.workload)
    dims = T.shape
    T_flat = synth.flat(T)
    Td = torch.from_numpy(T_flat).to(dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    opts = solve_options(cpd, args, extra)
    ws = torch.empty(cpd.cpd_workspace_size(dims, R, opts), dtype=torch.uint8, device=dev)

    # timed calls read no info record (no host synchronisation inside a step);
    # the record of the same solve is read after the timed region
    def step():
        return cpd.cpd_dgn_solve(Td, dims, R, opts, stream=stream, workspace=ws, want_info=False)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        start_barrier(world)
        torch.cuda.synchronize()
        l0 = cpd.cpd_launch_count()
        with ClockSampler(local_rank) as clk:
            ms, outs = _timed_steps(torch, step, flush, stream, args.steps)
        launches = cpd.cpd_launch_count() - l0
        W, lam, _, _ = outs[-1]
        info = cpd.cpd_dgn_solve(Td, dims, R, opts, stream=stream, workspace=ws)[2]
        infos = [info]
        # a replayed graph counts its refinement loop body once; the body ran
        # refine_iters times in each step (the library adds the difference
        # itself only when it reads the info record)
        launches += args.steps * 3 * (int(info["refine_iters"]) - 1)
        ms = max_over_ranks(ms, world, dev)
        value = whole_job_value(1, args.steps, world, ms)

        # per-stage device time: a second K-step region with CUDA-event scopes
        # around every launch (direct launches; graphs are bypassed while profiling)
        cpd.cpd_profile_enable(True)
        ms_prof, _ = _timed_steps(torch, step, flush, stream, args.steps)
        prof = cpd.cpd_profile_read()
        cpd.cpd_profile_enable(False)

        # end to end through the C ABI with host buffers: every step copies its
        # tensor from pinned host memory (H2D), solves it and reads W and lambda
        # back (D2H).  T is double-buffered on the device: the copy of step k+1
        # runs on a copy stream while step k is solved, as a caller streaming
        # tensors through the library would.  One span of CUDA events on the
        # compute stream brackets all K steps (the copy stream starts after the
        # opening event); the 400 MB inputs exceed L2, so no flush is needed.
        Th = torch.from_numpy(T_flat).pin_memory()
        Tbuf = [torch.empty_like(Td), torch.empty_like(Td)]
        copy_stream = torch.cuda.Stream(device=dev)
        n_out = R * sum(dims)
        Wh = torch.empty(n_out, dtype=torch.float32).pin_memory()
        lh = torch.empty(R, dtype=torch.float32).pin_memory()

        def e2e_run(K):
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            copied = [torch.cuda.Event(), torch.cuda.Event()]
            used = [torch.cuda.Event(), torch.cuda.Event()]
            torch.cuda.synchronize()
            t0.record(stream)
            copy_stream.wait_event(t0)
            with torch.cuda.stream(copy_stream):
                Tbuf[0].copy_(Th, non_blocking=True)
            copied[0].record(copy_stream)
            for k in range(K):
                b = k & 1
                if k + 1 < K:
                    nb = b ^ 1
                    if k >= 1:
                        copy_stream.wait_event(used[nb])       # step k-1 has read that buffer
                    with torch.cuda.stream(copy_stream):
                        Tbuf[nb].copy_(Th, non_blocking=True)
                    copied[nb].record(copy_stream)
                stream.wait_event(copied[b])
                W2, lam2, _, _ = cpd.cpd_dgn_solve(Tbuf[b], dims, R, opts, stream=stream, workspace=ws,
                                                   want_info=False)
                used[b].record(stream)
                Wh.copy_(torch.cat([w.t().reshape(-1) for w in W2]), non_blocking=True)
                lh.copy_(lam2, non_blocking=True)
            t1.record(stream)
            torch.cuda.synchronize()
            return t0.elapsed_time(t1)
        e2e_run(2)                                             # captures the graphs of both buffers
        start_barrier(world)
        e2e_ms = e2e_run(args.steps)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    e2e = dict(value=whole_job_value(1, args.steps, world, e2e_ms), unit=UNIT,
               h2d_bytes_per_step=int(Th.numel() * 4), d2h_bytes_per_step=int((n_out + R) * 4),
               pipeline="H2D of step k+1 on a copy stream during step k's solve (T double-buffered)",
               l2="no flush: every step's input (copied from the host) is larger than L2")

    if rank != 0:
        return 0
    pk = peaks()
    csum = clk.summary()
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"]) if prof else (None, None)
    roof = None
    if dom[0] is not None:
        per = dom[1]["ms"] / dom[1]["launches"]
        roof = algorithmic(dom[0], dims, R, infos[-1], per, pk, csum["sm_mhz"], sms=sms)
        roof.update(kernel=dom[0], launches=dom[1]["launches"], ms_per_launch=per, traffic=measured_traffic(dom[0]),
                    peak_source=pk["src"], region="separate profiled K-step region, direct launches")
    # the same roofline entry for the other stages that have a bound
    stage_roofs = {}
    for k, v in prof.items():
        if k == dom[0] or k not in ("gram_bf16_tc", "gram_fp32", "refine_pass", "project_T", "project"):
            continue
        n = v["launches"]
        if k == "refine_pass":
            # passes after the stop test exit at once: time the working ones
            passes = int(infos[-1].get("refine_iters", 0)) + 1
            if "full_start" in prof:       # dGN without compression: its iterations are passes too
                passes += int(infos[-1].get("iters", 0)) + 1
            n = min(n, args.steps * passes)
        r = algorithmic(k, dims, R, infos[-1], v["ms"] / max(n, 1), pk, csum["sm_mhz"],
                        gram_bf16=(args.gram == "bf16"), sms=sms)
        r.update(traffic=measured_traffic(k), working_launches=n)
        stage_roofs[k] = r
    stages = {k: dict(ms_per_step=v["ms"] / args.steps, launches_per_step=v["launches"] / args.steps)
              for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f32", data="synthetic",
                config=dict(workload=wname, tensor_dims=list(dims), start=extra.get("init", "mlsvd"),
                            rank=R, gram_precision=opts.gram_precision and "bf16" or "fp32",
                            refine_maxiter=int(opts.refine_maxiter), compress=int(opts.compress),
                            global_batch=world, parallelism=f"independent CPD per GPU x{world}",
                            l2="flushed between steps (256 MB write)", launch="cached CUDA graph per solve"),
                e2e=e2e, gpu_launches=int(launches), roofline=roof, stage_rooflines=stage_roofs, stages=stages,
                profiled_ms_per_step=ms_prof / args.steps,
                clocks=csum, solve=dict(core_iters=info["iters"], core_stop=info["stop_name"],
                                        core_cg=info["cg_total"], core_dims=info["core_dims"][:len(dims)],
                                        refine_iters=info["refine_iters"],
                                        refine_rel_err=info["refine_rel_err"]))
    if not args.no_cpu_baseline:
        Wg = [w.double().cpu().numpy() for w in W]
        lg = lam.double().cpu().numpy()
        cb = cpu_baseline(T, R, extra, wname, Wg, lg, budget_s=args.cpu_budget)
        line["parity"] = cb.pop("parity", None)
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)
    return 0


def run_batch_workload(args, rank, world, local_rank, torch, cpd, dev, stream, flush):
    """Optional line: the 4096-item uneven batch (modes U{8..48}, ranks U{2..8},
    noise 1e-6) in one persistent launch; CPDs/s of the whole batch."""
    items = synth.c4_batch()
    offs, o = [], 0
    for it in items:
        offs.append(o)
        o += it["T"].size
    flat = np.concatenate([synth.flat(it["T"]).astype(np.float32) for it in items])
    Tp = torch.from_numpy(flat).to(dev)
    dims = [list(it["T"].shape) for it in items]
    ranks = [it["R"] for it in items]
    # stop tolerance one decade below the noise level: the fit then agrees with
    # the oracle's within 1e-6 (with tol = noise the improvement test stops at
    # rounding-dependent points above the noise floor)
    opts = cpd.cpd_default_options(tol=1e-7)
    ws = torch.empty(cpd.cpd_batch_workspace_size(dims, ranks, opts), dtype=torch.uint8, device=dev)

    def step():
        return cpd.cpd_batch_solve(Tp, offs, dims, ranks, opts, stream=stream, workspace=ws, want_infos=False)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        start_barrier(world)
        torch.cuda.synchronize()
        l0 = cpd.cpd_launch_count()
        with ClockSampler(local_rank) as clk:
            ms, _ = _timed_steps(torch, step, flush, stream, args.steps)
        launches = cpd.cpd_launch_count() - l0
    ms = max_over_ranks(ms, world, dev)
    B = len(items)
    # what the autotuner chose between: each CTA size forced, one timed step
    cta_ms = {}
    for th in (64, 128, 256):
        o_th = cpd.cpd_default_options(block_threads=th, tol=1e-7)
        with torch.cuda.stream(stream):
            cpd.cpd_batch_solve(Tp, offs, dims, ranks, o_th, stream=stream, workspace=ws, want_infos=False)
            torch.cuda.synchronize()
            t_th, _ = _timed_steps(torch, lambda: cpd.cpd_batch_solve(Tp, offs, dims, ranks, o_th, stream=stream,
                                                                      workspace=ws, want_infos=False),
                                   flush, stream, 2)
        cta_ms[str(th)] = t_th / 2
    # the same problems one launch sequence per tensor (cpd_dgn_solve, graph
    # replays), on a seeded sample of 256 items
    pick = np.random.default_rng(7).choice(B, size=min(256, B), replace=False)
    per = [(torch.from_numpy(synth.flat(items[int(b)]["T"]).astype(np.float32)).to(dev), dims[int(b)],
            ranks[int(b)]) for b in pick]
    popts = cpd.cpd_default_options(tol=1e-7)
    pws = torch.empty(max(cpd.cpd_workspace_size(d, r, popts) for _, d, r in per), dtype=torch.uint8, device=dev)

    def per_tensor():
        for Tb, d, r in per:
            cpd.cpd_dgn_solve(Tb, d, r, popts, stream=stream, workspace=pws)
    with torch.cuda.stream(stream):
        per_tensor()
        torch.cuda.synchronize()
        pms, _ = _timed_steps(torch, per_tensor, flush, stream, 1)
    per_rate = len(per) / (pms * 1e-3)
    if rank != 0:
        return 0
    line = dict(metric="CPDs/sec (batched uneven CPDs)", value=whole_job_value(B, args.steps, world, ms),
                unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup, ms_per_step=ms / args.steps,
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload="batch_4096_uneven_3rd_order_r2-8_noise1e-6", tol=1e-7, global_batch=B * world,
                            parallelism=f"one persistent launch per GPU x{world}",
                            l2="flushed between steps (256 MB write)"),
                gpu_launches=int(launches), clocks=clk.summary(),
                ms_per_batch_by_cta_threads=cta_ms,
                per_tensor_launches=dict(cpds_per_s=per_rate, sample=f"{len(per)} seeded items of the batch, "
                                         "one cpd_dgn_solve (graph replay) each", per_gpu=True))
    print(json.dumps(line), flush=True)
    return 0


def run_initnet_workload(args, rank, world, local_rank, torch, cpd, dev, stream, flush):
    """Optional line: the learned initialiser.  Trains the network with the
    library's kernels on the cores of 196608 planted 16^3 problems (rank
    U{1..8}, collinearity U[0, 0.9], noise 1e-6) solved by the method, then
    times 4096 held-out problems solved from the learned start (MLSVD start
    as fallback) and from the MLSVD start alone; reports both, with mean dGN
    iterations and the fraction reaching the noise floor."""
    from paper_2110_05997_gb300 import initnet

    def pack(Tc, Rs):
        B = Tc.shape[0]
        return (torch.from_numpy(np.ascontiguousarray(Tc.reshape(-1))).to(dev), [b * 4096 for b in range(B)],
                [[16, 16, 16]] * B, [int(r) for r in Rs])
    t0 = time.perf_counter()
    Xs, Ms = [], []
    for c in range(12):
        Tc, Rs, _ = synth.c5_initnet(seed=synth.SEED_BASE + 500 + c, B=16384)
        Tp, to, d, r = pack(Tc, Rs)
        X, _, msk, *_ = cpd.cpd_batch_initnet_data(Tp, to, d, r, cpd.cpd_default_options(seed=1))
        Xs.append(X); Ms.append(msk)
    X, M = torch.cat(Xs), torch.cat(Ms)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    params = initnet.init_params(seed=3, device=dev)
    t0 = time.perf_counter()
    hist = initnet.train(params, X, None, M, epochs=20, batch=512, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del X, M, Xs, Ms
    Th, Rh, _ = synth.c5_initnet(seed=synth.SEED_BASE + 5, B=4096)
    Tp, to, d, r = pack(Th, Rh)
    opts = cpd.cpd_default_options(seed=7)
    ws = torch.empty(cpd.cpd_batch_ex_workspace_size(d, r, opts), dtype=torch.uint8, device=dev)

    def plain():
        return cpd.cpd_batch_solve(Tp, to, d, r, opts, stream=stream, workspace=ws, want_infos=False)

    def learned():
        return cpd.cpd_batch_solve_learned(Tp, to, d, r, params, opts, stream=stream, workspace=ws,
                                           want_infos=False)
    res = {}
    with torch.cuda.stream(stream):
        for name, fn in (("plain", plain), ("learned", learned)):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            start_barrier(world)
            torch.cuda.synchronize()
            l0 = cpd.cpd_launch_count()
            with ClockSampler(local_rank) as clk:
                ms, _ = _timed_steps(torch, fn, flush, stream, args.steps)
            ms = max_over_ranks(ms, world, dev)
            res[name] = dict(ms=ms / args.steps, launches=cpd.cpd_launch_count() - l0, clocks=clk.summary())
    _, _, _, _, ib = cpd.cpd_batch_solve(Tp, to, d, r, opts, workspace=ws)
    _, _, _, _, il = cpd.cpd_batch_solve_learned(Tp, to, d, r, params, opts, workspace=ws)
    if rank != 0:
        return 0
    stats = {}
    for name, inf in (("plain", ib), ("learned", il)):
        it = np.array([i["iters"] for i in inf]); e = np.array([i["rel_err"] for i in inf])
        stats[name] = dict(cpds_per_s=4096 / (res[name]["ms"] * 1e-3), ms_per_batch=res[name]["ms"],
                           mean_dgn_iters=float(it.mean()), converged_rel_err_lt_1e_5=float(np.mean(e < 1e-5)))
    stats["learned"]["learned_start_taken"] = float(np.mean([i["init_used"] for i in il]))
    line = dict(metric="CPDs/sec (batched 16^3 cores, learned start)", value=world * stats["learned"]["cpds_per_s"],
                unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=res["learned"]["ms"], higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="bf16 network, f32 dGN", data="synthetic",
                config=dict(workload="initnet_16^3_r1-8_rho0-0.9_noise1e-6", global_batch=4096 * world,
                            train_problems=196608, train_epochs=20, l2="flushed between steps (256 MB write)"),
                plain=stats["plain"], learned=stats["learned"], train_loss_first_last=[hist[0], hist[-1]],
                data_s=t_data, train_s=t_train, gpu_launches=int(res["learned"]["launches"]),
                clocks=res["learned"]["clocks"])
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--gram", choices=["fp32", "bf16"], default="bf16")
    workloads = ["order4", "compressed200", "full400", "full_order4", "batch", "initnet"]
    ap.add_argument("--workload", choices=workloads, default="order4")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
