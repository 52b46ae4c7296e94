#!/usr/bin/env python
"""Benchmark of the FMM-based NUFFT / INUFFT on GB300.

Workload (one step): forward NUFFT c -> g followed by the square inverse
g -> c on N = M = 2^20 complex128 data, y_j a 40 % jittered grid
(2 pi j/N + U(-0.4, 0.4) 2 pi/N), mixed precision at eps = 1e-6 (FP32 far
and near field, FP64 F_j / C_k / D_j / FFT).  The plan (binning, F_j, the
C_k / D_j log-sums) is built once, outside the timed region, as the paper
separates setting the data structure from evaluation (Sec. 3.3).

metric: non-uniform points per second, 2 M points per step (M through the
forward and M through the inverse).  The same step is also timed in the
plain FP64 path at eps = 1e-12 and reported under "fp64".

Multi-GPU (torchrun, N > 1): replicas only -- the transform has no exchange
step here, each rank runs the full workload on its own GPU; value is the
points of all ranks divided by the slowest rank's time.

--impl reference times the FP64 CPU oracle (the definition, O(N M)) on the
host cores for a bounded sample of targets of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

N_LOG2 = 20
EPS_MIXED = 1e-6
EPS_FP64 = 1e-12
JITTER = 0.4
METRIC = "NUFFT points/s (forward + square inverse, N=M=2^20, mixed eps=1e-6)"
# DRAM bytes (read + write) of the target-evaluation kernels per step (the
# forward's near-field and far-part launches, k_targets_fwd + k_far_fwd, and
# the inverse's, k_targets_grid2 in its near-field and far-part forms) from
# one ncu capture of this workload; reported only while the kernels' source
# text still hashes to `sha1` (a changed kernel reports null until it is
# captured again)
TARGETS_TRAFFIC = {"bytes_per_step": 134244096, "sha1": "ebb9f3d4bfb21e09e793b192dcd9f71ba03f65e2"}
STAGE_KERNELS = {"targets": "k_targets_fwd + k_far_fwd + k_targets_grid2 (near-field and far-part forms)", "fft": "k_fft_st",
                 "m2l": "k_down_fused (tensor-core levels: k_down_top + k_down_sub + k_m2l_tc)",
                 "p2m": "k_p2m_* + k_charges (when not inside k_up_fused)",
                 "m2m": "k_up_fused (with P2M and the charges when they fit)",
                 "level2": "k_level2"}
L2_FLUSH_BYTES = 512 << 20
E2E_FLUSH_BYTES = 256 << 20  # twice the 129 MB L2


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples during the timed region (median SM clock, reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- roofline model

def stage_work(stage: str, N: int, M: int, info: dict, io_bytes: int, fwd: int, bwd: int):
    """Algorithmic work of a stage per step of `fwd` forward and `bwd`
    adjoint / inverse sequences (each N grid points, M points, one signal):
    (flops, bytes, bound), counted from the method, not from the code.
      fft:     one read and one write of the N values per transform (io_bytes
               per complex value at the interface, 8 inside the FP32 path)
      p2m:     N pm (forward) or M pm (adjoint / inverse) complex-real FMA
               (4 flops each)
      m2m:     ~B parents x pm^2 complex-real FMA per pass
      m2l:     ~2B boxes x (3 p^2 + p^2 / 2) complex-real FMA per pass
      targets: per target (3s - 1) near pairs x 4 flops (the reciprocal
               counted as one flop) + p + 2q complex-real FMA (far field,
               regular part)"""
    L, p, q = info["lmax"], info["p"], info["q"]
    pm = max(p, 2 * q + 1)
    s = N >> L
    B = 1 << L
    nseq = fwd + bwd
    if stage == "fft":
        return 5 * N * math.log2(N) * nseq, (io_bytes + 8) * N * nseq, "hbm"
    if stage == "p2m":
        return 4 * (N * fwd + M * bwd) * pm, 0, "alu"
    if stage == "m2m":
        return 4 * B * pm * pm * nseq, 0, "alu"
    if stage == "m2l":
        return 4 * 2 * B * 3.5 * p * p * nseq, 0, "alu"
    if stage == "targets":
        per = (3 * s - 1) * 4 + 4 * p + 8 * q
        return per * (M * fwd + N * bwd), 0, "alu"
    return 0, 0, "other"


def stage_roofline(stages_ms: dict, N: int, M: int, info: dict, io_bytes: int, fwd: int, bwd: int,
                   peaks: dict) -> dict:
    """Per-stage achieved rate against its bound: FP32 ALU (152 SMs x 128
    lanes x 2 flops x max clock; for the targets, whose pair loop takes one
    reciprocal per pair, the special-function unit's 16 per clock per SM) or
    HBM (measured copy bandwidth)."""
    out = {}
    p2m_fused = stages_ms.get("p2m", 0.0) <= 0
    for st, ms in stages_ms.items():
        if ms <= 0:
            continue
        fl, by, bound = stage_work(st, N, M, info, io_bytes, fwd, bwd)
        if st == "m2m" and p2m_fused:  # the upward kernel formed the leaf multipoles too
            fl += stage_work("p2m", N, M, info, io_bytes, fwd, bwd)[0]
        if bound == "hbm":
            ach = by / (ms / 1e3) / 1e9
            out[st] = {"ms": ms, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
                       "unit": "GB/s", "frac": ach / peaks["hbm_gbs"]}
        elif bound == "alu":
            ach = fl / (ms / 1e3) / 1e12
            pk = fp32_peak_tflops(peaks)
            out[st] = {"ms": ms, "bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                       "frac": ach / pk}
            if st == "targets":
                # the pair loop's binding unit is the reciprocal (special-function)
                # pipe: pairs per second against its rate; beside it the FP32 FMA
                # pipe with 6 flops per pair (one division + 5) plus 4p per target
                L, p = info["lmax"], info["p"]
                pairs = near_pairs(N, M, L, fwd, bwd)
                tps = pairs / (ms / 1e3) / 1e12
                pk_pair = pair_peak_tps(peaks)
                fl6 = 6 * pairs + 4 * p * (M * fwd + N * bwd)
                out[st] = {"ms": ms, "bound": "alu", "achieved": tps, "peak": pk_pair,
                           "unit": "T pairs/s (one FP32 reciprocal each)", "frac": tps / pk_pair,
                           "pairs": pairs, "achieved_fp32_tflops": fl6 / (ms / 1e3) / 1e12,
                           "peak_fp32_fma": pk, "frac_fp32_fma": fl6 / (ms / 1e3) / 1e12 / pk}
        else:
            out[st] = {"ms": ms, "bound": None}
    return out


def targets_source_sha1() -> str:
    """SHA-1 of the near-field / target-kernel section of k_fmm.cu (the
    device code from the pair reciprocal to the first host function) and of
    the pair reciprocal itself (common.cuh)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1611_09379_gb300", "csrc")
    src = open(os.path.join(csrc, "k_fmm.cu")).read()
    a = src.index("// 1/t of a near-field pair")
    e = src.index("static inline unsigned nblk")
    com = open(os.path.join(csrc, "common.cuh")).read()
    ra = com.index("// 1/t of a near-field pair")
    re_ = com.index("// Leaf index and offset of a point")
    return hashlib.sha1((src[a:e] + com[ra:re_]).encode()).hexdigest()


# FP32 reciprocals and FMAs per SM per clock: measured at start-up by the
# library's probe (nufft_diag_pipe_rates); the CUDA C++ Programming Guide's
# arithmetic-throughput table gives 16 and 128 for this architecture.
PIPES = {"rcp_per_clk": 16.0, "ffma_per_clk": 128.0, "source": "CUDA C++ Programming Guide table"}
N_SM = 152


def fp32_peak_tflops(peaks):
    # SMs x measured FP32 FMAs per clock x 2 flops x max SM clock
    return N_SM * PIPES["ffma_per_clk"] * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def pair_peak_tps(peaks):
    # near-field pairs per second (1e12) if every SM's special-function unit
    # finishes one FP32 reciprocal per pair at its measured rate, max clock
    return N_SM * PIPES["rcp_per_clk"] * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def near_pairs(N: int, M: int, lmax: int, fwd: int, bwd: int) -> int:
    """Near-field pairs of one step: every target meets the 3s grid points
    (forward) or the sources (adjoint / inverse) of its leaf and the two
    neighbouring leaves, less the one pair per point handled in closed form
    (its nearest grid point): (3s - 1) M per forward, and, summed over the grid
    targets, 3 s M - M per adjoint / inverse (each leaf's sources are seen by
    the 3s grid points around them)."""
    s = N >> lmax
    return (3 * s - 1) * M * (fwd + bwd)


# ---------------------------------------------------------------- replicas

def ranks_max(x: float, ws: int, dev) -> float:
    """Largest value of x over the ranks (the slowest replica's time); the
    tensor lives on `dev` (the rank's GPU under NCCL, the CPU under gloo)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(points_per_replica: int, ms_slowest: float, ws: int) -> float:
    """Whole-job points/s of ws independent replicas: the points of all ranks
    over the slowest rank's time per step."""
    return ws * points_per_replica / (ms_slowest / 1e3)


# ---------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1611_09379_gb300 as nf
    from paper_1611_09379_gb300 import tune

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    # the pipe rates behind the targets' roofline, measured on this GPU
    try:
        rcp, ffma = nf.pipe_rates()
        PIPES.update({"rcp_per_clk": rcp, "ffma_per_clk": ffma,
                      "source": "measured (nufft_diag_pipe_rates: per-SM clock counters, median SM)"})
    except Exception as e:  # keep the table's counts, say so
        PIPES["source"] += f" (probe failed: {e!r})"

    N = M = 1 << N_LOG2
    y = workloads.points("jitter", M, N, seed=1234, jitter=JITTER)
    c = workloads.coeffs(N, seed=99)
    yd = torch.from_numpy(y).to(dev)
    cd = torch.from_numpy(c).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    results = {}
    tuning = {}
    arms = (("mixed", nf.MIXED, EPS_MIXED), ("fp64", nf.FP64, EPS_FP64),
            ("fp64_eps1e-6", nf.FP64, EPS_MIXED))
    if args.only_mixed:  # profiling runs: the headline arm alone
        arms = arms[:1]
    for tag, prec, eps in arms:
        prm = {}
        if not args.no_tune:
            # empirical l_max, p, q, tc_level for this point set (outside the timing,
            # like the plan: Sec. 3.3 separates setting up from evaluating)
            ent = tune.autotune(N, yd, eps, prec=prec, ops="fwd+inv", reps=5, tag="jitter0.4")
            prm = {k: ent["params"][k] for k in ("lmax", "p", "q", "tc_level", "tc_near")}
            chosen = [t for t in ent["trials"] if t["accepted"]]
            tuning[tag] = {"params": ent["params"], "seconds": ent["seconds"],
                           "from_table": ent["from_table"],
                           "formula_params": ent["trials"][0]["params"] if ent["trials"] else None,
                           "formula_ms": ent["trials"][0]["ms"] if ent["trials"] else None,
                           "tuned_ms": chosen[0]["ms"] if chosen else None,
                           "tuned_err_vs_fp64_fmm": chosen[0]["err"] if chosen else None,
                           "candidates": len(ent["trials"])}
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        plan = nf.Plan(N, yd, eps=eps, prec=prec, inverse=True, **prm)
        torch.cuda.synchronize(dev)
        t_plan = time.perf_counter() - t0
        g = torch.empty(M, dtype=torch.complex128, device=dev)
        c2 = torch.empty(N, dtype=torch.complex128, device=dev)

        def step():
            plan.forward(cd, out=g)
            plan.inverse(g, out=c2)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        with ClockSampler(local) as clk:
            for i in range(args.steps):
                flush.zero_()  # L2 flush outside the timed events
                ev[i][0].record(stream)
                step()
                ev[i][1].record(stream)
            torch.cuda.synchronize(dev)
        if ws > 1:
            dist.barrier()
        ms = [a.elapsed_time(b) for a, b in ev]
        # per-stage times from separate profiled steps (event-bracketed stages,
        # kernels launched one by one; the timed steps above replay graphs)
        plan.profile(True)
        for _ in range(args.steps):
            flush.zero_()
            step()
        stats = plan.stats()
        plan.profile(False)
        # accuracy on sampled targets (oracle definition), outside the timing
        results[tag] = {"ms": ms, "stats": stats, "info": plan.params(), "t_plan_s": t_plan,
                        "clocks": clk.summary(), "g": g, "c2": c2}
        # e2e through the public API with host buffers (pinned), every step's
        # copies inside one timed region: c in, g and c out, pipelined on two
        # copy streams (the next step's c goes in and this step's g, c come
        # out while the GPU computes); two slots of device and pinned host
        # buffers; L2 flushed (E2E_FLUSH_BYTES write) at the start of every
        # step inside the timed region
        if tag == "mixed":
            S = 2
            hc = [torch.from_numpy(c).pin_memory() for _ in range(S)]
            hg = [torch.empty(M, dtype=torch.complex128).pin_memory() for _ in range(S)]
            hc2 = [torch.empty(N, dtype=torch.complex128).pin_memory() for _ in range(S)]
            dcs = [torch.empty(N, dtype=torch.complex128, device=dev) for _ in range(S)]
            gs = [torch.empty(M, dtype=torch.complex128, device=dev) for _ in range(S)]
            c2s = [torch.empty(N, dtype=torch.complex128, device=dev) for _ in range(S)]
            fl = flush[: E2E_FLUSH_BYTES // 4]
            h2d = torch.cuda.Stream(dev)
            d2h = torch.cuda.Stream(dev)
            c_ready = [torch.cuda.Event() for _ in range(S)]
            fwd_done = [torch.cuda.Event() for _ in range(S)]
            inv_done = [torch.cuda.Event() for _ in range(S)]
            out_done = [torch.cuda.Event() for _ in range(S)]

            def h2d_issue(i):
                sl = i % S
                h2d.wait_event(fwd_done[sl])  # the slot's previous input consumed
                with torch.cuda.stream(h2d):
                    dcs[sl].copy_(hc[sl], non_blocking=True)
                c_ready[sl].record(h2d)

            def e2e_step(i):
                sl = i % S
                stream.wait_event(c_ready[sl])
                stream.wait_event(out_done[sl])  # the slot's previous outputs on the host
                fl.zero_()
                plan.forward(dcs[sl], out=gs[sl])
                fwd_done[sl].record(stream)
                plan.inverse(gs[sl], out=c2s[sl])
                inv_done[sl].record(stream)
                d2h.wait_event(fwd_done[sl])
                with torch.cuda.stream(d2h):
                    hg[sl].copy_(gs[sl], non_blocking=True)
                d2h.wait_event(inv_done[sl])
                with torch.cuda.stream(d2h):
                    hc2[sl].copy_(c2s[sl], non_blocking=True)
                out_done[sl].record(d2h)

            def e2e_run(first, count, ev_a=None):
                for k in range(count):
                    i = first + k
                    if k == 0:
                        if ev_a is not None:
                            h2d.wait_event(ev_a)
                        h2d_issue(i)
                    e2e_step(i)
                    if k + 1 < count:
                        h2d_issue(i + 1)

            e2e_run(0, args.warmup)
            torch.cuda.synchronize(dev)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            e2e_run(args.warmup, args.steps, a)
            stream.wait_stream(d2h)
            b.record(stream)
            torch.cuda.synchronize(dev)
            results[tag]["e2e_ms"] = [a.elapsed_time(b) / args.steps]
            results[tag]["e2e_bytes"] = (N * 16, M * 16 + N * 16)
            last = (args.warmup + args.steps - 1) % S
            results[tag]["e2e_check"] = float(np.abs(hc2[last].numpy() - c).max() /
                                              np.abs(c).max())
        plan.close()

    mx = results["mixed"]
    ms_step = ranks_max(sum(mx["ms"]) / len(mx["ms"]), ws, dev)
    value = replica_throughput(2 * M, ms_step, ws)
    if args.only_mixed:
        results["fp64"] = results["fp64_eps1e-6"] = dict(mx, g=mx["g"], c2=mx["c2"])
    fp = results["fp64"]
    ms_fp64 = ranks_max(sum(fp["ms"]) / len(fp["ms"]), ws, dev)
    fp6 = results["fp64_eps1e-6"]
    ms_fp64_6 = ranks_max(sum(fp6["ms"]) / len(fp6["ms"]), ws, dev)
    e2e_ms = ranks_max(sum(mx["e2e_ms"]) / len(mx["e2e_ms"]), ws, dev)

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return

    # accuracy (sampled 1024 targets / 512 coefficients against the oracle)
    acc = {}
    try:
        import oracle
        idx = workloads.sample_index(M, 1024)
        gref = oracle.nudft_fwd(c, y, idx)
        for tag in ("mixed", "fp64", "fp64_eps1e-6"):
            gh = results[tag]["g"].cpu().numpy()
            c2h = results[tag]["c2"].cpu().numpy()
            acc[tag] = {"fwd_rel_l2_sampled": oracle.rel_l2(gh[idx], gref),
                        "inv_roundtrip_rel_l2": oracle.rel_l2(c2h, c)}
    except Exception as e:  # accuracy is reported, not gating
        acc["error"] = repr(e)

    peaks, peak_src = _peaks()
    stats = mx["stats"]
    steps = args.steps
    launches = int(sum(v[1] for v in stats.values()))
    # dominant stage and its roofline
    per = {k: v[0] / steps for k, v in stats.items()}
    dom = max(per, key=per.get)
    info = mx["info"]
    sroof = stage_roofline(per, N, M, info, 16, 1, 1, peaks)
    r = sroof[dom]
    roof = {k: r[k] for k in ("bound", "achieved", "peak", "unit", "frac")}
    roof["traffic"] = None
    if dom == "targets" and TARGETS_TRAFFIC["bytes_per_step"] and \
            TARGETS_TRAFFIC["sha1"] == targets_source_sha1():
        roof["traffic"] = TARGETS_TRAFFIC["bytes_per_step"]
        roof["traffic_unit"] = "DRAM bytes per step (ncu dram__bytes_read + write, the four target launches)"
    roof["kernel_stage"] = dom
    roof["kernels"] = STAGE_KERNELS.get(dom)
    if roof["bound"] == "hbm":
        roof["peak_source"] = f"{peak_src}: MEASURED_PEAKS hbm_gbs"
    elif dom == "targets":
        roof["peak_source"] = (f"{N_SM} SM x {PIPES['rcp_per_clk']:.2f} FP32 reciprocals/clk "
                               f"({PIPES['source']}) x sm_max_mhz {peaks.get('sm_max_mhz')} "
                               f"({peak_src}); one reciprocal per near-field pair")
        roof["pairs_per_step"] = r["pairs"]
        roof["frac_fp32_fma"] = r["frac_fp32_fma"]
        roof["fp32_fma_peak_tflops"] = r["peak_fp32_fma"]
        roof["fp32_fma_count"] = "6 flops per near pair + 4p per target (far field)"
    else:
        roof["peak_source"] = (f"{peak_src}: {N_SM} SM x {PIPES['ffma_per_clk']:.1f} FP32 FMA/clk "
                               f"x 2 x sm_max_mhz")

    # cpu baseline: the oracle (direct forward definition) on sampled targets
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(c, y, budget_s=args.cpu_seconds)

    out = {
        "metric": METRIC,
        "value": value,
        "unit": "points/s",
        "n_gpus": ws,
        "steps": steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64 (mixed)",
        "data": "synthetic: y jittered grid (U(-0.4,0.4)), c iid N(0,1) complex128",
        "config": {"workload": "forward + square inverse NUFFT, N=M=2^20, complex128, jittered y, "
                               "mixed eps=1e-6",
                   "N": N, "M": M, "eps": EPS_MIXED, "lmax": info["lmax"], "p": info["p"],
                   "q": info["q"], "tc_level": info.get("tc_level"),
                   "params": "autotuned (nufft_autotune)" if tuning else "Eq. 18.2 / 25 formulas",
                   "l2": "flushed (512 MiB write) between timed steps",
                   "parallelism": "replicas" if ws > 1 else "1 gpu",
                   "plan_s": mx["t_plan_s"]},
        "stages_ms_per_step": {k: round(v, 5) for k, v in per.items()},
        "stage_roofline": sroof,
        "points_per_step": 2 * M,
        "value_per_transform": value / 2,
        "fp64": {"eps": EPS_FP64, "ms_per_step": ms_fp64, "value": replica_throughput(2 * M, ms_fp64, ws),
                 "params": fp["info"], "stages_ms_per_step":
                     {k: round(v[0] / steps, 5) for k, v in fp["stats"].items()},
                 "plan_s": fp["t_plan_s"]},
        "fp64_eps1e-6": {"eps": EPS_MIXED, "ms_per_step": ms_fp64_6,
                         "value": replica_throughput(2 * M, ms_fp64_6, ws), "params": fp6["info"],
                         "stages_ms_per_step":
                             {k: round(v[0] / steps, 5) for k, v in fp6["stats"].items()},
                         "mixed_speedup_same_eps": ms_fp64_6 / ms_step},
        "pipes": dict(PIPES),
        "accuracy": acc,
        "tuning": tuning or None,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": replica_throughput(2 * M, e2e_ms, ws), "unit": "points/s",
                "h2d_bytes_per_step": mx["e2e_bytes"][0], "d2h_bytes_per_step": mx["e2e_bytes"][1],
                "ms_per_step": e2e_ms,
                "timing": "one timed region over the steps: each step's c copied in, g and c "
                          "copied out (pinned host buffers, two slots, copies on two streams "
                          "beside the compute), L2 flushed (256 MiB write) at the start of "
                          "every step inside the region",
                "roundtrip_max_rel_err": mx["e2e_check"]},
        "gpu_launches": launches,
        "clocks": mx["clocks"],
    }
    if not args.no_batched:
        out["batched"] = run_batched(tune_params=not args.no_tune)
    if not args.no_large:
        out["large"] = run_large(tune_params=not args.no_tune)
    if not args.no_adaptive:
        out["adaptive_tree"] = run_adaptive(tune_params=not args.no_tune)
    if not args.no_lsq:
        out["inufft_lsq"] = run_lsq(budget_s=args.lsq_seconds, full=args.lsq_full)
    print(json.dumps(out))
    if ws > 1:
        dist.destroy_process_group()


def _timed(fn, flush, stream, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    ms = []
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return sum(ms) / len(ms)


def run_batched(steps: int = 5, warmup: int = 3, tune_params: bool = True):
    """Batched workloads, eps = 1e-6, mixed precision, complex64:
    (i) 64 signals sharing one uniform point set, N = M = 2^18, one batched
    forward; (ii) 256 independent forward transforms, N = M = 2^U with U
    uniform in {10..16}, own uniform points each, one CUDA graph launch."""
    import torch

    import paper_1611_09379_gb300 as nf
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    out = {}
    N = M = 1 << 18
    B = 64
    y = workloads.points("uniform", M, seed=1234)
    rng = workloads.rng(5)
    C = (rng.standard_normal((B, N)) + 1j * rng.standard_normal((B, N))).astype(np.complex64)
    yd = torch.from_numpy(y).cuda()
    prm, tuned = {}, None
    if tune_params:
        from paper_1611_09379_gb300 import tune
        ent = tune.autotune(N, yd, 1e-6, prec=nf.MIXED, io="c64", batch=B, ops="fwd", reps=3,
                            tag="uniform")
        prm = {k: ent["params"][k] for k in ("lmax", "p", "q", "tc_level", "tc_near")}
        tuned = {"seconds": ent["seconds"], "formula_ms": ent["trials"][0]["ms"],
                 "formula_params": ent["trials"][0]["params"]}
    plan = nf.Plan(N, yd, eps=1e-6, prec=nf.MIXED, io="c64", batch=B, **prm)
    Cd = torch.from_numpy(C).cuda()
    G = torch.empty((B, M), dtype=torch.complex64, device="cuda")
    ms = _timed(lambda: plan.forward(Cd, out=G), flush, stream, steps, warmup)
    plan.profile(True)
    _timed(lambda: plan.forward(Cd, out=G), flush, stream, steps, 0)
    stages = {k: round(v[0] / steps, 5) for k, v in plan.stats().items()}
    plan.profile(False)
    acc = None
    try:
        import oracle
        idx = workloads.sample_index(M, 256)
        Gh = G.cpu().numpy()
        acc = max(oracle.rel_l2(Gh[b][idx], oracle.nudft_fwd(C[b].astype(complex), y, idx)) for b in (0, 31, 63))
    except Exception as e:
        acc = repr(e)
    out["signals64"] = {"N": N, "M": M, "batch": B, "ms": ms, "value": B * M / (ms / 1e3),
                        "unit": "points/s", "params": plan.params(), "tuning": tuned,
                        "stages_ms": stages, "fwd_rel_l2_sampled_max": acc}
    plan.close()
    U = workloads.rng(6).integers(10, 17, size=256)
    Ns = [1 << int(u) for u in U]
    ys = [torch.from_numpy(workloads.points("uniform", n, seed=1000 + i)).cuda() for i, n in enumerate(Ns)]
    cs = [torch.from_numpy(workloads.coeffs(n, seed=2000 + i).astype(np.complex64)).cuda()
          for i, n in enumerate(Ns)]
    gs = [torch.empty(n, dtype=torch.complex64, device="cuda") for n in Ns]
    # parameters per size class (outside the timing, like the plans): the
    # autotuner once per N on the first transform of that size, its choice
    # used for every transform of the class
    t0 = time.perf_counter()
    per_class = {}
    if tune_params:
        from paper_1611_09379_gb300 import tune
        for n in sorted(set(Ns)):
            i0 = Ns.index(n)
            ent = tune.autotune(n, ys[i0], 1e-6, prec=nf.MIXED, io="c64", ops="fwd", reps=3,
                                tag="uniform")
            per_class[n] = {k: ent["params"][k] for k in ("lmax", "p", "q", "tc_level", "tc_near")}
    t_tune = time.perf_counter() - t0
    t0 = time.perf_counter()
    multi = nf.Multi(Ns, ys, eps=1e-6, prec=nf.MIXED, io="c64",
                     params=[per_class.get(n) for n in Ns] if per_class else None)
    t_plan = time.perf_counter() - t0
    ms = _timed(lambda: multi.forward(cs, gs), flush, stream, steps, warmup)
    acc = None
    try:
        import oracle
        worst = 0.0
        for i in (0, int(np.argmax(Ns)), 255):
            idx = workloads.sample_index(Ns[i], 64, seed=i)
            y_i = ys[i].cpu().numpy()
            ref = oracle.nudft_fwd(cs[i].cpu().numpy().astype(complex), y_i, idx)
            worst = max(worst, oracle.rel_l2(gs[i].cpu().numpy()[idx], ref))
        acc = worst
    except Exception as e:
        acc = repr(e)
    out["uneven256"] = {"count": 256, "points": int(sum(Ns)), "ms": ms,
                        "value": sum(Ns) / (ms / 1e3), "unit": "points/s", "plan_s": t_plan,
                        "tune_s": t_tune,
                        "params_per_N": {str(n): v for n, v in sorted(per_class.items())} or
                        "formulas",
                        "fwd_rel_l2_sampled_max": acc,
                        "launch": "one CUDA graph (64 forked streams)"}
    multi.close()
    return out


def run_large(steps: int = 5, warmup: int = 3, tune_params: bool = True):
    """Large workload: N = M = 2^24, complex64 data, uniform points, forward
    + adjoint at eps = 1e-6 (mixed precision), per-stage roofline."""
    import torch

    import paper_1611_09379_gb300 as nf
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    N = M = 1 << 24
    y = workloads.points("uniform", M, seed=1238)
    c = workloads.coeffs(N, seed=34).astype(np.complex64)
    gin = workloads.samples(M, seed=35).astype(np.complex64)
    yd = torch.from_numpy(y).cuda()
    prm, tuned = {}, None
    if tune_params:
        from paper_1611_09379_gb300 import tune
        ent = tune.autotune(N, yd, 1e-6, prec=nf.MIXED, io="c64", ops="fwd+adj", reps=3,
                            tag="uniform")
        prm = {k: ent["params"][k] for k in ("lmax", "p", "q", "tc_level", "tc_near")}
        tuned = {"seconds": ent["seconds"], "formula_ms": ent["trials"][0]["ms"],
                 "formula_params": ent["trials"][0]["params"]}
    plan = nf.Plan(N, yd, eps=1e-6, prec=nf.MIXED, io="c64", **prm)
    cd, gd = torch.from_numpy(c).cuda(), torch.from_numpy(gin).cuda()
    g = torch.empty(M, dtype=torch.complex64, device="cuda")
    a = torch.empty(N, dtype=torch.complex64, device="cuda")

    def step():
        plan.forward(cd, out=g)
        plan.adjoint(gd, out=a)

    ms = _timed(step, flush, stream, steps, warmup)
    plan.profile(True)
    _timed(step, flush, stream, steps, 0)
    per = {k: v[0] / steps for k, v in plan.stats().items()}
    plan.profile(False)
    peaks, _ = _peaks()
    info = plan.params()
    acc = None
    try:
        import oracle
        idx = workloads.sample_index(M, 64)
        kdx = workloads.sample_index(N, 64, seed=6)
        acc = {"fwd_rel_l2_sampled": oracle.rel_l2(g.cpu().numpy()[idx],
                                                   oracle.nudft_fwd(c.astype(complex), y, idx)),
               "adj_rel_l2_sampled": oracle.rel_l2(a.cpu().numpy()[kdx],
                                                   oracle.nudft_adj(gin.astype(complex), y, N, kdx))}
    except Exception as e:
        acc = repr(e)
    return {"workload": "forward + adjoint NUFFT, N=M=2^24, complex64, uniform y, mixed eps=1e-6",
            "ms": ms, "value": 2 * M / (ms / 1e3), "unit": "points/s", "params": info,
            "tuning": tuned, "stage_roofline": stage_roofline(per, N, M, info, 8, 1, 1, peaks),
            "accuracy": acc}


def run_adaptive(steps: int = 10, warmup: int = 3, tune_params: bool = True):
    """Forward and adjoint NUFFT on clustered points, N = M = 2^20,
    complex64, mixed eps = 1e-6: the uniform tree against the adaptive tree
    (NUFFT_ADAPTIVE, leaves refined where they hold more points than the
    mean), both with the parameters the autotuner picks for the uniform tree
    on these points, and the adaptive tree on a base one level coarser; for
    the eight-cluster mixture and for clusters of four widths over a uniform
    background."""
    import torch

    import paper_1611_09379_gb300 as nf
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    N = M = 1 << 20
    c = workloads.coeffs(N, seed=61).astype(np.complex64)
    gin = workloads.samples(M, seed=64).astype(np.complex64)
    cd, gd = torch.from_numpy(c).cuda(), torch.from_numpy(gin).cuda()
    out = {"workload": "forward and adjoint NUFFT, N=M=2^20, complex64, mixed eps=1e-6, "
                       "clustered y", "unit": "points/s", "cases": {}}
    for kind, seed in (("clustered", 62), ("multiscale", 63)):
        y = workloads.points(kind, M, seed=seed)
        yd = torch.from_numpy(y).cuda()
        prm = {}
        case = {}
        if tune_params:
            from paper_1611_09379_gb300 import tune
            ent = tune.autotune(N, yd, 1e-6, prec=nf.MIXED, io="c64", ops="fwd+adj", reps=3,
                                tag=kind)
            prm = {k: ent["params"][k] for k in ("lmax", "p", "q", "tc_level", "tc_near")}
            case["tuning_s"] = ent["seconds"]
        variants = (("uniform_tree", False, 0), ("adaptive_tree", True, 0),
                    ("adaptive_tree_coarser_base", True, -1))
        for name, ad, dl in variants:
            pv = dict(prm)
            if dl and pv:
                pv["lmax"] = pv["lmax"] + dl
            elif dl:
                continue
            try:
                plan = nf.Plan(N, yd, eps=1e-6, prec=nf.MIXED, io="c64", adaptive=ad, **pv)
            except nf.NufftError as e:  # e.g. a leaf of the coarser base over the binning's cap
                case[name] = {"refused": str(e), "params": pv}
                continue
            g = torch.empty(M, dtype=torch.complex64, device="cuda")
            a = torch.empty(N, dtype=torch.complex64, device="cuda")
            fwd = _timed(lambda: plan.forward(cd, out=g), flush, stream, steps, warmup)
            adj = _timed(lambda: plan.adjoint(gd, out=a), flush, stream, steps, warmup)
            per = {}
            for op, fn in (("fwd", lambda: plan.forward(cd, out=g)),
                           ("adj", lambda: plan.adjoint(gd, out=a))):
                plan.profile(True)
                _timed(fn, flush, stream, 3, 0)
                per[op] = {k: round(v[0] / 3, 4) for k, v in plan.stats().items() if v[1]}
                plan.profile(False)
            lv, cnt = plan.adaptive()
            r = {"fwd_ms": fwd, "adj_ms": adj, "fwd_value": M / (fwd / 1e3),
                 "adj_value": M / (adj / 1e3), "levels": lv, "class_counts": cnt,
                 "fwd_stage_ms": per["fwd"], "adj_stage_ms": per["adj"], "params": plan.params()}
            try:
                import oracle
                idx = workloads.sample_index(M, 64, seed=7)
                kdx = workloads.sample_index(N, 64, seed=9)
                r["fwd_rel_l2_sampled"] = oracle.rel_l2(
                    g.cpu().numpy()[idx], oracle.nudft_fwd(c.astype(complex), y, idx))
                r["adj_rel_l2_sampled"] = oracle.rel_l2(
                    a.cpu().numpy()[kdx], oracle.nudft_adj(gin.astype(complex), y, N, kdx))
            except Exception as e:
                r["rel_l2_sampled"] = repr(e)
            case[name] = r
            del plan
        out["cases"][kind] = case
    return out


def _first_below(hist, every, iters, level):
    for i, v in enumerate(hist):
        if v <= level:
            return min((i + 1) * every, iters)
    return None


def run_lsq(budget_s: float = 50.0, full: bool = False, check_every: int = 32):
    """Least-squares INUFFT (N = 2^16, M = 2^18, 1:100 contrast, complex128,
    consistent samples of a random band-limited c_true): CG with the shipped
    learned density compensation and plain CG, both stopped on the same test
    (the unweighted normal-equation residual, recomputed from the iterate,
    <= 1e-8).  Plan and weights outside the timed solves.  Within `budget_s`
    both solves get the same iteration cap (from a timed probe solve); each
    reports its time, iterations, final residual and the iterations at which
    the residual first fell below 1e-2, 1e-4, 1e-6, 1e-8.  full=True runs both
    to 1e-8 (about two minutes)."""
    import torch

    import paper_1611_09379_gb300 as nf
    from paper_1611_09379_gb300 import dcf
    N, M = 1 << 16, 1 << 18
    y = workloads.points("contrast", M, seed=1234)
    c_true = workloads.coeffs(N, seed=99)
    plan = nf.Plan(N, torch.from_numpy(y).cuda(), eps=1e-10)
    g = plan.forward(torch.from_numpy(c_true).cuda())
    mlp = dcf.load()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    w = dcf.weights(plan, mlp)
    torch.cuda.synchronize()
    t_w = time.perf_counter() - t0
    # iteration time from a short solve, then the common cap
    probe = 64
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan.solve_lsq(g, None, tol=1e-30, maxit=probe, check=False, check_every=check_every)
    torch.cuda.synchronize()
    t_it = (time.perf_counter() - t0) / probe
    maxit = 60000 if full else max(256, int(budget_s / 2 / t_it))
    out = {"workload": "least-squares INUFFT N=2^16 M=2^18 1:100 density contrast, complex128, FP64 FMM "
                       "eps=1e-10", "tol": 1e-8, "stopping_test": "||A^H (g - A c)|| / ||A^H g|| "
                       "recomputed from c every %d iterations (same for both)" % check_every,
           "plan": plan.info(), "weights_s": t_w, "ms_per_iteration_probe": 1e3 * t_it,
           "iteration_cap": maxit}
    for name, ww in (("learned", w), ("plain", None)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c, it, res = plan.solve_lsq(g, ww, tol=1e-8, maxit=maxit, check=False, check_every=check_every)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        info = plan.lsq_info
        hist = info["history"]
        err = float(torch.linalg.vector_norm(c - torch.from_numpy(c_true).cuda()) /
                    torch.linalg.vector_norm(torch.from_numpy(c_true).cuda()))
        out[name] = {"iterations": it, "converged": res <= 1e-8, "residual": res,
                     "residual_weighted": info["resid_w"], "data_residual": info["data_resid"],
                     "solve_s": dt, "ms_per_iteration": 1e3 * dt / max(it, 1),
                     "iterations_to": {f"{lv:.0e}": _first_below(hist, info["check_every"], it, lv)
                                       for lv in (1e-2, 1e-4, 1e-6, 1e-8)},
                     "coef_rel_err_vs_c_true": err}
    L, P = out["learned"], out["plain"]
    out["learned_over_plain"] = {
        "iterations_to_1e-6": (L["iterations_to"]["1e-06"] / P["iterations_to"]["1e-06"]
                               if L["iterations_to"]["1e-06"] and P["iterations_to"]["1e-06"] else None),
        "residual_at_cap": L["residual"] / P["residual"] if P["residual"] > 0 else None,
        "solve_s": L["solve_s"] / P["solve_s"]}
    plan.close()
    return out


def run_eps_scan(logs=(8, 10, 12, 14, 16, 18, 20, 22),
                 epss=(1e-4, 1e-6, 1e-8, 1e-10, 1e-12, 1e-13, 1e-14, 1e-15, 0.0)):
    """Accuracy floor of the FP64 path (Sec. 3.1's threshold error eps_th(N)
    for this implementation): for N = M = 2^L, uniform points, and each
    prescribed eps (0 = the library's machine-precision mode), the paper's
    analytic test (f = 1, eps_a = max_j |g_j - 1| over all M points), the
    relative L2 error of a random band-limited signal against the oracle on
    256 sampled targets, the forward time, and the parameters Eq. 18.2 gave."""
    import torch

    import oracle
    import paper_1611_09379_gb300 as nf
    stream = torch.cuda.current_stream()
    out = {}
    for L in logs:
        N = M = 1 << L
        y = workloads.points("uniform", M, seed=500 + L)
        yd = torch.from_numpy(y).cuda()
        e0 = torch.zeros(N, dtype=torch.complex128, device="cuda")
        e0[0] = 1.0
        c = workloads.coeffs(N, seed=L)
        cd = torch.from_numpy(c).cuda()
        idx = workloads.sample_index(M, 256, seed=L)
        gref = oracle.nudft_fwd(c, y, idx)
        row = {}
        for eps in epss:
            try:
                plan = nf.Plan(N, yd, eps=eps, prec=nf.FP64)
            except nf.NufftError as e:
                row[repr(eps)] = {"error": str(e)}
                continue
            g1 = plan.forward(e0)
            ea = float((g1 - 1.0).abs().max())
            g = plan.forward(cd)
            torch.cuda.synchronize()
            err = oracle.rel_l2(g.cpu().numpy()[idx], gref)
            ms = []
            for _ in range(5):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                plan.forward(cd, out=g)
                b.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            row[repr(eps)] = {"eps_a_f1": ea, "rel_l2": err, "ms": sorted(ms)[2], **plan.params()}
            plan.close()
        out[N] = row
    return out


def cpu_oracle_sample(c, y, budget_s: float = 15.0):
    import oracle
    probe = workloads.sample_index(y.size, 16, seed=7)
    t0 = time.perf_counter()
    oracle.nudft_fwd(c, y, probe)
    per_target = max((time.perf_counter() - t0) / probe.size, 1e-6)
    k = int(min(max(16, budget_s / per_target), 8192))
    idx = workloads.sample_index(y.size, k, seed=11)
    t0 = time.perf_counter()
    oracle.nudft_fwd(c, y, idx)
    dt = time.perf_counter() - t0
    return {"value": idx.size / dt, "unit": "points/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"direct forward NUDFT (Eq. p1, O(N) per target) on {idx.size} sampled targets of "
                      f"the N=M=2^20 workload, {dt:.1f} s; the inverse oracle needs all O(N^2) "
                      f"log-sums and is not sampled"}


# ---------------------------------------------------------------- reference arm (the oracle)

def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    oracle.build()
    N = M = 1 << N_LOG2
    y = workloads.points("jitter", M, N, seed=1234, jitter=JITTER)
    c = workloads.coeffs(N, seed=99)
    per_step = 64  # targets per step: a bounded sample of the workload
    times = []
    for i in range(args.warmup + args.steps):
        idx = workloads.sample_index(M, per_step, seed=100 + i)
        t0 = time.perf_counter()
        oracle.nudft_fwd(c, y, idx)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = per_step / (ms / 1e3)
    out = {
        "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (same seeds as the GPU arm)",
        "impl": "reference",
        "config": {"workload": "forward + square inverse NUFFT, N=M=2^20, complex128, jittered y, "
                               "mixed eps=1e-6", "N": N, "M": M},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": f"direct forward NUDFT on {per_step} sampled targets per step"},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-lsq", action="store_true",
                    help="skip the least-squares INUFFT, learned vs plain CG")
    ap.add_argument("--lsq-seconds", type=float, default=50.0,
                    help="time budget of the two least-squares solves (same iteration cap)")
    ap.add_argument("--lsq-full", action="store_true",
                    help="run both least-squares solves to the 1e-8 residual (~2 min)")
    ap.add_argument("--lsq-only", action="store_true", help="only the least-squares comparison")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched workloads")
    ap.add_argument("--no-tune", action="store_true",
                    help="use the formula parameters (Eq. 18.2, 25) instead of the autotuner's")
    ap.add_argument("--no-large", action="store_true", help="skip the 2^24 forward + adjoint")
    ap.add_argument("--only-mixed", action="store_true",
                    help="time the mixed-precision arm only (for profiling; the FP64 keys then "
                         "repeat it)")
    ap.add_argument("--eps-scan", action="store_true",
                    help="only the FP64 accuracy-floor scan over N and eps (Sec. 3.1)")
    ap.add_argument("--no-adaptive", action="store_true",
                    help="skip the clustered transforms on the uniform and adaptive trees")
    ap.add_argument("--adaptive-only", action="store_true",
                    help="only the clustered transforms on the uniform and adaptive trees")
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched workloads (steps / warmup as given)")
    args = ap.parse_args()
    if args.eps_scan:
        print(json.dumps({"eps_scan": run_eps_scan()}))
        return
    if args.lsq_only:
        print(json.dumps({"inufft_lsq": run_lsq(args.lsq_seconds, args.lsq_full)}))
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.batched_only:
        print(json.dumps({"batched": run_batched(args.steps, args.warmup, not args.no_tune)}))
        return
    if args.adaptive_only:
        print(json.dumps({"adaptive_tree": run_adaptive(args.steps, args.warmup,
                                                        not args.no_tune)}))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
