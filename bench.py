#!/usr/bin/env python3
"""Benchmark: block-CGrQ time to solution per right-hand side on one GB300.

Workload (default): 32^4 lattice, m = 0.01, N = 16 complex128 Gaussian
sources, FP64-form block-CGrQ (double-float iterations, native-FP64 reliable
updates) to a true relative residual <= 1e-10, seeded synthetic links
(fat exp(0.3 i H), long -1/24 exp(0.3 i H')).  One step = one complete solve
(every stage of the hot path: stencil, Grams, small dense algebra, fused
streaming update, reliable updates).  Inputs (links 4.8 GB, block fields
~3.6 GB) are far larger than the 129 MB L2, so no flush is needed between
steps.

Also reported on the same line: the N independent CG baseline on the same
sources (Sec. 7.1), the mixed-precision form, the Dslash GB/s sweep over N
(Fig. 1 analogue), the roofline of the dominant kernel measured with CUDA
events inside the timed solves, the end-to-end time through the public API
with host buffers, and the CPU oracle timed on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: launched by torchrun, one independent replica per GPU (the
workload partitions into independent right-hand-side blocks; no collective).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "block-CG time-to-solution per RHS & Dslash HBM GB/s vs N independent CG, 1 GB300"
UNIT = "ms/RHS"
LINK_SEED = 1001
SRC_SEED = 2100
SM_COUNT = 152
FP32_LANES = 128
SM_MAX_MHZ = 2070.0
DF_INSTR_PER_FLOP = 6.0   # 12 FP32 instructions per double-float multiply-add (2 flops)
STENCIL_FLOPS = 1158      # per site per right-hand side (Sec. 6.2)
TC_VARIANT = 8192         # blockcg_params.dslash_variant flag of the tensor-core stencil
TC_PAIRS = 21             # bf16 slice products per double-float product (s + t <= 5)
TC_USEFUL = 6.0 / 8.0     # output columns of the n8 MMA tile the stencil uses
TC_TRAFFIC_32x4_N16 = 767.6e6 * 524288 / 165888  # ncu DRAM bytes at 24^4, scaled by sites


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dims", type=int, nargs=4, default=[32, 32, 32, 32])
    ap.add_argument("--mass", type=float, default=0.01)
    ap.add_argument("--nrhs", type=int, default=16)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--prec", default="f64")
    ap.add_argument("--no-extras", action="store_true", help="skip CG/mixed/sweep/CPU legs")
    ap.add_argument("--dslash-only", action="store_true",
                    help="only the stencil sweep (Fig. 1 analogue) for --prec over --sweep")
    ap.add_argument("--sweep", type=int, nargs="+", default=[1, 4, 8, 16, 32])
    ap.add_argument("--dslash-variant", type=int, default=0,
                    help="force a stencil kernel (blockcg_params.dslash_variant) for the "
                         "headline solve and --dslash-only; 0 = autotuned")
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched leg (64 small problems, one CUDA graph)")
    ap.add_argument("--autograd-only", action="store_true",
                    help="only the differentiable-solve leg (16^4, N = 8)")
    ap.add_argument("--legs", nargs="*", default=None,
                    help="run only these context legs (cg f64_native mixed dslash width "
                         "fine_tol many config3 batched autograd cpu)")
    return ap.parse_args()


def replica_source_seed(rank: int) -> int:
    """Replicas only: every rank solves its own block of right-hand sides
    (seed per rank); ranks share no data and no collective on the solve."""
    return SRC_SEED + 1000 * rank


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time (all_reduce MAX; NCCL on GPUs, gloo on CPU)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def per_rhs(elapsed_ms: float, steps: int, n_rhs: int, world: int) -> float:
    """Whole-job ms per right-hand side: all ranks' RHS in the slowest rank's time."""
    return elapsed_ms / (steps * n_rhs * world)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def workload_name(a):
    d = "x".join(str(x) for x in a.dims)
    return f"{d} m={a.mass} N={a.nrhs} {a.prec} block-CGrQ to {a.tol:g}"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        # samples under load: the upper half of the power readings
        pmed = statistics.median(power)
        loaded = [s for s, p in zip(sm, power) if p >= pmed] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- CPU oracle
def oracle_sample(dims, mass, fat, lng, b0, budget_s=12.0):
    """Seconds per textbook-CG iteration of the C oracle on one right-hand side,
    measured on a bounded number of iterations (the oracle as it stands)."""
    from oracle import hisq
    t = time.time()
    hisq.cg_iterates(dims, fat, lng, mass, b0, 2)
    per = max((time.time() - t) / 2, 1e-6)
    k = max(2, int(budget_s / per))
    t = time.time()
    hisq.cg_iterates(dims, fat, lng, mass, b0, k)
    return (time.time() - t) / k, k


def oracle_full_solves():
    """Whole oracle solves (textbook CG to 1e-10, host cores) on the small
    workloads: 4^4, m = 0.1, N = 4 and 16^4, m = 0.01, N = 1."""
    import hisq_inputs as hi
    from oracle import hisq
    res = {}
    for name, dims, mass, n in (("4^4 m=0.1 N=4", (4, 4, 4, 4), 0.1, 4),
                                ("16^4 m=0.01 N=1", (16, 16, 16, 16), 0.01, 1)):
        fat, lng = hi.random_links(dims, 1001)
        b = hi.gaussian_sources(dims, n, 2001)
        t = time.time()
        _, iters, rr = hisq.cg(dims, fat, lng, mass, b, tol=1e-10, max_iter=20000)
        res[name] = {"s": time.time() - t, "iters": [int(i) for i in iters],
                     "true_rel_res_max": float(max(rr))}
    return res


def golden_cg_iterations(a):
    p = os.path.join(ROOT, "tests", "golden", "cg_iters_32x4.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if list(d["dims"]) != list(a.dims) or abs(d["mass"] - a.mass) > 0 or abs(d["tol"] - a.tol) > 0:
        return None
    return d["iterations_mean"]


def cpu_inputs(a):
    import hisq_inputs as hi
    fat, lng = hi.random_links_torch(tuple(a.dims), LINK_SEED, "cpu")
    b = hi.gaussian_sources(tuple(a.dims), a.nrhs, SRC_SEED)
    return fat, lng, b


def run_reference(a):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    from oracle import build as obuild
    obuild.build()
    fat, lng, b = cpu_inputs(a)
    fat, lng = fat.numpy(), lng.numpy()
    iters = golden_cg_iterations(a)
    if iters is None:
        print(json.dumps({"impl": "reference", "unavailable":
                          "no oracle CG iteration count stored for this workload"}))
        return
    from oracle import hisq
    dims = tuple(a.dims)
    per_step = []
    for i in range(a.warmup + a.steps):
        t = time.time()
        k = 4
        hisq.cg_iterates(dims, fat, lng, a.mass, b[0], k)
        sec_per_it = (time.time() - t) / k
        if i >= a.warmup:
            per_step.append(sec_per_it)
    sec = statistics.mean(per_step)
    value = sec * iters * 1e3
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"{k} oracle textbook-CG iterations per step on 1 of the {a.nrhs} sources, "
              f"extrapolated to the oracle's {iters:.0f} iterations to {a.tol:g}")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": sec * 1e3 * k,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_name(a)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# -------------------------------------------------------------------- ours
def batched_leg(tol, dev, count=64):
    """Many small independent problems solved together (blockcg_batch_solve):
    one CUDA graph per chunk of iterations, against plain per-problem streams
    and against solving the problems one after another."""
    import torch
    import hisq_inputs as hi
    from paper_1710_09745_gb300 import BlockCG, BlockCGBatch
    specs = hi.batch_problems(count, seed=4000)
    solvers, Bs = [], []
    for sp in specs:
        fat, lng = hi.random_links_torch(sp["dims"], sp["link_seed"], dev)
        solvers.append(BlockCG(sp["dims"], fat, lng, sp["mass"], prec="mixed_f32",
                               max_rhs=sp["n_rhs"], device=dev))
        Bs.append(torch.as_tensor(hi.gaussian_sources(sp["dims"], sp["n_rhs"],
                                                      sp["source_seed"])).to(dev))
    batch = BlockCGBatch(solvers)
    batch.solve(Bs, tol=tol, graph=True)  # tuning and first captures
    _, ig, bg = batch.solve(Bs, tol=tol, graph=True)
    _, ip, bp = batch.solve(Bs, tol=tol, graph=False)
    seq = 0.0
    for s, B in zip(solvers, Bs):
        _, i = s.solve(B, tol=tol)
        seq += i["ms_total"]
    batch.close()
    nrhs = sum(sp["n_rhs"] for sp in specs)
    return {"workload": f"{count} problems L^4, L in {{8,12,16}}, m ~ U[0.01,0.2], N in 2..16 "
                        "(seed 4000), mixed FP32 to 1e-10",
            "rhs": nrhs, "graph_ms": bg["ms_total"], "streams_ms": bp["ms_total"],
            "sequential_ms": seq, "graph_ms_per_rhs": bg["ms_total"] / nrhs,
            "sequential_ms_per_rhs": seq / nrhs, "speedup_vs_sequential": seq / bg["ms_total"],
            "speedup_vs_streams": bp["ms_total"] / bg["ms_total"],
            "graph_replays": bg["graph_replays"], "graph_captures": bg["graph_captures"],
            "graph_nodes": bg["graph_nodes"], "chunk": bg["chunk"], "launches": bg["launches"],
            "all_converged": all(i["status"] == 0 for i in ig + ip),
            "true_rel_res_max": max(i["true_rel_res_max"] for i in ig)}


def autograd_leg(dev, tol=1e-10):
    """Differentiable solve: L = sum_i phi_i^dag A^-1 phi_i on 16^4, m = 0.05,
    N = 8 (F64 form); one forward + backward (two block solves and the
    link-gradient kernel), and the gradient kernel alone."""
    import torch
    import hisq_inputs as hi
    from paper_1710_09745_gb300 import BlockCG
    from paper_1710_09745_gb300.autograd import hisq_solve
    dims, mass, N = (16, 16, 16, 16), 0.05, 8
    fat, lng = hi.random_links_torch(dims, 1300, dev)
    s = BlockCG(dims, fat, lng, mass, prec="f64", max_rhs=N, device=dev)
    phi = torch.as_tensor(hi.gaussian_sources(dims, N, 1301)).to(dev)
    f = fat.clone().requires_grad_(True)
    l = lng.clone().requires_grad_(True)

    def step():
        f.grad = None
        l.grad = None
        x = hisq_solve(f, l, phi, s, tol=tol)
        (phi.conj() * x).sum().real.backward()
        return x

    x = step()  # tuning
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record(stream)
    for _ in range(reps):
        x = step()
    e1.record(stream)
    e1.synchronize()
    fb = e0.elapsed_time(e1) / reps
    xd = x.detach()
    s.link_grad(xd, xd)
    e0.record(stream)
    for _ in range(10):
        s.link_grad(xd, xd)
    e1.record(stream)
    e1.synchronize()
    lg = e0.elapsed_time(e1) / 10
    V = 16 ** 4
    # blockcg_link_grad runs in native FP64: two D_oe halves (1158 N flops per
    # site) and the outer products (2 link kinds x 4 V links x N x 9 entries x
    # 8 multiply-adds); its roof is the FP64 rate, not HBM
    from paper_1710_09745_gb300.binding import bench_alu
    _, fp64_fma, _ = bench_alu(stream)
    flops = 2 * STENCIL_FLOPS * N * (V // 2) + 2 * 2 * 4 * V * N * 9 * 8
    return {"workload": "16^4 m=0.05 N=8, L = sum phi^dag A^-1 phi, F64 form to 1e-10",
            "ms_forward_backward": fb, "ms_link_grad": lg,
            "link_grad_gbs": (2 * 2 * 6 * (V // 2) * N * 8 + 2 * 4 * V * 18 * 8) / (lg * 1e-3) / 1e9,
            "link_grad_fp64_tflops": flops / (lg * 1e-3) / 1e12,
            "link_grad_fp64_frac": flops / (lg * 1e-3) / (2 * fp64_fma),
            "grad_finite": bool(torch.isfinite(f.grad).all().item())}


def dslash_only(a):
    """Stencil GB/s per N for one precision (no solve); one JSON line."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1710_09745_gb300 import BlockCG
    dims = tuple(a.dims)
    Vh = int(np.prod(dims)) // 2
    fat, lng, _ = cpu_inputs(a)
    dev = torch.device("cuda", 0)
    h = BlockCG(dims, fat.to(dev), lng.to(dev), a.mass, prec=a.prec, max_rhs=max(a.sweep),
                dslash_variant=a.dslash_variant, device=dev)
    hbm_peak, _ = load_peaks()
    bpr = {"f64": 8, "f64_native": 8, "mixed_f32": 4, "mixed_f16": 2, "mixed_bf16": 2}[a.prec]
    rows = {}
    for n in a.sweep:
        ms = h.bench_dslash(n, reps=max(a.steps, 1) * 10)
        gbs = (288 + 12 * n) * bpr * Vh / (ms * 1e-3) / 1e9
        rows[str(n)] = {"ms": ms, "gbs": gbs, "hbm_frac": gbs / hbm_peak,
                        "gflops": STENCIL_FLOPS * n * Vh / (ms * 1e-3) / 1e9}
    print(json.dumps({"dslash": rows, "prec": a.prec, "dims": list(dims),
                      "dslash_variant": a.dslash_variant}))


def main():
    a = parse_args()
    if a.impl == "reference":
        run_reference(a)
        return
    if a.dslash_only:
        dslash_only(a)
        return
    if a.batched_only or a.autograd_only:
        import torch
        dev = torch.device("cuda", 0)
        leg = batched_leg(a.tol, dev) if a.batched_only else autograd_leg(dev)
        print(json.dumps({"batched" if a.batched_only else "autograd": leg}))
        return
    world, rank, local = dist_env()
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1710_09745_gb300 import BlockCG

    dims = tuple(a.dims)
    V = int(np.prod(dims))
    Vh = V // 2
    N = a.nrhs
    fat_c, lng_c, b_np = cpu_inputs(a)
    if world > 1:  # independent replica per rank: its own sources
        import hisq_inputs as hi
        b_np = hi.gaussian_sources(dims, N, replica_source_seed(rank))
    fat = fat_c.to(dev)
    lng = lng_c.to(dev)
    B = torch.as_tensor(b_np).to(dev)
    s = BlockCG(dims, fat, lng, a.mass, prec=a.prec, max_rhs=max(N, 32), profile=True,
                dslash_variant=a.dslash_variant, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # measured FP32 / FP64 multiply-add rates of this GPU (the double-float roofline's basis)
    from paper_1710_09745_gb300.binding import bench_alu, bench_mma
    alu_f32, alu_f64, alu_sms = bench_alu(stream)
    mma_bf16 = bench_mma(stream)
    for _ in range(a.warmup):
        X, info = s.solve(B, tol=a.tol)
    barrier()
    clk = ClockSampler()
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    infos = []
    e0.record(stream)
    for _ in range(a.steps):
        X, info = s.solve(B, tol=a.tol)
        infos.append(info)
    e1.record(stream)
    barrier()
    clocks = clk.stop()
    elapsed = max_over_ranks(e0.elapsed_time(e1), world, dev)
    ms_per_step = elapsed / a.steps
    value = per_rhs(elapsed, a.steps, N, world)
    ok = all(i["status"] == 0 and i["true_rel_res_max"] <= a.tol for i in infos)

    # dominant kernel: the iteration's stencil, timed with events inside the solves
    n_st = sum(i["n_stencil"] for i in infos)
    ms_st = sum(i["ms_stencil"] for i in infos)
    ms_total = sum(i["ms_total"] for i in infos)
    avg_launch_ms = ms_st / max(n_st, 1)
    hbm_peak, peak_src = load_peaks()
    bytes_per_real = {"f64": 8, "f64_native": 8, "mixed_f32": 4, "mixed_f16": 2, "mixed_bf16": 2}[a.prec]
    alg_bytes = (288 + 12 * N) * bytes_per_real * Vh
    alg_flops = STENCIL_FLOPS * N * Vh
    variant = infos[-1]["stencil_variant"]
    hbm_view = {"achieved_gbs": alg_bytes / (avg_launch_ms * 1e-3) / 1e9, "peak_gbs": hbm_peak,
                "frac": alg_bytes / (avg_launch_ms * 1e-3) / 1e9 / hbm_peak}
    if a.prec == "f64" and (variant & TC_VARIANT) and N in (16, 32):
        # the tensor-core stencil: 6 chunks x 21 split products (m16n8k16, 4096 flops,
        # 6 of 8 output columns used) per site and 16 right-hand sides
        issued = 6 * 21 * (N // 16) * 4096.0 * Vh
        peak = mma_bf16 * TC_USEFUL / TC_PAIRS / 1e12
        achieved = alg_flops / (avg_launch_ms * 1e-3) / 1e12
        full = tuple(dims) == (32, 32, 32, 32) and N == 16
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": TC_TRAFFIC_32x4_N16 if full else None,
                "traffic_note": "ncu DRAM read+write of one k_dslash_tc launch at 24^4 N=16 "
                                "(767.6 MB, 1.21x its algorithmic bytes), scaled by sites to "
                                "32^4; profiles/k_dslash_tc_df_24x4_N16.md" if full else None,
                "kernel": "k_dslash_tc (tensor-core double-float stencil)",
                "peak_note": "FP64-equivalent rate of the split-product scheme: measured "
                             "mma.sync bf16 rate (blockcg_bench_mma, this run) x 6/8 used "
                             "output columns / 21 slice products per double-float product",
                "tensor_issued": {"tflops": issued / (avg_launch_ms * 1e-3) / 1e12,
                                  "mma_sync_peak_tflops": mma_bf16 / 1e12,
                                  "frac": issued / (avg_launch_ms * 1e-3) / mma_bf16},
                "ncu": {"profile": "profiles/k_dslash_tc_df_24x4_N16.md (24^4, N = 16)",
                        "tensor_pipe_active": 0.216, "issue_slots_active": 0.584,
                        "dram_throughput": 0.146, "warps_active": 0.243},
                "hbm_view": hbm_view,
                "share_of_solve": ms_st / ms_total if ms_total else None,
                "launches": n_st, "avg_launch_ms": avg_launch_ms, "variant": variant}
    elif a.prec == "f64":
        peak = SM_COUNT * FP32_LANES * SM_MAX_MHZ * 1e6 / DF_INSTR_PER_FLOP / 1e12
        achieved = alg_flops / (avg_launch_ms * 1e-3) / 1e12
        # ncu dram__bytes_read.sum + dram__bytes_write.sum of one 32^4 N=16 launch of the
        # tuned double-float stencil (k_dslash_async<StoreDF, 2, 1, 0, 3>), 2.0x the
        # algorithmic bytes; only that workload and kernel version
        full = tuple(dims) == (32, 32, 32, 32) and N == 16
        measured_peak = alu_f32 / DF_INSTR_PER_FLOP / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": 4.04e9 if full else None,
                "traffic_note": "ncu DRAM read+write of one k_dslash_async<StoreDF,2,1,0,3> "
                                "launch at 32^4 N=16 (algorithmic 2.013e9; "
                                "profiles/k_dslash_df_traffic_32x4_N16.md)" if full else None,
                "kernel": "k_dslash<StoreDF> (double-float stencil)",
                "peak_note": "FP32 issue rate 152 SM x 128 lanes x 2070 MHz / 6 instr per "
                             "FP64-equivalent flop (double-float: 12 FP32 instructions per "
                             "multiply-add); derived from unit counts and the maximum clock",
                "peak_measured": measured_peak,
                "frac_of_measured": achieved / measured_peak,
                "alu_probe": {"fp32_fma_per_s": alu_f32, "fp64_fma_per_s": alu_f64,
                              "sm_count": alu_sms,
                              "note": "blockcg_bench_alu in this run (FMA chains, 8 blocks of "
                                      "256 threads per SM); profiles/alu_issue_rates.md"},
                "ncu": {"profile": "profiles/k_dslash_df_24x4_N16.md (24^4, N = 16, same kernel)",
                        "issue_slots_active": 0.809, "fma_pipe_active": 0.681,
                        "dram_throughput": 0.195, "achieved_occupancy": 0.287},
                "hbm_view": hbm_view,
                "share_of_solve": ms_st / ms_total if ms_total else None,
                "launches": n_st, "avg_launch_ms": avg_launch_ms, "variant": variant}
    else:
        achieved = alg_bytes / (avg_launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None, "peak_source": peak_src,
                "share_of_solve": ms_st / ms_total if ms_total else None,
                "launches": n_st, "avg_launch_ms": avg_launch_ms}

    # end to end through the public API with host buffers
    B_host = torch.as_tensor(b_np).pin_memory()
    X_host = torch.empty_like(B_host).pin_memory()
    B_dev = torch.empty_like(B)
    X_dev = torch.empty_like(B)
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    barrier()
    e2.record(stream)
    for _ in range(a.steps):
        B_dev.copy_(B_host, non_blocking=True)
        X_dev.zero_()  # initial guess 0, solved in place
        Xd, _ = s.solve(B_dev, tol=a.tol, out=X_dev)
        X_host.copy_(Xd, non_blocking=True)
    e3.record(stream)
    barrier()
    e2e_ms = max_over_ranks(e2.elapsed_time(e3), world, dev)
    nbytes = B_host.numel() * B_host.element_size()
    e2e = {"value": per_rhs(e2e_ms, a.steps, N, world), "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"f64": "f64(double-float)", "f64_native": "f64", "mixed_f32": "f32+f64",
                  "mixed_f16": "f16+f32+f64", "mixed_bf16": "bf16+f32+f64"}[a.prec],
        "data": "synthetic",
        "config": {"workload": workload_name(a), "dims": list(dims), "mass": a.mass, "n_rhs": N,
                   "tol": a.tol, "prec": a.prec, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (no flush)",
                   "links": f"torch-cpu seed {LINK_SEED}", "sources": f"numpy seed {SRC_SEED}"},
        "clocks": clocks, "e2e": e2e,
        "gpu_launches": int(sum(i["launches"] for i in infos)),
        "roofline": roof,
        "solve": {"iters": infos[-1]["iters"], "reliable_updates": infos[-1]["reliable_updates"],
                  "true_rel_res_max": infos[-1]["true_rel_res_max"], "converged": ok,
                  "ms_breakdown": {k: sum(i[k] for i in infos) / a.steps for k in
                                   ("ms_stencil", "ms_stencil_fine", "ms_gram", "ms_stream",
                                    "ms_dense", "ms_total")}},
    }

    forms = {"f64": "iteration fields P, Q, AP, T, update X and links in double-float (FP32 "
                     "hi+lo pairs, ~48 significant bits) with error-free double-float arithmetic "
                     "on the FP32 pipes; reliable updates (Y, B, R, FP64 stencil, QR of R) and "
                     "all N x N algebra in native FP64",
             "f64_native": "native FP64 storage and arithmetic everywhere (the plain-FP64 form)",
             "mixed_f32": "sloppy P, Q, AP, T and links in FP32 with FP32 arithmetic; X in "
                          "double-float; native-FP64 reliable updates and N x N algebra",
             "mixed_f16": "as mixed_f32 with FP16 storage (2^4-scaled) and a reliable update "
                          "every 10 iterations"}
    out["forms"] = forms
    out["solve"]["true_rel_res"] = infos[-1]["true_rel_res"]

    def extras():
        """Context legs beside the headline line (outside the timed region)."""
        col0 = {"f64": X[0].cpu().numpy()}  # column 0 of each form's solution (oracle error)

        def leg(name, fn):
            """A context leg beside the headline (outside the timed region); its
            failure is recorded in the line instead of losing the line."""
            if a.legs and name not in a.legs:
                return
            try:
                fn()
            except Exception as exc:
                out.setdefault("leg_errors", {})[name] = f"{type(exc).__name__}: {exc}"

        def free_cuda():
            import gc
            gc.collect()
            torch.cuda.empty_cache()

        def cg_leg():
            # N independent CG solves on the same sources (Sec. 7.1 baseline)
            _, ic = s.solve_cg(B, tol=a.tol)
            out["cg_baseline"] = {"ms_per_rhs": ic["ms_total"] / N, "iters_per_rhs": ic["iters"] / N,
                                  "true_rel_res_max": ic["true_rel_res_max"],
                                  "block_speedup": (ic["ms_total"] / N) / value,
                                  "per_rhs_iteration_ratio": (value / out["solve"]["iters"]) /
                                  ((ic["ms_total"] / N) / (ic["iters"] / N)),
                                  "stencil_avg_launch_ms": ic["ms_stencil"] / max(ic["n_stencil"], 1)}

        def form_leg(key, prec, n_cg):
            """One solver form on the headline workload: block CGrQ (tuned
            first, then one timed solve) and n_cg independent CG solves."""
            sf = BlockCG(dims, fat, lng, a.mass, prec=prec, max_rhs=max(N, 32), profile=True,
                         device=dev)
            sf.tune(N)
            Xf, im = sf.solve(B, tol=a.tol)
            _, imc = sf.solve_cg(B[:n_cg], tol=a.tol)
            col0[prec] = Xf[0].cpu().numpy()
            ms_rhs = im["ms_total"] / N
            cg_rhs = imc["ms_total"] / n_cg
            out[key] = {"ms_per_rhs": ms_rhs, "iters": im["iters"],
                        "reliable_updates": im["reliable_updates"],
                        "true_rel_res_max": im["true_rel_res_max"],
                        "true_rel_res": im["true_rel_res"],
                        "converged": im["status"] == 0 and im["true_rel_res_max"] <= a.tol,
                        "ms_breakdown": {k: im[k] for k in ("ms_stencil", "ms_stencil_fine",
                                                            "ms_gram", "ms_stream", "ms_dense",
                                                            "ms_total")},
                        "stencil_variant": im["stencil_variant"],
                        "cg_rhs": n_cg, "cg_ms_per_rhs": cg_rhs, "cg_iters_per_rhs": imc["iters"] / n_cg,
                        "cg_true_rel_res_max": imc["true_rel_res_max"],
                        "block_speedup": cg_rhs / ms_rhs,
                        "per_rhs_iteration_ratio": (ms_rhs / im["iters"]) /
                        (cg_rhs / (imc["iters"] / n_cg))}
            return sf

        def f64_native_leg():
            # the plain-FP64 form: block CGrQ vs independent CG, native FP64 throughout
            sf = form_leg("f64_native", "f64_native", 4)
            del sf
            free_cuda()

        handles = {}

        def mixed_legs():
            handles["mixed_f32"] = form_leg("mixed", "mixed_f32", 4)
            handles["mixed_f16"] = form_leg("mixed_f16", "mixed_f16", 4)
            # the best CG of any form as a baseline for the 16-bit block solve
            best = min(out[k]["cg_ms_per_rhs"] for k in ("mixed", "mixed_f16"))
            if "cg_baseline" in out:
                best = min(best, out["cg_baseline"]["ms_per_rhs"])
            out["mixed_f16"]["block_speedup_vs_best_cg"] = best / out["mixed_f16"]["ms_per_rhs"]

        def dslash_leg():
            # Dslash GB/s per N (Fig. 1 analogue) for each storage format; "f32r12":
            # FP32 with two-row links, its GB/s counted with 18 reals per link as
            # for the others (the method's bytes), so it can exceed the HBM copy rate
            s32 = handles.get("mixed_f32") or BlockCG(dims, fat, lng, a.mass, prec="mixed_f32",
                                                      max_rhs=32, device=dev)
            s16 = handles.get("mixed_f16") or BlockCG(dims, fat, lng, a.mass, prec="mixed_f16",
                                                      max_rhs=32, device=dev)
            s32r = BlockCG(dims, fat, lng, a.mass, prec="mixed_f32", max_rhs=32, link_recon=12,
                           device=dev)
            sweep = {}
            for n in (1, 4, 8, 16, 32):
                row = {}
                for name, h, bpr in (("f32", s32, 4), ("f32r12", s32r, 4), ("f16", s16, 2),
                                     ("df", s, 8)):
                    ms = h.bench_dslash(n, reps=10)
                    gbs = (288 + 12 * n) * bpr * Vh / (ms * 1e-3) / 1e9
                    row[name] = {"ms": ms, "gbs": gbs, "hbm_frac": gbs / hbm_peak,
                                 "gflops": STENCIL_FLOPS * n * Vh / (ms * 1e-3) / 1e9}
                sweep[str(n)] = row
            out["dslash"] = sweep

        def width_leg():
            # time to solution per RHS against the block width (F64 form, same
            # sources: the first n columns of a 32-column block)
            import hisq_inputs as hi
            b32 = torch.as_tensor(hi.gaussian_sources(dims, 32, SRC_SEED)).to(dev)
            sN = BlockCG(dims, fat, lng, a.mass, prec=a.prec, max_rhs=32, device=dev)
            width = {}
            for n in (1, 4, 8, 16, 32):
                sN.tune(n)
                _, iN = sN.solve(b32[:n], tol=a.tol)
                width[str(n)] = {"ms_per_rhs": iN["ms_total"] / n, "iters": iN["iters"],
                                 "reliable_updates": iN["reliable_updates"],
                                 "true_rel_res_max": iN["true_rel_res_max"]}
            out["block_width"] = width

        def many_leg():
            # 64 right-hand sides in blocks whose width the library picks by
            # timing its first blocks (blockcg_solve_many), F64 form
            import hisq_inputs as hi
            b64 = torch.as_tensor(hi.gaussian_sources(dims, 64, SRC_SEED + 7)).to(dev)
            sM = BlockCG(dims, fat, lng, a.mass, prec=a.prec, max_rhs=32, device=dev)
            _, im = sM.solve_many(b64, tol=a.tol)
            out["solve_many"] = {
                "workload": f"{'x'.join(map(str, dims))} m={a.mass} 64 RHS {a.prec} to {a.tol:g}",
                "chosen_width": im["width"], "from_cache": im["from_cache"],
                "candidates_ms_per_rhs": {str(k): v for k, v in im["candidates"].items()},
                "blocks": im["blocks"], "ms_per_rhs": im["ms_total"] / 64,
                "true_rel_res_max": im["true_rel_res_max"], "status": im["status"]}
            del sM, b64
            free_cuda()

        def fine_tol_leg():
            # the F64 form at the paper's fine tolerance, for the solution error
            # against the oracle (column 0; the oracle solves to the same 1e-12)
            X12, i12 = s.solve(B, tol=1e-12)
            col0["f64@1e-12"] = X12[0].cpu().numpy()
            out["f64_tol_1e-12"] = {"ms_per_rhs": i12["ms_total"] / N, "iters": i12["iters"],
                                    "true_rel_res_max": i12["true_rel_res_max"]}

        def config3_leg():
            """48^3 x 96, m = 0.01, N = 32 in the mixed forms: FP16 storage with a
            reliable update every 10 iterations, and FP32 storage beside it."""
            import hisq_inputs as hi
            d3, n3, m3 = (48, 48, 48, 96), 32, 0.01
            f3, l3 = hi.random_links_torch(d3, 1003, dev)
            b3 = hi.gaussian_sources_torch(d3, n3, 2300, dev)
            res = {"workload": "48x48x48x96 m=0.01 N=32 to 1e-10 (links seed 1003, sources seed "
                               "2300)"}
            for key, prec, kw in (("mixed_f16", "mixed_f16", {"ru_every": 10}),
                                  ("mixed_f32", "mixed_f32", {})):
                h3 = BlockCG(d3, f3, l3, m3, prec=prec, max_rhs=n3, max_iter=5000, profile=True,
                             device=dev, **kw)
                h3.tune(n3)
                _, i3 = h3.solve(b3, tol=a.tol)
                res[key] = {"ms_per_rhs": i3["ms_total"] / n3, "ms_per_solve": i3["ms_total"],
                            "iters": i3["iters"], "reliable_updates": i3["reliable_updates"],
                            "true_rel_res_max": i3["true_rel_res_max"],
                            "converged": i3["status"] == 0 and i3["true_rel_res_max"] <= a.tol,
                            "ms_breakdown": {k: i3[k] for k in ("ms_stencil", "ms_stencil_fine",
                                                                "ms_gram", "ms_stream", "ms_dense")}}
                del h3
                free_cuda()
            out["config_48x96"] = res
            del f3, l3, b3
            free_cuda()

        def cpu_leg():
            # CPU oracle (rank 0, one GPU): one whole textbook-CG solve of source 0
            # of the workload to tol on the host cores (the baseline, measured, not
            # extrapolated), continued to 1e-12 for the solution error of every
            # form's column 0 against the FP64 oracle
            os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
            from oracle import build as obuild
            obuild.build()
            from oracle import hisq as ohisq
            import numpy as np
            fat_n, lng_n = fat_c.numpy(), lng_c.numpy()
            cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
            t0 = time.time()
            x10, it10, rr10 = ohisq.cg(dims, fat_n, lng_n, a.mass, b_np[:1], tol=a.tol, max_iter=5000)
            sec10 = time.time() - t0
            t0 = time.time()
            x12, it12, rr12 = ohisq.cg(dims, fat_n, lng_n, a.mass, b_np[:1], tol=1e-12, max_iter=5000,
                                       x0=x10)
            sec12 = time.time() - t0
            ref = x12[0]
            nref = np.linalg.norm(ref)
            errs = {k: float(np.linalg.norm(v - ref) / nref) for k, v in col0.items()}
            t0 = time.time()
            ohisq.apply_A(dims, fat_n, lng_n, a.mass, b_np[:1])
            apply_ms = (time.time() - t0) * 1e3
            prev = ohisq.set_threads(1)  # the same oracle on one core, shorter sample
            sec_it1, k1 = oracle_sample(dims, a.mass, fat_n, lng_n, b_np[0], budget_s=4.0)
            ohisq.set_threads(prev)
            out["cpu_baseline"] = {
                "value": sec10 * 1e3, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"one whole oracle textbook-CG solve of source 0 of the workload to "
                          f"{a.tol:g} ({int(it10[0])} iterations, {sec10:.1f} s, true residual "
                          f"{float(rr10[0]):.2e}) on {cores} host threads",
                "one_core": {"value": sec_it1 * int(it10[0]) * 1e3, "unit": UNIT, "cores": 1,
                             "sample": f"{k1} iterations ({sec_it1 * 1e3:.1f} ms each) x "
                                       f"{int(it10[0])}"},
                "apply_A_ms_per_rhs": apply_ms,
                "full_solves": oracle_full_solves()}
            out["oracle_error"] = {
                "what": "|x_0 - x_0^oracle| / |x_0^oracle| for column 0 of each form's solution; "
                        f"oracle = textbook CG in FP64 to 1e-12 ({int(it10[0] + it12[0])} iterations, "
                        f"true residual {float(rr12[0]):.2e})",
                "errors": errs,
                "bound_note": "|e|/|x| <= kappa |r|/|b|, kappa = lambda_max / m^2 ~ 4.3e4 at "
                              "m = 0.01: <= ~4e-6 at a 1e-10 residual, ~4e-8 at 1e-12"}

        leg("cg", cg_leg)
        leg("f64_native", f64_native_leg)
        leg("mixed", mixed_legs)
        leg("dslash", dslash_leg)
        handles.clear()
        free_cuda()
        leg("width", width_leg)
        leg("fine_tol", fine_tol_leg)
        leg("many", many_leg)
        leg("config3", config3_leg)
        leg("batched", lambda: out.__setitem__("batched", batched_leg(a.tol, dev)))
        leg("autograd", lambda: out.__setitem__("autograd", autograd_leg(dev)))
        if world == 1:
            leg("cpu", cpu_leg)

    if rank == 0 and not a.no_extras:
        extras()

    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
