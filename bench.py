"""Benchmark: eigenpairs/s at residual <= 1e-10 for the RF-DDES interface-filter solver.

One step = one full solve (quadrature, bordered-block factorisations, Schur complements, block
Lanczos on the interface filter, interior basis, Rayleigh-Ritz, completion passes) of the
workload, with the pencil already set up on the device (``value``).  ``e2e`` measures the same
metric through the C ABI with host buffers: setup (host->device upload), solve, and the copy of
eigenvalues, eigenvectors and residuals back to the host, every step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torch.distributed.run, one independent replica per GPU (the path does not
shard across GPUs here), value = eigenpairs of all ranks / max over ranks of the time.
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import rfdd_inputs as I  # noqa: E402

METRIC = "eigenpairs/s at residual<=1e-10, mixed vs FP64 plain, 1 GB300; p50/p99 latency"
UNIT = "eigenpairs/s"
WORKLOAD = "q1_3d_40"


def workload_config(w, precision):
    grid = tuple(w.grid) if w.grid is not None else (w.n,)
    splits = tuple(w.meta.get("splits", ())) if isinstance(w.meta, dict) else ()
    dims = "x".join(str(g) for g in grid)
    parts = "x".join(str(q) for q in splits) if splits else str(w.p)
    return {
        "workload": f"{len(grid)}D Q1 Laplacian pencil, {dims} interior grid (n={w.n}), {parts} geometric "
                    f"partition (p={w.p}), eigenvalues {w.meta['first']}..{w.meta['last']} "
                    f"(nev={w.expected_nev}), {w.n_nodes} {w.rule.replace('_', '-')} nodes",
        "name": w.name, "n": w.n, "p": w.p, "nev": w.expected_nev, "n_nodes": w.n_nodes,
        "interval": [w.alpha, w.beta], "precision": precision,
        "l2": "no flush: every step streams the bordered factors (tens of GB) through HBM, far above L2",
    }


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, max clock, throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
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
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        try:
            sm = [float(r[1]) for r in rows]
            mx = max(float(r[2]) for r in rows)
        except ValueError:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows)}


# DRAM traffic of the dominant kernel (tc_gemm_kernel).  A whole solve is far too large to capture
# under ncu, so the traffic is measured on one launch of the same kernel on a small case (a deep
# trailing-update shape: C = 8192 x 8192 complex, k = 256, about 1.1 GB on the device):
#   python bench.py --mode gemm --gemm 8192 8192 256 && \
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none -k regex:tc_gemm \
#       -s 1 -c 1 --csv --log-file tc_traffic_gemm.csv python bench.py --mode gemm --gemm 8192 8192 256
# and divided by the launch's compulsory bytes from the kernel's traffic model (C read and written
# once, packed operand tiles read once; rfdd_profile_bytes).  That launch runs the two-CTA kernel,
# which carries most of the GEMM time of a solve.  The full solve's traffic per launch is
# that ratio times the model bytes of the timed launches.  The ratio holds for the kernel's code as
# captured, so it is used only while the kernel's sources hash to the value below.
TC_TRAFFIC_RATIO = 1.06470        # measured / model DRAM bytes of the captured launch (1.2504e9 / 1.1744e9)
TC_TRAFFIC_KERNEL_SOURCES = ("common.cuh", "dense.cuh", "tc_gemm.cuh", "tc_gemm.cu")
TC_TRAFFIC_SOURCES_SHA256 = "3c32a42ad93bccff46d196a20bde6467e99a4a109be881d03eca494d025cc31c"


def kernel_sources_sha256(names=TC_TRAFFIC_KERNEL_SOURCES) -> str:
    import hashlib
    root = os.path.join(ROOT, "paper_1711_09487_gb300", "csrc")
    h = hashlib.sha256()
    for name in names:
        h.update(name.encode())
        with open(os.path.join(root, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def tc_traffic_per_launch(model_bytes_per_launch: float):
    """DRAM bytes per launch of the timed launches, or None while the captured ratio does not
    describe the kernel being timed."""
    if TC_TRAFFIC_RATIO is None or kernel_sources_sha256() != TC_TRAFFIC_SOURCES_SHA256:
        return None
    return TC_TRAFFIC_RATIO * model_bytes_per_launch


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


# --------------------------------------------------------------------------------------------
# CPU oracle sample (reference arm and cpu_baseline)
# --------------------------------------------------------------------------------------------

def oracle_sample(w, budget_s: float = 20.0):
    """Times the FP64 oracle's a2-a5 work (dense LU of B_j(zeta) plus the Schur update
    E_j^T B_j^{-1} E_j) on subdomain 0 at the first node, and extrapolates the oracle's whole
    factorisation phase (all subdomains x nodes, plus LU of every S(zeta)) by the flop model.
    Returns (estimated eigenpairs/s upper bound, sample seconds, description, threads)."""
    import scipy.linalg as sla
    from oracle import rfdd_oracle as O
    blk = O.Blocks(w.A.to_scipy(), w.M.to_scipy(), w.part, w.p)
    z, _ = O.quadrature(w.alpha, w.beta, w.n_nodes, w.rule)
    j = 0
    Bz = blk.B[j] - z[0] * blk.MB[j]
    Ez = (blk.E[j] - z[0] * blk.ME[j])[:, blk.sidx[j]]
    t0 = time.perf_counter()
    lu = sla.lu_factor(Bz)
    X = sla.lu_solve(lu, Ez)
    _ = Ez.T @ X
    t = time.perf_counter() - t0

    def work(d, sj):  # complex multiply-adds: LU d^3/3, two triangular solves d^2 sj, product d sj^2
        return d ** 3 / 3.0 + d * d * sj + d * sj * sj

    sample = work(blk.d[j], len(blk.sidx[j]))
    total = sum(work(blk.d[q], len(blk.sidx[q])) for q in range(blk.p)) * w.n_nodes + w.n_nodes * blk.s ** 3 / 3.0
    t_total = t * total / sample
    threads = os.cpu_count()
    try:
        from threadpoolctl import threadpool_info
        threads = max((i.get("num_threads", 0) for i in threadpool_info()), default=threads) or threads
    except Exception:
        pass
    desc = (f"oracle a2-a5 for subdomain 0 at node 0 (dense complex128 LU of {blk.d[j]}x{blk.d[j]} + Schur update "
            f"with {len(blk.sidx[j])} columns) = 1/{total / sample:.0f} of the factorisation work; value = nev / "
            f"extrapolated factorisation time (an upper bound on the oracle's full-solve throughput)")
    return w.expected_nev / t_total, t, desc, threads


def run_reference(args, rank, world):
    w = I.workload(args.workload)
    if rank != 0:
        return
    vals = []
    for i in range(args.warmup + args.steps):
        v, t, desc, threads = oracle_sample(w)
        if i >= args.warmup:
            vals.append((v, t))
    value = statistics.median(v for v, _ in vals)
    ms = statistics.median(t for _, t in vals) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": workload_config(w, "fp64-oracle"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------------
# multi-rank aggregation (one process per GPU, independent replicas)
# --------------------------------------------------------------------------------------------

def reduce_over_ranks(ms: float, units: float, dist, device) -> tuple[float, float]:
    """Whole-job figures of N replicas: the max over ranks of the timed milliseconds and the sum
    over ranks of the units (eigenpairs) processed.  ``dist`` is torch.distributed with an
    initialised process group (nccl on the GPU, gloo in the CPU tests)."""
    import torch
    mx = torch.tensor([ms], dtype=torch.float64, device=device)
    sm = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[0])


# --------------------------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------------------------

def run_fp64_plain(R, w, stream, ev_ref=None):
    """One solve of the workload on the plain FP64 path (FP64 factorisations and solves, no
    refinement needed), timed with CUDA events on its stream: eigenpairs with residual <= 1e-10
    per second, and how far its eigenvalues are from the mixed solve's."""
    import torch
    opts = R.rfdd_default_options(precision=R.RFDD_FP64, quad_rule=0 if w.rule == "midpoint" else 1,
                                  stream=stream.cuda_stream)
    h = R.rfdd_setup(w.A, w.M, w.part, w.p, opts)
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    r = R.rfdd_solve(h, w.alpha, w.beta, w.n_nodes)
    s1.record(stream)
    s1.synchronize()
    ms = s0.elapsed_time(s1)
    ev, _, rs = R.rfdd_result_get(r, vectors=False)
    info = R.rfdd_result_info(r)
    good = int(np.count_nonzero(rs <= 1e-10))
    out = {"value": good / (ms / 1e3), "unit": UNIT, "ms": ms, "eigenpairs": good,
           "max_resid": float(rs.max()) if len(rs) else None, "dtype": "c128",
           "phases_ms": {k: info[k] for k in ("t_factor_ms", "t_lanczos_ms", "t_interior_ms", "t_rr_ms",
                                               "t_complete_ms")}}
    if ev_ref is not None and len(ev_ref) == len(ev) and len(ev):
        out["max_rel_diff_vs_mixed"] = float(np.max(np.abs(ev - ev_ref) / np.abs(ev)))
    if w.exact is not None and len(ev):
        ex = w.exact[(w.exact > w.alpha) & (w.exact < w.beta)]
        if len(ex) == len(ev):
            out["max_rel_err_vs_closed_form"] = float(np.max(np.abs(ev - ex) / ex))
    del r, h
    return out


def oracle_model_check():
    """The flop model behind cpu_baseline, checked on the small 2D Q1 40^2 workload: the oracle's
    whole solve timed against the model's extrapolated factorisation time for the same workload."""
    from oracle import rfdd_oracle as O
    w1 = I.workload("q1_2d_40")
    t0 = time.perf_counter()
    O.rfdd_solve(w1.A.to_scipy(), w1.M.to_scipy(), w1.part, w1.p, w1.alpha, w1.beta, w1.n_nodes, w1.rule)
    full = time.perf_counter() - t0
    v, _, _, _ = oracle_sample(w1)
    model = w1.expected_nev / v
    return {"workload": w1.name, "full_oracle_solve_s": full, "model_factorisation_s": model,
            "full_over_model": full / model}


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1711_09487_gb300 as R

    torch.cuda.set_device(local_rank)
    R.load()
    dist = None
    if world > 1:
        import torch.distributed as dist
    w = I.workload(args.workload)
    precision = R.RFDD_MIXED if args.precision == "mixed" else R.RFDD_FP64
    stream = torch.cuda.Stream()
    opts = R.rfdd_default_options(precision=precision, quad_rule=0 if w.rule == "midpoint" else 1,
                                  stream=stream.cuda_stream)
    h = R.rfdd_setup(w.A, w.M, w.part, w.p, opts)

    def one_step():
        r = R.rfdd_solve(h, w.alpha, w.beta, w.n_nodes)
        return r, R.rfdd_result_info(r)

    # warm-up
    for _ in range(args.warmup):
        r, info = one_step()
        del r
    torch.cuda.synchronize()
    good_per_step = []
    lat = []
    clocks = ClockSampler(local_rank)
    R.rfdd_profile(True)
    launches0 = R.rfdd_kernel_launches()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        r, info = one_step()
        s1.record(stream)
        s1.synchronize()
        lat.append(s0.elapsed_time(s1))
        r_last_evals, _, rs_h = R.rfdd_result_get(r, vectors=False)
        good_per_step.append(int(np.count_nonzero(rs_h <= 1e-10)))
        del r
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = R.rfdd_kernel_launches() - launches0
    ms_total = e0.elapsed_time(e1)
    g_launch, g_ms, g_flops = R.rfdd_profile_get(0)
    t_launch, t_ms, t_flops = R.rfdd_profile_get(1)
    g_busy, t_busy = R.rfdd_profile_busy(0), R.rfdd_profile_busy(1)
    t_model_bytes = R.rfdd_profile_bytes(1)
    R.rfdd_profile(False)
    good = sum(good_per_step)
    if dist:
        ms_total, good = reduce_over_ranks(ms_total, good, dist, "cuda")
    value = good / (ms_total / 1e3)

    # end to end through the C ABI with host buffers (rank-local)
    e2e_times, h2d, d2h = [], 0, 0
    for _ in range(max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2 = R.rfdd_setup(w.A, w.M, w.part, w.p, opts)
        r2 = R.rfdd_solve(h2, w.alpha, w.beta, w.n_nodes)
        ev2, X2, rs2 = R.rfdd_result_get(r2)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        good2 = int(np.count_nonzero(rs2 <= 1e-10))
        h2d = (w.A.rowptr.nbytes + w.A.col.nbytes + w.A.val.nbytes + w.M.rowptr.nbytes + w.M.col.nbytes +
               w.M.val.nbytes + w.part.nbytes)
        d2h = ev2.nbytes + X2.nbytes + rs2.nbytes
        del r2, h2
    e2e_s, e2e_good = statistics.median(e2e_times), float(good2)
    if dist:
        e2e_ms, e2e_good = reduce_over_ranks(e2e_s * 1e3, e2e_good, dist, "cuda")
        e2e_s = e2e_ms / 1e3
    e2e_value = e2e_good / e2e_s

    # the plain FP64 path on the same workload (the metric's comparison arm): one solve, timed with
    # CUDA events on its stream, residual bar as for the mixed steps
    fp64 = None
    if args.fp64_plain == "on" or (args.fp64_plain == "auto" and world == 1 and precision == R.RFDD_MIXED):
        fp64 = run_fp64_plain(R, w, stream, ev_ref=r_last_evals)
    # the serving pattern on a short stream (the full 256-request stream: --mode serve)
    serving = None
    if args.serve_requests > 0 and world == 1:
        serving = serve_stream(R, args.serve_requests, args.load, args.inflight, min(4, args.capacity_sample))
        serving.pop("metric", None)
    if rank != 0:
        return
    peaks, src = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    # dominant kernel: complex-FP32 GEMM of the factorisations and triangular solves
    # Time basis: the union of the launches' CUDA-event intervals.  The real interior
    # factorisation runs on a second stream during the complex factorisations, so some GEMM
    # launches of the two streams run at the same time; the union counts that time once (with
    # no overlap it is the plain sum of the launch durations, also reported).
    if t_launch > 0:
        # achieved: the method's algorithmic complex flops (4M count, 8 real flops per complex
        # multiply-add) per second of busy time; peak: the TF32 tensor peak (measured sustained
        # bf16 x the nominal TF32/bf16 ratio 1.1/2.25), the rate of the unit the contraction runs on
        ach = t_flops / (t_busy / 1e3) / 1e12
        peak = float(peaks["bf16_tflops_sustained"]) * (1.1 / 2.25)
        traffic = tc_traffic_per_launch(t_model_bytes / t_launch)
        roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": traffic,
                "traffic_unit": "DRAM bytes per launch (model bytes x measured/model ratio of one captured launch)",
                "model_bytes_per_launch": t_model_bytes / t_launch,
                # executed tensor work: the realified complex product issues exactly the 4M count
                # of real multiply-adds, each as three TF32 products (3xTF32 split)
                "executed_tflops": 3.0 * ach, "executed_frac": 3.0 * ach / peak,
                "kernel": "tcgen05 3xTF32 complex GEMM", "launches": t_launch,
                "busy_ms": t_busy, "launch_ms_sum": t_ms,
                "peak_source": f"{src} bf16 sustained x 1.1/2.25 (TF32 tensor)"}
    else:
        ach = g_flops / (g_busy / 1e3) / 1e12 if g_busy > 0 else 0.0
        peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "kernel": "SIMT complex-FP32 GEMM (gemm_simt_kernel)", "launches": g_launch,
                "busy_ms": g_busy, "launch_ms_sum": g_ms,
                "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz ({src} max clock)"}
    # throughput probes of the units this path is bound by (context for the peaks above)
    probes = {}
    for name, which in (("tf32_mma_tflops", 0), ("fp64_fma_tflops", 1), ("fp32_fma_tflops", 2),
                        ("tf32_gemm_8192_tflops", 3)):
        try:
            probes[name] = R.rfdd_peak_probe(which)
        except Exception as ex:  # a probe is context, not part of the measurement
            probes[name] = f"failed: {ex}"
    if t_launch > 0 and isinstance(probes.get("tf32_mma_tflops"), float):
        # the same achieved rate against the tensor pipe's TF32 rate measured here (burst, MMAs from
        # shared memory): the stricter denominator when it exceeds the derived peak
        roof["probe_peak_tf32"] = probes["tf32_mma_tflops"]
        roof["frac_vs_probe"] = roof["achieved"] / probes["tf32_mma_tflops"]
        roof["executed_frac_vs_probe"] = roof["executed_tflops"] / probes["tf32_mma_tflops"]
    cpu_value, cpu_t, cpu_desc, cpu_threads = oracle_sample(w)
    model_check = oracle_model_check()
    lat_sorted = sorted(lat)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "c64+f64" if precision == R.RFDD_MIXED else "c128",
        "data": "synthetic", "config": workload_config(w, args.precision),
        "latency_ms": {"p50": lat_sorted[len(lat_sorted) // 2],
                       "p99": lat_sorted[min(len(lat_sorted) - 1, int(math.ceil(0.99 * len(lat_sorted))) - 1)]},
        "eigenpairs_per_step": good_per_step[-1], "solve_info": info,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roof,
        "cpu_baseline": {"value": cpu_value, "unit": UNIT, "cores": cpu_threads, "kind": "oracle",
                         "sample": cpu_desc, "model_check": model_check},
        "probes": probes,
        # the tile-shape autotuner's classes after the run: complex/real, K-depth and size buckets,
        # the kept kernel (0 one-CTA, 1 two-CTA) and each kernel's mean ms per GFLOP
        "autotune": [[e["complex"], e["kbucket"], e["tbucket"], e["winner"]] + e["ms_per_gflop"]
                     for e in R.rfdd_autotune_table()],
        "clocks": clk,
    }
    if fp64 is not None:
        line["fp64_plain"] = fp64
        line["mixed_over_fp64"] = value / fp64["value"] if fp64["value"] > 0 else None
    if serving is not None:
        line["serving"] = serving
    print(json.dumps(line), flush=True)


def run_one_solve(args):
    """One untimed solve of the workload (the command profiled for the kernel launch list)."""
    import torch
    import paper_1711_09487_gb300 as R
    torch.cuda.set_device(0)
    R.load()
    w = I.workload(args.workload)
    precision = R.RFDD_MIXED if args.precision == "mixed" else R.RFDD_FP64
    h = R.rfdd_setup(w.A, w.M, w.part, w.p,
                     R.rfdd_default_options(precision=precision, quad_rule=0 if w.rule == "midpoint" else 1))
    r = R.rfdd_solve(h, w.alpha, w.beta, w.n_nodes)
    info = R.rfdd_result_info(r)
    print(json.dumps({"mode": "one-solve", "workload": w.name, "precision": args.precision,
                      "eigenpairs_per_s": info["nev"] / (info["t_total_ms"] * 1e-3), "solve_info": info}), flush=True)


def run_compare(args):
    """RF-DDES (Algorithm 3 + completion) against RF-KRYLOV (Algorithm 1 + the same completion) on
    one workload, both on the same factorisation code and precision: the paper's comparison
    (Section 6.3: Krylov dimensions, accuracy before completion, time), here on one GPU."""
    import torch
    import paper_1711_09487_gb300 as R
    torch.cuda.set_device(0)
    R.load()
    w = I.workload(args.workload)
    precision = R.RFDD_MIXED if args.precision == "mixed" else R.RFDD_FP64
    stream = torch.cuda.Stream()
    extra = {} if args.nev_b is None else {"nev_b": args.nev_b}
    opts = R.rfdd_default_options(precision=precision, quad_rule=0 if w.rule == "midpoint" else 1,
                                  stream=stream.cuda_stream, **extra)
    h = R.rfdd_setup(w.A, w.M, w.part, w.p, opts)
    ex = w.exact[(w.exact > w.alpha) & (w.exact < w.beta)] if w.exact is not None else None
    out = {"mode": "compare", "workload": w.name, "n": w.n, "p": w.p, "n_nodes": w.n_nodes,
           "nev": w.expected_nev, "nev_b": opts.nev_b, "precision": args.precision, "steps": args.steps,
           "warmup": args.warmup}
    for name, call in (("rf_ddes", lambda: R.rfdd_solve(h, w.alpha, w.beta, w.n_nodes)),
                       ("rf_krylov", lambda: R.rfdd_rfkrylov(h, w.alpha, w.beta, w.n_nodes))):
        for _ in range(args.warmup):
            call()
        times, info, pre, good = [], None, None, 0
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = call()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            info = R.rfdd_result_info(r)
            pre = np.sort(R.rfdd_result_pre_evals(r))
            ev, _, rs = R.rfdd_result_get(r, vectors=False)
            good = int(np.count_nonzero(rs <= 1e-10))
            del r
        ms = statistics.median(times)
        d = {"eigenpairs_per_s": good / (ms / 1e3), "ms_median": ms, "eigenpairs": good,
             "krylov_dim": info["mu"], "rr_rank": info["k"], "passes": info["passes"],
             "max_resid": info["max_resid"], "status": info["status"], "fp64_basis": info["fp64_basis"],
             "phases_ms": {k: info[k] for k in ("t_factor_ms", "t_lanczos_ms", "t_interior_ms", "t_rr_ms",
                                                 "t_complete_ms")}}
        if ex is not None and len(pre) == len(ex) and len(ex):
            d["pre_completion_max_rel_err"] = float(np.max(np.abs(pre - ex) / np.abs(ex)))
        else:
            d["pre_completion_count"] = int(len(pre))
        if ex is not None and len(ev) == len(ex) and len(ex):
            d["final_max_rel_err"] = float(np.max(np.abs(np.sort(ev) - ex) / np.abs(ex)))
        out[name] = d
    out["ddes_over_krylov"] = out["rf_ddes"]["eigenpairs_per_s"] / max(out["rf_krylov"]["eigenpairs_per_s"], 1e-300)
    print(json.dumps(out), flush=True)


def run_levels(args):
    """Dense against two-level interface factorisation (rfdd_set_interface_groups) on one
    workload: factor-phase time, the device bytes of the factors, and whole solves, both
    completed to residual <= 1e-10 (median of --steps after --warmup)."""
    import torch
    import paper_1711_09487_gb300 as R
    torch.cuda.set_device(0)
    R.load()
    w = I.workload(args.workload)
    precision = R.RFDD_MIXED if args.precision == "mixed" else R.RFDD_FP64
    splits = w.meta["splits"]
    gs = tuple(int(x) for x in args.group_splits.split(",")) if args.group_splits else \
        tuple(max(1, k // 2) for k in splits)
    groups = I.subdomain_groups(splits, gs)
    stream = torch.cuda.Stream()
    extra = {} if args.nev_b is None else {"nev_b": args.nev_b}
    opts = R.rfdd_default_options(precision=precision, quad_rule=0 if w.rule == "midpoint" else 1,
                                  stream=stream.cuda_stream, **extra)
    h = R.rfdd_setup(w.A, w.M, w.part, w.p, opts)
    ex = w.exact[(w.exact > w.alpha) & (w.exact < w.beta)] if w.exact is not None else None
    _, _, s = R.rfdd_layout(h)
    out = {"mode": "levels", "workload": w.name, "n": w.n, "p": w.p, "s": s, "n_nodes": w.n_nodes,
           "nev": w.expected_nev, "nev_b": opts.nev_b, "precision": args.precision, "group_splits": list(gs),
           "steps": args.steps, "warmup": args.warmup}
    for name, grp in (("dense", None), ("two_level", groups)):
        R.rfdd_set_interface_groups(h, grp)
        cls, s2 = R.rfdd_interface_levels(h)
        mem = R.rfdd_memory_estimate(h, w.n_nodes, int(w.expected_nev or 100))
        for _ in range(args.warmup):
            R.rfdd_solve(h, w.alpha, w.beta, w.n_nodes)
        times, infos, good, err = [], [], 0, None
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = R.rfdd_solve(h, w.alpha, w.beta, w.n_nodes)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            infos.append(R.rfdd_result_info(r))
            ev, _, rs = R.rfdd_result_get(r, vectors=False)
            good = int(np.count_nonzero(rs <= 1e-10))
            if ex is not None and len(ev) == len(ex) and len(ex):
                err = float(np.max(np.abs(np.sort(ev) - ex) / np.abs(ex)))
            del r
        ms = statistics.median(times)
        tf = statistics.median(i["t_factor_ms"] for i in infos)
        d = {"eigenpairs_per_s": good / (ms / 1e3), "ms_median": ms, "eigenpairs": good, "t_factor_ms": tf,
             "memory_estimate_bytes": mem, "s2": s2, "level1": int(np.count_nonzero(cls >= 0)),
             "krylov_dim": infos[-1]["mu"], "passes": infos[-1]["passes"], "max_resid": infos[-1]["max_resid"],
             "status": infos[-1]["status"], "final_max_rel_err": err,
             "phases_ms": {k: infos[-1][k] for k in ("t_factor_ms", "t_lanczos_ms", "t_interior_ms", "t_rr_ms",
                                                      "t_complete_ms")}}
        out[name] = d
    out["two_level_over_dense"] = out["two_level"]["eigenpairs_per_s"] / max(out["dense"]["eigenpairs_per_s"], 1e-300)
    out["factor_speedup"] = out["dense"]["t_factor_ms"] / max(out["two_level"]["t_factor_ms"], 1e-300)
    print(json.dumps(out), flush=True)


def run_gemm(args):
    """One large complex GEMM C -= A B (m x k times k x n) on the tensor cores: the shape of the
    deep trailing updates of the factorisations (profiled alone with ncu)."""
    import paper_1711_09487_gb300 as R
    R.load()
    m, n, k = args.gemm
    g = np.random.default_rng(0)
    A = (g.standard_normal((m, k)) + 1j * g.standard_normal((m, k))).astype(np.complex64)
    B = (g.standard_normal((k, n)) + 1j * g.standard_normal((k, n))).astype(np.complex64)
    C = np.zeros((m, n), dtype=np.complex64)
    R.rfdd_cgemm(A, B, C, -1.0, 1.0, args.engine)  # warm-up
    R.rfdd_profile(True)
    R.rfdd_cgemm(A, B, C, -1.0, 1.0, args.engine)
    launches, ms, flops = R.rfdd_profile_get(1)
    model_bytes = R.rfdd_profile_bytes(1)
    R.rfdd_profile(False)
    print(json.dumps({"mode": "gemm", "m": m, "n": n, "k": k, "engine": args.engine, "kernel_ms": ms,
                      "model_bytes": model_bytes,
                      "tflops_4m": flops / (ms / 1e3) / 1e12 if ms > 0 else None}), flush=True)


def run_dgemm(args):
    """One Gram-type product C = Y^T Y (Y: k x n FP64, all output tiles formed) in the double-FP32
    arithmetic of the basis products (the Rayleigh-Ritz Gram shape; profiled alone with ncu)."""
    import paper_1711_09487_gb300 as R
    R.load()
    n, _, k = args.gemm
    Y = np.random.default_rng(0).standard_normal((k, n))
    C0 = np.zeros((n, n))
    R.rfdd_dgemm(Y, Y, C0, 1.0, 0.0, True, False, 1, False)  # warm-up
    R.rfdd_profile(True)
    R.rfdd_dgemm(Y, Y, C0, 1.0, 0.0, True, False, 1, False)
    launches, ms, flops = R.rfdd_profile_get(0)
    R.rfdd_profile(False)
    print(json.dumps({"mode": "dgemm", "n": n, "k": k, "kernel_ms": ms,
                      "fp64_equiv_tflops": flops / (ms / 1e3) / 1e12 if ms > 0 else None}), flush=True)


def run_serve(args):
    """The serving pattern on its own (bench.py --mode serve): prints the serve_stream() line."""
    import torch
    import paper_1711_09487_gb300 as R
    torch.cuda.set_device(0)
    R.load()
    print(json.dumps(serve_stream(R, args.requests, args.load, args.inflight, args.capacity_sample)), flush=True)


def serve_stream(R, requests, load, inflight, capacity_sample):
    """The serving pattern: a seeded Poisson stream of requests of mixed size and kind (2-D Q1 and
    3-D variable-coefficient pencils, 20..400 eigenvalues each, p in {4, 8, 16}, 8 nodes), each
    bringing its pencil, served by the library's continuous-batching server under a 150 GiB memory
    budget.  The arrival rate is `load` times the single-stream capacity, measured first on the
    stream's first requests run one at a time.  Returns eigenpairs/s (residual <= 1e-10) over the
    stream and the p50/p99 latency from arrival to result."""
    reqs = I.serving_stream(requests, seed=7)
    pencils = [I.serving_pencil(q) for q in reqs]          # built before any clock starts
    opts = R.rfdd_default_options(precision=R.RFDD_MIXED)
    budget = 150 << 30

    def submit(srv, q, pc):
        A, M, part, p = pc
        return srv.submit_pencil(A, M, part, p, q["alpha"], q["beta"], q["n_nodes"], nev_hint=q["nev"], opts=opts)

    # single-stream capacity: the first requests one at a time (after one warm-up request)
    k = min(capacity_sample, len(reqs))
    srv1 = R.Server(max_inflight=1, mem_budget=budget)
    r = srv1.wait(submit(srv1, reqs[0], pencils[0]))
    del r
    run_ms = []
    for q, pc in zip(reqs[:k], pencils[:k]):
        rid = submit(srv1, q, pc)
        r = srv1.wait(rid)
        run_ms.append(srv1.request_info(rid)["latency_ms"])
        del r
    srv1.close()
    capacity = 1000.0 / statistics.mean(run_ms)            # requests per second, one at a time
    rate = load * capacity
    gaps = np.random.default_rng(7).exponential(1.0 / rate, len(reqs))
    arrival = np.cumsum(gaps) - gaps[0]

    srv = R.Server(max_inflight=inflight, mem_budget=budget)
    ids, t_sub = [None] * len(reqs), [0.0] * len(reqs)
    t0 = time.perf_counter()
    for i, (q, pc) in enumerate(zip(reqs, pencils)):
        dt = t0 + arrival[i] - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        ids[i] = submit(srv, q, pc)
        t_sub[i] = time.perf_counter()
    good, wrong_count, lat, done_at = 0, 0, [], []
    per_kind, statuses, wrong = {}, {}, []
    for i, q in enumerate(reqs):
        r = srv.wait(ids[i])
        ev, _, rs = R.rfdd_result_get(r, vectors=False)
        info = srv.request_info(ids[i])
        rinfo = R.rfdd_result_info(r)
        del r
        g = int(np.count_nonzero(rs <= 1e-10))
        good += g
        statuses[str(info["status"])] = statuses.get(str(info["status"]), 0) + 1
        if len(ev) != q["nev"]:
            wrong_count += 1
            if len(wrong) < 24:
                wrong.append({"i": i, "kind": q["kind"], "N": q["N"], "splits": list(q["splits"]), "expected": q["nev"],
                              "got": len(ev), "good": g, "status": info["status"], "passes": rinfo["passes"],
                              "pre_nev": rinfo["pre_nev"], "max_resid": rinfo["max_resid"]})
        t_done = t_sub[i] - t0 + info["latency_ms"] / 1e3      # seconds after the first arrival
        done_at.append(t_done)
        lat.append((t_done - arrival[i]) * 1e3)
        k_ = per_kind.setdefault(q["kind"], {"requests": 0, "eigenpairs": 0})
        k_["requests"] += 1
        k_["eigenpairs"] += g
    st = srv.stats()
    srv.close()
    wall = max(done_at)
    lat_s = sorted(lat)
    line = {"mode": "serve", "metric": METRIC, "value": good / wall, "unit": UNIT, "requests": len(reqs),
            "eigenpairs": good, "wall_s": wall, "latency_ms": {
                "p50": lat_s[len(lat_s) // 2],
                "p99": lat_s[min(len(lat_s) - 1, int(math.ceil(0.99 * len(lat_s))) - 1)],
                "max": lat_s[-1]},
            "arrival_rate_per_s": rate, "load": load, "single_stream_capacity_per_s": capacity,
            "capacity_sample_requests": k, "max_inflight": inflight, "mem_budget_bytes": budget,
            "requests_with_wrong_count": wrong_count, "wrong_count_sample": wrong, "statuses": statuses,
            "per_kind": per_kind, "server": st,
            "config": {"workload": "serving stream: seeded Poisson arrivals, 50% 2D Q1 N in 64..256, 50% 3D "
                                   "variable-kappa 7-point N in 24..48, 20..400 eigenvalues, p in {4,8,16}, 8 nodes",
                       "seed": 7, "precision": "mixed"}}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mode", default="bench", choices=["bench", "one-solve", "gemm", "dgemm", "serve", "compare", "levels"])
    ap.add_argument("--requests", type=int, default=256, help="serve mode: requests in the stream")
    ap.add_argument("--load", type=float, default=0.7, help="serve mode: arrival rate / single-stream capacity")
    ap.add_argument("--inflight", type=int, default=4, help="serve mode: requests running at once")
    ap.add_argument("--capacity-sample", type=int, default=8, help="serve mode: requests timed one at a time")
    ap.add_argument("--serve-requests", type=int, default=24,
                    help="bench mode: requests of a short serving stream reported beside the solve line (0: none)")
    ap.add_argument("--gemm", type=int, nargs=3, default=[8192, 8192, 128], metavar=("M", "N", "K"))
    ap.add_argument("--engine", type=int, default=1, choices=[1, 2, 3],
                    help="gemm mode: 1 automatic kernel choice, 2 one-CTA kernel, 3 two-CTA kernel")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--group-splits", default=None,
                    help="levels mode: subdomain blocks per group along each axis, e.g. 2,2,2 "
                         "(default: half the subdomain splits)")
    ap.add_argument("--nev-b", type=int, default=None,
                    help="compare mode: eigenvectors per subdomain in the RF-DDES basis (default 100)")
    ap.add_argument("--fp64-plain", default="auto", choices=["auto", "on", "off"],
                    help="also time one solve on the plain FP64 path (auto: at N = 1 with --precision mixed)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.mode == "one-solve":
        run_one_solve(args)
        return
    if args.mode == "gemm":
        run_gemm(args)
        return
    if args.mode == "dgemm":
        run_dgemm(args)
        return
    if args.mode == "serve":
        run_serve(args)
        return
    if args.mode == "compare":
        run_compare(args)
        return
    if args.mode == "levels":
        run_levels(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
