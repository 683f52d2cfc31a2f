#!/usr/bin/env python
"""Benchmark: vertices+edges per second of edge-subdivision extraction.

Workload: the D=3 torus network (3-64-64-64-64-1, fitted to a torus SDF) on the
box [-1,1]^3, mixed precision (FP32 values, FP64 coordinates / t / filtered
sign predicates), one full extraction per step.  Inputs (the network
parameters) are resident in device memory when the timed region starts; the
L2 cache is flushed (a 512 MiB write) before every step, outside the step's
CUDA events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The JSON line (the last line on stdout) also carries the FP64 mode and the
pruned (level-set) extraction on the same workload (`variants`), the
rooflines of the neuron loop and of the tensor-core layer products on the
D=5 width-40 counting-sweep net, where HBM can bind (`large`; `--large 0`
skips it), and, last, the serving measurement (`serving`: a Poisson stream
of 2000 extraction requests through the batched server and the plain 1-slot
path; `--serve-requests 0` skips it).  Longer side measurements go to stderr,
one JSON line each: the counting sweep of Section 5.1.2 (random
four-hidden-layer nets of widths 10, 20, 40 for D = 1..5, five nets per
point; `--sweep-dims ''` skips it), the same net on a simplex domain
(`--domain 0` skips it) and the width-10 sweep nets for D = 6..10
(`--sweep-dims-w10 ''` skips it).

--impl reference times the FP64 CPU oracle as the reference arm
on the host cores.  Under torchrun (N > 1) every rank runs an independent
replica on its own GPU (the extraction does not shard); rank 0 prints one JSON
line with the whole-job throughput.
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
sys.path.insert(0, ROOT)

# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) per launch,
# averaged over the launches of one steady-state mixed-precision extraction,
# and a hash of the kernel sources they were taken with: the figures are
# reported only while the sources are unchanged (else traffic is null).
#   k_layer_torus      the D=3 torus workload, 5 k_layer launches
#   k_layer_d5w40      the D=5 width-40 counting-sweep net (seed 0), 5 launches
#   k_gemm_tc2_d5w40   the same net's 4 tensor-core layer products
KERNEL_DRAM = {"sources_sha16": "6e6aa921f3306f5b", "k_layer_torus": 231117670, "k_layer_d5w40": 30457925529,
               "k_gemm_tc2_d5w40": 1235692544}
KERNEL_SOURCES = ("pc_phases.cuh", "pc_core.cu", "pc_device.cuh", "pc_newton.cuh", "pc_gemm_tc.cu", "pc_polish.cu")

METRIC = "vertices+edges/s at D=3 (torus 3-64x4-1, box [-1,1]^3)"
UNIT = "(V+E)/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _workload():
    from paper_2306_07212_gb300 import workloads
    net, box = workloads.torus_d3()
    return net, box, {"workload": "torus SDF net D=3, MLP 3-64x4-1, box [-1,1]^3, one full extraction per step"}


# -- clocks -------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "0x1") or val == "Active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# -- algorithmic bytes of the neuron loop -------------------------------------

def kernel_traffic(key: str, precision: str) -> dict:
    """The captured DRAM bytes per launch (KERNEL_DRAM), or null when the
    kernel sources changed since the capture or the precision differs."""
    if precision == "mixed" and KERNEL_DRAM["sources_sha16"] == kernel_sources_sha16() and KERNEL_DRAM[key]:
        return {"traffic": KERNEL_DRAM[key],
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, averaged over the "
                                  "launches of one steady-state extraction of this workload"}
    return {"traffic": None, "traffic_source": "not captured for these kernel sources"}


def kernel_sources_sha16() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2306_07212_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def neuron_loop_bytes(net, stats, precision: str) -> list:
    """Algorithmic bytes of the per-neuron steps, per layer (one k_layer launch each).

    Per neuron step with V vertices, E edges, S splitting edges, K 2-face
    keys and P paired faces (the per-neuron counters):
      4 V                          the neuron's value row (zb bytes per value)
      8 E                          every edge's two endpoints
      S (3 (8D + zb H + 8W) + 16)  two endpoint records read and the new
                                   vertex's written (coordinates, the layer's
                                   H values, W sign words), 16 B of edges
      24 K                         each key's 12-byte slot written and read
      8 P                          each intersecting edge written
    zb = 4 (FP32 values) or 8 (FP64); W = 64-bit words per sign vector.
    Sign-word gathers and error scales are not counted (cache-resident).
    """
    D = net.D
    zb = 8 if precision == "fp64" else 4
    W = (2 * D + net.n_neurons + 31) // 32
    out, n = [], 0
    for l in range(net.L):
        H = net.widths[l + 1]
        tot = 0
        for _ in range(H):
            V, E, S, K, P = (int(stats[n, k]) for k in (0, 1, 2, 3, 4))
            tot += zb * V + 8 * E + S * (3 * (8 * D + H * zb + 8 * W) + 16) + 24 * K + 8 * P
            n += 1
        out.append(tot)
    return out


def gemm_bytes_flops(net, stats, precision: str) -> list:
    """Per layer l >= 1 (the tensor-core product): algorithmic bytes (read the
    previous layer's values and the vertices' sign words, write this layer's
    values) and useful flops 2 V H_{l-1} H_l, with V the vertices at the layer
    start."""
    zb = 8 if precision == "fp64" else 4
    W = (2 * net.D + net.n_neurons + 31) // 32
    out, off = [], 0
    for l in range(net.L):
        H, K = net.widths[l + 1], net.widths[l]
        V = int(stats[off, 0])
        out.append((zb * V * (K + H) + 8 * W * V, 2.0 * V * K * H))
        off += H
    return out


def measure_tf32_tflops(device: int) -> float:
    """Dense TF32 matmul rate of this GPU (torch.matmul, 8192^3, FP32 inputs
    with TF32 tensor cores allowed), best of 5 after a warm-up."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        n = 8192
        a = torch.randn(n, n, device=device)
        b = torch.randn(n, n, device=device)
        torch.matmul(a, b)
        best = 0.0
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            e1.synchronize()
            best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) / 1e3) / 1e12)
        del a, b
        return round(best, 1)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


# -- replicas: whole-job numbers --------------------------------------------

def max_over_ranks(seconds: float, dist=None) -> float:
    """The slowest rank's time (the job ends when the last replica does)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return seconds
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_step: int, steps: int, world: int, seconds: float) -> float:
    """Units all replicas processed (each the same workload) per second of the slowest."""
    return units_per_step * steps * world / seconds


# -- our arm -------------------------------------------------------------------

def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2306_07212_gb300 import Extractor

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    net, box, config = _workload()
    dev = torch.device("cuda", local_rank)
    params_dev = torch.from_numpy(net.flat_params()).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ex = Extractor(device=local_rank, precision=args.precision, execution=args.execution, timers=True)
    for _ in range(args.warmup):
        ex.extract(net, box, params=params_dev)
    c = ex.counts()
    units = c["nV"] + c["nE"]
    stats = ex.stats()
    layer_bytes = neuron_loop_bytes(net, stats, args.precision)
    launches0 = ex.diagnostics()["launches"]

    clocks = ClockSampler(local_rank)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, loop_ms, gemm_ms = [], [], []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ex.extract(net, box, params=params_dev)
        e1.record()
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        kt = ex.kernel_times_ms()
        loop_ms.append(kt[:, 1].copy())
        gemm_ms.append(kt[:, 0].copy())
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = ex.diagnostics()["launches"] - launches0
    assert ex.counts()["nV"] + ex.counts()["nE"] == units
    total_s = sum(step_ms) / 1e3
    total_s = max_over_ranks(total_s, dist)

    # end to end through the C ABI with host buffers: parameters from pinned
    # host memory each step, the complex copied back to pinned host memory
    params_host = torch.from_numpy(net.flat_params()).pin_memory()
    S = c["S"]
    Xh = torch.empty((c["D"], c["nV"]), dtype=torch.float64).pin_memory()
    Eh = torch.empty((2, c["nE"]), dtype=torch.int32).pin_memory()
    Sh = torch.empty((S, c["nV"]), dtype=torch.int64).pin_memory()
    lib, ctx = ex._lib, ex._ctx
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ex.extract(net, box, params=params_host)
        ex._check(lib.pc_vertices(ctx, None, None, Xh.data_ptr()))
        ex._check(lib.pc_edges(ctx, None, None, Eh.data_ptr()))
        ex._check(lib.pc_signvectors(ctx, None, None, Sh.data_ptr()))
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist)
    h2d = params_host.numel() * 8
    d2h = Xh.numel() * 8 + Eh.numel() * 4 + Sh.numel() * 8

    loop_avg = np.mean(np.stack(loop_ms), axis=0)  # per layer, ms
    gemm_avg = np.mean(np.stack(gemm_ms), axis=0)
    peak, peak_kind = _peaks()
    roofline = loop_roofline(layer_bytes, loop_avg, peak, peak_kind)
    roofline["share_of_step"] = round(float(loop_avg.sum() / statistics.mean(step_ms)), 3)
    roofline["forward_product_ms_per_step"] = round(float(gemm_avg.sum()), 4)
    roofline.update(kernel_traffic("k_layer_torus", args.precision))
    out = None
    if rank == 0:
        cpu = cpu_baseline(net, box) if world == 1 else None
        value = whole_job_rate(units, args.steps, world, total_s)
        out = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": round(total_s * 1e3 / args.steps, 4), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else
               {"fp32": "f32", "fp64": "f64"}[args.precision],
               "data": "synthetic (torus SDF net fitted from seed 0)",
               "config": dict(config, precision=args.precision, execution=args.execution, n_vertices=c["nV"],
                              n_edges=c["nE"], l2="flushed by a 512 MiB write before every step",
                              parallelism="replicas" if world > 1 else "single GPU"),
               "e2e": {"value": round(whole_job_rate(units, args.steps, world, e2e_s), 1), "unit": UNIT,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
               "gpu_launches": int(launches), "roofline": roofline, "clocks": clk,
               "step_ms_median": round(statistics.median(step_ms), 4)}
        if cpu:
            out["cpu_baseline"] = cpu
        if world == 1:
            variants = {}
            runs = [(p, {"precision": p}) for p in ("fp64", "mixed") if p != args.precision]
            runs.append(("prune", {"precision": args.precision, "prune": True}))
            for name, kw in runs:
                try:
                    variants[name] = time_variant(Extractor, local_rank, args, net, box, params_dev, flush, kw)
                except Exception as exc:  # a variant never takes the main line down
                    variants[name] = {"error": str(exc)[:200], **kw}
            out["variants"] = variants
            if args.large:
                try:
                    out["large"] = run_large(local_rank, args, flush, peak, peak_kind)
                except Exception as exc:
                    out["large"] = {"error": str(exc)[:300]}
        if args.serve_requests > 0 and world == 1:
            out["serving"] = run_serving_pair(args)
        # longer side measurements: one JSON line each on stderr, so that the
        # main line (the last line on stdout) stays short
        if world == 1:
            extras = {}
            if args.sweep_dims:
                extras["counting_sweep"] = lambda: run_counting_sweep(_dims(args.sweep_dims), args.sweep_seeds,
                                                                      local_rank, args.precision, args.execution)
            if args.domain:
                extras["domain"] = lambda: run_domain(net, params_dev, flush, local_rank, args)
            if args.sweep_dims_w10:
                extras["counting_sweep_w10"] = lambda: run_counting_sweep(
                    _dims(args.sweep_dims_w10), args.sweep_seeds, local_rank, args.precision, args.execution,
                    widths=(10,))
            for name, fn in extras.items():
                try:
                    block = fn()
                except Exception as exc:  # the main line stands on its own
                    block = {"error": str(exc)[:300]}
                print(json.dumps({"side_measurement": name, **block}), file=sys.stderr, flush=True)
    ex.close()
    if dist:
        dist.destroy_process_group()
    return out


def loop_roofline(layer_bytes, loop_ms, peak, peak_kind) -> dict:
    """HBM roofline of k_layer: algorithmic bytes per launch over the mean launch time."""
    import numpy as np
    achieved = sum(layer_bytes) / (float(np.sum(loop_ms)) / 1e3) / 1e9
    return {"kernel": "k_layer (persistent neuron loop, one launch per layer)", "bound": "hbm",
            "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "peak_source": peak_kind, "bytes_per_launch_avg": int(sum(layer_bytes) / len(layer_bytes)),
            "launch_ms_avg": round(float(np.mean(loop_ms)), 4)}


def time_variant(Extractor, device, args, net, box, params_dev, flush, kw, steps=None) -> dict:
    import torch
    steps = steps or args.steps
    with Extractor(device=device, execution=args.execution, **kw) as vx:
        for _ in range(args.warmup):
            vx.extract(net, box, params=params_dev)
        vms = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            vx.extract(net, box, params=params_dev)
            e1.record()
            e1.synchronize()
            vms.append(e0.elapsed_time(e1))
        vc = vx.counts()
    vunits = vc["nV"] + vc["nE"]
    return {"value": round(vunits * len(vms) / (sum(vms) / 1e3), 1), "unit": UNIT,
            "ms_per_step": round(sum(vms) / len(vms), 4), "steps": len(vms), "n_vertices": vc["nV"],
            "n_edges": vc["nE"], **kw}


def run_large(device: int, args, flush, peak, peak_kind) -> dict:
    """The kernels where HBM can bind: the counting-sweep net D=5, width 40
    (seed 0; 1.0e7 vertices, 4.8e7 edges), mixed precision.  Rooflines of
    the neuron loop (bytes model above) and of the tensor-core layer
    products (bytes, and useful flops against the measured TF32 rate)."""
    import numpy as np
    import torch
    from paper_2306_07212_gb300 import Extractor, workloads
    net, box = workloads.counting_sweep_net(5, 40, 0)
    params = torch.from_numpy(net.flat_params()).cuda(device)
    with Extractor(device=device, precision=args.precision, execution=args.execution, timers=True) as ex:
        ex.extract(net, box, params=params)  # grows the buffers
        step, loops, gemms = [], [], []
        for _ in range(2):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ex.extract(net, box, params=params)
            e1.record()
            e1.synchronize()
            step.append(e0.elapsed_time(e1))
            kt = ex.kernel_times_ms()
            loops.append(kt[:, 1].copy())
            gemms.append(kt[:, 0].copy())
        c = ex.counts()
        stats = ex.stats()
        polish_ms = ex.polish_time_ms()
    loop_ms = np.mean(np.stack(loops), axis=0)
    gemm_ms = np.mean(np.stack(gemms), axis=0)
    roof = loop_roofline(neuron_loop_bytes(net, stats, args.precision), loop_ms, peak, peak_kind)
    roof.update(kernel_traffic("k_layer_d5w40", args.precision))
    tf32 = measure_tf32_tflops(device)
    gb = gemm_bytes_flops(net, stats, args.precision)[1:]  # layers 2.. run on the tensor cores
    gms = gemm_ms[1:]
    gbytes = sum(b for b, _ in gb)
    gflops = sum(f for _, f in gb)
    gt = float(np.sum(gms)) / 1e3
    return {"workload": "counting-sweep net D=5, MLP 5-40x4-1 (seed 0), box [-1,1]^5, one extraction",
            "n_vertices": c["nV"], "n_edges": c["nE"], "ms": round(float(np.median(step)), 2),
            "value": round((c["nV"] + c["nE"]) / (float(np.median(step)) / 1e3), 1), "unit": UNIT,
            "loop_ms": round(float(np.sum(loop_ms)), 2), "forward_product_ms": round(float(np.sum(gemm_ms)), 2),
            "polish_ms": round(polish_ms, 2), "roofline": roof,
            "gemm_roofline": {"kernel": "k_gemm_tc2 (layers 2-5)", "bound": "hbm",
                              "achieved": round(gbytes / gt / 1e9, 2), "peak": peak, "unit": "GB/s",
                              "frac": round(gbytes / gt / 1e9 / peak, 4),
                              "tensor_tflops": round(gflops / gt / 1e12, 2), "tf32_peak_tflops": tf32,
                              "tensor_frac": round(gflops / gt / 1e12 / tf32, 4) if tf32 else None,
                              "bytes_per_launch_avg": int(gbytes / len(gb)),
                              "peak_source": "hbm " + peak_kind + "; TF32 measured in this run (torch.matmul 8192^3)",
                              **kernel_traffic("k_gemm_tc2_d5w40", args.precision)}}


def run_serving_pair(args) -> dict:
    """The serving workload through the batched server and the plain path."""
    serving = {"workload": f"Poisson stream, mean 200 req/s, {args.serve_requests} requests, D in {{2,3,4}}, "
                           "depth 2-6, width in {16,32,64,128}, He-normal FP32 weights, mixed precision; "
                           f"requests estimated above {args.serve_max_gib} GiB rejected"}
    for name, slots in (("batched", args.serve_slots), ("plain", 1)):
        try:
            serving[name] = run_serving(args.serve_requests, slots, int(args.serve_max_gib * (1 << 30)))
        except Exception as exc:  # the extraction numbers above stand on their own
            serving[name] = {"slots": slots, "error": str(exc)[:300]}
    return serving


def run_serving(n_requests: int, slots: int, request_max_bytes: int):
    """Poisson stream of extraction requests (serving workload); latencies in ms."""
    import numpy as np
    from paper_2306_07212_gb300 import binding, workloads
    reqs = workloads.serving_stream(n_requests)
    with binding.Server(max_slots=slots, request_max_bytes=request_max_bytes, mem_budget_bytes=160 << 30) as srv:
        t0 = time.perf_counter()
        ids = []
        for r in reqs:
            dt = r.arrival_s - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            ids.append(srv.submit(r.net, r.box))
        srv.wait_all(1800)
        res = [srv.poll(i)[1] for i in ids]
        errors = sorted({srv.error(i)[:160] for i, r in zip(ids, res) if r.status not in (0, 6)})
    ok = [r for r in res if r.status == 0]
    lat = np.array([r.finish_s - r.arrival_s for r in ok]) * 1e3
    span = max(r.finish_s for r in ok) - min(r.arrival_s for r in res)
    ve = sum(r.n_vertices + r.n_edges for r in ok)
    return {"slots": slots, "p50_ms": round(float(np.percentile(lat, 50)), 2),
            "p99_ms": round(float(np.percentile(lat, 99)), 2), "req_per_s": round(len(ok) / span, 2),
            "ve_per_s": round(ve / span, 1), "completed": len(ok),
            "rejected": sum(r.status == 6 for r in res), "failed": sum(r.status not in (0, 6) for r in res),
            "errors": errors[:4]}


def run_domain(net, params_dev, flush, device: int, args):
    """The workload's net on a polyhedral domain instead of the box (Section
    4.1; Section 5.2 suggests a simplex): the corner simplex of the box,
    x_d >= -1 and sum_d (x_d + 1) <= 2, same timing rules as the main line."""
    import torch
    from paper_2306_07212_gb300 import Extractor, workloads
    dom = workloads.Polytope.simplex(net.D)
    with Extractor(device=device, precision=args.precision, execution=args.execution) as dx:
        for _ in range(args.warmup):
            dx.extract_domain(net, dom, params=params_dev)
        ms = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            dx.extract_domain(net, dom, params=params_dev)
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        c = dx.counts()
    units = c["nV"] + c["nE"]
    return {"workload": f"same net on the simplex x_d >= -1, sum_d (x_d + 1) <= 2 ({len(dom.X0)} vertices, "
                        f"{len(dom.c)} facets)", "value": round(units * len(ms) / (sum(ms) / 1e3), 1), "unit": UNIT,
            "ms_per_step": round(sum(ms) / len(ms), 4), "steps": len(ms), "n_vertices": c["nV"],
            "n_edges": c["nE"]}


def zero_residual(net, box, X, words) -> float:
    """Section 5.1.1's validation: the largest |value| of a vertex's zero
    entries (facets and neuron pre-activations by a float64 forward pass at
    its coordinates), relative to the box's extent.  X: (nV, D) float64;
    words: (S, nV) packed sign vectors (entry j at bits 2 (j mod 32) of word
    j / 32, 00 = 0)."""
    import numpy as np
    X = np.asarray(X, np.float64)
    words = np.asarray(words, np.uint64)
    worst = 0.0
    for r0 in range(0, len(X), 1 << 20):  # bounded host memory
        x = X[r0:r0 + (1 << 20)]
        w = words[:, r0:r0 + (1 << 20)]
        facets = np.empty((len(x), 2 * net.D))
        facets[:, 0::2], facets[:, 1::2] = x - box.lo, box.hi - x
        cols, a = [facets], x
        for W, b in zip(net.W, net.b):
            z = a @ W.T + b
            cols.append(z)
            a = np.maximum(z, 0.0)
        allv = np.concatenate(cols, axis=1)
        for j in range(allv.shape[1]):
            on = ((w[j // 32] >> np.uint64(2 * (j % 32))) & np.uint64(3)) == 0
            if on.any():
                worst = max(worst, float(np.abs(allv[on, j]).max()))
    return worst / float(np.max(box.hi - box.lo))


def _dims(spec: str) -> list:
    """"1-4" or "1,2,5" -> sorted input dimensions."""
    dims = set()
    for part in spec.split(","):
        lo, _, hi = part.partition("-")
        dims.update(range(int(lo), int(hi or lo) + 1))
    return sorted(dims)


def run_counting_sweep(dims, seeds: int, device: int, precision: str, execution: str, widths=None):
    """Counting sweep (Section 5.1.2): per input dimension D and width w, nets
    of four hidden layers of w on [-1,1]^D, `seeds` random nets each; vertex
    and edge counts, extraction time and peak device memory, mean and standard
    deviation over the nets.  Each net gets a fresh context: `cold_ms` is its
    first extraction (capacity growth included), `ms` the median of three more,
    `peak_mib` the most device memory allocated above what was held before;
    at width 10 `zero_residual_rel` is the largest zero-entry residual of
    the first net (zero_residual; the paper validates one fixed 4-layer
    width-10 net per dimension)."""
    import numpy as np
    import torch
    from paper_2306_07212_gb300 import Extractor, workloads

    def timed(ex, net, box, params):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ex.extract(net, box, params=params)
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1)

    def ms(a):
        return [round(float(np.mean(a)), 3), round(float(np.std(a)), 3)]

    t_start = time.perf_counter()
    points = []
    widths = tuple(widths or workloads.COUNTING_WIDTHS)
    for width in widths:
        for D in dims:
            rows, residual = [], 0.0
            try:
                for seed in range(seeds):
                    net, box = workloads.counting_sweep_net(D, width, seed)
                    params = torch.from_numpy(net.flat_params()).cuda(device)
                    torch.cuda.synchronize()
                    base = torch.cuda.memory_allocated(device)
                    torch.cuda.reset_peak_memory_stats(device)
                    with Extractor(device=device, precision=precision, execution=execution,
                                   max_dim=8 if D <= 8 else 10) as ex:
                        cold = timed(ex, net, box, params)
                        peak = torch.cuda.max_memory_allocated(device) - base
                        warm = statistics.median([timed(ex, net, box, params) for _ in range(3)])
                        c = ex.counts()
                        if width == 10 and seed == 0:  # the paper validates one fixed 4-layer width-10 net
                            residual = zero_residual(net, box, ex.vertices(), ex.sign_words())
                    rows.append((c["nV"], c["nE"], cold, warm, peak / 2**20))
            except Exception as exc:  # e.g. a dimension the library does not take
                points.append({"D": D, "width": width, "error": str(exc)[:200]})
                continue
            a = np.array(rows, np.float64)
            points.append({"D": D, "width": width, "nV": ms(a[:, 0]), "nE": ms(a[:, 1]), "ms": ms(a[:, 3]),
                           "cold_ms": ms(a[:, 2]), "peak_mib": ms(a[:, 4]),
                           "ve_per_s": round(float(np.mean((a[:, 0] + a[:, 1]) / (a[:, 3] / 1e3))), 1)})
            if width == 10:
                points[-1]["zero_residual_rel"] = float(f"{residual:.3g}")
    return {"workload": f"Section 5.1.2 counting sweep: MLP [D, w, w, w, w, 1], w in "
                        f"{list(widths)}, D in {dims}, {seeds} uniformly initialised nets per "
                        f"point (FP32 weights), box [-1,1]^D, {precision} precision; values are [mean, std]",
            "points": points, "seconds": round(time.perf_counter() - t_start, 1)}


def host_cpu() -> dict:
    """Core count and CPU model of the host that runs the oracle."""
    info = {"nproc": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            key, _, val = line.partition(":")
            if key.strip() == "Model name":
                info["model"] = val.strip()
                break
    except Exception:
        pass
    return info


def cpu_baseline(net, box):
    import oracle
    t0 = time.perf_counter()
    r = oracle.extract(net, box)
    dt = time.perf_counter() - t0
    return {"value": round((r.nV + r.nE) / dt, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one full FP64 oracle extraction of the same workload ({r.nV} V, {r.nE} E) in {dt:.2f} s",
            "host": host_cpu()}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle
    net, box, config = _workload()
    for _ in range(args.warmup):
        oracle.extract(net, box)
    times = []
    units = 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.extract(net, box)
        times.append(time.perf_counter() - t0)
        units = r.nV + r.nE
    total = sum(times)
    value = units * args.steps / total
    cpu = {"value": round(value, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"full FP64 oracle extraction of the workload per step ({units} V+E)", "host": host_cpu()}
    return {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total * 1e3 / args.steps, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (torus SDF net fitted from seed 0)", "config": dict(config, precision="fp64"),
            "cpu_baseline": cpu,
            "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp32", "fp64"])
    ap.add_argument("--execution", default="persistent", choices=["persistent", "stepwise"])
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving stream to replay (0 = skip the serving measurement)")
    ap.add_argument("--sweep-dims", default="1-5",
                    help="input dimensions of the counting sweep, e.g. 1-4 or 1,2,5 ('' = skip it)")
    ap.add_argument("--sweep-seeds", type=int, default=5, help="random nets per counting-sweep point")
    ap.add_argument("--sweep-dims-w10", default="6-10",
                    help="input dimensions of the width-10 counting sweep beyond --sweep-dims ('' = skip it)")
    ap.add_argument("--domain", type=int, default=1, help="1: also time the net on a simplex domain")
    ap.add_argument("--large", type=int, default=1,
                    help="1: also the rooflines on the D=5, width-40 sweep net (1e7 vertices)")
    ap.add_argument("--serve-slots", type=int, default=8, help="slots of the batched server")
    ap.add_argument("--serve-max-gib", type=float, default=64.0,
                    help="serving: requests whose memory estimate exceeds this are rejected")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local_rank)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
