"""Benchmark of the PQ + IVF-ADC hot path on one GB300 (or N replicas).

Default workload (1M x 128 integer-valued mixture, M=16, Ks=256): one step is
the whole path -- PQ fit (k-means++ seeding + 25 Lloyd iterations), encode
with the reconstruction error, inverted-index build (coarse k-means
nlist=1024, 25 iterations, bucketing) and the IVF-ADC query of 10,000 queries
(nprobe=16, top-100).  `--workload pq_10m_d128_m16` times the precision form
(10M x 128, 20 iterations; fit + encode per step) and `--compare-fp32` adds
the plain FP32 form of the same fit + encode beside it.

value        fit+encode throughput, Mvec/s = N / (t_fit + t_encode), inputs
             resident in HBM, device time (CUDA events on the launch stream).
e2e          the same metric through the public API from pinned host buffers:
             X copied in, codes and codebooks copied out inside the timed region.
roofline     the kernel with the largest share of step time, its algorithmic
             work per launch over its measured average launch time.
cpu_baseline the FP64 oracle on the host cores, fit+encode on a bounded row
             sample of the same workload.
`--impl reference` times that oracle as the reference arm.

Multi-GPU: the path does not shard (one GPU per replica); with torchrun each
rank runs the same workload on its own GPU and value sums the ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2604_21645_gb300 import datagen  # noqa: E402

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_PATH = os.path.join(ROOT, "profiles", "traffic.json")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
SMS = 152


def load_peaks():
    try:
        with open(PEAKS_PATH) as f:
            return json.load(f), "measured"
    except OSError:
        return dict(FALLBACK_PEAKS), "fallback"


def fp32_peak_tflops(peaks):
    # 152 SMs x 128 FP32 lanes x 2 flop per FFMA x max SM clock
    return SMS * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def compare_peak_t(peaks):
    # 152 SMs x 128 FP32 lanes x one FMNMX per lane per clock x max SM clock (Tcmp/s)
    return SMS * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def source_hash(*names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2604_21645_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# algorithmic work per launch of each kernel, for the roofline of the dominant one:
# (bound, work, unit, peak kind)
def kernel_work(name, w, n_launch_rows):
    D, M, Ks = w.d, w.m, w.ks
    if name == "pq_pass_f32":
        # the plain form evaluates every (row, subspace, codeword) distance with Ds FFMAs
        return "alu", 2.0 * n_launch_rows * Ks * D, "TFLOP/s", "fp32"
    if name == "pq_pass_tc":
        # the argmin over Ks tensor-core scores needs one FP32 compare per score
        return "alu", float(n_launch_rows) * M * Ks, "Tcmp/s", "cmp"
    if name == "coarse_assign_tc":
        return "tensor", 2.0 * w.n * w.nlist * D, "TFLOP/s", "bf16_sustained"
    if name == "coarse_assign":
        return "alu", 2.0 * w.n * w.nlist * D, "TFLOP/s", "fp32"
    if name == "list_mean":
        return "hbm", float(w.n) * (4 * D + 8), "GB/s", "hbm"
    if name == "adc_scan":
        # codes of the probed lists (uniform-list expectation)
        return "hbm", float(w.nq) * w.nprobe * (w.n / w.nlist) * M, "GB/s", "hbm"
    return None, None, None, None


def roofline(kern, w, peaks, peak_src):
    """Roofline record of the kernel with the largest share of the timed region."""
    if not kern:
        return None
    dominant = max(kern, key=lambda n: kern[n]["ms"])
    k = kern[dominant]
    avg_s = k["ms"] / max(k["launches"], 1) / 1e3
    bound, work, unit, kind = kernel_work(dominant, w, w.n)
    share = k["ms"] / max(sum(v["ms"] for v in kern.values()), 1e-9)
    if work is None:
        return {"kernel": dominant, "bound": "latency", "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None, "avg_launch_ms": avg_s * 1e3, "share": share}
    if kind == "hbm":
        achieved, peak, src = work / avg_s / 1e9, peaks["hbm_gbs"], peak_src
    elif kind == "bf16_sustained":
        achieved, peak, src = work / avg_s / 1e12, peaks["bf16_tflops_sustained"], peak_src
    elif kind == "cmp":
        achieved, peak = work / avg_s / 1e12, compare_peak_t(peaks)
        src = "152 SMs x 128 FP32 lanes x 1 compare per clock x max SM clock"
    else:
        achieved, peak = work / avg_s / 1e12, fp32_peak_tflops(peaks)
        src = "152 SMs x 128 FP32 lanes x 2 flop per FFMA x max SM clock"
    traffic = None
    try:
        with open(TRAFFIC_PATH) as f:
            tr = json.load(f).get(dominant)
        if tr and tr.get("source_hash") == source_hash(*tr["sources"]) and tr.get("workload") == w.name:
            traffic = tr["bytes_per_launch"]
    except (OSError, KeyError, ValueError):
        traffic = None
    return {"kernel": dominant, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": traffic, "peak_source": src, "avg_launch_ms": avg_s * 1e3,
            "share": share}


def run_gpu(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2604_21645_gb300 import pqgb

    w = datagen.WORKLOADS[args.workload]
    ivf = w.nlist > 0
    prec = args.prec
    X = w.data()
    Xd = torch.from_numpy(X).cuda()
    if ivf:
        Qd = torch.from_numpy(w.queries()).cuda()
        out_ids = torch.empty((w.nq, w.topk), dtype=torch.int64, device="cuda")
        out_d = torch.empty((w.nq, w.topk), dtype=torch.float32, device="cuda")
    cbs = torch.empty((w.m, w.ks, w.d // w.m), dtype=torch.float32, device="cuda")
    codes = torch.empty((w.n, w.m), dtype=torch.uint8, device="cuda")
    sse = torch.zeros(1, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > L2
    stream = torch.cuda.current_stream()
    names = ["fit", "encode"] + (["ivf_build", "ivf_search"] if ivf else [])

    def step(p=prec, full=True):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
        ev[0].record(stream)
        pqgb.fit(Xd, w.m, w.ks, iters=w.iters, seed=w.init_seed, prec=p, out=cbs)
        ev[1].record(stream)
        pqgb.encode(Xd, cbs, prec=p, out=codes, sse=sse)
        ev[2].record(stream)
        idx = None
        if ivf and full:
            idx = pqgb.IVFIndex.build(Xd, codes, w.nlist, iters=w.ivf_iters, seed=w.coarse_seed, prec=p)
            ev[3].record(stream)
            idx.search(cbs, Qd, w.nprobe, w.topk, out_ids=out_ids, out_d=out_d)
            ev[4].record(stream)
        return ev, idx

    def timed(p, full, steps):
        n = len(names) if full else 2
        ph = np.zeros(n)
        for _ in range(steps):
            flush.zero_()
            ev, idx = step(p, full)
            torch.cuda.synchronize()
            ph += [ev[i].elapsed_time(ev[i + 1]) for i in range(n)]
            if idx is not None:
                idx.close()
        return ph / steps

    for _ in range(args.warmup):
        _, idx = step()
        if idx is not None:
            idx.close()
    torch.cuda.synchronize()

    launches0 = pqgb.launch_count()
    pqgb.profile_enable(True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        per_step = timed(prec, True, args.steps)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    launches = pqgb.launch_count() - launches0

    # per-kernel device time inside the timed region (events on the launch stream)
    kern = pqgb.profile_collect()
    pqgb.profile_enable(False)
    _, rmse = pqgb.decode_rmse(codes, cbs, Xd)

    t_fe = (per_step[0] + per_step[1]) / 1e3
    t_step = per_step.sum() / 1e3
    t_search = per_step[3] / 1e3 if ivf else 0.0
    if world > 1:
        t = torch.tensor([t_fe, t_step, t_search], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_fe, t_step, t_search = t.tolist()
    value = world * w.n / t_fe / 1e6

    # the plain FP32 form of the same fit + encode, for the precision comparison
    fp32_form = None
    if args.compare_fp32 and prec != "fp32":
        for _ in range(1):
            step("fp32", False)
        ph = timed("fp32", False, args.steps)
        _, rmse32 = pqgb.decode_rmse(codes, cbs, Xd)
        t32 = (ph[0] + ph[1]) / 1e3
        fp32_form = {"value": world * w.n / t32 / 1e6, "unit": "Mvec/s", "ms_fit": ph[0], "ms_encode": ph[1],
                     "rmse": rmse32, "rmse_rel_diff": abs(rmse - rmse32) / rmse32}

    # end-to-end through the public API from pinned host buffers (fit + encode)
    Xh = torch.from_numpy(X).pin_memory()
    codes_h = torch.empty((w.n, w.m), dtype=torch.uint8).pin_memory()
    cbs_h = torch.empty_like(cbs, device="cpu").pin_memory()
    Xe = torch.empty_like(Xd)
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Xe.copy_(Xh, non_blocking=True)
        pqgb.fit(Xe, w.m, w.ks, iters=w.iters, seed=w.init_seed, prec=prec, out=cbs)
        pqgb.encode(Xe, cbs, prec=prec, out=codes)
        codes_h.copy_(codes, non_blocking=True)
        cbs_h.copy_(cbs, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    t_e2e = float(np.mean(e2e_ms)) / 1e3
    if world > 1:
        t = torch.tensor([t_e2e], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_e2e = t.item()

    peaks, peak_src = load_peaks()
    cfg = {"workload": w.name, "N": w.n, "D": w.d, "M": w.m, "Ks": w.ks, "iters": w.iters}
    if ivf:
        cfg.update({"nlist": w.nlist, "ivf_iters": w.ivf_iters, "nq": w.nq, "nprobe": w.nprobe, "topk": w.topk})
    cfg.update({"prec": prec, "parallelism": f"replicas{world}",
                "l2": f"256 MB buffer written between steps; X ({X.nbytes // 10**6} MB) exceeds L2"})
    line = {
        "metric": "PQ fit+encode Mvec/s" + (" (IVF-ADC queries/s reported beside it)" if ivf else ""),
        "value": value,
        "unit": "Mvec/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_step * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if prec == "fp32" else "bf16",
        "data": "synthetic (seeded Gaussian mixture standing in for the paper's data)",
        "config": cfg,
        "phases_ms": dict(zip(names, per_step.tolist())),
        "rmse": rmse,
        "e2e": {"value": world * w.n / t_e2e / 1e6, "unit": "Mvec/s", "h2d_bytes_per_step": int(X.nbytes),
                "d2h_bytes_per_step": int(codes.numel() + cbs.numel() * 4)},
        "gpu_launches": int(launches),
        "kernels": kern,
        "roofline": roofline(kern, w, peaks, peak_src),
        "clocks": clk.summary(),
    }
    if ivf:
        line["queries_per_s"] = world * w.nq / t_search
    if fp32_form:
        line["fp32_form"] = fp32_form
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_rows)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def oracle_fit_encode(w, rows):
    import oracle as orc
    X = datagen.mixture(rows, w.d, w.n_comp, w.kind, w.seed)
    t0 = time.perf_counter()
    cb, _ = orc.pq_fit(X, w.m, w.ks, w.iters, w.init_seed)
    orc.pq_encode(X, cb)
    return time.perf_counter() - t0


def cpu_baseline(w, rows):
    import oracle as orc
    t = oracle_fit_encode(w, rows)
    return {"value": rows / t / 1e6, "unit": "Mvec/s", "cores": orc.num_threads(), "kind": "oracle",
            "sample": f"FP64 oracle pq_fit ({w.iters} Lloyd iterations, k-means++ seeding) + pq_encode on the first "
                      f"{rows} rows of the same seeded mixture, {t:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import oracle as orc
    w = datagen.WORKLOADS[args.workload]
    rows = args.cpu_rows
    for _ in range(args.warmup):
        oracle_fit_encode(w, rows // 4)
    times = [oracle_fit_encode(w, rows) for _ in range(args.steps)]
    t = float(np.mean(times))
    v = rows / t / 1e6
    print(json.dumps({
        "impl": "reference",
        "metric": "PQ fit+encode Mvec/s" + (" (IVF-ADC queries/s reported beside it)" if w.nlist else ""),
        "value": v, "unit": "Mvec/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (seeded Gaussian mixture standing in for the paper's data)",
        "config": {"workload": w.name, "N": w.n, "D": w.d, "M": w.m, "Ks": w.ks, "iters": w.iters,
                   "sample_rows": rows},
        "cpu_baseline": {"value": v, "unit": "Mvec/s", "cores": orc.num_threads(), "kind": "oracle",
                         "sample": f"fit+encode on the first {rows} of {w.n} rows per step"},
        "e2e": {"value": v, "unit": "Mvec/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=datagen.IVF_MEDIUM.name, choices=[datagen.IVF_MEDIUM.name,
                                                                            datagen.PQ_10M.name])
    ap.add_argument("--prec", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--compare-fp32", action="store_true", help="also time the plain FP32 form of fit + encode")
    ap.add_argument("--cpu-rows", type=int, default=50_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
