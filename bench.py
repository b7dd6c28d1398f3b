"""Benchmark of the PQ + IVF-ADC hot path on one GB300 (or N replicas).

Default workload (`pq_10m_d128_m16`): PQ fit + encode of 10M x 128 float32 rows
(integer-valued 4,096-component mixture), M=16, Ks=256, k-means++ seeding and 20
Lloyd iterations, in the BF16 tensor-core form with exact re-rank.  One step is
fit + encode with the reconstruction error.  Beside it the same line carries

fp32_form    the plain FP32 form of the same fit + encode (time, RMSE, ratio);
ivf_10m      IVF-ADC search of 10k queries (nprobe=16 of 1024 lists, top-100) over
             an index of the same 10M rows -- 160 MB of codes, larger than L2;
ivf_1m       the medium workload's search (1M x 128, nlist=1024, nprobe=16,
             top-100) with its recall against exhaustive FP64 neighbours.

`--workload ivf_1m_d128_m16_nlist1024` times the whole medium pipeline per step
(fit, encode, index build, search); `chunked_64x_d96_m12` and
`softpq_1m_d256_m32` time the batched and the soft-refinement forms.

value        fit+encode throughput, Mvec/s = N / (t_fit + t_encode), inputs
             resident in HBM, device time (CUDA events on the launch stream).
e2e          the same metric through the C ABI from pinned host buffers
             (pq_fit_encode_host: X copied in beside the seeding, which reads its
             subsample rows from host memory; codes and codebooks copied out),
             all inside the timed region.
roofline     the kernel with the largest share of the timed step, its
             algorithmic bytes (or flops) per launch over its measured average
             launch time.
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
# (bound, work, unit, peak kind).  `launch_rows` is the average number of rows one launch
# of the PQ pass processes; `encode_share` the fraction of those launches that also write codes.
def kernel_work(name, w, launch_rows, encode_share=0.0):
    D, M, Ks = w.d, w.m, w.ks
    if name == "pq_pass_f32":
        # the plain form evaluates every (row, subspace, codeword) distance with Ds FFMAs
        return "alu", 2.0 * launch_rows * Ks * D, "TFLOP/s", "fp32"
    if name in ("pq_pass_tc", "pq_fit_persistent_tc"):
        # HBM: each pass reads X once (D floats per row); the encode pass also writes M code bytes.
        # The persistent batched fit runs all the local passes in one launch (launch_rows = iters * N).
        return "hbm", float(launch_rows) * (4.0 * D + encode_share * M), "GB/s", "hbm"
    if name == "coarse_assign_tc":
        return "tensor", 2.0 * w.n * w.nlist * D, "TFLOP/s", "bf16_sustained"
    if name == "coarse_assign":
        return "alu", 2.0 * w.n * w.nlist * D, "TFLOP/s", "fp32"
    if name == "list_mean":
        return "hbm", float(w.n) * (4 * D + 8), "GB/s", "hbm"
    return None, None, None, None


def slowest_rank(values, world, device="cuda"):
    """Element-wise maximum of per-rank timings over all ranks (the replica job ends with its slowest rank)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def replica_throughput(units_per_rank, seconds, world):
    """Whole-job throughput of `world` replicas that each processed units_per_rank in (max) seconds."""
    return world * units_per_rank / seconds


def measured_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu capture, or None if absent or the kernel changed since."""
    try:
        with open(TRAFFIC_PATH) as f:
            tr = json.load(f).get(kernel)
        if tr and tr.get("source_hash") == source_hash(*tr["sources"]):
            return tr.get("per_workload", {}).get(workload)
    except (OSError, KeyError, ValueError):
        pass
    return None


def roofline_record(name, bound, work, unit, kind, avg_s, peaks, peak_src, workload, share=None):
    """{bound, achieved, peak, unit, frac, traffic} of one kernel from its algorithmic work per launch."""
    if kind == "hbm":
        achieved, peak, src = work / avg_s / 1e9, peaks["hbm_gbs"], f"{peak_src} HBM copy bandwidth"
    elif kind == "bf16_sustained":
        achieved, peak, src = work / avg_s / 1e12, peaks["bf16_tflops_sustained"], f"{peak_src} sustained bf16"
    else:
        achieved, peak = work / avg_s / 1e12, fp32_peak_tflops(peaks)
        src = "derived: 152 SMs x 128 FP32 lanes x 2 flop per FFMA x max SM clock"
    rec = {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
           "traffic": measured_traffic(name, workload), "peak_source": src, "avg_launch_ms": avg_s * 1e3,
           "work_per_launch": work}
    if share is not None:
        rec["share"] = share
    return rec


def roofline(kern, w, peaks, peak_src, launch_rows=None, encode_share=0.0):
    """Roofline record of the kernel with the largest share of the timed region."""
    if not kern:
        return None
    dominant = max(kern, key=lambda n: kern[n]["ms"])
    k = kern[dominant]
    avg_s = k["ms"] / max(k["launches"], 1) / 1e3
    bound, work, unit, kind = kernel_work(dominant, w, w.n if launch_rows is None else launch_rows, encode_share)
    share = k["ms"] / max(sum(v["ms"] for v in kern.values()), 1e-9)
    if work is None:
        return {"kernel": dominant, "bound": "latency", "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None, "avg_launch_ms": avg_s * 1e3, "share": share}
    return roofline_record(dominant, bound, work, unit, kind, avg_s, peaks, peak_src, w.name, share)


def run_gpu_pipeline(args):
    """The medium workload's whole path per step: fit, encode, index build and search."""
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
    _, est = pqgb.encode(Xd, cbs, prec=prec, stats=True)
    near_ties = est["fp64_rechecks"] / (w.n * w.m)

    t_fe = (per_step[0] + per_step[1]) / 1e3
    t_step = per_step.sum() / 1e3
    t_search = per_step[3] / 1e3 if ivf else 0.0
    t_fe, t_step, t_search = slowest_rank([t_fe, t_step, t_search], world)
    value = replica_throughput(w.n, t_fe, world) / 1e6

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

    # end-to-end through the C ABI from pinned host buffers (fit + encode in one call: the
    # seeding reads its subsample from host memory while X is copied to the device)
    Xh = torch.from_numpy(X).pin_memory()
    codes_h = torch.empty((w.n, w.m), dtype=torch.uint8).pin_memory()
    cbs_h = torch.empty_like(cbs, device="cpu").pin_memory()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pqgb.fit_encode_host(Xh, w.m, w.ks, iters=w.iters, seed=w.init_seed, prec=prec, codebooks=cbs_h,
                             codes=codes_h, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    t_e2e = slowest_rank([float(np.mean(e2e_ms)) / 1e3], world)[0]

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
        "exact_rerank_fraction": near_ties,
        "e2e": {"value": replica_throughput(w.n, t_e2e, world) / 1e6, "unit": "Mvec/s",
                # X copied once, plus the seeding's subsample rows read from host memory
                "h2d_bytes_per_step": int(X.nbytes + min(w.n, 100 * w.ks) * w.d * 4),
                "d2h_bytes_per_step": int(codes_h.numel() + cbs_h.numel() * 4)},
        "gpu_launches": int(launches),
        "kernels": kern,
        "roofline": roofline(kern, w, peaks, peak_src, encode_share=1.0 / (w.iters + 1)),
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


def _probe_bytes(torch, Qd, coarse, offsets, nprobe, M):
    """Code bytes the scan of each query reads: the sizes of its nprobe nearest lists (FP32 distances
    on the device; a near-tie at the cut can swap two lists, which moves the count negligibly)."""
    qn = (Qd * Qd).sum(1, keepdim=True)
    cn = (coarse * coarse).sum(1)[None, :]
    dist = qn - 2.0 * Qd @ coarse.T + cn
    probes = torch.topk(dist, nprobe, dim=1, largest=False).indices
    sizes = (offsets[1:] - offsets[:-1])[probes]
    return float(sizes.sum().item()) * M


def _exact_nn(torch, Xd, Qs):
    """Exhaustive FP64 nearest neighbour of each query row, on the device (FP64 distances
    ||x||^2 - 2 x.q + ||q||^2 in batches of 100 queries)."""
    X64 = Xd.double()
    xn = (X64 * X64).sum(1)
    out = []
    for b in range(0, Qs.shape[0], 100):
        q = Qs[b:b + 100].double()
        d = xn[None, :] - 2.0 * (q @ X64.T) + (q * q).sum(1, keepdim=True)
        out.append(torch.argmin(d, dim=1).cpu().numpy())
    del X64
    return np.concatenate(out)


def _time_search(torch, pqgb, idx, cbs, Qd, w, steps, warmup, flush):
    out_ids = torch.empty((Qd.shape[0], w.topk), dtype=torch.int64, device="cuda")
    out_d = torch.empty((Qd.shape[0], w.topk), dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        idx.search(cbs, Qd, w.nprobe, w.topk, out_ids=out_ids, out_d=out_d)
    torch.cuda.synchronize()
    pqgb.profile_enable(True)
    ms = _timed_steps(torch, lambda: idx.search(cbs, Qd, w.nprobe, w.topk, out_ids=out_ids, out_d=out_d), steps,
                      flush)
    kern = pqgb.profile_collect()
    pqgb.profile_enable(False)
    return float(np.mean(ms)), kern, out_ids, out_d


def run_gpu(args):
    """The precision form (10M x 128 fit + encode) and, beside it, the IVF-ADC search figures."""
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
    prec = args.prec
    X = w.data()
    Xd = torch.from_numpy(X).cuda()
    cbs = torch.empty((w.m, w.ks, w.d // w.m), dtype=torch.float32, device="cuda")
    codes = torch.empty((w.n, w.m), dtype=torch.uint8, device="cuda")
    sse = torch.zeros(1, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > L2
    stream = torch.cuda.current_stream()

    def step(p):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        pqgb.fit(Xd, w.m, w.ks, iters=w.iters, seed=w.init_seed, prec=p, out=cbs)
        ev[1].record(stream)
        pqgb.encode(Xd, cbs, prec=p, out=codes, sse=sse)
        ev[2].record(stream)
        return ev

    def timed(p, steps):
        ph = np.zeros(2)
        for _ in range(steps):
            flush.zero_()
            ev = step(p)
            torch.cuda.synchronize()
            ph += [ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])]
        return ph / steps

    for _ in range(args.warmup):
        step(prec)
    torch.cuda.synchronize()
    launches0 = pqgb.launch_count()
    pqgb.profile_enable(True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        per_step = timed(prec, args.steps)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    launches = pqgb.launch_count() - launches0
    kern = pqgb.profile_collect()
    pqgb.profile_enable(False)
    _, rmse = pqgb.decode_rmse(codes, cbs, Xd)
    _, est = pqgb.encode(Xd, cbs, prec=prec, stats=True)
    t_fe = slowest_rank([(per_step[0] + per_step[1]) / 1e3], world)[0]
    value = replica_throughput(w.n, t_fe, world) / 1e6
    peaks, peak_src = load_peaks()
    codes_main = codes.clone()
    cbs_main = cbs.clone()

    # the plain FP32 form of the same fit + encode
    fp32_form = None
    if not args.no_compare_fp32 and prec != "fp32":
        step("fp32")
        torch.cuda.synchronize()
        pqgb.profile_enable(True)
        ph = timed("fp32", args.steps)
        kern32 = pqgb.profile_collect()
        pqgb.profile_enable(False)
        _, rmse32 = pqgb.decode_rmse(codes, cbs, Xd)
        t32 = slowest_rank([(ph[0] + ph[1]) / 1e3], world)[0]
        v32 = replica_throughput(w.n, t32, world) / 1e6
        fp32_form = {"value": v32, "unit": "Mvec/s", "ms_fit": ph[0], "ms_encode": ph[1], "rmse": rmse32,
                     "rmse_rel_diff": abs(rmse - rmse32) / rmse32, "bf16_over_fp32": value / v32,
                     "roofline": roofline(kern32, w, peaks, peak_src)}

    # end-to-end through the C ABI from pinned host buffers
    Xh = torch.from_numpy(X).pin_memory()
    codes_h = torch.empty((w.n, w.m), dtype=torch.uint8).pin_memory()
    cbs_h = torch.empty_like(cbs, device="cpu").pin_memory()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pqgb.fit_encode_host(Xh, w.m, w.ks, iters=w.iters, seed=w.init_seed, prec=prec, codebooks=cbs_h,
                             codes=codes_h, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    t_e2e = slowest_rank([float(np.mean(e2e_ms)) / 1e3], world)[0]
    del Xh

    cfg = {"workload": w.name, "N": w.n, "D": w.d, "M": w.m, "Ks": w.ks, "iters": w.iters, "prec": prec,
           "parallelism": f"replicas{world}",
           "l2": f"256 MB buffer written between steps; X ({X.nbytes // 10**6} MB) exceeds L2"}
    line = {
        "metric": "PQ fit+encode Mvec/s (IVF-ADC queries/s reported beside it)",
        "value": value,
        "unit": "Mvec/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_fe * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if prec == "fp32" else "bf16",
        "data": "synthetic (seeded Gaussian mixture standing in for the paper's data)",
        "config": cfg,
        "phases_ms": {"fit": per_step[0], "encode": per_step[1]},
        "rmse": rmse,
        "exact_rerank_fraction": est["fp64_rechecks"] / (w.n * w.m),
        "e2e": {"value": replica_throughput(w.n, t_e2e, world) / 1e6, "unit": "Mvec/s",
                # X copied once, plus the seeding's subsample rows read from host memory
                "h2d_bytes_per_step": int(X.nbytes + min(w.n, 100 * w.ks) * w.d * 4),
                "d2h_bytes_per_step": int(codes_h.numel() + cbs_h.numel() * 4)},
        "gpu_launches": int(launches),
        "kernels": kern,
        "roofline": roofline(kern, w, peaks, peak_src, encode_share=1.0 / (w.iters + 1)),
        "clocks": clk.summary(),
    }
    if fp32_form:
        line["fp32_form"] = fp32_form

    if not args.no_search:
        # IVF-ADC search over the same 10M rows: 160 MB of codes, more than L2 holds
        wi = datagen.IVF_10M
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        idx = pqgb.IVFIndex.build(Xd, codes_main, wi.nlist, iters=wi.ivf_iters, seed=wi.coarse_seed, prec=prec)
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t0
        # the rows are not needed by the search: only the index (codes, ids, lists) stays on the device
        del Xd
        torch.cuda.empty_cache()
        Qd = torch.from_numpy(wi.queries()).cuda()
        ms, kern_s, _, _ = _time_search(torch, pqgb, idx, cbs_main, Qd, wi, args.steps, args.warmup, flush)
        off, _, _ = idx.lists()
        scanned = _probe_bytes(torch, Qd, idx.coarse(), off, wi.nprobe, wi.m)
        ivf10 = {"workload": wi.name, "queries_per_s": world * wi.nq / (ms / 1e3), "ms": ms, "build_s": t_build,
                 "nlist": wi.nlist, "nprobe": wi.nprobe, "topk": wi.topk, "nq": wi.nq,
                 "code_bytes_scanned": scanned, "kernels": kern_s}
        if "adc_scan" in kern_s:
            avg = kern_s["adc_scan"]["ms"] / max(kern_s["adc_scan"]["launches"], 1) / 1e3
            ivf10["roofline"] = roofline_record("adc_scan", "hbm", scanned, "GB/s", "hbm", avg, peaks, peak_src,
                                                wi.name)
        idx.close()
        del Qd
        line["ivf_10m"] = ivf10
        # the medium workload's index (1M x 128, 1,000 components) and its recall
        wm = datagen.IVF_MEDIUM
        Xm = torch.from_numpy(wm.data()).cuda()
        cm = pqgb.fit(Xm, wm.m, wm.ks, iters=wm.iters, seed=wm.init_seed, prec=prec)
        codes_m = pqgb.encode(Xm, cm, prec=prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        idx = pqgb.IVFIndex.build(Xm, codes_m, wm.nlist, iters=wm.ivf_iters, seed=wm.coarse_seed, prec=prec)
        torch.cuda.synchronize()
        t_b1 = time.perf_counter() - t0
        Qd = torch.from_numpy(wm.queries()).cuda()
        ms, kern_s, ids, _ = _time_search(torch, pqgb, idx, cm, Qd, wm, args.steps, args.warmup, flush)
        sample = np.random.default_rng(0).choice(wm.nq, 1000, replace=False)
        nn = _exact_nn(torch, Xm, Qd[torch.from_numpy(sample).cuda()])
        got = ids.cpu().numpy()[sample]
        recall = {f"recall@{r}": float(np.mean([nn[i] in got[i, :r] for i in range(len(sample))]))
                  for r in (1, 10, 100)}
        off, _, _ = idx.lists()
        scanned = _probe_bytes(torch, Qd, idx.coarse(), off, wm.nprobe, wm.m)
        ivf1 = {"workload": wm.name, "queries_per_s": world * wm.nq / (ms / 1e3), "ms": ms, "build_s": t_b1,
                "nlist": wm.nlist,
                "nprobe": wm.nprobe, "topk": wm.topk, "nq": wm.nq, "code_bytes_scanned": scanned,
                "recall": recall, "recall_sample": "exact FP64 1-NN of 1,000 sampled queries (torch on the device)",
                "l2_note": "the 16 MB code array is L2-resident"}
        idx.close()
        # the code-space index (Rii: centre codes by k-means over the PQ codes) over the same codes
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        idxc = pqgb.IVFIndex.build_codes(codes_m, cm, wm.nlist, iters=wm.ivf_iters, seed=wm.coarse_seed, prec=prec)
        torch.cuda.synchronize()
        t_bc = time.perf_counter() - t0
        ms_c, kern_c, ids_c, _ = _time_search(torch, pqgb, idxc, cm, Qd, wm, args.steps, args.warmup, flush)
        got_c = ids_c.cpu().numpy()[sample]
        recall_c = {f"recall@{r}": float(np.mean([nn[i] in got_c[i, :r] for i in range(len(sample))]))
                    for r in (1, 10, 100)}
        off_c, _, _ = idxc.lists()
        scanned_c = _probe_bytes(torch, Qd, idxc.coarse(), off_c, wm.nprobe, wm.m)
        idxc.close()
        ivf1["code_space"] = {"queries_per_s": world * wm.nq / (ms_c / 1e3), "ms": ms_c, "build_s": t_bc,
                              "code_bytes_scanned": scanned_c, "recall": recall_c,
                              "note": "centre codes by k-means over the PQ codes, probed by the query's ADC table"}
        line["ivf_1m"] = ivf1
        line["queries_per_s"] = ivf10["queries_per_s"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_rows)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _timed_steps(torch, step, steps, flush):
    """CUDA-event time (ms) of each of `steps` calls of step(), L2 flushed before each."""
    stream = torch.cuda.current_stream()
    out = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def _common_line(args, world, metric, value, unit, ms, dtype, cfg, kern, launches, clk):
    return {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype,
            "data": "synthetic (seeded Gaussian mixture standing in for the paper's data)", "config": cfg,
            "gpu_launches": int(launches), "kernels": kern, "clocks": clk.summary()}


def run_gpu_chunked(args):
    """Divide-and-conquer PQ over 64 lognormal chunks (Sec. 3): one step = pq_fit_chunked."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_2604_21645_gb300 import pqgb
    w = datagen.CHUNKED
    off = datagen.chunk_offsets(w)
    N = int(off[-1])
    X = datagen.mixture(N, w.d, w.n_comp, w.kind, w.seed)
    Xd = torch.from_numpy(X).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    offl = off.tolist()
    ctas, tune_ms = pqgb.tune_chunked(Xd, offl, w.m, w.ks, prec=args.prec)
    out = {}

    def step():
        out["r"] = pqgb.fit_chunked(Xd, offl, w.m, w.ks, iters=w.iters, seed=w.init_seed, prec=args.prec,
                                    want_rmse=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # the whole call (seeding, the persistent launch of every local pass, the global fit and the
    # encode) captured once as a CUDA graph; each timed step is one replay of it
    l0 = pqgb.launch_count()
    graph = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream()
    cs.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cs):
        with torch.cuda.graph(graph, stream=cs):
            step()
    torch.cuda.current_stream().wait_stream(cs)
    per_step = pqgb.launch_count() - l0
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms = _timed_steps(torch, graph.replay, args.steps, flush)
    launches = per_step * args.steps
    t = float(np.mean(ms)) / 1e3
    # per-kernel device times from the same call made eagerly (profiled): the dominant launch
    pqgb.profile_enable(True)
    ms_eager = _timed_steps(torch, step, args.steps, flush)
    kern = pqgb.profile_collect()
    pqgb.profile_enable(False)
    cb, codes, _ = out["r"]
    _, rmse = pqgb.decode_rmse(codes, cb, Xd)
    # e2e: rows from pinned host memory, codes and global codebooks back
    Xh = torch.from_numpy(X).pin_memory()
    Xe = torch.empty_like(Xd)
    codes_h = torch.empty(codes.shape, dtype=torch.uint8).pin_memory()
    cb_h = torch.empty(cb.shape, dtype=torch.float32).pin_memory()

    def step_e2e():
        Xe.copy_(Xh, non_blocking=True)
        c, k, _ = pqgb.fit_chunked(Xe, offl, w.m, w.ks, iters=w.iters, seed=w.init_seed, prec=args.prec,
                                   want_rmse=False)
        k_h = codes_h.copy_(k, non_blocking=True)
        cb_h.copy_(c, non_blocking=True)

    e2e = _timed_steps(torch, step_e2e, args.steps, flush)
    peaks, peak_src = load_peaks()
    pname = "pq_fit_persistent_tc" if args.prec == "bf16" else "pq_pass_f32"
    roof = None
    if pname == "pq_fit_persistent_tc" and pname in kern:
        # the dominant launch: every local Lloyd pass over all N rows, in one persistent launch
        secs = kern[pname]["ms"] / 1e3 / max(kern[pname]["launches"], 1)
        bound, work, unit, kind = kernel_work(pname, w, w.iters * N)
        roof = roofline_record(pname, bound, work, unit, kind, secs, peaks, peak_src, w.name,
                               kern[pname]["ms"] / max(sum(v["ms"] for v in kern.values()), 1e-9))
    elif pname in kern:
        # rows through the pass: every local iteration covers all N rows, the global fit the
        # n_chunks * Ks pooled codewords, the final encode N rows again
        n_launch = max(kern[pname]["launches"] // args.steps, 1)
        rows = w.iters * N + w.iters * len(offl[:-1]) * w.ks + N
        bound, work, unit, kind = kernel_work(pname, w, rows / n_launch, 1.0 / n_launch)
        secs = kern[pname]["ms"] / 1e3 / max(kern[pname]["launches"], 1)
        roof = roofline_record(pname, bound, work, unit, kind, secs, peaks, peak_src, w.name,
                               kern[pname]["ms"] / max(sum(v["ms"] for v in kern.values()), 1e-9))
    cfg = {"workload": w.name, "N": N, "n_chunks": w.n_chunks, "D": w.d, "M": w.m, "Ks": w.ks, "iters": w.iters,
           "chunk_rows": {"min": int(np.diff(off).min()), "median": int(np.median(np.diff(off))),
                          "max": int(np.diff(off).max())},
           "prec": args.prec, "tuned_ctas_per_group": ctas, "tuned_pass_ms": tune_ms, "parallelism": "replicas1",
           "graph": f"one CUDA graph replay per step ({per_step} kernel launches captured)",
           "eager_ms_per_step": float(np.mean(ms_eager)),
           "l2": f"256 MB buffer written between steps; X ({X.nbytes // 10**6} MB) exceeds L2"}
    line = _common_line(args, 1, "chunked PQ fit+encode Mvec/s", N / t / 1e6, "Mvec/s", t * 1e3,
                        "f32" if args.prec == "fp32" else "bf16", cfg, kern, launches, clk)
    line["rmse"] = rmse
    line["roofline"] = roof
    line["e2e"] = {"value": N / (float(np.mean(e2e)) / 1e3) / 1e6, "unit": "Mvec/s",
                   "h2d_bytes_per_step": int(X.nbytes), "d2h_bytes_per_step": int(codes.numel() + cb.numel() * 4)}
    if not args.no_cpu_baseline:
        import oracle as orc
        rows_c = 20_000
        off_s = np.arange(0, 4 * rows_c + 1, rows_c, dtype=np.int64)
        Xs = datagen.mixture(int(off_s[-1]), w.d, w.n_comp, w.kind, w.seed)
        t0 = time.perf_counter()
        orc.pq_fit_chunked(Xs, off_s, w.m, w.ks, w.iters, w.init_seed)
        tc = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": off_s[-1] / tc / 1e6, "unit": "Mvec/s", "cores": orc.num_threads(),
                                "kind": "oracle",
                                "sample": f"FP64 oracle pq_fit_chunked on 4 chunks of {rows_c} rows, {tc:.1f} s"}
    print(json.dumps(line), flush=True)


SOFTPQ_FLOPS_FWD = 34   # per (row, subspace, codeword): distance 16, exp 1, normaliser 1, soft reconstruction 16
SOFTPQ_FLOPS_BWD = 91   # recomputed weight 17, r.c 16, q 2, dX sum 16, dC sums 40


def run_gpu_softpq(args):
    """Soft-assignment refinement loss: one step = forward + backward (dL/dC and dL/dX)."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_2604_21645_gb300 import pqgb
    from paper_2604_21645_gb300.softpq import softpq_loss
    w = datagen.SOFTPQ
    X = w.data()
    Xd = torch.from_numpy(X).cuda()
    C0 = pqgb.fit(Xd, w.m, w.ks, iters=5, seed=w.init_seed, prec="bf16")  # starting codebooks, untimed
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    Xg = Xd.clone().requires_grad_(True)
    Cg = C0.clone().requires_grad_(True)
    out = {}

    def step():
        Xg.grad = None
        Cg.grad = None
        loss = softpq_loss(Xg, Cg, w.tau)
        loss.backward()
        out["loss"] = loss

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    l0 = pqgb.launch_count()
    pqgb.profile_enable(True)
    with ClockSampler(local) as clk:
        ms = _timed_steps(torch, step, args.steps, flush)
    launches = pqgb.launch_count() - l0
    kern = pqgb.profile_collect()
    pqgb.profile_enable(False)
    t = float(np.mean(ms)) / 1e3
    peaks, _ = load_peaks()
    scores = float(w.n) * w.m * w.ks
    roof = None
    dom = max(kern, key=lambda n: kern[n]["ms"]) if kern else None
    if dom in ("softpq_bwd", "softpq_fwd"):
        per = SOFTPQ_FLOPS_BWD if dom == "softpq_bwd" else SOFTPQ_FLOPS_FWD
        secs = kern[dom]["ms"] / 1e3 / max(kern[dom]["launches"], 1)
        ach = scores * per / secs / 1e12
        peak = fp32_peak_tflops(peaks)
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": measured_traffic(dom, w.name), "peak_source": "152 SMs x 128 FP32 lanes x 2 flop per FFMA x max SM clock",
                "avg_launch_ms": secs * 1e3,
                "share": kern[dom]["ms"] / max(sum(v["ms"] for v in kern.values()), 1e-9)}
    # e2e: rows and codebooks from pinned host memory, gradients and loss back
    Xh = torch.from_numpy(X).pin_memory()
    Ch = C0.cpu().pin_memory()
    dX_h = torch.empty_like(Xh).pin_memory()
    dC_h = torch.empty_like(Ch).pin_memory()
    loss_h = torch.empty((), dtype=torch.float32).pin_memory()

    def step_e2e():
        Xg.data.copy_(Xh, non_blocking=True)
        Cg.data.copy_(Ch, non_blocking=True)
        step()
        dX_h.copy_(Xg.grad, non_blocking=True)
        dC_h.copy_(Cg.grad, non_blocking=True)
        loss_h.copy_(out["loss"], non_blocking=True)

    e2e = _timed_steps(torch, step_e2e, args.steps, flush)
    cfg = {"workload": w.name, "N": w.n, "D": w.d, "M": w.m, "Ks": w.ks, "tau": w.tau, "parallelism": "replicas1",
           "l2": f"256 MB buffer written between steps; X ({X.nbytes // 10**6} MB) exceeds L2"}
    line = _common_line(args, 1, "soft-PQ loss forward+backward Mvec/s", w.n / t / 1e6, "Mvec/s", t * 1e3, "f32",
                        cfg, kern, launches, clk)
    line["loss"] = float(out["loss"].item())
    line["roofline"] = roof
    line["e2e"] = {"value": w.n / (float(np.mean(e2e)) / 1e3) / 1e6, "unit": "Mvec/s",
                   "h2d_bytes_per_step": int(X.nbytes + C0.numel() * 4),
                   "d2h_bytes_per_step": int(X.nbytes + C0.numel() * 4 + 4)}
    if not args.no_cpu_baseline:
        import oracle as orc
        rows = 2000
        Xs = X[:rows].astype(np.float64)
        Cs = C0.cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        orc.softpq_forward(Xs, Cs, w.tau)
        orc.softpq_backward(Xs, Cs, w.tau)
        tc = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": rows / tc / 1e6, "unit": "Mvec/s", "cores": 1, "kind": "oracle",
                                "sample": f"FP64 oracle softpq_forward + softpq_backward on the first {rows} rows, "
                                          f"{tc:.1f} s"}
    print(json.dumps(line), flush=True)


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


def _oracle_chunked_sample(w):
    import oracle as orc
    rows_c = 20_000
    off_s = np.arange(0, 4 * rows_c + 1, rows_c, dtype=np.int64)
    Xs = datagen.mixture(int(off_s[-1]), w.d, w.n_comp, w.kind, w.seed)
    t0 = time.perf_counter()
    orc.pq_fit_chunked(Xs, off_s, w.m, w.ks, w.iters, w.init_seed)
    return int(off_s[-1]), time.perf_counter() - t0, f"pq_fit_chunked on 4 chunks of {rows_c} rows"


def _oracle_softpq_sample(w):
    import oracle as orc
    rows = 2000
    Xs = w.data(rows).astype(np.float64)
    rng = np.random.default_rng(w.seed + 11)
    Cs = Xs[rng.integers(0, rows, size=w.ks)].reshape(w.ks, w.m, w.d // w.m).transpose(1, 0, 2).copy()
    t0 = time.perf_counter()
    orc.softpq_forward(Xs, Cs, w.tau)
    orc.softpq_backward(Xs, Cs, w.tau)
    return rows, time.perf_counter() - t0, f"softpq_forward + softpq_backward on {rows} rows"


def run_reference(args):
    """The FP64 oracle on the host cores, on a bounded sample of the same workload, per step."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import oracle as orc
    w = datagen.WORKLOADS[args.workload]
    if w.name == datagen.CHUNKED.name:
        sample, metric, cores = (lambda: _oracle_chunked_sample(w)), "chunked PQ fit+encode Mvec/s", orc.num_threads()
    elif w.name == datagen.SOFTPQ.name:
        sample, metric, cores = (lambda: _oracle_softpq_sample(w)), "soft-PQ loss forward+backward Mvec/s", 1
    else:
        rows = args.cpu_rows
        sample = lambda: (rows, oracle_fit_encode(w, rows), f"pq_fit + pq_encode on the first {rows} rows")
        metric = "PQ fit+encode Mvec/s (IVF-ADC queries/s reported beside it)"
        cores = orc.num_threads()
    for _ in range(args.warmup):
        sample()
    res = [sample() for _ in range(args.steps)]
    rows = res[0][0]
    t = float(np.mean([r[1] for r in res]))
    v = rows / t / 1e6
    print(json.dumps({
        "impl": "reference", "metric": metric, "value": v, "unit": "Mvec/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Gaussian mixture standing in for the paper's data)",
        "config": {"workload": w.name, "N": w.n, "D": w.d, "M": w.m, "Ks": w.ks, "iters": w.iters, "sample_rows": rows},
        "cpu_baseline": {"value": v, "unit": "Mvec/s", "cores": cores, "kind": "oracle",
                         "sample": f"FP64 oracle {res[0][2]} per step"},
        "e2e": {"value": v, "unit": "Mvec/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=datagen.PQ_10M.name,
                    choices=[datagen.PQ_10M.name, datagen.IVF_MEDIUM.name, datagen.CHUNKED.name, datagen.SOFTPQ.name])
    ap.add_argument("--prec", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--compare-fp32", action="store_true", help="medium pipeline: also time the plain FP32 form")
    ap.add_argument("--no-compare-fp32", action="store_true", help="precision form: skip the plain FP32 form")
    ap.add_argument("--no-search", action="store_true", help="precision form: skip the IVF-ADC search figures")
    ap.add_argument("--cpu-rows", type=int, default=300_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == datagen.CHUNKED.name:
        run_gpu_chunked(args)
    elif args.workload == datagen.SOFTPQ.name:
        run_gpu_softpq(args)
    elif args.workload == datagen.IVF_MEDIUM.name:
        run_gpu_pipeline(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
