#!/usr/bin/env python3
"""Benchmark of the CRISP GB300 engine (arXiv 2603.05180): QPS at recall@10 >= 0.95.

Workload (the paper's datasets are not available; synthetic rows of the Gist
shape stand in for them): N = 1,000,000 rows, D = 960, x = U diag(sqrt(l)) z
with l_i = i^-1.2 and U Haar-orthogonal (the CEV test triggers the rotation);
10,000 held-out queries from the same law; k = 10; M = 12 subspaces, K = 50
(the fastest M of a sweep over 12..32 at recall@10 >= 0.95).

A step is one crisp_search over the whole 10,000-query batch (Q1-Q7 of the
engine), inputs already resident in HBM; L2 (129 MB) is flushed by a 512 MB
write before every timed step, outside the timed events.  `value` is the
throughput of the plain FP32 engine at the operating point (mode, rho, alpha)
whose recall@10 on all 10,000 queries is reported beside it.  `e2e` is the
same metric through crisp_search_host (host buffers in, host buffers out,
copies inside the timed region).

Also printed: a roofline entry for the dominant kernel (algorithmic bytes per
launch over its CUDA-event duration, against the measured HBM copy bandwidth),
the CPU oracle timed on a bounded query sample on this machine's cores, SM
clocks sampled during the timed region, and the number of library kernels
launched inside it.

--impl reference times the CPU oracle itself on the same workload and
operating point (the reference arm of this benchmark).
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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "QPS at recall@10≥0.95 on 1 GB300 (plain FP32 vs learned+BF16), % HBM peak, p99 ms"
def workload_name(args):
    return (f"powerlaw N={args.n:,} D={args.dim} (lambda_i = i^-1.2, Haar mix), {args.nq:,} held-out queries, "
            f"k={args.k}, M={args.M} subspaces, K=50 centroids per half")
# operating point of the plain FP32 engine on this workload (recall@10 >= 0.95)
DEFAULT_POINT = dict(mode=0, rho=0.03, alpha=0.3)


def job_rate(torch, dist, dev, local_ms, units):
    """Whole-job rate over replicas: the slowest rank's time (max over ranks)
    and all ranks' units divided by it.  dist is torch.distributed or None."""
    total_ms = float(local_ms)
    if dist:
        tt = torch.tensor([total_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    return total_ms, units / (total_ms / 1e3)


def max_sm_mhz():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f).get("sm_max_mhz", 2070.0))
    return 2070.0


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# nominal dense tensor rates per GPU (PFLOP/s): TF32 is this fraction of BF16
TF32_PER_BF16 = 1.1 / 2.25


def bf16_peak():
    """BF16 tensor peak (TFLOP/s) for a kernel timed inside a long step: the
    measured sustained BF16 GEMM rate."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "measured"
    return 1700.0, "fallback"


def tf32_peak():
    """TF32 tensor peak (TFLOP/s) for a kernel timed inside a long step: the
    measured sustained BF16 GEMM rate times the nominal TF32 / BF16 ratio."""
    b, kind = bf16_peak()
    return b * TF32_PER_BF16, kind


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def start(self):
        self.tmp = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.tmp,
                                         stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.tmp.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.tmp.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------- ground truth
def ground_truth(torch, X, Q, k, extra=32):
    """Exact k-NN: FP32 expansion picks k+32 candidates, FP64 distances order them."""
    xn = (X * X).sum(1)
    nq = Q.shape[0]
    gd = torch.empty((nq, k), dtype=torch.float64, device=X.device)
    gi = torch.empty((nq, k), dtype=torch.int64, device=X.device)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    ch = max(1, min(1000, (1 << 30) // X.shape[0]))     # distance block of at most 4 GB
    for s in range(0, nq, ch):
        q = Q[s:s + ch]
        d = xn[None, :] - 2.0 * (q @ X.T)
        _, ci = torch.topk(d, k + extra, dim=1, largest=False)
        dd = ((X[ci].double() - q.double()[:, None, :]) ** 2).sum(-1)
        o = torch.argsort(dd, dim=1)[:, :k]
        gd[s:s + ch] = torch.gather(dd, 1, o)
        gi[s:s + ch] = torch.gather(ci, 1, o)
    torch.backends.cuda.matmul.allow_tf32 = prev
    return gi, gd


def recall_at_k(torch, X, Q, ids, gdk, rel=1e-5):
    """Tie-aware recall@k: a returned id counts if its FP64 distance is within (1 + rel) of the true k-th."""
    ids = ids.clone()
    valid = ids >= 0
    ids[~valid] = 0
    hits = 0
    for s in range(0, ids.shape[0], 2000):
        d = ((X[ids[s:s + 2000]].double() - Q[s:s + 2000].double()[:, None, :]) ** 2).sum(-1)
        hits += int(((d <= gdk[s:s + 2000, None] * (1 + rel)) & valid[s:s + 2000]).sum().item())
    return hits / (ids.shape[0] * ids.shape[1])


def d2_error(torch, X, Q, ids, d2):
    """Relative error of the returned FP32 squared distances against FP64
    distances recomputed from the original (unrotated) rows."""
    mx, tot, n = 0.0, 0.0, 0
    for s in range(0, ids.shape[0], 2000):
        i = ids[s:s + 2000]
        ok = i >= 0
        ex = ((X[i.clamp(min=0)].double() - Q[s:s + 2000].double()[:, None, :]) ** 2).sum(-1)
        rel = ((d2[s:s + 2000].double() - ex).abs() / ex.clamp(min=1e-30))[ok]
        if rel.numel():
            mx = max(mx, float(rel.max()))
            tot += float(rel.sum())
            n += rel.numel()
    return {"max_rel": mx, "mean_rel": tot / max(n, 1), "vs": "FP64 distances of the returned ids, original rows"}


def make_workload(args, device):
    import synthetic

    return synthetic.powerlaw(args.n, args.dim, args.nq, seed=args.seed, device=device)


# -------------------------------------------------------------- CPU oracle
def oracle_index(Xh, args):
    import oracle
    import synthetic

    draws = synthetic.method_draws(args.n, args.dim, args.M, 50, seed=args.seed)
    t = time.perf_counter()
    ix = oracle.build_index(Xh, M=args.M, draws=draws)
    return ix, time.perf_counter() - t


def oracle_time(ix, Qh, point, k, seconds):
    """Time the oracle's batched search on a bounded prefix of the queries."""
    import oracle

    p = oracle.SearchParams(k=k, mode=point["mode"], rho=point["rho"], alpha=point["alpha"])
    t = time.perf_counter()
    _, _, _, used = oracle.search(ix, Qh[:16], p)
    per_q = (time.perf_counter() - t) / 16
    n = int(max(16, min(Qh.shape[0], seconds / max(per_q, 1e-6))))
    t = time.perf_counter()
    _, _, _, used = oracle.search(ix, Qh[:n], p)
    dt = time.perf_counter() - t
    return n / dt, n, used, dt


# ---------------------------------------------------------------- arms
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch

    point = dict(DEFAULT_POINT)
    if args.mode is not None:
        point["mode"] = args.mode
    if args.rho is not None:
        point["rho"] = args.rho
    if args.alpha is not None:
        point["alpha"] = args.alpha
    device = "cuda" if torch.cuda.is_available() else "cpu"
    X, Q = make_workload(args, device)
    Xh = X.cpu().numpy() if device == "cuda" else X
    Qh = Q.cpu().numpy() if device == "cuda" else Q
    ix, build_s = oracle_index(Xh, args)
    import oracle

    p = oracle.SearchParams(k=args.k, mode=point["mode"], rho=point["rho"], alpha=point["alpha"])
    t = time.perf_counter()
    oracle.search(ix, Qh[:8], p)
    per_q = (time.perf_counter() - t) / 8
    nper = int(max(8, min(Qh.shape[0], args.ref_step_seconds / max(per_q, 1e-6))))
    times, used = [], 1
    for s in range(args.warmup + args.steps):
        lo = (s * nper) % max(1, Qh.shape[0] - nper + 1)
        t = time.perf_counter()
        _, _, _, used = oracle.search(ix, Qh[lo:lo + nper], p)
        if s >= args.warmup:
            times.append(time.perf_counter() - t)
    tot = sum(times)
    qps = nper * len(times) / tot
    sample = f"{nper} queries per step of the 10,000, on the oracle's own index (built in {build_s:.0f} s, not timed)"
    line = {"impl": "reference", "metric": METRIC, "value": qps, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args), **point, "k": args.k},
            "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": used, "kind": "oracle", "sample": sample},
            "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_crisp(args):
    import torch

    import paper_2603_05180_gb300 as crisp
    import synthetic

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream()
    peak, peak_kind = load_peaks()

    X, Q = make_workload(args, "cuda")
    N, D, nq, k = args.n, args.dim, args.nq, args.k
    draws = synthetic.method_draws(N, D, args.M, 50, seed=args.seed)
    torch.cuda.synchronize()
    t = time.perf_counter()
    ix = crisp.crisp_build(X, N, D, crisp.build_params(args.M, draws=draws, copies=3))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t
    info = ix.info()
    gi, gd = ground_truth(torch, X, Q, k)
    gdk = gd[:, k - 1].contiguous()

    ids = torch.empty((nq, k), dtype=torch.int64, device=dev)
    d2 = torch.empty((nq, k), dtype=torch.float32, device=dev)
    st = torch.empty((nq, 6), dtype=torch.int64, device=dev)

    def search(point, nqq=nq, Qx=Q, out=(ids, d2, st)):
        sp = crisp.search_params(k=k, mode=point["mode"], rho=point["rho"], alpha=point["alpha"],
                                 precision=point.get("precision", 0), shortlist=point.get("shortlist", 0),
                                 depth_margin=point.get("depth_margin", 0.0), short_margin=point.get("short_margin", 0.0))
        crisp.crisp_search(ix, Qx, nqq, sp, out[0][:nqq], out[1][:nqq], out[2][:nqq], stream)

    def timed(point, steps):
        for _ in range(3):
            search(point)
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            search(point)
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return nq * steps / (tot / 1e3), recall_at_k(torch, X, Q, ids, gdk), tot / steps

    # ---- operating point
    point = dict(DEFAULT_POINT)
    sweep_log = []
    if args.sweep:
        ns = 2000
        best = None
        for mode in (0, 1):
            for alpha in (0.1, 0.2, 0.3, 0.4, 0.5):
                for rho in (0.001, 0.002, 0.004, 0.007, 0.01, 0.015, 0.02, 0.03, 0.05):
                    pt = dict(mode=mode, rho=rho, alpha=alpha)
                    search(pt, ns)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    search(pt, ns)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    r = recall_at_k(torch, X, Q[:ns], ids[:ns], gdk[:ns])
                    q = ns / (e0.elapsed_time(e1) / 1e3)
                    sweep_log.append(dict(pt, recall=r, qps=q))
                    if r >= 0.955 and (best is None or q > best[1]):
                        best = (pt, q)
                    if r >= 0.995:
                        break
        if best:
            point = best[0]
    for key in ("mode", "rho", "alpha"):
        v = getattr(args, key)
        if v is not None:
            point[key] = v

    # ---- timed region: W warm-up steps, K timed steps, L2 flushed before each
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        search(point)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = crisp.crisp_kernel_launches()
    for s in range(args.steps):
        flush.zero_()
        ev[s][0].record(stream)
        search(point)
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    launches = crisp.crisp_kernel_launches() - launches0
    if dist:
        dist.barrier()
    clk = clocks.stop() if rank == 0 else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms, qps = job_rate(torch, dist, dev, sum(step_ms), world * nq * args.steps)
    rec = recall_at_k(torch, X, Q, ids, gdk)
    rec_sub = recall_at_k(torch, X, Q[:2000], ids[:2000], gdk[:2000])
    d2_err = d2_error(torch, X, Q, ids, d2)
    stats = st.cpu().numpy()

    # ---- stage-timed pass through the step entry points (same kernels, same launch shapes)
    stage = stage_pass(torch, crisp, ix, info, Q, point, k, args.steps, stream, flush)
    sl_stage = stage.pop("shortlist_bf16", None)
    shares = {n: v["ms"] for n, v in stage.items()}
    traffic_key = {"N": N, "D": D, "nq": nq, "M": args.M, "rho": point["rho"], "alpha": point["alpha"]}
    roofline, rooflines = stage_rooflines(stage, info, peak, peak_kind, traffic_key)
    roofline["stage_ms"] = {n: round(v, 4) for n, v in shares.items()}
    step_bytes = sum(v["bytes"] for v in stage.values())
    roofline_bf16 = None
    if sl_stage:
        a_bf = sl_stage["bytes"] / (sl_stage["ms"] / 1e3) / 1e9
        roofline_bf16 = {"kernel": sl_stage["kernel"], "bound": "hbm", "achieved": a_bf, "peak": peak, "unit": "GB/s",
                         "frac": a_bf / peak, "traffic": _ncu_traffic("shortlist_bf16", traffic_key),
                         "ms": round(sl_stage["ms"], 4), "algorithmic_bytes_per_launch": sl_stage["bytes"],
                         "note": "BF16 coarse scoring of the same candidates (the learned+BF16 path's shortlist "
                                 "step), shortlist of 50, timed on its own"}

    # ---- coarse-scoring variants (BF16 / FP8 rows, FP32 re-rank of a shortlist)
    variants = {}
    if not args.no_variants:
        ns = 2000
        for name, prec in (("bf16", 1), ("fp8", 2)):
            chosen = None
            for S in (50, 100, 200, 400, 800, 1600):
                pt = dict(point, precision=prec, shortlist=S)
                search(pt, ns)
                torch.cuda.synchronize()
                r = recall_at_k(torch, X, Q[:ns], ids[:ns], gdk[:ns])
                chosen = pt
                if r >= rec_sub - 0.002:
                    break
            q_v, r_v, ms_v = timed(chosen, args.steps)
            variants[name] = {"precision": name, "shortlist": chosen["shortlist"], "value": q_v, "recall_at_10": r_v,
                              "ms_per_step": ms_v, "speedup_vs_fp32": q_v / qps * world}

    leg_s = {}
    # ---- the same step with the re-rank bounds from one TF32 pass over the FP32
    # rows instead of one BF16 pass over the BF16 copy (identical results)
    tf32_rows = None
    if info.Xb:
        t_leg = time.perf_counter()
        os.environ["CRISP_RERANK_TF32"] = "1"
        try:
            q_t, r_t, ms_t = timed(point, args.steps)
        finally:
            del os.environ["CRISP_RERANK_TF32"]
        tf32_rows = {"value": q_t, "recall_at_10": r_t, "ms_per_step": ms_t,
                     "note": "re-rank bounds from one TF32 pass over the FP32 rows (CRISP_RERANK_TF32=1); the "
                             "headline value takes them from one BF16 pass over the index's BF16 copy; both return "
                             "the exact FP32 (CR32) top-k"}
        leg_s["tf32_rows"] = time.perf_counter() - t_leg

    # ---- learned depths + BF16 (F1): train the model on queries of the same law
    learned = None
    if not args.no_learned:
        t_leg = time.perf_counter()
        learned = learned_leg(torch, crisp, synthetic, ix, info, X, args, point, search, timed, qps, world, dev)
        leg_s["learned"] = time.perf_counter() - t_leg

    # ---- both modes at k = 10 and k = 100 on the same index
    modes = None
    if not args.no_modes:
        t_leg = time.perf_counter()
        modes = modes_leg(torch, crisp, ix, X, Q, args, dev)
        leg_s["modes"] = time.perf_counter() - t_leg

    # ---- the vMF (D = 3072) and low-rank (D = 4096) configurations, each on its
    # own index (with --full or their own flags: several minutes each)
    big = {}
    if world == 1:
        if args.vmf or (args.full and not args.no_vmf):
            t_leg = time.perf_counter()
            big["vmf_3072"] = vmf_leg(args, torch, crisp, synthetic, dev, flush, stream)
            leg_s["vmf_3072"] = time.perf_counter() - t_leg
        if args.lowrank or (args.full and not args.no_lowrank):
            t_leg = time.perf_counter()
            big["lowrank_4096"] = lowrank_leg(args, torch, crisp, synthetic, dev, flush, stream)
            leg_s["lowrank_4096"] = time.perf_counter() - t_leg

    # ---- continuous-batching serving (its own 5M x 1024 index; --full or --serve)
    serving = None
    if (args.serve or (args.full and not args.no_serve)) and world == 1:
        t_leg = time.perf_counter()
        serving = serving_leg(args, torch, crisp, synthetic, dev)
        leg_s["serving"] = time.perf_counter() - t_leg

    # ---- end to end through the host-buffer entry point
    Qh = torch.empty((nq, D), dtype=torch.float32, pin_memory=True)
    Qh.copy_(Q.cpu())
    ih = torch.empty((nq, k), dtype=torch.int64, pin_memory=True)
    dh = torch.empty((nq, k), dtype=torch.float32, pin_memory=True)
    sp = crisp.search_params(k=k, mode=point["mode"], rho=point["rho"], alpha=point["alpha"])
    crisp.crisp_search_host(ix, Qh, nq, sp, ih, dh, None, stream)
    e2e_t = []
    for s in range(max(3, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        crisp.crisp_search_host(ix, Qh, nq, sp, ih, dh, None, stream)
        e2e_t.append(time.perf_counter() - t)
    _, e2e_qps = job_rate(torch, dist, dev, 1e3 * sum(e2e_t), world * nq * len(e2e_t))

    # ---- CPU oracle baseline (rank 0, one GPU only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        Xh, Qhn = X.cpu().numpy(), Q.cpu().numpy()
        ixo, obuild = oracle_index(Xh, args)
        v, n, used, dt = oracle_time(ixo, Qhn, point, k, args.cpu_seconds)
        cpu = {"value": v, "unit": "queries/s", "cores": used, "kind": "oracle",
               "sample": f"first {n} of the 10,000 queries ({dt:.1f} s), on the oracle's own index of the same rows "
                         f"and draws (built in {obuild:.0f} s, not timed)"}

    if rank == 0:
        mode_name = "guaranteed" if point["mode"] == 0 else "optimized"
        line = {"metric": METRIC, "value": qps, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": workload_name(args), "N": N, "D": D, "nq": nq, "k": k, "M": args.M, "K": 50,
                           "mode": mode_name, "rho": point["rho"], "alpha": point["alpha"],
                           "parallelism": "replicas" if world > 1 else "single",
                           "l2": "flushed before every timed step (512 MB write, outside the timed events)",
                           "index_rotated": bool(info.rotated), "cev": info.cev, "build_s": round(build_s, 3)},
                "recall_at_10": rec, "sqdist_error": d2_err,
                "step_p50_ms": statistics.median(step_ms), "step_p99_ms": float(np.percentile(step_ms, 99)),
                "query_bytes_rate_vs_hbm": step_bytes / (total_ms / args.steps / 1e3) / 1e9 / peak,
                "query_bytes_note": "per-query algorithmic bytes of every stage (each candidate row counted once per "
                                    "query) over the step time, against the HBM copy peak: a reuse figure, not an "
                                    "HBM fraction (rows shared by a query group are fetched once)",
                "candidates_mean": float(stats[:, 0].mean()), "full_distances_mean": float(stats[:, 2].mean()),
                "roofline": roofline, "rooflines": rooflines, "roofline_bf16": roofline_bf16, "cpu_baseline": cpu,
                "e2e": {"value": e2e_qps, "unit": "queries/s", "h2d_bytes_per_step": nq * D * 4,
                        "d2h_bytes_per_step": nq * k * 12},
                "gpu_launches": launches, "clocks": clk,
                "coarse_scoring": variants, "learned_bf16": learned, "modes": modes, "tf32_rows": tf32_rows,
                "leg_seconds": leg_s, **big}
        if tf32_rows:   # the low-precision forms against the plain path that reads only the FP32 rows
            for v in list(variants.values()) + ([learned] if learned else []):
                v["speedup_vs_fp32_rows_only"] = v["value"] / tf32_rows["value"]
        if serving:
            ok = [r for r in serving["rates"] if r["achieved_qps"] >= 0.95 * r["offered_qps"]] or serving["rates"][:1]
            top = max(ok, key=lambda r: r["offered_qps"])
            line["p50_ms"], line["p99_ms"] = top["p50_ms"], top["p99_ms"]
            line["latency_note"] = (f"p50/p99: per-request latency of the serving loop at {top['offered_qps']} "
                                    "requests/s offered (the highest rate it sustained), see serving; step_p50/p99: "
                                    "one 10,000-query batch")
        line["serving"] = serving
        if sweep_log:
            line["sweep"] = sweep_log
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def learned_leg(torch, crisp, synthetic, ix, info, X, args, point, search, timed, plain_qps, world, dev):
    """Learned re-rank depths with BF16 coarse scores: labels from the plain
    search on training queries, GPU training, margins calibrated on validation
    queries to the plain path's recall, then timed on the evaluation queries."""
    N, D, k = args.n, args.dim, args.k
    M, F, H = info.M, 2 * info.M + 68, 256
    ntr, nva = args.train_queries, 2000
    _, Qtr = synthetic.powerlaw(1, D, ntr, seed=args.seed, device="cuda", query_sub=synthetic.SUB_TRAIN)
    _, Qva = synthetic.powerlaw(1, D, nva, seed=args.seed, device="cuda", query_sub=synthetic.SUB_VALID)
    sp = crisp.search_params(k=k, mode=0, rho=point["rho"], alpha=point["alpha"])
    feats = torch.empty((ntr, F), dtype=torch.float32, device=dev)
    labels = torch.empty((ntr, 2), dtype=torch.int64, device=dev)
    tg = torch.empty((ntr, 2), dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    crisp.crisp_learned_data(ix, Qtr, ntr, sp, feats, labels, tg)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    P = torch.empty(crisp.crisp_mlp_param_count(F, H, 2), dtype=torch.float32, device=dev)
    crisp.crisp_mlp_init(P, F, H, 2, seed=args.seed + 1)
    t0 = time.perf_counter()
    losses = crisp.crisp_mlp_train(P, F, H, 2, feats, tg, ntr, args.epochs, 1024, 1e-3, seed=args.seed + 2)
    t_train = time.perf_counter() - t0
    crisp.crisp_index_set_model(ix, P, H)
    # calibrate the margins on validation queries against the plain path's recall there
    _, gdv = ground_truth(torch, X, Qva, k)
    gdv = gdv[:, k - 1].contiguous()
    vi = torch.empty((nva, k), dtype=torch.int64, device=dev)
    vd = torch.empty((nva, k), dtype=torch.float32, device=dev)
    vs = torch.empty((nva, 6), dtype=torch.int64, device=dev)
    def val(pt):
        sp2 = crisp.search_params(k=k, mode=pt["mode"], rho=pt["rho"], alpha=pt["alpha"],
                                  depth_margin=pt.get("depth_margin", 0.0), short_margin=pt.get("short_margin", 0.0))
        crisp.crisp_search(ix, Qva, nva, sp2, vi, vd, vs)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        crisp.crisp_search(ix, Qva, nva, sp2, vi, vd, vs)
        b.record()
        torch.cuda.synchronize()
        return recall_at_k(torch, X, Qva, vi, gdv), nva / (a.elapsed_time(b) / 1e3)
    r_plain, _ = val(point)
    best = None
    for dm in (0.0, 0.5, 1.0, 1.5, 2.0, 3.0):
        for sm in (0.0, 1.0, 2.0):
            pt = dict(point, mode=2, depth_margin=dm, short_margin=sm)
            r, q = val(pt)
            if r >= max(r_plain - 0.002, 0.95) and (best is None or q > best[1]):
                best = (pt, q, r)
    if best is None:
        return {"status": "no margin reached the plain recall on the validation queries", "val_recall_plain": r_plain}
    pt = best[0]
    q_l, r_l, ms_l = timed(pt, args.steps)
    return {"value": q_l, "recall_at_10": r_l, "ms_per_step": ms_l, "speedup_vs_fp32": q_l / plain_qps * world,
            "depth_margin": pt["depth_margin"], "short_margin": pt["short_margin"], "train_queries": ntr,
            "epochs": args.epochs, "hidden": H, "features": F, "loss_first_epoch": losses[0],
            "loss_last_epoch": losses[-1], "label_seconds": round(t_data, 2), "train_seconds": round(t_train, 2),
            "val_recall_plain": r_plain, "val_recall_learned": best[2]}


def _search_fn(torch, crisp, ix, dev):
    """search(Qx, pt, out) -> None, and a timed(Qx, pt, steps) -> (qps, ms) helper for a leg's own index."""
    def search(Qx, pt, ids, d2, st=None):
        sp = crisp.search_params(k=pt["k"], mode=pt["mode"], rho=pt["rho"], alpha=pt["alpha"],
                                 precision=pt.get("precision", 0), shortlist=pt.get("shortlist", 0),
                                 depth_margin=pt.get("depth_margin", 0.0), short_margin=pt.get("short_margin", 0.0),
                                 patience_factor=pt.get("patience_factor", 40),
                                 max_candidates=pt.get("max_candidates", 0))
        crisp.crisp_search(ix, Qx, Qx.shape[0], sp, ids, d2, st)

    def timed(Qx, pt, ids, d2, steps, flush):
        search(Qx, pt, ids, d2)
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            search(Qx, pt, ids, d2)
            b.record()
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return Qx.shape[0] * steps / (tot / 1e3), tot / steps

    return search, timed


def _ladder(torch, X, Qv, gdv, search, pts, k, dev, target=0.955):
    """Recall on the validation queries along a ladder of points; the fastest
    reaching the target, else the one of highest recall."""
    n = Qv.shape[0]
    ids = torch.empty((n, k), dtype=torch.int64, device=dev)
    d2 = torch.empty((n, k), dtype=torch.float32, device=dev)
    log, best = [], None
    for pt in pts:
        search(Qv, pt, ids, d2)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        search(Qv, pt, ids, d2)
        b.record()
        torch.cuda.synchronize()
        r = recall_at_k(torch, X, Qv, ids, gdv)
        q = n / (a.elapsed_time(b) / 1e3)
        log.append(dict(pt, recall=r, qps=q))
        ok = r >= target
        if best is None or (ok and (not best[2] or q > best[1])) or (not ok and not best[2] and r > best[3]):
            best = (pt, q, ok, r)
    return best[0], best[2], log


def modes_leg(torch, crisp, ix, X, Q, args, dev):
    """Guaranteed and Optimized modes at k = 10 and k = 100 on the headline
    index (§4.3.2 Stages 2-3, §6.3): for each, the fastest point of a ladder
    (coverage, threshold; for Optimized also the patience factor) whose
    recall@k on 2,000 validation queries reaches 0.955, timed on the 10,000
    evaluation queries."""
    import synthetic

    _, Qva = synthetic.powerlaw(1, args.dim, 2000, seed=args.seed, device="cuda", query_sub=synthetic.SUB_VALID)
    _, gd = ground_truth(torch, X, Q, 100)
    _, gdv = ground_truth(torch, X, Qva, 100)
    search, timed = _search_fn(torch, crisp, ix, dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    out = {}
    nq = Q.shape[0]
    for k in (10, 100):
        ids = torch.empty((nq, k), dtype=torch.int64, device=dev)
        d2 = torch.empty((nq, k), dtype=torch.float32, device=dev)
        for mode, name in ((0, "guaranteed"), (1, "optimized")):
            if mode == 0:
                pts = [dict(k=k, mode=0, rho=r_, alpha=a_) for r_, a_ in
                       ((0.01, 0.3), (0.02, 0.3), (0.03, 0.3), (0.04, 0.3), (0.03, 0.25), (0.05, 0.25), (0.08, 0.2))]
            else:
                pts = [dict(k=k, mode=1, rho=r_, alpha=a_, patience_factor=pf, max_candidates=OPT_CAP)
                       for r_, a_ in ((0.01, 0.3), (0.02, 0.3), (0.03, 0.3), (0.04, 0.3), (0.05, 0.25))
                       for pf in (40, 100, 200, 400)]
            pt, ok, log = _ladder(torch, X, Qva, gdv[:, k - 1].contiguous(), search, pts, k, dev)
            q, ms = timed(Q, pt, ids, d2, min(args.steps, 5), flush)
            r = recall_at_k(torch, X, Q, ids, gd[:, k - 1].contiguous())
            out[f"{name}_k{k}"] = {"value": q, "unit": "queries/s", f"recall_at_{k}": r, "ms_per_step": ms,
                                   "point": pt, "reached_0_95": ok, "ladder": log}
    del flush
    return out


VMF_WORKLOAD = ("vMF N=1,000,000 D=3072 unit rows, 1,000 components, kappa=200 (Wood's sampler), 10,000 queries, "
                "k=10, M=16 subspaces, K=50")
LOWRANK_WORKLOAD = ("low-rank N=2,000,000 D=4096, rank-128 N(0,1) loadings, noise 0.05, 5% of dims x10 variance, "
                    "10,000 queries, k=10, M=16 subspaces, K=50")


def vmf_leg(args, torch, crisp, synthetic, dev, flush, stream):
    """Learned early termination + BF16 coarse scoring on near-isotropic unit
    rows (D = 3072): plain FP32 at the fastest point reaching recall@10 0.955 on
    validation queries (or the highest recall its ladder reaches, reported as
    such), the MLP trained on method-generated queries, then the learned+BF16
    path at the plain path's recall.  Each on its own index."""
    N, D, M, k = args.vmf_n, 3072, 16, 10
    seed = args.seed
    t0 = time.perf_counter()
    X, Q = synthetic.vmf(N, D, args.nq, seed=seed, device="cuda")
    _, Qva = synthetic.vmf(1, D, 2000, seed=seed, device="cuda", query_sub=synthetic.SUB_VALID)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    ix = crisp.crisp_build(X, N, D, crisp.build_params(M, draws=synthetic.method_draws(N, D, M, 50, seed=seed),
                                                       copies=1))
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    info = ix.info()
    _, gd = ground_truth(torch, X, Q, k)
    _, gdv = ground_truth(torch, X, Qva, k)
    gdk, gdvk = gd[:, k - 1].contiguous(), gdv[:, k - 1].contiguous()
    search, timed = _search_fn(torch, crisp, ix, dev)
    pts = [dict(k=k, mode=0, rho=r_, alpha=a_) for r_, a_ in
           ((0.02, 0.25), (0.05, 0.25), (0.05, 0.125), (0.1, 0.125), (0.2, 0.125), (0.3, 0.0625))]
    pt, ok, log = _ladder(torch, X, Qva, gdvk, search, pts, k, dev)
    nq = Q.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int64, device=dev)
    d2 = torch.empty((nq, k), dtype=torch.float32, device=dev)
    st = torch.empty((nq, 6), dtype=torch.int64, device=dev)
    steps = min(args.steps, 5)
    q_p, ms_p = timed(Q, pt, ids, d2, steps, flush)
    r_p = recall_at_k(torch, X, Q, ids, gdk)
    search(Q, pt, ids, d2, st)
    cands = float(st[:, 0].double().mean())
    stage = stage_pass(torch, crisp, ix, info, Q, pt, k, steps, stream, flush)
    stage.pop("shortlist_bf16", None)
    peak, peak_kind = load_peaks()
    roof, roofs = stage_rooflines(stage, info, peak, peak_kind, None)
    # learned depths: labels from the plain search on method-generated training queries
    F, H = 2 * M + 68, 256
    ntr = args.vmf_train
    t0 = time.perf_counter()
    _, Qtr = synthetic.vmf(1, D, ntr, seed=seed, device="cuda", query_sub=synthetic.SUB_TRAIN)
    feats = torch.empty((ntr, F), dtype=torch.float32, device=dev)
    labels = torch.empty((ntr, 2), dtype=torch.int64, device=dev)
    tg = torch.empty((ntr, 2), dtype=torch.float32, device=dev)
    crisp.crisp_learned_data(ix, Qtr, ntr, crisp.search_params(k=k, mode=0, rho=pt["rho"], alpha=pt["alpha"]), feats,
                             labels, tg)
    torch.cuda.synchronize()
    t_labels = time.perf_counter() - t0
    del Qtr
    P = torch.empty(crisp.crisp_mlp_param_count(F, H, 2), dtype=torch.float32, device=dev)
    crisp.crisp_mlp_init(P, F, H, 2, seed=seed + 1)
    t0 = time.perf_counter()
    losses = crisp.crisp_mlp_train(P, F, H, 2, feats, tg, ntr, args.epochs, 1024, 1e-3, seed=seed + 2)
    t_train = time.perf_counter() - t0
    del feats, labels, tg
    crisp.crisp_index_set_model(ix, P, H)
    vi = torch.empty((Qva.shape[0], k), dtype=torch.int64, device=dev)
    vd = torch.empty((Qva.shape[0], k), dtype=torch.float32, device=dev)
    search(Qva, pt, vi, vd)
    r_vplain = recall_at_k(torch, X, Qva, vi, gdvk)
    lpts = [dict(pt, mode=2, depth_margin=dm, short_margin=sm) for dm in (0.0, 0.5, 1.0, 2.0, 3.0)
            for sm in (0.0, 1.0, 2.0)]
    lpt, lok, llog = _ladder(torch, X, Qva, gdvk, search, lpts, k, dev, target=r_vplain - 0.002)
    q_l, ms_l = timed(Q, lpt, ids, d2, steps, flush)
    r_l = recall_at_k(torch, X, Q, ids, gdk)
    out = {"workload": VMF_WORKLOAD, "index_rotated": bool(info.rotated), "cev": info.cev,
           "data_s": round(t_data, 2), "build_s": round(t_build, 2),
           "plain_fp32": {"value": q_p, "unit": "queries/s", "recall_at_10": r_p, "ms_per_step": ms_p, "point": pt,
                          "reached_0_95": ok, "candidates_mean": cands, "ladder": log},
           "learned_bf16": {"value": q_l, "unit": "queries/s", "recall_at_10": r_l, "ms_per_step": ms_l,
                            "speedup_vs_fp32": q_l / q_p, "depth_margin": lpt["depth_margin"],
                            "short_margin": lpt["short_margin"], "matched_plain_recall": lok,
                            "train_queries": ntr, "epochs": args.epochs, "loss_first_epoch": losses[0],
                            "loss_last_epoch": losses[-1], "label_seconds": round(t_labels, 2),
                            "train_seconds": round(t_train, 2)},
           "roofline": roof, "rooflines": roofs,
           "stage_ms": {n: round(v["ms"], 4) for n, v in stage.items()}}
    ix.free()
    del X, Q, Qva, gd, gdv, ids, d2, st, vi, vd
    torch.cuda.empty_cache()
    return out


def lowrank_leg(args, torch, crisp, synthetic, dev, flush, stream):
    """FP8 E4M3 coarse scoring with per-row scales and an FP32 re-rank of the
    shortlist on low-rank rows (D = 4096, the CEV test rotates them), against
    the plain FP32 path at the same recall; its own index."""
    N, D, M, k = args.lowrank_n, 4096, 16, 10
    seed = args.seed
    t0 = time.perf_counter()
    X, Q = synthetic.lowrank(N, D, args.nq, seed=seed, device="cuda")
    _, Qva = synthetic.lowrank(1, D, 2000, seed=seed, device="cuda", query_sub=synthetic.SUB_VALID)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    ix = crisp.crisp_build(X, N, D, crisp.build_params(M, draws=synthetic.method_draws(N, D, M, 50, seed=seed),
                                                       copies=3))
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    info = ix.info()
    _, gd = ground_truth(torch, X, Q, k)
    _, gdv = ground_truth(torch, X, Qva, k)
    gdk, gdvk = gd[:, k - 1].contiguous(), gdv[:, k - 1].contiguous()
    search, timed = _search_fn(torch, crisp, ix, dev)
    pts = [dict(k=k, mode=0, rho=r_, alpha=a_) for r_, a_ in
           ((0.01, 0.25), (0.02, 0.25), (0.05, 0.2), (0.1, 0.15), (0.15, 0.125), (0.2, 0.125), (0.3, 0.0625))]
    pt, ok, log = _ladder(torch, X, Qva, gdvk, search, pts, k, dev)
    nq = Q.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int64, device=dev)
    d2 = torch.empty((nq, k), dtype=torch.float32, device=dev)
    st = torch.empty((nq, 6), dtype=torch.int64, device=dev)
    steps = min(args.steps, 5)
    q_p, ms_p = timed(Q, pt, ids, d2, steps, flush)
    r_p = recall_at_k(torch, X, Q, ids, gdk)
    search(Q, pt, ids, d2, st)
    cands = float(st[:, 0].double().mean())
    vi = torch.empty((Qva.shape[0], k), dtype=torch.int64, device=dev)
    vd = torch.empty((Qva.shape[0], k), dtype=torch.float32, device=dev)
    search(Qva, pt, vi, vd)
    r_vplain = recall_at_k(torch, X, Qva, vi, gdvk)
    fpts = [dict(pt, precision=2, shortlist=S) for S in (50, 100, 200, 400, 800, 1600)]
    fpt, fok, flog = _ladder(torch, X, Qva, gdvk, search, fpts, k, dev, target=r_vplain - 0.002)
    q_f, ms_f = timed(Q, fpt, ids, d2, steps, flush)
    r_f = recall_at_k(torch, X, Q, ids, gdk)
    stage = stage_pass(torch, crisp, ix, info, Q, pt, k, steps, stream, flush)
    stage.pop("shortlist_bf16", None)
    peak, peak_kind = load_peaks()
    roof, roofs = stage_rooflines(stage, info, peak, peak_kind, None)
    out = {"workload": LOWRANK_WORKLOAD, "index_rotated": bool(info.rotated), "cev": info.cev,
           "data_s": round(t_data, 2), "build_s": round(t_build, 2),
           "plain_fp32": {"value": q_p, "unit": "queries/s", "recall_at_10": r_p, "ms_per_step": ms_p, "point": pt,
                          "reached_0_95": ok, "candidates_mean": cands, "ladder": log},
           "fp8_e4m3": {"value": q_f, "unit": "queries/s", "recall_at_10": r_f, "ms_per_step": ms_f,
                        "shortlist": fpt["shortlist"], "speedup_vs_fp32": q_f / q_p, "matched_plain_recall": fok,
                        "ladder": flog},
           "roofline": roof, "rooflines": roofs,
           "stage_ms": {n: round(v["ms"], 4) for n, v in stage.items()}}
    ix.free()
    del X, Q, Qva, gd, gdv, ids, d2, st, vi, vd
    torch.cuda.empty_cache()
    return out


SERVE_WORKLOAD = ("serving: powerlaw N=5,000,000 D=1024 (lambda_i = i^-1.2, Haar mix), M=32; open-loop Poisson "
                  "arrivals; k in {1, 10, 100} uniform; mode Guaranteed : Optimized : Learned = 1 : 2 : 2")


OPT_CAP = 32768        # Optimized mode keeps at most this many candidates (the paper's optional cap)


def serving_leg(args, torch, crisp, synthetic, dev):
    """Continuous batching on the 5M x 1024 index: open-loop Poisson traces of
    mixed k and modes replayed through the server (native replay, so arrivals
    keep their schedule at any rate) at several offered rates.  Reports the
    per-request latency (scheduled arrival -> result on the host), throughput,
    batching and recall@k per class."""
    N, D, M, k10 = args.serve_n, args.serve_dim, args.serve_M, 10
    seed = args.seed + 1
    t0 = time.perf_counter()
    X, Qp = synthetic.powerlaw(N, D, args.serve_pool, seed=seed, device="cuda")
    _, Qva = synthetic.powerlaw(1, D, 1000, seed=seed, device="cuda", query_sub=synthetic.SUB_VALID)
    _, Qtr = synthetic.powerlaw(1, D, args.serve_train, seed=seed, device="cuda", query_sub=synthetic.SUB_TRAIN)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    ix = crisp.crisp_build(X, N, D, crisp.build_params(M, draws=synthetic.method_draws(N, D, M, 50, seed=seed),
                                                       copies=1))
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    info = ix.info()
    gi, gd = ground_truth(torch, X, Qp, 100)
    _, gdv = ground_truth(torch, X, Qva, k10)
    gdv = gdv[:, k10 - 1].contiguous()
    nva = Qva.shape[0]
    vi = torch.empty((nva, k10), dtype=torch.int64, device=dev)
    vd = torch.empty((nva, k10), dtype=torch.float32, device=dev)

    def val(sp):
        crisp.crisp_search(ix, Qva, nva, sp, vi, vd)
        torch.cuda.synchronize()
        return recall_at_k(torch, X, Qva, vi, gdv)

    # coverage / threshold: the cheapest rung of the ladder whose Guaranteed recall@10 reaches 0.955
    rho, alpha = 0.03, 0.3
    for r_, a_ in ((0.01, 0.2), (0.015, 0.2), (0.02, 0.2), (0.025, 0.25), (0.03, 0.25)):
        if val(crisp.search_params(k=k10, mode=0, rho=r_, alpha=a_)) >= 0.955:
            rho, alpha = r_, a_
            break
    # learned depths for this index (labels from its own plain search, trained on the GPU)
    F, H = 2 * M + 68, 256
    ntr = Qtr.shape[0]
    feats = torch.empty((ntr, F), dtype=torch.float32, device=dev)
    labels = torch.empty((ntr, 2), dtype=torch.int64, device=dev)
    tg = torch.empty((ntr, 2), dtype=torch.float32, device=dev)
    crisp.crisp_learned_data(ix, Qtr, ntr, crisp.search_params(k=k10, mode=0, rho=rho, alpha=alpha), feats, labels, tg)
    P = torch.empty(crisp.crisp_mlp_param_count(F, H, 2), dtype=torch.float32, device=dev)
    crisp.crisp_mlp_init(P, F, H, 2, seed=seed + 1)
    crisp.crisp_mlp_train(P, F, H, 2, feats, tg, ntr, args.epochs, 1024, 1e-3, seed=seed + 2)
    crisp.crisp_index_set_model(ix, P, H)
    del feats, labels, tg
    r_plain = val(crisp.search_params(k=k10, mode=0, rho=rho, alpha=alpha))
    dm = 3.0
    for d_ in (1.0, 2.0):
        if val(crisp.search_params(k=k10, mode=2, rho=rho, alpha=alpha, depth_margin=d_)) >= r_plain - 0.002:
            dm = d_
            break
    val_rec = {"guaranteed": r_plain,
               "optimized": val(crisp.search_params(k=k10, mode=1, rho=rho, alpha=alpha, max_candidates=OPT_CAP)),
               "learned": val(crisp.search_params(k=k10, mode=2, rho=rho, alpha=alpha, depth_margin=dm))}

    modes = (0, 1, 1, 2, 2)                       # Guaranteed : Optimized : Learned = 1 : 2 : 2
    ks = (1, 10, 100)
    params = [crisp.search_params(k=kk, mode=m, rho=rho, alpha=alpha, depth_margin=dm if m == 2 else 0.0,
                                  max_candidates=OPT_CAP if m == 1 else 0)
              for m in (0, 1, 2) for kk in ks]
    Qh = Qp.cpu().numpy()
    rng = np.random.default_rng(seed + 5)
    sv = crisp.crisp_server_create(ix, streams=args.serve_streams, max_batch=args.serve_batch)

    def trace(rate, n):
        arr = np.cumsum(rng.exponential(1e6 / rate, n))
        qidx = rng.integers(0, Qh.shape[0], n).astype(np.int32)
        m = np.array(modes)[rng.integers(0, len(modes), n)]
        kk = rng.integers(0, 3, n)
        return arr, qidx, (m * 3 + kk).astype(np.int32)

    arr, qidx, pidx = trace(20000, 2000)            # warm-up: pools, plans, pinned buffers
    crisp.crisp_server_replay(sv, Qh, qidx, params, pidx, arr, 100)
    # capacity: a burst of requests that all arrive at once (largest batches)
    arr, qidx, pidx = trace(1e9, args.serve_burst)
    _, _, _, wall = crisp.crisp_server_replay(sv, Qh, qidx, params, pidx, np.zeros(args.serve_burst), 100)
    capacity = args.serve_burst / (wall / 1e6)
    offered = sorted(set(list(args.serve_rates) + [int(f * capacity) for f in (0.25, 0.5, 0.75, 0.9)]))
    rates = []
    for rate in offered:
        n = int(min(args.serve_max_requests, rate * args.serve_seconds))
        arr, qidx, pidx = trace(rate, n)
        crisp.crisp_server_reset_stats(sv)
        ids, d2, lat, wall = crisp.crisp_server_replay(sv, Qh, qidx, params, pidx, arr, 100)
        st = crisp.crisp_server_get_stats(sv)
        idt = torch.from_numpy(ids).to(dev)
        qi = torch.from_numpy(qidx.astype(np.int64)).to(dev)
        rec_k, rec_m = {}, {}
        for j, kk in enumerate(ks):
            sel = torch.from_numpy(np.nonzero(pidx % 3 == j)[0]).to(dev)
            if sel.numel():
                rec_k[str(kk)] = recall_at_k(torch, X, Qp[qi[sel]], idt[sel, :kk].contiguous(),
                                             gd[qi[sel], kk - 1].contiguous())
        for mi, name in enumerate(("guaranteed", "optimized", "learned")):
            sel = torch.from_numpy(np.nonzero(pidx == mi * 3 + 1)[0]).to(dev)
            if sel.numel():
                rec_m[name] = recall_at_k(torch, X, Qp[qi[sel]], idt[sel, :k10].contiguous(),
                                          gd[qi[sel], k10 - 1].contiguous())
        rates.append({"offered_qps": rate, "requests": n, "achieved_qps": n / (wall / 1e6),
                      "p50_ms": float(np.percentile(lat, 50)) / 1e3, "p99_ms": float(np.percentile(lat, 99)) / 1e3,
                      "max_ms": float(lat.max()) / 1e3, "batches": int(st.batches), "mean_batch": st.mean_batch,
                      "failed": int(st.failed), "recall_at_k": rec_k, "recall_at_10_by_mode": rec_m})
    sv.free()
    out = {"workload": SERVE_WORKLOAD, "N": N, "D": D, "M": M, "rho": rho, "alpha": alpha,
           "learned_depth_margin": dm, "learned_train_queries": ntr, "query_pool": Qh.shape[0],
           "streams": args.serve_streams, "max_batch": args.serve_batch, "index_rotated": bool(info.rotated),
           "data_s": round(t_data, 2), "build_s": round(t_build, 2), "val_recall_at_10": val_rec,
           "capacity_qps": capacity, "capacity_note": f"{args.serve_burst} requests arriving at once",
           "latency": "scheduled arrival -> result in host memory, per request", "rates": rates}
    del ix, X, Qp, gi, gd
    torch.cuda.empty_cache()
    return out


TAU_POINTS = {"low": dict(rho=0.02, alpha=0.25), "high": dict(rho=0.1, alpha=0.2)}


def run_ablation(args):
    """The paper's ablations (§6, "Ablation Study") on the synthetic workloads:
    (1) the rotation threshold tau_CEV: per dataset its CEV, and recall@100 and
    QPS with the rotation forced off and on, then what each tau_CEV would
    choose; (2) the patience factor of the Optimized mode (20 / 40 / 60);
    (3) the verification sub-components: full (Hamming order + ADSampling),
    exact L2 (ADSampling off, eps0 = inf) and id order (Hamming re-ranking off);
    (4) the two build extensions of §7 (block-wise rotation, variance-aware
    subspace sizes) against the equal split with and without the global
    rotation, on skewed mixed data.  Prints one JSON line."""
    import torch

    import paper_2603_05180_gb300 as crisp
    import synthetic

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)

    def measure(ix, X, Q, gd, sp, k):
        nq = Q.shape[0]
        ids = torch.empty((nq, k), dtype=torch.int64, device=dev)
        d2 = torch.empty((nq, k), dtype=torch.float32, device=dev)
        crisp.crisp_search(ix, Q, nq, sp, ids, d2)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        crisp.crisp_search(ix, Q, nq, sp, ids, d2)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        return {"recall": recall_at_k(torch, X, Q, ids, gd[:, k - 1].contiguous()), "qps": nq / (ms / 1e3),
                "ms_per_query_batch": ms}

    out = {"workloads": {}}
    # (1) tau_CEV
    sets = []
    Xg, Qg = synthetic.gmm(N=20000, D=256, nq=1000)
    sets.append(("gmm 20k x 256", torch.from_numpy(Xg).to(dev), torch.from_numpy(Qg).to(dev), 8))
    Xp, Qp = synthetic.powerlaw(200000, 960, 1000, device="cuda")
    sets.append(("powerlaw 200k x 960", Xp, Qp, 20))
    Xv, Qv = synthetic.vmf(N=100000, D=768, nq=1000, n_comp=200)
    sets.append(("vmf 100k x 768", torch.from_numpy(Xv).to(dev), torch.from_numpy(Qv).to(dev), 16))
    Xl, Ql = synthetic.lowrank(N=100000, D=1024, nq=1000)
    sets.append(("lowrank 100k x 1024", torch.from_numpy(Xl).to(dev), torch.from_numpy(Ql).to(dev), 16))
    rows = []
    for name, X, Q, M in sets:
        N, D = X.shape
        _, gd = ground_truth(torch, X, Q, 100)
        res = {}
        cev = None
        for rot in (0, 1):
            ix = crisp.crisp_build(X, N, D, crisp.build_params(M, rotate=rot, draws=synthetic.method_draws(N, D, M, 50)))
            cev = ix.info().cev
            res[rot] = {pname: measure(ix, X, Q, gd, crisp.search_params(k=100, mode=0, **pt), 100)
                        for pname, pt in TAU_POINTS.items()}
            ix.free()
        rows.append({"dataset": name, "N": N, "D": D, "M": M, "cev": cev, "no_rotation": res[0], "rotation": res[1]})
    out["tau_cev"] = {"points": {k: f"Guaranteed, k=100, rho={v['rho']}, alpha={v['alpha']}, 1,000 queries"
                                 for k, v in TAU_POINTS.items()}, "datasets": rows,
                      "by_threshold": [{"tau_cev": t,
                                        "rotated": [r["dataset"] for r in rows if r["cev"] > t],
                                        **{f"mean_recall_at_100_{pn}": float(np.mean(
                                            [(r["rotation"] if r["cev"] > t else r["no_rotation"])[pn]["recall"]
                                             for r in rows])) for pn in TAU_POINTS}}
                                       for t in (0.7, 0.75, 0.8, 0.85, 0.9, 0.95)]}
    del sets, Xp, Qp
    torch.cuda.empty_cache()
    # (2) patience and (3) sub-components on the 1M x 960 power-law index
    N, D, M = 1_000_000, 960, 20
    X, Q = synthetic.powerlaw(N, D, 2000, device="cuda")
    ix = crisp.crisp_build(X, N, D, crisp.build_params(M, draws=synthetic.method_draws(N, D, M, 50)))
    _, gd = ground_truth(torch, X, Q, 100)
    out["patience"] = [dict(patience_factor=pf, **measure(ix, X, Q, gd, crisp.search_params(
        k=100, mode=1, rho=0.03, alpha=0.3, patience_factor=pf, max_candidates=OPT_CAP), 100)) for pf in (20, 40, 60)]
    sub = []
    for rho in (0.01, 0.02, 0.03):
        for name, kw in (("full", dict(eps0=2.1, verify_order=0)), ("exact L2 (no ADSampling)",
                                                                    dict(eps0=float("inf"), verify_order=0)),
                         ("no Hamming re-ranking", dict(eps0=2.1, verify_order=1))):
            sub.append(dict(config=name, rho=rho, **measure(ix, X, Q, gd, crisp.search_params(
                k=10, mode=1, rho=rho, alpha=0.3, max_candidates=OPT_CAP, **kw), 10)))
    out["subcomponents"] = {"point": "Optimized, k=10, alpha=0.3, patience 40 k, 2,000 queries, 1M x 960",
                            "points": sub}
    ix.free()
    del X, Q
    torch.cuda.empty_cache()
    # (4) §7 extensions on the mixed workload (a correlated 192-dim block beside
    # 768 independent dims with standard deviations 8 .. 1)
    N, D, M = 1_000_000, 960, 20
    Xh, Qh = synthetic.mixed(N, D, 2000, corr_dims=192, rank=8, skew=8.0)
    X, Q = torch.from_numpy(Xh).to(dev), torch.from_numpy(Qh).to(dev)
    del Xh, Qh
    _, gd = ground_truth(torch, X, Q, 10)
    draws = synthetic.method_draws(N, D, M, 50)
    ext = []
    for name, kw in (("equal split, no rotation", dict(rotate=0)), ("equal split, global rotation", dict(rotate=1)),
                     ("equal split, block-wise rotation (192-dim blocks)", dict(rotate=-1, block_dims=192)),
                     ("variance-aware subspaces, no rotation", dict(rotate=0, adaptive=1)),
                     ("variance-aware subspaces, block-wise rotation", dict(rotate=-1, block_dims=192, adaptive=1))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ix = crisp.crisp_build(X, N, D, crisp.build_params(M, draws=draws, **kw))
        build_s = time.perf_counter() - t0
        info = ix.info()
        w = np.diff(crisp.crisp_index_get_bounds(ix))
        ext.append(dict(config=name, build_s=build_s, rotated=int(info.rotated), rotated_blocks=int(info.rotated_blocks),
                        subspace_dims_min=int(w.min()), subspace_dims_max=int(w.max()),
                        points=[dict(rho=rho, **measure(ix, X, Q, gd, crisp.search_params(k=10, rho=rho, alpha=0.15),
                                                        10)) for rho in (0.05, 0.1, 0.2)]))
        ix.free()
    out["extensions"] = {"point": "Guaranteed, k=10, alpha=0.15, 2,000 queries, mixed 1M x 960, M=20",
                         "configs": ext}
    out["workloads"] = {"tau_cev": "gmm, powerlaw, vmf (200 components, kappa 200), lowrank (rank 128, 5% x10)",
                        "patience_subcomponents": "powerlaw 1M x 960, M=20",
                        "extensions": "mixed 1M x 960: rank-8 correlated block of 192 dims + 768 independent "
                                      "dims, std 8 .. 1"}
    print(json.dumps({"ablation": out}), flush=True)


def stage_rooflines(stage, info, hbm_peak, hbm_kind, traffic_key):
    """Roofline of the dominant kernel and of every timed stage.

    The tensor-core re-rank scorer is a dense contraction: its achieved rate is
    the flops it executes per launch (each (group, row) entry one row times the
    group's queries over Dp dims) over its CUDA-event duration, against the
    tensor peak of its pass: BF16 when it reads the index's BF16 copy, TF32
    when it reads the FP32 rows.  Its row traffic (entries x row bytes, from L2
    or HBM) and the pairs it serves per row fetch are reported beside it.  The
    other stages are measured in their algorithmic bytes against the HBM copy
    bandwidth."""
    rooflines = {}
    for n, v in stage.items():
        if v["bytes"]:
            a = v["bytes"] / (v["ms"] / 1e3) / 1e9
            rooflines[n] = {"kernel": v["kernel"], "bound": "hbm", "achieved": a, "peak": hbm_peak, "unit": "GB/s",
                            "frac": a / hbm_peak, "ms": round(v["ms"], 4), "algorithmic_bytes_per_launch": v["bytes"]}
    sc = stage.get("rerank", {}).get("scorer")
    if sc:
        bf = sc.get("elem_bytes", 4) == 2
        tpk, tkind = bf16_peak() if bf else tf32_peak()
        fl = sc["rows_per_launch"] * sc["group"] * 2 * sc["Dp"]
        t = sc["ms_per_launch"] / 1e3
        ach = fl / t / 1e12
        row_bytes = sc["rows_per_launch"] * sc.get("elem_bytes", 4) * sc["Dp"]
        traffic = _ncu_traffic("k_rerank_tc", traffic_key) if bf else None   # captured for the BF16 pass
        rooflines["rerank_scorer"] = {
            "kernel": "k_rerank_tc", "bound": "tensor", "achieved": ach, "peak": tpk, "unit": "TFLOP/s",
            "frac": ach / tpk, "traffic": traffic, "ms": round(sc["ms_per_launch"], 4),
            "pass": "BF16 (the index's BF16 copy, queries rounded to BF16)" if bf else "TF32 (the FP32 rows)",
            "peak_kind": (f"{tkind} sustained BF16 GEMM rate (MEASURED_PEAKS.json)" if bf else
                          f"{tkind} sustained BF16 GEMM rate (MEASURED_PEAKS.json) x {TF32_PER_BF16:.3f}, the nominal "
                          "TF32 / BF16 dense ratio"),
            "flops_per_launch": fl, "rows_per_launch": sc["rows_per_launch"], "pairs_per_launch": sc["pairs_per_launch"],
            "pairs_per_row_fetch": sc["pairs_per_launch"] / max(sc["rows_per_launch"], 1.0),
            "row_bytes_per_launch": row_bytes, "row_gbs": row_bytes / t / 1e9,
            "dram_gbs": traffic / t / 1e9 if traffic else None,
            "dram_frac": traffic / t / 1e9 / hbm_peak if traffic else None,
            "note": "flops: one pass of every (64-query group, listed row) entry; rows come from L2 when the "
                    "range-block order keeps them there; the exact FP32 re-measure and selection are separate "
                    "kernels"}
    timed_ms = {n: v["ms"] for n, v in stage.items()}
    dom_stage = max(timed_ms, key=lambda n: timed_ms[n])
    if dom_stage == "rerank" and "rerank_scorer" in rooflines:
        dom = dict(rooflines["rerank_scorer"])
    else:
        dom = dict(rooflines.get(dom_stage) or {"kernel": stage[dom_stage]["kernel"], "bound": "hbm", "achieved": None,
                                                "peak": hbm_peak, "unit": "GB/s", "frac": None})
        dom["traffic"] = _ncu_traffic(dom_stage, traffic_key)
        dom["peak_kind"] = f"{hbm_kind} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
    return dom, rooflines


def stage_pass(torch, crisp, ix, info, Q, point, k, steps, stream, flush):
    """Time each kernel of the search path with CUDA events on the launching stream,
    and count the algorithmic bytes each launch must move (the per-stage units of each kernel)."""
    nq, Dp, M, K = Q.shape[0], info.Dp, info.M, info.K
    dev = Q.device
    tau = crisp.tau(point["alpha"], M)
    bud = crisp.budget(point["rho"], info.N)
    w = 2 if point["mode"] == 1 else 1
    stride = min(info.N, max(-(-w * M * (bud + info.max_cell) // tau), k)) if tau > 0 else info.N
    Qr = torch.empty((nq, Dp), dtype=torch.float32, device=dev)
    act = torch.empty((nq, M, K * K), dtype=torch.int32, device=dev)
    nact = torch.empty((nq, M), dtype=torch.int32, device=dev)
    got = torch.empty((nq, M), dtype=torch.int64, device=dev)
    cand = torch.empty((nq, stride), dtype=torch.int32, device=dev)
    ncand = torch.empty((nq,), dtype=torch.int64, device=dev)
    how = torch.empty((nq,), dtype=torch.int32, device=dev)
    ids = torch.empty((nq, k), dtype=torch.int64, device=dev)
    d2 = torch.empty((nq, k), dtype=torch.float32, device=dev)
    nv = torch.empty((nq,), dtype=torch.int64, device=dev)
    nf = torch.empty((nq,), dtype=torch.int64, device=dev)
    nb = torch.empty((nq,), dtype=torch.int64, device=dev)
    names = ["rotate", "activate", "count_cut", "rerank" if point["mode"] == 0 else "verify_opt"]
    # batches of >= 256 queries with candidate lists >= 2,048 wide re-rank on the
    # tensor cores (k-d-ordered query groups, bounded TF32 scores, exact re-measure
    # of the candidates that can reach the top-k); smaller ones stream (k_dist_flat)
    grouped = nq >= 256 and stride >= 2048
    kernels = ["k_rotate", "k_activate", "k_count_cut",
               ("k_rerank_tc (+ order, union, bound select, exact re-measure)" if grouped else "k_dist_flat")
               if point["mode"] == 0 else "k_verify_opt"]
    bf16 = bool(info.Xb) and point["mode"] == 0
    if bf16:            # the F2 coarse-scoring kernel on the same candidates (timed on its own)
        names.append("shortlist_bf16")
        kernels.append("k_rerank_tc BF16 coarse bounds (+ order, union, bound select, exact scores of the kept)"
                       if grouped else "k_score_flat<BF16>")
        sl = torch.empty((nq, 64), dtype=torch.int32, device=dev)
        nsl = torch.empty((nq,), dtype=torch.int64, device=dev)
    acc = {n: 0.0 for n in names}

    def one():
        if info.rotated:
            crisp.crisp_rotate_rows(Q, nq, info.D, info.D, info.R32, Qr, Dp, stream)
        else:
            Qr.zero_()
            Qr[:, :info.D] = Q
        yield
        crisp.crisp_activate(ix, Qr, nq, point["mode"], k, bud, act, nact, got, stream)
        yield
        crisp.crisp_count_cut(ix, act, nact, nq, tau, k, 0, cand, stride, ncand, None, how, stream)
        yield
        if point["mode"] == 0:
            crisp.crisp_rerank(ix, Qr, nq, cand, stride, ncand, k, ids, d2, stream)
        else:
            crisp.crisp_verify_opt(ix, Qr, nq, cand, stride, ncand, k, 2.1, 40 * k, ids, d2, nv, nf, nb, stream)
        yield
        if bf16:
            crisp.crisp_shortlist(ix, Qr, nq, cand, stride, ncand, 1, 50, sl, 64, nsl, stream)
            yield

    prof = None
    for s in range(steps + 1):
        if s == 1:
            crisp.crisp_rerank_profile_read()          # drop the warm-up pass
        if s == 0:
            crisp.crisp_rerank_profile_enable(True)
        flush.zero_()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
        evs[0].record(stream)
        for i, _ in enumerate(one()):
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        if s == 0:
            continue            # warm-up
        for i, n in enumerate(names):
            acc[n] += evs[i].elapsed_time(evs[i + 1]) / steps
    prof = crisp.crisp_rerank_profile_read()
    crisp.crisp_rerank_profile_enable(False)
    C = float(ncand.sum().item())
    retr = float(got.sum().item())
    cells = float(nact.sum().item())
    W = Dp // 32
    out = {
        "rotate": {"ms": acc["rotate"], "bytes": 0, "kernel": "k_rotate"},
        "activate": {"ms": acc["activate"], "bytes": 0, "kernel": "k_activate"},
        # ids streamed from the CSR lists + 8 B per activated cell + candidate ids written
        "count_cut": {"ms": acc["count_cut"], "bytes": 4 * retr + 8 * cells + 4 * C, "kernel": "k_count_cut"},
    }
    if point["mode"] == 0:
        # every candidate row (Dp floats) + its id
        out["rerank"] = {"ms": acc["rerank"], "bytes": C * (4 * Dp + 4), "kernel": kernels[3]}
        if prof is not None and prof.launches > 0:
            # the tensor-core scorer alone (events around its launches inside the library):
            # per launch, its (group, row) entries each multiply one row by the group's
            # queries over Dp dims (2 flops per multiply-add); pairs are (row, query)
            # distances it bounds
            out["rerank"]["scorer"] = {"kernel": "k_rerank_tc", "launches": prof.launches,
                                       "ms_per_launch": prof.ms / prof.launches,
                                       "rows_per_launch": prof.rows / prof.launches,
                                       "pairs_per_launch": prof.pairs / prof.launches, "group": prof.group,
                                       "Dp": prof.Dp, "elem_bytes": prof.elem_bytes}
    else:
        blocks = float(nb.sum().item())
        out["verify_opt"] = {"ms": acc["verify_opt"], "bytes": C * (4 * W + 4) + 128 * blocks,
                             "kernel": "k_verify_opt"}
    if bf16:
        # every candidate's BF16 row (2 Dp bytes) + its id; the shortlist written is small
        out["shortlist_bf16"] = {"ms": acc["shortlist_bf16"], "bytes": C * (2 * Dp + 4)}
    for n, kn in zip(names, kernels):
        out[n]["kernel"] = kn
    return out


def _ncu_traffic(stage, workload):
    """DRAM bytes per launch from the committed ncu summary, when one exists for
    this kernel and was taken on this workload (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        if d.get("workload") != workload:
            return None
        return d.get("bytes_per_launch", {}).get(stage)
    return None


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["crisp", "reference"], default="crisp")
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--dim", type=int, default=960)
    ap.add_argument("--nq", type=int, default=10_000)
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--M", type=int, default=12)
    ap.add_argument("--mode", type=int, default=None)
    ap.add_argument("--rho", type=float, default=None)
    ap.add_argument("--alpha", type=float, default=None)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--sweep", action="store_true", help="pick the operating point by a recall/QPS sweep")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the BF16 / FP8 coarse-scoring measurements")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-depth + BF16 measurement")
    ap.add_argument("--train-queries", type=int, default=50000)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--full", action="store_true", help="also run the vMF D=3072, low-rank D=4096 and serving "
                    "configurations (several minutes each)")
    ap.add_argument("--vmf", action="store_true", help="run the vMF D=3072 learned+BF16 configuration")
    ap.add_argument("--lowrank", action="store_true", help="run the low-rank D=4096 FP8 configuration")
    ap.add_argument("--serve", action="store_true", help="run the continuous-batching serving configuration")
    ap.add_argument("--no-serve", action="store_true", help="skip the continuous-batching serving measurement")
    ap.add_argument("--no-modes", action="store_true", help="skip the Guaranteed / Optimized k=10 / k=100 points")
    ap.add_argument("--no-vmf", action="store_true", help="skip the vMF D=3072 learned+BF16 configuration")
    ap.add_argument("--no-lowrank", action="store_true", help="skip the low-rank D=4096 FP8 configuration")
    ap.add_argument("--vmf-n", type=int, default=1_000_000)
    ap.add_argument("--vmf-train", type=int, default=200_000)
    ap.add_argument("--lowrank-n", type=int, default=2_000_000)
    ap.add_argument("--ablation", action="store_true", help="run the paper's ablations (tau_CEV, patience, "
                                                            "verification sub-components) instead of the benchmark")
    ap.add_argument("--serve-n", type=int, default=5_000_000)
    ap.add_argument("--serve-dim", type=int, default=1024)
    ap.add_argument("--serve-M", type=int, default=32)
    ap.add_argument("--serve-pool", type=int, default=4096, help="distinct queries the requests draw from")
    ap.add_argument("--serve-train", type=int, default=20000)
    ap.add_argument("--serve-streams", type=int, default=4)
    ap.add_argument("--serve-batch", type=int, default=2048)
    ap.add_argument("--serve-rates", type=lambda v: [int(x) for x in v.split(",")], default=[20000, 50000, 100000, 200000])
    ap.add_argument("--serve-seconds", type=float, default=1.5)
    ap.add_argument("--serve-max-requests", type=int, default=60000)
    ap.add_argument("--serve-burst", type=int, default=20000, help="requests of the capacity burst")
    ap.add_argument("--ref-step-seconds", type=float, default=4.0)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.ablation:
        run_ablation(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_crisp(args)


if __name__ == "__main__":
    main()
