"""Benchmark of the randomized GSV solve on GB300.

One step = one full solve of the workload (every pair's two basis extractions
with q power iterations, the projections, the FP64 compressed-pair GSVD), inputs
resident in HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload batched|tf32_large|fp64_small|bf16_stress|learned] [--prec tf32|fp32|...]

--workload batched (the default): 256 uneven pairs (m, p ~ U[2000, 30000], n ~ U[100, 1000],
k = rank ~ U[10, 100], oversample 10, q = 1) per step, solved by one
gsvd_rand_solve_grouped call (every step one launch for all pairs, the launch
sequence replayed from a CUDA graph); --batched-mode workers runs
gsvd_rand_solve_batched over concurrent worker streams instead.

--workload learned: the learned (k, q) proposal (train on the GPU, then solve held-out
pairs; compared with Algorithm 1 alone and the plain fixed-rank method).

Multi-GPU (torchrun, N > 1): every rank solves its own independent pairs (the
units shard with no data-path collective): weak scaling, value = pairs of all
ranks / max-over-ranks time.
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

from paper_2404_09459_gb300.inputs import (PAIR_BF16_STRESS, PAIR_FP64_SMALL, PAIR_TF32_LARGE,  # noqa: E402
                                           aligned_rows, planted_pair, planted_pair_torch, uneven_batch)

WORKLOADS = {
    "tf32_large": (PAIR_TF32_LARGE, "tf32x3"),
    "fp64_small": (PAIR_FP64_SMALL, "fp64"),
    "bf16_stress": (PAIR_BF16_STRESS, "bf16"),
    "batched": (None, "tf32x3"),  # 256 uneven pairs, one batched call per step
    "learned": (None, "fp64"),    # learned (k, q) proposal: train, then held-out pairs
}
# context flags per precision: the BF16 mode runs its power steps on hi + lo halves (the
# single-product form misses the 1e-4 target on the slow-decay pair)
FLAGS = {"bf16": 4}
METRIC = "pairs/sec and sketch TFLOP/s at GSV rel-err <=1e-4, chosen form vs plain FP64"
DTYPE = {"tf32": "tf32", "tf32x3": "tf32x3", "bf16": "bf16", "fp32": "f32", "fp64": "f64"}


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest x over the ranks (a weak-scaling job takes as long as its slowest rank)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s own pair (the ranks solve independent pairs)."""
    return seed + 1000 * rank


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


def workload_desc(spec, prec):
    extra = ", G stored BF16, power steps on BF16 hi + lo" if prec == "bf16" else ""
    return (f"single pair m={spec.m} p={spec.p} n={spec.n} rank={spec.r} k={spec.kk} "
            f"oversample={spec.oversample} q={spec.q}, {prec} sketch/power/projection{extra}, FP64 small GSVD")


def sketch_traffic(prec, workload):
    """DRAM bytes per sketch launch from the committed ncu capture, or None when the capture
    does not cover this workload/precision or the kernel source changed since it was taken."""
    import hashlib
    files = {("tf32_large", "tf32x3"): "sketch_traffic_tf32x3_large_pair.json",
             ("bf16_stress", "bf16"): "sketch_traffic_bf16_stress_pair.json",
             ("batched", "tf32x3"): "sketch_traffic_grouped_batch.json"}
    if (workload, prec) not in files:
        return None
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", files[(workload, prec)])))
        src = open(os.path.join(ROOT, rec["source"]), "rb").read()
    except Exception:
        return None
    if hashlib.sha256(src).hexdigest() != rec["source_sha256"]:
        return None
    return rec.get("traffic_per_launch", rec.get("traffic_per_launch_both_sides_avg"))


def sketch_flops(spec):
    """Algorithmic GEMM flops of one solve: per side (2q+2) passes of 2 M n l."""
    return sum((2 * spec.q + 2) * 2.0 * M * spec.n * spec.l for M in (spec.m, spec.p))


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def cpu_baseline(spec, seconds=20.0):
    """The FP64 oracle (NumPy/LAPACK, all host cores) on a bounded sample: whole pairs."""
    from oracle import gsvd as O
    G1, G2, _, _ = planted_pair(spec)
    t0 = time.perf_counter()
    done = 0
    while True:
        O.rand_gsvd(G1, G2, spec.kk, spec.oversample, spec.q, spec.seed)
        done += 1
        if time.perf_counter() - t0 > seconds or done >= 8:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "pairs/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{done} full solve(s) of the workload pair with the FP64 oracle (OpenBLAS, "
                      f"{os.cpu_count()} threads)"}


def run_reference(args, rank, world):
    """--impl reference: the oracle timed on host cores (rank 0 only)."""
    spec, prec = WORKLOADS[args.workload]
    if rank != 0:
        return
    if spec is None and args.workload == "learned":
        from paper_2404_09459_gb300.inputs import learned_pairs
        s = oracle_learned_sample(learned_pairs(args.holdout, seed=2), seconds=10.0)
        line = {"impl": "reference", "metric": METRIC, "value": s["value"], "unit": "pairs/s", "n_gpus": world,
                "steps": 1, "warmup": 0, "ms_per_step": 1e3 / s["value"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"learned-proposal held-out pairs ({args.holdout}) (oracle on a sample)"},
                "cpu_baseline": s,
                "e2e": {"value": s["value"], "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    if spec is None:
        # batched: each step is the oracle's solve of one pair of the same 256-pair batch (pairs taken
        # in turn from the first few), so that --steps K --warmup W stays within minutes on host cores
        from oracle import gsvd as O
        specs = uneven_batch(args.pairs, seed=1)
        distinct = min(len(specs), 6)
        cache = {}

        def one(i):
            j = i % distinct
            if j not in cache:
                cache[j] = planted_pair(specs[j])[:2]
            G1, G2 = cache[j]
            s = specs[j]
            t0 = time.perf_counter()
            O.rand_gsvd(G1, G2, s.kk, s.oversample, s.q, s.seed, pair=j)
            return time.perf_counter() - t0

        for i in range(args.warmup):
            one(i)
        secs = sum(one(args.warmup + i) for i in range(args.steps))
        v = args.steps / secs
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "pairs/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": f"batch of {args.pairs} uneven pairs: m, p ~ U[2000, 30000], n ~ U[100, 1000], "
                                       "k = rank ~ U[10, 100], oversample 10, q 1; FP64 oracle, one pair per step "
                                       f"(the first {distinct} pairs in turn)"},
                "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": os.cpu_count(), "kind": "oracle",
                                 "sample": f"{args.steps} oracle solves of pairs 0..{distinct - 1} of the batch "
                                           f"(OpenBLAS, {os.cpu_count()} threads); input generation not timed"},
                "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    from oracle import gsvd as O
    G1, G2, _, _ = planted_pair(spec)
    for _ in range(args.warmup):
        O.rand_gsvd(G1, G2, spec.kk, spec.oversample, spec.q, spec.seed)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.rand_gsvd(G1, G2, spec.kk, spec.oversample, spec.q, spec.seed)
    dt = time.perf_counter() - t0
    v = args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_desc(spec, "fp64 oracle")},
            "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{args.steps} full solves of the workload pair"},
            "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def oracle_batch_sample(specs, seconds=20.0, max_pairs=16):
    """The FP64 oracle on the first pairs of a batch (only the solves are timed)."""
    from oracle import gsvd as O
    spent, done = 0.0, 0
    for s in specs[:max_pairs]:
        G1, G2, _, _ = planted_pair(s)
        t0 = time.perf_counter()
        O.rand_gsvd(G1, G2, s.kk, s.oversample, s.q, s.seed)
        spent += time.perf_counter() - t0
        done += 1
        if spent > seconds:
            break
    return {"value": done / spent, "unit": "pairs/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{done} pairs of the batch with the FP64 oracle (OpenBLAS, {os.cpu_count()} threads); "
                      "input generation not timed"}


def gsv_error_summary(pairs_out, refs):
    """Per-GSV error e_i = max(|alpha_i - alpha_ref_i|, |beta_i - beta_ref_i|) and the angular-distance
    error |theta_i - theta_ref_i| (theta = atan2(alpha, beta) - pi/4) over the compared pairs."""
    es, ts = [], []
    for (a, b), (ar, br) in zip(pairs_out, refs):
        a, b, ar, br = (np.asarray(x, dtype=np.float64) for x in (a, b, ar, br))
        es.append(np.maximum(np.abs(a - ar), np.abs(b - br)))
        ts.append(np.abs(np.arctan2(a, b) - np.arctan2(ar, br)))
    e, t = np.concatenate(es), np.concatenate(ts)
    return {"max": float(e.max()), "median": float(np.median(e)), "theta_abs_max": float(t.max()),
            "pairs": len(refs), "gsvs": int(e.size)}


def tensor_peak(prec, pk):
    """Tensor-core peak (TFLOP/s) for the products of `prec`: BF16 from MEASURED_PEAKS.json; TF32
    from the committed cuBLAS measurement in profiles/ (else half the BF16 peak, the nominal ratio)."""
    bf = pk.get("bf16_tflops", 1900.0)
    if prec == "bf16":
        return bf, "measured bf16_tflops (MEASURED_PEAKS.json)"
    try:
        rates = json.load(open(os.path.join(ROOT, "profiles", "measured_rates.json")))
        return float(rates["tf32_tflops"]), "measured TF32 cuBLAS GEMM (profiles/measured_rates.json)"
    except Exception:
        return 0.5 * bf, "measured bf16_tflops x 0.5 (TF32 nominal ratio)"


def run_batched(args, rank, world):
    """--workload batched (the default): one step = one grouped solve of 256 uneven pairs."""
    import torch
    import paper_2404_09459_gb300 as P
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    P._build.build()
    prec = args.prec or "tf32x3"
    npairs = args.pairs
    specs = uneven_batch(npairs, seed=1 + rank)
    dt = torch.float64 if prec == "fp64" else torch.float32
    # rows stored with a 16-byte-multiple stride, so that the tensor-core products read G in place
    mats = [tuple(aligned_rows(G) for G in planted_pair_torch(s, device=dev, dtype=dt)[:2]) for s in specs]
    pairs = [dict(G1=G1, G2=G2, k=s.kk, oversample=s.oversample, q=s.q, seed=s.seed, pair=i)
             for i, (s, (G1, G2)) in enumerate(zip(specs, mats))]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    ctx = P.Context(prec, device=local)
    grouped = args.batched_mode == "grouped"
    st = torch.cuda.current_stream()

    def step(c=ctx, pl=pairs):
        if grouped:
            return c.solve_grouped(pl)  # one launch per step for all pairs, replayed from a CUDA graph
        return c.solve_batched(pl, workers=args.workers)  # synchronous: returns after the worker streams

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    l0 = ctx.launch_count()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # timed region: CUDA events on the stream the library orders its work after and before
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)  # L2 flush between timed steps (outside the events)
            evs[i][0].record(st)
            outs = step()
            evs[i][1].record(st)
        barrier()
    launches = (ctx.launch_count() - l0) // max(args.steps, 1)
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), dist, dev)
    ms_step = ms / args.steps
    value = world * npairs * args.steps / (ms / 1e3)
    info = ctx.grouped_info() if grouped else None
    flops = sum(sketch_flops(s) for s in specs)

    # per-step device time of the replays by stage (CUDA events captured into the graph, on the
    # stream the kernels run on), for the stage split and the roofline of the Y = G X products
    stages, roof = None, None
    pk = peaks()
    if grouped:
        pctx = P.Context(prec, device=local, flags=P.FLAG_PROFILE)
        pctx.solve_grouped(pairs)
        pctx.profile(reset=True)
        reps = max(1, min(args.steps, 5))
        for i in range(reps):
            flush.fill_(i & 0xFF)
            pctx.solve_grouped(pairs)
        prof = pctx.profile()
        pctx.close()
        tot = sum(v[0] for k, v in prof.items() if k != "small")  # grouped steps carry the sub-stage tags
        stages = {k: {"ms_per_step": v[0] / reps, "launches_per_step": v[1] / reps,
                      "share": v[0] / tot if tot else None}
                  for k, v in prof.items() if v[1] and k != "small"}
        sk_ms, sk_calls = prof["sketch"]
        if sk_calls:
            # algorithmic bytes of the Y = G X launches of one solve: (1 + q) passes per side over G
            # (FP32), X (FP32, once) and Y (FP32 written); a launch covers every side still iterating
            passes = [(1 + s.q, M, s.n, s.l) for s in specs for M in (s.m, s.p)]
            bytes_step = sum(c * (M * n + n * l + M * l) * 4 for c, M, n, l in passes)
            flops_step = sum(c * 2.0 * M * n * l for c, M, n, l in passes)
            calls_step = sk_calls / reps
            launch_s = sk_ms / sk_calls / 1e3
            achieved = bytes_step / calls_step / launch_s / 1e9
            roof = {"kernel": "tc_group_kernel, Y = G X (all sides of the batch per launch)", "bound": "hbm",
                    "achieved": achieved, "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                    "frac": achieved / pk["hbm_gbs"], "traffic": sketch_traffic(prec, "batched"),
                    "bytes_per_launch": bytes_step / calls_step, "launch_ms": launch_s * 1e3,
                    "launches_per_step": calls_step,
                    "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if not pk.get("fallback") else "fallback"}
            tpk, src = tensor_peak(prec, pk)
            tach = flops_step / calls_step / launch_s / 1e12
            roof["tensor"] = {"achieved_tflops": tach, "peak_tflops": tpk, "frac": tach / tpk, "peak_source": src}

    # accuracy of the timed step's results: per-GSV error against the FP64 oracle on a sample of the
    # pairs (the oracle runs on host copies of the same FP32 matrices, same Philox streams)
    gsv = None
    sample = list(range(0, npairs, max(1, npairs // args.error_pairs)))[:args.error_pairs] if args.error_pairs else []
    refs, got = [], []
    if rank == 0 and sample:
        from oracle import gsvd as O
        for i in sample:
            s = specs[i]
            G1h = mats[i][0].double().cpu().numpy()
            G2h = mats[i][1].double().cpu().numpy()
            ref = O.rand_gsvd(G1h, G2h, s.kk, s.oversample, s.q, s.seed, pair=i)
            refs.append((ref["alpha"], ref["beta"]))
            got.append((outs[i]["alpha"].cpu().numpy(), outs[i]["beta"].cpu().numpy()))
        gsv = gsv_error_summary(got, refs)
        gsv.update({"tol": 1e-4 if prec != "tf32" else 1e-3, "against": "FP64 oracle, same FP32 inputs and Omega",
                    "sample": f"pairs {sample[0]}..{sample[-1]} step {max(1, npairs // args.error_pairs)}"})
        gsv["pass"] = gsv["max"] <= gsv["tol"] and gsv["theta_abs_max"] <= 1e-4

    # the other batched form on the same pairs (grouped vs concurrent per-pair workers)
    other = None
    if grouped and args.steps > 0:
        ctx.solve_batched(pairs, workers=args.workers)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.solve_batched(pairs, workers=args.workers)
        torch.cuda.synchronize()
        other = {"value": npairs / (time.perf_counter() - t0), "unit": "pairs/s",
                 "form": f"{args.workers} concurrent worker streams, per-pair launches",
                 "chol64_retries": ctx.chol64_retries() // 2}  # per call (two calls above)

    # plain FP64 GPU path on the same pairs (FP64 copies; the concurrent worker-stream form)
    fp64 = None
    if not args.no_fp64 and prec != "fp64":
        fpairs = [dict(d, G1=d["G1"].double(), G2=d["G2"].double()) for d in pairs]
        fctx = P.Context("fp64", device=local)
        fctx.solve_batched(fpairs[:args.workers], workers=args.workers)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fouts = fctx.solve_batched(fpairs, workers=args.workers)
        e1.record(st)
        torch.cuda.synchronize()
        fms = e0.elapsed_time(e1)
        fctx.close()
        fp64 = {"value": npairs / (fms / 1e3), "unit": "pairs/s", "ms_per_step": fms,
                "form": f"plain FP64 path, {args.workers} concurrent worker streams",
                "speedup_of_chosen_form": (value / world) / (npairs / (fms / 1e3))}
        if refs:
            fgot = [(fouts[i]["alpha"].cpu().numpy(), fouts[i]["beta"].cpu().numpy()) for i in sample]
            fp64["gsv_error"] = gsv_error_summary(fgot, refs)
        del fpairs, fouts
        torch.cuda.empty_cache()

    # end to end through the public API with host (pinned) buffers: every step copies the whole
    # batch into HBM inside the call (gsvd_rand_solve_grouped stages host inputs) and returns
    # alpha / beta in host memory
    e2e = None
    if not args.no_e2e:
        hpairs = []
        for d in pairs:
            h1 = torch.empty((d["G1"].shape[0], d["G1"].shape[1]), dtype=dt, pin_memory=True)
            h2 = torch.empty((d["G2"].shape[0], d["G2"].shape[1]), dtype=dt, pin_memory=True)
            h1.copy_(d["G1"])
            h2.copy_(d["G2"])
            hpairs.append(dict(d, G1=h1, G2=h2))
        ectx = P.Context(prec, device=local)
        for _ in range(2):
            step(ectx, hpairs)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step(ectx, hpairs)
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
        ectx.close()
        h2d = sum((d["G1"].shape[0] + d["G2"].shape[0]) * d["G1"].shape[1] for d in hpairs) * (8 if prec == "fp64" else 4)
        d2h = sum(2 * d["k"] * 8 + 2 * 8 + 4 for d in hpairs)
        e2e = {"value": world * npairs * args.steps / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h),
               "form": "gsvd_rand_solve_grouped on pinned host inputs (copied inside the call), host outputs; "
                       "host clock, device synchronised on both sides"}
        del hpairs

    # the same batch one pair after another (one stream), for the batching gain
    seq = None
    if grouped and not args.no_sequential:
        seq_ctx = P.Context(prec, device=local)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s, (G1, G2) in zip(specs, mats):
            seq_ctx.solve(G1, G2, s.kk, s.oversample, s.q, s.seed)
        torch.cuda.synchronize()
        seq_s = time.perf_counter() - t0
        seq_ctx.close()
        seq = {"value": npairs / seq_s, "unit": "pairs/s", "batching_speedup": value / world / (npairs / seq_s)}
    cpu = oracle_batch_sample(specs) if rank == 0 and not args.no_cpu_baseline else None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": DTYPE.get(prec, prec), "data": "synthetic",
                "config": {"workload": f"batch of {npairs} uneven pairs: m, p ~ U[2000, 30000], n ~ U[100, 1000], "
                                       f"k = rank ~ U[10, 100], oversample 10, q 1; {prec} products, FP64 small GSVD; "
                                       + ("grouped: one launch per step for all pairs (persistent grouped tcgen05 "
                                          "products, batched CholeskyQR and compressed-pair kernels), replayed from "
                                          "a captured CUDA graph" if grouped else
                                          f"{args.workers} concurrent worker streams"),
                           "l2": "flushed between timed steps (256 MiB write); the batch's G (17.6 GB) exceeds L2",
                           "timing": "CUDA events on the library's stream around each grouped call",
                           "parallelism": f"independent batches, {world} rank(s)"},
                "sketch_tflops": flops / (ms_step / 1e3) / 1e12, "roofline": roof, "gsv_error": gsv,
                "fp64_plain": fp64, "e2e": e2e, "sequential": seq, "cpu_baseline": cpu,
                "gpu_launches": int(launches), "clocks": clk.summary()}
        if info is not None:
            line["grouped"] = {"tuned_stages_ctas_per_sm": {"first_sketch": info["tuned"][0],
                                                            "power_sketch": info["tuned"][1],
                                                            "gtq_projection": info["tuned"][2]},
                               "graph_captures": info["captures"], "graph_replays": info["replays"],
                               "launches_per_replay": info["launches"]}
            line["worker_streams"] = other
            line["stages"] = stages
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def run_learned(args, rank, world):
    """--workload learned: the learned (k, q) proposal for whole groups of pairs of the uneven-batch
    laws (sigma 1e-9), mixed precision (3xTF32 products), residual tolerance --learned-tol.  Labels
    (the FP64 Algorithm 1 and fixed-rank bases at that tolerance) and training run on the GPU
    first (not timed).  One timed step = one grouped learned solve of every held-out pair (batched
    probes, one network forward and the device plans, the fixed-rank group with each pair's plan,
    one Algorithm 1 group for the misses).  The same group is also solved by the grouped Algorithm
    1 alone (b = 16), by the fixed-rank method at the one (k, q) the training labels need at most
    (a constant proposal through the same pipeline), and with the labels as a perfect proposal.  Timing: CUDA events around each grouped call on the
    library's stream, after one untimed call that captures its graphs."""
    import tempfile
    import torch
    import paper_2404_09459_gb300 as P
    from paper_2404_09459_gb300 import learn
    from paper_2404_09459_gb300.inputs import learned_pairs
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    P._build.build()
    tol, os_, b = args.learned_tol, 10, 16
    tr = learned_pairs(args.train, seed=1 + 7919 * rank)
    ho = learned_pairs(args.holdout, seed=2 + 7919 * rank)
    # labels at half the solve's tolerance: the FP32 residual estimate of the mixed solve then has
    # a margin over the FP64 labels' certified residual
    t0 = time.perf_counter()
    X, yk, yq, kad = learn.make_dataset(tr, tol / 2, os_, local, features_prec="tf32x3")
    t_label = time.perf_counter() - t0
    Xh, ykh, yqh, _ = learn.make_dataset(ho, tol / 2, os_, local, features_prec="tf32x3")
    t0 = time.perf_counter()
    params, norm, hist = learn.train(X, yk, yq, epochs=args.epochs, batch=256, lr=1e-3, device=local)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    pk, pq = learn.predict(params, norm, Xh, device=local, quantile=0.9)
    pk0, _ = learn.predict(params, norm, Xh, device=local)
    path = os.path.join(tempfile.mkdtemp(), "net.bin")
    learn.save(path, params, norm)
    # the held-out group: FP32 pairs with 16-byte rows (read in place by the grouped products)
    mats = [tuple(aligned_rows(G) for G in planted_pair_torch(s, device=dev, dtype=torch.float32)[:2]) for s in ho]
    kcap = 128 - os_
    kb_fix, qfix = int(yk.max()), int(yq.max())
    kfix = min(learn.k_of_bucket(kb_fix), kcap)
    cpath = os.path.join(tempfile.mkdtemp(), "constant.bin")
    learn.save(cpath, *learn.constant_net(kb_fix, qfix))
    st = torch.cuda.current_stream()

    def pairs_with(plans=None, k=None, q=1):
        out = []
        for i, (s, (G1, G2)) in enumerate(zip(ho, mats)):
            lm = min(s.m, s.p, s.n, 128) - os_
            kk, qq = plans[i] if plans is not None else (k, q)
            out.append(dict(G1=G1, G2=G2, k=max(1, min(kk, lm)), oversample=os_, q=qq, seed=s.seed, pair=i))
        return out

    def arm(make, pl, reps):
        with make() as ctx:
            ctx.solve_grouped(pl)  # capture and tuning
            ms = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                outs = ctx.solve_grouped(pl)
                e1.record(st)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            plans = ctx.grouped_plans(len(pl)) if getattr(ctx, "_learned", False) else None
        cert = float(np.mean([o["status"] == 0 and max(o["resid"]) <= tol for o in outs]))
        msm = statistics.median(ms)
        return {"value": len(pl) / (msm / 1e3), "unit": "pairs/s", "ms_per_call": msm, "certified": cert}, plans

    reps = max(1, args.steps)
    with ClockSampler(local) as clk:
        learned, plans = arm(lambda: P.Context("tf32x3", device=local, use_learned=True, mlp_path=path, tol=tol,
                                               block_b=b), pairs_with(k=kcap), reps)
    adaptive, _ = arm(lambda: P.Context("tf32x3", device=local, adaptive=True, tol=tol, block_b=b),
                      pairs_with(k=kcap), reps)
    # the plain fixed-rank method at the one (k, q) the training labels need at most, run through
    # the same pipeline as a constant proposal (probes, fixed-rank group, the same residual sums,
    # Algorithm 1 for the pairs it leaves above tol): what the trained network gains over it
    plain, plain_plans = arm(lambda: P.Context("tf32x3", device=local, use_learned=True, mlp_path=cpath, tol=tol,
                                               block_b=b), pairs_with(k=kcap), reps)
    plain["fallback_rate"] = float(np.mean([p_[2] for p_ in plain_plans])) if plain_plans else None
    # the labels as a perfect proposal (no fallback), the residual summed as the learned group sums it
    perfect, _ = arm(lambda: P.Context("tf32x3", device=local, flags=P.FLAG_ACC_RESID),
                     pairs_with(plans=[(learn.k_of_bucket(bb), int(qq)) for bb, qq in zip(ykh, yqh)]), reps)
    value = learned["value"]
    if dist is not None:
        value = world * len(ho) / max_over_ranks(len(ho) / value, dist, dev)
    fallback = float(np.mean([p_[2] for p_ in plans])) if plans else None
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = oracle_learned_sample(ho, tol=tol)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": reps,
                "warmup": 1, "ms_per_step": learned["ms_per_call"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "tf32x3", "data": "synthetic",
                "config": {"workload": (f"learned k/q proposal, grouped: {args.train} training + {args.holdout} "
                                        "held-out pairs of the uneven-batch laws (m, p ~ U[2000, 30000], n ~ "
                                        "U[100, 1000], r ~ U[10, 100], exp(-i/10) scale, sigma 1e-9), 3xTF32 "
                                        f"products, residual tol {tol:g}, oversample {os_}; one step = one grouped "
                                        "learned solve of every held-out pair"),
                           "timing": "CUDA events around each grouped call (median), after one capturing call",
                           "parallelism": f"independent groups, {world} rank(s)"},
                "arms": {"learned_grouped": learned, "adaptive_alg1_grouped_b16": adaptive,
                         "plain_fixed_rank_grouped": dict(plain, k=kfix, q=qfix), "perfect_proposal_grouped": perfect},
                "gain": {"vs_adaptive": value / adaptive["value"], "vs_plain_fixed_rank": value / plain["value"]},
                "learned": {"fallback_rate": fallback, "label_seconds": t_label, "train_seconds": t_train,
                            "train_pairs": args.train, "holdout_pairs": args.holdout,
                            "final_loss": float(hist[-1]), "holdout_k_bucket_acc": float(np.mean(pk0 == ykh)),
                            "holdout_q_acc": float(np.mean(pq == yqh)),
                            "holdout_under_k_at_q90": float(np.mean(pk < ykh)),
                            "label_q_counts": np.bincount(yq, minlength=5).tolist()},
                "cpu_baseline": cpu, "gpu_launches": None, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def oracle_learned_sample(specs, seconds=20.0, max_pairs=4, tol=1e-4):
    """The FP64 oracle's Algorithm 1 (b = 16) on a few held-out pairs (host cores)."""
    from oracle import gsvd as O
    done, t_total = 0, 0.0
    for s in specs[:max_pairs]:
        G1, G2, _, _ = planted_pair(s)
        t0 = time.perf_counter()
        O.rand_gsvd_adaptive(G1, G2, tol, 16, s.seed, 128)
        t_total += time.perf_counter() - t0
        done += 1
        if t_total > seconds:
            break
    return {"value": done / t_total, "unit": "pairs/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{done} held-out pairs solved by the oracle's Algorithm 1 (b = 16, tol {tol:g})"}


def measure_rates(device=0):
    """Dense GEMM rates of this GPU through cuBLAS (torch.matmul): TF32, FP32 and FP64, best of 10
    with CUDA events after warm-up (2 N^3 flops each).  The denominators of the TF32 tensor
    fraction and of the FP64 stages; printed as one JSON line."""
    import torch
    dev = torch.device("cuda", device)
    out = {}
    for name, dt, n, tf32 in (("tf32", torch.float32, 8192, True), ("fp32", torch.float32, 8192, False),
                              ("fp64", torch.float64, 4096, False)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device=dev, dtype=dt)
        b = torch.randn(n, n, device=dev, dtype=dt)
        for _ in range(3):
            torch.matmul(a, b)
        best = None
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None else min(best, t)
        out[f"{name}_tflops"] = 2.0 * n ** 3 / best / 1e12
        out[f"{name}_n"] = n
    torch.backends.cuda.matmul.allow_tf32 = False
    out["gpu_name"] = torch.cuda.get_device_name(dev)
    out["torch"] = torch.__version__
    out["how"] = "torch.matmul (cuBLAS) on N x N random operands, best of 10 with CUDA events after 3 warm-up calls"
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg with host buffers")
    ap.add_argument("--no-error", action="store_true", help="single pair: skip the GSV error against the oracle")
    ap.add_argument("--no-sequential", action="store_true", help="batched: skip the one-pair-at-a-time leg")
    ap.add_argument("--error-pairs", type=int, default=8,
                    help="batched: pairs whose GSVs are checked against the FP64 oracle (0: none)")
    ap.add_argument("--pairs", type=int, default=256, help="batched workload: pairs per step")
    ap.add_argument("--workers", type=int, default=16, help="batched workload: concurrent worker streams")
    ap.add_argument("--batched-mode", default="grouped", choices=["grouped", "workers"],
                    help="batched workload: one grouped solve (default) or concurrent per-pair solves")
    ap.add_argument("--train", type=int, default=4096, help="learned workload: training pairs")
    ap.add_argument("--holdout", type=int, default=512, help="learned workload: held-out pairs")
    ap.add_argument("--epochs", type=int, default=60, help="learned workload: training epochs")
    ap.add_argument("--learned-tol", type=float, default=2e-3,
                    help="learned workload: residual tolerance (mixed precision: above the ~4e-4 floor)")
    ap.add_argument("--measure-rates", action="store_true",
                    help="print the cuBLAS TF32 / FP32 / FP64 GEMM rates of this GPU and exit")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.measure_rates:
        return measure_rates(int(os.environ.get("LOCAL_RANK", "0")))

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batched":
        return run_batched(args, rank, world)
    if args.workload == "learned":
        return run_learned(args, rank, world)

    import torch
    import paper_2404_09459_gb300 as P

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    P._build.build()

    spec, default_prec = WORKLOADS[args.workload]
    prec = args.prec or default_prec
    # each rank draws its own pair (independent units)
    from dataclasses import replace
    rspec = replace(spec, seed=rank_seed(spec.seed, rank))
    dt = torch.float64 if prec == "fp64" else torch.float32
    G1, G2, a_true, b_true = planted_pair_torch(rspec, device=f"cuda:{local}", dtype=dt)
    G1u, G2u = G1, G2  # before BF16 storage rounding
    if prec == "bf16":
        dt = torch.bfloat16
        G1, G2 = G1.to(dt), G2.to(dt)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")  # > 129 MB L2
    flags = FLAGS.get(prec, 0)

    ctx = P.Context(prec, device=local, flags=flags)
    for _ in range(args.warmup):
        ctx.solve(G1, G2, spec.kk, spec.oversample, spec.q, rspec.seed)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    st = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = ctx.launch_count()
    barrier()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)  # L2 flush between timed steps (outside the events)
            evs[i][0].record(st)
            out = ctx.solve(G1, G2, spec.kk, spec.oversample, spec.q, rspec.seed)
            evs[i][1].record(st)
        barrier()
    launches = (ctx.launch_count() - l0) // args.steps
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), dist, f"cuda:{local}")
    ms_step = ms / args.steps
    value = world * args.steps / (ms / 1e3)
    tflops = sketch_flops(spec) / (ms_step / 1e3) / 1e12

    # per-stage device time of the same solve (CUDA events on the solve stream)
    pctx = P.Context(prec, device=local, flags=P.FLAG_PROFILE | flags)
    pctx.solve(G1, G2, spec.kk, spec.oversample, spec.q, rspec.seed)
    pctx.profile(reset=True)
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        pctx.solve(G1, G2, spec.kk, spec.oversample, spec.q, rspec.seed)
    prof = pctx.profile()
    pctx.close()
    tot = sum(v[0] for v in prof.values())
    stages = {k: {"ms_per_step": v[0] / args.steps, "calls_per_step": v[1] // args.steps,
                  "share": (v[0] / tot if tot else None)} for k, v in prof.items()}

    # roofline of the sketch product Y = G X (HBM-bound: G read once per launch)
    pk = peaks()
    sk_ms, sk_calls = prof["sketch"]
    el = 8 if prec == "fp64" else (2 if prec == "bf16" else 4)
    # algorithmic bytes of the Y = G X products of one solve ((1 + q) passes over both sides: G (el
    # bytes) + X (el) + Y (FP32 / FP64)), over their device time; a launch covers one side, or both
    # sides when the library groups them
    ey = 8 if prec == "fp64" else 4
    bytes_per_step = (1 + spec.q) * sum(M * spec.n * el + spec.l * spec.n * el + M * spec.l * ey
                                        for M in (spec.m, spec.p))
    calls_step = sk_calls / args.steps if sk_calls else 0
    bytes_per_launch = bytes_per_step / calls_step if calls_step else None
    launch_s = sk_ms / sk_calls / 1e3 if sk_calls else None
    achieved = bytes_per_launch / launch_s / 1e9 if sk_calls else None
    roof = {"kernel": "sketch product Y = G X", "bound": "hbm", "achieved": achieved,
            "peak": pk.get("hbm_gbs"), "unit": "GB/s",
            "frac": (achieved / pk["hbm_gbs"]) if achieved else None,
            "traffic": sketch_traffic(prec, args.workload), "bytes_per_launch": bytes_per_launch,
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if not pk.get("fallback") else "fallback"}
    if prec in ("bf16", "tf32", "tf32x3") and sk_calls:
        # the same launches against the tensor peak: BF16 measured; TF32 at half of it (nominal ratio)
        flops_per_launch = (1 + spec.q) * sum(2.0 * M * spec.n * spec.l for M in (spec.m, spec.p)) / calls_step
        tpk, src = tensor_peak(prec, pk)
        roof["tensor"] = {"achieved_tflops": flops_per_launch / launch_s / 1e12, "peak_tflops": tpk,
                          "frac": flops_per_launch / launch_s / 1e12 / tpk, "peak_source": src}

    # end to end through the public API with host (pinned) buffers
    h1 = torch.empty(G1.shape, dtype=dt, pin_memory=True)
    h2 = torch.empty(G2.shape, dtype=dt, pin_memory=True)
    h1.copy_(G1)
    h2.copy_(G2)
    n1, n2 = h1, h2  # host (pinned) tensors: the library stages them into HBM inside the call
    ectx = P.Context(prec, device=local, flags=flags)
    ectx.solve(n1, n2, spec.kk, spec.oversample, spec.q, rspec.seed)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        out = ectx.solve(n1, n2, spec.kk, spec.oversample, spec.q, rspec.seed)
    barrier()
    e2e_s = time.perf_counter() - t0
    ectx.close()
    e2e = {"value": world * args.steps / e2e_s, "unit": "pairs/s",
           "h2d_bytes_per_step": int((spec.m + spec.p) * spec.n * el),
           "d2h_bytes_per_step": int(2 * spec.kk * 8 + 2 * 8)}

    # plain FP64 GPU path on the same pair (the comparison the metric names)
    fp64 = None
    if not args.no_fp64 and prec != "fp64":
        g1d, g2d = G1.double(), G2.double()
        fctx = P.Context("fp64", device=local)
        fctx.solve(g1d, g2d, spec.kk, spec.oversample, spec.q, rspec.seed)
        torch.cuda.synchronize()
        reps = 2
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            fctx.solve(g1d, g2d, spec.kk, spec.oversample, spec.q, rspec.seed)
        e1.record(st)
        torch.cuda.synchronize()
        fms = e0.elapsed_time(e1) / reps
        fctx.close()
        del g1d, g2d
        fp64 = {"value": 1e3 / fms, "unit": "pairs/s", "ms_per_step": fms, "speedup_of_chosen_form": (1e3 / ms_step) / (1e3 / fms)}

    # accuracy of the timed solve's result against the FP64 oracle on the same stored input (same
    # Philox Omega; BF16: Omega rounded as the BF16 mode rounds it); in BF16 also against the oracle
    # on the unrounded pair (the error of BF16 storage itself) and against the planted pairs
    gsv = None
    if rank == 0 and not args.no_error:
        from oracle import gsvd as O
        got = [tuple(np.asarray(x.cpu() if hasattr(x, "cpu") else x) for x in (out["alpha"], out["beta"]))]
        h1, h2 = G1.double().cpu().numpy(), G2.double().cpu().numpy()
        ref = O.rand_gsvd(h1, h2, spec.kk, spec.oversample, spec.q, rspec.seed,
                          omega_round="bf16" if prec == "bf16" else None)
        del h1, h2
        gsv = gsv_error_summary(got, [(ref["alpha"], ref["beta"])])
        tol = 1e-10 if prec == "fp64" else (1e-3 if prec == "tf32" else 1e-4)
        gsv.update({"tol": tol, "against": "FP64 oracle, same stored input and Omega"})
        if prec == "bf16":
            u1, u2 = G1u.double().cpu().numpy(), G2u.double().cpu().numpy()
            refu = O.rand_gsvd(u1, u2, spec.kk, spec.oversample, spec.q, rspec.seed)
            del u1, u2
            gsv["storage_error_vs_unrounded_fp64"] = gsv_error_summary(got, [(refu["alpha"], refu["beta"])])
            gsv["oracle_unrounded_vs_rounded"] = gsv_error_summary([(ref["alpha"], ref["beta"])],
                                                                   [(refu["alpha"], refu["beta"])])
        gsv["vs_planted"] = gsv_error_summary(got, [(np.asarray(a_true), np.asarray(b_true))])
        gsv["pass"] = gsv["max"] <= tol and gsv["theta_abs_max"] <= 1e-4

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(spec)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": DTYPE.get(prec, prec), "data": "synthetic",
                "config": {"workload": workload_desc(spec, prec), "l2": "flushed between timed steps (256 MiB write)",
                           "parallelism": f"independent pairs, {world} rank(s)"},
                "sketch_tflops": tflops, "roofline": roof, "stages": stages, "gsv_error": gsv, "fp64_plain": fp64,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk.summary()}
        shapes = ctx.product_shapes()
        if any(s for sh in shapes for s in sh):
            # the timed solves' grouped two-side products: (stages, CTAs per SM) the tuner picked
            line["product_pipeline"] = {"first_sketch": shapes[0], "power_sketch": shapes[1],
                                        "gtq_projection": shapes[2]}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
