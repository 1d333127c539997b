#!/usr/bin/env python3
"""Secure decision-forest inference benchmark (COPSE, Algorithm 1) on GB300.

A step is one pass of the whole path over one batch of queries: encode and
encrypt the feature bit-planes, SecComp, reshuffle product, level products
with masks, product across levels, decrypt the leaf bits.  The headline
workload is the encrypted model (Section 8.3) of 32 complete depth-8 trees
(8160 branches, 32 features, 16-bit) at N = 2^15 with 16 primes, 64 queries
per step; further keys time the N = 2^14 plaintext-model forest (4 random
trees, 90..110 branches; one query per step, and the 32 queries one
ciphertext holds), batching, serving and the Table 6 forests.  ``value`` is
measured with the queries' feature words already in device memory; ``e2e``
goes through the C ABI with pinned host buffers (host-to-device copy of the
features and device-to-host copy of the leaf bits inside every step).
``cpu_baseline`` and ``--impl reference`` time the CPU oracle on the host.

Under torchrun (N > 1) every rank runs an independent replica (the method
has no exchange step); value = all ranks' inferences / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "secure inferences/s"
UNIT = "inferences/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--workload", default="encmodel32-n32768")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-stats", action="store_true", help="skip the per-kernel event timers")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (counter captures)")
    ap.add_argument("--profile", action="store_true", help="bracket the timed region with cudaProfilerStart/Stop")
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-serving", action="store_true", help="skip the Poisson-arrival serving leg")
    ap.add_argument("--no-table6", action="store_true", help="skip the per-stage microbenchmark sweep")
    ap.add_argument("--no-tune", action="store_true", help="fixed schedule (dnum 3, plain products, cluster NTT)")
    ap.add_argument("--schedule", default=None,
                    help="dnum,g_reshuffle,g_level,ntt_cluster_max[,ntt_fused_max] for the headline workload instead of tuning "
                         "(e.g. the values a tuned run printed, to profile that schedule)")
    ap.add_argument("--no-forest100", action="store_true", help="skip the N = 2^14 plaintext-model legs")
    ap.add_argument("--forest100-only", action="store_true",
                    help="run only the N = 2^14 plaintext-model legs and print them (counter captures of that step)")
    ap.add_argument("--forest100-steps", type=int, default=200,
                    help="steps of each N = 2^14 plaintext-model leg (one query, batched, plain)")
    return ap.parse_args()


# ---------------------------------------------------------------- distributed
def dist_setup():
    """One process per GPU (replicas: queries are independent, nothing is exchanged on the
    data path).  NCCL with CUDA, gloo without (host-side tests)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    """The slowest rank's time (the job's wall time for weak scaling)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, total_ms, ws):
    """Whole-job value: the units all ranks processed / the slowest rank's time."""
    return ws * units_per_rank / (max_over_ranks(total_ms, ws) / 1e3)


# ---------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = os.path.join("/tmp", f"copse_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.device), "-lms", "50"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.5)  # the sampler is running before the timed region starts
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- roofline inputs
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def ncu_traffic(family, workload, alg_bytes_per_launch, key="dram_bytes_per_unit"):
    """Per-launch DRAM bytes (or another per-unit counter, `key`) from the committed ncu summary
    of this kernel family on this workload, scaled from its per-unit figure to a launch of
    `alg_bytes_per_launch` algorithmic bytes; None when the summary is missing or was taken on a
    different source file than the one built now."""
    path = os.path.join(ROOT, "profiles", f"{family}_{workload}.md")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    kv = {}
    for ln in lines:
        if ln.startswith("- ") and ":" in ln:
            k, v = ln[2:].split(":", 1)
            kv[k.strip()] = v.strip()
    src = os.path.join(ROOT, "paper_2104_09583_gb300", "csrc", kv.get("source", ""))
    try:
        if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != kv.get("source_sha256_16"):
            return None
        units = alg_bytes_per_launch / float(kv["unit_algorithmic_bytes"])
        return float(kv[key]) * units
    except (OSError, KeyError, ValueError):
        return None


# ---------------------------------------------------------------- CUDA arm
# kernel families -> the measured integer rate their algorithmic operations are priced at
PEAK_KIND = {"enc_mac": "tensor", "ks_inner": "mac", **{f: "butterfly" for f in (
    "ntt_fwd", "ntt_inv", "ntt_inv_copy", "ntt_fwd_ms", "ntt_fwd_md", "ntt_fwd_mu", "ntt_fwd_mdd")}}
PEAK_UNIT = {"mac": ("G modular products/s", "exact 64-bit residue products in lazily reduced sums"),
             "butterfly": ("G butterflies/s", "lazy Shoup NTT butterflies"),
             "tensor": ("G flop/s", "dense f16 tensor-core multiply-adds (2 flops each)")}


def int_peaks(K, local):
    """Measured rates of the arithmetic the kernels are priced at: the modular arithmetic on
    this GPU (register-only microbenchmarks, best of 5 CUDA-event timed runs: exact products
    in lazily reduced sums, lazy Shoup butterflies, Barrett products), and the dense f16
    tensor-core rate, the sustained bf16 figure of MEASURED_PEAKS.json (f16 and bf16 have the
    same nominal dense rate, so the ratio is 1; sustained because the kernel runs inside a
    seconds-long step)."""
    ctx = K.copse_ctx_create(10, 55, 4, 2, device=local)
    try:
        out = {}
        for kind in ("mac", "butterfly", "barrett"):
            ops, ms = K.copse_measure_int_peak(ctx, kind, 5)
            out[kind] = {"ops_per_s": ops, "best_ms": ms}
    finally:
        K.copse_ctx_destroy(ctx)
    peaks, how = measured_peaks()
    tf = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    out["tensor"] = {"ops_per_s": tf * 1e12, "source": f"{how} bf16_tflops_sustained (cuBLAS bf16 GEMM, 4 s loop)"}
    return out


def family_roofline(fam, ops, peaks_hbm, how, ipk, workload, steps):
    """Roofline of the dominant kernel family (largest summed CUDA-event time) of an
    instrumented step: HBM bytes (algorithmic) and, where the family counts its modular
    products, the integer roof from the measured rate of that arithmetic."""
    top = max(fam, key=lambda k: fam[k]["ms"])
    v = fam[top]
    sec = v["ms"] * 1e-3
    achieved = v["bytes"] / sec / 1e9
    hbm = {"achieved": achieved, "peak": peaks_hbm, "unit": "GB/s", "frac": achieved / peaks_hbm,
           "peak_source": f"{how} hbm_gbs (copy)"}
    tr = ncu_traffic(top, workload, v["bytes"] / v["launches"])
    kind = PEAK_KIND.get(top)
    if ops.get(top) and kind and ipk:
        ach = ops[top] / sec
        peak = ipk[kind]["ops_per_s"]
        unit, what = PEAK_UNIT[kind]
        if kind == "tensor":
            roof = {"kernel": top, "bound": "tensor", "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                    "frac": ach / peak, "traffic": tr, "hbm": hbm,
                    "peak_source": ipk[kind]["source"] + "; achieved counts the f16 MMA flops issued "
                                   "(padding digits included)"}
        else:
            roof = {"kernel": top, "bound": "alu", "achieved": ach / 1e9, "peak": peak / 1e9,
                    "unit": unit, "frac": ach / peak, "traffic": tr, "hbm": hbm,
                    "peak_source": f"measured in this run: register-only microbenchmark of {what} ({kind}), best of 5"}
    else:
        roof = {"kernel": top, "bound": "hbm", "achieved": achieved, "peak": peaks_hbm, "unit": "GB/s",
                "frac": achieved / peaks_hbm, "traffic": tr, "peak_source": f"{how} hbm_gbs (copy)"}
    roof.update({"algorithmic_bytes_per_launch": v["bytes"] / v["launches"],
                 "avg_launch_us": v["ms"] * 1e3 / v["launches"], "launches_per_step": v["launches"] / steps,
                 "measured_on": "instrumented replay of the timed step (CUDA events around every launch)"})
    return roof


def family_table(fam, steps, ops=None, ipk=None, hbm=None):
    """Per kernel family: launches, time and share per step, HBM GB/s of its algorithmic bytes and,
    where it counts modular operations, their rate and its fraction of the measured peak."""
    tot = max(1e-9, sum(x["ms"] for x in fam.values()))
    out = {}
    for k, v in sorted(fam.items(), key=lambda kv: -kv[1]["ms"]):
        if not v["launches"]:
            continue
        row = {"launches_per_step": v["launches"] / steps, "ms_per_step": v["ms"] / steps, "share": v["ms"] / tot,
               "gbs": v["bytes"] / (v["ms"] * 1e-3) / 1e9 if v["ms"] else 0.0}
        if hbm:
            row["hbm_frac"] = row["gbs"] / hbm
        kind = PEAK_KIND.get(k)
        if ops and ops.get(k) and kind and ipk and v["ms"]:
            rate = ops[k] / (v["ms"] * 1e-3)
            row["int_rate_g"] = rate / 1e9
            row["int_frac"] = rate / ipk[kind]["ops_per_s"]
            row["int_unit"] = PEAK_UNIT[kind][0]
        out[k] = row
    return out


def step_roofline(kernels, ms_per_step):
    """The whole step against its roofs: each kernel family's time had it run at the roof that
    binds it (its measured time x the larger of its HBM and its integer or tensor fraction, at
    most 1), summed over the families, over the measured step time."""
    at_roofs = 0.0
    for row in (kernels or {}).values():
        frac = max(row.get("hbm_frac") or 0.0, row.get("int_frac") or 0.0)
        at_roofs += (row.get("ms_per_step") or 0.0) * min(frac, 1.0)
    if at_roofs <= 0.0 or not ms_per_step:
        return None
    return {"ms_at_roofs": at_roofs, "ms_measured": ms_per_step, "frac": at_roofs / ms_per_step,
            "how": "sum over kernel families of measured ms x max(hbm_frac, int_frac), over ms_per_step"}


def run_cuda(args, ws, rank, local):
    from paper_2104_09583_gb300 import copse as K

    ipk = int_peaks(K, local)
    if args.forest100_only:
        return run_forest100(args, ws, rank, local, ipk)
    line = run_headline(args, ws, rank, local, ipk)
    line["int_peaks"] = ipk
    if not args.no_forest100:
        line["forest100"] = run_forest100(args, ws, rank, local, ipk)
    line["serving"] = None if args.no_serving else run_serving(local, tune=not args.no_tune)
    line["batch3"] = None if args.no_serving else run_batch3(local, tune=not args.no_tune)
    line["table6"] = None if args.no_table6 else run_table6(local)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_baseline_encmodel(synth_workload(args.workload), args.cpu_budget)
        line["cpu_baseline"]["direct"] = oracle_direct("forest100-n16384")
    return line


def synth_workload(name):
    from paper_2104_09583_gb300 import synth
    return synth.WORKLOADS[name]


def run_headline(args, ws, rank, local, ipk):
    """The encrypted-model workload (Maurice = Diane): every model ciphertext (threshold planes,
    all reshuffle and level diagonals, masks) encrypted once; one step = the batch of queries
    encrypted, Algorithm 1 over all their ciphertexts, and the leaf bits decrypted, on one
    stream.  Baby-step sizes from a tuner sweep of this model (copse_tune_bsgs)."""
    import torch

    from paper_2104_09583_gb300 import copse as K

    W = synth_workload(args.workload)
    g = W.bsgs
    text = W.forest_texts()[0]
    N = 1 << W.log_n
    ctx = K.copse_ctx_create(W.log_n, W.bits, W.primes, W.dnum, device=local)
    model = K.copse_compile_forest(text, W.precision(), W.n_features(), W.log_n)
    K.copse_model_set_encrypted(model, True)
    K.copse_model_set_bsgs(model, *g)
    info = K.copse_model_info_get(model)
    per_ct = N // (info["block"] * info["n_segments"])
    t0 = time.perf_counter()
    keys, evk = K.copse_keygen(ctx, 29 + rank, [model])
    torch.cuda.synchronize()
    t_keys = time.perf_counter() - t0
    t0 = time.perf_counter()
    K.copse_encrypt_model(ctx, keys, model, 2024 + rank)
    t_enc = time.perf_counter() - t0
    nq = W.queries[0]
    qs = W.query_arrays()[0]
    want = K.copse_classify_plain(model, qs)
    L = info["n_leaves"]
    stream = torch.cuda.current_stream().cuda_stream
    d_q = torch.from_numpy(qs.astype(np.int32)).cuda()
    d_bits = torch.zeros(nq * L, dtype=torch.uint8, device="cuda")

    def step(seed):
        ct = K.copse_encrypt_features(ctx, keys, model, d_q.data_ptr(), seed, stream=stream, on_device=True,
                                      n_queries=nq)
        res = K.copse_infer(ctx, evk, model, ct, stream=stream)
        K.copse_decrypt_labels(ctx, keys, model, res, nq, stream=stream, out_device_ptr=d_bits.data_ptr())
        K.copse_ctbuf_destroy(res)
        K.copse_ctbuf_destroy(ct)

    for w in range(args.warmup):
        step(500 + 100 * w)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    if args.profile:
        torch.cuda.profiler.start()
    for i in range(args.steps):
        ev[i][0].record()
        step(900 + 100 * i)
        ev[i][1].record()
    torch.cuda.synchronize()
    if args.profile:
        torch.cuda.profiler.stop()
    ck = clocks.stop()
    barrier(ws)
    per = [ev[i][0].elapsed_time(ev[i][1]) for i in range(args.steps)]
    total_ms = max_over_ranks(ev[0][0].elapsed_time(ev[-1][1]), ws)
    ok = bool(np.array_equal(d_bits.cpu().numpy().reshape(nq, L), want))

    # per-kernel event timers over one instrumented step (the same launches as a timed step)
    fam, ops = {}, {}
    if not args.no_stats:
        K.copse_stats_reset()
        K.copse_stats_enable(True)
        step(7000)
        torch.cuda.synchronize()
        K.copse_stats_enable(False)
        fam = {k: v for k, v in K.copse_stats_all().items() if v["launches"]}
        ops = {k: K.copse_stats_get_ops(k) for k in fam}
    peaks, how = measured_peaks()
    roof = family_roofline(fam, ops, peaks["hbm_gbs"], how, ipk, W.name, 1) if fam else None
    launches_step = int(sum(v["launches"] for v in fam.values()))

    # end to end through the C ABI: pinned host features in, leaf bits back to pinned host memory
    h_q = torch.from_numpy(qs.astype(np.int32)).pin_memory()
    h_bits = torch.zeros(nq * L, dtype=torch.uint8).pin_memory()

    def e2e_step(seed):
        ct = K.copse_encrypt_features(ctx, keys, model, h_q.numpy().view(np.uint32), seed, stream=stream)
        res = K.copse_infer(ctx, evk, model, ct, stream=stream)
        K.copse_decrypt_labels(ctx, keys, model, res, nq, stream=stream, out=h_bits.numpy())
        K.copse_ctbuf_destroy(res)
        K.copse_ctbuf_destroy(ct)

    e_steps = 0 if args.no_e2e else max(3, args.steps // 4)
    if e_steps:
        e2e_step(3000)
    barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(e_steps):
        e2e_step(3100 + i)
    e1.record()
    torch.cuda.synchronize()
    e_ms = max(1e-9, max_over_ranks(e0.elapsed_time(e1), ws))
    e2e = {"value": ws * nq * e_steps / (e_ms / 1e3), "unit": UNIT, "steps": e_steps,
           "h2d_bytes_per_step": int(qs.astype(np.uint32).nbytes), "d2h_bytes_per_step": int(nq * L),
           "labels_ok": bool(np.array_equal(h_bits.numpy().reshape(nq, L), want)),
           "path": "copse_encrypt_features (pinned host features) + copse_infer + copse_decrypt_labels (pinned host bits)"}

    n_ct, words = model_ciphertexts(info, W, N)
    K.copse_keys_destroy(keys)
    K.copse_evk_destroy(evk)
    K.copse_model_destroy(model)
    K.copse_ctx_destroy(ctx)
    value = ws * nq * args.steps / (total_ms / 1e3)
    ktab = family_table(fam, 1, ops, ipk, peaks["hbm_gbs"])
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "p50_ms": float(np.percentile(per, 50)),
        "p99_ms": float(np.percentile(per, 99)), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64 (RNS residues mod 55-bit primes)", "data": "synthetic (seeded random forest and queries)",
        "config": {"workload": W.name, "ring_degree": N, "ciphertext_primes": W.primes, "prime_bits": W.bits,
                   "dnum": W.dnum, "model": "encrypted (thresholds, every reshuffle and level diagonal, masks)",
                   "trees": info["n_trees"], "branches": info["b"], "leaves": L, "depth": info["depth"],
                   "features": info["n_features"], "precision": info["precision"], "q": info["q"],
                   "row_segments": info["n_segments"], "block": info["block"],
                   "queries_per_step": nq, "queries_per_ciphertext": per_ct,
                   "query_ciphertexts": (nq + per_ct - 1) // per_ct, "bsgs": list(g),
                   "rotation_keys": info["n_rot_reshuffle"] + info["n_rot_level"], "parallelism": f"replicas{ws}",
                   "model_ciphertexts": n_ct, "model_gb_on_device": round(words * 8 / 1e9, 1),
                   "model_encryption_s": round(t_enc, 2), "keygen_s": round(t_keys, 2),
                   "l2": "inputs larger than L2 (the encrypted model alone is %.0f GB)" % (words * 8 / 1e9)},
        "labels_ok": ok, "path": "copse_encrypt_features + copse_infer + copse_decrypt_labels on one stream",
        "e2e": e2e, "gpu_launches": launches_step * args.steps, "roofline": roof,
        "kernels": ktab, "step_roofline": step_roofline(ktab, total_ms / args.steps), "clocks": ck,
    }


def model_ciphertexts(info, W, N):
    """Count and device words (c0 only) of the encrypted model: p threshold planes at the top level,
    q reshuffle diagonals at the level of Decisions, d (b + 1) level diagonals and masks one level
    lower, b the branch count of one slot block."""
    b = info["block_branches"]
    lvl_D = W.primes - 1 - (info["precision"] - 1).bit_length()
    n_ct = info["precision"] + info["q"] + info["depth"] * (b + 1)
    words = (info["precision"] * W.primes + info["q"] * lvl_D + info["depth"] * (b + 1) * (lvl_D - 1)) * N
    return n_ct, words


def run_forest100(args, ws, rank, local, ipk):
    """The N = 2^14 plaintext-model forest (4 random trees, 90..110 branches): one query per step
    through a recorded graph session, 32 queries per ciphertext batched, and the plain path
    (every kernel launched from the host, no graph)."""
    import torch

    from paper_2104_09583_gb300 import copse as K
    from paper_2104_09583_gb300 import synth

    W = synth.WORKLOADS["forest100-n16384"]
    text = W.forest_texts()[0]
    N = 1 << W.log_n
    model = K.copse_compile_forest(text, W.precision(), W.n_features(), W.log_n)
    dnum, tuning = W.dnum, None
    sched = [int(x) for x in args.schedule.split(",")] if args.schedule else None
    if sched:
        dnum = sched[0]
        K.copse_model_set_bsgs(model, sched[1], sched[2])
        tuning = {"fixed_schedule": sched}
    elif not args.no_tune:
        dnum, dn_ms = K.copse_tune_dnum(W.log_n, W.bits, W.primes, model, [1, 2, 3, 4], 1, 3, device=local)
        tuning = {"dnum_ms_per_inference": dn_ms}
    ctx = K.copse_ctx_create(W.log_n, W.bits, W.primes, dnum, device=local)
    if sched:
        K.copse_ctx_set_ntt_cluster_max(ctx, sched[3])
        if len(sched) > 4:
            K.copse_ctx_set_ntt_fused_max(ctx, sched[4])
    elif not args.no_tune:
        tuning.update(autotune(K, ctx, [model]))
    info = K.copse_model_info_get(model)
    keys, evk = K.copse_keygen(ctx, 7 + rank, [model])
    stream = torch.cuda.current_stream().cuda_stream
    per_ct = N // info["block"]
    nf, L = info["n_features"], info["n_leaves"]
    steps = args.forest100_steps

    def make_inputs(nq, seed):
        q = synth.random_queries(seed, nq, nf, W.precision())
        d_feats = torch.from_numpy(q.astype(np.int32)).cuda()
        d_bits = torch.zeros(max(nq * L, 1), dtype=torch.uint8, device="cuda")
        return q, d_feats, d_bits

    def step(nq, d_feats, d_bits, seed):
        ct = K.copse_encrypt_features(ctx, keys, model, d_feats.data_ptr(), seed, stream=stream, on_device=True,
                                      n_queries=nq)
        res = K.copse_infer(ctx, evk, model, ct, stream=stream)
        K.copse_decrypt_labels(ctx, keys, model, res, nq, stream=stream, out_device_ptr=d_bits.data_ptr())
        K.copse_ctbuf_destroy(res)
        K.copse_ctbuf_destroy(ct)

    def timed(nq, steps, warmup, seed0, stats=False):
        q, d_feats, d_bits = make_inputs(nq, seed0 + rank)
        for w in range(warmup):
            step(nq, d_feats, d_bits, 1000 + w)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        if stats:
            K.copse_stats_reset()
            K.copse_stats_enable(True)
        for i in range(steps):
            ev[i][0].record()
            step(nq, d_feats, d_bits, 2000 + i)
            ev[i][1].record()
        torch.cuda.synchronize()
        if stats:
            K.copse_stats_enable(False)
        per = [ev[i][0].elapsed_time(ev[i][1]) for i in range(steps)]
        total_ms = ev[0][0].elapsed_time(ev[-1][1])
        got = d_bits[: nq * L].cpu().numpy().reshape(nq, L)
        return total_ms, per, bool(np.array_equal(got, K.copse_classify_plain(model, q)))

    def timed_session(sess, nq, steps, warmup, seed0, profile=False):
        """Graph-replayed steps (copse_session_run) on device-resident features and bits."""
        q, d_feats, d_bits = make_inputs(nq, seed0 + rank)
        run = lambda seed: K.copse_session_run(sess, None, seed, stream=stream, feats_ptr=d_feats.data_ptr(),
                                               out_ptr=d_bits.data_ptr())
        for w in range(warmup):
            run(5000 + w)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        if profile:
            torch.cuda.profiler.start()
        for i in range(steps):
            ev[i][0].record()
            run(6000 + i)
            ev[i][1].record()
        torch.cuda.synchronize()
        if profile:
            torch.cuda.profiler.stop()
        per = [ev[i][0].elapsed_time(ev[i][1]) for i in range(steps)]
        total_ms = ev[0][0].elapsed_time(ev[-1][1])
        got = d_bits[: nq * L].cpu().numpy().reshape(nq, L)
        return total_ms, per, bool(np.array_equal(got, K.copse_classify_plain(model, q)))

    def leg(ms, per, ok, nq, n, path):
        return {"queries_per_step": nq, "value": nq * n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / n,
                "p50_ms": float(np.percentile(per, 50)), "p99_ms": float(np.percentile(per, 99)),
                "labels_ok": ok, "path": path}

    sess1 = K.copse_session_create(ctx, keys, evk, model, 1)
    sessB = K.copse_session_create(ctx, keys, evk, model, per_ct)
    one = leg(*timed_session(sess1, 1, steps, 3, 11, profile=args.profile and args.forest100_only), 1, steps,
              "graph session, one query per step")
    batched = leg(*timed_session(sessB, per_ct, steps, 3, 21), per_ct, steps,
                  f"graph session, {per_ct} queries per ciphertext")
    plain = leg(*timed(1, steps, 3, 31), 1, steps, "host-launched operations, one query, no graph")
    # per-kernel event timers over instrumented host-launched steps
    timed(1, steps, 1, 41, stats=True)
    fam = {k: v for k, v in K.copse_stats_all().items() if v["launches"]}
    ops = {k: K.copse_stats_get_ops(k) for k in fam}
    peaks, how = measured_peaks()
    K.copse_session_destroy(sess1)
    K.copse_session_destroy(sessB)
    K.copse_keys_destroy(keys)
    K.copse_evk_destroy(evk)
    K.copse_model_destroy(model)
    K.copse_ctx_destroy(ctx)
    n_rot = info["n_rot_reshuffle"] + info["n_rot_level"]
    alpha = -(-W.primes // dnum)
    key_gb = n_rot * dnum * 2 * (W.primes + alpha) * N * 8 / 1e9
    return {"workload": W.name, "ring_degree": N, "ciphertext_primes": W.primes, "dnum": dnum, "tuning": tuning,
            "branches": info["b"], "leaves": L, "depth": info["depth"], "one_query": one, "batched": batched,
            "plain_ops": plain, "kernels": family_table(fam, steps, ops, ipk, peaks["hbm_gbs"]),
            "roofline": family_roofline(fam, ops, peaks["hbm_gbs"], how, ipk, W.name, steps) if fam else None,
            "rotation_keys": n_rot,
            "key_working_set_gb": round(key_gb, 2), "l2": "working set > L2 (rotation keys %.1f GB)" % key_gb}


def autotune(K, ctx, models, g_r=(0, 16, 32, 64), g_l=(0, 4, 8), nq=1):
    """NTT kernel crossover for the context, then baby-step sizes per model (fastest stage times)."""
    lim, _ = K.copse_tune_ntt(ctx)
    plans = []
    for m in models:
        K.copse_tune_bsgs(ctx, m, list(g_r), list(g_l), nq, 3)
        plans.append(list(K.copse_model_get_bsgs(m)))
    # the fused transforms' crossover, by whole inferences of the largest model
    fused, fused_ms = K.copse_tune_fused(ctx, models[-1], n_queries=nq)
    return {"ntt_cluster_max_polys": lim, "ntt_fused_max_polys": fused, "fused_ms_per_inference": fused_ms,
            "bsgs_plans": plans}


# ---------------------------------------------------------------- serving
def run_serving(local, rate=200.0, n_req=1000, warm=100, seed=5, tune=True):
    """Poisson arrivals (mean `rate` per second) of single queries against four resident models,
    each chosen uniformly: the shapes of the three smaller workloads (1 tree of depth 3; 4 random
    trees, ~100 branches; 16 trees of depth 6) on an N = 2^14 server and a 64-tree depth-6 8-bit
    forest, whose query block needs N = 2^15, on a second server.  Each server batches its
    requests continuously into graph launches.  Latency is submit -> completion as the server
    measures it; throughput is completed requests over the offered time of the measured part."""
    import queue
    import threading

    from paper_2104_09583_gb300 import copse as K
    from paper_2104_09583_gb300 import synth

    Wt, Wf, Wb = (synth.WORKLOADS[n] for n in ("toy-n1024", "forest100-n16384", "batch3-n16384"))
    # (text, precision, features, ring) per model
    specs = [(Wt.forest_texts()[0], Wt.precision(), Wt.n_features(), 14),
             (Wf.forest_texts()[0], Wf.precision(), Wf.n_features(), 14),
             (Wb.forest_texts()[2], Wb.precision(2), Wb.n_features(2), 14),
             (synth.random_forest(5004, 64, 6, 16, 8, 4, complete=True), 8, 16, 15)]
    rings = {}
    for log_n in (14, 15):
        ids = [k for k, sp in enumerate(specs) if sp[3] == log_n]
        ctx = K.copse_ctx_create(log_n, Wf.bits, Wf.primes, 2, device=local)
        ms = [K.copse_compile_forest(specs[k][0], specs[k][1], specs[k][2], log_n) for k in ids]
        if tune:
            # the 64-tree reshuffle has ~3700 diagonals: its plain key set is not an option
            autotune(K, ctx, ms, g_r=(32, 64, 128) if log_n == 15 else (0, 16, 32, 64), g_l=(0, 8, 16))
        elif log_n == 15:
            K.copse_model_set_bsgs(ms[0], 64, 0)
        keys, evk = K.copse_keygen(ctx, 13, ms)
        srv = K.copse_server_create(ctx, keys, evk, ms)
        rings[log_n] = (ctx, ms, keys, evk, srv, ids)
    route = {}
    models = [None] * len(specs)
    for log_n, (ctx, ms, keys, evk, srv, ids) in rings.items():
        for local_id, k in enumerate(ids):
            route[k] = (srv, local_id)
            models[k] = ms[local_id]
    infos = [K.copse_model_info_get(m) for m in models]
    rng = np.random.default_rng(seed)
    total = warm + n_req
    choice = rng.integers(len(models), size=total)
    gaps = rng.exponential(1.0 / rate, size=total)
    qs = [synth.random_queries(10000 + i, 1, infos[k]["n_features"], specs[k][1])[0] for i, k in enumerate(choice)]
    tickets = queue.Queue()
    refused = [0]

    def submitter():
        t_next = time.perf_counter()
        for i in range(total):
            t_next += gaps[i]
            d = t_next - time.perf_counter()
            if d > 0:
                time.sleep(d)
            srv_k, mid = route[int(choice[i])]
            try:
                tickets.put((i, int(choice[i]), K.copse_server_submit(srv_k, mid, qs[i])))
            except K.CopseError:
                refused[0] += 1
                tickets.put((i, int(choice[i]), None))

    th = threading.Thread(target=submitter)
    t0 = time.perf_counter()
    th.start()
    lat, ok, t_first, t_last = [], True, None, None
    lat_by = {k: [] for k in range(len(specs))}
    for _ in range(total):
        i, k, t = tickets.get()
        if t is None:
            continue
        bits, ms = K.copse_server_poll(route[k][0], t, infos[k]["n_leaves"], 60000)
        ok &= bool(np.array_equal(bits, K.copse_classify_plain(models[k], qs[i][None, :])[0]))
        if i >= warm:
            lat.append(ms)
            lat_by[k].append(ms)
            now = time.perf_counter()
            t_first = t_first if t_first is not None else now
            t_last = now
    th.join()
    wall = time.perf_counter() - t0
    for ctx, ms, keys, evk, srv, ids in rings.values():
        K.copse_server_destroy(srv)
        K.copse_keys_destroy(keys)
        K.copse_evk_destroy(evk)
        for m in ms:
            K.copse_model_destroy(m)
        K.copse_ctx_destroy(ctx)
    measured_s = sum(gaps[warm:])
    return {"value": len(lat) / measured_s, "unit": UNIT, "offered_rate": rate, "requests": n_req,
            "warmup_requests": warm, "refused": refused[0], "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(np.mean(lat)), "labels_ok": ok,
            "models": [f"{i['n_trees']} trees, {i['b']} branches, block {i['block']}, N = 2^{sp[3]}"
                       for i, sp in zip(infos, specs)],
            "per_model": [{"requests": len(v), "p50_ms": float(np.percentile(v, 50)) if v else None,
                           "p99_ms": float(np.percentile(v, 99)) if v else None} for v in lat_by.values()],
            "wall_s": wall}


def run_batch3(local, steps=3, warmup=1, tune=True):
    """256 queries over three forests (1 x depth 3, 4 x depth 5, 16 x depth 6; 8/16/32 features, 8-bit)
    evaluated by one graph launch: one work item per ciphertext (32 + 3 x 32 + 32 x 4 queries)."""
    import torch

    from paper_2104_09583_gb300 import copse as K
    from paper_2104_09583_gb300 import synth

    W = synth.WORKLOADS["batch3-n16384"]
    texts = W.forest_texts()
    models = [K.copse_compile_forest(t, W.precision(k), W.n_features(k), W.log_n) for k, t in enumerate(texts)]
    dnum, tuning = W.dnum, None
    if tune:
        # digit count on the largest forest, then the NTT crossover and every forest's plan
        dnum, dn_ms = K.copse_tune_dnum(W.log_n, W.bits, W.primes, models[2], [2, 3, 4], 1, 2, device=local)
        tuning = {"dnum": dnum, "dnum_ms_per_inference": dn_ms}
    ctx = K.copse_ctx_create(W.log_n, W.bits, W.primes, dnum, device=local)
    if tune:
        tuning.update(autotune(K, ctx, models, g_r=(0, 16, 32, 64), g_l=(0, 8, 16)))
    keys, evk = K.copse_keygen(ctx, 17, models)
    infos = [K.copse_model_info_get(m) for m in models]
    per = [(1 << W.log_n) // i["block"] for i in infos]
    items = []
    for k, nq in enumerate(W.queries):
        while nq > 0:
            items.append((k, min(per[k], nq)))
            nq -= per[k]
    qa = W.query_arrays()
    feats, used = [], [0] * len(models)
    for k, n in items:
        feats.append(qa[k][used[k]: used[k] + n].reshape(-1))
        used[k] += n
    feats = np.concatenate(feats)
    out = np.zeros(sum(n * infos[k]["n_leaves"] for k, n in items), dtype=np.uint8)
    sess = K.copse_session_create_batch(ctx, keys, evk, [models[k] for k, _ in items], [n for _, n in items])
    stream = torch.cuda.current_stream().cuda_stream
    for w in range(warmup):
        K.copse_session_run(sess, feats, 70 + w, out, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for i in range(steps):
        K.copse_session_run(sess, feats, 80 + i, out, stream=stream)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ok, off, used = True, 0, [0] * len(models)
    for k, n in items:
        Lk = infos[k]["n_leaves"]
        want = K.copse_classify_plain(models[k], qa[k][used[k]: used[k] + n])
        ok &= bool(np.array_equal(out[off: off + n * Lk].reshape(n, Lk), want))
        off += n * Lk
        used[k] += n
    K.copse_session_destroy(sess)
    K.copse_keys_destroy(keys)
    K.copse_evk_destroy(evk)
    for m in models:
        K.copse_model_destroy(m)
    K.copse_ctx_destroy(ctx)
    return {"value": 256 / (ms / 1e3), "unit": UNIT, "ms_per_launch": ms, "queries_per_launch": 256,
            "items": len(items), "labels_ok": ok, "tuning": tuning,
            "forests": [f"{i['n_trees']} trees, {i['b']} branches, {i['n_rot_reshuffle']}+{i['n_rot_level']} "
                        f"rotations, {p} queries/ciphertext" for i, p in zip(infos, per)]}


# ---------------------------------------------------------------- Table 6 microbenchmarks
def run_table6(local, reps=7, warmup=2, log_n=14, bits=55, primes=11, dnum=3):
    """The eight microbenchmark forests of Section 8.4 (Table 6; 2 features, 3 labels),
    one query each, with the device time of every step of Algorithm 1 (comparison,
    reshuffling, level processing, aggregation): median over `reps` timed inferences."""
    from paper_2104_09583_gb300 import copse as K
    from paper_2104_09583_gb300 import synth

    ctx = K.copse_ctx_create(log_n, bits, primes, dnum, device=local)
    out = {}
    try:
        for name in sorted(synth.TABLE6):
            depth, p, per_tree = synth.TABLE6[name]
            text = synth.table6_forest(name)
            model = K.copse_compile_forest(text, p, synth.TABLE6_FEATURES, log_n)
            keys, evk = K.copse_keygen(ctx, 23, [model])
            info = K.copse_model_info_get(model)
            qs = synth.random_queries(200 + sorted(synth.TABLE6).index(name), 1, synth.TABLE6_FEATURES, p)
            want = K.copse_classify_plain(model, qs)
            rows, ok = [], True
            for r in range(warmup + reps):
                feats = K.copse_encrypt_features(ctx, keys, model, qs, 300 + r)
                res, ms = K.copse_infer_timed(ctx, evk, model, feats)
                bits_ = K.copse_decrypt_labels(ctx, keys, model, res, 1)
                ok &= bool(np.array_equal(bits_, want))
                K.copse_ctbuf_destroy(res)
                K.copse_ctbuf_destroy(feats)
                if r >= warmup:
                    rows.append([ms[k] for k in K.STAGES])
            med = np.median(np.asarray(rows), axis=0)
            out[name] = {"depth": depth, "precision": p, "trees": len(per_tree), "branches": int(info["b"]),
                         "rotations": int(info["n_rot_reshuffle"] + info["n_rot_level"]),
                         **{f"{k}_ms": round(float(v), 4) for k, v in zip(K.STAGES, med)},
                         "total_ms": round(float(med.sum()), 4), "labels_ok": ok}
            K.copse_keys_destroy(keys)
            K.copse_evk_destroy(evk)
            K.copse_model_destroy(model)
    finally:
        K.copse_ctx_destroy(ctx)
    return {"ring_degree": 1 << log_n, "ciphertext_primes": primes, "prime_bits": bits,
            "queries_per_inference": 1, "stat": f"median of {reps} (host-launched, per-stage CUDA events)",
            "models": out}


# ---------------------------------------------------------------- CPU oracle (baseline / reference arm)
class OracleBench:
    """The oracle on the encrypted-model workload: exact operation counts of one step (the
    batch of queries through Algorithm 1 with the model encrypted, under the same baby-step
    plan as the CUDA arm) and timed samples of each operation at the level where the circuit
    runs it.  A whole step takes the oracle days (millions of ciphertext products at
    N = 2^15), so the step time is extrapolated from the samples with the exact counts."""

    def __init__(self, W, text):
        from oracle import bgv as B
        from oracle import copse as Cp

        self.B, self.Cp, self.W = B, Cp, W
        self.m = m = Cp.compile_forest(text, W.precision(), W.n_features(), slots_per_row=1 << (W.log_n - 1))
        self.P = P = B.Params(logN=W.log_n, L=W.primes, bits=W.bits, dnum=W.dnum)
        self.bgv = B.Bgv(P)
        g = W.bsgs
        rs, ls = Cp.encrypted_rotation_sets(m, g)
        self.keys = self.bgv.keygen(7, [B.galois_rot(W.log_n, rs[0])])
        self.galois = B.galois_rot(W.log_n, rs[0])
        p, d = m.precision, m.d
        per_ct = (1 << W.log_n) // (m.block * m.n_seg)
        self.n_ct = -(-W.queries[0] // per_ct)
        gr, gl = g
        babies_r, babies_l = len({i % gr for i in range(m.q)} - {0}), len({i % gl for i in range(m.b)} - {0})
        giants_r, giants_l = len({i - i % gr for i in range(m.q)} - {0}), len({i - i % gl for i in range(m.b)} - {0})
        acc_r, acc_l = giants_r + 1, d * (giants_l + 1)
        c = self.n_ct
        self.lvl_D = P.L - 1 - (p - 1).bit_length()
        # per step: the operation counts of every query ciphertext
        self.n = {"enc": c * p, "mul_hi": c * (p + 2 * p - 3), "tensor_D": c * m.q, "tensor_B": c * d * m.b,
                  "relin": c * (acc_r + acc_l), "rot_D": c * (babies_r + giants_r),
                  "rot_B": c * (babies_l + d * giants_l), "mul_lo": c * (d - 1)}
        self._t = {}            # operation kind -> its timings (seconds); the estimate takes the median

    def _clock(self, f, *a):
        s = time.perf_counter()
        f(*a)
        return time.perf_counter() - s

    def _op(self, kind):
        B, bgv, P, k = self.B, self.bgv, self.P, self.keys
        if not hasattr(self, "_x"):
            z = np.zeros(P.N, dtype=np.int64)
            self._x = bgv.encrypt_slots(k.pk, z, 99, 0)
            self._xD = bgv.to_level(self._x, self.lvl_D)
            self._xB = bgv.to_level(self._x, self.lvl_D - 1)
            self._dD = bgv.encrypt_sk(k.sk, B.encode(P, z), 5, 1, self.lvl_D)
            self._dB = bgv.encrypt_sk(k.sk, B.encode(P, z), 5, 2, self.lvl_D - 1)
            self._t3 = bgv.tensor(self._dD, self._xD)
        if kind == "enc":
            return self._clock(bgv.encrypt_slots, k.pk, np.zeros(P.N, dtype=np.int64), 99, 1)
        if kind == "mul_hi":
            return self._clock(bgv.mul, self._x, self._x, k.rlk)
        if kind == "mul_lo":
            return self._clock(bgv.mul, self._xB, self._xB, k.rlk)
        if kind == "tensor_D":
            return self._clock(bgv.tensor, self._dD, self._xD)
        if kind == "tensor_B":
            return self._clock(bgv.tensor, self._dB, self._xB)
        if kind == "relin":
            return self._clock(bgv.relin, self._t3, k.rlk)
        if kind == "rot_D":
            return self._clock(bgv.rotate, self._xD, self.galois, k.gk[self.galois])
        return self._clock(bgv.rotate, self._xB, self.galois, k.gk[self.galois])

    def estimate(self):
        return sum(self.n[kd] * statistics.median(self._t[kd]) for kd in self.n)

    def sample_all(self):
        """Time every operation kind once -> (seconds per step, description)."""
        t0 = time.perf_counter()
        for kd in self.n:
            self._t.setdefault(kd, []).append(self._op(kd))
        return self.estimate(), self.describe(time.perf_counter() - t0)

    def sample_one(self, i):
        """One step of the reference arm: the i-th operation kind (round robin) timed again."""
        if not self._t:
            return self.sample_all()
        kinds = list(self.n)
        t0 = time.perf_counter()
        self._t[kinds[i % len(kinds)]].append(self._op(kinds[i % len(kinds)]))
        return self.estimate(), self.describe(time.perf_counter() - t0)

    def describe(self, cpu_s):
        n = self.n
        runs = sum(len(v) for v in self._t.values())
        return (f"oracle ({self.B.oracle_threads()} threads) timed on the step's operations at their levels "
                f"({runs} timings over the {len(self.n)} kinds, median per kind; {cpu_s:.1f} s of CPU work in this "
                f"sample: encrypt, ciphertext product at the top and bottom of the chain, tensor with an encrypted "
                f"diagonal at the reshuffle and level levels, relinearisation, rotation at both levels); one step of "
                f"{self.W.queries[0]} queries ({self.n_ct} query ciphertexts) extrapolated with its exact counts: "
                f"{n['enc']} encryptions, {n['mul_hi'] + n['mul_lo']} products, "
                f"{n['tensor_D'] + n['tensor_B']} tensors, {n['relin']} relinearisations, "
                f"{n['rot_D'] + n['rot_B']} rotations")


def oracle_baseline_encmodel(W, budget_s):
    """On all host cores: every operation kind timed once, then again round robin until about
    budget_s seconds of oracle work are spent; the step estimate takes each kind's median.  Then
    one timing of every kind on a single thread, for the same estimate at one core."""
    ob = OracleBench(W, W.forest_texts()[0])
    t0 = time.perf_counter()
    est, _ = ob.sample_all()
    i = 0
    while time.perf_counter() - t0 + statistics.median(ob._t[list(ob.n)[i % len(ob.n)]]) <= budget_s:
        est, _ = ob.sample_one(i)
        i += 1
    sample = ob.describe(time.perf_counter() - t0)
    cores = ob.B.oracle_threads()
    line = {"value": W.queries[0] / est, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "seconds_per_step_extrapolated": est}
    ob._t = {}
    ob.B.set_oracle_threads(1)
    try:
        t1 = time.perf_counter()
        est1, _ = ob.sample_all()
        line["one_core"] = {"value": W.queries[0] / est1, "unit": UNIT, "cores": 1,
                            "seconds_per_step_extrapolated": est1,
                            "sample": f"one timing of each of the {len(ob.n)} operation kinds on one thread "
                                      f"({time.perf_counter() - t1:.1f} s), extrapolated as above"}
    finally:
        ob.B.set_oracle_threads(cores)
    return line


def oracle_direct(name, seed=1):
    """The oracle's whole inference of one full query ciphertext of a plaintext-model workload,
    timed directly (no extrapolation): encrypt the queries' bit-planes, Algorithm 1, decrypt the
    leaf bits; keys are made before the timed region, as on the GPU."""
    from oracle import bgv as B
    from oracle import copse as Cp
    from paper_2104_09583_gb300 import synth

    W = synth.WORKLOADS[name]
    text = W.forest_texts()[0]
    m = Cp.compile_forest(text, W.precision(), W.n_features())
    P = B.Params(logN=W.log_n, L=W.primes, bits=W.bits, dnum=W.dnum)
    bgv = B.Bgv(P)
    keys = bgv.keygen(7, Cp.galois_elements(m, W.log_n))
    nq = P.N // m.block
    qs = synth.random_queries(seed, nq, W.n_features(), W.precision())
    t0 = time.perf_counter()
    X = Cp.encrypt_queries(bgv, keys, m, qs, 9)
    out = Cp.infer(Cp.BgvEngine(bgv, keys), m, X, P.N)
    bits = Cp.decode_labels(m, bgv.decrypt_slots(keys.sk, out), nq)
    dt = time.perf_counter() - t0
    _, trees = Cp.parse_forest(text)
    return {"workload": name, "value": nq / dt, "unit": UNIT, "cores": B.oracle_threads(), "queries": nq,
            "seconds": dt, "labels_ok": all(bits[j] == Cp.classify_plain(trees, qs[j]) for j in range(nq)),
            "sample": f"the oracle's whole inference of one query ciphertext ({nq} queries, N = {P.N}, "
                      f"{W.primes} primes): encryption, Algorithm 1 and decryption timed directly"}


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    W = synth_workload(args.workload)
    ob = OracleBench(W, W.forest_texts()[0])
    for i in range(args.warmup):
        ob.sample_one(i)
    ests, walls, sample = [], [], ""
    for i in range(args.steps):
        t0 = time.perf_counter()
        est, sample = ob.sample_one(i)
        walls.append(time.perf_counter() - t0)
        ests.append(est)
    est = statistics.mean(ests)
    value = W.queries[0] / est
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(walls) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64 (RNS residues mod 55-bit primes)",
            "data": "synthetic (seeded random forest and queries)", "config": {"workload": W.name},
            "ms_per_step_note": "each reference step is a bounded sample: one operation of the workload timed "
                                "(round robin); value re-estimates the whole 64-query step from the exact operation "
                                "counts (extrapolated_ms_per_full_step)",
            "extrapolated_ms_per_full_step": est * 1e3,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": ob.B.oracle_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        line = run_reference(args, ws, rank)
    else:
        line = run_cuda(args, ws, rank, local)
    if rank == 0 and line is not None:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
