#!/usr/bin/env python3
"""Secure decision-forest inference benchmark (COPSE, Algorithm 1) on GB300.

A step is one pass of the whole path over one batch of queries: encode and
encrypt the feature bit-planes, SecComp, reshuffle product, level products
with masks, product across levels, decrypt the leaf bits.  The default
workload is the N = 2^14, 10-prime forest (4 random trees, 90..110 branches,
8 features, 8-bit) with one query per step; the batched line packs the 32
queries one ciphertext holds.  ``value`` is measured with the queries'
feature words already in device memory; ``e2e`` goes through the C ABI with
pinned host buffers (host-to-device copy of the features and device-to-host
copy of the leaf bits inside every step).  ``--impl reference`` times the
CPU oracle on the host instead.

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
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["cuda", "reference"], default="cuda")
    ap.add_argument("--workload", default="forest100-n16384")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-stats", action="store_true", help="skip the per-kernel event timers")
    ap.add_argument("--profile", action="store_true", help="bracket the timed region with cudaProfilerStart/Stop")
    ap.add_argument("--cpu-budget", type=float, default=20.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-serving", action="store_true", help="skip the Poisson-arrival serving leg")
    ap.add_argument("--no-table6", action="store_true", help="skip the per-stage microbenchmark sweep")
    ap.add_argument("--no-tune", action="store_true", help="fixed schedule (dnum 3, plain products, cluster NTT)")
    ap.add_argument("--schedule", default=None,
                    help="dnum,g_reshuffle,g_level,ntt_cluster_max[,ntt_fused_max] for the headline workload instead of tuning "
                         "(e.g. the values a tuned run printed, to profile that schedule)")
    ap.add_argument("--no-encmodel", action="store_true", help="skip the encrypted-model leg")
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
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


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
def run_cuda(args, ws, rank, local):
    import torch

    from paper_2104_09583_gb300 import copse as K
    from paper_2104_09583_gb300 import synth

    W = synth.WORKLOADS[args.workload]
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

    def timed(nq, steps, warmup, seed0, stats=False, clocks=None, profile=False):
        q, d_feats, d_bits = make_inputs(nq, seed0 + rank)
        for w in range(warmup):
            step(nq, d_feats, d_bits, 1000 + w)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier(ws)
        torch.cuda.synchronize()
        if stats:
            K.copse_stats_reset()
            K.copse_stats_enable(True)
        if clocks:
            clocks.start()
        if profile:
            torch.cuda.profiler.start()
        for i in range(steps):
            ev[i][0].record()
            step(nq, d_feats, d_bits, 2000 + i)
            ev[i][1].record()
        torch.cuda.synchronize()
        if profile:
            torch.cuda.profiler.stop()
        ck = clocks.stop() if clocks else None
        if stats:
            K.copse_stats_enable(False)
        barrier(ws)
        per = [ev[i][0].elapsed_time(ev[i][1]) for i in range(steps)]
        total_ms = ev[0][0].elapsed_time(ev[-1][1])
        # decrypted bits of the last step against plaintext classification
        got = d_bits[: nq * L].cpu().numpy().reshape(nq, L)
        ok = bool(np.array_equal(got, K.copse_classify_plain(model, q)))
        return total_ms, per, ok, ck

    def timed_session(sess, nq, steps, warmup, seed0, clocks=None, profile=False):
        """Graph-replayed steps (copse_session_run) on device-resident features and bits."""
        q, d_feats, d_bits = make_inputs(nq, seed0 + rank)
        run = lambda seed: K.copse_session_run(sess, None, seed, stream=stream, feats_ptr=d_feats.data_ptr(),
                                               out_ptr=d_bits.data_ptr())
        for w in range(warmup):
            run(5000 + w)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier(ws)
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        if profile:
            torch.cuda.profiler.start()
        for i in range(steps):
            ev[i][0].record()
            run(6000 + i)
            ev[i][1].record()
        torch.cuda.synchronize()
        if profile:
            torch.cuda.profiler.stop()
        ck = clocks.stop() if clocks else None
        barrier(ws)
        per = [ev[i][0].elapsed_time(ev[i][1]) for i in range(steps)]
        total_ms = ev[0][0].elapsed_time(ev[-1][1])
        got = d_bits[: nq * L].cpu().numpy().reshape(nq, L)
        ok = bool(np.array_equal(got, K.copse_classify_plain(model, q)))
        return total_ms, per, ok, ck

    sess1 = K.copse_session_create(ctx, keys, evk, model, 1)
    sessB = K.copse_session_create(ctx, keys, evk, model, per_ct)
    clocks = Clocks(local)
    # headline: one query per step, the recorded graph replayed
    total_ms, per, ok, ck = timed_session(sess1, 1, args.steps, args.warmup, 11, clocks=clocks, profile=args.profile)
    total_ms = max_over_ranks(total_ms, ws)
    value = ws * args.steps / (total_ms / 1e3)
    # batched: every slot block of the ciphertext holds a query
    b_steps = max(3, args.steps // 2)
    b_ms, b_per, b_ok, _ = timed_session(sessB, per_ct, b_steps, args.warmup, 21)
    b_ms = max_over_ranks(b_ms, ws)
    batched = {"queries_per_step": per_ct, "value": ws * per_ct * b_steps / (b_ms / 1e3), "unit": UNIT,
               "ms_per_step": b_ms / b_steps, "p50_ms": float(np.percentile(b_per, 50)),
               "p99_ms": float(np.percentile(b_per, 99)), "labels_ok": b_ok, "path": "graph session"}
    # the plain GPU path: one query, every kernel launched from the host, no graph
    p_ms, p_per, p_ok, _ = timed(1, b_steps, args.warmup, 31)
    p_ms = max_over_ranks(p_ms, ws)
    plain_ops = {"queries_per_step": 1, "value": ws * b_steps / (p_ms / 1e3), "unit": UNIT,
                 "ms_per_step": p_ms / b_steps, "p50_ms": float(np.percentile(p_per, 50)),
                 "p99_ms": float(np.percentile(p_per, 99)), "labels_ok": p_ok, "path": "host-launched operations"}
    # per-kernel event timers over an instrumented replay of the same step (host-launched)
    fam = {}
    if not args.no_stats:
        timed(1, args.steps, 1, 41, stats=True)
        fam = K.copse_stats_all()

    # end to end through the C ABI: pinned host features in, leaf bits back to pinned host memory
    q = synth.random_queries(31 + rank, 1, nf, W.precision())
    h_feats = torch.from_numpy(q.copy()).pin_memory()
    h_bits = torch.zeros((1, L), dtype=torch.uint8).pin_memory()

    def e2e_step(seed):
        K.copse_session_run(sess1, h_feats.numpy(), seed, out=h_bits.numpy(), stream=stream)

    for w in range(args.warmup):
        e2e_step(3000 + w)
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(args.steps):
        e2e_step(4000 + i)
    e1.record()
    torch.cuda.synchronize()
    e_ms = max_over_ranks(e0.elapsed_time(e1), ws)
    e2e = {"value": ws * args.steps / (e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(q.nbytes) + 8,
           "d2h_bytes_per_step": int(L), "labels_ok": bool(np.array_equal(h_bits.numpy(), K.copse_classify_plain(model, q)))}
    K.copse_session_destroy(sess1)
    K.copse_session_destroy(sessB)

    # roofline of the dominant kernel family (largest summed event time)
    peaks, how = measured_peaks()
    roof = None
    launches_total = 0
    kern = {}
    if fam:
        # the graph replays exactly the kernels of the instrumented host-launched step
        launches_total = int(sum(v["launches"] for v in fam.values()))
        for k, v in fam.items():
            if v["launches"]:
                kern[k] = {"launches_per_step": v["launches"] / args.steps, "ms_per_step": v["ms"] / args.steps,
                           "share": v["ms"] / max(1e-9, sum(x["ms"] for x in fam.values())),
                           "gbs": v["bytes"] / (v["ms"] * 1e-3) / 1e9 if v["ms"] else 0.0}
        top = max(fam, key=lambda k: fam[k]["ms"])
        v = fam[top]
        achieved = v["bytes"] / (v["ms"] * 1e-3) / 1e9
        tr = ncu_traffic(top, args.workload, v["bytes"] / v["launches"])
        hbm = {"achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
               "peak_source": f"{how} hbm_gbs (copy)"}
        wi = ncu_traffic(top, args.workload, v["bytes"] / v["launches"], key="warp_instructions_per_unit")
        if wi is not None:
            # integer issue roof: 152 SMs x 4 schedulers x 1 warp instruction per clock at the
            # maximum SM clock; achieved = the ncu instruction count per unit scaled to the
            # average launch, over its CUDA-event duration
            peak_wi = 152 * 4 * 2.07e9 / 1e9
            ach_wi = wi / (v["ms"] * 1e-3 / v["launches"]) / 1e9
            roof = {"kernel": top, "bound": "alu", "achieved": ach_wi, "peak": peak_wi,
                    "unit": "G warp-instructions/s", "frac": ach_wi / peak_wi, "traffic": tr, "hbm": hbm,
                    "peak_source": "152 SMs x 4 schedulers x 1 warp instruction/clock x 2.07 GHz"}
        else:
            roof = {"kernel": top, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "traffic": tr, "peak_source": f"{how} hbm_gbs (copy)"}
        roof.update({"algorithmic_bytes_per_launch": v["bytes"] / v["launches"],
                     "avg_launch_us": v["ms"] * 1e3 / v["launches"],
                     "measured_on": "instrumented host-launched replay of the timed step (CUDA events per launch)"})

    serving = None if args.no_serving else run_serving(local, tune=not args.no_tune)
    batch3 = None if args.no_serving else run_batch3(local, tune=not args.no_tune)
    table6 = None if args.no_table6 else run_table6(local)
    encmodel = None if args.no_encmodel else run_encmodel(local)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(W, text, args.cpu_budget)

    for h in (keys,):
        K.copse_keys_destroy(h)
    K.copse_evk_destroy(evk)
    K.copse_model_destroy(model)
    K.copse_ctx_destroy(ctx)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "p50_ms": float(np.percentile(per, 50)),
        "p99_ms": float(np.percentile(per, 99)), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64 (RNS residues mod 55-bit primes)", "data": "synthetic (seeded random forest and queries)",
        "config": {"workload": W.name, "ring_degree": N, "ciphertext_primes": W.primes, "prime_bits": W.bits,
                   "dnum": dnum, "tuning": tuning, "trees": 4, "branches": info["b"], "leaves": L, "depth": info["depth"],
                   "features": nf, "precision": W.precision(), "queries_per_step": 1, "parallelism": f"replicas{ws}",
                   "l2": "working set > L2 (rotation keys with their Shoup companions alone are about %.1f GB)" % (
                       (info["n_rot_reshuffle"] + info["n_rot_level"]) * 3 * 2 * (W.primes + 4) * N * 8 * 2 / 1e9)},
        "labels_ok": ok, "path": "graph session", "batched": batched, "plain_ops": plain_ops, "e2e": e2e,
        "serving": serving, "batch3": batch3, "table6": table6, "encmodel": encmodel, "gpu_launches": launches_total,
        "roofline": roof, "kernels": kern, "clocks": ck, "cpu_baseline": cpu,
    }
    return line


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


# ---------------------------------------------------------------- encrypted model
def run_encmodel(local, steps=1, warmup=1, g=(128, 256)):
    """The encrypted-model workload (Maurice = Diane): 32 random trees of depth <= 8, 32 features,
    16-bit, 10 classes, N = 2^15 with 16 primes; every model ciphertext (thresholds, all reshuffle
    and level diagonals, masks) encrypted once; one step = the 64 queries (2 per ciphertext, 32
    ciphertexts) encrypted, inferred together and decrypted on one stream.  Baby-step sizes from
    a tuner sweep of this model (copse_tune_bsgs: 128 / 256 fastest)."""
    import torch

    from paper_2104_09583_gb300 import copse as K
    from paper_2104_09583_gb300 import synth

    W = synth.WORKLOADS["encmodel32-n32768"]
    text = W.forest_texts()[0]
    N = 1 << W.log_n
    ctx = K.copse_ctx_create(W.log_n, W.bits, W.primes, W.dnum, device=local)
    model = K.copse_compile_forest(text, W.precision(), W.n_features(), W.log_n)
    K.copse_model_set_encrypted(model, True)
    K.copse_model_set_bsgs(model, *g)
    info = K.copse_model_info_get(model)
    per_ct = N // info["block"]
    t0 = time.perf_counter()
    keys, evk = K.copse_keygen(ctx, 29, [model])
    torch.cuda.synchronize()
    t_keys = time.perf_counter() - t0
    t0 = time.perf_counter()
    K.copse_encrypt_model(ctx, keys, model, 2024)
    t_enc = time.perf_counter() - t0
    nq = W.queries[0]
    qs = W.query_arrays()[0]
    want = K.copse_classify_plain(model, qs)
    L = info["n_leaves"]
    stream = torch.cuda.current_stream().cuda_stream
    d_q = torch.from_numpy(qs.astype(np.int32)).cuda()
    d_bits = torch.zeros(nq * L, dtype=torch.uint8, device="cuda")

    def step(seed):
        # all query ciphertexts in one buffer: the products read each encrypted diagonal
        # (and regenerate its mask) once per group of query ciphertexts
        ct = K.copse_encrypt_features(ctx, keys, model, d_q.data_ptr(), seed, stream=stream, on_device=True,
                                      n_queries=nq)
        res = K.copse_infer(ctx, evk, model, ct, stream=stream)
        K.copse_decrypt_labels(ctx, keys, model, res, nq, stream=stream, out_device_ptr=d_bits.data_ptr())
        K.copse_ctbuf_destroy(res)
        K.copse_ctbuf_destroy(ct)

    for w in range(warmup):
        step(500 + 100 * w)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(steps):
        step(900 + 100 * i)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ok = bool(np.array_equal(d_bits.cpu().numpy().reshape(nq, L), want))
    # per-stage breakdown of one ciphertext's inference, then its kernels by family
    ct = K.copse_encrypt_features(ctx, keys, model, qs[:per_ct], 77)
    res, stages = K.copse_infer_timed(ctx, evk, model, ct)
    K.copse_ctbuf_destroy(res)
    K.copse_stats_reset()
    K.copse_stats_enable(True)
    res = K.copse_infer(ctx, evk, model, ct)
    torch.cuda.synchronize()
    K.copse_stats_enable(False)
    fam = {k: {"launches": v["launches"], "ms": round(v["ms"], 3)} for k, v in K.copse_stats_all().items()
           if v["launches"]}
    fam = dict(sorted(fam.items(), key=lambda kv: -kv[1]["ms"])[:8])
    K.copse_ctbuf_destroy(res)
    K.copse_ctbuf_destroy(ct)
    n_ct = info["precision"] + info["q"] + info["depth"] * (info["b"] + 1)
    lvl_D = W.primes - 1 - (info["precision"] - 1).bit_length()
    words = (info["precision"] * W.primes + info["q"] * lvl_D + info["depth"] * (info["b"] + 1) * (lvl_D - 1)) * N
    K.copse_keys_destroy(keys)
    K.copse_evk_destroy(evk)
    K.copse_model_destroy(model)
    K.copse_ctx_destroy(ctx)
    return {"value": nq / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "queries_per_step": nq,
            "ciphertexts_per_step": (nq + per_ct - 1) // per_ct, "labels_ok": ok,
            "stage_ms_one_ciphertext": stages, "kernels_one_ciphertext": fam, "model_ciphertexts": n_ct,
            "model_gb_on_device": round(words * 8 / 1e9, 1), "model_encryption_s": round(t_enc, 2),
            "keygen_s": round(t_keys, 2), "bsgs": list(g), "rotation_keys": info["n_rot_reshuffle"] + info["n_rot_level"],
            "model": f"{info['n_trees']} trees, {info['b']} branches, depth {info['depth']}, q {info['q']}, "
                     f"{info['precision']}-bit, N = 2^{W.log_n}, {W.primes} primes"}


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
    """The oracle on the benchmark workload: operation counts of one inference
    (exact, from the compiled model and the circuit's structure) and timed
    samples of its operations at the levels where the circuit runs them."""

    def __init__(self, W, text):
        from oracle import bgv as B
        from oracle import copse as Cp

        self.B, self.Cp = B, Cp
        self.m = m = Cp.compile_forest(text, W.precision(), W.n_features())
        self.P = P = B.Params(logN=W.log_n, L=W.primes, bits=W.bits, dnum=W.dnum)
        self.bgv = B.Bgv(P)
        self.rs, self.ls = Cp.rotation_sets(m)
        self.keys = self.bgv.keygen(7, [B.galois_rot(W.log_n, k) for k in self.rs[:2]])
        self.qs = W.query_arrays()[0]
        p = m.precision
        self.n = {"affine": 2 * p, "mul": max(0, 2 * p - 3) + (m.d - 1), "rot": len(self.rs) + len(self.ls),
                  "pt": len(Cp.reshuffle_diagonals(m)) + sum(len(Cp.level_diagonals(m, k, P.t))
                                                             for k in range(1, m.d + 1))}
        self.Rd = {i: Cp.tile_blocks(m, dg, P.N) for i, dg in Cp.reshuffle_diagonals(m).items()}

    def _clock(self, f, *a):
        s = time.perf_counter()
        r = f(*a)
        return r, time.perf_counter() - s

    def _op(self, kind):
        """Run and time one operation of the workload's inference (seconds)."""
        Cp, bgv, m = self.Cp, self.bgv, self.m
        if not hasattr(self, "_X"):
            self._X = Cp.encrypt_queries(bgv, self.keys, m, self.qs, 99)
            self._E = Cp.BgvEngine(bgv, self.keys)
            self._Y = self._E.thresholds(m)
            lvl_D = self.P.L - 1 - (m.precision - 1).bit_length()
            self._v = bgv.to_level(self._X[0], lvl_D)
        E, X, Y = self._E, self._X, self._Y
        if kind == "enc":
            return self._clock(Cp.encrypt_queries, bgv, self.keys, m, self.qs, 99)[1]
        if kind == "affine":
            return self._clock(E.affine, X[0], (-Y[0]) % E.t, Y[0])[1]
        if kind == "mul":
            return self._clock(E.mul, X[0], X[1 % len(X)])[1]
        k = self.rs[0]
        if kind == "rot":
            return self._clock(E.rot, self._v, k)[1]
        return self._clock(E.mul_plain, self._v, self.Rd[k])[1]

    def sample_small(self):
        """One step of the reference arm: one operation of the workload timed (round robin over
        encrypt of all planes, affine leaf, multiply, rotation, plaintext product; every one
        timed once first), the inference time extrapolated from the latest time of each with
        the inference's exact counts -> seconds per inference."""
        kinds = ("enc", "affine", "mul", "rot", "pt")
        if not hasattr(self, "_t"):
            self._t = {kd: self._op(kd) for kd in kinds}
            self._next = 0
        else:
            kd = kinds[self._next % len(kinds)]
            self._t[kd] = self._op(kd)
            self._next += 1
        t, n, m = self._t, self.n, self.m
        est = t["enc"] + n["affine"] * t["affine"] + n["mul"] * t["mul"] + n["rot"] * t["rot"] + n["pt"] * t["pt"]
        return est, (f"oracle, one operation of the workload timed per step (round robin over encrypt of "
                     f"{m.precision} planes, affine leaf, multiply, rotation at the reshuffle level, plaintext "
                     f"product); one inference extrapolated with its exact counts ({n['affine']} affine, "
                     f"{n['mul']} multiplies, {n['rot']} rotations, {n['pt']} plaintext products)")

    def sample_large(self, budget_s):
        """Encrypt and the whole SecComp, then reshuffle terms while the budget lasts -> s/inference."""
        Cp, bgv, m = self.Cp, self.bgv, self.m
        t0 = time.perf_counter()
        X = Cp.encrypt_queries(bgv, self.keys, m, self.qs, 99)
        t_enc = time.perf_counter() - t0
        times = {"mul": []}

        class Timed(Cp.BgvEngine):
            def mul(s_, a, b):
                s = time.perf_counter()
                r = Cp.BgvEngine.mul(s_, a, b)
                times["mul"].append(time.perf_counter() - s)
                return r

        E = Timed(bgv, self.keys)
        t1 = time.perf_counter()
        D = Cp.seccomp(E, X, E.thresholds(m), m.precision)
        t_sec = time.perf_counter() - t1
        t_rot, t_pt = [], []
        for k in self.rs[:2]:
            r, tr = self._clock(E.rot, D, k)
            _, tp = self._clock(E.mul_plain, r, self.Rd[k])
            t_rot.append(tr)
            t_pt.append(tp)
            if time.perf_counter() - t0 > budget_s:
                break
        n = self.n
        est = (t_enc + t_sec + n["rot"] * statistics.mean(t_rot) + n["pt"] * statistics.mean(t_pt)
               + (m.d - 1) * statistics.mean(times["mul"]))
        return est, (f"oracle timed on encrypt ({m.precision} planes), the whole SecComp, {len(t_rot)} rotations and "
                     f"plaintext products of the reshuffle ({time.perf_counter() - t0:.1f} s of CPU work); one "
                     f"inference extrapolated with its exact counts ({n['rot']} rotations, {n['pt']} plaintext "
                     f"products, {m.d - 1} more multiplies): {est:.1f} s/inference")


def oracle_baseline(W, text, budget_s):
    est, sample = OracleBench(W, text).sample_large(budget_s)
    return {"value": 1.0 / est, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}


def run_reference(args, ws, rank):
    from paper_2104_09583_gb300 import synth

    if rank != 0:
        return None
    W = synth.WORKLOADS[args.workload]
    ob = OracleBench(W, W.forest_texts()[0])
    for _ in range(args.warmup):
        ob.sample_small()
    ests, sample = [], ""
    for _ in range(args.steps):
        est, sample = ob.sample_small()
        ests.append(est)
    est = statistics.mean(ests)
    value = 1.0 / est
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": est * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64 (RNS residues mod 55-bit primes)",
            "data": "synthetic (seeded random forest and queries)", "config": {"workload": W.name},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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
