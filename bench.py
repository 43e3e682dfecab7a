"""Benchmark: amortized ms per encrypted Softmax (n = 256, N = 2^16, bootstrapping), batched vs plain.

Workload (default "m64"): 8192 Softmax of dimension 256 packed into m = 64 ciphertexts at
N = 2^16 (the paper's many-ciphertext setting, Sec. 4.2 / Table 6), inputs shaped like
attention logits q.k/sqrt(64), q, k ~ N(0, 1), shifted by a public bound and clipped to
[-128, 0].  "m1": 128 Softmax of dimension 256 in one ciphertext.

A step is one Softmax over the whole batch, ciphertexts already resident in HBM (a pristine
copy is restored into the working buffer inside the step): he_softmax_graph, i.e. a replay of
the circuit captured as one CUDA graph in the first warm-up step.  --method picks the circuit:
alg4 (default; Alg. 4 version B with the auxiliary thread of Alg. 3, Sec. 4.3: only the
auxiliary ciphertext is bootstrapped) or alg2 (Alg. 2 with Alg. 3, Sec. 4.2); the other one is
timed too (other_method).  Plain: he_softmax one ciphertext at a time, eager.  The timed region
is bracketed by a barrier and a synchronize, timed with CUDA events on the library's stream.
e2e: the same metric through he_softmax with the ciphertexts copied from pinned host memory
to the device and the results copied back, inside the timed region, every timed step;
e2e_x_to_y: FP64 inputs in host memory encrypted (he_encrypt), the Softmax, and the outputs
decrypted into host memory (he_decrypt), every timed step.
precision: worst/avg/std of the bits of max |error| against FP64 Softmax over seeds 0-4 and
three input recipes, and (with the CPU leg) the split into polynomial approximation
(the oracle's FP64 simulation of the circuit against FP64 Softmax) and CKKS noise
(decryption against that simulation).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                       [--workload m64|m1] [--method alg4|alg2] [--profile-kernel NAME]
Under torchrun each rank runs an independent replica (weak scaling, no collective on the
data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "amortized ms/Softmax (n=256, N=2^16, >=15-bit prec) batched vs plain; p99 ms"


def workload(name):
    if name == "m1":
        return {"workload": "1 ciphertext, 128 Softmax of dim 256, N=2^16, bootstrapping", "m": 1, "n": 256}
    return {"workload": "64 ciphertexts, 8192 Softmax of dim 256, N=2^16, bootstrapping", "m": 64, "n": 256}


def attention_logits(L, n, seed, M=128.0, d=64, bound=8.0):
    """q.k/sqrt(d) with q, k ~ N(0, 1) per row, minus a public bound, clipped to [-M, 0]."""
    from paper_2410_11184_gb300 import workloads

    return workloads.attention_logits(L, n, seed, M=M, d=d, bound=bound)


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes per limb (ncu dram__bytes_read.sum + dram__bytes_write.sum of both passes over the
# limbs of the launch) of the N = 2^16 transforms in 64-thread CTAs, the autotuner's usual pick:
# forward (167.9 + 112.8 + 173.1 + 107.6) MB over 320 limbs, inverse (409.2 + 341.9 + 402.9 + 347.3)
# MB over 768 limbs (python -m paper_2410_11184_gb300.profile_case keyswitch_small)
NTT_DRAM_PER_LIMB = {"fwd": (167.870464 + 112.770048 + 173.091072 + 107.571712) * 1e6 / 320,
                     "inv": (409.172224 + 341.905664 + 402.891520 + 347.335424) * 1e6 / 768}

# Warp instructions per limb of the N = 2^16 transforms (ncu smsp__inst_executed.sum of both passes
# of one capture, divided by the limbs of the launch), same captures: forward (63 283 200 +
# 72 744 960) over 320 limbs, inverse (166 232 064 + 210 173 952) over 768 limbs
# (profiles/ntt_instruction_mix_n65536.txt).  The NTT is bound by integer instruction issue (64-bit
# modular butterflies on 32-bit pipes), so its roofline is the SM issue limit: 152 SMs x 4
# sub-partitions x 1 warp instruction per cycle x 2070 MHz (the SM count and maximum SM clock of
# GB300; four schedulers per SM on this architecture).
NTT_WARP_INSTR_PER_LIMB = {"fwd": (63283200 + 72744960) / 320, "inv": (166232064 + 210173952) / 768}
ISSUE_PEAK_G = 152 * 4 * 2.070   # G warp instructions / s

# integer pipes of the NTT passes (ncu, same captures): issue active of the four passes weighted by
# their durations; ALU / FMA (IMAD) pipe cycles of the forward passes in 256-thread CTAs
NTT_INT_PIPES = {"issue_active_pct": 52.8, "alu_pct": 40.3, "fma_imad_pct": 38.3,
                 "source": "ncu, k_ntt_{cols,rows}_{fwd,inv}_rb<4> (profiles/ntt_instruction_mix_n65536.txt)"}

# circuits: the plan file entry each method evaluates at n = 256 on [-128, 0]
METHODS = {"alg4": ("n256_M128_B", "Alg. 4 (version B) + Alg. 3 auxiliary thread, Sec. 4.3"),
           "alg2": ("n256_M128", "Alg. 2 + Alg. 3 auxiliary thread, Sec. 4.2")}
# ciphertext key switches per step (he_counters of the GPU run) of each method and workload,
# used by the reference arm's scaling
KS_PER_STEP = {("alg2", "m64"): 7969, ("alg2", "m1"): 847, ("alg4", "m64"): 2744, ("alg4", "m1"): 1280}


def load_plan(he, method):
    name = METHODS[method][0]
    return he.load_plans_b()[name] if name.endswith("_B") else he.load_params()[1][name]


def bits(err):
    return -math.log2(err) if err > 0 else None


def stats_bits(errs):
    b = [-math.log2(e) for e in errs if e > 0]
    return {"worst": min(b), "avg": statistics.mean(b), "std": statistics.pstdev(b), "runs": len(b)} if b else None


def recipes(L, n, seed, M):
    """the three synthetic input recipes (stand-ins for the paper's LLaMa logits)"""
    from paper_2410_11184_gb300 import workloads as W

    return {"uniform": W.uniform_inputs(L, n, seed, M), "paper_normal": W.paper_normal_inputs(L, n, seed, M),
            "attention": W.attention_logits(L, n, seed, M=M)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return p["hbm_gbs"], "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_simulation(runs, plan):
    """The CPU leg's second part: the oracle's FP64 simulation of the circuit (its polynomials,
    no encryption) on the inputs of the precision runs; returns per run (max |O2 - O1|,
    max |dec - O2|): polynomial approximation and CKKS noise."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O

    out = []
    for x, y in runs:
        o2 = (O.simulate_b(x, plan) if plan.get("version") == "B" else O.simulate(x, plan))[0]
        out.append((float(np.abs(o2 - O.softmax_fp64(x)).max()), float(np.abs(y - o2).max())))
    return out


def cpu_full_toy_softmax():
    """One whole Softmax of the oracle at N = 2^12 (128 Softmax of dim 16 on [-8, 0], k = 2, no
    bootstrapping): a measured full run, not an extrapolation."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O

    chains, plans, _ = O.load_params()
    ch, pl = chains["toy"], plans["cfg1_n16_M8"]
    o = O.Oracle(ch)
    o.keygen(11)
    n = pl["n"]
    x = np.random.default_rng(0).uniform(-pl["M"], 0, (o.n0 // n, n))
    top = ch["user_top_level"]
    ct = o.encrypt(O.pack(x, 1, o.n0)[0], top, (2 / pl["M"]) * o.q[top], 5, 0)
    o.softmax([ct], pl)   # rotation keys made outside the timing
    t0 = time.perf_counter()
    o.softmax([ct], pl)
    dt = time.perf_counter() - t0
    return {"workload": "N=2^12, 1 ciphertext, 128 Softmax of dim 16, k=2, no bootstrapping",
            "ms": dt * 1e3, "ms_per_softmax": dt * 1e3 / (o.n0 // n)}


def cpu_baseline(steps_unit_ks, ms_per_softmax_scale):
    """Times the CPU oracle (as it stands) on a bounded sample: one relinearised multiplication
    at the top user level and one rotation at the top bootstrapping level of the N = 2^16
    chain; the mean key-switch time is scaled by the circuit's key-switch count per Softmax
    (counted by the GPU run).  That assumes every key switch of the step costs what these two
    do (it leaves out plaintext products, encodings and NTT-only work)."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O

    chains, plans, evalmod = O.load_params()
    ch = chains["fgb16"]
    o = O.Oracle(ch)
    o.keygen(11)
    rng = np.random.default_rng(0)
    a = o.encrypt(rng.uniform(-1, 1, o.n0), ch["user_top_level"], 2.0 ** 42, 3)
    top = len(o.q) - 1
    b = o.encrypt(rng.uniform(-1, 1, o.n0), top, 2.0 ** 42, 4)
    o.hmult(a, a)           # key generation outside the timing
    o.rotate(b, 1)
    t0 = time.perf_counter()
    reps = 3
    for _ in range(reps):
        o.hmult(a, a)
        o.rotate(b, 1)
    dt = time.perf_counter() - t0
    per_ks_ms = dt / (2 * reps) * 1e3
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {
        "value": per_ks_ms * steps_unit_ks * ms_per_softmax_scale,
        "unit": "ms/Softmax",
        "cores": cores,
        "kind": "oracle",
        "sample": "%d x (HMult at level %d + rotation at level %d), N=2^16, %.1f s; mean key switch %.0f ms "
                  "scaled by %d key switches per step / Softmax per step" % (reps, ch["user_top_level"], top, dt,
                                                                            per_ks_ms, steps_unit_ks),
    }


def run_reference(args, wl):
    """The CPU oracle timed as the reference arm: per step, the same bounded sample as the
    CPU baseline (key switches at the circuit's levels), scaled to ms/Softmax."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # ciphertext key switches per Softmax step of this workload (the circuit's operation list, as
    # counted by he_counters on the GPU path: 64-ciphertext batch / one ciphertext)
    ks_per_step = KS_PER_STEP[(args.method, args.workload)]
    L = wl["m"] * 32768 // wl["n"]
    vals = []
    for _ in range(args.warmup + args.steps):
        cb = cpu_baseline(ks_per_step, 1.0 / L)
        vals.append(cb["value"])
    v = statistics.median(vals[args.warmup:])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms/Softmax", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * L, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64 (RNS residues)", "data": "synthetic",
            "config": {"workload": wl["workload"], "n": wl["n"], "m": wl["m"], "softmax_per_step": L,
                       "method": METHODS[args.method][1]},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "ms/Softmax", "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_serve(args):
    """Serving workload: Poisson arrivals of one-ciphertext encrypted Softmax requests whose
    dimension is drawn from {128, 256, 1024, 4096, 32768} (inputs uniform on [-64, 0], N = 2^16
    with bootstrapping), admitted by HBM budget and batched by shape (serve.Server).  Dimensions
    up to 1024 use the Alg. 2 plans, 4096 and 32768 the Alg. 4 plans (Alg. 2 does not converge
    there on this chain).  Prints one JSON line with p50/p99 request latency, Softmax/s and
    the worst-case error per dimension."""
    print(json.dumps(serve_measure(args, args.requests, args.rate)))


def serve_measure(args, requests, rate):
    """The serving run of run_serve (its own contexts, keys and server); returns its line.
    --serve-lanes contexts with the same keys: batches of different shapes run concurrently."""
    import torch

    from paper_2410_11184_gb300 import he, serve, workloads

    chains, plans, evalmod = he.load_params()
    plans = dict(plans, **he.load_plans_b())
    names = ["n128_M64", "n256_M64", "n1024_M64", "n4096_M64_B"] + (["n32768_M64_B"] if "n32768_M64_B" in plans else [])
    ctxs = []
    for _ in range(max(1, args.serve_lanes)):
        c = he.Context(chains["fgb16"], evalmod["fgb16"])
        c.keygen(5)   # the same keys in every lane
        for nm in names:
            c.keygen_softmax(plans[nm]["n"], 1)
        ctxs.append(c)
    g = ctxs[0]
    rng = np.random.default_rng(args.seed)
    pool = {}
    for nm in names:   # a few distinct encrypted inputs per dimension, in pinned host memory
        pl = plans[nm]
        L = g.n0 // pl["n"]
        for v in range(3):
            x = workloads.uniform_inputs(L, pl["n"], 1000 + 10 * pl["n"] + v, pl["M"])
            ct = g.encrypt(x, pl["n"], 1, pl["M"], 77 + v)
            host = torch.empty(ct.tensor.numel(), dtype=torch.int64).pin_memory()
            host.copy_(ct.tensor)
            pool[(nm, v)] = (x, host, ct.level, ct.scale)
    # warm-up: one Softmax per dimension in every lane (first use of each plan's masks and diagonals)
    for c in ctxs:
        for nm in names:
            x, host, lv, sc = pool[(nm, 0)]
            w = c.alloc(lv, 1, sc)
            w.tensor.copy_(host)
            c.softmax_grouped(w, plans[nm], 1)
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    budget = 0.5 * free
    srv = serve.Server(ctxs, {nm: plans[nm] for nm in names}, budget, max_batch_ct=args.max_batch_ct)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, requests))
    picks = [(names[rng.integers(len(names))], int(rng.integers(3))) for _ in range(requests)]
    t0 = time.perf_counter()
    handles = []
    for t, key in zip(arrivals, picks):
        dt = t0 + t - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        x, host, lv, sc = pool[key]
        handles.append((key, srv.submit(key[0], host, 1, lv, sc)))
    for _, h in handles:
        h.wait(1800)
    srv.close()
    st = srv.stats()
    # precision of every distinct result (decrypted on the device)
    worst = {}
    for key, h in handles:
        x = pool[key][0]
        n = plans[key[0]]["n"]
        words = 2 * (h.out_level + 1) * g.n
        ct = g.alloc(h.out_level, 1, h.out_scale)
        ct.tensor.copy_(h.host_out[:words])
        e = np.exp(x - x.max(axis=1, keepdims=True))
        err = float(np.abs(g.decrypt(ct, n) - e / e.sum(axis=1, keepdims=True)).max())
        worst[n] = max(worst.get(n, 0.0), err)
    softmax_done = sum(g.n0 // plans[k[0]]["n"] for k, _ in handles)
    line = {
        "metric": "serving: request latency p50/p99 and Softmax/s (n in %s, N=2^16, bootstrapping)"
                  % sorted(plans[nm]["n"] for nm in names),
        "value": st["p99_ms"], "unit": "ms (p99 request latency)", "higher_is_better": False,
        "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
        "softmax_per_s": softmax_done / st["span_s"], "requests": st["requests"], "span_s": st["span_s"],
        "arrival_rate_per_s": rate, "batches": st["batches"], "mean_batch_requests": st["mean_batch_requests"],
        "lanes": st["lanes"],
        "precision_bits_by_n": {str(n): -math.log2(e) if e > 0 else None for n, e in sorted(worst.items())},
        "n_gpus": 1, "dtype": "u64 (RNS residues mod 42-60-bit primes)", "data": "synthetic",
        "config": {"workload": "Poisson arrivals, one ciphertext per request, dims %s on [-64, 0] (4096 and "
                                "32768 by Alg. 4)" % "/".join(str(plans[nm]["n"]) for nm in names),
                   "hbm_budget_gb": budget / 1e9, "max_batch_ct": args.max_batch_ct, "lanes": len(ctxs)},
    }
    srv = None
    del g, ctxs, c
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return line


def run_llama(args):
    """LLaMa-7B-shaped batch: 32 layers x 32 heads x 128 query rows = 131072 Softmax of dimension
    128 (context length 128), logits q.k/sqrt(128) with q, k ~ N(0, sigma^2), sigma ~ U[0.5, 1.5]
    per head, minus a public bound 16 and clipped to [-64, 0].  Each layer is one
    many-ciphertext group (4096 Softmax in 16 ciphertexts, n/m = 8, Sec. 4.2); a step runs all
    32 groups, --layers-per-pass of them per he_softmax_grouped call."""
    import torch

    from paper_2410_11184_gb300 import he, workloads

    chains, plans, evalmod = he.load_params()
    pl = he.load_plans_b()["n128_M64_B"] if args.method == "alg4" else plans["n128_M64"]
    n, M, layers, m = pl["n"], pl["M"], 32, 16
    stream = torch.cuda.Stream()
    g = he.Context(chains["fgb16"], evalmod["fgb16"], stream=stream)
    g.keygen(31)
    g.keygen_softmax(n, m)
    L = m * g.n0 // n   # 4096 Softmax per layer
    xs, cts = [], []
    for layer in range(layers):
        x = workloads.attention_logits(L, n, 500 + layer, M=M, d=128, bound=16.0, sigma="per_head",
                                       rows_per_head=128)
        xs.append(x)
        cts.append(g.encrypt(x, n, m, M, 600 + layer))
    per = args.layers_per_pass
    srcs = [he.Ciphertexts(g, torch.cat([c.tensor for c in cts[i:i + per]]), cts[0].level, cts[0].scale, per * m)
            for i in range(0, layers, per)]
    del cts
    works = [g.like(s) for s in srcs]

    def step():
        for s, w in zip(srcs, works):
            w.tensor.copy_(s.tensor)
            w.level, w.scale, w.n_ct = s.level, s.scale, s.n_ct
            g.softmax_grouped(w, pl, per)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        ev[0].record(stream)
        for i in range(args.steps):
            step()
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
    per_step = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    ms_step = ev[0].elapsed_time(ev[-1]) / args.steps
    bits = []
    for i, w in enumerate(works):   # every layer of the last step against FP64 Softmax
        lw = m * 2 * (w.level + 1) * g.n   # the output batch is stored compactly at its level
        for j in range(per):
            one = he.Ciphertexts(g, w.tensor[j * lw:(j + 1) * lw], w.level, w.scale, m)
            x = xs[i * per + j]
            e = np.exp(x - x.max(axis=1, keepdims=True))
            err = float(np.abs(g.decrypt(one, n) - e / e.sum(axis=1, keepdims=True)).max())
            bits.append(-math.log2(err))
    total = layers * L
    print(json.dumps({
        "metric": "amortized ms/Softmax (LLaMa-7B shape: 32 layers x 32 heads x 128 rows, n=128, N=2^16)",
        "value": ms_step / total, "unit": "ms/Softmax", "higher_is_better": False, "ms_per_step": ms_step,
        "p99_ms_per_step": max(per_step), "softmax_per_step": total, "steps": args.steps, "warmup": args.warmup,
        "precision_bits_min_over_layers": min(bits), "precision_bits_max_over_layers": max(bits),
        "n_gpus": 1, "dtype": "u64 (RNS residues mod 42-60-bit primes)", "data": "synthetic",
        "config": {"workload": "32 per-layer groups of 16 ciphertexts (4096 Softmax each), %d groups per pass" % per,
                   "n": n, "M": M, "k": pl["k"], "ciphertexts": layers * m,
                   "method": METHODS[args.method][1].replace("n = 256", "n = 128")},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="m64", choices=["m64", "m1", "serve", "llama"])
    ap.add_argument("--layers-per-pass", type=int, default=4, help="llama: layer groups per grouped pass")
    ap.add_argument("--rate", type=float, default=8.0, help="serve: request arrivals per second")
    ap.add_argument("--requests", type=int, default=64, help="serve: number of requests")
    ap.add_argument("--serve-requests", type=int, default=32,
                    help="default workload: requests of the serving leg (0: off)")
    ap.add_argument("--max-batch-ct", type=int, default=16, help="serve: ciphertexts per batched pass")
    ap.add_argument("--serve-lanes", type=int, default=1,
                    help="serve: contexts (same keys) whose batches run concurrently")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--profile-kernel", default="ntt")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-breakdown", action="store_true")
    ap.add_argument("--no-split", action="store_true", help="skip the split-packing (one problem per ciphertext) timing")
    ap.add_argument("--split-groups", type=int, default=16, help="split packing: problems per grouped pass")
    ap.add_argument("--latency-repeats", type=int, default=50, help="single-ciphertext latency repeats (0: off)")
    ap.add_argument("--method", default="alg4", choices=sorted(METHODS), help="Softmax circuit")
    ap.add_argument("--no-other", action="store_true", help="skip timing the other method")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch strategies")
    ap.add_argument("--precision-seeds", type=int, default=5, help="seeds per input recipe of the precision sweep")
    args = ap.parse_args()
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "llama":
        return run_llama(args)
    wl = workload(args.workload)
    if args.impl == "reference":
        return run_reference(args, wl)

    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2410_11184_gb300 import he, shard

    chains, plans, evalmod = he.load_params()
    ch, em = chains["fgb16"], evalmod["fgb16"]
    pl = load_plan(he, args.method)
    other = "alg2" if args.method == "alg4" else "alg4"
    pl_other = load_plan(he, other)
    stream = torch.cuda.Stream(dev)
    g = he.Context(ch, em, stream=stream, device=dev)
    m, n = wl["m"], wl["n"]
    L = m * g.n0 // n
    M = pl["M"]
    seeds = shard.replica_seeds(rank)   # independent replica per rank (weak scaling)
    g.keygen(seeds["key"])
    g.keygen_softmax(n, m)
    # autotuner: launch strategies timed on the device for every level of the chain and the two
    # batch sizes the circuit runs (the auxiliary ciphertext and the m main-thread ones)
    tune = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        g.autotune(list(range(1, len(ch["q"]))), sorted({1, m}), reps=2)
        table = g.tune_table()
        tune = {"seconds": round(time.perf_counter() - t0, 2), "entries": len(table),
                "keys": "(op, limbs, n_ct) for levels 1..%d and n_ct in %s" % (len(ch["q"]) - 1, sorted({1, m})),
                "non_default": [e for e in table if e["op"] not in ("ntt_small", "ntt_1pass")
                                and e["choice"] != ((0 if e["op"] == "fuse_conv" else 1) if e["n_ct"] <= 4 else 0)],
                "ntt_small_cta_at_limbs": {d: [e["limbs"] for e in table if e["op"] == "ntt_small"
                                               and e["n_ct"] == i and e["choice"] == 1]
                                           for i, d in enumerate(("forward", "inverse"))},
                "ntt_small_cta_ms": {"%s_%d" % ("fwd" if e["n_ct"] == 0 else "inv", e["limbs"]): e["ms"]
                                     for e in table if e["op"] == "ntt_small"},
                # one launch per limb cluster (distributed shared memory) against the two passes
                "ntt_1pass_at_limbs": {d: [e["limbs"] for e in table if e["op"] == "ntt_1pass"
                                           and e["n_ct"] == i and e["choice"] == 1]
                                       for i, d in enumerate(("forward", "inverse"))},
                "ntt_1pass_ms": {"%s_%d" % ("fwd" if e["n_ct"] == 0 else "inv", e["limbs"]): e["ms"]
                                 for e in table if e["op"] == "ntt_1pass"}}
    x = attention_logits(L, n, seed=seeds["inputs"])
    src = g.encrypt(x, n, m, M, seeds["encrypt"])
    work = g.like(src)

    def step(batched, graph=None, plan=None):
        # batched steps replay the circuit captured as one CUDA graph (captured in the first
        # warm-up step); plain steps run the per-ciphertext operation list eagerly
        work.tensor.copy_(src.tensor)  # (on torch's stream of `stream` below)
        work.level, work.scale, work.n_ct = src.level, src.scale, src.n_ct
        g.softmax(work, plan or pl, batched=batched, graph=batched if graph is None else graph)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def fp64_softmax(xx):
        e = np.exp(xx - xx.max(axis=1, keepdims=True))
        return e / e.sum(axis=1, keepdims=True)

    with torch.cuda.stream(stream):
        # the headline graph carries no timing events (captured in the first warm-up step)
        g.profile_kernel("")
        for _ in range(args.warmup):
            step(True)
        torch.cuda.synchronize(dev)
        # precision check of the warm-up output (FP64 Softmax of the same inputs)
        err = float(np.abs(g.decrypt(work, n) - fp64_softmax(x)).max())
        c0 = g.counters()
        l0 = g.launch_count()
        clocks = ClockSampler(local)
        clocks.start()
        barrier()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        torch.cuda.nvtx.range_push("timed")  # ncu --nvtx --nvtx-include "timed/" selects these launches
        ev[0].record(stream)
        for i in range(args.steps):
            step(True)
            ev[i + 1].record(stream)
        barrier()
        torch.cuda.nvtx.range_pop()
        clk = clocks.stop()
        per = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
        total_ms = ev[0].elapsed_time(ev[-1])
        c1 = g.counters()
        launches = g.launch_count() - l0
        ks_per_step = (c1["ks"] - c0["ks"]) // args.steps
        bts_per_step = (c1["bts"] - c0["bts"]) // args.steps
        # roofline pass: the same steps on a second buffer, whose graph carries CUDA events around
        # every launch of the profiled kernel family (the events cost time, so the headline above
        # is taken without them)
        work2 = g.like(src)

        def step_prof():
            work2.tensor.copy_(src.tensor)
            work2.level, work2.scale, work2.n_ct = src.level, src.scale, src.n_ct
            g.softmax(work2, pl, graph=True)

        # with branches on side streams, events around a launch would also time the kernels that
        # overlap it: the roofline graph runs every launch on one stream
        g.tune_force("branches", 0)
        g.profile_kernel(args.profile_kernel)
        step_prof()   # eager run + capture with the events inside
        step_prof()
        barrier()
        g.profile_read()  # drop the capture-time timings
        evp = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        evp[0].record(stream)
        for _ in range(args.steps):
            step_prof()
        evp[1].record(stream)
        barrier()
        prof_ms_step = evp[0].elapsed_time(evp[1]) / args.steps
        k_ms, k_launch, k_bytes = g.profile_read()   # the last replay's events
        g.profile_kernel("")
        g.tune_force("branches", -1)
        del work2
        # plain mode: the same operation list one ciphertext at a time
        plain_ms = None
        if not args.no_plain:
            t = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            step(False)  # warm-up of the per-ciphertext path
            barrier()
            t[0].record(stream)
            step(False)
            t[1].record(stream)
            barrier()
            plain_ms = t[0].elapsed_time(t[1])
        # per-family and per-phase breakdown of one more (untimed) step: CUDA events around every launch
        breakdown, phases = None, None
        if not args.no_breakdown:
            g.tune_force("branches", 0)   # one stream: the per-launch times add up to the step
            g.profile_kernel("all")
            step(True, graph=False)
            g.tune_force("branches", -1)
            breakdown, phases = {}, {}
            phase_family = {}
            for fam, (nl, ms, b) in g.profile_breakdown().items():
                if fam.startswith("pf:"):
                    _, ph, fm = fam.split(":", 2)
                    phase_family.setdefault(ph, {})[fm] = round(ms, 2)
                    continue
                if fam.startswith("phase:"):
                    phases[fam[6:]] = {"launches": nl, "ms": round(ms, 3)}
                    if fam.startswith("phase:bootstrap."):   # the sum of the bootstrapping's steps
                        tot = phases.setdefault("bootstrap", {"launches": 0, "ms": 0.0})
                        tot["launches"] += nl
                        tot["ms"] = round(tot["ms"] + ms, 3)
                    continue
                breakdown[fam] = {"launches": nl, "ms": round(ms, 3), "bytes": b}
                if b > 0 and ms > 0:
                    breakdown[fam]["gbs"] = round(b / (ms * 1e-3) / 1e9, 1)
            g.profile_kernel("")
        # the other method on the same batch: graph replays, one timed step
        other_line = None
        if not args.no_other:
            step(True, plan=pl_other)
            step(True, plan=pl_other)
            barrier()
            to = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            co0 = g.counters()
            to[0].record(stream)
            step(True, plan=pl_other)
            to[1].record(stream)
            barrier()
            co1 = g.counters()
            eo = float(np.abs(g.decrypt(work, n) - fp64_softmax(x)).max())
            other_line = {"method": METHODS[other][1], "ms_per_softmax": to[0].elapsed_time(to[1]) / L,
                          "precision_bits_vs_fp64": bits(eo), "key_switches_per_step": co1["ks"] - co0["ks"],
                          "bootstrappings_per_step": co1["bts"] - co0["bts"]}
        # e2e: pinned host ciphertexts in, results out, through he_softmax (every timed step)
        host_in = torch.empty_like(src.tensor, device="cpu").pin_memory()
        host_in.copy_(src.tensor)
        host_out = torch.empty_like(src.tensor, device="cpu").pin_memory()
        barrier()
        te = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        te[0].record(stream)
        out_words = 0
        for _ in range(args.steps):
            work.tensor.copy_(host_in, non_blocking=True)
            work.level, work.scale, work.n_ct = src.level, src.scale, src.n_ct
            g.softmax(work, pl, batched=True, graph=True)
            out_words = work.n_ct * 2 * (work.level + 1) * g.n
            host_out[:out_words].copy_(work.tensor[:out_words], non_blocking=True)
        te[1].record(stream)
        barrier()
        e2e_ms = te[0].elapsed_time(te[1]) / args.steps
        # e2e from FP64 inputs to FP64 outputs in host memory: he_encrypt, he_softmax, he_decrypt
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            g.encrypt(x, n, m, M, seeds["encrypt"], out=work)
            g.softmax(work, pl, batched=True, graph=True)
            y_host = g.decrypt(work, n)
        barrier()
        xy_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        # precision over seeds 0-4 and the three input recipes (graph replays on the same buffer)
        prec_runs, prec_err = [], {}
        for sd in range(args.precision_seeds):
            for rname, xx in recipes(L, n, 100 + sd, M).items():
                g.encrypt(xx, n, m, M, 500 + sd, out=work)
                g.softmax(work, pl, batched=True, graph=True)
                yy = g.decrypt(work, n)
                prec_err.setdefault(rname, []).append(float(np.abs(yy - fp64_softmax(xx)).max()))
                prec_runs.append((xx, yy))
        # latency of one Softmax call on a single ciphertext (128 Softmax of dim 256): graph
        # replays, each timed with CUDA events (p50 / p99 over the repeats)
        lat1 = None
        if args.latency_repeats > 0 or not args.no_split:
            g.keygen_softmax(n, 1)
        if args.latency_repeats > 0:
            x1 = attention_logits(g.n0 // n, n, seed=seeds["inputs"] + 1000)
            src1 = g.encrypt(x1, n, 1, M, seeds["encrypt"] + 1000)
            work1 = g.like(src1)

            def one():
                work1.tensor.copy_(src1.tensor)
                work1.level, work1.scale, work1.n_ct = src1.level, src1.scale, src1.n_ct
                g.softmax(work1, pl, graph=True)

            for _ in range(3):
                one()
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.latency_repeats)]
            for i in range(args.latency_repeats):
                evs[2 * i].record(stream)
                one()
                evs[2 * i + 1].record(stream)
            torch.cuda.synchronize(dev)
            ts = sorted(evs[2 * i].elapsed_time(evs[2 * i + 1]) for i in range(args.latency_repeats))
            lat1 = {"workload": "1 ciphertext, 128 Softmax of dim 256", "repeats": args.latency_repeats,
                    "p50_ms": ts[len(ts) // 2], "p99_ms": ts[min(len(ts) - 1, -(-99 * len(ts) // 100) - 1)],
                    "max_ms": ts[-1]}

        # the paper's split packing (Sec. 4.2, first paragraph of the many-ciphertext case): the
        # same L Softmax as m independent one-ciphertext problems of N0/n Softmax, each with its
        # own auxiliary thread (log n rotations per round instead of log(n/m)); timed as one
        # grouped batched pass (he_softmax_grouped, m groups of one ciphertext)
        split = None
        if not args.no_split:
            # passes of at most --split-groups problems: every problem carries its own auxiliary
            # ciphertext and bootstrappings, so one pass over all m would hold m of each at once
            rows = g.n0 // n
            gp = max(1, min(m, args.split_groups))
            try:
                torch.cuda.empty_cache()
                passes = []
                for p0 in range(0, m, gp):
                    parts = [g.encrypt(x[i * rows:(i + 1) * rows], n, 1, M, seeds["encrypt"] + 2000 + i)
                             for i in range(p0, min(m, p0 + gp))]
                    ssrc = he.Ciphertexts(g, torch.cat([p_.tensor for p_ in parts]), parts[0].level, parts[0].scale,
                                          len(parts))
                    passes.append((p0, ssrc, g.like(ssrc)))
                    del parts

                def split_step():
                    for _, ssrc, swork in passes:
                        swork.tensor.copy_(ssrc.tensor)
                        swork.level, swork.scale, swork.n_ct = ssrc.level, ssrc.scale, ssrc.n_ct
                        g.softmax_grouped(swork, pl, ssrc.n_ct)

                split_step()
                barrier()
                ts_ = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                ts_[0].record(stream)
                split_step()
                ts_[1].record(stream)
                barrier()
                serr = 0.0
                for p0, _, swork in passes:
                    w1 = 2 * (swork.level + 1) * g.n
                    for i in range(swork.n_ct):
                        one_ct = he.Ciphertexts(g, swork.tensor[i * w1:(i + 1) * w1], swork.level, swork.scale, 1)
                        yi = g.decrypt(one_ct, n)
                        xi = x[(p0 + i) * rows:(p0 + i + 1) * rows]
                        serr = max(serr, float(np.abs(yi - fp64_softmax(xi)).max()))
                split = {"workload": "%d one-ciphertext problems of %d Softmax (split packing)" % (m, rows),
                         "grouped_passes": len(passes), "problems_per_pass": gp,
                         "grouped_ms_per_softmax": ts_[0].elapsed_time(ts_[1]) / L,
                         "precision_bits_vs_fp64": bits(serr)}
                if lat1:
                    # one problem at a time: the single-ciphertext latency times m, per Softmax
                    split["sequential_ms_per_softmax"] = lat1["p50_ms"] * m / L
            except Exception as e:   # a side measurement: report it, keep the line
                split = {"error": ("%s: %s" % (type(e).__name__, e))[:200]}
            passes = None
            torch.cuda.synchronize(dev)
            torch.cuda.empty_cache()

    # serving (config 5's request loop, a short run): its own context beside this one
    serving = None
    if world == 1 and args.serve_requests > 0:
        try:
            sl = serve_measure(args, args.serve_requests, args.rate)
            serving = {k: sl[k] for k in ("p50_ms", "p99_ms", "max_ms", "softmax_per_s", "requests", "span_s",
                                          "arrival_rate_per_s", "batches", "mean_batch_requests", "lanes",
                                          "precision_bits_by_n")}
            serving["workload"] = sl["config"]["workload"]
        except Exception as e:   # a side measurement: report it, keep the line
            serving = {"error": ("%s: %s" % (type(e).__name__, e))[:200]}

    ms_step, e2e_ms, xy_ms = shard.max_over_ranks([total_ms / args.steps, e2e_ms, xy_ms], dist)
    if rank != 0:
        return
    value = ms_step / (L * world)   # each rank processes L Softmax; value is whole-job (weak scaling)
    hbm, peak_kind = peaks()
    roof = None
    if k_launch:
        gbs = (k_bytes / k_launch) / ((k_ms / k_launch) * 1e-3) / 1e9
        traffic = None
        hbm_view = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                    "peak_kind": peak_kind, "algorithmic_bytes": "16 N per limb (read + write)"}
        roof = dict(hbm_view, kernel=args.profile_kernel, traffic=traffic)
        if args.profile_kernel == "ntt" and breakdown:
            # limbs per direction from the eager breakdown (16 N algorithmic bytes per limb)
            lb = 16.0 * g.n
            fwd = sum(v["bytes"] for k, v in breakdown.items() if k.startswith("ntt") and not k.endswith("_inv")) / lb
            inv = sum(v["bytes"] for k, v in breakdown.items() if k.startswith("ntt") and k.endswith("_inv")) / lb
            per_limb = (fwd * NTT_WARP_INSTR_PER_LIMB["fwd"] + inv * NTT_WARP_INSTR_PER_LIMB["inv"]) / (fwd + inv)
            dram_limb = (fwd * NTT_DRAM_PER_LIMB["fwd"] + inv * NTT_DRAM_PER_LIMB["inv"]) / (fwd + inv)
            limbs = k_bytes / lb   # the timed replay's limbs
            traffic = dram_limb * limbs / k_launch   # DRAM bytes per launch
            ach = limbs * per_limb / (k_ms * 1e-3) / 1e9
            roof = {"bound": "alu", "kernel": "ntt", "achieved": ach, "peak": ISSUE_PEAK_G,
                    "unit": "G warp instructions/s", "frac": ach / ISSUE_PEAK_G, "traffic": traffic,
                    "peak_kind": "derived: 152 SMs x 4 schedulers x 1 warp instruction/cycle x 2070 MHz",
                    "work": "warp instructions per limb from ncu (forward %.0f, inverse %.0f), %.0f%% forward limbs"
                            % (NTT_WARP_INSTR_PER_LIMB["fwd"], NTT_WARP_INSTR_PER_LIMB["inv"],
                               100 * fwd / (fwd + inv)),
                    "hbm_view": hbm_view, "int_pipes": NTT_INT_PIPES}
        roof.update({"launches_per_step": k_launch, "kernel_ms_per_step": k_ms,
                     "share_of_step": k_ms / prof_ms_step, "profiled_ms_per_step": prof_ms_step,
                     "timed": "CUDA events inside a second captured graph of the same step, its last replay of %d"
                              % args.steps})
    all_err = [e for v in prec_err.values() for e in v]
    precision = {"gate_bits": 15, "vs": "FP64 Softmax, max |error| per run",
                 "seeds": list(range(100, 100 + args.precision_seeds)), "total": stats_bits(all_err),
                 "by_recipe": {k: stats_bits(v) for k, v in prec_err.items()},
                 "all_runs_pass_gate": all(e < 2 ** -15 for e in all_err)}
    line = {
        "metric": METRIC, "value": value, "unit": "ms/Softmax", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64 (RNS residues mod 42-60-bit primes)", "data": "synthetic",
        "config": {"workload": wl["workload"], "n": n, "m": m, "softmax_per_step": L * world, "M": M,
                   "k": pl["k"], "method": METHODS[args.method][1], "log_qp": round(ch["log_qp"], 2), "h": ch["h"],
                   "l2": "inputs 1.7 GB + evaluation keys > 12 GB per step, larger than L2 (no flush)"},
        "p50_ms_per_step": statistics.median(per), "p99_ms_per_step": max(per),
        "plain_ms_per_softmax": (plain_ms / L) if plain_ms else None,
        "batched_speedup_vs_plain": (plain_ms / ms_step) if plain_ms else None,
        "precision_bits_vs_fp64": bits(err),
        "precision": precision,
        "key_switches_per_step": ks_per_step,
        "bootstrappings_per_step": bts_per_step,
        "gpu_launches": launches,
        "clocks": clk,
        "roofline": roof,
        "breakdown_one_step": breakdown,
        "phase_ms_one_step": phases,
        "phase_family_ms_one_step": phase_family if not args.no_breakdown else None,
        "other_method": other_line,
        "autotune": tune,
        "single_ct_latency": lat1,
        "split_packing": split,
        "serving": serving,
        "e2e": {"value": e2e_ms / L, "unit": "ms/Softmax", "h2d_bytes_per_step": src.tensor.numel() * 8,
                "d2h_bytes_per_step": out_words * 8,
                "path": "pinned host ciphertexts -> he_softmax_graph -> host ciphertexts, every timed step"},
        "e2e_x_to_y": {"value": xy_ms / L, "unit": "ms/Softmax", "h2d_bytes_per_step": x.size * 8,
                       "d2h_bytes_per_step": y_host.size * 8,
                       "path": "host FP64 x -> he_encrypt -> he_softmax_graph -> he_decrypt -> host FP64 y, "
                               "every timed step (host wall clock)"},
    }
    if not args.no_cpu and world == 1:
        line["cpu_baseline"] = cpu_baseline(ks_per_step, 1.0 / L)
        line["cpu_baseline"]["full_toy_softmax"] = cpu_full_toy_softmax()
        split_err = cpu_simulation(prec_runs, pl)
        precision["approx"] = stats_bits([a for a, _ in split_err])
        precision["noise"] = stats_bits([b for _, b in split_err])
        precision["split"] = "approx: oracle FP64 simulation of the circuit vs FP64 Softmax; noise: decryption vs that simulation"
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
