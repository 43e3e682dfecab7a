"""Writes tests/golden/fullsize_fgb16.json: the CPU oracle's results at N = 2^16 (the fgb16
chain: log QP <= 1555, h = 192, bootstrapping) for cases too slow to recompute inside the GPU
tests, as SHA-256 hashes of every output limb (coefficient form, canonical residues in
[0, q_i), little-endian uint64) plus the output level (level_out) and scale (scale, as a hex
float).

Calls only oracle/ (and the seeded input generators, which hold none of the method's
arithmetic).  The oracle's results are the same on x86-64 and AArch64 hosts (every double
operation is one IEEE operation; the libm values it uses agree on both), so the file is valid
wherever the tests run.

    python tests/golden/make_fullsize.py [case ...]     # all cases by default; OMP threads: all cores

Cases (keys from seed 2024):
  bootstrap        one ciphertext at level 3 (uniform slots in [-1, 1], scale 2^42), gain 16
  softmax1_alg2    1 ciphertext = 128 Softmax of dim 256, plan n256_M128 (Alg. 2 + Alg. 3),
                   uniform inputs on [-128, 0]
  softmax1_alg4    the same inputs, plan n256_M128_B (Alg. 4 + Alg. 3)
  softmax64_alg2   64 ciphertexts = 8192 Softmax of dim 256 (many-ciphertext packing, Sec. 4.2),
                   attention-logit inputs, plan n256_M128
  softmax64_alg4   the same inputs, plan n256_M128_B
  softmax1_n32768_alg4   1 ciphertext = 1 Softmax of dim 32768 (the serving mix's largest
                   dimension), plan n32768_M64_B (Alg. 4 + Alg. 3), uniform inputs on [-64, 0]
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
for p in (ROOT, os.path.join(ROOT, "oracle")):
    if p not in sys.path:
        sys.path.insert(0, p)

import oracle as O  # noqa: E402
from paper_2410_11184_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "fullsize_fgb16.json")
KEY_SEED = 2024

# input recipes (shared with tests/test_gpu_fullsize.py through this file's JSON)
CASES = {
    "bootstrap": {"kind": "bootstrap", "slots_seed": 31, "level": 3, "in_scale": 2.0 ** 42, "enc_seed": 41,
                  "gain": 16.0, "out_scale": 2.0 ** 42},
    "softmax1_alg2": {"kind": "softmax", "plan": "n256_M128", "m": 1, "inputs": "uniform", "input_seed": 5,
                      "enc_seed": 99},
    "softmax1_alg4": {"kind": "softmax", "plan": "n256_M128_B", "m": 1, "inputs": "uniform", "input_seed": 5,
                      "enc_seed": 99},
    "softmax64_alg2": {"kind": "softmax", "plan": "n256_M128", "m": 64, "inputs": "attention", "input_seed": 7,
                       "enc_seed": 101},
    "softmax64_alg4": {"kind": "softmax", "plan": "n256_M128_B", "m": 64, "inputs": "attention", "input_seed": 7,
                       "enc_seed": 101},
    "softmax1_n32768_alg4": {"kind": "softmax", "plan": "n32768_M64_B", "m": 1, "inputs": "uniform",
                             "input_seed": 9, "enc_seed": 103},
}


def limb_hashes(data):
    """data [n_ct][2][L][N] or [2][L][N] uint64 -> nested lists of 16-hex-digit SHA-256 prefixes"""
    d = np.ascontiguousarray(data, dtype=np.uint64)
    if d.ndim == 3:
        d = d[None]
    return [[[hashlib.sha256(d[i, p, t].astype("<u8").tobytes()).hexdigest()[:16] for t in range(d.shape[2])]
             for p in range(2)] for i in range(d.shape[0])]


def softmax_inputs(case, n, L, M):
    if case["inputs"] == "uniform":
        return W.uniform_inputs(L, n, case["input_seed"], M)
    return W.attention_logits(L, n, case["input_seed"], M=M)


def plan_of(name):
    if name.endswith("_B"):
        return O.load_plans_b()[name]
    return O.load_params()[1][name]


def run(name, o, em):
    case = CASES[name]
    t0 = time.time()
    if case["kind"] == "bootstrap":
        rng = np.random.default_rng(case["slots_seed"])
        a = o.encrypt(rng.uniform(-1, 1, o.n0), case["level"], case["in_scale"], case["enc_seed"], 0)
        outs = [o.bootstrap(a, em, gain=case["gain"], out_scale=case["out_scale"])]
        ins = [a]
    else:
        pl = plan_of(case["plan"])
        n, m, M = pl["n"], case["m"], pl["M"]
        L = m * o.n0 // n
        x = softmax_inputs(case, n, L, M)
        top = o.chain["user_top_level"]
        slots = O.pack(x, m, o.n0)
        ins = [o.encrypt(slots[i], top, (2.0 / M) * o.q[top], case["enc_seed"], i) for i in range(m)]
        outs = o.softmax_b(ins, pl, em) if pl.get("version") == "B" else o.softmax(ins, pl, em)
        y = O.unpack(np.stack([o.decrypt(c).real for c in outs]), n)
        case = dict(case, bits_vs_fp64=float(-np.log2(np.abs(y - O.softmax_fp64(x)).max())))
    rec = dict(case, key_seed=KEY_SEED, in_hash=limb_hashes(np.stack([c.data for c in ins])),
               level_out=outs[0].level, scale=float(outs[0].scale).hex(),
               out_hash=limb_hashes(np.stack([c.data for c in outs])),
               oracle_seconds=round(time.time() - t0, 1), host_threads=int(os.environ.get("OMP_NUM_THREADS",
                                                                                        os.cpu_count())))
    return rec


def main(names):
    chains, _, evalmod = O.load_params()
    o = O.Oracle(chains["fgb16"])
    o.keygen(KEY_SEED)
    for name in names:
        rec = run(name, o, evalmod["fgb16"])
        data = {}
        if os.path.exists(OUT):
            with open(OUT) as fh:
                data = json.load(fh)
        data[name] = rec
        with open(OUT + ".tmp", "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(OUT + ".tmp", OUT)
        print(name, "%.0f s" % rec["oracle_seconds"], rec.get("bits_vs_fp64", ""), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
