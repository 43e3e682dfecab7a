"""Small fixed workloads for Nsight Compute captures (profiles/ summaries name the command).

  python -m paper_2410_11184_gb300.profile_case softmax       # one N=2^16 Softmax of dim 256 (1 ciphertext),
                                                              # Alg. 4, inside the NVTX range "softmax"
                                                              # (a first call outside fills the caches;
                                                              # transforms in 64-thread CTAs)
  python -m paper_2410_11184_gb300.profile_case softmax_alg2  # the same by Alg. 2
  python -m paper_2410_11184_gb300.profile_case keyswitch     # 4 HMults at level 12, 64 ciphertexts
                                                              # (inside the NVTX range "hmult")
  python -m paper_2410_11184_gb300.profile_case keyswitch_small   # the same with the transforms in
                                                              # 64-thread CTAs (the autotuner's usual pick)
  python -m paper_2410_11184_gb300.profile_case keyswitch_fused   # keyswitch_small with the basis
                                                              # conversions fused into the transforms
  python -m paper_2410_11184_gb300.profile_case keyswitch_1pass   # keyswitch_small with every plain
                                                              # transform as one cluster launch per limb
"""
import sys

import numpy as np
import torch

from paper_2410_11184_gb300 import he, workloads


def main(which):
    chains, plans, evalmod = he.load_params()
    ch, em = chains["fgb16"], evalmod["fgb16"]
    pl = plans["n256_M128"] if which == "softmax_alg2" else he.load_plans_b()["n256_M128_B"]
    if not which.startswith("softmax"):
        ch = dict(ch, bootstrap=0)  # relinearisation key only: a few GB on the device
        em = None
    g = he.Context(ch, em)
    g.keygen(5)
    if which in ("keyswitch_small", "keyswitch_fused", "keyswitch_1pass", "softmax", "softmax_alg2"):
        g.tune_force("ntt_small", 1)   # the transforms' 64-thread CTAs, the autotuner's pick at almost every size
    if which == "keyswitch_fused":
        g.tune_force("fuse_conv", 1)
    if which == "keyswitch_1pass":
        g.tune_force("ntt_1pass", 1)
    if which.startswith("softmax"):
        g.keygen_softmax(256, 1)
        x = workloads.attention_logits(128, 256, 1)
        cts = g.encrypt(x, 256, 1, pl["M"], 3)
        warm = g.like(cts)
        warm.tensor.copy_(cts.tensor)
        g.softmax(warm, pl)   # first call: encodes and caches the diagonals and masks
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("softmax")  # ncu --nvtx --nvtx-include "softmax/" selects these launches
        g.softmax(cts, pl)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    else:
        m = 64
        top = ch["user_top_level"]
        rng = np.random.default_rng(0)
        q = [int(v) for v in ch["q"]]
        d = np.zeros((m, 2, top + 1, g.n), dtype=np.uint64)
        for t in range(top + 1):
            d[:, :, t] = rng.integers(0, q[t], (m, 2, g.n), dtype=np.uint64)
        a = g.from_coeff(d, top, 2.0 ** 42)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("hmult")  # ncu --nvtx --nvtx-include "hmult/" selects these launches
        for _ in range(4):
            g.hmult(a, a)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    print("done", which, "launches", g.launch_count())


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "softmax")
