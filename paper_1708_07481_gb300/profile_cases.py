"""Small, self-contained cases for kernel profiling (ncu -k / -c on one kernel).

    python -m paper_1708_07481_gb300.profile_cases rr    # 3 Rayleigh-Ritz solves, m = 132, K = 44
    python -m paper_1708_07481_gb300.profile_cases rr64  # the same in FP64 (spread over SMs)
    python -m paper_1708_07481_gb300.profile_cases lob   # 3 LOBPCG passes, DC-SBM n = 50,000, K = 44
    python -m paper_1708_07481_gb300.profile_cases big   # 2 LOBPCG passes, DC-SBM n = 300,000, K = 160
    python -m paper_1708_07481_gb300.profile_cases kmeans  # k-means, 50,000 unit rows, d = k = 44
    python -m paper_1708_07481_gb300.profile_cases tall  # tall updates n = 50,000, 132 -> 44

`rr` feeds the dense Rayleigh-Ritz solve a 132 x 132 FP64 Gram with K = 44 small and 88 large
eigenvalues (the spectrum shape of the [X R P] projection at n = 50,000, K = 44).  `lob`
exercises the Cholesky-QR factors of 44 and 88 columns.  `big` runs the SpMM, the tensor-core
Gram and the tensor-core tall update on blocks (300,000 x 480 FP32 = 576 MB) larger than L2,
while holding only a few GB of device memory.  Every case goes through the C ABI and prints
"ok <case>" when it ends.
"""
import sys

import numpy as np

from . import sc
from . import workload as W


def main(argv=None):
    mode = (argv or sys.argv[1:] or ["rr"])[0]
    ctx = sc.sc_ctx_create(0)
    if mode in ("rr", "rr64"):
        rng = np.random.default_rng(0)
        m, K = 132, 44
        ev = np.concatenate([np.sort(rng.uniform(0, 12, K)),
                             np.sort(rng.uniform(10, 200, m - K))])
        Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
        G = (Q * ev) @ Q.T
        prec = sc.SC_PREC_FP32 if mode == "rr" else sc.SC_PREC_FP64
        for _ in range(3):
            sc.sc_rr_solve(ctx, G, K, prec)
    elif mode == "lob":
        g = W.dcsbm(50000, 44, seed=0)
        Gr = sc.sc_build_laplacian(ctx, g.n, g.src, g.dst)
        sc.sc_lobpcg(ctx, Gr, 44, iters=3, seed=0, cold=1, want_X=False)
    elif mode == "big":
        import torch
        g = W.dcsbm(300000, 160, seed=0)
        Gr = sc.sc_build_laplacian(ctx, g.n, torch.from_numpy(g.src).cuda(),
                                   torch.from_numpy(g.dst).cuda())
        sc.sc_lobpcg(ctx, Gr, 160, iters=2, seed=0, cold=1, want_X=False)
    elif mode == "kmeans":
        # unit rows around 44 centres (the embedding's shape at the bench workload); the
        # assignment path follows SC_TUNE_ASSIGN (1: tensor cores, 0: CUDA cores)
        rng = np.random.default_rng(0)
        C = rng.standard_normal((44, 44))
        E = C[rng.integers(0, 44, 50000)] + 0.05 * rng.standard_normal((50000, 44))
        E = (E / np.linalg.norm(E, axis=1, keepdims=True)).astype(np.float32)
        for _ in range(2):
            sc.sc_kmeans(ctx, E, 44, iters=50, seed=5)
    elif mode == "tall":
        # the update [X R P] Y of the bench workload (n = 50,000, 3K = 132 -> K = 44): three on
        # tensor cores, then three on CUDA cores
        rng = np.random.default_rng(0)
        A = rng.standard_normal((50000, 132), dtype=np.float32)
        Wm = rng.standard_normal((132, 44), dtype=np.float32)
        for prec in (sc.SC_PREC_MIXED, sc.SC_PREC_FP32):
            for _ in range(3):
                sc.sc_tall_update(ctx, A, Wm, prec=prec)
    else:
        raise SystemExit(f"unknown case {mode!r}: rr, rr64, lob, big, kmeans or tall")
    print("ok", mode)


if __name__ == "__main__":
    main()
