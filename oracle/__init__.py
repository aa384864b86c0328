"""FP64 CPU oracle for the spectral-clustering hot path (test infrastructure only).

This package is the plain, slow, obviously-correct reference that the CUDA library is
checked against.  It is imported only by the tests, by the smoke check and by the
benchmark's CPU-baseline leg; the library never calls it and it never calls the library.
Every function cites the passage of Zhuzhunashvili & Knyazev, "Preconditioned Spectral
Clustering for Stochastic Block Partition Streaming Graph Challenge" (HPEC 2017) it
follows; LOBPCG itself is Knyazev's (SIAM J. Sci. Comput. 2001), which the paper calls
through SciPy (Sec. II.B).
"""
from .spectral import (  # noqa: F401
    BreakdownError,
    LobpcgResult,
    cholqr,
    cholqr_drop,
    cpqr_assign,
    cpqr_pivots,
    eigengap_k,
    embed_rows,
    kmeans,
    kmeanspp_seed,
    lambda_max,
    lap_apply,
    laplacian_csr,
    laplacian_dense,
    lloyd,
    lobpcg,
    lobpcg_blocks,
    partition,
    partition_metrics,
    rayleigh_ritz,
    sin_theta,
)
