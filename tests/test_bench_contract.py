"""bench.py's roofline arithmetic on CPU: the algorithmic bytes and flops per launch that the
reported fractions divide by, against the per-unit figures written out by hand."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_spmm_bytes_per_launch():
    n, K, nnz = 50_000, 44, 1_995_908
    b, bound = bench.algorithmic_bytes("spmm", n, K, nnz, 3 * K)
    # row_ptr (n + 1) + col_idx (nnz) + degrees (n), int32/FP32; the 2K-column block read once
    # and its image written once, FP32
    assert bound == "hbm"
    assert b == 4 * (n + 1) + 4 * nnz + 4 * n + 2 * 4 * n * 88


def test_rayleigh_ritz_flops_per_launch():
    flops, bound = bench.algorithmic_bytes("rr_eig", 50_000, 44, 0, 132)
    assert bound == "alu"
    # (4/3) m^3 for the tridiagonalization + 2 m^2 K for the back-transformation, m = 3K
    assert flops == pytest.approx(4 / 3 * 132 ** 3 + 2 * 132 ** 2 * 44)
    assert flops == pytest.approx(4.60e6, rel=1e-3)


def test_streaming_kernels_and_unknown_names():
    n, K = 1000, 8
    assert bench.algorithmic_bytes("residual", n, K, 0, 24) == (4 * n * K * 3, "hbm")
    assert bench.algorithmic_bytes("gram", n, K, 0, 24) == (2 * 4 * n * 3 * K, "hbm")
    assert bench.algorithmic_bytes("tall_gemm", n, K, 0, 24) == (4 * n * 3 * K, "hbm")
    assert bench.algorithmic_bytes("kmeans_assign", n, K, 0, 24) == (None, None)


def test_traffic_table_covers_the_dominant_candidates():
    for k in ("rr_eig", "spmm", "tall_gemm", "chol_inv", "gram"):
        assert k in bench.NCU_TRAFFIC
        v = bench.NCU_TRAFFIC[k]
        assert v is None or (isinstance(v, int) and v > 0)
