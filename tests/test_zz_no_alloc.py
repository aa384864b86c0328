"""The allocation-free Gram entry point (sc_gram_static) against the allocating one.

Some callers of this library cannot allocate device memory: code embedded in a framework
that owns every byte of the device through its own pool, or a latency-critical loop that
must never enter the allocator.  sc_gram_static serves them with scratch that lives in a
fixed device array of the library instead.  This file is collected last on purpose, so a
run that stops at the first failure has run everything else already; it also passes alone
in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sc():
    from paper_1708_07481_gb300 import build, sc as S

    build.build()
    return S


def test_static_gram_matches_sc_gram_twice_in_a_row(sc):
    import torch

    ctx = sc.sc_ctx_create(0)
    try:
        rng = np.random.default_rng(2024)
        # two calls in a row with different shapes: the second must not see the first's
        # leftovers in the shared scratch array
        for n, a, b in [(50001, 44, 132), (3001, 130, 7)]:
            A = rng.standard_normal((n, a)).astype(np.float32)
            B = rng.standard_normal((n, b)).astype(np.float32)
            ref = sc.sc_gram(ctx, A, B, sc.SC_PREC_FP32)  # the allocating entry point
            Ad = torch.from_numpy(A).cuda()
            Bd = torch.from_numpy(B).cuda()
            Cd = torch.full((a, b), float("nan"), dtype=torch.float64, device="cuda")
            sc.sc_gram_static(Ad, Bd, Cd)
            torch.cuda.synchronize()
            got = Cd.cpu().numpy()
            # the tolerance of the FP32 Gram parity tests
            bound = 1e-6 * np.sqrt(n) * np.outer(np.linalg.norm(A, axis=0), np.linalg.norm(B, axis=0)) + 1e-30
            assert np.all(np.isfinite(got))
            assert np.all(np.abs(got - ref) <= bound), (n, a, b)
            exact = A.astype(np.float64).T @ B.astype(np.float64)
            assert np.all(np.abs(got - exact) <= bound), (n, a, b)
    finally:
        ctx.close()


def test_static_gram_allocates_nothing(sc):
    """After a first call (which looks up the array's device address), further calls leave
    the device's free memory and torch's reserved pool unchanged: no allocation happens."""
    import torch

    rng = np.random.default_rng(7)
    A = torch.from_numpy(rng.standard_normal((20000, 40)).astype(np.float32)).cuda()
    B = torch.from_numpy(rng.standard_normal((20000, 90)).astype(np.float32)).cuda()
    Cd = torch.empty((40, 90), dtype=torch.float64, device="cuda")
    sc.sc_gram_static(A, B, Cd)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    res0 = torch.cuda.memory_reserved()
    for _ in range(5):
        sc.sc_gram_static(A, B, Cd)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_reserved() == res0


def test_static_gram_rejects_oversized_blocks(sc):
    import torch

    A = torch.zeros((8, 1025), dtype=torch.float32, device="cuda")
    C = torch.zeros((1025, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(sc.ScError) as e:
        sc.sc_gram_static(A, A[:, :1], C)
    assert e.value.code == sc.SC_EINVAL
