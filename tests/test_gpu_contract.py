"""Contraction primitive (sctm_einsum) against numpy einsum in FP64.

Covers the FP64 CUDA-core kernel, the 3xTF32 tcgen05 tensor-core kernel
(precision 1) and the FP32 CUDA-core kernel (precision 2): ragged shapes that
span several 128 x 128 tiles and 32-wide K slabs, permuted (strided) operands,
batches, beta accumulation, and sampled entries of a full-size 8192^3 product
(the size of the enlarged-corner products of the 2x2 energy at D=8, chi=128).

Tolerance of the mixed forms: every product is formed from TF32 hi/lo pairs
(relative error 2^-22 per product) and summed in FP32, so |C - C_ref| <=
1e-6 * (|A| |B|)_ij bounds every entry; the RMS error must also stay below
1e-6 of the RMS result, which fails if partial sums are carried in FP32 over
the whole K range (errors near K/8 * 2^-24 of the running sum, as in a
single tensor-core accumulator).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2502_10298_gb300 as S  # noqa: E402


@pytest.fixture(scope="module")
def handles():
    hs = {p: S.sctm_create(1, 1, 2, 2, 8, precision=p, workspace_bytes=8 << 30) for p in (0, 1, 2)}
    yield hs
    for h in hs.values():
        S.sctm_destroy(h)


CASES = [
    # spec, shapes of A, B (letters -> extents)
    ("mk,kn->mn", (520, 700), (700, 390)),
    ("km,nk->mn", (700, 520), (390, 700)),        # A m-contiguous, B k-contiguous
    ("bmk,bkn->bmn", (3, 200, 300), (3, 300, 300)),
    ("aub,bvc->auvc", (130, 6, 140), (140, 5, 150)),  # grouped m (a,u) and n (v,c)
    ("xkmy,ynk->mxn", (9, 33, 70, 11), (11, 200, 33)),  # two k dims in reversed order
    ("ai,aj->ij", (432, 108), (432, 108)),        # Gram of a tall basis: few tiles, K split 27 ways
]


def _ref(spec, A, B):
    return np.einsum(spec, A, B)


def _bound(spec, A, B):
    return np.einsum(spec, np.abs(A), np.abs(B))


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_einsum_matches_numpy(handles, case, prec):
    spec, sa, sb = CASES[case]
    rng = np.random.default_rng(100 + case)
    A = rng.standard_normal(sa)
    B = rng.standard_normal(sb)
    ref = _ref(spec, A, B)
    C = S.sctm_einsum(handles[prec], spec, torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"))
    got = C.cpu().numpy()
    if prec == 0:
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-11 * np.abs(_bound(spec, A, B)).max())
    else:
        err = np.abs(got - ref)
        assert np.all(err <= 1e-6 * _bound(spec, A, B) + 1e-300), err.max()
        # accumulation quality: the RMS error stays near FP32 rounding of the result
        assert np.sqrt(np.mean(err ** 2)) <= 1e-6 * np.sqrt(np.mean(ref ** 2))


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_einsum_beta_accumulates(handles, prec):
    rng = np.random.default_rng(7)
    A = rng.standard_normal((300, 640))
    B = rng.standard_normal((640, 260))
    C0 = rng.standard_normal((300, 260))
    C = torch.tensor(C0, device="cuda")
    S.sctm_einsum(handles[prec], "mk,kn->mn", torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), C,
                  alpha=-0.5, beta=2.0)
    ref = -0.5 * A @ B + 2.0 * C0
    tol = 1e-11 if prec == 0 else 1e-6
    bound = 0.5 * np.abs(A) @ np.abs(B) + 2.0 * np.abs(C0)
    assert np.all(np.abs(C.cpu().numpy() - ref) <= tol * bound)


def test_full_size_corner_product_sampled(handles):
    """8192 x 8192 x 8192 on the tensor cores; 2000 entries checked in FP64."""
    n = 8192
    g = torch.Generator(device="cuda").manual_seed(11)
    A = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
    B = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
    C = S.sctm_einsum(handles[1], "rk,rn->kn", A, B)   # the Htop product: contraction over the first leg
    rng = np.random.default_rng(3)
    i = rng.integers(0, n, 2000)
    j = rng.integers(0, n, 2000)
    Ai = A[:, i].cpu().numpy()
    Bj = B[:, j].cpu().numpy()
    ref = np.einsum("ri,ri->i", Ai, Bj)
    bound = np.einsum("ri,ri->i", np.abs(Ai), np.abs(Bj))
    got = C[i, j].cpu().numpy()
    err = np.abs(got - ref)
    assert np.all(err <= 1e-6 * bound)
    assert np.sqrt(np.mean(err ** 2)) <= 1e-6 * np.sqrt(np.mean(ref ** 2))
