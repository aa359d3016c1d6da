"""Contraction primitive (sctm_einsum) against numpy einsum in FP64.

Covers the FP64 CUDA-core kernel, the 3xTF32 tcgen05 tensor-core kernel
(precision 1), the FP32 CUDA-core kernel (precision 2) and the BF16-slice
tcgen05 kernel (precision 4): ragged shapes that
span several 128 x 128 tiles and 32-wide K slabs, permuted (strided) operands,
batches, beta accumulation, and sampled entries of a full-size 8192^3 product
(the size of the enlarged-corner products of the 2x2 energy at D=8, chi=128).

Tolerance of the mixed forms: every product is formed from TF32 hi/lo pairs
(relative error 2^-22 per product) and summed in FP32, so |C - C_ref| <=
1e-6 * (|A| |B|)_ij bounds every entry; the RMS error must also stay below
1e-6 of the RMS result, which fails if partial sums are carried in FP32 over
the whole K range (errors near K/8 * 2^-24 of the running sum, as in a
single tensor-core accumulator).

Tolerance of the BF16-slice form (precision 4): with rows of A and columns of
B scaled to (-1, 1) by powers of two 2^eA_i, 2^eB_j, each product term carries
the dropped slice pairs and digit remainders (about 5 x 2^-32 of
2^(eA_i + eB_j)) and at most 2.3e-10 of it from the FP32 sums of the two
lowest levels; 2^(eA_i + eB_j) <= 4 max|A_i.| max|B_.j|, so
|C - C_ref| <= 2e-9 K max|A_i.| max|B_.j| bounds every entry.  Integer
operands small enough for exact level sums must come out bit-exact.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2502_10298_gb300 as S  # noqa: E402


@pytest.fixture(scope="module")
def handles():
    hs = {p: S.sctm_create(1, 1, 2, 2, 8, precision=p, workspace_bytes=8 << 30) for p in (0, 1, 2, 4)}
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
    ("mk,kn->mn", (1500, 128), (128, 700)),       # K = 128: whole rows in one pack tile
    ("km,nk->mn", (128, 1500), (700, 128)),       # the same with A m-contiguous, B k-contiguous
]


def _ref(spec, A, B):
    return np.einsum(spec, A, B)


def _bound(spec, A, B):
    return np.einsum(spec, np.abs(A), np.abs(B))


def _on_tensor_cores(spec, A, B):
    """The engine's rule: output and K wide enough for its tiles and at least
    1e8 flops; smaller contractions run on the CUDA cores (FP32 in the mixed
    precisions 1, 2 and 4)"""
    ins, out = spec.split("->")
    la, lb = ins.split(",")
    size = dict(zip(la, A.shape))
    size.update(zip(lb, B.shape))
    prod = lambda letters: int(np.prod([size[c] for c in letters])) if letters else 1
    bat = [c for c in out if c in la and c in lb]
    m = [c for c in la if c in out and c not in bat]
    n = [c for c in lb if c in out and c not in bat]
    k = [c for c in la if c in lb and c not in out]
    M, N, K, Bt = prod(m), prod(n), prod(k), prod(bat)
    return M >= 64 and N >= 64 and K >= 128 and 2.0 * Bt * M * N * K >= 1e8


def _slice_bound(spec, A, B):
    """2e-9 K max|A_i.| max|B_.j| per output entry: the maxima run over the
    contracted letters, the outer product over the others"""
    ins, out = spec.split("->")
    la, lb = ins.split(",")
    kl = [c for c in la if c in lb and c not in out]
    K = int(np.prod([A.shape[la.index(c)] for c in kl]))
    ma = np.abs(A).max(axis=tuple(la.index(c) for c in kl))
    mb = np.abs(B).max(axis=tuple(lb.index(c) for c in kl))
    ra = "".join(c for c in la if c not in kl)
    rb = "".join(c for c in lb if c not in kl)
    return 2e-9 * K * np.einsum(f"{ra},{rb}->{out}", ma, mb)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("prec", [0, 1, 2, 4])
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
    elif prec == 4 and _on_tensor_cores(spec, A, B):
        err = np.abs(got - ref)
        assert np.all(err <= _slice_bound(spec, A, B)), err.max()
    else:
        err = np.abs(got - ref)
        assert np.all(err <= 1e-6 * _bound(spec, A, B) + 1e-300), err.max()
        # accumulation quality: the RMS error stays near FP32 rounding of the result
        assert np.sqrt(np.mean(err ** 2)) <= 1e-6 * np.sqrt(np.mean(ref ** 2))


@pytest.mark.parametrize("prec", [0, 1, 2, 4])
def test_einsum_beta_accumulates(handles, prec):
    rng = np.random.default_rng(7)
    K = 1300 if prec == 4 else 640          # precision 4: enough work for the slice kernel
    A = rng.standard_normal((300, K))
    B = rng.standard_normal((K, 260))
    C0 = rng.standard_normal((300, 260))
    C = torch.tensor(C0, device="cuda")
    S.sctm_einsum(handles[prec], "mk,kn->mn", torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), C,
                  alpha=-0.5, beta=2.0)
    ref = -0.5 * A @ B + 2.0 * C0
    if prec == 4:
        assert _on_tensor_cores("mk,kn->mn", A, B)
        bound = 0.5 * _slice_bound("mk,kn->mn", A, B) + 1e-15 * 2.0 * np.abs(C0)
        assert np.all(np.abs(C.cpu().numpy() - ref) <= bound)
        return
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


@pytest.mark.parametrize("K", [2000, 128])
def test_slices_exact_on_small_integers(handles, K):
    """Integer operands |v| <= 127 are their own leading digit: every level sum
    is an exact integer below 2^24 in each 512-wide K window, and the windows
    are added without rounding, so the product must equal the FP64 one exactly
    (K = 2000 spans four windows and the two-pass packing; K = 128 packs whole
    rows in one pass; 600 x 700 spans ragged tiles)."""
    rng = np.random.default_rng(5)
    A = rng.integers(-127, 128, (600, K)).astype(np.float64)
    B = rng.integers(-127, 128, (K, 700)).astype(np.float64)
    assert _on_tensor_cores("mk,kn->mn", A, B)
    C = S.sctm_einsum(handles[4], "mk,kn->mn", torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"))
    assert np.array_equal(C.cpu().numpy(), A @ B)


def test_slices_full_size_corner_product_sampled(handles):
    """8192^3 in BF16 slices (precision 4); 2000 entries checked in FP64 against
    the slice bound 2e-9 K max|A_.i| max|B_.j|."""
    n = 8192
    g = torch.Generator(device="cuda").manual_seed(11)
    A = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
    B = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
    C = S.sctm_einsum(handles[4], "rk,rn->kn", A, B)
    rng = np.random.default_rng(3)
    i = rng.integers(0, n, 2000)
    j = rng.integers(0, n, 2000)
    Ai = A[:, i].cpu().numpy()
    Bj = B[:, j].cpu().numpy()
    ref = np.einsum("ri,ri->i", Ai, Bj)
    got = C[i, j].cpu().numpy()
    bound = 2e-9 * n * np.abs(Ai).max(axis=0) * np.abs(Bj).max(axis=0)
    assert np.all(np.abs(got - ref) <= bound)
