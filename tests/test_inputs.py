"""The seeded input recipe shared by the oracle and the CUDA path (CPU)."""
import numpy as np

import ipeps_inputs as I


def test_random_cell_recipe():
    """Site (x, y) is N(0,1) from PCG64 seed + x*Ly + y, divided by its max |entry|."""
    A = I.random_cell(2, 3, 2, 3, seed=5)
    assert A.shape == (2, 3, 2, 3, 3, 3, 3) and A.dtype == np.float64
    for x in range(2):
        for y in range(3):
            a = np.random.default_rng(5 + x * 3 + y).standard_normal((2, 3, 3, 3, 3))
            np.testing.assert_array_equal(A[x, y], a / np.abs(a).max())
            assert np.abs(A[x, y]).max() == 1.0
    np.testing.assert_array_equal(A, I.random_cell(2, 3, 2, 3, seed=5))


def test_neel_bias_of_the_d8_workload():
    """A += 0.5 e_sigma (x) e0^4 with sigma = up on (0,0), (1,1) and down on
    (0,1), (1,0), then each site divided by its max |entry| (reading R10)."""
    A, c = I.config("d8_chi128_2x2_j1j2")
    assert (c["D"], c["chi"], c["J2"]) == (8, 128, 0.5)
    R = I.random_cell(2, 2, 2, 8, seed=0)
    for x in range(2):
        for y in range(2):
            s = 0 if (x + y) % 2 == 0 else 1
            ref = R[x, y].copy()
            ref[s, 0, 0, 0, 0] += 0.5
            np.testing.assert_array_equal(A[x, y], ref / np.abs(ref).max())


def test_bond_operators():
    """S.S has eigenvalues -3/4 (singlet) and 1/4 (triplet, three times); the
    rotated operator is the same up to a sublattice rotation."""
    for h in (I.heisenberg_bond(), I.heisenberg_bond_rotated()):
        assert np.allclose(h, h.T)
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(h)), [-0.75, 0.25, 0.25, 0.25], atol=1e-14)
