"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds no arithmetic of the CTMRG method: it only draws random iPEPS
tensors, builds the two-site bond operators of the spin-1/2 Heisenberg model and
assembles exactly solvable "decoupled cluster" iPEPS from a small state vector.
Both the oracle (``oracle/``) and the GPU path (tests, ``bench.py``) take their
inputs from here, so the two sides see byte-identical float64 arrays.

Tensor layout (one site): ``A[s, u, l, d, r]`` with physical index ``s`` (size p)
and virtual legs up, left, down, right (size D each).  A unit cell is stored as
``A_cell[x, y, s, u, l, d, r]`` with x the row and y the column.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "random_cell", "neel_biased_cell", "config", "WORKLOADS",
    "pauli", "heisenberg_bond", "heisenberg_bond_rotated", "honeycomb_bond",
    "product_state_cell", "plaquette_cell", "dimer_cell", "dimer_pairs_cell",
    "gauge_transform_cell", "rotate_cell_90",
]


# ---------------------------------------------------------------- random iPEPS
def random_cell(Lx: int, Ly: int, p: int, D: int, seed: int = 0) -> np.ndarray:
    """Unit cell of i.i.d. N(0,1) tensors, each divided by its own max |entry|.

    Site (x, y) draws from ``np.random.default_rng(seed + x*Ly + y)`` (PCG64).
    """
    out = np.empty((Lx, Ly, p, D, D, D, D), dtype=np.float64)
    for x in range(Lx):
        for y in range(Ly):
            rng = np.random.default_rng(seed + x * Ly + y)
            a = rng.standard_normal((p, D, D, D, D))
            out[x, y] = a / np.abs(a).max()
    return out


def neel_biased_cell(p: int, D: int, seed: int = 0, bias: float = 0.5) -> np.ndarray:
    """2x2 cell of N(0,1) tensors plus a Neel-ordered product-state component.

    ``A += bias * e_sigma (x) e0 (x) e0 (x) e0 (x) e0`` with sigma = up (s=0) on
    (0,0),(1,1) and down (s=1) on (0,1),(1,0); each tensor is then divided by its
    max |entry|.
    """
    A = random_cell(2, 2, p, D, seed)
    for x in range(2):
        for y in range(2):
            s = 0 if (x + y) % 2 == 0 else 1
            A[x, y, s, 0, 0, 0, 0] += bias
            A[x, y] /= np.abs(A[x, y]).max()
    return A


# Workloads, named by bond dimension, environment dimension, unit cell and model:
# cell Lx x Ly, physical dimension p, D, chi, J2 / J1 of the diagonal bonds,
# rotated (sublattice-rotated bond operator of 1-site cells), neel (Neel bias)
WORKLOADS = {
    "d2_chi16_1x1": dict(Lx=1, Ly=1, p=2, D=2, chi=16, J2=0.0, rotated=True, sweeps=30),
    "d4_chi32_2x2": dict(Lx=2, Ly=2, p=2, D=4, chi=32, J2=0.0, rotated=False, sweeps=30),
    "d6_chi72_2x2": dict(Lx=2, Ly=2, p=2, D=6, chi=72, J2=0.0, rotated=False, sweeps=20, bench_precision=4),
    "d8_chi128_2x2_j1j2": dict(Lx=2, Ly=2, p=2, D=8, chi=128, J2=0.5, rotated=False, sweeps=10,
                               bench_precision=4, neel=True),
    "d10_chi200_1x1": dict(Lx=1, Ly=1, p=2, D=10, chi=200, J2=0.0, rotated=True, sweeps=10, bench_precision=4),
}


def config(name: str):
    """Return (A_cell, params) for a named workload; inputs are seeded (seed 0)."""
    c = dict(WORKLOADS[name])
    if c.get("neel"):
        A = neel_biased_cell(c["p"], c["D"], seed=0)
    else:
        A = random_cell(c["Lx"], c["Ly"], c["p"], c["D"], seed=0)
    return A, c


# --------------------------------------------------------------- bond operators
def pauli():
    """(I, X, iY, Z) for spin 1/2 as real 2x2 float64 matrices (iY = [[0,1],[-1,0]])."""
    I = np.eye(2)
    X = np.array([[0.0, 1.0], [1.0, 0.0]])
    iY = np.array([[0.0, 1.0], [-1.0, 0.0]])
    Z = np.array([[1.0, 0.0], [0.0, -1.0]])
    return I, X, iY, Z


def heisenberg_bond(J: float = 1.0) -> np.ndarray:
    """J * S_i . S_j as a real (4, 4) matrix, rows (t_i, t_j), cols (s_i, s_j).

    sigma^y (x) sigma^y = -(iY) (x) (iY) is real.
    """
    _, X, iY, Z = pauli()
    h = 0.25 * (np.kron(X, X) - np.kron(iY, iY) + np.kron(Z, Z))
    return J * h


def heisenberg_bond_rotated(J: float = 1.0) -> np.ndarray:
    """Heisenberg bond after a pi rotation about y on one sublattice.

    sigma^x -> -sigma^x, sigma^z -> -sigma^z on one site of the bond, so
    h = J/4 (-XX + YY - ZZ); it lets a one-site cell describe Neel order.
    """
    _, X, iY, Z = pauli()
    h = 0.25 * (-np.kron(X, X) - np.kron(iY, iY) - np.kron(Z, Z))
    return J * h


def honeycomb_bond(J: float = 1.0) -> np.ndarray:
    """Bond operator of the honeycomb Heisenberg model coarse-grained to the
    square lattice: every square-lattice site holds the two spins A and B of one
    honeycomb bond (physical dimension p = 4, index 2 a + b for spins a of A and
    b of B), and the other two honeycomb bonds of each spin connect B of a site
    to A of its right neighbour and to A of the neighbour below.  Both square
    bonds are then h = J S_B(first) . S_A(second), first = left or top site.  The
    intra-site term J S_A . S_B is shared out over the four bonds of each site,
    a quarter per bond end, so that the one-operator 2x2-patch energy gives
    <S_A.S_B> + <horizontal> + <vertical> per square site.  Real 16 x 16 matrix,
    rows (t_1, t_2), cols (s_1, s_2) as for ``heisenberg_bond``.
    """
    I2, X, iY, Z = pauli()
    I4 = np.eye(4)
    A_ops = [np.kron(X, I2), np.kron(iY, I2), np.kron(Z, I2)]    # spin A of a site (times 2)
    B_ops = [np.kron(I2, X), np.kron(I2, iY), np.kron(I2, Z)]    # spin B of a site (times 2)
    sign = [1.0, -1.0, 1.0]                                      # sigma^y sigma^y = -(iY)(iY)
    inter = 0.25 * sum(sg * np.kron(b, a) for sg, b, a in zip(sign, B_ops, A_ops))
    intra = 0.25 * sum(sg * a @ b for sg, a, b in zip(sign, A_ops, B_ops))   # S_A . S_B on one site
    return J * (inter + 0.25 * (np.kron(intra, I4) + np.kron(I4, intra)))


# ------------------------------------------------- exactly solvable test states
def product_state_cell(phis: np.ndarray, D: int = 1) -> np.ndarray:
    """Product state: A[x,y][s,0,0,0,0] = phi[x,y][s], zero-padded to bond dim D."""
    phis = np.asarray(phis, dtype=np.float64)
    Lx, Ly, p = phis.shape
    A = np.zeros((Lx, Ly, p, D, D, D, D))
    A[:, :, :, 0, 0, 0, 0] = phis
    return A


def plaquette_cell(psi: np.ndarray, D: int = 4) -> np.ndarray:
    """2x2 cell whose iPEPS is a product of identical 4-site plaquette states.

    ``psi[s00, s01, s10, s11]`` (spin 1/2) is the plaquette wavefunction.  Site
    (0,0) copies its spin to the right, (0,1) forwards (s00, s01) downwards as a
    4-valued index, (1,0) copies its spin to the right and (1,1) holds psi.  All
    bonds leaving the unit cell carry index 0 only, so the state factorises.
    Needs D >= 4.
    """
    assert D >= 4
    A = np.zeros((2, 2, 2, D, D, D, D))
    for s in range(2):
        A[0, 0, s, 0, 0, 0, s] = 1.0                    # r = s00
        A[1, 0, s, 0, 0, 0, s] = 1.0                    # r = s10
        for l in range(2):
            A[0, 1, s, 0, l, 2 * l + s, 0] = 1.0        # d = (s00, s01)
    for a in range(2):
        for b in range(2):
            for c in range(2):
                for s in range(2):
                    A[1, 1, s, 2 * a + b, c, 0, 0] = psi[a, b, c, s]
    return A


def dimer_cell(D: int = 2) -> np.ndarray:
    """2x2 cell: singlets on the horizontal bonds (x,0)-(x,1), nothing else."""
    A = np.zeros((2, 2, 2, D, D, D, D))
    for x in range(2):
        for s in range(2):
            A[x, 0, s, 0, 0, 0, s] = 1.0
            # amplitude of (s_left, s_right): (0,1) -> +1, (1,0) -> -1
            A[x, 1, s, 0, 1 - s, 0, 0] = 1.0 if s == 1 else -1.0
    return A


def dimer_pairs_cell(psis: np.ndarray, D: int = 2, vertical: bool = False) -> np.ndarray:
    """2x2 cell of generic two-site states on the bonds (x,0)-(x,1) (or (0,y)-(1,y)).

    ``psis[k]`` is a (p,p) amplitude matrix psi[s_first, s_second] for row k
    (column k when vertical).  The first site copies its state along the bond,
    the second holds psi; all other bonds carry index 0 only.  Needs D >= p.
    """
    p = np.asarray(psis).shape[1]
    assert D >= p
    A = np.zeros((2, 2, p, D, D, D, D))
    for k in range(2):
        for s in range(p):
            if not vertical:
                A[k, 0, s, 0, 0, 0, s] = 1.0
                for a in range(p):
                    A[k, 1, s, 0, a, 0, 0] = psis[k][a, s]
            else:
                A[0, k, s, 0, 0, s, 0] = 1.0
                for a in range(p):
                    A[1, k, s, a, 0, 0, 0] = psis[k][a, s]
    return A


def gauge_transform_cell(A: np.ndarray, seed: int = 1, scale: float = 0.3) -> np.ndarray:
    """Insert G G^{-1} on every virtual bond of the cell (G = 1 + scale*N(0,1)).

    The physical state is unchanged, so every expectation value is unchanged.
    Horizontal bond right of (x,y) gets G_h[x,y]; vertical bond below (x,y) gets G_v[x,y].
    """
    Lx, Ly, p, D = A.shape[0], A.shape[1], A.shape[2], A.shape[3]
    rng = np.random.default_rng(seed)
    Gh = np.eye(D) + scale * rng.standard_normal((Lx, Ly, D, D))
    Gv = np.eye(D) + scale * rng.standard_normal((Lx, Ly, D, D))
    out = A.copy()
    for x in range(Lx):
        for y in range(Ly):
            out[x, y] = np.einsum("suldr,rk->suldk", out[x, y], Gh[x, y])
            out[x, y] = np.einsum("suldr,dk->sulkr", out[x, y], Gv[x, y])
    for x in range(Lx):
        for y in range(Ly):
            yl = (y - 1) % Ly
            xu = (x - 1) % Lx
            out[x, y] = np.einsum("kl,suldr->sukdr", np.linalg.inv(Gh[x, yl]), out[x, y])
            out[x, y] = np.einsum("ku,suldr->skldr", np.linalg.inv(Gv[xu, y]), out[x, y])
    return out


def rotate_cell_90(A: np.ndarray) -> np.ndarray:
    """Rotate the lattice clockwise by 90 degrees: site (x,y) -> (y, Lx-1-x),
    legs left->up, down->left, right->down, up->right."""
    Lx, Ly = A.shape[:2]
    out = np.empty((Ly, Lx) + A.shape[2:], dtype=A.dtype)
    for x in range(Lx):
        for y in range(Ly):
            # new[s,u,l,d,r] = old[s, l, d, r, u]
            out[y, Lx - 1 - x] = np.transpose(A[x, y], (0, 2, 3, 4, 1))
    return out
