"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these tests retypes an oracle formula: each compares the oracle with an
independent value -- a closed form, a brute-force state-vector computation, a
linear-algebra identity, a symmetry, or a finite difference.
"""
import numpy as np
import pytest
import torch

import ipeps_inputs as I
from oracle import ctmrg as C
from oracle import energy as En
from oracle import statevector as SV
from oracle.fixed_point import implicit_energy_grad
from oracle.svd import svd as osvd

H = I.heisenberg_bond()
HR = I.heisenberg_bond_rotated()


def E_split(A, chi, sweeps, h, hd=None):
    env = C.split_ctmrg(A, chi=chi, sweeps=sweeps)
    return float(En.energy_per_site(A, env, h, hd))


# ------------------------------------------------------- closed forms (D = 1)
@pytest.mark.parametrize("D", [1, 2])
def test_product_state_rotated_one_site_is_minus_half(D):
    """Any real product state in the sublattice-rotated frame: -1/4 per bond,
    two bonds per site -> -1/2 (Bloch vector of a real state has unit length)."""
    rng = np.random.default_rng(0)
    phi = rng.standard_normal((1, 1, 2))
    A = I.product_state_cell(phi, D=D)
    assert abs(E_split(A, chi=8, sweeps=2, h=HR) + 0.5) < 1e-12


@pytest.mark.parametrize("D", [1, 2, 3])
def test_product_state_2x2_closed_form(D):
    """Real product state, 2x2 cell, J1-J2: every bond factorises."""
    rng = np.random.default_rng(1)
    phis = rng.standard_normal((2, 2, 2))
    A = I.product_state_cell(phis, D=D)
    if D > 1:
        A = I.gauge_transform_cell(A, seed=2)
    ref = SV.product_energy(phis, H, 0.5 * H)
    assert abs(E_split(A, chi=12, sweeps=2, h=H, hd=0.5 * H) - ref) < 1e-11


def test_neel_closed_form():
    """Neel in a 2x2 cell: -1/4 per NN bond, +1/4 per diagonal -> -1/2 + J2/2."""
    phis = np.zeros((2, 2, 2))
    phis[0, 0, 0] = phis[1, 1, 0] = 1.0
    phis[0, 1, 1] = phis[1, 0, 1] = 1.0
    A = I.product_state_cell(phis, D=2)
    for J2 in (0.0, 0.5):
        E = E_split(A, chi=4, sweeps=2, h=H, hd=J2 * H)
        assert abs(E - (-0.5 + 0.5 * J2)) < 1e-12


def test_singlet_dimers():
    """Singlets on horizontal bonds: -3/4 per singlet, 0 elsewhere -> -3/8 per site."""
    A = I.dimer_cell(D=2)
    assert abs(E_split(A, chi=8, sweeps=3, h=H, hd=0.5 * H) + 0.375) < 1e-12


# ------------------------------------------------ brute-force cluster states
@pytest.mark.parametrize("vertical", [False, True])
@pytest.mark.parametrize("D", [2, 3])
def test_generic_dimer_states_exact(vertical, D):
    """Product of generic two-site states (gauge-scrambled bonds, so every leg is
    dense): CTMRG must reproduce the state-vector energy exactly."""
    rng = np.random.default_rng(10 + D + 3 * vertical)
    psis = rng.standard_normal((2, 2, 2))
    A = I.gauge_transform_cell(I.dimer_pairs_cell(psis, D=D, vertical=vertical), seed=3)
    ref = SV.dimer_pairs_energy(psis, H, 0.5 * H, vertical=vertical)
    assert abs(E_split(A, chi=16, sweeps=3, h=H, hd=0.5 * H) - ref) < 1e-10


def test_plaquette_patch_bonds_exact():
    """Product of generic 4-site plaquettes: every bond of the patch that holds a
    whole plaquette (anchor (0,0)) equals the state-vector value, including both
    diagonals; bonds between plaquettes factorise."""
    rng = np.random.default_rng(4)
    psi = rng.standard_normal((2, 2, 2, 2))
    psi /= np.linalg.norm(psi)
    A = I.gauge_transform_cell(I.plaquette_cell(psi, D=4), seed=5, scale=0.2)
    env = C.split_ctmrg(A, chi=24, sweeps=3)
    _, bonds = En.energy_per_site(A, env, H, H, return_bonds=True)
    rdm1, rdm2 = SV._cluster_state_pairs(psi)
    v = bonds[(0, 0)]
    pairs = {"top": (0, 1), "bottom": (2, 3), "left": (0, 2), "right": (1, 3),
             "diag1": (0, 3), "diag2": (1, 2)}
    for k, (i, j) in pairs.items():
        assert abs(float(v[k]) - SV._two_site_value(rdm2[(i, j)], H)) < 1e-10, k
    # patch (1,1): all four sites in different plaquettes -> products
    w = bonds[(1, 1)]
    prod = lambda i, j: SV._two_site_value(np.einsum("sT,vU->svTU", rdm1[i], rdm1[j]), H)
    assert abs(float(w["top"]) - prod(3, 2)) < 1e-10
    assert abs(float(w["left"]) - prod(3, 1)) < 1e-10
    assert abs(float(w["diag1"]) - prod(3, 0)) < 1e-10


# ------------------------------------------------------ projector identities
def _env_after(A, chi, sweeps):
    Ac = C.as_cell(A)
    return Ac, C.split_ctmrg(Ac, chi=chi, sweeps=sweeps)


@pytest.mark.parametrize("order", ["standard", "alternative"])
@pytest.mark.parametrize("chi", [6, 40])
def test_projector_identities(chi, order):
    """For every colour, in both yellow/red orders (App. B): P_up P_dn = 1 on
    the kept space, P_dn P_up idempotent, and rho^B P_dn P_up rho^T equals the
    best rank-chi approximation of M (Eckart-Young: the residual is the norm of
    the discarded singular values)."""
    A = I.random_cell(2, 2, 2, 2, seed=7)
    Ac, env = _env_after(A, chi, 1)
    rec = {}
    E, a, K, Pg, Py, Pt, Pr, E2, a2 = C.split_column_projectors(Ac, env, 0, chi, record=rec, order=order)
    alt = order == "alternative"
    rhos = {
        "green": (C.green_rhoT(E[0], a[0]), C.green_rhoB(E[1], a[1])),
        "yellow": ((C.yellow_alt_rhoT(E[0], a[0]), C.yellow_alt_rhoB(E[0], a[0])) if alt else
                   (C.yellow_rhoT(E[0], a[0]), C.yellow_rhoB(E[0], a[0]))),
        "teal": (C.teal_rhoT(E[0], a[0], K[0], E2[0], a2[0]),
                 C.teal_rhoB(E[1], a[1], K[1], E2[1], a2[1])),
        "red": ((C.red_alt_rhoT(E[0], K[0], E2[0], a2[0]), C.red_alt_rhoB(E[0], a[0], K[0], E2[0], a2[0])) if alt
                else (C.red_rhoT(E[0], K[0], E2[0], a2[0]), C.red_rhoB(E[0], a[0], K[0], E2[0], a2[0]))),
    }
    for colour, (rT, rB) in rhos.items():
        up, dn, s = rec[colour][0]
        k = up.shape[0]
        M = rB @ rT
        sv = torch.linalg.svdvals(M)
        kept = int((s > 1e-8 * s[0]).sum())
        I_k = (up @ dn)[:kept, :kept]
        # rounding error of entry (i,j) scales like eps * s_max / sqrt(s_i s_j)
        cond = float(s[0]) / torch.sqrt(s[:kept, None] * s[None, :kept])
        err = (I_k - torch.eye(kept, dtype=I_k.dtype)).abs()
        assert bool((err <= 1e-12 * cond + 1e-12).all()), colour
        # idempotence on the well-conditioned part of the kept space
        kw = int((s > 1e-6 * s[0]).sum())
        Pw = dn[:, :kw] @ up[:kw]
        assert torch.allclose(Pw @ Pw, Pw, atol=1e-9 * max(1.0, float(Pw.abs().max()))), colour
        P = dn @ up
        resid = torch.linalg.norm(rB @ P @ rT - M)
        expect = torch.sqrt((sv[k:] ** 2).sum())
        assert abs(float(resid) - float(expect)) < 1e-8 * float(sv[0]), colour


def test_split_edges_contract_to_conventional():
    """Contracting T^ket T^bra over the interlayer bond gives the conventional
    double-layer edge when the split keeps the full rank (chi >= D^3)."""
    A = C.as_cell(I.random_cell(2, 2, 2, 2, seed=9))
    split = C.fuse(C.initial_env(A, chi=64, split=True))
    conv = C.initial_env(A, chi=64, split=False)
    for x in range(2):
        for y in range(2):
            for key in ("T1", "T2", "T3", "T4"):
                assert torch.allclose(split[x][y][key], conv[x][y][key], atol=1e-12)


# ------------------------------------------------------ symmetry / agreement
def _ising_peps(beta):
    """Tensor whose squared amplitude is the classical 2D Ising weight
    exp(beta * sum_<ij> s_i s_j): A = prod over legs of Q[s, leg], Q Q^T = W."""
    W = np.exp(0.5 * beta * np.array([[1.0, -1.0], [-1.0, 1.0]]))
    w, V = np.linalg.eigh(W)
    Q = V * np.sqrt(w)
    return np.einsum("su,sl,sd,sr->suldr", Q, Q, Q, Q)[None, None]


def _onsager_nn(beta):
    """Nearest-neighbour <s_i s_j> of the square-lattice Ising model (Onsager):
    u = -coth(2b) [1 + (2/pi)(2 tanh^2(2b) - 1) K(k)], k = 2 sinh(2b)/cosh^2(2b)."""
    from scipy.special import ellipk
    k = 2 * np.sinh(2 * beta) / np.cosh(2 * beta) ** 2
    return 0.5 / np.tanh(2 * beta) * (1 + (2 / np.pi) * (2 * np.tanh(2 * beta) ** 2 - 1) * ellipk(k * k))


@pytest.mark.parametrize("split", [True, False])
def test_ising_peps_matches_onsager(split):
    """<Z_i Z_j> of the Ising PEPS equals Onsager's exact value; the tensor is
    gauge-scrambled so that no leg permutation or corner transpose can hide."""
    beta = 0.3
    A = C.as_cell(I.gauge_transform_cell(_ising_peps(beta), seed=3, scale=0.4))
    ZZ = np.kron(np.diag([1.0, -1.0]), np.diag([1.0, -1.0]))
    env = C.split_ctmrg(A, 12, 25) if split else C.conv_ctmrg(A, 12, 25)
    _, bonds = En.energy_per_site(A, env, ZZ, split=split, return_bonds=True)
    ref = _onsager_nn(beta)
    for k in ("top", "bottom", "left", "right"):
        # the 1e-8 singular-value cutoff discards weight of that order
        assert abs(float(bonds[(0, 0)][k]) - ref) < 5e-7, k


@pytest.mark.parametrize("split", [True, False])
def test_run_to_fixed_point_matches_onsager(split):
    """Iterating full steps until the normalised corner spectra stop changing
    (ctmrg_run) reaches the true fixed point: for the Ising PEPS off
    criticality the change per step decays geometrically, the run stops on its
    own, and the converged correlator is Onsager's exact value."""
    beta = 0.3
    A = C.as_cell(I.gauge_transform_cell(_ising_peps(beta), seed=3, scale=0.4))
    env, n, hist = C.ctmrg_run(A, 12, 1e-9, 60, split=split)
    assert n < 60 and hist[-1] < 1e-9 and min(hist[:-1]) >= 1e-9
    assert all(b < a for a, b in zip(hist[2:], hist[3:])), hist
    ZZ = np.kron(np.diag([1.0, -1.0]), np.diag([1.0, -1.0]))
    _, bonds = En.energy_per_site(A, env, ZZ, split=split, return_bonds=True)
    assert abs(float(bonds[(0, 0)]["top"]) - _onsager_nn(beta)) < 5e-7


def test_run_stops_at_once_for_a_product_state():
    """A D=1 product state has rank-one corners: their normalised spectrum is
    (1, 0, ...) from the start, so the first step already changes nothing."""
    A = C.as_cell(np.array([0.8, 0.6]).reshape(1, 1, 2, 1, 1, 1, 1))
    _, n, hist = C.ctmrg_run(A, 4, 1e-12, 10)
    assert n == 1 and hist[0] < 1e-15


def _near_product(Lx, Ly, D, eps, seed):
    rng = np.random.default_rng(seed)
    A0 = np.zeros((Lx, Ly, 2, D, D, D, D))
    A0[:, :, 0, 0, 0, 0, 0] = 0.8
    A0[:, :, 1, 0, 0, 0, 0] = 0.6
    return A0 + eps * rng.standard_normal(A0.shape)


def test_split_agrees_with_conventional():
    """Split and conventional CTMRG converge to the same energy (Sec. III,
    Fig. 4a) on a generic correlated state; both are invariant under lattice
    rotation and reflection."""
    A0 = _near_product(1, 1, 2, 0.25, seed=5)
    vals = []
    for Av in (A0, I.rotate_cell_90(A0), A0.transpose(0, 1, 2, 3, 6, 5, 4)):
        A = C.as_cell(Av)
        vals.append(float(En.energy_per_site(A, C.split_ctmrg(A, 12, 20), HR)))
        vals.append(float(En.energy_per_site(A, C.conv_ctmrg(A, 12, 20), HR, split=False)))
    assert max(vals) - min(vals) < 5e-7


@pytest.mark.parametrize("split", [True, False])
def test_energy_converges_monotonically_in_chi(split):
    """The truncation error of the energy falls monotonically as chi grows, and
    vanishes to rounding once chi holds every singular value above the cutoff
    (Sec. III, Fig. 4a: the energy converges in the environment bond dimension).  A
    projector that kept the wrong singular vectors, or paired the halves of a
    cut the wrong way, would break the monotone decrease or the final agreement."""
    A = C.as_cell(_near_product(1, 1, 2, 0.25, seed=5))
    run = C.split_ctmrg if split else C.conv_ctmrg
    E = {chi: float(En.energy_per_site(A, run(A, chi, 30), HR, split=split)) for chi in (2, 4, 8, 12, 16, 20)}
    err = [abs(E[chi] - E[20]) for chi in (2, 4, 8, 12)]
    assert all(b < a for a, b in zip(err, err[1:])), err
    assert err[0] > 1e-3   # chi = 2 truncates visibly
    assert abs(E[16] - E[20]) < 1e-10


def test_split_conventional_gap_closes_with_chi():
    """The split and the conventional CTMRG approximate the same contraction
    with different truncations, so their energies approach each other as chi
    grows (Sec. III, Fig. 4a): on a random D=2 state the gap falls at every step
    chi = 2, 4, 8, 12, 16, 20, by five orders of magnitude in all."""
    A = C.as_cell(I.random_cell(1, 1, 2, 2, seed=0))
    gap = []
    for chi in (2, 4, 8, 12, 16, 20):
        e_s = float(En.energy_per_site(A, C.split_ctmrg(A, chi, 30), HR))
        e_c = float(En.energy_per_site(A, C.conv_ctmrg(A, chi, 30), HR, split=False))
        gap.append(abs(e_s - e_c))
    assert all(b < a for a, b in zip(gap, gap[1:])), gap
    assert gap[0] > 1e-2 and gap[-1] < 1e-6, gap


def test_interlayer_bond_dimension():
    """chi_I (the bond between a ket and a bra edge) is truncated separately
    from chi_E (Sec. II.B): the split edges are [chi_E, D, chi_I] and
    [chi_I, D, chi_E]; at fixed chi_E the energy approaches its chi_I = chi_E
    value as chi_I grows (Sec. III, Fig. 4b), and a pair (chi, chi) is the
    same computation as chi."""
    A = C.as_cell(_near_product(1, 1, 2, 0.25, seed=5))
    chi_e = 12
    E = {}
    for chi_i in (2, 4, 6, 8, 12):
        env = C.split_ctmrg(A, (chi_e, chi_i), 30)
        e = env[0][0]
        assert e["T1k"].shape[0] == e["T1b"].shape[2] == chi_e
        assert e["T1k"].shape[2] == e["T1b"].shape[0] <= chi_i
        assert e["T4b"].shape[0] == e["T4k"].shape[2] == chi_e
        assert e["T4b"].shape[2] == e["T4k"].shape[0] <= chi_i
        E[chi_i] = float(En.energy_per_site(A, env, HR))
    err = [abs(E[c] - E[chi_e]) for c in (2, 4, 6, 8)]
    assert all(b < a for a, b in zip(err, err[1:])) and err[-1] < 1e-5, err
    assert float(En.energy_per_site(A, C.split_ctmrg(A, (8, 8), 5), HR)) == \
        float(En.energy_per_site(A, C.split_ctmrg(A, 8, 5), HR))


def test_implicit_gradient_matches_unrolled_and_finite_differences():
    """The implicit (fixed-point) gradient of the converged energy equals the
    gradient taken through 30 unrolled steps, whose transient has died out, and
    a central difference of the converged energy along a random direction."""
    A = _near_product(1, 1, 2, 0.25, seed=5)
    chi = 8
    E, g, info = implicit_energy_grad(A, chi, HR)
    assert info["solver_iterations"] < 100
    At = torch.tensor(A).requires_grad_(True)
    Ac = [[At[0, 0]]]
    e = En.energy_per_site(Ac, C.split_ctmrg(Ac, chi, 30), HR)
    e.backward()
    assert abs(float(e.detach()) - E) < 1e-12
    assert float((At.grad - g).norm() / g.norm()) < 1e-10
    v = np.random.default_rng(1).standard_normal(A.shape)
    v /= np.linalg.norm(v)
    eps = 1e-5

    def converged(X):
        env, _, _ = C.ctmrg_run(X, chi, 1e-14, 300)
        return float(En.energy_per_site(C.as_cell(X), env, HR))
    fd = (converged(A + eps * v) - converged(A - eps * v)) / (2 * eps)
    assert abs(fd - float((g.numpy() * v).sum())) < 1e-7 * abs(fd)


def test_implicit_gradient_refuses_a_gauge_that_is_not_fixed():
    """The conventional scheme's tensors keep changing sign between steps even
    when its corner spectra have converged, with no short period: the
    fixed-point rule does not apply there."""
    A = _near_product(1, 1, 2, 0.25, seed=5)
    with pytest.raises(ValueError):
        implicit_energy_grad(A, 8, HR, split=False, max_sweeps=40)


@pytest.mark.parametrize("seed,period", [(0, 2), (3, None)])
def test_implicit_gradient_through_a_sign_cycle(seed, period):
    """A random D=2 state: at converged spectra the projector signs cycle, so
    the environment is a fixed point of a few steps only.  The rule applied to
    that p-step map must still give the derivative of the converged energy
    (central difference along a random direction, 1e-6) and report its period."""
    A = I.random_cell(1, 1, 2, 2, seed=seed)
    chi = 8
    E, g, info = implicit_energy_grad(A, chi, H)
    if period is not None:
        assert info["period"] == period
    v = np.random.default_rng(7).standard_normal(A.shape)
    v /= np.linalg.norm(v)
    eps = 1e-5

    def converged(X):
        env, _, _ = C.ctmrg_run(X, chi, 1e-14, 400)
        return float(En.energy_per_site(C.as_cell(X), env, H))
    fd = (converged(A + eps * v) - converged(A - eps * v)) / (2 * eps)
    assert abs(fd - float((g.numpy() * v).sum())) < 1e-6 * max(abs(fd), 1e-3)


def test_honeycomb_bond_closed_forms():
    """The coarse-grained honeycomb bond (p = 4: spins A, B of one honeycomb bond
    per site) on D=1 product states: intra-site singlets give -3/4 per site
    (singlet -3/4, inter-site bonds 0), Neel A-up B-down gives 3 x (-1/4), and a
    ferromagnet 3 x (+1/4).  A 1x2 cell fixes the orientation: the horizontal
    bond couples B of the left site to A of the right site."""
    h = I.honeycomb_bond()

    def energy(phis, **kw):
        phis = np.asarray(phis, dtype=np.float64)
        A = np.zeros(phis.shape[:2] + (4, 1, 1, 1, 1))
        A[:, :, :, 0, 0, 0, 0] = phis
        Ac = C.as_cell(A)
        return En.energy_per_site(Ac, C.split_ctmrg(Ac, 2, 2), h, **kw)

    r = 2 ** -0.5
    assert abs(float(energy([[[0, r, -r, 0]]])) + 0.75) < 1e-12
    assert abs(float(energy([[[0, 1, 0, 0]]])) + 0.75) < 1e-12
    assert abs(float(energy([[[0.5, 0.5, 0.5, 0.5]]])) - 0.75) < 1e-12
    # left site A-up B-up (index 0), right site A-down B-up (index 2): S_B(left).S_A(right) = -1/4,
    # and the two intra-site shares (+1/4 and -1/4, a quarter each) cancel
    _, bonds = energy([[[1, 0, 0, 0], [0, 0, 1, 0]]], return_bonds=True)
    assert abs(float(bonds[(0, 0)]["top"]) + 0.25) < 1e-12


@pytest.mark.parametrize("vertical", [False, True])
def test_p4_dimer_states_exact(vertical):
    """The paper's p = 4 sites (coarse-grained honeycomb bond, R13): a product of
    generic entangled two-site states (16 amplitudes each, gauge-scrambled
    bonds) gives the state-vector energy exactly."""
    h = I.honeycomb_bond()
    psis = np.random.default_rng(4).standard_normal((2, 4, 4))
    A = I.gauge_transform_cell(I.dimer_pairs_cell(psis, D=4, vertical=vertical), seed=3)
    ref = SV.dimer_pairs_energy(psis, h, None, vertical=vertical)
    assert abs(E_split(A, chi=16, sweeps=3, h=h) - ref) < 1e-12


def test_rotation_and_gauge_invariance():
    """The energy of an isotropic Hamiltonian does not change when the lattice
    is rotated by 90 degrees or when gauge matrices are put on every bond
    (2x2 cell, J1-J2)."""
    A = _near_product(2, 2, 2, 0.3, seed=21)
    e0 = E_split(A, chi=12, sweeps=12, h=H, hd=0.5 * H)
    e1 = E_split(I.rotate_cell_90(A), chi=12, sweeps=12, h=H, hd=0.5 * H)
    e2 = E_split(I.gauge_transform_cell(A, seed=22, scale=0.2), chi=12, sweeps=12, h=H, hd=0.5 * H)
    assert abs(e0 - e1) < 5e-7
    assert abs(e0 - e2) < 5e-7


def test_bond_values_physical():
    """Every <S_i . S_j> lies in [-3/4, 1/4]."""
    A = C.as_cell(_near_product(2, 2, 2, 0.5, seed=6))
    env = C.split_ctmrg(A, 12, 16)
    _, bonds = En.energy_per_site(A, env, H, H, return_bonds=True)
    for v in bonds.values():
        for k, val in v.items():
            if k != "norm":
                assert -0.75 - 1e-9 <= float(val) <= 0.25 + 1e-9


def test_frame_maps_are_involutions():
    A = C.as_cell(I.random_cell(2, 2, 2, 2, seed=8))
    env = C.initial_env(A, 16)
    for f in (C.transpose_frame, C.rot180_frame):
        A1, e1 = f(A, env)
        A2, e2 = f(A1, e1)
        for x in range(2):
            for y in range(2):
                assert torch.equal(A2[x][y], A[x][y])
                for k in C.SPLIT_KEYS:
                    assert torch.equal(e2[x][y][k], env[x][y][k])


# ---------------------------------------------------------------- gradients
def test_svd_backward_matches_finite_differences():
    torch.manual_seed(0)
    M = torch.randn(6, 6, dtype=torch.float64)
    W1 = torch.randn(6, 3, dtype=torch.float64)
    W2 = torch.randn(6, 3, dtype=torch.float64)

    def f(M):
        U, S, V = osvd(M)
        # sign-invariant function of the top-3 triplets
        return ((U[:, :3] * S[:3]) @ (V[:, :3].T @ W2) * W1.sum(1, keepdim=True)).sum() + (S[:3] ** 2).sum()

    Mg = M.clone().requires_grad_(True)
    f(Mg).backward()
    Dm = torch.randn(6, 6, dtype=torch.float64)
    h = 1e-6
    fd = (f(M + h * Dm) - f(M - h * Dm)) / (2 * h)
    assert abs(float((Mg.grad * Dm).sum()) - float(fd)) < 1e-6 * max(1.0, abs(float(fd)))


def test_oracle_gradient_matches_finite_differences():
    """Autograd through the whole oracle (init, sweeps, energy) equals the
    central finite difference (step 1e-5) along random directions."""
    A0 = torch.as_tensor(I.random_cell(1, 1, 2, 2, seed=3))

    def energy(At):
        Ac = [[At[0, 0]]]
        env = C.split_ctmrg(Ac, chi=8, sweeps=3)
        return En.energy_per_site(Ac, env, HR)

    Ag = A0.clone().requires_grad_(True)
    energy(Ag).backward()
    g = Ag.grad
    rng = np.random.default_rng(0)
    for _ in range(2):
        v = torch.as_tensor(rng.standard_normal(A0.shape))
        h = 1e-5
        fd = (energy(A0 + h * v) - energy(A0 - h * v)) / (2 * h)
        ad = (g * v).sum()
        assert abs(float(ad) - float(fd)) < 1e-6 * max(1e-3, abs(float(fd)))


def test_projector_pair_reduced_and_plain_forms_agree_on_rank_deficient_halves():
    """App. A's QR reduction (value-only runs) and the plain M = rhoB rhoT form
    (used when differentiating) give the same projectors; at rank-deficient
    halves the plain form's gradient is finite and matches a central
    difference (the kept values are separated from the zero ones)."""
    rng = np.random.default_rng(7)
    na, nb, rank, k = 12, 30, 7, 5
    X = torch.tensor(rng.standard_normal((na, rank)) @ rng.standard_normal((rank, nb)))
    Y = torch.tensor(rng.standard_normal((nb, rank)) @ rng.standard_normal((rank, na)))
    with torch.no_grad():
        up_r, dn_r, s_r = C.projector_pair(X, Y, k)
    Xg, Yg = X.clone().requires_grad_(True), Y.clone().requires_grad_(True)
    up_p, dn_p, s_p = C.projector_pair(Xg, Yg, k)
    assert torch.allclose(s_r[:k], s_p[:k].detach(), rtol=1e-12)
    # the kept product P_dn P_up is basis independent; P_up rows carry fixed signs
    assert torch.allclose(dn_r @ up_r, (dn_p @ up_p).detach(), atol=1e-10)
    assert torch.allclose(up_r, up_p.detach(), atol=1e-10)
    W = torch.tensor(rng.standard_normal((na, na)))
    f = ((dn_p @ up_p) * W).sum()
    f.backward()
    assert torch.isfinite(Xg.grad).all() and torch.isfinite(Yg.grad).all()
    dX, dY = torch.tensor(rng.standard_normal(X.shape)), torch.tensor(rng.standard_normal(Y.shape))
    h = 1e-6

    def fval(t):
        with torch.no_grad():
            u, d, _ = C.projector_pair(X + t * dX, Y + t * dY, k)
            return float(((d @ u) * W).sum())
    fd = (fval(h) - fval(-h)) / (2 * h)
    an = float((Xg.grad * dX).sum() + (Yg.grad * dY).sum())
    assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (fd, an)


# ------------------------------------ alternative yellow/red order (App. B)
def test_alternative_order_exact_states():
    """The alternative order (physical leg truncated by yellow) on states the
    CTMRG must reproduce exactly: Neel (-1/2 + J2/2 per site) and products of
    generic entangled two-site states (state-vector energy)."""
    phis = np.zeros((2, 2, 2))
    phis[0, 0, 0] = phis[1, 1, 0] = phis[0, 1, 1] = phis[1, 0, 1] = 1.0
    Ac = C.as_cell(I.product_state_cell(phis, D=2))
    e = float(En.energy_per_site(Ac, C.split_ctmrg(Ac, 4, 2, order="alternative"), H, 0.5 * H))
    assert abs(e - (-0.5 + 0.25)) < 1e-12
    for vertical in (False, True):
        rng = np.random.default_rng(12 + vertical)
        psis = rng.standard_normal((2, 2, 2))
        Ac = C.as_cell(I.gauge_transform_cell(I.dimer_pairs_cell(psis, D=2, vertical=vertical), seed=3))
        ref = SV.dimer_pairs_energy(psis, H, 0.5 * H, vertical=vertical)
        e = float(En.energy_per_site(Ac, C.split_ctmrg(Ac, 16, 3, order="alternative"), H, 0.5 * H))
        assert abs(e - ref) < 1e-10, (vertical, e, ref)


def test_alternative_order_agrees_with_standard_as_chi_grows():
    """App. B's alternative order changes only which projector truncates the
    physical leg, so at converged chi it must give the standard order's (and
    the conventional CTMRG's) energy: on a random D=2 state after 40 steps the
    differences shrink with chi and are below 2e-7 at chi = 24."""
    Ac = C.as_cell(I.random_cell(1, 1, 2, 2, seed=0))
    gaps = []
    with torch.no_grad():
        for chi in (8, 16, 24):
            e_alt = float(En.energy_per_site(Ac, C.split_ctmrg(Ac, chi, 40, order="alternative"), HR))
            e_std = float(En.energy_per_site(Ac, C.split_ctmrg(Ac, chi, 40), HR))
            e_conv = float(En.energy_per_site(Ac, C.conv_ctmrg(Ac, chi, 40), HR, split=False))
            gaps.append((abs(e_alt - e_conv), abs(e_alt - e_std)))
    assert gaps[0][0] > gaps[1][0] > gaps[2][0], gaps
    assert gaps[2][0] < 2e-7 and gaps[2][1] < 2e-7, gaps
