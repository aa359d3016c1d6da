"""GPU (C-ABI) vs FP64 oracle parity of the split-CTMRG hot path."""
import numpy as np
import pytest
import torch

import ipeps_inputs as I
from oracle import ctmrg as C
from oracle import energy as En

from gpu_helpers import env_max_rel_diff

pytestmark = pytest.mark.gpu

H = I.heisenberg_bond()
HR = I.heisenberg_bond_rotated()


@pytest.fixture(scope="module")
def S():
    import paper_2502_10298_gb300 as S
    S.load_library()
    return S


def _near(Lx, Ly, D, eps, seed):
    rng = np.random.default_rng(seed)
    A0 = np.zeros((Lx, Ly, 2, D, D, D, D))
    A0[:, :, 0, 0, 0, 0, 0] = 0.8
    A0[:, :, 1, 0, 0, 0, 0] = 0.6
    return A0 + eps * rng.standard_normal(A0.shape)


CASES = [(1, 1, 2, 8), (2, 2, 2, 8), (1, 2, 2, 6)]


@pytest.mark.parametrize("Lx,Ly,D,chi", CASES)
def test_initial_environment(S, Lx, Ly, D, chi):
    A = I.random_cell(Lx, Ly, 2, D, seed=11)
    with S.SplitCTMRG(Lx, Ly, 2, D, chi) as s:
        s.init(torch.tensor(A, device="cuda"))
        env = C.initial_env(C.as_cell(A), chi)
        assert env_max_rel_diff(s, env, chi) < 1e-12


@pytest.mark.parametrize("direction", [0, 1, 2, 3])
@pytest.mark.parametrize("Lx,Ly,D,chi", CASES)
def test_single_move(S, direction, Lx, Ly, D, chi):
    A = _near(Lx, Ly, D, 0.4, seed=12)
    with S.SplitCTMRG(Lx, Ly, 2, D, chi) as s:
        s.init(torch.tensor(A, device="cuda"))
        s.move(direction)
        Ac = C.as_cell(A)
        env = C.split_move(Ac, C.initial_env(Ac, chi), direction, chi)
        # entries tied to singular values within rounding of the 1e-8 cutoff
        # differ at that level; energies agree to 1e-10 (tests below)
        assert env_max_rel_diff(s, env, chi) < 1e-7


@pytest.mark.parametrize("Lx,Ly,D,chi", [(1, 1, 2, 8), (2, 2, 2, 8)])
def test_sweeps_environment_and_energy(S, Lx, Ly, D, chi):
    A = _near(Lx, Ly, D, 0.3, seed=13)
    h, hd = (HR, None) if Lx == 1 else (H, 0.5 * H)
    with S.SplitCTMRG(Lx, Ly, 2, D, chi) as s:
        s.init(torch.tensor(A, device="cuda"))
        s.sweeps(3)
        Ac = C.as_cell(A)
        env = C.split_ctmrg(Ac, chi, 3)
        assert env_max_rel_diff(s, env, chi) < 1e-8
        e_gpu = s.energy(h, hd)
        e_or = float(En.energy_per_site(Ac, env, h, hd))
        assert abs(e_gpu - e_or) < 1e-10 * abs(e_or)


def test_d2_chi16_thirty_sweeps_energy(S):
    """1x1, d=2, D=2, chi=16, 30 sweeps (rotated Heisenberg): energy vs oracle."""
    A, c = I.config("d2_chi16_1x1")
    with S.SplitCTMRG(1, 1, 2, 2, 16) as s:
        s.init(torch.tensor(A, device="cuda"))
        s.sweeps(30)
        e_gpu = s.energy(HR)
    Ac = C.as_cell(A)
    e_or = float(En.energy_per_site(Ac, C.split_ctmrg(Ac, 16, 30), HR))
    assert abs(e_gpu - e_or) < 1e-10 * abs(e_or)


def _through_inner(X, inner_up, inner_dn, k, rest):
    """P_dn P_up of teal (red) lives on alpha = (green (yellow) kept index, rest
    of the wires); mapped back through the green (yellow) pair of the same band
    it becomes an operator on the unprojected wires, independent of the basis
    and signs of the inner kept space: [(m, r), (m', r')]"""
    Xr = X.reshape(k, rest, k, rest)
    C = torch.einsum("ak,krls,lb->arbs", inner_dn, Xr, inner_up)
    m = inner_dn.shape[0]
    return C.reshape(m * rest, m * rest)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("colour", [0, 1, 2, 3])
def test_projectors(S, colour, order):
    """Projector pairs of the first left-move column at the initial environment:
    singular values, and the product P_dn P_up element by element for every
    colour.  Green and yellow compare P_dn P_up itself (independent of the
    basis and signs of their kept space).  Teal and red compare it mapped back
    through the green (yellow) pair their alpha index comes from, which
    removes the dependence on the inner pair's basis.  The oracle grows the
    environment leg of alpha while the GPU pads it to chi, so the oracle's
    alpha is embedded into the padded one and the padding must stay zero.
    order 1: the alternative yellow/red order of App. B."""
    Lx, Ly, D, chi, p = 2, 2, 2, 8, 2
    A = _near(Lx, Ly, D, 0.4, seed=14)
    Ac = C.as_cell(A)
    rec = {}
    C.split_column_projectors(Ac, C.initial_env(Ac, chi), 0, chi, record=rec, order=C.ORDERS[order])
    name = ["green", "teal", "yellow", "red"][colour]
    inner = {"teal": ("green", 0), "red": ("yellow", 2)}.get(name)
    up_o, dn_o, s_o = (t.detach() for t in rec[name][0])
    with S.SplitCTMRG(Lx, Ly, p, D, chi, projector_order=order) as s:
        s.init(torch.tensor(A, device="cuda"))
        up, dn, sv = s.projectors(0, 0, 0, colour)
        if inner:
            iup, idn, _ = s.projectors(0, 0, 0, inner[1])
    n = min(len(s_o), chi)
    assert np.allclose(sv[:n], s_o.numpy()[:n], rtol=1e-9, atol=1e-12 * float(s_o[0]))
    Po = dn_o @ up_o
    Pg = dn.cpu() @ up.cpu()
    if inner:
        rest = Pg.shape[0] // chi                             # wires of alpha beside the inner index
        iup_o, idn_o, _ = (t.detach() for t in rec[inner[0]][0])
        Po = _through_inner(Po, iup_o, idn_o, iup_o.shape[0], rest)
        Pg = _through_inner(Pg, iup.cpu(), idn.cpu(), chi, rest)
    lead = Pg.shape[0] // chi                                 # alpha = (env leg padded to chi, lead)
    e_o = Po.shape[0] // lead
    idx = (torch.arange(e_o)[:, None] * lead + torch.arange(lead)[None, :]).reshape(-1)
    # the product of one pair carries rounding amplified by s^-1/2 of values down
    # to the 1e-8 cutoff; a composite multiplies three such products
    tol = (1e-7 if inner else 1e-9) * float(Po.abs().max())
    diff = float((Pg[idx][:, idx] - Po).abs().max())
    assert diff <= tol, (name, diff, tol)
    rest_mask = torch.ones(Pg.shape[0], dtype=torch.bool)
    rest_mask[idx] = False
    if rest_mask.any():
        pad = max(float(Pg[rest_mask].abs().max()), float(Pg[:, rest_mask].abs().max()))
        assert pad <= 1e-12 * float(Po.abs().max()), (name, pad)


@pytest.mark.parametrize("Lx,Ly,D,chi,sweeps", [(1, 1, 2, 8, 2), (2, 2, 2, 6, 1)])
def test_gradient_matches_oracle_autograd(S, Lx, Ly, D, chi, sweeps):
    A = I.random_cell(Lx, Ly, 2, D, seed=3) if Lx == 1 else _near(Lx, Ly, D, 0.4, seed=15)
    h, hd = (HR, None) if Lx == 1 else (H, 0.5 * H)
    with S.SplitCTMRG(Lx, Ly, 2, D, chi) as s:
        e, g = s.energy_grad(torch.tensor(A, device="cuda"), sweeps, h, hd)
    Ao = torch.tensor(A).requires_grad_(True)
    Ac = [[Ao[x, y] for y in range(Ly)] for x in range(Lx)]
    eo = En.energy_per_site(Ac, C.split_ctmrg(Ac, chi, sweeps), h, hd)
    eo.backward()
    assert abs(e - float(eo)) < 1e-10 * abs(float(eo))
    rel = float((g.cpu() - Ao.grad).norm() / Ao.grad.norm())
    assert rel < 1e-7, rel


def test_fp64_d4_chi32_2x2_energy_and_gradient(S):
    """FP64 forward and reverse pass at the 2x2, D=4, chi=32 workload (random
    seeded tensors, Heisenberg J=1, two sweeps) against the oracle's autograd:
    energy to 1e-10 relative, gradient to 1e-7 (norm)."""
    A, c = I.config("d4_chi32_2x2")
    chi, sweeps = c["chi"], 2
    with S.SplitCTMRG(2, 2, 2, c["D"], chi) as s:
        e, g = s.energy_grad(torch.tensor(A, device="cuda"), sweeps, H, None)
    Ao = torch.tensor(A).requires_grad_(True)
    Ac = [[Ao[x, y] for y in range(2)] for x in range(2)]
    eo = En.energy_per_site(Ac, C.split_ctmrg(Ac, chi, sweeps), H, None)
    eo.backward()
    assert abs(e - float(eo.detach())) < 1e-10 * abs(float(eo.detach()))
    rel = float((g.cpu() - Ao.grad).norm() / Ao.grad.norm())
    assert rel < 1e-7, rel


def test_neel_and_ising_exact(S):
    phis = np.zeros((2, 2, 2))
    phis[0, 0, 0] = phis[1, 1, 0] = phis[0, 1, 1] = phis[1, 0, 1] = 1.0
    A = I.product_state_cell(phis, D=2)
    with S.SplitCTMRG(2, 2, 2, 2, 8) as s:
        s.init(torch.tensor(A, device="cuda"))
        s.sweeps(2)
        assert abs(s.energy(H, 0.5 * H) - (-0.5 + 0.25)) < 1e-12


@pytest.mark.parametrize("m,n", [(7, 7), (40, 40), (100, 60), (300, 256), (700, 200)])
def test_jacobi_svd_against_lapack(S, m, n):
    """Singular values to 1e-13 relative; U S V^T reproduces M; U, V orthonormal."""
    rng = np.random.default_rng(m + n)
    M = rng.standard_normal((m, n)) * np.logspace(0, -6, n)[None, :]
    with S.SplitCTMRG(1, 1, 2, 2, 4) as s:
        U, Sv, V = S.sctm_svd(s.h, torch.tensor(M, device="cuda"))
    U, Sv, V = U.cpu().numpy(), Sv.cpu().numpy(), V.cpu().numpy()
    ref = np.linalg.svd(M, compute_uv=False)
    assert np.allclose(Sv, ref, rtol=1e-12, atol=1e-14 * ref[0])
    assert np.abs(U * Sv[None, :] @ V.T - M).max() < 1e-13 * ref[0]
    assert np.abs(V.T @ V - np.eye(n)).max() < 1e-13
    assert np.abs(U.T @ U - np.eye(n)).max() < 1e-11


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("Lx,Ly,D,chi", [(1, 1, 3, 9), (2, 2, 3, 9)])
def test_mixed_mode_energy_and_gradient(S, Lx, Ly, D, chi, prec):
    """precision 1 (large contractions on the tensor cores) and 2 (FP32 on the
    CUDA cores) with their default cutoff: energy within 1e-6 per site and
    gradient within 1e-4 (norm) of the FP64 oracle (cutoff 1e-8)."""
    A = _near(Lx, Ly, D, 0.3, seed=21)
    h, hd = (HR, None) if Lx == 1 else (H, 0.5 * H)
    sweeps = 2
    with S.SplitCTMRG(Lx, Ly, 2, D, chi, precision=prec) as s:
        e, g = s.energy_grad(torch.tensor(A, device="cuda"), sweeps, h, hd)
    Ao = torch.tensor(A).requires_grad_(True)
    Ac = [[Ao[x, y] for y in range(Ly)] for x in range(Lx)]
    eo = En.energy_per_site(Ac, C.split_ctmrg(Ac, chi, sweeps), h, hd)
    eo.backward()
    assert abs(e - float(eo)) < 1e-6
    rel = float((g.cpu() - Ao.grad).norm() / Ao.grad.norm())
    assert rel < 1e-4, rel


def _randomized_case():
    D, chi = 4, 64
    return D, chi, torch.tensor(_near(1, 1, D, 0.3, seed=5), device="cuda")


def test_randomized_projectors_fp64_match_exact(S):
    """Randomized projectors (the default for the truncated spaces chi p D = 512
    of the yellow and red projectors, four times the chi + 32 sketch columns;
    green and teal, chi D = 256, stay exact) with FP64 arithmetic (precision 3): energy
    within 1e-8 and gradient within 2e-4 of the exact-SVD FP64 path at the same
    cutoff, two sweeps."""
    D, chi, At = _randomized_case()
    with S.SplitCTMRG(1, 1, 2, D, chi, precision=0, svd_cutoff=1e-6) as s:
        e0, g0 = s.energy_grad(At, 2, HR, None)
    with S.SplitCTMRG(1, 1, 2, D, chi, precision=3, svd_cutoff=1e-6) as s:
        e1, g1 = s.energy_grad(At, 2, HR, None)
    assert abs(e1 - e0) < 1e-8, (e0, e1)
    rel = float((g1 - g0).norm() / g0.norm())
    assert rel < 2e-4, rel


def test_mixed_randomized_matches_fp64_gpu(S):
    """Mixed mode with randomized projectors against the FP64 exact path at the
    same cutoff (1e-5, the mixed default).  This near-product state after two
    sweeps is ill-conditioned: the FP64 gradient itself moves by 7e-3 between
    cutoffs 1e-8 and 1e-5, so the gradient bound here is that scale, not 1e-4;
    the energy stays within 1e-6."""
    D, chi, At = _randomized_case()
    with S.SplitCTMRG(1, 1, 2, D, chi, precision=0, svd_cutoff=1e-5) as s:
        e0, g0 = s.energy_grad(At, 2, HR, None)
    with S.SplitCTMRG(1, 1, 2, D, chi, precision=1) as s:
        e1, g1 = s.energy_grad(At, 2, HR, None)
    assert abs(e1 - e0) < 1e-6, (e0, e1)
    rel = float((g1 - g0).norm() / g0.norm())
    assert rel < 3e-2, rel


@pytest.mark.parametrize("Lx,Ly,D,chi", [(1, 1, 2, 8), (2, 2, 2, 8)])
def test_conventional_ctmrg_energy_matches_oracle(S, Lx, Ly, D, chi):
    """Conventional double-layer CTMRG (algorithm 1) on the GPU against the
    oracle's conv_ctmrg: energy after three sweeps to 1e-10 relative."""
    A = _near(Lx, Ly, D, 0.3, seed=13)
    h, hd = (HR, None) if Lx == 1 else (H, 0.5 * H)
    with S.SplitCTMRG(Lx, Ly, 2, D, chi, algorithm=1) as s:
        s.init(torch.tensor(A, device="cuda"))
        s.sweeps(3)
        e_gpu = s.energy(h, hd)
        env = s.env(0, 0)
        assert set(env) == {"C1", "T1", "C2", "T2", "C3", "T3", "C4", "T4"}
    Ac = C.as_cell(A)
    e_or = float(En.energy_per_site(Ac, C.conv_ctmrg(Ac, chi, 3), h, hd, split=False))
    assert abs(e_gpu - e_or) < 1e-10 * abs(e_or)


def test_conventional_ctmrg_gradient_matches_oracle(S):
    """Gradient of the conventional CTMRG energy (two sweeps) against the
    oracle's autograd, 1e-7 relative."""
    Lx, Ly, D, chi, sweeps = 1, 1, 2, 8, 2
    A = I.random_cell(Lx, Ly, 2, D, seed=3)
    with S.SplitCTMRG(Lx, Ly, 2, D, chi, algorithm=1) as s:
        e, g = s.energy_grad(torch.tensor(A, device="cuda"), sweeps, HR, None)
    Ao = torch.tensor(A).requires_grad_(True)
    Ac = [[Ao[0, 0]]]
    eo = En.energy_per_site(Ac, C.conv_ctmrg(Ac, chi, sweeps), HR, None, split=False)
    eo.backward()
    assert abs(e - float(eo)) < 1e-10 * abs(float(eo))
    rel = float((g.cpu() - Ao.grad).norm() / Ao.grad.norm())
    assert rel < 1e-7, rel


@pytest.mark.parametrize("Lx,Ly,D,chi", [(1, 1, 2, 8), (2, 2, 2, 8)])
def test_alternative_order_sweeps_environment_and_energy(S, Lx, Ly, D, chi):
    """The alternative yellow/red order of App. B (projector_order 1) against
    the oracle's: environment after three sweeps to 1e-8, energy to 1e-10."""
    A = _near(Lx, Ly, D, 0.3, seed=13)
    h, hd = (HR, None) if Lx == 1 else (H, 0.5 * H)
    with S.SplitCTMRG(Lx, Ly, 2, D, chi, projector_order=1) as s:
        s.init(torch.tensor(A, device="cuda"))
        s.sweeps(3)
        Ac = C.as_cell(A)
        env = C.split_ctmrg(Ac, chi, 3, order="alternative")
        assert env_max_rel_diff(s, env, chi) < 1e-8
        e_gpu = s.energy(h, hd)
        e_or = float(En.energy_per_site(Ac, env, h, hd))
        assert abs(e_gpu - e_or) < 1e-10 * abs(e_or)


def test_alternative_order_gradient_matches_oracle_autograd(S):
    """Gradient through the alternative order, two sweeps, 1e-7 (norm)."""
    Lx, Ly, D, chi, sweeps = 1, 1, 2, 8, 2
    A = I.random_cell(Lx, Ly, 2, D, seed=3)
    with S.SplitCTMRG(Lx, Ly, 2, D, chi, projector_order=1) as s:
        e, g = s.energy_grad(torch.tensor(A, device="cuda"), sweeps, HR, None)
    Ao = torch.tensor(A).requires_grad_(True)
    eo = En.energy_per_site([[Ao[0, 0]]], C.split_ctmrg([[Ao[0, 0]]], chi, sweeps, order="alternative"), HR, None)
    eo.backward()
    assert abs(e - float(eo.detach())) < 1e-10 * abs(float(eo.detach()))
    rel = float((g.cpu() - Ao.grad).norm() / Ao.grad.norm())
    assert rel < 1e-7, rel


@pytest.mark.parametrize("Lx,Ly,D,chiE,chiI", [(1, 1, 2, 12, 8), (2, 2, 2, 10, 6)])
def test_interlayer_dimension_environment_and_energy(S, Lx, Ly, D, chiE, chiI):
    """chi_I below chi_E (the regime of the chi_I sweep in Sec. III): the
    environment after three sweeps to 1e-8 and the energy to 1e-10 against the
    oracle's (chi_E, chi_I) mode."""
    A = _near(Lx, Ly, D, 0.3, seed=13)
    h, hd = (HR, None) if Lx == 1 else (H, 0.5 * H)
    with S.SplitCTMRG(Lx, Ly, 2, D, chiE, chi_I=chiI) as s:
        s.init(torch.tensor(A, device="cuda"))
        s.sweeps(3)
        Ac = C.as_cell(A)
        env = C.split_ctmrg(Ac, (chiE, chiI), 3)
        assert env_max_rel_diff(s, env, chiE, chiI) < 1e-8
        e_gpu = s.energy(h, hd)
        e_or = float(En.energy_per_site(Ac, env, h, hd))
        assert abs(e_gpu - e_or) < 1e-10 * abs(e_or)


def test_interlayer_dimension_gradient_matches_oracle_autograd(S):
    """Gradient with chi_I = 6 < chi_E = 10, two sweeps, 1e-7 (norm)."""
    A = I.random_cell(1, 1, 2, 2, seed=3)
    with S.SplitCTMRG(1, 1, 2, 2, 10, chi_I=6) as s:
        e, g = s.energy_grad(torch.tensor(A, device="cuda"), 2, HR, None)
    Ao = torch.tensor(A).requires_grad_(True)
    eo = En.energy_per_site([[Ao[0, 0]]], C.split_ctmrg([[Ao[0, 0]]], (10, 6), 2), HR, None)
    eo.backward()
    assert abs(e - float(eo.detach())) < 1e-10 * abs(float(eo.detach()))
    rel = float((g.cpu() - Ao.grad).norm() / Ao.grad.norm())
    assert rel < 1e-7, rel
