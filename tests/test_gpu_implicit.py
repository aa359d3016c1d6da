"""Implicit (fixed-point) energy gradient on the GPU against the oracle's rule.

The oracle's ``implicit_energy_grad`` converges the environment, finds the
smallest number of full steps (up to four) after which it is an element-wise
fixed point, differentiates the energy there and solves the adjoint
fixed-point equation of that many steps (Sec. I, Sec. II.B, Sec. III;
implicit function theorem).  The engine's ``energy_grad_implicit``
takes the same steps in FP64.  Cases: near-product states, which the sign-
fixed projectors bring to an element-wise fixed point of one step, and states
whose projector signs still cycle at converged spectra, which are fixed points
of two or four steps (the rule then applies to that many steps).  Both sides
must find the same period, and refuse an environment with none.
"""
import numpy as np
import pytest
import torch

import ipeps_inputs as I
from oracle.fixed_point import implicit_energy_grad

pytestmark = pytest.mark.gpu

HR = I.heisenberg_bond_rotated()
H = I.heisenberg_bond()


@pytest.fixture(scope="module")
def S():
    import paper_2502_10298_gb300 as S
    S.load_library()
    return S


def _near_product(Lx, Ly, D, eps, seed):
    rng = np.random.default_rng(seed)
    A0 = np.zeros((Lx, Ly, 2, D, D, D, D))
    A0[:, :, 0, 0, 0, 0, 0] = 0.8
    A0[:, :, 1, 0, 0, 0, 0] = 0.6
    return A0 + eps * rng.standard_normal(A0.shape)


CASES = {
    "1x1_D2_chi8": (lambda: _near_product(1, 1, 2, 0.25, 5), 8, HR),
    "1x1_D3_chi12": (lambda: _near_product(1, 1, 3, 0.2, 3), 12, HR),
    "2x2_D2_chi8": (lambda: _near_product(2, 2, 2, 0.2, 7), 8, H),
    "1x1_D3_chi9_cycle": (lambda: _near_product(1, 1, 3, 0.25, 5), 9, HR),
    "1x1_D2_chi8_random": (lambda: I.random_cell(1, 1, 2, 2, seed=0), 8, H),
    "2x2_D2_chi8_random": (lambda: I.random_cell(2, 2, 2, 2, seed=4), 8, H),
}


@pytest.mark.parametrize("name", list(CASES))
def test_implicit_gradient_matches_oracle(S, name):
    mk, chi, h = CASES[name]
    A = mk()
    Eo, go, info_o = implicit_energy_grad(A, chi, h)
    Lx, Ly, p, D = A.shape[:4]
    with S.SplitCTMRG(Lx, Ly, p, D, chi, precision=0) as s:
        E, g, info = s.energy_grad_implicit(torch.tensor(A, device="cuda"), h)
    assert info["fixed_point_change"] < 1e-9
    assert info["period"] == info_o["period"], (info, info_o)
    assert info["solver_iterations"] < 200
    assert abs(E - Eo) < 1e-10 * abs(Eo), (E, Eo)
    rel = float(np.linalg.norm(g.cpu().numpy() - go.numpy()) / np.linalg.norm(go.numpy()))
    assert rel < 1e-7, rel


def test_implicit_agrees_with_the_checkpointed_gradient(S):
    """At a converged environment the unrolled gradient through 30 steps, whose
    transient has died out, equals the implicit one."""
    A = _near_product(1, 1, 2, 0.25, 5)
    At = torch.tensor(A, device="cuda")
    with S.SplitCTMRG(1, 1, 2, 2, 8, precision=0) as s:
        E, g, _ = s.energy_grad_implicit(At, HR)
        Eu, gu = s.energy_grad(At, 30, HR)
    assert abs(E - Eu) < 1e-12
    assert float((g - gu).norm() / g.norm()) < 1e-9


def test_implicit_refuses_an_environment_that_is_not_a_fixed_point(S):
    """Two sweeps leave the environment far from converged, and the
    conventional scheme's tensors do not settle into a short cycle: both are
    refused with ERR_NOT_FIXED_POINT (the oracle raises for the latter too), and
    the handle stays usable."""
    A = _near_product(1, 1, 2, 0.25, 5)
    At = torch.tensor(A, device="cuda")
    with S.SplitCTMRG(1, 1, 2, 2, 8, precision=0) as s:
        with pytest.raises(S.SctmError) as ei:
            s.energy_grad_implicit(At, HR, max_sweeps=2)
        assert ei.value.code == -7
        e, g = s.energy_grad(At, 2, HR)       # still usable
        assert np.isfinite(e) and torch.isfinite(g).all()
    with pytest.raises(ValueError):
        implicit_energy_grad(A, 8, HR, split=False, max_sweeps=40)
    with S.SplitCTMRG(1, 1, 2, 2, 8, precision=0, algorithm=1) as s:
        with pytest.raises(S.SctmError) as ei:
            s.energy_grad_implicit(At, HR, max_sweeps=40)
        assert ei.value.code == -7
