"""Mixed precision against the FP64 oracle where the benched machinery runs.

Spec tolerances for the mixed forms: energy within 1e-6 per site and
gradient within 1e-4 in norm of the FP64 oracle's.  Both cases are large
enough for the tensor-core contraction (its launch is asserted through the
engine's per-family profile) and for the randomized projectors, which take
truncated spaces of at least four sketch widths: the yellow and red ones at
D=4, chi=64 (512 against a sketch of 128) and the red ones at D=4, chi=32
(256 against 64).  The projector cutoff is the mixed default, 1e-5, on both
sides.
"""
import numpy as np
import pytest
import torch

import ipeps_inputs as I
from oracle import ctmrg as C
from oracle import energy as En

pytestmark = pytest.mark.gpu

CUTOFF = 1e-5


@pytest.fixture(scope="module")
def S():
    import paper_2502_10298_gb300 as S
    S.load_library()
    return S


def _near(D, eps, seed):
    rng = np.random.default_rng(seed)
    A0 = np.zeros((1, 1, 2, D, D, D, D))
    A0[:, :, 0, 0, 0, 0, 0] = 0.8
    A0[:, :, 1, 0, 0, 0, 0] = 0.6
    return A0 + eps * rng.standard_normal(A0.shape)


def _case(name):
    if name == "d4_chi64_1x1":        # near-product 1x1 state, rotated Heisenberg
        return _near(4, 0.3, 5), 64, 2, I.heisenberg_bond_rotated()
    A, c = I.config("d4_chi32_2x2")   # the 2x2, D=4, chi=32 workload: random tensors, Heisenberg J=1
    return A, c["chi"], 2, I.heisenberg_bond()


@pytest.fixture(scope="module")
def oracle_refs():
    cache = {}

    def get(name):
        if name not in cache:
            A, chi, sweeps, h = _case(name)
            old = C.CUTOFF
            C.CUTOFF = CUTOFF
            try:
                Ao = torch.tensor(A).requires_grad_(True)
                Lx, Ly = A.shape[:2]
                Ac = [[Ao[x, y] for y in range(Ly)] for x in range(Lx)]
                e = En.energy_per_site(Ac, C.split_ctmrg(Ac, chi, sweeps), h, None)
                e.backward()
            finally:
                C.CUTOFF = old
            cache[name] = (float(e.detach()), Ao.grad.numpy().copy())
        return cache[name]
    return get


@pytest.mark.parametrize("name", ["d4_chi32_2x2", "d4_chi64_1x1"])
@pytest.mark.parametrize("prec", [4])
def test_mixed_energy_and_gradient_match_oracle(S, oracle_refs, name, prec):
    A, chi, sweeps, h = _case(name)
    Lx, Ly, p, D = A.shape[:4]
    with S.SplitCTMRG(Lx, Ly, p, D, chi, precision=prec, svd_cutoff=CUTOFF) as s:
        S.sctm_profile(s.h, True)
        e, g = s.energy_grad(torch.tensor(A, device="cuda"), sweeps, h, None)
        fam = S.sctm_profile(s.h, False)
    assert fam["tensor"]["launches"] > 0
    eo, go = oracle_refs(name)
    assert abs(e - eo) < 1e-6, (e, eo)
    rel = float(np.linalg.norm(g.cpu().numpy() - go) / np.linalg.norm(go))
    assert rel < 1e-4, rel
