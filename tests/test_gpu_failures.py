"""Failure detection on the GPU without a GPU fault (host-side injection).

Each test lowers one bounded device loop through ``sctm_set_limits`` so that
the loop runs out, checks the error code the call returns, and then checks
that the same handle computes the right result once the limit is restored:
  - the Jacobi sweep limit -> SCTM_ERR_SVD_NOCONV;
  - the main-loop mbarrier wait limit of the tensor-core kernels (3xTF32 and
    BF16 slices) -> SCTM_ERR_CUDA.  A kernel that gives up still waits, with
    its full two-second limit, for the copies and MMAs it issued and frees its
    tensor memory, so the context stays usable.
"""
import numpy as np
import pytest
import torch

import ipeps_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import paper_2502_10298_gb300 as S
    S.load_library()
    return S


def test_jacobi_sweep_limit_reports_no_convergence_and_handle_recovers(S):
    A = torch.tensor(I.random_cell(1, 1, 2, 2, seed=3), device="cuda")
    h = I.heisenberg_bond_rotated()
    with S.SplitCTMRG(1, 1, 2, 2, 8) as ref:
        e0, g0 = ref.energy_grad(A, 2, h)
    with S.SplitCTMRG(1, 1, 2, 2, 8) as s:
        S.sctm_set_limits(s.h, 1, -1.0)
        with pytest.raises(S.SctmError) as ei:
            s.energy_grad(A, 2, h)
        assert ei.value.code == -3
        S.sctm_set_limits(s.h, 0, -1.0)
        e1, g1 = s.energy_grad(A, 2, h)
    # the same call on a fresh handle: equal up to the summation order of the
    # split-K atomics
    assert abs(e1 - e0) <= 1e-12 * abs(e0)
    assert float((g1 - g0).abs().max()) <= 1e-12 * float(g0.abs().max())


@pytest.mark.parametrize("prec", [1, 4])
def test_tensor_core_wait_timeout_reports_error_and_handle_recovers(S, prec):
    rng = np.random.default_rng(9)
    n = 2048
    X = torch.tensor(rng.standard_normal((n, n)), device="cuda")
    Y = torch.tensor(rng.standard_normal((n, n)), device="cuda")
    h = S.sctm_create(1, 1, 2, 2, 8, precision=prec, workspace_bytes=2 << 30)
    try:
        S.sctm_set_limits(h, 0, 0.0)
        with pytest.raises(S.SctmError) as ei:
            S.sctm_einsum(h, "ik,kj->ij", X, Y)
        assert ei.value.code == -2
        S.sctm_set_limits(h, 0, -1.0)
        Z = S.sctm_einsum(h, "ik,kj->ij", X, Y)
        ref = X @ Y
        bound = torch.abs(X) @ torch.abs(Y)
        assert bool(((Z - ref).abs() <= 1e-6 * bound).all())
    finally:
        S.sctm_destroy(h)
