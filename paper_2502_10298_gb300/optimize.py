"""Variational optimisation of an iPEPS unit cell with L-BFGS over the engine's
energy and gradient (the outer loop of Sec. III: every optimisation step needs
the CTMRG contraction and the energy gradient at least once).

The host only holds the optimiser state; every energy and gradient comes from
one ``energy_grad`` call of the C-ABI on the device buffers of the unit cell.
"""
from __future__ import annotations

import time

import torch

from .api import SplitCTMRG

__all__ = ["lbfgs"]


def lbfgs(A0: torch.Tensor, chi: int, sweeps: int, h_nn, h_diag=None, evaluations: int = 10,
          history: int = 10, lr: float = 1.0, **engine_kw):
    """Minimise the energy per site over the unit cell A0 ([Lx, Ly, p, D, D, D,
    D], CUDA float64) with L-BFGS (strong-Wolfe line search), stopping after
    ``evaluations`` energy+gradient evaluations.  engine_kw go to SplitCTMRG
    (precision, svd_cutoff, ...).  Returns (A, trace) with trace a list of
    dicts (evaluation, energy, gradient norm, seconds since the start)."""
    Lx, Ly, p, D = A0.shape[:4]
    A = A0.detach().clone().contiguous()
    A.requires_grad_(True)
    opt = torch.optim.LBFGS([A], lr=lr, max_iter=evaluations, max_eval=evaluations, history_size=history,
                            tolerance_grad=0.0, tolerance_change=0.0, line_search_fn="strong_wolfe")
    trace = []
    t0 = time.perf_counter()
    with SplitCTMRG(Lx, Ly, p, D, chi, **engine_kw) as s:

        def closure():
            opt.zero_grad()
            e, g = s.energy_grad(A.detach().contiguous(), sweeps, h_nn, h_diag)
            A.grad = g
            trace.append({"evaluation": len(trace) + 1, "energy": e, "grad_norm": float(g.norm()),
                          "seconds": time.perf_counter() - t0})
            return torch.tensor(e, dtype=torch.float64)

        opt.step(closure)
    return A.detach(), trace
