"""Energy gradient by implicit differentiation of the environment's fixed point.

Test infrastructure only (see ``oracle/__init__``).  The paper iterates full
CTMRG steps until the environment converges (Sec. II.B) and differentiates the
converged energy for its variational optimisation (Sec. I, Sec. III).  Besides
differentiating through the unrolled steps, the derivative of a converged
iteration env* = F(env*, A) follows from the implicit function theorem, the
reverse-mode fixed-point rule:

    dE/dA = dE/dA|_env*  +  x^T dF/dA|_env*,   x = dE/denv*  +  x^T dF/denv|_env*,

where the second equation is solved for x by iterating it from x = dE/denv*; it
converges when F contracts at the fixed point.  The rule needs env* to be a
fixed point of F element by element, not only in gauge-invariant quantities.
With F = f, one full directional step, that holds for near-product states;
elsewhere the signs of the sign-fixed projectors, and with them whole rows of
the environment tensors, still cycle from step to step at converged spectra.
The cycle closes after a few steps (two or four in every case seen), so F is
taken as f applied p times, p the smallest period up to ``max_period`` for which
one application of F changes no entry beyond ``fixed_point_tol``; the function
raises when there is none (the conventional scheme, whose steps do not settle).
The energy is gauge invariant, and any p gives the same gradient.

Every step here is a plain autograd call on the oracle's own functions.
"""
from __future__ import annotations

import torch

from . import ctmrg as C
from . import energy as En


def _keys(split):
    return C.SPLIT_KEYS if split else C.CONV_KEYS


def _flatten(env, split):
    return [e[k] for row in env for e in row for k in _keys(split)]


def _rebuild(flat, Lx, Ly, split):
    keys = _keys(split)
    it = iter(flat)
    return [[{k: next(it) for k in keys} for _ in range(Ly)] for _ in range(Lx)]


def implicit_energy_grad(A, chi, h_nn, h_diag=None, split: bool = True, tol: float = 1e-13,
                         max_sweeps: int = 300, solve_tol: float = 1e-12, max_iter: int = 500,
                         fixed_point_tol: float = 1e-9, max_period: int = 4):
    """Energy per site at the fixed point and its gradient with respect to every
    site tensor (same layout as ``A``, [Lx][Ly] of (p, D, D, D, D)).

    Steps: converge the environment (``ctmrg_run`` to ``tol``); find the smallest
    p <= max_period such that p more steps change no entry by more than
    ``fixed_point_tol`` of the tensor's largest entry (F = p steps); differentiate
    the energy at env*; solve the adjoint fixed-point equation of F to
    ``solve_tol``; add the A-part of F's vjp.
    Returns (E, grad, dict(sweeps=..., period=..., solver_iterations=...))."""
    A = A if isinstance(A, list) else C.as_cell(A)
    Lx, Ly = len(A), len(A[0])
    step = C.split_sweep if split else C.conv_sweep
    A0 = [[a.detach() for a in row] for row in A]
    with torch.no_grad():
        env, n, _ = C.ctmrg_run(A0, chi, tol, max_sweeps, split=split)
        ref = _flatten(env, split)
        nxt, period, changes = env, 0, []
        for q in range(1, max_period + 1):
            nxt = step(A0, nxt, chi)
            worst = max(float((b - a).abs().max() / a.abs().max()) for a, b in zip(ref, _flatten(nxt, split)))
            changes.append(worst)
            if worst <= fixed_point_tol:
                period = q
                break
    if not period:
        raise ValueError("environment is not an element-wise fixed point of up to "
                         f"{max_period} steps (changes {', '.join(f'{c:.1e}' for c in changes)})")
    Al = [[a.detach().clone().requires_grad_(True) for a in row] for row in A]
    Af = [a for row in Al for a in row]
    el = [t.detach().clone().requires_grad_(True) for t in _flatten(env, split)]
    envl = _rebuild(el, Lx, Ly, split)
    E = En.energy_per_site(Al, envl, h_nn, h_diag, split=split)
    g = torch.autograd.grad(E, el + Af, allow_unused=True)
    zero = lambda ts, gs: [torch.zeros_like(t) if v is None else v for t, v in zip(ts, gs)]
    gE_env, gE_A = zero(el, g[:len(el)]), zero(Af, g[len(el):])
    F = envl
    for _ in range(period):
        F = step(Al, F, chi)
    out = _flatten(F, split)
    x = gE_env
    it = 0
    for it in range(1, max_iter + 1):
        Jx = zero(el, torch.autograd.grad(out, el, grad_outputs=x, retain_graph=True, allow_unused=True))
        x_new = [a + b for a, b in zip(gE_env, Jx)]
        num = sum(float((a - b).pow(2).sum()) for a, b in zip(x_new, x)) ** 0.5
        den = sum(float(a.pow(2).sum()) for a in x_new) ** 0.5
        x = x_new
        if num <= solve_tol * den:
            break
    else:
        raise RuntimeError("adjoint fixed-point iteration did not converge")
    gA = zero(Af, torch.autograd.grad(out, Af, grad_outputs=x, allow_unused=True))
    grad = torch.stack([a + b for a, b in zip(gE_A, gA)]).reshape(Lx, Ly, *Af[0].shape)
    return float(E.detach()), grad, dict(sweeps=n, period=period, solver_iterations=it)
