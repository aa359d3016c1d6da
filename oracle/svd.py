"""Full real SVD with a Lorentzian-broadened reverse-mode rule (oracle).

Forward: ``M = U diag(S) V^T`` for a square real matrix, singular values in
descending order (LAPACK via torch.linalg.svd).

Backward (standard real SVD adjoint, written out from the chain rule): with
``J = U^T U_bar`` and ``K = V^T V_bar``,

    M_bar = U [ (F o (J - J^T)) S + diag(S_bar) + S (F o (K - K^T)) ] V^T,

``F_ij = 1/(s_j^2 - s_i^2)`` for i != j, broadened to
``F_ij = d / (d^2 + eps_L * s_max^4)`` with ``d = s_j^2 - s_i^2`` so that
degenerate or zero singular values give a finite result.  ``eps_L`` is taken
relative to ``s_max^4`` because the environment is rescaled every move and the
absolute scale of M is arbitrary.  Lorentzian broadening is not in the paper; it
is the stated backward of the build (eps_L = 1e-36 relative: it only acts on
(near-)degenerate pairs, so gradients through a non-degenerate spectrum are exact).
"""
import torch


class _SVD(torch.autograd.Function):
    @staticmethod
    def forward(ctx, M, eps_l):
        U, S, Vh = torch.linalg.svd(M, full_matrices=True)
        V = Vh.transpose(0, 1).contiguous()
        ctx.save_for_backward(U, S, V)
        ctx.eps_l = eps_l
        return U, S, V

    @staticmethod
    def backward(ctx, gU, gS, gV):
        U, S, V = ctx.saved_tensors
        n = S.shape[0]
        if gU is None:
            gU = torch.zeros_like(U)
        if gS is None:
            gS = torch.zeros_like(S)
        if gV is None:
            gV = torch.zeros_like(V)
        s2 = S * S
        d = s2[None, :] - s2[:, None]                    # d_ij = s_j^2 - s_i^2
        smax4 = (S.max() ** 4) if n > 0 else torch.tensor(0.0, dtype=S.dtype)
        F = d / (d * d + ctx.eps_l * smax4 + 1e-300)
        F.fill_diagonal_(0.0)
        J = U.T @ gU
        K = V.T @ gV
        inner = (F * (J - J.T)) * S[None, :] + torch.diag(gS) + S[:, None] * (F * (K - K.T))
        return U @ inner @ V.T, None


def svd(M: torch.Tensor, eps_l: float = 1e-36):
    """Return (U, S, V) with M = U diag(S) V^T (square M, full U and V)."""
    assert M.dim() == 2 and M.shape[0] == M.shape[1], "oracle SVD expects a square matrix"
    return _SVD.apply(M, eps_l)
