"""Energy per site from a 2x2 patch of the environment (oracle).

Test infrastructure only.  The paper reads local observables off the converged
environment (Sec. III); the build evaluates nearest-neighbour and diagonal bond
terms on a 2x2 patch.  The split environment is first fused into the
conventional one (a ket/bra edge pair contracted over the interlayer bond is the
conventional edge, Sec. II.B), then four enlarged corners are contracted.

Per-site energy (reading): each site (x,y) anchors the patch (x,y),(x,y+1),
(x+1,y),(x+1,y+1); the patch contributes half of each of its four
nearest-neighbour bonds (each lies in two patches) and both diagonals in full:

    E = (1/N) sum_patches [ (e_top + e_bottom + e_left + e_right)/2
                             + e_diag(TL,BR) + e_diag(TR,BL) ]

Each bond value is Tr(rho_ij h)/Tr(rho) with the two-site reduced density matrix
from the patch.  Operators are real (p^2, p^2) matrices indexed
h[(t_i,t_j),(s_i,s_j)] with s the ket and t the bra physical index; the first
site of a bond is the left (horizontal), upper (vertical), TL or TR (diagonals).
"""
from __future__ import annotations

import torch

from .ctmrg import as_cell, fuse, corner_TL, corner_TR, corner_BR, corner_BL, DT

es = torch.einsum


def _patch(envc, A, x, y):
    Lx, Ly = len(A), len(A[0])
    xp, yp = (x + 1) % Lx, (y + 1) % Ly
    TL = corner_TL(envc[x][y], A[x][y], True)
    TR = corner_TR(envc[x][yp], A[x][yp], True)
    BR = corner_BR(envc[xp][yp], A[xp][yp], True)
    BL = corner_BL(envc[xp][y], A[xp][y], True)
    return TL, TR, BR, BL


def _closed(Q):
    return es("abss->ab", Q)


def patch_bond_values(TL, TR, BR, BL, h_nn, h_diag):
    """Bond expectation values of one patch.  Corners carry open (s,t) legs.

    Returns dict with 'norm' and the six bond values (already normalised).
    """
    p = TL.shape[-1]
    hn = torch.as_tensor(h_nn, dtype=DT).reshape(p, p, p, p)   # [t_i,t_j,s_i,s_j]
    hd = None if h_diag is None else torch.as_tensor(h_diag, dtype=DT).reshape(p, p, p, p)
    cTL, cTR, cBR, cBL = _closed(TL), _closed(TR), _closed(BR), _closed(BL)
    # H_top[B_TL, B_TR] = sum_R TL[R,B_TL] TR[R,B_TR]; H_bot[T_BL, T_BR] = sum_L BL[T_BL,L] BR[T_BR,L]
    top_cc = es("ra,rb->ab", cTL, cTR)
    bot_cc = es("al,bl->ab", cBL, cBR)
    norm = (top_cc * bot_cc).sum()

    def val(rdm, hh):
        # sum h[t_i,t_j,s_i,s_j] rdm[s_i,t_i,s_j,t_j] / norm
        return es("TUsv,sTvU->", hh, rdm) / norm

    out = {"norm": norm}
    # top bond (TL, TR)
    top_oo = es("rast,rbuv->astbuv", TL, TR)              # [B_TL, s1, t1, B_TR, s2, t2]
    out["top"] = val(es("astbuv,ab->stuv", top_oo, bot_cc), hn)
    # bottom bond (BL, BR)
    bot_oo = es("alst,bluv->astbuv", BL, BR)
    out["bottom"] = val(es("ab,astbuv->stuv", top_cc, bot_oo), hn)
    # left bond (TL, BL): TL open, BL open, TR, BR closed
    top_oc = es("rast,rb->astb", TL, cTR)
    bot_oc = es("alst,bl->astb", BL, cBR)
    out["left"] = val(es("astb,auvb->stuv", top_oc, bot_oc), hn)
    # right bond (TR, BR)
    top_co = es("ra,rbst->abst", cTL, TR)
    bot_co = es("al,blst->abst", cBL, BR)
    out["right"] = val(es("abst,abuv->stuv", top_co, bot_co), hn)
    if hd is not None:
        # diagonal TL-BR and TR-BL
        out["diag1"] = val(es("astb,abuv->stuv", top_oc, bot_co), hd)
        out["diag2"] = val(es("abst,auvb->stuv", top_co, bot_oc), hd)
    return out


def energy_per_site(A, env, h_nn, h_diag=None, split: bool = True, return_bonds=False):
    """Energy per site (see module docstring).  ``env`` is split unless split=False."""
    A = A if isinstance(A, list) else as_cell(A)
    envc = fuse(env) if split else env
    Lx, Ly = len(A), len(A[0])
    total = torch.zeros((), dtype=DT)
    bonds = {}
    for x in range(Lx):
        for y in range(Ly):
            TL, TR, BR, BL = _patch(envc, A, x, y)
            v = patch_bond_values(TL, TR, BR, BL, h_nn, h_diag)
            bonds[(x, y)] = v
            e = 0.5 * (v["top"] + v["bottom"] + v["left"] + v["right"])
            if h_diag is not None:
                e = e + v["diag1"] + v["diag2"]
            total = total + e
    E = total / (Lx * Ly)
    return (E, bonds) if return_bonds else E
