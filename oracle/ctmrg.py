"""Split-CTMRG and conventional CTMRG, plain FP64 CPU reference (oracle).

Test infrastructure only (see ``oracle/__init__``).  Follows Naumann et al.,
"Variationally optimizing infinite PEPS at large bond dimensions: a split CTMRG
approach" (arXiv 2502.10298):

* environment definition: Fig. 2 (Sec. II.B); contracting a ket/bra edge pair
  over the interlayer bond gives the conventional edge tensor (Sec. II.B);
* left move, corners: Eqs. (splitCTMRG_C1), (splitCTMRG_C4);
* left move, edges: Eqs. (splitCTMRG_Tket), (splitCTMRG_Tbra);
* projectors: Fig. 3 and the equations for M, M~ and the resolution of the
  identity in Sec. II.B; yellow: Fig. 8 (App. A); teal and red: App. A
  (Figs. 7, 9 -- network figures missing, reading below);
* conventional CTMRG for comparison: Fig. 1 with the 2x2-patch projectors of
  Corboz et al. that the paper uses as its benchmark (Sec. III).

Leg order (the paper only draws diagrams; this order is shared by every file):

    A[s,u,l,d,r]                 ket; the bra is A itself (real tensors)
    C1[a,b]    a->T1k  b->T4k    T1k[a,u,i]  T1b[i,u',c]    C2[c,f]
    T2k[f,r,j] T2b[j,r',g]       C3[g,h]     T3b[h,d',k]    T3k[k,d,m]
    C4[m,n]    T4b[n,l',q]       T4k[q,l,b]

i.e. every tensor is [previous, PEPS leg, next] along the clockwise chain
C1 T1k T1b C2 T2k T2b C3 T3b T3k C4 T4b T4k.  Environment tensors are stored per
site ``env[x][y]`` (x row, y column); the left move writes column y+1 from column y.

Readings where the paper is silent (shared with the CUDA path):

* initial environment: double-layer corners/edges of the neighbouring A, edges
  split into ket/bra halves by an SVD truncated to chi_I;
* bond dimensions: ``chi`` is chi_E = chi_I or a pair (chi_E, chi_I); green and
  teal truncate to chi_E, yellow and red to chi_I (``chi_pair``);
* projector: keep min(chi, n) singular values, s^{-1/2} -> 0 for s < 1e-8 s_max
  (a smaller cutoff keeps directions amplified by s^{-1/2} > 1e4 and makes the
  map numerically non-differentiable);
  sign of each kept triplet fixed so the largest-|.| entry of the P_up row is > 0;
* teal / red rho networks (figures missing): upper / lower halves of the 2x2
  patch (columns y and y+1, as for the conventional projectors) with the
  ket-stage projectors of column y inside -- the "full" teal of App. B, whose
  cost with the QR pre-reduction is the O(chi_E^3 chi_B^4) the paper states;
  a one-column half leaves only the right-environment bond open, caps the bond
  dimension at its initial value and was measured to be biased;
* right/bottom moves: left/top moves after a 180 degree rotation with ket and bra
  relabelled (valid for real A), so they absorb the bra layer first;
* each new environment tensor is divided by its max |entry| after every move.
"""
from __future__ import annotations

import torch

from .svd import svd as _svd

DT = torch.float64
SPLIT_KEYS = ("C1", "T1k", "T1b", "C2", "T2k", "T2b", "C3", "T3b", "T3k", "C4", "T4b", "T4k")
CONV_KEYS = ("C1", "T1", "C2", "T2", "C3", "T3", "C4", "T4")
CUTOFF = 1e-8
EPS_L = 1e-36
es = torch.einsum


def chi_pair(chi):
    """(chi_E, chi_I): environment and interlayer bond dimensions.  An int sets
    both (chi_E = chi_I, the paper's default); a pair sets them separately
    (Sec. II.B: the split edges carry chi_E on their environment legs and chi_I
    on the bond between the ket and the bra edge)."""
    if isinstance(chi, (tuple, list)):
        return int(chi[0]), int(chi[1])
    return int(chi), int(chi)


# ----------------------------------------------------------------------- utils
def as_cell(A) -> list:
    """[Lx,Ly,p,D,D,D,D] array/tensor -> nested list of float64 tensors A[x][y]."""
    A = torch.as_tensor(A, dtype=DT)
    return [[A[x, y] for y in range(A.shape[1])] for x in range(A.shape[0])]


def rescale(t: torch.Tensor) -> torch.Tensor:
    """Divide by max |entry| (build reading: done after every move)."""
    m = t.detach().abs().max()
    if m == 0:
        return t
    return t / t.abs().max()


def projector_pair(rhoT: torch.Tensor, rhoB: torch.Tensor, chi: int,
                   cutoff: float = None, eps_l: float = EPS_L):
    """Projector pair from two half networks (Sec. II.B, Fig. 3).

    rhoT: (alpha, beta) upper half, rhoB: (beta, alpha) lower half, alpha being
    the wires to truncate.  M = rhoB rhoT = U S V^T; with the chi largest
    singular values,  P_up = S~^{-1/2} U~^T rhoB  (k x alpha, applied above the
    cut) and  P_dn = rhoT V~ S~^{-1/2}  (alpha x k, applied below), so that
    P_dn P_up ~ 1 on alpha and P_up P_dn = 1 on the kept space.

    When alpha < beta, M has rank <= alpha and both halves are first reduced by
    a QR decomposition (App. A: decompose rho^T and rho^B before multiplying):
    rhoT^T = Q_T R_T, rhoB = Q_B R_B, K = R_B R_T^T = U' S V'^T; then
    P_up = S^{-1/2} U'^T R_B and P_dn = R_T^T V' S^{-1/2}, which equals the
    unreduced formula because U = Q_B U', V = Q_T V'.  The reduction is used
    for values only: when a gradient is being recorded the projectors are
    formed from M = rhoB rhoT itself (Sec. II.B), because the reverse rule of
    QR divides by the pivots of R and is undefined when a half is
    rank-deficient (a truncated environment usually makes it so).
    ``cutoff`` defaults to the module's CUTOFF at call time.
    Returns (P_up, P_dn, s_kept).
    """
    cutoff = CUTOFF if cutoff is None else cutoff
    na, nb = rhoT.shape
    taped = torch.is_grad_enabled() and (rhoT.requires_grad or rhoB.requires_grad)
    if na < nb and not taped:
        _, RT = torch.linalg.qr(rhoT.T, mode="reduced")      # (alpha, alpha)
        _, RB = torch.linalg.qr(rhoB, mode="reduced")        # (alpha, alpha)
        left, right = RB, RT.T                               # K = RB @ RT^T
    else:
        left, right = rhoB, rhoT
    M = left @ right
    U, S, V = _svd(M, eps_l)
    k = min(chi, S.shape[0])
    U, S, V = U[:, :k], S[:k], V[:, :k]
    smax = S.detach()[0] if k > 0 else torch.tensor(0.0, dtype=DT)
    keep = S.detach() > cutoff * smax
    S_safe = torch.where(keep, S, torch.ones_like(S))
    sinv = torch.where(keep, S_safe.rsqrt(), torch.zeros_like(S))
    P_up = sinv[:, None] * (U.T @ left)
    P_dn = (right @ V) * sinv[None, :]
    with torch.no_grad():
        if k > 0:
            idx = P_up.abs().argmax(dim=1)
            sgn = torch.sign(P_up[torch.arange(k), idx])
            sgn[sgn == 0] = 1.0
        else:
            sgn = torch.ones(0, dtype=DT)
    return P_up * sgn[:, None], P_dn * sgn[None, :], S


# ------------------------------------------------------- initial environment
def _double_layer_pieces(A):
    """Double-layer corners and edges of one tensor (outward legs traced).

    Orders follow the conventional environment: C1[(r,r'),(d,d')],
    T1[(l,l'),d,d',(r,r')], C2[(l,l'),(d,d')], T2[(u,u'),l,l',(d,d')],
    C3[(u,u'),(l,l')], T3[(r,r'),u',u,(l,l')], C4[(r,r'),(u,u')],
    T4[(d,d'),r',r,(u,u')]; primed legs belong to the bra copy.
    """
    D = A.shape[1]
    D2 = D * D
    c1 = es("suldr,sulez->rzde", A, A).reshape(D2, D2)
    t1 = es("suldr,suvez->lvderz", A, A).reshape(D2, D, D, D2)
    c2 = es("suldr,suver->lvde", A, A).reshape(D2, D2)
    t2 = es("suldr,swver->uwlvde", A, A).reshape(D2, D, D, D2)
    c3 = es("suldr,swvdr->uwlv", A, A).reshape(D2, D2)
    t3 = es("suldr,swvdz->rzwulv", A, A).reshape(D2, D, D, D2)
    c4 = es("suldr,swldz->rzuw", A, A).reshape(D2, D2)
    t4 = es("suldr,swlez->dezruw", A, A).reshape(D2, D, D, D2)
    return c1, t1, c2, t2, c3, t3, c4, t4


def _split_edge(T: torch.Tensor, chi: int, cutoff: float = None):
    """Split a conventional edge T[p, k, k', n] into first[p,k,i] second[i,k',n].

    SVD of the matrix (p,k) x (k',n), truncated to chi and the cutoff;
    first = U sqrt(S), second = sqrt(S) V^T, sign fixed so the largest-|.|
    entry of every column of U is positive.  The first factor is the tensor that
    comes first along the clockwise chain.
    """
    cutoff = CUTOFF if cutoff is None else cutoff
    P, K, K2, N = T.shape
    Mt = T.reshape(P * K, K2 * N)
    U, S, Vh = torch.linalg.svd(Mt, full_matrices=False)
    k = min(chi, S.shape[0])
    U, S, Vh = U[:, :k], S[:k], Vh[:k]
    keep = S > cutoff * S[0]
    sq = torch.where(keep, S.clamp_min(0).sqrt(), torch.zeros_like(S))
    idx = U.abs().argmax(dim=0)
    sgn = torch.sign(U[idx, torch.arange(k)])
    sgn[sgn == 0] = 1.0
    U = U * sgn[None, :]
    Vh = Vh * sgn[:, None]
    first = (U * sq[None, :]).reshape(P, K, k)
    second = (sq[:, None] * Vh).reshape(k, K2, N)
    return first, second


def initial_env(A, chi: int, split: bool = True):
    """Environment built from the neighbours' own layer contractions.

    Site (x,y): C1 from A[x-1,y-1], T1 from A[x-1,y], C2 from A[x-1,y+1],
    T2 from A[x,y+1], C3 from A[x+1,y+1], T3 from A[x+1,y], C4 from A[x+1,y-1],
    T4 from A[x,y-1] (double layer, outward legs traced).  With split=True each
    edge is split into its ket and bra halves (chain order) by ``_split_edge``.
    """
    A = A if isinstance(A, list) else as_cell(A)
    Lx, Ly = len(A), len(A[0])
    pieces = [[_double_layer_pieces(A[x][y]) for y in range(Ly)] for x in range(Lx)]
    env = [[None] * Ly for _ in range(Lx)]
    for x in range(Lx):
        for y in range(Ly):
            xm, xp, ym, yp = (x - 1) % Lx, (x + 1) % Lx, (y - 1) % Ly, (y + 1) % Ly
            C1 = pieces[xm][ym][0]
            T1 = pieces[xm][y][1]
            C2 = pieces[xm][yp][2]
            T2 = pieces[x][yp][3]
            C3 = pieces[xp][yp][4]
            T3 = pieces[xp][y][5]
            C4 = pieces[xp][ym][6]
            T4 = pieces[x][ym][7]
            if not split:
                env[x][y] = dict(C1=C1, T1=T1, C2=C2, T2=T2, C3=C3, T3=T3, C4=C4, T4=T4)
                continue
            chi_i = chi_pair(chi)[1]   # the split cuts the interlayer bond
            T1k, T1b = _split_edge(T1, chi_i)
            T2k, T2b = _split_edge(T2, chi_i)
            T3b, T3k = _split_edge(T3, chi_i)
            T4b, T4k = _split_edge(T4, chi_i)
            env[x][y] = dict(C1=C1, T1k=T1k, T1b=T1b, C2=C2, T2k=T2k, T2b=T2b,
                             C3=C3, T3b=T3b, T3k=T3k, C4=C4, T4b=T4b, T4k=T4k)
    return env


def fuse(env):
    """Split environment -> conventional one by contracting each ket/bra pair
    over the interlayer bond (Sec. II.B)."""
    out = []
    for row in env:
        r = []
        for e in row:
            r.append(dict(
                C1=e["C1"], C2=e["C2"], C3=e["C3"], C4=e["C4"],
                T1=es("aui,iwc->auwc", e["T1k"], e["T1b"]),
                T2=es("frj,jzg->frzg", e["T2k"], e["T2b"]),
                T3=es("hek,kdm->hedm", e["T3b"], e["T3k"]),
                T4=es("nvq,qlb->nvlb", e["T4b"], e["T4k"]),
            ))
        out.append(r)
    return out


# ----------------------------------------------------------------------- frames
def _tp(t):
    return t.permute(*reversed(range(t.dim())))


def transpose_frame(A, env, split: bool = True):
    """Reflect the lattice about its main diagonal: (x,y) -> (y,x), up<->left,
    down<->right.  The ket stays up-left of the bra, so a left move in the new
    frame is a top move in the old one.  Every tensor is index-reversed and
    swapped with its partner (C2<->C4, T1<->T4, T2<->T3)."""
    Lx, Ly = len(A), len(A[0])
    A2 = [[A[x][y].permute(0, 2, 1, 4, 3) for x in range(Lx)] for y in range(Ly)]
    env2 = [[None] * Lx for _ in range(Ly)]
    for x in range(Lx):
        for y in range(Ly):
            e = env[x][y]
            if split:
                n = dict(C1=_tp(e["C1"]), T1k=_tp(e["T4k"]), T1b=_tp(e["T4b"]), C2=_tp(e["C4"]),
                         T2k=_tp(e["T3k"]), T2b=_tp(e["T3b"]), C3=_tp(e["C3"]), T3b=_tp(e["T2b"]),
                         T3k=_tp(e["T2k"]), C4=_tp(e["C2"]), T4b=_tp(e["T1b"]), T4k=_tp(e["T1k"]))
            else:
                n = dict(C1=_tp(e["C1"]), T1=_tp(e["T4"]), C2=_tp(e["C4"]), T2=_tp(e["T3"]),
                         C3=_tp(e["C3"]), T3=_tp(e["T2"]), C4=_tp(e["C2"]), T4=_tp(e["T1"]))
            env2[y][x] = n
    return A2, env2


def rot180_frame(A, env, split: bool = True):
    """Rotate the lattice by 180 degrees, (x,y) -> (-x,-y) mod cell, and relabel
    ket <-> bra (the norm network is symmetric under exchanging the layers for
    real A).  Edges keep their index order (T1k<->T3b, T1b<->T3k, T2k<->T4b,
    T2b<->T4k) and C2<->C4 too; C1 is stored [next, previous] along the chain
    while C3 is [previous, next], so C1<->C3 come with a transpose."""
    Lx, Ly = len(A), len(A[0])
    A2 = [[None] * Ly for _ in range(Lx)]
    env2 = [[None] * Ly for _ in range(Lx)]
    for x in range(Lx):
        for y in range(Ly):
            xn, yn = (-x) % Lx, (-y) % Ly
            A2[xn][yn] = A[x][y].permute(0, 3, 4, 1, 2)
            e = env[x][y]
            if split:
                n = dict(C1=_tp(e["C3"]), T1k=e["T3b"], T1b=e["T3k"], C2=e["C4"], T2k=e["T4b"],
                         T2b=e["T4k"], C3=_tp(e["C1"]), T3b=e["T1k"], T3k=e["T1b"], C4=e["C2"],
                         T4b=e["T2k"], T4k=e["T2b"])
            else:
                n = dict(C1=_tp(e["C3"]), T1=e["T3"], C2=e["C4"], T2=e["T4"], C3=_tp(e["C1"]),
                         T3=e["T1"], C4=e["C2"], T4=e["T2"])
            env2[xn][yn] = n
    return A2, env2


def in_frame(direction: int, fn, A, env, split: bool = True):
    """Run ``fn(A', env')`` (a left move) in the frame where ``direction`` is the
    left direction, and map the environment back.  0 left, 1 top, 2 right, 3 bottom."""
    if direction == 0:
        return fn(A, env)
    if direction == 1:
        A2, e2 = transpose_frame(A, env, split)
        out = fn(A2, e2)
        return transpose_frame(A2, out, split)[1]
    if direction == 2:
        A2, e2 = rot180_frame(A, env, split)
        out = fn(A2, e2)
        return rot180_frame(A2, out, split)[1]
    if direction == 3:
        A2, e2 = rot180_frame(A, env, split)
        A3, e3 = transpose_frame(A2, e2, split)
        out = fn(A3, e3)
        _, b2 = transpose_frame(A3, out, split)
        return rot180_frame(A2, b2, split)[1]
    raise ValueError("direction must be 0..3")


# --------------------------------------------------- split-CTMRG rho networks
def green_rhoT(E, A):
    """rho^T_green (Fig. 3a, upper box): everything of the site's norm network
    above the cut under its bra row.  Open (T4b.n, A.d | A'.d', T2b.g);
    returned as a matrix (alpha=(n, d)) x (beta=(d', g))."""
    X = es("ab,aui->bui", E["C1"], E["T1k"])
    X = es("bui,qlb->uiql", X, E["T4k"])
    X = es("uiql,sulkr->iqskr", X, A)
    X = es("iqskr,iwc->qskrwc", X, E["T1b"])
    X = es("qskrwc,cf->qskrwf", X, E["C2"])
    X = es("qskrwf,frj->qskwj", X, E["T2k"])
    X = es("qskwj,nvq->skwjnv", X, E["T4b"])
    X = es("skwjnv,swvez->kjnez", X, A)
    R = es("kjnez,jzg->nkeg", X, E["T2b"])
    n, k, e, g = R.shape
    return R.reshape(n * k, e * g)


def green_rhoB(E, A):
    """rho^B_green (Fig. 3a, lower box) of the site below the cut.  Open
    (T4k.b, A.u | A'.u', T2k.f); returned as (beta=(u', f)) x (alpha=(b, u))."""
    Y = es("mn,kdm->nkd", E["C4"], E["T3k"])
    Y = es("nkd,nvq->kdvq", Y, E["T4b"])
    Y = es("kdvq,hek->dvqhe", Y, E["T3b"])
    Y = es("dvqhe,gh->dvqeg", Y, E["C3"])
    Y = es("dvqeg,jzg->dvqejz", Y, E["T2b"])
    Y = es("dvqejz,swvez->dqjsw", Y, A)
    Y = es("dqjsw,qlb->djswlb", Y, E["T4k"])
    Y = es("djswlb,suldr->jwbur", Y, A)
    R = es("jwbur,frj->wfbu", Y, E["T2k"])
    w, f, b, u = R.shape
    return R.reshape(w * f, b * u)


def yellow_rhoT(E, A):
    """rho^T_yellow (Fig. 8, upper box): C1 T1k T1b C2 T2k T4k A.  Open
    (T4k.q, A.d | A.s, T1b.u', T2k.j) -> (alpha=(q, d)) x (beta=(s, u', j))."""
    X = es("ab,aui->bui", E["C1"], E["T1k"])
    X = es("bui,qlb->uiql", X, E["T4k"])
    X = es("uiql,sulkr->iqskr", X, A)
    X = es("iqskr,iwc->qskrwc", X, E["T1b"])
    X = es("qskrwc,cf->qskrwf", X, E["C2"])
    R = es("qskrwf,frj->qkswj", X, E["T2k"])
    q, k, s, w, j = R.shape
    return R.reshape(q * k, s * w * j)


def yellow_rhoB(E, A):
    """rho^B_yellow (Fig. 8, lower box): T4b A' T2b C3 T3b T3k C4.  Open
    (T4b.q, T3k.d | A'.s, A'.u', T2b.j) -> (beta=(s, u', j)) x (alpha=(q, d))."""
    Y = es("mn,kdm->nkd", E["C4"], E["T3k"])
    Y = es("nkd,nvq->kdvq", Y, E["T4b"])
    Y = es("kdvq,hek->dvqhe", Y, E["T3b"])
    Y = es("dvqhe,gh->dvqeg", Y, E["C3"])
    Y = es("dvqeg,jzg->dvqejz", Y, E["T2b"])
    Y = es("dvqejz,swvez->dqjsw", Y, A)
    R = es("dqjsw->swjqd", Y)
    s, w, j, q, d = R.shape
    return R.reshape(s * w * j, q * d)


def _upper_left_k(E, A, K):
    """Column y of the upper half after the ket stage: C1k T1b T4k_k T4b_k A'.
    Legs [r, c, t, e, z]: right (c = T1b.c, r = A.r, z = A'.r'), bottom (t, e = A'.d').
    The ket's physical leg s is open on T4k_k (standard order) or on T4b_k
    (alternative order, where yellow truncated it)."""
    if K["T4kk"].dim() == 3:                                   # alternative order
        X = es("ig,gry->iry", K["C1k"], K["T4kk"])
        X = es("iry,iwc->rywc", X, E["T1b"])
        X = es("rywc,yvts->rwcvts", X, K["T4bk"])
        return es("rwcvts,swvez->rctez", X, A)
    X = es("ig,grys->irys", K["C1k"], K["T4kk"])
    X = es("irys,iwc->ryswc", X, E["T1b"])
    X = es("ryswc,yvt->rswcvt", X, K["T4bk"])
    return es("rswcvt,swvez->rctez", X, A)


def _upper_right(E2, A2):
    """Column y+1 of the upper half: T1k T1b C2 T2k T2b A A' of site (x, y+1).
    Legs [c, l, v, D, E, g]: left (c = T1k.a, l = A.l, v = A'.l'), bottom
    (D = A.d, E = A'.d', g = T2b.g)."""
    Y = es("cui,iwC->cuwC", E2["T1k"], E2["T1b"])
    Y = es("cuwC,Cf->cuwf", Y, E2["C2"])
    Y = es("cuwf,fRj->cuwRj", Y, E2["T2k"])
    Y = es("cuwRj,jZg->cuwRZg", Y, E2["T2b"])
    Y = es("cuwRZg,SulDR->cwZgSlD", Y, A2)
    return es("cwZgSlD,SwvEZ->clvDEg", Y, A2)


def _lower_left_k(E, A, K):
    """Column y of the lower half after the ket stage: T4k_k T4b_k C4k A' T3b.
    Legs [h, w, z, g, r]: top (g = T4k_k.g, w = A'.u'), right (r, z, h = T3b.h)."""
    Z = es("tk,hek->the", K["C4k"], E["T3b"])
    if K["T4kk"].dim() == 3:                                   # alternative order
        Z = es("the,yvts->heyvs", Z, K["T4bk"])
        Z = es("heyvs,swvez->hywz", Z, A)
        return es("hywz,gry->hwzgr", Z, K["T4kk"])
    Z = es("the,yvt->heyv", Z, K["T4bk"])
    Z = es("heyv,swvez->hyswz", Z, A)
    return es("hyswz,grys->hwzgr", Z, K["T4kk"])


def _lower_right(E2, A2):
    """Column y+1 of the lower half: T2k T2b C3 T3b T3k A A' of site (x+1, y+1).
    Legs [U, W, f, h, l, v]: top (U = A.u, W = A'.u', f = T2k.f), left
    (h = T3k.m, l = A.l, v = A'.l')."""
    W = es("fRj,jZG->fRZG", E2["T2k"], E2["T2b"])
    W = es("fRZG,GH->fRZH", W, E2["C3"])
    W = es("fRZH,HEK->fRZEK", W, E2["T3b"])
    W = es("fRZEK,KDh->fRZEDh", W, E2["T3k"])
    W = es("fRZEDh,SUlDR->fZEhSUl", W, A2)
    return es("fZEhSUl,SWvEZ->UWfhlv", W, A2)


def teal_rhoT(E, A, K, E2, A2):
    """rho^T_teal (reading, App. A / Fig. 7 figure missing): upper half of the
    2x2 patch (columns y, y+1) with the ket-stage projectors of column y inside.
    Open (T4b_k.t, A'.d' | A.d, A'.d', T2b.g of column y+1)."""
    R = es("rctez,crzDEg->teDEg", _upper_left_k(E, A, K), _upper_right(E2, A2))
    t, e, D, E_, g = R.shape
    return R.reshape(t * e, D * E_ * g)


def teal_rhoB(E, A, K, E2, A2):
    """rho^B_teal (reading): lower half of the 2x2 patch.  Open
    (A.u, A'.u', T2k.f of column y+1) x (T4k_k.g, A'.u' of column y)."""
    R = es("UWfhlv,hwvgl->UWfgw", _lower_right(E2, A2), _lower_left_k(E, A, K))
    U, W, f, g, w = R.shape
    return R.reshape(U * W * f, g * w)


def red_rhoT(E, K, E2, A2):
    """rho^T_red (reading, App. A / Fig. 9 figure missing): ket rows of columns
    y (after the ket stage) and y+1.  Open (T4k_k.y, T4k_k.s, T1b.u' |
    A.d, A.s, T1b.u', T2k.j of column y+1)."""
    X = es("ig,grys->irys", K["C1k"], K["T4kk"])
    X = es("irys,iwc->ryswc", X, E["T1b"])
    Y = es("cui,iWC->cuWC", E2["T1k"], E2["T1b"])
    Y = es("cuWC,Cf->cuWf", Y, E2["C2"])
    Y = es("cuWf,fRj->cuWRj", Y, E2["T2k"])
    Y = es("cuWRj,SulDR->cWjSlD", Y, A2)
    R = es("ryswc,cWjSrD->yswDSWj", X, Y)
    y, s, w, D, S, W, j = R.shape
    return R.reshape(y * s * w, D * S * W * j)


def red_rhoB(E, A, K, E2, A2):
    """rho^B_red (reading): bra rows of columns y (after the ket stage) and y+1.
    Open (T3k.d, A'.s, A'.u', T2b.j of column y+1) x (T4b_k.y, A'.s, A'.u')."""
    Z = es("tk,hek->the", K["C4k"], E["T3b"])
    Z = es("the,yvt->heyv", Z, K["T4bk"])
    Z = es("heyv,swvez->hyswz", Z, A)
    W = es("jZG,GH->jZH", E2["T2b"], E2["C3"])
    W = es("jZH,HEK->jZEK", W, E2["T3b"])
    W = es("jZEK,KDh->jZEDh", W, E2["T3k"])
    W = es("jZEDh,SWvEZ->jDhSWv", W, A2)
    R = es("jDhSWv,hyswv->DSWjysw", W, Z)
    D, S, W_, j, y, s, w = R.shape
    return R.reshape(D * S * W_ * j, y * s * w)


# ------------------------------ alternative yellow/red order (App. B)
# App. B proposes to absorb the ket's physical leg into the yellow projectors
# instead of the red ones, which removes the p^3 factor of the red SVD:
# yellow then truncates (T4ket.q, A.d, A.s) -> chi_I on the same networks as
# Fig. 8 with the physical leg moved to the truncated side, and red truncates
# (yellow chi_I, T1bra.u') -> chi_I.  After the ket stage T4ket_k[g, r, y] has
# no physical leg and T4bra_k[y, l', g2, s] carries it to the bra layer, which
# closes it when the bra is absorbed.

def yellow_alt_rhoT(E, A):
    """rho^T_yellow of the alternative order: the network of yellow_rhoT with
    open (T4k.q, A.d, A.s | T1b.u', T2k.j) -> (alpha=(q, d, s)) x (beta=(u', j))."""
    X = es("ab,aui->bui", E["C1"], E["T1k"])
    X = es("bui,qlb->uiql", X, E["T4k"])
    X = es("uiql,sulkr->iqskr", X, A)
    X = es("iqskr,iwc->qskrwc", X, E["T1b"])
    X = es("qskrwc,cf->qskrwf", X, E["C2"])
    R = es("qskrwf,frj->qkswj", X, E["T2k"])
    q, k, s_, w, j = R.shape
    return R.reshape(q * k * s_, w * j)


def yellow_alt_rhoB(E, A):
    """rho^B_yellow of the alternative order: the network of yellow_rhoB with
    open (A'.u', T2b.j | T4b.q, T3k.d, A'.s) -> (beta=(u', j)) x (alpha=(q, d, s))."""
    Y = es("mn,kdm->nkd", E["C4"], E["T3k"])
    Y = es("nkd,nvq->kdvq", Y, E["T4b"])
    Y = es("kdvq,hek->dvqhe", Y, E["T3b"])
    Y = es("dvqhe,gh->dvqeg", Y, E["C3"])
    Y = es("dvqeg,jzg->dvqejz", Y, E["T2b"])
    Y = es("dvqejz,swvez->dqjsw", Y, A)
    R = es("dqjsw->wjqds", Y)
    w, j, q, d, s_ = R.shape
    return R.reshape(w * j, q * d * s_)


def red_alt_rhoT(E, K, E2, A2):
    """rho^T_red of the alternative order (two-column reading, as red_rhoT):
    open (T4k_k.y, T1b.u' | A.d, A.s, T1b.u', T2k.j of column y+1)."""
    X = es("ig,gry->iry", K["C1k"], K["T4kk"])
    X = es("iry,iwc->rywc", X, E["T1b"])
    Y = es("cui,iWC->cuWC", E2["T1k"], E2["T1b"])
    Y = es("cuWC,Cf->cuWf", Y, E2["C2"])
    Y = es("cuWf,fRj->cuWRj", Y, E2["T2k"])
    Y = es("cuWRj,SulDR->cWjSlD", Y, A2)
    R = es("rywc,cWjSrD->ywDSWj", X, Y)
    y, w, D, S, W, j = R.shape
    return R.reshape(y * w, D * S * W * j)


def red_alt_rhoB(E, A, K, E2, A2):
    """rho^B_red of the alternative order: open (T3k.d, A'.s, A'.u', T2b.j of
    column y+1) x (T4b_k.y, A'.u'); the bra closes the physical leg of T4b_k."""
    Z = es("tk,hek->the", K["C4k"], E["T3b"])
    Z = es("the,yvts->heyvs", Z, K["T4bk"])
    Z = es("heyvs,swvez->hywz", Z, A)
    W = es("jZG,GH->jZH", E2["T2b"], E2["C3"])
    W = es("jZH,HEK->jZEK", W, E2["T3b"])
    W = es("jZEK,KDh->jZEDh", W, E2["T3k"])
    W = es("jZEDh,SWvEZ->jDhSWv", W, A2)
    R = es("jDhSWv,hywv->DSWjyw", W, Z)
    D, S, W_, j, y, w = R.shape
    return R.reshape(D * S * W_ * j, y * w)


def ket_stage_alt(E, A, Pg_above, Py, Pg_below):
    """Ket stage of the alternative order: as ket_stage, with the yellow pair
    acting on (q, d, s); T4k_k[g, r, y], T4b_k[y, l', g2, s]."""
    gu_a, gd_a = Pg_above
    yu, yd = Py
    gu_b, gd_b = Pg_below
    X = es("ab,aui->bui", E["C1"], E["T1k"])
    C1k = es("bui,gbu->ig", X, gu_a)
    Z = es("bug,qlb->ugql", gd_a, E["T4k"])
    Z = es("ugql,suldr->gqsdr", Z, A)
    T4kk = es("gqsdr,yqds->gry", Z, yu)
    Z = es("qksy,nvq->ksynv", yd, E["T4b"])
    T4bk = es("ksynv,tnk->yvts", Z, gu_b)
    Z = es("mn,kdm->nkd", E["C4"], E["T3k"])
    C4k = es("nkd,ndt->tk", Z, gd_b)
    return dict(C1k=C1k, T4kk=T4kk, T4bk=T4bk, C4k=C4k)


def bra_stage_alt(E, A, K, Pt_above, Pr, Pt_below):
    """Bra stage of the alternative order: as bra_stage, with the red pair
    acting on (y, u') and the bra closing the physical leg of T4b_k."""
    tu_a, td_a = Pt_above
    ru, rd = Pr
    tu_b, td_b = Pt_below
    X = es("ig,iwc->gwc", K["C1k"], E["T1b"])
    C1n = es("gwc,Tgw->cT", X, tu_a)
    Z = es("gwT,gry->Twry", td_a, K["T4kk"])
    T4kn = es("Twry,Pyw->TrP", Z, ru)
    Z = es("ywP,yvts->wPvts", rd, K["T4bk"])
    Z = es("wPvts,swvez->Ptez", Z, A)
    T4bn = es("Ptez,Ote->PzO", Z, tu_b)
    Z = es("tk,hek->the", K["C4k"], E["T3b"])
    C4n = es("the,teO->Oh", Z, td_b)
    return dict(C1=C1n, T4k=T4kn.permute(2, 1, 0), T4b=T4bn.permute(2, 1, 0), C4=C4n.T)


ORDERS = ("standard", "alternative")


# ------------------------------------------------------------ split left move
def ket_stage(E, A, Pg_above, Py, Pg_below):
    """Absorb the ket layer of one site and apply green/yellow projectors.

    Eqs. (splitCTMRG_C1/C4/Tket/Tbra), first half: C1 T1k -> green;
    T4k A -> green above, yellow below; T4b -> yellow above, green below (basis
    change only); C4 T3k -> green.  Pg_above = (up, dn) of the band above the
    site, Pg_below of the band below, Py of the site's own ket|bra cut.
    """
    gu_a, gd_a = Pg_above
    yu, yd = Py
    gu_b, gd_b = Pg_below
    X = es("ab,aui->bui", E["C1"], E["T1k"])
    C1k = es("bui,gbu->ig", X, gu_a)
    Z = es("bug,qlb->ugql", gd_a, E["T4k"])
    Z = es("ugql,suldr->gqsdr", Z, A)
    T4kk = es("gqsdr,yqd->grys", Z, yu)
    Z = es("qky,nvq->kynv", yd, E["T4b"])
    T4bk = es("kynv,tnk->yvt", Z, gu_b)
    Z = es("mn,kdm->nkd", E["C4"], E["T3k"])
    C4k = es("nkd,ndt->tk", Z, gd_b)
    return dict(C1k=C1k, T4kk=T4kk, T4bk=T4bk, C4k=C4k)


def bra_stage(E, A, K, Pt_above, Pr, Pt_below):
    """Absorb the bra layer and apply teal/red projectors (second half of the
    same four equations).  Returns the new (C1, T4k, T4b, C4) in storage order."""
    tu_a, td_a = Pt_above
    ru, rd = Pr
    tu_b, td_b = Pt_below
    X = es("ig,iwc->gwc", K["C1k"], E["T1b"])
    C1n = es("gwc,Tgw->cT", X, tu_a)                       # [a=c, b=T]
    Z = es("gwT,grys->Twrys", td_a, K["T4kk"])
    T4kn = es("Twrys,Pysw->TrP", Z, ru)                    # [b, l, q] order reversed
    Z = es("yswP,yvt->swPvt", rd, K["T4bk"])
    Z = es("swPvt,swvez->Ptez", Z, A)
    T4bn = es("Ptez,Ote->PzO", Z, tu_b)                    # [q, l', n]
    Z = es("tk,hek->the", K["C4k"], E["T3b"])
    C4n = es("the,teO->Oh", Z, td_b)                       # [n, m]
    return dict(C1=C1n, T4k=T4kn.permute(2, 1, 0), T4b=T4bn.permute(2, 1, 0), C4=C4n.T)


def _pair_tensors(Pup, Pdn, shape_alpha):
    k = Pup.shape[0]
    return Pup.reshape(k, *shape_alpha), Pdn.reshape(*shape_alpha, k)


def split_column_projectors(A, env, y, chi, record=None, order="standard"):
    """All projectors and ket-stage tensors of one column (left move).
    order: "standard" (the physical leg truncated by red, Sec. II.B) or
    "alternative" (by yellow, App. B)."""
    assert order in ORDERS, order
    alt = order == "alternative"
    Lx, Ly = len(A), len(A[0])
    yp = (y + 1) % Ly
    E = [env[x][y] for x in range(Lx)]
    a = [A[x][y] for x in range(Lx)]
    E2 = [env[x][yp] for x in range(Lx)]
    a2 = [A[x][yp] for x in range(Lx)]
    D = a[0].shape[1]
    p = a[0].shape[0]
    chi_e, chi_i = chi_pair(chi)   # green, teal cut E-bands; yellow, red cut I-bands
    Pg, Py = [], []
    for x in range(Lx):
        xp = (x + 1) % Lx
        up, dn, s = projector_pair(green_rhoT(E[x], a[x]), green_rhoB(E[xp], a[xp]), chi_e)
        Pg.append(_pair_tensors(up, dn, (E[x]["T4b"].shape[0], D)))
        if record is not None:
            record.setdefault("green", []).append((up, dn, s))
    for x in range(Lx):
        if alt:
            up, dn, s = projector_pair(yellow_alt_rhoT(E[x], a[x]), yellow_alt_rhoB(E[x], a[x]), chi_i)
            Py.append(_pair_tensors(up, dn, (E[x]["T4k"].shape[0], D, p)))
        else:
            up, dn, s = projector_pair(yellow_rhoT(E[x], a[x]), yellow_rhoB(E[x], a[x]), chi_i)
            Py.append(_pair_tensors(up, dn, (E[x]["T4k"].shape[0], D)))
        if record is not None:
            record.setdefault("yellow", []).append((up, dn, s))
    stage = ket_stage_alt if alt else ket_stage
    K = [stage(E[x], a[x], Pg[(x - 1) % Lx], Py[x], Pg[x]) for x in range(Lx)]
    Pt, Pr = [], []
    for x in range(Lx):
        xp = (x + 1) % Lx
        up, dn, s = projector_pair(teal_rhoT(E[x], a[x], K[x], E2[x], a2[x]),
                                   teal_rhoB(E[xp], a[xp], K[xp], E2[xp], a2[xp]), chi_e)
        Pt.append(_pair_tensors(up, dn, (K[x]["T4bk"].shape[2], D)))
        if record is not None:
            record.setdefault("teal", []).append((up, dn, s))
    for x in range(Lx):
        if alt:
            up, dn, s = projector_pair(red_alt_rhoT(E[x], K[x], E2[x], a2[x]),
                                       red_alt_rhoB(E[x], a[x], K[x], E2[x], a2[x]), chi_i)
            Pr.append(_pair_tensors(up, dn, (K[x]["T4kk"].shape[2], D)))
        else:
            up, dn, s = projector_pair(red_rhoT(E[x], K[x], E2[x], a2[x]),
                                       red_rhoB(E[x], a[x], K[x], E2[x], a2[x]), chi_i)
            Pr.append(_pair_tensors(up, dn, (K[x]["T4kk"].shape[2], p, D)))
        if record is not None:
            record.setdefault("red", []).append((up, dn, s))
    return E, a, K, Pg, Py, Pt, Pr, E2, a2


def split_left_move(A, env, chi, record=None, order="standard"):
    """One directional left move over every column of the unit cell.

    Column y (in order y = 0..Ly-1) is absorbed into the left environment of
    column y, and the result becomes the left environment of column y+1 (mod Ly):
    C1[x,y+1], T4k[x,y+1], T4b[x,y+1], C4[x,y+1].
    """
    Lx, Ly = len(A), len(A[0])
    env = [list(row) for row in env]
    for y in range(Ly):
        E, a, K, Pg, Py, Pt, Pr, _, _ = split_column_projectors(A, env, y, chi, record, order)
        stage = bra_stage_alt if order == "alternative" else bra_stage
        new = [stage(E[x], a[x], K[x], Pt[(x - 1) % Lx], Pr[x], Pt[x]) for x in range(Lx)]
        yn = (y + 1) % Ly
        for x in range(Lx):
            d = dict(env[x][yn])
            for key, t in new[x].items():
                d[key] = rescale(t)
            env[x][yn] = d
    return env


def split_move(A, env, direction: int, chi: int, order: str = "standard"):
    """Directional move (0 left, 1 top, 2 right, 3 bottom) of the split CTMRG."""
    return in_frame(direction, lambda a, e: split_left_move(a, e, chi, order=order), A, env, split=True)


def split_sweep(A, env, chi, order: str = "standard"):
    """One full step: left, top, right, bottom moves in sequence."""
    for d in range(4):
        env = split_move(A, env, d, chi, order)
    return env


def split_ctmrg(A, chi: int, sweeps: int, env=None, order: str = "standard"):
    """Initial environment (if not given) followed by ``sweeps`` full steps.
    order: "standard" or "alternative" yellow/red order (App. B)."""
    A = A if isinstance(A, list) else as_cell(A)
    if env is None:
        env = initial_env(A, chi, split=True)
    for _ in range(sweeps):
        env = split_sweep(A, env, chi, order)
    return env


# --------------------------------------------------- conventional CTMRG
def corner_TL(e, A, open_phys=False):
    """Enlarged corner C1 T1 T4 a at the top-left: [(c,r,r'), (n,d,d')(, s, t)]."""
    X = es("ab,auwc->buwc", e["C1"], e["T1"])
    X = es("buwc,nvlb->uwcnvl", X, e["T4"])
    X = es("uwcnvl,suldr->wcnvsdr", X, A)
    if open_phys:
        Q = es("wcnvsdr,twvez->crzndest", X, A)
        c, r, z, n, d, ee, s, t = Q.shape
        return Q.reshape(c * r * z, n * d * ee, s, t)
    Q = es("wcnvsdr,swvez->crznde", X, A)
    c, r, z, n, d, ee = Q.shape
    return Q.reshape(c * r * z, n * d * ee)


def corner_TR(e, A, open_phys=False):
    """Enlarged corner T1 C2 T2 a at the top-right: [(a,l,l'), (d,d',g)(, s, t)]."""
    Y = es("auwc,cf->auwf", e["T1"], e["C2"])
    Y = es("auwf,frzg->auwrzg", Y, e["T2"])
    Y = es("auwrzg,suldr->awzgsld", Y, A)
    if open_phys:
        Q = es("awzgsld,twvez->alvdegst", Y, A)
        a_, l, v, d, ee, g, s, t = Q.shape
        return Q.reshape(a_ * l * v, d * ee * g, s, t)
    Q = es("awzgsld,swvez->alvdeg", Y, A)
    a_, l, v, d, ee, g = Q.shape
    return Q.reshape(a_ * l * v, d * ee * g)


def corner_BR(e, A, open_phys=False):
    """Enlarged corner T2 C3 T3 a at the bottom-right: [(u,u',f), (l,l',m)(, s, t)]."""
    Z = es("frzg,gh->frzh", e["T2"], e["C3"])
    Z = es("frzh,hedm->frzedm", Z, e["T3"])
    Z = es("frzedm,suldr->fzemsul", Z, A)
    if open_phys:
        Q = es("fzemsul,twvez->uwflvmst", Z, A)
        u, w, f, l, v, m, s, t = Q.shape
        return Q.reshape(u * w * f, l * v * m, s, t)
    Q = es("fzemsul,swvez->uwflvm", Z, A)
    u, w, f, l, v, m = Q.shape
    return Q.reshape(u * w * f, l * v * m)


def corner_BL(e, A, open_phys=False):
    """Enlarged corner T4 C4 T3 a at the bottom-left: [(b,u,u'), (r,r',h)(, s, t)]."""
    W = es("hedm,mn->hedn", e["T3"], e["C4"])
    W = es("hedn,nvlb->hedvlb", W, e["T4"])
    W = es("hedvlb,suldr->hevbsur", W, A)
    if open_phys:
        Q = es("hevbsur,twvez->buwrzhst", W, A)
        b, u, w, r, z, h, s, t = Q.shape
        return Q.reshape(b * u * w, r * z * h, s, t)
    Q = es("hevbsur,swvez->buwrzh", W, A)
    b, u, w, r, z, h = Q.shape
    return Q.reshape(b * u * w, r * z * h)


def conv_left_move(A, env, chi, record=None):
    """Left move of the conventional directional CTMRG with 2x2-patch projectors
    (upper half = TL . TR, lower half = BR . BL^T, truncating the column-y band)."""
    Lx, Ly = len(A), len(A[0])
    env = [list(row) for row in env]
    for y in range(Ly):
        yp = (y + 1) % Ly
        P = []
        for x in range(Lx):
            xp = (x + 1) % Lx
            TL = corner_TL(env[x][y], A[x][y])
            TR = corner_TR(env[x][yp], A[x][yp])
            BL = corner_BL(env[xp][y], A[xp][y])
            BR = corner_BR(env[xp][yp], A[xp][yp])
            up, dn, s = projector_pair(TL.T @ TR, BR @ BL.T, chi_pair(chi)[0])
            n = env[x][y]["T4"].shape[0]
            D = A[x][y].shape[1]
            k = up.shape[0]
            P.append((up.reshape(k, n, D, D), dn.reshape(n, D, D, k)))
            if record is not None:
                record.setdefault("conv", []).append((up, dn, s))
        new = []
        for x in range(Lx):
            e, a = env[x][y], A[x][y]
            pu_a, pd_a = P[(x - 1) % Lx]
            pu_b, pd_b = P[x]
            X = es("ab,auwc->buwc", e["C1"], e["T1"])
            C1n = es("buwc,kbuw->ck", X, pu_a)
            Z = es("buwK,nvlb->uwKnvl", pd_a, e["T4"])
            Z = es("uwKnvl,suldr->wKnvsdr", Z, a)
            Z = es("wKnvsdr,swvez->Kndrez", Z, a)
            T4n = es("Kndrez,Mnde->MzrK", Z, pu_b)
            Z = es("mn,hedm->nhed", e["C4"], e["T3"])
            C4n = es("nhed,ndeK->hK", Z, pd_b)
            new.append(dict(C1=C1n, T4=T4n, C4=C4n))
        for x in range(Lx):
            d = dict(env[x][yp])
            for key, t in new[x].items():
                d[key] = rescale(t)
            env[x][yp] = d
    return env


def conv_move(A, env, direction: int, chi: int):
    return in_frame(direction, lambda a, e: conv_left_move(a, e, chi), A, env, split=False)


def conv_sweep(A, env, chi):
    """One full step of the conventional CTMRG: left, top, right, bottom."""
    for d in range(4):
        env = conv_move(A, env, d, chi)
    return env


def conv_ctmrg(A, chi: int, sweeps: int, env=None):
    """Conventional double-layer directional CTMRG (the paper's benchmark)."""
    A = A if isinstance(A, list) else as_cell(A)
    if env is None:
        env = initial_env(A, chi, split=False)
    for _ in range(sweeps):
        env = conv_sweep(A, env, chi)
    return env


# ---------------------------------------------------------- fixed point
def corner_spectra(env, chi: int):
    """Singular values of the four corners of every site, each divided by its
    largest and padded with zeros to chi (the oracle's corners grow to chi)."""
    chi = chi_pair(chi)[0]   # corners carry environment bonds only
    out = []
    for row in env:
        for e in row:
            for k in ("C1", "C2", "C3", "C4"):
                s = torch.linalg.svdvals(e[k])
                v = torch.zeros(chi, dtype=DT)
                v[: s.numel()] = s / s[0]
                out.append(v)
    return out


def ctmrg_run(A, chi: int, tol: float, max_sweeps: int, split: bool = True):
    """Full steps until the environment reaches its fixed point (Sec. II.B says
    only that the steps are iterated until the environment converges; the
    measure is the reading shared with the GPU path): after each step,
    delta = max over corners of ||s_n - s_(n-1)||_2 of the normalised corner
    spectra (before the first step, those of the initial environment); stop at
    the first step with delta < tol or after max_sweeps steps.
    Returns (env, steps done, [delta after each step])."""
    A = A if isinstance(A, list) else as_cell(A)
    env = initial_env(A, chi, split=split)
    prev = corner_spectra(env, chi)
    deltas = []
    for n in range(1, max_sweeps + 1):
        env = split_sweep(A, env, chi) if split else conv_sweep(A, env, chi)
        cur = corner_spectra(env, chi)
        deltas.append(max(float(torch.linalg.vector_norm(a - b)) for a, b in zip(cur, prev)))
        prev = cur
        if deltas[-1] < tol:
            return env, n, deltas
    return env, max_sweeps, deltas
