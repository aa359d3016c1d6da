"""Brute-force expectation values for exactly solvable iPEPS (oracle pins).

Test infrastructure only.  These functions never touch a tensor network: they
work on explicit state vectors of at most four spins, so they pin the CTMRG
oracle independently of its own arithmetic.

* ``product_energy``   -- real product state on an Lx x Ly cell; every bond
  factorises into single-site expectation values.
* ``cluster_energy``   -- product of identical 4-site plaquettes (2x2 cell):
  bonds inside a plaquette from the 16-amplitude state vector, bonds between
  plaquettes from single-site expectation values.
* ``dimer_energy``     -- singlets on the horizontal (x,0)-(x,1) bonds.
"""
from __future__ import annotations

import numpy as np


def _h4(h):
    p = int(round(np.sqrt(h.shape[0])))
    return np.asarray(h, dtype=np.float64).reshape(p, p, p, p)   # [t_i,t_j,s_i,s_j]


def _two_site_value(rho_ij, h):
    """rho_ij[s_i,s_j,t_i,t_j] = psi_s psi_t (ket s, bra t) -> <h>."""
    return float(np.einsum("TUsv,svTU->", _h4(h), rho_ij))


def _product_bond(phi_i, phi_j, h):
    pi = phi_i / np.linalg.norm(phi_i)
    pj = phi_j / np.linalg.norm(phi_j)
    rho = np.einsum("s,v,T,U->svTU", pi, pj, pi, pj)
    return _two_site_value(rho, h)


def _bonds(Lx, Ly):
    """Per-site bonds: right, down (NN) and the two downward diagonals."""
    nn, dg = [], []
    for x in range(Lx):
        for y in range(Ly):
            nn.append(((x, y), (x, (y + 1) % Ly)))
            nn.append(((x, y), ((x + 1) % Lx, y)))
            dg.append(((x, y), ((x + 1) % Lx, (y + 1) % Ly)))
            dg.append(((x, (y + 1) % Ly), ((x + 1) % Lx, y)))   # TR - BL of the patch at (x,y)
    return nn, dg


def product_energy(phis, h_nn, h_diag=None):
    """Energy per site of the real product state phi[x][y] (Lx, Ly, p)."""
    phis = np.asarray(phis, dtype=np.float64)
    Lx, Ly = phis.shape[:2]
    nn, dg = _bonds(Lx, Ly)
    e = sum(_product_bond(phis[a], phis[b], h_nn) for a, b in nn)
    if h_diag is not None:
        e += sum(_product_bond(phis[a], phis[b], h_diag) for a, b in dg)
    return e / (Lx * Ly)


def _cluster_state_pairs(psi):
    """Reduced two-site density matrices of a normalised 4-spin state.

    Sites are labelled 0=(0,0), 1=(0,1), 2=(1,0), 3=(1,1)."""
    psi = np.asarray(psi, dtype=np.float64)
    psi = psi / np.linalg.norm(psi)
    letters = "abcd"
    rdm2 = {}
    for i in range(4):
        for j in range(4):
            if i == j:
                continue
            ket = list(letters)
            bra = list(letters)
            bra[i] = "T"
            bra[j] = "U"
            ket[i] = "s"
            ket[j] = "v"
            rdm2[(i, j)] = np.einsum(f"{''.join(ket)},{''.join(bra)}->svTU", psi, psi)
    rdm1 = {}
    for i in range(4):
        ket = list(letters)
        bra = list(letters)
        ket[i] = "s"
        bra[i] = "t"
        rdm1[i] = np.einsum(f"{''.join(ket)},{''.join(bra)}->st", psi, psi)
    return rdm1, rdm2


def cluster_energy(psi, h_nn, h_diag=None):
    """Energy per site of the product of 2x2 plaquettes psi[s00,s01,s10,s11]
    (the state of ``ipeps_inputs.plaquette_cell``)."""
    rdm1, rdm2 = _cluster_state_pairs(psi)
    idx = {(0, 0): 0, (0, 1): 1, (1, 0): 2, (1, 1): 3}

    def bond(a, b, h, same_cell):
        i, j = idx[a], idx[b]
        if same_cell:
            return _two_site_value(rdm2[(i, j)], h)
        rho = np.einsum("sT,vU->svTU", rdm1[i], rdm1[j])
        return _two_site_value(rho, h)

    e = 0.0
    # nearest neighbours: right and down of every site, wrapping -> other plaquette
    for x in range(2):
        for y in range(2):
            e += bond((x, y), (x, (y + 1) % 2), h_nn, y + 1 < 2)
            e += bond((x, y), ((x + 1) % 2, y), h_nn, x + 1 < 2)
            if h_diag is not None:
                e += bond((x, y), ((x + 1) % 2, (y + 1) % 2), h_diag, x + 1 < 2 and y + 1 < 2)
                e += bond((x, (y + 1) % 2), ((x + 1) % 2, y), h_diag, x + 1 < 2 and y + 1 < 2)
    return e / 4.0


def dimer_energy(h_nn, h_diag=None):
    """Energy per site of singlets on the bonds (x,0)-(x,1) of a 2x2 cell."""
    singlet = np.array([[0.0, 1.0], [-1.0, 0.0]]) / np.sqrt(2.0)   # psi[s_left, s_right]
    rho_in = np.einsum("sv,TU->svTU", singlet, singlet)
    half = np.eye(2) / 2.0
    rho_out = np.einsum("sT,vU->svTU", half, half)
    e = 0.0
    # per cell: 2 singlet bonds, 6 other NN bonds, 8 diagonals, all between
    # spins with zero single-site magnetisation
    e += 2 * _two_site_value(rho_in, h_nn) + 6 * _two_site_value(rho_out, h_nn)
    if h_diag is not None:
        e += 8 * _two_site_value(rho_out, h_diag)
    return e / 4.0


def dimer_pairs_energy(psis, h_nn, h_diag=None, vertical=False):
    """Energy per site of ``ipeps_inputs.dimer_pairs_cell(psis)``: generic two-site
    states psi_k[s_first, s_second] on (k,0)-(k,1) (or (0,k)-(1,k) if vertical)."""
    rho2, rho1 = [], []
    for k in range(2):
        ps = np.asarray(psis[k], dtype=np.float64)
        ps = ps / np.linalg.norm(ps)
        rho2.append(np.einsum("sv,TU->svTU", ps, ps))
        rho1.append((np.einsum("sv,Tv->sT", ps, ps), np.einsum("sv,sU->vU", ps, ps)))
    # single-site density matrices per site
    one = {}
    for k in range(2):
        a, b = ((k, 0), (k, 1)) if not vertical else ((0, k), (1, k))
        one[a], one[b] = rho1[k]

    def pair(a, b, h):
        for k in range(2):
            first, second = ((k, 0), (k, 1)) if not vertical else ((0, k), (1, k))
            if (a, b) == (first, second):
                return _two_site_value(rho2[k], h)
            if (a, b) == (second, first):
                return _two_site_value(np.einsum("svTU->vsUT", rho2[k]), h)
        return _two_site_value(np.einsum("sT,vU->svTU", one[a], one[b]), h)

    e = 0.0
    for x in range(2):
        for y in range(2):
            # a bond to the next cell connects different clusters
            same_r = (y + 1 < 2)
            same_d = (x + 1 < 2)
            r = (x, (y + 1) % 2)
            d = ((x + 1) % 2, y)
            e += pair((x, y), r, h_nn) if same_r else _two_site_value(np.einsum("sT,vU->svTU", one[(x, y)], one[r]), h_nn)
            e += pair((x, y), d, h_nn) if same_d else _two_site_value(np.einsum("sT,vU->svTU", one[(x, y)], one[d]), h_nn)
            if h_diag is not None:
                for a, b in [((x, y), ((x + 1) % 2, (y + 1) % 2)), ((x, (y + 1) % 2), ((x + 1) % 2, y))]:
                    e += _two_site_value(np.einsum("sT,vU->svTU", one[a], one[b]), h_diag)
    return e / 4.0
