// Split-CTMRG engine on one GPU: environment, directional moves, projectors,
// 2x2-patch energy and the reverse pass.
#pragma once
#include <array>
#include <vector>

#include "ops.h"

namespace sctm {

enum Key { C1, T1k, T1b, C2, T2k, T2b, C3, T3b, T3k, C4, T4b, T4k, NKEY };

// Environment of one site (Fig. 2).  Leg order of every tensor:
//   C1[a,b] a->T1k b->T4k;  C2[c,f]  C3[g,h]  C4[m,n]  ([previous, next] along
//   the clockwise chain for C2..C4, [next, previous] for C1);
//   T1k[a,u,i] T1b[i,u',c] T2k[f,r,j] T2b[j,r',g] T3b[h,d',k] T3k[k,d,m]
//   T4b[n,l',q] T4k[q,l,b]  ([previous, PEPS leg, next]).
using SiteEnv = std::array<Tensor, NKEY>;

struct Cell {
  int Lx = 0, Ly = 0;
  std::vector<Tensor> A;      // A[x*Ly + y] : [p, D, D, D, D]  (u, l, d, r)
  std::vector<SiteEnv> env;   // env[x*Ly + y]
  Tensor& a(int x, int y) { return A[((x % Lx + Lx) % Lx) * Ly + ((y % Ly + Ly) % Ly)]; }
  SiteEnv& e(int x, int y) { return env[((x % Lx + Lx) % Lx) * Ly + ((y % Ly + Ly) % Ly)]; }
};

struct Params {
  int Lx = 1, Ly = 1, p = 2, D = 2;
  int chi = 16;               // environment bond dimension chi_E (corners, environment legs of the edges)
  int chiI = 16;              // interlayer bond dimension chi_I (between a ket and a bra edge)
  double cutoff = 1e-8;       // relative cutoff on the projector singular values
  double gram_cutoff = 1e-15; // relative cutoff on Gram eigenvalues (reduction)
  double eps_l = 1e-36;       // Lorentzian broadening (relative to s_max^4)
  bool mixed = false;         // mixed mode: FP32 contractions, randomized projectors
  bool conventional = false;  // double-layer CTMRG (fused edges in both slots of a pair)
  int power_steps = 2;        // randomized projectors: power steps (mixed mode)
  int rank_extra = 0;         // randomized projectors: columns beyond chi (set from chi at creation)
  int adjoint_cg_steps = 0;   // randomized projectors' adjoint: CG steps for the complement coupling
  int adjoint_band = -1;      // randomized projectors' adjoint: computed triplets beyond chi coupled exactly (-1: all)
  int randomized_min = 256;   // randomized projectors only when the truncated space has >= this dimension
  int order = 0;              // 0: the physical leg truncated by red (Sec. II.B); 1: by yellow (App. B)
};

struct ProjPair {
  Tensor up, dn;   // up: [k, alpha...], dn: [alpha..., k]
  Tensor s;        // singular values of the decomposed core
};

// Projector pair from rhoT (alpha x beta) and rhoB (beta x alpha), keeping k
// singular values (chi_E for green and teal, chi_I for yellow and red).
ProjPair projector(Ctx& c, const Params& P, const Tensor& rhoT, const Tensor& rhoB, int k);

struct KetStage {
  // C1k[i,g] T4kk[g,r,y,s] T4bk[y,v,t] C4k[t,k]; in the alternative order
  // (physical leg truncated by yellow) T4kk[g,r,y] and T4bk[y,v,t,s]
  Tensor C1k, T4kk, T4bk, C4k;
  bool alt() const { return T4kk.nd == 3; }
};

// All projectors of one column of a left move (green, yellow, teal, red per
// row) and the ket-stage tensors.
struct ColumnProj {
  std::vector<ProjPair> g, y, t, r;
  std::vector<KetStage> K;
};
void column_projectors(Ctx& c, const Params& P, Cell& cell, int y, ColumnProj& out);

Cell frame_transpose(Cell& cell);
Cell frame_rot180(Cell& cell);

// one left move in the canonical frame (all columns, in order)
void left_move(Ctx& c, const Params& P, Cell& cell);
// directional move: 0 left, 1 top, 2 right, 3 bottom
void move(Ctx& c, const Params& P, Cell& cell, int dir);

// environment from the neighbours' double layers, padded to chi
void init_env(Ctx& c, const Params& P, Cell& cell);

// conventional (double-layer) CTMRG: initial environment and one left move
void conv_init_env(Ctx& c, const Params& P, Cell& cell);
void conv_left_move(Ctx& c, const Params& P, Cell& cell);

// Energy of one 2x2 patch: E_p = sum_t w_t <Htop(t1,t2), Hbot(b1,b2)> / <Htop(0,0), Hbot(0,0)>
// with Htop(o1, o2) = TL(o1)^T TR(o2) and Hbot(o3, o4) = BL(o3) BR(o4)^T over the
// enlarged corners of the patch, each carrying one operator slot o (0 = identity).
struct PatchTerm {
  int t1, t2, b1, b2;   // operator slots of TL, TR (top product) and BL, BR (bottom product)
  double w;
};
// bond operators split into one-site factors (operator-Schmidt decomposition);
// factors equal up to a scale share one slot, slot 0 is the identity
struct EnergyOps {
  struct Pair { int a, b; double w; };
  std::vector<Tensor> op;          // [p, p] device matrices
  std::vector<Pair> nn, diag;
};
EnergyOps energy_ops(Ctx& c, const Params& P, const double* h_nn, const double* h_diag);
// the bond terms of every patch (the same for all patches); nsites = Lx Ly
std::vector<PatchTerm> patch_terms(const EnergyOps& E, int nsites);
struct PatchCorners {
  std::vector<Tensor> TL, TR, BR, BL;   // by operator slot; data == nullptr where no term needs it
};
// the enlarged corners of the patch with top-left site (x, y) that `terms`
// need, taped when the tape is on
PatchCorners patch_corners(Ctx& c, const Params& P, Cell& cell, const EnergyOps& E,
                           const std::vector<PatchTerm>& terms, int x, int y);

}  // namespace sctm
