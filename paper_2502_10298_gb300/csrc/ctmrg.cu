// Split-CTMRG engine (see ctmrg.h).
//
// Paper: Naumann et al., arXiv 2502.10298.  Environment: Fig. 2.  Left move:
// Eqs. (splitCTMRG_C1), (splitCTMRG_C4), (splitCTMRG_Tket), (splitCTMRG_Tbra).
// Projectors: Sec. II.B (Fig. 3) and App. A (Figs. 7-9).  The other three
// moves are left moves in a transposed or 180-degree rotated frame; frames are
// pure stride/handle permutations, so they cost nothing on the device.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>

#include "ctmrg.h"

namespace sctm {

// ------------------------------------------------------------------ projector
static Tensor no_grad(Tensor t) {
  t.grad = nullptr;
  return t;
}

// Batched SVD of equally shaped square matrices (untaped, noise-level columns
// exempt from the convergence test): one kernel launch.
static std::vector<SVDResult> svd_batch(Ctx& c, const std::vector<Tensor>& Ms) {
  const int nb = (int)Ms.size();
  std::vector<SVDResult> out(nb);
  if (nb == 0) return out;
  const int n = Ms[0].shape[0];
  Tensor Mb = c.empty({nb, n, n}), Ub = c.empty({nb, n, n}), Sb = c.empty({nb, n}), Vb = c.empty({nb, n, n});
  for (int i = 0; i < nb; ++i) copy_into(c, Ms[i], Mb.sub(0, i));
  size_t wn = svd_work_doubles(n, n, nb);
  double* work = wn ? c.arena.alloc((long long)wn) : nullptr;
  // small factors of the randomized path: singular values at rounding level are
  // discarded afterwards, so their (noise-level) columns need not converge
  // the factors come from mixed-precision products (rounding about 1e-7), so
  // orthogonality to 1e-11 is ample
  launch_svd(n, n, nb, Mb.data, Ub.data, Sb.data, Vb.data, work, c.svd_status, c.stream, 2.0e-29, 1e-11,
             c.svd_max_sweeps);
  for (int i = 0; i < nb; ++i) out[i] = SVDResult{Ub.sub(0, i), Sb.sub(0, i), Vb.sub(0, i)};
  return out;
}

// Contractions of this scope run in FP64 arithmetic even in mixed mode.
struct Fp64Scope {
  Ctx& c;
  bool old, on = true;
  explicit Fp64Scope(Ctx& cx) : c(cx), old(cx.fp32_compute) { c.fp32_compute = false; }
  void end() {
    if (on) c.fp32_compute = old;
    on = false;
  }
  ~Fp64Scope() { end(); }
};

// In the BF16-slice mode (precision 4), contractions of this scope whose shape
// fits the tensor-core tiles take the slice kernel whatever their size, and the
// others run in FP64 on the CUDA cores: the randomized projectors resolve the
// small singular directions from products with rho, and their reverse pass
// divides by those singular values, so FP32-level rounding there would swamp
// the gradient.  No effect in the other precisions.
struct AccurateScope {
  Ctx& c;
  explicit AccurateScope(Ctx& cx) : c(cx) { ++c.accurate; }
  ~AccurateScope() { --c.accurate; }
};

// Operands used by many contractions of a scope (the rho halves of the
// randomized projectors: the power iteration, the projector formation and the
// reverse pass multiply each of them several times, in both orientations) are
// packed for the slice kernel once per layout and kept in the arena's high
// stack until the scope ends.  Their data must not change meanwhile.
struct SliceKeepScope {
  Ctx& c;
  size_t hi, nkeep, npanels;
  SliceKeepScope(Ctx& cx, const std::vector<Tensor>& keep)
      : c(cx), hi(cx.arena.mark_high()), nkeep(cx.slice_keep.size()), npanels(cx.slice_panels.size()) {
    if (c.bf16_slices)
      for (const Tensor& t : keep) c.slice_keep.push_back(t.data);
  }
  ~SliceKeepScope() {
    c.slice_keep.resize(nkeep);
    c.slice_panels.resize(npanels);
    c.arena.release_high(hi);
  }
};

// G = Y^T Y in FP64: the symmetric Gram kernel for row-major Y outside a
// taped region (upper-triangle tiles only, rows split over extra CTAs), else
// the general contraction.
static Tensor gram64(Ctx& c, const Tensor& Y) {
  if (Y.nd == 2 && Y.stride[1] == 1 && !c.tape.active) {
    const int r = Y.shape[1];
    Tensor G = c.empty({r, r});
    const size_t mk = c.arena.mark();
    double* W = c.arena.alloc((long long)r * r);
    launch_gram(Y.shape[0], r, Y.data, Y.stride[0], G.data, r, W, c.stream);
    c.arena.release(mk);   // stream-ordered: later work reuses the scratch after the kernels
    return G;
  }
  Fp64Scope f(c);
  return einsum(c, "ai,aj->ij", Y, Y);
}

// Orthonormal (or zero) columns spanning the columns of each Y_i (m_i x r):
// Cholesky QR with FP64 Gram matrices and deflation of dependent columns
// (pivots below 1e-13 of the largest), Q = Y R^+.  Two passes (CholeskyQR2;
// Yamamoto et al. 2015) give orthonormality to rounding for condition numbers
// up to about 1e8; one pass suffices for the intermediate bases of the power
// iteration, which only have to keep the directions apart.  Not taped.
static std::vector<Tensor> orthonormal_columns_batch(Ctx& c, const std::vector<Tensor>& Ys, int passes = 2) {
  const int nb = (int)Ys.size();
  if (nb == 0) return {};
  const int r = Ys[0].shape[1];
  std::vector<Tensor> Q = Ys;
  for (int pass = 0; pass < passes; ++pass) {
    Tensor Gb = c.empty({nb, r, r}), Tb = c.empty({nb, r, r});
    for (int i = 0; i < nb; ++i) copy_into(c, gram64(c, Q[i]), Gb.sub(0, i));
    launch_chol_qr_factor(r, nb, Gb.data, Tb.data, 1e-13, c.stream);
    for (int i = 0; i < nb; ++i) Q[i] = einsum(c, "ai,ij->aj", Q[i], Tb.sub(0, i));
  }
  return Q;
}

// Top-r singular triplets of M = rhoB rhoT (beta x beta, never formed) by
// randomized subspace iteration (Halko, Martinsson, Tropp 2011, Alg. 4.4):
// Q = orth(M Omega), then `power_steps` times Z = orth(M^T Q), Q = orth(M Z)
// (a basis after every product keeps the small directions resolvable), and
// finally B = Q^T M decomposed as below.  Returns U (beta x r), S (r),
// V (beta x r) with M ~ U S V^T.  Not taped.
struct Trunc {
  Tensor U, S, V;
};
static std::vector<Trunc> randomized_svd_batch(Ctx& c, const std::vector<Tensor>& rT, const std::vector<Tensor>& rB,
                                               int r, int power_steps) {
  AccurateScope acc(c);
  std::vector<Tensor> keep = rT;
  keep.insert(keep.end(), rB.begin(), rB.end());
  SliceKeepScope kept(c, keep);
  const size_t nb = rT.size();
  std::vector<Tensor> Y(nb);
  for (size_t i = 0; i < nb; ++i) {
    const int b = rT[i].shape[1];
    Tensor Om = c.empty({b, r});
    launch_gaussian(b, r, 0x5eedULL + (unsigned long long)b * 131 + r, Om.data, c.stream);
    Y[i] = einsum(c, "ab,bj->aj", rB[i], einsum(c, "ab,bj->aj", rT[i], Om));       // M Omega
  }
  std::vector<Tensor> Q = orthonormal_columns_batch(c, Y, power_steps > 0 ? 1 : 2);
  for (int q = 0; q < power_steps; ++q) {
    for (size_t i = 0; i < nb; ++i)
      Y[i] = einsum(c, "ba,bj->aj", rT[i], einsum(c, "ba,bj->aj", rB[i], Q[i]));    // M^T Q
    std::vector<Tensor> Z = orthonormal_columns_batch(c, Y, 1);
    for (size_t i = 0; i < nb; ++i)
      Y[i] = einsum(c, "ab,bj->aj", rB[i], einsum(c, "ab,bj->aj", rT[i], Z[i]));    // M Z
    Q = orthonormal_columns_batch(c, Y, q + 1 < power_steps ? 1 : 2);   // the final basis: two passes
  }
  // B^T = M^T Q = Q_B R_B (CholeskyQR2), R_B = U_R S V_R^T (FP64 Jacobi):
  // M ~ Q B = (Q V_R) S (Q_B U_R)^T with both factors orthonormal and no
  // division by small singular values (which would carry the contraction
  // rounding into V and spoil the reverse pass)
  std::vector<Tensor> Bt(nb);
  for (size_t i = 0; i < nb; ++i)
    Bt[i] = einsum(c, "ba,bj->aj", rT[i], einsum(c, "ba,bj->aj", rB[i], Q[i]));    // B^T = M^T Q
  std::vector<Tensor> QB = orthonormal_columns_batch(c, Bt, 2);
  std::vector<Tensor> RB(nb);
  {
    Fp64Scope f(c);
    for (size_t i = 0; i < nb; ++i) RB[i] = einsum(c, "ai,aj->ij", QB[i], Bt[i]);   // R_B = Q_B^T B^T
  }
  std::vector<SVDResult> e = svd_batch(c, RB);
  std::vector<Trunc> out(nb);
  for (size_t i = 0; i < nb; ++i) {
    // singular vectors of rounding-level values (below 1e-10 s_1, far under any
    // cutoff) are not resolved: zero them, so the reverse pass treats those
    // directions as part of the complement
    Tensor keep = spectrum_map(c, e[i].S, r, 1e-10, 2);
    out[i].S = e[i].S;
    out[i].U = scale_dim(c, einsum(c, "ai,ij->aj", Q[i], e[i].V), 1, keep);
    out[i].V = scale_dim(c, einsum(c, "ai,ij->aj", QB[i], e[i].U), 1, keep);
  }
  return out;
}

// Reverse pass of a truncated SVD (U_r, S_r, V_r) of M = rhoB rhoT (beta x
// beta, never formed).  Pairs inside the r computed triplets use the usual
// broadened coefficients; the coupling of triplet i to the unknown rest of the
// spectrum follows first-order perturbation theory summed over it: with
// P = 1 - U U^T, Q = 1 - V V^T the columns
//   y_i = (s_i^2 - P M M^T P)^-1 P (s_i u_bar_i + M v_bar_i),
//   z_i = (s_i^2 - Q M^T M Q)^-1 Q (M^T u_bar_i + s_i v_bar_i)
// are found by column-wise conjugate gradients (cg_steps of them), which only
// apply M and M^T; with cg_steps = 0 every column takes the first-order term
// y_i = P (s_i u_bar_i + M v_bar_i) / s_i^2, z_i = Q (M^T u_bar_i + s_i v_bar_i) / s_i^2
// (the expansion of the inverse to zeroth order in P M M^T P / s_i^2).
// Then
//   M_bar = U X V^T + Y V^T + U Z^T,
//   X = F o (J - J^T) S + diag(S_bar) + S F o (K - K^T), J = U^T U_bar, K = V^T V_bar,
// applied without forming M_bar:  rhoB_bar += M_bar rhoT^T, rhoT_bar += rhoB^T M_bar.
// The systems are positive definite when s_i > s_{r+1}, but the products with
// M carry the rounding of the contraction arithmetic (about 1e-7 s_1^2 in
// mixed mode), and the randomized basis leaks a little of the top spectrum
// into P M M^T P; so the solve is used for s_i >= 1e-3 s_1 only and a column's
// iteration stops where its operator is not safely positive definite (see
// launch_cg_update); smaller kept values take the first-order term.  Columns
// without cotangent stay zero.
static constexpr double kComplementMinRel = 1e-3;

static void truncated_svd_adjoint(Ctx& c, const Tensor& rhoT, const Tensor& rhoB, const Tensor& U, const Tensor& S,
                                  const Tensor& V, double eps_l, int cg_steps) {
  AccurateScope acc(c);
  SliceKeepScope kept(c, {rhoT, rhoB});
  const int k = S.shape[0];
  const int nb = U.shape[0];
  Tensor gU = no_grad(U), gV = no_grad(V), gS = no_grad(S);
  gU.data = U.grad;
  gV.data = V.grad;
  gS.data = S.grad;
  // products with M = rhoB rhoT and M^T on beta x k blocks
  auto Mx = [&](const Tensor& x) { return einsum(c, "ab,bj->aj", rhoB, einsum(c, "ab,bj->aj", rhoT, x)); };
  auto MTx = [&](const Tensor& x) { return einsum(c, "ba,bj->aj", rhoT, einsum(c, "ba,bj->aj", rhoB, x)); };
  auto project = [&](const Tensor& B, Tensor x) {   // x <- (1 - B B^T) x, in place
    einsum_into(c, "ai,ij->aj", B, einsum(c, "ai,aj->ij", B, x), x, -1.0, 1.0, false);
    return x;
  };
  // M Q v_bar and M^T P u_bar of the first-order coupling.  With exact
  // singular vectors P M V = 0 and these equal P M v_bar, P M^T u_bar; the
  // computed triplets are Ritz vectors whose residual P M V, divided by s_i^2,
  // would swamp the term, so only the parts of the cotangents outside the
  // computed spaces are multiplied (projections in FP64, products in the
  // accurate form of the handle's precision: their rounding is divided by s_i^2)
  Tensor Mv, Mu;
  {
    Fp64Scope f(c);
    Mv = project(V, copy(c, gV));
    Mu = project(U, copy(c, gU));
  }
  Mv = Mx(Mv);
  Mu = MTx(Mu);
  // FP64 arithmetic up to M_bar's factors: the complement terms divide
  // P U_bar by s_i, and P U_bar = U_bar - U (U^T U_bar) cancels; FP32-level
  // rounding of it, amplified by 1/s_i up to the inverse cutoff, swamps the
  // gradient.  The final products with rho run in the handle's precision.
  Fp64Scope f64(c);
  Tensor J = c.empty({k, k}), K = c.empty({k, k}), X = c.empty({k, k});
  einsum_into(c, "ai,aj->ij", U, gU, J, 1.0, 0.0, false);
  einsum_into(c, "ai,aj->ij", V, gV, K, 1.0, 0.0, false);
  launch_svd_adj_inner(k, S.data, J.data, K.data, gS.data, X.data, eps_l, c.stream);
  Tensor s2 = c.empty({k});
  einsum_into(c, "j,j->j", S, S, s2, 1.0, 0.0, false);   // s_j^2
  // masks: m_j = 1 for s_j >= kComplementMinRel s_1 (solved), else 0 (leading term)
  Tensor msk = spectrum_map(c, S, k, kComplementMinRel, 2);
  if (cg_steps <= 0) launch_fill(k, 0.0, msk.data, c.stream);   // leading term for every column
  Tensor nmsk = c.empty({k});
  launch_fill(k, 1.0, nmsk.data, c.stream);
  launch_axpy(k, -1.0, msk.data, nmsk.data, c.stream);
  Tensor sinv = spectrum_map(c, S, k, 1e-14, 0);              // s^-1/2
  // column-wise CG for (diag(s^2) - B) Y = rhs, B = P op P
  auto solve = [&](const Tensor& Bas, Tensor rhs, bool left) {
    Tensor Yv = c.zeros({nb, k});
    Tensor R = copy(c, rhs);
    Tensor Pd = copy(c, rhs);
    Tensor rr = c.empty({k}), rr2 = c.empty({k}), pq = c.empty({k}), pp = c.empty({k});
    int* frozen = reinterpret_cast<int*>(c.zeros({(k + 1) / 2}).data);
    launch_coldot(nb, k, R.data, R.data, rr.data, c.stream);
    for (int it = 0; it < cg_steps; ++it) {
      Tensor Bp = project(Bas, left ? Mx(MTx(Pd)) : MTx(Mx(Pd)));
      Tensor Q = scale_dim(c, Pd, 1, s2);
      launch_axpy(Q.numel(), -1.0, Bp.data, Q.data, c.stream);          // Q = s^2 p - B p
      launch_coldot(nb, k, Pd.data, Q.data, pq.data, c.stream);
      launch_coldot(nb, k, Pd.data, Pd.data, pp.data, c.stream);
      launch_cg_update(nb, k, Pd.data, Q.data, Yv.data, R.data, rr.data, pq.data, pp.data, s2.data, frozen,
                       c.stream);
      launch_coldot(nb, k, R.data, R.data, rr2.data, c.stream);
      launch_cg_direction(nb, k, Pd.data, R.data, rr2.data, rr.data, frozen, c.stream);
      std::swap(rr, rr2);
    }
    return Yv;
  };
  // right-hand sides: P (U_bar S + M V_bar), Q (M^T U_bar + V_bar S)
  Tensor bY, bZ;
  if (cg_steps > 0) {
    bY = scale_dim(c, gU, 1, S);
    launch_axpy(bY.numel(), 1.0, Mv.data, bY.data, c.stream);
    bY = project(U, bY);
    bZ = scale_dim(c, gV, 1, S);
    launch_axpy(bZ.numel(), 1.0, Mu.data, bZ.data, c.stream);
    bZ = project(V, bZ);
  }
  Tensor A = cg_steps > 0 ? solve(U, scale_dim(c, bY, 1, msk), true) : c.zeros({nb, k});
  Tensor Bm = cg_steps > 0 ? solve(V, scale_dim(c, bZ, 1, msk), false) : c.zeros({nb, k});
  // first-order terms for the unmasked columns:
  // P (U_bar S^-1 + M V_bar S^-2), Q (V_bar S^-1 + M^T U_bar S^-2)
  {
    Tensor w = c.empty({k}), w2 = c.empty({k});
    einsum_into(c, "j,j->j", sinv, sinv, w, 1.0, 0.0, false);   // 1/s
    einsum_into(c, "j,j->j", w, nmsk, w, 1.0, 0.0, false);
    einsum_into(c, "j,j->j", w, w, w2, 1.0, 0.0, false);        // 1/s^2 (masked)
    Tensor yl = scale_dim(c, gU, 1, w);
    launch_axpy(yl.numel(), 1.0, scale_dim(c, Mv, 1, w2).data, yl.data, c.stream);
    Tensor zl = scale_dim(c, gV, 1, w);
    launch_axpy(zl.numel(), 1.0, scale_dim(c, Mu, 1, w2).data, zl.data, c.stream);
    yl = project(U, yl);
    zl = project(V, zl);
    launch_axpy(A.numel(), 1.0, yl.data, A.data, c.stream);
    launch_axpy(Bm.numel(), 1.0, zl.data, Bm.data, c.stream);
  }
  // L1 = U X + Y
  Tensor L1 = c.empty({nb, k});
  einsum_into(c, "ai,ij->aj", U, X, L1, 1.0, 0.0, false);
  launch_axpy(L1.numel(), 1.0, A.data, L1.data, c.stream);
  f64.end();
  // rhoB_bar += L1 (V^T rhoT^T) + U (Z^T rhoT^T)
  if (rhoB.grad) {
    Tensor gB = no_grad(rhoB);
    gB.data = rhoB.grad;
    Tensor VR = c.empty({k, (int)rhoT.shape[0]}), BR = c.empty({k, (int)rhoT.shape[0]});
    einsum_into(c, "bj,ab->ja", V, rhoT, VR, 1.0, 0.0, false);
    einsum_into(c, "bj,ab->ja", Bm, rhoT, BR, 1.0, 0.0, false);
    einsum_into(c, "bj,ja->ba", L1, VR, gB, 1.0, 1.0, false);
    einsum_into(c, "bj,ja->ba", U, BR, gB, 1.0, 1.0, false);
  }
  // rhoT_bar += (rhoB^T L1) V^T + (rhoB^T U) Z^T
  if (rhoT.grad) {
    Tensor gT = no_grad(rhoT);
    gT.data = rhoT.grad;
    Tensor RL = c.empty({(int)rhoB.shape[1], k}), RU = c.empty({(int)rhoB.shape[1], k});
    einsum_into(c, "ba,bj->aj", rhoB, L1, RL, 1.0, 0.0, false);
    einsum_into(c, "ba,bj->aj", rhoB, U, RU, 1.0, 0.0, false);
    einsum_into(c, "aj,bj->ab", RL, V, gT, 1.0, 1.0, false);
    einsum_into(c, "aj,bj->ab", RU, Bm, gT, 1.0, 1.0, false);
  }
}

// rhoT: alpha x beta (upper half), rhoB: beta x alpha (lower half).
// M = rhoB rhoT has rank <= alpha; when alpha < beta both halves are reduced
// first (App. A: decompose rho^T and rho^B before multiplying them), here by
// thin SVDs computed with one-sided Jacobi (relative accuracy):
//   rhoT^T = Q_T S_T V_T^T -> rhoT = L_T Q_T^T with L_T = V_T S_T,
//   rhoB   = Q_B S_B V_B^T -> rhoB = Q_B L_B^T with L_B = V_B S_B,
//   K = L_B^T L_T = U S V^T,  P_up = S^-1/2 U^T L_B^T,  P_dn = L_T V S^-1/2,
// which equals S^-1/2 U~^T rhoB and rhoT V~ S^-1/2 for the full M.
// Mixed mode with alpha > 2 chi: the chi leading triplets of M come from a
// randomized subspace iteration (randomized_svd_batch) and the reverse pass uses
// the truncated-SVD adjoint above.
static ProjPair finish_randomized(Ctx& c, const Params& P, const Tensor& rhoT, const Tensor& rhoB, const Trunc& t,
                                  int k) {
  AccurateScope acc(c);
  SliceKeepScope kept(c, {rhoT, rhoB});
  bool tap = c.tape.active;
  {
    // leaves U_r, S_r, V_r with gradient buffers when taping; the projector
    // uses the first k triplets, the reverse pass couples them to all r
    Tensor Ur = copy(c, t.U), Vr = copy(c, t.V), Sr = copy(c, t.S);
    Tensor Uk = Ur, Vk = Vr, Sk = Sr;
    Uk.shape[1] = k;
    Vk.shape[1] = k;
    Sk.shape[0] = k;
    if (tap) {
      // the reverse pass couples the kept triplets exactly to the next
      // `adjoint_band` computed ones (all r by default); the rest of the
      // spectrum is treated as the complement
      const int kb = P.adjoint_band < 0 ? (int)Sr.shape[0] : std::min((int)Sr.shape[0], k + P.adjoint_band);
      Tensor rT = rhoT, rB = rhoB, U = Ur, S = Sr, V = Vr;
      U.shape[1] = kb;
      V.shape[1] = kb;
      S.shape[0] = kb;
      double eps = P.eps_l;
      int cg = P.adjoint_cg_steps;
      c.tape.push([&c, rT, rB, U, S, V, eps, cg]() {
        bool t2 = c.tape.active;
        c.tape.active = false;
        truncated_svd_adjoint(c, rT, rB, U, S, V, eps, cg);
        c.tape.active = t2;
      });
    }
    Tensor w = spectrum_map(c, Sk, k, P.cutoff, 0);
    Tensor up = scale_dim(c, einsum(c, "ik,ia->ka", Uk, rhoB), 0, w);
    Tensor dn = scale_dim(c, einsum(c, "ai,ik->ak", rhoT, Vk), 1, w);
    Tensor sg = row_signs(c, up);
    up = scale_dim(c, up, 0, sg);
    dn = scale_dim(c, dn, 1, sg);
    return ProjPair{up, dn, Sk};
  }
}

// Randomized projectors only for spaces at least kRandomizedRatio times the
// sketch width r = k + rank_extra (and at least randomized_min): nearer to r the
// sketch saves little work, and its gradient is the least accurate.  Measured
// at equal cutoff 1e-5 (two sweeps, precision 4), gradient against the exact
// FP64 one: at D=4, chi=64 (1x1 near-product state) the green and teal
// projectors (n = chi D = 2 r) randomized give 8e-5, exact 4e-5 with the
// others randomized; at D=6, chi=72 (2x2, n = 3 r) 7e-5 against 3e-5.
static constexpr int kRandomizedRatio = 4;

static bool use_randomized(const Params& P, const Tensor& rhoT, int k) {
  const int n = std::min(rhoT.shape[0], rhoT.shape[1]);
  return P.mixed && n >= kRandomizedRatio * (k + P.rank_extra) && n >= P.randomized_min;
}

// Projector pairs of several cuts, pair i keeping ks[i] values; the randomized
// decompositions of pairs with equal k run as one batch.
std::vector<ProjPair> projectors(Ctx& c, const Params& P, const std::vector<Tensor>& rT, const std::vector<Tensor>& rB,
                                 const std::vector<int>& ks) {
  std::vector<ProjPair> out(rT.size());
  std::vector<int> kvals;
  for (size_t i = 0; i < rT.size(); ++i) {
    if (!use_randomized(P, rT[i], ks[i])) {
      out[i] = projector(c, P, rT[i], rB[i], ks[i]);
    } else if (std::find(kvals.begin(), kvals.end(), ks[i]) == kvals.end()) {
      kvals.push_back(ks[i]);
    }
  }
  for (int k : kvals) {
    std::vector<int> ri;
    std::vector<Tensor> bT, bB;
    for (size_t i = 0; i < rT.size(); ++i)
      if (ks[i] == k && use_randomized(P, rT[i], k)) {
        ri.push_back((int)i);
        bT.push_back(rT[i]);
        bB.push_back(rB[i]);
      }
    const int r = k + P.rank_extra;
    std::vector<Trunc> t(ri.size());
    Ctx::DecompCache& dc = c.decomp;
    if (dc.mode == 2) {
      // replay the forward pass's decompositions of this move, in call order
      SCTM_CHECK(dc.next + ri.size() <= dc.entries.size(), "decomposition cache: fewer entries than calls");
      for (size_t j = 0; j < ri.size(); ++j) {
        const std::array<Tensor, 3>& e = dc.entries[dc.next++];
        SCTM_CHECK(e[0].shape[0] == bB[j].shape[0] && e[0].shape[1] == r, "decomposition cache: shape mismatch");
        t[j] = Trunc{e[0], e[1], e[2]};
      }
    } else {
      bool tap = c.tape.active;
      c.tape.active = false;
      t = randomized_svd_batch(c, bT, bB, r, P.power_steps);
      if (dc.mode == 1) {
        for (size_t j = 0; j < ri.size(); ++j) {
          std::array<Tensor, 3> e;
          const Tensor* src[3] = {&t[j].U, &t[j].S, &t[j].V};
          for (int q = 0; q < 3; ++q) {
            Tensor d = *src[q];
            d.grad = nullptr;
            d.data = c.arena.alloc_high(src[q]->numel());
            long long st = 1;
            for (int i = d.nd - 1; i >= 0; --i) d.stride[i] = st, st *= d.shape[i];
            copy_into(c, *src[q], d);
            e[q] = d;
          }
          dc.entries.push_back(e);
        }
      }
      c.tape.active = tap;
    }
    for (size_t j = 0; j < ri.size(); ++j) out[ri[j]] = finish_randomized(c, P, bT[j], bB[j], t[j], k);
  }
  return out;
}

ProjPair projector(Ctx& c, const Params& P, const Tensor& rhoT, const Tensor& rhoB, int k) {
  const int a = rhoT.shape[0], b = rhoT.shape[1];
  SCTM_CHECK(rhoB.shape[0] == b && rhoB.shape[1] == a, "projector: rho shapes do not match");
  if (use_randomized(P, rhoT, k)) {
    bool tap = c.tape.active;
    c.tape.active = false;
    Trunc t = randomized_svd_batch(c, {rhoT}, {rhoB}, k + P.rank_extra, P.power_steps)[0];
    c.tape.active = tap;
    return finish_randomized(c, P, rhoT, rhoB, t, k);
  }
  Tensor left, right;  // core = left @ right  (n x n), P_up = w U^T left, P_dn = right V w
  if (a < b) {
    SVDResult eT = svd(c, rhoT.rev(), P.eps_l);   // rhoT^T: b x a
    SVDResult eB = svd(c, rhoB, P.eps_l);         // b x a
    Tensor LT = scale_dim(c, eT.V, 1, eT.S);      // a x a
    Tensor LB = scale_dim(c, eB.V, 1, eB.S);
    left = LB.rev();                              // L_B^T
    right = LT;
  } else {
    left = rhoB;
    right = rhoT;
  }
  Tensor M = einsum(c, "ik,kj->ij", left, right);
  const int n = M.shape[0];
  SCTM_CHECK(k <= n, "projector: chi larger than the decomposed space");
  SVDResult r = svd(c, M, P.eps_l);
  Tensor w = spectrum_map(c, r.S, k, P.cutoff, 0);
  Tensor Uk = r.U, Vk = r.V;
  Uk.shape[1] = k;   // first k columns (view)
  Vk.shape[1] = k;
  Tensor up = einsum(c, "ik,ia->ka", Uk, left);
  Tensor dn = einsum(c, "ai,ik->ak", right, Vk);
  up = scale_dim(c, up, 0, w);
  dn = scale_dim(c, dn, 1, w);
  Tensor sg = row_signs(c, up);
  up = scale_dim(c, up, 0, sg);
  dn = scale_dim(c, dn, 1, sg);
  return ProjPair{up, dn, r.S};
}

// ------------------------------------------------------------------ frames
Cell frame_transpose(Cell& cell) {
  Cell o;
  o.Lx = cell.Ly;
  o.Ly = cell.Lx;
  o.A.resize(cell.A.size());
  o.env.resize(cell.env.size());
  for (int x = 0; x < cell.Lx; ++x)
    for (int y = 0; y < cell.Ly; ++y) {
      o.a(y, x) = cell.a(x, y).perm({0, 2, 1, 4, 3});
      SiteEnv& e = cell.e(x, y);
      SiteEnv& n = o.e(y, x);
      n[C1] = e[C1].rev();  n[T1k] = e[T4k].rev(); n[T1b] = e[T4b].rev();
      n[C2] = e[C4].rev();  n[T2k] = e[T3k].rev(); n[T2b] = e[T3b].rev();
      n[C3] = e[C3].rev();  n[T3b] = e[T2b].rev(); n[T3k] = e[T2k].rev();
      n[C4] = e[C2].rev();  n[T4b] = e[T1b].rev(); n[T4k] = e[T1k].rev();
    }
  return o;
}

// 180 degree rotation with the ket and bra layers relabelled (real A): edges and
// C2/C4 keep their leg order; C1 is stored [next, previous] and C3 [previous,
// next] along the chain, so these two are transposed when they trade places.
Cell frame_rot180(Cell& cell) {
  Cell o;
  o.Lx = cell.Lx;
  o.Ly = cell.Ly;
  o.A.resize(cell.A.size());
  o.env.resize(cell.env.size());
  for (int x = 0; x < cell.Lx; ++x)
    for (int y = 0; y < cell.Ly; ++y) {
      o.a(-x, -y) = cell.a(x, y).perm({0, 3, 4, 1, 2});
      SiteEnv& e = cell.e(x, y);
      SiteEnv& n = o.e(-x, -y);
      n[C1] = e[C3].rev(); n[T1k] = e[T3b]; n[T1b] = e[T3k];
      n[C2] = e[C4];       n[T2k] = e[T4b]; n[T2b] = e[T4k];
      n[C3] = e[C1].rev(); n[T3b] = e[T1k]; n[T3k] = e[T1b];
      n[C4] = e[C2];       n[T4b] = e[T2k]; n[T4k] = e[T2b];
    }
  return o;
}

// ------------------------------------------------------------------ rho networks
static Tensor mat(const Tensor& t, int nrow_dims) {
  long long r = 1, cc = 1;
  for (int i = 0; i < t.nd; ++i) (i < nrow_dims ? r : cc) *= t.shape[i];
  return t.reshape({(int)r, (int)cc});
}

// Fig. 3a, upper box: the site's network above the cut under its bra row.
// Open (T4b.n, A.d | A'.d', T2b.g).
static Tensor green_rhoT(Ctx& c, SiteEnv& E, const Tensor& A) {
  Tensor L = einsum(c, "ab,qlb->aql", E[C1], E[T4k]);
  L = einsum(c, "aql,aui->qlui", L, E[T1k]);
  L = einsum(c, "qlui,sulkr->qiskr", L, A);
  Tensor R = einsum(c, "cf,frj->crj", E[C2], E[T2k]);
  R = einsum(c, "iwc,crj->iwrj", E[T1b], R);
  Tensor X = einsum(c, "qiskr,iwrj->qskwj", L, R);
  X = einsum(c, "qskwj,nvq->skwjnv", X, E[T4b]);
  X = einsum(c, "skwjnv,swvez->kjnez", X, A);
  return mat(einsum(c, "kjnez,jzg->nkeg", X, E[T2b]), 2);
}

// Fig. 3a, lower box (site below the cut).  Rows (A'.u', T2k.f), cols (T4k.b, A.u).
static Tensor green_rhoB(Ctx& c, SiteEnv& E, const Tensor& A) {
  Tensor Y = einsum(c, "mn,kdm->nkd", E[C4], E[T3k]);
  Y = einsum(c, "nkd,nvq->kdvq", Y, E[T4b]);
  Tensor Z = einsum(c, "gh,hek->gek", E[C3], E[T3b]);
  Z = einsum(c, "jzg,gek->jzek", E[T2b], Z);
  Y = einsum(c, "kdvq,jzek->dvqjze", Y, Z);
  Y = einsum(c, "dvqjze,swvez->dqjsw", Y, A);
  Y = einsum(c, "dqjsw,qlb->djswlb", Y, E[T4k]);
  Y = einsum(c, "djswlb,suldr->jwbur", Y, A);
  return mat(einsum(c, "jwbur,frj->wfbu", Y, E[T2k]), 2);
}

// Upper part C1 T1k T4k A T1b C2 of the site, legs [q, s, k, r, w, f]
static Tensor upper_ket_row(Ctx& c, SiteEnv& E, const Tensor& A) {
  Tensor L = einsum(c, "ab,qlb->aql", E[C1], E[T4k]);
  L = einsum(c, "aql,aui->qlui", L, E[T1k]);
  L = einsum(c, "qlui,sulkr->qiskr", L, A);
  Tensor R = einsum(c, "iwc,cf->iwf", E[T1b], E[C2]);
  return einsum(c, "qiskr,iwf->qskrwf", L, R);
}

// Fig. 8 upper box.  Rows (T4k.q, A.d), cols (A.s, T1b.u', T2k.j).
static Tensor yellow_rhoT(Ctx& c, SiteEnv& E, const Tensor& A) {
  Tensor X = upper_ket_row(c, E, A);
  return mat(einsum(c, "qskrwf,frj->qkswj", X, E[T2k]), 2);
}

// Fig. 8 lower box.  Rows (A'.s, A'.u', T2b.j), cols (T4b.q, T3k.d).
static Tensor yellow_lower(Ctx& c, SiteEnv& E, const Tensor& A) {   // [d, v, q, j, z, e]
  Tensor Y = einsum(c, "mn,kdm->nkd", E[C4], E[T3k]);
  Y = einsum(c, "nkd,nvq->kdvq", Y, E[T4b]);
  Tensor Z = einsum(c, "gh,hek->gek", E[C3], E[T3b]);
  Z = einsum(c, "jzg,gek->jzek", E[T2b], Z);
  return einsum(c, "kdvq,jzek->dvqjze", Y, Z);
}
static Tensor yellow_rhoB(Ctx& c, SiteEnv& E, const Tensor& A) {
  return mat(einsum(c, "dvqjze,swvez->swjqd", yellow_lower(c, E, A), A), 3);
}

// Alternative order (App. B): the same networks with the ket's physical leg on
// the truncated side.  Rows (T4k.q, A.d, A.s), cols (T1b.u', T2k.j); and rows
// (A'.u', T2b.j), cols (T4b.q, T3k.d, A'.s).
static Tensor yellow_alt_rhoT(Ctx& c, SiteEnv& E, const Tensor& A) {
  Tensor X = upper_ket_row(c, E, A);
  return mat(einsum(c, "qskrwf,frj->qkswj", X, E[T2k]), 3);
}
static Tensor yellow_alt_rhoB(Ctx& c, SiteEnv& E, const Tensor& A) {
  return mat(einsum(c, "dvqjze,swvez->wjqds", yellow_lower(c, E, A), A), 2);
}

// Eqs. (splitCTMRG_*), ket layer: absorb A and apply green (E-cut) and yellow
// (I-cut) projectors.  ga = green pair of the band above the site, gb = below.
static KetStage ket_stage(Ctx& c, SiteEnv& E, const Tensor& A, const ProjPair& ga, const ProjPair& y,
                          const ProjPair& gb) {
  KetStage K;
  Tensor X = einsum(c, "ab,aui->bui", E[C1], E[T1k]);
  K.C1k = einsum(c, "bui,gbu->ig", X, ga.up);
  Tensor Z = einsum(c, "bug,qlb->ugql", ga.dn, E[T4k]);
  Z = einsum(c, "ugql,suldr->gqsdr", Z, A);
  if (y.up.nd == 4) {
    // alternative order: yellow acts on (q, d, s); the physical leg moves to T4b_k
    K.T4kk = einsum(c, "gqsdr,yqds->gry", Z, y.up);
    Z = einsum(c, "qksy,nvq->ksynv", y.dn, E[T4b]);
    K.T4bk = einsum(c, "ksynv,tnk->yvts", Z, gb.up);
  } else {
    K.T4kk = einsum(c, "gqsdr,yqd->grys", Z, y.up);
    Z = einsum(c, "qky,nvq->kynv", y.dn, E[T4b]);
    K.T4bk = einsum(c, "kynv,tnk->yvt", Z, gb.up);
  }
  Z = einsum(c, "mn,kdm->nkd", E[C4], E[T3k]);
  K.C4k = einsum(c, "nkd,ndt->tk", Z, gb.dn);
  return K;
}

// column y of the upper 2x2 half after the ket stage: [r, c, t, e, z]
static Tensor upper_left_k(Ctx& c, SiteEnv& E, const Tensor& A, const KetStage& K) {
  if (K.alt()) {
    Tensor X = einsum(c, "ig,gry->iry", K.C1k, K.T4kk);
    X = einsum(c, "iry,iwc->rywc", X, E[T1b]);
    X = einsum(c, "rywc,yvts->rwcvts", X, K.T4bk);
    return einsum(c, "rwcvts,swvez->rctez", X, A);
  }
  Tensor X = einsum(c, "ig,grys->irys", K.C1k, K.T4kk);
  X = einsum(c, "irys,iwc->ryswc", X, E[T1b]);
  X = einsum(c, "ryswc,yvt->rswcvt", X, K.T4bk);
  return einsum(c, "rswcvt,swvez->rctez", X, A);
}

// column y+1 of the upper half (site (x, y+1)): [c, l, v, D, E, g]
static Tensor upper_right(Ctx& c, SiteEnv& E, const Tensor& A) {
  Tensor Y = einsum(c, "cui,iwC->cuwC", E[T1k], E[T1b]);
  Y = einsum(c, "cuwC,Cf->cuwf", Y, E[C2]);
  Y = einsum(c, "cuwf,fRj->cuwRj", Y, E[T2k]);
  Y = einsum(c, "cuwRj,jZg->cuwRZg", Y, E[T2b]);
  Y = einsum(c, "cuwRZg,SulDR->cwZgSlD", Y, A);
  return einsum(c, "cwZgSlD,SwvEZ->clvDEg", Y, A);
}

// column y of the lower half after the ket stage: [h, w, z, g, r]
static Tensor lower_left_k(Ctx& c, SiteEnv& E, const Tensor& A, const KetStage& K) {
  Tensor Z = einsum(c, "tk,hek->the", K.C4k, E[T3b]);
  if (K.alt()) {
    Z = einsum(c, "the,yvts->heyvs", Z, K.T4bk);
    Z = einsum(c, "heyvs,swvez->hywz", Z, A);
    return einsum(c, "hywz,gry->hwzgr", Z, K.T4kk);
  }
  Z = einsum(c, "the,yvt->heyv", Z, K.T4bk);
  Z = einsum(c, "heyv,swvez->hyswz", Z, A);
  return einsum(c, "hyswz,grys->hwzgr", Z, K.T4kk);
}

// column y+1 of the lower half (site (x+1, y+1)): [U, W, f, h, l, v]
static Tensor lower_right(Ctx& c, SiteEnv& E, const Tensor& A) {
  Tensor W = einsum(c, "fRj,jZG->fRZG", E[T2k], E[T2b]);
  W = einsum(c, "fRZG,GH->fRZH", W, E[C3]);
  W = einsum(c, "fRZH,HEK->fRZEK", W, E[T3b]);
  W = einsum(c, "fRZEK,KDh->fRZEDh", W, E[T3k]);
  W = einsum(c, "fRZEDh,SUlDR->fZEhSUl", W, A);
  return einsum(c, "fZEhSUl,SWvEZ->UWfhlv", W, A);
}

// teal (two-column reading): rows (T4b_k.t, A'.d'), cols (A.d, A'.d', T2b.g of y+1)
static Tensor teal_rhoT(Ctx& c, SiteEnv& E, const Tensor& A, const KetStage& K, SiteEnv& E2, const Tensor& A2) {
  Tensor R = einsum(c, "rctez,crzDEg->teDEg", upper_left_k(c, E, A, K), upper_right(c, E2, A2));
  return mat(R, 2);
}

static Tensor teal_rhoB(Ctx& c, SiteEnv& E, const Tensor& A, const KetStage& K, SiteEnv& E2, const Tensor& A2) {
  Tensor R = einsum(c, "UWfhlv,hwvgl->UWfgw", lower_right(c, E2, A2), lower_left_k(c, E, A, K));
  return mat(R, 3);
}

// red (two-column reading): rows (T4k_k.y, T4k_k.s, T1b.u'), cols (A.d, A.s, T1b.u', T2k.j of y+1)
static Tensor red_rhoT(Ctx& c, SiteEnv& E, const KetStage& K, SiteEnv& E2, const Tensor& A2) {
  Tensor X = einsum(c, "ig,grys->irys", K.C1k, K.T4kk);
  X = einsum(c, "irys,iwc->ryswc", X, E[T1b]);
  Tensor Y = einsum(c, "cui,iWC->cuWC", E2[T1k], E2[T1b]);
  Y = einsum(c, "cuWC,Cf->cuWf", Y, E2[C2]);
  Y = einsum(c, "cuWf,fRj->cuWRj", Y, E2[T2k]);
  Y = einsum(c, "cuWRj,SulDR->cWjSlD", Y, A2);
  return mat(einsum(c, "ryswc,cWjSrD->yswDSWj", X, Y), 3);
}

static Tensor red_rhoB(Ctx& c, SiteEnv& E, const Tensor& A, const KetStage& K, SiteEnv& E2, const Tensor& A2) {
  Tensor Z = einsum(c, "tk,hek->the", K.C4k, E[T3b]);
  Z = einsum(c, "the,yvt->heyv", Z, K.T4bk);
  Z = einsum(c, "heyv,swvez->hyswz", Z, A);
  Tensor W = einsum(c, "jZG,GH->jZH", E2[T2b], E2[C3]);
  W = einsum(c, "jZH,HEK->jZEK", W, E2[T3b]);
  W = einsum(c, "jZEK,KDh->jZEDh", W, E2[T3k]);
  W = einsum(c, "jZEDh,SWvEZ->jDhSWv", W, A2);
  return mat(einsum(c, "jDhSWv,hyswv->DSWjysw", W, Z), 4);
}

// red of the alternative order: rows (T4k_k.y, T1b.u'), cols (A.d, A.s, T1b.u', T2k.j of y+1)
static Tensor red_alt_rhoT(Ctx& c, SiteEnv& E, const KetStage& K, SiteEnv& E2, const Tensor& A2) {
  Tensor X = einsum(c, "ig,gry->iry", K.C1k, K.T4kk);
  X = einsum(c, "iry,iwc->rywc", X, E[T1b]);
  Tensor Y = einsum(c, "cui,iWC->cuWC", E2[T1k], E2[T1b]);
  Y = einsum(c, "cuWC,Cf->cuWf", Y, E2[C2]);
  Y = einsum(c, "cuWf,fRj->cuWRj", Y, E2[T2k]);
  Y = einsum(c, "cuWRj,SulDR->cWjSlD", Y, A2);
  return mat(einsum(c, "rywc,cWjSrD->ywDSWj", X, Y), 2);
}

// rows (T3k.d, A'.s, A'.u', T2b.j of y+1), cols (T4b_k.y, A'.u'); the bra closes T4b_k's physical leg
static Tensor red_alt_rhoB(Ctx& c, SiteEnv& E, const Tensor& A, const KetStage& K, SiteEnv& E2,
                           const Tensor& A2) {
  Tensor Z = einsum(c, "tk,hek->the", K.C4k, E[T3b]);
  Z = einsum(c, "the,yvts->heyvs", Z, K.T4bk);
  Z = einsum(c, "heyvs,swvez->hywz", Z, A);
  Tensor W = einsum(c, "jZG,GH->jZH", E2[T2b], E2[C3]);
  W = einsum(c, "jZH,HEK->jZEK", W, E2[T3b]);
  W = einsum(c, "jZEK,KDh->jZEDh", W, E2[T3k]);
  W = einsum(c, "jZEDh,SWvEZ->jDhSWv", W, A2);
  return mat(einsum(c, "jDhSWv,hywv->DSWjyw", W, Z), 4);
}

static ProjPair shaped(const ProjPair& p, int a0, int a1, int a2 = 0) {
  ProjPair q = p;
  int k = p.up.shape[0];
  if (a2) {
    q.up = p.up.reshape({k, a0, a1, a2});
    q.dn = p.dn.reshape({a0, a1, a2, k});
  } else {
    q.up = p.up.reshape({k, a0, a1});
    q.dn = p.dn.reshape({a0, a1, k});
  }
  return q;
}

// ------------------------------------------------------------------ left move
void column_projectors(Ctx& c, const Params& P, Cell& cell, int y, ColumnProj& out) {
  const int Lx = cell.Lx;
  const int D = P.D, p = P.p, chi = P.chi, chiI = P.chiI;
  out.g.resize(Lx); out.y.resize(Lx); out.t.resize(Lx); out.r.resize(Lx); out.K.resize(Lx);
  // green and teal cut environment bonds (chi_E), yellow and red interlayer ones (chi_I)
  std::vector<int> ks(2 * Lx, chi);
  for (int x = 0; x < Lx; ++x) ks[Lx + x] = chiI;
  // ket stage: green (rows x | x+1) and yellow (row x) of every row, batched
  std::vector<Tensor> rT, rB;
  for (int x = 0; x < Lx; ++x) {
    rT.push_back(green_rhoT(c, cell.e(x, y), cell.a(x, y)));
    rB.push_back(green_rhoB(c, cell.e(x + 1, y), cell.a(x + 1, y)));
  }
  const bool alt = P.order == 1;
  for (int x = 0; x < Lx; ++x) {
    rT.push_back(alt ? yellow_alt_rhoT(c, cell.e(x, y), cell.a(x, y)) : yellow_rhoT(c, cell.e(x, y), cell.a(x, y)));
    rB.push_back(alt ? yellow_alt_rhoB(c, cell.e(x, y), cell.a(x, y)) : yellow_rhoB(c, cell.e(x, y), cell.a(x, y)));
  }
  std::vector<ProjPair> pk = projectors(c, P, rT, rB, ks);
  for (int x = 0; x < Lx; ++x) {
    out.g[x] = shaped(pk[x], chi, D);
    out.y[x] = alt ? shaped(pk[Lx + x], chiI, D, p) : shaped(pk[Lx + x], chiI, D);
  }
  for (int x = 0; x < Lx; ++x)
    out.K[x] = ket_stage(c, cell.e(x, y), cell.a(x, y), out.g[(x + Lx - 1) % Lx], out.y[x], out.g[x]);
  // bra stage: teal and red of every row, batched
  rT.clear();
  rB.clear();
  for (int x = 0; x < Lx; ++x) {
    int xp = (x + 1) % Lx;
    rT.push_back(teal_rhoT(c, cell.e(x, y), cell.a(x, y), out.K[x], cell.e(x, y + 1), cell.a(x, y + 1)));
    rB.push_back(teal_rhoB(c, cell.e(xp, y), cell.a(xp, y), out.K[xp], cell.e(xp, y + 1), cell.a(xp, y + 1)));
  }
  for (int x = 0; x < Lx; ++x) {
    if (alt) {
      rT.push_back(red_alt_rhoT(c, cell.e(x, y), out.K[x], cell.e(x, y + 1), cell.a(x, y + 1)));
      rB.push_back(red_alt_rhoB(c, cell.e(x, y), cell.a(x, y), out.K[x], cell.e(x, y + 1), cell.a(x, y + 1)));
    } else {
      rT.push_back(red_rhoT(c, cell.e(x, y), out.K[x], cell.e(x, y + 1), cell.a(x, y + 1)));
      rB.push_back(red_rhoB(c, cell.e(x, y), cell.a(x, y), out.K[x], cell.e(x, y + 1), cell.a(x, y + 1)));
    }
  }
  std::vector<ProjPair> pb = projectors(c, P, rT, rB, ks);
  for (int x = 0; x < Lx; ++x) {
    out.t[x] = shaped(pb[x], chi, D);
    out.r[x] = alt ? shaped(pb[Lx + x], chiI, D) : shaped(pb[Lx + x], chiI, p, D);
  }
}

void left_move(Ctx& c, const Params& P, Cell& cell) {
  const int Lx = cell.Lx, Ly = cell.Ly;
  for (int y = 0; y < Ly; ++y) {
    ColumnProj cp;
    column_projectors(c, P, cell, y, cp);
    std::vector<KetStage>& K = cp.K;
    std::vector<ProjPair>& t = cp.t;
    std::vector<ProjPair>& r = cp.r;
    // bra layer: absorb A' and apply teal (E-cut) and red (I-cut) projectors
    std::vector<std::array<Tensor, 4>> out(Lx);
    for (int x = 0; x < Lx; ++x) {
      SiteEnv& E = cell.e(x, y);
      const Tensor& A = cell.a(x, y);
      const ProjPair& ta = t[(x + Lx - 1) % Lx];
      const ProjPair& tb = t[x];
      Tensor X = einsum(c, "ig,iwc->gwc", K[x].C1k, E[T1b]);
      Tensor nC1 = einsum(c, "gwc,Tgw->cT", X, ta.up);
      Tensor Z, nT4k;
      if (K[x].alt()) {
        // alternative order: red acts on (y, u'); the bra closes T4b_k's physical leg
        Z = einsum(c, "gwT,gry->Twry", ta.dn, K[x].T4kk);
        nT4k = einsum(c, "Twry,Pyw->PrT", Z, r[x].up);
        Z = einsum(c, "ywP,yvts->wPvts", r[x].dn, K[x].T4bk);
        Z = einsum(c, "wPvts,swvez->Ptez", Z, A);
      } else {
        Z = einsum(c, "gwT,grys->Twrys", ta.dn, K[x].T4kk);
        nT4k = einsum(c, "Twrys,Pysw->PrT", Z, r[x].up);
        Z = einsum(c, "yswP,yvt->swPvt", r[x].dn, K[x].T4bk);
        Z = einsum(c, "swPvt,swvez->Ptez", Z, A);
      }
      Tensor nT4b = einsum(c, "Ptez,Ote->OzP", Z, tb.up);
      Z = einsum(c, "tk,hek->the", K[x].C4k, E[T3b]);
      Tensor nC4 = einsum(c, "the,teO->hO", Z, tb.dn);
      out[x] = {rescale(c, nC1), rescale(c, nT4k), rescale(c, nT4b), rescale(c, nC4)};
    }
    for (int x = 0; x < Lx; ++x) {
      SiteEnv& e = cell.e(x, y + 1);
      e[C1] = out[x][0];
      e[T4k] = out[x][1];
      e[T4b] = out[x][2];
      e[C4] = out[x][3];
    }
  }
}

static void any_left_move(Ctx& c, const Params& P, Cell& cell) {
  if (P.conventional)
    conv_left_move(c, P, cell);
  else
    left_move(c, P, cell);
}

void move(Ctx& c, const Params& P, Cell& cell, int dir) {
  if (dir == 0) {
    any_left_move(c, P, cell);
  } else if (dir == 1) {
    Cell t = frame_transpose(cell);
    Params q = P;
    std::swap(q.Lx, q.Ly);
    any_left_move(c, q, t);
    cell.env = frame_transpose(t).env;
  } else if (dir == 2) {
    Cell t = frame_rot180(cell);
    any_left_move(c, P, t);
    cell.env = frame_rot180(t).env;
  } else if (dir == 3) {
    Cell t = frame_rot180(cell);
    Cell u = frame_transpose(t);
    Params q = P;
    std::swap(q.Lx, q.Ly);
    any_left_move(c, q, u);
    t.env = frame_transpose(u).env;
    cell.env = frame_rot180(t).env;
  } else {
    throw ArgError("direction must be 0..3");
  }
}

// ------------------------------------------------------------------ init
// Split a conventional edge T[P,K,K2,N] (matrix (P K) x (K2 N)) into
// first[P,K,i] = U sqrt(S) and second[i,K2,N] = sqrt(S) V^T, keeping
// min(chi_I, rank) values above the cutoff, sign fixed on the columns of U,
// zero-padded to [chi_P, K, chi_I] and [chi_I, K2, chi_N].
// Split a double-layer edge T[prev, ket leg, bra leg, next] into its ket and
// bra halves from the SVD of ((prev, ket), (bra, next)) truncated to chi_I:
// first = U sqrt(S), second = sqrt(S) V^T, each zero-padded (chi_E legs to chi_E).
static void split_edge_from(Ctx& c, const Params& P, const Tensor& T, const SVDResult& r, Tensor& first,
                            Tensor& second, int padP, int padN) {
  const int Pd = T.shape[0], Kd = T.shape[1], K2 = T.shape[2], Nd = T.shape[3];
  const int rows = Pd * Kd;
  const int k = std::min(P.chiI, rows);
  Tensor q = spectrum_map(c, r.S, k, P.cutoff, 1);
  Tensor Uk = r.U, Vk = r.V;
  Uk.shape[1] = k;
  Vk.shape[1] = k;
  Tensor sg = row_signs(c, Uk.rev());     // sign of each U column
  Tensor Us = scale_dim(c, scale_dim(c, Uk, 1, q), 1, sg);
  Tensor Vs = scale_dim(c, scale_dim(c, Vk, 1, q), 1, sg);
  first = c.zeros({padP, Kd, P.chiI});
  second = c.zeros({P.chiI, K2, padN});
  Tensor fv = first, sv = second;
  fv.shape[0] = Pd; fv.shape[2] = k;
  sv.shape[0] = k;  sv.shape[2] = Nd;
  copy_into(c, Us.reshape({Pd, Kd, k}), fv);
  copy_into(c, copy(c, Vs.rev()).reshape({k, K2, Nd}), sv);
}

void init_env(Ctx& c, const Params& P, Cell& cell) {
  if (P.conventional) {
    conv_init_env(c, P, cell);
    return;
  }
  const int D = P.D, D2 = D * D, chi = P.chi;
  SCTM_CHECK(D2 <= chi, "chi must be at least D^2 (initial corner dimension)");
  struct Pieces { Tensor c1, t1, c2, t2, c3, t3, c4, t4; };
  std::vector<Pieces> pc(cell.Lx * cell.Ly);
  for (int x = 0; x < cell.Lx; ++x)
    for (int y = 0; y < cell.Ly; ++y) {
      const Tensor& A = cell.a(x, y);
      Pieces& q = pc[x * cell.Ly + y];
      q.c1 = einsum(c, "suldr,sulez->rzde", A, A).reshape({D2, D2});
      q.t1 = einsum(c, "suldr,suvez->lvderz", A, A).reshape({D2, D, D, D2});
      q.c2 = einsum(c, "suldr,suver->lvde", A, A).reshape({D2, D2});
      q.t2 = einsum(c, "suldr,swver->uwlvde", A, A).reshape({D2, D, D, D2});
      q.c3 = einsum(c, "suldr,swvdr->uwlv", A, A).reshape({D2, D2});
      q.t3 = einsum(c, "suldr,swvdz->rzwulv", A, A).reshape({D2, D, D, D2});
      q.c4 = einsum(c, "suldr,swldz->rzuw", A, A).reshape({D2, D2});
      q.t4 = einsum(c, "suldr,swlez->dezruw", A, A).reshape({D2, D, D, D2});
    }
  auto P_ = [&](int x, int y) -> Pieces& {
    x = (x % cell.Lx + cell.Lx) % cell.Lx;
    y = (y % cell.Ly + cell.Ly) % cell.Ly;
    return pc[x * cell.Ly + y];
  };
  auto padC = [&](const Tensor& m) {
    Tensor z = c.zeros({chi, chi});
    Tensor v = z;
    v.shape[0] = D2;
    v.shape[1] = D2;
    copy_into(c, m, v);
    return z;
  };
  // every edge split of the cell in one batched SVD
  struct Job { int x, y; const Tensor* T; Key a, b; };
  std::vector<Job> jobs;
  std::vector<Tensor> mats;
  for (int x = 0; x < cell.Lx; ++x)
    for (int y = 0; y < cell.Ly; ++y) {
      SiteEnv& e = cell.e(x, y);
      e[C1] = padC(P_(x - 1, y - 1).c1);
      e[C2] = padC(P_(x - 1, y + 1).c2);
      e[C3] = padC(P_(x + 1, y + 1).c3);
      e[C4] = padC(P_(x + 1, y - 1).c4);
      jobs.push_back({x, y, &P_(x - 1, y).t1, T1k, T1b});
      jobs.push_back({x, y, &P_(x, y + 1).t2, T2k, T2b});
      jobs.push_back({x, y, &P_(x + 1, y).t3, T3b, T3k});
      jobs.push_back({x, y, &P_(x, y - 1).t4, T4b, T4k});
    }
  for (const Job& j : jobs) {
    const Tensor& T = *j.T;
    SCTM_CHECK(T.shape[0] * T.shape[1] == T.shape[2] * T.shape[3], "edge split expects a square matrix");
    mats.push_back(T.reshape({T.shape[0] * T.shape[1], T.shape[2] * T.shape[3]}));
  }
  std::vector<SVDResult> rs;
  for (size_t i0 = 0; i0 < mats.size(); i0 += 64) {   // the batched kernel takes up to 64 matrices
    std::vector<Tensor> part(mats.begin() + i0, mats.begin() + std::min(mats.size(), i0 + 64));
    std::vector<SVDResult> pr = svd_many(c, part, P.eps_l);
    rs.insert(rs.end(), pr.begin(), pr.end());
  }
  for (size_t i = 0; i < jobs.size(); ++i) {
    SiteEnv& e = cell.e(jobs[i].x, jobs[i].y);
    split_edge_from(c, P, *jobs[i].T, rs[i], e[jobs[i].a], e[jobs[i].b], chi, chi);
  }
}

// ------------------------------------------------------------------ energy
// Two-site operators h[(t_i t_j), (s_i s_j)] are decomposed on the host into
// sum_k O_k (x) Q_k (operator Schmidt decomposition of a p^2 x p^2 matrix); the
// 2x2 patch is contracted as four enlarged corners with the operator O of a
// corner applied to its site (on the bra side, see half_TL).
// Bond value = <H_top(o1,o2), H_bot(o3,o4)> / <H_top(I,I), H_bot(I,I)>; the
// products H and the reverse pass through them live in the C-ABI driver.
static void host_svd(int n, std::vector<double> a, std::vector<double>& U, std::vector<double>& S,
                     std::vector<double>& V) {
  // one-sided Jacobi on an n x n host matrix (bond operator, n = p^2)
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    bool rot = false;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) {
        double al = 0, be = 0, ga = 0;
        for (int e = 0; e < n; ++e) al += a[e * n + i] * a[e * n + i], be += a[e * n + j] * a[e * n + j],
                                    ga += a[e * n + i] * a[e * n + j];
        if (std::fabs(ga) <= 1e-15 * std::sqrt(al * be) || ga == 0) continue;
        rot = true;
        double z = (be - al) / (2 * ga);
        double t = (z >= 0 ? 1.0 : -1.0) / (std::fabs(z) + std::sqrt(1 + z * z));
        double cs = 1 / std::sqrt(1 + t * t), sn = cs * t;
        for (int e = 0; e < n; ++e) {
          double x = a[e * n + i], y = a[e * n + j];
          a[e * n + i] = cs * x - sn * y, a[e * n + j] = sn * x + cs * y;
          double vx = V[e * n + i], vy = V[e * n + j];
          V[e * n + i] = cs * vx - sn * vy, V[e * n + j] = sn * vx + cs * vy;
        }
      }
    if (!rot) break;
  }
  S.assign(n, 0.0);
  U.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double s = 0;
    for (int e = 0; e < n; ++e) s += a[e * n + i] * a[e * n + i];
    S[i] = std::sqrt(s);
    for (int e = 0; e < n; ++e) U[e * n + i] = S[i] > 0 ? a[e * n + i] / S[i] : 0;
  }
}

struct OpTerm {
  std::vector<double> O, Q;   // p x p each, O[t*p+s]
};

static std::vector<OpTerm> decompose(int p, const double* h) {
  std::vector<OpTerm> out;
  if (!h) return out;
  const int n = p * p;
  // X[(t_i s_i), (t_j s_j)] = h[(t_i t_j), (s_i s_j)]
  std::vector<double> X(n * n);
  for (int ti = 0; ti < p; ++ti)
    for (int tj = 0; tj < p; ++tj)
      for (int si = 0; si < p; ++si)
        for (int sj = 0; sj < p; ++sj)
          X[(ti * p + si) * n + (tj * p + sj)] = h[(ti * p + tj) * n + (si * p + sj)];
  std::vector<double> U, S, V;
  host_svd(n, X, U, S, V);
  double smax = 0;
  for (double s : S) smax = std::max(smax, s);
  for (int k = 0; k < n; ++k) {
    if (S[k] <= 1e-14 * smax) continue;
    OpTerm t;
    t.O.resize(n);
    t.Q.resize(n);
    for (int r = 0; r < n; ++r) t.O[r] = U[r * n + k] * S[k], t.Q[r] = V[r * n + k];
    out.push_back(t);
  }
  return out;
}

static Tensor fuse_edge(Ctx& c, const Tensor& a, const Tensor& b, const char* spec) { return einsum(c, spec, a, b); }

// Enlarged corners (conventional edges): the environment part and the ket
// layer form an operator-independent half; the bra layer closes it.  A
// one-site operator O of the energy sits on the bra side, Ab = O^T A, which
// equals replacing the ket by O A: sum_{s,t} O[t,s] A[s] A[t].
static Tensor half_TL(Ctx& c, const Tensor& C1t, const Tensor& T1, const Tensor& T4, const Tensor& A) {
  Tensor X = einsum(c, "ab,auwc->buwc", C1t, T1);
  X = einsum(c, "buwc,nvlb->uwcnvl", X, T4);
  return einsum(c, "uwcnvl,suldr->wcnvsdr", X, A);
}
static Tensor finish_TL(Ctx& c, const Tensor& X, const Tensor& Ab) {
  return mat(einsum(c, "wcnvsdr,swvez->crznde", X, Ab), 3);   // [(c,r,z), (n,d,e)]
}
static Tensor half_TR(Ctx& c, const Tensor& T1, const Tensor& C2t, const Tensor& T2, const Tensor& A) {
  Tensor Y = einsum(c, "auwc,cf->auwf", T1, C2t);
  Y = einsum(c, "auwf,frzg->auwrzg", Y, T2);
  return einsum(c, "auwrzg,suldr->awzgsld", Y, A);
}
static Tensor finish_TR(Ctx& c, const Tensor& Y, const Tensor& Ab) {
  return mat(einsum(c, "awzgsld,swvez->alvdeg", Y, Ab), 3);   // [(a,l,v), (d,e,g)]
}
static Tensor half_BR(Ctx& c, const Tensor& T2, const Tensor& C3t, const Tensor& T3, const Tensor& A) {
  Tensor Z = einsum(c, "frzg,gh->frzh", T2, C3t);
  Z = einsum(c, "frzh,hedm->frzedm", Z, T3);
  return einsum(c, "frzedm,suldr->fzemsul", Z, A);
}
static Tensor finish_BR(Ctx& c, const Tensor& Z, const Tensor& Ab) {
  return mat(einsum(c, "fzemsul,swvez->uwflvm", Z, Ab), 3);   // [(u,w,f), (l,v,m)]
}
static Tensor half_BL(Ctx& c, const Tensor& T4, const Tensor& C4t, const Tensor& T3, const Tensor& A) {
  Tensor W = einsum(c, "hedm,mn->hedn", T3, C4t);
  W = einsum(c, "hedn,nvlb->hedvlb", W, T4);
  return einsum(c, "hedvlb,suldr->hevbsur", W, A);
}
static Tensor finish_BL(Ctx& c, const Tensor& W, const Tensor& Ab) {
  return mat(einsum(c, "hevbsur,swvez->buwrzh", W, Ab), 3);   // [(b,u,w), (r,z,h)]
}

EnergyOps energy_ops(Ctx& c, const Params& P, const double* h_nn, const double* h_diag) {
  const int p = P.p;
  std::vector<OpTerm> tn = decompose(p, h_nn), td = decompose(p, h_diag);
  // operator list: index 0 = identity; operators equal up to a factor share one
  // slot (Heisenberg: every factor of every bond), so corners are built once
  std::vector<std::vector<double>> ops;
  std::vector<double> I(p * p, 0.0);
  for (int i = 0; i < p; ++i) I[i * p + i] = 1.0;
  ops.push_back(I);
  auto intern = [&](const std::vector<double>& O, double& scale) -> int {
    int im = 0;
    for (int i = 1; i < (int)O.size(); ++i)
      if (std::fabs(O[i]) > std::fabs(O[im])) im = i;
    scale = O[im];
    std::vector<double> v(O.size());
    for (size_t i = 0; i < O.size(); ++i) v[i] = O[i] / scale;
    for (size_t j = 1; j < ops.size(); ++j) {
      double d = 0;
      for (size_t i = 0; i < v.size(); ++i) d = std::max(d, std::fabs(v[i] - ops[j][i]));
      if (d < 1e-12) return (int)j;
    }
    ops.push_back(v);
    return (int)ops.size() - 1;
  };
  EnergyOps E;
  std::vector<EnergyOps::Pair>& nnp = E.nn;
  std::vector<EnergyOps::Pair>& dgp = E.diag;
  for (auto& t : tn) {
    double sa, sb;
    int a = intern(t.O, sa), b = intern(t.Q, sb);
    nnp.push_back({a, b, sa * sb});
  }
  for (auto& t : td) {
    double sa, sb;
    int a = intern(t.O, sa), b = intern(t.Q, sb);
    dgp.push_back({a, b, sa * sb});
  }
  E.op.resize(ops.size());
  for (size_t i = 0; i < ops.size(); ++i) {
    bool t = c.tape.active;
    c.tape.active = false;
    E.op[i] = from_host(c, {p, p}, ops[i].data());
    c.tape.active = t;
  }
  return E;
}

std::vector<PatchTerm> patch_terms(const EnergyOps& E, int nsites) {
  std::vector<PatchTerm> t;
  const double inv_n = 1.0 / nsites;
  // nearest-neighbour bonds, half weight each (every bond lies in two patches)
  for (const auto& pr : E.nn) {
    const int o = pr.a, q = pr.b;
    const double w = 0.5 * inv_n * pr.w;
    t.push_back({o, q, 0, 0, w});   // top    (TL, TR)
    t.push_back({0, 0, o, q, w});   // bottom (BL, BR)
    t.push_back({o, 0, q, 0, w});   // left   (TL, BL)
    t.push_back({0, o, 0, q, w});   // right  (TR, BR)
  }
  for (const auto& pr : E.diag) {
    const int o = pr.a, q = pr.b;
    const double w = inv_n * pr.w;
    t.push_back({o, 0, 0, q, w});   // TL - BR
    t.push_back({0, o, q, 0, w});   // TR - BL
  }
  return t;
}

PatchCorners patch_corners(Ctx& c, const Params& P, Cell& cell, const EnergyOps& E,
                           const std::vector<PatchTerm>& terms, int x, int y) {
  const std::vector<Tensor>& opd = E.op;
  const size_t nops = opd.size();
  SiteEnv& eTL = cell.e(x, y);
  SiteEnv& eTR = cell.e(x, y + 1);
  SiteEnv& eBR = cell.e(x + 1, y + 1);
  SiteEnv& eBL = cell.e(x + 1, y);
  // conventional environments hold the fused edges already
  auto fused = [&](const Tensor& a, const Tensor& b, const char* spec) {
    return P.conventional ? a : fuse_edge(c, a, b, spec);
  };
  Tensor T1L = fused(eTL[T1k], eTL[T1b], "aui,iwc->auwc");
  Tensor T4T = fused(eTL[T4b], eTL[T4k], "nvq,qlb->nvlb");
  Tensor T1R = fused(eTR[T1k], eTR[T1b], "aui,iwc->auwc");
  Tensor T2T = fused(eTR[T2k], eTR[T2b], "frj,jzg->frzg");
  Tensor T2B = fused(eBR[T2k], eBR[T2b], "frj,jzg->frzg");
  Tensor T3R = fused(eBR[T3b], eBR[T3k], "hek,kdm->hedm");
  Tensor T3L = fused(eBL[T3b], eBL[T3k], "hek,kdm->hedm");
  Tensor T4B = fused(eBL[T4b], eBL[T4k], "nvq,qlb->nvlb");
  const Tensor& aTL = cell.a(x, y);
  const Tensor& aTR = cell.a(x, y + 1);
  const Tensor& aBR = cell.a(x + 1, y + 1);
  const Tensor& aBL = cell.a(x + 1, y);
  std::vector<char> nTL(nops, 0), nTR(nops, 0), nBR(nops, 0), nBL(nops, 0);
  nTL[0] = nTR[0] = nBR[0] = nBL[0] = 1;   // the norm <Htop(0,0), Hbot(0,0)>
  for (const PatchTerm& t : terms) nTL[t.t1] = nTR[t.t2] = nBL[t.b1] = nBR[t.b2] = 1;
  auto bra = [&](int o, const Tensor& a) { return o ? einsum(c, "ts,tuldr->suldr", opd[o], a) : a; };
  PatchCorners K;
  K.TL.resize(nops), K.TR.resize(nops), K.BR.resize(nops), K.BL.resize(nops);
  // operator-independent halves, built once; the bra layer closes them
  Tensor h = half_TL(c, eTL[C1], T1L, T4T, aTL);
  for (size_t o = 0; o < nops; ++o)
    if (nTL[o]) K.TL[o] = finish_TL(c, h, bra((int)o, aTL));
  h = half_TR(c, T1R, eTR[C2], T2T, aTR);
  for (size_t o = 0; o < nops; ++o)
    if (nTR[o]) K.TR[o] = finish_TR(c, h, bra((int)o, aTR));
  h = half_BR(c, T2B, eBR[C3], T3R, aBR);
  for (size_t o = 0; o < nops; ++o)
    if (nBR[o]) K.BR[o] = finish_BR(c, h, bra((int)o, aBR));
  h = half_BL(c, T4B, eBL[C4], T3L, aBL);
  for (size_t o = 0; o < nops; ++o)
    if (nBL[o]) K.BL[o] = finish_BL(c, h, bra((int)o, aBL));
  return K;
}

// ------------------------------------------------------------------ conventional CTMRG
// The double-layer (conventional) directional CTMRG that the paper benchmarks
// the split scheme against (Sec. III), with the 2x2-patch projectors of
// Corboz et al.: an edge is the fused ket-bra pair [previous, ket leg, bra leg,
// next] (the contraction of a split pair over the interlayer bond, Sec. II.B),
// stored in both slots of its pair (T1k = T1b, T2k = T2b, T3b = T3k,
// T4b = T4k), so the transposed and rotated frames of the split environment
// map it unchanged.

void conv_init_env(Ctx& c, const Params& P, Cell& cell) {
  const int D = P.D, D2 = D * D, chi = P.chi;
  SCTM_CHECK(D2 <= chi, "chi must be at least D^2 (initial corner dimension)");
  struct Pieces { Tensor c1, t1, c2, t2, c3, t3, c4, t4; };
  std::vector<Pieces> pc(cell.Lx * cell.Ly);
  for (int x = 0; x < cell.Lx; ++x)
    for (int y = 0; y < cell.Ly; ++y) {
      const Tensor& A = cell.a(x, y);
      Pieces& q = pc[x * cell.Ly + y];
      q.c1 = einsum(c, "suldr,sulez->rzde", A, A).reshape({D2, D2});
      q.t1 = einsum(c, "suldr,suvez->lvderz", A, A).reshape({D2, D, D, D2});
      q.c2 = einsum(c, "suldr,suver->lvde", A, A).reshape({D2, D2});
      q.t2 = einsum(c, "suldr,swver->uwlvde", A, A).reshape({D2, D, D, D2});
      q.c3 = einsum(c, "suldr,swvdr->uwlv", A, A).reshape({D2, D2});
      q.t3 = einsum(c, "suldr,swvdz->rzwulv", A, A).reshape({D2, D, D, D2});
      q.c4 = einsum(c, "suldr,swldz->rzuw", A, A).reshape({D2, D2});
      q.t4 = einsum(c, "suldr,swlez->dezruw", A, A).reshape({D2, D, D, D2});
    }
  auto P_ = [&](int x, int y) -> Pieces& {
    x = (x % cell.Lx + cell.Lx) % cell.Lx;
    y = (y % cell.Ly + cell.Ly) % cell.Ly;
    return pc[x * cell.Ly + y];
  };
  auto padC = [&](const Tensor& m) {
    Tensor z = c.zeros({chi, chi});
    Tensor v = z;
    v.shape[0] = D2;
    v.shape[1] = D2;
    copy_into(c, m, v);
    return z;
  };
  auto padT = [&](const Tensor& t) {
    Tensor z = c.zeros({chi, D, D, chi});
    Tensor v = z;
    v.shape[0] = D2;
    v.shape[3] = D2;
    copy_into(c, t, v);
    return z;
  };
  for (int x = 0; x < cell.Lx; ++x)
    for (int y = 0; y < cell.Ly; ++y) {
      SiteEnv& e = cell.e(x, y);
      e[C1] = padC(P_(x - 1, y - 1).c1);
      e[C2] = padC(P_(x - 1, y + 1).c2);
      e[C3] = padC(P_(x + 1, y + 1).c3);
      e[C4] = padC(P_(x + 1, y - 1).c4);
      e[T1k] = e[T1b] = padT(P_(x - 1, y).t1);
      e[T2k] = e[T2b] = padT(P_(x, y + 1).t2);
      e[T3b] = e[T3k] = padT(P_(x + 1, y).t3);
      e[T4b] = e[T4k] = padT(P_(x, y - 1).t4);
    }
}

void conv_left_move(Ctx& c, const Params& P, Cell& cell) {
  const int Lx = cell.Lx, Ly = cell.Ly, D = P.D, k = P.chi;
  for (int y = 0; y < Ly; ++y) {
    // projectors of the cuts below every row of column y: upper half TL^T TR,
    // lower half BR BL^T of the 2x2 patch anchored at (x, y)
    std::vector<Tensor> rT(Lx), rB(Lx);
    for (int x = 0; x < Lx; ++x) {
      SiteEnv& eTL = cell.e(x, y);
      SiteEnv& eTR = cell.e(x, y + 1);
      SiteEnv& eBR = cell.e(x + 1, y + 1);
      SiteEnv& eBL = cell.e(x + 1, y);
      const Tensor& aTL = cell.a(x, y);
      const Tensor& aTR = cell.a(x, y + 1);
      const Tensor& aBR = cell.a(x + 1, y + 1);
      const Tensor& aBL = cell.a(x + 1, y);
      Tensor TL = finish_TL(c, half_TL(c, eTL[C1], eTL[T1k], eTL[T4k], aTL), aTL);   // [(c,r,z), (n,d,e)]
      Tensor TR = finish_TR(c, half_TR(c, eTR[T1k], eTR[C2], eTR[T2k], aTR), aTR);   // [(a,l,v), (d,e,g)]
      Tensor BR = finish_BR(c, half_BR(c, eBR[T2k], eBR[C3], eBR[T3k], aBR), aBR);   // [(u,w,f), (l,v,m)]
      Tensor BL = finish_BL(c, half_BL(c, eBL[T4k], eBL[C4], eBL[T3k], aBL), aBL);   // [(b,u,w), (r,z,h)]
      rT[x] = einsum(c, "ra,rb->ab", TL, TR);   // alpha = TL's lower cut (n,d,e)  x  beta
      rB[x] = einsum(c, "al,bl->ab", BR, BL);   // beta x alpha
    }
    std::vector<ProjPair> pp = projectors(c, P, rT, rB, std::vector<int>(rT.size(), P.chi));
    const int n = cell.e(0, y)[T4k].shape[0];
    std::vector<std::array<Tensor, 3>> out(Lx);
    for (int x = 0; x < Lx; ++x) {
      SiteEnv& e = cell.e(x, y);
      const Tensor& a = cell.a(x, y);
      const ProjPair& pa = pp[(x + Lx - 1) % Lx];   // cut above row x
      const ProjPair& pb = pp[x];                   // cut below row x
      Tensor pua = pa.up.reshape({k, n, D, D}), pda = pa.dn.reshape({n, D, D, k});
      Tensor pub = pb.up.reshape({k, n, D, D}), pdb = pb.dn.reshape({n, D, D, k});
      Tensor X = einsum(c, "ab,auwc->buwc", e[C1], e[T1k]);
      Tensor nC1 = einsum(c, "buwc,kbuw->ck", X, pua);
      Tensor Z = einsum(c, "buwK,nvlb->uwKnvl", pda, e[T4k]);
      Z = einsum(c, "uwKnvl,suldr->wKnvsdr", Z, a);
      Z = einsum(c, "wKnvsdr,swvez->Kndrez", Z, a);
      Tensor nT4 = einsum(c, "Kndrez,Mnde->MzrK", Z, pub);
      Z = einsum(c, "mn,hedm->nhed", e[C4], e[T3k]);
      Tensor nC4 = einsum(c, "nhed,ndeK->hK", Z, pdb);
      out[x] = {rescale(c, nC1), rescale(c, nT4), rescale(c, nC4)};
    }
    for (int x = 0; x < Lx; ++x) {
      SiteEnv& e = cell.e(x, y + 1);
      e[C1] = out[x][0];
      e[T4b] = e[T4k] = out[x][1];
      e[C4] = out[x][2];
    }
  }
}

}  // namespace sctm
