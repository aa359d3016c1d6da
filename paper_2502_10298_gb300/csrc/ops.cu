// Differentiable device operations (see ops.h).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>

#include "ops.h"
#include "prof.h"

namespace sctm {

// ------------------------------------------------------------------ arena
Arena::~Arena() {
  if (base_) cudaFree(base_);
}

void Arena::reserve(size_t bytes) {
  if (base_) cudaFree(base_);
  base_ = nullptr;
  SCTM_CUDA(cudaMalloc(&base_, bytes));
  cap_ = bytes & ~(size_t)255;
  top_ = 0;
  hi_ = cap_;
}

double* Arena::alloc(long long n) {
  size_t bytes = ((size_t)std::max<long long>(n, 1) * sizeof(double) + 255) & ~(size_t)255;
  if (top_ + bytes > hi_)
    throw ArgError("device workspace exhausted (" + std::to_string((top_ + bytes + cap_ - hi_) >> 20) +
                   " MiB needed, " + std::to_string(cap_ >> 20) + " MiB reserved)");
  double* p = reinterpret_cast<double*>(base_ + top_);
  top_ += bytes;
  high_ = std::max(high_, top_ + (cap_ - hi_));
  return p;
}

double* Arena::alloc_high(long long n) {
  size_t bytes = ((size_t)std::max<long long>(n, 1) * sizeof(double) + 255) & ~(size_t)255;
  if (hi_ < top_ + bytes)
    throw ArgError("device workspace exhausted (" + std::to_string((top_ + bytes + cap_ - hi_) >> 20) +
                   " MiB needed, " + std::to_string(cap_ >> 20) + " MiB reserved)");
  hi_ -= bytes;
  high_ = std::max(high_, top_ + (cap_ - hi_));
  return reinterpret_cast<double*>(base_ + hi_);
}

Tensor Tensor::reshape(std::initializer_list<int> s) const {
  SCTM_CHECK(contiguous(), "reshape of a non-contiguous view");
  Tensor t;
  t.data = data;
  t.grad = grad;
  t.nd = (int)s.size();
  long long n = 1;
  int i = 0;
  for (int v : s) t.shape[i++] = v, n *= v;
  SCTM_CHECK(n == numel(), "reshape size mismatch");
  long long st = 1;
  for (int j = t.nd - 1; j >= 0; --j) t.stride[j] = st, st *= t.shape[j];
  return t;
}

// ------------------------------------------------------------------ ctx
Tensor Ctx::empty_shape(const int* shape, int nd) {
  Tensor t;
  t.nd = nd;
  long long st = 1;
  for (int j = nd - 1; j >= 0; --j) t.shape[j] = shape[j], t.stride[j] = st, st *= shape[j];
  t.data = arena.alloc(st);
  if (tape.active) {
    t.grad = arena.alloc(st);
    SCTM_CUDA(cudaMemsetAsync(t.grad, 0, st * sizeof(double), stream));
  }
  return t;
}

Tensor Ctx::empty(std::initializer_list<int> shape) {
  int s[kMaxDims];
  int i = 0;
  for (int v : shape) s[i++] = v;
  return empty_shape(s, i);
}

Tensor Ctx::zeros(std::initializer_list<int> shape) {
  Tensor t = empty(shape);
  SCTM_CUDA(cudaMemsetAsync(t.data, 0, t.numel() * sizeof(double), stream));
  return t;
}

Tensor Ctx::scalar() { return zeros({1}); }

void Ctx::zero_grad(const Tensor& t) {
  if (t.grad) SCTM_CUDA(cudaMemsetAsync(t.grad, 0, t.numel() * sizeof(double), stream));
}

void Ctx::ensure_grad(Tensor& t) {
  if (!t.grad) {
    SCTM_CHECK(t.contiguous(), "gradient buffer for a non-contiguous view");
    t.grad = arena.alloc(t.numel());
  }
  zero_grad(t);
}

static Tensor grad_view(const Tensor& t) {
  Tensor g = t;
  g.data = t.grad;
  g.grad = nullptr;
  return g;
}

// ------------------------------------------------------------------ einsum
struct Spec {
  std::string a, b, c;
};

static Spec parse(const char* spec) {
  std::string s(spec);
  size_t comma = s.find(','), arrow = s.find("->");
  SCTM_CHECK(comma != std::string::npos && arrow != std::string::npos, std::string("bad einsum spec ") + spec);
  return Spec{s.substr(0, comma), s.substr(comma + 1, arrow - comma - 1), s.substr(arrow + 2)};
}

static ContractDesc plan(const Spec& sp, const Tensor& A, const Tensor& B, const Tensor& C) {
  SCTM_CHECK((int)sp.a.size() == A.nd && (int)sp.b.size() == B.nd && (int)sp.c.size() == C.nd,
             "einsum rank mismatch: " + sp.a + "," + sp.b + "->" + sp.c);
  struct L {
    int size = -1;
    long long sa = 0, sb = 0, sc = 0;
    bool ia = false, ib = false, ic = false;
  };
  std::map<char, L> ls;
  std::string order;
  auto note = [&](char ch) {
    if (!ls.count(ch)) order.push_back(ch);
    return &ls[ch];
  };
  for (int i = 0; i < A.nd; ++i) {
    L* l = note(sp.a[i]);
    SCTM_CHECK(l->size < 0 || l->size == A.shape[i], "einsum size mismatch (A) in " + sp.a);
    l->size = A.shape[i], l->sa += A.stride[i], l->ia = true;
  }
  for (int i = 0; i < B.nd; ++i) {
    L* l = note(sp.b[i]);
    SCTM_CHECK(l->size < 0 || l->size == B.shape[i], "einsum size mismatch (B) in " + sp.a + "," + sp.b);
    l->size = B.shape[i], l->sb += B.stride[i], l->ib = true;
  }
  for (int i = 0; i < C.nd; ++i) {
    L* l = note(sp.c[i]);
    SCTM_CHECK(l->size < 0 || l->size == C.shape[i], "einsum size mismatch (C) in " + sp.c);
    l->size = C.shape[i], l->sc += C.stride[i], l->ic = true;
  }
  ContractDesc d;
  std::vector<char> gb, gm, gn, gk;
  for (char ch : order) {
    L& l = ls[ch];
    if (l.ia && l.ib && l.ic) gb.push_back(ch);
    else if (l.ia && l.ic) gm.push_back(ch);
    else if (l.ib && l.ic) gn.push_back(ch);
    else if (l.ia && l.ib) gk.push_back(ch);
    else SCTM_CHECK(false, std::string("einsum index only in one operand: ") + ch);
  }
  auto absl = [](long long v) { return v < 0 ? -v : v; };
  // within a group, the dim with the smallest stride of the operand that loads it goes last
  std::sort(gm.begin(), gm.end(), [&](char x, char y) { return absl(ls[x].sa) > absl(ls[y].sa); });
  std::sort(gk.begin(), gk.end(), [&](char x, char y) { return absl(ls[x].sa) > absl(ls[y].sa); });
  std::sort(gn.begin(), gn.end(), [&](char x, char y) { return absl(ls[x].sb) > absl(ls[y].sb); });
  auto fill = [&](Group& g, const std::vector<char>& v, long long& tot) {
    SCTM_CHECK((int)v.size() <= kMaxDims, "too many dims in an einsum group");
    g.nd = (int)v.size();
    tot = 1;
    for (int i = 0; i < g.nd; ++i) {
      L& l = ls[v[i]];
      g.size[i] = l.size, g.sa[i] = l.sa, g.sb[i] = l.sb, g.sc[i] = l.sc;
      tot *= l.size;
    }
  };
  fill(d.bat, gb, d.B);
  fill(d.m, gm, d.M);
  fill(d.n, gn, d.N);
  fill(d.k, gk, d.K);
  d.a_k_inner = 1;
  if (d.k.nd && absl(d.k.sa[d.k.nd - 1]) == 1) d.a_k_inner = 1;
  else if (d.m.nd && absl(d.m.sa[d.m.nd - 1]) == 1) d.a_k_inner = 0;
  d.b_n_inner = 1;
  if (d.n.nd && absl(d.n.sb[d.n.nd - 1]) == 1) d.b_n_inner = 1;
  else if (d.k.nd && absl(d.k.sb[d.k.nd - 1]) == 1) d.b_n_inner = 0;
  return d;
}

// The packed slice panel of an operand whose data pointer the current scope
// keeps (Ctx::slice_keep): packed into the arena's high stack on first use with
// this layout, reused afterwards.  Null for operands that are not kept.
static const SlicePanel* kept_slice_panel(Ctx& c, const ContractDesc& d, bool b_operand, const double* X,
                                          SlicePanel& out) {
  if (std::find(c.slice_keep.begin(), c.slice_keep.end(), X) == c.slice_keep.end()) return nullptr;
  const Group& rows = b_operand ? d.n : d.m;
  std::vector<long long> key{(long long)(uintptr_t)X, b_operand ? d.N : d.M, d.K, d.B};
  for (const Group* g : {&d.bat, &rows, &d.k}) {
    key.push_back(g->nd);
    for (int i = 0; i < g->nd; ++i) key.push_back(g->size[i]), key.push_back(b_operand ? g->sb[i] : g->sa[i]);
  }
  for (const auto& e : c.slice_panels)
    if (e.first == key) {
      out = e.second;
      return &out;
    }
  void* dst = c.arena.alloc_high((long long)(slice_panel_bytes(d, b_operand) + 7) / 8);
  out = slice_pack(d, b_operand, X, dst, c.stream);
  c.slice_panels.push_back({key, out});
  return &out;
}

// Split-K autotuner.  Contractions whose output has too few tiles to fill the
// GPU can split K over more CTAs; the kernels choose the count by a rule.
// With Ctx::autotune on, the first calls of each such shape (kernel, batch,
// M, N, K) run with the rule's count, half and twice it and no split, one per
// call -- each a complete contraction -- timed with events on the stream, and
// later calls use the fastest.  Returns the split count to request (0: rule).
static int tune_splits(Ctx& c, int kernel, const ContractDesc& d, int rule, int maxs, Ctx::Tune** slot) {
  *slot = nullptr;
  if (maxs < 2) return 0;
  const std::vector<long long> key{kernel, d.B, d.M, d.N, d.K};
  auto it = c.tune.find(key);
  if (it == c.tune.end()) {
    if (!c.autotune) return 0;
    Ctx::Tune t;
    for (int v : {rule, std::max(1, rule / 2), std::min(maxs, 2 * rule), 1})
      if (std::find(t.cand.begin(), t.cand.end(), v) == t.cand.end()) t.cand.push_back(v);
    t.ms.assign(t.cand.size(), 0.f);
    SCTM_CUDA(cudaEventCreate(&t.e0));
    SCTM_CUDA(cudaEventCreate(&t.e1));
    it = c.tune.emplace(key, t).first;
  }
  Ctx::Tune& t = it->second;
  if (t.pending >= 0) {   // the previous call's timing
    SCTM_CUDA(cudaEventSynchronize(t.e1));
    SCTM_CUDA(cudaEventElapsedTime(&t.ms[t.pending], t.e0, t.e1));
    t.pending = -1;
    if (t.next == (int)t.cand.size())
      t.chosen = t.cand[std::min_element(t.ms.begin(), t.ms.end()) - t.ms.begin()];
  }
  if (t.chosen) return t.chosen;
  if (!c.autotune || t.next >= (int)t.cand.size()) return 0;
  t.pending = t.next++;
  *slot = &t;
  return t.cand[t.pending];
}

void einsum_into(Ctx& c, const char* spec, const Tensor& A, const Tensor& B, const Tensor& C, double alpha,
                 double beta, bool record) {
  Spec sp = parse(spec);
  ContractDesc d = plan(sp, A, B, C);
  d.alpha = alpha;
  d.beta = beta;
  if (prof_enabled()) {
    char tag[160];
    std::snprintf(tag, sizeof(tag), "%s B%lld M%lld N%lld K%lld%s", spec, d.B, d.M, d.N, d.K,
                  c.fp32_compute ? "" : " f64");
    prof_set_tag(tag);
  }
  // inside an accurate scope of the BF16-slice mode, every contraction whose
  // shape fits the tiles takes the slice kernel and the rest run in FP64
  const bool accurate = c.bf16_slices && c.accurate > 0 && c.fp32_compute;
  Ctx::Tune* timed = nullptr;
  if (c.fp32_compute && c.tensor_cores && (accurate ? tc_shape_ok(d) : tc_eligible(d))) {
    size_t mk = c.arena.mark();
    if (c.bf16_slices) {
      SlicePanel pa, pb;
      const SlicePanel* ppa = kept_slice_panel(c, d, false, A.data, pa);
      const SlicePanel* ppb = kept_slice_panel(c, d, true, B.data, pb);
      void* scratch = c.arena.alloc((long long)(slice_scratch_bytes(d) + 7) / 8);
      const int sp = tune_splits(c, 3, d, slice_split_rule(d), slice_split_max(d), &timed);
      if (timed) SCTM_CUDA(cudaEventRecord(timed->e0, c.stream));
      launch_contract_slices(d, A.data, B.data, C.data, c.stream, scratch, c.svd_status + 32, c.pipe_wait_ns, ppa, ppb,
                             sp);
    } else {
      float* scratch = reinterpret_cast<float*>(c.arena.alloc((long long)(tc_scratch_floats(d) + 1) / 2));
      const int sp = tune_splits(c, 2, d, tc_split_rule(d), tc_split_max(d), &timed);
      if (timed) SCTM_CUDA(cudaEventRecord(timed->e0, c.stream));
      launch_contract_tc(d, A.data, B.data, C.data, c.stream, scratch, c.svd_status + 32, c.pipe_wait_ns, sp);
    }
    c.arena.release(mk);   // stream-ordered: later work on the stream reuses it after the GEMM
  } else {
    const size_t wn = contract_scratch_doubles(d);
    size_t mk = c.arena.mark();
    double* scratch = wn ? c.arena.alloc((long long)wn) : nullptr;
    const bool f32 = c.fp32_compute && !accurate;
    const int sp = tune_splits(c, f32 ? 1 : 0, d, contract_split_rule(d), contract_split_max(d), &timed);
    if (timed) SCTM_CUDA(cudaEventRecord(timed->e0, c.stream));
    launch_contract<double>(d, A.data, B.data, C.data, c.stream, f32, scratch, sp);
    c.arena.release(mk);
  }
  if (timed) SCTM_CUDA(cudaEventRecord(timed->e1, c.stream));
  if (prof_enabled()) prof_set_tag("");
  if (!record || !c.tape.active || !C.grad) return;
  std::string sa = sp.c + "," + sp.b + "->" + sp.a;
  std::string sb = sp.a + "," + sp.c + "->" + sp.b;
  Tensor a = A, b = B, cc = C;
  c.tape.push([&c, sa, sb, a, b, cc, alpha]() {
    Tensor gc = grad_view(cc);
    if (a.grad) einsum_into(c, sa.c_str(), gc, b, grad_view(a), alpha, 1.0, false);
    if (b.grad) einsum_into(c, sb.c_str(), a, gc, grad_view(b), alpha, 1.0, false);
  });
}

Tensor einsum(Ctx& c, const char* spec, const Tensor& A, const Tensor& B, double alpha) {
  Spec sp = parse(spec);
  int shape[kMaxDims];
  for (size_t i = 0; i < sp.c.size(); ++i) {
    char ch = sp.c[i];
    int sz = -1;
    for (int j = 0; j < A.nd; ++j)
      if (sp.a[j] == ch) sz = A.shape[j];
    for (int j = 0; j < B.nd; ++j)
      if (sp.b[j] == ch) sz = B.shape[j];
    SCTM_CHECK(sz >= 0, std::string("output index not found in inputs: ") + spec);
    shape[i] = sz;
  }
  Tensor C = c.empty_shape(shape, (int)sp.c.size());
  einsum_into(c, spec, A, B, C, alpha, 0.0, true);
  return C;
}

// ------------------------------------------------------------------ copies
static Group copy_group(const Tensor& X, const Tensor& Y) {
  SCTM_CHECK(X.nd == Y.nd, "copy rank mismatch");
  Group g;
  g.nd = X.nd;
  for (int i = 0; i < X.nd; ++i) {
    SCTM_CHECK(X.shape[i] == Y.shape[i], "copy shape mismatch");
    g.size[i] = X.shape[i], g.sa[i] = X.stride[i], g.sc[i] = Y.stride[i];
  }
  return g;
}

void copy_into(Ctx& c, const Tensor& X, const Tensor& Y) {
  launch_copy<double>(copy_group(X, Y), 1.0, X.data, 0.0, Y.data, c.stream);
  if (!c.tape.active || !Y.grad || !X.grad) return;
  Tensor x = X, y = Y;
  c.tape.push([&c, x, y]() {
    Group g = copy_group(grad_view(y), grad_view(x));
    launch_copy<double>(g, 1.0, y.grad, 1.0, x.grad, c.stream);
  });
}

Tensor copy(Ctx& c, const Tensor& X) {
  Tensor Y = c.empty_shape(X.shape, X.nd);
  copy_into(c, X, Y);
  return Y;
}

// ------------------------------------------------------------------ svd
// Reverse pass of M = U S V^T (square or tall):
// M_bar = U [ F o (J - J^T) S + diag(S_bar) + S F o (K - K^T) ] V^T,
// J = U^T U_bar, K = V^T V_bar.  For m > n the projector code uses only S and V
// (U_bar = 0), so the (1 - U U^T) U_bar S^-1 V^T term of the thin SVD vanishes.
static void record_svd_adjoint(Ctx& c, const SVDResult& r, const Tensor& Min, double eps_l) {
  const int m = r.U.shape[0], n = r.U.shape[1];
  Tensor U = r.U, S = r.S, V = r.V;
  c.tape.push([&c, U, S, V, Min, m, n, eps_l]() {
    bool t = c.tape.active;
    c.tape.active = false;
    Tensor gU = grad_view(U), gV = grad_view(V), gS = grad_view(S);
    Tensor J = c.empty({n, n}), K = c.empty({n, n}), inner = c.empty({n, n});
    einsum_into(c, "ai,aj->ij", U, gU, J, 1.0, 0.0, false);
    einsum_into(c, "ai,aj->ij", V, gV, K, 1.0, 0.0, false);
    launch_svd_adj_inner(n, S.data, J.data, K.data, gS.data, inner.data, eps_l, c.stream);
    Tensor T1 = c.empty({m, n});
    einsum_into(c, "ai,ij->aj", U, inner, T1, 1.0, 0.0, false);
    einsum_into(c, "aj,bj->ab", T1, V, grad_view(Min), 1.0, 1.0, false);
    c.tape.active = t;
  });
}

SVDResult svd(Ctx& c, const Tensor& M_in, double eps_l) { return svd_many(c, {M_in}, eps_l)[0]; }

std::vector<SVDResult> svd_many(Ctx& c, const std::vector<Tensor>& Ms, double eps_l) {
  const int nb = (int)Ms.size();
  std::vector<SVDResult> out(nb);
  if (nb == 0) return out;
  const int m = Ms[0].shape[0], n = Ms[0].shape[1];
  for (const Tensor& M : Ms)
    SCTM_CHECK(M.nd == 2 && M.shape[0] == m && M.shape[1] == n && m >= n,
               "svd expects equally shaped matrices with rows >= columns");
  bool tap = c.tape.active;
  // one contiguous batch (a view of the input when there is a single contiguous matrix)
  Tensor Mb;
  if (nb == 1 && Ms[0].contiguous()) {
    Mb = Ms[0];
  } else {
    c.tape.active = false;   // the inputs' adjoints are added explicitly below
    Mb = c.empty({nb, m, n});
    for (int i = 0; i < nb; ++i) copy_into(c, Ms[i], Mb.sub(0, i));
    c.tape.active = tap;
  }
  Tensor Ub = c.empty({nb, m, n}), Sb = c.empty({nb, n}), Vb = c.empty({nb, n, n});
  size_t mk = c.arena.mark();
  double* work = nullptr;
  size_t wn = svd_work_doubles(m, n, nb);
  if (wn) work = c.arena.alloc((long long)wn);
  // every column counts for convergence: the reverse pass couples the kept
  // triplets to the rest of the spectrum through the U columns of the
  // smallest singular values, which must come out orthonormal too
  launch_svd(m, n, nb, Mb.data, Ub.data, Sb.data, Vb.data, work, c.svd_status, c.stream, 0.0, 0.0,
             c.svd_max_sweeps);
  if (!tap) c.arena.release(mk);  // later work is stream-ordered after the kernel
  for (int i = 0; i < nb; ++i) {
    out[i] = SVDResult{Ub.sub(0, i), Sb.sub(0, i), Vb.sub(0, i)};
    if (tap && Ms[i].grad) record_svd_adjoint(c, out[i], Ms[i], eps_l);
  }
  return out;
}

// ------------------------------------------------------------------ spectrum
Tensor spectrum_map(Ctx& c, const Tensor& S, int kout, double cutoff, int mode) {
  const int n = S.shape[0];
  Tensor w = c.empty({kout});
  launch_spectrum_map(1, n, kout, S.data, w.data, cutoff, mode, c.stream);
  if (c.tape.active && S.grad && mode != 2) {
    Tensor s = S, ww = w;
    c.tape.push([&c, s, ww, n, kout, cutoff, mode]() {
      launch_spectrum_adj(n, kout, s.data, ww.grad, s.grad, cutoff, mode, c.stream);
    });
  }
  return w;
}

Tensor scale_dim(Ctx& c, const Tensor& X, int dim, const Tensor& v) {
  SCTM_CHECK(dim < X.nd && v.nd == 1 && v.shape[0] == X.shape[dim], "scale_dim shape");
  Tensor Y = c.empty_shape(X.shape, X.nd);
  Group g;
  g.nd = X.nd;
  for (int i = 0; i < X.nd; ++i) g.size[i] = X.shape[i], g.sa[i] = X.stride[i], g.sc[i] = Y.stride[i];
  launch_scale_dim(g, dim, X.data, v.data, 0.0, Y.data, c.stream);
  if (c.tape.active && Y.grad && (X.grad || v.grad)) {
    Tensor x = X, vv = v, y = Y;
    c.tape.push([&c, x, vv, y, dim]() {
      Group h;
      h.nd = x.nd;
      for (int i = 0; i < x.nd; ++i) h.size[i] = x.shape[i], h.sa[i] = y.stride[i], h.sc[i] = x.stride[i];
      if (x.grad) launch_scale_dim(h, dim, y.grad, vv.data, 1.0, x.grad, c.stream);   // xbar += ybar v
      if (vv.grad) {
        Group r;   // vbar[j] += sum ybar x
        r.nd = x.nd;
        for (int i = 0; i < x.nd; ++i) r.size[i] = x.shape[i], r.sa[i] = y.stride[i], r.sb[i] = x.stride[i];
        launch_scale_dim_reduce(r, dim, y.grad, x.data, vv.grad, c.stream);
      }
    });
  }
  return Y;
}

Tensor row_signs(Ctx& c, const Tensor& P) {
  SCTM_CHECK(P.nd == 2, "row_signs expects a matrix");
  bool t = c.tape.active;
  c.tape.active = false;
  Tensor s = c.empty({P.shape[0]});
  c.tape.active = t;
  launch_sign_find(P.shape[0], P.shape[1], P.data, P.stride[0], P.stride[1], s.data, c.stream);
  return s;
}

// ------------------------------------------------------------------ rescale
Tensor rescale(Ctx& c, const Tensor& X_in) {
  Tensor X = X_in.contiguous() ? X_in : copy(c, X_in);
  Tensor Y = copy(c, X);
  bool t = c.tape.active;
  c.tape.active = false;
  Tensor m = c.empty({1});
  c.tape.active = t;
  long long* k = reinterpret_cast<long long*>(c.arena.alloc(1));
  launch_rescale(1, Y.numel(), Y.data, 0, m.data, k, c.partial, c.stream);
  if (c.tape.active && X.grad) {
    // Y was registered as a copy of X; replace that adjoint by the rescale adjoint
    c.tape.ops.pop_back();
    Tensor x = X, y = Y, mm = m;
    c.tape.push([&c, x, y, mm, k]() {
      double* d = c.arena.alloc(1);
      launch_dot(1, y.numel(), y.grad, y.data, 0, d, c.partial, c.stream);
      launch_rescale_adj(y.numel(), y.grad, y.data, mm.data, k, nullptr, d, x.grad, c.stream);
    });
  }
  return Y;
}

// ------------------------------------------------------------------ dot
Tensor dot(Ctx& c, const Tensor& X_in, const Tensor& Y_in) {
  Tensor X = X_in.contiguous() ? X_in : copy(c, X_in);
  Tensor Y = Y_in.contiguous() ? Y_in : copy(c, Y_in);
  SCTM_CHECK(X.numel() == Y.numel(), "dot size mismatch");
  Tensor o = c.empty({1});
  launch_dot(1, X.numel(), X.data, Y.data, 0, o.data, c.partial, c.stream);
  if (c.tape.active && (X.grad || Y.grad)) {
    Tensor x = X, y = Y, oo = o;
    c.tape.push([&c, x, y, oo]() {
      // xbar += obar * y ; ybar += obar * x   (obar read on device)
      const long long n = x.numel();
      const double* ob = oo.grad;   // obar, on the device
      if (x.grad) launch_axpy_dev(n, ob, y.data, x.grad, c.stream);
      if (y.grad) launch_axpy_dev(n, ob, x.data, y.grad, c.stream);
    });
  }
  return o;
}

Tensor from_host(Ctx& c, std::initializer_list<int> shape, const double* host) {
  Tensor t = c.empty(shape);
  SCTM_CUDA(cudaMemcpyAsync(t.data, host, t.numel() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  return t;
}

std::vector<double> to_host(Ctx& c, const Tensor& t) {
  Tensor x = t.contiguous() ? t : copy(c, t);
  std::vector<double> h(x.numel());
  SCTM_CUDA(cudaMemcpyAsync(h.data(), x.data, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  SCTM_CUDA(cudaStreamSynchronize(c.stream));
  return h;
}

}  // namespace sctm
