// C ABI of the engine (declared in include/splitctmrg.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/splitctmrg.h"
#include "ctmrg.h"
#include "prof.h"

using namespace sctm;

struct sctm_ctx {
  Params P;
  Ctx c;
  std::string err;
  bool ready = false;
  // persistent device memory: A (+grad), environment store, checkpoints
  double* A = nullptr;
  double* Agrad = nullptr;
  double* store = nullptr;       // environment of every site
  long long env_site = 0;        // doubles per site
  long long key_off[NKEY] = {0};
  int key_shape[NKEY][4] = {{0}};
  int key_nd[NKEY] = {0};
  Cell cell;
  ~sctm_ctx() {
    if (A) cudaFree(A);
    if (Agrad) cudaFree(Agrad);
    if (store) cudaFree(store);
    if (c.partial) cudaFree(c.partial);
    if (c.svd_status) cudaFree(c.svd_status);
    for (auto& kv : c.tune) {
      if (kv.second.e0) cudaEventDestroy(kv.second.e0);
      if (kv.second.e1) cudaEventDestroy(kv.second.e1);
    }
  }
};

namespace {

// an error that carries its own return code
struct CodedError : std::runtime_error {
  int code;
  CodedError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

int fail(sctm_handle h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

void rollback(sctm_handle h, size_t arena_mark);

template <typename F>
int guard(sctm_handle h, F&& f) {
  if (!h) return SCTM_ERR_ARG;
  const size_t mk = h->c.arena.mark();
  try {
    f();
    return SCTM_OK;
  } catch (const ArgError& e) {
    rollback(h, mk);
    std::string m = e.what();
    return fail(h, m.find("workspace exhausted") != std::string::npos ? SCTM_ERR_OOM : SCTM_ERR_ARG, m);
  } catch (const CudaError& e) {
    rollback(h, mk);
    return fail(h, SCTM_ERR_CUDA, e.what());
  } catch (const CodedError& e) {
    rollback(h, mk);
    return fail(h, e.code, e.what());
  } catch (const std::exception& e) {
    rollback(h, mk);
    std::string m = e.what();
    if (m.find("no convergence") != std::string::npos) return fail(h, SCTM_ERR_SVD_NOCONV, m);
    if (m.find("non-finite") != std::string::npos) return fail(h, SCTM_ERR_NONFINITE, m);
    return fail(h, SCTM_ERR_ARG, m);
  }
}

long long site_index(sctm_handle h, int x, int y) {
  int Lx = h->P.Lx, Ly = h->P.Ly;
  return (long long)((x % Lx + Lx) % Lx) * Ly + ((y % Ly + Ly) % Ly);
}

Tensor key_view(sctm_handle h, double* base, int x, int y, int k) {
  Tensor t;
  t.data = base + site_index(h, x, y) * h->env_site + h->key_off[k];
  t.nd = h->key_nd[k];
  long long st = 1;
  for (int i = t.nd - 1; i >= 0; --i) t.shape[i] = h->key_shape[k][i], t.stride[i] = st, st *= t.shape[i];
  return t;
}

// A views of the persistent buffer (gradient pointer aligned with the data)
void bind_A(sctm_handle h, bool with_grad) {
  const int p = h->P.p, D = h->P.D;
  const long long per = (long long)p * D * D * D * D;
  h->cell.Lx = h->P.Lx;
  h->cell.Ly = h->P.Ly;
  h->cell.A.resize(h->P.Lx * h->P.Ly);
  h->cell.env.resize(h->P.Lx * h->P.Ly);
  for (int x = 0; x < h->P.Lx; ++x)
    for (int y = 0; y < h->P.Ly; ++y) {
      Tensor t;
      long long off = (x * (long long)h->P.Ly + y) * per;
      t.data = h->A + off;
      t.grad = with_grad ? h->Agrad + off : nullptr;
      t.nd = 5;
      int s[5] = {p, D, D, D, D};
      long long st = 1;
      for (int i = 4; i >= 0; --i) t.shape[i] = s[i], t.stride[i] = st, st *= s[i];
      h->cell.a(x, y) = t;
    }
}

// copy the current environment handles into `dst` (packed store layout)
void save_env(sctm_handle h, double* dst) {
  for (int x = 0; x < h->P.Lx; ++x)
    for (int y = 0; y < h->P.Ly; ++y)
      for (int k = 0; k < NKEY; ++k) {
        Tensor d = key_view(h, dst, x, y, k);
        Tensor& s = h->cell.e(x, y)[k];
        if (s.data == d.data) continue;
        bool t = h->c.tape.active;
        h->c.tape.active = false;
        copy_into(h->c, s, d);
        h->c.tape.active = t;
      }
}

// point the environment handles at the store (no gradient buffers)
void bind_store(sctm_handle h, double* base) {
  for (int x = 0; x < h->P.Lx; ++x)
    for (int y = 0; y < h->P.Ly; ++y)
      for (int k = 0; k < NKEY; ++k) h->cell.e(x, y)[k] = key_view(h, base, x, y, k);
}

// A call that failed part-way leaves nothing behind: its workspace is released,
// its tape dropped, and the handles point at the persistent store again (which
// holds the environment of the last call that completed).
void rollback(sctm_handle h, size_t arena_mark) {
  h->c.arena.release(arena_mark);
  h->c.arena.release_high(h->c.arena.capacity());   // forward-pass caches of the failed call
  h->c.decomp = Ctx::DecompCache();
  h->c.tape.active = false;
  h->c.tape.ops.clear();
  if (h->store && h->A) {
    bind_A(h, false);
    bind_store(h, h->store);
  }
}

// leaves for a taped region: arena copies of `base` with zeroed gradients
// the second key of each edge pair aliases the first in a conventional environment
bool alias_key(sctm_handle h, int k) {
  return h->P.conventional && (k == T1b || k == T2b || k == T3k || k == T4k);
}
int alias_of(int k) { return k - 1; }   // pairs (T1k,T1b) (T2k,T2b) (T3b,T3k) (T4b,T4k) are adjacent

void bind_leaves(sctm_handle h, double* base) {
  for (int x = 0; x < h->P.Lx; ++x)
    for (int y = 0; y < h->P.Ly; ++y)
      for (int k = 0; k < NKEY; ++k) {
        if (alias_key(h, k)) {   // one leaf (one gradient buffer) for both slots
          h->cell.e(x, y)[k] = h->cell.e(x, y)[alias_of(k)];
          continue;
        }
        Tensor src = key_view(h, base, x, y, k);
        Tensor t = h->c.empty_shape(src.shape, src.nd);   // tape active -> zeroed grad
        bool a = h->c.tape.active;
        h->c.tape.active = false;
        copy_into(h->c, src, t);
        h->c.tape.active = a;
        h->cell.e(x, y)[k] = t;
      }
}

// gradient buffers of the current handles <- / -> packed layout
void seed_env_grad(sctm_handle h, const double* g) {
  for (int x = 0; x < h->P.Lx; ++x)
    for (int y = 0; y < h->P.Ly; ++y)
      for (int k = 0; k < NKEY; ++k) {
        Tensor s = key_view(h, const_cast<double*>(g), x, y, k);
        Tensor& t = h->cell.e(x, y)[k];
        SCTM_CHECK(t.grad, "environment handle without gradient buffer");
        Tensor gv = t;
        gv.data = t.grad;
        gv.grad = nullptr;
        bool a = h->c.tape.active;
        h->c.tape.active = false;
        copy_into(h->c, s, gv);
        h->c.tape.active = a;
      }
}

void read_env_grad(sctm_handle h, double* g) {
  for (int x = 0; x < h->P.Lx; ++x)
    for (int y = 0; y < h->P.Ly; ++y)
      for (int k = 0; k < NKEY; ++k) {
        Tensor d = key_view(h, g, x, y, k);
        Tensor& t = h->cell.e(x, y)[k];
        Tensor gv = t;
        gv.data = t.grad;
        gv.grad = nullptr;
        bool a = h->c.tape.active;
        h->c.tape.active = false;
        copy_into(h->c, gv, d);
        h->c.tape.active = a;
      }
}

void check_svd(sctm_handle h) {
  // the SVD kernels record -1 in status word 0 when they ran out of sweeps; the
  // tensor-core contraction records -2 in word 32 when a pipeline wait timed out
  int st[33] = {0};
  SCTM_CUDA(cudaMemcpyAsync(st, h->c.svd_status, sizeof(st), cudaMemcpyDeviceToHost, h->c.stream));
  SCTM_CUDA(cudaStreamSynchronize(h->c.stream));
  if (st[32] < 0) {
    SCTM_CUDA(cudaMemsetAsync(h->c.svd_status + 32, 0, sizeof(int), h->c.stream));
    throw CudaError("tensor-core contraction: pipeline wait timed out");
  }
  if (st[0] < 0) {
    SCTM_CUDA(cudaMemsetAsync(h->c.svd_status, 0, sizeof(int), h->c.stream));
    throw std::runtime_error("svd: no convergence");
  }
}

// Singular values of the four corners of every site (batched FP64 Jacobi SVD of
// the stored chi x chi corners), each spectrum divided by its largest value:
// host vector [site][corner][chi]; zero-padded corners give trailing zeros.
std::vector<double> corner_spectra(sctm_handle h) {
  const int chi = h->P.chi;
  const int nc = h->P.Lx * h->P.Ly * 4;
  const long long mm = (long long)chi * chi;
  std::vector<double> out((size_t)nc * chi, 0.0);
  size_t mk = h->c.arena.mark();
  double* M = h->c.arena.alloc(nc * mm);
  double* U = h->c.arena.alloc(nc * mm);
  double* V = h->c.arena.alloc(nc * mm);
  double* S = h->c.arena.alloc((long long)nc * chi);
  const int corners[4] = {C1, C2, C3, C4};
  long long i = 0;
  for (int x = 0; x < h->P.Lx; ++x)
    for (int y = 0; y < h->P.Ly; ++y)
      for (int k : corners) {
        const Tensor t = key_view(h, h->store, x, y, k);
        SCTM_CUDA(cudaMemcpyAsync(M + i * mm, t.data, mm * sizeof(double), cudaMemcpyDeviceToDevice, h->c.stream));
        ++i;
      }
  for (int b0 = 0; b0 < nc; b0 += 64) {   // at most 64 matrices per SVD launch
    const int nb = std::min(64, nc - b0);
    const size_t wn = svd_work_doubles(chi, chi, nb);
    double* work = wn ? h->c.arena.alloc((long long)wn) : nullptr;
    // only the singular values are used: columns at rounding level (below
    // 1e-14 of the largest, which a converged corner has many of) rotate but do
    // not hold the sweeps back, and the orthogonality threshold is 1e-12
    launch_svd(chi, chi, nb, M + b0 * mm, U + b0 * mm, S + (long long)b0 * chi, V + b0 * mm, work,
               h->c.svd_status, h->c.stream, 1e-28, 1e-12);
  }
  check_svd(h);
  SCTM_CUDA(cudaMemcpyAsync(out.data(), S, out.size() * sizeof(double), cudaMemcpyDeviceToHost, h->c.stream));
  SCTM_CUDA(cudaStreamSynchronize(h->c.stream));
  h->c.arena.release(mk);
  for (int c = 0; c < nc; ++c) {   // S is descending: s[0] is the largest
    double* s = out.data() + (size_t)c * chi;
    const double top = s[0];
    if (top > 0)
      for (int j = 0; j < chi; ++j) s[j] /= top;
  }
  return out;
}

void sweep_untaped(sctm_handle h) {
  for (int d = 0; d < 4; ++d) {
    size_t mk = h->c.arena.mark();
    move(h->c, h->P, h->cell, d);
    save_env(h, h->store);
    bind_store(h, h->store);
    h->c.arena.release(mk);
  }
}

// Energy per site, one 2x2 patch at a time.  With `seed` the reverse pass of
// every patch runs right after it and accumulates into the leaves' gradient
// buffers.  Only the enlarged corners are taped; the products
// Htop(o1,o2) = TL(o1)^T TR(o2) and Hbot(o3,o4) = BL(o3) BR(o4)^T are plain
// buffers, and their reverse pass is written out (no gradient buffers for them):
//   E_p = sum_t w_t N_t / N0,  N_t = <Htop(k_t), Hbot(l_t)>,  N0 = <Htop(0,0), Hbot(0,0)>,
//   Htop^(k) = sum_{t: k_t = k} (w_t / N0) Hbot(l_t) - [k = (0,0)] (E_p / N0) Hbot(0,0),
//   Hbot^(l) = sum_{t: l_t = l} (w_t / N0) Htop(k_t) - [l = (0,0)] (E_p / N0) Htop(0,0),
//   TL_bar(o1) += TR(o2) Htop^(o1,o2)^T,  TR_bar(o2) += TL(o1) Htop^(o1,o2),
//   BL_bar(o3) += Hbot^(o3,o4) BR(o4),    BR_bar(o4) += Hbot^(o3,o4)^T BL(o3);
// then the corners' tape carries the adjoints to the environment and A.  To
// bound the memory only the Hbot are stored: each Htop is formed for its dot
// products and dropped, and formed once more for the Hbot^ sums.
double energy_value(sctm_handle h, const double* hn, const double* hd, bool seed) {
  Ctx& c = h->c;
  const Params& P = h->P;
  EnergyOps ops = energy_ops(c, P, hn, hd);
  const std::vector<PatchTerm> terms = patch_terms(ops, P.Lx * P.Ly);
  typedef std::pair<int, int> Key;
  std::vector<Key> tkeys{{0, 0}}, bkeys{{0, 0}};
  for (const PatchTerm& t : terms) {
    if (std::find(tkeys.begin(), tkeys.end(), Key(t.t1, t.t2)) == tkeys.end()) tkeys.push_back({t.t1, t.t2});
    if (std::find(bkeys.begin(), bkeys.end(), Key(t.b1, t.b2)) == bkeys.end()) bkeys.push_back({t.b1, t.b2});
  }
  auto idx = [](const std::vector<Key>& v, Key k) { return (int)(std::find(v.begin(), v.end(), k) - v.begin()); };
  auto plain = [](Tensor t) {
    t.grad = nullptr;
    return t;
  };
  auto gview = [](const Tensor& t) {
    Tensor g = t;
    g.data = t.grad;
    g.grad = nullptr;
    return g;
  };
  double E = 0;
  for (int x = 0; x < P.Lx; ++x)
    for (int y = 0; y < P.Ly; ++y) {
      size_t mk = c.arena.mark();
      const size_t tm = c.tape.mark();
      const bool tap = c.tape.active;
      PatchCorners K = patch_corners(c, P, h->cell, ops, terms, x, y);
      c.tape.active = false;
      auto top = [&](const Key& k) { return einsum(c, "ra,rb->ab", plain(K.TL[k.first]), plain(K.TR[k.second])); };
      const size_t mk_hb = c.arena.mark();
      std::vector<Tensor> Hb;
      for (const Key& k : bkeys) Hb.push_back(einsum(c, "al,bl->ab", plain(K.BL[k.first]), plain(K.BR[k.second])));
      // dot products: term i + 1, the norm N0 at 0
      std::vector<Tensor> dev(terms.size() + 1);
      for (size_t ik = 0; ik < tkeys.size(); ++ik) {
        Tensor Ht = top(tkeys[ik]);
        if (ik == 0) dev[0] = dot(c, Ht, Hb[0]);
        for (size_t i = 0; i < terms.size(); ++i)
          if (Key(terms[i].t1, terms[i].t2) == tkeys[ik])
            dev[i + 1] = dot(c, Ht, Hb[idx(bkeys, {terms[i].b1, terms[i].b2})]);
      }
      std::vector<double> v(dev.size());
      for (size_t i = 0; i < dev.size(); ++i)
        SCTM_CUDA(cudaMemcpyAsync(&v[i], dev[i].data, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
      SCTM_CUDA(cudaStreamSynchronize(c.stream));
      const double N0 = v[0];
      double Ep = 0;
      for (size_t i = 0; i < terms.size(); ++i) Ep += terms[i].w * v[i + 1] / N0;
      E += Ep;
      if (seed) {
        SCTM_CHECK(tap, "energy gradient without a tape");
        const int n0 = Hb[0].shape[0], n1 = Hb[0].shape[1];
        const long long nn = Hb[0].numel();
        // top products: Htop^(k) from the stored Hbot, then the cotangents of TL(o1), TR(o2)
        for (size_t ik = 0; ik < tkeys.size(); ++ik) {
          size_t m2 = c.arena.mark();
          Tensor Hh = c.zeros({n0, n1});
          for (size_t i = 0; i < terms.size(); ++i)
            if (Key(terms[i].t1, terms[i].t2) == tkeys[ik])
              launch_axpy(nn, terms[i].w / N0, Hb[idx(bkeys, {terms[i].b1, terms[i].b2})].data, Hh.data, c.stream);
          if (ik == 0) launch_axpy(nn, -Ep / N0, Hb[0].data, Hh.data, c.stream);
          const Tensor& TL = K.TL[tkeys[ik].first];
          const Tensor& TR = K.TR[tkeys[ik].second];
          einsum_into(c, "rb,ab->ra", plain(TR), Hh, gview(TL), 1.0, 1.0, false);
          einsum_into(c, "ra,ab->rb", plain(TL), Hh, gview(TR), 1.0, 1.0, false);
          c.arena.release(m2);
        }
        // bottom products: the Hbot^(l) sums from each Htop formed once more
        c.arena.release(mk_hb);   // the stored Hbot are no longer needed
        std::vector<Tensor> Hh;
        for (size_t il = 0; il < bkeys.size(); ++il) Hh.push_back(c.zeros({n0, n1}));
        for (size_t ik = 0; ik < tkeys.size(); ++ik) {
          size_t m2 = c.arena.mark();
          Tensor Ht = top(tkeys[ik]);
          for (size_t i = 0; i < terms.size(); ++i)
            if (Key(terms[i].t1, terms[i].t2) == tkeys[ik])
              launch_axpy(nn, terms[i].w / N0, Ht.data, Hh[idx(bkeys, {terms[i].b1, terms[i].b2})].data, c.stream);
          if (ik == 0) launch_axpy(nn, -Ep / N0, Ht.data, Hh[0].data, c.stream);
          c.arena.release(m2);
        }
        for (size_t il = 0; il < bkeys.size(); ++il) {
          const Tensor& BL = K.BL[bkeys[il].first];
          const Tensor& BR = K.BR[bkeys[il].second];
          einsum_into(c, "ab,bl->al", Hh[il], plain(BR), gview(BL), 1.0, 1.0, false);
          einsum_into(c, "ab,al->bl", Hh[il], plain(BL), gview(BR), 1.0, 1.0, false);
        }
        c.tape.active = tap;
        c.tape.backward_from(tm);
      }
      c.tape.active = tap;
      c.arena.release(mk);
    }
  if (!std::isfinite(E)) throw std::runtime_error("non-finite energy");
  return E;
}

}  // namespace

extern "C" {

int sctm_create(const sctm_config* cfg, void* stream, sctm_handle* out) {
  if (!cfg || !out) return SCTM_ERR_ARG;
  auto h = std::make_unique<sctm_ctx>();
  int rc = guard(h.get(), [&]() {
    SCTM_CHECK(cfg->Lx >= 1 && cfg->Ly >= 1 && cfg->p >= 1 && cfg->D >= 1 && cfg->chi >= 1, "bad dimensions");
    SCTM_CHECK(cfg->D * cfg->D <= cfg->chi, "chi must be >= D^2");
    SCTM_CHECK(cfg->precision >= 0 && cfg->precision <= 4, "precision must be 0 (FP64), 1, 2, 4 (mixed) or 3");
    Params& P = h->P;
    P.Lx = cfg->Lx, P.Ly = cfg->Ly, P.p = cfg->p, P.D = cfg->D, P.chi = cfg->chi;
    SCTM_CHECK(cfg->chi_I >= 0, "chi_I must be >= 0");
    P.chiI = cfg->chi_I > 0 ? cfg->chi_I : cfg->chi;
    SCTM_CHECK(cfg->algorithm == 0 || P.chiI == P.chi, "chi_I applies to the split CTMRG only");
    P.mixed = (cfg->precision >= 1);   // randomized projectors for large truncated spaces
    h->c.fp32_compute = (cfg->precision == 1 || cfg->precision == 2 || cfg->precision == 4);
    h->c.tensor_cores = (cfg->precision == 1 || cfg->precision == 4);
    h->c.bf16_slices = (cfg->precision == 4);
    // FP32-level contractions resolve the singular vectors of values near 1e-6 s_max
    // only to O(0.1); from 1e-5 s_max up they are accurate enough for the gradient
    if (P.mixed) P.cutoff = h->c.fp32_compute ? 1e-5 : 1e-6;
    if (cfg->svd_cutoff > 0) P.cutoff = cfg->svd_cutoff;
    SCTM_CHECK(cfg->power_steps >= 0 && cfg->power_steps <= 16, "power_steps must be in [0, 16]");
    if (cfg->power_steps > 0) P.power_steps = cfg->power_steps;
    if (cfg->randomized_min > 0) P.randomized_min = cfg->randomized_min;
    SCTM_CHECK(cfg->rank_extra >= 0, "rank_extra must be >= 0");
    // sketch of chi + max(32, chi / 2) columns (precision 4: chi + max(32, chi)).
    // The reverse pass couples the kept triplets exactly to the computed ones
    // and to the rest of the spectrum only to leading order, so the gradient
    // depends on the sketch width: at D=6, chi=72 (2x2, 2 sweeps, cutoff 1e-5)
    // it is 3.8e-4 from the exact one with chi + 36 columns and 7.4e-5 with
    // chi + 72, at 5 % more time; at D=4, chi=64 both stay within 1e-4
    P.rank_extra = cfg->rank_extra > 0 ? cfg->rank_extra
                                       : (cfg->precision == 4 ? std::max(32, P.chi) : std::max(32, P.chi / 2));
    SCTM_CHECK(cfg->adjoint_cg_steps >= 0 && cfg->adjoint_cg_steps <= 64, "adjoint_cg_steps must be in [0, 64]");
    P.adjoint_cg_steps = cfg->adjoint_cg_steps;
    SCTM_CHECK(cfg->adjoint_band >= 0, "adjoint_band must be >= 0");
    P.adjoint_band = cfg->adjoint_band > 0 ? cfg->adjoint_band - 1 : -1;
    if (cfg->lorentz_eps > 0) P.eps_l = cfg->lorentz_eps;
    SCTM_CHECK(cfg->projector_order == 0 || cfg->projector_order == 1, "projector_order must be 0 or 1");
    P.order = cfg->projector_order;
    h->c.stream = (cudaStream_t)stream;
    SCTM_CHECK(cfg->algorithm == 0 || cfg->algorithm == 1, "algorithm must be 0 (split) or 1 (conventional)");
    P.conventional = (cfg->algorithm == 1);
    const int chi = P.chi, chiI = P.chiI, D = P.D;
    long long off = 0;
    for (int k = 0; k < NKEY; ++k) {
      bool corner = (k == C1 || k == C2 || k == C3 || k == C4);
      if (alias_key(h.get(), k)) {   // conventional: same storage as the pair's first key
        h->key_off[k] = h->key_off[alias_of(k)];
        h->key_nd[k] = h->key_nd[alias_of(k)];
        for (int i = 0; i < 4; ++i) h->key_shape[k][i] = h->key_shape[alias_of(k)][i];
        continue;
      }
      h->key_off[k] = off;
      if (corner) {
        h->key_nd[k] = 2, h->key_shape[k][0] = chi, h->key_shape[k][1] = chi;
        off += (long long)chi * chi;
      } else if (P.conventional) {
        h->key_nd[k] = 4, h->key_shape[k][0] = chi, h->key_shape[k][1] = D, h->key_shape[k][2] = D;
        h->key_shape[k][3] = chi;
        off += (long long)chi * D * D * chi;
      } else {
        // the first edge of a pair along the chain (T1k, T2k, T3b, T4b) is
        // [chi_E, D, chi_I], the second (T1b, T2b, T3k, T4k) [chi_I, D, chi_E]
        const bool first = (k == T1k || k == T2k || k == T3b || k == T4b);
        h->key_nd[k] = 3, h->key_shape[k][0] = first ? chi : chiI, h->key_shape[k][1] = D;
        h->key_shape[k][2] = first ? chiI : chi;
        off += (long long)chi * D * chiI;
      }
    }
    h->env_site = off;
    const long long N = (long long)P.Lx * P.Ly;
    const long long nA = N * P.p * (long long)D * D * D * D;
    SCTM_CUDA(cudaMalloc(&h->A, nA * sizeof(double)));
    SCTM_CUDA(cudaMalloc(&h->Agrad, nA * sizeof(double)));
    SCTM_CUDA(cudaMalloc(&h->store, N * off * sizeof(double)));
    SCTM_CUDA(cudaMemset(h->store, 0, N * off * sizeof(double)));
    SCTM_CUDA(cudaMalloc(&h->c.partial, 4096 * sizeof(double)));
    SCTM_CUDA(cudaMalloc(&h->c.svd_status, 64 * sizeof(int)));
    SCTM_CUDA(cudaMemset(h->c.svd_status, 0, 64 * sizeof(int)));
    size_t ws = cfg->workspace_bytes ? cfg->workspace_bytes : ((size_t)4 << 30);
    h->c.arena.reserve(ws);
    bind_A(h.get(), false);
    bind_store(h.get(), h->store);
  });
  if (rc != SCTM_OK) {
    // report through a static buffer: the handle is released
    static thread_local std::string last;
    last = h->err;
    return rc;
  }
  *out = h.release();
  return SCTM_OK;
}

int sctm_destroy(sctm_handle h) {
  if (!h) return SCTM_ERR_ARG;
  cudaStreamSynchronize(h->c.stream);
  delete h;
  return SCTM_OK;
}

const char* sctm_last_error(sctm_handle h) { return h ? h->err.c_str() : "null handle"; }

int split_ctmrg_init(sctm_handle h, const double* A_cell_dev) {
  return guard(h, [&]() {
    SCTM_CHECK(A_cell_dev, "A_cell is null");
    const long long nA = (long long)h->P.Lx * h->P.Ly * h->P.p * (long long)h->P.D * h->P.D * h->P.D * h->P.D;
    SCTM_CUDA(cudaMemcpyAsync(h->A, A_cell_dev, nA * sizeof(double), cudaMemcpyDeviceToDevice, h->c.stream));
    bind_A(h, false);
    h->c.tape.active = false;
    size_t mk = h->c.arena.mark();
    init_env(h->c, h->P, h->cell);
    save_env(h, h->store);
    bind_store(h, h->store);
    h->c.arena.release(mk);
    h->ready = true;
  });
}

int split_ctmrg_move(sctm_handle h, int dir) {
  return guard(h, [&]() {
    SCTM_CHECK(h->ready, "split_ctmrg_init must come first");
    SCTM_CHECK(dir >= 0 && dir < 4, "dir must be 0..3");
    size_t mk = h->c.arena.mark();
    move(h->c, h->P, h->cell, dir);
    save_env(h, h->store);
    bind_store(h, h->store);
    h->c.arena.release(mk);
  });
}

int split_ctmrg_sweeps(sctm_handle h, int n) {
  return guard(h, [&]() {
    SCTM_CHECK(h->ready, "split_ctmrg_init must come first");
    for (int i = 0; i < n; ++i) sweep_untaped(h);
    check_svd(h);
  });
}

namespace {
// Full steps until the largest change of a normalised corner spectrum (L2 over
// its chi values, max over corners and sites) falls below tol (Sec. II.B:
// steps are iterated until the environment converges).
void run_to_tol(sctm_handle h, int max_sweeps, double tol, int* sweeps_done, double* last_delta) {
  const size_t chi = (size_t)h->P.chi;
  std::vector<double> prev = corner_spectra(h);
  double delta = HUGE_VAL;
  int n = 0;
  while (n < max_sweeps) {
    sweep_untaped(h);
    ++n;
    std::vector<double> cur = corner_spectra(h);
    delta = 0.0;
    for (size_t c = 0; c < cur.size() / chi; ++c) {
      double ss = 0.0;
      for (size_t j = 0; j < chi; ++j) {
        const double d = cur[c * chi + j] - prev[c * chi + j];
        ss += d * d;
      }
      if (!std::isfinite(ss)) throw std::runtime_error("non-finite corner spectrum");
      delta = std::max(delta, std::sqrt(ss));
    }
    prev.swap(cur);
    if (delta < tol) break;
  }
  if (sweeps_done) *sweeps_done = n;
  if (last_delta) *last_delta = delta;
}
}  // namespace

int split_ctmrg_run(sctm_handle h, int max_sweeps, double tol, int* sweeps_done, double* last_delta) {
  return guard(h, [&]() {
    SCTM_CHECK(h->ready, "split_ctmrg_init must come first");
    SCTM_CHECK(max_sweeps >= 0, "max_sweeps must be >= 0");
    if (!(tol > 0)) tol = h->c.fp32_compute ? 1e-7 : 1e-12;
    run_to_tol(h, max_sweeps, tol, sweeps_done, last_delta);
  });
}

int ctmrg_projectors(sctm_handle h, int dir, int x, int y, int colour, double* P_up_dev, double* P_dn_dev,
                     double* s_host) {
  return guard(h, [&]() {
    SCTM_CHECK(h->ready, "split_ctmrg_init must come first");
    SCTM_CHECK(!h->P.conventional, "projector colours belong to the split scheme");
    SCTM_CHECK(dir >= 0 && dir < 4 && colour >= 0 && colour < 4, "bad dir or colour");
    size_t mk = h->c.arena.mark();
    Cell fr;
    if (dir == 0) fr = h->cell;
    else if (dir == 1) fr = frame_transpose(h->cell);
    else if (dir == 2) fr = frame_rot180(h->cell);
    else {
      Cell t = frame_rot180(h->cell);
      fr = frame_transpose(t);
    }
    ColumnProj cp;
    column_projectors(h->c, h->P, fr, ((y % fr.Ly) + fr.Ly) % fr.Ly, cp);
    int xi = ((x % fr.Lx) + fr.Lx) % fr.Lx;
    const ProjPair& pp = colour == 0 ? cp.g[xi] : colour == 1 ? cp.t[xi] : colour == 2 ? cp.y[xi] : cp.r[xi];
    long long n = pp.up.numel();
    SCTM_CUDA(cudaMemcpyAsync(P_up_dev, pp.up.data, n * sizeof(double), cudaMemcpyDeviceToDevice, h->c.stream));
    SCTM_CUDA(cudaMemcpyAsync(P_dn_dev, pp.dn.data, n * sizeof(double), cudaMemcpyDeviceToDevice, h->c.stream));
    if (s_host)
      SCTM_CUDA(cudaMemcpyAsync(s_host, pp.s.data, pp.up.shape[0] * sizeof(double), cudaMemcpyDeviceToHost,
                                h->c.stream));
    SCTM_CUDA(cudaStreamSynchronize(h->c.stream));
    h->c.arena.release(mk);
  });
}

int energy_2x2(sctm_handle h, const double* h_nn_host, const double* h_diag_host, double* e_per_site) {
  return guard(h, [&]() {
    SCTM_CHECK(h->ready, "split_ctmrg_init must come first");
    SCTM_CHECK(h_nn_host && e_per_site, "null argument");
    size_t mk = h->c.arena.mark();
    h->c.tape.active = false;
    *e_per_site = energy_value(h, h_nn_host, h_diag_host, false);
    h->c.arena.release(mk);
  });
}

int energy_grad(sctm_handle h, const double* A_cell_dev, int sweeps, const double* h_nn_host,
                const double* h_diag_host, double* e_per_site, double* grad_dev) {
  return guard(h, [&]() {
    SCTM_CHECK(A_cell_dev && h_nn_host && e_per_site && grad_dev, "null argument");
    SCTM_CHECK(sweeps >= 0, "sweeps must be >= 0");
    Ctx& c = h->c;
    const Params& P = h->P;
    const long long N = (long long)P.Lx * P.Ly;
    const long long nA = N * P.p * (long long)P.D * P.D * P.D * P.D;
    const long long nE = N * h->env_site;
    SCTM_CUDA(cudaMemcpyAsync(h->A, A_cell_dev, nA * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    SCTM_CUDA(cudaMemsetAsync(h->Agrad, 0, nA * sizeof(double), c.stream));
    size_t base = c.arena.mark();
    // checkpoints of the environment before every directional move (+ final):
    // the reverse pass recomputes one move at a time, taped
    const int nmoves = 4 * sweeps;
    double* ck = c.arena.alloc(nE * (nmoves + 1));
    double* gbuf = c.arena.alloc(nE);
    // forward: the initial environment taped once (its tape segment and
    // intermediates are kept and reversed last), then the moves untaped
    bind_A(h, true);
    c.tape.active = true;
    const size_t init_mark = c.tape.mark();
    init_env(c, P, h->cell);
    std::vector<SiteEnv> init_out = h->cell.env;
    c.tape.active = false;
    save_env(h, ck);
    bind_store(h, ck);
    size_t top = c.arena.mark();
    // the randomized decompositions of every move are kept (arena high stack)
    // for the taped recomputation of that move in the reverse pass
    std::vector<std::vector<std::array<Tensor, 3>>> decomp(nmoves);
    std::vector<size_t> high_mark(nmoves);
    for (int mv = 0; mv < nmoves; ++mv) {
      high_mark[mv] = c.arena.mark_high();
      c.decomp = Ctx::DecompCache();
      c.decomp.mode = 1;
      move(c, P, h->cell, mv % 4);
      decomp[mv] = std::move(c.decomp.entries);
      c.decomp = Ctx::DecompCache();
      save_env(h, ck + (mv + 1) * nE);
      bind_store(h, ck + (mv + 1) * nE);
      c.arena.release(top);
    }
    check_svd(h);
    // energy on the final environment, taped patch by patch
    c.tape.active = true;
    bind_leaves(h, ck + nmoves * nE);
    *e_per_site = energy_value(h, h_nn_host, h_diag_host, true);
    read_env_grad(h, gbuf);
    c.tape.active = false;
    c.arena.release(top);
    // reverse through the moves, one checkpointed move at a time
    for (int mv = nmoves - 1; mv >= 0; --mv) {
      c.tape.active = true;
      bind_leaves(h, ck + mv * nE);
      std::vector<SiteEnv> leaves = h->cell.env;
      const size_t tm = c.tape.mark();
      c.decomp = Ctx::DecompCache();
      c.decomp.mode = 2;
      c.decomp.entries = std::move(decomp[mv]);
      move(c, P, h->cell, mv % 4);
      SCTM_CHECK(c.decomp.next == c.decomp.entries.size(), "decomposition cache: entries left over");
      c.decomp = Ctx::DecompCache();
      seed_env_grad(h, gbuf);
      c.tape.backward_from(tm);
      h->cell.env = leaves;
      read_env_grad(h, gbuf);
      c.tape.active = false;
      c.arena.release(top);
      c.arena.release_high(high_mark[mv]);
    }
    // reverse through the initial environment (recorded in the forward)
    h->cell.env = init_out;
    seed_env_grad(h, gbuf);
    c.tape.backward_from(init_mark);
    c.tape.active = false;
    check_svd(h);
    SCTM_CUDA(cudaMemcpyAsync(grad_dev, h->Agrad, nA * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    // leave the converged environment in the store
    bind_A(h, false);
    bind_store(h, ck + nmoves * nE);
    save_env(h, h->store);
    bind_store(h, h->store);
    SCTM_CUDA(cudaStreamSynchronize(c.stream));
    c.arena.release(base);
    h->ready = true;
  });
}

int energy_grad_host(sctm_handle h, const double* A_cell_host, int sweeps, const double* h_nn_host,
                     const double* h_diag_host, double* e_per_site, double* grad_host) {
  if (!h) return SCTM_ERR_ARG;
  if (!A_cell_host || !grad_host) return fail(h, SCTM_ERR_ARG, "null argument");
  const Params& P = h->P;
  const long long nA = (long long)P.Lx * P.Ly * P.p * (long long)P.D * P.D * P.D * P.D;
  const size_t mk = h->c.arena.mark();
  double* a = nullptr;
  double* g = nullptr;
  int rc = guard(h, [&]() {
    a = h->c.arena.alloc(nA);
    g = h->c.arena.alloc(nA);
    SCTM_CUDA(cudaMemcpyAsync(a, A_cell_host, nA * sizeof(double), cudaMemcpyHostToDevice, h->c.stream));
  });
  // energy_grad's own error code (e.g. SCTM_ERR_OOM) is passed through unchanged
  if (rc == SCTM_OK) rc = energy_grad(h, a, sweeps, h_nn_host, h_diag_host, e_per_site, g);
  if (rc == SCTM_OK)
    rc = guard(h, [&]() {
      SCTM_CUDA(cudaMemcpyAsync(grad_host, g, nA * sizeof(double), cudaMemcpyDeviceToHost, h->c.stream));
      SCTM_CUDA(cudaStreamSynchronize(h->c.stream));
    });
  h->c.arena.release(mk);
  return rc;
}

int energy_grad_implicit(sctm_handle h, const double* A_cell_dev, int max_sweeps, double tol,
                         const double* h_nn_host, const double* h_diag_host, double fixed_point_tol,
                         double solve_tol, int max_iter, int max_period, double* e_per_site, double* grad_dev,
                         int* sweeps_done, int* period_out, int* solver_iterations, double* fixed_point_change) {
  return guard(h, [&]() {
    SCTM_CHECK(A_cell_dev && h_nn_host && e_per_site && grad_dev, "null argument");
    SCTM_CHECK(max_sweeps >= 0 && max_iter >= 1, "max_sweeps must be >= 0 and max_iter >= 1");
    if (max_period <= 0) max_period = 4;
    SCTM_CHECK(max_period <= 16, "max_period must be at most 16");
    // defaults: FP64 as the rule's own tolerances; the mixed precisions carry
    // FP32-level rounding in the networks, which sets the floor of the
    // spectral change, of the step-to-step change and of the adjoint iterate
    const bool mixed = h->c.fp32_compute;
    if (!(tol > 0)) tol = mixed ? 1e-7 : 1e-13;
    if (!(fixed_point_tol > 0)) fixed_point_tol = mixed ? 1e-5 : 1e-9;
    if (!(solve_tol > 0)) solve_tol = mixed ? 1e-6 : 1e-12;
    Ctx& c = h->c;
    const Params& P = h->P;
    const long long N = (long long)P.Lx * P.Ly;
    const long long nA = N * P.p * (long long)P.D * P.D * P.D * P.D;
    const long long nE = N * h->env_site;
    SCTM_CUDA(cudaMemcpyAsync(h->A, A_cell_dev, nA * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    size_t base = c.arena.mark();
    const size_t high_base = c.arena.mark_high();
    // 1. the fixed point env*: initial environment, then full steps to tol
    bind_A(h, false);
    c.tape.active = false;
    init_env(c, P, h->cell);
    save_env(h, h->store);
    bind_store(h, h->store);
    c.arena.release(base);
    h->ready = true;
    int n = 0;
    run_to_tol(h, max_sweeps, tol, &n, nullptr);
    if (sweeps_done) *sweeps_done = n;
    // 2. the p-step map F = f^p: steps from env* with checkpoints ck[0] = env*,
    // ck[m] after move m, keeping the decompositions of every move for the taped
    // recomputations; p is the smallest number of steps (<= max_period) after
    // which no entry of any environment tensor has moved by more than
    // fixed_point_tol of that tensor's largest entry (the signs of the
    // projectors, and with them rows of the environment, may cycle at
    // converged spectra)
    const int max_moves = 4 * max_period;
    double* ck = c.arena.alloc(nE * (max_moves + 1));
    double* gE = c.arena.alloc(nE);     // dE/denv*
    double* x = c.arena.alloc(nE);      // adjoint iterate
    double* xn = c.arena.alloc(nE);
    double* gbuf = c.arena.alloc(nE);
    double* gA0 = c.arena.alloc(nA);    // dE/dA at fixed env*
    const long long ntens = N * NKEY;
    double* red = c.arena.alloc(2 * ntens + 4);
    save_env(h, ck);
    bind_store(h, ck);
    const size_t top = c.arena.mark();
    std::vector<std::vector<std::array<Tensor, 3>>> decomp(max_moves);
    int period = 0;
    double worst = 0.0;
    std::vector<double> hr(2 * ntens);
    for (int q = 1; q <= max_period && !period; ++q) {
      for (int d = 0; d < 4; ++d) {
        const int mv = 4 * (q - 1) + d;
        c.decomp = Ctx::DecompCache();
        c.decomp.mode = 1;
        move(c, P, h->cell, d);
        decomp[mv] = std::move(c.decomp.entries);
        c.decomp = Ctx::DecompCache();
        save_env(h, ck + (mv + 1) * nE);
        bind_store(h, ck + (mv + 1) * nE);
        c.arena.release(top);
      }
      check_svd(h);
      // element-wise change after q steps: max over tensors of max|F(env*) - env*| / max|env*|
      long long i = 0;
      for (int xx = 0; xx < P.Lx; ++xx)
        for (int yy = 0; yy < P.Ly; ++yy)
          for (int k = 0; k < NKEY; ++k, ++i) {
            const Tensor a0 = key_view(h, ck, xx, yy, k), b0 = key_view(h, ck + 4 * q * nE, xx, yy, k);
            launch_maxabs_pair(a0.numel(), b0.data, a0.data, red + 2 * i, c.stream);
          }
      SCTM_CUDA(cudaMemcpyAsync(hr.data(), red, hr.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
      SCTM_CUDA(cudaStreamSynchronize(c.stream));
      worst = 0.0;
      for (long long j = 0; j < ntens; ++j)
        if (hr[2 * j + 1] > 0) worst = std::max(worst, hr[2 * j] / hr[2 * j + 1]);
      if (worst <= fixed_point_tol) period = q;
    }
    if (fixed_point_change) *fixed_point_change = worst;
    if (period_out) *period_out = period;
    if (!period)
      throw CodedError(SCTM_ERR_NOT_FIXED_POINT,
                       "environment is not an element-wise fixed point of up to " + std::to_string(max_period) +
                           " steps (relative change " + std::to_string(worst) + ")");
    const int nmoves = 4 * period;
    // 3. energy at env*, taped: dE/denv* and dE/dA
    bind_A(h, true);
    SCTM_CUDA(cudaMemsetAsync(h->Agrad, 0, nA * sizeof(double), c.stream));
    c.tape.active = true;
    bind_leaves(h, ck);
    *e_per_site = energy_value(h, h_nn_host, h_diag_host, true);
    read_env_grad(h, gE);
    c.tape.active = false;
    c.arena.release(top);
    SCTM_CUDA(cudaMemcpyAsync(gA0, h->Agrad, nA * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    // out = x^T dF/denv through the moves of F, each recomputed taped from its
    // checkpoint (x^T dF/dA accumulates into the A gradient)
    auto vjp = [&](const double* xin, double* out) {
      SCTM_CUDA(cudaMemcpyAsync(gbuf, xin, nE * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
      for (int mv = nmoves - 1; mv >= 0; --mv) {
        c.tape.active = true;
        bind_leaves(h, ck + mv * nE);
        std::vector<SiteEnv> leaves = h->cell.env;
        const size_t tm = c.tape.mark();
        c.decomp = Ctx::DecompCache();
        c.decomp.mode = 2;
        c.decomp.entries = decomp[mv];
        move(c, P, h->cell, mv % 4);
        SCTM_CHECK(c.decomp.next == c.decomp.entries.size(), "decomposition cache: entries left over");
        c.decomp = Ctx::DecompCache();
        seed_env_grad(h, gbuf);
        c.tape.backward_from(tm);
        h->cell.env = leaves;
        read_env_grad(h, gbuf);
        c.tape.active = false;
        c.arena.release(top);
      }
      SCTM_CUDA(cudaMemcpyAsync(out, gbuf, nE * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    };
    // 4. x = dE/denv* + x^T dF/denv, iterated from x = dE/denv*
    SCTM_CUDA(cudaMemcpyAsync(x, gE, nE * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    int it = 0;
    bool converged = false;
    while (it < max_iter && !converged) {
      ++it;
      vjp(x, xn);
      launch_axpy(nE, 1.0, gE, xn, c.stream);                       // xn = dE/denv* + x^T dF/denv
      launch_axpy(nE, -1.0, xn, x, c.stream);                       // x <- x - xn (the change)
      launch_dot(1, nE, x, x, 0, red, c.partial, c.stream);
      launch_dot(1, nE, xn, xn, 0, red + 1, c.partial, c.stream);
      double nd[2];
      SCTM_CUDA(cudaMemcpyAsync(nd, red, sizeof(nd), cudaMemcpyDeviceToHost, c.stream));
      SCTM_CUDA(cudaStreamSynchronize(c.stream));
      if (!std::isfinite(nd[0]) || !std::isfinite(nd[1])) throw std::runtime_error("non-finite adjoint iterate");
      std::swap(x, xn);
      converged = std::sqrt(nd[0]) <= solve_tol * std::sqrt(nd[1]);
    }
    if (solver_iterations) *solver_iterations = it;
    if (!converged) throw CodedError(SCTM_ERR_NO_CONVERGENCE, "adjoint fixed-point iteration did not converge");
    check_svd(h);
    // 5. grad = dE/dA + x^T dF/dA
    SCTM_CUDA(cudaMemsetAsync(h->Agrad, 0, nA * sizeof(double), c.stream));
    vjp(x, xn);
    launch_axpy(nA, 1.0, gA0, h->Agrad, c.stream);
    check_svd(h);
    SCTM_CUDA(cudaMemcpyAsync(grad_dev, h->Agrad, nA * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    // env* stays in the store
    bind_A(h, false);
    bind_store(h, h->store);
    SCTM_CUDA(cudaStreamSynchronize(c.stream));
    c.arena.release(base);
    c.arena.release_high(high_base);
  });
}

int sctm_get_env(sctm_handle h, int x, int y, double* out_dev) {
  return guard(h, [&]() {
    SCTM_CHECK(out_dev, "null argument");
    SCTM_CUDA(cudaMemcpyAsync(out_dev, h->store + site_index(h, x, y) * h->env_site, h->env_site * sizeof(double),
                              cudaMemcpyDeviceToDevice, h->c.stream));
    SCTM_CUDA(cudaStreamSynchronize(h->c.stream));
  });
}

int sctm_svd(sctm_handle h, int m, int n, const double* M_dev, double* U_dev, double* S_dev, double* V_dev) {
  return guard(h, [&]() {
    SCTM_CHECK(m >= n && n >= 1 && M_dev && U_dev && S_dev && V_dev, "bad svd arguments");
    size_t mk = h->c.arena.mark();
    double* work = nullptr;
    size_t wn = svd_work_doubles(m, n, 1);
    if (wn) work = h->c.arena.alloc((long long)wn);
    launch_svd(m, n, 1, M_dev, U_dev, S_dev, V_dev, work, h->c.svd_status, h->c.stream, 0.0, 0.0,
               h->c.svd_max_sweeps);
    check_svd(h);
    h->c.arena.release(mk);
  });
}

int sctm_einsum(sctm_handle h, const char* spec, const double* A_dev, const int* shape_A, const double* B_dev,
                const int* shape_B, double* C_dev, const int* shape_C, double alpha, double beta) {
  return guard(h, [&]() {
    SCTM_CHECK(spec && A_dev && B_dev && C_dev && shape_A && shape_B && shape_C, "null argument");
    std::string s(spec);
    size_t comma = s.find(','), arrow = s.find("->");
    SCTM_CHECK(comma != std::string::npos && arrow != std::string::npos && comma < arrow, "bad einsum spec");
    const int nd[3] = {(int)comma, (int)(arrow - comma - 1), (int)(s.size() - arrow - 2)};
    const int* shp[3] = {shape_A, shape_B, shape_C};
    double* ptr[3] = {const_cast<double*>(A_dev), const_cast<double*>(B_dev), C_dev};
    Tensor t[3];
    for (int i = 0; i < 3; ++i) {
      SCTM_CHECK(nd[i] >= 1 && nd[i] <= kMaxDims, "einsum rank out of range");
      t[i].data = ptr[i];
      t[i].nd = nd[i];
      long long st = 1;
      for (int j = nd[i] - 1; j >= 0; --j) {
        SCTM_CHECK(shp[i][j] >= 1, "einsum extent must be >= 1");
        t[i].shape[j] = shp[i][j];
        t[i].stride[j] = st;
        st *= shp[i][j];
      }
    }
    bool tp = h->c.tape.active;
    h->c.tape.active = false;
    einsum_into(h->c, spec, t[0], t[1], t[2], alpha, beta, false);
    h->c.tape.active = tp;
    check_svd(h);
  });
}

int sctm_profile(sctm_handle h, int enable, double* out) {
  return guard(h, [&]() {
    if (enable) {
      SCTM_CUDA(cudaStreamSynchronize(h->c.stream));
      prof_enable(true);
    } else {
      SCTM_CHECK(out, "null output");
      SCTM_CUDA(cudaStreamSynchronize(h->c.stream));
      prof_collect(out);
      prof_enable(false);
    }
  });
}

int sctm_workspace_high_water(sctm_handle h, size_t* bytes) {
  return guard(h, [&]() { *bytes = h->c.arena.high_water(); });
}

int sctm_autotune(sctm_handle h, int enable) {
  return guard(h, [&]() { h->c.autotune = enable != 0; });
}

int sctm_autotune_table(sctm_handle h, double* out, int max_rows, int* rows) {
  return guard(h, [&]() {
    SCTM_CHECK(rows && (max_rows <= 0 || out), "null argument");
    SCTM_CUDA(cudaStreamSynchronize(h->c.stream));
    int n = 0;
    for (auto& kv : h->c.tune) {
      Ctx::Tune& t = kv.second;
      if (t.pending >= 0) {   // the last exploration call's timing
        SCTM_CUDA(cudaEventElapsedTime(&t.ms[t.pending], t.e0, t.e1));
        t.pending = -1;
        if (t.next == (int)t.cand.size())
          t.chosen = t.cand[std::min_element(t.ms.begin(), t.ms.end()) - t.ms.begin()];
      }
      if (!t.chosen) continue;
      if (n < max_rows) {
        double* r = out + 9 * (size_t)n;
        for (int i = 0; i < 5; ++i) r[i] = (double)kv.first[i];
        const int ic = (int)(std::find(t.cand.begin(), t.cand.end(), t.chosen) - t.cand.begin());
        r[5] = t.cand[0];
        r[6] = t.ms[0];
        r[7] = t.chosen;
        r[8] = t.ms[ic];
      }
      ++n;
    }
    *rows = n;
  });
}

int sctm_set_limits(sctm_handle h, int svd_max_sweeps, double pipeline_wait_s) {
  return guard(h, [&]() {
    SCTM_CHECK(pipeline_wait_s <= 60.0, "pipeline_wait_s must be at most 60 s");
    h->c.svd_max_sweeps = svd_max_sweeps > 0 ? svd_max_sweeps : 60;
    h->c.pipe_wait_ns = pipeline_wait_s < 0 ? 2000000000ull : (unsigned long long)(pipeline_wait_s * 1e9);
  });
}

}  // extern "C"
