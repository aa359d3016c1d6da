/* C ABI of the split-CTMRG engine for one GB300 GPU.
 *
 * Method: Naumann, Weerda, Eisert, Rizzi, Schmoll, "Variationally optimizing
 * infinite projected entangled-pair states at large bond dimensions: a split
 * corner transfer matrix renormalization group approach" (arXiv 2502.10298).
 *
 * Conventions
 *  - All floating point data is IEEE binary64 (double), row-major.
 *  - PEPS unit cell A_cell: [Lx][Ly][p][D][D][D][D], site (x, y) with x the row
 *    and y the column; per site the legs are (s, up, left, down, right).  The
 *    bra layer is the same real tensor (Sec. II.A).
 *  - Environment of a site (Fig. 2): C1, T1ket, T1bra, C2, T2ket, T2bra, C3,
 *    T3bra, T3ket, C4, T4bra, T4ket.  Every edge tensor is [previous, PEPS leg,
 *    next] along the clockwise chain C1 T1k T1b C2 T2k T2b C3 T3b T3k C4 T4b
 *    T4k; C2, C3, C4 are [previous, next] and C1 is [next (T1k), previous
 *    (T4k)].  Environment bonds have dimension chi_E = chi and interlayer
 *    bonds chi_I (sctm_config.chi_I, by default chi), zero-padded to those.
 *  - Bond operators are real p^2 x p^2 matrices h[(t_i t_j), (s_i s_j)] with s
 *    the ket and t the bra physical index.
 *  - "dev" pointers are device pointers owned by the caller; "host" pointers
 *    are host memory owned by the caller.  The library owns only the handle
 *    (environment, workspace, stream association).
 *  - Every call returns SCTM_OK (0) or a negative error code; a message is
 *    available from sctm_last_error().  Calls are asynchronous on the stream
 *    given at creation unless they return host values (those synchronise).
 */
#ifndef SPLITCTMRG_H
#define SPLITCTMRG_H

#include <stddef.h>

#if defined(__GNUC__)
#define SCTM_API __attribute__((visibility("default")))
#else
#define SCTM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SCTM_OK = 0,
  SCTM_ERR_ARG = -1,       /* invalid argument or shape                     */
  SCTM_ERR_CUDA = -2,      /* a CUDA call failed                            */
  SCTM_ERR_SVD_NOCONV = -3,/* a Jacobi SVD did not converge                 */
  SCTM_ERR_NONFINITE = -4, /* NaN or Inf in a result                        */
  SCTM_ERR_OOM = -5,       /* device workspace too small                    */
  SCTM_ERR_STATE = -6,     /* call order (e.g. move before init)            */
  SCTM_ERR_NOT_FIXED_POINT = -7, /* environment not an element-wise fixed point */
  SCTM_ERR_NO_CONVERGENCE = -8   /* an iteration reached its limit          */
};

typedef struct sctm_ctx* sctm_handle;

typedef struct {
  int Lx, Ly;            /* unit cell                                        */
  int p;                 /* physical dimension                               */
  int D;                 /* bulk bond dimension chi_B                        */
  int chi;               /* environment and interlayer bond dimension        */
  int precision;         /* 0: FP64 throughout (exact Jacobi SVDs).
                            1: mixed -- large contractions on the tcgen05 tensor cores
                               as 3xTF32 (operands split into TF32 hi + lo, FP32
                               accumulation), small ones in FP32 on the CUDA cores;
                               projectors from a randomized subspace iteration (chi +
                               rank_extra columns, Cholesky-QR bases, power_steps steps)
                               when the truncated space is at least four times that and
                               at least randomized_min;
                               decompositions and Gram matrices in FP64; default
                               cutoff 1e-5.
                            2: as 1 with every contraction on the CUDA cores (FP32).
                            3: FP64 arithmetic throughout with the randomized
                               projectors of 1 (cutoff default 1e-6).
                            4: as 1 with the large contractions on the tcgen05 tensor
                               cores as BF16 digit slices: every row of A and column
                               of B scaled by a power of two and split into four BF16
                               slices of 8 bits, ten BF16 products per multiply-add,
                               the two leading levels accumulated exactly in FP32
                               (error-free splitting of Ozaki et al. 2012); about
                               2^-32 relative to the largest terms, FP64 output.
                               Default cutoff 1e-5. */
  double svd_cutoff;     /* relative singular-value cutoff of projectors (<=0: 1e-8) */
  double lorentz_eps;    /* Lorentzian broadening of the SVD adjoint (<=0: 1e-36 s_max^4) */
  size_t workspace_bytes;/* device workspace; 0 = library default          */
  int power_steps;       /* mixed mode, randomized projectors: power steps, each
                            Z = orth(M^T Q), Q = orth(M Z) (0: default 2)        */
  int randomized_min;    /* mixed mode: randomized projectors only when the space
                            being truncated has at least this dimension (0: 256);
                            smaller ones use the exact FP64 decomposition        */
  int adjoint_cg_steps;  /* mixed mode, reverse pass of randomized projectors: 0 =
                            leading-order coupling to the unresolved spectrum;
                            n > 0 = n conjugate-gradient steps on the first-order
                            coupling (experimental)                                */
  int adjoint_band;      /* mixed mode, reverse pass of randomized projectors: 0 = all
                            chi + rank_extra computed triplets coupled exactly; n > 0 = only the
                            first chi + n - 1 (the rest of the spectrum is treated
                            as the complement)                                      */
  int rank_extra;        /* mixed mode, randomized projectors: columns beyond chi in the
                            sketch (0: max(32, chi / 2); precision 4: max(32, chi))  */
  int algorithm;         /* 0: split CTMRG (Sec. II.B).  1: the conventional double-
                            layer CTMRG the paper compares against (Sec. III), with
                            2x2-patch projectors; its edges are the fused ket-bra pairs
                            [previous, ket leg, bra leg, next] (chi x D x D x chi) and
                            the same calls (init, move, energy_2x2, energy_grad) apply;
                            ctmrg_projectors is not available for it                */
  int chi_I;             /* split CTMRG: interlayer bond dimension chi_I between a ket
                            and a bra edge (Sec. II.B; 0: chi_I = chi, the paper's
                            choice); chi is then chi_E.  Edges are [chi_E, D, chi_I]
                            (T1k, T2k, T3b, T4b) and [chi_I, D, chi_E] (T1b, T2b, T3k,
                            T4k); green and teal keep chi_E values, yellow, red and
                            the initial edge split chi_I                              */
  int projector_order;   /* split CTMRG: 0 = the physical leg of the ket is truncated
                            by the red projectors (Sec. II.B, App. A); 1 = by the
                            yellow ones (the alternative order of App. B, which
                            removes the p^3 factor of the red decomposition): yellow
                            then truncates (chi_I, D, p) and red (chi_I, D)         */
} sctm_config;

/* Create a handle.  stream: a cudaStream_t (NULL = legacy default stream). */
SCTM_API int sctm_create(const sctm_config* cfg, void* stream, sctm_handle* out);
SCTM_API int sctm_destroy(sctm_handle h);
SCTM_API const char* sctm_last_error(sctm_handle h);

/* Load A_cell (dev) and build the initial environment from the double-layer
 * contractions of the neighbouring tensors (corners and edges of the norm
 * network with their outward legs traced), each edge split into its ket and
 * bra halves by a truncated SVD (Sec. II.B: a ket/bra pair contracted over
 * the interlayer bond is the conventional edge).  Requires D*D <= chi. */
SCTM_API int split_ctmrg_init(sctm_handle h, const double* A_cell_dev);

/* One directional move over every column/row of the cell (Sec. II.B,
 * Eqs. splitCTMRG_C1, _C4, _Tket, _Tbra): dir 0 left, 1 top, 2 right,
 * 3 bottom.  Each new environment tensor is divided by its max |entry|. */
SCTM_API int split_ctmrg_move(sctm_handle h, int dir);

/* n full directional steps (left, top, right, bottom) = n sweeps. */
SCTM_API int split_ctmrg_sweeps(sctm_handle h, int n);

/* Full directional steps until the environment reaches its fixed point
 * (Sec. II.B iterates the steps until the environment converges; the paper
 * fixes no measure, this one is the engine's reading).  After each step the
 * singular values of every corner of every site, each divided by the largest,
 * are compared with those before the step; delta = max over corners of the
 * 2-norm of the difference.  Stops after the first step with delta < tol, or
 * after max_sweeps steps.  tol <= 0 selects 1e-12 when the contractions run
 * in FP64 (precision 0, 3) and 1e-7 when they run in FP32 (precision 1, 2).
 * sweeps_done and last_delta (host, may be NULL) receive the steps taken and
 * the last delta (HUGE_VAL when max_sweeps = 0); converged iff
 * *last_delta < tol.  Both algorithms.  Errors: SCTM_ERR_ARG (no init,
 * max_sweeps < 0), SCTM_ERR_SVD_NOCONV, SCTM_ERR_NONFINITE (a corner
 * spectrum is not finite), SCTM_ERR_CUDA.  Synchronises the stream. */
SCTM_API int split_ctmrg_run(sctm_handle h, int max_sweeps, double tol, int* sweeps_done, double* last_delta);

/* Projector pair of one cut of the move `dir` at the current environment,
 * without moving.  colour: 0 green, 1 teal, 2 yellow, 3 red (Sec. II.B, App. A).
 * (x, y) is the site in the frame of the move (the left-move frame is the
 * lattice itself).  P_up_dev: [k][alpha], P_dn_dev: [alpha][k] with k = chi_E
 * (green, teal) or chi_I (yellow, red) and alpha = k*D (green, teal; yellow in
 * order 0; red in order 1), k*p*D (red in order 0: [k][p][D]) or k*D*p (yellow
 * in order 1: [k][D][p]); s_host receives the k largest singular values of
 * the decomposed core. */
SCTM_API int ctmrg_projectors(sctm_handle h, int dir, int x, int y, int colour, double* P_up_dev, double* P_dn_dev,
                     double* s_host);

/* Energy per site from 2x2 patches of the environment: the expectation value of
 * the Hamiltonian that Sec. III reads off the (split or conventional) CTMRG
 * environment, here of a two-site bond operator on the square lattice.
 * (1/N) sum over patch anchors of half of the four nearest-neighbour bond
 * values plus both diagonal bond values; each bond value is Tr(rho h)/Tr(rho)
 * with rho the two-site reduced density matrix of the patch.
 * h_nn_host: p^2 x p^2 nearest-neighbour operator; h_diag_host: diagonal
 * operator or NULL.  Synchronises and writes *e_per_site (host). */
SCTM_API int energy_2x2(sctm_handle h, const double* h_nn_host, const double* h_diag_host, double* e_per_site);

/* Energy and its gradient with respect to A_cell: the variational gradient of
 * Sec. III, obtained by reverse-mode differentiation through the CTMRG at the
 * cost of the CTMRG itself (Sec. I, Sec. III).  Initial environment,
 * `sweeps` full steps, 2x2 energy, then the reverse pass through all of it
 * (one environment checkpoint per directional move, each move recomputed with
 * hand-written adjoints; SVD adjoint with Lorentzian broadening; the energy is
 * differentiated one 2x2 patch at a time).  grad_dev has the layout of A_cell.  Leaves the converged
 * environment in the handle. */
SCTM_API int energy_grad(sctm_handle h, const double* A_cell_dev, int sweeps, const double* h_nn_host,
                const double* h_diag_host, double* e_per_site, double* grad_dev);

/* The energy and gradient of energy_grad (Sec. III) with host buffers: copies
 * A_cell_host (layout of A_cell, caller-owned host memory) to the device, runs
 * energy_grad, and copies the gradient into grad_host (same layout, caller-
 * owned).  Synchronises; errors as energy_grad, plus SCTM_ERR_CUDA for a
 * failed copy. */
SCTM_API int energy_grad_host(sctm_handle h, const double* A_cell_host, int sweeps, const double* h_nn_host,
                     const double* h_diag_host, double* e_per_site, double* grad_host);

/* Energy per site at the converged environment and its gradient by implicit
 * differentiation of the fixed point env* = F(env*, A).  Sec. II.B iterates
 * full steps f (the four directional moves) until the environment converges,
 * and Sec. I / Sec. III differentiate the converged energy.  The rule follows
 * from the implicit function theorem:
 *   dE/dA = dE/dA|env* + x^T dF/dA|env*,  x = dE/denv* + x^T dF/denv|env*.
 * F is f applied p times, p the smallest number of steps (at most max_period;
 * <= 0: 4) after which no entry of any environment tensor has moved by more
 * than fixed_point_tol of that tensor's largest entry.  At converged spectra
 * the signs of the sign-fixed projectors, and with them rows of the
 * environment tensors, can still cycle from step to step; p closes the cycle.
 * Steps: initial environment, full steps until the corner spectra change by
 * less than tol (as split_ctmrg_run) or max_sweeps; the period search
 * (SCTM_ERR_NOT_FIXED_POINT when there is none); the energy's reverse pass at
 * env*; x by iterating its equation from x = dE/denv* until the change is below
 * solve_tol of |x|, at most max_iter times, else SCTM_ERR_NO_CONVERGENCE.  Each
 * iteration is one reverse pass through the 4p moves of F, recomputed from
 * checkpoints with the decompositions reused.
 * Tolerances <= 0 take the defaults: tol 1e-13, fixed_point_tol 1e-9,
 * solve_tol 1e-12 at precisions 0 and 3; 1e-7, 1e-5, 1e-6 in the precisions
 * with FP32-level contractions (1, 2, 4).
 * grad_dev (device, layout of A_cell) receives dE/dA.  Optional host outputs:
 * sweeps_done, period_out (p), solver_iterations, fixed_point_change (the
 * largest relative change after the last step tried).  Leaves env* in the
 * handle; synchronises. */
SCTM_API int energy_grad_implicit(sctm_handle h, const double* A_cell_dev, int max_sweeps, double tol,
                                  const double* h_nn_host, const double* h_diag_host, double fixed_point_tol,
                                  double solve_tol, int max_iter, int max_period, double* e_per_site,
                                  double* grad_dev, int* sweeps_done, int* period_out, int* solver_iterations,
                                  double* fixed_point_change);

/* Environment of site (x, y) (the split environment of Fig. 2, Sec. II.B; for
 * the conventional algorithm the environment of Fig. 1, Sec. II.A) into
 * out_dev (device, caller-owned), packed in the order C1 T1k T1b C2
 * T2k T2b C3 T3b T3k C4 T4b T4k (chi_E^2 doubles per corner, chi_E*D*chi_I per
 * edge, shapes as in sctm_config.chi_I); for the conventional algorithm C1 T1
 * C2 T2 C3 T3 C4 T4 (chi^2 or chi*D*D*chi each). */
SCTM_API int sctm_get_env(sctm_handle h, int x, int y, double* out_dev);

/* Singular value decomposition M = U diag(S) V^T of an m x n row-major
 * matrix (m >= n) by one-sided Jacobi in FP64 -- the decomposition behind
 * every projector (Sec. II.B).  U: m x n, S: n (descending), V: n x n, all
 * device buffers owned by the caller; the handle's workspace is the scratch.
 * Synchronises; SCTM_ERR_SVD_NOCONV if the sweep limit was reached. */
SCTM_API int sctm_svd(sctm_handle h, int m, int n, const double* M_dev, double* U_dev, double* S_dev,
                      double* V_dev);

/* The Jacobi SVD of sctm_svd without a handle and without any allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * must not allocate device memory while they run -- code running inside an
 * allocator callback, or a loop held to a fixed memory budget -- and that hold
 * no engine handle.  Its scratch is one statically sized device array per
 * device (16 MiB + 8 KiB), so:
 *  - sizes are limited to (m + n) * n <= 2^21 (e.g. m = n = 1024); larger
 *    matrices return SCTM_ERR_ARG without touching the device;
 *  - calls that overlap in time on one device (two streams, two host threads)
 *    race on that scratch: serialise them;
 *  - the first call on each device looks up the array's address and the
 *    kernel's occupancy; make it before any stream capture begins.
 * Arguments as for sctm_svd (m >= n, device buffers owned by the caller);
 * stream is a cudaStream_t (NULL = legacy default stream).  The call reads the
 * kernel's status word back and synchronises that stream before it returns
 * SCTM_OK, SCTM_ERR_ARG, SCTM_ERR_CUDA or
 * SCTM_ERR_SVD_NOCONV (sweep limit reached).  With sctm_profile recording,
 * the launch is timed with events like every other launch. */
SCTM_API int sctm_svd_noalloc(int m, int n, const double* M_dev, double* U_dev, double* S_dev, double* V_dev,
                              void* stream);

/* Tensor contraction C = alpha * einsum(spec, A, B) + beta * C on the handle's
 * stream, in the handle's precision: the primitive under every absorption,
 * rho network and projector application (Sec. II.B).  spec is an einsum string
 * such as "ab,bc->ac" (one letter per leg, every letter in at least two of the
 * three operands); A_dev, B_dev, C_dev are contiguous row-major device
 * buffers with extents shape_A/B/C (one int per letter).  With beta == 0, C
 * is not read.  Synchronises. */
SCTM_API int sctm_einsum(sctm_handle h, const char* spec, const double* A_dev, const int* shape_A,
                         const double* B_dev, const int* shape_B, double* C_dev, const int* shape_C,
                         double alpha, double beta);

/* Per-kernel-family timing.  enable=1 starts recording CUDA events around
 * every kernel launch (on the handle's stream); enable=0 stops and writes
 * out[4][4] = {CUDA-core contraction, svd, other, tensor-core contraction} x
 * {device ms, launches, algorithmic flops, algorithmic bytes}.  Not for timed regions of record: the events
 * themselves serialise nothing but add host overhead. */
SCTM_API int sctm_profile(sctm_handle h, int enable, double* out);

/* Device workspace high-water mark in bytes. */
SCTM_API int sctm_workspace_high_water(sctm_handle h, size_t* bytes);

/* Split-K autotuning, the engine's own tuner (the paper has no counterpart).
 * A contraction whose output has too few tiles to fill the GPU splits K over
 * more CTAs, by a rule in each kernel.  enable = 1: from now on, the first
 * calls of every such contraction shape (kernel, batch, M, N, K) run with the
 * rule's split count, half and twice it, and no split -- one candidate per
 * call, each a complete contraction, timed with events on the handle's stream
 * (the calls synchronise while a shape is being explored) -- and later calls
 * of that shape use the fastest.  enable = 0 stops exploring; shapes already
 * tuned keep their choice for the handle's lifetime.  Errors: none beyond
 * SCTM_ERR_ARG for a null handle. */
SCTM_API int sctm_autotune(sctm_handle h, int enable);

/* The tuner's choices: up to max_rows rows of nine doubles into out (host,
 * caller-owned): kernel (0 FP64 CUDA cores, 1 FP32 CUDA cores, 2 3xTF32
 * tensor cores, 3 BF16-slice tensor cores), batch, M, N, K, the rule's split
 * count and its milliseconds, the chosen count and its milliseconds.  *rows
 * receives the number of tuned shapes (which may exceed max_rows).
 * Synchronises the stream. */
SCTM_API int sctm_autotune_table(sctm_handle h, double* out, int max_rows, int* rows);

/* Limits of the handle's bounded device loops, for fault-injection tests (the
 * paper has no counterpart).  svd_max_sweeps: sweeps of every Jacobi SVD the
 * handle runs (<= 0: the default 60); a decomposition that reaches it makes
 * the call return SCTM_ERR_SVD_NOCONV.  pipeline_wait_s: how long the main
 * loop of a tensor-core contraction waits on one of its mbarriers before it
 * gives up (< 0: the default 2 s; 0: at the first wait not already
 * satisfied); a kernel that gives up waits with the full 2 s limit for the
 * copies and MMAs it issued, frees its tensor memory, returns, and the call
 * returns SCTM_ERR_CUDA.  In both cases the handle stays usable: the failed
 * call is rolled back.  Errors: SCTM_ERR_ARG for pipeline_wait_s > 60. */
SCTM_API int sctm_set_limits(sctm_handle h, int svd_max_sweeps, double pipeline_wait_s);

#ifdef __cplusplus
}
#endif
#endif /* SPLITCTMRG_H */
