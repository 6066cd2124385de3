/*
 * dftfe_gb300.h -- C ABI of a GB300 (sm_103a) implementation of one
 * Chebyshev-filtered subspace iteration (ChFSI) pass for the spectral
 * finite-element Kohn-Sham eigenproblem of DFT-FE 1.0 (Das, Motamarri,
 * Subramanian, Rogers, Gavini, Comput. Phys. Commun.).
 *
 * Problem (Sec. 2.3): the generalised eigenproblem H u = eps M u with C0
 * Lagrange elements on Gauss-Lobatto-Legendre (GLL) nodes (Eq. fem), lumped
 * diagonal M by GLL quadrature, is solved in the Loewdin form
 * H~ = M^-1/2 H M^-1/2 (Eq. hep).  H = H^loc + H^nl at the Gamma point
 * (Eq. discreteHam without the GGA term; Eq. nonlocalHamDiscrete), and at a Bloch
 * k-point on complex blocks through the _z calls (Sec. 2.1, the reduced equation).
 * The pass (Sec. 3.1-3.2): Chebyshev filter (Eq. chebyfilter), then
 * Cholesky-Gram-Schmidt and Rayleigh-Ritz (the orthonormalise-first reading of
 * Alg. 2), then residuals.
 *
 * Conventions shared by every call:
 *  - Every call returns dftfe_status; nothing throws or aborts across the ABI.
 *    On error, dftfe_last_error() returns a thread-local message.
 *  - Wavefunction blocks X are DoF-major (Sec. 4.3: all values of one DoF are
 *    contiguous): element (i, j) of an M x ncol block is X[i*ld + j], ld >= ncol,
 *    FP64, in DEVICE memory owned by the caller.
 *  - Handles own their device state and workspace; workspace is allocated on
 *    first use and freed by *_destroy.  A handle is not thread-safe; distinct
 *    handles are independent.  All device work of a ham is enqueued on the
 *    stream given to dftfe_ham_create and is asynchronous, except calls that
 *    return host scalars (they synchronise that stream and say so).
 *  - On DFTFE_ERR_ARG, outputs are untouched.
 *  - Numbering (the paper is silent; this library's contract): global node
 *    (ix, iy, iz) -> ix + gx*(iy + gy*iz), gx = ncell[0]*degree; cell
 *    (cx, cy, cz) -> cx + nx*(cy + ny*cz); cell-local node (a, b, c) ->
 *    a + (p+1)*(b + (p+1)*c); quadrature points in the same order, x fastest.
 *  - Periodic cubes/cuboids only, >= 2 cells per axis.
 */
#ifndef DFTFE_GB300_H
#define DFTFE_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DFTFE_OK = 0,
  DFTFE_ERR_ARG = 1,      /* invalid argument; outputs untouched */
  DFTFE_ERR_OOM = 2,      /* device allocation failed */
  DFTFE_ERR_CUDA = 3,     /* a CUDA runtime call or launch failed */
  DFTFE_ERR_NOT_SPD = 4,  /* overlap matrix S not positive definite (X untouched) */
  DFTFE_ERR_NOCONV = 5,   /* dense eigensolver did not converge */
  DFTFE_ERR_TIMEOUT = 6,  /* a bounded device-side wait gave up */
  DFTFE_ERR_STATE = 7     /* call out of order (e.g. no potential set) */
} dftfe_status;

typedef enum {
  DFTFE_FP64 = 0,          /* everything in FP64 */
  DFTFE_MIXED_BF16X3 = 1,  /* filter: cell products as 3-term BF16 splits (hi*hi + hi*lo +
                              lo*hi) on the tensor cores (tcgen05), FP32 accumulation, FP32
                              vectors; CholGS, Rayleigh-Ritz and residuals in FP64 */
  DFTFE_MIXED_TF32X3 = 2,  /* as above with 3-term TF32 splits (about 2^-21 relative per
                              product instead of 2^-16) */
  DFTFE_FP64_FLOAT_PAIRS = 3, /* dftfe_ham_apply(_z) only: FP64-accurate cell products from
                              pairs of floats (error-free products, TwoSum accumulation, about
                              44 significant bits) on the FP32 pipes; FP64 in and out */
  DFTFE_FP64_SLICES = 4     /* dftfe_ham_apply(_z) only: FP64-accurate cell products on the
                              tensor cores from exact digit products: each cell-matrix row and
                              each column of X as 41-bit fixed point (relative to its largest
                              entry) in six 7-bit bf16 digits, the 21 digit products of order
                              <= 5 accumulated exactly in FP32 (each sum stays below 2^24),
                              combined in 64-bit integers; error about 2^-39 |h|max |x|max per
                              term.  Degree <= 7 (DFTFE_ERR_ARG beyond); FP64 in and out */
  /* In dftfe_cholgs, dftfe_rayleigh_ritz and the pass, either mixed value selects the
     mixed overlap / projection / rotation of Sec. 3.2: diagonal entries of S and H^ and
     the diagonal part of each rotation in FP64, off-diagonal parts in FP32; W = H~X
     for the projection and the residuals uses the exact digit products of
     DFTFE_FP64_SLICES (the float pairs of DFTFE_FP64_FLOAT_PAIRS beyond degree 7; split
     products there would move the Ritz values by 1e-6 to 2e-6 Ha); the Cholesky
     factorisation and the eigensolve stay FP64. */
} dftfe_precision;

typedef struct dftfe_mesh_s* dftfe_mesh; /* opaque, library-owned */
typedef struct dftfe_ham_s* dftfe_ham;   /* opaque, library-owned */

/* Mesh description.  L: box lengths (bohr).  ncell: cells per axis (>= 2).
 * degree: FE degree p (1..8).  periodic: must be {1,1,1}.
 * vquad: rule for the local-potential term of Eq. quadLocal (the paper does not
 *   fix n_q): 0 = Gauss-Legendre with nq1d points per axis (dense V^c),
 *   1 = GLL collocated on the nodes (V^c diagonal).
 * nq1d: Gauss points per axis for vquad = 0 (0 means degree + 1, max 12). */
typedef struct {
  double L[3];
  int ncell[3];
  int degree;
  int periodic[3];
  int vquad;
  int nq1d;
} dftfe_mesh_desc;

/* Spectrum bounds for the filter (Eq. chebyfilter: Hbar = c1 H~ + c2 maps the
 * unwanted interval [a, b] to [-1, 1]).  a0: estimate of the lowest wanted
 * eigenvalue, used by the scaled recurrence (Zhou-Saad); NaN selects the
 * unscaled three-term recurrence T_{k+1} = 2 x T_k - T_{k-1}. */
typedef struct {
  double a, b, a0;
} dftfe_bounds;

/* ---------------------------------------------------------------- mesh (host) */

/* Create the mesh description and its 1D GLL / Gauss rules (Sec. 2.3, Eq. fem;
 * lumped M in the text after Eq. hep).  Host-only; no device memory. */
dftfe_status dftfe_mesh_create(const dftfe_mesh_desc* desc, dftfe_mesh* out);

/* Sizes: ndofs M = prod(ncell*degree), ncells, nodes_per_cell (p+1)^3,
 * quad_per_cell (nq1d^3 for vquad 0, (p+1)^3 for vquad 1).  Any pointer may be NULL. */
dftfe_status dftfe_mesh_info(dftfe_mesh mesh, int64_t* ndofs, int64_t* ncells,
                             int* nodes_per_cell, int* quad_per_cell);

/* Coordinates in HOST memory: node_xyz (M x 3) and, if non-NULL, quad_xyz
 * (ncells x quad_per_cell x 3) of the potential quadrature points, both in the
 * numbering above (used by callers to evaluate V and projectors).  Either may be NULL. */
dftfe_status dftfe_mesh_coords(dftfe_mesh mesh, double* node_xyz, double* quad_xyz);

dftfe_status dftfe_mesh_destroy(dftfe_mesh mesh);

/* ---------------------------------------------------------------- Hamiltonian */

/* Build the device operator state on the current CUDA device: cell -> global
 * map, lumped mass M (a1), the shared GLL stiffness, the packed product table
 * P of Eq. gemmLoc, and storage for the N_c dense cell matrices.  stream: a
 * cudaStream_t (NULL = legacy default stream) on which every later call of this
 * ham runs.  The mesh must outlive the ham. */
dftfe_status dftfe_ham_create(dftfe_mesh mesh, void* stream, dftfe_ham* out);

/* A second ham over src's mesh, on src's stream, that uses src's local operator: the cell
 * matrices H~^c that dftfe_ham_set_potential(src, ...) forms and every form the library
 * derives from them (the FP32 plane of the split products, the digit rows of the exact-slice
 * products, the float pairs), built once on first use and read by both.  The local term
 * -1/2 lap + V_loc is the same at every Bloch k-point of a system (Sec. 2.1: only the k terms
 * and the projector phases depend on k), so the k-point hams of one system made this way
 * hold one copy of it instead of one each.  The new ham has its own nonlocal term, k-point,
 * workspace, graphs and autotuner.  dftfe_ham_set_potential on it returns DFTFE_ERR_STATE
 * (set the potential on src; the change is seen by every ham that shares it), as does
 * dftfe_ham_destroy(src) while a ham made from it exists.  src must own its operator (not be
 * made by this call), and the current device must be src's (DFTFE_ERR_ARG otherwise). */
dftfe_status dftfe_ham_create_shared(dftfe_ham src, dftfe_ham* out);

/* Set the local potential (a2; Sec. 4.2, Eq. quadLocal / Eq. gemmLoc):
 * v_quad is DEVICE memory, ncells x quad_per_cell FP64 values V(x_q).  Forms
 * V^c for all cells with one packed-symmetric GEMM K = P V, adds the stiffness
 * K^c = 1/2 int grad N . grad N, and stores H~^c = D_c^-1/2 (K^c + V^c) D_c^-1/2.
 * Asynchronous; v_quad may be freed once the stream reaches this point. */
dftfe_status dftfe_ham_set_potential(dftfe_ham ham, const double* v_quad);

/* Set the nonlocal projector term (a3; Eq. nonlocalHamDiscrete, Alg. 4):
 * nproj projectors in CSR by projector, all in HOST memory: rowptr (nproj+1),
 * node (rowptr[nproj] global node indices), chi (projector values chi_a(x_j) at
 * those nodes), h (nproj couplings, Ha).  With GLL collocation C_ja = M_jj chi_a(x_j),
 * so the library stores C~ = M^1/2 chi and applies H~_nl = C~ diag(h) C~^T.
 * nproj = 0 removes the term.  Copies the inputs; synchronises the stream. */
dftfe_status dftfe_ham_set_nonlocal(dftfe_ham ham, int nproj, const double* h,
                                    const int64_t* rowptr, const int64_t* node,
                                    const double* chi);

dftfe_status dftfe_ham_destroy(dftfe_ham ham);

/* Copy device state out for inspection: mass (M doubles), cell_map
 * (ncells x nodes_per_cell int32), cell matrices of cells [c0, c0+count)
 * (count x n_c x n_c doubles).  All outputs DEVICE memory; any may be NULL. */
dftfe_status dftfe_ham_export(dftfe_ham ham, double* mass, int32_t* cell_map,
                              int64_t c0, int64_t count, double* cell_mats);

/* Y = H~ X for an M x ncol block (a4 + a5; Eq. celldgemm and Alg. 4): gather to
 * cells, dense per-cell product, colour-ordered scatter-add, plus C~ h C~^T X.
 * X and Y in DEVICE memory, must not overlap.  prec selects the FP64 cell kernel, the
 * split-precision tensor-core kernel (FP32 inside, converted at both ends; at most 512
 * nodes per cell, i.e. p <= 7), or one of the two FP64-accurate forms used for W in the
 * mixed passes (DFTFE_FP64_FLOAT_PAIRS; DFTFE_FP64_SLICES, p <= 7). */
dftfe_status dftfe_ham_apply(dftfe_ham ham, const double* X, int64_t ldx,
                             double* Y, int64_t ldy, int ncol, dftfe_precision prec);

/* Autotuner (no counterpart in the paper).  With enable = 1, the first FP64 cell-product
 * pass over the mesh for each column count (real columns: 2 ncol for the _z calls) times
 * every launch shape of the FP64 cell kernel -- 64, 128, ... rows of a cell per CTA, and the
 * built-in heuristic -- on the caller's block into a scratch output and keeps the fastest
 * for this ham (that first call synchronises the stream).  Likewise the first TF32x3
 * cell-product launch of the split-precision filter (Sec. 4.3's cell products on the tensor
 * cores) times every launch shape of that kernel -- the split A operand staged in tensor
 * memory (where the accumulators leave room: at most three 128-row M-tiles, p <= 6; with 6 or
 * 8 landing slots for the cell-matrix tiles) or in a shared-memory ring, and the cells dealt to the persistent CTAs round-robin or in contiguous
 * ranges -- on the launch's own operands and keeps the fastest (queried with
 * dftfe_autotune_query_mixed).  Tuning is skipped while the stream is being captured.  Every
 * shape gives bit-identical results.  enable = 0 restores the defaults; either call forgets
 * earlier choices. */
dftfe_status dftfe_ham_autotune(dftfe_ham ham, int enable);

/* The tuned TF32x3 cell-kernel shape of this ham's mesh: HOST atmem (1 = A operand in tensor
 * memory, 0 = in shared memory, -1 = not tuned yet), deep (with atmem: 0 = 6 landing slots for
 * the cell-matrix tiles and 4 stages for the gathered X, 1 = 8 and 3 in the same shared
 * memory), deal (0 = round-robin, 1 = contiguous ranges), best_ms and default_ms (one launch
 * over all cells in the chosen and in the default shape -- tensor memory where it fits, 6 and
 * 4, round-robin; may be NULL).  Every output -1 before tuning. */
dftfe_status dftfe_autotune_query_mixed(dftfe_ham ham, int* atmem, int* deep, int* deal, double* best_ms,
                                        double* default_ms);

/* The tuned shape for ncol real columns: HOST rows_per_cta (0 = the heuristic won, -1 = not
 * tuned yet), best_ms and heuristic_ms (one cell-product pass over the mesh; may be NULL). */
dftfe_status dftfe_autotune_query(dftfe_ham ham, int ncol, int* rows_per_cta, double* best_ms,
                                  double* heuristic_ms);

/* CUDA graphs (no counterpart in the paper).  With enable = 1, a WHOLE dftfe_chfsi_pass
 * (filter, Cholesky-Gram-Schmidt, Rayleigh-Ritz, residuals) runs as one CUDA graph launch with
 * a single host synchronisation at its end: the Cholesky and eigensolver statuses and the
 * tensor-core kernels' timeout flags stay on the device (the kernels that rotate X or W do no
 * work once the factorisation or the eigensolve has failed, so X is left as filtered) and are
 * read once, with the Ritz-value ends for the bounds update.  Errors are those of the plain
 * pass.  For dftfe_chfsi_pass_z the filter phase (every block's Chebyshev recurrence, about
 * degree x (3 + colours) launches per block) is one graph launch.  The first pass with given
 * (precision, ncol, block, degree) runs directly, later ones capture from the ham's stream and
 * update the cached executable (bounds change only kernel arguments).  Results are
 * bit-identical to enable = 0.  Per-kernel profiling timers (dftfe_profile_query) record
 * nothing inside a captured region.  Either call drops the cached graphs; synchronises the
 * stream. */
dftfe_status dftfe_ham_use_graphs(dftfe_ham ham, int enable);

/* HOST counts since dftfe_ham_use_graphs: graph launches and instantiations (an update that
 * the driver refuses, e.g. after a new potential adds the split-tile launches, instantiates
 * afresh). */
dftfe_status dftfe_graph_query(dftfe_ham ham, int64_t* replays, int64_t* instantiations);

/* --------------------------------------------------------------- ChFSI steps */

/* Counter-based SplitMix64 uniforms in [-1/2, 1/2) (Steele, Lea, Flood 2014):
 * out[i] = u(seed, offset + i) with u(s, k) = (mix(s + (k+1)*0x9E3779B97F4A7C15)
 * >> 11) * 2^-53 - 1/2.  out is DEVICE memory (n doubles); runs on `stream`.
 * For an M x ncol block with ld = ncol, element (i, j) uses k = i*ncol + j. */
dftfe_status dftfe_random_uniform(double* out, int64_t n, uint64_t seed,
                                  int64_t offset, void* stream);

/* k-step Lanczos with full reorthogonalisation on H~ (a7; the paper only says
 * the degree follows the upper bound of H~, Sec. 3.1).  v0: DEVICE start vector
 * (M doubles) or NULL to use dftfe_random_uniform(seed, offset 0).  Writes to
 * HOST out3 = {theta_min, theta_max, b}, b = theta_max + |beta_k| |s_k| (a
 * Ritz-residual upper bound).  Synchronises the stream. */
dftfe_status dftfe_lanczos(dftfe_ham ham, int k, const double* v0, uint64_t seed,
                           double* out3);

/* First-pass bounds from dftfe_lanczos: a0 = theta_min, b as above,
 * a = theta_min + (b - theta_min) * max(4 nstates / M, 0.05).  Host out. */
dftfe_status dftfe_spectrum_bounds(dftfe_ham ham, int k, uint64_t seed, int nstates,
                                   dftfe_bounds* out);

/* Chebyshev filter in place on ncol columns (a4-a6; Eq. chebyfilter): degree m
 * applications of H~ with the scaled (a0 finite) or unscaled (a0 = NaN)
 * three-term recurrence; X <- p_m(H~) X.  The caller filters a block of B_f
 * columns per call (Sec. 4.3 blocking).  Requires b > a, and a0 < a when scaled. */
dftfe_status dftfe_chebyshev_filter(dftfe_ham ham, double* X, int64_t ld, int ncol,
                                    int degree, const dftfe_bounds* bounds,
                                    dftfe_precision prec);

/* Cholesky-Gram-Schmidt in place (a8, a9; Alg. 2 steps 1a, 2a, 3b):
 * S = X^T X (lower triangle), S = L L^T, X <- X L^-T.  DFTFE_ERR_NOT_SPD when a
 * Cholesky pivot is not above 1e-14 times its diagonal entry of S (numerically
 * singular overlap); X is then untouched.  Synchronises the stream (reads the factorisation status). */
dftfe_status dftfe_cholgs(dftfe_ham ham, double* X, int64_t ld, int ncol,
                          dftfe_precision prec);

/* Rayleigh-Ritz on orthonormal X (a10-a12; Alg. 2 steps 1b, 2b-c, 3a):
 * W = H~ X, H^ = X^T W (lower triangle, symmetric), H^ = Q Theta Q^T with
 * Theta ascending and each column of Q signed so its largest-|.| entry is
 * positive, X <- X Q.  evals: DEVICE, ncol doubles.  HX: DEVICE M x ncol (ldhx)
 * receiving W Q = H~ X_new, or NULL (the library then uses its own workspace).
 * Synchronises the stream. */
dftfe_status dftfe_rayleigh_ritz(dftfe_ham ham, double* X, int64_t ld, int ncol,
                                 double* evals, double* HX, int64_t ldhx,
                                 dftfe_precision prec);

/* Residual norms (a13): kind 0 -> ||W_i - theta_i X_i||_2 in the Loewdin basis
 * (X orthonormal); kind 1 -> ||H psi - theta M psi|| / ||psi|| with
 * psi = M^-1/2 x (the generalised form).  X, HX (ld), evals, resid: DEVICE. */
dftfe_status dftfe_residuals(dftfe_ham ham, const double* X, const double* HX,
                             int64_t ld, int ncol, const double* evals,
                             double* resid, int kind);

/* One ChFSI pass (Sec. 3.1-3.2): filter each block of `block` columns with the
 * same bounds, CholGS on all ncol columns, Rayleigh-Ritz, Loewdin residuals,
 * then the bounds update a <- theta_ncol, a0 <- theta_1 (b kept; a0 stays NaN
 * for the unscaled filter).  evals, resid: DEVICE (ncol each).  inout: HOST.
 * Synchronises the stream. */
dftfe_status dftfe_chfsi_pass(dftfe_ham ham, double* X, int64_t ld, int ncol,
                              int block, int degree, dftfe_bounds* inout,
                              double* evals, double* resid, dftfe_precision prec);

/* ---------------------------------------------- spectrum splitting and density */

/* Spectrum-splitting Rayleigh-Ritz (Alg. 2 steps 1b, 2 and 3a) on an orthonormal X
 * (Psi_o, e.g. after dftfe_cholgs): all ncol Ritz values, ascending, to evals (DEVICE,
 * ncol), and the Ritz vectors of the top nfr values, Psi_fr = X Q'_fr, to Xfr (DEVICE
 * M x nfr, ldfr >= nfr; 1 <= nfr <= min(ncol, 512)).  X is not modified.  prec as in
 * dftfe_rayleigh_ritz.  Synchronises the stream. */
dftfe_status dftfe_rayleigh_ritz_split(dftfe_ham ham, const double* X, int64_t ld, int ncol,
                                       int nfr, double* evals, double* Xfr, int64_t ldfr,
                                       dftfe_precision prec);

/* Fermi level (Alg. 3 step 1): mu with 2 (n_oc + sum_i f(evals_fr[i], mu)) = n_elec,
 * f(e, mu) = 1 / (1 + exp((e - mu) / kT)) (kT in Ha; the paper uses T = 500 K), the
 * lowest n_oc states fully occupied.  evals_fr: DEVICE nfr values; f_fr: DEVICE nfr
 * occupations written; mu: HOST.  DFTFE_ERR_ARG unless 2 n_oc < n_elec < 2 (n_oc + nfr).
 * Runs on `stream` and synchronises it. */
dftfe_status dftfe_fermi_level(const double* evals_fr, int nfr, int n_oc, double n_elec,
                               double kT, double* f_fr, double* mu, void* stream);

/* Electron density (Alg. 3 steps 2-3) at the quadrature points of every cell (the
 * mesh's vquad rule): rho = 2 [ sum_i (n^T psi^_o,i)^2 + sum_k (f_k - 1)(n^T psi^_fr,k)^2 ]
 * with psi^ = M^-1/2 psi~.  Xo: DEVICE M x ncol (ldo), the orthonormal basis; Xfr: DEVICE
 * M x nfr (ldfr) and f_fr: DEVICE nfr (may be NULL when nfr = 0); rho: DEVICE
 * ncells x quad_per_cell.  FP64. */
dftfe_status dftfe_density(dftfe_ham ham, const double* Xo, int64_t ldo, int ncol,
                           const double* Xfr, int64_t ldfr, int nfr, const double* f_fr,
                           double* rho);

/* Allocation-free Cholesky-Gram-Schmidt (the paper has no counterpart; this is an
 * interface for callers that cannot allocate device memory at the call site, e.g.
 * inside a fixed memory pool or a framework step that forbids cudaMalloc).  Same
 * result as dftfe_cholgs (S = X^T X, S = L L^T, X <- X L^-T) on an M x ncol FP64
 * block X (DEVICE, ld), without a ham and without allocating: all scratch lives in
 * one static device array of about 20 MiB that every GPU loading this library holds
 * until exit.  ncol above DFTFE_NOALLOC_MAX_COLS returns DFTFE_ERR_ARG.
 * Work runs on `stream` (a cudaStream_t, NULL = legacy default) and the call
 * synchronises it (it reads the factorisation status).  The first call on each
 * device resolves the scratch address (cudaGetSymbolAddress; nothing is copied), so
 * make that first call before any stream capture.  X must be device memory of the
 * current device (else DFTFE_ERR_ARG).  Every call shares the one scratch array and
 * reuses whatever the last call left there (each call overwrites all scratch it
 * reads); calls that overlap on the GPU (other streams, other threads) race on it
 * and must be serialised by the caller.  DFTFE_ERR_NOT_SPD leaves X untouched. */
#define DFTFE_NOALLOC_MAX_COLS 512
dftfe_status dftfe_cholgs_noalloc(double* X, int64_t ld, int64_t M, int ncol, void* stream);

/* -------------------------------------------------------------- Bloch k-points */
/* The periodic part u of a Bloch state psi = e^{ik.x} u (Sec. 2.1, Eq. bloch) solves the reduced
 * equation after Eq. bloch.  Discretised with the same basis and quadratures as at the Gamma
 * point, its Loewdin form is
 *   H~^k = H~_loc + 1/2 |k|^2 - i sum_d k_d G~_d + C~^k diag(h) C~^k^H,
 * G~_d = M^-1/2 G_d M^-1/2 with G_d,jl = int N_j dN_l/dx_d by GLL quadrature on the nodes, and
 * C~^k_ja = M_jj^1/2 chi_a(x_j) e^{-ik.d_ja} with d_ja = x_j - R_a the minimum-image
 * displacement (the Bloch sum of the projector; projectors cut off within half the box).
 * The _z calls act on COMPLEX blocks: complex128, DoF-major, element (i, j) of an M x ncol
 * block at X[2 (i ld + j)] (real part) and X[2 (i ld + j) + 1] (imaginary part), ld >= ncol
 * counted in complex elements (the layout of C99 double complex and torch.complex128),
 * DEVICE memory owned by the caller.  Arithmetic is FP64 throughout.  The Gamma-point calls
 * of the same ham are unaffected.  The complex Rayleigh-Ritz multiplies each eigenvector
 * column of the subspace problem by the phase that makes its largest-|.| entry real and
 * positive (for deterministic output).  Every _z call other than dftfe_ham_set_kpoint returns
 * DFTFE_ERR_STATE before the first dftfe_ham_set_kpoint, and after a dftfe_ham_set_nonlocal
 * that came later than the last dftfe_ham_set_kpoint. */

/* Set the wave vector k (HOST, 3 doubles, bohr^-1) of the _z calls.  disp: HOST nnz x 3
 * displacements d_e = x_node(e) - R_atom (minimum image) of the entries e of the CSR passed to
 * the last dftfe_ham_set_nonlocal, in its order; NULL only when no projectors are set.
 * Non-finite k or displacements: DFTFE_ERR_ARG.  Synchronises the stream. */
dftfe_status dftfe_ham_set_kpoint(dftfe_ham ham, const double* k, const double* disp);

/* The k.grad stencil the _z calls apply (host only, no device work): on this structured
 * periodic mesh G~_d acts along axis d alone, G~_d = G~1_d with G~1_d = m_d^-1/2 G1_d m_d^-1/2,
 * G1_d the assembled 1D periodic matrix of int l_a l_b' (= w_a l_b'(x_a), exact under GLL) and
 * m_d the 1D lumped mass.  table: HOST 3 x p x (2p+1) doubles, entry (d, a, o + p) =
 * k_d G~1_d(i, i + o) for any node i with i mod p = a (zero outside the element couplings). */
dftfe_status dftfe_mesh_kpoint_stencil(dftfe_mesh mesh, const double* k, double* table);

/* Y = H~^k X for complex M x ncol blocks (X, Y DEVICE, not overlapping).  prec as in
 * dftfe_ham_apply: FP64; DFTFE_FP64_SLICES or DFTFE_FP64_FLOAT_PAIRS (local part from
 * exact digit products or float pairs on the real view, k terms and projectors FP64: the
 * W of a mixed complex pass uses the former); or a split precision (FP32 complex inside:
 * the split cell products act on the real view, the k terms and projectors in FP32). */
dftfe_status dftfe_ham_apply_z(dftfe_ham ham, const double* X, int64_t ldx, double* Y,
                               int64_t ldy, int ncol, dftfe_precision prec);

/* dftfe_lanczos on the real 2M x 2M form of H~^k (the same spectrum, each eigenvalue
 * twice), acting on the real view of one complex vector: v0 DEVICE, 2M doubles (M complex),
 * or NULL for dftfe_random_uniform(seed) over 2M values.  HOST out3 as in dftfe_lanczos. */
dftfe_status dftfe_lanczos_z(dftfe_ham ham, int k, const double* v0, uint64_t seed,
                             double* out3);

/* dftfe_spectrum_bounds from dftfe_lanczos_z.  Host out. */
dftfe_status dftfe_spectrum_bounds_z(dftfe_ham ham, int k, uint64_t seed, int nstates,
                                     dftfe_bounds* out);

/* dftfe_chebyshev_filter on a complex block with H~^k.  A split precision runs the
 * complex64 form: FP32 complex vectors, split cell products on the real view, the k terms
 * and projectors in FP32. */
dftfe_status dftfe_chebyshev_filter_z(dftfe_ham ham, double* X, int64_t ld, int ncol,
                                      int degree, const dftfe_bounds* bounds,
                                      dftfe_precision prec);

/* Cholesky-Gram-Schmidt on a complex block: S = X^H X, S = L L^H, X <- X L^-H
 * (1 <= ncol <= 1024).  A split precision selects the mixed overlap and rotation of
 * dftfe_cholgs on the real view of X.  DFTFE_ERR_NOT_SPD as dftfe_cholgs.  Synchronises the
 * stream. */
dftfe_status dftfe_cholgs_z(dftfe_ham ham, double* X, int64_t ld, int ncol, dftfe_precision prec);

/* Rayleigh-Ritz on an orthonormal complex block: W = H~^k X, H^ = X^H W (lower triangle,
 * Hermitian), H^ = Q Theta Q^H (Theta ascending, phases as above), X <- X Q.  evals: DEVICE
 * ncol doubles.  HX: DEVICE complex M x ncol (ldhx) receiving W Q, or NULL.  1 <= ncol <=
 * 1024.  Synchronises the stream. */
dftfe_status dftfe_rayleigh_ritz_z(dftfe_ham ham, double* X, int64_t ld, int ncol,
                                   double* evals, double* HX, int64_t ldhx,
                                   dftfe_precision prec);

/* Residual norms of complex columns as dftfe_residuals (kind 0: ||w_i - theta_i x_i||_2;
 * kind 1: the generalised form with psi = M^-1/2 x), |.| the complex modulus (X, HX complex
 * with ld; evals, resid DEVICE ncol doubles). */
dftfe_status dftfe_residuals_z(dftfe_ham ham, const double* X, const double* HX, int64_t ld,
                               int ncol, const double* evals, double* resid, int kind);

/* One ChFSI pass on a complex block at the ham's k-point, as dftfe_chfsi_pass
 * (1 <= ncol <= 1024): DFTFE_FP64 is the complex128 form; a split precision the complex64
 * form (filter in FP32 complex with split cell products; mixed overlap, projection and
 * rotations on the real view; W from float pairs; Cholesky, eigensolve and residuals FP64).
 * Synchronises the stream. */
dftfe_status dftfe_chfsi_pass_z(dftfe_ham ham, double* X, int64_t ld, int ncol, int block,
                                int degree, dftfe_bounds* inout, double* evals, double* resid,
                                dftfe_precision prec);

/* ------------------------------------------------------------ batched passes */
/* Several independent systems (FP64) of uneven mesh size, degree, state count and block
 * size -- each at the Gamma point or at its ham's Bloch k-point (item.kpoint), so several
 * k-points of one system are several hams of the same mesh and potential -- advanced by one
 * ChFSI pass each with shared launches: per Chebyshev step one launch forms the recurrence
 * terms of every Gamma-point system and one launch per colour runs the cell products of
 * every system's cells of that colour (a complex block through its real view); the k-point
 * terms, the nonlocal term, CholGS and Rayleigh-Ritz run per system.  Results are
 * bit-identical to dftfe_chfsi_pass / dftfe_chfsi_pass_z on each system alone (same
 * operations in the same order).  No counterpart in the paper, which runs one system per
 * job. */
typedef struct dftfe_batch_s* dftfe_batch;

typedef struct {
  double* X;            /* device, M x ncol, row stride ld (updated in place) */
  int64_t ld;
  int ncol;             /* 1..2048, <= M */
  int block;            /* filter block size, >= 1 */
  int degree;           /* Chebyshev degree, >= 0 */
  dftfe_bounds bounds;  /* in: filter bounds; out: updated as dftfe_chfsi_pass does */
  double* evals;        /* device, ncol: Ritz values (ascending) */
  double* resid;        /* device, ncol: residual norms */
  int kpoint;           /* 0: real block at the Gamma point; 1: complex block (complex128,
                           ld and ncol in complex elements, ncol <= 1024) at the k-point set on
                           the item's ham by dftfe_ham_set_kpoint, as in dftfe_chfsi_pass_z */
} dftfe_batch_item;

/* Build a batch over nsys (1..4096) distinct Hamiltonians created on one stream; the batch
 * keeps pointers to them (destroy the batch first).  Potentials may change between passes. */
dftfe_status dftfe_batch_create(const dftfe_ham* hams, int nsys, dftfe_batch* out);

/* One pass for every system; items[i] belongs to hams[i].  The systems' pass tails (CholGS,
 * Rayleigh-Ritz, residuals) run one after another and share one workspace that the batch owns
 * (sized by the largest system, freed by dftfe_batch_destroy), so a batch of many k-point
 * items holds one set of tail buffers instead of one per item.  prec is DFTFE_FP64 (shared FP64
 * launches as above) or DFTFE_MIXED_TF32X3: the split-precision filter of Sec. 4.3's cell
 * products on the tensor cores, where per Chebyshev step ONE persistent cell-product launch
 * per FE degree covers every cell of every system still filtering (a work list of
 * (system, cell) pairs; complex items as complex64 through their real view), the assembly
 * with the recurrence, the nonlocal and k-point terms run per system, and CholGS /
 * Rayleigh-Ritz as dftfe_chfsi_pass in that precision.  Either way the results are
 * bit-identical to the single-system passes in the same precision.  Errors as for
 * dftfe_chfsi_pass (checked for all items before any work); DFTFE_ERR_TIMEOUT if a bounded
 * wait of the tensor-core kernel gave up. */
dftfe_status dftfe_batch_chfsi_pass(dftfe_batch batch, dftfe_batch_item* items, dftfe_precision prec);

/* Synchronise the batch's stream and free it (NULL is a no-op). */
dftfe_status dftfe_batch_destroy(dftfe_batch batch);

/* CUDA graph of the batched filter phase (every round and step of every system, one graph
 * launch), as dftfe_ham_use_graphs for one ham: the first batched pass with given item shapes
 * runs directly, later ones capture and update the cached executable.  Bit-identical results.
 * Synchronises the stream and drops cached graphs. */
dftfe_status dftfe_batch_use_graphs(dftfe_batch batch, int enable);

/* HOST counts of graph launches and instantiations of the batch since dftfe_batch_use_graphs. */
dftfe_status dftfe_batch_graph_query(dftfe_batch batch, int64_t* replays, int64_t* instantiations);

/* Autotuner of the batched split-precision filter.  With enable = 1, every distinct
 * cell-product launch of a DFTFE_MIXED_TF32X3 batched pass (one FE degree's systems at one
 * Chebyshev step: keyed by nodes per cell, work items, systems and distinct cell-matrix
 * planes) is timed on its first appearance in every shape -- A operand in tensor memory or
 * shared memory, round-robin or contiguous dealing, and the (system, cell) work list
 * system-major or interleaved cell by cell across the systems, which lets the k-point hams of
 * one system that share a local operator (dftfe_ham_create_shared) read each cell's FP32 tiles
 * at about the same time, once from HBM -- and the fastest is used from then on.  Results are
 * bit-identical to untuned passes.  Synchronises the stream; either call forgets earlier
 * choices and makes the next graphed pass run directly. */
dftfe_status dftfe_batch_autotune(dftfe_batch batch, int enable);

/* The index-th tuned launch (in key order): HOST nodes per cell, work items, atmem, deep, deal
 * (as dftfe_autotune_query_mixed), order (0 = system-major, 1 = interleaved), best_ms and
 * default_ms (may be NULL); every output -1 (0 for the times) when index is past the last. */
dftfe_status dftfe_batch_autotune_query(dftfe_batch batch, int index, int* nodes_per_cell, int* work_items,
                                        int* atmem, int* deep, int* deal, int* order, double* best_ms,
                                        double* default_ms);

/* ------------------------------------------ learned degree / bounds proposer */
/* The network that proposes the Chebyshev degree and the unwanted-interval bounds of the
 * next pass from the last passes' Ritz values, residuals and bounds (a learned replacement
 * for the Lanczos bound estimate plus a fixed degree, which remain its fallback).  A
 * three-layer perceptron, FP32:
 *     h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = W3 h2 + b3,
 * parameters packed in one device vector: W1 (n_hidden x n_in, row-major), b1,
 * W2 (n_hidden x n_hidden), b2, W3 (n_out x n_hidden), b3.  Sizes: 1 <= n_in <= 64,
 * n_hidden in {32, 64, 96, 128}, 1 <= n_out <= 8.  All arrays are device memory, rows of X
 * and Y are samples (row-major); work is enqueued on `stream` (NULL = legacy default stream).
 * Nothing here comes from the paper, which fixes the degree from the bounds (Sec. 3.1). */

/* Number of packed parameters, or -1 for non-positive sizes. */
int64_t dftfe_mlp_param_count(int n_in, int n_hidden, int n_out);

/* Y[n x n_out] = network(X[n x n_in]).  DFTFE_ERR_ARG for sizes out of range or null
 * pointers (n = 0 is a no-op). */
dftfe_status dftfe_mlp_forward(const float* params, int n_in, int n_hidden, int n_out, const float* X,
                               int64_t n, float* Y, void* stream);

/* Training objective L = (1/n) sum_s sum_k w_k (y_sk - t_sk)^2 over the n >= 1 rows of X with
 * targets T[n x n_out] and per-output weights w[n_out] (NULL = all 1).  Writes L to *loss
 * (device, may be NULL) and dL/dparams to grad (device, dftfe_mlp_param_count floats), summed
 * in a fixed order (deterministic).  Uses a stream-ordered temporary of about
 * 2 x SMs x param_count floats. */
dftfe_status dftfe_mlp_loss_grad(const float* params, int n_in, int n_hidden, int n_out, const float* X,
                                 const float* T, const float* w, int64_t n, float* loss, float* grad,
                                 void* stream);

/* One Adam step (Kingma & Ba 2015) at step number t >= 1 on `count` parameters: moment
 * estimates m, v (device, zero before the first step) are updated in place, then
 * params -= lr * mhat / (sqrt(vhat) + eps) with the bias-corrected moments. */
dftfe_status dftfe_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t count, int t,
                            float lr, float beta1, float beta2, float eps, void* stream);

/* ------------------------------------------------------------ instrumentation */

/* Per-kernel timing with CUDA events recorded on the ham's stream around every
 * launch of the named kernel family ("cell_gemm_fp64", "cell_gemm_mixed",
 * "gram", "rotate", ...).  enable != 0 starts recording (and clears totals). */
dftfe_status dftfe_profile_enable(dftfe_ham ham, int enable);
/* Total milliseconds and number of timed launches of a kernel family since the
 * last enable.  Synchronises the stream. */
dftfe_status dftfe_profile_query(dftfe_ham ham, const char* kernel, double* total_ms,
                                 int64_t* launches);

/* Test hook for the bounded device waits (no counterpart in the paper).  The dense subspace
 * eigensolver (Rayleigh-Ritz, a cooperative launch whose CTAs meet at a grid barrier after
 * every Jacobi round) gives up a wait after a spin limit of about a second, records
 * DFTFE_ERR_TIMEOUT, lets every CTA return and leaves the context usable; the calling entry
 * point then returns DFTFE_ERR_TIMEOUT with X unchanged.  spin_limit > 0 replaces that limit
 * (iterations of a ~64 ns sleep; 0 restores the default) and withhold_arrival = 1 makes the
 * barrier expect one arrival more than the grid holds, so the first wait runs out for certain
 * (0 restores normal operation).  Both stay in force for later calls on this handle. */
dftfe_status dftfe_ham_set_wait_test(dftfe_ham ham, int64_t spin_limit, int withhold_arrival);

/* Number of kernels this library has launched in this process (all handles). */
int64_t dftfe_launch_count(void);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* dftfe_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DFTFE_GB300_H */
