// Internal declarations shared by the translation units of libdftfe_gb300.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>
#include <map>
#include <stdexcept>
#include <atomic>
#include <functional>

#include "../../include/dftfe_gb300.h"

namespace dftfe {

// ------------------------------------------------------------------ errors
struct Error : std::runtime_error {
  dftfe_status code;
  Error(dftfe_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};
void set_error(const std::string& msg);
void clear_error();
const char* last_error();

#define DFTFE_CHECK_CUDA(call)                                                        \
  do {                                                                                \
    cudaError_t e__ = (call);                                                         \
    if (e__ != cudaSuccess)                                                           \
      throw ::dftfe::Error(e__ == cudaErrorMemoryAllocation ? DFTFE_ERR_OOM : DFTFE_ERR_CUDA, \
                           std::string(#call) + ": " + cudaGetErrorString(e__));      \
  } while (0)

#define DFTFE_REQUIRE(cond, msg)                                     \
  do {                                                               \
    if (!(cond)) throw ::dftfe::Error(DFTFE_ERR_ARG, (msg));         \
  } while (0)

// Every kernel launch goes through this macro: it counts the launch and checks
// the launch status.
extern std::atomic<int64_t> g_launches;
#define DFTFE_LAUNCH(kernel, grid, block, smem, stream, ...)                     \
  do {                                                                           \
    kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                  \
    ::dftfe::g_launches.fetch_add(1, std::memory_order_relaxed);                 \
    DFTFE_CHECK_CUDA(cudaGetLastError());                                        \
  } while (0)

// ---------------------------------------------------------------- basis (host)
struct Rule1D {
  std::vector<double> x, w;
};
Rule1D gll_rule(int p);                         // p+1 GLL points
Rule1D gauss_rule(int n);                       // n Gauss-Legendre points
std::vector<double> barycentric_weights(const std::vector<double>& x);
// T[q*n + j] = l_j(pts[q]) for the Lagrange basis of nodes x (n = x.size()).
std::vector<double> lagrange_at(const std::vector<double>& x, const std::vector<double>& pts);
// D[i*n + j] = l_j'(x_i) at the nodes themselves.
std::vector<double> derivative_matrix(const std::vector<double>& x);

// ------------------------------------------------------------------- handles
}  // namespace dftfe

struct dftfe_mesh_s {
  double L[3];
  int n[3];
  int p, vquad, nq1d;
  int n1;        // p+1
  int nc;        // nodes per cell (p+1)^3
  int nq;        // quadrature points per cell
  int nq1;       // 1D quadrature points
  int64_t g[3];  // nodes per axis
  int64_t M;     // DoFs
  int64_t Nc;    // cells
  double h[3];
  double detJ;
  dftfe::Rule1D gll, quad;
  std::vector<double> D;      // n1 x n1 derivative matrix at GLL nodes
  std::vector<double> Lq;     // nq1 x n1: l_a at the potential quadrature points
  std::vector<double> m1[3];  // 1D lumped mass per axis
};

namespace dftfe {

// A grow-only device buffer.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  void* get(size_t need);
  void release();
};

// One autotuned launch shape of the FP64 cell kernel (rows of a cell per CTA; 0 = the
// built-in heuristic) with its time and the heuristic's for one local part.
struct TunedShape {
  int rows = 0;
  double best_ms = 0.0;
  double heuristic_ms = 0.0;
};

// A launch shape of the TF32x3 cell-product kernel, as the autotuner picks it: the split A
// operand staged in tensor memory (atmem = 1, at most three 128-row M-tiles) or in a
// shared-memory ring (0); with atmem, 6 landing slots for the FP32 plane and 4 stages for the
// gathered X (deep = 0) or 8 and 3 (deep = 1); work items dealt to the persistent CTAs round-robin (deal = 0) or
// in contiguous ranges (1); in a batched launch, the work list system-major (order = 0) or
// interleaved cell by cell across the systems (1, so the k-point items that share one FP32
// plane read each cell's tiles at about the same time).  Every shape computes every cell
// product the same way.  best_ms / default_ms: the timed launch in this shape and in the
// default one (0 when not tuned).
struct MixedShape {
  int atmem = 1, deep = 0, deal = 0, order = 0;
  double best_ms = 0.0, default_ms = 0.0;
};

// A CUDA graph of one enqueued region (graph.cu), re-captured on every call and applied to the
// cached executable by cudaGraphExecUpdate (new bounds change only kernel arguments).
struct GraphSlot {
  cudaGraphExec_t exec = nullptr;
  bool warm = false;      // the region has run once without capture (workspaces allocated)
  int64_t replays = 0;
  int64_t reinstantiations = 0;
};

struct KernelTimer {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
  size_t used = 0;
  double total_ms = 0;
  int64_t launches = 0;
};

}  // namespace dftfe

struct dftfe_ham_s {
  dftfe_mesh mesh = nullptr;
  cudaStream_t stream = nullptr;
  int device = 0;
  int sm_count = 0;
  // a1: mesh data on the device
  int32_t* d_map = nullptr;        // Nc x nc
  double* d_mass = nullptr;        // M
  double* d_minvsqrt = nullptr;    // M
  // colouring (cells grouped by colour; no two cells of one colour share a node)
  int ncolours = 0;
  std::vector<int64_t> colour_off; // ncolours + 1
  int32_t* d_colour_cells = nullptr;
  int32_t* d_node_ptr = nullptr;   // node -> (cell, local row) slots, CSR (built on first mixed use)
  int32_t* d_node_slot = nullptr;
  // a2: cell matrices
  double* d_K = nullptr;           // nc x nc shared stiffness
  double* d_P = nullptr;           // Msym x nq packed basis products (Eq. gemmLoc)
  int32_t* d_pairs = nullptr;      // Msym x 2 (j <= k)
  double* d_wq = nullptr;          // nq quadrature weights * detJ
  double* d_Nq = nullptr;          // nq x nc basis values at the quadrature points
  double* d_Hc = nullptr;          // Nc x nc x nc FP64
  bool has_potential = false;
  int64_t potential_version = 0;   // bumped by every set_potential
  int64_t mixed_version[2] = {-1, -1};  // potential version of the split tiles (bf16, tf32)
  int64_t df_version = -1;              // potential version of the float-pair cell matrices
  int64_t slices_version = -1;          // potential version of the digit rows (exact slices)
  // a3: nonlocal (CSR by projector and by node)
  int nproj = 0;
  double* d_h = nullptr;
  int64_t* d_prow = nullptr;  int32_t* d_pnode = nullptr;  double* d_pval = nullptr;
  int64_t nsup = 0;
  int32_t* d_snode = nullptr; int64_t* d_srow = nullptr;
  int32_t* d_sproj = nullptr; double* d_sval = nullptr;
  int64_t* d_nptr_all = nullptr;   // M + 1 offsets of every node's (sproj, sval) entries
  int64_t nnz = 0;                 // projector CSR entries
  int64_t* d_sperm = nullptr;      // node-major entry t = projector-major entry d_sperm[t]
  // Bloch k-point (complex entry points)
  bool has_kpoint = false;
  bool kpoint_nl = false;          // d_pval_z / d_sval_z hold the current projectors
  double kvec[3] = {0.0, 0.0, 0.0};
  double* d_ktab = nullptr;        // 3 x p x (2p+1): k_d G~1_d stencil per axis (see kpoint.cu)
  double* d_pval_z = nullptr;      // nnz complex, projector-major: M^1/2 chi e^{-ik.d}
  double* d_sval_z = nullptr;      // the same values node-major
  float* d_ktab32 = nullptr;       // FP32 copies for the mixed k-point filter
  float* d_pval_z32 = nullptr;
  float* d_sval_z32 = nullptr;
  // CUDA graphs of the pass's filter phase (dftfe_ham_use_graphs), one slot per shape
  bool use_graphs = false;
  std::map<std::string, dftfe::GraphSlot> graphs;
  cudaStream_t capture_stream = nullptr;   // private stream the regions are captured from
  // autotuner (dftfe_ham_autotune): FP64 cell-kernel shape per real column count
  bool autotune = false;
  std::map<int, dftfe::TunedShape> tuned_fp64;
  bool tuned_mixed_done = false;       // the TF32x3 cell-kernel shape of this mesh (one per ham)
  dftfe::MixedShape tuned_mixed;
  // bounded device waits (dftfe_ham_set_wait_test): spin limit of the eigensolver's grid
  // barrier (0 = the built-in limit of about a second) and arrivals withheld from it (a test
  // makes the wait run out with 1)
  long long wait_limit = 0;
  int wait_missing = 0;
  // a pass run as one CUDA graph (dftfe_ham_use_graphs): the statuses of the Cholesky
  // factorisation [0], the eigensolver [1] and the tensor-core kernels' bounded waits [2] stay
  // on the device (d_pass), the kernels that rotate X or W skip their work once [0] or [1] is
  // set, and the statuses with the Ritz-value ends are copied once, at the end of the pass,
  // to pinned host memory (h_pass: 4 ints, then 2 doubles)
  bool deferred = false;
  int* d_pass = nullptr;
  void* h_pass = nullptr;
  // a ham made by dftfe_ham_create_shared uses the local operator of local_src (its cell
  // matrices and every form derived from them, built on first use into local_src's
  // workspace); `sharers` counts the hams that use this one's
  dftfe_ham_s* local_src = nullptr;
  int sharers = 0;
  // while a batched pass runs this ham's tail: the batch's shared tail workspace, which the
  // tail's buffers (names in ws_get's list) come from instead of `ws`
  std::map<std::string, dftfe::DevBuf>* tail_ws = nullptr;
  // workspace
  std::map<std::string, dftfe::DevBuf> ws;
  // profiling
  bool profiling = false;
  std::map<std::string, dftfe::KernelTimer> timers;
};

namespace dftfe {

void* ws_get(dftfe_ham h, const char* name, size_t bytes);

// the ham that owns h's local operator (h itself unless it was made by
// dftfe_ham_create_shared)
inline dftfe_ham loc(dftfe_ham h) { return h->local_src ? h->local_src : h; }

// the device status words of a deferred pass that a rotation of X or W checks (NULL: none)
inline const int* rot_guard(dftfe_ham h) { return h->deferred ? h->d_pass : nullptr; }
// the timeout flag a tensor-core kernel records into: the pass's in a deferred pass (read
// once at its end), else `own`, which the caller zeroes and reads right away
inline int* tc_err_flag(dftfe_ham h, int* own) { return h->deferred ? h->d_pass + 2 : own; }

// Records an event pair around a kernel-family launch when profiling is on.
struct ProfScope {
  dftfe_ham h;
  KernelTimer* t = nullptr;
  cudaEvent_t e1 = nullptr;
  ProfScope(dftfe_ham h, const char* name);
  ~ProfScope();
};

// ------------------------------------------------------------ device kernels
// hx.cu
void apply_combo(dftfe_ham h, const double* X, int64_t ldx, const double* Xprev, int64_t ldp,
                 double* Z, int64_t ldz, int ncol, double alpha, double s1, double s2);
void chebyshev_filter(dftfe_ham h, double* X, int64_t ld, int ncol, int degree,
                      const dftfe_bounds& b);
void copy_block(cudaStream_t s, const double* src, int64_t lds, double* dst, int64_t ldd,
                int64_t rows, int ncol);
void zero_block(cudaStream_t s, double* dst, int64_t ldd, int64_t rows, int ncol);

// hx_mixed.cu
// ext_err: a device flag the caller zeroes and reads (a bounded wait timed out); NULL makes
// the call zero and read its own (and synchronise)
// kpoint: X is the real view of a complex block (ld, ncol in doubles) at the ham's k-point
void chebyshev_filter_mixed(dftfe_ham h, double* X, int64_t ld, int ncol, int degree,
                            const dftfe_bounds& b, bool tf32, int* ext_err = nullptr, bool kpoint = false);
void apply_mixed(dftfe_ham h, const double* X, int64_t ldx, double* Y, int64_t ldy, int ncol, bool tf32,
                 bool kpoint = false);
// one block of one system in a batched TF32x3 filter round (kpoint: X is the real view of a
// complex block, ncol real columns, at the ham's k-point)
struct MixedBlock {
  dftfe_ham h;
  double* X;
  int64_t ld;
  int ncol, degree;
  dftfe_bounds b;
  bool kpoint;
};
// the batched filter: per round the blocks of every system, with one cell-product launch per
// step, tile and degree group over all systems' cells.  Plans every round (workspaces, host
// descriptors uploaded into desc, staged through host_desc) and returns the closure that
// enqueues all launches on `stream`; err is zeroed and read by the caller.
// tuned: the batch's launch shapes by launch key, filled by timing the first appearance of a
// key (NULL: default shapes, no tuning)
std::function<void()> plan_mixed_batch(const std::vector<std::vector<MixedBlock>>& rounds, cudaStream_t stream,
                                       int* err, DevBuf& desc, std::vector<uint8_t>& host_desc,
                                       std::map<std::string, MixedShape>* tuned = nullptr);
// with_nl = false: the local part only (real view of a complex block)
void apply_df(dftfe_ham h, const double* X, int64_t ldx, double* Y, int64_t ldy, int ncol, bool with_nl = true);
// hx_slices.cu: Y = H~X from exact bf16 digit products on the tensor cores (FP64-accurate;
// false when the mesh degree is beyond what the exact accumulation allows), and the W = H~X
// of the mixed Rayleigh-Ritz step (those products where they apply, else float pairs)
bool slices_applicable(dftfe_ham h);
bool apply_slices(dftfe_ham h, const double* X, int64_t ldx, double* Y, int64_t ldy, int ncol, bool with_nl = true);
void apply_w(dftfe_ham h, const double* X, int64_t ldx, double* Y, int64_t ldy, int ncol, bool with_nl = true);
// kpoint.cu: Z += alpha (-i k.grad X + H~_nl^k X) on FP32 complex blocks given by their real
// views (ld in floats, ncolz complex columns); 1/2|k|^2 is the caller's
void kpoint_add32(dftfe_ham h, const float* X, int64_t ldx, float* Z, int64_t ldz, int ncolz, float alpha);
// hx.cu: Y = H~_nl X (Y overwritten; zero when there are no projectors), FP64
void apply_nonlocal_fp64(dftfe_ham h, const double* X, int64_t ldx, double* Y, int64_t ldy, int ncol);

// dense_mixed.cu (FP64 diagonal, FP32 off-diagonal)
void gram_lower_mixed(dftfe_ham h, const double* A, int64_t lda, const double* B, int64_t ldb, int64_t M, int N,
                      double* C);
void rotate_inplace_mixed(dftfe_ham h, double* X, int64_t ld, int64_t M, int N, const double* Z, bool upper);
// X <- X Z with the offdiagonal of Z as FP32-equivalent tensor-core products and its
// diagonal in FP64; false when not applicable
bool rotate_inplace_tc(dftfe_ham h, double* X, int64_t ld, int64_t M, int N, const double* Z, bool upper);
// the pass after its filter: CholGS, Rayleigh-Ritz, residuals, bounds update
void chfsi_pass_tail(dftfe_ham h, double* X, int64_t ld, int ncol, dftfe_bounds* inout, double* evals,
                     double* resid, dftfe_precision prec);
// Z += alpha H~_nl X in FP64 (no-op without projectors)
void nonlocal_add_fp64(dftfe_ham h, const double* X, int64_t ldx, double* Z, int64_t ldz, int ncol, double alpha);
// row splits of a cell for the FP64 wide cell kernel given the CTAs of one launch
int fp64_row_splits(dftfe_ham h, int64_t ctas, int nc);
// C = A^T B (both triangles) with FP32-equivalent tensor-core off-diagonal entries and the
// FP64 diagonal from column-dot partials dpart[nchunk][N]; false when not applicable
bool gram_lower_tc(dftfe_ham h, const double* A, int64_t lda, const double* B, int64_t ldb, int64_t M, int N,
                   double* C, const double* dpart, int nchunk);

// dense.cu
void gram_lower(dftfe_ham h, const double* A, int64_t lda, const double* B, int64_t ldb,
                int64_t M, int N, double* C, double* part, int nsplit);
int gram_nsplit(dftfe_ham h, int64_t M, int N);
void potrf(cudaStream_t s, double* A, int N, int* d_status);
void trtri_lower_to_upper_t(cudaStream_t s, const double* L, double* Z, int N);
// chol.cu: blocked multi-CTA forms of the two above (the lower triangle of A is factored in
// place, its strict upper triangle zeroed; d_status cleared, then DFTFE_ERR_NOT_SPD on a bad
// pivot; Z = L^-T upper triangular)
void cholesky_blocked(dftfe_ham h, double* A, int N, int* d_status);
void tri_inverse_blocked(dftfe_ham h, double* L, double* Z, int N);
void rotate_inplace(dftfe_ham h, double* X, int64_t ld, int64_t M, int N, const double* Z,
                    bool upper);
void syevd(dftfe_ham h, double* A, int N, double* evals, double* Q, int* d_status);
void tridiag_ql(cudaStream_t s, double* d, double* e, double* Z, int N, int* d_status);
// cw = 2: complex columns (interleaved real and imaginary parts, ld in doubles), one
// residual per complex column
void residual_norms(dftfe_ham h, const double* X, int64_t ldx, const double* W, int64_t ldw,
                    int64_t M, int ncol, const double* evals, double* resid, int kind, int cw = 1);
void random_uniform(cudaStream_t s, double* out, int64_t n, uint64_t seed, int64_t offset);
// cplx: Lanczos on the real 2M x 2M form of H~^k (vectors are the real views of complex ones)
void lanczos(dftfe_ham h, int k, const double* v0, uint64_t seed, double* out3, bool cplx = false);
// Hermitian A (N x N complex interleaved, lower triangle read) = Q Theta Q^H; Q row-major
// complex, columns ascending, each column's largest-|.| entry made real and positive
void syevd_z(dftfe_ham h, double* A, int N, double* evals, double* Q, int* d_status);

// hx.cu: Z += alpha H~_loc X over all colours (FP64 cell products), ncol real columns
void local_part_fp64(dftfe_ham h, const double* X, int64_t ldx, double* Z, int64_t ldz, int ncol, double alpha);

// graph.cu: run `enqueue` (work on h->stream only, no host synchronisation, no allocation
// once it has run with the same key) directly, or through the CUDA graph slot `key` when the
// ham uses graphs: the first call with a key runs directly, later ones capture and replay.
void run_region(dftfe_ham h, const std::string& key, const std::function<void()>& enqueue);
void free_graphs(dftfe_ham h);
// capture `enqueue` from stream `cap` (the variables in `streams`, all equal to `own`, point at
// it meanwhile; the flags in `prof` are cleared), update or instantiate slot.exec, launch on own
void capture_and_launch(GraphSlot& slot, cudaStream_t own, cudaStream_t cap, const std::vector<cudaStream_t*>& streams,
                        const std::vector<bool*>& prof, const std::function<void()>& enqueue);

// kpoint.cu: Z = alpha H~^k X + s1 X + s2 Xp on complex blocks (ld in complex elements)
void apply_combo_z(dftfe_ham h, const double* X, int64_t ldx, const double* Xp, int64_t ldp, double* Z,
                   int64_t ldz, int ncol, double alpha, double s1, double s2);
// the part of apply_combo_z before the cell products: Z = s1 X + s2 Xp + alpha (1/2|k|^2 X
// - i k.grad X + H~_nl^k X)
void kpoint_init_terms(dftfe_ham h, const double* X, int64_t ldx, const double* Xp, int64_t ldp, double* Z,
                       int64_t ldz, int ncol, double alpha, double s1, double s2);
void chebyshev_filter_z_fp64(dftfe_ham h, double* X, int64_t ld, int ncol, int degree, const dftfe_bounds& b);
void chfsi_pass_tail_z(dftfe_ham h, double* X, int64_t ld, int ncol, dftfe_bounds* inout, double* evals,
                       double* resid, dftfe_precision prec);
// DFTFE_ERR_STATE unless the potential and the k-point (with current projector phases) are set
void require_kpoint(dftfe_ham h);

}  // namespace dftfe

// Wraps the body of every extern "C" entry point: exceptions become status codes.
#define ABI_BEGIN \
  try {         \
    ::dftfe::clear_error();
#define ABI_END                                     \
  return DFTFE_OK;                                  \
  }                                                 \
  catch (const ::dftfe::Error& e) {                 \
    ::dftfe::set_error(e.what());                   \
    return e.code;                                  \
  }                                                 \
  catch (const std::bad_alloc&) {                   \
    ::dftfe::set_error("host allocation failed");   \
    return DFTFE_ERR_OOM;                           \
  }                                                 \
  catch (const std::exception& e) {                 \
    ::dftfe::set_error(e.what());                   \
    return DFTFE_ERR_CUDA;                          \
  }
