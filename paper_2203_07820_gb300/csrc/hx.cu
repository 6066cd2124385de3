// H~ X application (a4, a5) and the Chebyshev filter (a6).
//
// Local part (Sec. 4.3, Eq. celldgemm): Y = ASEMB_FEM{ H~^c X^c }.  One CTA takes one
// cell and up to 32 columns: it gathers the cell's rows of X into shared memory
// (each row is a contiguous run of columns, so the gather is coalesced, as in the
// paper's DoF-major layout), multiplies by the dense cell matrix and adds the result
// straight into the global output.  Cells are processed colour by colour (no two
// cells of one colour share a node), so the scatter-add needs no atomics and is
// deterministic.
// Nonlocal part (Alg. 4): P = C~^T X as a segmented reduction over each projector's
// support, P <- h P, then Y += C~ P as a gather over each support node's projectors.
// The recurrence (Eq. chebyfilter) is fused: the output is initialised to
// s1 X_k + s2 X_{k-1} and the local and nonlocal parts accumulate alpha H~ X_k on top.
#include "internal.h"
#include "cell_fp64.cuh"

#include <cmath>

namespace dftfe {

static unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Z = s1 X + s2 Xp (Xp may be null; s1 == 0 and Xp == null writes zeros).
__global__ void k_axpby_init(double* __restrict__ Z, int64_t ldz, const double* __restrict__ X,
                             int64_t ldx, const double* __restrict__ Xp, int64_t ldp,
                             int64_t M, int ncol, double s1, double s2) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t n = M * ncol;
  if (t >= n) return;
  int64_t i = t / ncol;
  int j = (int)(t - i * ncol);
  double v = 0.0;
  if (s1 != 0.0) v = s1 * X[i * ldx + j];
  if (Xp) v += s2 * Xp[i * ldp + j];
  Z[i * ldz + j] = v;
}

__global__ void k_copy_block(const double* __restrict__ src, int64_t lds, double* __restrict__ dst,
                             int64_t ldd, int64_t rows, int ncol) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= rows * ncol) return;
  int64_t i = t / ncol;
  int j = (int)(t - i * ncol);
  dst[i * ldd + j] = src[i * lds + j];
}

// P[a][col] = h_a * sum_{e in supp a} C~[e] X[node_e][col]; one CTA per (projector, 32 cols).
__global__ void __launch_bounds__(256) k_nl_coef(const double* __restrict__ X, int64_t ldx, int ncol,
                                                 const int64_t* __restrict__ prow,
                                                 const int32_t* __restrict__ pnode,
                                                 const double* __restrict__ pval,
                                                 const double* __restrict__ hcoup, double* __restrict__ P) {
  __shared__ double red[8][32];
  const int a = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.y * 32 + lane;
  double s = 0.0;
  if (col < ncol)
    for (int64_t e = prow[a] + warp; e < prow[a + 1]; e += 8)
      s = fma(pval[e], X[(int64_t)pnode[e] * ldx + col], s);
  red[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && col < ncol) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w][lane];
    P[(int64_t)a * ncol + col] = hcoup[a] * t;
  }
}

// Z[node][col] += alpha * sum_{t in node's projectors} C~[t] P[proj_t][col]; one warp per node.
__global__ void __launch_bounds__(256) k_nl_add(double* __restrict__ Z, int64_t ldz, int ncol,
                                                const int32_t* __restrict__ snode,
                                                const int64_t* __restrict__ srow,
                                                const int32_t* __restrict__ sproj,
                                                const double* __restrict__ sval,
                                                const double* __restrict__ P, int64_t nsup, double alpha) {
  const int lane = threadIdx.x & 31;
  const int64_t s = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int col = blockIdx.y * 32 + lane;
  if (s >= nsup || col >= ncol) return;
  double acc = 0.0;
  for (int64_t t = srow[s]; t < srow[s + 1]; ++t) acc = fma(sval[t], P[(int64_t)sproj[t] * ncol + col], acc);
  Z[(int64_t)snode[s] * ldz + col] += alpha * acc;
}

// Local part, wide form: one CTA = one cell x 32 columns (the body is shared with the batched
// kernel, see cell_fp64.cuh).
__global__ void __launch_bounds__(256, 2) k_cell_fp64_wide(
    const double* __restrict__ Hc, const int32_t* __restrict__ map,
    const int32_t* __restrict__ cells, int nc, const double* __restrict__ X, int64_t ldx,
    double* __restrict__ Z, int64_t ldz, int ncol, double alpha, int rows_per_split) {
  extern __shared__ double smem[];
  // blockIdx.z: a range of rows_per_split rows of the cell (a multiple of 64)
  const int rbeg = (int)blockIdx.z * rows_per_split;
  cell_fp64_wide_body(Hc, map, cells[blockIdx.x], nc, X, ldx, Z, ldz, ncol, alpha, (int)blockIdx.y, rbeg,
                      min(nc, rbeg + rows_per_split), smem);
}

// Local part, narrow form (ncol <= 4): one CTA = one cell; each warp reduces whole rows
// of H~^c against the gathered columns (lanes split the k index, shuffle reduction).
template <int NC>
__global__ void __launch_bounds__(256) k_cell_fp64_narrow(
    const double* __restrict__ Hc, const int32_t* __restrict__ map,
    const int32_t* __restrict__ cells, int nc, const double* __restrict__ X, int64_t ldx,
    double* __restrict__ Z, int64_t ldz, int ncol, double alpha) {
  extern __shared__ double smem[];
  double* xs = smem;                          // nc x NC
  int32_t* sm = (int32_t*)(smem + nc * NC);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t cell = cells[blockIdx.x];
  const int32_t* m = map + cell * nc;
  for (int k = threadIdx.x; k < nc; k += 256) sm[k] = m[k];
  __syncthreads();
  for (int t = threadIdx.x; t < nc * NC; t += 256) {
    int k = t / NC, c = t % NC;
    xs[t] = c < ncol ? X[(int64_t)sm[k] * ldx + c] : 0.0;
  }
  __syncthreads();
  const double* H = Hc + cell * (int64_t)nc * nc;
  for (int r = warp; r < nc; r += 8) {
    double acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.0;
    const double* Hr = H + (int64_t)r * nc;
    for (int k = lane; k < nc; k += 32) {
      const double hv = __ldg(Hr + k);
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = fma(hv, xs[k * NC + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], off);
    if (lane == 0) {
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if (c < ncol) Z[(int64_t)sm[r] * ldz + c] += alpha * acc[c];
    }
  }
}

void copy_block(cudaStream_t s, const double* src, int64_t lds, double* dst, int64_t ldd,
                int64_t rows, int ncol) {
  if (rows * ncol == 0) return;
  DFTFE_LAUNCH(k_copy_block, nblk(rows * ncol), 256, 0, s, src, lds, dst, ldd, rows, ncol);
}

void zero_block(cudaStream_t s, double* dst, int64_t ldd, int64_t rows, int ncol) {
  if (rows * ncol == 0) return;
  DFTFE_LAUNCH(k_axpby_init, nblk(rows * ncol), 256, 0, s, dst, ldd, nullptr, 0, nullptr, 0, rows, ncol, 0.0, 0.0);
}

static bool g_attr_set = false;
static void set_smem_attrs() {
  if (g_attr_set) return;
  const int big = 200 * 1024;
  DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_cell_fp64_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_cell_fp64_narrow<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_cell_fp64_narrow<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  g_attr_set = true;
}

// Row splits of a cell for the FP64 wide kernel: enough CTAs for two per SM when a colour
// holds few cells (the FP64 pipe of one SM needs long to finish a whole cell), at most one
// split per 64 rows.
int fp64_row_splits(dftfe_ham h, int64_t ctas, int nc) {
  const int64_t want = (2LL * h->sm_count + ctas - 1) / std::max<int64_t>(ctas, 1);
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (nc + 63) / 64));
}

// rows_per_cta > 0 forces that many rows of a cell per CTA (a multiple of 64) in every colour;
// 0 takes fp64_row_splits per colour.  Every choice gives the same bits (cell_fp64.cuh).
static void local_part_rows(dftfe_ham h, const double* X, int64_t ldx, double* Z, int64_t ldz, int ncol,
                            double alpha, int rows_per_cta) {
  auto* m = h->mesh;
  set_smem_attrs();
  const int nc = m->nc;
  for (int c = 0; c < h->ncolours; ++c) {
    const int64_t n = h->colour_off[c + 1] - h->colour_off[c];
    if (n == 0) continue;
    const int32_t* cells = h->d_colour_cells + h->colour_off[c];
    ProfScope ps(h, "cell_gemm_fp64");
    if (ncol <= 1) {
      size_t sh = (size_t)nc * 1 * sizeof(double) + nc * sizeof(int32_t);
      DFTFE_LAUNCH(k_cell_fp64_narrow<1>, (unsigned)n, 256, sh, h->stream, loc(h)->d_Hc, h->d_map, cells,
                   nc, X, ldx, Z, ldz, ncol, alpha);
    } else if (ncol <= 4) {
      size_t sh = (size_t)nc * 4 * sizeof(double) + nc * sizeof(int32_t);
      DFTFE_LAUNCH(k_cell_fp64_narrow<4>, (unsigned)n, 256, sh, h->stream, loc(h)->d_Hc, h->d_map, cells,
                   nc, X, ldx, Z, ldz, ncol, alpha);
    } else {
      size_t sh = (size_t)nc * 32 * sizeof(double) + nc * sizeof(int32_t);
      const int tiles = (ncol + 31) / 32;
      const int splits = fp64_row_splits(h, n * tiles, nc);
      const int rows = rows_per_cta > 0 ? rows_per_cta : ((nc + splits - 1) / splits + 63) / 64 * 64;
      dim3 grid((unsigned)n, (unsigned)tiles, (unsigned)((nc + rows - 1) / rows));
      DFTFE_LAUNCH(k_cell_fp64_wide, grid, 256, sh, h->stream, loc(h)->d_Hc, h->d_map, cells, nc, X, ldx, Z,
                   ldz, ncol, alpha, rows);
    }
  }
}

// Autotuner (no counterpart in the paper, whose cell GEMMs go to a vendor batched GEMM): the
// first local part of a given column count times every rows-per-CTA shape of the wide
// kernel (64, 128, ... rows of a cell per CTA, and the heuristic) on the caller's X into a
// scratch output, twice each (the first run warms up), and keeps the fastest for the ham.
static int tuned_rows(dftfe_ham h, const double* X, int64_t ldx, int ncol) {
  auto it = h->tuned_fp64.find(ncol);
  if (it != h->tuned_fp64.end()) return it->second.rows;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  DFTFE_CHECK_CUDA(cudaStreamIsCapturing(h->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) return 0;   // no timing inside a graph capture
  auto* m = h->mesh;
  double* Zs = (double*)ws_get(h, "tune_z", sizeof(double) * (size_t)m->M * ncol);
  DFTFE_CHECK_CUDA(cudaMemsetAsync(Zs, 0, sizeof(double) * (size_t)m->M * ncol, h->stream));
  struct Ev {
    cudaEvent_t e[2] = {nullptr, nullptr};
    ~Ev() { for (auto x : e) if (x) cudaEventDestroy(x); }
  } ev;
  for (auto& x : ev.e) DFTFE_CHECK_CUDA(cudaEventCreate(&x));
  const bool prof = h->profiling;
  h->profiling = false;
  TunedShape best;
  best.best_ms = 1e300;
  try {
    for (int r = 0; r <= (m->nc + 63) / 64 * 64; r += 64) {
      local_part_rows(h, X, ldx, Zs, ncol, ncol, 1.0, r);
      DFTFE_CHECK_CUDA(cudaEventRecord(ev.e[0], h->stream));
      local_part_rows(h, X, ldx, Zs, ncol, ncol, 1.0, r);
      DFTFE_CHECK_CUDA(cudaEventRecord(ev.e[1], h->stream));
      DFTFE_CHECK_CUDA(cudaEventSynchronize(ev.e[1]));
      float ms = 0.f;
      DFTFE_CHECK_CUDA(cudaEventElapsedTime(&ms, ev.e[0], ev.e[1]));
      if (r == 0) best.heuristic_ms = ms;
      if (ms < best.best_ms) {
        best.best_ms = ms;
        best.rows = r;
      }
    }
  } catch (...) {
    h->profiling = prof;
    throw;
  }
  h->profiling = prof;
  h->tuned_fp64[ncol] = best;
  return best.rows;
}

void local_part_fp64(dftfe_ham h, const double* X, int64_t ldx, double* Z, int64_t ldz, int ncol,
                     double alpha) {
  const int rows = h->autotune && ncol > 4 ? tuned_rows(h, X, ldx, ncol) : 0;
  local_part_rows(h, X, ldx, Z, ldz, ncol, alpha, rows);
}

// Z += alpha H~_nl X (FP64), nothing without projectors
void nonlocal_add_fp64(dftfe_ham h, const double* X, int64_t ldx, double* Z, int64_t ldz, int ncol, double alpha) {
  if (h->nproj <= 0) return;
  double* P = (double*)ws_get(h, "nl_coef", sizeof(double) * h->nproj * (size_t)ncol);
  dim3 g1((unsigned)h->nproj, (unsigned)((ncol + 31) / 32));
  DFTFE_LAUNCH(k_nl_coef, g1, 256, 0, h->stream, X, ldx, ncol, h->d_prow, h->d_pnode, h->d_pval, h->d_h, P);
  dim3 g2((unsigned)((h->nsup + 7) / 8), (unsigned)((ncol + 31) / 32));
  DFTFE_LAUNCH(k_nl_add, g2, 256, 0, h->stream, Z, ldz, ncol, h->d_snode, h->d_srow, h->d_sproj, h->d_sval, P,
               h->nsup, alpha);
}

void apply_combo(dftfe_ham h, const double* X, int64_t ldx, const double* Xprev, int64_t ldp,
                 double* Z, int64_t ldz, int ncol, double alpha, double s1, double s2) {
  if (!loc(h)->has_potential) throw Error(DFTFE_ERR_STATE, "set the potential before applying H");
  auto* m = h->mesh;
  if (ncol <= 0) return;
  set_smem_attrs();
  DFTFE_LAUNCH(k_axpby_init, nblk(m->M * ncol), 256, 0, h->stream, Z, ldz, X, ldx, Xprev, ldp, m->M,
               ncol, s1, s2);
  nonlocal_add_fp64(h, X, ldx, Z, ldz, ncol, alpha);
  local_part_fp64(h, X, ldx, Z, ldz, ncol, alpha);
}

void apply_nonlocal_fp64(dftfe_ham h, const double* X, int64_t ldx, double* Y, int64_t ldy, int ncol) {
  auto* m = h->mesh;
  DFTFE_LAUNCH(k_axpby_init, nblk(m->M * ncol), 256, 0, h->stream, Y, ldy, X, ldx, nullptr, 0, m->M, ncol, 0.0,
               0.0);
  if (h->nproj > 0) {
    double* P = (double*)ws_get(h, "nl_coef", sizeof(double) * h->nproj * (size_t)ncol);
    dim3 g1((unsigned)h->nproj, (unsigned)((ncol + 31) / 32));
    DFTFE_LAUNCH(k_nl_coef, g1, 256, 0, h->stream, X, ldx, ncol, h->d_prow, h->d_pnode, h->d_pval, h->d_h, P);
    dim3 g2((unsigned)((h->nsup + 7) / 8), (unsigned)((ncol + 31) / 32));
    DFTFE_LAUNCH(k_nl_add, g2, 256, 0, h->stream, Y, ldy, ncol, h->d_snode, h->d_srow, h->d_sproj, h->d_sval, P,
                 h->nsup, 1.0);
  }
}

// Eq. chebyfilter.  Unscaled: X1 = (H~ - c) X0 / e, X_{k+1} = 2 (H~ - c) X_k / e - X_{k-1}.
// Scaled (Zhou-Saad): sigma1 = e / (a0 - c), X1 = sigma1 (H~ - c) X0 / e,
// sigma_{k+1} = 1 / (2/sigma1 - sigma_k), X_{k+1} = 2 sigma_{k+1} (H~ - c) X_k / e
// - sigma_k sigma_{k+1} X_{k-1}.  Three buffers rotate: the caller's X and two workspaces.
void chebyshev_filter(dftfe_ham h, double* X, int64_t ld, int ncol, int degree, const dftfe_bounds& b) {
  if (degree <= 0 || ncol <= 0) return;
  auto* m = h->mesh;
  const double e = (b.b - b.a) / 2.0, c = (b.b + b.a) / 2.0;
  const bool scaled = !std::isnan(b.a0);
  double* w1 = (double*)ws_get(h, "cheb_w1", sizeof(double) * m->M * (size_t)ncol);
  double* w2 = (double*)ws_get(h, "cheb_w2", sizeof(double) * m->M * (size_t)ncol);
  double* buf[3] = {X, w1, w2};
  int64_t lds[3] = {ld, ncol, ncol};
  int cur = 0, prev = -1;
  double sigma = scaled ? e / (b.a0 - c) : 0.0;
  const double sigma1 = sigma, gamma = scaled ? 2.0 / sigma1 : 0.0;
  for (int k = 1; k <= degree; ++k) {
    int out = 0;
    while (out == cur || out == prev) ++out;
    double alpha, s1, s2 = 0.0;
    if (k == 1) {
      alpha = scaled ? sigma1 / e : 1.0 / e;
      s1 = -c * alpha;
    } else if (scaled) {
      const double sigma2 = 1.0 / (gamma - sigma);
      alpha = 2.0 * sigma2 / e;
      s1 = -c * alpha;
      s2 = -sigma * sigma2;
      sigma = sigma2;
    } else {
      alpha = 2.0 / e;
      s1 = -c * alpha;
      s2 = -1.0;
    }
    apply_combo(h, buf[cur], lds[cur], prev >= 0 ? buf[prev] : nullptr, prev >= 0 ? lds[prev] : 0,
                buf[out], lds[out], ncol, alpha, s1, s2);
    prev = cur;
    cur = out;
  }
  if (cur != 0) copy_block(h->stream, buf[cur], lds[cur], X, ld, m->M, ncol);
}

}  // namespace dftfe

using namespace dftfe;

extern "C" dftfe_status dftfe_ham_apply(dftfe_ham h, const double* X, int64_t ldx, double* Y,
                                        int64_t ldy, int ncol, dftfe_precision prec) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && X && Y, "null argument");
  DFTFE_REQUIRE(ncol >= 0 && ldx >= ncol && ldy >= ncol, "bad ncol / leading dimension");
  DFTFE_REQUIRE(prec == DFTFE_FP64 || prec == DFTFE_MIXED_BF16X3 || prec == DFTFE_MIXED_TF32X3 ||
                    prec == DFTFE_FP64_FLOAT_PAIRS || prec == DFTFE_FP64_SLICES,
                "unknown precision");
  if (!loc(h)->has_potential) throw Error(DFTFE_ERR_STATE, "set the potential first");
  if (prec == DFTFE_FP64_SLICES && !slices_applicable(h))
    throw Error(DFTFE_ERR_ARG, "exact-slice products need at most 682 nodes per cell (degree <= 7)");
  if (prec == DFTFE_FP64) apply_combo(h, X, ldx, nullptr, 0, Y, ldy, ncol, 1.0, 0.0, 0.0);
  else if (prec == DFTFE_FP64_FLOAT_PAIRS) apply_df(h, X, ldx, Y, ldy, ncol);
  else if (prec == DFTFE_FP64_SLICES) apply_slices(h, X, ldx, Y, ldy, ncol);
  else apply_mixed(h, X, ldx, Y, ldy, ncol, prec == DFTFE_MIXED_TF32X3);
  ABI_END
}

extern "C" dftfe_status dftfe_ham_autotune(dftfe_ham h, int enable) {
  ABI_BEGIN
  DFTFE_REQUIRE(h, "null ham");
  DFTFE_REQUIRE(enable == 0 || enable == 1, "enable must be 0 or 1");
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  h->autotune = enable == 1;
  h->tuned_fp64.clear();
  h->tuned_mixed_done = false;
  h->tuned_mixed = MixedShape{};
  // cached graphs hold the old launch shapes: the next pass of each runs directly again
  for (auto& kv : h->graphs) kv.second.warm = false;
  ABI_END
}

extern "C" dftfe_status dftfe_autotune_query(dftfe_ham h, int ncol, int* rows_per_cta, double* best_ms,
                                             double* heuristic_ms) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && rows_per_cta, "null argument");
  auto it = h->tuned_fp64.find(ncol);
  if (it == h->tuned_fp64.end()) {
    *rows_per_cta = -1;
    if (best_ms) *best_ms = 0.0;
    if (heuristic_ms) *heuristic_ms = 0.0;
  } else {
    *rows_per_cta = it->second.rows;
    if (best_ms) *best_ms = it->second.best_ms;
    if (heuristic_ms) *heuristic_ms = it->second.heuristic_ms;
  }
  ABI_END
}

extern "C" dftfe_status dftfe_chebyshev_filter(dftfe_ham h, double* X, int64_t ld, int ncol, int degree,
                                               const dftfe_bounds* bounds, dftfe_precision prec) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && X && bounds, "null argument");
  DFTFE_REQUIRE(ncol >= 0 && ld >= ncol && degree >= 0, "bad ncol / ld / degree");
  DFTFE_REQUIRE(bounds->b > bounds->a, "need b > a");
  DFTFE_REQUIRE(std::isnan(bounds->a0) || bounds->a0 < bounds->a, "need a0 < a for the scaled filter");
  DFTFE_REQUIRE(prec == DFTFE_FP64 || prec == DFTFE_MIXED_BF16X3 || prec == DFTFE_MIXED_TF32X3,
                "unknown precision");
  if (!loc(h)->has_potential) throw Error(DFTFE_ERR_STATE, "set the potential first");
  if (prec == DFTFE_FP64) chebyshev_filter(h, X, ld, ncol, degree, *bounds);
  else chebyshev_filter_mixed(h, X, ld, ncol, degree, *bounds, prec == DFTFE_MIXED_TF32X3);
  ABI_END
}

extern "C" dftfe_status dftfe_autotune_query_mixed(dftfe_ham h, int* atmem, int* deep, int* deal, double* best_ms,
                                                   double* default_ms) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && atmem && deep && deal, "null argument");
  const bool done = h->tuned_mixed_done;
  *atmem = done ? h->tuned_mixed.atmem : -1;
  *deep = done ? h->tuned_mixed.deep : -1;
  *deal = done ? h->tuned_mixed.deal : -1;
  if (best_ms) *best_ms = done ? h->tuned_mixed.best_ms : 0.0;
  if (default_ms) *default_ms = done ? h->tuned_mixed.default_ms : 0.0;
  ABI_END
}
