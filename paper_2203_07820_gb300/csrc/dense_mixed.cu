// Mixed-precision overlap, projection and subspace rotations (Sec. 3.2 and Sec. 4.4):
// as the filtered vectors approach eigenvectors, S = X^T X and H^ = X^T H~ X approach
// diagonal matrices and the rotation matrices approach diagonal ones, so the diagonal
// entries are formed in FP64 and the off-diagonal ones in FP32:
//   S, H^ : diagonal FP64 dot products, off-diagonal FP32 GEMM (per-split FP32
//           accumulation, FP64 sum over splits);
//   X <- X Z : X diag(Z) in FP64 plus X offdiag(Z) in FP32
//           (the paper's Psi_o = SP[Psi L^-T_od] + DP[Psi L^-T_d], applied to L^-T and to Q).
// The Cholesky factorisation, the dense eigensolver and H~X stay FP64.
#include "internal.h"

#include <cmath>
#include <vector>

namespace dftfe {

static unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------- FP32 Gram
constexpr int G32T = 128, G32K = 16;
// part[s][i][j] = sum over split s of A[m][i] B[m][j] (FP32 products and sums, stored FP64)
__global__ void __launch_bounds__(256, 1) k_gram32_partial(const double* __restrict__ A, int64_t lda,
                                                        const double* __restrict__ B, int64_t ldb, int64_t M,
                                                        int N, int64_t rows_per_split,
                                                        double* __restrict__ part) {
  __shared__ __align__(16) float As[G32K][G32T];
  __shared__ __align__(16) float Bs[G32K][G32T];
  // tile (ti, tj) of the lower triangle, row-major: blockIdx.x = ti (ti + 1) / 2 + tj
  const int t = blockIdx.x;
  int ti = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while (ti * (ti + 1) / 2 > t) --ti;
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  const int tj = t - ti * (ti + 1) / 2;
  const int i0 = ti * G32T, j0 = tj * G32T;
  const int64_t m0 = (int64_t)blockIdx.y * rows_per_split;
  const int64_t m1 = min(M, m0 + rows_per_split);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  for (int64_t mm = m0; mm < m1; mm += G32K) {
    for (int e = threadIdx.x; e < G32K * G32T; e += 256) {
      const int kk = e / G32T, c = e % G32T;
      const int64_t row = mm + kk;
      const bool rok = row < m1;
      As[kk][c] = (rok && i0 + c < N) ? (float)A[row * lda + i0 + c] : 0.0f;
      Bs[kk][c] = (rok && j0 + c < N) ? (float)B[row * ldb + j0 + c] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < G32K; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * 8 + 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8 + 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double* out = part + (int64_t)blockIdx.y * N * N;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gi = i0 + ty * 8 + i;
    if (gi >= N) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gj = j0 + tx * 8 + j;
      if (gj < N) out[(int64_t)gi * N + gj] = (double)acc[i][j];
    }
  }
}

// FP64 column dots d[j] = sum_m A[m][j] B[m][j], split over rows (partials per chunk)
__global__ void k_coldot_partial(const double* __restrict__ A, int64_t lda, const double* __restrict__ B,
                                 int64_t ldb, int64_t M, int N, int64_t rows, double* __restrict__ part) {
  const int64_t i0 = (int64_t)blockIdx.x * rows, i1 = min(M, i0 + rows);
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    double s = 0.0;
    for (int64_t i = i0; i < i1; ++i) s = fma(A[i * lda + j], B[i * ldb + j], s);
    part[(int64_t)blockIdx.x * N + j] = s;
  }
}

// C[i][j] = C[j][i] = sum_s part[s][i][j] (i > j, fixed order); C[i][i] = sum_c dpart[c][i]
__global__ void k_gram32_reduce(const double* __restrict__ part, int nsplit, const double* __restrict__ dpart,
                                int nchunk, int N, double* __restrict__ C) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * N) return;
  const int i = (int)(t / N), j = (int)(t % N);
  if (i < j) return;
  double s = 0.0;
  if (i == j)
    for (int c = 0; c < nchunk; ++c) s += dpart[(int64_t)c * N + i];
  else
    for (int k = 0; k < nsplit; ++k) s += part[(int64_t)k * N * N + t];
  C[(int64_t)i * N + j] = s;
  C[(int64_t)j * N + i] = s;
}

void gram_lower_mixed(dftfe_ham h, const double* A, int64_t lda, const double* B, int64_t ldb, int64_t M, int N,
                      double* C) {
  {
    // tensor cores (TF32x3 off-diagonal) with the FP64 column dots for the diagonal
    const int nchunk = (int)std::max<int64_t>(1, std::min<int64_t>(h->sm_count * 4, M / 64));
    const int64_t drows = (M + nchunk - 1) / nchunk;
    double* dpart = (double*)ws_get(h, "coldot_part", sizeof(double) * (size_t)nchunk * N);
    if (M >= 1) {
      {
        ProfScope ps(h, "coldot");
        DFTFE_LAUNCH(k_coldot_partial, nchunk, 256, 0, h->stream, A, lda, B, ldb, M, N, drows, dpart);
      }
      if (gram_lower_tc(h, A, lda, B, ldb, M, N, C, dpart, nchunk)) return;
    }
  }
  const int T = (N + G32T - 1) / G32T;
  const int ntiles = T * (T + 1) / 2;
  const int64_t want = (4LL * h->sm_count + ntiles - 1) / ntiles;
  const int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(want, M / 512));
  const int64_t rows = (M + nsplit - 1) / nsplit;
  double* part = (double*)ws_get(h, "gram32_part", sizeof(double) * (size_t)nsplit * N * N);
  const int nchunk = (int)std::max<int64_t>(1, std::min<int64_t>(h->sm_count * 4, M / 64));
  const int64_t drows = (M + nchunk - 1) / nchunk;
  double* dpart = (double*)ws_get(h, "coldot_part", sizeof(double) * (size_t)nchunk * N);
  {
    ProfScope ps(h, "gram_mixed");
    DFTFE_LAUNCH(k_gram32_partial, dim3(ntiles, nsplit), 256, 0, h->stream, A, lda, B, ldb, M, N, rows, part);
    DFTFE_LAUNCH(k_coldot_partial, nchunk, 256, 0, h->stream, A, lda, B, ldb, M, N, drows, dpart);
  }
  DFTFE_LAUNCH(k_gram32_reduce, nblk((int64_t)N * N), 256, 0, h->stream, part, nsplit, dpart, nchunk, N, C);
}

// --------------------------------------------------------- mixed rotation
// Zf = FP32 off-diagonal of Z (zero diagonal), zd = FP64 diagonal of Z
__global__ void k_split_rot(const double* __restrict__ Z, int N, float* __restrict__ Zf, double* __restrict__ zd) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * N) return;
  const int i = (int)(t / N), j = (int)(t % N);
  Zf[t] = (i == j) ? 0.0f : (float)Z[t];
  if (i == j) zd[i] = Z[t];
}

// X[r0:r0+R, :] <- X diag(zd) (FP64) + X offdiag(Z) (FP32), in place; the row panel is
// staged transposed (k-major) in shared memory as FP32.  Thread t owns columns t + 256 c.
template <int R, int CPT>
__global__ void __launch_bounds__(256) k_rotate_mixed(double* __restrict__ X, int64_t ld, int64_t M, int N,
                                                      const float* __restrict__ Zf, const double* __restrict__ zd,
                                                      int upper, const int* guard) {
  // a deferred pass whose factorisation or eigensolve failed leaves X as it is
  if (guard && (guard[0] != 0 || guard[1] != 0)) return;
  extern __shared__ __align__(16) float xsT[];  // N x R
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int rows = (int)min((int64_t)R, M - r0);
  for (int t = threadIdx.x; t < R * N; t += 256) {
    const int r = t / N, k = t % N;
    xsT[k * R + r] = r < rows ? (float)X[(r0 + r) * ld + k] : 0.0f;
  }
  __syncthreads();
  float acc[R][CPT];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[r][c] = 0.0f;
  int jmax = -1;
#pragma unroll
  for (int c = 0; c < CPT; ++c)
    if (threadIdx.x + 256 * c < N) jmax = threadIdx.x + 256 * c;
  const int kend = upper ? jmax + 1 : (jmax >= 0 ? N : 0);
  for (int k = 0; k < kend; ++k) {
    float z[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int j = threadIdx.x + 256 * c;
      z[c] = j < N ? __ldg(Zf + (int64_t)k * N + j) : 0.0f;
    }
#pragma unroll
    for (int r4 = 0; r4 < R; r4 += 4) {
      const float4 xv = *reinterpret_cast<const float4*>(&xsT[k * R + r4]);
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        acc[r4][c] = fmaf(xv.x, z[c], acc[r4][c]);
        acc[r4 + 1][c] = fmaf(xv.y, z[c], acc[r4 + 1][c]);
        acc[r4 + 2][c] = fmaf(xv.z, z[c], acc[r4 + 2][c]);
        acc[r4 + 3][c] = fmaf(xv.w, z[c], acc[r4 + 3][c]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (r >= rows) break;
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int j = threadIdx.x + 256 * c;
      if (j < N) {
        double* x = X + (r0 + r) * ld + j;
        *x = fma(*x, zd[j], (double)acc[r][c]);
      }
    }
  }
}

template <int R, int CPT>
static void launch_rotate_mixed(dftfe_ham h, double* X, int64_t ld, int64_t M, int N, const float* Zf,
                                const double* zd, bool upper) {
  static bool attr = false;
  if (!attr) {
    DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_rotate_mixed<R, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          200 * 1024));
    attr = true;
  }
  const size_t sh = (size_t)R * N * sizeof(float);
  ProfScope ps(h, "rotate_mixed");
  DFTFE_LAUNCH((k_rotate_mixed<R, CPT>), (unsigned)((M + R - 1) / R), 256, sh, h->stream, X, ld, M, N, Zf, zd,
               upper ? 1 : 0, rot_guard(h));
}

void rotate_inplace_mixed(dftfe_ham h, double* X, int64_t ld, int64_t M, int N, const double* Z, bool upper) {
  if (M == 0 || N == 0) return;
  // tensor cores (TF32x3 off-diagonal, FP64 diagonal) whenever the result panel fits TMEM
  if (rotate_inplace_tc(h, X, ld, M, N, Z, upper)) return;
  float* Zf = (float*)ws_get(h, "rotmix_Zf", sizeof(float) * (size_t)N * N);
  double* zd = (double*)ws_get(h, "rotmix_zd", sizeof(double) * (size_t)N);
  DFTFE_LAUNCH(k_split_rot, nblk((int64_t)N * N), 256, 0, h->stream, Z, N, Zf, zd);
  if (N <= 256) launch_rotate_mixed<32, 1>(h, X, ld, M, N, Zf, zd, upper);
  else if (N <= 512) launch_rotate_mixed<32, 2>(h, X, ld, M, N, Zf, zd, upper);
  else if (N <= 1024) launch_rotate_mixed<16, 4>(h, X, ld, M, N, Zf, zd, upper);
  else if (N <= 2048) launch_rotate_mixed<8, 8>(h, X, ld, M, N, Zf, zd, upper);
  else throw Error(DFTFE_ERR_ARG, "more than 2048 states are not supported");
}

}  // namespace dftfe
