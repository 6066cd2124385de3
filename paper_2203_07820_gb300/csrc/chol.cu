// Blocked Cholesky factorisation S = L L^T and triangular inverse Z = L^-T for the
// Cholesky-Gram-Schmidt step (Sec. 3.2, Alg. 2 steps 2a and 3b), FP64, on all SMs.
//
// Right-looking, 32 x 32 blocks (textbook blocked Cholesky): for every block column k
//   1. factor the diagonal block A_kk = L_kk L_kk^T and invert it (one CTA, shared memory),
//   2. L_ik = A_ik L_kk^-T for the blocks below it (one CTA per block),
//   3. A_ij -= L_ik L_jk^T for the trailing lower blocks k < j <= i (one CTA per block).
// The inverse is then formed block row by block row (block forward substitution):
//   (L^-1)_ii = L_ii^-1,  (L^-1)_ij = -L_ii^-1 sum_{k=j}^{i-1} L_ik (L^-1)_kj   (j < i),
// and written transposed as Z = L^-T (upper triangular), with L's strict upper triangle
// zeroed.  A pivot not above 1e-14 times its original diagonal entry (or not finite)
// records DFTFE_ERR_NOT_SPD; the later steps still run on finite stand-in values, so the
// caller reads the status once after the factorisation.
#include "internal.h"

namespace dftfe {

namespace chol {
constexpr int NB = 32;

__device__ __forceinline__ int rows_of(int blk, int N) { return min(NB, N - blk * NB); }

// load the 32 x 32 block (bi, bj) of A (row-major, N x N) into s (zero outside N)
__device__ __forceinline__ void load_block(const double* A, int N, int bi, int bj, double (*s)[NB + 1]) {
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    const int r = t / NB, c = t % NB;
    const int gi = bi * NB + r, gj = bj * NB + c;
    s[r][c] = (gi < N && gj < N) ? A[(int64_t)gi * N + gj] : 0.0;
  }
}
}  // namespace chol

// original diagonal (for the pivot test) and a cleared status word
__global__ void k_chol_save_diag(const double* __restrict__ A, int N, double* __restrict__ d0, int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) d0[i] = A[(int64_t)i * N + i];
  if (i == 0) *status = 0;
}

// step 1: factor and invert the diagonal block k
__global__ void __launch_bounds__(256) k_chol_diag(double* __restrict__ A, int N, int k, const double* __restrict__ d0,
                                                   double* __restrict__ Linv, int* status) {
  using namespace chol;
  __shared__ double a[NB][NB + 1];
  __shared__ double y[NB][NB + 1];
  __shared__ double piv;
  const int nb = rows_of(k, N), off = k * NB;
  load_block(A, N, k, k, a);
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      const double d = a[j][j], dorig = d0[off + j];
      if (!(d > 1e-14 * dorig) || !(dorig > 0.0) || !isfinite(d)) {
        atomicExch(status, (int)DFTFE_ERR_NOT_SPD);
        piv = 1.0;                                    // finite stand-in; the status stays set
      } else {
        piv = sqrt(d);
      }
      a[j][j] = piv;
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) a[i][j] /= piv;
    __syncthreads();
    // trailing update of the block's lower triangle
    const int m = nb - j - 1;
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
      const int i = j + 1 + t / m, l = j + 1 + t % m;
      if (l <= i) a[i][l] -= a[i][j] * a[l][j];
    }
    __syncthreads();
  }
  // L_kk^-1 column by column (thread c solves L y = e_c by forward substitution)
  if (threadIdx.x < NB) {
    const int c = threadIdx.x;
    for (int i = 0; i < NB; ++i) {
      double v = 0.0;
      if (c < nb && i < nb && i >= c) {
        double s = (i == c) ? 1.0 : 0.0;
        for (int l = c; l < i; ++l) s -= a[i][l] * y[l][c];
        v = s / a[i][i];
      }
      y[i][c] = v;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    const int r = t / NB, c = t % NB;
    if (r < nb && c < nb) {
      A[(int64_t)(off + r) * N + off + c] = c <= r ? a[r][c] : 0.0;
      Linv[(int64_t)(off + r) * N + off + c] = y[r][c];
    }
  }
}

// step 2: L_ik = A_ik L_kk^-T for the blocks i > k (block i = k + 1 + blockIdx.x)
__global__ void __launch_bounds__(256) k_chol_panel(double* __restrict__ A, int N, int k, const double* __restrict__ Linv) {
  using namespace chol;
  __shared__ double p[NB][NB + 1];
  __shared__ double li[NB][NB + 1];
  const int bi = k + 1 + blockIdx.x;
  load_block(A, N, bi, k, p);
  load_block(Linv, N, k, k, li);
  __syncthreads();
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    const int r = t / NB, c = t % NB;
    double s = 0.0;
#pragma unroll 8
    for (int l = 0; l <= c; ++l) s = fma(p[r][l], li[c][l], s);     // L_kk^-1 is lower
    const int gi = bi * NB + r, gj = k * NB + c;
    if (gi < N && gj < N) A[(int64_t)gi * N + gj] = s;
  }
}

// step 3: A_ij -= L_ik L_jk^T for k < j <= i (blockIdx.x enumerates the lower pairs)
__global__ void __launch_bounds__(256) k_chol_update(double* __restrict__ A, int N, int k) {
  using namespace chol;
  __shared__ double li[NB][NB + 1];
  __shared__ double lj[NB][NB + 1];
  // pair index t -> (i, j), i >= j, both counted from k + 1
  const int t = blockIdx.x;
  int i = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while (i * (i + 1) / 2 > t) --i;
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  const int j = t - i * (i + 1) / 2;
  const int bi = k + 1 + i, bj = k + 1 + j;
  load_block(A, N, bi, k, li);
  load_block(A, N, bj, k, lj);
  __syncthreads();
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    const int gi = bi * NB + r, gj = bj * NB + c;
    if (gi >= N || gj >= N || (bi == bj && c > r)) continue;
    double s = 0.0;
#pragma unroll 8
    for (int l = 0; l < NB; ++l) s = fma(li[r][l], lj[c][l], s);
    A[(int64_t)gi * N + gj] -= s;
  }
}

// inverse, block row i: (L^-1)_ij = -L_ii^-1 sum_{k=j}^{i-1} L_ik (L^-1)_kj, j = blockIdx.x < i
__global__ void __launch_bounds__(256) k_tri_inv_row(const double* __restrict__ L, int N, int i,
                                                     double* __restrict__ Linv) {
  using namespace chol;
  __shared__ double lk[NB][NB + 1];
  __shared__ double vk[NB][NB + 1];
  __shared__ double acc[NB][NB + 1];
  const int j = blockIdx.x;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) acc[e / NB][e % NB] = 0.0;
  for (int k = j; k < i; ++k) {
    __syncthreads();
    load_block(L, N, i, k, lk);
    load_block(Linv, N, k, j, vk);
    __syncthreads();
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
      const int r = e / NB, c = e % NB;
      double s = acc[r][c];
#pragma unroll 8
      for (int l = 0; l < NB; ++l) s = fma(lk[r][l], vk[l][c], s);
      acc[r][c] = s;
    }
  }
  __syncthreads();
  load_block(Linv, N, i, i, lk);
  __syncthreads();
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    double s = 0.0;
#pragma unroll 8
    for (int l = 0; l <= r; ++l) s = fma(lk[r][l], acc[l][c], s);
    const int gi = i * NB + r, gj = j * NB + c;
    if (gi < N && gj < N) Linv[(int64_t)gi * N + gj] = -s;
  }
}

// Z = (L^-1)^T (upper triangular, zero below the diagonal); L's strict upper triangle zeroed
__global__ void k_tri_finish(double* __restrict__ L, const double* __restrict__ Linv, double* __restrict__ Z, int N) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * N) return;
  const int r = (int)(t / N), c = (int)(t % N);
  Z[t] = c >= r ? Linv[(int64_t)c * N + r] : 0.0;
  if (c > r) L[t] = 0.0;
}

static unsigned nblk_c(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

void cholesky_blocked(dftfe_ham h, double* A, int N, int* d_status) {
  using namespace chol;
  cudaStream_t s = h->stream;
  const int nbk = (N + NB - 1) / NB;
  double* d0 = (double*)ws_get(h, "chol_d0", sizeof(double) * (size_t)N);
  double* Linv = (double*)ws_get(h, "chol_linv", sizeof(double) * (size_t)N * N);
  ProfScope ps(h, "potrf");
  DFTFE_LAUNCH(k_chol_save_diag, nblk_c(N), 256, 0, s, A, N, d0, d_status);
  for (int k = 0; k < nbk; ++k) {
    DFTFE_LAUNCH(k_chol_diag, 1, 256, 0, s, A, N, k, d0, Linv, d_status);
    const int below = nbk - k - 1;
    if (below == 0) break;
    DFTFE_LAUNCH(k_chol_panel, below, 256, 0, s, A, N, k, Linv);
    DFTFE_LAUNCH(k_chol_update, below * (below + 1) / 2, 256, 0, s, A, N, k);
  }
}

void tri_inverse_blocked(dftfe_ham h, double* L, double* Z, int N) {
  using namespace chol;
  cudaStream_t s = h->stream;
  const int nbk = (N + NB - 1) / NB;
  double* Linv = (double*)ws_get(h, "chol_linv", sizeof(double) * (size_t)N * N);
  ProfScope ps(h, "trtri");
  for (int i = 1; i < nbk; ++i) DFTFE_LAUNCH(k_tri_inv_row, i, 256, 0, s, L, N, i, Linv);
  DFTFE_LAUNCH(k_tri_finish, nblk_c((int64_t)N * N), 256, 0, s, L, Linv, Z, N);
}

}  // namespace dftfe
