// Dense FP64 kernels of Cholesky-Gram-Schmidt and Rayleigh-Ritz (a8-a13), the Lanczos
// bound (a7) and the counter-based random numbers.
//
//  gram_lower   C = A^T B, lower triangle (Alg. 2 steps 1a/1b; only the lower triangle
//               is formed, as in Sec. 4.4), split over the long M dimension with a
//               fixed-order second-stage sum (deterministic).
//  potrf        S = L L^T, left-looking, one CTA (Alg. 2 step 2a).
//  trtri        Z = L^-T, one thread per column of L^-1 (forward substitution).
//  rotate       X <- X Z in place, row panels staged in shared memory (steps 3a/3b).
//  syevd        H^ = Q Theta Q^T: parallel cyclic Jacobi in one cooperative launch, then
//               ascending sort and the sign convention (step 2b-c); syevd_z is the
//               Hermitian form for Bloch k-points.
//  tridiag_ql   implicit-shift QL on a tridiagonal (Bowdler, Martin, Reinsch, Wilkinson,
//               Numer. Math. 11, 1968), for the Lanczos bound.
//  residuals    ||W_i - theta_i X_i|| or the generalised form (a13), real or complex.
#include "internal.h"

#include <cmath>
#include <vector>

namespace dftfe {

static unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ----------------------------------------------------------- block reduction
template <int NT>
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < NT / 32; ++w) t += red[w];
    red[NT / 32] = t;
  }
  __syncthreads();
  return red[NT / 32];
}

// ------------------------------------------------------------------ Gram
constexpr int GT = 64, GK = 16;
__global__ void __launch_bounds__(256) k_gram_partial(const double* __restrict__ A, int64_t lda,
                                                      const double* __restrict__ B, int64_t ldb,
                                                      int64_t M, int N, int64_t rows_per_split,
                                                      double* __restrict__ part) {
  __shared__ double As[GK][GT];
  __shared__ double Bs[GK][GT];
  // tile (ti, tj) of the lower triangle, row-major: blockIdx.x = ti (ti + 1) / 2 + tj
  const int t = blockIdx.x;
  int ti = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
  while (ti * (ti + 1) / 2 > t) --ti;
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  const int tj = t - ti * (ti + 1) / 2;
  const int i0 = ti * GT, j0 = tj * GT;
  const int64_t m0 = (int64_t)blockIdx.y * rows_per_split;
  const int64_t m1 = min(M, m0 + rows_per_split);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  for (int64_t mm = m0; mm < m1; mm += GK) {
    for (int e = threadIdx.x; e < GK * GT; e += 256) {
      const int kk = e / GT, c = e % GT;
      const int64_t row = mm + kk;
      const bool rok = row < m1;
      As[kk][c] = (rok && i0 + c < N) ? A[row * lda + i0 + c] : 0.0;
      Bs[kk][c] = (rok && j0 + c < N) ? B[row * ldb + j0 + c] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double* out = part + (int64_t)blockIdx.y * N * N;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = i0 + ty + 16 * i;
    if (gi >= N) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = j0 + tx + 16 * j;
      if (gj < N) out[(int64_t)gi * N + gj] = acc[i][j];
    }
  }
}

// C[i][j] = C[j][i] = sum_s part[s][i][j] for i >= j (fixed order over s).
__global__ void k_gram_reduce(const double* __restrict__ part, int nsplit, int N, double* __restrict__ C) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * N) return;
  const int i = (int)(t / N), j = (int)(t % N);
  if (i < j) return;
  double s = 0.0;
  for (int k = 0; k < nsplit; ++k) s += part[(int64_t)k * N * N + t];
  C[(int64_t)i * N + j] = s;
  C[(int64_t)j * N + i] = s;
}

int gram_nsplit(dftfe_ham h, int64_t M, int N) {
  const int T = (N + GT - 1) / GT;
  const int ntiles = T * (T + 1) / 2;
  int64_t want = (4LL * h->sm_count + ntiles - 1) / ntiles;
  int64_t maxs = std::max<int64_t>(1, M / 256);
  return (int)std::max<int64_t>(1, std::min(want, maxs));
}

void gram_lower(dftfe_ham h, const double* A, int64_t lda, const double* B, int64_t ldb, int64_t M,
                int N, double* C, double* part, int nsplit) {
  // no host data: the kernel decodes its tile from the block index, so the launch can be
  // captured in a CUDA graph and replayed
  const int T = (N + GT - 1) / GT;
  const int ntiles = T * (T + 1) / 2;
  const int64_t rows = (M + nsplit - 1) / nsplit;
  {
    ProfScope ps(h, "gram");
    DFTFE_LAUNCH(k_gram_partial, dim3(ntiles, nsplit), 256, 0, h->stream, A, lda, B, ldb, M, N,
                 rows, part);
  }
  DFTFE_LAUNCH(k_gram_reduce, nblk((int64_t)N * N), 256, 0, h->stream, part, nsplit, N, C);
}

// ---------------------------------------------------------------- Cholesky
// Left-looking Cholesky of the lower triangle of A (N x N, row-major) in place; the
// strict upper triangle is zeroed.  status = DFTFE_ERR_NOT_SPD when a pivot is not
// larger than 1e-14 times its original diagonal entry (S numerically singular).
__global__ void __launch_bounds__(1024) k_potrf(double* A, int N, int* status) {
  __shared__ double diag, dorig;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < N; ++j) {
    if (threadIdx.x == 0) dorig = A[(int64_t)j * N + j];
    __syncthreads();
    for (int i = j + threadIdx.x; i < N; i += blockDim.x) {
      double s = A[(int64_t)i * N + j];
      const double* Li = A + (int64_t)i * N;
      const double* Lj = A + (int64_t)j * N;
      for (int k = 0; k < j; ++k) s -= Li[k] * Lj[k];
      A[(int64_t)i * N + j] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const double d = A[(int64_t)j * N + j];
      if (!(d > 1e-14 * dorig) || !(dorig > 0.0) || !isfinite(d)) bad = 1;
      else {
        diag = sqrt(d);
        A[(int64_t)j * N + j] = diag;
      }
    }
    __syncthreads();
    if (bad) break;
    for (int i = j + 1 + threadIdx.x; i < N; i += blockDim.x) A[(int64_t)i * N + j] /= diag;
    __syncthreads();
  }
  if (!bad)
    for (int64_t t = threadIdx.x; t < (int64_t)N * N; t += blockDim.x) {
      const int i = (int)(t / N), j = (int)(t % N);
      if (j > i) A[t] = 0.0;
    }
  if (threadIdx.x == 0) *status = bad ? (int)DFTFE_ERR_NOT_SPD : 0;
}

void potrf(cudaStream_t s, double* A, int N, int* d_status) {
  DFTFE_LAUNCH(k_potrf, 1, 1024, 0, s, A, N, d_status);
}

// Z = L^-T: thread j solves L y = e_j by forward substitution and stores y as row j of Z.
__global__ void k_trtri(const double* __restrict__ L, double* __restrict__ Z, int N) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double* y = Z + (int64_t)j * N;
  for (int i = 0; i < j; ++i) y[i] = 0.0;
  for (int i = j; i < N; ++i) {
    double s = (i == j) ? 1.0 : 0.0;
    const double* Li = L + (int64_t)i * N;
    for (int k = j; k < i; ++k) s -= Li[k] * y[k];
    y[i] = s / Li[i];
  }
}

void trtri_lower_to_upper_t(cudaStream_t s, const double* L, double* Z, int N) {
  DFTFE_LAUNCH(k_trtri, nblk(N, 128), 128, 0, s, L, Z, N);
}

// ------------------------------------------------------------------ rotate
// X[r0:r0+R, :] <- X[r0:r0+R, :] Z, in place.  Thread t owns columns t + 256 c.
template <int R, int CPT>
__global__ void __launch_bounds__(256) k_rotate(double* __restrict__ X, int64_t ld, int64_t M, int N,
                                                const double* __restrict__ Z, int upper, const int* guard) {
  // a deferred pass whose factorisation or eigensolve failed leaves X as it is
  if (guard && (guard[0] != 0 || guard[1] != 0)) return;
  extern __shared__ double xs[];  // R x N
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int rows = (int)min((int64_t)R, M - r0);
  for (int t = threadIdx.x; t < R * N; t += 256) {
    const int r = t / N, k = t % N;
    xs[t] = r < rows ? X[(r0 + r) * ld + k] : 0.0;
  }
  __syncthreads();
  double acc[R][CPT];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[r][c] = 0.0;
  int jmax = -1;
#pragma unroll
  for (int c = 0; c < CPT; ++c)
    if (threadIdx.x + 256 * c < N) jmax = threadIdx.x + 256 * c;
  const int kend = upper ? jmax + 1 : (jmax >= 0 ? N : 0);
  for (int k = 0; k < kend; ++k) {
    double z[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int j = threadIdx.x + 256 * c;
      z[c] = j < N ? __ldg(Z + (int64_t)k * N + j) : 0.0;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const double xv = xs[r * N + k];
#pragma unroll
      for (int c = 0; c < CPT; ++c) acc[r][c] = fma(xv, z[c], acc[r][c]);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (r >= rows) break;
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int j = threadIdx.x + 256 * c;
      if (j < N) X[(r0 + r) * ld + j] = acc[r][c];
    }
  }
}

template <int R, int CPT>
static void launch_rotate(dftfe_ham h, double* X, int64_t ld, int64_t M, int N, const double* Z, bool upper) {
  const size_t sh = (size_t)R * N * sizeof(double);
  static bool attr = false;
  if (!attr) {
    DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_rotate<R, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          200 * 1024));
    attr = true;
  }
  const unsigned grid = (unsigned)((M + R - 1) / R);
  ProfScope ps(h, "rotate");
  DFTFE_LAUNCH((k_rotate<R, CPT>), grid, 256, sh, h->stream, X, ld, M, N, Z, upper ? 1 : 0, rot_guard(h));
}

void rotate_inplace(dftfe_ham h, double* X, int64_t ld, int64_t M, int N, const double* Z, bool upper) {
  if (M == 0 || N == 0) return;
  if (N <= 256) launch_rotate<32, 1>(h, X, ld, M, N, Z, upper);
  else if (N <= 512) launch_rotate<32, 2>(h, X, ld, M, N, Z, upper);
  else if (N <= 1024) launch_rotate<16, 4>(h, X, ld, M, N, Z, upper);
  else if (N <= 2048) launch_rotate<8, 8>(h, X, ld, M, N, Z, upper);
  else throw Error(DFTFE_ERR_ARG, "more than 2048 states are not supported");
}

// -------------------------------------------------------------- eigensolver
// Dense symmetric eigensolver: cyclic two-sided Jacobi with the round-robin (circle)
// pairing, so each round rotates N/2 disjoint planes at once (Golub & Van Loan, parallel
// Jacobi).  One cooperative launch runs all sweeps; the CTAs meet at a bounded grid
// barrier after every round.  Every CTA computes all N/2 rotations of a round from the
// same matrix entries, so all agree on them and on convergence without exchanging them.
namespace jac {

constexpr long kBarrierSpins = 20000000L;   // x 64 ns sleep: about a second

struct Barrier {
  unsigned int count;
  unsigned int gen;
  int abort;
  unsigned int reads;   // CTAs that have read the rotation inputs, summed over rounds
  long long limit;      // spin iterations before a wait gives up
  unsigned int missing; // arrivals the barrier expects beyond the grid (0; 1 only in the wait test)
};

// every call starts from a cleared barrier with its spin limit and expected arrivals
__global__ void k_bar_init(Barrier* b, long long limit, unsigned int missing) {
  b->count = 0;
  b->gen = 0;
  b->abort = 0;
  b->reads = 0;
  b->limit = limit > 0 ? limit : (long long)kBarrierSpins;
  b->missing = missing;
}

// split barrier: the rotation inputs of a round (A_pp, A_qq, A_pq of every pair) may be
// overwritten only once every CTA has read them
__device__ void arrive_read(Barrier* b) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&b->reads, 1u);
  }
}

__device__ bool wait_reads(Barrier* b, unsigned int target, int* status) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int* vr = &b->reads;
    volatile int* vabort = &b->abort;
    const long long lim = b->limit;
    long long it = 0;
    while (*vr < target) {
      if (*vabort || ++it > lim) {
        ok = 0;
        atomicExch(&b->abort, 1);
        atomicCAS(status, 0, (int)DFTFE_ERR_TIMEOUT);
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// grid-wide barrier (all CTAs are co-resident under the cooperative launch); false when
// a wait ran out or another CTA gave up
__device__ bool grid_barrier(Barrier* b, int* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int* vgen = &b->gen;
    volatile int* vabort = &b->abort;
    const unsigned int g = *vgen;
    const long long lim = b->limit;
    __threadfence();
    if (atomicAdd(&b->count, 1u) == gridDim.x - 1 + b->missing) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      long long it = 0;
      while (*vgen == g) {
        if (*vabort || ++it > lim) {
          ok = 0;
          atomicExch(&b->abort, 1);
          atomicCAS(status, 0, (int)DFTFE_ERR_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// players a, b of pair P in round k of the circle method on Ne (even) indices
__device__ __forceinline__ void pairing(int k, int P, int Ne, int& p, int& q) {
  const int m = Ne - 1;
  int a, b;
  if (P == 0) {
    a = 0;
    b = 1 + k % m;
  } else {
    a = 1 + (k + P) % m;
    b = 1 + (k - P + m) % m;
  }
  p = min(a, b);
  q = max(a, b);
}

}  // namespace jac

// A (N x N symmetric, only the lower triangle is read) -> VT (rows = eigenvectors) and
// d (eigenvalues, unsorted).  Dynamic shared memory: 3 doubles + 2 ints per pair.
__global__ void __launch_bounds__(256) k_jacobi(double* __restrict__ A, double* __restrict__ VT, double* __restrict__ d,
                                                int N, int max_sweeps, const double* __restrict__ anorm_p,
                                                jac::Barrier* bar, int* status) {
  extern __shared__ double jsm[];
  const int Ne = N + (N & 1), NP = Ne / 2, m = Ne - 1;
  double* cs = jsm;
  double* sn = cs + NP;
  double* tn = sn + NP;
  int* pp = reinterpret_cast<int*>(tn + NP);
  int* qq = pp + NP;
  __shared__ int rotated;
  const double anorm = *anorm_p;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  // full symmetric copy from the lower triangle, VT = I
  for (int64_t w = gtid; w < (int64_t)N * N; w += gthreads) {
    const int i = (int)(w / N), j = (int)(w % N);
    if (i < j) A[w] = A[(int64_t)j * N + i];
    VT[w] = i == j ? 1.0 : 0.0;
  }
  if (!jac::grid_barrier(bar, status)) return;
  bool converged = false;
  unsigned int round = 0;
  for (int sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int k = 0; k < m; ++k) {
      // the N/2 rotations of this round (Golub & Van Loan's symmetric 2x2 Schur form)
      for (int P = threadIdx.x; P < NP; P += blockDim.x) {
        int p, q;
        jac::pairing(k, P, Ne, p, q);
        double c = 1.0, s = 0.0, t = 0.0;
        if (q < N) {
          const double apq = A[(int64_t)p * N + q];
          const double app = A[(int64_t)p * N + p], aqq = A[(int64_t)q * N + q];
          const double small = fmax(1e-15 * sqrt(fabs(app) * fabs(aqq)), 1e-18 * anorm);
          if (fabs(apq) > small) {
            const double tau = (aqq - app) / (2.0 * apq);
            t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(fma(tau, tau, 1.0)));
            c = 1.0 / sqrt(fma(t, t, 1.0));
            s = t * c;
            rotated = 1;
          }
        }
        cs[P] = c;
        sn[P] = s;
        tn[P] = t;
        pp[P] = p;
        qq[P] = q;
      }
      jac::arrive_read(bar);   // ends with the CTA's rotations in shared memory
      ++round;
      // A <- J^T A J, one 2 x 2 block (row pair P, column pair R) per work item; the
      // diagonal blocks (which hold the rotation inputs) come last
      for (int64_t w = gtid; w < (int64_t)NP * NP; w += gthreads) {
        const int P = (int)(w / NP), R = (int)(w % NP);
        const double c = cs[P], s = sn[P], c2 = cs[R], s2 = sn[R];
        if ((s == 0.0 && s2 == 0.0) || P == R) continue;
        const int p = pp[P], q = qq[P], p2 = pp[R], q2 = qq[R];
        // with N odd one pair per round holds the absent index N: that row / column is
        // left out (its entries count as zero), the rest of the block is rotated as usual
        const bool hq = q < N, hq2 = q2 < N;
        double* rp = A + (int64_t)p * N;
        double* rq = A + (int64_t)(hq ? q : p) * N;
        const double x00 = rp[p2], x01 = hq2 ? rp[q2] : 0.0;
        const double x10 = hq ? rq[p2] : 0.0, x11 = hq && hq2 ? rq[q2] : 0.0;
        const double t00 = c * x00 - s * x10, t01 = c * x01 - s * x11;
        const double t10 = s * x00 + c * x10, t11 = s * x01 + c * x11;
        rp[p2] = t00 * c2 - t01 * s2;
        if (hq2) rp[q2] = t00 * s2 + t01 * c2;
        if (hq) rq[p2] = t10 * c2 - t11 * s2;
        if (hq && hq2) rq[q2] = t10 * s2 + t11 * c2;
      }
      if (!jac::wait_reads(bar, round * gridDim.x, status)) return;
      for (int64_t P = gtid; P < NP; P += gthreads) {
        if (sn[P] == 0.0) continue;
        double* rp = A + (int64_t)pp[P] * N;
        double* rq = A + (int64_t)qq[P] * N;
        const int p = pp[P], q = qq[P];
        const double apq = rp[q], t = tn[P];
        rp[p] -= t * apq;
        rq[q] += t * apq;
        rp[q] = 0.0;
        rq[p] = 0.0;
      }
      // V <- V J on the rows of VT
      for (int64_t w = gtid; w < (int64_t)NP * N; w += gthreads) {
        const int P = (int)(w / N), i = (int)(w % N);
        const double s = sn[P];
        if (s == 0.0 || qq[P] >= N) continue;
        const double c = cs[P];
        double* vp = VT + (int64_t)pp[P] * N + i;
        double* vq = VT + (int64_t)qq[P] * N + i;
        const double a = *vp, b = *vq;
        *vp = c * a - s * b;
        *vq = s * a + c * b;
      }
      if (!jac::grid_barrier(bar, status)) return;
    }
    converged = rotated == 0;   // same in every CTA
    __syncthreads();            // everyone has read the flag before it is reset
  }
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) d[i] = A[(int64_t)i * N + i];
    if (threadIdx.x == 0 && !converged) atomicCAS(status, 0, (int)DFTFE_ERR_NOCONV);
  }
}

// complex helpers for the Hermitian Jacobi
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 zlin(double a, double2 x, double b, double2 y) {   // a x + b y
  return make_double2(a * x.x + b * y.x, a * x.y + b * y.y);
}

// Hermitian form of k_jacobi: A (N x N complex, lower triangle read) -> VT (row p = column p
// of V, not conjugated) and d.  A rotation of the pair (p, q) first makes a_pq real and
// non-negative with the diagonal unitary D = diag(1, conj(w)), w = a_pq / |a_pq| (row q of A
// times w, column q times conj(w)), then applies k_jacobi's real symmetric rotation R to the
// resulting real 2 x 2 problem: J = D R, A <- J^H A J, V <- V J.  Same pairing, barriers,
// convergence test and work split as k_jacobi.  Dynamic shared memory: 4 doubles, one
// complex and 2 ints per pair.
__global__ void __launch_bounds__(256) k_jacobi_z(double2* __restrict__ A, double2* __restrict__ VT,
                                                  double* __restrict__ d, int N, int max_sweeps,
                                                  const double* __restrict__ anorm_p, jac::Barrier* bar,
                                                  int* status) {
  extern __shared__ double jsm[];
  const int Ne = N + (N & 1), NP = Ne / 2, m = Ne - 1;
  double* cs = jsm;
  double* sn = cs + NP;
  double* tn = sn + NP;
  double* mg = tn + NP;
  double2* om = reinterpret_cast<double2*>(mg + NP);   // 4 NP doubles in: 16-byte aligned
  int* pp = reinterpret_cast<int*>(om + NP);
  int* qq = pp + NP;
  __shared__ int rotated;
  const double anorm = *anorm_p;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  // full Hermitian copy from the lower triangle (real diagonal), VT = I
  for (int64_t w = gtid; w < (int64_t)N * N; w += gthreads) {
    const int i = (int)(w / N), j = (int)(w % N);
    if (i < j) A[w] = zconj(A[(int64_t)j * N + i]);
    else if (i == j) A[w].y = 0.0;
    VT[w] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  if (!jac::grid_barrier(bar, status)) return;
  bool converged = false;
  unsigned int round = 0;
  for (int sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int k = 0; k < m; ++k) {
      for (int P = threadIdx.x; P < NP; P += blockDim.x) {
        int p, q;
        jac::pairing(k, P, Ne, p, q);
        double c = 1.0, s = 0.0, t = 0.0, mag = 0.0;
        double2 w = make_double2(1.0, 0.0);
        if (q < N) {
          const double2 apq = A[(int64_t)p * N + q];
          mag = hypot(apq.x, apq.y);
          const double app = A[(int64_t)p * N + p].x, aqq = A[(int64_t)q * N + q].x;
          const double small = fmax(1e-15 * sqrt(fabs(app) * fabs(aqq)), 1e-18 * anorm);
          if (mag > small) {
            const double tau = (aqq - app) / (2.0 * mag);
            t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(fma(tau, tau, 1.0)));
            c = 1.0 / sqrt(fma(t, t, 1.0));
            s = t * c;
            w = make_double2(apq.x / mag, apq.y / mag);
            rotated = 1;
          }
        }
        cs[P] = c;
        sn[P] = s;
        tn[P] = t;
        mg[P] = mag;
        om[P] = w;
        pp[P] = p;
        qq[P] = q;
      }
      jac::arrive_read(bar);
      ++round;
      // A <- J^H A J on the off-diagonal 2 x 2 blocks (row pair P, column pair R)
      for (int64_t wi = gtid; wi < (int64_t)NP * NP; wi += gthreads) {
        const int P = (int)(wi / NP), R = (int)(wi % NP);
        const double c = cs[P], s = sn[P], c2 = cs[R], s2 = sn[R];
        if ((s == 0.0 && s2 == 0.0) || P == R) continue;
        const int p = pp[P], q = qq[P], p2 = pp[R], q2 = qq[R];
        const bool hq = q < N, hq2 = q2 < N;
        double2* rp = A + (int64_t)p * N;
        double2* rq = A + (int64_t)(hq ? q : p) * N;
        const double2 z0 = make_double2(0.0, 0.0);
        const double2 x00 = rp[p2], x01 = hq2 ? rp[q2] : z0;
        const double2 x10 = hq ? rq[p2] : z0, x11 = hq && hq2 ? rq[q2] : z0;
        const double2 wP = om[P], wRc = zconj(om[R]);
        const double2 y10 = zmul(wP, x10), y11 = zmul(wP, x11);          // row q times w_P
        const double2 t00 = zlin(c, x00, -s, y10), t01 = zlin(c, x01, -s, y11);
        const double2 t10 = zlin(s, x00, c, y10), t11 = zlin(s, x01, c, y11);
        const double2 u01 = zmul(wRc, t01), u11 = zmul(wRc, t11);         // column q2 times conj(w_R)
        rp[p2] = zlin(c2, t00, -s2, u01);
        if (hq2) rp[q2] = zlin(s2, t00, c2, u01);
        if (hq) rq[p2] = zlin(c2, t10, -s2, u11);
        if (hq && hq2) rq[q2] = zlin(s2, t10, c2, u11);
      }
      if (!jac::wait_reads(bar, round * gridDim.x, status)) return;
      for (int64_t P = gtid; P < NP; P += gthreads) {
        if (sn[P] == 0.0) continue;
        double2* rp = A + (int64_t)pp[P] * N;
        double2* rq = A + (int64_t)qq[P] * N;
        const int p = pp[P], q = qq[P];
        const double tm = tn[P] * mg[P];
        rp[p].x -= tm;
        rq[q].x += tm;
        rp[q] = make_double2(0.0, 0.0);
        rq[p] = make_double2(0.0, 0.0);
      }
      // V <- V J on the rows of VT
      for (int64_t wi = gtid; wi < (int64_t)NP * N; wi += gthreads) {
        const int P = (int)(wi / N), i = (int)(wi % N);
        const double s = sn[P];
        if (s == 0.0 || qq[P] >= N) continue;
        const double c = cs[P];
        double2* vp = VT + (int64_t)pp[P] * N + i;
        double2* vq = VT + (int64_t)qq[P] * N + i;
        const double2 a = *vp, b = zmul(zconj(om[P]), *vq);
        *vp = zlin(c, a, -s, b);
        *vq = zlin(s, a, c, b);
      }
      if (!jac::grid_barrier(bar, status)) return;
    }
    converged = rotated == 0;
    __syncthreads();
  }
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) d[i] = A[(int64_t)i * N + i].x;
    if (threadIdx.x == 0 && !converged) atomicCAS(status, 0, (int)DFTFE_ERR_NOCONV);
  }
}

// Frobenius norm of a Hermitian matrix from its lower triangle (complex, interleaved)
__global__ void k_fro_norm_z(const double2* __restrict__ A, int N, double* out) {
  __shared__ double red[9];
  double s = 0.0;
  for (int64_t w = threadIdx.x; w < (int64_t)N * N; w += blockDim.x) {
    const int i = (int)(w / N), j = (int)(w % N);
    const double a2 = A[w].x * A[w].x + A[w].y * A[w].y;
    if (i >= j) s += i > j ? 2.0 * a2 : a2;
  }
  s = block_sum<256>(s, red);
  if (threadIdx.x == 0) *out = sqrt(s);
}

__global__ void k_fro_norm(const double* __restrict__ A, int N, double* out) {
  __shared__ double red[9];
  double s = 0.0;
  for (int64_t w = threadIdx.x; w < (int64_t)N * N; w += blockDim.x) {
    const int i = (int)(w / N), j = (int)(w % N);
    if (i >= j) s = fma(i > j ? 2.0 * A[w] : A[w], A[w], s);   // lower triangle, off-diagonal twice
  }
  s = block_sum<256>(s, red);
  if (threadIdx.x == 0) *out = sqrt(s);
}

// Implicit QL with Wilkinson shifts on (d, e); rotations are replayed on the rows of Z
// this CTA holds in shared memory.  Every CTA runs the same scalar recurrence (lane 0),
// so all agree on d; CTA 0 writes it back.
__global__ void __launch_bounds__(32) k_tql(double* __restrict__ dg, double* __restrict__ eg,
                                            double* __restrict__ Z, int N, int R, int* status) {
  extern __shared__ double sm[];
  double* d = sm;                 // N
  double* e = d + N;              // N
  double* cs = e + N;             // N
  double* sn = cs + N;            // N
  double* zr = sn + N;            // R x (N+1)
  __shared__ int nrot, base, fail;
  const int r0 = blockIdx.x * R;
  const int myrow = r0 + threadIdx.x;
  const bool have = threadIdx.x < R && myrow < N;
  for (int i = threadIdx.x; i < N; i += 32) {
    d[i] = dg[i];
    e[i] = (i < N - 1) ? eg[i] : 0.0;
  }
  for (int r = 0; r < R; ++r)
    if (r0 + r < N)
      for (int j = threadIdx.x; j < N; j += 32) zr[r * (N + 1) + j] = Z[(int64_t)(r0 + r) * N + j];
  if (threadIdx.x == 0) fail = 0;
  __syncwarp();
  const double eps = 2.220446049250313e-16;
  for (int l = 0; l < N; ++l) {
    int iter = 0;
    while (true) {
      // lane 0 performs one QL sweep (or detects convergence) and records the rotations
      if (threadIdx.x == 0) {
        nrot = 0;
        int m = l;
        for (; m < N - 1; ++m) {
          const double dd = fabs(d[m]) + fabs(d[m + 1]);
          if (fabs(e[m]) <= eps * dd) break;
        }
        if (m == l) {
          nrot = -1;
        } else if (iter >= 60) {
          nrot = -1;
          fail = 1;
        } else {
          ++iter;
          double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
          double r = sqrt(fma(g, g, 1.0));
          g = d[m] - d[l] + e[l] / (g + copysign(r, g));
          double s = 1.0, c = 1.0, p = 0.0;
          int i = m - 1;
          bool early = false;
          for (; i >= l; --i) {
            const double f = s * e[i], b = c * e[i];
            // Givens rotation from (f, g): one reciprocal square root instead of a
            // hypot and two divisions (the FP64 pipe is slow; this loop is serial)
            const double r2 = fma(f, f, g * g);
            if (r2 == 0.0) {
              e[i + 1] = 0.0;
              d[i + 1] -= p;
              e[m] = 0.0;
              early = true;
              break;
            }
            const double rinv = rsqrt(r2);
            r = r2 * rinv;
            e[i + 1] = r;
            s = f * rinv;
            c = g * rinv;
            g = d[i + 1] - p;
            r = (d[i] - g) * s + 2.0 * c * b;
            p = s * r;
            d[i + 1] = g + p;
            g = c * r - b;
            cs[nrot] = c;
            sn[nrot] = s;
            ++nrot;
          }
          base = m - 1;  // rotation t acts on columns (base - t, base - t + 1)
          if (!early) {
            d[l] -= p;
            e[l] = g;
            e[m] = 0.0;
          }
        }
      }
      __syncwarp();
      const int nr = nrot;
      if (nr < 0) break;
      if (have) {
        double* z = zr + threadIdx.x * (N + 1);
        const int b0 = base;
        for (int t = 0; t < nr; ++t) {
          const int i = b0 - t;
          const double f = z[i + 1];
          z[i + 1] = sn[t] * z[i] + cs[t] * f;
          z[i] = cs[t] * z[i] - sn[t] * f;
        }
      }
      __syncwarp();
    }
    if (fail) break;
  }
  __syncwarp();
  if (have)
    for (int j = 0; j < N; ++j) Z[(int64_t)myrow * N + j] = zr[threadIdx.x * (N + 1) + j];
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < N; i += 32) dg[i] = d[i];
    if (threadIdx.x == 0) *status = fail ? (int)DFTFE_ERR_NOCONV : 0;
  }
}

void tridiag_ql(cudaStream_t s, double* d, double* e, double* Z, int N, int* d_status) {
  int R = (int)std::min<int64_t>(32, std::max<int64_t>(1, 131072 / ((int64_t)(N + 1) * 8)));
  size_t sh = (size_t)(4 * N + R * (N + 1)) * sizeof(double);
  static bool attr = false;
  if (!attr) {
    DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_tql, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    attr = true;
  }
  if (sh > 220 * 1024) throw Error(DFTFE_ERR_ARG, "dense eigensolver: N too large");
  DFTFE_LAUNCH(k_tql, (unsigned)((N + R - 1) / R), 32, sh, s, d, e, Z, N, R, d_status);
}

// ascending order (ties by index) and the sign convention: the largest-|.| entry of each
// eigenvector (first one on ties) is made positive.
// ascending order by a strict total order (NaN after every number, ties by index), so perm
// is a permutation whatever d holds (an eigensolver that gave up leaves d unspecified)
__global__ void k_rank(const double* d, int N, int* perm, double* evals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double di = d[i];
  const bool ni = isnan(di);
  int r = 0;
  for (int j = 0; j < N; ++j) {
    const double dj = d[j];
    const bool nj = isnan(dj);
    r += ni ? (!nj || j < i) : (!nj && (dj < di || (dj == di && j < i)));
  }
  perm[r] = i;
  evals[r] = di;
}

// Z holds the eigenvectors as rows (Z[src * N + r] = component r of vector src)
__global__ void __launch_bounds__(256) k_sign_copy(const double* __restrict__ Z, const int* perm, int N,
                                                   double* __restrict__ Q) {
  __shared__ double bv[256];
  __shared__ int bi[256];
  const int c = blockIdx.x;
  int src = perm[c];
  if (src < 0 || src >= N) src = c;               // defensive: perm comes from k_rank
  double best = -1.0;
  int bidx = N;
  for (int r = threadIdx.x; r < N; r += 256) {
    const double a = fabs(Z[(int64_t)src * N + r]);
    if (a > best || (a == best && r < bidx)) { best = a; bidx = r; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = bidx;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double o = bv[threadIdx.x + s];
      const int oi = bi[threadIdx.x + s];
      if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
        bv[threadIdx.x] = o;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const double sgn = Z[(int64_t)src * N + bi[0]] < 0.0 ? -1.0 : 1.0;
  for (int r = threadIdx.x; r < N; r += 256) Q[(int64_t)r * N + c] = sgn * Z[(int64_t)src * N + r];
}

void syevd(dftfe_ham h, double* A, int N, double* evals, double* Q, int* d_status) {
  cudaStream_t s = h->stream;
  ProfScope ps(h, "syevd");
  const int NP = (N + (N & 1)) / 2;
  double* VT = (double*)ws_get(h, "eig_V", sizeof(double) * (size_t)N * N);
  double* vec = (double*)ws_get(h, "eig_vec", sizeof(double) * (size_t)N + 64);
  double* d = vec;
  double* anorm = vec + N;
  jac::Barrier* bar = (jac::Barrier*)ws_get(h, "eig_bar", sizeof(jac::Barrier));
  int* perm = (int*)ws_get(h, "eig_perm", sizeof(int) * (size_t)N);
  const size_t sh = (size_t)NP * (3 * sizeof(double) + 2 * sizeof(int));
  static bool attr = false;
  if (!attr) {
    DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, 48 * 1024));
    attr = true;
  }
  if (sh > 48 * 1024) throw Error(DFTFE_ERR_ARG, "dense eigensolver: N too large");
  int per_sm = 0;
  DFTFE_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi, 256, sh));
  if (per_sm < 1) throw Error(DFTFE_ERR_CUDA, "dense eigensolver: kernel does not fit on an SM");
  // enough CTAs for the widest round, never more than can be co-resident
  const int want = (int)std::min<int64_t>(h->sm_count, ((int64_t)NP * N + 255) / 256);
  int grid = std::max(1, want);
  DFTFE_LAUNCH(jac::k_bar_init, 1, 1, 0, s, bar, h->wait_limit, (unsigned int)h->wait_missing);
  DFTFE_CHECK_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), s));
  DFTFE_LAUNCH(k_fro_norm, 1, 256, 0, s, A, N, anorm);
  int maxs = 60;
  void* args[] = {&A, &VT, &d, &N, &maxs, &anorm, &bar, &d_status};
  DFTFE_CHECK_CUDA(cudaLaunchCooperativeKernel((const void*)k_jacobi, dim3(grid), dim3(256), args, sh, s));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  DFTFE_LAUNCH(k_rank, nblk(N, 128), 128, 0, s, d, N, perm, evals);
  DFTFE_LAUNCH(k_sign_copy, N, 256, 0, s, VT, perm, N, Q);
}

// complex eigenvectors (rows of VT) -> columns of Q in ascending order, each multiplied by
// the phase that makes its largest-|.| entry (first on ties) real and positive
__global__ void __launch_bounds__(256) k_phase_copy_z(const double2* __restrict__ VT, const int* perm, int N,
                                                      double2* __restrict__ Q) {
  __shared__ double bv[256];
  __shared__ int bi[256];
  const int c = blockIdx.x;
  int src = perm[c];
  if (src < 0 || src >= N) src = c;               // defensive: perm comes from k_rank
  double best = -1.0;
  int bidx = N;
  for (int r = threadIdx.x; r < N; r += 256) {
    const double2 v = VT[(int64_t)src * N + r];
    const double a = hypot(v.x, v.y);
    if (a > best || (a == best && r < bidx)) { best = a; bidx = r; }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = bidx;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double o = bv[threadIdx.x + s];
      const int oi = bi[threadIdx.x + s];
      if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
        bv[threadIdx.x] = o;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const double2 pv = VT[(int64_t)src * N + bi[0]];
  const double a = bv[0];
  const double2 ph = a > 0.0 ? make_double2(pv.x / a, -pv.y / a) : make_double2(1.0, 0.0);
  for (int r = threadIdx.x; r < N; r += 256) Q[(int64_t)r * N + c] = zmul(ph, VT[(int64_t)src * N + r]);
}

void syevd_z(dftfe_ham h, double* Ad, int N, double* evals, double* Qd, int* d_status) {
  cudaStream_t s = h->stream;
  ProfScope ps(h, "syevd_z");
  double2* A = reinterpret_cast<double2*>(Ad);
  double2* Q = reinterpret_cast<double2*>(Qd);
  const int NP = (N + (N & 1)) / 2;
  double2* VT = (double2*)ws_get(h, "eigz_V", sizeof(double2) * (size_t)N * N);
  double* vec = (double*)ws_get(h, "eig_vec", sizeof(double) * (size_t)N + 64);
  double* d = vec;
  double* anorm = vec + N;
  jac::Barrier* bar = (jac::Barrier*)ws_get(h, "eig_bar", sizeof(jac::Barrier));
  int* perm = (int*)ws_get(h, "eig_perm", sizeof(int) * (size_t)N);
  const size_t sh = (size_t)NP * (6 * sizeof(double) + 2 * sizeof(int));
  static bool attr = false;
  if (!attr) {
    DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_jacobi_z, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
    attr = true;
  }
  if (sh > 64 * 1024) throw Error(DFTFE_ERR_ARG, "dense eigensolver: N too large");
  int per_sm = 0;
  DFTFE_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_z, 256, sh));
  if (per_sm < 1) throw Error(DFTFE_ERR_CUDA, "dense eigensolver: kernel does not fit on an SM");
  const int want = (int)std::min<int64_t>(h->sm_count, ((int64_t)NP * N + 255) / 256);
  int grid = std::max(1, want);
  DFTFE_LAUNCH(jac::k_bar_init, 1, 1, 0, s, bar, h->wait_limit, (unsigned int)h->wait_missing);
  DFTFE_CHECK_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), s));
  DFTFE_LAUNCH(k_fro_norm_z, 1, 256, 0, s, A, N, anorm);
  int maxs = 60;
  void* args[] = {&A, &VT, &d, &N, &maxs, &anorm, &bar, &d_status};
  DFTFE_CHECK_CUDA(cudaLaunchCooperativeKernel((const void*)k_jacobi_z, dim3(grid), dim3(256), args, sh, s));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  DFTFE_LAUNCH(k_rank, nblk(N, 128), 128, 0, s, d, N, perm, evals);
  DFTFE_LAUNCH(k_phase_copy_z, N, 256, 0, s, VT, perm, N, Q);
}

// ----------------------------------------------------------------- residuals
// cw doubles per column: 1 (real) or 2 (complex, real and imaginary parts interleaved)
__global__ void k_resid_partial(const double* __restrict__ X, int64_t ldx, const double* __restrict__ W,
                                int64_t ldw, int64_t M, int ncol, const double* __restrict__ evals,
                                const double* __restrict__ mass, int kind, int64_t rows, int cw,
                                double* __restrict__ part) {
  const int64_t i0 = (int64_t)blockIdx.x * rows;
  const int64_t i1 = min(M, i0 + rows);
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
    const double th = evals[c];
    double num = 0.0, den = 0.0;
    for (int64_t i = i0; i < i1; ++i)
      for (int u = 0; u < cw; ++u) {
        const double x = X[i * ldx + c * cw + u];
        const double r = W[i * ldw + c * cw + u] - th * x;
        if (kind == 0) num = fma(r, r, num);
        else {
          const double m = mass[i];
          num = fma(m * r, r, num);
          den = fma(x / m, x, den);
        }
      }
    part[((int64_t)blockIdx.x * ncol + c) * 2] = num;
    part[((int64_t)blockIdx.x * ncol + c) * 2 + 1] = den;
  }
}

__global__ void k_resid_final(const double* __restrict__ part, int nchunk, int ncol, int kind,
                              double* __restrict__ resid) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncol) return;
  double num = 0.0, den = 0.0;
  for (int k = 0; k < nchunk; ++k) {
    num += part[((int64_t)k * ncol + c) * 2];
    den += part[((int64_t)k * ncol + c) * 2 + 1];
  }
  resid[c] = kind == 0 ? sqrt(num) : sqrt(num) / sqrt(den);
}

void residual_norms(dftfe_ham h, const double* X, int64_t ldx, const double* W, int64_t ldw, int64_t M,
                     int ncol, const double* evals, double* resid, int kind, int cw) {
  if (ncol <= 0) return;
  const int nchunk = (int)std::max<int64_t>(1, std::min<int64_t>(h->sm_count * 4, M / 64));
  const int64_t rows = (M + nchunk - 1) / nchunk;
  double* part = (double*)ws_get(h, "resid_part", sizeof(double) * 2 * (size_t)nchunk * ncol);
  DFTFE_LAUNCH(k_resid_partial, nchunk, 256, 0, h->stream, X, ldx, W, ldw, M, ncol, evals, h->d_mass,
               kind, rows, cw, part);
  DFTFE_LAUNCH(k_resid_final, nblk(ncol, 128), 128, 0, h->stream, part, nchunk, ncol, kind, resid);
}

// --------------------------------------------------------- random numbers
__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__global__ void k_random(double* out, int64_t n, uint64_t seed, int64_t offset) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const uint64_t idx = (uint64_t)(offset + t);
  const uint64_t z = splitmix_mix(seed + (idx + 1ULL) * 0x9E3779B97F4A7C15ULL);
  out[t] = (double)(z >> 11) * 0x1.0p-53 - 0.5;
}

void random_uniform(cudaStream_t s, double* out, int64_t n, uint64_t seed, int64_t offset) {
  if (n <= 0) return;
  DFTFE_LAUNCH(k_random, nblk(n), 256, 0, s, out, n, seed, offset);
}

// ------------------------------------------------------------------ Lanczos
constexpr int LZ_G = 512;
// part[v*G + b] = partial dot of V[v] (stride M) with w over block b's rows.
__global__ void __launch_bounds__(256) k_multidot_partial(const double* __restrict__ Vm, int nv,
                                                          const double* __restrict__ w, int64_t M,
                                                          double* __restrict__ part) {
  __shared__ double red[9];
  const int64_t rows = (M + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * rows, i1 = min(M, i0 + rows);
  for (int v = 0; v < nv; ++v) {
    const double* x = Vm + (int64_t)v * M;
    double s = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += 256) s = fma(x[i], w[i], s);
    s = block_sum<256>(s, red);
    if (threadIdx.x == 0) part[v * gridDim.x + blockIdx.x] = s;
  }
}

// out[v] = sum_b part[v*G + b] (fixed order); mode 1 stores sqrt.
__global__ void k_multidot_final(const double* part, int nv, int G, double* out, int mode) {
  const int v = threadIdx.x;
  if (v >= nv) return;
  double s = 0.0;
  for (int b = 0; b < G; ++b) s += part[v * G + b];
  out[v] = mode == 1 ? sqrt(s) : s;
}

// w = (w - a v) - b u   (a = *pa, b = *pb or 0)
__global__ void k_lz_three_term(double* w, const double* v, const double* u, const double* pa,
                                const double* pb, int64_t M) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= M) return;
  double x = w[i] - pa[0] * v[i];
  if (u) x = x - pb[0] * u[i];
  w[i] = x;
}

// w -= sum_v hcoef[v] V[v]
__global__ void k_lz_reorth(double* w, const double* Vm, int nv, const double* hcoef, int64_t M) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= M) return;
  double s = 0.0;
  for (int v = 0; v < nv; ++v) s = fma(hcoef[v], Vm[(int64_t)v * M + i], s);
  w[i] -= s;
}

// out = w / *pn (0 if the norm is 0)
__global__ void k_lz_scale(double* out, const double* w, const double* pn, int64_t M) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= M) return;
  const double n = pn[0];
  out[i] = n > 0.0 ? w[i] / n : 0.0;
}

__global__ void k_lz_tridiag(const double* alpha, const double* beta, int k, double* d, double* e, double* Z) {
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    d[i] = alpha[i];
    e[i] = i < k - 1 ? beta[i] : 0.0;
  }
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) Z[t] = (t / k == t % k) ? 1.0 : 0.0;
}

__global__ void k_lz_bound(const double* d, const double* Z, const double* beta, int k, double* out3) {
  if (threadIdx.x != 0) return;
  int imin = 0, imax = 0;
  for (int i = 1; i < k; ++i) {
    if (d[i] < d[imin]) imin = i;
    if (d[i] > d[imax]) imax = i;
  }
  out3[0] = d[imin];
  out3[1] = d[imax];
  // upper-bound estimator of Zhou and Saad: the largest Ritz value plus the norm of the last
  // Lanczos residual |beta_k|.  (theta_max + |beta_k| |s_k|, the residual of that Ritz pair
  // alone, undershoots when the top of the spectrum is clustered: measured on a periodic
  // 27-cell p = 4 box, 30.21 against lambda_max = 30.54.)
  (void)Z;
  out3[2] = d[imax] + fabs(beta[k - 1]);
}

void lanczos(dftfe_ham h, int k, const double* v0, uint64_t seed, double* out3, bool cplx) {
  auto* m = h->mesh;
  // vector length: M, or 2M for the real view of a complex vector (the dot products below are
  // then those of the real 2M x 2M form of H~^k, which has H~^k's spectrum, each value twice)
  const int64_t M = cplx ? 2 * m->M : m->M;
  cudaStream_t s = h->stream;
  double* Vm = (double*)ws_get(h, "lz_V", sizeof(double) * (size_t)(k + 1) * M);
  double* w = (double*)ws_get(h, "lz_w", sizeof(double) * (size_t)M);
  double* sc = (double*)ws_get(h, "lz_scal", sizeof(double) * (size_t)(4 * k + 8 + k * k + 2 * k));
  double* part = (double*)ws_get(h, "lz_part", sizeof(double) * (size_t)(k + 1) * LZ_G);
  int* st = (int*)ws_get(h, "lz_status", sizeof(int));
  double* alpha = sc;
  double* beta = sc + k;
  double* hco = sc + 2 * k;        // k + 1
  double* nrm = sc + 3 * k + 1;    // 1
  double* d = sc + 3 * k + 2;      // k
  double* e = d + k;               // k
  double* Z = e + k;               // k*k
  double* d_out = Z + k * k;       // 3
  if (v0) DFTFE_CHECK_CUDA(cudaMemcpyAsync(w, v0, sizeof(double) * M, cudaMemcpyDeviceToDevice, s));
  else random_uniform(s, w, M, seed, 0);
  DFTFE_LAUNCH(k_multidot_partial, LZ_G, 256, 0, s, w, 1, w, M, part);
  DFTFE_LAUNCH(k_multidot_final, 1, 32, 0, s, part, 1, LZ_G, nrm, 1);
  DFTFE_LAUNCH(k_lz_scale, nblk(M), 256, 0, s, Vm, w, nrm, M);
  for (int j = 0; j < k; ++j) {
    double* vj = Vm + (int64_t)j * M;
    if (cplx) apply_combo_z(h, vj, 1, nullptr, 0, w, 1, 1, 1.0, 0.0, 0.0);
    else apply_combo(h, vj, 1, nullptr, 0, w, 1, 1, 1.0, 0.0, 0.0);
    DFTFE_LAUNCH(k_multidot_partial, LZ_G, 256, 0, s, vj, 1, w, M, part);
    DFTFE_LAUNCH(k_multidot_final, 1, 32, 0, s, part, 1, LZ_G, alpha + j, 0);
    DFTFE_LAUNCH(k_lz_three_term, nblk(M), 256, 0, s, w, vj, j > 0 ? vj - M : nullptr, alpha + j,
                 j > 0 ? beta + j - 1 : alpha + j, M);
    for (int rep = 0; rep < 2; ++rep) {
      DFTFE_LAUNCH(k_multidot_partial, LZ_G, 256, 0, s, Vm, j + 1, w, M, part);
      DFTFE_LAUNCH(k_multidot_final, 1, 256, 0, s, part, j + 1, LZ_G, hco, 0);
      DFTFE_LAUNCH(k_lz_reorth, nblk(M), 256, 0, s, w, Vm, j + 1, hco, M);
    }
    DFTFE_LAUNCH(k_multidot_partial, LZ_G, 256, 0, s, w, 1, w, M, part);
    DFTFE_LAUNCH(k_multidot_final, 1, 32, 0, s, part, 1, LZ_G, beta + j, 1);
    DFTFE_LAUNCH(k_lz_scale, nblk(M), 256, 0, s, Vm + (int64_t)(j + 1) * M, w, beta + j, M);
  }
  DFTFE_LAUNCH(k_lz_tridiag, 1, 256, 0, s, alpha, beta, k, d, e, Z);
  tridiag_ql(s, d, e, Z, k, st);
  DFTFE_LAUNCH(k_lz_bound, 1, 32, 0, s, d, Z, beta, k, d_out);
  int hst = 0;
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(out3, d_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(&hst, st, sizeof(int), cudaMemcpyDeviceToHost, s));
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(s));
  if (hst) throw Error(DFTFE_ERR_NOCONV, "Lanczos tridiagonal eigensolve did not converge");
}

}  // namespace dftfe

// ------------------------------------------------ stream-only launchers
// Launch the kernels above with caller-provided scratch and a plain stream (no handle,
// no workspace).  Used by the allocation-free CholGS entry point.
namespace dftfe {

void gram_partial_launch(cudaStream_t s, const double* A, int64_t lda, const double* B, int64_t ldb,
                         int64_t M, int N, int nsplit, int ntiles, double* part) {
  const int64_t rows = (M + nsplit - 1) / nsplit;
  DFTFE_LAUNCH(k_gram_partial, dim3(ntiles, nsplit), 256, 0, s, A, lda, B, ldb, M, N, rows, part);
}

void gram_reduce_launch(cudaStream_t s, const double* part, int nsplit, int N, double* C) {
  DFTFE_LAUNCH(k_gram_reduce, nblk((int64_t)N * N), 256, 0, s, part, nsplit, N, C);
}

template <int R, int CPT>
static void rotate_launch_t(cudaStream_t s, double* X, int64_t ld, int64_t M, int N, const double* Z,
                            bool upper) {
  DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_rotate<R, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        200 * 1024));
  const size_t sh = (size_t)R * N * sizeof(double);
  DFTFE_LAUNCH((k_rotate<R, CPT>), (unsigned)((M + R - 1) / R), 256, sh, s, X, ld, M, N, Z, upper ? 1 : 0,
               (const int*)nullptr);
}

void rotate_launch(cudaStream_t s, double* X, int64_t ld, int64_t M, int N, const double* Z, bool upper) {
  if (M == 0 || N == 0) return;
  if (N <= 256) rotate_launch_t<32, 1>(s, X, ld, M, N, Z, upper);
  else if (N <= 512) rotate_launch_t<32, 2>(s, X, ld, M, N, Z, upper);
  else throw Error(DFTFE_ERR_ARG, "rotate_launch: at most 512 columns");
}

}  // namespace dftfe
