// Spectrum splitting and electron density (Alg. 2 step 3a, Alg. 3).
//
//   Psi_fr = Psi_o Q'_fr        top N_fr Ritz vectors of the orthonormal basis (RRGEP-ST-F)
//   mu from 2 (N_oc + sum_fr f(eps_i, mu)) = N_e, f Fermi-Dirac (bisection, one thread)
//   rho(x_q) = 2 [ sum_i (n^T psi^_o,i)^2 + sum_fr (f_k - 1) (n^T psi^_fr,k)^2 ],
//              psi^ = M^-1/2 psi~, n = basis values at the quadrature point (Alg. 3)
#include "internal.h"

#include <cmath>

namespace dftfe {

static unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// out[r][j] = sum_k X[r][k] Z[k][j], j < nout; the row panel of X is staged in shared
// memory, thread t owns output columns t + 256 c.
template <int R, int CPT>
__global__ void __launch_bounds__(256) k_rotate_out(const double* __restrict__ X, int64_t ldx, int64_t M, int N,
                                                    const double* __restrict__ Z, int64_t ldz, int nout,
                                                    double* __restrict__ out, int64_t ldo) {
  extern __shared__ double xs[];  // R x N
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const int rows = (int)min((int64_t)R, M - r0);
  for (int t = threadIdx.x; t < R * N; t += 256) {
    const int r = t / N, k = t % N;
    xs[t] = r < rows ? X[(r0 + r) * ldx + k] : 0.0;
  }
  __syncthreads();
  double acc[R][CPT];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[r][c] = 0.0;
  for (int k = 0; k < N; ++k) {
    double z[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int j = threadIdx.x + 256 * c;
      z[c] = j < nout ? __ldg(Z + (int64_t)k * ldz + j) : 0.0;
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
      if (j < nout) out[(r0 + r) * ldo + j] = acc[r][c];
    }
  }
}

template <int R, int CPT>
static void launch_rotate_out(dftfe_ham h, const double* X, int64_t ldx, int64_t M, int N, const double* Z,
                              int64_t ldz, int nout, double* out, int64_t ldo) {
  static bool attr = false;
  if (!attr) {
    DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_rotate_out<R, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          200 * 1024));
    attr = true;
  }
  ProfScope ps(h, "rotate_split");
  DFTFE_LAUNCH((k_rotate_out<R, CPT>), (unsigned)((M + R - 1) / R), 256, (size_t)R * N * sizeof(double), h->stream,
               X, ldx, M, N, Z, ldz, nout, out, ldo);
}

static void rotate_out(dftfe_ham h, const double* X, int64_t ldx, int64_t M, int N, const double* Z, int64_t ldz,
                       int nout, double* out, int64_t ldo) {
  if (M == 0 || nout == 0) return;
  if (nout > 512) throw Error(DFTFE_ERR_ARG, "at most 512 split states");
  // rows per panel so that the panel stays within 128 KB of shared memory
  if (N <= 512) {
    if (nout <= 256) launch_rotate_out<32, 1>(h, X, ldx, M, N, Z, ldz, nout, out, ldo);
    else launch_rotate_out<32, 2>(h, X, ldx, M, N, Z, ldz, nout, out, ldo);
  } else if (N <= 1024) {
    if (nout <= 256) launch_rotate_out<16, 1>(h, X, ldx, M, N, Z, ldz, nout, out, ldo);
    else launch_rotate_out<16, 2>(h, X, ldx, M, N, Z, ldz, nout, out, ldo);
  } else {
    if (nout <= 256) launch_rotate_out<8, 1>(h, X, ldx, M, N, Z, ldz, nout, out, ldo);
    else launch_rotate_out<8, 2>(h, X, ldx, M, N, Z, ldz, nout, out, ldo);
  }
}

// ---------------------------------------------------------------- Fermi level
__device__ __forceinline__ double fermi_dirac(double eps, double mu, double kT) {
  const double x = (eps - mu) / kT;
  if (x > 0.0) {
    const double e = exp(-x);
    return e / (1.0 + e);
  }
  return 1.0 / (1.0 + exp(x));
}

// one thread: bisection on the electron count (increasing in mu), 200 halvings
__global__ void k_fermi(const double* __restrict__ eps, int nfr, int n_oc, double n_elec, double kT,
                        double* __restrict__ f, double* __restrict__ mu_out, int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (!(2.0 * n_oc < n_elec && n_elec < 2.0 * (n_oc + nfr))) {
    *status = (int)DFTFE_ERR_ARG;
    return;
  }
  double lo = eps[0], hi = eps[0];
  for (int i = 1; i < nfr; ++i) {
    lo = fmin(lo, eps[i]);
    hi = fmax(hi, eps[i]);
  }
  lo -= 50.0 * kT;
  hi += 50.0 * kT;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    double s = 0.0;
    for (int i = 0; i < nfr; ++i) s += fermi_dirac(eps[i], mid, kT);
    if (2.0 * (n_oc + s) < n_elec) lo = mid;
    else hi = mid;
  }
  const double mu = 0.5 * (lo + hi);
  for (int i = 0; i < nfr; ++i) f[i] = fermi_dirac(eps[i], mu, kT);
  *mu_out = mu;
  *status = 0;
}

// ---------------------------------------------------------------- density
// One CTA per cell.  Columns of [Xo | Xfr] are processed 32 at a time: the cell's rows are
// gathered into shared memory scaled by M^-1/2, each warp interpolates 8 quadrature points
// at a time (rows of Nq, warp-uniform loads), squares, weights (1 for Psi_o, f - 1 for
// Psi_fr) and reduces across the lanes; quadrature point q is always owned by the same
// warp, so the per-point sums are race-free and deterministic.
constexpr int DN_ROWS = 8;
__global__ void __launch_bounds__(256, 2) k_density(const double* __restrict__ Nq, const int32_t* __restrict__ map,
                                                    const double* __restrict__ minvsqrt, int nc, int nq,
                                                    const double* __restrict__ Xo, int64_t ldo, int ncol,
                                                    const double* __restrict__ Xfr, int64_t ldf, int nfr,
                                                    const double* __restrict__ f_fr, double* __restrict__ rho) {
  extern __shared__ double sm[];
  double* xs = sm;                    // nc x 32
  double* racc = xs + nc * 32;        // nq
  double* dm = racc + nq;             // nc
  int32_t* gm = (int32_t*)(dm + nc);  // nc
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t cell = blockIdx.x;
  for (int k = threadIdx.x; k < nc; k += 256) {
    gm[k] = map[cell * nc + k];
    dm[k] = minvsqrt[gm[k]];
  }
  for (int q = threadIdx.x; q < nq; q += 256) racc[q] = 0.0;
  __syncthreads();
  const int T = ncol + nfr;
  for (int c0 = 0; c0 < T; c0 += 32) {
    const int col = c0 + lane;
    double w = 0.0;
    if (col < ncol) w = 1.0;
    else if (col < T) w = f_fr[col - ncol] - 1.0;
    for (int k = warp; k < nc; k += 8) {
      double v = 0.0;
      if (col < ncol) v = Xo[(int64_t)gm[k] * ldo + col];
      else if (col < T) v = Xfr[(int64_t)gm[k] * ldf + (col - ncol)];
      xs[k * 32 + lane] = dm[k] * v;
    }
    __syncthreads();
    for (int q0 = warp * DN_ROWS; q0 < nq; q0 += 8 * DN_ROWS) {
      const int nr = min(DN_ROWS, nq - q0);
      double acc[DN_ROWS];
#pragma unroll
      for (int i = 0; i < DN_ROWS; ++i) acc[i] = 0.0;
      const double* Nr = Nq + (int64_t)q0 * nc;
      for (int k = 0; k < nc; ++k) {
        const double x = xs[k * 32 + lane];
#pragma unroll
        for (int i = 0; i < DN_ROWS; ++i)
          if (i < nr) acc[i] = fma(__ldg(Nr + (int64_t)i * nc + k), x, acc[i]);
      }
#pragma unroll
      for (int i = 0; i < DN_ROWS; ++i) {
        double v = w * acc[i] * acc[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0 && i < nr) racc[q0 + i] += 2.0 * v;
      }
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < nq; q += 256) rho[cell * nq + q] = racc[q];
}

}  // namespace dftfe

using namespace dftfe;

extern "C" dftfe_status dftfe_rayleigh_ritz_split(dftfe_ham h, const double* X, int64_t ld, int ncol, int nfr,
                                                  double* evals, double* Xfr, int64_t ldfr, dftfe_precision prec) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && X && evals && Xfr, "null argument");
  DFTFE_REQUIRE(ncol >= 1 && ncol <= 2048 && ld >= ncol, "bad ncol / ld");
  DFTFE_REQUIRE(nfr >= 1 && nfr <= ncol && nfr <= 512 && ldfr >= nfr, "bad nfr / ldfr");
  DFTFE_REQUIRE(prec == DFTFE_FP64 || prec == DFTFE_MIXED_BF16X3 || prec == DFTFE_MIXED_TF32X3,
                "unknown precision");
  if (!loc(h)->has_potential) throw Error(DFTFE_ERR_STATE, "set the potential first");
  auto* m = h->mesh;
  const int N = ncol;
  const bool mixed = prec != DFTFE_FP64;
  double* W = (double*)ws_get(h, "W", sizeof(double) * (size_t)m->M * N);
  if (mixed) apply_w(h, X, ld, W, N, N);
  else apply_combo(h, X, ld, nullptr, 0, W, N, N, 1.0, 0.0, 0.0);
  double* Hh = (double*)ws_get(h, "Hhat", sizeof(double) * (size_t)N * N);
  double* Q = (double*)ws_get(h, "Q", sizeof(double) * (size_t)N * N);
  int* st = (int*)ws_get(h, "status", sizeof(int) * 4);
  if (mixed) {
    gram_lower_mixed(h, X, ld, W, N, m->M, N, Hh);
  } else {
    const int nsplit = gram_nsplit(h, m->M, N);
    double* part = (double*)ws_get(h, "gram_part", sizeof(double) * (size_t)nsplit * N * N);
    gram_lower(h, X, ld, W, N, m->M, N, Hh, part, nsplit);
  }
  syevd(h, Hh, N, evals, Q, st);
  int s = 0;
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(&s, st, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  if (s == DFTFE_ERR_NOCONV) throw Error(DFTFE_ERR_NOCONV, "subspace eigensolver did not converge");
  if (s != 0) throw Error((dftfe_status)s, "subspace eigensolver: a bounded grid wait timed out");
  // Psi_fr = X Q'_fr: the last nfr columns of Q (row stride N)
  rotate_out(h, X, ld, m->M, N, Q + (N - nfr), N, nfr, Xfr, ldfr);
  ABI_END
}

extern "C" dftfe_status dftfe_fermi_level(const double* evals_fr, int nfr, int n_oc, double n_elec, double kT,
                                          double* f_fr, double* mu, void* stream) {
  ABI_BEGIN
  DFTFE_REQUIRE(evals_fr && f_fr && mu, "null argument");
  DFTFE_REQUIRE(nfr >= 1 && n_oc >= 0 && kT > 0.0 && std::isfinite(n_elec), "bad sizes / temperature");
  DFTFE_REQUIRE(2.0 * n_oc < n_elec && n_elec < 2.0 * (n_oc + nfr),
                "the electron count must fall inside the fractionally occupied window");
  cudaStream_t s = (cudaStream_t)stream;
  double* d_mu = nullptr;
  int* d_st = nullptr;
  // two scalars of scratch: allocated per call (the call is outside the pass's hot loop)
  DFTFE_CHECK_CUDA(cudaMallocAsync((void**)&d_mu, sizeof(double) + sizeof(int) * 2, s));
  d_st = (int*)(d_mu + 1);
  DFTFE_LAUNCH(k_fermi, 1, 32, 0, s, evals_fr, nfr, n_oc, n_elec, kT, f_fr, d_mu, d_st);
  double hmu = 0.0;
  int hst = 0;
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(&hmu, d_mu, sizeof(double), cudaMemcpyDeviceToHost, s));
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(&hst, d_st, sizeof(int), cudaMemcpyDeviceToHost, s));
  DFTFE_CHECK_CUDA(cudaFreeAsync(d_mu, s));
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(s));
  if (hst) throw Error(DFTFE_ERR_ARG, "the electron count must fall inside the fractionally occupied window");
  *mu = hmu;
  ABI_END
}

extern "C" dftfe_status dftfe_density(dftfe_ham h, const double* Xo, int64_t ldo, int ncol, const double* Xfr,
                                      int64_t ldfr, int nfr, const double* f_fr, double* rho) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && Xo && rho, "null argument");
  DFTFE_REQUIRE(ncol >= 0 && ldo >= ncol && nfr >= 0, "bad sizes");
  DFTFE_REQUIRE(nfr == 0 || (Xfr && f_fr && ldfr >= nfr), "null split-state inputs");
  auto* m = h->mesh;
  static bool attr = false;
  if (!attr) {
    DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_density, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  const size_t sh = (size_t)m->nc * 32 * sizeof(double) + (size_t)m->nq * sizeof(double) +
                    (size_t)m->nc * (sizeof(double) + sizeof(int32_t));
  ProfScope ps(h, "density");
  DFTFE_LAUNCH(k_density, (unsigned)m->Nc, 256, sh, h->stream, h->d_Nq, h->d_map, h->d_minvsqrt, m->nc, m->nq, Xo,
               ldo, ncol, Xfr, ldfr, nfr, f_fr, rho);
  ABI_END
}
