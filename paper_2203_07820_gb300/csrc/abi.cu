// Orchestration of the pass steps behind the C ABI: Lanczos bounds (a7),
// Cholesky-Gram-Schmidt (a8, a9), Rayleigh-Ritz (a10-a12), residuals (a13), the pass
// (Sec. 3.1-3.2 with Alg. 2 read as orthonormalise-first), random numbers, profiling.
#include "internal.h"

#include <cmath>
#include <string>

namespace dftfe {

static int read_status(dftfe_ham h, int* d_status) {
  int st = 0;
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  return st;
}

static void cholgs_impl(dftfe_ham h, double* X, int64_t ld, int ncol, bool mixed) {
  auto* m = h->mesh;
  const int N = ncol;
  double* S = (double*)ws_get(h, "S", sizeof(double) * (size_t)N * N);
  double* Z = (double*)ws_get(h, "Zinv", sizeof(double) * (size_t)N * N);
  // a deferred pass keeps the status on the device (read at its end); the rotation below
  // then skips its work if the factorisation failed
  int* st = h->deferred ? h->d_pass : (int*)ws_get(h, "status", sizeof(int) * 4);
  if (mixed) {
    gram_lower_mixed(h, X, ld, X, ld, m->M, N, S);
  } else {
    const int nsplit = gram_nsplit(h, m->M, N);
    double* part = (double*)ws_get(h, "gram_part", sizeof(double) * (size_t)nsplit * N * N);
    gram_lower(h, X, ld, X, ld, m->M, N, S, part, nsplit);
  }
  cholesky_blocked(h, S, N, st);
  if (!h->deferred && read_status(h, st) == DFTFE_ERR_NOT_SPD)
    throw Error(DFTFE_ERR_NOT_SPD, "overlap matrix is not positive definite");
  tri_inverse_blocked(h, S, Z, N);
  if (mixed) rotate_inplace_mixed(h, X, ld, m->M, N, Z, true);
  else rotate_inplace(h, X, ld, m->M, N, Z, true);
}

static void rr_impl(dftfe_ham h, double* X, int64_t ld, int ncol, double* evals, double* W, int64_t ldw,
                    dftfe_precision prec) {
  auto* m = h->mesh;
  const int N = ncol;
  const bool mixed = prec != DFTFE_FP64;
  // W = H~X must be FP64-accurate in every precision (split-precision cell products here
  // move the Ritz values by 1e-6 to 2e-6 Ha, the size of the mixed tolerance): FP64 in
  // the FP64 pass, float pairs (about 44 bits) on the FP32 pipes in a mixed pass
  if (mixed) apply_w(h, X, ld, W, ldw, N);
  else apply_combo(h, X, ld, nullptr, 0, W, ldw, N, 1.0, 0.0, 0.0);
  double* Hh = (double*)ws_get(h, "Hhat", sizeof(double) * (size_t)N * N);
  double* Q = (double*)ws_get(h, "Q", sizeof(double) * (size_t)N * N);
  int* st = h->deferred ? h->d_pass + 1 : (int*)ws_get(h, "status", sizeof(int) * 4);
  if (mixed) {
    gram_lower_mixed(h, X, ld, W, ldw, m->M, N, Hh);
  } else {
    const int nsplit = gram_nsplit(h, m->M, N);
    double* part = (double*)ws_get(h, "gram_part", sizeof(double) * (size_t)nsplit * N * N);
    gram_lower(h, X, ld, W, ldw, m->M, N, Hh, part, nsplit);
  }
  syevd(h, Hh, N, evals, Q, st);
  if (!h->deferred) {
    const int s = read_status(h, st);
    if (s == DFTFE_ERR_NOCONV) throw Error(DFTFE_ERR_NOCONV, "subspace eigensolver did not converge");
    if (s != 0) throw Error((dftfe_status)s, "subspace eigensolver: a bounded grid wait timed out");
  }
  if (mixed) {
    rotate_inplace_mixed(h, X, ld, m->M, N, Q, false);
    rotate_inplace_mixed(h, W, ldw, m->M, N, Q, false);
  } else {
    rotate_inplace(h, X, ld, m->M, N, Q, false);
    rotate_inplace(h, W, ldw, m->M, N, Q, false);
  }
}

// The pass after the filter (Alg. 2 read as orthonormalise-first): CholGS, Rayleigh-Ritz,
// residuals, bounds update a <- theta_N, a0 <- theta_1 (a0 kept NaN for the unscaled filter).
void chfsi_pass_tail(dftfe_ham h, double* X, int64_t ld, int ncol, dftfe_bounds* inout, double* evals,
                     double* resid, dftfe_precision prec) {
  auto* m = h->mesh;
  {
    ProfScope ps(h, "pass_cholgs");
    cholgs_impl(h, X, ld, ncol, prec != DFTFE_FP64);
  }
  double* W = (double*)ws_get(h, "W", sizeof(double) * (size_t)m->M * ncol);
  {
    ProfScope ps(h, "pass_rr");
    rr_impl(h, X, ld, ncol, evals, W, ncol, prec);
  }
  residual_norms(h, X, ld, W, ncol, m->M, ncol, evals, resid, 0);
  if (h->deferred) {
    // statuses and the Ritz-value ends to pinned host memory; the caller synchronises once
    double* ends = (double*)((char*)h->h_pass + 16);
    DFTFE_CHECK_CUDA(cudaMemcpyAsync(h->h_pass, h->d_pass, 4 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    DFTFE_CHECK_CUDA(cudaMemcpyAsync(&ends[0], evals, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    DFTFE_CHECK_CUDA(cudaMemcpyAsync(&ends[1], evals + ncol - 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return;
  }
  double ends[2];
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(&ends[0], evals, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(&ends[1], evals + ncol - 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  inout->a = ends[1];
  if (!std::isnan(inout->a0)) inout->a0 = ends[0];
}

// The whole pass as one enqueued region (filter, CholGS, Rayleigh-Ritz, residuals) with the
// statuses deferred: one CUDA graph per shape when the ham uses graphs, one host
// synchronisation at the end either way.  Errors are reported after the region in the order
// the plain pass would meet them; a failed factorisation or eigensolve leaves X as filtered.
static void chfsi_pass_graphed(dftfe_ham h, double* X, int64_t ld, int ncol, int block, int degree,
                               dftfe_bounds* inout, double* evals, double* resid, dftfe_precision prec) {
  if (!h->d_pass) h->d_pass = (int*)ws_get(h, "pass_status", sizeof(int) * 4);
  if (!h->h_pass) DFTFE_CHECK_CUDA(cudaHostAlloc(&h->h_pass, 64, cudaHostAllocDefault));
  const dftfe_bounds bnd = *inout;
  const std::string key = "wholepass/" + std::to_string((int)prec) + "/" + std::to_string(ncol) + "/" +
                          std::to_string(block) + "/" + std::to_string(degree) + "/" + std::to_string((int64_t)ld);
  dftfe_bounds out = bnd;
  h->deferred = true;
  try {
    run_region(h, key, [&]() {
      DFTFE_CHECK_CUDA(cudaMemsetAsync(h->d_pass, 0, sizeof(int) * 4, h->stream));
      for (int j0 = 0; j0 < ncol; j0 += block) {
        const int nb = std::min(block, ncol - j0);
        if (prec == DFTFE_FP64) chebyshev_filter(h, X + j0, ld, nb, degree, bnd);
        else chebyshev_filter_mixed(h, X + j0, ld, nb, degree, bnd, prec == DFTFE_MIXED_TF32X3, h->d_pass + 2);
      }
      chfsi_pass_tail(h, X, ld, ncol, &out, evals, resid, prec);
    });
  } catch (...) {
    h->deferred = false;
    throw;
  }
  h->deferred = false;
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  const int* st = (const int*)h->h_pass;
  const double* ends = (const double*)((const char*)h->h_pass + 16);
  if (st[0] == DFTFE_ERR_NOT_SPD) throw Error(DFTFE_ERR_NOT_SPD, "overlap matrix is not positive definite");
  if (st[2]) throw Error(DFTFE_ERR_TIMEOUT, "tensor-core kernel: a bounded wait timed out");
  if (st[1] == DFTFE_ERR_NOCONV) throw Error(DFTFE_ERR_NOCONV, "subspace eigensolver did not converge");
  if (st[1] != 0) throw Error((dftfe_status)st[1], "subspace eigensolver: a bounded grid wait timed out");
  inout->a = ends[1];
  if (!std::isnan(inout->a0)) inout->a0 = ends[0];
}

}  // namespace dftfe

using namespace dftfe;

extern "C" dftfe_status dftfe_random_uniform(double* out, int64_t n, uint64_t seed, int64_t offset,
                                             void* stream) {
  ABI_BEGIN
  DFTFE_REQUIRE(n >= 0 && offset >= 0, "negative size");
  DFTFE_REQUIRE(out || n == 0, "null output");
  random_uniform((cudaStream_t)stream, out, n, seed, offset);
  ABI_END
}

extern "C" dftfe_status dftfe_lanczos(dftfe_ham h, int k, const double* v0, uint64_t seed, double* out3) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && out3, "null argument");
  DFTFE_REQUIRE(k >= 1 && k <= 200, "k must be in 1..200");
  if (!loc(h)->has_potential) throw Error(DFTFE_ERR_STATE, "set the potential first");
  lanczos(h, k, v0, seed, out3);
  ABI_END
}

extern "C" dftfe_status dftfe_spectrum_bounds(dftfe_ham h, int k, uint64_t seed, int nstates,
                                              dftfe_bounds* out) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && out, "null argument");
  DFTFE_REQUIRE(k >= 1 && k <= 200 && nstates >= 1, "bad k / nstates");
  if (!loc(h)->has_potential) throw Error(DFTFE_ERR_STATE, "set the potential first");
  double r[3];
  lanczos(h, k, nullptr, seed, r);
  const double frac = std::max(4.0 * nstates / (double)h->mesh->M, 0.05);
  out->a0 = r[0];
  out->b = r[2];
  out->a = r[0] + (r[2] - r[0]) * frac;
  ABI_END
}

extern "C" dftfe_status dftfe_cholgs(dftfe_ham h, double* X, int64_t ld, int ncol, dftfe_precision prec) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && X, "null argument");
  DFTFE_REQUIRE(ncol >= 1 && ncol <= 2048 && ld >= ncol, "bad ncol / ld");
  DFTFE_REQUIRE(ncol <= h->mesh->M, "more columns than DoFs");
  DFTFE_REQUIRE(prec == DFTFE_FP64 || prec == DFTFE_MIXED_BF16X3 || prec == DFTFE_MIXED_TF32X3, "unknown precision");
  cholgs_impl(h, X, ld, ncol, prec != DFTFE_FP64);
  ABI_END
}

extern "C" dftfe_status dftfe_rayleigh_ritz(dftfe_ham h, double* X, int64_t ld, int ncol, double* evals,
                                            double* HX, int64_t ldhx, dftfe_precision prec) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && X && evals, "null argument");
  DFTFE_REQUIRE(ncol >= 1 && ncol <= 2048 && ld >= ncol, "bad ncol / ld");
  DFTFE_REQUIRE(!HX || ldhx >= ncol, "bad ldhx");
  DFTFE_REQUIRE(prec == DFTFE_FP64 || prec == DFTFE_MIXED_BF16X3 || prec == DFTFE_MIXED_TF32X3, "unknown precision");
  if (!loc(h)->has_potential) throw Error(DFTFE_ERR_STATE, "set the potential first");
  double* W = HX;
  int64_t ldw = ldhx;
  if (!W) {
    W = (double*)ws_get(h, "W", sizeof(double) * (size_t)h->mesh->M * ncol);
    ldw = ncol;
  }
  rr_impl(h, X, ld, ncol, evals, W, ldw, prec);
  ABI_END
}

extern "C" dftfe_status dftfe_residuals(dftfe_ham h, const double* X, const double* HX, int64_t ld, int ncol,
                                        const double* evals, double* resid, int kind) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && X && HX && evals && resid, "null argument");
  DFTFE_REQUIRE(ncol >= 1 && ld >= ncol, "bad ncol / ld");
  DFTFE_REQUIRE(kind == 0 || kind == 1, "kind must be 0 or 1");
  residual_norms(h, X, ld, HX, ld, h->mesh->M, ncol, evals, resid, kind);
  ABI_END
}

extern "C" dftfe_status dftfe_chfsi_pass(dftfe_ham h, double* X, int64_t ld, int ncol, int block, int degree,
                                         dftfe_bounds* inout, double* evals, double* resid,
                                         dftfe_precision prec) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && X && inout && evals && resid, "null argument");
  DFTFE_REQUIRE(ncol >= 1 && ncol <= 2048 && ld >= ncol && block >= 1 && degree >= 0, "bad sizes");
  DFTFE_REQUIRE(ncol <= h->mesh->M, "more columns than DoFs");
  DFTFE_REQUIRE(inout->b > inout->a, "need b > a");
  DFTFE_REQUIRE(std::isnan(inout->a0) || inout->a0 < inout->a, "need a0 < a for the scaled filter");
  DFTFE_REQUIRE(prec == DFTFE_FP64 || prec == DFTFE_MIXED_BF16X3 || prec == DFTFE_MIXED_TF32X3,
                "unknown precision");
  if (!loc(h)->has_potential) throw Error(DFTFE_ERR_STATE, "set the potential first");
  if (h->use_graphs) {
    chfsi_pass_graphed(h, X, ld, ncol, block, degree, inout, evals, resid, prec);
    return DFTFE_OK;
  }
  {
    ProfScope ps(h, "pass_filter");
    // the mixed cell kernel's timeout flag is zeroed before the filter and read after it, so
    // the filter phase has no host read and can run as one CUDA graph
    int* err = nullptr;
    if (prec != DFTFE_FP64) {
      err = (int*)ws_get(h, "mx_err", sizeof(int));
      DFTFE_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), h->stream));
    }
    const dftfe_bounds bnd = *inout;
    const std::string key = "pass/" + std::to_string((int)prec) + "/" + std::to_string(ncol) + "/" +
                            std::to_string(block) + "/" + std::to_string(degree);
    run_region(h, key, [&]() {
      for (int j0 = 0; j0 < ncol; j0 += block) {
        const int nb = std::min(block, ncol - j0);
        if (prec == DFTFE_FP64) chebyshev_filter(h, X + j0, ld, nb, degree, bnd);
        else chebyshev_filter_mixed(h, X + j0, ld, nb, degree, bnd, prec == DFTFE_MIXED_TF32X3, err);
      }
    });
    if (err) {
      int herr = 0;
      DFTFE_CHECK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
      DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
      if (herr) throw Error(DFTFE_ERR_TIMEOUT, "mixed cell kernel: a bounded wait timed out");
    }
  }
  chfsi_pass_tail(h, X, ld, ncol, inout, evals, resid, prec);
  ABI_END
}

extern "C" dftfe_status dftfe_ham_set_wait_test(dftfe_ham h, int64_t spin_limit, int withhold_arrival) {
  ABI_BEGIN
  DFTFE_REQUIRE(h, "null ham");
  DFTFE_REQUIRE(spin_limit >= 0 && (withhold_arrival == 0 || withhold_arrival == 1), "bad wait-test arguments");
  h->wait_limit = (long long)spin_limit;
  h->wait_missing = withhold_arrival;
  ABI_END
}

extern "C" dftfe_status dftfe_profile_enable(dftfe_ham h, int enable) {
  ABI_BEGIN
  DFTFE_REQUIRE(h, "null ham");
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  for (auto& kv : h->timers) {
    kv.second.used = 0;
    kv.second.launches = 0;
    kv.second.total_ms = 0;
  }
  h->profiling = enable != 0;
  ABI_END
}

extern "C" dftfe_status dftfe_profile_query(dftfe_ham h, const char* kernel, double* total_ms,
                                            int64_t* launches) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && kernel && total_ms && launches, "null argument");
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  auto it = h->timers.find(kernel);
  double ms = 0.0;
  int64_t n = 0;
  if (it != h->timers.end()) {
    for (size_t i = 0; i < it->second.used; ++i) {
      float t = 0.f;
      DFTFE_CHECK_CUDA(cudaEventElapsedTime(&t, it->second.events[i].first, it->second.events[i].second));
      ms += t;
    }
    n = it->second.launches;
  }
  *total_ms = ms;
  *launches = n;
  ABI_END
}
