// Allocation-free Cholesky-Gram-Schmidt.
//
// Some callers cannot call cudaMalloc at the point where they orthonormalise a
// block: code running inside a pre-sized memory pool that must not grow, a host
// framework that forbids device allocations in its step function, or a process
// whose allocator is owned by another runtime.  dftfe_cholgs_noalloc gives them the
// same result as dftfe_cholgs without a handle and without any allocation: its
// scratch (the split-K partial overlaps, S/L, L^-T and a status word) is one
// file-scope device array of fixed size, which every GPU that loads this library
// holds until the process exits.
#include "internal.h"

#include <algorithm>
#include <mutex>

namespace dftfe {
void gram_partial_launch(cudaStream_t s, const double* A, int64_t lda, const double* B, int64_t ldb,
                         int64_t M, int N, int nsplit, int ntiles, double* part);
void gram_reduce_launch(cudaStream_t s, const double* part, int nsplit, int N, double* C);
void rotate_launch(cudaStream_t s, double* X, int64_t ld, int64_t M, int N, const double* Z, bool upper);
}  // namespace dftfe

namespace {

constexpr int kMaxCols = DFTFE_NOALLOC_MAX_COLS;              // 512
constexpr int kTileCols = 64;                                 // Gram tile width
constexpr int kMaxTiles1D = (kMaxCols + kTileCols - 1) / kTileCols;
constexpr int kMaxTiles = kMaxTiles1D * (kMaxTiles1D + 1) / 2;
// scratch = 8 partial overlaps + S/L + L^-T at the largest size, plus one status word
constexpr size_t kScratchDoubles = (size_t)10 * kMaxCols * kMaxCols + 32;

static __device__ __align__(256) double g_scratch[kScratchDoubles];


struct DeviceSetup {
  bool ready = false;
  double* scratch = nullptr;   // device address of g_scratch on this device
  int sm_count = 0;
};
constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Once per device, with that device current: resolve the arrays' device addresses (host code
// may not use the symbols themselves as pointers) and the SM count.  Nothing is copied.
const DeviceSetup& setup_current_device() {
  int dev = 0;
  DFTFE_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) throw dftfe::Error(DFTFE_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& d = g_setup[dev];
  if (d.ready) return d;
  DFTFE_CHECK_CUDA(cudaGetSymbolAddress((void**)&d.scratch, g_scratch));
  DFTFE_CHECK_CUDA(cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev));
  d.ready = true;
  return d;
}

}  // namespace

using namespace dftfe;

extern "C" dftfe_status dftfe_cholgs_noalloc(double* X, int64_t ld, int64_t M, int ncol, void* stream) {
  ABI_BEGIN
  DFTFE_REQUIRE(X, "null X");
  DFTFE_REQUIRE(ncol >= 1 && ld >= ncol && M >= ncol, "bad sizes: need 1 <= ncol <= M and ld >= ncol");
  if (ncol > kMaxCols)
    throw Error(DFTFE_ERR_ARG, "dftfe_cholgs_noalloc: ncol exceeds the static scratch limit of " +
                                   std::to_string(kMaxCols) + " columns");
  const DeviceSetup& d = setup_current_device();
  // X must be device memory of the current device, whose static scratch the kernels use
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, X) != cudaSuccess) {
    cudaGetLastError();
    throw Error(DFTFE_ERR_ARG, "dftfe_cholgs_noalloc: X is not a device pointer");
  }
  int cur = 0;
  DFTFE_CHECK_CUDA(cudaGetDevice(&cur));
  if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)
    throw Error(DFTFE_ERR_ARG, "dftfe_cholgs_noalloc: X is not device memory");
  if (pa.device != cur) throw Error(DFTFE_ERR_ARG, "dftfe_cholgs_noalloc: X lives on another device");
  cudaStream_t s = (cudaStream_t)stream;
  const int N = ncol;
  const int T = (N + kTileCols - 1) / kTileCols;
  const int ntiles = T * (T + 1) / 2;
  const size_t n2 = (size_t)N * N;
  // split count: as many as fill the GPU, bounded by the rows and by the scratch
  const int64_t want = (4LL * d.sm_count + ntiles - 1) / ntiles;
  const int64_t by_rows = std::max<int64_t>(1, M / 256);
  const int64_t by_scratch = (int64_t)((kScratchDoubles - 32) / n2) - 2;
  const int nsplit = (int)std::max<int64_t>(1, std::min(want, std::min(by_rows, by_scratch)));
  double* part = d.scratch;                       // nsplit x N x N, fully overwritten
  double* S = part + (size_t)nsplit * n2;         // N x N: S, then L in place
  double* Z = S + n2;                             // N x N: L^-T
  int* status = (int*)(Z + n2);                   // written by the Cholesky kernel
  gram_partial_launch(s, X, ld, X, ld, M, N, nsplit, ntiles, part);
  gram_reduce_launch(s, part, nsplit, N, S);
  potrf(s, S, N, status);
  int st = 0;
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(s));
  if (st == DFTFE_ERR_NOT_SPD) throw Error(DFTFE_ERR_NOT_SPD, "overlap matrix is not positive definite");
  trtri_lower_to_upper_t(s, S, Z, N);
  rotate_launch(s, X, ld, M, N, Z, true);
  ABI_END
}
