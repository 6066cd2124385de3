// Mixed-precision subspace GEMMs on the tensor cores (Sec. 3.2 and Sec. 4.4): the FP32
// off-diagonal parts of the Gram matrices S = X^T X, H^ = X^T W and of the rotations
// X <- X Z (Z = L^-T in CholGS, Z = Q in Rayleigh-Ritz) run as TF32 split products with
// FP32 accumulation; the diagonals stay FP64 (column dots; X diag(Z) in the epilogue pass).
//
// Precision.  Each FP64 operand is narrowed to FP32 and cut into three TF32 slices (exact:
// 11 + 11 + 2 bits); the six slice products of order <= 2 (a1 b1, a1 b2, a2 b1, a1 b3,
// a2 b2, a3 b1) give FP32-equivalent products.  The tensor cores' FP32 accumulation loses
// accuracy systematically with the length of an accumulation chain, so every 32-deep chunk
// of the contraction goes to a fresh accumulator (two in tensor memory, alternating) and
// epilogue warps add the chunk products into FP32 registers rounded to nearest, as a plain
// FP32 dot product would.
//
// k_rot_tc: one CTA per (panel of 128 rows of X, tile of 128 output columns), the four
// column tiles of a panel adjacent in launch order so the panel is re-read from L2.  The
// FP32 product X offdiag(Z) goes to a buffer; k_rot_diag then forms X diag(Z) + product in
// FP64, in place.  Warp roles:
//   warp 0      B producer: bulk copies of the pre-split Z^T tiles (2-stage ring)
//   warp 1      TMEM owner and MMA issuer (one elected lane)
//   warps 2-5   A producers: each warp reads rows of the panel (one 256-byte line per row,
//               its next chunk ahead), narrows and splits them and writes the swizzled
//               K-major tiles
//   warps 6-9   epilogue: chunk products of one TMEM lane quadrant into FP32 registers
// Every wait is bounded; on a time-out the kernel records DFTFE_ERR_TIMEOUT, drains its own
// copies and MMAs (bounded), frees its tensor memory and returns.
#include "internal.h"
#include "tcgen05.h"

#include <algorithm>

namespace dftfe {

namespace st {

constexpr int kThreads = 320;
constexpr int kStages = 2;
constexpr int kSlices = 3;
constexpr int kTile = 16384;                 // 128 rows x 128 bytes, one slice
constexpr int kOperand = kSlices * kTile;    // one 128 x 32 operand block, all slices
constexpr int kStage = 2 * kOperand;         // A | B

struct Bars {
  uint64_t a_full[kStages], b_full[kStages], empty[kStages];
  uint64_t acc_full[2], acc_empty[2], drain;
  uint32_t tmem;
  int abort;
};

constexpr size_t smem_bytes() { return 1024 + kStages * (size_t)kStage + sizeof(Bars); }

// the three TF32 slices of an FP32 value (exact); each rounding by the two-integer-operation
// form of cvt.rna.tf32.f32 (identical for every finite input), which keeps the conversion off
// the instruction the producers would otherwise issue three times per value
__device__ __forceinline__ void slices3(float f, uint32_t& s1, uint32_t& s2, uint32_t& s3) {
  s1 = tc::tf32_rn_bits(__float_as_uint(f));
  const float r1 = f - __uint_as_float(s1);
  s2 = tc::tf32_rn_bits(__float_as_uint(r1));
  s3 = tc::tf32_rn_bits(__float_as_uint(r1 - __uint_as_float(s2)));
}

// the six slice products of one 32-deep chunk into accumulator d (fresh)
__device__ __forceinline__ void chunk_mma(uint32_t d, uint32_t a0, uint32_t b0) {
  const uint32_t id = tc::idesc(2u, 128, 128);
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    const uint32_t o = ks * 32;
    tc::mma_tf32(d, tc::sdesc(a0 + o), tc::sdesc(b0 + o), id, ks > 0 ? 1u : 0u);
    tc::mma_tf32(d, tc::sdesc(a0 + o), tc::sdesc(b0 + kTile + o), id, 1u);
    tc::mma_tf32(d, tc::sdesc(a0 + kTile + o), tc::sdesc(b0 + o), id, 1u);
    tc::mma_tf32(d, tc::sdesc(a0 + o), tc::sdesc(b0 + 2 * kTile + o), id, 1u);
    tc::mma_tf32(d, tc::sdesc(a0 + kTile + o), tc::sdesc(b0 + kTile + o), id, 1u);
    tc::mma_tf32(d, tc::sdesc(a0 + 2 * kTile + o), tc::sdesc(b0 + o), id, 1u);
  }
}

// epilogue: add chunk kc's 32 x 128 accumulator block of this warp's quadrant into acc
__device__ __forceinline__ bool drain_chunk(Bars* sh, uint32_t tmem, int q, int kc, float* acc,
                                            volatile int* abort, int* err) {
  const int buf = kc & 1;
  if (!tc::mbar_wait(&sh->acc_full[buf], (kc >> 1) & 1, abort, err)) return false;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
  for (int cb = 0; cb < 4; ++cb) {
    uint32_t r[32];
    tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(128 * buf + 32 * cb), r);
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[32 * cb + j] += __uint_as_float(r[j]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  tc::mbar_arrive(&sh->acc_empty[buf]);
  return true;
}

}  // namespace st

// Zt tiles: tile (kc, nt) holds rows n = 128 nt + r (r < 128) and k = 32 kc + kk (kk < 32)
// of Z^T, i.e. Z[k][n], as three TF32 slices, K-major 128-byte swizzle; zero on the
// diagonal, outside N x N, and (upper) below the diagonal.  zd = diag(Z) in FP64.
__global__ void k_rot_tiles(const double* __restrict__ Z, int N, int upper, int nkc, int nt,
                            uint8_t* __restrict__ Bt, double* __restrict__ zd) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)nkc * nt * 128 * 32;
  if (t >= total) return;
  const int kk = (int)(t % 32);
  const int r = (int)((t / 32) % 128);
  const int64_t tile = t / (32 * 128);       // kc * nt + column tile
  const int ct = (int)(tile % nt), kc = (int)(tile / nt);
  const int n = 128 * ct + r, k = 32 * kc + kk;
  double v = 0.0;
  if (n < N && k < N && k != n && (!upper || k < n)) v = Z[(int64_t)k * N + n];
  uint32_t s1, s2, s3;
  st::slices3(tc::narrow_f64(v), s1, s2, s3);
  uint8_t* base = Bt + tile * (int64_t)st::kOperand;
  const uint32_t off = tc::sw128((uint32_t)r, (uint32_t)(4 * kk));
  *reinterpret_cast<uint32_t*>(base + off) = s1;
  *reinterpret_cast<uint32_t*>(base + st::kTile + off) = s2;
  *reinterpret_cast<uint32_t*>(base + 2 * st::kTile + off) = s3;
  if (n < N && k == n) zd[n] = Z[(int64_t)k * N + n];
}

__global__ void __launch_bounds__(st::kThreads, 1) k_rot_tc(const double* __restrict__ X, int64_t ld, int64_t M,
                                                            int N, const uint8_t* __restrict__ Bt, int nkc_all, int nt,
                                                            int upper, float* __restrict__ Yo, int64_t ldo, int* err) {
  using namespace st;
  using namespace tc;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  Bars* sh = (Bars*)(base + kStages * kStage);
  volatile int* abort = &sh->abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ct = (int)(blockIdx.x % nt);               // output column tile
  const int64_t m0 = (int64_t)(blockIdx.x / nt) * 128;
  // an upper triangular Z (strict part) has no entries below row 128 ct + 127 in column
  // tile ct: its chunks kc > 4 ct + 3 are zero and are skipped
  const int nkc = upper ? min(nkc_all, 4 * ct + 4) : nkc_all;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sh->a_full[s], 128);
      mbar_init(&sh->b_full[s], 1);
      mbar_init(&sh->empty[s], 1);
    }
    for (int t = 0; t < 2; ++t) {
      mbar_init(&sh->acc_full[t], 1);
      mbar_init(&sh->acc_empty[t], 128);
    }
    mbar_init(&sh->drain, 1);
    sh->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&sh->tmem)), "r"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sh->tmem;

  if (warp == 0) {
    // ------------------------------------------------------------ B producer
    if (lane == 0) {
      int kc = 0;
      for (; kc < nkc && !*abort; ++kc) {
        const int s = kc % kStages;
        if (!mbar_wait(&sh->empty[s], ((kc / kStages) & 1) ^ 1, abort, err)) break;
        const uint32_t full = smem_u32(&sh->b_full[s]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(full), "r"(kOperand) : "memory");
        const uint8_t* src = Bt + ((int64_t)kc * nt + ct) * kOperand;
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     :: "r"(smem_u32(base + s * kStage + kOperand)), "l"(src), "r"(kOperand), "r"(full)
                     : "memory");
      }
      // drain: every issued copy has landed before the CTA may exit
      for (int u = max(0, kc - kStages); u < kc; ++u) {
        volatile int no_abort = 0;
        mbar_wait(&sh->b_full[u % kStages], (u / kStages) & 1, &no_abort, err);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      for (int kc = 0; kc < nkc && !*abort; ++kc) {
        const int s = kc % kStages, buf = kc & 1;
        if (!mbar_wait(&sh->acc_empty[buf], ((kc >> 1) & 1) ^ 1, abort, err)) break;
        if (!mbar_wait(&sh->a_full[s], (kc / kStages) & 1, abort, err)) break;
        if (!mbar_wait(&sh->b_full[s], (kc / kStages) & 1, abort, err)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_u32(base + s * kStage);
        chunk_mma(tmem + (uint32_t)(128 * buf), a0, a0 + kOperand);
        tc_commit(&sh->empty[s]);
        tc_commit(&sh->acc_full[buf]);
      }
      tc_commit(&sh->drain);
      volatile int no_abort = 0;
      mbar_wait(&sh->drain, 0, &no_abort, err);
    }
  } else if (warp < 6) {
    // ------------------------------------------------------------ A producers
    // warp w writes panel rows 32 w .. 32 w + 31 of each chunk, lane l holding column
    // k = 32 kc + l of a row; the raw FP64 values of the next chunk are loaded before the
    // current one is narrowed, split and stored
    const int w = warp - 2;
    double raw[32];
    auto load_a = [&](int kc) {
      const int k = 32 * kc + lane;
#pragma unroll
      for (int rr = 0; rr < 32; ++rr) {
        const int64_t m = m0 + 32 * w + rr;
        raw[rr] = (m < M && k < N) ? X[m * ld + k] : 0.0;
      }
    };
    if (nkc > 0) load_a(0);
    for (int kc = 0; kc < nkc && !*abort; ++kc) {
      const int s = kc % kStages;
      float v[32];
#pragma unroll
      for (int rr = 0; rr < 32; ++rr) v[rr] = narrow_f64(raw[rr]);
      if (kc + 1 < nkc) load_a(kc + 1);
      if (!mbar_wait(&sh->empty[s], ((kc / kStages) & 1) ^ 1, abort, err)) break;
      uint8_t* tile = base + s * kStage;
#pragma unroll
      for (int rr = 0; rr < 32; ++rr) {
        uint32_t s1, s2, s3;
        slices3(v[rr], s1, s2, s3);
        const uint32_t off = sw128((uint32_t)(32 * w + rr), (uint32_t)(4 * lane));
        *reinterpret_cast<uint32_t*>(tile + off) = s1;
        *reinterpret_cast<uint32_t*>(tile + kTile + off) = s2;
        *reinterpret_cast<uint32_t*>(tile + 2 * kTile + off) = s3;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&sh->a_full[s]);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    float acc[128];
#pragma unroll
    for (int j = 0; j < 128; ++j) acc[j] = 0.0f;
    bool ok = true;
    for (int kc = 0; kc < nkc && ok; ++kc) ok = drain_chunk(sh, tmem, q, kc, acc, abort, err);
    const int64_t m = m0 + 32 * q + lane;
    const int n0 = 128 * ct;
    if (ok && m < M) {
      float* y = Yo + m * ldo + n0;
      const int ncols = min(128, N - n0);
      if (ncols == 128) {
#pragma unroll
        for (int j = 0; j < 128; j += 4)
          *reinterpret_cast<float4*>(y + j) = make_float4(acc[j], acc[j + 1], acc[j + 2], acc[j + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 128; ++j)
          if (j < ncols) y[j] = acc[j];
      }
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(256));
}

// X[m][n] <- X[m][n] zd[n] + Yo[m][n] in FP64 (the diagonal of the rotation), two columns
// per thread
__global__ void k_rot_diag(double* __restrict__ X, int64_t ld, const float* __restrict__ Yo, int64_t ldo, int64_t M,
                           int N, const double* __restrict__ zd, const int* guard) {
  // a deferred pass whose factorisation or eigensolve failed leaves X as it is
  if (guard && (guard[0] != 0 || guard[1] != 0)) return;
  const int nh = (N + 1) / 2;
  const int64_t total = M * nh;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = t / nh;
    const int n = 2 * (int)(t - m * nh);
    double* x = X + m * ld + n;
    const float* y = Yo + m * ldo + n;
    x[0] = fma(x[0], zd[n], (double)y[0]);
    if (n + 1 < N) x[1] = fma(x[1], zd[n + 1], (double)y[1]);
  }
}

// ----------------------------------------------------------------------- Gram
// k_gram_tc: part[s][i][j] = sum over the rows m of split s of A[m][i] B[m][j] for one
// 128 x 128 block (bi, bj), bi >= bj, of the lower triangle (three TF32 slices, 32-row
// chunks into alternating accumulators, FP32 register sums; see the top of this file).
// Both operands are read transposed: a producer warp covers 32 columns, lane l loads
// column c0 + l of 32 consecutive rows (one 256-byte line per warp load), narrows and
// splits them and writes the lane's row of the K-major tile as 16-byte chunks.
// Warp roles: warp 1 TMEM owner and MMA issuer; warps 2-5 producers (the A and the B unit
// of each chunk); warps 6-9 epilogue.  Warp 0 only takes part in set-up and teardown.
__global__ void __launch_bounds__(st::kThreads, 1) k_gram_tc(const double* __restrict__ A, int64_t lda,
                                                             const double* __restrict__ B, int64_t ldb, int64_t M,
                                                             int N, int npairs, int64_t rows_per_split,
                                                             float* __restrict__ part, int* err) {
  using namespace st;
  using namespace tc;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  Bars* sh = (Bars*)(base + kStages * kStage);
  volatile int* abort = &sh->abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pidx = (int)(blockIdx.x % npairs);
  const int64_t sidx = blockIdx.x / npairs;
  int bi = (int)((sqrtf(8.0f * pidx + 1.0f) - 1.0f) * 0.5f);
  while (bi * (bi + 1) / 2 > pidx) --bi;
  while ((bi + 1) * (bi + 2) / 2 <= pidx) ++bi;
  const int bj = pidx - bi * (bi + 1) / 2;
  const int64_t k0 = sidx * rows_per_split;
  const int64_t k1 = min(M, k0 + rows_per_split);
  const int nkc = (int)((max((int64_t)0, k1 - k0) + 31) / 32);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sh->a_full[s], 128);
      mbar_init(&sh->b_full[s], 1);                     // unused here
      mbar_init(&sh->empty[s], 1);
    }
    for (int t = 0; t < 2; ++t) {
      mbar_init(&sh->acc_full[t], 1);
      mbar_init(&sh->acc_empty[t], 128);
    }
    mbar_init(&sh->drain, 1);
    sh->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&sh->tmem)), "r"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sh->tmem;

  if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      for (int kc = 0; kc < nkc && !*abort; ++kc) {
        const int s = kc % kStages, buf = kc & 1;
        if (!mbar_wait(&sh->acc_empty[buf], ((kc >> 1) & 1) ^ 1, abort, err)) break;
        if (!mbar_wait(&sh->a_full[s], (kc / kStages) & 1, abort, err)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_u32(base + s * kStage);
        chunk_mma(tmem + (uint32_t)(128 * buf), a0, a0 + kOperand);
        tc_commit(&sh->empty[s]);
        tc_commit(&sh->acc_full[buf]);
      }
      tc_commit(&sh->drain);
      volatile int no_abort = 0;
      mbar_wait(&sh->drain, 0, &no_abort, err);
    }
  } else if (warp >= 2 && warp < 6) {
    // ------------------------------------------------------------ producers
    // per chunk: the A unit (columns 128 bi + 32 w) and the B unit (columns 128 bj + 32 w);
    // the raw FP64 values of the next unit are loaded before the current one is narrowed,
    // split and stored
    const int w = warp - 2;
    const int total = 2 * nkc;
    double raw[32];
    auto load = [&](int u) {
      const int kc = u >> 1;
      const bool isA = (u & 1) == 0;
      const double* src = isA ? A : B;
      const int64_t ldm = isA ? lda : ldb;
      const int c = 128 * (isA ? bi : bj) + 32 * w + lane;
#pragma unroll
      for (int kk = 0; kk < 32; ++kk) {
        const int64_t m = k0 + 32 * kc + kk;
        raw[kk] = (c < N && m < k1) ? src[m * ldm + c] : 0.0;
      }
    };
    if (total > 0) load(0);
    for (int u = 0; u < total && !*abort; ++u) {
      const int kc = u >> 1, s = kc % kStages;
      const bool isA = (u & 1) == 0;
      float v[32];
#pragma unroll
      for (int kk = 0; kk < 32; ++kk) v[kk] = narrow_f64(raw[kk]);
      if (u + 1 < total) load(u + 1);
      if (isA && !mbar_wait(&sh->empty[s], ((kc / kStages) & 1) ^ 1, abort, err)) break;
      uint8_t* tile = base + s * kStage + (isA ? 0 : kOperand);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        uint32_t s1[4], s2[4], s3[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) slices3(v[4 * c + e], s1[e], s2[e], s3[e]);
        const uint32_t off = sw128((uint32_t)(32 * w + lane), (uint32_t)(16 * c));
        *reinterpret_cast<uint4*>(tile + off) = make_uint4(s1[0], s1[1], s1[2], s1[3]);
        *reinterpret_cast<uint4*>(tile + kTile + off) = make_uint4(s2[0], s2[1], s2[2], s2[3]);
        *reinterpret_cast<uint4*>(tile + 2 * kTile + off) = make_uint4(s3[0], s3[1], s3[2], s3[3]);
      }
      if (!isA) {                                      // the stage is complete (A and B written)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&sh->a_full[s]);
      }
    }
  } else if (warp >= 6) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    float acc[128];
#pragma unroll
    for (int j = 0; j < 128; ++j) acc[j] = 0.0f;
    bool ok = true;
    for (int kc = 0; kc < nkc && ok; ++kc) ok = drain_chunk(sh, tmem, q, kc, acc, abort, err);
    const int i = 128 * bi + 32 * q + lane;
    if (ok && i < N) {
      float* out = part + sidx * (int64_t)N * N + (int64_t)i * N + 128 * bj;
      const int ncols = min(128, N - 128 * bj);
#pragma unroll
      for (int j = 0; j < 128; ++j)
        if (j < ncols) out[j] = acc[j];
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(256));
}

// C[i][j] = C[j][i] = sum_s part[s][i][j] (i > j, FP64 sum in split order); C[i][i] = sum of
// the FP64 column-dot partials
__global__ void k_gram_tc_reduce(const float* __restrict__ part, int nsplit, const double* __restrict__ dpart,
                                 int nchunk, int N, double* __restrict__ C) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * N) return;
  const int i = (int)(t / N), j = (int)(t % N);
  if (i < j) return;
  double s = 0.0;
  if (i == j)
    for (int c = 0; c < nchunk; ++c) s += dpart[(int64_t)c * N + i];
  else
    for (int k = 0; k < nsplit; ++k) s += (double)part[(int64_t)k * N * N + t];
  C[(int64_t)i * N + j] = s;
  C[(int64_t)j * N + i] = s;
}

static unsigned nblk_tc(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// X <- X Z (in place) for N <= 512 with the tensor-core kernel; false when not applicable
bool rotate_inplace_tc(dftfe_ham h, double* X, int64_t ld, int64_t M, int N, const double* Z, bool upper) {
  if (N < 1 || M < 1) return false;
  static bool attr = false;
  if (!attr) {
    DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_rot_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)st::smem_bytes()));
    attr = true;
  }
  const int nkc = (N + 31) / 32, nt = (N + 127) / 128;
  uint8_t* Bt = (uint8_t*)ws_get(h, "rot_tc_tiles", (size_t)nkc * nt * st::kOperand);
  double* zd = (double*)ws_get(h, "rot_tc_zd", sizeof(double) * (size_t)N);
  int* err = tc_err_flag(h, (int*)ws_get(h, "rot_tc_err", sizeof(int)));
  if (!h->deferred) DFTFE_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), h->stream));
  DFTFE_LAUNCH(k_rot_tiles, nblk_tc((int64_t)nkc * nt * 128 * 32), 256, 0, h->stream, Z, N, upper ? 1 : 0, nkc, nt,
               Bt, zd);
  // the FP32 product X offdiag(Z) goes through a buffer of at most 2 GiB: row slabs of a
  // multiple of 128 rows, each rotated and then given its FP64 diagonal part in place
  const int64_t ldo = (N + 3) / 4 * 4;
  const int64_t cap_rows = std::max<int64_t>(128, ((int64_t)(2LL << 30) / (ldo * 4)) / 128 * 128);
  const int64_t slab = std::min<int64_t>((M + 127) / 128 * 128, cap_rows);
  float* Yo = (float*)ws_get(h, "rot_tc_out", sizeof(float) * (size_t)slab * ldo);
  for (int64_t r0 = 0; r0 < M; r0 += slab) {
    const int64_t ms = std::min<int64_t>(slab, M - r0);
    double* Xs = X + r0 * ld;
    {
      ProfScope ps(h, "rotate_tc");
      DFTFE_LAUNCH(k_rot_tc, (unsigned)(((ms + 127) / 128) * nt), st::kThreads, st::smem_bytes(), h->stream, Xs, ld, ms,
                   N, Bt, nkc, nt, upper ? 1 : 0, Yo, ldo, err);
    }
    {
      ProfScope ps(h, "rotate_diag");
      DFTFE_LAUNCH(k_rot_diag, (unsigned)std::min<int64_t>((int64_t)h->sm_count * 16, nblk_tc(ms * ((N + 1) / 2))), 256,
                   0, h->stream, Xs, ld, Yo, ldo, ms, N, zd, rot_guard(h));
    }
  }
  if (h->deferred) return true;
  int herr = 0;
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  if (herr) throw Error(DFTFE_ERR_TIMEOUT, "tensor-core rotation: a bounded wait timed out");
  return true;
}

}  // namespace dftfe

namespace dftfe {

// C (N x N, both triangles) = A^T B with TF32x3 off-diagonal entries and FP64 diagonal
// (N <= 512); false when not applicable
bool gram_lower_tc(dftfe_ham h, const double* A, int64_t lda, const double* B, int64_t ldb, int64_t M, int N,
                   double* C, const double* dpart, int nchunk) {
  if (N < 1 || M < 1) return false;
  static bool attr = false;
  if (!attr) {
    DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)st::smem_bytes()));
    attr = true;
  }
  const int NB = (N + 127) / 128;
  const int npairs = NB * (NB + 1) / 2;
  // row splits: at least two CTAs per SM in all, and (one CTA per SM at a time) a split
  // count whose CTAs fill their last wave: the count in [want, 8 want] with the least idle
  // SM slots in the last wave, per CTA-wave of work (36 blocks at N = 1,024 take 38 splits,
  // 9 full waves, where 9 splits left 0.87 of the third wave idle)
  const int64_t sm = std::max(1, h->sm_count);
  const int64_t want = std::max<int64_t>(1, (2 * sm + npairs - 1) / npairs);
  int64_t pick = want;
  double best = 1e300;
  for (int64_t c = want; c <= 8 * want; ++c) {
    const int64_t ctas = c * npairs, waves = (ctas + sm - 1) / sm;
    const double t = (double)waves / (double)c;          // time ~ waves x rows per split
    if (t < best * (1.0 - 1e-9)) {
      best = t;
      pick = c;
    }
  }
  const int64_t nsplit = std::max<int64_t>(1, std::min<int64_t>(pick, (M + 1023) / 1024));
  const int64_t rows = ((M + nsplit - 1) / nsplit + 31) / 32 * 32;
  const int64_t ns = (M + rows - 1) / rows;
  float* part = (float*)ws_get(h, "gram_tc_part", sizeof(float) * (size_t)ns * N * N);
  int* err = tc_err_flag(h, (int*)ws_get(h, "gram_tc_err", sizeof(int)));
  if (!h->deferred) DFTFE_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), h->stream));
  {
    ProfScope ps(h, "gram_tc");
    DFTFE_LAUNCH(k_gram_tc, (unsigned)(ns * npairs), st::kThreads, st::smem_bytes(), h->stream, A, lda, B, ldb, M, N,
                 npairs, rows, part, err);
  }
  DFTFE_LAUNCH(k_gram_tc_reduce, nblk_tc((int64_t)N * N), 256, 0, h->stream, part, (int)ns, dpart, nchunk, N, C);
  if (h->deferred) return true;
  int herr = 0;
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  if (herr) throw Error(DFTFE_ERR_TIMEOUT, "tensor-core Gram: a bounded wait timed out");
  return true;
}

}  // namespace dftfe
