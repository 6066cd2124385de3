// Mixed-precision H~X for the Chebyshev filter: the dense cell products
// Y^c = H~^c X^c (Sec. 4.3, Eq. celldgemm) as 3-term split products on the fifth-generation
// tensor cores (tcgen05), FP32 accumulation in tensor memory, FP32 vectors.
//
//   H~^c = H_hi + H_lo, X^c = X_hi + X_lo  (each term TF32 or BF16, rounded to nearest)
//   Y^c ~= H_hi X_hi + H_hi X_lo + H_lo X_hi
//
// Operand layout: K-major, 128-byte swizzle (rows of 128 bytes, 8-row atoms of 1024 bytes,
// 16-byte chunks XOR-ed with the row index mod 8).  The split cell matrices are laid out in
// HBM in exactly this tile order at set-up, so the kernel streams them with plain bulk
// copies (cp.async.bulk) into shared memory.  The cell's columns of X are gathered by four
// producer warps, split, and written transposed (K-major) into the B tiles.
//
// One CTA per SM walks the cells (all of them, in one launch per 128-column tile) and
// writes each product Y^c with plain stores to a per-cell buffer; a separate assembly
// kernel sums every node's cell contributions in fixed order, fused with the recurrence
// terms, so the tensor-core kernel never waits on a read-modify-write.  Warp roles:
//   warp 0      A producer (bulk copies of the split cell-matrix tiles, 4-stage ring)
//   warp 1      TMEM owner and MMA issuer (one elected lane)
//   warps 2-5   B producers (coalesced gather + split of X^c, 2-stage ring, loads one
//               chunk ahead)
//   warps 6-9   epilogue (tcgen05.ld of the accumulators, stores of the rows of Y^c)
// Every wait is bounded; on a time-out the kernel records DFTFE_ERR_TIMEOUT, drains its
// own copies and MMAs (bounded), frees its tensor memory and returns.
#include "internal.h"
#include "tcgen05.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <memory>

namespace dftfe {

namespace mx {

constexpr int kThreads = 320;
constexpr int kStagesA = 4, kStagesB = 2;
constexpr int kTile = 16384;                       // one 128-row x 128-byte operand tile
constexpr int kStageBytes = 2 * kTile;             // hi + lo
constexpr int kMaxMTiles = 4;                      // 4 x 128 accumulator columns = 512 TMEM columns
constexpr int kPatchLd = 36;                       // epilogue patch row stride (floats)
constexpr int kPatchBytes = 4 * 32 * kPatchLd * 4;

using tc::idesc;
using tc::mbar_arrive;
using tc::mbar_init;
using tc::mbar_wait;
using tc::sdesc;
using tc::smem_u32;
using tc::sw128;
using tc::tc_commit;
using tc::tf32_rn;

struct Shared {
  uint64_t a_full[kStagesA], a_empty[kStagesA];
  uint64_t b_full[kStagesB], b_empty[kStagesB];
  uint64_t acc_full, acc_empty[kMaxMTiles], drain;   // acc_empty per 128-column accumulator
  uint32_t tmem;
  int abort;
};

template <bool TF32>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  constexpr uint32_t id = idesc(TF32 ? 2u : 1u, 128, 128);
  if (TF32)
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                 :: "r"(d), "l"(a), "l"(b), "r"(id), "r"(acc));
  else
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 :: "r"(d), "l"(a), "l"(b), "r"(id), "r"(acc));
}

// split x into two terms of the operand type, packed as the 16-byte chunk layout needs
template <bool TF32> struct Split;
template <> struct Split<true> {
  static constexpr int G = 4;  // elements per 16-byte chunk
  __device__ static void run(const float* v, uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      h[i] = tf32_rn(v[i]);
      l[i] = tf32_rn(v[i] - __uint_as_float(h[i]));
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
  }
};
template <> struct Split<false> {
  static constexpr int G = 8;
  __device__ static void run(const float* v, uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __nv_bfloat16 a = __float2bfloat16_rn(v[2 * i]), b = __float2bfloat16_rn(v[2 * i + 1]);
      __nv_bfloat16 c = __float2bfloat16_rn(v[2 * i] - __bfloat162float(a));
      __nv_bfloat16 d = __float2bfloat16_rn(v[2 * i + 1] - __bfloat162float(b));
      h[i] = (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
      l[i] = (uint32_t)__bfloat16_as_ushort(c) | ((uint32_t)__bfloat16_as_ushort(d) << 16);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
  }
};

}  // namespace mx

// Set-up: split the FP64 cell matrices into the tile order the kernel streams:
// A[cell][kc][mt][hi|lo][16 KB tile]; tile row r <-> matrix row mt*128 + r, tile byte b <->
// column kc*KC + b/esize; zero outside nc x nc.
template <bool TF32>
__global__ void k_split_cells(const double* __restrict__ Hc, uint8_t* __restrict__ A, int64_t Nc, int nc,
                              int nkc, int nmt) {
  constexpr int ES = TF32 ? 4 : 2, KC = 128 / ES;
  const int64_t per_cell = (int64_t)nkc * nmt * 128 * KC;   // elements (each yields hi and lo)
  const int64_t total = Nc * per_cell;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = t / per_cell;
    int64_t rem = t - cell * per_cell;
    const int e = (int)(rem % KC);
    rem /= KC;
    const int r = (int)(rem % 128);
    rem /= 128;
    const int mt = (int)(rem % nmt);
    const int kc = (int)(rem / nmt);
    const int m = mt * 128 + r, k = kc * KC + e;
    const double h = (m < nc && k < nc) ? Hc[(cell * nc + m) * (int64_t)nc + k] : 0.0;
    uint8_t* tile = A + (((cell * nkc + kc) * nmt + mt) * 2) * (int64_t)mx::kTile;
    const uint32_t off = mx::sw128((uint32_t)r, (uint32_t)(e * ES));
    if (TF32) {
      const uint32_t hi = mx::tf32_rn(__double2float_rn(h));
      const uint32_t lo = mx::tf32_rn(__double2float_rn(h - (double)__uint_as_float(hi)));
      *reinterpret_cast<uint32_t*>(tile + off) = hi;
      *reinterpret_cast<uint32_t*>(tile + mx::kTile + off) = lo;
    } else {
      const __nv_bfloat16 hi = __double2bfloat16(h);
      const __nv_bfloat16 lo = __double2bfloat16(h - (double)__bfloat162float(hi));
      *reinterpret_cast<__nv_bfloat16*>(tile + off) = hi;
      *reinterpret_cast<__nv_bfloat16*>(tile + mx::kTile + off) = lo;
    }
  }
}

template <bool TF32>
__global__ void __launch_bounds__(mx::kThreads, 1) k_cell_mixed(
    const uint8_t* __restrict__ A, const int32_t* __restrict__ map, int ncells, int nc, int nkc, int nmt, const float* __restrict__ X, int64_t ldx,
    float* __restrict__ Yc, int col0, int ncol, int* err) {
  using namespace mx;
  constexpr int ES = TF32 ? 4 : 2, KC = 128 / ES, G = Split<TF32>::G;
  // cell of the i-th work item of this CTA (cells dealt round-robin over the grid)
  auto cell_of = [&](int64_t i) -> int64_t { return blockIdx.x + i * gridDim.x; };
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;                                    // kStagesA x (hi 16K | lo 16K)
  uint8_t* sB = base + kStagesA * kStageBytes;           // kStagesB x (hi 16K | lo 16K)
  uint8_t* sP = sB + kStagesB * kStageBytes;            // 4 epilogue patches of 32 x kPatchLd floats
  Shared* sh = (Shared*)(sP + kPatchBytes);
  volatile int* abort = &sh->abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStagesA; ++s) { mbar_init(&sh->a_full[s], 1); mbar_init(&sh->a_empty[s], 1); }
    for (int s = 0; s < kStagesB; ++s) { mbar_init(&sh->b_full[s], 128); mbar_init(&sh->b_empty[s], 1); }
    mbar_init(&sh->acc_full, 1);
    for (int t = 0; t < kMaxMTiles; ++t) mbar_init(&sh->acc_empty[t], 128);
    mbar_init(&sh->drain, 1);
    sh->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&sh->tmem)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sh->tmem;
  const int my_cells = ncells > (int)blockIdx.x ? (ncells - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int last_rows8 = ((nc - 128 * (nmt - 1)) + 7) / 8 * 8;   // rows of the last M-tile, in atoms

  if (warp == 0) {
    // ------------------------------------------------------------ A producer
    if (lane == 0) {
      uint32_t ta = 0;
      for (int i = 0; i < my_cells && !*abort; ++i) {
        const int64_t cell = cell_of(i);
        for (int kc = 0; kc < nkc && !*abort; ++kc)
          for (int mt = 0; mt < nmt; ++mt, ++ta) {
            const int s = ta % kStagesA;
            if (!mbar_wait(&sh->a_empty[s], ((ta / kStagesA) & 1) ^ 1, abort, err)) break;
            const uint32_t full = smem_u32(&sh->a_full[s]);
            // only the 8-row atoms that hold matrix rows are streamed: the rows of the last
            // M-tile beyond n_c keep stale data, which only reaches accumulator rows that the
            // epilogue never stores (row m of a product depends on row m of A alone)
            const uint32_t bytes = mt == nmt - 1 ? (uint32_t)last_rows8 * 128u : (uint32_t)kTile;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(full), "r"(2 * bytes) : "memory");
            const uint8_t* src = A + (((cell * nkc + kc) * nmt + mt) * 2) * (int64_t)kTile;
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(smem_u32(sA + s * kStageBytes)), "l"(src), "r"(bytes), "r"(full) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(smem_u32(sA + s * kStageBytes + kTile)), "l"(src + kTile), "r"(bytes), "r"(full)
                         : "memory");
          }
      }
      // drain: every issued copy has landed before the CTA may exit
      for (uint32_t t = (ta > (uint32_t)kStagesA ? ta - kStagesA : 0); t < ta; ++t) {
        volatile int no_abort = 0;
        mbar_wait(&sh->a_full[t % kStagesA], (t / kStagesA) & 1, &no_abort, err);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t ta = 0, tb = 0;
      for (int i = 0; i < my_cells && !*abort; ++i) {
        for (int kc = 0; kc < nkc && !*abort; ++kc, ++tb) {
          const int sb = tb % kStagesB;
          if (!mbar_wait(&sh->b_full[sb], (tb / kStagesB) & 1, abort, err)) break;
          const uint32_t bhi = smem_u32(sB + sb * kStageBytes), blo = bhi + kTile;
          for (int mt = 0; mt < nmt; ++mt, ++ta) {
            const int sa = ta % kStagesA;
            // the first product into accumulator mt waits until the epilogue has read
            // that accumulator of the previous cell (it drains them in the same order)
            if (kc == 0 && !mbar_wait(&sh->acc_empty[mt], (i & 1) ^ 1, abort, err)) break;
            if (!mbar_wait(&sh->a_full[sa], (ta / kStagesA) & 1, abort, err)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ahi = smem_u32(sA + sa * kStageBytes), alo = ahi + kTile;
            const uint32_t d = tmem + (uint32_t)(mt * 128);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              const uint32_t o = ks * 32;
              mma<TF32>(d, sdesc(ahi + o), sdesc(bhi + o), (kc > 0 || ks > 0) ? 1u : 0u);
              mma<TF32>(d, sdesc(ahi + o), sdesc(blo + o), 1u);
              mma<TF32>(d, sdesc(alo + o), sdesc(bhi + o), 1u);
            }
            tc_commit(&sh->a_empty[sa]);
          }
          tc_commit(&sh->b_empty[sb]);
        }
        tc_commit(&sh->acc_full);
      }
      // drain: all issued MMAs complete before tensor memory is released
      tc_commit(&sh->drain);
      volatile int no_abort = 0;
      mbar_wait(&sh->drain, 0, &no_abort, err);
    }
  } else if (warp >= 2 && warp < 6) {
    // ------------------------------------------------------------ B producers
    // warp w covers tile rows (columns of X) n = 32w + lane: for every row k of the chunk
    // the warp reads 32 consecutive floats of X row map[k] (one 128-byte line), so lane
    // l holds column n for all k of the chunk without any exchange between lanes.
    const int w = warp - 2;
    const int n = 32 * w + lane;
    const int col = col0 + n;
    constexpr int QN = KC / 4;                   // row quads per K-chunk
    // loads of chunk tb+1 are issued before chunk tb is split and stored
    const uint32_t nchunks = (uint32_t)my_cells * (uint32_t)nkc;
    float v[KC], vn[KC];
    auto load_chunk = [&](uint32_t t, float* dst) {
      const int64_t cell = cell_of(t / nkc);
      const int kc = (int)(t % nkc);
      const int32_t* cm = map + cell * nc;
#pragma unroll
      for (int j = 0; j < KC; ++j) {
        const int k = kc * KC + j;
        dst[j] = 0.0f;
        if (k < nc && col < ncol) dst[j] = __ldg(X + (int64_t)__ldg(cm + k) * ldx + col);
      }
    };
    if (nchunks > 0) load_chunk(0, v);
    for (uint32_t tb = 0; tb < nchunks && !*abort; ++tb) {
      {
        if (tb + 1 < nchunks) load_chunk(tb + 1, vn);
        const int sb = tb % kStagesB;
        if (!mbar_wait(&sh->b_empty[sb], ((tb / kStagesB) & 1) ^ 1, abort, err)) break;
        uint8_t* bhi = sB + sb * kStageBytes;
        uint8_t* blo = bhi + kTile;
#pragma unroll
        for (int q = 0; q < QN; q += G / 4) {     // one 16-byte chunk of the row per step
          uint4 hi, lo;
          Split<TF32>::run(v + 4 * q, hi, lo);
          const uint32_t off = sw128((uint32_t)n, (uint32_t)((q / (G / 4)) * 16));
          *reinterpret_cast<uint4*>(bhi + off) = hi;
          *reinterpret_cast<uint4*>(blo + off) = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&sh->b_full[sb]);
      }
#pragma unroll
      for (int j = 0; j < KC; ++j) v[j] = vn[j];
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // each warp reads 32 accumulator rows x 32 columns at a time (lane = row), turns them
    // around in its shared-memory patch (row stride 36 floats) and writes 4 rows x 128 B
    // per store instruction; accumulator mt is released as soon as it has been read.
    const int q = warp & 3;                       // TMEM lane quadrant of this warp
    float* patch = reinterpret_cast<float*>(sP) + q * (32 * kPatchLd);
    for (int i = 0; i < my_cells; ++i) {
      if (!mbar_wait(&sh->acc_full, i & 1, abort, err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int64_t cell = cell_of(i);
      for (int mt = 0; mt < nmt; ++mt) {
        const int row0 = mt * 128 + q * 32;       // first accumulator row of this warp
        for (int cb = 0; cb < 4; ++cb) {
          uint32_t r[32];
          const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(mt * 128 + cb * 32);
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                       "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                       : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                         "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                         "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                         "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                       : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (row0 >= nc) continue;               // whole patch is padding (warp-uniform)
#pragma unroll
          for (int j = 0; j < 32; j += 4)
            *reinterpret_cast<uint4*>(patch + lane * kPatchLd + j) = make_uint4(r[j], r[j + 1], r[j + 2], r[j + 3]);
          __syncwarp();
#pragma unroll
          for (int it = 0; it < 8; ++it) {
            const int rl = it * 4 + (lane >> 3);  // patch row of this lane
            const int row = row0 + rl;
            const float4 val = *reinterpret_cast<const float4*>(patch + rl * kPatchLd + 4 * (lane & 7));
            // row `row` of Y^c is slot cell * nc + row of the per-cell output (128 floats)
            if (row < nc)
              *reinterpret_cast<float4*>(Yc + (cell * nc + row) * (int64_t)128 + cb * 32 + 4 * (lane & 7)) = val;
          }
          __syncwarp();
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&sh->acc_empty[mt]);
      }
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512));
}

// ------------------------------------------------------------ TF32x3 from one FP32 plane
// The TF32x3 form streams the cell matrices as ONE FP32 plane (4 bytes per entry, rounded to
// nearest from FP64) and splits every tile into its hi and lo TF32 terms on chip:
//   plane layout: per (cell, K-chunk of 32 columns) the M-tiles of 128 rows in order, each a
//   K-major 128-byte-swizzled tile of 128 x 32 floats; the last M-tile holds only its rows in
//   8-row atoms (88 of 128 for p = 6), so a cell streams (nmt - 1) x 16 KB + rows8 x 128 B per
//   K-chunk -- the nc x nc matrix plus the K padding, nothing else.
// The FP32 tiles land in a ring that is released as soon as a tile is converted, so several
// 16 KB bulk copies stay in flight per SM.  Measured on GB300, 128 x 128 x 8 TF32 MMAs with
// both operands in shared memory issue at about half the nominal TF32 rate; with at most
// three M-tiles (p <= 6) the converters therefore write the hi and lo A tiles into tensor
// memory (2 slots x 64 columns beside the 3 x 128 accumulator columns) and the MMAs read A
// from there (tcgen05.mma A-in-TMEM form), halving the shared-memory operand traffic.  With
// four M-tiles (p = 7) the accumulators fill tensor memory and the hi/lo A tiles go to a
// 2-slot shared-memory ring instead.
// Warp roles (448 threads):
//   warp 0        A producer: one bulk copy per tile into the landing ring
//   warp 1        TMEM owner and MMA issuer (one elected lane)
//   warps 2-5     B producers: cp.async gather of the cell's rows of X (each warp 32 columns,
//                 into its own 4 KB slice of the stage's lo slot, kStagesB - 1 chunks ahead;
//                 the cell map entries of the next chunk are loaded one chunk ahead), then
//                 the split of the chunk into the swizzled hi and lo B tiles
//   warps 6-9     epilogue (tcgen05.ld of the accumulators, 32-byte stores of Y^c rows)
//   warps 10-13   A converters: landing tile -> hi = rn_tf32(f), lo = rn_tf32(f - hi), into
//                 tensor memory (one row per thread) or the shared-memory ring
// Every wait is bounded; on a time-out the kernel records DFTFE_ERR_TIMEOUT, drains its own
// copies and MMAs (bounded), frees its tensor memory and returns.
namespace mp {
constexpr int kThreads = 448;
constexpr int kTile = 16384;
constexpr int kStage = 2 * kTile;                  // hi | lo
constexpr int kMaxMTiles = 4;
constexpr int kConv = 2;
constexpr uint32_t kAcolBase = 384;                // first TMEM column of the A slots (TMEM form)
// DEEP: the same shared memory as 8 landing slots and 3 B stages instead of 6 and 4 (more of
// the A stream in flight, less lookahead for the X gathers); a launch shape the tuner times
template <bool ATMEM, bool DEEP = false> struct Cfg {
  static constexpr int kLand = ATMEM ? (DEEP ? 8 : 6) : 4;      // landing ring slots (FP32 tiles)
  static constexpr int kStagesB = ATMEM ? (DEEP ? 3 : 4) : 3;   // B ring stages
  static constexpr int kConvSmem = ATMEM ? 0 : kConv;
};
template <bool ATMEM, bool DEEP = false> struct Shared {
  uint64_t land_full[Cfg<ATMEM, DEEP>::kLand], land_empty[Cfg<ATMEM, DEEP>::kLand];
  uint64_t conv_full[kConv], conv_empty[kConv];
  uint64_t b_full[Cfg<ATMEM, DEEP>::kStagesB], b_empty[Cfg<ATMEM, DEEP>::kStagesB];
  uint64_t acc_full, acc_empty[kMaxMTiles], drain;
  uint32_t tmem;
  int abort;
};
template <bool ATMEM, bool DEEP = false> constexpr size_t smem_bytes() {
  using C = Cfg<ATMEM, DEEP>;
  return 1024 + (size_t)C::kLand * kTile + (size_t)C::kConvSmem * kStage + (size_t)C::kStagesB * kStage +
         sizeof(Shared<ATMEM, DEEP>);
}
static_assert(smem_bytes<true, true>() <= 227 * 1024 && smem_bytes<true, false>() <= 227 * 1024 &&
                  smem_bytes<false, false>() <= 227 * 1024,
              "TF32x3 cell kernel: shared memory above the 227 KB per CTA");
__host__ __device__ inline int64_t kc_block_bytes(int nmt, int rows8) {
  return (int64_t)(nmt - 1) * kTile + (int64_t)rows8 * 128;
}
// the operands of one system in a launch: its FP32 plane, cell map, FP32 block (ld a multiple
// of 32 floats) with the launch's columns col0 .. col0 + 127 (ncol in all), and its
// per-cell product buffer
struct Item {
  const uint8_t* A;
  const int32_t* map;
  const float* X;
  float* Yc;
  int64_t ldx;
  int col0, ncol;
};

// one TF32 MMA with A from tensor memory (column address a_tmem), B from a shared-memory
// descriptor
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t acc) {
  constexpr uint32_t id = tc::idesc(2u, 128, 128);
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}"
               :: "r"(d), "r"(a_tmem), "l"(b), "r"(id), "r"(acc));
}

// 32 consecutive 32-bit TMEM columns of this warp's 32 lanes from registers (lane = row)
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t* r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
               "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
               :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
                  "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
                  "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
                  "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
               : "memory");
}
}  // namespace mp

// Set-up: the FP32 plane in the tile order above (written in physical order, so the stores
// are coalesced; each physical position is mapped back through the swizzle).
__global__ void k_plane_cells(const double* __restrict__ Hc, float* __restrict__ A, int64_t Nc, int nc, int nkc,
                              int nmt, int rows8) {
  const int64_t per_kc = mp::kc_block_bytes(nmt, rows8) / 4;      // floats per (cell, K-chunk)
  const int64_t total = Nc * nkc * per_kc;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blk = t / per_kc;
    const int w = (int)(t - blk * per_kc);
    const int64_t cell = blk / nkc;
    const int kc = (int)(blk - cell * nkc);
    const int mt = w >> 12;                                        // 4096 floats per tile
    const uint32_t p = (uint32_t)(w & 4095) * 4u;                  // physical byte in the tile
    const uint32_t r = p >> 7;
    const uint32_t lchunk = ((p >> 4) & 7u) ^ (r & 7u);
    const int e = (int)(lchunk * 4u + ((p & 15u) >> 2));
    const int m = mt * 128 + (int)r, k = kc * 32 + e;
    A[t] = (m < nc && k < nc) ? __double2float_rn(Hc[(cell * nc + m) * (int64_t)nc + k]) : 0.0f;
  }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(bytes) : "memory");
}

// Work item g of a launch: cell g of `single` (work == NULL), or the (system, cell) pair
// work[g] of the systems `items` (all of one degree: nc, nkc, nmt are the launch's).  Items
// are dealt to the persistent grid round-robin (deal = 0: CTA b takes b, b + grid, ...) or in
// contiguous ranges (deal = 1: CTA b takes the b-th of grid near-equal ranges), a launch shape
// the autotuner picks; every item is computed the same way either way.
template <bool ATMEM, bool DEEP>
__global__ void __launch_bounds__(mp::kThreads, 1) k_cell_tf32p(mp::Item single, const mp::Item* __restrict__ items,
                                                                const int2* __restrict__ work, int nwork, int nc,
                                                                int nkc, int nmt, int deal, int* err) {
  using namespace mp;
  using tc::mbar_arrive;
  using tc::mbar_init;
  using tc::mbar_wait;
  using tc::sdesc;
  using tc::smem_u32;
  using tc::sw128;
  using tc::tc_commit;
  constexpr int kLand = Cfg<ATMEM, DEEP>::kLand, kStagesB = Cfg<ATMEM, DEEP>::kStagesB;
  // the CTA's i-th work item: its system's operands and its cell
  const int q_deal = nwork / (int)gridDim.x, r_deal = nwork % (int)gridDim.x;
  const int64_t first = deal ? (int64_t)blockIdx.x * q_deal + min((int)blockIdx.x, r_deal) : 0;
  auto item_of = [&](int64_t i, int64_t& cell) -> Item {
    const int64_t g = deal ? first + i : blockIdx.x + i * gridDim.x;
    if (!work) {
      cell = g;
      return single;
    }
    const int2 w = work[g];
    cell = w.y;
    return items[w.x];
  };
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sL = base;                                        // landing ring: kLand x 16 KB FP32
  uint8_t* sC = sL + kLand * kTile;                          // shared-memory hi/lo ring (not ATMEM)
  uint8_t* sB = sC + Cfg<ATMEM, DEEP>::kConvSmem * kStage;   // B ring: kStagesB x (hi | lo)
  Shared<ATMEM, DEEP>* sh = (Shared<ATMEM, DEEP>*)(sB + kStagesB * kStage);
  volatile int* abort = &sh->abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kLand; ++s) {
      mbar_init(&sh->land_full[s], 1);
      mbar_init(&sh->land_empty[s], 128);
    }
    for (int s = 0; s < kConv; ++s) {
      mbar_init(&sh->conv_full[s], 128);
      mbar_init(&sh->conv_empty[s], 1);
    }
    for (int s = 0; s < kStagesB; ++s) { mbar_init(&sh->b_full[s], 128); mbar_init(&sh->b_empty[s], 1); }
    mbar_init(&sh->acc_full, 1);
    for (int t = 0; t < kMaxMTiles; ++t) mbar_init(&sh->acc_empty[t], 128);
    mbar_init(&sh->drain, 1);
    sh->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&sh->tmem)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sh->tmem;
  const int my_cells = deal ? q_deal + ((int)blockIdx.x < r_deal ? 1 : 0)
                            : (nwork > (int)blockIdx.x ? (nwork - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0);
  const int rows8 = ((nc - 128 * (nmt - 1)) + 7) / 8 * 8;   // rows of the last M-tile, in atoms
  const int64_t kcb = kc_block_bytes(nmt, rows8);

  if (warp == 0) {
    // ------------------------------------------------------------ A producer
    if (lane == 0) {
      uint32_t ta = 0;
      bool go = true;
      for (int i = 0; i < my_cells && go; ++i) {
        int64_t cell;
        const uint8_t* A = item_of(i, cell).A;
        for (int kc = 0; kc < nkc && go; ++kc)
          for (int mt = 0; mt < nmt; ++mt, ++ta) {
            const int s = ta % kLand;
            if (!mbar_wait(&sh->land_empty[s], ((ta / kLand) & 1) ^ 1, abort, err)) { go = false; break; }
            const uint32_t full = smem_u32(&sh->land_full[s]);
            const uint32_t bytes = mt == nmt - 1 ? (uint32_t)rows8 * 128u : (uint32_t)kTile;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(full), "r"(bytes) : "memory");
            const uint8_t* src = A + (cell * nkc + kc) * kcb + (int64_t)mt * kTile;
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(smem_u32(sL + s * kTile)), "l"(src), "r"(bytes), "r"(full) : "memory");
          }
      }
      // drain: every issued copy has landed before the CTA may exit
      for (uint32_t t = (ta > (uint32_t)kLand ? ta - kLand : 0); t < ta; ++t) {
        volatile int no_abort = 0;
        mbar_wait(&sh->land_full[t % kLand], (t / kLand) & 1, &no_abort, err);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t ta = 0, tb = 0;
      bool go = true;
      for (int i = 0; i < my_cells && go; ++i) {
        for (int kc = 0; kc < nkc && go; ++kc, ++tb) {
          const int sb = tb % kStagesB;
          if (!mbar_wait(&sh->b_full[sb], (tb / kStagesB) & 1, abort, err)) { go = false; break; }
          const uint32_t bhi = smem_u32(sB + sb * kStage), blo = bhi + kTile;
          for (int mt = 0; mt < nmt; ++mt, ++ta) {
            const int sa = ta % kConv;
            if (kc == 0 && !mbar_wait(&sh->acc_empty[mt], (i & 1) ^ 1, abort, err)) { go = false; break; }
            if (!mbar_wait(&sh->conv_full[sa], (ta / kConv) & 1, abort, err)) { go = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t d = tmem + (uint32_t)(mt * 128);
            if constexpr (ATMEM) {
              const uint32_t ahi = tmem + kAcolBase + (uint32_t)(sa * 64), alo = ahi + 32;
#pragma unroll
              for (int ks = 0; ks < 4; ++ks) {
                const uint32_t o = ks * 32;
                mma_ts(d, ahi + 8 * ks, sdesc(bhi + o), (kc > 0 || ks > 0) ? 1u : 0u);
                mma_ts(d, ahi + 8 * ks, sdesc(blo + o), 1u);
                mma_ts(d, alo + 8 * ks, sdesc(bhi + o), 1u);
              }
            } else {
              const uint32_t ahi = smem_u32(sC + sa * kStage), alo = ahi + kTile;
#pragma unroll
              for (int ks = 0; ks < 4; ++ks) {
                const uint32_t o = ks * 32;
                mx::mma<true>(d, sdesc(ahi + o), sdesc(bhi + o), (kc > 0 || ks > 0) ? 1u : 0u);
                mx::mma<true>(d, sdesc(ahi + o), sdesc(blo + o), 1u);
                mx::mma<true>(d, sdesc(alo + o), sdesc(bhi + o), 1u);
              }
            }
            tc_commit(&sh->conv_empty[sa]);
          }
          if (go) tc_commit(&sh->b_empty[sb]);
        }
        if (go) tc_commit(&sh->acc_full);
      }
      // drain: all issued MMAs complete before tensor memory is released
      tc_commit(&sh->drain);
      volatile int no_abort = 0;
      mbar_wait(&sh->drain, 0, &no_abort, err);
    }
  } else if (warp >= 2 && warp < 6) {
    // ------------------------------------------------------------ B producers
    // warp w gathers columns col0 + 32 w .. +31 of the chunk's 32 rows into its 4 KB slice of
    // the stage's lo slot (row i of the chunk at byte 128 i), each lane copying 16 bytes of
    // one row per instruction; the slice is exactly where the warp's 32 rows of the lo B
    // tile go, so the split overwrites only what the warp itself staged.  Lane l holds the
    // node of row l of the next chunk to issue (loaded one chunk ahead) and hands it to the
    // lanes that copy that row by a shuffle.
    constexpr int kAhead = kStagesB - 1;
    const int w = warp - 2;
    const int n = 32 * w + lane;
    const uint32_t nchunks = (uint32_t)my_cells * (uint32_t)nkc;
    auto node_of = [&](uint32_t t) -> int {
      if (t >= nchunks) return 0;
      int64_t cell;
      const Item it = item_of(t / nkc, cell);
      const int k = (int)(t % nkc) * 32 + lane;
      return k < nc ? __ldg(it.map + cell * nc + k) : 0;
    };
    int node_next = node_of(0);
    auto issue = [&](uint32_t t) -> bool {
      const int sb = t % kStagesB;
      const int node_t = node_next;
      node_next = node_of(t + 1);                       // the next chunk's nodes, in flight
      if (!mbar_wait(&sh->b_empty[sb], ((t / kStagesB) & 1) ^ 1, abort, err)) return false;
      int64_t cell;
      const Item it = item_of(t / nkc, cell);
      const int kc = (int)(t % nkc);
      const uint32_t dst = smem_u32(sB + sb * kStage + kTile + w * 4096);
      const int seg = lane & 7;
      const int c = it.col0 + 32 * w + 4 * seg;
      const int cvalid = min(max(it.ncol - c, 0), 4) * 4;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int row = 4 * j + (lane >> 3);
        const int node = __shfl_sync(0xffffffffu, node_t, row);
        const bool ok = kc * 32 + row < nc && cvalid > 0;
        const float* src = ok ? it.X + (int64_t)node * it.ldx + c : it.X;
        cp_async16(dst + row * 128 + seg * 16, src, ok ? (uint32_t)cvalid : 0u);
      }
      return true;
    };
    bool go = true;
    for (uint32_t t = 0; t < (uint32_t)kAhead; ++t) {
      if (go && t < nchunks) go = issue(t);
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (uint32_t tb = 0; tb < nchunks && go; ++tb) {
      // every group but the newest kAhead - 1 complete: chunk tb has landed
      asm volatile("cp.async.wait_group %0;" :: "n"(kAhead - 1) : "memory");
      __syncwarp();
      const int sb = tb % kStagesB;
      uint8_t* bhi = sB + sb * kStage;
      uint8_t* blo = bhi + kTile;
      const float* raw = reinterpret_cast<const float*>(blo + w * 4096);
      float v[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = raw[k * 32 + lane];
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        uint4 hi, lo;
        tc::split_tf32_bits(__float_as_uint(v[4 * q]), hi.x, lo.x);
        tc::split_tf32_bits(__float_as_uint(v[4 * q + 1]), hi.y, lo.y);
        tc::split_tf32_bits(__float_as_uint(v[4 * q + 2]), hi.z, lo.z);
        tc::split_tf32_bits(__float_as_uint(v[4 * q + 3]), hi.w, lo.w);
        const uint32_t off = sw128((uint32_t)n, (uint32_t)(q * 16));
        *reinterpret_cast<uint4*>(bhi + off) = hi;
        *reinterpret_cast<uint4*>(blo + off) = lo;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&sh->b_full[sb]);
      if (tb + kAhead < nchunks) go = issue(tb + kAhead);
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp >= 6 && warp < 10) {
    // ------------------------------------------------------------ epilogue
    // lane = accumulator row: 32 consecutive columns of the row per tcgen05.ld, written as
    // four 32-byte stores (one full sector each) into the row of Y^c
    const int q = warp & 3;                       // TMEM lane quadrant of this warp
    for (int i = 0; i < my_cells; ++i) {
      if (!mbar_wait(&sh->acc_full, i & 1, abort, err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int64_t cell;
      float* Yc = item_of(i, cell).Yc;
      for (int mt = 0; mt < nmt; ++mt) {
        const int row = mt * 128 + q * 32 + lane;
        const bool any = mt * 128 + q * 32 < nc;  // warp-uniform: the quadrant holds rows
        for (int cb = 0; cb < 4 && any; ++cb) {
          uint32_t r[32];
          tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(mt * 128 + cb * 32), r);
          if (row < nc) {
            float* y = Yc + (cell * nc + row) * (int64_t)128 + cb * 32;
#pragma unroll
            for (int j = 0; j < 32; j += 8)
              asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                           :: "l"(y + j), "r"(r[j]), "r"(r[j + 1]), "r"(r[j + 2]), "r"(r[j + 3]), "r"(r[j + 4]),
                              "r"(r[j + 5]), "r"(r[j + 6]), "r"(r[j + 7]) : "memory");
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&sh->acc_empty[mt]);
      }
    }
  } else {
    // ------------------------------------------------------------ A converters
    const int tid = threadIdx.x - 320;            // 0 .. 127
    const int q = warp & 3;                       // TMEM lane quadrant (ATMEM)
    const uint32_t row = (uint32_t)(32 * q + lane);   // the tile row this thread converts (ATMEM)
    uint32_t ta = 0;
    bool go = true;
    for (int i = 0; i < my_cells && go; ++i)
      for (int kc = 0; kc < nkc && go; ++kc)
        for (int mt = 0; mt < nmt; ++mt, ++ta) {
          const int s = ta % kLand, sc = ta % kConv;
          if (!mbar_wait(&sh->land_full[s], (ta / kLand) & 1, abort, err)) { go = false; break; }
          if (!mbar_wait(&sh->conv_empty[sc], ((ta / kConv) & 1) ^ 1, abort, err)) { go = false; break; }
          if constexpr (ATMEM) {
            // row `row` of the tile: its 32 values in K order from the swizzled landing tile;
            // rows of the last M-tile beyond the landed atoms hold whatever the slot held
            // before (possibly never written), so they enter tensor memory as zeros: measured
            // on GB300, non-finite stale values in such rows of a tensor-memory A operand
            // corrupted other rows of the product, although their own rows are never stored
            const uint8_t* L = sL + s * kTile;
            const bool landed = mt != nmt - 1 || (int)row < rows8;
            uint32_t hv[32], lv[32];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              uint4 u = make_uint4(0u, 0u, 0u, 0u);
              if (landed) u = *reinterpret_cast<const uint4*>(L + sw128(row, (uint32_t)(16 * c)));
              tc::split_tf32_bits(u.x, hv[4 * c], lv[4 * c]);
              tc::split_tf32_bits(u.y, hv[4 * c + 1], lv[4 * c + 1]);
              tc::split_tf32_bits(u.z, hv[4 * c + 2], lv[4 * c + 2]);
              tc::split_tf32_bits(u.w, hv[4 * c + 3], lv[4 * c + 3]);
            }
            // the landing slot may take the next bulk copy: the proxy fence orders these
            // ordinary shared-memory reads before that async-proxy write (measured on GB300:
            // without it the next tile overwrote rows still being read, at many cells per CTA)
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&sh->land_empty[s]);
            // the MMAs that read this A slot have completed (conv_empty): order the stores below
            // after that wait
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ta_hi = tmem + ((uint32_t)(32 * q) << 16) + kAcolBase + (uint32_t)(sc * 64);
            tmem_st32(ta_hi, hv);
            tmem_st32(ta_hi + 32, lv);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          } else {
            const int nchunk16 = (mt == nmt - 1 ? rows8 : 128) * 8;
            const uint4* src = reinterpret_cast<const uint4*>(sL + s * kTile);
            uint4* hi = reinterpret_cast<uint4*>(sC + sc * kStage);
            uint4* lo = reinterpret_cast<uint4*>(sC + sc * kStage + kTile);
            uint4 u[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int c = tid + 128 * j;
              if (c < nchunk16) u[j] = src[c];
            }
            // the landing slot may take the next bulk copy (async proxy) once these reads are
            // ordered before it
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&sh->land_empty[s]);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int c = tid + 128 * j;
              if (c < nchunk16) {
                uint4 h4, l4;
                tc::split_tf32_bits(u[j].x, h4.x, l4.x);
                tc::split_tf32_bits(u[j].y, h4.y, l4.y);
                tc::split_tf32_bits(u[j].z, h4.z, l4.z);
                tc::split_tf32_bits(u[j].w, h4.w, l4.w);
                hi[c] = h4;
                lo[c] = l4;
              }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          }
          mbar_arrive(&sh->conv_full[sc]);
        }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512));
}

// one launch in the given shape (the A-in-TMEM form needs at most three M-tiles beside the A
// slots; the default shape is that form where it fits, with round-robin dealing)
static void launch_cell_tf32p(cudaStream_t s, unsigned grid, const mp::Item& one, const mp::Item* items,
                              const int2* work, int nwork, int nc, int nkc, int nmt, int* err,
                              const MixedShape& shape = MixedShape{}) {
  if (nmt <= 3 && shape.atmem && shape.deep)
    DFTFE_LAUNCH((k_cell_tf32p<true, true>), grid, mp::kThreads, (mp::smem_bytes<true, true>()), s, one, items, work,
                 nwork, nc, nkc, nmt, shape.deal, err);
  else if (nmt <= 3 && shape.atmem)
    DFTFE_LAUNCH((k_cell_tf32p<true, false>), grid, mp::kThreads, (mp::smem_bytes<true, false>()), s, one, items,
                 work, nwork, nc, nkc, nmt, shape.deal, err);
  else
    DFTFE_LAUNCH((k_cell_tf32p<false, false>), grid, mp::kThreads, (mp::smem_bytes<false, false>()), s, one, items,
                 work, nwork, nc, nkc, nmt, shape.deal, err);
}

static bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  DFTFE_CHECK_CUDA(cudaStreamIsCapturing(s, &st));
  return st != cudaStreamCaptureStatusNone;
}

// The autotuner of the TF32x3 cell-product launch: every candidate shape (A operand in tensor
// memory where it fits, or in shared memory; round-robin or contiguous dealing; with
// work_alt, the interleaved work list too) runs once untimed and three times timed (CUDA
// events on the launch stream) on the launch's own operands, and the fastest is kept.  The
// launches only write the per-cell products, which the real launch that follows rewrites, so
// tuning changes no result.  The first candidate is the default shape.
static MixedShape tune_cell_tf32p(cudaStream_t s, int sm, const mp::Item& one, const mp::Item* items, const int2* work,
                                  const int2* work_alt, int nwork, int nc, int nkc, int nmt, int* err) {
  std::vector<MixedShape> cands;
  for (int order = 0; order < (work_alt ? 2 : 1); ++order)
    for (int atmem = (nmt <= 3 ? 1 : 0); atmem >= 0; --atmem)
      for (int deep = 0; deep < (atmem ? 2 : 1); ++deep)
        for (int deal = 0; deal < 2; ++deal) {
          MixedShape c;
          c.atmem = atmem;
          c.deep = deep;
          c.deal = deal;
          c.order = order;
          cands.push_back(c);
        }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  DFTFE_CHECK_CUDA(cudaEventCreate(&e0));
  DFTFE_CHECK_CUDA(cudaEventCreate(&e1));
  const unsigned grid = (unsigned)std::min(nwork, sm);
  MixedShape best = cands[0];
  double tbest = 1e300, tdef = 0.0;
  try {
    for (size_t ci = 0; ci < cands.size(); ++ci) {
      const MixedShape& c = cands[ci];
      const int2* w = c.order ? work_alt : work;
      launch_cell_tf32p(s, grid, one, items, w, nwork, nc, nkc, nmt, err, c);
      DFTFE_CHECK_CUDA(cudaEventRecord(e0, s));
      for (int r = 0; r < 3; ++r) launch_cell_tf32p(s, grid, one, items, w, nwork, nc, nkc, nmt, err, c);
      DFTFE_CHECK_CUDA(cudaEventRecord(e1, s));
      DFTFE_CHECK_CUDA(cudaEventSynchronize(e1));
      float ms = 0.0f;
      DFTFE_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      const double t = ms / 3.0;
      if (ci == 0) tdef = t;
      if (t < tbest) {
        tbest = t;
        best = c;
      }
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  best.best_ms = tbest;
  best.default_ms = tdef;
  return best;
}

static void set_tf32p_attrs() {
  DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_cell_tf32p<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)mp::smem_bytes<true, false>()));
  DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_cell_tf32p<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)mp::smem_bytes<true, true>()));
  DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_cell_tf32p<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)mp::smem_bytes<false, false>()));
}

// ------------------------------------------------------------ FP32 helpers

__global__ void k_to_f32(const double* __restrict__ X, int64_t ldx, float* __restrict__ Y, int64_t ldy,
                         int64_t M, int ncol) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= M * ncol) return;
  const int64_t i = t / ncol;
  const int j = (int)(t - i * ncol);
  Y[i * ldy + j] = __double2float_rn(X[i * ldx + j]);
}

__global__ void k_to_f64(const float* __restrict__ Y, int64_t ldy, double* __restrict__ X, int64_t ldx,
                         int64_t M, int ncol) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= M * ncol) return;
  const int64_t i = t / ncol;
  const int j = (int)(t - i * ncol);
  X[i * ldx + j] = (double)Y[i * ldy + j];
}

// Projector coefficients in two stages for parallelism: stage 1, CTA (a, s) sums split s
// of projector a's support (8 warps x 4 unrolled loads per lane); stage 2 adds the splits
// in a fixed order and scales by h_a.
constexpr int kNlSplits = 8;
__global__ void __launch_bounds__(256) k_nl_coef32_part(const float* __restrict__ X, int64_t ldx, int ncol,
                                                        const int64_t* __restrict__ prow,
                                                        const int32_t* __restrict__ pnode,
                                                        const double* __restrict__ pval, float* __restrict__ part) {
  // CTA (a, s): split s of projector a's support; warp w takes every 8th entry; lane l
  // holds columns 4l..4l+3 of a 128-column tile (blockIdx.y), read as one float4
  __shared__ float4 red[8][32];
  const int a = blockIdx.x / kNlSplits, sidx = blockIdx.x % kNlSplits;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c0 = blockIdx.y * 128 + 4 * lane;
  const int64_t e0 = prow[a], e1 = prow[a + 1];
  const int64_t len = (e1 - e0 + kNlSplits - 1) / kNlSplits;
  const int64_t s0 = e0 + sidx * len, s1 = min(e1, s0 + len);
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  if (c0 < ncol) {
    for (int64_t e = s0 + warp; e < s1; e += 8) {
      const float w = (float)pval[e];
      const float4 x = __ldg(reinterpret_cast<const float4*>(X + (int64_t)pnode[e] * ldx + c0));
      s.x = fmaf(w, x.x, s.x); s.y = fmaf(w, x.y, s.y); s.z = fmaf(w, x.z, s.z); s.w = fmaf(w, x.w, s.w);
    }
  }
  red[warp][lane] = s;
  __syncthreads();
  if (warp == 0) {
    float4 t = red[0][lane];
#pragma unroll
    for (int w = 1; w < 8; ++w) {
      const float4 u = red[w][lane];
      t.x += u.x; t.y += u.y; t.z += u.z; t.w += u.w;
    }
    const float v[4] = {t.x, t.y, t.z, t.w};
    for (int j = 0; j < 4; ++j)
      if (c0 + j < ncol) part[((int64_t)blockIdx.x) * ncol + c0 + j] = v[j];
  }
}

__global__ void k_nl_coef32_reduce(const float* __restrict__ part, const double* __restrict__ hcoup, int nproj,
                                   int ncol, float* __restrict__ P, int ldP) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nproj * ncol) return;
  const int a = (int)(t / ncol), col = (int)(t % ncol);
  float s = 0.0f;
  for (int k = 0; k < kNlSplits; ++k) s += part[((int64_t)a * kNlSplits + k) * ncol + col];
  P[(int64_t)a * ldP + col] = (float)hcoup[a] * s;
}


static unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

static size_t mixed_smem() {
  return 1024 + (size_t)mx::kStagesA * mx::kStageBytes + (size_t)mx::kStagesB * mx::kStageBytes + mx::kPatchBytes +
         sizeof(mx::Shared);
}

// build (once per potential and precision) the split cell-matrix tiles
static uint8_t* mixed_tiles(dftfe_ham h, bool tf32, int* nkc_out, int* nmt_out) {
  auto* m = h->mesh;
  const int es = tf32 ? 4 : 2, kc = 128 / es;
  const int nkc = (m->nc + kc - 1) / kc, nmt = (m->nc + 127) / 128;
  *nkc_out = nkc;
  *nmt_out = nmt;
  if (nmt > mx::kMaxMTiles) throw Error(DFTFE_ERR_ARG, "mixed precision supports at most 512 nodes per cell (p <= 7)");
  const int fmt = tf32 ? 1 : 0;
  dftfe_ham o = loc(h);                 // the owner of the cell matrices and their split forms
  if (tf32) {
    // TF32x3: one FP32 plane, split in shared memory by the kernel
    const int rows8 = ((m->nc - 128 * (nmt - 1)) + 7) / 8 * 8;
    const size_t bytes = (size_t)m->Nc * nkc * (size_t)mp::kc_block_bytes(nmt, rows8);
    uint8_t* A = (uint8_t*)ws_get(o, "mixed_plane_tf32", bytes);
    if (o->mixed_version[fmt] != o->potential_version) {
      DFTFE_LAUNCH(k_plane_cells, h->sm_count * 16, 256, 0, h->stream, o->d_Hc, (float*)A, m->Nc, m->nc, nkc, nmt,
                   rows8);
      o->mixed_version[fmt] = o->potential_version;
    }
    return A;
  }
  const char* name = "mixed_tiles_bf16";
  const size_t bytes = (size_t)m->Nc * nkc * nmt * 2 * mx::kTile;
  uint8_t* A = (uint8_t*)ws_get(o, name, bytes);
  if (o->mixed_version[fmt] != o->potential_version) {
    const int grid = h->sm_count * 16;
    if (tf32)
      DFTFE_LAUNCH(k_split_cells<true>, grid, 256, 0, h->stream, o->d_Hc, A, m->Nc, m->nc, nkc, nmt);
    else
      DFTFE_LAUNCH(k_split_cells<false>, grid, 256, 0, h->stream, o->d_Hc, A, m->Nc, m->nc, nkc, nmt);
    o->mixed_version[fmt] = o->potential_version;
  }
  return A;
}

// Assembly of the per-cell products fused with the recurrence and the nonlocal term:
//   Z[g] = s1 X[g] + s2 Xp[g] + alpha (sum_{slots (c, l) of node g} Y^c[l] + sum_t w_t P[a_t])
// one warp per node, lane l owns columns col0 + 4l .. +3 (float4); the slots of a node are
// summed in increasing cell order, so the result is deterministic.  P (nproj x ncol, FP32)
// (row stride ldP) holds h_a (C~^T X)_a; (a_t, w_t) are the node's projector entries (none off
// the supports).
__global__ void __launch_bounds__(256) k_assemble32(float* __restrict__ Z, int64_t ldz, const float* __restrict__ X,
                                                    int64_t ldx, const float* __restrict__ Xp, int64_t ldp,
                                                    const float* __restrict__ Yc, const int32_t* __restrict__ nptr,
                                                    const int32_t* __restrict__ nslot, const int64_t* __restrict__ nlptr,
                                                    const int32_t* __restrict__ nlproj, const double* __restrict__ nlval,
                                                    const float* __restrict__ P, int ldP, int64_t M, int col0,
                                                    int ncol, float alpha, float s1, float s2) {
  const int lane = threadIdx.x & 31;
  const int64_t g = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int c = col0 + 4 * lane;
  if (g >= M || c >= ncol) return;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int t = nptr[g]; t < nptr[g + 1]; ++t) {
    const float4 y = __ldg(reinterpret_cast<const float4*>(Yc + (int64_t)nslot[t] * 128 + 4 * lane));
    acc.x += y.x; acc.y += y.y; acc.z += y.z; acc.w += y.w;
  }
  if (nlptr) {
    for (int64_t t = nlptr[g]; t < nlptr[g + 1]; ++t) {
      const float w = (float)nlval[t];
      const float* pa = P + (int64_t)nlproj[t] * ldP + c;      // ldP % 4 == 0, c < ldP
      const float4 pv = *reinterpret_cast<const float4*>(pa);
      acc.x = fmaf(w, pv.x, acc.x); acc.y = fmaf(w, pv.y, acc.y);
      acc.z = fmaf(w, pv.z, acc.z); acc.w = fmaf(w, pv.w, acc.w);
    }
  }
  const float4 x = *reinterpret_cast<const float4*>(X + g * ldx + c);     // in bounds: ld % 32 == 0
  float4 o = make_float4(fmaf(alpha, acc.x, s1 * x.x), fmaf(alpha, acc.y, s1 * x.y),
                         fmaf(alpha, acc.z, s1 * x.z), fmaf(alpha, acc.w, s1 * x.w));
  if (Xp) {
    const float4 p = *reinterpret_cast<const float4*>(Xp + g * ldp + c);
    o.x = fmaf(s2, p.x, o.x); o.y = fmaf(s2, p.y, o.y); o.z = fmaf(s2, p.z, o.z); o.w = fmaf(s2, p.w, o.w);
  }
  float* z = Z + g * ldz + c;
  if (c + 3 < ncol) {
    *reinterpret_cast<float4*>(z) = o;
  } else {
    const float v[4] = {o.x, o.y, o.z, o.w};
    for (int j = 0; c + j < ncol; ++j) z[j] = v[j];
  }
}

// node -> (cell, local row) slots in CSR, cells in increasing order (built once per ham)
static void node_slots(dftfe_ham h, const int32_t** ptr, const int32_t** slots) {
  auto* m = h->mesh;
  if (!h->d_node_ptr) {
    // the cell map itself (cell c, local row l) -> node, read back once
    const int nc = m->nc;
    DFTFE_REQUIRE(m->Nc * (int64_t)nc < INT32_MAX, "too many cell rows for 32-bit slots");
    std::vector<int32_t> map((size_t)m->Nc * nc);
    DFTFE_CHECK_CUDA(cudaMemcpyAsync(map.data(), h->d_map, sizeof(int32_t) * map.size(), cudaMemcpyDeviceToHost,
                                     h->stream));
    DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    std::vector<int32_t> cnt(m->M + 1, 0);
    auto node_of = [&](int64_t c, int l) -> int64_t { return map[c * nc + l]; };
    for (int64_t c = 0; c < m->Nc; ++c)
      for (int l = 0; l < nc; ++l) cnt[node_of(c, l) + 1]++;
    for (int64_t g = 0; g < m->M; ++g) cnt[g + 1] += cnt[g];
    std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1), sl((size_t)m->Nc * nc);
    for (int64_t c = 0; c < m->Nc; ++c)
      for (int l = 0; l < nc; ++l) sl[fill[node_of(c, l)]++] = (int32_t)(c * nc + l);
    DFTFE_CHECK_CUDA(cudaMalloc(&h->d_node_ptr, sizeof(int32_t) * cnt.size()));
    DFTFE_CHECK_CUDA(cudaMalloc(&h->d_node_slot, sizeof(int32_t) * sl.size()));
    DFTFE_CHECK_CUDA(cudaMemcpy(h->d_node_ptr, cnt.data(), sizeof(int32_t) * cnt.size(), cudaMemcpyHostToDevice));
    DFTFE_CHECK_CUDA(cudaMemcpy(h->d_node_slot, sl.data(), sizeof(int32_t) * sl.size(), cudaMemcpyHostToDevice));
  }
  *ptr = h->d_node_ptr;
  *slots = h->d_node_slot;
}

// Z = alpha H~ X + s1 X + s2 Xp on FP32 blocks (ld multiple of 32), mixed cell products:
// per 128-column tile, one launch of the cell kernel over all cells (per-cell outputs,
// plain stores) and one assembly launch; then the nonlocal part.
// kpoint: X, Xp, Z are the real views of complex blocks (ncol real columns): the real nonlocal
// term is left out and the k-dependent terms (1/2|k|^2, -i k.grad, complex nonlocal) are
// added after the assembly in FP32 (kpoint_add32).
static void apply_combo_mixed(dftfe_ham h, bool tf32, const uint8_t* A, int nkc, int nmt, const float* X, int64_t ldx,
                              const float* Xp, int64_t ldp, float* Z, int64_t ldz, int ncol, float alpha, float s1,
                              float s2, int* err, bool kpoint = false) {
  auto* m = h->mesh;
  if (kpoint) {
    const double k2 = h->kvec[0] * h->kvec[0] + h->kvec[1] * h->kvec[1] + h->kvec[2] * h->kvec[2];
    s1 += (float)(0.5 * (double)alpha * k2);
  }
  const int32_t *nptr, *nslot;
  node_slots(h, &nptr, &nslot);
  float* Yc = (float*)ws_get(h, "mx_yc", sizeof(float) * (size_t)m->Nc * m->nc * 128);
  const size_t sh = mixed_smem();
  const unsigned grid = (unsigned)std::min<int64_t>(m->Nc, h->sm_count);
  // nonlocal coefficients P = h (C~^T X) first: the assembly adds C~ P with the cell sums
  float* P = nullptr;
  const int ldP = (ncol + 3) / 4 * 4;
  if (h->nproj > 0 && !kpoint) {
    P = (float*)ws_get(h, "nl_coef32", sizeof(float) * h->nproj * (size_t)ldP);
    float* Pp = (float*)ws_get(h, "nl_coef32_part", sizeof(float) * h->nproj * (size_t)kNlSplits * ncol);
    dim3 g1((unsigned)(h->nproj * kNlSplits), (unsigned)((ncol + 127) / 128));
    DFTFE_LAUNCH(k_nl_coef32_part, g1, 256, 0, h->stream, X, ldx, ncol, h->d_prow, h->d_pnode, h->d_pval, Pp);
    DFTFE_LAUNCH(k_nl_coef32_reduce, nblk((int64_t)h->nproj * ncol), 256, 0, h->stream, Pp, h->d_h, h->nproj,
                 ncol, P, ldP);
  }
  for (int col0 = 0; col0 < ncol; col0 += 128) {
    {
      ProfScope ps(h, tf32 ? "cell_gemm_tf32x3" : "cell_gemm_bf16x3");
      if (tf32) {
        const mp::Item one{A, h->d_map, X, Yc, ldx, col0, ncol};
        if (h->autotune && !h->tuned_mixed_done && !capturing(h->stream)) {
          h->tuned_mixed = tune_cell_tf32p(h->stream, h->sm_count, one, nullptr, nullptr, nullptr, (int)m->Nc, m->nc,
                                           nkc, nmt, err);
          h->tuned_mixed_done = true;
        }
        launch_cell_tf32p(h->stream, grid, one, nullptr, nullptr, (int)m->Nc, m->nc, nkc, nmt, err,
                          h->autotune && h->tuned_mixed_done ? h->tuned_mixed : MixedShape{});
      } else
        DFTFE_LAUNCH(k_cell_mixed<false>, grid, mx::kThreads, sh, h->stream, A, h->d_map, (int)m->Nc, m->nc,
                     nkc, nmt, X, ldx, Yc, col0, ncol, err);
    }
    ProfScope ps(h, "assemble32");
    DFTFE_LAUNCH(k_assemble32, nblk((m->M + 7) / 8 * 256), 256, 0, h->stream, Z, ldz, X, ldx, Xp, ldp, Yc, nptr, nslot,
                 P ? h->d_nptr_all : nullptr, h->d_sproj, h->d_sval, P, ldP, m->M, col0, ncol, alpha, s1, s2);
  }
  if (kpoint) kpoint_add32(h, X, ldx, Z, ldz, ncol / 2, alpha);
}

static bool g_mixed_attr = false;

// Eq. chebyfilter with FP32 vectors and split-precision cell products; the caller's FP64
// block is converted in and out.
void chebyshev_filter_mixed(dftfe_ham h, double* X, int64_t ld, int ncol, int degree, const dftfe_bounds& b,
                            bool tf32, int* ext_err, bool kpoint) {
  if (degree <= 0 || ncol <= 0) return;
  auto* m = h->mesh;
  if (!g_mixed_attr) {
    set_tf32p_attrs();
    DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_cell_mixed<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mixed_smem()));
    g_mixed_attr = true;
  }
  int nkc, nmt;
  const uint8_t* A = mixed_tiles(h, tf32, &nkc, &nmt);
  const int64_t ld32 = (ncol + 31) / 32 * 32;
  float* buf[3];
  buf[0] = (float*)ws_get(h, "mx_v0", sizeof(float) * m->M * (size_t)ld32);
  buf[1] = (float*)ws_get(h, "mx_v1", sizeof(float) * m->M * (size_t)ld32);
  buf[2] = (float*)ws_get(h, "mx_v2", sizeof(float) * m->M * (size_t)ld32);
  // with ext_err the caller owns the timeout flag (zeroed and read by the caller, so a whole
  // pass can be enqueued, or captured in a graph, without a host read in between)
  int* err = ext_err ? ext_err : (int*)ws_get(h, "mx_err", sizeof(int));
  if (!ext_err) DFTFE_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), h->stream));
  DFTFE_LAUNCH(k_to_f32, nblk(m->M * ncol), 256, 0, h->stream, X, ld, buf[0], ld32, m->M, ncol);
  const double e = (b.b - b.a) / 2.0, c = (b.b + b.a) / 2.0;
  const bool scaled = !std::isnan(b.a0);
  double sigma = scaled ? e / (b.a0 - c) : 0.0;
  const double sigma1 = sigma, gamma = scaled ? 2.0 / sigma1 : 0.0;
  int cur = 0, prev = -1;
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
    apply_combo_mixed(h, tf32, A, nkc, nmt, buf[cur], ld32, prev >= 0 ? buf[prev] : nullptr, ld32, buf[out], ld32,
                      ncol, (float)alpha, (float)s1, (float)s2, err, kpoint);
    prev = cur;
    cur = out;
  }
  DFTFE_LAUNCH(k_to_f64, nblk(m->M * ncol), 256, 0, h->stream, buf[cur], ld32, X, ld, m->M, ncol);
  if (ext_err) return;
  int herr = 0;
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  if (herr) throw Error(DFTFE_ERR_TIMEOUT, "mixed cell kernel: a bounded wait timed out");
}

// Batched TF32x3 filter: per round, one block of every system (X_s, ld_s, ncol_s real
// columns -- the real view of a complex block for a k-point item), each with its own degree
// and bounds.  Per Chebyshev step and 128-column tile, ONE persistent cell-product launch per
// degree group covers every cell of every system still filtering (a work list of
// (system, cell) pairs); the nonlocal coefficients, the assembly fused with the recurrence
// and the k-point terms run per system.  Each system's operations, and their order, are
// those of its single-system filter, so the results are bit-identical to it.  Planning forms
// the launch descriptors of every round on the host and uploads them once; the returned
// closure enqueues all launches with no host work in between (it can be captured as one
// CUDA graph).
namespace {
struct MixedRoundPlan {
  struct Sys {
    const uint8_t* A = nullptr;
    int nkc = 0, nmt = 0;
    const int32_t *nptr = nullptr, *nslot = nullptr;
    float* Yc = nullptr;
    float* buf[3] = {nullptr, nullptr, nullptr};
    int64_t ld32 = 0;
  };
  struct StepSys {
    int cur, prev, out;
    float alpha, s1, s2;
  };
  struct CellLaunch {
    int k, tile, nc, nkc, nmt;
    size_t item_off, work_off, work_off_alt;   // system-major and interleaved work lists
    int nwork, nitems;
    MixedShape shape;
  };
  std::vector<MixedBlock> blk;
  std::vector<Sys> sy;
  std::vector<std::vector<StepSys>> steps;
  std::vector<CellLaunch> launches;
  int maxdeg = 0, ntiles = 0;
  size_t item_base = 0, work_base = 0;     // element offsets of the round in the uploads
};
}  // namespace

static void plan_mixed_round(MixedRoundPlan& R, std::vector<mp::Item>& items, std::vector<int2>& work) {
  std::vector<MixedBlock>& blk = R.blk;
  const int ns = (int)blk.size();
  if (!g_mixed_attr) {
    set_tf32p_attrs();
    DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_cell_mixed<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mixed_smem()));
    g_mixed_attr = true;
  }
  using Sys = MixedRoundPlan::Sys;
  using StepSys = MixedRoundPlan::StepSys;
  using CellLaunch = MixedRoundPlan::CellLaunch;
  std::vector<Sys>& sy = R.sy;
  sy.assign(ns, Sys{});
  int& maxdeg = R.maxdeg;
  int& ntiles = R.ntiles;
  for (int s = 0; s < ns; ++s) {
    const MixedBlock& b = blk[s];
    if (b.degree <= 0 || b.ncol <= 0) continue;
    dftfe_ham h = b.h;
    auto* m = h->mesh;
    Sys& y = sy[s];
    y.A = mixed_tiles(h, true, &y.nkc, &y.nmt);
    node_slots(h, &y.nptr, &y.nslot);
    y.Yc = (float*)ws_get(h, "mx_yc", sizeof(float) * (size_t)m->Nc * m->nc * 128);
    y.ld32 = (b.ncol + 31) / 32 * 32;
    y.buf[0] = (float*)ws_get(h, "mx_v0", sizeof(float) * m->M * (size_t)y.ld32);
    y.buf[1] = (float*)ws_get(h, "mx_v1", sizeof(float) * m->M * (size_t)y.ld32);
    y.buf[2] = (float*)ws_get(h, "mx_v2", sizeof(float) * m->M * (size_t)y.ld32);
    maxdeg = std::max(maxdeg, b.degree);
    ntiles = std::max(ntiles, (b.ncol + 127) / 128);
  }
  // buffer rotation and recurrence coefficients of every system and step, as the single filter
  // forms them
  std::vector<std::vector<StepSys>>& steps = R.steps;
  steps.assign(ns, {});
  for (int s = 0; s < ns; ++s) {
    const MixedBlock& bb = blk[s];
    if (bb.degree <= 0 || bb.ncol <= 0) continue;
    const dftfe_bounds& b = bb.b;
    const double e = (b.b - b.a) / 2.0, c = (b.b + b.a) / 2.0;
    const bool scaled = !std::isnan(b.a0);
    double sigma = scaled ? e / (b.a0 - c) : 0.0;
    const double sigma1 = sigma, gamma = scaled ? 2.0 / sigma1 : 0.0;
    int cur = 0, prev = -1;
    for (int k = 1; k <= bb.degree; ++k) {
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
      StepSys st{cur, prev, out, (float)alpha, (float)s1, (float)s2};
      if (bb.kpoint) {
        const double* kv = bb.h->kvec;
        const double k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2];
        st.s1 += (float)(0.5 * (double)st.alpha * k2);
      }
      steps[s].push_back(st);
      prev = cur;
      cur = out;
    }
  }
  // launch descriptors: per (step, tile, degree group) the items of the systems still
  // filtering, and one work list per distinct set of systems
  std::map<std::vector<int>, std::pair<size_t, int>> lists;
  std::map<std::vector<int>, size_t> lists_alt;
  std::vector<CellLaunch>& launches = R.launches;
  launches.clear();
  std::vector<int> ncs;
  for (int s = 0; s < ns; ++s)
    if (!steps[s].empty() && std::find(ncs.begin(), ncs.end(), blk[s].h->mesh->nc) == ncs.end())
      ncs.push_back(blk[s].h->mesh->nc);
  for (int k = 1; k <= maxdeg; ++k)
    for (int t = 0; t < ntiles; ++t)
      for (int nc : ncs) {
        std::vector<int> act;
        for (int s = 0; s < ns; ++s)
          if ((int)steps[s].size() >= k && blk[s].h->mesh->nc == nc && blk[s].ncol > 128 * t) act.push_back(s);
        if (act.empty()) continue;
        CellLaunch L{k, t, nc, sy[act[0]].nkc, sy[act[0]].nmt, items.size() - R.item_base, 0, 0, 0,
                     (int)act.size(), MixedShape{}};
        for (int s : act) {
          const StepSys& st = steps[s][k - 1];
          items.push_back(mp::Item{sy[s].A, blk[s].h->d_map, sy[s].buf[st.cur], sy[s].Yc, sy[s].ld32, 128 * t,
                                   blk[s].ncol});
        }
        auto it = lists.find(act);
        if (it == lists.end()) {
          const size_t off = work.size() - R.work_base;
          for (int li = 0; li < (int)act.size(); ++li) {
            const int64_t Nc = blk[act[li]].h->mesh->Nc;
            for (int64_t cidx = 0; cidx < Nc; ++cidx) work.push_back(make_int2(li, (int)cidx));
          }
          it = lists.emplace(act, std::make_pair(off, (int)(work.size() - R.work_base - off))).first;
          // the same pairs interleaved: cell 0 of every system, then cell 1, ...
          const size_t off_alt = work.size() - R.work_base;
          int64_t ncmax = 0;
          for (int s : act) ncmax = std::max<int64_t>(ncmax, blk[s].h->mesh->Nc);
          for (int64_t cidx = 0; cidx < ncmax; ++cidx)
            for (int li = 0; li < (int)act.size(); ++li)
              if (cidx < blk[act[li]].h->mesh->Nc) work.push_back(make_int2(li, (int)cidx));
          lists_alt.emplace(act, off_alt);
        }
        L.work_off = it->second.first;
        L.work_off_alt = lists_alt.at(act);
        L.nwork = it->second.second;
        launches.push_back(L);
      }
}

static void enqueue_mixed_round(const MixedRoundPlan& R, cudaStream_t stream, int* err, const mp::Item* d_items,
                                const int2* d_work) {
  using StepSys = MixedRoundPlan::StepSys;
  using CellLaunch = MixedRoundPlan::CellLaunch;
  const std::vector<MixedBlock>& blk = R.blk;
  const int ns = (int)blk.size();
  const auto& sy = R.sy;
  const auto& steps = R.steps;
  const auto& launches = R.launches;
  const int maxdeg = R.maxdeg, ntiles = R.ntiles;
  if (maxdeg == 0) return;
  const int sm = blk[0].h->sm_count;

  for (int s = 0; s < ns; ++s)
    if (!steps[s].empty()) {
      auto* m = blk[s].h->mesh;
      DFTFE_LAUNCH(k_to_f32, nblk(m->M * blk[s].ncol), 256, 0, stream, blk[s].X, blk[s].ld, sy[s].buf[0], sy[s].ld32,
                   m->M, blk[s].ncol);
    }
  size_t li = 0;
  for (int k = 1; k <= maxdeg; ++k) {
    // nonlocal coefficients P = h (C~^T X) of the Gamma-point systems with projectors
    std::vector<float*> P(ns, nullptr);
    std::vector<int> ldP(ns, 0);
    for (int s = 0; s < ns; ++s) {
      if ((int)steps[s].size() < k) continue;
      dftfe_ham h = blk[s].h;
      if (h->nproj <= 0 || blk[s].kpoint) continue;
      const int ncol = blk[s].ncol;
      ldP[s] = (ncol + 3) / 4 * 4;
      P[s] = (float*)ws_get(h, "nl_coef32", sizeof(float) * h->nproj * (size_t)ldP[s]);
      float* Pp = (float*)ws_get(h, "nl_coef32_part", sizeof(float) * h->nproj * (size_t)kNlSplits * ncol);
      const StepSys& st = steps[s][k - 1];
      dim3 g1((unsigned)(h->nproj * kNlSplits), (unsigned)((ncol + 127) / 128));
      DFTFE_LAUNCH(k_nl_coef32_part, g1, 256, 0, stream, sy[s].buf[st.cur], sy[s].ld32, ncol, h->d_prow, h->d_pnode,
                   h->d_pval, Pp);
      DFTFE_LAUNCH(k_nl_coef32_reduce, nblk((int64_t)h->nproj * ncol), 256, 0, stream, Pp, h->d_h, h->nproj, ncol,
                   P[s], ldP[s]);
    }
    for (int t = 0; t < ntiles; ++t) {
      for (; li < launches.size() && launches[li].k == k && launches[li].tile == t; ++li) {
        const CellLaunch& L = launches[li];
        ProfScope ps(blk[0].h, "batch_cell_tf32x3");
        const mp::Item none{};
        launch_cell_tf32p(stream, (unsigned)std::min(L.nwork, sm), none, d_items + R.item_base + L.item_off,
                          d_work + R.work_base + (L.shape.order ? L.work_off_alt : L.work_off), L.nwork, L.nc, L.nkc,
                          L.nmt, err, L.shape);
      }
      for (int s = 0; s < ns; ++s) {
        if ((int)steps[s].size() < k || blk[s].ncol <= 128 * t) continue;
        dftfe_ham h = blk[s].h;
        auto* m = h->mesh;
        const StepSys& st = steps[s][k - 1];
        float* const* b3 = sy[s].buf;
        const int64_t l = sy[s].ld32;
        ProfScope ps(h, "batch_assemble32");
        DFTFE_LAUNCH(k_assemble32, nblk((m->M + 7) / 8 * 256), 256, 0, stream, b3[st.out], l, b3[st.cur], l,
                     st.prev >= 0 ? b3[st.prev] : nullptr, l, sy[s].Yc, sy[s].nptr, sy[s].nslot,
                     P[s] ? h->d_nptr_all : nullptr, h->d_sproj, h->d_sval, P[s], ldP[s], m->M, 128 * t, blk[s].ncol,
                     st.alpha, st.s1, st.s2);
      }
    }
    for (int s = 0; s < ns; ++s) {
      if ((int)steps[s].size() < k || !blk[s].kpoint) continue;
      const StepSys& st = steps[s][k - 1];
      kpoint_add32(blk[s].h, sy[s].buf[st.cur], sy[s].ld32, sy[s].buf[st.out], sy[s].ld32, blk[s].ncol / 2, st.alpha);
    }
  }
  for (int s = 0; s < ns; ++s)
    if (!steps[s].empty()) {
      auto* m = blk[s].h->mesh;
      DFTFE_LAUNCH(k_to_f64, nblk(m->M * blk[s].ncol), 256, 0, stream, sy[s].buf[steps[s].back().out], sy[s].ld32,
                   blk[s].X, blk[s].ld, m->M, blk[s].ncol);
    }
}

std::function<void()> plan_mixed_batch(const std::vector<std::vector<MixedBlock>>& rounds, cudaStream_t stream,
                                       int* err, DevBuf& desc, std::vector<uint8_t>& host_desc,
                                       std::map<std::string, MixedShape>* tuned) {
  if (!g_mixed_attr) {
    set_tf32p_attrs();
    DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_cell_mixed<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mixed_smem()));
    g_mixed_attr = true;
  }
  auto plans = std::make_shared<std::vector<MixedRoundPlan>>(rounds.size());
  std::vector<mp::Item> items;
  std::vector<int2> work;
  for (size_t j = 0; j < rounds.size(); ++j) {
    MixedRoundPlan& R = (*plans)[j];
    R.blk = rounds[j];
    R.item_base = items.size();
    R.work_base = work.size();
    plan_mixed_round(R, items, work);
  }
  const size_t ib = items.size() * sizeof(mp::Item), wb = work.size() * sizeof(int2);
  const size_t woff = (ib + 255) / 256 * 256;
  host_desc.resize(std::max<size_t>(woff + wb, 1));
  if (ib) std::memcpy(host_desc.data(), items.data(), ib);
  if (wb) std::memcpy(host_desc.data() + woff, work.data(), wb);
  uint8_t* ddesc = (uint8_t*)desc.get(host_desc.size());
  // from pageable memory: the call returns once the data is staged, so the host copy may be
  // rewritten by the next pass
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(ddesc, host_desc.data(), host_desc.size(), cudaMemcpyHostToDevice, stream));
  const mp::Item* d_items = reinterpret_cast<const mp::Item*>(ddesc);
  const int2* d_work = reinterpret_cast<const int2*>(ddesc + woff);
  // launch shapes: the tuned shape of each distinct launch (FE degree, systems, work items),
  // timed on its first appearance when the batch tunes, else the default shape
  if (tuned) {
    const int sm = rounds.empty() || rounds[0].empty() ? 1 : rounds[0][0].h->sm_count;
    for (MixedRoundPlan& R : *plans)
      for (auto& L : R.launches) {
        // key: FE degree (nodes per cell), work items, systems and distinct cell-matrix planes
        std::vector<const uint8_t*> planes;
        for (int q = 0; q < L.nitems; ++q) planes.push_back(items[R.item_base + L.item_off + q].A);
        std::sort(planes.begin(), planes.end());
        const size_t nplanes = (size_t)(std::unique(planes.begin(), planes.end()) - planes.begin());
        const std::string key = std::to_string(L.nc) + "/" + std::to_string(L.nwork) + "/" +
                                std::to_string(L.nitems) + "/" + std::to_string(nplanes);
        auto it = tuned->find(key);
        if (it == tuned->end()) {
          if (capturing(stream)) continue;
          const mp::Item none{};
          MixedShape sh = tune_cell_tf32p(stream, sm, none, d_items + R.item_base + L.item_off,
                                          d_work + R.work_base + L.work_off, d_work + R.work_base + L.work_off_alt,
                                          L.nwork, L.nc, L.nkc, L.nmt, err);
          it = tuned->emplace(key, sh).first;
        }
        L.shape = it->second;
      }
  }
  return [plans, stream, err, d_items, d_work]() {
    for (const MixedRoundPlan& R : *plans) enqueue_mixed_round(R, stream, err, d_items, d_work);
  };
}

// Y = H~ X with the mixed cell products (FP64 in and out, FP32 inside); for parity tests.
void apply_mixed(dftfe_ham h, const double* X, int64_t ldx, double* Y, int64_t ldy, int ncol, bool tf32, bool kpoint) {
  auto* m = h->mesh;
  if (!g_mixed_attr) {
    set_tf32p_attrs();
    DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_cell_mixed<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mixed_smem()));
    g_mixed_attr = true;
  }
  int nkc, nmt;
  const uint8_t* A = mixed_tiles(h, tf32, &nkc, &nmt);
  const int64_t ld32 = (ncol + 31) / 32 * 32;
  float* x32 = (float*)ws_get(h, "mx_v0", sizeof(float) * m->M * (size_t)ld32);
  float* y32 = (float*)ws_get(h, "mx_v1", sizeof(float) * m->M * (size_t)ld32);
  int* err = (int*)ws_get(h, "mx_err", sizeof(int));
  DFTFE_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), h->stream));
  DFTFE_LAUNCH(k_to_f32, nblk(m->M * ncol), 256, 0, h->stream, X, ldx, x32, ld32, m->M, ncol);
  apply_combo_mixed(h, tf32, A, nkc, nmt, x32, ld32, nullptr, 0, y32, ld32, ncol, 1.0f, 0.0f, 0.0f, err, kpoint);
  DFTFE_LAUNCH(k_to_f64, nblk(m->M * ncol), 256, 0, h->stream, y32, ld32, Y, ldy, m->M, ncol);
  int herr = 0;
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  if (herr) throw Error(DFTFE_ERR_TIMEOUT, "mixed cell kernel: a bounded wait timed out");
}

}  // namespace dftfe

// ---------------------------------------------------------------------------------
// FP64-accurate H~X on the FP32 pipes (GB300 issues FP32 about 60x faster than FP64):
// each entry as an unevaluated pair of floats h = h_hi + h_lo, x likewise; a product is
// h_hi x_hi plus its exact rounding error (one FMA) plus the two cross terms, and the
// running sum is kept as a pair with Knuth's TwoSum, so the result carries about 44
// significant bits.  Same colour-ordered gather / cell product / scatter-add structure as
// the FP64 kernel; output FP64.
namespace dftfe {

__global__ void k_split_df(const double* __restrict__ Hc, float2* __restrict__ Hdf, int64_t n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double h = Hc[t];
  const float hi = __double2float_rn(h);
  Hdf[t] = make_float2(hi, __double2float_rn(h - (double)hi));
}

constexpr int DF_ROWS = 8;
__global__ void __launch_bounds__(256, 2) k_cell_df_wide(const float2* __restrict__ Hdf,
                                                         const int32_t* __restrict__ map,
                                                         const int32_t* __restrict__ cells, int nc,
                                                         const double* __restrict__ X, int64_t ldx,
                                                         double* __restrict__ Z, int64_t ldz, int ncol) {
  extern __shared__ float2 xs2[];                       // nc x 32 pairs
  int32_t* sm = (int32_t*)(xs2 + nc * 32);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t cell = cells[blockIdx.x];
  const int col = blockIdx.y * 32 + lane;
  const bool colok = col < ncol;
  const int32_t* m = map + cell * nc;
  for (int k = threadIdx.x; k < nc; k += 256) sm[k] = m[k];
  __syncthreads();
  for (int k = warp; k < nc; k += 8) {
    const double xd = colok ? X[(int64_t)sm[k] * ldx + col] : 0.0;
    const float hi = __double2float_rn(xd);
    xs2[k * 32 + lane] = make_float2(hi, __double2float_rn(xd - (double)hi));
  }
  __syncthreads();
  const float2* H = Hdf + cell * (int64_t)nc * nc;
  for (int r0 = warp * DF_ROWS; r0 < nc; r0 += 8 * DF_ROWS) {
    const int nr = min(DF_ROWS, nc - r0);
    float ah[DF_ROWS], al[DF_ROWS];
#pragma unroll
    for (int i = 0; i < DF_ROWS; ++i) ah[i] = al[i] = 0.0f;
    const float2* Hr = H + (int64_t)r0 * nc;
    // pair product + TwoSum: exact error of the leading product, cross terms, and the
    // rounding error of the running sum all go to the low word
#define DF_MAC(i)                                                   \
  {                                                                 \
    const float2 h = __ldg(Hr + (int64_t)(i) * nc + k);            \
    const float p = h.x * x.x;                                      \
    float e = fmaf(h.x, x.x, -p);                                   \
    e = fmaf(h.x, x.y, e);                                          \
    e = fmaf(h.y, x.x, e);                                          \
    const float s = ah[i] + p;                                      \
    const float bb = s - ah[i];                                     \
    const float err = (ah[i] - (s - bb)) + (p - bb);                \
    ah[i] = s;                                                      \
    al[i] += err + e;                                               \
  }
    if (nr == DF_ROWS) {
      for (int k = 0; k < nc; ++k) {
        const float2 x = xs2[k * 32 + lane];
#pragma unroll
        for (int i = 0; i < DF_ROWS; ++i) DF_MAC(i)
      }
    } else {
      for (int k = 0; k < nc; ++k) {
        const float2 x = xs2[k * 32 + lane];
#pragma unroll
        for (int i = 0; i < DF_ROWS; ++i)
          if (i < nr) DF_MAC(i)
      }
    }
#undef DF_MAC
    if (colok) {
#pragma unroll
      for (int i = 0; i < DF_ROWS; ++i)
        if (i < nr) Z[(int64_t)sm[r0 + i] * ldz + col] += (double)ah[i] + (double)al[i];
    }
  }
}

static unsigned nblk2(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Tiled float-pair cell products.  The cell matrix is stored k-major as pairs,
// Hk[cell][k][r] = H~^c[r][k] with rows padded to RP = 32 TM (zeros), and streamed in
// chunks of kDfKt values of k by bulk copies into a double buffer; X^c (32 columns) sits
// in shared memory as pairs.  Thread (rg, cg) = (lane, warp) owns rows rg + 32 i (i < TM)
// and columns 4 cg .. 4 cg + 3: per k it reads TM row entries (consecutive across the warp)
// and one broadcast 32-byte column group, then runs 4 TM independent pair products.
constexpr int kDfKt = 16;
constexpr long kDfSpin = 40000000L;

__global__ void k_split_df_k(const double* __restrict__ Hc, float2* __restrict__ Hk, int64_t Nc, int nc, int RP) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Nc * nc * RP) return;
  const int r = (int)(t % RP);
  const int64_t ck = t / RP;                 // cell * nc + k
  const int k = (int)(ck % nc);
  const int64_t cell = ck / nc;
  float2 v = make_float2(0.f, 0.f);
  if (r < nc) {
    const double h = Hc[(cell * nc + r) * nc + k];
    const float hi = __double2float_rn(h);
    v = make_float2(hi, __double2float_rn(h - (double)hi));
  }
  Hk[t] = v;
}

__device__ __forceinline__ bool df_wait(uint64_t* b, uint32_t parity, int* err) {
  const uint32_t addr = mx::smem_u32(b);
  for (long it = 0; it < kDfSpin; ++it) {
    uint32_t done;
    asm volatile("{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n selp.b32 %0, 1, 0, P1;\n}"
                 : "=r"(done) : "r"(addr), "r"(parity) : "memory");
    if (done) return true;
  }
  atomicExch(err, (int)DFTFE_ERR_TIMEOUT);
  return false;
}

template <int TM>
__global__ void __launch_bounds__(256, 1) k_cell_df_tiled(const float2* __restrict__ Hk,
                                                          const int32_t* __restrict__ map,
                                                          const int32_t* __restrict__ cells, int nc,
                                                          const double* __restrict__ X, int64_t ldx,
                                                          double* __restrict__ Z, int64_t ldz, int ncol, int* err) {
  constexpr int RP = 32 * TM;
  extern __shared__ __align__(16) uint8_t dsm[];
  // [0, hbytes): two H chunks (kDfKt x RP pairs each), later the output patch (RP x 33 doubles)
  constexpr size_t hbytes = (size_t)RP * 33 * 8 > (size_t)2 * kDfKt * RP * 8 ? (size_t)RP * 33 * 8
                                                                             : (size_t)2 * kDfKt * RP * 8;
  float2* hs = reinterpret_cast<float2*>(dsm);
  float2* xs = reinterpret_cast<float2*>(dsm + hbytes);           // nc x 32 pairs
  int32_t* sm = reinterpret_cast<int32_t*>(xs + (size_t)nc * 32);  // nc node ids
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + ((nc + 3) & ~3));  // 2 mbarriers (8-byte aligned)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t cell = cells[blockIdx.x];
  const int col0 = blockIdx.y * 32;
  const int nkt = (nc + kDfKt - 1) / kDfKt;
  const float2* Hc = Hk + cell * (int64_t)nc * RP;
  auto issue = [&](int t) {
    const int k0 = t * kDfKt;
    const uint32_t bytes = (uint32_t)(min(kDfKt, nc - k0) * RP * 8);
    const uint32_t b = mx::smem_u32(&bar[t & 1]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(b), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(mx::smem_u32(hs + (size_t)(t & 1) * kDfKt * RP)), "l"(Hc + (size_t)k0 * RP), "r"(bytes), "r"(b)
                 : "memory");
  };
  if (threadIdx.x == 0) {
    mx::mbar_init(&bar[0], 1);
    mx::mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    issue(0);
    if (nkt > 1) issue(1);
  }
  const int32_t* cm = map + cell * nc;
  for (int k = threadIdx.x; k < nc; k += 256) sm[k] = cm[k];
  __syncthreads();
  {
    // eight rows per warp in flight; the pair split keeps the FP64 pipe to one subtraction
    // (the narrowing and widening are integer operations)
    const int col = col0 + lane;
    for (int k0 = warp; k0 < nc; k0 += 64) {
      double xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = k0 + 8 * u;
        xv[u] = (k < nc && col < ncol) ? X[(int64_t)sm[k] * ldx + col] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = k0 + 8 * u;
        if (k < nc) {
          const float hi = tc::narrow_f64(xv[u]);
          xs[k * 32 + lane] = make_float2(hi, tc::narrow_f64(xv[u] - tc::widen_f32(hi)));
        }
      }
    }
  }
  __syncthreads();
  float ah[TM][4], al[TM][4];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) ah[i][j] = al[i][j] = 0.0f;
  bool ok = true;
  int issued = nkt > 1 ? 2 : 1;                    // chunks handed to the copy engine (thread 0)
  for (int t = 0; t < nkt && ok; ++t) {
    const bool got = df_wait(&bar[t & 1], (t >> 1) & 1, err);
    if (got) {
      const float2* hb = hs + (size_t)(t & 1) * kDfKt * RP + lane;
      const float2* xb = xs + (size_t)t * kDfKt * 32 + 4 * warp;
      const int kt = min(kDfKt, nc - t * kDfKt);
#pragma unroll 2
      for (int kk = 0; kk < kt; ++kk) {
        const float4 xa = *reinterpret_cast<const float4*>(xb + kk * 32);
        const float4 xc = *reinterpret_cast<const float4*>(xb + kk * 32 + 2);
        const float2 x[4] = {make_float2(xa.x, xa.y), make_float2(xa.z, xa.w), make_float2(xc.x, xc.y),
                             make_float2(xc.z, xc.w)};
#pragma unroll
        for (int i = 0; i < TM; ++i) {
          const float2 h = hb[kk * RP + 32 * i];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            // pair product (exact error of the leading term + cross terms) and TwoSum
            const float p = h.x * x[j].x;
            float e = fmaf(h.x, x[j].x, -p);
            e = fmaf(h.x, x[j].y, e);
            e = fmaf(h.y, x[j].x, e);
            const float s = ah[i][j] + p;
            const float bb = s - ah[i][j];
            const float er = (ah[i][j] - (s - bb)) + (p - bb);
            ah[i][j] = s;
            al[i][j] += er + e;
          }
        }
      }
    }
    ok = __syncthreads_and(got) != 0;               // chunk t fully read, by every thread
    if (threadIdx.x == 0 && ok && t + 2 < nkt) {
      issue(t + 2);
      issued = t + 3;
    }
  }
  if (!ok) {
    // let the copies still in flight land before shared memory is given up: the last
    // chunk issued into each buffer (bounded waits)
    if (threadIdx.x == 0)
      for (int t = max(0, issued - 2); t < issued; ++t) df_wait(&bar[t & 1], (t >> 1) & 1, err);
    __syncthreads();
    return;
  }
  // output patch over the (now idle) H buffers: RP x 33 doubles, then coalesced row updates
  double* out = reinterpret_cast<double*>(dsm);
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) out[(lane + 32 * i) * 33 + 4 * warp + j] = (double)ah[i][j] + (double)al[i][j];
  __syncthreads();
  const int col = col0 + lane;
  if (col < ncol)
    for (int r = warp; r < nc; r += 8) Z[(int64_t)sm[r] * ldz + col] += out[r * 33 + lane];
}

template <int TM>
static size_t df_tiled_smem(int nc) {
  const size_t RP = 32 * TM;
  const size_t hbytes = std::max(RP * 33 * 8, (size_t)2 * kDfKt * RP * 8);
  return hbytes + (size_t)nc * 32 * 8 + (size_t)((nc + 3) & ~3) * 4 + 16;
}

// Y = H~_nl X (with_nl) or 0, before the cell products add H~_loc X
static void df_init(dftfe_ham h, const double* X, int64_t ldx, double* Y, int64_t ldy, int ncol, bool with_nl) {
  if (with_nl) apply_nonlocal_fp64(h, X, ldx, Y, ldy, ncol);
  else zero_block(h->stream, Y, ldy, h->mesh->M, ncol);
}

template <int TM>
static bool apply_df_tiled(dftfe_ham h, const double* X, int64_t ldx, double* Y, int64_t ldy, int ncol, bool with_nl) {
  auto* m = h->mesh;
  const int nc = m->nc;
  if (nc > 32 * TM || nc <= 32 * (TM - 1)) return false;
  const size_t sh = df_tiled_smem<TM>(nc);
  if (sh > 227 * 1024) return false;
  static bool attr = false;
  if (!attr) {
    DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_cell_df_tiled<TM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr = true;
  }
  const int RP = 32 * TM;
  const size_t n2 = (size_t)m->Nc * nc * RP;
  dftfe_ham o = loc(h);
  float2* Hk = (float2*)ws_get(o, "cells_df_k", sizeof(float2) * n2);
  if (o->df_version != o->potential_version) {
    DFTFE_LAUNCH(k_split_df_k, nblk2((int64_t)n2), 256, 0, h->stream, o->d_Hc, Hk, (int64_t)m->Nc, nc, RP);
    o->df_version = o->potential_version;
  }
  int* err = tc_err_flag(h, (int*)ws_get(h, "df_err", sizeof(int)));
  if (!h->deferred) DFTFE_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), h->stream));
  df_init(h, X, ldx, Y, ldy, ncol, with_nl);
  for (int c = 0; c < h->ncolours; ++c) {
    const int64_t n = h->colour_off[c + 1] - h->colour_off[c];
    if (n == 0) continue;
    const int32_t* cells = h->d_colour_cells + h->colour_off[c];
    ProfScope ps(h, "cell_gemm_df");
    dim3 grid((unsigned)n, (unsigned)((ncol + 31) / 32));
    DFTFE_LAUNCH(k_cell_df_tiled<TM>, grid, 256, sh, h->stream, Hk, h->d_map, cells, nc, X, ldx, Y, ldy, ncol, err);
  }
  if (h->deferred) return true;
  int herr = 0;
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  if (herr) throw Error(DFTFE_ERR_TIMEOUT, "float-pair cell kernel: a bounded wait timed out");
  return true;
}

// Y = H~ X with the pair-of-floats cell products (nonlocal part FP64).
void apply_df(dftfe_ham h, const double* X, int64_t ldx, double* Y, int64_t ldy, int ncol, bool with_nl) {
  // tiled kernel for the degrees it is instantiated for (rows per thread TM = ceil(nc/32))
  if (apply_df_tiled<1>(h, X, ldx, Y, ldy, ncol, with_nl) || apply_df_tiled<2>(h, X, ldx, Y, ldy, ncol, with_nl) ||
      apply_df_tiled<4>(h, X, ldx, Y, ldy, ncol, with_nl) || apply_df_tiled<7>(h, X, ldx, Y, ldy, ncol, with_nl) ||
      apply_df_tiled<11>(h, X, ldx, Y, ldy, ncol, with_nl))
    return;
  auto* m = h->mesh;
  const int nc = m->nc;
  static bool attr = false;
  if (!attr) {
    DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_cell_df_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  const size_t n2 = (size_t)m->Nc * nc * nc;
  dftfe_ham o = loc(h);
  float2* Hdf = (float2*)ws_get(o, "cells_df", sizeof(float2) * n2);
  if (o->df_version != o->potential_version) {
    DFTFE_LAUNCH(k_split_df, nblk2((int64_t)n2), 256, 0, h->stream, o->d_Hc, Hdf, (int64_t)n2);
    o->df_version = o->potential_version;
  }
  // zero output and the FP64 nonlocal part, then the cell products colour by colour
  df_init(h, X, ldx, Y, ldy, ncol, with_nl);
  const size_t sh = (size_t)nc * 32 * sizeof(float2) + nc * sizeof(int32_t);
  for (int c = 0; c < h->ncolours; ++c) {
    const int64_t n = h->colour_off[c + 1] - h->colour_off[c];
    if (n == 0) continue;
    const int32_t* cells = h->d_colour_cells + h->colour_off[c];
    ProfScope ps(h, "cell_gemm_df");
    dim3 grid((unsigned)n, (unsigned)((ncol + 31) / 32));
    DFTFE_LAUNCH(k_cell_df_wide, grid, 256, sh, h->stream, Hdf, h->d_map, cells, nc, X, ldx, Y, ldy, ncol);
  }
}

}  // namespace dftfe
