// FP64-accurate H~X on the tensor cores from exact digit products (the W = H~X of the
// Rayleigh-Ritz step, Sec. 3.2, which must keep FP64 accuracy when the filter runs in FP32).
//
// Each FP64 operand is written as a 41-bit fixed-point integer relative to a power of two:
// a cell-matrix entry relative to the largest entry of its row (2^eA), an entry of X relative
// to the largest entry of its column (2^eX).  The integer is cut into six balanced base-128
// digits (|digit| <= 64), each held exactly by a bf16.  A cell product is then
//     sum_k a_rk x_kc ~ 2^(eA + eX - 47) sum_{d=0..5} acc_d 2^(7 (5 - d)),
//     acc_d = sum_{s + t = d} sum_k A_s[r][k] X_t[k][c],
// the 21 digit products of order <= 5.  Every product is an integer of at most 13 bits and
// each accumulator sums at most 6 x 343 of them (p = 6), below 2^24 in magnitude, so the
// FP32 tensor-core accumulation in tensor memory is exact; the dropped products of order
// >= 6 and the rounding of the fixed-point integers leave about 2^-39 of |a|max |x|max per
// term.  The epilogue turns the six exact accumulators into one 64-bit integer (Horner in
// base 128), converts it to FP64 once and adds it into Y.
//
// Kernel k_cell_slices: one persistent CTA per SM over the (cell, 64-column) items of one
// colour (no two cells of a colour share a node, so the FP64 read-modify-write of Y needs no
// atomics and the sum order is fixed).  D[128 cell rows][64 columns] per digit order: six
// accumulators (384 tensor-memory columns); the cell-matrix digits are the A operand, read
// from tensor memory (two slots of one 16-deep K-step: 6 digits x 8 columns each); the X
// digits are the B operand in shared memory, gathered row by row from digit planes
// (node-major, so the tiles are MN-major: each 128-byte row is one node's 64 columns).
// Warp roles (448 threads):
//   warp 0        bulk copies of the A digit rows of each (M-tile, K-step) into a 3-slot ring
//   warp 1        tensor-memory owner and MMA issuer (one elected lane)
//   warps 2-5     B producers: cp.async gather of 32 nodes x 64 columns x 6 digits per stage
//   warps 6-9     epilogue: exact accumulators -> FP64 (staged in shared memory), then a
//                 row-coalesced FP64 add into Y
//   warps 10-13   A converters: digit rows of the landing slot -> tensor memory
// Every wait is bounded; on a time-out the kernel records DFTFE_ERR_TIMEOUT, drains its own
// copies and MMAs (bounded), frees its tensor memory and returns.
#include "internal.h"
#include "tcgen05.h"

#include <algorithm>

namespace dftfe {

namespace oz {

constexpr int kDig = 6;                   // digits per operand
constexpr int kFix = 41;                  // fixed-point bits: |F| <= 2^41
constexpr int kThreads = 448;
constexpr int kN = 64;                    // columns of one work item (MMA N)
constexpr int kBlk = 128;                 // columns of one digit-plane block
constexpr int kKc = 32;                   // nodes per B stage (two 16-deep K-steps)
constexpr int kRowBytes = kDig * 32;      // one row of one K-step of A: 6 digits x 16 bf16
constexpr int kASlot = 128 * kRowBytes;   // 24 KB
constexpr int kBTile = kKc * 128;         // one digit of one stage: 32 nodes x 64 bf16
constexpr int kBStage = kDig * kBTile;    // 24 KB
constexpr int kLand = 3, kStagesB = 3, kConv = 2;
constexpr uint32_t kAccCols = kDig * kN;  // 384 accumulator columns
constexpr uint32_t kASlotCols = kDig * 8; // 48 columns per A slot
constexpr int kStagePitch = kN * 8 + 16;  // bytes per staged output row (bank offset 4 words)

struct Shared {
  uint64_t land_full[kLand], land_empty[kLand];
  uint64_t conv_full[kConv], conv_empty[kConv];
  uint64_t b_full[kStagesB], b_empty[kStagesB];
  uint64_t acc_full, acc_empty, drain;
  uint32_t tmem;
  int abort;
};

constexpr size_t smem_bytes() {
  return 1024 + (size_t)kLand * kASlot + (size_t)kStagesB * kBStage + (size_t)128 * kStagePitch + sizeof(Shared);
}

struct Args {
  const uint8_t* A;       // digit rows of the cell matrices (layout: see k_cell_digits)
  const int32_t* eA;      // row exponents, Nc x (nmt 128)
  const int32_t* map;     // Nc x nc
  const int32_t* cells;   // the launch's cells (one colour)
  int ncells, nhalf;      // cells; 64-column items per cell (1 or 2)
  const uint16_t* Xd;     // kDig digit planes, each M x 128 bf16
  int64_t plane;          // elements per plane
  const int32_t* ebx;     // biased exponent of the largest |x| of each block column
  double* Z;              // output block (its column 0 is the block's)
  int64_t ldz;
  int ncol;               // valid columns of the block
  int nc, nmt, rows8, nks;
  int* err;
};

__device__ __forceinline__ int biased_exp(double v) {
  return (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7FFull);
}

// F = round(v 2^(kFix - E)) for |v| < 2^E (ties away from zero; subnormals as zero), as
// kDig balanced base-128 digits, most significant first: F = sum_s dg[s] 128^(kDig-1-s),
// |dg[s]| <= 64.  Integer operations only.
__device__ __forceinline__ void fixed_digits(double v, int E, int* dg) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const int eb = (int)((u >> 52) & 0x7FFull);
  long long F = 0;
  const int sh = 1075 - kFix + E - eb;      // v = mant 2^(eb - 1075); >= 12 when |v| < 2^E
  if (eb != 0 && sh >= 1 && sh <= 53) {
    const unsigned long long mant = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    F = (long long)((mant + (1ull << (sh - 1))) >> sh);
    if (u >> 63) F = -F;
  }
#pragma unroll
  for (int s = kDig - 1; s > 0; --s) {
    int r = (int)(F & 127);
    if (r > 63) r -= 128;
    dg[s] = r;
    F = (F - r) >> 7;
  }
  dg[0] = (int)F;
}

__device__ __forceinline__ uint32_t bf16_bits(int d) { return __float_as_uint((float)d) >> 16; }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(bytes) : "memory");
}

// BF16 MMA, A from tensor memory (K-major, two bf16 per column), B an MN-major
// 128-byte-swizzled shared-memory tile, D F32 in tensor memory: M = 128, N = 64
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t acc) {
  constexpr uint32_t id = tc::idesc(1u, 128, kN) | (1u << 16);
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}"
               :: "r"(d), "r"(a_tmem), "l"(b), "r"(id), "r"(acc));
}

// descriptor of an MN-major SW128 tile holding one 64-element atom column along N: 8-row
// groups along K are 1024 bytes apart (given as both offsets)
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(1024 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
               :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
}

// S 2^e in FP64 (S exact below 2^59; one rounding to 53 bits), the exponent added to the
// bits while the result stays normal
__device__ __forceinline__ double scaled(long long S, int e) {
  if (S == 0) return 0.0;
  const double v = (double)S;
  const long long b = __double_as_longlong(v);
  const int ne = (int)((b >> 52) & 0x7FF) + e;
  if (ne > 0 && ne < 2047) return __longlong_as_double(b + ((long long)e << 52));
  return ldexp(v, e);
}

}  // namespace oz

// Set-up: digit rows of every cell matrix.  Per cell, M-tile mt (rows 128 mt ..; the last
// M-tile holds rows8 rows) and K-step ks (columns 16 ks .. 16 ks + 15), the tile's rows in
// order, each 192 bytes: digit s (most significant first) as 16 bf16 in column order.  Rows
// and columns beyond nc hold zero digits; eA[cell][r] = exponent E of the row (|h| < 2^E).
__global__ void k_cell_digits(const double* __restrict__ Hc, int64_t Nc, int nc, int nmt, int rows8, int nks,
                              uint8_t* __restrict__ A, int32_t* __restrict__ eA) {
  using namespace oz;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Nc * nmt * 128) return;
  const int64_t cell = t / (nmt * 128);
  const int r = (int)(t - cell * nmt * 128);
  const int mt = r >> 7, rt = r & 127;
  const int rows = mt == nmt - 1 ? rows8 : 128;
  const bool real_row = r < nc;
  const double* hr = Hc + (cell * nc + (real_row ? r : 0)) * (int64_t)nc;
  int emax = 0;
  if (real_row)
    for (int k = 0; k < nc; ++k) emax = max(emax, biased_exp(hr[k]));
  const int E = emax - 1022;
  eA[t] = real_row ? E : 0;
  if (rt >= rows) return;                          // row not stored (last M-tile)
  const int64_t cell_bytes = (int64_t)nks * ((nmt - 1) * 128 + rows8) * kRowBytes;
  uint8_t* dst0 = A + cell * cell_bytes + (int64_t)mt * nks * 128 * kRowBytes + (int64_t)rt * kRowBytes;
  for (int ks = 0; ks < nks; ++ks) {
    uint32_t w[kDig][8];
#pragma unroll
    for (int s = 0; s < kDig; ++s)
#pragma unroll
      for (int j = 0; j < 8; ++j) w[s][j] = 0u;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int k = 16 * ks + j;
      const double v = (real_row && k < nc) ? hr[k] : 0.0;
      int dg[kDig];
      fixed_digits(v, E, dg);
#pragma unroll
      for (int s = 0; s < kDig; ++s) w[s][j >> 1] |= bf16_bits(dg[s]) << (16 * (j & 1));
    }
    uint4* dst = reinterpret_cast<uint4*>(dst0 + (int64_t)ks * rows * kRowBytes);
#pragma unroll
    for (int s = 0; s < kDig; ++s) {
      dst[2 * s] = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
      dst[2 * s + 1] = make_uint4(w[s][4], w[s][5], w[s][6], w[s][7]);
    }
  }
}

// ebx[c] = largest biased exponent of |X[:, c]| over the M rows (c < ncol; ebx zeroed first)
__global__ void k_col_exponent(const double* __restrict__ X, int64_t ldx, int64_t M, int ncol, int* ebx) {
  __shared__ int mx[2][128];
  const int c = threadIdx.x & 127, half = threadIdx.x >> 7;
  int m = 0;
  if (c < ncol)
    for (int64_t r = 2 * (int64_t)blockIdx.x + half; r < M; r += 2 * (int64_t)gridDim.x)
      m = max(m, oz::biased_exp(X[r * ldx + c]));
  mx[half][c] = m;
  __syncthreads();
  if (half == 0 && c < ncol) {
    m = max(m, mx[1][c]);
    if (m > 0) atomicMax(ebx + c, m);
  }
}

// digit planes of a block of (up to) 128 columns: Xd[s][node][c], zero beyond ncol; two
// columns per thread
__global__ void k_x_digits(const double* __restrict__ X, int64_t ldx, int64_t M, int ncol, const int* __restrict__ ebx,
                           uint32_t* __restrict__ Xd) {
  using namespace oz;
  const int64_t total = M * (kBlk / 2);
  const int64_t plane2 = M * (kBlk / 2);           // 32-bit words per plane
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / (kBlk / 2);
    const int c = 2 * (int)(t - r * (kBlk / 2));
    int d0[kDig], d1[kDig];
#pragma unroll
    for (int s = 0; s < kDig; ++s) d0[s] = d1[s] = 0;
    if (c < ncol) fixed_digits(X[r * ldx + c], ebx[c] - 1022, d0);
    if (c + 1 < ncol) fixed_digits(X[r * ldx + c + 1], ebx[c + 1] - 1022, d1);
#pragma unroll
    for (int s = 0; s < kDig; ++s) Xd[s * plane2 + t] = bf16_bits(d0[s]) | (bf16_bits(d1[s]) << 16);
  }
}

__global__ void __launch_bounds__(oz::kThreads, 1) k_cell_slices(oz::Args g) {
  using namespace oz;
  using tc::mbar_arrive;
  using tc::mbar_init;
  using tc::mbar_wait;
  using tc::smem_u32;
  using tc::sw128;
  using tc::tc_commit;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;                                   // A landing ring
  uint8_t* sB = sA + kLand * kASlot;                    // B stages (1024-aligned)
  uint8_t* sO = sB + kStagesB * kBStage;                // staged FP64 outputs
  Shared* sh = (Shared*)(sO + 128 * kStagePitch);
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
    for (int s = 0; s < kStagesB; ++s) {
      mbar_init(&sh->b_full[s], 128);
      mbar_init(&sh->b_empty[s], 1);
    }
    mbar_init(&sh->acc_full, 1);
    mbar_init(&sh->acc_empty, 128);
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

  const int nitems = g.ncells * g.nhalf;
  const int my = nitems > (int)blockIdx.x ? (nitems - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  // the CTA's i-th item: its cell and first column within the block; the two 64-column
  // halves of a cell go to adjacent CTAs, which read its digit rows at about the same time
  auto item = [&](int i, int& cell, int& c0) {
    const int w = (int)blockIdx.x + i * (int)gridDim.x;
    cell = g.cells[w / g.nhalf];
    c0 = (w % g.nhalf) * kN;
  };
  const int nkc = (g.nks + 1) / 2;
  const int64_t cell_bytes = (int64_t)g.nks * ((g.nmt - 1) * 128 + g.rows8) * kRowBytes;

  if (warp == 0) {
    // ------------------------------------------------------------ A producer
    if (lane == 0) {
      uint32_t ta = 0;
      bool go = true;
      for (int i = 0; i < my && go; ++i) {
        int cell, c0;
        item(i, cell, c0);
        const uint8_t* Ac = g.A + (int64_t)cell * cell_bytes;
        for (int mt = 0; mt < g.nmt && go; ++mt) {
          const int rows = mt == g.nmt - 1 ? g.rows8 : 128;
          const uint8_t* At = Ac + (int64_t)mt * g.nks * 128 * kRowBytes;
          for (int ks = 0; ks < g.nks; ++ks, ++ta) {
            const int s = ta % kLand;
            if (!mbar_wait(&sh->land_empty[s], ((ta / kLand) & 1) ^ 1, abort, g.err)) { go = false; break; }
            const uint32_t full = smem_u32(&sh->land_full[s]);
            const uint32_t bytes = (uint32_t)rows * kRowBytes;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(full), "r"(bytes) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(smem_u32(sA + s * kASlot)), "l"(At + (int64_t)ks * rows * kRowBytes), "r"(bytes),
                            "r"(full)
                         : "memory");
          }
        }
      }
      // drain: every issued copy has landed before the CTA may exit
      for (uint32_t t = (ta > (uint32_t)kLand ? ta - kLand : 0); t < ta; ++t) {
        volatile int no_abort = 0;
        mbar_wait(&sh->land_full[t % kLand], (t / kLand) & 1, &no_abort, g.err);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t ta = 0, tb = 0, tm = 0;
      bool go = true;
      for (int i = 0; i < my && go; ++i) {
        for (int mt = 0; mt < g.nmt && go; ++mt, ++tm) {
          if (!mbar_wait(&sh->acc_empty, (tm & 1) ^ 1, abort, g.err)) { go = false; break; }
          for (int kc = 0; kc < nkc && go; ++kc, ++tb) {
            const int sb = tb % kStagesB;
            if (!mbar_wait(&sh->b_full[sb], (tb / kStagesB) & 1, abort, g.err)) { go = false; break; }
            const uint32_t bst = smem_u32(sB + sb * kBStage);
            for (int kk = 0; kk < 2 && go; ++kk) {
              const int ks = 2 * kc + kk;
              if (ks >= g.nks) break;
              const int sa = ta % kConv;
              if (!mbar_wait(&sh->conv_full[sa], (ta / kConv) & 1, abort, g.err)) { go = false; break; }
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              const uint32_t aslot = tmem + kAccCols + (uint32_t)sa * kASlotCols;
#pragma unroll
              for (int d = 0; d < kDig; ++d)
#pragma unroll
                for (int s = 0; s <= d; ++s)
                  mma_ts(tmem + (uint32_t)(d * kN), aslot + (uint32_t)(8 * s),
                         sdesc_mn(bst + (uint32_t)((d - s) * kBTile + kk * 2048)), (ks > 0 || s > 0) ? 1u : 0u);
              tc_commit(&sh->conv_empty[sa]);
              ++ta;
            }
            if (go) tc_commit(&sh->b_empty[sb]);
          }
          if (go) tc_commit(&sh->acc_full);
        }
      }
      // drain: all issued MMAs complete before tensor memory is released
      tc_commit(&sh->drain);
      volatile int no_abort = 0;
      mbar_wait(&sh->drain, 0, &no_abort, g.err);
    }
  } else if (warp < 6) {
    // ------------------------------------------------------------ B producers
    // stage = nodes 32 kc .. 32 kc + 31 of the item's cell, its 64 columns, all digits: thread
    // pt copies (node row pt / 8, 16-byte column chunk pt % 8) and the same for pt + 128, for
    // each digit; rows beyond nc are zero-filled
    const int pt = threadIdx.x - 64;
    constexpr int kAhead = kStagesB - 1;
    const uint32_t per_item = (uint32_t)(g.nmt * nkc);
    const uint32_t nchunks = (uint32_t)my * per_item;
    auto issue = [&](uint32_t t) -> bool {
      const int sb = t % kStagesB;
      if (!mbar_wait(&sh->b_empty[sb], ((t / kStagesB) & 1) ^ 1, abort, g.err)) return false;
      int cell, c0;
      item((int)(t / per_item), cell, c0);
      const int kc = (int)(t % (uint32_t)nkc);
      const uint32_t st = smem_u32(sB + sb * kBStage);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int pr = pt + 128 * j;
        const int k = pr >> 3, c = pr & 7;
        const int kg = kc * kKc + k;
        const bool ok = kg < g.nc;
        const int node = ok ? __ldg(g.map + (int64_t)cell * g.nc + kg) : 0;
        const uint16_t* src = g.Xd + (int64_t)node * kBlk + c0 + 8 * c;
        const uint32_t dst = st + sw128((uint32_t)k, (uint32_t)(16 * c));
#pragma unroll
        for (int s = 0; s < kDig; ++s) cp_async16(dst + s * kBTile, src + s * g.plane, ok ? 16u : 0u);
      }
      return true;
    };
    bool go = true;
    for (uint32_t t = 0; t < (uint32_t)kAhead; ++t) {
      if (go && t < nchunks) go = issue(t);
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (uint32_t tb = 0; tb < nchunks && go; ++tb) {
      // every group but the newest kAhead - 1 complete: stage tb has landed
      asm volatile("cp.async.wait_group %0;" :: "n"(kAhead - 1) : "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&sh->b_full[tb % kStagesB]);
      if (tb + kAhead < nchunks) go = issue(tb + kAhead);
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp < 10) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;                       // TMEM lane quadrant
    const int rt = 32 * q + lane;                 // accumulator row = tile row
    uint32_t tm = 0;
    bool go = true;
    for (int i = 0; i < my && go; ++i) {
      int cell, c0;
      item(i, cell, c0);
      for (int mt = 0; mt < g.nmt; ++mt, ++tm) {
        if (!mbar_wait(&sh->acc_full, tm & 1, abort, g.err)) { go = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int r = mt * 128 + rt;
        const int ea = __ldg(g.eA + (int64_t)cell * g.nmt * 128 + r) - 47;
        double* orow = reinterpret_cast<double*>(sO + rt * kStagePitch);
        for (int cg = 0; cg < kN / 16; ++cg) {
          uint32_t a[kDig][16];
#pragma unroll
          for (int d = 0; d < kDig; ++d)
            oz::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(d * kN + 16 * cg), a[d]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            long long S = 0;
#pragma unroll
            for (int d = 0; d < kDig; ++d) S = S * 128 + (long long)__float2int_rn(__uint_as_float(a[d][j]));
            const int col = c0 + 16 * cg + j;
            orow[16 * cg + j] = scaled(S, ea + __ldg(g.ebx + col) - 1022);
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&sh->acc_empty);
        __syncwarp();
        // Y[node(row)][c0 + c] += staged, one row of 64 doubles per warp step, the loads of
        // eight rows ahead of their stores
        const int node_l = r < g.nc ? __ldg(g.map + (int64_t)cell * g.nc + r) : -1;
        const int c = lane, colA = c0 + c, colB = c0 + c + 32;
        for (int r0 = 0; r0 < 32; r0 += 8) {
          double va[8], vb[8];
          int nd[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            nd[u] = __shfl_sync(0xffffffffu, node_l, r0 + u);
            double* zr = g.Z + (int64_t)max(nd[u], 0) * g.ldz;
            va[u] = (nd[u] >= 0 && colA < g.ncol) ? zr[colA] : 0.0;
            vb[u] = (nd[u] >= 0 && colB < g.ncol) ? zr[colB] : 0.0;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            if (nd[u] < 0) continue;
            const double* srow = reinterpret_cast<const double*>(sO + (32 * q + r0 + u) * kStagePitch);
            double* zr = g.Z + (int64_t)nd[u] * g.ldz;
            if (colA < g.ncol) zr[colA] = va[u] + srow[c];
            if (colB < g.ncol) zr[colB] = vb[u] + srow[c + 32];
          }
        }
        __syncwarp();
      }
    }
  } else {
    // ------------------------------------------------------------ A converters
    const int q = warp & 3;
    const int rt = 32 * q + lane;
    uint32_t ta = 0;
    bool go = true;
    for (int i = 0; i < my && go; ++i)
      for (int mt = 0; mt < g.nmt && go; ++mt) {
        const int rows = mt == g.nmt - 1 ? g.rows8 : 128;
        // rows of the last M-tile beyond the landed ones hold stale bytes: zeros instead
        const bool landed = rt < rows;
        for (int ks = 0; ks < g.nks; ++ks, ++ta) {
          const int s = ta % kLand, sc = ta % kConv;
          if (!mbar_wait(&sh->land_full[s], (ta / kLand) & 1, abort, g.err)) { go = false; break; }
          if (!mbar_wait(&sh->conv_empty[sc], ((ta / kConv) & 1) ^ 1, abort, g.err)) { go = false; break; }
          uint32_t w[kDig * 8];
          const uint4* src = reinterpret_cast<const uint4*>(sA + s * kASlot + rt * kRowBytes);
#pragma unroll
          for (int c = 0; c < 2 * kDig; ++c) {
            const uint4 u = landed ? src[c] : make_uint4(0u, 0u, 0u, 0u);
            w[4 * c] = u.x;
            w[4 * c + 1] = u.y;
            w[4 * c + 2] = u.z;
            w[4 * c + 3] = u.w;
          }
          // the landing slot may take the next bulk copy once these reads are ordered before it
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_arrive(&sh->land_empty[s]);
          // the MMAs that read this A slot have completed (conv_empty)
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t slot = tmem + ((uint32_t)(32 * q) << 16) + kAccCols + (uint32_t)sc * kASlotCols;
#pragma unroll
          for (int d = 0; d < kDig; ++d) oz::tmem_st8(slot + 8 * d, w + 8 * d);
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          mbar_arrive(&sh->conv_full[sc]);
        }
      }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512));
}

static unsigned nblk_oz(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// the exact-slice products apply when each accumulator stays below 2^24 (nc <= 682, p <= 7)
bool slices_applicable(dftfe_ham h) { return (int64_t)6 * 4096 * h->mesh->nc < (1 << 24); }

// Y = H~ X (H~_nl in FP64 when with_nl, else the local part only) with the cell products
// from exact digit products on the tensor cores.  False when not applicable.
bool apply_slices(dftfe_ham h, const double* X, int64_t ldx, double* Y, int64_t ldy, int ncol, bool with_nl) {
  using namespace oz;
  if (!slices_applicable(h)) return false;
  auto* m = h->mesh;
  const int nc = m->nc;
  const int nmt = (nc + 127) / 128;
  const int rows8 = ((nc - 128 * (nmt - 1)) + 7) / 8 * 8;
  const int nks = (nc + 15) / 16;
  static bool attr = false;
  if (!attr) {
    DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_cell_slices, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem_bytes()));
    attr = true;
  }
  const int64_t cell_bytes = (int64_t)nks * ((nmt - 1) * 128 + rows8) * kRowBytes;
  dftfe_ham o = loc(h);                 // the owner of the cell matrices and their digit rows
  uint8_t* A = (uint8_t*)ws_get(o, "cells_slices", (size_t)(m->Nc * cell_bytes));
  int32_t* eA = (int32_t*)ws_get(o, "cells_slices_e", sizeof(int32_t) * (size_t)m->Nc * nmt * 128);
  if (o->slices_version != o->potential_version) {
    DFTFE_LAUNCH(k_cell_digits, nblk_oz(m->Nc * nmt * 128, 128), 128, 0, h->stream, o->d_Hc, m->Nc, nc, nmt, rows8,
                 nks, A, eA);
    o->slices_version = o->potential_version;
  }
  int* err = tc_err_flag(h, (int*)ws_get(h, "slices_err", sizeof(int)));
  if (!h->deferred) DFTFE_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), h->stream));
  if (with_nl) apply_nonlocal_fp64(h, X, ldx, Y, ldy, ncol);
  else zero_block(h->stream, Y, ldy, m->M, ncol);
  uint16_t* Xd = (uint16_t*)ws_get(h, "slices_x", sizeof(uint16_t) * (size_t)kDig * m->M * kBlk);
  int* ebx = (int*)ws_get(h, "slices_xe", sizeof(int) * kBlk);
  const unsigned gx = (unsigned)std::max(1, h->sm_count) * 4;
  for (int b0 = 0; b0 < ncol; b0 += kBlk) {
    const int nb = std::min(kBlk, ncol - b0);
    DFTFE_CHECK_CUDA(cudaMemsetAsync(ebx, 0, sizeof(int) * kBlk, h->stream));
    {
      ProfScope ps(h, "slices_digits");
      DFTFE_LAUNCH(k_col_exponent, gx, 256, 0, h->stream, X + b0, ldx, m->M, nb, ebx);
      DFTFE_LAUNCH(k_x_digits, gx * 2, 256, 0, h->stream, X + b0, ldx, m->M, nb, ebx, (uint32_t*)Xd);
    }
    const int nhalf = (nb + kN - 1) / kN;
    for (int c = 0; c < h->ncolours; ++c) {
      const int64_t n = h->colour_off[c + 1] - h->colour_off[c];
      if (n == 0) continue;
      Args a{A, eA, h->d_map, h->d_colour_cells + h->colour_off[c], (int)n, nhalf, Xd, m->M * (int64_t)kBlk, ebx,
             Y + b0, ldy, nb, nc, nmt, rows8, nks, err};
      const unsigned grid = (unsigned)std::min<int64_t>(n * nhalf, std::max(1, h->sm_count));
      ProfScope ps(h, "cell_gemm_slices");
      DFTFE_LAUNCH(k_cell_slices, grid, kThreads, smem_bytes(), h->stream, a);
    }
  }
  if (h->deferred) return true;
  int herr = 0;
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  if (herr) throw Error(DFTFE_ERR_TIMEOUT, "exact-slice cell kernel: a bounded wait timed out");
  return true;
}

// W = H~X for the mixed Rayleigh-Ritz step: exact digit products where they apply, else the
// float-pair products
void apply_w(dftfe_ham h, const double* X, int64_t ldx, double* Y, int64_t ldy, int ncol, bool with_nl) {
  if (!apply_slices(h, X, ldx, Y, ldy, ncol, with_nl)) apply_df(h, X, ldx, Y, ldy, ncol, with_nl);
}

}  // namespace dftfe
