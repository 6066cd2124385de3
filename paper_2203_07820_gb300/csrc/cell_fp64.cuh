// FP64 cell product body shared by the per-colour kernel (hx.cu) and the batched kernel
// (batch.cu), so both compute bit-identical results.
#pragma once

#include <cstdint>

namespace dftfe {

constexpr int CW_ROWS = 8;

// One cell's product Z[rows rbeg..rend-1 of the cell] += alpha H~^c X^c for the 32 columns of
// tile `ytile`, 256 threads: the cell's rows of X are gathered into shared memory (nc x 32
// doubles + nc node ids); each warp owns rows r0..r0+7 of H~^c in turn (lanes = columns) and
// reads them as warp-uniform loads.  Every output row is formed by one warp in the same order
// whatever the row range, so splitting a cell's rows over CTAs does not change the result.
__device__ __forceinline__ void cell_fp64_wide_body(const double* __restrict__ Hc, const int32_t* __restrict__ map,
                                                    int64_t cell, int nc, const double* __restrict__ X, int64_t ldx,
                                                    double* __restrict__ Z, int64_t ldz, int ncol, double alpha,
                                                    int ytile, int rbeg, int rend, double* smem) {
  double* xs = smem;                          // nc x 32
  int32_t* sm = (int32_t*)(smem + nc * 32);   // nc
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = ytile * 32 + lane;
  const bool colok = col < ncol;
  const int32_t* m = map + cell * nc;
  for (int k = threadIdx.x; k < nc; k += 256) sm[k] = m[k];
  __syncthreads();
  for (int k = warp; k < nc; k += 8) xs[k * 32 + lane] = colok ? X[(int64_t)sm[k] * ldx + col] : 0.0;
  __syncthreads();
  const double* H = Hc + cell * (int64_t)nc * nc;
  for (int r0 = rbeg + warp * CW_ROWS; r0 < rend; r0 += 8 * CW_ROWS) {
    const int nr = min(CW_ROWS, rend - r0);
    double acc[CW_ROWS];
#pragma unroll
    for (int i = 0; i < CW_ROWS; ++i) acc[i] = 0.0;
    const double* Hr = H + (int64_t)r0 * nc;
    if (nr == CW_ROWS) {
      for (int k = 0; k < nc; ++k) {
        const double x = xs[k * 32 + lane];
#pragma unroll
        for (int i = 0; i < CW_ROWS; ++i) acc[i] = fma(__ldg(Hr + (int64_t)i * nc + k), x, acc[i]);
      }
    } else {
      for (int k = 0; k < nc; ++k) {
        const double x = xs[k * 32 + lane];
#pragma unroll
        for (int i = 0; i < CW_ROWS; ++i)
          if (i < nr) acc[i] = fma(__ldg(Hr + (int64_t)i * nc + k), x, acc[i]);
      }
    }
    if (colok) {
#pragma unroll
      for (int i = 0; i < CW_ROWS; ++i)
        if (i < nr) {
          double* z = Z + (int64_t)sm[r0 + i] * ldz + col;
          *z += alpha * acc[i];
        }
    }
  }
}


}  // namespace dftfe
