// Bloch k-points (Sec. 2.1: psi = e^{ik.x} u, Eq. bloch, and the reduced Kohn-Sham equation
// after it): H~^k on complex blocks and the complex ChFSI steps, FP64 (complex128).
//
//   H~^k = H~_loc + 1/2 |k|^2 - i sum_d k_d G~_d + C~^k diag(h) C~^k^H,
//   G_d,jl = int N_j dN_l/dx_d (GLL quadrature on the nodes), G~_d = M^-1/2 G_d M^-1/2,
//   C~^k_ja = M_jj^1/2 chi_a(x_j) e^{-ik.d_ja}, d_ja the minimum-image displacement x_j - R_a.
//
// Layout: a complex block is complex128 DoF-major (real and imaginary parts interleaved), so
// its real view is an M x 2 ncol FP64 block.  H~_loc is real: it acts on that real view as on
// 2 ncol real columns, through the same FP64 cell products as at the Gamma point.
//
// The k.grad term is separable on the structured periodic mesh: with GLL quadrature on the
// nodes, G_d is the 1D periodic derivative matrix G1_d (entries int l_a l_b' = w_a l_b'(x_a),
// exact under GLL) along axis d times the 1D lumped masses of the two other axes, and the
// Loewdin scaling cancels those, so G~_d = G~1_d along axis d with G~1_d = m_d^-1/2 G1_d
// m_d^-1/2.  A stencil kernel applies it (p+1 neighbours per axis inside an element, 2p+1
// on element faces), fused with the recurrence terms.  Dense complex cell matrices (the
// paper's form) would make every cell product four real FP64 products; here the cell
// products stay real and the k-dependent part costs 3 (p+2) complex-by-real multiply-adds
// per entry on average (the kernel is bound by GB300's FP64 pipe, not by HBM).
//
// CholGS and Rayleigh-Ritz work on the real view.  With Xr the real view of X (M x 2N), the
// real Gram G = Xr^T Xr holds every real inner product, and the complex S = X^H X is
//   S_ab = (G[2a,2b] + G[2a+1,2b+1]) + i (G[2a,2b+1] - G[2a+1,2b]).
// Right multiplication by a complex matrix A acts on the real view as the real 2N x 2N
// matrix rho(A): rho(A)[2a,2b] = rho(A)[2a+1,2b+1] = Re A_ab, rho(A)[2a,2b+1] = Im A_ab,
// rho(A)[2a+1,2b] = -Im A_ab, with rho(AB) = rho(A) rho(B) and rho(A^H) = rho(A)^T.  So
// rho(S) = rho(L) rho(L)^T for S = L L^H, and rho(L) is lower triangular with a positive
// diagonal: the real Cholesky factor of rho(S) IS rho(L) (uniqueness), and the real CholGS
// steps on (rho(S), Xr) give X L^-H exactly.  The Rayleigh-Ritz eigensolve is Hermitian
// (syevd_z); its eigenvectors rotate the real views through rho(Q).
#include "internal.h"

#include <cmath>
#include <string>
#include <vector>

namespace dftfe {

static unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

static int read_status_z(dftfe_ham h, int* d_status) {
  int st = 0;
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  return st;
}

// ------------------------------------------------------------------ kernels
// Z = s1 X + s2 Xp - i alpha sum_d (G~1_d along axis d) X; tab = 3 x p x (2p+1), entry
// (d, a, o + p) = k_d G~1_d(i, i + o) for a node i with i mod p = a (uniform mesh).
// Z and Xp may be the same array (each thread reads Xp before it writes Z at one entry)
__global__ void __launch_bounds__(256) k_kin_init(double2* Z, int64_t ldz,
                                                  const double2* __restrict__ X, int64_t ldx,
                                                  const double2* Xp, int64_t ldp, int64_t M,
                                                  int ncol, double s1, double s2, double alpha,
                                                  const double* __restrict__ tab, int p, int64_t g0,
                                                  int64_t g1, int kbits) {
  extern __shared__ double ts[];
  const int W = 2 * p + 1;
  for (int t = threadIdx.x; t < 3 * p * W; t += blockDim.x) ts[t] = tab[t];
  __syncthreads();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= M * ncol) return;
  const int64_t i = t / ncol;
  const int c = (int)(t - i * ncol);
  const int64_t ix = i % g0, iy = (i / g0) % g1, iz = i / (g0 * g1);
  const int64_t g2 = M / (g0 * g1);
  const int64_t pos[3] = {ix, iy, iz};
  const int64_t ext[3] = {g0, g1, g2};
  const int64_t stride[3] = {1, g0, g0 * g1};
  const bool kmask[3] = {(kbits & 1) != 0, (kbits & 2) != 0, (kbits & 4) != 0};   // k_d != 0
  double sr = 0.0, si = 0.0;
  // the structural non-zeros of row a: offsets -a..p-a within the node's cell, and for a = 0
  // also -p..-1 in the previous cell (integer bounds: the FP64 pipe only does the products)
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (!kmask[d]) continue;
    const int a = (int)(pos[d] % p);
    const double* T = ts + ((size_t)d * p + a) * W + p;
    const int olo = a == 0 ? -p : -a;
    for (int o = olo; o <= p - a; ++o) {
      int64_t j = pos[d] + o;
      j += j < 0 ? ext[d] : (j >= ext[d] ? -ext[d] : 0);
      const double2 v = X[(i + (j - pos[d]) * stride[d]) * ldx + c];
      sr = fma(T[o], v.x, sr);
      si = fma(T[o], v.y, si);
    }
  }
  const double2 xv = X[i * ldx + c];
  double2 z = make_double2(fma(s1, xv.x, alpha * si), fma(s1, xv.y, -alpha * sr));
  if (Xp) {
    const double2 pv = Xp[i * ldp + c];
    z.x = fma(s2, pv.x, z.x);
    z.y = fma(s2, pv.y, z.y);
  }
  Z[i * ldz + c] = z;
}

// The same coefficients split over each projector's support, so that a long support does not
// run as one latency-bound chain of dependent loads per warp: CTA (a, s) sums split s of
// projector a's entries (warp w every 8th entry of the split, lane l complex column
// 32 blockIdx.y + l) into part[a S + s][col]; k_nl_coefz_reduce adds the S splits in order and
// scales by h_a.  C is float2 (the complex64 filter) or double2.
constexpr int kNlzSplits = 8;
template <typename C>
__global__ void __launch_bounds__(256) k_nl_coefz_part(const C* __restrict__ X, int64_t ldx, int ncol,
                                                       const int64_t* __restrict__ prow,
                                                       const int32_t* __restrict__ pnode, const C* __restrict__ pval,
                                                       C* __restrict__ part) {
  using R = decltype(C::x);
  __shared__ C red[8][32];
  const int a = blockIdx.x / kNlzSplits, sidx = blockIdx.x % kNlzSplits;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.y * 32 + lane;
  const int64_t e0 = prow[a], e1 = prow[a + 1];
  const int64_t len = (e1 - e0 + kNlzSplits - 1) / kNlzSplits;
  const int64_t s0 = e0 + sidx * len, s1 = min(e1, s0 + len);
  R sr = 0, si = 0;
  if (col < ncol) {
#pragma unroll 4
    for (int64_t e = s0 + warp; e < s1; e += 8) {
      const C cv = pval[e];
      const C xv = X[(int64_t)pnode[e] * ldx + col];
      sr = fma(cv.x, xv.x, fma(cv.y, xv.y, sr));
      si = fma(cv.x, xv.y, fma(-cv.y, xv.x, si));
    }
  }
  C v;
  v.x = sr;
  v.y = si;
  red[warp][lane] = v;
  __syncthreads();
  if (warp == 0 && col < ncol) {
    R tr = 0, ti = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      tr += red[w][lane].x;
      ti += red[w][lane].y;
    }
    C o;
    o.x = tr;
    o.y = ti;
    part[(int64_t)blockIdx.x * ncol + col] = o;
  }
}

template <typename C>
__global__ void k_nl_coefz_reduce(const C* __restrict__ part, const double* __restrict__ hcoup, int nproj, int ncol,
                                  C* __restrict__ P) {
  using R = decltype(C::x);
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nproj * ncol) return;
  const int a = (int)(t / ncol), col = (int)(t % ncol);
  R sr = 0, si = 0;
  for (int k = 0; k < kNlzSplits; ++k) {
    const C v = part[((int64_t)a * kNlzSplits + k) * ncol + col];
    sr += v.x;
    si += v.y;
  }
  const R hv = (R)hcoup[a];
  C o;
  o.x = hv * sr;
  o.y = hv * si;
  P[t] = o;
}

// P = h (C~^kH X) for ncol complex columns through the split kernels above
template <typename C>
static void nl_coef_z_split(dftfe_ham h, const C* X, int64_t ldx, int ncol, const C* pval, C* P) {
  C* part = (C*)ws_get(h, sizeof(C) == 8 ? "nl_coefz32_part" : "nl_coefz_part",
                       sizeof(C) * (size_t)h->nproj * kNlzSplits * ncol);
  dim3 g1((unsigned)(h->nproj * kNlzSplits), (unsigned)((ncol + 31) / 32));
  DFTFE_LAUNCH(k_nl_coefz_part<C>, g1, 256, 0, h->stream, X, ldx, ncol, h->d_prow, h->d_pnode, pval, part);
  DFTFE_LAUNCH(k_nl_coefz_reduce<C>, nblk((int64_t)h->nproj * ncol), 256, 0, h->stream, part, h->d_h, h->nproj,
               ncol, P);
}

// Z[node][col] += alpha sum_{t in node's projectors} C~^k_t P[proj_t][col]; one warp per node
__global__ void __launch_bounds__(256) k_nl_add_z(double2* __restrict__ Z, int64_t ldz, int ncol,
                                                  const int32_t* __restrict__ snode,
                                                  const int64_t* __restrict__ srow,
                                                  const int32_t* __restrict__ sproj,
                                                  const double2* __restrict__ sval,
                                                  const double2* __restrict__ P, int64_t nsup, double alpha) {
  const int lane = threadIdx.x & 31;
  const int64_t s = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int col = blockIdx.y * 32 + lane;
  if (s >= nsup || col >= ncol) return;
  double ar = 0.0, ai = 0.0;
  for (int64_t t = srow[s]; t < srow[s + 1]; ++t) {
    const double2 cv = sval[t];
    const double2 pv = P[(int64_t)sproj[t] * ncol + col];
    ar = fma(cv.x, pv.x, fma(-cv.y, pv.y, ar));
    ai = fma(cv.x, pv.y, fma(cv.y, pv.x, ai));
  }
  double2* z = Z + (int64_t)snode[s] * ldz + col;
  z->x += alpha * ar;
  z->y += alpha * ai;
}

// FP32 forms for the mixed filter (complex64 vectors): Z += alpha (-i) sum_d G~1_d X along
// axis d (the 1/2|k|^2 and recurrence terms are in the assembly that precedes it)
__global__ void __launch_bounds__(256) k_kin_add32(float2* __restrict__ Z, int64_t ldz,
                                                   const float2* __restrict__ X, int64_t ldx, int64_t M, int ncol,
                                                   float alpha, const float* __restrict__ tab, int p, int64_t g0,
                                                   int64_t g1, int kbits) {
  // one warp per node (its mesh position computed once, in 32-bit arithmetic: M < 2^31);
  // lane l takes complex columns 64 blockIdx.y + 2l and + 1 (one 16-byte load per
  // neighbour row); the neighbours are summed axis by axis in increasing offset, per column
  extern __shared__ float tsf[];
  const int W = 2 * p + 1;
  for (int t = threadIdx.x; t < 3 * p * W; t += blockDim.x) tsf[t] = tab[t];
  __syncthreads();
  const unsigned i = blockIdx.x * 8u + (threadIdx.x >> 5);
  const int c = blockIdx.y * 64 + 2 * (threadIdx.x & 31);
  if ((int64_t)i >= M || c >= ncol) return;
  const bool two = c + 1 < ncol;
  const unsigned G0 = (unsigned)g0, G1 = (unsigned)g1, G2 = (unsigned)M / (G0 * G1);
  const unsigned iy_all = i / G0;
  const unsigned pos[3] = {i - iy_all * G0, iy_all % G1, iy_all / G1};
  const unsigned ext[3] = {G0, G1, G2};
  const unsigned stride[3] = {1u, G0, G0 * G1};
  float sr0 = 0.f, si0 = 0.f, sr1 = 0.f, si1 = 0.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (!(kbits & (1 << d))) continue;
    const int a = (int)(pos[d] % (unsigned)p);
    const float* T = tsf + (d * p + a) * W + p;
    for (int o = a == 0 ? -p : -a; o <= p - a; ++o) {
      int j = (int)pos[d] + o;
      j += j < 0 ? (int)ext[d] : (j >= (int)ext[d] ? -(int)ext[d] : 0);
      const unsigned row = i + (unsigned)(j - (int)pos[d]) * stride[d];
      const float2* src = X + (int64_t)row * ldx + c;
      const float t = T[o];
      if (two) {
        const float4 v = *reinterpret_cast<const float4*>(src);
        sr0 = fmaf(t, v.x, sr0);
        si0 = fmaf(t, v.y, si0);
        sr1 = fmaf(t, v.z, sr1);
        si1 = fmaf(t, v.w, si1);
      } else {
        const float2 v = *src;
        sr0 = fmaf(t, v.x, sr0);
        si0 = fmaf(t, v.y, si0);
      }
    }
  }
  float2* z = Z + (int64_t)i * ldz + c;
  if (two) {
    float4 zv = *reinterpret_cast<float4*>(z);
    zv.x = fmaf(alpha, si0, zv.x);
    zv.y = fmaf(-alpha, sr0, zv.y);
    zv.z = fmaf(alpha, si1, zv.z);
    zv.w = fmaf(-alpha, sr1, zv.w);
    *reinterpret_cast<float4*>(z) = zv;
  } else {
    z->x = fmaf(alpha, si0, z->x);
    z->y = fmaf(-alpha, sr0, z->y);
  }
}

__global__ void __launch_bounds__(256) k_nl_add32_z(float2* __restrict__ Z, int64_t ldz, int ncol,
                                                    const int32_t* __restrict__ snode,
                                                    const int64_t* __restrict__ srow,
                                                    const int32_t* __restrict__ sproj,
                                                    const float2* __restrict__ sval,
                                                    const float2* __restrict__ P, int64_t nsup, float alpha) {
  const int lane = threadIdx.x & 31;
  const int64_t s = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int col = blockIdx.y * 32 + lane;
  if (s >= nsup || col >= ncol) return;
  float ar = 0.f, ai = 0.f;
  for (int64_t t = srow[s]; t < srow[s + 1]; ++t) {
    const float2 cv = sval[t];
    const float2 pv = P[(int64_t)sproj[t] * ncol + col];
    ar = fmaf(cv.x, pv.x, fmaf(-cv.y, pv.y, ar));
    ai = fmaf(cv.x, pv.y, fmaf(cv.y, pv.x, ai));
  }
  float2* z = Z + (int64_t)snode[s] * ldz + col;
  z->x = fmaf(alpha, ar, z->x);
  z->y = fmaf(alpha, ai, z->y);
}

__global__ void k_to_f2(float2* __restrict__ dst, const double2* __restrict__ src, int64_t n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) dst[t] = make_float2((float)src[t].x, (float)src[t].y);
}

// pz[e] = pval[e] e^{-i k.disp_e}
__global__ void k_phase_vals(double2* __restrict__ pz, const double* __restrict__ pval,
                             const double* __restrict__ disp, double k0, double k1, double k2, int64_t nnz) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  const double th = k0 * disp[3 * e] + k1 * disp[3 * e + 1] + k2 * disp[3 * e + 2];
  double sn, cs;
  sincos(th, &sn, &cs);
  pz[e] = make_double2(pval[e] * cs, -pval[e] * sn);
}

__global__ void k_gather_z(double2* __restrict__ dst, const double2* __restrict__ src,
                           const int64_t* __restrict__ perm, int64_t n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) dst[t] = src[perm[t]];
}

// In place on the lower triangle of the real Gram G (2N x 2N) of a real view: G -> rho(S),
// S = X^H X.  One thread per 2 x 2 block (a, b), a >= b.
__global__ void k_herm_expand(double* __restrict__ G, int N) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * N) return;
  const int a = (int)(t / N), b = (int)(t % N);
  if (a < b) return;
  const int64_t n2 = 2 * (int64_t)N;
  double* r0 = G + (2 * (int64_t)a) * n2;
  double* r1 = r0 + n2;
  const double sr = r0[2 * b] + r1[2 * b + 1];
  const double si = a > b ? r0[2 * b + 1] - r1[2 * b] : 0.0;
  r0[2 * b] = sr;
  r1[2 * b + 1] = sr;
  if (a > b) r0[2 * b + 1] = si;
  r1[2 * b] = -si;
}

// Lower triangle of the real product G = Xr^T Wr (2N x 2N) -> lower triangle of the complex
// H^ = X^H W (N x N, interleaved), with a real diagonal
__global__ void k_herm_pack(const double* __restrict__ G, int N, double2* __restrict__ H) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * N) return;
  const int a = (int)(t / N), b = (int)(t % N);
  if (a < b) return;
  const int64_t n2 = 2 * (int64_t)N;
  const double* r0 = G + (2 * (int64_t)a) * n2;
  const double* r1 = r0 + n2;
  const double hr = r0[2 * b] + r1[2 * b + 1];
  const double hi = a > b ? r0[2 * b + 1] - r1[2 * b] : 0.0;
  H[t] = make_double2(hr, hi);
}

// rho(Q) (2N x 2N real, row-major) of a complex N x N Q (row-major, interleaved)
__global__ void k_realify(const double2* __restrict__ Q, int N, double* __restrict__ R) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * N) return;
  const int a = (int)(t / N), b = (int)(t % N);
  const double2 q = Q[t];
  const int64_t n2 = 2 * (int64_t)N;
  double* r0 = R + (2 * (int64_t)a) * n2 + 2 * b;
  double* r1 = r0 + n2;
  r0[0] = q.x;
  r0[1] = q.y;
  r1[0] = -q.y;
  r1[1] = q.x;
}

// -------------------------------------------------------------- host side
// k_d G~1_d stencil tables (see the file comment)
// host: tab[(d p + a)(2p+1) + o + p] = k_d G~1_d(i, i + o) for nodes i with i mod p = a
static void stencil_table(const dftfe_mesh_s* m, const double* kvec, double* tab) {
  const int p = m->p, n1 = m->n1, W = 2 * p + 1;
  const auto& w = m->gll.w;
  const auto& D = m->D;
  for (int d = 0; d < 3; ++d) {
    const int64_t gd = m->g[d];
    for (int a = 0; a < p; ++a)
      for (int o = -p; o <= p; ++o) {
        double g = 0.0;
        if (a + o >= 0 && a + o <= p) g += w[a] * D[(size_t)a * n1 + a + o];     // the cell where the node is local a
        if (a == 0 && o <= 0) g += w[p] * D[(size_t)p * n1 + p + o];           // a = 0: also local p of the previous cell
        const int64_t j = ((a + o) % gd + gd) % gd;
        tab[((size_t)d * p + a) * W + (o + p)] = kvec[d] * g / std::sqrt(m->m1[d][a] * m->m1[d][j]);
      }
  }
}

static void build_ktab(dftfe_ham h) {
  auto* m = h->mesh;
  const int p = m->p, W = 2 * p + 1;
  std::vector<double> tab(3 * (size_t)p * W, 0.0);
  stencil_table(m, h->kvec, tab.data());
  if (!h->d_ktab) DFTFE_CHECK_CUDA(cudaMalloc(&h->d_ktab, sizeof(double) * tab.size()));
  if (!h->d_ktab32) DFTFE_CHECK_CUDA(cudaMalloc(&h->d_ktab32, sizeof(float) * tab.size()));
  std::vector<float> tab32(tab.begin(), tab.end());
  DFTFE_CHECK_CUDA(cudaMemcpy(h->d_ktab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice));
  DFTFE_CHECK_CUDA(cudaMemcpy(h->d_ktab32, tab32.data(), sizeof(float) * tab32.size(), cudaMemcpyHostToDevice));
}

static int kbits_of(dftfe_ham h) {
  return (h->kvec[0] != 0.0 ? 1 : 0) | (h->kvec[1] != 0.0 ? 2 : 0) | (h->kvec[2] != 0.0 ? 4 : 0);
}

void require_kpoint(dftfe_ham h) {
  if (!loc(h)->has_potential) throw Error(DFTFE_ERR_STATE, "set the potential first");
  if (!h->has_kpoint) throw Error(DFTFE_ERR_STATE, "set the k-point first (dftfe_ham_set_kpoint)");
  if (h->nproj > 0 && !h->kpoint_nl)
    throw Error(DFTFE_ERR_STATE, "the projectors changed: call dftfe_ham_set_kpoint again");
}

void kpoint_init_terms(dftfe_ham h, const double* X, int64_t ldx, const double* Xp, int64_t ldp, double* Z,
                       int64_t ldz, int ncol, double alpha, double s1, double s2) {
  auto* m = h->mesh;
  const double k2 = h->kvec[0] * h->kvec[0] + h->kvec[1] * h->kvec[1] + h->kvec[2] * h->kvec[2];
  const int p = m->p;
  {
    ProfScope ps(h, "kin_k");
    const size_t sh = sizeof(double) * 3 * p * (2 * p + 1);
    DFTFE_LAUNCH(k_kin_init, nblk(m->M * ncol), 256, sh, h->stream, (double2*)Z, ldz, (const double2*)X, ldx,
                 (const double2*)Xp, ldp, m->M, ncol, s1 + 0.5 * alpha * k2, s2, alpha, h->d_ktab, p, m->g[0],
                 m->g[1], kbits_of(h));
  }
  if (h->nproj > 0) {
    ProfScope ps(h, "nl_z");
    double2* P = (double2*)ws_get(h, "nl_coef_z", sizeof(double2) * h->nproj * (size_t)ncol);
    nl_coef_z_split(h, (const double2*)X, ldx, ncol, (const double2*)h->d_pval_z, P);
    dim3 g2((unsigned)((h->nsup + 7) / 8), (unsigned)((ncol + 31) / 32));
    DFTFE_LAUNCH(k_nl_add_z, g2, 256, 0, h->stream, (double2*)Z, ldz, ncol, h->d_snode, h->d_srow, h->d_sproj,
                 (const double2*)h->d_sval_z, P, h->nsup, alpha);
  }
}

void apply_combo_z(dftfe_ham h, const double* X, int64_t ldx, const double* Xp, int64_t ldp, double* Z,
                   int64_t ldz, int ncol, double alpha, double s1, double s2) {
  require_kpoint(h);
  if (ncol <= 0) return;
  kpoint_init_terms(h, X, ldx, Xp, ldp, Z, ldz, ncol, alpha, s1, s2);
  local_part_fp64(h, X, 2 * ldx, Z, 2 * ldz, 2 * ncol, alpha);
}

void kpoint_add32(dftfe_ham h, const float* X, int64_t ldx, float* Z, int64_t ldz, int ncolz, float alpha) {
  require_kpoint(h);
  auto* m = h->mesh;
  if (ncolz <= 0) return;
  const int p = m->p;
  {
    ProfScope ps(h, "kin_k32");
    const size_t sh = sizeof(float) * 3 * p * (2 * p + 1);
    // 8 nodes per CTA, 64 complex columns per blockIdx.y; the complex row strides ldx / 2 and
    // ldz / 2 are multiples of 2, so the two-column accesses are 16-byte aligned
    dim3 grid((unsigned)((m->M + 7) / 8), (unsigned)((ncolz + 63) / 64));
    DFTFE_LAUNCH(k_kin_add32, grid, 256, sh, h->stream, (float2*)Z, ldz / 2, (const float2*)X, ldx / 2,
                 m->M, ncolz, alpha, h->d_ktab32, p, m->g[0], m->g[1], kbits_of(h));
  }
  if (h->nproj > 0) {
    ProfScope ps(h, "nl_z32");
    float2* P = (float2*)ws_get(h, "nl_coef32_z", sizeof(float2) * h->nproj * (size_t)ncolz);
    nl_coef_z_split(h, (const float2*)X, ldx / 2, ncolz, (const float2*)h->d_pval_z32, P);
    dim3 g2((unsigned)((h->nsup + 7) / 8), (unsigned)((ncolz + 31) / 32));
    DFTFE_LAUNCH(k_nl_add32_z, g2, 256, 0, h->stream, (float2*)Z, ldz / 2, ncolz, h->d_snode, h->d_srow, h->d_sproj,
                 (const float2*)h->d_sval_z32, P, h->nsup, alpha);
  }
}

// W = H~^k X with an FP64-accurate local part on the real view (prec: DFTFE_FP64_SLICES, the
// exact digit products, or DFTFE_FP64_FLOAT_PAIRS) and the k-dependent and nonlocal terms in
// FP64: the W of a mixed complex Rayleigh-Ritz
static void apply_z_df(dftfe_ham h, const double* X, int64_t ldx, double* Y, int64_t ldy, int ncol,
                       dftfe_precision prec) {
  require_kpoint(h);
  auto* m = h->mesh;
  if (prec == DFTFE_FP64_SLICES) apply_w(h, X, 2 * ldx, Y, 2 * ldy, 2 * ncol, false);
  else apply_df(h, X, 2 * ldx, Y, 2 * ldy, 2 * ncol, false);
  const double k2 = h->kvec[0] * h->kvec[0] + h->kvec[1] * h->kvec[1] + h->kvec[2] * h->kvec[2];
  const int p = m->p;
  {
    // in place: Y = 1/2|k|^2 X + 1 * Y - i k.grad X (each thread reads and writes its own entry)
    ProfScope ps(h, "kin_k");
    const size_t sh = sizeof(double) * 3 * p * (2 * p + 1);
    DFTFE_LAUNCH(k_kin_init, nblk(m->M * ncol), 256, sh, h->stream, (double2*)Y, ldy, (const double2*)X, ldx,
                 (const double2*)Y, ldy, m->M, ncol, 0.5 * k2, 1.0, 1.0, h->d_ktab, p, m->g[0], m->g[1], kbits_of(h));
  }
  if (h->nproj > 0) {
    ProfScope ps(h, "nl_z");
    double2* P = (double2*)ws_get(h, "nl_coef_z", sizeof(double2) * h->nproj * (size_t)ncol);
    nl_coef_z_split(h, (const double2*)X, ldx, ncol, (const double2*)h->d_pval_z, P);
    dim3 g2((unsigned)((h->nsup + 7) / 8), (unsigned)((ncol + 31) / 32));
    DFTFE_LAUNCH(k_nl_add_z, g2, 256, 0, h->stream, (double2*)Y, ldy, ncol, h->d_snode, h->d_srow, h->d_sproj,
                 (const double2*)h->d_sval_z, P, h->nsup, 1.0);
  }
}

// Eq. chebyfilter on a complex block (the recurrence of chebyshev_filter, real coefficients)
void chebyshev_filter_z_fp64(dftfe_ham h, double* X, int64_t ld, int ncol, int degree, const dftfe_bounds& b) {
  if (degree <= 0 || ncol <= 0) return;
  auto* m = h->mesh;
  const double e = (b.b - b.a) / 2.0, c = (b.b + b.a) / 2.0;
  const bool scaled = !std::isnan(b.a0);
  double* w1 = (double*)ws_get(h, "cheb_w1", sizeof(double) * 2 * m->M * (size_t)ncol);
  double* w2 = (double*)ws_get(h, "cheb_w2", sizeof(double) * 2 * m->M * (size_t)ncol);
  double* buf[3] = {X, w1, w2};
  int64_t lds[3] = {ld, ncol, ncol};
  int cur = 0, prev = -1;
  double sigma = scaled ? e / (b.a0 - c) : 0.0;
  const double sigma1 = sigma, gamma = scaled ? 2.0 / sigma1 : 0.0;
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
    apply_combo_z(h, buf[cur], lds[cur], prev >= 0 ? buf[prev] : nullptr, prev >= 0 ? lds[prev] : 0, buf[out],
                  lds[out], ncol, alpha, s1, s2);
    prev = cur;
    cur = out;
  }
  if (cur != 0) copy_block(h->stream, buf[cur], 2 * lds[cur], X, 2 * ld, m->M, 2 * ncol);
}

// S = X^H X = L L^H, X <- X L^-H, through the real view (file comment)
// mixed: the real-view Gram with FP64 diagonal and FP32-accuracy off-diagonal entries and the
// mixed rotation (the Gamma-point mixed scheme applied to the real view)
static void real_view_gram(dftfe_ham h, const double* A, int64_t lda, const double* B, int64_t ldb, int N2,
                           double* C, bool mixed) {
  auto* m = h->mesh;
  if (mixed) {
    gram_lower_mixed(h, A, lda, B, ldb, m->M, N2, C);
  } else {
    const int nsplit = gram_nsplit(h, m->M, N2);
    double* part = (double*)ws_get(h, "gram_part", sizeof(double) * (size_t)nsplit * N2 * N2);
    gram_lower(h, A, lda, B, ldb, m->M, N2, C, part, nsplit);
  }
}

static void cholgs_z(dftfe_ham h, double* X, int64_t ld, int ncol, bool mixed) {
  auto* m = h->mesh;
  const int N2 = 2 * ncol;
  double* S = (double*)ws_get(h, "S", sizeof(double) * (size_t)N2 * N2);
  double* Z = (double*)ws_get(h, "Zinv", sizeof(double) * (size_t)N2 * N2);
  int* st = (int*)ws_get(h, "status", sizeof(int) * 4);
  real_view_gram(h, X, 2 * ld, X, 2 * ld, N2, S, mixed);
  DFTFE_LAUNCH(k_herm_expand, nblk((int64_t)ncol * ncol), 256, 0, h->stream, S, ncol);
  cholesky_blocked(h, S, N2, st);
  if (read_status_z(h, st) == DFTFE_ERR_NOT_SPD)
    throw Error(DFTFE_ERR_NOT_SPD, "overlap matrix is not positive definite");
  tri_inverse_blocked(h, S, Z, N2);
  if (mixed) rotate_inplace_mixed(h, X, 2 * ld, m->M, N2, Z, true);
  else rotate_inplace(h, X, 2 * ld, m->M, N2, Z, true);
}

// W = H~^k X, H^ = X^H W = Q Theta Q^H, X <- X Q, W <- W Q
static void rayleigh_ritz_z(dftfe_ham h, double* X, int64_t ld, int ncol, double* evals, double* W, int64_t ldw,
                            bool mixed) {
  auto* m = h->mesh;
  const int N2 = 2 * ncol;
  // W FP64-accurate in both precisions (float pairs for the local part of a mixed pass)
  if (mixed) apply_z_df(h, X, ld, W, ldw, ncol, DFTFE_FP64_SLICES);
  else apply_combo_z(h, X, ld, nullptr, 0, W, ldw, ncol, 1.0, 0.0, 0.0);
  double* G = (double*)ws_get(h, "Hhat", sizeof(double) * (size_t)N2 * N2);
  real_view_gram(h, X, 2 * ld, W, 2 * ldw, N2, G, mixed);
  double* Hz = (double*)ws_get(h, "Hz", sizeof(double2) * (size_t)ncol * ncol);
  double* Qz = (double*)ws_get(h, "Qz", sizeof(double2) * (size_t)ncol * ncol);
  double* Qr = (double*)ws_get(h, "Q", sizeof(double) * (size_t)N2 * N2);
  int* st = (int*)ws_get(h, "status", sizeof(int) * 4);
  DFTFE_LAUNCH(k_herm_pack, nblk((int64_t)ncol * ncol), 256, 0, h->stream, G, ncol, (double2*)Hz);
  syevd_z(h, Hz, ncol, evals, Qz, st);
  const int s = read_status_z(h, st);
  if (s == DFTFE_ERR_NOCONV) throw Error(DFTFE_ERR_NOCONV, "subspace eigensolver did not converge");
  if (s != 0) throw Error((dftfe_status)s, "subspace eigensolver: a bounded grid wait timed out");
  DFTFE_LAUNCH(k_realify, nblk((int64_t)ncol * ncol), 256, 0, h->stream, (const double2*)Qz, ncol, Qr);
  if (mixed) {
    rotate_inplace_mixed(h, X, 2 * ld, m->M, N2, Qr, false);
    rotate_inplace_mixed(h, W, 2 * ldw, m->M, N2, Qr, false);
  } else {
    rotate_inplace(h, X, 2 * ld, m->M, N2, Qr, false);
    rotate_inplace(h, W, 2 * ldw, m->M, N2, Qr, false);
  }
}

static bool valid_prec(dftfe_precision prec) {
  return prec == DFTFE_FP64 || prec == DFTFE_MIXED_BF16X3 || prec == DFTFE_MIXED_TF32X3;
}

// the filter of one complex column block in the pass's precision (mixed: FP32 complex vectors,
// split cell products on the real view, FP32 k-terms; err as for chebyshev_filter_mixed)
static void filter_z_any(dftfe_ham h, double* X, int64_t ld, int ncol, int degree, const dftfe_bounds& b,
                         dftfe_precision prec, int* err) {
  if (prec == DFTFE_FP64) chebyshev_filter_z_fp64(h, X, ld, ncol, degree, b);
  else chebyshev_filter_mixed(h, X, 2 * ld, 2 * ncol, degree, b, prec == DFTFE_MIXED_TF32X3, err, true);
}

// the complex pass after its filter: CholGS, Rayleigh-Ritz, residuals, bounds update
void chfsi_pass_tail_z(dftfe_ham h, double* X, int64_t ld, int ncol, dftfe_bounds* inout, double* evals,
                       double* resid, dftfe_precision prec) {
  auto* m = h->mesh;
  const bool mixed = prec != DFTFE_FP64;
  {
    ProfScope ps(h, "pass_cholgs");
    cholgs_z(h, X, ld, ncol, mixed);
  }
  double* W = (double*)ws_get(h, "W", sizeof(double) * 2 * (size_t)m->M * ncol);
  {
    ProfScope ps(h, "pass_rr");
    rayleigh_ritz_z(h, X, ld, ncol, evals, W, ncol, mixed);
  }
  residual_norms(h, X, 2 * ld, W, 2 * (int64_t)ncol, m->M, ncol, evals, resid, 0, 2);
  double ends[2];
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(&ends[0], evals, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(&ends[1], evals + ncol - 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  inout->a = ends[1];
  if (!std::isnan(inout->a0)) inout->a0 = ends[0];
}

}  // namespace dftfe

using namespace dftfe;

extern "C" dftfe_status dftfe_mesh_kpoint_stencil(dftfe_mesh m, const double* kvec, double* table) {
  ABI_BEGIN
  DFTFE_REQUIRE(m && kvec && table, "null argument");
  for (int d = 0; d < 3; ++d) DFTFE_REQUIRE(std::isfinite(kvec[d]), "k must be finite");
  stencil_table(m, kvec, table);
  ABI_END
}

extern "C" dftfe_status dftfe_ham_set_kpoint(dftfe_ham h, const double* kvec, const double* disp) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && kvec, "null argument");
  for (int d = 0; d < 3; ++d) DFTFE_REQUIRE(std::isfinite(kvec[d]), "k must be finite");
  DFTFE_REQUIRE(h->nnz == 0 || disp, "projectors are set: their displacements are required");
  for (int64_t e = 0; disp && e < 3 * h->nnz; ++e) DFTFE_REQUIRE(std::isfinite(disp[e]), "non-finite displacement");
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  for (int d = 0; d < 3; ++d) h->kvec[d] = kvec[d];
  build_ktab(h);
  h->kpoint_nl = false;
  if (h->nnz > 0) {
    const int64_t nnz = h->nnz;
    cudaFree(h->d_pval_z);
    cudaFree(h->d_sval_z);
    h->d_pval_z = h->d_sval_z = nullptr;
    DFTFE_CHECK_CUDA(cudaMalloc(&h->d_pval_z, sizeof(double2) * nnz));
    DFTFE_CHECK_CUDA(cudaMalloc(&h->d_sval_z, sizeof(double2) * nnz));
    struct DevFree {
      double* p = nullptr;
      ~DevFree() { cudaFree(p); }
    } disp_buf;
    DFTFE_CHECK_CUDA(cudaMalloc(&disp_buf.p, sizeof(double) * 3 * nnz));
    double* d_disp = disp_buf.p;
    DFTFE_CHECK_CUDA(cudaMemcpyAsync(d_disp, disp, sizeof(double) * 3 * nnz, cudaMemcpyHostToDevice, h->stream));
    DFTFE_LAUNCH(k_phase_vals, nblk(nnz), 256, 0, h->stream, (double2*)h->d_pval_z, h->d_pval, d_disp, kvec[0],
                 kvec[1], kvec[2], nnz);
    DFTFE_LAUNCH(k_gather_z, nblk(nnz), 256, 0, h->stream, (double2*)h->d_sval_z, (const double2*)h->d_pval_z,
                 h->d_sperm, nnz);
    cudaFree(h->d_pval_z32);
    cudaFree(h->d_sval_z32);
    h->d_pval_z32 = h->d_sval_z32 = nullptr;
    DFTFE_CHECK_CUDA(cudaMalloc(&h->d_pval_z32, sizeof(float2) * nnz));
    DFTFE_CHECK_CUDA(cudaMalloc(&h->d_sval_z32, sizeof(float2) * nnz));
    DFTFE_LAUNCH(k_to_f2, nblk(nnz), 256, 0, h->stream, (float2*)h->d_pval_z32, (const double2*)h->d_pval_z, nnz);
    DFTFE_LAUNCH(k_to_f2, nblk(nnz), 256, 0, h->stream, (float2*)h->d_sval_z32, (const double2*)h->d_sval_z, nnz);
    DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    h->kpoint_nl = true;
  }
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  h->has_kpoint = true;
  ABI_END
}

extern "C" dftfe_status dftfe_ham_apply_z(dftfe_ham h, const double* X, int64_t ldx, double* Y, int64_t ldy,
                                          int ncol, dftfe_precision prec) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && X && Y, "null argument");
  DFTFE_REQUIRE(ncol >= 0 && ldx >= ncol && ldy >= ncol, "bad ncol / leading dimension");
  DFTFE_REQUIRE(valid_prec(prec) || prec == DFTFE_FP64_FLOAT_PAIRS || prec == DFTFE_FP64_SLICES,
                "unknown precision");
  require_kpoint(h);
  if (prec == DFTFE_FP64_SLICES && !slices_applicable(h))
    throw Error(DFTFE_ERR_ARG, "exact-slice products need at most 682 nodes per cell (degree <= 7)");
  if (prec == DFTFE_FP64) apply_combo_z(h, X, ldx, nullptr, 0, Y, ldy, ncol, 1.0, 0.0, 0.0);
  else if (prec == DFTFE_FP64_FLOAT_PAIRS || prec == DFTFE_FP64_SLICES) apply_z_df(h, X, ldx, Y, ldy, ncol, prec);
  else apply_mixed(h, X, 2 * ldx, Y, 2 * ldy, 2 * ncol, prec == DFTFE_MIXED_TF32X3, true);
  ABI_END
}

extern "C" dftfe_status dftfe_lanczos_z(dftfe_ham h, int k, const double* v0, uint64_t seed, double* out3) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && out3, "null argument");
  DFTFE_REQUIRE(k >= 1 && k <= 200, "k must be in 1..200");
  require_kpoint(h);
  lanczos(h, k, v0, seed, out3, true);
  ABI_END
}

extern "C" dftfe_status dftfe_spectrum_bounds_z(dftfe_ham h, int k, uint64_t seed, int nstates,
                                                dftfe_bounds* out) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && out, "null argument");
  DFTFE_REQUIRE(k >= 1 && k <= 200 && nstates >= 1, "bad k / nstates");
  require_kpoint(h);
  double r[3];
  lanczos(h, k, nullptr, seed, r, true);
  const double frac = std::max(4.0 * nstates / (double)h->mesh->M, 0.05);
  out->a0 = r[0];
  out->b = r[2];
  out->a = r[0] + (r[2] - r[0]) * frac;
  ABI_END
}

extern "C" dftfe_status dftfe_chebyshev_filter_z(dftfe_ham h, double* X, int64_t ld, int ncol, int degree,
                                                 const dftfe_bounds* bounds, dftfe_precision prec) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && X && bounds, "null argument");
  DFTFE_REQUIRE(ncol >= 0 && ld >= ncol && degree >= 0, "bad ncol / ld / degree");
  DFTFE_REQUIRE(bounds->b > bounds->a, "need b > a");
  DFTFE_REQUIRE(std::isnan(bounds->a0) || bounds->a0 < bounds->a, "need a0 < a for the scaled filter");
  DFTFE_REQUIRE(valid_prec(prec), "unknown precision");
  require_kpoint(h);
  filter_z_any(h, X, ld, ncol, degree, *bounds, prec, nullptr);
  ABI_END
}

extern "C" dftfe_status dftfe_cholgs_z(dftfe_ham h, double* X, int64_t ld, int ncol, dftfe_precision prec) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && X, "null argument");
  DFTFE_REQUIRE(ncol >= 1 && ncol <= 1024 && ld >= ncol, "bad ncol / ld (at most 1024 complex columns)");
  DFTFE_REQUIRE(ncol <= h->mesh->M, "more columns than DoFs");
  DFTFE_REQUIRE(valid_prec(prec), "unknown precision");
  cholgs_z(h, X, ld, ncol, prec != DFTFE_FP64);
  ABI_END
}

extern "C" dftfe_status dftfe_rayleigh_ritz_z(dftfe_ham h, double* X, int64_t ld, int ncol, double* evals,
                                              double* HX, int64_t ldhx, dftfe_precision prec) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && X && evals, "null argument");
  DFTFE_REQUIRE(ncol >= 1 && ncol <= 1024 && ld >= ncol, "bad ncol / ld (at most 1024 complex columns)");
  DFTFE_REQUIRE(!HX || ldhx >= ncol, "bad ldhx");
  DFTFE_REQUIRE(valid_prec(prec), "unknown precision");
  require_kpoint(h);
  double* W = HX;
  int64_t ldw = ldhx;
  if (!W) {
    W = (double*)ws_get(h, "W", sizeof(double) * 2 * (size_t)h->mesh->M * ncol);
    ldw = ncol;
  }
  rayleigh_ritz_z(h, X, ld, ncol, evals, W, ldw, prec != DFTFE_FP64);
  ABI_END
}

extern "C" dftfe_status dftfe_residuals_z(dftfe_ham h, const double* X, const double* HX, int64_t ld, int ncol,
                                          const double* evals, double* resid, int kind) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && X && HX && evals && resid, "null argument");
  DFTFE_REQUIRE(ncol >= 1 && ld >= ncol, "bad ncol / ld");
  DFTFE_REQUIRE(kind == 0 || kind == 1, "kind must be 0 or 1");
  residual_norms(h, X, 2 * ld, HX, 2 * ld, h->mesh->M, ncol, evals, resid, kind, 2);
  ABI_END
}

extern "C" dftfe_status dftfe_chfsi_pass_z(dftfe_ham h, double* X, int64_t ld, int ncol, int block, int degree,
                                           dftfe_bounds* inout, double* evals, double* resid, dftfe_precision prec) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && X && inout && evals && resid, "null argument");
  DFTFE_REQUIRE(ncol >= 1 && ncol <= 1024 && ld >= ncol && block >= 1 && degree >= 0,
                "bad sizes (at most 1024 complex columns)");
  DFTFE_REQUIRE(ncol <= h->mesh->M, "more columns than DoFs");
  DFTFE_REQUIRE(inout->b > inout->a, "need b > a");
  DFTFE_REQUIRE(std::isnan(inout->a0) || inout->a0 < inout->a, "need a0 < a for the scaled filter");
  DFTFE_REQUIRE(valid_prec(prec), "unknown precision");
  require_kpoint(h);
  const bool mixed = prec != DFTFE_FP64;
  {
    ProfScope ps(h, "pass_filter");
    int* err = nullptr;
    if (mixed) {
      err = (int*)ws_get(h, "mx_err", sizeof(int));
      DFTFE_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), h->stream));
    }
    const dftfe_bounds bnd = *inout;
    const std::string key = "pass_z/" + std::to_string((int)prec) + "/" + std::to_string(ncol) + "/" +
                            std::to_string(block) + "/" + std::to_string(degree);
    run_region(h, key, [&]() {
      for (int j0 = 0; j0 < ncol; j0 += block)
        filter_z_any(h, X + 2 * (int64_t)j0, ld, std::min(block, ncol - j0), degree, bnd, prec, err);
    });
    if (err) {
      int herr = 0;
      DFTFE_CHECK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
      DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
      if (herr) throw Error(DFTFE_ERR_TIMEOUT, "mixed cell kernel: a bounded wait timed out");
    }
  }
  chfsi_pass_tail_z(h, X, ld, ncol, inout, evals, resid, prec);
  ABI_END
}
