// Mesh (a1), cell Hamiltonians (a2) and nonlocal projector setup (a3).
//
// a1 (Sec. 2.3): structured periodic hexahedral mesh of GLL spectral elements, the
//    cell -> global map and the lumped diagonal mass M (text after Eq. hep).  On a
//    uniform periodic mesh M = M1x (x) M1y (x) M1z with M1 the 1D lumped mass, which
//    is how the device builds it.
// a2 (Sec. 4.2, Eq. quadLocal / Eq. gemmLoc): V^c for all cells by one packed-symmetric
//    GEMM K^{eff,loc} = P V with P_{I,q} = N_j(x_q) N_k(x_q) (j <= k) and
//    V_{q,c} = w_q detJ V(x_q^c); the GLL stiffness K^c = 1/2 int grad N . grad N is
//    shared by all cells; H~^c = D_c^-1/2 (K^c + V^c) D_c^-1/2 (Eq. hep, Eq. celldgemm).
// a3 (Eq. nonlocalHamDiscrete, Alg. 4): C_ja = M_jj chi_a(x_j) (GLL collocation), stored
//    as C~ = M^1/2 chi in CSR by projector and by node.
#include "internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace dftfe {

std::atomic<int64_t> g_launches{0};
static thread_local std::string t_last_error;
void set_error(const std::string& msg) { t_last_error = msg; }
void clear_error() { t_last_error.clear(); }
const char* last_error() { return t_last_error.c_str(); }


void* DevBuf::get(size_t need) {
  if (need <= bytes && ptr) return ptr;
  if (ptr) {
    cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
  }
  size_t alloc = std::max<size_t>(need, 256);
  DFTFE_CHECK_CUDA(cudaMalloc(&ptr, alloc));
  bytes = alloc;
  return ptr;
}
void DevBuf::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
}

// buffers that live only inside one pass tail (CholGS, Rayleigh-Ritz, residuals): in a batched
// pass they come from the batch's shared tail workspace
static bool tail_buffer(const char* name) {
  static const char* const names[] = {"S", "Zinv", "gram_part", "Hhat", "Q", "W", "chol_d0", "chol_linv",
                                      "eig_V", "eigz_V", "eig_vec", "eig_perm", "resid_part", "coldot_part",
                                      "gram32_part", "rotmix_Zf", "rotmix_zd", "Hz", "Qz", "rot_tc_tiles",
                                      "rot_tc_zd", "rot_tc_out", "gram_tc_part", "slices_x", "slices_xe"};
  for (const char* n : names)
    if (std::strcmp(n, name) == 0) return true;
  return false;
}

void* ws_get(dftfe_ham h, const char* name, size_t bytes) {
  DevBuf& b = (h->tail_ws && tail_buffer(name)) ? (*h->tail_ws)[name] : h->ws[name];
  if (bytes > b.bytes && b.ptr) DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  return b.get(bytes);
}

ProfScope::ProfScope(dftfe_ham ham, const char* name) : h(ham) {
  if (!h || !h->profiling) return;
  t = &h->timers[name];
  if (t->used == t->events.size()) {
    cudaEvent_t a, b;
    DFTFE_CHECK_CUDA(cudaEventCreate(&a));
    DFTFE_CHECK_CUDA(cudaEventCreate(&b));
    t->events.push_back({a, b});
  }
  auto& ev = t->events[t->used++];
  e1 = ev.second;
  DFTFE_CHECK_CUDA(cudaEventRecord(ev.first, h->stream));
}
ProfScope::~ProfScope() {
  if (t) {
    cudaEventRecord(e1, h->stream);
    t->launches++;
  }
}

// ------------------------------------------------------------------ kernels

// cell_map[c*nc + (a + n1*(b + n1*cc))] = global node of local (a, b, cc) in cell c
__global__ void k_cell_map(int32_t* map, int64_t Nc, int n1, int p, int nx, int ny,
                           int64_t gx, int64_t gy, int64_t gz) {
  const int nc = n1 * n1 * n1;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Nc * nc) return;
  int64_t c = t / nc;
  int l = (int)(t % nc);
  int a = l % n1, b = (l / n1) % n1, cc = l / (n1 * n1);
  int64_t cx = c % nx, cy = (c / nx) % ny, cz = c / ((int64_t)nx * ny);
  int64_t ix = (cx * p + a) % gx, iy = (cy * p + b) % gy, iz = (cz * p + cc) % gz;
  map[t] = (int32_t)(ix + gx * (iy + gy * iz));
}

// M_jj = m1x[ix] m1y[iy] m1z[iz]; also M^-1/2.
__global__ void k_mass(double* mass, double* minvsqrt, const double* m1x, const double* m1y,
                       const double* m1z, int64_t gx, int64_t gy, int64_t M) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= M) return;
  int64_t ix = j % gx, iy = (j / gx) % gy, iz = j / (gx * gy);
  double m = m1x[ix] * m1y[iy] * m1z[iz];
  mass[j] = m;
  minvsqrt[j] = 1.0 / sqrt(m);
}

// P[I*nq + q] = N_j(x_q) N_k(x_q), (j, k) = pairs[I], tensor-product basis values.
__global__ void k_products(double* P, const int32_t* pairs, const double* Lq, int64_t Msym,
                           int nq1, int n1) {
  const int nq = nq1 * nq1 * nq1;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= Msym * nq) return;
  int64_t I = t / nq;
  int q = (int)(t % nq);
  int j = pairs[2 * I], k = pairs[2 * I + 1];
  int qa = q % nq1, qb = (q / nq1) % nq1, qc = q / (nq1 * nq1);
  int ja = j % n1, jb = (j / n1) % n1, jc = j / (n1 * n1);
  int ka = k % n1, kb = (k / n1) % n1, kc = k / (n1 * n1);
  double Nj = Lq[qa * n1 + ja] * Lq[qb * n1 + jb] * Lq[qc * n1 + jc];
  double Nk = Lq[qa * n1 + ka] * Lq[qb * n1 + kb] * Lq[qc * n1 + kc];
  P[t] = Nj * Nk;
}

// Packed-symmetric DHM GEMM with the Loewdin epilogue:
//   Keff[I, c] = sum_q P[I, q] (wq[q] V[c, q]);
//   Hc[c][j][k] = Hc[c][k][j] = d_j (K[j][k] + Keff[I, c]) d_k, d = M^-1/2 at the cell's nodes.
constexpr int PV_BM = 64, PV_BN = 64, PV_BK = 16;
__global__ void __launch_bounds__(256) k_pv_gemm(
    const double* __restrict__ P, const double* __restrict__ V, const double* __restrict__ wq,
    const int32_t* __restrict__ pairs, const double* __restrict__ K,
    const int32_t* __restrict__ map, const double* __restrict__ minvsqrt,
    double* __restrict__ Hc, int64_t Msym, int64_t Nc, int nq, int nc) {
  __shared__ double As[PV_BK][PV_BM + 1];
  __shared__ double Bs[PV_BK][PV_BN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t I0 = blockIdx.x * (int64_t)PV_BM;
  const int64_t c0 = blockIdx.y * (int64_t)PV_BN;
  double acc[4][4] = {};
  for (int q0 = 0; q0 < nq; q0 += PV_BK) {
    for (int e = threadIdx.x; e < PV_BK * PV_BM; e += 256) {
      int kk = e % PV_BK, i = e / PV_BK;
      int64_t I = I0 + i;
      int q = q0 + kk;
      As[kk][i] = (I < Msym && q < nq) ? P[I * nq + q] : 0.0;
      int64_t c = c0 + i;
      Bs[kk][i] = (c < Nc && q < nq) ? V[c * nq + q] * wq[q] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < PV_BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t I = I0 + ty * 4 + i;
    if (I >= Msym) continue;
    int jn = pairs[2 * I], kn = pairs[2 * I + 1];
    double kv = K[(int64_t)jn * nc + kn];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t c = c0 + tx * 4 + j;
      if (c >= Nc) continue;
      double dj = minvsqrt[map[c * nc + jn]];
      double dk = minvsqrt[map[c * nc + kn]];
      double v = dj * (kv + acc[i][j]) * dk;
      double* H = Hc + c * (int64_t)nc * nc;
      H[(int64_t)jn * nc + kn] = v;
      if (jn != kn) H[(int64_t)kn * nc + jn] = v;
    }
  }
}

__global__ void k_scale_by_sqrt_mass(double* out, const double* chi, const int32_t* node,
                                     const double* mass, int64_t n) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) out[t] = sqrt(mass[node[t]]) * chi[t];
}

__global__ void k_gather_vals(double* out, const double* in, const int64_t* perm, int64_t n) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) out[t] = in[perm[t]];
}

static unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

template <class T>
static T* dev_upload(const std::vector<T>& v, cudaStream_t s) {
  T* p = nullptr;
  DFTFE_CHECK_CUDA(cudaMalloc(&p, std::max<size_t>(v.size(), 1) * sizeof(T)));
  if (!v.empty())
    DFTFE_CHECK_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return p;
}

static void free_nonlocal(dftfe_ham h) {
  cudaFree(h->d_h); cudaFree(h->d_prow); cudaFree(h->d_pnode); cudaFree(h->d_pval);
  cudaFree(h->d_snode); cudaFree(h->d_srow); cudaFree(h->d_sproj); cudaFree(h->d_sval);
  cudaFree(h->d_nptr_all); cudaFree(h->d_sperm); cudaFree(h->d_pval_z); cudaFree(h->d_sval_z);
  cudaFree(h->d_pval_z32); cudaFree(h->d_sval_z32);
  h->d_pval_z32 = nullptr; h->d_sval_z32 = nullptr;
  h->d_h = nullptr; h->d_prow = nullptr; h->d_pnode = nullptr; h->d_pval = nullptr;
  h->d_snode = nullptr; h->d_srow = nullptr; h->d_sproj = nullptr; h->d_sval = nullptr;
  h->d_nptr_all = nullptr; h->d_sperm = nullptr; h->d_pval_z = nullptr; h->d_sval_z = nullptr;
  h->nproj = 0;
  h->nsup = 0;
  h->nnz = 0;
  h->kpoint_nl = false;   // the phased projector values belong to the old CSR
}

}  // namespace dftfe

using namespace dftfe;

extern "C" dftfe_status dftfe_mesh_create(const dftfe_mesh_desc* d, dftfe_mesh* out) {
  ABI_BEGIN
  DFTFE_REQUIRE(d && out, "null argument");
  DFTFE_REQUIRE(d->degree >= 1 && d->degree <= 8, "degree must be in 1..8");
  DFTFE_REQUIRE(d->vquad == 0 || d->vquad == 1, "vquad must be 0 or 1");
  DFTFE_REQUIRE(d->nq1d >= 0 && d->nq1d <= 12, "nq1d must be in 0..12");
  for (int a = 0; a < 3; ++a) {
    DFTFE_REQUIRE(d->ncell[a] >= 2, "need at least 2 cells per axis");
    DFTFE_REQUIRE(d->L[a] > 0 && std::isfinite(d->L[a]), "box lengths must be positive");
    DFTFE_REQUIRE(d->periodic[a] == 1, "only fully periodic meshes are supported");
  }
  auto* m = new dftfe_mesh_s();
  m->p = d->degree;
  m->n1 = m->p + 1;
  m->nc = m->n1 * m->n1 * m->n1;
  m->vquad = d->vquad;
  m->nq1d = d->nq1d ? d->nq1d : m->p + 1;
  m->nq1 = m->vquad == 1 ? m->n1 : m->nq1d;
  m->nq = m->nq1 * m->nq1 * m->nq1;
  m->M = 1;
  m->Nc = 1;
  for (int a = 0; a < 3; ++a) {
    m->L[a] = d->L[a];
    m->n[a] = d->ncell[a];
    m->g[a] = (int64_t)d->ncell[a] * m->p;
    m->h[a] = d->L[a] / d->ncell[a];
    m->M *= m->g[a];
    m->Nc *= m->n[a];
  }
  if (m->M >= (int64_t)INT32_MAX) {
    delete m;
    throw Error(DFTFE_ERR_ARG, "more than 2^31-1 DoFs");
  }
  m->detJ = m->h[0] * m->h[1] * m->h[2] / 8.0;
  m->gll = gll_rule(m->p);
  m->quad = m->vquad == 1 ? m->gll : gauss_rule(m->nq1);
  m->D = derivative_matrix(m->gll.x);
  m->Lq = lagrange_at(m->gll.x, m->quad.x);
  for (int a = 0; a < 3; ++a) {
    m->m1[a].assign(m->g[a], 0.0);
    for (int c = 0; c < m->n[a]; ++c)
      for (int i = 0; i <= m->p; ++i)
        m->m1[a][(c * (int64_t)m->p + i) % m->g[a]] += m->gll.w[i] * m->h[a] / 2.0;
  }
  *out = m;
  ABI_END
}

extern "C" dftfe_status dftfe_mesh_info(dftfe_mesh m, int64_t* ndofs, int64_t* ncells,
                                        int* nodes_per_cell, int* quad_per_cell) {
  ABI_BEGIN
  DFTFE_REQUIRE(m, "null mesh");
  if (ndofs) *ndofs = m->M;
  if (ncells) *ncells = m->Nc;
  if (nodes_per_cell) *nodes_per_cell = m->nc;
  if (quad_per_cell) *quad_per_cell = m->nq;
  ABI_END
}

extern "C" dftfe_status dftfe_mesh_coords(dftfe_mesh m, double* node_xyz, double* quad_xyz) {
  ABI_BEGIN
  DFTFE_REQUIRE(m, "null mesh");
  if (node_xyz) {
    for (int64_t j = 0; j < m->M; ++j) {
      int64_t idx[3] = {j % m->g[0], (j / m->g[0]) % m->g[1], j / (m->g[0] * m->g[1])};
      for (int a = 0; a < 3; ++a) {
        int64_t cell = idx[a] / m->p;
        int loc = (int)(idx[a] % m->p);
        node_xyz[3 * j + a] = cell * m->h[a] + (m->gll.x[loc] + 1.0) * m->h[a] / 2.0;
      }
    }
  }
  if (quad_xyz) {
    const int nq1 = m->nq1;
    for (int64_t c = 0; c < m->Nc; ++c) {
      int64_t cc[3] = {c % m->n[0], (c / m->n[0]) % m->n[1], c / ((int64_t)m->n[0] * m->n[1])};
      for (int q = 0; q < m->nq; ++q) {
        int qi[3] = {q % nq1, (q / nq1) % nq1, q / (nq1 * nq1)};
        for (int a = 0; a < 3; ++a)
          quad_xyz[(c * m->nq + q) * 3 + a] = cc[a] * m->h[a] + (m->quad.x[qi[a]] + 1.0) * m->h[a] / 2.0;
      }
    }
  }
  ABI_END
}

extern "C" dftfe_status dftfe_mesh_destroy(dftfe_mesh m) {
  ABI_BEGIN
  delete m;
  ABI_END
}

// ----------------------------------------------------------------- ABI: ham
// A ham over mesh m on `stream`; with src, one that uses src's local operator (no cell
// matrices or packed basis products of its own).
static dftfe_ham create_ham(dftfe_mesh m, void* stream, dftfe_ham src) {
  auto* h = new dftfe_ham_s();
  try {
    h->mesh = m;
    h->local_src = src;
    h->stream = (cudaStream_t)stream;
    DFTFE_CHECK_CUDA(cudaGetDevice(&h->device));
    DFTFE_CHECK_CUDA(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device));
    cudaStream_t s = h->stream;
    const int nc = m->nc, n1 = m->n1;
    // a1: map and lumped mass
    DFTFE_CHECK_CUDA(cudaMalloc(&h->d_map, sizeof(int32_t) * m->Nc * nc));
    DFTFE_LAUNCH(k_cell_map, nblk(m->Nc * nc), 256, 0, s, h->d_map, m->Nc, n1, m->p, m->n[0],
                 m->n[1], m->g[0], m->g[1], m->g[2]);
    DFTFE_CHECK_CUDA(cudaMalloc(&h->d_mass, sizeof(double) * m->M));
    DFTFE_CHECK_CUDA(cudaMalloc(&h->d_minvsqrt, sizeof(double) * m->M));
    {
      double* m1[3];
      for (int a = 0; a < 3; ++a) m1[a] = dev_upload(m->m1[a], s);
      DFTFE_LAUNCH(k_mass, nblk(m->M), 256, 0, s, h->d_mass, h->d_minvsqrt, m1[0], m1[1], m1[2],
                   m->g[0], m->g[1], m->M);
      DFTFE_CHECK_CUDA(cudaStreamSynchronize(s));
      for (int a = 0; a < 3; ++a) cudaFree(m1[a]);
    }
    // colouring: per axis 2 colours (even count) or 3 (odd count, last cell apart)
    {
      int ncol_ax[3];
      for (int a = 0; a < 3; ++a) ncol_ax[a] = (m->n[a] % 2 == 0) ? 2 : 3;
      h->ncolours = ncol_ax[0] * ncol_ax[1] * ncol_ax[2];
      std::vector<std::vector<int32_t>> lists(h->ncolours);
      for (int64_t c = 0; c < m->Nc; ++c) {
        int64_t cc[3] = {c % m->n[0], (c / m->n[0]) % m->n[1], c / ((int64_t)m->n[0] * m->n[1])};
        int k[3];
        for (int a = 0; a < 3; ++a)
          k[a] = (ncol_ax[a] == 3 && cc[a] == m->n[a] - 1) ? 2 : (int)(cc[a] % 2);
        lists[k[0] + ncol_ax[0] * (k[1] + ncol_ax[1] * k[2])].push_back((int32_t)c);
      }
      std::vector<int32_t> flat;
      h->colour_off.assign(1, 0);
      for (auto& l : lists) {
        flat.insert(flat.end(), l.begin(), l.end());
        h->colour_off.push_back((int64_t)flat.size());
      }
      h->d_colour_cells = dev_upload(flat, s);
    }
    // a2 reference-cell tables: stiffness (Kronecker form of the GLL quadrature) and P
    {
      const auto& w = m->gll.w;
      const auto& D = m->D;
      std::vector<double> k1[3], mm1[3];
      for (int a = 0; a < 3; ++a) {
        k1[a].assign(n1 * n1, 0.0);
        mm1[a].assign(n1, 0.0);
        for (int i = 0; i < n1; ++i) {
          mm1[a][i] = m->h[a] / 2.0 * w[i];
          for (int j = 0; j < n1; ++j) {
            double s1 = 0.0;
            for (int q = 0; q < n1; ++q) s1 += w[q] * D[q * n1 + i] * D[q * n1 + j];
            k1[a][i * n1 + j] = 2.0 / m->h[a] * s1;
          }
        }
      }
      std::vector<double> K((size_t)nc * nc, 0.0);
      for (int j = 0; j < nc; ++j) {
        int a = j % n1, b = (j / n1) % n1, c = j / (n1 * n1);
        for (int k = 0; k < nc; ++k) {
          int d = k % n1, e = (k / n1) % n1, f = k / (n1 * n1);
          double v = 0.0;
          if (b == e && c == f) v += k1[0][a * n1 + d] * mm1[1][b] * mm1[2][c];
          if (a == d && c == f) v += mm1[0][a] * k1[1][b * n1 + e] * mm1[2][c];
          if (a == d && b == e) v += mm1[0][a] * mm1[1][b] * k1[2][c * n1 + f];
          K[(size_t)j * nc + k] = 0.5 * v;
        }
      }
      h->d_K = dev_upload(K, s);
      const int64_t Msym = (int64_t)nc * (nc + 1) / 2;
      std::vector<int32_t> pairs(2 * Msym);
      int64_t I = 0;
      for (int j = 0; j < nc; ++j)
        for (int k = j; k < nc; ++k) {
          pairs[2 * I] = j;
          pairs[2 * I + 1] = k;
          ++I;
        }
      h->d_pairs = dev_upload(pairs, s);
      std::vector<double> wq(m->nq);
      for (int q = 0; q < m->nq; ++q) {
        int qa = q % m->nq1, qb = (q / m->nq1) % m->nq1, qc = q / (m->nq1 * m->nq1);
        wq[q] = m->quad.w[qa] * m->quad.w[qb] * m->quad.w[qc] * m->detJ;
      }
      h->d_wq = dev_upload(wq, s);
      std::vector<double> Nq((size_t)m->nq * nc);
      for (int q = 0; q < m->nq; ++q) {
        const int qa = q % m->nq1, qb = (q / m->nq1) % m->nq1, qc = q / (m->nq1 * m->nq1);
        for (int j = 0; j < nc; ++j) {
          const int a = j % n1, b = (j / n1) % n1, c = j / (n1 * n1);
          Nq[(size_t)q * nc + j] = m->Lq[qa * n1 + a] * m->Lq[qb * n1 + b] * m->Lq[qc * n1 + c];
        }
      }
      h->d_Nq = dev_upload(Nq, s);
      if (!src) {
        double* d_Lq = dev_upload(m->Lq, s);
        DFTFE_CHECK_CUDA(cudaMalloc(&h->d_P, sizeof(double) * Msym * m->nq));
        DFTFE_LAUNCH(k_products, nblk(Msym * m->nq), 256, 0, s, h->d_P, h->d_pairs, d_Lq, Msym,
                     m->nq1, n1);
        DFTFE_CHECK_CUDA(cudaStreamSynchronize(s));
        cudaFree(d_Lq);
      }
    }
    if (!src) DFTFE_CHECK_CUDA(cudaMalloc(&h->d_Hc, sizeof(double) * m->Nc * (int64_t)nc * nc));
  } catch (...) {
    h->local_src = nullptr;
    dftfe_ham_destroy(h);
    throw;
  }
  if (src) src->sharers++;
  return h;
}

extern "C" dftfe_status dftfe_ham_create(dftfe_mesh m, void* stream, dftfe_ham* out) {
  ABI_BEGIN
  DFTFE_REQUIRE(m && out, "null argument");
  *out = create_ham(m, stream, nullptr);
  ABI_END
}

extern "C" dftfe_status dftfe_ham_create_shared(dftfe_ham src, dftfe_ham* out) {
  ABI_BEGIN
  DFTFE_REQUIRE(src && out, "null argument");
  DFTFE_REQUIRE(!src->local_src, "src must own its local operator (not itself made by dftfe_ham_create_shared)");
  int dev = -1;
  DFTFE_CHECK_CUDA(cudaGetDevice(&dev));
  DFTFE_REQUIRE(dev == src->device, "the current device must be src's");
  *out = create_ham(src->mesh, (void*)src->stream, src);
  ABI_END
}

extern "C" dftfe_status dftfe_ham_set_potential(dftfe_ham h, const double* v_quad) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && v_quad, "null argument");
  if (h->local_src)
    throw Error(DFTFE_ERR_STATE, "this ham uses another ham's local operator: set the potential on that ham");
  auto* m = h->mesh;
  const int64_t Msym = (int64_t)m->nc * (m->nc + 1) / 2;
  dim3 grid((unsigned)((Msym + PV_BM - 1) / PV_BM), (unsigned)((m->Nc + PV_BN - 1) / PV_BN));
  {
    ProfScope ps(h, "dhm_gemm");
    DFTFE_LAUNCH(k_pv_gemm, grid, 256, 0, h->stream, h->d_P, v_quad, h->d_wq, h->d_pairs, h->d_K,
                 h->d_map, h->d_minvsqrt, h->d_Hc, Msym, m->Nc, m->nq, m->nc);
  }
  h->has_potential = true;
  h->potential_version++;
  ABI_END
}

extern "C" dftfe_status dftfe_ham_set_nonlocal(dftfe_ham h, int nproj, const double* hcoup,
                                               const int64_t* rowptr, const int64_t* node,
                                               const double* chi) {
  ABI_BEGIN
  DFTFE_REQUIRE(h, "null ham");
  DFTFE_REQUIRE(nproj >= 0, "nproj must be >= 0");
  auto* m = h->mesh;
  if (nproj == 0) {
    DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
    free_nonlocal(h);
    return DFTFE_OK;
  }
  DFTFE_REQUIRE(hcoup && rowptr && node && chi, "null CSR input");
  DFTFE_REQUIRE(rowptr[0] == 0, "rowptr[0] must be 0");
  for (int a = 0; a < nproj; ++a) DFTFE_REQUIRE(rowptr[a + 1] >= rowptr[a], "rowptr not monotone");
  const int64_t nnz = rowptr[nproj];
  for (int64_t e = 0; e < nnz; ++e)
    DFTFE_REQUIRE(node[e] >= 0 && node[e] < m->M, "projector node index out of range");
  // node-major transpose (counting sort over the support nodes)
  std::vector<int32_t> pnode(nnz);
  for (int64_t e = 0; e < nnz; ++e) pnode[e] = (int32_t)node[e];
  std::vector<int64_t> order(nnz);
  for (int64_t e = 0; e < nnz; ++e) order[e] = e;
  std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return node[x] < node[y]; });
  std::vector<int32_t> snode, sproj(nnz);
  std::vector<int64_t> srow;
  std::vector<int64_t> eproj(nnz);
  for (int a = 0; a < nproj; ++a)
    for (int64_t e = rowptr[a]; e < rowptr[a + 1]; ++e) eproj[e] = a;
  for (int64_t t = 0; t < nnz; ++t) {
    int64_t e = order[t];
    if (snode.empty() || snode.back() != (int32_t)node[e]) {
      snode.push_back((int32_t)node[e]);
      srow.push_back(t);
    }
    sproj[t] = (int32_t)eproj[e];
  }
  srow.push_back(nnz);
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  free_nonlocal(h);
  cudaStream_t s = h->stream;
  h->nproj = nproj;
  h->nnz = nnz;
  h->nsup = (int64_t)snode.size();
  h->d_h = dev_upload(std::vector<double>(hcoup, hcoup + nproj), s);
  h->d_prow = dev_upload(std::vector<int64_t>(rowptr, rowptr + nproj + 1), s);
  h->d_pnode = dev_upload(pnode, s);
  double* d_chi = dev_upload(std::vector<double>(chi, chi + nnz), s);
  DFTFE_CHECK_CUDA(cudaMalloc(&h->d_pval, sizeof(double) * std::max<int64_t>(nnz, 1)));
  if (nnz)
    DFTFE_LAUNCH(k_scale_by_sqrt_mass, nblk(nnz), 256, 0, s, h->d_pval, d_chi, h->d_pnode,
                 h->d_mass, nnz);
  h->d_snode = dev_upload(snode, s);
  h->d_srow = dev_upload(srow, s);
  {
    // the same node-major entries indexed by every node (empty ranges off the supports)
    std::vector<int64_t> nall(m->M + 1, 0);
    for (size_t k = 0; k < snode.size(); ++k) nall[(size_t)snode[k] + 1] = srow[k + 1] - srow[k];
    for (int64_t g = 0; g < m->M; ++g) nall[g + 1] += nall[g];
    h->d_nptr_all = dev_upload(nall, s);
  }
  h->d_sproj = dev_upload(sproj, s);
  // node-major position t holds projector-major entry sperm[t] (kept for the k-point values)
  h->d_sperm = dev_upload(order, s);
  DFTFE_CHECK_CUDA(cudaMalloc(&h->d_sval, sizeof(double) * std::max<int64_t>(nnz, 1)));
  if (nnz) DFTFE_LAUNCH(k_gather_vals, nblk(nnz), 256, 0, s, h->d_sval, h->d_pval, h->d_sperm, nnz);
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(s));
  cudaFree(d_chi);
  ABI_END
}

extern "C" dftfe_status dftfe_ham_destroy(dftfe_ham h) {
  ABI_BEGIN
  if (!h) return DFTFE_OK;
  if (h->sharers > 0)
    throw Error(DFTFE_ERR_STATE, "hams made by dftfe_ham_create_shared still use this ham: destroy them first");
  if (h->local_src) h->local_src->sharers--;
  cudaStreamSynchronize(h->stream);
  free_graphs(h);
  if (h->h_pass) cudaFreeHost(h->h_pass);
  free_nonlocal(h);
  cudaFree(h->d_map); cudaFree(h->d_mass); cudaFree(h->d_minvsqrt);
  cudaFree(h->d_colour_cells); cudaFree(h->d_node_ptr); cudaFree(h->d_node_slot); cudaFree(h->d_K); cudaFree(h->d_P); cudaFree(h->d_pairs);
  cudaFree(h->d_wq); cudaFree(h->d_Hc); cudaFree(h->d_Nq); cudaFree(h->d_ktab); cudaFree(h->d_ktab32);
  for (auto& kv : h->ws) kv.second.release();
  for (auto& kv : h->timers)
    for (auto& ev : kv.second.events) {
      cudaEventDestroy(ev.first);
      cudaEventDestroy(ev.second);
    }
  delete h;
  ABI_END
}

extern "C" dftfe_status dftfe_ham_export(dftfe_ham h, double* mass, int32_t* cell_map, int64_t c0,
                                         int64_t count, double* cell_mats) {
  ABI_BEGIN
  DFTFE_REQUIRE(h, "null ham");
  auto* m = h->mesh;
  cudaStream_t s = h->stream;
  if (mass)
    DFTFE_CHECK_CUDA(cudaMemcpyAsync(mass, h->d_mass, sizeof(double) * m->M, cudaMemcpyDeviceToDevice, s));
  if (cell_map)
    DFTFE_CHECK_CUDA(cudaMemcpyAsync(cell_map, h->d_map, sizeof(int32_t) * m->Nc * m->nc,
                                     cudaMemcpyDeviceToDevice, s));
  if (cell_mats) {
    DFTFE_REQUIRE(c0 >= 0 && count >= 0 && c0 + count <= m->Nc, "cell range out of bounds");
    DFTFE_REQUIRE(loc(h)->has_potential, "no potential set");
    const int64_t n2 = (int64_t)m->nc * m->nc;
    DFTFE_CHECK_CUDA(cudaMemcpyAsync(cell_mats, loc(h)->d_Hc + c0 * n2, sizeof(double) * count * n2,
                                     cudaMemcpyDeviceToDevice, s));
  }
  ABI_END
}

extern "C" int64_t dftfe_launch_count(void) { return g_launches.load(); }
extern "C" const char* dftfe_last_error(void) { return dftfe::last_error(); }
