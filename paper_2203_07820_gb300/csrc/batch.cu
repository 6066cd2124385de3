// Batched ChFSI passes (FP64): independent systems of uneven mesh size, degree, state count
// and block size -- at the Gamma point or, item by item, at the ham's Bloch k-point with a
// complex block -- filtered with shared launches.  Per Chebyshev step one launch forms
// s1 X_k + s2 X_{k-1} for every real system (a complex system forms it with its k.grad
// stencil, as a single k-point pass does), and one launch per colour runs the cell products
// of every system's cells of that colour (a work list of (system, cell) pairs built once; a
// complex block enters as its real view); the nonlocal term is added per system.  The
// orthonormalisation and Rayleigh-Ritz steps then run per system.  Each system's
// arithmetic, and its order, is that of a single pass (the cell body is shared with the
// per-colour kernel), so the results are bit-identical to passes run one system at a time;
// the gain is fewer, fuller launches for small systems.
#include "internal.h"
#include "cell_fp64.cuh"

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <string>
#include <vector>



namespace dftfe {

namespace bt {
struct SysStep {
  const double* Hc;
  const int32_t* map;
  const double* X;
  const double* Xp;
  double* Z;
  int64_t ldx, ldp, ldz, M;
  int nc, ncol, active;
  int cplx;                // real view of a complex block: the init is the k-point kernel's
  double alpha, s1, s2;
};
}  // namespace bt

}  // namespace dftfe

struct dftfe_batch_s {
  std::vector<dftfe_ham> hams;
  cudaStream_t stream = nullptr;
  int ncolours = 0;                         // most colours of any system
  std::vector<int64_t> work_off;            // per colour: range in the work list
  int32_t* d_wsys = nullptr;                // work list: system of each item
  int32_t* d_wcell = nullptr;               // work list: cell of each item
  int nc_max = 0;
  void* d_steps = nullptr;                  // per-step system descriptors
  size_t steps_bytes = 0;
  std::vector<dftfe::bt::SysStep> host_steps;   // their host copy (kept until the next pass)
  // descriptors of the batched split-precision filter (device buffer and its host staging)
  dftfe::DevBuf mixed_desc;
  std::vector<uint8_t> mixed_host;
  // autotuner of the split-precision cell-product launches (dftfe_batch_autotune)
  bool autotune = false;
  std::map<std::string, dftfe::MixedShape> tuned;
  // workspace of the per-system pass tails (CholGS, Rayleigh-Ritz, residuals), which run one
  // system after another on the batch's stream: shared by every ham of the batch during its
  // tail, sized by the largest, freed with the batch
  std::map<std::string, dftfe::DevBuf> tail_ws;
  // CUDA graph of the filter phase (dftfe_batch_use_graphs)
  bool use_graphs = false;
  std::map<std::string, dftfe::GraphSlot> graphs;
  cudaStream_t capture_stream = nullptr;
};

namespace dftfe {

// Z = s1 X + s2 Xp for every active system (blockIdx.y = system); the same operations in the
// same order as the single-system k_axpby_init
__global__ void k_batch_axpby(const bt::SysStep* __restrict__ st) {
  const bt::SysStep& d = st[blockIdx.y];
  if (!d.active || d.cplx) return;
  const int64_t n = d.M * d.ncol;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / d.ncol;
    const int j = (int)(t - i * d.ncol);
    double v = 0.0;
    if (d.s1 != 0.0) v = d.s1 * d.X[i * d.ldx + j];
    if (d.Xp) v += d.s2 * d.Xp[i * d.ldp + j];
    d.Z[i * d.ldz + j] = v;
  }
}

// one CTA per (work item of this colour, 32-column tile, range of 64-row groups)
__global__ void __launch_bounds__(256, 2) k_batch_cell(const bt::SysStep* __restrict__ st,
                                                       const int32_t* __restrict__ wsys,
                                                       const int32_t* __restrict__ wcell, int rows_per_split) {
  extern __shared__ double smem[];
  const bt::SysStep& d = st[wsys[blockIdx.x]];
  const int rbeg = (int)blockIdx.z * rows_per_split;
  if (!d.active || (int)blockIdx.y * 32 >= d.ncol || rbeg >= d.nc) return;
  cell_fp64_wide_body(d.Hc, d.map, wcell[blockIdx.x], d.nc, d.X, d.ldx, d.Z, d.ldz, d.ncol, d.alpha,
                      (int)blockIdx.y, rbeg, min(d.nc, rbeg + rows_per_split), smem);
}

// Chebyshev coefficients of step k (1-based) for bounds b, as the single-system filter forms
// them; sigma carries the scaled recurrence's state
static void cheb_coef(const dftfe_bounds& b, int k, double& sigma, double& alpha, double& s1, double& s2) {
  const double e = (b.b - b.a) / 2.0, c = (b.b + b.a) / 2.0;
  const bool scaled = !std::isnan(b.a0);
  s2 = 0.0;
  if (k == 1) {
    sigma = scaled ? e / (b.a0 - c) : 0.0;
    alpha = scaled ? sigma / e : 1.0 / e;
    s1 = -c * alpha;
  } else if (scaled) {
    const double sigma1 = e / (b.a0 - c), gamma = 2.0 / sigma1;
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
}

// One round = block j of every system.  The descriptors of every round and step are formed
// on the host and uploaded before any launch, so the launches of the whole filter phase need
// no host work in between and can be captured as one CUDA graph.
struct RoundPlan {
  std::vector<int> nb;                       // real columns of block j (0: none / alone)
  std::vector<int> alone;                    // blocks of at most 4 real columns: single filter
  std::vector<int> cur;                      // buffer holding the result after the last step
  std::vector<std::array<double*, 3>> buf;
  std::vector<std::array<int64_t, 3>> lds;
  int maxtiles = 0;
  int64_t maxwork = 0;
};

static void batch_filter(dftfe_batch bt, dftfe_batch_item* items) {
  const int ns = (int)bt->hams.size();
  int rounds = 0, maxdeg = 0;
  for (int s = 0; s < ns; ++s) {
    rounds = std::max(rounds, (items[s].ncol + items[s].block - 1) / items[s].block);
    maxdeg = std::max(maxdeg, items[s].degree);
  }
  const size_t per_round = (size_t)std::max(maxdeg, 1) * ns;
  const size_t need = sizeof(bt::SysStep) * per_round * std::max(rounds, 1);
  if (need > bt->steps_bytes) {
    if (bt->d_steps) DFTFE_CHECK_CUDA(cudaFree(bt->d_steps));
    bt->d_steps = nullptr;
    DFTFE_CHECK_CUDA(cudaMalloc(&bt->d_steps, need));
    bt->steps_bytes = need;
  }
  bt::SysStep* dsteps = (bt::SysStep*)bt->d_steps;
  const size_t sh = (size_t)bt->nc_max * 32 * sizeof(double) + bt->nc_max * sizeof(int32_t);
  DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_batch_cell, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
  // the two recurrence workspaces of each system, at the size of its widest block (all
  // rounds' descriptors point into them, so they must not be reallocated between rounds)
  std::vector<double*> w1(ns, nullptr), w2(ns, nullptr);
  for (int s = 0; s < ns; ++s) {
    const int cw = items[s].kpoint ? 2 : 1;
    const int widest = cw * std::min(items[s].block, items[s].ncol);
    if (widest <= 4 || items[s].degree <= 0) continue;
    dftfe_ham h = bt->hams[s];
    w1[s] = (double*)ws_get(h, "cheb_w1", sizeof(double) * h->mesh->M * (size_t)widest);
    w2[s] = (double*)ws_get(h, "cheb_w2", sizeof(double) * h->mesh->M * (size_t)widest);
  }
  bt->host_steps.assign(per_round * std::max(rounds, 1), bt::SysStep{});
  std::vector<RoundPlan> plan(rounds);
  for (int j = 0; j < rounds; ++j) {
    RoundPlan& r = plan[j];
    r.nb.assign(ns, 0);
    r.cur.assign(ns, 0);
    r.buf.resize(ns);
    r.lds.resize(ns);
    std::vector<int> prev(ns, -1);
    for (int s = 0; s < ns; ++s) {
      // a complex block is handled through its real view: 2 doubles per complex column
      const int cw = items[s].kpoint ? 2 : 1;
      int nb = cw * std::min(items[s].block, items[s].ncol - j * items[s].block);
      if (nb <= 0 || items[s].degree <= 0) continue;
      if (nb <= 4) {
        r.alone.push_back(s);
        continue;
      }
      r.nb[s] = nb;
      r.buf[s] = {items[s].X + (int64_t)cw * j * items[s].block, w1[s], w2[s]};
      r.lds[s] = {cw * items[s].ld, nb, nb};
      r.maxtiles = std::max(r.maxtiles, (nb + 31) / 32);
      r.maxwork = std::max<int64_t>(r.maxwork, bt->hams[s]->mesh->M * nb);
    }
    std::vector<double> sigma(ns, 0.0);
    for (int k = 1; k <= maxdeg; ++k)
      for (int s = 0; s < ns; ++s) {
        bt::SysStep& d = bt->host_steps[(size_t)j * per_round + (size_t)(k - 1) * ns + s];
        if (r.nb[s] == 0 || k > items[s].degree) continue;
        dftfe_ham h = bt->hams[s];
        int out = 0;
        while (out == r.cur[s] || out == prev[s]) ++out;
        double alpha, s1, s2;
        cheb_coef(items[s].bounds, k, sigma[s], alpha, s1, s2);
        d.Hc = loc(h)->d_Hc;
        d.map = h->d_map;
        d.X = r.buf[s][r.cur[s]];
        d.ldx = r.lds[s][r.cur[s]];
        d.Xp = prev[s] >= 0 ? r.buf[s][prev[s]] : nullptr;
        d.ldp = prev[s] >= 0 ? r.lds[s][prev[s]] : 0;
        d.Z = r.buf[s][out];
        d.ldz = r.lds[s][out];
        d.M = h->mesh->M;
        d.nc = h->mesh->nc;
        d.ncol = r.nb[s];
        d.active = 1;
        d.cplx = items[s].kpoint ? 1 : 0;
        d.alpha = alpha;
        d.s1 = s1;
        d.s2 = s2;
        prev[s] = r.cur[s];
        r.cur[s] = out;
      }
  }
  // from pageable memory: the call returns once the data is staged, so the host descriptors
  // may be rewritten by the next pass
  DFTFE_CHECK_CUDA(cudaMemcpyAsync(dsteps, bt->host_steps.data(), sizeof(bt::SysStep) * bt->host_steps.size(),
                                   cudaMemcpyHostToDevice, bt->stream));

  auto enqueue = [&]() {
    for (int j = 0; j < rounds; ++j) {
      const RoundPlan& r = plan[j];
      for (int k = 1; k <= maxdeg; ++k) {
        const size_t off = (size_t)j * per_round + (size_t)(k - 1) * ns;
        const bt::SysStep* dk = dsteps + off;
        if (r.maxwork > 0) {
          const unsigned gx = (unsigned)std::min<int64_t>((r.maxwork + 255) / 256, 4096);
          DFTFE_LAUNCH(k_batch_axpby, dim3(std::max(gx, 1u), (unsigned)ns), 256, 0, bt->stream, dk);
        }
        for (int s = 0; s < ns; ++s) {
          const bt::SysStep& d = bt->host_steps[off + s];
          if (!d.active) continue;
          if (d.cplx)      // the recurrence terms, 1/2|k|^2, -i k.grad and the phased projectors
            kpoint_init_terms(bt->hams[s], d.X, d.ldx / 2, d.Xp, d.ldp / 2, d.Z, d.ldz / 2, d.ncol / 2, d.alpha,
                              d.s1, d.s2);
          else
            nonlocal_add_fp64(bt->hams[s], d.X, d.ldx, d.Z, d.ldz, d.ncol, d.alpha);
        }
        for (int c = 0; c < bt->ncolours; ++c) {
          const int64_t n = bt->work_off[c + 1] - bt->work_off[c];
          if (n == 0 || r.maxtiles == 0) continue;
          ProfScope ps(bt->hams[0], "batch_cell");
          const int splits = fp64_row_splits(bt->hams[0], n * r.maxtiles, bt->nc_max);
          const int rows = ((bt->nc_max + splits - 1) / splits + 63) / 64 * 64;
          DFTFE_LAUNCH(k_batch_cell, dim3((unsigned)n, (unsigned)r.maxtiles, (unsigned)((bt->nc_max + rows - 1) / rows)),
                       256, sh, bt->stream, dk, bt->d_wsys + bt->work_off[c], bt->d_wcell + bt->work_off[c], rows);
        }
      }
      for (int s = 0; s < ns; ++s)
        if (r.nb[s] > 0 && r.cur[s] != 0)
          copy_block(bt->stream, r.buf[s][r.cur[s]], r.lds[s][r.cur[s]], r.buf[s][0], r.lds[s][0],
                     bt->hams[s]->mesh->M, r.nb[s]);
      for (int s : r.alone) {
        const int n = std::min(items[s].block, items[s].ncol - j * items[s].block);
        if (items[s].kpoint)
          chebyshev_filter_z_fp64(bt->hams[s], items[s].X + 2 * (int64_t)j * items[s].block, items[s].ld, n,
                                  items[s].degree, items[s].bounds);
        else
          chebyshev_filter(bt->hams[s], items[s].X + (int64_t)j * items[s].block, items[s].ld, n, items[s].degree,
                           items[s].bounds);
      }
    }
  };
  if (!bt->use_graphs) {
    enqueue();
    return;
  }
  std::string key = "batch";
  for (int s = 0; s < ns; ++s)
    key += "/" + std::to_string(items[s].ncol) + "," + std::to_string(items[s].block) + "," +
           std::to_string(items[s].degree) + "," + std::to_string(items[s].kpoint);
  GraphSlot& slot = bt->graphs[key];
  if (!slot.warm) {
    enqueue();
    slot.warm = true;
    return;
  }
  if (!bt->capture_stream) DFTFE_CHECK_CUDA(cudaStreamCreateWithFlags(&bt->capture_stream, cudaStreamNonBlocking));
  std::vector<cudaStream_t*> streams = {&bt->stream};
  std::vector<bool*> prof;
  for (auto h : bt->hams) {
    streams.push_back(&h->stream);
    prof.push_back(&h->profiling);
  }
  capture_and_launch(slot, bt->stream, bt->capture_stream, streams, prof, enqueue);
}

// The split-precision (TF32x3) filter phase of a batched pass: rounds j = block j of every
// system, each round's cell products in one persistent launch per step and degree group over
// all systems' cells (plan_mixed_batch); optionally one CUDA graph for the whole phase.
static void batch_filter_mixed(dftfe_batch bt, dftfe_batch_item* items, int* err) {
  const int ns = (int)bt->hams.size();
  int rounds = 0;
  for (int s = 0; s < ns; ++s) rounds = std::max(rounds, (items[s].ncol + items[s].block - 1) / items[s].block);
  std::vector<std::vector<MixedBlock>> plan(rounds);
  for (int j = 0; j < rounds; ++j)
    for (int s = 0; s < ns; ++s) {
      const int cw = items[s].kpoint ? 2 : 1;
      const int nb = std::min(items[s].block, items[s].ncol - j * items[s].block);
      if (nb <= 0 || items[s].degree <= 0) continue;
      plan[j].push_back(MixedBlock{bt->hams[s], items[s].X + (int64_t)cw * j * items[s].block, cw * items[s].ld,
                                   cw * nb, items[s].degree, items[s].bounds, items[s].kpoint != 0});
    }
  auto enqueue = plan_mixed_batch(plan, bt->stream, err, bt->mixed_desc, bt->mixed_host,
                                  bt->autotune ? &bt->tuned : nullptr);
  if (!bt->use_graphs) {
    enqueue();
    return;
  }
  std::string key = "batch_tf32x3";
  for (int s = 0; s < ns; ++s)
    key += "/" + std::to_string(items[s].ncol) + "," + std::to_string(items[s].block) + "," +
           std::to_string(items[s].degree) + "," + std::to_string(items[s].kpoint);
  GraphSlot& slot = bt->graphs[key];
  if (!slot.warm) {
    enqueue();
    slot.warm = true;
    return;
  }
  if (!bt->capture_stream) DFTFE_CHECK_CUDA(cudaStreamCreateWithFlags(&bt->capture_stream, cudaStreamNonBlocking));
  std::vector<cudaStream_t*> streams = {&bt->stream};
  std::vector<bool*> prof;
  for (auto h : bt->hams) {
    streams.push_back(&h->stream);
    prof.push_back(&h->profiling);
  }
  capture_and_launch(slot, bt->stream, bt->capture_stream, streams, prof, enqueue);
}

}  // namespace dftfe

using namespace dftfe;

extern "C" dftfe_status dftfe_batch_create(const dftfe_ham* hams, int nsys, dftfe_batch* out) {
  ABI_BEGIN
  DFTFE_REQUIRE(hams && out && nsys >= 1 && nsys <= 4096, "need 1..4096 Hamiltonians");
  cudaStream_t s = hams[0] ? hams[0]->stream : nullptr;
  for (int i = 0; i < nsys; ++i) {
    DFTFE_REQUIRE(hams[i], "null Hamiltonian");
    DFTFE_REQUIRE(hams[i]->stream == s, "all Hamiltonians of a batch must use one stream");
    for (int j = 0; j < i; ++j) DFTFE_REQUIRE(hams[j] != hams[i], "a Hamiltonian appears twice");
  }
  auto* b = new dftfe_batch_s();
  try {
    b->hams.assign(hams, hams + nsys);
    b->stream = s;
    for (auto h : b->hams) {
      b->ncolours = std::max(b->ncolours, h->ncolours);
      b->nc_max = std::max(b->nc_max, h->mesh->nc);
    }
    // work list: colour by colour, the cells of every system with that colour
    std::vector<int32_t> wsys, wcell;
    b->work_off.assign(1, 0);
    std::vector<std::vector<int32_t>> cells(nsys);
    for (int i = 0; i < nsys; ++i) {
      auto h = b->hams[i];
      cells[i].resize(h->colour_off.back());
      if (!cells[i].empty())
        DFTFE_CHECK_CUDA(cudaMemcpy(cells[i].data(), h->d_colour_cells, sizeof(int32_t) * cells[i].size(),
                                    cudaMemcpyDeviceToHost));
    }
    for (int c = 0; c < b->ncolours; ++c) {
      for (int i = 0; i < nsys; ++i) {
        auto h = b->hams[i];
        if (c >= h->ncolours) continue;
        for (int64_t t = h->colour_off[c]; t < h->colour_off[c + 1]; ++t) {
          wsys.push_back(i);
          wcell.push_back(cells[i][t]);
        }
      }
      b->work_off.push_back((int64_t)wsys.size());
    }
    DFTFE_CHECK_CUDA(cudaMalloc(&b->d_wsys, sizeof(int32_t) * std::max<size_t>(wsys.size(), 1)));
    DFTFE_CHECK_CUDA(cudaMalloc(&b->d_wcell, sizeof(int32_t) * std::max<size_t>(wcell.size(), 1)));
    if (!wsys.empty()) {
      DFTFE_CHECK_CUDA(cudaMemcpy(b->d_wsys, wsys.data(), sizeof(int32_t) * wsys.size(), cudaMemcpyHostToDevice));
      DFTFE_CHECK_CUDA(cudaMemcpy(b->d_wcell, wcell.data(), sizeof(int32_t) * wcell.size(), cudaMemcpyHostToDevice));
    }
  } catch (...) {
    cudaFree(b->d_wsys);
    cudaFree(b->d_wcell);
    delete b;
    throw;
  }
  *out = b;
  ABI_END
}

extern "C" dftfe_status dftfe_batch_destroy(dftfe_batch b) {
  ABI_BEGIN
  if (!b) return DFTFE_OK;
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(b->stream));
  cudaFree(b->d_wsys);
  cudaFree(b->d_wcell);
  cudaFree(b->d_steps);
  for (auto& kv : b->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  for (auto& kv : b->tail_ws) kv.second.release();
  delete b;
  ABI_END
}

extern "C" dftfe_status dftfe_batch_chfsi_pass(dftfe_batch b, dftfe_batch_item* items, dftfe_precision prec) {
  ABI_BEGIN
  DFTFE_REQUIRE(b && items, "null argument");
  DFTFE_REQUIRE(prec == DFTFE_FP64 || prec == DFTFE_MIXED_TF32X3, "batched passes are FP64 or TF32x3");
  const int ns = (int)b->hams.size();
  for (int s = 0; s < ns; ++s) {
    const dftfe_batch_item& it = items[s];
    dftfe_ham h = b->hams[s];
    DFTFE_REQUIRE(it.X && it.evals && it.resid, "null array in a batch item");
    DFTFE_REQUIRE(it.kpoint == 0 || it.kpoint == 1, "kpoint must be 0 or 1");
    DFTFE_REQUIRE(it.ncol >= 1 && it.ncol <= (it.kpoint ? 1024 : 2048) && it.ld >= it.ncol && it.block >= 1 &&
                      it.degree >= 0,
                  "bad sizes in a batch item");
    if (it.kpoint) require_kpoint(h);
    DFTFE_REQUIRE(it.ncol <= h->mesh->M, "more columns than DoFs");
    DFTFE_REQUIRE(it.bounds.b > it.bounds.a, "need b > a");
    DFTFE_REQUIRE(std::isnan(it.bounds.a0) || it.bounds.a0 < it.bounds.a, "need a0 < a for the scaled filter");
    if (!loc(h)->has_potential) throw Error(DFTFE_ERR_STATE, "set the potential first");
  }
  {
    ProfScope ps(b->hams[0], "batch_filter");
    if (prec == DFTFE_FP64) {
      batch_filter(b, items);
    } else {
      int* err = (int*)ws_get(b->hams[0], "mx_err_batch", sizeof(int));
      DFTFE_CHECK_CUDA(cudaMemsetAsync(err, 0, sizeof(int), b->stream));
      batch_filter_mixed(b, items, err);
      int herr = 0;
      DFTFE_CHECK_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
      DFTFE_CHECK_CUDA(cudaStreamSynchronize(b->stream));
      if (herr) throw Error(DFTFE_ERR_TIMEOUT, "batched mixed cell kernel: a bounded wait timed out");
    }
  }
  for (int s = 0; s < ns; ++s) {
    dftfe_ham h = b->hams[s];
    struct TailWs {         // the batch's shared tail workspace while this system's tail runs
      dftfe_ham h;
      TailWs(dftfe_ham h_, std::map<std::string, DevBuf>* w) : h(h_) { h->tail_ws = w; }
      ~TailWs() { h->tail_ws = nullptr; }
    } guard(h, &b->tail_ws);
    if (items[s].kpoint)
      chfsi_pass_tail_z(h, items[s].X, items[s].ld, items[s].ncol, &items[s].bounds, items[s].evals,
                        items[s].resid, prec);
    else
      chfsi_pass_tail(h, items[s].X, items[s].ld, items[s].ncol, &items[s].bounds, items[s].evals,
                      items[s].resid, prec);
  }
  ABI_END
}

extern "C" dftfe_status dftfe_batch_autotune(dftfe_batch b, int enable) {
  ABI_BEGIN
  DFTFE_REQUIRE(b, "null batch");
  DFTFE_REQUIRE(enable == 0 || enable == 1, "enable must be 0 or 1");
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(b->stream));
  b->autotune = enable == 1;
  b->tuned.clear();
  for (auto& kv : b->graphs) kv.second.warm = false;   // cached graphs hold the old shapes
  ABI_END
}

extern "C" dftfe_status dftfe_batch_autotune_query(dftfe_batch b, int index, int* nodes_per_cell, int* work_items,
                                                   int* atmem, int* deep, int* deal, int* order, double* best_ms,
                                                   double* default_ms) {
  ABI_BEGIN
  DFTFE_REQUIRE(b && nodes_per_cell && work_items && atmem && deep && deal && order, "null argument");
  DFTFE_REQUIRE(index >= 0, "index must be >= 0");
  if (index >= (int)b->tuned.size()) {
    *nodes_per_cell = *work_items = *atmem = *deep = *deal = *order = -1;
    if (best_ms) *best_ms = 0.0;
    if (default_ms) *default_ms = 0.0;
    return DFTFE_OK;
  }
  auto it = b->tuned.begin();
  std::advance(it, index);
  *nodes_per_cell = std::atoi(it->first.c_str());
  *work_items = std::atoi(it->first.c_str() + it->first.find('/') + 1);
  *atmem = it->second.atmem;
  *deep = it->second.deep;
  *deal = it->second.deal;
  *order = it->second.order;
  if (best_ms) *best_ms = it->second.best_ms;
  if (default_ms) *default_ms = it->second.default_ms;
  ABI_END
}

extern "C" dftfe_status dftfe_batch_use_graphs(dftfe_batch b, int enable) {
  ABI_BEGIN
  DFTFE_REQUIRE(b, "null batch");
  DFTFE_REQUIRE(enable == 0 || enable == 1, "enable must be 0 or 1");
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(b->stream));
  for (auto& kv : b->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  b->graphs.clear();
  b->use_graphs = enable == 1;
  ABI_END
}

extern "C" dftfe_status dftfe_batch_graph_query(dftfe_batch b, int64_t* replays, int64_t* instantiations) {
  ABI_BEGIN
  DFTFE_REQUIRE(b && replays && instantiations, "null argument");
  int64_t r = 0, n = 0;
  for (auto& kv : b->graphs) {
    r += kv.second.replays;
    n += kv.second.reinstantiations;
  }
  *replays = r;
  *instantiations = n;
  ABI_END
}
