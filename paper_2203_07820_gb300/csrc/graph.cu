// CUDA graphs of the pass's filter phase (no counterpart in the paper).  A Chebyshev filter is
// degree x (recurrence init + nonlocal + one cell launch per colour) short launches; for small
// systems the gaps between them cost as much as the kernels.  With graphs on, the region is
// captured from the ham's stream on every call (capture records launches without submitting
// them) and applied to the cached executable with cudaGraphExecUpdate: the topology of a
// filter depends only on its shapes (the slot key), while bounds, and so the recurrence
// coefficients, change every pass and only change kernel arguments.  The first call with a
// key runs directly, so every workspace exists before any capture (capture cannot allocate).
// Capture runs on a private stream (the ham's own may be the legacy default stream, which
// cannot be captured): the region is enqueued with the ham's stream temporarily set to it,
// and the graph is launched on the ham's stream, so it is ordered with everything before.
#include "internal.h"

namespace dftfe {

// The capture itself, shared by single hams and batches: every stream variable in `streams`
// (all holding the stream `own`) points at `cap` while `enqueue` runs, and every profiling
// flag in `prof` is cleared (per-kernel timers would record events inside the graph; the
// caller times the region as a whole).
void capture_and_launch(GraphSlot& slot, cudaStream_t own, cudaStream_t cap, const std::vector<cudaStream_t*>& streams,
                        const std::vector<bool*>& prof, const std::function<void()>& enqueue) {
  std::vector<bool> saved;
  for (bool* f : prof) saved.push_back(*f);
  auto restore = [&]() {
    for (auto* sp : streams) *sp = own;
    for (size_t i = 0; i < prof.size(); ++i) *prof[i] = saved[i];
  };
  cudaGraph_t g = nullptr;
  DFTFE_CHECK_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  for (auto* sp : streams) *sp = cap;
  for (bool* f : prof) *f = false;
  try {
    enqueue();
  } catch (...) {
    restore();
    cudaStreamEndCapture(cap, &g);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    throw;
  }
  restore();
  DFTFE_CHECK_CUDA(cudaStreamEndCapture(cap, &g));
  if (slot.exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(slot.exec, g, &info) != cudaSuccess) {
      cudaGetLastError();   // clear the update failure: the graph is instantiated afresh
      cudaGraphExecDestroy(slot.exec);
      slot.exec = nullptr;
    }
  }
  if (!slot.exec) {
    const cudaError_t e = cudaGraphInstantiate(&slot.exec, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      slot.exec = nullptr;
      throw Error(DFTFE_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    ++slot.reinstantiations;
  }
  cudaGraphDestroy(g);
  DFTFE_CHECK_CUDA(cudaGraphLaunch(slot.exec, own));
  ++slot.replays;
}

void run_region(dftfe_ham h, const std::string& key, const std::function<void()>& enqueue) {
  if (!h->use_graphs) {
    enqueue();
    return;
  }
  GraphSlot& slot = h->graphs[key];
  if (!slot.warm) {
    enqueue();
    slot.warm = true;
    return;
  }
  if (!h->capture_stream) DFTFE_CHECK_CUDA(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
  capture_and_launch(slot, h->stream, h->capture_stream, {&h->stream}, {&h->profiling}, enqueue);
}

void free_graphs(dftfe_ham h) {
  for (auto& kv : h->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  h->graphs.clear();
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  h->capture_stream = nullptr;
}

}  // namespace dftfe

using namespace dftfe;

extern "C" dftfe_status dftfe_ham_use_graphs(dftfe_ham h, int enable) {
  ABI_BEGIN
  DFTFE_REQUIRE(h, "null ham");
  DFTFE_REQUIRE(enable == 0 || enable == 1, "enable must be 0 or 1");
  DFTFE_CHECK_CUDA(cudaStreamSynchronize(h->stream));
  free_graphs(h);
  h->use_graphs = enable == 1;
  ABI_END
}

extern "C" dftfe_status dftfe_graph_query(dftfe_ham h, int64_t* replays, int64_t* instantiations) {
  ABI_BEGIN
  DFTFE_REQUIRE(h && replays && instantiations, "null argument");
  int64_t r = 0, n = 0;
  for (auto& kv : h->graphs) {
    r += kv.second.replays;
    n += kv.second.reinstantiations;
  }
  *replays = r;
  *instantiations = n;
  ABI_END
}
