// The learned degree/bounds proposer's network on the GPU (FP32): a three-layer perceptron
// x -> tanh(W1 x + b1) -> tanh(W2 h1 + b2) -> W3 h2 + b3, its weighted mean-squared loss
// with the gradient by the chain rule (training), and Adam.  Parameters are one packed
// vector: W1 (n_h x n_in, row-major), b1, W2 (n_h x n_h), b2, W3 (n_out x n_h), b3.
//
// Kernels: one CTA of n_h threads (thread j = hidden unit j) walks a contiguous range of
// samples with the parameters in shared memory.  In the backward pass thread j owns row j of
// W1 and W2, column j of W3 and b1[j], b2[j] (threads < n_out also b3), so the per-CTA
// gradient sums in shared memory need no atomics; a second kernel adds the CTA partials in a
// fixed order, so the gradient is deterministic.
#include "internal.h"

#include <cmath>

namespace dftfe {

namespace nn {

constexpr int kMaxIn = 64, kMaxHidden = 128, kMaxOut = 8;

struct Shape {
  int nin, nh, nout;
  __host__ __device__ int64_t count() const {
    return (int64_t)nh * nin + nh + (int64_t)nh * nh + nh + (int64_t)nout * nh + nout;
  }
  __host__ __device__ int64_t oW1() const { return 0; }
  __host__ __device__ int64_t ob1() const { return (int64_t)nh * nin; }
  __host__ __device__ int64_t oW2() const { return ob1() + nh; }
  __host__ __device__ int64_t ob2() const { return oW2() + (int64_t)nh * nh; }
  __host__ __device__ int64_t oW3() const { return ob2() + nh; }
  __host__ __device__ int64_t ob3() const { return oW3() + (int64_t)nout * nh; }
};

// forward of one sample held in xs (shared); leaves h1, h2 (shared) and y (shared)
__device__ __forceinline__ void fwd_sample(const Shape& s, const float* P, const float* xs, float* h1, float* h2,
                                           float* y) {
  const int j = threadIdx.x;
  float z = P[s.ob1() + j];
  const float* w1 = P + s.oW1() + (int64_t)j * s.nin;
  for (int i = 0; i < s.nin; ++i) z = fmaf(w1[i], xs[i], z);
  h1[j] = tanhf(z);
  __syncthreads();
  z = P[s.ob2() + j];
  const float* w2 = P + s.oW2() + (int64_t)j * s.nh;
  for (int i = 0; i < s.nh; ++i) z = fmaf(w2[i], h1[i], z);
  h2[j] = tanhf(z);
  __syncthreads();
  if (j < s.nout) {
    float o = P[s.ob3() + j];
    const float* w3 = P + s.oW3() + (int64_t)j * s.nh;
    for (int i = 0; i < s.nh; ++i) o = fmaf(w3[i], h2[i], o);
    y[j] = o;
  }
  __syncthreads();
}

}  // namespace nn

__global__ void k_mlp_forward(const float* __restrict__ params, nn::Shape s, const float* __restrict__ X,
                              int64_t n, int64_t per_cta, float* __restrict__ Y) {
  extern __shared__ float nsm[];
  const int64_t P = s.count();
  float* Ps = nsm;
  float* xs = Ps + P;
  float* h1 = xs + nn::kMaxIn;
  float* h2 = h1 + nn::kMaxHidden;
  float* y = h2 + nn::kMaxHidden;
  for (int64_t i = threadIdx.x; i < P; i += blockDim.x) Ps[i] = params[i];
  __syncthreads();
  const int64_t r0 = blockIdx.x * per_cta, r1 = min(n, r0 + per_cta);
  for (int64_t r = r0; r < r1; ++r) {
    for (int i = threadIdx.x; i < s.nin; i += blockDim.x) xs[i] = X[r * s.nin + i];
    __syncthreads();
    nn::fwd_sample(s, Ps, xs, h1, h2, y);
    if (threadIdx.x < s.nout) Y[r * s.nout + threadIdx.x] = y[threadIdx.x];
    __syncthreads();
  }
}

// per-CTA partial gradient (P floats) and partial loss of L = (1/n) sum w_k (y - t)^2
__global__ void k_mlp_grad_partial(const float* __restrict__ params, nn::Shape s, const float* __restrict__ X,
                                   const float* __restrict__ T, const float* __restrict__ wk, int64_t n,
                                   int64_t per_cta, float* __restrict__ gpart, float* __restrict__ lpart) {
  extern __shared__ float nsm[];
  const int64_t P = s.count();
  float* Ps = nsm;
  float* G = Ps + P;
  float* xs = G + P;
  float* h1 = xs + nn::kMaxIn;
  float* h2 = h1 + nn::kMaxHidden;
  float* y = h2 + nn::kMaxHidden;
  float* dy = y + nn::kMaxOut;
  float* dz2 = dy + nn::kMaxOut;
  const int j = threadIdx.x;
  for (int64_t i = j; i < P; i += blockDim.x) {
    Ps[i] = params[i];
    G[i] = 0.0f;
  }
  __syncthreads();
  const float inv_n = 1.0f / (float)n;
  float lacc = 0.0f;
  const int64_t r0 = blockIdx.x * per_cta, r1 = min(n, r0 + per_cta);
  for (int64_t r = r0; r < r1; ++r) {
    for (int i = j; i < s.nin; i += blockDim.x) xs[i] = X[r * s.nin + i];
    __syncthreads();
    nn::fwd_sample(s, Ps, xs, h1, h2, y);
    if (j < s.nout) {
      const float e = y[j] - T[r * s.nout + j];
      const float w = wk ? wk[j] : 1.0f;
      lacc = fmaf(w * e, e * inv_n, lacc);
      dy[j] = 2.0f * w * e * inv_n;
      G[s.ob3() + j] += dy[j];
    }
    __syncthreads();
    // layer 3 and the second hidden layer
    float dh2 = 0.0f;
    for (int k = 0; k < s.nout; ++k) {
      G[s.oW3() + (int64_t)k * s.nh + j] += dy[k] * h2[j];
      dh2 = fmaf(Ps[s.oW3() + (int64_t)k * s.nh + j], dy[k], dh2);
    }
    const float z2 = dh2 * (1.0f - h2[j] * h2[j]);
    dz2[j] = z2;
    G[s.ob2() + j] += z2;
    float* gw2 = G + s.oW2() + (int64_t)j * s.nh;
    for (int i = 0; i < s.nh; ++i) gw2[i] = fmaf(z2, h1[i], gw2[i]);
    __syncthreads();
    // the first hidden layer
    float dh1 = 0.0f;
    for (int i = 0; i < s.nh; ++i) dh1 = fmaf(Ps[s.oW2() + (int64_t)i * s.nh + j], dz2[i], dh1);
    const float z1 = dh1 * (1.0f - h1[j] * h1[j]);
    G[s.ob1() + j] += z1;
    float* gw1 = G + s.oW1() + (int64_t)j * s.nin;
    for (int i = 0; i < s.nin; ++i) gw1[i] = fmaf(z1, xs[i], gw1[i]);
    __syncthreads();
  }
  for (int64_t i = j; i < P; i += blockDim.x) gpart[(int64_t)blockIdx.x * P + i] = G[i];
  // loss: threads < n_out hold partial sums
  __shared__ float lred[nn::kMaxOut];
  if (j < s.nout) lred[j] = lacc;
  __syncthreads();
  if (j == 0) {
    float t = 0.0f;
    for (int k = 0; k < s.nout; ++k) t += lred[k];
    lpart[blockIdx.x] = t;
  }
}

__global__ void k_mlp_grad_reduce(const float* __restrict__ gpart, const float* __restrict__ lpart, int nparts,
                                  int64_t P, float* __restrict__ grad, float* __restrict__ loss) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < P) {
    float g = 0.0f;
    for (int c = 0; c < nparts; ++c) g += gpart[(int64_t)c * P + i];
    grad[i] = g;
  }
  if (i == 0 && loss) {
    float l = 0.0f;
    for (int c = 0; c < nparts; ++c) l += lpart[c];
    *loss = l;
  }
}

// Adam (Kingma & Ba): m, v moving averages; c1 = 1/(1 - beta1^t), c2 = 1/(1 - beta2^t)
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t count, float lr, float beta1, float beta2, float eps, float c1,
                       float c2) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float mi = fmaf(beta1, m[i], (1.0f - beta1) * gi);
  const float vi = fmaf(beta2, v[i], (1.0f - beta2) * gi * gi);
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

static nn::Shape check_shape(int nin, int nh, int nout) {
  DFTFE_REQUIRE(nin >= 1 && nin <= nn::kMaxIn, "n_in must be in 1..64");
  DFTFE_REQUIRE(nh >= 32 && nh <= nn::kMaxHidden && nh % 32 == 0, "n_hidden must be 32, 64, 96 or 128");
  DFTFE_REQUIRE(nout >= 1 && nout <= nn::kMaxOut && nout <= nh, "n_out must be in 1..8");
  return nn::Shape{nin, nh, nout};
}

static int mlp_ctas(int64_t n) {
  int dev = 0, sms = 0;
  DFTFE_CHECK_CUDA(cudaGetDevice(&dev));
  DFTFE_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)2 * sms, (n + 15) / 16));
}

}  // namespace dftfe

using namespace dftfe;

extern "C" int64_t dftfe_mlp_param_count(int n_in, int n_hidden, int n_out) {
  if (n_in < 1 || n_hidden < 1 || n_out < 1) return -1;
  return nn::Shape{n_in, n_hidden, n_out}.count();
}

extern "C" dftfe_status dftfe_mlp_forward(const float* params, int n_in, int n_hidden, int n_out, const float* X,
                                          int64_t n, float* Y, void* stream) {
  ABI_BEGIN
  const nn::Shape s = check_shape(n_in, n_hidden, n_out);
  DFTFE_REQUIRE(params && (X || n == 0) && (Y || n == 0) && n >= 0, "null argument or negative n");
  if (n == 0) return DFTFE_OK;
  const int ctas = mlp_ctas(n);
  const int64_t per = (n + ctas - 1) / ctas;
  const size_t sh = sizeof(float) * ((size_t)s.count() + nn::kMaxIn + 2 * nn::kMaxHidden + nn::kMaxOut);
  if (sh > 48 * 1024)
    DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
  DFTFE_LAUNCH(k_mlp_forward, (unsigned)ctas, n_hidden, sh, (cudaStream_t)stream, params, s, X, n, per, Y);
  ABI_END
}

extern "C" dftfe_status dftfe_mlp_loss_grad(const float* params, int n_in, int n_hidden, int n_out, const float* X,
                                            const float* T, const float* w, int64_t n, float* loss, float* grad,
                                            void* stream) {
  ABI_BEGIN
  const nn::Shape s = check_shape(n_in, n_hidden, n_out);
  DFTFE_REQUIRE(params && X && T && grad && n >= 1, "null argument or empty batch");
  const int ctas = mlp_ctas(n);
  const int64_t per = (n + ctas - 1) / ctas;
  const int64_t P = s.count();
  float* gpart = nullptr;
  float* lpart = nullptr;
  // partials in a stream-ordered allocation (freed on the same stream)
  DFTFE_CHECK_CUDA(cudaMallocAsync(&gpart, sizeof(float) * (size_t)(ctas * P + ctas), (cudaStream_t)stream));
  lpart = gpart + (size_t)ctas * P;
  const size_t sh = sizeof(float) * ((size_t)2 * P + nn::kMaxIn + 2 * nn::kMaxHidden + 2 * nn::kMaxOut + nn::kMaxHidden);
  if (sh > 48 * 1024)
    DFTFE_CHECK_CUDA(cudaFuncSetAttribute(k_mlp_grad_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
  DFTFE_LAUNCH(k_mlp_grad_partial, (unsigned)ctas, n_hidden, sh, (cudaStream_t)stream, params, s, X, T, w, n, per,
               gpart, lpart);
  DFTFE_LAUNCH(k_mlp_grad_reduce, (unsigned)((P + 255) / 256), 256, 0, (cudaStream_t)stream, gpart, lpart, ctas, P,
               grad, loss);
  DFTFE_CHECK_CUDA(cudaFreeAsync(gpart, (cudaStream_t)stream));
  ABI_END
}

extern "C" dftfe_status dftfe_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t count, int t,
                                       float lr, float beta1, float beta2, float eps, void* stream) {
  ABI_BEGIN
  DFTFE_REQUIRE(params && grad && m && v && count >= 0 && t >= 1, "null argument, negative count or t < 1");
  DFTFE_REQUIRE(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && lr > 0.f && eps > 0.f, "bad hyper-parameters");
  if (count == 0) return DFTFE_OK;
  const double c1 = 1.0 / (1.0 - std::pow((double)beta1, t)), c2 = 1.0 / (1.0 - std::pow((double)beta2, t));
  DFTFE_LAUNCH(k_adam, (unsigned)((count + 255) / 256), 256, 0, (cudaStream_t)stream, params, grad, m, v, count, lr,
               beta1, beta2, eps, (float)c1, (float)c2);
  ABI_END
}
