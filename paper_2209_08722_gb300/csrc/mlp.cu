// A small multilayer perceptron for the learned warm start of the inner solve:
// in -> H -> H -> out with GELU after both hidden layers,
//     Z1 = W1 X + b1, A1 = gelu(Z1), Z2 = W2 A1 + b2, A2 = gelu(Z2), Y = W3 A2 + b3,
// trained by mean-squared error, L = 1/(2B) sum_b ||Y_b - T_b||^2, with Adam.
//
// Layout: a batch of B samples is a column-major (features x B) matrix, i.e.
// each sample is contiguous; weights are column-major (rows = outputs).  The
// three matrix products of a forward pass and the six of a backward pass run
// on the project's tcgen05 GEMM (mlp_gemm.cu: split-TF32 operands, FP32
// accumulation in tensor memory), single-sample prediction on its FP32 GEMV;
// the element-wise work is in this file's kernels: bias + GELU (keeping Z for
// the backward pass), the GELU derivative fused with the bias-gradient row
// sums, the loss and its gradient, and the Adam update.  GELU is the exact
// 0.5 z (1 + erf(z / sqrt 2)) with derivative Phi(z) + z phi(z).
#include "internal.h"

#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "../../include/lp_sketch_ipm.h"

namespace lpk {

namespace {

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float z) {
  const float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * z * z);
  return cdf + z * pdf;
}

// Z += b (per row), A = gelu(Z) (or A = Z for the output layer)
__global__ void k_bias_act(int rows, int cols, const float* __restrict__ b, float* __restrict__ z,
                           float* __restrict__ a, int act) {
  const long long total = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % rows);
    const float v = z[e] + b[r];
    z[e] = v;
    if (a) a[e] = act ? gelu(v) : v;
  }
}

// dZ = dA * gelu'(Z) in place (act) ; db[r] = sum_c dZ[r, c]   (one warp per row)
__global__ void k_act_back(int rows, int cols, const float* __restrict__ z, float* __restrict__ d,
                           float* __restrict__ db, int act) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = warp; r < rows; r += nw) {
    float s = 0.0f;
    for (int c = lane; c < cols; c += 32) {
      const size_t e = (size_t)c * rows + r;
      float g = d[e];
      if (act) {
        g *= gelu_grad(z[e]);
        d[e] = g;
      }
      s += g;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) db[r] = s;
  }
}

// y = sum of the GEMV's column-slice partials (in slice order) + b, then the
// activation (single-sample prediction)
__global__ void k_slices_bias_act(int rows, int slices, const float* __restrict__ part,
                                  const float* __restrict__ b, float* __restrict__ y, int act) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  float s = 0.0f;
  for (int q = 0; q < slices; ++q) s += part[(size_t)q * rows + r];
  const float v = s + b[r];
  y[r] = act ? gelu(v) : v;
}

// dY = (Y - T) / B; loss partial sums
__global__ void k_mse(long long total, int batch, const float* __restrict__ y, const float* __restrict__ t,
                      float* __restrict__ dy, double* __restrict__ loss) {
  __shared__ double red[32];
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const float r = y[e] - t[e];
    dy[e] = r / (float)batch;
    acc += (double)r * (double)r;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) atomicAdd(loss, acc / (2.0 * batch));
}

__global__ void k_adam(long long count, float* __restrict__ w, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.0f - b1) * gi;
    const float vi = b2 * v[e] + (1.0f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    w[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

int grid_for(long long count, int num_sms) {
  return (int)std::max<long long>(1, std::min<long long>((count + 255) / 256, (long long)num_sms * 8));
}

}  // namespace
}  // namespace lpk

using namespace lpk;

struct lp_mlp {
  int in = 0, hid = 0, out = 0;
  int num_sms = 1;
  cudaStream_t st = nullptr;
  int* err = nullptr;        // device status word of the GEMMs' bounded waits
  int* herr = nullptr;       // pinned host copy
  // parameters: W1 (hid x in), b1, W2 (hid x hid), b2, W3 (out x hid), b3, in one buffer
  float* param = nullptr;
  float* grad = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  long long nparam = 0;
  long long steps = 0;
  // activations for the current batch capacity
  int cap = 0;
  float *z1 = nullptr, *a1 = nullptr, *z2 = nullptr, *a2 = nullptr, *y = nullptr, *d3 = nullptr;
  float *d2 = nullptr, *d1 = nullptr;
  double* loss = nullptr;
  std::vector<void*> allocs;

  float* W1() { return param; }
  float* b1() { return W1() + (size_t)hid * in; }
  float* W2() { return b1() + hid; }
  float* b2() { return W2() + (size_t)hid * hid; }
  float* W3() { return b2() + hid; }
  float* b3() { return W3() + (size_t)out * hid; }
  float* g(float* p) { return grad + (p - param); }

  ~lp_mlp() {
    for (void* p : allocs) cudaFree(p);
    if (herr) cudaFreeHost(herr);
  }
  template <typename T>
  bool alloc(T** p, size_t count) {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return false;
    try {
      allocs.push_back(q);
    } catch (const std::bad_alloc&) {  // never throw out of a C ABI call
      cudaFree(q);
      return false;
    }
    *p = static_cast<T*>(q);
    return true;
  }
  bool ensure_batch(int B) {
    if (B <= cap) return true;
    if (!alloc(&z1, (size_t)hid * B) || !alloc(&a1, (size_t)hid * B) || !alloc(&z2, (size_t)hid * B) ||
        !alloc(&a2, (size_t)hid * B) || !alloc(&y, (size_t)out * B) || !alloc(&d3, (size_t)out * B) ||
        !alloc(&d2, (size_t)hid * B) || !alloc(&d1, (size_t)hid * B))
      return false;
    cap = B;
    return true;
  }
  // C = op(A) op(B) on the tensor cores (ta / tb: transpose A / B)
  bool gemm(bool ta, bool tb, int m, int n, int k, const float* A, int lda, const float* B, int ldb, float* C,
            int ldc) {
    return launch_gemm_tf32x3(ta, tb, m, n, k, A, lda, B, ldb, C, ldc, err, st) == cudaSuccess;
  }
  // the GEMMs' status word after the stream is done: LP_ERR_DEVICE_TIMEOUT
  // when a wait gave up (the word is cleared again)
  int status() {
    if (cudaMemcpyAsync(herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return LP_ERR_CUDA;
    if (*herr == ERR_NONE) return LP_OK;
    if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return LP_ERR_CUDA;
    return LP_ERR_DEVICE_TIMEOUT;
  }
  // Y (out x B) from X (in x B); activations kept for backward
  int forward(const float* X, int B) {
    if (!ensure_batch(B)) return LP_ERR_OOM;
    if (!gemm(false, false, hid, B, in, W1(), hid, X, in, z1, hid)) return LP_ERR_CUDA;
    k_bias_act<<<grid_for((long long)hid * B, num_sms), 256, 0, st>>>(hid, B, b1(), z1, a1, 1);
    if (!gemm(false, false, hid, B, hid, W2(), hid, a1, hid, z2, hid)) return LP_ERR_CUDA;
    k_bias_act<<<grid_for((long long)hid * B, num_sms), 256, 0, st>>>(hid, B, b2(), z2, a2, 1);
    if (!gemm(false, false, out, B, hid, W3(), out, a2, hid, y, out)) return LP_ERR_CUDA;
    k_bias_act<<<grid_for((long long)out * B, num_sms), 256, 0, st>>>(out, B, b3(), y, nullptr, 0);
    g_launches.fetch_add(3, std::memory_order_relaxed);
    return cudaGetLastError() == cudaSuccess ? LP_OK : LP_ERR_CUDA;
  }
  // gradients of the loss from dY (= d3, out x B) for the batch X
  int backward(const float* X, int B) {
    const int wg = std::max(1, std::min(num_sms * 4, (out + 7) / 8));
    k_act_back<<<wg, 256, 0, st>>>(out, B, y, d3, g(b3()), 0);
    if (!gemm(false, true, out, hid, B, d3, out, a2, hid, g(W3()), out)) return LP_ERR_CUDA;
    if (!gemm(true, false, hid, B, out, W3(), out, d3, out, d2, hid)) return LP_ERR_CUDA;
    const int hg = std::max(1, std::min(num_sms * 4, (hid + 7) / 8));
    k_act_back<<<hg, 256, 0, st>>>(hid, B, z2, d2, g(b2()), 1);
    if (!gemm(false, true, hid, hid, B, d2, hid, a1, hid, g(W2()), hid)) return LP_ERR_CUDA;
    if (!gemm(true, false, hid, B, hid, W2(), hid, d2, hid, d1, hid)) return LP_ERR_CUDA;
    k_act_back<<<hg, 256, 0, st>>>(hid, B, z1, d1, g(b1()), 1);
    if (!gemm(false, true, hid, in, B, d1, hid, X, in, g(W1()), hid)) return LP_ERR_CUDA;
    g_launches.fetch_add(3, std::memory_order_relaxed);
    return cudaGetLastError() == cudaSuccess ? LP_OK : LP_ERR_CUDA;
  }
};

extern "C" {

static int mlp_create_impl(lp_mlp** out, int32_t in, int32_t hidden, int32_t outdim, uint64_t seed,
                           void* stream) {
  std::unique_ptr<lp_mlp> M(new lp_mlp());  // freed on every early return
  M->in = in;
  M->hid = hidden;
  M->out = outdim;
  M->st = static_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&M->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    return LP_ERR_CUDA;
  }
  if (cudaMallocHost(&M->herr, sizeof(int)) != cudaSuccess) {
    M->herr = nullptr;
    return LP_ERR_OOM;
  }
  M->nparam = (long long)hidden * in + hidden + (long long)hidden * hidden + hidden + (long long)outdim * hidden + outdim;
  if (!M->alloc(&M->param, M->nparam) || !M->alloc(&M->grad, M->nparam) || !M->alloc(&M->adam_m, M->nparam) ||
      !M->alloc(&M->adam_v, M->nparam) || !M->alloc(&M->loss, 1) || !M->alloc(&M->err, 1)) {
    return LP_ERR_OOM;
  }
  // He-style initialisation from SplitMix64 (host), biases zero; the output
  // layer starts small so an untrained model predicts nearly zero
  std::vector<float> h((size_t)M->nparam, 0.0f);
  auto fill = [&](size_t off, int rows, int cols, double scale) {
    for (size_t e = 0; e < (size_t)rows * cols; ++e) {
      const uint64_t v1 = sm64_draw(seed, 2 * (off + e)), v2 = sm64_draw(seed, 2 * (off + e) + 1);
      const double u1 = ((double)(v1 >> 11) + 1.0) * 0x1p-53, u2 = (double)(v2 >> 11) * 0x1p-53;
      h[off + e] = (float)(scale * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
    }
  };
  const size_t o1 = 0, o2 = (size_t)hidden * in + hidden, o3 = o2 + (size_t)hidden * hidden + hidden;
  fill(o1, hidden, in, std::sqrt(2.0 / in));
  fill(o2, hidden, hidden, std::sqrt(2.0 / hidden));
  fill(o3, outdim, hidden, 0.01 * std::sqrt(1.0 / hidden));
  if (cudaMemcpy(M->param, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(M->adam_m, 0, sizeof(float) * M->nparam) != cudaSuccess ||
      cudaMemset(M->err, 0, sizeof(int)) != cudaSuccess ||
      cudaMemset(M->adam_v, 0, sizeof(float) * M->nparam) != cudaSuccess) {
    return LP_ERR_CUDA;
  }
  *out = M.release();
  return LP_OK;
}

// no C++ exception crosses the C ABI: a failed host allocation is LP_ERR_OOM
int lp_mlp_create(lp_mlp** out, int32_t in, int32_t hidden, int32_t outdim, uint64_t seed, void* stream) {
  if (!out || in <= 0 || hidden <= 0 || outdim <= 0) return LP_ERR_ARG;
  *out = nullptr;
  try {
    return mlp_create_impl(out, in, hidden, outdim, seed, stream);
  } catch (const std::bad_alloc&) {
    return LP_ERR_OOM;
  } catch (...) {
    return LP_ERR_ARG;
  }
}

int lp_mlp_destroy(lp_mlp* M) {
  delete M;
  return LP_OK;
}

int64_t lp_mlp_num_params(const lp_mlp* M) { return M ? M->nparam : -1; }

int lp_mlp_get_params(lp_mlp* M, float* host) {
  if (!M || !host) return LP_ERR_ARG;
  if (cudaStreamSynchronize(M->st) != cudaSuccess) return LP_ERR_CUDA;
  return cudaMemcpy(host, M->param, sizeof(float) * M->nparam, cudaMemcpyDeviceToHost) == cudaSuccess ? LP_OK
                                                                                                   : LP_ERR_CUDA;
}

int lp_mlp_set_params(lp_mlp* M, const float* host) {
  if (!M || !host) return LP_ERR_ARG;
  if (cudaStreamSynchronize(M->st) != cudaSuccess) return LP_ERR_CUDA;
  return cudaMemcpy(M->param, host, sizeof(float) * M->nparam, cudaMemcpyHostToDevice) == cudaSuccess ? LP_OK
                                                                                                   : LP_ERR_CUDA;
}

int lp_mlp_get_grads(lp_mlp* M, float* host) {
  if (!M || !host) return LP_ERR_ARG;
  if (cudaStreamSynchronize(M->st) != cudaSuccess) return LP_ERR_CUDA;
  return cudaMemcpy(host, M->grad, sizeof(float) * M->nparam, cudaMemcpyDeviceToHost) == cudaSuccess ? LP_OK
                                                                                                  : LP_ERR_CUDA;
}

int lp_mlp_forward(lp_mlp* M, const float* X, int32_t batch, float* Y) {
  if (!M || !X || !Y || batch <= 0) return LP_ERR_ARG;
  const int rc = M->forward(X, batch);
  if (rc != LP_OK) return rc;
  if (cudaMemcpyAsync(Y, M->y, sizeof(float) * (size_t)M->out * batch, cudaMemcpyDeviceToDevice, M->st) !=
      cudaSuccess)
    return LP_ERR_CUDA;
  return M->status();
}

int lp_mlp_loss_grad(lp_mlp* M, const float* X, const float* T, int32_t batch, double* loss) {
  if (!M || !X || !T || batch <= 0) return LP_ERR_ARG;
  int rc = M->forward(X, batch);
  if (rc != LP_OK) return rc;
  if (cudaMemsetAsync(M->loss, 0, sizeof(double), M->st) != cudaSuccess) return LP_ERR_CUDA;
  const long long total = (long long)M->out * batch;
  k_mse<<<grid_for(total, M->num_sms), 256, 0, M->st>>>(total, batch, M->y, T, M->d3, M->loss);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  rc = M->backward(X, batch);
  if (rc != LP_OK) return rc;
  if (loss && cudaMemcpyAsync(loss, M->loss, sizeof(double), cudaMemcpyDeviceToHost, M->st) != cudaSuccess)
    return LP_ERR_CUDA;
  return M->status();
}

int lp_mlp_train_step(lp_mlp* M, const float* X, const float* T, int32_t batch, float lr, double* loss) {
  const int rc = lp_mlp_loss_grad(M, X, T, batch, loss);
  if (rc != LP_OK) return rc;
  M->steps += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, (float)M->steps), c2 = 1.0f - std::pow(b2, (float)M->steps);
  k_adam<<<grid_for(M->nparam, M->num_sms), 256, 0, M->st>>>(M->nparam, M->param, M->grad, M->adam_m,
                                                               M->adam_v, lr, b1, b2, 1e-8f, c1, c2);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaStreamSynchronize(M->st) == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

}  // extern "C"

// used by the solver's warm start: Y (out x 1) from X (in x 1) into the
// caller's scratch (mlp_predict_scratch_floats floats) on the caller's
// stream, so the model is only read and handles solving concurrently may
// share it.
namespace lpk {
void mlp_dims(const lp_mlp* M, int* in, int* out, int* hid) {
  *in = M->in;
  *out = M->out;
  if (hid) *hid = M->hid;
}

size_t mlp_predict_scratch_floats(const lp_mlp* M) {
  return 2 * (size_t)M->hid + (size_t)32 * std::max(M->hid, M->out);
}

int mlp_predict(lp_mlp* M, const float* X, float* scratch, float* Y, cudaStream_t st) {
  float* h1 = scratch;
  float* h2 = scratch + M->hid;
  float* part = scratch + 2 * (size_t)M->hid;
  const int hid = M->hid, in = M->in, out = M->out;
  auto layer = [&](int rows, int cols, const float* W, const float* b, const float* x, float* y, int act) {
    if (launch_gemv_cm(rows, cols, W, x, part, st) != cudaSuccess) return false;
    k_slices_bias_act<<<(rows + 127) / 128, 128, 0, st>>>(rows, gemv_slices(cols), part, b, y, act);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError() == cudaSuccess;
  };
  if (!layer(hid, in, M->W1(), M->b1(), X, h1, 1)) return LP_ERR_CUDA;
  if (!layer(hid, hid, M->W2(), M->b2(), h1, h2, 1)) return LP_ERR_CUDA;
  if (!layer(out, hid, M->W3(), M->b3(), h2, Y, 0)) return LP_ERR_CUDA;
  return LP_OK;
}
}  // namespace lpk
