// A small multilayer perceptron for the learned warm start of the inner solve:
// in -> H -> H -> out with GELU after both hidden layers,
//     Z1 = W1 X + b1, A1 = gelu(Z1), Z2 = W2 A1 + b2, A2 = gelu(Z2), Y = W3 A2 + b3,
// trained by mean-squared error, L = 1/(2B) sum_b ||Y_b - T_b||^2, with Adam.
//
// Layout: a batch of B samples is a column-major (features x B) matrix, i.e.
// each sample is contiguous; weights are column-major (rows = outputs).  The
// three matrix products per pass are plain library GEMMs (cuBLAS SGEMM); the
// element-wise work is in this file's kernels: bias + GELU (keeping Z for the
// backward pass), the GELU derivative fused with the bias-gradient row sums,
// the loss and its gradient, and the Adam update.  GELU is the exact
// 0.5 z (1 + erf(z / sqrt 2)) with derivative Phi(z) + z phi(z).
#include "internal.h"

#include <cublas_v2.h>

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
  cublasHandle_t blas = nullptr;
  cudaStream_t st = nullptr;
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
    if (blas) cublasDestroy(blas);
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
  bool gemm(cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, const float* A, int lda,
            const float* B, int ldb, float beta, float* C, int ldc) {
    const float one = 1.0f;
    return cublasSgemm(blas, ta, tb, m, n, k, &one, A, lda, B, ldb, &beta, C, ldc) == CUBLAS_STATUS_SUCCESS;
  }
  // Y (out x B) from X (in x B); activations kept for backward
  int forward(const float* X, int B) {
    if (!ensure_batch(B)) return LP_ERR_OOM;
    if (!gemm(CUBLAS_OP_N, CUBLAS_OP_N, hid, B, in, W1(), hid, X, in, 0.0f, z1, hid)) return LP_ERR_CUDA;
    k_bias_act<<<grid_for((long long)hid * B, num_sms), 256, 0, st>>>(hid, B, b1(), z1, a1, 1);
    if (!gemm(CUBLAS_OP_N, CUBLAS_OP_N, hid, B, hid, W2(), hid, a1, hid, 0.0f, z2, hid)) return LP_ERR_CUDA;
    k_bias_act<<<grid_for((long long)hid * B, num_sms), 256, 0, st>>>(hid, B, b2(), z2, a2, 1);
    if (!gemm(CUBLAS_OP_N, CUBLAS_OP_N, out, B, hid, W3(), out, a2, hid, 0.0f, y, out)) return LP_ERR_CUDA;
    k_bias_act<<<grid_for((long long)out * B, num_sms), 256, 0, st>>>(out, B, b3(), y, nullptr, 0);
    g_launches.fetch_add(3, std::memory_order_relaxed);
    return cudaGetLastError() == cudaSuccess ? LP_OK : LP_ERR_CUDA;
  }
  // gradients of the loss from dY (= d3, out x B) for the batch X
  int backward(const float* X, int B) {
    const int wg = std::max(1, std::min(num_sms * 4, (out + 7) / 8));
    k_act_back<<<wg, 256, 0, st>>>(out, B, y, d3, g(b3()), 0);
    if (!gemm(CUBLAS_OP_N, CUBLAS_OP_T, out, hid, B, d3, out, a2, hid, 0.0f, g(W3()), out)) return LP_ERR_CUDA;
    if (!gemm(CUBLAS_OP_T, CUBLAS_OP_N, hid, B, out, W3(), out, d3, out, 0.0f, d2, hid)) return LP_ERR_CUDA;
    const int hg = std::max(1, std::min(num_sms * 4, (hid + 7) / 8));
    k_act_back<<<hg, 256, 0, st>>>(hid, B, z2, d2, g(b2()), 1);
    if (!gemm(CUBLAS_OP_N, CUBLAS_OP_T, hid, hid, B, d2, hid, a1, hid, 0.0f, g(W2()), hid)) return LP_ERR_CUDA;
    if (!gemm(CUBLAS_OP_T, CUBLAS_OP_N, hid, B, hid, W2(), hid, d2, hid, 0.0f, d1, hid)) return LP_ERR_CUDA;
    k_act_back<<<hg, 256, 0, st>>>(hid, B, z1, d1, g(b1()), 1);
    if (!gemm(CUBLAS_OP_N, CUBLAS_OP_T, hid, in, B, d1, hid, X, in, 0.0f, g(W1()), hid)) return LP_ERR_CUDA;
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
  if (cublasCreate(&M->blas) != CUBLAS_STATUS_SUCCESS || cublasSetStream(M->blas, M->st) != CUBLAS_STATUS_SUCCESS) {
    return LP_ERR_CUDA;
  }
  M->nparam = (long long)hidden * in + hidden + (long long)hidden * hidden + hidden + (long long)outdim * hidden + outdim;
  if (!M->alloc(&M->param, M->nparam) || !M->alloc(&M->grad, M->nparam) || !M->alloc(&M->adam_m, M->nparam) ||
      !M->alloc(&M->adam_v, M->nparam) || !M->alloc(&M->loss, 1)) {
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
  return cudaStreamSynchronize(M->st) == cudaSuccess ? LP_OK : LP_ERR_CUDA;
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
  return cudaStreamSynchronize(M->st) == cudaSuccess ? LP_OK : LP_ERR_CUDA;
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

// used by the solver's warm start: Y (out x 1) from X (in x 1) on the caller's
// cuBLAS handle (bound to the caller's stream) and scratch (2 hid floats), so
// the model is only read: handles solving concurrently may share it, and no
// cuBLAS stream switch (which resets its workspace) happens per call.
namespace lpk {
void mlp_dims(const lp_mlp* M, int* in, int* out, int* hid) {
  *in = M->in;
  *out = M->out;
  if (hid) *hid = M->hid;
}

int mlp_predict(lp_mlp* M, cublasHandle_t blas, const float* X, float* scratch, float* Y,
                cudaStream_t st) {
  const float one = 1.0f, zero = 0.0f;
  float* h1 = scratch;
  float* h2 = scratch + M->hid;
  const int hid = M->hid, in = M->in, out = M->out;
  auto gemv = [&](int rows, int cols, const float* W, const float* x, float* y) {
    return cublasSgemv(blas, CUBLAS_OP_N, rows, cols, &one, W, rows, x, 1, &zero, y, 1) ==
           CUBLAS_STATUS_SUCCESS;
  };
  if (!gemv(hid, in, M->W1(), X, h1)) return LP_ERR_CUDA;
  k_bias_act<<<grid_for(hid, M->num_sms), 256, 0, st>>>(hid, 1, M->b1(), h1, h1, 1);
  if (!gemv(hid, hid, M->W2(), h1, h2)) return LP_ERR_CUDA;
  k_bias_act<<<grid_for(hid, M->num_sms), 256, 0, st>>>(hid, 1, M->b2(), h2, h2, 1);
  if (!gemv(out, hid, M->W3(), h2, Y)) return LP_ERR_CUDA;
  k_bias_act<<<grid_for(out, M->num_sms), 256, 0, st>>>(out, 1, M->b3(), Y, nullptr, 0);
  g_launches.fetch_add(3, std::memory_order_relaxed);
  return cudaGetLastError() == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}
}  // namespace lpk
