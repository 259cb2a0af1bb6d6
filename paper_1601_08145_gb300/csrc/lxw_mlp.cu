// lxw_mlp.cu -- training of the learned troubled-cell indicator: an MLP
// 24 -> 64 (ReLU) -> 64 (ReLU) -> 1 (sigmoid) fitted by mean-squared error to
// the shock-capturing limiter's theta (Sec. 4.1) on features of cells the
// method itself produces.  Forward, backward and Adam are the kernels below
// (FP32); the step kernels read a BF16 copy of the weights (FP32 accumulate).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lxw_internal.h"

using namespace lxw;

namespace {

constexpr int TB = 16;   // GEMM tile

// C[M][N] = alpha * op(A) op(B) + beta * C, row-major; op(A) is M x K
// (A stored K x M when ta), op(B) is K x N (B stored N x K when tb).
__global__ void k_gemm(int M, int N, int K, const float* __restrict__ A, int ta, const float* __restrict__ B,
                       int tb, float* __restrict__ C, float alpha, float beta) {
  __shared__ float As[TB][TB + 1], Bs[TB][TB + 1];
  const int r = blockIdx.y * TB + threadIdx.y, c = blockIdx.x * TB + threadIdx.x;
  float acc = 0.0f;
  for (int k0 = 0; k0 < K; k0 += TB) {
    const int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
    const int ar = blockIdx.y * TB + threadIdx.y;
    As[threadIdx.y][threadIdx.x] = (ar < M && ka < K) ? (ta ? A[(size_t)ka * M + ar] : A[(size_t)ar * K + ka]) : 0.0f;
    Bs[threadIdx.y][threadIdx.x] = (kb < K && c < N) ? (tb ? B[(size_t)c * K + kb] : B[(size_t)kb * N + c]) : 0.0f;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TB; ++k) acc = fmaf(As[threadIdx.y][k], Bs[k][threadIdx.x], acc);
    __syncthreads();
  }
  if (r < M && c < N) C[(size_t)r * N + c] = alpha * acc + (beta != 0.0f ? beta * C[(size_t)r * N + c] : 0.0f);
}

// Z += b (broadcast over rows); H = relu(Z)
__global__ void k_bias_relu(int B, int N, float* __restrict__ Z, const float* __restrict__ b, float* __restrict__ H) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * N) return;
  const float z = Z[idx] + b[idx % N];
  Z[idx] = z;
  H[idx] = fmaxf(z, 0.0f);
}

// output layer: yhat = sigmoid(z + b3); loss += (yhat - y)^2 / B; dz = 2 (yhat - y) yhat (1 - yhat) / B
__global__ void k_head(int B, const float* __restrict__ z, const float* __restrict__ b3, const float* __restrict__ y,
                       float* __restrict__ yhat, float* __restrict__ dz, float* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.0f;
  if (i < B) {
    const float s = 1.0f / (1.0f + expf(-(z[i] + b3[0])));
    if (yhat) yhat[i] = s;
    if (y) {
      const float d = s - y[i];
      l = d * d / B;
      if (dz) dz[i] = 2.0f * d * s * (1.0f - s) / B;
    }
  }
  if (loss) {
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
  }
}

// dZ = dH * (Z > 0)
__global__ void k_relu_back(int n, float* __restrict__ dH, const float* __restrict__ Z) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n && !(Z[idx] > 0.0f)) dH[idx] = 0.0f;
}

// db[N] = sum over rows of dZ[B][N]
__global__ void k_colsum(int B, int N, const float* __restrict__ dZ, float* __restrict__ db) {
  const int c = blockIdx.x;
  float acc = 0.0f;
  for (int r = threadIdx.x; r < B; r += blockDim.x) acc += dZ[(size_t)r * N + c];
  __shared__ float red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[c] = red[0];
}

__global__ void k_adam(int n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi, vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi; v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_gather(int B, const int* __restrict__ idx, const float* __restrict__ X, const float* __restrict__ y,
                         float* __restrict__ Xb, float* __restrict__ yb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * lxw::kMlpIn) return;
  const int r = t / lxw::kMlpIn, c = t % lxw::kMlpIn;
  const int s = idx[r];
  Xb[t] = X[(size_t)s * lxw::kMlpIn + c];
  if (c == 0) yb[r] = y[s];
}

// order-preserving int key of a float (NaN excluded), and back
__device__ __forceinline__ int fkey(float x) {
  const int i = __float_as_int(x);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
inline float fkey_inv(int k) {
  const int i = k >= 0 ? k : k ^ 0x7fffffff;
  float x;
  std::memcpy(&x, &i, sizeof x);
  return x;
}

// per-feature minimum and maximum of X[count][24]: one column per lane
// group, atomics on the order-preserving keys
__global__ void k_feature_range(int count, const float* __restrict__ X, int* __restrict__ keys) {
  const int c = threadIdx.x % lxw::kMlpIn;
  const int r0 = blockIdx.x * (blockDim.x / lxw::kMlpIn) + threadIdx.x / lxw::kMlpIn;
  const int rs = gridDim.x * (blockDim.x / lxw::kMlpIn);
  if (threadIdx.x >= (blockDim.x / lxw::kMlpIn) * lxw::kMlpIn) return;
  int lo = 0x7fffffff, hi = (int)0x80000000;
  for (int r = r0; r < count; r += rs) {
    const int k = fkey(X[(size_t)r * lxw::kMlpIn + c]);
    lo = min(lo, k); hi = max(hi, k);
  }
  atomicMin(keys + c, lo);
  atomicMax(keys + lxw::kMlpIn + c, hi);
}

// round to nearest even (the parameters are finite)
__device__ __forceinline__ unsigned short bf16_rne(float x) {
  unsigned u = __float_as_uint(x);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (unsigned short)(u >> 16);
}
__device__ __forceinline__ float bf16_widen(unsigned short h) { return __uint_as_float((unsigned)h << 16); }

// parameter vector -> GateWeights (zero padding included)
__global__ void k_gate_layout(const float* __restrict__ p, GateWeights* __restrict__ g) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kMlpH * kMlpH; k += gridDim.x * blockDim.x) {
    const int n = k / kMlpH, c = k % kMlpH;            // output unit n, input c
    g->w2[umma_kmajor(n, c, kMlpH)] = bf16_rne(p[kW2 + c * kMlpH + n]);
    if (c < kGateK1) g->w1[umma_kmajor(n, c, kGateK1)] = c < kMlpIn ? bf16_rne(p[kW1 + c * kMlpH + n]) : (unsigned short)0;
    if (n == 0) {
      g->b1[c] = bf16_widen(bf16_rne(p[kB1 + c]));
      g->b2[c] = bf16_widen(bf16_rne(p[kB2 + c]));
      g->w3[c] = bf16_widen(bf16_rne(p[kW3 + c]));
    }
    if (k == 0) { g->b3 = bf16_widen(bf16_rne(p[kB3])); g->pad[0] = g->pad[1] = g->pad[2] = 0.0f; }
  }
}

}  // namespace

struct lxw_mlp {
  int maxB = 0;
  cudaStream_t stream = nullptr;
  // envelope of the training features: the gate uses the prediction only
  // for cells whose features lie inside it (unbounded until set or trained)
  bool env_set = false;
  float lo[kMlpIn], hi[kMlpIn];
  int* env_keys = nullptr;                  // device: order-preserving keys of min [24], max [24]
  float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  float *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr, *z3 = nullptr, *yhat = nullptr, *dz = nullptr;
  float *dH = nullptr, *Xb = nullptr, *yb = nullptr, *loss = nullptr;
  int* idx = nullptr;
  int adam_t = 0;
  std::vector<void*> allocs;
  ~lxw_mlp() { for (void* p : allocs) cudaFree(p); }
};

namespace {

inline dim3 gemm_grid(int M, int N) { return dim3((N + TB - 1) / TB, (M + TB - 1) / TB); }

// forward on rows X[B][24]; leaves Z1, H1, Z2, H2, z3 (pre-bias) in the workspace
void forward(lxw_mlp* n, const float* X, int B) {
  cudaStream_t st = n->stream;
  const float* P = n->params;
  k_gemm<<<gemm_grid(B, kMlpH), dim3(TB, TB), 0, st>>>(B, kMlpH, kMlpIn, X, 0, P + kW1, 0, n->Z1, 1.0f, 0.0f);
  k_bias_relu<<<(B * kMlpH + 255) / 256, 256, 0, st>>>(B, kMlpH, n->Z1, P + kB1, n->H1);
  k_gemm<<<gemm_grid(B, kMlpH), dim3(TB, TB), 0, st>>>(B, kMlpH, kMlpH, n->H1, 0, P + kW2, 0, n->Z2, 1.0f, 0.0f);
  k_bias_relu<<<(B * kMlpH + 255) / 256, 256, 0, st>>>(B, kMlpH, n->Z2, P + kB2, n->H2);
  k_gemm<<<gemm_grid(B, 1), dim3(TB, TB), 0, st>>>(B, 1, kMlpH, n->H2, 0, P + kW3, 0, n->z3, 1.0f, 0.0f);
}

// mean-squared-error loss and its gradient w.r.t. every parameter
void backward(lxw_mlp* n, const float* X, const float* y, int B) {
  cudaStream_t st = n->stream;
  const float* P = n->params;
  float* G = n->grad;
  k_head<<<(B + 255) / 256, 256, 0, st>>>(B, n->z3, P + kB3, y, n->yhat, n->dz, n->loss);
  // output layer
  k_gemm<<<gemm_grid(kMlpH, 1), dim3(TB, TB), 0, st>>>(kMlpH, 1, B, n->H2, 1, n->dz, 0, G + kW3, 1.0f, 0.0f);
  k_colsum<<<1, 256, 0, st>>>(B, 1, n->dz, G + kB3);
  // dH2 = dz w3^T, masked by Z2 > 0
  k_gemm<<<gemm_grid(B, kMlpH), dim3(TB, TB), 0, st>>>(B, kMlpH, 1, n->dz, 0, P + kW3, 0, n->dH, 1.0f, 0.0f);
  k_relu_back<<<(B * kMlpH + 255) / 256, 256, 0, st>>>(B * kMlpH, n->dH, n->Z2);
  k_gemm<<<gemm_grid(kMlpH, kMlpH), dim3(TB, TB), 0, st>>>(kMlpH, kMlpH, B, n->H1, 1, n->dH, 0, G + kW2, 1.0f, 0.0f);
  k_colsum<<<kMlpH, 256, 0, st>>>(B, kMlpH, n->dH, G + kB2);
  // dH1 = dZ2 W2^T, masked by Z1 > 0 (H2 buffer reused)
  k_gemm<<<gemm_grid(B, kMlpH), dim3(TB, TB), 0, st>>>(B, kMlpH, kMlpH, n->dH, 0, P + kW2, 1, n->H2, 1.0f, 0.0f);
  k_relu_back<<<(B * kMlpH + 255) / 256, 256, 0, st>>>(B * kMlpH, n->H2, n->Z1);
  k_gemm<<<gemm_grid(kMlpIn, kMlpH), dim3(TB, TB), 0, st>>>(kMlpIn, kMlpH, B, X, 1, n->H2, 0, G + kW1, 1.0f, 0.0f);
  k_colsum<<<kMlpH, 256, 0, st>>>(B, kMlpH, n->H2, G + kB1);
}

thread_local std::string g_mlp_err;
lxw_status mfail(lxw_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

uint64_t splitmix(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double unif(uint64_t& x) { return (double)(splitmix(x) >> 11) * (1.0 / 9007199254740992.0); }

}  // namespace

extern "C" {

lxw_status lxw_mlp_create(int max_batch, unsigned long long seed, void* stream, lxw_mlp** out) {
  if (!out || max_batch < 1 || max_batch > (1 << 22)) return mfail(LXW_ERR_ARG, "lxw_mlp_create: bad argument");
  lxw_mlp* n = new (std::nothrow) lxw_mlp;
  if (!n) return mfail(LXW_ERR_NOMEM, "lxw_mlp_create: out of memory");
  n->maxB = max_batch;
  n->stream = (cudaStream_t)stream;
  auto al = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    n->allocs.push_back(p);
    return p;
  };
  const size_t B = max_batch, H = kMlpH;
  n->params = (float*)al(sizeof(float) * kMlpParams);
  n->grad = (float*)al(sizeof(float) * kMlpParams);
  n->m = (float*)al(sizeof(float) * kMlpParams);
  n->v = (float*)al(sizeof(float) * kMlpParams);
  n->Z1 = (float*)al(sizeof(float) * B * H); n->H1 = (float*)al(sizeof(float) * B * H);
  n->Z2 = (float*)al(sizeof(float) * B * H); n->H2 = (float*)al(sizeof(float) * B * H);
  n->dH = (float*)al(sizeof(float) * B * H);
  n->z3 = (float*)al(sizeof(float) * B); n->yhat = (float*)al(sizeof(float) * B); n->dz = (float*)al(sizeof(float) * B);
  n->Xb = (float*)al(sizeof(float) * B * kMlpIn); n->yb = (float*)al(sizeof(float) * B);
  n->idx = (int*)al(sizeof(int) * B);
  n->loss = (float*)al(sizeof(float));
  n->env_keys = (int*)al(sizeof(int) * 2 * kMlpIn);
  for (int k = 0; k < kMlpIn; ++k) { n->lo[k] = -INFINITY; n->hi[k] = INFINITY; }
  for (void* p : n->allocs)
    if (!p) { delete n; return mfail(LXW_ERR_NOMEM, "lxw_mlp_create: device allocation failed"); }
  // He initialisation from SplitMix64 (Box-Muller), zero biases
  std::vector<float> P(kMlpParams, 0.0f);
  uint64_t x = seed;
  auto gauss = [&]() { double u1 = unif(x), u2 = unif(x); return std::sqrt(-2.0 * std::log(u1 + 1e-300)) * std::cos(6.283185307179586 * u2); };
  for (int k = 0; k < kMlpIn * kMlpH; ++k) P[kW1 + k] = (float)(gauss() * std::sqrt(2.0 / kMlpIn));
  for (int k = 0; k < kMlpH * kMlpH; ++k) P[kW2 + k] = (float)(gauss() * std::sqrt(2.0 / kMlpH));
  for (int k = 0; k < kMlpH; ++k) P[kW3 + k] = (float)(gauss() * std::sqrt(1.0 / kMlpH));
  P[kB3] = 2.0f;   // start near theta = 1 (most cells are not limited)
  if (cudaMemcpy(n->params, P.data(), sizeof(float) * kMlpParams, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(n->m, 0, sizeof(float) * kMlpParams) != cudaSuccess ||
      cudaMemset(n->v, 0, sizeof(float) * kMlpParams) != cudaSuccess) {
    delete n;
    return mfail(LXW_ERR_CUDA, "lxw_mlp_create: upload failed");
  }
  *out = n;
  return LXW_OK;
}

void lxw_mlp_destroy(lxw_mlp* n) { delete n; }

int lxw_mlp_num_params(void) { return kMlpParams; }

lxw_status lxw_mlp_get_params(lxw_mlp* n, float* params_dev) {
  if (!n || !params_dev) return mfail(LXW_ERR_ARG, "lxw_mlp_get_params: null argument");
  if (cudaMemcpyAsync(params_dev, n->params, sizeof(float) * kMlpParams, cudaMemcpyDeviceToDevice, n->stream))
    return mfail(LXW_ERR_CUDA, "lxw_mlp_get_params: copy failed");
  return LXW_OK;
}

lxw_status lxw_mlp_set_params(lxw_mlp* n, const float* params_dev) {
  if (!n || !params_dev) return mfail(LXW_ERR_ARG, "lxw_mlp_set_params: null argument");
  if (cudaMemcpyAsync(n->params, params_dev, sizeof(float) * kMlpParams, cudaMemcpyDeviceToDevice, n->stream))
    return mfail(LXW_ERR_CUDA, "lxw_mlp_set_params: copy failed");
  return LXW_OK;
}

lxw_status lxw_mlp_forward(lxw_mlp* n, const float* X, int B, float* yhat) {
  if (!n || !X || !yhat || B < 1 || B > n->maxB) return mfail(LXW_ERR_ARG, "lxw_mlp_forward: bad argument");
  forward(n, X, B);
  k_head<<<(B + 255) / 256, 256, 0, n->stream>>>(B, n->z3, n->params + kB3, nullptr, yhat, nullptr, nullptr);
  return cudaGetLastError() == cudaSuccess ? LXW_OK : mfail(LXW_ERR_CUDA, "lxw_mlp_forward: launch failed");
}

lxw_status lxw_mlp_loss_grad(lxw_mlp* n, const float* X, const float* y, int B, float* loss_host, float* grad_dev) {
  if (!n || !X || !y || B < 1 || B > n->maxB) return mfail(LXW_ERR_ARG, "lxw_mlp_loss_grad: bad argument");
  cudaMemsetAsync(n->loss, 0, sizeof(float), n->stream);
  forward(n, X, B);
  backward(n, X, y, B);
  if (grad_dev) cudaMemcpyAsync(grad_dev, n->grad, sizeof(float) * kMlpParams, cudaMemcpyDeviceToDevice, n->stream);
  if (loss_host) {
    if (cudaMemcpyAsync(loss_host, n->loss, sizeof(float), cudaMemcpyDeviceToHost, n->stream) ||
        cudaStreamSynchronize(n->stream))
      return mfail(LXW_ERR_CUDA, "lxw_mlp_loss_grad: copy failed");
  }
  return cudaGetLastError() == cudaSuccess ? LXW_OK : mfail(LXW_ERR_CUDA, "lxw_mlp_loss_grad: launch failed");
}

lxw_status lxw_mlp_set_envelope(lxw_mlp* n, const float* lo, const float* hi) {
  if (!n || (!lo) != (!hi)) return mfail(LXW_ERR_ARG, "lxw_mlp_set_envelope: bad argument");
  for (int k = 0; k < kMlpIn; ++k) {
    if (lo && !(lo[k] <= hi[k])) return mfail(LXW_ERR_ARG, "lxw_mlp_set_envelope: needs lo <= hi");
    n->lo[k] = lo ? lo[k] : -INFINITY;
    n->hi[k] = hi ? hi[k] : INFINITY;
  }
  n->env_set = lo != nullptr;
  return LXW_OK;
}

lxw_status lxw_mlp_get_envelope(const lxw_mlp* n, float* lo, float* hi) {
  if (!n || !lo || !hi) return mfail(LXW_ERR_ARG, "lxw_mlp_get_envelope: null argument");
  for (int k = 0; k < kMlpIn; ++k) { lo[k] = n->lo[k]; hi[k] = n->hi[k]; }
  return LXW_OK;
}

lxw_status lxw_mlp_train(lxw_mlp* n, const float* X, const float* y, int count, int epochs, int batch, float lr,
                         unsigned long long seed, float* last_loss) {
  if (!n || !X || !y || count < 1 || epochs < 1 || batch < 1 || batch > n->maxB || !(lr > 0.0f))
    return mfail(LXW_ERR_ARG, "lxw_mlp_train: bad argument");
  {  // widen the envelope by these features (the first training call sets it)
    int keys[2 * kMlpIn];
    for (int k = 0; k < kMlpIn; ++k) { keys[k] = 0x7fffffff; keys[kMlpIn + k] = (int)0x80000000; }
    const int blocks = std::min(1024, (count + 9) / 10);
    if (cudaMemcpyAsync(n->env_keys, keys, sizeof keys, cudaMemcpyHostToDevice, n->stream))
      return mfail(LXW_ERR_CUDA, "lxw_mlp_train: copy failed");
    k_feature_range<<<blocks, 240, 0, n->stream>>>(count, X, n->env_keys);
    if (cudaMemcpyAsync(keys, n->env_keys, sizeof keys, cudaMemcpyDeviceToHost, n->stream) ||
        cudaStreamSynchronize(n->stream))
      return mfail(LXW_ERR_CUDA, "lxw_mlp_train: feature range failed");
    for (int k = 0; k < kMlpIn; ++k) {
      const float lo = fkey_inv(keys[k]), hi = fkey_inv(keys[kMlpIn + k]);
      n->lo[k] = n->env_set ? std::min(n->lo[k], lo) : lo;
      n->hi[k] = n->env_set ? std::max(n->hi[k], hi) : hi;
    }
    n->env_set = true;
  }
  uint64_t x = seed;
  std::vector<int> perm(count);
  float loss = 0.0f;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int k = 0; k < count; ++k) perm[k] = k;
    for (int k = count - 1; k > 0; --k) {
      int j = (int)(splitmix(x) % (uint64_t)(k + 1));
      std::swap(perm[k], perm[j]);
    }
    for (int b0 = 0; b0 + batch <= count; b0 += batch) {
      if (cudaMemcpyAsync(n->idx, perm.data() + b0, sizeof(int) * batch, cudaMemcpyHostToDevice, n->stream))
        return mfail(LXW_ERR_CUDA, "lxw_mlp_train: copy failed");
      k_gather<<<(batch * kMlpIn + 255) / 256, 256, 0, n->stream>>>(batch, n->idx, X, y, n->Xb, n->yb);
      cudaMemsetAsync(n->loss, 0, sizeof(float), n->stream);
      forward(n, n->Xb, batch);
      backward(n, n->Xb, n->yb, batch);
      ++n->adam_t;
      const float b1 = 0.9f, b2 = 0.999f;
      k_adam<<<(kMlpParams + 255) / 256, 256, 0, n->stream>>>(kMlpParams, n->params, n->grad, n->m, n->v, lr, b1, b2,
                                                              1e-8f, 1.0f - std::pow(b1, (float)n->adam_t),
                                                              1.0f - std::pow(b2, (float)n->adam_t));
      if (cudaStreamSynchronize(n->stream)) return mfail(LXW_ERR_CUDA, "lxw_mlp_train: step failed");
    }
  }
  if (cudaMemcpy(&loss, n->loss, sizeof(float), cudaMemcpyDeviceToHost)) return mfail(LXW_ERR_CUDA, "lxw_mlp_train: copy");
  if (last_loss) *last_loss = loss;
  return LXW_OK;
}

}  // extern "C"

namespace lxw {
int mlp_gate_weights(lxw_mlp* n, GateWeights* out) {
  k_gate_layout<<<(kMlpH * kMlpH + 255) / 256, 256, 0, n->stream>>>(n->params, out);
  if (cudaMemcpyAsync(out->lo, n->lo, sizeof n->lo, cudaMemcpyHostToDevice, n->stream) ||
      cudaMemcpyAsync(out->hi, n->hi, sizeof n->hi, cudaMemcpyHostToDevice, n->stream))
    return -1;
  return cudaStreamSynchronize(n->stream) == cudaSuccess ? 0 : -1;
}
}  // namespace lxw
