// Warm-start network of libsos: a multilayer perceptron trained and run on
// the tensor cores with hand-written kernels.
//
//   h1 = relu(X W1^T + b1), h2 = relu(h1 W2^T + b2), y = h2 W3^T + b3
//
// trained on the mean squared error of standardised targets with Adam.  Every
// matrix product is one tcgen05 GEMM kernel: operands are rounded to BF16 when
// they are staged into shared memory, products accumulate in FP32 in tensor
// memory, and the epilogue applies bias, ReLU or the ReLU derivative.  Master
// weights, activations, gradients and Adam moments are FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "../../include/sos.h"
#include "setup.h"
#include "tcgen05.cuh"

namespace sos {
namespace {

constexpr int kTM = 128, kTN = 64, kKC = 64;
constexpr size_t kGemmSmem = (kTM + kTN) * kKC * 2;  // BF16 A and B chunks

enum Epi : int32_t { kEpiStore = 0, kEpiBiasRelu = 1, kEpiBias = 2, kEpiReluGrad = 3 };

struct GemmArgs {
  const float* A;  // element (m, k) = A[m * lda + k], or A[k * lda + m] when a_t
  const float* B;  // element (n, k) = B[n * ldb + k], or B[k * ldb + n] when b_t
  float* C;        // C[m * ldc + n]
  const float* bias;  // [N] (bias epilogues)
  const float* H;     // [M x ldc] activations whose positive part masks the ReLU derivative
  int M, N, K, lda, ldb, ldc;
  int a_t, b_t, epi;
  int32_t* err;
};

__device__ __forceinline__ uint32_t core_off(int r, int k) {
  return static_cast<uint32_t>((r >> 3) * ((kKC / 8) * 128) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// rows [r0, r0 + R) x k in [k0, k0 + kKC) of an operand, zero outside [0, rows) x [0, K)
__device__ __forceinline__ void stage(const float* X, int ld, int trans, int rows, int K, int r0, int R, int k0,
                                      unsigned char* dst) {
  for (int idx = threadIdx.x; idx < R * kKC; idx += blockDim.x) {
    int r, k;
    if (trans) {  // consecutive threads walk r: coalesced for a transposed read
      k = idx / R;
      r = idx - k * R;
    } else {
      r = idx / kKC;
      k = idx - r * kKC;
    }
    const int gr = r0 + r, gk = k0 + k;
    float x = 0.f;
    if (gr < rows && gk < K) x = trans ? X[static_cast<int64_t>(gk) * ld + gr] : X[static_cast<int64_t>(gr) * ld + gk];
    *reinterpret_cast<__nv_bfloat16*>(dst + core_off(r, k)) = __float2bfloat16_rn(x);
  }
}

__global__ void __launch_bounds__(256) k_gemm(GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
  unsigned char* sa = sm;
  unsigned char* sb = sm + kTM * kKC * 2;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_base)),
                 "r"(kTN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t LBO = 128, SBO = (kKC / 8) * 128;
  constexpr uint32_t idesc = tc::idesc_bf16(kTM, kTN);
  uint32_t phase = 0;
  bool ok = true;
  for (int k0 = 0; k0 < g.K; k0 += kKC) {
    stage(g.A, g.lda, g.a_t, g.M, g.K, m0, kTM, k0, sa);
    stage(g.B, g.ldb, g.b_t, g.N, g.K, n0, kTN, k0, sb);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (threadIdx.x == 0 && ok) {
      const uint32_t a0 = tc::smem_u32(sa), b0 = tc::smem_u32(sb);
      for (int s = 0; s < kKC / 16; ++s) {
        const uint32_t so = s * 2 * LBO;
        tc::mma(tmem, tc::desc(a0 + so, LBO, SBO), tc::desc(b0 + so, LBO, SBO), idesc, (k0 > 0 || s > 0) ? 1u : 0u);
      }
      tc::commit(&mbar);
    }
    if (ok && !tc::wait(&mbar, phase)) ok = false;
    phase ^= 1u;
    tc::fence_after();
  }
  if (ok) {
    const int wq = (threadIdx.x >> 5) & 3, ch = threadIdx.x >> 7;
    const int row = m0 + wq * 32 + (threadIdx.x & 31);
    for (int c0 = ch * 32; c0 < ch * 32 + 32; c0 += 8) {
      float v[8];
      tc::ld8(tmem + (static_cast<uint32_t>(wq * 32) << 16) + c0, v);
      if (row >= g.M) continue;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int col = n0 + c0 + j;
        if (col >= g.N) continue;
        const int64_t o = static_cast<int64_t>(row) * g.ldc + col;
        float x = v[j];
        if (g.epi == kEpiBiasRelu) x = fmaxf(x + g.bias[col], 0.f);
        else if (g.epi == kEpiBias) x += g.bias[col];
        else if (g.epi == kEpiReluGrad) x = g.H[o] > 0.f ? x : 0.f;
        g.C[o] = x;
      }
    }
  } else {
    tc::wait(&mbar, phase ^ 1u);  // one more bounded wait for MMAs still in flight
    if (threadIdx.x == 0) atomicExch(g.err, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTN));
}

// column sums: out[j] = sum_i X[i * ld + j]
__global__ void k_colsum(const float* X, int rows, int cols, int ld, float* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float s = 0.f;
  for (int i = 0; i < rows; ++i) s += X[static_cast<int64_t>(i) * ld + j];
  out[j] = s;
}

// dY = 2 (y - (Y - mu) / sd) / (B n_out) and per-block partial sums of the squared error
__global__ void k_loss(const float* y, const float* Y, const float* mu, const float* sd, int B, int n, float* dY,
                       double* partial) {
  __shared__ double red[256];
  double acc = 0.0;
  const int64_t total = static_cast<int64_t>(B) * n;
  const float scale = 2.f / static_cast<float>(total);
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < total;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int j = static_cast<int>(q % n);
    const float t = (Y[q] - mu[j]) / sd[j];
    const float r = y[q] - t;
    dY[q] = scale * r;
    acc += static_cast<double>(r) * r;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Adam (bias-corrected moments), in place over the flat parameter vector
__global__ void k_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < n;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.f - b1) * gq;
    const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    p[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
  }
}

// y = mu + sd * yhat (de-standardised prediction)
__global__ void k_unscale(float* y, const float* mu, const float* sd, int B, int n) {
  const int64_t total = static_cast<int64_t>(B) * n;
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < total;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int j = static_cast<int>(q % n);
    y[q] = mu[j] + sd[j] * y[q];
  }
}

// per-column mean and standard deviation (floored) of Y [rows x n]
__global__ void k_colstats(const float* Y, int rows, int n, float* mu, float* sd) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0, s2 = 0.0;
  for (int i = 0; i < rows; ++i) {
    const double x = Y[static_cast<int64_t>(i) * n + j];
    s += x;
    s2 += x * x;
  }
  const double mean = s / rows;
  const double var = fmax(s2 / rows - mean * mean, 0.0);
  mu[j] = static_cast<float>(mean);
  sd[j] = static_cast<float>(fmax(sqrt(var), 1e-6));
}

thread_local std::string g_mlp_err;

}  // namespace
}  // namespace sos

using namespace sos;

struct sos_mlp {
  int n_in = 0, n_hid = 0, n_out = 0;
  cudaStream_t s = nullptr;
  int64_t n_param = 0;
  float *param = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  float *mu = nullptr, *sd = nullptr;
  float *h1 = nullptr, *h2 = nullptr, *y = nullptr, *d2 = nullptr, *d1 = nullptr, *dy = nullptr;
  double* partial = nullptr;
  int32_t* err = nullptr;
  int cap = 0;  // batch capacity of the activation buffers
  int64_t step = 0;
  std::vector<void*> allocs;
  // offsets into the flat parameter vector
  int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
};

namespace {

int mfail(int code, const std::string& msg) {
  set_global_error(msg);
  return code;
}

#define MCK(call)                                                                                       \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) return mfail(SOS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename V>
int malloc_track(sos_mlp* net, V** p, size_t count) {
  void* q = nullptr;
  MCK(cudaMalloc(&q, sizeof(V) * (count ? count : 1)));
  MCK(cudaMemsetAsync(q, 0, sizeof(V) * (count ? count : 1), net->s));
  net->allocs.push_back(q);
  *p = static_cast<V*>(q);
  return SOS_OK;
}

int ensure_batch(sos_mlp* net, int B) {
  if (B <= net->cap) return SOS_OK;
  for (float** b : {&net->h1, &net->h2, &net->d2, &net->d1})
    if (*b) {
      cudaFree(*b);
      *b = nullptr;
    }
  if (net->y) cudaFree(net->y);
  if (net->dy) cudaFree(net->dy);
  net->y = net->dy = nullptr;
  auto mk = [&](float** p, size_t n) -> int {
    MCK(cudaMalloc(reinterpret_cast<void**>(p), sizeof(float) * n));
    return SOS_OK;
  };
  const size_t bh = static_cast<size_t>(B) * net->n_hid, bo = static_cast<size_t>(B) * net->n_out;
  int rc;
  if ((rc = mk(&net->h1, bh)) || (rc = mk(&net->h2, bh)) || (rc = mk(&net->d2, bh)) || (rc = mk(&net->d1, bh)) ||
      (rc = mk(&net->y, bo)) || (rc = mk(&net->dy, bo)))
    return rc;
  net->cap = B;
  return SOS_OK;
}

cudaError_t gemm(sos_mlp* net, const float* A, int lda, int a_t, const float* B, int ldb, int b_t, float* C, int ldc,
                 int M, int N, int K, int epi, const float* bias, const float* H) {
  GemmArgs g{A, B, C, bias, H, M, N, K, lda, ldb, ldc, a_t, b_t, epi, net->err};
  dim3 grid((N + kTN - 1) / kTN, (M + kTM - 1) / kTM);
  k_gemm<<<grid, 256, kGemmSmem, net->s>>>(g);
  return cudaGetLastError();
}

int forward(sos_mlp* net, const float* X, int B) {
  float* P = net->param;
  MCK(gemm(net, X, net->n_in, 0, P + net->oW1, net->n_in, 0, net->h1, net->n_hid, B, net->n_hid, net->n_in,
           kEpiBiasRelu, P + net->ob1, nullptr));
  MCK(gemm(net, net->h1, net->n_hid, 0, P + net->oW2, net->n_hid, 0, net->h2, net->n_hid, B, net->n_hid, net->n_hid,
           kEpiBiasRelu, P + net->ob2, nullptr));
  MCK(gemm(net, net->h2, net->n_hid, 0, P + net->oW3, net->n_hid, 0, net->y, net->n_out, B, net->n_out, net->n_hid,
           kEpiBias, P + net->ob3, nullptr));
  return SOS_OK;
}

int backward(sos_mlp* net, const float* X, const float* Y, int B, double* loss) {
  const int nh = net->n_hid, no = net->n_out, ni = net->n_in;
  k_loss<<<256, 256, 0, net->s>>>(net->y, Y, net->mu, net->sd, B, no, net->dy, net->partial);
  MCK(cudaGetLastError());
  float* G = net->grad;
  float* P = net->param;
  // layer 3: dW3 = dy^T h2, db3 = colsum(dy), dh2 = dy W3 masked by h2 > 0
  MCK(gemm(net, net->dy, no, 1, net->h2, nh, 1, G + net->oW3, nh, no, nh, B, kEpiStore, nullptr, nullptr));
  k_colsum<<<(no + 255) / 256, 256, 0, net->s>>>(net->dy, B, no, no, G + net->ob3);
  MCK(gemm(net, net->dy, no, 0, P + net->oW3, nh, 1, net->d2, nh, B, nh, no, kEpiReluGrad, nullptr, net->h2));
  // layer 2
  MCK(gemm(net, net->d2, nh, 1, net->h1, nh, 1, G + net->oW2, nh, nh, nh, B, kEpiStore, nullptr, nullptr));
  k_colsum<<<(nh + 255) / 256, 256, 0, net->s>>>(net->d2, B, nh, nh, G + net->ob2);
  MCK(gemm(net, net->d2, nh, 0, P + net->oW2, nh, 1, net->d1, nh, B, nh, nh, kEpiReluGrad, nullptr, net->h1));
  // layer 1
  MCK(gemm(net, net->d1, nh, 1, X, ni, 1, G + net->oW1, ni, nh, ni, B, kEpiStore, nullptr, nullptr));
  k_colsum<<<(nh + 255) / 256, 256, 0, net->s>>>(net->d1, B, nh, nh, G + net->ob1);
  MCK(cudaGetLastError());
  if (loss) {
    std::vector<double> part(256);
    MCK(cudaMemcpyAsync(part.data(), net->partial, sizeof(double) * 256, cudaMemcpyDeviceToHost, net->s));
    MCK(cudaStreamSynchronize(net->s));
    double t = 0.0;
    for (double x : part) t += x;
    *loss = t / (static_cast<double>(B) * no);
  }
  return SOS_OK;
}

int check_err(sos_mlp* net) {
  int32_t e = 0;
  MCK(cudaMemcpyAsync(&e, net->err, sizeof(int32_t), cudaMemcpyDeviceToHost, net->s));
  MCK(cudaStreamSynchronize(net->s));
  if (e) {
    cudaMemsetAsync(net->err, 0, sizeof(int32_t), net->s);
    return mfail(SOS_ERR_TIMEOUT, "a bounded device-side wait expired in the network kernels");
  }
  return SOS_OK;
}

}  // namespace

extern "C" {

int sos_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed, void* stream, sos_mlp** out) {
  if (!out || n_in < 1 || n_hidden < 1 || n_out < 1) return mfail(SOS_ERR_INVALID_ARG, "sos_mlp_create: bad sizes");
  *out = nullptr;
  auto* net = new sos_mlp();
  net->n_in = n_in;
  net->n_hid = n_hidden;
  net->n_out = n_out;
  net->s = static_cast<cudaStream_t>(stream);
  net->oW1 = 0;
  net->ob1 = net->oW1 + static_cast<int64_t>(n_hidden) * n_in;
  net->oW2 = net->ob1 + n_hidden;
  net->ob2 = net->oW2 + static_cast<int64_t>(n_hidden) * n_hidden;
  net->oW3 = net->ob2 + n_hidden;
  net->ob3 = net->oW3 + static_cast<int64_t>(n_out) * n_hidden;
  net->n_param = net->ob3 + n_out;
  int rc = SOS_OK;
  if ((rc = malloc_track(net, &net->param, net->n_param)) || (rc = malloc_track(net, &net->grad, net->n_param)) ||
      (rc = malloc_track(net, &net->m, net->n_param)) || (rc = malloc_track(net, &net->v, net->n_param)) ||
      (rc = malloc_track(net, &net->mu, n_out)) || (rc = malloc_track(net, &net->sd, n_out)) ||
      (rc = malloc_track(net, &net->partial, 256)) || (rc = malloc_track(net, &net->err, 1))) {
    sos_mlp_destroy(net);
    return rc;
  }
  if (cudaFuncSetAttribute(k_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kGemmSmem)) !=
      cudaSuccess) {
    sos_mlp_destroy(net);
    return mfail(SOS_ERR_CUDA, "sos_mlp_create: shared memory attribute");
  }
  // He-uniform weights, zero biases; identity output scaling
  std::mt19937_64 rng(seed);
  std::vector<float> h(net->n_param, 0.f);
  auto fill = [&](int64_t off, int rows, int cols) {
    std::uniform_real_distribution<float> u(-std::sqrt(6.f / cols), std::sqrt(6.f / cols));
    for (int64_t q = 0; q < static_cast<int64_t>(rows) * cols; ++q) h[off + q] = u(rng);
  };
  fill(net->oW1, n_hidden, n_in);
  fill(net->oW2, n_hidden, n_hidden);
  fill(net->oW3, n_out, n_hidden);
  std::vector<float> one(n_out, 1.f);
  if (cudaMemcpyAsync(net->param, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, net->s) != cudaSuccess ||
      cudaMemcpyAsync(net->sd, one.data(), sizeof(float) * n_out, cudaMemcpyHostToDevice, net->s) != cudaSuccess ||
      cudaStreamSynchronize(net->s) != cudaSuccess) {
    sos_mlp_destroy(net);
    return mfail(SOS_ERR_CUDA, "sos_mlp_create: upload");
  }
  *out = net;
  return SOS_OK;
}

void sos_mlp_destroy(sos_mlp* net) {
  if (!net) return;
  if (net->s) cudaStreamSynchronize(net->s);
  for (void* p : net->allocs) cudaFree(p);
  for (float* p : {net->h1, net->h2, net->y, net->d2, net->d1, net->dy})
    if (p) cudaFree(p);
  delete net;
}

int64_t sos_mlp_param_count(const sos_mlp* net) { return net ? net->n_param : -1; }

int sos_mlp_set_params(sos_mlp* net, const float* host) {
  if (!net || !host) return mfail(SOS_ERR_INVALID_ARG, "sos_mlp_set_params: NULL");
  MCK(cudaMemcpyAsync(net->param, host, sizeof(float) * net->n_param, cudaMemcpyHostToDevice, net->s));
  MCK(cudaMemsetAsync(net->m, 0, sizeof(float) * net->n_param, net->s));
  MCK(cudaMemsetAsync(net->v, 0, sizeof(float) * net->n_param, net->s));
  net->step = 0;
  MCK(cudaStreamSynchronize(net->s));
  return SOS_OK;
}

int sos_mlp_get_params(const sos_mlp* net, float* host) {
  if (!net || !host) return mfail(SOS_ERR_INVALID_ARG, "sos_mlp_get_params: NULL");
  MCK(cudaMemcpyAsync(host, net->param, sizeof(float) * net->n_param, cudaMemcpyDeviceToHost, net->s));
  MCK(cudaStreamSynchronize(net->s));
  return SOS_OK;
}

int sos_mlp_fit_scaling(sos_mlp* net, const float* Y, int32_t rows) {
  if (!net || !Y || rows < 1) return mfail(SOS_ERR_INVALID_ARG, "sos_mlp_fit_scaling: bad arguments");
  k_colstats<<<(net->n_out + 255) / 256, 256, 0, net->s>>>(Y, rows, net->n_out, net->mu, net->sd);
  MCK(cudaGetLastError());
  MCK(cudaStreamSynchronize(net->s));
  return SOS_OK;
}

int sos_mlp_gradients(sos_mlp* net, const float* X, const float* Y, int32_t batch, double* loss, float* grad_host) {
  if (!net || !X || !Y || batch < 1) return mfail(SOS_ERR_INVALID_ARG, "sos_mlp_gradients: bad arguments");
  int rc;
  if ((rc = ensure_batch(net, batch)) || (rc = forward(net, X, batch)) || (rc = backward(net, X, Y, batch, loss)))
    return rc;
  if (grad_host) MCK(cudaMemcpyAsync(grad_host, net->grad, sizeof(float) * net->n_param, cudaMemcpyDeviceToHost, net->s));
  MCK(cudaStreamSynchronize(net->s));
  return check_err(net);
}

int sos_mlp_train_step(sos_mlp* net, const float* X, const float* Y, int32_t batch, float lr, double* loss) {
  if (!net || !X || !Y || batch < 1 || !(lr > 0)) return mfail(SOS_ERR_INVALID_ARG, "sos_mlp_train_step: bad arguments");
  int rc;
  if ((rc = ensure_batch(net, batch)) || (rc = forward(net, X, batch)) || (rc = backward(net, X, Y, batch, loss)))
    return rc;
  net->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, static_cast<float>(net->step)), c2 = 1.f - std::pow(b2, static_cast<float>(net->step));
  k_adam<<<512, 256, 0, net->s>>>(net->param, net->grad, net->m, net->v, net->n_param, lr, b1, b2, 1e-8f, c1, c2);
  MCK(cudaGetLastError());
  return loss ? check_err(net) : SOS_OK;
}

int sos_mlp_predict(sos_mlp* net, const float* X, float* Y, int32_t batch) {
  if (!net || !X || !Y || batch < 1) return mfail(SOS_ERR_INVALID_ARG, "sos_mlp_predict: bad arguments");
  int rc;
  if ((rc = ensure_batch(net, batch)) || (rc = forward(net, X, batch))) return rc;
  MCK(cudaMemcpyAsync(Y, net->y, sizeof(float) * static_cast<size_t>(batch) * net->n_out, cudaMemcpyDeviceToDevice, net->s));
  k_unscale<<<256, 256, 0, net->s>>>(Y, net->mu, net->sd, batch, net->n_out);
  MCK(cudaGetLastError());
  MCK(cudaStreamSynchronize(net->s));
  return check_err(net);
}

}  // extern "C"
