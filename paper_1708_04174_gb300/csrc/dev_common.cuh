// Device helpers shared by the kernel translation units of libsos:
// deterministic block reductions, the projection input of a Gram entry,
// the packed (svec) index and the bounded grid-wide barrier of the
// cooperative kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace sos {
namespace {


__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum; result valid in every thread.
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (w == 0) {
    double x = (l < nw) ? sh[l] : 0.0;
    x = warp_sum(x);
    if (l == 0) sh[32] = x;
  }
  __syncthreads();
  return sh[32];
}

// Block maximum (inputs >= 0); result valid in every thread.
__device__ double block_max(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (w == 0) {
    double x = (l < nw) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (l == 0) sh[32] = x;
  }
  __syncthreads();
  return sh[32];
}

template <typename T>
__device__ __forceinline__ double d(T x) {
  return static_cast<double>(x);
}

// Input of the PSD projection for packed entry e of block bd:
//   plain:    W_e = u_e + a_e u_hat_2[row(e)]
//   weighted: W_e = u_e + z_j - s g_j      (j = low-rank column of e)
template <typename T>
__device__ __forceinline__ T proj_input(const DevPlan<T>& p, const BlockDesc& bd, int64_t k, bool off, double s) {
  const int64_t e = bd.x_off + k;
  if (bd.kind == kRaw) return p.ux[e];
  if (bd.kind == kPlain) {
    const int row = p.ent_row[e] & ~kEntOffBit;
    const T a = off ? static_cast<T>(kSqrt2) : static_cast<T>(1);
    return p.ux[e] + a * p.uh2[row];
  }
  const int j = bd.lr_first + static_cast<int>(k);
  return static_cast<T>(d(p.ux[e]) + p.zlr[j] - s * p.lr_g[j]);
}

__device__ __forceinline__ int64_t packed_index(int i, int j, int N) {  // i >= j
  return static_cast<int64_t>(j) * N - static_cast<int64_t>(j) * (j - 1) / 2 + (i - j);
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* ptr) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ptr) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* ptr, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(ptr), "r"(v) : "memory");
}

// Grid-wide barrier.  bar[0] counts arrivals (zeroed before the launch),
// bar[1] holds the last released generation; the CTA that completes a
// generation releases it, the others poll bar[1].  Ordering comes from the
// atomics themselves, not from full fences: __syncthreads orders the CTA's
// writes before thread 0's arrival, the arrival is an acquire-release
// read-modify-write at GPU scope (so the last arriver acquires every earlier
// arrival), the release is a store-release and the pollers load-acquire it.
// Bounded spin (limit in clock cycles): on expiry (or when another CTA
// already raised the error word) every CTA returns false.
__device__ bool grid_barrier(unsigned* bar, unsigned target, int32_t* err, long long limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = target / gridDim.x;
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(bar) : "memory");
    int good = 1;
    if (old == target - 1) {
      st_release_u32(bar + 1, gen);
    } else {
      const long long t0 = clock64();
      while (ld_acquire_u32(bar + 1) < gen) {
        if (*reinterpret_cast<volatile int32_t*>(err) != 0) {
          good = 0;
          break;
        }
        if (clock64() - t0 > limit) {
          atomicExch(err, 1);
          good = 0;
          break;
        }
      }
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

template <typename T>
__device__ __forceinline__ T ldg_cg(const T* ptr) {
  return __ldcg(ptr);
}
}  // namespace
}  // namespace sos
