// CUDA kernels of libsos for sm_103a (GB300).
//
// One ADMM iteration (eq. (20)) on a batch of instances is:
//
//   k_rows_r      r = w2hat - A w1hat, x = P^{-1} r           (eq. (27b), Appendix)
//   k_lr_y        y = A_L^T x                                  (Appendix)
//   k_woodbury    z = (L L^T)^{-1} y with the cached factor     (eq. (28))
//   k_rows_sigma2 sigma_2 = x - P^{-1} A_L z                    (Appendix)
//   k_inst_scalar Sherman-Morrison scalar, u_hat_3, tau/kappa,
//                 free variables                                (eq. (24b), (25), (20b-c))
//   k_rows_y      u_hat_2 = sigma_2 - s h_2; y-part of (20b-c)
//   k_psd_*       Gram blocks: W = u_hat_1 - v, u = P_S+(W),
//                 v = u - W                                     (eq. (20b-c))
//
// Identities used to avoid extra passes (exact in exact arithmetic):
//   A_L^T sigma_2 = z            (since (I + A_L^T P^{-1} A_L) z = A_L^T P^{-1} r)
//   u_hat_1 = w1hat - s c + A^T u_hat_2, and for a plain Gram entry
//   W_e = u_hat_1,e - v_e = u_e + a_e u_hat_2[row(e)].
#include <cuda_bf16.h>

#include <algorithm>
#include <cfloat>
#include <cstdio>

#include "dev_common.cuh"
#include "kernels.h"
#include "tcgen05.cuh"

namespace sos {
namespace {


// ---------------------------------------------------------------------------
// affine step
// ---------------------------------------------------------------------------

// r = w2_hat - A w1_hat and x = P^-1 r for every row (eq. (27b)).  Rows are
// walked one per thread through the sliced lists (a warp's 32 rows read
// element k of each row from 32 consecutive words), and the low-rank part
// uses w1_hat of each column, stored once per iteration in wl: one FP64
// multiply-add per A_L nonzero.  The row index must advance in whole warps.
template <typename T>
__device__ void d_rows_r(const DevPlan<T>& p, int64_t g0, int64_t stride) {
  for (int64_t a = g0; a < p.M; a += stride) {
    const int i = p.row_inst[a];
    if (!p.active[i]) continue;
    const double om3 = p.tau[i] + p.kappa[i];
    double acc = d(p.uy[a]) + d(p.vy[a]) + p.b[a] * om3;  // w2hat
    const int64_t sl = a >> 5;
    const int lane = static_cast<int>(a & 31);
    const int ne = p.row_ptr[a + 1] - p.row_ptr[a];
    const uint32_t* ent = p.ent_sl + p.ent_sl_off[sl] + lane;
#pragma unroll 4
    for (int k = 0; k < ne; ++k) {
      const uint32_t v = __ldcs(ent + 32 * k);  // read once: streaming load
      const uint32_t e = v & ~kOffDiagBit;
      const double w = d(p.ux[e]) + d(p.vx[e]);
      const double wt = (v & kOffDiagBit) ? kSqrt2 : 1.0;  // selected, not multiplied
      acc = fma(-wt, w, acc);                              // two FP64 operations per entry
    }
    const int nl = p.lrr_ptr[a + 1] - p.lrr_ptr[a];
    const int64_t lb = p.lr_sl_off[sl] + lane;
#pragma unroll 4
    for (int k = 0; k < nl; ++k) acc -= __ldcs(p.lr_sl_val + lb + 32 * k) * p.wl[__ldcs(p.lr_sl_col + lb + 32 * k)];
    p.xP[a] = acc * p.pinv[a];
  }
}

template <typename T>
__global__ void k_rows_r(DevPlan<T> p) {
  d_rows_r(p, static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x, static_cast<int64_t>(gridDim.x) * blockDim.x);
}

// y = A_L^T x (eq. (28)), eight lanes per column: four columns per warp,
// lanes striding over a column's nonzeros, a three-step shuffle reduction.
template <typename T>
__device__ void d_lr_y(const DevPlan<T>& p, int warp, int nwarps) {
  const int lane = threadIdx.x & 31, sub = lane & 7, grp = lane >> 3;
  for (int j0 = warp * 4; j0 < p.TL; j0 += nwarps * 4) {  // warp-uniform loop
    const int jq = j0 + grp;
    const int j = jq < p.TL ? p.col_perm[jq] : 0;  // columns of similar length share a warp
    const bool on = jq < p.TL && p.active[p.lr_inst[j]];
    double acc = 0.0;
    if (on) {
      const int k1 = p.lr_ptr[j + 1];
#pragma unroll 4
      for (int k = p.lr_ptr[j] + sub; k < k1; k += 8) acc += __ldcs(p.lr_val + k) * p.xP[__ldcs(p.lr_row + k)];
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (on && sub == 0) p.ylr[j] = acc;
  }
}

template <typename T>
__global__ void k_lr_y(DevPlan<T> p) {
  d_lr_y(p, (blockIdx.x * blockDim.x + threadIdx.x) >> 5, (gridDim.x * blockDim.x) >> 5);
}

// z = L^{-T} L^{-1} y per instance (one CTA per instance).
template <typename T>
__device__ void d_woodbury(const DevPlan<T>& p, int i, double* sh) {
  if (!p.active[i]) return;
  const InstInfo in = p.inst[i];
  const int te = in.t_eff;
  if (te == 0) return;
  double* y = sh;
  double* q = sh + te;
  const double* Li = p.linv + in.linv_off;
  for (int k = threadIdx.x; k < te; k += blockDim.x) y[k] = p.ylr[in.lr_off + k];
  __syncthreads();
  const double* Lt = p.linv_t + in.linv_off;  // the same matrix, column-major
  for (int r = threadIdx.x; r < te; r += blockDim.x) {  // q = L^{-1} y, one thread per row
    double acc = 0.0;
#pragma unroll 4
    for (int k = 0; k <= r; ++k) acc += Lt[static_cast<int64_t>(k) * te + r] * y[k];  // coalesced across rows
    q[r] = acc;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < te + 31; j += blockDim.x) {  // z = L^{-T} q, one thread per column;
    const int r0 = j & ~31;  // the lanes of a warp walk the same rows together (coalesced row reads)
    double acc = 0.0;
    for (int r = r0; r < te; ++r)
      if (j < te && r >= j) acc += Li[static_cast<int64_t>(r) * te + j] * q[r];
    if (j < te) p.zlr[in.lr_off + j] = acc;
  }
}

template <typename T>
__global__ void k_woodbury(DevPlan<T> p) {
  extern __shared__ double shw[];
  d_woodbury(p, blockIdx.x, shw);
}

// The same two triangular products for a single instance with a wide core,
// spread over the GPU: every row of L^{-1} (first pass) or of L^{-T} (second
// pass, the rows of the column-major copy) is one warp's dot product, its
// lanes striding along the row (coalesced) with four independent partial
// sums, then a warp reduction.  The first pass writes q = L^{-1} y to wq.
template <typename T>
__global__ void __launch_bounds__(256) k_woodbury_wide(DevPlan<T> p, int pass) {
  if (!p.active[0]) return;
  const InstInfo in = p.inst[0];
  const int te = in.t_eff;
  const int lane = threadIdx.x & 31;
  const int nw = static_cast<int>((static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5);
  const double* x = (pass == 0 ? p.ylr : p.wq) + in.lr_off;
  for (int r = static_cast<int>((static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5); r < te;
       r += nw) {
    // pass 0: sum_{k <= r} Li[r][k] y[k]; pass 1: sum_{k >= r} Li[k][r] q[k] = sum_k Lt[r][k] q[k]
    const double* row = (pass == 0 ? p.linv : p.linv_t) + in.linv_off + static_cast<int64_t>(r) * te;
    const int k0 = pass == 0 ? 0 : r, k1 = pass == 0 ? r + 1 : te;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int k = k0 + lane;
    for (; k + 96 < k1; k += 128) {
      a0 = fma(row[k], x[k], a0);
      a1 = fma(row[k + 32], x[k + 32], a1);
      a2 = fma(row[k + 64], x[k + 64], a2);
      a3 = fma(row[k + 96], x[k + 96], a3);
    }
    for (; k < k1; k += 32) a0 = fma(row[k], x[k], a0);
    const double acc = warp_sum((a0 + a1) + (a2 + a3));
    if (lane == 0) {
      if (pass == 0)
        p.wq[in.lr_off + r] = acc;
      else
        p.zlr[in.lr_off + r] = acc;
    }
  }
}

template <typename T>
void launch_woodbury(const DevPlan<T>& p, cudaStream_t s) {
  if (woodbury_wide(p.n_inst, p.max_teff)) {
    const int grid = (p.max_teff + 7) / 8;  // one warp per row
    k_woodbury_wide<T><<<grid, 256, 0, s>>>(p, 0);
    k_woodbury_wide<T><<<grid, 256, 0, s>>>(p, 1);
    return;
  }
  const size_t wsm = sizeof(double) * 2 * static_cast<size_t>(p.max_teff > 0 ? p.max_teff : 1);
  k_woodbury<T><<<p.n_inst, 256, wsm, s>>>(p);
}

template <typename T>
__device__ void d_rows_sigma2(const DevPlan<T>& p, int64_t g0, int64_t stride) {
  for (int64_t a = g0; a < p.M; a += stride) {  // rows advance in whole warps
    if (!p.active[p.row_inst[a]]) continue;
    double acc = 0.0;
    const int nl = p.lrr_ptr[a + 1] - p.lrr_ptr[a];
    const int64_t lb = p.lr_sl_off[a >> 5] + (a & 31);
#pragma unroll 4
    for (int k = 0; k < nl; ++k) acc += __ldcs(p.lr_sl_val + lb + 32 * k) * p.zlr[__ldcs(p.lr_sl_col + lb + 32 * k)];
    p.sig2[a] = p.xP[a] - acc * p.pinv[a];
  }
}

template <typename T>
__global__ void k_rows_sigma2(DevPlan<T> p) {
  d_rows_sigma2(p, static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x, static_cast<int64_t>(gridDim.x) * blockDim.x);
}

// Per instance: b^T sigma_2, c^T sigma_1, Sherman-Morrison coefficient,
// u_hat_3, the tau/kappa update and the free variables.
template <typename T>
__device__ void d_inst_scalar(const DevPlan<T>& p, int i) {
  __shared__ double sh[40];
  if (!p.active[i]) return;
  const InstInfo in = p.inst[i];
  const double tau = p.tau[i], kappa = p.kappa[i];
  const double om3 = tau + kappa;
  double bs = 0.0;
#pragma unroll 4
  for (int a = threadIdx.x; a < in.m; a += blockDim.x) bs += p.b[in.y_off + a] * p.sig2[in.y_off + a];
  const double bsig2 = block_sum(bs, sh);
  double cs = 0.0;
  for (int j = threadIdx.x; j < in.t; j += blockDim.x) {
    const int jl = in.lr_off + j;
    const double w = p.lr_c[jl];
    cs += w * (p.wl[jl] + p.zlr[jl]);  // c^T sigma_1, sigma_1 = w1hat + A^T sigma_2 = w1hat + z
  }
  const double csig1 = block_sum(cs, sh);
  const double zs = csig1 - bsig2;                 // zeta^T sigma
  const double s = zs / (1.0 + in.zeta_h);         // eq. (25)
  const double uh3 = om3 + zs - s * in.zeta_h;     // eq. (24b): w3 + c^T u1 - b^T u2
  const double tn = fmax(uh3 - kappa, 0.0);
  const double kn = kappa - uh3 + tn;
  for (int j = threadIdx.x; j < in.t; j += blockDim.x) {
    const int jl = in.lr_off + j;
    const double w = p.lr_c[jl];
    const int64_t e = in.x_off + j;
    const double wv = d(p.ux[e]) - w * (om3 + s) + p.zlr[jl] - s * p.lr_g[jl];
    const T un = static_cast<T>(wv);
    p.ux[e] = un;                // free: projection is the identity
    p.vx[e] = static_cast<T>(0);  // dual of a free variable is 0
    p.wl[jl] = d(un) - w * (tn + kn);  // w1_hat of the next iteration
  }
  if (threadIdx.x == 0) {
    p.tau[i] = tn;
    p.kappa[i] = kn;
    p.st[i].s = s;
    p.st[i].omega3 = om3;
    p.st[i].cs1 = csig1;
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_inst_scalar(DevPlan<T> p) {
  d_inst_scalar(p, blockIdx.x);
}

// A single instance gets a whole 1024-thread CTA for its reductions over m.
template <typename T>
int inst_scalar_threads(const DevPlan<T>& p, const LaunchShape& ls) {
  return p.n_inst == 1 ? 1024 : ls.inst_threads;
}

template <typename T>
__device__ void d_rows_y(const DevPlan<T>& p, int64_t g0, int64_t stride) {
  for (int64_t a = g0; a < p.M; a += stride) {
    const int i = p.row_inst[a];
    if (!p.active[i]) continue;
    const double uh2 = p.sig2[a] - p.st[i].s * p.h2[a];
    const double vy = d(p.vy[a]);
    const double un = uh2 - vy;
    p.uy[a] = static_cast<T>(un);
    p.vy[a] = static_cast<T>((vy - uh2) + un);
    p.uh2[a] = static_cast<T>(uh2);
  }
}

template <typename T>
__global__ void k_rows_y(DevPlan<T> p) {
  d_rows_y(p, static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x, static_cast<int64_t>(gridDim.x) * blockDim.x);
}


// Round-robin (circle method) pairing: pair k of round r, for Np even.
// q = x / d, r = x % d for 0 <= x < 2^24 without an integer division: the
// float estimate is off by at most one and is corrected exactly.
__device__ __forceinline__ void divmod_small(int x, int d, float invd, int& q, int& r) {
  q = __float2int_rz(static_cast<float>(x) * invd);
  r = x - q * d;
  if (r >= d) {
    ++q;
    r -= d;
  } else if (r < 0) {
    --q;
    r += d;
  }
}

__device__ __forceinline__ void rr_pair(int k, int r, int Np, int& a, int& b) {
  const int m1 = Np - 1;
  a = (k == 0) ? 0 : 1 + (k - 1 + r) % m1;
  b = 1 + (Np - 2 - k + r) % m1;
  if (a > b) {
    const int t = a;
    a = b;
    b = t;
  }
}

template <typename T>
__device__ __forceinline__ T rsqrt2() {
  return static_cast<T>(0.70710678118654752440);
}

template <typename T>
__device__ __forceinline__ T teps();
template <>
__device__ __forceinline__ double teps<double>() {
  return DBL_EPSILON;
}
template <>
__device__ __forceinline__ float teps<float>() {
  return FLT_EPSILON;
}

// Rutishauser's rotation zeroing a_pq: a'_pp = a_pp - t a_pq, a'_qq = a_qq + t a_pq.
template <typename T>
__device__ __forceinline__ void jacobi_rot(T app, T aqq, T apq, T& c, T& s, T& t) {
  const T theta = (aqq - app) / (static_cast<T>(2) * apq);
  const T at = fabs(theta);
  T tt;
  if (at > static_cast<T>(1e150) && sizeof(T) == 8)
    tt = static_cast<T>(0.5) / theta;
  else if (at > static_cast<T>(1e18) && sizeof(T) == 4)
    tt = static_cast<T>(0.5) / theta;
  else
    tt = static_cast<T>(1) / (at + sqrt(theta * theta + static_cast<T>(1)));
  if (theta < 0) tt = -tt;
  c = static_cast<T>(1) / sqrt(tt * tt + static_cast<T>(1));
  s = tt * c;
  t = tt;
}

// ---------------------------------------------------------------------------
// PSD projection, small blocks: one CTA per block, cyclic Jacobi in shared
// memory with the round-robin parallel ordering.  Each round applies Np/2
// disjoint rotations as 2x2-block updates of A = J^T A J and column updates
// V = V J.  A sweep without any rotation above eps |W|_F ends the solve.
// T is the storage type of the iterates, TC the compute type.
// Warm start: the eigenvectors of the previous iteration (kept per block,
// re-orthonormalised by one Newton-Schulz step V (3 I - V^T V) / 2 before
// they are stored) give B = V^T W V, nearly diagonal after the first
// iterations, so few sweeps remain.
// ---------------------------------------------------------------------------
// Row i >= column j of lower-triangle entry t = i (i + 1) / 2 + j.
__device__ __forceinline__ void lower_ij(int t, int& i, int& j) {
  i = static_cast<int>((sqrtf(8.0f * static_cast<float>(t) + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= t) ++i;  // integer correction of the float estimate
  while (i * (i + 1) / 2 > t) --i;
  j = t - i * (i + 1) / 2;
}

// Compensated FP32 dot-product step (Ogita, Rump & Oishi, "Accurate sum and
// dot product", 2005): s + c accumulates a*b with the product split exactly
// by an FMA (a*b = p + e) and the sum split exactly by TwoSum (s + p = t + r).
// The intrinsics keep the compiler from contracting the error-free steps.
// The result is as accurate as if computed in twice the working precision:
// error <= eps |sum| + O(n eps^2) sum |a_k b_k|.
__device__ __forceinline__ void dot2_step(float a, float b, float& s, float& c) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  const float r = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s = t;
  c = __fadd_rn(c, __fadd_rn(r, e));
}

// Refinement of an FP32 Jacobi projection (FP64 iterates, FP32 projections).
// An FP32 Jacobi solve accumulates one rounding error per rotation in V and
// in the rotated matrix, so V V^T - I and the backward error reach
// ~1e-5 |W| after a few hundred rotations per column, and ADMM runs that need
// thousands of iterations stall near a 1e-3 residual.  One correction step
// restores FP32 accuracy (~1e-7 |W|):
//   F  = V^T V - I                     (compensated sums)
//   V' = V (I - F / 2)                 (orthonormal to O(|F|^2 + eps))
//   B  = V'^T W V'                     (W as an FP32 pair hi + lo, compensated sums)
//   M  = diag(max(b_ii, 0)) + G o offdiag(B),
//        g_ij = (max(b_ii,0) - max(b_jj,0)) / (b_ii - b_jj)
//   U  = V' M V'^T                     (FP32)
// M is P_S+(B) to first order in offdiag(B) (the derivative of the
// eigenvalue map x -> max(x, 0) at a diagonal matrix: g_ij = 1 when both
// Ritz values are positive, 0 when neither is, and in (0, 1) across zero).
// The products that need more than FP32 use the compensated dot product
// above (2 N^3 steps of ~10 FP32 operations), not FP64: FP64 runs at under
// 2% of the FP32 rate on GB300.  On entry V holds the Jacobi
// eigenvectors; on exit A holds V'.  The pair copy of W and then W V' live
// where V and T1 were (2 Np ld floats >= 2 N^2); M is held in registers
// until W V' is dead and then written where T1 was, so the refinement needs
// no shared memory beyond the Jacobi's three buffers.
template <typename T, typename TC>
__device__ void psd_small_refine(const DevPlan<T>& p, const BlockDesc& bd, double s_sm, int N, int ld, TC* A, TC* V,
                                 TC* T1, double* lam64) {
  static_assert(sizeof(TC) == 4, "the refinement works on FP32 data");
  const int tid = threadIdx.x, nt = blockDim.x;
  __syncthreads();
  for (int q = tid; q < N * N; q += nt) {  // T1 = F (lower and mirrored)
    const int i = q / N, j = q - i * N;
    if (i < j) continue;
    float sh = 0.f, c = 0.f;
    for (int k = 0; k < N; ++k) dot2_step(V[k * ld + i], V[k * ld + j], sh, c);
    if (i == j) sh = __fsub_rn(sh, 1.0f);  // exact: sh lies in [1/2, 2]
    const TC f = __fadd_rn(sh, c);
    T1[i * ld + j] = f;
    T1[j * ld + i] = f;
  }
  __syncthreads();
  for (int q = tid; q < N * N; q += nt) {  // A = V' = V - V F / 2
    const int i = q / N, j = q - i * N;
    TC acc = 0;
    for (int k = 0; k < N; ++k) acc += V[i * ld + k] * T1[k * ld + j];
    A[i * ld + j] = V[i * ld + j] - static_cast<TC>(0.5) * acc;
  }
  __syncthreads();
  float2* W2 = reinterpret_cast<float2*>(V);  // W as (hi, lo), row-major, leading dimension N
  for (int q = tid; q < N * N; q += nt) {
    const int i = q / N, j = q - i * N;
    if (i < j) continue;
    const double w = d(proj_input(p, bd, packed_index(i, j, N), i != j, s_sm));
    const double x = (i == j) ? w : w * 0.70710678118654752440;
    const float hi = static_cast<float>(x);
    const float2 v2 = make_float2(hi, static_cast<float>(x - static_cast<double>(hi)));
    W2[i * N + j] = v2;
    W2[j * N + i] = v2;
  }
  __syncthreads();
  // W2 <- W V' in place, a chunk of rows at a time: each thread computes a
  // 4-row x 1-column tile of the chunk and holds it across the barrier
  const int groups = nt / N > 0 ? nt / N : 1;
  for (int r0 = 0; r0 < N; r0 += 4 * groups) {
    const int g = tid / N, j = tid - g * N;
    const bool act = g < groups && r0 + 4 * g < N;
    float sh[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    if (act) {
      const int i0 = r0 + 4 * g;
      for (int k = 0; k < N; ++k) {
        const float v = A[k * ld + j];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          if (i0 + t < N) {
            const float2 w = W2[(i0 + t) * N + k];
            dot2_step(w.x, v, sh[t], c[t]);
            c[t] = __fmaf_rn(w.y, v, c[t]);
          }
        }
      }
    }
    __syncthreads();
    if (act) {
      const int i0 = r0 + 4 * g;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (i0 + t < N) {
          const float hi = __fadd_rn(sh[t], c[t]);
          W2[(i0 + t) * N + j] = make_float2(hi, __fadd_rn(__fsub_rn(sh[t], hi), c[t]));
        }
      }
    }
    __syncthreads();
  }
  for (int i = tid; i < N; i += nt) {  // Ritz values b_ii
    float sh = 0.f, c = 0.f;
    for (int k = 0; k < N; ++k) {
      const float v = A[k * ld + i];
      const float2 t2 = W2[k * N + i];
      dot2_step(v, t2.x, sh, c);
      c = __fmaf_rn(v, t2.y, c);
    }
    lam64[i] = static_cast<double>(sh) + static_cast<double>(c);
  }
  __syncthreads();
  // M, one lower-triangle entry t = i (i + 1) / 2 + j per thread and slot,
  // held in registers until W V' is dead, then written where T1 was
  constexpr int kMaxLower = 25;  // ceil(112 * 113 / 2 / 256): N <= 112 with 256 threads
  const int L = N * (N + 1) / 2;
  if (L > kMaxLower * nt) {  // uniform: the size classes keep N <= 112
    if (tid == 0) atomicExch(p.err, 3);
    return;
  }
  float mreg[kMaxLower];
#pragma unroll
  for (int r = 0; r < kMaxLower; ++r) {
    const int t = tid + r * nt;
    mreg[r] = 0.f;
    if (t < L) {
      int i, j;
      lower_ij(t, i, j);
      const double li = lam64[i], lj = lam64[j];
      double m;
      if (i == j) {
        m = fmax(li, 0.0);
      } else {
        double g;
        if (li > 0.0 && lj > 0.0)
          g = 1.0;
        else if (li <= 0.0 && lj <= 0.0)
          g = 0.0;
        else
          g = (fmax(li, 0.0) - fmax(lj, 0.0)) / (li - lj);  // one of them > 0 >= the other: |li - lj| > 0
        m = 0.0;
        if (g != 0.0) {
          float sh = 0.f, c = 0.f;
          for (int k = 0; k < N; ++k) {
            const float v = A[k * ld + i];
            const float2 t2 = W2[k * N + j];
            dot2_step(v, t2.x, sh, c);
            c = __fmaf_rn(v, t2.y, c);
          }
          m = g * (static_cast<double>(sh) + static_cast<double>(c));
        }
      }
      mreg[r] = static_cast<float>(m);
    }
  }
  __syncthreads();  // W V' is dead from here
#pragma unroll
  for (int r = 0; r < kMaxLower; ++r) {
    const int t = tid + r * nt;
    if (t < L) {
      int i, j;
      lower_ij(t, i, j);
      T1[i * ld + j] = mreg[r];
      T1[j * ld + i] = mreg[r];
    }
  }
  __syncthreads();
  for (int q = tid; q < N * N; q += nt) {  // V region (as TC) = Y = V' M
    const int i = q / N, j = q - i * N;
    TC acc = 0;
    for (int k = 0; k < N; ++k) acc += A[i * ld + k] * T1[k * ld + j];
    V[i * ld + j] = acc;
  }
  __syncthreads();
  for (int q = tid; q < N * N; q += nt) {  // U = Y V'^T; outputs u = svec(U), v = u - W
    const int i = q / N, j = q - i * N;
    if (i < j) continue;
    TC u = 0;
    for (int k = 0; k < N; ++k) u += V[i * ld + k] * A[j * ld + k];
    const int64_t kk = packed_index(i, j, N);
    const T w = proj_input(p, bd, kk, i != j, s_sm);
    const T uu = (i != j) ? static_cast<T>(d(u) * kSqrt2) : static_cast<T>(u);
    p.ux[bd.x_off + kk] = uu;
    const T vv = uu - w;
    p.vx[bd.x_off + kk] = vv;
    if (bd.kind == kWeighted) p.wl[bd.lr_first + kk] = d(uu) + d(vv);  // w1_hat of the next iteration (c = 0)
  }
}

template <typename T, typename TC>
__device__ void d_psd_small(const DevPlan<T>& p, int bid, const SmallWarm<TC>& wm, unsigned char* smraw) {
  __shared__ double red[40];
  __shared__ int last_rot;  // index of the last round that had a rotation
  const BlockDesc bd = p.blocks[bid];
  if (!p.active[bd.inst]) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) last_rot = -1;  // block_sum below orders this before any use
  const double s_sm = p.st[bd.inst].s;
  const int N = bd.N, Np = N + (N & 1), ld = Np + 1, H = Np / 2;
  constexpr bool kRefine = sizeof(T) == 8 && sizeof(TC) == 4;  // FP64 iterates, FP32 projections
  TC* A = reinterpret_cast<TC*>(smraw);
  TC* V = A + Np * ld;
  TC* T1 = V + Np * ld;
  double* lam64 = reinterpret_cast<double*>(T1 + Np * ld);  // refinement only: Ritz values
  TC* rc = kRefine ? reinterpret_cast<TC*>(lam64 + Np) : T1 + Np * ld;
  TC* rs = rc + H;
  TC* rt = rs + H;
  TC* lam = rt + H;
  int* rp = reinterpret_cast<int*>(lam + Np);
  int* rq = rp + H;
  TC* gV = (wm.V != nullptr && bd.v_off >= 0) ? wm.V + bd.v_off : nullptr;
  const int wc = gV ? wm.count[bid] : 0;
  const bool warm = wc > 0 && wc < wm.limit;

  double nrm = 0.0;
  for (int q = tid; q < Np * Np; q += nt) {
    const int i = q / Np, j = q - i * Np;
    if (i >= N || j >= N) {
      A[i * ld + j] = static_cast<TC>(0);
      V[i * ld + j] = (i == j) ? static_cast<TC>(1) : static_cast<TC>(0);
      continue;
    }
    V[i * ld + j] = warm ? gV[i * N + j] : ((i == j) ? static_cast<TC>(1) : static_cast<TC>(0));
    if (i < j) continue;
    const T w = proj_input(p, bd, packed_index(i, j, N), i != j, s_sm);
    nrm += d(w) * d(w);
    const TC a = (i == j) ? static_cast<TC>(w) : static_cast<TC>(d(w) * 0.70710678118654752440);
    A[i * ld + j] = a;
    A[j * ld + i] = a;
  }
  // FP64: sweeps stop below 1e-10 |W|_F and the reconstruction corrects
  // for the remaining off-diagonal to first order.  FP32 with the refinement
  // (mixed form): stop below 4 eps |W|_F, the refinement's first-order
  // correction absorbs the rest (same ~1e-7 |W| result, one sweep fewer);
  // plain FP32: to the roundoff.
  const TC thr = static_cast<TC>(sqrt(block_sum(nrm, red))) *
                 (sizeof(TC) == 8 ? static_cast<TC>(1e-10) : (kRefine ? 4 * teps<TC>() : teps<TC>()));
  if (warm) {
    for (int q = tid; q < N * N; q += nt) {  // T1 = W V
      const int i = q / N, j = q - i * N;
      TC acc = 0;
      for (int k = 0; k < N; ++k) acc += A[i * ld + k] * V[k * ld + j];
      T1[i * ld + j] = acc;
    }
    __syncthreads();
    for (int q = tid; q < N * N; q += nt) {  // A = V^T T1, lower triangle mirrored
      const int i = q / N, j = q - i * N;
      if (i < j) continue;
      TC acc = 0;
      for (int k = 0; k < N; ++k) acc += V[k * ld + i] * T1[k * ld + j];
      A[i * ld + j] = acc;
      A[j * ld + i] = acc;
    }
    __syncthreads();
  }

  int sweeps_done = 0;
  int round_id = 0;
  const float invH1 = 1.0f / static_cast<float>(H + 1);
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    bool rotated = false;
    sweeps_done = sweep + 1;
    for (int r = 0; r < Np - 1; ++r, ++round_id) {
      for (int k = tid; k < H; k += nt) {
        int a, b;
        rr_pair(k, r, Np, a, b);
        TC c = 1, s = 0, t = 0;
        if (b < N) {
          const TC apq = A[a * ld + b];
          if (fabs(apq) > thr) {
            jacobi_rot(A[a * ld + a], A[b * ld + b], apq, c, s, t);
            last_rot = round_id;
          }
        }
        rp[k] = a;
        rq[k] = b;
        rc[k] = c;
        rs[k] = s;
        rt[k] = t;
      }
      __syncthreads();
      if (last_rot != round_id) continue;  // no rotation this round (uniform)
      rotated = true;
      // A <- J^T A J as 2x2-block tasks; V <- V J as (pair, row group)
      // tasks: each loads its rotation once and walks the rows g, g + G, ...
      // (consecutive threads on consecutive rows: odd ld, no bank conflicts)
      // the H (H + 1) / 2 pair combinations k1 <= k2 are enumerated with
      // rows r and H - 1 - r paired (H + 1 combinations per paired row)
      const int nblk = H * (H + 1) / 2;
      const int G = nt / H > 1 ? nt / H : 1;  // row groups per pair
      for (int task = tid; task < nblk + G * H; task += nt) {
        if (task < nblk) {
          int rr, cc, k1, k2;
          divmod_small(task, H + 1, invH1, rr, cc);
          if (cc < H - rr) {
            k1 = rr;
            k2 = rr + cc;
          } else {
            k1 = H - 1 - rr;
            k2 = k1 + cc - (H - rr);
          }
          const int p1 = rp[k1], q1 = rq[k1], p2 = rp[k2], q2 = rq[k2];
          const TC c1 = rc[k1], s1 = rs[k1];
          if (k1 == k2) {
            if (s1 != static_cast<TC>(0)) {
              const TC apq = A[p1 * ld + q1], t1 = rt[k1];
              A[p1 * ld + p1] -= t1 * apq;
              A[q1 * ld + q1] += t1 * apq;
              A[p1 * ld + q1] = static_cast<TC>(0);
              A[q1 * ld + p1] = static_cast<TC>(0);
            }
            continue;
          }
          const TC c2 = rc[k2], s2 = rs[k2];
          if (s1 == static_cast<TC>(0) && s2 == static_cast<TC>(0)) continue;
          const TC x11 = A[p1 * ld + p2], x12 = A[p1 * ld + q2], x21 = A[q1 * ld + p2], x22 = A[q1 * ld + q2];
          const TC y11 = c1 * x11 - s1 * x21, y12 = c1 * x12 - s1 * x22;
          const TC y21 = s1 * x11 + c1 * x21, y22 = s1 * x12 + c1 * x22;
          const TC z11 = c2 * y11 - s2 * y12, z12 = s2 * y11 + c2 * y12;
          const TC z21 = c2 * y21 - s2 * y22, z22 = s2 * y21 + c2 * y22;
          A[p1 * ld + p2] = z11;
          A[p1 * ld + q2] = z12;
          A[q1 * ld + p2] = z21;
          A[q1 * ld + q2] = z22;
          A[p2 * ld + p1] = z11;
          A[q2 * ld + p1] = z12;
          A[p2 * ld + q1] = z21;
          A[q2 * ld + q1] = z22;
        } else {
          int k, g;
          divmod_small(task - nblk, G, 1.0f / static_cast<float>(G), k, g);
          const TC s = rs[k];
          if (s == static_cast<TC>(0)) continue;
          const TC c = rc[k];
          const int pp = rp[k], qq = rq[k];
          for (int row = g; row < N; row += G) {
            const TC vp = V[row * ld + pp], vq = V[row * ld + qq];
            V[row * ld + pp] = c * vp - s * vq;
            V[row * ld + qq] = s * vp + c * vq;
          }
        }
      }
      __syncthreads();
    }
    if (!rotated) break;
  }

  if (tid == 0) p.blk_sweeps[bid] = sweeps_done;
  if constexpr (kRefine) {
    psd_small_refine(p, bd, s_sm, N, ld, A, V, T1, lam64);
    if (gV) {  // keep the re-orthonormalised V' for the next iteration
      for (int q = tid; q < N * N; q += nt) {
        const int i = q / N, j = q - i * N;
        gV[i * N + j] = A[i * ld + j];
      }
      if (tid == 0) wm.count[bid] = warm ? wc + 1 : 1;
    }
  } else {
  // P_S+(W) = V max(Lambda, 0) V^T; v = u - W (in the storage type).  FP64:
  // V M V^T with M = diag(max(b_kk, 0)) + G o offdiag(B), the first-order
  // projection of the nearly diagonal B (T1 = V M first).
  for (int k = tid; k < N; k += nt) lam[k] = fmax(A[k * ld + k], static_cast<TC>(0));
  __syncthreads();
  if constexpr (sizeof(TC) == 8) {
    TC* bdiag = rc;  // rc, rs, rt are contiguous: 3 H >= N entries, free after the sweeps
    for (int k = tid; k < N; k += nt) bdiag[k] = A[k * ld + k];
    __syncthreads();
    for (int q = tid; q < N * N; q += nt) {  // A <- M in place (each entry from itself and the diagonal)
      const int l = q / N, k = q - l * N;
      const TC bl = bdiag[l], bk = bdiag[k];
      TC m;
      if (l == k)
        m = lam[k];
      else if (bl > 0 && bk > 0)
        m = A[l * ld + k];
      else if (bl <= 0 && bk <= 0)
        m = 0;
      else
        m = (lam[l] - lam[k]) / (bl - bk) * A[l * ld + k];  // |bl - bk| > 0 here
      A[l * ld + k] = m;
    }
    __syncthreads();
    for (int q = tid; q < N * N; q += nt) {  // T1 = V M
      const int i = q / N, k = q - i * N;
      TC acc = 0;
      for (int l = 0; l < N; ++l) acc += V[i * ld + l] * A[l * ld + k];
      T1[i * ld + k] = acc;
    }
    __syncthreads();
  }
  for (int q = tid; q < N * N; q += nt) {
    const int i = q / N, j = q - i * N;
    if (i < j) continue;
    TC u = 0;
    if constexpr (sizeof(TC) == 8) {
      for (int k = 0; k < N; ++k) u += T1[i * ld + k] * V[j * ld + k];
    } else {
      for (int k = 0; k < N; ++k) u += V[i * ld + k] * lam[k] * V[j * ld + k];
    }
    const int64_t kk = packed_index(i, j, N);
    const T w = proj_input(p, bd, kk, i != j, s_sm);
    const T uu = (i != j) ? static_cast<T>(d(u) * kSqrt2) : static_cast<T>(u);
    p.ux[bd.x_off + kk] = uu;
    const T vv = uu - w;
    p.vx[bd.x_off + kk] = vv;
    if (bd.kind == kWeighted) p.wl[bd.lr_first + kk] = d(uu) + d(vv);  // w1_hat of the next iteration (c = 0)
  }
  if (gV) {  // keep V for the next iteration: V (3 I - V^T V) / 2
    __syncthreads();  // T1 may still be read by the reconstruction above
    for (int q = tid; q < N * N; q += nt) {
      const int i = q / N, j = q - i * N;
      TC acc = 0;
      for (int k = 0; k < N; ++k) acc += V[k * ld + i] * V[k * ld + j];
      T1[i * ld + j] = ((i == j) ? static_cast<TC>(1.5) : static_cast<TC>(0)) - static_cast<TC>(0.5) * acc;
    }
    __syncthreads();
    for (int q = tid; q < N * N; q += nt) {
      const int i = q / N, j = q - i * N;
      TC acc = 0;
      for (int k = 0; k < N; ++k) acc += V[i * ld + k] * T1[k * ld + j];
      gV[i * N + j] = acc;
    }
    if (tid == 0) wm.count[bid] = warm ? wc + 1 : 1;
  }
  }
}

template <typename T, typename TC>
__global__ void __launch_bounds__(512) k_psd_small(DevPlan<T> p, const int32_t* ids, SmallWarm<TC> wm) {
  extern __shared__ __align__(16) unsigned char smraw[];
  d_psd_small(p, ids[blockIdx.x], wm, smraw);
}

// ---------------------------------------------------------------------------
// PSD projection, large blocks: one cooperative grid per block.  Same Jacobi
// as above with the matrix in global memory (L2 resident), warm-started
// from the previous iteration's eigenvectors V: B = V^T W V, then sweeps on
// B (double buffered; each round's rotations are recomputed by every task
// from the current buffer), then U = V max(diag B, 0) V^T.
// ---------------------------------------------------------------------------


// C tile (16x16, 256 threads) of one of:
//   mode 0: C = A B           mode 1: C = A^T B        (A, B: Np x Np, ld Np)
template <typename T>
__device__ T tile_mm(const T* A, const T* B, int Np, int ti, int tj, int mode, T* sA, T* sB) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i = ti * 16 + ty, j = tj * 16 + tx;
  T acc = 0;
  for (int k0 = 0; k0 < Np; k0 += 16) {
    {
      const int r = ty, k = tx;  // element (r, k) of the A tile and (k=ty, c=tx) of the B tile
      const int gi = ti * 16 + r, gk = k0 + k;
      T av = 0;
      if (gi < Np && gk < Np) av = (mode == 0) ? ldg_cg(A + static_cast<int64_t>(gi) * Np + gk)
                                               : ldg_cg(A + static_cast<int64_t>(gk) * Np + gi);
      sA[r * 17 + k] = av;
      const int bk = k0 + ty, bj = tj * 16 + tx;
      sB[ty * 17 + tx] = (bk < Np && bj < Np) ? ldg_cg(B + static_cast<int64_t>(bk) * Np + bj) : static_cast<T>(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc += sA[ty * 17 + k] * sB[k * 17 + tx];
    __syncthreads();
  }
  (void)i;
  (void)j;
  return acc;
}

template <typename T, typename TC>
__global__ void __launch_bounds__(256, 1) k_psd_large(DevPlan<T> p, int bid, LargeScratch<TC> L) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double red[40];
  __shared__ TC sA[16 * 17], sB[16 * 17];
  __shared__ int any_rot;
  const BlockDesc bd = p.blocks[bid];
  if (!p.active[bd.inst]) return;
  if (sizeof(TC) == 8 && sizeof(T) == 8 && tri_path(bd.N) && __ldcg(L.flags) == 1) return;  // projected already
  if (threadIdx.x == 0) any_rot = -1;  // the load phase's block_sum orders this before any use
  const double s_sm = p.st[bd.inst].s;
  const int N = bd.N, Np = N + (N & 1), H = Np / 2;
  const int64_t gt = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t gs = static_cast<int64_t>(gridDim.x) * blockDim.x;
  unsigned gen = 0;
  const unsigned G = gridDim.x;
  int32_t* err = p.err;
  const int warm_count = __ldcg(L.warm);
  const bool warm = warm_count > 0 && warm_count < L.warm_limit;
  TC* Wf = L.Wf;
  TC* V = L.V;

  // load W (full symmetric, svec unscaled), norm, V = I when cold
  double nrm = 0.0;
  for (int64_t q = gt; q < static_cast<int64_t>(Np) * Np; q += gs) {
    const int i = static_cast<int>(q / Np), j = static_cast<int>(q - static_cast<int64_t>(i) * Np);
    if (!warm) V[q] = (i == j) ? static_cast<TC>(1) : static_cast<TC>(0);
    if (i >= N || j >= N) {
      Wf[q] = static_cast<TC>(0);
      continue;
    }
    const int ii = i >= j ? i : j, jj = i >= j ? j : i;
    const T w = proj_input(p, bd, packed_index(ii, jj, N), ii != jj, s_sm);
    if (i >= j) nrm += d(w) * d(w);
    Wf[q] = (i == j) ? static_cast<TC>(w) : static_cast<TC>(d(w) * 0.70710678118654752440);
  }
  const double part = block_sum(nrm, red);
  if (threadIdx.x == 0) L.partial[blockIdx.x] = part;
  if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
  double tot = 0.0;
  for (unsigned c = 0; c < G; ++c) tot += __ldcg(L.partial + c);
  // FP64: the sweeps stop once every off-diagonal entry is below
  // 1e-10 |W|_F and the reconstruction corrects for the rest to first order
  // (second-order error <= |E|^2 / gap, and never above |E|); FP32 sweeps run
  // to the unit roundoff.
  const TC thr = static_cast<TC>(sqrt(tot)) * (sizeof(TC) == 8 ? static_cast<TC>(1e-10) : teps<TC>());

  const int nt = (Np + 15) / 16;
  TC* cur = Wf;
  if (warm) {
    for (int tile = blockIdx.x; tile < nt * nt; tile += G) {  // T1 = W V
      const int ti = tile / nt, tj = tile - ti * nt;
      const TC v = tile_mm(Wf, V, Np, ti, tj, 0, sA, sB);
      const int i = ti * 16 + (threadIdx.x >> 4), j = tj * 16 + (threadIdx.x & 15);
      if (i < Np && j < Np) L.T1[static_cast<int64_t>(i) * Np + j] = v;
    }
    if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
    for (int tile = blockIdx.x; tile < nt * nt; tile += G) {  // B = V^T T1 (lower tiles, mirrored)
      const int ti = tile / nt, tj = tile - ti * nt;
      if (ti < tj) continue;
      const TC v = tile_mm(V, L.T1, Np, ti, tj, 1, sA, sB);
      const int i = ti * 16 + (threadIdx.x >> 4), j = tj * 16 + (threadIdx.x & 15);
      if (i < Np && j < Np && i >= j) {
        Wf[static_cast<int64_t>(i) * Np + j] = v;
        Wf[static_cast<int64_t>(j) * Np + i] = v;
      }
    }
    if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
  }

  // Jacobi sweeps, double buffered (cur -> nxt).  Every CTA computes all
  // rotations of a round into shared memory from cur, so all CTAs take the
  // same decisions: a round without rotations writes nothing and is skipped
  // without a barrier, and the sweep loop ends everywhere at once.  Reads of
  // cur never race with writes, which only go to nxt.
  TC* nxt = L.B0;
  TC* rc = reinterpret_cast<TC*>(dsm);
  TC* rs = rc + H;
  TC* rt = rs + H;
  int* rp = reinterpret_cast<int*>(rt + H);
  int* rq = rp + H;
  int sweeps = 0;
  int round_id = 0;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    bool sweep_rot = false;
    sweeps = sweep + 1;
    {
      // A sweep in which no off-diagonal entry exceeds thr rotates nothing
      // and leaves the matrix as it is: one grid-wide maximum decides that
      // up front (the same value in every CTA) instead of N - 1 rounds of
      // rotation parameters.  The partial maxima alternate between two
      // buffers: check k + 2 cannot overwrite check k's partials before
      // every CTA has passed check k + 1's barrier.
      TC mx = 0;
      for (int64_t q = gt; q < static_cast<int64_t>(N) * Np; q += gs) {
        const int i = static_cast<int>(q / Np), j = static_cast<int>(q - static_cast<int64_t>(i) * Np);
        if (j > i && j < N) mx = fmax(mx, fabs(ldg_cg(cur + q)));
      }
      const double bm = block_max(d(mx), red);
      double* part = L.partial + static_cast<int64_t>(1 + (sweep & 1)) * G;
      if (threadIdx.x == 0) part[blockIdx.x] = bm;
      if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
      double gv = 0.0;
      for (unsigned c = threadIdx.x; c < G; c += blockDim.x) gv = fmax(gv, __ldcg(part + c));
      const double gm = block_max(gv, red);
      if (!(gm > d(thr))) break;
    }
    for (int r = 0; r < Np - 1; ++r, ++round_id) {
      for (int k = threadIdx.x; k < H; k += blockDim.x) {
        int a, b;
        rr_pair(k, r, Np, a, b);
        TC c = 1, s = 0, t = 0;
        if (b < N) {
          const TC apq = ldg_cg(cur + static_cast<int64_t>(a) * Np + b);
          if (fabs(apq) > thr) {
            jacobi_rot(ldg_cg(cur + static_cast<int64_t>(a) * Np + a), ldg_cg(cur + static_cast<int64_t>(b) * Np + b), apq,
                       c, s, t);
            any_rot = round_id;
          }
        }
        rp[k] = a;
        rq[k] = b;
        rc[k] = c;
        rs[k] = s;
        rt[k] = t;
      }
      __syncthreads();
      if (any_rot != round_id) continue;  // same decision in every CTA
      sweep_rot = true;
      // 2x2 tasks over pairs k1 <= k2 only (numbered k2 (k2 + 1) / 2 + k1),
      // then N x H row tasks of V: on 152 CTAs of 256 threads at most one task
      // per thread up to N = 248
      const int64_t nblk = static_cast<int64_t>(H) * (H + 1) / 2;
      for (int64_t task = gt; task < nblk + static_cast<int64_t>(N) * H; task += gs) {
        if (task < nblk) {
          int k2 = static_cast<int>((sqrtf(8.0f * static_cast<float>(task) + 1.0f) - 1.0f) * 0.5f);
          while (k2 > 0 && static_cast<int64_t>(k2) * (k2 + 1) / 2 > task) --k2;
          while (k2 < H - 1 && static_cast<int64_t>(k2 + 1) * (k2 + 2) / 2 <= task) ++k2;
          const int k1 = static_cast<int>(task - static_cast<int64_t>(k2) * (k2 + 1) / 2);
          const int p1 = rp[k1], q1 = rq[k1], p2 = rp[k2], q2 = rq[k2];
          const TC c1 = rc[k1], s1 = rs[k1], c2 = rc[k2], s2 = rs[k2];
          if (k1 == k2) {
            const TC a1 = ldg_cg(cur + static_cast<int64_t>(p1) * Np + q1);
            const TC app = ldg_cg(cur + static_cast<int64_t>(p1) * Np + p1);
            const TC aqq = ldg_cg(cur + static_cast<int64_t>(q1) * Np + q1);
            if (s1 != static_cast<TC>(0)) {
              const TC t1 = rt[k1];
              nxt[static_cast<int64_t>(p1) * Np + p1] = app - t1 * a1;
              nxt[static_cast<int64_t>(q1) * Np + q1] = aqq + t1 * a1;
              nxt[static_cast<int64_t>(p1) * Np + q1] = static_cast<TC>(0);
              nxt[static_cast<int64_t>(q1) * Np + p1] = static_cast<TC>(0);
            } else {
              nxt[static_cast<int64_t>(p1) * Np + p1] = app;
              nxt[static_cast<int64_t>(q1) * Np + q1] = aqq;
              nxt[static_cast<int64_t>(p1) * Np + q1] = a1;
              nxt[static_cast<int64_t>(q1) * Np + p1] = a1;
            }
            continue;
          }
          const TC x11 = ldg_cg(cur + static_cast<int64_t>(p1) * Np + p2);
          const TC x12 = ldg_cg(cur + static_cast<int64_t>(p1) * Np + q2);
          const TC x21 = ldg_cg(cur + static_cast<int64_t>(q1) * Np + p2);
          const TC x22 = ldg_cg(cur + static_cast<int64_t>(q1) * Np + q2);
          const TC y11 = c1 * x11 - s1 * x21, y12 = c1 * x12 - s1 * x22;
          const TC y21 = s1 * x11 + c1 * x21, y22 = s1 * x12 + c1 * x22;
          const TC z11 = c2 * y11 - s2 * y12, z12 = s2 * y11 + c2 * y12;
          const TC z21 = c2 * y21 - s2 * y22, z22 = s2 * y21 + c2 * y22;
          nxt[static_cast<int64_t>(p1) * Np + p2] = z11;
          nxt[static_cast<int64_t>(p1) * Np + q2] = z12;
          nxt[static_cast<int64_t>(q1) * Np + p2] = z21;
          nxt[static_cast<int64_t>(q1) * Np + q2] = z22;
          nxt[static_cast<int64_t>(p2) * Np + p1] = z11;
          nxt[static_cast<int64_t>(q2) * Np + p1] = z12;
          nxt[static_cast<int64_t>(p2) * Np + q1] = z21;
          nxt[static_cast<int64_t>(q2) * Np + q1] = z22;
        } else {
          const int64_t t2i = task - nblk;
          const int row = static_cast<int>(t2i / H), k = static_cast<int>(t2i - static_cast<int64_t>(row) * H);
          const TC s = rs[k];
          if (s == static_cast<TC>(0)) continue;
          const TC c = rc[k];
          const int pp = rp[k], qq = rq[k];
          TC* vr = V + static_cast<int64_t>(row) * Np;
          const TC vp = ldg_cg(vr + pp), vq = ldg_cg(vr + qq);
          vr[pp] = c * vp - s * vq;
          vr[qq] = s * vp + c * vq;
        }
      }
      if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
      TC* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
    if (!sweep_rot) break;
  }

  const int ntl = (N + 15) / 16;
  if constexpr (sizeof(TC) == 8) {
    // U = V M V^T with M = diag(max(b_kk, 0)) + G o offdiag(B): the first-order
    // projection of the nearly diagonal B (the derivative of the eigenvalue
    // map max(., 0) at diag(B); g_lk = 1 when both diagonal entries are
    // positive, 0 when neither is, in (0, 1) across zero).  M into B1 (free
    // in FP64), then T1 = V M.
    for (int64_t q = gt; q < static_cast<int64_t>(Np) * Np; q += gs) {
      const int l = static_cast<int>(q / Np), k = static_cast<int>(q - static_cast<int64_t>(l) * Np);
      TC m = 0;
      if (l < N && k < N) {
        const TC bl = ldg_cg(cur + static_cast<int64_t>(l) * Np + l), bk = ldg_cg(cur + static_cast<int64_t>(k) * Np + k);
        if (l == k)
          m = fmax(bl, static_cast<TC>(0));
        else if (bl > 0 && bk > 0)
          m = ldg_cg(cur + q);
        else if (bl <= 0 && bk <= 0)
          m = 0;
        else
          m = (fmax(bl, static_cast<TC>(0)) - fmax(bk, static_cast<TC>(0))) / (bl - bk) * ldg_cg(cur + q);  // |bl - bk| > 0
      }
      L.B1[q] = m;
    }
    if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
    for (int tile = blockIdx.x; tile < nt * nt; tile += G) {
      const int ti = tile / nt, tj = tile - ti * nt;
      const TC v = tile_mm(V, L.B1, Np, ti, tj, 0, sA, sB);
      const int i = ti * 16 + (threadIdx.x >> 4), j = tj * 16 + (threadIdx.x & 15);
      if (i < Np && j < Np) L.T1[static_cast<int64_t>(i) * Np + j] = v;
    }
    if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
  }
  // U = (V M or V max(diag B, 0)) V^T on lower tiles; write u and v = u - W
  for (int tile = blockIdx.x; tile < ntl * ntl; tile += G) {
    const int ti = tile / ntl, tj = tile - ti * ntl;
    if (ti < tj) continue;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i = ti * 16 + ty, j = tj * 16 + tx;
    TC acc = 0;
    for (int k0 = 0; k0 < N; k0 += 16) {
      const int gk = k0 + tx;
      const int ri = ti * 16 + ty, rj = tj * 16 + ty;
      if constexpr (sizeof(TC) == 8) {
        sA[ty * 17 + tx] = (ri < N && gk < N) ? ldg_cg(L.T1 + static_cast<int64_t>(ri) * Np + gk) : static_cast<TC>(0);
      } else {
        TC lk = 0;
        if (gk < N) lk = fmax(ldg_cg(cur + static_cast<int64_t>(gk) * Np + gk), static_cast<TC>(0));
        sA[ty * 17 + tx] = (ri < N && gk < N) ? ldg_cg(V + static_cast<int64_t>(ri) * Np + gk) * lk : static_cast<TC>(0);
      }
      sB[ty * 17 + tx] = (rj < N && gk < N) ? ldg_cg(V + static_cast<int64_t>(rj) * Np + gk) : static_cast<TC>(0);
      __syncthreads();
#pragma unroll
      for (int k = 0; k < 16; ++k) acc += sA[ty * 17 + k] * sB[tx * 17 + k];
      __syncthreads();
    }
    if (i < N && j < N && i >= j) {
      const int64_t kk = packed_index(i, j, N);
      const T w = proj_input(p, bd, kk, i != j, s_sm);
      const T u = (i != j) ? static_cast<T>(d(acc) * kSqrt2) : static_cast<T>(acc);
      p.ux[bd.x_off + kk] = u;
      const T vv = u - w;
      p.vx[bd.x_off + kk] = vv;
      if (bd.kind == kWeighted) p.wl[bd.lr_first + kk] = d(u) + d(vv);  // w1_hat of the next iteration (c = 0)
    }
  }
  if (sizeof(TC) < 8) {  // FP32 eigenvectors: V <- V (3 I - V^T V) / 2 before they are kept
    if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
    for (int tile = blockIdx.x; tile < nt * nt; tile += G) {
      const int ti = tile / nt, tj = tile - ti * nt;
      const TC v = tile_mm(V, V, Np, ti, tj, 1, sA, sB);
      const int i = ti * 16 + (threadIdx.x >> 4), j = tj * 16 + (threadIdx.x & 15);
      if (i < Np && j < Np)
        L.T1[static_cast<int64_t>(i) * Np + j] = ((i == j) ? static_cast<TC>(1.5) : static_cast<TC>(0)) - static_cast<TC>(0.5) * v;
    }
    if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
    for (int tile = blockIdx.x; tile < nt * nt; tile += G) {
      const int ti = tile / nt, tj = tile - ti * nt;
      const TC v = tile_mm(V, L.T1, Np, ti, tj, 0, sA, sB);
      const int i = ti * 16 + (threadIdx.x >> 4), j = tj * 16 + (threadIdx.x & 15);
      if (i < Np && j < Np) L.B1[static_cast<int64_t>(i) * Np + j] = v;
    }
    if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
    for (int64_t q = gt; q < static_cast<int64_t>(Np) * Np; q += gs) V[q] = __ldcg(L.B1 + q);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *L.sweeps_out = sweeps;
    p.blk_sweeps[bid] = sweeps;
    *L.warm = warm ? warm_count + 1 : 1;
  }
}

// ---------------------------------------------------------------------------
// PSD projection of large blocks on the tensor cores (FP32-compute forms).
// P_S+(W) = (W + W sign(W)) / 2, sign(W) by the Newton-Schulz iteration
// X <- (3 X - X^3) / 2 from X_0 = W / |W|_F (Higham, Functions of Matrices,
// ch. 5).  Every product is a tcgen05.mma GEMM: BF16 operands split into a
// high and a low part (x = x_hi + x_lo, so X Y ~ X_hi Y_hi + X_hi Y_lo +
// X_lo Y_hi) with FP32 accumulation in tensor memory.  The iterates are
// symmetric polynomials of W, so each CTA computes one 128 x 64 tile of the
// lower triangle (using rows of both operands, K-major) and writes it and its
// mirror.  Operands are staged from L2 into shared memory in the no-swizzle
// core-matrix layout (8 rows x 16 bytes per core matrix).
// ---------------------------------------------------------------------------


constexpr int kNsTM = 128, kNsTN = 64, kNsKC = 64, kNsStages = 3;
constexpr uint32_t kNsStrip = 8 * kNsKC * 2;                      // bytes of an 8-row strip of a K chunk
constexpr uint32_t kNsABytes = kNsTM * kNsKC * 2;                  // one BF16 part of an A chunk
constexpr uint32_t kNsBBytes = kNsTN * kNsKC * 2;                  // one BF16 part of a B chunk
constexpr uint32_t kNsStageBytes = 3 * (kNsABytes + kNsBBytes);    // three parts of both chunks
constexpr size_t kNsSmem = static_cast<size_t>(kNsStages) * kNsStageBytes;

// The split operand layout of an Np x Np matrix (Np a multiple of 128),
// three parts of BF16 (x = x_hi + x_mid + x_lo, each the rounding of what the
// previous parts leave): part q, K chunk kc (kNsKC columns), row group rg (8
// rows) is one strip of kNsStrip bytes in the no-swizzle K-major
// core-matrix layout (core matrix (rg, k/8) at byte (k % kNsKC / 8) * 128,
// row r % 8 at + 16 (r % 8)), strips ordered [q][kc][rg].  The A chunk of rows m0 .. m0 + 127 (or the B
// chunk of rows n0 .. n0 + 63) of chunk kc is then one contiguous range, and
// a stage of the product pipeline is six bulk copies.
__device__ __forceinline__ size_t ns_strip(int Np, int q, int kc, int rg) {
  return (static_cast<size_t>(q) * (Np / kNsKC) + kc) * (Np / 8) + rg;
}

__device__ __forceinline__ void ns_split8(const float (&x)[8], uint4& h, uint4& m, uint4& l) {
  __nv_bfloat16 hh[8], mm[8], ll[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    hh[j] = __float2bfloat16_rn(x[j]);
    const float r1 = x[j] - __bfloat162float(hh[j]);
    mm[j] = __float2bfloat16_rn(r1);
    ll[j] = __float2bfloat16_rn(r1 - __bfloat162float(mm[j]));
  }
  h = *reinterpret_cast<const uint4*>(hh);
  m = *reinterpret_cast<const uint4*>(mm);
  l = *reinterpret_cast<const uint4*>(ll);
}

// Entries (r, c0 .. c0 + 7) of a matrix into its split layout (c0 % 8 == 0):
// one 16-byte core-matrix row per part.
__device__ __forceinline__ void ns_put8(unsigned char* S, int Np, int r, int c0, const float (&x)[8]) {
  uint4 h, m, l;
  ns_split8(x, h, m, l);
  const size_t o = ((c0 % kNsKC) >> 3) * 128 + (r & 7) * 16;
  *reinterpret_cast<uint4*>(S + ns_strip(Np, 0, c0 / kNsKC, r >> 3) * kNsStrip + o) = h;
  *reinterpret_cast<uint4*>(S + ns_strip(Np, 1, c0 / kNsKC, r >> 3) * kNsStrip + o) = m;
  *reinterpret_cast<uint4*>(S + ns_strip(Np, 2, c0 / kNsKC, r >> 3) * kNsStrip + o) = l;
}

// Entries (r, c0 + j), j < 8, of a symmetric matrix computed by this thread,
// those on or below the diagonal, to the split layout (and to the FP32 copy
// F when given).  Their mirrors are written by ns_put_mirror.
__device__ __forceinline__ void ns_put_lower(unsigned char* S, float* F, int Np, int r, int c0, const float (&x)[8]) {
  if (c0 + 7 <= r) {  // the whole group on or below the diagonal
    ns_put8(S, Np, r, c0, x);
    if (F) {
      float4* dst = reinterpret_cast<float4*>(F + static_cast<int64_t>(r) * Np + c0);
      dst[0] = make_float4(x[0], x[1], x[2], x[3]);
      dst[1] = make_float4(x[4], x[5], x[6], x[7]);
    }
  } else if (c0 <= r) {  // straddles the diagonal: entries c0 .. r only
    uint4 h, m, l;
    ns_split8(x, h, m, l);
    const uint16_t* ph = reinterpret_cast<const uint16_t*>(&h);
    const uint16_t* pm = reinterpret_cast<const uint16_t*>(&m);
    const uint16_t* pl = reinterpret_cast<const uint16_t*>(&l);
    const size_t o = ((c0 % kNsKC) >> 3) * 128 + (r & 7) * 16;
    for (int j = 0; j <= r - c0; ++j) {
      reinterpret_cast<uint16_t*>(S + ns_strip(Np, 0, c0 / kNsKC, r >> 3) * kNsStrip + o)[j] = ph[j];
      reinterpret_cast<uint16_t*>(S + ns_strip(Np, 1, c0 / kNsKC, r >> 3) * kNsStrip + o)[j] = pm[j];
      reinterpret_cast<uint16_t*>(S + ns_strip(Np, 2, c0 / kNsKC, r >> 3) * kNsStrip + o)[j] = pl[j];
      if (F) F[static_cast<int64_t>(r) * Np + c0 + j] = x[j];
    }
  }
}

// Mirrors of the strictly-lower entries of this CTA's 128 x 64 tile (rows
// m0.., columns n0..), staged in shared memory T[128][65] by the epilogue:
// entry (c, r) = T[r - m0][c - n0] for r > c, written as rows c of the
// split layout (eight consecutive r per 16-byte store) and of F.  Each entry
// of the lower triangle is computed by exactly one CTA, so the stored matrix
// is exactly symmetric (the iteration doubles any antisymmetric part once
// X^T X is near I).  Call with the whole CTA after a barrier that made T
// visible.
__device__ __forceinline__ void ns_put_mirror(unsigned char* S, float* F, int Np, int m0, int n0, const float* T) {
  for (int g = threadIdx.x; g < kNsTN * (kNsTM / 8); g += blockDim.x) {
    const int cl = g % kNsTN, rg = g / kNsTN;  // consecutive threads: consecutive columns (no bank conflicts)
    const int c = n0 + cl, r0 = m0 + 8 * rg;
    if (r0 + 7 <= c) continue;  // no entry of the group below the diagonal
    float x[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) x[t] = T[(8 * rg + t) * (kNsTN + 1) + cl];
    if (r0 > c) {  // all eight strictly below
      ns_put8(S, Np, c, r0, x);
      if (F) {
        float4* dst = reinterpret_cast<float4*>(F + static_cast<int64_t>(c) * Np + r0);
        dst[0] = make_float4(x[0], x[1], x[2], x[3]);
        dst[1] = make_float4(x[4], x[5], x[6], x[7]);
      }
    } else {
      uint4 h, m, l;
      ns_split8(x, h, m, l);
      const uint16_t* pp[3] = {reinterpret_cast<const uint16_t*>(&h), reinterpret_cast<const uint16_t*>(&m),
                               reinterpret_cast<const uint16_t*>(&l)};
      const size_t o = ((r0 % kNsKC) >> 3) * 128 + (c & 7) * 16;
      for (int t = 0; t < 8; ++t) {
        if (r0 + t <= c) continue;
#pragma unroll
        for (int q = 0; q < 3; ++q)
          reinterpret_cast<uint16_t*>(S + ns_strip(Np, q, r0 / kNsKC, c >> 3) * kNsStrip + o)[t] = pp[q][t];
        if (F) F[static_cast<int64_t>(c) * Np + r0 + t] = x[t];
      }
    }
  }
}

// Pipeline state of the products of one CTA (thread 0 drives the copies and
// the MMAs; every thread waits on `done`).
struct NsPipe {
  uint64_t* full;   // [kNsStages] bulk copies of a stage landed
  uint64_t* empty;  // [kNsStages] MMAs that read a stage completed
  uint64_t* done;   // all MMAs of a product completed
  uint32_t fph[kNsStages], eph[kNsStages], dph;  // phases awaited next
  int epend[kNsStages];                           // a commit on empty[s] not yet waited for
  int fpend[kNsStages];                           // bulk copies into stage s not yet waited for
  uint32_t tmem;
  long long limit;  // bound of each wait, clock cycles
  bool ok;
};

// acc[128 x 64] (TMEM) = A[m0.., :] B[n0.., :]^T over k in [0, Np) from the
// split layouts, with the six products of the three-part split whose
// exponent sum is at most 2^-16.  kNsStages stages: thread 0 refills the
// stage of chunk kc - 1 with chunk kc - 1 + kNsStages once its MMAs have
// completed, while the MMAs of chunk kc run.  On return (every thread) the accumulator is ready,
// or P.ok is false after an expired wait.
__device__ void ns_gemm(const unsigned char* As, const unsigned char* Bs, int Np, int m0, int n0,
                        unsigned char* smem, NsPipe& P) {
  constexpr uint32_t LBO = 128, SBO = (kNsKC / 8) * 128;
  constexpr uint32_t idesc = tc::idesc_bf16(kNsTM, kNsTN);
  const int pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
  const int nk = Np / kNsKC;
  if (threadIdx.x == 0) {
    // the operands were written by generic stores of other CTAs before the
    // grid barrier this thread acquired: order that view before the bulk
    // copies (async proxy) that read them
    asm volatile("fence.proxy.async.global;" ::: "memory");
    auto load = [&](int kc) {
      const int s = kc % kNsStages;
      if (P.epend[s]) {  // the stage's previous chunk must be consumed
        if (P.ok) P.ok = tc::wait(P.empty + s, P.eph[s], P.limit);
        P.eph[s] ^= 1u;
        P.epend[s] = 0;
      }
      if (!P.ok) return;
      unsigned char* base = smem + s * kNsStageBytes;
      tc::arrive_expect_tx(P.full + s, kNsStageBytes);
      P.fpend[s] = 1;
      for (int q = 0; q < 3; ++q) {
        tc::bulk_g2s(base + q * kNsABytes, As + ns_strip(Np, q, kc, m0 / 8) * kNsStrip, kNsABytes, P.full + s);
        tc::bulk_g2s(base + 3 * kNsABytes + q * kNsBBytes, Bs + ns_strip(Np, q, kc, n0 / 8) * kNsStrip, kNsBBytes,
                     P.full + s);
      }
    };
    for (int kc = 0; kc < nk && kc < kNsStages; ++kc) load(kc);
    for (int kc = 0; kc < nk && P.ok; ++kc) {
      const int s = kc % kNsStages;
      P.ok = tc::wait(P.full + s, P.fph[s], P.limit);
      if (!P.ok) break;  // left pending: the kernel's cleanup waits for these copies once more
      P.fph[s] ^= 1u;
      P.fpend[s] = 0;
      tc::fence_after();
      unsigned char* base = smem + s * kNsStageBytes;
      for (int ks = 0; ks < kNsKC / 16; ++ks) {
        const uint32_t so = ks * 2 * LBO;
        for (int q = 0; q < 6; ++q) {
          const uint32_t acc = (kc > 0 || ks > 0 || q > 0) ? 1u : 0u;
          tc::mma(P.tmem, tc::desc(tc::smem_u32(base + pa[q] * kNsABytes) + so, LBO, SBO),
                  tc::desc(tc::smem_u32(base + 3 * kNsABytes + pb[q] * kNsBBytes) + so, LBO, SBO), idesc, acc);
        }
      }
      tc::commit(P.empty + s);
      P.epend[s] = 1;
      if (kc >= 1 && kc - 1 + kNsStages < nk) load(kc - 1 + kNsStages);
    }
    tc::commit(P.done);  // arrives once every MMA issued so far has completed
  }
  __syncthreads();
  const bool good = tc::wait(P.done, P.dph, P.limit);
  P.dph ^= 1u;
  // every commit on empty[] precedes the one on done: their phases have
  // completed too (thread 0's bookkeeping)
  if (threadIdx.x == 0)
    for (int s = 0; s < kNsStages; ++s)
      if (P.epend[s]) {
        P.eph[s] ^= 1u;
        P.epend[s] = 0;
      }
  tc::fence_after();
  const int bad = __syncthreads_or(!good || (threadIdx.x == 0 && !P.ok));
  P.ok = !bad;
}


__host__ __device__ __forceinline__ int ns_np(int N) { return (N + kNsTM - 1) / kNsTM * kNsTM; }
__host__ __device__ __forceinline__ int ns_tiles(int N) {
  const int nti = ns_np(N) / kNsTM;
  return nti * (nti + 1) * (kNsTM / kNsTN) / 2;
}

template <typename T>
__global__ void __launch_bounds__(256) k_psd_ns(DevPlan<T> p, int bid, NsScratch S) {
  extern __shared__ __align__(1024) unsigned char nsm[];
  __shared__ __align__(8) uint64_t mbar[2 * kNsStages + 1];
  __shared__ uint32_t tmem_base;
  __shared__ double red[40];
  const BlockDesc bd = p.blocks[bid];
  if (!p.active[bd.inst]) return;
  const double s_sm = p.st[bd.inst].s;
  const int N = bd.N, Np = ns_np(N);
  const unsigned G = gridDim.x;
  unsigned gen = 0;
  int32_t* err = p.err;
  const int64_t gt = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t gs = static_cast<int64_t>(G) * blockDim.x;
  // this CTA's lower tile: row tile ti holds column tiles 0 .. 2 ti + 1 (the
  // products are symmetric; the epilogues write each lower entry and its mirror)
  int ti = 0, rem = blockIdx.x;
  while (rem >= (ti + 1) * (kNsTM / kNsTN)) {
    rem -= (ti + 1) * (kNsTM / kNsTN);
    ++ti;
  }
  const int m0 = ti * kNsTM, n0 = rem * kNsTN;
  const size_t sb = ns_split_bytes(Np);
  unsigned char* Wsp = S.split;
  unsigned char* Xsp = S.split + sb;
  unsigned char* Xnsp = S.split + 2 * sb;
  unsigned char* Ysp = S.split + 3 * sb;

  NsPipe P;
  P.full = mbar;
  P.empty = mbar + kNsStages;
  P.done = mbar + 2 * kNsStages;
  for (int s = 0; s < kNsStages; ++s) {
    P.fph[s] = P.eph[s] = 0;
    P.epend[s] = P.fpend[s] = 0;
  }
  P.dph = 0;
  P.limit = p.wait_limit;
  P.ok = true;
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2 * kNsStages + 1; ++s) tc::mbar_init(mbar + s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_base)),
                 "r"(kNsTN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }

  bool alive = true;
  // the split layouts written by this CTA's threads become operands of bulk
  // copies (async proxy) in other CTAs after the barrier
#define NS_SYNC()                                                \
  do {                                                           \
    asm volatile("fence.proxy.async.global;" ::: "memory");     \
    tc::fence_before();                                          \
    alive = grid_barrier(S.bar, (++gen) * G, err, p.wait_limit); \
    tc::fence_after();                                           \
  } while (0)
  // W (unscaled, FP32, and split) and its Frobenius norm; groups of eight
  // consecutive columns
  double nrm = 0.0;
  const int gpr = Np / 8;  // groups per row
  for (int64_t g = gt; g < static_cast<int64_t>(Np) * gpr; g += gs) {
    const int i = static_cast<int>(g / gpr), c0 = static_cast<int>(g - static_cast<int64_t>(i) * gpr) * 8;
    float w8[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int j = c0 + t;
      float w = 0.f;
      if (i < N && j < N) {
        const int ii = i >= j ? i : j, jj = i >= j ? j : i;
        const T wv = proj_input(p, bd, packed_index(ii, jj, N), ii != jj, s_sm);
        if (i >= j) nrm += d(wv) * d(wv);
        w = (i == j) ? static_cast<float>(wv) : static_cast<float>(d(wv) * 0.70710678118654752440);
      }
      w8[t] = w;
    }
    float4* dst = reinterpret_cast<float4*>(S.Wf + static_cast<int64_t>(i) * Np + c0);
    dst[0] = make_float4(w8[0], w8[1], w8[2], w8[3]);
    dst[1] = make_float4(w8[4], w8[5], w8[6], w8[7]);
    ns_put8(Wsp, Np, i, c0, w8);
  }
  const double part = block_sum(nrm, red);
  if (threadIdx.x == 0) S.partial[blockIdx.x] = part;
  NS_SYNC();
  P.tmem = tmem_base;
  const int wq = (threadIdx.x >> 5) & 3;  // TMEM lane quarter of this warp
  const int chalf = (threadIdx.x >> 7);   // warps 4..7 take the upper 32 columns
  const int row = m0 + wq * 32 + (threadIdx.x & 31);
  // an epilogue stages its tile for the mirror writes in the product
  // pipeline's shared memory, which no copy targets between products
  float* tile = reinterpret_cast<float*>(nsm);
  int it = 0;
  float* X = S.X;
  float* Xn = S.Xn;
  if (alive) {
    double tot = 0.0;
    for (unsigned c = 0; c < G; ++c) tot += __ldcg(S.partial + c);
    const float inv = tot > 0.0 ? static_cast<float>(1.0 / sqrt(tot)) : 0.f;
    for (int64_t g = gt; g < static_cast<int64_t>(Np) * gpr; g += gs) {
      const int i = static_cast<int>(g / gpr), c0 = static_cast<int>(g - static_cast<int64_t>(i) * gpr) * 8;
      const float4* src = reinterpret_cast<const float4*>(S.Wf + static_cast<int64_t>(i) * Np + c0);
      const float4 a = __ldcg(src), b = __ldcg(src + 1);
      float x8[8] = {a.x * inv, a.y * inv, a.z * inv, a.w * inv, b.x * inv, b.y * inv, b.z * inv, b.w * inv};
      float4* dst = reinterpret_cast<float4*>(X + static_cast<int64_t>(i) * Np + c0);
      dst[0] = make_float4(x8[0], x8[1], x8[2], x8[3]);
      dst[1] = make_float4(x8[4], x8[5], x8[6], x8[7]);
      ns_put8(Xsp, Np, i, c0, x8);
    }
    NS_SYNC();

    // Plain Newton-Schulz, X <- (3 X - X^3) / 2: eigenvalues of X in (0, 1]
    // converge to sign(lambda) quadratically near 1 and grow by 1.5x per step
    // near 0.  The optimally scaled variant (step a-dependent, a > 1) sends
    // eigenvalues near 1 down to the current floor ell before they return; in
    // FP32 with split-BF16 products those lose their relative accuracy there and
    // the outer ADMM iteration stalls near a 2e-4 dual residual, so it is not used.
    // The first step alone is rescaled: |X|_2 <= c = |X^2|_F^(1/2) <= |X|_F = 1,
    // so X / c still has its eigenvalues in [-1, 1] and every one of them
    // starts a factor 1/c higher (c is about r^(-1/4) for r eigenvalues of
    // comparable size), which saves log_1.5(1/c) steps.
    float alpha = 1.5f, beta = 0.5f;
    for (it = 0; alive && it < S.max_iter; ++it) {
      // Y = X X
      ns_gemm(Xsp, Xsp, Np, m0, n0, nsm, P);
      if (!P.ok) break;
      float ysq = 0.f;
      for (int c0 = chalf * 32; c0 < chalf * 32 + 32; c0 += 8) {
        float v[8];
        tc::ld8(P.tmem + (static_cast<uint32_t>(wq * 32) << 16) + c0, v);
        ns_put_lower(Ysp, nullptr, Np, row, n0 + c0, v);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          tile[(row - m0) * (kNsTN + 1) + c0 + j] = v[j];
          const int col = n0 + c0 + j;
          if (row >= col) ysq = fmaf((row == col ? 1.f : 2.f) * v[j], v[j], ysq);
        }
      }
      __syncthreads();
      ns_put_mirror(Ysp, nullptr, Np, m0, n0, tile);
      if (it == 0) {
        const double py = block_sum(static_cast<double>(ysq), red);
        if (threadIdx.x == 0) S.partial[G + blockIdx.x] = py;
      }
      NS_SYNC();
      if (!alive) break;
      if (it == 0) {
        double ytot = 0.0;
        for (unsigned c = 0; c < G; ++c) ytot += __ldcg(S.partial + G + c);  // same order in every CTA
        const double c = sqrt(sqrt(ytot));
        if (c > 0.0 && c < 1.0) {
          alpha = static_cast<float>(1.5 / c);
          beta = static_cast<float>(0.5 / (c * c * c));
        }
      } else {
        alpha = 1.5f;
        beta = 0.5f;
      }
      // X_next = 1.5 X - 0.5 Y X, and |X_next - X|^2
      ns_gemm(Ysp, Xsp, Np, m0, n0, nsm, P);
      if (!P.ok) break;
      float dsq = 0.f;  // FP32: the FP64 pipe is 1/64 of the FP32 one here
      float4 xq[8];     // this thread's 32 entries of X, loaded together
#pragma unroll
      for (int q = 0; q < 8; ++q)
        xq[q] = __ldcg(reinterpret_cast<const float4*>(X + static_cast<int64_t>(row) * Np + n0 + chalf * 32) + q);
#pragma unroll
      for (int c0 = chalf * 32; c0 < chalf * 32 + 32; c0 += 8) {
        float v[8];
        tc::ld8(P.tmem + (static_cast<uint32_t>(wq * 32) << 16) + c0, v);
        const float4 a = xq[(c0 - chalf * 32) / 4], b = xq[(c0 - chalf * 32) / 4 + 1];
        const float x[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        float xn[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          xn[j] = alpha * x[j] - beta * v[j];
          const int col = n0 + c0 + j;
          const float df = xn[j] - x[j];
          if (row >= col) dsq = fmaf((row == col ? 1.f : 2.f) * df, df, dsq);
        }
        ns_put_lower(Xnsp, Xn, Np, row, n0 + c0, xn);
#pragma unroll
        for (int j = 0; j < 8; ++j) tile[(row - m0) * (kNsTN + 1) + c0 + j] = xn[j];
      }
      __syncthreads();
      ns_put_mirror(Xnsp, Xn, Np, m0, n0, tile);
      const double pd = block_sum(static_cast<double>(dsq), red);
      if (threadIdx.x == 0) S.partial[blockIdx.x] = pd;
      NS_SYNC();
      if (!alive) break;
      double dtot = 0.0;
      for (unsigned c = 0; c < G; ++c) dtot += __ldcg(S.partial + c);
      float* tmp = X;
      X = Xn;
      Xn = tmp;
      unsigned char* tsp = Xsp;
      Xsp = Xnsp;
      Xnsp = tsp;
      if (dtot <= static_cast<double>(S.tol) * S.tol * Np) {  // same decision in every CTA
        ++it;
        break;
      }
    }
  }
  // U = (W + W S) / 2 with S = sign(W) ~ X; outputs u = svec(U), v = u - W
  // (lower triangle: the tile entries with row >= col)
  if (alive && P.ok) ns_gemm(Wsp, Xsp, Np, m0, n0, nsm, P);
  if (alive && P.ok) {
    for (int c0 = chalf * 32; c0 < chalf * 32 + 32; c0 += 8) {
      float v[8];
      tc::ld8(P.tmem + (static_cast<uint32_t>(wq * 32) << 16) + c0, v);
      for (int j = 0; j < 8; ++j) {
        const int col = n0 + c0 + j;
        if (row >= col && row < N && col < N) {
          const float w = __ldcg(S.Wf + static_cast<int64_t>(row) * Np + col);
          const float u = 0.5f * (w + v[j]);
          const int64_t kk = packed_index(row, col, N);
          const T wv = proj_input(p, bd, kk, row != col, s_sm);
          const T uu = (row != col) ? static_cast<T>(static_cast<double>(u) * kSqrt2) : static_cast<T>(u);
          p.ux[bd.x_off + kk] = uu;
          const T vv = uu - wv;
          p.vx[bd.x_off + kk] = vv;
          if (bd.kind == kWeighted) p.wl[bd.lr_first + kk] = d(uu) + d(vv);  // w1_hat of the next iteration (c = 0)
        }
      }
    }
  }
#undef NS_SYNC
  // cleanup on every path: after a failed wait, MMAs still in flight get one
  // more bounded wait (on a fresh commit), then the tensor memory is released
  if (!P.ok) {
    if (threadIdx.x == 0) {
      for (int s = 0; s < kNsStages; ++s)
        if (P.fpend[s]) tc::wait(P.full + s, P.fph[s], P.limit);  // bulk copies still in flight
      tc::commit(P.done);
    }
    __syncthreads();
    tc::wait(P.done, P.dph, P.limit);
  }
  tc::fence_before();
  __syncthreads();
  if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(P.tmem), "r"(kNsTN));
  if (!P.ok && threadIdx.x == 0) atomicExch(err, 1);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *S.iters_out = it;
    p.blk_sweeps[bid] = it;
  }
}

// ---------------------------------------------------------------------------
// residuals (every k_check iterations)
// ---------------------------------------------------------------------------
template <typename T>
__device__ void d_res_rows(const DevPlan<T>& p, int64_t g0, int64_t stride) {
  for (int64_t a = g0; a < p.M; a += stride) {
    if (!p.active[p.row_inst[a]]) continue;
    double acc = 0.0;
    const int k1 = p.row_ptr[a + 1];
    for (int k = p.row_ptr[a]; k < k1; ++k) {
      const uint32_t v = p.row_ent[k];
      const double x = d(p.ux[v & ~kOffDiagBit]);
      acc += (v & kOffDiagBit) ? kSqrt2 * x : x;
    }
    const int l1 = p.lrr_ptr[a + 1];
    for (int k = p.lrr_ptr[a]; k < l1; ++k) acc += p.lrr_val[k] * d(p.ux[p.lr_ent[p.lrr_col[k]]]);
    p.ra[a] = acc;  // (A u_xi)_a
  }
}

template <typename T>
__global__ void k_res_rows(DevPlan<T> p) {
  d_res_rows(p, static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x, static_cast<int64_t>(gridDim.x) * blockDim.x);
}

template <typename T>
__device__ void d_res_lr(const DevPlan<T>& p, int warp, int nwarps) {
  const int lane = threadIdx.x & 31;
  for (int j = warp; j < p.TL; j += nwarps) {
    if (!p.active[p.lr_inst[j]]) continue;
    double acc = 0.0;
    const int k1 = p.lr_ptr[j + 1];
    for (int k = p.lr_ptr[j] + lane; k < k1; k += 32) acc += p.lr_val[k] * d(p.uy[p.lr_row[k]]);
    acc = warp_sum(acc);
    if (lane == 0) p.atyl[j] = acc;  // (A_L^T u_y)_j
  }
}

template <typename T>
__global__ void k_res_lr(DevPlan<T> p) {
  d_res_lr(p, (blockIdx.x * blockDim.x + threadIdx.x) >> 5, (gridDim.x * blockDim.x) >> 5);
}

template <typename T>
__device__ void d_res_inst(const DevPlan<T>& p, int i) {
  __shared__ double sh[40];
  if (!p.active[i]) return;
  const InstInfo in = p.inst[i];
  const double tau = p.tau[i];
  double pr = 0, ax = 0, by = 0, bad = 0;
  for (int a = threadIdx.x; a < in.m; a += blockDim.x) {
    const int64_t g = in.y_off + a;
    const double axv = p.ra[g];
    const double r = axv - p.b[g] * tau;
    pr += r * r;
    ax += axv * axv;
    const double uy = d(p.uy[g]);
    by += p.b[g] * uy;
    if (!isfinite(uy) || !isfinite(axv)) bad += 1.0;
  }
  double dr = 0, aty = 0, cx = 0;
  for (int k = threadIdx.x; k < in.nx; k += blockDim.x) {
    const int64_t e = in.x_off + k;
    const int er = p.ent_row[e];
    double at, c = 0.0;
    if (er >= 0) {  // plain Gram entry: one nonzero a_e (1 or sqrt 2) at its row
      const double u = d(p.uy[er & ~kEntOffBit]);
      at = (er & kEntOffBit) ? kSqrt2 * u : u;
    } else {  // low-rank column j
      const int j = -er - 1;
      at = p.atyl[j];
      c = p.lr_c[j];
    }
    const double vz = d(p.vx[e]);
    const double ux = d(p.ux[e]);
    if (!isfinite(vz) || !isfinite(ux)) bad += 1.0;
    const double q = at + vz;
    dr += (q - c * tau) * (q - c * tau);
    aty += q * q;
    cx += c * ux;
  }
  const double spr = block_sum(pr, sh), sax = block_sum(ax, sh), sby = block_sum(by, sh);
  const double sdr = block_sum(dr, sh), saty = block_sum(aty, sh), scx = block_sum(cx, sh);
  const double sbad = block_sum(bad, sh);
  if (threadIdx.x == 0) {
    InstResid R;
    R.tau = tau;
    R.kappa = p.kappa[i];
    R.pr2 = spr;
    R.ax2 = sax;
    R.by = sby;
    R.dr2 = sdr;
    R.aty2 = saty;
    R.cx = scx;
    R.nonfinite = sbad;
    p.resid[i] = R;
  }
}

template <typename T>
__global__ void k_res_inst(DevPlan<T> p) {
  d_res_inst(p, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Persistent batched solver: one cooperative launch runs many iterations of
// every instance.  The phases of an iteration are the device functions used
// by the per-kernel path, separated by grid barriers.  Every k_check
// iterations the residuals are reduced and each instance is checked on the
// device (same rule as sos_solve); a finished instance is frozen and the
// launch ends when none is running.  Gram blocks are handed to CTAs either
// round-robin over a fixed order (largest first) or from an atomic work queue.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void d_check(const DevPlan<T>& p, int i, int it, double tol, double infeas_tol, InstReport* rep, int32_t* active,
                        int32_t* n_active) {
  if (threadIdx.x != 0 || !active[i]) return;
  const InstInfo in = p.inst[i];
  const InstResid r = p.resid[i];
  InstReport R;
  R.rp = R.rd = R.gap = R.pobj = R.dobj = nan("");
  double res = INFINITY;
  if (r.tau > 1e-12 * (r.kappa + 1.0)) {
    R.rp = sqrt(r.pr2) / r.tau / (1.0 + in.norm_b);
    R.rd = sqrt(r.dr2) / r.tau / (1.0 + in.norm_c);
    R.pobj = r.cx / r.tau;
    R.dobj = r.by / r.tau;
    R.gap = fabs(R.pobj - R.dobj) / (1.0 + fabs(R.pobj) + fabs(R.dobj));
    res = fmax(R.rp, fmax(R.rd, R.gap));
  }
  const double pinf = r.by > 0 ? sqrt(r.aty2) / r.by : INFINITY;
  const double dinf = r.cx < 0 ? sqrt(r.ax2) / (-r.cx) : INFINITY;
  int st = 0;
  if (r.nonfinite > 0 || !isfinite(r.tau) || !isfinite(r.kappa))
    st = 5;  // NUMERICAL
  else if (res <= tol)
    st = 1;  // SOLVED
  else if (r.kappa > r.tau && pinf <= infeas_tol)  // certificates only while kappa > tau
    st = 2;  // PRIMAL_INFEASIBLE
  else if (r.kappa > r.tau && dinf <= infeas_tol)
    st = 3;  // DUAL_INFEASIBLE
  R.status = st;
  R.iters = it;
  rep[i] = R;
  if (st != 0) {
    active[i] = 0;
    atomicSub(n_active, 1);
  }
}

template <typename T, typename TC>
__global__ void __launch_bounds__(256) k_persistent(DevPlan<T> p, PersistArgs<TC> a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ int s_item;
  const unsigned G = gridDim.x;
  unsigned gen = 0;
  const int64_t gt = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t gs = static_cast<int64_t>(G) * blockDim.x;
  const int warp0 = static_cast<int>(gt >> 5), nwarps = static_cast<int>(gs >> 5);
  int32_t* err = p.err;
#define SOS_GRID_SYNC() \
  if (!grid_barrier(a.bar, (++gen) * G, err, p.wait_limit)) return
  int it = 0;
  for (it = 1; it <= a.max_iter; ++it) {
    d_rows_r(p, gt, gs);
    SOS_GRID_SYNC();
    d_lr_y(p, warp0, nwarps);
    SOS_GRID_SYNC();
    for (int i = blockIdx.x; i < p.n_inst; i += G) d_woodbury(p, i, reinterpret_cast<double*>(dsm));
    SOS_GRID_SYNC();
    d_rows_sigma2(p, gt, gs);
    SOS_GRID_SYNC();
    for (int i = blockIdx.x; i < p.n_inst; i += G) d_inst_scalar(p, i);
    SOS_GRID_SYNC();
    d_rows_y(p, gt, gs);
    SOS_GRID_SYNC();
    if (a.dynamic) {
      const int64_t base = static_cast<int64_t>(it - 1) * (a.n_sched + G);
      while (true) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = static_cast<int>(static_cast<int64_t>(atomicAdd(a.queue, 1u)) - base);
        __syncthreads();
        const int k = s_item;
        if (k >= a.n_sched) break;
        d_psd_small(p, a.sched[k], a.wm, dsm);
      }
    } else {
      for (int k = blockIdx.x; k < a.n_sched; k += G) d_psd_small(p, a.sched[k], a.wm, dsm);
    }
    SOS_GRID_SYNC();
    if (a.k_check > 0 && (it % a.k_check == 0 || it == a.max_iter)) {
      d_res_rows(p, gt, gs);
      d_res_lr(p, warp0, nwarps);
      SOS_GRID_SYNC();
      for (int i = blockIdx.x; i < p.n_inst; i += G) {
        d_res_inst(p, i);
        d_check(p, i, it, a.tol, a.infeas_tol, a.rep, a.active, a.n_active);
      }
      SOS_GRID_SYNC();
      if (__ldcg(a.n_active) == 0) break;
    }
  }
#undef SOS_GRID_SYNC
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.iters_done = it > a.max_iter ? a.max_iter : it;
}

int grid_for(int64_t n, int threads, int sms) {
  int64_t g = (n + threads - 1) / threads;
  const int64_t cap = static_cast<int64_t>(sms) * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

}  // namespace

template <typename T>
cudaError_t launch_affine(const DevPlan<T>& p, const LaunchShape& ls, cudaStream_t s) {
  const int rt = ls.row_threads;
  k_rows_r<T><<<grid_for(p.M, rt, ls.sms), rt, 0, s>>>(p);
  if (p.TL > 0) {
    k_lr_y<T><<<grid_for(static_cast<int64_t>(p.TL) * 32, 256, ls.sms), 256, 0, s>>>(p);
    launch_woodbury(p, s);
  }
  k_rows_sigma2<T><<<grid_for(p.M, rt, ls.sms), rt, 0, s>>>(p);
  k_inst_scalar<T><<<p.n_inst, inst_scalar_threads(p, ls), 0, s>>>(p);
  k_rows_y<T><<<grid_for(p.M, rt, ls.sms), rt, 0, s>>>(p);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_init_wl(DevPlan<T> p) {
  for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < p.TL;
       j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int i = p.lr_inst[j];
    const int64_t e = p.lr_ent[j];
    p.wl[j] = d(p.ux[e]) + d(p.vx[e]) - p.lr_c[j] * (p.tau[i] + p.kappa[i]);
  }
}

template <typename T>
cudaError_t launch_init_wl(const DevPlan<T>& p, cudaStream_t s) {
  if (p.TL == 0) return cudaSuccess;
  k_init_wl<T><<<static_cast<int>((p.TL + 255) / 256), 256, 0, s>>>(p);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_affine_part(const DevPlan<T>& p, const LaunchShape& ls, int part, cudaStream_t s) {
  const int rt = ls.row_threads;
  switch (part) {
    case 0:
      k_rows_r<T><<<grid_for(p.M, rt, ls.sms), rt, 0, s>>>(p);
      break;
    case 1:
      if (p.TL > 0) k_lr_y<T><<<grid_for(static_cast<int64_t>(p.TL) * 32, 256, ls.sms), 256, 0, s>>>(p);
      break;
    case 2:
      if (p.TL > 0) launch_woodbury(p, s);
      break;
    case 3:
      k_rows_sigma2<T><<<grid_for(p.M, rt, ls.sms), rt, 0, s>>>(p);
      break;
    case 4:
      k_inst_scalar<T><<<p.n_inst, inst_scalar_threads(p, ls), 0, s>>>(p);
      break;
    case 5:
      k_rows_y<T><<<grid_for(p.M, rt, ls.sms), rt, 0, s>>>(p);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

size_t psd_small_smem_bytes(int maxN, int form) {
  const int Np = maxN + (maxN & 1), ld = Np + 1, H = Np / 2;
  const size_t es = form == kFormFP64 ? 8 : 4;
  const size_t lam64 = form == kFormMixed ? sizeof(double) * Np : 0;  // Ritz values of the refinement
  return es * (3 * static_cast<size_t>(Np) * ld + 3 * H + Np) + lam64 + sizeof(int) * 2 * H;
}

int psd_small_max_n(int form) { return form == kFormFP64 ? 96 : (form == kFormMixed ? 112 : 128); }

template <typename T, typename TC>
cudaError_t launch_psd_small(const DevPlan<T>& p, const int32_t* ids, int count, int maxN, const SmallWarm<TC>& wm,
                             cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const size_t sm = psd_small_smem_bytes(maxN, form_of<T, TC>());
  const int threads = maxN > 64 ? 512 : 256;  // more warps per SM where blocks are large
  k_psd_small<T, TC><<<count, threads, sm, s>>>(p, ids, wm);
  return cudaGetLastError();
}

int large_grid_size(int N) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  (void)N;
  return sms;  // one CTA per SM: co-resident, and fewer barrier arrivals
}

size_t large_smem_bytes(int N, size_t es) {
  const size_t H = static_cast<size_t>(N + (N & 1)) / 2;
  return H * (3 * es + 2 * sizeof(int));
}

template <typename T, typename TC>
cudaError_t launch_psd_large_part(const DevPlan<T>& p, int bid, int N, const LargeScratch<TC>& ls, int grid,
                                  int part, cudaStream_t s) {
  if (part < 4 || part == 5) {  // 5: the warm attempt of the tridiagonal path
    if constexpr (sizeof(T) == 8 && sizeof(TC) == 8) {
      if (tri_path(N) && (part < 4 || ls.tri_warm)) return launch_psd_tri_part(p, bid, N, ls, grid, part == 5 ? 4 : part, s);
    }
    return cudaSuccess;
  }
  if (part != 4) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(ls.bar, 0, 2 * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = large_smem_bytes(N, sizeof(TC));
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_psd_large<T, TC>, p, bid, ls);
}

template <typename T, typename TC>
cudaError_t launch_psd_large(const DevPlan<T>& p, int bid, int N, const LargeScratch<TC>& ls, int grid,
                             cudaStream_t s) {
  for (int part : {5, 0, 1, 2, 3, 4}) {
    const cudaError_t e = launch_psd_large_part<T, TC>(p, bid, N, ls, grid, part, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_residuals(const DevPlan<T>& p, const LaunchShape& ls, cudaStream_t s) {
  k_res_rows<T><<<grid_for(p.M, ls.row_threads, ls.sms), ls.row_threads, 0, s>>>(p);
  if (p.TL > 0) k_res_lr<T><<<grid_for(static_cast<int64_t>(p.TL) * 32, 256, ls.sms), 256, 0, s>>>(p);
  k_res_inst<T><<<p.n_inst, 512, 0, s>>>(p);
  return cudaGetLastError();
}

template <typename T, typename TC>
cudaError_t prepare_kernels(int max_small_n, int max_teff) {
  cudaError_t e = cudaSuccess;
  if (max_small_n > 0) {
    const size_t sm = psd_small_smem_bytes(max_small_n, form_of<T, TC>());
    e = cudaFuncSetAttribute(k_psd_small<T, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    if (e != cudaSuccess) return e;
  }
  const size_t wsm = sizeof(double) * 2 * static_cast<size_t>(max_teff > 0 ? max_teff : 1);
  if (wsm > 48 * 1024) e = cudaFuncSetAttribute(k_woodbury<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(wsm));
  return e;
}


template <typename T, typename TC>
size_t persistent_smem_bytes(int max_small_n, int max_teff) {
  size_t a = psd_small_smem_bytes(max_small_n, form_of<T, TC>());
  size_t b = sizeof(double) * 2 * static_cast<size_t>(max_teff > 0 ? max_teff : 1);
  return a > b ? a : b;
}

template <typename T, typename TC>
int persistent_max_ctas_per_sm(int max_small_n, int max_teff) {
  const size_t sm = persistent_smem_bytes<T, TC>(max_small_n, max_teff);
  if (cudaFuncSetAttribute(k_persistent<T, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm)) !=
      cudaSuccess)
    return 0;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persistent<T, TC>, 256, sm) != cudaSuccess) return 0;
  return per;
}

template <typename T, typename TC>
cudaError_t launch_persistent(const DevPlan<T>& p, const PersistArgs<TC>& a, int grid, int max_small_n, int max_teff,
                              cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.bar, 0, 2 * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.queue, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = persistent_smem_bytes<T, TC>(max_small_n, max_teff);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_persistent<T, TC>, p, a);
}

int ns_grid(int N) { return ns_tiles(N); }
int ns_padded(int N) { return ns_np(N); }
size_t ns_smem_bytes() { return kNsSmem; }

template <typename T>
cudaError_t launch_psd_ns(const DevPlan<T>& p, int bid, int N, const NsScratch& S, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_psd_ns<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kNsSmem));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(S.bar, 0, 2 * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ns_tiles(N));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = kNsSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_psd_ns<T>, p, bid, S);
}

#define SOS_INSTANTIATE(T)                                                                       \
  template cudaError_t launch_affine<T>(const DevPlan<T>&, const LaunchShape&, cudaStream_t);    \
  template cudaError_t launch_affine_part<T>(const DevPlan<T>&, const LaunchShape&, int, cudaStream_t);    \
  template cudaError_t launch_init_wl<T>(const DevPlan<T>&, cudaStream_t);    \
  template cudaError_t launch_residuals<T>(const DevPlan<T>&, const LaunchShape&, cudaStream_t);             \
  template cudaError_t launch_psd_ns<T>(const DevPlan<T>&, int, int, const NsScratch&, cudaStream_t);

#define SOS_INSTANTIATE_PROJ(T, TC)                                                                          \
  template cudaError_t launch_psd_small<T, TC>(const DevPlan<T>&, const int32_t*, int, int, const SmallWarm<TC>&, \
                                               cudaStream_t);                                               \
  template cudaError_t launch_psd_large<T, TC>(const DevPlan<T>&, int, int, const LargeScratch<TC>&, int,     \
                                               cudaStream_t);                                               \
  template cudaError_t launch_psd_large_part<T, TC>(const DevPlan<T>&, int, int, const LargeScratch<TC>&, int, \
                                                    int, cudaStream_t);                                      \
  template cudaError_t prepare_kernels<T, TC>(int, int);                                                     \
  template int persistent_max_ctas_per_sm<T, TC>(int, int);                                                  \
  template cudaError_t launch_persistent<T, TC>(const DevPlan<T>&, const PersistArgs<TC>&, int, int, int,     \
                                                cudaStream_t);

SOS_INSTANTIATE(double)
SOS_INSTANTIATE(float)
SOS_INSTANTIATE_PROJ(double, double)
SOS_INSTANTIATE_PROJ(double, float)
SOS_INSTANTIATE_PROJ(float, float)

// ---------------------------------------------------------------------------
// Iterate exchange with caller device buffers (layout in kernels.h)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_gather_iterate(DevPlan<T> p, const int64_t* map, int64_t total, double* u, double* v) {
  const int64_t NX = p.NX, M = p.M;
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < total;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t src = map[q];
    if (src < NX) {
      u[q] = static_cast<double>(p.ux[src]);
      v[q] = static_cast<double>(p.vx[src]);
    } else if (src < NX + M) {
      u[q] = static_cast<double>(p.uy[src - NX]);
      v[q] = static_cast<double>(p.vy[src - NX]);
    } else {
      u[q] = p.tau[src - NX - M];
      v[q] = p.kappa[src - NX - M];
    }
  }
}

template <typename T>
__global__ void k_scatter_iterate(DevPlan<T> p, const int64_t* map, int64_t total, const double* u, const double* v,
                                  int32_t* active) {
  const int64_t NX = p.NX, M = p.M;
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < total;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t dst = map[q];
    if (dst < NX) {
      p.ux[dst] = static_cast<T>(u[q]);
      p.vx[dst] = static_cast<T>(v[q]);
    } else if (dst < NX + M) {
      p.uy[dst - NX] = static_cast<T>(u[q]);
      p.vy[dst - NX] = static_cast<T>(v[q]);
    } else {
      p.tau[dst - NX - M] = u[q];
      p.kappa[dst - NX - M] = v[q];
      active[dst - NX - M] = 1;
    }
  }
}

template <typename T>
cudaError_t launch_gather_iterate(const DevPlan<T>& p, const int64_t* map, int64_t total, double* u, double* v,
                                  cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  const int grid = static_cast<int>(std::min<int64_t>((total + 255) / 256, 152 * 16));
  k_gather_iterate<T><<<grid, 256, 0, s>>>(p, map, total, u, v);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scatter_iterate(const DevPlan<T>& p, const int64_t* map, int64_t total, const double* u,
                                   const double* v, int32_t* active, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  const int grid = static_cast<int>(std::min<int64_t>((total + 255) / 256, 152 * 16));
  k_scatter_iterate<T><<<grid, 256, 0, s>>>(p, map, total, u, v, active);
  return cudaGetLastError();
}

template cudaError_t launch_gather_iterate<double>(const DevPlan<double>&, const int64_t*, int64_t, double*, double*,
                                                   cudaStream_t);
template cudaError_t launch_gather_iterate<float>(const DevPlan<float>&, const int64_t*, int64_t, double*, double*,
                                                  cudaStream_t);
template cudaError_t launch_scatter_iterate<double>(const DevPlan<double>&, const int64_t*, int64_t, const double*,
                                                    const double*, int32_t*, cudaStream_t);
template cudaError_t launch_scatter_iterate<float>(const DevPlan<float>&, const int64_t*, int64_t, const double*,
                                                   const double*, int32_t*, cudaStream_t);

}  // namespace sos
