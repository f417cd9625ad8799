// PSD projection of one large Gram block in the plain FP64 form (eq. (20b))
// through a reduction to tridiagonal form.
//
// The projection needs the eigen-decomposition W = V diag(lambda) V^T of a
// symmetric N x N block (33 <= N <= 232 here).  Jacobi rotations need N - 1
// synchronised rounds per sweep and several sweeps per ADMM iteration; on
// GB300 a grid-wide round costs microseconds, a dependent FP64 operation 64
// cycles (an FP64 division several hundred) and the FP64 pipe delivers 1/60
// of the FP32 one.  So the sequential work runs in FP32 and FP64 is kept
// for bulk products on every SM, where the accuracy is decided:
//
//   k_tri_reduce   one CTA: W (scaled by 1/|W|_F) in FP32 shared memory,
//                  Householder reduction Q^T W Q = T (T tridiagonal), the
//                  reflector vectors kept for the back-transformation.
//   k_tri_vectors  one warp per eigenvalue i (FP32): bisection on Sturm
//                  counts of T brackets lambda_i, two steps of inverse
//                  iteration on T give its eigenvector z_i, and the
//                  reflectors map it back: v_i = Q z_i (four at a time).
//   k_tri_recon    cooperative grid, FP64 products: V made orthonormal to the
//                  unit roundoff (one second-order step of the inverse
//                  square root of V^T V, or Newton-Schulz V (3I - V^T V) / 2
//                  repeated for larger deviations),
//                  B = V^T W V, a check of the first-order projection of B,
//                  and while that fails (at most twice) a Newton correction
//                  of V (Ogita and Aishima's refinement step) and another
//                  pass; then M = diag(max(b_kk, 0)) + G o offdiag(B), g_lk
//                  the divided difference of max(., 0) at (b_ll, b_kk), and
//                  U = V M V^T, written as u and v = u - W.
//
// The first-order projection of B is exact for pairs of eigenvalues of the
// same sign (g = 1 or 0 there, and the block is linear in B) and leaves
// |b_lk|^2 / (|b_ll| + |b_kk|) at second order for a pair of opposite signs;
// the check asks that sum to stay below 1e-14 |W|_F.  FP32 eigenvectors
// carry |offdiag B| of order 1e-7 |W|, so the check passes without a
// correction where the spectrum keeps away from zero and needs one where
// eigenvalues of both signs crowd it.  If V^T V deviates from I by more
// than 0.25 (or Newton-Schulz stops converging), or three passes do not pass
// the check, the grid Jacobi kernel launched after this one takes the block
// over (flag word 0; started from V when V is orthonormal).
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "dev_common.cuh"
#include "kernels.h"

namespace sos {
namespace {

constexpr int kTriThreads = 256;   // reduction CTA (8 warps: little redundant per-warp work)
constexpr int kVecThreads = 128;   // four eigenvectors per CTA (one warp per scheduler)
constexpr int kRecThreads = 128;   // one warpgroup: the threads of a product tile
constexpr int kRecBlock = 2 * kRecThreads;  // refinement CTAs: two warpgroups split each product's K
constexpr int kTriSlots = (kTriMaxN + 31) / 32;  // per-lane register slots of a length-N vector
constexpr int kTriRows = 256;                     // columns of a lane's two float4 slots
constexpr int kTriPcol = (kTriThreads / 32) * kTriRows;  // per-warp column sums of one step

// Output of the reduction inside LargeScratch::B0 (as floats):
//   U[k * N + j]   entry j (>= k + 2) of reflector k; its entry k + 1 is 1
//   d[N], e[N]     diagonal and subdiagonal of T (e[N - 1] = 0)
//   tau[N]         FP32 Householder scalars (0: the reflector is the identity)
struct TriOut {
  float* U;
  float* d;
  float* e;
  float* tau;
};

__device__ __forceinline__ TriOut tri_out(double* B0, int N) {
  TriOut o;
  float* f = reinterpret_cast<float*>(B0);
  o.U = f;
  o.d = f + static_cast<size_t>(N) * N;
  o.e = o.d + N;
  o.tau = o.e + N;
  return o;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Householder reduction to tridiagonal form (FP32, one CTA).
//
// Step k annihilates A[k+2.., k] with H_k = I - tau v v^T (v_0 = 1):
//   beta = -sign(alpha) |A[k+1.., k]|,  tau = (beta - alpha) / beta,
//   v = A[k+1.., k] / (alpha - beta),   p = tau A22 v,
//   w = p - (tau / 2)(p^T v) v,         A22 <- A22 - v w^T - w v^T,
// with A22 the trailing block A[k+1.., k+1..].
//
// Layout: the whole symmetric matrix, index-reversed, B[i][j] = A[N-1-i][N-1-j],
// rows padded to a multiple of 4 floats.  The trailing block of step k is
// then the leading m x m block of B (m = N - 1 - k) and every access is an
// aligned float4 along a row: lane l holds columns 4 l + 128 s .. + 3
// (s = 0, 1), warp w owns the row chunks q = w + 8 t (rows 4 q .. 4 q + 3,
// whose entries of a chunked vector sit in lane q mod 32).  The update of step k and the
// product A22 v of step k + 1 are one pass over each owned row (the next
// reflector comes from row m - 1 of the updated block, which every warp
// forms for itself), so a step reads and writes each element once and needs
// one barrier.
// ---------------------------------------------------------------------------

// Sums of eight per-lane values over the warp, spread out: on return lane l
// holds the total of value (l >> 2) & 7 (nine shuffles instead of forty).
__device__ __forceinline__ float warp_sum8(float (&a)[8], int lane) {
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
  float b[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float send = h16 ? a[j] : a[j + 4], keep = h16 ? a[j + 4] : a[j];
    b[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float c[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float send = h8 ? b[j] : b[j + 2], keep = h8 ? b[j + 2] : b[j];
    c[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float x = (h4 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, h4 ? c[0] : c[1], 4);
  x += __shfl_xor_sync(0xffffffffu, x, 2);
  x += __shfl_xor_sync(0xffffffffu, x, 1);
  return x;
}

__device__ __forceinline__ float f4get(const float4& a, int c) { return c == 0 ? a.x : (c == 1 ? a.y : (c == 2 ? a.z : a.w)); }

// Entry i of a vector held as float4 chunks (lane l: entries 4 l + 128 s ..).
__device__ __forceinline__ float chunk_entry(const float4 (&v)[2], int i) {
  const int src = (i >> 2) & 31;
  const float4 a = (i >> 7) ? v[1] : v[0];
  return __shfl_sync(0xffffffffu, f4get(a, i & 3), src);
}

// Reflector from x (entries 0 .. mk-1 in chunks; the pivot alpha is entry
// mk - 1): v (pivot entry 1, zero from mk on), tau and beta; the same
// arithmetic in every warp.
__device__ __forceinline__ void make_reflector(const float4 (&x)[2], int mk, int lane, float4 (&v)[2], float& tau,
                                               float& beta) {
  float s2 = 0.f;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int j0 = 128 * s + 4 * lane;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float e = f4get(x[s], c);
      if (j0 + c < mk - 1) s2 = fmaf(e, e, s2);
    }
  }
  s2 = warp_sum_f(s2);
  const float alpha = chunk_entry(x, mk - 1);
  tau = 0.f;
  beta = alpha;
  float sc = 0.f;
  if (s2 > 0.f) {  // fast square root and reciprocals: the FP64 refinement
                    // restores the accuracy these steps give away
    const float a2 = fmaf(alpha, alpha, s2);
    beta = -copysignf(a2 * rsqrtf(a2), alpha);
    tau = (beta - alpha) * __fdividef(1.f, beta);
    sc = __fdividef(1.f, alpha - beta);
  }
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int j0 = 128 * s + 4 * lane;
    float e[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + c;
      e[c] = j < mk - 1 ? f4get(x[s], c) * sc : (j == mk - 1 ? 1.f : 0.f);
    }
    v[s] = make_float4(e[0], e[1], e[2], e[3]);
  }
}

// One pass over the rows i < nrows owned by this warp (row chunks q = warp
// + 8 t, rows 4 q .. 4 q + 3): a = a - v_i w - w_i v on the columns j < ncols,
// and this warp's share of the next product, sum over its rows i of
// v'_i a_ij for every column j (A symmetric: the column sums are the row
// products), written to pc[warp][j] -- no reduction across lanes.  All
// eight rows of two chunks are loaded before any is used; rows past the
// block are read at clamped addresses and not written (v' is zero there);
// columns past ncols are not written and their sums are never used.
// SL: float4 slots per lane (columns 4 lane + 128 s), 1 when ncols <= 128.
template <int SL>
__device__ __forceinline__ void fused_rows(float* B, int LD, int N, int nrows, int ncols, int warp, int lane,
                                           const float4 (&v)[2], const float4 (&w)[2], const float4 (&vn)[2],
                                           float* pc) {
  float4 cs[SL];
#pragma unroll
  for (int s = 0; s < SL; ++s) cs[s] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int t0 = 0; t0 < 8; t0 += 2) {
    if (4 * (warp + 8 * t0) >= nrows) break;  // warp-uniform: later chunks are further out
    float vi[8], wi[8], ni[8];
    int row[8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int t = t0 + h, src = warp + 8 * (t & 3);
      const float4 vq = t < 4 ? v[0] : v[1], wq = t < 4 ? w[0] : w[1], nq = t < 4 ? vn[0] : vn[1];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        vi[4 * h + c] = __shfl_sync(0xffffffffu, f4get(vq, c), src);
        wi[4 * h + c] = __shfl_sync(0xffffffffu, f4get(wq, c), src);
        ni[4 * h + c] = __shfl_sync(0xffffffffu, f4get(nq, c), src);
        row[4 * h + c] = 4 * (warp + 8 * t) + c;
      }
    }
    float4 a[8][SL];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int s = 0; s < SL; ++s) {
        const int i = min(row[r], N - 1), j0 = min(128 * s + 4 * lane, LD - 4);
        a[r][s] = *reinterpret_cast<const float4*>(B + i * LD + j0);
      }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const bool rok = row[r] < nrows;
#pragma unroll
      for (int s = 0; s < SL; ++s) {
        const int j0 = 128 * s + 4 * lane;
        float4 t = a[r][s];
        t.x = fmaf(-vi[r], w[s].x, fmaf(-wi[r], v[s].x, t.x));
        t.y = fmaf(-vi[r], w[s].y, fmaf(-wi[r], v[s].y, t.y));
        t.z = fmaf(-vi[r], w[s].z, fmaf(-wi[r], v[s].z, t.z));
        t.w = fmaf(-vi[r], w[s].w, fmaf(-wi[r], v[s].w, t.w));
        if (rok && j0 < ncols) *reinterpret_cast<float4*>(B + row[r] * LD + j0) = t;
        cs[s].x = fmaf(ni[r], t.x, cs[s].x);
        cs[s].y = fmaf(ni[r], t.y, cs[s].y);
        cs[s].z = fmaf(ni[r], t.z, cs[s].z);
        cs[s].w = fmaf(ni[r], t.w, cs[s].w);
      }
    }
  }
#pragma unroll
  for (int s = 0; s < SL; ++s) *reinterpret_cast<float4*>(pc + warp * kTriRows + 128 * s + 4 * lane) = cs[s];
}

constexpr int kGatherCtas = 64;

// W of the block into the reduction's layout (index-reversed, both
// triangles, FP32, unscaled) in L.T1, and per-CTA partial sums of |W|_F^2
// (FP64) in L.partial: many CTAs do the dependent gathers of the
// projection input, so the one-CTA reduction reads a dense array.
template <typename T>
__global__ void __launch_bounds__(256) k_tri_gather(DevPlan<T> p, int bid, LargeScratch<double> L) {
  __shared__ double red[40];
  const BlockDesc bd = p.blocks[bid];
  if (!p.active[bd.inst]) return;
  if (L.tri_warm && __ldcg(L.flags) == 1) return;  // the warm attempt projected the block
  const int N = bd.N, LD = (N + 3) & ~3;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), nwg = gridDim.x * (blockDim.x / 32);
  float* Bg = reinterpret_cast<float*>(L.T1);
  const double s_sm = p.st[bd.inst].s;
  double nrm2 = 0.0;
  for (int c = gw; c < N; c += nwg) {
    const int64_t base = packed_index(c, c, N);
#pragma unroll 4
    for (int r = c + lane; r < N; r += 32) {
      const double w = d(proj_input(p, bd, base + (r - c), r != c, s_sm));
      nrm2 += w * w;  // packed entries carry sqrt(2): w^2 counts both halves
      const float a = static_cast<float>(r == c ? w : w * 0.70710678118654752440);
      Bg[(N - 1 - r) * LD + (N - 1 - c)] = a;
      Bg[(N - 1 - c) * LD + (N - 1 - r)] = a;
    }
  }
  if (blockIdx.x == 0)
    for (int q = threadIdx.x; q < N * (LD - N); q += blockDim.x) Bg[(q / (LD - N)) * LD + N + q % (LD - N)] = 0.f;
  nrm2 = block_sum(nrm2, red);
  if (threadIdx.x == 0) L.partial[blockIdx.x] = nrm2;
}

template <typename T>
__global__ void __launch_bounds__(kTriThreads, 1) k_tri_reduce(DevPlan<T> p, int bid, LargeScratch<double> L) {
  extern __shared__ __align__(16) float tsm[];
  __shared__ double redd[40];
  const BlockDesc bd = p.blocks[bid];
  if (!p.active[bd.inst]) return;
  if (L.tri_warm && __ldcg(L.flags) == 1) return;  // the warm attempt projected the block
  const int N = bd.N, LD = (N + 3) & ~3;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* B = tsm;
  // per-warp column sums [8][kTriRows] (read at the start of a step, before
  // the barrier after which the step's fused pass rewrites them), and p
  float* pcol = B + static_cast<size_t>(N) * LD;
  float* pfin = pcol + kTriPcol;
  const TriOut out = tri_out(L.B0, N);

  // W (dense FP32 copy from k_tri_gather), scaled by 1 / |W|_F
  {
    double nrm2 = 0.0;
    for (int c = tid; c < kGatherCtas; c += kTriThreads) nrm2 += __ldcg(L.partial + c);  // same order everywhere
    nrm2 = block_sum(nrm2, redd);
    const float scale = nrm2 > 0.0 ? static_cast<float>(1.0 / sqrt(nrm2)) : 1.f;
    const float4* src = reinterpret_cast<const float4*>(L.T1);
    float4* dst = reinterpret_cast<float4*>(B);
#pragma unroll 4
    for (int q = tid; q < N * LD / 4; q += kTriThreads) {
      float4 a = __ldcg(src + q);
      a.x *= scale;
      a.y *= scale;
      a.z *= scale;
      a.w *= scale;
      dst[q] = a;
    }
    for (int q = tid; q < kTriPcol + kTriRows; q += kTriThreads) pcol[q] = 0.f;
  }
  __syncthreads();

  // reflector 0 from column 0 of A: row N - 1 of B (its entries 0 .. N-2)
  float4 vk[2], wk[2], vn[2];
  float tauk, beta;
  {
    float4 x[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int j0 = 128 * s + 4 * lane;
      x[s] = j0 < LD ? *reinterpret_cast<const float4*>(B + (N - 1) * LD + j0) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    make_reflector(x, N - 1, lane, vk, tauk, beta);
    if (tid == 0) {
      out.d[0] = B[(N - 1) * LD + N - 1];
      out.e[0] = beta;
      out.tau[0] = tauk;
    }
  }
  // p = tau A22 v for step 0 (no update before it)
  {
    const float4 zero[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
    fused_rows<2>(B, LD, N, N - 1, N - 1, warp, lane, vk, zero, vk, pcol);
  }
  __syncthreads();

  for (int k = 0; k < N - 2; ++k) {
    const int m = N - 1 - k;        // trailing block of step k: B[0..m-1][0..m-1]
    const float* pc = pcol;
    float* pn = pcol;
    // p = tau A v: warp w sums the per-warp column sums of columns
    // 32 w .. 32 w + 31 once, then every warp reads the whole p
    {
      const int j = 32 * warp + lane;
      float q = 0.f;
#pragma unroll
      for (int w = 0; w < kTriThreads / 32; ++w) q += pc[w * kTriRows + j];
      pfin[j] = j < m ? tauk * q : 0.f;  // sums past the block may be stale or non-finite
    }
    __syncthreads();
    // w_k = p - (tau / 2)(p^T v) v, every warp for itself
    {
      float dot = 0.f;
      float4 pk[2];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int j0 = 128 * s + 4 * lane;
        pk[s] = *reinterpret_cast<const float4*>(pfin + j0);
        dot = fmaf(pk[s].x, vk[s].x, fmaf(pk[s].y, vk[s].y, fmaf(pk[s].z, vk[s].z, fmaf(pk[s].w, vk[s].w, dot))));
      }
      const float K = -0.5f * tauk * warp_sum_f(dot);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int j0 = 128 * s + 4 * lane;
        float e[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) e[c] = (j0 + c < m) ? fmaf(K, f4get(vk[s], c), f4get(pk[s], c)) : 0.f;
        wk[s] = make_float4(e[0], e[1], e[2], e[3]);
      }
      if (tauk == 0.f) {  // H_k = I
#pragma unroll
        for (int s = 0; s < 2; ++s) wk[s] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    // row m - 1 of the updated block: the diagonal entry d_{k+1} and the next
    // reflector's column (entries 0 .. m-2)
    float taun = 0.f;
    {
      const float vm = chunk_entry(vk, m - 1), wm = chunk_entry(wk, m - 1);
      float4 y[2];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int j0 = 128 * s + 4 * lane;
        float4 t = j0 < LD ? *reinterpret_cast<const float4*>(B + (m - 1) * LD + j0) : make_float4(0.f, 0.f, 0.f, 0.f);
        t.x = fmaf(-vm, wk[s].x, fmaf(-wm, vk[s].x, t.x));
        t.y = fmaf(-vm, wk[s].y, fmaf(-wm, vk[s].y, t.y));
        t.z = fmaf(-vm, wk[s].z, fmaf(-wm, vk[s].z, t.z));
        t.w = fmaf(-vm, wk[s].w, fmaf(-wm, vk[s].w, t.w));
        y[s] = t;
      }
      const float dn = chunk_entry(y, m - 1);
      if (k + 1 <= N - 3) {
        make_reflector(y, m - 1, lane, vn, taun, beta);
        if (tid == 0) {
          out.d[k + 1] = dn;
          out.e[k + 1] = beta;
          out.tau[k + 1] = taun;
        }
      } else {  // the last 2 x 2 block: no reflector
        const float e_last = chunk_entry(y, 0);
        if (tid == 0) {
          out.d[k + 1] = dn;
          out.e[k + 1] = e_last;
          out.tau[k + 1] = 0.f;
        }
#pragma unroll
        for (int s = 0; s < 2; ++s) vn[s] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    // reflector k for the back-transformation (A order: entries k + 2 .. N-1
    // = B entries 0 .. m - 2, reversed)
    if (warp < 2) {
      const int j0 = 128 * warp + 4 * lane;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = j0 + c;
        if (j < m - 1) out.U[static_cast<int64_t>(k) * N + (N - 1 - j)] = f4get(vk[warp], c);
      }
    }
    // own rows i < m - 1: update with (v_k, w_k), then the product with v_{k+1}
    if (m > 129)
      fused_rows<2>(B, LD, N, m - 1, m, warp, lane, vk, wk, vn, pn);
    else
      fused_rows<1>(B, LD, N, m - 1, m, warp, lane, vk, wk, vn, pn);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 2; ++s) vk[s] = vn[s];
    tauk = taun;
  }
  if (tid == 0) out.d[N - 1] = B[0];
}

// ---------------------------------------------------------------------------
// Eigenvector i of T, mapped back by the reflectors (one CTA per eigenvalue,
// FP32: on this GPU a dependent FP64 operation takes 64 cycles and an FP64
// division several hundred, so every sequential recurrence here is FP32 and
// the FP64 accuracy comes from the refinement of the reconstruction kernel).
// ---------------------------------------------------------------------------

// Number of eigenvalues of T below x (Sturm sequence of the LDL^T pivots;
// a pivot of magnitude below pivmin is replaced by -pivmin).
// Sturm counts of T - x0 I and T - x1 I (the number of eigenvalues below
// x0 and x1): the pivots of the LDL^T recurrence q_k = d_k - x - e_{k-1}^2 /
// q_{k-1}, two independent chains interleaved; a pivot smaller than pivmin
// is replaced by -pivmin.
__device__ __forceinline__ void sturm_count2(const float* __restrict__ d, const float* __restrict__ e2, int N,
                                             float x0, float x1, float pivmin, int& c0, int& c1) {
  float q0 = d[0] - x0, q1 = d[0] - x1;
  q0 = fabsf(q0) < pivmin ? -pivmin : q0;
  q1 = fabsf(q1) < pivmin ? -pivmin : q1;
  int a0 = q0 < 0.f, a1 = q1 < 0.f;
#pragma unroll 4
  for (int k = 1; k < N; ++k) {
    const float dk = d[k], ek = e2[k - 1];
    q0 = (dk - x0) - __fdividef(ek, q0);
    q1 = (dk - x1) - __fdividef(ek, q1);
    q0 = fabsf(q0) < pivmin ? -pivmin : q0;
    q1 = fabsf(q1) < pivmin ? -pivmin : q1;
    a0 += q0 < 0.f;
    a1 += q1 < 0.f;
  }
  c0 = a0;
  c1 = a1;
}

// Deterministic start vector entries in (-1, 1).
__device__ __forceinline__ float start_entry(int i, int j) {
  uint32_t h = static_cast<uint32_t>(i) * 0x9E3779B1u ^ (static_cast<uint32_t>(j) + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  return (static_cast<float>(h & 0xFFFFFFu) + 0.5f) / 8388608.0f - 1.0f;
}

constexpr int kVecGroup = 4;                                   // reflectors applied per warp reduction
constexpr int kVecChunk = kVecGroup * (kVecThreads / 32);      // reflectors staged at a time: one group per warp
constexpr int kVecPairs = kVecGroup * (kVecGroup - 1) / 2;     // products u_r^T u_t, t < r, of a group

__host__ __device__ __forceinline__ int vec_ld(int N) { return (N + 3) & ~3; }

// Shared memory of k_tri_vectors: d, e, e^2, tau of T; per warp the
// eigenvector z and the pivoted LU of the inverse iteration (1 / pivot,
// first and second superdiagonal of U, multipliers); two chunks of
// reflectors; the products of the reflectors within each group of a chunk;
// per warp the row exchanges (bytes).
size_t tri_vectors_smem(int N) {
  constexpr int nw = kVecThreads / 32;
  return sizeof(float) * (static_cast<size_t>(4 + 5 * nw) * N + 2 * kVecChunk * static_cast<size_t>(vec_ld(N)) +
                          (kVecChunk / kVecGroup) * kVecPairs) +
         sizeof(bool) * nw * static_cast<size_t>(N);
}

__global__ void __launch_bounds__(kVecThreads) k_tri_vectors(DevPlan<double> p, int bid, LargeScratch<double> L) {
  extern __shared__ __align__(16) float vsm[];
  __shared__ float s_g[3][kVecThreads / 32];
  const BlockDesc bd = p.blocks[bid];
  if (!p.active[bd.inst]) return;
  if (L.tri_warm && __ldcg(L.flags) == 1) return;  // the warm attempt projected the block
  const int N = bd.N, ldu = vec_ld(N);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nw = kVecThreads / 32;
  const TriOut out = tri_out(L.B0, N);
  float* df = vsm;       // diagonal of T
  float* ef = df + N;    // subdiagonal, split entries zeroed
  float* e2f = ef + N;   // its squares
  float* tau_s = e2f + N;
  float* z = tau_s + N + warp * 5 * N;  // this warp's eigenvector of T and the
  float* rinv = z + N;   // pivoted LU of T - sigma I: reciprocal pivots, first
  float* du = rinv + N;  // and second superdiagonal of U, multipliers
  float* du2 = du + N;
  float* dl = du2 + N;
  float* ubuf = tau_s + N + nw * 5 * N;      // [2][kVecChunk][ldu] reflectors
  float* gbuf = ubuf + 2 * kVecChunk * ldu;  // [kVecChunk / kVecGroup][kVecPairs]
  bool* pv = reinterpret_cast<bool*>(gbuf + (kVecChunk / kVecGroup) * kVecPairs) + warp * N;  // row exchanges

  // T, the Gershgorin bounds and the splits (|e_k| <= 1e-10 |T| set to zero)
  float tn = 0.f, glo = FLT_MAX, ghi = -FLT_MAX;
  for (int k = tid; k < N; k += kVecThreads) {
    const float dk = out.d[k], ek = k < N - 1 ? fabsf(out.e[k]) : 0.f, em = k > 0 ? fabsf(out.e[k - 1]) : 0.f;
    tn = fmaxf(tn, fabsf(dk) + ek + em);
    glo = fminf(glo, dk - ek - em);
    ghi = fmaxf(ghi, dk + ek + em);
  }
  for (int o = 16; o > 0; o >>= 1) {
    tn = fmaxf(tn, __shfl_xor_sync(0xffffffffu, tn, o));
    glo = fminf(glo, __shfl_xor_sync(0xffffffffu, glo, o));
    ghi = fmaxf(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
  }
  if (lane == 0) {
    s_g[0][warp] = tn;
    s_g[1][warp] = glo;
    s_g[2][warp] = ghi;
  }
  __syncthreads();
  tn = 0.f;
  glo = FLT_MAX;
  ghi = -FLT_MAX;
  for (int w = 0; w < nw; ++w) {
    tn = fmaxf(tn, s_g[0][w]);
    glo = fminf(glo, s_g[1][w]);
    ghi = fmaxf(ghi, s_g[2][w]);
  }
  const float split = 1e-10f * tn;
  int has_split = 0;
  for (int k = tid; k < N; k += kVecThreads) {
    float ek = k < N - 1 ? out.e[k] : 0.f;
    if (fabsf(ek) <= split) {
      ek = 0.f;
      has_split |= k < N - 1;
    }
    df[k] = out.d[k];
    ef[k] = ek;
    e2f[k] = ek * ek;
    tau_s[k] = out.tau[k];
  }
  has_split = __syncthreads_or(has_split);
  const int i = blockIdx.x * nw + warp;  // this warp's eigenvalue (ascending order)
  const bool valid = i < N;              // a warp past N still stages reflectors below

  if (valid) {
    // bisection: 64 points per pass (two per lane), keeping
    // count(lo) <= i < count(hi)
    const float pivmin = 1e-30f;
    float lo = glo - 1e-6f * tn - 1e-30f, hi = ghi + 1e-6f * tn + 1e-30f;
    for (int pass = 0; pass < 4; ++pass) {
      const float step = (hi - lo) * (1.f / 65.f);
      const float x0 = fmaf(step, static_cast<float>(lane + 1), lo);
      const float x1 = fmaf(step, static_cast<float>(lane + 33), lo);
      int c0, c1;
      sturm_count2(df, e2f, N, x0, x1, pivmin, c0, c1);
      float nlo = fmaxf(c0 <= i ? x0 : -FLT_MAX, c1 <= i ? x1 : -FLT_MAX);
      float nhi = fminf(c0 >= i + 1 ? x0 : FLT_MAX, c1 >= i + 1 ? x1 : FLT_MAX);
      for (int o = 16; o > 0; o >>= 1) {
        nlo = fmaxf(nlo, __shfl_xor_sync(0xffffffffu, nlo, o));
        nhi = fminf(nhi, __shfl_xor_sync(0xffffffffu, nhi, o));
      }
      if (nlo > lo && nlo < hi) lo = nlo;
      if (nhi < hi && nhi > lo) hi = nhi;
    }

    // the unreduced block of T that holds eigenvalue i (the whole matrix
    // unless T split), found by lane 0 from block-wise Sturm counts
    int b0 = 0, b1 = N - 1;
    if (has_split) {
      if (lane == 0) {
        int clo = 0;
        {
          float q = 0.f;
          for (int k = 0; k < N; ++k) {
            q = (k == 0 || e2f[k - 1] == 0.f) ? df[k] - lo : (df[k] - lo) - __fdividef(e2f[k - 1], q);
            if (fabsf(q) < pivmin) q = -pivmin;
            clo += q < 0.f;
          }
        }
        const int want = i - clo;  // position of eigenvalue i among those in (lo, hi], by block
        int run = 0, start = 0, cl = 0, ch = 0;
        float ql = 0.f, qh = 0.f;
        bool found = false;
        for (int k = 0; k < N && !found; ++k) {
          if (k == 0 || e2f[k - 1] == 0.f) {
            start = k;
            cl = ch = 0;
            ql = df[k] - lo;
            qh = df[k] - hi;
          } else {
            ql = (df[k] - lo) - __fdividef(e2f[k - 1], ql);
            qh = (df[k] - hi) - __fdividef(e2f[k - 1], qh);
          }
          if (fabsf(ql) < pivmin) ql = -pivmin;
          if (fabsf(qh) < pivmin) qh = -pivmin;
          cl += ql < 0.f;
          ch += qh < 0.f;
          if (k == N - 1 || e2f[k] == 0.f) {  // end of a block
            const int inb = ch - cl;
            if (run + inb > want) {
              b0 = start;
              b1 = k;
              found = true;
            }
            run += inb;
          }
        }
        if (!found) {  // inconsistent counts: the whole matrix
          b0 = 0;
          b1 = N - 1;
        }
      }
      b0 = __shfl_sync(0xffffffffu, b0, 0);
      b1 = __shfl_sync(0xffffffffu, b1, 0);
    }

    // inverse iteration, two steps with the shift at the centre of the
    // bracket: lane 0 factors T_b - sigma I once with partial pivoting (the
    // first right side eliminated in the same pass) and substitutes
    // backward; the warp normalises; lane 0 repeats the forward elimination
    // and backward substitution on the result.  (Emulated on ADMM inputs of
    // a 231 x 231 block, two steps at a fixed shift give the same
    // orthogonality and Ritz off-diagonal as three with Rayleigh shifts.)
    float nrm = 0.f;
    for (int k = lane; k < N; k += 32) {
      const float v = (k >= b0 && k <= b1) ? start_entry(i, k) : 0.f;
      z[k] = v;
      nrm = fmaf(v, v, nrm);
    }
    nrm = rsqrtf(warp_sum_f(nrm));
    for (int k = lane; k < N; k += 32) z[k] *= nrm;
    __syncwarp();
    if (b1 > b0) {
      const float tiny = 1.2e-7f * tn + 1e-30f;
      const float sigma = 0.5f * (lo + hi);
      float* __restrict__ zR = z;
      float* __restrict__ rR = rinv;
      float* __restrict__ uR = du;
      float* __restrict__ u2R = du2;
      float* __restrict__ lR = dl;
      // backward substitution with U; the next step's operands are loaded
      // one step ahead
      auto backward = [&](float zk) {
        float y1 = zk * rR[b1], y2 = 0.f;
        zR[b1] = y1;
        float zc = zR[b1 - 1], uc = uR[b1 - 1], u2c = u2R[b1 - 1], rc = rR[b1 - 1];
        for (int k = b1 - 1; k >= b0; --k) {
          const bool more = k > b0;
          const float zp = more ? zR[k - 1] : 0.f, up = more ? uR[k - 1] : 0.f;
          const float u2p = more ? u2R[k - 1] : 0.f, rp = more ? rR[k - 1] : 0.f;
          const float y = fmaf(-u2c, y2, fmaf(-uc, y1, zc)) * rc;
          zR[k] = y;
          y2 = y1;
          y1 = y;
          zc = zp;
          uc = up;
          u2c = u2p;
          rc = rp;
        }
      };
      auto normalise = [&]() {
        __syncwarp();
        float n2 = 0.f;
        for (int k = b0 + lane; k <= b1; k += 32) n2 = fmaf(z[k], z[k], n2);
        const float sc = rsqrtf(warp_sum_f(n2));
        for (int k = b0 + lane; k <= b1; k += 32) z[k] *= sc;
        __syncwarp();
      };
      if (lane == 0) {
        const float* __restrict__ dR = df;
        const float* __restrict__ eR = ef;
        // operands of the next step are loaded one step ahead, so the
        // dependent chain of a step holds no shared-memory load; step k
        // keeps its multiplier in lR and its row exchange in pv
        float dk = dR[b0] - sigma, uk = eR[b0], zk = zR[b0];
        float lk = eR[b0], dn = dR[b0 + 1] - sigma, zn = zR[b0 + 1];
        float un = b0 + 1 < b1 ? eR[b0 + 1] : 0.f;
        for (int k = b0; k < b1; ++k) {
          const bool more = k + 1 < b1;
          const float dn2 = more ? dR[k + 2] - sigma : 0.f;
          const float zn2 = more ? zR[k + 2] : 0.f;
          const float un2 = k + 2 < b1 ? eR[k + 2] : 0.f;
          const bool sw = fabsf(lk) > fabsf(dk);  // rows k and k + 1 exchanged
          const float pd = fabsf(dk) < tiny ? (dk < 0.f ? -tiny : tiny) : dk;
          const float r = __fdividef(1.f, sw ? lk : pd);
          const float l = (sw ? dk : lk) * r;
          rR[k] = r;
          uR[k] = sw ? dn : uk;
          u2R[k] = sw ? un : 0.f;
          lR[k] = l;
          pv[k] = sw;
          zR[k] = sw ? zn : zk;  // forward elimination of the right side
          const float dk1 = sw ? fmaf(-l, dn, uk) : fmaf(-l, uk, dn);
          const float uk1 = sw ? -l * un : un;
          const float zk1 = sw ? fmaf(-l, zn, zk) : fmaf(-l, zk, zn);
          dk = dk1;
          uk = uk1;
          zk = zk1;
          lk = un;  // e_{k+1}
          dn = dn2;
          zn = zn2;
          un = un2;
        }
        rR[b1] = __fdividef(1.f, fabsf(dk) < tiny ? (dk < 0.f ? -tiny : tiny) : dk);
        backward(zk);
      }
      normalise();
      if (lane == 0) {  // second step: the same factors
        float zk = zR[b0], zn = zR[b0 + 1], l = lR[b0];
        bool sw = pv[b0];
        for (int k = b0; k < b1; ++k) {
          const bool more = k + 1 < b1;
          const float zn2 = more ? zR[k + 2] : 0.f, l2 = more ? lR[k + 1] : 0.f;
          const bool sw2 = more ? pv[k + 1] : false;
          zR[k] = sw ? zn : zk;
          zk = sw ? fmaf(-l, zn, zk) : fmaf(-l, zk, zn);
          zn = zn2;
          l = l2;
          sw = sw2;
        }
        backward(zk);
      }
      normalise();
    }
  }
  __syncwarp();

  // v_i = H_0 H_1 ... H_{N-3} z.  Lane l holds entries l + 32 s.  The CTA
  // stages kVecChunk reflectors at a time in shared memory (entry k + 1 set
  // to 1, entries up to k zero), loading the next chunk while the current
  // one is applied.  A warp applies a group of kVecGroup reflectors
  // u_0, u_1, ... (in the order they act) with one reduction: with
  // d_r = u_r^T z and g_rt = u_r^T u_t, reflector r meets
  // z - sum_{t < r} alpha_t u_t, so alpha_r = tau_r (d_r - sum_{t < r}
  // alpha_t g_rt), and z -= sum_r alpha_r u_r.  The g_rt depend on the
  // reflectors only: warp w forms those of group w of each chunk for the CTA.
  float zr[kTriSlots];
#pragma unroll
  for (int s = 0; s < kTriSlots; ++s) {
    const int j = lane + 32 * s;
    zr[s] = (valid && j < N) ? z[j] : 0.f;
  }
  const int nref = N - 2;  // reflectors 0 .. N - 3, applied from N - 3 down
  const int nchunk = (nref + kVecChunk - 1) / kVecChunk;
  constexpr int kPer = (kVecChunk * ((kTriMaxN + 3) & ~3) + kVecThreads - 1) / kVecThreads;
  float pre[kPer];
  // chunk c holds reflectors k = N - 3 - c kVecChunk - r, r = 0 .. kVecChunk - 1
  auto load_chunk = [&](int c) {
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
      const int q = tid + t * kVecThreads;
      const int r = q / ldu, j = q - r * ldu;
      const int k = N - 3 - c * kVecChunk - r;
      float v = 0.f;
      if (r < kVecChunk && k >= 0 && j < N)
        v = j == k + 1 ? 1.f : (j >= k + 2 ? __ldcg(out.U + static_cast<int64_t>(k) * N + j) : 0.f);
      pre[t] = v;
    }
  };
  auto store_chunk = [&](int buf) {
    float* dst = ubuf + buf * kVecChunk * ldu;
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
      const int q = tid + t * kVecThreads;
      if (q < kVecChunk * ldu) dst[q] = pre[t];
    }
  };
  auto load_group = [&](const float* ub, int g, float (&u)[kVecGroup][kTriSlots]) {
#pragma unroll
    for (int r = 0; r < kVecGroup; ++r)
#pragma unroll
      for (int s = 0; s < kTriSlots; ++s) {
        const int j = lane + 32 * s;
        u[r][s] = j < ldu ? ub[(g + r) * ldu + j] : 0.f;
      }
  };
  load_chunk(0);
  store_chunk(0);
  __syncthreads();
  for (int c = 0; c < nchunk; ++c) {
    if (c + 1 < nchunk) load_chunk(c + 1);
    const float* ub = ubuf + (c & 1) * kVecChunk * ldu;
    {  // g_rt of group `warp` of this chunk
      float u[kVecGroup][kTriSlots];
      load_group(ub, warp * kVecGroup, u);
      float gv[kVecPairs];
      int q = 0;
#pragma unroll
      for (int r = 1; r < kVecGroup; ++r)
#pragma unroll
        for (int t = 0; t < r; ++t) {
          float acc = 0.f;
#pragma unroll
          for (int s = 0; s < kTriSlots; ++s) acc = fmaf(u[r][s], u[t][s], acc);
          gv[q++] = acc;
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q2 = 0; q2 < kVecPairs; ++q2) gv[q2] += __shfl_xor_sync(0xffffffffu, gv[q2], o);
      if (lane < kVecPairs) {
        float x = gv[0];
#pragma unroll
        for (int q2 = 1; q2 < kVecPairs; ++q2) x = lane == q2 ? gv[q2] : x;
        gbuf[warp * kVecPairs + lane] = x;
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int g = 0; g < kVecChunk; g += kVecGroup) {
      const int k0 = N - 3 - c * kVecChunk - g;  // first reflector of the group
      if (k0 < 0) break;
      float u[kVecGroup][kTriSlots];
      load_group(ub, g, u);
      float dv[kVecGroup];
#pragma unroll
      for (int r = 0; r < kVecGroup; ++r) {
        float acc = 0.f;
#pragma unroll
        for (int s = 0; s < kTriSlots; ++s) acc = fmaf(u[r][s], zr[s], acc);
        dv[r] = acc;
      }
      // transposed reduction: after the xor-16 and xor-8 exchanges lane l
      // holds a partial of d_{(l >> 3) & 3}; three more steps finish it, and
      // lanes 0, 8, 16, 24 broadcast d_0 .. d_3
      const bool h16 = lane & 16, h8 = lane & 8;
      const float b0 = (h16 ? dv[2] : dv[0]) + __shfl_xor_sync(0xffffffffu, h16 ? dv[0] : dv[2], 16);
      const float b1 = (h16 ? dv[3] : dv[1]) + __shfl_xor_sync(0xffffffffu, h16 ? dv[1] : dv[3], 16);
      float x = (h8 ? b1 : b0) + __shfl_xor_sync(0xffffffffu, h8 ? b0 : b1, 8);
      x += __shfl_xor_sync(0xffffffffu, x, 4);
      x += __shfl_xor_sync(0xffffffffu, x, 2);
      x += __shfl_xor_sync(0xffffffffu, x, 1);
      float dsum[kVecGroup];
#pragma unroll
      for (int r = 0; r < kVecGroup; ++r) dsum[r] = __shfl_sync(0xffffffffu, x, 8 * r);
      const float* gg = gbuf + (g / kVecGroup) * kVecPairs;
      float al[kVecGroup];
#pragma unroll
      for (int r = 0; r < kVecGroup; ++r) {
        float dd = dsum[r];
#pragma unroll
        for (int t = 0; t < r; ++t) dd = fmaf(-al[t], gg[r * (r - 1) / 2 + t], dd);  // g_rt
        const int k = k0 - r;
        al[r] = k >= 0 ? tau_s[k] * dd : 0.f;
      }
#pragma unroll
      for (int r = 0; r < kVecGroup; ++r)
#pragma unroll
        for (int s = 0; s < kTriSlots; ++s) zr[s] = fmaf(-al[r], u[r][s], zr[s]);
    }
    // buffer (c + 1) & 1 last served chunk c - 1, which every warp finished
    // before the barrier that opened chunk c; gbuf is rewritten only after
    // the next barrier
    if (c + 1 < nchunk) store_chunk((c + 1) & 1);
    __syncthreads();
  }
  if (!valid) return;
  const int Np = N + (N & 1);
#pragma unroll
  for (int s = 0; s < kTriSlots; ++s) {
    const int j = lane + 32 * s;
    if (j < N) L.V[static_cast<int64_t>(j) * Np + i] = static_cast<double>(zr[s]);
  }
}

// ---------------------------------------------------------------------------
// FP64 refinement and reconstruction on every SM (cooperative).
// ---------------------------------------------------------------------------
constexpr int kKC = 16;

// Tile (TM x TN) of C = op(A) op(B), op(A) n x n, op(B) n x n, leading
// dimension ld, on the CTA's two warpgroups: warpgroup w multiplies the K
// chunks w, w + 2, ... with its own shared-memory buffers and its own named
// barrier, and the partial sums meet at the end.  Thread t of a warpgroup
// computes row t % TM and the columns t / TM + 8 q; the result is valid in
// warpgroup 0 (threads 0..127).  op(X) = X^T where the flag is set.
// xb(k, j, x) maps an element of op(B) as it is staged.  The next chunk is
// loaded into registers while the current one is multiplied.  A and B are
// stored as G and multiplied as F (rounded as they are staged).  sA and sB
// hold two buffers each (2 TM (kKC + 1) and 2 kKC (TN + 1) elements of F).
template <typename F, int TM, int TN, bool TA, bool TB, class XB, typename G = F>
__device__ __forceinline__ void gemm_tile(const G* A, const G* B, int ld, int n, int i0, int j0, XB xb,
                                          F (&acc)[TM * TN / kRecThreads], F* sA, F* sB) {
  constexpr int PT = TM * TN / kRecThreads;
  constexpr int LA = TM * kKC / kRecThreads, LB = kKC * TN / kRecThreads;
  static_assert(LA * kRecThreads == TM * kKC && LB * kRecThreads == kKC * TN, "tile shape");
  static_assert(TM * TN <= kKC * (TN + 1), "partial sums fit the B buffer");
  const int wg = threadIdx.x / kRecThreads;
  const int t = threadIdx.x - wg * kRecThreads, r = t % TM, g = t / TM;
  F* mA = sA + wg * TM * (kKC + 1);
  F* mB = sB + wg * kKC * (TN + 1);
  auto wg_sync = [&]() { asm volatile("bar.sync %0, %1;" ::"r"(1 + wg), "n"(kRecThreads) : "memory"); };
  G ra[LA], rb[LB];
  auto load = [&](int k0) {
#pragma unroll
    for (int u = 0; u < LA; ++u) {
      const int e = t + u * kRecThreads;
      int ii, kk;
      if (TA) {
        kk = e / TM;
        ii = e - kk * TM;
      } else {
        ii = e / kKC;
        kk = e - ii * kKC;
      }
      const int gi = i0 + ii, gk = k0 + kk;
      ra[u] = (gi < n && gk < n)
                  ? __ldcg(TA ? A + static_cast<int64_t>(gk) * ld + gi : A + static_cast<int64_t>(gi) * ld + gk)
                  : G(0);
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int e = t + u * kRecThreads;
      int jj, kk;
      if (TB) {
        jj = e / kKC;
        kk = e - jj * kKC;
      } else {
        kk = e / TN;
        jj = e - kk * TN;
      }
      const int gj = j0 + jj, gk = k0 + kk;
      rb[u] = (gj < n && gk < n)
                  ? __ldcg(TB ? B + static_cast<int64_t>(gj) * ld + gk : B + static_cast<int64_t>(gk) * ld + gj)
                  : G(0);
    }
  };
  auto store = [&](int k0) {
#pragma unroll
    for (int u = 0; u < LA; ++u) {
      const int e = t + u * kRecThreads;
      int ii, kk;
      if (TA) {
        kk = e / TM;
        ii = e - kk * TM;
      } else {
        ii = e / kKC;
        kk = e - ii * kKC;
      }
      mA[ii * (kKC + 1) + kk] = static_cast<F>(ra[u]);
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int e = t + u * kRecThreads;
      int jj, kk;
      if (TB) {
        jj = e / kKC;
        kk = e - jj * kKC;
      } else {
        kk = e / TN;
        jj = e - kk * TN;
      }
      const int gj = j0 + jj, gk = k0 + kk;
      mB[kk * (TN + 1) + jj] = (gj < n && gk < n) ? static_cast<F>(xb(gk, gj, rb[u])) : F(0);
    }
  };
  // KS independent partial sums per output (interleaved k): four warps per
  // SM leave the dependent multiply-add latency exposed with one chain per
  // output
  constexpr int KS = 2;
  F part[KS][PT];
#pragma unroll
  for (int h = 0; h < KS; ++h)
#pragma unroll
    for (int q = 0; q < PT; ++q) part[h][q] = F(0);
  load(wg * kKC);
  for (int k0 = wg * kKC; k0 < n; k0 += 2 * kKC) {
    store(k0);
    wg_sync();
    if (k0 + 2 * kKC < n) load(k0 + 2 * kKC);
#pragma unroll
    for (int kk = 0; kk < kKC; kk += KS) {
#pragma unroll
      for (int h = 0; h < KS; ++h) {
        const F a = mA[r * (kKC + 1) + kk + h];
#pragma unroll
        for (int q = 0; q < PT; ++q) part[h][q] = fma(a, mB[(kk + h) * (TN + 1) + g + 8 * q], part[h][q]);
      }
    }
    wg_sync();
  }
#pragma unroll
  for (int q = 0; q < PT; ++q) {
#pragma unroll
    for (int h = 1; h < KS; ++h) part[0][q] += part[h][q];
  }
  // warpgroup 1 hands its sums to warpgroup 0 through the first B buffer
  // (warpgroup 1's next stores go to its own buffers; warpgroup 0 reads
  // these before its own next store)
  __syncthreads();
  if (wg == 1)
#pragma unroll
    for (int q = 0; q < PT; ++q) sB[t * PT + q] = part[0][q];
  __syncthreads();
  if (wg == 0)
#pragma unroll
    for (int q = 0; q < PT; ++q) acc[q] = part[0][q] + sB[t * PT + q];
}

struct Ident {
  template <typename X>
  __device__ __forceinline__ X operator()(int, int, X x) const { return x; }
};

// Correction part (I - V^T V) / 2 of the Newton-Schulz factor, from the
// stored V^T V.
struct NsCorr {
  __device__ __forceinline__ double operator()(int k, int j, double x) const {
    return 0.5 * ((k == j ? 1.0 : 0.0) - x);
  }
};

// Newton-Schulz factor (3 I - V^T V) / 2 from the stored V^T V.
struct NsFactor {
  __device__ __forceinline__ double operator()(int k, int j, double x) const {
    return (k == j ? 1.5 : 0.0) - 0.5 * x;
  }
};

// Second-order factor I + E/2 + 3 E^2 / 8 of the inverse square root of
// V^T V = I - E, from the stored E^2 (staged) and V^T V (read).
struct NsFactor2 {
  const double* G;
  int ld;
  __device__ __forceinline__ double operator()(int k, int j, double e2) const {
    const double g = __ldcg(G + static_cast<int64_t>(k) * ld + j);
    return (k == j ? 1.0 + 0.5 * (1.0 - g) : -0.5 * g) + 0.375 * e2;
  }
};

// First-order projection of B = V^T W V at its diagonal (see the file header).
struct FirstOrder {
  const double* B;
  int ld;
  __device__ __forceinline__ double operator()(int k, int j, double x) const {
    const double bk = __ldcg(B + static_cast<int64_t>(k) * ld + k), bj = __ldcg(B + static_cast<int64_t>(j) * ld + j);
    if (k == j) return fmax(bk, 0.0);
    if (bk > 0.0 && bj > 0.0) return x;
    if (bk <= 0.0 && bj <= 0.0) return 0.0;
    return (fmax(bk, 0.0) - fmax(bj, 0.0)) / (bk - bj) * x;  // |bk - bj| > 0 here
  }
};

// C = A + A X for FP64 A and a small correction X = xb(stored), the
// product A X in FP32 (relative error about 1e-6 of |X|): for steps whose
// result the next check measures again in FP64 (a Newton rotation, a
// Newton-Schulz step far from orthonormal), never for the last one.
template <class XB>
__device__ void gemm_corr(const double* A, const double* X, double* C, int N, int ld, XB xb, float* sA, float* sB) {
  const int ntn = (N + 23) / 24, nfull = ((N + 15) / 16) * ntn;
  for (int t = blockIdx.x; t < nfull; t += gridDim.x) {
    const int ti = t / ntn, tj = t - ti * ntn;
    float acc[3];
    gemm_tile<float, 16, 24, false, false, XB, double>(A, X, ld, N, ti * 16, tj * 24, xb, acc, sA, sB);
    if (threadIdx.x >= kRecThreads) continue;
    const int r = threadIdx.x % 16, g = threadIdx.x / 16;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int ii = ti * 16 + r, jj = tj * 24 + g + 8 * q;
      if (ii < N && jj < N) {
        const int64_t o = static_cast<int64_t>(ii) * ld + jj;
        C[o] = __ldcg(A + o) + static_cast<double>(acc[q]);
      }
    }
  }
}

// Lower-triangle tile index -> (ti, tj), ti >= tj.
__device__ __forceinline__ void lower_tile(int t, int& ti, int& tj) {
  ti = static_cast<int>((sqrtf(8.0f * static_cast<float>(t) + 1.0f) - 1.0f) * 0.5f);
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  while (ti * (ti + 1) / 2 > t) --ti;
  tj = t - ti * (ti + 1) / 2;
}

// C = op(A) op(B) over all 16 x 24 tiles (full) into C.
template <bool TA, bool TB, class XB, typename F>
__device__ void gemm_full(const F* A, const F* B, F* C, int N, int ld, XB xb, F* sA, F* sB) {
  const int ntn = (N + 23) / 24, nfull = ((N + 15) / 16) * ntn;
  for (int t = blockIdx.x; t < nfull; t += gridDim.x) {
    const int ti = t / ntn, tj = t - ti * ntn;
    F acc[3];
    gemm_tile<F, 16, 24, TA, TB>(A, B, ld, N, ti * 16, tj * 24, xb, acc, sA, sB);
    if (threadIdx.x >= kRecThreads) continue;
    const int r = threadIdx.x % 16, g = threadIdx.x / 16;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int ii = ti * 16 + r, jj = tj * 24 + g + 8 * q;
      if (ii < N && jj < N) C[static_cast<int64_t>(ii) * ld + jj] = acc[q];
    }
  }
}

// Symmetric C = op(A) op(B) over the lower 16 x 16 tiles, mirrored; f(i, j,
// c) sees each lower entry (i >= j) once.  CT: the type the products are
// computed in (FP32 only where the result's rounding is far below what it
// is used for).
template <bool TA, bool TB, class F, typename CT = double>
__device__ void gemm_sym(const double* A, const double* B, double* C, int N, int ld, F f, double* sA, double* sB) {
  const int nt = (N + 15) / 16, nlow = nt * (nt + 1) / 2;
  for (int t = blockIdx.x; t < nlow; t += gridDim.x) {
    int ti, tj;
    lower_tile(t, ti, tj);
    CT acc[2];
    gemm_tile<CT, 16, 16, TA, TB, Ident, double>(A, B, ld, N, ti * 16, tj * 16, Ident(), acc,
                                                 reinterpret_cast<CT*>(sA), reinterpret_cast<CT*>(sB));
    if (threadIdx.x >= kRecThreads) continue;
    const int r = threadIdx.x % 16, g = threadIdx.x / 16;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int ii = ti * 16 + r, jj = tj * 16 + g + 8 * q;
      if (ii < N && jj < N && ii >= jj) {
        if (C) {
          C[static_cast<int64_t>(ii) * ld + jj] = acc[q];
          C[static_cast<int64_t>(jj) * ld + ii] = acc[q];
        }
        f(ii, jj, acc[q]);
      }
    }
  }
}

struct NoOp {
  __device__ __forceinline__ void operator()(int, int, double) const {}
};

// |G - I| of a Gram matrix G = V^T V, NaN counted as non-orthonormal.
struct OrthMax {
  double* m;
  __device__ __forceinline__ void operator()(int i, int j, double x) const {
    const double dv = fabs(x - (i == j ? 1.0 : 0.0));
    *m = (dv == dv) ? fmax(*m, dv) : 1e300;
  }
};

// Newton correction of Ogita and Aishima ("Iterative refinement for
// symmetric eigenvalue decomposition", 2018) for orthonormal V with
// S = V^T W V: V' = V (I + E), e_ij = s_ij / (s_jj - s_ii) where that is a
// small rotation (|e_ij| <= 0.1), else 0 (the pair is left as a cluster).
// E is written over S's storage companion C (N x N, leading dimension ld).
// With F32 (the Rayleigh-quotient update below), also FP32 copies of E and
// of the off-diagonal of S, the diagonal of S in dsave, and this thread's
// largest |e| and largest off-diagonal |s_ij| in emax and omax.
__device__ void newton_correction(const double* S, double* C, int N, int ld, float* Ef, float* Of, double* dsave,
                                  double& emax, double& omax) {
  const int64_t gt = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t gs = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t q = gt; q < static_cast<int64_t>(N) * N; q += gs) {
    const int i = static_cast<int>(q / N), j = static_cast<int>(q - static_cast<int64_t>(i) * N);
    const int64_t o = static_cast<int64_t>(i) * ld + j;
    double e = 0.0;
    const double sij = __ldcg(S + o);
    if (i != j) {
      const double den = __ldcg(S + static_cast<int64_t>(j) * ld + j) - __ldcg(S + static_cast<int64_t>(i) * ld + i);
      if (den != 0.0 && fabs(sij) <= 0.1 * fabs(den)) e = sij / den;
    }
    C[o] = e;
    emax = fmax(emax, fabs(e));
    if (i != j) omax = fmax(omax, fabs(sij));
    if (Ef) {
      Ef[o] = static_cast<float>(e);
      Of[o] = i != j ? static_cast<float>(sij) : 0.f;
      if (i == j) dsave[i] = sij;
    }
  }
}

// V (I + E + E^2 / 2) from the stored E (staged) and FP32 E^2 (read): the
// exponential of the antisymmetric E to second order, orthogonal to O(E^4).
struct ExpE {
  const float* E2;
  int ld;
  __device__ __forceinline__ double operator()(int k, int j, double e) const {
    return (k == j ? 1.0 : 0.0) + e + 0.5 * static_cast<double>(__ldcg(E2 + static_cast<int64_t>(k) * ld + j));
  }
};

// Grid-wide maximum of one value per CTA (same result in every CTA).  The
// per-CTA values go to slots of their own, alternating between two sets by
// the barrier count: a CTA that runs ahead cannot overwrite values another
// CTA is still reading, neither those of the check (slots 0..4G) nor those of
// the previous maximum when no barrier lies between the two.
__device__ bool grid_max(double v, double* red, LargeScratch<double>& L, unsigned& gen, int32_t* err, long long limit,
                         double& out) {
  const unsigned G = gridDim.x;
  double* slot = L.partial + (4 + (gen & 1)) * static_cast<size_t>(G);
  v = block_max(v, red);
  if (threadIdx.x == 0) slot[blockIdx.x] = v;
  if (!grid_barrier(L.bar, (++gen) * G, err, limit)) return false;
  double m = 0.0;
  for (unsigned c = threadIdx.x; c < G; c += blockDim.x) m = fmax(m, __ldcg(slot + c));
  out = block_max(m, red);
  return true;
}

// Exact plane rotations for the pairs the Newton step leaves alone
// (|b_lk| > 0.1 |b_ll - b_kk|: eigenvalues close enough that the change of
// W mixes their eigenvectors by a large angle).  Each row l proposes its
// largest such coupling b_lk, k < l (one warp per row); a proposal is taken
// when it is the largest of all proposals that share an index with it (ties
// to the smaller row), so the taken pairs are disjoint and their rotations
// commute.  Each rotation is the Jacobi rotation that zeroes b_lk (angle at
// most pi/4); V <- V Q and B <- Q^T B Q in place.  Pairs left out wait for
// the next pass.  `gb` holds 5 N doubles: proposals (value, column), then
// per index the rotation's cosine, partner coefficient and partner.
// Returns false if a grid wait expired.
__device__ bool pair_rotations(double* B, double* V, int N, int ld, double* gb, double* red, LargeScratch<double>& L,
                               unsigned& gen, int32_t* err, long long limit) {
  double* pv = gb;
  double* pk = gb + N;
  double* qc = gb + 2 * N;
  double* qs = gb + 3 * N;
  double* qp = gb + 4 * N;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  double found = 0.0;
  for (int64_t l = warp; l < N; l += nwarps) {
    const double bll = __ldcg(B + l * ld + l);
    double best = 0.0;
    int bk = -1;
    for (int k = lane; k < l; k += 32) {
      const double x = fabs(__ldcg(B + l * ld + k));
      const double den = fabs(__ldcg(B + static_cast<int64_t>(k) * ld + k) - bll);
      if (x > 0.1 * den && x > best) {  // NaN never qualifies
        best = x;
        bk = k;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
      if (ob > best || (ob == best && ok >= 0 && (bk < 0 || ok < bk))) {
        best = ob;
        bk = ok;
      }
    }
    if (lane == 0) {
      pv[l] = best;
      pk[l] = bk;
      qc[l] = 1.0;
      qs[l] = 0.0;
      qp[l] = static_cast<double>(l);
    }
    found = fmax(found, best);
  }
  double any = 0.0;
  if (!grid_max(found, red, L, gen, err, limit, any)) return false;
  if (!(any > 0.0)) return true;
  // a proposal (l, k) is taken when no other proposal touching l or k is larger
  for (int64_t l = warp; l < N; l += nwarps) {
    const int k = static_cast<int>(__ldcg(pk + l));
    if (k < 0) continue;  // warp-uniform
    const double v = __ldcg(pv + l);
    bool beaten = false;
    for (int m = lane; m < N; m += 32) {
      if (m == l) continue;
      const int km = static_cast<int>(__ldcg(pk + m));
      if (km < 0) continue;
      if (m == k || km == l || km == k) {
        const double vm = __ldcg(pv + m);
        if (vm > v || (vm == v && m < l)) beaten = true;
      }
    }
    if (__any_sync(0xffffffffu, beaten)) continue;
    if (lane == 0) {
      // Jacobi rotation of the 2 x 2 block (k, l): tau = (b_ll - b_kk) / (2 b_kl),
      // t = tan(theta) = sign(tau) / (|tau| + sqrt(1 + tau^2)), |t| <= 1
      const double bkk = __ldcg(B + static_cast<int64_t>(k) * ld + k), bll = __ldcg(B + l * ld + l);
      const double bkl = __ldcg(B + l * ld + k);
      const double tau = (bll - bkk) / (2.0 * bkl);
      const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      const double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
      // column k of V Q is c v_k - s v_l, column l is c v_l + s v_k
      qc[k] = c;
      qs[k] = -sn;
      qp[k] = static_cast<double>(l);
      qc[l] = c;
      qs[l] = sn;
      qp[l] = static_cast<double>(k);
    }
  }
  if (!grid_barrier(L.bar, (++gen) * gridDim.x, err, limit)) return false;
  const int64_t gt = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t gs = static_cast<int64_t>(gridDim.x) * blockDim.x;
  // V Q: each pair of columns once per row (j the smaller index)
  for (int64_t q = gt; q < static_cast<int64_t>(N) * N; q += gs) {
    const int r = static_cast<int>(q / N), j = static_cast<int>(q - static_cast<int64_t>(r) * N);
    const int pj = static_cast<int>(__ldcg(qp + j));
    if (pj <= j) continue;
    double* row = V + static_cast<int64_t>(r) * ld;
    const double x = __ldcg(row + j), y = __ldcg(row + pj);
    row[j] = __ldcg(qc + j) * x + __ldcg(qs + j) * y;
    row[pj] = __ldcg(qc + pj) * y + __ldcg(qs + pj) * x;
  }
  // Q^T B Q: the entries {i, p(i)} x {j, p(j)} together, by the thread of
  // the smaller index of each side; (Q^T B Q)_xy = sum_ab Q_ax B_ab Q_by with
  // Q_xx = qc[x] and Q_p(x)x = qs[x]
  for (int64_t q = gt; q < static_cast<int64_t>(N) * N; q += gs) {
    const int i = static_cast<int>(q / N), j = static_cast<int>(q - static_cast<int64_t>(i) * N);
    const int pi = static_cast<int>(__ldcg(qp + i)), pj = static_cast<int>(__ldcg(qp + j));
    if (pi < i || pj < j || (pi == i && pj == j)) continue;
    const int xs[2] = {i, pi}, ys[2] = {j, pj};
    const int nx = pi != i ? 2 : 1, ny = pj != j ? 2 : 1;
    double o[2][2], nv[2][2];
    for (int a = 0; a < nx; ++a)
      for (int b = 0; b < ny; ++b) o[a][b] = __ldcg(B + static_cast<int64_t>(xs[a]) * ld + ys[b]);
    for (int x = 0; x < nx; ++x)
      for (int y = 0; y < ny; ++y) {
        double acc = 0.0;
        for (int a = 0; a < nx; ++a) {
          const double qa = a == x ? __ldcg(qc + xs[x]) : __ldcg(qs + xs[x]);
          for (int b = 0; b < ny; ++b) {
            const double qb = b == y ? __ldcg(qc + ys[y]) : __ldcg(qs + ys[y]);
            acc += qa * o[a][b] * qb;
          }
        }
        nv[x][y] = acc;
      }
    for (int x = 0; x < nx; ++x)
      for (int y = 0; y < ny; ++y) B[static_cast<int64_t>(xs[x]) * ld + ys[y]] = nv[x][y];
  }
  return grid_barrier(L.bar, (++gen) * gridDim.x, err, limit);
}

// Leaves the block to the Jacobi kernel launched after this one: cold, or
// started from the eigenvectors in L.V.
__device__ void hand_over(LargeScratch<double>& L, bool warm) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    L.flags[0] = 0;
    L.flags[3] = 0;
    *L.warm = warm ? 1 : 0;
  }
}

// A warm attempt that gave up: the cold path (gather, reduction,
// eigenvectors, refinement) projects the block.  The next attempt waits 16
// iterations after a start far from converged (given up at the first check,
// which costs about one W V product) and 4 after a near miss (given up after
// one or two Newton passes).
__device__ void warm_abort(LargeScratch<double>& L, bool near) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    L.flags[0] = 0;
    L.flags[1] = near ? 4 : 16;
  }
}

// 256 threads at most 128 registers each (32 K of the SM's 64 K): the
// cooperative grid needs a CTA on every SM, and the small-block projections
// running beside it on another stream keep room for theirs (at 255
// registers each CTA filled its SM and waited for those to finish).
template <typename T>
__global__ void __maxnreg__(128) k_tri_recon(DevPlan<T> p, int bid, LargeScratch<double> L,
                                                         int warm_mode) {
  __shared__ double sA[2 * 16 * (kKC + 1)], sB[2 * kKC * (24 + 1)];
  __shared__ double red[40];
  const BlockDesc bd = p.blocks[bid];
  if (!p.active[bd.inst]) return;
  if (warm_mode) {
    // start from the previous iteration's eigenvectors (kept in L.V) when
    // they are there and no cool-down is running; otherwise leave the block
    // to the cold path launched after this kernel
    if (!(__ldcg(L.flags + 3) == 1 && __ldcg(L.flags + 1) == 0)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) L.flags[0] = 0;
      return;
    }
  } else if (L.tri_warm && __ldcg(L.flags) == 1) {
    return;  // the warm attempt of this iteration projected the block
  }
  const int N = bd.N, Np = N + (N & 1);
  const unsigned G = gridDim.x;
  unsigned gen = 0;
  int32_t* err = p.err;
  const double s_sm = p.st[bd.inst].s;
  const int64_t gt = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t gs = static_cast<int64_t>(G) * blockDim.x;

  // W, full and FP64
  for (int64_t q = gt; q < static_cast<int64_t>(N) * N; q += gs) {
    const int i = static_cast<int>(q / N), j = static_cast<int>(q - static_cast<int64_t>(i) * N);
    if (i < j) continue;
    const double w = d(proj_input(p, bd, packed_index(i, j, N), i != j, s_sm));
    const double wf = (i == j) ? w : w * 0.70710678118654752440;
    L.Wf[static_cast<int64_t>(i) * Np + j] = wf;
    L.Wf[static_cast<int64_t>(j) * Np + i] = wf;
  }
  // Vc alternates between L.V and L.B1; each pass makes it orthonormal to
  // the unit roundoff (Newton-Schulz V (3 I - V^T V) / 2), forms
  // B = Vc^T W Vc and checks the first-order projection of B; a failed check
  // takes one Newton correction of Vc and another pass (three at most)
  double* Vc = L.V;
  double* Vn = L.B1;
  int work = 0;  // refinement GEMM passes beyond the reconstruction (reported per block)
  bool fresh = false;  // B = V^T W V already updated for the current V (Rayleigh-quotient update)
  double rk0 = 0.0;     // the first check's largest same-sign coupling (warm attempts)
  for (int pass = 0;; ++pass) {
   if (!fresh) {
    // V^T V = I to the unit roundoff: a Newton-Schulz step takes the
    // largest deviation g to about (3/4) g^2 and ends it for g <= 3e-8; for
    // g <= 1.5e-5 (FP32 eigenvectors of separated eigenvalues) one
    // second-order step ends it; above that Newton-Schulz steps repeat with
    // a new V^T V.  Eigenvectors of close eigenvalues from separate inverse
    // iterations overlap by up to about eps_32 / gap (6e-4 for a gap of
    // 1e-5 |W|); a deviation above 0.25, or one that does not shrink, goes
    // to the Jacobi kernel from a cold start.
    double gm = 0.0;
    for (int ns = 0;; ++ns) {
      double rmax = 0.0;
      gemm_sym<true, false>(Vc, Vc, L.T1, N, Np, OrthMax{&rmax}, sA, sB);
      const double prev = gm;
      if (!grid_max(rmax, red, L, gen, err, p.wait_limit, gm)) return;
      if (!(gm <= 0.25) || (ns > 0 && !(gm < prev)) || ns == 6) {  // not converging
        if (warm_mode)
          warm_abort(L, pass > 0);
        else
          hand_over(L, false);
        return;
      }
      if (gm <= 1e-15) break;
      if (gm > 3e-8 && gm <= 1.5e-5) {
        // one second-order step V (I + E/2 + 3 E^2 / 8), E = I - V^T V
        // exact in FP64 from the stored V^T V: it leaves about
        // (5/16) g^3 <= 1e-15 where two first-order steps would take a
        // second V^T V and a second full product
        for (int64_t q = gt; q < static_cast<int64_t>(N) * Np; q += gs) {
          const int k = static_cast<int>(q / Np), j = static_cast<int>(q - static_cast<int64_t>(k) * Np);
          Vn[q] = j < N ? (k == j ? 1.0 : 0.0) - __ldcg(L.T1 + q) : 0.0;
        }
        if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
        // E^2 (E symmetric) in FP32: its entries are at most g^2 <= 2.3e-10,
        // so its rounding (about 1e-6 relative) stays below 1e-15
        gemm_sym<true, false, NoOp, float>(Vn, Vn, L.B0, N, Np, NoOp(), sA, sB);
        if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
        gemm_full<false, false>(Vc, L.B0, Vn, N, Np, NsFactor2{L.T1, Np}, sA, sB);
        if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
        double* t = Vc;
        Vc = Vn;
        Vn = t;
        work += 2;
        break;
      }
      // far from orthonormal the step's product may be FP32 (the next
      // V^T V measures the result again); the last step is FP64
      if (gm > 1.5e-5)
        gemm_corr(Vc, L.T1, Vn, N, Np, NsCorr(), reinterpret_cast<float*>(sA), reinterpret_cast<float*>(sB));
      else
        gemm_full<false, false>(Vc, L.T1, Vn, N, Np, NsFactor(), sA, sB);
      if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
      double* t = Vc;
      Vc = Vn;
      Vn = t;
      ++work;
      if (gm <= 3e-8) break;
    }
    gemm_full<false, false>(L.Wf, Vc, L.T1, N, Np, Ident(), sA, sB);
    if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
    gemm_sym<true, false>(Vc, L.T1, L.B0, N, Np, NoOp(), sA, sB);
    if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
   }
   fresh = false;

    // check of the first-order projection of B: a pair of diagonal entries
    // of opposite signs adds |b_lk|^2 / (|b_ll| + |b_kk|) at second order
    // (and its rotation angle must be small), a pair of the same sign adds
    // nothing unless its coupling can move an eigenvalue across zero
    // (|b_lk|^2 > 1e-6 |b_ll b_kk|)
    double angle = 0.0, second = 0.0, risky = 0.0, fro2 = 0.0;
    for (int64_t q = gt; q < static_cast<int64_t>(N) * N; q += gs) {
      const int i = static_cast<int>(q / N), j = static_cast<int>(q - static_cast<int64_t>(i) * N);
      if (i < j) continue;
      const double bij = __ldcg(L.B0 + static_cast<int64_t>(i) * Np + j);
      fro2 += (i == j ? 1.0 : 2.0) * bij * bij;
      if (i == j) continue;
      const double bi = __ldcg(L.B0 + static_cast<int64_t>(i) * Np + i);
      const double bj = __ldcg(L.B0 + static_cast<int64_t>(j) * Np + j);
      const double e = fabs(bij);
      if ((bi > 0.0) != (bj > 0.0)) {
        const double gsum = fabs(bi) + fabs(bj);
        angle = fmax(angle, e / gsum);
        second += e * e / gsum;
      } else if (e * e > 1e-6 * fabs(bi * bj)) {
        risky = fmax(risky, e);
      }
    }
    angle = (angle == angle) ? angle : 1e300;
    angle = block_max(angle, red);
    risky = block_max(risky, red);
    second = block_sum(second, red);
    fro2 = block_sum(fro2, red);
    if (threadIdx.x == 0) {
      L.partial[blockIdx.x] = angle;
      L.partial[G + blockIdx.x] = risky;
      L.partial[2 * G + blockIdx.x] = second;
      L.partial[3 * G + blockIdx.x] = fro2;
    }
    if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
    double a = 0.0, rk = 0.0, sc = 0.0, f2 = 0.0;
    for (unsigned c = threadIdx.x; c < G; c += blockDim.x) {
      a = fmax(a, __ldcg(L.partial + c));
      rk = fmax(rk, __ldcg(L.partial + G + c));
    }
    a = block_max(a, red);
    rk = block_max(rk, red);
    for (unsigned c = threadIdx.x; c < G; c += blockDim.x) {  // same order in every CTA
      sc += __ldcg(L.partial + 2 * G + c);
      f2 += __ldcg(L.partial + 3 * G + c);
    }
    sc = block_sum(sc, red);
    f2 = block_sum(f2, red);
    const double wn = sqrt(f2);
    if (a <= 1e-3 && rk <= 1e-13 * wn && sc <= 1e-14 * wn) break;
    if (pass == 0) rk0 = rk;
    if (warm_mode) {
      // Two Newton passes take a second-order sum s to about s^4 / |B|^3,
      // so a start above 1e-6 |B|_F cannot reach the check; an angle
      // beyond 0.05 meets the step's 0.1 clip; same-sign couplings of
      // close eigenvalues (a cluster the step leaves alone) stay where they
      // are, so a start above 1e-4 |B|_F, or a first pass that does not
      // halve them, does not converge either.
      const bool far = pass == 0 && (a > 0.05 || sc > 1e-6 * wn || rk > 1e-4 * wn);
      const bool stuck = pass == 1 && rk > 1e-13 * wn && rk > 0.5 * rk0;
      if (far || stuck || pass == 2) {
        warm_abort(L, !far);
        return;
      }
    }
    if (!warm_mode && pass == 2) {  // still not accurate: the Jacobi kernel finishes from these eigenvectors
      if (Vc != L.V)
        for (int64_t q = gt; q < static_cast<int64_t>(N) * Np; q += gs) L.V[q] = __ldcg(Vc + q);
      hand_over(L, true);
      return;
    }
    const size_t fs = static_cast<size_t>(N) * Np;  // one FP32 slot of L.F32
    float* F0 = L.F32;
    double* dsv = L.partial + 6 * G;
    if (!pair_rotations(L.B0, Vc, N, Np, dsv + N, red, L, gen, err, p.wait_limit)) return;
    double emax = 0.0, omax = 0.0;
    newton_correction(L.B0, L.T1, N, Np, F0, F0 ? F0 + fs : nullptr, dsv, emax, omax);
    // the update needs |E| <= 1e-5 and |O| <= 1e-4 |B|_F (so the FP32 terms
    // stay below 1e-15 |B|_F); one grid maximum decides both
    double eg;
    const double ratio = fmax(emax / 1e-5, omax / (1e-4 * wn));
    if (!grid_max(ratio == ratio ? ratio : 1e300, red, L, gen, err, p.wait_limit, eg)) return;
    if (F0 && eg <= 1.0) {
      // Rayleigh-quotient update for small E: V' = V M, M = I + C,
      // C = E + E^2/2 (orthogonal to O(E^4), so V' needs no new V^T V), and
      // B' = M^T B M = B + D C + (D C)^T + O C + (O C)^T + C^T (S C) with
      // B = D + O (diagonal, off-diagonal), S C = D C + O C.  The terms
      // O C and C^T S C (of order |O| |E| and |E|^2) go through FP32
      // products, the others stay FP64; W V and V^T W V are not formed again.
      float* Ef = F0;            // E (slot 0; later S C)
      float* Of = F0 + fs;       // O (slot 1; later C^T S C)
      float* E2 = F0 + 2 * fs;   // E^2
      float* Cf = F0 + 3 * fs;   // C
      float* OC = F0 + 4 * fs;   // O C
      float* sAf = reinterpret_cast<float*>(sA);
      float* sBf = reinterpret_cast<float*>(sB);
      gemm_full<false, false>(Ef, Ef, E2, N, Np, Ident(), sAf, sBf);
      if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
      gemm_full<false, false>(Vc, L.T1, Vn, N, Np, ExpE{E2, Np}, sA, sB);
      for (int64_t q = gt; q < fs; q += gs) Cf[q] = __ldcg(Ef + q) + 0.5f * __ldcg(E2 + q);
      if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
      gemm_full<false, false>(Of, Cf, OC, N, Np, Ident(), sAf, sBf);
      if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
      float* SC = Ef;
      for (int64_t q = gt; q < static_cast<int64_t>(N) * N; q += gs) {
        const int i = static_cast<int>(q / N), j = static_cast<int>(q - static_cast<int64_t>(i) * N);
        const int64_t o = static_cast<int64_t>(i) * Np + j;
        SC[o] = static_cast<float>(__ldcg(dsv + i)) * __ldcg(Cf + o) + __ldcg(OC + o);
      }
      if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
      float* CSC = Of;
      gemm_full<true, false>(Cf, SC, CSC, N, Np, Ident(), sAf, sBf);
      if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
      for (int64_t q = gt; q < static_cast<int64_t>(N) * N; q += gs) {
        const int i = static_cast<int>(q / N), j = static_cast<int>(q - static_cast<int64_t>(i) * N);
        const int64_t o = static_cast<int64_t>(i) * Np + j, ot = static_cast<int64_t>(j) * Np + i;
        const double cij = __ldcg(L.T1 + o) + 0.5 * static_cast<double>(__ldcg(E2 + o));
        const double cji = __ldcg(L.T1 + ot) + 0.5 * static_cast<double>(__ldcg(E2 + ot));
        const double small = static_cast<double>(__ldcg(OC + o)) + static_cast<double>(__ldcg(OC + ot)) +
                             static_cast<double>(__ldcg(CSC + o));
        L.B0[o] = __ldcg(L.B0 + o) + __ldcg(dsv + i) * cij + __ldcg(dsv + j) * cji + small;
      }
      if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
      fresh = true;
    } else {
      // V (I + E), E in FP32: the next pass orthonormalises the result and
      // measures V^T W V again in FP64
      gemm_corr(Vc, L.T1, Vn, N, Np, Ident(), reinterpret_cast<float*>(sA), reinterpret_cast<float*>(sB));
      if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
    }
    double* t = Vc;
    Vc = Vn;
    Vn = t;
    work += 2;
  }
  // T1 = V M with M the first-order projection of B, then U = T1 V^T on the
  // lower triangle; u = svec(U), v = u - W
  {  // M once into the free V buffer (one division per entry, not one per
     // staging of the entry by every tile row), then T1 = V M
    const FirstOrder fo{L.B0, Np};
    for (int64_t q = gt; q < static_cast<int64_t>(N) * Np; q += gs) {
      const int k = static_cast<int>(q / Np), j = static_cast<int>(q - static_cast<int64_t>(k) * Np);
      Vn[q] = j < N ? fo(k, j, __ldcg(L.B0 + q)) : 0.0;
    }
  }
  if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
  gemm_full<false, false>(Vc, Vn, L.T1, N, Np, Ident(), sA, sB);
  if (!grid_barrier(L.bar, (++gen) * G, err, p.wait_limit)) return;
  auto emit = [&](int ii, int jj, double x) {
    const int64_t kk = packed_index(ii, jj, N);
    const T w = proj_input(p, bd, kk, ii != jj, s_sm);
    const T u = (ii != jj) ? static_cast<T>(x * kSqrt2) : static_cast<T>(x);
    p.ux[bd.x_off + kk] = u;
    const T vv = u - w;
    p.vx[bd.x_off + kk] = vv;
    if (bd.kind == kWeighted) p.wl[bd.lr_first + kk] = d(u) + d(vv);  // w1_hat of the next iteration (c = 0)
  };
  gemm_sym<false, true>(L.T1, Vc, static_cast<double*>(nullptr), N, Np, emit, sA, sB);
  // keep V for the next iteration's warm attempt (L.V last held M, which the
  // product above has consumed)
  if (L.tri_warm && Vc != L.V)
    for (int64_t q = gt; q < static_cast<int64_t>(N) * Np; q += gs) L.V[q] = __ldcg(Vc + q);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    L.flags[0] = 1;
    L.flags[3] = 1;
    if (warm_mode) {
      L.flags[1] = 0;  // stay warm
    } else if (L.flags[4] == 0) {
      L.flags[4] = 1;  // first cold projection: the first attempt waits 16 iterations
      L.flags[1] = 16;
    } else if (L.flags[1] > 0) {
      --L.flags[1];
    }
    *L.sweeps_out = 0;
    p.blk_sweeps[bid] = work;
    *L.warm = 0;
  }
}

size_t tri_reduce_smem(int N) {
  return sizeof(float) * (static_cast<size_t>(N) * ((N + 3) & ~3) + kTriPcol + kTriRows);
}


}  // namespace

cudaError_t launch_psd_tri_part(const DevPlan<double>& p, int bid, int N, const LargeScratch<double>& L, int grid,
                                int part, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  switch (part) {
    case 0:
      k_tri_gather<double><<<kGatherCtas, 256, 0, s>>>(p, bid, L);
      return cudaGetLastError();
    case 1: {
      const size_t sm1 = tri_reduce_smem(N);
      e = cudaFuncSetAttribute(k_tri_reduce<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm1));
      if (e != cudaSuccess) return e;
      k_tri_reduce<double><<<1, kTriThreads, sm1, s>>>(p, bid, L);
      return cudaGetLastError();
    }
    case 2: {
      const size_t sm2 = tri_vectors_smem(N);
      e = cudaFuncSetAttribute(k_tri_vectors, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm2));
      if (e != cudaSuccess) return e;
      k_tri_vectors<<<(N + kVecThreads / 32 - 1) / (kVecThreads / 32), kVecThreads, sm2, s>>>(p, bid, L);
      return cudaGetLastError();
    }
    case 3:
    case 4: {  // 3: refinement after the cold path; 4: warm attempt from the previous eigenvectors
      const int warm_mode = part == 4 ? 1 : 0;
      e = cudaMemsetAsync(L.bar, 0, 2 * sizeof(uint32_t), s);
      if (e != cudaSuccess) return e;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(grid);
      cfg.blockDim = dim3(kRecBlock);
      cfg.dynamicSmemBytes = 0;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, k_tri_recon<double>, p, bid, L, warm_mode);
    }
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_psd_tri(const DevPlan<double>& p, int bid, int N, const LargeScratch<double>& L, int grid,
                           cudaStream_t s) {
  if (L.tri_warm) {
    const cudaError_t e = launch_psd_tri_part(p, bid, N, L, grid, 4, s);
    if (e != cudaSuccess) return e;
  }
  for (int part = 0; part < 4; ++part) {
    const cudaError_t e = launch_psd_tri_part(p, bid, N, L, grid, part, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sos
