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
//                  counts of T brackets lambda_i, inverse iteration with
//                  Rayleigh shifts on T gives its eigenvector z_i, and the
//                  reflectors map it back: v_i = Q z_i.
//   k_tri_recon    cooperative grid, FP64 products: V made orthonormal to the
//                  unit roundoff (Newton-Schulz V (3I - V^T V) / 2),
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
// eigenvalues of both signs crowd it.  If V is not even FP32-orthonormal, or
// three passes do not pass the check, the grid Jacobi kernel launched after
// this one takes the block over (flag word 0; started from V when V is
// orthonormal).
#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "dev_common.cuh"
#include "kernels.h"

namespace sos {
namespace {

constexpr int kTriThreads = 1024;  // reduction CTA
constexpr int kVecThreads = 256;   // one CTA per eigenvector
constexpr int kRecThreads = 128;   // reconstruction CTAs
constexpr int kTriSlots = (kTriMaxN + 31) / 32;  // per-lane register slots of a length-N vector

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
// with A22 the trailing block A[k+1.., k+1..].  Only the lower triangle is
// kept (row-major, odd leading dimension, so that a row and a column of it
// are both read without shared-memory bank conflicts).  Warp w owns the rows
// r = w (mod 32) of the product and of the update, its lanes the columns
// c = lane (mod 32); every warp forms the reflector itself from the column
// (held in registers), and the update also sums the squares of the next
// column, so a step needs two barriers.
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

template <typename T>
__global__ void __launch_bounds__(kTriThreads, 1) k_tri_reduce(DevPlan<T> p, int bid, LargeScratch<double> L) {
  static_assert(kTriSlots == 8, "the row reduction handles eight rows per warp");
  extern __shared__ __align__(16) float tsm[];
  __shared__ double redd[40];
  __shared__ float sg_part[32];
  const BlockDesc bd = p.blocks[bid];
  if (!p.active[bd.inst]) return;
  const int N = bd.N, LD = N | 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* A = tsm;
  float* pp = A + static_cast<size_t>(N) * LD;
  const TriOut out = tri_out(L.B0, N);
  const double s_sm = p.st[bd.inst].s;

  // the lower triangle in FP32 (column j by warp j mod 32, coalesced over the
  // packed column), |W|_F in FP64, then the scaling by 1 / |W|_F
  double nrm2 = 0.0;
  for (int j = warp; j < N; j += 32) {
    const int64_t base = packed_index(j, j, N);
#pragma unroll 4
    for (int i = j + lane; i < N; i += 32) {
      const double w = d(proj_input(p, bd, base + (i - j), i != j, s_sm));
      nrm2 += w * w;  // packed entries carry sqrt(2): w^2 counts both halves
      A[i * LD + j] = static_cast<float>(i == j ? w : w * 0.70710678118654752440);
    }
  }
  nrm2 = block_sum(nrm2, redd);
  {
    const float scale = nrm2 > 0.0 ? static_cast<float>(1.0 / sqrt(nrm2)) : 1.f;
    float sg = 0.f;
    for (int j = warp; j < N; j += 32)
      for (int i = j + lane; i < N; i += 32) {
        const float x = A[i * LD + j] * scale;
        A[i * LD + j] = x;
        if (j == 0 && i >= 2) sg = fmaf(x, x, sg);  // squares of column 0 below the subdiagonal
      }
    sg = warp_sum_f(sg);
    if (lane == 0) sg_part[warp] = sg;
  }
  __syncthreads();

  for (int k = 0; k < N - 2; ++k) {
    const int m = N - k - 1;
    float* A22 = A + (k + 1) * LD + (k + 1);  // A22[r * LD + c], r >= c
    const float* col = A + (k + 1) * LD + k;  // col[r * LD] = A[k+1+r][k]
    // the reflector (the same arithmetic in every warp)
    const float s2 = warp_sum_f(sg_part[lane]);
    const float alpha = col[0];
    float tau = 0.f, beta = alpha, sc = 0.f;
    if (s2 > 0.f) {
      beta = -copysignf(sqrtf(fmaf(alpha, alpha, s2)), alpha);
      tau = (beta - alpha) / beta;
      sc = 1.f / (alpha - beta);
    }
    if (tid == 0) {
      out.d[k] = A[k * LD + k];
      out.e[k] = beta;
      out.tau[k] = tau;
    }
    if (tau == 0.f) {  // H_k = I: only the squares of the next column
      float sg = 0.f;
      for (int r = 2 + tid; r < m; r += kTriThreads) sg = fmaf(A22[r * LD], A22[r * LD], sg);
      __syncthreads();  // every warp has read sg_part
      sg = warp_sum_f(sg);
      if (lane == 0) sg_part[warp] = sg;
      __syncthreads();
      continue;
    }
    float vr[kTriSlots];
#pragma unroll
    for (int q = 0; q < kTriSlots; ++q) {
      const int c = lane + 32 * q;
      vr[q] = c == 0 ? 1.f : (c < m ? col[c * LD] * sc : 0.f);
    }
    if (warp < kTriSlots) {  // reflector k for the back-transformation: entries k + 2 ..
      const int c = lane + 32 * warp;
      if (c >= 1 && c < m) out.U[static_cast<int64_t>(k) * N + k + 1 + c] = vr[warp];
    }
    // p = tau A22 v for the rows r = warp + 32 i; slots of 32 columns wholly
    // on or below the diagonal read a row, wholly above it a column
    {
      float acc[kTriSlots];
#pragma unroll
      for (int i = 0; i < kTriSlots; ++i) {
        acc[i] = 0.f;
        const int r = warp + 32 * i;
        if (r < m) {
#pragma unroll
          for (int q = 0; q < kTriSlots; ++q) {
            const int c = lane + 32 * q;
            if (32 * q + 31 <= r) {
              acc[i] = fmaf(A22[r * LD + c], vr[q], acc[i]);
            } else if (32 * q > r) {
              if (32 * q < m && c < m) acc[i] = fmaf(A22[c * LD + r], vr[q], acc[i]);
            } else if (c < m) {
              acc[i] = fmaf(c <= r ? A22[r * LD + c] : A22[c * LD + r], vr[q], acc[i]);
            }
          }
        }
      }
      const float tot = warp_sum8(acc, lane);
      const int r = warp + 32 * ((lane >> 2) & 7);
      if ((lane & 3) == 0 && r < m) pp[r] = tau * tot;
    }
    __syncthreads();
    // w = p - (tau / 2)(p^T v) v (every warp forms p^T v itself)
    float wr[kTriSlots];
    float pv = 0.f;
#pragma unroll
    for (int q = 0; q < kTriSlots; ++q) {
      const int c = lane + 32 * q;
      wr[q] = c < m ? pp[c] : 0.f;
      pv = fmaf(wr[q], vr[q], pv);
    }
    const float K = -0.5f * tau * warp_sum_f(pv);
#pragma unroll
    for (int q = 0; q < kTriSlots; ++q) wr[q] = fmaf(K, vr[q], wr[q]);
    // A22 <- A22 - v w^T - w v^T on the lower triangle; squares of its column 0 (the next reflector's)
    float sg = 0.f;
#pragma unroll
    for (int i = 0; i < kTriSlots; ++i) {
      const int r = warp + 32 * i;
      if (r < m) {
        const float vrr = __shfl_sync(0xffffffffu, vr[i], warp), wrr = __shfl_sync(0xffffffffu, wr[i], warp);
#pragma unroll
        for (int q = 0; q < kTriSlots; ++q) {
          const int c = lane + 32 * q;
          if (32 * q > r) continue;
          if (32 * q + 31 <= r || c <= r) {
            float* a = A22 + r * LD + c;
            const float x = fmaf(-vrr, wr[q], fmaf(-wrr, vr[q], *a));
            *a = x;
            if (q == 0 && c == 0 && r >= 2) sg = fmaf(x, x, sg);
          }
        }
      }
    }
    sg = warp_sum_f(sg);
    if (lane == 0) sg_part[warp] = sg;
    __syncthreads();
  }
  if (tid == 0) {
    out.d[N - 2] = A[(N - 2) * LD + N - 2];
    out.d[N - 1] = A[(N - 1) * LD + N - 1];
    out.e[N - 2] = A[(N - 1) * LD + N - 2];
    out.e[N - 1] = 0.f;
    out.tau[N - 2] = 0.f;
    out.tau[N - 1] = 0.f;
  }
}

// ---------------------------------------------------------------------------
// Eigenvector i of T, mapped back by the reflectors (one CTA per eigenvalue,
// FP32: on this GPU a dependent FP64 operation takes 64 cycles and an FP64
// division several hundred, so every sequential recurrence here is FP32 and
// the FP64 accuracy comes from the refinement of the reconstruction kernel).
// ---------------------------------------------------------------------------

// Number of eigenvalues of T below x (Sturm sequence of the LDL^T pivots;
// a pivot of magnitude below pivmin is replaced by -pivmin).
__device__ __forceinline__ int sturm_count(const float* d, const float* e2, int N, float x, float pivmin) {
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int c = q < 0.f;
  for (int k = 1; k < N; ++k) {
    q = (d[k] - x) - __fdividef(e2[k - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
  }
  return c;
}

// Deterministic start vector entries in (-1, 1).
__device__ __forceinline__ float start_entry(int i, int j) {
  uint32_t h = static_cast<uint32_t>(i) * 0x9E3779B1u ^ (static_cast<uint32_t>(j) + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  return (static_cast<float>(h & 0xFFFFFFu) + 0.5f) / 8388608.0f - 1.0f;
}

__global__ void __launch_bounds__(kVecThreads) k_tri_vectors(DevPlan<double> p, int bid, LargeScratch<double> L) {
  extern __shared__ __align__(16) float vsm[];
  __shared__ float s_g[3][kVecThreads / 32];
  const BlockDesc bd = p.blocks[bid];
  if (!p.active[bd.inst]) return;
  const int N = bd.N;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nw = kVecThreads / 32;
  const TriOut out = tri_out(L.B0, N);
  float* df = vsm;       // diagonal of T
  float* ef = df + N;    // subdiagonal, split entries zeroed
  float* e2f = ef + N;   // its squares
  float* tau_s = e2f + N;
  float* z = tau_s + N + warp * 5 * N;  // this warp's eigenvector of T and
  float* rinv = z + N;   // the pivoted LU of T - sigma I: reciprocal pivots,
  float* du = rinv + N;  // first and second superdiagonal of U,
  float* du2 = du + N;
  float* dl = du2 + N;   // multipliers
  int* piv = reinterpret_cast<int*>(tau_s + N + nw * 5 * N) + warp * N;

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
  for (int k = tid; k < N; k += kVecThreads) {
    float ek = k < N - 1 ? out.e[k] : 0.f;
    if (fabsf(ek) <= split) ek = 0.f;
    df[k] = out.d[k];
    ef[k] = ek;
    e2f[k] = ek * ek;
    tau_s[k] = out.tau[k];
  }
  __syncthreads();
  const int i = blockIdx.x * nw + warp;  // this warp's eigenvalue (ascending order)
  if (i >= N) return;

  // bisection: 32 points per pass, keeping count(lo) <= i < count(hi)
  const float pivmin = 1e-30f;
  float lo = glo - 1e-6f * tn - 1e-30f, hi = ghi + 1e-6f * tn + 1e-30f;
  for (int pass = 0; pass < 5; ++pass) {
    const float x = lo + (hi - lo) * (static_cast<float>(lane + 1) / 33.f);
    const int c = sturm_count(df, e2f, N, x, pivmin);
    float nlo = c <= i ? x : -FLT_MAX;
    float nhi = c >= i + 1 ? x : FLT_MAX;
    for (int o = 16; o > 0; o >>= 1) {
      nlo = fmaxf(nlo, __shfl_xor_sync(0xffffffffu, nlo, o));
      nhi = fminf(nhi, __shfl_xor_sync(0xffffffffu, nhi, o));
    }
    if (nlo > lo && nlo < hi) lo = nlo;
    if (nhi < hi && nhi > lo) hi = nhi;
  }

  // lane 0: the unreduced block of T that holds eigenvalue i, then inverse
  // iteration on it with Rayleigh-quotient shifts kept by the bracket
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
    int run = 0, b0 = 0, b1 = N - 1, start = 0, cl = 0, ch = 0;
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
    for (int k = 0; k < N; ++k) z[k] = 0.f;
    if (b1 == b0) {
      z[b0] = 1.f;
    } else {
      const float tiny = 1.2e-7f * tn + 1e-30f;
      const float wid = (hi - lo) + 1e-6f * tn;
      float sigma = 0.5f * (lo + hi);
      float nrm = 0.f;
      for (int k = b0; k <= b1; ++k) {
        z[k] = start_entry(i, k);
        nrm = fmaf(z[k], z[k], nrm);
      }
      nrm = rsqrtf(nrm);
      for (int k = b0; k <= b1; ++k) z[k] *= nrm;
      for (int it = 0; it < 3; ++it) {
        // LU with partial pivoting of T_b - sigma I
        float dk = df[b0] - sigma, uk = ef[b0];
        for (int k = b0; k < b1; ++k) {
          const float lk = ef[k], dn = df[k + 1] - sigma, un = k + 1 < b1 ? ef[k + 1] : 0.f;
          if (fabsf(dk) >= fabsf(lk)) {
            const float pv = fabsf(dk) < tiny ? (dk < 0.f ? -tiny : tiny) : dk;
            const float r = __fdividef(1.f, pv);
            const float l = lk * r;
            piv[k] = 0;
            rinv[k] = r;
            du[k] = uk;
            du2[k] = 0.f;
            dl[k] = l;
            dk = fmaf(-l, uk, dn);
            uk = un;
          } else {  // rows k and k + 1 exchanged
            const float r = __fdividef(1.f, lk);
            const float l = dk * r;
            piv[k] = 1;
            rinv[k] = r;
            du[k] = dn;
            du2[k] = un;
            dl[k] = l;
            dk = fmaf(-l, dn, uk);
            uk = -l * un;
          }
        }
        rinv[b1] = __fdividef(1.f, fabsf(dk) < tiny ? (dk < 0.f ? -tiny : tiny) : dk);
        // L U y = z: forward with the exchanges, then backward
        float zk = z[b0];
        for (int k = b0; k < b1; ++k) {
          const float zn = z[k + 1];
          if (piv[k]) {
            z[k] = zn;
            zk = fmaf(-dl[k], zn, zk);
          } else {
            z[k] = zk;
            zk = fmaf(-dl[k], zk, zn);
          }
        }
        float y2 = 0.f, y1 = zk * rinv[b1];
        z[b1] = y1;
        nrm = y1 * y1;
        for (int k = b1 - 1; k >= b0; --k) {
          const float y = (z[k] - du[k] * y1 - du2[k] * y2) * rinv[k];
          z[k] = y;
          nrm = fmaf(y, y, nrm);
          y2 = y1;
          y1 = y;
        }
        nrm = rsqrtf(nrm);
        float rq = 0.f, prev = 0.f;
        for (int k = b0; k <= b1; ++k) {
          const float zz = z[k] * nrm;
          z[k] = zz;
          rq = fmaf(df[k] * zz, zz, rq);
          if (k > b0) rq = fmaf(2.f * ef[k - 1] * prev, zz, rq);
          prev = zz;
        }
        if (rq > lo - wid && rq < hi + wid) sigma = rq;  // Rayleigh quotient z^T T z as the next shift
      }
    }
  }
  __syncwarp();

  // v_i = H_0 H_1 ... H_{N-3} z; lane l holds entries l + 32 s, and the next
  // reflector's entries are loaded while the current one is applied
  float zr[kTriSlots], un[kTriSlots];
#pragma unroll
  for (int s = 0; s < kTriSlots; ++s) {
    const int j = lane + 32 * s;
    zr[s] = j < N ? z[j] : 0.f;
  }
  auto fetch = [&](int k, float (&u)[kTriSlots]) {
    const float* Uk = out.U + static_cast<int64_t>(k > 0 ? k : 0) * N;
#pragma unroll
    for (int s = 0; s < kTriSlots; ++s) {
      const int j = lane + 32 * s;
      u[s] = (k >= 0 && j >= k + 2 && j < N) ? __ldcg(Uk + j) : 0.f;
    }
  };
  fetch(N - 3, un);
  for (int k = N - 3; k >= 0; --k) {
    float ur[kTriSlots];
#pragma unroll
    for (int s = 0; s < kTriSlots; ++s) ur[s] = un[s];
    fetch(k - 1, un);
    const float tau = tau_s[k];
    if (tau == 0.f) continue;  // H_k = I
    float dsum = 0.f;
#pragma unroll
    for (int s = 0; s < kTriSlots; ++s) {
      const int j = lane + 32 * s;
      if (j == k + 1) ur[s] = 1.f;
      dsum = fmaf(ur[s], zr[s], dsum);
    }
    dsum = tau * warp_sum_f(dsum);
#pragma unroll
    for (int s = 0; s < kTriSlots; ++s) zr[s] = fmaf(-dsum, ur[s], zr[s]);
  }
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
// dimension ld, 128 threads; thread t computes row t % TM and the columns
// t / TM + 8 q.  op(X) = X^T where the flag is set.  xb(k, j, x) maps an
// element of op(B) as it is staged.  The next K chunk is loaded into
// registers while the current one is multiplied.
template <int TM, int TN, bool TA, bool TB, class XB>
__device__ __forceinline__ void gemm_tile(const double* A, const double* B, int ld, int n, int i0, int j0, XB xb,
                                          double (&acc)[TM * TN / kRecThreads], double* sA, double* sB) {
  constexpr int PT = TM * TN / kRecThreads;
  constexpr int LA = TM * kKC / kRecThreads, LB = kKC * TN / kRecThreads;
  static_assert(LA * kRecThreads == TM * kKC && LB * kRecThreads == kKC * TN, "tile shape");
  const int t = threadIdx.x, r = t % TM, g = t / TM;
  double ra[LA], rb[LB];
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
                  : 0.0;
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
                  : 0.0;
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
      sA[ii * (kKC + 1) + kk] = ra[u];
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
      sB[kk * (TN + 1) + jj] = (gj < n && gk < n) ? xb(gk, gj, rb[u]) : 0.0;
    }
  };
#pragma unroll
  for (int q = 0; q < PT; ++q) acc[q] = 0.0;
  load(0);
  for (int k0 = 0; k0 < n; k0 += kKC) {
    store(k0);
    __syncthreads();
    if (k0 + kKC < n) load(k0 + kKC);
#pragma unroll
    for (int kk = 0; kk < kKC; ++kk) {
      const double a = sA[r * (kKC + 1) + kk];
#pragma unroll
      for (int q = 0; q < PT; ++q) acc[q] = fma(a, sB[kk * (TN + 1) + g + 8 * q], acc[q]);
    }
    __syncthreads();
  }
}

struct Ident {
  __device__ __forceinline__ double operator()(int, int, double x) const { return x; }
};

// I + X for a stored correction X (X = E of the refinement step).
struct PlusIdent {
  __device__ __forceinline__ double operator()(int k, int j, double x) const { return (k == j ? 1.0 : 0.0) + x; }
};

// Newton-Schulz factor (3 I - V^T V) / 2 from the stored V^T V.
struct NsFactor {
  __device__ __forceinline__ double operator()(int k, int j, double x) const {
    return (k == j ? 1.5 : 0.0) - 0.5 * x;
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

// Lower-triangle tile index -> (ti, tj), ti >= tj.
__device__ __forceinline__ void lower_tile(int t, int& ti, int& tj) {
  ti = static_cast<int>((sqrtf(8.0f * static_cast<float>(t) + 1.0f) - 1.0f) * 0.5f);
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  while (ti * (ti + 1) / 2 > t) --ti;
  tj = t - ti * (ti + 1) / 2;
}

// C = op(A) op(B) over all 16 x 24 tiles (full) into C.
template <bool TA, bool TB, class XB>
__device__ void gemm_full(const double* A, const double* B, double* C, int N, int ld, XB xb, double* sA, double* sB) {
  const int ntn = (N + 23) / 24, nfull = ((N + 15) / 16) * ntn;
  for (int t = blockIdx.x; t < nfull; t += gridDim.x) {
    const int ti = t / ntn, tj = t - ti * ntn;
    double acc[3];
    gemm_tile<16, 24, TA, TB>(A, B, ld, N, ti * 16, tj * 24, xb, acc, sA, sB);
    const int r = threadIdx.x % 16, g = threadIdx.x / 16;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int ii = ti * 16 + r, jj = tj * 24 + g + 8 * q;
      if (ii < N && jj < N) C[static_cast<int64_t>(ii) * ld + jj] = acc[q];
    }
  }
}

// Symmetric C = op(A) op(B) over the lower 16 x 16 tiles, mirrored; f(i, j,
// c) sees each lower entry (i >= j) once.
template <bool TA, bool TB, class F>
__device__ void gemm_sym(const double* A, const double* B, double* C, int N, int ld, F f, double* sA, double* sB) {
  const int nt = (N + 15) / 16, nlow = nt * (nt + 1) / 2;
  for (int t = blockIdx.x; t < nlow; t += gridDim.x) {
    int ti, tj;
    lower_tile(t, ti, tj);
    double acc[2];
    gemm_tile<16, 16, TA, TB>(A, B, ld, N, ti * 16, tj * 16, Ident(), acc, sA, sB);
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
__device__ void newton_correction(const double* S, double* C, int N, int ld) {
  const int64_t gt = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t gs = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t q = gt; q < static_cast<int64_t>(N) * N; q += gs) {
    const int i = static_cast<int>(q / N), j = static_cast<int>(q - static_cast<int64_t>(i) * N);
    const int64_t o = static_cast<int64_t>(i) * ld + j;
    double e = 0.0;
    if (i != j) {
      const double den = __ldcg(S + static_cast<int64_t>(j) * ld + j) - __ldcg(S + static_cast<int64_t>(i) * ld + i);
      const double sij = __ldcg(S + o);
      if (den != 0.0 && fabs(sij) <= 0.1 * fabs(den)) e = sij / den;
    }
    C[o] = e;
  }
}

// Grid-wide maximum of one value per CTA (same result in every CTA).
__device__ bool grid_max(double v, double* red, LargeScratch<double>& L, unsigned& gen, int32_t* err, double& out) {
  v = block_max(v, red);
  if (threadIdx.x == 0) L.partial[blockIdx.x] = v;
  if (!grid_barrier(L.bar, (++gen) * gridDim.x, err)) return false;
  double m = 0.0;
  for (unsigned c = threadIdx.x; c < gridDim.x; c += blockDim.x) m = fmax(m, __ldcg(L.partial + c));
  out = block_max(m, red);
  return true;
}

// Leaves the block to the Jacobi kernel launched after this one: cold, or
// started from the eigenvectors in L.V.
__device__ void hand_over(LargeScratch<double>& L, bool warm) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    L.flags[0] = 0;
    *L.warm = warm ? 1 : 0;
  }
}

template <typename T>
__global__ void __launch_bounds__(kRecThreads) k_tri_recon(DevPlan<T> p, int bid, LargeScratch<double> L) {
  __shared__ double sA[16 * (kKC + 1)], sB[kKC * (24 + 1)];
  __shared__ double red[40];
  const BlockDesc bd = p.blocks[bid];
  if (!p.active[bd.inst]) return;
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
  for (int pass = 0;; ++pass) {
    double rmax = 0.0;
    gemm_sym<true, false>(Vc, Vc, L.T1, N, Np, OrthMax{&rmax}, sA, sB);
    double gm;
    if (!grid_max(rmax, red, L, gen, err, gm)) return;
    if (!(gm <= 1e-3)) {  // not even FP32-orthonormal
      hand_over(L, false);
      return;
    }
    if (gm > 1e-15) {
      gemm_full<false, false>(Vc, L.T1, Vn, N, Np, NsFactor(), sA, sB);
      if (!grid_barrier(L.bar, (++gen) * G, err)) return;
      double* t = Vc;
      Vc = Vn;
      Vn = t;
      ++work;
    }
    gemm_full<false, false>(L.Wf, Vc, L.T1, N, Np, Ident(), sA, sB);
    if (!grid_barrier(L.bar, (++gen) * G, err)) return;
    gemm_sym<true, false>(Vc, L.T1, L.B0, N, Np, NoOp(), sA, sB);
    if (!grid_barrier(L.bar, (++gen) * G, err)) return;

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
    if (!grid_barrier(L.bar, (++gen) * G, err)) return;
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
    if (pass == 2) {  // still not accurate: the Jacobi kernel finishes from these eigenvectors
      if (Vc != L.V)
        for (int64_t q = gt; q < static_cast<int64_t>(N) * Np; q += gs) L.V[q] = __ldcg(Vc + q);
      hand_over(L, true);
      return;
    }
    newton_correction(L.B0, L.T1, N, Np);
    if (!grid_barrier(L.bar, (++gen) * G, err)) return;
    gemm_full<false, false>(Vc, L.T1, Vn, N, Np, PlusIdent(), sA, sB);
    if (!grid_barrier(L.bar, (++gen) * G, err)) return;
    double* t = Vc;
    Vc = Vn;
    Vn = t;
    work += 2;
  }
  // T1 = V M with M the first-order projection of B, then U = T1 V^T on the
  // lower triangle; u = svec(U), v = u - W
  gemm_full<false, false>(Vc, L.B0, L.T1, N, Np, FirstOrder{L.B0, Np}, sA, sB);
  if (!grid_barrier(L.bar, (++gen) * G, err)) return;
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
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    L.flags[0] = 1;
    *L.sweeps_out = 0;
    p.blk_sweeps[bid] = work;
    *L.warm = 0;
  }
}

size_t tri_reduce_smem(int N) { return sizeof(float) * (static_cast<size_t>(N) * (N | 1) + kTriMaxN); }

size_t tri_vectors_smem(int N) {
  return (sizeof(float) * (4 + 5 * (kVecThreads / 32)) + sizeof(int) * (kVecThreads / 32)) * static_cast<size_t>(N);
}

}  // namespace

cudaError_t launch_psd_tri(const DevPlan<double>& p, int bid, int N, const LargeScratch<double>& L, int grid,
                           cudaStream_t s) {
  const size_t sm1 = tri_reduce_smem(N), sm2 = tri_vectors_smem(N);
  cudaError_t e = cudaFuncSetAttribute(k_tri_reduce<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sm1));
  if (e != cudaSuccess) return e;
  k_tri_reduce<double><<<1, kTriThreads, sm1, s>>>(p, bid, L);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_tri_vectors, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm2));
  if (e != cudaSuccess) return e;
  k_tri_vectors<<<(N + kVecThreads / 32 - 1) / (kVecThreads / 32), kVecThreads, sm2, s>>>(p, bid, L);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(L.bar, 0, 2 * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kRecThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_tri_recon<double>, p, bid, L);
}

}  // namespace sos
