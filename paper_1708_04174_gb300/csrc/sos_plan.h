// Internal data layout of libsos (host setup <-> device kernels).
//
// A "problem set" concatenates every instance of a batch:
//   x vectors  (u_xi, v_z)  : NX = sum_i n_x(i)  entries, instance-major
//   y vectors  (u_y, v_s)   : M  = sum_i m(i)
//   low-rank columns        : TL = sum_i t_eff(i)  (free u first, then the
//                             packed entries of weighted blocks)
// Per instance, x = [u (t); svec X_1; svec X_2; ...] with the packed order of
// include/sos.h.
//
// Column classes (Prop. 1, Prop. 3): an entry of a plain Gram block has one
// nonzero, at row ent_row[e] with coefficient 1 (diagonal) or sqrt(2)
// (off-diagonal, svec scaling).  Free variables and weighted-block entries
// form the low-rank part A_L, stored both by column (CSC) and by row (CSR).
#pragma once
#include <cstdint>

namespace sos {

constexpr double kSqrt2 = 1.4142135623730950488;
constexpr uint32_t kOffDiagBit = 0x80000000u;  // in row_ent: entry is off-diagonal
constexpr int32_t kEntOffBit = 0x40000000;     // in ent_row: plain entry is off-diagonal

struct InstInfo {
  int64_t x_off;      // first x entry
  int64_t y_off;      // first row
  int32_t nx, m;
  int32_t t, t_eff;
  int32_t lr_off;     // first low-rank column
  int32_t extra_form; // 1: weighted blocks rewritten with extra polynomials
  int64_t linv_off;   // dense t_eff x t_eff lower-triangular L^{-1}, row-major
  double zeta_h;      // zeta^T h with h = M^{-1} zeta (eq. (25))
  double norm_b, norm_c;
};

// Mutable per-instance scalars (device).
struct InstState {
  double omega3;      // u_tau + v_kappa at the start of the current iteration
  double s;           // Sherman-Morrison coefficient (zeta^T sigma)/(1 + zeta^T h)
  double cs1;         // c^T sigma_1
};

// Residual accumulators written every check (device -> host).
struct InstResid {
  double tau, kappa;
  double pr2;         // |A u_xi - b tau|^2
  double dr2;         // |A^T u_y + v_z - c tau|^2
  double ax2;         // |A u_xi|^2
  double aty2;        // |A^T u_y + v_z|^2
  double cx, by;      // c^T u_xi, b^T u_y
  double nonfinite;   // > 0 if a non-finite value was seen
};

// kRaw: the projection input is the stored vector itself (standalone projection).
enum BlockKind : int32_t { kPlain = 0, kWeighted = 1, kRaw = 2 };

struct BlockDesc {
  int64_t x_off;      // first packed entry of the block in x
  int64_t v_off;      // eigenvector storage (large blocks) or -1
  int32_t N;
  int32_t inst;
  int32_t kind;
  int32_t lr_first;   // weighted: low-rank column of the block's first entry
};

}  // namespace sos
