// Host-side setup of libsos: coefficient matching, index map, column classes,
// Woodbury core factorisation and Sherman-Morrison data.
//
// Paper references: coefficient matching eq. (11)-(12); indicator matrices
// B_alpha eq. (8) (a Gram entry (i, j) belongs to row beta_i + beta_j);
// weighted blocks eq. (38)-(40) (row beta_i + beta_j + delta for every term of
// the weight); Prop. 1 / Prop. 3 (plain Gram columns are orthogonal, so
// P = I + A_D A_D^T is diagonal); eq. (28) and the Appendix (Woodbury with a
// cached Cholesky factor of I + A_L^T P^{-1} A_L); eq. (25) (h = M^{-1} zeta).
#include "setup.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <thread>

namespace sos {
namespace {

// ---------------------------------------------------------------------------
// exponent-vector hash table (open addressing, FNV-1a over the int32 digits)
// ---------------------------------------------------------------------------
class ExpTable {
 public:
  ExpTable(int n_vars, const int32_t* exps, int32_t count) : n_(n_vars), exps_(exps), count_(count) {
    size_t cap = 16;
    while (cap < 2 * static_cast<size_t>(count) + 1) cap <<= 1;
    slots_.assign(cap, -1);
    mask_ = cap - 1;
  }
  // Inserts all rows; returns false on a duplicate.
  bool build() {
    for (int32_t r = 0; r < count_; ++r) {
      const int32_t* e = exps_ + static_cast<int64_t>(r) * n_;
      size_t s = hash(e) & mask_;
      while (slots_[s] >= 0) {
        if (equal(e, exps_ + static_cast<int64_t>(slots_[s]) * n_)) return false;
        s = (s + 1) & mask_;
      }
      slots_[s] = r;
    }
    return true;
  }
  int32_t find(const int32_t* e) const {
    size_t s = hash(e) & mask_;
    while (slots_[s] >= 0) {
      if (equal(e, exps_ + static_cast<int64_t>(slots_[s]) * n_)) return slots_[s];
      s = (s + 1) & mask_;
    }
    return -1;
  }

 private:
  size_t hash(const int32_t* e) const {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < n_; ++i) {
      uint32_t v = static_cast<uint32_t>(e[i]);
      for (int k = 0; k < 4; ++k) {
        h ^= (v >> (8 * k)) & 0xffu;
        h *= 1099511628211ull;
      }
    }
    return static_cast<size_t>(h ^ (h >> 29));
  }
  bool equal(const int32_t* a, const int32_t* b) const { return std::memcmp(a, b, sizeof(int32_t) * n_) == 0; }
  int n_;
  const int32_t* exps_;
  int32_t count_;
  std::vector<int32_t> slots_;
  size_t mask_;
};

struct LocalBlock {
  int64_t x_off;
  int32_t N, kind, lr_first;
};

// One instance, all indices local to it.
struct Local {
  int32_t nx = 0, m = 0, t = 0, t_eff = 0;
  std::vector<double> b, P, h2, g, linv, lr_c;
  std::vector<int32_t> ent_row;                 // nx
  std::vector<std::vector<std::pair<int32_t, double>>> cols;  // low-rank columns (row, value)
  std::vector<int32_t> lr_ent;
  std::vector<std::vector<uint32_t>> row_plain; // per row: entries | offdiag bit
  std::vector<LocalBlock> blocks;
  double zeta_h = 0, norm_b = 0, norm_c = 0;
  int extra_form = 0;  // 1: weighted blocks rewritten with extra polynomials
  int code = SOS_OK;
  std::string err;
};

int fail(Local& L, int code, const std::string& msg) {
  L.code = code;
  L.err = msg;
  return code;
}

// Barrier for the threads of one dense factorisation (spins, then yields).
class SpinBarrier {
 public:
  explicit SpinBarrier(int n) : n_(n) {}
  void wait() {
    const int g = gen_.load(std::memory_order_acquire);
    if (count_.fetch_add(1, std::memory_order_acq_rel) == n_ - 1) {
      count_.store(0, std::memory_order_relaxed);
      gen_.fetch_add(1, std::memory_order_release);
      return;
    }
    for (int spin = 0; gen_.load(std::memory_order_acquire) == g; ++spin)
      if (spin > 256) std::this_thread::yield();
  }

 private:
  const int n_;
  std::atomic<int> count_{0}, gen_{0};
};

// Dense FP64 Cholesky C = L L^T (row-major, lower), in place.  false if not
// SPD.  Column j: L_jj = sqrt(C_jj - sum_k<j L_jk^2), then every row below it
// L_ij = (C_ij - sum_k<j L_ik L_jk) / L_jj, the sums in ascending k.  With
// nth > 1 the rows of a column are shared cyclically among threads (one
// barrier per column; the owner of row j + 1 also forms L_{j+1,j+1}); every
// entry is computed by the same operations in the same order as with one
// thread.
bool cholesky(std::vector<double>& C, int n, int nth) {
  double* A = C.data();
  auto row_entry = [&](int i, int j, double d) {
    double s = A[static_cast<size_t>(i) * n + j];
    for (int k = 0; k < j; ++k) s -= A[static_cast<size_t>(i) * n + k] * A[static_cast<size_t>(j) * n + k];
    A[static_cast<size_t>(i) * n + j] = s / d;
  };
  auto diag = [&](int j) {  // false if not positive
    double d = A[static_cast<size_t>(j) * n + j];
    for (int k = 0; k < j; ++k) d -= A[static_cast<size_t>(j) * n + k] * A[static_cast<size_t>(j) * n + k];
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    A[static_cast<size_t>(j) * n + j] = std::sqrt(d);
    return true;
  };
  nth = std::max(1, std::min(nth, n / 64));
  bool ok = true;
  if (nth == 1) {
    for (int j = 0; j < n && ok; ++j) {
      ok = diag(j);
      if (!ok) break;
      const double d = A[static_cast<size_t>(j) * n + j];
      for (int i = j + 1; i < n; ++i) row_entry(i, j, d);
    }
  } else {
    ok = n < 1 || diag(0);
    std::atomic<bool> bad{!ok};
    SpinBarrier bar(nth);
    auto work = [&](int t) {
      for (int j = 0; j < n - 1; ++j) {
        const double d = A[static_cast<size_t>(j) * n + j];
        if ((j + 1) % nth == t) {  // row j + 1 first, then the next diagonal
          row_entry(j + 1, j, d);
          if (!diag(j + 1)) bad.store(true, std::memory_order_relaxed);
        }
        for (int i = j + 2 + ((t - (j + 2)) % nth + nth) % nth; i < n; i += nth) row_entry(i, j, d);
        bar.wait();
        if (bad.load(std::memory_order_relaxed)) return;
      }
    };
    if (ok) {
      std::vector<std::thread> pool;
      for (int t = 1; t < nth; ++t) pool.emplace_back(work, t);
      work(0);
      for (auto& th : pool) th.join();
    }
    ok = !bad.load();
  }
  if (!ok) return false;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) A[static_cast<size_t>(i) * n + j] = 0.0;
  return true;
}

// Inverse of a lower-triangular matrix (row-major), FP64.  Column c of L^{-1}
// solves L x = e_c and depends on no other column, so threads take chunks of
// columns; inside a chunk row i is formed from the rows k < i by contiguous
// multiply-adds: X_ic = -(sum_{k=c}^{i-1} L_ik X_kc) / L_ii (ascending k),
// X_ii = 1 / L_ii.
std::vector<double> tri_inverse(const std::vector<double>& Lm, int n, int nth) {
  std::vector<double> X(static_cast<size_t>(n) * n, 0.0);
  constexpr int kChunk = 32;
  const int nchunk = (n + kChunk - 1) / kChunk;
  auto chunk = [&](int q) {
    const int c0 = q * kChunk, c1 = std::min(n, c0 + kChunk);
    for (int i = c0; i < n; ++i) {
      double* xi = &X[static_cast<size_t>(i) * n];
      const double* li = &Lm[static_cast<size_t>(i) * n];
      for (int k = c0; k < i; ++k) {
        const double a = li[k];
        const double* xk = &X[static_cast<size_t>(k) * n];
        const int ce = std::min(k + 1, c1);
        for (int c = c0; c < ce; ++c) xi[c] += a * xk[c];
      }
      const double lii = li[i];
      const int ce = std::min(i, c1);
      for (int c = c0; c < ce; ++c) xi[c] = -xi[c] / lii;
      if (i < c1) xi[i] = 1.0 / lii;
    }
  };
  nth = std::max(1, std::min(nth, nchunk));
  std::vector<std::thread> pool;
  for (int t = 1; t < nth; ++t)
    pool.emplace_back([&, t]() {
      for (int q = t; q < nchunk; q += nth) chunk(q);
    });
  for (int q = 0; q < nchunk; q += nth) chunk(q);
  for (auto& th : pool) th.join();
  return X;
}

// ---------------------------------------------------------------------------
// Extra-polynomial form of weighted SOS constraints (end of Section II): a
// weighted term p(x) s(x), s = v^T X v, becomes p(x) r(x) with r a free
// polynomial r = sum_beta r_beta x^beta over the monomials beta of v v^T,
// plus a new identity r(x) = v^T X v in which X is a plain Gram block.  The
// coefficients r_beta follow the original t variables (weighted blocks in
// program order, beta in the order of eq. (4)); each new identity follows the
// original constraints (same order) and owns its block, which leaves the
// weighted term's constraint.  Every Gram block of the result is plain, and
// the low-rank part holds only free variables.
// ---------------------------------------------------------------------------
struct ExtraForm {
  std::vector<double> w;
  std::vector<sos_constraint> cons;
  std::deque<std::vector<sos_block>> blocks;
  std::deque<std::vector<int32_t>> i32;
  std::deque<std::vector<double>> f64;
  sos_program prog{};
};

// Structural checks of one program (sizes and pointers), before anything
// reads its arrays; the coefficient matching reports the rest.
const char* program_error(const sos_program& pg) {
  if (pg.n_vars < 1) return "n_vars must be >= 1";
  if (pg.t < 0 || (pg.t > 0 && !pg.w)) return "t < 0 or w missing";
  if (pg.n_constraints < 1 || !pg.constraints) return "no constraints";
  for (int j = 0; j < pg.n_constraints; ++j) {
    const sos_constraint& c = pg.constraints[j];
    if (c.n_rows < 1 || !c.row_exps) return "constraint without rows";
    if (c.n_terms < 0 || (c.n_terms > 0 && (!c.term_poly || !c.term_exps || !c.term_coef)))
      return "term arrays missing";
    if (c.n_blocks < 0 || (c.n_blocks > 0 && !c.blocks)) return "block array missing";
    for (int k = 0; k < c.n_blocks; ++k) {
      const sos_block& bk = c.blocks[k];
      if (bk.N < 1 || !bk.basis_exps) return "block with N < 1";
      if (bk.n_weight_terms < 0 || (bk.n_weight_terms > 0 && (!bk.weight_exps || !bk.weight_coef)))
        return "weight arrays missing";
    }
    if (c.matrix_r < 0) return "matrix_r < 0";
    if (c.matrix_r > 0) {
      if (c.n_blocks != 1 || c.blocks[0].n_weight_terms != 0)
        return "a matrix-valued constraint takes exactly one unweighted block";
      if (c.n_terms > 0 && !c.term_pair) return "term_pair missing";
      for (int64_t k = 0; k < c.n_terms; ++k) {
        const int32_t a = c.term_pair[2 * k], b = c.term_pair[2 * k + 1];
        if (a < 0 || a > b || b >= c.matrix_r) return "term_pair outside 0 <= i <= j < matrix_r";
      }
    }
  }
  return nullptr;
}

bool has_matrix(const sos_program& pg) {
  for (int j = 0; j < pg.n_constraints; ++j)
    if (pg.constraints[j].matrix_r > 0) return true;
  return false;
}

// A program with matrix-valued constraints (Section V) as one with scalar
// constraints only, in the variables (x, y_1..y_R), R the largest size:
// the basis entry (i, a) of I_r (x) v becomes y_i x^a, the row triple
// (alpha, i, j), i <= j, becomes y_i y_j x^alpha, and a term c x^e of entry
// (i, j) of P_h becomes c' x^e y_i y_j with c' = c on the diagonal and 2 c
// off it -- the coefficient of y_i y_j x^e in y^T P_h(x) y.  An entry (p, q)
// of Y then meets row (alpha_p + alpha_q, i_p, i_q) through the same
// exponent lookup as a scalar Gram entry (Prop. 2).  Scalar constraints get
// zero exponents in y.
struct MatrixForm {
  std::vector<sos_constraint> cons;
  std::deque<std::vector<sos_block>> blocks;
  std::deque<std::vector<int32_t>> i32;
  std::deque<std::vector<double>> f64;
  sos_program prog{};
};

void to_scalar_form(const sos_program& pg, MatrixForm& F) {
  const int n = pg.n_vars;
  int R = 0;
  for (int j = 0; j < pg.n_constraints; ++j) R = std::max(R, pg.constraints[j].matrix_r);
  const int nv = n + R;
  auto pad = [&](const int32_t* e, int64_t count) -> const int32_t* {
    std::vector<int32_t> out(static_cast<size_t>(count) * nv, 0);
    for (int64_t q = 0; q < count; ++q)
      for (int a = 0; a < n; ++a) out[q * nv + a] = e[q * n + a];
    F.i32.push_back(std::move(out));
    return F.i32.back().data();
  };
  F.cons.assign(pg.constraints, pg.constraints + pg.n_constraints);
  for (int j = 0; j < pg.n_constraints; ++j) {
    const sos_constraint& c = pg.constraints[j];
    sos_constraint& o = F.cons[j];
    o.matrix_r = 0;
    o.term_pair = nullptr;
    if (c.matrix_r == 0) {
      o.row_exps = pad(c.row_exps, c.n_rows);
      o.term_exps = pad(c.term_exps, c.n_terms);
      F.blocks.emplace_back(c.blocks, c.blocks + c.n_blocks);
      for (auto& bk : F.blocks.back()) {
        bk.basis_exps = pad(bk.basis_exps, bk.N);
        if (bk.n_weight_terms > 0) bk.weight_exps = pad(bk.weight_exps, bk.n_weight_terms);
      }
      o.blocks = F.blocks.back().data();
      continue;
    }
    const int r = c.matrix_r;
    // rows: pairs i <= j row-major, then alpha
    std::vector<int32_t> rows;
    for (int i = 0; i < r; ++i)
      for (int jj = i; jj < r; ++jj)
        for (int32_t q = 0; q < c.n_rows; ++q) {
          std::vector<int32_t> e(nv, 0);
          for (int a = 0; a < n; ++a) e[a] = c.row_exps[static_cast<int64_t>(q) * n + a];
          e[n + i] += 1;
          e[n + jj] += 1;
          rows.insert(rows.end(), e.begin(), e.end());
        }
    F.i32.push_back(std::move(rows));
    o.row_exps = F.i32.back().data();
    o.n_rows = c.n_rows * r * (r + 1) / 2;
    // terms
    std::vector<int32_t> tp(c.n_terms), te(static_cast<size_t>(c.n_terms) * nv, 0);
    std::vector<double> tc(c.n_terms);
    for (int64_t k = 0; k < c.n_terms; ++k) {
      const int32_t i = c.term_pair[2 * k], jj = c.term_pair[2 * k + 1];
      tp[k] = c.term_poly[k];
      for (int a = 0; a < n; ++a) te[k * nv + a] = c.term_exps[k * n + a];
      te[k * nv + n + i] += 1;
      te[k * nv + n + jj] += 1;
      tc[k] = (i == jj ? 1.0 : 2.0) * c.term_coef[k];
    }
    F.i32.push_back(std::move(tp));
    o.term_poly = F.i32.back().data();
    F.i32.push_back(std::move(te));
    o.term_exps = F.i32.back().data();
    F.f64.push_back(std::move(tc));
    o.term_coef = F.f64.back().data();
    // one block: y_i x^a, block-major
    const sos_block& b0 = c.blocks[0];
    std::vector<int32_t> bas(static_cast<size_t>(r) * b0.N * nv, 0);
    for (int i = 0; i < r; ++i)
      for (int a = 0; a < b0.N; ++a) {
        int32_t* e = bas.data() + (static_cast<size_t>(i) * b0.N + a) * nv;
        for (int v = 0; v < n; ++v) e[v] = b0.basis_exps[static_cast<int64_t>(a) * n + v];
        e[n + i] = 1;
      }
    F.i32.push_back(std::move(bas));
    sos_block nb{};
    nb.N = r * b0.N;
    nb.basis_exps = F.i32.back().data();
    nb.n_weight_terms = 0;
    F.blocks.emplace_back(1, nb);
    o.blocks = F.blocks.back().data();
    o.n_blocks = 1;
  }
  F.prog = pg;
  F.prog.n_vars = nv;
  F.prog.constraints = F.cons.data();
}

bool has_weighted(const sos_program& pg) {
  for (int j = 0; j < pg.n_constraints; ++j)
    for (int k = 0; k < pg.constraints[j].n_blocks; ++k)
      if (pg.constraints[j].blocks[k].n_weight_terms > 0) return true;
  return false;
}

// eq. (42) with packed Gram blocks: the direct form pays off while the
// Woodbury core, t + sum N_i (N_i + 1) / 2 for the weighted blocks, stays
// smaller than m.
bool choose_extra_form(const sos_program& pg, int form) {
  if (form == 1 || !has_weighted(pg)) return false;
  if (form == 2) return true;
  int64_t width = pg.t, m = 0;
  for (int j = 0; j < pg.n_constraints; ++j) {
    const sos_constraint& c = pg.constraints[j];
    m += c.n_rows;
    for (int k = 0; k < c.n_blocks; ++k)
      if (c.blocks[k].n_weight_terms > 0) width += static_cast<int64_t>(c.blocks[k].N) * (c.blocks[k].N + 1) / 2;
  }
  return width >= m;
}

void to_extra_form(const sos_program& pg, ExtraForm& F) {
  const int nv = pg.n_vars;
  struct Weighted {
    int j, k;
    int32_t first;                          // index of r_beta for the first beta
    std::vector<std::vector<int32_t>> beta;  // monomials of v v^T, eq. (4) order
  };
  std::vector<Weighted> ws;
  int32_t t2 = pg.t;
  for (int j = 0; j < pg.n_constraints; ++j)
    for (int k = 0; k < pg.constraints[j].n_blocks; ++k) {
      const sos_block& bk = pg.constraints[j].blocks[k];
      if (bk.n_weight_terms <= 0) continue;
      std::vector<std::vector<int32_t>> bs;
      for (int jj = 0; jj < bk.N; ++jj)
        for (int ii = jj; ii < bk.N; ++ii) {
          std::vector<int32_t> e(nv);
          for (int q = 0; q < nv; ++q)
            e[q] = bk.basis_exps[static_cast<int64_t>(ii) * nv + q] + bk.basis_exps[static_cast<int64_t>(jj) * nv + q];
          bs.push_back(std::move(e));
        }
      auto degree = [](const std::vector<int32_t>& e) {
        int64_t d = 0;
        for (int32_t v : e) d += v;
        return d;
      };
      std::sort(bs.begin(), bs.end(), [&](const std::vector<int32_t>& a, const std::vector<int32_t>& b) {
        const int64_t da = degree(a), db = degree(b);
        return da != db ? da < db : a > b;  // graded, then x1-major descending
      });
      bs.erase(std::unique(bs.begin(), bs.end()), bs.end());
      ws.push_back({j, k, t2, std::move(bs)});
      t2 += static_cast<int32_t>(ws.back().beta.size());
    }
  F.w.assign(pg.w, pg.w + pg.t);
  F.w.resize(t2, 0.0);
  size_t wi = 0;
  for (int j = 0; j < pg.n_constraints; ++j) {
    const sos_constraint& c = pg.constraints[j];
    auto& tp = F.i32.emplace_back(c.term_poly, c.term_poly + c.n_terms);
    auto& te = F.i32.emplace_back(c.term_exps, c.term_exps + c.n_terms * nv);
    auto& tc = F.f64.emplace_back(c.term_coef, c.term_coef + c.n_terms);
    auto& bl = F.blocks.emplace_back();
    for (int k = 0; k < c.n_blocks; ++k) {
      const sos_block& bk = c.blocks[k];
      if (bk.n_weight_terms <= 0) {
        bl.push_back(bk);
        continue;
      }
      const Weighted& W = ws[wi++];
      // g_beta = p(x) x^beta on the identity's left side
      for (size_t q = 0; q < W.beta.size(); ++q)
        for (int d = 0; d < bk.n_weight_terms; ++d) {
          tp.push_back(W.first + static_cast<int32_t>(q) + 1);
          for (int v = 0; v < nv; ++v) te.push_back(W.beta[q][v] + bk.weight_exps[static_cast<int64_t>(d) * nv + v]);
          tc.push_back(bk.weight_coef[d]);
        }
    }
    sos_constraint nc = c;
    nc.n_terms = static_cast<int64_t>(tp.size());
    nc.term_poly = tp.data();
    nc.term_exps = te.data();
    nc.term_coef = tc.data();
    nc.n_blocks = static_cast<int32_t>(bl.size());
    nc.blocks = bl.data();
    F.cons.push_back(nc);
  }
  for (const Weighted& W : ws) {
    const sos_block& bk = pg.constraints[W.j].blocks[W.k];
    auto& rows = F.i32.emplace_back();
    auto& tp = F.i32.emplace_back();
    auto& tc = F.f64.emplace_back();
    for (size_t q = 0; q < W.beta.size(); ++q) {
      rows.insert(rows.end(), W.beta[q].begin(), W.beta[q].end());
      tp.push_back(W.first + static_cast<int32_t>(q) + 1);
      tc.push_back(-1.0);  // 0 - sum_beta r_beta (-x^beta) = v^T X v
    }
    auto& bl = F.blocks.emplace_back();
    sos_block plain = bk;
    plain.n_weight_terms = 0;
    plain.weight_exps = nullptr;
    plain.weight_coef = nullptr;
    bl.push_back(plain);
    sos_constraint nc{};
    nc.n_rows = static_cast<int32_t>(W.beta.size());
    nc.row_exps = rows.data();
    nc.n_terms = static_cast<int64_t>(tp.size());
    nc.term_poly = tp.data();
    nc.term_exps = rows.data();  // term q is x^beta_q, the q-th row
    nc.term_coef = tc.data();
    nc.n_blocks = 1;
    nc.blocks = bl.data();
    F.cons.push_back(nc);
  }
  F.prog = pg;
  F.prog.t = t2;
  F.prog.w = F.w.data();
  F.prog.n_constraints = static_cast<int32_t>(F.cons.size());
  F.prog.constraints = F.cons.data();
}

// inner_threads: threads the dense factorisation of this instance may use
// (1 while the instances of a plan are built in parallel)
int build_instance(const sos_program& pg, Local& L, int inner_threads) {
  const int nv = pg.n_vars;
  if (nv < 1) return fail(L, SOS_ERR_INVALID_ARG, "n_vars must be >= 1");
  if (pg.t < 0 || (pg.t > 0 && !pg.w)) return fail(L, SOS_ERR_INVALID_ARG, "t < 0 or w missing");
  if (pg.n_constraints < 1 || !pg.constraints) return fail(L, SOS_ERR_INVALID_ARG, "no constraints");
  L.t = pg.t;

  // rows of every constraint, concatenated
  std::vector<int32_t> row_base(pg.n_constraints);
  std::vector<ExpTable> tables;
  tables.reserve(pg.n_constraints);
  int32_t m = 0;
  for (int j = 0; j < pg.n_constraints; ++j) {
    const sos_constraint& c = pg.constraints[j];
    if (c.n_rows < 1 || !c.row_exps) return fail(L, SOS_ERR_INVALID_ARG, "constraint without rows");
    row_base[j] = m;
    m += c.n_rows;
    tables.emplace_back(nv, c.row_exps, c.n_rows);
    if (!tables.back().build()) return fail(L, SOS_ERR_INVALID_ARG, "duplicate row monomial");
  }
  L.m = m;
  L.b.assign(m, 0.0);
  L.row_plain.assign(m, {});

  // packed x layout: free u, then every block of every constraint
  int64_t nx = pg.t;
  for (int j = 0; j < pg.n_constraints; ++j)
    for (int k = 0; k < pg.constraints[j].n_blocks; ++k) {
      const sos_block& bk = pg.constraints[j].blocks[k];
      if (bk.N < 1 || !bk.basis_exps) return fail(L, SOS_ERR_INVALID_ARG, "block with N < 1");
      nx += static_cast<int64_t>(bk.N) * (bk.N + 1) / 2;
    }
  if (nx > (1ll << 30)) return fail(L, SOS_ERR_UNSUPPORTED, "instance too large");
  L.nx = static_cast<int32_t>(nx);
  L.ent_row.assign(L.nx, -1);

  // free columns (A_1) and b, coefficient matching eq. (11)
  std::vector<std::map<int32_t, double>> freecols(pg.t);
  for (int j = 0; j < pg.n_constraints; ++j) {
    const sos_constraint& c = pg.constraints[j];
    for (int64_t k = 0; k < c.n_terms; ++k) {
      int32_t p = c.term_poly[k];
      if (p < 0 || p > pg.t) return fail(L, SOS_ERR_INVALID_ARG, "term_poly out of range");
      int32_t r = tables[j].find(c.term_exps + k * nv);
      if (r < 0) return fail(L, SOS_ERR_INVALID_ARG, "a term of g_i is not among the constraint's rows");
      r += row_base[j];
      if (p == 0)
        L.b[r] += c.term_coef[k];
      else
        freecols[p - 1][r] += c.term_coef[k];
    }
  }
  for (int i = 0; i < pg.t; ++i) {
    std::vector<std::pair<int32_t, double>> col;
    for (auto& kv : freecols[i])
      if (kv.second != 0.0) col.push_back(kv);
    L.cols.push_back(std::move(col));
    L.lr_ent.push_back(i);
    L.lr_c.push_back(pg.w[i]);
  }

  // Gram blocks: index map of eq. (8) / eq. (38)
  std::vector<int32_t> sum(nv);
  int64_t xo = pg.t;
  for (int j = 0; j < pg.n_constraints; ++j) {
    const sos_constraint& c = pg.constraints[j];
    for (int k = 0; k < c.n_blocks; ++k) {
      const sos_block& bk = c.blocks[k];
      const int N = bk.N;
      const bool weighted = bk.n_weight_terms > 0;
      LocalBlock lb{xo, N, weighted ? kWeighted : kPlain, weighted ? static_cast<int32_t>(L.cols.size()) : -1};
      L.blocks.push_back(lb);
      int64_t e = xo;
      for (int jj = 0; jj < N; ++jj) {
        const int32_t* bj = bk.basis_exps + static_cast<int64_t>(jj) * nv;
        for (int ii = jj; ii < N; ++ii, ++e) {
          const int32_t* bi = bk.basis_exps + static_cast<int64_t>(ii) * nv;
          for (int q = 0; q < nv; ++q) sum[q] = bi[q] + bj[q];
          const bool off = ii != jj;
          if (!weighted) {
            int32_t r = tables[j].find(sum.data());
            if (r < 0) return fail(L, SOS_ERR_INVALID_ARG, "a Gram product monomial is not among the rows");
            r += row_base[j];
            L.ent_row[e] = r | (off ? kEntOffBit : 0);
            L.row_plain[r].push_back(static_cast<uint32_t>(e) | (off ? kOffDiagBit : 0u));
          } else {
            std::vector<std::pair<int32_t, double>> col;
            std::vector<int32_t> s2(nv);
            for (int w = 0; w < bk.n_weight_terms; ++w) {
              const int32_t* d = bk.weight_exps + static_cast<int64_t>(w) * nv;
              for (int q = 0; q < nv; ++q) s2[q] = sum[q] + d[q];
              int32_t r = tables[j].find(s2.data());
              if (r < 0) return fail(L, SOS_ERR_INVALID_ARG, "a weighted Gram product monomial is not among the rows");
              col.emplace_back(r + row_base[j], bk.weight_coef[w] * (off ? kSqrt2 : 1.0));
            }
            std::sort(col.begin(), col.end());
            std::vector<std::pair<int32_t, double>> merged;
            for (auto& p : col) {
              if (!merged.empty() && merged.back().first == p.first)
                merged.back().second += p.second;
              else
                merged.push_back(p);
            }
            L.cols.push_back(std::move(merged));
            L.lr_ent.push_back(static_cast<int32_t>(e));
            L.lr_c.push_back(0.0);
          }
        }
      }
      xo = e;
    }
  }
  const int te = static_cast<int>(L.cols.size());
  L.t_eff = te;

  // P = I + A_D A_D^T, diagonal by Prop. 1 (svec: 1 per diagonal, 2 per off-diagonal entry)
  L.P.assign(m, 1.0);
  for (int32_t r = 0; r < m; ++r)
    for (uint32_t v : L.row_plain[r]) L.P[r] += (v & kOffDiagBit) ? 2.0 : 1.0;

  // low-rank rows
  std::vector<std::vector<std::pair<int32_t, double>>> lrrows(m);
  for (int jc = 0; jc < te; ++jc)
    for (auto& p : L.cols[jc]) lrrows[p.first].emplace_back(jc, p.second);

  // Woodbury core I + A_L^T P^{-1} A_L (eq. (28)) and its FP64 Cholesky factor
  std::vector<double> C(static_cast<size_t>(te) * te, 0.0);
  for (int i = 0; i < te; ++i) C[static_cast<size_t>(i) * te + i] = 1.0;
  for (int32_t r = 0; r < m; ++r) {
    const double pi = 1.0 / L.P[r];
    const auto& row = lrrows[r];
    for (size_t a = 0; a < row.size(); ++a) {
      const double va = row[a].second * pi;
      double* Ci = &C[static_cast<size_t>(row[a].first) * te];
      for (size_t c2 = 0; c2 < row.size(); ++c2) Ci[row[c2].first] += va * row[c2].second;
    }
  }
  std::vector<double> Lf = C;
  if (!cholesky(Lf, te, inner_threads)) return fail(L, SOS_ERR_FACTOR, "Woodbury core is not positive definite");
  L.linv = tri_inverse(Lf, te, inner_threads);

  // h = M^{-1} zeta, zeta = [c; -b] (eq. (25)), via eq. (27) with the Cholesky factor
  //   r = -b - A c ; sigma2 = (P + A_L A_L^T)^{-1} r ; sigma1 = c + A^T sigma2
  std::vector<double> r(m);
  for (int32_t i = 0; i < m; ++i) r[i] = -L.b[i];
  for (int i = 0; i < pg.t; ++i)
    for (auto& p : L.cols[i]) r[p.first] -= p.second * pg.w[i];
  std::vector<double> xw(m), y(te, 0.0), z(te, 0.0);
  for (int32_t i = 0; i < m; ++i) xw[i] = r[i] / L.P[i];
  for (int jc = 0; jc < te; ++jc)
    for (auto& p : L.cols[jc]) y[jc] += p.second * xw[p.first];
  for (int i = 0; i < te; ++i) {  // forward substitution L q = y
    double s = y[i];
    for (int k = 0; k < i; ++k) s -= Lf[static_cast<size_t>(i) * te + k] * z[k];
    z[i] = s / Lf[static_cast<size_t>(i) * te + i];
  }
  for (int i = te - 1; i >= 0; --i) {  // back substitution L^T z = q
    double s = z[i];
    for (int k = i + 1; k < te; ++k) s -= Lf[static_cast<size_t>(k) * te + i] * z[k];
    z[i] = s / Lf[static_cast<size_t>(i) * te + i];
  }
  L.h2.assign(m, 0.0);
  for (int32_t i = 0; i < m; ++i) {
    double acc = 0.0;
    for (auto& p : lrrows[i]) acc += p.second * z[p.first];
    L.h2[i] = xw[i] - acc / L.P[i];
  }
  // g = A_L^T h_2 (equals z up to rounding; recomputed from h_2 directly)
  L.g.assign(te, 0.0);
  for (int jc = 0; jc < te; ++jc)
    for (auto& p : L.cols[jc]) L.g[jc] += p.second * L.h2[p.first];
  double ch1 = 0.0, bh2 = 0.0, nb = 0.0, nc = 0.0;
  for (int i = 0; i < pg.t; ++i) {
    ch1 += pg.w[i] * (pg.w[i] + L.g[i]);  // h_1 = c + A^T h_2 on the free columns
    nc += pg.w[i] * pg.w[i];
  }
  for (int32_t i = 0; i < m; ++i) {
    bh2 += L.b[i] * L.h2[i];
    nb += L.b[i] * L.b[i];
  }
  L.zeta_h = ch1 - bh2;
  L.norm_b = std::sqrt(nb);
  L.norm_c = std::sqrt(nc);
  if (!(1.0 + L.zeta_h > 0.0)) return fail(L, SOS_ERR_FACTOR, "1 + zeta^T h is not positive");
  return SOS_OK;
}

}  // namespace

int64_t enumerate_monomials(int32_t n_vars, int32_t degree, int32_t* out, int64_t capacity) {
  // graded; inside a degree, x1-major descending (eq. (4))
  int64_t count = 0;
  std::vector<int32_t> e(n_vars);
  for (int32_t deg = 0; deg <= degree; ++deg) {
    // first exponent of the level: (deg, 0, ..., 0)
    std::fill(e.begin(), e.end(), 0);
    e[0] = deg;
    while (true) {
      if (out && count < capacity) std::memcpy(out + count * n_vars, e.data(), sizeof(int32_t) * n_vars);
      ++count;
      // next in descending lex order among compositions of deg
      int k = n_vars - 2;
      while (k >= 0 && e[k] == 0) --k;
      if (k < 0) break;
      e[k] -= 1;
      int32_t rest = 0;
      for (int q = k + 1; q < n_vars; ++q) rest += e[q];
      for (int q = k + 1; q < n_vars; ++q) e[q] = 0;
      e[k + 1] = rest + 1;
    }
  }
  return count;
}

int build_plan(const sos_program* progs, int32_t n_progs, HostPlan& P, std::string& err, int weighted_form) {
  if (!progs || n_progs < 1) {
    err = "need at least one program";
    return SOS_ERR_INVALID_ARG;
  }
  std::vector<Local> loc(n_progs);
  unsigned nth = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  // few programs: one builder thread, and the dense factorisations of the
  // Woodbury cores use the cores instead
  const int inner = n_progs < 4 ? static_cast<int>(nth) : 1;
  if (n_progs < 4) nth = 1;
  std::vector<std::thread> pool;
  for (unsigned w = 0; w < nth; ++w)
    pool.emplace_back([&, w]() {
      for (int32_t i = static_cast<int32_t>(w); i < n_progs; i += static_cast<int32_t>(nth)) {
        if (const char* msg = program_error(progs[i])) {
          fail(loc[i], SOS_ERR_INVALID_ARG, msg);
          continue;
        }
        MatrixForm MF;
        const sos_program* pg = &progs[i];
        if (has_matrix(*pg)) {
          to_scalar_form(*pg, MF);
          pg = &MF.prog;
        }
        if (choose_extra_form(*pg, weighted_form)) {
          ExtraForm F;
          to_extra_form(*pg, F);
          build_instance(F.prog, loc[i], inner);
          loc[i].extra_form = 1;
        } else {
          build_instance(*pg, loc[i], inner);
        }
      }
    });
  for (auto& th : pool) th.join();
  for (int32_t i = 0; i < n_progs; ++i)
    if (loc[i].code != SOS_OK) {
      err = "instance " + std::to_string(i) + ": " + loc[i].err;
      return loc[i].code;
    }

  // merge with global offsets
  P.n_inst = n_progs;
  int64_t NX = 0, M = 0, nnzD = 0, nnzL = 0, nlinv = 0;
  int64_t TL = 0;
  for (auto& L : loc) {
    NX += L.nx;
    M += L.m;
    TL += L.t_eff;
    nlinv += static_cast<int64_t>(L.t_eff) * L.t_eff;
    for (auto& r : L.row_plain) nnzD += static_cast<int64_t>(r.size());
    for (auto& c : L.cols) nnzL += static_cast<int64_t>(c.size());
  }
  if (NX >= (1ll << 31) || M >= (1ll << 30) || TL >= (1ll << 31) || nnzL >= (1ll << 31) || nnzD >= (1ll << 31)) {
    err = "problem set too large for 32-bit indices";
    return SOS_ERR_UNSUPPORTED;
  }
  P.NX = NX;
  P.M = M;
  P.TL = static_cast<int32_t>(TL);
  P.n_linv = nlinv;
  P.b.reserve(M);
  P.pinv.reserve(M);
  P.h2.reserve(M);
  P.row_inst.reserve(M);
  P.row_ptr.reserve(M + 1);
  P.row_ent.reserve(nnzD);
  P.ent_row.reserve(NX);
  P.lr_ptr.reserve(TL + 1);
  P.lr_row.reserve(nnzL);
  P.lr_val.reserve(nnzL);
  P.linv.reserve(nlinv);
  P.row_ptr.push_back(0);
  P.lr_ptr.push_back(0);
  int64_t xoff = 0, yoff = 0, loff = 0;
  int32_t lroff = 0;
  for (int32_t i = 0; i < n_progs; ++i) {
    Local& L = loc[i];
    InstInfo in{};
    in.x_off = xoff;
    in.y_off = yoff;
    in.nx = L.nx;
    in.m = L.m;
    in.t = L.t;
    in.t_eff = L.t_eff;
    in.lr_off = lroff;
    in.extra_form = L.extra_form;
    in.linv_off = loff;
    in.zeta_h = L.zeta_h;
    in.norm_b = L.norm_b;
    in.norm_c = L.norm_c;
    P.inst.push_back(in);
    P.x_inst_start.push_back(xoff);
    for (int32_t r = 0; r < L.m; ++r) {
      P.b.push_back(L.b[r]);
      P.pinv.push_back(1.0 / L.P[r]);
      P.h2.push_back(L.h2[r]);
      P.row_inst.push_back(i);
      for (uint32_t v : L.row_plain[r]) {
        uint32_t e = (v & ~kOffDiagBit) + static_cast<uint32_t>(xoff);
        P.row_ent.push_back(e | (v & kOffDiagBit));
      }
      P.row_ptr.push_back(static_cast<int32_t>(P.row_ent.size()));
    }
    for (int32_t e = 0; e < L.nx; ++e) {
      const int32_t er = L.ent_row[e];
      P.ent_row.push_back(er >= 0 ? static_cast<int32_t>(((er & ~kEntOffBit) + yoff) | (er & kEntOffBit)) : -1);
    }
    for (int jc = 0; jc < L.t_eff; ++jc) {
      P.ent_row[xoff + L.lr_ent[jc]] = -(lroff + jc + 1);
      for (auto& p : L.cols[jc]) {
        P.lr_row.push_back(static_cast<int32_t>(p.first + yoff));
        P.lr_val.push_back(p.second);
      }
      P.lr_ptr.push_back(static_cast<int32_t>(P.lr_row.size()));
      P.lr_ent.push_back(L.lr_ent[jc] + xoff);
      P.lr_inst.push_back(i);
      P.lr_c.push_back(L.lr_c[jc]);
      P.lr_g.push_back(L.g[jc]);
    }
    P.linv.insert(P.linv.end(), L.linv.begin(), L.linv.end());
    for (auto& lb : L.blocks) {
      BlockDesc bd{};
      bd.x_off = lb.x_off + xoff;
      bd.v_off = -1;
      bd.N = lb.N;
      bd.inst = i;
      bd.kind = lb.kind;
      bd.lr_first = lb.kind == kWeighted ? lb.lr_first + lroff : -1;
      P.blocks.push_back(bd);
    }
    xoff += L.nx;
    yoff += L.m;
    loff += static_cast<int64_t>(L.t_eff) * L.t_eff;
    lroff += L.t_eff;
    L = Local();  // release
  }
  P.x_inst_start.push_back(xoff);
  // CSR of A_L by rows (global)
  P.lrr_ptr.assign(M + 1, 0);
  for (int64_t k = 0; k < static_cast<int64_t>(P.lr_row.size()); ++k) P.lrr_ptr[P.lr_row[k] + 1]++;
  for (int64_t r = 0; r < M; ++r) P.lrr_ptr[r + 1] += P.lrr_ptr[r];
  P.lrr_col.assign(P.lr_row.size(), 0);
  P.lrr_val.assign(P.lr_row.size(), 0.0);
  std::vector<int32_t> fillp(P.lrr_ptr.begin(), P.lrr_ptr.end() - 1);
  for (int32_t jc = 0; jc < P.TL; ++jc)
    for (int32_t k = P.lr_ptr[jc]; k < P.lr_ptr[jc + 1]; ++k) {
      int32_t r = P.lr_row[k];
      P.lrr_col[fillp[r]] = jc;
      P.lrr_val[fillp[r]] = P.lr_val[k];
      fillp[r]++;
    }
  return SOS_OK;
}

}  // namespace sos
