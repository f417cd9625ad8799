// C-ABI of libsos: handle lifetime, device memory, the per-iteration CUDA
// graph, the solve loop with residual checks, iterate I/O.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <memory>
#include <string>
#include <vector>

#include "../../include/sos.h"
#include "kernels.h"
#include "setup.h"

using namespace sos;

namespace {
thread_local std::string g_setup_error;
}  // namespace

void sos::set_global_error(const std::string& msg) { g_setup_error = msg; }

namespace {

struct SmallClass {
  int maxN;
  int count;
  int32_t* ids;  // device
};

template <typename T>
struct LargeBlock {
  int bid, N, grid;
  LargeScratch<T> scratch;
};

struct NsBlock {
  int bid, N;
  NsScratch s;
};
}  // namespace

struct sos_handle {
  int32_t precision = SOS_PREC_FP64;
  int32_t k_check = 10;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int32_t n_inst = 0;
  int64_t NX = 0, M = 0;
  int32_t TL = 0;
  std::vector<InstInfo> inst;
  std::vector<BlockDesc> blocks;
  std::vector<void*> allocs;
  DevPlan<double> d64;
  DevPlan<float> d32;
  LaunchShape shape;
  std::vector<SmallClass> small;
  std::vector<LargeBlock<double>> large64;  // FP64 projections
  std::vector<LargeBlock<float>> large32;   // FP32 projections
  SmallWarm<double> warm64;
  SmallWarm<float> warm32;
  std::vector<NsBlock> ns_large;  // large blocks projected by Newton-Schulz on the tensor cores
  int32_t large_method = 0;
  double infeas_tol = 1e-7;   // tolerance of the infeasibility certificates
  int32_t wait_limit_us = 0;  // bound of the grid-wide waits (0: about 2 s)
  int32_t* active = nullptr;  // device
  std::vector<int32_t> active_h;
  std::vector<int32_t> iters_h, status_h;
  int64_t iter_count = 0;
  int32_t* blk_sweeps = nullptr;  // device
  int32_t large_grid_best = 0;    // grid chosen for the cooperative Jacobi kernel
  int64_t stage_bytes[16] = {0};  // algorithmic bytes of each profiling stage
  std::vector<int32_t> row_perm;  // device row q holds the constraint row row_perm[q]
  int64_t* cat_map = nullptr;     // device iterate exchange: source of each concatenated position (lazy)
  int64_t cat_total = 0;
  double* cat_stage = nullptr;    // 2 x cat_total doubles: device staging of the host iterate exchange (lazy)
  // persistent batched path
  bool persistent = false;
  int32_t solve_mode = 0;
  int32_t weighted_form = 0;  // 0 eq. (42), 1 direct, 2 extra polynomials
  int32_t p_grid = 0, p_dynamic = 0, p_tried = 0, p_max_small = 0, p_max_teff = 0;
  float p_best_ms = 0.f;
  uint32_t *p_bar = nullptr, *p_queue = nullptr;
  int32_t *p_nactive = nullptr, *p_iters = nullptr, *p_sched = nullptr;
  int32_t p_nsched = 0;
  InstReport* p_rep = nullptr;
  cudaGraphExec_t graph = nullptr;
  bool graph_tried = false;
  // small-block projections of an iteration run beside the large-block ones
  // (disjoint blocks): forked onto this stream after the affine step, joined
  // before the next step
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::string err;
};

namespace {

int set_err(sos_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return set_err(h, SOS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename V>
int upload(sos_handle* h, const std::vector<V>& v, V** out) {
  *out = nullptr;
  size_t bytes = std::max<size_t>(1, v.size()) * sizeof(V);
  void* p = nullptr;
  CK(cudaMalloc(&p, bytes));
  h->allocs.push_back(p);
  if (!v.empty()) CK(cudaMemcpy(p, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice));
  *out = static_cast<V*>(p);
  return SOS_OK;
}

template <typename V>
int alloc(sos_handle* h, size_t count, V** out) {
  void* p = nullptr;
  CK(cudaMalloc(&p, std::max<size_t>(1, count) * sizeof(V)));
  CK(cudaMemset(p, 0, std::max<size_t>(1, count) * sizeof(V)));
  h->allocs.push_back(p);
  *out = static_cast<V*>(p);
  return SOS_OK;
}

#define TRY(x)            \
  do {                    \
    int r_ = (x);         \
    if (r_ != SOS_OK) return r_; \
  } while (0)

// Shared (type-independent) device arrays, filled once.
struct Common {
  const InstInfo* inst;
  InstState* st;
  InstResid* resid;
  const BlockDesc* blocks;
  const double *b, *pinv, *h2, *lr_val, *lrr_val, *lr_c, *lr_g, *linv, *linv_t;
  const int32_t *row_inst, *row_ptr, *ent_row, *lr_ptr, *lr_row, *lrr_ptr, *lrr_col, *lr_inst;
  const uint32_t* row_ent;
  const int64_t* lr_ent;
  const int64_t *ent_sl_off, *lr_sl_off;
  const int32_t* col_perm;
  const uint32_t* ent_sl;
  const int32_t* lr_sl_col;
  const double* lr_sl_val;
  double* wl;
  double *tau, *kappa, *xP, *ylr, *zlr, *wq, *sig2, *ra, *atyl;
  int32_t* err;
  int32_t* blk_sweeps;
};

// Clock cycles of a wait bound given in microseconds (0: about 2 s).
long long wait_cycles(int32_t us) {
  if (us <= 0) return 4000000000ll;
  int dev = 0, khz = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess || khz <= 0) khz = 2070000;
  return static_cast<long long>(us) * khz / 1000;
}

template <typename T>
int make_devplan(sos_handle* h, const Common& c, int32_t max_teff, DevPlan<T>& p) {
  p.n_inst = h->n_inst;
  p.NX = h->NX;
  p.M = h->M;
  p.TL = h->TL;
  p.max_teff = max_teff;
  p.inst = c.inst;
  p.st = c.st;
  p.active = h->active;
  p.resid = c.resid;
  p.blocks = c.blocks;
  p.b = c.b;
  p.pinv = c.pinv;
  p.h2 = c.h2;
  p.row_inst = c.row_inst;
  p.row_ptr = c.row_ptr;
  p.row_ent = c.row_ent;
  p.ent_row = c.ent_row;
  p.lr_ptr = c.lr_ptr;
  p.lr_row = c.lr_row;
  p.lr_val = c.lr_val;
  p.lrr_ptr = c.lrr_ptr;
  p.lrr_col = c.lrr_col;
  p.lrr_val = c.lrr_val;
  p.lr_ent = c.lr_ent;
  p.lr_inst = c.lr_inst;
  p.lr_c = c.lr_c;
  p.lr_g = c.lr_g;
  p.linv = c.linv;
  p.linv_t = c.linv_t;
  p.col_perm = c.col_perm;
  p.ent_sl_off = c.ent_sl_off;
  p.ent_sl = c.ent_sl;
  p.lr_sl_off = c.lr_sl_off;
  p.lr_sl_col = c.lr_sl_col;
  p.lr_sl_val = c.lr_sl_val;
  p.wl = c.wl;
  p.tau = c.tau;
  p.kappa = c.kappa;
  p.xP = c.xP;
  p.ylr = c.ylr;
  p.zlr = c.zlr;
  p.wq = c.wq;
  p.sig2 = c.sig2;
  p.ra = c.ra;
  p.atyl = c.atyl;
  p.err = c.err;
  p.blk_sweeps = c.blk_sweeps;
  TRY(alloc(h, h->NX, &p.ux));
  TRY(alloc(h, h->NX, &p.vx));
  TRY(alloc(h, h->M, &p.uy));
  TRY(alloc(h, h->M, &p.vy));
  TRY(alloc(h, h->M, &p.uh2));
  p.wait_limit = wait_cycles(h->wait_limit_us);
  return SOS_OK;
}

template <typename T>
int make_large(sos_handle* h, std::vector<LargeBlock<T>>& out, const std::vector<int>& bids) {
  for (int bid : bids) {
    LargeBlock<T> lb{};
    lb.bid = bid;
    lb.N = h->blocks[bid].N;
    const size_t Np = lb.N + (lb.N & 1);
    lb.grid = large_grid_size(lb.N);
    TRY(alloc(h, Np * Np, &lb.scratch.Wf));
    TRY(alloc(h, Np * Np, &lb.scratch.B0));
    TRY(alloc(h, Np * Np, &lb.scratch.B1));
    TRY(alloc(h, Np * Np, &lb.scratch.V));
    TRY(alloc(h, Np * Np, &lb.scratch.T1));
    TRY(alloc(h, large_partials_size(lb.grid, lb.N), &lb.scratch.partial));
    TRY(alloc(h, kMaxSweeps, &lb.scratch.flags));
    TRY(alloc(h, 2, &lb.scratch.bar));
    TRY(alloc(h, 1, &lb.scratch.sweeps_out));
    TRY(alloc(h, 1, &lb.scratch.warm));
    if (sizeof(T) == 8 && tri_path(lb.N)) TRY(alloc(h, 5 * Np * Np, &lb.scratch.F32));
    lb.scratch.warm_limit = h->warm64.limit;  // same restart period as the small blocks
    out.push_back(lb);
  }
  return SOS_OK;
}

template <typename T, typename TC>
cudaError_t enqueue_stage(sos_handle* h, const DevPlan<T>& p, std::vector<LargeBlock<TC>>& large,
                          const SmallWarm<TC>& wm, int stage) {
  cudaError_t e = cudaSuccess;
  if (stage >= 4 && stage <= 9) return launch_affine_part<T>(p, h->shape, stage - 4, h->stream);
  if (stage >= 10 && stage <= 15) {
    for (auto& lb : large) {
      e = launch_psd_large_part<T, TC>(p, lb.bid, lb.N, lb.scratch, lb.grid, stage - 10, h->stream);
      if (e != cudaSuccess) return e;
    }
    return e;
  }
  if (stage == 0 || stage == 3) {
    e = launch_affine<T>(p, h->shape, h->stream);
    if (e != cudaSuccess) return e;
  }
  const bool fork = stage == 3 && h->side && !h->small.empty() && (!large.empty() || !h->ns_large.empty());
  if (fork) {
    e = cudaEventRecord(h->ev_fork, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->ev_fork, 0);
    if (e != cudaSuccess) return e;
  }
  if (stage == 1 || stage == 3)
    for (auto& c : h->small) {
      e = launch_psd_small<T, TC>(p, c.ids, c.count, c.maxN, wm, fork ? h->side : h->stream);
      if (e != cudaSuccess) return e;
    }
  if (fork) {
    e = cudaEventRecord(h->ev_join, h->side);
    if (e != cudaSuccess) return e;
  }
  if (stage == 2 || stage == 3) {
    for (auto& lb : large) {
      e = launch_psd_large<T, TC>(p, lb.bid, lb.N, lb.scratch, lb.grid, h->stream);
      if (e != cudaSuccess) return e;
    }
    for (auto& nb : h->ns_large) {
      e = launch_psd_ns<T>(p, nb.bid, nb.N, nb.s, h->stream);
      if (e != cudaSuccess) return e;
    }
  }
  if (fork) e = cudaStreamWaitEvent(h->stream, h->ev_join, 0);
  return e;
}

cudaError_t enqueue_any(sos_handle* h, int stage) {
  if (h->precision == SOS_PREC_FP64) return enqueue_stage<double, double>(h, h->d64, h->large64, h->warm64, stage);
  if (h->precision == SOS_PREC_MIXED) return enqueue_stage<double, float>(h, h->d64, h->large32, h->warm32, stage);
  return enqueue_stage<float, float>(h, h->d32, h->large32, h->warm32, stage);
}

cudaError_t enqueue_iteration(sos_handle* h) { return enqueue_any(h, 3); }

bool iter64(const sos_handle* h) { return h->precision != SOS_PREC_FP32; }

void reset_warm(sos_handle* h) {
  for (auto& lb : h->large64) cudaMemsetAsync(lb.scratch.warm, 0, sizeof(int32_t), h->stream);
  for (auto& lb : h->large32) cudaMemsetAsync(lb.scratch.warm, 0, sizeof(int32_t), h->stream);
  if (h->warm64.count) cudaMemsetAsync(h->warm64.count, 0, sizeof(int32_t) * h->blocks.size(), h->stream);
  if (h->warm32.count) cudaMemsetAsync(h->warm32.count, 0, sizeof(int32_t) * h->blocks.size(), h->stream);
}

int check_err_word(sos_handle* h) {
  int32_t e = 0;
  CK(cudaMemcpyAsync(&e, h->d64.err, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (e != 0) {
    cudaMemsetAsync(h->d64.err, 0, sizeof(int32_t), h->stream);
    return set_err(h, SOS_ERR_TIMEOUT, "a bounded device-side wait expired");
  }
  return SOS_OK;
}

int init_wl(sos_handle* h) {
  CK(iter64(h) ? launch_init_wl<double>(h->d64, h->stream) : launch_init_wl<float>(h->d32, h->stream));
  return SOS_OK;
}

int cold_start(sos_handle* h) {
  std::vector<double> one(h->n_inst, 1.0);
  CK(cudaMemcpyAsync(h->d64.tau, one.data(), sizeof(double) * h->n_inst, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->d64.kappa, one.data(), sizeof(double) * h->n_inst, cudaMemcpyHostToDevice, h->stream));
  if (iter64(h)) {
    CK(cudaMemsetAsync(h->d64.ux, 0, sizeof(double) * h->NX, h->stream));
    CK(cudaMemsetAsync(h->d64.vx, 0, sizeof(double) * h->NX, h->stream));
    CK(cudaMemsetAsync(h->d64.uy, 0, sizeof(double) * h->M, h->stream));
    CK(cudaMemsetAsync(h->d64.vy, 0, sizeof(double) * h->M, h->stream));
  } else {
    CK(cudaMemsetAsync(h->d32.ux, 0, sizeof(float) * h->NX, h->stream));
    CK(cudaMemsetAsync(h->d32.vx, 0, sizeof(float) * h->NX, h->stream));
    CK(cudaMemsetAsync(h->d32.uy, 0, sizeof(float) * h->M, h->stream));
    CK(cudaMemsetAsync(h->d32.vy, 0, sizeof(float) * h->M, h->stream));
  }
  TRY(init_wl(h));
  std::fill(h->active_h.begin(), h->active_h.end(), 1);
  CK(cudaMemcpyAsync(h->active, h->active_h.data(), sizeof(int32_t) * h->n_inst, cudaMemcpyHostToDevice, h->stream));
  std::fill(h->iters_h.begin(), h->iters_h.end(), 0);
  std::fill(h->status_h.begin(), h->status_h.end(), SOS_RUNNING);
  h->iter_count = 0;
  reset_warm(h);
  CK(cudaStreamSynchronize(h->stream));
  return SOS_OK;
}

template <typename T, typename TC>
PersistArgs<TC> persist_args(sos_handle* h, const SmallWarm<TC>& wm, int32_t max_iter, int32_t k_check, double tol) {
  PersistArgs<TC> a;
  a.max_iter = max_iter;
  a.k_check = k_check;
  a.tol = tol;
  a.infeas_tol = h->infeas_tol;
  a.bar = h->p_bar;
  a.queue = h->p_queue;
  a.active = h->active;
  a.n_active = h->p_nactive;
  a.rep = h->p_rep;
  a.sched = h->p_sched;
  a.n_sched = h->p_nsched;
  a.dynamic = h->p_dynamic;
  a.wm = wm;
  a.iters_done = h->p_iters;
  return a;
}

cudaError_t launch_persist(sos_handle* h, int32_t max_iter, int32_t k_check, double tol) {
  if (h->precision == SOS_PREC_FP64)
    return launch_persistent<double, double>(h->d64, persist_args<double, double>(h, h->warm64, max_iter, k_check, tol),
                                             h->p_grid, h->p_max_small, h->p_max_teff, h->stream);
  if (h->precision == SOS_PREC_MIXED)
    return launch_persistent<double, float>(h->d64, persist_args<double, float>(h, h->warm32, max_iter, k_check, tol),
                                            h->p_grid, h->p_max_small, h->p_max_teff, h->stream);
  return launch_persistent<float, float>(h->d32, persist_args<float, float>(h, h->warm32, max_iter, k_check, tol),
                                         h->p_grid, h->p_max_small, h->p_max_teff, h->stream);
}

int max_ctas_per_sm(sos_handle* h) {
  if (h->precision == SOS_PREC_FP64) return persistent_max_ctas_per_sm<double, double>(h->p_max_small, h->p_max_teff);
  if (h->precision == SOS_PREC_MIXED) return persistent_max_ctas_per_sm<double, float>(h->p_max_small, h->p_max_teff);
  return persistent_max_ctas_per_sm<float, float>(h->p_max_small, h->p_max_teff);
}

int cold_start(sos_handle* h);
}  // namespace
extern "C" int sos_iterate(sos_handle* h, int32_t iters);
namespace {

// Autotuner of the persistent launch: times a few iterations for every
// (CTAs per SM, schedule) candidate from the cold start, keeps the fastest,
// and returns the iterate to the cold start.
int autotune_persistent(sos_handle* h) {
  const int occ = max_ctas_per_sm(h);
  if (occ < 1) return set_err(h, SOS_ERR_CUDA, "persistent kernel cannot be resident");
  const int max_per = occ < 4 ? occ : 4;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_grid = h->shape.sms, best_dyn = 0, tried = 0;
  const int32_t reps = 3;
  for (int per = 1; per <= max_per; ++per)
    for (int dyn = 0; dyn <= 1; ++dyn) {
      h->p_grid = h->shape.sms * per;
      h->p_dynamic = dyn;
      CK(launch_persist(h, 1, 0, 0.0));  // warm-up of this shape
      CK(cudaEventRecord(e0, h->stream));
      CK(launch_persist(h, reps, 0, 0.0));
      CK(cudaEventRecord(e1, h->stream));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      ++tried;
      if (ms < best) {
        best = ms;
        best_grid = h->p_grid;
        best_dyn = dyn;
      }
    }
  // the per-phase kernel path (one CUDA graph per iteration) is a candidate too
  float graph_ms = 1e30f;
  if (h->solve_mode == 0) {
    h->persistent = false;
    int rc = sos_iterate(h, 1);  // builds the graph
    if (rc != SOS_OK) return rc;
    CK(cudaEventRecord(e0, h->stream));
    rc = sos_iterate(h, reps);
    if (rc != SOS_OK) return rc;
    CK(cudaEventRecord(e1, h->stream));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&graph_ms, e0, e1));
    ++tried;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->persistent = !(graph_ms < best);
  h->p_grid = best_grid;
  h->p_dynamic = best_dyn;
  h->p_tried = tried;
  h->p_best_ms = (h->persistent ? best : graph_ms) / reps;
  return cold_start(h);
}

// Grid size of the cooperative Jacobi kernel of each large block: times one
// projection (after one affine step from the cold start, so the input is a
// realistic W) for 1/4, 1/2 and all SMs, keeps the fastest, and resets the
// iterate.  Fewer CTAs make each grid barrier cheaper; more give more FP64
// and FP32 throughput per round.  FP64 blocks on the tridiagonal path take
// every SM without a trial: there the grid only sizes the tile products of
// the refinement and reconstruction, which divide evenly over the CTAs.
template <typename TC>
int autotune_large(sos_handle* h, std::vector<LargeBlock<TC>>& large) {
  if (large.empty()) return SOS_OK;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(enqueue_any(h, 0));
  const int sms = h->shape.sms;
  const int cands[3] = {sms / 4, sms / 2, sms};
  for (auto& lb : large) {
    float best = 1e30f;
    int best_g = sms;
    if (sizeof(TC) == 8 && tri_path(lb.N)) {
      lb.grid = sms;
      h->large_grid_best = sms;
      continue;
    }
    for (int g : cands) {
      if (g < 1) continue;
      lb.grid = g;
      for (auto& other : large) CK(cudaMemsetAsync(other.scratch.warm, 0, sizeof(int32_t), h->stream));
      CK(cudaEventRecord(e0, h->stream));
      CK(enqueue_any(h, 2));
      CK(cudaEventRecord(e1, h->stream));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        best_g = g;
      }
    }
    lb.grid = best_g;
    h->large_grid_best = best_g;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return check_err_word(h);
}

// Renumbers the rows of each instance in order of decreasing length (A_L
// nonzeros, then plain Gram entries) so that 32 consecutive rows have similar
// lengths: a warp of the row kernels then keeps its lanes busy, and every
// row-indexed array is read and written contiguously.  perm[new] = old; the
// host converts the y part of iterates and results with it.
void renumber_rows(HostPlan& P, std::vector<int32_t>& perm) {
  const int64_t M = P.M;
  perm.resize(M);
  for (int64_t a = 0; a < M; ++a) perm[a] = static_cast<int32_t>(a);
  for (const InstInfo& in : P.inst) {
    auto first = perm.begin() + in.y_off, last = first + in.m;
    std::stable_sort(first, last, [&](int32_t x, int32_t y) {
      const int lx = P.lrr_ptr[x + 1] - P.lrr_ptr[x], ly = P.lrr_ptr[y + 1] - P.lrr_ptr[y];
      if (lx != ly) return lx > ly;
      return P.row_ptr[x + 1] - P.row_ptr[x] > P.row_ptr[y + 1] - P.row_ptr[y];
    });
  }
  std::vector<int32_t> inv(M);
  for (int64_t q = 0; q < M; ++q) inv[perm[q]] = static_cast<int32_t>(q);
  auto permute = [&](auto& v) {
    auto w = v;
    for (int64_t q = 0; q < M; ++q) w[q] = v[perm[q]];
    v.swap(w);
  };
  permute(P.b);
  permute(P.pinv);
  permute(P.h2);
  permute(P.row_inst);
  {  // plain entries per row
    std::vector<int32_t> ptr(M + 1, 0);
    std::vector<uint32_t> ent;
    ent.reserve(P.row_ent.size());
    for (int64_t q = 0; q < M; ++q) {
      const int32_t a = perm[q];
      for (int k = P.row_ptr[a]; k < P.row_ptr[a + 1]; ++k) ent.push_back(P.row_ent[k]);
      ptr[q + 1] = static_cast<int32_t>(ent.size());
    }
    P.row_ptr.swap(ptr);
    P.row_ent.swap(ent);
  }
  {  // A_L rows
    std::vector<int32_t> ptr(M + 1, 0), col;
    std::vector<double> val;
    col.reserve(P.lrr_col.size());
    val.reserve(P.lrr_val.size());
    for (int64_t q = 0; q < M; ++q) {
      const int32_t a = perm[q];
      for (int k = P.lrr_ptr[a]; k < P.lrr_ptr[a + 1]; ++k) {
        col.push_back(P.lrr_col[k]);
        val.push_back(P.lrr_val[k]);
      }
      ptr[q + 1] = static_cast<int32_t>(col.size());
    }
    P.lrr_ptr.swap(ptr);
    P.lrr_col.swap(col);
    P.lrr_val.swap(val);
  }
  for (auto& r : P.ent_row)  // row of each plain entry (flag bit kept)
    if (r >= 0) r = inv[r & ~kEntOffBit] | (r & kEntOffBit);
  for (auto& r : P.lr_row) r = inv[r];  // rows of the A_L columns
}

// Algorithmic bytes of each profiling stage (sos_stage_bytes): every array
// element the stage has to read or write, counted once.  es is the size of an
// iterate element, tcs the element size of the stored eigenvectors.
void compute_stage_bytes(sos_handle* h, const HostPlan& P, const std::vector<int>& large) {
  const int64_t es = h->precision == SOS_PREC_FP32 ? 4 : 8;
  const int64_t tcs = h->precision == SOS_PREC_FP64 ? 8 : 4;
  const int64_t M = P.M, nent = static_cast<int64_t>(P.row_ent.size());
  const int64_t nnz = static_cast<int64_t>(P.lr_row.size()), TL = P.TL, ni = P.n_inst;
  int64_t tri = 0, te_sum = 0, t_sum = 0;
  for (const InstInfo& in : P.inst) {
    tri += static_cast<int64_t>(in.t_eff) * (in.t_eff + 1) / 2;
    te_sum += in.t_eff;
    t_sum += in.t;
  }
  int64_t* b = h->stage_bytes;
  // rows_r: rows (row_inst, u_y, v_y, b, pinv, row_ptr, lrr_ptr, x), plain
  // entries (row_ent, u, v), A_L rows (lrr_col, lrr_val), low-rank columns
  // (lr_ent, u, v, lr_c), per instance tau, kappa, active
  b[4] = M * (4 + 2 * es + 8 + 8 + 4 + 4 + 8) + nent * (4 + 2 * es) + nnz * 12 + TL * (16 + 2 * es) + ni * 20;
  // lr_y: A_L columns (lr_ptr, lr_inst, y_L), nonzeros (lr_val, lr_row), x
  b[5] = TL * 16 + nnz * 12 + M * 8 + ni * 4;
  // woodbury: the lower triangle of L^-1, y_L in, z out
  b[6] = tri * 8 + te_sum * 16 + ni * static_cast<int64_t>(sizeof(InstInfo));
  // rows_sigma2: rows (row_inst, lrr_ptr, x, pinv, sigma_2), nonzeros, z
  b[7] = M * 32 + nnz * 12 + TL * 8;
  // inst_scalar: b and sigma_2 per row; per free variable lr_c, u, v, z and
  // the writes of u, v
  b[8] = M * 16 + t_sum * (8 + 2 * es + 8 + 8 + 2 * es) + ni * 64;
  // rows_y: rows (row_inst, sigma_2, h_2, v_y in; u_y, v_y, u_hat_2 out)
  b[9] = M * (4 + 8 + 8 + 4 * es) + ni * 8;
  b[0] = b[4] + b[5] + b[6] + b[7] + b[8] + b[9];
  // projections: per packed entry the input (u, ent_row, u_hat_2 / z), the
  // outputs u and v, and the stored eigenvectors read and written
  std::vector<char> is_large(P.blocks.size(), 0);
  for (int bid : large) is_large[bid] = 1;
  b[1] = b[2] = 0;
  for (size_t k = 0; k < P.blocks.size(); ++k) {
    const int64_t N = P.blocks[k].N, L = N * (N + 1) / 2;
    b[is_large[k] ? 2 : 1] += L * (4 + 3 * es) + 2 * N * N * tcs;
  }
  b[3] = b[0] + b[1] + b[2];
}

int build(sos_handle* h, const sos_program* progs, int32_t n_progs) {
  HostPlan P;
  std::string err;
  int rc = build_plan(progs, n_progs, P, err, h->weighted_form);
  if (rc != SOS_OK) return set_err(h, rc, err);
  renumber_rows(P, h->row_perm);
  h->n_inst = P.n_inst;
  h->NX = P.NX;
  h->M = P.M;
  h->TL = P.TL;
  h->inst = P.inst;
  h->blocks = P.blocks;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&h->shape.sms, cudaDevAttrMultiProcessorCount, dev));

  Common c{};
  InstInfo* inst;
  TRY(upload(h, P.inst, &inst));
  c.inst = inst;
  InstState* st;
  TRY(alloc(h, h->n_inst, &st));
  c.st = st;
  InstResid* resid;
  TRY(alloc(h, h->n_inst, &resid));
  c.resid = resid;
  BlockDesc* bl;
  TRY(upload(h, P.blocks, &bl));
  c.blocks = bl;
  double* dp;
  TRY(upload(h, P.b, &dp));
  c.b = dp;
  TRY(upload(h, P.pinv, &dp));
  c.pinv = dp;
  TRY(upload(h, P.h2, &dp));
  c.h2 = dp;
  TRY(upload(h, P.lr_val, &dp));
  c.lr_val = dp;
  TRY(upload(h, P.lrr_val, &dp));
  c.lrr_val = dp;
  TRY(upload(h, P.lr_c, &dp));
  c.lr_c = dp;
  TRY(upload(h, P.lr_g, &dp));
  c.lr_g = dp;
  TRY(upload(h, P.linv, &dp));
  c.linv = dp;
  {  // column-major copy of every L^-1
    std::vector<double> lt(P.linv.size(), 0.0);
    for (const InstInfo& in : P.inst) {
      const int64_t te = in.t_eff;
      const double* src = P.linv.data() + in.linv_off;
      double* dst = lt.data() + in.linv_off;
      for (int64_t r = 0; r < te; ++r)
        for (int64_t k = 0; k <= r; ++k) dst[k * te + r] = src[r * te + k];
    }
    TRY(upload(h, lt, &dp));
    c.linv_t = dp;
  }
  int32_t* ip;
  TRY(upload(h, P.row_inst, &ip));
  c.row_inst = ip;
  TRY(upload(h, P.row_ptr, &ip));
  c.row_ptr = ip;
  TRY(upload(h, P.ent_row, &ip));
  c.ent_row = ip;
  TRY(upload(h, P.lr_ptr, &ip));
  c.lr_ptr = ip;
  TRY(upload(h, P.lr_row, &ip));
  c.lr_row = ip;
  TRY(upload(h, P.lrr_ptr, &ip));
  c.lrr_ptr = ip;
  TRY(upload(h, P.lrr_col, &ip));
  c.lrr_col = ip;
  TRY(upload(h, P.lr_inst, &ip));
  c.lr_inst = ip;
  uint32_t* up;
  TRY(upload(h, P.row_ent, &up));
  c.row_ent = up;
  int64_t* lp;
  TRY(upload(h, P.lr_ent, &lp));
  c.lr_ent = lp;
  {  // sliced row lists: 32 consecutive rows (already ordered by length by
     // renumber_rows) form a slice, element k of row a lies at
     // off[a / 32] + 32 k + a % 32
    const int64_t n_sl = (h->M + 31) / 32;
    std::vector<int64_t> eoff(n_sl + 1, 0), loff(n_sl + 1, 0);
    for (int64_t sl = 0; sl < n_sl; ++sl) {
      int we = 0, wlr = 0;
      for (int64_t a = sl * 32; a < std::min<int64_t>(h->M, sl * 32 + 32); ++a) {
        we = std::max(we, P.row_ptr[a + 1] - P.row_ptr[a]);
        wlr = std::max(wlr, P.lrr_ptr[a + 1] - P.lrr_ptr[a]);
      }
      eoff[sl + 1] = eoff[sl] + 32 * static_cast<int64_t>(we);
      loff[sl + 1] = loff[sl] + 32 * static_cast<int64_t>(wlr);
    }
    std::vector<uint32_t> esl(std::max<int64_t>(eoff[n_sl], 1), 0u);
    std::vector<int32_t> lcol(std::max<int64_t>(loff[n_sl], 1), 0);
    std::vector<double> lval(std::max<int64_t>(loff[n_sl], 1), 0.0);
    for (int64_t a = 0; a < h->M; ++a) {
      const int64_t sl = a / 32, lane = a % 32;
      for (int k = P.row_ptr[a]; k < P.row_ptr[a + 1]; ++k)
        esl[eoff[sl] + 32 * static_cast<int64_t>(k - P.row_ptr[a]) + lane] = P.row_ent[k];
      for (int k = P.lrr_ptr[a]; k < P.lrr_ptr[a + 1]; ++k) {
        const int64_t q = loff[sl] + 32 * static_cast<int64_t>(k - P.lrr_ptr[a]) + lane;
        lcol[q] = P.lrr_col[k];
        lval[q] = P.lrr_val[k];
      }
    }
    int64_t* op;
    TRY(upload(h, eoff, &op));
    c.ent_sl_off = op;
    TRY(upload(h, loff, &op));
    c.lr_sl_off = op;
    uint32_t* eup;
    TRY(upload(h, esl, &eup));
    c.ent_sl = eup;
    int32_t* pp;
    // columns of A_L (CSC) ordered by decreasing length within each instance,
    // so the four columns a warp takes together have similar lengths
    std::vector<int32_t> cperm(std::max<int32_t>(h->TL, 1), 0);
    for (int32_t j = 0; j < h->TL; ++j) cperm[j] = j;
    for (const InstInfo& in : P.inst) {
      auto first = cperm.begin() + in.lr_off, last = first + in.t_eff;
      std::stable_sort(first, last, [&](int32_t x, int32_t y) {
        return P.lr_ptr[x + 1] - P.lr_ptr[x] > P.lr_ptr[y + 1] - P.lr_ptr[y];
      });
    }
    TRY(upload(h, cperm, &pp));
    c.col_perm = pp;
    int32_t* cp;
    TRY(upload(h, lcol, &cp));
    c.lr_sl_col = cp;
    double* vp;
    TRY(upload(h, lval, &vp));
    c.lr_sl_val = vp;
  }
  TRY(alloc(h, std::max<int64_t>(h->TL, 1), &c.wl));
  TRY(alloc(h, h->n_inst, &c.tau));
  TRY(alloc(h, h->n_inst, &c.kappa));
  TRY(alloc(h, h->M, &c.xP));
  TRY(alloc(h, h->TL, &c.ylr));
  TRY(alloc(h, h->TL, &c.zlr));
  TRY(alloc(h, h->TL, &c.wq));
  TRY(alloc(h, h->M, &c.sig2));
  TRY(alloc(h, h->M, &c.ra));
  TRY(alloc(h, h->TL, &c.atyl));
  TRY(alloc(h, 1, &c.err));
  TRY(alloc(h, P.blocks.size(), &c.blk_sweeps));
  h->blk_sweeps = c.blk_sweeps;
  TRY(alloc(h, h->n_inst, &h->active));
  h->active_h.assign(h->n_inst, 1);
  h->iters_h.assign(h->n_inst, 0);
  h->status_h.assign(h->n_inst, SOS_RUNNING);

  int32_t max_teff = 0;
  for (auto& in : P.inst) max_teff = std::max(max_teff, in.t_eff);

  // projection classes: small blocks (shared-memory Jacobi) by size class, large blocks (grid Jacobi)
  const bool fp64 = h->precision == SOS_PREC_FP64;  // FP64 projections
  const int form = fp64 ? kFormFP64 : (h->precision == SOS_PREC_MIXED ? kFormMixed : kFormFP32);
  // A one-CTA FP64 Jacobi runs on a single SM's FP64 pipe; with one program
  // (a few blocks) the grid path, which spreads each round over every SM, is
  // faster from N > 32 on (N = 91: 4.5 -> ~1 ms per iteration).  Batches keep
  // the one-CTA kernel, which fills the GPU with blocks.
  const int small_cap = (fp64 && P.n_inst == 1 && h->solve_mode != 2) ? 32 : psd_small_max_n(form);
  constexpr int kClasses = 7;
  const int caps[kClasses] = {16, 32, 48, 64, 96, 112, 128};
  std::vector<std::vector<int32_t>> cls(kClasses);
  std::vector<int> large;
  int max_small = 0;
  for (int b = 0; b < static_cast<int>(P.blocks.size()); ++b) {
    const int N = P.blocks[b].N;
    if (N > small_cap) {
      large.push_back(b);
      continue;
    }
    for (int k = 0; k < kClasses; ++k)
      if (N <= caps[k]) {
        cls[k].push_back(b);
        break;
      }
  }
  // shared memory of a class is sized for its largest member (rounded up to
  // even), so e.g. a batch of N = 66 blocks fits three CTAs per SM
  int cls_n[kClasses] = {0};
  for (int k = 0; k < kClasses; ++k) {
    for (int32_t b : cls[k]) cls_n[k] = std::max(cls_n[k], P.blocks[b].N + (P.blocks[b].N & 1));
    max_small = std::max(max_small, cls_n[k]);
  }
  compute_stage_bytes(h, P, large);
  // eigenvector storage of small blocks (warm start)
  int64_t voff = 0;
  for (int k = 0; k < kClasses; ++k)
    for (int32_t b : cls[k]) {
      P.blocks[b].v_off = voff;
      voff += static_cast<int64_t>(P.blocks[b].N) * P.blocks[b].N;
    }
  h->blocks = P.blocks;
  BlockDesc* bl2;
  TRY(upload(h, P.blocks, &bl2));
  c.blocks = bl2;
  if (fp64) {
    TRY(alloc(h, static_cast<size_t>(voff), &h->warm64.V));
    TRY(alloc(h, P.blocks.size(), &h->warm64.count));
  } else {
    TRY(alloc(h, static_cast<size_t>(voff), &h->warm32.V));
    TRY(alloc(h, P.blocks.size(), &h->warm32.count));
  }
  for (int k = 0; k < kClasses; ++k)
    if (!cls[k].empty()) {
      SmallClass sc{cls_n[k], static_cast<int>(cls[k].size()), nullptr};
      TRY(upload(h, cls[k], &sc.ids));
      h->small.push_back(sc);
    }
  if (h->precision == SOS_PREC_FP64) {
    TRY(make_devplan(h, c, max_teff, h->d64));
    TRY(make_large(h, h->large64, large));
    // the iterations of a solve first try each tridiagonal-path block's
    // refinement from the previous iteration's eigenvectors
    for (auto& lb : h->large64) lb.scratch.tri_warm = 1;
    CK((prepare_kernels<double, double>(max_small, max_teff)));
  } else {
    // FP32 projections: large blocks by Newton-Schulz on the tensor cores
    // unless the Jacobi grid kernel is requested
    std::vector<int> jac;
    for (int b : large) {
      if (h->large_method == 1) {
        jac.push_back(b);
        continue;
      }
      NsBlock nb{};
      nb.bid = b;
      nb.N = P.blocks[b].N;
      const size_t Np = static_cast<size_t>(ns_padded(nb.N));
      TRY(alloc(h, Np * Np, &nb.s.Wf));
      TRY(alloc(h, Np * Np, &nb.s.X));
      TRY(alloc(h, Np * Np, &nb.s.Xn));
      TRY(alloc(h, 4 * ns_split_bytes(static_cast<int>(Np)), &nb.s.split));
      TRY(alloc(h, 2 * static_cast<size_t>(ns_grid(nb.N)), &nb.s.partial));
      TRY(alloc(h, 2, &nb.s.bar));
      TRY(alloc(h, 1, &nb.s.iters_out));
      h->ns_large.push_back(nb);
    }
    if (h->precision == SOS_PREC_MIXED) {
      TRY(make_devplan(h, c, max_teff, h->d64));
      TRY(make_large(h, h->large32, jac));
      CK((prepare_kernels<double, float>(max_small, max_teff)));
    } else {
      TRY(make_devplan(h, c, max_teff, h->d32));
      TRY(make_large(h, h->large32, jac));
      CK((prepare_kernels<float, float>(max_small, max_teff)));
    }
  }
  h->d64.tau = c.tau;  // FP64 scalars shared by every form
  h->d64.kappa = c.kappa;
  h->d64.err = c.err;
  h->d64.resid = c.resid;
  if (!h->small.empty() && !large.empty()) {  // small and large projections side by side
    CK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  }
  // persistent batched path: every block small, and either requested or a batch
  const bool eligible = large.empty();
  h->persistent = eligible && (h->solve_mode == 2 || (h->solve_mode == 0 && n_progs > 1));
  // (auto mode keeps the persistent launch only if the autotuner finds it faster)
  if (h->solve_mode == 2 && !eligible)
    return set_err(h, SOS_ERR_UNSUPPORTED, "the persistent solver needs every Gram block to be small");
  // grid size of the large-block Jacobi kernel
  TRY(cold_start(h));
  TRY(h->precision == SOS_PREC_FP64 ? autotune_large(h, h->large64) : autotune_large(h, h->large32));
  if (h->persistent) {
    std::vector<int32_t> order;
    for (int k = 5; k >= 0; --k)
      for (int32_t b : cls[k]) order.push_back(b);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t x, int32_t y) { return P.blocks[x].N > P.blocks[y].N; });
    h->p_nsched = static_cast<int32_t>(order.size());
    TRY(upload(h, order, &h->p_sched));
    TRY(alloc(h, 2, &h->p_bar));
    TRY(alloc(h, 1, &h->p_queue));
    TRY(alloc(h, 1, &h->p_nactive));
    TRY(alloc(h, 1, &h->p_iters));
    TRY(alloc(h, h->n_inst, &h->p_rep));
    h->p_max_small = max_small;
    h->p_max_teff = max_teff;
    TRY(cold_start(h));
    return autotune_persistent(h);
  }
  return cold_start(h);
}

template <typename T>
int copy_iterate_out(sos_handle* h, const DevPlan<T>& p, std::vector<double>& ux, std::vector<double>& vx,
                     std::vector<double>& uy, std::vector<double>& vy, std::vector<double>& tau,
                     std::vector<double>& kappa) {
  std::vector<T> a(h->NX), b(h->NX), c(h->M), dd(h->M);
  CK(cudaMemcpyAsync(a.data(), p.ux, sizeof(T) * h->NX, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(b.data(), p.vx, sizeof(T) * h->NX, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(c.data(), p.uy, sizeof(T) * h->M, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(dd.data(), p.vy, sizeof(T) * h->M, cudaMemcpyDeviceToHost, h->stream));
  tau.resize(h->n_inst);
  kappa.resize(h->n_inst);
  CK(cudaMemcpyAsync(tau.data(), h->d64.tau, sizeof(double) * h->n_inst, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(kappa.data(), h->d64.kappa, sizeof(double) * h->n_inst, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  ux.assign(a.begin(), a.end());
  vx.assign(b.begin(), b.end());
  uy.resize(h->M);
  vy.resize(h->M);
  for (int64_t q = 0; q < h->M; ++q) {  // back to the order of the constraint rows
    uy[h->row_perm[q]] = c[q];
    vy[h->row_perm[q]] = dd[q];
  }
  return SOS_OK;
}

int get_all(sos_handle* h, std::vector<double>& ux, std::vector<double>& vx, std::vector<double>& uy,
            std::vector<double>& vy, std::vector<double>& tau, std::vector<double>& kappa) {
  if (iter64(h)) return copy_iterate_out(h, h->d64, ux, vx, uy, vy, tau, kappa);
  return copy_iterate_out(h, h->d32, ux, vx, uy, vy, tau, kappa);
}

}  // namespace

extern "C" {

int sos_setup(const sos_program* progs, int32_t n_progs, const sos_options* opts, sos_handle** out) {
  if (!out) return SOS_ERR_INVALID_ARG;
  *out = nullptr;
  auto h = std::make_unique<sos_handle>();
  if (opts) {
    if (opts->precision != SOS_PREC_FP64 && opts->precision != SOS_PREC_MIXED && opts->precision != SOS_PREC_FP32) {
      g_setup_error = "unknown precision";
      return SOS_ERR_INVALID_ARG;
    }
    h->precision = opts->precision;
    h->k_check = opts->k_check > 0 ? opts->k_check : 10;
    h->stream = static_cast<cudaStream_t>(opts->cuda_stream);
    h->solve_mode = opts->solve_mode;
    h->large_method = opts->large_method;
    if (h->large_method < 0 || h->large_method > 2 || (h->large_method == 2 && h->precision == SOS_PREC_FP64)) {
      g_setup_error = "large_method must be 0, 1, or 2 (2 needs FP32 projections)";
      return SOS_ERR_INVALID_ARG;
    }
    if (h->solve_mode < 0 || h->solve_mode > 2) {
      g_setup_error = "unknown solve_mode";
      return SOS_ERR_INVALID_ARG;
    }
    if (opts->warm_restart < 0) {
      g_setup_error = "warm_restart must be >= 0";
      return SOS_ERR_INVALID_ARG;
    }
    if (opts->infeas_tol < 0) {
      g_setup_error = "infeas_tol must be >= 0";
      return SOS_ERR_INVALID_ARG;
    }
    if (opts->weighted_form < 0 || opts->weighted_form > 2) {
      g_setup_error = "unknown weighted_form";
      return SOS_ERR_INVALID_ARG;
    }
    h->weighted_form = opts->weighted_form;
    if (opts->infeas_tol > 0) h->infeas_tol = opts->infeas_tol;
    if (opts->wait_limit_us < 0 || opts->reserved != 0) {
      g_setup_error = "wait_limit_us must be >= 0 and reserved 0";
      return SOS_ERR_INVALID_ARG;
    }
    h->wait_limit_us = opts->wait_limit_us;
    if (opts->warm_restart > 0)
      h->warm64.limit = h->warm32.limit = opts->warm_restart;
  }
  if (!h->stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      g_setup_error = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
      return SOS_ERR_CUDA;
    }
    h->own_stream = true;
  }
  int rc = build(h.get(), progs, n_progs);
  if (rc != SOS_OK) {
    g_setup_error = h->err;
    sos_destroy(h.release());
    return rc;
  }
  *out = h.release();
  return SOS_OK;
}

void sos_destroy(sos_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->side) {
    cudaStreamSynchronize(h->side);
    cudaStreamDestroy(h->side);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  for (void* p : h->allocs) cudaFree(p);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

const char* sos_last_error(const sos_handle* h) { return h ? h->err.c_str() : g_setup_error.c_str(); }

int sos_dims(const sos_handle* h, int32_t inst, int64_t dims[6]) {
  if (!h || !dims || inst < 0 || inst >= h->n_inst) return SOS_ERR_INVALID_ARG;
  const InstInfo& in = h->inst[inst];
  dims[0] = in.nx;
  dims[1] = in.m;
  dims[2] = in.t;
  dims[3] = in.t_eff;
  int64_t nb = 0, ent = 0;
  for (auto& b : h->blocks)
    if (b.inst == inst) {
      ++nb;
      ent += static_cast<int64_t>(b.N) * (b.N + 1) / 2;
    }
  dims[4] = nb;
  dims[5] = ent;
  return SOS_OK;
}

int sos_iterate(sos_handle* h, int32_t iters) {
  if (!h || iters < 0) return SOS_ERR_INVALID_ARG;
  if (h->persistent) {
    if (iters == 0) return SOS_OK;
    int32_t na = 0;
    for (int i = 0; i < h->n_inst; ++i) na += h->active_h[i];
    CK(cudaMemcpyAsync(h->p_nactive, &na, sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    CK(launch_persist(h, iters, 0, 0.0));
    h->iter_count += iters;
    for (int i = 0; i < h->n_inst; ++i)
      if (h->active_h[i]) h->iters_h[i] += iters;
    CK(cudaStreamSynchronize(h->stream));  // na lives on this stack frame
    return SOS_OK;
  }
  if (!h->graph_tried) {
    h->graph_tried = true;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      cudaError_t e = enqueue_iteration(h);
      cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
      if (e == cudaSuccess && e2 == cudaSuccess && g) {
        if (cudaGraphInstantiate(&h->graph, g, 0) != cudaSuccess) h->graph = nullptr;
      }
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();  // clear a failed capture
  }
  for (int k = 0; k < iters; ++k) {
    cudaError_t e = h->graph ? cudaGraphLaunch(h->graph, h->stream) : enqueue_iteration(h);
    if (e != cudaSuccess) return set_err(h, SOS_ERR_CUDA, std::string("iteration launch: ") + cudaGetErrorString(e));
  }
  h->iter_count += iters;
  for (int i = 0; i < h->n_inst; ++i)
    if (h->active_h[i]) h->iters_h[i] += iters;
  return SOS_OK;
}

int sos_sync(sos_handle* h) {
  if (!h) return SOS_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(h->stream));
  return check_err_word(h);
}

int sos_solve(sos_handle* h, double tol, int32_t max_iter, sos_result* results) {
  if (!h || max_iter < 0 || !(tol > 0)) return SOS_ERR_INVALID_ARG;
  std::vector<InstResid> R(h->n_inst);
  std::vector<double> rp(h->n_inst, NAN), rd(h->n_inst, NAN), gp(h->n_inst, NAN), po(h->n_inst, NAN),
      dobj(h->n_inst, NAN);
  int32_t done = 0;
  for (int i = 0; i < h->n_inst; ++i) done += h->active_h[i] ? 0 : 1;
  int32_t it = 0;
  if (h->persistent && done < h->n_inst && max_iter > 0) {
    int32_t na = h->n_inst - done;
    CK(cudaMemcpyAsync(h->p_nactive, &na, sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    CK(launch_persist(h, max_iter, h->k_check, tol));
    std::vector<InstReport> rp_h(h->n_inst);
    std::vector<int32_t> act(h->n_inst);
    int32_t ran = 0;
    CK(cudaMemcpyAsync(rp_h.data(), h->p_rep, sizeof(InstReport) * h->n_inst, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(act.data(), h->active, sizeof(int32_t) * h->n_inst, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&ran, h->p_iters, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    int rc = check_err_word(h);
    if (rc != SOS_OK) return rc;
    h->iter_count += ran;
    for (int i = 0; i < h->n_inst; ++i) {
      if (!h->active_h[i]) continue;
      if (!act[i]) {
        h->status_h[i] = rp_h[i].status;
        h->iters_h[i] += rp_h[i].iters;
        h->active_h[i] = 0;
      } else {
        h->iters_h[i] += ran;
      }
      rp[i] = rp_h[i].rp;
      rd[i] = rp_h[i].rd;
      gp[i] = rp_h[i].gap;
      po[i] = rp_h[i].pobj;
      dobj[i] = rp_h[i].dobj;
    }
    it = max_iter;
  }
  while (it < max_iter && done < h->n_inst) {
    const int32_t k = std::min(h->k_check, max_iter - it);
    int rc = sos_iterate(h, k);
    if (rc != SOS_OK) return rc;
    it += k;
    cudaError_t e = iter64(h) ? launch_residuals<double>(h->d64, h->shape, h->stream)
                              : launch_residuals<float>(h->d32, h->shape, h->stream);
    if (e != cudaSuccess) return set_err(h, SOS_ERR_CUDA, std::string("residuals: ") + cudaGetErrorString(e));
    CK(cudaMemcpyAsync(R.data(), h->d64.resid, sizeof(InstResid) * h->n_inst, cudaMemcpyDeviceToHost, h->stream));
    rc = check_err_word(h);  // synchronises
    if (rc != SOS_OK) return rc;
    bool changed = false;
    for (int i = 0; i < h->n_inst; ++i) {
      if (!h->active_h[i]) continue;
      const InstInfo& in = h->inst[i];
      const InstResid& r = R[i];
      int st = SOS_RUNNING;
      double res = std::numeric_limits<double>::infinity();
      if (r.tau > 1e-12 * (r.kappa + 1.0)) {
        rp[i] = std::sqrt(r.pr2) / r.tau / (1.0 + in.norm_b);
        rd[i] = std::sqrt(r.dr2) / r.tau / (1.0 + in.norm_c);
        po[i] = r.cx / r.tau;
        dobj[i] = r.by / r.tau;
        gp[i] = std::fabs(po[i] - dobj[i]) / (1.0 + std::fabs(po[i]) + std::fabs(dobj[i]));
        res = std::max(rp[i], std::max(rd[i], gp[i]));
      }
      const double pinf = r.by > 0 ? std::sqrt(r.aty2) / r.by : std::numeric_limits<double>::infinity();
      const double dinf = r.cx < 0 ? std::sqrt(r.ax2) / (-r.cx) : std::numeric_limits<double>::infinity();
      if (r.nonfinite > 0 || !std::isfinite(r.tau) || !std::isfinite(r.kappa))
        st = SOS_NUMERICAL;
      else if (res <= tol)
        st = SOS_SOLVED;
      else if (r.kappa > r.tau && pinf <= h->infeas_tol)  // an embedding solution with kappa > 0 is a certificate
        st = SOS_PRIMAL_INFEASIBLE;
      else if (r.kappa > r.tau && dinf <= h->infeas_tol)
        st = SOS_DUAL_INFEASIBLE;
      if (st != SOS_RUNNING) {
        h->status_h[i] = st;
        h->active_h[i] = 0;
        ++done;
        changed = true;
      }
    }
    if (changed)
      CK(cudaMemcpyAsync(h->active, h->active_h.data(), sizeof(int32_t) * h->n_inst, cudaMemcpyHostToDevice, h->stream));
  }
  if (!results) return SOS_OK;
  std::vector<double> ux, vx, uy, vy, tau, kappa;
  TRY(get_all(h, ux, vx, uy, vy, tau, kappa));
  for (int i = 0; i < h->n_inst; ++i) {
    sos_result& out = results[i];
    const InstInfo& in = h->inst[i];
    out.status = h->status_h[i] == SOS_RUNNING ? SOS_MAX_ITER : h->status_h[i];
    out.iters = h->iters_h[i];
    out.res_primal = rp[i];
    out.res_dual = rd[i];
    out.gap = gp[i];
    out.obj_primal = po[i];
    out.obj_dual = dobj[i];
    out.tau = tau[i];
    out.kappa = kappa[i];
    const double it = tau[i] > 0 ? 1.0 / tau[i] : 0.0;
    if (out.x)
      for (int k = 0; k < in.nx; ++k) out.x[k] = ux[in.x_off + k] * it;
    if (out.s)
      for (int k = 0; k < in.nx; ++k) out.s[k] = vx[in.x_off + k] * it;
    if (out.y)
      for (int k = 0; k < in.m; ++k) out.y[k] = uy[in.y_off + k] * it;
  }
  return SOS_OK;
}

static int ensure_cat_map(sos_handle* h) {
  if (h->cat_map) return SOS_OK;
  std::vector<int32_t> inv(h->M);
  for (int64_t q = 0; q < h->M; ++q) inv[h->row_perm[q]] = static_cast<int32_t>(q);
  std::vector<int64_t> map;
  for (int i = 0; i < h->n_inst; ++i) {
    const InstInfo& in = h->inst[i];
    for (int k = 0; k < in.nx; ++k) map.push_back(in.x_off + k);
    for (int k = 0; k < in.m; ++k) map.push_back(h->NX + inv[in.y_off + k]);
    map.push_back(h->NX + h->M + i);
  }
  h->cat_total = static_cast<int64_t>(map.size());
  return upload(h, map, &h->cat_map);
}

int sos_get_iterate_device(sos_handle* h, double* u, double* v) {
  if (!h || !u || !v) return SOS_ERR_INVALID_ARG;
  TRY(ensure_cat_map(h));
  CK(iter64(h) ? launch_gather_iterate<double>(h->d64, h->cat_map, h->cat_total, u, v, h->stream)
               : launch_gather_iterate<float>(h->d32, h->cat_map, h->cat_total, u, v, h->stream));
  return SOS_OK;
}

int sos_set_iterate_device(sos_handle* h, const double* u, const double* v) {
  if (!h || !u || !v) return SOS_ERR_INVALID_ARG;
  TRY(ensure_cat_map(h));
  CK(iter64(h) ? launch_scatter_iterate<double>(h->d64, h->cat_map, h->cat_total, u, v, h->active, h->stream)
               : launch_scatter_iterate<float>(h->d32, h->cat_map, h->cat_total, u, v, h->active, h->stream));
  TRY(init_wl(h));
  std::fill(h->active_h.begin(), h->active_h.end(), 1);
  std::fill(h->iters_h.begin(), h->iters_h.end(), 0);
  std::fill(h->status_h.begin(), h->status_h.end(), SOS_RUNNING);
  return SOS_OK;
}

// Host iterate exchange: one contiguous copy each way through a device
// staging buffer, the reordering done by the device gather / scatter kernels
// (no host-side loops; pinned caller buffers copy at full link speed).
static int ensure_cat_stage(sos_handle* h) {
  TRY(ensure_cat_map(h));
  if (!h->cat_stage) TRY(alloc(h, 2 * static_cast<size_t>(h->cat_total), &h->cat_stage));
  return SOS_OK;
}

int sos_get_iterate(sos_handle* h, double* u, double* v) {
  if (!h || !u || !v) return SOS_ERR_INVALID_ARG;
  TRY(ensure_cat_stage(h));
  double* su = h->cat_stage;
  double* sv = h->cat_stage + h->cat_total;
  const size_t bytes = sizeof(double) * static_cast<size_t>(h->cat_total);
  CK(iter64(h) ? launch_gather_iterate<double>(h->d64, h->cat_map, h->cat_total, su, sv, h->stream)
               : launch_gather_iterate<float>(h->d32, h->cat_map, h->cat_total, su, sv, h->stream));
  CK(cudaMemcpyAsync(u, su, bytes, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(v, sv, bytes, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SOS_OK;
}

int sos_set_iterate(sos_handle* h, const double* u, const double* v) {
  if (!h || !u || !v) return SOS_ERR_INVALID_ARG;
  TRY(ensure_cat_stage(h));
  double* su = h->cat_stage;
  double* sv = h->cat_stage + h->cat_total;
  const size_t bytes = sizeof(double) * static_cast<size_t>(h->cat_total);
  CK(cudaMemcpyAsync(su, u, bytes, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(sv, v, bytes, cudaMemcpyHostToDevice, h->stream));
  // the scatter also marks every instance active
  CK(iter64(h) ? launch_scatter_iterate<double>(h->d64, h->cat_map, h->cat_total, su, sv, h->active, h->stream)
               : launch_scatter_iterate<float>(h->d32, h->cat_map, h->cat_total, su, sv, h->active, h->stream));
  TRY(init_wl(h));
  std::fill(h->active_h.begin(), h->active_h.end(), 1);
  std::fill(h->iters_h.begin(), h->iters_h.end(), 0);
  std::fill(h->status_h.begin(), h->status_h.end(), SOS_RUNNING);
  CK(cudaStreamSynchronize(h->stream));
  return SOS_OK;
}

int sos_monomials(int32_t n_vars, int32_t degree, int32_t* out, int64_t capacity, int64_t* count) {
  if (n_vars < 1 || degree < 0 || !count || capacity < 0) return SOS_ERR_INVALID_ARG;
  *count = enumerate_monomials(n_vars, degree, out, capacity);
  return SOS_OK;
}

int sos_host_plan(const sos_program* prog, int32_t weighted_form, int64_t dims[6], int32_t* ent_row, double* p_diag,
                  double* b, double* zeta_h) {
  if (!prog || !dims || weighted_form < 0 || weighted_form > 2) return SOS_ERR_INVALID_ARG;
  HostPlan P;
  std::string err;
  const int rc = build_plan(prog, 1, P, err, weighted_form);
  if (rc != SOS_OK) {
    g_setup_error = err;
    return rc;
  }
  const InstInfo& in = P.inst[0];
  dims[0] = in.nx;
  dims[1] = in.m;
  dims[2] = in.t;
  dims[3] = in.t_eff;
  dims[4] = static_cast<int64_t>(P.blocks.size());
  int64_t ent = 0;
  for (auto& bk : P.blocks) ent += static_cast<int64_t>(bk.N) * (bk.N + 1) / 2;
  dims[5] = ent;
  if (ent_row)
    for (int64_t e = 0; e < in.nx; ++e) ent_row[e] = P.ent_row[e] >= 0 ? (P.ent_row[e] & ~kEntOffBit) : -1;
  if (p_diag)
    for (int64_t r = 0; r < in.m; ++r) p_diag[r] = 1.0 / P.pinv[r];
  if (b)
    for (int64_t r = 0; r < in.m; ++r) b[r] = P.b[r];
  if (zeta_h) *zeta_h = in.zeta_h;
  return SOS_OK;
}

namespace {
// One PSD projection of a packed block: FP64 Jacobi (mixed = false) or FP32
// Jacobi with the FP64-accumulated refinement (mixed = true, small blocks).
int psd_project_one(const double* in, double* out, int32_t N, void* stream, bool mixed) {
  if (!in || !out || N < 1) return SOS_ERR_INVALID_ARG;
  if (mixed && N > psd_small_max_n(kFormMixed)) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (ns_grid(N) > sms) {
      g_setup_error = "the mixed projection of N = " + std::to_string(N) + " needs more SMs than this GPU has";
      return SOS_ERR_UNSUPPORTED;
    }
  }
  sos_handle tmp;  // owns the scratch allocations of this call
  sos_handle* h = &tmp;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t len = static_cast<int64_t>(N) * (N + 1) / 2;
  h->stream = s;
  auto release = [&]() {
    cudaStreamSynchronize(s);
    for (void* p : h->allocs) cudaFree(p);
    h->allocs.clear();
  };
  const bool small = N <= psd_small_max_n(kFormFP64);
  BlockDesc bd{};
  bd.x_off = 0;
  bd.v_off = -1;
  bd.N = N;
  bd.inst = 0;
  bd.kind = kRaw;
  bd.lr_first = -1;
  h->blocks.assign(1, bd);
  h->n_inst = 1;
  h->NX = len;
  DevPlan<double> p;
  int rc = SOS_OK;
  do {
    BlockDesc* dbd;
    if ((rc = upload(h, h->blocks, &dbd)) != SOS_OK) break;
    std::vector<int32_t> one(1, 1), zero_id(1, 0);
    int32_t *act, *ids, *sw, *err;
    if ((rc = upload(h, one, &act)) != SOS_OK) break;
    if ((rc = upload(h, zero_id, &ids)) != SOS_OK) break;
    if ((rc = alloc(h, 1, &sw)) != SOS_OK) break;
    if ((rc = alloc(h, 1, &err)) != SOS_OK) break;
    InstState* st;
    if ((rc = alloc(h, 1, &st)) != SOS_OK) break;
    double* v;
    if ((rc = alloc(h, len, &v)) != SOS_OK) break;
    p.n_inst = 1;
    p.NX = len;
    p.blocks = dbd;
    p.active = act;
    p.st = st;
    p.blk_sweeps = sw;
    p.err = err;
    p.ux = out;
    p.vx = v;
    if (cudaMemcpyAsync(out, in, sizeof(double) * len, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      rc = set_err(h, SOS_ERR_CUDA, "copy of the input failed");
      break;
    }
    cudaError_t e;
    if (mixed && N > psd_small_max_n(kFormMixed)) {  // Newton-Schulz on the tensor cores
      NsScratch S{};
      const size_t Np = static_cast<size_t>(ns_padded(N));
      if ((rc = alloc(h, Np * Np, &S.Wf)) != SOS_OK || (rc = alloc(h, Np * Np, &S.X)) != SOS_OK ||
          (rc = alloc(h, 4 * ns_split_bytes(static_cast<int>(Np)), &S.split)) != SOS_OK ||
          (rc = alloc(h, Np * Np, &S.Xn)) != SOS_OK ||
          (rc = alloc(h, 2 * static_cast<size_t>(ns_grid(N)), &S.partial)) != SOS_OK || (rc = alloc(h, 2, &S.bar)) != SOS_OK ||
          (rc = alloc(h, 1, &S.iters_out)) != SOS_OK)
        break;
      e = launch_psd_ns<double>(p, 0, N, S, s);
    } else if (mixed) {
      const int cap = N <= 16 ? 16 : N <= 32 ? 32 : N <= 48 ? 48 : N <= 64 ? 64 : N <= 96 ? 96 : 112;
      e = prepare_kernels<double, float>(cap, 0);
      if (e == cudaSuccess) e = launch_psd_small<double, float>(p, ids, 1, cap, SmallWarm<float>(), s);
    } else if (small) {
      const int cap = N <= 16 ? 16 : N <= 32 ? 32 : N <= 48 ? 48 : N <= 64 ? 64 : 96;
      e = prepare_kernels<double, double>(cap, 0);
      if (e == cudaSuccess) e = launch_psd_small<double, double>(p, ids, 1, cap, SmallWarm<double>(), s);
    } else {
      std::vector<LargeBlock<double>> lb;
      if ((rc = make_large(h, lb, std::vector<int>(1, 0))) != SOS_OK) break;
      e = launch_psd_large<double, double>(p, 0, N, lb[0].scratch, lb[0].grid, s);
    }
    if (e != cudaSuccess) {
      rc = set_err(h, SOS_ERR_CUDA, std::string("projection launch: ") + cudaGetErrorString(e));
      break;
    }
    int32_t ew = 0;
    if (cudaMemcpyAsync(&ew, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = set_err(h, SOS_ERR_CUDA, "projection failed");
      break;
    }
    if (ew != 0) rc = set_err(h, SOS_ERR_TIMEOUT, "a bounded device-side wait expired");
  } while (false);
  if (rc != SOS_OK) g_setup_error = h->err;
  release();
  return rc;
}
}  // namespace

int sos_psd_project(const double* in, double* out, int32_t N, void* stream) {
  return psd_project_one(in, out, N, stream, false);
}

int sos_psd_project_mixed(const double* in, double* out, int32_t N, void* stream) {
  return psd_project_one(in, out, N, stream, true);
}

int sos_stats(sos_handle* h, int64_t out[4]) {
  if (!h || !out) return SOS_ERR_INVALID_ARG;
  std::vector<int32_t> sw(h->blocks.size());
  if (!sw.empty())
    CK(cudaMemcpyAsync(sw.data(), h->blk_sweeps, sizeof(int32_t) * sw.size(), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  out[0] = h->iter_count;
  out[1] = static_cast<int64_t>(sw.size());
  out[2] = 0;
  out[3] = 0;
  for (int32_t s : sw) {
    out[2] = std::max<int64_t>(out[2], s);
    out[3] += s;
  }
  return SOS_OK;
}

int sos_tuning(const sos_handle* h, int32_t out[5]) {
  if (!h || !out) return SOS_ERR_INVALID_ARG;
  out[0] = h->persistent ? 1 : 0;
  out[1] = h->p_grid;
  out[2] = h->p_dynamic;
  out[3] = h->p_tried;
  out[4] = static_cast<int32_t>(h->p_best_ms * 1000.f);
  if (!h->persistent && h->large_grid_best > 0) out[1] = h->large_grid_best;
  return SOS_OK;
}

int sos_set_wait_limit(sos_handle* h, int32_t us) {
  if (!h || us < 0) return SOS_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(h->stream));
  h->wait_limit_us = us;
  h->d64.wait_limit = h->d32.wait_limit = wait_cycles(us);
  if (h->graph) {  // the captured launches hold the old bound
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  h->graph_tried = false;
  return SOS_OK;
}

int sos_launches_per_iteration(const sos_handle* h) {
  if (!h) return SOS_ERR_INVALID_ARG;
  if (h->persistent) return 0;  // one launch for all iterations of a call
  const int teff = h->precision == SOS_PREC_FP32 ? h->d32.max_teff : h->d64.max_teff;
  int affine = h->TL > 0 ? 6 : 4;
  if (h->TL > 0 && woodbury_wide(h->n_inst, teff)) affine += 1;
  int large = 0;
  for (const auto& lb : h->large64) large += tri_path(lb.N) ? (lb.scratch.tri_warm ? 6 : 5) : 1;  // warm attempt, gather, reduce, vectors, recon, Jacobi
  return affine + static_cast<int>(h->small.size()) + large +
         static_cast<int>(h->large32.size() + h->ns_large.size());
}

void* sos_stream(sos_handle* h) { return h ? static_cast<void*>(h->stream) : nullptr; }

int sos_stage_bytes(const sos_handle* h, int32_t stage, int64_t* bytes) {
  if (!h || !bytes || stage < 0 || stage > 15) return SOS_ERR_INVALID_ARG;
  *bytes = h->stage_bytes[stage];
  return SOS_OK;
}

int sos_run_stage(sos_handle* h, int32_t stage) {
  if (!h || stage < 0 || stage > 15) return SOS_ERR_INVALID_ARG;
  cudaError_t e = enqueue_any(h, stage);
  if (e != cudaSuccess) return set_err(h, SOS_ERR_CUDA, std::string("stage launch: ") + cudaGetErrorString(e));
  return SOS_OK;
}

}  // extern "C"
