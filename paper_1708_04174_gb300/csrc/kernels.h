// Device kernels of libsos and their launch wrappers (host-callable).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "sos_plan.h"

namespace sos {

// Device pointers of one problem set; T is the iterate type (double for the
// plain FP64 form, float for the FP32 form).  Woodbury data, tau/kappa and
// every reduction stay in FP64.
template <typename T>
struct DevPlan {
  int32_t n_inst = 0;
  int64_t NX = 0, M = 0;
  int32_t TL = 0;
  int32_t max_teff = 0;
  const InstInfo* inst = nullptr;
  InstState* st = nullptr;
  const int32_t* active = nullptr;  // 1 while the instance iterates
  InstResid* resid = nullptr;
  const BlockDesc* blocks = nullptr;
  const double* b = nullptr;
  const double* pinv = nullptr;
  const double* h2 = nullptr;
  const int32_t* row_inst = nullptr;
  const int32_t* row_ptr = nullptr;
  const uint32_t* row_ent = nullptr;
  const int32_t* ent_row = nullptr;   // plain: row | kEntOffBit if off-diagonal; low-rank: -(column + 1)
  const int32_t* lr_ptr = nullptr;
  const int32_t* lr_row = nullptr;
  const double* lr_val = nullptr;
  const int32_t* lrr_ptr = nullptr;
  const int32_t* lrr_col = nullptr;
  const double* lrr_val = nullptr;
  const int64_t* lr_ent = nullptr;
  const int32_t* lr_inst = nullptr;
  const double* lr_c = nullptr;
  const double* lr_g = nullptr;
  const double* linv = nullptr;
  const double* linv_t = nullptr;  // L^-1 of each instance, column-major (first triangular pass)
  // sliced copies of the row lists: rows are numbered in order of decreasing
  // length within each instance, 32 consecutive rows per slice, element k of
  // row a at off[a / 32] + 32 k + a % 32, so a warp's loads coalesce and its
  // lanes run similar lengths
  const int32_t* col_perm = nullptr;  // A_L columns by decreasing length within each instance
  const int64_t* ent_sl_off = nullptr;  // plain Gram entries (as row_ent)
  const uint32_t* ent_sl = nullptr;
  const int64_t* lr_sl_off = nullptr;   // A_L rows (as lrr_col / lrr_val)
  const int32_t* lr_sl_col = nullptr;
  const double* lr_sl_val = nullptr;
  double* wl = nullptr;  // w1_hat on the low-rank columns: u + v - c (tau + kappa) (TL)
  // iterates
  T* ux = nullptr;
  T* vx = nullptr;
  T* uy = nullptr;
  T* vy = nullptr;
  double* tau = nullptr;
  double* kappa = nullptr;
  // per-iteration work
  double* xP = nullptr;    // P^{-1} r (M)
  double* ylr = nullptr;   // A_L^T P^{-1} r (TL)
  double* zlr = nullptr;   // core^{-1} ylr (TL)
  double* wq = nullptr;    // L^{-1} ylr of a single wide instance (TL)
  double* sig2 = nullptr;  // sigma_2 (M)
  T* uh2 = nullptr;        // u_hat_2 (M)
  double* ra = nullptr;    // residual work (M)
  double* atyl = nullptr;  // residual work (TL)
  int32_t* err = nullptr;  // device error word (nonzero: a bounded wait expired)
  int32_t* blk_sweeps = nullptr;  // Jacobi sweeps of each block in the last iteration
  long long wait_limit = 4000000000ll;  // bound of each grid-wide wait, clock cycles (~2 s)
};

// Scratch of the large-block (cooperative) projection, one per large block.
template <typename T>
struct LargeScratch {
  T* Wf = nullptr;   // Np x Np symmetric input
  T* B0 = nullptr;   // Jacobi working matrix (double buffered)
  T* B1 = nullptr;
  T* V = nullptr;    // eigenvectors, kept across iterations (warm start)
  T* T1 = nullptr;   // GEMM temporary
  double* partial = nullptr;   // large_partials_size(grid, N) doubles
  // [0]: 1 if the tridiagonal path projected the block in this iteration;
  // with tri_warm, [1]: iterations before the next warm attempt, [3]: 1 if V
  // holds the last iteration's eigenvectors, [4]: 1 once a cold projection
  // has set the first wait
  int32_t* flags = nullptr;
  uint32_t* bar = nullptr;     // grid barrier: [arrivals, released generation], zeroed before each launch
  int32_t* sweeps_out = nullptr;  // number of sweeps of the last launch
  int32_t* warm = nullptr;     // 1 if V holds the previous eigenvectors
  int32_t warm_limit = 1024;   // cold restart after this many warm iterations
  int32_t tri_warm = 0;        // 1: each iteration first tries the refinement from the last eigenvectors
  float* F32 = nullptr;        // five N x Np FP32 work matrices of the refinement's Rayleigh-quotient update, or none
};

constexpr int kMaxSweeps = 40;
// LargeScratch::partial: kLargePartials doubles per CTA (the Jacobi kernel
// uses three: norm and two alternating sweep checks; the tridiagonal path's
// refinement four for its check and two sets for grid maxima), then 6 N + 1
// doubles of the refinement (diagonal of B, pair-rotation proposals and
// rotations)
constexpr int kLargePartials = 6;
__host__ __device__ constexpr size_t large_partials_size(int grid, int N) {
  return static_cast<size_t>(kLargePartials) * static_cast<size_t>(grid) + 6 * static_cast<size_t>(N) + 1;
}

// FP64 large blocks of kTriMinN <= N <= kTriMaxN are projected through a
// tridiagonal reduction (csrc/eigproj.cu); the grid Jacobi kernel launched
// after it does nothing unless that path left the block to it (flags[0] = 0).
constexpr int kTriMinN = 33, kTriMaxN = 232;
__host__ __device__ constexpr bool tri_path(int N) { return N >= kTriMinN && N <= kTriMaxN; }
cudaError_t launch_psd_tri(const DevPlan<double>& p, int bid, int N, const LargeScratch<double>& L, int grid,
                           cudaStream_t s);
// one kernel of that path (profiling): 0 gather, 1 reduction, 2 eigenvectors,
// 3 FP64 refinement and reconstruction, 4 the warm attempt (refinement from
// the last iteration's eigenvectors, launched first when tri_warm is set)
cudaError_t launch_psd_tri_part(const DevPlan<double>& p, int bid, int N, const LargeScratch<double>& L, int grid,
                                int part, cudaStream_t s);

// Scratch of the Newton-Schulz projection (tensor cores) of one large block.
struct NsScratch {
  float* Wf = nullptr;  // W, Np x Np (Np = N rounded up to 128)
  float* X = nullptr;
  float* Xn = nullptr;
  // W, X, Xn, Y as three BF16 parts each, in the operand layout of the
  // tensor-core products (ns_split_bytes(Np) bytes per matrix)
  unsigned char* split = nullptr;
  double* partial = nullptr;  // two per CTA
  uint32_t* bar = nullptr;    // grid barrier [2], zeroed by the launcher
  int32_t* iters_out = nullptr;
  int32_t max_iter = 60;
  float tol = 2e-5f;          // stop when |X_next - X|_F <= tol sqrt(Np)
};

// Eigenvectors kept across iterations for the shared-memory projection.
template <typename TC>
struct SmallWarm {
  TC* V = nullptr;          // per block N x N (offset BlockDesc::v_off), or nullptr: always cold
  int32_t* count = nullptr; // per block: iterations since the last cold start (0 = cold)
  int32_t limit = 1024;     // cold restart after this many warm iterations
};

// Per-instance result of the device-side checks of the persistent solver.
struct InstReport {
  double rp, rd, gap, pobj, dobj;
  int32_t status;  // SOS_* status (0 while running)
  int32_t iters;   // iteration of the last check
};

template <typename TC>
struct PersistArgs {
  int32_t max_iter = 0;
  int32_t k_check = 0;        // 0: no checks (fixed number of iterations)
  double tol = 0.0;
  double infeas_tol = 1e-7;    // tolerance of the infeasibility certificates
  uint32_t* bar = nullptr;     // grid barrier [2], zeroed by the launcher
  uint32_t* queue = nullptr;   // work queue counter, zeroed by the launcher
  int32_t* active = nullptr;   // same array as DevPlan::active
  int32_t* n_active = nullptr; // running instances
  InstReport* rep = nullptr;
  const int32_t* sched = nullptr;  // Gram blocks, largest first
  int32_t n_sched = 0;
  int32_t dynamic = 0;         // 1: atomic work queue, 0: round-robin
  SmallWarm<TC> wm;
  int32_t* iters_done = nullptr;
};

struct LaunchShape {
  int sms = 152;
  int row_threads = 256;
  int inst_threads = 256;
};

template <typename T>
cudaError_t launch_affine(const DevPlan<T>& p, const LaunchShape& ls, cudaStream_t s);
// A single instance whose Woodbury core is at least 64 wide applies it with
// two launches spread over the GPU (one warp per row) instead of one CTA.
inline bool woodbury_wide(int n_inst, int max_teff) { return n_inst == 1 && max_teff >= 64; }
// w1_hat on the low-rank columns from the stored iterate (after a start or
// sos_set_iterate; during the iteration the producers of u and v write it)
template <typename T>
cudaError_t launch_init_wl(const DevPlan<T>& p, cudaStream_t s);
// one kernel of the affine step: 0 rows_r, 1 lr_y, 2 woodbury, 3 rows_sigma2,
// 4 inst_scalar, 5 rows_y (profiling)
template <typename T>
cudaError_t launch_affine_part(const DevPlan<T>& p, const LaunchShape& ls, int part, cudaStream_t s);
template <typename T, typename TC>
cudaError_t launch_psd_small(const DevPlan<T>& p, const int32_t* ids, int count, int maxN, const SmallWarm<TC>& wm,
                             cudaStream_t s);
template <typename T, typename TC>
cudaError_t launch_psd_large(const DevPlan<T>& p, int bid, int N, const LargeScratch<TC>& ls, int grid,
                             cudaStream_t s);
// one kernel of the large-block projection (profiling): parts 0..3 the
// tridiagonal path (FP64 form, kTriMinN <= N <= kTriMaxN), part 4 the grid
// Jacobi kernel (which does nothing after a successful tridiagonal path),
// part 5 the warm attempt of the tridiagonal path (launched first)
template <typename T, typename TC>
cudaError_t launch_psd_large_part(const DevPlan<T>& p, int bid, int N, const LargeScratch<TC>& ls, int grid,
                                  int part, cudaStream_t s);
int large_grid_size(int N);
template <typename T, typename TC>
cudaError_t prepare_kernels(int max_small_n, int max_teff);
template <typename T>
cudaError_t launch_residuals(const DevPlan<T>& p, const LaunchShape& ls, cudaStream_t s);
template <typename T>
cudaError_t launch_psd_ns(const DevPlan<T>& p, int bid, int N, const NsScratch& S, cudaStream_t s);
int ns_grid(int N);
int ns_padded(int N);
// bytes of one matrix in the split operand layout (three BF16 parts)
__host__ __device__ inline size_t ns_split_bytes(int Np) { return static_cast<size_t>(6) * Np * Np; }
template <typename T, typename TC>
int persistent_max_ctas_per_sm(int max_small_n, int max_teff);
template <typename T, typename TC>
cudaError_t launch_persistent(const DevPlan<T>& p, const PersistArgs<TC>& a, int grid, int max_small_n, int max_teff,
                              cudaStream_t s);
// projection forms of the small-block kernel: FP64; FP32 Jacobi with an FP64
// refinement (FP64 iterates); plain FP32 (FP32 iterates)
constexpr int kFormFP64 = 0, kFormMixed = 1, kFormFP32 = 2;
template <typename T, typename TC>
constexpr int form_of() {
  return sizeof(TC) == 8 ? kFormFP64 : (sizeof(T) == 8 ? kFormMixed : kFormFP32);
}
// Iterate exchange with caller DEVICE buffers in the concatenated layout
// (per instance [xi (n_x), y (m), tau] for u, [z, s, kappa] for v): map[q]
// is the source of position q, an index into x (< NX), into the device rows
// (NX .. NX + M) or an instance (NX + M + i) for tau / kappa.  The scatter
// also marks every instance running.
template <typename T>
cudaError_t launch_gather_iterate(const DevPlan<T>& p, const int64_t* map, int64_t total, double* u, double* v,
                                  cudaStream_t s);
template <typename T>
cudaError_t launch_scatter_iterate(const DevPlan<T>& p, const int64_t* map, int64_t total, const double* u,
                                   const double* v, int32_t* active, cudaStream_t s);
size_t psd_small_smem_bytes(int maxN, int form);
size_t large_smem_bytes(int N, size_t es);
int psd_small_max_n(int form);

}  // namespace sos
