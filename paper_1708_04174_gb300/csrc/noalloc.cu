// sos_psd_project_noalloc: the PSD projection of sos_psd_project for callers
// that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or unsafe --
// under a memory pool or allocator that owns all device memory, in a
// real-time loop that may not block on the allocator, or in a plugin whose
// host forbids allocations after start-up.  Such callers pass only their
// input and output buffers; every piece of scratch comes from the fixed
// array below, which is part of the library image and is resident on every
// GPU that loads the library, for as long as the process lives.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "../../include/sos.h"
#include "kernels.h"
#include "setup.h"

namespace sos {
namespace {

constexpr int kNoAllocMaxN = SOS_NOALLOC_MAX_N;
constexpr int kMaxDevices = 64;
constexpr int kMaxGrid = 2048;  // CTAs of the grid path (one per SM)

// Byte layout of the scratch array (all offsets 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }
constexpr size_t kNp = kNoAllocMaxN + (kNoAllocMaxN & 1);
constexpr size_t kMat = align256(sizeof(double) * kNp * kNp);
constexpr size_t kPacked = align256(sizeof(double) * kNoAllocMaxN * (kNoAllocMaxN + 1) / 2);
constexpr size_t kOffV = 0;                       // v = u - W output (packed)
constexpr size_t kOffMats = kOffV + kPacked;      // Wf, B0, B1, V, T1
constexpr size_t kOffPartial = kOffMats + 5 * kMat;
constexpr size_t kOffSmall = kOffPartial + align256(sizeof(double) * large_partials_size(kMaxGrid, kNoAllocMaxN));
// small words: block descriptor, instance state, ids/flags
constexpr size_t kOffDesc = kOffSmall;
constexpr size_t kOffState = kOffDesc + align256(sizeof(BlockDesc));
constexpr size_t kOffWords = kOffState + align256(sizeof(InstState));
constexpr int kWordActive = 0, kWordId = 1, kWordSweeps = 2, kWordErr = 3, kWordBar = 4, kWordSweepsOut = 6,
              kWordWarm = 7, kWordFlags = 8;
constexpr size_t kWordsBytes = align256(sizeof(int32_t) * (kWordFlags + kMaxSweeps));
constexpr size_t kScratchBytes = kOffWords + kWordsBytes;

// The scratch itself.  Every call of the entry point uses all of it, and it
// keeps the previous call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_ptr[kMaxDevices] = {};  // device address of the scratch, per device

int fail(int code, const std::string& msg) {
  set_global_error(msg);
  return code;
}

}  // namespace
}  // namespace sos

using namespace sos;

extern "C" int sos_psd_project_noalloc(const double* in, double* out, int32_t N, void* stream) {
  if (!in || !out) return fail(SOS_ERR_INVALID_ARG, "sos_psd_project_noalloc: NULL buffer");
  if (N < 1 || N > kNoAllocMaxN)
    return fail(SOS_ERR_INVALID_ARG, "sos_psd_project_noalloc: N = " + std::to_string(N) + " is outside 1.." +
                                         std::to_string(kNoAllocMaxN) + " (fixed scratch size)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(SOS_ERR_CUDA, "sos_psd_project_noalloc: no current CUDA device");
  unsigned char* base = nullptr;
  {
    // One-time set-up per device, with that device current: look up the
    // device address of the scratch array (the host-side symbol is only a
    // stand-in and must never be passed to a kernel).
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return fail(SOS_ERR_CUDA, std::string("sos_psd_project_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_ptr[dev] = static_cast<unsigned char*>(p);
    }
    base = g_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t len = static_cast<int64_t>(N) * (N + 1) / 2;
  int32_t* words = reinterpret_cast<int32_t*>(base + kOffWords);

  // descriptors of the single block, and the words that must start at zero
  BlockDesc bd{};
  bd.x_off = 0;
  bd.v_off = -1;
  bd.N = N;
  bd.inst = 0;
  bd.kind = kRaw;
  bd.lr_first = -1;
  int32_t w0[kWordFlags] = {};
  w0[kWordActive] = 1;
  w0[kWordId] = 0;
  if (cudaMemcpyAsync(base + kOffDesc, &bd, sizeof(bd), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(base + kOffState, 0, sizeof(InstState), s) != cudaSuccess ||
      cudaMemcpyAsync(words, w0, sizeof(w0), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(out, in, sizeof(double) * len, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return fail(SOS_ERR_CUDA, "sos_psd_project_noalloc: staging copies failed");

  DevPlan<double> p;
  p.n_inst = 1;
  p.NX = len;
  p.blocks = reinterpret_cast<const BlockDesc*>(base + kOffDesc);
  p.st = reinterpret_cast<InstState*>(base + kOffState);
  p.active = words + kWordActive;
  p.blk_sweeps = words + kWordSweeps;
  p.err = words + kWordErr;
  p.ux = out;
  p.vx = reinterpret_cast<double*>(base + kOffV);

  cudaError_t e;
  if (N <= psd_small_max_n(kFormFP64)) {
    const int cap = N <= 16 ? 16 : N <= 32 ? 32 : N <= 48 ? 48 : N <= 64 ? 64 : 96;
    e = prepare_kernels<double, double>(cap, 0);
    if (e == cudaSuccess) e = launch_psd_small<double, double>(p, words + kWordId, 1, cap, SmallWarm<double>(), s);
  } else {
    const int grid = large_grid_size(N);
    if (grid > kMaxGrid) return fail(SOS_ERR_UNSUPPORTED, "sos_psd_project_noalloc: too many SMs for the scratch");
    const size_t Np = N + (N & 1);
    LargeScratch<double> ls;
    double* mats = reinterpret_cast<double*>(base + kOffMats);
    const size_t stride = kMat / sizeof(double);
    (void)Np;
    ls.Wf = mats;
    ls.B0 = mats + stride;
    ls.B1 = mats + 2 * stride;
    ls.V = mats + 3 * stride;
    ls.T1 = mats + 4 * stride;
    ls.partial = reinterpret_cast<double*>(base + kOffPartial);
    ls.bar = reinterpret_cast<uint32_t*>(words + kWordBar);  // zeroed by the launch
    ls.sweeps_out = words + kWordSweepsOut;
    ls.warm = words + kWordWarm;  // zeroed above: always a cold start
    ls.flags = words + kWordFlags;
    e = launch_psd_large<double, double>(p, 0, N, ls, grid, s);
  }
  if (e != cudaSuccess)
    return fail(SOS_ERR_CUDA, std::string("sos_psd_project_noalloc: launch: ") + cudaGetErrorString(e));
  int32_t ew = 0;
  if (cudaMemcpyAsync(&ew, words + kWordErr, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(SOS_ERR_CUDA, "sos_psd_project_noalloc: projection failed");
  if (ew != 0) return fail(SOS_ERR_TIMEOUT, "sos_psd_project_noalloc: a bounded device-side wait expired");
  return SOS_OK;
}
