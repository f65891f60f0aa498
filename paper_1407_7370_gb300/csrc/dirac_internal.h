// dirac_internal.h -- what the library's translation units share (not part of
// the public ABI): error reporting and a read-only view of a single-problem
// context.
#pragma once

#include "dirac.h"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>

namespace dirac {

// NVTX range around a public call, so that timeline tools show the library's
// calls; without a tool attached the push and pop do nothing.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// Records a printf-style message for dirac_last_error() and returns `s`.
dirac_status fail(dirac_status s, const char* fmt, ...);

// The operator and fields of a context as set by dirac_create / dirac_set_fields.
struct CtxView {
  int nx, ny;
  double dx, dy, mass, c;
  int order, boundary;
  const double* V;        // FP64 potential energy on the grid (device), or null for V = 0
  double vmin, vmax;      // range of V (0, 0 when V = 0)
  double ax, ay;          // uniform vector potential (static fields)
  double shift;           // energy shift s: the operator is H - s
  bool fields_set;
  cudaStream_t stream;
  long long* launches;    // the context's kernel-launch counter
  bool profiling;         // dirac_profile_enable is on: time kernels with CUDA events
  int precision;          // DIRAC_FP64 or DIRAC_MIXED
  int m_max;
  const void* dev_state;  // the problem's DevState (device): T, norms, k of the last step
  void* basis;            // its Krylov basis q^_2 .. q^_{m_max} (device), consecutive fields
};

dirac_status ctx_view(dirac_ctx* ctx, CtxView* v);

struct ChebParams;
struct LaunchParams;
struct CoopArgs;

// Resident CTAs per SM of `kernel` (threads, dynamic shared memory smem) on
// the current device.  Computed once per device -- after raising the
// kernel's dynamic shared memory limit there -- and kept in cache[device],
// an array of OCC_MAX_DEVICES zero-initialised entries that the caller
// declares once per kernel.  Threads may race on the first call: each
// computes the same value.
constexpr int OCC_MAX_DEVICES = 64;
template <class Kernel>
cudaError_t occupancy_on_device(std::atomic<int>* cache, Kernel kernel, int threads, size_t smem, int* occ) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= OCC_MAX_DEVICES) return cudaErrorInvalidDevice;
  int v = cache[dev].load(std::memory_order_acquire);
  if (v == 0) {
    if (smem > 0) {
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    if (v > 0) cache[dev].store(v, std::memory_order_release);
  }
  *occ = v;
  return cudaSuccess;
}

// FP32 passes stage their tiles by asynchronous copies from this many tiles
// per CTA on (below that the extra barrier costs more than it hides)
constexpr int ASYNC_MIN_TILES = 4;

// Tile height of the mixed-precision one-launch step (tiles of 32 x 16 sites).
constexpr int M32_TILE_H = 16;

// One mixed-precision time step of every problem in `p` as one cooperative
// launch (lanczos_step_m32): one CTA per SM, bulk-copy staging, compensated
// FP32 stencil.  The tile list must use M32_TILE_H; ca.slots holds 2 x 3 x
// ca.cap doubles (one problem) and ca.bar GRID_SYNC_WORDS zeroed words;
// ca.bar_count on entry: extra arrivals the barriers wait for (0; 1 only in
// the test of the barrier timeout).
cudaError_t launch_step_m32(int order, bool diri, const LaunchParams& p, int n_sm, const CoopArgs& ca,
                            cudaStream_t s);

// One time step of the single problem in `p` as one cooperative launch
// (lanczos_step); sets the grid, the chunks and ca.G.  ca.bar_count on entry:
// arrivals the barriers wait for beyond the launch's CTAs (0; 1 only in the
// test of the barrier timeout).
cudaError_t launch_step(int precision, int th, int order, bool diri, bool hasv, const LaunchParams& p, int n_sm,
                        const CoopArgs& ca, cudaStream_t s);

// [c0 - half, c0 + half] contains the spectrum of H - s for any vector
// potential with |A_x| <= ax_max, |A_y| <= ay_max
dirac_status operator_interval(dirac_ctx* ctx, double ax_max, double ay_max, double* c0, double* half);

// Chebyshev coefficients of exp(-i (H - s) dt) e_1 on that interval (dt > 0)
dirac_status cheb_params(double c0, double half, double dt, double shift, ChebParams* cp);

}  // namespace dirac
