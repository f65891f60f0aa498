// dirac_step.cu -- launcher of the FP64 one-launch time step (`lanczos_step`):
// all Lanczos passes of a step of one problem and its recombination in one
// cooperative launch, the passes separated by grid-wide barriers.  Kept in a
// translation unit of its own so that it compiles in parallel with the
// per-pass kernels.
#include "dirac.h"
#include "dirac_internal.h"
#include "dirac_kernels.cuh"

#include <cuda_runtime.h>

#include <algorithm>

namespace dirac {

namespace {

template <class S, int R, int TH, bool D, bool V, bool AY>
cudaError_t launch_step_t(LaunchParams p, int n_sm, CoopArgs ca, cudaStream_t s) {
  static std::atomic<int> occ_dev[OCC_MAX_DEVICES];
  constexpr int SUB = step_workers<S, TH>();
  constexpr int NT = SUB * 32 * (TH / rows_per_thread<S, TH>());
  constexpr size_t smem = dyn_smem_bytes<S, R, TH, SUB>();
  int occ = 0;
  cudaError_t e = occupancy_on_device(occ_dev, lanczos_step<S, R, TH, D, V, AY>, NT, smem, &occ);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorCooperativeLaunchTooLarge;
  // every CTA resident (a cooperative launch checks it) and each with at
  // least one tile, so that every CTA writes its partial in every pass
  const int grid = std::max(1, std::min(std::min(p.total_tiles, n_sm * occ), ca.cap));
  p.chunk_q = p.total_tiles / grid;
  p.chunk_r = p.total_tiles % grid;
  p.async_tiles = p.chunk_q >= ASYNC_MIN_TILES;
  ca.bar_count = grid + ca.bar_count;   // ca.bar_count comes in as the extra arrivals to wait for
  ca.G = grid;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, lanczos_step<S, R, TH, D, V, AY>, p, ca);
}

template <class S, int R, int TH, bool D, bool V>
cudaError_t launch_step_ay(const LaunchParams& p, int n_sm, const CoopArgs& ca, cudaStream_t s) {
  if constexpr (sizeof(S) == sizeof(double)) {
    if (!p.has_ay) return launch_step_t<S, R, TH, D, V, false>(p, n_sm, ca, s);
  }
  return launch_step_t<S, R, TH, D, V, true>(p, n_sm, ca, s);
}

template <class S, int TH>
cudaError_t launch_step_s(int order, bool diri, bool hasv, const LaunchParams& p, int n_sm, const CoopArgs& ca,
                          cudaStream_t s) {
  if (order == 2) {
    if (diri) return hasv ? launch_step_ay<S, 1, TH, true, true>(p, n_sm, ca, s)
                          : launch_step_ay<S, 1, TH, true, false>(p, n_sm, ca, s);
    return hasv ? launch_step_ay<S, 1, TH, false, true>(p, n_sm, ca, s)
                : launch_step_ay<S, 1, TH, false, false>(p, n_sm, ca, s);
  }
  if (diri) return hasv ? launch_step_ay<S, 2, TH, true, true>(p, n_sm, ca, s)
                        : launch_step_ay<S, 2, TH, true, false>(p, n_sm, ca, s);
  return hasv ? launch_step_ay<S, 2, TH, false, true>(p, n_sm, ca, s)
              : launch_step_ay<S, 2, TH, false, false>(p, n_sm, ca, s);
}

}  // namespace

cudaError_t launch_step(int precision, int th, int order, bool diri, bool hasv, const LaunchParams& p, int n_sm,
                        const CoopArgs& ca, cudaStream_t s) {
  // the mixed path has its own one-launch step (dirac_step32.cu)
  if (precision != DIRAC_FP64) return cudaErrorInvalidValue;
  if (th == 16) return launch_step_s<double, 16>(order, diri, hasv, p, n_sm, ca, s);
  return launch_step_s<double, 32>(order, diri, hasv, p, n_sm, ca, s);
}

}  // namespace dirac
