// dirac_capi.cu -- host side of the GB300 Dirac Lanczos propagator: problem
// tables, workspace, launch sequencing and the C ABI of include/dirac.h.
#include "dirac.h"
#include "dirac_internal.h"
#include "dirac_kernels.cuh"

#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

using namespace dirac;

namespace dirac {

thread_local char g_err[512] = "";

dirac_status fail(dirac_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

}  // namespace dirac

namespace {

#define CUDA_TRY(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return fail(DIRAC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
bool aligned32(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 31u) == 0; }
size_t site_bytes(int precision) { return precision == DIRAC_FP64 ? sizeof(double4_32a) : sizeof(float4); }

// ---------------------------------------------------------------------------
// small exponential: Jacobi-Anger coefficients on an a-priori interval
// ---------------------------------------------------------------------------

// Bessel functions J_0..J_{n-1}(x), x > 0, by Miller's backward recurrence
// J_{k-1} = (2k/x) J_k - J_{k+1} started far above n and normalised with
// J_0 + 2 sum_{k>=1} J_{2k} = 1.  Stack storage only.
bool bessel_j(int n, double x, double* out) {
  constexpr int NJ = 512;
  double j[NJ + 2];
  const int start = 2 * ((std::max(n, (int)x) + 40 + (int)std::sqrt(40.0 * std::max(x, 1.0))) / 2);
  if (start > NJ) return false;
  for (int k = 0; k <= start + 1; ++k) j[k] = 0.0;
  j[start] = 1e-300;
  for (int k = start; k >= 1; --k) {
    j[k - 1] = (2.0 * k / x) * j[k] - j[k + 1];
    if (std::fabs(j[k - 1]) > 1e250)      // rescale to stay in range
      for (int t = k - 1; t <= start; ++t) j[t] *= 1e-250;
  }
  double norm = j[0];
  for (int k = 2; k <= start; k += 2) norm += 2.0 * j[k];
  for (int k = 0; k < n; ++k) out[k] = j[k] / norm;
  return true;
}

// Rigorous interval [c0 - half, c0 + half] containing the spectrum of H - s:
// H = H0(A) + V with spec(H0(A)) = {+-E_k}, E_k <= sqrt(m^2c^4 + c^2 (P_x+|A_x|)^2
// + c^2 (P_y+|A_y|)^2), P = max |stencil momentum| (1/h for order 2, for order
// 4 the maximum of (8 sin t - sin 2t)/(6h)), and V_min <= V <= V_max.
void spectral_interval(int order, double dx, double dy, double mass, double c, double ax_max,
                       double ay_max, double vmin, double vmax, double shift, double& c0,
                       double& half) {
  double pf = 1.0;
  if (order == 4) {
    const double cs = 1.0 - std::sqrt(6.0) / 2.0;    // cos t at the maximum
    pf = std::sqrt(1.0 - cs * cs) * (4.0 - cs) / 3.0;
  }
  const double px = pf / dx + ax_max, py = pf / dy + ay_max;
  const double mc2 = mass * c * c;
  const double emax = std::sqrt(mc2 * mc2 + c * c * (px * px + py * py));
  c0 = 0.5 * (vmin + vmax) - shift;
  half = (emax + 0.5 * (vmax - vmin)) * (1.0 + 1e-8) + 1e-12;
}

dirac_status make_cheb(double c0, double half, double dt, double shift, ChebParams& cp) {
  const double R = half * dt;
  if (!(R > 0.0) || R > 90.0)
    return fail(DIRAC_EINVAL, "dt * ||H|| = %.3g outside (0, 90]: take smaller steps", R);
  double J[CHEB_MAX];
  if (!bessel_j(CHEB_MAX, R, J)) return fail(DIRAC_EINVAL, "dt too large");
  int n = 2;
  for (int k = 0; k < CHEB_MAX; ++k)
    if (std::fabs(J[k]) > 1e-18 || k <= (int)R + 1) n = k + 1;
  if (n >= CHEB_MAX) return fail(DIRAC_EINVAL, "Chebyshev expansion needs more than %d terms", CHEB_MAX);
  cp.n = std::max(n, 2);
  cp.c0 = c0;
  cp.inv_half = 1.0 / half;
  const double ph = -(c0 + shift) * dt;
  cp.ph_re = std::cos(ph);
  cp.ph_im = std::sin(ph);
  for (int k = 0; k < CHEB_MAX; ++k) {
    const double a = (k == 0 ? 1.0 : 2.0) * (k < cp.n ? J[k] : 0.0);
    switch (k & 3) {           // (-i)^k
      case 0: cp.cr[k] = a;  cp.ci[k] = 0.0; break;
      case 1: cp.cr[k] = 0.0; cp.ci[k] = -a; break;
      case 2: cp.cr[k] = -a; cp.ci[k] = 0.0; break;
      default: cp.cr[k] = 0.0; cp.ci[k] = a; break;
    }
  }
  return DIRAC_OK;
}

// ---------------------------------------------------------------------------
// tensor maps of the mixed one-launch step
// ---------------------------------------------------------------------------

// cuTensorMapEncodeTiled through the runtime's driver entry point (the
// library does not link against the driver library itself)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::atomic<void*> fn{nullptr};
  void* f = fn.load();
  if (!f) {
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !f)
      return nullptr;
    fn.store(f);
  }
  return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
}

// Map of `fields` consecutive nx x ny spinor fields (byte stride fstride
// between fields) as a tensor of FP32 (complex64 spinors, 4 floats per site)
// or FP64 (complex128) elements, of rank 3 ({4 nx, ny, fields}) or, with
// fields = 0, rank 2, with a box of one tile and its halo, 4 (32 + 2R) x
// (th + 2R) (x 1) elements, zeros outside.  False if the driver refuses the
// shape (the kernel then copies row by row).
bool encode_field_map(CUtensorMap* map, bool fp64, const void* base, int nx, int ny, int fields, size_t fstride,
                      int R, int th) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t eb = fp64 ? 8 : 4;
  const cuuint64_t dims[3] = {4ull * (cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)(fields > 0 ? fields : 1)};
  const cuuint64_t strides[2] = {4ull * (cuuint64_t)nx * eb, (cuuint64_t)fstride};
  const cuuint32_t box[3] = {(cuuint32_t)(4 * (TILE_W + 2 * R)), (cuuint32_t)(th + 2 * R), 1u};
  const cuuint32_t es[3] = {1u, 1u, 1u};
  const CUresult r = enc(map, fp64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                         fields > 0 ? 3u : 2u, const_cast<void*>(base), dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------

// DIRAC_NO_PDL=1 in the environment turns the launch overlap off (debugging aid).
bool pdl_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("DIRAC_NO_PDL");
    return !(v && v[0] == '1');
  }();
  return on;
}

// Launch with programmatic stream serialisation: the kernel may be scheduled
// while the previous kernel in the stream finishes; it waits for it (and sees
// its writes) at its griddepcontrol.wait.
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

struct LaunchShape {
  int n_sm;          // SMs of the device
  int th;            // tile height (32 or 16; FP64 always 32)
  int cta_cap;       // 0: as many CTAs per SM as fit; else at most this many
};

// Persistent launch: as many CTAs as are resident at once (at most one per
// tile), each taking a contiguous chunk of the tile list whose size differs
// from the others' by at most one tile.
template <class S, int R, int TH, bool D, bool V, bool AY>
cudaError_t launch_pass_t(LaunchParams p, const LaunchShape& ls, cudaStream_t s) {
  static std::atomic<int> occ_dev[OCC_MAX_DEVICES];
  constexpr int NT = sub_workers<S>() * 32 * (TH / rows_per_thread<S, TH>());
  constexpr size_t smem = dyn_smem_bytes<S, R, TH, sub_workers<S>()>();
  int occ = 0;
  cudaError_t e = occupancy_on_device(occ_dev, lanczos_pass<S, R, TH, D, V, AY>, NT, smem, &occ);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  const int per_sm = ls.cta_cap > 0 ? std::min(occ, ls.cta_cap) : occ;
  const int slots = std::max(1, ls.n_sm * per_sm);
  const int grid = std::max(1, std::min(p.total_tiles, slots));
  p.chunk_q = p.total_tiles / grid;
  p.chunk_r = p.total_tiles % grid;
  p.async_tiles = p.chunk_q >= ASYNC_MIN_TILES;
  return launch_pdl(lanczos_pass<S, R, TH, D, V, AY>, grid, NT, smem, s, p);
}

// FP64: a kernel without the c A_y terms (four FMAs per site of ~54) when no
// step of the launch has A_y != 0 (linear polarisation along x, static
// fields); the FP32 pass, bound by memory, keeps one kernel
template <class S, int R, int TH, bool D, bool V>
cudaError_t launch_pass_ay(const LaunchParams& p, const LaunchShape& ls, cudaStream_t s) {
  if constexpr (sizeof(S) == sizeof(double)) {
    if (!p.has_ay) return launch_pass_t<S, R, TH, D, V, false>(p, ls, s);
  }
  return launch_pass_t<S, R, TH, D, V, true>(p, ls, s);
}

template <class S, int TH>
cudaError_t launch_pass_s(int order, bool diri, bool hasv, const LaunchParams& p, const LaunchShape& ls,
                          cudaStream_t s) {
  if (order == 2) {
    if (diri) return hasv ? launch_pass_ay<S, 1, TH, true, true>(p, ls, s) : launch_pass_ay<S, 1, TH, true, false>(p, ls, s);
    return hasv ? launch_pass_ay<S, 1, TH, false, true>(p, ls, s) : launch_pass_ay<S, 1, TH, false, false>(p, ls, s);
  }
  if (diri) return hasv ? launch_pass_ay<S, 2, TH, true, true>(p, ls, s) : launch_pass_ay<S, 2, TH, true, false>(p, ls, s);
  return hasv ? launch_pass_ay<S, 2, TH, false, true>(p, ls, s) : launch_pass_ay<S, 2, TH, false, false>(p, ls, s);
}

// FP64 path: everything complex128.  Mixed path: complex64 basis (passes 1
// and 2 read the complex128 state as q^_1; the kernel picks per problem).
cudaError_t launch_pass(int precision, int order, bool diri, bool hasv, const LaunchParams& p,
                        const LaunchShape& ls, cudaStream_t s) {
  if (precision == DIRAC_FP64) {
    if (ls.th == 16) return launch_pass_s<double, 16>(order, diri, hasv, p, ls, s);
    return launch_pass_s<double, 32>(order, diri, hasv, p, ls, s);
  }
  if (ls.th == 16) return launch_pass_s<float, 16>(order, diri, hasv, p, ls, s);
  return launch_pass_s<float, 32>(order, diri, hasv, p, ls, s);
}

// Re-runs of a pass allowed per step (each costs one spare launch, which
// exits at once when unused) and the cancellation ratio kappa = Y / s2 that
// triggers one.  With y^ stored to unit roundoff u, s2 = ||y^||^2 - P^2/X
// keeps about u * kappa relative accuracy, and the rounding of P leaves a
// component of about u sqrt(kappa) of q^_i in q^_{i+1}.  FP64: 1e12.  FP32:
// 100, i.e. a pass whose stencil shift missed alpha_i by more than ten times
// beta_i is re-run -- in practice pass 2 of a context's first step, before
// the previous step's T can supply the shifts.
int redo_budget(int precision, int m) { return precision == DIRAC_FP64 ? 2 : 2 + m / 5; }
double kappa_redo(int precision) { return precision == DIRAC_FP64 ? 1e12 : 1e2; }

cudaError_t launch_recombine(int precision, const RecombParams& rp, int grid, cudaStream_t s) {
  if (precision == DIRAC_FP64) return launch_pdl(recombine<false>, grid, 256, 0, s, rp);
  return launch_pdl(recombine<true>, grid, 256, 0, s, rp);
}

// FP64 -> FP32 pair: hi = (float)v, lo = (float)(v - hi)
__global__ void split_float_kernel(const double* in, float* hi, float* lo, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = in[i];
    const float h = (float)v;
    hi[i] = h;
    lo[i] = (float)(v - (double)h);
  }
}

__global__ void minmax_kernel(const double* v, long long n, double* out) {
  __shared__ double smin[256], smax[256];
  double lo = 1e308, hi = -1e308;
  bool bad = false;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = v[i];
    lo = fmin(lo, x);
    hi = fmax(hi, x);
    if (!isfinite(x)) bad = true;
  }
  if (bad) { lo = -INFINITY; hi = INFINITY; }
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] = smin[0]; out[1] = smax[0]; }
}

// ---------------------------------------------------------------------------
// Engine: N independent problems sharing precision, stencil, boundary, m_max
// ---------------------------------------------------------------------------
enum { KIND_PASS = 0, KIND_RECOMBINE = 1, KIND_STEP = 2, KIND_END = -1 };

struct HostProblem {
  int nx = 0, ny = 0;
  double dx = 0, dy = 0;
  long long n = 0;
  int tiles_x = 0, ntiles = 0, tile_begin = 0;
  int rblk_begin = 0, rblk_count = 0;
  size_t slot_off = 0;             // first partial slot (3 doubles each)
  void* basis = nullptr;
  void* ybuf[2] = {nullptr, nullptr};
  void* V = nullptr;               // double (FP64) or float (mixed) copy
  float* Vlo = nullptr;            // mixed: V - (float)V
  double* V64 = nullptr;           // double copy (== V on the FP64 path)
  bool has_v = false;
  double vmin = 0, vmax = 0;
  double ax = 0, ay = 0, shift = 0;
  bool fields_set = false;
  // mixed precision: tensor maps of the complex64 fields (set at creation)
  // and of the state (re-encoded when the state's address changes)
  CUtensorMap map_basis{}, map_ybuf{};
  bool map_v_ok = false;
  CUtensorMap map_psi{};
  const void* map_psi_addr = nullptr;
  bool map_psi_ok = false;
};

struct Engine {
  int order = 2, boundary = DIRAC_PERIODIC, precision = DIRAC_FP64, m_max = 1;
  double mass = 1, c = 137.036;
  cudaStream_t stream = nullptr;
  LaunchShape shape{0, 32, 0};
  std::vector<HostProblem> P;
  int total_tiles = 0, rgrid = 0;
  void* vec_mem = nullptr;         // all basis / y^ fields
  DevState* d_st = nullptr;        // nprob states
  DevState* h_st = nullptr;        // pinned mirror for read-back
  double* d_partials = nullptr;
  // one-launch step (single problem): CTA partials by pass parity, barrier words
  double* d_coop_slots = nullptr;
  unsigned* d_coop_bar = nullptr;
  int coop_cap = 0;                // CTAs the slot buffer holds
  int step_mode = DIRAC_STEP_AUTO;
  int barrier_extra = 0;           // 1 only inside dirac_debug_barrier_timeout
  int* d_blk_prob = nullptr;
  int* d_step = nullptr;
  // per-call tables: [Problem x nprob][ChebParams x nprob][FieldStep x nfield]
  void* d_tab = nullptr;
  void* h_tab = nullptr;           // pinned staging
  size_t tab_cap = 0;
  cudaEvent_t tab_ev = nullptr;    // last upload of the staging buffer
  bool tab_ev_live = false;
  bool need_probe = true;
  long long launches = 0;
  vec4* psi_own = nullptr;         // staging for the host-buffer call
  // CUDA graph of one step (captured on a private stream, replayed on `stream`)
  bool use_graphs = true;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t step_graph = nullptr;
  std::vector<unsigned char> graph_key;
  int graph_kernels = 0;
  // per-kernel CUDA-event timing
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_kind;
  size_t ev_used = 0;

  int nprob() const { return (int)P.size(); }
  // FP64, one problem: one cooperative launch per step (lanczos_step)
  bool use_step_kernel(int np) const {
    if (np != 1 || !d_coop_slots || precision != DIRAC_FP64) return false;
    return step_mode == DIRAC_STEP_AUTO || step_mode == DIRAC_STEP_ONE_LAUNCH;
  }
  // mixed precision, any number of problems: one cooperative launch per step
  // (lanczos_step_m32) when asked for; per-pass launches are the default
  // (measured faster: 1024^2 0.51 vs 0.66 ms per step, 2048^2 1.58 vs 2.07
  // ms, the 256-packet batch 9.2 vs 12.5 ms)
  bool use_m32() const { return precision == DIRAC_MIXED && step_mode == DIRAC_STEP_ONE_LAUNCH; }
  cudaError_t mark(int kind);
  dirac_status init(int n, const int* nx, const int* ny, const double* dx, const double* dy, double mass_,
                    double c_, int order_, int boundary_, int precision_, int m_max_, void* stream_);
  void release();
  dirac_status set_fields(int b, const double* V_dev, double ax, double ay, double shift);
  dirac_status run(vec4* const* psi, int nsteps, double dt, int m, double tol, const double* a_xy);
  dirac_status read_state(dirac_step_info* info);
  dirac_status set_stream(cudaStream_t s);
};

cudaError_t Engine::mark(int kind) {
  if (!profiling) return cudaSuccess;
  if (ev_used == ev_pool.size()) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return e;
    ev_pool.push_back(ev);
    ev_kind.push_back(kind);
  }
  ev_kind[ev_used] = kind;
  return cudaEventRecord(ev_pool[ev_used++], stream);
}

dirac_status check_common(double mass, double c, int order, int boundary, int precision, int m_max) {
  if (!(c > 0) || !std::isfinite(c)) return fail(DIRAC_EINVAL, "c must be finite and > 0");
  if (!(mass >= 0) || !std::isfinite(mass)) return fail(DIRAC_EINVAL, "mass must be finite and >= 0");
  if (order != 2 && order != 4) return fail(DIRAC_EINVAL, "stencil_order must be 2 or 4");
  if (boundary != DIRAC_PERIODIC && boundary != DIRAC_DIRICHLET) return fail(DIRAC_EINVAL, "bad boundary");
  if (precision != DIRAC_FP64 && precision != DIRAC_MIXED)
    return fail(DIRAC_EINVAL, "precision must be DIRAC_FP64 or DIRAC_MIXED");
  if (m_max < 1 || m_max > DIRAC_KRYLOV_MAX) return fail(DIRAC_EINVAL, "m_max must be 1..%d", DIRAC_KRYLOV_MAX);
  return DIRAC_OK;
}

dirac_status check_grid(int nx, int ny, double dx, double dy) {
  if (nx < 1 || ny < 1) return fail(DIRAC_EINVAL, "grid %d x %d must be at least 1 x 1", nx, ny);
  if ((long long)nx * ny > (1LL << 31)) return fail(DIRAC_EINVAL, "grid too large");
  if (!(dx > 0) || !(dy > 0) || !std::isfinite(dx) || !std::isfinite(dy))
    return fail(DIRAC_EINVAL, "dx, dy must be finite and > 0");
  return DIRAC_OK;
}

// tiles of a problem at tile height th
int tiles_of(int nx, int ny, int th) { return ((nx + TILE_W - 1) / TILE_W) * ((ny + th - 1) / th); }

// FP64 tile height when none is set.  One CTA per SM streams its chunk of
// tiles, so the SM with the most tiles sets the pass time:
// ceil(tiles / SMs) x (rows + about a quarter row of per-tile cost: halo,
// barriers).  16-row tiles win on grids that leave SMs idle or end with a
// nearly empty last tile per SM; 32-row tiles otherwise.
int fp64_tile_height(const std::vector<HostProblem>& P, int n_sm) {
  double best = 1e300;
  int pick = 32;
  for (int th : {32, 16}) {
    long long t = 0;
    for (const HostProblem& q : P) t += tiles_of(q.nx, q.ny, th);
    const long long per_sm = (t + n_sm - 1) / std::max(1, n_sm);
    const double cost = (double)per_sm * (th + 0.25);
    if (cost < best) { best = cost; pick = th; }
  }
  return pick;
}

dirac_status Engine::init(int n, const int* nx, const int* ny, const double* dx, const double* dy,
                          double mass_, double c_, int order_, int boundary_, int precision_, int m_max_,
                          void* stream_) {
  order = order_; boundary = boundary_; precision = precision_; m_max = m_max_;
  mass = mass_; c = c_; stream = (cudaStream_t)stream_;
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&shape.n_sm, cudaDevAttrMultiProcessorCount, dev));
  shape.th = 0;    // 0: chosen per run
  P.resize(n);
  long long sites = 0;
  size_t slots = 0;
  for (int b = 0; b < n; ++b) {
    HostProblem& q = P[b];
    q.nx = nx[b]; q.ny = ny[b]; q.dx = dx[b]; q.dy = dy[b];
    q.n = (long long)q.nx * q.ny;
    q.tiles_x = (q.nx + TILE_W - 1) / TILE_W;
    q.slot_off = slots;
    slots += (size_t)tiles_of(q.nx, q.ny, 16);   // at least one tile per slot
    sites += q.n;
  }
  // workspace: (m_max - 1) basis fields + 2 y^ fields per problem, one block
  const size_t sb = site_bytes(precision);
  const int nbasis = std::max(1, m_max - 1);
  size_t vec_bytes = 0;
  for (const HostProblem& q : P) vec_bytes += (size_t)(nbasis + 2) * align256((size_t)q.n * sb);
  cudaError_t e = cudaMalloc(&vec_mem, vec_bytes);
  if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? DIRAC_ENOMEM : DIRAC_ECUDA,
                                    "workspace (%zu bytes): %s", vec_bytes, cudaGetErrorString(e));
  char* p = static_cast<char*>(vec_mem);
  for (HostProblem& q : P) {
    const size_t f = align256((size_t)q.n * sb);
    q.basis = p; p += (size_t)nbasis * f;
    q.ybuf[0] = p; p += f;
    q.ybuf[1] = p; p += f;
    if (precision == DIRAC_MIXED) {   // the basis vectors are packed; the y^ buffers `f` apart
      q.map_v_ok = encode_field_map(&q.map_basis, false, q.basis, q.nx, q.ny, nbasis, (size_t)q.n * sb,
                                    order / 2, M32_TILE_H) &&
                   encode_field_map(&q.map_ybuf, false, q.ybuf[0], q.nx, q.ny, 2, f, order / 2, M32_TILE_H);
    }
  }
  CUDA_TRY(cudaMalloc(&d_partials, 3 * sizeof(double) * std::max<size_t>(slots, 1)));
  CUDA_TRY(cudaMalloc(&d_st, sizeof(DevState) * n));
  CUDA_TRY(cudaMallocHost(&h_st, sizeof(DevState) * n));
  CUDA_TRY(cudaMalloc(&d_step, sizeof(int)));
  if (n == 1) {
    coop_cap = shape.n_sm * 8;     // the most resident CTAs of any pass kernel
    CUDA_TRY(cudaMalloc(&d_coop_slots, 2 * 3 * sizeof(double) * coop_cap));
  }
  CUDA_TRY(cudaMalloc(&d_coop_bar, GRID_SYNC_WORDS * sizeof(unsigned)));
  CUDA_TRY(cudaMemsetAsync(d_st, 0, sizeof(DevState) * n, stream));
  CUDA_TRY(cudaEventCreateWithFlags(&tab_ev, cudaEventDisableTiming));
  // recombination blocks in proportion to the problem sizes
  const long long rmax = std::max<long long>(n, (long long)shape.n_sm * 8);
  std::vector<int> blk;
  for (int b = 0; b < n; ++b) {
    HostProblem& q = P[b];
    long long want = (long long)((double)rmax * (double)q.n / (double)sites + 0.5);
    want = std::max<long long>(1, std::min<long long>(want, (q.n + 255) / 256));
    q.rblk_begin = (int)blk.size();
    q.rblk_count = (int)want;
    for (long long k = 0; k < want; ++k) blk.push_back(b);
  }
  rgrid = (int)blk.size();
  CUDA_TRY(cudaMalloc(&d_blk_prob, sizeof(int) * blk.size()));
  CUDA_TRY(cudaMemcpy(d_blk_prob, blk.data(), sizeof(int) * blk.size(), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaStreamSynchronize(stream));
  return DIRAC_OK;
}

void Engine::release() {
  cudaStreamSynchronize(stream);
  if (step_graph) cudaGraphExecDestroy(step_graph);
  if (cap_stream) cudaStreamDestroy(cap_stream);
  for (cudaEvent_t ev : ev_pool) cudaEventDestroy(ev);
  ev_pool.clear();
  if (tab_ev) cudaEventDestroy(tab_ev);
  cudaFree(vec_mem);
  for (HostProblem& q : P) {
    if (q.V64 != q.V) cudaFree(q.V64);
    cudaFree(q.V);
    cudaFree(q.Vlo);
  }
  cudaFree(d_st);
  cudaFreeHost(h_st);
  cudaFree(d_partials);
  cudaFree(d_coop_slots);
  cudaFree(d_coop_bar);
  cudaFree(d_blk_prob);
  cudaFree(d_step);
  cudaFree(d_tab);
  cudaFreeHost(h_tab);
  cudaFree(psi_own);
}

dirac_status Engine::set_stream(cudaStream_t s) {
  if (s != stream) {
    // order the new stream after everything already queued on the old one
    cudaEvent_t ev;
    CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CUDA_TRY(cudaEventRecord(ev, stream));
    CUDA_TRY(cudaStreamWaitEvent(s, ev, 0));
    CUDA_TRY(cudaEventDestroy(ev));
    stream = s;
  }
  return DIRAC_OK;
}

dirac_status Engine::set_fields(int b, const double* V_dev, double ax, double ay, double shift) {
  if (b < 0 || b >= nprob()) return fail(DIRAC_EINVAL, "problem index %d out of range", b);
  if (!std::isfinite(ax) || !std::isfinite(ay) || !std::isfinite(shift))
    return fail(DIRAC_EINVAL, "non-finite field scalar");
  HostProblem& q = P[b];
  if (V_dev) {
    const bool f32 = precision != DIRAC_FP64;
    if (!q.V) CUDA_TRY(cudaMalloc(&q.V, (f32 ? sizeof(float) : sizeof(double)) * q.n));
    if (f32) {
      if (!q.Vlo) CUDA_TRY(cudaMalloc(&q.Vlo, sizeof(float) * q.n));
      split_float_kernel<<<256, 256, 0, stream>>>(V_dev, static_cast<float*>(q.V), q.Vlo, q.n);
      ++launches;
      CUDA_TRY(cudaGetLastError());
      if (!q.V64) CUDA_TRY(cudaMalloc(&q.V64, sizeof(double) * q.n));
    } else {
      q.V64 = static_cast<double*>(q.V);
    }
    CUDA_TRY(cudaMemcpyAsync(q.V64, V_dev, sizeof(double) * q.n, cudaMemcpyDeviceToDevice, stream));
    double* mm = d_partials;   // two doubles of scratch (rewritten by every pass)
    minmax_kernel<<<1, 256, 0, stream>>>(V_dev, q.n, mm);
    ++launches;
    CUDA_TRY(cudaGetLastError());
    double h[2];
    CUDA_TRY(cudaMemcpyAsync(h, mm, sizeof(h), cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    if (!std::isfinite(h[0]) || !std::isfinite(h[1])) return fail(DIRAC_EINVAL, "V has non-finite entries");
    q.vmin = h[0];
    q.vmax = h[1];
    q.has_v = true;
  } else {
    q.has_v = false;
    q.vmin = q.vmax = 0.0;
  }
  q.ax = ax;
  q.ay = ay;
  q.shift = shift;
  q.fields_set = true;
  need_probe = true;
  return DIRAC_OK;
}

dirac_status Engine::run(vec4* const* psi, int nsteps, double dt, int m, double tol, const double* a_xy) {
  const int np = nprob();
  for (int b = 0; b < np; ++b) {
    if (!P[b].fields_set) return fail(DIRAC_ESTATE, "fields of problem %d not set", b);
    if (!psi[b] || !aligned32(psi[b])) return fail(DIRAC_EINVAL, "psi of problem %d null or not 32-byte aligned", b);
  }
  if (m < 1 || m > m_max) return fail(DIRAC_EINVAL, "m = %d outside 1..m_max = %d", m, m_max);
  if (!(dt != 0.0) || !std::isfinite(dt)) return fail(DIRAC_EINVAL, "dt must be finite and nonzero");
  const bool backward = dt < 0.0;   // exp(+i H |dt|): the conjugate of the forward coefficients
  dt = std::fabs(dt);
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(DIRAC_EINVAL, "tol must be finite and >= 0");
  if (nsteps < 0) return fail(DIRAC_EINVAL, "nsteps < 0");
  if (nsteps == 0) return DIRAC_OK;
  if (a_xy)
    for (long long k = 0; k < 2LL * nsteps * np; ++k)
      if (!std::isfinite(a_xy[k])) return fail(DIRAC_EINVAL, "non-finite vector potential in the schedule");
  const bool m32 = use_m32();
  const int th = m32 ? M32_TILE_H
                     : (shape.th ? shape.th : (precision == DIRAC_FP64 ? fp64_tile_height(P, shape.n_sm) : 16));
  // tile list for this tile height
  int tt = 0;
  for (HostProblem& q : P) {
    q.ntiles = tiles_of(q.nx, q.ny, th);
    q.tile_begin = tt;
    tt += q.ntiles;
  }
  total_tiles = tt;
  // tables: problems, Chebyshev parameters, fields of every step
  const int nfield = a_xy ? nsteps * np : np;
  const size_t off_cheb = align256(sizeof(Problem) * np);
  const size_t off_field = off_cheb + align256(sizeof(ChebParams) * np);
  const size_t off_maps = off_field + align256(sizeof(FieldStep) * nfield);
  const size_t bytes = off_maps + (m32 ? align256(sizeof(TmaMaps) * np) : 0);
  if (tab_ev_live) CUDA_TRY(cudaEventSynchronize(tab_ev));   // staging free again
  if (bytes > tab_cap) {
    CUDA_TRY(cudaStreamSynchronize(stream));
    cudaFree(d_tab);
    cudaFreeHost(h_tab);
    d_tab = h_tab = nullptr;
    tab_cap = 0;
    CUDA_TRY(cudaMalloc(&d_tab, bytes));
    CUDA_TRY(cudaMallocHost(&h_tab, bytes));
    tab_cap = bytes;
  }
  char* hb = static_cast<char*>(h_tab);
  char* db = static_cast<char*>(d_tab);
  Problem* hp = reinterpret_cast<Problem*>(hb);
  ChebParams* hc = reinterpret_cast<ChebParams*>(hb + off_cheb);
  FieldStep* hf = reinterpret_cast<FieldStep*>(hb + off_field);
  TmaMaps* hm = m32 ? reinterpret_cast<TmaMaps*>(hb + off_maps) : nullptr;
  const double kfac = (order == 2) ? 2.0 : 12.0;
  const double mcc = mass * c * c;
  bool hasv = false;
  for (int b = 0; b < np; ++b) {
    HostProblem& q = P[b];
    double axm = std::fabs(q.ax), aym = std::fabs(q.ay);
    if (a_xy) {
      axm = aym = 0.0;
      for (int s = 0; s < nsteps; ++s) {
        axm = std::max(axm, std::fabs(a_xy[2 * ((size_t)s * np + b)]));
        aym = std::max(aym, std::fabs(a_xy[2 * ((size_t)s * np + b) + 1]));
      }
      q.ax = a_xy[2 * ((size_t)(nsteps - 1) * np + b)];
      q.ay = a_xy[2 * ((size_t)(nsteps - 1) * np + b) + 1];
    }
    double c0, half;
    spectral_interval(order, q.dx, q.dy, mass, c, axm, aym, q.has_v ? q.vmin : 0.0,
                      q.has_v ? q.vmax : 0.0, q.shift, c0, half);
    dirac_status s = make_cheb(c0, half, dt, q.shift, hc[b]);
    if (s != DIRAC_OK) return s;
    Problem& d = hp[b];
    std::memset(&d, 0, sizeof(d));
    d.nx = q.nx; d.ny = q.ny; d.tiles_x = q.tiles_x; d.tile_begin = q.tile_begin; d.ntiles = q.ntiles;
    d.rblk_begin = q.rblk_begin; d.rblk_count = q.rblk_count;
    d.psi = psi[b];
    d.basis = q.basis; d.ybuf0 = q.ybuf[0]; d.ybuf1 = q.ybuf[1];
    d.V = q.has_v ? q.V : nullptr;
    d.Vlo = q.has_v ? q.Vlo : nullptr;
    d.st = d_st + b;
    d.partials = d_partials + 3 * q.slot_off;
    d.cheb = reinterpret_cast<const ChebParams*>(db + off_cheb) + b;
    d.kx = c / (kfac * q.dx);
    d.ky = c / (kfac * q.dy);
    d.kxf = (float)d.kx;
    d.kyf = (float)d.ky;
    d.kxf_lo = (float)(d.kx - (double)d.kxf);
    d.kyf_lo = (float)(d.ky - (double)d.kyf);
    d.shift = q.shift;
    d.probe_coef = make_coef(1.0, 0.0, 0.0, mcc - q.shift, -mcc - q.shift);
    if (m32) {
      if (q.map_psi_addr != psi[b]) {
        q.map_psi_ok = encode_field_map(&q.map_psi, true, psi[b], q.nx, q.ny, 0, 0, order / 2, M32_TILE_H);
        q.map_psi_addr = psi[b];
      }
      hm[b].basis = q.map_basis;
      hm[b].ybuf = q.map_ybuf;
      hm[b].psi = q.map_psi;
      d.tma = (q.map_v_ok && q.map_psi_ok) ? 1 : 0;
    }
    hasv = hasv || q.has_v;
  }
  bool has_ay = false;
  for (int k = 0; k < nfield; ++k) {
    const int b = k % np;
    const double ax = a_xy ? a_xy[2 * (size_t)k] : P[b].ax;
    const double ay = a_xy ? a_xy[2 * (size_t)k + 1] : P[b].ay;
    has_ay = has_ay || ay != 0.0;
    FieldStep& f = hf[k];
    f.cAx = c * ax;   // electron: p - qA = p + A
    f.cAy = c * ay;
    f.cAxf = (float)f.cAx;
    f.cAyf = (float)f.cAy;
    f.cAxf_lo = (float)(f.cAx - (double)f.cAxf);
    f.cAyf_lo = (float)(f.cAy - (double)f.cAyf);
  }
  CUDA_TRY(cudaMemcpyAsync(d_tab, h_tab, bytes, cudaMemcpyHostToDevice, stream));
  CUDA_TRY(cudaEventRecord(tab_ev, stream));
  tab_ev_live = true;
  CUDA_TRY(cudaMemsetAsync(d_step, 0, sizeof(int), stream));

  LaunchParams lp;
  std::memset(&lp, 0, sizeof(lp));
  lp.probs = reinterpret_cast<const Problem*>(d_tab);
  lp.maps = m32 ? reinterpret_cast<const TmaMaps*>(db + off_maps) : nullptr;
  lp.states = d_st;
  lp.fields = reinterpret_cast<const FieldStep*>(db + off_field);
  lp.fstride = a_xy ? np : 0;
  lp.nprob = np;
  lp.total_tiles = total_tiles;
  lp.m = m;
  lp.mcc = mcc;
  lp.dt = dt;
  lp.conj_coef = backward ? 1 : 0;
  lp.has_ay = has_ay ? 1 : 0;
  lp.diri = boundary == DIRAC_DIRICHLET ? 1 : 0;
  lp.tol = tol;
  lp.step = d_step;
  lp.redo_budget = redo_budget(precision, m);
  lp.kappa_redo = kappa_redo(precision);
  RecombParams rp;
  rp.probs = lp.probs;
  rp.blk_prob = d_blk_prob;
  rp.step = d_step;
  rp.redo_budget = lp.redo_budget;
  LaunchShape ls = shape;
  ls.th = th;
  const bool diri = boundary == DIRAC_DIRICHLET;
  if (need_probe) {
    lp.pass = 1;
    lp.probe = 1;
    CUDA_TRY(mark(KIND_PASS));
    CUDA_TRY(launch_pass(precision, order, diri, hasv, lp, ls, stream));
    ++launches;
    lp.probe = 0;
    need_probe = false;
  }
  if (use_step_kernel(np)) {
    // one cooperative launch per step (the barrier words restart at zero)
    CoopArgs ca;
    ca.slots = d_coop_slots;
    ca.bar = d_coop_bar;
    ca.G = 0;
    ca.cap = coop_cap;
    ca.bar_count = barrier_extra;
    for (int s = 0; s < nsteps; ++s) {
      CUDA_TRY(cudaMemsetAsync(d_coop_bar, 0, GRID_SYNC_WORDS * sizeof(unsigned), stream));
      CUDA_TRY(mark(KIND_STEP));
      CUDA_TRY(launch_step(precision, th, order, diri, hasv, lp, shape.n_sm, ca, stream));
      ++launches;
    }
    CUDA_TRY(mark(KIND_END));
    return DIRAC_OK;
  }
  // One step: m passes plus the spare launches for re-runs (every problem
  // runs its own next pass; launches with nothing left to do exit at once),
  // then the recombination.  The launches are the same at every step (the
  // fields come from the table through the device step counter).
  CoopArgs ca32;
  ca32.slots = d_coop_slots;
  ca32.bar = d_coop_bar;
  ca32.G = 0;
  ca32.cap = coop_cap;
  ca32.bar_count = barrier_extra;
  auto enqueue_step = [&](cudaStream_t st, bool count) -> dirac_status {
    if (m32) {   // the whole step in one launch (the barrier words restart at zero)
      CUDA_TRY(cudaMemsetAsync(d_coop_bar, 0, GRID_SYNC_WORDS * sizeof(unsigned), st));
      if (count) CUDA_TRY(mark(KIND_STEP));
      CUDA_TRY(launch_step_m32(order, diri, lp, shape.n_sm, ca32, st));
      if (count) {
        ++launches;
        CUDA_TRY(mark(KIND_END));
      }
      return DIRAC_OK;
    }
    for (int i = 1; i <= m + lp.redo_budget; ++i) {
      lp.pass = i;
      if (count) CUDA_TRY(mark(KIND_PASS));
      CUDA_TRY(launch_pass(precision, order, diri, hasv, lp, ls, st));
      if (count) ++launches;
    }
    if (count) CUDA_TRY(mark(KIND_RECOMBINE));
    CUDA_TRY(launch_recombine(precision, rp, rgrid, st));
    if (count) {
      ++launches;
      CUDA_TRY(mark(KIND_END));
    }
    return DIRAC_OK;
  };
  if (use_graphs && !profiling && nsteps >= 2) {
    // capture once per launch configuration, replay every step
    std::vector<unsigned char> key(sizeof(LaunchParams) + sizeof(RecombParams) + sizeof(LaunchShape) + 3 * sizeof(int));
    unsigned char* kp = key.data();
    LaunchParams lk = lp;
    lk.pass = 0;
    std::memcpy(kp, &lk, sizeof(lk)); kp += sizeof(lk);
    std::memcpy(kp, &rp, sizeof(rp)); kp += sizeof(rp);
    std::memcpy(kp, &ls, sizeof(ls)); kp += sizeof(ls);
    const int extra[3] = {precision + 2 * (int)m32, (int)hasv, rgrid};
    std::memcpy(kp, extra, sizeof(extra));
    if (!step_graph || key != graph_key) {
      if (!cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
      if (step_graph) { cudaGraphExecDestroy(step_graph); step_graph = nullptr; }
      cudaGraph_t g = nullptr;
      CUDA_TRY(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal));
      dirac_status st = enqueue_step(cap_stream, false);
      cudaError_t e = cudaStreamEndCapture(cap_stream, &g);
      if (st != DIRAC_OK) { if (g) cudaGraphDestroy(g); return st; }
      if (e != cudaSuccess) return fail(DIRAC_ECUDA, "step capture: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&step_graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) { step_graph = nullptr; return fail(DIRAC_ECUDA, "graph instantiate: %s", cudaGetErrorString(e)); }
      graph_key = key;
      graph_kernels = m32 ? 1 : m + lp.redo_budget + 1;
    }
    for (int s = 0; s < nsteps; ++s) {
      CUDA_TRY(cudaGraphLaunch(step_graph, stream));
      launches += graph_kernels;
    }
  } else {
    for (int s = 0; s < nsteps; ++s) {
      dirac_status st = enqueue_step(stream, true);
      if (st != DIRAC_OK) return st;
    }
  }
  return DIRAC_OK;
}

dirac_status Engine::read_state(dirac_step_info* info) {
  const int np = nprob();
  CUDA_TRY(cudaMemcpyAsync(h_st, d_st, sizeof(DevState) * np, cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  bool bad = false;
  for (int b = 0; b < np; ++b) bad = bad || h_st[b].error;
  if (bad) {
    const int zero[2] = {0, 0};
    for (int b = 0; b < np; ++b) {
      if (!h_st[b].error) continue;
      CUDA_TRY(cudaMemcpyAsync(&d_st[b].stopped, &zero[0], sizeof(int), cudaMemcpyHostToDevice, stream));
      CUDA_TRY(cudaMemcpyAsync(&d_st[b].error, &zero[1], sizeof(int), cudaMemcpyHostToDevice, stream));
    }
    CUDA_TRY(cudaStreamSynchronize(stream));
    need_probe = true;
  }
  if (info) {
    for (int b = 0; b < np; ++b) {
      const DevState& h = h_st[b];
      dirac_step_info& o = info[b];
      std::memset(&o, 0, sizeof(o));
      o.k_used = h.k_used;
      o.breakdown = h.breakdown;
      o.err_est = h.err_est;
      o.cum_err = h.cum_err;
      o.norm = h.psi_norm;
      o.energy = h.energy;
      o.kappa_max = h.kappa_max;
      for (int j = 0; j < h.k_used && j < DIRAC_KRYLOV_MAX; ++j) {
        o.alpha[j] = h.alpha[j + 1];
        o.beta[j] = h.beta[j + 1];
      }
    }
  }
  if (bad) {
    for (int b = 0; b < np; ++b)
      if (h_st[b].error == ERR_BARRIER)
        return fail(DIRAC_ECUDA, "a grid barrier of the one-launch step timed out; psi left unchanged");
    return fail(DIRAC_ENONFINITE, "non-finite value in a Lanczos reduction; psi left unchanged");
  }
  return DIRAC_OK;
}

dirac_status profile_read(Engine& e, double* ms, long long* launches) {
  for (int k = 0; k < DIRAC_KERNEL_KINDS; ++k) { ms[k] = 0.0; launches[k] = 0; }
  if (e.ev_used > 0) CUDA_TRY(cudaEventSynchronize(e.ev_pool[e.ev_used - 1]));
  for (size_t j = 0; j + 1 < e.ev_used; ++j) {
    const int k = e.ev_kind[j];
    if (k < 0) continue;
    float t = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&t, e.ev_pool[j], e.ev_pool[j + 1]));
    ms[k] += t;
    launches[k] += 1;
  }
  e.ev_used = 0;
  return DIRAC_OK;
}

}  // namespace

struct dirac_ctx {
  Engine e;
};

struct dirac_batch {
  Engine e;
};

namespace dirac {

dirac_status ctx_view(dirac_ctx* ctx, CtxView* v) {
  if (!ctx) return fail(DIRAC_EINVAL, "null context");
  const Engine& e = ctx->e;
  const HostProblem& q = e.P[0];
  v->nx = q.nx; v->ny = q.ny; v->dx = q.dx; v->dy = q.dy;
  v->mass = e.mass; v->c = e.c; v->order = e.order; v->boundary = e.boundary;
  v->V = q.has_v ? q.V64 : nullptr;
  v->vmin = q.vmin; v->vmax = q.vmax;
  v->ax = q.ax; v->ay = q.ay; v->shift = q.shift;
  v->fields_set = q.fields_set;
  v->stream = e.stream;
  v->launches = &ctx->e.launches;
  v->profiling = e.profiling;
  v->precision = e.precision;
  v->m_max = e.m_max;
  v->dev_state = e.d_st;
  v->basis = q.basis;
  return DIRAC_OK;
}

dirac_status operator_interval(dirac_ctx* ctx, double ax_max, double ay_max, double* c0, double* half) {
  if (!ctx) return fail(DIRAC_EINVAL, "null context");
  const Engine& e = ctx->e;
  const HostProblem& q = e.P[0];
  spectral_interval(e.order, q.dx, q.dy, e.mass, e.c, ax_max, ay_max, q.vmin, q.vmax, q.shift, *c0, *half);
  return DIRAC_OK;
}

dirac_status cheb_params(double c0, double half, double dt, double shift, ChebParams* cp) {
  return make_cheb(c0, half, dt, shift, *cp);
}

}  // namespace dirac

namespace {

// ----------------------------- measured peak -------------------------------

// Independent fused multiply-add chains, eight per thread, iterated to a
// bounded fixed point (x -> a x + b with |a| < 1): no overflow, no
// subnormals, and a result the compiler cannot drop.
template <class T>
__global__ void __launch_bounds__(256) fma_peak_kernel(T* sink, int iters, T a, T b) {
  constexpr int C = 8;
  T x[C];
#pragma unroll
  for (int c = 0; c < C; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < C; ++c) x[c] = fma(x[c], a, b);
  }
  T t = (T)0;
#pragma unroll
  for (int c = 0; c < C; ++c) t += x[c];
  if (t == (T)-1.0) sink[blockIdx.x] = t;   // never true: keeps the chains live
}

template <class T>
dirac_status measure_fma_peak(int iters, double* tflops) {
  int dev = 0, n_sm = 0, occ = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fma_peak_kernel<T>, 256, 0));
  const int grid = n_sm * std::max(occ, 1);
  T* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t st = nullptr;
  CUDA_TRY(cudaMalloc(&sink, sizeof(T) * grid));
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const T a = (T)(1.0 - 1.0 / 1048576.0), b = (T)(1.0 / 1024.0);
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first run warms up
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
      fma_peak_kernel<T><<<grid, 256, 0, st>>>(sink, iters, a, b);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0) best = std::min(best, ms);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(sink);
  if (e != cudaSuccess) return fail(DIRAC_ECUDA, "peak measurement: %s", cudaGetErrorString(e));
  const double fmas = (double)grid * 256.0 * 8.0 * (double)iters;
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  return DIRAC_OK;
}

}  // namespace

extern "C" {

const char* dirac_status_string(dirac_status s) {
  switch (s) {
    case DIRAC_OK: return "ok";
    case DIRAC_EINVAL: return "invalid argument";
    case DIRAC_ENOMEM: return "out of memory";
    case DIRAC_ECUDA: return "CUDA error";
    case DIRAC_ENONFINITE: return "non-finite value";
    case DIRAC_ESTATE: return "call out of order";
  }
  return "unknown status";
}

const char* dirac_last_error(void) { return g_err; }

dirac_status dirac_create(dirac_ctx** out, int nx, int ny, double dx, double dy, double mass,
                          double c, int stencil_order, int boundary, int precision, int m_max,
                          void* cuda_stream) {
  g_err[0] = 0;
  if (!out) return fail(DIRAC_EINVAL, "null output pointer");
  *out = nullptr;
  dirac_status s = check_grid(nx, ny, dx, dy);
  if (s == DIRAC_OK) s = check_common(mass, c, stencil_order, boundary, precision, m_max);
  if (s != DIRAC_OK) return s;
  dirac_ctx* ctx = new (std::nothrow) dirac_ctx;
  if (!ctx) return fail(DIRAC_ENOMEM, "host allocation failed");
  s = ctx->e.init(1, &nx, &ny, &dx, &dy, mass, c, stencil_order, boundary, precision, m_max, cuda_stream);
  if (s != DIRAC_OK) {
    ctx->e.release();
    delete ctx;
    return s;
  }
  *out = ctx;
  return DIRAC_OK;
}

void dirac_destroy(dirac_ctx* ctx) {
  if (!ctx) return;
  ctx->e.release();
  delete ctx;
}

dirac_status dirac_set_stream(dirac_ctx* ctx, void* cuda_stream) {
  if (!ctx) return fail(DIRAC_EINVAL, "null context");
  return ctx->e.set_stream((cudaStream_t)cuda_stream);
}

dirac_status dirac_set_fields(dirac_ctx* ctx, const double* V_dev, double A_x, double A_y,
                              double energy_shift) {
  if (!ctx) return fail(DIRAC_EINVAL, "null context");
  return ctx->e.set_fields(0, V_dev, A_x, A_y, energy_shift);
}

dirac_status dirac_set_vector_potential(dirac_ctx* ctx, double A_x, double A_y) {
  if (!ctx) return fail(DIRAC_EINVAL, "null context");
  if (!std::isfinite(A_x) || !std::isfinite(A_y)) return fail(DIRAC_EINVAL, "non-finite vector potential");
  ctx->e.P[0].ax = A_x;
  ctx->e.P[0].ay = A_y;
  return DIRAC_OK;
}

dirac_status dirac_lanczos_step(dirac_ctx* ctx, void* psi_dev, double dt, int m, double tol,
                                dirac_step_info* info) {
  return dirac_lanczos_steps(ctx, psi_dev, 1, dt, m, tol, nullptr, info);
}

dirac_status dirac_lanczos_steps(dirac_ctx* ctx, void* psi_dev, int nsteps, double dt, int m,
                                 double tol, const double* A_xy_host, dirac_step_info* info) {
  dirac::TraceRange trace("dirac_lanczos_steps");
  if (!ctx) return fail(DIRAC_EINVAL, "null context");
  if (!psi_dev) return fail(DIRAC_EINVAL, "null psi");
  vec4* psi = static_cast<vec4*>(psi_dev);
  dirac_status s = ctx->e.run(&psi, nsteps, dt, m, tol, A_xy_host);
  if (s != DIRAC_OK) return s;
  if (info) return ctx->e.read_state(info);
  return DIRAC_OK;
}

dirac_status dirac_propagate_host(dirac_ctx* ctx, void* psi_host, int nsteps, double dt, int m,
                                  double tol, const double* A_xy_host, dirac_step_info* info) {
  dirac::TraceRange trace("dirac_propagate_host");
  if (!ctx) return fail(DIRAC_EINVAL, "null context");
  if (!psi_host) return fail(DIRAC_EINVAL, "null psi");
  Engine& e = ctx->e;
  const size_t bytes = (size_t)e.P[0].n * sizeof(vec4);
  if (!e.psi_own) CUDA_TRY(cudaMalloc(&e.psi_own, bytes));
  CUDA_TRY(cudaMemcpyAsync(e.psi_own, psi_host, bytes, cudaMemcpyHostToDevice, e.stream));
  dirac_status s = e.run(&e.psi_own, nsteps, dt, m, tol, A_xy_host);
  if (s != DIRAC_OK) return s;
  CUDA_TRY(cudaMemcpyAsync(psi_host, e.psi_own, bytes, cudaMemcpyDeviceToHost, e.stream));
  return e.read_state(info);
}

dirac_status dirac_sync(dirac_ctx* ctx) {
  if (!ctx) return fail(DIRAC_EINVAL, "null context");
  return ctx->e.read_state(nullptr);
}

size_t dirac_state_bytes(const dirac_ctx* ctx) {
  return ctx ? sizeof(DevState) * ctx->e.P.size() : 0;
}

dirac_status dirac_export_state(dirac_ctx* ctx, void* host, size_t bytes) {
  if (!ctx || !host) return fail(DIRAC_EINVAL, "null context or buffer");
  Engine& e = ctx->e;
  if (bytes != sizeof(DevState) * e.P.size()) return fail(DIRAC_EINVAL, "state buffer of %zu bytes, need %zu",
                                                           bytes, sizeof(DevState) * e.P.size());
  if (e.need_probe) return fail(DIRAC_ESTATE, "no step has run since the context was created or re-armed");
  dirac_status s = e.read_state(nullptr);   // waits, and reports a pending device error
  if (s != DIRAC_OK) return s;
  std::memcpy(host, e.h_st, bytes);
  return DIRAC_OK;
}

dirac_status dirac_import_state(dirac_ctx* ctx, const void* host, size_t bytes) {
  if (!ctx || !host) return fail(DIRAC_EINVAL, "null context or buffer");
  Engine& e = ctx->e;
  if (bytes != sizeof(DevState) * e.P.size()) return fail(DIRAC_EINVAL, "state buffer of %zu bytes, need %zu",
                                                           bytes, sizeof(DevState) * e.P.size());
  const DevState* st = static_cast<const DevState*>(host);
  for (size_t b = 0; b < e.P.size(); ++b)
    if (st[b].error || st[b].stopped || !st[b].sigma_valid || st[b].cur_pass != 1)
      return fail(DIRAC_EINVAL, "not a state exported between steps");
  CUDA_TRY(cudaStreamSynchronize(e.stream));
  CUDA_TRY(cudaMemcpy(e.d_st, host, bytes, cudaMemcpyHostToDevice));
  e.need_probe = false;   // the imported stencil shift is the one the next step uses
  return DIRAC_OK;
}

double dirac_pulse_sin2_mean(double t0, double dt, double a0, double omega, double duration) {
  // sin^2(pi t/T) sin(w t) = sin(w t)/2 - sin((w+W) t)/4 - sin((w-W) t)/4, W = 2 pi / T
  if (!(dt > 0.0) || !(duration > 0.0)) return 0.0;
  const double a = std::max(t0, 0.0), b = std::min(t0 + dt, duration);
  if (b <= a) return 0.0;
  const double W = 2.0 * M_PI / duration;
  auto integ = [&](double nu) {   // integral of sin(nu t) over [a, b]
    if (nu == 0.0) return 0.0;
    return 2.0 * std::sin(0.5 * nu * (a + b)) * std::sin(0.5 * nu * (b - a)) / nu;
  };
  return a0 * (0.5 * integ(omega) - 0.25 * integ(omega + W) - 0.25 * integ(omega - W)) / dt;
}

dirac_status dirac_pulse_sine_basis_means(int nsteps, double dt, int n_coef, double duration, double* W) {
  if (nsteps < 1 || n_coef < 1 || !W) return fail(DIRAC_EINVAL, "bad sizes or null output");
  if (!(dt > 0.0) || !(duration > 0.0) || !std::isfinite(dt) || !std::isfinite(duration))
    return fail(DIRAC_EINVAL, "dt and duration must be finite and > 0");
  for (int n = 0; n < nsteps; ++n) {
    const double a = n * dt, b = a + dt;
    for (int k = 0; k < n_coef; ++k) {
      const double w = (k + 1) * M_PI / duration;
      // (cos(w a) - cos(w b)) / (w dt), written without cancellation
      W[(size_t)n * n_coef + k] = 2.0 * std::sin(0.5 * w * (a + b)) * std::sin(0.5 * w * dt) / (w * dt);
    }
  }
  return DIRAC_OK;
}

long long dirac_kernel_launches(const dirac_ctx* ctx) { return ctx ? ctx->e.launches : 0; }

dirac_status dirac_profile_enable(dirac_ctx* ctx, int enable) {
  if (!ctx) return fail(DIRAC_EINVAL, "null context");
  ctx->e.profiling = enable != 0;
  return DIRAC_OK;
}

dirac_status dirac_profile_read(dirac_ctx* ctx, double* ms, long long* launches) {
  if (!ctx || !ms || !launches) return fail(DIRAC_EINVAL, "null argument");
  return profile_read(ctx->e, ms, launches);
}

// ----------------------------- batches -------------------------------------

dirac_status dirac_batch_create(dirac_batch** out, int n_problems, const int* nx, const int* ny,
                                const double* dx, const double* dy, double mass, double c,
                                int stencil_order, int boundary, int precision, int m_max,
                                void* cuda_stream) {
  g_err[0] = 0;
  if (!out) return fail(DIRAC_EINVAL, "null output pointer");
  *out = nullptr;
  if (n_problems < 1 || !nx || !ny || !dx || !dy) return fail(DIRAC_EINVAL, "need n_problems >= 1 and sizes");
  for (int b = 0; b < n_problems; ++b) {
    dirac_status s = check_grid(nx[b], ny[b], dx[b], dy[b]);
    if (s != DIRAC_OK) return s;
  }
  dirac_status s = check_common(mass, c, stencil_order, boundary, precision, m_max);
  if (s != DIRAC_OK) return s;
  dirac_batch* bt = new (std::nothrow) dirac_batch;
  if (!bt) return fail(DIRAC_ENOMEM, "host allocation failed");
  s = bt->e.init(n_problems, nx, ny, dx, dy, mass, c, stencil_order, boundary, precision, m_max, cuda_stream);
  if (s != DIRAC_OK) {
    bt->e.release();
    delete bt;
    return s;
  }
  *out = bt;
  return DIRAC_OK;
}

void dirac_batch_destroy(dirac_batch* bt) {
  if (!bt) return;
  bt->e.release();
  delete bt;
}

dirac_status dirac_batch_set_fields(dirac_batch* bt, int problem, const double* V_dev, double A_x,
                                    double A_y, double energy_shift) {
  if (!bt) return fail(DIRAC_EINVAL, "null batch");
  return bt->e.set_fields(problem, V_dev, A_x, A_y, energy_shift);
}

dirac_status dirac_batch_set_launch_shape(dirac_batch* bt, int tile_height, int ctas_per_sm) {
  if (!bt) return fail(DIRAC_EINVAL, "null batch");
  if (tile_height != 16 && tile_height != 32) return fail(DIRAC_EINVAL, "tile height must be 16 or 32");
  if (ctas_per_sm < 0) return fail(DIRAC_EINVAL, "ctas_per_sm < 0");
  bt->e.shape.th = tile_height;
  bt->e.shape.cta_cap = ctas_per_sm;
  return DIRAC_OK;
}

dirac_status dirac_batch_steps(dirac_batch* bt, void* const* psi_dev, int nsteps, double dt, int m,
                               double tol, const double* A_xy_host, dirac_step_info* info) {
  dirac::TraceRange trace("dirac_batch_steps");
  if (!bt) return fail(DIRAC_EINVAL, "null batch");
  if (!psi_dev) return fail(DIRAC_EINVAL, "null psi table");
  dirac_status s = bt->e.run(reinterpret_cast<vec4* const*>(psi_dev), nsteps, dt, m, tol, A_xy_host);
  if (s != DIRAC_OK) return s;
  if (info) return bt->e.read_state(info);
  return DIRAC_OK;
}

dirac_status dirac_batch_sync(dirac_batch* bt, dirac_step_info* info) {
  if (!bt) return fail(DIRAC_EINVAL, "null batch");
  return bt->e.read_state(info);
}

dirac_status dirac_batch_profile_enable(dirac_batch* bt, int enable) {
  if (!bt) return fail(DIRAC_EINVAL, "null batch");
  bt->e.profiling = enable != 0;
  return DIRAC_OK;
}

dirac_status dirac_batch_profile_read(dirac_batch* bt, double* ms, long long* launches) {
  if (!bt || !ms || !launches) return fail(DIRAC_EINVAL, "null argument");
  return profile_read(bt->e, ms, launches);
}

long long dirac_batch_kernel_launches(const dirac_batch* bt) { return bt ? bt->e.launches : 0; }

dirac_status dirac_batch_use_graphs(dirac_batch* bt, int enable) {
  if (!bt) return fail(DIRAC_EINVAL, "null batch");
  bt->e.use_graphs = enable != 0;
  return DIRAC_OK;
}

dirac_status dirac_use_graphs(dirac_ctx* ctx, int enable) {
  if (!ctx) return fail(DIRAC_EINVAL, "null context");
  ctx->e.use_graphs = enable != 0;
  return DIRAC_OK;
}

dirac_status dirac_debug_barrier_timeout(dirac_ctx* ctx, void* psi_dev, double dt, int m) {
  if (!ctx) return fail(DIRAC_EINVAL, "null context");
  if (!psi_dev) return fail(DIRAC_EINVAL, "null psi");
  Engine& e = ctx->e;
  if (!e.d_coop_slots) return fail(DIRAC_ESTATE, "no one-launch step on this context");
  const int mode = e.step_mode;
  e.step_mode = DIRAC_STEP_ONE_LAUNCH;
  e.barrier_extra = 1;
  vec4* psi = static_cast<vec4*>(psi_dev);
  dirac_status s = e.run(&psi, 1, dt, m, 0.0, nullptr);
  e.barrier_extra = 0;
  e.step_mode = mode;
  if (s != DIRAC_OK) return s;
  return e.read_state(nullptr);
}

dirac_status dirac_set_step_mode(dirac_ctx* ctx, int mode) {
  if (!ctx) return fail(DIRAC_EINVAL, "null context");
  if (mode != DIRAC_STEP_AUTO && mode != DIRAC_STEP_PASSES && mode != DIRAC_STEP_ONE_LAUNCH)
    return fail(DIRAC_EINVAL, "unknown step mode %d", mode);
  ctx->e.step_mode = mode;
  return DIRAC_OK;
}

dirac_status dirac_batch_set_step_mode(dirac_batch* bt, int mode) {
  if (!bt) return fail(DIRAC_EINVAL, "null batch");
  if (mode != DIRAC_STEP_AUTO && mode != DIRAC_STEP_PASSES && mode != DIRAC_STEP_ONE_LAUNCH)
    return fail(DIRAC_EINVAL, "unknown step mode %d", mode);
  bt->e.step_mode = mode;
  return DIRAC_OK;
}

// Autotuner: time each candidate launch shape on scratch copies of the
// states (the caller's states and the scalar blocks are left as they were),
// keep the fastest, remember it in the cache file named by
// DIRAC_AUTOTUNE_CACHE (one line per problem signature).
dirac_status dirac_batch_autotune(dirac_batch* bt, void* const* psi_dev, double dt, int m,
                                  const double* A_xy_host, int steps, dirac_tune_result* out) {
  if (!bt || !psi_dev) return fail(DIRAC_EINVAL, "null argument");
  if (steps < 1) return fail(DIRAC_EINVAL, "steps must be >= 1");
  Engine& e = bt->e;
  const int np = e.nprob();
  long long sites = 0;
  for (const HostProblem& q : e.P) sites += q.n;
  char sig[256];
  {
    int dev = 0;
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
    for (char* c = prop.name; *c; ++c) if (*c == ' ') *c = '_';
    snprintf(sig, sizeof(sig), "prec=%d,order=%d,bnd=%d,nprob=%d,sites=%lld,m=%d,sm=%d,gpu=%s", e.precision,
             e.order, e.boundary, np, sites, m, e.shape.n_sm, prop.name);
  }
  const char* cache = std::getenv("DIRAC_AUTOTUNE_CACHE");
  if (cache && cache[0]) {
    if (FILE* f = std::fopen(cache, "r")) {
      char line[512], key[300];
      int th = 0, cap = 0;
      double ms = 0;
      bool found = false;
      while (std::fgets(line, sizeof(line), f)) {
        if (std::sscanf(line, "%299s %d %d %lf", key, &th, &cap, &ms) == 4 && std::strcmp(key, sig) == 0) {
          found = true;
          break;
        }
      }
      std::fclose(f);
      if (found && (th == 16 || th == 32) && cap >= 0) {
        e.shape.th = th;
        e.shape.cta_cap = cap;
        if (out) { out->tile_height = th; out->ctas_per_sm = cap; out->ms_per_step = ms; out->from_cache = 1; out->candidates = 0; }
        return DIRAC_OK;
      }
    }
  }
  // scratch states and a copy of the scalar blocks
  std::vector<size_t> off(np + 1, 0);
  for (int b = 0; b < np; ++b) off[b + 1] = off[b] + align256((size_t)e.P[b].n * sizeof(vec4));
  char* scratch = nullptr;
  DevState* st_save = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaMalloc(&scratch, off[np]));
  cudaError_t ce = cudaMalloc(&st_save, sizeof(DevState) * np);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(st_save, e.d_st, sizeof(DevState) * np, cudaMemcpyDeviceToDevice, e.stream);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  std::vector<vec4*> sp(np);
  for (int b = 0; b < np; ++b) sp[b] = reinterpret_cast<vec4*>(scratch + off[b]);
  struct Cand { int th, cap; };
  std::vector<Cand> cands;
  if (e.precision == DIRAC_FP64) cands = {{32, 0}, {16, 0}};
  else cands = {{16, 0}, {16, 4}, {32, 0}, {32, 2}};
  const LaunchShape keep = e.shape;
  const bool probe_keep = e.need_probe;
  double best = 1e300;
  Cand pick = cands[0];
  dirac_status s = DIRAC_OK;
  for (const Cand& cd : cands) {
    if (ce != cudaSuccess) break;
    for (int b = 0; b < np && ce == cudaSuccess; ++b)
      ce = cudaMemcpyAsync(sp[b], psi_dev[b], (size_t)e.P[b].n * sizeof(vec4), cudaMemcpyDeviceToDevice, e.stream);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(e.d_st, st_save, sizeof(DevState) * np, cudaMemcpyDeviceToDevice, e.stream);
    if (ce != cudaSuccess) break;
    e.need_probe = true;
    e.shape.th = cd.th;
    e.shape.cta_cap = cd.cap;
    s = e.run(sp.data(), 1, dt, m, 0.0, A_xy_host);                       // warm-up
    if (s == DIRAC_OK) ce = cudaEventRecord(e0, e.stream);
    if (s == DIRAC_OK && ce == cudaSuccess) s = e.run(sp.data(), steps, dt, m, 0.0, A_xy_host);
    if (s == DIRAC_OK && ce == cudaSuccess) ce = cudaEventRecord(e1, e.stream);
    if (s == DIRAC_OK && ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    if (s != DIRAC_OK || ce != cudaSuccess) break;
    float ms = 0.f;
    ce = cudaEventElapsedTime(&ms, e0, e1);
    const double per = ms / steps;
    if (per < best) { best = per; pick = cd; }
  }
  // leave everything as it was, with the chosen shape
  if (ce == cudaSuccess && st_save) ce = cudaMemcpyAsync(e.d_st, st_save, sizeof(DevState) * np, cudaMemcpyDeviceToDevice, e.stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(e.stream);
  e.need_probe = probe_keep;
  cudaFree(scratch);
  cudaFree(st_save);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s != DIRAC_OK) { e.shape = keep; return s; }
  if (ce != cudaSuccess) { e.shape = keep; return fail(DIRAC_ECUDA, "autotune: %s", cudaGetErrorString(ce)); }
  e.shape.th = pick.th;
  e.shape.cta_cap = pick.cap;
  if (cache && cache[0]) {
    if (FILE* f = std::fopen(cache, "a")) {
      std::fprintf(f, "%s %d %d %.6f\n", sig, pick.th, pick.cap, best);
      std::fclose(f);
    }
  }
  if (out) {
    out->tile_height = pick.th; out->ctas_per_sm = pick.cap; out->ms_per_step = best;
    out->from_cache = 0; out->candidates = (int)cands.size();
  }
  return DIRAC_OK;
}

// ----------------------------- test hook -----------------------------------

dirac_status dirac_measure_peak(int kind, double* tflops) {
  if (!tflops) return fail(DIRAC_EINVAL, "null output");
  // about 50 ms per launch on a GB300 at full clock
  if (kind == DIRAC_PEAK_FP64) return measure_fma_peak<double>(12000, tflops);
  if (kind == DIRAC_PEAK_FP32) return measure_fma_peak<float>(600000, tflops);
  return fail(DIRAC_EINVAL, "unknown peak kind %d", kind);
}

dirac_status dirac_debug_tridiag_expm(const double* alpha, const double* beta, int k, double dt,
                                      double lo, double hi, double* v_re, double* v_im) {
  if (k < 1 || k > DIRAC_KRYLOV_MAX) return fail(DIRAC_EINVAL, "k outside 1..%d", DIRAC_KRYLOV_MAX);
  if (!(lo <= hi) || !alpha || !v_re || !v_im || (k > 1 && !beta)) return fail(DIRAC_EINVAL, "bad arguments");
  ChebParams cp;
  const double half = std::max(0.5 * (hi - lo), 1e-300) * (1.0 + 1e-8) + 1e-12;
  dirac_status s = make_cheb(0.5 * (lo + hi), half, dt, 0.0, cp);
  if (s != DIRAC_OK) return s;
  double h[4 * (KMAX + 2)] = {0};
  for (int j = 0; j < k; ++j) h[j + 1] = alpha[j];
  for (int j = 0; j + 1 < k; ++j) h[(KMAX + 2) + j + 1] = beta[j];
  double* d = nullptr;
  CUDA_TRY(cudaMalloc(&d, sizeof(h)));
  cudaError_t e = cudaMemcpy(d, h, sizeof(h), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    debug_tridiag_expm<<<1, 32>>>(cp, k, d, d + (KMAX + 2), d + 2 * (KMAX + 2), d + 3 * (KMAX + 2));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(DIRAC_ECUDA, "debug_tridiag_expm: %s", cudaGetErrorString(e));
  for (int j = 0; j < k; ++j) { v_re[j] = h[2 * (KMAX + 2) + j]; v_im[j] = h[3 * (KMAX + 2) + j]; }
  return DIRAC_OK;
}

}  // extern "C"

// ===========================================================================
// Allocation-free single step (dirac_lanczos_step_noalloc).
//
// For callers that may not allocate device memory at all: a host framework
// that owns every device allocation and forbids libraries from calling
// cudaMalloc, a fixed memory budget decided up front, or a per-step loop in
// which the latency or the failure of an allocation is not acceptable.  The
// step keeps its whole workspace (problem table, scalar block, per-CTA
// partial sums, the two y^ fields and the Krylov basis) in one file-scope
// device array of fixed size, shared by every call in the process, and calls
// no cudaMalloc, cudaFree or other allocating routine (host or device).
// ===========================================================================
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 8u << 20;   // 8 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::atomic<void*> g_noalloc_ptr[NOALLOC_MAX_DEVICES];

// Device address of the scratch array on the current device.  In host code
// `g_noalloc_scratch` names a host-side shadow, not device memory, so the
// address is looked up once per device (with that device current) and kept
// for the life of the process.  cudaDeviceReset unloads the module; the kept
// address is then stale, so a process that resets a device must not call the
// allocation-free step on it again.
dirac_status noalloc_scratch(unsigned char** out) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(DIRAC_EINVAL, "device index %d too large", dev);
  void* p = g_noalloc_ptr[dev].load();
  if (!p) {
    CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev].store(p);
  }
  *out = static_cast<unsigned char*>(p);
  return DIRAC_OK;
}

// The per-call tables travel as kernel arguments (no host buffer is read
// after the call returns): one CTA writes them into the scratch and clears
// the step counter, the block map (every block is problem 0) and the scalar
// block, which the scratch keeps from the previous call.
struct NoallocTables {
  Problem pr;
  ChebParams cheb;
  FieldStep fs;
};

__global__ void noalloc_setup(const __grid_constant__ NoallocTables t, Problem* pr, ChebParams* cheb,
                              FieldStep* fs, int* step_and_blocks, int n_words, DevState* st) {
  if (threadIdx.x == 0) {
    *pr = t.pr;
    *fs = t.fs;
  }
  const double* src = reinterpret_cast<const double*>(&t.cheb);
  double* dst = reinterpret_cast<double*>(cheb);
  for (int w = threadIdx.x; w < (int)(sizeof(ChebParams) / sizeof(double)); w += blockDim.x) dst[w] = src[w];
  for (int w = threadIdx.x; w < n_words; w += blockDim.x) step_and_blocks[w] = 0;
  unsigned* sw = reinterpret_cast<unsigned*>(st);
  for (int w = threadIdx.x; w < (int)(sizeof(DevState) / sizeof(unsigned)); w += blockDim.x) sw[w] = 0u;
}

}  // namespace

extern "C" size_t dirac_noalloc_scratch_bytes(void) { return NOALLOC_SCRATCH_BYTES; }

extern "C" dirac_status dirac_lanczos_step_noalloc(const dirac_problem* pb, void* psi_dev, double dt,
                                                   int m, double tol, void* cuda_stream,
                                                   dirac_step_info* info) {
  if (!pb || !psi_dev) return fail(DIRAC_EINVAL, "null argument");
  dirac_status s = check_grid(pb->nx, pb->ny, pb->dx, pb->dy);
  if (s == DIRAC_OK) s = check_common(pb->mass, pb->c, pb->stencil_order, pb->boundary, DIRAC_FP64, m);
  if (s != DIRAC_OK) return s;
  if (!std::isfinite(pb->A_x) || !std::isfinite(pb->A_y) || !std::isfinite(pb->energy_shift))
    return fail(DIRAC_EINVAL, "non-finite field scalar");
  if (!(dt != 0.0) || !std::isfinite(dt)) return fail(DIRAC_EINVAL, "dt must be finite and nonzero");
  const bool backward = dt < 0.0;   // exp(+i H |dt|): the conjugate of the forward coefficients
  dt = std::fabs(dt);
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(DIRAC_EINVAL, "tol must be finite and >= 0");
  if (!aligned32(psi_dev)) return fail(DIRAC_EINVAL, "psi must be 32-byte aligned");

  // scratch layout: Problem | ChebParams | FieldStep | step counter and block
  //                 map | DevState | partials | y^[2] | basis[m-1]
  const int nx = pb->nx, ny = pb->ny;
  const long long n = (long long)nx * ny;
  const int tiles_x = (nx + TILE_W - 1) / TILE_W;
  const int ntiles = tiles_of(nx, ny, 32);
  constexpr int RB_MAX = 64;                   // recombination blocks
  const size_t field = align256((size_t)n * sizeof(vec4));
  const size_t off_cheb = align256(sizeof(Problem));
  const size_t off_field = off_cheb + align256(sizeof(ChebParams));
  const size_t off_step = off_field + align256(sizeof(FieldStep));
  const size_t off_st = off_step + align256(sizeof(int) * (1 + RB_MAX));
  const size_t off_part = off_st + align256(sizeof(DevState));
  const size_t off_y = off_part + align256(3 * sizeof(double) * ntiles);
  const size_t off_basis = off_y + 2 * field;
  const size_t need = off_basis + (size_t)std::max(1, m - 1) * field;
  if (need > NOALLOC_SCRATCH_BYTES)
    return fail(DIRAC_EINVAL, "grid %d x %d with m = %d needs %zu bytes of scratch; the static scratch "
                "holds %zu bytes (use dirac_create for larger problems)", nx, ny, m, need,
                NOALLOC_SCRATCH_BYTES);
  unsigned char* base = nullptr;
  s = noalloc_scratch(&base);
  if (s != DIRAC_OK) return s;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  int n_sm = 0, dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  DevState* st = reinterpret_cast<DevState*>(base + off_st);
  double* partials = reinterpret_cast<double*>(base + off_part);
  int* step = reinterpret_cast<int*>(base + off_step);
  int* blk = step + 1;

  // spectral interval of H - s (needs the range of V: read back two doubles)
  double vmin = 0.0, vmax = 0.0;
  if (pb->V_dev) {
    minmax_kernel<<<1, 256, 0, stream>>>(pb->V_dev, n, partials);
    CUDA_TRY(cudaGetLastError());
    double h[2];
    CUDA_TRY(cudaMemcpyAsync(h, partials, sizeof(h), cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    if (!std::isfinite(h[0]) || !std::isfinite(h[1])) return fail(DIRAC_EINVAL, "V has non-finite entries");
    vmin = h[0];
    vmax = h[1];
  }
  static_assert(sizeof(ChebParams) % sizeof(double) == 0, "ChebParams copied as doubles");
  NoallocTables host;   // passed by value to the setup kernel
  std::memset(&host, 0, sizeof(host));
  double c0, half;
  spectral_interval(pb->stencil_order, pb->dx, pb->dy, pb->mass, pb->c, std::fabs(pb->A_x),
                    std::fabs(pb->A_y), vmin, vmax, pb->energy_shift, c0, half);
  s = make_cheb(c0, half, dt, pb->energy_shift, host.cheb);
  if (s != DIRAC_OK) return s;
  const double kfac = (pb->stencil_order == 2) ? 2.0 : 12.0;
  const double mcc = pb->mass * pb->c * pb->c;
  const int rblocks = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, RB_MAX));
  Problem& d = host.pr;
  d.nx = nx; d.ny = ny; d.tiles_x = tiles_x; d.tile_begin = 0; d.ntiles = ntiles;
  d.rblk_begin = 0; d.rblk_count = rblocks;
  d.psi = static_cast<vec4*>(psi_dev);
  d.basis = base + off_basis;
  d.ybuf0 = base + off_y;
  d.ybuf1 = base + off_y + field;
  d.V = pb->V_dev;
  d.st = st;
  d.partials = partials;
  d.cheb = reinterpret_cast<const ChebParams*>(base + off_cheb);
  d.kx = pb->c / (kfac * pb->dx);
  d.ky = pb->c / (kfac * pb->dy);
  d.kxf = (float)d.kx;
  d.kyf = (float)d.ky;
  d.kxf_lo = (float)(d.kx - (double)d.kxf);
  d.kyf_lo = (float)(d.ky - (double)d.kyf);
  d.shift = pb->energy_shift;
  d.probe_coef = make_coef(1.0, 0.0, 0.0, mcc - pb->energy_shift, -mcc - pb->energy_shift);
  host.fs.cAx = pb->c * pb->A_x;
  host.fs.cAy = pb->c * pb->A_y;
  host.fs.cAxf = (float)host.fs.cAx;
  host.fs.cAyf = (float)host.fs.cAy;
  host.fs.cAxf_lo = (float)(host.fs.cAx - (double)host.fs.cAxf);
  host.fs.cAyf_lo = (float)(host.fs.cAy - (double)host.fs.cAyf);
  noalloc_setup<<<1, 256, 0, stream>>>(host, reinterpret_cast<Problem*>(base),
                                       reinterpret_cast<ChebParams*>(base + off_cheb),
                                       reinterpret_cast<FieldStep*>(base + off_field), step, 1 + RB_MAX, st);
  CUDA_TRY(cudaGetLastError());

  LaunchParams lp;
  std::memset(&lp, 0, sizeof(lp));
  lp.probs = reinterpret_cast<const Problem*>(base);
  lp.states = st;
  lp.fields = reinterpret_cast<const FieldStep*>(base + off_field);
  lp.fstride = 0;
  lp.nprob = 1;
  lp.total_tiles = ntiles;
  lp.has_ay = pb->A_y != 0.0 ? 1 : 0;
  lp.m = m;
  lp.mcc = mcc;
  lp.dt = dt;
  lp.conj_coef = backward ? 1 : 0;
  lp.tol = tol;
  lp.step = step;
  lp.redo_budget = redo_budget(DIRAC_FP64, m);
  lp.kappa_redo = kappa_redo(DIRAC_FP64);
  LaunchShape ls{n_sm, 32, 0};
  const bool diri = pb->boundary == DIRAC_DIRICHLET, hasv = pb->V_dev != nullptr;
  lp.pass = 1;
  lp.probe = 1;
  CUDA_TRY(launch_pass(DIRAC_FP64, pb->stencil_order, diri, hasv, lp, ls, stream));
  lp.probe = 0;
  for (int i = 1; i <= m + lp.redo_budget; ++i) {
    lp.pass = i;
    CUDA_TRY(launch_pass(DIRAC_FP64, pb->stencil_order, diri, hasv, lp, ls, stream));
  }
  RecombParams rp;
  rp.probs = lp.probs;
  rp.blk_prob = blk;
  rp.step = step;
  rp.redo_budget = lp.redo_budget;
  CUDA_TRY(launch_recombine(DIRAC_FP64, rp, rblocks, stream));

  if (info) {
    DevState h;
    CUDA_TRY(cudaMemcpyAsync(&h, st, sizeof(DevState), cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    if (h.error) return fail(DIRAC_ENONFINITE, "non-finite value in a Lanczos reduction; psi left unchanged");
    std::memset(info, 0, sizeof(*info));
    info->k_used = h.k_used;
    info->breakdown = h.breakdown;
    info->err_est = h.err_est;
    info->cum_err = h.err_est;
    info->norm = h.psi_norm;
    info->energy = h.energy;
    for (int k = 0; k < h.k_used && k < DIRAC_KRYLOV_MAX; ++k) {
      info->alpha[k] = h.alpha[k + 1];
      info->beta[k] = h.beta[k + 1];
    }
  }
  return DIRAC_OK;
}
