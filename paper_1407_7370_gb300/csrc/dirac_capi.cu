// dirac_capi.cu -- host side of the GB300 Dirac Lanczos propagator: context,
// workspace, launch sequencing and the C ABI declared in include/dirac.h.
#include "dirac.h"
#include "dirac_kernels.cuh"

#include <cuda_runtime.h>

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

namespace {

thread_local char g_err[512] = "";

dirac_status fail(dirac_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

#define CUDA_TRY(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return fail(DIRAC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Bessel functions J_0..J_{n-1}(x), x > 0, by Miller's backward recurrence
// J_{k-1} = (2k/x) J_k - J_{k+1} started far above n and normalised with
// J_0 + 2 sum_{k>=1} J_{2k} = 1.
std::vector<double> bessel_j(int n, double x) {
  const int start = 2 * ((std::max(n, (int)x) + 40 + (int)std::sqrt(40.0 * std::max(x, 1.0))) / 2);
  std::vector<double> j(start + 2, 0.0);
  j[start + 1] = 0.0;
  j[start] = 1e-300;
  for (int k = start; k >= 1; --k) {
    j[k - 1] = (2.0 * k / x) * j[k] - j[k + 1];
    if (std::fabs(j[k - 1]) > 1e250) {      // rescale to stay in range
      for (int t = k - 1; t <= start; ++t) j[t] *= 1e-250;
    }
  }
  double norm = j[0];
  for (int k = 2; k <= start; k += 2) norm += 2.0 * j[k];
  std::vector<double> out(n);
  for (int k = 0; k < n; ++k) out[k] = j[k] / norm;
  return out;
}

}  // namespace

struct dirac_ctx {
  int nx = 0, ny = 0, order = 2, boundary = DIRAC_PERIODIC, precision = DIRAC_FP64, m_max = 1;
  double dx = 0, dy = 0, mass = 1, c = 137.036;
  cudaStream_t stream = nullptr;
  long long n_sites = 0;
  void* basis = nullptr;          // q^_2 .. q^_m (complex128, or complex64 when mixed)
  void* ybuf[2] = {nullptr, nullptr};
  vec4* psi_own = nullptr;        // staging for the host-buffer call
  void* V = nullptr;              // double, or float when mixed
  bool has_v = false;
  double vmin = 0, vmax = 0;
  double ax = 0, ay = 0, shift = 0;
  bool fields_set = false;
  bool need_probe = true;
  DevState* st = nullptr;
  DevState* st_host = nullptr;    // pinned
  double* partials = nullptr;
  dim3 grid;
  long long launches = 0;
  int n_sm = 0;
  // per-kernel CUDA-event timing (dirac_profile_*)
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_kind;
  size_t ev_used = 0;
};

namespace {

// Rigorous interval [c0 - half, c0 + half] containing the spectrum of H - s:
// H = H0(A) + V with spec(H0(A)) = {+-E_k}, E_k <= sqrt(m^2c^4 + c^2 (P_x+|A_x|)^2
// + c^2 (P_y+|A_y|)^2), P = max |stencil momentum| (1/h for order 2, for order
// 4 the maximum of (8 sin t - sin 2t)/(6h)), and V_min <= V <= V_max.
void spectral_interval(const dirac_ctx* c, double& c0, double& half) {
  double pf = 1.0;
  if (c->order == 4) {
    const double cs = 1.0 - std::sqrt(6.0) / 2.0;    // cos t at the maximum
    const double sn = std::sqrt(1.0 - cs * cs);
    pf = sn * (4.0 - cs) / 3.0;
  }
  const double px = pf / c->dx + std::fabs(c->ax), py = pf / c->dy + std::fabs(c->ay);
  const double mc2 = c->mass * c->c * c->c;
  const double emax = std::sqrt(mc2 * mc2 + c->c * c->c * (px * px + py * py));
  const double vmin = c->has_v ? c->vmin : 0.0, vmax = c->has_v ? c->vmax : 0.0;
  c0 = 0.5 * (vmin + vmax) - c->shift;
  half = (emax + 0.5 * (vmax - vmin)) * (1.0 + 1e-8) + 1e-12;
}

dirac_status make_cheb(double c0, double half, double dt, double shift, ChebParams& cp) {
  const double R = half * dt;
  if (!(R > 0.0) || R > 90.0)
    return fail(DIRAC_EINVAL, "dt * ||H|| = %.3g outside (0, 90]: take smaller steps", R);
  std::vector<double> J = bessel_j(CHEB_MAX, R);
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

// Launch with programmatic stream serialisation: the kernel may be scheduled
// while the previous kernel in the stream finishes; it waits for it (and sees
// its writes) at its griddepcontrol.wait.
// DIRAC_NO_PDL=1 in the environment turns the overlap off (debugging aid).
bool pdl_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("DIRAC_NO_PDL");
    return !(v && v[0] == '1');
  }();
  return on;
}

template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Persistent launch: as many CTAs as fit on the GPU at once (never more than
// there are tiles); each CTA walks the tiles with a grid stride.
template <class S, int R, bool D, bool V, bool Q64>
cudaError_t launch_pass_t(const PassParams& p, int n_sm, cudaStream_t s) {
  static int occ = 0;
  if (occ == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lanczos_pass<S, R, D, V, Q64>, NTP, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
  }
  // FP32 (memory-bound): equal work per CTA, T = ceil(tiles / resident CTAs)
  // tiles each; FP64 (FP64-pipe-bound): fill every slot to hide latency
  const int slots = std::max(1, n_sm * occ);
  const int per = (p.ntiles + slots - 1) / slots;
  const int grid = sizeof(S) == sizeof(float) ? std::max(1, (p.ntiles + per - 1) / per)
                                              : std::max(1, std::min(p.ntiles, slots));
  return launch_pdl(lanczos_pass<S, R, D, V, Q64>, grid, NTP, s, p);
}

template <class S, bool Q64>
cudaError_t launch_pass_s(const dirac_ctx* c, const PassParams& p) {
  const bool d = c->boundary == DIRAC_DIRICHLET, v = c->has_v;
  if (c->order == 2) {
    if (d) return v ? launch_pass_t<S, 1, true, true, Q64>(p, c->n_sm, c->stream) : launch_pass_t<S, 1, true, false, Q64>(p, c->n_sm, c->stream);
    return v ? launch_pass_t<S, 1, false, true, Q64>(p, c->n_sm, c->stream) : launch_pass_t<S, 1, false, false, Q64>(p, c->n_sm, c->stream);
  }
  if (d) return v ? launch_pass_t<S, 2, true, true, Q64>(p, c->n_sm, c->stream) : launch_pass_t<S, 2, true, false, Q64>(p, c->n_sm, c->stream);
  return v ? launch_pass_t<S, 2, false, true, Q64>(p, c->n_sm, c->stream) : launch_pass_t<S, 2, false, false, Q64>(p, c->n_sm, c->stream);
}

// FP64 path: everything complex128.  Mixed path: passes 1 and 2 read the
// complex128 state as q^_1, later passes read complex64 basis vectors.
cudaError_t launch_pass(const dirac_ctx* c, const PassParams& p) {
  if (c->precision == DIRAC_FP64) return launch_pass_s<double, true>(c, p);
  if (p.pass <= 2) return launch_pass_s<float, true>(c, p);
  return launch_pass_s<float, false>(c, p);
}

size_t site_bytes(int precision) { return precision == DIRAC_FP64 ? sizeof(double4_32a) : sizeof(float4); }

bool aligned32(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 31u) == 0; }

enum { KIND_PASS = 0, KIND_RECOMBINE = 1, KIND_END = -1 };

// with profiling on, an event is recorded before every launch and after each step
cudaError_t mark(dirac_ctx* c, int kind) {
  if (!c->profiling) return cudaSuccess;
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return e;
    c->ev_pool.push_back(ev);
    c->ev_kind.push_back(kind);
  }
  c->ev_kind[c->ev_used] = kind;
  return cudaEventRecord(c->ev_pool[c->ev_used++], c->stream);
}

// enqueue one full time step on psi (device)
dirac_status enqueue_step(dirac_ctx* c, vec4* psi, double dt, int m, double tol) {
  PassParams p;
  std::memset(&p, 0, sizeof(p));
  double c0, half;
  spectral_interval(c, c0, half);
  dirac_status s = make_cheb(c0, half, dt, c->shift, p.cheb);
  if (s != DIRAC_OK) return s;
  const double kfac = (c->order == 2) ? 2.0 : 12.0;
  p.psi = psi;
  p.V = c->has_v ? c->V : nullptr;
  p.st = c->st;
  p.partials = c->partials;
  p.nx = c->nx;
  p.ny = c->ny;
  p.tiles_x = c->grid.x;
  p.ntiles = c->grid.x * c->grid.y;
  p.m = m;
  p.kx = c->c / (kfac * c->dx);
  p.ky = c->c / (kfac * c->dy);
  p.mcc = c->mass * c->c * c->c;
  p.cAx = c->c * c->ax;   // electron: p - qA = p + A
  p.cAy = c->c * c->ay;
  p.shift = c->shift;
  p.dt = dt;
  p.tol = tol;
  p.kxf = (float)p.kx; p.kyf = (float)p.ky; p.cAxf = (float)p.cAx; p.cAyf = (float)p.cAy;
  p.probe_coef = make_coef(1.0, 0.0, 0.0, p.mcc - p.shift, -p.mcc - p.shift);
  const long long n = c->n_sites;
  const size_t sb = site_bytes(c->precision);
  char* basis = static_cast<char*>(c->basis);
  if (c->need_probe) {
    p.pass = 1;
    p.probe = 1;
    CUDA_TRY(mark(c, KIND_PASS));
    CUDA_TRY(launch_pass(c, p));
    ++c->launches;
    p.probe = 0;
    c->need_probe = false;
  }
  for (int i = 1; i <= m; ++i) {
    p.pass = i;
    p.y_prev = (i >= 2) ? c->ybuf[(i - 1) & 1] : nullptr;
    p.q_prev = (i == 2) ? (const void*)psi : (i >= 3 ? (const void*)(basis + (size_t)(i - 3) * n * sb) : nullptr);
    p.q_out = (i >= 2) ? (void*)(basis + (size_t)(i - 2) * n * sb) : nullptr;
    p.y_out = (i < m) ? c->ybuf[i & 1] : nullptr;
    CUDA_TRY(mark(c, KIND_PASS));
    CUDA_TRY(launch_pass(c, p));
    ++c->launches;
  }
  const int rb = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)c->n_sm * 8));
  CUDA_TRY(mark(c, KIND_RECOMBINE));
  if (c->precision == DIRAC_FP64)
    CUDA_TRY(launch_pdl(recombine, rb, 256, c->stream, psi, static_cast<const vec4*>(c->basis), n, c->st));
  else
    CUDA_TRY(launch_pdl(recombine_mixed, rb, 256, c->stream, psi, static_cast<const float4*>(c->basis), n, c->st));
  ++c->launches;
  CUDA_TRY(mark(c, KIND_END));
  return DIRAC_OK;
}

dirac_status read_state(dirac_ctx* c, dirac_step_info* info) {
  CUDA_TRY(cudaMemcpyAsync(c->st_host, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  const DevState& h = *c->st_host;
  if (h.error) {
    const int zero[2] = {0, 0};
    CUDA_TRY(cudaMemcpyAsync(&c->st->stopped, &zero[0], sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(&c->st->error, &zero[1], sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->need_probe = true;
    return fail(DIRAC_ENONFINITE, "non-finite value in a Lanczos reduction; psi left unchanged");
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->k_used = h.k_used;
    info->breakdown = h.breakdown;
    info->err_est = h.err_est;
    info->cum_err = h.cum_err;
    info->norm = h.psi_norm;
    info->energy = h.energy;
    for (int j = 0; j < h.k_used && j < DIRAC_KRYLOV_MAX; ++j) {
      info->alpha[j] = h.alpha[j + 1];
      info->beta[j] = h.beta[j + 1];
    }
  }
  return DIRAC_OK;
}

dirac_status check_step_args(dirac_ctx* c, const void* psi, double dt, int m, double tol, bool device) {
  if (!c) return fail(DIRAC_EINVAL, "null context");
  if (!c->fields_set) return fail(DIRAC_ESTATE, "dirac_set_fields must be called before stepping");
  if (!psi) return fail(DIRAC_EINVAL, "null psi");
  if (device && !aligned32(psi)) return fail(DIRAC_EINVAL, "psi must be 32-byte aligned");
  if (m < 1 || m > c->m_max) return fail(DIRAC_EINVAL, "m = %d outside 1..m_max = %d", m, c->m_max);
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(DIRAC_EINVAL, "dt must be finite and > 0");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(DIRAC_EINVAL, "tol must be finite and >= 0");
  return DIRAC_OK;
}

dirac_status run_steps(dirac_ctx* c, vec4* psi, int nsteps, double dt, int m, double tol,
                       const double* a_xy) {
  for (int n = 0; n < nsteps; ++n) {
    if (a_xy) {
      if (!std::isfinite(a_xy[2 * n]) || !std::isfinite(a_xy[2 * n + 1]))
        return fail(DIRAC_EINVAL, "non-finite vector potential at step %d", n);
      c->ax = a_xy[2 * n];
      c->ay = a_xy[2 * n + 1];
    }
    dirac_status s = enqueue_step(c, psi, dt, m, tol);
    if (s != DIRAC_OK) return s;
  }
  return DIRAC_OK;
}

__global__ void to_float_kernel(const double* in, float* out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

__global__ void minmax_kernel(const double* v, long long n, double* out) {
  __shared__ double smin[256], smax[256];
  double lo = 1e308, hi = -1e308;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = v[i];
    lo = fmin(lo, x);
    hi = fmax(hi, x);
    if (!isfinite(x)) { lo = -INFINITY; hi = INFINITY; }
  }
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
  if (nx < 1 || ny < 1) return fail(DIRAC_EINVAL, "grid %d x %d must be at least 1 x 1", nx, ny);
  if (!(dx > 0) || !(dy > 0) || !std::isfinite(dx) || !std::isfinite(dy))
    return fail(DIRAC_EINVAL, "dx, dy must be finite and > 0");
  if (!(c > 0) || !std::isfinite(c)) return fail(DIRAC_EINVAL, "c must be finite and > 0");
  if (!(mass >= 0) || !std::isfinite(mass)) return fail(DIRAC_EINVAL, "mass must be finite and >= 0");
  if (stencil_order != 2 && stencil_order != 4) return fail(DIRAC_EINVAL, "stencil_order must be 2 or 4");
  if (boundary != DIRAC_PERIODIC && boundary != DIRAC_DIRICHLET) return fail(DIRAC_EINVAL, "bad boundary");
  if (precision != DIRAC_FP64 && precision != DIRAC_MIXED)
    return fail(DIRAC_EINVAL, "precision must be DIRAC_FP64 or DIRAC_MIXED");
  if (m_max < 1 || m_max > DIRAC_KRYLOV_MAX) return fail(DIRAC_EINVAL, "m_max must be 1..%d", DIRAC_KRYLOV_MAX);
  const long long n = (long long)nx * ny;
  if (n > (1LL << 31)) return fail(DIRAC_EINVAL, "grid too large");

  dirac_ctx* ctx = new (std::nothrow) dirac_ctx;
  if (!ctx) return fail(DIRAC_ENOMEM, "host allocation failed");
  ctx->nx = nx; ctx->ny = ny; ctx->dx = dx; ctx->dy = dy; ctx->mass = mass; ctx->c = c;
  ctx->order = stencil_order; ctx->boundary = boundary; ctx->precision = precision;
  ctx->m_max = m_max; ctx->stream = (cudaStream_t)cuda_stream; ctx->n_sites = n;
  ctx->grid = dim3((nx + TILE - 1) / TILE, (ny + TILE - 1) / TILE);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, dev);
  const size_t vb = (size_t)n * site_bytes(precision);
  const int nbasis = std::max(1, m_max - 1);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->basis, vb * nbasis);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->ybuf[0], vb);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->ybuf[1], vb);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->st, sizeof(DevState));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->partials, sizeof(double) * 3 * (size_t)ctx->grid.x * ctx->grid.y);
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->st_host, sizeof(DevState));
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->st, 0, sizeof(DevState), ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    const bool oom = (e == cudaErrorMemoryAllocation);
    dirac_destroy(ctx);
    return fail(oom ? DIRAC_ENOMEM : DIRAC_ECUDA, "create: %s", cudaGetErrorString(e));
  }
  *out = ctx;
  return DIRAC_OK;
}

void dirac_destroy(dirac_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  for (cudaEvent_t ev : ctx->ev_pool) cudaEventDestroy(ev);
  cudaFree(ctx->basis);
  cudaFree(ctx->ybuf[0]);
  cudaFree(ctx->ybuf[1]);
  cudaFree(ctx->psi_own);
  cudaFree(ctx->V);
  cudaFree(ctx->st);
  cudaFree(ctx->partials);
  cudaFreeHost(ctx->st_host);
  delete ctx;
}

dirac_status dirac_set_stream(dirac_ctx* ctx, void* cuda_stream) {
  if (!ctx) return fail(DIRAC_EINVAL, "null context");
  if ((cudaStream_t)cuda_stream != ctx->stream) {
    // order the new stream after everything already queued on the old one
    cudaEvent_t ev;
    CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CUDA_TRY(cudaEventRecord(ev, ctx->stream));
    CUDA_TRY(cudaStreamWaitEvent((cudaStream_t)cuda_stream, ev, 0));
    CUDA_TRY(cudaEventDestroy(ev));
    ctx->stream = (cudaStream_t)cuda_stream;
  }
  return DIRAC_OK;
}

dirac_status dirac_set_fields(dirac_ctx* ctx, const double* V_dev, double A_x, double A_y,
                              double energy_shift) {
  if (!ctx) return fail(DIRAC_EINVAL, "null context");
  if (!std::isfinite(A_x) || !std::isfinite(A_y) || !std::isfinite(energy_shift))
    return fail(DIRAC_EINVAL, "non-finite field scalar");
  if (V_dev) {
    const bool f32 = ctx->precision != DIRAC_FP64;
    if (!ctx->V) CUDA_TRY(cudaMalloc(&ctx->V, (f32 ? sizeof(float) : sizeof(double)) * ctx->n_sites));
    if (f32) {
      to_float_kernel<<<256, 256, 0, ctx->stream>>>(V_dev, static_cast<float*>(ctx->V), ctx->n_sites);
      ++ctx->launches;
      CUDA_TRY(cudaGetLastError());
    } else {
      CUDA_TRY(cudaMemcpyAsync(ctx->V, V_dev, sizeof(double) * ctx->n_sites, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    double* mm = nullptr;
    CUDA_TRY(cudaMalloc(&mm, 2 * sizeof(double)));
    minmax_kernel<<<1, 256, 0, ctx->stream>>>(V_dev, ctx->n_sites, mm);
    ++ctx->launches;
    double h[2];
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, mm, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(mm);
    if (e != cudaSuccess) return fail(DIRAC_ECUDA, "set_fields: %s", cudaGetErrorString(e));
    if (!std::isfinite(h[0]) || !std::isfinite(h[1])) return fail(DIRAC_EINVAL, "V has non-finite entries");
    ctx->vmin = h[0];
    ctx->vmax = h[1];
    ctx->has_v = true;
  } else {
    ctx->has_v = false;
    ctx->vmin = ctx->vmax = 0.0;
  }
  ctx->ax = A_x;
  ctx->ay = A_y;
  ctx->shift = energy_shift;
  ctx->fields_set = true;
  ctx->need_probe = true;
  return DIRAC_OK;
}

dirac_status dirac_set_vector_potential(dirac_ctx* ctx, double A_x, double A_y) {
  if (!ctx) return fail(DIRAC_EINVAL, "null context");
  if (!std::isfinite(A_x) || !std::isfinite(A_y)) return fail(DIRAC_EINVAL, "non-finite vector potential");
  ctx->ax = A_x;
  ctx->ay = A_y;
  return DIRAC_OK;
}

dirac_status dirac_lanczos_step(dirac_ctx* ctx, void* psi_dev, double dt, int m, double tol,
                                dirac_step_info* info) {
  return dirac_lanczos_steps(ctx, psi_dev, 1, dt, m, tol, nullptr, info);
}

dirac_status dirac_lanczos_steps(dirac_ctx* ctx, void* psi_dev, int nsteps, double dt, int m,
                                 double tol, const double* A_xy_host, dirac_step_info* info) {
  dirac_status s = check_step_args(ctx, psi_dev, dt, m, tol, true);
  if (s != DIRAC_OK) return s;
  if (nsteps < 0) return fail(DIRAC_EINVAL, "nsteps < 0");
  s = run_steps(ctx, (vec4*)psi_dev, nsteps, dt, m, tol, A_xy_host);
  if (s != DIRAC_OK) return s;
  if (info) return read_state(ctx, info);
  return DIRAC_OK;
}

dirac_status dirac_propagate_host(dirac_ctx* ctx, void* psi_host, int nsteps, double dt, int m,
                                  double tol, const double* A_xy_host, dirac_step_info* info) {
  dirac_status s = check_step_args(ctx, psi_host, dt, m, tol, false);
  if (s != DIRAC_OK) return s;
  if (nsteps < 0) return fail(DIRAC_EINVAL, "nsteps < 0");
  const size_t bytes = (size_t)ctx->n_sites * sizeof(vec4);
  if (!ctx->psi_own) CUDA_TRY(cudaMalloc(&ctx->psi_own, bytes));
  CUDA_TRY(cudaMemcpyAsync(ctx->psi_own, psi_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
  s = run_steps(ctx, ctx->psi_own, nsteps, dt, m, tol, A_xy_host);
  if (s != DIRAC_OK) return s;
  CUDA_TRY(cudaMemcpyAsync(psi_host, ctx->psi_own, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  return read_state(ctx, info);
}

dirac_status dirac_sync(dirac_ctx* ctx) {
  if (!ctx) return fail(DIRAC_EINVAL, "null context");
  return read_state(ctx, nullptr);
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

long long dirac_kernel_launches(const dirac_ctx* ctx) { return ctx ? ctx->launches : 0; }

dirac_status dirac_profile_enable(dirac_ctx* ctx, int enable) {
  if (!ctx) return fail(DIRAC_EINVAL, "null context");
  ctx->profiling = enable != 0;
  return DIRAC_OK;
}

dirac_status dirac_profile_read(dirac_ctx* ctx, double* ms, long long* launches) {
  if (!ctx || !ms || !launches) return fail(DIRAC_EINVAL, "null argument");
  for (int k = 0; k < DIRAC_KERNEL_KINDS; ++k) { ms[k] = 0.0; launches[k] = 0; }
  if (ctx->ev_used > 0) CUDA_TRY(cudaEventSynchronize(ctx->ev_pool[ctx->ev_used - 1]));
  for (size_t j = 0; j + 1 < ctx->ev_used; ++j) {
    const int k = ctx->ev_kind[j];
    if (k < 0) continue;
    float t = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&t, ctx->ev_pool[j], ctx->ev_pool[j + 1]));
    ms[k] += t;
    launches[k] += 1;
  }
  ctx->ev_used = 0;
  return DIRAC_OK;
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
// step keeps its whole workspace (scalar block, per-CTA partial sums, the two
// y^ fields and the Krylov basis) in one file-scope device array of fixed
// size, shared by every call in the process, and calls no cudaMalloc,
// cudaFree or other allocating routine (host or device).
// ===========================================================================
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 8u << 20;   // 8 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::atomic<void*> g_noalloc_ptr[NOALLOC_MAX_DEVICES];

// Device address of the scratch array on the current device.  In host code
// `g_noalloc_scratch` names a host-side shadow, not device memory, so the
// address is looked up once per device (with that device current).
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

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

// Chebyshev coefficients as make_cheb, with stack storage only.
dirac_status noalloc_cheb(double c0, double half, double dt, double shift, ChebParams& cp) {
  const double R = half * dt;
  if (!(R > 0.0) || R > 90.0)
    return fail(DIRAC_EINVAL, "dt * ||H|| = %.3g outside (0, 90]: take smaller steps", R);
  constexpr int NJ = 512;
  double j[NJ + 2];
  const int start = 2 * ((std::max(CHEB_MAX, (int)R) + 40 + (int)std::sqrt(40.0 * std::max(R, 1.0))) / 2);
  if (start > NJ) return fail(DIRAC_EINVAL, "dt too large");
  for (int k = 0; k <= start + 1; ++k) j[k] = 0.0;
  j[start] = 1e-300;
  for (int k = start; k >= 1; --k) {
    j[k - 1] = (2.0 * k / R) * j[k] - j[k + 1];
    if (std::fabs(j[k - 1]) > 1e250)
      for (int t = k - 1; t <= start; ++t) j[t] *= 1e-250;
  }
  double norm = j[0];
  for (int k = 2; k <= start; k += 2) norm += 2.0 * j[k];
  int n = 2;
  for (int k = 0; k < CHEB_MAX; ++k)
    if (std::fabs(j[k] / norm) > 1e-18 || k <= (int)R + 1) n = k + 1;
  if (n >= CHEB_MAX) return fail(DIRAC_EINVAL, "Chebyshev expansion needs more than %d terms", CHEB_MAX);
  cp.n = std::max(n, 2);
  cp.c0 = c0;
  cp.inv_half = 1.0 / half;
  const double ph = -(c0 + shift) * dt;
  cp.ph_re = std::cos(ph);
  cp.ph_im = std::sin(ph);
  for (int k = 0; k < CHEB_MAX; ++k) {
    const double a = (k == 0 ? 1.0 : 2.0) * (k < cp.n ? j[k] / norm : 0.0);
    switch (k & 3) {
      case 0: cp.cr[k] = a;  cp.ci[k] = 0.0; break;
      case 1: cp.cr[k] = 0.0; cp.ci[k] = -a; break;
      case 2: cp.cr[k] = -a; cp.ci[k] = 0.0; break;
      default: cp.cr[k] = 0.0; cp.ci[k] = a; break;
    }
  }
  return DIRAC_OK;
}

}  // namespace

extern "C" size_t dirac_noalloc_scratch_bytes(void) { return NOALLOC_SCRATCH_BYTES; }

extern "C" dirac_status dirac_lanczos_step_noalloc(const dirac_problem* pb, void* psi_dev, double dt,
                                                   int m, double tol, void* cuda_stream,
                                                   dirac_step_info* info) {
  if (!pb || !psi_dev) return fail(DIRAC_EINVAL, "null argument");
  const int nx = pb->nx, ny = pb->ny;
  if (nx < 1 || ny < 1) return fail(DIRAC_EINVAL, "grid %d x %d must be at least 1 x 1", nx, ny);
  if (!(pb->dx > 0) || !(pb->dy > 0) || !std::isfinite(pb->dx) || !std::isfinite(pb->dy))
    return fail(DIRAC_EINVAL, "dx, dy must be finite and > 0");
  if (!(pb->c > 0) || !std::isfinite(pb->c)) return fail(DIRAC_EINVAL, "c must be finite and > 0");
  if (!(pb->mass >= 0) || !std::isfinite(pb->mass)) return fail(DIRAC_EINVAL, "mass must be finite and >= 0");
  if (pb->stencil_order != 2 && pb->stencil_order != 4) return fail(DIRAC_EINVAL, "stencil_order must be 2 or 4");
  if (pb->boundary != DIRAC_PERIODIC && pb->boundary != DIRAC_DIRICHLET) return fail(DIRAC_EINVAL, "bad boundary");
  if (!std::isfinite(pb->A_x) || !std::isfinite(pb->A_y) || !std::isfinite(pb->energy_shift))
    return fail(DIRAC_EINVAL, "non-finite field scalar");
  if (m < 1 || m > DIRAC_KRYLOV_MAX) return fail(DIRAC_EINVAL, "m = %d outside 1..%d", m, DIRAC_KRYLOV_MAX);
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(DIRAC_EINVAL, "dt must be finite and > 0");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(DIRAC_EINVAL, "tol must be finite and >= 0");
  if (!aligned32(psi_dev)) return fail(DIRAC_EINVAL, "psi must be 32-byte aligned");

  // scratch layout: DevState | partials | y^[2] | basis[m-1]
  const long long n = (long long)nx * ny;
  const dim3 grid((nx + TILE - 1) / TILE, (ny + TILE - 1) / TILE);
  const size_t ncta = (size_t)grid.x * grid.y;
  const size_t field = round256((size_t)n * sizeof(vec4));
  const size_t off_part = round256(sizeof(DevState));
  const size_t off_y = off_part + round256(3 * sizeof(double) * ncta);
  const size_t off_basis = off_y + 2 * field;
  const size_t need = off_basis + (size_t)std::max(1, m - 1) * field;
  if (need > NOALLOC_SCRATCH_BYTES)
    return fail(DIRAC_EINVAL, "grid %d x %d with m = %d needs %zu bytes of scratch; the static scratch "
                "holds %zu bytes (use dirac_create for larger problems)", nx, ny, m, need,
                NOALLOC_SCRATCH_BYTES);
  unsigned char* base = nullptr;
  dirac_status s = noalloc_scratch(&base);
  if (s != DIRAC_OK) return s;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  DevState* st = reinterpret_cast<DevState*>(base);
  double* partials = reinterpret_cast<double*>(base + off_part);
  vec4* ybuf[2] = {reinterpret_cast<vec4*>(base + off_y), reinterpret_cast<vec4*>(base + off_y + field)};
  vec4* basis = reinterpret_cast<vec4*>(base + off_basis);
  vec4* psi = static_cast<vec4*>(psi_dev);

  // the scratch keeps the previous call's contents: restart the scalar block
  CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(DevState), stream));

  // spectral interval of H - s (needs the range of V: read back two doubles)
  double vmin = 0.0, vmax = 0.0;
  if (pb->V_dev) {
    double* mm = partials;   // two doubles of scratch, rewritten by the passes later
    minmax_kernel<<<1, 256, 0, stream>>>(pb->V_dev, n, mm);
    CUDA_TRY(cudaGetLastError());
    double h[2];
    CUDA_TRY(cudaMemcpyAsync(h, mm, sizeof(h), cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    if (!std::isfinite(h[0]) || !std::isfinite(h[1])) return fail(DIRAC_EINVAL, "V has non-finite entries");
    vmin = h[0];
    vmax = h[1];
  }
  double pf = 1.0;
  if (pb->stencil_order == 4) {
    const double cs = 1.0 - std::sqrt(6.0) / 2.0;
    pf = std::sqrt(1.0 - cs * cs) * (4.0 - cs) / 3.0;
  }
  const double px = pf / pb->dx + std::fabs(pb->A_x), py = pf / pb->dy + std::fabs(pb->A_y);
  const double mc2 = pb->mass * pb->c * pb->c;
  const double emax = std::sqrt(mc2 * mc2 + pb->c * pb->c * (px * px + py * py));
  const double c0 = 0.5 * (vmin + vmax) - pb->energy_shift;
  const double half = (emax + 0.5 * (vmax - vmin)) * (1.0 + 1e-8) + 1e-12;

  PassParams p;
  std::memset(&p, 0, sizeof(p));
  s = noalloc_cheb(c0, half, dt, pb->energy_shift, p.cheb);
  if (s != DIRAC_OK) return s;
  const double kfac = (pb->stencil_order == 2) ? 2.0 : 12.0;
  p.psi = psi;
  p.V = pb->V_dev;
  p.st = st;
  p.partials = partials;
  p.nx = nx;
  p.ny = ny;
  p.tiles_x = grid.x;
  p.ntiles = grid.x * grid.y;
  p.m = m;
  p.kx = pb->c / (kfac * pb->dx);
  p.ky = pb->c / (kfac * pb->dy);
  p.mcc = mc2;
  p.cAx = pb->c * pb->A_x;
  p.cAy = pb->c * pb->A_y;
  p.shift = pb->energy_shift;
  p.dt = dt;
  p.tol = tol;
  p.kxf = (float)p.kx; p.kyf = (float)p.ky; p.cAxf = (float)p.cAx; p.cAyf = (float)p.cAy;
  p.probe_coef = make_coef(1.0, 0.0, 0.0, p.mcc - p.shift, -p.mcc - p.shift);

  int n_sm = 0, dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  dirac_ctx view;   // launch configuration only; owns nothing
  view.nx = nx; view.ny = ny; view.order = pb->stencil_order; view.boundary = pb->boundary;
  view.has_v = pb->V_dev != nullptr; view.grid = grid; view.stream = stream;
  view.precision = DIRAC_FP64; view.n_sm = n_sm;
  p.pass = 1;
  p.probe = 1;
  CUDA_TRY(launch_pass(&view, p));
  p.probe = 0;
  for (int i = 1; i <= m; ++i) {
    p.pass = i;
    p.y_prev = (i >= 2) ? ybuf[(i - 1) & 1] : nullptr;
    p.q_prev = (i == 2) ? (const void*)psi : (i >= 3 ? (const void*)(basis + (size_t)(i - 3) * n) : nullptr);
    p.q_out = (i >= 2) ? (void*)(basis + (size_t)(i - 2) * n) : nullptr;
    p.y_out = (i < m) ? (void*)ybuf[i & 1] : nullptr;
    CUDA_TRY(launch_pass(&view, p));
  }
  const int rb = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)n_sm * 8));
  CUDA_TRY(launch_pdl(recombine, rb, 256, stream, psi, (const vec4*)basis, n, st));

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
