// dirac_adjoint.cu -- gradients of a final-state observable through the
// time-discrete propagation psi_{n+1} = exp(-i H_n dt) psi_n (Sec. 4, Eq. 16
// and 17) with respect to the potential V on the grid and the step-mean
// vector potential A_n of every step.
//
// Adjoint (reverse) sweep.  With lambda_N = dL/d conj(psi_N) and
// lambda_n = exp(+i H_n dt) lambda_{n+1} (a backward Lanczos step), a
// parameter theta with dH_n/dtheta = E contributes
//     dL/dtheta += 2 dt Im int_0^1 <a(s), E b(s)> ds,
//     a(s) = exp(+i H_n dt s) lambda_{n+1},  b(s) = exp(-i H_n dt (1-s)) psi_n,
// the Frechet derivative of the exponential paired with the adjoint.  In the
// Krylov spaces of psi_n (basis Q, matrix T) and of lambda_{n+1} (Q', T'):
//     a(s) = ||lambda|| Q' conj(e(s)),  e(s) = exp(-i (T' + s_h) dt s) e_1,
//     b(s) = ||psi||    Q  v(s),        v(s) = exp(-i (T + s_h) dt (1-s)) e_1,
// so the integral is sum_jl M_jl <Q'_j, E Q_l> with the small matrix
//     M_jl = ||lambda|| ||psi|| int_0^1 e_j(s) v_l(s) ds,
// evaluated by Gauss-Legendre quadrature in s with the device Chebyshev
// exponential at every node (the node count makes the quadrature error of
// the fastest oscillation, 2 |dt| times the half width of the spectral
// interval, negligible against rounding).  E is the identity on one site for
// V (dL/dV(x) is then a per-site bilinear form in the two bases) and
// c sigma_x, c sigma_y for A_x, A_y (the same bilinear form, summed).
//
// The forward states are kept every `checkpoint_every` steps and recomputed
// segment by segment on the way back; each backward step re-runs the forward
// step from the stored psi_n (its Krylov basis is needed) and the backward
// step of lambda in a second context.  All sums are in a fixed order.
#include "dirac.h"
#include "dirac_internal.h"
#include "dirac_kernels.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace dirac {
namespace adj {

using v4 = double4_32a;
constexpr int QMAX = 32;   // Gauss-Legendre nodes at most (one warp each)

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// per-block sum of v into out[blockIdx.x] (fixed order)
__device__ void block_partial2(double a, double b, double* out) {
  __shared__ double ra[32], rb[32];
  a = wsum(a);
  b = wsum(b);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) { ra[warp] = a; rb[warp] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < nw; ++w) { sa += ra[w]; sb += rb[w]; }
    out[2 * blockIdx.x] = sa;
    out[2 * blockIdx.x + 1] = sb;
  }
}

// ---------------------------------------------------------------------------
// observables: L and lambda_N = dL/d conj(psi_N)
// ---------------------------------------------------------------------------
struct PxArgs {
  int nx, ny, order, diri;
  double inv_h;          // 1 / (2 dx) (order 2) or 1 / (12 dx) (order 4)
  double w;              // dx dy
  const v4* psi;
  v4* lam;
  double* part;          // per block: Re <psi, p_x psi>, 0
};

__device__ __forceinline__ v4 site_or_zero(const v4* f, int x, int y, int nx, int ny, bool diri) {
  if (diri) {
    if (x < 0 || x >= nx) { v4 z; z.x = z.y = z.z = z.w = 0.0; return z; }
  } else {
    x = ((x % nx) + nx) % nx;
  }
  return f[(size_t)y * nx + x];
}

// lambda = w p_x psi with p_x = -i D_x (central difference); partial sums of
// Re <psi, p_x psi>
__global__ void __launch_bounds__(256) adj_obs_px(const PxArgs a) {
  double acc = 0.0;
  const long long n = (long long)a.nx * a.ny;
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(s % a.nx), y = (int)(s / a.nx);
    const bool d = a.diri != 0;
    const v4 p1 = site_or_zero(a.psi, x + 1, y, a.nx, a.ny, d), m1 = site_or_zero(a.psi, x - 1, y, a.nx, a.ny, d);
    double D[4] = {p1.x - m1.x, p1.y - m1.y, p1.z - m1.z, p1.w - m1.w};
    if (a.order == 4) {
      const v4 p2 = site_or_zero(a.psi, x + 2, y, a.nx, a.ny, d), m2 = site_or_zero(a.psi, x - 2, y, a.nx, a.ny, d);
      D[0] = fma(8.0, D[0], m2.x - p2.x);
      D[1] = fma(8.0, D[1], m2.y - p2.y);
      D[2] = fma(8.0, D[2], m2.z - p2.z);
      D[3] = fma(8.0, D[3], m2.w - p2.w);
    }
    // p = -i D: (re, im) -> (D.im, -D.re)
    v4 p;
    p.x = D[1] * a.inv_h; p.y = -D[0] * a.inv_h; p.z = D[3] * a.inv_h; p.w = -D[2] * a.inv_h;
    const v4 c = a.psi[s];
    acc = fma(c.x, p.x, fma(c.y, p.y, fma(c.z, p.z, fma(c.w, p.w, acc))));
    v4 l;
    l.x = a.w * p.x; l.y = a.w * p.y; l.z = a.w * p.z; l.w = a.w * p.w;
    a.lam[s] = l;
  }
  block_partial2(acc, 0.0, a.part);
}

// partial sums of <phi, psi>
__global__ void __launch_bounds__(256) adj_obs_dot(const v4* phi, const v4* psi, long long n, double* part) {
  double re = 0.0, im = 0.0;
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (long long)gridDim.x * blockDim.x) {
    const v4 f = phi[s], p = psi[s];
    re = fma(f.x, p.x, fma(f.y, p.y, fma(f.z, p.z, fma(f.w, p.w, re))));
    im = fma(f.x, p.y, fma(-f.y, p.x, fma(f.z, p.w, fma(-f.w, p.z, im))));
  }
  block_partial2(re, im, part);
}

// fixed-order sum of the block partials: out[0] = loss, out[1..2] = the
// complex factor of lambda (proj: w amp), by one warp
__global__ void adj_obs_finish(const double* part, int nblk, int kind, double w, double* out) {
  double re = 0.0, im = 0.0;
  for (int b = threadIdx.x; b < nblk; b += 32) { re += part[2 * b]; im += part[2 * b + 1]; }
  re = wsum(re);
  im = wsum(im);
  if (threadIdx.x != 0) return;
  if (kind == DIRAC_OBS_PX) {
    out[0] = w * re;
    out[1] = out[2] = 0.0;
  } else {
    const double ar = w * re, ai = w * im;   // amp = w <phi, psi>
    out[0] = ar * ar + ai * ai;
    out[1] = w * ar;                          // lambda = w amp phi
    out[2] = w * ai;
  }
}

__global__ void __launch_bounds__(256) adj_obs_scale(const v4* phi, long long n, const double* fac, v4* lam) {
  const double fr = fac[1], fi = fac[2];
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (long long)gridDim.x * blockDim.x) {
    const v4 f = phi[s];
    v4 l;
    l.x = fr * f.x - fi * f.y; l.y = fr * f.y + fi * f.x;
    l.z = fr * f.z - fi * f.w; l.w = fr * f.w + fi * f.z;
    lam[s] = l;
  }
}

// ---------------------------------------------------------------------------
// the small matrix M (scaled for the unnormalised bases): one warp per node
// ---------------------------------------------------------------------------
struct MArgs {
  const DevState* fwd;        // Krylov space of psi_n: T, norms, k
  const DevState* bwd;        // of lambda_{n+1}
  const ChebParams* cp;       // cp[r]: exp(-i (T + s_h) dt s_r) e_1; s_{R-1-r} = 1 - s_r
  const double* wq;           // quadrature weights on [0, 1]
  int R;
  double two_dt;              // 2 |dt|
  double2* M;                 // QMAX x KMAX, row j (adjoint basis), column l (forward basis)
};

__global__ void __launch_bounds__(QMAX * 32) adj_mmat(const MArgs a) {
  __shared__ double2 E[QMAX][KMAX], Vv[QMAX][KMAX];
  const int lane = threadIdx.x & 31, r = threadIdx.x >> 5;
  const int kf = a.fwd->k_used, kb = a.bwd->k_used;
  if (r < a.R) {
    // e(s_r) on T'
    {
      const DevState* st = a.bwd;
      const double aj = lane < kb ? st->alpha[lane + 1] : 0.0;
      const double bh = lane + 1 < kb ? st->beta[lane + 1] : 0.0;
      const double bl = __shfl_up_sync(0xffffffffu, bh, 1);
      double vr, vi;
      cheb_expm_e1(a.cp[r], kb, aj, bl, bh, vr, vi);
      E[r][lane] = make_double2(vr, vi);
    }
    // v(s_r) = exp(-i (T + s_h) dt (1 - s_r)) e_1 on T
    {
      const DevState* st = a.fwd;
      const double aj = lane < kf ? st->alpha[lane + 1] : 0.0;
      const double bh = lane + 1 < kf ? st->beta[lane + 1] : 0.0;
      const double bl = __shfl_up_sync(0xffffffffu, bh, 1);
      double vr, vi;
      cheb_expm_e1(a.cp[a.R - 1 - r], kf, aj, bl, bh, vr, vi);
      Vv[r][lane] = make_double2(vr, vi);
    }
  }
  __syncthreads();
  const double scale = a.two_dt * a.bwd->psi_norm * a.fwd->psi_norm;
  for (int t = threadIdx.x; t < QMAX * KMAX; t += blockDim.x) {
    const int j = t / KMAX, l = t % KMAX;
    double mr = 0.0, mi = 0.0;
    if (j < kb && l < kf) {
      for (int q = 0; q < a.R; ++q) {
        const double2 e = E[q][j], v = Vv[q][l];
        const double w = a.wq[q];
        mr = fma(w, e.x * v.x - e.y * v.y, mr);
        mi = fma(w, e.x * v.y + e.y * v.x, mi);
      }
      const double f = scale * a.bwd->inv_nu[j + 1] * a.fwd->inv_nu[l + 1];
      mr *= f;
      mi *= f;
    }
    a.M[t] = make_double2(mr, mi);
  }
}

// ---------------------------------------------------------------------------
// per-site contraction: with w_j = sum_l M_jl q^_l (each component),
//   dV(x) += Im sum_j conj(q^'_j) . w_j,   A_x: Im sum_j conj(q^'_j) . sigma_x w_j,
//   A_y: Im sum_j conj(q^'_j) . sigma_y w_j (summed over sites).
// JW lanes per site (lane j holds the adjoint basis index j).
// ---------------------------------------------------------------------------
struct CArgs {
  const DevState* fwd;
  const DevState* bwd;
  const v4* q1;               // psi_n  (q^_1 of the forward space)
  const v4* qf;               // forward basis q^_2 ..
  const v4* p1;               // lambda_{n+1}
  const v4* pb;               // backward basis
  const double2* M;
  long long n;
  double* gV;                 // += per site
  double* part;               // per block: (A_x, A_y) sums
};

template <int JW>
__global__ void __launch_bounds__(256) adj_contract(const CArgs a) {
  __shared__ double2 Ms[KMAX][KMAX];
  const int kf = a.fwd->k_used, kb = a.bwd->k_used;
  for (int t = threadIdx.x; t < KMAX * KMAX; t += blockDim.x) Ms[t / KMAX][t % KMAX] = a.M[t];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int grp = lane / JW, j = lane % JW;   // site slot in the warp, adjoint index
  constexpr int SPW = 32 / JW;                // sites per warp
  const long long warp_g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  double accx = 0.0, accy = 0.0;
  for (long long base = warp_g * SPW; base < a.n; base += nwarps * SPW) {
    const long long x = base + grp;
    const bool valid = x < a.n;
    // this lane's forward vector l = j and adjoint vector j at site x
    v4 ql, pj;
    ql.x = ql.y = ql.z = ql.w = 0.0;
    pj = ql;
    if (valid && j < kf) ql = (j == 0) ? a.q1[x] : a.qf[(size_t)(j - 1) * a.n + x];
    if (valid && j < kb) pj = (j == 0) ? a.p1[x] : a.pb[(size_t)(j - 1) * a.n + x];
    double ur = 0.0, ui = 0.0, dr = 0.0, di = 0.0;   // w_j (upper, lower)
    for (int l = 0; l < kf; ++l) {
      const int src = grp * JW + l;
      const double qx = __shfl_sync(0xffffffffu, ql.x, src), qy = __shfl_sync(0xffffffffu, ql.y, src);
      const double qz = __shfl_sync(0xffffffffu, ql.z, src), qw = __shfl_sync(0xffffffffu, ql.w, src);
      const double2 m = Ms[j < kb ? j : 0][l];
      ur = fma(m.x, qx, fma(-m.y, qy, ur));
      ui = fma(m.x, qy, fma(m.y, qx, ui));
      dr = fma(m.x, qz, fma(-m.y, qw, dr));
      di = fma(m.x, qw, fma(m.y, qz, di));
    }
    if (!(valid && j < kb)) { ur = ui = dr = di = 0.0; }
    // Im conj(p) . w for the identity, sigma_x (swap) and sigma_y (u' = -i d, d' = i u)
    const double dv = (pj.x * ui - pj.y * ur) + (pj.z * di - pj.w * dr);
    const double dax = (pj.x * di - pj.y * dr) + (pj.z * ui - pj.w * ur);
    const double day = -(pj.x * dr + pj.y * di) + (pj.z * ur + pj.w * ui);
    double sv = dv;
#pragma unroll
    for (int o = JW / 2; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
    if (valid && j == 0) a.gV[x] += sv;
    accx += dax;
    accy += day;
  }
  block_partial2(accx, accy, a.part);
}

// gA[n] = (c sum_blocks A_x, c sum_blocks A_y), one warp
__global__ void adj_finish_a(const double* part, int nblk, double c, double* gA_n) {
  double x = 0.0, y = 0.0;
  for (int b = threadIdx.x; b < nblk; b += 32) { x += part[2 * b]; y += part[2 * b + 1]; }
  x = wsum(x);
  y = wsum(y);
  if (threadIdx.x == 0) { gA_n[0] = c * x; gA_n[1] = c * y; }
}

// sums over blocks of bx x by sites (one thread per block)
__global__ void adj_pool(const double* gV, int nx, int ny, int bx, int by, double* out) {
  const int nbx = nx / bx, nby = ny / by;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nbx * nby) return;
  const int ix = t % nbx, iy = t / nbx;
  double s = 0.0;
  for (int yy = 0; yy < by; ++yy)
    for (int xx = 0; xx < bx; ++xx) s += gV[(size_t)(iy * by + yy) * nx + ix * bx + xx];
  out[t] = s;
}

// da_k = sum_n W[n][k] gA[n][0] (fixed order), one thread per k
__global__ void adj_coef(const double* W, const double* gA, int nsteps, int ncoef, double* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ncoef) return;
  double s = 0.0;
  for (int n = 0; n < nsteps; ++n) s = fma(W[(size_t)n * ncoef + k], gA[2 * n], s);
  out[k] = s;
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
};

struct CtxGuard {
  dirac_ctx* c = nullptr;
  ~CtxGuard() { if (c) dirac_destroy(c); }
};

#define ADJ_TRY(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return fail(DIRAC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define ADJ_CHECK(call)                                                                 \
  do {                                                                                  \
    dirac_status s_ = (call);                                                           \
    if (s_ != DIRAC_OK) return s_;                                                      \
  } while (0)

// Gauss-Legendre nodes x and weights w on [-1, 1] (Newton on P_R from the
// three-term recurrence)
void gauss_legendre(int R, std::vector<double>& x, std::vector<double>& w) {
  x.assign(R, 0.0);
  w.assign(R, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < R; ++i) {
    double z = std::cos(pi * (i + 0.75) / (R + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= R; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      // P_R = p1, P_{R-1} = p0
      dp = R * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// nodes needed so that Gauss-Legendre integrates exp(i omega s) on [0, 1]
// to ~1e-17 for |omega| <= omega_max: (omega/2)^(2R) / (2R)! < 1e-17
int quad_nodes(double omega_max) {
  for (int R = 4; R <= QMAX; ++R) {
    const double lg = 2.0 * R * std::log(std::max(omega_max, 1e-30) / 2.0) - std::lgamma(2.0 * R + 1.0);
    if (lg < std::log(1e-17)) return R;
  }
  return -1;
}

}  // namespace adj
}  // namespace dirac

using namespace dirac;
using namespace dirac::adj;

extern "C" {

dirac_status dirac_adjoint_gradient(dirac_ctx* ctx, const void* psi0_dev, int nsteps, double dt, int m,
                                    const double* A_xy_host, const dirac_adjoint_opts* opts,
                                    double* loss_out, void* psiN_dev, void* dV_dev, double* dA_host,
                                    double* da_host, dirac_adjoint_info* info) {
  dirac::TraceRange trace("dirac_adjoint_gradient");
  CtxView v;
  ADJ_CHECK(ctx_view(ctx, &v));
  if (!v.fields_set) return fail(DIRAC_ESTATE, "dirac_set_fields has not been called");
  if (v.precision != DIRAC_FP64) return fail(DIRAC_EINVAL, "the adjoint needs an FP64 context");
  if (!opts || !A_xy_host || !loss_out) return fail(DIRAC_EINVAL, "null argument");
  if (nsteps < 1) return fail(DIRAC_EINVAL, "nsteps must be >= 1");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(DIRAC_EINVAL, "dt must be finite and > 0");
  if (m < 1 || m > v.m_max) return fail(DIRAC_EINVAL, "m must be 1..m_max (%d)", v.m_max);
  if (opts->observable != DIRAC_OBS_PX && opts->observable != DIRAC_OBS_PROJ)
    return fail(DIRAC_EINVAL, "unknown observable");
  if (opts->observable == DIRAC_OBS_PROJ && !opts->phi_dev) return fail(DIRAC_EINVAL, "proj needs phi_dev");
  if (opts->checkpoint_every < 1) return fail(DIRAC_EINVAL, "checkpoint_every must be >= 1");
  const int bx = opts->block_x, by = opts->block_y;
  if (dV_dev && (bx < 1 || by < 1 || v.nx % bx || v.ny % by))
    return fail(DIRAC_EINVAL, "blocks %d x %d must tile the %d x %d grid", bx, by, v.nx, v.ny);
  if (da_host && (opts->n_coef < 1 || !opts->W_host)) return fail(DIRAC_EINVAL, "da needs n_coef and W_host");
  auto misaligned = [](const void* p) { return p && (reinterpret_cast<uintptr_t>(p) & 31u); };
  if (!psi0_dev || misaligned(psi0_dev) || misaligned(psiN_dev) || misaligned(opts->phi_dev))
    return fail(DIRAC_EINVAL, "state pointers must be non-null (psi0) and 32-byte aligned");
  for (int k = 0; k < 2 * nsteps; ++k)
    if (!std::isfinite(A_xy_host[k])) return fail(DIRAC_EINVAL, "non-finite vector potential");
  if (info) std::memset(info, 0, sizeof(*info));

  const long long n = (long long)v.nx * v.ny;
  const size_t vb = sizeof(v4) * (size_t)n;
  const int K = std::min(opts->checkpoint_every, nsteps);
  const int n_ckpt = (nsteps + K - 1) / K;
  cudaStream_t s = v.stream;

  // quadrature of the Frechet integral on the spectral interval of every H_n
  double axm = 0.0, aym = 0.0;
  for (int k = 0; k < nsteps; ++k) {
    axm = std::max(axm, std::fabs(A_xy_host[2 * k]));
    aym = std::max(aym, std::fabs(A_xy_host[2 * k + 1]));
  }
  double c0 = 0.0, half = 0.0;
  ADJ_CHECK(operator_interval(ctx, axm, aym, &c0, &half));
  const int R = quad_nodes(2.0 * half * dt);
  if (R < 0) return fail(DIRAC_EINVAL, "dt * ||H|| too large for the adjoint quadrature");
  std::vector<double> gx, gw;
  gauss_legendre(R, gx, gw);
  std::vector<ChebParams> hcp(R);
  std::vector<double> hw(R);
  for (int r = 0; r < R; ++r) {
    const double sr = 0.5 * (1.0 + gx[r]);            // node on [0, 1]
    hw[r] = 0.5 * gw[r];
    ADJ_CHECK(cheb_params(c0, half, dt * sr, v.shift, &hcp[r]));
  }
  // the nodes come in pairs s, 1 - s: cp[R-1-r] must be the partner of cp[r]
  for (int r = 0; r < R; ++r)
    if (std::fabs((0.5 * (1.0 + gx[r])) + (0.5 * (1.0 + gx[R - 1 - r])) - 1.0) > 1e-14)
      return fail(DIRAC_EINVAL, "quadrature nodes not symmetric");

  // memory
  size_t free_b = 0, total_b = 0;
  ADJ_TRY(cudaMemGetInfo(&free_b, &total_b));
  const size_t n_vec = (size_t)n_ckpt + K + 3;
  if (vb * n_vec + sizeof(double) * (size_t)n > free_b)
    return fail(DIRAC_ENOMEM, "adjoint needs %.3g GB, %.3g GB free", (vb * n_vec + 8.0 * n) / 1e9, free_b / 1e9);
  DevBuf vec_mem, small_mem;
  ADJ_TRY(cudaMalloc(&vec_mem.p, vb * n_vec));
  v4* ckpt = static_cast<v4*>(vec_mem.p);
  v4* seg = ckpt + (size_t)n_ckpt * n;
  v4* work = seg + (size_t)K * n;
  v4* lam = work + n;
  v4* lam1 = lam + n;
  const int nblk = 304;
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
  const size_t o_gV = take(sizeof(double) * (size_t)n);
  const size_t o_gA = take(sizeof(double) * 2 * (size_t)nsteps);
  const size_t o_part = take(sizeof(double) * 2 * nblk);
  const size_t o_obs = take(sizeof(double) * 4);
  const size_t o_M = take(sizeof(double2) * KMAX * KMAX);
  const size_t o_cp = take(sizeof(ChebParams) * R);
  const size_t o_w = take(sizeof(double) * R);
  const size_t o_W = take(sizeof(double) * (da_host ? (size_t)nsteps * opts->n_coef : 1));
  const size_t o_da = take(sizeof(double) * (da_host ? opts->n_coef : 1));
  ADJ_TRY(cudaMalloc(&small_mem.p, off));
  char* sb = static_cast<char*>(small_mem.p);
  double* gV = reinterpret_cast<double*>(sb + o_gV);
  double* gA = reinterpret_cast<double*>(sb + o_gA);
  double* part = reinterpret_cast<double*>(sb + o_part);
  double* obs = reinterpret_cast<double*>(sb + o_obs);
  double2* Mm = reinterpret_cast<double2*>(sb + o_M);
  ChebParams* dcp = reinterpret_cast<ChebParams*>(sb + o_cp);
  double* dw = reinterpret_cast<double*>(sb + o_w);
  ADJ_TRY(cudaMemsetAsync(gV, 0, sizeof(double) * (size_t)n, s));
  ADJ_TRY(cudaMemsetAsync(gA, 0, sizeof(double) * 2 * (size_t)nsteps, s));
  ADJ_TRY(cudaMemcpyAsync(dcp, hcp.data(), sizeof(ChebParams) * R, cudaMemcpyHostToDevice, s));
  ADJ_TRY(cudaMemcpyAsync(dw, hw.data(), sizeof(double) * R, cudaMemcpyHostToDevice, s));

  // the adjoint's own context: same operator and fields
  CtxGuard back;
  ADJ_CHECK(dirac_create(&back.c, v.nx, v.ny, v.dx, v.dy, v.mass, v.c, v.order, v.boundary, DIRAC_FP64, m,
                         (void*)s));
  ADJ_CHECK(dirac_set_fields(back.c, v.V, v.ax, v.ay, v.shift));
  CtxView vb_view;
  ADJ_CHECK(ctx_view(back.c, &vb_view));
  long long launches = 0;
  cudaEvent_t ev[3];
  for (auto& e : ev) ADJ_TRY(cudaEventCreate(&e));
  struct EvGuard {
    cudaEvent_t* e;
    ~EvGuard() { for (int i = 0; i < 3; ++i) cudaEventDestroy(e[i]); }
  } evg{ev};
  const long long l0 = *v.launches;

  // forward sweep with checkpoints
  ADJ_TRY(cudaEventRecord(ev[0], s));
  ADJ_TRY(cudaMemcpyAsync(work, psi0_dev, vb, cudaMemcpyDeviceToDevice, s));
  for (int c = 0; c < n_ckpt; ++c) {
    const int n0 = c * K, cnt = std::min(K, nsteps - n0);
    ADJ_TRY(cudaMemcpyAsync(ckpt + (size_t)c * n, work, vb, cudaMemcpyDeviceToDevice, s));
    ADJ_CHECK(dirac_lanczos_steps(ctx, work, cnt, dt, m, 0.0, A_xy_host + 2 * n0, nullptr));
  }
  if (psiN_dev) ADJ_TRY(cudaMemcpyAsync(psiN_dev, work, vb, cudaMemcpyDeviceToDevice, s));

  // loss and lambda_N
  const double w = v.dx * v.dy;
  if (opts->observable == DIRAC_OBS_PX) {
    PxArgs pa;
    pa.nx = v.nx; pa.ny = v.ny; pa.order = v.order; pa.diri = v.boundary == DIRAC_DIRICHLET;
    pa.inv_h = 1.0 / ((v.order == 2 ? 2.0 : 12.0) * v.dx);
    pa.w = w; pa.psi = work; pa.lam = lam; pa.part = part;
    adj_obs_px<<<nblk, 256, 0, s>>>(pa);
    ADJ_TRY(cudaGetLastError());
    adj_obs_finish<<<1, 32, 0, s>>>(part, nblk, DIRAC_OBS_PX, w, obs);
    ADJ_TRY(cudaGetLastError());
    launches += 2;
  } else {
    adj_obs_dot<<<nblk, 256, 0, s>>>(static_cast<const v4*>(opts->phi_dev), work, n, part);
    ADJ_TRY(cudaGetLastError());
    adj_obs_finish<<<1, 32, 0, s>>>(part, nblk, DIRAC_OBS_PROJ, w, obs);
    ADJ_TRY(cudaGetLastError());
    adj_obs_scale<<<nblk, 256, 0, s>>>(static_cast<const v4*>(opts->phi_dev), n, obs, lam);
    ADJ_TRY(cudaGetLastError());
    launches += 3;
  }
  double hobs[4];
  ADJ_TRY(cudaMemcpyAsync(hobs, obs, sizeof(hobs), cudaMemcpyDeviceToHost, s));
  ADJ_TRY(cudaEventRecord(ev[1], s));
  ADJ_TRY(cudaStreamSynchronize(s));
  *loss_out = hobs[0];
  if (!std::isfinite(hobs[0])) return fail(DIRAC_ENONFINITE, "non-finite observable");

  // backward sweep (skipped when no gradient is asked for, or when lambda_N
  // vanishes: then every gradient is zero)
  const bool need_grad = dV_dev || dA_host || da_host;
  const bool zero_adjoint = !need_grad ||
                            (opts->observable == DIRAC_OBS_PROJ && hobs[1] == 0.0 && hobs[2] == 0.0);
  const int jw = m <= 16 ? 16 : 32;
  MArgs ma;
  ma.fwd = static_cast<const DevState*>(v.dev_state);
  ma.bwd = static_cast<const DevState*>(vb_view.dev_state);
  ma.cp = dcp; ma.wq = dw; ma.R = R; ma.two_dt = 2.0 * dt; ma.M = Mm;
  CArgs ca;
  ca.fwd = ma.fwd; ca.bwd = ma.bwd;
  ca.qf = static_cast<const v4*>(v.basis);
  ca.pb = static_cast<const v4*>(vb_view.basis);
  ca.p1 = lam1; ca.M = Mm; ca.n = n; ca.gV = gV; ca.part = part;
  // CUDA-event timing of the contraction kernels while the context profiles
  cudaEvent_t cev[2];
  for (auto& e : cev) ADJ_TRY(cudaEventCreate(&e));
  struct CevGuard {
    cudaEvent_t* e;
    ~CevGuard() { for (int i = 0; i < 2; ++i) cudaEventDestroy(e[i]); }
  } cevg{cev};
  double ms_contract = 0.0;
  for (int c = n_ckpt - 1; c >= 0 && !zero_adjoint; --c) {
    const int n0 = c * K, cnt = std::min(K, nsteps - n0);
    // the segment's states psi_{n0} .. psi_{n0+cnt-1}
    ADJ_TRY(cudaMemcpyAsync(seg, ckpt + (size_t)c * n, vb, cudaMemcpyDeviceToDevice, s));
    for (int k = 1; k < cnt; ++k) {
      ADJ_TRY(cudaMemcpyAsync(seg + (size_t)k * n, seg + (size_t)(k - 1) * n, vb, cudaMemcpyDeviceToDevice, s));
      ADJ_CHECK(dirac_lanczos_steps(ctx, seg + (size_t)k * n, 1, dt, m, 0.0, A_xy_host + 2 * (n0 + k - 1),
                                    nullptr));
    }
    for (int k = cnt - 1; k >= 0; --k) {
      const int step = n0 + k;
      const double* a = A_xy_host + 2 * step;
      // Krylov space of psi_n (the step's result in `work` is not used)
      ADJ_TRY(cudaMemcpyAsync(work, seg + (size_t)k * n, vb, cudaMemcpyDeviceToDevice, s));
      ADJ_CHECK(dirac_lanczos_steps(ctx, work, 1, dt, m, 0.0, a, nullptr));
      // Krylov space of lambda_{n+1}, and lambda_n = exp(+i H_n dt) lambda_{n+1}
      ADJ_TRY(cudaMemcpyAsync(lam1, lam, vb, cudaMemcpyDeviceToDevice, s));
      ADJ_CHECK(dirac_lanczos_steps(back.c, lam, 1, -dt, m, 0.0, a, nullptr));
      adj_mmat<<<1, QMAX * 32, 0, s>>>(ma);
      ADJ_TRY(cudaGetLastError());
      ca.q1 = seg + (size_t)k * n;
      if (v.profiling) ADJ_TRY(cudaEventRecord(cev[0], s));
      if (jw == 16) adj_contract<16><<<nblk, 256, 0, s>>>(ca);
      else adj_contract<32><<<nblk, 256, 0, s>>>(ca);
      ADJ_TRY(cudaGetLastError());
      if (v.profiling) {   // profiling only: wait for this launch and add its time
        float t = 0.f;
        ADJ_TRY(cudaEventRecord(cev[1], s));
        ADJ_TRY(cudaEventSynchronize(cev[1]));
        ADJ_TRY(cudaEventElapsedTime(&t, cev[0], cev[1]));
        ms_contract += t;
      }
      adj_finish_a<<<1, 32, 0, s>>>(part, nblk, v.c, gA + 2 * step);   // dH/dA = c sigma (electron)
      ADJ_TRY(cudaGetLastError());
      launches += 3;
    }
  }
  // errors of the steps surface here
  ADJ_CHECK(dirac_sync(ctx));
  ADJ_CHECK(dirac_sync(back.c));

  if (dV_dev) {
    const int nout = (v.nx / bx) * (v.ny / by);
    adj_pool<<<(nout + 255) / 256, 256, 0, s>>>(gV, v.nx, v.ny, bx, by, static_cast<double*>(dV_dev));
    ADJ_TRY(cudaGetLastError());
    ++launches;
  }
  if (dA_host) ADJ_TRY(cudaMemcpyAsync(dA_host, gA, sizeof(double) * 2 * (size_t)nsteps, cudaMemcpyDeviceToHost, s));
  if (da_host) {
    double* dW = reinterpret_cast<double*>(sb + o_W);
    double* dda = reinterpret_cast<double*>(sb + o_da);
    ADJ_TRY(cudaMemcpyAsync(dW, opts->W_host, sizeof(double) * (size_t)nsteps * opts->n_coef,
                            cudaMemcpyHostToDevice, s));
    adj_coef<<<(opts->n_coef + 127) / 128, 128, 0, s>>>(dW, gA, nsteps, opts->n_coef, dda);
    ADJ_TRY(cudaGetLastError());
    ++launches;
    ADJ_TRY(cudaMemcpyAsync(da_host, dda, sizeof(double) * opts->n_coef, cudaMemcpyDeviceToHost, s));
  }
  ADJ_TRY(cudaEventRecord(ev[2], s));
  ADJ_TRY(cudaStreamSynchronize(s));
  const long long steps_launches = (*v.launches - l0) + dirac_kernel_launches(back.c);
  *v.launches += launches;
  if (info) {
    float f = 0.f, b = 0.f;
    ADJ_TRY(cudaEventElapsedTime(&f, ev[0], ev[1]));
    ADJ_TRY(cudaEventElapsedTime(&b, ev[1], ev[2]));
    info->ms_forward = f;
    info->ms_backward = b;
    info->quadrature_nodes = R;
    info->checkpoints = n_ckpt;
    info->launches = launches + steps_launches;
    info->ms_contract = ms_contract;
  }
  return DIRAC_OK;
}

}  // extern "C"
