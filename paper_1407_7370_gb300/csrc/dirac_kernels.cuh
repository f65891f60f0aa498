// dirac_kernels.cuh -- device code of the GB300 Dirac Lanczos propagator (FP64 path).
//
// One time step (Sec. 4, Eq. 17) is m launches of `lanczos_pass` (one Lanczos
// iteration each, Fig. 1 / Eq. 4) and one launch of `recombine`.
//
// Pass i (1-based) works on unnormalised vectors whose scales are tracked by
// device scalars:
//   q^_1 = psi                                  (no copy: psi is read in place)
//   q^_i = g_{i-1} (y^_{i-1} - d_{i-1} q^_{i-1})  formed on the fly, i >= 2
//   y^_i = (H - s - sigma_i) q^_i - e_i q^_{i-1}  the stencil product
// and reduces P = Re<q^_i, y^_i>, Y = ||y^_i||^2, X = ||q^_i||^2 in the same
// pass.  With q_i = q^_i / nu_i (nu_i = sqrt X) one has y^_i = nu_i (z_i -
// sigma_i q_i), z_i = A q_i - beta_{i-1} q_{i-1} being the vector of Fig. 1,
// so that exactly (in exact arithmetic)
//   alpha_i  = sigma_i + P / X                         (Eq. 4)
//   d_i      = P / X,   ||z_i - alpha_i q_i||^2 nu_i^2 = Y - P d_i =: s2_i
//   beta_{i-1} = nu_i / (g_{i-1} nu_{i-1})               (a posteriori, exact)
//   g_i = 1 / sqrt(s2_i),  e_{i+1} = sqrt(s2_i) / X,  sigma_{i+1} = alpha_i.
// The shift sigma_i = alpha_{i-1} keeps s2 free of cancellation (Y ~ s2),
// and beta_{i-1} is taken from the measured norm of the next vector rather
// than from s2, so the tridiagonal T of Fig. 1 is reproduced to rounding.
// The last CTA of each pass sums the per-CTA partials in a fixed order
// (deterministic, no floating-point atomics) and updates the scalars.
//
// exp(-i T dt) e_1 (Sec. 4) is evaluated on one warp by a Chebyshev expansion
// over an a-priori spectral interval of H (Jacobi-Anger coefficients computed
// on the host).  The paper diagonalises T; on this GPU FP64 division and
// square root have latencies of several hundred cycles, which would make a
// serial eigensolver dominate small steps, while the Chebyshev recurrence is
// FMA-only and warp-parallel.  Both give exp(-i T dt) e_1 to rounding.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dirac {

constexpr int KMAX = 32;        // Krylov dimension limit (one warp holds T)
constexpr int CHEB_MAX = 160;   // Chebyshev terms limit
constexpr int TX = 32;          // tile width (sites, x)
constexpr int TY = 8;           // tile height (sites, y)
constexpr int NT = TX * TY;     // threads per tile CTA
constexpr int ERR_NONFINITE = 4;

using vec4 = double4_32a;       // one site: (u.re, u.im, d.re, d.im)

struct DevState {
  double alpha[KMAX + 2];   // T diagonal of H - s, index 1..k
  double beta[KMAX + 2];    // beta[i] couples i and i+1; beta[k] = beta_k estimate
  double nu[KMAX + 2];      // ||q^_i||
  double sigma[KMAX + 2];   // stencil shift of pass i
  double g[KMAX + 2];
  double d[KMAX + 2];
  double e[KMAX + 2];
  double coef_re[KMAX + 2]; // recombination coefficients C_j, j = 1..k
  double coef_im[KMAX + 2];
  double scale;             // running max(|alpha_j + s|, beta_j) for breakdown
  double psi_norm, energy, err_est, cum_err, beta_last, kappa_max;
  int stopped;              // passes of this step are done (or an error is pending)
  int k_used, breakdown, error, sigma_valid;
  unsigned counter;         // last-CTA ticket of the running pass
};

struct ChebParams {
  int n;                    // number of terms
  double c0;                // centre of the spectral interval of H - s
  double inv_half;          // 1 / half width
  double ph_re, ph_im;      // exp(-i (c0 + s) dt)
  double cr[CHEB_MAX];      // eps_n (-i)^n J_n(half * dt), real part
  double ci[CHEB_MAX];      //                               imaginary part
};

struct PassParams {
  const vec4* psi;          // q^_1 (the state, read in place)
  const vec4* y_prev;       // y^_{i-1}
  const vec4* q_prev;       // q^_{i-1}
  vec4* q_out;              // q^_i  (i >= 2)
  vec4* y_out;              // y^_i  (NULL on the last pass)
  const double* V;          // potential energy [ny][nx] or NULL
  DevState* st;
  double* partials;         // 3 doubles per CTA
  int nx, ny;
  int pass, m, probe;
  double kx, ky;            // c/(2dx) (order 2) or c/(12dx) (order 4)
  double mcc, cAx, cAy, shift, dt, tol;
  ChebParams cheb;
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// grid coordinate -> array index; `outside` marks a Dirichlet zero
template <bool DIRI>
__device__ __forceinline__ int wrap(int g, int n, bool& outside) {
  if (g >= 0 && g < n) { outside = false; return g; }
  if (DIRI) { outside = true; return 0; }
  outside = false;
  int r = g % n;
  return r < 0 ? r + n : r;
}

// ---------------------------------------------------------------------------
// exp(-i T dt) e_1 on one warp: lane j holds component j+1 (k <= 32).
// T diagonal alpha[1..k], off-diagonal beta[1..k-1] (1-based arrays).
// X = (T - c0) / half has its spectrum in [-1, 1]; exp(-i R X) with
// R = half * dt is sum_n eps_n (-i)^n J_n(R) T_n(X) (Jacobi-Anger), summed
// with the three-term Chebyshev recurrence T_{n+1} = 2 X T_n - T_{n-1}.
// ---------------------------------------------------------------------------
__device__ void cheb_expm_e1(const ChebParams& cp, int k, const volatile double* alpha,
                             const volatile double* beta, double& vr, double& vi) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  double a = 0.0, bl = 0.0, bh = 0.0;
  if (lane < k) {
    a = (alpha[lane + 1] - cp.c0) * cp.inv_half;
    if (lane >= 1) bl = beta[lane] * cp.inv_half;
    if (lane + 1 < k) bh = beta[lane + 1] * cp.inv_half;
  }
  double t0 = (lane == 0) ? 1.0 : 0.0;
  double up = __shfl_up_sync(full, t0, 1);
  double dn = __shfl_down_sync(full, t0, 1);
  double t1 = fma(a, t0, fma(bl, up, bh * dn));
  double r = cp.cr[0] * t0 + cp.cr[1] * t1;
  double im = cp.ci[0] * t0 + cp.ci[1] * t1;
  const double a2 = 2.0 * a, bl2 = 2.0 * bl, bh2 = 2.0 * bh;
  for (int n = 2; n < cp.n; ++n) {
    up = __shfl_up_sync(full, t1, 1);
    dn = __shfl_down_sync(full, t1, 1);
    const double t2 = fma(a2, t1, fma(bl2, up, fma(bh2, dn, -t0)));
    r = fma(cp.cr[n], t2, r);
    im = fma(cp.ci[n], t2, im);
    t0 = t1;
    t1 = t2;
  }
  vr = r * cp.ph_re - im * cp.ph_im;
  vi = r * cp.ph_im + im * cp.ph_re;
}

// ---------------------------------------------------------------------------
// Scalar update after pass i: run by warp 0 of the last CTA with the grid
// totals P, Y, X in every lane.
// ---------------------------------------------------------------------------
__device__ void finish_pass(const PassParams& p, double P, double Y, double X) {
  volatile DevState* st = p.st;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int i = p.pass;
  const bool ok = isfinite(P) && isfinite(Y) && isfinite(X) && X > 0.0;
  if (p.probe) {   // Rayleigh quotient of psi: the first stencil shift
    if (lane == 0) {
      if (ok) { st->sigma[1] = st->sigma[1] + P / X; st->sigma_valid = 1; }
      else { st->error = ERR_NONFINITE; st->stopped = 1; }
    }
    return;
  }
  if (!ok) {
    if (lane == 0) { st->error = ERR_NONFINITE; st->stopped = 1; }
    return;
  }
  int stop = 0, brk = 0;
  double beta_hat = 0.0;
  if (lane == 0) {
    const double nu = sqrt(X);
    const double dd = P / X;
    const double alpha = st->sigma[i] + dd;
    st->nu[i] = nu;
    st->alpha[i] = alpha;
    st->d[i] = dd;
    double scale = (i == 1) ? 0.0 : st->scale;
    if (i == 1) {
      st->psi_norm = nu;
      st->energy = alpha + p.shift;
    } else {
      const double b = nu / (st->g[i - 1] * st->nu[i - 1]);
      st->beta[i - 1] = b;
      scale = fmax(scale, b);
    }
    scale = fmax(scale, fabs(alpha + p.shift));
    st->scale = scale;
    const double s2 = Y - P * dd;
    const double sq = s2 > 0.0 ? sqrt(s2) : 0.0;
    beta_hat = sq / nu;
    st->beta[i] = beta_hat;
    if (s2 > 0.0) st->kappa_max = fmax(st->kappa_max, Y / s2);
    brk = beta_hat <= 1e-12 * scale;
    stop = (i >= p.m) || brk;
    if (!stop) {
      st->g[i] = 1.0 / sq;
      st->e[i + 1] = sq / X;
      st->sigma[i + 1] = alpha;
    }
  }
  stop = __shfl_sync(full, stop, 0);
  brk = __shfl_sync(full, brk, 0);
  beta_hat = __shfl_sync(full, beta_hat, 0);
  __syncwarp();
  double vr = 0.0, vi = 0.0;
  bool have_v = false;
  if (!stop && p.tol > 0.0) {   // adaptive Krylov dimension (Sec. 4, Eq. 18)
    cheb_expm_e1(p.cheb, i, st->alpha, st->beta, vr, vi);
    have_v = true;
    const double vk = __shfl_sync(full, sqrt(vr * vr + vi * vi), i - 1);
    stop = (beta_hat * p.dt * vk <= p.tol);
  }
  if (!stop) return;
  if (!have_v) cheb_expm_e1(p.cheb, i, st->alpha, st->beta, vr, vi);
  // C_j = nu_1 / nu_j * v_j applied to q^_j; Eq. 18 estimate from v_k
  const double vk = __shfl_sync(full, sqrt(vr * vr + vi * vi), i - 1);
  if (lane < i) {
    const double f = st->nu[1] / st->nu[lane + 1];
    st->coef_re[lane + 1] = f * vr;
    st->coef_im[lane + 1] = f * vi;
  }
  if (lane == 0) {
    const double err = p.dt * beta_hat * st->psi_norm * vk;
    st->err_est = err;
    st->cum_err = st->cum_err + err;
    st->k_used = i;
    st->breakdown = brk;
    st->beta_last = beta_hat;
    st->sigma[1] = st->alpha[1];   // next step's first shift
    st->sigma_valid = 1;
    st->stopped = 1;
  }
}

// ---------------------------------------------------------------------------
// One Lanczos iteration: stencil product with fused reductions.
// R = stencil half width (1: order 2, 2: order 4).
// ---------------------------------------------------------------------------
template <int R, bool DIRI, bool HAS_V>
__global__ void __launch_bounds__(NT) lanczos_pass(const __grid_constant__ PassParams p) {
  __shared__ vec4 tile[TY + 2 * R][TX + 2 * R];
  __shared__ double red[NT / 32][3];
  __shared__ int last_cta;
  volatile DevState* st = p.st;
  if (st->stopped) return;

  const int i = p.pass;
  const double sigma = st->sigma[i];
  double g = 1.0, gd = 0.0, e = 0.0;
  if (i >= 2) {
    g = st->g[i - 1];
    gd = g * st->d[i - 1];
    e = st->e[i];
  }
  const int nx = p.nx, ny = p.ny;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;

  // value of q^_i at grid point (gx, gy), possibly outside the grid
  auto form = [&](int gx, int gy, vec4& qprev_out) -> vec4 {
    bool ox, oy;
    const int ix = wrap<DIRI>(gx, nx, ox), iy = wrap<DIRI>(gy, ny, oy);
    vec4 v;
    if (ox || oy) { v.x = v.y = v.z = v.w = 0.0; qprev_out = v; return v; }
    const size_t idx = (size_t)iy * nx + ix;
    if (i == 1) {
      v = p.psi[idx];
      qprev_out = v;
    } else {
      const vec4 yv = p.y_prev[idx];
      const vec4 qv = p.q_prev[idx];
      v.x = fma(-gd, qv.x, g * yv.x);
      v.y = fma(-gd, qv.y, g * yv.y);
      v.z = fma(-gd, qv.z, g * yv.z);
      v.w = fma(-gd, qv.w, g * yv.w);
      qprev_out = qv;
    }
    return v;
  };

  // centre slots: one per thread, keeping q^_{i-1} of the own site
  vec4 qprev;
  tile[ty + R][tx + R] = form(x0 + tx, y0 + ty, qprev);
  // halo slots (cross shape, no corners)
  constexpr int NH_ROW = 2 * R * TX, NH = NH_ROW + 2 * R * TY;
  if (threadIdx.x < NH) {
    int row, col;
    const int h = threadIdx.x;
    if (h < NH_ROW) {
      const int r = h / TX;
      row = (r < R) ? r : TY + r;
      col = (h % TX) + R;
    } else {
      const int h2 = h - NH_ROW;
      row = h2 / (2 * R) + R;
      const int c = h2 % (2 * R);
      col = (c < R) ? c : TX + c;
    }
    vec4 dummy;
    tile[row][col] = form(x0 + col - R, y0 + row - R, dummy);
  }
  __syncthreads();

  const int x = x0 + tx, y = y0 + ty;
  double P = 0.0, Y = 0.0, Xn = 0.0;
  if (x < nx && y < ny) {
    const size_t idx = (size_t)y * nx + x;
    const int r = ty + R, c = tx + R;
    const vec4 C = tile[r][c];
    double dxu_r, dxu_i, dxd_r, dxd_i, dyu_r, dyu_i, dyd_r, dyd_i;
    {
      const vec4 E1 = tile[r][c + 1], W1 = tile[r][c - 1];
      const vec4 N1 = tile[r + 1][c], S1 = tile[r - 1][c];
      dxu_r = E1.x - W1.x; dxu_i = E1.y - W1.y; dxd_r = E1.z - W1.z; dxd_i = E1.w - W1.w;
      dyu_r = N1.x - S1.x; dyu_i = N1.y - S1.y; dyd_r = N1.z - S1.z; dyd_i = N1.w - S1.w;
      if constexpr (R == 2) {
        const vec4 E2 = tile[r][c + R], W2 = tile[r][c - R];
        const vec4 N2 = tile[r + R][c], S2 = tile[r - R][c];
        dxu_r = fma(8.0, dxu_r, W2.x - E2.x); dxu_i = fma(8.0, dxu_i, W2.y - E2.y);
        dxd_r = fma(8.0, dxd_r, W2.z - E2.z); dxd_i = fma(8.0, dxd_i, W2.w - E2.w);
        dyu_r = fma(8.0, dyu_r, S2.x - N2.x); dyu_i = fma(8.0, dyu_i, S2.y - N2.y);
        dyd_r = fma(8.0, dyd_r, S2.z - N2.z); dyd_i = fma(8.0, dyd_i, S2.w - N2.w);
      }
    }
    double au = p.mcc - p.shift - sigma, ad = -p.mcc - p.shift - sigma;
    if (HAS_V) {
      const double v = p.V[idx];
      au += v;
      ad += v;
    }
    const double kx = p.kx, ky = p.ky, cAx = p.cAx, cAy = p.cAy;
    vec4 yv;
    // upper: (mc^2+V-s-sigma) u + c[-i D_x d - D_y d + (A_x - i A_y) d]
    yv.x = au * C.x + kx * dxd_i - ky * dyd_r + cAx * C.z + cAy * C.w;
    yv.y = au * C.y - kx * dxd_r - ky * dyd_i + cAx * C.w - cAy * C.z;
    // lower: (-mc^2+V-s-sigma) d + c[-i D_x u + D_y u + (A_x + i A_y) u]
    yv.z = ad * C.z + kx * dxu_i + ky * dyu_r + cAx * C.x - cAy * C.y;
    yv.w = ad * C.w - kx * dxu_r + ky * dyu_i + cAx * C.y + cAy * C.x;
    if (i >= 2) {
      yv.x = fma(-e, qprev.x, yv.x);
      yv.y = fma(-e, qprev.y, yv.y);
      yv.z = fma(-e, qprev.z, yv.z);
      yv.w = fma(-e, qprev.w, yv.w);
    }
    if (!p.probe) {
      if (p.q_out) p.q_out[idx] = C;
      if (p.y_out) p.y_out[idx] = yv;
    }
    P = C.x * yv.x + C.y * yv.y + C.z * yv.z + C.w * yv.w;
    Y = yv.x * yv.x + yv.y * yv.y + yv.z * yv.z + yv.w * yv.w;
    Xn = C.x * C.x + C.y * C.y + C.z * C.z + C.w * C.w;
  }

  // CTA reduction in a fixed order
  P = warp_sum(P);
  Y = warp_sum(Y);
  Xn = warp_sum(Xn);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red[warp][0] = P; red[warp][1] = Y; red[warp][2] = Xn; }
  __syncthreads();
  const unsigned ncta = gridDim.x * gridDim.y;
  const unsigned cta = blockIdx.y * gridDim.x + blockIdx.x;
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) { s0 += red[w][0]; s1 += red[w][1]; s2 += red[w][2]; }
    p.partials[3 * (size_t)cta + 0] = s0;
    p.partials[3 * (size_t)cta + 1] = s1;
    p.partials[3 * (size_t)cta + 2] = s2;
    __threadfence();
    const unsigned ticket = atomicAdd((unsigned*)&p.st->counter, 1u);
    last_cta = (ticket == ncta - 1);
  }
  __syncthreads();
  if (!last_cta) return;

  // last CTA: sum all partials in a fixed order
  __threadfence();
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (unsigned b = threadIdx.x; b < ncta; b += NT) {
    s0 += __ldcg(p.partials + 3 * (size_t)b + 0);
    s1 += __ldcg(p.partials + 3 * (size_t)b + 1);
    s2 += __ldcg(p.partials + 3 * (size_t)b + 2);
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  __syncthreads();
  if (lane == 0) { red[warp][0] = s0; red[warp][1] = s1; red[warp][2] = s2; }
  __syncthreads();
  if (warp == 0) {
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) { t0 += red[w][0]; t1 += red[w][1]; t2 += red[w][2]; }
    if (lane == 0) st->counter = 0u;
    finish_pass(p, t0, t1, t2);
  }
}

// ---------------------------------------------------------------------------
// psi <- sum_j C_j q^_j (Eq. 17), q^_1 = psi, q^_j = basis[j-2] for j >= 2.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) recombine(vec4* psi, const vec4* __restrict__ basis,
                                                 long long n_sites, DevState* st_) {
  __shared__ double cr[KMAX + 2], ci[KMAX + 2];
  __shared__ int k_s, err_s;
  volatile DevState* st = st_;
  if (threadIdx.x == 0) { k_s = st->k_used; err_s = st->error; }
  if (threadIdx.x <= KMAX) { cr[threadIdx.x] = st->coef_re[threadIdx.x]; ci[threadIdx.x] = st->coef_im[threadIdx.x]; }
  __syncthreads();
  if (err_s) return;                                   // leave psi untouched
  if (blockIdx.x == 0 && threadIdx.x == 0) st->stopped = 0;   // re-arm the next step
  const int k = k_s;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n_sites; s += stride) {
    const vec4 q = psi[s];
    double ur = cr[1] * q.x - ci[1] * q.y, ui = cr[1] * q.y + ci[1] * q.x;
    double dr = cr[1] * q.z - ci[1] * q.w, di = cr[1] * q.w + ci[1] * q.z;
    for (int j = 2; j <= k; ++j) {
      const vec4 b = basis[(size_t)(j - 2) * n_sites + s];
      const double a = cr[j], bb = ci[j];
      ur = fma(a, b.x, fma(-bb, b.y, ur));
      ui = fma(a, b.y, fma(bb, b.x, ui));
      dr = fma(a, b.z, fma(-bb, b.w, dr));
      di = fma(a, b.w, fma(bb, b.z, di));
    }
    vec4 o;
    o.x = ur; o.y = ui; o.z = dr; o.w = di;
    psi[s] = o;
  }
}

// ---------------------------------------------------------------------------
// test hook: exp(-i T dt) e_1 for a given T with the device routine
// ---------------------------------------------------------------------------
__global__ void debug_tridiag_expm(const __grid_constant__ ChebParams cp, int k, const double* alpha1,
                                   const double* beta1, double* out_re, double* out_im) {
  double vr, vi;
  cheb_expm_e1(cp, k, alpha1, beta1, vr, vi);
  const int lane = threadIdx.x & 31;
  if (lane < k) { out_re[lane] = vr; out_im[lane] = vi; }
}

}  // namespace dirac
