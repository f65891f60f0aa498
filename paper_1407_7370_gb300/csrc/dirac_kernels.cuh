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

#include <cuda/atomic>

namespace dirac {

constexpr int KMAX = 32;        // Krylov dimension limit (one warp holds T)
constexpr int CHEB_MAX = 160;   // Chebyshev terms limit
constexpr int ERR_NONFINITE = 4;

using vec4 = double4_32a;       // one site: (u.re, u.im, d.re, d.im)

// Coefficients one pass needs, prepared by the finisher of the pass before
// (FP64 values and FP32 copies, so that no thread converts on the FP64 pipe).
struct PassCoef {
  double g, gd, e, au0, ad0;          // q^ = g y^ - gd q^_prev; y^ -= e q^_prev; diagonals
  float gf, gdf, ef, au_hi, au_lo, ad_hi, ad_lo, pad;
};

__host__ __device__ inline PassCoef make_coef(double g, double gd, double e, double au0, double ad0) {
  PassCoef c;
  c.g = g; c.gd = gd; c.e = e; c.au0 = au0; c.ad0 = ad0;
  c.gf = (float)g; c.gdf = (float)gd; c.ef = (float)e;
  // the diagonals (up to ~2 m c^2) as a rounded float plus its remainder, so
  // that on the FP32 path their rounding does not act as a constant
  // perturbation of the mass term
  c.au_hi = (float)au0; c.au_lo = (float)(au0 - (double)c.au_hi);
  c.ad_hi = (float)ad0; c.ad_lo = (float)(ad0 - (double)c.ad_hi);
  c.pad = 0.f;
  return c;
}

struct DevState {
  PassCoef pc[KMAX + 2];    // coefficients of pass i (pc[1]: first pass of a step)
  double alpha[KMAX + 2];   // T diagonal of H - s, index 1..k
  double beta[KMAX + 2];    // beta[i] couples i and i+1; beta[k] = beta_k estimate
  double nu[KMAX + 2];      // ||q^_i||
  double inv_nu[KMAX + 2];  // 1 / ||q^_i||
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
  const void* psi;          // q^_1 (the FP64 state, read in place)
  const void* y_prev;       // y^_{i-1}
  const void* q_prev;       // q^_{i-1}
  void* q_out;              // q^_i  (i >= 2)
  void* y_out;              // y^_i  (NULL on the last pass)
  const void* V;            // potential energy [ny][nx] (double) or NULL
  DevState* st;
  double* partials;         // 3 doubles per CTA
  int nx, ny;
  int tiles_x, ntiles;      // tiles of TILE x TILE sites (grid-stride over them)
  int pass, m, probe;
  double kx, ky;            // c/(2dx) (order 2) or c/(12dx) (order 4)
  double mcc, cAx, cAy, shift, dt, tol;
  float kxf, kyf, cAxf, cAyf; // the same four in FP32 (rounded on the host)
  PassCoef probe_coef;      // coefficients of the probe pass (shift 0)
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
__device__ void cheb_expm_e1(const ChebParams& cp, int k, double alpha_j, double beta_lo,
                             double beta_hi, double& vr, double& vi) {
  // lane j holds alpha_{j+1} and the couplings to its neighbours (0 outside)
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  double a = 0.0, bl = 0.0, bh = 0.0;
  if (lane < k) {
    a = (alpha_j - cp.c0) * cp.inv_half;
    if (lane >= 1) bl = beta_lo * cp.inv_half;
    if (lane + 1 < k) bh = beta_hi * cp.inv_half;
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
// totals P, Y, X in every lane.  Values written by earlier launches are read
// with plain loads up front; new values travel by shuffles.  rsqrt gives
// sqrt(X), 1/X, sqrt(s2) and 1/sqrt(s2) with few dependent FP64 operations.
// ---------------------------------------------------------------------------
__device__ void finish_pass(const PassParams& p, double P, double Y, double X) {
  DevState* st = p.st;
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int i = p.pass;
  const bool ok = isfinite(P) && isfinite(Y) && isfinite(X) && X > 0.0;
  if (p.probe) {   // Rayleigh quotient of psi: the first stencil shift
    if (lane == 0) {
      if (ok) {
        const double s1 = P / X;   // the probe ran with shift 0
        st->sigma[1] = s1;
        st->pc[1] = make_coef(1.0, 0.0, 0.0, p.mcc - p.shift - s1, -p.mcc - p.shift - s1);
        st->sigma_valid = 1;
      } else {
        st->error = ERR_NONFINITE; st->stopped = 1;
      }
    }
    return;
  }
  if (!ok) {
    if (lane == 0) { st->error = ERR_NONFINITE; st->stopped = 1; }
    return;
  }
  // earlier T entries (lane j: component j+1), issued before the scalar chain
  const double a_old = (lane + 1 < i) ? st->alpha[lane + 1] : 0.0;
  const double b_old = (lane + 2 < i) ? st->beta[lane + 1] : 0.0;   // exact beta_{j+1}
  const double invnu_old = (lane + 1 < i) ? st->inv_nu[lane + 1] : 0.0;
  const double sigma = st->sigma[i];
  const double scale_old = (i == 1) ? 0.0 : st->scale;
  const double bhat_prev = (i == 1) ? 0.0 : st->beta[i - 1];       // estimate from pass i-1
  const double nu1_old = (i == 1) ? 0.0 : st->nu[1];
  const double psi_norm_old = st->psi_norm, cum_old = st->cum_err;

  // scalar chain (every lane computes it; no broadcast needed)
  const double y = rsqrt(X);            // 1 / nu_i
  const double nu = X * y;
  const double rX = y * y;
  const double dd = P * rX;             // alpha_i - sigma_i
  const double alpha = sigma + dd;
  const double s2 = fma(-P, dd, Y);     // nu_i^2 beta_i^2 (estimate)
  const double rs = s2 > 0.0 ? rsqrt(s2) : 0.0;
  const double sq = s2 > 0.0 ? s2 * rs : 0.0;
  const double beta_hat = sq * y;
  const double bprev = nu * bhat_prev;  // exact beta_{i-1} from the measured norm
  double scale = fmax(scale_old, fabs(alpha + p.shift));
  if (i > 1) scale = fmax(scale, bprev);
  const int brk = beta_hat <= 1e-12 * scale;
  int stop = (i >= p.m) || brk;
  const double nu1 = (i == 1) ? nu : nu1_old;
  const double psi_norm = (i == 1) ? nu : psi_norm_old;
  if (lane == 0) {
    st->nu[i] = nu;
    st->inv_nu[i] = y;
    st->alpha[i] = alpha;
    st->d[i] = dd;
    st->beta[i] = beta_hat;
    if (i > 1) st->beta[i - 1] = bprev;
    st->scale = scale;
    if (i == 1) { st->psi_norm = nu; st->energy = alpha + p.shift; }
    if (s2 > 0.0) st->kappa_max = fmax(st->kappa_max, Y * rs * rs);
    if (!stop) {
      st->g[i] = rs;
      st->e[i + 1] = sq * rX;
      st->sigma[i + 1] = alpha;
      st->pc[i + 1] = make_coef(rs, rs * dd, sq * rX, p.mcc - p.shift - alpha, -p.mcc - p.shift - alpha);
    }
  }
  // this lane's row of T^(i)
  const double a_j = (lane + 1 == i) ? alpha : a_old;
  const double b_hi = (lane + 2 == i) ? bprev : b_old;               // couples j+1, j+2
  const double b_lo = __shfl_up_sync(full, b_hi, 1);                 // couples j, j+1
  const double inv_nu_j = (lane + 1 == i) ? y : invnu_old;
  double vr = 0.0, vi = 0.0;
  bool have_v = false;
  if (!stop && p.tol > 0.0) {   // adaptive Krylov dimension (Sec. 4, Eq. 18)
    cheb_expm_e1(p.cheb, i, a_j, b_lo, b_hi, vr, vi);
    have_v = true;
    const double vk = __shfl_sync(full, sqrt(vr * vr + vi * vi), i - 1);
    stop = (beta_hat * p.dt * vk <= p.tol);
  }
  if (!stop) return;
  if (!have_v) cheb_expm_e1(p.cheb, i, a_j, b_lo, b_hi, vr, vi);
  // C_j = nu_1 / nu_j * v_j applied to q^_j; Eq. 18 estimate from v_k
  const double vk = __shfl_sync(full, sqrt(vr * vr + vi * vi), i - 1);
  if (lane < i) {
    const double f = nu1 * inv_nu_j;
    st->coef_re[lane + 1] = f * vr;
    st->coef_im[lane + 1] = f * vi;
  }
  if (lane == 0) {
    const double err = p.dt * beta_hat * psi_norm * vk;
    st->err_est = err;
    st->cum_err = cum_old + err;
    st->k_used = i;
    st->breakdown = brk;
    st->beta_last = beta_hat;
    const double s1 = (i == 1) ? alpha : st->alpha[1];   // next step's first shift
    st->sigma[1] = s1;
    st->pc[1] = make_coef(1.0, 0.0, 0.0, p.mcc - p.shift - s1, -p.mcc - p.shift - s1);
    st->sigma_valid = 1;
    st->stopped = 1;
  }
}

// ---------------------------------------------------------------------------
// One Lanczos iteration: stencil product with fused reductions.
//
// S    arithmetic type of the stencil (double: FP64 path; float: mixed path)
// R    stencil half width (1: order 2, 2: order 4)
// QIN64  q^_{i-1} (and psi) are complex128 (FP64 path, and passes 1-2 of the
//      mixed path, whose q^_1 is the FP64 state itself); otherwise they are
//      stored like y^ (complex64 in the mixed path)
//
// A CTA owns a TILE x TILE block of sites; thread (tx, tg) handles column tx
// and rows tg, tg + NG, tg + 2 NG, tg + 3 NG (NG = TILE / RPT), so every warp
// touches one contiguous row segment per access.  The tile and a cross-shaped
// halo of q^_i are formed in shared memory from y^_{i-1} and q^_{i-1}.
// ---------------------------------------------------------------------------
template <class S> struct Vec4;
template <> struct Vec4<double> { using T = double4_32a; };
template <> struct Vec4<float> { using T = float4; };

template <class To, class From>
__device__ __forceinline__ void cvt4(const From& a, To (&o)[4]) {
  o[0] = (To)a.x; o[1] = (To)a.y; o[2] = (To)a.z; o[3] = (To)a.w;
}

template <class S>
__device__ __forceinline__ S warp_sum_t(S v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int TILE = 32;          // tile edge (sites)
constexpr int RPT = 4;            // rows per thread
constexpr int NG = TILE / RPT;    // row groups
constexpr int NTP = 32 * NG;      // threads per CTA (256)

template <class S, int R, bool DIRI, bool HAS_V, bool QIN64>
__global__ void __launch_bounds__(NTP, sizeof(S) == sizeof(float) ? 5 : 2)
lanczos_pass(const __grid_constant__ PassParams p) {
  using T4 = typename Vec4<S>::T;           // storage of y^ and (if !QIN64) q^
  constexpr int W = TILE + 2 * R;
  __shared__ __align__(32) S tile[TILE + 2 * R][W][4];
  __shared__ double red[NTP / 32][3];
  __shared__ int last_cta;
  // programmatic dependent launch: everything above may overlap the tail of
  // the previous kernel; nothing it wrote is read before this point
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const DevState* st = p.st;   // written by earlier launches: plain loads
  if (st->stopped) return;
  const int i = p.pass;
  const PassCoef pc = p.probe ? p.probe_coef : st->pc[i];
  constexpr bool F32 = sizeof(S) == sizeof(float);
  const S gS = F32 ? (S)pc.gf : (S)pc.g;
  const S gdS = F32 ? (S)pc.gdf : (S)pc.gd;
  const S eS = F32 ? (S)pc.ef : (S)pc.e;
  const int nx = p.nx, ny = p.ny;
  const int tx = threadIdx.x & 31, tg = threadIdx.x >> 5;
  const T4* yprev = static_cast<const T4*>(p.y_prev);
  const S kx = F32 ? (S)p.kxf : (S)p.kx, ky = F32 ? (S)p.kyf : (S)p.ky;
  const S cAx = F32 ? (S)p.cAxf : (S)p.cAx, cAy = F32 ? (S)p.cAyf : (S)p.cAy;
  const S au_hi = F32 ? (S)pc.au_hi : (S)pc.au0, au_lo = F32 ? (S)pc.au_lo : S(0);
  const S ad_hi = F32 ? (S)pc.ad_hi : (S)pc.ad0, ad_lo = F32 ? (S)pc.ad_lo : S(0);
  S accP = S(0), accY = S(0), accX = S(0);
  int x0 = 0, y0 = 0;

  // q^_i at grid point (gx, gy) (zero outside for Dirichlet) into smem slot
  auto form = [&](int gx, int gy, int row, int col, S (&qp)[4]) {
    bool ox, oy;
    const int ix = wrap<DIRI>(gx, nx, ox), iy = wrap<DIRI>(gy, ny, oy);
    S q[4] = {S(0), S(0), S(0), S(0)};
    qp[0] = qp[1] = qp[2] = qp[3] = S(0);
    if (!(ox || oy)) {
      const size_t idx = (size_t)iy * nx + ix;
      if constexpr (QIN64) {
        const double4_32a* qsrc = static_cast<const double4_32a*>(i == 1 ? p.psi : p.q_prev);
        cvt4(qsrc[idx], qp);
      } else {
        cvt4(static_cast<const T4*>(p.q_prev)[idx], qp);
      }
      if (i == 1) {
#pragma unroll
        for (int c = 0; c < 4; ++c) q[c] = qp[c];
      } else {
        S yv[4];
        cvt4(yprev[idx], yv);
#pragma unroll
        for (int c = 0; c < 4; ++c) q[c] = fma(-gdS, qp[c], gS * yv[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) tile[row][col][c] = q[c];
  };

  for (int t = blockIdx.x; t < p.ntiles; t += gridDim.x) {
  x0 = (t % p.tiles_x) * TILE;
  y0 = (t / p.tiles_x) * TILE;
  S qprev[RPT][4];
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int r = tg + k * NG;
    form(x0 + tx, y0 + r, r + R, tx + R, qprev[k]);
  }
  constexpr int NH_ROW = 2 * R * TILE, NH = 2 * NH_ROW;
  for (int h = threadIdx.x; h < NH; h += NTP) {
    int row, col;
    if (h < NH_ROW) {               // rows above / below
      const int r = h / TILE;
      row = (r < R) ? r : TILE + r;
      col = (h % TILE) + R;
    } else {                        // columns left / right
      const int h2 = h - NH_ROW;
      row = h2 / (2 * R) + R;
      const int c = h2 % (2 * R);
      col = (c < R) ? c : TILE + c;
    }
    S dummy[4];
    form(x0 + col - R, y0 + row - R, row, col, dummy);
  }
  __syncthreads();

#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int ry = tg + k * NG;
    const int x = x0 + tx, y = y0 + ry;
    if (x < nx && y < ny) {
      const size_t idx = (size_t)y * nx + x;
      const int r = ry + R, c = tx + R;
      S C[4], dxv[4], dyv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        C[q] = tile[r][c][q];
        dxv[q] = tile[r][c + 1][q] - tile[r][c - 1][q];
        dyv[q] = tile[r + 1][c][q] - tile[r - 1][c][q];
        if constexpr (R == 2) {
          dxv[q] = fma(S(8), dxv[q], tile[r][c - 2][q] - tile[r][c + 2][q]);
          dyv[q] = fma(S(8), dyv[q], tile[r - 2][c][q] - tile[r + 2][c][q]);
        }
      }
      S au, ad;
      if constexpr (HAS_V) {       // V stored in S (float copy on the mixed path)
        const S v = static_cast<const S*>(p.V)[idx];
        au = au_hi + v;
        ad = ad_hi + v;
      } else {
        au = au_hi;
        ad = ad_hi;
      }
      // C = (u.re, u.im, d.re, d.im); dxv/dyv likewise
      S yv[4];
      // upper: (mc^2+V-s-sigma) u + c[-i D_x d - D_y d + (A_x - i A_y) d]
      yv[0] = au * C[0] + kx * dxv[3] - ky * dyv[2] + cAx * C[2] + cAy * C[3];
      yv[1] = au * C[1] - kx * dxv[2] - ky * dyv[3] + cAx * C[3] - cAy * C[2];
      // lower: (-mc^2+V-s-sigma) d + c[-i D_x u + D_y u + (A_x + i A_y) u]
      yv[2] = ad * C[2] + kx * dxv[1] + ky * dyv[0] + cAx * C[0] - cAy * C[1];
      yv[3] = ad * C[3] - kx * dxv[0] + ky * dyv[1] + cAx * C[1] + cAy * C[0];
      if constexpr (sizeof(S) == sizeof(float)) {
        yv[0] = fma(au_lo, C[0], yv[0]);
        yv[1] = fma(au_lo, C[1], yv[1]);
        yv[2] = fma(ad_lo, C[2], yv[2]);
        yv[3] = fma(ad_lo, C[3], yv[3]);
      }
      if (i >= 2) {
#pragma unroll
        for (int q = 0; q < 4; ++q) yv[q] = fma(-eS, qprev[k][q], yv[q]);
      }
      if (!p.probe) {
        if (p.q_out) {
          T4 o; o.x = C[0]; o.y = C[1]; o.z = C[2]; o.w = C[3];
          static_cast<T4*>(p.q_out)[idx] = o;
        }
        if (p.y_out) {
          T4 o; o.x = yv[0]; o.y = yv[1]; o.z = yv[2]; o.w = yv[3];
          static_cast<T4*>(p.y_out)[idx] = o;
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        accP = fma(C[q], yv[q], accP);
        accY = fma(yv[q], yv[q], accY);
        accX = fma(C[q], C[q], accX);
      }
    }
  }
  __syncthreads();   // the tile is reused by the next iteration
  }

  // the next kernel may be scheduled now (it waits for our completion)
  asm volatile("griddepcontrol.launch_dependents;");
  // reductions: thread -> warp in S, warp -> CTA in double (fixed order)
  accP = warp_sum_t(accP);
  accY = warp_sum_t(accY);
  accX = warp_sum_t(accX);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red[warp][0] = (double)accP; red[warp][1] = (double)accY; red[warp][2] = (double)accX; }
  __syncthreads();
  const unsigned ncta = gridDim.x;
  const unsigned cta = blockIdx.x;
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
    for (int w = 0; w < NTP / 32; ++w) { s0 += red[w][0]; s1 += red[w][1]; s2 += red[w][2]; }
    p.partials[3 * (size_t)cta + 0] = s0;
    p.partials[3 * (size_t)cta + 1] = s1;
    p.partials[3 * (size_t)cta + 2] = s2;
    // release our partials / acquire everybody else's
    cuda::atomic_ref<unsigned, cuda::thread_scope_device> ticket(p.st->counter);
    last_cta = (ticket.fetch_add(1u, cuda::memory_order_acq_rel) == ncta - 1);
  }
  __syncthreads();
  if (!last_cta || warp != 0) return;

  // last CTA, warp 0: sum all partials in a fixed order
  double t0 = 0.0, t1 = 0.0, t2 = 0.0;
  for (unsigned b = lane; b < ncta; b += 32) {
    t0 += __ldcg(p.partials + 3 * (size_t)b + 0);
    t1 += __ldcg(p.partials + 3 * (size_t)b + 1);
    t2 += __ldcg(p.partials + 3 * (size_t)b + 2);
  }
  t0 = warp_sum(t0);
  t1 = warp_sum(t1);
  t2 = warp_sum(t2);
  if (lane == 0) p.st->counter = 0u;
  finish_pass(p, t0, t1, t2);
}

// ---------------------------------------------------------------------------
// psi <- sum_j C_j q^_j (Eq. 17), q^_1 = psi, q^_j = basis[j-2] for j >= 2.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) recombine(vec4* psi, const vec4* __restrict__ basis,
                                                 long long n_sites, DevState* st_) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
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
// Mixed path: psi <- C_1 psi + sum_{j>=2} C_j q^_j with psi complex128 and the
// basis complex64.  C_1 psi is formed in FP64 so that the FP32 rounding of the
// basis only enters the (small) Krylov corrections.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) recombine_mixed(double4_32a* psi, const float4* __restrict__ basis,
                                                       long long n_sites, DevState* st_) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __shared__ double c1r, c1i;
  __shared__ float cr[KMAX + 2], ci[KMAX + 2];
  __shared__ int k_s, err_s;
  volatile DevState* st = st_;
  if (threadIdx.x == 0) {
    k_s = st->k_used; err_s = st->error;
    c1r = st->coef_re[1]; c1i = st->coef_im[1];
  }
  if (threadIdx.x <= KMAX) { cr[threadIdx.x] = (float)st->coef_re[threadIdx.x]; ci[threadIdx.x] = (float)st->coef_im[threadIdx.x]; }
  __syncthreads();
  if (err_s) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) st->stopped = 0;
  const int k = k_s;
  const double ar = c1r, ai = c1i;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n_sites; s += stride) {
    float ur = 0.f, ui = 0.f, dr = 0.f, di = 0.f;
    for (int j = 2; j <= k; ++j) {
      const float4 b = basis[(size_t)(j - 2) * n_sites + s];
      const float a = cr[j], bb = ci[j];
      ur = fmaf(a, b.x, fmaf(-bb, b.y, ur));
      ui = fmaf(a, b.y, fmaf(bb, b.x, ui));
      dr = fmaf(a, b.z, fmaf(-bb, b.w, dr));
      di = fmaf(a, b.w, fmaf(bb, b.z, di));
    }
    const double4_32a q = psi[s];
    double4_32a o;
    o.x = fma(ar, q.x, fma(-ai, q.y, (double)ur));
    o.y = fma(ar, q.y, fma(ai, q.x, (double)ui));
    o.z = fma(ar, q.z, fma(-ai, q.w, (double)dr));
    o.w = fma(ar, q.w, fma(ai, q.z, (double)di));
    psi[s] = o;
  }
}

// ---------------------------------------------------------------------------
// test hook: exp(-i T dt) e_1 for a given T with the device routine
// ---------------------------------------------------------------------------
__global__ void debug_tridiag_expm(const __grid_constant__ ChebParams cp, int k, const double* alpha1,
                                   const double* beta1, double* out_re, double* out_im) {
  double vr, vi;
  const int lane = threadIdx.x & 31;
  const double a = lane < k ? alpha1[lane + 1] : 0.0;
  const double bl = (lane >= 1 && lane < k) ? beta1[lane] : 0.0;
  const double bh = (lane + 1 < k) ? beta1[lane + 1] : 0.0;
  cheb_expm_e1(cp, k, a, bl, bh, vr, vi);
  if (lane < k) { out_re[lane] = vr; out_im[lane] = vi; }
}

}  // namespace dirac
