// dirac_kernels.cuh -- device code of the GB300 Dirac Lanczos propagator.
//
// One time step (Sec. 4, Eq. 17) is m launches of `lanczos_pass` (one Lanczos
// iteration each, Fig. 1 / Eq. 4) and one launch of `recombine`.  Every launch
// covers a table of independent problems (grids of any size); a single
// propagation is a table of one.  For a single problem the same pass body can
// instead run inside `lanczos_step`, one cooperative launch per time step
// whose passes are separated by grid-wide barriers (see there).
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
//   g_i = 1 / sqrt(s2_i),  e_{i+1} = sqrt(s2_i) / X.
// The stencil shift sigma_i only moves rounding: any value gives the same T
// in exact arithmetic.  It predicts alpha_i so that s2 is free of
// cancellation (Y ~ s2): the previous step's alpha_i where there is one (T
// changes little between steps), else alpha_{i-2} (the Krylov vectors of a
// packet with a negative-energy admixture alternate between the two bands),
// else alpha_{i-1}.  beta_{i-1} is taken from the measured norm of the next
// vector rather than from s2, so the tridiagonal T of Fig. 1 is reproduced
// to rounding.
//
// Work split: the tiles of all problems form one list of T tiles; persistent
// CTA c of G takes a contiguous chunk of T / G or T / G + 1 tiles.  A CTA may hold SUB independent tile workers (groups
// of warps with their own tile buffer and named barrier) that take the
// chunk's tiles in turn, so that one CTA per SM still overlaps one worker's
// loads with another's arithmetic.  Per problem it touches, a CTA writes one
// partial (P, Y, X) into slot c - (first CTA of that problem) and adds its
// tile count to the problem's ticket; the CTA that completes a problem sums
// that problem's slots in a fixed order (deterministic, no floating-point
// atomics) and updates its scalars.
//
// exp(-i T dt) e_1 (Sec. 4) is evaluated on one warp by a Chebyshev expansion
// over an a-priori spectral interval of H (Jacobi-Anger coefficients computed
// on the host).  The paper diagonalises T; on this GPU FP64 division and
// square root have latencies of several hundred cycles, which would make a
// serial eigensolver dominate small steps, while the Chebyshev recurrence is
// FMA-only and warp-parallel.  Both give exp(-i T dt) e_1 to rounding.
//
// Precision: S = double is the FP64 path.  S = float is the mixed path:
// complex64 basis and y^, FP32 stencil, warp sums converted to FP64, FP64
// scalars; q^_1 is the complex128 state itself (passes 1-2 read it).
#pragma once
#include <cuda.h>           // CUtensorMap (the type only; the library calls the driver through the runtime)
#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda/atomic>

namespace dirac {

constexpr int KMAX = 32;        // Krylov dimension limit (one warp holds T)
constexpr int CHEB_MAX = 160;   // Chebyshev terms limit
constexpr int ERR_NONFINITE = 4;
constexpr int TILE_W = 32;      // tile width in sites (one warp)

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
  PassCoef pc_cur;          // coefficients of the next pass to run
  PassCoef pc_prev;         // those of the last accepted pass (its stencil shift and coupling)
  int cur_pass;             // the next pass to run (1-based; 0 reads as 1)
  int redo_left;            // re-runs of a pass still allowed in this step
  double alpha[KMAX + 2];   // T diagonal of H - s, index 1..k
  double beta[KMAX + 2];    // beta[i] couples i and i+1; beta[k] = beta_k estimate
  double nu[KMAX + 2];      // ||q^_i||
  double inv_nu[KMAX + 2];  // 1 / ||q^_i||
  double sigma[KMAX + 2];   // stencil shift of pass i
  double coef_re[KMAX + 2]; // recombination coefficients C_j, j = 1..k
  double coef_im[KMAX + 2];
  double scale;             // running max(|alpha_j + s|, beta_j) for breakdown
  double psi_norm, energy, err_est, cum_err, beta_last, kappa_max;
  int stopped;              // passes of this step are done (or an error is pending)
  int k_used, breakdown, error, sigma_valid;
  unsigned counter;         // tiles of the running pass completed so far
};

struct ChebParams {
  int n;                    // number of terms
  double c0;                // centre of the spectral interval of H - s
  double inv_half;          // 1 / half width
  double ph_re, ph_im;      // exp(-i (c0 + s) dt)
  double cr[CHEB_MAX];      // eps_n (-i)^n J_n(half * dt), real part
  double ci[CHEB_MAX];      //                               imaginary part
};

// c * A of one step (electron: p - qA = p + A), FP64 and as FP32 pairs
// (rounded value and remainder)
struct FieldStep {
  double cAx, cAy;
  float cAxf, cAyf, cAxf_lo, cAyf_lo;
};

// One independent propagation problem.
struct Problem {
  int nx, ny, tiles_x, tile_begin, ntiles;   // tiles of TILE_W x TH sites
  int rblk_begin, rblk_count;                // recombination blocks
  const vec4* psi;          // the state (complex128), q^_1
  void* basis;              // q^_2 .. q^_m
  void* ybuf0;              // y^ ping-pong
  void* ybuf1;
  const void* V;            // potential energy in S, or NULL
  const void* Vlo;          // mixed path: V - (float)V as float, or NULL
  DevState* st;
  double* partials;         // 3 doubles per slot
  const ChebParams* cheb;
  double kx, ky, shift;     // c/(2dx) (order 2) or c/(12dx) (order 4); energy shift
  float kxf, kyf;           // kx, ky rounded to FP32
  float kxf_lo, kyf_lo;     // and their remainders
  int tma;                  // the mixed one-launch step stages tiles by tensor copies (maps valid)
  PassCoef probe_coef;      // coefficients of the probe pass (stencil shift 0)
};

// Tensor maps of one problem for the bulk tensor copies of the mixed
// one-launch step, each with a box of one tile and its halo and zeros
// outside the grid: `basis` covers the complex64 basis vectors q^_2 ..
// (packed, nx ny 16 bytes apart) as a 3D FP32 tensor {4 nx, ny, vectors},
// `ybuf` the two y^ buffers as {4 nx, ny, 2}, `psi` the complex128 state as a
// 2D FP64 tensor {4 nx, ny}.
struct TmaMaps {
  CUtensorMap basis;
  CUtensorMap ybuf;
  CUtensorMap psi;
};

struct LaunchParams {
  const Problem* probs;
  const TmaMaps* maps;      // one per problem (mixed one-launch step only), else NULL
  int redo_budget;          // re-runs allowed per step (the spare launches)
  double kappa_redo;        // re-run a pass whose ||y^||^2 / s2 exceeds this
  DevState* states;         // one per problem, same order
  const FieldStep* fields;  // fields[step * fstride + problem]
  int fstride;              // 0: one FieldStep per problem for every step
  int nprob, total_tiles;
  int chunk_q, chunk_r;     // tiles per CTA: q + 1 for the first r CTAs, then q
  int pass, m, probe;
  int conj_coef;            // 1: backward step (dt < 0): exp(+i H |dt|), the conjugate coefficients
  int async_tiles;          // FP32 basis: stage passes >= 3 by asynchronous copies (many tiles per CTA)
  int has_ay;               // 0: A_y = 0 in every step and problem (host: picks the kernel)
  int diri;                 // Dirichlet boundaries (kernels that take the boundary at run time)
  double mcc, dt, tol;      // dt = |dt|
  const int* step;          // step counter of the running call (index into fields)
};

struct RecombParams {
  const Problem* probs;
  const int* blk_prob;      // problem of each block
  int* step;                // advanced once per step
  int redo_budget;
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
template <class S>
__device__ __forceinline__ S warp_sum(S v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// compensated FP32 arithmetic (value s plus error accumulator e)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& r) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  r = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e  +=  (kh + kl) * a
__device__ __forceinline__ void acc_prod(float kh, float kl, float a, float& s, float& e) {
  const float p = __fmul_rn(kh, a);
  const float pe = fmaf(kh, a, -p);
  float t, r;
  two_sum(s, p, t, r);
  s = t;
  e = __fadd_rn(e, __fadd_rn(pe, r));
  e = fmaf(kl, a, e);
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

// asynchronous 16-byte global -> shared copy (bytes = 0: zero fill, nothing read)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// read-only (non-coherent) loads: the inputs of a pass are not written
// during it, and the compiler may then move these loads ahead of the shared
// memory stores in between
__device__ __forceinline__ vec4 ldg4(const vec4* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  const double2 a = __ldg(q), b = __ldg(q + 1);
  vec4 r;
  r.x = a.x; r.y = a.y; r.z = b.x; r.w = b.y;
  return r;
}
__device__ __forceinline__ float4 ldg4(const float4* p) { return __ldg(p); }

// plain (coherent) loads for the one-launch step: its own earlier passes
// wrote the data, so the read-only path may not serve it; the grid barrier's
// acquire orders these loads after the other CTAs' stores
__device__ __forceinline__ vec4 ldw4(const vec4* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  const double2 a = q[0], b = q[1];
  vec4 r;
  r.x = a.x; r.y = a.y; r.z = b.x; r.w = b.y;
  return r;
}
__device__ __forceinline__ float4 ldw4(const float4* p) { return *p; }

template <bool COHERENT, class T>
__device__ __forceinline__ T ld4(const T* p) {
  if constexpr (COHERENT) return ldw4(p);
  else return ldg4(p);
}

template <class S> struct Vec4;
template <> struct Vec4<double> { using T = double4_32a; };
template <> struct Vec4<float> { using T = float4; };

template <class To, class From>
__device__ __forceinline__ void cvt4(const From& a, To (&o)[4]) {
  o[0] = (To)a.x; o[1] = (To)a.y; o[2] = (To)a.z; o[3] = (To)a.w;
}

// ---------------------------------------------------------------------------
// exp(-i T dt) e_1 on one warp: lane j holds component j+1 (k <= 32).
// X = (T - c0) / half has its spectrum in [-1, 1]; exp(-i R X) with
// R = half * dt is sum_n eps_n (-i)^n J_n(R) T_n(X) (Jacobi-Anger), summed
// with the three-term Chebyshev recurrence T_{n+1} = 2 X T_n - T_{n-1}.
// ---------------------------------------------------------------------------
__device__ inline void cheb_expm_e1(const ChebParams& cp, int k, double alpha_j, double beta_lo,
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
// Scalar update of one problem after pass i: run by one warp with the grid
// totals P, Y, X in every lane.  Values written by earlier launches are read
// with plain loads up front; new values travel by shuffles.  rsqrt gives
// sqrt(X), 1/X, sqrt(s2) and 1/sqrt(s2) with few dependent FP64 operations.
// ---------------------------------------------------------------------------
__device__ inline void finish_pass(const LaunchParams& lp, const Problem* pr, DevState* st, int i, double P,
                                   double Y, double X) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const double shift = pr->shift;
  const bool ok = isfinite(P) && isfinite(Y) && isfinite(X) && X > 0.0;
  // psi = 0 exactly: exp(-i H dt) 0 = 0, a step that changes nothing
  const bool zero = X == 0.0 && P == 0.0 && Y == 0.0;
  if (lp.probe) {   // Rayleigh quotient of psi: the first stencil shift
    if (lane == 0) {
      if (ok || zero) {
        const double s1 = ok ? P / X : 0.0;   // the probe ran with stencil shift 0
        st->sigma[1] = s1;
        st->pc_cur = make_coef(1.0, 0.0, 0.0, lp.mcc - shift - s1, -lp.mcc - shift - s1);
        st->cur_pass = 1;
        st->redo_left = lp.redo_budget;
        st->sigma_valid = 1;
      } else {
        st->error = ERR_NONFINITE; st->stopped = 1;
      }
    }
    return;
  }
  if (zero && i == 1) {   // recombination with C_1 = 0 keeps psi = 0
    if (lane == 0) {
      st->nu[1] = 0.0;
      st->inv_nu[1] = 0.0;
      st->alpha[1] = st->sigma[1];
      st->beta[1] = 0.0;
      st->coef_re[1] = 0.0;
      st->coef_im[1] = 0.0;
      st->psi_norm = 0.0;
      st->energy = 0.0;          // no state, no energy
      st->err_est = 0.0;
      st->k_used = 1;
      st->breakdown = 1;
      st->beta_last = 0.0;
      st->pc_cur = make_coef(1.0, 0.0, 0.0, lp.mcc - shift - st->sigma[1], -lp.mcc - shift - st->sigma[1]);
      st->sigma_valid = 1;
      st->stopped = 1;
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
  const double alpha1_old = (i == 1) ? 0.0 : st->alpha[1];
  const double psi_norm_old = st->psi_norm, cum_old = st->cum_err;
  const int redo_left = st->redo_left;
  // candidates for the next pass's stencil shift: alpha_{i+1} of the previous
  // step (still in place: this step has not reached pass i + 1) and
  // alpha_{i-1} of this one
  const int k_prev = st->k_used;
  const double alpha_next_prev = (i + 1 <= k_prev && i + 1 <= KMAX) ? st->alpha[i + 1] : 0.0;
  const double alpha_im1 = (i >= 2) ? st->alpha[i - 1] : 0.0;
  const PassCoef pc_now = st->pc_cur;
  __syncwarp();   // every lane has read the state before lane 0 updates it

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
  // The stencil shift sigma_i was too far from alpha_i for the precision of
  // y^ (s2 is then cancellation noise): run pass i again with sigma_i =
  // alpha_i, which makes s2 ~ Y.  Everything derived from X (nu, beta_{i-1})
  // is unchanged by the re-run.
  if ((!(s2 > 0.0) || Y > lp.kappa_redo * s2) && redo_left > 0) {
    if (lane == 0) {
      st->redo_left = redo_left - 1;
      st->sigma[i] = alpha;
      st->pc_cur = make_coef(pc_now.g, pc_now.gd, pc_now.e, lp.mcc - shift - alpha,
                             -lp.mcc - shift - alpha);
      if (s2 > 0.0) st->kappa_max = fmax(st->kappa_max, Y * rs * rs);
    }
    return;
  }
  double scale = fmax(scale_old, fabs(alpha + shift));
  if (i > 1) scale = fmax(scale, bprev);
  const int brk = beta_hat <= 1e-12 * scale;
  int stop = (i >= lp.m) || brk;
  const double nu1 = (i == 1) ? nu : nu1_old;
  const double psi_norm = (i == 1) ? nu : psi_norm_old;
  if (lane == 0) {
    st->nu[i] = nu;
    st->inv_nu[i] = y;
    st->alpha[i] = alpha;
    st->beta[i] = beta_hat;
    if (i > 1) st->beta[i - 1] = bprev;
    st->scale = scale;
    if (i == 1) { st->psi_norm = nu; st->energy = alpha + shift; }
    if (s2 > 0.0) st->kappa_max = fmax(st->kappa_max, Y * rs * rs);
    if (!stop) {
      // The stencil shift of pass i + 1, a prediction of alpha_{i+1} (any
      // value is exact; a close one keeps s2 free of cancellation).  T hardly
      // changes from one step to the next -- for static fields its entries
      // are moments of H in psi, which the propagation conserves -- so the
      // previous step's alpha_{i+1} is the best guess when that step got so
      // far.  Else alpha_{i-1}: the Krylov vectors of a positive-energy packet
      // with a small negative-energy admixture alternate between the two
      // bands, so alpha_{i+1} is close to alpha_{i-1}, not to alpha_i.
      const double sig = (i + 1 <= k_prev) ? alpha_next_prev : (i >= 2 ? alpha_im1 : alpha);
      st->sigma[i + 1] = sig;
      st->pc_prev = pc_now;
      st->pc_cur = make_coef(rs, rs * dd, sq * rX, lp.mcc - shift - sig, -lp.mcc - shift - sig);
      st->cur_pass = i + 1;
    }
  }
  // this lane's row of T^(i)
  const double a_j = (lane + 1 == i) ? alpha : a_old;
  const double b_hi = (lane + 2 == i) ? bprev : b_old;               // couples j+1, j+2
  const double b_lo = __shfl_up_sync(full, b_hi, 1);                 // couples j, j+1
  const double inv_nu_j = (lane + 1 == i) ? y : invnu_old;
  double vr = 0.0, vi = 0.0;
  bool have_v = false;
  if (!stop && lp.tol > 0.0) {   // adaptive Krylov dimension (Sec. 4, Eq. 18)
    cheb_expm_e1(*pr->cheb, i, a_j, b_lo, b_hi, vr, vi);
    have_v = true;
    const double vk = __shfl_sync(full, sqrt(vr * vr + vi * vi), i - 1);
    stop = (beta_hat * lp.dt * vk <= lp.tol);
  }
  if (!stop) return;
  if (!have_v) cheb_expm_e1(*pr->cheb, i, a_j, b_lo, b_hi, vr, vi);
  // C_j = nu_1 / nu_j * v_j applied to q^_j; Eq. 18 estimate from v_k
  const double vk = __shfl_sync(full, sqrt(vr * vr + vi * vi), i - 1);
  if (lane < i) {
    const double f = nu1 * inv_nu_j;
    st->coef_re[lane + 1] = f * vr;
    st->coef_im[lane + 1] = lp.conj_coef ? -f * vi : f * vi;   // T real: exp(+iT dt) e_1 = conj(exp(-iT dt) e_1)
  }
  if (lane == 0) {
    const double err = lp.dt * beta_hat * psi_norm * vk;
    st->err_est = err;
    st->cum_err = cum_old + err;
    st->k_used = i;
    st->breakdown = brk;
    st->beta_last = beta_hat;
    const double s1 = (i == 1) ? alpha : alpha1_old;   // next step's first shift
    st->sigma[1] = s1;
    st->pc_cur = make_coef(1.0, 0.0, 0.0, lp.mcc - shift - s1, -lp.mcc - shift - s1);
    st->sigma_valid = 1;
    st->stopped = 1;
  }
}

// ---------------------------------------------------------------------------
// One Lanczos iteration over every problem of the table: stencil product
// with fused reductions.
//
// S    arithmetic type of the stencil (double: FP64 path; float: mixed path)
// R    stencil half width (1: order 2, 2: order 4)
// TH   tile height in sites (tiles are TILE_W x TH; TH / RPT warps per tile
//      worker, RPT rows per thread)
//
// Each problem runs its own next pass (DevState::cur_pass), so that a pass
// can be re-run (see finish_pass) without the host knowing.  q^_{i-1} (and
// psi) are complex128 on the FP64 path and in passes 1-2 of the mixed path
// (whose q^_1 is the FP64 state itself), else complex64.
//
// Thread (tx, tg) handles column tx and rows tg, tg + NG, ..., so every warp
// touches one contiguous row segment per access.  The tile and a
// cross-shaped halo of q^_i are formed in shared memory from y^_{i-1} and
// q^_{i-1}.
// ---------------------------------------------------------------------------
template <class S, int TH, int SUB>
__host__ __device__ constexpr int min_blocks() { return sizeof(S) == sizeof(float) ? (TH == 32 ? 4 : 8) : (SUB == 2 ? 1 : 2); }

// rows per thread: four, except two on FP64 16-row tiles, which keep eight
// warps per tile worker and halve the unit of work: a grid of a few tiles per
// worker then ends with a shorter partial round
template <class S, int TH>
__host__ __device__ constexpr int rows_per_thread() { return (sizeof(S) == sizeof(double) && TH == 16) ? 2 : 4; }

// tile workers per CTA: two on the FP64 path (one CTA per SM), one otherwise
template <class S>
__host__ __device__ constexpr int sub_workers() { return sizeof(S) == sizeof(double) ? 2 : 1; }

// shared memory of one tile worker: the tile of q^_i with its halo, and on
// the mixed path the staging buffer of q^_{i-1} on the same rectangle
template <class S, int R, int TH>
__host__ __device__ constexpr size_t tile_bytes() { return sizeof(S) * 4 * (TH + 2 * R) * (TILE_W + 2 * R); }
template <class S, int R, int TH>
__host__ __device__ constexpr size_t qbuf_bytes() {
  return sizeof(S) == sizeof(float) ? sizeof(float4) * (TH + 2 * R) * (TILE_W + 2 * R) : 0;
}
template <class S, int R, int TH>
__host__ __device__ constexpr size_t worker_bytes() { return tile_bytes<S, R, TH>() + qbuf_bytes<S, R, TH>(); }

// tile workers per CTA of the one-launch step: one CTA per SM on both paths
// (two workers of eight warps on FP64; 768 threads on FP32 -- six 128-thread
// or three 256-thread workers, 80 registers each, where 1024 threads at 64
// registers spilled), so that a grid barrier and its partial sums involve one
// CTA per SM
template <class S, int TH>
__host__ __device__ constexpr int step_workers() {
  return sizeof(S) == sizeof(double) ? 2 : 768 / (32 * (TH / 4));
}

// Chunks of the tile list: CTA c takes q + 1 tiles if c < r, else q (q = T / G,
// r = T % G), starting at c q + min(c, r).  The CTA whose chunk holds tile t:
__device__ __forceinline__ int cta_of_tile(int t, int q, int r) {
  const int big = r * (q + 1);
  return t < big ? t / (q + 1) : r + (t - big) / q;
}

// shared memory of the tile workers: a static array for one worker, the
// dynamic allocation for several (more than the 48 KiB of static memory)
template <class S, int R, int TH, int SUB>
__host__ __device__ constexpr size_t dyn_smem_bytes() { return SUB == 1 ? 0 : SUB * worker_bytes<S, R, TH>(); }

// The body of one pass over this CTA's chunk.  COOP = false: a launch of
// its own (lanczos_pass): per-problem tickets, the last CTA finishes.
// COOP = true: inside the one-launch step (lanczos_step): one problem, the
// state read from `coop_st`, coherent loads, and the CTA's partial sums
// written to coop_slots[3 * blockIdx.x ...]; the caller synchronises the grid
// and finishes.
template <class S, int R, int TH, bool DIRI, bool HAS_V, bool HAS_AY, bool COOP, int SUB>
__device__ __forceinline__ void pass_body(const LaunchParams& lp, const DevState* coop_st, double* coop_slots,
                                          int step) {
  using T4 = typename Vec4<S>::T;           // storage of y^ (and of q^ on the mixed path)
  constexpr int RPT = rows_per_thread<S, TH>();
  constexpr int NG = TH / RPT;              // row groups = warps of a worker
  constexpr int NTS = 32 * NG;              // threads of a worker
  constexpr int NT = SUB * NTS;             // threads
  constexpr int NW = SUB * NG;              // warps
  constexpr int W = TILE_W + 2 * R;
  extern __shared__ __align__(32) unsigned char dyn_smem[];
  __shared__ double red[NW][3];
  __shared__ int last_flag;

  const int cq = lp.chunk_q, cr = lp.chunk_r;
  const int t_begin = blockIdx.x * cq + min((int)blockIdx.x, cr);
  const int t_end = t_begin + cq + ((int)blockIdx.x < cr ? 1 : 0);
  const int sub = SUB == 1 ? 0 : (int)threadIdx.x / NTS;   // this thread's worker
  const int ltid = (int)threadIdx.x - sub * NTS;
  const int tx = ltid & 31, tg = ltid >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr bool F32 = sizeof(S) == sizeof(float);
  __shared__ __align__(32) S tile_s[SUB == 1 ? TH + 2 * R : 1][W][4];
  S(*const tile)[W][4] = SUB == 1 ? &tile_s[0]
                                  : reinterpret_cast<S(*)[W][4]>(dyn_smem + sub * worker_bytes<S, R, TH>());
  // mixed path, passes >= 3: q^_{i-1} on the tile and halo, copied asynchronously
  constexpr int NSQ = (F32 && SUB == 1) ? (TH + 2 * R) * W : 1;
  __shared__ __align__(16) float4 qbuf_s[NSQ];
  float4* const qbuf = SUB == 1 ? qbuf_s
                                : reinterpret_cast<float4*>(dyn_smem + sub * worker_bytes<S, R, TH>() +
                                                            tile_bytes<S, R, TH>());
  // barrier of this worker's threads (the whole CTA when there is one worker)
  auto sub_sync = [&]() {
    if constexpr (SUB == 1) {
      __syncthreads();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(1 + sub), "r"(NTS) : "memory");
    }
  };

  // problem of the first tile (problems are sorted by tile_begin)
  int b = 0;
  {
    int lo = 0, hi = lp.nprob - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (lp.probs[mid].tile_begin <= t_begin) lo = mid; else hi = mid - 1;
    }
    b = lo;
  }
  for (int t = t_begin; t < t_end; ++b) {
    const Problem* pr = lp.probs + b;
    const DevState* st = COOP ? coop_st : lp.states + b;
    // independent loads first (all addresses are valid), then the branch
    const int stopped = st->stopped;
    const int i = lp.probe ? 1 : max(1, st->cur_pass);
    const PassCoef pc = lp.probe ? pr->probe_coef : st->pc_cur;
    const FieldStep fs = lp.fields[step * lp.fstride + b];
    const int seg_end = min(t_end, pr->tile_begin + pr->ntiles);
    const int seg_tiles = seg_end - t;
    if (stopped) { t = seg_end; continue; }
    const S gS = F32 ? (S)pc.gf : (S)pc.g;
    const S gdS = F32 ? (S)pc.gdf : (S)pc.gd;
    const S eS = F32 ? (S)pc.ef : (S)pc.e;
    const S kx = F32 ? (S)pr->kxf : (S)pr->kx, ky = F32 ? (S)pr->kyf : (S)pr->ky;
    const S cAx = F32 ? (S)fs.cAxf : (S)fs.cAx, cAy = F32 ? (S)fs.cAyf : (S)fs.cAy;
    const S au_hi = F32 ? (S)pc.au_hi : (S)pc.au0, au_lo = F32 ? (S)pc.au_lo : S(0);
    const S ad_hi = F32 ? (S)pc.ad_hi : (S)pc.ad0, ad_lo = F32 ? (S)pc.ad_lo : S(0);
    // FP32: remainders of the stencil and vector-potential coefficients
    const S kx_lo = F32 ? (S)pr->kxf_lo : S(0), ky_lo = F32 ? (S)pr->kyf_lo : S(0);
    const S cAx_lo = F32 ? (S)fs.cAxf_lo : S(0), cAy_lo = F32 ? (S)fs.cAyf_lo : S(0);
    const int nx = pr->nx, ny = pr->ny;
    const size_t n = (size_t)nx * ny;
    // this pass's vectors
    constexpr int SB = F32 ? (int)sizeof(float4) : (int)sizeof(double4_32a);
    const char* basis = static_cast<const char*>(pr->basis);
    const void* y_prev = (i >= 2) ? (((i - 1) & 1) ? pr->ybuf1 : pr->ybuf0) : nullptr;
    const void* q_prev = (i == 2) ? (const void*)pr->psi
                                  : (i >= 3 ? (const void*)(basis + (size_t)(i - 3) * n * SB) : nullptr);
    void* q_out = (i >= 2) ? (void*)(basis + (size_t)(i - 2) * n * SB) : nullptr;
    void* y_out = (i < lp.m) ? ((i & 1) ? pr->ybuf1 : pr->ybuf0) : nullptr;
    const T4* yprev = static_cast<const T4*>(y_prev);
    const bool q64 = !F32 || i <= 2;                // q^_{i-1} stored as complex128
    const S* Vp = static_cast<const S*>(pr->V);   // NULL: V = 0 for this problem
    const float* Vlo = static_cast<const float*>(pr->Vlo);   // mixed path: V - (float)V, or NULL

    // q^_i at grid point (gx, gy) (zero outside for Dirichlet) into smem slot
    auto form = [&](int gx, int gy, int row, int col, S (&qp)[4]) {
      bool ox, oy;
      const int ix = wrap<DIRI>(gx, nx, ox), iy = wrap<DIRI>(gy, ny, oy);
      S q[4] = {S(0), S(0), S(0), S(0)};
      qp[0] = qp[1] = qp[2] = qp[3] = S(0);
      if (!(ox || oy)) {
        const size_t idx = (size_t)iy * nx + ix;
        if (q64) {
          const vec4* qsrc = (i == 1) ? pr->psi : static_cast<const vec4*>(q_prev);
          cvt4(ld4<COOP>(qsrc + idx), qp);
        } else {
          cvt4(ld4<COOP>(static_cast<const float4*>(q_prev) + idx), qp);
        }
        if (i == 1) {
#pragma unroll
          for (int c = 0; c < 4; ++c) q[c] = qp[c];
        } else {
          S yv[4];
          cvt4(ld4<COOP>(yprev + idx), yv);
#pragma unroll
          for (int c = 0; c < 4; ++c) q[c] = fma(-gdS, qp[c], gS * yv[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) tile[row][col][c] = q[c];
    };

    S accP = S(0), accY = S(0), accX = S(0);
    // y^_i at one site from q^_i there (C) and its differences, q^_{i-1}
    // (qp) and V; stores q^_i and y^_i and accumulates P, Y, X
    auto site_update = [&](size_t idx, const S (&C)[4], const S (&dxv)[4], const S (&dyv)[4],
                           const S (&qp)[4]) {
      S au, ad, aul = au_lo, adl = ad_lo;
      if (HAS_V && Vp != nullptr) {   // V stored in S (float copy on the mixed path)
        const S v = Vp[idx];
        if constexpr (F32) {
          // the FP32 sum with the diagonal (up to 2 m c^2) rounds differently at
          // every site: its error and V's own remainder go into the low part
          float ru, rd;
          two_sum(au_hi, v, au, ru);
          two_sum(ad_hi, v, ad, rd);
          const float vl = Vlo ? Vlo[idx] : 0.f;
          aul = au_lo + vl + ru;
          adl = ad_lo + vl + rd;
        } else {
          au = au_hi + v;
          ad = ad_hi + v;
        }
      } else {
        au = au_hi;
        ad = ad_hi;
      }
      // C = (u.re, u.im, d.re, d.im); dxv/dyv likewise
      S yv[4];
      // upper: (mc^2+V-s-sigma) u + c[-i D_x d - D_y d + (A_x - i A_y) d]
      yv[0] = au * C[0] + kx * dxv[3] - ky * dyv[2] + cAx * C[2];
      yv[1] = au * C[1] - kx * dxv[2] - ky * dyv[3] + cAx * C[3];
      // lower: (-mc^2+V-s-sigma) d + c[-i D_x u + D_y u + (A_x + i A_y) u]
      yv[2] = ad * C[2] + kx * dxv[1] + ky * dyv[0] + cAx * C[0];
      yv[3] = ad * C[3] - kx * dxv[0] + ky * dyv[1] + cAx * C[1];
      if constexpr (HAS_AY) {   // else A_y = 0 in every step of the launch
        yv[0] = fma(cAy, C[3], yv[0]);
        yv[1] = fma(-cAy, C[2], yv[1]);
        yv[2] = fma(-cAy, C[1], yv[2]);
        yv[3] = fma(cAy, C[0], yv[3]);
      }
      if constexpr (F32) {
        yv[0] = fma(aul, C[0], fma(kx_lo, dxv[3], fma(-ky_lo, dyv[2], fma(cAx_lo, C[2], yv[0]))));
        yv[1] = fma(aul, C[1], fma(-kx_lo, dxv[2], fma(-ky_lo, dyv[3], fma(cAx_lo, C[3], yv[1]))));
        yv[2] = fma(adl, C[2], fma(kx_lo, dxv[1], fma(ky_lo, dyv[0], fma(cAx_lo, C[0], yv[2]))));
        yv[3] = fma(adl, C[3], fma(-kx_lo, dxv[0], fma(ky_lo, dyv[1], fma(cAx_lo, C[1], yv[3]))));
        if constexpr (HAS_AY) {
          yv[0] = fma(cAy_lo, C[3], yv[0]);
          yv[1] = fma(-cAy_lo, C[2], yv[1]);
          yv[2] = fma(-cAy_lo, C[1], yv[2]);
          yv[3] = fma(cAy_lo, C[0], yv[3]);
        }
      }
      if (i >= 2) {
#pragma unroll
        for (int q = 0; q < 4; ++q) yv[q] = fma(-eS, qp[q], yv[q]);
      }
      if (!lp.probe) {
        if (q_out) {
          T4 o; o.x = C[0]; o.y = C[1]; o.z = C[2]; o.w = C[3];
          static_cast<T4*>(q_out)[idx] = o;
        }
        if (y_out) {
          T4 o; o.x = yv[0]; o.y = yv[1]; o.z = yv[2]; o.w = yv[3];
          static_cast<T4*>(y_out)[idx] = o;
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        accP = fma(C[q], yv[q], accP);
        accY = fma(yv[q], yv[q], accY);
        accX = fma(C[q], C[q], accX);
      }
    };
    // the stencil on the formed tile; qprev(k, r, c) gives q^_{i-1} of row k
    auto stencil_rows = [&](int x0, int y0, auto&& qprev) {
#pragma unroll
      for (int k = 0; k < RPT; ++k) {
        const int ry = tg + k * NG;
        const int x = x0 + tx, y = y0 + ry;
        if (x < nx && y < ny) {
          const size_t idx = (size_t)y * nx + x;
          const int r = ry + R, c = tx + R;
          S C[4], dxv[4], dyv[4], qp[4];
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
          qprev(k, r, c, qp);
          site_update(idx, C, dxv, dyv, qp);
        }
      }
    };

    bool done_async = false;
    if constexpr (F32) {
     if (!q64 && lp.async_tiles) {
      done_async = true;
      // mixed path, passes >= 3: y^_{i-1} and q^_{i-1} of the tile and its
      // halo (a full rectangle) go to shared memory by asynchronous copies,
      // all in flight at once and without registers; q^_i is formed in place
      constexpr int NS = (TH + 2 * R) * W;
      float4* const tf = reinterpret_cast<float4*>(&tile[0][0][0]);
      const float4* const qsrc = static_cast<const float4*>(q_prev);
      for (int tt = t + sub; tt < seg_end; tt += SUB) {
        const int lt = tt - pr->tile_begin;
        const int x0 = (lt % pr->tiles_x) * TILE_W;
        const int y0 = (lt / pr->tiles_x) * TH;
        for (int e = ltid; e < NS; e += NTS) {
          const int r = e / W, c = e - r * W;
          bool ox, oy;
          const int ix = wrap<DIRI>(x0 - R + c, nx, ox), iy = wrap<DIRI>(y0 - R + r, ny, oy);
          const bool in = !(ox || oy);
          const size_t idx = in ? (size_t)iy * nx + ix : 0;
          cp_async16(tf + e, reinterpret_cast<const float4*>(yprev) + idx, in ? 16 : 0);
          cp_async16(qbuf + e, qsrc + idx, in ? 16 : 0);
        }
        cp_async_commit_wait();
        sub_sync();
        for (int e = ltid; e < NS; e += NTS) {
          const float4 yv = tf[e], qp = qbuf[e];
          tf[e] = make_float4(fmaf(-(float)gdS, qp.x, (float)gS * yv.x), fmaf(-(float)gdS, qp.y, (float)gS * yv.y),
                              fmaf(-(float)gdS, qp.z, (float)gS * yv.z), fmaf(-(float)gdS, qp.w, (float)gS * yv.w));
        }
        sub_sync();
        stencil_rows(x0, y0, [&](int, int r, int c, S (&qp)[4]) {
          const float4 v = qbuf[r * W + c];
          qp[0] = (S)v.x; qp[1] = (S)v.y; qp[2] = (S)v.z; qp[3] = (S)v.w;
        });
        sub_sync();   // tile and qbuf are reused next
      }
     }
    }
    if (!done_async) {
      for (int tt = t + sub; tt < seg_end; tt += SUB) {
        const int lt = tt - pr->tile_begin;
        const int x0 = (lt % pr->tiles_x) * TILE_W;
        const int y0 = (lt / pr->tiles_x) * TH;
        S qprev[RPT][4];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
          const int r = tg + k * NG;
          form(x0 + tx, y0 + r, r + R, tx + R, qprev[k]);
        }
        constexpr int NH_ROW = 2 * R * TILE_W, NH = NH_ROW + 2 * R * TH;
        for (int h = ltid; h < NH; h += NTS) {
          int row, col;
          if (h < NH_ROW) {               // rows above / below
            const int r = h / TILE_W;
            row = (r < R) ? r : TH + r;
            col = (h % TILE_W) + R;
          } else {                        // columns left / right
            const int h2 = h - NH_ROW;
            row = h2 / (2 * R) + R;
            const int c = h2 % (2 * R);
            col = (c < R) ? c : TILE_W + c;
          }
          S dummy[4];
          form(x0 + col - R, y0 + row - R, row, col, dummy);
        }
        sub_sync();
        stencil_rows(x0, y0, [&](int k, int, int, S (&qp)[4]) {
#pragma unroll
          for (int q = 0; q < 4; ++q) qp[q] = qprev[k][q];
        });
        sub_sync();   // the tile buffer is reused next
      }
    }
    t = seg_end;

    // this CTA's share of the problem: thread -> warp in S, warps -> CTA in
    // double, one partial per (problem, CTA) slot, then the ticket
    accP = warp_sum(accP);
    accY = warp_sum(accY);
    accX = warp_sum(accX);
    if (lane == 0) { red[warp][0] = (double)accP; red[warp][1] = (double)accY; red[warp][2] = (double)accX; }
    __syncthreads();
    if (warp == 0) {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      if (lane < NW) { s0 = red[lane][0]; s1 = red[lane][1]; s2 = red[lane][2]; }
#pragma unroll
      for (int o = (NW > 16 ? 16 : 8); o > 0; o >>= 1) {   // NW <= 32 warps
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      }
      if (lane == 0) {
        if constexpr (COOP) {
          coop_slots[3 * blockIdx.x + 0] = s0;
          coop_slots[3 * blockIdx.x + 1] = s1;
          coop_slots[3 * blockIdx.x + 2] = s2;
          last_flag = 0;
        } else {
          const int slot = blockIdx.x - cta_of_tile(pr->tile_begin, cq, cr);
          pr->partials[3 * slot + 0] = s0;
          pr->partials[3 * slot + 1] = s1;
          pr->partials[3 * slot + 2] = s2;
          // release our partial / acquire everybody else's
          cuda::atomic_ref<unsigned, cuda::thread_scope_device> ticket(pr->st->counter);
          last_flag = (ticket.fetch_add((unsigned)seg_tiles, cuda::memory_order_acq_rel) + seg_tiles ==
                       (unsigned)pr->ntiles);
        }
      }
    }
    __syncthreads();
    if (!COOP && last_flag) {
      // the problem is complete: the whole CTA sums its slots in a fixed
      // order (thread-strided, the warp tree, then the warps in turn), the
      // loads of SB slots per thread in flight at once, so that a pass of
      // eight CTAs per SM waits for two L2 round trips here, not five
      const int cta_lo = cta_of_tile(pr->tile_begin, cq, cr);
      const int nslots = cta_of_tile(pr->tile_begin + pr->ntiles - 1, cq, cr) - cta_lo + 1;
      constexpr int SB = 5;
      double t0 = 0.0, t1 = 0.0, t2 = 0.0;
      for (int s0 = threadIdx.x; s0 < nslots; s0 += SB * NT) {
        double v[SB][3];
#pragma unroll
        for (int k = 0; k < SB; ++k) {
          const int s = s0 + k * NT;
          const double* ps = pr->partials + 3 * (s < nslots ? s : 0);
          v[k][0] = s < nslots ? __ldcg(ps + 0) : 0.0;
          v[k][1] = s < nslots ? __ldcg(ps + 1) : 0.0;
          v[k][2] = s < nslots ? __ldcg(ps + 2) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < SB; ++k) { t0 += v[k][0]; t1 += v[k][1]; t2 += v[k][2]; }
      }
      t0 = warp_sum(t0);
      t1 = warp_sum(t1);
      t2 = warp_sum(t2);
      if (lane == 0) { red[warp][0] = t0; red[warp][1] = t1; red[warp][2] = t2; }
      __syncthreads();
      if (warp == 0) {
        t0 = red[0][0]; t1 = red[0][1]; t2 = red[0][2];
#pragma unroll
        for (int w = 1; w < NW; ++w) { t0 += red[w][0]; t1 += red[w][1]; t2 += red[w][2]; }
        if (lane == 0) pr->st->counter = 0u;
        finish_pass(lp, pr, pr->st, i, t0, t1, t2);
      }
    }
    __syncthreads();
  }
}

template <class S, int R, int TH, bool DIRI, bool HAS_V, bool HAS_AY>
__global__ void __launch_bounds__(sub_workers<S>() * 32 * (TH / rows_per_thread<S, TH>()),
                                  (min_blocks<S, TH, sub_workers<S>()>()))
lanczos_pass(const __grid_constant__ LaunchParams lp) {
  // programmatic dependent launch: nothing the previous kernel wrote is read
  // before this point
  asm volatile("griddepcontrol.wait;" ::: "memory");
  pass_body<S, R, TH, DIRI, HAS_V, HAS_AY, false, sub_workers<S>()>(lp, nullptr, nullptr, *lp.step);
  // the next kernel may be scheduled now (it waits for our completion)
  asm volatile("griddepcontrol.launch_dependents;");
}

// psi <- C_1 psi + sum_{j >= 2} C_j q^_j at site s: the complex64 basis
// terms accumulated in compensated FP32 (coefficients as FP32 pairs, exact
// products, two-sum accumulation), added to the FP64 term C_1 psi at the end.
// Loads of DEPTH basis vectors are issued before their products (more loads
// in flight per thread, against more registers).
template <int DEPTH>
__device__ __forceinline__ void recombine_site_df(vec4* psi, const float4* basis, size_t n, size_t s, int k,
                                                  const double* cr, const double* ci, const float* crh,
                                                  const float* crl, const float* cih, const float* cil) {
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, e0 = 0.f, e1 = 0.f, e2 = 0.f, e3 = 0.f;
  for (int j0 = 2; j0 <= k; j0 += DEPTH) {
    float4 v[DEPTH];
#pragma unroll
    for (int u = 0; u < DEPTH; ++u)
      if (j0 + u <= k) v[u] = __ldcs(basis + (size_t)(j0 + u - 2) * n + s);
#pragma unroll
    for (int u = 0; u < DEPTH; ++u) {
      if (j0 + u <= k) {
        const int j = j0 + u;
        const float ah = crh[j], al = crl[j], bh = cih[j], bl = cil[j];
        // (a + i b)(q.re + i q.im) for the upper (x, y) and lower (z, w) component
        acc_prod(ah, al, v[u].x, s0, e0);
        acc_prod(-bh, -bl, v[u].y, s0, e0);
        acc_prod(ah, al, v[u].y, s1, e1);
        acc_prod(bh, bl, v[u].x, s1, e1);
        acc_prod(ah, al, v[u].z, s2, e2);
        acc_prod(-bh, -bl, v[u].w, s2, e2);
        acc_prod(ah, al, v[u].w, s3, e3);
        acc_prod(bh, bl, v[u].z, s3, e3);
      }
    }
  }
  const vec4 q = psi[s];
  const double ar = cr[1], ai = ci[1];
  vec4 o;
  o.x = fma(ar, q.x, fma(-ai, q.y, (double)s0 + (double)e0));
  o.y = fma(ar, q.y, fma(ai, q.x, (double)s1 + (double)e1));
  o.z = fma(ar, q.z, fma(-ai, q.w, (double)s2 + (double)e2));
  o.w = fma(ar, q.w, fma(ai, q.z, (double)s3 + (double)e3));
  psi[s] = o;
}

// ---------------------------------------------------------------------------
// psi <- sum_j C_j q^_j (Eq. 17), q^_1 = psi, q^_j = basis[j-2] for j >= 2.
// FP64 path: complex128 throughout.  Mixed path: the basis is complex64;
// C_1 psi is formed in FP64 so that the FP32 rounding of the basis only
// enters the (small) Krylov corrections, and those are summed with
// compensation (recombine_site_df): plain FP32 accumulation of the
// corrections was the largest error of the mixed path on fast packets.
// Blocks are dealt to problems in proportion to their size.
// ---------------------------------------------------------------------------
template <bool MIXED>
__device__ __forceinline__ void recombine_site(vec4* psi, const void* basis_v, long long n, long long s, int k,
                                               const double* cr, const double* ci, const float* fr,
                                               const float* fi) {
  if constexpr (!MIXED) {
    const vec4* basis = static_cast<const vec4*>(basis_v);
    const vec4 q = psi[s];
    double ur = cr[1] * q.x - ci[1] * q.y, ui = cr[1] * q.y + ci[1] * q.x;
    double dr = cr[1] * q.z - ci[1] * q.w, di = cr[1] * q.w + ci[1] * q.z;
    for (int j = 2; j <= k; ++j) {
      const vec4* vp = basis + (size_t)(j - 2) * n + s;
      const vec4 v = *vp;
      const double a = cr[j], bb = ci[j];
      ur = fma(a, v.x, fma(-bb, v.y, ur));
      ui = fma(a, v.y, fma(bb, v.x, ui));
      dr = fma(a, v.z, fma(-bb, v.w, dr));
      di = fma(a, v.w, fma(bb, v.z, di));
    }
    vec4 o;
    o.x = ur; o.y = ui; o.z = dr; o.w = di;
    psi[s] = o;
  } else {
    const float4* basis = static_cast<const float4*>(basis_v);
    const double ar = cr[1], ai = ci[1];
    float ur = 0.f, ui = 0.f, dr = 0.f, di = 0.f;
    for (int j = 2; j <= k; ++j) {
      const float4* vp = basis + (size_t)(j - 2) * n + s;
      const float4 v = *vp;
      const float a = fr[j], bb = fi[j];
      ur = fmaf(a, v.x, fmaf(-bb, v.y, ur));
      ui = fmaf(a, v.y, fmaf(bb, v.x, ui));
      dr = fmaf(a, v.z, fmaf(-bb, v.w, dr));
      di = fmaf(a, v.w, fmaf(bb, v.z, di));
    }
    const vec4 q = psi[s];
    vec4 o;
    o.x = fma(ar, q.x, fma(-ai, q.y, (double)ur));
    o.y = fma(ar, q.y, fma(ai, q.x, (double)ui));
    o.z = fma(ar, q.z, fma(-ai, q.w, (double)dr));
    o.w = fma(ar, q.w, fma(ai, q.z, (double)di));
    psi[s] = o;
  }
}

// Three CTAs per SM (at most 85 registers), so that enough warps keep loads
// in flight: the compensated sums make the mixed form arithmetic-heavy.
template <bool MIXED>
__global__ void __launch_bounds__(256, 3) recombine(const __grid_constant__ RecombParams rp) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __shared__ double cr[KMAX + 2], ci[KMAX + 2];
  __shared__ float fr[KMAX + 2], fi[KMAX + 2], frl[KMAX + 2], fil[KMAX + 2];
  __shared__ int k_s, err_s;
  const int b = rp.blk_prob[blockIdx.x];
  const Problem* pr = rp.probs + b;
  DevState* st = pr->st;
  if (threadIdx.x == 0) { k_s = st->k_used; err_s = st->error; }
  if (threadIdx.x <= KMAX) {
    const double a = st->coef_re[threadIdx.x], c = st->coef_im[threadIdx.x];
    cr[threadIdx.x] = a;
    ci[threadIdx.x] = c;
    fr[threadIdx.x] = (float)a;
    fi[threadIdx.x] = (float)c;
    frl[threadIdx.x] = (float)(a - (double)fr[threadIdx.x]);
    fil[threadIdx.x] = (float)(c - (double)fi[threadIdx.x]);
  }
  __syncthreads();
  const int lb = blockIdx.x - pr->rblk_begin;
  if (blockIdx.x == 0 && threadIdx.x == 0) *rp.step += 1;   // the next step's fields
  if (err_s) return;                                         // leave psi untouched
  if (lb == 0 && threadIdx.x == 0) {                         // re-arm the next step
    st->stopped = 0;
    st->cur_pass = 1;
    st->redo_left = rp.redo_budget;
  }
  const int k = k_s;
  const long long n = (long long)pr->nx * pr->ny;
  const long long stride = (long long)pr->rblk_count * blockDim.x;
  vec4* psi = const_cast<vec4*>(pr->psi);
  for (long long s = (long long)lb * blockDim.x + threadIdx.x; s < n; s += stride) {
    if constexpr (MIXED)
      recombine_site_df<8>(psi, static_cast<const float4*>(pr->basis), (size_t)n, (size_t)s, k, cr, ci, fr, frl,
                           fi, fil);
    else
      recombine_site<false>(psi, pr->basis, n, s, k, cr, ci, fr, fi);
  }
  asm volatile("griddepcontrol.launch_dependents;");
}

// ---------------------------------------------------------------------------
// One time step of one problem in one cooperative launch (every CTA
// resident): the passes separated by grid-wide barriers instead of kernel
// boundaries, then the recombination.  After each pass every CTA sums all
// CTA partials in the same fixed order and runs the scalar update on its own
// shared-memory copy of the state, so that all copies stay identical
// (bitwise: same inputs, same operations) and no second barrier is needed.
// Partials are double-buffered by pass parity: a CTA can run at most one
// pass ahead of the slowest one, which is still reading the other buffer.
// ---------------------------------------------------------------------------
constexpr int ERR_BARRIER = 8;                    // a grid barrier timed out
constexpr unsigned GRID_SYNC_SPIN_MAX = 1u << 20; // polls (~100 ns nap + an L2 round trip each: about a second)
constexpr int GRID_SYNC_WORDS = 4;                // arrivals, generation, timeout flag, spare

struct CoopArgs {
  double* slots;   // 2 x 3 x cap doubles: CTA partials (P, Y, X) by pass parity
  unsigned* bar;   // GRID_SYNC_WORDS words, zeroed before each launch
  int G;           // CTAs of the launch
  int cap;         // CTAs the slot buffer holds
  int bar_count;   // CTAs each grid barrier waits for: G (G + 1 only in the timeout test)
};

// Barrier of all CTAs of a cooperative launch.  Thread 0 of each CTA arrives
// (release of the CTA's writes, ordered by the __syncthreads before it) and
// waits for the generation to advance (acquire).  False after a timeout
// (bar[2] set), after which every waiting CTA gives up as well.  One counter
// and one polled word serve the one-CTA-per-SM launches of the FP64 path
// well; with many CTAs per SM their contention outweighs what the launch
// boundaries cost, which is why the FP32 path keeps per-pass launches.
__device__ __forceinline__ bool grid_sync(unsigned* bar, unsigned G) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned, cuda::thread_scope_device> arrived(bar[0]), gen(bar[1]), timeout(bar[2]);
    const unsigned g0 = gen.load(cuda::memory_order_acquire);
    int ok = 1;
    __threadfence();
    if (arrived.fetch_add(1u, cuda::memory_order_acq_rel) == G - 1u) {
      arrived.store(0u, cuda::memory_order_relaxed);
      gen.store(g0 + 1u, cuda::memory_order_release);
    } else {
      unsigned spins = 0;
      while (gen.load(cuda::memory_order_acquire) == g0) {
        if (timeout.load(cuda::memory_order_relaxed) != 0u || ++spins > GRID_SYNC_SPIN_MAX) {
          timeout.store(1u, cuda::memory_order_relaxed);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

template <class S, int R, int TH, bool DIRI, bool HAS_V, bool HAS_AY>
__global__ void __launch_bounds__(step_workers<S, TH>() * 32 * (TH / rows_per_thread<S, TH>()), 1)
lanczos_step(const __grid_constant__ LaunchParams lp, const __grid_constant__ CoopArgs ca) {
  constexpr bool F32 = sizeof(S) == sizeof(float);
  constexpr int SUB = step_workers<S, TH>();
  constexpr int NT = SUB * 32 * (TH / rows_per_thread<S, TH>());
  __shared__ DevState sst;
  __shared__ double cr_s[KMAX + 2], ci_s[KMAX + 2];
  __shared__ float fr_s[KMAX + 2], fi_s[KMAX + 2];
  const Problem* pr = lp.probs;
  DevState* gst = lp.states;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  {
    const unsigned* src = reinterpret_cast<const unsigned*>(gst);
    unsigned* dst = reinterpret_cast<unsigned*>(&sst);
    for (int w = threadIdx.x; w < (int)(sizeof(DevState) / sizeof(unsigned)); w += NT) dst[w] = __ldcg(src + w);
  }
  const int step = __ldcg(lp.step);
  __syncthreads();
  const int max_iter = lp.m + lp.redo_budget;
  int iter = 0;
  while (!sst.stopped && iter < max_iter) {
    const int i = max(1, sst.cur_pass);
    double* slots = ca.slots + (iter & 1) * 3 * ca.G;
    pass_body<S, R, TH, DIRI, HAS_V, HAS_AY, true, SUB>(lp, &sst, slots, step);
    ++iter;
    if (!grid_sync(ca.bar, (unsigned)ca.bar_count)) {
      if (threadIdx.x == 0) { gst->error = ERR_BARRIER; gst->stopped = 1; }
      return;   // psi untouched; the host reports the timeout
    }
    if (warp == 0) {   // the grid totals, in the same order in every CTA
      constexpr int SB = 4;   // loads in flight per lane
      double t0 = 0.0, t1 = 0.0, t2 = 0.0;
      for (int c0 = lane; c0 < ca.G; c0 += SB * 32) {
        double v[SB][3];
#pragma unroll
        for (int k = 0; k < SB; ++k) {
          const int c = c0 + k * 32;
          const double* ps = slots + 3 * (c < ca.G ? c : 0);
          v[k][0] = c < ca.G ? __ldcg(ps) : 0.0;
          v[k][1] = c < ca.G ? __ldcg(ps + 1) : 0.0;
          v[k][2] = c < ca.G ? __ldcg(ps + 2) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < SB; ++k) { t0 += v[k][0]; t1 += v[k][1]; t2 += v[k][2]; }
      }
      t0 = warp_sum(t0);
      t1 = warp_sum(t1);
      t2 = warp_sum(t2);
      finish_pass(lp, pr, &sst, i, t0, t1, t2);
    }
    __syncthreads();
  }
  const int err = sst.error;
  if (!err) {
    // psi <- sum_j C_j q^_j on this CTA's tiles (no CTA reads psi any more)
    if (threadIdx.x <= KMAX) {
      cr_s[threadIdx.x] = sst.coef_re[threadIdx.x];
      ci_s[threadIdx.x] = sst.coef_im[threadIdx.x];
      fr_s[threadIdx.x] = (float)cr_s[threadIdx.x];
      fi_s[threadIdx.x] = (float)ci_s[threadIdx.x];
    }
    __syncthreads();
    const int cq = lp.chunk_q, cr = lp.chunk_r;
    const int t_begin = blockIdx.x * cq + min((int)blockIdx.x, cr);
    const int t_end = t_begin + cq + ((int)blockIdx.x < cr ? 1 : 0);
    const long long n = (long long)pr->nx * pr->ny;
    const int k = sst.k_used;
    vec4* psi = const_cast<vec4*>(pr->psi);
    for (int tt = t_begin; tt < t_end; ++tt) {
      const int x0 = (tt % pr->tiles_x) * TILE_W, y0 = (tt / pr->tiles_x) * TH;
      for (int e = threadIdx.x; e < TILE_W * TH; e += NT) {
        const int x = x0 + (e & (TILE_W - 1)), y = y0 + e / TILE_W;
        if (x < pr->nx && y < pr->ny)
          recombine_site<F32>(psi, pr->basis, n, (long long)y * pr->nx + x, k, cr_s, ci_s, fr_s, fi_s);
      }
    }
  }
  if (blockIdx.x == 0) {   // publish the state (identical in every CTA), re-armed for the next step
    __syncthreads();
    if (threadIdx.x == 0) {
      if (!err) { sst.stopped = 0; sst.cur_pass = 1; sst.redo_left = lp.redo_budget; }
      *const_cast<int*>(lp.step) = step + 1;
    }
    __syncthreads();
    const unsigned* src = reinterpret_cast<const unsigned*>(&sst);
    unsigned* dst = reinterpret_cast<unsigned*>(gst);
    for (int w = threadIdx.x; w < (int)(sizeof(DevState) / sizeof(unsigned)); w += NT) dst[w] = src[w];
  }
}

// ---------------------------------------------------------------------------
// test hook: exp(-i T dt) e_1 for a given T with the device routine
// ---------------------------------------------------------------------------
static __global__ void debug_tridiag_expm(const __grid_constant__ ChebParams cp, int k, const double* alpha1,
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
