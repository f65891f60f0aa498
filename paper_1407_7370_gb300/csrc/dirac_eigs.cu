// dirac_eigs.cu -- eigenvalue mode of the Dirac Lanczos library (Sec. 2, Sec. 5)
// and the plain Hamiltonian product.
//
// Lanczos on A = H - s (direct) or A = (H - s - sigma)^2 (shift-folded), with
// full reorthogonalisation by classical Gram-Schmidt applied twice (Sec. 2),
// Ritz values of T_k checked every few iterations against the Eq. 9 bound
// |beta_k t_i^k|, and Ritz vectors Q t_i (Eq. 8) on request.
//
// Iteration i (0-based) with basis slots q^_0..q^_i (q_j = s_j q^_j, s_j the
// reciprocal norm of slot j, so no vector is ever rescaled in memory):
//   apply   z = s_i A q^_i - beta_{i-1} s_{i-1} q^_{i-1}  into slot i+1; the
//           prologue turns the norm partials of slot i into beta_{i-1} and s_i
//           and applies the breakdown test
//   twice:  h_j = <q_j, z> for j <= i  (dot + finish: fixed-order sums)
//           z -= sum_j h_j q_j         (update; the second also yields ||z||^2
//                                       partials for beta_i)
//   alpha_i = Re(h_i) summed over both passes.
// Without reorthogonalisation one pass against q_i alone with the real part
// of h_i only (Fig. 1, Eq. 4).
//
// Every sum is taken in a fixed order (per-CTA partials, then one warp), so
// results are bitwise reproducible.  No kernel waits on another CTA.
//
// The Ritz values come from a Sturm-sequence multisection on T_k (one warp
// per eigenvalue, 32 points per round), their vectors from inverse iteration
// with a partially pivoted LU of T_k - theta (two solves, orthogonalised
// within clusters of close values); T_k is scaled by a power of two so that
// the characteristic-polynomial recurrence stays in range.
#include "dirac.h"
#include "dirac_internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

namespace dirac {
namespace eig {

using v4 = double4_32a;   // one site: (u.re, u.im, d.re, d.im)

constexpr int RITZ_CAP = DIRAC_EIG_RITZ_MAX;   // Ritz values examined per check
constexpr int MAX_ITER = DIRAC_EIG_ITER_MAX;
constexpr int CH_MAX = 1024;                   // sites per dot-kernel chunk
constexpr double BREAKDOWN_REL = 1e-12;

struct EigDev {
  int breakdown;   // 1 once beta_i <= 1e-12 * scale (invariant subspace)
  int k_final;     // size of T at the breakdown
  int error;       // 1: non-finite value or zero start vector
  int pad;
  double scale;    // max(|alpha_j + s_a|, beta_j) so far, s_a the shift of A
};

struct RitzOut {
  int k;           // size of T_k
  int n_lo, n_hi;  // eigenvalue indices of T_k in the window (folded: 0, k)
  int n_exam;      // examined: indices n_lo .. n_lo + n_exam - 1
  int breakdown, error, exp2;   // exp2: T was scaled by 2^-exp2
  int pad;
  double beta_last;             // beta_k of Eq. 9
  double g_lo, g_hi;            // Gershgorin interval of the scaled T
  double theta[RITZ_CAP];
  double bound[RITZ_CAP];
};

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double wmax(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double wmin(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------------------------
// A q: the Hamiltonian of Eq. 12 (electron, central differences) minus e0
// ---------------------------------------------------------------------------
struct ApplyArgs {
  int nx, ny;
  double kx, ky;        // c / (2h) (order 2) or c / (12h) (order 4)
  double cax, cay;      // c A (p - qA = p + A for the electron)
  double au, ad;        // mc^2 - e0, -mc^2 - e0
  const double* V;      // potential energy or null
  const v4* in;
  const v4* sub;        // q^_{i-1} (Lanczos mode) or null
  v4* out;
  EigDev* ed;           // null: plain product out = (H - e0) in
  const double* norm_part;
  int n_part;
  double* beta;
  double* s;
  int iter;
  int prologue;         // 1: s_i and beta_{i-1} from norm_part, breakdown test, scale by s_i
};

template <bool DIRI, class T>
__device__ __forceinline__ void load_site(const v4* __restrict__ in, int gx, int gy, int nx, int ny,
                                          T (&o)[4]) {
  if (DIRI) {
    if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) { o[0] = o[1] = o[2] = o[3] = 0.0; return; }
  } else {
    gx = ((gx % nx) + nx) % nx;
    gy = ((gy % ny) + ny) % ny;
  }
  const v4 v = in[(size_t)gy * nx + gx];
  o[0] = (T)v.x; o[1] = (T)v.y; o[2] = (T)v.z; o[3] = (T)v.w;
}

// T = double: the FP64 product.  T = float: the mixed-precision product --
// the off-diagonal part (differences and vector potential) on FP32 copies of
// the vector, the diagonal (m c^2 + V - e0 and -m c^2 + V - e0) on the FP64
// vector itself, so that the -2 m c^2 of the lower components adds no
// u32 * 2 m c^2 rounding to the product; the Lanczos combination
// s_i y - c q^_{i-1} in FP64.
template <int R, bool DIRI, bool HAS_V, class T>
__global__ void __launch_bounds__(256) eig_apply(const ApplyArgs a) {
  __shared__ double sh_nrm;
  __shared__ int sh_stop;
  double s_in = 1.0, csub = 0.0;
  if (a.ed) {
    // one read of the flags per block (the lead CTA of a prologue launch may
    // set them meanwhile), so that every thread takes the same branch
    if (threadIdx.x == 0) sh_stop = a.ed->breakdown | a.ed->error;
    if (a.prologue && threadIdx.x < 32) {
      double nrm = 0.0;
      for (int c = threadIdx.x; c < a.n_part; c += 32) nrm += a.norm_part[c];
      nrm = wsum(nrm);
      if (threadIdx.x == 0) sh_nrm = nrm;
    }
    __syncthreads();
    if (sh_stop) return;
    const int i = a.iter;
    if (a.prologue) {
      const double bt = sqrt(sh_nrm);          // ||q^_i||: beta_{i-1}, or ||start|| at i = 0
      const bool lead = blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0;
      if (!isfinite(bt) || !(bt > 0.0)) {
        if (lead) a.ed->error = 1;
        return;
      }
      if (i >= 1 && bt <= BREAKDOWN_REL * a.ed->scale) {
        if (lead) { a.ed->breakdown = 1; a.ed->k_final = i; a.beta[i - 1] = bt; }
        return;
      }
      s_in = 1.0 / bt;
      if (i >= 1 && a.sub) csub = bt * a.s[i - 1];
      if (lead) {
        a.s[i] = s_in;
        if (i >= 1) a.beta[i - 1] = bt;
      }
    } else if (a.sub && i >= 1) {
      csub = a.beta[i - 1] * a.s[i - 1];
    }
  }
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= a.nx || y >= a.ny) return;
  const int nx = a.nx, ny = a.ny;
  T C[4], xp[4], xm[4], yp[4], ym[4], dxv[4], dyv[4];
  double C64[4];
  load_site<DIRI>(a.in, x, y, nx, ny, C64);
#pragma unroll
  for (int q = 0; q < 4; ++q) C[q] = (T)C64[q];
  load_site<DIRI>(a.in, x + 1, y, nx, ny, xp);
  load_site<DIRI>(a.in, x - 1, y, nx, ny, xm);
  load_site<DIRI>(a.in, x, y + 1, nx, ny, yp);
  load_site<DIRI>(a.in, x, y - 1, nx, ny, ym);
#pragma unroll
  for (int q = 0; q < 4; ++q) { dxv[q] = xp[q] - xm[q]; dyv[q] = yp[q] - ym[q]; }
  if constexpr (R == 2) {
    load_site<DIRI>(a.in, x + 2, y, nx, ny, xp);
    load_site<DIRI>(a.in, x - 2, y, nx, ny, xm);
    load_site<DIRI>(a.in, x, y + 2, nx, ny, yp);
    load_site<DIRI>(a.in, x, y - 2, nx, ny, ym);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      dxv[q] = fma(T(8), dxv[q], xm[q] - xp[q]);
      dyv[q] = fma(T(8), dyv[q], ym[q] - yp[q]);
    }
  }
  const size_t idx = (size_t)y * nx + x;
  double au = a.au, ad = a.ad;
  if (HAS_V) {
    const double v = a.V[idx];
    au += v;
    ad += v;
  }
  const T kx = (T)a.kx, ky = (T)a.ky, cax = (T)a.cax, cay = (T)a.cay;
  // off-diagonal part
  T ot[4];
  // upper: c[-i D_x d - D_y d + (A_x - i A_y) d]
  ot[0] = kx * dxv[3] - ky * dyv[2] + cax * C[2] + cay * C[3];
  ot[1] = -kx * dxv[2] - ky * dyv[3] + cax * C[3] - cay * C[2];
  // lower: c[-i D_x u + D_y u + (A_x + i A_y) u]
  ot[2] = kx * dxv[1] + ky * dyv[0] + cax * C[0] - cay * C[1];
  ot[3] = -kx * dxv[0] + ky * dyv[1] + cax * C[1] + cay * C[0];
  // plus the diagonal: (mc^2+V-e0) u and (-mc^2+V-e0) d
  const double o[4] = {fma(au, C64[0], (double)ot[0]), fma(au, C64[1], (double)ot[1]),
                       fma(ad, C64[2], (double)ot[2]), fma(ad, C64[3], (double)ot[3])};
  v4 r;
  if (csub != 0.0) {
    const v4 sv = a.sub[idx];
    r.x = fma(s_in, o[0], -csub * sv.x);
    r.y = fma(s_in, o[1], -csub * sv.y);
    r.z = fma(s_in, o[2], -csub * sv.z);
    r.w = fma(s_in, o[3], -csub * sv.w);
  } else {
    r.x = s_in * o[0]; r.y = s_in * o[1]; r.z = s_in * o[2]; r.w = s_in * o[3];
  }
  a.out[idx] = r;
}

// ---------------------------------------------------------------------------
// h_j = <q^_j, z> for j = j0..j1: per-CTA partials, z chunk staged in shared
// memory, one warp per basis vector at a time
// ---------------------------------------------------------------------------
struct DotArgs {
  const v4* z;
  const v4* basis;
  long long n;
  int j0, j1;
  int cs;               // sites per chunk (multiple of 32, <= CH_MAX)
  double2* part;        // [j - j0][CTA]
  const EigDev* ed;
};

__global__ void __launch_bounds__(256) eig_dot(const DotArgs a) {
  extern __shared__ __align__(32) unsigned char smem[];
  if (a.ed && (a.ed->breakdown | a.ed->error)) return;
  v4* zc = reinterpret_cast<v4*>(smem);
  double2* acc = reinterpret_cast<double2*>(smem + (size_t)a.cs * sizeof(v4));
  const int count = a.j1 - a.j0 + 1;
  for (int t = threadIdx.x; t < count; t += blockDim.x) acc[t] = make_double2(0.0, 0.0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long long nchunks = (a.n + a.cs - 1) / a.cs;
  for (long long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const long long base = ch * a.cs;
    const int len = (int)min((long long)a.cs, a.n - base);
    __syncthreads();
    for (int t = threadIdx.x; t < len; t += blockDim.x) zc[t] = a.z[base + t];
    __syncthreads();
    for (int jj = warp; jj < count; jj += nw) {
      const v4* __restrict__ q = a.basis + (size_t)(a.j0 + jj) * a.n + base;
      double re0 = 0.0, im0 = 0.0, re1 = 0.0, im1 = 0.0;
      int t = lane;
      for (; t + 32 < len; t += 64) {
        const v4 qa = q[t], qb = q[t + 32];
        const v4 za = zc[t], zb = zc[t + 32];
        re0 = fma(qa.x, za.x, fma(qa.y, za.y, fma(qa.z, za.z, fma(qa.w, za.w, re0))));
        im0 = fma(qa.x, za.y, fma(-qa.y, za.x, fma(qa.z, za.w, fma(-qa.w, za.z, im0))));
        re1 = fma(qb.x, zb.x, fma(qb.y, zb.y, fma(qb.z, zb.z, fma(qb.w, zb.w, re1))));
        im1 = fma(qb.x, zb.y, fma(-qb.y, zb.x, fma(qb.z, zb.w, fma(-qb.w, zb.z, im1))));
      }
      if (t < len) {
        const v4 qa = q[t], za = zc[t];
        re0 = fma(qa.x, za.x, fma(qa.y, za.y, fma(qa.z, za.z, fma(qa.w, za.w, re0))));
        im0 = fma(qa.x, za.y, fma(-qa.y, za.x, fma(qa.z, za.w, fma(-qa.w, za.z, im0))));
      }
      const double re = wsum(re0 + re1), im = wsum(im0 + im1);
      if (lane == 0) { acc[jj].x += re; acc[jj].y += im; }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < count; t += blockDim.x)
    a.part[(size_t)t * gridDim.x + blockIdx.x] = acc[t];
}

// ---------------------------------------------------------------------------
// grid sums of the dot partials -> update coefficients, alpha_i
// ---------------------------------------------------------------------------
struct FinishArgs {
  const double2* part;
  int n_cta;
  int j0, j1;
  int iter, pass, last, reorth;
  const double* s;
  double2* coef;        // coefficient of q^_j in the update: s_j h_j
  double* alpha;
  const double* beta;
  EigDev* ed;
  double ashift;        // shift of A for the breakdown scale (s direct, 0 folded)
};

__global__ void __launch_bounds__(256) eig_dot_finish(const FinishArgs a) {
  if (a.ed->breakdown | a.ed->error) return;
  const int lane = threadIdx.x & 31;
  const int jj = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (jj > a.j1 - a.j0) return;
  double re = 0.0, im = 0.0;
  const double2* p = a.part + (size_t)jj * a.n_cta;
  for (int c = lane; c < a.n_cta; c += 32) { re += p[c].x; im += p[c].y; }
  re = wsum(re);
  im = wsum(im);
  if (lane != 0) return;
  const int j = a.j0 + jj;
  const double sj = a.s[j];
  const double hr = sj * re;                      // h_j = <q_j, z>
  const double hi = a.reorth ? sj * im : 0.0;     // Fig. 1 removes alpha_i q_i, alpha real
  a.coef[jj] = make_double2(sj * hr, sj * hi);
  if (j == a.iter) {
    if (!isfinite(hr) || !isfinite(hi)) a.ed->error = 1;
    const double al = (a.pass == 0 ? 0.0 : a.alpha[j]) + hr;
    a.alpha[j] = al;
    if (a.last) {
      double sc = fmax(a.ed->scale, fabs(al + a.ashift));
      if (j >= 1) sc = fmax(sc, a.beta[j - 1]);
      a.ed->scale = sc;
    }
  }
}

// ---------------------------------------------------------------------------
// z -= sum_j coef_j q^_j; with `last`, per-CTA partials of ||z||^2
// ---------------------------------------------------------------------------
struct UpdArgs {
  v4* z;
  const v4* basis;
  long long n;
  int j0, j1;
  const double2* coef;
  int last;
  double* norm_part;
  const EigDev* ed;
};

__device__ __forceinline__ void axpy_c(v4& z, double cr, double ci, const v4& q) {
  z.x = fma(-cr, q.x, fma(ci, q.y, z.x));
  z.y = fma(-cr, q.y, fma(-ci, q.x, z.y));
  z.z = fma(-cr, q.z, fma(ci, q.w, z.z));
  z.w = fma(-cr, q.w, fma(-ci, q.z, z.w));
}

__device__ void block_partial(double v, double* out) {
  __shared__ double red[32];
  v = wsum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    t = wsum(t);
    if (lane == 0) *out = t;
  }
}

__global__ void __launch_bounds__(256) eig_update(const UpdArgs a) {
  if (a.ed && (a.ed->breakdown | a.ed->error)) return;
  const int count = a.j1 - a.j0 + 1;
  double nrm = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < a.n; x += stride) {
    v4 zv = a.z[x];
    const v4* __restrict__ q = a.basis + (size_t)a.j0 * a.n + x;
    int jj = 0;
    for (; jj + 4 <= count; jj += 4) {
      const v4 q0 = q[(size_t)jj * a.n], q1 = q[(size_t)(jj + 1) * a.n];
      const v4 q2 = q[(size_t)(jj + 2) * a.n], q3 = q[(size_t)(jj + 3) * a.n];
      const double2 c0 = __ldg(a.coef + jj), c1 = __ldg(a.coef + jj + 1);
      const double2 c2 = __ldg(a.coef + jj + 2), c3 = __ldg(a.coef + jj + 3);
      axpy_c(zv, c0.x, c0.y, q0);
      axpy_c(zv, c1.x, c1.y, q1);
      axpy_c(zv, c2.x, c2.y, q2);
      axpy_c(zv, c3.x, c3.y, q3);
    }
    for (; jj < count; ++jj) {
      const double2 c = __ldg(a.coef + jj);
      axpy_c(zv, c.x, c.y, q[(size_t)jj * a.n]);
    }
    a.z[x] = zv;
    nrm = fma(zv.x, zv.x, fma(zv.y, zv.y, fma(zv.z, zv.z, fma(zv.w, zv.w, nrm))));
  }
  if (a.last) block_partial(nrm, a.norm_part + blockIdx.x);
}

// slot 0 = start, with the ||start||^2 partials
__global__ void __launch_bounds__(256) eig_start(const v4* in, v4* out, long long n, double* norm_part) {
  double nrm = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
    const v4 v = in[x];
    out[x] = v;
    nrm = fma(v.x, v.x, fma(v.y, v.y, fma(v.z, v.z, fma(v.w, v.w, nrm))));
  }
  block_partial(nrm, norm_part + blockIdx.x);
}

// ---------------------------------------------------------------------------
// Ritz values of T_k (Sec. 2) and the Eq. 9 bounds
// ---------------------------------------------------------------------------
struct RitzArgs {
  int k;
  const double* alpha;
  double* beta;
  const double* norm_part;
  int n_part;
  EigDev* ed;
  double lo, hi;        // examined range (energies of A); use_window = 0: the lowest values
  int use_window;
  int exam_max;         // most Ritz values examined (<= RITZ_CAP)
  double* th_s;         // scaled Ritz values, RITZ_CAP
  double* as;           // scaled T: diagonal, off-diagonal, squared off-diagonal
  double* bs;
  double* b2s;
  RitzOut* out;
  double* X;            // eigenvectors, RITZ_CAP rows of kmax
  double* lu;           // LU scratch, RITZ_CAP x 4 x kmax
  int* piv;             // RITZ_CAP x kmax
  int kmax;
};

// Number of eigenvalues of the scaled T below x: sign changes of the
// characteristic polynomials p_j(x) = det(T_j - x) from the three-term
// recurrence p_j = (a_j - x) p_{j-1} - b_{j-1}^2 p_{j-2}.  The pair is rescaled
// by a power of two every 8 terms; an exact zero takes the sign opposite to
// its predecessor (it counts as an eigenvalue at or below x of T_j).
__device__ int sturm_count(const double* __restrict__ as, const double* __restrict__ b2s, int k, double x) {
  double p1 = 1.0, p2 = 0.0;
  int cnt = 0;
  for (int j = 0; j < k; ++j) {
    const double t = (j > 0) ? b2s[j - 1] * p2 : 0.0;
    double p = fma(as[j] - x, p1, -t);
    if (p == 0.0) p = (p1 > 0.0 ? -1.0 : 1.0) * fabs(p1) * 0x1p-60;
    cnt += (p < 0.0) != (p1 < 0.0);
    p2 = p1;
    p1 = p;
    if ((j & 7) == 7) {
      const int e = ilogb(fmax(fabs(p1), fabs(p2)));
      if (e > 400 || e < -400) {
        const double f = ldexp(1.0, -e);
        p1 *= f;
        p2 *= f;
      }
    }
  }
  return cnt;
}

// max (or min, with `mx` false) over a block of up to 1024 threads; every
// thread gets the result
__device__ double block_extreme(double v, bool mx) {
  __shared__ double red[32];
  v = mx ? wmax(v) : wmin(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = red[0];
  for (int w = 1; w < nw; ++w) r = mx ? fmax(r, red[w]) : fmin(r, red[w]);
  return r;
}

__global__ void __launch_bounds__(256) eig_ritz_prep(const RitzArgs a) {
  __shared__ int shk;
  RitzOut* o = a.out;
  if (threadIdx.x < 32) {
    // beta_k: from the last norm partials, or the one that broke down
    const bool broke = a.ed->breakdown != 0;
    const int kb = broke ? a.ed->k_final : a.k;
    double nrm = 0.0;
    if (!broke)
      for (int c = threadIdx.x; c < a.n_part; c += 32) nrm += a.norm_part[c];
    nrm = wsum(nrm);
    if (threadIdx.x == 0) {
      int k = kb;
      const double bt = broke ? a.beta[kb - 1] : sqrt(nrm);
      o->error = 0;
      if (a.ed->error || !isfinite(bt)) {
        o->error = 1;
        a.ed->error = 1;
        k = 0;
      } else if (!broke) {
        a.beta[k - 1] = bt;
        if (bt <= BREAKDOWN_REL * a.ed->scale) { a.ed->breakdown = 1; a.ed->k_final = k; }
      }
      o->k = k;
      o->n_lo = o->n_hi = o->n_exam = 0;
      o->breakdown = a.ed->breakdown;
      o->beta_last = bt;
      shk = k;
    }
  }
  __syncthreads();
  const int k = shk;
  if (k == 0) return;
  // scale T by 2^-e, 2^e above the Gershgorin bound max_j |a_j| + b_{j-1} + b_j,
  // so that the scaled norm is <= 1
  double g = 0.0;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const double bl = j > 0 ? a.beta[j - 1] : 0.0, br = j < k - 1 ? a.beta[j] : 0.0;
    g = fmax(g, fabs(a.alpha[j]) + bl + br);
  }
  g = block_extreme(g, true);
  const int e = g > 0.0 ? ilogb(g) + 1 : 0;
  const double f = ldexp(1.0, -e);
  double glo = 1e300, ghi = -1e300;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const double aj = a.alpha[j] * f;
    const double bl = j > 0 ? a.beta[j - 1] * f : 0.0, br = j < k - 1 ? a.beta[j] * f : 0.0;
    a.as[j] = aj;
    if (j < k - 1) { a.bs[j] = br; a.b2s[j] = br * br; }
    glo = fmin(glo, aj - bl - br);
    ghi = fmax(ghi, aj + bl + br);
  }
  glo = block_extreme(glo, false);
  ghi = block_extreme(ghi, true);
  __syncthreads();   // the scaled arrays are complete
  if (threadIdx.x == 0) {
    // widen by a few ulps so that the interval brackets every eigenvalue
    const double pad = 8.0 * DBL_EPSILON * fmax(1.0, fmax(fabs(glo), fabs(ghi)));
    o->g_lo = glo - pad;
    o->g_hi = ghi + pad;
    o->exp2 = e;
    o->n_lo = a.use_window ? sturm_count(a.as, a.b2s, k, a.lo * f) : 0;
  }
  if (threadIdx.x == 32) o->n_hi = a.use_window ? sturm_count(a.as, a.b2s, k, a.hi * f) : k;
  __syncthreads();
  if (threadIdx.x == 0) o->n_exam = min(o->n_hi - o->n_lo, a.exam_max);
}

// LU of the scaled T - theta with partial pivoting (row interchanges kept in
// piv): d diagonal of U, u1/u2 its first/second superdiagonal, l the
// multipliers.  One thread.
__device__ void tridiag_lu(const double* __restrict__ as, const double* __restrict__ bs, int k, double theta,
                           double* d, double* u1, double* u2, double* l, int* piv) {
  const double tiny = DBL_EPSILON;   // T is scaled to norm <= 1
  for (int j = 0; j < k; ++j) {
    d[j] = as[j] - theta;
    u1[j] = j < k - 1 ? bs[j] : 0.0;
    u2[j] = 0.0;
  }
  for (int j = 0; j < k - 1; ++j) {
    const double low = bs[j];                 // entry (j+1, j)
    if (fabs(d[j]) >= fabs(low)) {
      if (d[j] == 0.0) d[j] = tiny;
      const double m = low / d[j];
      l[j] = m;
      d[j + 1] -= m * u1[j];
      piv[j] = 0;
    } else {                                  // rows j and j+1 change places
      const double m = d[j] / low;
      const double dn = d[j + 1], un = (j + 1 < k - 1) ? u1[j + 1] : 0.0;
      const double uj = u1[j];
      d[j] = low;
      u1[j] = dn;
      u2[j] = un;
      d[j + 1] = uj - m * dn;
      if (j + 1 < k - 1) u1[j + 1] = -m * un;
      l[j] = m;
      piv[j] = 1;
    }
  }
  if (d[k - 1] == 0.0) d[k - 1] = tiny;
}

// x <- (T - theta)^{-1} x with the factors of tridiag_lu; one thread
__device__ void tridiag_solve(int k, const double* d, const double* u1, const double* u2, const double* l,
                              const int* piv, double* x) {
  for (int j = 0; j < k - 1; ++j) {
    if (piv[j]) { const double t = x[j]; x[j] = x[j + 1]; x[j + 1] = t; }
    x[j + 1] -= l[j] * x[j];
  }
  x[k - 1] /= d[k - 1];
  if (k >= 2) x[k - 2] = (x[k - 2] - u1[k - 2] * x[k - 1]) / d[k - 2];
  for (int j = k - 3; j >= 0; --j) x[j] = (x[j] - u1[j] * x[j + 1] - u2[j] * x[j + 2]) / d[j];
}

// x /= ||x|| by one warp (x in global memory; the warp is synchronised on return)
__device__ void warp_normalise(double* x, int k) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  double mx = 0.0;
  for (int j = lane; j < k; j += 32) mx = fmax(mx, fabs(x[j]));
  mx = wmax(mx);
  const double inv_mx = mx > 0.0 ? 1.0 / mx : 1.0;
  double nrm = 0.0;
  for (int j = lane; j < k; j += 32) { const double t = x[j] * inv_mx; nrm = fma(t, t, nrm); }
  nrm = wsum(nrm);
  const double f = inv_mx / sqrt(nrm);
  for (int j = lane; j < k; j += 32) x[j] *= f;
  __syncwarp();
}

// Ritz values: multisection for the r-th smallest eigenvalue (0-based) of the
// scaled T, one warp each, 32 Sturm counts per round
__global__ void __launch_bounds__(128) eig_ritz_values(const RitzArgs a) {
  const RitzOut* o = a.out;
  if (o->error || o->k == 0) return;
  const int lane = threadIdx.x & 31;
  const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (w >= o->n_exam) return;
  const int k = o->k;
  const int r = o->n_lo + w;
  double lo = o->g_lo, hi = o->g_hi;
  for (int round = 0; round < 80; ++round) {
    const double width = hi - lo;
    if (width <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + 2.0 * DBL_EPSILON) break;
    const double xq = lo + width * (double)(lane + 1) * (1.0 / 33.0);
    const int c = sturm_count(a.as, a.b2s, k, xq);
    const unsigned above = __ballot_sync(0xffffffffu, c > r);   // points past the eigenvalue
    const int f = above ? __ffs(above) - 1 : 32;
    const double nlo = __shfl_sync(0xffffffffu, xq, f > 0 ? f - 1 : 0);
    const double nhi = __shfl_sync(0xffffffffu, xq, f < 32 ? f : 31);
    if (f > 0) lo = nlo;
    if (f < 32) hi = nhi;
  }
  if (lane == 0) {
    const double th = 0.5 * (lo + hi);
    a.th_s[w] = th;
    a.out->theta[w] = ldexp(th, o->exp2);
  }
}

// Ritz vectors of T (t_i, for Eq. 9 and Eq. 8) by inverse iteration, two
// solves from a fixed pseudo-random start.  Values closer than CLUSTER (in
// units of the scaled norm) form a cluster, handled by one warp in order:
// each member's iterate is orthogonalised against the members before it
// (modified Gram-Schmidt) and a value equal to its predecessor is nudged by a
// few ulps so that the factorisations differ.
constexpr double CLUSTER = 1e-7;

__global__ void __launch_bounds__(128) eig_ritz_tvecs(const RitzArgs a) {
  const RitzOut* o = a.out;
  if (o->error || o->k == 0) return;
  const int lane = threadIdx.x & 31;
  const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int ne = o->n_exam;
  if (w >= ne) return;
  if (w > 0 && a.th_s[w] - a.th_s[w - 1] <= CLUSTER) return;   // not the first of its cluster
  const int k = o->k;
  double* lu = a.lu + (size_t)w * 4 * a.kmax;
  double *d = lu, *u1 = lu + a.kmax, *u2 = lu + 2 * a.kmax, *l = lu + 3 * a.kmax;
  int* piv = a.piv + (size_t)w * a.kmax;
  double th_prev = 0.0;
  for (int m = w; m < ne && (m == w || a.th_s[m] - a.th_s[m - 1] <= CLUSTER); ++m) {
    double th = a.th_s[m];
    if (m > w && th - th_prev < 10.0 * DBL_EPSILON) th = th_prev + 10.0 * DBL_EPSILON;
    th_prev = th;
    double* x = a.X + (size_t)m * a.kmax;
    if (lane == 0) tridiag_lu(a.as, a.bs, k, th, d, u1, u2, l, piv);
    for (int j = lane; j < k; j += 32) {
      unsigned h = (unsigned)j * 2654435761u + 0x9e3779b9u;
      h ^= h >> 15; h *= 0x85ebca6bu; h ^= h >> 13;
      x[j] = 0.5 + (double)(h >> 8) * (1.0 / 16777216.0);
    }
    __syncwarp();
    for (int it = 0; it < 2; ++it) {
      if (lane == 0) tridiag_solve(k, d, u1, u2, l, piv, x);
      warp_normalise(x, k);
      for (int p = w; p < m; ++p) {         // against the earlier members of the cluster
        const double* xp = a.X + (size_t)p * a.kmax;
        double dot = 0.0;
        for (int j = lane; j < k; j += 32) dot = fma(xp[j], x[j], dot);
        dot = wsum(dot);
        for (int j = lane; j < k; j += 32) x[j] = fma(-dot, xp[j], x[j]);
        __syncwarp();
      }
      if (m > w) warp_normalise(x, k);
    }
    if (lane == 0) a.out->bound[m] = fabs(o->beta_last * x[k - 1]);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Ritz vectors y_l = sum_j q_j t_{j,l} = sum_j q^_j (s_j t_{j,l})  (Eq. 8)
// ---------------------------------------------------------------------------
struct RvArgs {
  const v4* basis;
  const double* s;
  const double* X;
  int kmax, k;
  const int* sel;       // rows of X
  int n_sel;
  long long n;
  v4* out;              // n_sel consecutive fields
};

__global__ void __launch_bounds__(256) eig_ritz_vectors(const RvArgs a) {
  __shared__ double w[4][256];
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (int l0 = 0; l0 < a.n_sel; l0 += 4) {
    const int nl = min(4, a.n_sel - l0);
    double acc[4][4];
#pragma unroll
    for (int l = 0; l < 4; ++l) acc[l][0] = acc[l][1] = acc[l][2] = acc[l][3] = 0.0;
    for (int jb = 0; jb < a.k; jb += 256) {
      __syncthreads();
      const int j = jb + threadIdx.x;
#pragma unroll
      for (int l = 0; l < 4; ++l)
        w[l][threadIdx.x] = (l < nl && j < a.k) ? a.s[j] * a.X[(size_t)a.sel[l0 + l] * a.kmax + j] : 0.0;
      __syncthreads();
      if (x < a.n) {
        const int jn = min(256, a.k - jb);
        for (int jj = 0; jj < jn; ++jj) {
          const v4 q = a.basis[(size_t)(jb + jj) * a.n + x];
#pragma unroll
          for (int l = 0; l < 4; ++l) {
            const double c = w[l][jj];
            acc[l][0] = fma(c, q.x, acc[l][0]);
            acc[l][1] = fma(c, q.y, acc[l][1]);
            acc[l][2] = fma(c, q.z, acc[l][2]);
            acc[l][3] = fma(c, q.w, acc[l][3]);
          }
        }
      }
    }
    if (x < a.n) {
      for (int l = 0; l < nl; ++l) {
        v4 r;
        r.x = acc[l][0]; r.y = acc[l][1]; r.z = acc[l][2]; r.w = acc[l][3];
        a.out[(size_t)(l0 + l) * a.n + x] = r;
      }
    }
  }
}

// folded mode: lambda = sigma + sign(rho) sqrt(theta), rho = <y, (H - s - sigma) y>
__global__ void eig_fold_finish(const double2* part, int n_cta, double theta, double bound, double sigma,
                                double* out) {
  double re = 0.0;
  for (int c = threadIdx.x; c < n_cta; c += 32) re += part[c].x;
  re = wsum(re);
  if (threadIdx.x != 0) return;
  const double th = fmax(theta, 0.0), rt = sqrt(th);
  out[0] = sigma + copysign(rt, re);
  out[1] = th > 0.0 ? fmin(sqrt(bound), bound / rt) : sqrt(bound);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct DevMem {
  void* p = nullptr;
  ~DevMem() { if (p) cudaFree(p); }
};

#define EIG_TRY(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return fail(DIRAC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

ApplyArgs apply_args(const CtxView& v, double e0) {
  ApplyArgs a;
  std::memset(&a, 0, sizeof(a));
  const double kfac = v.order == 2 ? 2.0 : 12.0;
  const double mc2 = v.mass * v.c * v.c;
  a.nx = v.nx; a.ny = v.ny;
  a.kx = v.c / (kfac * v.dx);
  a.ky = v.c / (kfac * v.dy);
  a.cax = v.c * v.ax;
  a.cay = v.c * v.ay;
  a.au = mc2 - e0;
  a.ad = -mc2 - e0;
  a.V = v.V;
  return a;
}

template <int R, bool D, class T>
cudaError_t launch_apply_rd(const ApplyArgs& a, cudaStream_t s) {
  const dim3 grid((a.nx + 31) / 32, (a.ny + 7) / 8);
  if (a.V) eig_apply<R, D, true, T><<<grid, 256, 0, s>>>(a);
  else eig_apply<R, D, false, T><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_apply_t(const CtxView& v, const ApplyArgs& a) {
  if (v.order == 2) return v.boundary == DIRAC_DIRICHLET ? launch_apply_rd<1, true, T>(a, v.stream)
                                                         : launch_apply_rd<1, false, T>(a, v.stream);
  return v.boundary == DIRAC_DIRICHLET ? launch_apply_rd<2, true, T>(a, v.stream)
                                       : launch_apply_rd<2, false, T>(a, v.stream);
}

// f32: the mixed-precision product (the Lanczos steps of a DIRAC_MIXED context)
cudaError_t launch_apply(const CtxView& v, const ApplyArgs& a, bool f32 = false) {
  return f32 ? launch_apply_t<float>(v, a) : launch_apply_t<double>(v, a);
}

// Device time per kernel kind from CUDA events recorded between consecutive
// launches on one stream (active only while the context is profiling).
enum { K_APPLY = 0, K_DOT = 1, K_UPDATE = 2, K_OTHER = 3, K_START = -1 };

struct KindTimer {
  bool on = false;
  cudaStream_t s = nullptr;
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;      // kind of the kernel that ends at event j
  size_t used = 0;
  double ms[4] = {0.0, 0.0, 0.0, 0.0};
  long long n = 0;            // kernels launched (counted also when not timing)

  // after a launch of `k` (K_START: before the first launch of a segment)
  cudaError_t mark(int k) {
    if (k >= 0) ++n;
    if (!on) return cudaSuccess;
    if (used == ev.size()) {
      cudaEvent_t e;
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return r;
      ev.push_back(e);
      kind.push_back(k);
    }
    kind[used] = k;
    return cudaEventRecord(ev[used++], s);
  }
  // after the stream has been synchronised: add up and start a new segment
  cudaError_t flush() {
    if (!on) return cudaSuccess;
    for (size_t j = 1; j < used; ++j) {
      if (kind[j] < 0) continue;
      float t = 0.f;
      cudaError_t r = cudaEventElapsedTime(&t, ev[j - 1], ev[j]);
      if (r != cudaSuccess) return r;
      ms[kind[j]] += t;
    }
    used = 0;
    return cudaSuccess;
  }
  ~KindTimer() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

int n_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return std::max(1, n);
}

}  // namespace eig
}  // namespace dirac

using namespace dirac;
using namespace dirac::eig;

extern "C" {

dirac_status dirac_apply_hamiltonian(dirac_ctx* ctx, const void* in_dev, void* out_dev) {
  CtxView v;
  dirac_status st = ctx_view(ctx, &v);
  if (st != DIRAC_OK) return st;
  if (!v.fields_set) return fail(DIRAC_ESTATE, "dirac_set_fields has not been called");
  if (!in_dev || !out_dev) return fail(DIRAC_EINVAL, "null vector");
  if ((reinterpret_cast<uintptr_t>(in_dev) | reinterpret_cast<uintptr_t>(out_dev)) & 31u)
    return fail(DIRAC_EINVAL, "vectors must be 32-byte aligned");
  if (in_dev == out_dev) return fail(DIRAC_EINVAL, "in and out must not alias");
  ApplyArgs a = apply_args(v, v.shift);
  a.in = static_cast<const v4*>(in_dev);
  a.out = static_cast<v4*>(out_dev);
  EIG_TRY(launch_apply(v, a));
  ++*v.launches;
  return DIRAC_OK;
}

dirac_status dirac_lanczos_eigs(dirac_ctx* ctx, const void* start_dev, int n_want, int max_iter,
                                int check_every, double tol, double e_lo, double e_hi, int reorth,
                                int fold, double sigma, double* eigs_out, double* bounds_out,
                                void* vecs_dev, dirac_eig_info* info) {
  dirac::TraceRange trace("dirac_lanczos_eigs");
  CtxView v;
  dirac_status st = ctx_view(ctx, &v);
  if (st != DIRAC_OK) return st;
  if (!v.fields_set) return fail(DIRAC_ESTATE, "dirac_set_fields has not been called");
  if (!start_dev || (reinterpret_cast<uintptr_t>(start_dev) & 31u))
    return fail(DIRAC_EINVAL, "start vector must be a non-null 32-byte aligned device pointer");
  if (vecs_dev && (reinterpret_cast<uintptr_t>(vecs_dev) & 31u))
    return fail(DIRAC_EINVAL, "vecs_dev must be 32-byte aligned");
  if (n_want < 1 || n_want > RITZ_CAP) return fail(DIRAC_EINVAL, "n_want must be 1..%d", RITZ_CAP);
  if (max_iter < 1 || max_iter > MAX_ITER) return fail(DIRAC_EINVAL, "max_iter must be 1..%d", MAX_ITER);
  if (check_every < 1) return fail(DIRAC_EINVAL, "check_every must be >= 1");
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(DIRAC_EINVAL, "tol must be finite and >= 0");
  if (!fold && !(e_lo < e_hi)) return fail(DIRAC_EINVAL, "window needs e_lo < e_hi");
  if (fold && !std::isfinite(sigma)) return fail(DIRAC_EINVAL, "fold sigma must be finite");
  if (!eigs_out || !bounds_out) return fail(DIRAC_EINVAL, "null output array");
  if (info) std::memset(info, 0, sizeof(*info));

  const long long n = (long long)v.nx * v.ny;
  const size_t vb = sizeof(v4) * (size_t)n;
  const int kmax = max_iter;
  const int sm = n_sms();
  cudaStream_t s = v.stream;

  // launch geometry, fixed for the call
  int cs = (int)std::min<long long>(CH_MAX, std::max<long long>(32, (n + 2LL * sm - 1) / (2LL * sm)));
  cs = (cs + 31) / 32 * 32;
  const int n_dot = (int)std::min<long long>(2LL * sm, (n + cs - 1) / cs);
  const int n_upd = (int)std::min<long long>(4LL * sm, std::max<long long>(1, (n + 255) / 256));
  const size_t dot_smem_max = (size_t)cs * sizeof(v4) + sizeof(double2) * (size_t)(kmax + 1);
  EIG_TRY(cudaFuncSetAttribute(eig_dot, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dot_smem_max));

  // device memory: basis slots 0..max_iter, then (folded) one product buffer
  // and the n_want Ritz vectors before sorting
  const size_t n_vec = (size_t)kmax + 1 + (fold ? 1 + (size_t)n_want : 0);
  size_t free_b = 0, total_b = 0;
  EIG_TRY(cudaMemGetInfo(&free_b, &total_b));
  if (vb * n_vec > free_b)
    return fail(DIRAC_ENOMEM, "eigen mode needs %.3g GB for %zu vectors, %.3g GB free", vb * n_vec / 1e9,
                n_vec, free_b / 1e9);
  DevMem basis_mem, small_mem;
  EIG_TRY(cudaMalloc(&basis_mem.p, vb * n_vec));
  v4* basis = static_cast<v4*>(basis_mem.p);
  v4* tmp = fold ? basis + (size_t)(kmax + 1) * n : nullptr;
  v4* fold_vecs = fold ? tmp + n : nullptr;

  // small arrays
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
  const size_t o_ed = take(sizeof(EigDev));
  const size_t o_ro = take(sizeof(RitzOut));
  const size_t o_alpha = take(sizeof(double) * (kmax + 1));
  const size_t o_beta = take(sizeof(double) * (kmax + 1));
  const size_t o_s = take(sizeof(double) * (kmax + 1));
  const size_t o_coef = take(sizeof(double2) * (kmax + 1));
  const size_t o_dpart = take(sizeof(double2) * (size_t)n_dot * (kmax + 1));
  const size_t o_npart = take(sizeof(double) * n_upd);
  const size_t o_as = take(sizeof(double) * kmax);
  const size_t o_bs = take(sizeof(double) * kmax);
  const size_t o_b2s = take(sizeof(double) * kmax);
  const size_t o_X = take(sizeof(double) * (size_t)RITZ_CAP * kmax);
  const size_t o_lu = take(sizeof(double) * (size_t)RITZ_CAP * 4 * kmax);
  const size_t o_piv = take(sizeof(int) * (size_t)RITZ_CAP * kmax);
  const size_t o_sel = take(sizeof(int) * RITZ_CAP);
  const size_t o_fres = take(sizeof(double) * 2 * RITZ_CAP);
  const size_t o_ths = take(sizeof(double) * RITZ_CAP);
  EIG_TRY(cudaMalloc(&small_mem.p, off));
  char* sb = static_cast<char*>(small_mem.p);
  EigDev* ed = reinterpret_cast<EigDev*>(sb + o_ed);
  RitzOut* ro = reinterpret_cast<RitzOut*>(sb + o_ro);
  double* alpha = reinterpret_cast<double*>(sb + o_alpha);
  double* beta = reinterpret_cast<double*>(sb + o_beta);
  double* sarr = reinterpret_cast<double*>(sb + o_s);
  double2* coef = reinterpret_cast<double2*>(sb + o_coef);
  double2* dpart = reinterpret_cast<double2*>(sb + o_dpart);
  double* npart = reinterpret_cast<double*>(sb + o_npart);
  int* d_sel = reinterpret_cast<int*>(sb + o_sel);
  double* d_fres = reinterpret_cast<double*>(sb + o_fres);
  EIG_TRY(cudaMemsetAsync(ed, 0, sizeof(EigDev), s));
  EIG_TRY(cudaMemsetAsync(alpha, 0, sizeof(double) * (kmax + 1), s));
  EIG_TRY(cudaMemsetAsync(beta, 0, sizeof(double) * (kmax + 1), s));

  RitzArgs ra;
  ra.alpha = alpha; ra.beta = beta; ra.norm_part = npart; ra.n_part = n_upd; ra.ed = ed;
  ra.lo = e_lo; ra.hi = e_hi; ra.use_window = fold ? 0 : 1;
  ra.exam_max = fold ? n_want : RITZ_CAP;
  ra.as = reinterpret_cast<double*>(sb + o_as);
  ra.bs = reinterpret_cast<double*>(sb + o_bs);
  ra.b2s = reinterpret_cast<double*>(sb + o_b2s);
  ra.out = ro;
  ra.X = reinterpret_cast<double*>(sb + o_X);
  ra.lu = reinterpret_cast<double*>(sb + o_lu);
  ra.piv = reinterpret_cast<int*>(sb + o_piv);
  ra.th_s = reinterpret_cast<double*>(sb + o_ths);
  ra.kmax = kmax;

  KindTimer tm;
  tm.on = v.profiling;
  tm.s = s;
  // every exit from here on adds the launches to the context and fills info
  struct Finish {
    KindTimer& tm;
    CtxView& v;
    dirac_eig_info* info;
    ~Finish() {
      *v.launches += tm.n;
      if (info) {
        info->launches = tm.n;
        info->ms_apply = tm.ms[K_APPLY];
        info->ms_dot = tm.ms[K_DOT];
        info->ms_update = tm.ms[K_UPDATE];
        info->ms_other = tm.ms[K_OTHER];
      }
    }
  } finish_guard{tm, v, info};

  EIG_TRY(tm.mark(K_START));
  eig_start<<<n_upd, 256, 0, s>>>(static_cast<const v4*>(start_dev), basis, n, npart);
  EIG_TRY(cudaGetLastError());
  EIG_TRY(tm.mark(K_OTHER));

  const double e0 = v.shift + (fold ? sigma : 0.0);   // A = H - e0 (direct) or (H - e0)^2
  const double ashift = fold ? 0.0 : v.shift;
  std::vector<unsigned char> ro_host(sizeof(RitzOut));
  RitzOut& h = *reinterpret_cast<RitzOut*>(ro_host.data());
  std::vector<int> sel;
  int k_done = 0;
  bool finished = false;

  for (int i = 0; i < max_iter && !finished; ++i) {
    v4* z = basis + (size_t)(i + 1) * n;
    const v4* qi = basis + (size_t)i * n;
    const v4* qim = i >= 1 ? basis + (size_t)(i - 1) * n : nullptr;
    ApplyArgs a = apply_args(v, e0);
    a.ed = ed; a.norm_part = npart; a.n_part = n_upd; a.beta = beta; a.s = sarr; a.iter = i;
    a.prologue = 1;
    a.in = qi;
    const bool f32 = v.precision == DIRAC_MIXED;
    if (!fold) {
      a.sub = qim;
      a.out = z;
      EIG_TRY(launch_apply(v, a, f32));
      EIG_TRY(tm.mark(K_APPLY));
    } else {
      a.sub = nullptr;
      a.out = tmp;
      EIG_TRY(launch_apply(v, a, f32));
      EIG_TRY(tm.mark(K_APPLY));
      a.prologue = 0;
      a.in = tmp;
      a.sub = qim;
      a.out = z;
      EIG_TRY(launch_apply(v, a, f32));
      EIG_TRY(tm.mark(K_APPLY));
    }
    const int passes = reorth ? 2 : 1;
    const int j0 = reorth ? 0 : i;
    const int count = i - j0 + 1;
    for (int p = 0; p < passes; ++p) {
      DotArgs da{z, basis, n, j0, i, cs, dpart, ed};
      const size_t smem = (size_t)cs * sizeof(v4) + sizeof(double2) * (size_t)count;
      eig_dot<<<n_dot, 256, smem, s>>>(da);
      EIG_TRY(cudaGetLastError());
      EIG_TRY(tm.mark(K_DOT));
      FinishArgs fa{dpart, n_dot, j0, i, i, p, p == passes - 1, reorth ? 1 : 0, sarr, coef, alpha, beta, ed, ashift};
      eig_dot_finish<<<(count + 7) / 8, 256, 0, s>>>(fa);
      EIG_TRY(cudaGetLastError());
      EIG_TRY(tm.mark(K_OTHER));
      UpdArgs ua{z, basis, n, j0, i, coef, p == passes - 1 ? 1 : 0, npart, ed};
      eig_update<<<n_upd, 256, 0, s>>>(ua);
      EIG_TRY(cudaGetLastError());
      EIG_TRY(tm.mark(K_UPDATE));
    }
    const int it = i + 1;
    if (it % check_every != 0 && it != max_iter) continue;

    ra.k = it;
    eig_ritz_prep<<<1, 256, 0, s>>>(ra);
    EIG_TRY(cudaGetLastError());
    eig_ritz_values<<<(RITZ_CAP + 3) / 4, 128, 0, s>>>(ra);
    EIG_TRY(cudaGetLastError());
    eig_ritz_tvecs<<<(RITZ_CAP + 3) / 4, 128, 0, s>>>(ra);
    EIG_TRY(cudaGetLastError());
    EIG_TRY(tm.mark(K_OTHER));
    tm.n += 2;
    EIG_TRY(cudaMemcpyAsync(ro_host.data(), ro, sizeof(RitzOut), cudaMemcpyDeviceToHost, s));
    EIG_TRY(cudaStreamSynchronize(s));
    EIG_TRY(tm.flush());
    EIG_TRY(tm.mark(K_START));
    if (h.error) return fail(DIRAC_ENONFINITE, "eigen mode: non-finite value or zero start vector");
    k_done = h.k;
    const int n_exam = h.n_exam;
    std::vector<int> conv;
    for (int w = 0; w < n_exam; ++w) {
      const double th = h.theta[w];
      bool c = h.bound[w] <= tol * std::max(1.0, std::fabs(th));
      if (!fold) c = c && th > e_lo && th < e_hi;
      if (c) conv.push_back(w);
    }
    const bool done = it >= max_iter || h.breakdown;
    bool ok;
    if (!fold) {
      ok = (int)conv.size() >= n_want;
    } else {
      ok = n_exam >= n_want && (int)conv.size() >= n_want && conv[n_want - 1] == n_want - 1;
    }
    if (info) {
      info->iterations = k_done;
      info->n_in_window = h.n_hi - h.n_lo;
      info->n_converged = (int)conv.size();
      info->breakdown = h.breakdown;
    }
    if (ok || done) {
      finished = true;
      if (!fold) {
        sel.assign(conv.begin(), conv.begin() + std::min<size_t>(conv.size(), (size_t)n_want));
      } else {
        for (int w : conv) if (w < n_want) sel.push_back(w);
      }
    }
  }
  const int n_sel = (int)sel.size();
  if (info) info->n_found = n_sel;
  if (n_sel == 0) return DIRAC_OK;

  const int vgrid = (int)((n + 255) / 256);
  if (!fold) {
    for (int l = 0; l < n_sel; ++l) {
      eigs_out[l] = h.theta[sel[l]];
      bounds_out[l] = h.bound[sel[l]];
    }
    if (vecs_dev) {
      EIG_TRY(cudaMemcpyAsync(d_sel, sel.data(), sizeof(int) * n_sel, cudaMemcpyHostToDevice, s));
      RvArgs rv{basis, sarr, ra.X, kmax, k_done, d_sel, n_sel, n, static_cast<v4*>(vecs_dev)};
      eig_ritz_vectors<<<vgrid, 256, 0, s>>>(rv);
      EIG_TRY(cudaGetLastError());
      EIG_TRY(tm.mark(K_OTHER));
      EIG_TRY(cudaStreamSynchronize(s));
      EIG_TRY(tm.flush());
    }
    return DIRAC_OK;
  }

  // folded: Ritz vectors, the sign of each from its Rayleigh quotient with
  // H - s - sigma, lambda ascending
  EIG_TRY(cudaMemcpyAsync(d_sel, sel.data(), sizeof(int) * n_sel, cudaMemcpyHostToDevice, s));
  RvArgs rv{basis, sarr, ra.X, kmax, k_done, d_sel, n_sel, n, fold_vecs};
  eig_ritz_vectors<<<vgrid, 256, 0, s>>>(rv);
  EIG_TRY(cudaGetLastError());
  EIG_TRY(tm.mark(K_OTHER));
  for (int l = 0; l < n_sel; ++l) {
    ApplyArgs a = apply_args(v, e0);
    a.in = fold_vecs + (size_t)l * n;
    a.out = tmp;
    EIG_TRY(launch_apply(v, a));
    EIG_TRY(tm.mark(K_APPLY));
    DotArgs da{tmp, fold_vecs + (size_t)l * n, n, 0, 0, cs, dpart, nullptr};
    eig_dot<<<n_dot, 256, (size_t)cs * sizeof(v4) + sizeof(double2), s>>>(da);
    EIG_TRY(cudaGetLastError());
    EIG_TRY(tm.mark(K_DOT));
    eig_fold_finish<<<1, 32, 0, s>>>(dpart, n_dot, h.theta[sel[l]], h.bound[sel[l]], sigma, d_fres + 2 * l);
    EIG_TRY(cudaGetLastError());
    EIG_TRY(tm.mark(K_OTHER));
  }
  std::vector<double> fres(2 * n_sel);
  EIG_TRY(cudaMemcpyAsync(fres.data(), d_fres, sizeof(double) * 2 * n_sel, cudaMemcpyDeviceToHost, s));
  EIG_TRY(cudaStreamSynchronize(s));
  EIG_TRY(tm.flush());
  std::vector<int> order(n_sel);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return fres[2 * p] < fres[2 * q]; });
  for (int l = 0; l < n_sel; ++l) {
    eigs_out[l] = fres[2 * order[l]];
    bounds_out[l] = fres[2 * order[l] + 1];
    if (vecs_dev)
      EIG_TRY(cudaMemcpyAsync(static_cast<v4*>(vecs_dev) + (size_t)l * n, fold_vecs + (size_t)order[l] * n, vb,
                              cudaMemcpyDeviceToDevice, s));
  }
  EIG_TRY(cudaStreamSynchronize(s));
  return DIRAC_OK;
}

}  // extern "C"
