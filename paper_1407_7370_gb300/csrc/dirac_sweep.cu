// dirac_sweep.cu -- the mixed-precision time step as one cooperative launch
// in which every Lanczos pass (Fig. 1, Eq. 4) is a register sweep over the
// grid and nothing but the Krylov basis is written.
//
// Pass i needs q^_i = g_{i-1} (y^_{i-1} - d_{i-1} q^_{i-1}) and y^_i =
// (H - s - sigma_i) q^_i - e_i q^_{i-1}.  Instead of storing y^_{i-1} in pass
// i - 1 and reading it back (the fused scheme of the per-pass kernel, 64 bytes
// per site and pass in complex64), this kernel recomputes y^_{i-1} =
// (H - s - sigma_{i-1}) q^_{i-1} - e_{i-1} q^_{i-2} from the two basis vectors
// it reads anyway.  A pass then reads q^_{i-1} and q^_{i-2} and writes q^_i:
// 48 bytes per site, the algorithmic minimum, for twice the stencil
// arithmetic, which the FP32 pipe has room for.  The recomputation runs the
// same FP32 instructions on the same stored values, so the y^_{i-1} it gets
// is the one whose sums P, Y, X were reduced in pass i - 1.
//
// Work: strips of W = 32 - 4R columns by SWEEP_H rows ("units"), one warp
// each.  Lane l holds column x0 - 2R + l; the warp walks down the strip one
// row per iteration, keeping the last 2R + 1 rows of q^_{i-1} and of q^_i in
// registers (vertical neighbours) and taking horizontal neighbours by warp
// shuffles, so no shared memory and no block-wide barrier is involved; rows
// are loaded a few iterations ahead.  Lanes R .. 31 - R have y^_{i-1} and
// q^_i, lanes 2R .. 31 - 2R (the strip) y^_i.
//
// Between passes: a bounded grid barrier; then, as in the other one-launch
// steps, every CTA sums the CTA partials in a fixed order and updates its own
// shared-memory copy of the scalars (one problem), or the last CTA to finish
// a problem's units updates its scalars in global memory (several problems).
// At the end the compensated recombination (recombine_site_df).
#include "dirac.h"
#include "dirac_internal.h"
#include "dirac_kernels.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

namespace dirac {
namespace sweep {

constexpr int NWARP = 16;                 // warps per CTA, one CTA per SM (up to 128 registers)
constexpr int NT = 32 * NWARP;
constexpr int H = SWEEP_H;
template <int R> __host__ __device__ constexpr int strip_w() { return 32 - 4 * R; }

// the fields a pass reads, by pass number
enum Mode { FIRST = 0, SECOND = 1, THIRD = 2, LATER = 3 };
// pass 1: q^_1 = psi (complex128), y^_1 only.  Pass 2: q^_1 = psi, no q^_0.
// Pass 3: q^_2 from the basis, q^_1 = psi.  Later: both from the basis.
template <int MODE> __host__ __device__ constexpr bool a_is_f64() { return MODE <= SECOND; }
template <int MODE> __host__ __device__ constexpr bool has_b() { return MODE >= THIRD; }
template <int MODE> __host__ __device__ constexpr bool b_is_f64() { return MODE == THIRD; }
// rows loaded ahead (two: more registers cost more in warps per SM than
// they gain in loads in flight)
template <int R, int MODE> __host__ __device__ constexpr int prefetch() { return 2; }

// the stencil coefficients shared by both applications of a pass
struct KCoef {
  float kxh, kxl, kyh, kyl;   // c / (2 dx), c / (2 dy) (order 2) or c / (12 h) (order 4), value + remainder
  float axh, axl, ayh, ayl;   // c A_x, c A_y
  bool has_ay;
};
// diagonal and coupling of one application: (H - s - sigma) q - e q_prev
struct DCoef {
  float auh, aul, adh, adl;   // m c^2 - s - sigma, -m c^2 - s - sigma
  float e;
};
__device__ __forceinline__ DCoef dcoef(const PassCoef& pc, bool with_e) {
  DCoef d;
  d.auh = pc.au_hi; d.aul = pc.au_lo; d.adh = pc.ad_hi; d.adl = pc.ad_lo;
  d.e = with_e ? pc.ef : 0.f;
  return d;
}

// one spinor site in registers
struct F4 {
  float x, y, z, w;
};
__device__ __forceinline__ F4 f4(float4 v) { return F4{v.x, v.y, v.z, v.w}; }
__device__ __forceinline__ F4 f4(const vec4& v) { return F4{(float)v.x, (float)v.y, (float)v.z, (float)v.w}; }
__device__ __forceinline__ F4 zero4() { return F4{0.f, 0.f, 0.f, 0.f}; }

// loads of the inputs of a pass: written by other CTAs in earlier passes of
// this launch, so through L2 (after the grid barrier's acquire)
__device__ __forceinline__ float4 ld_field(const float4* p) { return __ldcg(p); }
__device__ __forceinline__ vec4 ld_field(const vec4* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  const double2 a = __ldcg(q), b = __ldcg(q + 1);
  vec4 r;
  r.x = a.x; r.y = a.y; r.z = b.x; r.w = b.y;
  return r;
}
// differences of the neighbours along x by shuffles: lane l gets
// v[l+1] - v[l-1] (order 2) or 8 (v[l+1] - v[l-1]) - (v[l+2] - v[l-2])
// (order 4); the outermost R lanes get values of no use
template <int R>
__device__ __forceinline__ float dxs(float v) {
  const unsigned full = 0xffffffffu;
  float d = __shfl_down_sync(full, v, 1) - __shfl_up_sync(full, v, 1);
  if constexpr (R == 2) d = fmaf(8.f, d, __shfl_up_sync(full, v, 2) - __shfl_down_sync(full, v, 2));
  return d;
}

// (H - s - sigma) C - e qp at one site, C's neighbours given by the window
// w[0 .. 2R] of rows (C = w[R]) and shuffles; V (when has_v) as an FP32
// pair (vh, vl).
// FP32 products and sums, every coefficient as a value plus its remainder
// and the diagonal plus V by an exact two-sum, as in the per-pass kernel.
template <int R>
__device__ __forceinline__ F4 apply_h(const F4 (&w)[2 * R + 1], const KCoef& k, const DCoef& d, bool has_v,
                                      float vh, float vl, const F4& qp) {
  const F4 C = w[R];
  float dx[4] = {dxs<R>(C.x), dxs<R>(C.y), dxs<R>(C.z), dxs<R>(C.w)};
  float dy[4] = {w[R + 1].x - w[R - 1].x, w[R + 1].y - w[R - 1].y, w[R + 1].z - w[R - 1].z,
                 w[R + 1].w - w[R - 1].w};
  if constexpr (R == 2) {
    dy[0] = fmaf(8.f, dy[0], w[0].x - w[4].x);
    dy[1] = fmaf(8.f, dy[1], w[0].y - w[4].y);
    dy[2] = fmaf(8.f, dy[2], w[0].z - w[4].z);
    dy[3] = fmaf(8.f, dy[3], w[0].w - w[4].w);
  }
  float au = d.auh, ad = d.adh, aul = d.aul, adl = d.adl;
  if (has_v) {
    float ru, rd;
    two_sum(d.auh, vh, au, ru);
    two_sum(d.adh, vh, ad, rd);
    aul = d.aul + vl + ru;
    adl = d.adl + vl + rd;
  }
  // upper: (mc^2+V-s-sigma) u + c[-i D_x d - D_y d + (A_x - i A_y) d]
  // lower: (-mc^2+V-s-sigma) d + c[-i D_x u + D_y u + (A_x + i A_y) u]
  float y0 = au * C.x + k.kxh * dx[3] - k.kyh * dy[2] + k.axh * C.z;
  float y1 = au * C.y - k.kxh * dx[2] - k.kyh * dy[3] + k.axh * C.w;
  float y2 = ad * C.z + k.kxh * dx[1] + k.kyh * dy[0] + k.axh * C.x;
  float y3 = ad * C.w - k.kxh * dx[0] + k.kyh * dy[1] + k.axh * C.y;
  if (k.has_ay) {
    y0 = fmaf(k.ayh, C.w, y0); y1 = fmaf(-k.ayh, C.z, y1);
    y2 = fmaf(-k.ayh, C.y, y2); y3 = fmaf(k.ayh, C.x, y3);
    y0 = fmaf(k.ayl, C.w, y0); y1 = fmaf(-k.ayl, C.z, y1);
    y2 = fmaf(-k.ayl, C.y, y2); y3 = fmaf(k.ayl, C.x, y3);
  }
  y0 = fmaf(aul, C.x, fmaf(k.kxl, dx[3], fmaf(-k.kyl, dy[2], fmaf(k.axl, C.z, fmaf(-d.e, qp.x, y0)))));
  y1 = fmaf(aul, C.y, fmaf(-k.kxl, dx[2], fmaf(-k.kyl, dy[3], fmaf(k.axl, C.w, fmaf(-d.e, qp.y, y1)))));
  y2 = fmaf(adl, C.z, fmaf(k.kxl, dx[1], fmaf(k.kyl, dy[0], fmaf(k.axl, C.x, fmaf(-d.e, qp.z, y2)))));
  y3 = fmaf(adl, C.w, fmaf(-k.kxl, dx[0], fmaf(k.kyl, dy[1], fmaf(k.axl, C.y, fmaf(-d.e, qp.w, y3)))));
  return F4{y0, y1, y2, y3};
}

// What one unit of a pass reads and writes.
struct UnitArgs {
  int nx, ny;
  bool diri;
  const void* A;        // q^_{i-1}; pass 1: psi = q^_1
  const void* B;        // q^_{i-2} (pass 3: psi), or null
  float4* q_out;        // q^_i (basis vector i - 2); null in pass 1
  const float* Vh;      // V as FP32 pairs (value, remainder), or null
  const float* Vl;
  KCoef k;
  DCoef d1;             // y^_{i-1}: stencil shift sigma_{i-1}, coupling e_{i-1}
  DCoef d2;             // y^_i (pass 1: the only application)
  float g, gd;          // q^_i = g y^_{i-1} - gd q^_{i-1}
};

// grid index of coordinate v along an axis of n points: periodic images, or
// `out` (a Dirichlet zero) outside
__device__ __forceinline__ int axis_index(int v, int n, bool diri, bool& out) {
  out = false;
  if (v >= 0 && v < n) return v;
  if (diri) { out = true; return 0; }
  int r = v % n;
  return r < 0 ? r + n : r;
}

// One unit (strip x0 .. x0 + W - 1, rows y0 .. y0 + H - 1) of a pass:
// stores q^_i on the strip and adds this lane's terms of P, Y, X.  Row
// iteration j loads row ya = y0 - LAG + j of A (and row ya - R of B and V);
// it completes y^_{i-1} and q^_i on row ya - R and y^_i on row ya - 2R
// (pass 1: y^_1 on row ya - R).
template <int R, int MODE>
__device__ __forceinline__ void sweep_unit(const UnitArgs& u, int x0, int y0, float& tP, float& tY, float& tX) {
  using TA = std::conditional_t<a_is_f64<MODE>(), vec4, float4>;
  using TB = std::conditional_t<b_is_f64<MODE>(), vec4, float4>;
  constexpr int PF = prefetch<R, MODE>();
  constexpr int LAG = (MODE == FIRST) ? R : 2 * R;
  constexpr int NA = H + 2 * LAG;
  constexpr int W = strip_w<R>();
  const int lane = threadIdx.x & 31;
  const int nx = u.nx, ny = u.ny;
  const int gx = x0 - 2 * R + lane;
  bool xout;
  const int ix = axis_index(gx, nx, u.diri, xout);
  const bool out_lane = lane >= 2 * R && lane < 2 * R + W && gx < nx;
  const TA* A = static_cast<const TA*>(u.A);
  const TB* B = static_cast<const TB*>(u.B);
  const bool has_v = u.Vh != nullptr;

  auto site = [&](int gy, bool& out) -> size_t {
    bool yout;
    const int iy = axis_index(gy, ny, u.diri, yout);
    out = xout || yout;
    return out ? 0 : (size_t)iy * nx + ix;
  };
  // loads return the raw value (of site 0 outside a Dirichlet grid) and set
  // `out`; the zero is applied where the row is used, so that nothing waits
  // for a load before then
  auto load_a = [&](int j, bool& out) -> TA { return ld_field(A + site(y0 - LAG + j, out)); };
  auto load_b = [&](int j, bool& out) -> TB { return ld_field(B + site(y0 - LAG + j - R, out)); };
  auto load_v = [&](int j, float& vh, float& vl) {
    bool out;
    const size_t s = site(y0 - LAG + j - R, out);
    vh = has_v ? __ldg(u.Vh + s) : 0.f;
    vl = has_v ? __ldg(u.Vl + s) : 0.f;
  };

  TA pa[PF];
  TB pb[PF];
  bool pao[PF], pbo[PF];
  float pvh[PF], pvl[PF];
#pragma unroll
  for (int p = 0; p < PF; ++p) {
    pa[p] = load_a(p, pao[p]);
    pbo[p] = true;
    if constexpr (has_b<MODE>()) {
      if (p >= 2 * R) pb[p] = load_b(p, pbo[p]);
    }
    if (p >= 2 * R) load_v(p, pvh[p], pvl[p]);
  }
  F4 Aw[2 * R + 1], Qw[2 * R + 1];
  float Vwh[R + 1], Vwl[R + 1];
#pragma unroll
  for (int s = 0; s <= 2 * R; ++s) { Aw[s] = zero4(); Qw[s] = zero4(); }
#pragma unroll
  for (int s = 0; s <= R; ++s) { Vwh[s] = 0.f; Vwl[s] = 0.f; }

  // rolled in groups of PF rows (slot = j mod PF stays a constant), so that
  // the code of a unit stays small and the loads of a group are consumed
  // only in the next one
#pragma unroll 1
  for (int j0 = 0; j0 < NA; j0 += PF) {
#pragma unroll
    for (int slot = 0; slot < PF; ++slot) {
      const int j = j0 + slot;
      if (j >= NA) break;
      // the new row of A, then the load PF rows ahead into the freed slot
#pragma unroll
      for (int s = 0; s < 2 * R; ++s) Aw[s] = Aw[s + 1];
      Aw[2 * R] = pao[slot] ? zero4() : f4(pa[slot]);
      F4 Bv = zero4();
      if (j >= 2 * R) {
        if constexpr (has_b<MODE>()) Bv = pbo[slot] ? zero4() : f4(pb[slot]);
#pragma unroll
        for (int s = 0; s < R; ++s) { Vwh[s] = Vwh[s + 1]; Vwl[s] = Vwl[s + 1]; }
        Vwh[R] = pvh[slot];
        Vwl[R] = pvl[slot];
      }
      if (j + PF < NA) {
        pa[slot] = load_a(j + PF, pao[slot]);
        if (j + PF >= 2 * R) {
          if constexpr (has_b<MODE>()) pb[slot] = load_b(j + PF, pbo[slot]);
          load_v(j + PF, pvh[slot], pvl[slot]);
        }
      }
      if constexpr (MODE == FIRST) {
        // y^_1 = (H - s - sigma_1) q^_1 on row ya - R
        if (j >= 2 * R) {
          const int yc = y0 + j - 2 * LAG;
          const F4 y = apply_h<R>(Aw, u.k, u.d2, has_v, Vwh[R], Vwl[R], zero4());
          if (out_lane && yc < ny) {
            const F4 C = Aw[R];
            tP = fmaf(C.x, y.x, fmaf(C.y, y.y, fmaf(C.z, y.z, fmaf(C.w, y.w, tP))));
            tY = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, tY))));
            tX = fmaf(C.x, C.x, fmaf(C.y, C.y, fmaf(C.z, C.z, fmaf(C.w, C.w, tX))));
          }
        }
      } else {
        if (j >= 2 * R) {
          // y^_{i-1} and q^_i on row yb = ya - R (lanes R .. 31 - R)
          const int yb = y0 + j - LAG - R;
          const F4 y1 = apply_h<R>(Aw, u.k, u.d1, has_v, Vwh[R], Vwl[R], Bv);
          const F4 qa = Aw[R];
          F4 q = F4{fmaf(-u.gd, qa.x, u.g * y1.x), fmaf(-u.gd, qa.y, u.g * y1.y), fmaf(-u.gd, qa.z, u.g * y1.z),
                    fmaf(-u.gd, qa.w, u.g * y1.w)};
          if (u.diri && (xout || yb < 0 || yb >= ny)) q = zero4();
#pragma unroll
          for (int s = 0; s < 2 * R; ++s) Qw[s] = Qw[s + 1];
          Qw[2 * R] = q;
        }
        if (j >= 4 * R) {
          // y^_i on row yc = yb - R (lanes 2R .. 31 - 2R), coupling to q^_{i-1} = Aw[0]
          const int yc = y0 + j - 2 * LAG;
          const F4 y = apply_h<R>(Qw, u.k, u.d2, has_v, Vwh[0], Vwl[0], Aw[0]);
          if (out_lane && yc < ny) {
            const F4 C = Qw[R];
            u.q_out[(size_t)yc * nx + gx] = make_float4(C.x, C.y, C.z, C.w);
            tP = fmaf(C.x, y.x, fmaf(C.y, y.y, fmaf(C.z, y.z, fmaf(C.w, y.w, tP))));
            tY = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, tY))));
            tX = fmaf(C.x, C.x, fmaf(C.y, C.y, fmaf(C.z, C.z, fmaf(C.w, C.w, tX))));
          }
        }
      }
    }
  }
}

__device__ __forceinline__ int problem_of_unit(const LaunchParams& lp, int t) {
  int lo = 0, hi = lp.nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (lp.probs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// fields and coefficients of pass i of problem pr; pc: this pass's
// coefficients, pp: those of pass i - 1 (its stencil shift and coupling)
template <int R>
__device__ __forceinline__ UnitArgs unit_args(const LaunchParams& lp, const Problem* pr, const FieldStep& fs,
                                              const PassCoef& pc, const PassCoef& pp, int i) {
  UnitArgs u;
  u.nx = pr->nx;
  u.ny = pr->ny;
  u.diri = lp.diri != 0;
  const size_t n = (size_t)pr->nx * pr->ny;
  char* basis = static_cast<char*>(pr->basis);
  u.A = (i <= 2) ? static_cast<const void*>(pr->psi) : static_cast<const void*>(basis + (size_t)(i - 3) * n * 16);
  u.B = (i == 3) ? static_cast<const void*>(pr->psi)
                 : (i >= 4 ? static_cast<const void*>(basis + (size_t)(i - 4) * n * 16) : nullptr);
  u.q_out = (i >= 2) ? reinterpret_cast<float4*>(basis + (size_t)(i - 2) * n * 16) : nullptr;
  u.Vh = static_cast<const float*>(pr->V);
  u.Vl = static_cast<const float*>(pr->Vlo);
  u.k.kxh = pr->kxf; u.k.kxl = pr->kxf_lo; u.k.kyh = pr->kyf; u.k.kyl = pr->kyf_lo;
  u.k.axh = fs.cAxf; u.k.axl = fs.cAxf_lo; u.k.ayh = fs.cAyf; u.k.ayl = fs.cAyf_lo;
  u.k.has_ay = fs.cAy != 0.0;
  u.d1 = dcoef(pp, i >= 3);   // y^_1 has no coupling term
  u.d2 = dcoef(pc, i >= 2);
  u.g = pc.gf;
  u.gd = pc.gdf;
  return u;
}

template <int R, bool SINGLE>
__global__ void __launch_bounds__(NT, 1) lanczos_sweep(const __grid_constant__ LaunchParams lp,
                                                      const __grid_constant__ CoopArgs ca) {
  constexpr int W = strip_w<R>();
  __shared__ DevState sst;              // one problem: this CTA's copy of its scalars
  __shared__ double red[NWARP][3];
  __shared__ double cr_s[KMAX + 2], ci_s[KMAX + 2];
  __shared__ float crh_s[KMAX + 2], crl_s[KMAX + 2], cih_s[KMAX + 2], cil_s[KMAX + 2];
  __shared__ int rk_s, rerr_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cq = lp.chunk_q, crm = lp.chunk_r;
  const int t_begin = blockIdx.x * cq + min((int)blockIdx.x, crm);
  const int t_end = t_begin + cq + ((int)blockIdx.x < crm ? 1 : 0);
  const bool probe = lp.probe != 0;
  if (SINGLE) {
    const unsigned* src = reinterpret_cast<const unsigned*>(lp.states);
    unsigned* dst = reinterpret_cast<unsigned*>(&sst);
    for (int w = threadIdx.x; w < (int)(sizeof(DevState) / sizeof(unsigned)); w += NT) dst[w] = __ldcg(src + w);
  }
  const int step = __ldcg(lp.step);
  __syncthreads();

  const int max_iter = probe ? 1 : lp.m + lp.redo_budget;
  bool failed = false;
  for (int iter = 0; iter < max_iter; ++iter) {
    if (SINGLE && !probe && sst.stopped) break;
    double* slots = ca.slots + (iter & 1) * 3 * ca.G;
    const int i_single = SINGLE ? (probe ? 1 : max(1, sst.cur_pass)) : 0;
    int b = problem_of_unit(lp, t_begin);
    for (int t = t_begin; t < t_end; ++b) {
      const Problem* pr = lp.probs + b;
      const DevState* gst = lp.states + b;
      const int seg_end = min(t_end, pr->tile_begin + pr->ntiles);
      const int seg_units = seg_end - t;
      int i;
      if (probe) {
        i = 1;
      } else if (SINGLE) {
        i = i_single;
      } else {
        if (__ldcg(&gst->stopped)) { t = seg_end; continue; }
        i = max(1, __ldcg(&gst->cur_pass));
      }
      PassCoef pc, pp;
      if (probe) {
        pc = pr->probe_coef;
        pp = pc;
      } else if (SINGLE) {
        pc = sst.pc_cur;
        pp = sst.pc_prev;
      } else {
        const double* s1 = reinterpret_cast<const double*>(&gst->pc_cur);
        const double* s2 = reinterpret_cast<const double*>(&gst->pc_prev);
        double* d1 = reinterpret_cast<double*>(&pc);
        double* d2 = reinterpret_cast<double*>(&pp);
        for (int w = 0; w < (int)(sizeof(PassCoef) / sizeof(double)); ++w) {
          d1[w] = __ldcg(s1 + w);
          d2[w] = __ldcg(s2 + w);
        }
      }
      const FieldStep fs = lp.fields[step * lp.fstride + b];
      const UnitArgs u = unit_args<R>(lp, pr, fs, pc, pp, i);
      // per-lane sums over the warp's units: FP32 values with two-sum
      // compensation (FP64 adds would cost more than a unit's stencils)
      float sP = 0.f, sY = 0.f, sX = 0.f, cP = 0.f, cY = 0.f, cX = 0.f;
      for (int tt = t + warp; tt < seg_end; tt += NWARP) {
        const int lt = tt - pr->tile_begin;
        const int x0 = (lt % pr->tiles_x) * W;
        const int y0 = (lt / pr->tiles_x) * H;
        float tP = 0.f, tY = 0.f, tX = 0.f;
        if (i == 1) sweep_unit<R, FIRST>(u, x0, y0, tP, tY, tX);
        else if (i == 2) sweep_unit<R, SECOND>(u, x0, y0, tP, tY, tX);
        else if (i == 3) sweep_unit<R, THIRD>(u, x0, y0, tP, tY, tX);
        else sweep_unit<R, LATER>(u, x0, y0, tP, tY, tX);
        float s, r;
        two_sum(sP, tP, s, r); sP = s; cP += r;
        two_sum(sY, tY, s, r); sY = s; cY += r;
        two_sum(sX, tX, s, r); sX = s; cX += r;
      }
      // this CTA's share of problem b: lanes -> warp in FP64, warps -> CTA
      const double wP = warp_sum((double)sP + (double)cP);
      const double wY = warp_sum((double)sY + (double)cY);
      const double wX = warp_sum((double)sX + (double)cX);
      if (lane == 0) { red[warp][0] = wP; red[warp][1] = wY; red[warp][2] = wX; }
      __syncthreads();
      if (warp == 0) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        if (lane < NWARP) { s0 = red[lane][0]; s1 = red[lane][1]; s2 = red[lane][2]; }
#pragma unroll
        for (int o = NWARP / 2; o > 0; o >>= 1) {
          s0 += __shfl_xor_sync(0xffffffffu, s0, o);
          s1 += __shfl_xor_sync(0xffffffffu, s1, o);
          s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (SINGLE) {
          if (lane == 0) {
            slots[3 * blockIdx.x + 0] = s0;
            slots[3 * blockIdx.x + 1] = s1;
            slots[3 * blockIdx.x + 2] = s2;
          }
        } else {
          int last = 0;
          if (lane == 0) {
            const int slot = blockIdx.x - cta_of_tile(pr->tile_begin, cq, crm);
            pr->partials[3 * slot + 0] = s0;
            pr->partials[3 * slot + 1] = s1;
            pr->partials[3 * slot + 2] = s2;
            cuda::atomic_ref<unsigned, cuda::thread_scope_device> ticket(pr->st->counter);
            last = ticket.fetch_add((unsigned)seg_units, cuda::memory_order_acq_rel) + seg_units ==
                   (unsigned)pr->ntiles;
          }
          last = __shfl_sync(0xffffffffu, last, 0);
          if (last) {
            // the problem is complete: its slots in a fixed order, then the scalars
            const int cta_lo = cta_of_tile(pr->tile_begin, cq, crm);
            const int nslots = cta_of_tile(pr->tile_begin + pr->ntiles - 1, cq, crm) - cta_lo + 1;
            double t0 = 0.0, t1 = 0.0, t2 = 0.0;
            for (int q = lane; q < nslots; q += 32) {
              t0 += __ldcg(pr->partials + 3 * q + 0);
              t1 += __ldcg(pr->partials + 3 * q + 1);
              t2 += __ldcg(pr->partials + 3 * q + 2);
            }
            t0 = warp_sum(t0);
            t1 = warp_sum(t1);
            t2 = warp_sum(t2);
            if (lane == 0) pr->st->counter = 0u;
            finish_pass(lp, pr, pr->st, i, t0, t1, t2);
          }
        }
      }
      __syncthreads();   // red[] is reused by the next problem
      t = seg_end;
    }
    if (!grid_sync(ca.bar, (unsigned)ca.bar_count)) {
      failed = true;
      break;
    }
    if (SINGLE) {
      if (warp == 0) {   // the grid totals, in the same order in every CTA
        double t0 = 0.0, t1 = 0.0, t2 = 0.0;
        for (int c0 = 0; c0 < ca.G; c0 += 5 * 32) {   // five slots per lane in flight at once
          double v[5][3];
#pragma unroll
          for (int w = 0; w < 5; ++w) {
            const int c = c0 + lane + 32 * w;
            const double* ps = slots + 3 * (c < ca.G ? c : 0);
            v[w][0] = c < ca.G ? __ldcg(ps + 0) : 0.0;
            v[w][1] = c < ca.G ? __ldcg(ps + 1) : 0.0;
            v[w][2] = c < ca.G ? __ldcg(ps + 2) : 0.0;
          }
#pragma unroll
          for (int w = 0; w < 5; ++w) { t0 += v[w][0]; t1 += v[w][1]; t2 += v[w][2]; }
        }
        t0 = warp_sum(t0);
        t1 = warp_sum(t1);
        t2 = warp_sum(t2);
        finish_pass(lp, lp.probs, &sst, i_single, t0, t1, t2);
      }
      __syncthreads();
    }
  }
  if (failed) {   // a grid barrier timed out: record it, leave psi untouched
    if (threadIdx.x == 0) {
      for (int b = 0; b < lp.nprob; ++b) { lp.states[b].error = ERR_BARRIER; lp.states[b].stopped = 1; }
    }
    return;
  }
  if (!probe) {
    // psi <- sum_j C_j q^_j on this CTA's units, problem by problem
    int b = problem_of_unit(lp, t_begin);
    for (int t = t_begin; t < t_end; ++b) {
      const Problem* pr = lp.probs + b;
      const int seg_end = min(t_end, pr->tile_begin + pr->ntiles);
      const DevState* stp = SINGLE ? &sst : lp.states + b;
      if (threadIdx.x <= KMAX) {
        const double a = SINGLE ? stp->coef_re[threadIdx.x] : __ldcg(&stp->coef_re[threadIdx.x]);
        const double c = SINGLE ? stp->coef_im[threadIdx.x] : __ldcg(&stp->coef_im[threadIdx.x]);
        cr_s[threadIdx.x] = a;
        ci_s[threadIdx.x] = c;
        const float ah = (float)a, ch = (float)c;
        crh_s[threadIdx.x] = ah; crl_s[threadIdx.x] = (float)(a - (double)ah);
        cih_s[threadIdx.x] = ch; cil_s[threadIdx.x] = (float)(c - (double)ch);
      }
      if (threadIdx.x == 0) {
        rk_s = SINGLE ? stp->k_used : __ldcg(&stp->k_used);
        rerr_s = SINGLE ? stp->error : __ldcg(&stp->error);
      }
      __syncthreads();
      if (!rerr_s) {
        const long long n = (long long)pr->nx * pr->ny;
        vec4* psi = const_cast<vec4*>(pr->psi);
        for (int tt = t; tt < seg_end; ++tt) {
          const int lt = tt - pr->tile_begin;
          const int x0 = (lt % pr->tiles_x) * W, y0 = (lt / pr->tiles_x) * H;
          for (int e = threadIdx.x; e < W * H; e += NT) {
            const int x = x0 + e % W, y = y0 + e / W;
            if (x < pr->nx && y < pr->ny)
              recombine_site_df<16>(psi, static_cast<const float4*>(pr->basis), (size_t)n, (size_t)y * pr->nx + x,
                                    rk_s, cr_s, ci_s, crh_s, crl_s, cih_s, cil_s);
          }
        }
        // re-arm the problem for the next step (the CTA holding its first unit)
        if (!SINGLE && threadIdx.x == 0 && t == pr->tile_begin) {
          DevState* st = lp.states + b;
          st->stopped = 0;
          st->cur_pass = 1;
          st->redo_left = lp.redo_budget;
        }
      }
      __syncthreads();
      t = seg_end;
    }
  }
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0 && !probe) *const_cast<int*>(lp.step) = step + 1;
    if (SINGLE) {   // publish the state (identical in every CTA), re-armed for the next step
      __syncthreads();
      if (threadIdx.x == 0 && !probe && !sst.error) {
        sst.stopped = 0;
        sst.cur_pass = 1;
        sst.redo_left = lp.redo_budget;
      }
      __syncthreads();
      const unsigned* src = reinterpret_cast<const unsigned*>(&sst);
      unsigned* dst = reinterpret_cast<unsigned*>(lp.states);
      for (int w = threadIdx.x; w < (int)(sizeof(DevState) / sizeof(unsigned)); w += NT) dst[w] = src[w];
    }
  }
}

template <int R, bool SINGLE>
cudaError_t launch_t(LaunchParams p, int n_sm, CoopArgs ca, cudaStream_t s) {
  static std::atomic<int> occ_dev[OCC_MAX_DEVICES];
  int occ = 0;
  cudaError_t e = occupancy_on_device(occ_dev, lanczos_sweep<R, SINGLE>, NT, 0, &occ);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorCooperativeLaunchTooLarge;
  // one CTA per SM, at most one per unit, so that every CTA has a unit in
  // every pass
  int grid = std::max(1, std::min(p.total_tiles, n_sm * occ));
  if (SINGLE) grid = std::min(grid, ca.cap);
  p.chunk_q = p.total_tiles / grid;
  p.chunk_r = p.total_tiles % grid;
  ca.bar_count = grid + ca.bar_count;
  ca.G = grid;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, lanczos_sweep<R, SINGLE>, p, ca);
}

}  // namespace sweep

cudaError_t launch_step_sweep(int order, bool diri, const LaunchParams& p, int n_sm, const CoopArgs& ca,
                              cudaStream_t s) {
  LaunchParams q = p;
  q.diri = diri ? 1 : 0;
  const bool single = p.nprob == 1;
  if (order == 2)
    return single ? sweep::launch_t<1, true>(q, n_sm, ca, s) : sweep::launch_t<1, false>(q, n_sm, ca, s);
  return single ? sweep::launch_t<2, true>(q, n_sm, ca, s) : sweep::launch_t<2, false>(q, n_sm, ca, s);
}

}  // namespace dirac
