// dirac_step32.cu -- the mixed-precision time step as one cooperative launch:
// every Lanczos pass (Fig. 1, Eq. 4) of every problem of a table and the
// recombination (Eq. 17), with the tiles of each pass streamed into shared
// memory by bulk asynchronous tensor copies, and the recombination summed in
// compensated FP32 arithmetic.
//
// Launch: every CTA resident (cooperative; two per SM where the shared
// memory allows, for more warps to hide latency), each owning the same
// contiguous chunk of the tile list in every pass (the tiles it writes in a
// pass are the ones it reads in the next, apart from halos).  Warp roles:
//   * producer (the last warp): for each tile of the chunk, the tile and its
//     halo of the pass's two input fields (y^_{i-1} and q^_{i-1}; the
//     complex128 state psi in passes 1 and 2) are copied into a ring of
//     STAGES shared-memory stages by one tensor copy per field (a box of
//     (32 + 2R) x (16 + 2R) sites; zeros outside the grid), completion counted
//     in bytes on the stage's "full" mbarrier.  Where the driver refuses a
//     tensor map the rows are copied one by one with cp.async.bulk instead.
//   * consumers (NCW warps): wait for a stage, form q^_i = g y^_{i-1} -
//     gd q^_{i-1} on the tile and its halo into a formed-tile buffer, release
//     the stage, then apply the stencil, store q^_i and y^_i, and accumulate
//     P = Re<q^_i, y^_i>, Y = ||y^_i||^2, X = ||q^_i||^2 (FP32 within a tile,
//     compensated FP32 across a thread's tiles, FP64 across threads).
// Between passes: a bounded grid barrier.  One problem: every CTA sums all CTA
// partials in the same order and updates its own shared-memory copy of the
// scalars (identical everywhere).  Several problems: the last CTA to finish a
// problem's tiles sums that problem's partials and updates its scalars in
// global memory before the barrier (as the per-pass kernel does).
//
// Precision.  The stencil product runs in FP32 on the complex64 tile, each
// coefficient (c / 2dx, c A, the diagonal m c^2 - s - sigma + V) entering as
// an FP32 value plus its remainder.  The recombination sums its complex64
// terms with compensation (exact products, two-sum accumulation): measured
// on 500 steps of the fastest packets of the batched workload, plain FP32
// accumulation there tripled the error, while a compensated stencil product
// did not lower the largest error.
#include "dirac.h"
#include "dirac_internal.h"
#include "dirac_kernels.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>

namespace dirac {
namespace m32 {

constexpr int TH = M32_TILE_H;     // tile height (sites)
constexpr int NCW = 8;             // consumer warps
constexpr int NC = 32 * NCW;       // consumer threads
constexpr int NT = NC + 32;        // and the producer warp
constexpr int RPT = TH / NCW;      // rows per consumer thread
constexpr int STAGES = 3;          // shared-memory ring depth (two CTAs share an SM)
constexpr long long WAIT_CYCLES = 4000000000LL;   // bounded waits: about two seconds at 2 GHz

constexpr int round128(int b) { return (b + 127) & ~127; }

template <int R>
struct Geo {
  static constexpr int W = TILE_W + 2 * R;   // row of a tile with its halo
  static constexpr int HR = TH + 2 * R;      // rows with the halo
  static constexpr int NS = W * HR;          // sites of the rectangle
  static constexpr int A_BYTES = round128(NS * 16);   // y^_{i-1}: complex64 spinors
  static constexpr int B_BYTES = round128(NS * 32);   // q^_{i-1}: complex128 (psi) or complex64
  static constexpr int STAGE = A_BYTES + B_BYTES;     // tensor-copy destinations stay 128-byte aligned
  static constexpr int QT = round128(NS * 16);        // formed q^_i (complex64)
  static constexpr int SMEM = STAGES * STAGE + 2 * QT + 128;   // + alignment slack
};

// ---------------------------------------------------------------------------
// shared-memory barriers and bulk copies
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned saddr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of `bar` with parity `parity`.  Bounded: false once
// *abort is raised (by anyone) or after WAIT_CYCLES, which raises it.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, volatile int* abort) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (*abort) return false;
    if (clock64() - t0 > WAIT_CYCLES) {
      *abort = 1;
      return false;
    }
  }
}

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// global -> shared bulk copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned), completion counted on `bar`
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(bar)), "l"(pol)
      : "memory");
}

// one box of a tensor map (2D: {x, y}; 3D: {x, y, z}) -> shared memory,
// completion counted on `bar`; elements outside the tensor arrive as zeros
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar,
                                            uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(saddr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(saddr(bar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar,
                                            uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(saddr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(saddr(bar)), "l"(pol)
      : "memory");
}

// the tensor maps live in global memory, written by the host before the
// launch: make them visible to the tensor copies of this kernel
__device__ __forceinline__ void fence_tensormap(const CUtensorMap* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

// generic-proxy writes to global memory (other CTAs' stores of the previous
// pass) made visible to this thread's later bulk copies, and the reverse
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NC) : "memory"); }

// Coefficients of one pass of one problem, FP32 pairs.
struct StencilCoef {
  float kxh, kxl, kyh, kyl;       // c / (2 dx) (order 2) or c / (12 dx) (order 4)
  float axh, axl, ayh, ayl;       // c A_x, c A_y
  float auh, aul, adh, adl;       // m c^2 - s - sigma, -m c^2 - s - sigma
  float e;                        // coupling to q^_{i-1}
  bool has_ay;
};

// (H - s - sigma) q^ - e q^_{i-1} at one site of the formed tile (row r,
// column c of the rectangle), V given as a pair (vh, vl).  FP32 products and
// sums; every coefficient enters as a value plus its remainder, so that its
// own rounding is not a constant perturbation of the operator (the diagonal
// m c^2 - s - sigma reaches 2 m c^2).
template <int R>
__device__ __forceinline__ void site_stencil(const float4* qt, int r, int c, const StencilCoef& k, float vh, float vl,
                                             const float (&qp)[4], float4& C, float (&y)[4]) {
  constexpr int W = Geo<R>::W;
  C = qt[r * W + c];
  const float4 E1 = qt[r * W + c + 1], W1 = qt[r * W + c - 1];
  const float4 N1 = qt[(r + 1) * W + c], S1 = qt[(r - 1) * W + c];
  float dx[4] = {E1.x - W1.x, E1.y - W1.y, E1.z - W1.z, E1.w - W1.w};
  float dy[4] = {N1.x - S1.x, N1.y - S1.y, N1.z - S1.z, N1.w - S1.w};
  if constexpr (R == 2) {   // D f = 8 (f[j+1] - f[j-1]) - (f[j+2] - f[j-2]), coefficient c / (12 h)
    const float4 E2 = qt[r * W + c + 2], W2 = qt[r * W + c - 2];
    const float4 N2 = qt[(r + 2) * W + c], S2 = qt[(r - 2) * W + c];
    dx[0] = fmaf(8.f, dx[0], W2.x - E2.x); dx[1] = fmaf(8.f, dx[1], W2.y - E2.y);
    dx[2] = fmaf(8.f, dx[2], W2.z - E2.z); dx[3] = fmaf(8.f, dx[3], W2.w - E2.w);
    dy[0] = fmaf(8.f, dy[0], S2.x - N2.x); dy[1] = fmaf(8.f, dy[1], S2.y - N2.y);
    dy[2] = fmaf(8.f, dy[2], S2.z - N2.z); dy[3] = fmaf(8.f, dy[3], S2.w - N2.w);
  }
  // diagonals with V as FP32 pairs: the sum (up to 2 m c^2) rounds differently
  // at every site, so its rounding error goes into the remainder
  float au, ad, ru, rd;
  two_sum(k.auh, vh, au, ru);
  two_sum(k.adh, vh, ad, rd);
  const float aul = k.aul + vl + ru, adl = k.adl + vl + rd;
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
  // remainders of the coefficients, and the coupling to q^_{i-1}
  y0 = fmaf(aul, C.x, fmaf(k.kxl, dx[3], fmaf(-k.kyl, dy[2], fmaf(k.axl, C.z, fmaf(-k.e, qp[0], y0)))));
  y1 = fmaf(aul, C.y, fmaf(-k.kxl, dx[2], fmaf(-k.kyl, dy[3], fmaf(k.axl, C.w, fmaf(-k.e, qp[1], y1)))));
  y2 = fmaf(adl, C.z, fmaf(k.kxl, dx[1], fmaf(k.kyl, dy[0], fmaf(k.axl, C.x, fmaf(-k.e, qp[2], y2)))));
  y3 = fmaf(adl, C.w, fmaf(-k.kxl, dx[0], fmaf(k.kyl, dy[1], fmaf(k.axl, C.y, fmaf(-k.e, qp[3], y3)))));
  y[0] = y0; y[1] = y1; y[2] = y2; y[3] = y3;
}

// The input fields of pass i of problem pr: A = y^_{i-1} (complex64; none in
// pass 1), B = q^_{i-1} (passes 1 and 2: the complex128 state psi, which is
// q^_1; later the complex64 basis vector q^_{i-1}).
struct PassFields {
  const char* A;
  const char* B;
  int sbB;          // bytes per site of B
};
__device__ __forceinline__ PassFields pass_fields(const Problem* pr, int i) {
  PassFields f;
  const size_t n = (size_t)pr->nx * pr->ny;
  f.A = (i >= 2) ? static_cast<const char*>(((i - 1) & 1) ? pr->ybuf1 : pr->ybuf0) : nullptr;
  if (i <= 2) {
    f.B = reinterpret_cast<const char*>(pr->psi);
    f.sbB = 32;
  } else {
    f.B = static_cast<const char*>(pr->basis) + (size_t)(i - 3) * n * 16;
    f.sbB = 16;
  }
  return f;
}

// One row of a field for the rectangle of a tile, done by one producer
// thread: generic writes first (zeros, small-grid elements) when `generic`,
// else the bulk copies; returns the bytes of the bulk copies.
template <int R>
__device__ __forceinline__ unsigned row_copy(bool generic, const char* field, int sb, char* dst_row, int nx, int ny,
                                             int x0, int gy, bool diri, uint64_t* bar, uint64_t pol) {
  constexpr int W = Geo<R>::W;
  unsigned bytes = 0;
  const bool yout = gy < 0 || gy >= ny;
  if (diri && yout) {           // a row outside the grid: zeros
    if (generic)
      for (int c = 0; c < W * sb / 16; ++c) reinterpret_cast<float4*>(dst_row)[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    return 0;
  }
  int iy = gy % ny;
  if (iy < 0) iy += ny;
  const char* src_row = field + (size_t)iy * nx * sb;
  if (nx >= W) {
    // columns c <-> gx = x0 - R + c; [cl, cr) lie inside the grid
    const int cl = x0 - R < 0 ? R - x0 : 0;
    const int cr = min(W, nx - x0 + R);
    if (!generic) {
      const int mid = cr - cl;
      bulk_load(dst_row + cl * sb, src_row + (size_t)(x0 - R + cl) * sb, (unsigned)(mid * sb), bar, pol);
      bytes += (unsigned)(mid * sb);
      if (!diri) {
        if (cl > 0) {           // left halo wraps to the end of the row
          bulk_load(dst_row, src_row + (size_t)(nx - cl) * sb, (unsigned)(cl * sb), bar, pol);
          bytes += (unsigned)(cl * sb);
        }
        if (cr < W) {           // right part wraps to the start of the row
          bulk_load(dst_row + cr * sb, src_row, (unsigned)((W - cr) * sb), bar, pol);
          bytes += (unsigned)((W - cr) * sb);
        }
      }
    } else if (diri) {
      float4* d = reinterpret_cast<float4*>(dst_row);
      const int q = sb / 16;
      for (int c = 0; c < cl * q; ++c) d[c] = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int c = cr * q; c < W * q; ++c) d[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    return bytes;
  }
  if (generic) {                // narrow grid: element by element
    const int q = sb / 16;
    for (int c = 0; c < W; ++c) {
      const int gx = x0 - R + c;
      const bool xout = gx < 0 || gx >= nx;
      int ix = gx % nx;
      if (ix < 0) ix += nx;
      for (int h = 0; h < q; ++h) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (!(diri && xout)) v = reinterpret_cast<const float4*>(src_row + (size_t)ix * sb)[h];
        reinterpret_cast<float4*>(dst_row + c * sb)[h] = v;
      }
    }
  }
  return 0;
}

// Producer: the stage of one tile (all 32 threads of the producer warp).
// By tensor copies, one box per field (zeros outside the grid; the
// consumers patch periodic halos); else row by row.  Either way every byte
// in flight is announced (expect-tx) before its copy is issued, and the
// warp's single arrival comes last.
template <int R>
__device__ __forceinline__ void produce_tile(const LaunchParams& lp, int b, const Problem* pr, int i, int tt,
                                             unsigned char* stage, uint64_t* full, bool diri, uint64_t pol) {
  using G = Geo<R>;
  const int lane = threadIdx.x & 31;
  const int lt = tt - pr->tile_begin;
  const int x0 = (lt % pr->tiles_x) * TILE_W;
  const int y0 = (lt / pr->tiles_x) * TH;
  char* A = reinterpret_cast<char*>(stage);
  char* B = reinterpret_cast<char*>(stage) + G::A_BYTES;
  if (pr->tma) {
    if (lane == 0) {
      const TmaMaps* mp = lp.maps + b;
      const int xe = 4 * (x0 - R), ye = y0 - R;   // element coordinates (16- or 32-byte multiples)
      const unsigned bytes = (i >= 2 ? G::NS * 16u : 0u) + (i <= 2 ? G::NS * 32u : G::NS * 16u);
      mbar_arrive_expect_tx(full, bytes);
      if (i >= 2) tma_load_3d(A, &mp->ybuf, xe, ye, (i - 1) & 1, full, pol);
      if (i <= 2) tma_load_2d(B, &mp->psi, xe, ye, full, pol);
      else tma_load_3d(B, &mp->basis, xe, ye, i - 3, full, pol);
    }
    return;
  }
  const PassFields f = pass_fields(pr, i);
  const int nf = (i == 1) ? 1 : 2;     // pass 1 reads psi only
  unsigned bytes = 0;
  // generic writes first (zeros, narrow grids)
  for (int p = lane; p < nf * G::HR; p += 32) {
    const bool fb = (nf == 1) || p >= G::HR;
    const int r = fb && nf == 2 ? p - G::HR : p;
    const int sb = fb ? f.sbB : 16;
    row_copy<R>(true, fb ? f.B : f.A, sb, (fb ? B : A) + r * G::W * sb, pr->nx, pr->ny, x0, y0 - R + r, diri, full,
                pol);
  }
  // bytes of this thread's copies (the same plan, without issuing)
  for (int p = lane; p < nf * G::HR; p += 32) {
    const bool fb = (nf == 1) || p >= G::HR;
    const int r = fb && nf == 2 ? p - G::HR : p;
    const int sb = fb ? f.sbB : 16;
    const int gy = y0 - R + r;
    if (diri && (gy < 0 || gy >= pr->ny)) continue;
    if (pr->nx < G::W) continue;
    const int cl = x0 - R < 0 ? R - x0 : 0;
    const int cr = min(G::W, pr->nx - x0 + R);
    bytes += (unsigned)((cr - cl) * sb);
    if (!diri) bytes += (unsigned)((cl + (G::W - cr)) * sb);
  }
  if (bytes) mbar_expect_tx(full, bytes);
  for (int p = lane; p < nf * G::HR; p += 32) {
    const bool fb = (nf == 1) || p >= G::HR;
    const int r = fb && nf == 2 ? p - G::HR : p;
    const int sb = fb ? f.sbB : 16;
    row_copy<R>(false, fb ? f.B : f.A, sb, (fb ? B : A) + r * G::W * sb, pr->nx, pr->ny, x0, y0 - R + r, diri, full,
                pol);
  }
  __syncwarp();
  if (lane == 0) mbar_arrive(full);
}

__device__ __forceinline__ int problem_of_tile(const LaunchParams& lp, int t) {
  int lo = 0, hi = lp.nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (lp.probs[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// scalars of problem b at the start of a pass: the CTA's shared copy (one
// problem) or the global block written before the grid barrier
template <bool SINGLE>
__device__ __forceinline__ void pass_state(const LaunchParams& lp, const DevState* sst, int b, int& stopped, int& i) {
  if (SINGLE) {
    stopped = sst->stopped;
    i = max(1, sst->cur_pass);
  } else {
    const DevState* st = lp.states + b;
    stopped = __ldcg(&st->stopped);
    i = max(1, __ldcg(&st->cur_pass));
  }
}

template <int R, bool SINGLE>
__global__ void __launch_bounds__(NT, 2) lanczos_step_m32(const __grid_constant__ LaunchParams lp,
                                                         const __grid_constant__ CoopArgs ca) {
  using G = Geo<R>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* const smem = smem_raw + ((128u - (saddr(smem_raw) & 127u)) & 127u);
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES];
  __shared__ DevState sst;              // one problem: this CTA's copy of its scalars
  __shared__ double red[NCW][3];
  __shared__ int abort_s;
  __shared__ double cr_s[KMAX + 2], ci_s[KMAX + 2];
  __shared__ float crh_s[KMAX + 2], crl_s[KMAX + 2], cih_s[KMAX + 2], cil_s[KMAX + 2];
  __shared__ int rk_s, rerr_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool producer = warp == NCW;
  const int cq = lp.chunk_q, crm = lp.chunk_r;
  const int t_begin = blockIdx.x * cq + min((int)blockIdx.x, crm);
  const int t_end = t_begin + cq + ((int)blockIdx.x < crm ? 1 : 0);
  const bool diri = lp.diri != 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    abort_s = 0;
  }
  if (SINGLE) {
    const unsigned* src = reinterpret_cast<const unsigned*>(lp.states);
    unsigned* dst = reinterpret_cast<unsigned*>(&sst);
    for (int w = threadIdx.x; w < (int)(sizeof(DevState) / sizeof(unsigned)); w += NT) dst[w] = __ldcg(src + w);
  }
  const int step = __ldcg(lp.step);
  __syncthreads();

  const int max_iter = lp.m + lp.redo_budget;
  unsigned it = 0;            // tiles streamed so far in this launch (ring position)
  int iter = 0;
  bool failed = false;
  const uint64_t pol = policy_evict_first();
  while (iter < max_iter) {
    if (SINGLE && sst.stopped) break;
    double* slots = ca.slots + (iter & 1) * 3 * ca.G;
    int i_single = SINGLE ? max(1, sst.cur_pass) : 0;
    if (producer) {
      fence_proxy_async_global();
      int b = problem_of_tile(lp, t_begin);
      for (int t = t_begin; t < t_end && !failed; ++b) {
        const Problem* pr = lp.probs + b;
        int stopped, i;
        pass_state<SINGLE>(lp, &sst, b, stopped, i);
        const int seg_end = min(t_end, pr->tile_begin + pr->ntiles);
        if (!stopped) {
          if (pr->tma && lane == 0) {
            fence_tensormap(&lp.maps[b].basis);
            fence_tensormap(&lp.maps[b].ybuf);
            fence_tensormap(&lp.maps[b].psi);
          }
          for (int tt = t; tt < seg_end; ++tt, ++it) {
            const int s = it % STAGES;
            const unsigned ph = (it / STAGES) & 1u;
            if (!mbar_wait(&empty_bar[s], ph ^ 1u, &abort_s)) { failed = true; break; }
            produce_tile<R>(lp, b, pr, i, tt, smem + (size_t)s * G::STAGE, &full_bar[s], diri, pol);
          }
        }
        t = seg_end;
      }
    } else {
      const int ctid = threadIdx.x;             // 0 .. NC-1
      const int tx = lane, tg = warp;
      int b = problem_of_tile(lp, t_begin);
      for (int t = t_begin; t < t_end; ++b) {
        const Problem* pr = lp.probs + b;
        int stopped, i;
        pass_state<SINGLE>(lp, &sst, b, stopped, i);
        const int seg_end = min(t_end, pr->tile_begin + pr->ntiles);
        const int seg_tiles = seg_end - t;
        if (stopped) { t = seg_end; continue; }
        const DevState* stp = SINGLE ? &sst : lp.states + b;
        PassCoef pc;
        if (SINGLE) {
          pc = sst.pc_cur;
        } else {
          const double* src = reinterpret_cast<const double*>(&stp->pc_cur);
          double* dst = reinterpret_cast<double*>(&pc);
          for (int w = 0; w < (int)(sizeof(PassCoef) / sizeof(double)); ++w) dst[w] = __ldcg(src + w);
        }
        const FieldStep fs = lp.fields[step * lp.fstride + b];
        StencilCoef k;
        k.kxh = pr->kxf; k.kxl = pr->kxf_lo; k.kyh = pr->kyf; k.kyl = pr->kyf_lo;
        k.axh = fs.cAxf; k.axl = fs.cAxf_lo; k.ayh = fs.cAyf; k.ayl = fs.cAyf_lo;
        k.auh = pc.au_hi; k.aul = pc.au_lo; k.adh = pc.ad_hi; k.adl = pc.ad_lo;
        k.e = (i >= 2) ? pc.ef : 0.f;
        k.has_ay = fs.cAy != 0.0;
        const float gS = pc.gf, gdS = pc.gdf;
        const int nx = pr->nx, ny = pr->ny;
        const size_t n = (size_t)nx * ny;
        const PassFields f = pass_fields(pr, i);
        float4* q_out = (i >= 2) ? reinterpret_cast<float4*>(static_cast<char*>(pr->basis) + (size_t)(i - 2) * n * 16)
                                 : nullptr;
        float4* y_out = (i < lp.m) ? static_cast<float4*>((i & 1) ? pr->ybuf1 : pr->ybuf0) : nullptr;
        const float* Vh = static_cast<const float*>(pr->V);
        const float* Vl = static_cast<const float*>(pr->Vlo);
        // per-thread sums over the segment's tiles: FP32 values with two-sum
        // compensation (FP64 arithmetic per tile would cost more than the
        // tile's stencil: the FP64 pipe issues 1/64 of the FP32 rate)
        float sP = 0.f, sY = 0.f, sX = 0.f, cP = 0.f, cY = 0.f, cX = 0.f;
        for (int tt = t; tt < seg_end; ++tt, ++it) {
          const int s = it % STAGES;
          const unsigned ph = (it / STAGES) & 1u;
          const int lt = tt - pr->tile_begin;
          const int x0 = (lt % pr->tiles_x) * TILE_W;
          const int y0 = (lt / pr->tiles_x) * TH;
          const unsigned char* stage = smem + (size_t)s * G::STAGE;
          const float4* A = reinterpret_cast<const float4*>(stage);
          const unsigned char* B = stage + G::A_BYTES;
          float4* qt = reinterpret_cast<float4*>(smem + (size_t)STAGES * G::STAGE + (size_t)(it & 1u) * G::QT);
          if (!mbar_wait(&full_bar[s], ph, &abort_s)) failed = true;
          // a tile staged by tensor copies holds zeros outside the grid; on
          // periodic grids those elements are read from their images instead
          const bool wrapfix = pr->tma && !diri &&
                               (x0 < R || x0 + TILE_W + R > nx || y0 < R || y0 + TH + R > ny);
          // q^_i at rectangle element e = (r, c) (B holds q^_{i-1} at sbB bytes per site)
          auto formed = [&](int e, int r, int c, float (&qp)[4]) -> float4 {
            bool glob = false;
            size_t gi = 0;
            if (wrapfix) {
              const int gx = x0 - R + c, gy = y0 - R + r;
              if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) {
                int ix = gx % nx, iy = gy % ny;
                if (ix < 0) ix += nx;
                if (iy < 0) iy += ny;
                glob = true;
                gi = (size_t)iy * nx + ix;
              }
            }
            if (f.sbB == 32) {
              const double4_32a v = glob ? ldw4(reinterpret_cast<const vec4*>(f.B) + gi)
                                         : reinterpret_cast<const double4_32a*>(B)[e];
              qp[0] = (float)v.x; qp[1] = (float)v.y; qp[2] = (float)v.z; qp[3] = (float)v.w;
            } else {
              const float4 v = glob ? reinterpret_cast<const float4*>(f.B)[gi] : reinterpret_cast<const float4*>(B)[e];
              qp[0] = v.x; qp[1] = v.y; qp[2] = v.z; qp[3] = v.w;
            }
            if (i == 1) return make_float4(qp[0], qp[1], qp[2], qp[3]);
            const float4 yv = glob ? reinterpret_cast<const float4*>(f.A)[gi] : A[e];
            return make_float4(fmaf(-gdS, qp[0], gS * yv.x), fmaf(-gdS, qp[1], gS * yv.y),
                               fmaf(-gdS, qp[2], gS * yv.z), fmaf(-gdS, qp[3], gS * yv.w));
          };
          float qp[RPT][4];
          if (!failed) {
#pragma unroll
            for (int kk = 0; kk < RPT; ++kk) {
              const int r = tg + kk * NCW + R;
              const int e = r * G::W + tx + R;
              qt[e] = formed(e, r, tx + R, qp[kk]);
            }
            constexpr int NH_ROW = 2 * R * G::W, NH = NH_ROW + 2 * R * TH;
            for (int h = ctid; h < NH; h += NC) {
              int r, c;
              if (h < NH_ROW) {         // the rows above and below (full width)
                const int rr = h / G::W;
                r = (rr < R) ? rr : TH + rr;
                c = h % G::W;
              } else {                  // the columns left and right
                const int h2 = h - NH_ROW;
                const int cc = h2 % (2 * R);
                r = h2 / (2 * R) + R;
                c = (cc < R) ? cc : TILE_W + cc;
              }
              const int e = r * G::W + c;
              float dummy[4];
              qt[e] = formed(e, r, c, dummy);
            }
          }
          consumer_sync();
          if (ctid == 0) mbar_arrive(&empty_bar[s]);   // the stage may be refilled
          if (!failed) {
            float tP = 0.f, tY = 0.f, tX = 0.f;
#pragma unroll
            for (int kk = 0; kk < RPT; ++kk) {
              const int ry = tg + kk * NCW;
              const int x = x0 + tx, y = y0 + ry;
              if (x < nx && y < ny) {
                const size_t idx = (size_t)y * nx + x;
                float vh = 0.f, vl = 0.f;
                if (Vh) { vh = __ldg(Vh + idx); vl = __ldg(Vl + idx); }
                float4 C;
                float yv[4];
                site_stencil<R>(qt, ry + R, tx + R, k, vh, vl, qp[kk], C, yv);
                if (q_out) q_out[idx] = C;
                if (y_out) y_out[idx] = make_float4(yv[0], yv[1], yv[2], yv[3]);
                tP = fmaf(C.x, yv[0], fmaf(C.y, yv[1], fmaf(C.z, yv[2], fmaf(C.w, yv[3], tP))));
                tY = fmaf(yv[0], yv[0], fmaf(yv[1], yv[1], fmaf(yv[2], yv[2], fmaf(yv[3], yv[3], tY))));
                tX = fmaf(C.x, C.x, fmaf(C.y, C.y, fmaf(C.z, C.z, fmaf(C.w, C.w, tX))));
              }
            }
            float t, r;
            two_sum(sP, tP, t, r); sP = t; cP += r;
            two_sum(sY, tY, t, r); sY = t; cY += r;
            two_sum(sX, tX, t, r); sX = t; cX += r;
          }
        }
        // this CTA's share of problem b: warps -> CTA, one partial per slot
        double accP = warp_sum((double)sP + (double)cP);
        double accY = warp_sum((double)sY + (double)cY);
        double accX = warp_sum((double)sX + (double)cX);
        if (lane == 0) { red[warp][0] = accP; red[warp][1] = accY; red[warp][2] = accX; }
        consumer_sync();
        if (warp == 0) {
          double s0 = 0.0, s1 = 0.0, s2 = 0.0;
          if (lane < NCW) { s0 = red[lane][0]; s1 = red[lane][1]; s2 = red[lane][2]; }
#pragma unroll
          for (int o = NCW / 2; o > 0; o >>= 1) {
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
              last = ticket.fetch_add((unsigned)seg_tiles, cuda::memory_order_acq_rel) + seg_tiles ==
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
        consumer_sync();   // red[] is reused by the next problem
        t = seg_end;
      }
      // this thread's stores of the pass, visible to the bulk copies of the next
      fence_proxy_async_global();
    }
    ++iter;
    if (__syncthreads_or(failed ? 1 : 0)) failed = true;
    if (failed || !grid_sync(ca.bar, (unsigned)ca.bar_count)) {
      failed = true;
      break;
    }
    if (SINGLE) {
      if (warp == 0) {   // the grid totals, in the same order in every CTA
        double t0 = 0.0, t1 = 0.0, t2 = 0.0;
        for (int c0 = 0; c0 < ca.G; c0 += 5 * 32) {   // five slots per lane in flight at once
          double v[5][3];
#pragma unroll
          for (int u = 0; u < 5; ++u) {
            const int c = c0 + lane + 32 * u;
            const double* ps = slots + 3 * (c < ca.G ? c : 0);
            v[u][0] = c < ca.G ? __ldcg(ps + 0) : 0.0;
            v[u][1] = c < ca.G ? __ldcg(ps + 1) : 0.0;
            v[u][2] = c < ca.G ? __ldcg(ps + 2) : 0.0;
          }
#pragma unroll
          for (int u = 0; u < 5; ++u) { t0 += v[u][0]; t1 += v[u][1]; t2 += v[u][2]; }
        }
        t0 = warp_sum(t0);
        t1 = warp_sum(t1);
        t2 = warp_sum(t2);
        finish_pass(lp, lp.probs, &sst, i_single, t0, t1, t2);
      }
      __syncthreads();
    }
  }
  if (failed) {
    // a bounded wait gave up: let every copy already issued land before the
    // CTA exits (bounded too), record the error, leave psi untouched
    if (producer) {
      for (unsigned q = (it >= STAGES ? it - STAGES : 0); q < it; ++q) {
        const int s = q % STAGES;
        volatile int never = 0;
        mbar_wait(&full_bar[s], (q / STAGES) & 1u, &never);
      }
    }
    if (threadIdx.x == 0) {
      for (int b = 0; b < lp.nprob; ++b) { lp.states[b].error = ERR_BARRIER; lp.states[b].stopped = 1; }
    }
    return;
  }
  // psi <- sum_j C_j q^_j on this CTA's tiles, problem by problem
  {
    int b = problem_of_tile(lp, t_begin);
    for (int t = t_begin; t < t_end; ++b) {
      const Problem* pr = lp.probs + b;
      const int seg_end = min(t_end, pr->tile_begin + pr->ntiles);
      const DevState* stp = SINGLE ? &sst : lp.states + b;
      if (threadIdx.x <= KMAX) {
        const double a = SINGLE ? stp->coef_re[threadIdx.x] : __ldcg(&stp->coef_re[threadIdx.x]);
        const double c = SINGLE ? stp->coef_im[threadIdx.x] : __ldcg(&stp->coef_im[threadIdx.x]);
        cr_s[threadIdx.x] = a; ci_s[threadIdx.x] = c;
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
          const int x0 = (lt % pr->tiles_x) * TILE_W, y0 = (lt / pr->tiles_x) * TH;
          for (int e = threadIdx.x; e < TILE_W * TH; e += NT) {
            const int x = x0 + (e & (TILE_W - 1)), y = y0 + e / TILE_W;
            if (x < pr->nx && y < pr->ny)
              recombine_site_df<16>(psi, static_cast<const float4*>(pr->basis), (size_t)n, (size_t)y * pr->nx + x, rk_s,
                                cr_s, ci_s, crh_s, crl_s, cih_s, cil_s);
          }
        }
        // re-arm the problem for the next step (the CTA holding its first tile)
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
    if (threadIdx.x == 0) *const_cast<int*>(lp.step) = step + 1;
    if (SINGLE) {   // publish the state (identical in every CTA), re-armed for the next step
      __syncthreads();
      if (threadIdx.x == 0 && !sst.error) { sst.stopped = 0; sst.cur_pass = 1; sst.redo_left = lp.redo_budget; }
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
  constexpr size_t smem = Geo<R>::SMEM;
  int occ = 0;
  cudaError_t e = occupancy_on_device(occ_dev, lanczos_step_m32<R, SINGLE>, NT, smem, &occ);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorCooperativeLaunchTooLarge;
  // as many CTAs as are resident (two per SM for the order-2 stencil, whose
  // rings fit twice in shared memory), at most one per tile, so that every
  // CTA has a tile in every pass
  int grid = std::max(1, std::min(p.total_tiles, n_sm * occ));
  if (SINGLE) grid = std::min(grid, ca.cap);
  p.chunk_q = p.total_tiles / grid;
  p.chunk_r = p.total_tiles % grid;
  ca.bar_count = grid + ca.bar_count;
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
  return cudaLaunchKernelEx(&cfg, lanczos_step_m32<R, SINGLE>, p, ca);
}

}  // namespace m32

cudaError_t launch_step_m32(int order, bool diri, const LaunchParams& p, int n_sm, const CoopArgs& ca,
                            cudaStream_t s) {
  LaunchParams q = p;
  q.diri = diri ? 1 : 0;
  q.probe = 0;
  const bool single = p.nprob == 1;
  if (order == 2) return single ? m32::launch_t<1, true>(q, n_sm, ca, s) : m32::launch_t<1, false>(q, n_sm, ca, s);
  return single ? m32::launch_t<2, true>(q, n_sm, ca, s) : m32::launch_t<2, false>(q, n_sm, ca, s);
}

}  // namespace dirac
