// qpm_adjoint.cu -- relaxed d_eff and its hand-written adjoint.
//
// Relaxation: d_j = tanh(theta_j) in (-1, 1).  The closed form of the Sec. 2.1
// integral holds for any real piecewise-constant d:
//   D = phi1 phi2 sum_j a_j P_j + psi sum_j d_j^2 q_j,
//   a_j = d_j p2_j, b_j = d_j p1_j, P_j = sum_{m<j} b_m, q_j = p1_j p2_j,
// and f = |D|^2.  Its derivative with respect to d_k is
//   dD/dd_k = phi1 phi2 (p2_k P_k + p1_k R_k) + 2 psi d_k q_k,  R_k = sum_{j>k} a_j,
//   df/dtheta_k = 2 Re(conj(D) dD/dd_k) (1 - d_k^2).
//
// Work split (both passes): a warp takes 32 rows (lane = row) and one segment of
// L domains (L a multiple of 32 fixed by N alone, at most 256) and sweeps the
// segment in index order in steps of 32 domains.  A step's 32 x 32 theta tile
// arrives in shared memory ahead of its use: for 16-byte aligned rows as one 2-D
// TMA copy (cp.async.bulk.tensor, 128-byte swizzle, zero fill past the row ends and
// the last row) that completes on a per-warp mbarrier, otherwise through registers.
// Every lane then walks its own row: the running sums are plain sequential sums and
// every phasor read is a broadcast.  The warps of a CTA take consecutive row groups
// of the same segment and share its staged phasors.
//
// Forward: every (row, segment) writes its partial sums (A_s, B_s, C_s, E_s) into
// the row's saved block; a second kernel (a warp per row, lanes over segments,
// launched as a programmatic dependent so that its launch overlaps the first one's
// tail) combines the segments in index order (C = sum_s C_s + A_s Bpre_s with
// Bpre_s the b-sum of the segments before s), closes D and overwrites each segment's
// (A_s, B_s) with the exclusive prefixes (Apre_s, Bpre_s).
// Backward: each (row, segment) starts from those prefixes (P = Bpre_s,
// R = A - Apre_s), updates P_k and R_k as it goes and writes the gradient back
// through the same tile: a 2-D TMA store where the gradient rows are 16-byte
// aligned and the tile lies wholly inside the matrix, coalesced stores otherwise.
//
// Every wait on an mbarrier is bounded by %globaltimer.  A wait that runs out fills
// its tile with NaN, so that the call's results (d_eff, fit, gradient) come out NaN
// instead of silently wrong, and the warp stops issuing copies.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>

#include <algorithm>
#include <mutex>

#include "qpm_common.cuh"
#include "qpm_internal.h"
#include "qpm_tma.cuh"

namespace qpm {

static constexpr int RX_STEP = 32;   // domains per step (one per lane of a tile row)
static constexpr int RX_LMAX = 256;  // longest segment
static constexpr int RX_WPC = 4;     // warps (row groups of 32) per CTA
static constexpr int RX_TILE = RX_STEP * RX_STEP * 4;  // bytes of one 32 x 32 tile
static constexpr int RX_NST_F = 2;   // tile buffers per warp, forward (one step ahead)
static constexpr int RX_NST_B = 2;   // backward

struct RelaxShape {
  int B, N, L, S;  // rows, domains, segment length, segments
  int64_t ld;      // theta leading dimension
  int64_t sf;      // floats per row of the saved block
};

// segment length: S = ceil(N / L) is about 32 for short rows, L = 256 for long ones
// (4096 x 4096: 32 segments of 128 domains, 4096 warps of work)
static constexpr int RX_SEGQ = 1024;  // about N / 32, rounded up to whole steps
static int rx_seg_len(int N) { return std::min(RX_LMAX, RX_STEP * ((N + RX_SEGQ - 1) / RX_SEGQ)); }
static int rx_nseg(int N) { return (N + rx_seg_len(N) - 1) / rx_seg_len(N); }
// saved block of a row: [A (2 floats), 2 unused, then per segment 8 floats]
static int64_t rx_saved_floats(int N) { return 4 + 8 * (int64_t)rx_nseg(N); }

// Packed FP32 pairs (sm_100+): one 64-bit register pair holds (re, im) of a complex
// sum, and add/mul/fma.rn.f32x2 apply the IEEE-rounded single operation to both
// halves in one instruction.  The forward keeps its a-, b- and d^2 q-sums this way
// (operands straight from the phasor loads); its a P product stays scalar.
typedef unsigned long long f2x;
__device__ __forceinline__ f2x f2_pack(float lo, float hi) {
  f2x r; asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi)); return r; }
__device__ __forceinline__ float2 f2_unpack(f2x v) {
  float2 r; asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v)); return r; }
__device__ __forceinline__ f2x f2_fma(f2x a, f2x b, f2x c) {
  f2x r; asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c)); return r; }
__device__ __forceinline__ f2x f2_mul(f2x a, f2x b) {
  f2x r; asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b)); return r; }
__device__ __forceinline__ f2x f2_add(f2x a, f2x b) {
  f2x r; asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b)); return r; }
// ------------------------------------------------------------- tanh and tiles
__device__ __forceinline__ float ex2_approx(float y) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
  return r;
}

__device__ __forceinline__ float rcp_approx(float y) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
  return r;
}

// d = tanh(x) from one exponential.  With r = 1 / (1 + e^{2|x|}):
//   tanh|x| = 1 - 2r,   1 - tanh^2 x = 4 r (1 - r).
// The second identity keeps the derivative accurate to a few ulp where d is
// close to +-1 (1 - d*d cancels there).  d is accurate to about 3e-7 absolute
// (the hardware 2^y and 1/y approximations, see the parity tests).
__device__ __forceinline__ float tanh_r(float x, float &r) {
  const float E = ex2_approx(fabsf(x) * 2.8853900817779268f);  // 2 log2(e) |x|
  r = rcp_approx(1.f + E);
  return copysignf(fmaf(-2.f, r, 1.f), x);
}

// The per-warp tile holds 32 rows x 32 domains as float4 [row][c4], the column
// xor-swizzled by the row: 8 columns of one row (a quarter-warp of the staging
// stores) and 8 rows of one column (a quarter-warp of the row walks) both fall
// into 8 different 16-byte bank groups.  This is the layout a TMA copy with the
// 128-byte swizzle writes into a 1024-byte aligned tile.
__device__ __forceinline__ int tix(int row, int c4) { return row * 8 + (c4 ^ (row & 7)); }

// Step registers: lane l holds float4 k * 32 + l of the 32 x 8 float4 step,
// i.e. row 4k + l / 8, column l % 8 (4 rows x 128 contiguous bytes per load).
// Any alignment; the path for rows a TMA copy cannot take.
__device__ __forceinline__ void load_step(const float *__restrict__ theta, const RelaxShape &sh,
                                          int r0, int ms, float4 R[8]) {
  const int lane = threadIdx.x & 31;
  const int m = ms + 4 * (lane & 7);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int gr = r0 + 4 * k + (lane >> 3);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gr < sh.B) {
      const float *rp = theta + (int64_t)gr * sh.ld;
      if (m < sh.N) v.x = __ldg(rp + m);
      if (m + 1 < sh.N) v.y = __ldg(rp + m + 1);
      if (m + 2 < sh.N) v.z = __ldg(rp + m + 2);
      if (m + 3 < sh.N) v.w = __ldg(rp + m + 3);
    }
    R[k] = v;
  }
}

__device__ __forceinline__ void put_step(float4 *T, const float4 R[8]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 8; ++k) T[tix(4 * k + (lane >> 3), lane & 7)] = R[k];
}

// after a wait ran out at step t_fail no further copies were issued; the copies of
// steps t_fail and t_fail + 1 may still be in flight: wait for them (bounded again)
// before the CTA's shared memory goes away
__device__ __forceinline__ void drain_loads(unsigned bar0, int nst, int t_fail, int nsteps) {
  if ((threadIdx.x & 31) != 0) return;
  for (int k = t_fail; k < min(t_fail + 2, nsteps); ++k) mbar_wait(bar0 + 8 * (k % nst), (k / nst) & 1);
}

__device__ __forceinline__ void nan_tile(float4 *T) {
  const int lane = threadIdx.x & 31;
  const float n = __int_as_float(0x7fc00000);
#pragma unroll
  for (int c4 = 0; c4 < 8; ++c4) T[tix(lane, c4)] = make_float4(n, n, n, n);
}

// ---------------------------------------------------------- staged phasors
// per domain of the CTA's segment: p = (p1.re, p1.im, p2.re, p2.im) and q = p1 p2
struct Ph {
  float4 p;
  float2 q;
  float2 pad;  // 32 bytes: one entry never straddles two 128-byte lines
};

__device__ __forceinline__ float2 q_of(const float4 &p) {  // q = p1 p2
  return make_float2(p.x * p.z - p.y * p.w, p.x * p.w + p.y * p.z);
}

// phasors of the CTA's segment [m0, m0 + L) (zero beyond N), then a CTA barrier
__device__ __forceinline__ void stage_segment(Ph *ph, const float4 *gtab, int m0, int L, int N) {
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    const int m = m0 + i;
    const float4 p = m < N ? __ldg(gtab + m) : make_float4(0.f, 0.f, 0.f, 0.f);
    ph[i].p = p;
    ph[i].q = q_of(p);
  }
  __syncthreads();
}

// dynamic shared memory: [phasors (L entries)][tiles, 1024-byte aligned][mbarriers]
template <int NST>
static size_t rx_smem_bytes(int L) {
  return 1024 + ((sizeof(Ph) * L + 1023) & ~(size_t)1023) + (size_t)RX_WPC * NST * RX_TILE +
         (size_t)RX_WPC * NST * 8;
}
template <int NST>
__device__ __forceinline__ void rx_carve(unsigned char *raw, int L, Ph *&ph, float4 *&tiles,
                                         unsigned long long *&bars) {
  unsigned char *base =
      raw + ((1024 - (smem_u32(raw) & 1023)) & 1023);  // 1024-byte aligned for the swizzle
  ph = (Ph *)base;
  tiles = (float4 *)(base + ((sizeof(Ph) * L + 1023) & ~(size_t)1023));
  bars = (unsigned long long *)((unsigned char *)tiles + (size_t)RX_WPC * NST * RX_TILE);
}

// The forward sweep of one (row group, segment): (A_s, B_s, C_s, E_s) of its rows
template <bool TMA>
__device__ __forceinline__ void fwd_sweep(const CUtensorMap *tmap, const float *__restrict__ theta,
                                          const RelaxShape &sh, const Ph *ph, float4 *wt,
                                          unsigned bar0, int r0, int m0, float4 R[8], Mono &acc,
                                          float2 &E) {
  constexpr int NST = RX_NST_F;
  const int lane = threadIdx.x & 31;
  const int nsteps = sh.L / RX_STEP;
  bool ok = true;
  int t_fail = -1;  // first step whose tile did not arrive in time
  f2x A2 = 0ull, B2 = 0ull, E2 = 0ull;
  float Cx = 0.f, Cy = 0.f;
  for (int t = 0; t < nsteps; ++t) {
    float4 *T = wt + (t % NST) * (RX_TILE / 16);
    if constexpr (TMA) {
      if (lane == 0 && ok && t + 1 < nsteps) {  // the buffer of step t - 1 is free (see below)
        const int b = (t + 1) % NST;
        fence_async_smem();
        mbar_expect_tx(bar0 + 8 * b, RX_TILE);
        tma_load_tile(wt + b * (RX_TILE / 16), tmap, m0 + (t + 1) * RX_STEP, r0, bar0 + 8 * b);
      }
      const bool arrived = ok && mbar_wait(bar0 + 8 * (t % NST), (t / NST) & 1);
      if (!__all_sync(0xffffffffu, arrived)) {  // ok is uniform across the warp
        if (ok) t_fail = t;
        ok = false;
        nan_tile(T);
      }
      __syncwarp();
    } else {
      __syncwarp();
      put_step(T, R);
      __syncwarp();
      if (t + 1 < nsteps) load_step(theta, sh, r0, m0 + (t + 1) * RX_STEP, R);
    }
    const Ph *pe = ph + t * RX_STEP;
#pragma unroll
    for (int c4 = 0; c4 < 8; ++c4) {
      const float4 x = T[tix(lane, c4)];
      const float th[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float rc;
        const float d = tanh_r(th[j], rc);
        const ulonglong2 pp = *(const ulonglong2 *)&pe[4 * c4 + j].p;
        const f2x qq = *(const f2x *)&pe[4 * c4 + j].q;
        const f2x dd = f2_pack(d, d);
        const f2x a = f2_mul(dd, pp.y);
        const float2 av = f2_unpack(a), bv = f2_unpack(B2);
        Cx = fmaf(av.x, bv.x, Cx);
        Cx = fmaf(-av.y, bv.y, Cx);
        Cy = fmaf(av.x, bv.y, Cy);
        Cy = fmaf(av.y, bv.x, Cy);
        A2 = f2_add(A2, a);
        B2 = f2_fma(dd, pp.x, B2);
        E2 = f2_fma(f2_mul(dd, dd), qq, E2);
      }
    }
    __syncwarp();  // every lane has read T before the copy NST - 1 steps on refills it
  }
  if constexpr (TMA) {
    if (!ok) drain_loads(bar0, NST, t_fail, nsteps);
  }
  acc.A = f2_unpack(A2);
  acc.B = f2_unpack(B2);
  acc.C = make_float2(Cx, Cy);
  E = f2_unpack(E2);
}

// exclusive prefix over lanes of a float2 (lane 0 gets 0); total in `tot`
__device__ __forceinline__ float2 warp_excl_scan2(float2 v, float2 &tot) {
  const int lane = threadIdx.x & 31;
  float2 inc = v;
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
    const float ox = __shfl_up_sync(0xffffffffu, inc.x, s);
    const float oy = __shfl_up_sync(0xffffffffu, inc.y, s);
    if (lane >= s) {
      inc.x += ox;
      inc.y += oy;
    }
  }
  tot.x = __shfl_sync(0xffffffffu, inc.x, 31);
  tot.y = __shfl_sync(0xffffffffu, inc.y, 31);
  return make_float2(inc.x - v.x, inc.y - v.y);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
  return v;
}

// One warp combines the segments of rows [r_begin, r_end), one row at a time, lanes
// over segments (a row's partials are contiguous: coalesced loads, the next row's
// already in flight): C = sum_s C_s + A_s Bpre_s with Bpre_s the b-sum of the
// segments before s; closes D and f, keeps the row's a-sum A and overwrites each
// segment's (A_s, B_s) with the exclusive prefixes (Apre_s, Bpre_s) that the
// backward starts from.
__device__ __forceinline__ void combine_rows(const RelaxShape &sh, const float2 *__restrict__ konst,
                                             float *__restrict__ saved, float2 *__restrict__ Dout,
                                             float *__restrict__ fout, int r_begin, int r_end) {
  const int lane = threadIdx.x & 31;
  const float2 phi12 = konst[0], psi = konst[2];
  const bool one_chunk = sh.S <= 32;
  float4 nab = make_float4(0.f, 0.f, 0.f, 0.f), nce = nab;  // next row's first chunk
  if (one_chunk && r_begin < r_end && lane < sh.S) {
    const float4 *in = (const float4 *)(saved + (int64_t)r_begin * sh.sf + 4 + 8 * lane);
    nab = __ldcg(in);
    nce = __ldcg(in + 1);
  }
  for (int row = r_begin; row < r_end; ++row) {
    float *sv = saved + (int64_t)row * sh.sf;
    float2 cA = make_float2(0.f, 0.f), cB = cA, Cl = cA, El = cA;
    for (int c = 0; c < sh.S; c += 32) {
      const int s = c + lane;
      float4 ab, ce;
      if (one_chunk) {
        ab = nab;
        ce = nce;
        if (row + 1 < r_end && lane < sh.S) {
          const float4 *in = (const float4 *)(sv + sh.sf + 4 + 8 * lane);
          nab = __ldcg(in);
          nce = __ldcg(in + 1);
        }
      } else {
        ab = make_float4(0.f, 0.f, 0.f, 0.f);
        ce = ab;
        if (s < sh.S) {
          const float4 *in = (const float4 *)(sv + 4 + 8 * (int64_t)s);
          ab = __ldcg(in);
          ce = __ldcg(in + 1);
        }
      }
      float2 tA, tB;
      const float2 xA = warp_excl_scan2(make_float2(ab.x, ab.y), tA);
      const float2 xB = warp_excl_scan2(make_float2(ab.z, ab.w), tB);
      const float2 Ap = make_float2(cA.x + xA.x, cA.y + xA.y);
      const float2 Bp = make_float2(cB.x + xB.x, cB.y + xB.y);
      // this segment's pairs plus its a-sum times every b before it
      Cl.x += ce.x + (ab.x * Bp.x - ab.y * Bp.y);
      Cl.y += ce.y + (ab.x * Bp.y + ab.y * Bp.x);
      El.x += ce.z;
      El.y += ce.w;
      if (s < sh.S) __stcg((float4 *)(sv + 4 + 8 * (int64_t)s), make_float4(Ap.x, Ap.y, Bp.x, Bp.y));
      cA.x += tA.x;
      cA.y += tA.y;
      cB.x += tB.x;
      cB.y += tB.y;
    }
    const float Cr = warp_sum(Cl.x), Ci = warp_sum(Cl.y);
    const float Er = warp_sum(El.x), Ei = warp_sum(El.y);
    if (lane == 0) {
      const float2 D = make_float2(phi12.x * Cr - phi12.y * Ci + (psi.x * Er - psi.y * Ei),
                                   phi12.x * Ci + phi12.y * Cr + (psi.x * Ei + psi.y * Er));
      Dout[row] = D;
      if (fout) fout[row] = fit_of(D);
      sv[0] = cA.x;
      sv[1] = cA.y;
    }
  }
}

// one warp per row.  Launched as a programmatic dependent of the forward: its CTAs
// are scheduled as the forward's retire and wait here until the forward's writes
// are visible.
static __global__ void k_relaxed_combine(RelaxShape sh, const float2 *__restrict__ konst,
                                         float *__restrict__ saved, float2 *__restrict__ Dout,
                                         float *__restrict__ fout) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row < sh.B) combine_rows(sh, konst, saved, Dout, fout, row, row + 1);
}

// grid (ceil(row groups / RX_WPC), S), block RX_WPC warps
template <bool TMA>
static __global__ void __launch_bounds__(RX_WPC * 32, 5)
    k_relaxed_fwd(const __grid_constant__ CUtensorMap tmap, const float *__restrict__ theta,
                  RelaxShape sh, const float4 *__restrict__ gtab, float *__restrict__ saved) {
  constexpr int NST = RX_NST_F;
  extern __shared__ unsigned char rx_raw[];
  Ph *ph;
  float4 *tiles;
  unsigned long long *bars;
  rx_carve<NST>(rx_raw, sh.L, ph, tiles, bars);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int seg = blockIdx.y, m0 = seg * sh.L;
  const int r0 = (blockIdx.x * RX_WPC + warp) * 32;
  float4 *wt = tiles + (size_t)warp * NST * (RX_TILE / 16);  // this warp's NST tiles
  const unsigned bar0 = smem_u32(bars + warp * NST);
  float4 R[TMA ? 1 : 8];
  if (r0 < sh.B) {  // the first step is in flight while the table is staged
    if constexpr (TMA) {
      if (lane == 0) {
        for (int k = 0; k < NST; ++k) mbar_init(bar0 + 8 * k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
        mbar_expect_tx(bar0, RX_TILE);
        tma_load_tile(wt, &tmap, m0, r0, bar0);
      }
    } else {
      load_step(theta, sh, r0, m0, R);
    }
  }
  stage_segment(ph, gtab, m0, sh.L, sh.N);
  if (r0 >= sh.B) return;
  Mono acc = mono_zero();
  float2 E = make_float2(0.f, 0.f);
  fwd_sweep<TMA>(&tmap, theta, sh, ph, wt, bar0, r0, m0, R, acc, E);
  const int row = r0 + lane;
  if (row < sh.B) {
    float4 *o = (float4 *)(saved + (int64_t)row * sh.sf + 4 + 8 * (int64_t)seg);
    o[0] = make_float4(acc.A.x, acc.A.y, acc.B.x, acc.B.y);
    o[1] = make_float4(acc.C.x, acc.C.y, E.x, E.y);
  }
}

// TMA_IN: theta tiles by TMA (else through registers); TMA_OUT: gradient tiles by
// TMA store where they lie wholly inside (else coalesced stores, 16-byte ones when
// VECG)
template <bool TMA_IN, bool TMA_OUT, bool VECG>
static __global__ void __launch_bounds__(RX_WPC * 32, 5)
    k_relaxed_bwd(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap gmap,
                  const float *__restrict__ theta, RelaxShape sh, const float4 *__restrict__ gtab,
                  const float2 *__restrict__ konst, const float2 *__restrict__ Din,
                  const float *__restrict__ saved, const float *__restrict__ gf,
                  float *__restrict__ grad, int64_t ldg) {
  constexpr int NST = RX_NST_B;
  extern __shared__ unsigned char rx_raw[];
  Ph *ph;
  float4 *tiles;
  unsigned long long *bars;
  rx_carve<NST>(rx_raw, sh.L, ph, tiles, bars);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int seg = blockIdx.y, m0 = seg * sh.L;
  const int r0 = (blockIdx.x * RX_WPC + warp) * 32;
  const int nsteps = sh.L / RX_STEP;
  float4 *wt = tiles + (size_t)warp * NST * (RX_TILE / 16);
  const unsigned bar0 = smem_u32(bars + warp * NST);
  float4 R4[TMA_IN ? 1 : 8];
  if (r0 < sh.B) {
    if constexpr (TMA_IN) {
      if (lane == 0) {
        for (int k = 0; k < NST; ++k) mbar_init(bar0 + 8 * k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
        mbar_expect_tx(bar0, RX_TILE);
        tma_load_tile(wt, &tmap, m0, r0, bar0);
      }
    } else {
      load_step(theta, sh, r0, m0, R4);
    }
  }
  stage_segment(ph, gtab, m0, sh.L, sh.N);
  if (r0 >= sh.B) return;
  const int row = r0 + lane;
  // u = 8 g conj(D) phi1 phi2, v = 16 g conj(D) psi: df/dtheta_k =
  //   [Re(u (p2 P + p1 R)) + d Re(v q)] r (1 - r)   with (1 - d^2) = 4 r (1 - r)
  float2 D = make_float2(0.f, 0.f), P = D, Rs = D;
  float g = 0.f;
  if (row < sh.B) {
    const float *sv = saved + (int64_t)row * sh.sf;
    D = Din[row];
    const float4 pre = *(const float4 *)(sv + 4 + 8 * (int64_t)seg);
    Rs = make_float2(sv[0] - pre.x, sv[1] - pre.y);  // sum of a from the segment start on
    P = make_float2(pre.z, pre.w);                  // sum of b before the segment
    g = gf ? gf[row] : 1.0f;
  }
  const float2 phi12 = konst[0], psi = konst[2];
  const float ur = 8.f * g * (D.x * phi12.x + D.y * phi12.y);
  const float ui = 8.f * g * (D.x * phi12.y - D.y * phi12.x);
  const float vr = 16.f * g * (D.x * psi.x + D.y * psi.y);
  const float vi = 16.f * g * (D.x * psi.y - D.y * psi.x);
  bool ok = true;
  int t_fail = -1;
  for (int t = 0; t < nsteps; ++t) {
    const int ms = m0 + t * RX_STEP;
    float4 *T = wt + (t % NST) * (RX_TILE / 16);
    if constexpr (TMA_IN) {
      if (lane == 0 && ok && t + 1 < nsteps) {
        // buffer (t + 1) % NST last held step t + 1 - NST, whose tile store must
        // have finished reading it (with two buffers that store left at the end
        // of the previous step: reading 4 KB of shared memory is soon done)
        const int b = (t + 1) % NST;
        if constexpr (TMA_OUT) tma_store_wait_read<NST - 2>();
        fence_async_smem();
        mbar_expect_tx(bar0 + 8 * b, RX_TILE);
        tma_load_tile(wt + b * (RX_TILE / 16), &tmap, ms + RX_STEP, r0, bar0 + 8 * b);
      }
      const bool arrived = ok && mbar_wait(bar0 + 8 * (t % NST), (t / NST) & 1);
      if (!__all_sync(0xffffffffu, arrived)) {  // ok is uniform across the warp
        if (ok) t_fail = t;
        ok = false;
        nan_tile(T);
      }
      __syncwarp();
    } else {
      // buffer t % NST last held step t - NST; later steps' stores may still read
      if constexpr (TMA_OUT) {
        if (lane == 0) tma_store_wait_read<NST - 1>();
      }
      __syncwarp();
      put_step(T, R4);
      __syncwarp();
      if (t + 1 < nsteps) load_step(theta, sh, r0, ms + RX_STEP, R4);
    }
    const Ph *pe = ph + t * RX_STEP;
#pragma unroll
    for (int c4 = 0; c4 < 8; ++c4) {
      const float4 x = T[tix(lane, c4)];
      const float th[4] = {x.x, x.y, x.z, x.w};
      float out[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float rc;
        const float d = tanh_r(th[j], rc);
        const float4 p = pe[4 * c4 + j].p;
        const float2 q = pe[4 * c4 + j].q;
        Rs.x = fmaf(-d, p.z, Rs.x);  // R_k: sum of a after this domain
        Rs.y = fmaf(-d, p.w, Rs.y);
        // w = p2 P + p1 R and the bracket, as chains of fused multiply-adds
        const float wr = fmaf(p.z, P.x, fmaf(-p.w, P.y, fmaf(p.x, Rs.x, -p.y * Rs.y)));
        const float wi = fmaf(p.z, P.y, fmaf(p.w, P.x, fmaf(p.x, Rs.y, p.y * Rs.x)));
        const float vq = fmaf(vr, q.x, -vi * q.y);
        const float s = fmaf(ur, wr, fmaf(-ui, wi, d * vq));
        out[j] = s * fmaf(-rc, rc, rc);
        P.x = fmaf(d, p.x, P.x);
        P.y = fmaf(d, p.y, P.y);
      }
      T[tix(lane, c4)] = make_float4(out[0], out[1], out[2], out[3]);
    }
    // a tile wholly inside the gradient leaves by TMA store; an edge tile (past the
    // last row or the row end) by plain stores, so that nothing past the rows' N
    // floats is written whatever the pitch
    if (TMA_OUT && ms + RX_STEP <= sh.N && r0 + 32 <= sh.B) {
      fence_async_smem();  // this lane's tile writes, before the async-proxy read
      __syncwarp();
      if (lane == 0) tma_store_tile(&gmap, ms, r0, T);
    } else {
      __syncwarp();
      // the step's gradient leaves through the tile with the load pattern
      const int m = ms + 4 * (lane & 7);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int tr = 4 * k + (lane >> 3), gr = r0 + tr;
        if (gr < sh.B) {
          const float4 v = T[tix(tr, lane & 7)];
          float *gp = grad + (int64_t)gr * ldg;
          if (VECG && m + 4 <= sh.N) {
            *(float4 *)(gp + m) = v;
          } else {
            if (m < sh.N) gp[m] = v.x;
            if (m + 1 < sh.N) gp[m + 1] = v.y;
            if (m + 2 < sh.N) gp[m + 2] = v.z;
            if (m + 3 < sh.N) gp[m + 3] = v.w;
          }
        }
      }
    }
    __syncwarp();  // every lane has read T before it is refilled
  }
  if constexpr (TMA_IN) {
    if (!ok) drain_loads(bar0, NST, t_fail, nsteps);
  }
  if constexpr (TMA_OUT) {
    if (lane == 0) tma_store_wait_all();
  }
}

// ---------------------------------------------------------------- host side
// the caller's lease stays alive until its launches are enqueued
static qpm_status relaxed_setup(const qpm_problem *prob, const float *theta, int64_t ld,
                                int32_t B, const void *saved, cudaStream_t s, TableLease &lease,
                                RelaxShape *sh, const float4 **tab, const float2 **konst) {
  if (!prob || !theta || !saved) return fail(QPM_ERR_ARG, "relaxed: NULL theta or saved block");
  if (prob->N < 1 || B < 1) return fail(QPM_ERR_ARG, "relaxed: need N >= 1 and B >= 1");
  if (ld < prob->N) return fail(QPM_ERR_ARG, "relaxed: leading dimension smaller than the row");
  if (((uintptr_t)saved & 15) != 0) return fail(QPM_ERR_ARG, "relaxed: saved block not 16-byte aligned");
  if (rx_nseg(prob->N) > 65535) return fail(QPM_ERR_ARG, "relaxed: N too large");
  qpm_status st = lease.table(prob, s, tab, konst);
  if (st != QPM_OK) return st;
  sh->B = B;
  sh->N = prob->N;
  sh->L = rx_seg_len(prob->N);
  sh->S = rx_nseg(prob->N);
  sh->ld = ld;
  sh->sf = rx_saved_floats(prob->N);
  return QPM_OK;
}

static dim3 rx_grid(const RelaxShape &sh) {
  const int groups = (sh.B + 31) / 32;
  return dim3((groups + RX_WPC - 1) / RX_WPC, sh.S);
}

// dynamic shared memory above the default 48 KB: the kernel's opt-in, set before each
// launch (a host-side attribute write) to what the longest segment needs, so that a
// launch with shorter segments never lowers it under one captured earlier
template <int NST, class K>
static qpm_status rx_launch_attr(K kernel) {
  QPM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)rx_smem_bytes<NST>(RX_LMAX)));
  return QPM_OK;
}

}  // namespace qpm

using namespace qpm;

extern "C" int64_t qpm_relaxed_saved_floats(int32_t N) { return N < 1 ? 0 : rx_saved_floats(N); }

extern "C" qpm_status qpm_deff_relaxed_fwd(const qpm_problem *prob, const float *theta, int64_t ld,
                                           int32_t B, float *d_eff, float *fit, float *saved,
                                           qpm_stream_t stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!d_eff) return fail(QPM_ERR_ARG, "qpm_deff_relaxed_fwd: NULL d_eff");
  if (!prob) return fail(QPM_ERR_ARG, "relaxed: NULL problem");
  TableLease lease(prob, 1);
  RelaxShape sh;
  const float4 *tab;
  const float2 *konst;
  qpm_status st = relaxed_setup(prob, theta, ld, B, saved, s, lease, &sh, &tab, &konst);
  if (st != QPM_OK) return st;
  float2 *D = (float2 *)d_eff;
  const dim3 grid = rx_grid(sh);
  CUtensorMap tmap{};
  const bool tma = make_tile_map(&tmap, theta, B, sh.N, ld);
  const size_t smem = rx_smem_bytes<RX_NST_F>(sh.L);
  if (tma) {
    if ((st = rx_launch_attr<RX_NST_F>(k_relaxed_fwd<true>)) != QPM_OK) return st;
    k_relaxed_fwd<true><<<grid, RX_WPC * 32, smem, s>>>(tmap, theta, sh, tab, saved);
  } else {
    if ((st = rx_launch_attr<RX_NST_F>(k_relaxed_fwd<false>)) != QPM_OK) return st;
    k_relaxed_fwd<false><<<grid, RX_WPC * 32, smem, s>>>(tmap, theta, sh, tab, saved);
  }
  QPM_CUDA(cudaGetLastError());
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((B + 7) / 8);
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  QPM_CUDA(cudaLaunchKernelEx(&cfg, k_relaxed_combine, sh, konst, saved, D, fit));
  return QPM_OK;
}

template <bool TI, bool TO, bool VG>
static qpm_status launch_bwd(dim3 grid, size_t smem, cudaStream_t s, const CUtensorMap &tmap,
                             const CUtensorMap &gmap, const float *theta, const RelaxShape &sh,
                             const float4 *tab, const float2 *konst, const float2 *D,
                             const float *saved, const float *gf, float *grad, int64_t ldg) {
  qpm_status st = rx_launch_attr<RX_NST_B>(k_relaxed_bwd<TI, TO, VG>);
  if (st != QPM_OK) return st;
  k_relaxed_bwd<TI, TO, VG><<<grid, RX_WPC * 32, smem, s>>>(tmap, gmap, theta, sh, tab, konst, D,
                                                            saved, gf, grad, ldg);
  QPM_CUDA(cudaGetLastError());
  return QPM_OK;
}

extern "C" qpm_status qpm_deff_relaxed_bwd(const qpm_problem *prob, const float *theta, int64_t ld,
                                           int32_t B, const float *d_eff, const float *saved,
                                           const float *grad_fit, float *grad_theta,
                                           int64_t ld_grad, qpm_stream_t stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!d_eff || !grad_theta)
    return fail(QPM_ERR_ARG, "qpm_deff_relaxed_bwd: NULL d_eff or grad_theta");
  if (!prob) return fail(QPM_ERR_ARG, "relaxed: NULL problem");
  if (ld_grad < prob->N)
    return fail(QPM_ERR_ARG, "qpm_deff_relaxed_bwd: gradient leading dimension smaller than the row");
  TableLease lease(prob, 1);
  RelaxShape sh;
  const float4 *tab;
  const float2 *konst;
  qpm_status st = relaxed_setup(prob, theta, ld, B, saved, s, lease, &sh, &tab, &konst);
  if (st != QPM_OK) return st;
  const bool vg = (ld_grad % 4 == 0) && (((uintptr_t)grad_theta & 15) == 0);
  const float2 *D = (const float2 *)d_eff;
  const dim3 grid = rx_grid(sh);
  CUtensorMap tmap{}, gmap{};
  const bool ti = make_tile_map(&tmap, theta, B, sh.N, ld);
  const bool to = make_tile_map(&gmap, grad_theta, B, sh.N, ld_grad);
  const size_t smem = rx_smem_bytes<RX_NST_B>(sh.L);
  if (ti && to)  // a TMA-ready gradient has 16-byte aligned rows: VECG for the edge tiles
    return launch_bwd<true, true, true>(grid, smem, s, tmap, gmap, theta, sh, tab, konst, D, saved,
                                        grad_fit, grad_theta, ld_grad);
  if (ti)
    return vg ? launch_bwd<true, false, true>(grid, smem, s, tmap, gmap, theta, sh, tab, konst, D,
                                              saved, grad_fit, grad_theta, ld_grad)
              : launch_bwd<true, false, false>(grid, smem, s, tmap, gmap, theta, sh, tab, konst, D,
                                               saved, grad_fit, grad_theta, ld_grad);
  if (to)
    return launch_bwd<false, true, true>(grid, smem, s, tmap, gmap, theta, sh, tab, konst, D, saved,
                                         grad_fit, grad_theta, ld_grad);
  return vg ? launch_bwd<false, false, true>(grid, smem, s, tmap, gmap, theta, sh, tab, konst, D,
                                             saved, grad_fit, grad_theta, ld_grad)
            : launch_bwd<false, false, false>(grid, smem, s, tmap, gmap, theta, sh, tab, konst, D,
                                              saved, grad_fit, grad_theta, ld_grad);
}
