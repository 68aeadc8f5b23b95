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
// segment in index order in steps of 32 domains.  Each step's 32 x 32 theta
// values arrive one step ahead as coalesced 16-byte asynchronous copies
// (cp.async, zero-filled past the row ends) straight into a double-buffered
// per-warp shared-memory tile, transposed by its swizzle, so no registers hold
// the prefetch (rows that are not 16-byte aligned use register loads instead);
// every lane then walks its own row:
// the running prefixes of a and b are plain sequential sums and every phasor
// read is a broadcast.  The warps of a CTA take consecutive row groups of the
// same segment and share its staged phasors (p1, p2, q = p1 p2).
//
// Forward: every (row, segment) writes its partial sums (A_s, B_s, C_s, E_s) into
// the row's saved block; a second kernel (a warp per row, lanes over segments)
// combines the segments in index order (C = sum_s C_s + A_s Bpre_s with Bpre_s
// the b-sum of the segments before s), closes D and overwrites each segment's
// (A_s, B_s) with the exclusive prefixes (Apre_s, Bpre_s).
// Backward: each (row, segment) starts from those prefixes (P = Bpre_s,
// R = A - Apre_s), updates P_k and R_k as it goes and writes the gradient back
// through the same tile with coalesced stores.
#include <math.h>

#include <algorithm>

#include "qpm_common.cuh"
#include "qpm_internal.h"

namespace qpm {

static constexpr int RX_STEP = 32;   // domains per step (one per lane of a tile row)
static constexpr int RX_LMAX = 256;  // longest segment
static constexpr int RX_WPC = 4;     // warps (row groups of 32) per CTA

struct RelaxShape {
  int B, N, L, S;  // rows, domains, segment length, segments
  int64_t ld;      // theta leading dimension
  int64_t sf;      // floats per row of the saved block
  bool vec;        // theta rows 16-byte aligned with ld % 4 == 0
};

// segment length: S = ceil(N / L) is about 32 for short rows, L = 256 for long ones
// (4096 x 4096: 32 segments of 128 domains, 4096 warps of work)
static constexpr int RX_SEGQ = 1024;  // about N / 32, rounded up to whole steps
static int rx_seg_len(int N) { return std::min(RX_LMAX, RX_STEP * ((N + RX_SEGQ - 1) / RX_SEGQ)); }
static int rx_nseg(int N) { return (N + rx_seg_len(N) - 1) / rx_seg_len(N); }
// saved block of a row: [A (2 floats), 2 unused, then per segment 8 floats]
static int64_t rx_saved_floats(int N) { return 4 + 8 * (int64_t)rx_nseg(N); }

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

__device__ __forceinline__ float2 q_of(const float4 &p) {  // q = p1 p2
  return make_float2(p.x * p.z - p.y * p.w, p.x * p.w + p.y * p.z);
}

// The per-warp tile holds 32 rows x 32 domains as float4 [row][c4], the column
// xor-swizzled by the row: 8 columns of one row (a quarter-warp of the staging
// stores) and 8 rows of one column (a quarter-warp of the row walks) both fall
// into 8 different 16-byte bank groups.
__device__ __forceinline__ int tix(int row, int c4) { return row * 8 + (c4 ^ (row & 7)); }

// Step registers: lane l holds float4 k * 32 + l of the 32 x 8 float4 step,
// i.e. row 4k + l / 8, column l % 8 (4 rows x 128 contiguous bytes per load).
template <bool VEC>
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
      if (VEC && m + 4 <= sh.N) {
        v = __ldg((const float4 *)(rp + m));
      } else {
        if (m < sh.N) v.x = __ldg(rp + m);
        if (m + 1 < sh.N) v.y = __ldg(rp + m + 1);
        if (m + 2 < sh.N) v.z = __ldg(rp + m + 2);
        if (m + 3 < sh.N) v.w = __ldg(rp + m + 3);
      }
    }
    R[k] = v;
  }
}

__device__ __forceinline__ void put_step(float4 *T, const float4 R[8]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 8; ++k) T[tix(4 * k + (lane >> 3), lane & 7)] = R[k];
}

// one step (32 domains from ms) of rows r0..r0+31 copied asynchronously into the
// tile T with the layout of put_step; 16-byte aligned rows (ld % 4 == 0) only
__device__ __forceinline__ void copy_step(float4 *T, const float *__restrict__ theta,
                                          const RelaxShape &sh, int r0, int ms) {
  const int lane = threadIdx.x & 31;
  const int m = ms + 4 * (lane & 7);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int tr = 4 * k + (lane >> 3), gr = r0 + tr;
    const float *src = theta;
    int bytes = 0;
    if (gr < sh.B && m < sh.N) {
      src = theta + (int64_t)gr * sh.ld + m;
      bytes = 4 * min(4, sh.N - m);
    }
    cp_async16(&T[tix(tr, lane & 7)], src, bytes);
  }
  cp_async_commit();
}

// phasors of the CTA's segment [m0, m0 + L) (zero beyond N), then a CTA barrier
__device__ __forceinline__ void stage_segment(float4 *sp, float2 *sq, const float4 *gtab, int m0,
                                              int L, int N) {
  for (int i = threadIdx.x; i < L; i += blockDim.x) {
    const int m = m0 + i;
    const float4 p = m < N ? __ldg(gtab + m) : make_float4(0.f, 0.f, 0.f, 0.f);
    sp[i] = p;
    sq[i] = q_of(p);
  }
  __syncthreads();
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

// grid (ceil(row groups / RX_WPC), S), block RX_WPC warps
template <bool VEC>
static __global__ void __launch_bounds__(RX_WPC * 32)
    k_relaxed_fwd(const float *__restrict__ theta, RelaxShape sh, const float4 *__restrict__ gtab,
                  float *__restrict__ saved) {
  __shared__ float4 sp[RX_LMAX];
  __shared__ float2 sq[RX_LMAX];
  __shared__ float4 tile[RX_WPC][2][RX_STEP * RX_STEP / 4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int seg = blockIdx.y, m0 = seg * sh.L;
  const int r0 = (blockIdx.x * RX_WPC + warp) * 32;
  const int nsteps = sh.L / RX_STEP;
  float4 R[VEC ? 1 : 8];
  if (r0 < sh.B) {  // the first step is in flight while the table is staged
    if constexpr (VEC) copy_step(tile[warp][0], theta, sh, r0, m0);
    else load_step<false>(theta, sh, r0, m0, R);
  }
  stage_segment(sp, sq, gtab, m0, sh.L, sh.N);
  if (r0 >= sh.B) return;
  Mono acc = mono_zero();
  float2 E = make_float2(0.f, 0.f);
  for (int t = 0; t < nsteps; ++t) {
    float4 *T = tile[warp][t & 1];
    if constexpr (VEC) {
      if (t + 1 < nsteps) {
        copy_step(tile[warp][(t + 1) & 1], theta, sh, r0, m0 + (t + 1) * RX_STEP);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncwarp();
    } else {
      __syncwarp();
      put_step(T, R);
      __syncwarp();
      if (t + 1 < nsteps) load_step<false>(theta, sh, r0, m0 + (t + 1) * RX_STEP, R);
    }
    const int e0 = t * RX_STEP;
#pragma unroll
    for (int c4 = 0; c4 < 8; ++c4) {
      const float4 x = T[tix(lane, c4)];
      const float th[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float rc;
        const float d = tanh_r(th[j], rc);
        const int e = e0 + 4 * c4 + j;
        const float4 p = sp[e];
        const float2 q = sq[e];
        mono_push(acc, d, p);
        const float d2 = d * d;
        E.x = fmaf(d2, q.x, E.x);
        E.y = fmaf(d2, q.y, E.y);
      }
    }
    __syncwarp();  // every lane has read T before the copy two steps on refills it
  }
  const int row = r0 + lane;
  if (row < sh.B) {
    float4 *o = (float4 *)(saved + (int64_t)row * sh.sf + 4 + 8 * (int64_t)seg);
    o[0] = make_float4(acc.A.x, acc.A.y, acc.B.x, acc.B.y);
    o[1] = make_float4(acc.C.x, acc.C.y, E.x, E.y);
  }
}

// one warp per row: segments in index order -> D, f, A; (A_s, B_s) -> prefixes
static __global__ void k_relaxed_combine(RelaxShape sh, const float2 *__restrict__ konst,
                                         float *__restrict__ saved, float2 *__restrict__ Dout,
                                         float *__restrict__ fout) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= sh.B) return;
  float *sv = saved + (int64_t)row * sh.sf;
  float2 cA = make_float2(0.f, 0.f), cB = cA, Cl = cA, El = cA;
  for (int c = 0; c < sh.S; c += 32) {
    const int s = c + lane;
    float4 ab = make_float4(0.f, 0.f, 0.f, 0.f), ce = ab;
    if (s < sh.S) {
      const float4 *in = (const float4 *)(sv + 4 + 8 * (int64_t)s);
      ab = in[0];
      ce = in[1];
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
    if (s < sh.S) *(float4 *)(sv + 4 + 8 * (int64_t)s) = make_float4(Ap.x, Ap.y, Bp.x, Bp.y);
    cA.x += tA.x;
    cA.y += tA.y;
    cB.x += tB.x;
    cB.y += tB.y;
  }
  const float Cr = warp_sum(Cl.x), Ci = warp_sum(Cl.y);
  const float Er = warp_sum(El.x), Ei = warp_sum(El.y);
  if (lane == 0) {
    const float2 phi12 = konst[0], psi = konst[2];
    const float2 D = make_float2(phi12.x * Cr - phi12.y * Ci + (psi.x * Er - psi.y * Ei),
                                 phi12.x * Ci + phi12.y * Cr + (psi.x * Ei + psi.y * Er));
    Dout[row] = D;
    if (fout) fout[row] = fit_of(D);
    sv[0] = cA.x;
    sv[1] = cA.y;
  }
}

template <bool VEC, bool VECG>
static __global__ void __launch_bounds__(RX_WPC * 32)
    k_relaxed_bwd(const float *__restrict__ theta, RelaxShape sh, const float4 *__restrict__ gtab,
                  const float2 *__restrict__ konst, const float2 *__restrict__ Din,
                  const float *__restrict__ saved, const float *__restrict__ gf,
                  float *__restrict__ grad, int64_t ldg) {
  __shared__ float4 sp[RX_LMAX];
  __shared__ float2 sq[RX_LMAX];
  __shared__ float4 tile[RX_WPC][2][RX_STEP * RX_STEP / 4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int seg = blockIdx.y, m0 = seg * sh.L;
  const int r0 = (blockIdx.x * RX_WPC + warp) * 32;
  const int nsteps = sh.L / RX_STEP;
  float4 R[VEC ? 1 : 8];
  if (r0 < sh.B) {
    if constexpr (VEC) copy_step(tile[warp][0], theta, sh, r0, m0);
    else load_step<false>(theta, sh, r0, m0, R);
  }
  stage_segment(sp, sq, gtab, m0, sh.L, sh.N);
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
  for (int t = 0; t < nsteps; ++t) {
    const int ms = m0 + t * RX_STEP;
    float4 *T = tile[warp][t & 1];
    if constexpr (VEC) {
      if (t + 1 < nsteps) {
        copy_step(tile[warp][(t + 1) & 1], theta, sh, r0, ms + RX_STEP);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncwarp();
    } else {
      __syncwarp();
      put_step(T, R);
      __syncwarp();
      if (t + 1 < nsteps) load_step<false>(theta, sh, r0, ms + RX_STEP, R);
    }
    const int e0 = t * RX_STEP;
#pragma unroll
    for (int c4 = 0; c4 < 8; ++c4) {
      const float4 x = T[tix(lane, c4)];
      const float th[4] = {x.x, x.y, x.z, x.w};
      float out[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float rc;
        const float d = tanh_r(th[j], rc);
        const int e = e0 + 4 * c4 + j;
        const float4 p = sp[e];
        const float2 q = sq[e];
        Rs.x = fmaf(-d, p.z, Rs.x);  // R_k: sum of a after this domain
        Rs.y = fmaf(-d, p.w, Rs.y);
        // w = p2 P + p1 R
        const float wr = p.z * P.x - p.w * P.y + (p.x * Rs.x - p.y * Rs.y);
        const float wi = p.z * P.y + p.w * P.x + (p.x * Rs.y + p.y * Rs.x);
        const float s = (ur * wr - ui * wi) + d * (vr * q.x - vi * q.y);
        out[j] = s * fmaf(-rc, rc, rc);
        P.x = fmaf(d, p.x, P.x);
        P.y = fmaf(d, p.y, P.y);
      }
      T[tix(lane, c4)] = make_float4(out[0], out[1], out[2], out[3]);
    }
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
    __syncwarp();  // every lane has read T before the copy two steps on refills it
  }
}

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
  sh->vec = (ld % 4 == 0) && (((uintptr_t)theta & 15) == 0);
  return QPM_OK;
}

static dim3 rx_grid(const RelaxShape &sh) {
  const int groups = (sh.B + 31) / 32;
  return dim3((groups + RX_WPC - 1) / RX_WPC, sh.S);
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
  if (sh.vec)
    k_relaxed_fwd<true><<<grid, RX_WPC * 32, 0, s>>>(theta, sh, tab, saved);
  else
    k_relaxed_fwd<false><<<grid, RX_WPC * 32, 0, s>>>(theta, sh, tab, saved);
  QPM_CUDA(cudaGetLastError());
  k_relaxed_combine<<<(B + 7) / 8, 256, 0, s>>>(sh, konst, saved, D, fit);
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
  if (!prob || ld_grad < prob->N)
    return fail(QPM_ERR_ARG, "qpm_deff_relaxed_bwd: gradient leading dimension smaller than the row");
  if (!prob) return fail(QPM_ERR_ARG, "relaxed: NULL problem");
  TableLease lease(prob, 1);
  RelaxShape sh;
  const float4 *tab;
  const float2 *konst;
  qpm_status st = relaxed_setup(prob, theta, ld, B, saved, s, lease, &sh, &tab, &konst);
  if (st != QPM_OK) return st;
  const bool vg = (ld_grad % 4 == 0) && (((uintptr_t)grad_theta & 15) == 0);
  const float2 *D = (const float2 *)d_eff;
  const dim3 grid = rx_grid(sh);
  if (sh.vec && vg)
    k_relaxed_bwd<true, true><<<grid, RX_WPC * 32, 0, s>>>(theta, sh, tab, konst, D, saved, grad_fit,
                                                           grad_theta, ld_grad);
  else if (sh.vec)
    k_relaxed_bwd<true, false><<<grid, RX_WPC * 32, 0, s>>>(theta, sh, tab, konst, D, saved,
                                                            grad_fit, grad_theta, ld_grad);
  else if (vg)
    k_relaxed_bwd<false, true><<<grid, RX_WPC * 32, 0, s>>>(theta, sh, tab, konst, D, saved,
                                                            grad_fit, grad_theta, ld_grad);
  else
    k_relaxed_bwd<false, false><<<grid, RX_WPC * 32, 0, s>>>(theta, sh, tab, konst, D, saved,
                                                             grad_fit, grad_theta, ld_grad);
  QPM_CUDA(cudaGetLastError());
  return QPM_OK;
}
