// qpm_adjoint.cu -- relaxed d_eff and its hand-written adjoint.
//
// Relaxation: d_j = tanh(theta_j) in (-1, 1).  The closed form of the Sec. 2.1
// integral holds for any real piecewise-constant d:
//   D = phi1 phi2 sum_j a_j P_j + psi sum_j d_j^2 q_j,
//   a_j = d_j p2_j, b_j = d_j p1_j, P_j = sum_{m<j} b_m, q_j = p1_j p2_j,
// and f = |D|^2.  Its derivative with respect to d_k is
//   dD/dd_k = phi1 phi2 (p2_k P_k + p1_k R_k) + 2 psi d_k q_k,  R_k = sum_{j>k} a_j,
//   df/dtheta_k = 2 Re(conj(D) dD/dd_k) (1 - d_k^2).
// The forward pass keeps D and A = sum_j a_j per row; the backward pass
// recomputes d, sweeps the row once in index order and forms P_k as a running
// prefix and R_k = A - (prefix of a through k).
//
// Work split: one warp per row; the row is cut into tiles of 256 domains, lane l
// owns the 8 contiguous domains [8l, 8l+8) of every tile (two coalesced float4
// accesses per tile).  Because C = sum_j a_j P_j is bilinear, each lane keeps its
// own share of C, of A and of E across the whole row; only the prefix of b
// entering each lane's 8 domains needs a warp exclusive scan per tile, and the
// shares are summed once per row.  The phasor table (p1, p2) is staged once per
// CTA in shared memory in a [tile][e][lane] layout, which makes every table read
// conflict-free; the next tile's theta is requested before the current one is
// processed, so one tile of loads is always in flight per warp.
#include <math.h>

#include <algorithm>

#include "qpm_common.cuh"
#include "qpm_internal.h"

namespace qpm {

static constexpr int RX_WARPS = 8;
static constexpr int RX_TILE = 256;
static constexpr size_t RX_SMEM_MAX = 192 * 1024;

struct RelaxShape {
  int B, N, ntiles;
  int64_t ld;
  bool vec;  // 16-byte aligned rows with ld % 4 == 0
};

// table entry of (tile, lane, e) in the staged layout
__device__ __forceinline__ const float4 &tab(const float4 *sm, int tile, int e, int lane) {
  return sm[((size_t)tile * 8 + e) * 32 + lane];
}

template <bool SMT>
__device__ __forceinline__ float4 tab_get(const float4 *sm, const float4 *gtab, int tile, int e,
                                          int lane, int m, int N) {
  if (SMT) return tab(sm, tile, e, lane);
  return m < N ? __ldg(gtab + m) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// the 8 values of lane `lane` in tile `tile` of a row (0 beyond N)
template <bool VEC>
__device__ __forceinline__ void load8(const float *row, int m0, int N, float v[8]) {
  if (VEC && m0 + 8 <= N) {
    const float4 x = __ldg((const float4 *)(row + m0));
    const float4 y = __ldg((const float4 *)(row + m0 + 4));
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = (m0 + e < N) ? __ldg(row + m0 + e) : 0.f;
  }
}

template <bool VEC>
__device__ __forceinline__ void store8(float *row, int m0, int N, const float v[8]) {
  if (VEC && m0 + 8 <= N) {
    *(float4 *)(row + m0) = make_float4(v[0], v[1], v[2], v[3]);
    *(float4 *)(row + m0 + 4) = make_float4(v[4], v[5], v[6], v[7]);
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e)
      if (m0 + e < N) row[m0 + e] = v[e];
  }
}

// stage the natural-order table into shared memory ([tile][e][lane], zero padded);
// consecutive threads write consecutive shared-memory slots
__device__ void stage_table(float4 *sm, const float4 *gtab, int N, int ntiles) {
  for (int o = threadIdx.x; o < ntiles * RX_TILE; o += blockDim.x) {
    const int tile = o / RX_TILE, rem = o - tile * RX_TILE, e = rem >> 5, lane = rem & 31;
    const int m = tile * RX_TILE + lane * 8 + e;
    sm[o] = m < N ? __ldg(gtab + m) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
}

__device__ __forceinline__ float2 q_of(const float4 &p) {  // q = p1 p2
  return make_float2(p.x * p.z - p.y * p.w, p.x * p.w + p.y * p.z);
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

// this warp's work list: rows r = gw, gw + nw, ...; (row, tile) pairs in order.
// next() advances and prefetches the theta of the following pair.
template <bool VEC>
struct RowWalker {
  const float *theta;
  int64_t ld;
  int N, B, ntiles, nw;
  int r, tile;
  float nxt[8];
  __device__ __forceinline__ void fetch(int rr, int tt) {
    if (rr < B) load8<VEC>(theta + (int64_t)rr * ld, tt * RX_TILE + (threadIdx.x & 31) * 8, N, nxt);
  }
  __device__ __forceinline__ void start(int gw) {
    r = gw;
    tile = 0;
    fetch(r, 0);
  }
  // copies the prefetched values of (r, tile) into v and requests the next pair
  __device__ __forceinline__ void take(float v[8]) {
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = nxt[e];
    const int nt = tile + 1 < ntiles ? tile + 1 : 0;
    const int nr = tile + 1 < ntiles ? r : r + nw;
    fetch(nr, nt);
  }
  __device__ __forceinline__ bool advance() {  // true when a new row starts
    if (++tile < ntiles) return false;
    tile = 0;
    r += nw;
    return true;
  }
};

template <bool VEC, bool SMT>
static __global__ void __launch_bounds__(RX_WARPS * 32)
    k_relaxed_fwd(const float *__restrict__ theta, RelaxShape sh, const float4 *__restrict__ gtab,
                  const float2 *__restrict__ konst, float2 *__restrict__ Dout,
                  float *__restrict__ fout, float2 *__restrict__ Aout) {
  extern __shared__ float4 smt[];
  if (SMT) stage_table(smt, gtab, sh.N, sh.ntiles);
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nw = gridDim.x * (blockDim.x >> 5);
  const float2 phi12 = konst[0], psi = konst[2];
  RowWalker<VEC> w{theta, sh.ld, sh.N, sh.B, sh.ntiles, nw, 0, 0, {}};
  w.start(gw);
  while (w.r < sh.B) {
    const int r = w.r;
    float2 Cl = make_float2(0.f, 0.f), Al = Cl, El = Cl;  // this lane's shares
    float2 Brun = make_float2(0.f, 0.f);                   // sum of b before this tile
    bool row_done = false;
    while (!row_done) {
      const int tile = w.tile;
      const int m0 = tile * RX_TILE + lane * 8;
      float th[8];
      w.take(th);
      Mono loc = mono_zero();
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float d = tanhf(th[e]);
        const float4 p = tab_get<SMT>(smt, gtab, tile, e, lane, m0 + e, sh.N);
        mono_push(loc, d, p);
        const float2 q = q_of(p);
        const float d2 = d * d;
        El.x = fmaf(d2, q.x, El.x);
        El.y = fmaf(d2, q.y, El.y);
      }
      float2 Bt;
      const float2 Bex = warp_excl_scan2(loc.B, Bt);
      // C share: the lane's own pairs plus its a-sum times every b before the lane
      const float br = Brun.x + Bex.x, bi = Brun.y + Bex.y;
      Cl.x += loc.C.x + (loc.A.x * br - loc.A.y * bi);
      Cl.y += loc.C.y + (loc.A.x * bi + loc.A.y * br);
      Al.x += loc.A.x;
      Al.y += loc.A.y;
      Brun.x += Bt.x;
      Brun.y += Bt.y;
      row_done = w.advance();
    }
    const float Cr = warp_sum(Cl.x), Ci = warp_sum(Cl.y);
    const float Er = warp_sum(El.x), Ei = warp_sum(El.y);
    const float Ar = warp_sum(Al.x), Ai = warp_sum(Al.y);
    if (lane == 0) {
      const float2 D = make_float2(phi12.x * Cr - phi12.y * Ci + (psi.x * Er - psi.y * Ei),
                                   phi12.x * Ci + phi12.y * Cr + (psi.x * Ei + psi.y * Er));
      Dout[r] = D;
      if (fout) fout[r] = fit_of(D);
      if (Aout) Aout[r] = make_float2(Ar, Ai);
    }
  }
}

template <bool VEC, bool SMT>
static __global__ void __launch_bounds__(RX_WARPS * 32)
    k_relaxed_bwd(const float *__restrict__ theta, RelaxShape sh, const float4 *__restrict__ gtab,
                  const float2 *__restrict__ konst, const float2 *__restrict__ Din,
                  const float2 *__restrict__ Ain, const float *__restrict__ gf,
                  float *__restrict__ grad, int64_t ldg) {
  extern __shared__ float4 smt[];
  if (SMT) stage_table(smt, gtab, sh.N, sh.ntiles);
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nw = gridDim.x * (blockDim.x >> 5);
  const float2 phi12 = konst[0], psi = konst[2];
  RowWalker<VEC> wk{theta, sh.ld, sh.N, sh.B, sh.ntiles, nw, 0, 0, {}};
  wk.start(gw);
  while (wk.r < sh.B) {
    const int r = wk.r;
    float *grow = grad + (int64_t)r * ldg;
    const float2 D = Din[r];
    const float2 Atot = Ain[r];
    const float g = gf ? gf[r] : 1.0f;
    // u = 2 g conj(D) phi1 phi2, v = 4 g conj(D) psi: df/dtheta_k =
    //   [Re(u (p2 P + p1 R)) + d Re(v q)] (1 - d^2)
    const float ur = 2.f * g * (D.x * phi12.x + D.y * phi12.y);
    const float ui = 2.f * g * (D.x * phi12.y - D.y * phi12.x);
    const float vr = 4.f * g * (D.x * psi.x + D.y * psi.y);
    const float vi = 4.f * g * (D.x * psi.y - D.y * psi.x);
    float2 Brun = make_float2(0.f, 0.f), Arun = make_float2(0.f, 0.f);
    bool row_done = false;
    while (!row_done) {
      const int tile = wk.tile;
      const int m0 = tile * RX_TILE + lane * 8;
      float th[8], d[8];
      wk.take(th);
      float2 la = make_float2(0.f, 0.f), lb = make_float2(0.f, 0.f);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        d[e] = tanhf(th[e]);
        const float4 p = tab_get<SMT>(smt, gtab, tile, e, lane, m0 + e, sh.N);
        la.x = fmaf(d[e], p.z, la.x);
        la.y = fmaf(d[e], p.w, la.y);
        lb.x = fmaf(d[e], p.x, lb.x);
        lb.y = fmaf(d[e], p.y, lb.y);
      }
      float2 ta, tb;
      const float2 ea = warp_excl_scan2(la, ta), eb = warp_excl_scan2(lb, tb);
      float2 P = make_float2(Brun.x + eb.x, Brun.y + eb.y);   // sum of b before this lane
      float2 Ap = make_float2(Arun.x + ea.x, Arun.y + ea.y);  // sum of a before this lane
      float out[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float4 p = tab_get<SMT>(smt, gtab, tile, e, lane, m0 + e, sh.N);
        Ap.x = fmaf(d[e], p.z, Ap.x);
        Ap.y = fmaf(d[e], p.w, Ap.y);
        const float Rr = Atot.x - Ap.x, Ri = Atot.y - Ap.y;  // sum of a after this domain
        // w = p2 P + p1 R
        const float wr = p.z * P.x - p.w * P.y + (p.x * Rr - p.y * Ri);
        const float wi = p.z * P.y + p.w * P.x + (p.x * Ri + p.y * Rr);
        const float2 q = q_of(p);
        const float sv = (ur * wr - ui * wi) + d[e] * (vr * q.x - vi * q.y);
        out[e] = sv * (1.f - d[e] * d[e]);
        P.x = fmaf(d[e], p.x, P.x);
        P.y = fmaf(d[e], p.y, P.y);
      }
      store8<VEC>(grow, m0, sh.N, out);
      Brun.x += tb.x;
      Brun.y += tb.y;
      Arun.x += ta.x;
      Arun.y += ta.y;
      row_done = wk.advance();
    }
  }
}

static qpm_status relaxed_setup(const qpm_problem *prob, const float *theta, int64_t ld,
                                int32_t B, cudaStream_t s, RelaxShape *sh, const float4 **tab,
                                const float2 **konst, size_t *smem, int *grid) {
  if (!prob || !theta) return fail(QPM_ERR_ARG, "relaxed: NULL pointer");
  if (prob->N < 1 || B < 1) return fail(QPM_ERR_ARG, "relaxed: need N >= 1 and B >= 1");
  if (ld < prob->N) return fail(QPM_ERR_ARG, "relaxed: leading dimension smaller than the row");
  qpm_status st = cached_table(prob, s, tab, konst);
  if (st != QPM_OK) return st;
  sh->B = B;
  sh->N = prob->N;
  sh->ntiles = (prob->N + RX_TILE - 1) / RX_TILE;
  sh->ld = ld;
  sh->vec = (ld % 4 == 0) && (((uintptr_t)theta & 15) == 0);
  const size_t need = sizeof(float4) * (size_t)sh->ntiles * RX_TILE;
  *smem = need <= RX_SMEM_MAX ? need : 0;
  const int per_sm = *smem ? (int)std::max<size_t>(1, (228 * 1024) / (*smem + 1024)) : 4;
  *grid = sm_count() * std::min(per_sm, 4);
  const int rows_per_cta = RX_WARPS;
  *grid = std::max(1, std::min(*grid, (B + rows_per_cta - 1) / rows_per_cta));
  return QPM_OK;
}

}  // namespace qpm

using namespace qpm;

#define QPM_RX_DISPATCH(KERNEL, ...)                                                       \
  do {                                                                                     \
    const void *fn;                                                                        \
    if (sh.vec) fn = smem ? (const void *)KERNEL<true, true> : (const void *)KERNEL<true, false>; \
    else fn = smem ? (const void *)KERNEL<false, true> : (const void *)KERNEL<false, false>;      \
    if (smem) QPM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                            (int)RX_SMEM_MAX));                            \
    void *args[] = {__VA_ARGS__};                                                          \
    QPM_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(RX_WARPS * 32), args, smem, s));         \
  } while (0)

extern "C" qpm_status qpm_deff_relaxed_fwd(const qpm_problem *prob, const float *theta, int64_t ld,
                                           int32_t B, float *d_eff, float *fit, float *sum_a,
                                           qpm_stream_t stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!d_eff) return fail(QPM_ERR_ARG, "qpm_deff_relaxed_fwd: NULL d_eff");
  RelaxShape sh;
  const float4 *tab;
  const float2 *konst;
  size_t smem;
  int grid;
  qpm_status st = relaxed_setup(prob, theta, ld, B, s, &sh, &tab, &konst, &smem, &grid);
  if (st != QPM_OK) return st;
  float2 *D = (float2 *)d_eff, *A = (float2 *)sum_a;
  QPM_RX_DISPATCH(k_relaxed_fwd, (void *)&theta, &sh, &tab, &konst, &D, &fit, &A);
  return QPM_OK;
}

extern "C" qpm_status qpm_deff_relaxed_bwd(const qpm_problem *prob, const float *theta, int64_t ld,
                                           int32_t B, const float *d_eff, const float *sum_a,
                                           const float *grad_fit, float *grad_theta,
                                           int64_t ld_grad, qpm_stream_t stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!d_eff || !sum_a || !grad_theta)
    return fail(QPM_ERR_ARG, "qpm_deff_relaxed_bwd: NULL d_eff, sum_a or grad_theta");
  if (!prob || ld_grad < prob->N)
    return fail(QPM_ERR_ARG, "qpm_deff_relaxed_bwd: gradient leading dimension smaller than the row");
  RelaxShape sh;
  const float4 *tab;
  const float2 *konst;
  size_t smem;
  int grid;
  qpm_status st = relaxed_setup(prob, theta, ld, B, s, &sh, &tab, &konst, &smem, &grid);
  if (st != QPM_OK) return st;
  if (sh.vec && (ld_grad % 4 != 0 || ((uintptr_t)grad_theta & 15) != 0)) sh.vec = false;
  const float2 *D = (const float2 *)d_eff, *A = (const float2 *)sum_a;
  QPM_RX_DISPATCH(k_relaxed_bwd, (void *)&theta, &sh, &tab, &konst, (void *)&D, (void *)&A,
                  (void *)&grad_fit, &grad_theta, &ld_grad);
  return QPM_OK;
}
