// qpm_objectives.cu -- the other objectives of the paper's designs.
//
// SHG field (Sec. 2.1, the single integral before the cascade):
//   E2 prop. to int_0^L d(z) e^{-i dk z} dz = phi(kappa) sum_j d_j e^{-i kappa j},
// used by the multi-wavelength SHG designs of Sec. 5.  A plain complex sum per
// row: each CTA takes 8 rows, each thread 4-domain groups spaced by the CTA width
// (coalesced float4 loads), so one phasor read serves the 8 rows.
//
// Multi-wavelength objective (Sec. 5): f = sum_k |G0 - G_k| + beta (G_max - G_min)
// with G_k = |d_eff(kappa1_k, kappa2_k)|, to be minimised.  The K cascaded scans
// share one read of the genes: the row sweep of qpm_eval (qpm_rows.cuh) with the
// K sign-block tables streamed side by side, every block of 4 domains appended to K
// running monoids.  For K = 1 this is qpm_eval's arithmetic, operation for operation.
#include <math.h>

#include <algorithm>
#include <vector>

#include "qpm_common.cuh"
#include "qpm_internal.h"
#include "qpm_rows.cuh"

namespace qpm {

// ------------------------------------------------------------------ SHG field
static constexpr int SHG_ROWS = 8;
static constexpr int SHG_THREADS = 256;

template <bool VEC>
static __global__ void __launch_bounds__(SHG_THREADS)
    k_shg(const float *__restrict__ genes, int64_t ld, int NP, int N,
          const float4 *__restrict__ table, const float2 *__restrict__ konst,
          float2 *__restrict__ eout, float *__restrict__ fout) {
  __shared__ float2 red[SHG_THREADS / 32][SHG_ROWS];
  const int r0 = blockIdx.x * SHG_ROWS;
  float2 S[SHG_ROWS];
#pragma unroll
  for (int r = 0; r < SHG_ROWS; ++r) S[r] = make_float2(0.f, 0.f);
  for (int m = 4 * threadIdx.x; m < N; m += 4 * SHG_THREADS) {
    float2 p[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 t = m + q < N ? __ldg(table + m + q) : make_float4(0.f, 0.f, 0.f, 0.f);
      p[q] = make_float2(t.x, t.y);  // e^{-i kappa m}
    }
#pragma unroll
    for (int r = 0; r < SHG_ROWS; ++r) {
      if (r0 + r >= NP) break;
      const float *row = genes + (int64_t)(r0 + r) * ld;
      float x[4];
      if (VEC && m + 4 <= N) {
        const float4 v = __ldg((const float4 *)(row + m));
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = m + q < N ? __ldg(row + m + q) : 0.f;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float d = x[q] < 0.f ? -1.f : 1.f;
        S[r].x = fmaf(d, p[q].x, S[r].x);
        S[r].y = fmaf(d, p[q].y, S[r].y);
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < SHG_ROWS; ++r) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      S[r].x += __shfl_xor_sync(0xffffffffu, S[r].x, s);
      S[r].y += __shfl_xor_sync(0xffffffffu, S[r].y, s);
    }
    if (lane == 0) red[warp][r] = S[r];
  }
  __syncthreads();
  if (threadIdx.x < SHG_ROWS && r0 + (int)threadIdx.x < NP) {
    const int r = threadIdx.x;
    float2 t = red[0][r];
    for (int w = 1; w < SHG_THREADS / 32; ++w) {
      t.x += red[w][r].x;
      t.y += red[w][r].y;
    }
    const float2 ph = konst[3];  // phi(kappa)
    const float2 E = make_float2(ph.x * t.x - ph.y * t.y, ph.x * t.y + ph.y * t.x);
    eout[r0 + r] = E;
    if (fout) fout[r0 + r] = fit_of(E);
  }
}

// ------------------------------------------------- multi-wavelength objective
static constexpr int MW_KMAX = 4;

struct MultiTables {
  const float4 *t[MW_KMAX];  // sign-block tables (launch_block_table), read as float4
  const float2 *konst[MW_KMAX];
};

// The qpm_eval sweeps with K sign-block tables: the same segments and order for the
// same rows, so K = 1 reproduces qpm_eval's plain scan bit for bit.  Partials as for
// qpm_eval, one set per problem: part[((3k + comp) * S + s) * NPpad + i].
// grid (S, ceil(groups / ER_WPC)).

// 16-byte aligned rows: er_ring_sweep with K tables; K x 12 KB + 48 KB of shared memory
// per CTA (about 1 KB more with TMA tiles), so 3 CTAs per SM for K <= 2 and 2 for K = 3, 4
__host__ __device__ constexpr int mw_ring_ctas(int K) { return K <= 2 ? 3 : 2; }
// TMA: the gene tiles by TMA copies (er_ring_sweep_tma, `gmap`), else by cp.async
template <int K, bool TMA>
static __global__ void __launch_bounds__(ER_WPC * 32, mw_ring_ctas(K))
    k_multi_rows_ring(const __grid_constant__ CUtensorMap gmap, const float *__restrict__ genes,
                      int64_t ld, EvalShape sh, MultiTables mt, float2 *__restrict__ part) {
  extern __shared__ float4 dyn_raw[];
  float4 *dyn = dyn_raw;
  if constexpr (TMA)  // 1024-byte aligned for the swizzled tiles (the launch adds the slack)
    dyn = (float4 *)((unsigned char *)dyn_raw + ((1024 - (smem_u32(dyn_raw) & 1023)) & 1023));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int s = blockIdx.x, m0 = s * sh.L, m1 = min(sh.N, m0 + sh.L);
  const int r0 = (blockIdx.y * ER_WPC + warp) * 32;
  const bool live = r0 < sh.NP;
  Mono acc[K];
#pragma unroll
  for (int p = 0; p < K; ++p) acc[p] = mono_zero();
  auto push = [&](uint32_t e, const float2 *E, int b) {
#pragma unroll
    for (int p = 0; p < K; ++p) er_push_block(acc[p], e, E + (size_t)p * 2 * ER_STEP_F4_P + b * BLK_F2);
  };
  if constexpr (TMA) er_ring_sweep_tma<K>(dyn, &gmap, sh, mt.t, m0, m1, r0, live, push);
  else er_ring_sweep<K>(dyn, genes, ld, sh, mt.t, m0, m1, r0, live, push);
  if (!live) return;
  const size_t stride = (size_t)sh.S * sh.NPpad;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const size_t o = (size_t)(3 * k) * stride + (size_t)s * sh.NPpad + r0 + lane;
    part[o] = acc[k].A;
    part[o + stride] = acc[k].B;
    part[o + 2 * stride] = acc[k].C;
  }
}

// other rows: scalar gene loads one sub-step ahead in registers.  Dynamic shared
// memory: two steps of the K tables' entries, [2][K][ER_STEP_F4_P] float4.
template <int K>
static __global__ void __launch_bounds__(ER_WPC * 32)
    k_multi_rows(const float *__restrict__ genes, int64_t ld, EvalShape sh, MultiTables mt,
                 float2 *__restrict__ part) {
  extern __shared__ float4 tb[];
  __shared__ float4 tile[ER_WPC][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int s = blockIdx.x, m0 = s * sh.L, m1 = min(sh.N, m0 + sh.L);
  const int r0 = (blockIdx.y * ER_WPC + warp) * 32;
  const bool live = r0 < sh.NP;
  const int nb = (sh.N + 3) >> 2, nsteps = (m1 - m0 + 127) >> 7;
  float4 R[8];
  if (live) er_load_genes<false>(genes, ld, sh, r0, m0, R);
  // step k of problem p in buffer ((k & 1) * K + p); one commit group per step
#pragma unroll
  for (int p = 0; p < K; ++p) er_stage_step(tb + p * ER_STEP_F4_P, mt.t[p], m0, 0, nb);
  const float2 *bt = (const float2 *)tb;
  Mono acc[K];
#pragma unroll
  for (int p = 0; p < K; ++p) acc[p] = mono_zero();
  float4 *T = tile[warp];
  for (int k = 0; k < nsteps; ++k) {
    cp_async_wait<0>();
    __syncthreads();
    if (k + 1 < nsteps) {
#pragma unroll
      for (int p = 0; p < K; ++p)
        er_stage_step(tb + (((k + 1) & 1) * K + p) * ER_STEP_F4_P, mt.t[p], m0, k + 1, nb);
    }
    if (!live) continue;
    const float2 *bp = bt + (size_t)(k & 1) * K * 2 * ER_STEP_F4_P;
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      const int ms = m0 + 128 * k + 32 * q;
      if (ms >= m1) break;
      __syncwarp();
#pragma unroll
      for (int j = 0; j < 8; ++j) T[er_tix(4 * j + (lane >> 3), lane & 7)] = R[j];
      __syncwarp();
      if (ms + 32 < m1) er_load_genes<false>(genes, ld, sh, r0, ms + 32, R);
#pragma unroll 2
      for (int c4 = 0; c4 < 8; ++c4) {
        const uint32_t e = er_pattern(T[er_tix(lane, c4)]);
#pragma unroll
        for (int p = 0; p < K; ++p)
          er_push_block(acc[p], e, bp + (size_t)p * 2 * ER_STEP_F4_P + (8 * q + c4) * BLK_F2);
      }
    }
  }
  if (!live) return;
  const size_t stride = (size_t)sh.S * sh.NPpad;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const size_t o = (size_t)(3 * k) * stride + (size_t)s * sh.NPpad + r0 + lane;
    part[o] = acc[k].A;
    part[o + stride] = acc[k].B;
    part[o + 2 * stride] = acc[k].C;
  }
}

// one warp per row: the K combined scans (as in qpm_eval), then the objective
template <int K>
static __global__ void k_multi_combine(EvalShape sh, const float2 *__restrict__ part, MultiTables mt,
                                       float G0, float beta, float2 *__restrict__ deff,
                                       float *__restrict__ obj) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= sh.NP) return;
  const size_t set = (size_t)3 * sh.S * sh.NPpad;  // the partials of one problem
  float f = 0.f, gmax = -1.f, gmin = 3.0e38f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const Mono acc = combine_segments(part + k * set, sh.S, sh.NPpad, row);
    const float2 D = deff_from(acc, mt.konst[k][0], mt.konst[k][1]);
    if (deff && (threadIdx.x & 31) == 0) deff[(size_t)row * K + k] = D;
    const float G = sqrtf(fit_of(D));
    f += fabsf(G0 - G);
    gmax = fmaxf(gmax, G);
    gmin = fminf(gmin, G);
  }
  if ((threadIdx.x & 31) == 0) obj[row] = f + beta * (gmax - gmin);
}

}  // namespace qpm

using namespace qpm;

extern "C" qpm_status qpm_eval_shg(const qpm_problem *prob, const float *genes, int64_t ld,
                                   int32_t NP, float *e_shg, float *fit, qpm_stream_t stream) {
  if (!prob || !genes || !e_shg) return fail(QPM_ERR_ARG, "qpm_eval_shg: NULL pointer");
  if (prob->N < 1 || NP < 1) return fail(QPM_ERR_ARG, "qpm_eval_shg: need N >= 1 and NP >= 1");
  if (ld < prob->N) return fail(QPM_ERR_ARG, "qpm_eval_shg: leading dimension smaller than the row");
  cudaStream_t s = (cudaStream_t)stream;
  TableLease lease(prob, 1);  // held until the launch below is enqueued
  const float4 *table;
  const float2 *konst;
  qpm_status st = lease.table(prob, s, &table, &konst);
  if (st != QPM_OK) return st;
  const bool vec = (ld % 4 == 0) && (((uintptr_t)genes & 15) == 0);
  const int grid = (NP + SHG_ROWS - 1) / SHG_ROWS;
  if (vec)
    k_shg<true><<<grid, SHG_THREADS, 0, s>>>(genes, ld, NP, prob->N, table, konst, (float2 *)e_shg, fit);
  else
    k_shg<false><<<grid, SHG_THREADS, 0, s>>>(genes, ld, NP, prob->N, table, konst, (float2 *)e_shg, fit);
  QPM_CUDA(cudaGetLastError());
  return QPM_OK;
}

extern "C" qpm_status qpm_eval_multi(const qpm_problem *probs, int32_t K, const float *genes,
                                     int64_t ld, int32_t NP, float G0, float beta, float *d_eff,
                                     float *objective, void *scratch, size_t scratch_bytes,
                                     qpm_stream_t stream) {
  if (!probs || !genes || !objective) return fail(QPM_ERR_ARG, "qpm_eval_multi: NULL pointer");
  if (K < 1 || K > MW_KMAX) return fail(QPM_ERR_ARG, "qpm_eval_multi: need 1 <= K <= 4");
  const int N = probs[0].N;
  for (int k = 1; k < K; ++k)
    if (probs[k].N != N) return fail(QPM_ERR_ARG, "qpm_eval_multi: all problems need the same N");
  if (N < 1 || NP < 1) return fail(QPM_ERR_ARG, "qpm_eval_multi: need N >= 1 and NP >= 1");
  if (ld < N) return fail(QPM_ERR_ARG, "qpm_eval_multi: leading dimension smaller than the row");
  cudaStream_t s = (cudaStream_t)stream;
  MultiTables mt;
  for (int k = 0; k < MW_KMAX; ++k) {
    mt.t[k] = nullptr;
    mt.konst[k] = nullptr;
  }
  if (NP > ER_WPC * 32 * 65535) return fail(QPM_ERR_UNSUPPORTED, "qpm_eval_multi: too many rows");
  // one lease for all K lookups and the launches: room for the K tables is made
  // before the first lookup, so no lookup can evict a table returned before it
  TableLease lease(probs, K);
  for (int k = 0; k < K; ++k) {
    const float2 *blk;
    qpm_status st = lease.block_table(&probs[k], s, &blk, &mt.konst[k]);
    if (st != QPM_OK) return st;
    mt.t[k] = (const float4 *)blk;
  }
  const bool vec = (ld % 4 == 0) && (((uintptr_t)genes & 15) == 0);
  const EvalShape sh = eval_rows_shape(NP, N, vec ? ER_WPC * mw_ring_ctas(K) : 20);
  const size_t need = sizeof(float2) * 3 * (size_t)K * sh.S * sh.NPpad;
  if (!scratch || scratch_bytes < need)
    return fail(QPM_ERR_ARG, "qpm_eval_multi: scratch smaller than qpm_eval_multi_scratch_bytes()");
  float2 *part = (float2 *)scratch;
  const dim3 grid(sh.S, (sh.groups + ER_WPC - 1) / ER_WPC);
  CUtensorMap gmap{};
  const bool tma = vec && make_tile_map(&gmap, genes, NP, N, ld);
#define QPM_MW(KK)                                                                          \
  {                                                                                         \
    const void *fn = !vec ? (const void *)k_multi_rows<KK>                                  \
                     : tma ? (const void *)k_multi_rows_ring<KK, true>                     \
                           : (const void *)k_multi_rows_ring<KK, false>;                   \
    const size_t smem = !vec ? sizeof(float4) * 2 * (size_t)KK * ER_STEP_F4_P               \
                        : tma ? 1024 + er_ring_smem_tma(KK) : er_ring_smem(KK);             \
    QPM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    EvalShape shv = sh;                                                                     \
    int64_t ldv = ld;                                                                       \
    void *args_ring[] = {(void *)&gmap, (void *)&genes, &ldv, &shv, &mt, &part};           \
    void *args_rows[] = {(void *)&genes, &ldv, &shv, &mt, &part};                           \
    QPM_CUDA(cudaLaunchKernel(fn, grid, dim3(ER_WPC * 32), vec ? args_ring : args_rows, smem, s)); \
    k_multi_combine<KK><<<(NP + 7) / 8, 256, 0, s>>>(sh, part, mt, G0, beta,               \
                                                      (float2 *)d_eff, objective);          \
  }
  if (K == 1) QPM_MW(1) else if (K == 2) QPM_MW(2) else if (K == 3) QPM_MW(3) else QPM_MW(4)
#undef QPM_MW
  QPM_CUDA(cudaGetLastError());
  return QPM_OK;
}

// sized for the split of unaligned rows: fewer resident warps (the ring form of aligned
// rows) only lengthen the segments, so no split the call takes has more of them
extern "C" size_t qpm_eval_multi_scratch_bytes(int32_t K, int32_t N, int32_t NP) {
  if (K < 1 || N < 1 || NP < 1) return 0;
  const EvalShape sh = eval_rows_shape(NP, N, 20);
  return sizeof(float2) * 3 * (size_t)K * sh.S * sh.NPpad;
}
