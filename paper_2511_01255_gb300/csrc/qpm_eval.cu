// qpm_eval.cu -- fitness of caller-supplied sign sequences (Sec. 2.1).
//
// Work split: a warp takes 32 rows (lane = row) and one segment of L domains (L a
// multiple of 128) and sweeps it in index order, so every row's running monoid
// (A, B, C) is a plain sequential accumulation.  The sweep appends a block of 4
// domains per lookup in the sign-block table (the block's monoid triple for its sign
// pattern, precomputed in FP64), whose entries are streamed into shared memory per
// step of 128 domains, the next step's with cp.async while this one is swept.
// Float genes arrive 32 domains at a time and are transposed through per-warp
// shared-memory tiles: rows that are 16-byte aligned through a ring of ER_RING tiles
// filled by cp.async ER_RING - 1 sub-steps ahead, other rows with register loads one
// sub-step ahead.  Packed sign
// words (32 domains each) are read four at a time straight into the lane of their
// row.  The warps of a CTA take consecutive row groups of the same segment and
// synchronise once per step of 128 domains.  A second kernel (a warp per row) combines
// the S segment partials of every row in index order and closes
// d_eff = phi1 phi2 C + cdiag.
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "qpm_common.cuh"
#include "qpm_internal.h"
#include "qpm_rows.cuh"

namespace qpm {

// partial monoids, structure of arrays: part[(comp * S + s) * NPpad + i], comp in A,B,C
// Float genes of rows that are not 16-byte aligned (scalar loads, one sub-step ahead
// in registers).  blk: the problem's sign-block table, read as float4.
// grid (S, ceil(groups / ER_WPC)).
template <bool COMP>
static __global__ void __launch_bounds__(ER_WPC * 32, 5)
    k_eval_rows(const float *__restrict__ src, int64_t ld, EvalShape sh,
                const float4 *__restrict__ blk, float2 *__restrict__ part) {
  extern __shared__ float4 tb[];  // two steps of sign-block entries
  __shared__ float4 tile[ER_WPC][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int s = blockIdx.x, m0 = s * sh.L, m1 = min(sh.N, m0 + sh.L);
  const int r0 = (blockIdx.y * ER_WPC + warp) * 32;
  const bool live = r0 < sh.NP;
  const int nb = (sh.N + 3) >> 2, nsteps = (m1 - m0 + 127) >> 7;
  float4 R[8];
  if (live) er_load_genes<false>(src, ld, sh, r0, m0, R);
  er_stage_step(tb, blk, m0, 0, nb);
  const float2 *bt = (const float2 *)tb;
  ErAcc<COMP> acc;
  acc.zero();
  float4 *T = tile[warp];
  for (int k = 0; k < nsteps; ++k) {
    cp_async_wait<0>();  // this thread's copies of step k
    __syncthreads();     // everyone's copies of step k; everyone done with step k - 1
    if (k + 1 < nsteps) er_stage_step(tb + ((k + 1) & 1) * ER_STEP_F4_P, blk, m0, k + 1, nb);
    if (!live) continue;
    const float2 *bp = bt + (size_t)(k & 1) * 2 * ER_STEP_F4_P;
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {  // 4 sub-steps of 32 domains
      const int ms = m0 + 128 * k + 32 * q;
      if (ms >= m1) break;
      __syncwarp();
#pragma unroll
      for (int j = 0; j < 8; ++j) T[er_tix(4 * j + (lane >> 3), lane & 7)] = R[j];
      __syncwarp();
      if (ms + 32 < m1) er_load_genes<false>(src, ld, sh, r0, ms + 32, R);
#pragma unroll
      for (int c4 = 0; c4 < 8; ++c4) {  // the sub-step's 8 blocks of 4 domains
        er_push_block(acc.m, er_pattern(T[er_tix(lane, c4)]), bp + (8 * q + c4) * BLK_F2);
        if ((c4 & 3) == 3) acc.fold();
      }
    }
  }
  if (!live) return;
  acc.fold();
  const Mono run = acc.get();
  const size_t stride = (size_t)sh.S * sh.NPpad;
  const size_t o = (size_t)s * sh.NPpad + r0 + lane;
  part[o] = run.A;
  part[stride + o] = run.B;
  part[2 * stride + o] = run.C;
}

// Float genes of 16-byte aligned rows through the per-warp ring of er_ring_sweep (60 KB
// of shared memory per CTA, 3 CTAs per SM); the accumulation order equals k_eval_rows'.
// grid (S, ceil(groups / ER_WPC)).
constexpr int ER_RING_CTAS = 3;  // resident CTAs per SM (shared memory)
// TMA: the gene tiles come by TMA copies (er_ring_sweep_tma, `gmap`), else by cp.async.
template <bool COMP, bool TMA>
static __global__ void __launch_bounds__(ER_WPC * 32, ER_RING_CTAS)
    k_eval_rows_ring(const __grid_constant__ CUtensorMap gmap, const float *__restrict__ src,
                     int64_t ld, EvalShape sh, const float4 *__restrict__ blk,
                     float2 *__restrict__ part) {
  extern __shared__ float4 dyn_raw[];
  float4 *dyn = dyn_raw;
  if constexpr (TMA)  // 1024-byte aligned for the swizzled tiles (the launch adds the slack)
    dyn = (float4 *)((unsigned char *)dyn_raw + ((1024 - (smem_u32(dyn_raw) & 1023)) & 1023));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int s = blockIdx.x, m0 = s * sh.L, m1 = min(sh.N, m0 + sh.L);
  const int r0 = (blockIdx.y * ER_WPC + warp) * 32;
  const bool live = r0 < sh.NP;
  const float4 *const tabs[1] = {blk};
  ErAcc<COMP> acc;
  acc.zero();
  auto push = [&](uint32_t e, const float2 *E, int b) {
    er_push_block(acc.m, e, E + b * BLK_F2);
    if ((b & 3) == 3) acc.fold();
  };
  if constexpr (TMA) er_ring_sweep_tma<1>(dyn, &gmap, sh, tabs, m0, m1, r0, live, push);
  else er_ring_sweep<1>(dyn, src, ld, sh, tabs, m0, m1, r0, live, push);
  if (!live) return;
  acc.fold();
  const Mono run = acc.get();
  const size_t stride = (size_t)sh.S * sh.NPpad;
  const size_t o = (size_t)s * sh.NPpad + r0 + lane;
  part[o] = run.A;
  part[stride + o] = run.B;
  part[2 * stride + o] = run.C;
}

// Packed sign words: the sign-block sweep.  A CTA of ER_WPC_P warps takes ER_WPC_P
// row groups of one segment; per block of 4 domains the lane's 4 sign bits select the
// block's triple among the staged sign-block entries (conflict-free: the 8 entries of
// a block fall in distinct banks).  The entries are streamed per step of 128 domains
// (32 blocks, 6 KB) into two buffers with cp.async, the next step's while this one
// is swept, behind one CTA barrier per step; the sign words come one step ahead in
// registers.  Compensation folds every 4 blocks.  VECW: 16-byte word loads.
// grid (S, ceil(groups / ER_WPC_P)).
template <bool VECW, bool COMP>
static __global__ void __launch_bounds__(ER_WPC_P * 32)
    k_eval_packed(const uint32_t *__restrict__ src, int64_t ld, EvalShape sh,
                  const float4 *__restrict__ blk, float2 *__restrict__ part) {
  extern __shared__ float4 tb[];  // two steps of sign-block entries
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int s = blockIdx.x, m0 = s * sh.L, m1 = min(sh.N, m0 + sh.L);
  const int r0 = (blockIdx.y * ER_WPC_P + warp) * 32;
  const bool live = r0 < sh.NP;
  const int nb = (sh.N + 3) >> 2, nsteps = (m1 - m0 + 127) >> 7;
  uint4 W = make_uint4(0u, 0u, 0u, 0u);
  if (live) W = er_load_words<VECW>(src, ld, sh, r0 + lane, m0);
  er_stage_step(tb, blk, m0, 0, nb);
  const float2 *bt = (const float2 *)tb;
  ErAcc<COMP> acc;
  acc.zero();
  for (int k = 0; k < nsteps; ++k) {
    cp_async_wait<0>();  // this thread's copies of step k
    __syncthreads();     // everyone's copies of step k; everyone done with step k - 1
    if (k + 1 < nsteps) er_stage_step(tb + ((k + 1) & 1) * ER_STEP_F4_P, blk, m0, k + 1, nb);
    if (live) {
      const int ms = m0 + 128 * k;
      const uint4 cur = W;
      if (ms + 128 < m1) W = er_load_words<VECW>(src, ld, sh, r0 + lane, ms + 128);
      const float2 *bp = bt + (size_t)(k & 1) * 2 * ER_STEP_F4_P;
      const uint32_t ws[4] = {cur.x, cur.y, cur.z, cur.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const ErWord f = er_fold_word(ws[q]);
#pragma unroll
        for (int j = 0; j < 8; ++j) {  // the word's 8 blocks of 4 domains
          er_push_entry(acc.m, (f.folded >> (4 * j + 1)) & 7u, (f.lo << (31 - 4 * j)) & 0x80000000u,
                        bp + (8 * q + j) * BLK_F2);
          if ((j & 3) == 3) acc.fold();
        }
      }
    }
  }
  if (!live) return;
  acc.fold();
  const Mono run = acc.get();
  const size_t stride = (size_t)sh.S * sh.NPpad;
  const size_t o = (size_t)s * sh.NPpad + r0 + lane;
  part[o] = run.A;
  part[stride + o] = run.B;
  part[2 * stride + o] = run.C;
}

// one warp per row: d_eff = phi1 phi2 C + cdiag of the combined segments
static __global__ void k_eval_combine(EvalShape sh, const float2 *__restrict__ part,
                                      const float2 *__restrict__ konst, float2 *__restrict__ deff,
                                      float *__restrict__ fit) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= sh.NP) return;
  const Mono acc = combine_segments(part, sh.S, sh.NPpad, row);
  if ((threadIdx.x & 31) == 0) {
    const float2 D = deff_from(acc, konst[0], konst[1]);
    deff[row] = D;
    if (fit) fit[row] = fit_of(D);
  }
}

// ------------------------------------------------------------- caches (host)
namespace {
struct TableEntry {
  float4 *table = nullptr;
  double2 *part = nullptr;
  float2 *konst = nullptr;
  cudaEvent_t ready = nullptr;
  float2 *blk = nullptr;  // sign-block table, built on the first packed call
  cudaEvent_t blk_ready = nullptr;
};
struct ScratchEntry {
  void *ptr = nullptr;
  size_t bytes = 0;
};
std::mutex g_mu;
std::map<std::tuple<int, int32_t, double, double>, TableEntry> g_tables;
std::map<std::pair<int, cudaStream_t>, ScratchEntry> g_scratch;
constexpr size_t MAX_TABLES = 64;

qpm_status release_device_caches(int dev) {
  QPM_CUDA(cudaDeviceSynchronize());
  for (auto it = g_tables.begin(); it != g_tables.end();) {
    if (std::get<0>(it->first) == dev) {
      cudaFree(it->second.table);
      cudaFree(it->second.part);
      cudaFree(it->second.konst);
      cudaEventDestroy(it->second.ready);
      if (it->second.blk) cudaFree(it->second.blk);
      if (it->second.blk_ready) cudaEventDestroy(it->second.blk_ready);
      it = g_tables.erase(it);
    } else {
      ++it;
    }
  }
  for (auto it = g_scratch.begin(); it != g_scratch.end();) {
    if (it->first.first == dev) {
      cudaFree(it->second.ptr);
      it = g_scratch.erase(it);
    } else {
      ++it;
    }
  }
  return QPM_OK;
}

size_t device_table_count(int dev) {
  size_t n = 0;
  for (const auto &kv : g_tables) n += (std::get<0>(kv.first) == dev);
  return n;
}

// phasor table in natural order for (device, problem); built on `stream` on a miss.
// blk (if non-NULL) receives the sign-block table, built on `stream` the first time
// it is asked for.  Never evicts: TableLease makes room before its first lookup.
// Caller holds g_mu.
qpm_status get_table(const qpm_problem *p, cudaStream_t stream, const float4 **table,
                     const float2 **konst, const float2 **blk = nullptr) {
  int dev = 0;
  QPM_CUDA(cudaGetDevice(&dev));
  auto key = std::make_tuple(dev, p->N, p->kappa1, p->kappa2);
  auto it = g_tables.find(key);
  if (it == g_tables.end()) {
    TableEntry e;
    const int32_t Npad = (p->N + 3) & ~3;
    cudaError_t ce = cudaMalloc(&e.table, sizeof(float4) * (size_t)Npad);
    if (ce == cudaSuccess) ce = cudaMalloc(&e.part, sizeof(double2) * (size_t)table_part_count(Npad));
    if (ce == cudaSuccess) ce = cudaMalloc(&e.konst, sizeof(float2) * 4);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&e.ready, cudaEventDisableTiming);
    qpm_status st = ce == cudaSuccess ? QPM_OK : cuda_fail(ce, "allocating a phasor table");
    if (st == QPM_OK) {
      TableSpec s{p->N, Npad, 1, Npad, p->kappa1, p->kappa2};
      st = launch_table(s, e.table, e.part, e.konst, nullptr, stream);
    }
    if (st == QPM_OK && (ce = cudaEventRecord(e.ready, stream)) != cudaSuccess)
      st = cuda_fail(ce, "cudaEventRecord");
    if (st != QPM_OK) {  // the cache keeps no half-built entry
      cudaFree(e.table);
      cudaFree(e.part);
      cudaFree(e.konst);
      if (e.ready) cudaEventDestroy(e.ready);
      return st;
    }
    it = g_tables.emplace(key, e).first;
  } else {
    QPM_CUDA(cudaStreamWaitEvent(stream, it->second.ready, 0));
  }
  *table = it->second.table;
  *konst = it->second.konst;
  if (blk) {
    TableEntry &e = it->second;
    if (!e.blk) {
      const size_t nb = (size_t)(p->N + 3) / 4;
      float2 *b = nullptr;
      cudaEvent_t ev = nullptr;
      QPM_CUDA(cudaMalloc(&b, sizeof(float2) * BLK_F2 * nb));
      cudaError_t ce = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      qpm_status st = ce == cudaSuccess ? launch_block_table(p->N, p->kappa1, p->kappa2, b, stream)
                                        : cuda_fail(ce, "cudaEventCreateWithFlags");
      if (st == QPM_OK && (ce = cudaEventRecord(ev, stream)) != cudaSuccess)
        st = cuda_fail(ce, "cudaEventRecord");
      if (st != QPM_OK) {  // the entry keeps no half-built table
        cudaFree(b);
        if (ev) cudaEventDestroy(ev);
        return st;
      }
      e.blk = b;
      e.blk_ready = ev;
    } else {
      QPM_CUDA(cudaStreamWaitEvent(stream, e.blk_ready, 0));
    }
    *blk = e.blk;
  }
  return QPM_OK;
}

qpm_status get_scratch(cudaStream_t stream, size_t bytes, void **ptr) {
  int dev = 0;
  QPM_CUDA(cudaGetDevice(&dev));
  ScratchEntry &e = g_scratch[std::make_pair(dev, stream)];
  if (e.bytes < bytes) {
    if (e.ptr) {
      QPM_CUDA(cudaStreamSynchronize(stream));
      QPM_CUDA(cudaFree(e.ptr));
      e.ptr = nullptr;
      e.bytes = 0;
    }
    QPM_CUDA(cudaMalloc(&e.ptr, bytes));
    e.bytes = bytes;
  }
  *ptr = e.ptr;
  return QPM_OK;
}
}  // namespace

// split for the row sweep: about `warps_per_sm` warps per SM in total (20 suit
// float genes; the packed sweep holds fewer registers and runs best near 32),
// segments a multiple of ER_LQ domains and at most ER_LMAX
EvalShape eval_rows_shape(int NP, int N, int warps_per_sm, int lmax) {
  EvalShape sh;
  sh.NP = NP;
  sh.N = N;
  sh.groups = (NP + 31) / 32;
  sh.NPpad = sh.groups * 32;
  const int target = sm_count() * warps_per_sm;
  const int S0 = std::max(1, (target + sh.groups - 1) / sh.groups);
  int L = (N + S0 - 1) / S0;
  L = (L + ER_LQ - 1) / ER_LQ * ER_LQ;
  L = std::min(std::max(L, ER_LQ), lmax > 0 ? lmax : ER_LMAX);
  sh.L = L;
  sh.S = (N + L - 1) / L;
  return sh;
}

// shape of the float-gene sweep: the ring kernel for aligned rows keeps ER_WPC x
// ER_RING_CTAS warps per SM, the register-prefetch kernel 20
static EvalShape eval_genes_shape(int NP, int N, bool aligned) {
  return eval_rows_shape(NP, N, aligned ? ER_WPC * ER_RING_CTAS : 20);
}

static qpm_status launch_eval_rows(bool aligned, bool comp, const float *g, int64_t ld,
                                   const EvalShape &sh, const float2 *blk, float2 *part,
                                   cudaStream_t stream) {
  const dim3 grid(sh.S, (sh.groups + ER_WPC - 1) / ER_WPC);
  const float4 *b4 = (const float4 *)blk;
  if (aligned) {
    CUtensorMap gmap{};
    const bool tma = make_tile_map(&gmap, g, sh.NP, sh.N, ld);
    const void *fn = tma ? (comp ? (const void *)k_eval_rows_ring<true, true>
                                 : (const void *)k_eval_rows_ring<false, true>)
                         : (comp ? (const void *)k_eval_rows_ring<true, false>
                                 : (const void *)k_eval_rows_ring<false, false>);
    const size_t smem = tma ? 1024 + er_ring_smem_tma(1) : er_ring_smem(1);
    QPM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    void *args[] = {(void *)&gmap, (void *)&g, (void *)&ld, (void *)&sh, (void *)&b4, (void *)&part};
    QPM_CUDA(cudaLaunchKernel(fn, grid, dim3(ER_WPC * 32), args, smem, stream));
  } else {
    const size_t smem = sizeof(float4) * 2 * ER_STEP_F4_P;
    if (comp) k_eval_rows<true><<<grid, ER_WPC * 32, smem, stream>>>(g, ld, sh, b4, part);
    else k_eval_rows<false><<<grid, ER_WPC * 32, smem, stream>>>(g, ld, sh, b4, part);
  }
  return QPM_OK;
}

static void launch_eval_packed(bool vecw, bool comp, const uint32_t *src, int64_t ld,
                               const EvalShape &sh, const float2 *blk, float2 *part,
                               cudaStream_t stream) {
  const dim3 grid(sh.S, (sh.groups + ER_WPC_P - 1) / ER_WPC_P);
  const size_t smem = sizeof(float4) * 2 * ER_STEP_F4_P;
  const float4 *b4 = (const float4 *)blk;
#define QPM_EP(V, C) k_eval_packed<V, C><<<grid, ER_WPC_P * 32, smem, stream>>>(src, ld, sh, b4, part)
  if (vecw) {
    if (comp) QPM_EP(true, true); else QPM_EP(true, false);
  } else {
    if (comp) QPM_EP(false, true); else QPM_EP(false, false);
  }
#undef QPM_EP
}

static qpm_status eval_common(const qpm_problem *prob, const void *src, int64_t ld, int32_t NP,
                              int kind, float *d_eff, float *fit, int32_t comp,
                              cudaStream_t stream) {
  if (!prob || !src || !d_eff) return fail(QPM_ERR_ARG, "qpm_eval: NULL pointer");
  if (prob->N < 1 || NP < 1) return fail(QPM_ERR_ARG, "qpm_eval: need N >= 1 and NP >= 1");
  if (prob->N > (1 << 28)) return fail(QPM_ERR_UNSUPPORTED, "qpm_eval: N too large");
  if (kind == 2 ? (ld < (prob->N + 31) / 32) : (ld < prob->N))
    return fail(QPM_ERR_ARG, "qpm_eval: leading dimension smaller than the row");
  TableLease lease(prob, 1);  // held until the launches below are enqueued
  const float2 *konst, *blk = nullptr;
  qpm_status st = lease.block_table(prob, stream, &blk, &konst);
  if (st != QPM_OK) return st;
  if (NP > ER_WPC * 32 * 65535) return fail(QPM_ERR_UNSUPPORTED, "qpm_eval: too many rows");
  const bool aligned = (ld % 4 == 0) && (((uintptr_t)src & 15) == 0);
  const EvalShape sh = kind == 2 ? eval_rows_shape(NP, prob->N, 32, ER_LMAX_P)
                                 : eval_genes_shape(NP, prob->N, aligned);
  void *scratch;
  st = get_scratch(stream, sizeof(float2) * 3 * (size_t)sh.S * sh.NPpad, &scratch);
  if (st != QPM_OK) return st;
  float2 *part = (float2 *)scratch;
  if (kind == 2) {
    launch_eval_packed(aligned, comp != 0, (const uint32_t *)src, ld, sh, blk, part, stream);
  } else {
    st = launch_eval_rows(aligned, comp != 0, (const float *)src, ld, sh, blk, part, stream);
    if (st != QPM_OK) return st;
  }
  QPM_CUDA(cudaGetLastError());
  k_eval_combine<<<(NP + 7) / 8, 256, 0, stream>>>(sh, part, konst, (float2 *)d_eff, fit);
  QPM_CUDA(cudaGetLastError());
  return QPM_OK;
}


// ---------------------------------------------------------------------------
// Allocation-free variant of qpm_eval.  For callers that must not allocate device
// memory: host callbacks and other code that may not call into the allocator,
// processes whose device memory is all owned by an external allocator, and real-time
// paths where the implicit device synchronisation of cudaMalloc/cudaFree is not
// acceptable.  Its scratch (sign-block table, the constants' reduction, segment
// partials) lives in one file-scope device array of fixed size that every GPU
// loading this library holds until the process exits.
// ---------------------------------------------------------------------------
static constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)16 << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[128] = {nullptr};  // device address of g_noalloc_scratch, per device

// One-time set-up per device (with that device current): the host name
// g_noalloc_scratch is only a host-side stand-in, so its device address is
// looked up once and cached.
qpm_status noalloc_base(void **out) {
  int dev = 0;
  QPM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return fail(QPM_ERR_UNSUPPORTED, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return QPM_OK;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// bytes of the fixed array one call uses: the sign-block table (192 bytes per block of
// 4 domains), the reduction partials of the constants, the constants, and the segment
// partials of the scan (3 float2 per segment and padded row)
size_t noalloc_bytes(int32_t N, const EvalShape &sh) {
  const int32_t Npad = (N + 3) & ~3;
  return up256(sizeof(float2) * BLK_F2 * (size_t)(Npad / 4)) +
         up256(sizeof(double2) * (size_t)table_part_count(Npad)) + 256 +
         up256(sizeof(float2) * 3 * (size_t)sh.S * sh.NPpad);
}
}  // namespace

}  // namespace qpm

extern "C" qpm_status qpm_eval_noalloc(const qpm_problem *prob, const float *genes, int64_t ld,
                                       int32_t NP, float *d_eff, float *fit, int32_t compensated,
                                       qpm_stream_t stream) {
  using namespace qpm;
  if (!prob || !genes || !d_eff) return fail(QPM_ERR_ARG, "qpm_eval_noalloc: NULL pointer");
  if (prob->N < 1 || NP < 1) return fail(QPM_ERR_ARG, "qpm_eval_noalloc: need N >= 1 and NP >= 1");
  if (ld < prob->N) return fail(QPM_ERR_ARG, "qpm_eval_noalloc: leading dimension smaller than the row");
  if (prob->N > (1 << 28) || NP > (1 << 26))
    return fail(QPM_ERR_ARG, "qpm_eval_noalloc: N above 2^28 or NP above 2^26");
  if (NP > ER_WPC * 32 * 65535) return fail(QPM_ERR_UNSUPPORTED, "qpm_eval_noalloc: too many rows");
  const bool vec = (ld % 4 == 0) && (((uintptr_t)genes & 15) == 0);
  const EvalShape sh = eval_genes_shape(NP, prob->N, vec);
  const int32_t Npad = (prob->N + 3) & ~3;
  const size_t need = noalloc_bytes(prob->N, sh);
  if (need > NOALLOC_SCRATCH_BYTES)
    return fail(QPM_ERR_ARG, "qpm_eval_noalloc: N and NP need " + std::to_string(need) +
                                 " bytes of scratch, more than the fixed 16 MiB (16777216)");
  void *base = nullptr;
  qpm_status st = noalloc_base(&base);
  if (st != QPM_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  char *p = (char *)base;
  const size_t b_blk = up256(sizeof(float2) * BLK_F2 * (size_t)(Npad / 4));
  const size_t b_tpart = up256(sizeof(double2) * (size_t)table_part_count(Npad));
  float2 *blk = (float2 *)p;
  double2 *tpart = (double2 *)(p + b_blk);
  float2 *konst = (float2 *)(p + b_blk + b_tpart);
  float2 *part = (float2 *)(p + b_blk + b_tpart + 256);
  // every word read below is written first in this call (the sign-block table, the
  // constants and their partial sums, every segment partial of every padded row), so
  // nothing needs zeroing; the constants come from k_table without a phasor table
  TableSpec ts{prob->N, Npad, 1, Npad, prob->kappa1, prob->kappa2};
  st = launch_table(ts, nullptr, tpart, konst, nullptr, s);
  if (st != QPM_OK) return st;
  st = launch_block_table(prob->N, prob->kappa1, prob->kappa2, blk, s);
  if (st != QPM_OK) return st;
  st = launch_eval_rows(vec, compensated != 0, genes, ld, sh, blk, part, s);
  if (st != QPM_OK) return st;
  QPM_CUDA(cudaGetLastError());
  k_eval_combine<<<(NP + 7) / 8, 256, 0, s>>>(sh, part, konst, (float2 *)d_eff, fit);
  QPM_CUDA(cudaGetLastError());
  return QPM_OK;
}

qpm::TableLease::TableLease(const qpm_problem *problems, int count) {
  g_mu.lock();
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    st_ = cuda_fail(e, "cudaGetDevice");
    return;
  }
  size_t misses = 0;
  for (int k = 0; k < count; ++k) {
    const qpm_problem &p = problems[k];
    bool seen = g_tables.count(std::make_tuple(dev, p.N, p.kappa1, p.kappa2)) != 0;
    for (int m = 0; m < k && !seen; ++m)
      seen = problems[m].N == p.N && problems[m].kappa1 == p.kappa1 &&
             problems[m].kappa2 == p.kappa2;
    misses += !seen;
  }
  if (misses > 0 && device_table_count(dev) + misses > MAX_TABLES)
    st_ = release_device_caches(dev);
}

qpm::TableLease::~TableLease() { g_mu.unlock(); }

qpm_status qpm::TableLease::table(const qpm_problem *p, cudaStream_t stream, const float4 **table,
                                  const float2 **konst) {
  if (st_ != QPM_OK) return st_;
  return get_table(p, stream, table, konst);
}

qpm_status qpm::TableLease::block_table(const qpm_problem *p, cudaStream_t stream,
                                        const float2 **blk, const float2 **konst) {
  if (st_ != QPM_OK) return st_;
  const float4 *table;
  return get_table(p, stream, &table, konst, blk);
}

extern "C" qpm_status qpm_eval(const qpm_problem *prob, const float *genes, int64_t ld,
                               int32_t NP, float *d_eff, float *fit, int32_t compensated,
                               qpm_stream_t stream) {
  return qpm::eval_common(prob, genes, ld, NP, 1, d_eff, fit, compensated,
                          (cudaStream_t)stream);
}

extern "C" qpm_status qpm_eval_packed(const qpm_problem *prob, const uint32_t *signs,
                                      int64_t ld_words, int32_t NP, float *d_eff, float *fit,
                                      int32_t compensated, qpm_stream_t stream) {
  return qpm::eval_common(prob, signs, ld_words, NP, 2, d_eff, fit, compensated,
                          (cudaStream_t)stream);
}

extern "C" qpm_status qpm_release_caches(void) {
  std::lock_guard<std::mutex> lock(qpm::g_mu);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return qpm::cuda_fail(e, "cudaGetDevice");
  return qpm::release_device_caches(dev);
}
