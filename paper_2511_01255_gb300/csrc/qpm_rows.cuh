// qpm_rows.cuh -- the row sweep shared by the fitness kernels of qpm_eval and of
// the multi-wavelength objective: a warp takes 32 rows (lane = row) and one
// segment of L domains (a multiple of ER_LQ) and walks it in index order, one block
// of 4 domains at a time: a block of +-1 domains takes one of 16 sign patterns and
// its monoid triple depends on the pattern only, so the sign-block table
// (launch_block_table) holds the triples and the sweep appends one per lookup.  The
// table entries are streamed into shared memory per step of 128 domains.
#pragma once
#include "qpm_common.cuh"
#include "qpm_internal.h"
#include "qpm_tma.cuh"

namespace qpm {

constexpr int ER_WPC = 4;      // warps (row groups of 32) per CTA of the float sweeps
constexpr int ER_LQ = 128;     // segment length quantum (domains)
constexpr int ER_LMAX = 1920;  // longest segment of the float sweeps

// per-warp tile: 32 rows x 32 domains as float4 [row][c4], the column xor-swizzled by
// the row so that both the staging stores (8 columns of a row per quarter-warp) and
// the row walks (8 rows of a column) are free of bank conflicts
__device__ __forceinline__ int er_tix(int row, int c4) { return row * 8 + (c4 ^ (row & 7)); }

// float genes of one step (32 domains from ms) of rows r0..r0+31: lane l holds
// float4 k * 32 + l, i.e. row 4k + l / 8, columns 4 (l % 8) .. +3
template <bool VEC>
__device__ __forceinline__ void er_load_genes(const float *__restrict__ g, int64_t ld,
                                              const EvalShape &sh, int r0, int ms, float4 R[8]) {
  const int lane = threadIdx.x & 31;
  const int m = ms + 4 * (lane & 7);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int gr = r0 + 4 * k + (lane >> 3);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gr < sh.NP) {
      const float *rp = g + (int64_t)gr * ld;
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

// the same step copied asynchronously (cp.async, not committed) into the per-warp
// tile T in the layout of er_tix: lane l's copy k lands at row 4k + l / 8, columns
// 4 (l % 8) .. +3.  16-byte aligned rows (ld % 4 == 0) only; genes past the row
// end and rows past NP are zero-filled.
__device__ __forceinline__ void er_copy_genes(float4 *T, const float *__restrict__ g, int64_t ld,
                                              const EvalShape &sh, int r0, int ms) {
  const int lane = threadIdx.x & 31;
  const int m = ms + 4 * (lane & 7);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int tr = 4 * k + (lane >> 3), gr = r0 + tr;
    const float *src = g;
    int bytes = 0;
    if (gr < sh.NP && m < sh.N) {
      src = g + (int64_t)gr * ld + m;
      bytes = 4 * min(4, sh.N - m);
    }
    cp_async16(&T[er_tix(tr, lane & 7)], src, bytes);
  }
}

// sign words of one packed step (128 domains from ms, a multiple of 128) of row
// `row`; words beyond the row's last domain are zero
template <bool VECW>
__device__ __forceinline__ uint4 er_load_words(const uint32_t *__restrict__ w, int64_t ld,
                                               const EvalShape &sh, int row, int ms) {
  uint4 v = make_uint4(0u, 0u, 0u, 0u);
  if (row < sh.NP) {
    const uint32_t *rp = w + (int64_t)row * ld + (ms >> 5);
    const int nw = (sh.N - ms + 31) >> 5;  // words of this row from ms on
    if (VECW && nw >= 4) {
      v = __ldg((const uint4 *)rp);
    } else {
      if (nw > 0) v.x = __ldg(rp);
      if (nw > 1) v.y = __ldg(rp + 1);
      if (nw > 2) v.z = __ldg(rp + 2);
      if (nw > 3) v.w = __ldg(rp + 3);
    }
  }
  return v;
}

// sign pattern of 4 genes: bit j set iff gene j < 0 (d_j = -1; -0.0 counts as +1)
__device__ __forceinline__ uint32_t er_pattern(const float4 &x) {
  return (x.x < 0.f ? 1u : 0u) | (x.y < 0.f ? 2u : 0u) | (x.z < 0.f ? 4u : 0u) |
         (x.w < 0.f ? 8u : 0u);
}

constexpr int ER_WPC_P = 8;      // warps (row groups of 32) per CTA of the packed sweep
constexpr int ER_LMAX_P = 4096;  // longest segment of the packed sweep
constexpr int ER_STEP_F4_P = 32 * BLK_F2 / 2;  // float4 of entries per step of 128 domains

// the sign-block entries of step k of a segment starting at m0 (blocks
// m0 / 4 + 32 k .. + 31) into buf, copied with cp.async by the whole CTA (not
// committed); blocks past the last of the problem are zero
__device__ __forceinline__ void er_stage_entries(float4 *buf, const float4 *__restrict__ blk,
                                                 int m0, int k, int nb) {
  const int b0 = (m0 >> 2) + 32 * k;
  for (int i = threadIdx.x; i < ER_STEP_F4_P; i += blockDim.x) {
    if (b0 + i / (BLK_F2 / 2) < nb) cp_async16(buf + i, blk + (size_t)b0 * (BLK_F2 / 2) + i);
    else buf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// er_stage_entries committed as one group
__device__ __forceinline__ void er_stage_step(float4 *buf, const float4 *__restrict__ blk, int m0,
                                              int k, int nb) {
  er_stage_entries(buf, blk, m0, k, nb);
  cp_async_commit();
}

// Ring sweep of one warp over its segment [m0, m1) for float genes in 16-byte aligned
// rows, with NT sign-block tables.  Sub-step u (32 domains) of the warp's 32 rows lands
// by cp.async in slot u % ER_RING of the warp's ring of 4 KB tiles, issued ER_RING - 1
// sub-steps before it is swept, so 8 KB of each warp's loads stay in flight without
// holding registers.  Every sub-step commits one cp.async group (empty past the
// segment's end) holding the genes of sub-step u + ER_RING - 1 and, at the start of a
// 128-domain step, the next step's entries of every table; waiting until at most
// ER_RING - 2 groups are pending therefore completes sub-step u's genes and, for
// ER_RING <= 5, its step's entries.  Shared memory `dyn`: [2 steps][NT][ER_STEP_F4_P]
// entries, then ER_WPC rings of ER_RING tiles.  push(e, E, b) appends block b (0..31)
// of the current step with sign pattern e; table t's entries of the step start at
// E + t * 2 * ER_STEP_F4_P (float2).  Every thread of the CTA must call this (it holds
// CTA barriers); warps without rows (live false) only stage entries.
constexpr int ER_RING = 3;
static_assert(ER_RING >= 2 && ER_RING <= 5, "a step's entries must complete with its first sub-step");
__host__ __device__ constexpr size_t er_ring_smem(int NT) {
  return sizeof(float4) * (2 * (size_t)NT * ER_STEP_F4_P + (size_t)ER_WPC * ER_RING * 256);
}

template <int NT, class Push>
__device__ __forceinline__ void er_ring_sweep(float4 *dyn, const float *__restrict__ g, int64_t ld,
                                              const EvalShape &sh, const float4 *const *tabs,
                                              int m0, int m1, int r0, bool live, Push &&push) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4 *ring = dyn + 2 * NT * ER_STEP_F4_P + warp * (ER_RING * 256);
  const int nb = (sh.N + 3) >> 2, nsteps = (m1 - m0 + 127) >> 7, nsub = (m1 - m0 + 31) >> 5;
#pragma unroll
  for (int t = 0; t < NT; ++t) er_stage_entries(dyn + t * ER_STEP_F4_P, tabs[t], m0, 0, nb);
  cp_async_commit();
#pragma unroll
  for (int u = 0; u < ER_RING - 1; ++u) {
    if (live && u < nsub) er_copy_genes(ring + u * 256, g, ld, sh, r0, m0 + 32 * u);
    cp_async_commit();
  }
  int slot = 0;  // u % ER_RING
  for (int k = 0; k < nsteps; ++k) {
    const float2 *bp = (const float2 *)dyn + (size_t)(k & 1) * NT * 2 * ER_STEP_F4_P;
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {  // 4 sub-steps of 32 domains
      const int u = 4 * k + q;
      if (u >= nsub) break;
      cp_async_wait<ER_RING - 2>();  // this thread's copies of sub-step u (and of step k)
      if (q == 0) __syncthreads();   // everyone's; everyone done with step k - 1
      else __syncwarp();             // the warp's lanes' copies; done with sub-step u - 1
      const int ua = u + ER_RING - 1;
      const int sa = slot == 0 ? ER_RING - 1 : slot - 1;  // the slot swept at u - 1
      if (live && ua < nsub) er_copy_genes(ring + sa * 256, g, ld, sh, r0, m0 + 32 * ua);
      if (q == 0 && k + 1 < nsteps) {
#pragma unroll
        for (int t = 0; t < NT; ++t)
          er_stage_entries(dyn + (((k + 1) & 1) * NT + t) * ER_STEP_F4_P, tabs[t], m0, k + 1, nb);
      }
      cp_async_commit();
      const float4 *T = ring + slot * 256;
      slot = slot + 1 == ER_RING ? 0 : slot + 1;
      if (!live) continue;
#pragma unroll
      for (int c4 = 0; c4 < 8; ++c4) push(er_pattern(T[er_tix(lane, c4)]), bp, 8 * q + c4);
    }
  }
  cp_async_wait<0>();
}

// The same sweep with each sub-step's 32 x 32 gene tile brought in by one TMA copy
// (`gmap`: the genes as an NP x N float matrix, 32 x 32 boxes, 128-byte swizzle, zero
// fill past the row end and the last row) that completes on the slot's mbarrier; the
// steps' sign-block entries still come by cp.async, one group per step.  `dyn` must be
// 1024-byte aligned (the tiles follow the NT tables' 12 KB per table and step); the
// mbarriers follow the rings: er_ring_smem_tma bytes in all.  A wait that runs out
// (bounded by %globaltimer) fills the tile with NaN, which makes the rows' results NaN.
__host__ __device__ constexpr size_t er_ring_smem_tma(int NT) {
  return er_ring_smem(NT) + (size_t)ER_WPC * ER_RING * 8;
}
__device__ __forceinline__ void er_nan_tile(float4 *T) {
  const float n = __int_as_float(0x7fc00000);
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int c4 = 0; c4 < 8; ++c4) T[er_tix(lane, c4)] = make_float4(n, n, n, n);
}
template <int NT, class Push>
__device__ __forceinline__ void er_ring_sweep_tma(float4 *dyn, const CUtensorMap *gmap,
                                                  const EvalShape &sh, const float4 *const *tabs,
                                                  int m0, int m1, int r0, bool live, Push &&push) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4 *ring = dyn + 2 * NT * ER_STEP_F4_P + warp * (ER_RING * 256);
  const unsigned bar0 =
      smem_u32(dyn + 2 * NT * ER_STEP_F4_P + ER_WPC * ER_RING * 256) + warp * ER_RING * 8;
  const int nb = (sh.N + 3) >> 2, nsteps = (m1 - m0 + 127) >> 7, nsub = (m1 - m0 + 31) >> 5;
#pragma unroll
  for (int t = 0; t < NT; ++t) er_stage_entries(dyn + t * ER_STEP_F4_P, tabs[t], m0, 0, nb);
  cp_async_commit();
  if (live && lane == 0) {
    for (int k = 0; k < ER_RING; ++k) mbar_init(bar0 + 8 * k, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
    for (int u = 0; u < ER_RING - 1 && u < nsub; ++u) {
      mbar_expect_tx(bar0 + 8 * u, 4096);
      tma_load_tile(ring + u * 256, gmap, m0 + 32 * u, r0, bar0 + 8 * u);
    }
  }
  bool ok = true;
  int u_fail = -1;  // first sub-step whose tile did not arrive in time
  int slot = 0;     // u % ER_RING
  for (int k = 0; k < nsteps; ++k) {
    const float2 *bp = (const float2 *)dyn + (size_t)(k & 1) * NT * 2 * ER_STEP_F4_P;
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {  // 4 sub-steps of 32 domains
      const int u = 4 * k + q;
      if (u >= nsub) break;
      if (q == 0) {
        cp_async_wait<0>();  // this thread's copies of step k's entries
        __syncthreads();     // everyone's; everyone done with step k - 1
      } else {
        __syncwarp();  // the warp's lanes are done with sub-step u - 1's tile
      }
      const int ua = u + ER_RING - 1;
      const int sa = slot == 0 ? ER_RING - 1 : slot - 1;  // the slot swept at u - 1
      if (live && lane == 0 && ok && ua < nsub) {
        fence_async_smem();
        mbar_expect_tx(bar0 + 8 * sa, 4096);
        tma_load_tile(ring + sa * 256, gmap, m0 + 32 * ua, r0, bar0 + 8 * sa);
      }
      if (q == 0 && k + 1 < nsteps) {
#pragma unroll
        for (int t = 0; t < NT; ++t)
          er_stage_entries(dyn + (((k + 1) & 1) * NT + t) * ER_STEP_F4_P, tabs[t], m0, k + 1, nb);
        cp_async_commit();
      }
      float4 *T = ring + slot * 256;
      const unsigned bar = bar0 + 8 * slot;
      slot = slot + 1 == ER_RING ? 0 : slot + 1;
      if (!live) continue;
      const bool arrived = ok && mbar_wait(bar, (u / ER_RING) & 1);
      if (!__all_sync(0xffffffffu, arrived)) {  // ok is uniform across the warp
        if (ok) u_fail = u;
        ok = false;
        er_nan_tile(T);
        __syncwarp();
      }
#pragma unroll
      for (int c4 = 0; c4 < 8; ++c4) push(er_pattern(T[er_tix(lane, c4)]), bp, 8 * q + c4);
    }
  }
  cp_async_wait<0>();
  if (!ok && lane == 0) {  // copies issued after u_fail may still be in flight
    for (int v = u_fail; v < min(u_fail + ER_RING - 1, nsub); ++v)
      mbar_wait(bar0 + 8 * (v % ER_RING), (v / ER_RING) & 1);
  }
}

// append stored entry idx (0..7, the pattern with d_0 = +1) of a block whose 8
// entries start at E8, with A and B negated when sm = 0x80000000 (the block's pattern
// has d_0 = -1 and is the complement of entry idx: an exact sign flip, C unchanged)
__device__ __forceinline__ void er_push_entry(Mono &m, uint32_t idx, uint32_t sm, const float2 *E8) {
  const float2 *E = E8 + 3 * idx;
  const float2 a = E[0], b = E[1];
  Mono R;
  R.A = make_float2(__uint_as_float(__float_as_uint(a.x) ^ sm), __uint_as_float(__float_as_uint(a.y) ^ sm));
  R.B = make_float2(__uint_as_float(__float_as_uint(b.x) ^ sm), __uint_as_float(__float_as_uint(b.y) ^ sm));
  R.C = E[2];
  m = mono_combine(m, R);
}

// append the block with sign pattern e (bit j: d_j = -1)
__device__ __forceinline__ void er_push_block(Mono &m, uint32_t e, const float2 *E8) {
  const uint32_t neg = 0u - (e & 1u);  // all ones when d_0 = -1
  er_push_entry(m, ((e ^ neg) & 0xFu) >> 1, neg & 0x80000000u, E8);
}

// the 8 sign patterns of a packed word folded onto the stored entries at once: every
// nibble whose d_0 bit is set is complemented, so stored entry j of the word's block j
// is bits 4j+1 .. 4j+3 of the result and its sign flip is bit 4j of `lo`
struct ErWord {
  uint32_t folded, lo;
};
__device__ __forceinline__ ErWord er_fold_word(uint32_t w) {
  const uint32_t lo = w & 0x11111111u;
  return {w ^ (lo * 0xFu), lo};
}

// Running monoid of a lane's row: plain FP32 sums, or (COMP) plain sums over 16
// domains (4 sign blocks) Kahan-folded into a compensated triple.
template <bool COMP>
struct ErAcc {
  Mono m;
  MonoK k;
  __device__ __forceinline__ void zero() {
    m = mono_zero();
    if (COMP) k = monok_zero();
  }
  __device__ __forceinline__ void fold() {
    if (COMP) {
      monok_fold_in(k, m);
      m = mono_zero();
    }
  }
  __device__ __forceinline__ Mono get() { return COMP ? monok_fold(k) : m; }
};

// The S segment partials of row `row` combined in index order by one warp: lane l
// folds its contiguous run of segments [l c, l c + c), c = ceil(S / 32), then the
// 32 lane results are combined pairwise in lane order.  part is the structure of
// arrays [comp][S][NPpad] (comp = A, B, C); the result is valid in lane 0.
__device__ __forceinline__ Mono combine_segments(const float2 *__restrict__ part, int S, int NPpad,
                                                 int row) {
  const int lane = threadIdx.x & 31;
  const size_t stride = (size_t)S * NPpad;
  const int c = (S + 31) >> 5;
  const int s0 = lane * c, s1 = min(S, s0 + c);
  Mono acc = mono_zero();
  for (int s = s0; s < s1; ++s) {
    const size_t o = (size_t)s * NPpad + row;
    Mono r;
    r.A = part[o];
    r.B = part[stride + o];
    r.C = part[2 * stride + o];
    acc = mono_combine(acc, r);
  }
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    Mono r;
    r.A.x = __shfl_down_sync(0xffffffffu, acc.A.x, off);
    r.A.y = __shfl_down_sync(0xffffffffu, acc.A.y, off);
    r.B.x = __shfl_down_sync(0xffffffffu, acc.B.x, off);
    r.B.y = __shfl_down_sync(0xffffffffu, acc.B.y, off);
    r.C.x = __shfl_down_sync(0xffffffffu, acc.C.x, off);
    r.C.y = __shfl_down_sync(0xffffffffu, acc.C.y, off);
    if ((lane & (2 * off - 1)) == 0) acc = mono_combine(acc, r);
  }
  return acc;
}

}  // namespace qpm
