// qpm_hwsda.cu -- the HWSDA generation step (Sec. 3.2, Steps 1-7) on sm_103a.
//
// One CTA is the team for one individual at a time: its T threads split the
// N domains into contiguous chunks of c domains (c a multiple of 4), every thread
// builds its chunk of the new vector (DE trial or GWO candidate) straight from
// the generator and the parent rows, scans it into a monoid partial, and the CTA
// combines the partials in index order to d_eff.  The population is stored in
// the matching permuted order, so that every warp-wide float4 access to a row
// (target, donors, leaders, new vector, phasor table) is one contiguous 512 B
// segment.
//
// Every individual owns two row slots; the new vector is always written to the
// slot that is not current and survives by flipping a per-individual slot
// selector, so no row is ever copied.  DE reads selectors of generation parity
// p and writes those of parity p^1; GWO works in place on parity p^1 (it only
// moves omega wolves and only reads the leaders).
//
// Per generation: k_de (all NP trials + greedy selection + leader choice by the
// last CTA) and k_gwo (omega wolves + greedy selection + generation counter by
// the last CTA); or one cooperative persistent kernel that runs both phases for
// many generations with bounded grid barriers in between; or, for many
// instances, one launch of k_batch in which thread-block clusters take whole
// instances from a queue.
#include <math.h>

#include <string.h>

#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "qpm_common.cuh"
#include "qpm_internal.h"
#include "qpm_sync.cuh"

namespace qpm {

struct InstDev {
  int32_t N, Npad, NP, T, c, G;
  int32_t combine, compensated;
  float F, CR;
  uint32_t crthr;  // cr_threshold(CR)
  uint32_t inst;
  uint2 key;
  double kappa1, kappa2;
  float *pop;            // [NP][2][Npad], permuted rows
  int32_t *sel0, *sel1;  // slot selectors, parity 0 / 1
  float *fit;            // [NP]
  float2 *dval;          // [NP]
  float4 *table;         // [Npad], permuted
  double2 *tpart;        // table reduction scratch
  float2 *konst;         // phi1 phi2, cdiag
  double2 *konst64;      // phi1 phi2, cdiag, psi, phi1 (FP64)
  int32_t *lead;         // [3] (four for the discrete GWO)
  unsigned long long *topk;  // [2][NP * 3] partial leader keys (by generation parity)
  unsigned *ctr;         // [4] CTA-completion counters
  int32_t *gen;          // [1] completed generations
  int32_t *best;         // [1] best index (get_best)
  float *trace;          // optional fitness trace
  float *Fsched;         // [G + 1] F of every generation, or NULL for constant F; the
                         // adaptive F (f_schedule 2) writes entry g + 1 during generation g
  const float *Fbase;    // [G + 1] adaptive F only: the schedule of its intermediate state
  int32_t adaptive;      // f_schedule == 2
  // the objective (qpm_objective): kind, problems of the multi-wavelength kinds (the
  // first one's table and constants are table / konst), G0, beta; minimised for the
  // multi-wavelength kinds
  int32_t obj, K, minimize;
  const uint32_t *dthr;  // [G][7] discrete GWO (combine 2): social, flip, plus[0..4] thresholds
  float G0, beta;
  const float4 *mtab[8];   // [Npad] permuted phasor tables of the K problems
  const float2 *mkonst[8];  // their FP32 constants
  unsigned long long *dekey;  // [NP] persistent form: DE survivor keys (lead_key) for Step 3
};

template <bool NC>
__device__ __forceinline__ float4 ld4(const float *p) {
  if (NC) return __ldg((const float4 *)p);
  return *(const float4 *)p;
}
// phasor table entry: from shared memory (TS) or through the read-only path
template <bool TS>
__device__ __forceinline__ float4 ldt(const float4 *p) {
  if (TS) return *p;
  return __ldg(p);
}

// Running monoid of a thread's chunk.  Plain: FP32 sums.  Compensated: the
// domains are summed plainly in blocks of 8 and every block is Kahan-folded into
// the running triple (blocked Kahan summation: error of order 8 eps instead of c eps).
template <bool COMP>
struct Acc {
  Mono m;   // plain sums / current block
  MonoK k;  // compensated running triple
  __device__ __forceinline__ void zero() {
    m = mono_zero();
    if (COMP) k = monok_zero();
  }
  __device__ __forceinline__ void push(float d, const float4 &p) { mono_push(m, d, p); }
  // end of a block of domains
  __device__ __forceinline__ void fold() {
    if (COMP) {
      monok_fold_in(k, m);
      m = mono_zero();
    }
  }
  __device__ __forceinline__ Mono get() {
    if (COMP) {
      fold();
      return monok_fold(k);
    }
    return m;
  }
};

__device__ __forceinline__ float sgn(float x) { return x < 0.f ? -1.f : 1.f; }

// ----------------------------------------------------------------- objectives
// The fitness the optimiser works on (qpm_objective.kind): the cascaded d_eff of Sec. 2.1
// (|d_eff|^2, maximised; the default), the SHG field of Sec. 2.1's first step (|E|^2,
// maximised), or the multi-wavelength objective of Sec. 5, sum_k |G0 - G_k| + beta
// (G_max - G_min) over K problems, G_k the cascaded or the SHG field magnitude
// (minimised).  The two single kinds share the one scan (the SHG field is
// phi(kappa1) sum_j d_j e^{-i kappa1 j}, the scan's B); the multi-wavelength kinds run K
// scans of the same vector in their own kernel variants (MK).
constexpr int OBJ_THG = 0, OBJ_SHG = 1, OBJ_MULTI_THG = 2, OBJ_MULTI_SHG = 3;

// the field of a single kind from its reduced scan
__device__ __forceinline__ float2 field_of(const InstDev &I, const Mono &m) {
  if (I.obj == OBJ_SHG) {
    const float2 ph = I.konst[3];  // phi(kappa1)
    return make_float2(ph.x * m.B.x - ph.y * m.B.y, ph.x * m.B.y + ph.y * m.B.x);
  }
  return deff_from(m, I.konst[0], I.konst[1]);
}

// selection key of fitness f of individual i: a larger key is a better individual,
// ties to the lower index (an objective to minimise is >= 0, so ~bits orders it)
__device__ __forceinline__ unsigned long long sel_key(bool minimize, float f, int i) {
  const uint32_t b = __float_as_uint(f);
  return ((unsigned long long)(minimize ? ~b : b) << 32) | (0xFFFFFFFFu - (uint32_t)i);
}

// a phasor-table entry of a multi-wavelength kind: read-only path, kept in L1 ahead of
// other lines (every team on the SM sweeps the same K tables for every individual)
__device__ __forceinline__ float4 ld_table_keep(const float4 *p) {
  float4 v;
  asm("ld.global.nc.L1::evict_last.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(p));
  return v;
}

// MK != 0: the K scans of a multi-wavelength kind, plain FP32 sums, phasors from the
// problems' tables in global memory (cached in L1 and L2)
// smt (optional): the K tables copied into shared memory by the CTA, [K][Npad] in the
// same permuted order, float4 (p1, p2) entries for the cascaded kind and float2 (p1)
// entries for the SHG kind, which needs p1 only
template <int MK>
struct MultiAcc {
  static constexpr int KMAX = MK == OBJ_MULTI_THG ? 4 : (MK == OBJ_MULTI_SHG ? 8 : 1);
  Mono m[KMAX];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < KMAX; ++k) m[k] = mono_zero();
  }
  // one domain of problem k with sign d and its phasors p (p.zw unused for SHG)
  __device__ __forceinline__ void push1(int k, float d, const float4 &p) {
    if (MK == OBJ_MULTI_THG) {
      mono_push(m[k], d, p);
    } else {  // the SHG field needs the running sum of d p1 only
      m[k].B.x = fmaf(d, p.x, m[k].B.x);
      m[k].B.y = fmaf(d, p.y, m[k].B.y);
    }
  }
  // group k4 of this thread's chunk (4 domains of signs u); one uniform branch picks
  // the tables' place for the whole group
  __device__ __forceinline__ void push4(const InstDev &I, int k4, int t, float4 u,
                                        const void *smt = nullptr) {
    const float d[4] = {sgn(u.x), sgn(u.y), sgn(u.z), sgn(u.w)};
    if (smt) {
      const int e0 = k4 * 4 * I.T + t;
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        if (k < I.K) {
          const int ek = k * I.Npad + e0;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float4 p;
            if (MK == OBJ_MULTI_SHG) {
              const float2 p1 = ((const float2 *)smt)[ek + q * I.T];
              p = make_float4(p1.x, p1.y, 0.f, 0.f);
            } else {
              p = ((const float4 *)smt)[ek + q * I.T];
            }
            push1(k, d[q], p);
          }
        }
      }
      return;
    }
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      if (k < I.K) {
        const float4 *tb = I.mtab[k] + ((uint32_t)k4 * 4u * (uint32_t)I.T + (uint32_t)t);
#pragma unroll
        for (int q = 0; q < 4; ++q) push1(k, d[q], ld_table_keep(tb + (size_t)q * I.T));
      }
    }
  }
};

// ordered warp reduction of the b-sums alone (the SHG field): the same tree and the
// same additions as warp_reduce's B
__device__ __forceinline__ float2 warp_reduce_b(float2 b) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
    const float rx = __shfl_down_sync(0xffffffffu, b.x, s);
    const float ry = __shfl_down_sync(0xffffffffu, b.y, s);
    if ((lane & (2 * s - 1)) == 0) b = make_float2(b.x + rx, b.y + ry);
  }
  return b;
}

// reduce the K scans (WT: a warp team) and form the objective: f and the first
// problem's field D0 are valid in the team's first thread; every thread returns.
// The K warp reductions are independent and run together; a CTA team then passes
// the warps' partials through shared memory once (sh holds KMAX x warps monoids)
// and its thread 0 combines them in warp order, as block_reduce does.
// Several teams per CTA (the multi-wavelength kinds with shared-memory tables): a team
// is the T consecutive threads [team T, team T + T); team_sync is the team's own
// named barrier (1 + team), a warp barrier for one-warp teams, or the CTA barrier
// when the CTA is one team.
__device__ __forceinline__ int team_thread(const InstDev &I) { return (int)threadIdx.x & (I.T - 1); }
__device__ __forceinline__ void team_sync(const InstDev &I) {
  if ((int)blockDim.x == I.T) {
    __syncthreads();
  } else if (I.T == 32) {
    __syncwarp();
  } else {
    const int team = (int)threadIdx.x / I.T;
    asm volatile("bar.sync %0, %1;" ::"r"(1 + team), "r"(I.T) : "memory");
  }
}

template <int MK, bool WT>
__device__ void multi_finish(const InstDev &I, MultiAcc<MK> &acc, Mono *sh, float &f, float2 &D0) {
  constexpr int KM = MultiAcc<MK>::KMAX;
  constexpr bool SHG = MK == OBJ_MULTI_SHG;
  const int t = WT ? (int)(threadIdx.x & 31) : team_thread(I);
#pragma unroll
  for (int k = 0; k < KM; ++k) {
    if (k < I.K) {
      if (SHG) acc.m[k].B = warp_reduce_b(acc.m[k].B);
      else acc.m[k] = warp_reduce(acc.m[k]);
    }
  }
  if (!WT) {
    // the team's warps and its share of the scratch
    const int lane = threadIdx.x & 31, warp = t >> 5, nw = I.T >> 5;
    sh += (size_t)((int)threadIdx.x / I.T) * KM * nw;
    if (nw > 1) {
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < KM; ++k)
          if (k < I.K) {
            if (SHG) sh[k * nw + warp].B = acc.m[k].B;
            else sh[k * nw + warp] = acc.m[k];
          }
      }
      team_sync(I);
      if (t == 0) {
#pragma unroll
        for (int k = 0; k < KM; ++k)
          if (k < I.K)
            for (int w = 1; w < nw; ++w) {
              const Mono &r = sh[k * nw + w];
              if (SHG) acc.m[k].B = make_float2(acc.m[k].B.x + r.B.x, acc.m[k].B.y + r.B.y);
              else acc.m[k] = mono_combine(acc.m[k], r);
            }
      }
    }
  }
  float obj = 0.f, gmax = -1.f, gmin = 3.0e38f;
  if (t == 0) {
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      if (k < I.K) {
        const Mono &mk = acc.m[k];
        float2 Dk;
        if (MK == OBJ_MULTI_THG) {
          Dk = deff_from(mk, I.mkonst[k][0], I.mkonst[k][1]);
        } else {
          const float2 ph = I.mkonst[k][3];
          Dk = make_float2(ph.x * mk.B.x - ph.y * mk.B.y, ph.x * mk.B.y + ph.y * mk.B.x);
        }
        const float G = sqrtf(fit_of(Dk));
        obj += fabsf(I.G0 - G);
        gmax = fmaxf(gmax, G);
        gmin = fminf(gmin, G);
        if (k == 0) D0 = Dk;
      }
    }
  }
  f = obj + I.beta * (gmax - gmin);
}

// push the 4 domains of group k4 of this thread's chunk
template <bool COMP, bool TS>
__device__ __forceinline__ void push4(Acc<COMP> &acc, const float4 *tbl, int T, int k4, int t,
                                      float4 u) {
  const float4 *tb = tbl + ((uint32_t)k4 * 4u * (uint32_t)T + (uint32_t)t);
  acc.push(sgn(u.x), ldt<TS>(tb));
  acc.push(sgn(u.y), ldt<TS>(tb + T));
  acc.push(sgn(u.z), ldt<TS>(tb + 2 * T));
  acc.push(sgn(u.w), ldt<TS>(tb + 3 * T));
}

__device__ __forceinline__ float *row_ptr(const InstDev &I, int i, int slot) {
  return I.pop + ((size_t)2 * i + slot) * I.Npad;
}

// float4 group `off` of individual i's current row.  DUAL: both slots are read
// together with the selector, which takes the selector load off the critical path.
template <bool NC, bool DUAL>
__device__ __forceinline__ float4 ld_cur(const InstDev &I, int i, int slot, uint32_t off) {
  if (DUAL) {
    const float *r0 = I.pop + (size_t)2 * i * I.Npad + off;
    const float4 v0 = ld4<NC>(r0), v1 = ld4<NC>(r0 + I.Npad);
    return slot ? v1 : v0;
  }
  return ld4<NC>(row_ptr(I, i, slot) + off);
}

// ---------------------------------------------------- Step 1: initialisation
template <bool COMP, int MK = 0>
__device__ void init_individual(const InstDev &I, int i, Mono *sh) {
  const int t = threadIdx.x;
  const PhiloxKey K = philox_schedule(I.key);
  float *row = row_ptr(I, i, 0);
  Acc<COMP> acc;
  acc.zero();
  MultiAcc<MK> macc;
  if (MK) macc.zero();
  for (int k4 = 0; k4 < I.c / 4; ++k4) {
    const int j0 = t * I.c + 4 * k4;
    const uint4 w = rng4(K, I.inst, TAG_INIT, GEN_INIT, (uint32_t)i, (uint32_t)(j0 >> 2));
    float4 x;
    x.x = __fsub_rn(__fmul_rn(2.0f, u24(w.x)), 1.0f);
    x.y = __fsub_rn(__fmul_rn(2.0f, u24(w.y)), 1.0f);
    x.z = __fsub_rn(__fmul_rn(2.0f, u24(w.z)), 1.0f);
    x.w = __fsub_rn(__fmul_rn(2.0f, u24(w.w)), 1.0f);
    *(float4 *)(row + ((size_t)k4 * I.T + t) * 4) = x;
    if (MK) {
      macc.push4(I, k4, t, x);
    } else {
      push4<COMP, false>(acc, I.table, I.T, k4, t, x);
      if (k4 & 1) acc.fold();
    }
  }
  float2 D = make_float2(0.f, 0.f);
  float f = 0.f;
  if constexpr (MK != 0) {
    multi_finish<MK, false>(I, macc, sh, f, D);
  } else {
    const Mono m = block_reduce(acc.get(), sh);
    if (t == 0) {
      D = field_of(I, m);
      f = fit_of(D);
    }
  }
  if (t == 0) {
    I.fit[i] = f;
    I.dval[i] = D;
    I.sel0[i] = 0;
    I.sel1[i] = 0;
    if (I.trace) I.trace[i] = f;
  }
}

template <bool COMP, int MK = 0>
static __global__ void k_init(InstDev I) {
  extern __shared__ Mono sh[];
  for (int i = blockIdx.x; i < I.NP; i += gridDim.x) {
    if (i != (int)blockIdx.x) __syncthreads();  // the reduction scratch is reused
    init_individual<COMP, MK>(I, i, sh);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *I.gen = 0;
    for (int k = 0; k < 4; ++k) I.ctr[k] = 0u;
  }
}

// ------------------------------------------------------------- row staging
// Row staging (STG): the four rows an update reads (own + three donors or leaders)
// and, when the phasor table is not in shared memory (!TS), the group's four table
// entries are copied ahead into shared memory with cp.async, so the next group's
// loads are in flight during this group's arithmetic without holding registers.
// Two stages (one group ahead): a third stage, measured where the table comes from
// global memory, sped the memory-bound DE phase up by 2 % and slowed the GWO phase
// down by 7 %.  Each thread owns its slots
// stg[(stage * SPS + k) * blockDim.x + threadIdx.x] (SPS = 4 rows, + 4 table
// entries when !TS) and reads back only what it copied itself, so no barrier is
// needed.
__host__ __device__ constexpr int stg_stages(bool) { return 2; }
__host__ __device__ constexpr int stg_f4_per_thread(bool ts) {
  return stg_stages(ts) * (ts ? 4 : 8);
}
// copies of group k (4 domains: rows at float offset ((k T + t) 4), table entries
// tbl[(4 k + q) T + t]) into stage `stage`
template <bool TS>
__device__ __forceinline__ void stage_group(float4 *stg, int stage, int k, int T, int t,
                                            const float *r0, const float *r1, const float *r2,
                                            const float *r3, const float4 *tbl) {
  constexpr int SPS = stg_f4_per_thread(TS) / stg_stages(TS);
  const int nt = blockDim.x;
  const uint32_t off = ((uint32_t)k * (uint32_t)T + (uint32_t)t) * 4u;
  float4 *s = stg + ((uint32_t)(stage * SPS * nt) + threadIdx.x);
  cp_async16(s, r0 + off);
  cp_async16(s + nt, r1 + off);
  cp_async16(s + 2 * nt, r2 + off);
  cp_async16(s + 3 * nt, r3 + off);
  if (!TS) {
    const float4 *tb = tbl + ((uint32_t)k * 4u * (uint32_t)T + (uint32_t)t);
    cp_async16(s + 4 * nt, tb);
    cp_async16(s + 5 * nt, tb + T);
    cp_async16(s + 6 * nt, tb + 2 * T);
    cp_async16(s + 7 * nt, tb + 3 * T);
  }
}
// before the loop: groups 0 .. NS - 2, one commit group each (possibly empty)
template <bool TS>
__device__ __forceinline__ void stage_prologue(float4 *stg, int n4, int T, int t, const float *r0,
                                               const float *r1, const float *r2, const float *r3,
                                               const float4 *tbl) {
#pragma unroll
  for (int k = 0; k < stg_stages(TS) - 1; ++k) {
    if (k < n4) stage_group<TS>(stg, k, k, T, t, r0, r1, r2, r3, tbl);
    cp_async_commit();
  }
}
// group k4: commits the copies of group k4 + NS - 1 first when there is one, waits
// until group k4 has landed and returns this thread's stage base (rows at
// [0, 4 nt), table entries at [4 nt, 8 nt) if !TS)
template <bool TS>
__device__ __forceinline__ const float4 *staged_group(float4 *stg, int k4, int n4, int T, int t,
                                                      const float *r0, const float *r1,
                                                      const float *r2, const float *r3,
                                                      const float4 *tbl) {
  constexpr int NS = stg_stages(TS), SPS = stg_f4_per_thread(TS) / NS;
  const int kn = k4 + NS - 1;
  if (kn < n4) stage_group<TS>(stg, kn % NS, kn, T, t, r0, r1, r2, r3, tbl);
  cp_async_commit();  // possibly empty: keeps one group per iteration
  cp_async_wait<NS - 1>();
  return stg + ((uint32_t)((k4 % NS) * SPS) * blockDim.x + threadIdx.x);
}
// the push of one staged group: table entries from the stage when !TS
template <bool COMP, bool TS>
__device__ __forceinline__ void push4_staged(Acc<COMP> &acc, const float4 *tbl, int T, int k4,
                                             int t, const float4 *st, float4 u) {
  if (TS) push4<COMP, true>(acc, tbl, T, k4, t, u);
  else push4<COMP, true>(acc, st + 4 * blockDim.x, blockDim.x, 0, 0, u);
}

// ------------------------------------------ Step 2: DE rand/1/bin + selection
// returns (in thread 0) the key of the survivor for the leader choice
// WT: the team is one warp (t = lane, warp reduction) instead of the whole CTA
// r = (r1, r2, r3, jrand) from de_indices
// STG: rows staged through stg (known slots only, so not with DUAL)
// has_wcr: wcr is the crossover word of the thread's first group of 4 domains, drawn
// earlier (while waiting at the grid barrier)
template <bool COMP, bool NC, bool TS, bool DUAL, bool WT = false, bool STG = false, int MK = 0>
__device__ unsigned long long de_individual(const InstDev &I, const PhiloxKey &K,
                                            const float4 *tbl, int g, int i, const int4 r,
                                            const int32_t *sel_in, int32_t *sel_out, Mono *sh,
                                            int *slot_out = nullptr, float4 *stg = nullptr,
                                            bool has_wcr = false,
                                            uint4 wcr = make_uint4(0u, 0u, 0u, 0u),
                                            int own_slot = -1, int *impr_out = nullptr,
                                            const void *smt = nullptr) {
  static_assert(!(STG && DUAL), "staged rows need known slots");
  // only the multi-wavelength kinds put several teams in a CTA
  const int t = WT ? (int)(threadIdx.x & 31) : (MK ? team_thread(I) : (int)threadIdx.x);
  const float fx = (t == 0) ? I.fit[i] : 0.f;  // issued early, used after the scan
  // own_slot >= 0: the individual's current slot, known to the caller
  const int si = own_slot >= 0 ? own_slot : sel_in[i];
  const int s1 = sel_in[r.x], s2 = sel_in[r.y], s3 = sel_in[r.z];
  float *out = row_ptr(I, i, si ^ 1);
  const float F = I.Fsched ? I.Fsched[g] : I.F;
  const uint32_t crthr = I.crthr;
  const int n4 = I.c / 4;
  const float *ra = row_ptr(I, i, si), *rb = row_ptr(I, r.x, s1);
  const float *rp = row_ptr(I, r.y, s2), *rq = row_ptr(I, r.z, s3);
  if (STG) stage_prologue<TS>(stg, n4, I.T, t, ra, rb, rp, rq, tbl);
  Acc<COMP> acc;
  acc.zero();
  MultiAcc<MK> macc;
  if (MK) macc.zero();
  for (int k4 = 0; k4 < n4; ++k4) {
    const uint32_t off = ((uint32_t)k4 * (uint32_t)I.T + (uint32_t)t) * 4u;
    float4 a, b, p, q;
    const float4 *st = nullptr;
    if (STG) {
      st = staged_group<TS>(stg, k4, n4, I.T, t, ra, rb, rp, rq, tbl);
      const int nt = blockDim.x;
      a = st[0];
      b = st[nt];
      p = st[2 * nt];
      q = st[3 * nt];
    } else {
      a = ld_cur<NC, DUAL>(I, i, si, off);
      b = ld_cur<NC, DUAL>(I, r.x, s1, off);
      p = ld_cur<NC, DUAL>(I, r.y, s2, off);
      q = ld_cur<NC, DUAL>(I, r.z, s3, off);
    }
    const int j0 = t * I.c + 4 * k4;
    const uint4 w = (has_wcr && k4 == 0)
                        ? wcr
                        : rng4(K, I.inst, TAG_CR, (uint32_t)g, (uint32_t)i, (uint32_t)(j0 >> 2));
    float4 u;
    // v = fl(x_r1 + fl(F fl(x_r2 - x_r3))) (no FMA), clamped;
    // u = v if U <= CR (integer form) or j == jrand, else x
#define QPM_DE1(C, W, J)                                                              \
    {                                                                                 \
      const float v = clamp1(__fadd_rn(b.C, __fmul_rn(F, __fsub_rn(p.C, q.C))));      \
      u.C = (w.W <= crthr || (J) == r.w) ? v : a.C;                                   \
    }
    QPM_DE1(x, x, j0)
    QPM_DE1(y, y, j0 + 1)
    QPM_DE1(z, z, j0 + 2)
    QPM_DE1(w, w, j0 + 3)
#undef QPM_DE1
    *(float4 *)(out + off) = u;
    if (MK) {
      macc.push4(I, k4, t, u, smt);
    } else {
      if (STG) push4_staged<COMP, TS>(acc, tbl, I.T, k4, t, st, u);
      else push4<COMP, TS>(acc, tbl, I.T, k4, t, u);
      if (k4 & 1) acc.fold();
    }
  }
  float2 D = make_float2(0.f, 0.f);
  float f = 0.f;
  if constexpr (MK != 0) {
    multi_finish<MK, WT>(I, macc, sh, f, D);
  } else {
    // a single group of 4 domains per thread needs no compensation (its plain sums are
    // what the fold would return, up to the sign of a zero), and skipping the fold
    // takes a dependent chain off the phase's critical path
    const Mono mine = (COMP && !WT && n4 == 1) ? acc.m : acc.get();
    const Mono m = WT ? warp_reduce(mine) : block_reduce(mine, sh);
    if (t == 0) {
      D = field_of(I, m);
      f = fit_of(D);
    }
  }
  unsigned long long key = 0ull;
  if (t == 0) {
    // greedy one-to-one selection: maximising, or minimising the multi-wavelength kinds
    const bool accept = MK ? (f <= fx) : (f >= fx);
    sel_out[i] = accept ? (si ^ 1) : si;
    if (accept) {
      I.fit[i] = f;
      I.dval[i] = D;
    }
    if (I.trace) I.trace[(size_t)I.NP * (1 + 2 * (size_t)g) + i] = f;
    key = sel_key(MK != 0, accept ? f : fx, i);
    if (slot_out) *slot_out = accept ? (si ^ 1) : si;  // the survivor's slot
    if (impr_out) *impr_out = MK ? (f < fx) : (f > fx);  // a strict improvement (adaptive F)
  }
  return key;
}

// ------------------------------------------------ Step 4-5: GWO + selection
// PRE: the three GWO random words of the thread's first group of 4 domains were
// drawn earlier (while waiting at the grid barrier) and are passed in wpre.
// One word per leader and gene gives that leader's (r1, r2) as its 16-bit halves.
template <bool COMP, bool NC, bool TS, bool DUAL, bool WT = false, bool PRE = false,
          bool STG = false, int MK = 0>
__device__ void gwo_individual(const InstDev &I, const PhiloxKey &K, const float4 *tbl, int g,
                               int i, int32_t *sel, int la, int lb, int ld, Mono *sh,
                               const uint4 *wpre = nullptr,
                               float4 own0 = make_float4(0.f, 0.f, 0.f, 0.f),
                               float4 own1 = make_float4(0.f, 0.f, 0.f, 0.f),
                               const int32_t *lslot = nullptr, float4 *stg = nullptr,
                               int own_slot = -1, int *slot_out = nullptr,
                               const void *smt = nullptr) {
  static_assert(!(STG && (DUAL || PRE)), "staged rows need known slots and no prefetched row");
  // only the multi-wavelength kinds put several teams in a CTA
  const int t = WT ? (int)(threadIdx.x & 31) : (MK ? team_thread(I) : (int)threadIdx.x);
  const float fx = (t == 0) ? I.fit[i] : 0.f;
  // lslot: the leaders' current slots, when the leader search delivered them;
  // own_slot >= 0: the individual's current slot, known to the caller
  const int si = own_slot >= 0 ? own_slot : sel[i];
  const int sa = lslot ? lslot[0] : sel[la], sb = lslot ? lslot[1] : sel[lb];
  const int sd = lslot ? lslot[2] : sel[ld];
  float *out = row_ptr(I, i, si ^ 1);
  const float a = __fdiv_rn((float)(2 * (I.G - g)), (float)I.G);
  const float two_a = __fmul_rn(2.0f, a);
  const int n4 = I.c / 4;
  const float *rx = row_ptr(I, i, si), *r0 = row_ptr(I, la, sa), *r1 = row_ptr(I, lb, sb);
  const float *r2 = row_ptr(I, ld, sd);
  if (STG) stage_prologue<TS>(stg, n4, I.T, t, rx, r0, r1, r2, tbl);
  Acc<COMP> acc;
  acc.zero();
  MultiAcc<MK> macc;
  if (MK) macc.zero();
  for (int k4 = 0; k4 < n4; ++k4) {
    const uint32_t off = ((uint32_t)k4 * (uint32_t)I.T + (uint32_t)t) * 4u;
    float4 x, L0, L1, L2;
    const float4 *st = nullptr;
    if (STG) {
      st = staged_group<TS>(stg, k4, n4, I.T, t, rx, r0, r1, r2, tbl);
      const int nt = blockDim.x;
      x = st[0];
      L0 = st[nt];
      L1 = st[2 * nt];
      L2 = st[3 * nt];
    } else {
      x = (PRE && k4 == 0) ? (si ? own1 : own0) : ld_cur<NC, DUAL>(I, i, si, off);
      // a known slot needs one row read, not both
      L0 = lslot ? ld_cur<NC, false>(I, la, sa, off) : ld_cur<NC, DUAL>(I, la, sa, off);
      L1 = lslot ? ld_cur<NC, false>(I, lb, sb, off) : ld_cur<NC, DUAL>(I, lb, sb, off);
      L2 = lslot ? ld_cur<NC, false>(I, ld, sd, off) : ld_cur<NC, DUAL>(I, ld, sd, off);
    }
    const uint32_t jg = (uint32_t)((t * I.c + 4 * k4) >> 2);
    uint4 w[3];
    if (PRE && k4 == 0) {
#pragma unroll
      for (int k = 0; k < 3; ++k) w[k] = wpre[k];
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k) w[k] = rng4(K, I.inst, TAG_GWO + k, (uint32_t)g, (uint32_t)i, jg);
    }
    float4 y;
    // A = fl(fl(2a r1) - a), C = 2 r2, D = |fl(fl(C Xp) - x)|, Y = fl(Xp - fl(A D)),
    // in this order, no FMA
#define QPM_PULL(Xp, xv, rw, out_)                                                     \
    {                                                                                  \
      const float A = __fsub_rn(__fmul_rn(two_a, u16hi(rw)), a);                        \
      const float C = twice_u16lo(rw);                                                  \
      const float dist = fabsf(__fsub_rn(__fmul_rn(C, Xp), xv));                        \
      out_ = __fsub_rn(Xp, __fmul_rn(A, dist));                                         \
    }
#define QPM_GWO1(CMP)                                                                  \
    {                                                                                  \
      float Y0, Y1, Y2;                                                                \
      QPM_PULL(L0.CMP, x.CMP, w[0].CMP, Y0)                                            \
      QPM_PULL(L1.CMP, x.CMP, w[1].CMP, Y1)                                            \
      QPM_PULL(L2.CMP, x.CMP, w[2].CMP, Y2)                                            \
      float v;                                                                         \
      if (I.combine == 0) {                                                            \
        v = div3_rn(__fadd_rn(__fadd_rn(Y0, Y1), Y2));                                \
      } else {                                                                         \
        const float m0 = fabsf(Y0), m1 = fabsf(Y1), m2 = fabsf(Y2);                    \
        const float s = __fadd_rn(__fadd_rn(m0, m1), m2);                              \
        const float num = __fadd_rn(__fadd_rn(__fmul_rn(m0, Y0), __fmul_rn(m1, Y1)),   \
                                    __fmul_rn(m2, Y2));                                \
        v = (s == 0.0f) ? 0.0f : __fdiv_rn(num, __fmul_rn(3.0f, s));                   \
      }                                                                                \
      y.CMP = clamp1(v);                                                               \
    }
    QPM_GWO1(x)
    QPM_GWO1(y)
    QPM_GWO1(z)
    QPM_GWO1(w)
#undef QPM_GWO1
#undef QPM_PULL
    *(float4 *)(out + off) = y;
    if (MK) {
      macc.push4(I, k4, t, y, smt);
    } else {
      if (STG) push4_staged<COMP, TS>(acc, tbl, I.T, k4, t, st, y);
      else push4<COMP, TS>(acc, tbl, I.T, k4, t, y);
      if (k4 & 1) acc.fold();
    }
  }
  float2 D = make_float2(0.f, 0.f);
  float f = 0.f;
  if constexpr (MK != 0) {
    multi_finish<MK, WT>(I, macc, sh, f, D);
  } else {
    // a single group of 4 domains per thread needs no compensation (its plain sums are
    // what the fold would return, up to the sign of a zero), and skipping the fold
    // takes a dependent chain off the phase's critical path
    const Mono mine = (COMP && !WT && n4 == 1) ? acc.m : acc.get();
    const Mono m = WT ? warp_reduce(mine) : block_reduce(mine, sh);
    if (t == 0) {
      D = field_of(I, m);
      f = fit_of(D);
    }
  }
  if (t == 0) {
    const bool accept = MK ? (f <= fx) : (f >= fx);
    if (accept) {
      sel[i] = si ^ 1;
      I.fit[i] = f;
      I.dval[i] = D;
    }
    if (I.trace) I.trace[(size_t)I.NP * (2 + 2 * (size_t)g) + i] = f;
    if (slot_out) *slot_out = accept ? (si ^ 1) : si;  // the survivor's slot
  }
}

// The keys carry the survivor's slot and whether its trial strictly improved on the
// target: fitness bits << 32 | (0x3FFFFFFF - i) << 2 | improved << 1 | slot, which
// orders like lead_key (the two low bits never separate two individuals).
__device__ __forceinline__ unsigned long long slot_key(unsigned long long key, int i, int slot,
                                                       int improved = 0) {
  return (key & 0xFFFFFFFF00000000ull) |
         (unsigned long long)(((0x3FFFFFFFu - (uint32_t)i) << 2) | ((uint32_t)improved << 1) |
                              (uint32_t)slot);
}
__device__ __forceinline__ int slot_key_index(unsigned long long k) {
  return (int)(0x3FFFFFFFu - ((uint32_t)k >> 2));
}

// ------------------------------------------------------------- adaptive F
// Sec. 3.1.1's adaptive F (f_schedule 2).  The paper keeps F in [0.01, 0.1], raises it
// when the population's diversity is low (standard deviation below a threshold, or a
// convergence rate below 0.1), lowers it when diversity is too high or the fitness
// range small (deviation above a threshold, or range below 10^3), and otherwise lets
// it follow the cosine-times-quadratic decay.  Readings (the paper gives neither the
// thresholds nor the steps): after the DE phase of generation g, over the DE survivors,
// cv = the fitness' standard deviation over its mean, the convergence rate = the
// fraction of trials that strictly improved on their target; cv < 0.05 or a rate below
// 0.1 raises F to min(0.1, 1.25 F); cv > 0.5 or max f - min f < 10^3 lowers it to
// max(0.01, 0.8 F); otherwise F = Fbase[g + 1] = 0.1 (cos(pi (g+1) / 2G) + 1) / 2
// (1 - 0.2 ((g+1)/G)^2).  The decision uses exact integer statistics, so that it does
// not depend on a summation order: with E such that 2^(E-1) <= max f < 2^E, every
// fitness is quantised to n = floor(f 2^(20 - E)) by shifting its significand, and
// S1 = sum n, S2 = sum n^2 are 64-bit integers (NP <= 2^23); cv^2 < t^2 is tested as
// NP S2 - S1^2 < t^2 S1^2 with every FP64 operation rounded once.
constexpr float AF_FMIN = 0.01f, AF_FMAX = 0.1f, AF_UP = 1.25f, AF_DOWN = 0.8f;

// n = floor(f 2^(20 - E)) for the fitness bits fb (f >= 0) and the exponent field emax
// (>= 1) of the largest fitness: f = m 2^(e - 150), m the 24-bit significand
__device__ __forceinline__ uint32_t af_quantise(uint32_t fb, uint32_t emax) {
  uint32_t e = (fb >> 23) & 0xFFu, m = fb & 0x7FFFFFu;
  if (e == 0) e = 1;
  else m |= 0x800000u;
  const uint32_t sh = 4u + emax - e;
  return sh >= 24u ? 0u : m >> sh;
}

// F of generation g + 1 from the survivor keys of generation g (slot_key layout), by
// every thread of one CTA; thread 0 writes it to I.Fsched[g + 1].  Every thread returns
// after a CTA barrier.
__device__ void adaptive_F_block(const InstDev &I, const unsigned long long *keys, int g) {
  __shared__ uint32_t red_u[3][32];
  __shared__ unsigned long long red_s[2][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t mx = 0u, mn = 0xFFFFFFFFu, cnt = 0u;
  for (int i = threadIdx.x; i < I.NP; i += blockDim.x) {
    const unsigned long long k = keys[i];
    const uint32_t fb = I.minimize ? ~(uint32_t)(k >> 32) : (uint32_t)(k >> 32);  // f's bits
    mx = max(mx, fb);
    mn = min(mn, fb);
    cnt += ((uint32_t)k >> 1) & 1u;
  }
  mx = __reduce_max_sync(0xffffffffu, mx);
  mn = __reduce_min_sync(0xffffffffu, mn);
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if (lane == 0) {
    red_u[0][warp] = mx;
    red_u[1][warp] = mn;
    red_u[2][warp] = cnt;
  }
  __syncthreads();
  mx = 0u;
  mn = 0xFFFFFFFFu;
  cnt = 0u;
  for (int w = 0; w < nw; ++w) {
    mx = max(mx, red_u[0][w]);
    mn = min(mn, red_u[1][w]);
    cnt += red_u[2][w];
  }
  uint32_t emax = (mx >> 23) & 0xFFu;
  if (emax == 0) emax = 1;
  unsigned long long s1 = 0ull, s2 = 0ull;
  for (int i = threadIdx.x; i < I.NP; i += blockDim.x) {
    const uint32_t hi = (uint32_t)(keys[i] >> 32);
    const uint32_t n = af_quantise(I.minimize ? ~hi : hi, emax);
    s1 += n;
    s2 += (unsigned long long)n * n;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (lane == 0) {
    red_s[0][warp] = s1;
    red_s[1][warp] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s1 = s2 = 0ull;
    for (int w = 0; w < nw; ++w) {
      s1 += red_s[0][w];
      s2 += red_s[1][w];
    }
    const double a = __dmul_rn((double)I.NP, (double)s2);
    const double b = __dmul_rn((double)s1, (double)s1);
    const double num = __dsub_rn(a, b);
    const float range = __fsub_rn(__uint_as_float(mx), __uint_as_float(mn));
    const bool low = (s1 == 0ull) || (num < __dmul_rn(0.0025, b)) ||
                     (10ull * cnt < (unsigned long long)I.NP);
    const bool high = !low && ((num > __dmul_rn(0.25, b)) || (range < 1000.0f));
    const float Fg = I.Fsched[g];
    I.Fsched[g + 1] = low ? fminf(AF_FMAX, __fmul_rn(Fg, AF_UP))
                          : (high ? fmaxf(AF_FMIN, __fmul_rn(Fg, AF_DOWN)) : I.Fbase[g + 1]);
  }
  __syncthreads();
}

// ------------------------------------------- four-leader discrete GWO (Sec. 3.1.2)
// The paper describes it only qualitatively (continuous positions mapped to +-1; state
// transitions from the four leaders' state distribution with a dispersion parameter;
// much disturbance early, the dominant state and rare flips late; a falling social-
// learning rate that copies a random leader).  Reading, per omega wolf and gene, with
// n the number of the four leaders whose gene is +1 and tau = g / G: with probability
// sigma = 0.3 (1 - tau) take leader kl's state (kl uniform in 0..3), else +1 with
// probability P_n = (1 - delta) q_n + delta / 2, delta = 0.5 (1 - tau),
// q_n = (1 - tau) n / 4 + tau [n > 2, or 1/2 for n = 2]; then flip with probability
// mu = 0.1 (1 - tau) + 0.01 tau.  The probabilities are 16-bit thresholds per
// generation (computed on the host in FP64, I.dthr), tested against the 16-bit halves
// of two words per gene (tag GWO: social high, transition low; tag GWO + 1: flip high,
// kl the low two bits).  The new genes are +-1.
__device__ __forceinline__ void top4_insert(unsigned long long &k0, unsigned long long &k1,
                                            unsigned long long &k2, unsigned long long &k3,
                                            unsigned long long x) {
  if (x > k0) { k3 = k2; k2 = k1; k1 = k0; k0 = x; }
  else if (x > k1) { k3 = k2; k2 = k1; k1 = x; }
  else if (x > k2) { k3 = k2; k2 = x; }
  else if (x > k3) { k3 = x; }
}

// the generation's thresholds: social, flip, and P(+1) for 0 .. 4 leaders at +1
struct DiscThr {
  uint32_t soc, flip, p0, p1, p2, p3, p4;
};

// the new state of one gene from the four leaders' genes and the two random words
__device__ __forceinline__ float disc_gene(float a, float b, float c, float d, uint32_t w1,
                                           uint32_t w2, const DiscThr &th) {
  const float s0 = sgn(a), s1 = sgn(b), s2 = sgn(c), s3 = sgn(d);
  const int n = (s0 > 0.f) + (s1 > 0.f) + (s2 > 0.f) + (s3 > 0.f);
  const uint32_t kl = w2 & 3u;
  float v;
  if ((w1 >> 16) < th.soc) {  // social learning: a random leader's state
    v = kl == 0u ? s0 : (kl == 1u ? s1 : (kl == 2u ? s2 : s3));
  } else {  // transition from the leaders' state distribution
    const uint32_t tp = n == 0 ? th.p0 : (n == 1 ? th.p1 : (n == 2 ? th.p2 : (n == 3 ? th.p3 : th.p4)));
    v = (w1 & 0xFFFFu) < tp ? 1.f : -1.f;
  }
  return (w2 >> 16) < th.flip ? -v : v;  // disturbance
}

// one candidate of the discrete GWO for omega wolf i and its greedy selection, by the
// CTA (team T); L: the four leaders' current rows
template <bool COMP>
__device__ void gwo_discrete_individual(const InstDev &I, const PhiloxKey &K, int g, int i,
                                        int32_t *sel, const float *L0, const float *L1,
                                        const float *L2, const float *L3, Mono *sh) {
  const int t = threadIdx.x;
  const float fx = (t == 0) ? I.fit[i] : 0.f;
  const int si = sel[i];
  float *out = row_ptr(I, i, si ^ 1);
  const uint32_t *tg = I.dthr + (size_t)7 * g;
  const DiscThr th{tg[0], tg[1], tg[2], tg[3], tg[4], tg[5], tg[6]};
  Acc<COMP> acc;
  acc.zero();
  const int n4 = I.c / 4;
  for (int k4 = 0; k4 < n4; ++k4) {
    const uint32_t off = ((uint32_t)k4 * (uint32_t)I.T + (uint32_t)t) * 4u;
    const float4 l0 = __ldg((const float4 *)(L0 + off)), l1 = __ldg((const float4 *)(L1 + off));
    const float4 l2 = __ldg((const float4 *)(L2 + off)), l3 = __ldg((const float4 *)(L3 + off));
    const uint32_t jg = (uint32_t)((t * I.c + 4 * k4) >> 2);
    const uint4 w1 = rng4(K, I.inst, TAG_GWO, (uint32_t)g, (uint32_t)i, jg);
    const uint4 w2 = rng4(K, I.inst, TAG_GWO + 1, (uint32_t)g, (uint32_t)i, jg);
    float4 y;
    y.x = disc_gene(l0.x, l1.x, l2.x, l3.x, w1.x, w2.x, th);
    y.y = disc_gene(l0.y, l1.y, l2.y, l3.y, w1.y, w2.y, th);
    y.z = disc_gene(l0.z, l1.z, l2.z, l3.z, w1.z, w2.z, th);
    y.w = disc_gene(l0.w, l1.w, l2.w, l3.w, w1.w, w2.w, th);
    *(float4 *)(out + off) = y;
    push4<COMP, false>(acc, I.table, I.T, k4, t, y);
    if (k4 & 1) acc.fold();
  }
  const Mono m = block_reduce(acc.get(), sh);
  if (t == 0) {
    const float2 D = field_of(I, m);
    const float f = fit_of(D);
    const bool accept = f >= fx;
    if (accept) {
      sel[i] = si ^ 1;
      I.fit[i] = f;
      I.dval[i] = D;
    }
    if (I.trace) I.trace[(size_t)I.NP * (2 + 2 * (size_t)g) + i] = f;
  }
}

// top-3 merge over the CTA: every thread passes its sorted triple, thread 0 gets the result
__device__ void block_top3(unsigned long long &k0, unsigned long long &k1, unsigned long long &k2,
                           unsigned long long *sh) {
  for (int s = 16; s > 0; s >>= 1) {
    const unsigned long long p0 = __shfl_xor_sync(0xffffffffu, k0, s);
    const unsigned long long p1 = __shfl_xor_sync(0xffffffffu, k1, s);
    const unsigned long long p2 = __shfl_xor_sync(0xffffffffu, k2, s);
    top3_insert(k0, k1, k2, p0);
    top3_insert(k0, k1, k2, p1);
    top3_insert(k0, k1, k2, p2);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) {
    sh[3 * warp] = k0;
    sh[3 * warp + 1] = k1;
    sh[3 * warp + 2] = k2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w) {
      top3_insert(k0, k1, k2, sh[3 * w]);
      top3_insert(k0, k1, k2, sh[3 * w + 1]);
      top3_insert(k0, k1, k2, sh[3 * w + 2]);
    }
  }
  __syncthreads();
}

// merge all per-CTA partial triples in topk[0 .. 3*nparts) into the leaders; warp 0
// does the work, every thread returns after the CTA barrier (thread 0 writes lead)
__device__ void merge_leaders(const unsigned long long *topk, int nparts, int32_t *lead,
                              int32_t *lead_sh) {
  if (threadIdx.x < 32) {
    unsigned long long k0 = 0, k1 = 0, k2 = 0;
    for (int e = threadIdx.x; e < 3 * nparts; e += 32) top3_insert(k0, k1, k2, topk[e]);
    for (int s = 16; s > 0; s >>= 1) {
      const unsigned long long p0 = __shfl_xor_sync(0xffffffffu, k0, s);
      const unsigned long long p1 = __shfl_xor_sync(0xffffffffu, k1, s);
      const unsigned long long p2 = __shfl_xor_sync(0xffffffffu, k2, s);
      top3_insert(k0, k1, k2, p0);
      top3_insert(k0, k1, k2, p1);
      top3_insert(k0, k1, k2, p2);
    }
    if (threadIdx.x == 0) {
      const int l0 = key_index(k0), l1 = key_index(k1), l2 = key_index(k2);
      if (lead) { lead[0] = l0; lead[1] = l1; lead[2] = l2; }
      if (lead_sh) { lead_sh[0] = l0; lead_sh[1] = l1; lead_sh[2] = l2; }
    }
  }
  __syncthreads();
}

// the same for four leaders (the discrete GWO): topk holds 4 keys per part
__device__ void merge_leaders4(const unsigned long long *topk, int nparts, int32_t *lead) {
  if (threadIdx.x < 32) {
    unsigned long long k0 = 0, k1 = 0, k2 = 0, k3 = 0;
    for (int e = threadIdx.x; e < 4 * nparts; e += 32) top4_insert(k0, k1, k2, k3, topk[e]);
    for (int s = 16; s > 0; s >>= 1) {
      const unsigned long long p0 = __shfl_xor_sync(0xffffffffu, k0, s);
      const unsigned long long p1 = __shfl_xor_sync(0xffffffffu, k1, s);
      const unsigned long long p2 = __shfl_xor_sync(0xffffffffu, k2, s);
      const unsigned long long p3 = __shfl_xor_sync(0xffffffffu, k3, s);
      top4_insert(k0, k1, k2, k3, p0);
      top4_insert(k0, k1, k2, k3, p1);
      top4_insert(k0, k1, k2, k3, p2);
      top4_insert(k0, k1, k2, k3, p3);
    }
    if (threadIdx.x == 0) {
      lead[0] = key_index(k0);
      lead[1] = key_index(k1);
      lead[2] = key_index(k2);
      lead[3] = key_index(k3);
    }
  }
  __syncthreads();
}

// true in every thread of the last CTA to finish (classic fence + counter pattern)
__device__ bool last_cta(unsigned *ctr) {
  __shared__ bool is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(ctr, 1u);
    is_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// dynamic shared memory of k_de and k_gwo: [row + table staging (long rows)][reduction]
// The multi-wavelength kinds (MK) stage the rows only: their K phasor tables are read
// through L1, which keeps them (the rows bypass it).
template <bool COMP, bool DUAL, int MK = 0>
static __global__ void k_de(InstDev I) {
  constexpr bool STG = !DUAL, TSS = MK != 0;
  extern __shared__ float4 dyn[];
  float4 *stg = dyn;
  Mono *sh = (Mono *)(dyn + (STG ? stg_f4_per_thread(TSS) * blockDim.x : 0));
  const int g = *I.gen;
  const PhiloxKey K = philox_schedule(I.key);
  const int32_t *sel_in = (g & 1) ? I.sel1 : I.sel0;
  int32_t *sel_out = (g & 1) ? I.sel0 : I.sel1;
  const bool four = I.combine == 2;  // the discrete GWO's four leaders
  unsigned long long k0 = 0, k1 = 0, k2 = 0, k3 = 0;
  for (int i = blockIdx.x; i < I.NP; i += gridDim.x) {
    if (i != (int)blockIdx.x) __syncthreads();  // the reduction scratch is reused
    int slot = 0, impr = 0;
    const unsigned long long key =
        de_individual<COMP, true, TSS, DUAL, false, STG, MK>(
            I, K, I.table, g, i, de_indices(K, I.inst, (uint32_t)g, i, I.NP, I.N), sel_in, sel_out, sh,
            &slot, stg, false, make_uint4(0u, 0u, 0u, 0u), -1, &impr);
    if (threadIdx.x == 0) {
      if (four) top4_insert(k0, k1, k2, k3, key);
      else top3_insert(k0, k1, k2, key);
      if (I.adaptive) I.dekey[i] = slot_key(key, i, slot, impr);
    }
  }
  if (threadIdx.x == 0) {
    if (four) {
      I.topk[4 * blockIdx.x] = k0;
      I.topk[4 * blockIdx.x + 1] = k1;
      I.topk[4 * blockIdx.x + 2] = k2;
      I.topk[4 * blockIdx.x + 3] = k3;
    } else {
      I.topk[3 * blockIdx.x] = k0;
      I.topk[3 * blockIdx.x + 1] = k1;
      I.topk[3 * blockIdx.x + 2] = k2;
    }
  }
  if (last_cta(&I.ctr[0])) {
    if (four) merge_leaders4(I.topk, gridDim.x, I.lead);  // Step 3
    else merge_leaders(I.topk, gridDim.x, I.lead, nullptr);
    if (I.adaptive) adaptive_F_block(I, I.dekey, g);     // Step 6: the next F
    if (threadIdx.x == 0) I.ctr[0] = 0u;
  }
}

template <bool COMP, bool DUAL, int MK = 0>
static __global__ void k_gwo(InstDev I) {
  constexpr bool STG = !DUAL, TSS = MK != 0;
  extern __shared__ float4 dyn[];
  float4 *stg = dyn;
  Mono *sh = (Mono *)(dyn + (STG ? stg_f4_per_thread(TSS) * blockDim.x : 0));
  const int g = *I.gen;
  const PhiloxKey K = philox_schedule(I.key);
  int32_t *sel = (g & 1) ? I.sel0 : I.sel1;
  const int la = I.lead[0], lb = I.lead[1], ld = I.lead[2];
  for (int i = blockIdx.x; i < I.NP; i += gridDim.x) {
    if (i == la || i == lb || i == ld) continue;  // the leaders do not move
    __syncthreads();  // the reduction scratch is reused
    gwo_individual<COMP, true, TSS, DUAL, false, false, STG, MK>(
        I, K, I.table, g, i, sel, la, lb, ld, sh, nullptr, make_float4(0.f, 0.f, 0.f, 0.f),
        make_float4(0.f, 0.f, 0.f, 0.f), nullptr, stg);
  }
  if (I.trace && blockIdx.x == 0 && threadIdx.x < 3) {
    const int l = threadIdx.x == 0 ? la : (threadIdx.x == 1 ? lb : ld);
    I.trace[(size_t)I.NP * (2 + 2 * (size_t)g) + l] = __int_as_float(0x7fc00000);
  }
  if (last_cta(&I.ctr[1])) {
    if (threadIdx.x == 0) {
      *I.gen = g + 1;  // Step 6/7: next generation (a is derived from g)
      I.ctr[1] = 0u;
    }
  }
}

// ------------------------------- the multi-wavelength kinds, tables in shared memory
// When their K tables fit, the multi-wavelength kinds run several teams of T threads
// per CTA (threads [team T, team T + T) are the team of one individual, with its own
// named barrier, or none for one-warp teams) so that one copy of the K tables in
// shared memory serves every team
// on the SM: read through L1, the tables of three N = 3000 problems (147 KB) did not
// stay there.  The cascaded kind keeps (p1, p2) per domain, the SHG kind p1 only.
// Dynamic shared memory: [K tables][row staging][reduction scratch of every team].
// Teams take individuals from a counter (ctr[2] in DE, ctr[3] in GWO, reset by the
// phase's last CTA), so that every SM ends within about one individual of the others
// (a fixed deal of 5000 individuals to 152 x 8 teams leaves the fifth round 11 % full).
// Which team evaluates an individual does not change any result.
__device__ __forceinline__ int mt_next(const InstDev &I, unsigned *ctr, int &cur) {
  __shared__ int next_sh[16];
  const int team = (int)threadIdx.x / I.T;
  if (team_thread(I) == 0) next_sh[team] = cur;
  team_sync(I);  // also: the previous individual's reduction scratch is free again
  const int i = next_sh[team];
  // the one after, requested while this one is evaluated
  if (i < I.NP && team_thread(I) == 0) cur = (int)atomicAdd(ctr, 1u);
  return i;
}

template <int MK>
__host__ __device__ constexpr size_t mt_entry_bytes() {
  return MK == OBJ_MULTI_SHG ? sizeof(float2) : sizeof(float4);
}
template <int MK>
__device__ void mt_load_tables(const InstDev &I, void *smt) {
#pragma unroll
  for (int k = 0; k < MultiAcc<MK>::KMAX; ++k) {
    if (k < I.K) {
      const float4 *src = I.mtab[k];
      for (int j = threadIdx.x; j < I.Npad; j += blockDim.x) {
        const float4 p = __ldg(src + j);
        const size_t e = (size_t)k * I.Npad + j;
        if (MK == OBJ_MULTI_SHG) ((float2 *)smt)[e] = make_float2(p.x, p.y);
        else ((float4 *)smt)[e] = p;
      }
    }
  }
  __syncthreads();
}
template <int MK>
__device__ __forceinline__ void mt_layout(const InstDev &I, void *&smt, float4 *&stg, Mono *&sh) {
  extern __shared__ float4 dyn[];
  smt = dyn;
  stg = (float4 *)((char *)dyn + (size_t)I.K * I.Npad * mt_entry_bytes<MK>());
  sh = (Mono *)(stg + stg_f4_per_thread(true) * blockDim.x);
}

template <int MK>
static __global__ void k_de_mt(InstDev I) {
  // launched as a programmatic dependent of the phase before: the next phase's CTAs may
  // start as this grid's retire, and every CTA loads its tables (fixed per problem)
  // before it waits for the phase before to complete and its writes to be visible
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  void *smt;
  float4 *stg;
  Mono *sh;
  mt_layout<MK>(I, smt, stg, sh);
  mt_load_tables<MK>(I, smt);
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int g = *I.gen;
  const PhiloxKey K = philox_schedule(I.key);
  const int32_t *sel_in = (g & 1) ? I.sel1 : I.sel0;
  int32_t *sel_out = (g & 1) ? I.sel0 : I.sel1;
  const int nteams = (int)blockDim.x / I.T, team = (int)threadIdx.x / I.T, t = team_thread(I);
  unsigned long long k0 = 0, k1 = 0, k2 = 0;
  int cur = t == 0 ? (int)atomicAdd(&I.ctr[2], 1u) : 0;
  for (;;) {
    const int i = mt_next(I, &I.ctr[2], cur);
    if (i >= I.NP) break;
    int slot = 0, impr = 0;
    const unsigned long long key = de_individual<false, true, true, false, false, true, MK>(
        I, K, I.table, g, i, de_indices(K, I.inst, (uint32_t)g, i, I.NP, I.N), sel_in, sel_out,
        sh, &slot, stg, false, make_uint4(0u, 0u, 0u, 0u), -1, &impr, smt);
    if (t == 0) {
      top3_insert(k0, k1, k2, key);
      if (I.adaptive) I.dekey[i] = slot_key(key, i, slot, impr);
    }
  }
  // the teams' top three, merged by thread 0 (team 0's first thread)
  __shared__ unsigned long long tk[3 * 16];
  if (t == 0) {
    tk[3 * team] = k0;
    tk[3 * team + 1] = k1;
    tk[3 * team + 2] = k2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int m = 1; m < nteams; ++m)
      for (int e = 0; e < 3; ++e) top3_insert(k0, k1, k2, tk[3 * m + e]);
    I.topk[3 * blockIdx.x] = k0;
    I.topk[3 * blockIdx.x + 1] = k1;
    I.topk[3 * blockIdx.x + 2] = k2;
  }
  if (last_cta(&I.ctr[0])) {
    merge_leaders(I.topk, gridDim.x, I.lead, nullptr);  // Step 3
    if (I.adaptive) adaptive_F_block(I, I.dekey, g);     // Step 6: the next F
    if (threadIdx.x == 0) {
      I.ctr[0] = 0u;
      I.ctr[2] = 0u;
    }
  }
}

template <int MK>
static __global__ void k_gwo_mt(InstDev I) {
  // launched as a programmatic dependent of the phase before: the next phase's CTAs may
  // start as this grid's retire, and every CTA loads its tables (fixed per problem)
  // before it waits for the phase before to complete and its writes to be visible
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  void *smt;
  float4 *stg;
  Mono *sh;
  mt_layout<MK>(I, smt, stg, sh);
  mt_load_tables<MK>(I, smt);
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int g = *I.gen;
  const PhiloxKey K = philox_schedule(I.key);
  int32_t *sel = (g & 1) ? I.sel0 : I.sel1;
  const int la = I.lead[0], lb = I.lead[1], ld = I.lead[2];
  int cur = team_thread(I) == 0 ? (int)atomicAdd(&I.ctr[3], 1u) : 0;
  for (;;) {
    const int i = mt_next(I, &I.ctr[3], cur);
    if (i >= I.NP) break;
    if (i == la || i == lb || i == ld) continue;  // the leaders do not move
    gwo_individual<false, true, true, false, false, false, true, MK>(
        I, K, I.table, g, i, sel, la, lb, ld, sh, nullptr, make_float4(0.f, 0.f, 0.f, 0.f),
        make_float4(0.f, 0.f, 0.f, 0.f), nullptr, stg, -1, nullptr, smt);
  }
  if (I.trace && blockIdx.x == 0 && threadIdx.x < 3) {
    const int l = threadIdx.x == 0 ? la : (threadIdx.x == 1 ? lb : ld);
    I.trace[(size_t)I.NP * (2 + 2 * (size_t)g) + l] = __int_as_float(0x7fc00000);
  }
  if (last_cta(&I.ctr[1])) {
    if (threadIdx.x == 0) {
      *I.gen = g + 1;  // Step 6/7: next generation (a is derived from g)
      I.ctr[1] = 0u;
      I.ctr[3] = 0u;
    }
  }
}

// Steps 4-5 with the four-leader discrete GWO (launches form)
template <bool COMP>
static __global__ void k_gwo_disc(InstDev I) {
  extern __shared__ float4 dyn[];
  Mono *sh = (Mono *)dyn;
  const int g = *I.gen;
  const PhiloxKey K = philox_schedule(I.key);
  int32_t *sel = (g & 1) ? I.sel0 : I.sel1;
  // the leaders do not move in this phase
  const int la = I.lead[0], lb = I.lead[1], lc = I.lead[2], ld = I.lead[3];
  const float *L0 = row_ptr(I, la, sel[la]), *L1 = row_ptr(I, lb, sel[lb]);
  const float *L2 = row_ptr(I, lc, sel[lc]), *L3 = row_ptr(I, ld, sel[ld]);
  for (int i = blockIdx.x; i < I.NP; i += gridDim.x) {
    if (i == la || i == lb || i == lc || i == ld) continue;
    __syncthreads();  // the reduction scratch is reused
    gwo_discrete_individual<COMP>(I, K, g, i, sel, L0, L1, L2, L3, sh);
  }
  if (I.trace && blockIdx.x == 0 && threadIdx.x < 4)
    I.trace[(size_t)I.NP * (2 + 2 * (size_t)g) + I.lead[threadIdx.x]] = __int_as_float(0x7fc00000);
  if (last_cta(&I.ctr[1])) {
    if (threadIdx.x == 0) {
      *I.gen = g + 1;
      I.ctr[1] = 0u;
    }
  }
}

// ------------------------------------------------------ persistent kernel
// Step 3 of the persistent form, after the grid barrier that follows DE: the top
// three of the DE survivor keys of all individuals; every thread returns after the
// CTA barrier with lead_sh and the leaders' current slots (slot_sh) set.  Two forms:
// REDUX (short rows, where a generation is bound by its serial latency): every thread
// reads its share of the keys, every warp takes its top three with redux.sync and warp
// 0 those of the warps (7.89 -> 7.31 us per generation at N = 1000, NP = 256);
// otherwise warp 0 reads all keys and merges lane triples by shuffles, which measured
// 2.6 % faster on the 1e5-domain rows (753 against 773 us per generation), where the
// search is a negligible part of a generation.  The keys are written in
// the DE phase only, so a CTA that is still choosing leaders never sees a fitness
// already changed by another CTA's GWO selection.
template <bool REDUX>
__device__ void leaders_from_keys(const unsigned long long *keys, int NP, int32_t *lead,
                                  int32_t *lead_sh, int32_t *slot_sh) {
  if (!REDUX) {
    if (threadIdx.x < 32) {
      unsigned long long k0 = 0, k1 = 0, k2 = 0;
      for (int i = threadIdx.x; i < NP; i += 32) top3_insert(k0, k1, k2, keys[i]);
      for (int s = 16; s > 0; s >>= 1) {
        const unsigned long long p0 = __shfl_xor_sync(0xffffffffu, k0, s);
        const unsigned long long p1 = __shfl_xor_sync(0xffffffffu, k1, s);
        const unsigned long long p2 = __shfl_xor_sync(0xffffffffu, k2, s);
        top3_insert(k0, k1, k2, p0);
        top3_insert(k0, k1, k2, p1);
        top3_insert(k0, k1, k2, p2);
      }
      if (threadIdx.x == 0) {
        lead_sh[0] = slot_key_index(k0);
        lead_sh[1] = slot_key_index(k1);
        lead_sh[2] = slot_key_index(k2);
        slot_sh[0] = (int32_t)(k0 & 1u);
        slot_sh[1] = (int32_t)(k1 & 1u);
        slot_sh[2] = (int32_t)(k2 & 1u);
        if (lead) { lead[0] = lead_sh[0]; lead[1] = lead_sh[1]; lead[2] = lead_sh[2]; }
      }
    }
    __syncthreads();
    return;
  }
  __shared__ unsigned long long wtop[3 * 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long k0 = 0, k1 = 0, k2 = 0;
  for (int i = threadIdx.x; i < NP; i += blockDim.x) top3_insert(k0, k1, k2, keys[i]);
  warp_top3(k0, k1, k2);
  if (lane == 0) {
    wtop[3 * warp] = k0;
    wtop[3 * warp + 1] = k1;
    wtop[3 * warp + 2] = k2;
  }
  __syncthreads();
  if (warp == 0) {
    k0 = k1 = k2 = 0ull;
    if (lane < nw) {
      k0 = wtop[3 * lane];
      k1 = wtop[3 * lane + 1];
      k2 = wtop[3 * lane + 2];
    }
    warp_top3(k0, k1, k2);
    if (lane == 0) {
      lead_sh[0] = slot_key_index(k0);
      lead_sh[1] = slot_key_index(k1);
      lead_sh[2] = slot_key_index(k2);
      slot_sh[0] = (int32_t)(k0 & 1u);
      slot_sh[1] = (int32_t)(k1 & 1u);
      slot_sh[2] = (int32_t)(k2 & 1u);
      if (lead) { lead[0] = lead_sh[0]; lead[1] = lead_sh[1]; lead[2] = lead_sh[2]; }
    }
  }
  __syncthreads();
}

// All generations [*gen, g_end) in one cooperative launch; every CTA keeps the
// same individuals (i = blockIdx.x + k gridDim.x), the phasor table sits in
// shared memory when it fits (TS).  Two grid barriers per generation: after DE
// (the leaders need every DE survivor) and after GWO (the next donors are any
// individuals).  With one individual per CTA and 4 domains per thread, the GWO
// random words are drawn between the arrival at the first barrier and the wait.
// MAXT: the largest team the variant runs (256: two CTAs per SM; 512: one)
template <bool COMP, bool TS, bool DUAL, int MAXT = 256>
static __global__ void __launch_bounds__(MAXT, MAXT > 256 ? 1 : 2)
    k_persist(InstDev I, int g_end, Barrier bar) {
  // dynamic shared memory: [row staging (long rows)][phasor table (TS)][reduction]
  constexpr bool STG = !DUAL;
  extern __shared__ float4 dyn[];
  __shared__ int32_t lead_sh[3], lslot_sh[3], own_slot_sh;
  float4 *stg = dyn;
  float4 *tab = dyn + (STG ? stg_f4_per_thread(TS) * blockDim.x : 0);
  Mono *sh = (Mono *)(tab + (TS ? I.Npad : 0));
  if (TS) {
    for (int e = threadIdx.x; e < I.Npad; e += blockDim.x) tab[e] = __ldg(I.table + e);
    __syncthreads();
  }
  const float4 *tbl = TS ? (const float4 *)tab : I.table;
  const PhiloxKey K = philox_schedule(I.key);
  const bool pre = DUAL && (I.c == 4) && (gridDim.x == (unsigned)I.NP);
  unsigned target = 0;
  int g = *I.gen;
  // pre (one individual per CTA, one group of 4 domains per thread): the DE donors
  // and the crossover word of a generation depend on (g, i) only and are drawn
  // while the previous generation's last barrier completes
  const uint32_t jg0 = (uint32_t)((threadIdx.x * I.c) >> 2);
  // pre: own_slot_sh carries the individual's current slot from one phase to the next
  // (set by thread 0 after its selection), so its selector is not read back; the first
  // DE phase of a launch reads it
  bool own_known = false;
  int4 r_pre = make_int4(0, 0, 0, 0);
  uint4 wcr_pre = make_uint4(0u, 0u, 0u, 0u);
  if (pre && g < g_end) {
    r_pre = de_indices(K, I.inst, (uint32_t)g, blockIdx.x, I.NP, I.N);
    wcr_pre = rng4(K, I.inst, TAG_CR, (uint32_t)g, (uint32_t)blockIdx.x, jg0);
  }
  for (; g < g_end; ++g) {
    const int32_t *sel_in = (g & 1) ? I.sel1 : I.sel0;
    int32_t *sel_out = (g & 1) ? I.sel0 : I.sel1;
    for (int i = blockIdx.x; i < I.NP; i += gridDim.x) {
      if (i != (int)blockIdx.x) __syncthreads();  // the reduction scratch is reused
      const int4 r = pre ? r_pre : de_indices(K, I.inst, (uint32_t)g, i, I.NP, I.N);
      int slot = 0, impr = 0;
      const unsigned long long key =
          de_individual<COMP, false, TS, DUAL, false, STG>(I, K, tbl, g, i, r, sel_in, sel_out,
                                                            sh, &slot, stg, pre, wcr_pre,
                                                            own_known ? own_slot_sh : -1, &impr);
      // ordered before the barrier's release
      if (threadIdx.x == 0) {
        I.dekey[i] = slot_key(key, i, slot, impr);
        own_slot_sh = slot;  // read after the barrier's CTA synchronisation
      }
    }
    grid_arrive(bar, target);
    uint4 wpre[3];
    if (pre) {
      const uint32_t jg = (uint32_t)((threadIdx.x * I.c) >> 2);
#pragma unroll
      for (int k = 0; k < 3; ++k)
        wpre[k] = rng4(K, I.inst, TAG_GWO + k, (uint32_t)g, (uint32_t)blockIdx.x, jg);
    }
    if (!grid_wait(bar, target)) return;
    // the own row (its current slot, known from this CTA's own selection) is
    // requested before the leaders are known, so that its latency overlaps the
    // leader search
    float4 own0 = make_float4(0.f, 0.f, 0.f, 0.f), own1 = own0;
    if (pre) {
      const float *r0 = I.pop + ((size_t)2 * blockIdx.x + own_slot_sh) * I.Npad +
                        (size_t)threadIdx.x * 4;
      own0 = *(const float4 *)r0;
      own1 = own0;
    }
    // every CTA finds the leaders itself (Sec. 3.2 Step 3) from the DE keys
    leaders_from_keys<DUAL>(I.dekey, I.NP, blockIdx.x == 0 ? I.lead : nullptr, lead_sh, lslot_sh);
    const int la = lead_sh[0], lb = lead_sh[1], ld = lead_sh[2];
    for (int i = blockIdx.x; i < I.NP; i += gridDim.x) {
      if (i == la || i == lb || i == ld) continue;
      if (i != (int)blockIdx.x) __syncthreads();  // the reduction scratch is reused
      if (pre) {
        int gslot = 0;
        gwo_individual<COMP, false, TS, DUAL, false, true>(I, K, tbl, g, i, sel_out, la, lb, ld,
                                                           sh, wpre, own0, own1, lslot_sh,
                                                           nullptr, own_slot_sh, &gslot);
        // read by every thread after the next barrier's CTA synchronisation
        if (threadIdx.x == 0) own_slot_sh = gslot;
      }
      else
        gwo_individual<COMP, false, TS, DUAL, false, false, STG>(
            I, K, tbl, g, i, sel_out, la, lb, ld, sh, nullptr, make_float4(0.f, 0.f, 0.f, 0.f),
            make_float4(0.f, 0.f, 0.f, 0.f), lslot_sh, stg);
    }
    if (I.trace && blockIdx.x == 0 && threadIdx.x < 3) {
      const int l = threadIdx.x == 0 ? la : (threadIdx.x == 1 ? lb : ld);
      I.trace[(size_t)I.NP * (2 + 2 * (size_t)g) + l] = __int_as_float(0x7fc00000);
    }
    // Step 6, the adaptive F of the next generation, by the CTA of the alpha leader
    // (which moves no wolf when it holds one individual): the survivor keys stay
    // unchanged until the next DE phase, which the barrier below keeps after this
    if (I.adaptive && (int)blockIdx.x == la % (int)gridDim.x) adaptive_F_block(I, I.dekey, g);
    // the next DE phase reads any individual: every CTA must have finished GWO
    grid_arrive(bar, target);
    own_known = pre;
    if (pre && g + 1 < g_end) {
      r_pre = de_indices(K, I.inst, (uint32_t)(g + 1), blockIdx.x, I.NP, I.N);
      wcr_pre = rng4(K, I.inst, TAG_CR, (uint32_t)(g + 1), (uint32_t)blockIdx.x, jg0);
    }
    if (!grid_wait(bar, target)) return;
  }
  // every CTA read the start generation before its first barrier; later kernels
  // see the new value after this launch completes
  if (blockIdx.x == 0 && threadIdx.x == 0) *I.gen = g_end;
}

// ------------------------------------------------------------ batched form
// Many independent instances in one launch.  Each thread-block cluster (1, 2, 4
// or 8 CTAs on as many SMs) takes whole instances from a queue (largest first)
// and runs them for the requested generations: every warp is the team of one
// individual (instances use T = 32), the individuals of an instance are dealt to
// the warps of all CTAs of the cluster, and the two dependencies of a generation
// are cluster barriers (release/acquire at cluster scope, which also orders the
// population writes in global memory).  Each CTA's leader candidates are read by
// the others through distributed shared memory.  No cluster waits for another,
// so no co-residency beyond the cluster's own is needed.  Splitting an instance
// over a cluster keeps the largest instance from setting the batch's makespan.
static constexpr int BATCH_WARPS = 16;

__device__ __forceinline__ unsigned cluster_rank() {
  return cooperative_groups::this_cluster().block_rank();
}
__device__ __forceinline__ unsigned cluster_size() {
  return cooperative_groups::this_cluster().num_blocks();
}
// every thread of every CTA of the cluster (CL) or of the CTA; writes before it
// (shared and global) are visible to every thread of the cluster after it
template <bool CL>
__device__ __forceinline__ void cluster_sync_all() {
  if (CL) cooperative_groups::this_cluster().sync();
  else __syncthreads();
}
// the word at `p` in the shared memory of CTA `rank` of this cluster
__device__ __forceinline__ unsigned long long ld_dsmem_u64(unsigned long long *p, unsigned rank) {
  return *cooperative_groups::this_cluster().map_shared_rank(p, rank);
}

// one instance, generations [*gen, min(*gen + gens, G)), by the whole CTA
// CL: the instance is shared by the CTAs of a cluster (more than one)
template <bool COMP, bool TS, bool CL>
__device__ void batch_instance(const InstDev &I, int gens, float4 *dyn, unsigned long long *wk,
                               unsigned long long *ck, int32_t *lead_sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned crank = CL ? cluster_rank() : 0u, csize = CL ? cluster_size() : 1u;
  const int gw = (int)crank * nw + warp, gstride = (int)csize * nw;  // warp in the cluster
  // dynamic shared memory: [row staging][phasor table (TS)]
  float4 *stg = dyn, *tab = dyn + stg_f4_per_thread(TS) * blockDim.x;
  if (TS) {
    for (int e = threadIdx.x; e < I.Npad; e += blockDim.x) tab[e] = __ldg(I.table + e);
  }
  const float4 *tbl = TS ? (const float4 *)tab : I.table;
  const PhiloxKey K = philox_schedule(I.key);
  int g = *I.gen;
  const int g_end = min(g + gens, I.G);
  __syncthreads();
  for (; g < g_end; ++g) {
    const int32_t *sel_in = (g & 1) ? I.sel1 : I.sel0;
    int32_t *sel_out = (g & 1) ? I.sel0 : I.sel1;
    // each warp's running top three lives in shared memory (lane 0), which keeps
    // six registers free across the DE loop
    if (lane == 0) wk[3 * warp] = wk[3 * warp + 1] = wk[3 * warp + 2] = 0ull;
    for (int i = gw; i < I.NP; i += gstride) {
      int impr = 0;
      const unsigned long long key =
          de_individual<COMP, false, TS, false, true, true>(
              I, K, tbl, g, i, de_indices(K, I.inst, (uint32_t)g, i, I.NP, I.N), sel_in, sel_out,
              nullptr, nullptr, stg, false, make_uint4(0u, 0u, 0u, 0u), -1, &impr);
      if (lane == 0 && I.adaptive) I.dekey[i] = slot_key(key, i, 0, impr);
      if (lane == 0) {
        unsigned long long a = wk[3 * warp], b = wk[3 * warp + 1], c = wk[3 * warp + 2];
        top3_insert(a, b, c, key);
        wk[3 * warp] = a;
        wk[3 * warp + 1] = b;
        wk[3 * warp + 2] = c;
      }
    }
    __syncthreads();
    unsigned long long k0 = wk[0], k1 = wk[1], k2 = wk[2];
    if (threadIdx.x == 0) {  // this CTA's candidates
      for (int w = 1; w < nw; ++w) {
        top3_insert(k0, k1, k2, wk[3 * w]);
        top3_insert(k0, k1, k2, wk[3 * w + 1]);
        top3_insert(k0, k1, k2, wk[3 * w + 2]);
      }
      ck[0] = k0;
      ck[1] = k1;
      ck[2] = k2;
    }
    // every DE survivor of the instance and every CTA's candidates are now visible
    cluster_sync_all<CL>();
    if (threadIdx.x == 0) {  // Step 3: leaders of this instance (the same in every CTA)
      for (unsigned r = 0; CL && r < csize; ++r) {
        if (r == crank) continue;
        top3_insert(k0, k1, k2, ld_dsmem_u64(ck, r));
        top3_insert(k0, k1, k2, ld_dsmem_u64(ck + 1, r));
        top3_insert(k0, k1, k2, ld_dsmem_u64(ck + 2, r));
      }
      lead_sh[0] = key_index(k0);
      lead_sh[1] = key_index(k1);
      lead_sh[2] = key_index(k2);
      if (crank == 0) {
        I.lead[0] = lead_sh[0];
        I.lead[1] = lead_sh[1];
        I.lead[2] = lead_sh[2];
      }
    }
    __syncthreads();
    // Step 6: the adaptive F of the next generation, by the cluster's first CTA; the
    // cluster barrier after the GWO phase orders it before the next DE phase
    if (I.adaptive && crank == 0) adaptive_F_block(I, I.dekey, g);
    const int la = lead_sh[0], lb = lead_sh[1], ld = lead_sh[2];
    for (int i = gw; i < I.NP; i += gstride) {
      if (i == la || i == lb || i == ld) continue;
      gwo_individual<COMP, false, TS, false, true, false, true>(
          I, K, tbl, g, i, sel_out, la, lb, ld, nullptr, nullptr, make_float4(0.f, 0.f, 0.f, 0.f),
          make_float4(0.f, 0.f, 0.f, 0.f), nullptr, stg);
    }
    if (I.trace && crank == 0 && threadIdx.x < 3) {
      const int l = threadIdx.x == 0 ? la : (threadIdx.x == 1 ? lb : ld);
      I.trace[(size_t)I.NP * (2 + 2 * (size_t)g) + l] = __int_as_float(0x7fc00000);
    }
    // the next DE reads any individual, and ck is rewritten only after every CTA read it
    cluster_sync_all<CL>();
  }
  if (crank == 0 && threadIdx.x == 0) *I.gen = g_end;
}

template <bool TS, bool CL>
static __global__ void __launch_bounds__(BATCH_WARPS * 32, 1)
    k_batch(const InstDev *__restrict__ insts, const int32_t *__restrict__ order, int n_inst,
            unsigned *queue, int gens) {
  extern __shared__ float4 dyn[];
  __shared__ unsigned long long wk[3 * BATCH_WARPS];
  __shared__ unsigned long long ck[3];  // this CTA's leader candidates, read by the cluster
  __shared__ int32_t lead_sh[3];
  __shared__ unsigned long long job_sh;
  for (;;) {
    int job;
    {
      const unsigned crank = CL ? cluster_rank() : 0u;
      if (crank == 0 && threadIdx.x == 0) job_sh = (unsigned long long)atomicAdd(queue, 1u);
      cluster_sync_all<CL>();
      job = (int)(crank == 0 ? job_sh : ld_dsmem_u64(&job_sh, 0));
      cluster_sync_all<CL>();  // every CTA has the job before rank 0 takes the next one
    }
    if (job >= n_inst) break;
    const InstDev I = insts[order[job]];
    if (I.compensated) batch_instance<true, TS, CL>(I, gens, dyn, wk, ck, lead_sh);
    else batch_instance<false, TS, CL>(I, gens, dyn, wk, ck, lead_sh);
  }
}

// ------------------------------------------------ outputs: best, FP64, layout
static __global__ void k_best(InstDev I, int32_t *index_out) {
  __shared__ unsigned long long shk[3 * 32];
  unsigned long long k0 = 0, k1 = 0, k2 = 0;
  for (int i = threadIdx.x; i < I.NP; i += blockDim.x)
    top3_insert(k0, k1, k2, sel_key(I.minimize != 0, I.fit[i], i));
  block_top3(k0, k1, k2, shk);
  if (threadIdx.x == 0) {
    *I.best = key_index(k0);
    if (index_out) *index_out = key_index(k0);
  }
}

__device__ __forceinline__ size_t perm_pos(const InstDev &I, int j) {
  const int t = j / I.c, e = j - t * I.c;
  return ((size_t)(e >> 2) * I.T + t) * 4 + (e & 3);
}

static __global__ void k_unpermute(InstDev I, int i_fixed, float *out, int64_t ld) {
  const int i = i_fixed >= 0 ? i_fixed : (i_fixed == -2 ? *I.best : (int)blockIdx.x);
  const int32_t *sel = (*I.gen & 1) ? I.sel1 : I.sel0;
  const float *row = row_ptr(I, i, sel[i]);
  float *o = out + (i_fixed == -1 ? (int64_t)i * ld : 0);
  for (int j = threadIdx.x; j < I.N; j += blockDim.x) o[j] = row[perm_pos(I, j)];
}

static __global__ void k_copy_fit(InstDev I, float *fit_out, float2 *d_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= I.NP) return;
  if (fit_out) fit_out[i] = I.fit[i];
  if (d_out) d_out[i] = I.dval[i];
}

struct Mono64 {
  double2 A, B, C;
};
__device__ __forceinline__ Mono64 m64_combine(const Mono64 &L, const Mono64 &R) {
  Mono64 o;
  o.A = make_double2(L.A.x + R.A.x, L.A.y + R.A.y);
  o.B = make_double2(L.B.x + R.B.x, L.B.y + R.B.y);
  o.C = make_double2(L.C.x + R.C.x + (R.A.x * L.B.x - R.A.y * L.B.y),
                     L.C.y + R.C.y + (R.A.x * L.B.y + R.A.y * L.B.x));
  return o;
}

// A11: FP64 re-evaluation of the best individual's d_eff (closed form, FP64 phasors)
static __global__ void k_recheck64(InstDev I, double *d64_out, float *fit_out) {
  __shared__ Mono64 sh[256];
  const int i = *I.best;
  const int32_t *sel = (*I.gen & 1) ? I.sel1 : I.sel0;
  const float *row = row_ptr(I, i, sel[i]);
  const int nt = blockDim.x, t = threadIdx.x;
  const int per = (I.N + nt - 1) / nt;
  const int j0 = min(I.N, t * per), j1 = min(I.N, j0 + per);
  Mono64 m;
  m.A = m.B = m.C = make_double2(0.0, 0.0);
  for (int j = j0; j < j1; ++j) {
    const double d = row[perm_pos(I, j)] < 0.f ? -1.0 : 1.0;
    double s1, c1, s2, c2;
    sincos(reduce_2pi((double)j * I.kappa1), &s1, &c1);
    sincos(reduce_2pi((double)j * I.kappa2), &s2, &c2);
    const double ar = d * c2, ai = -d * s2;  // a = d p2
    m.C.x += ar * m.B.x - ai * m.B.y;
    m.C.y += ar * m.B.y + ai * m.B.x;
    m.A.x += ar;
    m.A.y += ai;
    m.B.x += d * c1;  // b = d p1
    m.B.y -= d * s1;
  }
  sh[t] = m;
  __syncthreads();
  if (t == 0) {
    Mono64 acc = sh[0];
    for (int k = 1; k < nt; ++k) acc = m64_combine(acc, sh[k]);
    double re, im;
    if (I.obj == OBJ_SHG || I.obj == OBJ_MULTI_SHG) {  // SHG field: phi(kappa1) sum d p1
      const double2 ph = I.konst64[3];
      re = ph.x * acc.B.x - ph.y * acc.B.y;
      im = ph.x * acc.B.y + ph.y * acc.B.x;
    } else {  // cascaded d_eff
      const double2 p12 = I.konst64[0], cd = I.konst64[1];
      re = p12.x * acc.C.x - p12.y * acc.C.y + cd.x;
      im = p12.x * acc.C.y + p12.y * acc.C.x + cd.y;
    }
    if (d64_out) {
      d64_out[0] = re;
      d64_out[1] = im;
    }
    if (fit_out) fit_out[0] = I.fit[i];
  }
}

// ------------------------------------------------------------ leader polish
// The three best individuals are polished on the relaxed fitness: theta = tau x,
// `steps` ascent steps theta += lr g / max|g| (g = df/dtheta from the adjoint
// kernels), then x' = clamp(theta / tau, -1, 1) is re-mapped to +-1 and kept
// only if its +-1 fitness is at least the current one (the same greedy rule as
// Sec. 2.2.1 step 4).
static __global__ void k_polish_pick(InstDev I, int32_t *lead_out) {
  __shared__ unsigned long long shk[3 * 32];
  unsigned long long k0 = 0, k1 = 0, k2 = 0;
  for (int i = threadIdx.x; i < I.NP; i += blockDim.x)
    top3_insert(k0, k1, k2, sel_key(I.minimize != 0, I.fit[i], i));
  block_top3(k0, k1, k2, shk);
  if (threadIdx.x == 0) {
    lead_out[0] = key_index(k0);
    lead_out[1] = key_index(k1);
    lead_out[2] = key_index(k2);
  }
}

__device__ __forceinline__ size_t perm_pos_of(const InstDev &I, int j) {
  const int t = j / I.c, e = j - t * I.c;
  return ((size_t)(e >> 2) * I.T + t) * 4 + (e & 3);
}

static __global__ void k_polish_theta(InstDev I, const int32_t *lead, float tau, float *theta) {
  const int k = blockIdx.x, i = lead[k];
  const int32_t *sel = (*I.gen & 1) ? I.sel1 : I.sel0;
  const float *row = row_ptr(I, i, sel[i]);
  for (int j = threadIdx.x; j < I.N; j += blockDim.x)
    theta[(size_t)k * I.Npad + j] = __fmul_rn(tau, row[perm_pos_of(I, j)]);
}

static __global__ void k_polish_step(int N, int64_t ld, float lr, float *theta, const float *grad) {
  __shared__ float red[32];
  const float *g = grad + (size_t)blockIdx.x * ld;
  float *th = theta + (size_t)blockIdx.x * ld;
  float m = 0.f;
  for (int j = threadIdx.x; j < N; j += blockDim.x) m = fmaxf(m, fabsf(g[j]));
  for (int s = 16; s > 0; s >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, s));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    red[0] = m;
  }
  __syncthreads();
  m = red[0];
  if (m > 0.f && isfinite(m)) {
    const float s = lr / m;
    for (int j = threadIdx.x; j < N; j += blockDim.x) th[j] = fmaf(s, g[j], th[j]);
  }
}

// one CTA (team of T threads) per leader
template <bool COMP>
static __global__ void k_polish_accept(InstDev I, const int32_t *lead, float tau,
                                       const float *theta, int32_t *accepted) {
  extern __shared__ Mono sh[];
  const int k = blockIdx.x, i = lead[k], t = threadIdx.x;
  int32_t *sel = (*I.gen & 1) ? I.sel1 : I.sel0;
  const int si = sel[i];
  float *out = row_ptr(I, i, si ^ 1);
  const float *th = theta + (size_t)k * I.Npad;
  Acc<COMP> acc;
  acc.zero();
  for (int k4 = 0; k4 < I.c / 4; ++k4) {
    const int j0 = t * I.c + 4 * k4;
    float4 x;
    x.x = j0 < I.N ? clamp1(__fdiv_rn(th[j0], tau)) : 0.f;
    x.y = j0 + 1 < I.N ? clamp1(__fdiv_rn(th[j0 + 1], tau)) : 0.f;
    x.z = j0 + 2 < I.N ? clamp1(__fdiv_rn(th[j0 + 2], tau)) : 0.f;
    x.w = j0 + 3 < I.N ? clamp1(__fdiv_rn(th[j0 + 3], tau)) : 0.f;
    *(float4 *)(out + ((size_t)k4 * I.T + t) * 4) = x;
    push4<COMP, false>(acc, I.table, I.T, k4, t, x);
    if (k4 & 1) acc.fold();
  }
  const Mono m = block_reduce(acc.get(), sh);
  if (t == 0) {
    const float2 D = deff_from(m, I.konst[0], I.konst[1]);
    const float f = fit_of(D);
    const bool accept = f >= I.fit[i];
    if (accept) {
      sel[i] = si ^ 1;
      I.fit[i] = f;
      I.dval[i] = D;
    }
    if (accepted) accepted[k] = accept ? 1 : 0;
  }
}

// ------------------------------------------------------ checkpoint / resume
// Natural-order genes [NP][ld] -> slot 0 of every row (permuted), both selectors
// 0, fitness recomputed with the same scan as every other evaluation (so it is
// bit-identical to the value the run had), generation counter set.
template <bool COMP, int MK = 0>
static __global__ void k_load_population(InstDev I, const float *__restrict__ genes, int64_t ld,
                                         int generation) {
  extern __shared__ Mono sh[];
  const int t = threadIdx.x;
  for (int i = blockIdx.x; i < I.NP; i += gridDim.x) {
    if (i != (int)blockIdx.x) __syncthreads();  // the reduction scratch is reused
    float *row = row_ptr(I, i, 0);
    const float *src = genes + (int64_t)i * ld;
    Acc<COMP> acc;
    acc.zero();
    MultiAcc<MK> macc;
    if (MK) macc.zero();
    for (int k4 = 0; k4 < I.c / 4; ++k4) {
      const int j0 = t * I.c + 4 * k4;
      float4 x;
      x.x = j0 < I.N ? src[j0] : 0.f;
      x.y = j0 + 1 < I.N ? src[j0 + 1] : 0.f;
      x.z = j0 + 2 < I.N ? src[j0 + 2] : 0.f;
      x.w = j0 + 3 < I.N ? src[j0 + 3] : 0.f;
      *(float4 *)(row + ((size_t)k4 * I.T + t) * 4) = x;
      if (MK) {
        macc.push4(I, k4, t, x);
      } else {
        push4<COMP, false>(acc, I.table, I.T, k4, t, x);
        if (k4 & 1) acc.fold();
      }
    }
    float2 D = make_float2(0.f, 0.f);
    float f = 0.f;
    if constexpr (MK != 0) {
      multi_finish<MK, false>(I, macc, sh, f, D);
    } else {
      const Mono m = block_reduce(acc.get(), sh);
      if (t == 0) {
        D = field_of(I, m);
        f = fit_of(D);
      }
    }
    if (t == 0) {
      I.fit[i] = f;
      I.dval[i] = D;
      I.sel0[i] = 0;
      I.sel1[i] = 0;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *I.gen = generation;
    for (int k = 0; k < 4; ++k) I.ctr[k] = 0u;
  }
}

}  // namespace qpm

// =========================================================== host: the state
using qpm::InstDev;

struct qpm_state {
  int dev = 0;
  int n = 0;
  std::vector<InstDev> h;
  std::vector<qpm_problem> probs;
  std::vector<qpm_params> params;
  std::vector<int> grid_plain, grid_persist;
  std::vector<int> grid_mt;  // CTAs of the multi-team kernels of the multi-wavelength kinds
  void *arena = nullptr;
  int g = 0;
  int G_min = 0;
  bool inited = false;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_n = -1;
  unsigned *bar = nullptr;  // [0] count, [1] unused, [2] err, [3] batch queue
  unsigned long long timeout_ns = 5000000000ull;
  InstDev *d_insts = nullptr;  // device copy of the descriptors (batched form)
  int32_t *d_order = nullptr;  // instances by decreasing work
  size_t batch_smem = 0;       // dynamic shared memory of the batched kernel
  bool batch_ts = false;       // phasor tables in shared memory (else read from global)
  int grid_batch = 0;
  int batch_cluster = 1;       // CTAs per thread-block cluster in the batched form
  cudaGraphExec_t gexec_b = nullptr;
  int graph_b_n = -1;
  void *polish = nullptr;  // leader-polish scratch (allocated on first use)
  size_t polish_bytes = 0;
  std::vector<qpm_objective> objs;  // per instance (kind 0 unless qpm_set_objective)
  std::vector<void *> objmem;       // tables of a multi-wavelength kind's problems 2 .. K
};

namespace qpm {

// threads per individual: the smallest power of two in [32, 256] giving at most
// 4 domains per thread; beyond 1024 domains the 256 threads take more each
static int choose_team(int N) {
  int T = 32;
  while (T < 256 && N > 4 * T) T *= 2;
  return T;
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static size_t smem_bytes(int T) { return sizeof(Mono) * (size_t)(T / 32 + 1); }
// the reduction scratch of the multi-wavelength kinds: one monoid per problem and warp
static size_t smem_bytes_multi(int T) { return sizeof(Mono) * (size_t)(8 * (T / 32) + 1); }

// kernel variants of one instance
struct Variant {
  const void *de, *gwo, *persist;
  size_t smem, persist_smem;
  int block = 0;  // threads per CTA of de / gwo (0: the team width)
};

static constexpr int TS_MAX_NPAD = 4096;  // phasor table in shared memory up to 64 KB
static constexpr size_t BATCH_TS_MAX_BYTES = 160 * 1024;  // batched form: table in smem up to 160 KB

template <bool COMP, bool DUAL>
static Variant variant2(const InstDev &I) {
  Variant v;
  v.de = (const void *)k_de<COMP, DUAL>;
  v.gwo = (const void *)k_gwo<COMP, DUAL>;
  // k_de / k_gwo read the table from global memory: long rows stage rows and table
  v.smem = (DUAL ? 0 : sizeof(float4) * stg_f4_per_thread(false) * (size_t)I.T) + smem_bytes(I.T);
  const bool wide = I.T > 256;
  // row staging of the long-row variants (DUAL false)
  const bool ts = I.Npad <= TS_MAX_NPAD;
  const size_t stg = DUAL ? 0 : sizeof(float4) * stg_f4_per_thread(ts) * (size_t)I.T;
  if (ts) {
    v.persist = wide ? (const void *)k_persist<COMP, true, DUAL, 512>
                     : (const void *)k_persist<COMP, true, DUAL>;
    v.persist_smem = stg + sizeof(float4) * (size_t)I.Npad + smem_bytes(I.T);
  } else {
    v.persist = wide ? (const void *)k_persist<COMP, false, DUAL, 512>
                     : (const void *)k_persist<COMP, false, DUAL>;
    v.persist_smem = stg + smem_bytes(I.T);
  }
  return v;
}

// the multi-wavelength kinds: launches form only, rows staged; their K tables in shared
// memory shared by the teams of a CTA of up to 512 threads (at most 8 teams with their
// named barriers, 16 one-warp teams) where they fit, else through L1
static size_t optin_smem() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  return (size_t)v;
}
// the dynamic shared memory the multi-team kernels may take: the opt-in limit less their
// own static shared memory (their attribute is set to it, so states of any size can
// take turns on the same kernels)
template <int MK>
static size_t mt_smem_cap() {
  static const size_t cap = [] {
    cudaFuncAttributes a{}, b{};
    const size_t optin = optin_smem();
    if (cudaFuncGetAttributes(&a, (const void *)k_de_mt<MK>) != cudaSuccess ||
        cudaFuncGetAttributes(&b, (const void *)k_gwo_mt<MK>) != cudaSuccess)
      return (size_t)0;
    const size_t st = std::max(a.sharedSizeBytes, b.sharedSizeBytes);
    return optin > st ? optin - st : (size_t)0;
  }();
  return cap;
}
template <int MK>
static Variant variant_multi(const InstDev &I) {
  Variant v;
  // at most 8 named barriers (1 .. 8); one-warp teams need none (16 per CTA)
  const int nteams = std::max(1, std::min(I.T == 32 ? 16 : 8, 512 / I.T));
  const int block = nteams * I.T;
  const size_t mt = (size_t)I.K * I.Npad * mt_entry_bytes<MK>() +
                    sizeof(float4) * stg_f4_per_thread(true) * (size_t)block +
                    sizeof(Mono) * (size_t)MultiAcc<MK>::KMAX * (I.T / 32) * nteams;
  if (mt <= mt_smem_cap<MK>()) {
    v.de = (const void *)k_de_mt<MK>;
    v.gwo = (const void *)k_gwo_mt<MK>;
    v.smem = mt;
    v.block = block;
    v.persist = nullptr;
    v.persist_smem = 0;
    return v;
  }
  v.de = (const void *)k_de<false, false, MK>;
  v.gwo = (const void *)k_gwo<false, false, MK>;
  v.smem = sizeof(float4) * stg_f4_per_thread(true) * (size_t)I.T + smem_bytes_multi(I.T);
  v.persist = nullptr;
  v.persist_smem = 0;
  return v;
}

static Variant variant_of(const InstDev &I) {
  if (I.obj == OBJ_MULTI_THG) return variant_multi<OBJ_MULTI_THG>(I);
  if (I.obj == OBJ_MULTI_SHG) return variant_multi<OBJ_MULTI_SHG>(I);
  const bool dual = I.c <= 8;
  Variant v = I.compensated ? (dual ? variant2<true, true>(I) : variant2<true, false>(I))
                            : (dual ? variant2<false, true>(I) : variant2<false, false>(I));
  if (I.combine == 2)  // the discrete GWO (launches form): its own GWO kernel
    v.gwo = I.compensated ? (const void *)k_gwo_disc<true> : (const void *)k_gwo_disc<false>;
  return v;
}

// the shared-memory attribute of a persistent variant is the same for every
// instance (the largest any instance can need), so occupancy figures computed
// for one instance stay valid after another instance is set up
static size_t persist_smem_cap(bool ts) {
  return sizeof(float4) * stg_f4_per_thread(ts) * 512 + smem_bytes(512) +
         (ts ? sizeof(float4) * (size_t)TS_MAX_NPAD : 0);
}

static const void *batch_kernel(bool ts, bool cl) {
  if (ts) return cl ? (const void *)k_batch<true, true> : (const void *)k_batch<true, false>;
  return cl ? (const void *)k_batch<false, true> : (const void *)k_batch<false, false>;
}

// co-resident CTAs of the batched kernel for clusters of `cs` CTAs (a multiple of cs)
static qpm_status batch_grid(const qpm_state *st, int cs, int *grid) {
  const void *kb = batch_kernel(st->batch_ts, cs > 1);
  // the largest any state of this kernel variant can need, so that a state with smaller
  // tables cannot fail the captured launch of another
  const size_t cap = sizeof(float4) * stg_f4_per_thread(st->batch_ts) * BATCH_WARPS * 32 +
                     (st->batch_ts ? BATCH_TS_MAX_BYTES : 0);
  QPM_CUDA(cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(cs * sm_count()));
  cfg.blockDim = dim3(BATCH_WARPS * 32);
  cfg.dynamicSmemBytes = st->batch_smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  QPM_CUDA(cudaOccupancyMaxActiveClusters(&clusters, kb, &cfg));
  if (clusters < 1) return fail(QPM_ERR_UNSUPPORTED, "batched form: clusters of this size do not fit");
  *grid = clusters * cs;
  return QPM_OK;
}

static qpm_status occupancy(const InstDev &I, int *plain, int *persist) {
  const Variant v = variant_of(I);
  int a = 0, a2 = 0, b = 0;
  QPM_CUDA(cudaFuncSetAttribute(v.persist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)persist_smem_cap(I.Npad <= TS_MAX_NPAD)));
  // the largest dynamic shared memory any instance's k_de / k_gwo can need
  const int plain_cap = (int)(sizeof(float4) * stg_f4_per_thread(false) * 512 + smem_bytes(512));
  QPM_CUDA(cudaFuncSetAttribute(v.de, cudaFuncAttributeMaxDynamicSharedMemorySize, plain_cap));
  QPM_CUDA(cudaFuncSetAttribute(v.gwo, cudaFuncAttributeMaxDynamicSharedMemorySize, plain_cap));
  QPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, v.de, I.T, v.smem));
  QPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a2, v.gwo, I.T, v.smem));
  QPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, v.persist, I.T, v.persist_smem));
  *plain = std::max(1, std::min(a, a2));
  *persist = std::max(1, b);
  return QPM_OK;
}

static qpm_status enqueue_step(qpm_state *st, cudaStream_t s) {
  for (int k = 0; k < st->n; ++k) {
    InstDev I = st->h[k];
    const Variant v = variant_of(I);
    void *args[] = {&I};
    const bool mt = v.block != 0;  // several teams per CTA
    const dim3 grid(mt ? st->grid_mt[k] : st->grid_plain[k]), block(mt ? v.block : I.T);
    if (mt) {  // each phase a programmatic dependent of the one before
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = grid;
      cfg.blockDim = block;
      cfg.dynamicSmemBytes = v.smem;
      cfg.stream = s;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      QPM_CUDA(cudaLaunchKernelExC(&cfg, v.de, args));
      QPM_CUDA(cudaLaunchKernelExC(&cfg, v.gwo, args));
      continue;
    }
    QPM_CUDA(cudaLaunchKernel(v.de, grid, block, args, v.smem, s));
    QPM_CUDA(cudaLaunchKernel(v.gwo, grid, block, args, v.smem, s));
  }
  return QPM_OK;
}

static qpm_status check_state(qpm_state *st, int gens) {
  if (!st) return fail(QPM_ERR_ARG, "NULL state");
  if (!st->inited) return fail(QPM_ERR_STATE, "qpm_init has not been called");
  if (gens < 0) return fail(QPM_ERR_ARG, "negative generation count");
  if (st->g + gens > st->G_min)
    return fail(QPM_ERR_ARG, "running past the last generation G of an instance");
  int dev = -1;
  QPM_CUDA(cudaGetDevice(&dev));
  if (dev != st->dev) return fail(QPM_ERR_STATE, "state belongs to another device");
  return QPM_OK;
}

}  // namespace qpm

using namespace qpm;

extern "C" qpm_status qpm_create(const qpm_problem *probs, const qpm_params *params,
                                 int32_t n_inst, qpm_state **out) {
  if (!probs || !params || !out) return fail(QPM_ERR_ARG, "qpm_create: NULL pointer");
  if (n_inst < 1) return fail(QPM_ERR_ARG, "qpm_create: n_inst < 1");
  *out = nullptr;
  for (int k = 0; k < n_inst; ++k) {
    const qpm_problem &p = probs[k];
    const qpm_params &q = params[k];
    if (p.N < 1) return fail(QPM_ERR_ARG, "qpm_create: N < 1");
    if (p.N > (1 << 26)) return fail(QPM_ERR_UNSUPPORTED, "qpm_create: N too large");
    if (q.NP < 4) return fail(QPM_ERR_ARG, "qpm_create: NP < 4 (rand/1 needs three donors)");
    if (q.NP > (1 << 28)) return fail(QPM_ERR_UNSUPPORTED, "qpm_create: NP above 2^28");
    if (q.G < 1) return fail(QPM_ERR_ARG, "qpm_create: G < 1");
    if (!(q.F >= 0.f && q.F <= 2.f)) return fail(QPM_ERR_ARG, "qpm_create: F outside [0, 2]");
    if (!(q.CR >= 0.f && q.CR <= 1.f)) return fail(QPM_ERR_ARG, "qpm_create: CR outside [0, 1]");
    if (q.gwo_combine < 0 || q.gwo_combine > 2)
      return fail(QPM_ERR_ARG, "qpm_create: gwo_combine must be 0, 1 or 2");
    if (q.team != 0 && q.team != 32 && q.team != 64 && q.team != 128 && q.team != 256 &&
        q.team != 512)
      return fail(QPM_ERR_ARG, "qpm_create: team must be 0, 32, 64, 128, 256 or 512");
    if (q.f_schedule < 0 || q.f_schedule > 2)
      return fail(QPM_ERR_ARG, "qpm_create: f_schedule must be 0, 1 or 2");
    if (q.f_schedule == 2 && q.NP > (1 << 23))
      return fail(QPM_ERR_UNSUPPORTED, "qpm_create: the adaptive F needs NP <= 2^23");
    if (!std::isfinite(p.kappa1) || !std::isfinite(p.kappa2))
      return fail(QPM_ERR_ARG, "qpm_create: kappa must be finite");
  }
  qpm_state *st = new qpm_state();
  cudaError_t e = cudaGetDevice(&st->dev);
  if (e != cudaSuccess) { delete st; return cuda_fail(e, "cudaGetDevice"); }
  st->n = n_inst;
  st->probs.assign(probs, probs + n_inst);
  st->params.assign(params, params + n_inst);
  st->h.resize(n_inst);
  st->grid_plain.resize(n_inst);
  st->grid_mt.assign(n_inst, 0);
  st->grid_persist.resize(n_inst);
  st->objs.assign(n_inst, qpm_objective{});
  st->objmem.assign(n_inst, nullptr);
  st->G_min = params[0].G;
  const int nsm = sm_count();
  size_t total = 0;
  std::vector<size_t> base(n_inst);
  for (int k = 0; k < n_inst; ++k) {
    const qpm_problem &p = probs[k];
    const qpm_params &q = params[k];
    InstDev &I = st->h[k];
    memset(&I, 0, sizeof(I));
    I.N = p.N;
    I.T = q.team ? q.team : (n_inst > 1 ? 32 : choose_team(p.N));
    I.Npad = (int32_t)align_up((size_t)p.N, 4 * (size_t)I.T);
    I.c = I.Npad / I.T;
    I.NP = q.NP;
    I.G = q.G;
    I.combine = q.gwo_combine;
    I.compensated = q.compensated ? 1 : 0;
    I.F = q.F;
    I.CR = q.CR;
    I.crthr = cr_threshold(q.CR);
    I.inst = (uint32_t)k;
    I.key = make_uint2((uint32_t)q.seed, (uint32_t)(q.seed >> 32));
    I.kappa1 = p.kappa1;
    I.kappa2 = p.kappa2;
    st->G_min = std::min(st->G_min, q.G);
    int occ_plain = 1, occ_persist = 1;
    qpm_status s2 = occupancy(I, &occ_plain, &occ_persist);
    if (s2 != QPM_OK) { delete st; return s2; }
    if (q.team == 0 && n_inst == 1 && I.T == 256 && I.c >= 16) {
      // long rows: 512 threads per individual (one CTA per SM) when that leaves fewer
      // CTA slots idle in the last round of individuals of a phase
      InstDev W = I;
      W.T = 512;
      W.Npad = (int32_t)align_up((size_t)p.N, 4 * (size_t)W.T);
      W.c = W.Npad / W.T;
      int wp = 1, wq = 1;
      s2 = occupancy(W, &wp, &wq);
      if (s2 != QPM_OK) { delete st; return s2; }
      auto fill = [&](int slots) {
        const int rounds = (I.NP + slots - 1) / slots;
        return (double)I.NP / ((double)rounds * slots);
      };
      if (fill(wq * nsm) > fill(occ_persist * nsm) + 0.05) {
        I.T = W.T;
        I.Npad = W.Npad;
        I.c = W.c;
        occ_plain = wp;
        occ_persist = wq;
      }
    }
    st->grid_plain[k] = std::min(I.NP, occ_plain * nsm);
    st->grid_persist[k] = std::min(I.NP, occ_persist * nsm);
    base[k] = total;
    const size_t NP = (size_t)I.NP, Np = (size_t)I.Npad;
    total += align_up(2 * NP * Np * sizeof(float), 256);
    total += 2 * align_up(NP * sizeof(int32_t), 256);
    total += align_up(NP * sizeof(float), 256) + align_up(NP * sizeof(float2), 256);
    total += align_up(Np * sizeof(float4), 256);
    total += align_up((size_t)table_part_count(I.Npad) * sizeof(double2), 256);
    total += 256 + 256 + 256;  // konst, konst64, lead
    total += align_up(6 * NP * sizeof(unsigned long long), 256);
    total += align_up(NP * sizeof(unsigned long long), 256);  // DE survivor keys
    total += 2 * align_up((size_t)(q.G + 1) * sizeof(float), 256);  // F history, F base
    total += align_up((size_t)q.G * 7 * sizeof(uint32_t), 256);     // discrete GWO thresholds
    total += 256 + 256 + 256;  // ctr, gen, best
  }
  const size_t desc_off = total;
  total += align_up(sizeof(InstDev) * (size_t)n_inst, 256);
  const size_t order_off = total;
  total += align_up(sizeof(int32_t) * (size_t)n_inst, 256);
  total += 256;  // barrier words
  e = cudaMalloc(&st->arena, total);
  if (e != cudaSuccess) { delete st; return cuda_fail(e, "cudaMalloc(state arena)"); }
  e = cudaMemset(st->arena, 0, total);
  if (e != cudaSuccess) { cudaFree(st->arena); delete st; return cuda_fail(e, "cudaMemset"); }
  for (int k = 0; k < n_inst; ++k) {
    InstDev &I = st->h[k];
    char *p = (char *)st->arena + base[k];
    auto take = [&](size_t bytes) { char *r = p; p += align_up(bytes, 256); return (void *)r; };
    const size_t NP = (size_t)I.NP, Np = (size_t)I.Npad;
    I.pop = (float *)take(2 * NP * Np * sizeof(float));
    I.sel0 = (int32_t *)take(NP * sizeof(int32_t));
    I.sel1 = (int32_t *)take(NP * sizeof(int32_t));
    I.fit = (float *)take(NP * sizeof(float));
    I.dval = (float2 *)take(NP * sizeof(float2));
    I.table = (float4 *)take(Np * sizeof(float4));
    I.tpart = (double2 *)take((size_t)table_part_count(I.Npad) * sizeof(double2));
    I.konst = (float2 *)take(4 * sizeof(float2));
    I.K = 1;  // the cascaded d_eff of the problem until qpm_set_objective
    I.mtab[0] = I.table;
    I.mkonst[0] = I.konst;
    I.konst64 = (double2 *)take(4 * sizeof(double2));
    I.lead = (int32_t *)take(4 * sizeof(int32_t));  // four for the discrete GWO
    I.topk = (unsigned long long *)take(6 * NP * sizeof(unsigned long long));
    I.dekey = (unsigned long long *)take(NP * sizeof(unsigned long long));
    {
      float *fs = (float *)take((size_t)(I.G + 1) * sizeof(float));
      float *fb = (float *)take((size_t)(I.G + 1) * sizeof(float));
      I.Fsched = st->params[k].f_schedule ? fs : nullptr;
      I.Fbase = st->params[k].f_schedule == 2 ? fb : nullptr;
      I.adaptive = st->params[k].f_schedule == 2 ? 1 : 0;
    }
    {
      uint32_t *th = (uint32_t *)take((size_t)I.G * 7 * sizeof(uint32_t));
      I.dthr = I.combine == 2 ? th : nullptr;
    }
    I.ctr = (unsigned *)take(4 * sizeof(unsigned));
    I.gen = (int32_t *)take(sizeof(int32_t));
    I.best = (int32_t *)take(sizeof(int32_t));
  }
  st->bar = (unsigned *)((char *)st->arena + total - 256);
  st->d_insts = (InstDev *)((char *)st->arena + desc_off);
  st->d_order = (int32_t *)((char *)st->arena + order_off);
  {
    // largest instances first (longest-processing-time order for the batch queue)
    std::vector<int32_t> order(n_inst);
    for (int k = 0; k < n_inst; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      return (long long)st->h[a].NP * st->h[a].Npad > (long long)st->h[b].NP * st->h[b].Npad;
    });
    // F schedules (Sec. 3.1.1): cosine decay times a quadratic factor 1.0 -> 0.8, for
    // generations 0 .. G; from F (f_schedule 1), or from the top 0.1 of the adaptive
    // F's interval (f_schedule 2: its intermediate state's values in Fbase, and its
    // first generation's F in the history)
    // thresholds of the discrete GWO (Sec. 3.1.2): per generation g (tau = g / G) the
    // social rate, the disturbance and P(+1) for 0 .. 4 leaders at +1, as 16-bit
    // thresholds floor(65536 p), evaluated in FP64
    for (int k = 0; k < n_inst && e == cudaSuccess; ++k) {
      if (!st->h[k].dthr) continue;
      const int G = st->h[k].G;
      std::vector<uint32_t> th((size_t)G * 7);
      for (int g = 0; g < G; ++g) {
        const double tau = (double)g / (double)G;
        const double delta = 0.5 * (1.0 - tau), sigma = 0.3 * (1.0 - tau);
        const double mu = 0.1 * (1.0 - tau) + 0.01 * tau;
        th[7 * (size_t)g] = (uint32_t)std::floor(65536.0 * sigma);
        th[7 * (size_t)g + 1] = (uint32_t)std::floor(65536.0 * mu);
        for (int n = 0; n <= 4; ++n) {
          const double m = n > 2 ? 1.0 : (n < 2 ? 0.0 : 0.5);
          const double qn = (1.0 - tau) * ((double)n / 4.0) + tau * m;
          th[7 * (size_t)g + 2 + n] = (uint32_t)std::floor(65536.0 * ((1.0 - delta) * qn + 0.5 * delta));
        }
      }
      e = cudaMemcpy((void *)st->h[k].dthr, th.data(), sizeof(uint32_t) * th.size(),
                     cudaMemcpyHostToDevice);
    }
    for (int k = 0; k < n_inst && e == cudaSuccess; ++k) {
      if (!st->h[k].Fsched) continue;
      const int G = st->h[k].G;
      const bool adaptive = st->h[k].adaptive != 0;
      const double top = adaptive ? 0.1 : (double)st->params[k].F;
      std::vector<float> F(G + 1);
      for (int g = 0; g <= G; ++g) {
        const double x = (double)g / (double)G;
        const double c = 0.5 * (std::cos(M_PI * (double)g / (2.0 * (double)G)) + 1.0);
        const double qd = 1.0 - 0.2 * x * x;
        F[g] = (float)(top * c * qd);
      }
      e = cudaMemcpy(st->h[k].Fsched, F.data(), sizeof(float) * (G + 1), cudaMemcpyHostToDevice);
      if (e == cudaSuccess && adaptive)
        e = cudaMemcpy((void *)st->h[k].Fbase, F.data(), sizeof(float) * (G + 1),
                       cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess)
      e = cudaMemcpy(st->d_order, order.data(), sizeof(int32_t) * n_inst, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(st->d_insts, st->h.data(), sizeof(InstDev) * n_inst, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(st->arena); delete st; return cuda_fail(e, "cudaMemcpy"); }
    int maxpad = 0;
    for (int k = 0; k < n_inst; ++k) maxpad = std::max(maxpad, st->h[k].Npad);
    st->batch_ts = (size_t)maxpad * sizeof(float4) <= BATCH_TS_MAX_BYTES;
    st->batch_smem = sizeof(float4) * stg_f4_per_thread(st->batch_ts) * BATCH_WARPS * 32 +
                     (st->batch_ts ? (size_t)maxpad * sizeof(float4) : 0);
    st->grid_batch = 0;  // set on the first batched run (or by qpm_set_batch_cluster)
  }
  e = cudaStreamCreateWithFlags(&st->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) { cudaFree(st->arena); delete st; return cuda_fail(e, "cudaStreamCreate"); }
  *out = st;
  return QPM_OK;
}

extern "C" qpm_status qpm_set_trace(qpm_state *st, int32_t inst, float *trace) {
  if (!st || inst < 0 || inst >= st->n) return fail(QPM_ERR_ARG, "qpm_set_trace: bad instance");
  st->h[inst].trace = trace;
  if (st->gexec) {
    cudaGraphExecDestroy(st->gexec);
    st->gexec = nullptr;
    st->graph_n = -1;
  }
  cudaError_t e = cudaMemcpy(st->d_insts + inst, &st->h[inst], sizeof(InstDev), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(descriptor)");
  return QPM_OK;
}

extern "C" qpm_status qpm_init(qpm_state *st, qpm_stream_t stream) {
  if (!st) return fail(QPM_ERR_ARG, "NULL state");
  cudaStream_t s = (cudaStream_t)stream;
  for (int k = 0; k < st->n; ++k) {
    const InstDev &I = st->h[k];
    TableSpec ts{I.N, I.Npad, I.T, I.c, I.kappa1, I.kappa2};
    qpm_status r = launch_table(ts, I.table, I.tpart, I.konst, I.konst64, s);
    if (r != QPM_OK) return r;
    // the other problems of a multi-wavelength kind (one after the other: they share
    // the reduction scratch on this stream)
    for (int q = 1; q < (I.obj >= OBJ_MULTI_THG ? I.K : 1); ++q) {
      TableSpec tq{I.N, I.Npad, I.T, I.c, st->objs[k].kappa1[q], st->objs[k].kappa2[q]};
      r = launch_table(tq, (float4 *)I.mtab[q], I.tpart, (float2 *)I.mkonst[q], nullptr, s);
      if (r != QPM_OK) return r;
    }
    const size_t sm = smem_bytes(I.T), smm = smem_bytes_multi(I.T);
    if (I.obj == OBJ_MULTI_THG) k_init<false, OBJ_MULTI_THG><<<st->grid_plain[k], I.T, smm, s>>>(I);
    else if (I.obj == OBJ_MULTI_SHG) k_init<false, OBJ_MULTI_SHG><<<st->grid_plain[k], I.T, smm, s>>>(I);
    else if (I.compensated) k_init<true><<<st->grid_plain[k], I.T, sm, s>>>(I);
    else k_init<false><<<st->grid_plain[k], I.T, sm, s>>>(I);
    QPM_CUDA(cudaGetLastError());
  }
  st->g = 0;
  st->inited = true;
  return QPM_OK;
}

extern "C" qpm_status qpm_step(qpm_state *st, qpm_stream_t stream) {
  qpm_status r = check_state(st, 1);
  if (r != QPM_OK) return r;
  r = enqueue_step(st, (cudaStream_t)stream);
  if (r == QPM_OK) st->g += 1;
  return r;
}

extern "C" qpm_status qpm_run(qpm_state *st, int32_t generations, int32_t mode,
                              qpm_stream_t stream) {
  qpm_status r = check_state(st, generations);
  if (r != QPM_OK) return r;
  cudaStream_t s = (cudaStream_t)stream;
  if (generations == 0) return QPM_OK;
  if (mode == QPM_RUN_LAUNCHES) {
    for (int g = 0; g < generations; ++g) {
      r = enqueue_step(st, s);
      if (r != QPM_OK) return r;
    }
  } else if (mode == QPM_RUN_GRAPH) {
    if (st->graph_n != generations || !st->gexec) {
      if (st->gexec) {
        cudaGraphExecDestroy(st->gexec);
        st->gexec = nullptr;
      }
      QPM_CUDA(cudaStreamBeginCapture(st->cap_stream, cudaStreamCaptureModeThreadLocal));
      for (int g = 0; g < generations; ++g) {
        r = enqueue_step(st, st->cap_stream);
        if (r != QPM_OK) {
          cudaGraph_t junk;
          cudaStreamEndCapture(st->cap_stream, &junk);
          if (junk) cudaGraphDestroy(junk);
          return r;
        }
      }
      cudaGraph_t graph;
      QPM_CUDA(cudaStreamEndCapture(st->cap_stream, &graph));
      cudaError_t e = cudaGraphInstantiate(&st->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
      st->graph_n = generations;
    }
    QPM_CUDA(cudaGraphLaunch(st->gexec, s));
  } else if (mode == QPM_RUN_PERSISTENT) {
    for (int k = 0; k < st->n; ++k)
      if (st->h[k].obj >= OBJ_MULTI_THG || st->h[k].combine == 2)
        return fail(QPM_ERR_UNSUPPORTED, "the multi-wavelength objectives and the discrete GWO "
                                         "run in the launches and graph forms");
    QPM_CUDA(cudaMemsetAsync(st->bar, 0, 3 * sizeof(unsigned), s));
    for (int k = 0; k < st->n; ++k) {
      InstDev I = st->h[k];
      const Variant v = variant_of(I);
      int g_end = st->g + generations;
      // each instance gets a fresh arrival counter; the error word is shared
      QPM_CUDA(cudaMemsetAsync(st->bar, 0, sizeof(unsigned), s));
      Barrier b{st->bar, (int32_t *)(st->bar + 2), st->timeout_ns};
      void *args[] = {&I, &g_end, &b};
      QPM_CUDA(cudaLaunchCooperativeKernel(v.persist, st->grid_persist[k], I.T, args,
                                           v.persist_smem, s));
    }
    int32_t err = 0;
    QPM_CUDA(cudaMemcpyAsync(&err, st->bar + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    QPM_CUDA(cudaStreamSynchronize(s));
    if (err != 0) {
      st->g += generations;
      return fail(QPM_ERR_TIMEOUT, "persistent kernel: a bounded grid-barrier wait gave up");
    }
  } else if (mode == QPM_RUN_BATCHED) {
    for (int k = 0; k < st->n; ++k)
      if (st->h[k].obj >= OBJ_MULTI_THG || st->h[k].combine == 2)
        return fail(QPM_ERR_UNSUPPORTED, "the multi-wavelength objectives and the discrete GWO "
                                         "run in the launches and graph forms");
    for (int k = 0; k < st->n; ++k)
      if (st->h[k].T != 32)
        return fail(QPM_ERR_UNSUPPORTED, "batched form needs 32 threads per individual (team 32)");
    if (st->grid_batch == 0) {
      qpm_status r = batch_grid(st, st->batch_cluster, &st->grid_batch);
      if (r != QPM_OK) return r;
    }
    if (st->graph_b_n != generations || !st->gexec_b) {
      if (st->gexec_b) {
        cudaGraphExecDestroy(st->gexec_b);
        st->gexec_b = nullptr;
      }
      QPM_CUDA(cudaStreamBeginCapture(st->cap_stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = cudaMemsetAsync(st->bar + 3, 0, sizeof(unsigned), st->cap_stream);
      if (e == cudaSuccess) {
        int n = st->n, gens = generations;
        unsigned *queue = st->bar + 3;
        void *args[] = {&st->d_insts, &st->d_order, &n, &queue, &gens};
        const void *kb = batch_kernel(st->batch_ts, st->batch_cluster > 1);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)st->batch_cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)st->grid_batch);
        cfg.blockDim = dim3(BATCH_WARPS * 32);
        cfg.dynamicSmemBytes = st->batch_smem;
        cfg.stream = st->cap_stream;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelExC(&cfg, kb, args);
      }
      cudaGraph_t graph = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(st->cap_stream, &graph);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(e != cudaSuccess ? e : e2, "capturing the batched launch");
      }
      e = cudaGraphInstantiate(&st->gexec_b, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
      st->graph_b_n = generations;
    }
    QPM_CUDA(cudaGraphLaunch(st->gexec_b, s));
  } else {
    return fail(QPM_ERR_ARG, "qpm_run: unknown mode");
  }
  st->g += generations;
  return QPM_OK;
}

extern "C" qpm_status qpm_set_batch_cluster(qpm_state *st, int32_t ctas) {
  if (!st) return fail(QPM_ERR_ARG, "qpm_set_batch_cluster: NULL state");
  if (ctas != 1 && ctas != 2 && ctas != 4 && ctas != 8)
    return fail(QPM_ERR_ARG, "qpm_set_batch_cluster: ctas must be 1, 2, 4 or 8");
  int dev = -1;
  QPM_CUDA(cudaGetDevice(&dev));
  if (dev != st->dev) return fail(QPM_ERR_STATE, "state belongs to another device");
  int grid = 0;
  qpm_status r = batch_grid(st, ctas, &grid);
  if (r != QPM_OK) return r;
  if (st->gexec_b) {  // the captured launch has the old shape
    QPM_CUDA(cudaDeviceSynchronize());
    cudaGraphExecDestroy(st->gexec_b);
    st->gexec_b = nullptr;
    st->graph_b_n = -1;
  }
  st->batch_cluster = ctas;
  st->grid_batch = grid;
  return QPM_OK;
}

extern "C" qpm_status qpm_set_objective(qpm_state *st, int32_t inst, const qpm_objective *o) {
  if (!st || inst < 0 || inst >= st->n || !o) return fail(QPM_ERR_ARG, "qpm_set_objective: bad arguments");
  if (st->inited) return fail(QPM_ERR_STATE, "qpm_set_objective: call it before qpm_init");
  if (o->kind < OBJ_THG || o->kind > OBJ_MULTI_SHG)
    return fail(QPM_ERR_ARG, "qpm_set_objective: kind must be one of QPM_OBJ_*");
  const bool multi = o->kind >= OBJ_MULTI_THG;
  const int kmax = o->kind == OBJ_MULTI_THG ? 4 : 8;
  if (multi && (o->K < 1 || o->K > kmax))
    return fail(QPM_ERR_ARG, "qpm_set_objective: need 1 <= K <= 4 (THG) or 8 (SHG)");
  for (int k = 0; multi && k < o->K; ++k)
    if (!std::isfinite(o->kappa1[k]) || !std::isfinite(o->kappa2[k]))
      return fail(QPM_ERR_ARG, "qpm_set_objective: kappa must be finite");
  if (multi && (!std::isfinite(o->G0) || !(o->beta >= 0.f) || !std::isfinite(o->beta)))
    return fail(QPM_ERR_ARG, "qpm_set_objective: need finite G0 and beta >= 0");
  int dev = -1;
  QPM_CUDA(cudaGetDevice(&dev));
  if (dev != st->dev) return fail(QPM_ERR_STATE, "state belongs to another device");
  InstDev &I = st->h[inst];
  if (multi && I.combine == 2)
    return fail(QPM_ERR_UNSUPPORTED, "qpm_set_objective: the discrete GWO optimises the single kinds");
  if (st->objmem[inst]) {
    QPM_CUDA(cudaFree(st->objmem[inst]));
    st->objmem[inst] = nullptr;
  }
  I.obj = o->kind;
  I.minimize = multi ? 1 : 0;
  I.K = multi ? o->K : 1;
  I.G0 = multi ? o->G0 : 0.f;
  I.beta = multi ? o->beta : 0.f;
  for (int k = 0; k < 8; ++k) {
    I.mtab[k] = nullptr;
    I.mkonst[k] = nullptr;
  }
  I.mtab[0] = I.table;
  I.mkonst[0] = I.konst;
  if (multi) {
    // the first problem is the instance's own: its table, constants and FP64 re-check
    I.kappa1 = o->kappa1[0];
    I.kappa2 = o->kappa2[0];
    st->probs[inst].kappa1 = o->kappa1[0];
    st->probs[inst].kappa2 = o->kappa2[0];
    if (o->K > 1) {
      const size_t tb = align_up(sizeof(float4) * (size_t)I.Npad, 256);
      void *mem = nullptr;
      QPM_CUDA(cudaMalloc(&mem, (size_t)(o->K - 1) * (tb + 256)));
      st->objmem[inst] = mem;
      for (int k = 1; k < o->K; ++k) {
        char *p = (char *)mem + (size_t)(k - 1) * (tb + 256);
        I.mtab[k] = (const float4 *)p;
        I.mkonst[k] = (const float2 *)(p + tb);
      }
    }
  }
  st->objs[inst] = *o;
  // the kernel variants of the kind and their occupancy
  int occ_plain = 1, occ_persist = 1;
  if (multi && variant_of(I).block != 0) {
    // several teams per CTA sharing the K tables in shared memory
    const Variant v = variant_of(I);
    int a = 0, b = 0;
    // the largest any state can need: a smaller value would fail another state's launch
    const int cap = (int)(I.obj == OBJ_MULTI_THG ? mt_smem_cap<OBJ_MULTI_THG>()
                                                 : mt_smem_cap<OBJ_MULTI_SHG>());
    for (const void *fn : {v.de, v.gwo})
      QPM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
    QPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, v.de, v.block, v.smem));
    QPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, v.gwo, v.block, v.smem));
    if (std::min(a, b) < 1) return fail(QPM_ERR_UNSUPPORTED, "qpm_set_objective: kernels do not fit");
    const int nteams = v.block / I.T;
    st->grid_mt[inst] = std::min((I.NP + nteams - 1) / nteams, std::min(a, b) * sm_count());
    // k_init and k_load_population keep one team per CTA
    int c = 0;
    QPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &c, I.obj == OBJ_MULTI_THG ? (const void *)k_init<false, OBJ_MULTI_THG>
                                   : (const void *)k_init<false, OBJ_MULTI_SHG>,
        I.T, smem_bytes_multi(I.T)));
    st->grid_plain[inst] = std::min(I.NP, std::max(1, c) * sm_count());
  } else if (multi) {
    const Variant v = variant_of(I);
    // the largest dynamic shared memory a team of up to 512 threads needs
    const int cap = (int)(sizeof(float4) * stg_f4_per_thread(true) * 512 + smem_bytes_multi(512));
    int a = 0, b = 0;
    for (const void *fn : {v.de, v.gwo}) {
      QPM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
      QPM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    (int)cudaSharedmemCarveoutDefault));
    }
    QPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, v.de, I.T, v.smem));
    QPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, v.gwo, I.T, v.smem));
    occ_plain = std::max(1, std::min(a, b));
    // ask for no more shared memory than the resident CTAs use, so that the rest of
    // the SM's L1 holds the K phasor tables; kept only if the occupancy stays
    int dev = 0, smem_sm = 0;
    QPM_CUDA(cudaGetDevice(&dev));
    QPM_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    const int pct = (int)std::min<size_t>(
        100, (100 * (size_t)occ_plain * (v.smem + 1024) + (size_t)smem_sm - 1) / (size_t)smem_sm);
    for (const void *fn : {v.de, v.gwo})
      QPM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
    int a2 = 0, b2 = 0;
    QPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a2, v.de, I.T, v.smem));
    QPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, v.gwo, I.T, v.smem));
    if (std::min(a2, b2) < occ_plain)
      for (const void *fn : {v.de, v.gwo})
        QPM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutDefault));
    st->grid_plain[inst] = std::min(I.NP, occ_plain * sm_count());
  } else {
    qpm_status r = occupancy(I, &occ_plain, &occ_persist);
    if (r != QPM_OK) return r;
    st->grid_plain[inst] = std::min(I.NP, occ_plain * sm_count());
    st->grid_persist[inst] = std::min(I.NP, occ_persist * sm_count());
  }
  if (st->gexec) {
    cudaGraphExecDestroy(st->gexec);
    st->gexec = nullptr;
    st->graph_n = -1;
  }
  QPM_CUDA(cudaMemcpy(st->d_insts + inst, &I, sizeof(InstDev), cudaMemcpyHostToDevice));
  return QPM_OK;
}

extern "C" qpm_status qpm_team_of(const qpm_state *st, int32_t inst, int32_t *team_out) {
  if (!st || !team_out || inst < 0 || inst >= st->n) return fail(QPM_ERR_ARG, "bad arguments");
  *team_out = st->h[inst].T;
  return QPM_OK;
}

extern "C" qpm_status qpm_instance_shape(const qpm_state *st, int32_t inst, int32_t *N_out,
                                         int32_t *NP_out, int32_t *G_out) {
  if (!st || inst < 0 || inst >= st->n) return fail(QPM_ERR_ARG, "bad state or instance");
  if (N_out) *N_out = st->h[inst].N;
  if (NP_out) *NP_out = st->h[inst].NP;
  if (G_out) *G_out = st->h[inst].G;
  return QPM_OK;
}

static __global__ void k_copy_F(InstDev I, float *out) {
  for (int g = threadIdx.x + blockIdx.x * blockDim.x; g <= I.G; g += blockDim.x * gridDim.x)
    out[g] = I.Fsched ? I.Fsched[g] : I.F;
}

extern "C" qpm_status qpm_get_F(qpm_state *st, int32_t inst, float *F_out, qpm_stream_t stream) {
  if (!st || inst < 0 || inst >= st->n || !F_out) return fail(QPM_ERR_ARG, "bad arguments");
  if (!st->inited) return fail(QPM_ERR_STATE, "qpm_init has not been called");
  const InstDev &I = st->h[inst];
  k_copy_F<<<(I.G + 256) / 256, 256, 0, (cudaStream_t)stream>>>(I, F_out);
  QPM_CUDA(cudaGetLastError());
  return QPM_OK;
}

extern "C" qpm_status qpm_set_F(qpm_state *st, int32_t inst, const float *F_in, qpm_stream_t stream) {
  if (!st || inst < 0 || inst >= st->n || !F_in) return fail(QPM_ERR_ARG, "bad arguments");
  const InstDev &I = st->h[inst];
  if (!I.Fsched) return fail(QPM_ERR_ARG, "qpm_set_F: constant F (f_schedule 0) has no history");
  QPM_CUDA(cudaMemcpyAsync(I.Fsched, F_in, sizeof(float) * (size_t)(I.G + 1),
                           cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return QPM_OK;
}

extern "C" qpm_status qpm_generation(const qpm_state *st, int32_t *g_out) {
  if (!st || !g_out) return fail(QPM_ERR_ARG, "NULL pointer");
  *g_out = st->g;
  return QPM_OK;
}

extern "C" qpm_status qpm_set_population(qpm_state *st, int32_t inst, const float *genes,
                                         int64_t ld, int32_t generation, qpm_stream_t stream) {
  if (!st || inst < 0 || inst >= st->n || !genes) return fail(QPM_ERR_ARG, "bad arguments");
  const InstDev &I = st->h[inst];
  if (ld < I.N) return fail(QPM_ERR_ARG, "ld < N");
  if (generation < 0 || generation > I.G) return fail(QPM_ERR_ARG, "generation outside [0, G]");
  if (!st->inited) return fail(QPM_ERR_STATE, "qpm_init has not been called");
  for (int k = 0; k < st->n; ++k)
    if (k != inst && generation != st->g)
      return fail(QPM_ERR_UNSUPPORTED, "all instances of a state share one generation count");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t sm = smem_bytes(I.T), smm = smem_bytes_multi(I.T);
  if (I.obj == OBJ_MULTI_THG)
    k_load_population<false, OBJ_MULTI_THG><<<st->grid_plain[inst], I.T, smm, s>>>(I, genes, ld, generation);
  else if (I.obj == OBJ_MULTI_SHG)
    k_load_population<false, OBJ_MULTI_SHG><<<st->grid_plain[inst], I.T, smm, s>>>(I, genes, ld, generation);
  else if (I.compensated)
    k_load_population<true><<<st->grid_plain[inst], I.T, sm, s>>>(I, genes, ld, generation);
  else
    k_load_population<false><<<st->grid_plain[inst], I.T, sm, s>>>(I, genes, ld, generation);
  QPM_CUDA(cudaGetLastError());
  st->g = generation;
  return QPM_OK;
}

extern "C" qpm_status qpm_get_population(qpm_state *st, int32_t inst, float *genes_out, int64_t ld,
                                         float *fit_out, float *d_eff_out, qpm_stream_t stream) {
  if (!st || inst < 0 || inst >= st->n) return fail(QPM_ERR_ARG, "bad state or instance");
  if (!st->inited) return fail(QPM_ERR_STATE, "qpm_init has not been called");
  const InstDev &I = st->h[inst];
  if (genes_out && ld < I.N) return fail(QPM_ERR_ARG, "ld < N");
  cudaStream_t s = (cudaStream_t)stream;
  if (genes_out) k_unpermute<<<I.NP, 256, 0, s>>>(I, -1, genes_out, ld);
  if (fit_out || d_eff_out)
    k_copy_fit<<<(I.NP + 255) / 256, 256, 0, s>>>(I, fit_out, (float2 *)d_eff_out);
  QPM_CUDA(cudaGetLastError());
  return QPM_OK;
}

extern "C" qpm_status qpm_get_best(qpm_state *st, int32_t inst, float *genes_out,
                                   double *d_eff64_out, float *fit_out, int32_t *index_out,
                                   qpm_stream_t stream) {
  if (!st || inst < 0 || inst >= st->n) return fail(QPM_ERR_ARG, "bad state or instance");
  if (!st->inited) return fail(QPM_ERR_STATE, "qpm_init has not been called");
  const InstDev &I = st->h[inst];
  cudaStream_t s = (cudaStream_t)stream;
  k_best<<<1, 256, 0, s>>>(I, index_out);
  if (d_eff64_out || fit_out) k_recheck64<<<1, 256, 0, s>>>(I, d_eff64_out, fit_out);
  if (genes_out) k_unpermute<<<1, 256, 0, s>>>(I, -2, genes_out, 0);
  QPM_CUDA(cudaGetLastError());
  return QPM_OK;
}

extern "C" qpm_status qpm_destroy(qpm_state *st) {
  if (!st) return QPM_OK;
  cudaDeviceSynchronize();
  if (st->gexec) cudaGraphExecDestroy(st->gexec);
  if (st->gexec_b) cudaGraphExecDestroy(st->gexec_b);
  if (st->polish) cudaFree(st->polish);
  for (void *p : st->objmem)
    if (p) cudaFree(p);
  if (st->cap_stream) cudaStreamDestroy(st->cap_stream);
  cudaFree(st->arena);
  delete st;
  return QPM_OK;
}

extern "C" qpm_status qpm_set_wait_timeout_ns(qpm_state *st, uint64_t ns) {
  if (!st) return fail(QPM_ERR_ARG, "NULL state");
  st->timeout_ns = ns;
  return QPM_OK;
}

extern "C" qpm_status qpm_polish_leaders(qpm_state *st, int32_t inst, int32_t steps, float lr,
                                         float tau, int32_t *accepted_out, qpm_stream_t stream) {
  if (!st || inst < 0 || inst >= st->n) return fail(QPM_ERR_ARG, "bad state or instance");
  if (!st->inited) return fail(QPM_ERR_STATE, "qpm_init has not been called");
  if (steps < 0 || !(lr >= 0.f) || !(tau > 0.f))
    return fail(QPM_ERR_ARG, "qpm_polish_leaders: need steps >= 0, lr >= 0, tau > 0");
  const InstDev &I = st->h[inst];
  if (I.obj != OBJ_THG)
    return fail(QPM_ERR_UNSUPPORTED, "qpm_polish_leaders: the cascaded |d_eff|^2 objective only");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t Np = (size_t)I.Npad;
  const size_t saved_bytes = align_up(3 * (size_t)qpm_relaxed_saved_floats(I.N) * sizeof(float), 256);
  const size_t need = 256 + align_up(3 * Np * sizeof(float), 256) * 2 + 256 + saved_bytes;
  if (st->polish_bytes < need) {
    if (st->polish) {
      QPM_CUDA(cudaDeviceSynchronize());
      QPM_CUDA(cudaFree(st->polish));
      st->polish = nullptr;
      st->polish_bytes = 0;
    }
    QPM_CUDA(cudaMalloc(&st->polish, need));
    st->polish_bytes = need;
  }
  char *p = (char *)st->polish;
  int32_t *lead = (int32_t *)p;
  float *theta = (float *)(p + 256);
  float *grad = (float *)(p + 256 + align_up(3 * Np * sizeof(float), 256));
  float *D = (float *)(p + 256 + 2 * align_up(3 * Np * sizeof(float), 256));
  float *saved = D + 256 / sizeof(float);
  k_polish_pick<<<1, 256, 0, s>>>(I, lead);
  k_polish_theta<<<3, 256, 0, s>>>(I, lead, tau, theta);
  QPM_CUDA(cudaGetLastError());
  const qpm_problem prob = st->probs[inst];
  for (int k = 0; k < steps; ++k) {
    qpm_status r = qpm_deff_relaxed_fwd(&prob, theta, (int64_t)Np, 3, D, nullptr, saved, stream);
    if (r != QPM_OK) return r;
    r = qpm_deff_relaxed_bwd(&prob, theta, (int64_t)Np, 3, D, saved, nullptr, grad, (int64_t)Np,
                             stream);
    if (r != QPM_OK) return r;
    k_polish_step<<<3, 256, 0, s>>>(I.N, (int64_t)Np, lr, theta, grad);
  }
  if (I.compensated)
    k_polish_accept<true><<<3, I.T, smem_bytes(I.T), s>>>(I, lead, tau, theta, accepted_out);
  else
    k_polish_accept<false><<<3, I.T, smem_bytes(I.T), s>>>(I, lead, tau, theta, accepted_out);
  QPM_CUDA(cudaGetLastError());
  return QPM_OK;
}

extern "C" qpm_status qpm_solve(const qpm_problem *prob, const qpm_params *params, int32_t mode,
                                float *best_genes_host, double *best_deff64_host,
                                float *best_fit_host) {
  if (!prob || !params) return fail(QPM_ERR_ARG, "qpm_solve: NULL pointer");
  qpm_state *st = nullptr;
  qpm_status r = qpm_create(prob, params, 1, &st);
  if (r != QPM_OK) return r;
  cudaStream_t s = st->cap_stream;
  float *dgenes = nullptr;
  double *dd = nullptr;
  float *df = nullptr;
  cudaError_t e = cudaMalloc(&dgenes, sizeof(float) * (size_t)prob->N + 64);
  if (e == cudaSuccess) e = cudaMalloc(&dd, 2 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&df, sizeof(float));
  if (e != cudaSuccess) r = cuda_fail(e, "cudaMalloc");
  if (r == QPM_OK && mode == QPM_RUN_GRAPH) mode = QPM_RUN_LAUNCHES;  // one pass: nothing to reuse
  if (r == QPM_OK) r = qpm_init(st, (qpm_stream_t)s);
  if (r == QPM_OK) r = qpm_run(st, params->G, mode, (qpm_stream_t)s);
  if (r == QPM_OK) r = qpm_get_best(st, 0, dgenes, dd, df, nullptr, (qpm_stream_t)s);
  if (r == QPM_OK && best_genes_host) {
    e = cudaMemcpyAsync(best_genes_host, dgenes, sizeof(float) * (size_t)prob->N,
                        cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) r = cuda_fail(e, "cudaMemcpyAsync");
  }
  if (r == QPM_OK && best_deff64_host) {
    e = cudaMemcpyAsync(best_deff64_host, dd, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) r = cuda_fail(e, "cudaMemcpyAsync");
  }
  if (r == QPM_OK && best_fit_host) {
    e = cudaMemcpyAsync(best_fit_host, df, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) r = cuda_fail(e, "cudaMemcpyAsync");
  }
  if (r == QPM_OK) {
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) r = cuda_fail(e, "cudaStreamSynchronize");
  }
  cudaFree(dgenes);
  cudaFree(dd);
  cudaFree(df);
  qpm_destroy(st);
  return r;
}
