// qpm_common.cuh -- device building blocks shared by the sm_103a kernels.
//
// Fitness (Sec. 2.1).  For piecewise-constant d over unit domains the double
// integral closes exactly:
//   d_eff = phi1 phi2 * sum_j a_j (sum_{m<j} b_m) + psi * sum_j d_j^2 p1_j p2_j
// with p1_m = e^{-i k1 m}, p2_m = e^{-i k2 m}, b_m = d_m p1_m, a_j = d_j p2_j,
// phi(k) = int_0^1 e^{-iks} ds, psi = int_0^1 e^{-i k2 s} int_0^s e^{-i k1 t} dt ds.
// The double sum is a reduction over the monoid of triples (A, B, C) =
// (sum a, sum b, sum_{m<j} a_j b_m) with
//   (A, B, C) (+) (A', B', C') = (A + A', B + B', C + C' + A' B),
// which is associative but not commutative, so every tree below keeps the
// left operand on the lower domain indices.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace qpm {

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, SC'11: 10 rounds, multipliers 0xD2511F53 and
// 0xCD9E8D57, Weyl key increments 0x9E3779B9 and 0xBB67AE85.  The round keys
// depend on the seed only, so a thread builds them once and reuses them.
struct PhiloxKey {
  uint32_t k0[10], k1[10];
};
__device__ __forceinline__ PhiloxKey philox_schedule(uint2 key) {
  PhiloxKey K;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    K.k0[r] = key.x + (uint32_t)r * 0x9E3779B9u;
    K.k1[r] = key.y + (uint32_t)r * 0xBB67AE85u;
  }
  return K;
}
__device__ __forceinline__ uint4 philox10(uint4 c, const PhiloxKey &K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ K.k0[r], (uint32_t)p1,
                   (uint32_t)(p0 >> 32) ^ c.w ^ K.k1[r], (uint32_t)p0);
  }
  return c;
}

// Random-number contract: key = seed, counter = (j/4, i, g, instance<<8 | tag);
// word j%4 of the output serves gene j.  Tags: 0 init (with g = 0xFFFFFFFF), 1 DE
// indices, 2 crossover, 3-5 GWO (one word per leader and gene: r1 its high, r2 its
// low 16 bits).
enum : uint32_t { TAG_INIT = 0, TAG_DEIDX = 1, TAG_CR = 2, TAG_GWO = 3, TAG_THETA = 16 };
constexpr uint32_t GEN_INIT = 0xFFFFFFFFu;  // the generation word of the initial draw

__device__ __forceinline__ uint4 rng4(const PhiloxKey &K, uint32_t inst, uint32_t tag, uint32_t g,
                                      uint32_t i, uint32_t jgroup) {
  return philox10(make_uint4(jgroup, i, g, (inst << 8) | tag), K);
}
// U in [0, 1) on the 24-bit grid (exact in FP32)
__device__ __forceinline__ float u24(uint32_t w) {
  return __fmul_rn(__uint2float_rn(w >> 8), 0x1p-24f);
}
// The GWO pair of one leader and gene: r1 = (w >> 16) 2^-16 and r2 = (w & 0xFFFF) 2^-16.
// The update needs r1 and C = 2 r2, built without a conversion: the 16 bits go to the
// top of the significand of a float in [1, 2) (for r1) or [2, 4) (for 2 r2), which is
// then 1 + r1 or 2 + 2 r2, and one exact subtraction leaves the value.
__device__ __forceinline__ float u16hi(uint32_t w) {  // r1
  return __fsub_rn(__uint_as_float(0x3F800000u | ((w >> 9) & 0x007FFF80u)), 1.0f);
}
__device__ __forceinline__ float twice_u16lo(uint32_t w) {  // 2 r2
  return __fsub_rn(__uint_as_float(0x40000000u | ((w << 7) & 0x007FFF80u)), 2.0f);
}
// crossover test U <= CR for U = (w >> 8) 2^-24 and CR in [0, 1], as one integer
// compare: (w >> 8) <= floor(2^24 CR)  <=>  w <= 256 floor(2^24 CR) + 255
static inline uint32_t cr_threshold(float CR) {
  const double k = floor((double)CR * 16777216.0);
  return k >= 16777216.0 ? 0xFFFFFFFFu : ((uint32_t)k << 8) | 0xFFu;
}
// index in [0, m): Lemire's multiply-shift
__device__ __forceinline__ uint32_t lemire(uint32_t w, uint32_t m) { return __umulhi(w, m); }

// DE rand/1 donors r1, r2, r3 (distinct, != i) and the forced crossover index jrand.
// Each draw is mapped onto the values not yet excluded by skipping the excluded
// ones in ascending order (a bijection, so every allowed value is equally likely).
__device__ __forceinline__ int4 de_indices(const PhiloxKey &K, uint32_t inst, uint32_t g, int i,
                                           int NP, int N) {
  const uint4 w = rng4(K, inst, TAG_DEIDX, g, (uint32_t)i, 0u);
  int r1 = (int)lemire(w.x, (uint32_t)(NP - 1));
  r1 += (r1 >= i);
  int e0 = min(i, r1), e1 = max(i, r1);
  int r2 = (int)lemire(w.y, (uint32_t)(NP - 2));
  r2 += (r2 >= e0);
  r2 += (r2 >= e1);
  // sorted triple of excluded values
  int s0 = e0, s1 = e1, s2 = r2;
  if (s2 < s1) { int t = s1; s1 = s2; s2 = t; }
  if (s1 < s0) { int t = s0; s0 = s1; s1 = t; }
  int r3 = (int)lemire(w.z, (uint32_t)(NP - 3));
  r3 += (r3 >= s0);
  r3 += (r3 >= s1);
  r3 += (r3 >= s2);
  return make_int4(r1, r2, r3, (int)lemire(w.w, (uint32_t)N));
}

__device__ __forceinline__ float clamp1(float v) { return fminf(fmaxf(v, -1.0f), 1.0f); }

// x / 3 rounded to nearest even, by Markstein's residual correction: q = RN(x r)
// with r = RN(1/3) is within one ulp of the quotient, the residual x - 3q is exact
// in one FMA, and RN(q + (x - 3q) r) is the correctly rounded quotient.  A zero
// residual (x = +-0 keeps its sign) or a NaN one (x = +-inf) returns q itself.
// qpm_selfcheck(0) compares it with the IEEE division over every float.
__device__ __forceinline__ float div3_rn(float x) {
  const float r = 0x1.555556p-2f;  // RN(1/3)
  const float q = __fmul_rn(x, r);
  const float rem = __fmaf_rn(-q, 3.0f, x);
  return fabsf(rem) > 0.0f ? __fmaf_rn(rem, r, q) : q;
}

// ------------------------------------------------------- asynchronous copies
// 16 bytes global -> shared through L2 (cp.async.cg), no registers held while in
// flight; bytes < 16 zero-fills the rest.  A thread sees its own copies after
// cp_async_wait; other threads need a barrier as well.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int bytes = 16) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(a), "l"(gmem), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most PENDING of this thread's committed groups are still in flight
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

// ------------------------------------------------------------------ the monoid
struct Mono {
  float2 A, B, C;
};
__device__ __forceinline__ Mono mono_zero() {
  Mono m;
  m.A = m.B = m.C = make_float2(0.f, 0.f);
  return m;
}
// L (+) R, L on the lower indices
__device__ __forceinline__ Mono mono_combine(const Mono &L, const Mono &R) {
  Mono o;
  o.A = make_float2(L.A.x + R.A.x, L.A.y + R.A.y);
  o.B = make_float2(L.B.x + R.B.x, L.B.y + R.B.y);
  float cr = L.C.x + R.C.x, ci = L.C.y + R.C.y;
  cr = fmaf(R.A.x, L.B.x, cr);
  cr = fmaf(-R.A.y, L.B.y, cr);
  ci = fmaf(R.A.x, L.B.y, ci);
  ci = fmaf(R.A.y, L.B.x, ci);
  o.C = make_float2(cr, ci);
  return o;
}

// append one domain with sign d (+-1.0f) and phasors p = (p1.re, p1.im, p2.re, p2.im)
__device__ __forceinline__ void mono_push(Mono &m, float d, const float4 &p) {
  const float ar = d * p.z, ai = d * p.w;  // a = d p2
  m.C.x = fmaf(ar, m.B.x, m.C.x);
  m.C.x = fmaf(-ai, m.B.y, m.C.x);
  m.C.y = fmaf(ar, m.B.y, m.C.y);
  m.C.y = fmaf(ai, m.B.x, m.C.y);
  m.A.x += ar;
  m.A.y += ai;
  m.B.x = fmaf(d, p.x, m.B.x);  // b = d p1, added after its use: strict prefix
  m.B.y = fmaf(d, p.y, m.B.y);
}

// compensated running triple: every running sum carries its Kahan compensation term
struct MonoK {
  Mono s;
  float2 eA, eB, eC;
};
__device__ __forceinline__ MonoK monok_zero() {
  MonoK m;
  m.s = mono_zero();
  m.eA = m.eB = m.eC = make_float2(0.f, 0.f);
  return m;
}
__device__ __forceinline__ void kahan_add(float &s, float &e, float x) {
  const float y = __fsub_rn(x, e);
  const float t = __fadd_rn(s, y);
  e = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}
__device__ __forceinline__ Mono monok_fold(const MonoK &m) {
  Mono o;
  o.A = make_float2(__fsub_rn(m.s.A.x, m.eA.x), __fsub_rn(m.s.A.y, m.eA.y));
  o.B = make_float2(__fsub_rn(m.s.B.x, m.eB.x), __fsub_rn(m.s.B.y, m.eB.y));
  o.C = make_float2(__fsub_rn(m.s.C.x, m.eC.x), __fsub_rn(m.s.C.y, m.eC.y));
  return o;
}

// Kahan-fold a plain partial R (the next domains) into the compensated running
// monoid m: C += C_R + A_R B, B += B_R, A += A_R, each sum with its compensation
__device__ __forceinline__ void monok_fold_in(MonoK &m, const Mono &R) {
  const float br = __fsub_rn(m.s.B.x, m.eB.x), bi = __fsub_rn(m.s.B.y, m.eB.y);
  const float xr = __fadd_rn(R.C.x, __fsub_rn(__fmul_rn(R.A.x, br), __fmul_rn(R.A.y, bi)));
  const float xi = __fadd_rn(R.C.y, __fadd_rn(__fmul_rn(R.A.x, bi), __fmul_rn(R.A.y, br)));
  kahan_add(m.s.C.x, m.eC.x, xr);
  kahan_add(m.s.C.y, m.eC.y, xi);
  kahan_add(m.s.B.x, m.eB.x, R.B.x);
  kahan_add(m.s.B.y, m.eB.y, R.B.y);
  kahan_add(m.s.A.x, m.eA.x, R.A.x);
  kahan_add(m.s.A.y, m.eA.y, R.A.y);
}

__device__ __forceinline__ Mono mono_shfl_down(const Mono &m, int s) {
  Mono o;
  o.A.x = __shfl_down_sync(0xffffffffu, m.A.x, s);
  o.A.y = __shfl_down_sync(0xffffffffu, m.A.y, s);
  o.B.x = __shfl_down_sync(0xffffffffu, m.B.x, s);
  o.B.y = __shfl_down_sync(0xffffffffu, m.B.y, s);
  o.C.x = __shfl_down_sync(0xffffffffu, m.C.x, s);
  o.C.y = __shfl_down_sync(0xffffffffu, m.C.y, s);
  return o;
}

// ordered reduction over the 32 lanes of a warp (lane 0 gets lanes 0..31 combined)
__device__ __forceinline__ Mono warp_reduce(Mono m) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
    const Mono r = mono_shfl_down(m, s);
    if ((lane & (2 * s - 1)) == 0) m = mono_combine(m, r);
  }
  return m;
}

// ordered reduction over the whole CTA (threads in index order); the result is
// valid in thread 0 only.  Each warp reduces by shuffles, lane 0 parks the warp
// total in sh[warp] (blockDim.x/32 entries) and thread 0 folds them in order.
// `sh` is reused by the next call: a caller that reduces again before any other
// CTA barrier must put a __syncthreads() in between.
__device__ __forceinline__ Mono block_reduce(Mono m, Mono *sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  m = warp_reduce(m);
  if (nw == 1) return m;
  if (lane == 0) sh[warp] = m;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < nw; ++w) m = mono_combine(m, sh[w]);
  return m;
}

// d_eff = phi1 phi2 C + cdiag  (cdiag = psi sum_j p1_j p2_j for +-1 domains)
__device__ __forceinline__ float2 deff_from(const Mono &m, float2 phi12, float2 cdiag) {
  return make_float2(fmaf(phi12.x, m.C.x, fmaf(-phi12.y, m.C.y, cdiag.x)),
                     fmaf(phi12.x, m.C.y, fmaf(phi12.y, m.C.x, cdiag.y)));
}
__device__ __forceinline__ float fit_of(float2 D) { return fmaf(D.x, D.x, D.y * D.y); }

// leader keys: larger key = larger f, ties -> lower index
__device__ __forceinline__ unsigned long long lead_key(float f, int i) {
  return ((unsigned long long)__float_as_uint(f) << 32) | (0xFFFFFFFFu - (uint32_t)i);
}
__device__ __forceinline__ int key_index(unsigned long long k) {
  return (int)(0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFull));
}
__device__ __forceinline__ void top3_insert(unsigned long long &k0, unsigned long long &k1,
                                            unsigned long long &k2, unsigned long long x) {
  if (x > k0) { k2 = k1; k1 = k0; k0 = x; }
  else if (x > k1) { k2 = k1; k1 = x; }
  else if (x > k2) { k2 = x; }
}
// The warp's three largest keys (keys distinct, 0 = none) from each lane's sorted
// triple k0 >= k1 >= k2, returned in every lane: three rounds of a two-word maximum
// (redux.sync on the high word, then on the low word among the lanes holding that
// high word), after each of which the lane holding the winner moves its triple up.
__device__ __forceinline__ void warp_top3(unsigned long long &k0, unsigned long long &k1,
                                          unsigned long long &k2) {
  unsigned long long out[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const uint32_t hi = (uint32_t)(k0 >> 32), lo = (uint32_t)k0;
    const uint32_t mhi = __reduce_max_sync(0xffffffffu, hi);
    const uint32_t mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
    out[r] = ((unsigned long long)mhi << 32) | mlo;
    if (k0 != 0ull && hi == mhi && lo == mlo) {
      k0 = k1;
      k1 = k2;
      k2 = 0ull;
    }
  }
  k0 = out[0];
  k1 = out[1];
  k2 = out[2];
}

// ----------------------------------------------- FP64 phase argument reduction
// r = x - 2 pi n with n = rint(x / 2pi), 2pi split into a double-double
__device__ __forceinline__ double reduce_2pi(double x) {
  const double TWO_PI_HI = 6.283185307179586232;
  const double TWO_PI_LO = 2.4492935982947064e-16;
  const double INV_TWO_PI = 0.15915494309189533577;
  const double n = rint(x * INV_TWO_PI);
  double r = fma(-n, TWO_PI_HI, x);
  r = fma(-n, TWO_PI_LO, r);
  return r;
}

// ------------------------------------------------------- bounded device waits
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

}  // namespace qpm
