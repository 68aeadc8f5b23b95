// qpm_eval.cu -- fitness of caller-supplied sign sequences (Sec. 2.1).
//
// Work split: a CTA takes 32 rows and one segment of the domains.  It walks the
// segment in steps of 256 domains: the 32 x 256 genes (or their sign words) are
// copied into shared memory with fully coalesced loads, the 256 phasors beside
// them, then warp w scans domains [32w, 32w + 32) of the step for all 32 rows
// (lane = row, so each phasor read is a broadcast) and the 8 warp partials are
// combined in index order into the CTA's running monoid (A, B, C).  A second
// kernel combines the S segment partials of every row in index order and closes
// d_eff = phi1 phi2 C + cdiag.
#include <math.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "qpm_common.cuh"
#include "qpm_internal.h"

namespace qpm {

static constexpr int EV_WARPS = 8;
static constexpr int EV_STEP = 256;  // domains staged per step (32 per warp)

// genes of the step as float4 [column c4 = d/4][row], the row xor-swizzled by the
// low 3 bits of the column: 8 consecutive columns of one row (a quarter-warp of
// the coalesced staging stores) and 8 rows of one column (a quarter-warp of the
// scan reads) both fall into 8 different 16-byte bank groups
__device__ __forceinline__ int tile4_idx(int c4, int row) { return c4 * 32 + (row ^ (c4 & 7)); }

// the genes (or sign word) of step `ms` that this thread stages, loaded into
// registers ahead of time
template <int KIND>
struct StepRegs {
  float4 v[8];
  uint32_t w;
  float4 p;
};

template <int KIND>
__device__ __forceinline__ void load_step(const void *src, int64_t ld, const EvalShape &sh,
                                          const float4 *table, int r0, int ms, StepRegs<KIND> &R) {
  const int m = ms + threadIdx.x;
  R.p = m < sh.N ? __ldg(table + m) : make_float4(0.f, 0.f, 0.f, 0.f);
  if (KIND == 2) {
    const int row = threadIdx.x >> 3, wd = threadIdx.x & 7;
    const int gr = r0 + row;
    R.w = 0u;
    if (gr < sh.NP && ms + wd * 32 < sh.N)
      R.w = __ldg((const uint32_t *)src + (int64_t)gr * ld + (ms >> 5) + wd);
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int f = threadIdx.x + k * EV_WARPS * 32;  // float4 slot: 32 rows x 64 columns
      const int row = f >> 6, c4 = f & 63;
      const int gr = r0 + row, mm = ms + 4 * c4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gr < sh.NP) {
        const float *rp = (const float *)src + (int64_t)gr * ld;
        if (KIND == 0 && mm + 4 <= sh.N) {
          v = __ldg((const float4 *)(rp + mm));
        } else {
          if (mm < sh.N) v.x = __ldg(rp + mm);
          if (mm + 1 < sh.N) v.y = __ldg(rp + mm + 1);
          if (mm + 2 < sh.N) v.z = __ldg(rp + mm + 2);
          if (mm + 3 < sh.N) v.w = __ldg(rp + mm + 3);
        }
      }
      R.v[k] = v;
    }
  }
}

// partial monoids, structure of arrays: part[(comp * S + s) * NPpad + i], comp in A,B,C
template <int KIND, bool COMP>  // KIND 0: float genes (vector loads), 1: float genes (scalar), 2: packed bits
static __global__ void __launch_bounds__(EV_WARPS * 32)
    k_eval_seg(const void *__restrict__ src, int64_t ld, EvalShape sh,
               const float4 *__restrict__ table, float2 *__restrict__ part) {
  __shared__ float4 tile4[EV_STEP / 4 * 32];         // genes, or sign words for KIND 2
  __shared__ float4 tb[EV_STEP];                    // phasors of the step
  __shared__ Mono wpart[EV_WARPS][32];              // per-warp partials of the step
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int s = blockIdx.x, grp = blockIdx.y;
  const int r0 = grp * 32;
  const int m0 = s * sh.L;
  const int m1 = min(sh.N, m0 + sh.L);
  Mono run = mono_zero();   // running monoid of the segment (warp 0, lane = row)
  MonoK runk = monok_zero();
  StepRegs<KIND> R;
  if (m0 < m1) load_step<KIND>(src, ld, sh, table, r0, m0, R);
  for (int ms = m0; ms < m1; ms += EV_STEP) {
    __syncthreads();  // the previous step's tile and partials have been consumed
    tb[threadIdx.x] = R.p;
    if (KIND == 2) {
      ((uint32_t *)tile4)[threadIdx.x] = R.w;  // [row][8 words]
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int f = threadIdx.x + k * EV_WARPS * 32;
        tile4[tile4_idx(f & 63, f >> 6)] = R.v[k];
      }
    }
    __syncthreads();
    // the next step's loads are in flight while this step is scanned
    if (ms + EV_STEP < m1) load_step<KIND>(src, ld, sh, table, r0, ms + EV_STEP, R);
    // ---- warp w: domains [32w, 32w + 32) of the step for rows r0 + lane
    Mono acc = mono_zero();
    const int d0 = warp * 32;
    if (KIND == 2) {
      const uint32_t w = ((const uint32_t *)tile4)[lane * 8 + warp];
#pragma unroll 8
      for (int e = 0; e < 32; ++e) mono_push(acc, ((w >> e) & 1u) ? -1.0f : 1.0f, tb[d0 + e]);
    } else {
#pragma unroll 2
      for (int e4 = 0; e4 < 8; ++e4) {
        const int c4 = (d0 >> 2) + e4;
        const float4 x = tile4[tile4_idx(c4, lane)];
        const float4 *pp = tb + 4 * c4;
        mono_push(acc, x.x < 0.f ? -1.f : 1.f, pp[0]);
        mono_push(acc, x.y < 0.f ? -1.f : 1.f, pp[1]);
        mono_push(acc, x.z < 0.f ? -1.f : 1.f, pp[2]);
        mono_push(acc, x.w < 0.f ? -1.f : 1.f, pp[3]);
      }
    }
    wpart[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int w = 0; w < EV_WARPS; ++w) {
        if (COMP) monok_fold_in(runk, wpart[w][lane]);
        else run = mono_combine(run, wpart[w][lane]);
      }
    }
  }
  if (warp == 0) {
    if (COMP) run = monok_fold(runk);
    const size_t stride = (size_t)sh.S * sh.NPpad;
    const size_t o = (size_t)s * sh.NPpad + r0 + lane;
    part[o] = run.A;
    part[stride + o] = run.B;
    part[2 * stride + o] = run.C;
  }
}

template <bool COMP>
static __global__ void k_eval_combine(EvalShape sh, const float2 *__restrict__ part,
                                      const float2 *__restrict__ konst, float2 *__restrict__ deff,
                                      float *__restrict__ fit) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= sh.NP) return;
  const size_t stride = (size_t)sh.S * sh.NPpad;
  Mono acc = mono_zero();
  float2 eB = make_float2(0.f, 0.f), eC = make_float2(0.f, 0.f);
  for (int s = 0; s < sh.S; ++s) {
    const size_t o = (size_t)s * sh.NPpad + i;
    Mono r;
    r.A = part[o];
    r.B = part[stride + o];
    r.C = part[2 * stride + o];
    if (COMP) {
      // C += C' + A' B and B += B' with Kahan compensation on C and B
      const float br = __fsub_rn(acc.B.x, eB.x), bi = __fsub_rn(acc.B.y, eB.y);
      const float xr = __fadd_rn(r.C.x, __fsub_rn(__fmul_rn(r.A.x, br), __fmul_rn(r.A.y, bi)));
      const float xi = __fadd_rn(r.C.y, __fadd_rn(__fmul_rn(r.A.x, bi), __fmul_rn(r.A.y, br)));
      kahan_add(acc.C.x, eC.x, xr);
      kahan_add(acc.C.y, eC.y, xi);
      kahan_add(acc.B.x, eB.x, r.B.x);
      kahan_add(acc.B.y, eB.y, r.B.y);
      acc.A.x += r.A.x;
      acc.A.y += r.A.y;
    } else {
      acc = mono_combine(acc, r);
    }
  }
  if (COMP) acc.C = make_float2(__fsub_rn(acc.C.x, eC.x), __fsub_rn(acc.C.y, eC.y));
  const float2 D = deff_from(acc, konst[0], konst[1]);
  deff[i] = D;
  if (fit) fit[i] = fit_of(D);
}

// ------------------------------------------------------------- caches (host)
namespace {
struct TableEntry {
  float4 *table = nullptr;
  double2 *part = nullptr;
  float2 *konst = nullptr;
  cudaEvent_t ready = nullptr;
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

// phasor table in natural order for (device, problem); built on `stream` on a miss
qpm_status get_table(const qpm_problem *p, cudaStream_t stream, const float4 **table,
                     const float2 **konst) {
  int dev = 0;
  QPM_CUDA(cudaGetDevice(&dev));
  auto key = std::make_tuple(dev, p->N, p->kappa1, p->kappa2);
  auto it = g_tables.find(key);
  if (it == g_tables.end()) {
    if (g_tables.size() >= MAX_TABLES) {
      qpm_status st = release_device_caches(dev);
      if (st != QPM_OK) return st;
    }
    TableEntry e;
    const int32_t Npad = (p->N + 3) & ~3;
    QPM_CUDA(cudaMalloc(&e.table, sizeof(float4) * (size_t)Npad));
    QPM_CUDA(cudaMalloc(&e.part, sizeof(double2) * (size_t)table_part_count(Npad)));
    QPM_CUDA(cudaMalloc(&e.konst, sizeof(float2) * 4));
    QPM_CUDA(cudaEventCreateWithFlags(&e.ready, cudaEventDisableTiming));
    TableSpec s{p->N, Npad, 1, Npad, p->kappa1, p->kappa2};
    qpm_status st = launch_table(s, e.table, e.part, e.konst, nullptr, stream);
    if (st != QPM_OK) return st;
    QPM_CUDA(cudaEventRecord(e.ready, stream));
    it = g_tables.emplace(key, e).first;
  } else {
    QPM_CUDA(cudaStreamWaitEvent(stream, it->second.ready, 0));
  }
  *table = it->second.table;
  *konst = it->second.konst;
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

EvalShape eval_shape(int NP, int N) {
  EvalShape sh;
  sh.NP = NP;
  sh.N = N;
  sh.groups = (NP + 31) / 32;
  sh.NPpad = sh.groups * 32;
  const int target_ctas = sm_count() * 6;
  int S = (target_ctas + sh.groups - 1) / sh.groups;
  const int maxS = (N + EV_STEP - 1) / EV_STEP;  // at least one step per segment
  if (S > maxS) S = maxS;
  if (S < 1) S = 1;
  int L = (N + S - 1) / S;
  L = (L + EV_STEP - 1) / EV_STEP * EV_STEP;
  sh.S = (N + L - 1) / L;
  sh.L = L;
  return sh;
}

static qpm_status eval_common(const qpm_problem *prob, const void *src, int64_t ld, int32_t NP,
                              int kind, float *d_eff, float *fit, int32_t comp,
                              cudaStream_t stream) {
  if (!prob || !src || !d_eff) return fail(QPM_ERR_ARG, "qpm_eval: NULL pointer");
  if (prob->N < 1 || NP < 1) return fail(QPM_ERR_ARG, "qpm_eval: need N >= 1 and NP >= 1");
  if (prob->N > (1 << 28)) return fail(QPM_ERR_UNSUPPORTED, "qpm_eval: N too large");
  if (kind == 2 ? (ld < (prob->N + 31) / 32) : (ld < prob->N))
    return fail(QPM_ERR_ARG, "qpm_eval: leading dimension smaller than the row");
  std::lock_guard<std::mutex> lock(g_mu);
  const float4 *table;
  const float2 *konst;
  qpm_status st = get_table(prob, stream, &table, &konst);
  if (st != QPM_OK) return st;
  const EvalShape sh = eval_shape(NP, prob->N);
  void *scratch;
  st = get_scratch(stream, sizeof(float2) * 3 * (size_t)sh.S * sh.NPpad, &scratch);
  if (st != QPM_OK) return st;
  float2 *part = (float2 *)scratch;
  dim3 grid(sh.S, sh.groups);
  if (kind != 2 && (ld % 4 == 0) && (((uintptr_t)src & 15) == 0)) kind = 0;
  else if (kind != 2) kind = 1;
#define QPM_EV(K, C) k_eval_seg<K, C><<<grid, EV_WARPS * 32, 0, stream>>>(src, ld, sh, table, part)
  if (kind == 0) { if (comp) QPM_EV(0, true); else QPM_EV(0, false); }
  else if (kind == 1) { if (comp) QPM_EV(1, true); else QPM_EV(1, false); }
  else { if (comp) QPM_EV(2, true); else QPM_EV(2, false); }
#undef QPM_EV
  QPM_CUDA(cudaGetLastError());
  const int cb = 128;
  if (comp)
    k_eval_combine<true><<<(NP + cb - 1) / cb, cb, 0, stream>>>(sh, part, konst, (float2 *)d_eff, fit);
  else
    k_eval_combine<false><<<(NP + cb - 1) / cb, cb, 0, stream>>>(sh, part, konst, (float2 *)d_eff, fit);
  QPM_CUDA(cudaGetLastError());
  return QPM_OK;
}


// ---------------------------------------------------------------------------
// Allocation-free variant of qpm_eval.  For callers that must not allocate
// device memory: code running where cudaMalloc is not allowed or not wanted,
// e.g. while a CUDA stream is being captured into a graph, inside a host
// callback, under an external allocator that owns all device memory, or on a
// real-time path where an allocation's implicit device synchronisation is not
// acceptable.  Its scratch (phasor table, table reduction, segment partials)
// lives in one file-scope device array of fixed size that every GPU loading
// this library holds until the process exits.
// ---------------------------------------------------------------------------
static constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)8 << 20;  // 8 MiB
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
    return fail(QPM_ERR_ARG, "qpm_eval_noalloc: problem exceeds the fixed scratch (8 MiB)");
  const EvalShape sh = eval_shape(NP, prob->N);
  const int32_t Npad = (prob->N + 3) & ~3;
  const size_t b_table = up256(sizeof(float4) * (size_t)Npad);
  const size_t b_tpart = up256(sizeof(double2) * (size_t)table_part_count(Npad));
  const size_t b_konst = 256;
  const size_t b_part = up256(sizeof(float2) * 3 * (size_t)sh.S * sh.NPpad);
  const size_t need = b_table + b_tpart + b_konst + b_part;
  if (need > NOALLOC_SCRATCH_BYTES)
    return fail(QPM_ERR_ARG, "qpm_eval_noalloc: N and NP need " + std::to_string(need) +
                                 " bytes of scratch, more than the fixed 8 MiB (8388608)");
  void *base = nullptr;
  qpm_status st = noalloc_base(&base);
  if (st != QPM_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  char *p = (char *)base;
  float4 *table = (float4 *)p;
  double2 *tpart = (double2 *)(p + b_table);
  float2 *konst = (float2 *)(p + b_table + b_tpart);
  float2 *part = (float2 *)(p + b_table + b_tpart + b_konst);
  // every word read below is written first in this call (table, its partial
  // sums, every segment partial of every padded row), so nothing needs zeroing
  TableSpec ts{prob->N, Npad, 1, Npad, prob->kappa1, prob->kappa2};
  st = launch_table(ts, table, tpart, konst, nullptr, s);
  if (st != QPM_OK) return st;
  dim3 grid(sh.S, sh.groups);
  const bool vec = (ld % 4 == 0) && (((uintptr_t)genes & 15) == 0);
  if (vec) {
    if (compensated) k_eval_seg<0, true><<<grid, EV_WARPS * 32, 0, s>>>(genes, ld, sh, table, part);
    else k_eval_seg<0, false><<<grid, EV_WARPS * 32, 0, s>>>(genes, ld, sh, table, part);
  } else {
    if (compensated) k_eval_seg<1, true><<<grid, EV_WARPS * 32, 0, s>>>(genes, ld, sh, table, part);
    else k_eval_seg<1, false><<<grid, EV_WARPS * 32, 0, s>>>(genes, ld, sh, table, part);
  }
  QPM_CUDA(cudaGetLastError());
  const int cb = 128;
  if (compensated)
    k_eval_combine<true><<<(NP + cb - 1) / cb, cb, 0, s>>>(sh, part, konst, (float2 *)d_eff, fit);
  else
    k_eval_combine<false><<<(NP + cb - 1) / cb, cb, 0, s>>>(sh, part, konst, (float2 *)d_eff, fit);
  QPM_CUDA(cudaGetLastError());
  return QPM_OK;
}

qpm_status qpm::cached_table(const qpm_problem *p, cudaStream_t stream, const float4 **table,
                             const float2 **konst) {
  std::lock_guard<std::mutex> lock(g_mu);
  return get_table(p, stream, table, konst);
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
