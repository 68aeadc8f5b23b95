// qpm_peaks.cu -- issue-rate microbenchmarks for the ALU roofline, and exhaustive
// self-checks of the library's own arithmetic helpers against CUDA's.
//
// The generation step is bound by FP32 and integer issue (fitness monoid steps,
// Philox rounds), for which no vendor figure is measured on this machine.  Each
// kernel runs PK_CHAINS independent dependency chains of one instruction kind per
// thread, long enough that launch and tail effects vanish, and writes its result
// only under a condition the chains never meet, so nothing is optimised away.
// Lane-ops/s = threads x iterations x chains x ops per chain step / elapsed time,
// with the op counts of the roofline's own convention: a 32 x 32 -> 64 multiply
// counts 2, a three-input logic op 1, an FFMA 1; kind 3 reports whole calls of the
// generator's Philox4x32-10 per second.
#include <cuda_runtime.h>

#include <vector>

#include "qpm_common.cuh"
#include "qpm_internal.h"
#include "qpm_sync.cuh"

namespace qpm {

static constexpr int PK_CHAINS = 8;
static constexpr int PK_ITERS = 4096;
static constexpr int PK_THREADS = 512;

// x <- x * a + b in FP32 (one FFMA per chain and iteration)
static __global__ void __launch_bounds__(PK_THREADS) k_peak_ffma(float a, float b, float *sink) {
  float x[PK_CHAINS];
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) x[c] = (float)(threadIdx.x + c);
  for (int it = 0; it < PK_ITERS; ++it) {
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
  if (s == -1.2345f) sink[blockIdx.x] = s;
}

// x <- hi(x * m) ^ lo(x * m): the 32 x 32 -> 64 multiply of a Philox round
// (one wide multiply and one xor per chain and iteration)
static __global__ void __launch_bounds__(PK_THREADS) k_peak_imul(uint32_t m, uint32_t *sink) {
  uint32_t x[PK_CHAINS];
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) x[c] = threadIdx.x * 2654435761u + c;
  for (int it = 0; it < PK_ITERS; ++it) {
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) {
      const uint64_t p = (uint64_t)x[c] * m;
      x[c] = (uint32_t)(p >> 32) ^ (uint32_t)p;
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) s ^= x[c];
  if (s == 0x9E3779B9u && m == 0u) sink[blockIdx.x] = s;
}

// x <- x ^ y ^ k: a three-input logic op (one LOP3 per chain and iteration)
static __global__ void __launch_bounds__(PK_THREADS) k_peak_lop3(uint32_t k, uint32_t *sink) {
  uint32_t x[PK_CHAINS], y[PK_CHAINS];
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) {
    x[c] = threadIdx.x + c;
    y[c] = (threadIdx.x << 3) ^ (uint32_t)c * 0x85EBCA6Bu;
  }
  for (int it = 0; it < PK_ITERS; ++it) {
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) {
      x[c] = x[c] ^ y[c] ^ (k + (uint32_t)it);
      y[c] = y[c] ^ x[c] ^ k;
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) s ^= x[c] ^ y[c];
  if (s == 0x12345678u && k == 0u) sink[blockIdx.x] = s;
}

// whole Philox4x32-10 calls of the library's generator (the counter of each chain
// is the previous output, so nothing is hoisted); one "op" per call here
static constexpr int PK_PHILOX_ITERS = 256;
static __global__ void __launch_bounds__(PK_THREADS) k_peak_philox(uint2 key, uint32_t *sink) {
  const PhiloxKey K = philox_schedule(key);
  uint4 c[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) c[k] = make_uint4(threadIdx.x, blockIdx.x, k, 7u);
  for (int it = 0; it < PK_PHILOX_ITERS; ++it) {
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k] = philox10(c[k], K);
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) s ^= c[k].x ^ c[k].y ^ c[k].z ^ c[k].w;
  if (s == 0x2545F491u && key.x == 0u) sink[blockIdx.x] = s;
}

// every float bit pattern x: div3_rn(x) against the IEEE division x / 3 (bitwise;
// two NaNs agree); per-thread counts and first bad pattern, one atomic each
static __global__ void k_check_div3(unsigned long long *bad, uint32_t *first) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  unsigned long long n = 0;
  uint32_t f = 0xFFFFFFFFu;
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < (1ull << 32); b += stride) {
    const float x = __uint_as_float((uint32_t)b);
    const float q = div3_rn(x), ref = __fdiv_rn(x, 3.0f);
    const bool same = __float_as_uint(q) == __float_as_uint(ref) || (q != q && ref != ref);
    if (!same) {
      ++n;
      f = min(f, (uint32_t)b);
    }
  }
  if (n) {
    atomicAdd(bad, n);
    atomicMin(first, f);
  }
}

// every 32-bit word w: the GWO's r1 and 2 r2 built in the significand against the
// same values through conversions, r = (16-bit half) 2^-16 (bitwise)
static __global__ void k_check_gwo_uniforms(unsigned long long *bad, uint32_t *first) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  unsigned long long n = 0;
  uint32_t f = 0xFFFFFFFFu;
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < (1ull << 32); b += stride) {
    const uint32_t w = (uint32_t)b;
    const float r1 = __fmul_rn(__uint2float_rn(w >> 16), 0x1p-16f);
    const float r2 = __fmul_rn(__uint2float_rn(w & 0xFFFFu), 0x1p-16f);
    const bool same = __float_as_uint(u16hi(w)) == __float_as_uint(r1) &&
                      __float_as_uint(twice_u16lo(w)) == __float_as_uint(__fmul_rn(2.0f, r2));
    if (!same) {
      ++n;
      f = min(f, w);
    }
  }
  if (n) {
    atomicAdd(bad, n);
    atomicMin(first, f);
  }
}

// every 32-bit word w and each of ncr crossover rates: the integer test against
// cr_threshold(CR) against U <= CR with U = (w >> 8) 2^-24 in FP32
struct CrCases {
  float cr[8];
  uint32_t thr[8];
  int n;
};
static __global__ void k_check_cr(CrCases c, unsigned long long *bad, uint32_t *first) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  unsigned long long n = 0;
  uint32_t f = 0xFFFFFFFFu;
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; b < (1ull << 32); b += stride) {
    const uint32_t w = (uint32_t)b;
    const float u = u24(w);
    for (int k = 0; k < c.n; ++k) {
      if ((w <= c.thr[k]) != (u <= c.cr[k])) {
        ++n;
        f = min(f, w);
      }
    }
  }
  if (n) {
    atomicAdd(bad, n);
    atomicMin(first, f);
  }
}

}  // namespace qpm

using namespace qpm;

extern "C" qpm_status qpm_selfcheck(int32_t kind, uint64_t *mismatches, uint32_t *first_bad,
                                    qpm_stream_t stream) {
  if (!mismatches || !first_bad || kind < 0 || kind > 2)
    return fail(QPM_ERR_ARG, "qpm_selfcheck: kind must be 0, 1 or 2 and both outputs non-NULL");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long *bad = nullptr;
  QPM_CUDA(cudaMalloc(&bad, sizeof(unsigned long long) + sizeof(uint32_t)));
  uint32_t *first = (uint32_t *)(bad + 1);
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(first, 0xFF, sizeof(uint32_t), s);
  if (e == cudaSuccess) {
    const int blocks = sm_count() * 8;
    if (kind == 0) {
      k_check_div3<<<blocks, 256, 0, s>>>(bad, first);
    } else if (kind == 1) {
      k_check_gwo_uniforms<<<blocks, 256, 0, s>>>(bad, first);
    } else {
      // the edges of [0, 1], the rate of the workloads and its FP32 neighbours
      const float cr[8] = {0.0f, 0x1p-24f, 0x1.8p-24f, 0.5f, nextafterf(0.9f, 0.0f), 0.9f,
                           nextafterf(0.9f, 1.0f), 1.0f};
      CrCases c;
      c.n = 8;
      for (int k = 0; k < 8; ++k) {
        c.cr[k] = cr[k];
        c.thr[k] = cr_threshold(cr[k]);
      }
      k_check_cr<<<blocks, 256, 0, s>>>(c, bad, first);
    }
    e = cudaGetLastError();
  }
  unsigned long long h = 0;
  uint32_t hf = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, bad, sizeof h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hf, first, sizeof hf, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(bad);
  if (e != cudaSuccess) return cuda_fail(e, "qpm_selfcheck");
  *mismatches = (uint64_t)h;
  *first_bad = hf;
  return QPM_OK;
}

extern "C" qpm_status qpm_measure_issue_peak(int32_t kind, double *lane_ops_per_s,
                                             qpm_stream_t stream) {
  if (!lane_ops_per_s || kind < 0 || kind > 3)
    return fail(QPM_ERR_ARG, "qpm_measure_issue_peak: kind must be 0, 1, 2 or 3");
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = sm_count() * 4;  // 2048 threads per SM: every scheduler full
  void *sink = nullptr;
  QPM_CUDA(cudaMalloc(&sink, sizeof(uint32_t) * blocks));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f;
  // ops per chain step: FFMA 1; wide multiply (2) + xor (1); two three-input xors;
  // kind 3 counts whole Philox calls (4 chains of PK_PHILOX_ITERS)
  const double per_step = kind == 0 ? 1.0 : (kind == 1 ? 3.0 : 2.0);
  const double per_thread = kind == 3 ? (double)PK_PHILOX_ITERS * 4
                                      : (double)PK_ITERS * PK_CHAINS * per_step;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {  // the first launch warms up
    e = cudaEventRecord(e0, s);
    if (kind == 0) k_peak_ffma<<<blocks, PK_THREADS, 0, s>>>(1.000001f, 1e-7f, (float *)sink);
    else if (kind == 1) k_peak_imul<<<blocks, PK_THREADS, 0, s>>>(0xD2511F53u, (uint32_t *)sink);
    else if (kind == 2) k_peak_lop3<<<blocks, PK_THREADS, 0, s>>>(0xCD9E8D57u, (uint32_t *)sink);
    else k_peak_philox<<<blocks, PK_THREADS, 0, s>>>(make_uint2(1u, 2u), (uint32_t *)sink);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "qpm_measure_issue_peak");
  *lane_ops_per_s = (double)blocks * PK_THREADS * per_thread / (ms * 1e-3);
  return QPM_OK;
}

// ------------------------------------------------------- latency probes
// The latency floor of a generation of the persistent kernel: its two grid barriers
// and its dependent L2 round trips (donor rows, survivor keys, leader rows).
namespace qpm {

static constexpr int LP_THREADS = 256;  // the team width of the 1000-domain workload

// `reps` grid barriers of the persistent kernel's own form, back to back
static __global__ void __launch_bounds__(LP_THREADS) k_probe_barrier(Barrier b, int reps) {
  unsigned target = 0;
  for (int r = 0; r < reps; ++r)
    if (!grid_sync(b, target)) return;
}

// The ways a grid could synchronise, for comparison with the barrier above (reps
// rounds each, every wait bounded by an iteration count that records QPM_ERR_TIMEOUT):
//   2: the same counter barrier with relaxed arrival and polling -- how fast an
//      arrival reaches the pollers at all, without the ordering the kernel needs;
//   3: a gpu-scope fence between two CTA barriers, no cross-CTA wait -- the price of
//      the ordering alone;
//   4: an all-to-all exchange without a counter: every CTA publishes a round-tagged
//      8-byte word (single-copy atomic, relaxed) and its threads poll the words of
//      all CTAs, one thread per word (what a fence-free leader search would need).
// words: [2][ctas] u64, zero before the launch (rounds alternate between the halves,
// so a fast CTA never overwrites a word a slow one still waits for).
static constexpr unsigned LP_SPIN_LIMIT = 1u << 22;
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
static __global__ void __launch_bounds__(LP_THREADS)
    k_probe_sync(Barrier b, int kind, unsigned long long *words, int reps) {
  __shared__ int bad;
  unsigned target = 0;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int r = 0; r < reps; ++r) {
    if (kind == 2) {
      __syncthreads();
      target += gridDim.x;
      if (threadIdx.x == 0) {
        asm volatile("red.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(b.count) : "memory");
        unsigned it = 0;
        while ((int)(ld_relaxed_u32(b.count) - target) < 0)
          if (++it > LP_SPIN_LIMIT) {
            atomicCAS(b.err, 0, (int)QPM_ERR_TIMEOUT);
            bad = 1;
            break;
          }
      }
      __syncthreads();
    } else if (kind == 3) {
      __syncthreads();
      if (threadIdx.x == 0) asm volatile("fence.acq_rel.gpu;" ::: "memory");
      __syncthreads();
    } else {
      const unsigned tag = (unsigned)r + 1u;
      unsigned long long *half = words + (size_t)(r & 1) * gridDim.x;
      if (threadIdx.x == 0) st_relaxed_u64(half + blockIdx.x, ((unsigned long long)tag << 32) | blockIdx.x);
      for (unsigned c = threadIdx.x; c < gridDim.x; c += blockDim.x) {
        unsigned it = 0;
        while ((unsigned)(ld_relaxed_u64(half + c) >> 32) != tag)
          if (++it > LP_SPIN_LIMIT) {
            atomicCAS(b.err, 0, (int)QPM_ERR_TIMEOUT);
            bad = 1;
            break;
          }
      }
      __syncthreads();
    }
    if (bad) return;
  }
}

// one thread follows a cyclic permutation with L2-cached loads: every load depends
// on the one before, so the time per step is the latency of a load served by L2
static __global__ void k_probe_chase(const uint32_t *__restrict__ next, int steps,
                                     uint32_t *sink) {
  uint32_t i = 0;
  for (int s = 0; s < steps; ++s) i = __ldcg(next + i);
  if (i == 0xFFFFFFFFu) *sink = i;
}

}  // namespace qpm

extern "C" qpm_status qpm_measure_latency(int32_t kind, int32_t ctas, double *ns_out,
                                          qpm_stream_t stream) {
  using namespace qpm;
  if (!ns_out) return fail(QPM_ERR_ARG, "qpm_measure_latency: NULL output");
  if (kind < 0 || kind > 4) return fail(QPM_ERR_ARG, "qpm_measure_latency: kind outside [0, 4]");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  QPM_CUDA(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ce, "cudaEventCreate");
  }
  qpm_status st = QPM_OK;
  void *buf = nullptr;
  // elapsed ms of one launch made by `launch`
  auto timed = [&](auto launch, float *ms) -> qpm_status {
    cudaError_t e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    return e == cudaSuccess ? QPM_OK : cuda_fail(e, "latency probe launch");
  };
  if (kind != 1) {
    const void *fn = kind == 0 ? (const void *)k_probe_barrier : (const void *)k_probe_sync;
    int occ = 0;
    ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, LP_THREADS, 0);
    if (ce != cudaSuccess) st = cuda_fail(ce, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    else if (ctas < 1 || ctas > occ * sm_count())
      st = fail(QPM_ERR_ARG, "qpm_measure_latency: ctas outside [1, co-resident CTAs]");
    // [count, ..., err at word 32, ...] then the exchanged words [2][ctas]
    const size_t words_off = 256, bytes = words_off + 2 * sizeof(unsigned long long) * (size_t)ctas;
    if (st == QPM_OK) {
      ce = cudaMalloc(&buf, bytes);
      if (ce == cudaSuccess) ce = cudaMemsetAsync(buf, 0, bytes, s);
      if (ce != cudaSuccess) st = cuda_fail(ce, "cudaMalloc(barrier words)");
    }
    float t[2] = {0.f, 0.f};
    const int reps[2] = {100, 2100};  // the difference removes the launch cost
    for (int k = 0; k < 2 && st == QPM_OK; ++k) {
      for (int w = 0; w < 2 && st == QPM_OK; ++w) {  // the second launch is the timed one
        Barrier b{(unsigned *)buf, (int32_t *)buf + 32, 1000000000ull};  // 1 s per wait
        int r = reps[k], kd = kind;
        unsigned long long *words = (unsigned long long *)((char *)buf + words_off);
        void *args0[] = {&b, &r};
        void *args[] = {&b, &kd, &words, &r};
        st = timed([&] {
          cudaError_t e = cudaMemsetAsync(buf, 0, bytes, s);
          return e == cudaSuccess ? cudaLaunchCooperativeKernel(fn, ctas, LP_THREADS,
                                                                kind == 0 ? args0 : args, 0, s)
                                  : e;
        }, &t[k]);
      }
    }
    int32_t err = 0;
    if (st == QPM_OK) {
      ce = cudaMemcpy(&err, (int32_t *)buf + 32, sizeof(int32_t), cudaMemcpyDeviceToHost);
      if (ce != cudaSuccess) st = cuda_fail(ce, "cudaMemcpy");
      else if (err != 0) st = fail(QPM_ERR_TIMEOUT, "qpm_measure_latency: a barrier wait gave up");
    }
    if (st == QPM_OK) *ns_out = 1e6 * (double)(t[1] - t[0]) / (double)(reps[1] - reps[0]);
  } else {
    const size_t n = (size_t)4 << 20;  // 16 MB of uint32: in L2 after the first pass
    std::vector<uint32_t> h(n);
    // one cycle through all n words in a scrambled order (an affine map modulo n,
    // odd multiplier: a permutation of the ring; consecutive steps land far apart)
    for (size_t i = 0; i < n; ++i) h[i] = (uint32_t)((i * 2654435761ull + 40503ull) % n);
    std::vector<uint32_t> nx(n);
    {
      // follow the permutation's order to make next[] a single cycle
      std::vector<uint32_t> order(n);
      for (size_t i = 0; i < n; ++i) order[i] = h[i];
      for (size_t i = 0; i < n; ++i) nx[order[i]] = order[(i + 1) % n];
    }
    ce = cudaMalloc(&buf, n * sizeof(uint32_t) + 256);
    if (ce == cudaSuccess)
      ce = cudaMemcpy(buf, nx.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) st = cuda_fail(ce, "latency probe buffer");
    const uint32_t *next = (const uint32_t *)buf;
    uint32_t *sink = (uint32_t *)((char *)buf + n * sizeof(uint32_t));
    float t[2] = {0.f, 0.f};
    const int steps[2] = {1024, 9216};
    for (int k = 0; k < 2 && st == QPM_OK; ++k) {
      for (int w = 0; w < 2 && st == QPM_OK; ++w) {
        const int stp = w == 0 ? (int)n / 8 : steps[k];  // warm pass brings lines into L2
        st = timed([&] {
          k_probe_chase<<<1, 1, 0, s>>>(next, stp, sink);
          return cudaGetLastError();
        }, &t[k]);
      }
    }
    if (st == QPM_OK) *ns_out = 1e6 * (double)(t[1] - t[0]) / (double)(steps[1] - steps[0]);
  }
  if (buf) cudaFree(buf);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}
