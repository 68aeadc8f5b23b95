// qpm_tma.cuh -- the TMA tile copies, mbarriers and tensor maps shared by the sweeps
// that stream 32 x 32 float tiles (32 rows x 32 domains, 4 KB) through shared memory.
//
// A tile lands with the 128-byte swizzle (16-byte chunk c of row r at chunk c ^ (r & 7)
// of a 1024-byte aligned tile), which is the row-walk layout the sweeps index.  Loads
// complete on an mbarrier with an expected transaction count; every wait on one is
// bounded by %globaltimer.  Past the row end and the last row a load reads zeros.
// Stores leave as bulk groups; a store of a tile that reaches past the row end was
// measured writing into the row's padding (N = 4097 in rows of 4100 floats), so callers
// store only tiles that lie wholly inside the matrix.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "qpm_common.cuh"

namespace qpm {

static constexpr unsigned long long TMA_WAIT_NS = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase with the given parity to complete
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (!mbar_try(bar, parity))
    if (globaltimer_ns() - t0 > TMA_WAIT_NS) return false;
  return true;
}
// generic-proxy accesses to shared memory before this point are ordered before
// later async-proxy (TMA) accesses
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 32 x 32 float tile at (x = domain, y = row) into shared memory, completing on bar
__device__ __forceinline__ void tma_load_tile(void *dst, const CUtensorMap *map, int x, int y,
                                              unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
// the tile back to global memory (the part inside the tensor), as one bulk group
__device__ __forceinline__ void tma_store_tile(const CUtensorMap *map, int x, int y, const void *src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];"
               ::"l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_u32(src))
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// at most N of this thread's bulk store groups still reading shared memory
template <int N>
__device__ __forceinline__ void tma_store_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void tma_store_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------- host side
// cuTensorMapEncodeTiled from the driver, looked up once
static inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// rows x cols float matrix with leading dimension ld as 32 x 32 tiles, 128-byte
// swizzle, zero fill outside; false where a TMA copy cannot take it (address not
// 16-byte aligned, row pitch not a multiple of 16 bytes) or the driver refused
static inline bool make_tile_map(CUtensorMap *map, const float *base, int rows, int cols, int64_t ld) {
  if (((uintptr_t)base & 15) != 0 || (ld % 4) != 0 || ld >= ((int64_t)1 << 37)) return false;
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  const cuuint32_t box[2] = {32, 32};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace qpm
