// qpm_internal.h -- host-side declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "qpm.h"

namespace qpm {

void set_error(const std::string &msg);
qpm_status fail(qpm_status s, const std::string &msg);
qpm_status cuda_fail(cudaError_t e, const char *what);

#define QPM_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return ::qpm::cuda_fail(e_, #call); \
  } while (0)

// Phasor table layout: dimension m of a row split over T threads of c dims each
// (c a multiple of 4) lives at float4 index ((k4 * 4 + q) * T + t) with t = m / c,
// k4 = (m % c) / 4, q = m % 4.  T = 1, c = Npad is the natural order.
struct TableSpec {
  int32_t N, Npad, T, c;
  double kappa1, kappa2;
};

// float2 konst[4] = {phi1*phi2, cdiag, psi, phi1}; double2 konst64[4] = {phi1*phi2, cdiag, psi, phi1}
// part: scratch of table_part_count(Npad) double2; table may be NULL (constants only)
int table_part_count(int32_t Npad);
qpm_status launch_table(const TableSpec &s, float4 *table, double2 *part, float2 *konst,
                        double2 *konst64, cudaStream_t stream);

// sign-block table of the row sweeps: 8 patterns x (A, B, C) as float2 for every
// block of 4 domains, float2 blk[(8 b + e) * 3 + k], ceil(N / 4) blocks (24 float2
// = 192 bytes each); built in FP64, rounded to FP32
qpm_status launch_block_table(int32_t N, double kappa1, double kappa2, float2 *blk,
                              cudaStream_t stream);
constexpr int BLK_F2 = 24;  // float2 per block of 4 domains

// Access to the per-(device, N, kappa1, kappa2) cache of phasor tables, FP32
// constants and sign-block tables.  A lease holds the cache's lock from its
// construction to its destruction: the caller keeps it alive from the first lookup
// until the last launch that uses the returned pointers has been enqueued, so no
// other host thread can evict those tables in between.  The cache holds at most
// MAX_TABLES problems per device; a lease that will look up `problems` distinct
// problems makes room for all of them when it is created (freeing every table of
// the device once, after a device synchronisation), never between two lookups.
class TableLease {
 public:
  TableLease(const qpm_problem *problems, int count);
  ~TableLease();
  TableLease(const TableLease &) = delete;
  TableLease &operator=(const TableLease &) = delete;
  // status of the set-up (a failed eviction is reported by the first lookup)
  qpm_status status() const { return st_; }
  // natural-order phasor table and FP32 constants; built on `stream` on a miss
  qpm_status table(const qpm_problem *p, cudaStream_t stream, const float4 **table,
                   const float2 **konst);
  // the same entry's sign-block table (built on `stream` the first time) and constants
  qpm_status block_table(const qpm_problem *p, cudaStream_t stream, const float2 **blk,
                         const float2 **konst);

 private:
  qpm_status st_ = QPM_OK;
};

// split of qpm_eval-style work: S segments of L domains, rows in groups of 32
struct EvalShape {
  int NP, N, S, L;
  int groups;  // ceil(NP / 32)
  int NPpad;   // groups * 32
};
// split of the row sweep (qpm_rows.cuh): segments a multiple of 128 domains,
// about warps_per_sm warps of work per SM
// (lmax: longest segment, 0 for the phasor sweep's default)
EvalShape eval_rows_shape(int NP, int N, int warps_per_sm, int lmax = 0);

// current device's SM count (cached per device)
int sm_count();

}  // namespace qpm
