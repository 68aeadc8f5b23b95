// qpm_table.cu -- per-problem phasor table and closed-form constants.
//
// The exact form of the Sec. 2.1 integral over unit domains needs, for every
// domain m, p1_m = e^{-i k1 m} and p2_m = e^{-i k2 m}, and three per-problem
// constants phi1 = phi(k1), phi2 = phi(k2), psi (see qpm_common.cuh).  The
// phase m*k is formed and reduced modulo 2 pi in FP64 (m*k reaches 1e5 rad for
// 1e5 domains, far beyond FP32's resolution), then the reduced argument is
// rounded to FP32 and passed to sincosf.  The diagonal sum sum_m p1_m p2_m that
// +-1 domains need is accumulated in FP64 with a fixed-order (deterministic)
// reduction.
#include <math.h>

#include <algorithm>

#include "qpm_common.cuh"
#include "qpm_internal.h"

namespace qpm {

static constexpr int TBL_THREADS = 256;

static __global__ void __launch_bounds__(TBL_THREADS)
    k_table(TableSpec s, float4 *__restrict__ table, double2 *__restrict__ part) {
  __shared__ double2 red[TBL_THREADS];
  double2 acc = make_double2(0.0, 0.0);
  const double ks = s.kappa1 + s.kappa2;
  for (int m = blockIdx.x * TBL_THREADS + threadIdx.x; m < s.Npad;
       m += gridDim.x * TBL_THREADS) {
    float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
    if (m < s.N) {
      const double dm = (double)m;
      float sn, cs;
      sincosf((float)reduce_2pi(dm * s.kappa1), &sn, &cs);
      e.x = cs;
      e.y = -sn;
      sincosf((float)reduce_2pi(dm * s.kappa2), &sn, &cs);
      e.z = cs;
      e.w = -sn;
      double sd, cd;
      sincos(reduce_2pi(dm * ks), &sd, &cd);
      acc.x += cd;
      acc.y -= sd;
    }
    if (table) {  // NULL: only the constants' diagonal sum is wanted
      const int t = m / s.c, r = m - t * s.c, k4 = r >> 2, q = r & 3;
      table[((size_t)k4 * 4 + q) * s.T + t] = e;
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = TBL_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[threadIdx.x].x += red[threadIdx.x + w].x;
      red[threadIdx.x].y += red[threadIdx.x + w].y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// phi(k) = int_0^1 e^{-iks} ds = e^{-ik/2} sin(k/2)/(k/2)
static __device__ double2 phi64(double k) {
  if (k == 0.0) return make_double2(1.0, 0.0);
  const double h = 0.5 * k;
  const double sc = sin(h) / h;
  return make_double2(cos(h) * sc, -sin(h) * sc);
}

static __device__ double2 psi64(double k1, double k2) {
  if (fabs(k1) > 1e-7) {
    // (phi(k2) - phi(k1 + k2)) / (i k1)
    const double2 a = phi64(k2), b = phi64(k1 + k2);
    const double xr = a.x - b.x, xi = a.y - b.y;
    return make_double2(xi / k1, -xr / k1);
  }
  // k1 -> 0: int_0^1 s e^{-i k2 s} ds
  if (fabs(k2) > 1e-4) {
    const double c = cos(k2), s = -sin(k2);  // e^{-i k2}
    // e^{-ik2} (1 + i k2) - 1, divided by k2^2
    const double re = c - s * k2 - 1.0, im = s + c * k2;
    return make_double2(re / (k2 * k2), im / (k2 * k2));
  }
  return make_double2(0.5 - k2 * k2 / 8.0, -k2 / 3.0);
}

static __global__ void k_table_finalize(int nparts, const double2 *__restrict__ part,
                                        double k1, double k2, float2 *konst, double2 *konst64) {
  if (threadIdx.x != 0) return;
  double sr = 0.0, si = 0.0;
  for (int b = 0; b < nparts; ++b) {
    sr += part[b].x;
    si += part[b].y;
  }
  const double2 p1 = phi64(k1), p2 = phi64(k2), ps = psi64(k1, k2);
  const double2 phi12 = make_double2(p1.x * p2.x - p1.y * p2.y, p1.x * p2.y + p1.y * p2.x);
  const double2 cdiag = make_double2(ps.x * sr - ps.y * si, ps.x * si + ps.y * sr);
  konst[0] = make_float2((float)phi12.x, (float)phi12.y);
  konst[1] = make_float2((float)cdiag.x, (float)cdiag.y);
  konst[2] = make_float2((float)ps.x, (float)ps.y);
  konst[3] = make_float2((float)p1.x, (float)p1.y);
  if (konst64) {
    konst64[0] = phi12;
    konst64[1] = cdiag;
    konst64[2] = ps;
    konst64[3] = p1;
  }
}

// Sign-block table of the row sweeps (qpm_eval, qpm_eval_packed, qpm_eval_multi).
// For +-1 domains a block of 4 consecutive domains 4b .. 4b+3 takes one of 16 sign
// patterns, and its monoid triple (A, B, C) = (sum_j a_j, sum_j b_j,
// sum_{j<k} a_k b_j), a = d p2, b = d p1, depends on the pattern only.  The 8
// patterns with d_{4b} = +1 are stored: pattern e has d_{4b+j} = -1 iff bit j of
// e << 1 is set (j = 1, 2, 3); the complement of a pattern has A and B negated and
// C unchanged (C is a sum of products of two signs).  Phases are reduced and their
// sines and cosines taken in FP64, the triples accumulated in FP64 in index order
// and rounded once to FP32.  Domains past N have p = 0.
// Layout: float2 blk[(8 b + e) * 3 + {0: A, 1: B, 2: C}], b < ceil(N / 4).
static __global__ void __launch_bounds__(TBL_THREADS)
    k_block_table(int N, int NB, double k1, double k2, float2 *__restrict__ blk) {
  for (int b = blockIdx.x * TBL_THREADS + threadIdx.x; b < NB; b += gridDim.x * TBL_THREADS) {
    double p1r[4], p1i[4], p2r[4], p2i[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = 4 * b + j;
      p1r[j] = p1i[j] = p2r[j] = p2i[j] = 0.0;
      if (m < N) {
        double sn, cs;
        sincos(reduce_2pi((double)m * k1), &sn, &cs);
        p1r[j] = cs;
        p1i[j] = -sn;
        sincos(reduce_2pi((double)m * k2), &sn, &cs);
        p2r[j] = cs;
        p2i[j] = -sn;
      }
    }
    for (int e = 0; e < 8; ++e) {
      double Ar = 0.0, Ai = 0.0, Br = 0.0, Bi = 0.0, Cr = 0.0, Ci = 0.0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const double d = (j > 0 && ((e >> (j - 1)) & 1)) ? -1.0 : 1.0;
        const double ar = d * p2r[j], ai = d * p2i[j];
        Cr += ar * Br - ai * Bi;  // a_j times the strictly earlier b
        Ci += ar * Bi + ai * Br;
        Ar += ar;
        Ai += ai;
        Br += d * p1r[j];
        Bi += d * p1i[j];
      }
      float2 *o = blk + ((size_t)8 * b + e) * 3;
      o[0] = make_float2((float)Ar, (float)Ai);
      o[1] = make_float2((float)Br, (float)Bi);
      o[2] = make_float2((float)Cr, (float)Ci);
    }
  }
}

qpm_status launch_block_table(int32_t N, double kappa1, double kappa2, float2 *blk,
                              cudaStream_t stream) {
  const int NB = (N + 3) / 4;
  const int nb = std::min(1024, (NB + TBL_THREADS - 1) / TBL_THREADS);
  k_block_table<<<nb, TBL_THREADS, 0, stream>>>(N, NB, kappa1, kappa2, blk);
  QPM_CUDA(cudaGetLastError());
  return QPM_OK;
}

int table_part_count(int32_t Npad) {
  const int n = (Npad + TBL_THREADS - 1) / TBL_THREADS;
  return n < 1024 ? (n < 1 ? 1 : n) : 1024;
}

qpm_status launch_table(const TableSpec &s, float4 *table, double2 *part, float2 *konst,
                        double2 *konst64, cudaStream_t stream) {
  const int nb = table_part_count(s.Npad);
  k_table<<<nb, TBL_THREADS, 0, stream>>>(s, table, part);
  QPM_CUDA(cudaGetLastError());
  k_table_finalize<<<1, 32, 0, stream>>>(nb, part, s.kappa1, s.kappa2, konst, konst64);
  QPM_CUDA(cudaGetLastError());
  return QPM_OK;
}

}  // namespace qpm
