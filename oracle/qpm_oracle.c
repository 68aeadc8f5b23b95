/*
 * qpm_oracle.c -- plain, slow, obviously-correct CPU oracle for the cascaded-THG
 * quasi-phase-matching design method (HWSDA: DE + grey-wolf hybrid).
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  The product path (the CUDA
 * library) never calls it, shares no code with it, and fails loudly when its own
 * extension is missing.
 *
 * What it computes, and where the paper defines it:
 *   - d_eff (Sec. 2.1, the double integral that closes the derivation):
 *       d_eff = int_0^L d(z) e^{-i dk2 z} ( int_0^z d(x) e^{-i dk1 x} dx ) dz
 *     over N equal-width domains, d(z) = +-1 per domain (Sec. 2.1: +1 up, -1 down).
 *     Here it is integrated DIRECTLY: the integrand is split at the domain walls
 *     (the only places it is not smooth) and every piece is integrated with a
 *     Q-node Gauss-Legendre rule, the inner integral nested inside the outer one.
 *     Lengths are in units of the domain width w, so kappa = dk*w and the
 *     physical value is w^2 times the returned one.
 *   - the relaxed gradient d|d_eff|^2/d(theta_k), d_k = tanh(theta_k), by exact
 *     differentiation of the same quadrature sum, and by central differences.
 *   - the HWSDA loop (Sec. 2.2.1 DE, Sec. 2.2.2 GWO, Sec. 3.2 Steps 1-7) with
 *     FP32 genes and FP32 update arithmetic in a fixed operation order (no FMA:
 *     build with -ffp-contract=off), random numbers from Philox4x32-10
 *     (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 *     SC'11), written here from that published definition.
 *
 * Readings of the paper taken here (garbled or silent passages):
 *   - objective: maximise |d_eff|^2 (Sec. 2.1 asks for the largest d_eff); the loop can
 *     also maximise the SHG field |E|^2 or minimise the multi-wavelength objective of
 *     Sec. 5, sum_k |G0 - G_k| + beta (G_max - G_min), with G_k the cascaded or SHG
 *     field magnitude of each (kappa1, kappa2) pair (orc_cfg.obj); selection keeps the
 *     trial when it is at least as good in the objective's direction;
 *   - greedy selection keeps the trial when f(trial) >= f(target) (Sec. 2.2.1
 *     step 4 is printed garbled and for minimisation; mirrored for maximisation);
 *   - binomial crossover takes the mutant gene when U <= CR or j == jrand;
 *   - GWO: X2 uses d_beta and X3 uses d_gamma (the paper prints d_alpha in all
 *     three, a typo); combination is the plain mean (X1+X2+X3)/3 by default, or
 *     the paper's |X_k|-weighted form read per dimension;
 *   - only the omega wolves move in the GWO phase; the three leaders are the
 *     top three by fitness after the DE phase (Sec. 3.2 Step 3), ties broken
 *     towards the lower index;
 *   - real gene -> domain sign: d = (x < 0) ? -1 : +1;
 *   - genes are clamped to [-1, 1] after mutation and after the GWO move;
 *   - the update formulas are evaluated in FP32 in the order they are written,
 *     every operation rounded: v = fl(x_r1 + fl(F fl(x_r2 - x_r3))),
 *     A = fl(fl(2a r1) - a), C = fl(2 r2), D = |fl(fl(C X_p) - X)|,
 *     X_k = fl(X_p - fl(A D)), y = fl(fl(fl(X_1 + X_2) + X_3) / 3);
 *   - a decays linearly from 2 to 0: a_g = 2(G-g)/G, one rounded FP32 division.
 * Parity status: every function here is pinned by the CPU test-suite
 * (closed forms, invariants, an independent analytic closed form, brute force,
 * curand's host Philox); none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------- */
/* Gauss-Legendre rule on [-1, 1] (Newton iteration on P_Q, three-term recurrence) */
/* ------------------------------------------------------------------------- */
#define QMAX 32
static int g_Q = 0;
static double g_t[QMAX], g_w[QMAX];

static void legendre(int Q, double x, double *p, double *dp) {
  double p0 = 1.0, p1 = x;
  for (int k = 2; k <= Q; ++k) {
    double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = pk;
  }
  *p = p1;
  *dp = Q * (x * p1 - p0) / (x * x - 1.0);
}

ORC_API int orc_gauss_legendre(int Q, double *t, double *w) {
  if (Q < 2 || Q > QMAX) return -1;
  for (int k = 0; k < Q; ++k) {
    double x = cos(M_PI * (k + 0.75) / (Q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(Q, x, &p, &dp);
      double dx = p / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    double p, dp;
    legendre(Q, x, &p, &dp);
    t[k] = x;
    w[k] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  return 0;
}

static void ensure_rule(int Q) {
  if (g_Q != Q) {
    orc_gauss_legendre(Q, g_t, g_w);
    g_Q = Q;
  }
}

/* e^{-i k x} */
static inline void cis_neg(double k, double x, double *re, double *im) {
  double ph = k * x;
  *re = cos(ph);
  *im = -sin(ph);
}

/* Neumaier-compensated complex accumulator */
typedef struct { double sr, si, cr, ci; } acc_t;
static inline void acc_add(acc_t *a, double xr, double xi) {
  double t = a->sr + xr;
  if (fabs(a->sr) >= fabs(xr)) a->cr += (a->sr - t) + xr; else a->cr += (xr - t) + a->sr;
  a->sr = t;
  t = a->si + xi;
  if (fabs(a->si) >= fabs(xi)) a->ci += (a->si - t) + xi; else a->ci += (xi - t) + a->si;
  a->si = t;
}
static inline double acc_re(const acc_t *a) { return a->sr + a->cr; }
static inline double acc_im(const acc_t *a) { return a->si + a->ci; }

/* ------------------------------------------------------------------------- */
/* d_eff by nested quadrature (Sec. 2.1).                                     */
/*   domain j covers z in [j, j+1]; for z in that domain                      */
/*   I1(z) = sum_{m<j} d_m int_m^{m+1} e^{-ik1 x}dx + d_j int_j^z e^{-ik1 x}dx */
/*   d_eff = sum_j d_j int_j^{j+1} e^{-ik2 z} I1(z) dz                         */
/* ------------------------------------------------------------------------- */
static void deff_quad_one(int N, double k1, double k2, const double *d, int Q,
                          double *Dre, double *Dim) {
  ensure_rule(Q);
  acc_t D = {0, 0, 0, 0};
  acc_t C = {0, 0, 0, 0}; /* running inner integral over whole domains m < j */
  for (int j = 0; j < N; ++j) {
    double Cre = acc_re(&C), Cim = acc_im(&C);
    double outr = 0.0, outi = 0.0;
    for (int q = 0; q < Q; ++q) {
      double z = j + 0.5 * (1.0 + g_t[q]);
      double wq = 0.5 * g_w[q];
      double h = z - j; /* inner partial-domain integral over [j, z] */
      double inr = 0.0, ini = 0.0;
      for (int r = 0; r < Q; ++r) {
        double x = j + 0.5 * h * (1.0 + g_t[r]);
        double er, ei;
        cis_neg(k1, x, &er, &ei);
        inr += 0.5 * h * g_w[r] * er;
        ini += 0.5 * h * g_w[r] * ei;
      }
      double I1r = Cre + d[j] * inr, I1i = Cim + d[j] * ini;
      double er, ei;
      cis_neg(k2, z, &er, &ei);
      outr += wq * (er * I1r - ei * I1i);
      outi += wq * (er * I1i + ei * I1r);
    }
    acc_add(&D, d[j] * outr, d[j] * outi);
    /* whole-domain inner integral of domain j, added for the domains after it */
    double fr = 0.0, fi = 0.0;
    for (int r = 0; r < Q; ++r) {
      double x = j + 0.5 * (1.0 + g_t[r]);
      double er, ei;
      cis_neg(k1, x, &er, &ei);
      fr += 0.5 * g_w[r] * er;
      fi += 0.5 * g_w[r] * ei;
    }
    acc_add(&C, d[j] * fr, d[j] * fi);
  }
  *Dre = acc_re(&D);
  *Dim = acc_im(&D);
}

/* D[2*i], D[2*i+1] = d_eff of row i of d (rows of length N, leading dim ld) */
ORC_API void orc_deff_quad(int NP, int N, int64_t ld, double kappa1, double kappa2,
                           const double *d, int Q, double *D) {
  ensure_rule(Q);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < NP; ++i)
    deff_quad_one(N, kappa1, kappa2, d + (int64_t)i * ld, Q, &D[2 * i], &D[2 * i + 1]);
}

/* same, from FP32 genes mapped to domain signs d = (x < 0) ? -1 : +1 */
ORC_API void orc_deff_genes(int NP, int N, int64_t ld, double kappa1, double kappa2,
                            const float *X, int Q, double *D) {
  ensure_rule(Q);
#pragma omp parallel
  {
    double *d = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
#pragma omp for schedule(dynamic, 1)
    for (int i = 0; i < NP; ++i) {
      for (int j = 0; j < N; ++j) d[j] = (X[(int64_t)i * ld + j] < 0.0f) ? -1.0 : 1.0;
      deff_quad_one(N, kappa1, kappa2, d, Q, &D[2 * i], &D[2 * i + 1]);
    }
    free(d);
  }
}

/* ------------------------------------------------------------------------- */
/* d_eff by the closed form of the same integral for unit domains (Sec. 2.1): */
/*   int_j^{j+1} e^{-ik2 z} dz = e^{-ik2 j} phi2 and                         */
/*   int_m^{m+1} e^{-ik1 x} dx = e^{-ik1 m} phi1 turn the off-diagonal part   */
/*   into phi1 phi2 sum_j d_j e^{-ik2 j} sum_{m<j} d_m e^{-ik1 m}, and the     */
/*   diagonal part (x and z in the same domain j) into                        */
/*   psi sum_j d_j^2 e^{-i(k1+k2) j}, with phi(k) = int_0^1 e^{-iks} ds and      */
/*   psi = int_0^1 e^{-ik2 s} int_0^s e^{-ik1 t} dt ds, both taken here by the */
/*   same Gauss-Legendre rule (exact to rounding for these smooth integrands). */
/* FP64, rows in index order: a CPU throughput reference, pinned against the  */
/* quadrature.                                                                */
/* ------------------------------------------------------------------------- */
static void unit_integrals(double k1, double k2, int Q, double phi1[2], double phi2[2],
                           double psi[2]) {
  ensure_rule(Q);
  phi1[0] = phi1[1] = phi2[0] = phi2[1] = psi[0] = psi[1] = 0.0;
  for (int q = 0; q < Q; ++q) {
    const double s = 0.5 * (1.0 + g_t[q]), w = 0.5 * g_w[q];
    double er, ei;
    cis_neg(k1, s, &er, &ei);
    phi1[0] += w * er;
    phi1[1] += w * ei;
    cis_neg(k2, s, &er, &ei);
    phi2[0] += w * er;
    phi2[1] += w * ei;
    double inr = 0.0, ini = 0.0; /* int_0^s e^{-ik1 t} dt */
    for (int r = 0; r < Q; ++r) {
      const double t = 0.5 * s * (1.0 + g_t[r]);
      double fr, fi;
      cis_neg(k1, t, &fr, &fi);
      inr += 0.5 * s * g_w[r] * fr;
      ini += 0.5 * s * g_w[r] * fi;
    }
    psi[0] += w * (er * inr - ei * ini);
    psi[1] += w * (er * ini + ei * inr);
  }
}

ORC_API void orc_deff_closed(int NP, int N, int64_t ld, double kappa1, double kappa2,
                             const float *X, int Q, double *D) {
  double p1[2], p2[2], ps[2];
  unit_integrals(kappa1, kappa2, Q, p1, p2, ps);
  const double p12r = p1[0] * p2[0] - p1[1] * p2[1], p12i = p1[0] * p2[1] + p1[1] * p2[0];
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < NP; ++i) {
    acc_t S = {0, 0, 0, 0};   /* sum_{m<j} d_m e^{-ik1 m} */
    acc_t off = {0, 0, 0, 0}; /* sum_j d_j e^{-ik2 j} S_j */
    acc_t dg = {0, 0, 0, 0};  /* sum_j d_j^2 e^{-i(k1+k2) j} */
    for (int j = 0; j < N; ++j) {
      const double d = (X[(int64_t)i * ld + j] < 0.0f) ? -1.0 : 1.0;
      double ar, ai, br, bi, cr, ci;
      cis_neg(kappa2, (double)j, &ar, &ai);
      const double sr = acc_re(&S), si = acc_im(&S);
      acc_add(&off, d * (ar * sr - ai * si), d * (ar * si + ai * sr));
      cis_neg(kappa1, (double)j, &br, &bi);
      acc_add(&S, d * br, d * bi);
      cis_neg(kappa1 + kappa2, (double)j, &cr, &ci);
      acc_add(&dg, d * d * cr, d * d * ci);
    }
    const double orr = acc_re(&off), oi = acc_im(&off), gr = acc_re(&dg), gi = acc_im(&dg);
    D[2 * i] = (p12r * orr - p12i * oi) + (ps[0] * gr - ps[1] * gi);
    D[2 * i + 1] = (p12r * oi + p12i * orr) + (ps[0] * gi + ps[1] * gr);
  }
}

/* exhaustive search over all 2^N sign patterns (bit m set -> d_m = -1).
 * Writes f = |d_eff|^2 of every pattern to fit[2^N] (may be NULL) and returns
 * the best value; best_mask gets the lowest pattern index attaining it. */
ORC_API double orc_bruteforce(int N, double kappa1, double kappa2, int Q, double *fit,
                              int64_t *best_mask) {
  if (N < 1 || N > 24) return -1.0;
  ensure_rule(Q);
  int64_t M = (int64_t)1 << N;
  double best = -1.0;
  int64_t bm = 0;
#pragma omp parallel
  {
    double d[24];
    double lb = -1.0;
    int64_t lm = 0;
#pragma omp for schedule(static)
    for (int64_t s = 0; s < M; ++s) {
      for (int m = 0; m < N; ++m) d[m] = ((s >> m) & 1) ? -1.0 : 1.0;
      double re, im;
      deff_quad_one(N, kappa1, kappa2, d, Q, &re, &im);
      double f = re * re + im * im;
      if (fit) fit[s] = f;
      if (f > lb) { lb = f; lm = s; }
    }
#pragma omp critical
    {
      if (lb > best || (lb == best && lm < bm)) { best = lb; bm = lm; }
    }
  }
  if (best_mask) *best_mask = bm;
  return best;
}

/* ------------------------------------------------------------------------- */
/* SHG field integral (Sec. 2.1, first step of the derivation):              */
/*   E2(L) prop. to int_0^L d(z) e^{-i dk z} dz = sum_j d_j int_j^{j+1} e^{-ik z} dz */
/* each domain integrated with the Q-node Gauss-Legendre rule.                 */
/* ------------------------------------------------------------------------- */
static void shg_quad_one(int N, double k, const double *d, int Q, double *re, double *im) {
  acc_t S = {0, 0, 0, 0};
  for (int j = 0; j < N; ++j) {
    double fr = 0.0, fi = 0.0;
    for (int r = 0; r < Q; ++r) {
      double x = j + 0.5 * (1.0 + g_t[r]);
      double er, ei;
      cis_neg(k, x, &er, &ei);
      fr += 0.5 * g_w[r] * er;
      fi += 0.5 * g_w[r] * ei;
    }
    acc_add(&S, d[j] * fr, d[j] * fi);
  }
  *re = acc_re(&S);
  *im = acc_im(&S);
}

ORC_API void orc_shg_genes(int NP, int N, int64_t ld, double kappa, const float *X, int Q,
                           double *E) {
  ensure_rule(Q);
#pragma omp parallel
  {
    double *d = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
#pragma omp for schedule(dynamic, 1)
    for (int i = 0; i < NP; ++i) {
      for (int j = 0; j < N; ++j) d[j] = (X[(int64_t)i * ld + j] < 0.0f) ? -1.0 : 1.0;
      shg_quad_one(N, kappa, d, Q, &E[2 * i], &E[2 * i + 1]);
    }
    free(d);
  }
}

/* Multi-wavelength objective (Sec. 5, multi-wavelength designs):
 *   f = sum_i |G0 - G_i| + beta (G_max - G_min),  G_i = |d_eff| at (kappa1_i, kappa2_i)
 * (to be minimised; G0 a large reference value, beta a weight).  D[2*(i*K+k)]. */
ORC_API void orc_multi_objective(int NP, int N, int64_t ld, int K, const double *kappa1,
                                 const double *kappa2, const float *X, double G0, double beta,
                                 int Q, double *D, double *obj) {
  ensure_rule(Q);
#pragma omp parallel
  {
    double *d = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
#pragma omp for schedule(dynamic, 1)
    for (int i = 0; i < NP; ++i) {
      for (int j = 0; j < N; ++j) d[j] = (X[(int64_t)i * ld + j] < 0.0f) ? -1.0 : 1.0;
      double f = 0.0, gmax = -1.0, gmin = 1e300;
      for (int k = 0; k < K; ++k) {
        double re, im;
        deff_quad_one(N, kappa1[k], kappa2[k], d, Q, &re, &im);
        D[2 * ((int64_t)i * K + k)] = re;
        D[2 * ((int64_t)i * K + k) + 1] = im;
        double G = sqrt(re * re + im * im);
        f += fabs(G0 - G);
        if (G > gmax) gmax = G;
        if (G < gmin) gmin = G;
      }
      obj[i] = f + beta * (gmax - gmin);
    }
    free(d);
  }
}

/* ------------------------------------------------------------------------- */
/* Relaxed gradient: d_k = tanh(theta_k), f = |D|^2.                          */
/* D is a quadratic form in d; its derivative is taken term by term from the  */
/* quadrature sum of deff_quad_one:                                           */
/*   D = sum_j d_j O_j,  O_j = sum_q wq e^{-ik2 z_q} (C_j + d_j in_{j,q}),     */
/*   C_j = sum_{m<j} d_m F1_m                                                 */
/*   dD/dd_k = O_k + d_k S_k + F1_k sum_{j>k} d_j F2_j                        */
/* with S_k = sum_q wq e^{-ik2 z_q} in_{k,q} and F2_j = sum_q wq e^{-ik2 z_q}. */
/* ------------------------------------------------------------------------- */
ORC_API void orc_grad_relaxed(int N, double kappa1, double kappa2, const double *theta,
                              int Q, double *grad, double *Dout) {
  ensure_rule(Q);
  double *d = (double *)malloc(sizeof(double) * N);
  double *O = (double *)malloc(sizeof(double) * 2 * N);
  double *S = (double *)malloc(sizeof(double) * 2 * N);
  double *F1 = (double *)malloc(sizeof(double) * 2 * N);
  double *F2 = (double *)malloc(sizeof(double) * 2 * N);
  for (int j = 0; j < N; ++j) d[j] = tanh(theta[j]);
  acc_t C = {0, 0, 0, 0}, D = {0, 0, 0, 0};
  for (int j = 0; j < N; ++j) {
    double Cre = acc_re(&C), Cim = acc_im(&C);
    double outr = 0, outi = 0, sr = 0, si = 0, f2r = 0, f2i = 0;
    for (int q = 0; q < Q; ++q) {
      double z = j + 0.5 * (1.0 + g_t[q]);
      double wq = 0.5 * g_w[q];
      double h = z - j;
      double inr = 0.0, ini = 0.0;
      for (int r = 0; r < Q; ++r) {
        double x = j + 0.5 * h * (1.0 + g_t[r]);
        double er, ei;
        cis_neg(kappa1, x, &er, &ei);
        inr += 0.5 * h * g_w[r] * er;
        ini += 0.5 * h * g_w[r] * ei;
      }
      double er, ei;
      cis_neg(kappa2, z, &er, &ei);
      double I1r = Cre + d[j] * inr, I1i = Cim + d[j] * ini;
      outr += wq * (er * I1r - ei * I1i);
      outi += wq * (er * I1i + ei * I1r);
      sr += wq * (er * inr - ei * ini);
      si += wq * (er * ini + ei * inr);
      f2r += wq * er;
      f2i += wq * ei;
    }
    O[2 * j] = outr; O[2 * j + 1] = outi;
    S[2 * j] = sr; S[2 * j + 1] = si;
    F2[2 * j] = f2r; F2[2 * j + 1] = f2i;
    acc_add(&D, d[j] * outr, d[j] * outi);
    double fr = 0.0, fi = 0.0;
    for (int r = 0; r < Q; ++r) {
      double x = j + 0.5 * (1.0 + g_t[r]);
      double er, ei;
      cis_neg(kappa1, x, &er, &ei);
      fr += 0.5 * g_w[r] * er;
      fi += 0.5 * g_w[r] * ei;
    }
    F1[2 * j] = fr; F1[2 * j + 1] = fi;
    acc_add(&C, d[j] * fr, d[j] * fi);
  }
  double Dre = acc_re(&D), Dim = acc_im(&D);
  acc_t R = {0, 0, 0, 0}; /* suffix sum_{j>k} d_j F2_j */
  for (int k = N - 1; k >= 0; --k) {
    double Rr = acc_re(&R), Ri = acc_im(&R);
    double gr = O[2 * k] + d[k] * S[2 * k] + (F1[2 * k] * Rr - F1[2 * k + 1] * Ri);
    double gi = O[2 * k + 1] + d[k] * S[2 * k + 1] + (F1[2 * k] * Ri + F1[2 * k + 1] * Rr);
    /* df/dd_k = 2 Re(conj(D) dD/dd_k);  dd_k/dtheta_k = 1 - d_k^2 */
    grad[k] = 2.0 * (Dre * gr + Dim * gi) * (1.0 - d[k] * d[k]);
    acc_add(&R, d[k] * F2[2 * k], d[k] * F2[2 * k + 1]);
  }
  if (Dout) { Dout[0] = Dre; Dout[1] = Dim; }
  free(d); free(O); free(S); free(F1); free(F2);
}

/* f = |D|^2 of the relaxed sequence d = tanh(theta) */
ORC_API double orc_fit_relaxed(int N, double kappa1, double kappa2, const double *theta,
                               int Q, double *Dout) {
  ensure_rule(Q);
  double *d = (double *)malloc(sizeof(double) * N);
  for (int j = 0; j < N; ++j) d[j] = tanh(theta[j]);
  double re, im;
  deff_quad_one(N, kappa1, kappa2, d, Q, &re, &im);
  free(d);
  if (Dout) { Dout[0] = re; Dout[1] = im; }
  return re * re + im * im;
}

/* central finite differences of f(theta) at the coordinates idx[0..n) */
ORC_API void orc_fd_grad(int N, double kappa1, double kappa2, const double *theta,
                         const int32_t *idx, int n, double h, int Q, double *out) {
  ensure_rule(Q);
#pragma omp parallel
  {
    double *t = (double *)malloc(sizeof(double) * N);
    double *d = (double *)malloc(sizeof(double) * N);
#pragma omp for schedule(dynamic, 1)
    for (int c = 0; c < n; ++c) {
      memcpy(t, theta, sizeof(double) * N);
      int k = idx[c];
      double fp, fm, re, im;
      t[k] = theta[k] + h;
      for (int j = 0; j < N; ++j) d[j] = tanh(t[j]);
      deff_quad_one(N, kappa1, kappa2, d, Q, &re, &im);
      fp = re * re + im * im;
      t[k] = theta[k] - h;
      for (int j = 0; j < N; ++j) d[j] = tanh(t[j]);
      deff_quad_one(N, kappa1, kappa2, d, Q, &re, &im);
      fm = re * re + im * im;
      out[c] = (fp - fm) / (2.0 * h);
    }
    free(t);
    free(d);
  }
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 Philox round,  */
/* multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 /      */
/* 0xBB67AE85 (the golden ratio and sqrt(3)-1 in 0.32 fixed point).           */
/* ------------------------------------------------------------------------- */
ORC_API void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------- */
/* Random-number contract of this implementation (the paper fixes none):     */
/*   key = (seed low word, seed high word)                                    */
/*   counter = (j/4, i, g, (instance << 8) | tag); word j%4 serves gene j     */
/*   (g = 0xFFFFFFFF for the initial draw)                                    */
/*   tags: 0 init, 1 DE indices (counter word 0 = 0), 2 crossover,            */
/*         3..5 GWO for alpha, beta, gamma                                    */
/*   uniform U = (w >> 8) * 2^-24 in [0, 1) for init and crossover; the GWO   */
/*   pair (r1, r2) of a leader and gene = (w >> 16, w & 0xFFFF) * 2^-16       */
/*   index in [0, m): (w * m) >> 32  (Lemire multiply-shift)                  */
/* ------------------------------------------------------------------------- */
enum { TAG_INIT = 0, TAG_DEIDX = 1, TAG_CR = 2, TAG_GWO = 3 };
#define GEN_INIT 0xFFFFFFFFu /* the generation word of the initial draw */

static inline uint32_t rng_word(uint64_t seed, uint32_t inst, uint32_t tag, uint32_t g,
                                uint32_t i, uint32_t j) {
  uint32_t ctr[4] = {j >> 2, i, g, (inst << 8) | tag};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox(ctr, key, out);
  return out[j & 3];
}
static inline float u24(uint32_t w) { return (float)(w >> 8) * 0x1p-24f; }
/* the two 16-bit halves of one word as uniforms on [0, 1) (exact in FP32) */
static inline float u16hi(uint32_t w) { return (float)(w >> 16) * 0x1p-16f; }
static inline float u16lo(uint32_t w) { return (float)(w & 0xFFFFu) * 0x1p-16f; }
static inline uint32_t lemire(uint32_t w, uint32_t m) {
  return (uint32_t)(((uint64_t)w * m) >> 32);
}

ORC_API float orc_uniform(uint64_t seed, uint32_t inst, uint32_t tag, uint32_t g, uint32_t i,
                          uint32_t j) {
  return u24(rng_word(seed, inst, tag, g, i, j));
}

/* DE rand/1 donor indices r1, r2, r3 (distinct, != i; NP >= 4, Sec. 2.2.1 step 2) and
 * the forced crossover dimension jrand (rnbr(i) in Sec. 2.2.1 step 3). */
ORC_API void orc_de_indices(uint64_t seed, uint32_t inst, uint32_t g, int32_t i, int32_t NP,
                            int32_t N, int32_t out[4]) {
  uint32_t ctr[4] = {0, (uint32_t)i, g, (inst << 8) | TAG_DEIDX};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t w[4];
  orc_philox(ctr, key, w);
  int32_t ex[4];
  int ne = 0;
  ex[ne++] = i;
  int32_t r[3];
  for (int k = 0; k < 3; ++k) {
    int32_t t = (int32_t)lemire(w[k], (uint32_t)(NP - 1 - k));
    /* skip the excluded values in ascending order: a bijection onto the rest */
    int32_t s[3];
    for (int a = 0; a < ne; ++a) s[a] = ex[a];
    for (int a = 1; a < ne; ++a)
      for (int b = a; b > 0 && s[b - 1] > s[b]; --b) { int32_t tmp = s[b]; s[b] = s[b - 1]; s[b - 1] = tmp; }
    for (int a = 0; a < ne; ++a)
      if (t >= s[a]) ++t;
    r[k] = t;
    ex[ne++] = t;
  }
  out[0] = r[0]; out[1] = r[1]; out[2] = r[2];
  out[3] = (int32_t)lemire(w[3], (uint32_t)N);
}

typedef struct {
  int32_t NP, N;
  int64_t ld;
  int32_t G;
  float F, CR;
  uint64_t seed;
  uint32_t inst;
  int32_t combine; /* 0 = mean of X1..X3, 1 = |X_k|-weighted per dimension,
                      2 = the four-leader discrete GWO of Sec. 3.1.2 */
  int32_t f_schedule; /* 0 = constant F; 1 = decaying F of Sec. 3.1.1;
                         2 = the adaptive F of Sec. 3.1.1 (orc_adaptive_F) */
  /* the fitness the loop optimises (Sec. 2.1 and Sec. 5):
   *   0: |d_eff(kappa1, kappa2)|^2 of the cascaded integral, maximised (Sec. 2.1);
   *   1: |E_SHG(kappa1)|^2 of the single SHG integral, maximised;
   *   2: the multi-wavelength objective sum_k |G0 - G_k| + beta (G_max - G_min) with
   *      G_k = |d_eff(kap1[k], kap2[k])|, minimised (Sec. 5, cascaded THG designs);
   *   3: the same with G_k = |E_SHG(kap1[k])|, minimised (Sec. 5, SHG designs) */
  int32_t obj, K;
  double kap1[8], kap2[8];
  float G0, beta;
} orc_cfg;

/* the objective direction: the multi-wavelength objectives are minimised */
static inline int minimising(const orc_cfg *c) { return c->obj >= 2; }
/* a at least as good as b / strictly better, in the objective's direction */
static inline int better_eq(const orc_cfg *c, double a, double b) {
  return minimising(c) ? (a <= b) : (a >= b);
}
static inline int better(const orc_cfg *c, double a, double b) {
  return minimising(c) ? (a < b) : (a > b);
}

/* F of generation g.  Sec. 3.1.1 lets F follow (cos(pi g / 2G) + 1) / 2 times a
 * quadratic factor that falls from 1.0 to 0.8 over the run; the reading taken
 * here is F_g = F (cos(pi g / 2G) + 1) / 2 (1 - 0.2 (g/G)^2) in FP64, rounded to
 * FP32.  Its diversity-triggered adjustments have unstated thresholds and are not
 * modelled. */
ORC_API float orc_F_of(const orc_cfg *c, int32_t g) {
  if (!c->f_schedule) return c->F;
  const double x = (double)g / (double)c->G;
  const double cs = 0.5 * (cos(M_PI * (double)g / (2.0 * (double)c->G)) + 1.0);
  const double qd = 1.0 - 0.2 * x * x;
  /* adaptive form: the decay is the schedule of its intermediate state, scaled to the
   * interval [0.01, 0.1] that Sec. 3.1.1 keeps F in (its top) */
  const double top = c->f_schedule == 2 ? 0.1 : (double)c->F;
  return (float)(top * cs * qd);
}

/* ------------------------------------------------------------------------- */
/* Adaptive F (Sec. 3.1.1, "dual mechanism").  The paper keeps F in [0.01, 0.1]  */
/* and moves it by the population's state: when diversity is low (the standard  */
/* deviation below a threshold, or the convergence rate below 0.1) F is raised; */
/* when diversity is too high or the fitness range is small (the deviation above */
/* a threshold, or the range below 10^3) F is lowered; otherwise F follows the   */
/* cosine decay (cos(pi g / 2G) + 1) / 2 times a factor falling from 1.0 to 0.8. */
/* It states neither the thresholds, the step sizes, which deviation, nor what   */
/* the convergence rate is.  Readings taken (all after the DE phase of g, on the */
/* DE survivors, deciding the F of generation g + 1):                            */
/*   deviation: of the survivors' fitness, relative to its mean (coefficient of  */
/*     variation cv); thresholds cv < 0.05 (low) and cv > 0.5 (high);             */
/*   convergence rate: the fraction of the NP trials that strictly improved on    */
/*     their target;                                                              */
/*   range: max f - min f of the survivors, in the library's fitness units        */
/*     (|d_eff / w^2|^2), against 10^3;                                           */
/*   raise: F <- min(0.1, 1.25 F); lower: F <- max(0.01, 0.8 F); otherwise        */
/*     F <- 0.1 (cos(pi (g+1) / 2G) + 1) / 2 (1 - 0.2 ((g+1)/G)^2) (orc_F_of);    */
/*     the low test is taken first; F of generation 0 is the schedule's 0.1.      */
/* So that both implementations take every decision identically whatever their  */
/* summation order, the deviation is computed from exact integers: with E such   */
/* that 2^(E-1) <= max f < 2^E, every fitness is quantised to                    */
/* n = floor(f 2^(20 - E)) in [0, 2^20) by shifting its significand (exact), the */
/* sums S1 = sum n and S2 = sum n^2 are exact 64-bit integers (NP <= 2^23), and  */
/* cv^2 = (NP S2 - S1^2) / S1^2 is compared as NP S2 - S1^2 against t^2 S1^2 in  */
/* FP64, each operation rounded once (no contraction).  All f = 0 counts as low  */
/* diversity.                                                                     */
/* ------------------------------------------------------------------------- */
#define AF_FMIN 0.01f
#define AF_FMAX 0.1f
#define AF_UP 1.25f
#define AF_DOWN 0.8f

/* n = floor(f 2^(20 - E)) for f >= 0 given the biased exponent field emax of max f
 * (emax >= 1), from the bits: f = m 2^(e - 150) with m its 24-bit significand */
static inline uint32_t af_quantise(float f, uint32_t emax) {
  uint32_t u;
  memcpy(&u, &f, sizeof u);
  uint32_t e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  if (e == 0) e = 1; else m |= 0x800000u; /* subnormal: no hidden bit */
  const uint32_t sh = 4u + emax - e;     /* >= 4 since e <= emax */
  return sh >= 24u ? 0u : m >> sh;
}

/* F of generation g + 1 from the survivors' fitness f[NP] (the decision precision)
 * and the strict-improvement flags of the generation's trials; returns the branch
 * taken (0 schedule, 1 raised, 2 lowered), *F_next the new F.  stats (may be NULL)
 * receives {cv^2 (as the FP64 ratio, for reports), improved fraction, range}. */
ORC_API int orc_adaptive_F(const orc_cfg *c, int32_t g, const float *f, const uint8_t *improved,
                           float F_g, float *F_next, double *stats) {
  const int32_t NP = c->NP;
  float fmax = 0.0f, fmin = f[0];
  int64_t nimp = 0;
  for (int32_t i = 0; i < NP; ++i) {
    if (f[i] > fmax) fmax = f[i];
    if (f[i] < fmin) fmin = f[i];
    nimp += improved[i] ? 1 : 0;
  }
  uint32_t ub;
  memcpy(&ub, &fmax, sizeof ub);
  uint32_t emax = (ub >> 23) & 0xFFu;
  if (emax == 0) emax = 1;
  uint64_t S1 = 0, S2 = 0;
  for (int32_t i = 0; i < NP; ++i) {
    const uint64_t n = af_quantise(f[i], emax);
    S1 += n;
    S2 += n * n;
  }
  const double a = (double)NP * (double)S2;
  const double b = (double)S1 * (double)S1;
  const double num = a - b;
  const float range = fmax - fmin;
  const int low = (S1 == 0) || (num < 0.0025 * b) || (10 * nimp < (int64_t)NP);
  const int high = !low && ((num > 0.25 * b) || (range < 1000.0f));
  if (stats) {
    stats[0] = b > 0.0 ? num / b : 0.0;
    stats[1] = (double)nimp / (double)NP;
    stats[2] = (double)range;
  }
  if (low) {
    *F_next = fminf(AF_FMAX, F_g * AF_UP);
    return 1;
  }
  if (high) {
    *F_next = fmaxf(AF_FMIN, F_g * AF_DOWN);
    return 2;
  }
  *F_next = orc_F_of(c, g + 1);
  return 0;
}

static inline float clamp1(float v) { return fminf(fmaxf(v, -1.0f), 1.0f); }

/* Step 1 / Sec. 2.2.1 step 1: x_ij = U(-1, 1), computed as 2U - 1 (exact in FP32) */
ORC_API void orc_init_population(const orc_cfg *c, float *X) {
  for (int32_t i = 0; i < c->NP; ++i)
    for (int32_t j = 0; j < c->N; ++j) {
      float U = u24(rng_word(c->seed, c->inst, TAG_INIT, GEN_INIT, (uint32_t)i, (uint32_t)j));
      X[(int64_t)i * c->ld + j] = 2.0f * U - 1.0f;
    }
}

/* Sec. 2.2.1 steps 2-3 for target i: mutant v = x_r1 + F (x_r2 - x_r3), clamped,
 * then binomial crossover with the target -> trial u */
static void de_trial_one(const orc_cfg *c, uint32_t g, float F, int32_t i, const float *X,
                         float *u) {
  int32_t r[4];
  orc_de_indices(c->seed, c->inst, g, i, c->NP, c->N, r);
  const float *x = X + (int64_t)i * c->ld;
  const float *x1 = X + (int64_t)r[0] * c->ld;
  const float *x2 = X + (int64_t)r[1] * c->ld;
  const float *x3 = X + (int64_t)r[2] * c->ld;
  for (int32_t j = 0; j < c->N; ++j) {
    float diff = x2[j] - x3[j];
    float step = F * diff;
    float v = clamp1(x1[j] + step);
    float randb = u24(rng_word(c->seed, c->inst, TAG_CR, g, (uint32_t)i, (uint32_t)j));
    u[j] = (randb <= c->CR || j == r[3]) ? v : x[j];
  }
}

/* trials of every target with the scale factor F of generation g */
static void de_trials_F(const orc_cfg *c, uint32_t g, float F, const float *X, float *U) {
#pragma omp parallel for schedule(static)
  for (int32_t i = 0; i < c->NP; ++i) de_trial_one(c, g, F, i, X, U + (int64_t)i * c->ld);
}

ORC_API void orc_de_trials(const orc_cfg *c, uint32_t g, const float *X, float *U) {
  de_trials_F(c, g, orc_F_of(c, (int32_t)g), X, U);
}

/* Sec. 3.2 Step 3: the three best wolves (descending f, ties to the lower index) */
ORC_API void orc_top3(int32_t NP, const float *f, int32_t lead[3]) {
  for (int k = 0; k < 3; ++k) lead[k] = -1;
  for (int32_t i = 0; i < NP; ++i) {
    for (int k = 0; k < 3; ++k) {
      if (lead[k] < 0 || f[i] > f[lead[k]]) {
        for (int m = 2; m > k; --m) lead[m] = lead[m - 1];
        lead[k] = i;
        break;
      }
    }
  }
}

/* a_g = 2 (G - g) / G  (linear decay from 2 towards 0, Sec. 2.2.2) */
ORC_API float orc_a_of(int32_t g, int32_t G) {
  return (float)(2 * (G - g)) / (float)G;
}

/* Sec. 2.2.2: encircling of the prey by the three leaders, then the combination */
static void gwo_cand_one(const orc_cfg *c, uint32_t g, int32_t i, const float *X,
                         const int32_t lead[3], float *y) {
  float a = orc_a_of((int32_t)g, c->G);
  float two_a = 2.0f * a;
  const float *x = X + (int64_t)i * c->ld;
  for (int32_t j = 0; j < c->N; ++j) {
    float Xk[3];
    for (int k = 0; k < 3; ++k) {
      const float *Xp = X + (int64_t)lead[k] * c->ld; /* alpha, beta, gamma */
      /* r1 and r2 of leader k: the high and low 16 bits of one word (tag GWO + k) */
      const uint32_t w = rng_word(c->seed, c->inst, TAG_GWO + k, g, (uint32_t)i, (uint32_t)j);
      float r1 = u16hi(w);
      float r2 = u16lo(w);
      float A = two_a * r1 - a;             /* A = 2 a r1 - a */
      float C = 2.0f * r2;                  /* C = 2 r2 */
      float dist = fabsf(C * Xp[j] - x[j]); /* d = |C Xp - X| */
      Xk[k] = Xp[j] - A * dist;             /* X_k = Xp - A d */
    }
    float yj;
    if (c->combine == 0) {
      yj = ((Xk[0] + Xk[1]) + Xk[2]) / 3.0f;
    } else {
      float m0 = fabsf(Xk[0]), m1 = fabsf(Xk[1]), m2 = fabsf(Xk[2]);
      float s = (m0 + m1) + m2;
      float num = ((m0 * Xk[0]) + (m1 * Xk[1])) + (m2 * Xk[2]);
      yj = (s == 0.0f) ? 0.0f : num / (3.0f * s);
    }
    y[j] = clamp1(yj);
  }
}

/* ------------------------------------------------------------------------- */
/* Improved discrete GWO with four leaders (Sec. 3.1.2), combine = 2.  The paper */
/* describes it only qualitatively: continuous positions map to +-1 states; the  */
/* state of a wolf follows transition probabilities taken from the four leaders' */
/* state distribution, with random disturbance whose strength a dispersion      */
/* parameter sets; early iterations explore with much disturbance, late ones     */
/* follow the dominant state with only a small flip probability; a social-      */
/* learning rate that falls with the iterations lets a wolf copy a random       */
/* leader's state.  Reading taken (tau = g / G), per omega wolf and gene j, with */
/* n = the number of the four leaders whose gene j is +1:                        */
/*   dispersion delta = 0.5 (1 - tau), social rate sigma = 0.3 (1 - tau),        */
/*   disturbance mu = 0.1 (1 - tau) + 0.01 tau;                                  */
/*   q_n = (1 - tau) n / 4 + tau m_n, m_n the majority vote (1 for n > 2, 0 for   */
/*   n < 2, 1/2 for n = 2); P_n = (1 - delta) q_n + delta / 2 (the chance of +1); */
/*   with probability sigma the wolf takes the state of leader kl (uniform among  */
/*   the four), else +1 with probability P_n; then the state flips with          */
/*   probability mu.  Every probability p becomes the 16-bit threshold           */
/*   floor(65536 p) (FP64, once per generation), tested as u < threshold on      */
/*   16-bit uniforms from two words per gene: tag 3 gives the social (high) and  */
/*   transition (low) halves, tag 4 the flip half (high) and kl (low two bits).   */
/* The new genes are +-1.0.                                                      */
/* ------------------------------------------------------------------------- */
typedef struct { uint32_t social, flip, plus[5]; } disc_thr;

ORC_API void orc_discrete_thresholds(int32_t g, int32_t G, uint32_t out[7]) {
  const double tau = (double)g / (double)G;
  const double delta = 0.5 * (1.0 - tau), sigma = 0.3 * (1.0 - tau);
  const double mu = 0.1 * (1.0 - tau) + 0.01 * tau;
  out[0] = (uint32_t)floor(65536.0 * sigma);
  out[1] = (uint32_t)floor(65536.0 * mu);
  for (int n = 0; n <= 4; ++n) {
    const double m = n > 2 ? 1.0 : (n < 2 ? 0.0 : 0.5);
    const double qn = (1.0 - tau) * ((double)n / 4.0) + tau * m;
    const double P = (1.0 - delta) * qn + 0.5 * delta;
    out[2 + n] = (uint32_t)floor(65536.0 * P);
  }
}

static void gwo_discrete_one(const orc_cfg *c, uint32_t g, int32_t i, const float *X,
                             const int32_t lead[4], float *y) {
  uint32_t th[7];
  orc_discrete_thresholds((int32_t)g, c->G, th);
  for (int32_t j = 0; j < c->N; ++j) {
    float s[4];
    int n = 0;
    for (int k = 0; k < 4; ++k) {
      s[k] = (X[(int64_t)lead[k] * c->ld + j] < 0.0f) ? -1.0f : 1.0f;
      n += s[k] > 0.0f;
    }
    const uint32_t w1 = rng_word(c->seed, c->inst, TAG_GWO, g, (uint32_t)i, (uint32_t)j);
    const uint32_t w2 = rng_word(c->seed, c->inst, TAG_GWO + 1, g, (uint32_t)i, (uint32_t)j);
    float v;
    if ((w1 >> 16) < th[0]) v = s[w2 & 3u];           /* social learning */
    else v = ((w1 & 0xFFFFu) < th[2 + n]) ? 1.0f : -1.0f; /* transition */
    if ((w2 >> 16) < th[1]) v = -v;                   /* disturbance */
    y[j] = v;
  }
}

/* candidate positions for every omega wolf (rows of leaders are left untouched in Y) */
/* number of leaders: four for the discrete GWO, three otherwise */
static inline int n_leaders(const orc_cfg *c) { return c->combine == 2 ? 4 : 3; }
static inline int is_leader(const int32_t *lead, int nl, int32_t i) {
  for (int k = 0; k < nl; ++k)
    if (lead[k] == i) return 1;
  return 0;
}

/* lead: three leaders (four for the discrete GWO, combine = 2) */
ORC_API void orc_gwo_candidates(const orc_cfg *c, uint32_t g, const float *X,
                                const int32_t *lead, float *Y) {
  const int nl = n_leaders(c);
#pragma omp parallel for schedule(static)
  for (int32_t i = 0; i < c->NP; ++i) {
    if (is_leader(lead, nl, i)) continue;
    if (c->combine == 2) gwo_discrete_one(c, g, i, X, lead, Y + (int64_t)i * c->ld);
    else gwo_cand_one(c, g, i, X, lead, Y + (int64_t)i * c->ld);
  }
}

/* the objective of one +-1 row d (cfg->obj), by the quadratures of Sec. 2.1 */
static double row_objective(const orc_cfg *c, double kappa1, double kappa2, int Q,
                            const double *d) {
  double re, im;
  if (c->obj == 0 || c->obj == 1) {
    if (c->obj == 0) deff_quad_one(c->N, kappa1, kappa2, d, Q, &re, &im);
    else shg_quad_one(c->N, kappa1, d, Q, &re, &im);
    return re * re + im * im;
  }
  double f = 0.0, gmax = -1.0, gmin = 1e300;
  for (int k = 0; k < c->K; ++k) {
    if (c->obj == 2) deff_quad_one(c->N, c->kap1[k], c->kap2[k], d, Q, &re, &im);
    else shg_quad_one(c->N, c->kap1[k], d, Q, &re, &im);
    const double G = sqrt(re * re + im * im);
    f += fabs((double)c->G0 - G);
    if (G > gmax) gmax = G;
    if (G < gmin) gmin = G;
  }
  return f + (double)c->beta * (gmax - gmin);
}

static void eval_rows(const orc_cfg *c, double kappa1, double kappa2, int Q, const float *X,
                      const uint8_t *mask, double *f64) {
#pragma omp parallel
  {
    double *d = (double *)malloc(sizeof(double) * (size_t)c->N);
#pragma omp for schedule(dynamic, 1)
    for (int32_t i = 0; i < c->NP; ++i) {
      if (mask && !mask[i]) { f64[i] = NAN; continue; }
      for (int32_t j = 0; j < c->N; ++j) d[j] = (X[(int64_t)i * c->ld + j] < 0.0f) ? -1.0 : 1.0;
      f64[i] = row_objective(c, kappa1, kappa2, Q, d);
    }
    free(d);
  }
}

/* the objective of every row of X (the loop's fitness, in FP64) */
ORC_API void orc_objective_rows(const orc_cfg *c, double kappa1, double kappa2, int Q,
                                const float *X, double *f64) {
  ensure_rule(Q);
  eval_rows(c, kappa1, kappa2, Q, X, NULL, f64);
}

/* the nl best of f in the objective's direction, ties to the lower index */
static void topn_dir(const orc_cfg *c, int nl, const float *f, int32_t *lead) {
  for (int k = 0; k < nl; ++k) lead[k] = -1;
  for (int32_t i = 0; i < c->NP; ++i)
    for (int k = 0; k < nl; ++k)
      if (lead[k] < 0 || better(c, f[i], f[lead[k]])) {
        for (int m = nl - 1; m > k; --m) lead[m] = lead[m - 1];
        lead[k] = i;
        break;
      }
}

/* One generation of the HWSDA loop (Sec. 3.2 Steps 2-6) from population X.
 *   X[NP*ld]      in/out FP32 genes
 *   fdec[NP]      in/out FP32 fitness used for the decisions (lockstep mode)
 *   f64[NP]       in/out FP64 fitness of the current individuals (may be stale
 *                 for individuals whose new fitness was not evaluated)
 *   lock_trial, lock_cand: if non-NULL (lockstep), FP32 fitness of this
 *                 generation's trials / GWO candidates that decide selection
 *                 and leaders; otherwise the oracle's own FP64 values decide
 *   eval_mask[NP]: if non-NULL, only rows with a non-zero entry get their FP64
 *                 fitness computed (lockstep only; decisions do not need them)
 *   tr_trial, tr_cand: if non-NULL, receive the FP64 fitness of trials and
 *                 candidates (NaN where not evaluated)
 *   lead_out:     if non-NULL, receives the leaders of this generation (three, or
 *                 four for the discrete GWO)
 *   F_io:         adaptive F (f_schedule = 2) only: in, the F of generation g; out,
 *                 the F of generation g + 1 (orc_adaptive_F on the DE survivors);
 *                 NULL otherwise (F then follows orc_F_of)
 *   branch_out:   if non-NULL (adaptive F), receives orc_adaptive_F's branch */
ORC_API int orc_hwsda_generation(const orc_cfg *c, double kappa1, double kappa2, int Q, int32_t g,
                                 float *X, float *fdec, double *f64, const float *lock_trial,
                                 const float *lock_cand, const uint8_t *eval_mask,
                                 double *tr_trial, double *tr_cand, int32_t *lead_out,
                                 float *F_io, int32_t *branch_out) {
  ensure_rule(Q);
  const int lock = (lock_trial != NULL);
  if (!lock && eval_mask) return -1;
  if ((c->f_schedule == 2) != (F_io != NULL)) return -2;
  int32_t NP = c->NP;
  int64_t sz = (int64_t)NP * c->ld;
  float *U = (float *)calloc((size_t)sz, sizeof(float));
  double *ft = (double *)malloc(sizeof(double) * NP);
  uint8_t *mask = (uint8_t *)malloc((size_t)NP);
  /* Step 2: mutation, crossover and selection over all NP individuals */
  de_trials_F(c, (uint32_t)g, F_io ? *F_io : orc_F_of(c, g), X, U);
  eval_rows(c, kappa1, kappa2, Q, U, eval_mask, ft);
  if (tr_trial) memcpy(tr_trial, ft, sizeof(double) * NP);
  for (int32_t i = 0; i < NP; ++i) {
    /* strict improvement of the trial over its target, in the decision precision */
    mask[i] = lock ? better(c, lock_trial[i], fdec[i]) : better(c, (float)ft[i], fdec[i]);
    int accept = lock ? better_eq(c, lock_trial[i], fdec[i]) : better_eq(c, ft[i], f64[i]);
    if (accept) {
      memcpy(X + (int64_t)i * c->ld, U + (int64_t)i * c->ld, sizeof(float) * c->N);
      f64[i] = ft[i];
      fdec[i] = lock ? lock_trial[i] : (float)ft[i];
    }
  }
  /* Sec. 3.2 Step 6 for the adaptive F, from the DE survivors (Sec. 3.1.1) */
  if (F_io) {
    float Fn;
    const int br = orc_adaptive_F(c, g, fdec, mask, *F_io, &Fn, NULL);
    *F_io = Fn;
    if (branch_out) *branch_out = br;
  }
  /* Step 3: the three leaders (four for the discrete GWO) */
  const int nl = n_leaders(c);
  int32_t lead[4] = {-1, -1, -1, -1};
  if (lock) {
    topn_dir(c, nl, fdec, lead);
  } else {
    for (int32_t i = 0; i < NP; ++i)
      for (int k = 0; k < nl; ++k)
        if (lead[k] < 0 || better(c, f64[i], f64[lead[k]])) {
          for (int m = nl - 1; m > k; --m) lead[m] = lead[m - 1];
          lead[k] = i;
          break;
        }
  }
  if (lead_out)
    for (int k = 0; k < nl; ++k) lead_out[k] = lead[k];
  /* Step 4: move the omega wolves; Step 5: greedy selection again */
  orc_gwo_candidates(c, (uint32_t)g, X, lead, U);
  for (int32_t i = 0; i < NP; ++i)
    mask[i] = !is_leader(lead, nl, i) && (!eval_mask || eval_mask[i]);
  eval_rows(c, kappa1, kappa2, Q, U, mask, ft);
  if (tr_cand) memcpy(tr_cand, ft, sizeof(double) * NP);
  for (int32_t i = 0; i < NP; ++i) {
    if (is_leader(lead, nl, i)) continue;
    int accept = lock ? better_eq(c, lock_cand[i], fdec[i]) : better_eq(c, ft[i], f64[i]);
    if (accept) {
      memcpy(X + (int64_t)i * c->ld, U + (int64_t)i * c->ld, sizeof(float) * c->N);
      f64[i] = ft[i];
      fdec[i] = lock ? lock_cand[i] : (float)ft[i];
    }
  }
  /* Step 6: F and CR stay constant; a follows from g in the next generation */
  free(U); free(ft); free(mask);
  return 0;
}

/* The HWSDA loop of Sec. 3.2 (Steps 1-7), one instance.
 *   X[NP*ld]   out: final population (FP32 genes)
 *   fcur[NP]   out: FP64 fitness of the final population
 *   lockstep:  if non-NULL, selection and leader decisions are taken from these
 *              FP32 fitness values instead of the oracle's own FP64 ones, so that
 *              an FP32 implementation can be followed bit for bit:
 *              lockstep[0 .. NP)                       fitness after init
 *              lockstep[NP*(1+2g) .. NP*(2+2g))        trial fitness of generation g
 *              lockstep[NP*(2+2g) .. NP*(3+2g))        GWO candidate fitness of gen g
 *   trace64:   if non-NULL, same layout, filled with the oracle's FP64 fitness
 *   Fhist:     if non-NULL, [G + 1]: the F of every generation (the last entry: the
 *              F the run would use next)
 *   Returns 0. */
ORC_API int orc_hwsda_run(const orc_cfg *c, double kappa1, double kappa2, int Q, float *X,
                          double *fcur, const float *lockstep, double *trace64, float *Fhist) {
  ensure_rule(Q);
  int32_t NP = c->NP;
  float *fdec = (float *)malloc(sizeof(float) * NP);
  orc_init_population(c, X);
  eval_rows(c, kappa1, kappa2, Q, X, NULL, fcur);
  if (trace64) memcpy(trace64, fcur, sizeof(double) * NP);
  for (int32_t i = 0; i < NP; ++i) fdec[i] = lockstep ? lockstep[i] : (float)fcur[i];
  float F = orc_F_of(c, 0); /* the adaptive F starts from the schedule */
  for (int32_t g = 0; g < c->G; ++g) {
    const float *lt = lockstep ? lockstep + (int64_t)NP * (1 + 2 * g) : NULL;
    const float *lc = lockstep ? lockstep + (int64_t)NP * (2 + 2 * g) : NULL;
    double *tt = trace64 ? trace64 + (int64_t)NP * (1 + 2 * g) : NULL;
    double *tc = trace64 ? trace64 + (int64_t)NP * (2 + 2 * g) : NULL;
    if (Fhist) Fhist[g] = c->f_schedule == 2 ? F : orc_F_of(c, g);
    orc_hwsda_generation(c, kappa1, kappa2, Q, g, X, fdec, fcur, lt, lc, NULL, tt, tc, NULL,
                         c->f_schedule == 2 ? &F : NULL, NULL);
  }
  if (Fhist) Fhist[c->G] = c->f_schedule == 2 ? F : orc_F_of(c, c->G);
  free(fdec);
  return 0;
}

ORC_API int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
