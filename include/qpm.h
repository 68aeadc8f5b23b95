/*
 * qpm.h -- C ABI of the GB300 (sm_103a) library for quasi-phase-matching crystal
 * design by the hybrid wolf-swarm differential algorithm (HWSDA: differential
 * evolution + grey-wolf optimiser) of arXiv 2511.01255.
 *
 * Conventions shared by every entry point
 *   - Lengths are in units of the domain width w.  A problem is N domains of width
 *     w with phase mismatches dk1 (SHG) and dk2 (SFG); the library takes
 *     kappa1 = dk1*w and kappa2 = dk2*w in radians.  The returned d_eff is in
 *     units of w^2 (multiply by w^2 for physical units).
 *   - d_eff is the double integral of Sec. 2.1 (the expression that ends the
 *     derivation of the cascaded third-harmonic field):
 *         d_eff = int_0^L d(z) e^{-i dk2 z} ( int_0^z d(x) e^{-i dk1 x} dx ) dz
 *     evaluated exactly for piecewise-constant d(z).  The fitness is
 *     f = |d_eff|^2, which the optimiser maximises (Sec. 2.1 asks for the
 *     largest d_eff).
 *   - Domain signs: a real gene x maps to d = (x < 0) ? -1 : +1 (Sec. 3.1.2's
 *     continuous-to-(+1/-1) mapping); in packed form bit (j % 32) of word j / 32
 *     set means d_j = -1.
 *   - Complex values are two consecutive floats (re, im), i.e. float2 layout.
 *   - Every pointer named "device" is CUDA device memory owned by the caller;
 *     the library never frees it and never keeps it past the call.  Host
 *     pointers are named "host".
 *   - Every call that takes a stream enqueues its work on that stream
 *     (NULL = the legacy default stream) and returns without synchronising,
 *     unless stated otherwise.
 *   - Every call returns a qpm_status.  On failure nothing is enqueued (argument
 *     errors) or the CUDA error is reported (QPM_ERR_CUDA); qpm_last_error()
 *     gives a message for the calling thread.  No exception crosses the ABI.
 *     There is no CPU fallback: without a usable sm_103a device every call that
 *     computes returns QPM_ERR_CUDA.
 */
#ifndef QPM_H_
#define QPM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *qpm_stream_t; /* same type as cudaStream_t */

typedef enum {
  QPM_OK = 0,
  QPM_ERR_ARG = 1,         /* invalid argument (size, alignment, NULL pointer) */
  QPM_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  QPM_ERR_TIMEOUT = 3,     /* a bounded device-side wait gave up (persistent kernel) */
  QPM_ERR_UNSUPPORTED = 4, /* request outside what this build supports */
  QPM_ERR_STATE = 5        /* call out of order (e.g. step before init) */
} qpm_status;

/* One design problem: N domains, kappa = dk * w in radians. */
typedef struct {
  int32_t N;
  double kappa1; /* SHG mismatch dk1 * w */
  double kappa2; /* SFG mismatch dk2 * w */
} qpm_problem;

/* HWSDA parameters (Sec. 2.2.1, 2.2.2, 3.2). */
typedef struct {
  int32_t NP;          /* population size, >= 4 (rand/1 needs 3 donors != target) */
  int32_t G;           /* generations; a decays linearly 2 -> 0 over them */
  float F;             /* DE scale factor, [0, 2] */
  float CR;            /* crossover rate, [0, 1] */
  uint64_t seed;       /* Philox4x32-10 key */
  int32_t gwo_combine; /* the GWO update of the omega wolves: 0: (X1+X2+X3)/3; 1: |X_k|-
                          weighted, per dimension; 2: the four-leader discrete GWO of
                          Sec. 3.1.2 (launches and graph forms, single objectives): with
                          tau = g / G and n of the four leaders' genes at +1, take a random
                          leader's state with probability 0.3 (1 - tau), else +1 with
                          probability (1 - delta) q_n + delta / 2, delta = 0.5 (1 - tau),
                          q_n = (1 - tau) n / 4 + tau [majority of the four, 1/2 on a tie];
                          then flip with probability 0.1 (1 - tau) + 0.01 tau; genes +-1 */
  int32_t compensated; /* 0: plain FP32 scan; 1: Kahan-compensated FP32 scan */
  int32_t team;        /* threads per individual: 0 = automatic (the smallest power of two in
                          [32, 256] with at most 4 domains per thread; 512 for a single
                          long-row instance when one 512-thread CTA per SM leaves fewer CTA
                          slots idle), else 32, 64, 128, 256 or 512 */
  int32_t f_schedule;  /* 0: F constant; 1: decaying F of Sec. 3.1.1,
                          F_g = F (cos(pi g / 2G) + 1) / 2 (1 - 0.2 (g / G)^2),
                          evaluated in FP64 and rounded to FP32;
                          2: the adaptive F of Sec. 3.1.1 (the field F is unused):
                          F in [0.01, 0.1], F_0 = 0.1; after the DE phase of generation
                          g, over the DE survivors, with cv their fitness' standard
                          deviation over its mean and rho the fraction of trials that
                          strictly improved on their target: cv < 0.05 or rho < 0.1
                          -> F = min(0.1, 1.25 F); else cv > 0.5 or max f - min f < 1e3
                          -> F = max(0.01, 0.8 F); else F = 0.1 (cos(pi (g+1) / 2G)
                          + 1) / 2 (1 - 0.2 ((g+1) / G)^2).  cv is decided from exact
                          integer statistics (fitness quantised to 20 bits against the
                          population maximum), so the decision is independent of any
                          summation order.  NP <= 2^23.  A run resumed with
                          qpm_set_population continues from the F history the state
                          holds (qpm_get_F; another state takes it with qpm_set_F) */
} qpm_params;

/* The fitness an optimiser state works on (qpm_set_objective; no call: QPM_OBJ_THG).
 *   QPM_OBJ_THG        |d_eff|^2 of the cascaded integral of Sec. 2.1 at the problem's
 *                      (kappa1, kappa2), maximised
 *   QPM_OBJ_SHG        |E|^2 of the SHG field integral of Sec. 2.1's first step,
 *                      E = int_0^L d(z) e^{-i dk z} dz with dk w = the problem's kappa1,
 *                      maximised
 *   QPM_OBJ_MULTI_THG  the multi-wavelength objective of Sec. 5,
 *                      f = sum_k |G0 - G_k| + beta (G_max - G_min), G_k = |d_eff| of the
 *                      cascaded integral at (kappa1[k], kappa2[k]), k < K <= 4, minimised
 *   QPM_OBJ_MULTI_SHG  the same with G_k = |E| of the SHG integral at kappa1[k],
 *                      k < K <= 8, minimised
 * The optimiser's d_eff outputs (qpm_get_population, qpm_get_best) hold the field of the
 * objective (for the multi-wavelength kinds: of the first problem), its fitness
 * outputs the objective.  The multi-wavelength kinds run in the launches and graph
 * forms of qpm_run, with plain FP32 scans; their states take (kappa1[0], kappa2[0]) as
 * the instance's problem. */
enum { QPM_OBJ_THG = 0, QPM_OBJ_SHG = 1, QPM_OBJ_MULTI_THG = 2, QPM_OBJ_MULTI_SHG = 3 };
typedef struct {
  int32_t kind;       /* QPM_OBJ_* */
  int32_t K;          /* multi-wavelength kinds: the number of problems */
  double kappa1[8];   /* multi-wavelength kinds: dk1 w (THG) or dk w (SHG) of problem k */
  double kappa2[8];   /* QPM_OBJ_MULTI_THG: dk2 w of problem k */
  float G0, beta;     /* multi-wavelength kinds: the reference value and the spread weight */
} qpm_objective;

/* Execution modes of qpm_run. */
enum {
  QPM_RUN_LAUNCHES = 0,   /* two kernels per generation, launched one by one */
  QPM_RUN_GRAPH = 1,      /* the same launches captured once into a CUDA graph */
  QPM_RUN_PERSISTENT = 2, /* one cooperative persistent kernel for all generations */
  QPM_RUN_BATCHED = 3     /* many instances in one launch (captured in a CUDA graph): each
                             thread-block cluster (qpm_set_batch_cluster) runs whole
                             instances from a largest-first queue; needs team = 32, the
                             default when n_inst > 1 */
};

const char *qpm_last_error(void);
const char *qpm_status_string(qpm_status s);
int32_t qpm_abi_version(void);

/* ---------------------------------------------------------------------------
 * Fitness (Sec. 2.1): d_eff and f = |d_eff|^2 of NP sign sequences.
 *   genes   device, float [NP][ld], row-major, ld >= N; only the sign is used
 *   signs   device, uint32 [NP][ld_words], ld_words >= ceil(N / 32)
 *   d_eff   device, float2 [NP] (re, im), units of w^2
 *   fit     device, float [NP] = |d_eff|^2 (may be NULL)
 *   compensated: 0 plain FP32 scan, 1 Kahan-compensated
 * The per-problem phasor table is built on first use of (device, N, kappa1,
 * kappa2) and cached by the library (library-owned device memory, released by
 * qpm_release_caches); the scan's partial results use a library-owned scratch
 * buffer grown on demand.  The cache holds at most 64 problems per device: a call
 * that needs room for new problems first synchronises the device and frees all of
 * that device's tables and scratch (never while another host thread's call is
 * between its table lookup and its launches).  Rows that start on 16-byte boundaries (genes or
 * signs 16-byte aligned, ld or ld_words a multiple of 4) are read with 16-byte
 * accesses; other rows are read 4 bytes at a time, which is slower but gives
 * results within the same tolerance.  Errors: N < 1, NP < 1, ld < N ->
 * QPM_ERR_ARG.
 * ------------------------------------------------------------------------- */
qpm_status qpm_eval(const qpm_problem *prob, const float *genes, int64_t ld, int32_t NP,
                    float *d_eff, float *fit, int32_t compensated, qpm_stream_t stream);
qpm_status qpm_eval_packed(const qpm_problem *prob, const uint32_t *signs, int64_t ld_words,
                           int32_t NP, float *d_eff, float *fit, int32_t compensated,
                           qpm_stream_t stream);

/* ---------------------------------------------------------------------------
 * Other objectives of the paper's designs (Sec. 2.1 and Sec. 5).
 * qpm_eval_shg: the SHG field integral int_0^L d(z) e^{-i dk z} dz (units of w) of
 *   each row, with dk w = prob->kappa1 (prob->kappa2 is ignored); e_shg device
 *   float2 [NP], fit device float [NP] = |e_shg|^2 (may be NULL).
 * qpm_eval_multi: the multi-wavelength objective of Sec. 5,
 *     f = sum_k |G0 - G_k| + beta (G_max - G_min),  G_k = |d_eff(probs[k])|,
 *   to be minimised, for K <= 4 problems of equal N sharing one read of the
 *   genes.  d_eff device float2 [NP][K] (may be NULL), objective device float [NP].
 *   scratch: caller-owned device memory of at least
 *   qpm_eval_multi_scratch_bytes(K, N, NP) bytes (segment partials).
 * Phasor tables as for qpm_eval.  Errors: K outside [1, 4], unequal N, N < 1,
 * NP < 1, ld < N, small scratch -> QPM_ERR_ARG.
 * ------------------------------------------------------------------------- */
qpm_status qpm_eval_shg(const qpm_problem *prob, const float *genes, int64_t ld, int32_t NP,
                        float *e_shg, float *fit, qpm_stream_t stream);
qpm_status qpm_eval_multi(const qpm_problem *probs, int32_t K, const float *genes, int64_t ld,
                          int32_t NP, float G0, float beta, float *d_eff, float *objective,
                          void *scratch, size_t scratch_bytes, qpm_stream_t stream);
size_t qpm_eval_multi_scratch_bytes(int32_t K, int32_t N, int32_t NP);

/* Allocation-free qpm_eval (no counterpart in the paper).  It exists for callers
 * that cannot allocate device memory: host callbacks and other code that must not
 * call into the allocator, processes whose device memory is all owned by an
 * external allocator, and real-time paths that cannot afford the implicit device
 * synchronisation of cudaMalloc/cudaFree.  Same arguments, layouts and result as
 * qpm_eval; it allocates nothing (no cudaMalloc/cudaFree, no allocating library
 * routine).  Its scratch lives in one fixed 16 MiB array in the library's device
 * image, which every GPU that loads the library holds until the process exits:
 *   bytes = 192 ceil(N / 4) (sign-block table, rounded up to 256)
 *         + 16 min(1024, ceil(N / 256)) + 256 (the constants and their partial sums)
 *         + 24 S NPpad (segment partials; NPpad = 32 ceil(NP / 32), S the number of
 *           segments the row sweep splits N into, which grows with the SM count)
 *   must not exceed 16777216.  On a 152-SM GB300 that admits N up to about 3.1e5
 *   domains for up to 256 rows, 2.75e5 for 1024 rows and 1.7e5 for 4096 rows.
 *   - The first call on each device looks up that array's device address
 *     (cudaGetSymbolAddress) with the device current; make this first call
 *     before any stream capture on that device.
 *   - Sizes whose scratch exceeds 16 MiB are rejected with QPM_ERR_ARG and a
 *     message stating the bytes needed; nothing is enqueued.
 *   - Every call rebuilds its tables in the shared array, so calls that overlap on
 *     the GPU (for example on different streams) race on it and must be serialised
 *     by the caller.  Nothing in the array needs to start at zero: each call
 *     writes every word it reads. */
qpm_status qpm_eval_noalloc(const qpm_problem *prob, const float *genes, int64_t ld, int32_t NP,
                            float *d_eff, float *fit, int32_t compensated, qpm_stream_t stream);

/* Free the cached phasor tables and scratch of the current device (synchronises it). */
qpm_status qpm_release_caches(void);

/* Measured issue rate of the current device for the ALU roofline (no counterpart
 * in the paper): kind 0 FFMA, 1 the 32 x 32 -> 64 multiply and xor of a Philox
 * round, 2 three-input xor (lane-ops per second, a wide multiply counting 2 ops),
 * 3 whole Philox4x32-10 calls of the library's generator per second; the result in
 * *lane_ops_per_s (host double).  Synchronous (about 10 ms); allocates and frees a
 * small device buffer.  Errors: kind outside [0, 3] -> QPM_ERR_ARG. */
qpm_status qpm_measure_issue_peak(int32_t kind, double *lane_ops_per_s, qpm_stream_t stream);

/* Measured latency on the current device for the latency floor of a generation of
 * the persistent form (no counterpart in the paper), in nanoseconds (*ns_out, host):
 *   kind 0: one grid barrier of the persistent kernel (the same code: release
 *           reduction on a counter, bounded acquire polling), `ctas` co-resident CTAs of
 *           256 threads, averaged over 2000 barriers in one cooperative launch;
 *   kind 1: one dependent load served by L2 (a single thread chasing a scrambled
 *           cyclic permutation of 16 MB that is L2-resident), averaged over 8192 loads;
 *           `ctas` is ignored;
 *   kind 2: the kind 0 barrier with relaxed arrival and polling (no ordering: how
 *           fast an arrival reaches the pollers at all);
 *   kind 3: one gpu-scope fence per CTA between two CTA barriers, no cross-CTA wait;
 *   kind 4: an all-to-all exchange without a counter: every CTA publishes a
 *           round-tagged 8-byte word and its threads poll every CTA's word;
 *   kinds 2-4 per round, `ctas` CTAs of 256 threads, 2000 rounds as for kind 0.
 * Synchronous (a few ms); allocates and frees its device buffers (256 bytes plus 16
 * per CTA, or 16 MB).  Errors: NULL output, kind outside [0, 4], ctas outside [1, the
 * co-resident CTA count] for kinds 0 and 2-4 -> QPM_ERR_ARG; a wait that ran out (1 s,
 * or 2^22 polls for kinds 2 and 4) -> QPM_ERR_TIMEOUT. */
qpm_status qpm_measure_latency(int32_t kind, int32_t ctas, double *ns_out, qpm_stream_t stream);

/* Exhaustive self-check of one of the library's arithmetic shortcuts against
 * the plain operation it replaces (no counterpart in the paper), over all 2^32
 * 32-bit patterns x:
 *   kind 0: the GWO mean's division by 3 (Markstein's residual correction of
 *           x * RN(1/3)) against the IEEE division x / 3 (two NaNs agree);
 *   kind 1: the GWO's r1 and 2 r2 built in the significand of a float in [1, 2)
 *           or [2, 4) against the same values through int-to-float conversions,
 *           r1 = (x >> 16) 2^-16, r2 = (x & 0xFFFF) 2^-16;
 *   kind 2: the crossover test as one integer compare (x <= 256 floor(2^24 CR)
 *           + 255) against U <= CR in FP32, U = (x >> 8) 2^-24, for CR = 0,
 *           2^-24, 1.5 2^-24, 0.5, 0.9f and its two neighbours, 1.
 * *mismatches (host) receives the number of differing results (bitwise for
 * values), *first_bad (host) the smallest pattern with one, or 0xFFFFFFFF.
 * Synchronous (a few ms); allocates and frees 12 device bytes.
 * Errors: kind outside [0, 2] or a NULL output -> QPM_ERR_ARG. */
qpm_status qpm_selfcheck(int32_t kind, uint64_t *mismatches, uint32_t *first_bad,
                         qpm_stream_t stream);

/* ---------------------------------------------------------------------------
 * Relaxed fitness and its adjoint (no counterpart in the paper's method, which
 * works on +-1 domains; used to polish the GWO leaders and exposed for
 * gradient-based design).  Each row theta_r[0..N) defines real domain values
 * d_j = tanh(theta_j); d_eff is the Sec. 2.1 integral for that piecewise-
 * constant d (exact for real d: phi1 phi2 sum_j a_j P_j + psi sum_j d_j^2 p1_j p2_j).
 *   theta      device float [B][ld], ld >= N
 *   d_eff      device float2 [B] (fwd out, bwd in)
 *   fit        device float [B] = |d_eff|^2 (fwd, may be NULL)
 *   saved      device float [B][qpm_relaxed_saved_floats(N)], 16-byte aligned,
 *              caller-owned: the forward fills it (it is also the forward's
 *              workspace) and the backward reads it.  Floats 0-1 of each row
 *              hold sum_a = sum_j d_j e^{-i kappa2 j}; the rest holds the
 *              row's prefix sums at segment starts (about N/16 floats).
 *   grad_fit   device float [B] upstream gradient dL/df (NULL = all ones)
 *   grad_theta device float [B][ld_grad] out: dL/dtheta = grad_fit * df/dtheta
 * Phasor table as for qpm_eval (cached per problem).  Errors: N < 1, B < 1,
 * ld < N, NULL theta, d_eff, saved or grad_theta, misaligned saved -> QPM_ERR_ARG.
 * Rows whose pitch is a multiple of 16 bytes are read as TMA tiles, whose device
 * waits are bounded (2 s): a wait that runs out makes that call's d_eff, fit or
 * gradient NaN rather than returning an error (the calls are asynchronous).
 * Nothing past a row's N floats is read into the sums or written.
 * ------------------------------------------------------------------------- */
int64_t qpm_relaxed_saved_floats(int32_t N);
qpm_status qpm_deff_relaxed_fwd(const qpm_problem *prob, const float *theta, int64_t ld,
                                int32_t B, float *d_eff, float *fit, float *saved,
                                qpm_stream_t stream);
qpm_status qpm_deff_relaxed_bwd(const qpm_problem *prob, const float *theta, int64_t ld,
                                int32_t B, const float *d_eff, const float *saved,
                                const float *grad_fit, float *grad_theta, int64_t ld_grad,
                                qpm_stream_t stream);

/* ---------------------------------------------------------------------------
 * Optimiser state: n_inst independent HWSDA instances (uneven N, kappa, NP
 * allowed), all resident on the current device.
 *   qpm_create   allocates the state (library-owned device memory) and returns
 *                it in *out; synchronous; nothing is launched.
 *   qpm_init     Step 1 of Sec. 3.2: phasor tables, x_ij = U(-1,1) (Sec. 2.2.1
 *                step 1) and the fitness of every individual; generation := 0.
 *   qpm_step     one generation (Sec. 3.2 Steps 2-6) of every instance.
 *   qpm_run      `generations` generations in the given QPM_RUN_* mode (every
 *                instance advances by the same count).
 *                QPM_RUN_PERSISTENT returns QPM_ERR_TIMEOUT if a bounded
 *                device-side wait gave up (checked after synchronising the stream).
 *   qpm_destroy  frees the state (synchronises the device first).
 * Errors: NP < 4, N < 1, G < 1, F outside [0, 2] or CR outside [0, 1] -> QPM_ERR_ARG;
 * qpm_step/qpm_run before qpm_init -> QPM_ERR_STATE; running past G -> QPM_ERR_ARG.
 * ------------------------------------------------------------------------- */
typedef struct qpm_state qpm_state;

qpm_status qpm_create(const qpm_problem *probs, const qpm_params *params, int32_t n_inst,
                      qpm_state **out);
qpm_status qpm_init(qpm_state *st, qpm_stream_t stream);
qpm_status qpm_step(qpm_state *st, qpm_stream_t stream);
qpm_status qpm_run(qpm_state *st, int32_t generations, int32_t mode, qpm_stream_t stream);
qpm_status qpm_destroy(qpm_state *st);

/* Size of instance `inst` (host int32 outs, each may be NULL): domains N, population
 * NP and generations G, as given to qpm_create.  Lets a caller size the buffers of
 * the calls below.  Errors: bad state or instance -> QPM_ERR_ARG. */
qpm_status qpm_instance_shape(const qpm_state *st, int32_t inst, int32_t *N_out, int32_t *NP_out,
                              int32_t *G_out);

/* The F of every generation of instance `inst`: F_out device float [G + 1], entry g
 * the F the DE phase of generation g uses (constant F: F everywhere; decaying F: the
 * schedule; adaptive F: the values computed so far, entry g + 1 written during
 * generation g).  Enqueued on `stream`.  Errors: bad state, instance or NULL output ->
 * QPM_ERR_ARG; before qpm_init -> QPM_ERR_STATE. */
qpm_status qpm_get_F(qpm_state *st, int32_t inst, float *F_out, qpm_stream_t stream);

/* Restore the F history of instance `inst` from F_in (device float [G + 1], e.g. from
 * qpm_get_F of the run being resumed), so that an adaptive-F run (f_schedule 2) resumed
 * with qpm_set_population in another state uses the F it would have used.  Enqueued on
 * `stream`.  Errors: bad state, instance or NULL input, or f_schedule 0 -> QPM_ERR_ARG. */
qpm_status qpm_set_F(qpm_state *st, int32_t inst, const float *F_in, qpm_stream_t stream);

/* generation counter of the state as seen by the host (host int32 out) */
qpm_status qpm_generation(const qpm_state *st, int32_t *g_out);

/* Current population of instance `inst`, in natural order:
 *   genes_out device float [NP][ld] (ld >= N), fit_out device float [NP] (may be NULL),
 *   d_eff_out device float2 [NP] (may be NULL).  Enqueued on `stream`. */
qpm_status qpm_get_population(qpm_state *st, int32_t inst, float *genes_out, int64_t ld,
                              float *fit_out, float *d_eff_out, qpm_stream_t stream);

/* Checkpoint / resume: replace the population of instance `inst` (after qpm_init)
 * by genes (device float [NP][ld], natural order, e.g. from qpm_get_population)
 * and set the generation counter to `generation`.  Fitness is recomputed with the
 * library's own scan, so it equals the value the saved run held bit for bit; since
 * every random number is a function of (seed, instance, generation, individual,
 * gene), continuing from a checkpoint reproduces the uninterrupted run exactly.
 * Single-instance states, or states whose instances are all at `generation`.
 * Errors: generation outside [0, G], ld < N -> QPM_ERR_ARG. */
qpm_status qpm_set_population(qpm_state *st, int32_t inst, const float *genes, int64_t ld,
                              int32_t generation, qpm_stream_t stream);

/* Best individual of instance `inst` (largest f, lowest index on ties) with its
 * d_eff re-evaluated in FP64 on the device:
 *   genes_out device float [N], d_eff64_out device double [2], fit_out device float [1]
 *   (each may be NULL), index_out device int32 [1] (may be NULL). */
qpm_status qpm_get_best(qpm_state *st, int32_t inst, float *genes_out, double *d_eff64_out,
                        float *fit_out, int32_t *index_out, qpm_stream_t stream);

/* Gradient polish of the three best individuals of instance `inst` (build
 * add-on; the paper has no counterpart): theta = tau x, `steps` ascent steps
 * theta += lr g / max_j |g_j| with g the adjoint of the relaxed fitness
 * (qpm_deff_relaxed_*), then x' = clamp(theta / tau, -1, 1); x' replaces x only if
 * its +-1 fitness is >= the current one.  accepted_out (device int32 [3], may be
 * NULL) receives 1 where a leader was replaced.  Allocates a small state-owned
 * scratch on first use (call once before any stream capture).  Errors: steps < 0,
 * lr < 0 or tau <= 0 -> QPM_ERR_ARG. */
qpm_status qpm_polish_leaders(qpm_state *st, int32_t inst, int32_t steps, float lr, float tau,
                              int32_t *accepted_out, qpm_stream_t stream);

/* The objective of instance `inst` (Sec. 2.1, Sec. 5; see qpm_objective): host call,
 * before qpm_init; allocates the other problems' phasor tables of a multi-wavelength
 * kind (state-owned).  Errors: an unknown kind, K outside its range, non-finite
 * kappa or G0, beta < 0 -> QPM_ERR_ARG; after qpm_init or on another device ->
 * QPM_ERR_STATE.  qpm_run then returns QPM_ERR_UNSUPPORTED for the multi-wavelength
 * kinds in the persistent and batched forms, and qpm_polish_leaders for every kind
 * but QPM_OBJ_THG. */
qpm_status qpm_set_objective(qpm_state *st, int32_t inst, const qpm_objective *obj);

/* Threads per individual the state uses for instance `inst` (host int32 out). */
qpm_status qpm_team_of(const qpm_state *st, int32_t inst, int32_t *team_out);

/* Batched form (QPM_RUN_BATCHED): CTAs per thread-block cluster, 1 (default), 2, 4
 * or 8.  An instance is run by all CTAs of one cluster (its individuals dealt to
 * their warps, the generation's two dependencies as cluster barriers), so a large
 * instance no longer holds one SM while the others have finished; the per-
 * individual arithmetic, and hence every result, is the same for every size.  An
 * execution choice with no counterpart in the paper; autotune.py picks it by
 * measurement.  Host call; synchronises the device if a batched launch was already
 * captured.  Errors: other values -> QPM_ERR_ARG; a size the device cannot
 * co-schedule -> QPM_ERR_UNSUPPORTED; the current device is not the state's ->
 * QPM_ERR_STATE. */
qpm_status qpm_set_batch_cluster(qpm_state *st, int32_t ctas);

/* Test hook: record FP32 fitness values of instance `inst` into trace (device,
 * float [NP * (1 + 2G)]): [0, NP) after init, then for generation g the trial
 * fitness at NP*(1+2g) and the GWO candidate fitness at NP*(2+2g) (NaN for the
 * three leaders, which do not move).  NULL disables.  Must be set before qpm_init. */
qpm_status qpm_set_trace(qpm_state *st, int32_t inst, float *trace);

/* Upper bound, in nanoseconds, on every device-side wait of the persistent kernel
 * (grid barriers; default 5 s).  A wait that reaches it makes the kernel record
 * QPM_ERR_TIMEOUT and return; qpm_run then reports QPM_ERR_TIMEOUT.  No GPU
 * trap is ever raised.  Test hook and safety valve; host-only, takes effect at
 * the next qpm_run. */
qpm_status qpm_set_wait_timeout_ns(qpm_state *st, uint64_t ns);

/* End to end with host buffers: create, init, run all G generations (mode as in
 * qpm_run), copy the best genes (host float [N]) and its FP64 d_eff (host
 * double [2]) back, destroy.  Synchronous.  best_fit (host float [1]) may be NULL. */
qpm_status qpm_solve(const qpm_problem *prob, const qpm_params *params, int32_t mode,
                     float *best_genes_host, double *best_deff64_host, float *best_fit_host);

#ifdef __cplusplus
}
#endif
#endif /* QPM_H_ */
