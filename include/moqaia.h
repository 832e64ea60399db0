/*
 * moqaia.h -- C ABI of the B300 library for multi-objective MaxCut sampled by
 * noise-injected simulated bifurcation (NI-SB), after "Multi-Objective Optimization
 * by Quantum-Annealing-Inspired Algorithms" (arXiv 2604.26477).
 *
 * Pipeline (one round): weight vectors -> moq_sample (SB replicas, packed spins)
 * -> moq_evaluate_cuts (exact K-objective cut values) -> moq_pareto_front (dedup +
 * non-dominated filter merged into a device archive) -> moq_hypervolume (exact).
 *
 * Conventions shared by every call:
 *  - Return value: MOQ_OK (0) or a negative MOQ_ERR_* code. No C++ exception and no
 *    abort crosses this interface. moq_last_error_message() gives a per-thread text.
 *  - Memory: pointers documented "device" are caller-owned device memory of the
 *    current CUDA device; "host" pointers are ordinary host memory. The library
 *    allocates device memory only inside instance and archive handles, at creation,
 *    and frees it in the matching destroy call.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream). Calls are
 *    stream-ordered and asynchronous unless documented as synchronising.
 *  - Spin packing: a configuration s in {-1,+1}^n is W = ceil(n/64) uint64 words;
 *    bit (i mod 64) of word i/64 is 1 exactly when s_i = -1. Bits >= n are 0.
 *    Arrays of configurations are row-major: sample m occupies words [m*W, m*W+W).
 *  - Cut vectors are int64, row-major M x K.
 *  - Limits: 2 <= n, n <= 2^24 (sampler: n <= 1024 per replica block), 2 <= K <= 8,
 *    weights are int32, E < 2^31.
 */
#ifndef MOQAIA_H
#define MOQAIA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif
#if defined(__GNUC__)
#pragma GCC visibility push(default) /* the library is built with hidden visibility */
#endif

/* ---- status codes ------------------------------------------------------------- */
#define MOQ_OK 0
#define MOQ_ERR_ARG -1         /* invalid argument (range, duplicate edge, NULL) */
#define MOQ_ERR_OOM -2         /* device allocation failed */
#define MOQ_ERR_CUDA -3        /* a CUDA runtime call or kernel launch failed */
#define MOQ_ERR_TIMEOUT -4     /* a device-side wait ran out of its budget */
#define MOQ_ERR_CAPACITY -5    /* the archive (or a buffer) is too small */
#define MOQ_ERR_OVERFLOW -6    /* a result would leave the exact integer range */
#define MOQ_ERR_UNSUPPORTED -7 /* valid request outside what the library implements */

/* ---- SB variants ("Simulated Bifurcation with Gaussian noise") ----------------- */
#define MOQ_DSB 0 /* discrete SB: phi(x) = sgn(x) */
#define MOQ_BSB 1 /* ballistic SB: phi(x) = x */
#define MOQ_PREC_FP32 0 /* state and step arithmetic in FP32 */
#define MOQ_PREC_FP16 1 /* state and step arithmetic in FP16, the paper's float16 (moq_sample) */
#define MOQ_LAYOUT_PLAIN -1  /* moq_create_instance_layout: slots by decreasing degree, rows by column */
#define MOQ_LAYOUT_DEFAULT 0 /* moq_create_instance_layout: the bank-conflict planner at its default effort */

typedef struct moq_instance moq_instance;
typedef struct moq_archive moq_archive;

/* Summary of an instance, filled by moq_instance_get_info. */
typedef struct moq_instance_info {
    int32_t n, K;
    int64_t E;
    int32_t max_degree;
    int32_t words;            /* W = ceil(n/64) */
    int64_t weight_sum[8];    /* W_k = sum_E J^(k) */
    int64_t abs_sum[8];       /* sum_E |J^(k)|, bounds every cut range */
    int64_t ref_point[8];     /* r_k = sum_E min(0, J^(k)): C_k(s) >= r_k for every s */
    float features[8];        /* graph statistics of the learned proposal (not in the paper):
                                 log n, mean degree / 10, mean_k mean|w_k| / rms(w_k),
                                 mean_k std(w_k) / rms(w_k), fraction of positive weights,
                                 mean, min, max pairwise Pearson correlation of the w_k */
} moq_instance_info;

/* Parameters of one sampling call ("Simulated Bifurcation with Gaussian noise"). */
typedef struct moq_sample_params {
    int32_t variant;       /* MOQ_DSB or MOQ_BSB */
    int32_t steps;         /* T >= 0 Euler steps */
    float dt;              /* time step (paper: 1) */
    float a0;              /* pump ceiling a0 (paper: 1) */
    float alpha;           /* noise amplitude of Eq. NI-SB (0 = plain SB) */
    float init_amp;        /* x, y start uniform in [-init_amp, init_amp) */
    int32_t noise_sqrt_dt; /* 0: y += dt*alpha*eta (Euler of Eq. NI-SB); 1: alpha*sqrt(dt)*eta */
    const float* schedule; /* device, T entries a_m, or NULL for a_m = a0*m/(T-1) */
    const float* x_init;   /* device R x n, or NULL (Philox start) */
    const float* y_init;   /* device R x n, or NULL (zero when x_init is given) */
    float* x_out;          /* device R x n final positions, or NULL */
    float* y_out;          /* device R x n final momenta, or NULL */
    uint32_t replica_offset; /* added to r in the Philox replica counter (batches: the instance's offset) */
    int32_t precision;     /* MOQ_PREC_FP32 (default) or MOQ_PREC_FP16 (moq_sample and per-instance batches only) */
} moq_sample_params;

/* Result of moq_hypervolume: value = hi * 2^64 + (uint64)lo (a signed 128-bit int). */
typedef struct moq_hv {
    int64_t lo;
    int64_t hi;
    double approx; /* the same value rounded to double */
} moq_hv;

/* Fills p with the paper's defaults: dSB, T = 1000, dt = 1, a0 = 1, alpha = 0,
 * init_amp = 0.1, noise y += dt*alpha*eta, linear pump, no optional arrays. */
void moq_default_params(moq_sample_params* p);

/* ---- a1: instance build ("Hamiltonian formulation of multi-objective MaxCut") ---
 * Graph G = (V, E), |V| = n, edge e = (ei[e], ej[e]) with 0 <= ei[e] < ej[e] < n, and K
 * integer weight sets: w[k*E + e] = J^(k) of edge e (host, row k = objective k).
 * Builds the device graph (both-direction CSR with per-entry weights, integer row
 * sums sum_j J^(k)_ij, W_k, sum |J^(k)|, r_k). Synchronises `stream`.
 * Errors: MOQ_ERR_ARG (n < 2, K outside [2, 8], E < 0, an endpoint out of range,
 * ei >= ej, a repeated edge, NULL pointers with E > 0), MOQ_ERR_OOM, MOQ_ERR_CUDA.
 * Ownership: inputs are copied; *out is owned by the caller until destroyed. */
int moq_create_instance(int32_t n, int32_t K, int64_t E, const int32_t* ei, const int32_t* ej,
                        const int32_t* w, void* stream, moq_instance** out);
/* a1 with the sparse samplers' memory layout chosen by the caller instead of the environment
 * (the layout is an implementation detail with no counterpart in the paper; it changes the
 * order of the FP32 force sums only, see moq_plan_gather_layout): layout = MOQ_LAYOUT_PLAIN
 * keeps slots by decreasing degree and rows by column (no host search: 0.2 ms for a 1024-spin
 * build instead of several ms, the better choice when the instance is sampled for only a few
 * short rounds), MOQ_LAYOUT_DEFAULT runs the bank-conflict planner, m > 0 adds the longer
 * search with m slot exchanges per spin. Reads no environment variable, so builds on several
 * host threads may each pass their own layout. Everything else is moq_create_instance.
 * Errors: MOQ_ERR_ARG (layout < MOQ_LAYOUT_PLAIN), then those of moq_create_instance. */
int moq_create_instance_layout(int32_t n, int32_t K, int64_t E, const int32_t* ei, const int32_t* ej,
                               const int32_t* w, int32_t layout, void* stream, moq_instance** out);
/* a1 for a dense weight matrix: J_upper (host, K x n(n-1)/2, row k = objective k) holds
 * J^(k)_ij for the pairs i < j in row order ((0,1), (0,2), .., (0,n-1), (1,2), ..). The
 * pairs with a non-zero weight in some objective become the edges, in that order; the
 * rest is moq_create_instance. Errors: MOQ_ERR_ARG (n outside [2, 65536], K outside
 * [2, 8], NULL), then those of moq_create_instance. Synchronises `stream`. */
int moq_create_instance_dense(int32_t n, int32_t K, const int32_t* J_upper, void* stream, moq_instance** out);
/* The sparse samplers' memory layout as moq_create_instance chooses it for graphs of n <= 1024
 * with degrees <= 8 (an implementation detail with no counterpart in the paper): the slot of
 * each spin in the samplers' shared-memory state and the order in which each spin gathers its
 * neighbours, chosen by a seeded local search against shared-memory bank conflicts (a warp's
 * 4-byte reads conflict-free when their words differ modulo 32, 8-byte reads when each
 * half-warp's differ modulo 16). Gather order changes only the order of the FP32 force sums.
 * Host only (no GPU, no allocation visible to the caller). Out: slot_spin[n] (slot -> spin);
 * gather[2E] (rows in spin order, row i holding spin i's neighbours in gather order, row
 * lengths the degrees); passes[4] or NULL: 8-byte and 4-byte shared-memory passes of one
 * gather step over all warps for the column layout, then for the chosen one. Setting
 * MOQ_SB_LAYOUT=0 in the environment makes moq_create_instance keep slots by decreasing
 * degree and rows by column (moq_create_instance_layout takes the choice as an argument); MOQ_SB_LAYOUT_EFFORT=m > 0 adds, for regular graphs whose blocks
 * hold one replica per slot, a longer search (m * n slot exchanges, about 0.15 ms per exchange
 * per spin at n = 1024: worth it for long jobs) aimed at the 8-byte gathers, kept where it is
 * better; both are read on every call. Errors: MOQ_ERR_ARG (NULL outputs), MOQ_ERR_UNSUPPORTED (n
 * outside [2, 1024], a degree above 8, an invalid or repeated edge, E = 0). */
int moq_plan_gather_layout(int32_t n, int64_t E, const int32_t* ei, const int32_t* ej, int32_t* slot_spin, int32_t* gather,
                           int64_t* passes);
void moq_destroy_instance(moq_instance* inst);
int moq_instance_get_info(const moq_instance* inst, moq_instance_info* out);

/* ---- a2..a5: sampling ("Simulated Bifurcation with Gaussian noise", Eq. NI-SB) ---
 * R replicas; replica r runs SB on J(c) = sum_k c_k J^(k) with c = lambda[r*K..r*K+K)
 * (device, float, Eq. H_total; rows are used as given, the paper takes sum c = 1):
 *   c0 = 1/max_i |sum_j J(c)_ij| (1/max_i sum_j |J(c)_ij| if all row sums vanish,
 *   1 if J(c) = 0); force c0 * sum_j (-J(c)_ij) phi(x_j) (the negated coupling, so that
 *   the attractors minimise H_total, i.e. maximise the weighted cut);
 *   y += dt*(-(a0 - a_m) x + force + alpha*eta); x += dt*a0*y; |x| > 1 -> x = sgn x, y = 0;
 *   s = sgn(x) with sgn(0) = +1, written to bits (device, R x W words).
 * eta comes from Philox4x32-10 with key = seed and counter (m >> 3, i, o + r, round)
 * (o = p->replica_offset): word (m & 7) >> 1 gives two Gaussians by Box-Muller on its
 * 16-bit halves, u1 = (low + 1) 2^-16, u2 = high 2^-16 (cosine for even m, sine for odd m);
 * the start state from counter (0xFFFFFFFF, i, o + r, round). `seed` and `round` fully
 * determine the output on a given GPU build. The whole trajectory of a block of replicas
 * runs on-chip in one launch; each thread runs one spin of one replica or, where that keeps
 * more replicas in flight per SM (degree bound <= 4), of two (same results; the
 * environment variable MOQ_SB_PAIR = 0 / 1 forces a form).
 * p->precision = MOQ_PREC_FP16 runs the paper's float16 ("Results and discussion": SB in
 * float16): x, y, the couplings -c0 J(c), phi and every multiply-add of a step in FP16
 * (two replicas per thread as packed half2; c0 and J(c) formed in FP32, then rounded once);
 * the start state, the pump value and eta are the FP32 form's, rounded to FP16. Degree
 * bound 8. Per-step force error against FP64: at most (deg + 2) 2^-11 c0 sum_j |J(c)_ij phi_j|.
 * Errors: MOQ_ERR_ARG (R < 0, steps < 0, bad variant or precision, NULL lambda/bits with
 * R > 0), MOQ_ERR_UNSUPPORTED (n > 1024, max degree > 16, or > 8 with FP16), MOQ_ERR_CUDA.
 * Asynchronous. */
int moq_sample(const moq_instance* inst, const float* lambda, int32_t R, const moq_sample_params* p,
               uint64_t seed, uint64_t round, uint64_t* bits, void* stream);

/* ---- batched sampling of many instances (the paper runs every weight vector and replica
 * "in parallel in a single run", "Results and discussion") ------------------------------
 * A batch fixes `count` instances (same K, n <= 1024, max degree <= 8; host array of
 * handles, kept alive by the caller) and replicas[b] replicas of each. Inputs and outputs are
 * concatenated: lambda_all holds sum_b replicas[b] rows of K floats, instance b starting at
 * row replica_offsets[b]; bits_all holds instance b's replicas[b] x W_b words from word
 * word_offsets[b] (moq_batch_layout fills both arrays, count + 1 entries each). One
 * persistent launch runs every (instance, replica block) work item, longest first, from a
 * device queue; instance b's replicas use Philox replica counters replica_offsets[b] + r, so
 * the result equals moq_sample on instance b with p->replica_offset = replica_offsets[b].
 * The tile shape (threads per block, spin slots per thread) affects speed only; results
 * do not depend on it. moq_batch_create allocates the work tables (device); errors:
 * MOQ_ERR_ARG, MOQ_ERR_UNSUPPORTED, MOQ_ERR_OOM. */
typedef struct moq_batch moq_batch;
int moq_batch_create(const moq_instance* const* insts, int32_t count, const int32_t* replicas, moq_batch** out);
void moq_batch_destroy(moq_batch* b);
int moq_batch_layout(const moq_batch* b, int64_t* replica_offsets, int64_t* word_offsets);
/* block_threads in {256, 512, 1024}, slots_per_thread in {1, 2}, block_threads *
 * slots_per_thread >= the largest n; *items_out (may be NULL) = work items. (0, 0) selects
 * per-instance mode: moq_sample_batch then launches the single-instance sampler once per
 * instance (largest first, replica counters from the instance's offset), whose blocks are
 * sized per instance, round-robin over internal streams (MOQ_BATCH_STREAMS, default 4,
 * created by the first such call) that fork from and join back into the caller's stream;
 * the samples are the same bits either way. Synchronous. */
int moq_batch_set_tiles(moq_batch* b, int32_t block_threads, int32_t slots_per_thread, int32_t* items_out);
/* Active replicas per instance (host array of count entries): instance b then samples, and
 * moq_evaluate_cuts_batch evaluates, its first replicas[b] replicas only (0 skips it), with
 * the layout and the noise counters of the batch unchanged, so a driver can drop the
 * instances that have reached their target. 0 <= replicas[b] <= the count given at
 * creation, else MOQ_ERR_ARG. Synchronous (the persistent kernel's work list is rebuilt). */
int moq_batch_set_replicas(moq_batch* b, const int32_t* replicas);
/* Samples every active replica of every instance (asynchronous; p's state arrays must be
 * NULL; p->precision = MOQ_PREC_FP16 runs in the per-instance mode only). */
int moq_sample_batch(moq_batch* b, const float* lambda_all, const moq_sample_params* p, uint64_t seed, uint64_t round,
                     uint64_t* bits_all, void* stream);
/* Exact cut values (Eq. single_obj) of every sample: cuts_all row replica_offsets[b] + m
 * holds C(s) of instance b's sample m (device, sum replicas x K int64). Asynchronous. */
int moq_evaluate_cuts_batch(const moq_batch* b, const uint64_t* bits_all, int64_t* cuts_all, void* stream);

/* ---- a3 dense: tensor-core sampler (same dynamics as moq_sample; the force
 * c0 sum_k c_k (J^(k) Phi)_i is a matrix product) -----------------------------------------
 * moq_dense_create copies the instance's couplings into K zero-padded n_pad x n_pad BF16
 * matrices (n_pad = n rounded up to 128; integers |J| <= 256 are exact), their residuals
 * (moq_sample_dense_split) and E4M3 matrices with row scales (moq_sample_dense_fp8), and
 * allocates the replica state for up to max_replicas (x, y FP32, four BF16 and two E4M3 phi
 * buffers, each ceil(max_replicas/128)*128 x n_pad). K <= 4, n <= 16384. The instance must outlive it.
 * moq_sample_dense runs T step kernels (tcgen05.mma BF16 -> FP32 products for every
 * objective, fused update/wall/phi epilogue) on `stream`, then writes the packed signs
 * (and x_out/y_out if given); with n_pad = 128 and K <= 3 one launch runs all T steps with
 * J, phi and the state held on chip (same results; MOQ_DENSE_RESIDENT=0 at create time keeps
 * the per-step kernels). Differences from moq_sample: phi is rounded to BF16 for the
 * products (exact for dSB), the force is combined as -c0 sum_k c_k G_k, and the noise of
 * step m for replica r is Gaussian number r & 7 of Philox(key = seed, counter = (m, i,
 * 2^30 + (r >> 3), round)) (word (r & 7) >> 1, Box-Muller on 16-bit halves as in
 * moq_sample); the start state uses the same counter as moq_sample.
 * replica_offset must be 0. Errors: MOQ_ERR_ARG, MOQ_ERR_UNSUPPORTED, MOQ_ERR_OOM,
 * MOQ_ERR_CUDA; a device wait that ran out of its 2 s budget is reported as
 * MOQ_ERR_TIMEOUT by moq_dense_status (synchronises, clears the flag). */
typedef struct moq_dense moq_dense;
int moq_dense_create(const moq_instance* inst, int32_t max_replicas, moq_dense** out);
void moq_dense_destroy(moq_dense* d);
int moq_sample_dense(moq_dense* d, const float* lambda, int32_t R, const moq_sample_params* p, uint64_t seed, uint64_t round,
                     uint64_t* bits, void* stream);
int moq_dense_status(moq_dense* d, void* stream);

/* FP8 form of the dense dSB step (precision growth of the force contraction): the couplings
 * as E4M3 with one power-of-two scale per row and objective (J^(k)_ij = 2^e J8_ij, e >= 0
 * the smallest with max_j |J^(k)_ij| <= 448 2^e; integers |J| <= 16 are exact, larger ones
 * round to 4 significant bits) and phi = sgn(x) as exact +-1 E4M3, multiplied by
 * tcgen05.mma kind::f8f6f4 with FP32 accumulation; the row scale is applied to each
 * accumulator in the epilogue. Same arguments, start state, noise and update as
 * moq_sample_dense (with |J| <= 16 the two give identical results); the per-step kernel is
 * used for every n. dSB only: p->variant = MOQ_BSB returns MOQ_ERR_UNSUPPORTED (x would
 * round to 4 significant bits). Buffers are allocated by moq_dense_create. Errors as
 * moq_sample_dense; a timed-out device wait shows in moq_dense_status. */
int moq_sample_dense_fp8(moq_dense* d, const float* lambda, int32_t R, const moq_sample_params* p, uint64_t seed,
                         uint64_t round, uint64_t* bits, void* stream);

/* Split-precision form of the dense step on the tensor cores: J = BF16(J) + J_res with the
 * residual J - BF16(J) exact in BF16 (|J| <= 65408), and for bSB phi = phi_hi + phi_lo with
 * phi_hi = BF16(x), phi_lo = BF16(x - phi_hi); each K-chunk is multiplied in passes into the
 * same FP32 accumulator: (BF16(J) + J_res) phi for dSB -- the exact integer products, so the
 * results equal those of moq_sample_dense_fp32 whenever every row sum of |J| stays below
 * 2^24 -- and BF16(J) phi_hi + J_res phi_hi + BF16(J) phi_lo for bSB (relative error of the
 * products about 2^-16, inside the FP32 force bound 1e-5). Two (dSB) or three (bSB) times
 * the products of moq_sample_dense. Same arguments, start state, noise and update as
 * moq_sample_dense; the per-step kernel is used for every n. Errors as moq_sample_dense,
 * and MOQ_ERR_UNSUPPORTED when some |J| > 65408. */
int moq_sample_dense_split(moq_dense* d, const float* lambda, int32_t R, const moq_sample_params* p, uint64_t seed,
                           uint64_t round, uint64_t* bits, void* stream);

/* ---- a3 dense, plain FP32 form on the CUDA cores (same dynamics as moq_sample_dense)
 * The force c0 sum_k c_k (J^(k) Phi)_i of the SB equations with J^(k) and phi in FP32 and
 * every product and sum in FP32: the full-precision comparison for the tensor-core form.
 * moq_dense_fp32_create copies the couplings into K zero-padded n_pad x n_pad FP32 matrices
 * (n_pad = n rounded up to 64; integers |J| < 2^24 are exact) and allocates x, y and two
 * phi buffers (FP32, ceil(max_replicas/128)*128 x n_pad each). K <= 4, n <= 16384. The
 * instance must outlive the handle. moq_sample_dense_fp32 takes the arguments of
 * moq_sample_dense and draws the same start state and the same noise (the counters of
 * moq_sample_dense), combines the force in the same order and applies the same update, so
 * for dSB with integer couplings whose row sums of |J| stay below 2^24 (every per-objective
 * product exact in both forms) and |J| <= 256 (exact in BF16) the two forms give identical
 * results; otherwise they differ by the BF16 rounding of J (and of x for bSB) only.
 * Asynchronous on `stream`; replica_offset must be 0. Errors: MOQ_ERR_ARG,
 * MOQ_ERR_UNSUPPORTED, MOQ_ERR_OOM, MOQ_ERR_CUDA. */
typedef struct moq_dense_fp32 moq_dense_fp32;
int moq_dense_fp32_create(const moq_instance* inst, int32_t max_replicas, moq_dense_fp32** out);
void moq_dense_fp32_destroy(moq_dense_fp32* d);
int moq_sample_dense_fp32(moq_dense_fp32* d, const float* lambda, int32_t R, const moq_sample_params* p, uint64_t seed,
                          uint64_t round, uint64_t* bits, void* stream);

/* a6 for dense instances on the tensor cores, exact: C_k(s) (Eq. single_obj) of M packed
 * configurations bits (device, M x W words, bit set for s_i = -1; M <= max_replicas) into
 * cuts (device, M x K int64, row-major), the same values as moq_evaluate_cuts. Uses
 * s^T J_k s = 2 sum_E J_e s_i s_j, so C_k = (2 W_k - s^T J_k s) / 4, with J_k split as
 * 256 J_hi + J_lo (both exact in BF16) and products accumulated exactly in FP32 tiles then
 * 64-bit integers. Reuses the handle's buffers: stream-ordered with moq_sample_dense on
 * the same handle. Errors: MOQ_ERR_ARG (M out of range, NULL pointers),
 * MOQ_ERR_UNSUPPORTED (some |J| > 65408: use moq_evaluate_cuts), MOQ_ERR_CUDA.
 * Asynchronous; a device wait that ran out of its budget shows in moq_dense_status. */
int moq_dense_evaluate_cuts(moq_dense* d, const uint64_t* bits, int32_t M, int64_t* cuts, void* stream);

/* ---- a6: exact cut values, Eq. (single_obj) -------------------------------------
 * cuts[m*K + k] = C_k(s^(m)) = sum over edges with s_i != s_j of J^(k)_ij, for the M
 * packed configurations bits (device, M x W) into cuts (device, M x K int64).
 * Exact (integer). Errors: MOQ_ERR_ARG, MOQ_ERR_CUDA. Asynchronous. */
int moq_evaluate_cuts(const moq_instance* inst, const uint64_t* bits, int64_t M, int64_t* cuts, void* stream);

/* ---- a7: Pareto filter with dedup into a device archive ("Pareto filtering") ----
 * The archive holds the distinct non-dominated cut vectors seen so far (maximisation:
 * u dominates v iff u_k >= v_k for all k and u_j > v_j for some j), each with one
 * representative configuration -- the one with the lowest global sample index,
 * canonicalised to s_0 = +1 (C(s) = C(-s)) -- and that index.
 * capacity: most vectors the archive can hold; max_batch: most candidates per call.
 * Device memory for both is allocated here. Errors: MOQ_ERR_ARG, MOQ_ERR_OOM. */
int moq_archive_create(int32_t n, int32_t K, int64_t capacity, int64_t max_batch, moq_archive** out);
void moq_archive_destroy(moq_archive* a);
/* Empties the archive (stream-ordered). */
int moq_archive_reset(moq_archive* a, void* stream);
/* Merges M candidates (cuts: device M x K int64; bits: device M x W) whose global
 * sample indices are index_base + m; callers give increasing index_base across calls,
 * so earlier members win ties. If front_size_out is non-NULL the call synchronises and
 * writes the new archive size there (and reports a capacity overflow as
 * MOQ_ERR_CAPACITY); otherwise it is asynchronous and an overflow -- which leaves
 * the archive unchanged -- is reported by the next synchronising archive call.
 * Errors: MOQ_ERR_ARG (M < 0 or M > max_batch, NULL), MOQ_ERR_CAPACITY, MOQ_ERR_CUDA. */
int moq_pareto_front(moq_archive* a, const int64_t* cuts, const uint64_t* bits, int64_t M, int64_t index_base,
                     int64_t* front_size_out, void* stream);
/* The front of the union of two sample sets ("Pareto filtering": the non-dominated set of a
 * pool does not depend on how the pool was split): merges every member of src (its cut
 * vector, configuration and global sample index) into dst, in batches of dst's max_batch.
 * On a cut vector present in both, dst's member is kept. The exchange step of a run split
 * over several devices or processes (gather the parts' fronts, merge them). Synchronises
 * once to read src's size; the merge itself is stream-ordered and src must not change
 * meanwhile. Errors: MOQ_ERR_ARG (NULL, dst == src, different n or K), MOQ_ERR_CAPACITY
 * (pending in src, or reported by the next synchronising call on dst), MOQ_ERR_CUDA. */
int moq_archive_merge(moq_archive* dst, const moq_archive* src, void* stream);
/* Archive size (synchronises). Returns a pending capacity error, if any. */
int moq_archive_size(const moq_archive* a, int64_t* size_out, void* stream);
/* Copies up to cap members to host arrays (cuts_host cap x K, bits_host cap x W,
 * index_host cap; any may be NULL) and the size to *n_out. Synchronises. */
int moq_archive_copy_out(const moq_archive* a, int64_t* cuts_host, uint64_t* bits_host, int64_t* index_host,
                         int64_t cap, int64_t* n_out, void* stream);
/* Device pointers to the current archive arrays (valid until the next merge/reset). */
int moq_archive_device_view(const moq_archive* a, const int64_t** cuts, const uint64_t** bits,
                            const int64_t** index, const int64_t** size_dev);

/* ---- a8: hypervolume ("Hamiltonian formulation" Eq. HV, Appendix A) -------------
 * Exact Lebesgue measure of the union of boxes prod_k [ref_k, y_k] over the archive
 * front (maximisation), in 128-bit integers; points with some y_k < ref_k span an
 * empty box and are left out. ref: host, K int64. *out: host. K in {2, 3, 4}.
 * Synchronises. Errors: MOQ_ERR_ARG, MOQ_ERR_UNSUPPORTED (K > 4),
 * MOQ_ERR_OVERFLOW (product of the K side lengths >= 2^125), MOQ_ERR_CUDA. */
int moq_hypervolume(const moq_archive* a, const int64_t* ref, moq_hv* out, void* stream);
/* a8 for several archives at once, the stop test of a driver over many instances (the
 * repeat-until-covered loop of "Results and discussion", one hypervolume per instance and
 * round): out[i] = moq_hypervolume(archives[i], refs + i*K), the same exact integer value,
 * with two synchronisations of `stream` in all instead of two per archive (the front sizes
 * are read back together, then every archive's computation is queued and the results are
 * read back together). archives: `count` handles of one K (2..4); refs: host, count x K,
 * row i = the reference point of archive i; out: host, count results (zero for an empty
 * front). Errors: MOQ_ERR_ARG (count < 0, NULL, archives of different K),
 * MOQ_ERR_UNSUPPORTED (K > 4), MOQ_ERR_CAPACITY (an archive overflowed: reported for the
 * first such archive, every such latch cleared, as moq_archive_size does), MOQ_ERR_OVERFLOW,
 * MOQ_ERR_CUDA; on an error the outputs past the failing archive are left zero. */
int moq_hypervolume_many(const moq_archive* const* archives, const int64_t* refs, int32_t count, moq_hv* out,
                         void* stream);
/* The same for an arbitrary point set: pts device F x K int64 (need not be
 * non-dominated). workspace: device scratch of moq_hypervolume_workspace_size(F, K)
 * bytes, 256-byte aligned, owned by the caller. */
int64_t moq_hypervolume_workspace_size(int64_t F, int32_t K);
int moq_hypervolume_points(const int64_t* pts, int64_t F, int32_t K, const int64_t* ref, void* workspace,
                           moq_hv* out, void* stream);
/* Allocation-free variant of moq_hypervolume_points (the paper has no counterpart: it
 * exists for callers that cannot allocate device memory when they need a result, e.g.
 * code whose device memory is owned by another allocator, or loops where a cudaMalloc
 * or cudaFree would stall the whole device). The scratch is a fixed array in the
 * library's own device memory, sized for moq_hypervolume_noalloc_max_points() points
 * (16384) of up to 4 objectives, about 1.4 MB on every GPU that loads the library,
 * held until the process exits. The call allocates nothing; the caller still owns pts,
 * ref and out, and the 20 result bytes are read back into the call's own stack frame (no
 * pinned host buffer either). Every call looks up the current device's address of the
 * array, so a cudaDeviceReset between calls, which can move it, is harmless. Every call
 * shares the one array and leaves its contents behind, so calls that overlap on the GPU
 * (e.g. from two streams at once) race; calls in sequence are safe (the call
 * synchronises its stream).
 * Errors: MOQ_ERR_CAPACITY (F above the limit), otherwise as moq_hypervolume_points. */
int64_t moq_hypervolume_noalloc_max_points(void);
int moq_hypervolume_points_noalloc(const int64_t* pts, int64_t F, int32_t K, const int64_t* ref, moq_hv* out,
                                   void* stream);

/* ---- a2: weight vectors ("Scalarization via the weighted sum method", App. B) ----
 * Das-Dennis lattice of resolution H: c in {0, 1/H, .., 1}^K with sum 1 (interior != 0:
 * every c_k > 0, the paper's choice), lexicographically ascending in (m_1..m_K), c = m/H.
 * Writes min(count, capacity) rows to lambda (device, float) and count to *count_out.
 * Errors: MOQ_ERR_ARG, MOQ_ERR_CAPACITY (count > capacity). Asynchronous. */
int moq_lambda_das_dennis(int32_t K, int32_t H, int32_t interior, float* lambda, int64_t capacity,
                          int64_t* count_out, void* stream);
/* R vectors uniform on the simplex (Dirichlet(1,..,1)): c_k = e_k / sum e, e_k = -ln u_k,
 * u_k = ((word >> 8) + 1) 2^-24 with word k & 3 of Philox4x32-10(key = seed,
 * counter = (r, k >> 2, 0x4C414D42, round)). lambda: device R x K float. Asynchronous. */
int moq_lambda_dirichlet(int32_t K, int32_t R, uint64_t seed, uint64_t round, float* lambda, void* stream);

/* ---- a9 learned weight-vector proposal (not in the paper) ----------------------------
 * A surrogate MLP (d_in -> 128 -> 128 -> d_out, ReLU; d_in <= 16, d_out <= 8) predicts the
 * normalised cut vector an SB replica reaches for a given weight vector and graph
 * statistics: y = W3 relu(W2 relu(W1 x + b1) + b2) + b3. Parameters are one flat vector
 * (W1 [128 x d_in], b1, W2 [128 x 128], b2, W3 [d_out x 128], b3, row-major): an FP32
 * master copy for the optimiser and a BF16 copy that every kernel computes with (FP32
 * accumulation). moq_mlp_create allocates parameters, Adam state, per-block gradient slots
 * for up to max_batch rows and proposal scratch for up to max_candidates, and initialises
 * the weights He-uniform from Philox(seed) (biases 0). */
typedef struct moq_mlp moq_mlp;
int moq_mlp_create(int32_t d_in, int32_t d_out, int32_t max_batch, int32_t max_candidates, uint64_t seed, moq_mlp** out);
void moq_mlp_destroy(moq_mlp* m);
int64_t moq_mlp_param_count(const moq_mlp* m);
/* Host copies of the parameters (synchronous): set writes the FP32 master and refreshes the
 * BF16 copy; get reads the master, or the BF16 copy widened to float if bf16_rounded. */
int moq_mlp_set_params(moq_mlp* m, const float* params_host);
int moq_mlp_get_params(const moq_mlp* m, float* params_host, int32_t bf16_rounded);
/* Y (device B x d_out) = MLP(X) for X (device B x d_in). Asynchronous. */
int moq_mlp_forward(const moq_mlp* m, const float* X, int32_t B, float* Y, void* stream);
/* Mean squared error L = 1/(B d_out) sum (y - t)^2 of the batch X, T (device, B <= max_batch)
 * and its gradient, kept for moq_mlp_adam_step; grad_out (device, P floats) and loss_out
 * (device, 1 float) receive copies when non-NULL. Deterministic (fixed reduction order). */
int moq_mlp_gradient(moq_mlp* m, const float* X, const float* T, int32_t B, float* grad_out, float* loss_out, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with the last gradient. */
int moq_mlp_adam_step(moq_mlp* m, float lr, void* stream);
/* moq_mlp_gradient followed by moq_mlp_adam_step in two launches instead of three (the
 * gradient sum and the update share one pass): the same parameters bit for bit. loss_out
 * (device, 1 float) may be NULL. Asynchronous; errors: MOQ_ERR_ARG. */
int moq_mlp_train_step(moq_mlp* m, const float* X, const float* T, int32_t B, float lr, float* loss_out, void* stream);
/* Which kernels run the products of moq_mlp_forward, moq_mlp_gradient, moq_mlp_train_step and
 * the proposal's predictions (set per handle; default MOQ_MLP_CUDA_CORES):
 *  MOQ_MLP_CUDA_CORES   FP32 activations, FP32 multiply-adds on the CUDA cores;
 *  MOQ_MLP_TENSOR_CORES every matrix product (forward, the backward products and the weight
 *                       gradients) a tcgen05 MMA with BF16 operands and FP32 accumulation in
 *                       TMEM, one CTA per 128-row tile: inputs, activations and the
 *                       backpropagated deltas are rounded to BF16 where they enter a product;
 *                       sums, relu masks, the loss and the bias gradients stay FP32. Its
 *                       gradient is that of the FP64 network with those roundings (within FP32
 *                       summation error), and within a few BF16 units (2^-8) of the exact
 *                       network's. Deterministic (fixed reduction order).
 * Errors: MOQ_ERR_ARG. */
#define MOQ_MLP_CUDA_CORES 0
#define MOQ_MLP_TENSOR_CORES 1
int moq_mlp_set_engine(moq_mlp* m, int32_t engine);
/* Synchronises `stream`; MOQ_ERR_TIMEOUT if a tensor-core wait of an earlier call ran out of
 * its 2 s budget (the call then left its outputs unwritten), which also clears the flag. */
int moq_mlp_status(moq_mlp* m, void* stream);
/* Training rows from M samples (device): X[m] = [lambda[m] (K), features (host, n_features)],
 * T[m][k] = (cuts[m][k] - offset[k]) / scale[k] (host offset, scale: K int64; the learned
 * proposal uses the reference point and sum |J^(k)|, so targets lie in [0, 1]). X: M x
 * (K + n_features), T: M x K, device float. Asynchronous. */
int moq_mlp_make_rows(int32_t K, int32_t n_features, const float* lambda, const int64_t* cuts, int64_t M, const float* features,
                      const int64_t* offset, const int64_t* scale, float* X, float* T, void* stream);
/* Proposes R weight vectors: n_candidates uniform-simplex candidates (moq_lambda_dirichlet
 * with seed, round) get the MLP prediction p from [candidate, features]; each is scored by
 * gap(p) = min over archive members f of max_k (p_k - (f_k - offset_k) / scale_k), the
 * distance by which the prediction reaches beyond the nearest front member, and the R best
 * (ties: lower candidate index) are written to lambda_out (device R x K) in score order.
 * d_in must equal K + n_features. offset, scale: host K int64 (the cut normalisation used for
 * the targets). Asynchronous. */
int moq_lambda_propose(moq_mlp* m, const moq_archive* a, const float* features, int32_t n_features, const int64_t* offset,
                       const int64_t* scale, int32_t n_candidates, uint64_t seed, uint64_t round, float* lambda_out, int32_t R,
                       void* stream);

/* ---- handle memory --------------------------------------------------------------
 * Instances and archives take their device arrays from a memory pool the library keeps
 * per device: memory freed by moq_destroy_instance / moq_archive_destroy stays reserved
 * for the next handle instead of going back to the driver. moq_release_cached_memory
 * returns the unused part of the current device's pool to the driver (synchronises the
 * device; handles that are alive keep their memory). Errors: MOQ_ERR_CUDA. */
int moq_release_cached_memory(void);

/* ---- errors -------------------------------------------------------------------- */
/* moq_strerror: a fixed text for a status code. moq_last_error_message and moq_last_status:
 * the message and the code of the last call on this thread that failed (a successful call
 * leaves both unchanged; "" and MOQ_OK before any failure). */
const char* moq_strerror(int code);
const char* moq_last_error_message(void);
int moq_last_status(void);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif
#ifdef __cplusplus
}
#endif
#endif /* MOQAIA_H */
