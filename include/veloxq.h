/*
 * veloxq.h -- C ABI of a GB300 (sm_103a) implementation of the data-parallel
 * hot path of the physics-inspired QUBO solver benchmarked in
 * "VeloxQ: A Fast and Efficient QUBO Solver" (arXiv:2501.19221).
 *
 * The problem (Sec. 2, eq. qubo_model; read as a sum over every stored entry):
 *     minimise  E(x) = sum_{i,j} Q_ij x_i x_j + sum_i c_i x_i ,  x in {0,1}^n .
 * Ising input (Sec. 2, eq. ising_model) H(s) = sum_{i<j} J_ij s_i s_j +
 * sum_i h_i s_i is mapped to a QUBO by App. A (eq. qij_SK).
 *
 * The solver integrates R replicas of a ballistic simulated-bifurcation
 * system (App. B, eqs. sbm2/sbm without the quartic term, with walls at
 * |s| = 1) in lockstep. With Qs = (Q + Q^T)/2, Qoff its off-diagonal part and
 * b = Qs 1 + c, one step k (of K) is
 *     F   = Qoff s                       (local field, the dominant product)
 *     phi = -(F + b)/2
 *     y  <- y + dt (-(a0 - a_k) s + c0 phi)
 *     s  <- s + dt a0 y ;   |s| > 1 => s = sign(s), y = 0
 * and the readout is x = [s > 0] (App. B, s_i = sign(q_i)). The exact energy of
 * the read-out vectors is kept as best-so-far per replica; the result is the
 * lowest energy over replicas (lowest replica index on ties).
 *
 * Conventions shared by every entry point:
 *  - Every call returns a veloxq_status (0 = OK) and never aborts. On failure
 *    veloxq_last_error() returns a thread-local message.
 *  - Host pointers are owned by the caller and only read or written during
 *    the call. Calls that take host pointers synchronise their stream before
 *    returning.
 *  - Entry points whose name ends in _dev take DEVICE pointers (for instance
 *    from PyTorch tensors) owned by the caller; they are enqueued on the
 *    context's stream and return without synchronising.
 *  - State blocks (S, Y, F) are replica-major float32: element (r, i) of R
 *    replicas of n variables is at r*n + i. Binary batches are uint8 [B][n]
 *    with values 0/1.
 *  - A context owns every device buffer it allocates; veloxq_destroy frees
 *    them. A context is not thread-safe; different contexts are independent
 *    (they may be created, used and destroyed from different threads at once).
 *  - Freed device buffers (of contexts and of a call's temporaries) go to a
 *    cache of the library, after the device has finished the work issued so
 *    far, and later buffers of the same device reuse them: up to 8 GiB per
 *    device stays allocated for the process's lifetime. An allocation that
 *    fails frees that device's cache and is tried once more. Setting the
 *    environment variable VELOXQ_ALLOC_CACHE=0 before the first call sends
 *    every freed buffer back to cudaFree instead.
 *  - A context lives on the device that was current when it was created;
 *    every later call on it needs that device current (EINVAL otherwise).
 */
#ifndef VELOXQ_H
#define VELOXQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct veloxq_ctx veloxq_ctx; /* opaque, library-owned */

typedef enum {
    VELOXQ_OK = 0,
    VELOXQ_EINVAL = -1,      /* invalid argument or input (message says which) */
    VELOXQ_ENOMEM = -2,      /* device or host allocation failed */
    VELOXQ_ECUDA = -3,       /* CUDA runtime error (no device, launch failure) */
    VELOXQ_ETIMEDOUT = -4,   /* a bounded device-side wait gave up */
    VELOXQ_EUNSUPPORTED = -5 /* a valid request that the library or the device cannot run */
} veloxq_status;

/* Element type of a coupling array passed in. */
typedef enum { VELOXQ_I8 = 0, VELOXQ_I32 = 1, VELOXQ_F32 = 2, VELOXQ_F64 = 3 } veloxq_vtype;

/* Operand precision of the dense local-field product F = Qoff S. FP32 runs on
 * the CUDA cores; the others run on the tcgen05 tensor cores; all accumulate
 * in FP32. Sparse contexts always use FP32 (or exact int8 couplings).
 *   BF16:          bf16(Qoff) x bf16(s).
 *   FP8:           Qoff as E4M3 with one FP32 scale per row (amax_i / 448);
 *                  S (whose entries the walls keep in [-1, 1]) with the fixed
 *                  scale 448 as two E4M3 terms, v = 448 s, hi = e4m3(v),
 *                  lo = e4m3(v - hi), both multiplied by the same Qoff operand
 *                  into one FP32 accumulator. The field's error is then that of
 *                  Qoff's rounding (about 2.7% normwise on Gaussian couplings).
 *   FP8_ONE_TERM:  the same with S as hi alone: half the tensor-core work, but
 *                  both operands rounded to 4 significant bits (about 3.7%
 *                  normwise). Parallel Annealing's operand (+-1) is exact in one
 *                  term, so FP8 runs it this way too.
 * BF16 and FP8 run every step up to a readout in one persistent launch; its
 * tiles go column block (256 replicas) by column block, in groups of two
 * blocks for BF16 and FP8_ONE_TERM. The environment variable
 * VELOXQ_TC_COLGROUP (1 to 16 blocks per group) fixes the group; the results
 * are the same bits for every group. */
typedef enum {
    VELOXQ_PREC_FP32 = 0,
    VELOXQ_PREC_BF16 = 1,
    VELOXQ_PREC_FP8 = 2,
    VELOXQ_PREC_FP8_ONE_TERM = 3
} veloxq_prec;

/* Kernel path selection. VELOXQ_PATH_AUTO picks by size and format: BF16 and
 * FP8 on dense contexts take the dense path; FP32 on dense contexts the
 * resident kernel when it fits, else the dense path; sparse contexts the
 * resident kernel when its couplings fit in shared memory, else the
 * streaming path. */
typedef enum {
    VELOXQ_PATH_AUTO = 0,
    VELOXQ_PATH_RESIDENT = 1,  /* sparse rows, whole run in one launch, state in shared memory */
    VELOXQ_PATH_STREAM = 2,    /* sparse rows, one fused launch per step, state in HBM */
    VELOXQ_PATH_DENSE = 3      /* dense Q, one fused field+update launch per step */
} veloxq_path;

/* Integrator (App. B). Each step forms the field F = Qoff o of an operand o
 * of the state (s, y) and applies one update, with phi = -(F + b)/2:
 *   BSB: ballistic simulated bifurcation (default). o = s;
 *        y <- y + dt(-(a0 - a_k) s + c0 phi), s <- s + dt a0 y, and
 *        |s| > 1 => s = sign(s), y = 0.
 *   ASB: adiabatic simulated bifurcation as App. B prints it (quartic
 *        potential, no walls). o = s;
 *        y <- y + dt(-(s^2 + a0 - a_k) s + c0 phi), s <- s + dt a0 y.
 *        Not available with the FP8 precisions (|s| is unbounded).
 *   PA:  Parallel Annealing (App. B): s holds the analog spins x, y the
 *        momenta m; o = sign(s) (+1 where s > 0, else -1);
 *        g = lambda_k s - c0 phi with lambda_k = (a0 - a_k)/a0,
 *        m <- momentum m - dt g, x <- clip(x + m, -1, 1).
 * The readout is x = [s > 0] for all three. veloxq_grad needs BSB. */
typedef enum { VELOXQ_METHOD_BSB = 0, VELOXQ_METHOD_ASB = 1, VELOXQ_METHOD_PA = 2 } veloxq_method;

/* Integration schedule. App. B fixes a0 = 1, c0 = 1/lambda_max(J) and a(t)
 * increasing linearly through the bifurcation at a(t) ~ a0; the rest is not
 * given by the paper and has the defaults below. The Ising coupling of the
 * dynamics is J = -Qoff/2, so the default c0 is kappa / rho(J) with rho the
 * spectral radius, estimated when the context is created (48 Lanczos steps;
 * power iteration in one CTA for small sparse instances): from below, within
 * 2% of rho on the instance families the tests cover. */
typedef struct {
    float dt;               /* step size; default 0.5 */
    float a0;               /* default 1 */
    float kappa;            /* c0 = kappa / rho(J) unless c0 > 0; default 1 */
    float c0;               /* > 0 overrides kappa / rho(J); default 0 */
    float sigma0;           /* initial s, y ~ U(-sigma0, sigma0); default 0.1 */
    int32_t n_knots;        /* 0 => a(t) through {0, a0}, i.e. a_k = a0 k/(K-1) */
    const float* a_knots;   /* host, n_knots values spread evenly over steps 0..K-1 */
    int32_t readout_every;  /* read out every this many steps (and after the last); 0 => last only */
    veloxq_prec prec;       /* dense field operand precision; default FP32 */
    veloxq_path path;       /* default AUTO */
    veloxq_method method;   /* integrator; default BSB */
    float momentum;         /* PA momentum alpha in [0, 1); default 0.9 */
} veloxq_schedule;

/* Context facts computed at creation. */
typedef struct {
    int64_t n;              /* variables */
    int64_t nnz_field;      /* stored off-diagonal entries of Qs (n*(n-1) for dense) */
    int32_t is_dense;       /* 1 for dense contexts */
    int32_t is_integer;     /* 1 when Q and c are integer-valued: energies are exact int64 */
    double rho;             /* spectral radius of Qoff (Lanczos or power-iteration estimate) */
    double K0;              /* E(x) = s^T Qoff s / 4 + b^T s / 2 + K0 for s = 2x - 1 */
    double ising_offset;    /* Ising contexts: H(s) = 2 E(x) + ising_offset; else 0 */
} veloxq_info;

/* Device timing of the last veloxq_solve or veloxq_grad on a context, from
 * CUDA events recorded on the stream the kernels run on. For veloxq_grad,
 * ms_main is the reverse sweep (the adjoint step kernels, 3 launches per
 * step) and path is VELOXQ_PATH_STREAM. */
typedef struct {
    double ms_total;        /* first to last kernel of the solve (or gradient) */
    double ms_main;         /* the integration: the resident kernel, or the captured steps up to the last one */
    int64_t launches;       /* kernels this library launched for the solve */
    int32_t path;           /* veloxq_path that ran */
    int32_t main_launches;  /* launches inside ms_main (1 for the resident kernel, else the step kernels) */
    int32_t stream_gather;  /* streaming path: couplings gathered at a time (1, 4 or 6; timed per context
                               and replica count, or fixed by the environment variable
                               VELOXQ_STREAM_FORM="gather chunk", chunk in replicas as in stream_chunk,
                               EINVAL if it does not fit); else 0 */
    int32_t stream_chunk;   /* streaming path: replicas per chunk of the step's thread order (every row of
                               one chunk before the next; 0: all replicas at once); else 0 */
    int32_t batch_stages;   /* one-launch veloxq_solve_batch: pipeline stages of the autotuned form; else 0 */
    int32_t batch_group;    /* one-launch veloxq_solve_batch: replicas per work item (an instance's
                               replicas in groups of this size, each on its own CTA); else 0 */
} veloxq_timing;

/* Fill *s with the defaults listed above. */
void veloxq_schedule_default(veloxq_schedule* s);

/* ---------------------------------------------------------------------------
 * Creation (Sec. 2 problem statement; inputs as biases and couplings in dense
 * or sparse form, Sec. "Comparison of VeloxQ SDK and D-Wave Ocean SDK").
 * ------------------------------------------------------------------------- */

/* Dense QUBO. Q: host, n*n row-major of type vt, used as given (need not be
 * symmetric); c: host, n doubles, or NULL for c = 0. stream: a cudaStream_t to
 * run on, or NULL for the default stream. Q and c are copied to the device,
 * Qs/Qoff/b/K0 are formed there, and rho is estimated (see veloxq_schedule).
 * Errors: EINVAL for n < 1, NULL Q, non-finite values or n > 2^20; ENOMEM. */
int veloxq_create_dense(veloxq_ctx** out, int64_t n, veloxq_vtype vt, const void* Q,
                        const double* c, void* stream);

/* Sparse QUBO in CSR form. rowptr: host, n+1 int64 (rowptr[0] = 0,
 * non-decreasing); col: host, rowptr[n] int32 in [0, n), strictly increasing
 * within a row; val: host, rowptr[n] values of type vt. Diagonal entries are
 * linear terms. The sparsity pattern must be structurally symmetric (values
 * may differ: the dynamics use (Q + Q^T)/2, the energy uses Q as given).
 * Errors: EINVAL for a malformed CSR or non-finite values; EUNSUPPORTED for a
 * structurally non-symmetric pattern; ENOMEM. */
int veloxq_create_csr(veloxq_ctx** out, int64_t n, const int64_t* rowptr, const int32_t* col,
                      veloxq_vtype vt, const void* val, const double* c, void* stream);

/* Dense Ising model (Sec. 2, eq. ising_model): J host n*n row-major of type
 * vt, read from its strict upper triangle; h host n doubles or NULL. Mapped to
 * the QUBO of App. A (eq. qij_SK) on the device: Q_ij = J_ij (i != j),
 * Q_ii = h_i - sum_l J_il, with H(s) = 2 E(x) + ising_offset,
 * ising_offset = sum_{i<j} J_ij - sum_i h_i. Errors as veloxq_create_dense. */
int veloxq_create_ising_dense(veloxq_ctx** out, int64_t n, veloxq_vtype vt, const void* J,
                              const double* h, void* stream);

/* Sparse Ising model in CSR form (structurally symmetric pattern, no diagonal
 * entries; the coupling of a pair is the value stored at its (i<j) position).
 * Mapped to a QUBO as veloxq_create_ising_dense. Errors as veloxq_create_csr,
 * plus EINVAL for a stored diagonal entry. */
int veloxq_create_ising_csr(veloxq_ctx** out, int64_t n, const int64_t* rowptr, const int32_t* col,
                            veloxq_vtype vt, const void* J, const double* h, void* stream);

/* Third-order Ising cost function (HUBO, Sec. "HUBO" eqs. nn and mw3s)
 *   H(s) = sum_i h_i s_i + sum_q J_q s_pi s_pj + sum_q K_q s_ti s_tj s_tk
 * reduced to second order by the gadget of eq. reduction: one auxiliary
 * spin a_q (index n + q) per cubic term, which adds
 *   |K| [3 + sgn(K)(s_i + s_j + s_k + 2a) + 2a(s_i + s_j + s_k) + s_i s_j + s_j s_k + s_i s_k],
 * so that min over the auxiliary spins of the result equals H(s). Host only
 * (no device use). Inputs (host): h (n values, or NULL for 0), n2 pairs
 * (pi, pj, J2; i != j, repeated pairs add), n3 triples (ti, tj, tk, K3;
 * distinct indices). Outputs (host, caller-allocated): *n_out = n + n3;
 * rowptr (n + n3 + 1), col and val (capacity 2 (n2 + 6 n3)): the reduced
 * Ising couplings in the CSR form veloxq_create_ising_csr takes (each pair
 * at both positions with the same value, summed in the order of the terms;
 * columns sorted), *nnz_out
 * the stored entries; lin (n + n3) the reduced fields; *offset the constant,
 * so H_reduced(s, a) = sum_{i<j} J s s + sum lin s + *offset.
 * Errors: EINVAL (bad sizes, indices out of range or repeated within a term,
 * non-finite values, NULL arrays, n + n3 >= 2^31). */
int veloxq_hubo3_reduce(int64_t n, const double* h, int64_t n2, const int64_t* pi, const int64_t* pj,
                        const double* J2, int64_t n3, const int64_t* ti, const int64_t* tj, const int64_t* tk,
                        const double* K3, int64_t* n_out, int64_t* nnz_out, int64_t* rowptr, int32_t* col,
                        double* val, double* lin, double* offset);

/* The same reduction, numbered for locality: the original spins keep their
 * order, and each is followed by the auxiliary spins of the cubic terms whose
 * largest index it is (in term order), so that a term's auxiliary spin sits
 * next to its variables (for the chain of eq. nn: spin i at 2i - 2 from i = 2
 * on, term q's auxiliary right after spin q + 2). index (host,
 * caller-allocated, n + n3 entries) receives the reduced index of every spin:
 * original v at index[v], auxiliary q at index[n + q]; every other output is
 * veloxq_hubo3_reduce's relabeled by index, bit for bit. Errors: those of
 * veloxq_hubo3_reduce, and EINVAL for a NULL index. */
int veloxq_hubo3_reduce_local(int64_t n, const double* h, int64_t n2, const int64_t* pi, const int64_t* pj,
                              const double* J2, int64_t n3, const int64_t* ti, const int64_t* tj,
                              const int64_t* tk, const double* K3, int64_t* n_out, int64_t* nnz_out,
                              int64_t* rowptr, int32_t* col, double* val, double* lin, double* offset,
                              int64_t* index);

/* Failure-path self-test of the bounded device waits (the paper has no
 * counterpart; this is a property of the library). Launches one small
 * kernel that waits, with the same bounded wait every tensor-core kernel
 * uses, on a barrier that nothing arrives on: the wait gives up after
 * budget_cycles SM cycles, records its code and returns, and the device
 * stays usable. Returns VELOXQ_ETIMEDOUT (with the code in the message) when
 * that happened, ECUDA otherwise; EINVAL for a budget outside [1e3, 1e10].
 * Runs on the current device and the default stream. */
int veloxq_selftest_timeout(int64_t budget_cycles);

/* Release every device and host resource of ctx (NULL is a no-op). */
void veloxq_destroy(veloxq_ctx* ctx);

/* Thread-local message describing the last non-OK status of this thread. */
const char* veloxq_last_error(void);

/* Context facts (host struct written). */
int veloxq_get_info(veloxq_ctx* ctx, veloxq_info* info);

/* Change the stream later calls run on (a cudaStream_t, or NULL). A solve on
 * a NULL stream runs on a stream the context owns, ordered after the legacy
 * default stream; on a non-NULL stream it runs (and is graph-captured) there. */
int veloxq_set_stream(veloxq_ctx* ctx, void* stream);

/* Timing of the last veloxq_solve or veloxq_grad on ctx (EINVAL if none ran yet). */
int veloxq_last_timing(veloxq_ctx* ctx, veloxq_timing* timing);

/* ---------------------------------------------------------------------------
 * Solve (App. B dynamics, replicas evolved in parallel and the best kept;
 * the returned state comes with its energy, Sec. "Structure-exploiting
 * solvers"; the per-replica energies are the low-energy spectrum of
 * Sec. "Pegasus topology").
 * ------------------------------------------------------------------------- */

/* Run `replicas` replicas for `steps` steps from a Philox4x32-10 initial state
 * keyed by seed (counter (i_lo, i_hi, r, 0); word 0 -> s, word 1 -> y).
 * sched: NULL for defaults. Outputs (host; any may be NULL):
 *   x_best        n bytes 0/1, the best vector (lowest energy, lowest replica);
 *   E_best        its energy as a double;
 *   E_best_int    its exact int64 energy (integer contexts only, else untouched);
 *   E_per_replica `replicas` doubles, each replica's best energy.
 * Errors: EINVAL (replicas < 1 or > 2^20, steps < 1, bad schedule), EUNSUPPORTED (path
 * or precision not available for this context), ENOMEM, ECUDA. */
int veloxq_solve(veloxq_ctx* ctx, int32_t replicas, int32_t steps, const veloxq_schedule* sched,
                 uint64_t seed, uint8_t* x_best, double* E_best, int64_t* E_best_int,
                 double* E_per_replica);

/* Solve several independent contexts (for instance a batch of instances of
 * uneven size) with the same replicas, steps, schedule and seed. x_best[m] is
 * a host buffer of n_m bytes (or NULL), E_best[m] the best energy. Errors as
 * veloxq_solve; m-th failure reported with its index. */
int veloxq_solve_batch(veloxq_ctx* const* ctxs, int32_t count, int32_t replicas, int32_t steps,
                       const veloxq_schedule* sched, uint64_t seed, uint8_t* const* x_best,
                       double* E_best);
/* (veloxq_solve_batch, continued) When every context is dense, replicas is a
 * multiple of 16 in [16, 128], sched->prec is BF16, FP8 or FP8_ONE_TERM (not
 * with adiabatic SB) and sched->readout_every is 0, the whole batch runs as ONE
 * persistent tensor-core launch followed by the exact final-readout energies
 * of every instance in two more launches, captured as one CUDA graph that is
 * replayed by later solves of the same contexts, replicas, steps and schedule
 * (any seed); otherwise each context is solved in turn. The launch's work items are
 * replica groups of instances, assigned to CTAs longest-first; its form
 * (pipeline depth, replicas per work item) is picked by timing a short probe
 * of each candidate the first time a kind of batch is seen on a device, kept
 * for the process and, when the environment variable VELOXQ_TUNE_CACHE names
 * a file, read from and appended to it ("key=stages group" lines); the
 * environment variable VELOXQ_BATCH_FORM="stages group" fixes the form instead
 * (EINVAL if it does not fit). Every integrator (sched->method) runs in both
 * forms. */

/* Final state of context ctx after the last veloxq_solve_batch that ran the
 * persistent batched kernel (dense instances, readout only after the last
 * step): S, Y device [R][n] float32, R the replicas of that batch.
 * Errors: EINVAL if no such state is held for R replicas. */
int veloxq_batch_state_dev(veloxq_ctx* ctx, int32_t R, float* S, float* Y);

/* ---------------------------------------------------------------------------
 * Energies (Sec. 2, eq. qubo_model)
 * ------------------------------------------------------------------------- */

/* E(x) for a host batch X [batch][n] of 0/1 bytes. E: host, batch doubles (or
 * NULL); E_int: host, batch int64 (integer contexts only, else must be NULL).
 * Errors: EINVAL (batch < 0, NULL X with batch > 0, E_int on a real context). */
int veloxq_energy(veloxq_ctx* ctx, int64_t batch, const uint8_t* X, double* E, int64_t* E_int);

/* As veloxq_energy with device pointers; asynchronous on the context stream. */
int veloxq_energy_dev(veloxq_ctx* ctx, int64_t batch, const uint8_t* X, double* E, int64_t* E_int);

/* The same energies as veloxq_energy_dev for callers that must not allocate
 * device memory during the call: code running inside a custom or pooling
 * allocator (an allocation callback, an out-of-memory handler) that must not
 * re-enter cudaMalloc, processes that reserve their whole device-memory budget
 * up front and refuse later allocations, and loops that cannot afford the
 * device synchronisation an allocation may cause. (The paper has no
 * counterpart; this is a property of the library.)
 * Scratch is a fixed 4 MiB array in device memory that every GPU loading the
 * library keeps until the process exits; nothing is allocated or freed. The
 * first call on a device (and the first after a device reset) looks up that
 * array's device address, a one-time set-up that may load the library's
 * device code, so make that first call before any stream capture; the
 * context's device must be the current one (EINVAL otherwise). Limits:
 * batch <= 65535 and batch * groups <= 2^19, groups = 64 for sparse contexts
 * and ceil(n/64) for dense ones; larger batches are rejected with EINVAL and
 * a message giving the largest accepted batch. Every partial sum is written
 * before it is read, so nothing needs clearing between calls, but all calls
 * share the one array: calls that overlap on the GPU (different streams, or
 * different contexts on one device) race and must be serialised by the
 * caller. X, E, E_int: device pointers as in veloxq_energy_dev; asynchronous
 * on the context's stream. */
int veloxq_energy_dev_noalloc(veloxq_ctx* ctx, int64_t batch, const uint8_t* X, double* E, int64_t* E_int);

/* ---------------------------------------------------------------------------
 * Pieces of the step, for parity tests and for callers that drive the
 * integration themselves (device pointers, asynchronous).
 * ------------------------------------------------------------------------- */

/* Philox initial state S, Y [R][n] for seed and sigma0 (same draw as solve). */
int veloxq_init_state_dev(veloxq_ctx* ctx, int32_t R, uint64_t seed, float sigma0, float* S, float* Y);

/* Local field F = Qoff S for S [R][n] in the given operand precision (the FP8
 * forms quantise S with the fixed scale 448, so S must lie in [-1, 1]; FP8
 * takes two E4M3 terms of S, FP8_ONE_TERM one). Errors: EUNSUPPORTED for
 * BF16/FP8 on a sparse context. */
int veloxq_field_dev(veloxq_ctx* ctx, int32_t R, veloxq_prec prec, const float* S, float* F);

/* Advance S, Y [R][n] in place by steps k_begin .. k_begin+k_count-1 of a
 * K-step schedule, on the kernel path the schedule selects (the same kernels
 * veloxq_solve runs). If F_last is not NULL it receives the field used in the
 * last step. Errors: EINVAL for k_begin < 0 or k_begin + k_count > K. */
int veloxq_steps_dev(veloxq_ctx* ctx, int32_t R, int32_t k_begin, int32_t k_count, int32_t K,
                     const veloxq_schedule* sched, float* S, float* Y, float* F_last);

/* Spectral radius of Qoff as used for the default c0 (the creation-time estimate). */
int veloxq_spectral_radius(veloxq_ctx* ctx, double* rho);

/* ---------------------------------------------------------------------------
 * Differentiation of the unrolled integrator (adjoint of the step).
 * ------------------------------------------------------------------------- */

/* Loss L = mean_r E_relax(s_K,r) with E_relax(s) = s^T Qoff s/4 + b^T s/2 + K0
 * (the QUBO energy identity under x = (1+s)/2, evaluated at continuous s),
 * after `steps` steps from the Philox state of seed. Returns L and its
 * gradient w.r.t. dt, kappa (c0 = kappa/rho(J); w.r.t. c0 itself when
 * sched->c0 > 0) and the a(t) knots (n_knots values, or the 2 default knots).
 * Forward states are checkpointed every ckpt_every steps and each segment is
 * recomputed in the reverse sweep. Host outputs; any may be NULL. */
int veloxq_grad(veloxq_ctx* ctx, int32_t replicas, int32_t steps, const veloxq_schedule* sched,
                uint64_t seed, int32_t ckpt_every, double* loss, double* d_dt, double* d_kappa,
                double* d_knots);
/* (veloxq_grad, continued) Runs on the sparse-row path (CSR contexts);
 * device memory: (ceil(steps/ckpt_every) + ckpt_every + 2) x 2 x replicas x n
 * floats. Errors: EINVAL (replicas, steps or ckpt_every < 1, more than 64
 * knots), EUNSUPPORTED (dense context), ENOMEM. */

#ifdef __cplusplus
}
#endif
#endif /* VELOXQ_H */
