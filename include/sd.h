/*
 * sd.h -- C ABI of the simultaneous-diagonalisation Trotter simulator.
 *
 * The method (Kawase & Fujii, arXiv:2206.11664): the Hamiltonian
 * H = sum_j c_j P_j (Sec. 2.2, real c_j, P_j in {I,X,Y,Z}^n) is split on the
 * host into groups of mutually commuting terms (Sec. 2.3, greedy); each
 * group g is mapped by a Clifford circuit C_g found with the binary tableau
 * (Sec. 2.4 and 3.2, Algorithms 1-6) to diagonal Z-strings,
 *     P_j = C_g^dag (-1)^{r_j} Z^{m_j} C_g            (Eq. hami_sim_diag),
 * and one Trotter step applies, group after group, C_g, the diagonal phase
 *     psi[x] *= exp(-i dt sum_j c_j (-1)^{r_j + |x & m_j|})   (Sec. 3.4 item 3)
 * and C_g^dag (Eq. trotter_simul_diag).  All state-vector work runs in
 * CUDA kernels for sm_103a; the host does planning and scheduling only.
 *
 * Conventions.
 *   - Qubit q (the paper's qubit q+1) is bit q of every mask and of the
 *     amplitude index (Sec. 2.1 numbers basis states with qubit 1 as the
 *     least significant digit).
 *   - A Pauli string is a pair of n-bit masks (x, z): I (0,0), X (1,0),
 *     Z (0,1), Y (1,1).  Text strings: character q is qubit q.
 *   - A state is 2^n contiguous amplitudes in device memory, interleaved
 *     (re, im): float pairs for SD_C64, double pairs for SD_C128, starting
 *     on a 16-byte boundary (other addresses give SD_EINVAL; the library's
 *     copies move 16 bytes at a time).
 *
 * Errors.  Every call returns an sd_status; on failure nothing the caller
 * owns has been modified, except that a CUDA error (SD_ECUDA) or a timeout
 * raised after kernels were launched may leave the state partly updated.
 * sd_last_error() returns a message for the last failing call on a
 * context.  A context is not thread safe.
 *
 * Ownership.  The library copies terms and coefficients, owns the plan and
 * every device work buffer it allocates; the caller owns state buffers and
 * host output arrays.  No call frees or reallocates caller memory.
 *
 * Ordering.  sd_evolve, sd_evolve_observe, sd_evolve_pauli, sd_evolve_host
 * and sd_evolve_batch are asynchronous on the given CUDA stream (NULL =
 * legacy default stream); sd_expect and sd_grad synchronise the stream to
 * return host values.  sd_prepare, sd_prepare_batch and sd_autotune are
 * synchronous; sd_plan, sd_get_plan, sd_get_schedule and sd_count_passes are
 * host only.  A call whose programs are built (by sd_prepare or an earlier
 * identical call) only launches kernels and may be captured into a CUDA
 * graph.
 */
#ifndef SD_H
#define SD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sd_ctx sd_ctx;

typedef enum {
    SD_OK = 0,
    SD_EINVAL = 1,     /* invalid argument; nothing modified */
    SD_ENOMEM = 2,     /* host or device allocation failed */
    SD_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed */
    SD_ENOPLAN = 4,    /* sd_plan has not been called on this context */
    SD_ETIMEOUT = 5,   /* reserved: no kernel of this library waits on another
                          block, kernel or device, so no call returns it */
    SD_EINTERNAL = 6   /* a planner invariant failed (e.g. a term not diagonal) */
} sd_status;

typedef enum { SD_C64 = 0, SD_C128 = 1 } sd_dtype;

/* Gate kinds in plan views (application order). */
enum { SD_GATE_H = 0, SD_GATE_S = 1, SD_GATE_CNOT = 2, SD_GATE_CZ = 3 };

/* Planner options (sd_plan).  Zero-initialised = defaults. */
typedef struct {
    /* Skip rule of Sec. 3.2 (after Algorithm 5): 0 = none (every qubit goes
     * through steps (i)-(iv)); 1 = the paper's rule (qubits carrying only
     * I/Z are left alone, only I/X get H, both leave steps (i)-(iv));
     * 2 = rule 1 plus qubits carrying only I/Y get S then H.  -1 = default (2). */
    int skip_rule;
    /* Tile size of the state-vector passes, log2 amplitudes per CTA tile:
     * 0 = default (13 for complex64, 12 for complex128, or what sd_autotune
     * chose), else 9..13. */
    int tile_bits;
    /* Run-time specialisation of the tile passes (each pass compiled with
     * NVRTC for sm_103a, cached in memory and under $SD_JIT_CACHE or
     * ~/.cache/sd_jit): 0 = automatic (states of 20+ qubits with at most 512
     * passes per program), 1 = always on the tile path, -1 = never.  Falls
     * back to the precompiled interpreter kernel if NVRTC is unavailable. */
    int jit;
    /* Order of the greedy commuting partition (Sec. 2.3 asks only for a
     * greedy method): 0 = first fit in input order (default); 1 = first fit
     * in order of decreasing number of anticommuting terms (largest first);
     * 2 = DSATUR colouring; 3 = first fit in order of decreasing |c_j| (the
     * coefficients at sd_plan time).  1 and 2 take O(m^2) time. */
    int grouping;
    /* Register layout of the complex64 passes compiled at run time:
     * -1 = plain (16 amplitudes per thread as (re, im) pairs); 1 = paired
     * (qubit 0 kept in registers, so that a thread's amplitudes pair up along
     * it and its one-qubit gates, rotations, shared-memory exchanges and
     * global accesses run on packed pairs: fewer instructions, one more
     * register round in some passes); 0 = default (plain, or what
     * sd_autotune_shape chose).  Complex128 passes ignore it. */
    int layout;
    /* Prefetch buffers of the passes compiled at run time: 1 = one (the
     * next tile is loaded into it once every thread has read the current
     * one); 2 = two (the next two tiles are in flight while a block works on
     * a third; 64 KB more shared memory, used only where it fits); 3 = two
     * in the passes without a group exponential, one in the others; 0 =
     * default (what sd_autotune_shape chose, else 1 for complex64 and 2 for
     * complex128 states). */
    int prefetch;
    int reserved[2];
} sd_plan_opts;

/* Result of sd_autotune_shape: the shape kept, and milliseconds per step
 * for tile sizes K = 9..13 (last index) in the plain layout with one prefetch
 * buffer and with the dtype's two-buffer form (prefetch 3 for complex64, 2
 * for complex128) (first index 0, 1) and in the paired layout with the same
 * two (2, 3); 0 where not run. */
typedef struct {
    int best_k;
    int best_layout;          /* -1 plain, 1 paired; 0 on the on-chip path */
    int best_prefetch;        /* sd_plan_opts.prefetch value kept; 0 on the on-chip path */
    double ms[4][5];
} sd_tune_result;

/* Read-only view of a plan; pointers stay valid until the next sd_plan or
 * sd_destroy on the context. */
typedef struct {
    int n;
    int64_t m;
    int64_t n_groups;
    const int64_t *group_offsets;  /* n_groups + 1 offsets into group_terms   */
    const int64_t *group_terms;    /* m term indices, grouped, input order    */
    const uint64_t *masks;         /* m: Z mask m_j of C_g P_j C_g^dag         */
    const uint8_t *signs;          /* m: sign bit r_j                          */
    const int64_t *gate_offsets;   /* n_groups + 1 offsets (in gates)          */
    const int32_t *gates;          /* 3 int32 per gate: kind, a, b (b=-1 for 1q) */
    const uint64_t *cnot_cols;     /* n_groups * n: A_g e_q for the CNOT map x -> A_g x */
    const uint64_t *cnot_inv_cols; /* n_groups * n: A_g^-1 e_q                 */
} sd_plan_view;

/* Schedule statistics for one Trotter step of the tile path. */
typedef struct {
    int tile_bits;            /* K: log2 amplitudes per tile                */
    int64_t passes_per_step;  /* state passes (HBM read + write) per step  */
    int64_t rounds_per_step;  /* register rounds over all passes           */
    int64_t diag_passes;      /* passes that apply a group phase            */
    int onchip;               /* 1 if the whole state stays on chip (small n) */
} sd_schedule_stats;

/* Create a context for H = sum_j coeffs[j] * P_(xmask[j], zmask[j]) on n
 * qubits (Sec. 2.2).  1 <= n <= 40, m >= 1; a mask bit at or above n gives
 * SD_EINVAL.  Identity terms are allowed (a global phase).  Inputs are
 * copied. */
sd_status sd_create(int n, int64_t m, const uint64_t *xmask, const uint64_t *zmask,
                    const double *coeffs, sd_ctx **out);

/* Same, from text strings of length n over {I,X,Y,Z} (character q = qubit q;
 * lower-case letters are accepted; any other character gives SD_EINVAL). */
sd_status sd_create_str(int n, int64_t m, const char *const *paulis, const double *coeffs,
                        sd_ctx **out);

/* Replace the m coefficients (input term order) of a context.  The plan
 * (groups, circuits, masks) depends only on the Pauli strings and is kept;
 * device programs built for the old coefficients are dropped. */
sd_status sd_set_coeffs(sd_ctx *ctx, const double *coeffs);

/* Host planning: greedy partition into commuting groups (Sec. 2.3; first
 * fit in input order unless opts->grouping chooses another order),
 * independent generators (Appendix, Algorithm 6) completed to n commuting
 * rows, synthesis steps (i)-(iv) (Algorithms 2-5), and masks/signs of every
 * term by replaying the circuit on the full tableau (Eq. hami_sim_diag).
 * opts may be NULL.  Host only: no device memory is touched here. */
sd_status sd_plan(sd_ctx *ctx, const sd_plan_opts *opts);

/* Fills *out with a read-only view of the plan (layout in sd_plan_view);
 * SD_ENOPLAN before sd_plan.  Host only. */
sd_status sd_get_plan(const sd_ctx *ctx, sd_plan_view *out);

/* Statistics of the pass schedule that sd_evolve would run for this dtype
 * and Trotter order (1 or 2).  Host only. */
sd_status sd_get_schedule(sd_ctx *ctx, sd_dtype dtype, int order, sd_schedule_stats *out);

/* Builds, without launching anything, every program that
 * sd_evolve(ctx, ., dtype, dt, steps, order, .) runs: pass schedules, their
 * device tables and the kernels compiled at run time.  A later sd_evolve
 * with the same arguments then starts launching at once.  Synchronous;
 * SD_EINVAL / SD_ENOPLAN as for sd_evolve. */
sd_status sd_prepare(sd_ctx *ctx, sd_dtype dtype, double dt, int64_t steps, int order);

/* sd_evolve on a state held in host memory: the 2^n amplitudes of
 * `dtype` at host_state (page-locked: cudaHostAlloc, cudaHostRegister or
 * torch pin_memory; pageable memory gives SD_EINVAL) are copied to d_work
 * (a caller-owned device buffer of the same size), evolved there, and copied
 * back, the copies done by kernels that read and write the host buffer
 * through its mapped address.  Asynchronous on the stream: host_state holds
 * the result once the stream has reached this point. */
sd_status sd_evolve_host(sd_ctx *ctx, void *host_state, void *d_work, sd_dtype dtype, double dt,
                         int64_t steps, int order, void *cuda_stream);

/* Tile-size autotuner.  For each tile size K = kmin..kmax (9 <= kmin <=
 * kmax <= 13; a tile is 2^K amplitudes staged in one block's shared memory),
 * runs sd_evolve(., dt, steps, order) once to build and compile its programs
 * and once timed with CUDA events, on a scratch state of 2^n amplitudes of
 * `dtype` that the call allocates and frees (caller states are untouched).
 * The fastest K is kept for this dtype and used by later calls of the
 * context (a tile size given to sd_plan overrides it; sd_plan clears it).
 * best_k (may be NULL) receives it; times_ms (may be NULL, kmax - kmin + 1
 * doubles) receives milliseconds per step, 0 for sizes not run.  Sizes the
 * scheduler cannot use are skipped.  On the on-chip path nothing is tuned
 * (best_k = 0).  Synchronous; SD_ENOMEM if the scratch state does not fit. */
sd_status sd_autotune(sd_ctx *ctx, sd_dtype dtype, double dt, int64_t steps, int order, int kmin,
                      int kmax, int *best_k, double *times_ms);

/* Shape autotuner: as sd_autotune, over tile sizes K = kmin..kmax and, for
 * states whose passes are compiled at run time, over the prefetch depth (one
 * buffer or the dtype's two-buffer form, see sd_plan_opts.prefetch) and, for
 * complex64, both
 * register layouts (plain and paired, see sd_plan_opts.layout); the fastest
 * shape is kept for this dtype until the next sd_plan (a tile size, layout
 * or prefetch depth given to sd_plan overrides the tuned one).  Synchronous;
 * scratch state and errors as for sd_autotune; *out may not be NULL. */
sd_status sd_autotune_shape(sd_ctx *ctx, sd_dtype dtype, double dt, int64_t steps, int order, int kmin,
                            int kmax, sd_tune_result *out);

/* Compiles, host only (no GPU, no CUDA driver needed: NVRTC only), the
 * kernels that sd_evolve(ctx, ., dtype, ., steps, order, .) would compile
 * at run time, into the on-disk kernel cache ($SD_JIT_CACHE, else
 * $XDG_CACHE_HOME/sd_jit or ~/.cache/sd_jit) that later sd_evolve calls on
 * a GPU read.  The kernels do not depend on dt.  *compiled (may be NULL)
 * receives the number of NVRTC programs compiled (0 when all were cached,
 * or when nothing is compiled at run time for this call).  SD_EINVAL if
 * NVRTC is unavailable. */
sd_status sd_precompile(sd_ctx *ctx, sd_dtype dtype, int64_t steps, int order, int64_t *compiled);

/* Number of tile-pass kernels sd_evolve(ctx, ., dtype, ., steps, order, .)
 * launches; each reads and writes the state once.  0 when the state stays
 * on chip (one launch then runs every step).  A call of several steps merges
 * up to 4 steps (first order) or cores (second order) into one pass schedule,
 * so this is not steps times sd_get_schedule's passes_per_step.  Host only. */
sd_status sd_count_passes(sd_ctx *ctx, sd_dtype dtype, int order, int64_t steps, int64_t *out);

/* Trotter evolution in place (Eq. trotter_simul_diag): `steps` steps of
 * size dt of order 1 (groups 1..G) or 2 (Strang: groups 1..G-1 at dt/2, G
 * at dt, G-1..1 at dt/2; the half steps of group 1 that meet between
 * consecutive steps of one call are merged).  d_state: 2^n amplitudes of
 * `dtype` in device memory, owned by the caller.  Phases are formed from
 * angles dt*c_j/(2 pi) reduced mod 1 in FP64 and summed exactly in Q0.64
 * fixed point. */
sd_status sd_evolve(sd_ctx *ctx, void *d_state, sd_dtype dtype, double dt, int64_t steps,
                    int order, void *cuda_stream);

/* As sd_evolve, and after every step writes <psi|O|psi> for the Pauli-sum
 * observable O = sum_k oc[k] P_(ox[k], oz[k]) into d_trace[step] (device
 * memory, `steps` doubles, caller-owned).  The host arrays ox, oz, oc are
 * copied in stream order before the call returns and may be reused at once;
 * a later call on the same stream with another observable does not disturb
 * this one. */
sd_status sd_evolve_observe(sd_ctx *ctx, void *d_state, sd_dtype dtype, double dt,
                            int64_t steps, int order, int64_t mo, const uint64_t *ox,
                            const uint64_t *oz, const double *oc, double *d_trace,
                            void *cuda_stream);

/* Baseline path (Eq. trotter_decomp without grouping, Sec. 4): one state pass
 * per term, psi <- (cos a - i sin a P_j) psi with a = c_j dt, terms in
 * group order (so the product equals sd_evolve's up to rounding). */
sd_status sd_evolve_pauli(sd_ctx *ctx, void *d_state, sd_dtype dtype, double dt,
                          int64_t steps, int order, void *cuda_stream);

/* <psi|O|psi> for O = sum_k oc[k] P_(ox[k], oz[k]) (host arrays, mo terms),
 * reduced in FP64, written to *out_host.  Synchronises the stream. */
sd_status sd_expect(sd_ctx *ctx, const void *d_state, sd_dtype dtype, int64_t mo,
                    const uint64_t *ox, const uint64_t *oz, const double *oc,
                    double *out_host, void *cuda_stream);

/* Value f = <psi_T|O|psi_T> and gradient df/dc_j (m doubles, input term
 * order) of the evolution sd_evolve(d_state0, dt, steps, order) by an
 * adjoint sweep that undoes each group exponential (no checkpoints).
 * d_state0 is not modified; two device work vectors of the state's size are
 * allocated by the library and kept for later calls.  Needs n >= 4 (the
 * per-term sums run over 16-amplitude register groups); smaller n gives
 * SD_EINVAL.  Synchronises the stream. */
sd_status sd_grad(sd_ctx *ctx, const void *d_state0, sd_dtype dtype, double dt,
                  int64_t steps, int order, int64_t mo, const uint64_t *ox,
                  const uint64_t *oz, const double *oc, double *value_out,
                  double *grad_out, void *cuda_stream);

/* Evolve `count` independent problems (each its own planned context and
 * device state; qubit counts may differ) with the same dt/steps/order.
 * Problems whose states fit one block's shared memory run in one launch
 * each; the others are grouped by tile size and advanced pass level by pass
 * level, one launch per level covering every problem of the group, with the
 * blocks of a launch shared among the problems in proportion to their
 * sizes.  Asynchronous on the stream; at most 65535 problems.  The first
 * call with given (ctxs, d_states, dtype, dt, steps, order) builds the
 * programs and the device descriptors of the batch synchronously; repeated
 * calls reuse them and only launch kernels, so such a call can be captured
 * into a CUDA graph.  Under stream capture a batch that is not prepared
 * gives SD_EINVAL.  The descriptors are dropped when a context of the batch
 * frees its programs (another dt, sd_set_coeffs, sd_plan, sd_destroy); the
 * library keeps those of the 8 most recent batches. */
sd_status sd_evolve_batch(sd_ctx *const *ctxs, void *const *d_states, int64_t count,
                          sd_dtype dtype, double dt, int64_t steps, int order,
                          void *cuda_stream);

/* Builds, without launching anything, the programs and device descriptors
 * that sd_evolve_batch with the same arguments uses (for example before
 * capturing that call into a CUDA graph).  Synchronous; errors as for
 * sd_evolve_batch. */
sd_status sd_prepare_batch(sd_ctx *const *ctxs, void *const *d_states, int64_t count,
                           sd_dtype dtype, double dt, int64_t steps, int order);

/* <psi|O|psi> like sd_expect, for callers that cannot allocate device
 * memory (a fixed budget owned by another allocator, or a loop that must not
 * pay cudaMalloc's implicit synchronisation).  The paper has no counterpart:
 * this is a service of the library.  No context is needed and nothing is
 * allocated: the scratch (per-block partial sums of one term, one result per
 * term) lives in a file-scope static device array of about 41 KB that every
 * GPU loading the library keeps until the process exits.  n qubits, state as
 * in sd_evolve; mo <= 4096 terms (more gives SD_EINVAL, with a message in
 * sd_last_error(NULL)); the observable arrays are host arrays; the value is
 * written to *out_host after the stream is synchronised.  Each term costs
 * one read of the state (sd_expect folds all Z-only terms into one read),
 * so for observables with many terms on large states it is slower than
 * sd_expect.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current.  All calls share the array, so calls that overlap on
 * the GPU (other streams or host threads) race and must be serialised by the
 * caller. */
sd_status sd_expect_noalloc(int n, const void *d_state, sd_dtype dtype, int64_t mo,
                            const uint64_t *ox, const uint64_t *oz, const double *oc,
                            double *out_host, void *cuda_stream);

/* Message for the last failing call on ctx (ctx may be NULL: last global error). */
const char *sd_last_error(const sd_ctx *ctx);

void sd_destroy(sd_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SD_H */
