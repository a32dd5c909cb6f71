/*
 * nbgpu.h — C ABI of the GB300 (sm_103a) regular-force library.
 *
 * The library computes the regular-force step of the NBODY6++GPU method
 * (Wang et al. 2015, MNRAS 450, 4070): every particle of an active block gets
 * its acceleration, the time derivative of the acceleration (jerk) and its
 * potential from all N predicted particles, plus the list of its neighbours
 * inside the radius r_s (Sec. 2, Ahmad-Cohen neighbour scheme; Sec. 3.2.1,
 * regular force, potential and neighbour list on the GPU; Table 2, O(N_i N)
 * work per regular step).  All particles are first predicted to the block time
 * (Sec. 3.3.3; the fourth-order Hermite predictor of Sec. 2).
 *
 * Conventions shared by every entry point
 *  - Units are whatever the caller uses with G = 1 (the paper uses N-body units).
 *  - Vectors are row-major (n, 3) arrays of double; scalars per particle are (n).
 *  - The caller owns every buffer it passes; the library owns only the
 *    context's internal device state and scratch.
 *  - `on_device` = 1: every array argument of that call is a device pointer and
 *    the call is asynchronous on the context stream (results are valid after
 *    nb_sync or any later stream-ordered operation).  `on_device` = 0: every
 *    array argument is a host pointer; the call copies in, computes, copies out
 *    and returns after the results are in host memory.
 *  - Errors never abort the process.  Every function returns an nb_status;
 *    nb_last_error() gives a one-line description of the last failure.  After a
 *    CUDA error the context is unusable (NB_ERR_STATE) and should be freed.
 *  - A context is not thread-safe: use one per host thread / stream.
 *  - Sums over j run over all j != i.  The sum over particles outside r_s only
 *    (the Ahmad-Cohen regular force proper) is this result minus the sum over the
 *    neighbour list, which the caller forms.  No softening is applied; two
 *    distinct particles at the same position give inf/NaN.
 */
#ifndef NBGPU_H
#define NBGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nb_ctx nb_ctx; /* opaque */

typedef enum {
    NB_OK = 0,
    NB_ERR_ARG = 1,          /* invalid argument (null pointer, size, index out of range) */
    NB_ERR_STATE = 2,        /* call order violated, or context broken by an earlier CUDA error */
    NB_ERR_OOM = 3,          /* device allocation failed */
    NB_ERR_CUDA = 4,         /* a CUDA runtime call failed */
    NB_ERR_NB_OVERFLOW = 5,  /* warning: results valid, some neighbour lists were cut at nb_cap
                                or the CSR output capacity was too small */
    NB_ERR_TIMEOUT = 6,      /* a bounded device-side wait expired */
    NB_ERR_DEVICE = 7        /* a device-side consistency check failed */
} nb_status;

typedef enum {
    NB_FP64 = 0,  /* every step in FP64 */
    NB_MIXED = 1  /* FP64 predictor; pairwise arithmetic in FP32 on double-single
                     coordinate differences; per-tile sums promoted to FP64 */
} nb_precision;

typedef struct {
    int64_t n_max;      /* largest particle count the context will hold (>= 1) */
    int32_t precision;  /* nb_precision */
    int32_t nb_cap;     /* neighbours stored per active particle (>= 1); the true count is
                           always reported */
    int32_t device;     /* CUDA device ordinal */
    int32_t flags;      /* reserved, must be 0 */
    void *stream;       /* cudaStream_t to run on; NULL = a stream the context creates */
} nb_config;

/* Library version as 10000*major + 100*minor + patch. */
int32_t nb_version(void);

/* Create a context on cfg->device.  *out receives the handle (NULL on failure). */
nb_status nb_init(nb_ctx **out, const nb_config *cfg);

/* Destroy a context and free its device memory.  Safe on NULL. */
nb_status nb_free(nb_ctx *ctx);

/* Run subsequent calls on `stream` (a cudaStream_t; NULL = CUDA's default stream). */
nb_status nb_set_stream(nb_ctx *ctx, void *stream);

/* Load the Hermite state of n particles (1 <= n <= n_max): positions x, velocities
 * v, acceleration a and jerk at each particle's last step time t_last, and masses m
 * — the inputs of the predictor.  Arrays are copied; the caller keeps ownership. */
nb_status nb_set_particles(nb_ctx *ctx, int64_t n, const double *x, const double *v,
                           const double *a, const double *jerk, const double *m,
                           const double *t_last, int32_t on_device);

/* Predict all n particles to time t (Sec. 3.3.3):
 *   dt = t - t_last;  x_p = x + v dt + a dt^2/2 + jerk dt^3/6;  v_p = v + a dt + jerk dt^2/2,
 * in FP64, and build the j-records the force kernels read. */
nb_status nb_predict(nb_ctx *ctx, double t);

/* Load an already predicted state (x_p, v_p, m) of n particles directly, in place
 * of nb_set_particles + nb_predict (used by the autograd binding and the chained
 * integrator, whose predictor runs outside the library). */
nb_status nb_set_predicted(nb_ctx *ctx, int64_t n, const double *xp, const double *vp,
                           const double *m, int32_t on_device);

/* Copy the predicted positions and velocities (n,3) out of the context. */
nb_status nb_get_predicted(nb_ctx *ctx, double *xp, double *vp, int32_t on_device);

/* Copy the j-records of the n predicted particles, the data the force kernels stream (built
 * by nb_predict or nb_set_predicted; Sec. 3.2.1: the j-particles' predicted positions,
 * velocities and masses), into out:
 *   mixed: 12 floats per particle, {x_hi, y_hi, z_hi, m} {x_lo, y_lo, z_lo, 0} {vx, vy, vz, 0},
 *          where hi is the FP64 position with its 29 low mantissa bits cleared (exactly a
 *          float), lo = x - hi rounded to FP32, and v and m are rounded to FP32 (to nearest);
 *   fp64:  8 doubles per particle, {x, y, z, m} {vx, vy, vz, 0}.
 * out holds n * 48 bytes (mixed) or n * 64 bytes (fp64), host or device memory as on_device
 * says; the caller owns it.  NB_ERR_STATE before any predicted state exists. */
nb_status nb_get_records(nb_ctx *ctx, void *out, int32_t on_device);

/* Regular force step for the active block idx[0..n_i) (Sec. 2, Sec. 3.2.1):
 *   acc_k  = sum_{j != i} m_j r / |r|^3
 *   jerk_k = sum_{j != i} m_j [ w / |r|^3 - 3 (r.w) r / |r|^5 ]
 *   pot_k  = - sum_{j != i} m_j / |r|
 * with i = idx[k], r = x_p,j - x_p,i, w = v_p,j - v_p,i, over all n predicted particles
 * (or over the source range set by nb_set_source_range).
 * Neighbours: j != i with |r|^2 < rs2 (rs2[k], or rs2[0] for all when rs2_scalar != 0).
 *
 * idx:           (n_i) int32, unique, each in [0, n); output row k is for idx[k].
 * acc, jerk:     (n_i, 3) double, overwritten.   pot: (n_i) double, overwritten.
 * nb_off:        (n_i + 1) int64 CSR offsets, overwritten (may be NULL with nb_idx NULL).
 * nb_idx:        (nb_idx_capacity) int32: the neighbours of row k, ascending j, are
 *                nb_idx[nb_off[k] .. nb_off[k+1]); each list holds at most nb_cap entries
 *                (the smallest j's).  If the lists need more than nb_idx_capacity entries
 *                in total, the CSR is cut there and NB_ERR_NB_OVERFLOW is reported.
 *                With nb_idx NULL only the counts (and nb_off, if given) are produced, and
 *                nothing is reported about a capacity.
 * nb_count_true: (n_i) int32, the untruncated neighbour count of each row (may be NULL).
 * n_i = 0 is allowed (only nb_off[0] = 0 is written).
 * Status: NB_ERR_NB_OVERFLOW (a warning, results valid) is returned by this call when
 * on_device = 0, and by the next nb_sync when on_device = 1. */
nb_status nb_regular_force(nb_ctx *ctx, int64_t n_i, const int32_t *idx, const double *rs2,
                           int32_t rs2_scalar, double *acc, double *jerk, double *pot,
                           int64_t *nb_off, int32_t *nb_idx, int64_t nb_idx_capacity,
                           int32_t *nb_count_true, int32_t on_device);

/* Restrict the source particles of subsequent nb_regular_force calls to j in [j_lo, j_hi):
 * the split of the particle set between the GPUs of one node (Sec. 3.4: every GPU holds a
 * similar share of the particles for the regular force, and together they cover the whole
 * set).  The active particles idx may be anywhere in [0, n).  The call then returns the
 * sums over the range only, the neighbours found in the range (global indices, ascending
 * j, at most nb_cap per row) and the range's true counts.  Adding the sums of disjoint
 * ranges that cover [0, n), concatenating the lists in range order (each cut at nb_cap)
 * and adding the counts gives the unrestricted result; the sums agree with it up to the
 * order of the FP64 additions.
 * j_lo must be a multiple of NB_SOURCE_ALIGN and 0 <= j_lo < j_hi <= n_max; at call time
 * j_hi must not exceed the loaded particle count n and must be a multiple of
 * NB_SOURCE_ALIGN unless it equals n (else that call returns NB_ERR_STATE).
 * (0, 0) restores the full set.  nb_regular_force_backward returns NB_ERR_STATE while a
 * range is set; the batched form ignores it. */
#define NB_SOURCE_ALIGN 256
nb_status nb_set_source_range(nb_ctx *ctx, int64_t j_lo, int64_t j_hi);

/* Vector-Jacobian product of nb_regular_force's (acc, jerk, pot) w.r.t. the predicted
 * positions, velocities and masses of all n particles (no counterpart in the paper;
 * obtained by differentiating the sums above).  For
 *   L = sum_k g_acc[k].acc_k + g_jerk[k].jerk_k + g_pot[k] pot_k
 * it writes g_x = dL/dx_p, g_v = dL/dv_p (n,3) and g_m = dL/dm (n), overwriting them.
 * Uses the state of the last nb_predict / nb_set_predicted.  idx: (n_i) int32, unique, each
 * in [0, n); g_acc, g_jerk (n_i,3) and g_pot (n_i) are the cotangents of row k = idx[k].  An
 * index outside [0, n) or named twice makes the call fail with NB_ERR_ARG (returned by this
 * call when on_device = 0, by the next nb_sync when on_device = 1), its outputs unspecified;
 * with unique indices every sum has a fixed order and runs are bitwise reproducible. */
nb_status nb_regular_force_backward(nb_ctx *ctx, int64_t n_i, const int32_t *idx,
                                    const double *g_acc, const double *g_jerk,
                                    const double *g_pot, double *g_x, double *g_v, double *g_m,
                                    int32_t on_device);

/* Batched ensemble form (many independent clusters, one launch; a mixed-precision context).
 * The particles of all clusters are loaded as one state (nb_set_particles + nb_predict, or
 * nb_set_predicted) in cluster order: cluster c owns particles cluster_off[c] ..
 * cluster_off[c+1]-1 and the active rows active_off[c] .. active_off[c+1]-1; each cluster
 * only feels its own particles.
 * nb_batch_plan (host arrays of n_clusters+1 entries, both starting at 0) builds the work
 * items — (cluster, a tile of up to 128/256/512 active rows), sorted by cost, largest first —
 * uploads them, and grows every scratch buffer the launch needs; `variant` selects the tile
 * (0: 512 rows, 1: 256, 2: 128; -1: the largest tile that still gives 8 items per SM).
 * nb_regular_force_batched then runs one persistent kernel that pops the items from a device
 * counter, plus the reduction and the neighbour CSR: it allocates nothing and synchronises
 * nothing (device pointers only; deferred status via nb_sync).  Arguments as for
 * nb_regular_force over the concatenated active list idx (global particle indices, every
 * one inside its own cluster, rows grouped by cluster), with rs2[c] the squared neighbour
 * radius of cluster c.  No counterpart in the paper (a batching service for many small
 * independent integrations). */
nb_status nb_batch_plan(nb_ctx *ctx, int64_t n_clusters, const int64_t *cluster_off,
                        const int64_t *active_off, int32_t variant);
nb_status nb_regular_force_batched(nb_ctx *ctx, const int32_t *idx, const double *rs2, double *acc,
                                   double *jerk, double *pot, int64_t *nb_off, int32_t *nb_idx,
                                   int64_t nb_idx_capacity, int32_t *nb_count_true);

/* Irregular force of the Ahmad-Cohen scheme (Sec. 2; Sec. 3.2.2): for the active rows
 * idx[0..n_i), the sums of nb_regular_force restricted to each row's neighbour list,
 *   acc_k = sum_{j in L_k, j != i} m_j r/|r|^3   (jerk and pot likewise),
 * with L_k = nb_idx[nb_off[k] .. nb_off[k+1]) (any CSR list of particle indices; typically
 * the one nb_regular_force returned).  The particles are predicted from the Hermite state
 * of nb_set_particles to time t: only i and its listed neighbours while N_i is below n/128
 * (FP64 context) or n/8 (mixed) (neighbour-only prediction, Sec. 3.3.3), else all particles
 * once (the cheaper choice once the lists name many more particles than there are, as
 * Sec. 3.3.3 notes).  The predictor is
 * nb_predict's, so in an FP64 context both forms give bit-identical results.  The pair
 * arithmetic follows the context precision (FP64, or mixed: double-single position
 * differences, FP32 pair terms, FP64 row sums; the neighbour-only form adds the Taylor
 * increments in FP32).
 * acc, jerk: (n_i, 3), pot: (n_i) double, overwritten.
 * acc_reg, jerk_reg, pot_reg: all NULL, or all given; then on input the all-j sums of the
 * same rows at the same time (from nb_regular_force) and on output the part from outside
 * the lists (input minus the irregular sums): the regular force of the scheme.
 * Requires nb_set_particles (NB_ERR_STATE after nb_set_predicted alone).  Host mode
 * validates every index and offset (NB_ERR_ARG); device mode flags a bad one in the
 * deferred status and writes zeros for that row. */
nb_status nb_irregular_force(nb_ctx *ctx, double t, int64_t n_i, const int32_t *idx,
                             const int64_t *nb_off, const int32_t *nb_idx, double *acc,
                             double *jerk, double *pot, double *acc_reg, double *jerk_reg,
                             double *pot_reg, int32_t on_device);

/* Per-phase device timing: with timing enabled, every phase of every later call is
 * bracketed by CUDA events on the context stream.  nb_get_timings synchronises the
 * stream and returns, per phase, the summed device time in ms and the number of kernels
 * launched since the previous nb_get_timings (launch counts are kept even with timing
 * off), then resets both.  Phases: 0 predict (and the array predictor and corrector),
 * 1 force, 2 partial reduction, 3 neighbour CSR, 4 backward (and the predictor's and the
 * corrector's VJPs), 5 irregular force, 6 row order (the spatial order of the active rows
 * that the anchored force kernel takes).  ms and launches have NB_PHASES
 * entries each. */
#define NB_PHASES 7
nb_status nb_set_timing(nb_ctx *ctx, int32_t enable);
nb_status nb_get_timings(nb_ctx *ctx, double *ms, int64_t *launches);

/* Wait for all work queued on the context stream and return the first deferred
 * status (NB_OK, NB_ERR_NB_OVERFLOW, NB_ERR_TIMEOUT, NB_ERR_DEVICE or a CUDA error)
 * raised since the previous nb_sync; the deferred status is then cleared. */
nb_status nb_sync(nb_ctx *ctx);

/* Fault injection for testing error handling (no counterpart in the paper).  Arms a
 * simulated runtime failure on the host: after `after` more operations of `kind`, the next
 * one reports the error the CUDA runtime would, and the GPU is never touched:
 *   NB_FAULT_ALLOC  a device allocation of the context's scratch -> NB_ERR_OOM; the context
 *                   stays usable (the call can be retried);
 *   NB_FAULT_SYNC   a stream synchronisation -> NB_ERR_CUDA, as after a failed kernel; the
 *                   context becomes unusable (NB_ERR_STATE from then on; nb_free it);
 *   NB_FAULT_STATUS the read of the deferred device status -> NB_ERR_CUDA, likewise.
 * kind 0 disarms.  The environment variable NB_FAULT = "alloc:N", "sync:N" or "status:N"
 * arms the same at nb_init. */
#define NB_FAULT_ALLOC 1
#define NB_FAULT_SYNC 2
#define NB_FAULT_STATUS 3
nb_status nb_inject_fault(nb_ctx *ctx, int32_t kind, int32_t after);

/* One-line description of the last error on this context (never NULL). */
const char *nb_last_error(const nb_ctx *ctx);

/* ---------------------------------------------------------------------------------------
 * The Hermite predictor and corrector over caller arrays, and their vector-Jacobian
 * products: the O(N) steps of a block-step integration that a differentiable chain of block
 * steps (predictor -> nb_regular_force -> corrector) runs between force calls, and runs
 * backwards for its gradient (Sec. 2: the fourth-order Hermite scheme after Makino 1991;
 * Sec. 3.3.3: prediction).  All arrays are device arrays, (n,3) row-major for vectors and (n)
 * for t_last; the calls are asynchronous on the context stream and read no context state.
 * Outputs are overwritten (and must not alias inputs).  NB_ERR_ARG for n < 0 or a null array
 * (n = 0 does nothing).  t and t_last are not differentiated.
 * --------------------------------------------------------------------------------------- */

/* Predict to time t: dt_k = t - t_last[k], xp = x + dt (v + dt/2 (a + dt/3 jerk)),
 * vp = v + dt (a + dt/2 jerk), in the same operation order as nb_predict (bit-identical). */
nb_status nb_hermite_predict(nb_ctx *ctx, int64_t n, double t, const double *x, const double *v,
                             const double *a, const double *jerk, const double *t_last, double *xp,
                             double *vp);

/* VJP of nb_hermite_predict: g_x = g_xp, g_v = dt g_xp + g_vp, g_a = dt^2/2 g_xp + dt g_vp,
 * g_jerk = dt^3/6 g_xp + dt^2/2 g_vp. */
nb_status nb_hermite_predict_backward(nb_ctx *ctx, int64_t n, double t, const double *t_last,
                                      const double *g_xp, const double *g_vp, double *g_x, double *g_v,
                                      double *g_a, double *g_jerk);

/* Fourth-order Hermite corrector of n rows stepping from t_last[k] to t (h = t - t_last[k] > 0):
 * a2 = (-6 (a0 - a1) - h (4 j0 + 2 j1)) / h^2, a3 = (12 (a0 - a1) + 6 h (j0 + j1)) / h^3,
 * x1 = xp + h^4/24 a2 + h^5/120 a3, v1 = vp + h^3/6 a2 + h^4/24 a3, with xp, vp the predicted
 * state, a0, j0 the force and jerk at t_last and a1, j1 at t (the operation order of that
 * definition, without FMA contraction: the same arithmetic as the device integrator). */
nb_status nb_hermite_correct(nb_ctx *ctx, int64_t n, double t, const double *t_last, const double *xp,
                             const double *vp, const double *a0, const double *j0, const double *a1,
                             const double *j1, double *x1, double *v1);

/* VJP of nb_hermite_correct (the corrector is linear in its inputs): g_xp = g_x1, g_vp = g_v1,
 * g_a0 = -3h^2/20 g_x1 - h/2 g_v1, g_j0 = -7h^3/60 g_x1 - 5h^2/12 g_v1, g_a1 = -g_a0,
 * g_j1 = -h^3/30 g_x1 - h^2/12 g_v1. */
nb_status nb_hermite_correct_backward(nb_ctx *ctx, int64_t n, double t, const double *t_last,
                                      const double *g_x1, const double *g_v1, double *g_xp, double *g_vp,
                                      double *g_a0, double *g_j0, double *g_a1, double *g_j1);

/* Spatial order of an active block's rows: the permutation that the anchored mixed force
 * kernel (plan variants 10-19) takes before it runs, and that a caller may use to lay out its
 * own blocks (no counterpart in the paper; a locality device of this GPU design).  The rows
 * idx (n_i, device int32) are ordered along the Morton (Z) curve of their predicted positions,
 * quantised to 8 bits per coordinate over the block's bounding box (the hi parts of the mixed
 * j-records of the last nb_predict / nb_set_predicted); ties keep row order (a stable sort), so
 * the order is deterministic.  Writes perm (n_i, device int32): perm[r] is the row taken r-th.
 * Rows whose index is outside [0, n) come last.  Asynchronous on the context stream.
 * NB_ERR_STATE for an FP64 context or before a prediction; NB_ERR_ARG for n_i < 0 or null
 * arrays (n_i = 0 does nothing). */
nb_status nb_row_order(nb_ctx *ctx, int64_t n_i, const int32_t *idx, int32_t *perm);

/* Describe the launch plan nb_regular_force would use (host-only, no GPU work):
 * out[0] = kernel id (0 = FP64 tiled, 1 = mixed tiled, 2 = mixed j-streamed,
 * 3 = FP64 j-streamed), out[1] = i-particles per CTA, out[2] = j-splits, out[3] = CTAs,
 * out[4] = j-tile (0 for the j-streamed kernels), out[5] = kernel variant. */
nb_status nb_plan(const nb_ctx *ctx, int64_t n, int64_t n_i, int64_t *out);

/* Force the launch plan of later nb_regular_force calls on this context (used to tune and
 * benchmark individual kernel variants): kernel and variant as reported by nb_plan (mixed
 * tiled kernel variants: 0-3 scalar double-single, 4-9 packed FP32x2 double-single, 10-14
 * packed with anchor-relative separations over the spatial row order, 15-19 the same with the
 * neighbour hits staged in shared memory and written as whole 32- or 64-byte groups; mixed
 * j-streamed variants: 0 one row a CTA, 1-3 four, eight and two rows a CTA as FP32x2 pairs),
 * `splits` j-splits (clipped to the tile count; 0 with the mixed tiled kernel = the
 * planner's split count for that variant).  kernel < 0 restores automatic planning.
 * NB_ERR_ARG if the kernel does not match the context's precision. */
nb_status nb_set_plan_override(nb_ctx *ctx, int32_t kernel, int32_t variant, int32_t splits);

/* Install tuned plans (from the project's autotuner): entry q applies to active blocks with
 * n_i <= ni_max[q] not covered by an earlier entry (ni_max strictly increasing); kernel,
 * variant and splits as for nb_set_plan_override.  Blocks beyond the last entry use the
 * automatic plan; an override, while set, takes precedence.  n_entries = 0 clears it. */
nb_status nb_set_plan_table(nb_ctx *ctx, int32_t n_entries, const int64_t *ni_max,
                            const int32_t *kernel, const int32_t *variant, const int32_t *splits);

/* The automatic plan for a given device shape, without a context or a GPU (host-only):
 * num_sms SMs, ctas_per_sm[0..20] resident CTAs of the twenty mixed tiled variants and the
 * FP64 tiled kernel (NULL = 1 each), and the context's nb_cap. */
nb_status nb_plan_for(int32_t precision, int32_t num_sms, const int32_t *ctas_per_sm, int64_t n,
                      int64_t n_i, int32_t nb_cap, int64_t *out);

/* Regular force, jerk and potential of a small active block without allocating any device
 * memory (the paper has no counterpart: this is a service for callers that cannot allocate
 * device memory while they integrate, such as a host code whose memory manager owns the
 * whole device, or a time-step loop that must never reach cudaMalloc/cudaFree because they
 * can synchronise the device).  No context is needed.
 *
 * Computes, in FP64, the same sums as nb_regular_force (no neighbour lists):
 *   acc_k, jerk_k, pot_k over all j != idx[k], from the caller's predicted state.
 * n:          particles, 1 <= n <= 2^31-1.
 * xp, vp:     (n,3) device arrays of predicted positions and velocities; m: (n) masses.
 * idx:        (n_i) int32 device array, 0 <= n_i <= 65536; an entry outside [0, n) gives a
 *             zero row.
 * acc, jerk:  (n_i,3) device outputs; pot: (n_i) device output (overwritten).
 * stream:     cudaStream_t to run on (NULL = CUDA's default stream); the call is
 *             asynchronous on it and runs on the current device.
 * err:        optional host buffer of err_len bytes for a one-line error message.
 * Scratch: the per-split partial sums live in a fixed 4 MiB device array inside the
 * library (every GPU that loads the library holds it until the process exits).  n_i above
 * 65536 is rejected with NB_ERR_ARG.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  A lookup that fails returns NB_ERR_CUDA and is tried again by the
 * next call; once it has succeeded the address is kept.  A CUDA error already pending on
 * the calling thread (left by earlier, unrelated work) makes the call return NB_ERR_CUDA
 * without running anything and without clearing that error.  All calls share the one array: calls that overlap on the GPU (on
 * different streams, or from different host threads without ordering) race and corrupt
 * each other's results.  Every scratch element a call reads is written earlier in the same
 * call, so no clearing is needed between calls. */
nb_status nb_regular_force_noalloc(int64_t n, const double *xp, const double *vp, const double *m,
                                   int64_t n_i, const int32_t *idx, double *acc, double *jerk,
                                   double *pot, void *stream, char *err, int32_t err_len);

/* ---------------------------------------------------------------------------------------
 * Block-step scheduler: the time-step sorting list of Sec. 3.3.1.
 *
 * Particle i has a level L_i (step 2^-L_i, Sec. 2: steps are integer powers of 1/2) and is
 * advanced at every multiple of its step; all particles start at time 0.  The scheduler
 * keeps the device list of all particle indices sorted by step, smallest first (level
 * descending), and the number of particles per level (the boundary offsets of the list).
 * nb_sched_next moves to the next block time, T + (smallest step), and reports the active
 * particles: all those whose step divides the new time, which are the first n_active
 * entries of the list.  nb_sched_update then takes the levels the integrator requests for
 * them and applies the block rule: a request is clamped to [level_min, level_max], a larger
 * step than twice the current one is cut to one doubling, and a doubling is granted only
 * when the block time is a multiple of the doubled step (else the level stays).  Only the
 * first n_active entries are re-sorted (O(N_i), stable: ties keep their list order), so the
 * result is deterministic.  Times are exact multiples of 2^-48.
 * --------------------------------------------------------------------------------------- */
typedef struct nb_sched nb_sched;

/* Create a scheduler for n particles with initial levels (n) int32 in [level_min,
 * level_max], 0 <= level_min <= level_max <= 48, on `device`, running on `stream` (a
 * cudaStream_t; NULL = a stream the scheduler creates).  Levels are read from host memory,
 * or device memory when on_device != 0.  NB_ERR_ARG on a level outside the range. */
nb_status nb_sched_init(nb_sched **out, int64_t n, const int32_t *levels, int32_t level_min,
                        int32_t level_max, int32_t device, void *stream, int32_t on_device);

/* Destroy a scheduler.  Safe on NULL. */
nb_status nb_sched_free(nb_sched *s);

/* Advance to the next block time (host only, O(levels)): *t_block receives the time, and
 * *n_active the number of active particles, which are (*d_list)[0 .. n_active) — *d_list is
 * the device list (n int32 entries), valid until the next nb_sched_update, and may serve
 * directly as the idx of nb_regular_force.  NB_ERR_STATE if the previous block step has
 * not been committed with nb_sched_update. */
nb_status nb_sched_next(nb_sched *s, double *t_block, int64_t *n_active, const int32_t **d_list);

/* Commit the block step: want (n_active) int32, in list order, holds the requested levels;
 * granted (n_active, optional) receives the levels granted by the block rule, in the same
 * order.  Host pointers when on_device = 0, else device pointers.  Re-sorts the active
 * part of the list; synchronises the scheduler's stream (the level counts come back). */
nb_status nb_sched_update(nb_sched *s, const int32_t *want, int32_t *granted, int32_t on_device);

/* Copy out the whole list and/or the level of every particle (n int32 each; either may
 * be NULL) and the time of the last committed block step.  Synchronises. */
nb_status nb_sched_get(nb_sched *s, int32_t *list, int32_t *levels, double *t_now, int32_t on_device);

/* Particles per level, counts[64] (index = level), as of the last committed step. */
nb_status nb_sched_counts(const nb_sched *s, int64_t *counts);

/* Set the time of the last committed block step (a scheduler created from the levels of a
 * run resumed at time t; every particle's last step time must be the latest multiple of
 * its step not above t).  t must be a multiple of 2^-48 and of the smallest step present;
 * only between block steps. */
nb_status nb_sched_set_time(nb_sched *s, double t);

/* Time of the next block step, without advancing (host only). */
nb_status nb_sched_peek(const nb_sched *s, double *t_next);

/* One-line description of the last error of this scheduler (never NULL). */
const char *nb_sched_last_error(const nb_sched *s);

/* ---------------------------------------------------------------------------------------
 * Ahmad-Cohen Hermite integrator on the device (Sec. 2: the force on a particle is split
 * into the irregular part from its neighbours inside r_s, recomputed at every irregular
 * step, and the regular part from all other particles, recomputed at the longer regular
 * steps and extrapolated with its derivatives in between; NBODY6++ adjusts r_s towards a
 * target neighbour number, App. A).  The paper prints no formulas; the scheme, step for
 * step:
 *  - block step: the scheduler above selects the particles whose irregular step ends at
 *    the new block time t; when some of them also end a regular step, all particles are
 *    predicted to t (nb_predict), otherwise only the active particles and their neighbours,
 *    on load (the neighbour-only prediction of Sec. 3.3.3);
 *  - every active particle gets the irregular force over its current list; one whose
 *    regular step also ends at t gets the all-j sums (nb_regular_force, which also yields
 *    its new list) and the irregular force over the new list;
 *  - new total force: all-j sums on a regular step, else list sums plus the regular force
 *    extrapolated to third order from its last regular step;
 *  - fourth-order Hermite corrector on the total force; irregular step from the Aarseth
 *    criterion on the total force (eta_irr); on a regular step, the regular force's second
 *    and third derivatives from the Hermite interpolation of the regular force with the
 *    old list, the regular step from the criterion on it (eta_reg), the new regular force
 *    and jerk (all-j minus new-list sums), and r_s^2 scaled by (nb_opt / N_b)^(2/3) clamped
 *    to [1/2, 2] (nb_opt <= 0 keeps r_s);
 *  - steps are powers of 1/2, halved as needed, doubled at most once and only at a time
 *    that is a multiple of the doubled step, never above dt_max; irregular <= regular: on a
 *    regular step the regular step is raised to the new irregular step if shorter, on an
 *    irregular step the irregular step is capped at the regular one.
 * Start: all forces and lists at t = 0, zero higher regular derivatives, steps from
 * eta_s |F| / |dF/dt| of the total and of the regular force (the regular one raised to the
 * irregular one if shorter).
 * The context provides the particle state, precision and list capacity (its nb_cap). */
typedef struct {
    double eta_irr, eta_reg, eta_s;  /* accuracy parameters of the step criteria */
    double dt_max;                   /* largest step: a power of 1/2 */
    int32_t nb_opt;                  /* target neighbour number (<= 0: r_s stays fixed) */
    int32_t level_max;               /* smallest step 2^-level_max, level_max <= 48 */
} nb_ac_params;
typedef struct nb_ac nb_ac;

/* Start an integration of n particles (masses m, positions x, velocities v (n,3) at t = 0,
 * squared neighbour radii rs2 (n); host or device pointers) on the context ctx (n <= its
 * n_max; the context's particle state is taken over and evolved in place by the integrator:
 * load no other state into the context while the integrator lives). */
nb_status nb_ac_init(nb_ac **out, nb_ctx *ctx, int64_t n, const double *m, const double *x, const double *v,
                     const double *rs2, const nb_ac_params *params, int32_t on_device);

/* One block step.  *t_block, *n_active, *n_regular (any may be NULL) receive the block
 * time, the particles stepped and those among them that took a regular step. */
nb_status nb_ac_step(nb_ac *s, double *t_block, int64_t *n_active, int64_t *n_regular);

/* Block steps until the next one would pass t_end, or max_blocks steps (0: no limit;
 * NB_ERR_STATE when reached).  Runs of block steps without a regular subset are driven from
 * the device: one kernel per step (irregular force, corrector, re-sort of the time-step list
 * and the next step's selection), enqueued in batches with one host synchronisation per
 * batch; a step with a regular subset, or with more than 4096 active particles, is taken by
 * the host path of nb_ac_step.  Both give the same bits.  stats (6 doubles, optional): block
 * steps, irregular particle steps, regular particle steps, neighbour-list pair terms, all-j
 * pair terms, block steps driven from the device. */
nb_status nb_ac_run(nb_ac *s, double t_end, int64_t max_blocks, double *stats);

/* Copy out (each may be NULL; n entries, x and v (n,3), lists n x nb_cap): positions and
 * velocities at each particle's last step time t, irregular and regular steps dt and DT,
 * the last regular step time T, r_s^2, list lengths and lists (ascending j). */
nb_status nb_ac_get(nb_ac *s, double *x, double *v, double *t, double *dt, double *DT, double *T,
                    double *rs2, int32_t *nb_count, int32_t *nb_lists, int32_t on_device);

/* Checkpoint / resume.  nb_ac_snapshot_bytes gives the size of a snapshot; nb_ac_save
 * writes the integrator's complete state between block steps (particles, regular-force
 * history, steps, lists, r_s^2, time, counters) into the host buffer buf; nb_ac_restore
 * creates an integrator on ctx (same precision and nb_cap as the saved one, n <= its n_max)
 * from such a buffer.  The kernels give every particle the same result whatever the order
 * of the active rows, so a resumed run continues bit for bit as the uninterrupted one. */
nb_status nb_ac_snapshot_bytes(nb_ac *s, size_t *bytes);
nb_status nb_ac_save(nb_ac *s, void *buf, size_t bytes);
nb_status nb_ac_restore(nb_ac **out, nb_ctx *ctx, const void *buf, size_t bytes);

/* Destroy the integrator (the context stays valid).  Safe on NULL. */
nb_status nb_ac_free(nb_ac *s);

/* One-line description of the last error of this integrator (never NULL). */
const char *nb_ac_last_error(const nb_ac *s);

#ifdef __cplusplus
}
#endif
#endif /* NBGPU_H */
