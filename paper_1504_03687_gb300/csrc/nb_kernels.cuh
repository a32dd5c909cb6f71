// nb_kernels.cuh — host-side launchers of the library's kernels (internal; not part of the ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

struct nb_ctx;
struct nb_sched;

namespace nbgpu {

// ---- device-driven block steps ------------------------------------------------------------
// The parameters of one block step held in device memory, so that a batch of block steps can
// be enqueued with no host work in between: the step's begin kernel (ac.cu) writes them from
// the scheduler's device state, and every later kernel of the step reads them.  A nonzero
// halt turns every kernel of the step, and of every step queued after it, into a no-op.
struct StepParams {
    double t;          // block time
    int64_t t_ticks;   // block time in ticks of 2^-48
    int64_t n_act;     // active particles: the list prefix [0, n_act)
    float t_hi, t_lo;  // the block time as a double-single pair
    int32_t lstar;     // coarsest active level
    int32_t halt;      // 0 run; 1 end time passed; 2 a regular step is due; 3 prefix too long; 4 batch done
};
enum { STEP_RUN = 0, STEP_END = 1, STEP_REGULAR = 2, STEP_LONG = 3, STEP_BUDGET = 4 };

// The begin of a device-driven block step (Sec. 3.3.1's block-step selection), one warp;
// lane l holds the counts of levels l and l + 32 and T is the current time in ticks.  The
// next block time is T + 2^-Lmax, Lmax the finest level present; its active particles are
// the levels >= L* = 48 - ctz(T_new), the list prefix of their total count.  The run halts
// when no particle is left, the time passes t_end, the budget is spent, the prefix is longer
// than max_prefix, or halt_hist (the regular-level histogram) holds a particle at a level
// >= L* (a regular step is due: the host takes it).  Otherwise P receives the step and the
// budget words are advanced: [0] steps left, [1] steps taken, [2] active rows taken.
struct StepBegin {
    StepParams *P;
    const int32_t *halt_hist;  // [64]
    double t_end;
    int64_t *budget;
    int64_t max_prefix;
};

// The inputs of step_begin that do not change during a device-driven step, read ahead.
struct StepBeginIn {
    int32_t r_lo, r_hi;  // halt_hist[lane], halt_hist[lane + 32]
    int64_t left;        // budget[0]
};
__device__ __forceinline__ StepBeginIn step_begin_inputs(const StepBegin &B, int lane)
{
    return StepBeginIn{B.halt_hist[lane], B.halt_hist[lane + 32], B.budget[0]};
}

__device__ __forceinline__ void step_begin(const StepBegin &B, int64_t c_lo, int64_t c_hi, int64_t T, int lane,
                                           const StepBeginIn &in)
{
    constexpr int kTicks = 48;
    const int32_t r_lo = in.r_lo, r_hi = in.r_hi;
    const int64_t left = in.left;
    StepParams *P = B.P;
    if (left <= 0) {
        if (lane == 0) P->halt = STEP_BUDGET;
        return;
    }
    const unsigned m_hi = __ballot_sync(0xffffffffu, c_hi != 0), m_lo = __ballot_sync(0xffffffffu, c_lo != 0);
    const int lmax = m_hi ? 63 - __clz(m_hi) : (m_lo ? 31 - __clz(m_lo) : -1);
    if (lmax < 0) {
        if (lane == 0) P->halt = STEP_END;
        return;
    }
    const int64_t T_new = T + ((int64_t)1 << (kTicks - lmax));
    const double t = ldexp((double)T_new, -kTicks);
    if (t > B.t_end) {
        if (lane == 0) P->halt = STEP_END;
        return;
    }
    int lstar = kTicks - (__ffsll(T_new) - 1);
    if (lstar < 0) lstar = 0;
    int64_t na = (lane >= lstar ? c_lo : 0) + (lane + 32 >= lstar ? c_hi : 0);
    int64_t nr = (lane >= lstar ? r_lo : 0) + (lane + 32 >= lstar ? r_hi : 0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        na += __shfl_xor_sync(0xffffffffu, na, o);
        nr += __shfl_xor_sync(0xffffffffu, nr, o);
    }
    if (lane != 0) return;
    if (nr > 0 || na > B.max_prefix) {
        P->halt = nr > 0 ? STEP_REGULAR : STEP_LONG;
        return;
    }
    P->t = t;
    P->t_ticks = T_new;
    P->n_act = na;
    P->lstar = lstar;
    P->t_hi = (float)t;
    P->t_lo = (float)(t - (double)P->t_hi);
    B.budget[0] = left - 1;
    B.budget[1] += 1;
    B.budget[2] += na;
}

// The scheduler's state on the device for device-driven steps (sched.cu): the list, device
// copies of the per-level counts and of the current time, and the longest prefix one device
// re-sort takes (one CTA).
struct SchedDevice {
    int32_t *list;
    int64_t *count;  // [64]
    int64_t *T;
    int64_t max_prefix;
};
bool sched_device(::nb_sched *s, SchedDevice *out);  // allocates the device copies on first use
bool sched_push(::nb_sched *s);                      // host counts and time -> device (stream-ordered)
bool sched_pull(::nb_sched *s);                      // device -> host (synchronises the stream)

// Predicted j-records.
//  FP64 : 2 dvec4 per particle  {x, y, z, m}, {vx, vy, vz, 0}                   (64 B)
//  mixed: 3 float4 per particle {x_hi, y_hi, z_hi, m}, {x_lo, y_lo, z_lo, 0},
//                               {vx, vy, vz, 0}                                 (48 B)
// x_hi = x with its 29 low mantissa bits cleared (a float), x_lo = fl32(x - x_hi), so
// |x - (x_hi + x_lo)| <= 2^-48 |x|.  Records n .. n_pad-1 are padding: mass 0,
// position 1e18, so whole tiles can be read without a bounds check.
//
// Neighbour capture.  The j-range is cut into G ordered segments; for every (segment g,
// active row k) exactly one thread (tiled kernels) or one warp (j-streamed kernels) walks
// the segment in ascending j and appends hits to seg_slots[(g*n_i + k)*L ...] (at most L
// kept, all counted in seg_cnt[g*n_i + k]; the anchored kernels index both by the row's
// position r in their spatial order instead).  The CSR row k is then the concatenation of
// its segments in order, cut at nb_cap: ascending j, deterministic, no atomics, no sort.
// L = min(nb_cap, longest segment) suffices because a segment that holds more than L
// hits can only be reached when L = nb_cap.

struct ForceArgs {
    const void *rec;        // dvec4* (FP64) or float4* (mixed)
    int64_t n;              // particles
    int64_t j_lo, j_hi;     // source range [j_lo, j_hi); j_lo is a multiple of the record padding
    int64_t n_tiles;        // j-tiles of the launch's tile size covering the source range
    const int32_t *idx;     // active indices
    int64_t n_i;
    const int32_t *perm;    // anchored kernel: row order (the r-th row is row perm[r]); null = identity
    const double *rs2;      // (n_i) or scalar
    int32_t rs2_scalar;
    int32_t want_nb;        // 0: skip neighbour capture
    int32_t S;              // j-splits (blockIdx.y)
    int32_t L;              // neighbour slots per (segment, row); 0 = count only
    double *part;           // partial sums [S][7][n_i] at row k (the anchored kernels: at row-order position r)
    int32_t *seg_cnt;       // [G][n_i]
    int32_t *seg_slots;     // [G][n_i][L]
    unsigned *status;
};

// Batched ensemble: one work item = (cluster, up to rows-per-item consecutive active rows).
struct BatchItem {
    int32_t cluster, row0, rows, pad;
};

struct BatchArgs {
    const float4 *rec;
    const int64_t *cluster_off;  // [C+1] particle offsets of the concatenated clusters
    const double *rs2;           // [C] squared neighbour radius per cluster
    const int32_t *idx;          // [n_i] global active indices, rows grouped by cluster
    int64_t n_i;
    const BatchItem *items;
    int32_t n_items;
    int32_t want_nb;
    int32_t L;                   // neighbour slots per row (0: counts only)
    unsigned *queue;             // item counter, zero at launch
    double *part;                // [7][n_i]
    int32_t *seg_cnt;            // [n_i]
    int32_t *seg_slots;          // [n_i][L]
    unsigned *status;
};

struct Plan {
    int kernel;     // 0 FP64 tiled, 1 mixed tiled, 2 mixed j-streamed, 3 FP64 j-streamed
    int variant;    // kernel-specific template variant
    int i_per_cta;  // active particles per CTA
    int S;          // j-splits
    int64_t ctas;
    int tj;         // j-tile (tiled kernels) or 0
    int segs_per_split;   // neighbour segments per split (1 tiled, warps per CTA j-streamed)
    int64_t seg_len;      // longest neighbour segment (j's)
};

// Launch-shape planner (pure host function; no CUDA calls).
Plan plan_force(int precision, int num_sms, const int *ctas_per_sm, int64_t n, int64_t n_i, int nb_cap);
// Occupancy of each kernel variant (filled once per context).
void query_occupancy(int *ctas_per_sm /* [8] */);

void launch_predict(cudaStream_t st, int64_t n, int64_t n_pad, double t, const double *x,
                    const double *v, const double *a, const double *jk, const double *tl,
                    const double *m, double *xp, double *vp, void *rec64, void *rec32);
void launch_pack_predicted(cudaStream_t st, int64_t n, int64_t n_pad, const double *xp,
                           const double *vp, const double *m, void *rec64, void *rec32);

void launch_force(cudaStream_t st, const Plan &p, ForceArgs a);

// Spatial (Morton) order of an active block's rows for the anchored force kernel
// (roworder.cu): writes a permutation of [0, n_i) into scratch and returns the launches.
size_t roworder_scratch_bytes(int64_t n_i);
void roworder_configure();
int launch_row_order(cudaStream_t st, const void *rec, const int32_t *idx, int64_t n, int64_t n_i, void *scratch,
                     const int32_t **perm_out);

// The fixed-order sum of S partial-sum sets; position r of part holds row perm[r] (perm null:
// row r), as the anchored force kernel writes them.
void launch_reduce(cudaStream_t st, const double *part, int S, int64_t n_i, double *acc,
                   double *jerk, double *pot, const int32_t *perm = nullptr);

// Neighbour CSR from the segment lists: counts -> offsets -> ordered gather.
// Returns the number of kernels launched.
// row_total: (n_i) int32 scratch used when there are many segments per row or a perm (may be
// NULL when G is small and perm is NULL).  perm: the segments of position r belong to row
// perm[r] (the anchored force kernel's spatial order); NULL = row r.
int launch_neighbour_csr(cudaStream_t st, int64_t G, int64_t n_i, int L, int cap,
                         const int32_t *seg_cnt, const int32_t *seg_slots, int64_t *off,
                         int32_t *nb_idx, int64_t nb_capacity, int32_t *count_true,
                         int64_t *scan_tmp, int32_t *row_total, unsigned *status,
                         const int32_t *perm = nullptr);

size_t neighbour_scan_tmp_elems(int64_t n_i);

// Device state of a context, for the integrator inside the library (nb_api.cu).
struct CtxState {
    double *x, *v, *a, *jk, *tl, *m, *xp, *vp;
    void *rec;  // predicted j-records of the last nb_predict
    unsigned *status;
    cudaStream_t stream;
    int precision, cap, num_sms, device;
    int64_t n, n_pad;
};
bool ctx_state(::nb_ctx *c, CtxState *out);
void ctx_state_changed(::nb_ctx *c);  // the state arrays were rewritten in place

// Hermite predictor and corrector over caller arrays, and their VJPs (hermite.cu).
void launch_hermite_predict(cudaStream_t st, int64_t n, double t, const double *x, const double *v, const double *a,
                            const double *j, const double *tl, double *xp, double *vp);
void launch_hermite_predict_vjp(cudaStream_t st, int64_t n, double t, const double *tl, const double *gxp,
                                const double *gvp, double *gx, double *gv, double *ga, double *gj);
void launch_hermite_correct(cudaStream_t st, int64_t n, double t, const double *tl, const double *xp, const double *vp,
                            const double *a0, const double *j0, const double *a1, const double *j1, double *x1,
                            double *v1);
void launch_hermite_correct_vjp(cudaStream_t st, int64_t n, double t, const double *tl, const double *gx1,
                                const double *gv1, double *gxp, double *gvp, double *ga0, double *gj0, double *ga1,
                                double *gj1);

// Irregular force (irregular.cu).  Lists as CSR (off) or, with ell_stride > 0, per
// particle: particle i's list is nb[i * ell_stride .. + ell_cnt[i]).
void launch_irregular(cudaStream_t st, int precision, int num_sms, const void *srec, int predicted, int64_t n,
                      double t, int64_t n_i, const int32_t *idx, const int64_t *off, const int32_t *nb, double *acc,
                      double *jerk, double *pot, double *acc_reg, double *jerk_reg, double *pot_reg, unsigned *status,
                      const int32_t *ell_cnt = nullptr, int64_t ell_stride = 0, const StepParams *dyn = nullptr);
// State records of the predict-on-load form (pack_state_one layout) for particles 0..n-1.
size_t state_record_bytes(int precision, int64_t n);
void launch_pack_state(cudaStream_t st, int precision, int64_t n, const double *x, const double *v, const double *a,
                       const double *jk, const double *tl, const double *m, void *srec);

}  // namespace nbgpu
