// nb_kernels.cuh — host-side launchers of the library's kernels (internal; not part of the ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "nb_force.cuh"  // the regular-force kernels' arguments and record layouts
#include "nb_step.cuh"   // device-driven block steps: StepParams, step_begin, the scheduler's device state

struct nb_ctx;
struct nb_sched;

namespace nbgpu {

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

// Reduction and neighbour CSR of a tiny active block (n_i <= kTinyRows, rows in caller order)
// in one launch, in place of launch_reduce + launch_neighbour_csr, with the same results:
// the same bits of the sums, the same offsets, counts, lists and status flags.  seg_cnt null:
// sums only; nb_idx null or L = 0: counts and offsets only.  It stages the G x n_i segment
// counts in shared memory, so it applies while tiny_epilogue_fits(G, n_i).
constexpr int kTinyRows = 8;  // one CTA does it all: past a few rows the work outgrows the launches saved
constexpr int kTinySmemMax = 100 * 1024;
bool tiny_epilogue_fits(int64_t G, int64_t n_i);
void launch_tiny_epilogue(cudaStream_t st, const double *part, int S, int64_t n_i, double *acc, double *jerk,
                          double *pot, int64_t G, int L, int cap, const int32_t *seg_cnt, const int32_t *seg_slots,
                          int64_t *off, int32_t *nb_idx, int64_t nb_capacity, int32_t *count_true, unsigned *status);

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
                      const int32_t *ell_cnt = nullptr, int64_t ell_stride = 0);
// State records of the predict-on-load form (pack_state_one layout) for particles 0..n-1.
size_t state_record_bytes(int precision, int64_t n);
void launch_pack_state(cudaStream_t st, int precision, int64_t n, const double *x, const double *v, const double *a,
                       const double *jk, const double *tl, const double *m, void *srec);

}  // namespace nbgpu
