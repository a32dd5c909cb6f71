// nb_kernels.cuh — host-side launchers of the library's kernels (internal; not part of the ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace nbgpu {

// Predicted j-records.
//  FP64 : 2 dvec4 per particle  {x, y, z, m}, {vx, vy, vz, 0}                 (64 B)
//  mixed: 3 float4  per particle  {x_hi, y_hi, z_hi, m}, {x_lo, y_lo, z_lo, 0},
//                                 {vx, vy, vz, 0}                               (48 B)
// x_hi = fl32(x), x_lo = fl32(x - x_hi).  Records n .. n_pad-1 are padding: mass 0,
// position 1e18, so whole tiles can be read without a bounds check.

struct ForceArgs {
    const void *rec;        // dvec4* (FP64) or float4* (mixed)
    int64_t n;              // particles
    int64_t n_tiles;        // j-tiles of the launch's tile size covering n_pad
    const int32_t *idx;     // active indices
    int64_t n_i;
    const double *rs2;      // (n_i) or scalar
    int32_t rs2_scalar;
    int32_t want_nb;        // 0: skip neighbour capture
    int32_t S;              // j-splits (blockIdx.y)
    int32_t cap;            // neighbour slots per active particle in nb_tmp
    double *part;           // partial sums [S][7][n_i]
    int32_t *nb_cnt;        // (n_i) neighbour counters (zeroed by the caller)
    int32_t *nb_tmp;        // (n_i, cap) unordered neighbour slots
    unsigned *status;
};

struct Plan {
    int kernel;     // 0 FP64 tiled, 1 mixed tiled, 2 mixed j-streamed, 3 FP64 j-streamed
    int variant;    // kernel-specific template variant
    int i_per_cta;  // active particles per CTA
    int S;          // j-splits
    int64_t ctas;
    int tj;         // j-tile (tiled kernels) or 0
};

// Launch-shape planner (pure host function; no CUDA calls).
Plan plan_force(int precision, int num_sms, const int *ctas_per_sm, int64_t n, int64_t n_i);
// Occupancy of each kernel variant (filled once per context).
void query_occupancy(int *ctas_per_sm /* [8] */);

void launch_predict(cudaStream_t st, int64_t n, int64_t n_pad, double t, const double *x,
                    const double *v, const double *a, const double *jk, const double *tl,
                    const double *m, double *xp, double *vp, void *rec64, void *rec32);
void launch_pack_predicted(cudaStream_t st, int64_t n, int64_t n_pad, const double *xp,
                           const double *vp, const double *m, void *rec64, void *rec32);

void launch_force(cudaStream_t st, const Plan &p, ForceArgs a);

void launch_reduce(cudaStream_t st, const double *part, int S, int64_t n_i, double *acc,
                   double *jerk, double *pot);

// Neighbour CSR: counts -> offsets -> sorted lists; lists over nb_cap are recomputed in
// ascending j order.  `rec` / `precision` select the distance arithmetic.
void launch_neighbour_csr(cudaStream_t st, int precision, const void *rec, int64_t n,
                          const int32_t *idx, int64_t n_i, const double *rs2, int rs2_scalar,
                          const int32_t *nb_cnt, const int32_t *nb_tmp, int cap,
                          int64_t *off, int32_t *nb_idx, int64_t nb_capacity,
                          int32_t *count_true, int64_t *scan_tmp, int32_t *over_list,
                          unsigned *status, int num_sms);

size_t neighbour_scan_tmp_elems(int64_t n_i);

void launch_backward(cudaStream_t st, int precision, const void *rec, int64_t n, const int32_t *idx,
                     int64_t n_i, const double *g_acc, const double *g_jerk, const double *g_pot,
                     double *g_x, double *g_v, double *g_m, int32_t *mark, unsigned *status,
                     int num_sms);

}  // namespace nbgpu
