// nb_force.cuh — the arguments of the regular-force kernels and the layouts they read and
// write (internal; not part of the ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace nbgpu {

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

// With at most this many j-splits the anchored kernels read, at the start of a CTA, the
// neighbour counts that the CTAs of the earlier segments of its rows have written, and store
// only the hits a row can still keep (nb_cap minus the hits before it).
constexpr int kPriorSegMax = 64;

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
    int32_t cap;            // nb_cap; 0 = store every hit up to L (see prior_count below)
    double *part;           // partial sums [S][7][n_i] at row k (the anchored kernels: at row-order position r)
    int32_t *seg_cnt;       // [G][n_i]
    int32_t *seg_slots;     // [G][n_i][L]
    unsigned *status;
};

}  // namespace nbgpu
