// force_fp64.cu — K2: regular force, jerk, potential and neighbour capture with every
// operation in FP64 (paper Sec. 3.2.1).  The reference-precision GPU path: same work
// decomposition as the mixed kernels (tiled for large active blocks, j-streamed for tiny
// ones), FP64 partial sums [split][7][n_i] added in a fixed order by k_reduce, and the
// same ordered neighbour segments.
//
// The neighbour test uses r^2 = (rx*rx + ry*ry) + rz*rz with IEEE round-to-nearest and no
// contraction, the same arithmetic as a plain C evaluation of the definition.
#include "nb_common.cuh"
#include "nb_kernels.cuh"

namespace nbgpu {

template <int BLOCK, int TJ>
__global__ void __launch_bounds__(BLOCK) k_force_fp64_tiled(ForceArgs A)
{
    __shared__ dvec4 sj[2][2 * TJ];
    const int tid = threadIdx.x;
    const int64_t k = (int64_t)blockIdx.x * BLOCK + tid;
    const int s = blockIdx.y;
    const int64_t tb = A.j_lo / TJ;  // first tile of the source range
    const int64_t t0 = tb + (A.n_tiles * s) / A.S, t1 = tb + (A.n_tiles * (s + 1)) / A.S;
    const dvec4 *rec = static_cast<const dvec4 *>(A.rec);

    int64_t g = -1;
    if (k < A.n_i) {
        g = A.idx[k];
        if (g < 0 || g >= A.n) {
            if (s == 0) atomicOr(A.status, ST_BAD_INDEX);
            g = -1;
        }
    }
    double xi[3] = {0, 0, 0}, vi[3] = {0, 0, 0}, rs2 = -1.0;
    if (g >= 0) {
        const dvec4 p0 = rec[2 * g], p1 = rec[2 * g + 1];
        xi[0] = p0.x; xi[1] = p0.y; xi[2] = p0.z;
        vi[0] = p1.x; vi[1] = p1.y; vi[2] = p1.z;
        if (A.want_nb) rs2 = A.rs2[A.rs2_scalar ? 0 : k];
    }
    int32_t *slot = A.seg_slots + ((int64_t)s * A.n_i + (k < A.n_i ? k : 0)) * A.L;
    int cnt = 0;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};

    auto load_tile = [&](int buf, int64_t t) {
        const dvec4 *src = rec + t * (2 * TJ);
        // each dvec4 is two 16-byte halves
        for (int e = tid; e < 4 * TJ; e += BLOCK)
            cp_async16(reinterpret_cast<char *>(&sj[buf][0]) + 16 * e,
                       reinterpret_cast<const char *>(src) + 16 * e);
        cp_async_commit();
    };
    if (t0 < t1) load_tile(0, t0);
    for (int64_t t = t0; t < t1; ++t) {
        const int buf = (int)((t - t0) & 1);
        if (t + 1 < t1) {
            load_tile(buf ^ 1, t + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int64_t jb = t * TJ;
#pragma unroll 2
        for (int jj = 0; jj < TJ; ++jj) {
            const int64_t j = jb + jj;
            const double r2 = pair_f64(sj[buf][2 * jj], sj[buf][2 * jj + 1], xi, vi, j == g, acc);
            if (r2 < rs2 && j != g && j < A.j_hi) {
                if (cnt < A.L) slot[cnt] = (int32_t)j;
                ++cnt;
            }
        }
        __syncthreads();
    }
    if (k < A.n_i) {
#pragma unroll
        for (int c = 0; c < 7; ++c) A.part[((int64_t)s * 7 + c) * A.n_i + k] = acc[c];
        if (A.want_nb) A.seg_cnt[(int64_t)s * A.n_i + k] = cnt;
    }
}

template <int IB, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_force_fp64_jstream(ForceArgs A)
{
    constexpr int W = BLOCK / 32;
    __shared__ double red[W][IB][7];
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int s = blockIdx.y;
    const int64_t k0 = (int64_t)blockIdx.x * IB;
    const int64_t j0 = A.j_lo + ((A.j_hi - A.j_lo) * s) / A.S, j1 = A.j_lo + ((A.j_hi - A.j_lo) * (s + 1)) / A.S;
    const int64_t w0 = j0 + ((j1 - j0) * w) / W, w1 = j0 + ((j1 - j0) * (w + 1)) / W;
    const int64_t seg = (int64_t)s * W + w;
    const dvec4 *rec = static_cast<const dvec4 *>(A.rec);

    double xi[IB][3], vi[IB][3], rs2[IB];
    int64_t gi[IB];
    int cnt[IB];
#pragma unroll
    for (int q = 0; q < IB; ++q) {
        const int64_t k = k0 + q;
        int64_t g = -1;
        if (k < A.n_i) {
            g = A.idx[k];
            if (g < 0 || g >= A.n) {
                if (s == 0 && tid == 0) atomicOr(A.status, ST_BAD_INDEX);
                g = -1;
            }
        }
        gi[q] = g;
        cnt[q] = 0;
        rs2[q] = -1.0;
        if (g >= 0) {
            const dvec4 p0 = rec[2 * g], p1 = rec[2 * g + 1];
            xi[q][0] = p0.x; xi[q][1] = p0.y; xi[q][2] = p0.z;
            vi[q][0] = p1.x; vi[q][1] = p1.y; vi[q][2] = p1.z;
            if (A.want_nb) rs2[q] = A.rs2[A.rs2_scalar ? 0 : k];
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) xi[q][c] = vi[q][c] = 0.0;
        }
    }
    double acc[IB][7];
#pragma unroll
    for (int q = 0; q < IB; ++q)
#pragma unroll
        for (int c = 0; c < 7; ++c) acc[q][c] = 0.0;
    const unsigned below = (1u << lane) - 1u;
    for (int64_t base = w0; base < w1; base += 32) {  // warp-uniform trip count
        const int64_t j = base + lane;
        const bool valid = j < w1;
        dvec4 p0 = make_dvec4(1e18, 1e18, 1e18, 0.0), p1 = make_dvec4(0.0, 0.0, 0.0, 0.0);
        if (valid) {
            p0 = rec[2 * j];
            p1 = rec[2 * j + 1];
        }
#pragma unroll
        for (int q = 0; q < IB; ++q) {
            const double r2 = pair_f64(p0, p1, xi[q], vi[q], j == gi[q], acc[q]);
            const bool hit = valid && r2 < rs2[q] && j != gi[q];
            const unsigned mask = __ballot_sync(0xffffffffu, hit);
            if (mask) {
                const int pos = cnt[q] + __popc(mask & below);
                if (hit && pos < A.L) A.seg_slots[(seg * A.n_i + k0 + q) * A.L + pos] = (int32_t)j;
                cnt[q] += __popc(mask);
            }
        }
    }
    if (A.want_nb && lane == 0) {
#pragma unroll
        for (int q = 0; q < IB; ++q)
            if (k0 + q < A.n_i) A.seg_cnt[seg * A.n_i + k0 + q] = cnt[q];
    }
#pragma unroll
    for (int q = 0; q < IB; ++q)
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            const double v = warp_sum(acc[q][c]);
            if (lane == 0) red[w][q][c] = v;
        }
    __syncthreads();
    for (int e = tid; e < IB * 7; e += BLOCK) {
        const int q = e / 7, c = e % 7;
        const int64_t k = k0 + q;
        if (k < A.n_i) {
            double sum = 0.0;
#pragma unroll
            for (int ww = 0; ww < W; ++ww) sum += red[ww][q][c];
            A.part[((int64_t)s * 7 + c) * A.n_i + k] = sum;
        }
    }
}

void *fp64_tiled_fn() { return (void *)k_force_fp64_tiled<128, 64>; }
int fp64_jstream_ib(int v) { return v == 0 ? 1 : 4; }

void launch_force_fp64(cudaStream_t st, int kernel, int variant, int64_t ctas_x, int S, ForceArgs a)
{
    dim3 grid((unsigned)ctas_x, (unsigned)S);
    if (kernel == 0) {
        k_force_fp64_tiled<128, 64><<<grid, 128, 0, st>>>(a);
    } else if (variant == 0) {
        k_force_fp64_jstream<1, 256><<<grid, 256, 0, st>>>(a);
    } else {
        k_force_fp64_jstream<4, 256><<<grid, 256, 0, st>>>(a);
    }
}

}  // namespace nbgpu
