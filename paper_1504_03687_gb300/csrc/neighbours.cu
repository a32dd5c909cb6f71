// neighbours.cu — K4 (fixed-order reduction of the per-split partial sums) and K5 (the
// neighbour lists as CSR in ascending j; paper Sec. 3.2.1: the GPU accumulates the
// neighbour list during the regular force calculation).
//
// The force kernels append neighbour indices to per-particle slot arrays with atomics, so
// a list arrives unordered.  K5 turns the counts into offsets (exclusive scan of
// min(count, nb_cap)), sorts each list with a warp-wide bitonic sort and writes it.  A
// list whose true count exceeds nb_cap holds an arbitrary subset of its neighbours, so it
// is recomputed by one CTA that scans j in ascending order with the same distance
// arithmetic and keeps the first nb_cap hits.
#include <climits>

#include "nb_common.cuh"
#include "nb_kernels.cuh"

namespace nbgpu {

// ------------------------------------------------------------------------------ K4
__global__ void k_reduce(const double *__restrict__ part, int S, int64_t n_i, double *__restrict__ acc,
                         double *__restrict__ jerk, double *__restrict__ pot)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_i;
         k += (int64_t)gridDim.x * blockDim.x) {
        double v[7];
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            double sum = 0.0;
            for (int s = 0; s < S; ++s) sum += part[((int64_t)s * 7 + c) * n_i + k];
            v[c] = sum;
        }
        acc[3 * k] = v[0];
        acc[3 * k + 1] = v[1];
        acc[3 * k + 2] = v[2];
        jerk[3 * k] = v[3];
        jerk[3 * k + 1] = v[4];
        jerk[3 * k + 2] = v[5];
        pot[k] = v[6];
    }
}

void launch_reduce(cudaStream_t st, const double *part, int S, int64_t n_i, double *acc, double *jerk,
                   double *pot)
{
    int64_t g = (n_i + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    k_reduce<<<(unsigned)g, 256, 0, st>>>(part, S, n_i, acc, jerk, pot);
}

// ------------------------------------------------------------------------------ scan
constexpr int SCAN_BLOCK = 1024;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *wsum, int64_t &total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t s = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) wsum[lane] = s;  // inclusive warp sums
    }
    __syncthreads();
    total = wsum[nw - 1];
    const int64_t before = w > 0 ? wsum[w - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void k_scan_local(const int32_t *__restrict__ cnt, int64_t n_i, int cap, int64_t *__restrict__ off,
                             int64_t *__restrict__ bsum, int32_t *__restrict__ count_true, unsigned *status)
{
    __shared__ int64_t wsum[32];
    const int64_t k = blockIdx.x * (int64_t)SCAN_BLOCK + threadIdx.x;
    int64_t kept = 0;
    if (k < n_i) {
        const int c = cnt[k];
        kept = c < cap ? c : cap;
        if (c > cap) atomicOr(status, ST_NB_TRUNCATED);
        if (count_true) count_true[k] = c;
    }
    int64_t total;
    const int64_t ex = block_exclusive_scan(kept, wsum, total);
    if (k < n_i) off[k] = ex;
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// Exclusive scan of the nb block sums in one CTA (chunks of SCAN_BLOCK with a carry);
// bsum[nb] receives the grand total.
__global__ void k_scan_blocks(int64_t *bsum, int64_t nb)
{
    __shared__ int64_t wsum[32];
    int64_t carry = 0;
    for (int64_t base = 0; base < nb; base += SCAN_BLOCK) {
        const int64_t b = base + threadIdx.x;
        const int64_t v = b < nb ? bsum[b] : 0;
        int64_t total;
        const int64_t ex = block_exclusive_scan(v, wsum, total);
        if (b < nb) bsum[b] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void k_scan_add(int64_t *__restrict__ off, const int64_t *__restrict__ bsum, int64_t n_i,
                           int64_t nb, int64_t capacity, unsigned *status)
{
    const int64_t k = blockIdx.x * (int64_t)SCAN_BLOCK + threadIdx.x;
    if (k < n_i) off[k] += bsum[blockIdx.x];
    if (k == 0) {
        off[n_i] = bsum[nb];
        if (bsum[nb] > capacity) atomicOr(status, ST_CSR_FULL);
    }
}

size_t neighbour_scan_tmp_elems(int64_t n_i) { return (size_t)((n_i + SCAN_BLOCK - 1) / SCAN_BLOCK) + 2; }

// ------------------------------------------------------------------------------ sort + write
// One warp per active particle; the warp's slots are sorted in shared memory.
__global__ void k_sort_write(const int32_t *__restrict__ cnt, const int32_t *__restrict__ tmp, int cap,
                             int pow2cap, int64_t n_i, const int64_t *__restrict__ off,
                             int32_t *__restrict__ nb_idx, int64_t capacity,
                             int32_t *__restrict__ over_list, unsigned *status)
{
    extern __shared__ int32_t sbuf[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t k = blockIdx.x * (int64_t)(blockDim.x >> 5) + w;
    if (k >= n_i) return;
    const int c = cnt[k];
    if (c > cap) {
        if (lane == 0) {
            const unsigned slot = atomicAdd(status + SS_OVERFLOW_COUNT, 1u);
            over_list[slot] = (int32_t)k;
        }
        return;
    }
    if (c == 0) return;
    int P = 1;
    while (P < c) P <<= 1;
    int32_t *s = sbuf + (int64_t)w * pow2cap;
    const int32_t *src = tmp + k * (int64_t)cap;
    for (int e = lane; e < P; e += 32) s[e] = e < c ? src[e] : INT_MAX;
    __syncwarp();
    for (int kk = 2; kk <= P; kk <<= 1) {
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int e = lane; e < P; e += 32) {
                const int p = e ^ jj;
                if (p > e) {
                    const int32_t a = s[e], b = s[p];
                    const bool up = (e & kk) == 0;
                    if ((a > b) == up) {
                        s[e] = b;
                        s[p] = a;
                    }
                }
            }
            __syncwarp();
        }
    }
    const int64_t o = off[k];
    for (int e = lane; e < c; e += 32)
        if (o + e < capacity) nb_idx[o + e] = s[e];
}

// ------------------------------------------------------------------------------ ordered recompute
template <bool MIXED>
__global__ void __launch_bounds__(256) k_recompute(const void *__restrict__ recv, int64_t n,
                                                   const int32_t *__restrict__ idx, const double *__restrict__ rs2,
                                                   int rs2_scalar, int cap, const int64_t *__restrict__ off,
                                                   int32_t *__restrict__ nb_idx, int64_t capacity,
                                                   const int32_t *__restrict__ over_list, const unsigned *status)
{
    __shared__ int wt[8];
    const unsigned n_over = status[SS_OVERFLOW_COUNT];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (unsigned o = blockIdx.x; o < n_over; o += gridDim.x) {
        const int64_t k = over_list[o];
        const int64_t g = idx[k];
        const int64_t base_out = off[k];
        int base = 0;
        if (MIXED) {
            const float4 *rec = static_cast<const float4 *>(recv);
            const float4 ih = rec[3 * g], il = rec[3 * g + 1];
            const float r2max = __double2float_rn(rs2[rs2_scalar ? 0 : k]);
            for (int64_t jb = 0; jb < n && base < cap; jb += 256) {
                const int64_t j = jb + threadIdx.x;
                bool f = false;
                if (j < n && j != g) {
                    const float4 jh = rec[3 * j], jl = rec[3 * j + 1];
                    const float r2 = r2_f32(ds_diff(jh.x, jl.x, ih.x, il.x), ds_diff(jh.y, jl.y, ih.y, il.y),
                                            ds_diff(jh.z, jl.z, ih.z, il.z));
                    f = r2 < r2max;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, f);
                if (lane == 0) wt[w] = __popc(bal);
                __syncthreads();
                int woff = 0, tot = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    woff += q < w ? wt[q] : 0;
                    tot += wt[q];
                }
                const int pos = base + woff + __popc(bal & ((1u << lane) - 1u));
                if (f && pos < cap && base_out + pos < capacity) nb_idx[base_out + pos] = (int32_t)j;
                __syncthreads();
                base += tot;
            }
        } else {
            const dvec4 *rec = static_cast<const dvec4 *>(recv);
            const dvec4 xi = rec[2 * g];
            const double r2max = rs2[rs2_scalar ? 0 : k];
            for (int64_t jb = 0; jb < n && base < cap; jb += 256) {
                const int64_t j = jb + threadIdx.x;
                bool f = false;
                if (j < n && j != g) {
                    const dvec4 xj = rec[2 * j];
                    const double r2 = r2_f64(__dsub_rn(xj.x, xi.x), __dsub_rn(xj.y, xi.y), __dsub_rn(xj.z, xi.z));
                    f = r2 < r2max;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, f);
                if (lane == 0) wt[w] = __popc(bal);
                __syncthreads();
                int woff = 0, tot = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    woff += q < w ? wt[q] : 0;
                    tot += wt[q];
                }
                const int pos = base + woff + __popc(bal & ((1u << lane) - 1u));
                if (f && pos < cap && base_out + pos < capacity) nb_idx[base_out + pos] = (int32_t)j;
                __syncthreads();
                base += tot;
            }
        }
    }
}

void launch_neighbour_csr(cudaStream_t st, int precision, const void *rec, int64_t n, const int32_t *idx,
                          int64_t n_i, const double *rs2, int rs2_scalar, const int32_t *nb_cnt,
                          const int32_t *nb_tmp, int cap, int64_t *off, int32_t *nb_idx, int64_t nb_capacity,
                          int32_t *count_true, int64_t *scan_tmp, int32_t *over_list, unsigned *status,
                          int num_sms)
{
    const int64_t nb = (n_i + SCAN_BLOCK - 1) / SCAN_BLOCK;
    k_scan_local<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(nb_cnt, n_i, cap, off, scan_tmp, count_true, status);
    k_scan_blocks<<<1, SCAN_BLOCK, 0, st>>>(scan_tmp, nb);
    k_scan_add<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(off, scan_tmp, n_i, nb, nb_capacity, status);
    if (!nb_idx) return;
    int pow2cap = 1;
    while (pow2cap < cap) pow2cap <<= 1;
    int warps = 8;
    while (warps > 1 && (size_t)warps * pow2cap * 4 > 48 * 1024) warps >>= 1;
    const int64_t blocks = (n_i + warps - 1) / warps;
    k_sort_write<<<(unsigned)blocks, 32 * warps, (size_t)warps * pow2cap * 4, st>>>(
        nb_cnt, nb_tmp, cap, pow2cap, n_i, off, nb_idx, nb_capacity, over_list, status);
    const int grid = 2 * (num_sms > 0 ? num_sms : 152);
    if (precision == 1)
        k_recompute<true><<<grid, 256, 0, st>>>(rec, n, idx, rs2, rs2_scalar, cap, off, nb_idx, nb_capacity,
                                                over_list, status);
    else
        k_recompute<false><<<grid, 256, 0, st>>>(rec, n, idx, rs2, rs2_scalar, cap, off, nb_idx, nb_capacity,
                                                 over_list, status);
}

}  // namespace nbgpu
