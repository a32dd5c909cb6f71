// neighbours.cu — K4 (fixed-order reduction of the per-split partial sums) and K5 (the
// neighbour lists as CSR in ascending j; paper Sec. 3.2.1: the GPU accumulates the
// neighbour list during the regular force calculation).
//
// The force kernels leave, for every (segment g, active row k), the first L neighbours of
// that j-segment in ascending order and their true count.  K5 sums the counts per row
// (the untruncated neighbour number), scans min(count, nb_cap) into CSR offsets, and
// gathers each row's segments in segment order until nb_cap entries are written.
#include <atomic>

#include "nb_common.cuh"
#include "nb_kernels.cuh"

namespace nbgpu {

// ------------------------------------------------------------------------------ K4
// The partial sums of position r are those of row perm[r] (perm == null: row r).  The anchored
// force kernel writes them at the position of its spatial row order, so that its stores are
// whole sectors; the reduction reads them in that order and writes each row's sums in place.
__global__ void k_reduce(const double *__restrict__ part, int S, int64_t n_i, const int32_t *__restrict__ perm,
                         double *__restrict__ acc, double *__restrict__ jerk, double *__restrict__ pot)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_i;
         r += (int64_t)gridDim.x * blockDim.x) {
        double v[7];
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            double sum = 0.0;
            for (int s = 0; s < S; ++s) sum += part[((int64_t)s * 7 + c) * n_i + r];
            v[c] = sum;
        }
        const int64_t k = perm ? perm[r] : r;
        acc[3 * k] = v[0];
        acc[3 * k + 1] = v[1];
        acc[3 * k + 2] = v[2];
        jerk[3 * k] = v[3];
        jerk[3 * k + 1] = v[4];
        jerk[3 * k + 2] = v[5];
        pot[k] = v[6];
    }
}

// Many splits: one CTA per position, warp c sums component c; lane l adds the splits s = l,
// l+32, ... in increasing order, then the warp adds the 32 lane sums with a fixed butterfly,
// so the result is deterministic for a given split count.
__global__ void __launch_bounds__(256) k_reduce_wide(const double *__restrict__ part, int S, int64_t n_i,
                                                     const int32_t *__restrict__ perm, double *__restrict__ acc,
                                                     double *__restrict__ jerk, double *__restrict__ pot)
{
    const int64_t r = blockIdx.x;
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (c >= 7) return;  // warp-uniform
    double sum = 0.0;
    for (int s = lane; s < S; s += 32) sum += part[((int64_t)s * 7 + c) * n_i + r];
    sum = warp_sum(sum);
    if (lane == 0) {
        const int64_t k = perm ? perm[r] : r;
        if (c < 3)
            acc[3 * k + c] = sum;
        else if (c < 6)
            jerk[3 * k + c - 3] = sum;
        else
            pot[k] = sum;
    }
}

// Many splits and a few thousand positions: one warp per position, the seven components in turn, each
// summed as in k_reduce_wide (lanes over the splits, the same butterfly), so the two kernels
// give the same bits.
__global__ void __launch_bounds__(256) k_reduce_warp(const double *__restrict__ part, int S, int64_t n_i,
                                                     const int32_t *__restrict__ perm, double *__restrict__ acc,
                                                     double *__restrict__ jerk, double *__restrict__ pot)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= n_i) return;  // warp-uniform
    double v[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) {
        double sum = 0.0;
        for (int s = lane; s < S; s += 32) sum += part[((int64_t)s * 7 + c) * n_i + r];
        v[c] = warp_sum(sum);
    }
    if (lane < 7) {
        const int64_t k = perm ? perm[r] : r;
        double x = v[0];
#pragma unroll
        for (int c = 1; c < 7; ++c)
            if (lane == c) x = v[c];
        if (lane < 3)
            acc[3 * k + lane] = x;
        else if (lane < 6)
            jerk[3 * k + lane - 3] = x;
        else
            pot[k] = x;
    }
}

void launch_reduce(cudaStream_t st, const double *part, int S, int64_t n_i, double *acc, double *jerk,
                   double *pot, const int32_t *perm)
{
    if (S > 16 && n_i <= 1024) {  // a warp per component and position: the split loop in parallel
        k_reduce_wide<<<(unsigned)n_i, 256, 0, st>>>(part, S, n_i, perm, acc, jerk, pot);
        return;
    }
    if (S > 16 && n_i <= 4096) {  // a warp per position (above, the coalesced thread-per-position form)
        k_reduce_warp<<<(unsigned)((n_i + 7) / 8), 256, 0, st>>>(part, S, n_i, perm, acc, jerk, pot);
        return;
    }
    int64_t g = (n_i + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    k_reduce<<<(unsigned)g, 256, 0, st>>>(part, S, n_i, perm, acc, jerk, pot);
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

// Per row: true count = sum over segments; kept = min(count, cap); block-local scan. A launch
// of one CTA (n_i <= SCAN_BLOCK) has the whole scan: it writes the total and checks the
// capacity itself, and the block-sum passes are skipped.
__global__ void k_seg_scan_local(const int32_t *__restrict__ seg_cnt, int64_t G, int64_t n_i, int cap,
                                 int64_t *__restrict__ off, int64_t *__restrict__ bsum,
                                 int32_t *__restrict__ count_true, unsigned *status, int64_t capacity)
{
    __shared__ int64_t wsum[32];
    const int64_t k = blockIdx.x * (int64_t)SCAN_BLOCK + threadIdx.x;
    int64_t kept = 0;
    if (k < n_i) {
        int64_t c = 0;
        for (int64_t g = 0; g < G; ++g) c += seg_cnt[g * n_i + k];
        kept = c < cap ? c : cap;
        if (c > cap) atomicOr(status, ST_NB_TRUNCATED);
        if (count_true) count_true[k] = (int32_t)(c < INT32_MAX ? c : INT32_MAX);
    }
    int64_t total;
    const int64_t ex = block_exclusive_scan(kept, wsum, total);
    if (k < n_i) off[k] = ex;
    if (threadIdx.x == 0) {
        bsum[blockIdx.x] = total;
        if (gridDim.x == 1) {
            off[n_i] = total;
            if (total > capacity) atomicOr(status, ST_CSR_FULL);
        }
    }
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

// ------------------------------------------------------------------------------ ordered gather
// One warp per row: segments are visited 32 at a time; a warp scan of their kept sizes gives
// each segment's place in the row, then the warp copies segment after segment (coalesced).
__global__ void k_seg_gather(const int32_t *__restrict__ seg_cnt, const int32_t *__restrict__ seg_slots, int64_t G,
                             int64_t n_i, int L, const int64_t *__restrict__ off, int32_t *__restrict__ nb_idx,
                             int64_t capacity, const int32_t *__restrict__ perm)
{
    const int lane = threadIdx.x & 31;
    const int64_t k = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);  // segment position
    if (k >= n_i) return;  // warp-uniform
    const int64_t row = perm ? perm[k] : k;
    const int64_t o0 = off[row];
    const int64_t kept = off[row + 1] - o0;
    int64_t done = 0;
    for (int64_t g0 = 0; g0 < G && done < kept; g0 += 32) {
        const int64_t g = g0 + lane;
        int c = g < G ? seg_cnt[g * n_i + k] : 0;
        c = c < L ? c : L;
        int x = c;  // inclusive warp scan of the kept sizes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const int64_t start = done + x - c;
        for (int q = 0; q < 32; ++q) {
            const int64_t st = __shfl_sync(0xffffffffu, start, q);
            int cq = __shfl_sync(0xffffffffu, c, q);
            if (st >= kept) break;  // warp-uniform
            if (st + cq > kept) cq = (int)(kept - st);
            const int32_t *src = seg_slots + ((g0 + q) * n_i + k) * (int64_t)L;
            for (int e = lane; e < cq; e += 32)
                if (o0 + st + e < capacity) nb_idx[o0 + st + e] = src[e];
        }
        done += __shfl_sync(0xffffffffu, x, 31);
    }
}

// ------------------------------------------------------------------------------ many segments
// With tiny active blocks the j-streamed kernels leave thousands of segments per row; these
// block-per-row versions walk them with all threads of a CTA instead of one thread or warp.
constexpr int ROW_BLOCK = 256;

// True neighbour count of every row: block-wide sum over the row's segments.
__global__ void __launch_bounds__(ROW_BLOCK) k_seg_count_rows(const int32_t *__restrict__ seg_cnt, int64_t G,
                                                              int64_t n_i, int32_t *__restrict__ total,
                                                              const int32_t *__restrict__ perm)
{
    __shared__ int64_t ws[ROW_BLOCK / 32];
    const int64_t k = blockIdx.x;  // segment position (row perm[k])
    int64_t c = 0;
    for (int64_t g = threadIdx.x; g < G; g += ROW_BLOCK) c += seg_cnt[g * n_i + k];
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t s = 0;
        for (int w = 0; w < ROW_BLOCK / 32; ++w) s += ws[w];
        total[perm ? perm[k] : k] = (int32_t)(s < INT32_MAX ? s : INT32_MAX);
    }
}

// The same with few segments: a thread per position.
__global__ void k_seg_count_pos(const int32_t *__restrict__ seg_cnt, int64_t G, int64_t n_i,
                                int32_t *__restrict__ total, const int32_t *__restrict__ perm)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_i; k += (int64_t)gridDim.x * blockDim.x) {
        int64_t c = 0;
        for (int64_t g = 0; g < G; ++g) c += seg_cnt[g * n_i + k];
        total[perm[k]] = (int32_t)(c < INT32_MAX ? c : INT32_MAX);
    }
}

// Ordered gather of one row with a whole CTA: thread t owns the contiguous segment range
// [t*G/B, (t+1)*G/B); a block scan of the owned kept sizes places every segment in the row.
__global__ void __launch_bounds__(ROW_BLOCK) k_seg_gather_rows(const int32_t *__restrict__ seg_cnt,
                                                               const int32_t *__restrict__ seg_slots, int64_t G,
                                                               int64_t n_i, int L, const int64_t *__restrict__ off,
                                                               int32_t *__restrict__ nb_idx, int64_t capacity,
                                                               const int32_t *__restrict__ perm)
{
    __shared__ int64_t wsum[32];
    const int64_t k = blockIdx.x;  // segment position (row perm[k])
    const int64_t g0 = (G * threadIdx.x) / ROW_BLOCK, g1 = (G * (threadIdx.x + 1)) / ROW_BLOCK;
    int64_t mine = 0;
    for (int64_t g = g0; g < g1; ++g) {
        const int c = seg_cnt[g * n_i + k];
        mine += c < L ? c : L;
    }
    int64_t total;
    int64_t pos = block_exclusive_scan(mine, wsum, total);
    const int64_t row = perm ? perm[k] : k;
    const int64_t o0 = off[row], kept = off[row + 1] - o0;
    for (int64_t g = g0; g < g1 && pos < kept; ++g) {
        int c = seg_cnt[g * n_i + k];
        c = c < L ? c : L;
        if (pos + c > kept) c = (int)(kept - pos);
        const int32_t *src = seg_slots + (g * n_i + k) * (int64_t)L;
        for (int e = 0; e < c; ++e)
            if (o0 + pos + e < capacity) nb_idx[o0 + pos + e] = src[e];
        pos += c;
    }
}

// ------------------------------------------------------------------------------ tiny blocks
// Reduction and neighbour CSR of a tiny active block (at most kTinyRows rows, in caller order)
// in one CTA, in place of the reduce kernel and the three CSR kernels: for such a block the
// dependent launches, not the work, are the cost (with more rows the one CTA's own work, FP64
// adds on one SM and the copies of dense rows, outgrows the launches saved).  The partial sums
// are added in the order launch_reduce takes for S splits (a warp per row and component:
// lanes over the splits and the warp butterfly for S > 16, one lane in split order
// otherwise), so they carry the same bits.  The lists are those of the CSR kernels: the
// G x n_i segment counts are staged in shared memory (row r's segments contiguous, row stride
// Gp odd so the transposing stores do not collide in a bank); one block scan over the
// (row, segment) items, each thread owning a contiguous run of them, gives every row's true
// count, kept = min(count, cap), the offsets (a scan over the rows) and every segment's place
// in its row, which replaces its count in shared memory; then every output position finds its
// row and, by binary search over the places, the segment entry it takes.
constexpr int kTinyBlock = 1024;
constexpr int kTinyPer = (kTinySmemMax / 4 + kTinyBlock - 1) / kTinyBlock;  // counts a thread loads

__global__ void __launch_bounds__(kTinyBlock) k_tiny_epilogue(
    const double *__restrict__ part, int S, int n_i, double *__restrict__ acc, double *__restrict__ jerk,
    double *__restrict__ pot, int G, int L, int cap, const int32_t *__restrict__ seg_cnt,
    const int32_t *__restrict__ seg_slots, int64_t *__restrict__ off, int32_t *__restrict__ nb_idx, int64_t capacity,
    int32_t *__restrict__ count_true, unsigned *status)
{
    extern __shared__ int32_t cnt_s[];  // [n_i][Gp]
    __shared__ int64_t wsum[32];
    __shared__ int64_t base_l[kTinyRows + 1], base_t[kTinyRows + 1], row_off[kTinyRows], row_kept[kTinyRows];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int Gp = G | 1;
    const int F = G * n_i;  // at most kTinySmemMax / 4 items
    // segment counts into shared memory: every load of a thread issued before the first
    // store (a single CTA cannot hide the latency of one load at a time), in global order
    if (seg_cnt) {
        int v[kTinyPer];
#pragma unroll
        for (int i = 0; i < kTinyPer; ++i) {
            const int f = tid + i * kTinyBlock;
            v[i] = f < F ? seg_cnt[f] : 0;
        }
        // f = tid + i * kTinyBlock is segment f / n_i of row f % n_i: stepped, not divided
        int r = tid % n_i, g = tid / n_i;
        const int dr = kTinyBlock % n_i, dg = kTinyBlock / n_i;
#pragma unroll
        for (int i = 0; i < kTinyPer; ++i) {
            if (tid + i * kTinyBlock < F) cnt_s[r * Gp + g] = v[i];
            r += dr;
            g += dg;
            if (r >= n_i) r -= n_i, ++g;
        }
    }
    // the sums: item e = (row e / 7, component e % 7), a warp each
    for (int e = w; e < n_i * 7; e += kTinyBlock / 32) {
        const int r = e / 7, c = e % 7;
        const double *pc = part + (int64_t)c * n_i + r;  // split s at pc[s * 7 * n_i]
        const int64_t ps = (int64_t)7 * n_i;
        double sum = 0.0;
        if (S > 16) {
#pragma unroll 8
            for (int s = lane; s < S; s += 32) sum += pc[s * ps];
            sum = warp_sum(sum);
        } else if (lane == 0) {
#pragma unroll 8
            for (int s = 0; s < S; ++s) sum += pc[s * ps];
        }
        if (lane == 0) {
            if (c < 3)
                acc[3 * r + c] = sum;
            else if (c < 6)
                jerk[3 * r + c - 3] = sum;
            else
                pot[r] = sum;
        }
    }
    if (!seg_cnt) return;  // no neighbour output wanted
    __syncthreads();
    // thread-contiguous runs [f0, f1) of the flattened items f = r * G + g
    const int per = (F + kTinyBlock - 1) / kTinyBlock;
    const int f0 = tid * per < F ? tid * per : F, f1 = f0 + per < F ? f0 + per : F;
    const int r0 = f0 / G, g0 = f0 % G;
    int64_t sl = 0, st = 0;  // stored (at most L a segment) and true counts of the run
    for (int f = f0, r = r0, g = g0; f < f1; ++f) {
        const int c = cnt_s[r * Gp + g];
        sl += c < L ? c : L;
        st += c;
        if (++g == G) g = 0, ++r;
    }
    int64_t tot_l, tot_t;
    const int64_t ex_l = block_exclusive_scan(sl, wsum, tot_l);
    const int64_t ex_t = block_exclusive_scan(st, wsum, tot_t);
    {  // the prefixes at the first segment of every row
        int64_t pl = ex_l, pt = ex_t;
        for (int f = f0, r = r0, g = g0; f < f1; ++f) {
            const int c = cnt_s[r * Gp + g];
            if (g == 0) {
                base_l[r] = pl;
                base_t[r] = pt;
            }
            pl += c < L ? c : L;
            pt += c;
            if (++g == G) g = 0, ++r;
        }
        if (tid == 0) {
            base_l[n_i] = tot_l;
            base_t[n_i] = tot_t;
        }
    }
    __syncthreads();
    if (w == 0) {  // rows: true and kept counts, offsets (a warp scan over at most 32 rows)
        int64_t c = 0, kept = 0;
        if (lane < n_i) {
            c = base_t[lane + 1] - base_t[lane];
            kept = c < cap ? c : cap;
            if (c > cap) atomicOr(status, ST_NB_TRUNCATED);
            if (count_true) count_true[lane] = (int32_t)(c < INT32_MAX ? c : INT32_MAX);
        }
        int64_t x = kept;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane < n_i) {
            off[lane] = x - kept;
            row_off[lane] = x - kept;
            row_kept[lane] = kept;
        }
        if (lane == 31) {
            off[n_i] = x;
            if (x > capacity) atomicOr(status, ST_CSR_FULL);
        }
    }
    if (!nb_idx || L <= 0) return;
    // every count becomes its segment's place in the row: the entries the row's earlier
    // segments store (each run is read and overwritten by its own thread only)
    {
        int64_t pl = ex_l;
        for (int f = f0, r = r0, g = g0; f < f1; ++f) {
            int32_t *q = &cnt_s[r * Gp + g];
            const int c = *q;
            *q = (int32_t)(pl - base_l[r]);
            pl += c < L ? c : L;
            if (++g == G) g = 0, ++r;
        }
    }
    __syncthreads();
    // the copies, spread over the output positions: position o of the CSR lies in row r
    // (row_off[r] <= o < row_off[r] + kept_r) at place q of it, taken from the last segment
    // whose place is <= q (a binary search over the row's places); a dense row's entries come
    // from few segments, so a thread per segment would copy them one after another
    const int64_t total = row_off[n_i - 1] + row_kept[n_i - 1];
    const int64_t last = total < capacity ? total : capacity;
    for (int64_t o = tid; o < last; o += kTinyBlock) {
        int r = 0, rh = n_i;  // the last row whose offset is <= o
        while (rh - r > 1) {
            const int mid = (r + rh) >> 1;
            if (row_off[mid] <= o) r = mid; else rh = mid;
        }
        const int q = (int)(o - row_off[r]);
        const int32_t *P = cnt_s + r * Gp;
        int lo = 0, hi = G;  // the first segment whose place exceeds q is hi
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (P[mid] <= q) lo = mid + 1; else hi = mid;
        }
        const int g = lo - 1;
        nb_idx[o] = seg_slots[((int64_t)g * n_i + r) * L + (q - P[g])];
    }
}

bool tiny_epilogue_fits(int64_t G, int64_t n_i)
{
    return n_i >= 1 && n_i <= kTinyRows && (G | 1) * n_i * 4 <= kTinySmemMax;
}

void launch_tiny_epilogue(cudaStream_t st, const double *part, int S, int64_t n_i, double *acc, double *jerk,
                          double *pot, int64_t G, int L, int cap, const int32_t *seg_cnt, const int32_t *seg_slots,
                          int64_t *off, int32_t *nb_idx, int64_t nb_capacity, int32_t *count_true, unsigned *status)
{
    const size_t smem = seg_cnt ? (size_t)(G | 1) * n_i * 4 : 0;
    if (smem > 48 * 1024) {  // the opt-in above 48 KB of dynamic shared memory, once per device
        static std::atomic<unsigned long long> done{0};  // a bit per device 0..63; others set it every call
        int dev = 0;
        cudaGetDevice(&dev);
        const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
        if (!bit || !(done.load() & bit)) {
            if (cudaFuncSetAttribute(k_tiny_epilogue, cudaFuncAttributeMaxDynamicSharedMemorySize, kTinySmemMax) ==
                cudaSuccess)
                done.fetch_or(bit);
        }
    }
    k_tiny_epilogue<<<1, kTinyBlock, smem, st>>>(part, S, (int)n_i, acc, jerk, pot, (int)G, L, cap, seg_cnt, seg_slots,
                                                 off, nb_idx, nb_capacity, count_true, status);
}

int launch_neighbour_csr(cudaStream_t st, int64_t G, int64_t n_i, int L, int cap, const int32_t *seg_cnt,
                         const int32_t *seg_slots, int64_t *off, int32_t *nb_idx, int64_t nb_capacity,
                         int32_t *count_true, int64_t *scan_tmp, int32_t *row_total, unsigned *status,
                         const int32_t *perm)
{
    const int64_t nb = (n_i + SCAN_BLOCK - 1) / SCAN_BLOCK;
    int kernels = 0;
    // segments at spatial-order positions: the per-row totals are put in row order first
    const bool many = (G > 64 || perm) && row_total != nullptr;
    if (many && (G > 64 || !perm)) {  // sum the segments of every row in parallel first
        k_seg_count_rows<<<(unsigned)n_i, ROW_BLOCK, 0, st>>>(seg_cnt, G, n_i, row_total, perm);
        ++kernels;
    } else if (many) {
        int64_t g = (n_i + 255) / 256;
        if (g > 152 * 16) g = 152 * 16;
        k_seg_count_pos<<<(unsigned)(g < 1 ? 1 : g), 256, 0, st>>>(seg_cnt, G, n_i, row_total, perm);
        ++kernels;
    }
    k_seg_scan_local<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(many ? row_total : seg_cnt, many ? 1 : G, n_i, cap, off,
                                                          scan_tmp, count_true, status, nb_capacity);
    ++kernels;
    if (nb > 1) {
        k_scan_blocks<<<1, SCAN_BLOCK, 0, st>>>(scan_tmp, nb);
        k_scan_add<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(off, scan_tmp, n_i, nb, nb_capacity, status);
        kernels += 2;
    }
    if (!nb_idx || L <= 0) return kernels;
    if (G > 64 && row_total != nullptr) {
        k_seg_gather_rows<<<(unsigned)n_i, ROW_BLOCK, 0, st>>>(seg_cnt, seg_slots, G, n_i, L, off, nb_idx, nb_capacity,
                                                               perm);
    } else {
        const int64_t blocks = (n_i + 7) / 8;
        k_seg_gather<<<(unsigned)blocks, 256, 0, st>>>(seg_cnt, seg_slots, G, n_i, L, off, nb_idx, nb_capacity, perm);
    }
    return kernels + 1;
}

}  // namespace nbgpu
