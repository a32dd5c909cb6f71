// roworder.cu — spatial order of an active block's rows for the anchored force kernel.
//
// The anchored kernel measures every position from one anchor per CTA (the predicted
// position of one of the CTA's rows), so it wants the rows of a CTA to lie close together.
// The rows of an active block arrive in the caller's order (the time-step list, which is not
// spatial), so before such a launch they are put into Morton (Z-curve) order of their
// predicted positions: 8 bits per coordinate over the block's bounding box, 24-bit keys,
// sorted by a stable three-pass LSD radix sort (8 bits a pass).  The result is a permutation
// perm of [0, n_i): the kernel's r-th row is row perm[r] of the call, and every output stays
// at its row's own place.  The order only affects speed — the anchored kernel is exact for
// any order — but it is deterministic (integer keys from fixed float operations, a stable
// sort), so results are reproducible bit for bit.
//
// Blocks of up to kRoChunk rows are ordered by one CTA in shared memory (one launch).  Larger
// blocks take a bounding-box pass and, per radix pass, a ranking pass (every CTA ranks its
// kRoChunk rows per digit in row order: a warp match within each round of 256 rows, warp
// counts scanned across the round, running counts across the rounds), a one-CTA exclusive scan
// of the per-CTA digit counts stored digit-major (so equal digits keep CTA order), and a
// scatter to base + rank.  Rows whose index is outside [0, n) get the largest key (they sort
// last; the force kernel reports them).
#include "nb_common.cuh"
#include "nb_kernels.cuh"

namespace nbgpu {

constexpr int kRoThreads = 256;
constexpr int kRoWarps = kRoThreads / 32;
constexpr int kRoItems = 16;
constexpr int kRoChunk = kRoThreads * kRoItems;  // rows per CTA (4096)
constexpr int kRoBins = 256;                     // 8-bit digits
constexpr int kRoPasses = 3;                     // 24-bit keys
constexpr uint32_t kRoBadKey = 0xFFFFFFu;
static_assert(kRoBins == kRoThreads, "one digit per thread in the count loops");

// order-preserving unsigned image of a float (larger float -> larger unsigned)
__device__ __forceinline__ unsigned ro_ord(float f)
{
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ro_unord(unsigned u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// bit k of an 8-bit value to bit 3k
__device__ __forceinline__ uint32_t ro_spread(uint32_t a)
{
    a &= 0xffu;
    a = (a | (a << 8)) & 0x00F00Fu;
    a = (a | (a << 4)) & 0x0C30C3u;
    a = (a | (a << 2)) & 0x249249u;
    return a;
}

struct RoRows {
    const float4 *rec;   // mixed j-records (x_hi in the first float4 of each particle)
    const int32_t *idx;  // active indices; null: row r is particle r (n_i = n)
    int64_t n, n_i;
    __device__ __forceinline__ int64_t particle(int64_t r) const { return idx ? (int64_t)idx[r] : r; }
};

// The bounding box is kept as ordered unsigned images, the minimum complemented, so that both
// halves are atomic maxima over words that start at zero: box = {~min x, ~min y, ~min z,
// max x, max y, max z}.
__device__ __forceinline__ void ro_frame(const unsigned *box, float (&lo)[3], float (&inv)[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lo[c] = ro_unord(~box[c]);
        const float hi = ro_unord(box[3 + c]);
        const float ext = __fsub_rn(hi, lo[c]);
        inv[c] = ext > 0.f ? __fdiv_rn(256.f, ext) : 0.f;
    }
}

__device__ __forceinline__ uint32_t ro_key(const RoRows &R, int64_t r, const float (&lo)[3], const float (&inv)[3])
{
    const int64_t g = R.particle(r);
    if (g < 0 || g >= R.n) return kRoBadKey;
    const float4 p = R.rec[3 * g];
    const float x[3] = {p.x, p.y, p.z};
    uint32_t key = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        int q = __float2int_rz(__fmul_rn(__fsub_rn(x[c], lo[c]), inv[c]));
        q = q < 0 ? 0 : (q > 255 ? 255 : q);
        key |= ro_spread((uint32_t)q) << c;
    }
    return key;
}

__device__ __forceinline__ float ro_warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float ro_warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide bounding box of rows [r0, r1) (stride kRoThreads) into s_box (ordered images,
// minimum complemented), merged by atomic maxima; s_box starts at zero.
__device__ void ro_box_rows(const RoRows &R, int64_t r0, int64_t r1, int64_t stride, unsigned *s_box)
{
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t r = r0; r < r1; r += stride) {
        const int64_t g = R.particle(r);
        if (g < 0 || g >= R.n) continue;
        const float4 p = R.rec[3 * g];
        mn[0] = fminf(mn[0], p.x); mn[1] = fminf(mn[1], p.y); mn[2] = fminf(mn[2], p.z);
        mx[0] = fmaxf(mx[0], p.x); mx[1] = fmaxf(mx[1], p.y); mx[2] = fmaxf(mx[2], p.z);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        mn[c] = ro_warp_min(mn[c]);
        mx[c] = ro_warp_max(mx[c]);
    }
    if ((threadIdx.x & 31) == 0 && mn[0] <= mx[0]) {  // this warp saw a valid row
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            atomicMax(s_box + c, ~ro_ord(mn[c]));
            atomicMax(s_box + 3 + c, ro_ord(mx[c]));
        }
    }
}

// Ranks of the rows of one CTA chunk by digit, in row order (stable).  d_of(it) gives the
// digit of round it's row (kRoBins for a row past the end); rank(it, r) receives its rank
// among the chunk's rows with the same digit.  Only the first `rounds` rounds hold rows (the
// same count for the whole CTA).  On return s_run holds the chunk's digit counts.
template <typename DigitOf, typename Rank>
__device__ __forceinline__ void ro_rank_chunk(DigitOf d_of, Rank rank, int rounds, int32_t (*s_wcnt)[kRoBins],
                                              int32_t *s_run)
{
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    s_run[tid] = 0;
#pragma unroll
    for (int q = 0; q < kRoWarps; ++q) s_wcnt[q][tid] = 0;
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kRoItems; ++it) {
        if (it >= rounds) break;
        const int d = d_of(it);
        const bool valid = d < kRoBins;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int lr = __popc(peers & ((1u << lane) - 1u));
        if (valid && lr == 0) s_wcnt[w][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int r = s_run[d] + lr;
            for (int q = 0; q < w; ++q) r += s_wcnt[q][d];
            rank(it, r);
        }
        __syncthreads();
        int t = 0;
#pragma unroll
        for (int q = 0; q < kRoWarps; ++q) {
            t += s_wcnt[q][tid];
            s_wcnt[q][tid] = 0;
        }
        s_run[tid] += t;
        __syncthreads();
    }
}

// Exclusive scan of kRoBins counts in place (one entry per thread).
__device__ __forceinline__ void ro_scan_bins(int32_t *s_run, int32_t *s_warp)
{
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int v = s_run[tid];
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    int before = 0;
    for (int q = 0; q < w; ++q) before += s_warp[q];
    __syncthreads();
    s_run[tid] = before + x - v;
    __syncthreads();
}

// ---- one CTA: blocks of up to kRoChunk rows ------------------------------------------------
__global__ void __launch_bounds__(kRoThreads) k_ro_single(RoRows R, int32_t *__restrict__ perm)
{
    extern __shared__ unsigned long long ro_buf[];  // [2][kRoChunk]: key << 32 | row
    __shared__ int32_t s_wcnt[kRoWarps][kRoBins];
    __shared__ int32_t s_run[kRoBins];
    __shared__ int32_t s_warp[kRoWarps];
    __shared__ unsigned s_box[6];
    const int tid = threadIdx.x;
    const int64_t n_i = R.n_i;
    if (tid < 6) s_box[tid] = 0u;
    __syncthreads();
    ro_box_rows(R, tid, n_i, kRoThreads, s_box);
    __syncthreads();
    float lo[3], inv[3];
    ro_frame(s_box, lo, inv);
#pragma unroll
    for (int it = 0; it < kRoItems; ++it) {
        const int64_t e = (int64_t)it * kRoThreads + tid;
        if (e < n_i) ro_buf[e] = ((unsigned long long)ro_key(R, e, lo, inv) << 32) | (unsigned long long)e;
    }
    __syncthreads();
    int src = 0;
    for (int pass = 0; pass < kRoPasses; ++pass) {
        const int shift = 32 + 8 * pass;
        const unsigned long long *in = ro_buf + src * kRoChunk;
        unsigned long long *out = ro_buf + (src ^ 1) * kRoChunk;
        int32_t rk[kRoItems];
        ro_rank_chunk(
            [&](int it) {
                const int64_t e = (int64_t)it * kRoThreads + tid;
                return e < n_i ? (int)((in[e] >> shift) & 0xffu) : kRoBins;
            },
            [&](int it, int r) { rk[it] = r; }, (int)((n_i + kRoThreads - 1) / kRoThreads), s_wcnt, s_run);
        ro_scan_bins(s_run, s_warp);
#pragma unroll
        for (int it = 0; it < kRoItems; ++it) {
            const int64_t e = (int64_t)it * kRoThreads + tid;
            if (e < n_i) {
                const unsigned long long v = in[e];
                out[s_run[(int)((v >> shift) & 0xffu)] + rk[it]] = v;
            }
        }
        __syncthreads();
        src ^= 1;
    }
    const unsigned long long *fin = ro_buf + src * kRoChunk;
    for (int64_t e = tid; e < n_i; e += kRoThreads) perm[e] = (int32_t)(fin[e] & 0xffffffffull);
}

// ---- many CTAs -----------------------------------------------------------------------------
__global__ void __launch_bounds__(kRoThreads) k_ro_box(RoRows R, unsigned *__restrict__ box)
{
    __shared__ unsigned s_box[6];
    if (threadIdx.x < 6) s_box[threadIdx.x] = 0u;
    __syncthreads();
    ro_box_rows(R, (int64_t)blockIdx.x * kRoThreads + threadIdx.x, R.n_i, (int64_t)gridDim.x * kRoThreads, s_box);
    __syncthreads();
    if (threadIdx.x < 6 && s_box[threadIdx.x] != 0u) atomicMax(box + threadIdx.x, s_box[threadIdx.x]);
}

struct RoPass {
    uint32_t *key_in;         // keys of the rows in their current order (pass 0: written by its rank pass)
    const int32_t *val_in;    // rows in their current order; null = the identity (pass 0)
    uint32_t *key_out;
    int32_t *val_out;
    int32_t *rank;            // (n_i) rank of every row within its (CTA, digit)
    int32_t *hist;            // [kRoBins][ctas] digit counts, then bases
    int64_t n_i;
    int shift, ctas;
};

template <bool FIRST>
__global__ void __launch_bounds__(kRoThreads) k_ro_rank(RoPass P, RoRows R, const unsigned *__restrict__ box)
{
    __shared__ int32_t s_wcnt[kRoWarps][kRoBins];
    __shared__ int32_t s_run[kRoBins];
    const int tid = threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.x * kRoChunk;
    float lo[3] = {0.f, 0.f, 0.f}, inv[3] = {0.f, 0.f, 0.f};
    if (FIRST) ro_frame(box, lo, inv);
    // every round's digit first, so that the loads of all rounds are in flight together
    int dig[kRoItems];
#pragma unroll
    for (int it = 0; it < kRoItems; ++it) {
        const int64_t e = c0 + (int64_t)it * kRoThreads + tid;
        dig[it] = kRoBins;
        if (e < P.n_i) {
            uint32_t key;
            if (FIRST) {
                key = ro_key(R, e, lo, inv);
                P.key_in[e] = key;
            } else {
                key = P.key_in[e];
            }
            dig[it] = (int)((key >> P.shift) & 0xffu);
        }
    }
    const int64_t left = P.n_i - c0;
    const int rounds = left >= kRoChunk ? kRoItems : (int)((left + kRoThreads - 1) / kRoThreads);
    ro_rank_chunk([&](int it) { return dig[it]; },
                  [&](int it, int r) { P.rank[c0 + (int64_t)it * kRoThreads + tid] = r; }, rounds, s_wcnt, s_run);
    P.hist[(int64_t)tid * P.ctas + blockIdx.x] = s_run[tid];
}

// Exclusive scan of the m digit-major counts in place, one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_ro_scan(int32_t *__restrict__ hist, int64_t m)
{
    __shared__ int32_t s_warp[32];
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int64_t per = (m + 1023) / 1024;
    const int64_t b = (int64_t)tid * per, e = b + per < m ? b + per : m;
    int32_t sum = 0;
    for (int64_t q = b; q < e; ++q) sum += hist[q];
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    int before = 0;
    for (int q = 0; q < w; ++q) before += s_warp[q];
    int32_t run = before + x - sum;
    for (int64_t q = b; q < e; ++q) {
        const int32_t v = hist[q];
        hist[q] = run;
        run += v;
    }
}

__global__ void __launch_bounds__(kRoThreads) k_ro_scatter(RoPass P)
{
    const int64_t c0 = (int64_t)blockIdx.x * kRoChunk;
#pragma unroll 4
    for (int it = 0; it < kRoItems; ++it) {
        const int64_t e = c0 + (int64_t)it * kRoThreads + threadIdx.x;
        if (e < P.n_i) {
            const uint32_t key = P.key_in[e];
            const int d = (int)((key >> P.shift) & 0xffu);
            const int64_t pos = (int64_t)P.hist[(int64_t)d * P.ctas + blockIdx.x] + P.rank[e];
            P.key_out[pos] = key;
            P.val_out[pos] = P.val_in ? P.val_in[e] : (int32_t)e;
        }
    }
}

static size_t ro_align(size_t b) { return (b + 255) & ~(size_t)255; }

size_t roworder_scratch_bytes(int64_t n_i)
{
    if (n_i <= kRoChunk) return ro_align((size_t)n_i * 4);
    const int64_t ctas = (n_i + kRoChunk - 1) / kRoChunk;
    return 6 * ro_align((size_t)n_i * 4) + ro_align((size_t)kRoBins * ctas * 4) + ro_align(6 * sizeof(unsigned));
}

void roworder_configure()
{
    cudaFuncSetAttribute((const void *)k_ro_single, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         2 * kRoChunk * (int)sizeof(unsigned long long));
    cudaGetLastError();
}

int launch_row_order(cudaStream_t st, const void *rec, const int32_t *idx, int64_t n, int64_t n_i, void *scratch,
                     const int32_t **perm_out)
{
    RoRows R{static_cast<const float4 *>(rec), idx, n, n_i};
    char *p = static_cast<char *>(scratch);
    if (n_i <= kRoChunk) {
        int32_t *perm = reinterpret_cast<int32_t *>(p);
        k_ro_single<<<1, kRoThreads, 2 * kRoChunk * sizeof(unsigned long long), st>>>(R, perm);
        *perm_out = perm;
        return 1;
    }
    const int64_t ctas = (n_i + kRoChunk - 1) / kRoChunk;
    const size_t a = ro_align((size_t)n_i * 4);
    uint32_t *kt = reinterpret_cast<uint32_t *>(p);
    uint32_t *ka = reinterpret_cast<uint32_t *>(p + a);
    uint32_t *kb = reinterpret_cast<uint32_t *>(p + 2 * a);
    int32_t *va = reinterpret_cast<int32_t *>(p + 3 * a);
    int32_t *vb = reinterpret_cast<int32_t *>(p + 4 * a);
    int32_t *rank = reinterpret_cast<int32_t *>(p + 5 * a);
    int32_t *hist = reinterpret_cast<int32_t *>(p + 6 * a);
    unsigned *box = reinterpret_cast<unsigned *>(p + 6 * a + ro_align((size_t)kRoBins * ctas * 4));
    cudaMemsetAsync(box, 0, 6 * sizeof(unsigned), st);
    int64_t gb = (n_i + kRoThreads - 1) / kRoThreads;
    if (gb > 152 * 4) gb = 152 * 4;
    k_ro_box<<<(unsigned)gb, kRoThreads, 0, st>>>(R, box);
    // pass 0: keys into kt, (kt, rows) -> (ka, va); pass 1: -> (kb, vb); pass 2: -> (kt, va)
    uint32_t *kin[kRoPasses] = {kt, ka, kb};
    const int32_t *vin[kRoPasses] = {nullptr, va, vb};
    uint32_t *kout[kRoPasses] = {ka, kb, kt};
    int32_t *vout[kRoPasses] = {va, vb, va};
    for (int pass = 0; pass < kRoPasses; ++pass) {
        RoPass P{kin[pass], vin[pass], kout[pass], vout[pass], rank, hist, n_i, 8 * pass, (int)ctas};
        if (pass == 0)
            k_ro_rank<true><<<(unsigned)ctas, kRoThreads, 0, st>>>(P, R, box);
        else
            k_ro_rank<false><<<(unsigned)ctas, kRoThreads, 0, st>>>(P, R, box);
        k_ro_scan<<<1, 1024, 0, st>>>(hist, (int64_t)kRoBins * ctas);
        k_ro_scatter<<<(unsigned)ctas, kRoThreads, 0, st>>>(P);
    }
    *perm_out = va;
    return 1 + 3 * kRoPasses;
}

}  // namespace nbgpu
