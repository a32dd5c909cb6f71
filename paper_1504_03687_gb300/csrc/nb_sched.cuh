// nb_sched.cuh — the per-CTA pieces of the time-step sorting list's re-sort (Sec. 3.3.1):
// ranking a chunk of the list prefix by the granted levels, and the whole re-sort of a prefix
// that fits one CTA.  Shared by the scheduler's sort kernels (sched.cu, 1024 threads) and the
// integrator's fused block-step kernel (ac.cu), whose last CTA re-sorts the step's prefix.
#pragma once

#include "nb_common.cuh"
#include "nb_kernels.cuh"

namespace nbgpu {

constexpr int kTick = 48;        // time unit 2^-48
constexpr int kBins = 64;        // level bins
constexpr int kSortThreads = 1024;
constexpr int kSortItems = 16;   // rounds of 32 entries per warp
constexpr int kChunk = kSortThreads * kSortItems;  // entries per CTA of the scheduler's sorts (16384)
constexpr int kSortWarps = kSortThreads / 32;

struct SortArgs {
    int32_t *list;          // the list; the prefix [0, n_act) is re-sorted
    int32_t *level;         // (n) level of every particle
    const int32_t *want;    // (n_act) requested levels in list order, or null (initial sort)
    int32_t *granted;       // (n_act) optional: the granted levels in list order
    int64_t n_act;
    int32_t lstar, lmin, lmax;
    int32_t *keep_part;     // multi-CTA: particle of every entry
    int32_t *keep_rank;     // multi-CTA: rank of every entry within its CTA and level
    int8_t *keep_lev;       // multi-CTA: new level of every entry
    int32_t *cta_count;     // [ctas][kBins]
    int64_t *totals;        // [kBins] entries per new level (written by the scan)
    int32_t *bad;           // set when a stored level is outside [0, kBins) (initial sort)
    const StepParams *dyn;  // device-driven step: n_act and lstar from here (nothing when halted)
    int64_t *dev_count;     // device-driven step: the device counts of levels >= lstar are set
    int64_t *dev_T;         // ... and the device time advanced to the step's block time
    const uint4 *rec_new;   // optional (single CTA): records of the prefix in list order, copied ...
    uint4 *rec;             // ... to rec[particle] before the re-sort; rec_u4 (<= 8) 16-byte words each
    int32_t rec_u4;
    StepBegin next;         // optional (device-driven, next.P set): the following step's begin
};

// One CTA of THREADS threads: read its chunk of the prefix (ITEMS rounds of THREADS
// entries), apply the block rule, and rank every entry within (CTA, new level) in list order.
// Entry e of the chunk is handled in round e / THREADS by warp (e % THREADS) / 32, lane e % 32;
// the rank counts earlier rounds of all warps, then earlier warps of the same round, then
// earlier lanes.  With REC, each entry's new record (A.rec_new) is copied to its particle.
// Returns the per-level counts in s_cnt.
template <int THREADS, int ITEMS, bool REC = false>
__device__ void rank_chunk(const SortArgs &A, int64_t c0, int32_t (&part)[ITEMS], int32_t (&lev)[ITEMS],
                           int32_t (&rank)[ITEMS], int32_t *s_cnt, int32_t (*s_warp)[kBins])
{
    constexpr int WARPS = THREADS / 32;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int b = tid; b < kBins; b += THREADS) s_cnt[b] = 0;
    const unsigned lt = (1u << lane) - 1u;
    // rounds past the end of the prefix hold no entry (the same count for the whole CTA)
    const int64_t left = A.n_act - c0;
    const int rounds = left >= (int64_t)THREADS * ITEMS ? ITEMS : (int)((left + THREADS - 1) / THREADS);
    __syncthreads();  // s_cnt is zeroed
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
        part[r] = -1;
        lev[r] = 0;
        rank[r] = 0;
        if (r >= rounds) continue;  // the same for the whole CTA
        const int64_t e = c0 + (int64_t)r * THREADS + tid;
        const bool in = e < A.n_act;
        int32_t p = -1, L = 0;
        if (in) {
            // every load of the entry before its stores: a store would hold the later loads
            // behind it (the compiler cannot tell the arrays apart)
            p = A.list[e];
            L = A.level[p];
            const int32_t g0 = A.want ? A.want[e] : 0;
            uint4 q[REC ? 8 : 1];
            if constexpr (REC)
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (u < A.rec_u4) q[u] = A.rec_new[e * A.rec_u4 + u];
            if (L < 0 || L >= kBins) {  // only possible for levels handed to the initial sort
                atomicOr(A.bad, 1);
                L = L < 0 ? 0 : kBins - 1;
            }
            if (A.want) {
                int32_t g = g0 < A.lmin ? A.lmin : (g0 > A.lmax ? A.lmax : g0);
                if (g < L - 1) g = L - 1;
                if (g == L - 1 && L <= A.lstar) g = L;
                L = g;
                if (A.granted) A.granted[e] = g;
            }
            if constexpr (REC)  // the entry's new record, read whole above
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (u < A.rec_u4) A.rec[(int64_t)p * A.rec_u4 + u] = q[u];
        }
        part[r] = p;
        lev[r] = L;
        const int key = in ? L : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        // per-warp count of this round per level, then offsets across the warps
        for (int b = lane; b < kBins; b += 32) s_warp[w][b] = 0;
        __syncwarp();
        if (in && (peers & lt) == 0) s_warp[w][L] = __popc(peers);
        __syncthreads();
        // exclusive scan over warps, per level (one thread per level)
        if (tid < kBins) {
            int acc = s_cnt[tid];
            for (int ww = 0; ww < WARPS; ++ww) {
                const int c = s_warp[ww][tid];
                s_warp[ww][tid] = acc;
                acc += c;
            }
            s_cnt[tid] = acc;
        }
        __syncthreads();
        rank[r] = in ? s_warp[w][L] + __popc(peers & lt) : 0;
        __syncthreads();  // s_warp is rewritten in the next round
    }
}

// The re-sort of a prefix of at most THREADS * ITEMS entries by one CTA: rank, scan the 64
// counts, scatter in place, update the levels; for a device-driven step (STEP: A.dyn, A.rec
// and A.rec_new set) also the new records, the device counts and time and, with A.next.P, the
// begin of the following step.  A.n_act and A.lstar are the step's.  THREADS >= 64.
template <int THREADS, int ITEMS, bool STEP = false>
__device__ void sort_prefix_cta(const SortArgs &A, int32_t *s_cnt, int32_t *s_base, int32_t (*s_warp)[kBins])
{
    static_assert(THREADS >= kBins, "one thread per level");
    // the next step's begin reads the counts of the levels this step leaves alone, the
    // regular-level histogram and the budget: requested now, used at the end
    const bool begin = STEP && A.next.P && threadIdx.x < 32;
    int64_t old_lo = 0, old_hi = 0;
    StepBeginIn bin{};
    if (begin) {
        old_lo = A.dev_count[threadIdx.x];
        old_hi = A.dev_count[threadIdx.x + 32];
        bin = step_begin_inputs(A.next, threadIdx.x);
    }
    int32_t part[ITEMS], lev[ITEMS], rank[ITEMS];
    rank_chunk<THREADS, ITEMS, STEP>(A, 0, part, lev, rank, s_cnt, s_warp);
    if (threadIdx.x < 32) {  // bases in list order (level descending): an exclusive warp scan
        const int l = threadIdx.x;
        const int32_t v_hi = s_cnt[63 - l], v_lo = s_cnt[31 - l];  // levels 63..32, then 31..0
        int32_t in_hi = v_hi, in_lo = v_lo;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t u_hi = __shfl_up_sync(0xffffffffu, in_hi, o), u_lo = __shfl_up_sync(0xffffffffu, in_lo, o);
            if (l >= o) {
                in_hi += u_hi;
                in_lo += u_lo;
            }
        }
        const int32_t tot_hi = __shfl_sync(0xffffffffu, in_hi, 31);
        s_base[63 - l] = in_hi - v_hi;
        s_base[31 - l] = tot_hi + in_lo - v_lo;
    }
    if (A.totals && threadIdx.x < kBins) A.totals[threadIdx.x] = s_cnt[threadIdx.x];
    if constexpr (STEP) {  // the scheduler's device state moves on to the step's block time
        if (threadIdx.x < kBins && threadIdx.x >= A.lstar) A.dev_count[threadIdx.x] = s_cnt[threadIdx.x];
        if (threadIdx.x == 0) *A.dev_T = A.dyn->t_ticks;
    }
    __syncthreads();  // every entry is in registers: the in-place scatter is safe
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
        if (part[r] < 0) continue;
        A.list[s_base[lev[r]] + rank[r]] = part[r];
        A.level[part[r]] = lev[r];
    }
    if (begin) {  // the next step's begin on the new counts
        const int l = threadIdx.x;
        const int64_t c_lo = l >= A.lstar ? (int64_t)s_cnt[l] : old_lo;
        const int64_t c_hi = l + 32 >= A.lstar ? (int64_t)s_cnt[l + 32] : old_hi;
        step_begin(A.next, c_lo, c_hi, A.dyn->t_ticks, l, bin);
    }
}

// The arguments of a device-driven step's re-sort (the scheduler's list, levels, bounds and
// device state), for a kernel that re-sorts the prefix itself with sort_prefix_cta.
SortArgs sched_device_sort_args(::nb_sched *s, const int32_t *want, const StepParams *P, const void *rec_new,
                                void *rec, int rec_bytes, const StepBegin *next);

}  // namespace nbgpu
