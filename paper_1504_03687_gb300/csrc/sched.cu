// sched.cu — the time-step sorting list of Sec. 3.3.1 on the device: selection of the active
// particles of hierarchical power-of-two block steps and the O(N_i) re-sort after a step.
//
// The list holds all particle indices sorted by step, smallest first (level L descending,
// step 2^-L).  Times are integers in ticks of 2^-kTick.  With every particle of level L
// updated at each multiple of 2^-L:
//   * the next block time is T + 2^-Lmax, Lmax the largest level present;
//   * the particles active at T_new are exactly those of level >= L* = kTick - ctz(T_new),
//     so they are the prefix of the list up to the boundary of level L* (the paper's
//     boundary offsets I_off are the per-level counts kept on the host);
//   * after the step an active particle at level L takes the requested level w under the
//     block rule (w clamped to [level_min, level_max], at most one doubling, a doubling only
//     when T_new is a multiple of the doubled step, i.e. L > L*), so every new level is still
//     >= L*: only the prefix changes and it is re-sorted in place, the rest of the list
//     stays as it is.
// The re-sort is a stable counting sort over the levels (64 bins): every CTA ranks its
// chunk of the prefix per level (warp match on the level, rounds of 32 consecutive
// entries, warp offsets scanned in shared memory), a one-CTA scan turns the per-CTA counts
// into bases in list order (level descending, then CTA), and a scatter writes each entry
// to base + rank.  The order within a level is the previous list order, so the result does
// not depend on timing.  Prefixes of up to one chunk are sorted by a single CTA in place.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "nbgpu.h"
#include "nb_common.cuh"
#include "nb_kernels.cuh"
#include "nb_sched.cuh"

namespace nbgpu {

// Prefix within one chunk: rank, scan the 64 counts, scatter in place, update the levels.
__global__ void __launch_bounds__(kSortThreads) k_sort_single(SortArgs A)
{
    __shared__ int32_t s_cnt[kBins];
    __shared__ int32_t s_base[kBins];
    __shared__ int32_t s_warp[kSortWarps][kBins];
    sort_prefix_cta<kSortThreads, kSortItems>(A, s_cnt, s_base, s_warp);
}

// Multi-CTA pass 1: rank each chunk, keep (particle, level, rank), write the CTA's counts.
__global__ void __launch_bounds__(kSortThreads) k_sort_rank(SortArgs A)
{
    __shared__ int32_t s_cnt[kBins];
    __shared__ int32_t s_warp[kSortWarps][kBins];
    int32_t part[kSortItems], lev[kSortItems], rank[kSortItems];
    const int64_t c0 = (int64_t)blockIdx.x * kChunk;
    rank_chunk<kSortThreads, kSortItems>(A, c0, part, lev, rank, s_cnt, s_warp);
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t e = c0 + (int64_t)r * kSortThreads + threadIdx.x;
        if (e < A.n_act) {
            A.keep_part[e] = part[r];
            A.keep_rank[e] = rank[r];
            A.keep_lev[e] = (int8_t)lev[r];
        }
    }
    if (threadIdx.x < kBins) A.cta_count[(int64_t)blockIdx.x * kBins + threadIdx.x] = s_cnt[threadIdx.x];
}

// Multi-CTA pass 2 (one CTA): bases in list order, level descending then CTA ascending;
// cta_count is overwritten with the bases.  One thread per level, then a scan over levels.
__global__ void k_sort_scan(SortArgs A, int ctas)
{
    __shared__ int64_t s_tot[kBins];
    const int b = threadIdx.x;
    if (b < kBins) {
        int64_t acc = 0;
        for (int c = 0; c < ctas; ++c) {
            const int32_t v = A.cta_count[(int64_t)c * kBins + b];
            A.cta_count[(int64_t)c * kBins + b] = (int32_t)acc;
            acc += v;
        }
        s_tot[b] = acc;
        A.totals[b] = acc;
    }
    __syncthreads();
    if (b < kBins) {
        int64_t base = 0;
        for (int q = kBins - 1; q > b; --q) base += s_tot[q];
        for (int c = 0; c < ctas; ++c) A.cta_count[(int64_t)c * kBins + b] += (int32_t)base;
    }
}

// Multi-CTA pass 3: scatter into the list (reads only the kept copies) and set the levels.
__global__ void k_sort_scatter(SortArgs A)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < A.n_act;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / kChunk);
        const int32_t p = A.keep_part[e];
        const int L = A.keep_lev[e];
        A.list[A.cta_count[(int64_t)c * kBins + L] + A.keep_rank[e]] = p;
        A.level[p] = L;
    }
}

__global__ void k_iota(int32_t *list, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        list[i] = (int32_t)i;
}

}  // namespace nbgpu

using namespace nbgpu;

struct nb_sched {
    int device = 0;
    cudaStream_t stream = nullptr, own_stream = nullptr;
    int64_t n = 0;
    int32_t lmin = 0, lmax = 0;
    int64_t T = 0, T_new = 0, n_active = 0;
    int32_t lstar = 0;
    bool pending = false;  // nb_sched_next called, update not yet
    int64_t count[kBins] = {0};
    int32_t *list = nullptr, *level = nullptr, *want_stage = nullptr, *granted_stage = nullptr;
    int32_t *keep_part = nullptr, *keep_rank = nullptr, *bad = nullptr, *h_bad = nullptr;
    int8_t *keep_lev = nullptr;
    int32_t *cta_count = nullptr;
    // level totals: pinned host memory mapped into the device, written by the sort kernels
    // themselves (no copy to issue); totals is the device address of h_totals
    int64_t *totals = nullptr, *h_totals = nullptr;
    // device copies of count and T for device-driven block steps (allocated on first use)
    int64_t *d_count = nullptr, *d_T = nullptr;
    char err[256] = {0};
};

static nb_status sfail(nb_sched *s, nb_status st, const char *fmt, ...)
{
    if (s) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(s->err, sizeof(s->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

#define SCK(call, what)                                                                           \
    do {                                                                                          \
        cudaError_t _e = (call);                                                                  \
        if (_e != cudaSuccess) return sfail(s, NB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(_e)); \
    } while (0)

// Sort the prefix [0, n_act) (want == null: the whole list by the current levels).
static nb_status sched_sort(nb_sched *s, int64_t n_act, const int32_t *d_want, int32_t *d_granted)
{
    SortArgs A;
    A.list = s->list;
    A.level = s->level;
    A.want = d_want;
    A.granted = d_granted;
    A.n_act = n_act;
    A.lstar = s->lstar;
    A.lmin = s->lmin;
    A.lmax = s->lmax;
    A.keep_part = s->keep_part;
    A.keep_rank = s->keep_rank;
    A.keep_lev = s->keep_lev;
    A.cta_count = s->cta_count;
    A.totals = s->totals;
    A.bad = s->bad;
    A.dyn = nullptr;
    A.dev_count = nullptr;
    A.dev_T = nullptr;
    A.rec_new = nullptr;
    A.rec = nullptr;
    A.rec_u4 = 0;
    A.next = StepBegin{};
    if (n_act <= kChunk) {
        k_sort_single<<<1, kSortThreads, 0, s->stream>>>(A);
    } else {
        const int ctas = (int)((n_act + kChunk - 1) / kChunk);
        k_sort_rank<<<ctas, kSortThreads, 0, s->stream>>>(A);
        k_sort_scan<<<1, kBins, 0, s->stream>>>(A, ctas);
        int64_t g = (n_act + 255) / 256;
        if (g > 152 * 16) g = 152 * 16;
        k_sort_scatter<<<(int)g, 256, 0, s->stream>>>(A);
    }
    SCK(cudaGetLastError(), "sort launch");
    // the flag can only be raised by stored levels out of range: the initial sort's
    if (!d_want) SCK(cudaMemcpyAsync(s->h_bad, s->bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream), "copy flag");
    SCK(cudaStreamSynchronize(s->stream), "cudaStreamSynchronize");
    return NB_OK;
}

// ---- device-driven block steps (the integrator's batched loop) ---------------------------
namespace nbgpu {

bool sched_device(nb_sched *s, SchedDevice *out)
{
    if (!s || s->pending) return false;
    if (!s->d_count) {
        if (cudaMalloc(&s->d_count, kBins * sizeof(int64_t)) != cudaSuccess ||
            cudaMalloc(&s->d_T, sizeof(int64_t)) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
    }
    out->list = s->list;
    out->count = s->d_count;
    out->T = s->d_T;
    out->max_prefix = kChunk;
    return true;
}

bool sched_push(nb_sched *s)
{
    // pageable sources: the copies have taken the host words when the calls return
    return cudaMemcpyAsync(s->d_count, s->count, kBins * sizeof(int64_t), cudaMemcpyHostToDevice, s->stream) ==
               cudaSuccess &&
           cudaMemcpyAsync(s->d_T, &s->T, sizeof(int64_t), cudaMemcpyHostToDevice, s->stream) == cudaSuccess;
}

bool sched_pull(nb_sched *s)
{
    return cudaMemcpyAsync(s->count, s->d_count, kBins * sizeof(int64_t), cudaMemcpyDeviceToHost, s->stream) ==
               cudaSuccess &&
           cudaMemcpyAsync(&s->T, s->d_T, sizeof(int64_t), cudaMemcpyDeviceToHost, s->stream) == cudaSuccess &&
           cudaStreamSynchronize(s->stream) == cudaSuccess;
}

SortArgs sched_device_sort_args(nb_sched *s, const int32_t *want, const StepParams *P, const void *rec_new,
                                void *rec, int rec_bytes, const StepBegin *next)
{
    SortArgs A;
    A.list = s->list;
    A.level = s->level;
    A.want = want;
    A.granted = nullptr;
    A.n_act = 0;   // from P
    A.lstar = 0;   // from P
    A.lmin = s->lmin;
    A.lmax = s->lmax;
    A.keep_part = s->keep_part;
    A.keep_rank = s->keep_rank;
    A.keep_lev = s->keep_lev;
    A.cta_count = s->cta_count;
    A.totals = nullptr;  // the host reads the device counts after the batch instead
    A.bad = s->bad;
    A.dyn = P;
    A.dev_count = s->d_count;
    A.dev_T = s->d_T;
    A.rec_new = static_cast<const uint4 *>(rec_new);
    A.rec = static_cast<uint4 *>(rec);
    A.rec_u4 = rec_bytes / 16;
    A.next = next ? *next : StepBegin{};
    return A;
}

}  // namespace nbgpu

extern "C" {

nb_status nb_sched_init(nb_sched **out, int64_t n, const int32_t *levels, int32_t level_min, int32_t level_max,
                        int32_t device, void *stream, int32_t on_device)
{
    if (!out) return NB_ERR_ARG;
    *out = nullptr;
    if (n < 1 || n > (int64_t)INT32_MAX || !levels || level_min < 0 || level_max < level_min || level_max > kTick)
        return NB_ERR_ARG;
    if (!on_device)
        for (int64_t i = 0; i < n; ++i)
            if (levels[i] < level_min || levels[i] > level_max) return NB_ERR_ARG;
    nb_sched *s = new (std::nothrow) nb_sched();
    if (!s) return NB_ERR_OOM;
    s->device = device;
    s->n = n;
    s->lmin = level_min;
    s->lmax = level_max;
    auto bail = [&](nb_status st) {
        nb_sched_free(s);
        return st;
    };
    if (cudaSetDevice(device) != cudaSuccess) return bail(NB_ERR_CUDA);
    if (stream) {
        s->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&s->own_stream, cudaStreamNonBlocking) != cudaSuccess) return bail(NB_ERR_CUDA);
        s->stream = s->own_stream;
    }
    const int64_t chunks = (n + kChunk - 1) / kChunk;
    if (cudaMalloc(&s->list, n * 4) != cudaSuccess || cudaMalloc(&s->level, n * 4) != cudaSuccess ||
        cudaMalloc(&s->want_stage, n * 4) != cudaSuccess || cudaMalloc(&s->granted_stage, n * 4) != cudaSuccess ||
        cudaMalloc(&s->bad, 4) != cudaSuccess || cudaMallocHost(&s->h_bad, 4) != cudaSuccess ||
        cudaMalloc(&s->keep_part, n * 4) != cudaSuccess ||
        cudaMalloc(&s->keep_rank, n * 4) != cudaSuccess || cudaMalloc(&s->keep_lev, n) != cudaSuccess ||
        cudaMalloc(&s->cta_count, chunks * kBins * 4) != cudaSuccess ||
        cudaHostAlloc(&s->h_totals, kBins * sizeof(int64_t), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(&s->totals, s->h_totals, 0) != cudaSuccess) {
        cudaGetLastError();
        return bail(NB_ERR_OOM);
    }
    if (cudaMemcpyAsync(s->level, levels, n * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        s->stream) != cudaSuccess)
        return bail(NB_ERR_CUDA);
    if (cudaMemsetAsync(s->bad, 0, 4, s->stream) != cudaSuccess) return bail(NB_ERR_CUDA);
    int64_t g = (n + 255) / 256;
    k_iota<<<(int)(g > 152 * 16 ? 152 * 16 : g), 256, 0, s->stream>>>(s->list, n);
    // the initial list: all particles sorted by level (stable in the index)
    if (sched_sort(s, n, nullptr, nullptr) != NB_OK) return bail(NB_ERR_CUDA);
    if (*s->h_bad) return bail(NB_ERR_ARG);
    int64_t tot = 0;
    for (int b = 0; b < kBins; ++b) {
        s->count[b] = s->h_totals[b];
        tot += s->count[b];
        if (s->count[b] && (b < level_min || b > level_max)) return bail(NB_ERR_ARG);
    }
    if (tot != n) return bail(NB_ERR_ARG);
    *out = s;
    return NB_OK;
}

nb_status nb_sched_free(nb_sched *s)
{
    if (!s) return NB_OK;
    cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    void *p[] = {s->list,      s->level,    s->want_stage, s->granted_stage, s->keep_part,
                 s->keep_rank, s->keep_lev, s->cta_count,  s->bad,           s->d_count, s->d_T};
    for (void *q : p)
        if (q) cudaFree(q);
    if (s->h_totals) cudaFreeHost(s->h_totals);
    if (s->h_bad) cudaFreeHost(s->h_bad);
    if (s->own_stream) cudaStreamDestroy(s->own_stream);
    delete s;
    return NB_OK;
}

nb_status nb_sched_next(nb_sched *s, double *t_block, int64_t *n_active, const int32_t **d_list)
{
    if (!s || !t_block || !n_active) return NB_ERR_ARG;
    if (s->pending) return sfail(s, NB_ERR_STATE, "nb_sched_next twice without nb_sched_update");
    int lmax_present = -1;
    for (int b = kBins - 1; b >= 0; --b)
        if (s->count[b]) {
            lmax_present = b;
            break;
        }
    const int64_t T_new = s->T + ((int64_t)1 << (kTick - lmax_present));
    if (T_new <= s->T || T_new >= ((int64_t)1 << 62)) return sfail(s, NB_ERR_STATE, "block time out of range");
    int tz = 0;
    while (((T_new >> tz) & 1) == 0) ++tz;
    int lstar = kTick - tz;
    if (lstar < 0) lstar = 0;
    int64_t na = 0;
    for (int b = lstar; b < kBins; ++b) na += s->count[b];
    s->T_new = T_new;
    s->lstar = lstar;
    s->n_active = na;
    s->pending = true;
    *t_block = std::ldexp((double)T_new, -kTick);
    *n_active = na;
    if (d_list) *d_list = s->list;
    return NB_OK;
}

nb_status nb_sched_update(nb_sched *s, const int32_t *want, int32_t *granted, int32_t on_device)
{
    if (!s) return NB_ERR_ARG;
    if (!s->pending) return sfail(s, NB_ERR_STATE, "nb_sched_update without nb_sched_next");
    if (!want) return sfail(s, NB_ERR_ARG, "null want");
    if (cudaSetDevice(s->device) != cudaSuccess) return sfail(s, NB_ERR_CUDA, "cudaSetDevice");
    const int32_t *d_want = want;
    int32_t *d_granted = granted;
    if (!on_device) {
        SCK(cudaMemcpyAsync(s->want_stage, want, s->n_active * 4, cudaMemcpyHostToDevice, s->stream), "copy want");
        d_want = s->want_stage;
        d_granted = granted ? s->granted_stage : nullptr;
    }
    nb_status st = sched_sort(s, s->n_active, d_want, d_granted);
    if (st == NB_OK && !on_device && granted)
        SCK(cudaMemcpy(granted, s->granted_stage, s->n_active * 4, cudaMemcpyDeviceToHost), "copy granted");
    if (st != NB_OK) return st;
    for (int b = s->lstar; b < kBins; ++b) s->count[b] = s->h_totals[b];
    s->T = s->T_new;
    s->pending = false;
    return NB_OK;
}

nb_status nb_sched_get(nb_sched *s, int32_t *list, int32_t *levels, double *t_now, int32_t on_device)
{
    if (!s) return NB_ERR_ARG;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (list) SCK(cudaMemcpyAsync(list, s->list, s->n * 4, k, s->stream), "copy list");
    if (levels) SCK(cudaMemcpyAsync(levels, s->level, s->n * 4, k, s->stream), "copy levels");
    if (t_now) *t_now = std::ldexp((double)s->T, -kTick);
    SCK(cudaStreamSynchronize(s->stream), "cudaStreamSynchronize");
    return NB_OK;
}

nb_status nb_sched_counts(const nb_sched *s, int64_t *counts)
{
    if (!s || !counts) return NB_ERR_ARG;
    for (int b = 0; b < kBins; ++b) counts[b] = s->count[b];
    return NB_OK;
}

nb_status nb_sched_set_time(nb_sched *s, double t)
{
    if (!s) return NB_ERR_ARG;
    if (s->pending) return sfail(s, NB_ERR_STATE, "a block step is open");
    const double ticks = std::ldexp(t, kTick);
    if (!(t >= 0.0) || ticks >= std::ldexp(1.0, 62) || ticks != std::floor(ticks))
        return sfail(s, NB_ERR_ARG, "time %.17g is not a multiple of 2^-%d in range", t, kTick);
    const int64_t T = (int64_t)ticks;
    // a block time is a multiple of the smallest step present (its particles step every time)
    int lmax_present = 0;
    for (int b = kBins - 1; b >= 0; --b)
        if (s->count[b]) {
            lmax_present = b;
            break;
        }
    if ((T & (((int64_t)1 << (kTick - lmax_present)) - 1)) != 0)
        return sfail(s, NB_ERR_ARG, "time %.17g is not a multiple of the smallest step 2^-%d", t, lmax_present);
    s->T = T;
    return NB_OK;
}

nb_status nb_sched_peek(const nb_sched *s, double *t_next)
{
    if (!s || !t_next) return NB_ERR_ARG;
    int lmax_present = -1;
    for (int b = kBins - 1; b >= 0; --b)
        if (s->count[b]) {
            lmax_present = b;
            break;
        }
    if (lmax_present < 0) return NB_ERR_STATE;
    *t_next = std::ldexp((double)(s->T + ((int64_t)1 << (kTick - lmax_present))), -kTick);
    return NB_OK;
}

const char *nb_sched_last_error(const nb_sched *s) { return s ? s->err : "null scheduler"; }

}  // extern "C"
