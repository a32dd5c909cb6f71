// nb_api.cu — the context part of the C ABI declared in include/nbgpu.h: the context and
// its device buffers, validation, launch planning (automatic, override or tuned table), and
// the call sequences:
//   nb_predict            : K1 predictor -> j-records
//   nb_regular_force      : K2/K3 force (+ neighbour capture, optional source range)
//                           -> K4 reduce -> K5 neighbour CSR
//   nb_regular_force_backward : K6 adjoint passes
//   nb_batch_plan / nb_regular_force_batched : the persistent ensemble launch
//   nb_irregular_force    : state or predicted records -> K10 list sums (+ split)
// plus per-phase timing, the deferred device status and the fault-injection hook.  The
// scheduler (sched.cu), the AC integrator (ac.cu) and the allocation-free call (noalloc.cu)
// have their own files.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <initializer_list>

#include "nbgpu.h"
#include "nb_common.cuh"
#include "nb_kernels.cuh"

using namespace nbgpu;

namespace nbgpu {
void *mixed_tiled_fn(int v);
int mixed_tiled_i_per_cta(int v);
int mixed_tiled_block(int v);
int mixed_tiled_tj(int v);
int mixed_jstream_ib(int v);
int jstream_warps();
int mixed_tiled_dyn_smem(int v);
int mixed_tiled_anchored(int v);
void mixed_tiled_configure();
int mixed_batched_rows_per_item(int v);
int mixed_batched_variants();
int mixed_batched_occupancy(int v);
void launch_force_mixed_batched(cudaStream_t st, int variant, int ctas, const BatchArgs &a);
void *fp64_tiled_fn();
int fp64_jstream_ib(int v);
void launch_force_mixed(cudaStream_t st, int kernel, int variant, int64_t ctas_x, int S, ForceArgs a);
void launch_force_fp64(cudaStream_t st, int kernel, int variant, int64_t ctas_x, int S, ForceArgs a);
void adjoint_configure();
size_t adjoint_scratch_bytes(int precision, int64_t n, int64_t n_i, int num_sms, int64_t *rows_pad_out, int *SA,
                             int *SB);
int launch_adjoint(cudaStream_t st, int precision, const void *rec, int64_t n, const int32_t *idx, int64_t n_i,
                   const double *g_acc, const double *g_jerk, const double *g_pot, double *g_x, double *g_v,
                   double *g_m, void *scratch, unsigned *status, int num_sms);
}  // namespace nbgpu

static constexpr int kTilePad = 256;   // j-record arrays are padded to a multiple of this
static constexpr int kMixedTiledVariants = 20;  // entries of the mixed tiled variant table
static constexpr int kOccFp64 = 20;             // occupancy slot of the FP64 tiled kernel
static constexpr int kOccSlots = 21;
static_assert(kOccSlots == kMixedTiledVariants + 1, "one occupancy slot per mixed tiled variant, then the FP64 kernel");
static constexpr int kMaxCap = 8192;   // largest nb_cap (sort buffers live in shared memory)
// Irregular force: predict all particles once when N_i * factor >= N.  Measured on this GPU
// (King cluster, N = 2^20, r_s for a median of 80 neighbours): in FP64 the per-pair prediction
// (25 FP64 operations) makes predict-all pay already at N/128 active rows; in mixed precision
// the 80-byte state gathers only lose to one full predictor pass above about N/8.
static constexpr int64_t kIrrAllFactorFp64 = 128;
static constexpr int64_t kIrrAllFactorMixed = 8;

struct nb_ctx {
    int device = 0, precision = 0, cap = 0, num_sms = 0;
    int occ[kOccSlots] = {0};  // resident CTAs per SM of every planned kernel variant
    int force_kernel = -1, force_variant = 0, force_splits = 0;  // plan override (-1: none)
    struct TableEntry {
        int64_t ni_max;
        int kernel, variant, splits;
    };
    std::vector<TableEntry> table;  // tuned plans by active-block size (nb_set_plan_table)
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    int64_t n_max = 0, n = 0, n_pad = 0;
    int64_t src_lo = 0, src_hi = 0;  // source range of nb_regular_force (src_hi 0: all particles)
    bool have_state = false, have_pred = false, broken = false;
    double *x = nullptr, *v = nullptr, *a = nullptr, *jk = nullptr, *m = nullptr, *tl = nullptr;
    double *xp = nullptr, *vp = nullptr;
    void *rec = nullptr;  // dvec4[2*n_pad] or float4[3*n_pad]
    unsigned *status = nullptr;
    // grow-only scratch
    double *part = nullptr; size_t part_cap = 0;
    int32_t *seg_slots = nullptr; size_t seg_slots_cap = 0;
    int32_t *seg_cnt = nullptr; size_t seg_cnt_cap = 0;
    int32_t *row_total = nullptr; size_t row_total_cap = 0;
    int64_t *scan = nullptr; size_t scan_cap = 0;
    char *stage = nullptr; size_t stage_cap = 0;
    char *adj = nullptr; size_t adj_cap = 0;
    void *srec = nullptr; size_t srec_cap = 0;  // Hermite-state records of the irregular force
    bool srec_valid = false;
    void *prec = nullptr; size_t prec_cap = 0;  // predicted j-records of its predict-all form
    // batched ensemble plan (nb_batch_plan)
    void *b_items = nullptr; size_t b_items_cap = 0;
    int64_t *b_cluster_off = nullptr; size_t b_cluster_off_cap = 0;
    void *ro = nullptr; size_t ro_cap = 0;  // row order of the anchored force kernel
    int64_t b_clusters = 0, b_rows = 0, b_items_n = 0, b_n = 0;
    int b_variant = -1, b_ctas = 0, b_L = 0;
    char err[512] = {0};
    // per-phase device timing (CUDA events on the context stream) and launch counters
    bool timing = false;
    struct Span {
        cudaEvent_t a, b;
        int phase;
    };
    std::vector<Span> spans;
    std::vector<cudaEvent_t> evpool;
    int64_t launches[NB_PHASES] = {0};  // kernels launched per phase since nb_get_timings
    // test hook (nb_inject_fault / NB_FAULT): the operation of kind fault_kind that comes
    // after fault_after more of its kind reports the failure the CUDA runtime would
    int fault_kind = 0, fault_after = 0;
};

enum { PH_PREDICT = 0, PH_FORCE = 1, PH_REDUCE = 2, PH_NEIGHBOURS = 3, PH_BACKWARD = 4, PH_IRREGULAR = 5, PH_ORDER = 6,
       PH_COUNT = 7 };
static_assert(PH_COUNT == NB_PHASES, "one timing phase per NB_PHASES entry");

static cudaEvent_t ev_take(nb_ctx *c)
{
    if (!c->evpool.empty()) {
        cudaEvent_t e = c->evpool.back();
        c->evpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

static cudaEvent_t span_begin(nb_ctx *c)
{
    if (!c->timing) return nullptr;
    cudaEvent_t a = ev_take(c);
    if (a) cudaEventRecord(a, c->stream);
    return a;
}

static void span_end(nb_ctx *c, int phase, cudaEvent_t a, int kernels)
{
    c->launches[phase] += kernels;
    if (!c->timing || !a) return;
    cudaEvent_t b = ev_take(c);
    if (!b) return;
    cudaEventRecord(b, c->stream);
    c->spans.push_back({a, b, phase});
}

// ------------------------------------------------------------------------------ helpers
static nb_status fail(nb_ctx *c, nb_status s, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

static nb_status cuda_fail(nb_ctx *c, cudaError_t e, const char *what)
{
    if (c) {
        snprintf(c->err, sizeof(c->err), "%s: %s", what, cudaGetErrorString(e));
        // errors that poison the context are sticky
        if (e != cudaErrorMemoryAllocation && e != cudaErrorInvalidValue) c->broken = true;
    }
    return e == cudaErrorMemoryAllocation ? NB_ERR_OOM : NB_ERR_CUDA;
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t _e = (call);                        \
        if (_e != cudaSuccess) return cuda_fail(c, _e, what); \
    } while (0)

#define CK_LAUNCH(what) CK(cudaGetLastError(), what)

// Simulated runtime failure for the fault-injection hook: true once, when the armed kind's
// countdown reaches zero.  Nothing touches the GPU.
static bool take_fault(nb_ctx *c, int kind)
{
    if (!c || c->fault_kind != kind) return false;
    if (c->fault_after-- > 0) return false;
    c->fault_kind = 0;
    return true;
}

static cudaError_t ctx_sync(nb_ctx *c)
{
    if (take_fault(c, NB_FAULT_SYNC)) return cudaErrorLaunchFailure;
    return cudaStreamSynchronize(c->stream);
}

static nb_status grow(nb_ctx *c, void **p, size_t *cap, size_t need_bytes, const char *what)
{
    if (need_bytes <= *cap && *p) return NB_OK;
    if (*p) {
        // the old buffer may still be read by queued work
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
        cudaFree(*p);
        *p = nullptr;
        *cap = 0;
    }
    size_t bytes = need_bytes < 256 ? 256 : need_bytes;
    bytes = bytes + bytes / 4;  // headroom to avoid regrowth on small changes
    cudaError_t e = take_fault(c, NB_FAULT_ALLOC) ? cudaErrorMemoryAllocation : cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(c, e, what);
    }
    *cap = bytes;
    return NB_OK;
}

static nb_status check_usable(nb_ctx *c)
{
    if (!c) return NB_ERR_ARG;
    if (c->broken) return fail(c, NB_ERR_STATE, "context unusable after an earlier CUDA error: %s", c->err);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return NB_OK;
}

static nb_status status_from_flags(nb_ctx *c, unsigned f)
{
    if (f & ST_BAD_INDEX)
        return fail(c, NB_ERR_ARG, "an active or neighbour index was outside [0, n), or CSR offsets decreased");
    if (f & ST_DUP_INDEX) return fail(c, NB_ERR_ARG, "an active index appears more than once");
    if (f & ST_TIMEOUT) return fail(c, NB_ERR_TIMEOUT, "a bounded device-side wait expired");
    if (f & ST_DEVICE) return fail(c, NB_ERR_DEVICE, "a device-side consistency check failed");
    if (f & ST_CSR_FULL) return fail(c, NB_ERR_NB_OVERFLOW, "neighbour CSR capacity too small; lists cut");
    if (f & ST_NB_TRUNCATED) return fail(c, NB_ERR_NB_OVERFLOW, "some neighbour lists were cut at nb_cap");
    return NB_OK;
}

static nb_status sync_and_collect(nb_ctx *c)
{
    CK(ctx_sync(c), "cudaStreamSynchronize");
    unsigned f = 0;
    CK(take_fault(c, NB_FAULT_STATUS) ? cudaErrorUnknown
                                      : cudaMemcpy(&f, c->status + SS_FLAGS, sizeof(unsigned), cudaMemcpyDeviceToHost),
       "read status");
    CK(cudaMemset(c->status + SS_FLAGS, 0, sizeof(unsigned)), "clear status");
    return status_from_flags(c, f);
}

// ------------------------------------------------------------------------------ planner
namespace nbgpu {

static double wave_eff(int64_t ctas, int64_t P)
{
    if (P <= 0) return 1.0;
    const int64_t waves = (ctas + P - 1) / P;
    return (double)ctas / (double)(waves * P);
}

// Picks the kernel, its variant and the j-split S.  Tiny active blocks take the j-streamed
// kernel (every CTA streams a contiguous j-chunk for a few i); larger ones the tiled kernel,
// with S chosen so that the CTA count fills whole waves of the GPU (each split must keep at
// least two j-tiles).  Relative per-pair speed of the tiled variants weights the choice.
// Splits whose neighbour slot arrays (S x n_i x min(nb_cap, split length) int32) would
// exceed kSlotBudget are not considered (S = 1 always is).
static constexpr double kSlotBudget = 6.0e9;

static void jstream_segments(Plan &p, int64_t n)
{
    const int W = jstream_warps();
    p.segs_per_split = W;
    const int64_t chunk = (n + p.S - 1) / p.S;
    p.seg_len = (chunk + W - 1) / W + 1;
}

static Plan plan_force_variant(int precision, int num_sms, const int *occ, int64_t n, int64_t n_i, int nb_cap,
                               int only_variant);

Plan plan_force(int precision, int num_sms, const int *occ, int64_t n, int64_t n_i, int nb_cap)
{
    return plan_force_variant(precision, num_sms, occ, n, n_i, nb_cap, -1);
}

// only_variant >= 0 restricts the tiled search to that mixed variant (and always takes the
// tiled kernel).
static Plan plan_force_variant(int precision, int num_sms, const int *occ, int64_t n, int64_t n_i, int nb_cap,
                               int only_variant)
{
    Plan p{};
    if (num_sms <= 0) num_sms = 152;
    const int64_t n_pad = ((n + kTilePad - 1) / kTilePad) * kTilePad;
    if (precision == NB_MIXED) {
        if (n_i <= 32 && only_variant < 0) {
            // one row a CTA up to two rows, then the packed forms: two rows a CTA (three CTAs an
            // SM) up to 16 rows, four rows a CTA above (measured on a GB300, King W0 = 6, 2^20)
            p.kernel = 2;
            p.variant = n_i <= 2 ? 0 : (n_i <= 16 ? 3 : 1);
            p.i_per_cta = mixed_jstream_ib(p.variant);
            const int64_t batches = (n_i + p.i_per_cta - 1) / p.i_per_cta;
            const int64_t per_sm = p.variant == 3 ? 3 : 4;
            int64_t S = (per_sm * (int64_t)num_sms + batches - 1) / batches;
            const int64_t smax = n / 2048 > 1 ? n / 2048 : 1;  // >= 2048 j per CTA
            if (S > smax) S = smax;
            if (S < 1) S = 1;
            p.S = (int)S;
            p.ctas = batches * S;
            p.tj = 0;
            jstream_segments(p, n);
            return p;
        }
        // relative per-pair speed of the tiled variants (scalar NI=4/2/1, NI=4 x 256 threads,
        // packed FP32x2 NI=4/2, NI=4 with 128-j tiles, NI=2 x 256 threads), measured on a
        // GB300 at N = 2^20, N_i = 2^17 (King W0 = 6); the two small-tile packed variants
        // (NI=2 x 64 and x 32 threads) estimated from their occupancy; the anchored variants
        // measured the same way (10-12) or estimated (13, 14: the small-tile packed ones x 1.1;
        // 15-19: the staged-hit forms of 10-12, measured)
        static const double speed[kMixedTiledVariants] = {0.81, 0.87, 0.71, 0.76, 0.99, 0.92, 1.0, 0.91, 0.85,
                                                           0.75, 1.12, 1.08, 1.125, 0.94, 0.82, 1.107, 1.06, 1.027, 1.111, 1.036};
        double best = -1.0;
        for (int v = 0; v < kMixedTiledVariants; ++v) {
            if (only_variant >= 0 && v != only_variant) continue;
            const int ipc = mixed_tiled_i_per_cta(v), tj = mixed_tiled_tj(v);
            const int64_t tiles = n_pad / tj;
            const int64_t itiles = (n_i + ipc - 1) / ipc;
            const int64_t P = (int64_t)num_sms * (occ && occ[v] > 0 ? occ[v] : 1);
            const double util = (double)n_i / (double)(itiles * ipc);
            int64_t smax = tiles / 2 > 1 ? tiles / 2 : 1;
            if (smax > 2048) smax = 2048;
            for (int64_t S = 1; S <= smax; ++S) {
                const int64_t ctas = itiles * S;
                const int64_t seg = (tiles + S - 1) / S * tj;
                const double slots = (double)S * (double)n_i * (double)(seg < nb_cap ? seg : nb_cap) * 4.0;
                if (S > 1 && slots > kSlotBudget) break;
                // a split costs one partial-sum write per i; penalise many splits slightly
                const double score = speed[v] * util * wave_eff(ctas, P) * (1.0 - 0.0005 * (double)S);
                if (score > best + 1e-12) {
                    best = score;
                    p.kernel = 1;
                    p.variant = v;
                    p.i_per_cta = ipc;
                    p.S = (int)S;
                    p.ctas = ctas;
                    p.tj = tj;
                    p.segs_per_split = 1;
                    p.seg_len = seg;
                }
                if (ctas >= 64 * P) break;
            }
        }
        return p;
    }
    // FP64
    if (n_i <= 64) {
        p.kernel = 3;
        p.variant = n_i <= 4 ? 0 : 1;
        p.i_per_cta = fp64_jstream_ib(p.variant);
        const int64_t batches = (n_i + p.i_per_cta - 1) / p.i_per_cta;
        int64_t S = (4 * (int64_t)num_sms + batches - 1) / batches;
        const int64_t smax = n / 1024 > 1 ? n / 1024 : 1;
        if (S > smax) S = smax;
        if (S < 1) S = 1;
        p.S = (int)S;
        p.ctas = batches * S;
        p.tj = 0;
        jstream_segments(p, n);
        return p;
    }
    const int ipc = 128, tj = 64;
    const int64_t tiles = n_pad / tj;
    const int64_t itiles = (n_i + ipc - 1) / ipc;
    const int64_t P = (int64_t)num_sms * (occ && occ[kOccFp64] > 0 ? occ[kOccFp64] : 1);
    int64_t smax = tiles / 2 > 1 ? tiles / 2 : 1;
    if (smax > 2048) smax = 2048;
    double best = -1.0;
    for (int64_t S = 1; S <= smax; ++S) {
        const int64_t ctas = itiles * S;
        const int64_t seg = (tiles + S - 1) / S * tj;
        const double slots = (double)S * (double)n_i * (double)(seg < nb_cap ? seg : nb_cap) * 4.0;
        if (S > 1 && slots > kSlotBudget) break;
        const double score = wave_eff(ctas, P) * (1.0 - 0.0005 * (double)S);
        if (score > best + 1e-12) {
            best = score;
            p.kernel = 0;
            p.variant = 0;
            p.i_per_cta = ipc;
            p.S = (int)S;
            p.ctas = ctas;
            p.tj = tj;
            p.segs_per_split = 1;
            p.seg_len = seg;
        }
        if (ctas >= 64 * P) break;
    }
    return p;
}

void query_occupancy(int *occ)
{
    mixed_tiled_configure();
    roworder_configure();
    adjoint_configure();
    for (int v = 0; v < kMixedTiledVariants; ++v) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, mixed_tiled_fn(v), mixed_tiled_block(v),
                                                          (size_t)mixed_tiled_dyn_smem(v)) != cudaSuccess)
            b = 1;
        occ[v] = b > 0 ? b : 1;
    }
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fp64_tiled_fn(), 128, 0) != cudaSuccess) b = 1;
    occ[kOccFp64] = b > 0 ? b : 1;
    cudaGetLastError();
}

// A forced plan (autotuning and benchmarking of individual variants): kernel < 0 = none.
static Plan forced_plan(int precision, int num_sms, const int *occ, int64_t n, int64_t n_i, int nb_cap,
                        int kernel, int variant, int splits)
{
    if (kernel == 1 && splits <= 0 && precision == NB_MIXED)  // forced variant, automatic splits
        return plan_force_variant(precision, num_sms, occ, n, n_i, nb_cap, variant);
    Plan p = plan_force(precision, num_sms, occ, n, n_i, nb_cap);
    if (kernel < 0) return p;
    const int64_t n_pad = ((n + kTilePad - 1) / kTilePad) * kTilePad;
    p.kernel = kernel;
    p.variant = variant;
    if (kernel == 1) {
        p.i_per_cta = mixed_tiled_i_per_cta(variant);
        p.tj = mixed_tiled_tj(variant);
    } else if (kernel == 0) {
        p.i_per_cta = 128;
        p.tj = 64;
    } else {
        p.i_per_cta = kernel == 2 ? mixed_jstream_ib(variant) : fp64_jstream_ib(variant);
        p.tj = 0;
    }
    int64_t S = splits > 0 ? splits : 1;
    if (splits <= 0 && p.tj == 0) {  // j-streamed kernel, automatic splits: ~4 CTAs per SM (3 for the
                                     // two-row packed form, which fits three)
        const int64_t batches = (n_i + p.i_per_cta - 1) / p.i_per_cta;
        const int64_t per_sm = (kernel == 2 && variant == 3) ? 3 : 4;
        S = (per_sm * (int64_t)(num_sms > 0 ? num_sms : 152) + batches - 1) / (batches > 0 ? batches : 1);
        const int64_t per = kernel == 2 ? 2048 : 1024;
        const int64_t smax = n / per > 1 ? n / per : 1;
        if (S > smax) S = smax;
        if (S < 1) S = 1;
    }
    if (p.tj > 0) {
        const int64_t tiles = n_pad / p.tj;
        if (S > tiles) S = tiles;
        p.segs_per_split = 1;
        p.seg_len = (tiles + S - 1) / S * p.tj;
    } else {
        if (S > n) S = n;
    }
    p.S = (int)S;
    p.ctas = (n_i + p.i_per_cta - 1) / p.i_per_cta * S;
    if (p.tj == 0) jstream_segments(p, n);
    return p;
}

void launch_force(cudaStream_t st, const Plan &p, ForceArgs a)
{
    const int64_t ctas_x = p.ctas / p.S;
    a.S = p.S;
    // records past n are massless padding up to the next multiple of kTilePad
    const int64_t hi_pad = ((a.j_hi + kTilePad - 1) / kTilePad) * kTilePad;
    a.n_tiles = p.tj > 0 ? (hi_pad - a.j_lo) / p.tj : 0;
    if (p.kernel == 1 || p.kernel == 2)
        launch_force_mixed(st, p.kernel, p.variant, ctas_x, p.S, a);
    else
        launch_force_fp64(st, p.kernel, p.variant, ctas_x, p.S, a);
}

}  // namespace nbgpu

namespace nbgpu {
bool ctx_state(nb_ctx *c, CtxState *o)
{
    if (!c || c->broken || !c->have_state) return false;
    *o = CtxState{c->x, c->v, c->a, c->jk, c->tl, c->m, c->xp, c->vp, c->rec, c->status, c->stream,
                  c->precision, c->cap, c->num_sms, c->device, c->n, c->n_pad};
    return true;
}

// The state arrays were rewritten in place (by the integrator): what the context derived from
// them (the state records of the irregular force) must be rebuilt on next use.
void ctx_state_changed(nb_ctx *c)
{
    if (c) c->srec_valid = false;
}
}  // namespace nbgpu

// ------------------------------------------------------------------------------ ABI
extern "C" {

int32_t nb_version(void) { return 100; }

nb_status nb_init(nb_ctx **out, const nb_config *cfg)
{
    if (!out) return NB_ERR_ARG;
    *out = nullptr;
    if (!cfg) return NB_ERR_ARG;
    if (cfg->n_max < 1 || cfg->nb_cap < 1 || cfg->nb_cap > kMaxCap || cfg->flags != 0 ||
        (cfg->precision != NB_FP64 && cfg->precision != NB_MIXED) || cfg->n_max > (int64_t)INT32_MAX - kTilePad)
        return NB_ERR_ARG;
    nb_ctx *c = new (std::nothrow) nb_ctx();
    if (!c) return NB_ERR_OOM;
    c->device = cfg->device;
    c->precision = cfg->precision;
    c->cap = cfg->nb_cap;
    c->n_max = cfg->n_max;
    if (const char *f = getenv("NB_FAULT")) {  // "alloc:N", "sync:N" or "status:N"
        int after = 0;
        char kind[16] = {0};
        if (sscanf(f, "%15[a-z]:%d", kind, &after) >= 1) {
            c->fault_after = after;
            c->fault_kind = !strcmp(kind, "alloc") ? NB_FAULT_ALLOC
                            : !strcmp(kind, "sync") ? NB_FAULT_SYNC
                            : !strcmp(kind, "status") ? NB_FAULT_STATUS : 0;
        }
    }
    auto bail = [&](nb_status s) {
        nb_free(c);
        return s;
    };
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return bail(NB_ERR_CUDA);
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        return bail(NB_ERR_CUDA);
    if (cfg->stream) {
        c->stream = (cudaStream_t)cfg->stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) return bail(NB_ERR_CUDA);
        c->stream = c->own_stream;
    }
    query_occupancy(c->occ);
    const int64_t nm = c->n_max, npad = ((nm + kTilePad - 1) / kTilePad) * kTilePad;
    const size_t v3 = (size_t)nm * 3 * sizeof(double), s1 = (size_t)nm * sizeof(double);
    const size_t rec_bytes = c->precision == NB_FP64 ? (size_t)npad * 2 * sizeof(dvec4) : (size_t)npad * 3 * sizeof(float4);
    if (cudaMalloc(&c->x, v3) != cudaSuccess || cudaMalloc(&c->v, v3) != cudaSuccess ||
        cudaMalloc(&c->a, v3) != cudaSuccess || cudaMalloc(&c->jk, v3) != cudaSuccess ||
        cudaMalloc(&c->m, s1) != cudaSuccess || cudaMalloc(&c->tl, s1) != cudaSuccess ||
        cudaMalloc(&c->xp, v3) != cudaSuccess || cudaMalloc(&c->vp, v3) != cudaSuccess ||
        cudaMalloc(&c->rec, rec_bytes) != cudaSuccess ||
        cudaMalloc(&c->status, SS_WORDS * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return bail(NB_ERR_OOM);
    }
    if (cudaMemset(c->status, 0, SS_WORDS * sizeof(unsigned)) != cudaSuccess) return bail(NB_ERR_CUDA);
    *out = c;
    return NB_OK;
}

nb_status nb_free(nb_ctx *c)
{
    if (!c) return NB_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    void *ptrs[] = {c->x, c->v, c->a, c->jk, c->m, c->tl, c->xp, c->vp, c->rec, c->status,
                    c->part, c->seg_slots, c->seg_cnt, c->row_total, c->scan, c->stage, c->adj, c->b_items,
                    c->b_cluster_off, c->srec, c->prec, c->ro};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    for (auto &sp : c->spans) {
        cudaEventDestroy(sp.a);
        cudaEventDestroy(sp.b);
    }
    for (auto e : c->evpool) cudaEventDestroy(e);
    delete c;
    return NB_OK;
}

nb_status nb_set_stream(nb_ctx *c, void *stream)
{
    nb_status s = check_usable(c);
    if (s != NB_OK) return s;
    // NULL is CUDA's default (legacy) stream, which is what a framework reports when it
    // runs on the default stream; work then orders with the framework's own kernels.
    c->stream = (cudaStream_t)stream;
    return NB_OK;
}

static nb_status copy_in(nb_ctx *c, void *dst, const void *src, size_t bytes, int on_device)
{
    CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       c->stream),
       "cudaMemcpyAsync (in)");
    return NB_OK;
}

nb_status nb_set_particles(nb_ctx *c, int64_t n, const double *x, const double *v, const double *a,
                           const double *jerk, const double *m, const double *t_last, int32_t on_device)
{
    nb_status s = check_usable(c);
    if (s != NB_OK) return s;
    if (n < 1 || n > c->n_max) return fail(c, NB_ERR_ARG, "n=%lld outside [1, n_max=%lld]", (long long)n, (long long)c->n_max);
    if (!x || !v || !a || !jerk || !m || !t_last) return fail(c, NB_ERR_ARG, "null array");
    const size_t b3 = (size_t)n * 3 * sizeof(double), b1 = (size_t)n * sizeof(double);
    if ((s = copy_in(c, c->x, x, b3, on_device)) || (s = copy_in(c, c->v, v, b3, on_device)) ||
        (s = copy_in(c, c->a, a, b3, on_device)) || (s = copy_in(c, c->jk, jerk, b3, on_device)) ||
        (s = copy_in(c, c->m, m, b1, on_device)) || (s = copy_in(c, c->tl, t_last, b1, on_device)))
        return s;
    c->n = n;
    c->n_pad = ((n + kTilePad - 1) / kTilePad) * kTilePad;
    c->have_state = true;
    c->srec_valid = false;
    c->have_pred = false;
    if (!on_device) CK(ctx_sync(c), "cudaStreamSynchronize");
    return NB_OK;
}

nb_status nb_predict(nb_ctx *c, double t)
{
    nb_status s = check_usable(c);
    if (s != NB_OK) return s;
    if (!c->have_state) return fail(c, NB_ERR_STATE, "nb_predict before nb_set_particles");
    cudaEvent_t t0 = span_begin(c);
    launch_predict(c->stream, c->n, c->n_pad, t, c->x, c->v, c->a, c->jk, c->tl, c->m, c->xp, c->vp,
                   c->precision == NB_FP64 ? c->rec : nullptr, c->precision == NB_MIXED ? c->rec : nullptr);
    CK_LAUNCH("k_predict launch");
    span_end(c, PH_PREDICT, t0, 1);
    c->have_pred = true;
    return NB_OK;
}

nb_status nb_set_predicted(nb_ctx *c, int64_t n, const double *xp, const double *vp, const double *m,
                           int32_t on_device)
{
    nb_status s = check_usable(c);
    if (s != NB_OK) return s;
    if (n < 1 || n > c->n_max) return fail(c, NB_ERR_ARG, "n=%lld outside [1, n_max=%lld]", (long long)n, (long long)c->n_max);
    if (!xp || !vp || !m) return fail(c, NB_ERR_ARG, "null array");
    const size_t b3 = (size_t)n * 3 * sizeof(double), b1 = (size_t)n * sizeof(double);
    if ((s = copy_in(c, c->xp, xp, b3, on_device)) || (s = copy_in(c, c->vp, vp, b3, on_device)) ||
        (s = copy_in(c, c->m, m, b1, on_device)))
        return s;
    c->n = n;
    c->n_pad = ((n + kTilePad - 1) / kTilePad) * kTilePad;
    launch_pack_predicted(c->stream, n, c->n_pad, c->xp, c->vp, c->m, c->precision == NB_FP64 ? c->rec : nullptr,
                          c->precision == NB_MIXED ? c->rec : nullptr);
    CK_LAUNCH("k_pack launch");
    c->have_state = false;
    c->have_pred = true;
    if (!on_device) CK(ctx_sync(c), "cudaStreamSynchronize");
    return NB_OK;
}

nb_status nb_get_predicted(nb_ctx *c, double *xp, double *vp, int32_t on_device)
{
    nb_status s = check_usable(c);
    if (s != NB_OK) return s;
    if (!c->have_pred) return fail(c, NB_ERR_STATE, "no predicted state");
    if (!xp || !vp) return fail(c, NB_ERR_ARG, "null array");
    const size_t b3 = (size_t)c->n * 3 * sizeof(double);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(xp, c->xp, b3, kind, c->stream), "cudaMemcpyAsync");
    CK(cudaMemcpyAsync(vp, c->vp, b3, kind, c->stream), "cudaMemcpyAsync");
    if (!on_device) CK(ctx_sync(c), "cudaStreamSynchronize");
    return NB_OK;
}

nb_status nb_get_records(nb_ctx *c, void *out, int32_t on_device)
{
    nb_status s = check_usable(c);
    if (s != NB_OK) return s;
    if (!c->have_pred) return fail(c, NB_ERR_STATE, "no predicted state");
    if (!out) return fail(c, NB_ERR_ARG, "null array");
    const size_t b = (size_t)c->n * (c->precision == NB_FP64 ? 2 * sizeof(dvec4) : 3 * sizeof(float4));
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(out, c->rec, b, kind, c->stream), "cudaMemcpyAsync");
    if (!on_device) CK(ctx_sync(c), "cudaStreamSynchronize");
    return NB_OK;
}

// The plan of a call: the override if one is set, else the first tuned table entry whose
// bucket holds n_i, else the automatic plan.
static Plan ctx_plan(const nb_ctx *c, int64_t n, int64_t n_i)
{
    if (c->force_kernel >= 0)
        return forced_plan(c->precision, c->num_sms, c->occ, n, n_i, c->cap, c->force_kernel, c->force_variant,
                           c->force_splits);
    for (const auto &e : c->table)
        if (n_i <= e.ni_max)
            return forced_plan(c->precision, c->num_sms, c->occ, n, n_i, c->cap, e.kernel, e.variant, e.splits);
    return plan_force(c->precision, c->num_sms, c->occ, n, n_i, c->cap);
}

static bool plan_valid(int precision, int kernel, int variant, int splits)
{
    const bool ok = (kernel == 1 && precision == NB_MIXED && variant >= 0 && variant < kMixedTiledVariants) ||
                    (kernel == 2 && precision == NB_MIXED && variant >= 0 && variant <= 3) ||
                    (kernel == 0 && precision == NB_FP64 && variant == 0) ||
                    (kernel == 3 && precision == NB_FP64 && variant >= 0 && variant <= 1);
    return ok && splits >= 0 && !(splits == 0 && kernel == 0);
}

nb_status nb_set_plan_table(nb_ctx *c, int32_t n_entries, const int64_t *ni_max, const int32_t *kernel,
                            const int32_t *variant, const int32_t *splits)
{
    if (!c || n_entries < 0 || (n_entries > 0 && (!ni_max || !kernel || !variant || !splits))) return NB_ERR_ARG;
    std::vector<nb_ctx::TableEntry> t;
    for (int32_t q = 0; q < n_entries; ++q) {
        if (!plan_valid(c->precision, kernel[q], variant[q], splits[q]) || (q > 0 && ni_max[q] <= ni_max[q - 1]))
            return fail(c, NB_ERR_ARG, "plan table entry %d invalid (kernel %d, variant %d, splits %d)", q, kernel[q],
                        variant[q], splits[q]);
        t.push_back({ni_max[q], kernel[q], variant[q], splits[q]});
    }
    c->table.swap(t);
    return NB_OK;
}

// ---- Hermite predictor / corrector over caller arrays (differentiable integration) -------
static nb_status hermite_args(nb_ctx *c, int64_t n, std::initializer_list<const void *> arrays)
{
    nb_status s = check_usable(c);
    if (s != NB_OK) return s;
    if (n < 0) return fail(c, NB_ERR_ARG, "n=%lld out of range", (long long)n);
    for (const void *p : arrays)
        if (n > 0 && !p) return fail(c, NB_ERR_ARG, "null array");
    return NB_OK;
}

nb_status nb_hermite_predict(nb_ctx *c, int64_t n, double t, const double *x, const double *v, const double *a,
                             const double *jerk, const double *t_last, double *xp, double *vp)
{
    nb_status s = hermite_args(c, n, {x, v, a, jerk, t_last, xp, vp});
    if (s != NB_OK || n == 0) return s;
    cudaEvent_t t0 = span_begin(c);
    launch_hermite_predict(c->stream, n, t, x, v, a, jerk, t_last, xp, vp);
    CK_LAUNCH("k_hermite_predict launch");
    span_end(c, PH_PREDICT, t0, 1);
    return NB_OK;
}

nb_status nb_hermite_predict_backward(nb_ctx *c, int64_t n, double t, const double *t_last, const double *g_xp,
                                      const double *g_vp, double *g_x, double *g_v, double *g_a, double *g_jerk)
{
    nb_status s = hermite_args(c, n, {t_last, g_xp, g_vp, g_x, g_v, g_a, g_jerk});
    if (s != NB_OK || n == 0) return s;
    cudaEvent_t t0 = span_begin(c);
    launch_hermite_predict_vjp(c->stream, n, t, t_last, g_xp, g_vp, g_x, g_v, g_a, g_jerk);
    CK_LAUNCH("k_hermite_predict_vjp launch");
    span_end(c, PH_BACKWARD, t0, 1);
    return NB_OK;
}

nb_status nb_hermite_correct(nb_ctx *c, int64_t n, double t, const double *t_last, const double *xp,
                             const double *vp, const double *a0, const double *j0, const double *a1,
                             const double *j1, double *x1, double *v1)
{
    nb_status s = hermite_args(c, n, {t_last, xp, vp, a0, j0, a1, j1, x1, v1});
    if (s != NB_OK || n == 0) return s;
    cudaEvent_t t0 = span_begin(c);
    launch_hermite_correct(c->stream, n, t, t_last, xp, vp, a0, j0, a1, j1, x1, v1);
    CK_LAUNCH("k_hermite_correct launch");
    span_end(c, PH_PREDICT, t0, 1);
    return NB_OK;
}

nb_status nb_hermite_correct_backward(nb_ctx *c, int64_t n, double t, const double *t_last, const double *g_x1,
                                      const double *g_v1, double *g_xp, double *g_vp, double *g_a0, double *g_j0,
                                      double *g_a1, double *g_j1)
{
    nb_status s = hermite_args(c, n, {t_last, g_x1, g_v1, g_xp, g_vp, g_a0, g_j0, g_a1, g_j1});
    if (s != NB_OK || n == 0) return s;
    cudaEvent_t t0 = span_begin(c);
    launch_hermite_correct_vjp(c->stream, n, t, t_last, g_x1, g_v1, g_xp, g_vp, g_a0, g_j0, g_a1, g_j1);
    CK_LAUNCH("k_hermite_correct_vjp launch");
    span_end(c, PH_BACKWARD, t0, 1);
    return NB_OK;
}

nb_status nb_row_order(nb_ctx *c, int64_t n_i, const int32_t *idx, int32_t *perm)
{
    nb_status s = check_usable(c);
    if (s != NB_OK) return s;
    if (c->precision != NB_MIXED) return fail(c, NB_ERR_STATE, "nb_row_order reads the mixed j-records: mixed context only");
    if (!c->have_pred) return fail(c, NB_ERR_STATE, "nb_row_order before nb_predict / nb_set_predicted");
    if (n_i < 0 || n_i > (int64_t)INT32_MAX) return fail(c, NB_ERR_ARG, "n_i=%lld out of range", (long long)n_i);
    if (n_i == 0) return NB_OK;
    if (!idx || !perm) return fail(c, NB_ERR_ARG, "null array");
    if ((s = grow(c, &c->ro, &c->ro_cap, roworder_scratch_bytes(n_i), "row order")) != NB_OK) return s;
    cudaEvent_t t0 = span_begin(c);
    const int32_t *out = nullptr;
    const int kernels = launch_row_order(c->stream, c->rec, idx, c->n, n_i, c->ro, &out);
    CK_LAUNCH("row order launch");
    CK(cudaMemcpyAsync(perm, out, (size_t)n_i * 4, cudaMemcpyDeviceToDevice, c->stream), "copy order");
    span_end(c, PH_ORDER, t0, kernels);
    return NB_OK;
}

nb_status nb_plan(const nb_ctx *c, int64_t n, int64_t n_i, int64_t *out)
{
    if (!c || !out || n < 1 || n_i < 0) return NB_ERR_ARG;
    Plan p = ctx_plan(c, n, n_i);
    out[0] = p.kernel;
    out[1] = p.i_per_cta;
    out[2] = p.S;
    out[3] = p.ctas;
    out[4] = p.tj;
    out[5] = p.variant;
    return NB_OK;
}

nb_status nb_plan_for(int32_t precision, int32_t num_sms, const int32_t *ctas_per_sm, int64_t n, int64_t n_i,
                      int32_t nb_cap, int64_t *out)
{
    if (!out || n < 1 || n_i < 0 || nb_cap < 1 || (precision != NB_FP64 && precision != NB_MIXED)) return NB_ERR_ARG;
    int occ[kOccSlots];
    for (int q = 0; q < kOccSlots; ++q) occ[q] = 1;
    if (ctas_per_sm)
        for (int q = 0; q < kOccSlots; ++q) occ[q] = ctas_per_sm[q];
    Plan p = plan_force(precision, num_sms, occ, n, n_i, nb_cap);
    out[0] = p.kernel;
    out[1] = p.i_per_cta;
    out[2] = p.S;
    out[3] = p.ctas;
    out[4] = p.tj;
    out[5] = p.variant;
    return NB_OK;
}

nb_status nb_set_plan_override(nb_ctx *c, int32_t kernel, int32_t variant, int32_t splits)
{
    if (!c) return NB_ERR_ARG;
    if (kernel < 0) {
        c->force_kernel = -1;
        return NB_OK;
    }
    const bool ok = (kernel == 1 && c->precision == NB_MIXED && variant >= 0 && variant < kMixedTiledVariants) ||
                    (kernel == 2 && c->precision == NB_MIXED && variant >= 0 && variant <= 3) ||
                    (kernel == 0 && c->precision == NB_FP64 && variant == 0) ||
                    (kernel == 3 && c->precision == NB_FP64 && variant >= 0 && variant <= 1);
    if (!ok || splits < 0 || (splits == 0 && kernel == 0))
        return fail(c, NB_ERR_ARG, "plan override (%d, %d, %d) invalid for this context", kernel, variant, splits);
    c->force_kernel = kernel;
    c->force_variant = variant;
    c->force_splits = splits;
    return NB_OK;
}

nb_status nb_inject_fault(nb_ctx *c, int32_t kind, int32_t after)
{
    if (!c || kind < 0 || kind > NB_FAULT_STATUS || after < 0) return NB_ERR_ARG;
    c->fault_kind = kind;
    c->fault_after = after;
    return NB_OK;
}

nb_status nb_set_source_range(nb_ctx *c, int64_t j_lo, int64_t j_hi)
{
    if (!c) return NB_ERR_ARG;
    if (j_lo == 0 && j_hi == 0) {
        c->src_lo = c->src_hi = 0;
        return NB_OK;
    }
    if (j_lo < 0 || j_hi <= j_lo || j_hi > c->n_max || j_lo % kTilePad != 0)
        return fail(c, NB_ERR_ARG, "source range [%lld, %lld) invalid: need 0 <= j_lo < j_hi <= n_max, j_lo %% %d == 0",
                    (long long)j_lo, (long long)j_hi, kTilePad);
    c->src_lo = j_lo;
    c->src_hi = j_hi;
    return NB_OK;
}

nb_status nb_regular_force(nb_ctx *c, int64_t n_i, const int32_t *idx, const double *rs2, int32_t rs2_scalar,
                           double *acc, double *jerk, double *pot, int64_t *nb_off, int32_t *nb_idx,
                           int64_t nb_idx_capacity, int32_t *nb_count_true, int32_t on_device)
{
    nb_status s = check_usable(c);
    if (s != NB_OK) return s;
    if (!c->have_pred) return fail(c, NB_ERR_STATE, "nb_regular_force before nb_predict / nb_set_predicted");
    if (n_i < 0 || n_i > (int64_t)INT32_MAX) return fail(c, NB_ERR_ARG, "n_i=%lld out of range", (long long)n_i);
    if (nb_idx && (!nb_off || nb_idx_capacity < 0)) return fail(c, NB_ERR_ARG, "nb_idx needs nb_off and a capacity >= 0");
    if (n_i > 0 && (!idx || !rs2 || !acc || !jerk || !pot)) return fail(c, NB_ERR_ARG, "null array");
    const bool want_nb = nb_off || nb_count_true;
    if (n_i == 0) {
        if (nb_off) {
            if (on_device) CK(cudaMemsetAsync(nb_off, 0, sizeof(int64_t), c->stream), "cudaMemsetAsync");
            else nb_off[0] = 0;
        }
        return NB_OK;
    }
    const int64_t n = c->n;
    const int64_t j_lo = c->src_hi ? c->src_lo : 0, j_hi = c->src_hi ? c->src_hi : n;
    if (j_hi > n || (j_hi != n && j_hi % kTilePad != 0))
        return fail(c, NB_ERR_STATE, "source range [%lld, %lld) does not fit the %lld loaded particles",
                    (long long)j_lo, (long long)j_hi, (long long)n);
    // host mode: validate on the host and stage everything on the device
    const int32_t *d_idx = idx;
    const double *d_rs2 = rs2;
    double *d_acc = acc, *d_jerk = jerk, *d_pot = pot;
    int64_t *d_off = nb_off;
    int32_t *d_nbidx = nb_idx, *d_cnt_true = nb_count_true;
    const size_t n_rs2 = rs2_scalar ? 1 : (size_t)n_i;
    if (!on_device) {
        for (int64_t k = 0; k < n_i; ++k)
            if (idx[k] < 0 || idx[k] >= n) return fail(c, NB_ERR_ARG, "idx[%lld]=%d outside [0, %lld)", (long long)k, idx[k], (long long)n);
        const size_t cap_nb = nb_idx ? (size_t)nb_idx_capacity : 0;
        const size_t bytes = 256 * 8 + (size_t)n_i * 4 + n_rs2 * 8 + (size_t)n_i * 7 * 8 + ((size_t)n_i + 1) * 8 +
                             cap_nb * 4 + (size_t)n_i * 4;
        if ((s = grow(c, (void **)&c->stage, &c->stage_cap, bytes, "staging buffer")) != NB_OK) return s;
        char *p = c->stage;
        auto take = [&](size_t b) {
            char *q = p;
            p += (b + 255) & ~(size_t)255;
            return q;
        };
        d_idx = (int32_t *)take((size_t)n_i * 4);
        d_rs2 = (double *)take(n_rs2 * 8);
        d_acc = (double *)take((size_t)n_i * 24);
        d_jerk = (double *)take((size_t)n_i * 24);
        d_pot = (double *)take((size_t)n_i * 8);
        d_off = nb_off ? (int64_t *)take(((size_t)n_i + 1) * 8) : nullptr;
        d_nbidx = nb_idx ? (int32_t *)take(cap_nb * 4 + 4) : nullptr;
        d_cnt_true = nb_count_true ? (int32_t *)take((size_t)n_i * 4) : nullptr;
        CK(cudaMemcpyAsync((void *)d_idx, idx, (size_t)n_i * 4, cudaMemcpyHostToDevice, c->stream), "copy idx");
        CK(cudaMemcpyAsync((void *)d_rs2, rs2, n_rs2 * 8, cudaMemcpyHostToDevice, c->stream), "copy rs2");
    }
    Plan p = ctx_plan(c, j_hi - j_lo, n_i);
    const size_t part_bytes = (size_t)p.S * 7 * (size_t)n_i * sizeof(double);
    if ((s = grow(c, (void **)&c->part, &c->part_cap, part_bytes, "partial sums")) != NB_OK) return s;
    // neighbour segments: G ordered j-segments, L slots each per row (0: counts only)
    const int64_t G = (int64_t)p.S * p.segs_per_split;
    const int L = d_nbidx ? (int)(p.seg_len < c->cap ? p.seg_len : c->cap) : 0;
    const size_t scan_elems = neighbour_scan_tmp_elems(n_i) + (d_off ? 0 : (size_t)n_i + 1);
    if (want_nb) {
        if ((s = grow(c, (void **)&c->seg_cnt, &c->seg_cnt_cap, (size_t)G * n_i * 4, "neighbour counts")) != NB_OK) return s;
        if ((s = grow(c, (void **)&c->row_total, &c->row_total_cap, (size_t)n_i * 4, "neighbour totals")) != NB_OK)
            return s;
        if (L > 0 &&
            (s = grow(c, (void **)&c->seg_slots, &c->seg_slots_cap, (size_t)G * n_i * L * 4, "neighbour slots")) != NB_OK)
            return s;
        if ((s = grow(c, (void **)&c->scan, &c->scan_cap, scan_elems * 8, "scan scratch")) != NB_OK) return s;
    }
    ForceArgs fa{};
    if (p.kernel == 1 && mixed_tiled_anchored(p.variant)) {  // spatial order of the rows first
        if ((s = grow(c, &c->ro, &c->ro_cap, roworder_scratch_bytes(n_i), "row order")) != NB_OK) return s;
        cudaEvent_t t0 = span_begin(c);
        const int kernels = launch_row_order(c->stream, c->rec, d_idx, n, n_i, c->ro, &fa.perm);
        CK_LAUNCH("row order launch");
        span_end(c, PH_ORDER, t0, kernels);
    }
    fa.rec = c->rec;
    fa.n = n;
    fa.j_lo = j_lo;
    fa.j_hi = j_hi;
    fa.idx = d_idx;
    fa.n_i = n_i;
    fa.rs2 = d_rs2;
    fa.rs2_scalar = rs2_scalar ? 1 : 0;
    fa.want_nb = want_nb ? 1 : 0;
    fa.L = L;
    // the anchored kernels skip storing hits that earlier segments of the row already make
    // surplus; they read those segments' counts, which start as -1 (not yet known)
    if (want_nb && p.S > 1 && p.S <= kPriorSegMax && p.kernel == 1 && mixed_tiled_anchored(p.variant)) {
        fa.cap = c->cap;
        CK(cudaMemsetAsync(c->seg_cnt, 0xff, (size_t)p.S * n_i * 4, c->stream), "clear counts");
    }
    fa.part = c->part;
    fa.seg_cnt = c->seg_cnt;
    fa.seg_slots = c->seg_slots;
    fa.status = c->status;
    cudaEvent_t t0 = span_begin(c);
    launch_force(c->stream, p, fa);
    CK_LAUNCH("force kernel launch");
    span_end(c, PH_FORCE, t0, 1);
    // counts only: the scan still needs an offsets buffer, taken from the scan scratch
    int64_t *off_buf = want_nb ? (d_off ? d_off : c->scan + neighbour_scan_tmp_elems(n_i)) : nullptr;
    const bool tiny = !fa.perm && n_i <= kTinyRows && (!want_nb || tiny_epilogue_fits(G, n_i));
    if (tiny) {  // a tiny block: the sums and the lists in one launch (timed as the reduction)
        t0 = span_begin(c);
        launch_tiny_epilogue(c->stream, c->part, p.S, n_i, d_acc, d_jerk, d_pot, G, L, c->cap,
                             want_nb ? c->seg_cnt : nullptr, c->seg_slots, off_buf, d_nbidx,
                             d_nbidx ? nb_idx_capacity : INT64_MAX, d_cnt_true, c->status);
        CK_LAUNCH("tiny-block epilogue launch");
        span_end(c, PH_REDUCE, t0, 1);
    } else {
        t0 = span_begin(c);
        launch_reduce(c->stream, c->part, p.S, n_i, d_acc, d_jerk, d_pot, fa.perm);  // anchored: row-order positions
        CK_LAUNCH("k_reduce launch");
        span_end(c, PH_REDUCE, t0, 1);
    }
    if (want_nb && !tiny) {
        t0 = span_begin(c);
        const int kernels = launch_neighbour_csr(c->stream, G, n_i, L, c->cap, c->seg_cnt, c->seg_slots, off_buf,
                                                 d_nbidx, d_nbidx ? nb_idx_capacity : INT64_MAX, d_cnt_true, c->scan,
                                                 c->row_total, c->status, fa.perm);
        CK_LAUNCH("neighbour CSR launch");
        span_end(c, PH_NEIGHBOURS, t0, kernels);
    }
    if (on_device) return NB_OK;
    // host mode: copy results back and report the deferred status of this call
    CK(cudaMemcpyAsync(acc, d_acc, (size_t)n_i * 24, cudaMemcpyDeviceToHost, c->stream), "copy acc");
    CK(cudaMemcpyAsync(jerk, d_jerk, (size_t)n_i * 24, cudaMemcpyDeviceToHost, c->stream), "copy jerk");
    CK(cudaMemcpyAsync(pot, d_pot, (size_t)n_i * 8, cudaMemcpyDeviceToHost, c->stream), "copy pot");
    if (nb_count_true)
        CK(cudaMemcpyAsync(nb_count_true, d_cnt_true, (size_t)n_i * 4, cudaMemcpyDeviceToHost, c->stream), "copy counts");
    if (nb_off) {
        CK(cudaMemcpyAsync(nb_off, d_off, ((size_t)n_i + 1) * 8, cudaMemcpyDeviceToHost, c->stream), "copy offsets");
        CK(ctx_sync(c), "cudaStreamSynchronize");
        if (nb_idx) {
            int64_t tot = nb_off[n_i] < nb_idx_capacity ? nb_off[n_i] : nb_idx_capacity;
            if (tot > 0)
                CK(cudaMemcpyAsync(nb_idx, d_nbidx, (size_t)tot * 4, cudaMemcpyDeviceToHost, c->stream), "copy lists");
        }
    }
    return sync_and_collect(c);
}

nb_status nb_regular_force_backward(nb_ctx *c, int64_t n_i, const int32_t *idx, const double *g_acc,
                                    const double *g_jerk, const double *g_pot, double *g_x, double *g_v,
                                    double *g_m, int32_t on_device)
{
    nb_status s = check_usable(c);
    if (s != NB_OK) return s;
    if (!c->have_pred) return fail(c, NB_ERR_STATE, "nb_regular_force_backward before nb_predict / nb_set_predicted");
    if (n_i < 0 || n_i > (int64_t)INT32_MAX) return fail(c, NB_ERR_ARG, "n_i=%lld out of range", (long long)n_i);
    if (!g_x || !g_v || !g_m || (n_i > 0 && (!idx || !g_acc || !g_jerk || !g_pot)))
        return fail(c, NB_ERR_ARG, "null array");
    if (c->src_hi) return fail(c, NB_ERR_STATE, "nb_regular_force_backward needs the full source range");
    const int64_t n = c->n;
    const int32_t *d_idx = idx;
    const double *d_ga = g_acc, *d_gj = g_jerk, *d_gp = g_pot;
    double *d_gx = g_x, *d_gv = g_v, *d_gm = g_m;
    if (!on_device) {
        for (int64_t k = 0; k < n_i; ++k)
            if (idx[k] < 0 || idx[k] >= n) return fail(c, NB_ERR_ARG, "idx[%lld]=%d outside [0, %lld)", (long long)k, idx[k], (long long)n);
        const size_t bytes = 8 * 256 + (size_t)n_i * (4 + 56) + (size_t)n * 56;
        if ((s = grow(c, (void **)&c->stage, &c->stage_cap, bytes, "staging buffer")) != NB_OK) return s;
        char *p = c->stage;
        auto take = [&](size_t b) {
            char *q = p;
            p += (b + 255) & ~(size_t)255;
            return q;
        };
        d_idx = (int32_t *)take((size_t)n_i * 4);
        d_ga = (double *)take((size_t)n_i * 24);
        d_gj = (double *)take((size_t)n_i * 24);
        d_gp = (double *)take((size_t)n_i * 8);
        d_gx = (double *)take((size_t)n * 24);
        d_gv = (double *)take((size_t)n * 24);
        d_gm = (double *)take((size_t)n * 8);
        if (n_i > 0) {
            CK(cudaMemcpyAsync((void *)d_idx, idx, (size_t)n_i * 4, cudaMemcpyHostToDevice, c->stream), "copy idx");
            CK(cudaMemcpyAsync((void *)d_ga, g_acc, (size_t)n_i * 24, cudaMemcpyHostToDevice, c->stream), "copy g_acc");
            CK(cudaMemcpyAsync((void *)d_gj, g_jerk, (size_t)n_i * 24, cudaMemcpyHostToDevice, c->stream), "copy g_jerk");
            CK(cudaMemcpyAsync((void *)d_gp, g_pot, (size_t)n_i * 8, cudaMemcpyHostToDevice, c->stream), "copy g_pot");
        }
    }
    int64_t rows_pad = 0;
    int SA = 0, SB = 0;
    const size_t need = adjoint_scratch_bytes(c->precision, n, n_i, c->num_sms, &rows_pad, &SA, &SB);
    if ((s = grow(c, (void **)&c->adj, &c->adj_cap, need, "adjoint scratch")) != NB_OK) return s;
    cudaEvent_t t0 = span_begin(c);
    const int kernels = launch_adjoint(c->stream, c->precision, c->rec, n, d_idx, n_i, d_ga, d_gj, d_gp, d_gx, d_gv,
                                       d_gm, c->adj, c->status, c->num_sms);
    CK_LAUNCH("adjoint kernels launch");
    span_end(c, PH_BACKWARD, t0, kernels);
    if (on_device) return NB_OK;
    CK(cudaMemcpyAsync(g_x, d_gx, (size_t)n * 24, cudaMemcpyDeviceToHost, c->stream), "copy g_x");
    CK(cudaMemcpyAsync(g_v, d_gv, (size_t)n * 24, cudaMemcpyDeviceToHost, c->stream), "copy g_v");
    CK(cudaMemcpyAsync(g_m, d_gm, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream), "copy g_m");
    return sync_and_collect(c);
}

nb_status nb_irregular_force(nb_ctx *c, double t, int64_t n_i, const int32_t *idx, const int64_t *nb_off,
                             const int32_t *nb_idx, double *acc, double *jerk, double *pot, double *acc_reg,
                             double *jerk_reg, double *pot_reg, int32_t on_device)
{
    nb_status s = check_usable(c);
    if (s != NB_OK) return s;
    if (!c->have_state) return fail(c, NB_ERR_STATE, "nb_irregular_force needs the Hermite state of nb_set_particles");
    if (n_i < 0 || n_i > (int64_t)INT32_MAX) return fail(c, NB_ERR_ARG, "n_i=%lld out of range", (long long)n_i);
    const int nreg = (acc_reg != nullptr) + (jerk_reg != nullptr) + (pot_reg != nullptr);
    if (nreg != 0 && nreg != 3) return fail(c, NB_ERR_ARG, "acc_reg, jerk_reg and pot_reg: all three or none");
    if (n_i == 0) return NB_OK;
    if (!idx || !nb_off || !nb_idx || !acc || !jerk || !pot) return fail(c, NB_ERR_ARG, "null array");
    const int64_t n = c->n;
    // Neighbour-only prediction, or (Sec. 3.3.3) one prediction of all particles when the
    // lists of the block name many more particles than there are.
    const bool predict_all = n_i * (c->precision == NB_FP64 ? kIrrAllFactorFp64 : kIrrAllFactorMixed) >= n;
    cudaEvent_t t0 = span_begin(c);
    int kernels = 1;
    const void *records = c->srec;
    if (predict_all) {
        const size_t rb = (size_t)c->n_pad * (c->precision == NB_FP64 ? 2 * sizeof(dvec4) : 3 * sizeof(float4));
        if ((s = grow(c, &c->prec, &c->prec_cap, rb, "predicted records")) != NB_OK) return s;
        launch_predict(c->stream, n, c->n_pad, t, c->x, c->v, c->a, c->jk, c->tl, c->m, nullptr, nullptr,
                       c->precision == NB_FP64 ? c->prec : nullptr, c->precision == NB_MIXED ? c->prec : nullptr);
        CK_LAUNCH("k_predict launch");
        records = c->prec;
        kernels = 2;
    } else if (!c->srec_valid) {
        if ((s = grow(c, &c->srec, &c->srec_cap, state_record_bytes(c->precision, n), "state records")) != NB_OK)
            return s;
        launch_pack_state(c->stream, c->precision, n, c->x, c->v, c->a, c->jk, c->tl, c->m, c->srec);
        CK_LAUNCH("k_pack_state launch");
        c->srec_valid = true;
        records = c->srec;
        kernels = 2;
    }
    const int32_t *d_idx = idx, *d_nb = nb_idx;
    const int64_t *d_off = nb_off;
    double *d_acc = acc, *d_jerk = jerk, *d_pot = pot, *d_ar = acc_reg, *d_jr = jerk_reg, *d_pr = pot_reg;
    if (!on_device) {
        // host mode: validate the rows and lists on the host and stage them
        if (nb_off[0] < 0) return fail(c, NB_ERR_ARG, "nb_off[0]=%lld < 0", (long long)nb_off[0]);
        for (int64_t k = 0; k < n_i; ++k) {
            if (idx[k] < 0 || idx[k] >= n) return fail(c, NB_ERR_ARG, "idx[%lld]=%d outside [0, %lld)", (long long)k, idx[k], (long long)n);
            if (nb_off[k + 1] < nb_off[k]) return fail(c, NB_ERR_ARG, "nb_off decreases at row %lld", (long long)k);
        }
        const int64_t tot = nb_off[n_i];
        for (int64_t e = 0; e < tot; ++e)
            if (nb_idx[e] < 0 || nb_idx[e] >= n) return fail(c, NB_ERR_ARG, "nb_idx[%lld]=%d outside [0, %lld)", (long long)e, nb_idx[e], (long long)n);
        const size_t bytes = 256 * 10 + (size_t)n_i * 4 + ((size_t)n_i + 1) * 8 + (size_t)tot * 4 +
                             (size_t)n_i * 56 * (nreg ? 2 : 1);
        if ((s = grow(c, (void **)&c->stage, &c->stage_cap, bytes, "staging buffer")) != NB_OK) return s;
        char *p = c->stage;
        auto take = [&](size_t b) {
            char *q = p;
            p += (b + 255) & ~(size_t)255;
            return q;
        };
        d_idx = (int32_t *)take((size_t)n_i * 4);
        d_off = (int64_t *)take(((size_t)n_i + 1) * 8);
        d_nb = (int32_t *)take((size_t)tot * 4 + 4);
        d_acc = (double *)take((size_t)n_i * 24);
        d_jerk = (double *)take((size_t)n_i * 24);
        d_pot = (double *)take((size_t)n_i * 8);
        CK(cudaMemcpyAsync((void *)d_idx, idx, (size_t)n_i * 4, cudaMemcpyHostToDevice, c->stream), "copy idx");
        CK(cudaMemcpyAsync((void *)d_off, nb_off, ((size_t)n_i + 1) * 8, cudaMemcpyHostToDevice, c->stream), "copy nb_off");
        if (tot > 0)
            CK(cudaMemcpyAsync((void *)d_nb, nb_idx, (size_t)tot * 4, cudaMemcpyHostToDevice, c->stream), "copy nb_idx");
        if (nreg) {
            d_ar = (double *)take((size_t)n_i * 24);
            d_jr = (double *)take((size_t)n_i * 24);
            d_pr = (double *)take((size_t)n_i * 8);
            CK(cudaMemcpyAsync(d_ar, acc_reg, (size_t)n_i * 24, cudaMemcpyHostToDevice, c->stream), "copy acc_reg");
            CK(cudaMemcpyAsync(d_jr, jerk_reg, (size_t)n_i * 24, cudaMemcpyHostToDevice, c->stream), "copy jerk_reg");
            CK(cudaMemcpyAsync(d_pr, pot_reg, (size_t)n_i * 8, cudaMemcpyHostToDevice, c->stream), "copy pot_reg");
        }
    }
    launch_irregular(c->stream, c->precision, c->num_sms, records, predict_all ? 1 : 0, n, t, n_i, d_idx, d_off, d_nb,
                     d_acc, d_jerk, d_pot, d_ar, d_jr, d_pr, c->status);
    CK_LAUNCH("irregular force launch");
    span_end(c, PH_IRREGULAR, t0, kernels);
    if (on_device) return NB_OK;
    CK(cudaMemcpyAsync(acc, d_acc, (size_t)n_i * 24, cudaMemcpyDeviceToHost, c->stream), "copy acc");
    CK(cudaMemcpyAsync(jerk, d_jerk, (size_t)n_i * 24, cudaMemcpyDeviceToHost, c->stream), "copy jerk");
    CK(cudaMemcpyAsync(pot, d_pot, (size_t)n_i * 8, cudaMemcpyDeviceToHost, c->stream), "copy pot");
    if (nreg) {
        CK(cudaMemcpyAsync(acc_reg, d_ar, (size_t)n_i * 24, cudaMemcpyDeviceToHost, c->stream), "copy acc_reg");
        CK(cudaMemcpyAsync(jerk_reg, d_jr, (size_t)n_i * 24, cudaMemcpyDeviceToHost, c->stream), "copy jerk_reg");
        CK(cudaMemcpyAsync(pot_reg, d_pr, (size_t)n_i * 8, cudaMemcpyDeviceToHost, c->stream), "copy pot_reg");
    }
    return sync_and_collect(c);
}

nb_status nb_set_timing(nb_ctx *c, int32_t enable)
{
    nb_status s = check_usable(c);
    if (s != NB_OK) return s;
    c->timing = enable != 0;
    return NB_OK;
}

nb_status nb_get_timings(nb_ctx *c, double *ms, int64_t *launches)
{
    nb_status s = check_usable(c);
    if (s != NB_OK) return s;
    if (!ms || !launches) return fail(c, NB_ERR_ARG, "null array");
    CK(ctx_sync(c), "cudaStreamSynchronize");
    for (int q = 0; q < PH_COUNT; ++q) {
        ms[q] = 0.0;
        launches[q] = c->launches[q];
        c->launches[q] = 0;
    }
    for (auto &sp : c->spans) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, sp.a, sp.b) == cudaSuccess) ms[sp.phase] += t;
        c->evpool.push_back(sp.a);
        c->evpool.push_back(sp.b);
    }
    c->spans.clear();
    cudaGetLastError();
    return NB_OK;
}

nb_status nb_batch_plan(nb_ctx *c, int64_t n_clusters, const int64_t *cluster_off, const int64_t *active_off,
                        int32_t variant)
{
    nb_status s = check_usable(c);
    if (s != NB_OK) return s;
    if (c->precision != NB_MIXED) return fail(c, NB_ERR_STATE, "the batched form needs a mixed-precision context");
    if (n_clusters < 1 || !cluster_off || !active_off) return fail(c, NB_ERR_ARG, "bad cluster description");
    if (variant >= mixed_batched_variants()) return fail(c, NB_ERR_ARG, "batched variant %d unknown", variant);
    if (cluster_off[0] != 0 || active_off[0] != 0) return fail(c, NB_ERR_ARG, "offsets must start at 0");
    int64_t max_n = 0;
    for (int64_t q = 0; q < n_clusters; ++q) {
        const int64_t nc = cluster_off[q + 1] - cluster_off[q], ac = active_off[q + 1] - active_off[q];
        if (nc < 1 || ac < 0 || ac > nc) return fail(c, NB_ERR_ARG, "cluster %lld: bad sizes", (long long)q);
        if (nc > max_n) max_n = nc;
    }
    const int64_t n = cluster_off[n_clusters], rows = active_off[n_clusters];
    if (n > c->n_max) return fail(c, NB_ERR_ARG, "clusters hold %lld particles > n_max", (long long)n);
    if (rows > (int64_t)INT32_MAX) return fail(c, NB_ERR_ARG, "too many active rows");
    // variant: the tuned one, else the largest items whose count still fills the GPU
    int v = variant;
    if (v < 0) {
        v = 0;
        for (int q = 0; q < mixed_batched_variants(); ++q) {
            const int rpi = mixed_batched_rows_per_item(q);
            int64_t items = 0;
            for (int64_t cl = 0; cl < n_clusters; ++cl) items += (active_off[cl + 1] - active_off[cl] + rpi - 1) / rpi;
            v = q;
            if (items >= 8 * (int64_t)c->num_sms) break;
        }
    }
    const int rpi = mixed_batched_rows_per_item(v);
    std::vector<BatchItem> items;
    for (int64_t cl = 0; cl < n_clusters; ++cl) {
        const int64_t a0 = active_off[cl], a1 = active_off[cl + 1];
        for (int64_t r = a0; r < a1; r += rpi) {
            BatchItem it{(int32_t)cl, (int32_t)r, (int32_t)(a1 - r < rpi ? a1 - r : rpi), 0};
            items.push_back(it);
        }
    }
    // largest (cost = row-tile x cluster size) first: the dynamic queue then balances the tail
    std::vector<size_t> order(items.size());
    for (size_t q = 0; q < order.size(); ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        const double ca = (double)(cluster_off[items[a].cluster + 1] - cluster_off[items[a].cluster]);
        const double cb = (double)(cluster_off[items[b].cluster + 1] - cluster_off[items[b].cluster]);
        return ca > cb;
    });
    std::vector<BatchItem> sorted(items.size());
    for (size_t q = 0; q < order.size(); ++q) sorted[q] = items[order[q]];
    if ((s = grow(c, &c->b_items, &c->b_items_cap, sorted.size() * sizeof(BatchItem) + 16, "batch items")) != NB_OK)
        return s;
    if ((s = grow(c, (void **)&c->b_cluster_off, &c->b_cluster_off_cap, (size_t)(n_clusters + 1) * 8, "cluster offsets")) !=
        NB_OK)
        return s;
    if (!sorted.empty())
        CK(cudaMemcpyAsync(c->b_items, sorted.data(), sorted.size() * sizeof(BatchItem), cudaMemcpyHostToDevice,
                           c->stream), "copy items");
    CK(cudaMemcpyAsync(c->b_cluster_off, cluster_off, (size_t)(n_clusters + 1) * 8, cudaMemcpyHostToDevice, c->stream),
       "copy cluster offsets");
    // scratch of the launch, grown here so that the launch itself never allocates
    const int L = (int)(max_n < c->cap ? max_n : c->cap);
    const size_t r = (size_t)(rows > 0 ? rows : 1);
    if ((s = grow(c, (void **)&c->part, &c->part_cap, 7 * r * 8, "partial sums")) != NB_OK) return s;
    if ((s = grow(c, (void **)&c->seg_cnt, &c->seg_cnt_cap, r * 4, "neighbour counts")) != NB_OK) return s;
    if ((s = grow(c, (void **)&c->seg_slots, &c->seg_slots_cap, r * (size_t)L * 4, "neighbour slots")) != NB_OK) return s;
    if ((s = grow(c, (void **)&c->scan, &c->scan_cap, (neighbour_scan_tmp_elems(rows) + r + 1) * 8, "scan scratch")) !=
        NB_OK)
        return s;
    CK(ctx_sync(c), "cudaStreamSynchronize");
    const int occ = mixed_batched_occupancy(v);
    int64_t ctas = (int64_t)occ * c->num_sms;
    if (ctas > (int64_t)sorted.size()) ctas = (int64_t)sorted.size();
    c->b_clusters = n_clusters;
    c->b_rows = rows;
    c->b_items_n = (int64_t)sorted.size();
    c->b_variant = v;
    c->b_ctas = (int)(ctas > 0 ? ctas : 1);
    c->b_L = L;
    c->b_n = n;
    return NB_OK;
}

nb_status nb_regular_force_batched(nb_ctx *c, const int32_t *idx, const double *rs2, double *acc, double *jerk,
                                   double *pot, int64_t *nb_off, int32_t *nb_idx, int64_t nb_idx_capacity,
                                   int32_t *nb_count_true)
{
    nb_status s = check_usable(c);
    if (s != NB_OK) return s;
    if (c->b_variant < 0) return fail(c, NB_ERR_STATE, "nb_regular_force_batched before nb_batch_plan");
    if (!c->have_pred) return fail(c, NB_ERR_STATE, "nb_regular_force_batched before nb_predict / nb_set_predicted");
    if (c->n != c->b_n)
        return fail(c, NB_ERR_STATE, "the loaded state has %lld particles, the batch plan %lld", (long long)c->n,
                    (long long)c->b_n);
    const int64_t rows = c->b_rows;
    if (rows > 0 && (!idx || !rs2 || !acc || !jerk || !pot)) return fail(c, NB_ERR_ARG, "null array");
    if (nb_idx && (!nb_off || nb_idx_capacity < 0)) return fail(c, NB_ERR_ARG, "nb_idx needs nb_off and a capacity >= 0");
    const bool want_nb = nb_off || nb_count_true;
    if (rows == 0) {
        if (nb_off) CK(cudaMemsetAsync(nb_off, 0, sizeof(int64_t), c->stream), "cudaMemsetAsync");
        return NB_OK;
    }
    BatchArgs ba{};
    ba.rec = static_cast<const float4 *>(c->rec);
    ba.cluster_off = c->b_cluster_off;
    ba.rs2 = rs2;
    ba.idx = idx;
    ba.n_i = rows;
    ba.items = static_cast<const BatchItem *>(c->b_items);
    ba.n_items = (int32_t)c->b_items_n;
    ba.want_nb = want_nb ? 1 : 0;
    ba.L = nb_idx ? c->b_L : 0;
    ba.queue = c->status + SS_QUEUE;
    ba.part = c->part;
    ba.seg_cnt = c->seg_cnt;
    ba.seg_slots = c->seg_slots;
    ba.status = c->status;
    cudaEvent_t t0 = span_begin(c);
    CK(cudaMemsetAsync(c->status + SS_QUEUE, 0, sizeof(unsigned), c->stream), "cudaMemsetAsync");
    launch_force_mixed_batched(c->stream, c->b_variant, c->b_ctas, ba);
    CK_LAUNCH("batched force kernel launch");
    span_end(c, PH_FORCE, t0, 1);
    t0 = span_begin(c);
    launch_reduce(c->stream, c->part, 1, rows, acc, jerk, pot);
    CK_LAUNCH("k_reduce launch");
    span_end(c, PH_REDUCE, t0, 1);
    if (want_nb) {
        int64_t *off_buf = nb_off ? nb_off : c->scan + neighbour_scan_tmp_elems(rows);
        t0 = span_begin(c);
        const int kernels = launch_neighbour_csr(c->stream, 1, rows, ba.L, c->cap, c->seg_cnt, c->seg_slots, off_buf,
                                                 nb_idx, nb_idx ? nb_idx_capacity : 0, nb_count_true, c->scan,
                                                 nullptr, c->status);
        CK_LAUNCH("neighbour CSR launch");
        span_end(c, PH_NEIGHBOURS, t0, kernels);
    }
    return NB_OK;
}

nb_status nb_sync(nb_ctx *c)
{
    nb_status s = check_usable(c);
    if (s != NB_OK) return s;
    return sync_and_collect(c);
}

const char *nb_last_error(const nb_ctx *c)
{
    if (!c) return "null context";
    return c->err;
}

}  // extern "C"
