// ac.cu — K9: the Ahmad-Cohen Hermite block step on the device (paper Sec. 2; the scheme
// is stated with the declarations in nbgpu.h).  One block step is a fixed sequence of
// launches on the context stream:
//   nb_sched_next (host)          -> block time t, active particles = list prefix
//   k_ac_classify                 -> which active particles also take a regular step (only
//                                    when the regular-level histogram predicts some)
//   with a regular subset:
//     nb_predict(t)               -> all particles predicted, j-records built
//     nb_regular_force (regular)  -> all-j sums and the new lists of the regular subset
//     irregular force, old lists  -> list sums of every active particle (predicted records)
//     irregular force, new lists  -> list sums of the regular subset over its new lists
//   without one (most block steps):
//     irregular force, old lists  -> list sums, i and its neighbours predicted on load from
//                                    the state records (Sec. 3.3.3): no O(N) work
//   k_ac_correct                  -> corrector, step criteria, regular bookkeeping, r_s; the
//                                    state records of the corrected particles
//   k_ac_lists                    -> the new lists replace the old ones
//   nb_sched_update               -> the requested levels re-sort the active prefix
// The corrector's FP64 arithmetic is written operation by operation in the order of the
// plain definition and this file is compiled without FMA contraction, so an FP64 context
// follows the reference integration to rounding.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "nbgpu.h"
#include "nb_common.cuh"
#include "nb_kernels.cuh"

namespace nbgpu {

constexpr int kAcTick = 48;  // the scheduler's time unit 2^-48

struct AcDev {
    // context state
    double *x, *v, *a, *jk, *tl, *m;
    dvec4 *s64;   // state records of the predict-on-load irregular force (FP64 context) ...
    float4 *s32;  // ... or mixed context; the other is null
    // integrator state
    double *Fr, *Jr, *D2, *D3, *rs2;
    double *Tr;
    int32_t *LR, *LI;
    int32_t *ell, *ell_cnt;
    int32_t *lr_hist;  // [64] particles per regular level (kept current by the corrector)
    unsigned *tickets; // [2] CTAs done in the classify and corrector launches (last-CTA epilogues)
    int32_t *io;       // device address of the pinned host words the corrector publishes:
                       // [0, 64) the regular-level histogram, [64] the step's status flags
    int32_t cap, lmin, lmax;
    double eta_irr, eta_reg, dt_max;
    int32_t nb_opt;
};

__device__ __forceinline__ double norm3d(double a, double b, double c) { return sqrt(a * a + b * b + c * c); }

// sqrt(eta (|a||a2| + |j|^2) / (|j||a3| + |a2|^2)); +inf where the ratio is undefined.
__device__ double ac_crit(double eta, const double *a, const double *j, const double *a2, const double *a3)
{
    const double na = norm3d(a[0], a[1], a[2]), nj = norm3d(j[0], j[1], j[2]);
    const double n2 = norm3d(a2[0], a2[1], a2[2]), n3 = norm3d(a3[0], a3[1], a3[2]);
    const double num = na * n2 + nj * nj, den = nj * n3 + n2 * n2;
    if (!(den > 0.0) || !(num > 0.0)) return __longlong_as_double(0x7ff0000000000000LL);  // +inf
    return sqrt(eta * num / den);
}

// The step rule on levels (step 2^-L): halve until not above crit, or double once when
// crit >= 2 h, 2 h <= dt_max and the time t (ticks of 2^-48) is a multiple of 2 h.
__device__ int ac_level_rule(int L, double crit, int64_t t_ticks, int lmin, int lmax)
{
    const double h = ldexp(1.0, -L);
    if (crit < h) {
        int Ln = L;
        double hn = h;
        while (hn > crit && Ln < lmax) {  // steps below 2^-lmax are not representable in ticks
            hn *= 0.5;
            ++Ln;
        }
        return Ln;
    }
    if (crit >= 2.0 * h && L - 1 >= lmin && (t_ticks & (((int64_t)1 << (kAcTick - (L - 1))) - 1)) == 0)
        return L - 1;
    return L;
}

// Largest power of two (level) not above crit and not above dt_max.
__device__ int ac_quantise(double crit, int lmin, int lmax)
{
    int L = lmin;
    double dt = ldexp(1.0, -lmin);
    while (dt > crit && L < lmax) {
        dt *= 0.5;
        ++L;
    }
    return L;
}

__global__ void k_iota32(int32_t *p, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}

// Start: regular part = all-j minus list sums, zero higher derivatives, initial levels.
__global__ void k_ac_init(AcDev D, int64_t n, const double *Fa, const double *Ja, const double *Fl, const double *Jl,
                          const int64_t *off, const int32_t *csr, double eta_s, int32_t *levels_out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double fr[3], jr[3];
        for (int c = 0; c < 3; ++c) {
            fr[c] = Fa[3 * i + c] - Fl[3 * i + c];
            jr[c] = Ja[3 * i + c] - Jl[3 * i + c];
            D.Fr[3 * i + c] = fr[c];
            D.Jr[3 * i + c] = jr[c];
            D.D2[3 * i + c] = 0.0;
            D.D3[3 * i + c] = 0.0;
            D.a[3 * i + c] = Fa[3 * i + c];
            D.jk[3 * i + c] = Ja[3 * i + c];
        }
        D.tl[i] = 0.0;
        D.Tr[i] = 0.0;
        const double ni = norm3d(Fa[3 * i], Fa[3 * i + 1], Fa[3 * i + 2]);
        const double nji = norm3d(Ja[3 * i], Ja[3 * i + 1], Ja[3 * i + 2]);
        const double nr = norm3d(fr[0], fr[1], fr[2]), njr = norm3d(jr[0], jr[1], jr[2]);
        const int LI = nji > 0.0 ? ac_quantise(eta_s * ni / nji, D.lmin, D.lmax) : D.lmin;
        int LR = njr > 0.0 ? ac_quantise(eta_s * nr / njr, D.lmin, D.lmax) : D.lmin;
        if (LR > LI) LR = LI;  // the regular step is at least the irregular one
        D.LI[i] = LI;
        D.LR[i] = LR;
        atomicAdd(&D.lr_hist[LR], 1);
        pack_state_one(i, D.x + 3 * i, D.v + 3 * i, Fa + 3 * i, Ja + 3 * i, 0.0, D.m[i], D.s64, D.s32);
        levels_out[i] = LI;
        const int64_t e0 = off[i], len = off[i + 1] - off[i];
        D.ell_cnt[i] = (int32_t)len;
        for (int64_t e = 0; e < len; ++e) D.ell[i * D.cap + e] = csr[e0 + e];
    }
}

// Active row k: regular step too?  Compacts the regular subset (order of the subset is
// irrelevant: every row's sums are independent of the others).
__global__ void k_ac_classify(AcDev D, int64_t n_act, const int32_t *list, int64_t t_ticks, unsigned *counter,
                              int32_t *reg_pos, int32_t *reg_idx, double *reg_rs2, int64_t expected, unsigned *status)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_act; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = list[k];
        const int LR = D.LR[i];
        const bool reg = (t_ticks & (((int64_t)1 << (kAcTick - LR)) - 1)) == 0;
        int32_t p = -1;
        if (reg) {
            p = (int32_t)atomicAdd(counter, 1u);
            reg_idx[p] = i;
            reg_rs2[p] = D.rs2[i];
        }
        reg_pos[k] = p;
    }
    // the last CTA to finish checks the count against the host's prediction (a mismatch is a
    // device error of the step) and leaves the counter at zero for the next step
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && atomicAdd(&D.tickets[0], 1u) == gridDim.x - 1) {
        __threadfence();
        if (atomicAdd(counter, 0u) != (unsigned)expected) atomicOr(status, ST_DEVICE);
        atomicExch(counter, 0u);
        atomicExch(&D.tickets[0], 0u);
    }
}

__global__ void k_ac_correct(AcDev D, int64_t n_act, const int32_t *list, double t, int64_t t_ticks,
                             const int32_t *reg_pos, const double *Fo, const double *Jo, const double *Fa,
                             const double *Ja, const double *Fn, const double *Jn, const int32_t *cnt_true,
                             int32_t *want, unsigned long long *pairs, unsigned *status)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_act; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = list[k];
        // reg_pos == null: the host predicted no regular particle in this step and skipped the
        // classify launch; a particle that is due for a regular step is then a device error
        int32_t p = -1;
        if (reg_pos) {
            p = reg_pos[k];
        } else if ((t_ticks & (((int64_t)1 << (kAcTick - D.LR[i])) - 1)) == 0) {
            atomicOr(status, ST_DEVICE);
        }
        atomicAdd(pairs, (unsigned long long)D.ell_cnt[i]);
        double a1[3], j1[3];
        int lr_old = -1;
        if (p < 0) {
            const double tau = t - D.Tr[i];
            for (int c = 0; c < 3; ++c) {
                const int64_t q = 3 * i + c;
                const double Fx = D.Fr[q] + D.Jr[q] * tau + D.D2[q] * tau * tau / 2.0 + D.D3[q] * tau * tau * tau / 6.0;
                const double Jx = D.Jr[q] + D.D2[q] * tau + D.D3[q] * tau * tau / 2.0;
                a1[c] = Fo[3 * k + c] + Fx;
                j1[c] = Jo[3 * k + c] + Jx;
            }
        } else {
            double Fold[3], Jold[3], a2r[3], a3r[3];
            const double H = t - D.Tr[i];
            lr_old = D.LR[i];
            for (int c = 0; c < 3; ++c) {
                const int64_t q = 3 * i + c;
                a1[c] = Fa[3 * p + c];
                j1[c] = Ja[3 * p + c];
                Fold[c] = a1[c] - Fo[3 * k + c];
                Jold[c] = j1[c] - Jo[3 * k + c];
                const double df = D.Fr[q] - Fold[c];
                const double a2 = (-6.0 * df - H * (4.0 * D.Jr[q] + 2.0 * Jold[c])) / (H * H);
                const double a3 = (12.0 * df + 6.0 * H * (D.Jr[q] + Jold[c])) / (H * H * H);
                a2r[c] = a2 + H * a3;
                a3r[c] = a3;
            }
            const double critR = ac_crit(D.eta_reg, Fold, Jold, a2r, a3r);
            D.LR[i] = ac_level_rule(D.LR[i], critR, t_ticks, D.lmin, D.lmax);
            for (int c = 0; c < 3; ++c) {
                const int64_t q = 3 * i + c;
                D.Fr[q] = a1[c] - Fn[3 * p + c];
                D.Jr[q] = j1[c] - Jn[3 * p + c];
                D.D2[q] = a2r[c];
                D.D3[q] = a3r[c];
            }
            D.Tr[i] = t;
            if (D.nb_opt > 0) {
                const int32_t ct = cnt_true[p];
                double f = pow((double)D.nb_opt / (double)(ct > 0 ? ct : 1), 2.0 / 3.0);
                f = f < 0.5 ? 0.5 : (f > 2.0 ? 2.0 : f);
                D.rs2[i] *= f;
            }
        }
        // Hermite corrector on the total force; the predicted state is recomputed here with
        // the predictor's own function (bit-identical to the all-particle predictor)
        const double h = t - D.tl[i];
        double a2[3], a3[3], a2e[3];
        for (int c = 0; c < 3; ++c) {
            const int64_t q = 3 * i + c;
            double xp, vp;
            hermite_taylor(D.x[q], D.v[q], D.a[q], D.jk[q], h, xp, vp);
            double x1, v1;
            hermite_correct(xp, vp, D.a[q], D.jk[q], a1[c], j1[c], h, x1, v1, a2[c], a3[c]);
            D.x[q] = x1;
            D.v[q] = v1;
            D.a[q] = a1[c];
            D.jk[q] = j1[c];
            a2e[c] = a2[c] + h * a3[c];
        }
        D.tl[i] = t;
        const double crit = ac_crit(D.eta_irr, a1, j1, a2e, a3);
        int L = ac_level_rule(D.LI[i], crit, t_ticks, D.lmin, D.lmax);
        if (p >= 0) {
            if (D.LR[i] > L) D.LR[i] = L;  // regular step at least the new irregular step
            if (D.LR[i] != lr_old) {
                atomicSub(&D.lr_hist[lr_old], 1);
                atomicAdd(&D.lr_hist[D.LR[i]], 1);
            }
        } else if (L < D.LR[i]) {
            L = D.LR[i];  // irregular step at most the regular step
        }
        D.LI[i] = L;
        want[k] = L;
        pack_state_one(i, D.x + 3 * i, D.v + 3 * i, D.a + 3 * i, D.jk + 3 * i, t, D.m[i], D.s64, D.s32);
    }
    // the last CTA to finish publishes the final histogram and the step's status flags to the
    // host words (read after the scheduler's synchronisation) and clears the flags
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&D.tickets[1], 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) {
        __threadfence();
        for (int b = threadIdx.x; b < 64; b += blockDim.x) D.io[b] = __ldcg(&D.lr_hist[b]);
        if (threadIdx.x == 0) {
            D.io[64] = (int32_t)atomicExch(status, 0u);
            atomicExch(&D.tickets[1], 0u);
        }
    }
}

// The regular subset's new lists (CSR) replace the old per-particle lists; one warp per row.
__global__ void k_ac_lists(AcDev D, int64_t n_reg, const int32_t *reg_idx, const int64_t *off, const int32_t *csr)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = w0; p < n_reg; p += nw) {
        const int32_t i = reg_idx[p];
        const int64_t e0 = off[p], len = off[p + 1] - off[p];
        for (int64_t e = lane; e < len; e += 32) D.ell[(int64_t)i * D.cap + e] = csr[e0 + e];
        if (lane == 0) D.ell_cnt[i] = (int32_t)len;
    }
}

// The regular subset the classifier found must be the one the level histogram predicted.

__global__ void k_ac_hist(AcDev D, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&D.lr_hist[D.LR[i]], 1);
}

__global__ void k_ac_get_steps(const AcDev D, int64_t n, double *dt, double *DT, double *T)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (dt) dt[i] = ldexp(1.0, -D.LI[i]);
        if (DT) DT[i] = ldexp(1.0, -D.LR[i]);
        if (T) T[i] = D.Tr[i];
    }
}

static int grid_of(int64_t n, int block, int cap_ctas)
{
    int64_t g = (n + block - 1) / block;
    if (g > cap_ctas) g = cap_ctas;
    return g < 1 ? 1 : (int)g;
}

}  // namespace nbgpu

using namespace nbgpu;

struct nb_ac {
    nb_ctx *ctx = nullptr;
    nb_sched *sched = nullptr;
    CtxState cs{};
    AcDev D{};
    int64_t n = 0;
    nb_ac_params p{};
    // scratch
    int32_t *reg_pos = nullptr, *reg_idx = nullptr, *want = nullptr, *cnt_true = nullptr, *csr = nullptr;
    int64_t *off = nullptr;
    double *reg_rs2 = nullptr, *Fo = nullptr, *Jo = nullptr, *Po = nullptr, *Fa = nullptr, *Ja = nullptr,
           *Pa = nullptr, *Fn = nullptr, *Jn = nullptr, *Pn = nullptr;
    unsigned *counter = nullptr;  // regular rows classified so far in this step (reset by the last CTA)
    void *srec = nullptr;  // state records (pack_state_one layout of the context's precision)
    unsigned long long *pairs = nullptr;
    int32_t *h_io = nullptr;       // pinned, mapped: [0, 64) regular-level histogram, [64] status flags
    int32_t *h_lr = nullptr;       // = h_io
    unsigned *h_status = nullptr;  // = h_io + 64: the context's status flags of the last block step
    bool overflow = false;         // some neighbour list was cut at nb_cap
    double stats[6] = {0, 0, 0, 0, 0, 0};
    char err[384] = {0};
};

static nb_status afail(nb_ac *s, nb_status st, const char *fmt, ...)
{
    if (s) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(s->err, sizeof(s->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

#define ACK(call, what)                                                                            \
    do {                                                                                           \
        cudaError_t _e = (call);                                                                   \
        if (_e != cudaSuccess) return afail(s, NB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(_e)); \
    } while (0)

#define ANB(call, what)                                                                  \
    do {                                                                                 \
        nb_status _s = (call);                                                           \
        if (_s != NB_OK && _s != NB_ERR_NB_OVERFLOW)                                     \
            return afail(s, _s, "%s: %s", what, nb_last_error(s->ctx));                  \
    } while (0)

// Device arrays of the integrator and its per-step scratch (sizes from n and the list cap).
static bool ac_alloc(nb_ac *s, int64_t n, int cap)
{
    const size_t v3 = (size_t)n * 3 * sizeof(double);
    AcDev &D = s->D;
    const bool ok =
        cudaMalloc(&D.Fr, v3) == cudaSuccess && cudaMalloc(&D.Jr, v3) == cudaSuccess &&
        cudaMalloc(&D.D2, v3) == cudaSuccess && cudaMalloc(&D.D3, v3) == cudaSuccess &&
        cudaMalloc(&D.rs2, n * 8) == cudaSuccess && cudaMalloc(&D.Tr, n * 8) == cudaSuccess &&
        cudaMalloc(&D.LR, n * 4) == cudaSuccess && cudaMalloc(&D.LI, n * 4) == cudaSuccess &&
        cudaMalloc(&D.ell, (size_t)n * cap * 4) == cudaSuccess && cudaMalloc(&D.ell_cnt, n * 4) == cudaSuccess &&
        cudaMalloc(&s->reg_pos, n * 4) == cudaSuccess && cudaMalloc(&s->reg_idx, n * 4) == cudaSuccess &&
        cudaMalloc(&s->want, n * 4) == cudaSuccess && cudaMalloc(&s->cnt_true, n * 4) == cudaSuccess &&
        cudaMalloc(&s->csr, (size_t)n * cap * 4 + 4) == cudaSuccess && cudaMalloc(&s->off, (n + 1) * 8) == cudaSuccess &&
        cudaMalloc(&s->reg_rs2, n * 8) == cudaSuccess && cudaMalloc(&s->Fo, v3) == cudaSuccess &&
        cudaMalloc(&s->Jo, v3) == cudaSuccess && cudaMalloc(&s->Po, n * 8) == cudaSuccess &&
        cudaMalloc(&s->Fa, v3) == cudaSuccess && cudaMalloc(&s->Ja, v3) == cudaSuccess &&
        cudaMalloc(&s->Pa, n * 8) == cudaSuccess && cudaMalloc(&s->Fn, v3) == cudaSuccess &&
        cudaMalloc(&s->Jn, v3) == cudaSuccess && cudaMalloc(&s->Pn, n * 8) == cudaSuccess &&
        cudaMalloc(&s->counter, 4) == cudaSuccess &&
        cudaMalloc(&s->pairs, 8) == cudaSuccess && cudaMalloc(&D.lr_hist, 64 * 4) == cudaSuccess &&
        cudaMalloc(&D.tickets, 2 * 4) == cudaSuccess &&
        cudaHostAlloc(&s->h_io, 80 * 4, cudaHostAllocMapped) == cudaSuccess &&
        cudaHostGetDevicePointer((void **)&D.io, s->h_io, 0) == cudaSuccess &&
        cudaMemset(D.lr_hist, 0, 64 * 4) == cudaSuccess && cudaMemset(s->pairs, 0, 8) == cudaSuccess &&
        cudaMemset(D.tickets, 0, 2 * 4) == cudaSuccess && cudaMemset(s->counter, 0, 4) == cudaSuccess &&
        cudaMalloc(&s->srec, state_record_bytes(s->cs.precision, n)) == cudaSuccess;
    if (!ok) cudaGetLastError();
    s->h_lr = s->h_io;
    s->h_status = s->h_io ? reinterpret_cast<unsigned *>(s->h_io + 64) : nullptr;
    return ok;
}

static void ac_bind(nb_ac *s, const nb_ac_params *p, int lmin)
{
    AcDev &D = s->D;
    D.x = s->cs.x; D.v = s->cs.v; D.a = s->cs.a; D.jk = s->cs.jk; D.tl = s->cs.tl; D.m = s->cs.m;
    D.s64 = s->cs.precision == NB_FP64 ? static_cast<dvec4 *>(s->srec) : nullptr;
    D.s32 = s->cs.precision == NB_FP64 ? nullptr : static_cast<float4 *>(s->srec);
    D.cap = s->cs.cap;
    D.lmin = lmin;
    D.lmax = p->level_max;
    D.eta_irr = p->eta_irr;
    D.eta_reg = p->eta_reg;
    D.dt_max = p->dt_max;
    D.nb_opt = p->nb_opt;
}

// Level of dt_max = 2^-lmin, or -1 if dt_max is not a power of 1/2 in range.
// The scheduler must order its work after the integrator's kernels: it runs on the context's
// stream, which for a context on the legacy default stream is named by its handle (a null
// stream would give the scheduler a stream of its own).
static void *sched_stream(cudaStream_t st) { return st ? (void *)st : (void *)cudaStreamLegacy; }

static int params_lmin(const nb_ac_params *p)
{
    if (!(p->dt_max > 0.0) || p->level_max > kAcTick || !(p->eta_irr > 0.0) || !(p->eta_reg > 0.0) ||
        !(p->eta_s > 0.0))
        return -1;
    int fe = 0;
    const double fr = std::frexp(p->dt_max, &fe);
    const int lmin = 1 - fe;
    return (fr != 0.5 || lmin < 0 || lmin > p->level_max) ? -1 : lmin;
}

// Snapshot layout: header, then the arrays in this order.
struct AcSnapshotHeader {
    char magic[8];
    int64_t n;
    int32_t cap, precision;
    nb_ac_params params;
    double t_now;
    double stats[6];
};
static constexpr char kSnapMagic[8] = {'N', 'B', 'A', 'C', 'S', 'N', 'P', '1'};

struct SnapField {
    void *dev;
    size_t bytes;
};

static int snap_fields(nb_ac *s, SnapField *f)
{
    const int64_t n = s->n;
    const size_t v3 = (size_t)n * 24, s1 = (size_t)n * 8, i1 = (size_t)n * 4;
    const AcDev &D = s->D;
    int k = 0;
    f[k++] = {D.x, v3};  f[k++] = {D.v, v3};  f[k++] = {D.a, v3};  f[k++] = {D.jk, v3};
    f[k++] = {D.tl, s1}; f[k++] = {D.m, s1};
    f[k++] = {D.Fr, v3}; f[k++] = {D.Jr, v3}; f[k++] = {D.D2, v3}; f[k++] = {D.D3, v3};
    f[k++] = {D.rs2, s1}; f[k++] = {D.Tr, s1};
    f[k++] = {D.LR, i1}; f[k++] = {D.LI, i1}; f[k++] = {D.ell_cnt, i1};
    f[k++] = {D.ell, (size_t)n * D.cap * 4};
    return k;
}

extern "C" {

nb_status nb_ac_init(nb_ac **out, nb_ctx *ctx, int64_t n, const double *m, const double *x, const double *v,
                     const double *rs2, const nb_ac_params *p, int32_t on_device)
{
    if (!out) return NB_ERR_ARG;
    *out = nullptr;
    if (!ctx || !m || !x || !v || !rs2 || !p || n < 1) return NB_ERR_ARG;
    const int lmin = params_lmin(p);  // dt_max = 2^-lmin
    if (lmin < 0) return NB_ERR_ARG;
    nb_ac *s = new (std::nothrow) nb_ac();
    if (!s) return NB_ERR_OOM;
    s->ctx = ctx;
    s->n = n;
    s->p = *p;
    auto bail = [&](nb_status st) {
        nb_ac_free(s);
        return st;
    };
    // the context takes the state at t = 0: zero force and jerk until the first evaluation
    {
        double *z = nullptr;
        if (cudaMalloc(&z, (size_t)n * 3 * sizeof(double)) != cudaSuccess) return bail(NB_ERR_OOM);
        cudaMemset(z, 0, (size_t)n * 3 * sizeof(double));
        const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        double *dx = nullptr, *dv = nullptr, *dm = nullptr;
        if (cudaMalloc(&dx, n * 24) != cudaSuccess || cudaMalloc(&dv, n * 24) != cudaSuccess ||
            cudaMalloc(&dm, n * 8) != cudaSuccess) {
            cudaFree(z); cudaFree(dx); cudaFree(dv); cudaFree(dm);
            return bail(NB_ERR_OOM);
        }
        cudaMemcpy(dx, x, n * 24, k);
        cudaMemcpy(dv, v, n * 24, k);
        cudaMemcpy(dm, m, n * 8, k);
        nb_status st = nb_set_particles(ctx, n, dx, dv, z, z, dm, z, 1);
        if (st == NB_OK) st = nb_sync(ctx);
        cudaFree(z); cudaFree(dx); cudaFree(dv); cudaFree(dm);
        if (st != NB_OK) return bail(afail(s, st, "nb_set_particles: %s", nb_last_error(ctx)));
    }
    if (!ctx_state(ctx, &s->cs)) return bail(NB_ERR_STATE);
    if (!ac_alloc(s, n, s->cs.cap)) return bail(NB_ERR_OOM);
    ac_bind(s, p, lmin);
    const int cap = s->cs.cap;
    cudaStream_t st = s->cs.stream;
    AcDev &D = s->D;
    ACK(cudaMemcpyAsync(D.rs2, rs2, n * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st),
        "copy rs2");
    // all forces and lists at t = 0
    ANB(nb_predict(ctx, 0.0), "nb_predict");
    k_iota32<<<grid_of(n, 256, 152 * 16), 256, 0, st>>>(s->reg_idx, n);
    ANB(nb_regular_force(ctx, n, s->reg_idx, D.rs2, 0, s->Fa, s->Ja, s->Pa, s->off, s->csr, n * cap, s->cnt_true, 1),
        "nb_regular_force");
    launch_irregular(st, s->cs.precision, s->cs.num_sms, s->cs.rec, 1, n, 0.0, n, s->reg_idx, s->off, s->csr, s->Fn,
                     s->Jn, s->Pn, nullptr, nullptr, nullptr, s->cs.status);
    k_ac_init<<<grid_of(n, 256, 152 * 16), 256, 0, st>>>(D, n, s->Fa, s->Ja, s->Fn, s->Jn, s->off, s->csr, p->eta_s,
                                                          s->want);
    ACK(cudaGetLastError(), "init launch");
    ACK(cudaMemcpyAsync(s->h_lr, D.lr_hist, 64 * 4, cudaMemcpyDeviceToHost, st), "copy histogram");
    ANB(nb_sync(ctx), "initial forces");
    nb_status ss = nb_sched_init(&s->sched, n, s->want, lmin, p->level_max, s->cs.device, sched_stream(st), 1);
    if (ss != NB_OK) return bail(afail(s, ss, "nb_sched_init"));
    *out = s;
    return NB_OK;
}

// One block step with a single host synchronisation (inside nb_sched_update): the size of the
// regular subset follows from the histogram of regular levels published by the previous step
// (a particle takes a regular step exactly when its regular level is >= L*, the coarsest
// level whose step divides the block time), so the regular force is launched without
// waiting. The last CTA of the classify launch checks that size against the classified
// count; the last CTA of the corrector writes the new histogram and the step's status flags
// into mapped host words, which the scheduler's synchronisation makes visible. A step with no
// regular particle is three launches (irregular force, corrector, re-sort: the corrector
// then checks that no particle was due for a regular step) and one synchronisation.
nb_status nb_ac_step(nb_ac *s, double *t_block, int64_t *n_active, int64_t *n_regular)
{
    if (!s) return NB_ERR_ARG;
    double t = 0.0;
    int64_t na = 0;
    const int32_t *list = nullptr;
    nb_status ss = nb_sched_next(s->sched, &t, &na, &list);
    if (ss != NB_OK) return afail(s, ss, "nb_sched_next: %s", nb_sched_last_error(s->sched));
    const CtxState &cs = s->cs;
    cudaStream_t st = cs.stream;
    const int64_t t_ticks = (int64_t)std::ldexp(t, kAcTick);
    int tz = 0;
    while (tz < kAcTick && ((t_ticks >> tz) & 1) == 0) ++tz;
    const int lstar = kAcTick - tz;
    int64_t nr = 0;
    for (int b = lstar; b < 64; ++b) nr += s->h_lr[b];
    const int cap = cs.cap;
    if (nr > 0) {  // with no regular particle predicted the corrector makes the check itself
        k_ac_classify<<<grid_of(na, 256, 152 * 16), 256, 0, st>>>(s->D, na, list, t_ticks, s->counter, s->reg_pos,
                                                                   s->reg_idx, s->reg_rs2, nr, cs.status + SS_FLAGS);
        ACK(cudaGetLastError(), "classify launch");
    }
    if (nr > 0) {
        ANB(nb_predict(s->ctx, t), "nb_predict");
        ANB(nb_regular_force(s->ctx, nr, s->reg_idx, s->reg_rs2, 0, s->Fa, s->Ja, s->Pa, s->off, s->csr, nr * cap,
                             s->cnt_true, 1),
            "nb_regular_force");
        launch_irregular(st, cs.precision, cs.num_sms, cs.rec, 1, cs.n, t, na, list, nullptr, s->D.ell, s->Fo, s->Jo,
                         s->Po, nullptr, nullptr, nullptr, cs.status, s->D.ell_cnt, cap);
        launch_irregular(st, cs.precision, cs.num_sms, cs.rec, 1, cs.n, t, nr, s->reg_idx, s->off, s->csr, s->Fn,
                         s->Jn, s->Pn, nullptr, nullptr, nullptr, cs.status);
    } else {  // no all-particle work: the active particles and their neighbours predicted on load
        launch_irregular(st, cs.precision, cs.num_sms, s->srec, 0, cs.n, t, na, list, nullptr, s->D.ell, s->Fo,
                         s->Jo, s->Po, nullptr, nullptr, nullptr, cs.status, s->D.ell_cnt, cap);
    }
    k_ac_correct<<<grid_of(na, 128, 152 * 32), 128, 0, st>>>(s->D, na, list, t, t_ticks,
                                                              nr > 0 ? s->reg_pos : nullptr, s->Fo, s->Jo,
                                                              s->Fa, s->Ja, s->Fn, s->Jn, s->cnt_true, s->want,
                                                              s->pairs, cs.status + SS_FLAGS);
    if (nr > 0) k_ac_lists<<<grid_of(nr * 32, 256, 152 * 16), 256, 0, st>>>(s->D, nr, s->reg_idx, s->off, s->csr);
    ACK(cudaGetLastError(), "corrector launch");
    ctx_state_changed(s->ctx);  // the corrector rewrote the context's state arrays
    ss = nb_sched_update(s->sched, s->want, nullptr, 1);  // synchronises the stream
    if (ss != NB_OK) return afail(s, ss, "nb_sched_update: %s", nb_sched_last_error(s->sched));
    const unsigned f = *s->h_status;
    if (f & (ST_BAD_INDEX | ST_DUP_INDEX | ST_DEVICE | ST_TIMEOUT))
        return afail(s, NB_ERR_DEVICE, "block step at t = %.17g: device status 0x%x", t, f);
    if (f & (ST_NB_TRUNCATED | ST_CSR_FULL)) s->overflow = true;
    s->stats[0] += 1;
    s->stats[1] += (double)na;
    s->stats[2] += (double)nr;
    s->stats[4] += (double)nr * (double)(cs.n - 1);
    if (t_block) *t_block = t;
    if (n_active) *n_active = na;
    if (n_regular) *n_regular = nr;
    return NB_OK;
}

// Counters of the run so far (the neighbour-pair count lives on the device).
static nb_status ac_read_stats(nb_ac *s)
{
    unsigned long long pairs = 0;
    ACK(cudaMemcpyAsync(&pairs, s->pairs, 8, cudaMemcpyDeviceToHost, s->cs.stream), "copy pairs");
    ACK(cudaStreamSynchronize(s->cs.stream), "cudaStreamSynchronize");
    s->stats[3] = (double)pairs;
    return NB_OK;
}

nb_status nb_ac_run(nb_ac *s, double t_end, int64_t max_blocks, double *stats)
{
    if (!s) return NB_ERR_ARG;
    int64_t b = 0;
    nb_status rc = NB_OK;
    for (;;) {
        double tn = 0.0;
        nb_status ss = nb_sched_peek(s->sched, &tn);
        if (ss != NB_OK) return afail(s, ss, "nb_sched_peek");
        if (tn > t_end) break;
        if (max_blocks > 0 && b >= max_blocks) {
            rc = NB_ERR_STATE;
            afail(s, rc, "max_blocks reached");
            break;
        }
        if ((ss = nb_ac_step(s, nullptr, nullptr, nullptr)) != NB_OK) return ss;
        ++b;
    }
    if (stats) {
        nb_status ss = ac_read_stats(s);
        if (ss != NB_OK) return ss;
        memcpy(stats, s->stats, sizeof(s->stats));
    }
    return rc;
}

nb_status nb_ac_get(nb_ac *s, double *x, double *v, double *t, double *dt, double *DT, double *T, double *rs2,
                    int32_t *nb_count, int32_t *nb_lists, int32_t on_device)
{
    if (!s) return NB_ERR_ARG;
    const int64_t n = s->n;
    cudaStream_t st = s->cs.stream;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (x) ACK(cudaMemcpyAsync(x, s->D.x, n * 24, k, st), "copy x");
    if (v) ACK(cudaMemcpyAsync(v, s->D.v, n * 24, k, st), "copy v");
    if (t) ACK(cudaMemcpyAsync(t, s->D.tl, n * 8, k, st), "copy t");
    if (rs2) ACK(cudaMemcpyAsync(rs2, s->D.rs2, n * 8, k, st), "copy rs2");
    if (nb_count) ACK(cudaMemcpyAsync(nb_count, s->D.ell_cnt, n * 4, k, st), "copy counts");
    if (nb_lists) ACK(cudaMemcpyAsync(nb_lists, s->D.ell, (size_t)n * s->D.cap * 4, k, st), "copy lists");
    if (dt || DT || T) {
        double *tmp = s->Fo;  // 3n doubles of scratch
        k_ac_get_steps<<<grid_of(n, 256, 152 * 16), 256, 0, st>>>(s->D, n, dt ? tmp : nullptr, DT ? tmp + n : nullptr,
                                                                   T ? tmp + 2 * n : nullptr);
        ACK(cudaGetLastError(), "steps launch");
        if (dt) ACK(cudaMemcpyAsync(dt, tmp, n * 8, k, st), "copy dt");
        if (DT) ACK(cudaMemcpyAsync(DT, tmp + n, n * 8, k, st), "copy DT");
        if (T) ACK(cudaMemcpyAsync(T, tmp + 2 * n, n * 8, k, st), "copy T");
    }
    ACK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    return NB_OK;
}

nb_status nb_ac_snapshot_bytes(nb_ac *s, size_t *bytes)
{
    if (!s || !bytes) return NB_ERR_ARG;
    SnapField f[32];
    const int k = snap_fields(s, f);
    size_t b = sizeof(AcSnapshotHeader);
    for (int q = 0; q < k; ++q) b += f[q].bytes;
    *bytes = b;
    return NB_OK;
}

nb_status nb_ac_save(nb_ac *s, void *buf, size_t bytes)
{
    if (!s || !buf) return NB_ERR_ARG;
    size_t need = 0;
    nb_ac_snapshot_bytes(s, &need);
    if (bytes < need) return afail(s, NB_ERR_ARG, "snapshot needs %zu bytes", need);
    AcSnapshotHeader h{};
    memcpy(h.magic, kSnapMagic, 8);
    h.n = s->n;
    h.cap = s->D.cap;
    h.precision = s->cs.precision;
    h.params = s->p;
    nb_status ss = nb_sched_get(s->sched, nullptr, nullptr, &h.t_now, 0);
    if (ss != NB_OK) return afail(s, ss, "nb_sched_get");
    if ((ss = ac_read_stats(s)) != NB_OK) return ss;
    memcpy(h.stats, s->stats, sizeof(h.stats));
    char *out = static_cast<char *>(buf);
    memcpy(out, &h, sizeof(h));
    size_t o = sizeof(h);
    SnapField f[32];
    const int k = snap_fields(s, f);
    for (int q = 0; q < k; ++q) {
        ACK(cudaMemcpyAsync(out + o, f[q].dev, f[q].bytes, cudaMemcpyDeviceToHost, s->cs.stream), "copy state");
        o += f[q].bytes;
    }
    ACK(cudaStreamSynchronize(s->cs.stream), "cudaStreamSynchronize");
    return NB_OK;
}

nb_status nb_ac_restore(nb_ac **out, nb_ctx *ctx, const void *buf, size_t bytes)
{
    if (!out) return NB_ERR_ARG;
    *out = nullptr;
    if (!ctx || !buf || bytes < sizeof(AcSnapshotHeader)) return NB_ERR_ARG;
    AcSnapshotHeader h;
    memcpy(&h, buf, sizeof(h));
    const int lmin = params_lmin(&h.params);
    if (memcmp(h.magic, kSnapMagic, 8) != 0 || h.n < 1 || lmin < 0) return NB_ERR_ARG;
    nb_ac *s = new (std::nothrow) nb_ac();
    if (!s) return NB_ERR_OOM;
    s->ctx = ctx;
    s->n = h.n;
    s->p = h.params;
    memcpy(s->stats, h.stats, sizeof(h.stats));
    auto bail = [&](nb_status st) {
        nb_ac_free(s);
        return st;
    };
    const int64_t n = h.n;
    const char *in = static_cast<const char *>(buf);
    const size_t v3 = (size_t)n * 24, s1 = (size_t)n * 8, o0 = sizeof(h);
    // the particle state goes to the context first (it checks n against its capacity)
    const double *hx = (const double *)(in + o0), *hv = (const double *)(in + o0 + v3),
                 *ha = (const double *)(in + o0 + 2 * v3), *hj = (const double *)(in + o0 + 3 * v3),
                 *ht = (const double *)(in + o0 + 4 * v3), *hm = (const double *)(in + o0 + 4 * v3 + s1);
    nb_status st0 = nb_set_particles(ctx, n, hx, hv, ha, hj, hm, ht, 0);
    if (st0 != NB_OK) return bail(afail(s, st0, "nb_set_particles: %s", nb_last_error(ctx)));
    if (!ctx_state(ctx, &s->cs)) return bail(NB_ERR_STATE);
    if (s->cs.cap != h.cap || s->cs.precision != h.precision)
        return bail(afail(s, NB_ERR_ARG, "the context's nb_cap / precision differ from the snapshot's"));
    if (!ac_alloc(s, n, h.cap)) return bail(NB_ERR_OOM);
    ac_bind(s, &h.params, lmin);
    SnapField f[32];
    const int k = snap_fields(s, f);
    size_t need = sizeof(h);
    for (int q = 0; q < k; ++q) need += f[q].bytes;
    if (bytes < need) return bail(afail(s, NB_ERR_ARG, "snapshot truncated"));
    size_t o = sizeof(h);
    for (int q = 0; q < k; ++q) {
        if (cudaMemcpyAsync(f[q].dev, in + o, f[q].bytes, cudaMemcpyHostToDevice, s->cs.stream) != cudaSuccess)
            return bail(NB_ERR_CUDA);
        o += f[q].bytes;
    }
    launch_pack_state(s->cs.stream, s->cs.precision, n, s->D.x, s->D.v, s->D.a, s->D.jk, s->D.tl, s->D.m, s->srec);
    // LI follows x, v, a, jk (4 v3), tl, m (2 s1), Fr, Jr, D2, D3 (4 v3), rs2, Tr (2 s1), LR
    const int32_t *levels = (const int32_t *)(in + sizeof(h) + 8 * v3 + 4 * s1 + (size_t)n * 4);
    nb_status ss =
        nb_sched_init(&s->sched, n, levels, lmin, h.params.level_max, s->cs.device, sched_stream(s->cs.stream), 0);
    if (ss == NB_OK) ss = nb_sched_set_time(s->sched, h.t_now);
    if (ss != NB_OK) return bail(afail(s, ss, "scheduler"));
    const unsigned long long pairs = (unsigned long long)h.stats[3];
    if (cudaMemcpyAsync(s->pairs, &pairs, 8, cudaMemcpyHostToDevice, s->cs.stream) != cudaSuccess)
        return bail(NB_ERR_CUDA);
    k_ac_hist<<<grid_of(n, 256, 152 * 16), 256, 0, s->cs.stream>>>(s->D, n);
    if (cudaMemcpyAsync(s->h_lr, s->D.lr_hist, 64 * 4, cudaMemcpyDeviceToHost, s->cs.stream) != cudaSuccess)
        return bail(NB_ERR_CUDA);
    if (cudaStreamSynchronize(s->cs.stream) != cudaSuccess) return bail(NB_ERR_CUDA);
    *out = s;
    return NB_OK;
}

nb_status nb_ac_free(nb_ac *s)
{
    if (!s) return NB_OK;
    if (s->cs.stream) cudaStreamSynchronize(s->cs.stream);
    if (s->sched) nb_sched_free(s->sched);
    void *p[] = {s->D.Fr, s->D.Jr, s->D.D2, s->D.D3, s->D.rs2, s->D.Tr, s->D.LR, s->D.LI, s->D.ell, s->D.ell_cnt,
                 s->reg_pos, s->reg_idx, s->want, s->cnt_true, s->csr, s->off, s->reg_rs2, s->Fo, s->Jo, s->Po,
                 s->Fa, s->Ja, s->Pa, s->Fn, s->Jn, s->Pn, s->counter, s->pairs, s->D.lr_hist, s->D.tickets, s->srec};
    for (void *q : p)
        if (q) cudaFree(q);
    if (s->h_io) cudaFreeHost(s->h_io);
    delete s;
    return NB_OK;
}

const char *nb_ac_last_error(const nb_ac *s) { return s ? s->err : "null integrator"; }

}  // extern "C"
