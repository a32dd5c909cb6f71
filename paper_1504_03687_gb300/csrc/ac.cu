// ac.cu — K9: the Ahmad-Cohen Hermite block step on the device (paper Sec. 2; the scheme
// is stated with the declarations in nbgpu.h).  One block step is a fixed sequence of
// launches on the context stream:
//   nb_sched_next (host)          -> block time t, active particles = list prefix
//   k_ac_classify_count, _place   -> which active particles also take a regular step, in
//                                    list order (only when the regular-level histogram
//                                    predicts some)
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
// nb_ac_run drives runs of block steps without a regular subset from the device instead: per
// step one launch of k_ac_irregular_step (irregular force, corrector, step rule; its last CTA
// re-sorts the prefix and selects the next step into StepParams), enqueued in batches sized
// from the level histograms, each launch a programmatic dependent of the one before, one host
// synchronisation per batch.  Both paths give the same bits.
// The corrector's FP64 arithmetic is written operation by operation in the order of the
// plain definition (its divisions by powers of two as exact scalings) and this file is
// compiled without FMA contraction, so an FP64 context follows the reference integration to
// rounding.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "nbgpu.h"
#include "nb_common.cuh"
#include "nb_irregular.cuh"
#include "nb_kernels.cuh"
#include "nb_sched.cuh"

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
    unsigned *tickets; // [2] CTAs done in the fused block-step and corrector launches (last-CTA epilogues)
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
    const double h = pow2i(-L);
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

// The step rule's level for the criterion of ac_crit, decided on an FP32 estimate where that
// is provably the FP64 decision; -1 where it is not (the caller then evaluates ac_crit).  A, J,
// A2, A3 are FP32 sums of squares of the FP32-rounded components of a, jerk, a2 and a3, so
//   crit^2 = eta (sqrt(A A2) + J) / (sqrt(J A3) + A2)
// is the square of ac_crit's value, computed to a relative error below 18 * 2^-24 < 2^-19 (as
// long as every quantity is a normal FP32 number; ac_crit's own rounding is far smaller).  The
// rule compares crit only with powers of two, so where the estimate of crit^2 is at least
// 2^-14 (relative) from every power of two, the FP64 criterion lies on the same side of each
// of them and the rule on the estimate gives the same level.  Only a row whose crit^2 falls
// within that margin of a power of two (about one in 8000) takes the FP64 criterion.
__device__ __forceinline__ int ac_level_rule_est(int L, float A, float J, float A2, float A3, float eta,
                                                 int64_t t_ticks, int lmin, int lmax)
{
    const float AA2 = __fmul_rn(A, A2), JA3 = __fmul_rn(J, A3);
    const float num = __fadd_rn(__fsqrt_rn(AA2), J), den = __fadd_rn(__fsqrt_rn(JA3), A2);
    const float c2 = __fdiv_rn(__fmul_rn(eta, num), den);
    auto normal = [](float x) { return x >= 1.17549435e-38f && x <= 3.40282347e38f; };  // false for NaN
    if (!(normal(A) && normal(J) && normal(A2) && normal(A3) && normal(AA2) && normal(JA3) && normal(num) &&
          normal(den) && normal(c2)))
        return -1;
    const unsigned m = __float_as_uint(c2) & 0x7FFFFFu;
    if (m < (1u << 9) || m > 0x7FFFFFu - (1u << 9)) return -1;  // within 2^-14 of a power of two
    const float crit = __fsqrt_rn(c2);
    const float h = __uint_as_float((unsigned)(127 - L) << 23);  // 2^-L, exactly
    if (crit < h) {
        int Ln = L;
        float hn = h;
        while (hn > crit && Ln < lmax) {
            hn *= 0.5f;
            ++Ln;
        }
        return Ln;
    }
    if (crit >= 2.0f * h && L - 1 >= lmin && (t_ticks & (((int64_t)1 << (kAcTick - (L - 1))) - 1)) == 0)
        return L - 1;
    return L;
}

// ac_level_rule(L, ac_crit(eta, a, j, a2, a3), ...) for one thread's three components: decided
// on the FP32 estimate where that provably gives the same level, on the FP64 criterion
// otherwise (the sums of squares are formed as in the fused step kernel, ((x0^2 + x1^2) + x2^2)).
__device__ __forceinline__ int ac_level_rule_vec(double eta, const double *a, const double *j, const double *a2,
                                                 const double *a3, int L, int64_t t_ticks, int lmin, int lmax)
{
    float sq[4] = {0.f, 0.f, 0.f, 0.f};
    const double *v[4] = {a, j, a2, a3};
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float x = __double2float_rn(v[u][c]);
            sq[u] = c == 0 ? __fmul_rn(x, x) : __fadd_rn(sq[u], __fmul_rn(x, x));
        }
    const int Le = ac_level_rule_est(L, sq[0], sq[1], sq[2], sq[3], (float)eta, t_ticks, lmin, lmax);
    return Le >= 0 ? Le : ac_level_rule(L, ac_crit(eta, a, j, a2, a3), t_ticks, lmin, lmax);
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

// Active row k: regular step too?  The regular subset is compacted in list order (the order
// is deterministic, so the regular force, whose anchored kernel groups rows into CTAs by their
// order, gives the same bits every run): CTA b owns the list chunk [b kClassifyChunk,
// (b + 1) kClassifyChunk); the count pass writes the chunk's regular rows, the place pass turns
// the counts before b into the chunk's base and ranks its rows in order.
constexpr int kClassifyBlock = 256, kClassifyChunk = 1024;

__device__ __forceinline__ bool ac_regular_row(const AcDev &D, const int32_t *list, int64_t k, int64_t t_ticks)
{
    const int LR = D.LR[list[k]];
    return (t_ticks & (((int64_t)1 << (kAcTick - LR)) - 1)) == 0;
}

__global__ void __launch_bounds__(kClassifyBlock) k_ac_classify_count(AcDev D, int64_t n_act, const int32_t *list,
                                                                    int64_t t_ticks, int32_t *cta_count)
{
    __shared__ int32_t s_warp[kClassifyBlock / 32];
    const int64_t c0 = (int64_t)blockIdx.x * kClassifyChunk;
    int cnt = 0;
    for (int64_t k = c0 + threadIdx.x; k < n_act && k < c0 + kClassifyChunk; k += kClassifyBlock)
        cnt += ac_regular_row(D, list, k, t_ticks);
    cnt = warp_sum(cnt);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < kClassifyBlock / 32; ++w) tot += s_warp[w];
        cta_count[blockIdx.x] = tot;
    }
}

__global__ void __launch_bounds__(kClassifyBlock)
    k_ac_classify_place(AcDev D, int64_t n_act, const int32_t *list, int64_t t_ticks, const int32_t *cta_count,
                        int32_t *reg_pos, int32_t *reg_idx, double *reg_rs2, int64_t expected, unsigned *status)
{
    __shared__ int32_t s_warp[kClassifyBlock / 32];
    __shared__ int64_t s_part[kClassifyBlock / 32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    // the regular rows of the chunks before this one (CTA 0: of all chunks, for the check)
    const int nb = blockIdx.x == 0 ? (int)gridDim.x : (int)blockIdx.x;
    int64_t part = 0;
    for (int b = tid; b < nb; b += kClassifyBlock) part += cta_count[b];
    part = warp_sum(part);
    if (lane == 0) s_part[w] = part;
    __syncthreads();
    int64_t tot = 0;
    for (int q = 0; q < kClassifyBlock / 32; ++q) tot += s_part[q];
    // the host's prediction must be the classified count (else a device error of the step)
    if (blockIdx.x == 0 && tid == 0 && tot != expected) atomicOr(status, ST_DEVICE);
    int64_t run = blockIdx.x == 0 ? 0 : tot;
    const int64_t c0 = (int64_t)blockIdx.x * kClassifyChunk;
    for (int64_t r0 = c0; r0 < c0 + kClassifyChunk && r0 < n_act; r0 += kClassifyBlock) {
        const int64_t k = r0 + tid;
        const bool reg = k < n_act && ac_regular_row(D, list, k, t_ticks);
        const unsigned m = __ballot_sync(0xffffffffu, reg);
        if (lane == 0) s_warp[w] = __popc(m);
        __syncthreads();
        int64_t before = run;
        int round_total = 0;
        for (int q = 0; q < kClassifyBlock / 32; ++q) {
            if (q < w) before += s_warp[q];
            round_total += s_warp[q];
        }
        if (k < n_act) {
            int32_t p = -1;
            if (reg) {
                p = (int32_t)(before + __popc(m & ((1u << lane) - 1u)));
                const int32_t i = list[k];
                reg_idx[p] = i;
                reg_rs2[p] = D.rs2[i];
            }
            reg_pos[k] = p;
        }
        run += round_total;
        __syncthreads();  // s_warp is rewritten in the next round
    }
}

__global__ void k_ac_correct(AcDev D, int64_t n_act, const int32_t *list, double t, int64_t t_ticks,
                             const int32_t *reg_pos, const double *Fo, const double *Jo, const double *Fa,
                             const double *Ja, const double *Fn, const double *Jn, const int32_t *cnt_true,
                             int32_t *want, unsigned long long *pairs, unsigned *status)
{
    // CTAs past the rows have nothing to do and take no part in the last-CTA epilogue
    const int64_t per = (int64_t)gridDim.x * blockDim.x;
    const int64_t used = n_act <= 0 ? 1 : (n_act < per ? (n_act + blockDim.x - 1) / blockDim.x : gridDim.x);
    if (blockIdx.x >= used) return;
    unsigned long long my_pairs = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_act; k += per) {
        // every input is loaded before the first store: the state arrays are separate
        // allocations, but the compiler cannot know it and would otherwise order each load
        // behind the stores before it, a chain of dependent memory round trips per row
        const int32_t i = list[k];
        // reg_pos == null: the host predicted no regular particle in this step and skipped the
        // classify launch; a particle that is due for a regular step is then a device error
        const int32_t p = reg_pos ? reg_pos[k] : -1;
        const int LR0 = D.LR[i], LI0 = D.LI[i];
        const double Tr = D.Tr[i], tl = D.tl[i], mi = D.m[i];
        double x0[3], v0[3], a0[3], j0[3], Fr[3], Jr[3], D2[3], D3[3], fo[3], jo[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int64_t q = 3 * i + c;
            x0[c] = D.x[q];
            v0[c] = D.v[q];
            a0[c] = D.a[q];
            j0[c] = D.jk[q];
            Fr[c] = D.Fr[q];
            Jr[c] = D.Jr[q];
            D2[c] = D.D2[q];
            D3[c] = D.D3[q];
            fo[c] = Fo[3 * k + c];
            jo[c] = Jo[3 * k + c];
        }
        my_pairs += (unsigned long long)D.ell_cnt[i];
        if (!reg_pos && (t_ticks & (((int64_t)1 << (kAcTick - LR0)) - 1)) == 0) atomicOr(status, ST_DEVICE);
        double a1[3], j1[3];
        int LR = LR0;
        if (p < 0) {
            const double tau = t - Tr;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double Fx = Fr[c] + Jr[c] * tau + D2[c] * tau * tau / 2.0 + D3[c] * tau * tau * tau / 6.0;
                const double Jx = Jr[c] + D2[c] * tau + D3[c] * tau * tau / 2.0;
                a1[c] = fo[c] + Fx;
                j1[c] = jo[c] + Jx;
            }
        } else {
            double Fold[3], Jold[3], a2r[3], a3r[3], fn[3], jn[3];
            const double H = t - Tr, iH = 1.0 / H;  // H is the regular step, a power of two
            const int32_t ct = cnt_true[p];
            const double rs2 = D.rs2[i];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                a1[c] = Fa[3 * p + c];
                j1[c] = Ja[3 * p + c];
                fn[c] = Fn[3 * p + c];
                jn[c] = Jn[3 * p + c];
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                Fold[c] = a1[c] - fo[c];
                Jold[c] = j1[c] - jo[c];
                const double df = Fr[c] - Fold[c];
                // the definition's divisions by H^2 and H^3, as exact scalings
                const double a2 = (-6.0 * df - H * (4.0 * Jr[c] + 2.0 * Jold[c])) * (iH * iH);
                const double a3 = (12.0 * df + 6.0 * H * (Jr[c] + Jold[c])) * (iH * iH * iH);
                a2r[c] = a2 + H * a3;
                a3r[c] = a3;
            }
            LR = ac_level_rule_vec(D.eta_reg, Fold, Jold, a2r, a3r, LR0, t_ticks, D.lmin, D.lmax);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int64_t q = 3 * i + c;
                D.Fr[q] = a1[c] - fn[c];
                D.Jr[q] = j1[c] - jn[c];
                D.D2[q] = a2r[c];
                D.D3[q] = a3r[c];
            }
            D.Tr[i] = t;
            if (D.nb_opt > 0) {
                double f = pow((double)D.nb_opt / (double)(ct > 0 ? ct : 1), 2.0 / 3.0);
                f = f < 0.5 ? 0.5 : (f > 2.0 ? 2.0 : f);
                D.rs2[i] = rs2 * f;
            }
        }
        // Hermite corrector on the total force; the predicted state is recomputed here with
        // the predictor's own function (bit-identical to the all-particle predictor)
        const double h = t - tl, ih = 1.0 / h;  // h is the irregular step, a power of two
        double a2[3], a3[3], a2e[3], x1[3], v1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double xp, vp;
            hermite_taylor(x0[c], v0[c], a0[c], j0[c], h, xp, vp);
            hermite_correct_pow2(xp, vp, a0[c], j0[c], a1[c], j1[c], h, ih, x1[c], v1[c], a2[c], a3[c]);
            a2e[c] = a2[c] + h * a3[c];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int64_t q = 3 * i + c;
            D.x[q] = x1[c];
            D.v[q] = v1[c];
            D.a[q] = a1[c];
            D.jk[q] = j1[c];
        }
        D.tl[i] = t;
        int L = ac_level_rule_vec(D.eta_irr, a1, j1, a2e, a3, LI0, t_ticks, D.lmin, D.lmax);
        if (p >= 0) {
            if (LR > L) LR = L;  // regular step at least the new irregular step
            D.LR[i] = LR;
            if (LR != LR0) {
                atomicSub(&D.lr_hist[LR0], 1);
                atomicAdd(&D.lr_hist[LR], 1);
            }
        } else if (L < LR) {
            L = LR;  // irregular step at most the regular step
        }
        D.LI[i] = L;
        want[k] = L;
        pack_state_one(i, x1, v1, a1, j1, t, mi, D.s64, D.s32);
    }
    // one atomic per warp for the neighbour-pair count (a row's count is at most nb_cap)
    const unsigned wp = __reduce_add_sync(0xffffffffu, (unsigned)my_pairs);
    if ((threadIdx.x & 31) == 0 && wp) atomicAdd(pairs, (unsigned long long)wp);
    // the last CTA to finish publishes the final histogram and the step's status flags to the
    // host words (read after the scheduler's synchronisation; the flags are OR-ed in) and
    // clears the device flags
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&D.tickets[1], 1u) == (unsigned)used - 1;
    __syncthreads();
    if (last) {
        __threadfence();
        for (int b = threadIdx.x; b < 64; b += blockDim.x) D.io[b] = __ldcg(&D.lr_hist[b]);
        if (threadIdx.x == 0) {
            D.io[64] |= (int32_t)atomicExch(status, 0u);  // the host clears it after reading
            atomicExch(&D.tickets[1], 0u);
        }
    }
}

// A device-driven block step without a regular subset, in one kernel.  For every row of the
// step's prefix one warp computes the irregular force (the irregular force kernels' own
// per-row code: the lanes stride over the row's list, neighbours predicted on load from the
// state records, the same fixed-order warp reduction) and then the corrector of k_ac_correct's
// irregular branch, lane c < 3 taking component c (GB300's FP64 pipe takes about as long for a
// warp instruction with three lanes active as with 32, so three component chains in one
// instruction stream cost one).  The step rule is decided on an FP32 estimate of the criterion
// where that provably gives the FP64 decision (ac_level_rule_est), else on ac_crit.  The
// corrected state records go to rec_new[k] (list position), not to the records other rows are
// reading.  Rows go four to a CTA, one to each SM sub-partition, so a short prefix occupies
// few CTAs (few tickets) and no sub-partition runs two rows.  The last CTA to finish (a ticket, no
// waiting) then re-sorts the prefix by the new levels with sort_prefix_cta, copying the new
// records in on the way, and begins the next step.  The arithmetic is k_irregular_* followed
// by k_ac_correct, operation for operation, and the re-sort is the scheduler's, so the state
// after the step is the same bits as the host path's.
constexpr int kStepWarps = 8;
constexpr int kStepThreads = kStepWarps * 32;
constexpr int kStepSortItems = 16;
constexpr int64_t kDevicePrefix = (int64_t)kStepThreads * kStepSortItems;  // the longest prefix (4096)

template <bool MIXED>
__global__ void __launch_bounds__(kStepThreads) k_ac_irregular_step(AcDev D, int64_t n, uint4 *rec_new,
                                                                    unsigned long long *pairs, unsigned *status,
                                                                    SortArgs SA)
{
    __shared__ int32_t s_cnt[kBins];
    __shared__ int32_t s_base[kBins];
    __shared__ int32_t s_warp[kStepWarps][kBins];
    __shared__ bool s_last;
    pdl_trigger();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // rows in rounds of 8 G: the first 4 G go four to a CTA, one to each of its warps 0-3 (one
    // per SM sub-partition), the next 4 G likewise to warps 4-7
    const int64_t k_first = 4 * (int64_t)blockIdx.x + (w & 3) + (int64_t)(w >> 2) * 4 * gridDim.x;
    const int64_t k_step = (int64_t)gridDim.x * kStepWarps;
    const StepParams *dyn = SA.dyn;
    const int32_t *list = SA.list;
    int32_t *want = const_cast<int32_t *>(SA.want);
    pdl_wait();
    // the first row's particle is requested with the step's parameters (the list holds n entries)
    const int32_t i_first = k_first < n ? list[k_first] : 0;
    if (dyn->halt) return;
    IrrArgs A{};
    A.srec = MIXED ? (const void *)D.s32 : (const void *)D.s64;
    A.n = n;
    A.n_i = dyn->n_act;
    A.idx = list;
    A.nb = D.ell;
    A.t = dyn->t;
    A.t_hi = dyn->t_hi;
    A.t_lo = dyn->t_lo;
    A.status = status;
    A.ell_cnt = D.ell_cnt;
    A.ell_stride = D.cap;
    const int64_t t_ticks = dyn->t_ticks;
    const double t = A.t;
    // CTAs past the rows have nothing to do and take no part in the ticket
    const int64_t used = A.n_i <= 0 ? 1 : ((A.n_i + 3) / 4 < gridDim.x ? (A.n_i + 3) / 4 : gridDim.x);
    if (blockIdx.x >= used) return;
    const int c = lane < 3 ? lane : 0;  // the component lanes 0-2 correct (the others shadow 0)
    const float eta_f = (float)D.eta_irr;
    unsigned my_pairs = 0;
    for (int64_t k = k_first; k < A.n_i; k += k_step) {
        // row k's particle and list range (irr_row's checks)
        const int64_t i = k == k_first ? i_first : list[k];
        const bool ok = i >= 0 && i < n;
        const int64_t e0 = ok ? i * A.ell_stride : 0, e1 = ok ? e0 + D.ell_cnt[i] : 0;
        if (!ok && lane == 0) atomicOr(status, ST_BAD_INDEX);
        // the corrector's inputs do not depend on the force: requested before the list pass
        const int64_t ii = ok ? i : 0, q = 3 * ii + c;
        const int LR0 = D.LR[ii], LI0 = D.LI[ii];
        const double Tr = D.Tr[ii], tl = D.tl[ii], mi = D.m[ii];
        const double x0 = D.x[q], v0 = D.v[q], a0 = D.a[q], j0 = D.jk[q];
        const double Fr = D.Fr[q], Jr = D.Jr[q], D2 = D.D2[q], D3 = D.D3[q];
        double fo, jo;  // the irregular force and jerk, component c
        // the corrector's steps that do not need the force, in lanes 0-2 (FP64), are placed
        // where the force pass waits for its first gathers: the extrapolated regular force and
        // jerk at t and the predicted position and velocity
        double Fx = 0.0, Jx = 0.0, xp = 0.0, vp = 0.0;
        const double h = t - tl;  // the irregular step, a power of two
        auto prework = [&]() {
            if (lane < 3) {
                const double tau = t - Tr;
                Fx = Fr + Jr * tau + D2 * tau * tau / 2.0 + D3 * tau * tau * tau / 6.0;
                Jx = Jr + D2 * tau + D3 * tau * tau / 2.0;
                hermite_taylor(x0, v0, a0, j0, h, xp, vp);
            }
        };
        if constexpr (MIXED) {
            const float4 *S = static_cast<const float4 *>(A.srec);
            float ih[3] = {0, 0, 0}, il[3] = {0, 0, 0}, iv[3] = {0, 0, 0}, iD[3] = {0, 0, 0}, iE[3] = {0, 0, 0};
            float4 Pi[5];
            if (ok)
#pragma unroll
                for (int u = 0; u < 5; ++u) Pi[u] = S[5 * i + u];
            // the lane's list entries four rounds (128 entries a row) at a time: a batch's indices
            // and then its records are requested together, so a batch costs two round trips
            // whatever its length, and the first batch is in flight during the FP64 work (the
            // per-lane order of the terms is the irregular force kernel's)
            constexpr int kBatch = 4;
            int32_t jb[kBatch];
            float4 Rb[kBatch][5];
            auto fetch = [&](int64_t eb) {
#pragma unroll
                for (int r = 0; r < kBatch; ++r) jb[r] = irr_neighbour(A, eb + 32 * r, e1);
#pragma unroll
                for (int r = 0; r < kBatch; ++r)
                    if (jb[r] >= 0)
#pragma unroll
                        for (int u = 0; u < 5; ++u) Rb[r][u] = S[5 * (int64_t)jb[r] + u];
            };
            fetch(e0 + lane);
            prework();
            if (ok) {
                const float4 P = Pi[0], L = Pi[1], V = Pi[2], Ac = Pi[3], J = Pi[4];
                const float dt = __fadd_rn(__fsub_rn(A.t_hi, L.w), __fsub_rn(A.t_lo, V.w));
                ih[0] = P.x; ih[1] = P.y; ih[2] = P.z;
                il[0] = L.x; il[1] = L.y; il[2] = L.z;
                iv[0] = V.x; iv[1] = V.y; iv[2] = V.z;
                incr_f32(V.x, Ac.x, J.x, dt, iD[0], iE[0]);
                incr_f32(V.y, Ac.y, J.y, dt, iD[1], iE[1]);
                incr_f32(V.z, Ac.z, J.z, dt, iD[2], iE[2]);
            }
            float f[7] = {0, 0, 0, 0, 0, 0, 0};
            for (int64_t eb = e0 + lane; eb < e1; eb += 32 * kBatch) {
#pragma unroll
                for (int r = 0; r < kBatch; ++r)
                    if (jb[r] >= 0 && jb[r] != i) state_pair_mixed(Rb[r], A.t_hi, A.t_lo, ih, il, iv, iD, iE, f);
                if (eb + 32 * kBatch < e1) fetch(eb + 32 * kBatch);
            }
            float h, l;
            warp_sum7_df(f, lane, h, l);
            const double v = ok ? __dadd_rn((double)h, (double)l) : 0.0;  // lane 4 c': component c'
            fo = __shfl_sync(0xffffffffu, v, 4 * c);
            jo = __shfl_sync(0xffffffffu, v, 4 * (c + 3));
        } else {
            const dvec4 *S = static_cast<const dvec4 *>(A.srec);
            prework();
            double own = 0.0;
            if (ok && lane < 6) {
                const int cc = lane < 3 ? lane : lane - 3;
                const dvec4 P = S[4 * i], V = S[4 * i + 1], Ac = S[4 * i + 2], J = S[4 * i + 3];
                auto pick = [cc](const dvec4 &u) { return cc == 0 ? u.x : (cc == 1 ? u.y : u.z); };
                double xp, vp;
                hermite_taylor(pick(P), pick(V), pick(Ac), pick(J), __dsub_rn(A.t, P.w), xp, vp);
                own = lane < 3 ? xp : vp;
            }
            double xi[3], vi[3];
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                xi[u] = __shfl_sync(0xffffffffu, own, u);
                vi[u] = __shfl_sync(0xffffffffu, own, 3 + u);
            }
            double sum[7] = {0, 0, 0, 0, 0, 0, 0};
            for (int64_t e = e0 + lane; e < e1; e += 32) {
                const int64_t j = A.nb[e];
                if (j < 0 || j >= A.n) {
                    atomicOr(A.status, ST_BAD_INDEX);
                    continue;
                }
                if (j == i) continue;
                const dvec4 P = S[4 * j], V = S[4 * j + 1], Ac = S[4 * j + 2], J = S[4 * j + 3];
                const double dt = __dsub_rn(A.t, P.w);
                double x0j, x1j, x2j, v0j, v1j, v2j;
                hermite_taylor(P.x, V.x, Ac.x, J.x, dt, x0j, v0j);
                hermite_taylor(P.y, V.y, Ac.y, J.y, dt, x1j, v1j);
                hermite_taylor(P.z, V.z, Ac.z, J.z, dt, x2j, v2j);
                pair_f64_fma(make_dvec4(x0j, x1j, x2j, V.w), make_dvec4(v0j, v1j, v2j, 0.0), xi, vi, sum);
            }
#pragma unroll
            for (int u = 0; u < 7; ++u) sum[u] = warp_sum(sum[u]);
            fo = jo = 0.0;
#pragma unroll
            for (int u = 0; u < 3; ++u)
                if (c == u) {
                    fo = sum[u];
                    jo = sum[3 + u];
                }
            if (!ok) fo = jo = 0.0;
        }
        if (!ok) continue;  // (warp-uniform) the status bit is set; the row is left as it was
        // k_ac_correct's irregular branch, lane c < 3 component c: the extrapolated regular
        // force, then the Hermite corrector on the total force
        double x1 = 0.0, v1 = 0.0, a1 = 0.0, j1 = 0.0, a2e = 0.0, a3 = 0.0;
        float sq[4] = {0.f, 0.f, 0.f, 0.f};  // FP32 squares of a1, j1, a2e, a3 for the estimate
        if (lane < 3) {
            a1 = fo + Fx;
            j1 = jo + Jx;
            double a2;
            hermite_correct_pow2(xp, vp, a0, j0, a1, j1, h, recip_pow2(h), x1, v1, a2, a3);
            a2e = a2 + h * a3;
            const float q4[4] = {__double2float_rn(a1), __double2float_rn(j1), __double2float_rn(a2e),
                                 __double2float_rn(a3)};
#pragma unroll
            for (int u = 0; u < 4; ++u) sq[u] = __fmul_rn(q4[u], q4[u]);
        }
        float tot[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            tot[u] = __fadd_rn(__fadd_rn(sq[u], __shfl_sync(0xffffffffu, sq[u], 1)), __shfl_sync(0xffffffffu, sq[u], 2));
        int L = ac_level_rule_est(LI0, tot[0], tot[1], tot[2], tot[3], eta_f, t_ticks, D.lmin, D.lmax);
        L = __shfl_sync(0xffffffffu, L, 0);
        if (L < 0) {  // within the estimate's margin of a power of two: the FP64 criterion
            double A1[3], J1[3], A2E[3], A3[3];
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                A1[u] = __shfl_sync(0xffffffffu, a1, u);
                J1[u] = __shfl_sync(0xffffffffu, j1, u);
                A2E[u] = __shfl_sync(0xffffffffu, a2e, u);
                A3[u] = __shfl_sync(0xffffffffu, a3, u);
            }
            L = ac_level_rule(LI0, ac_crit(D.eta_irr, A1, J1, A2E, A3), t_ticks, D.lmin, D.lmax);
        }
        if (L < LR0) L = LR0;  // irregular step at most the regular step
        if (lane < 3) {
            D.x[q] = x1;
            D.v[q] = v1;
            D.a[q] = a1;
            D.jk[q] = j1;
        }
        // the new state record (pack_state_one's layout and conversions), lane c its component
        if constexpr (MIXED) {
            float *R = reinterpret_cast<float *>(rec_new + 5 * k);
            if (lane < 3) {
                const float hx = __double2float_rn(x1);
                R[c] = hx;
                R[4 + c] = __double2float_rn(__dsub_rn(x1, (double)hx));
                R[8 + c] = __double2float_rn(v1);
                R[12 + c] = __double2float_rn(a1);
                R[16 + c] = __double2float_rn(j1);
            } else if (lane == 3) {
                const float th = __double2float_rn(t);
                R[3] = __double2float_rn(mi);
                R[7] = th;
                R[11] = __double2float_rn(__dsub_rn(t, (double)th));
                R[15] = 0.f;
                R[19] = 0.f;
            }
        } else {
            double *R = reinterpret_cast<double *>(rec_new + 8 * k);
            if (lane < 3) {
                R[c] = x1;
                R[4 + c] = v1;
                R[8 + c] = a1;
                R[12 + c] = j1;
            } else if (lane == 3) {
                R[3] = t;
                R[7] = mi;
                R[11] = 0.0;
                R[15] = 0.0;
            }
        }
        if (lane == 0) {
            if ((t_ticks & (((int64_t)1 << (kAcTick - LR0)) - 1)) == 0) atomicOr(status, ST_DEVICE);
            D.tl[i] = t;
            D.LI[i] = L;
            want[k] = L;
            my_pairs += (unsigned)D.ell_cnt[i];
        }
    }
    if (lane == 0 && my_pairs) atomicAdd(pairs, (unsigned long long)my_pairs);
    // the last CTA to finish re-sorts the prefix (every other CTA's writes are visible to it:
    // each fenced them before taking its ticket) and begins the next step
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&D.tickets[0], 1u) == (unsigned)used - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) D.tickets[0] = 0u;  // the next step's kernel starts after this one ends
    SA.n_act = A.n_i;
    SA.lstar = dyn->lstar;
    sort_prefix_cta<kStepThreads, kStepSortItems, true>(SA, s_cnt, s_base, s_warp);
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

// The begin of the first step of a batch of device-driven block steps (one warp, step_begin):
// the next block time and the active prefix from the scheduler's device counts, as
// nb_sched_next finds them on the host.  The step halts, and with it every step queued after
// it, when that time passes t_end, when the regular-level histogram says some particle takes a
// regular step there (the host path runs those), when the prefix is longer than the step
// kernel's re-sort takes, or when the batch's budget dstep[0] is spent; otherwise it counts the
// step (dstep[1]) and its rows (dstep[2]).  Later steps begin in the last CTA of the step before.
__global__ void __launch_bounds__(32) k_ac_begin(StepBegin B, SchedDevice S)
{
    // one warp: lane l holds the levels l and l + 32
    pdl_trigger();
    pdl_wait();
    if (B.P->halt) return;
    step_begin(B, S.count[threadIdx.x], S.count[threadIdx.x + 32], *S.T, threadIdx.x,
               step_begin_inputs(B, threadIdx.x));
}

// The host words after a batch of device-driven steps: the regular-level histogram and the
// status flags the batch's steps raised (cleared on the device; the host clears its copy).
__global__ void k_ac_publish(AcDev D, unsigned *status)
{
    D.io[threadIdx.x] = __ldcg(&D.lr_hist[threadIdx.x]);
    if (threadIdx.x == 0) D.io[64] |= (int32_t)atomicExch(status, 0u);
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
    int32_t *cta_count = nullptr;  // regular rows per list chunk of the classify passes
    void *srec = nullptr;  // state records (pack_state_one layout of the context's precision)
    unsigned long long *pairs = nullptr;
    int32_t *h_io = nullptr;       // pinned, mapped: [0, 64) regular-level histogram, [64] status flags
    int32_t *h_lr = nullptr;       // = h_io
    unsigned *h_status = nullptr;  // = h_io + 64: the context's status flags since the host last read them
    StepParams *P = nullptr;       // device-driven steps: the current step's parameters
    int64_t *dstep = nullptr;      // device-driven steps: [0] budget left, [1] steps done, [2] active rows
    uint4 *rec_new = nullptr;      // device-driven steps: the corrected records of a step's prefix
    int64_t rec_rows = 0;          // ... for up to this many rows
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
        cudaMalloc(&s->cta_count, ((n + kClassifyChunk - 1) / kClassifyChunk + 1) * 4) == cudaSuccess &&
        cudaMalloc(&s->pairs, 8) == cudaSuccess && cudaMalloc(&D.lr_hist, 64 * 4) == cudaSuccess &&
        cudaMalloc(&D.tickets, 2 * 4) == cudaSuccess &&
        cudaHostAlloc(&s->h_io, 80 * 4, cudaHostAllocMapped) == cudaSuccess &&
        cudaHostGetDevicePointer((void **)&D.io, s->h_io, 0) == cudaSuccess &&
        cudaMemset(D.lr_hist, 0, 64 * 4) == cudaSuccess && cudaMemset(s->pairs, 0, 8) == cudaSuccess &&
        cudaMemset(D.tickets, 0, 2 * 4) == cudaSuccess &&
        cudaMalloc(&s->srec, state_record_bytes(s->cs.precision, n)) == cudaSuccess &&
        cudaMalloc(&s->P, sizeof(StepParams)) == cudaSuccess && cudaMalloc(&s->dstep, 3 * sizeof(int64_t)) == cudaSuccess &&
        cudaMemset(s->P, 0, sizeof(StepParams)) == cudaSuccess &&
        cudaMalloc(&s->rec_new, state_record_bytes(s->cs.precision, n < kDevicePrefix ? n : kDevicePrefix)) ==
            cudaSuccess;
    s->rec_rows = n < kDevicePrefix ? n : kDevicePrefix;
    if (!ok) cudaGetLastError();
    if (s->h_io) memset(s->h_io, 0, 80 * 4);
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
        const int cg = (int)((na + kClassifyChunk - 1) / kClassifyChunk);
        k_ac_classify_count<<<cg, kClassifyBlock, 0, st>>>(s->D, na, list, t_ticks, s->cta_count);
        k_ac_classify_place<<<cg, kClassifyBlock, 0, st>>>(s->D, na, list, t_ticks, s->cta_count, s->reg_pos,
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
    *s->h_status = 0;
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

// Whether the block step at time t has a regular subset, from the regular-level histogram
// the last corrector published (the test nb_ac_step makes before it launches).
static bool ac_regular_due(const nb_ac *s, double t)
{
    const int64_t t_ticks = (int64_t)std::ldexp(t, kAcTick);
    int tz = 0;
    while (tz < kAcTick && ((t_ticks >> tz) & 1) == 0) ++tz;
    int64_t nr = 0;
    for (int b = kAcTick - tz; b < 64; ++b) nr += s->h_lr[b];
    return nr > 0;
}

// Up to K block steps without a regular subset, driven by the device: per step the begin
// kernel, the irregular force (predict on load), the corrector and the scheduler's re-sort,
// all reading the step's parameters from device memory, so the host enqueues the whole batch
// and synchronises once.  The first step that needs the host (a regular subset, a prefix too
// long for one re-sort CTA) or the end time halts the rest.  *done: the steps taken.
static nb_status ac_device_steps(nb_ac *s, double t_end, int64_t K, int64_t *done)
{
    *done = 0;
    SchedDevice S;
    if (!sched_device(s->sched, &S)) return afail(s, NB_ERR_OOM, "device scheduler state");
    if (S.max_prefix > s->rec_rows) S.max_prefix = s->rec_rows;  // longer prefixes: the host path
    if (!sched_push(s->sched)) return afail(s, NB_ERR_CUDA, "scheduler state to the device");
    const CtxState &cs = s->cs;
    cudaStream_t st = cs.stream;
    int64_t h[3] = {K, 0, 0};
    int32_t halt = 0;
    ACK(cudaMemsetAsync(&s->P->halt, 0, sizeof(int32_t), st), "clear halt");
    ACK(cudaMemcpyAsync(s->dstep, h, sizeof(h), cudaMemcpyHostToDevice, st), "step budget");
    // the first step's begin, then one kernel per step: the fused irregular force, corrector
    // and re-sort, which ends with the next step's begin; each a programmatic dependent of the
    // kernel before it
    const int rb = (int)state_record_bytes(cs.precision, 1);
    auto step_kernel = cs.precision == 0 ? k_ac_irregular_step<false> : k_ac_irregular_step<true>;
    StepBegin B{s->P, s->D.lr_hist, t_end, s->dstep, S.max_prefix};
    const SortArgs SA = sched_device_sort_args(s->sched, s->want, s->P, s->rec_new, s->srec, rb, &B);
    k_ac_begin<<<1, 32, 0, st>>>(B, S);
    for (int64_t k = 0; k < K; ++k)
        ACK(launch_pdl(true, step_kernel, dim3(cs.num_sms), dim3(kStepThreads), st, s->D, cs.n, s->rec_new, s->pairs,
                       cs.status + SS_FLAGS, SA),
            "block-step launch");
    k_ac_publish<<<1, 64, 0, st>>>(s->D, cs.status + SS_FLAGS);
    ACK(cudaGetLastError(), "device step launches");
    ACK(cudaMemcpyAsync(h, s->dstep, sizeof(h), cudaMemcpyDeviceToHost, st), "step counters");
    ACK(cudaMemcpyAsync(&halt, &s->P->halt, sizeof(halt), cudaMemcpyDeviceToHost, st), "halt flag");
    if (!sched_pull(s->sched)) return afail(s, NB_ERR_CUDA, "scheduler state from the device");  // synchronises
    if (h[1] > 0) ctx_state_changed(s->ctx);  // the correctors rewrote the context's state arrays
    const unsigned f = *s->h_status;
    *s->h_status = 0;
    if (f & (ST_BAD_INDEX | ST_DUP_INDEX | ST_DEVICE | ST_TIMEOUT))
        return afail(s, NB_ERR_DEVICE, "device-driven block steps: device status 0x%x", f);
    if (f & (ST_NB_TRUNCATED | ST_CSR_FULL)) s->overflow = true;
    *done = h[1];
    s->stats[0] += (double)h[1];
    s->stats[1] += (double)h[2];
    s->stats[5] += (double)h[1];
    return NB_OK;
}

// The number of block steps from the next one (at tn) up to, not including, the next step
// with a regular subset or the first step past t_end, if the levels stay as they are: the
// block time advances by the finest irregular step present, and the next regular subset falls
// on the first multiple of the finest regular step present (the published histogram).
static int64_t ac_run_length(nb_ac *s, double tn, double t_end)
{
    int64_t counts[64];
    if (nb_sched_counts(s->sched, counts) != NB_OK) return 1;
    int li = -1, lr = -1;
    for (int b = 63; b >= 0; --b)
        if (li < 0 && counts[b]) li = b;
    for (int b = 63; b >= 0; --b)
        if (lr < 0 && s->h_lr[b]) lr = b;
    if (li < 0) return 1;
    const double dt = std::ldexp(1.0, -li);
    double t_stop = t_end + dt;  // the first block time past t_end
    if (lr >= 0) {
        const double DT = std::ldexp(1.0, -lr);
        const double t_reg = std::ceil(tn / DT) * DT;  // the next regular time (tn is not one)
        if (t_reg < t_stop) t_stop = t_reg;
    }
    const double k = (t_stop - tn) / dt;
    return k < 1.0 ? 1 : (k > 1e6 ? 1000000 : (int64_t)k);
}

nb_status nb_ac_run(nb_ac *s, double t_end, int64_t max_blocks, double *stats)
{
    if (!s) return NB_ERR_ARG;
    constexpr int64_t kMaxBatch = 128;
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
        int64_t done = 0;
        if (!ac_regular_due(s, tn)) {  // a run of steps without regular subsets: the device drives them
            // as many steps as the run should hold (a finer level ends the batch early, through its
            // budget; a coarser one halts it at the regular step, the rest of the batch no-ops)
            int64_t k = ac_run_length(s, tn, t_end);
            if (k > kMaxBatch) k = kMaxBatch;
            if (max_blocks > 0 && max_blocks - b < k) k = max_blocks - b;
            if ((ss = ac_device_steps(s, t_end, k, &done)) != NB_OK) return ss;
            b += done;
        }
        if (done == 0) {  // a regular subset is due (or the device took no step): the host path
            if ((ss = nb_ac_step(s, nullptr, nullptr, nullptr)) != NB_OK) return ss;
            ++b;
        }
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
                 s->Fa, s->Ja, s->Pa, s->Fn, s->Jn, s->Pn, s->cta_count, s->pairs, s->D.lr_hist, s->D.tickets, s->srec,
                 s->P, s->dstep, s->rec_new};
    for (void *q : p)
        if (q) cudaFree(q);
    if (s->h_io) cudaFreeHost(s->h_io);
    delete s;
    return NB_OK;
}

const char *nb_ac_last_error(const nb_ac *s) { return s ? s->err : "null integrator"; }

}  // extern "C"
