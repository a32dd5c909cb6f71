// irregular.cu — K10: the irregular force of the Ahmad-Cohen scheme (paper Sec. 2; Sec.
// 3.2.2 "Prediction and irregular force").  For every active particle i, acceleration, jerk
// and potential summed over its neighbour list only (a CSR list, e.g. the one the regular
// force returned), with i and each listed neighbour predicted to the block time on load
// from its Hermite state: the neighbour-only prediction of Sec. 3.3.3.  Optionally the same
// pass splits a regular-force result of the same rows into its part from outside the lists
// (all-j sums minus the irregular sums).
//
// Work: one warp per active row, the lanes striding over the row's list (lists hold tens to
// hundreds of entries), a fixed xor-butterfly reduction over the lanes (results do not
// depend on timing).  The gathers hit a per-particle state record (below) that a 2^20-body
// system keeps within the 129 MB L2 (mixed) or mostly within it (FP64).
//
// Two precisions, as the context's:
//  * FP64: the predictor is hermite_taylor, so a neighbour predicted here is bit-identical to
//    the same particle after nb_predict; the pair is pair_f64_fma (pair_f64's sums, fused).
//  * mixed: r = (x_j - x_i) + (D_j - D_i) with the base difference in double-single (as in
//    the mixed regular force) and the Taylor increments D = dt (v + dt (a/2 + dt jerk/6)) in
//    FP32; likewise w = (v_j - v_i) + (E_j - E_i), E = dt (a + dt jerk/2).  dt = t - t_last
//    is formed in double-single from hi/lo halves of t and t_last, so that small steps at
//    late times keep their digits.  Pair arithmetic in FP32, lane sums in FP32 (at most a
//    few dozen terms), the warp reduction in double-float with one FP64 add per component.
#include "nb_common.cuh"
#include "nb_irregular.cuh"
#include "nb_kernels.cuh"

namespace nbgpu {

// State records: the layout is that of pack_state_one (nb_common.cuh).
__global__ void k_pack_state(int64_t n, const double *__restrict__ x, const double *__restrict__ v,
                             const double *__restrict__ a, const double *__restrict__ jk,
                             const double *__restrict__ tl, const double *__restrict__ m, dvec4 *__restrict__ s64,
                             float4 *__restrict__ s32)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        pack_state_one(i, x + 3 * i, v + 3 * i, a + 3 * i, jk + 3 * i, tl[i], m[i], s64, s32);
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_irregular_fp64(IrrArgs A)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)BLOCK + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * BLOCK) >> 5;
    const dvec4 *S = static_cast<const dvec4 *>(A.srec);
    for (int64_t k = w0; k < A.n_i; k += nw) {
        int64_t i, e0, e1;
        const bool ok = irr_row(A, k, lane, i, e0, e1);
        // the active particle: lanes 0-2 predict x_p, lanes 3-5 v_p, one component each
        double own = 0.0;
        if (ok && lane < 6) {
            const int c = lane < 3 ? lane : lane - 3;
            const dvec4 P = S[4 * i], V = S[4 * i + 1], Ac = S[4 * i + 2], J = S[4 * i + 3];
            auto pick = [c](const dvec4 &q) { return c == 0 ? q.x : (c == 1 ? q.y : q.z); };
            double xp, vp;
            hermite_taylor(pick(P), pick(V), pick(Ac), pick(J), __dsub_rn(A.t, P.w), xp, vp);
            own = lane < 3 ? xp : vp;
        }
        double xi[3], vi[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xi[c] = __shfl_sync(0xffffffffu, own, c);
            vi[c] = __shfl_sync(0xffffffffu, own, 3 + c);
        }
        double s[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const int64_t j = A.nb[e];
            if (j < 0 || j >= A.n) {
                atomicOr(A.status, ST_BAD_INDEX);
                continue;
            }
            if (j == i) continue;
            const dvec4 P = S[4 * j], V = S[4 * j + 1], Ac = S[4 * j + 2], J = S[4 * j + 3];
            const double dt = __dsub_rn(A.t, P.w);
            double x0, x1, x2, v0, v1, v2;
            hermite_taylor(P.x, V.x, Ac.x, J.x, dt, x0, v0);
            hermite_taylor(P.y, V.y, Ac.y, J.y, dt, x1, v1);
            hermite_taylor(P.z, V.z, Ac.z, J.z, dt, x2, v2);
            pair_f64_fma(make_dvec4(x0, x1, x2, V.w), make_dvec4(v0, v1, v2, 0.0), xi, vi, s);
        }
#pragma unroll
        for (int c = 0; c < 7; ++c) s[c] = warp_sum(s[c]);
        irr_store(A, k, lane, s, ok);
    }
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_irregular_mixed(IrrArgs A)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)BLOCK + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * BLOCK) >> 5;
    const float4 *S = static_cast<const float4 *>(A.srec);
    for (int64_t k = w0; k < A.n_i; k += nw) {
        int64_t i, e0, e1;
        const bool ok = irr_row(A, k, lane, i, e0, e1);
        float ih[3] = {0, 0, 0}, il[3] = {0, 0, 0}, iv[3] = {0, 0, 0}, iD[3] = {0, 0, 0}, iE[3] = {0, 0, 0};
        if (ok) {
            const float4 P = S[5 * i], L = S[5 * i + 1], V = S[5 * i + 2], Ac = S[5 * i + 3], J = S[5 * i + 4];
            const float dt = __fadd_rn(__fsub_rn(A.t_hi, L.w), __fsub_rn(A.t_lo, V.w));
            ih[0] = P.x; ih[1] = P.y; ih[2] = P.z;
            il[0] = L.x; il[1] = L.y; il[2] = L.z;
            iv[0] = V.x; iv[1] = V.y; iv[2] = V.z;
            incr_f32(V.x, Ac.x, J.x, dt, iD[0], iE[0]);
            incr_f32(V.y, Ac.y, J.y, dt, iD[1], iE[1]);
            incr_f32(V.z, Ac.z, J.z, dt, iD[2], iE[2]);
        }
        float f[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const int32_t j = irr_neighbour(A, e, e1);
            if (j < 0 || j == i) continue;
            float4 R[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) R[q] = S[5 * (int64_t)j + q];
            state_pair_mixed(R, A.t_hi, A.t_lo, ih, il, iv, iD, iE, f);
        }
        float h, l;
        warp_sum7_df(f, lane, h, l);
        irr_store_df(A, k, lane, h, l, ok);
    }
}

// ------------------------------------------------------------------------------------------
// Predict-all form.  Sec. 3.3.3 notes that predicting every particle once is cheaper than
// predicting each neighbour when <N_b> N_i exceeds N.  Then one pass of the all-particle
// predictor (k_predict, records only) writes the compact j-records of the regular force —
// FP64 {x_p, m} {v_p, 0}, mixed {x_hi, m} {x_lo, 0} {v, 0} — and the list pass gathers 64 or
// 48 bytes per neighbour instead of 128 or 80, with no prediction per pair.  FP64 positions
// are the same bits as in the neighbour-only form (one predictor), so FP64 results agree
// bit for bit between the forms; the mixed form predicts in FP64 here.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_irregular_rec_fp64(IrrArgs A)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)BLOCK + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * BLOCK) >> 5;
    const dvec4 *R = static_cast<const dvec4 *>(A.srec);
    for (int64_t k = w0; k < A.n_i; k += nw) {
        int64_t i, e0, e1;
        const bool ok = irr_row(A, k, lane, i, e0, e1);
        double xi[3] = {0, 0, 0}, vi[3] = {0, 0, 0};
        if (ok) {
            const dvec4 P = R[2 * i], V = R[2 * i + 1];
            xi[0] = P.x; xi[1] = P.y; xi[2] = P.z;
            vi[0] = V.x; vi[1] = V.y; vi[2] = V.z;
        }
        double s[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const int64_t j = A.nb[e];
            if (j < 0 || j >= A.n) {
                atomicOr(A.status, ST_BAD_INDEX);
                continue;
            }
            if (j == i) continue;
            pair_f64_fma(R[2 * j], R[2 * j + 1], xi, vi, s);
        }
#pragma unroll
        for (int c = 0; c < 7; ++c) s[c] = warp_sum(s[c]);
        irr_store(A, k, lane, s, ok);
    }
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 4) k_irregular_rec_mixed(IrrArgs A)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)BLOCK + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * BLOCK) >> 5;
    const float4 *R = static_cast<const float4 *>(A.srec);
    for (int64_t k = w0; k < A.n_i; k += nw) {
        int64_t i, e0, e1;
        const bool ok = irr_row(A, k, lane, i, e0, e1);
        float ih[3] = {0, 0, 0}, il[3] = {0, 0, 0}, iv[3] = {0, 0, 0};
        if (ok) {
            const float4 P = R[3 * i], L = R[3 * i + 1], V = R[3 * i + 2];
            ih[0] = P.x; ih[1] = P.y; ih[2] = P.z;
            il[0] = L.x; il[1] = L.y; il[2] = L.z;
            iv[0] = V.x; iv[1] = V.y; iv[2] = V.z;
        }
        float f[7] = {0, 0, 0, 0, 0, 0, 0};
        // two list entries per lane per round (e and e + 32): both records are requested
        // before either is used, so each lane keeps two gathers in flight; the per-lane order
        // of the terms is unchanged
        for (int64_t e = e0 + lane; e < e1; e += 64) {
            const int32_t ja = irr_neighbour(A, e, e1), jb = irr_neighbour(A, e + 32, e1);
            float4 Ra[3], Rb[3];
            if (ja >= 0)
#pragma unroll
                for (int q = 0; q < 3; ++q) Ra[q] = R[3 * (int64_t)ja + q];
            if (jb >= 0)
#pragma unroll
                for (int q = 0; q < 3; ++q) Rb[q] = R[3 * (int64_t)jb + q];
            if (ja >= 0 && ja != i) rec_pair_mixed(Ra, ih, il, iv, f);
            if (jb >= 0 && jb != i) rec_pair_mixed(Rb, ih, il, iv, f);
        }
        float h, l;
        warp_sum7_df(f, lane, h, l);
        irr_store_df(A, k, lane, h, l, ok);
    }
}

constexpr int kIrrBlock = 256;

void launch_pack_state(cudaStream_t st, int precision, int64_t n, const double *x, const double *v, const double *a,
                       const double *jk, const double *tl, const double *m, void *srec)
{
    int64_t g = (n + 255) / 256;
    if (g > 152 * 32) g = 152 * 32;
    k_pack_state<<<(int)(g < 1 ? 1 : g), 256, 0, st>>>(n, x, v, a, jk, tl, m,
                                                         precision == 0 ? (dvec4 *)srec : nullptr,
                                                         precision == 0 ? nullptr : (float4 *)srec);
}

size_t state_record_bytes(int precision, int64_t n) { return (size_t)n * (precision == 0 ? 4 * 32 : 5 * 16); }

// records: the state records (neighbour-only prediction) or, with predicted != 0, the compact
// predicted j-records of the predict-all form.
void launch_irregular(cudaStream_t st, int precision, int num_sms, const void *srec, int predicted, int64_t n,
                      double t, int64_t n_i, const int32_t *idx, const int64_t *off, const int32_t *nb, double *acc,
                      double *jerk, double *pot, double *acc_reg, double *jerk_reg, double *pot_reg, unsigned *status,
                      const int32_t *ell_cnt, int64_t ell_stride)
{
    IrrArgs A;
    A.srec = srec;
    A.n = n;
    A.n_i = n_i;
    A.idx = idx;
    A.off = off;
    A.nb = nb;
    A.t = t;
    A.t_hi = (float)t;
    A.t_lo = (float)(t - (double)A.t_hi);
    A.acc = acc;
    A.jerk = jerk;
    A.pot = pot;
    A.acc_reg = acc_reg;
    A.jerk_reg = jerk_reg;
    A.pot_reg = pot_reg;
    A.status = status;
    A.ell_cnt = ell_cnt;
    A.ell_stride = ell_stride;
    constexpr int rows_per_cta = kIrrBlock / 32;
    int64_t g = (n_i + rows_per_cta - 1) / rows_per_cta;
    const int64_t gmax = (int64_t)num_sms * 8;  // 8 CTAs of 8 warps: 64 warps per SM
    if (g > gmax) g = gmax;
    if (predicted) {
        if (precision == 0)
            k_irregular_rec_fp64<kIrrBlock><<<(int)g, kIrrBlock, 0, st>>>(A);
        else
            k_irregular_rec_mixed<kIrrBlock><<<(int)g, kIrrBlock, 0, st>>>(A);
    } else if (precision == 0) {
        k_irregular_fp64<kIrrBlock><<<(int)g, kIrrBlock, 0, st>>>(A);
    } else {
        k_irregular_mixed<kIrrBlock><<<(int)g, kIrrBlock, 0, st>>>(A);
    }
}

}  // namespace nbgpu
