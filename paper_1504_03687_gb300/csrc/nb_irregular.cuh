// nb_irregular.cuh — the per-row pieces of the irregular force (Sec. 3.2.2): the launch
// arguments, a row's checked list range, the neighbour pair of either precision with
// prediction on load, and the fixed-order warp reductions.  Shared by the irregular force
// kernels and the integrator's fused block-step kernel; both units are compiled without FMA
// contraction, so the two give the same bits for the same row.
#pragma once

#include "nb_common.cuh"
#include "nb_kernels.cuh"

namespace nbgpu {

struct IrrArgs {
    const void *srec;
    int64_t n, n_i;
    const int32_t *idx;
    const int64_t *off;
    const int32_t *nb;
    double t;
    float t_hi, t_lo;
    double *acc, *jerk, *pot;
    double *acc_reg, *jerk_reg, *pot_reg;  // optional: all-j sums in, outside-list part out
    unsigned *status;
    const int32_t *ell_cnt;  // per-particle lists: i's list is nb[i * ell_stride .. + ell_cnt[i])
    int64_t ell_stride;      // 0: CSR lists (off)
};

// Row k's checked index and list range (an empty range and a status bit when malformed).
__device__ __forceinline__ bool irr_row(const IrrArgs &A, int64_t k, int lane, int64_t &i, int64_t &e0, int64_t &e1)
{
    i = A.idx[k];
    if (A.ell_stride > 0) {
        const bool in = i >= 0 && i < A.n;
        e0 = in ? i * A.ell_stride : 0;
        e1 = in ? e0 + A.ell_cnt[i] : 0;
    } else {
        e0 = A.off[k];
        e1 = A.off[k + 1];
    }
    const bool ok = i >= 0 && i < A.n && e0 >= 0 && e1 >= e0;
    if (!ok) {
        if (lane == 0) atomicOr(A.status, ST_BAD_INDEX);
        e0 = e1 = 0;
    }
    return ok;
}

// Lanes 0..6 hold the row's seven sums after the butterfly: lane c writes component c and,
// when asked, replaces the all-j value by the outside-list part.
__device__ __forceinline__ void irr_store(const IrrArgs &A, int64_t k, int lane, const double (&s)[7], bool ok)
{
    if (lane >= 7) return;
    double v = 0.0;
#pragma unroll
    for (int c = 0; c < 7; ++c)
        if (lane == c) v = s[c];
    if (!ok) v = 0.0;
    double *out = lane < 3 ? A.acc + 3 * k + lane : lane < 6 ? A.jerk + 3 * k + (lane - 3) : A.pot + k;
    *out = v;
    if (A.acc_reg) {
        double *reg = lane < 3 ? A.acc_reg + 3 * k + lane : lane < 6 ? A.jerk_reg + 3 * k + (lane - 3) : A.pot_reg + k;
        *reg = __dsub_rn(*reg, v);
    }
}

// (h, l) += (h2, l2) in double-float: TwoSum of the high parts (exact error term), the low
// parts added to that error, renormalised by FastTwoSum. The error of the pair is about
// 2^-44 of the sum, far below the FP32 lane sums it adds up.
__device__ __forceinline__ void df_add(float &h, float &l, float h2, float l2)
{
    const float s = __fadd_rn(h, h2);
    const float bp = __fsub_rn(s, h);
    const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(h2, bp));
    const float t = __fadd_rn(e, __fadd_rn(l, l2));
    h = __fadd_rn(s, t);
    l = __fsub_rn(t, __fsub_rn(h, s));
}

// The seven FP32 lane sums f[0..6] of a row summed over the warp, transposed: at the xor-16,
// -8 and -4 steps every lane keeps half of its components and sends the other half, so lane L
// ends with component c = L >> 2 (bits 4, 3, 2 of L pick the halves) summed over eight lanes;
// the xor-2 and xor-1 steps complete the 32-lane sum. Nine double-float adds and 14 shuffles
// per row instead of 35 FP64 adds: GB300's FP64 pipe is 1/64 of its FP32 rate. Lane 4c
// (c < 7) writes component c.
__device__ __forceinline__ void warp_sum7_df(const float (&f)[7], int lane, float &h, float &l)
{
    const unsigned full = 0xffffffffu;
    const bool b16 = lane & 16, b8 = lane & 8, b4 = lane & 4;
    float v4[4], h2[2], l2[2];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float lo_c = f[k], hi_c = k + 4 < 7 ? f[k + 4] : 0.f;
        const float send = b16 ? lo_c : hi_c;
        v4[k] = b16 ? hi_c : lo_c;
        float z = 0.f;
        df_add(v4[k], z, __shfl_xor_sync(full, send, 16), 0.f);
        if (k < 2) { h2[k] = v4[k]; l2[k] = z; }
        else {  // pair component k with k - 2 for the xor-8 step
            const float sh = b8 ? h2[k - 2] : v4[k], sl = b8 ? l2[k - 2] : z;
            const float kh = b8 ? v4[k] : h2[k - 2], kl = b8 ? z : l2[k - 2];
            h2[k - 2] = kh;
            l2[k - 2] = kl;
            df_add(h2[k - 2], l2[k - 2], __shfl_xor_sync(full, sh, 8), __shfl_xor_sync(full, sl, 8));
        }
    }
    {
        const float sh = b4 ? h2[0] : h2[1], sl = b4 ? l2[0] : l2[1];
        h = b4 ? h2[1] : h2[0];
        l = b4 ? l2[1] : l2[0];
        df_add(h, l, __shfl_xor_sync(full, sh, 4), __shfl_xor_sync(full, sl, 4));
    }
    df_add(h, l, __shfl_xor_sync(full, h, 2), __shfl_xor_sync(full, l, 2));
    df_add(h, l, __shfl_xor_sync(full, h, 1), __shfl_xor_sync(full, l, 1));
}

// Store of a row reduced by warp_sum7_df: lane 4c writes component c in FP64.
__device__ __forceinline__ void irr_store_df(const IrrArgs &A, int64_t k, int lane, float h, float l, bool ok)
{
    if ((lane & 3) != 0 || lane >= 28) return;
    const int c = lane >> 2;
    const double v = ok ? __dadd_rn((double)h, (double)l) : 0.0;
    double *out = c < 3 ? A.acc + 3 * k + c : c < 6 ? A.jerk + 3 * k + (c - 3) : A.pot + k;
    *out = v;
    if (A.acc_reg) {
        double *reg = c < 3 ? A.acc_reg + 3 * k + c : c < 6 ? A.jerk_reg + 3 * k + (c - 3) : A.pot_reg + k;
        *reg = __dsub_rn(*reg, v);
    }
}

// One FP64 pair of the irregular force (pair_f64's sums) with every multiply-add written as an
// explicit fused operation: the same bits under any contraction setting, and FMA-dense on the
// narrow FP64 pipe (the irregular units are compiled without automatic contraction).
__device__ __forceinline__ void pair_f64_fma(const dvec4 &p0, const dvec4 &p1, const double (&xi)[3],
                                             const double (&vi)[3], double *acc)
{
    const double rx = __dsub_rn(p0.x, xi[0]), ry = __dsub_rn(p0.y, xi[1]), rz = __dsub_rn(p0.z, xi[2]);
    const double r2 = __fma_rn(rz, rz, __fma_rn(ry, ry, __dmul_rn(rx, rx)));
    const double rinv = rsqrt(r2);
    const double wx = __dsub_rn(p1.x, vi[0]), wy = __dsub_rn(p1.y, vi[1]), wz = __dsub_rn(p1.z, vi[2]);
    const double rw = __fma_rn(rz, wz, __fma_rn(ry, wy, __dmul_rn(rx, wx)));
    const double rinv2 = __dmul_rn(rinv, rinv);
    const double mr = __dmul_rn(p0.w, rinv);
    const double mr3 = __dmul_rn(mr, rinv2);
    const double beta = __dmul_rn(-3.0, __dmul_rn(rw, rinv2));
    acc[0] = __fma_rn(mr3, rx, acc[0]);
    acc[1] = __fma_rn(mr3, ry, acc[1]);
    acc[2] = __fma_rn(mr3, rz, acc[2]);
    acc[3] = __fma_rn(mr3, __fma_rn(beta, rx, wx), acc[3]);
    acc[4] = __fma_rn(mr3, __fma_rn(beta, ry, wy), acc[4]);
    acc[5] = __fma_rn(mr3, __fma_rn(beta, rz, wz), acc[5]);
    acc[6] = __dsub_rn(acc[6], mr);
}

// Taylor increments of the mixed path: D = dt (v + dt (a/2 + dt jerk/6)), E = dt (a + dt jerk/2).
__device__ __forceinline__ void incr_f32(float v, float a, float j, float dt, float &D, float &E)
{
    constexpr float kSixth = 1.f / 6.f;
    D = __fmul_rn(dt, __fmaf_rn(dt, __fmaf_rn(dt, __fmul_rn(j, kSixth), __fmul_rn(a, 0.5f)), v));
    E = __fmul_rn(dt, __fmaf_rn(dt, __fmul_rn(j, 0.5f), a));
}

// List entry e of the row (index checked; -1 past the row's end or for a bad index).
__device__ __forceinline__ int32_t irr_neighbour(const IrrArgs &A, int64_t e, int64_t e1)
{
    if (e >= e1) return -1;
    const int32_t j = A.nb[e];
    if (j < 0 || j >= A.n) {
        atomicOr(A.status, ST_BAD_INDEX);
        return -1;
    }
    return j;
}

// One pair of the neighbour-only mixed form from j's state record R (5 float4).
__device__ __forceinline__ void state_pair_mixed(const float4 (&R)[5], float t_hi, float t_lo, const float (&ih)[3],
                                                 const float (&il)[3], const float (&iv)[3], const float (&iD)[3],
                                                 const float (&iE)[3], float (&f)[7])
{
    const float4 P = R[0], L = R[1], V = R[2], Ac = R[3], J = R[4];
    const float dt = __fadd_rn(__fsub_rn(t_hi, L.w), __fsub_rn(t_lo, V.w));
    const float ph[3] = {P.x, P.y, P.z}, pl[3] = {L.x, L.y, L.z}, pv[3] = {V.x, V.y, V.z}, pa[3] = {Ac.x, Ac.y, Ac.z},
                pj[3] = {J.x, J.y, J.z};
    float r[3], w[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float D, E;
        incr_f32(pv[c], pa[c], pj[c], dt, D, E);
        r[c] = __fadd_rn(ds_diff(ph[c], pl[c], ih[c], il[c]), __fsub_rn(D, iD[c]));
        w[c] = __fadd_rn(__fsub_rn(pv[c], iv[c]), __fsub_rn(E, iE[c]));
    }
    const float r2 = r2_f32(r[0], r[1], r[2]);
    const float rinv = rsqrtf(r2);
    const float rw = r[0] * w[0] + r[1] * w[1] + r[2] * w[2];
    const float rinv2 = rinv * rinv;
    const float mr = P.w * rinv;
    const float mr3 = mr * rinv2;
    const float beta = rw * (rinv2 * -3.f);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        f[c] += mr3 * r[c];
        f[3 + c] += mr3 * (w[c] + beta * r[c]);
    }
    f[6] -= mr;
}

// One pair of the predict-all mixed form from j's predicted record R (3 float4).
__device__ __forceinline__ void rec_pair_mixed(const float4 (&R)[3], const float (&ih)[3], const float (&il)[3],
                                               const float (&iv)[3], float (&f)[7])
{
    const float4 P = R[0], L = R[1], V = R[2];
    const float r[3] = {ds_diff(P.x, L.x, ih[0], il[0]), ds_diff(P.y, L.y, ih[1], il[1]), ds_diff(P.z, L.z, ih[2], il[2])};
    const float w[3] = {V.x - iv[0], V.y - iv[1], V.z - iv[2]};
    const float r2 = r2_f32(r[0], r[1], r[2]);
    const float rinv = rsqrtf(r2);
    const float rw = r[0] * w[0] + r[1] * w[1] + r[2] * w[2];
    const float rinv2 = rinv * rinv;
    const float mr = P.w * rinv;
    const float mr3 = mr * rinv2;
    const float beta = rw * (rinv2 * -3.f);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        f[c] += mr3 * r[c];
        f[3 + c] += mr3 * (w[c] + beta * r[c]);
    }
    f[6] -= mr;
}

}  // namespace nbgpu
