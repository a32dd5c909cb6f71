// adjoint.cu — K6: vector-Jacobian product of the regular force step (no counterpart in the
// paper; derived by differentiating the sums of Sec. 2 / Sec. 3.2.1).
//
// For cotangents (ga_i, gj_i, s_i) of (acc_i, jerk_i, pot_i) and one pair with r = x_j - x_i,
// w = v_j - v_i, q = r.w, ar = ga.r, jr = gj.r, jw = gj.w, b = 3/|r|^2:
//   dL/dr   = m_j |r|^-3 [ ga + alpha r + beta w + gamma gj ]
//   dL/dw   = m_j |r|^-3 [ gj + beta r ]
//   dL/dm_j = |r|^-3 (ar + jw + gamma jr) - s / |r|
// with beta = -b jr, gamma = -b q, alpha = s - b (ar + jw - 5 q jr / |r|^2).
// Then g_x[j] += dL/dr, g_x[i] -= dL/dr (same for v), g_m[j] += dL/dm_j.
//
// Two passes without atomics in the pair loops:
//   i-side : each active i (in registers) over all j (j-tiles in shared memory, cp.async)
//            -> partial sums of dL/dr, dL/dw per i, per j-split
//   j-side : each particle j (in registers) over all active i (i-records with the
//            cotangents in shared memory) -> partial sums of dL/dr, dL/dw, dL/dm per j
// A combine kernel adds the partials in a fixed order and scatters the i-side sums with
// one atomic per (active i, component); for unique indices the result is deterministic.
// For dense blocks (n_i >= 3n/4), in either precision, one fused pass replaces the two: every
// particle carries its (possibly zero) cotangents, and each pair evaluated once gives both
// directions (i as the active row against j, and j as the active row against i).  In mixed
// precision the fused pass takes the particles in spatial order and measures separations from
// one anchor per CTA (k_adj_fused_anchored_x2), with close pairs replayed in double-single form.
// Self pairs are skipped by r^2 == 0 (distinct particles never coincide).
#include "nb_common.cuh"
#include "nb_kernels.cuh"

namespace nbgpu {

struct AdjArgs {
    const void *rec;     // j-records (as the forward)
    const void *irec;    // active i-records with cotangents (see k_pack_irec)
    int64_t n, n_i, n_tiles_j, n_tiles_i;
    const int32_t *idx;
    const double *g_acc, *g_jerk, *g_pot;
    int32_t S;           // splits of the streamed dimension
    double *part;        // [S][C][rows]
    unsigned *status;
};

// Pair terms: adds rinv^3 [ga + alpha r + beta w + gamma gj] to gr, rinv^3 [gj + beta r] to gv,
// and (optionally) dm.  rinv = 0 for the self pair.
template <typename T, bool WANT_DM>
__device__ __forceinline__ void adj_pair(T rx, T ry, T rz, T wx, T wy, T wz, T rinv, const T *ga, const T *gj, T s,
                                         T mscale, T *gr, T *gv, T &dm)
{
    const T rinv2 = rinv * rinv;
    const T rinv3 = rinv * rinv2 * mscale;
    const T q = rx * wx + ry * wy + rz * wz;
    const T ar = ga[0] * rx + ga[1] * ry + ga[2] * rz;
    const T jr = gj[0] * rx + gj[1] * ry + gj[2] * rz;
    const T jw = gj[0] * wx + gj[1] * wy + gj[2] * wz;
    const T b = T(3) * rinv2;
    const T t = ar + jw;
    const T beta = -b * jr;
    const T gamma = -b * q;
    const T alpha = s - b * (t - T(5) * rinv2 * q * jr);
    gr[0] += rinv3 * (ga[0] + alpha * rx + beta * wx + gamma * gj[0]);
    gr[1] += rinv3 * (ga[1] + alpha * ry + beta * wy + gamma * gj[1]);
    gr[2] += rinv3 * (ga[2] + alpha * rz + beta * wz + gamma * gj[2]);
    gv[0] += rinv3 * (gj[0] + beta * rx);
    gv[1] += rinv3 * (gj[1] + beta * ry);
    gv[2] += rinv3 * (gj[2] + beta * rz);
    if (WANT_DM) dm += rinv3 * (t + gamma * jr) - s * rinv;
}

// ---------------------------------------------------------------- i-record packing
// mixed: 4 float4 {xh,yh,zh,s} {xl,yl,zl,gj0} {vx,vy,vz,gj1} {ga0,ga1,ga2,gj2}
// FP64 : 4 dvec4  {x,y,z,s} {vx,vy,vz,gj0} {ga0,ga1,ga2,gj1} {gj2,0,0,0}
// Rows n_i .. n_tiles_i*TI-1 are padding with zero cotangents far away.
__global__ void k_pack_irec(AdjArgs A, int mixed, int64_t rows_pad)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < rows_pad;
         k += (int64_t)gridDim.x * blockDim.x) {
        int64_t g = -1;
        if (k < A.n_i) {
            g = A.idx[k];
            if (g < 0 || g >= A.n) {
                atomicOr(A.status, ST_BAD_INDEX);
                g = -1;
            }
        }
        if (mixed) {
            float4 *o = (float4 *)A.irec + 4 * k;
            if (g < 0) {
                o[0] = make_float4(kPadPos, kPadPos, kPadPos, 0.f);
                o[1] = o[2] = o[3] = make_float4(0.f, 0.f, 0.f, 0.f);
                continue;
            }
            const float4 *r = (const float4 *)A.rec + 3 * g;
            const float4 h = r[0], l = r[1], v = r[2];
            const double *ga = A.g_acc + 3 * k, *gj = A.g_jerk + 3 * k;
            o[0] = make_float4(h.x, h.y, h.z, (float)A.g_pot[k]);
            o[1] = make_float4(l.x, l.y, l.z, (float)gj[0]);
            o[2] = make_float4(v.x, v.y, v.z, (float)gj[1]);
            o[3] = make_float4((float)ga[0], (float)ga[1], (float)ga[2], (float)gj[2]);
        } else {
            dvec4 *o = (dvec4 *)A.irec + 4 * k;
            if (g < 0) {
                o[0] = make_dvec4(1e18, 1e18, 1e18, 0.0);
                o[1] = o[2] = o[3] = make_dvec4(0.0, 0.0, 0.0, 0.0);
                continue;
            }
            const dvec4 *r = (const dvec4 *)A.rec + 2 * g;
            const dvec4 x = r[0], v = r[1];
            const double *ga = A.g_acc + 3 * k, *gj = A.g_jerk + 3 * k;
            o[0] = make_dvec4(x.x, x.y, x.z, A.g_pot[k]);
            o[1] = make_dvec4(v.x, v.y, v.z, gj[0]);
            o[2] = make_dvec4(ga[0], ga[1], ga[2], gj[1]);
            o[3] = make_dvec4(gj[2], 0.0, 0.0, 0.0);
        }
    }
}

// ---------------------------------------------------------------- packed FP32x2 passes
// The mixed passes, with __ffma2_rn / __fadd2_rn / __fmul2_rn on pairs of rows: i-side rows
// (pass A) or j-side particles (pass B) are held two per packed register, the streamed side
// is expanded once per tile into a duplicated shared-memory layout.  The pair terms are the
// ones adj_pair states, with r, w and the differences in double-single form as in the
// forward kernels.
__device__ __forceinline__ float2 a2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 a2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 a2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Same terms as adj_pair for two pairs at once; rinv = 0 for a self pair.  gr, gv += rinv3
// [...] scaled by mscale; dm += rinv3 (t + gamma jr) - s rinv.
template <bool WANT_DM>
__device__ __forceinline__ void adj_pair_x2(const float2 (&r)[3], const float2 (&w)[3], float2 rinv,
                                            const float2 (&ga)[3], const float2 (&gj)[3], float2 s, float2 mscale,
                                            float2 (&gr)[3], float2 (&gv)[3], float2 &dm)
{
    const float2 rinv2 = a2mul(rinv, rinv);
    const float2 rinv3 = a2mul(rinv, rinv2);
    const float2 rinv3m = a2mul(rinv3, mscale);
    const float2 q = a2fma(r[2], w[2], a2fma(r[1], w[1], a2mul(r[0], w[0])));
    const float2 ar = a2fma(ga[2], r[2], a2fma(ga[1], r[1], a2mul(ga[0], r[0])));
    const float2 jr = a2fma(gj[2], r[2], a2fma(gj[1], r[1], a2mul(gj[0], r[0])));
    const float2 jw = a2fma(gj[2], w[2], a2fma(gj[1], w[1], a2mul(gj[0], w[0])));
    const float2 t = a2add(ar, jw);
    const float2 b3 = a2mul(rinv2, make_float2(-3.f, -3.f));
    const float2 beta = a2mul(b3, jr);
    const float2 gamma = a2mul(b3, q);
    const float2 v5 = a2mul(a2mul(q, jr), rinv2);
    const float2 alpha = a2fma(b3, a2fma(make_float2(-5.f, -5.f), v5, t), s);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 in = a2fma(gamma, gj[c], a2fma(beta, w[c], a2fma(alpha, r[c], ga[c])));
        gr[c] = a2fma(rinv3m, in, gr[c]);
        gv[c] = a2fma(rinv3m, a2fma(beta, r[c], gj[c]), gv[c]);
    }
    if (WANT_DM) {
        const float2 ns = make_float2(-s.x, -s.y);
        dm = a2add(dm, a2fma(ns, rinv, a2mul(rinv3, a2fma(gamma, jr, t))));
    }
}

__device__ __forceinline__ float2 rsqrt_nz(float2 r2)
{
    return make_float2(r2.x > 0.f ? rsqrtf(r2.x) : 0.f, r2.y > 0.f ? rsqrtf(r2.y) : 0.f);
}

template <int NI, int BLOCK, int TJ>
constexpr int adj_iside_x2_smem()
{
    return 3 * TJ * 16 + 5 * TJ * 16 + 6 * NI * BLOCK * 8;
}

// Pass A: NI active rows per thread (NI/2 packed pairs) against j-tiles of all particles.
template <int NI, int BLOCK, int TJ, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_adj_iside_x2(AdjArgs A)
{
    constexpr int NP = NI / 2;
    extern __shared__ __align__(16) float4 adj_smem[];
    float4 *raw = adj_smem;
    float4 *dup = adj_smem + 3 * TJ;
    double *dacc = reinterpret_cast<double *>(adj_smem + 8 * TJ);  // [6][NI][BLOCK]
    const int tid = threadIdx.x;
    const int64_t kbase = (int64_t)blockIdx.x * (BLOCK * NI);
    const int s = blockIdx.y;
    const int64_t t0 = (A.n_tiles_j * s) / A.S, t1 = (A.n_tiles_j * (s + 1)) / A.S;
    const float4 *rec = static_cast<const float4 *>(A.rec);
    const float4 *irec = static_cast<const float4 *>(A.irec);
    float2 nh[NP][3], nl[NP][3], nv[NP][3], ga[NP][3], gj[NP][3], gs[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float4 a[2], b[2], c[2], d[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {  // irec rows are padded: always readable
            const int64_t k = kbase + (2 * p + u) * BLOCK + tid;
            a[u] = irec[4 * k]; b[u] = irec[4 * k + 1]; c[u] = irec[4 * k + 2]; d[u] = irec[4 * k + 3];
        }
        nh[p][0] = make_float2(-a[0].x, -a[1].x); nh[p][1] = make_float2(-a[0].y, -a[1].y);
        nh[p][2] = make_float2(-a[0].z, -a[1].z); gs[p] = make_float2(a[0].w, a[1].w);
        nl[p][0] = make_float2(-b[0].x, -b[1].x); nl[p][1] = make_float2(-b[0].y, -b[1].y);
        nl[p][2] = make_float2(-b[0].z, -b[1].z); gj[p][0] = make_float2(b[0].w, b[1].w);
        nv[p][0] = make_float2(-c[0].x, -c[1].x); nv[p][1] = make_float2(-c[0].y, -c[1].y);
        nv[p][2] = make_float2(-c[0].z, -c[1].z); gj[p][1] = make_float2(c[0].w, c[1].w);
        ga[p][0] = make_float2(d[0].x, d[1].x); ga[p][1] = make_float2(d[0].y, d[1].y);
        ga[p][2] = make_float2(d[0].z, d[1].z); gj[p][2] = make_float2(d[0].w, d[1].w);
    }
#pragma unroll
    for (int e = 0; e < 6 * NI; ++e) dacc[e * BLOCK + tid] = 0.0;
    auto load_tile = [&](int64_t t) {
        const float4 *src = rec + t * (3 * TJ);
#pragma unroll
        for (int e = tid; e < 3 * TJ; e += BLOCK) cp_async16(&raw[e], src + e);
        cp_async_commit();
    };
    if (t0 < t1) load_tile(t0);
    for (int64_t t = t0; t < t1; ++t) {
        cp_async_wait<0>();
        __syncthreads();
#pragma unroll
        for (int jj = tid; jj < TJ; jj += BLOCK) {
            const float4 p0 = raw[3 * jj], p1 = raw[3 * jj + 1], p2 = raw[3 * jj + 2];
            dup[5 * jj] = make_float4(p0.x, p0.x, p0.y, p0.y);
            dup[5 * jj + 1] = make_float4(p0.z, p0.z, p0.w, p0.w);
            dup[5 * jj + 2] = make_float4(p1.x, p1.x, p1.y, p1.y);
            dup[5 * jj + 3] = make_float4(p1.z, p1.z, p2.x, p2.x);
            dup[5 * jj + 4] = make_float4(p2.y, p2.y, p2.z, p2.z);
        }
        __syncthreads();
        if (t + 1 < t1) load_tile(t + 1);
        float2 gr[NP][3], gv[NP][3], dm_unused = make_float2(0.f, 0.f);
#pragma unroll
        for (int p = 0; p < NP; ++p)
#pragma unroll
            for (int c = 0; c < 3; ++c) gr[p][c] = gv[p][c] = make_float2(0.f, 0.f);
#pragma unroll 2
        for (int jj = 0; jj < TJ; ++jj) {
            const float4 a = dup[5 * jj], b = dup[5 * jj + 1], c = dup[5 * jj + 2], d = dup[5 * jj + 3],
                         e = dup[5 * jj + 4];
            const float2 XH[3] = {make_float2(a.x, a.y), make_float2(a.z, a.w), make_float2(b.x, b.y)};
            const float2 M = make_float2(b.z, b.w);
            const float2 XL[3] = {make_float2(c.x, c.y), make_float2(c.z, c.w), make_float2(d.x, d.y)};
            const float2 V[3] = {make_float2(d.z, d.w), make_float2(e.x, e.y), make_float2(e.z, e.w)};
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                float2 r[3], w[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    r[k] = a2add(a2add(XH[k], nh[p][k]), a2add(XL[k], nl[p][k]));
                    w[k] = a2add(V[k], nv[p][k]);
                }
                const float2 r2 = a2fma(r[2], r[2], a2fma(r[1], r[1], a2mul(r[0], r[0])));
                adj_pair_x2<false>(r, w, rsqrt_nz(r2), ga[p], gj[p], gs[p], M, gr[p], gv[p], dm_unused);
            }
        }
#pragma unroll
        for (int p = 0; p < NP; ++p)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dacc[(c * NI + 2 * p) * BLOCK + tid] += (double)gr[p][c].x;
                dacc[(c * NI + 2 * p + 1) * BLOCK + tid] += (double)gr[p][c].y;
                dacc[((3 + c) * NI + 2 * p) * BLOCK + tid] += (double)gv[p][c].x;
                dacc[((3 + c) * NI + 2 * p + 1) * BLOCK + tid] += (double)gv[p][c].y;
            }
    }
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int64_t k = kbase + q * BLOCK + tid;
        if (k < A.n_i)
#pragma unroll
            for (int c = 0; c < 6; ++c) A.part[((int64_t)s * 6 + c) * A.n_i + k] = dacc[(c * NI + q) * BLOCK + tid];
    }
}

template <int NJ, int BLOCK, int TI>
constexpr int adj_jside_x2_smem()
{
    return 4 * TI * 16 + 8 * TI * 16 + 7 * NJ * BLOCK * 8;
}

// Pass B: NJ particles per thread (NJ/2 packed pairs) against tiles of the active rows with
// their cotangents.  Expanded i-record, eight float4 per row:
//   {-xh,-xh,-yh,-yh} {-zh,-zh,s,s} {-xl,-xl,-yl,-yl} {-zl,-zl,-vx,-vx}
//   {-vy,-vy,-vz,-vz} {ga0,ga0,ga1,ga1} {ga2,ga2,gj0,gj0} {gj1,gj1,gj2,gj2}
template <int NJ, int BLOCK, int TI, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_adj_jside_x2(AdjArgs A)
{
    constexpr int NP = NJ / 2;
    extern __shared__ __align__(16) float4 adj_smem[];
    float4 *raw = adj_smem;                 // 4*TI float4
    float4 *dup = adj_smem + 4 * TI;        // 8*TI float4
    double *dacc = reinterpret_cast<double *>(adj_smem + 12 * TI);  // [7][NJ][BLOCK]
    const int tid = threadIdx.x;
    const int64_t jbase = (int64_t)blockIdx.x * (BLOCK * NJ);
    const int s = blockIdx.y;
    const int64_t t0 = (A.n_tiles_i * s) / A.S, t1 = (A.n_tiles_i * (s + 1)) / A.S;
    const float4 *rec = static_cast<const float4 *>(A.rec);
    const float4 *irec = static_cast<const float4 *>(A.irec);
    float2 jh[NP][3], jl[NP][3], jv[NP][3], jm[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float4 a[2], b[2], c[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t j = jbase + (2 * p + u) * BLOCK + tid;
            if (j < A.n) {
                a[u] = rec[3 * j]; b[u] = rec[3 * j + 1]; c[u] = rec[3 * j + 2];
            } else {  // beyond the particles: a massless row far away (never written)
                a[u] = make_float4(kPadPos, kPadPos, kPadPos, 0.f);
                b[u] = c[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        jh[p][0] = make_float2(a[0].x, a[1].x); jh[p][1] = make_float2(a[0].y, a[1].y);
        jh[p][2] = make_float2(a[0].z, a[1].z); jm[p] = make_float2(a[0].w, a[1].w);
        jl[p][0] = make_float2(b[0].x, b[1].x); jl[p][1] = make_float2(b[0].y, b[1].y);
        jl[p][2] = make_float2(b[0].z, b[1].z);
        jv[p][0] = make_float2(c[0].x, c[1].x); jv[p][1] = make_float2(c[0].y, c[1].y);
        jv[p][2] = make_float2(c[0].z, c[1].z);
    }
#pragma unroll
    for (int e = 0; e < 7 * NJ; ++e) dacc[e * BLOCK + tid] = 0.0;
    auto load_tile = [&](int64_t t) {
        const float4 *src = irec + t * (4 * TI);
#pragma unroll
        for (int e = tid; e < 4 * TI; e += BLOCK) cp_async16(&raw[e], src + e);
        cp_async_commit();
    };
    if (t0 < t1) load_tile(t0);
    for (int64_t t = t0; t < t1; ++t) {
        cp_async_wait<0>();
        __syncthreads();
#pragma unroll
        for (int ii = tid; ii < TI; ii += BLOCK) {
            const float4 a = raw[4 * ii], b = raw[4 * ii + 1], c = raw[4 * ii + 2], d = raw[4 * ii + 3];
            dup[8 * ii] = make_float4(-a.x, -a.x, -a.y, -a.y);
            dup[8 * ii + 1] = make_float4(-a.z, -a.z, a.w, a.w);
            dup[8 * ii + 2] = make_float4(-b.x, -b.x, -b.y, -b.y);
            dup[8 * ii + 3] = make_float4(-b.z, -b.z, -c.x, -c.x);
            dup[8 * ii + 4] = make_float4(-c.y, -c.y, -c.z, -c.z);
            dup[8 * ii + 5] = make_float4(d.x, d.x, d.y, d.y);
            dup[8 * ii + 6] = make_float4(d.z, d.z, b.w, b.w);
            dup[8 * ii + 7] = make_float4(c.w, c.w, d.w, d.w);
        }
        __syncthreads();
        if (t + 1 < t1) load_tile(t + 1);
        float2 gr[NP][3], gv[NP][3], dm[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            dm[p] = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < 3; ++c) gr[p][c] = gv[p][c] = make_float2(0.f, 0.f);
        }
#pragma unroll 2
        for (int ii = 0; ii < TI; ++ii) {
            const float4 a = dup[8 * ii], b = dup[8 * ii + 1], c = dup[8 * ii + 2], d = dup[8 * ii + 3],
                         e = dup[8 * ii + 4], f = dup[8 * ii + 5], g = dup[8 * ii + 6], h = dup[8 * ii + 7];
            const float2 NH[3] = {make_float2(a.x, a.y), make_float2(a.z, a.w), make_float2(b.x, b.y)};
            const float2 S = make_float2(b.z, b.w);
            const float2 NL[3] = {make_float2(c.x, c.y), make_float2(c.z, c.w), make_float2(d.x, d.y)};
            const float2 NV[3] = {make_float2(d.z, d.w), make_float2(e.x, e.y), make_float2(e.z, e.w)};
            const float2 GA[3] = {make_float2(f.x, f.y), make_float2(f.z, f.w), make_float2(g.x, g.y)};
            const float2 GJ[3] = {make_float2(g.z, g.w), make_float2(h.x, h.y), make_float2(h.z, h.w)};
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                float2 r[3], w[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    r[k] = a2add(a2add(jh[p][k], NH[k]), a2add(jl[p][k], NL[k]));
                    w[k] = a2add(jv[p][k], NV[k]);
                }
                const float2 r2 = a2fma(r[2], r[2], a2fma(r[1], r[1], a2mul(r[0], r[0])));
                adj_pair_x2<true>(r, w, rsqrt_nz(r2), GA, GJ, S, make_float2(1.f, 1.f), gr[p], gv[p], dm[p]);
            }
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                dacc[(c * NJ + 2 * p) * BLOCK + tid] += (double)gr[p][c].x;
                dacc[(c * NJ + 2 * p + 1) * BLOCK + tid] += (double)gr[p][c].y;
                dacc[((3 + c) * NJ + 2 * p) * BLOCK + tid] += (double)gv[p][c].x;
                dacc[((3 + c) * NJ + 2 * p + 1) * BLOCK + tid] += (double)gv[p][c].y;
            }
            dacc[(6 * NJ + 2 * p) * BLOCK + tid] += (double)dm[p].x;
            dacc[(6 * NJ + 2 * p + 1) * BLOCK + tid] += (double)dm[p].y;
        }
    }
#pragma unroll
    for (int q = 0; q < NJ; ++q) {
        const int64_t j = jbase + q * BLOCK + tid;
        if (j < A.n) {
            const double mj = (double)(q & 1 ? jm[q >> 1].y : jm[q >> 1].x);
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                const double v = dacc[(c * NJ + q) * BLOCK + tid];
                A.part[((int64_t)s * 7 + c) * A.n + j] = c < 6 ? v * mj : v;
            }
        }
    }
}

// ---------------------------------------------------------------- fused single pass (mixed)
// For dense active blocks.  Every particle k is a row; its cotangents (zero when k is not
// active, summed when idx names k twice) live in a per-particle record next to its position:
//   crec (five float4): {xh,yh,zh,m} {xl,yl,zl,s} {vx,vy,vz,gj0} {ga0,ga1,ga2,gj1} {gj2,0,0,0}
// For the pair (k, m) with r = x_m - x_k, w = v_m - v_k the shared terms (r, w, 1/|r|, r.w)
// are formed once and both directions are added:
//   k as receiver (cotangents of k):  g_x[k] -= m_m V(r, w; c_k),  g_v[k] -= m_m U(r, w; c_k)
//   m as receiver (cotangents of m):  g_x[k] += m_k V(-r, -w; c_m), g_v[k] += m_k U(-r, -w; c_m),
//                                     g_m[k] += D(-r, -w; c_m)
// with V, U, D the bracketed terms of adj_pair.  In terms of P = ga_m.r, Q = gj_m.r,
// R = gj_m.w and E = P + R - 5 q Q / |r|^2 the reversed pair reads
//   V = ga_m - (s_m + 3 E / |r|^2) r - 3 Q w / |r|^2 + gamma gj_m,  U = gj_m - 3 Q r / |r|^2,
//   D = -|r|^-3 (P + R + gamma Q) - s_m / |r|,  gamma = -3 q / |r|^2.
// Every active index must appear once: each row's cotangents are written into its particle's
// record, and the i-side sums are added into g_x, g_v of that particle.  claim (n words) is
// zero on entry; a second claim of the same particle flags ST_DUP_INDEX (the call then fails
// with NB_ERR_ARG and its outputs are unspecified).
__global__ void k_check_unique(int64_t n, int64_t n_i, const int32_t *__restrict__ idx, unsigned *__restrict__ claim,
                               unsigned *status)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_i; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx[q];
        if (i < 0 || i >= n) continue;  // reported by the kernels that use the row
        if (atomicExch(claim + i, 1u) != 0u) atomicOr(status, ST_DUP_INDEX);
    }
}

__global__ void k_build_crec(int64_t n, int64_t n_pad, const float4 *__restrict__ rec, float4 *__restrict__ crec)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_pad; k += (int64_t)gridDim.x * blockDim.x) {
        float4 a = make_float4(kPadPos, kPadPos, kPadPos, 0.f), b = make_float4(0.f, 0.f, 0.f, 0.f), c = b;
        if (k < n) {
            a = rec[3 * k];
            b = rec[3 * k + 1];
            c = rec[3 * k + 2];
        }
        crec[5 * k] = a;
        crec[5 * k + 1] = make_float4(b.x, b.y, b.z, 0.f);
        crec[5 * k + 2] = make_float4(c.x, c.y, c.z, 0.f);
        crec[5 * k + 3] = make_float4(0.f, 0.f, 0.f, 0.f);
        crec[5 * k + 4] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__global__ void k_scatter_cotangents(int64_t n, int64_t n_i, const int32_t *__restrict__ idx,
                                     const double *__restrict__ g_acc, const double *__restrict__ g_jerk,
                                     const double *__restrict__ g_pot, float *__restrict__ crec, unsigned *status)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_i; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx[q];
        if (i < 0 || i >= n) {
            atomicOr(status, ST_BAD_INDEX);
            continue;
        }
        // idx is checked for duplicates first (k_check_unique), so one row writes each record
        float *r = crec + 20 * i;  // five float4 = 20 floats
        r[7] = (float)g_pot[q];         // s
        r[11] = (float)g_jerk[3 * q];   // gj0
        r[12] = (float)g_acc[3 * q];    // ga0
        r[13] = (float)g_acc[3 * q + 1];
        r[14] = (float)g_acc[3 * q + 2];
        r[15] = (float)g_jerk[3 * q + 1];  // gj1
        r[16] = (float)g_jerk[3 * q + 2];  // gj2
    }
}

// FP32 sums of one row pair over a j-tile in the fused pass, and their promotion to the FP64
// running sums dacc[c][2][BLOCK] (c: g_x 0-2, g_v 3-5, g_m 6).
struct AdjTileSums {
    float2 s0, s1, A1[3], B1[3], C1[3], v2[3], u2[3], d2;
    __device__ __forceinline__ void zero()
    {
        s0 = s1 = d2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 3; ++c) A1[c] = B1[c] = C1[c] = v2[c] = u2[c] = make_float2(0.f, 0.f);
    }
    template <int BLOCK>
    __device__ __forceinline__ void promote(const float2 (&ga)[3], const float2 (&gj)[3], float2 mk, double *dacc,
                                            int tid) const
    {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 v1 = a2add(a2fma(ga[c], s0, a2mul(gj[c], s1)), a2add(A1[c], B1[c]));
            const float2 u1 = a2fma(gj[c], s0, C1[c]);
            const float2 gx = a2fma(mk, v2[c], make_float2(-v1.x, -v1.y));
            const float2 gv = a2fma(mk, u2[c], make_float2(-u1.x, -u1.y));
            dacc[(c * 2) * BLOCK + tid] += (double)gx.x;
            dacc[(c * 2 + 1) * BLOCK + tid] += (double)gx.y;
            dacc[((3 + c) * 2) * BLOCK + tid] += (double)gv.x;
            dacc[((3 + c) * 2 + 1) * BLOCK + tid] += (double)gv.y;
        }
        dacc[12 * BLOCK + tid] += (double)d2.x;
        dacc[13 * BLOCK + tid] += (double)d2.y;
    }
};

// One pair (row pair k against source m) of the fused pass: separation r = x_m - x_k, w =
// v_m - v_k, rinv = 1/|r| (0 zeroes every term: the self pair, or a pair handled elsewhere);
// m's mass M, its cotangents Sm, GAm, GJm; k's cotangents ga, gj, gs.
__device__ __forceinline__ void adj_fused_pair(const float2 (&r)[3], const float2 (&w)[3], float2 rinv, float2 M,
                                               float2 Sm, const float2 (&GAm)[3], const float2 (&GJm)[3],
                                               const float2 (&ga)[3], const float2 (&gj)[3], float2 gs,
                                               AdjTileSums &S)
{
    const float2 m3 = make_float2(-3.f, -3.f), m5 = make_float2(-5.f, -5.f);
    const float2 rinv2 = a2mul(rinv, rinv);
    const float2 rinv3 = a2mul(rinv, rinv2);
    const float2 q = a2fma(r[2], w[2], a2fma(r[1], w[1], a2mul(r[0], w[0])));
    const float2 b3 = a2mul(rinv2, m3);
    const float2 gamma = a2mul(b3, q);
    // k as receiver (cotangents of k), source mass m_m
    {
        const float2 ar = a2fma(ga[2], r[2], a2fma(ga[1], r[1], a2mul(ga[0], r[0])));
        const float2 jr = a2fma(gj[2], r[2], a2fma(gj[1], r[1], a2mul(gj[0], r[0])));
        const float2 jw = a2fma(gj[2], w[2], a2fma(gj[1], w[1], a2mul(gj[0], w[0])));
        const float2 tt = a2add(ar, jw);
        const float2 beta = a2mul(b3, jr);
        const float2 alpha = a2fma(b3, a2fma(m5, a2mul(a2mul(q, jr), rinv2), tt), gs);
        const float2 rinv3m = a2mul(rinv3, M);
        S.s0 = a2add(S.s0, rinv3m);
        S.s1 = a2fma(rinv3m, gamma, S.s1);
        const float2 ra = a2mul(rinv3m, alpha), rb = a2mul(rinv3m, beta);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            S.A1[c] = a2fma(ra, r[c], S.A1[c]);
            S.B1[c] = a2fma(rb, w[c], S.B1[c]);
            S.C1[c] = a2fma(rb, r[c], S.C1[c]);
        }
    }
    // m as receiver (cotangents of m), source k (mass m_k applied per tile)
    {
        const float2 P = a2fma(GAm[2], r[2], a2fma(GAm[1], r[1], a2mul(GAm[0], r[0])));
        const float2 Q = a2fma(GJm[2], r[2], a2fma(GJm[1], r[1], a2mul(GJm[0], r[0])));
        const float2 R = a2fma(GJm[2], w[2], a2fma(GJm[1], w[1], a2mul(GJm[0], w[0])));
        const float2 PR = a2add(P, R);
        const float2 b3Q = a2mul(b3, Q);
        const float2 E = a2fma(m5, a2mul(a2mul(q, Q), rinv2), PR);
        // alpha' = s_m - b3 E, applied as -alpha' r
        const float2 nalpha = a2fma(b3, E, make_float2(-Sm.x, -Sm.y));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 in = a2fma(gamma, GJm[c], a2fma(b3Q, w[c], a2fma(nalpha, r[c], GAm[c])));
            S.v2[c] = a2fma(rinv3, in, S.v2[c]);
            S.u2[c] = a2fma(rinv3, a2fma(b3Q, r[c], GJm[c]), S.u2[c]);
        }
        const float2 nd = a2fma(rinv3, a2fma(gamma, Q, PR), a2mul(Sm, rinv));
        S.d2 = a2add(S.d2, make_float2(-nd.x, -nd.y));
    }
}

// ---------------------------------------------------------------- anchored fused pass (mixed)
// The fused pass with the anchored separations of the forward's anchored kernel: the rows (all
// particles) are taken in the spatial order perm (Morton order, so a CTA's rows lie close
// together), every position is measured from one anchor B per CTA (the predicted position of
// its middle row), e_k = ds(x_k - B) once per row and f_m = ds(x_m - B) once per source and CTA,
// rounded to FP32, and the separation is the single subtraction f_m - e_k (3 FP32 lane-operations
// a pair where the double-single difference takes 9).  Its error is at most about
// 4u |x_k - B| + 3u |r| (u = 2^-24); pairs with |r| below |x_k - B| / 16, where that is not small
// against |r|, and the self pair (separation exactly zero), are masked out of the loop (inverse
// distance 0 zeroes every term) and replayed after each 32-source chunk with the double-single
// separation ((hi - hi) + (lo - lo), as in the forward kernels), so every pair is computed to
// the double-single accuracy or better.
// Duplicated tile, nine float4 per source:
//   {fx,fx,fy,fy} {fz,fz,m,m} {vx,vx,vy,vy} {vz,vz,s,s} {ga0,ga0,ga1,ga1} {ga2,ga2,gj0,gj0}
//   {gj1,gj1,gj2,gj2} {xh,yh,zh,xl} {yl,zl,0,0}
// (the loop reads the first seven; the replay also reads the absolute hi/lo position).  The
// rows' own hi/lo positions are kept in shared memory for the replay.
template <int BLOCK, int TJ>
constexpr int adj_anchored_smem()
{
    return 5 * TJ * 16 + 9 * TJ * 16 + 7 * 2 * BLOCK * 8 + 6 * 2 * BLOCK * 4;
}

template <int BLOCK, int TJ, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB)
    k_adj_fused_anchored_x2(AdjArgs A, const float4 *__restrict__ crec, const int32_t *__restrict__ perm)
{
    extern __shared__ __align__(16) float4 adj_smem[];
    float4 *raw = adj_smem;                 // 5*TJ
    float4 *dup = adj_smem + 5 * TJ;        // 9*TJ
    double *dacc = reinterpret_cast<double *>(adj_smem + 14 * TJ);  // [7][2][BLOCK]
    float *spos = reinterpret_cast<float *>(dacc + 14 * BLOCK);     // [6][2][BLOCK]: hi xyz, lo xyz
    __shared__ float s_anchor[6];
    const int tid = threadIdx.x;
    const int64_t kbase = (int64_t)blockIdx.x * (2 * BLOCK);
    const int s = blockIdx.y;
    const int64_t t0 = (A.n_tiles_j * s) / A.S, t1 = (A.n_tiles_j * (s + 1)) / A.S;
    if (tid == 0) {  // anchor: the middle row of the CTA's valid rows
        const int64_t rows = A.n - kbase < 2 * BLOCK ? A.n - kbase : 2 * BLOCK;
        const int64_t ka = perm[kbase + (rows > 0 ? rows / 2 : 0)];
        const float4 h = crec[5 * ka], l = crec[5 * ka + 1];
        s_anchor[0] = h.x; s_anchor[1] = h.y; s_anchor[2] = h.z;
        s_anchor[3] = l.x; s_anchor[4] = l.y; s_anchor[5] = l.z;
    }
    __syncthreads();
    const float Bh[3] = {s_anchor[0], s_anchor[1], s_anchor[2]}, Bl[3] = {s_anchor[3], s_anchor[4], s_anchor[5]};
    float2 ne[3], nv[3], ga[3], gj[3], gs, mk, tm;
    int64_t krow[2];
    {
        float4 a[2], b[2], c[2], d[2], e[2];
        float tmu[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {  // crec is padded to the tile multiple; rows past n are padding
            const int64_t r = kbase + u * BLOCK + tid;
            const int64_t k = r < A.n ? perm[r] : r;
            krow[u] = k;
            a[u] = crec[5 * k]; b[u] = crec[5 * k + 1]; c[u] = crec[5 * k + 2];
            d[u] = crec[5 * k + 3]; e[u] = crec[5 * k + 4];
            const float ex = ds_diff(a[u].x, b[u].x, Bh[0], Bl[0]);
            const float ey = ds_diff(a[u].y, b[u].y, Bh[1], Bl[1]);
            const float ez = ds_diff(a[u].z, b[u].z, Bh[2], Bl[2]);
            const int slot = u * BLOCK + tid;
            spos[0 * 2 * BLOCK + slot] = a[u].x; spos[1 * 2 * BLOCK + slot] = a[u].y; spos[2 * 2 * BLOCK + slot] = a[u].z;
            spos[3 * 2 * BLOCK + slot] = b[u].x; spos[4 * 2 * BLOCK + slot] = b[u].y; spos[5 * 2 * BLOCK + slot] = b[u].z;
            if (u == 0) { ne[0].x = -ex; ne[1].x = -ey; ne[2].x = -ez; }
            else { ne[0].y = -ex; ne[1].y = -ey; ne[2].y = -ez; }
            tmu[u] = r < A.n ? fmaxf(r2_f32(ex, ey, ez) * (1.f / 256.f), 1.17549435e-38f) : -1.f;
        }
        mk = make_float2(a[0].w, a[1].w);
        gs = make_float2(b[0].w, b[1].w);
        nv[0] = make_float2(-c[0].x, -c[1].x); nv[1] = make_float2(-c[0].y, -c[1].y);
        nv[2] = make_float2(-c[0].z, -c[1].z); gj[0] = make_float2(c[0].w, c[1].w);
        ga[0] = make_float2(d[0].x, d[1].x); ga[1] = make_float2(d[0].y, d[1].y);
        ga[2] = make_float2(d[0].z, d[1].z); gj[1] = make_float2(d[0].w, d[1].w);
        gj[2] = make_float2(e[0].x, e[1].x);
        tm = make_float2(tmu[0], tmu[1]);
    }
#pragma unroll
    for (int e = 0; e < 14; ++e) dacc[e * BLOCK + tid] = 0.0;
    auto load_tile = [&](int64_t t) {
        const float4 *src = crec + t * (5 * TJ);
#pragma unroll
        for (int e = tid; e < 5 * TJ; e += BLOCK) cp_async16(&raw[e], src + e);
        cp_async_commit();
    };
    if (t0 < t1) load_tile(t0);
    for (int64_t t = t0; t < t1; ++t) {
        cp_async_wait<0>();
        __syncthreads();
#pragma unroll
        for (int jj = tid; jj < TJ; jj += BLOCK) {
            const float4 a = raw[5 * jj], b = raw[5 * jj + 1], c = raw[5 * jj + 2], d = raw[5 * jj + 3],
                         e = raw[5 * jj + 4];
            const float fx = ds_diff(a.x, b.x, Bh[0], Bl[0]);
            const float fy = ds_diff(a.y, b.y, Bh[1], Bl[1]);
            const float fz = ds_diff(a.z, b.z, Bh[2], Bl[2]);
            dup[9 * jj] = make_float4(fx, fx, fy, fy);
            dup[9 * jj + 1] = make_float4(fz, fz, a.w, a.w);
            dup[9 * jj + 2] = make_float4(c.x, c.x, c.y, c.y);
            dup[9 * jj + 3] = make_float4(c.z, c.z, b.w, b.w);
            dup[9 * jj + 4] = make_float4(d.x, d.x, d.y, d.y);
            dup[9 * jj + 5] = make_float4(d.z, d.z, c.w, c.w);
            dup[9 * jj + 6] = make_float4(d.w, d.w, e.x, e.x);
            dup[9 * jj + 7] = make_float4(a.x, a.y, a.z, b.x);
            dup[9 * jj + 8] = make_float4(b.y, b.z, 0.f, 0.f);
        }
        __syncthreads();
        if (t + 1 < t1) load_tile(t + 1);
        AdjTileSums S;
        S.zero();
        for (int jc = 0; jc < TJ; jc += 32) {
            const float4 *sc = dup + 9 * jc;
            unsigned hm0 = 0, hm1 = 0;
#pragma unroll 2
            for (int u = 0; u < 32; ++u) {
                const float4 q0 = sc[9 * u], q1 = sc[9 * u + 1], q2 = sc[9 * u + 2], q3 = sc[9 * u + 3],
                             q4 = sc[9 * u + 4], q5 = sc[9 * u + 5], q6 = sc[9 * u + 6];
                const float2 M = make_float2(q1.z, q1.w), Sm = make_float2(q3.z, q3.w);
                const float2 GAm[3] = {make_float2(q4.x, q4.y), make_float2(q4.z, q4.w), make_float2(q5.x, q5.y)};
                const float2 GJm[3] = {make_float2(q5.z, q5.w), make_float2(q6.x, q6.y), make_float2(q6.z, q6.w)};
                float2 r[3], w[3];
                r[0] = a2add(make_float2(q0.x, q0.y), ne[0]);
                r[1] = a2add(make_float2(q0.z, q0.w), ne[1]);
                r[2] = a2add(make_float2(q1.x, q1.y), ne[2]);
                w[0] = a2add(make_float2(q2.x, q2.y), nv[0]);
                w[1] = a2add(make_float2(q2.z, q2.w), nv[1]);
                w[2] = a2add(make_float2(q3.x, q3.y), nv[2]);
                const float2 r2 = a2fma(r[2], r[2], a2fma(r[1], r[1], a2mul(r[0], r[0])));
                const bool m0 = r2.x < tm.x, m1 = r2.y < tm.y;
                hm0 |= (unsigned)m0 << u;
                hm1 |= (unsigned)m1 << u;
                float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                rinv.x = m0 ? 0.f : rinv.x;
                rinv.y = m1 ? 0.f : rinv.y;
                adj_fused_pair(r, w, rinv, M, Sm, GAm, GJm, ga, gj, gs, S);
            }
            // masked pairs: the double-single separation, one row of the pair at a time
            unsigned hm = hm0 | hm1;
            while (hm) {
                const int u = __ffs(hm) - 1;
                hm &= hm - 1;
                const float4 q0 = sc[9 * u + 1], q2 = sc[9 * u + 2], q3 = sc[9 * u + 3], q4 = sc[9 * u + 4],
                             q5 = sc[9 * u + 5], q6 = sc[9 * u + 6], q7 = sc[9 * u + 7], q8 = sc[9 * u + 8];
                const float2 M = make_float2(q0.z, q0.w), Sm = make_float2(q3.z, q3.w);
                const float2 GAm[3] = {make_float2(q4.x, q4.y), make_float2(q4.z, q4.w), make_float2(q5.x, q5.y)};
                const float2 GJm[3] = {make_float2(q5.z, q5.w), make_float2(q6.x, q6.y), make_float2(q6.z, q6.w)};
                const float jh[3] = {q7.x, q7.y, q7.z}, jl[3] = {q7.w, q8.x, q8.y};
                float2 w[3];
                w[0] = a2add(make_float2(q2.x, q2.y), nv[0]);
                w[1] = a2add(make_float2(q2.z, q2.w), nv[1]);
                w[2] = a2add(make_float2(q3.x, q3.y), nv[2]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (!(((h ? hm1 : hm0) >> u) & 1u)) continue;
                    const int slot = h * BLOCK + tid;
                    float2 r[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float d = ds_diff(jh[c], jl[c], spos[c * 2 * BLOCK + slot], spos[(3 + c) * 2 * BLOCK + slot]);
                        r[c] = make_float2(d, d);
                    }
                    const float r2 = r2_f32(r[0].x, r[1].x, r[2].x);
                    const float ri = r2 > 0.f ? rsqrtf(r2) : 0.f;  // the self pair has r = 0
                    adj_fused_pair(r, w, h ? make_float2(0.f, ri) : make_float2(ri, 0.f), M, Sm, GAm, GJm, ga, gj, gs, S);
                }
            }
        }
        S.promote<BLOCK>(ga, gj, mk, dacc, tid);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int64_t k = krow[u];
        if (k < A.n)
#pragma unroll
            for (int c = 0; c < 7; ++c) A.part[((int64_t)s * 7 + c) * A.n + k] = dacc[(c * 2 + u) * BLOCK + tid];
    }
}

// ---------------------------------------------------------------- fused single pass (FP64)
// The same pair algebra as the mixed fused pass (adj_fused_pair), in FP64 with one row per thread and the sums kept
// in FP64 registers.  Records (four dvec4):
//   {x,y,z,m} {vx,vy,vz,s} {ga0,ga1,ga2,gj0} {gj1,gj2,0,0}
__global__ void k_build_crec64(int64_t n, int64_t n_pad, const dvec4 *__restrict__ rec, dvec4 *__restrict__ crec)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_pad; k += (int64_t)gridDim.x * blockDim.x) {
        dvec4 a = make_dvec4(1e18, 1e18, 1e18, 0.0), b = make_dvec4(0.0, 0.0, 0.0, 0.0);
        if (k < n) {
            a = rec[2 * k];
            b = rec[2 * k + 1];
        }
        crec[4 * k] = a;
        crec[4 * k + 1] = make_dvec4(b.x, b.y, b.z, 0.0);
        crec[4 * k + 2] = make_dvec4(0.0, 0.0, 0.0, 0.0);
        crec[4 * k + 3] = make_dvec4(0.0, 0.0, 0.0, 0.0);
    }
}

__global__ void k_scatter_cotangents64(int64_t n, int64_t n_i, const int32_t *__restrict__ idx,
                                       const double *__restrict__ g_acc, const double *__restrict__ g_jerk,
                                       const double *__restrict__ g_pot, double *__restrict__ crec, unsigned *status)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_i; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx[q];
        if (i < 0 || i >= n) {
            atomicOr(status, ST_BAD_INDEX);
            continue;
        }
        double *r = crec + 16 * i;  // four dvec4 = 16 doubles; one row writes each record
        r[7] = g_pot[q];       // s
        r[8] = g_acc[3 * q];   // ga
        r[9] = g_acc[3 * q + 1];
        r[10] = g_acc[3 * q + 2];
        r[11] = g_jerk[3 * q];  // gj
        r[12] = g_jerk[3 * q + 1];
        r[13] = g_jerk[3 * q + 2];
    }
}

template <int BLOCK, int TJ>
__global__ void __launch_bounds__(BLOCK) k_adj_fused_f64(AdjArgs A, const dvec4 *__restrict__ crec)
{
    __shared__ dvec4 sj[2][4 * TJ];
    const int tid = threadIdx.x;
    const int64_t k = (int64_t)blockIdx.x * BLOCK + tid;  // crec is padded past every row
    const int s = blockIdx.y;
    const int64_t t0 = (A.n_tiles_j * s) / A.S, t1 = (A.n_tiles_j * (s + 1)) / A.S;
    const dvec4 a = crec[4 * k], b = crec[4 * k + 1], c = crec[4 * k + 2], d = crec[4 * k + 3];
    const double xk[3] = {a.x, a.y, a.z}, vk[3] = {b.x, b.y, b.z}, ga[3] = {c.x, c.y, c.z}, gj[3] = {c.w, d.x, d.y};
    const double mk = a.w, gs = b.w;
    // k as receiver: its cotangents factor out of the j-sums (see AdjTileSums)
    double s0 = 0.0, s1 = 0.0, A1[3] = {0, 0, 0}, B1[3] = {0, 0, 0}, C1[3] = {0, 0, 0};
    // m as receiver
    double v2[3] = {0, 0, 0}, u2[3] = {0, 0, 0}, d2 = 0.0;
    auto load_tile = [&](int buf, int64_t t) {
        const dvec4 *src = crec + t * (4 * TJ);
        for (int e = tid; e < 8 * TJ; e += BLOCK)
            cp_async16(reinterpret_cast<char *>(&sj[buf][0]) + 16 * e, reinterpret_cast<const char *>(src) + 16 * e);
        cp_async_commit();
    };
    if (t0 < t1) load_tile(0, t0);
    for (int64_t t = t0; t < t1; ++t) {
        const int buf = (int)((t - t0) & 1);
        if (t + 1 < t1) {
            load_tile(buf ^ 1, t + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        for (int jj = 0; jj < TJ; ++jj) {
            const dvec4 P0 = sj[buf][4 * jj], P1 = sj[buf][4 * jj + 1], P2 = sj[buf][4 * jj + 2],
                        P3 = sj[buf][4 * jj + 3];
            const double r[3] = {P0.x - xk[0], P0.y - xk[1], P0.z - xk[2]};
            const double w[3] = {P1.x - vk[0], P1.y - vk[1], P1.z - vk[2]};
            const double GAm[3] = {P2.x, P2.y, P2.z}, GJm[3] = {P2.w, P3.x, P3.y};
            const double Mm = P0.w, Sm = P1.w;
            const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
            const double rinv = r2 > 0.0 ? rsqrt(r2) : 0.0;
            const double rinv2 = rinv * rinv, rinv3 = rinv * rinv2;
            const double q = r[0] * w[0] + r[1] * w[1] + r[2] * w[2];
            const double b3 = -3.0 * rinv2;
            const double gamma = b3 * q;
            {  // k as receiver
                const double ar = ga[0] * r[0] + ga[1] * r[1] + ga[2] * r[2];
                const double jr = gj[0] * r[0] + gj[1] * r[1] + gj[2] * r[2];
                const double jw = gj[0] * w[0] + gj[1] * w[1] + gj[2] * w[2];
                const double beta = b3 * jr;
                const double alpha = b3 * (ar + jw - 5.0 * q * jr * rinv2) + gs;
                const double rm = rinv3 * Mm;
                s0 += rm;
                s1 += rm * gamma;
                const double ra = rm * alpha, rb = rm * beta;
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    A1[cc] += ra * r[cc];
                    B1[cc] += rb * w[cc];
                    C1[cc] += rb * r[cc];
                }
            }
            {  // m as receiver
                const double P = GAm[0] * r[0] + GAm[1] * r[1] + GAm[2] * r[2];
                const double Q = GJm[0] * r[0] + GJm[1] * r[1] + GJm[2] * r[2];
                const double R = GJm[0] * w[0] + GJm[1] * w[1] + GJm[2] * w[2];
                const double PR = P + R;
                const double b3Q = b3 * Q;
                const double nalpha = b3 * (PR - 5.0 * q * Q * rinv2) - Sm;
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    v2[cc] += rinv3 * (GAm[cc] + nalpha * r[cc] + b3Q * w[cc] + gamma * GJm[cc]);
                    u2[cc] += rinv3 * (GJm[cc] + b3Q * r[cc]);
                }
                d2 -= rinv3 * (PR + gamma * Q) + Sm * rinv;
            }
        }
        __syncthreads();
    }
    if (k < A.n) {
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            const double v1 = ga[cc] * s0 + gj[cc] * s1 + A1[cc] + B1[cc];
            const double u1 = gj[cc] * s0 + C1[cc];
            A.part[((int64_t)s * 7 + cc) * A.n + k] = mk * v2[cc] - v1;
            A.part[((int64_t)s * 7 + 3 + cc) * A.n + k] = mk * u2[cc] - u1;
        }
        A.part[((int64_t)s * 7 + 6) * A.n + k] = d2;
    }
}

// ---------------------------------------------------------------- FP64 passes
template <int BLOCK, int TJ>
__global__ void __launch_bounds__(BLOCK) k_adj_iside_f64(AdjArgs A)
{
    __shared__ dvec4 sj[2][2 * TJ];
    const int tid = threadIdx.x;
    const int64_t k = (int64_t)blockIdx.x * BLOCK + tid;
    const int s = blockIdx.y;
    const int64_t t0 = (A.n_tiles_j * s) / A.S, t1 = (A.n_tiles_j * (s + 1)) / A.S;
    const dvec4 *rec = static_cast<const dvec4 *>(A.rec);
    const dvec4 *irec = static_cast<const dvec4 *>(A.irec);
    const dvec4 a = irec[4 * k], b = irec[4 * k + 1], c = irec[4 * k + 2], d = irec[4 * k + 3];
    const double xi[3] = {a.x, a.y, a.z}, vi[3] = {b.x, b.y, b.z};
    const double ga[3] = {c.x, c.y, c.z}, gj[3] = {b.w, c.w, d.x};
    const double gs = a.w;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    auto load_tile = [&](int buf, int64_t t) {
        const dvec4 *src = rec + t * (2 * TJ);
        for (int e = tid; e < 4 * TJ; e += BLOCK)
            cp_async16(reinterpret_cast<char *>(&sj[buf][0]) + 16 * e, reinterpret_cast<const char *>(src) + 16 * e);
        cp_async_commit();
    };
    if (t0 < t1) load_tile(0, t0);
    for (int64_t t = t0; t < t1; ++t) {
        const int buf = (int)((t - t0) & 1);
        if (t + 1 < t1) {
            load_tile(buf ^ 1, t + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        for (int jj = 0; jj < TJ; ++jj) {
            const dvec4 p0 = sj[buf][2 * jj], p1 = sj[buf][2 * jj + 1];
            const double rx = p0.x - xi[0], ry = p0.y - xi[1], rz = p0.z - xi[2];
            const double r2 = rx * rx + ry * ry + rz * rz;
            const double rinv = r2 > 0.0 ? rsqrt(r2) : 0.0;
            double dm = 0.0;
            adj_pair<double, false>(rx, ry, rz, p1.x - vi[0], p1.y - vi[1], p1.z - vi[2], rinv, ga, gj, gs, p0.w, acc,
                                    acc + 3, dm);
        }
        __syncthreads();
    }
    if (k < A.n_i)
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) A.part[((int64_t)s * 6 + cc) * A.n_i + k] = acc[cc];
}

template <int BLOCK, int TI>
__global__ void __launch_bounds__(BLOCK) k_adj_jside_f64(AdjArgs A)
{
    __shared__ dvec4 si[2][4 * TI];
    const int tid = threadIdx.x;
    const int64_t j = (int64_t)blockIdx.x * BLOCK + tid;
    const int s = blockIdx.y;
    const int64_t t0 = (A.n_tiles_i * s) / A.S, t1 = (A.n_tiles_i * (s + 1)) / A.S;
    const dvec4 *rec = static_cast<const dvec4 *>(A.rec);
    const dvec4 *irec = static_cast<const dvec4 *>(A.irec);
    const dvec4 p0 = rec[2 * j], p1 = rec[2 * j + 1];
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    auto load_tile = [&](int buf, int64_t t) {
        const dvec4 *src = irec + t * (4 * TI);
        for (int e = tid; e < 8 * TI; e += BLOCK)
            cp_async16(reinterpret_cast<char *>(&si[buf][0]) + 16 * e, reinterpret_cast<const char *>(src) + 16 * e);
        cp_async_commit();
    };
    if (t0 < t1) load_tile(0, t0);
    for (int64_t t = t0; t < t1; ++t) {
        const int buf = (int)((t - t0) & 1);
        if (t + 1 < t1) {
            load_tile(buf ^ 1, t + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        for (int ii = 0; ii < TI; ++ii) {
            const dvec4 a = si[buf][4 * ii], b = si[buf][4 * ii + 1], c = si[buf][4 * ii + 2], d = si[buf][4 * ii + 3];
            const double ga[3] = {c.x, c.y, c.z}, gj[3] = {b.w, c.w, d.x};
            const double rx = p0.x - a.x, ry = p0.y - a.y, rz = p0.z - a.z;
            const double r2 = rx * rx + ry * ry + rz * rz;
            const double rinv = r2 > 0.0 ? rsqrt(r2) : 0.0;
            adj_pair<double, true>(rx, ry, rz, p1.x - b.x, p1.y - b.y, p1.z - b.z, rinv, ga, gj, a.w, 1.0, acc, acc + 3,
                                   acc[6]);
        }
        __syncthreads();
    }
    if (j < A.n)
#pragma unroll
        for (int c = 0; c < 7; ++c) A.part[((int64_t)s * 7 + c) * A.n + j] = c < 6 ? acc[c] * p0.w : acc[c];
}

// ---------------------------------------------------------------- combine
__global__ void k_adj_combine_j(const double *__restrict__ partB, int SB, int64_t n, double *__restrict__ g_x,
                                double *__restrict__ g_v, double *__restrict__ g_m)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double v[7];
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            double sum = 0.0;
            for (int s = 0; s < SB; ++s) sum += partB[((int64_t)s * 7 + c) * n + j];
            v[c] = sum;
        }
        g_x[3 * j] = v[0];
        g_x[3 * j + 1] = v[1];
        g_x[3 * j + 2] = v[2];
        g_v[3 * j] = v[3];
        g_v[3 * j + 1] = v[4];
        g_v[3 * j + 2] = v[5];
        g_m[j] = v[6];
    }
}

__global__ void k_adj_combine_i(const double *__restrict__ partA, int SA, int64_t n_i, const int32_t *__restrict__ idx,
                                int64_t n, double *__restrict__ g_x, double *__restrict__ g_v)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_i; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx[k];
        if (i < 0 || i >= n) continue;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            double sum = 0.0;
            for (int s = 0; s < SA; ++s) sum += partA[((int64_t)s * 6 + c) * n_i + k];
            double *dst = c < 3 ? g_x + 3 * i + c : g_v + 3 * i + (c - 3);
            atomicAdd(dst, -sum);
        }
    }
}

// ---------------------------------------------------------------- planning + launch
constexpr int kAdjNI = 4, kAdjNJ = 4, kAdjBlock = 128, kAdjTJ = 128, kAdjTI = 64;

size_t adjoint_scratch_bytes(int precision, int64_t n, int64_t n_i, int num_sms, int64_t *rows_pad_out, int *SA,
                             int *SB);

// The fused single pass does N x N pair work with ~96 FP32 operations (~81 in FP64), the two
// passes 2 x N_i x N with ~56 and ~60 (~63 each in FP64): the fused pass wins for dense blocks.
constexpr int kFusedBlock = 128, kFusedTJ = 128;     // mixed: one packed row pair a thread
constexpr int kFused64Block = 128, kFused64TJ = 64;  // FP64: one row a thread
static bool use_fused(int precision, int64_t n, int64_t n_i) { return 4 * n_i >= 3 * n; }

// Splits of the streamed dimension for ctas_x CTAs along the other one, P resident CTAs:
// the count with the least time in whole waves of the GPU, ceil(ctas_x S / P) / S, each
// split charged 0.05 % for its partial sums and their combine, and each keeping >= 2
// streamed tiles.
static int splits_for(int64_t ctas_x, int64_t tiles, int64_t P)
{
    const int64_t smax = tiles / 2 > 1 ? tiles / 2 : 1;
    if (ctas_x < 1) ctas_x = 1;
    int64_t S = 1;
    double best = 1e300;
    for (int64_t q = 1; q <= smax && q <= 64; ++q) {
        const double waves = (double)((ctas_x * q + P - 1) / P) / (double)q * (1.0 + 0.0005 * (double)q);
        if (waves < best * (1.0 - 1e-9)) {
            best = waves;
            S = q;
        }
    }
    return (int)S;
}

struct FusedGeom {
    int64_t n_pad, n_tiles, ctas;
    int S;
};

static FusedGeom fused_geom(int precision, int64_t n, int num_sms)
{
    FusedGeom f{};
    const int64_t sms = num_sms > 0 ? num_sms : 152;
    f.n_pad = ((n + 255) / 256) * 256;  // a multiple of both tile depths and of the row blocks
    if (precision == 1) {
        f.n_tiles = f.n_pad / kFusedTJ;
        f.ctas = (n + 2 * kFusedBlock - 1) / (2 * kFusedBlock);
        f.S = splits_for(f.ctas, f.n_tiles, sms * 3);  // 3 CTAs per SM
    } else {
        f.n_tiles = f.n_pad / kFused64TJ;
        f.ctas = (n + kFused64Block - 1) / kFused64Block;
        f.S = splits_for(f.ctas, f.n_tiles, sms * 4);  // 4 CTAs per SM
    }
    return f;
}

// Bytes of the fused pass's per-particle records.
static size_t fused_rec_bytes(int precision, int64_t n_pad) { return (size_t)n_pad * (precision == 1 ? 80 : 128); }

// Geometry shared by the scratch sizing and the launch.
struct AdjGeom {
    int ti_a, tj_a, tj_b, ti_b;  // i-side: i per CTA, j-tile; j-side: j per CTA, i-tile
    int64_t rows_pad, n_tiles_j, n_tiles_i, ctas_a, ctas_b;
    int SA, SB;
};

static AdjGeom adj_geom(int precision, int64_t n, int64_t n_i, int num_sms)
{
    AdjGeom g{};
    const int64_t P = (int64_t)(num_sms > 0 ? num_sms : 152) * 3;
    const int64_t n_pad = ((n + 255) / 256) * 256;
    if (precision == 1) {
        g.ti_a = kAdjNI * kAdjBlock; g.tj_a = kAdjTJ;   // i-side: packed, NI=4, BLOCK=128
        g.tj_b = kAdjNJ * kAdjBlock; g.ti_b = kAdjTI;   // j-side: packed, NJ=4, BLOCK=128
    } else {
        g.ti_a = 128; g.tj_a = 64;
        g.tj_b = 128; g.ti_b = 64;
    }
    const int64_t lcm_rows = (int64_t)(g.ti_a > g.ti_b ? g.ti_a : g.ti_b);
    g.rows_pad = ((n_i + lcm_rows - 1) / lcm_rows) * lcm_rows;
    if (g.rows_pad == 0) g.rows_pad = lcm_rows;
    g.n_tiles_j = n_pad / g.tj_a;
    g.n_tiles_i = g.rows_pad / g.ti_b;
    g.ctas_a = (n_i + g.ti_a - 1) / g.ti_a;
    g.ctas_b = (n + g.tj_b - 1) / g.tj_b;
    g.SA = splits_for(g.ctas_a, g.n_tiles_j, P);
    g.SB = splits_for(g.ctas_b, g.n_tiles_i, P);
    return g;
}

// Bytes of the pass scratch (records and partial sums); the duplicate check's n claim words
// follow at the next 256-byte boundary.
static size_t adjoint_core_bytes(int precision, int64_t n, int64_t n_i, int num_sms);
static size_t claim_offset(int precision, int64_t n, int64_t n_i, int num_sms)
{
    return (adjoint_core_bytes(precision, n, n_i, num_sms) + 255) & ~(size_t)255;
}

size_t adjoint_scratch_bytes(int precision, int64_t n, int64_t n_i, int num_sms, int64_t *rows_pad_out, int *SA,
                             int *SB)
{
    const AdjGeom g = adj_geom(precision, n, n_i, num_sms);
    *rows_pad_out = g.rows_pad;
    *SA = g.SA;
    *SB = g.SB;
    return claim_offset(precision, n, n_i, num_sms) + (size_t)n * sizeof(unsigned);
}

static size_t adjoint_core_bytes(int precision, int64_t n, int64_t n_i, int num_sms)
{
    const AdjGeom g = adj_geom(precision, n, n_i, num_sms);
    const size_t irec = (size_t)g.rows_pad * (precision == 1 ? 64 : 128);
    const size_t pa = (size_t)g.SA * 6 * (size_t)n_i * 8, pb = (size_t)g.SB * 7 * (size_t)n * 8;
    size_t need = irec + 256 + pa + 256 + pb;
    if (use_fused(precision, n, n_i)) {
        const FusedGeom f = fused_geom(precision, n, num_sms);
        size_t fb = fused_rec_bytes(precision, f.n_pad) + 256 + (size_t)f.S * 7 * (size_t)n * 8;
        if (precision == 1) fb = ((fb + 255) & ~(size_t)255) + roworder_scratch_bytes(n);  // row order
        if (fb > need) need = fb;
    }
    return need;
}

// Dynamic shared-memory limit of the anchored fused pass (just above the 48 KB default).
void adjoint_configure()
{
    cudaFuncSetAttribute((const void *)k_adj_fused_anchored_x2<kFusedBlock, kFusedTJ, 3>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, adj_anchored_smem<kFusedBlock, kFusedTJ>());
    cudaGetLastError();
}

int launch_adjoint(cudaStream_t st, int precision, const void *rec, int64_t n, const int32_t *idx, int64_t n_i,
                   const double *g_acc, const double *g_jerk, const double *g_pot, double *g_x, double *g_v,
                   double *g_m, void *scratch, unsigned *status, int num_sms)
{
    {
        unsigned *claim = reinterpret_cast<unsigned *>(static_cast<char *>(scratch) +
                                                       claim_offset(precision, n, n_i, num_sms));
        cudaMemsetAsync(claim, 0, (size_t)n * sizeof(unsigned), st);
        int64_t gq = (n_i + 255) / 256;
        if (gq > 152 * 8) gq = 152 * 8;
        if (gq < 1) gq = 1;
        k_check_unique<<<(unsigned)gq, 256, 0, st>>>(n, n_i, idx, claim, status);
    }
    if (use_fused(precision, n, n_i)) {  // dense block: one fused pass over all pairs
        const FusedGeom f = fused_geom(precision, n, num_sms);
        double *part = reinterpret_cast<double *>(static_cast<char *>(scratch) +
                                                  ((fused_rec_bytes(precision, f.n_pad) + 255) & ~(size_t)255));
        int64_t gr = (f.n_pad + 255) / 256;
        if (gr > 152 * 8) gr = 152 * 8;
        int64_t gq = (n_i + 255) / 256;
        if (gq > 152 * 8) gq = 152 * 8;
        if (gq < 1) gq = 1;
        AdjArgs A{};
        A.n = n;
        A.n_i = n_i;
        A.n_tiles_j = f.n_tiles;
        A.S = f.S;
        A.part = part;
        A.status = status;
        int order_kernels = 0;
        if (precision == 1) {
            float4 *crec = static_cast<float4 *>(scratch);
            k_build_crec<<<(unsigned)gr, 256, 0, st>>>(n, f.n_pad, static_cast<const float4 *>(rec), crec);
            k_scatter_cotangents<<<(unsigned)gq, 256, 0, st>>>(n, n_i, idx, g_acc, g_jerk, g_pot,
                                                               reinterpret_cast<float *>(crec), status);
            // every particle is a row: spatial order of all of them, then the anchored pass
            const size_t fb = fused_rec_bytes(precision, f.n_pad) + 256 + (size_t)f.S * 7 * (size_t)n * 8;
            void *ro = static_cast<char *>(scratch) + ((fb + 255) & ~(size_t)255);
            const int32_t *perm = nullptr;
            order_kernels = launch_row_order(st, rec, nullptr, n, n, ro, &perm);
            k_adj_fused_anchored_x2<kFusedBlock, kFusedTJ, 3>
                <<<dim3((unsigned)f.ctas, (unsigned)f.S), kFusedBlock, adj_anchored_smem<kFusedBlock, kFusedTJ>(),
                   st>>>(A, crec, perm);
        } else {
            dvec4 *crec = static_cast<dvec4 *>(scratch);
            k_build_crec64<<<(unsigned)gr, 256, 0, st>>>(n, f.n_pad, static_cast<const dvec4 *>(rec), crec);
            k_scatter_cotangents64<<<(unsigned)gq, 256, 0, st>>>(n, n_i, idx, g_acc, g_jerk, g_pot,
                                                                 reinterpret_cast<double *>(crec), status);
            k_adj_fused_f64<kFused64Block, kFused64TJ>
                <<<dim3((unsigned)f.ctas, (unsigned)f.S), kFused64Block, 0, st>>>(A, crec);
        }
        int64_t gj = (n + 255) / 256;
        if (gj > 152 * 16) gj = 152 * 16;
        k_adj_combine_j<<<(unsigned)gj, 256, 0, st>>>(part, f.S, n, g_x, g_v, g_m);
        return 5 + order_kernels;
    }
    const AdjGeom g = adj_geom(precision, n, n_i, num_sms);
    char *p = static_cast<char *>(scratch);
    const size_t irec_bytes = (size_t)g.rows_pad * (precision == 1 ? 64 : 128);
    void *irec = p;
    double *partA = reinterpret_cast<double *>(p + ((irec_bytes + 255) & ~(size_t)255));
    double *partB = partA + (((size_t)g.SA * 6 * (size_t)n_i + 31) & ~(size_t)31);
    AdjArgs A{};
    A.rec = rec;
    A.irec = irec;
    A.n = n;
    A.n_i = n_i;
    A.n_tiles_j = g.n_tiles_j;
    A.n_tiles_i = g.n_tiles_i;
    A.idx = idx;
    A.g_acc = g_acc;
    A.g_jerk = g_jerk;
    A.g_pot = g_pot;
    A.status = status;
    int kernels = 1;  // k_check_unique
    {
        int64_t gr = (g.rows_pad + 255) / 256;
        if (gr > 152 * 8) gr = 152 * 8;
        k_pack_irec<<<(unsigned)gr, 256, 0, st>>>(A, precision == 1, g.rows_pad);
        ++kernels;
    }
    if (n_i > 0) {
        A.S = g.SA;
        A.part = partA;
        if (precision == 1)
            k_adj_iside_x2<kAdjNI, kAdjBlock, kAdjTJ, 3>
                <<<dim3((unsigned)g.ctas_a, (unsigned)g.SA), kAdjBlock,
                   adj_iside_x2_smem<kAdjNI, kAdjBlock, kAdjTJ>(), st>>>(A);
        else
            k_adj_iside_f64<128, 64><<<dim3((unsigned)g.ctas_a, (unsigned)g.SA), 128, 0, st>>>(A);
        ++kernels;
    }
    A.S = g.SB;
    A.part = partB;
    if (precision == 1)
        k_adj_jside_x2<kAdjNJ, kAdjBlock, kAdjTI, 3>
            <<<dim3((unsigned)g.ctas_b, (unsigned)g.SB), kAdjBlock, adj_jside_x2_smem<kAdjNJ, kAdjBlock, kAdjTI>(),
               st>>>(A);
    else
        k_adj_jside_f64<128, 64><<<dim3((unsigned)g.ctas_b, (unsigned)g.SB), 128, 0, st>>>(A);
    ++kernels;
    int64_t gj = (n + 255) / 256;
    if (gj > 152 * 16) gj = 152 * 16;
    k_adj_combine_j<<<(unsigned)gj, 256, 0, st>>>(partB, g.SB, n, g_x, g_v, g_m);
    ++kernels;
    if (n_i > 0) {
        int64_t gi = (n_i + 255) / 256;
        if (gi > 152 * 16) gi = 152 * 16;
        k_adj_combine_i<<<(unsigned)gi, 256, 0, st>>>(partA, g.SA, n_i, idx, n, g_x, g_v);
        ++kernels;
    }
    return kernels;
}

}  // namespace nbgpu
