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

// ---------------------------------------------------------------- i-side pass, mixed
template <int NI, int BLOCK, int TJ>
__global__ void __launch_bounds__(BLOCK) k_adj_iside_mixed(AdjArgs A)
{
    __shared__ __align__(16) float4 sj[2][3 * TJ];
    const int tid = threadIdx.x;
    const int64_t kbase = (int64_t)blockIdx.x * (BLOCK * NI);
    const int s = blockIdx.y;
    const int64_t t0 = (A.n_tiles_j * s) / A.S, t1 = (A.n_tiles_j * (s + 1)) / A.S;
    const float4 *rec = static_cast<const float4 *>(A.rec);
    const float4 *irec = static_cast<const float4 *>(A.irec);
    float ih[NI][3], il[NI][3], iv[NI][3], ga[NI][3], gj[NI][3], gs[NI];
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int64_t k = kbase + q * BLOCK + tid;  // irec rows are padded: always readable
        const float4 a = irec[4 * k], b = irec[4 * k + 1], c = irec[4 * k + 2], d = irec[4 * k + 3];
        ih[q][0] = a.x; ih[q][1] = a.y; ih[q][2] = a.z; gs[q] = a.w;
        il[q][0] = b.x; il[q][1] = b.y; il[q][2] = b.z; gj[q][0] = b.w;
        iv[q][0] = c.x; iv[q][1] = c.y; iv[q][2] = c.z; gj[q][1] = c.w;
        ga[q][0] = d.x; ga[q][1] = d.y; ga[q][2] = d.z; gj[q][2] = d.w;
    }
    double dacc[NI][6];
#pragma unroll
    for (int q = 0; q < NI; ++q)
#pragma unroll
        for (int c = 0; c < 6; ++c) dacc[q][c] = 0.0;
    auto load_tile = [&](int buf, int64_t t) {
        const float4 *src = rec + t * (3 * TJ);
#pragma unroll
        for (int e = tid; e < 3 * TJ; e += BLOCK) cp_async16(&sj[buf][e], src + e);
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
        float acc[NI][6];
#pragma unroll
        for (int q = 0; q < NI; ++q)
#pragma unroll
            for (int c = 0; c < 6; ++c) acc[q][c] = 0.f;
#pragma unroll 2
        for (int jj = 0; jj < TJ; ++jj) {
            const float4 p0 = sj[buf][3 * jj], p1 = sj[buf][3 * jj + 1], p2 = sj[buf][3 * jj + 2];
#pragma unroll
            for (int q = 0; q < NI; ++q) {
                const float rx = ds_diff(p0.x, p1.x, ih[q][0], il[q][0]);
                const float ry = ds_diff(p0.y, p1.y, ih[q][1], il[q][1]);
                const float rz = ds_diff(p0.z, p1.z, ih[q][2], il[q][2]);
                const float r2 = r2_f32(rx, ry, rz);
                const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
                float dm = 0.f;
                adj_pair<float, false>(rx, ry, rz, p2.x - iv[q][0], p2.y - iv[q][1], p2.z - iv[q][2], rinv, ga[q],
                                       gj[q], gs[q], p0.w, acc[q], acc[q] + 3, dm);
            }
        }
#pragma unroll
        for (int q = 0; q < NI; ++q)
#pragma unroll
            for (int c = 0; c < 6; ++c) dacc[q][c] += (double)acc[q][c];
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int64_t k = kbase + q * BLOCK + tid;
        if (k < A.n_i)
#pragma unroll
            for (int c = 0; c < 6; ++c) A.part[((int64_t)s * 6 + c) * A.n_i + k] = dacc[q][c];
    }
}

// ---------------------------------------------------------------- j-side pass, mixed
template <int NJ, int BLOCK, int TI>
__global__ void __launch_bounds__(BLOCK) k_adj_jside_mixed(AdjArgs A)
{
    __shared__ __align__(16) float4 si[2][4 * TI];
    const int tid = threadIdx.x;
    const int64_t jbase = (int64_t)blockIdx.x * (BLOCK * NJ);
    const int s = blockIdx.y;
    const int64_t t0 = (A.n_tiles_i * s) / A.S, t1 = (A.n_tiles_i * (s + 1)) / A.S;
    const float4 *rec = static_cast<const float4 *>(A.rec);
    const float4 *irec = static_cast<const float4 *>(A.irec);
    float jh[NJ][3], jl[NJ][3], jv[NJ][3], jm[NJ];
#pragma unroll
    for (int q = 0; q < NJ; ++q) {
        const int64_t j = jbase + q * BLOCK + tid;  // rec is padded to the tile multiple
        const float4 a = rec[3 * j], b = rec[3 * j + 1], c = rec[3 * j + 2];
        jh[q][0] = a.x; jh[q][1] = a.y; jh[q][2] = a.z; jm[q] = a.w;
        jl[q][0] = b.x; jl[q][1] = b.y; jl[q][2] = b.z;
        jv[q][0] = c.x; jv[q][1] = c.y; jv[q][2] = c.z;
    }
    double dacc[NJ][7];
#pragma unroll
    for (int q = 0; q < NJ; ++q)
#pragma unroll
        for (int c = 0; c < 7; ++c) dacc[q][c] = 0.0;
    auto load_tile = [&](int buf, int64_t t) {
        const float4 *src = irec + t * (4 * TI);
#pragma unroll
        for (int e = tid; e < 4 * TI; e += BLOCK) cp_async16(&si[buf][e], src + e);
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
        float acc[NJ][7];
#pragma unroll
        for (int q = 0; q < NJ; ++q)
#pragma unroll
            for (int c = 0; c < 7; ++c) acc[q][c] = 0.f;
#pragma unroll 2
        for (int ii = 0; ii < TI; ++ii) {
            const float4 a = si[buf][4 * ii], b = si[buf][4 * ii + 1], c = si[buf][4 * ii + 2],
                         d = si[buf][4 * ii + 3];
            const float ga[3] = {d.x, d.y, d.z}, gj[3] = {b.w, c.w, d.w};
#pragma unroll
            for (int q = 0; q < NJ; ++q) {
                const float rx = ds_diff(jh[q][0], jl[q][0], a.x, b.x);
                const float ry = ds_diff(jh[q][1], jl[q][1], a.y, b.y);
                const float rz = ds_diff(jh[q][2], jl[q][2], a.z, b.z);
                const float r2 = r2_f32(rx, ry, rz);
                const float rinv = r2 > 0.f ? rsqrtf(r2) : 0.f;
                adj_pair<float, true>(rx, ry, rz, jv[q][0] - c.x, jv[q][1] - c.y, jv[q][2] - c.z, rinv, ga, gj, a.w,
                                      1.f, acc[q], acc[q] + 3, acc[q][6]);
            }
        }
#pragma unroll
        for (int q = 0; q < NJ; ++q)
#pragma unroll
            for (int c = 0; c < 7; ++c) dacc[q][c] += (double)acc[q][c];
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < NJ; ++q) {
        const int64_t j = jbase + q * BLOCK + tid;
        if (j < A.n)
#pragma unroll
            for (int c = 0; c < 7; ++c)
                A.part[((int64_t)s * 7 + c) * A.n + j] = c < 6 ? dacc[q][c] * (double)jm[q] : dacc[q][c];
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
static int splits_for(int64_t ctas_x, int64_t tiles, int64_t P)
{
    // enough CTAs for ~4 waves, each split keeping >= 2 streamed tiles
    int64_t S = (4 * P + ctas_x - 1) / (ctas_x > 0 ? ctas_x : 1);
    const int64_t smax = tiles / 2 > 1 ? tiles / 2 : 1;
    if (S > smax) S = smax;
    if (S < 1) S = 1;
    return (int)S;
}

size_t adjoint_scratch_bytes(int precision, int64_t n, int64_t n_i, int num_sms, int64_t *rows_pad_out, int *SA,
                             int *SB);

// Geometry shared by the scratch sizing and the launch.
struct AdjGeom {
    int ti_a, tj_a, tj_b, ti_b;  // i-side: i per CTA, j-tile; j-side: j per CTA, i-tile
    int64_t rows_pad, n_tiles_j, n_tiles_i, ctas_a, ctas_b;
    int SA, SB;
};

static AdjGeom adj_geom(int precision, int64_t n, int64_t n_i, int num_sms)
{
    AdjGeom g{};
    const int64_t P = (int64_t)(num_sms > 0 ? num_sms : 152) * 2;
    const int64_t n_pad = ((n + 255) / 256) * 256;
    if (precision == 1) {
        g.ti_a = 2 * 128; g.tj_a = 256;   // i-side: NI=2, BLOCK=128
        g.tj_b = 2 * 128; g.ti_b = 128;   // j-side: NJ=2, BLOCK=128, i-tile 128
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

size_t adjoint_scratch_bytes(int precision, int64_t n, int64_t n_i, int num_sms, int64_t *rows_pad_out, int *SA,
                             int *SB)
{
    const AdjGeom g = adj_geom(precision, n, n_i, num_sms);
    *rows_pad_out = g.rows_pad;
    *SA = g.SA;
    *SB = g.SB;
    const size_t irec = (size_t)g.rows_pad * (precision == 1 ? 64 : 128);
    const size_t pa = (size_t)g.SA * 6 * (size_t)n_i * 8, pb = (size_t)g.SB * 7 * (size_t)n * 8;
    return irec + 256 + pa + 256 + pb;
}

int launch_adjoint(cudaStream_t st, int precision, const void *rec, int64_t n, const int32_t *idx, int64_t n_i,
                   const double *g_acc, const double *g_jerk, const double *g_pot, double *g_x, double *g_v,
                   double *g_m, void *scratch, unsigned *status, int num_sms)
{
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
    int kernels = 0;
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
            k_adj_iside_mixed<2, 128, 256><<<dim3((unsigned)g.ctas_a, (unsigned)g.SA), 128, 0, st>>>(A);
        else
            k_adj_iside_f64<128, 64><<<dim3((unsigned)g.ctas_a, (unsigned)g.SA), 128, 0, st>>>(A);
        ++kernels;
    }
    A.S = g.SB;
    A.part = partB;
    if (precision == 1)
        k_adj_jside_mixed<2, 128, 128><<<dim3((unsigned)g.ctas_b, (unsigned)g.SB), 128, 0, st>>>(A);
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
