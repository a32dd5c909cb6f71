// force_mixed.cu — K3: regular force, jerk, potential and neighbour capture in mixed
// precision (paper Sec. 3.2.1: the regular force and neighbour list on the GPU).
//
// Precision scheme: positions arrive as FP64 split into hi/lo floats; the coordinate
// difference is formed in double-single ((hi - hi) + (lo - lo)), every other pairwise
// operation runs in FP32 on the CUDA cores (one MUFU rsqrt per pair), per-i sums are
// accumulated in FP32 over one j-tile, or two in the packed variants other than the
// four-row one at 3 CTAs per SM (128 to 512 j), and promoted to FP64 after it.
// Not a dense contraction, so no tensor cores.
//
// Kernels:
//  * tiled (scalar) : CTA = NI*BLOCK active particles (NI per thread, register-blocked) x
//                     one j-range; j-tiles of TJ records are staged in shared memory with
//                     cp.async (double-buffered) and broadcast to all threads.
//  * tiled (packed) : the same decomposition with two rows in every FP32x2 operation and a
//                     duplicated j-tile layout (k_force_mixed_tiled_x2; the default for
//                     blocks of more than a few dozen rows).  FMA-pipe bound.
//  * j-streamed     : for tiny active blocks.  CTA = IB active particles x one j-chunk;
//                     every warp streams its own contiguous sub-chunk (coalesced) and the
//                     block reduces the IB x 7 partial sums with warp shuffles.  HBM /
//                     latency bound.  One row a CTA in scalar form; two, four or eight rows
//                     as row pairs in FP32x2 operations (k_force_mixed_jstream_x2).
//  * batched        : many independent clusters in one persistent launch (a work queue of
//                     cost-sorted items), the packed inner loop.
// The per-call kernels write FP64 partial sums [split][7][n_i] that k_reduce adds in a fixed
// order, so results are bitwise reproducible for a given launch plan.  Neighbour segments:
// one per split (tiled, owned by the thread holding the row) or one per warp (j-streamed,
// ordered within the warp by ballot).
#include "nb_common.cuh"
#include "nb_kernels.cuh"

namespace nbgpu {

// One pair (i <- j) in mixed precision; returns r^2 for the neighbour test.
// acc[0..2] += m r/|r|^3 ; acc[3..5] += m (w - 3 (r.w) r/|r|^2)/|r|^3 ; acc[6] += m/|r|
template <bool MASK>
__device__ __forceinline__ float pair_mixed(float jxh, float jyh, float jzh, float jm, float jxl,
                                            float jyl, float jzl, float jvx, float jvy, float jvz,
                                            float ixh, float iyh, float izh, float ixl, float iyl,
                                            float izl, float ivx, float ivy, float ivz, bool self,
                                            float *acc)
{
    const float dx = ds_diff(jxh, jxl, ixh, ixl);
    const float dy = ds_diff(jyh, jyl, iyh, iyl);
    const float dz = ds_diff(jzh, jzl, izh, izl);
    const float r2 = r2_f32(dx, dy, dz);
    float rinv = rsqrtf(r2);
    if (MASK) rinv = self ? 0.f : rinv;
    const float wx = jvx - ivx, wy = jvy - ivy, wz = jvz - ivz;
    const float rw = dx * wx + dy * wy + dz * wz;
    const float rinv2 = rinv * rinv;
    const float mr = jm * rinv;
    const float mr3 = mr * rinv2;
    const float beta = rw * (rinv2 * -3.f);
    acc[0] += mr3 * dx;
    acc[1] += mr3 * dy;
    acc[2] += mr3 * dz;
    acc[3] += mr3 * (wx + beta * dx);
    acc[4] += mr3 * (wy + beta * dy);
    acc[5] += mr3 * (wz + beta * dz);
    acc[6] += mr;
    return r2;
}

template <int NI, bool MASK, int TJ>
__device__ __forceinline__ void tile_mixed(const float4 *__restrict__ sj, int64_t jb, const ForceArgs &A,
                                           const float (&ih)[NI][3], const float (&il)[NI][3],
                                           const float (&iv)[NI][3], const float (&rs2f)[NI],
                                           const int64_t (&gi)[NI], int32_t *const (&slot)[NI],
                                           int (&cnt)[NI], float (&acc)[NI][7])
{
#pragma unroll 4
    for (int jj = 0; jj < TJ; ++jj) {
        const float4 p0 = sj[3 * jj], p1 = sj[3 * jj + 1], p2 = sj[3 * jj + 2];
        const int64_t j = jb + jj;
        float r2[NI];
        bool hit = false;
#pragma unroll
        for (int q = 0; q < NI; ++q) {
            r2[q] = pair_mixed<MASK>(p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p2.x, p2.y, p2.z,
                                     ih[q][0], ih[q][1], ih[q][2], il[q][0], il[q][1], il[q][2],
                                     iv[q][0], iv[q][1], iv[q][2], MASK && (j == gi[q]), acc[q]);
            hit |= r2[q] < rs2f[q];
        }
        if (hit) {  // rare: record in ascending j, the first L per segment
#pragma unroll
            for (int q = 0; q < NI; ++q)
                if (r2[q] < rs2f[q] && j != gi[q] && j < A.j_hi) {
                    if (cnt[q] < A.L) slot[q][cnt[q]] = (int32_t)j;
                    ++cnt[q];
                }
        }
    }
}

template <int NI, int BLOCK, int TJ, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_force_mixed_tiled(ForceArgs A)
{
    __shared__ __align__(16) float4 sj[2][3 * TJ];
    const int tid = threadIdx.x;
    const int64_t kbase = (int64_t)blockIdx.x * (BLOCK * NI);
    const int s = blockIdx.y;
    const int64_t tb = A.j_lo / TJ;  // first tile of the source range
    const int64_t t0 = tb + (A.n_tiles * s) / A.S, t1 = tb + (A.n_tiles * (s + 1)) / A.S;
    const float4 *rec = static_cast<const float4 *>(A.rec);

    float ih[NI][3], il[NI][3], iv[NI][3], rs2f[NI];
    int64_t gi[NI];
    int32_t *slot[NI];
    int cnt[NI];
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int64_t k = kbase + q * BLOCK + tid;
        int64_t g = -1;
        if (k < A.n_i) {
            g = A.idx[k];
            if (g < 0 || g >= A.n) {
                if (s == 0) atomicOr(A.status, ST_BAD_INDEX);
                g = -1;
            }
        }
        gi[q] = g;
        cnt[q] = 0;
        slot[q] = A.seg_slots + ((int64_t)s * A.n_i + (k < A.n_i ? k : 0)) * A.L;
        if (g >= 0) {
            const float4 p0 = rec[3 * g], p1 = rec[3 * g + 1], p2 = rec[3 * g + 2];
            ih[q][0] = p0.x; ih[q][1] = p0.y; ih[q][2] = p0.z;
            il[q][0] = p1.x; il[q][1] = p1.y; il[q][2] = p1.z;
            iv[q][0] = p2.x; iv[q][1] = p2.y; iv[q][2] = p2.z;
            rs2f[q] = A.want_nb ? __double2float_rn(A.rs2[A.rs2_scalar ? 0 : k]) : -1.f;
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) ih[q][c] = il[q][c] = iv[q][c] = 0.f;
            rs2f[q] = -1.f;
        }
    }
    double dacc[NI][7];
#pragma unroll
    for (int q = 0; q < NI; ++q)
#pragma unroll
        for (int c = 0; c < 7; ++c) dacc[q][c] = 0.0;

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
        const int64_t jb = t * TJ;
        bool mine = false;
#pragma unroll
        for (int q = 0; q < NI; ++q) mine |= (gi[q] >= jb && gi[q] < jb + TJ);
        float acc[NI][7];
#pragma unroll
        for (int q = 0; q < NI; ++q)
#pragma unroll
            for (int c = 0; c < 7; ++c) acc[q][c] = 0.f;
        if (__any_sync(0xffffffffu, mine))
            tile_mixed<NI, true, TJ>(sj[buf], jb, A, ih, il, iv, rs2f, gi, slot, cnt, acc);
        else
            tile_mixed<NI, false, TJ>(sj[buf], jb, A, ih, il, iv, rs2f, gi, slot, cnt, acc);
#pragma unroll
        for (int q = 0; q < NI; ++q)
#pragma unroll
            for (int c = 0; c < 7; ++c) dacc[q][c] += (double)acc[q][c];
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int64_t k = kbase + q * BLOCK + tid;
        if (k < A.n_i) {
#pragma unroll
            for (int c = 0; c < 7; ++c)
                A.part[((int64_t)s * 7 + c) * A.n_i + k] = (c == 6) ? -dacc[q][c] : dacc[q][c];
            if (A.want_nb) A.seg_cnt[(int64_t)s * A.n_i + k] = cnt[q];
        }
    }
}

// j-streamed kernel for small active blocks: blockIdx.x = batch of IB active particles,
// blockIdx.y = j-chunk [j0, j1).  Warp w of the CTA walks the contiguous sub-chunk w of
// the chunk, 32 consecutive j per step, so its neighbour segment (g = s*W + w) is built
// in ascending j by ballot.
template <int IB, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_force_mixed_jstream(ForceArgs A)
{
    constexpr int W = BLOCK / 32;
    __shared__ double red[W][IB][7];
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int s = blockIdx.y;
    const int64_t k0 = (int64_t)blockIdx.x * IB;
    const int64_t j0 = A.j_lo + ((A.j_hi - A.j_lo) * s) / A.S, j1 = A.j_lo + ((A.j_hi - A.j_lo) * (s + 1)) / A.S;
    const int64_t w0 = j0 + ((j1 - j0) * w) / W, w1 = j0 + ((j1 - j0) * (w + 1)) / W;
    const int64_t g = (int64_t)s * W + w;
    const float4 *rec = static_cast<const float4 *>(A.rec);

    float ih[IB][3], il[IB][3], iv[IB][3], rs2f[IB];
    int64_t gi[IB];
    int cnt[IB];
#pragma unroll
    for (int q = 0; q < IB; ++q) {
        const int64_t k = k0 + q;
        int64_t gg = -1;
        if (k < A.n_i) {
            gg = A.idx[k];
            if (gg < 0 || gg >= A.n) {
                if (s == 0 && tid == 0) atomicOr(A.status, ST_BAD_INDEX);
                gg = -1;
            }
        }
        gi[q] = gg;
        cnt[q] = 0;
        if (gg >= 0) {
            const float4 p0 = rec[3 * gg], p1 = rec[3 * gg + 1], p2 = rec[3 * gg + 2];
            ih[q][0] = p0.x; ih[q][1] = p0.y; ih[q][2] = p0.z;
            il[q][0] = p1.x; il[q][1] = p1.y; il[q][2] = p1.z;
            iv[q][0] = p2.x; iv[q][1] = p2.y; iv[q][2] = p2.z;
            rs2f[q] = A.want_nb ? __double2float_rn(A.rs2[A.rs2_scalar ? 0 : k]) : -1.f;
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) ih[q][c] = il[q][c] = iv[q][c] = 0.f;
            rs2f[q] = -1.f;
        }
    }
    float acc[IB][7];
#pragma unroll
    for (int q = 0; q < IB; ++q)
#pragma unroll
        for (int c = 0; c < 7; ++c) acc[q][c] = 0.f;

    const unsigned below = (1u << lane) - 1u;
    for (int64_t base = w0; base < w1; base += 32) {  // warp-uniform trip count
        const int64_t j = base + lane;
        const bool valid = j < w1;
        float4 p0 = make_float4(kPadPos, kPadPos, kPadPos, 0.f), p1 = make_float4(0.f, 0.f, 0.f, 0.f), p2 = p1;
        if (valid) {
            p0 = __ldg(rec + 3 * j);
            p1 = __ldg(rec + 3 * j + 1);
            p2 = __ldg(rec + 3 * j + 2);
        }
#pragma unroll
        for (int q = 0; q < IB; ++q) {
            const float r2 = pair_mixed<true>(p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p2.x, p2.y, p2.z, ih[q][0],
                                              ih[q][1], ih[q][2], il[q][0], il[q][1], il[q][2], iv[q][0], iv[q][1],
                                              iv[q][2], j == gi[q], acc[q]);
            const bool hit = valid && r2 < rs2f[q] && j != gi[q];
            const unsigned mask = __ballot_sync(0xffffffffu, hit);
            if (mask) {
                const int pos = cnt[q] + __popc(mask & below);
                if (hit && pos < A.L) A.seg_slots[(g * A.n_i + k0 + q) * A.L + pos] = (int32_t)j;
                cnt[q] += __popc(mask);
            }
        }
    }
    if (A.want_nb && lane == 0) {
#pragma unroll
        for (int q = 0; q < IB; ++q)
            if (k0 + q < A.n_i) A.seg_cnt[g * A.n_i + k0 + q] = cnt[q];
    }
    // block reduction: warp shuffles, then one FP64 slot per warp, summed in warp order
#pragma unroll
    for (int q = 0; q < IB; ++q)
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            const float v = warp_sum(acc[q][c]);
            if (lane == 0) red[w][q][c] = (double)v;
        }
    __syncthreads();
    for (int e = tid; e < IB * 7; e += BLOCK) {
        const int q = e / 7, c = e % 7;
        const int64_t k = k0 + q;
        if (k < A.n_i) {
            double sum = 0.0;
#pragma unroll
            for (int ww = 0; ww < W; ++ww) sum += red[ww][q][c];
            A.part[((int64_t)s * 7 + c) * A.n_i + k] = (c == 6) ? -sum : sum;
        }
    }
}

// ------------------------------------------------------------------------------------------
// Packed-FP32x2 tiled kernel.  Each thread holds NI active rows as NI/2 row pairs; every
// FP32 operation of a pair interaction is one __ffma2_rn / __fadd2_rn / __fmul2_rn acting on
// both rows of a pair against the same j (half the FP32 instructions of the scalar kernel).
// The j-tile is copied raw (cp.async, double-buffered) and expanded once per tile into a
// duplicated layout, five float4 per j:
//   {xh,xh,yh,yh} {zh,zh,m,m} {xl,xl,yl,yl} {zl,zl,vx,vx} {vy,vy,vz,vz}
// so that each 16-byte shared load yields two broadcast pairs.  The arithmetic and its
// rounding order are those of pair_mixed (x - y is computed as x + (-y), which IEEE
// rounds identically), so neighbour decisions are bit-identical to the scalar kernel.
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// r^2 of two rows against one j of the duplicated tile, in the rounding order of pair_mixed;
// the neighbour pass recomputes it with this same function, so its decisions are those the
// interaction loop saw.
__device__ __forceinline__ float2 x2_r2(const float4 &a, const float4 &b, const float4 &c, const float4 &d,
                                        const float2 (&h)[3], const float2 (&l)[3], float2 &dx, float2 &dy,
                                        float2 &dz)
{
    dx = f2add(f2add(make_float2(a.x, a.y), h[0]), f2add(make_float2(c.x, c.y), l[0]));
    dy = f2add(f2add(make_float2(a.z, a.w), h[1]), f2add(make_float2(c.z, c.w), l[1]));
    dz = f2add(f2add(make_float2(b.x, b.y), h[2]), f2add(make_float2(d.x, d.y), l[2]));
    return f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx)));
}

// The interaction loop only sets bit u of a 32-bit mask when j = jb + u lies inside r_s of
// any of the thread's rows; the rare hits are recorded after each 32-j chunk, in ascending j,
// so that the loop body has no branch and the compiler can interleave consecutive j.
template <int NP>
__device__ __forceinline__ void x2_record_hits(const float4 *__restrict__ sd, int64_t jb, unsigned hm, int64_t jend,
                                            int L, const float2 (&nh)[NP][3], const float2 (&nl)[NP][3],
                                            const float2 (&rs2f)[NP], const int32_t (&gi)[NP][2],
                                            int32_t *slot0, int64_t sstride, int (&cnt)[NP][2])
{
    while (hm) {
        const int u = __ffs(hm) - 1;
        hm &= hm - 1;
        const int64_t j = jb + u;
        const int32_t j32 = (int32_t)j;
        const float4 a = sd[5 * u], b = sd[5 * u + 1], c = sd[5 * u + 2], d = sd[5 * u + 3];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            float2 dx, dy, dz;
            const float2 r2 = x2_r2(a, b, c, d, nh[q], nl[q], dx, dy, dz);
            if (r2.x < rs2f[q].x && j32 != gi[q][0] && j < jend) {
                if (cnt[q][0] < L) slot0[(2 * q) * sstride + cnt[q][0]] = j32;
                ++cnt[q][0];
            }
            if (r2.y < rs2f[q].y && j32 != gi[q][1] && j < jend) {
                if (cnt[q][1] < L) slot0[(2 * q + 1) * sstride + cnt[q][1]] = j32;
                ++cnt[q][1];
            }
        }
    }
}

template <int NP, bool MASK, int TJ, int UJ>
__device__ __forceinline__ void tile_mixed_x2(const float4 *__restrict__ sd, int64_t jb, int64_t jend, int L,
                                              const float2 (&nh)[NP][3], const float2 (&nl)[NP][3],
                                              const float2 (&nv)[NP][3], const float2 (&rs2f)[NP],
                                              const int32_t (&gi)[NP][2], int32_t *slot0, int64_t sstride,
                                              int (&cnt)[NP][2], float2 (&acc)[NP][7])
{
    static_assert(TJ % 32 == 0, "tiles are whole 32-j chunks");
    const float2 m3 = make_float2(-3.f, -3.f);
    for (int jc = 0; jc < TJ; jc += 32) {
        const float4 *sc = sd + 5 * jc;
        unsigned hm = 0;
#pragma unroll UJ
        for (int u = 0; u < 32; ++u) {
            const float4 a = sc[5 * u], b = sc[5 * u + 1], c = sc[5 * u + 2], d = sc[5 * u + 3], e = sc[5 * u + 4];
            const float2 M = make_float2(b.z, b.w), VX = make_float2(d.z, d.w), VY = make_float2(e.x, e.y);
            const float2 VZ = make_float2(e.z, e.w);
            bool hit = false;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                float2 dx, dy, dz;
                const float2 r2 = x2_r2(a, b, c, d, nh[q], nl[q], dx, dy, dz);
                float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                if (MASK) {
                    const int32_t j = (int32_t)(jb + jc + u);
                    rinv.x = (j == gi[q][0]) ? 0.f : rinv.x;
                    rinv.y = (j == gi[q][1]) ? 0.f : rinv.y;
                }
                const float2 wx = f2add(VX, nv[q][0]), wy = f2add(VY, nv[q][1]), wz = f2add(VZ, nv[q][2]);
                const float2 rw = f2fma(dz, wz, f2fma(dy, wy, f2mul(dx, wx)));
                const float2 rinv2 = f2mul(rinv, rinv);
                const float2 mr = f2mul(M, rinv);
                const float2 mr3 = f2mul(mr, rinv2);
                const float2 beta = f2mul(rw, f2mul(rinv2, m3));
                acc[q][0] = f2fma(mr3, dx, acc[q][0]);
                acc[q][1] = f2fma(mr3, dy, acc[q][1]);
                acc[q][2] = f2fma(mr3, dz, acc[q][2]);
                acc[q][3] = f2fma(mr3, f2fma(beta, dx, wx), acc[q][3]);
                acc[q][4] = f2fma(mr3, f2fma(beta, dy, wy), acc[q][4]);
                acc[q][5] = f2fma(mr3, f2fma(beta, dz, wz), acc[q][5]);
                acc[q][6] = f2add(acc[q][6], mr);
                hit |= (r2.x < rs2f[q].x) | (r2.y < rs2f[q].y);
            }
            hm |= (unsigned)hit << u;
        }
        if (hm) x2_record_hits<NP>(sc, jb + jc, hm, jend, L, nh, nl, rs2f, gi, slot0, sstride, cnt);
    }
}

// Packed j-streamed kernel for small active blocks (IB = 2, 4 or 8 rows a CTA).  The
// decomposition is that of k_force_mixed_jstream: warp w walks the contiguous sub-chunk w of
// the CTA's j-chunk, 32 consecutive j a round, one j a lane, and its neighbour segment
// (g = s*W + w) is built in ascending j by ballot.  Every lane holds the IB rows as IB/2 row
// pairs, so that each FP32x2 operation of the pair interaction updates two rows against the
// lane's j (the operations and their order are those of tile_mixed_x2; r^2 is bit-identical
// to pair_mixed's, so the neighbour decisions are the scalar kernel's).  The self-pair mask
// is applied only in the one round of a warp that holds a row's own index, and the per-row
// ballots run only in rounds where some lane has a hit, when that lane's r^2 is recomputed
// with the same operations.
// One round of the packed j-streamed kernel: the lane's j in the duplicated layout of the
// tiled kernel ({xh,xh,yh,yh} {zh,zh,m,m} {xl,xl,yl,yl} {zl,zl,vx,vx}, and vy, vz) against
// its NP row pairs; returns whether any of the rows has j inside its r_s.
template <int NP, bool MASK>
__device__ __forceinline__ bool js_round_x2(const float4 &a, const float4 &b, const float4 &c, const float4 &d,
                                            float2 VY, float2 VZ, int32_t j32, const float2 (&nh)[NP][3],
                                            const float2 (&nl)[NP][3], const float2 (&nv)[NP][3],
                                            const float2 (&rs2f)[NP], const int32_t (&gi)[NP][2],
                                            float2 (&acc)[NP][7])
{
    const float2 M = make_float2(b.z, b.w), VX = make_float2(d.z, d.w);
    const float2 m3 = make_float2(-3.f, -3.f);
    bool hit = false;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        float2 dx, dy, dz;
        const float2 r2 = x2_r2(a, b, c, d, nh[q], nl[q], dx, dy, dz);
        float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
        if (MASK) {
            rinv.x = (j32 == gi[q][0]) ? 0.f : rinv.x;
            rinv.y = (j32 == gi[q][1]) ? 0.f : rinv.y;
        }
        const float2 wx = f2add(VX, nv[q][0]), wy = f2add(VY, nv[q][1]), wz = f2add(VZ, nv[q][2]);
        const float2 rw = f2fma(dz, wz, f2fma(dy, wy, f2mul(dx, wx)));
        const float2 rinv2 = f2mul(rinv, rinv);
        const float2 mr = f2mul(M, rinv);
        const float2 mr3 = f2mul(mr, rinv2);
        const float2 beta = f2mul(rw, f2mul(rinv2, m3));
        acc[q][0] = f2fma(mr3, dx, acc[q][0]);
        acc[q][1] = f2fma(mr3, dy, acc[q][1]);
        acc[q][2] = f2fma(mr3, dz, acc[q][2]);
        acc[q][3] = f2fma(mr3, f2fma(beta, dx, wx), acc[q][3]);
        acc[q][4] = f2fma(mr3, f2fma(beta, dy, wy), acc[q][4]);
        acc[q][5] = f2fma(mr3, f2fma(beta, dz, wz), acc[q][5]);
        acc[q][6] = f2add(acc[q][6], mr);
        hit |= (r2.x < rs2f[q].x) | (r2.y < rs2f[q].y);
    }
    return hit;
}

template <int IB, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_force_mixed_jstream_x2(ForceArgs A)
{
    static_assert(IB % 2 == 0, "rows come in pairs");
    constexpr int W = BLOCK / 32, NP = IB / 2;
    __shared__ double red[W][IB][7];
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int s = blockIdx.y;
    const int64_t k0 = (int64_t)blockIdx.x * IB;
    const int64_t j0 = A.j_lo + ((A.j_hi - A.j_lo) * s) / A.S, j1 = A.j_lo + ((A.j_hi - A.j_lo) * (s + 1)) / A.S;
    const int64_t w0 = j0 + ((j1 - j0) * w) / W, w1 = j0 + ((j1 - j0) * (w + 1)) / W;
    const int64_t g = (int64_t)s * W + w;
    const float4 *rec = static_cast<const float4 *>(A.rec);

    // the rows, negated (x - y is computed as x + (-y), which IEEE rounds identically)
    float2 nh[NP][3], nl[NP][3], nv[NP][3], rs2f[NP];
    int32_t gi[NP][2];
    int cnt[IB];
#pragma unroll
    for (int q = 0; q < IB; ++q) {
        const int64_t k = k0 + q;
        int64_t gg = -1;
        if (k < A.n_i) {
            gg = A.idx[k];
            if (gg < 0 || gg >= A.n) {
                if (s == 0 && tid == 0) atomicOr(A.status, ST_BAD_INDEX);
                gg = -1;
            }
        }
        float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f}, v[3] = {0.f, 0.f, 0.f}, r = -1.f;
        if (gg >= 0) {
            const float4 p0 = rec[3 * gg], p1 = rec[3 * gg + 1], p2 = rec[3 * gg + 2];
            h[0] = -p0.x; h[1] = -p0.y; h[2] = -p0.z;
            l[0] = -p1.x; l[1] = -p1.y; l[2] = -p1.z;
            v[0] = -p2.x; v[1] = -p2.y; v[2] = -p2.z;
            if (A.want_nb) r = __double2float_rn(A.rs2[A.rs2_scalar ? 0 : k]);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (q & 1) {
                nh[q / 2][c].y = h[c]; nl[q / 2][c].y = l[c]; nv[q / 2][c].y = v[c];
            } else {
                nh[q / 2][c].x = h[c]; nl[q / 2][c].x = l[c]; nv[q / 2][c].x = v[c];
            }
        }
        if (q & 1) rs2f[q / 2].y = r; else rs2f[q / 2].x = r;
        gi[q / 2][q & 1] = (int32_t)gg;  // -1 matches no j
        cnt[q] = 0;
    }
    float2 acc[NP][7];
#pragma unroll
    for (int q = 0; q < NP; ++q)
#pragma unroll
        for (int c = 0; c < 7; ++c) acc[q][c] = make_float2(0.f, 0.f);

    const unsigned below = (1u << lane) - 1u;
    for (int64_t base = w0; base < w1; base += 32) {  // warp-uniform trip count
        const int64_t j = base + lane;
        const bool valid = j < w1;
        const int32_t j32 = (int32_t)j;
        float4 a, b, c, d;
        float2 VY, VZ;
        {
            float4 p0 = make_float4(kPadPos, kPadPos, kPadPos, 0.f), p1 = make_float4(0.f, 0.f, 0.f, 0.f), p2 = p1;
            if (valid) {
                p0 = __ldg(rec + 3 * j);
                p1 = __ldg(rec + 3 * j + 1);
                p2 = __ldg(rec + 3 * j + 2);
            }
            a = make_float4(p0.x, p0.x, p0.y, p0.y);
            b = make_float4(p0.z, p0.z, p0.w, p0.w);
            c = make_float4(p1.x, p1.x, p1.y, p1.y);
            d = make_float4(p1.z, p1.z, p2.x, p2.x);
            VY = make_float2(p2.y, p2.y);
            VZ = make_float2(p2.z, p2.z);
        }
        bool self = false;  // warp-uniform: does a row's own index fall in this round?
#pragma unroll
        for (int q = 0; q < NP; ++q)
            self |= (gi[q][0] >= base && gi[q][0] < base + 32) | (gi[q][1] >= base && gi[q][1] < base + 32);
        const bool hit = self ? js_round_x2<NP, true>(a, b, c, d, VY, VZ, j32, nh, nl, nv, rs2f, gi, acc)
                              : js_round_x2<NP, false>(a, b, c, d, VY, VZ, j32, nh, nl, nv, rs2f, gi, acc);
        if (__any_sync(0xffffffffu, hit)) {  // rare: record this round's hits row by row
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                float2 dx, dy, dz;
                const float2 r2 = x2_r2(a, b, c, d, nh[q], nl[q], dx, dy, dz);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int row = 2 * q + h;
                    const bool hq = valid && (h ? r2.y < rs2f[q].y : r2.x < rs2f[q].x) && j32 != gi[q][h];
                    const unsigned mask = __ballot_sync(0xffffffffu, hq);
                    if (mask) {
                        const int pos = cnt[row] + __popc(mask & below);
                        if (hq && pos < A.L) A.seg_slots[(g * A.n_i + k0 + row) * A.L + pos] = j32;
                        cnt[row] += __popc(mask);
                    }
                }
            }
        }
    }
    if (A.want_nb && lane == 0) {
#pragma unroll
        for (int q = 0; q < IB; ++q)
            if (k0 + q < A.n_i) A.seg_cnt[g * A.n_i + k0 + q] = cnt[q];
    }
    // block reduction: warp shuffles, then one FP64 slot per warp, summed in warp order
#pragma unroll
    for (int q = 0; q < IB; ++q)
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            const float v = warp_sum((q & 1) ? acc[q / 2][c].y : acc[q / 2][c].x);
            if (lane == 0) red[w][q][c] = (double)v;
        }
    __syncthreads();
    for (int e = tid; e < IB * 7; e += BLOCK) {
        const int q = e / 7, c = e % 7;
        const int64_t k = k0 + q;
        if (k < A.n_i) {
            double sum = 0.0;
#pragma unroll
            for (int ww = 0; ww < W; ++ww) sum += red[ww][q][c];
            A.part[((int64_t)s * 7 + c) * A.n_i + k] = (c == 6) ? -sum : sum;
        }
    }
}

// Dynamic shared memory of k_force_mixed_tiled_x2: the raw tile (cp.async target), the
// duplicated tile, and the FP64 running sums of every row, dacc[c][q][thread].
template <int NI, int BLOCK, int TJ>
constexpr int x2_smem_bytes()
{
    return 3 * TJ * 16 + 5 * TJ * 16 + 7 * NI * BLOCK * 8;
}

template <int NI, int BLOCK, int TJ, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_force_mixed_tiled_x2(ForceArgs A)
{
    constexpr int NP = NI / 2;
    // j per unrolled body: four for two rows a thread, two for four rows, one where four rows
    // must fit in 128 registers (more would spill)
    constexpr int UJ = NI >= 4 ? (MINB >= 4 ? 1 : 2) : 4;
    extern __shared__ __align__(16) float4 x2_smem[];
    float4 *raw = x2_smem;              // 3*TJ float4
    float4 *dup = x2_smem + 3 * TJ;     // 5*TJ float4
    double *dacc = reinterpret_cast<double *>(x2_smem + 8 * TJ);  // [7][NI][BLOCK]
    const int tid = threadIdx.x;
    const int64_t kbase = (int64_t)blockIdx.x * (BLOCK * NI);
    const int s = blockIdx.y;
    const int64_t tb = A.j_lo / TJ;  // first tile of the source range
    const int64_t t0 = tb + (A.n_tiles * s) / A.S, t1 = tb + (A.n_tiles * (s + 1)) / A.S;
    const float4 *rec = static_cast<const float4 *>(A.rec);

    // rows q*BLOCK + tid (q = 0..NI-1); pair p holds rows 2p and 2p+1
    // the neighbour segment of row q starts at slot0 + q * sstride (rows past n_i never hit)
    float2 nh[NP][3], nl[NP][3], nv[NP][3], rs2f[NP];
    int32_t gi[NP][2];
    int cnt[NP][2];
    int32_t *const slot0 = A.seg_slots + ((int64_t)s * A.n_i + kbase + tid) * A.L;
    const int64_t sstride = (int64_t)BLOCK * A.L;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float h[2][3], l[2][3], v[2][3], r[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t k = kbase + (2 * p + u) * BLOCK + tid;
            int64_t g = -1;
            if (k < A.n_i) {
                g = A.idx[k];
                if (g < 0 || g >= A.n) {
                    if (s == 0) atomicOr(A.status, ST_BAD_INDEX);
                    g = -1;
                }
            }
            gi[p][u] = (int32_t)g;
            cnt[p][u] = 0;
            if (g >= 0) {
                const float4 p0 = rec[3 * g], p1 = rec[3 * g + 1], p2 = rec[3 * g + 2];
                h[u][0] = -p0.x; h[u][1] = -p0.y; h[u][2] = -p0.z;
                l[u][0] = -p1.x; l[u][1] = -p1.y; l[u][2] = -p1.z;
                v[u][0] = -p2.x; v[u][1] = -p2.y; v[u][2] = -p2.z;
                r[u] = A.want_nb ? __double2float_rn(A.rs2[A.rs2_scalar ? 0 : k]) : -1.f;
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) h[u][c] = l[u][c] = v[u][c] = 0.f;
                r[u] = -1.f;
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            nh[p][c] = make_float2(h[0][c], h[1][c]);
            nl[p][c] = make_float2(l[0][c], l[1][c]);
            nv[p][c] = make_float2(v[0][c], v[1][c]);
        }
        rs2f[p] = make_float2(r[0], r[1]);
    }
#pragma unroll
    for (int e = 0; e < 7 * NI; ++e) dacc[e * BLOCK + tid] = 0.0;

    auto load_tile = [&](int64_t t) {
        const float4 *src = rec + t * (3 * TJ);
#pragma unroll
        for (int e = tid; e < 3 * TJ; e += BLOCK) cp_async16(&raw[e], src + e);
        cp_async_commit();
    };

    // FP32 sums of PT consecutive tiles, then promoted to the FP64 running sums: every two
    // tiles, except for four rows at 3 CTAs per SM, where the longer FP32 chain was slower
    constexpr int PT = (NI >= 4 && MINB < 4) ? 1 : 2;
    float2 acc[NP][7];
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int c = 0; c < 7; ++c) acc[p][c] = make_float2(0.f, 0.f);
    // one raw buffer: tile t+1 lands in it while tile t is computed from dup
    if (t0 < t1) load_tile(t0);
    for (int64_t t = t0; t < t1; ++t) {
        cp_async_wait<0>();
        __syncthreads();  // raw holds tile t; every thread is done with the previous dup
#pragma unroll
        for (int jj = tid; jj < TJ; jj += BLOCK) {
            const float4 p0 = raw[3 * jj], p1 = raw[3 * jj + 1], p2 = raw[3 * jj + 2];
            dup[5 * jj] = make_float4(p0.x, p0.x, p0.y, p0.y);
            dup[5 * jj + 1] = make_float4(p0.z, p0.z, p0.w, p0.w);
            dup[5 * jj + 2] = make_float4(p1.x, p1.x, p1.y, p1.y);
            dup[5 * jj + 3] = make_float4(p1.z, p1.z, p2.x, p2.x);
            dup[5 * jj + 4] = make_float4(p2.y, p2.y, p2.z, p2.z);
        }
        __syncthreads();  // dup complete; raw is free again
        if (t + 1 < t1) load_tile(t + 1);
        const int64_t jb = t * TJ;
        bool mine = false;
#pragma unroll
        for (int p = 0; p < NP; ++p) mine |= (gi[p][0] >= jb && gi[p][0] < jb + TJ) | (gi[p][1] >= jb && gi[p][1] < jb + TJ);
        if (__any_sync(0xffffffffu, mine))
            tile_mixed_x2<NP, true, TJ, UJ>(dup, jb, A.j_hi, A.L, nh, nl, nv, rs2f, gi, slot0, sstride, cnt, acc);
        else
            tile_mixed_x2<NP, false, TJ, UJ>(dup, jb, A.j_hi, A.L, nh, nl, nv, rs2f, gi, slot0, sstride, cnt, acc);
        if ((t - t0) % PT == PT - 1 || t + 1 == t1) {
#pragma unroll
            for (int p = 0; p < NP; ++p)
#pragma unroll
                for (int c = 0; c < 7; ++c) {
                    dacc[(c * NI + 2 * p) * BLOCK + tid] += (double)acc[p][c].x;
                    dacc[(c * NI + 2 * p + 1) * BLOCK + tid] += (double)acc[p][c].y;
                    acc[p][c] = make_float2(0.f, 0.f);
                }
        }
    }
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int64_t k = kbase + q * BLOCK + tid;
        if (k < A.n_i) {
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                const double v = dacc[(c * NI + q) * BLOCK + tid];
                A.part[((int64_t)s * 7 + c) * A.n_i + k] = (c == 6) ? -v : v;
            }
            if (A.want_nb) A.seg_cnt[(int64_t)s * A.n_i + k] = cnt[q >> 1][q & 1];
        }
    }
}

// ------------------------------------------------------------------------------------------
// Anchored packed kernel.  The rows of a CTA are taken in the order A.perm (Morton order of
// their positions, so a CTA's rows lie close together) and every position is measured from
// one anchor B per CTA, the predicted position of the CTA's middle row: e_i = ds(x_i - B) once
// per row and f_j = ds(x_j - B) once per j and CTA (in the tile expansion), both rounded to
// FP32, with ds the double-single difference of the other kernels.  The pair separation is
// then the single FP32 subtraction f_j - e_i: 3 lane-operations per pair where the
// double-single difference takes 9 (27 instead of 33 FP32 lane-operations a pair), at an
// error of at most about 4u |x_i - B| + 3u |r| (u = 2^-24) in the separation.  Pairs for which
// that is not small against |r| — |r| below r_c,i = |x_i - B| / 16, where the bound is 67u |r| —
// are masked out of the interaction loop (their inverse distance set to 0) and added by the
// chunk replay with the double-single separation, exactly as the other kernels compute them.
// The replay also decides the neighbours, from the double-single r^2 of the other kernels, so
// the lists are bit-identical to theirs.  The loop's hit mask marks j that is either masked
// (anchored r^2 < r_c,i^2) or possibly a neighbour (anchored r^2 < max(r_s^2, r_c,i^2) (1 +
// 2^-10), a margin far above the anchored r^2 error at those distances).  The self pair has
// separation exactly 0 (e_i and f_i are the same computation) and is masked like any pair.
// Correct for any row order; the order only decides how many pairs are masked.
//
// Duplicated tile layout, five float4 per j:
//   {fx,fx,fy,fy} {fz,fz,m,m} {vx,vx,vy,vy} {vz,vz,xh,yh} {zh,xl,yl,zl}
// (the loop reads the first four; the replay also reads the absolute hi/lo position).
// Per-row data the replay needs live in shared memory: index, output row, neighbour count,
// r_s^2 (float) and the row's hi/lo position.
enum { AR_GI = 0, AR_K = 1, AR_CNT = 2, AR_RS2 = 3, AR_LIM = 4, AR_WORDS = 5 };

// HITS > 0: every row's neighbour hits are gathered in shared memory, HITS at a time (8: one
// 32-byte sector, 16: two), and written out as whole aligned groups instead of one 4-byte store
// a hit, which leaves partly written sectors that the memory system completes with extra DRAM
// reads and writes.
template <int NI, int BLOCK, int TJ, int HITS = 0>
constexpr int anchored_smem_bytes()
{
    return 3 * TJ * 16 + 5 * TJ * 16 + 7 * NI * BLOCK * 8 + (AR_WORDS + HITS) * NI * BLOCK * 4;
}

// Writes the staged hits first .. last (inclusive, one group of HITS) of one row to its
// neighbour segment: a whole aligned group as 16-byte stores, a partial one entry by entry.
template <int HITS>
__device__ __forceinline__ void flush_staged(int32_t *seg, const int32_t *sbuf, int stride, int first, int last,
                                             bool aligned)
{
    // streaming (evict-first) stores: the lists are read once, by the CSR gather
    if (aligned && last - first == HITS - 1) {
        int4 *dst = reinterpret_cast<int4 *>(seg + first);
#pragma unroll
        for (int q = 0; q < HITS / 4; ++q)
            __stcs(dst + q, make_int4(sbuf[(4 * q) * stride], sbuf[(4 * q + 1) * stride], sbuf[(4 * q + 2) * stride],
                                      sbuf[(4 * q + 3) * stride]));
    } else {
        for (int q = first; q <= last; ++q) __stcs(seg + q, sbuf[(q & (HITS - 1)) * stride]);
    }
}

template <int NP, int BLOCK, int TJ, int UJ, int HITS>
__device__ __forceinline__ void tile_mixed_anchored(const float4 *__restrict__ sd, int64_t jb, const ForceArgs &A,
                                                    int s, const float2 (&ne)[NP][3], const float2 (&nv)[NP][3],
                                                    const float2 (&tm)[NP], const float2 (&th)[NP],
                                                    int32_t *__restrict__ srow, float2 (&acc)[NP][7])
{
    static_assert(TJ % 32 == 0, "tiles are whole 32-j chunks");
    constexpr int NR = 2 * NP;  // rows a thread
    const float2 m3 = make_float2(-3.f, -3.f);
    const int tid = threadIdx.x;
    for (int jc = 0; jc < TJ; jc += 32) {
        const float4 *sc = sd + 5 * jc;
        unsigned hm = 0;
#pragma unroll UJ
        for (int u = 0; u < 32; ++u) {
            const float4 a = sc[5 * u], b = sc[5 * u + 1], c = sc[5 * u + 2], d = sc[5 * u + 3];
            const float2 M = make_float2(b.z, b.w), VX = make_float2(c.x, c.y), VY = make_float2(c.z, c.w);
            const float2 VZ = make_float2(d.x, d.y);
            bool hit = false;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const float2 dx = f2add(make_float2(a.x, a.y), ne[q][0]);
                const float2 dy = f2add(make_float2(a.z, a.w), ne[q][1]);
                const float2 dz = f2add(make_float2(b.x, b.y), ne[q][2]);
                const float2 r2 = f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx)));
                float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                rinv.x = r2.x < tm[q].x ? 0.f : rinv.x;
                rinv.y = r2.y < tm[q].y ? 0.f : rinv.y;
                const float2 wx = f2add(VX, nv[q][0]), wy = f2add(VY, nv[q][1]), wz = f2add(VZ, nv[q][2]);
                const float2 rw = f2fma(dz, wz, f2fma(dy, wy, f2mul(dx, wx)));
                const float2 rinv2 = f2mul(rinv, rinv);
                const float2 mr = f2mul(M, rinv);
                const float2 mr3 = f2mul(mr, rinv2);
                const float2 beta = f2mul(rw, f2mul(rinv2, m3));
                acc[q][0] = f2fma(mr3, dx, acc[q][0]);
                acc[q][1] = f2fma(mr3, dy, acc[q][1]);
                acc[q][2] = f2fma(mr3, dz, acc[q][2]);
                acc[q][3] = f2fma(mr3, f2fma(beta, dx, wx), acc[q][3]);
                acc[q][4] = f2fma(mr3, f2fma(beta, dy, wy), acc[q][4]);
                acc[q][5] = f2fma(mr3, f2fma(beta, dz, wz), acc[q][5]);
                acc[q][6] = f2add(acc[q][6], mr);
                hit |= (r2.x < th[q].x) | (r2.y < th[q].y);
            }
            hm |= (unsigned)hit << u;
        }
        // replay of the chunk's rare hits, in ascending j
        while (hm) {
            const int u = __ffs(hm) - 1;
            hm &= hm - 1;
            const int64_t j = jb + jc + u;
            const int32_t j32 = (int32_t)j;
            const float4 a = sc[5 * u], b = sc[5 * u + 1], c = sc[5 * u + 2], d = sc[5 * u + 3], e = sc[5 * u + 4];
            const float jh[3] = {d.z, d.w, e.x}, jl[3] = {e.y, e.z, e.w}, jv[3] = {c.x, c.z, d.x};
            const float jm = b.z;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const float2 dx = f2add(make_float2(a.x, a.y), ne[q][0]);
                const float2 dy = f2add(make_float2(a.z, a.w), ne[q][1]);
                const float2 dz = f2add(make_float2(b.x, b.y), ne[q][2]);
                const float2 r2 = f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx)));
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float r2a = h ? r2.y : r2.x;
                    if (!(r2a < (h ? th[q].y : th[q].x))) continue;
                    const int slot = (2 * q + h) * BLOCK + tid;
                    const int32_t gi = srow[AR_GI * NR * BLOCK + slot];
                    if (j32 == gi) continue;
                    const float *xr = reinterpret_cast<const float *>(srow);
                    // the row's double-single position from its j-record (a candidate pair is
                    // rare, and shared memory is what bounds the staged variants' occupancy)
                    const float4 *recp = static_cast<const float4 *>(A.rec);
                    const float4 ph = __ldg(recp + 3 * (int64_t)gi), pl = __ldg(recp + 3 * (int64_t)gi + 1);
                    const float xh3[3] = {ph.x, ph.y, ph.z}, xl3[3] = {pl.x, pl.y, pl.z};
                    float r[3];
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) r[cc] = ds_diff(jh[cc], jl[cc], xh3[cc], xl3[cc]);
                    const float r2p = r2_f32(r[0], r[1], r[2]);
                    if (r2p < xr[AR_RS2 * NR * BLOCK + slot] && j < A.j_hi) {
                        int32_t *cp = srow + AR_CNT * NR * BLOCK + slot;
                        const int cnt = *cp;
                        const int lim = srow[AR_LIM * NR * BLOCK + slot];
                        if (cnt < lim) {
                            // the row's segment at its position in the spatial order
                            const int64_t r = (int64_t)blockIdx.x * (NR * BLOCK) + slot;
                            int32_t *seg = A.seg_slots + ((int64_t)s * A.n_i + r) * A.L;
                            if (HITS > 0) {
                                int32_t *sbuf = srow + AR_WORDS * NR * BLOCK + slot;
                                sbuf[(cnt & (HITS - 1)) * NR * BLOCK] = j32;
                                if ((cnt & (HITS - 1)) == HITS - 1 || cnt == lim - 1)
                                    flush_staged<HITS>(seg, sbuf, NR * BLOCK, cnt & ~(HITS - 1), cnt,
                                                       (A.L & (HITS - 1)) == 0);
                            } else {
                                __stcs(seg + cnt, j32);
                            }
                        }
                        *cp = cnt + 1;
                    }
                    if (r2a < (h ? tm[q].y : tm[q].x)) {  // masked: add the pair in double-single form
                        const float rinv = rsqrtf(r2p);
                        const float w0 = jv[0] + (h ? nv[q][0].y : nv[q][0].x);
                        const float w1 = jv[1] + (h ? nv[q][1].y : nv[q][1].x);
                        const float w2 = jv[2] + (h ? nv[q][2].y : nv[q][2].x);
                        const float rw = r[0] * w0 + r[1] * w1 + r[2] * w2;
                        const float rinv2 = rinv * rinv;
                        const float mr = jm * rinv;
                        const float mr3 = mr * rinv2;
                        const float beta = rw * (rinv2 * -3.f);
                        const float t[7] = {mr3 * r[0], mr3 * r[1], mr3 * r[2], mr3 * (w0 + beta * r[0]),
                                            mr3 * (w1 + beta * r[1]), mr3 * (w2 + beta * r[2]), mr};
#pragma unroll
                        for (int cc = 0; cc < 7; ++cc) {
                            if (h) acc[q][cc].y += t[cc];
                            else acc[q][cc].x += t[cc];
                        }
                    }
                }
            }
        }
    }
}

template <int NI, int BLOCK, int TJ, int MINB, int HITS>
__device__ __forceinline__ void anchored_body(const ForceArgs &A)
{
    constexpr int NP = NI / 2;
    constexpr int UJ = NI >= 4 ? (MINB >= 4 ? 1 : 2) : 4;
    constexpr int PT = TJ >= 256 ? 1 : 256 / TJ;  // FP32 sums over 256 j, then promoted to FP64
    extern __shared__ __align__(16) float4 an_smem[];
    float4 *raw = an_smem;                                           // 3*TJ float4
    float4 *dup = an_smem + 3 * TJ;                                  // 5*TJ float4
    double *dacc = reinterpret_cast<double *>(an_smem + 8 * TJ);     // [7][NI][BLOCK]
    int32_t *srow = reinterpret_cast<int32_t *>(dacc + 7 * NI * BLOCK);  // [AR_WORDS][NI*BLOCK]
    float *srowf = reinterpret_cast<float *>(srow);
    __shared__ float s_anchor[6];  // B as hi (x, y, z) and lo (x, y, z)
    const int tid = threadIdx.x;
    const int64_t kbase = (int64_t)blockIdx.x * (BLOCK * NI);
    const int s = blockIdx.y;
    const int64_t tb = A.j_lo / TJ;
    const int64_t t0 = tb + (A.n_tiles * s) / A.S, t1 = tb + (A.n_tiles * (s + 1)) / A.S;
    const float4 *rec = static_cast<const float4 *>(A.rec);

    if (tid == 0) {
        const int64_t rows = A.n_i - kbase < NI * BLOCK ? A.n_i - kbase : NI * BLOCK;
        const int64_t ra = kbase + rows / 2;
        const int64_t ka = A.perm ? A.perm[ra] : ra;
        const int64_t ga = (ka >= 0 && ka < A.n_i) ? A.idx[ka] : -1;
        float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
        if (ga >= 0 && ga < A.n) {
            h = rec[3 * ga];
            l = rec[3 * ga + 1];
        }
        s_anchor[0] = h.x; s_anchor[1] = h.y; s_anchor[2] = h.z;
        s_anchor[3] = l.x; s_anchor[4] = l.y; s_anchor[5] = l.z;
    }
    __syncthreads();
    const float Bh[3] = {s_anchor[0], s_anchor[1], s_anchor[2]}, Bl[3] = {s_anchor[3], s_anchor[4], s_anchor[5]};

    float2 ne[NP][3], nv[NP][3], tm[NP], th[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float e[2][3], v[2][3], tmask[2], thit[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int slot = (2 * p + u) * BLOCK + tid;
            const int64_t r = kbase + slot;
            int64_t k = -1, g = -1;
            if (r < A.n_i) {
                k = A.perm ? A.perm[r] : r;
                g = A.idx[k];
                if (g < 0 || g >= A.n) {
                    if (s == 0) atomicOr(A.status, ST_BAD_INDEX);
                    g = -1;
                }
            }
            float h3[3] = {0.f, 0.f, 0.f}, l3[3] = {0.f, 0.f, 0.f}, rs2f = -1.f;
            v[u][0] = v[u][1] = v[u][2] = 0.f;
            if (g >= 0) {
                const float4 p0 = rec[3 * g], p1 = rec[3 * g + 1], p2 = rec[3 * g + 2];
                h3[0] = p0.x; h3[1] = p0.y; h3[2] = p0.z;
                l3[0] = p1.x; l3[1] = p1.y; l3[2] = p1.z;
                v[u][0] = -p2.x; v[u][1] = -p2.y; v[u][2] = -p2.z;
                if (A.want_nb) rs2f = __double2float_rn(A.rs2[A.rs2_scalar ? 0 : k]);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) e[u][c] = -ds_diff(h3[c], l3[c], Bh[c], Bl[c]);
            const float ee = r2_f32(e[u][0], e[u][1], e[u][2]);
            const float rc2 = fmaxf(ee * (1.f / 256.f), 1.17549435e-38f);
            tmask[u] = g >= 0 ? rc2 : -1.f;
            thit[u] = g >= 0 ? fmaxf(rs2f, rc2) * (1.f + 1.f / 1024.f) : -1.f;
            srow[AR_GI * NI * BLOCK + slot] = (int32_t)g;
            srow[AR_K * NI * BLOCK + slot] = (int32_t)k;
            srow[AR_CNT * NI * BLOCK + slot] = 0;
            int32_t lim = A.L;
            if (A.cap > 0 && s > 0 && k >= 0) {
                // the hits the row's earlier segments hold, from the counts their CTAs have
                // written by now (-1: not yet written, taken as none): only nb_cap minus those
                // can reach the row's list, so no more are stored (the count stays complete)
                int64_t prior = 0;
                for (int q2 = 0; q2 < s; ++q2) {
                    const int32_t c2 = __ldcg(A.seg_cnt + (int64_t)q2 * A.n_i + r);
                    if (c2 > 0) prior += c2;
                }
                const int64_t room = (int64_t)A.cap - prior;
                lim = room <= 0 ? 0 : (room < A.L ? (int32_t)room : A.L);
            }
            srow[AR_LIM * NI * BLOCK + slot] = lim;
            srowf[AR_RS2 * NI * BLOCK + slot] = rs2f;

        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ne[p][c] = make_float2(e[0][c], e[1][c]);
            nv[p][c] = make_float2(v[0][c], v[1][c]);
        }
        tm[p] = make_float2(tmask[0], tmask[1]);
        th[p] = make_float2(thit[0], thit[1]);
    }
#pragma unroll
    for (int e = 0; e < 7 * NI; ++e) dacc[e * BLOCK + tid] = 0.0;

    const uint64_t keep = l2_keep_policy();  // the j-records stay in L2 past the list stores
    auto load_tile = [&](int64_t t) {
        const float4 *src = rec + t * (3 * TJ);
#pragma unroll
        for (int e = tid; e < 3 * TJ; e += BLOCK) cp_async16_keep(&raw[e], src + e, keep);
        cp_async_commit();
    };
    float2 acc[NP][7];
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
        for (int c = 0; c < 7; ++c) acc[p][c] = make_float2(0.f, 0.f);
    if (t0 < t1) load_tile(t0);
    for (int64_t t = t0; t < t1; ++t) {
        cp_async_wait<0>();
        __syncthreads();  // raw holds tile t; every thread is done with the previous dup
#pragma unroll
        for (int jj = tid; jj < TJ; jj += BLOCK) {
            const float4 p0 = raw[3 * jj], p1 = raw[3 * jj + 1], p2 = raw[3 * jj + 2];
            const float fx = ds_diff(p0.x, p1.x, Bh[0], Bl[0]);
            const float fy = ds_diff(p0.y, p1.y, Bh[1], Bl[1]);
            const float fz = ds_diff(p0.z, p1.z, Bh[2], Bl[2]);
            dup[5 * jj] = make_float4(fx, fx, fy, fy);
            dup[5 * jj + 1] = make_float4(fz, fz, p0.w, p0.w);
            dup[5 * jj + 2] = make_float4(p2.x, p2.x, p2.y, p2.y);
            dup[5 * jj + 3] = make_float4(p2.z, p2.z, p0.x, p0.y);
            dup[5 * jj + 4] = make_float4(p0.z, p1.x, p1.y, p1.z);
        }
        __syncthreads();  // dup complete; raw is free again
        if (t + 1 < t1) load_tile(t + 1);
        tile_mixed_anchored<NP, BLOCK, TJ, UJ, HITS>(dup, t * TJ, A, s, ne, nv, tm, th, srow, acc);
        if ((t - t0) % PT == PT - 1 || t + 1 == t1) {
#pragma unroll
            for (int p = 0; p < NP; ++p)
#pragma unroll
                for (int c = 0; c < 7; ++c) {
                    dacc[(c * NI + 2 * p) * BLOCK + tid] += (double)acc[p][c].x;
                    dacc[(c * NI + 2 * p + 1) * BLOCK + tid] += (double)acc[p][c].y;
                    acc[p][c] = make_float2(0.f, 0.f);
                }
        }
    }
#pragma unroll
    for (int q = 0; q < NI; ++q) {
        const int slot = q * BLOCK + tid;
        const int64_t k = srow[AR_K * NI * BLOCK + slot];
        if (k >= 0) {
            // the sums at the row's position in the spatial order (consecutive threads,
            // consecutive positions: whole sectors); the reduction puts them back in row order
            const int64_t r = kbase + slot;
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                const double v = dacc[(c * NI + q) * BLOCK + tid];
                __stcs(A.part + ((int64_t)s * 7 + c) * A.n_i + r, (c == 6) ? -v : v);
            }
            if (A.want_nb) {  // the count and the last group, at the position too
                const int cnt = srow[AR_CNT * NI * BLOCK + slot];
                A.seg_cnt[(int64_t)s * A.n_i + r] = cnt;
                const int lim = srow[AR_LIM * NI * BLOCK + slot];
                const int c = cnt;  // staged hits not yet written (a last, partial group)
                if (HITS > 0 && cnt < lim && (c & (HITS - 1)) != 0) {
                    // with L a multiple of HITS the whole group is written (the slots past the
                    // count hold stale values that nothing reads), so every list store is a
                    // whole aligned chunk
                    const bool whole = (A.L & (HITS - 1)) == 0;
                    flush_staged<HITS>(A.seg_slots + ((int64_t)s * A.n_i + r) * A.L,
                                       srow + AR_WORDS * NI * BLOCK + slot, NI * BLOCK, c & ~(HITS - 1),
                                       whole ? (c | (HITS - 1)) : c - 1, whole);
                }
            }
        }
    }
}

template <int NI, int BLOCK, int TJ, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_force_mixed_anchored_x2(ForceArgs A)
{
    anchored_body<NI, BLOCK, TJ, MINB, 0>(A);
}

// The anchored kernel with the neighbour hits staged in shared memory and written in whole
// 32-byte sectors (8 hits), or in pairs of sectors (16 hits: the two-row variant).
template <int NI, int BLOCK, int TJ, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_force_mixed_staged_x2(ForceArgs A)
{
    anchored_body<NI, BLOCK, TJ, MINB, NI >= 4 ? 8 : 16>(A);
}

// The same with 16 hits (64 bytes) a group whatever the rows per thread.  HBM is written in
// 64-byte units: a group of 8 hits is half a unit, which the memory system completes with a
// read of the other half.
template <int NI, int BLOCK, int TJ, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_force_mixed_staged16_x2(ForceArgs A)
{
    anchored_body<NI, BLOCK, TJ, MINB, 16>(A);
}

// ------------------------------------------------------------------------------------------
// Batched ensemble kernel: many independent clusters in one persistent launch.  The particle
// arrays of all clusters are concatenated; cluster c owns the j-range
// [cluster_off[c], cluster_off[c+1]) and the active rows it lists.  Work items (cluster, up to
// NI*BLOCK consecutive active rows) are popped from a device counter in the order the host
// sorted them (largest cost first), so uneven clusters balance across the SMs.  Each item
// walks its cluster's j-range in ragged tiles (records past the range are replaced by
// massless padding during the tile expansion) with the packed-FP32x2 inner loop, and writes
// its rows' sums and neighbour segment directly (one split per row).  The pop is a single
// atomicAdd: no CTA ever waits on another.
template <int NI, int BLOCK, int TJ, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_force_mixed_batched(BatchArgs A)
{
    constexpr int NP = NI / 2;
    // j per unrolled body: four for two rows a thread, two for four rows, one where four rows
    // must fit in 128 registers (more would spill)
    constexpr int UJ = NI >= 4 ? (MINB >= 4 ? 1 : 2) : 4;
    extern __shared__ __align__(16) float4 x2_smem[];
    float4 *raw = x2_smem;
    float4 *dup = x2_smem + 3 * TJ;
    double *dacc = reinterpret_cast<double *>(x2_smem + 8 * TJ);  // [7][NI][BLOCK]
    __shared__ int s_item;
    const int tid = threadIdx.x;

    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(A.queue, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();  // every thread holds `it` before thread 0 pops again
        if (it >= A.n_items) break;
        const BatchItem W = A.items[it];
        const int64_t j0 = A.cluster_off[W.cluster], j1 = A.cluster_off[W.cluster + 1];
        const float rs2c = A.want_nb ? __double2float_rn(A.rs2[W.cluster]) : -1.f;

        float2 nh[NP][3], nl[NP][3], nv[NP][3], rs2f[NP];
        int32_t gi[NP][2];
        int cnt[NP][2];
        int32_t *const slot0 = A.seg_slots + ((int64_t)W.row0 + tid) * A.L;  // row q: + q * sstride
        const int64_t sstride = (int64_t)BLOCK * A.L;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float h[2][3], l[2][3], v[2][3], r[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int rr = (2 * p + u) * BLOCK + tid;
                const int64_t k = (int64_t)W.row0 + rr;
                int64_t g = -1;
                if (rr < W.rows) {
                    g = A.idx[k];
                    if (g < j0 || g >= j1) {  // every active index must lie in its cluster
                        atomicOr(A.status, ST_BAD_INDEX);
                        g = -1;
                    }
                }
                gi[p][u] = (int32_t)g;
                cnt[p][u] = 0;
                if (g >= 0) {
                    const float4 p0 = A.rec[3 * g], p1 = A.rec[3 * g + 1], p2 = A.rec[3 * g + 2];
                    h[u][0] = -p0.x; h[u][1] = -p0.y; h[u][2] = -p0.z;
                    l[u][0] = -p1.x; l[u][1] = -p1.y; l[u][2] = -p1.z;
                    v[u][0] = -p2.x; v[u][1] = -p2.y; v[u][2] = -p2.z;
                    r[u] = rs2c;
                } else {
#pragma unroll
                    for (int c = 0; c < 3; ++c) h[u][c] = l[u][c] = v[u][c] = 0.f;
                    r[u] = -1.f;
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                nh[p][c] = make_float2(h[0][c], h[1][c]);
                nl[p][c] = make_float2(l[0][c], l[1][c]);
                nv[p][c] = make_float2(v[0][c], v[1][c]);
            }
            rs2f[p] = make_float2(r[0], r[1]);
        }
#pragma unroll
        for (int e = 0; e < 7 * NI; ++e) dacc[e * BLOCK + tid] = 0.0;

        const int64_t n_t = (j1 - j0 + TJ - 1) / TJ;
        auto load_tile = [&](int64_t t) {
            const int64_t jb = j0 + t * TJ;
            const int valid = (int)((j1 - jb) < TJ ? (j1 - jb) : TJ);
            const float4 *src = A.rec + jb * 3;
            for (int e = tid; e < 3 * valid; e += BLOCK) cp_async16(&raw[e], src + e);
            cp_async_commit();
        };
        if (n_t > 0) load_tile(0);
        for (int64_t t = 0; t < n_t; ++t) {
            const int64_t jb = j0 + t * TJ;
            const int valid = (int)((j1 - jb) < TJ ? (j1 - jb) : TJ);
            cp_async_wait<0>();
            __syncthreads();
#pragma unroll
            for (int jj = tid; jj < TJ; jj += BLOCK) {
                if (jj < valid) {
                    const float4 p0 = raw[3 * jj], p1 = raw[3 * jj + 1], p2 = raw[3 * jj + 2];
                    dup[5 * jj] = make_float4(p0.x, p0.x, p0.y, p0.y);
                    dup[5 * jj + 1] = make_float4(p0.z, p0.z, p0.w, p0.w);
                    dup[5 * jj + 2] = make_float4(p1.x, p1.x, p1.y, p1.y);
                    dup[5 * jj + 3] = make_float4(p1.z, p1.z, p2.x, p2.x);
                    dup[5 * jj + 4] = make_float4(p2.y, p2.y, p2.z, p2.z);
                } else {  // massless, far away: contributes exactly zero
                    dup[5 * jj] = make_float4(kPadPos, kPadPos, kPadPos, kPadPos);
                    dup[5 * jj + 1] = make_float4(kPadPos, kPadPos, 0.f, 0.f);
                    dup[5 * jj + 2] = make_float4(0.f, 0.f, 0.f, 0.f);
                    dup[5 * jj + 3] = make_float4(0.f, 0.f, 0.f, 0.f);
                    dup[5 * jj + 4] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            __syncthreads();
            if (t + 1 < n_t) load_tile(t + 1);
            bool mine = false;
#pragma unroll
            for (int p = 0; p < NP; ++p)
                mine |= (gi[p][0] >= jb && gi[p][0] < jb + TJ) | (gi[p][1] >= jb && gi[p][1] < jb + TJ);
            float2 acc[NP][7];
#pragma unroll
            for (int p = 0; p < NP; ++p)
#pragma unroll
                for (int c = 0; c < 7; ++c) acc[p][c] = make_float2(0.f, 0.f);
            if (__any_sync(0xffffffffu, mine))
                tile_mixed_x2<NP, true, TJ, UJ>(dup, jb, j1, A.L, nh, nl, nv, rs2f, gi, slot0, sstride, cnt, acc);
            else
                tile_mixed_x2<NP, false, TJ, UJ>(dup, jb, j1, A.L, nh, nl, nv, rs2f, gi, slot0, sstride, cnt, acc);
#pragma unroll
            for (int p = 0; p < NP; ++p)
#pragma unroll
                for (int c = 0; c < 7; ++c) {
                    dacc[(c * NI + 2 * p) * BLOCK + tid] += (double)acc[p][c].x;
                    dacc[(c * NI + 2 * p + 1) * BLOCK + tid] += (double)acc[p][c].y;
                }
        }
#pragma unroll
        for (int q = 0; q < NI; ++q) {
            const int rr = q * BLOCK + tid;
            if (rr < W.rows) {
                const int64_t k = (int64_t)W.row0 + rr;
#pragma unroll
                for (int c = 0; c < 7; ++c) {
                    const double v = dacc[(c * NI + q) * BLOCK + tid];
                    A.part[(int64_t)c * A.n_i + k] = (c == 6) ? -v : v;
                }
                if (A.want_nb) A.seg_cnt[k] = cnt[q >> 1][q & 1];
            }
        }
    }
}

#define NB_MIXED_BATCHED_VARIANTS(X)              \
    X(0, 4, 128, 128, 4)                          \
    X(1, 2, 128, 128, 4)                          \
    X(2, 2, 64, 128, 6)

static int batched_smem(int ni, int block, int tj) { return 3 * tj * 16 + 5 * tj * 16 + 7 * ni * block * 8; }

int mixed_batched_rows_per_item(int v)
{
    switch (v) {
#define NB_BV_ROWS(id, NI, B, TJ, MB) \
    case id: return NI * B;
        NB_MIXED_BATCHED_VARIANTS(NB_BV_ROWS)
#undef NB_BV_ROWS
    default: return 0;
    }
}

int mixed_batched_variants() { return 3; }

// Resident CTAs per SM of a batched variant (sets the dynamic shared-memory limit first).
int mixed_batched_occupancy(int v)
{
    int b = 0;
    switch (v) {
#define NB_BV_OCC(id, NI, B, TJ, MB)                                                                   \
    case id:                                                                                           \
        cudaFuncSetAttribute((const void *)k_force_mixed_batched<NI, B, TJ, MB>,                       \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, batched_smem(NI, B, TJ));    \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_force_mixed_batched<NI, B, TJ, MB>, B,      \
                                                      batched_smem(NI, B, TJ));                        \
        break;
        NB_MIXED_BATCHED_VARIANTS(NB_BV_OCC)
#undef NB_BV_OCC
    default: break;
    }
    cudaGetLastError();
    return b > 0 ? b : 1;
}

void launch_force_mixed_batched(cudaStream_t st, int variant, int ctas, const BatchArgs &a)
{
    switch (variant) {
#define NB_BV_LAUNCH(id, NI, B, TJ, MB)                                                            \
    case id:                                                                                       \
        k_force_mixed_batched<NI, B, TJ, MB><<<ctas, B, batched_smem(NI, B, TJ), st>>>(a);         \
        break;
        NB_MIXED_BATCHED_VARIANTS(NB_BV_LAUNCH)
#undef NB_BV_LAUNCH
    default: break;
    }
}

// ------------------------------------------------------------------------------------------
// Variants of the tiled kernel: (id, kernel, NI, BLOCK, TJ, min CTAs per SM, kind).  The plan's
// `variant` indexes this list; ids 0-3 are the scalar kernel, 4-9 the packed-FP32x2 one
// (8 and 9: row tiles of 128 and 64 for blocks of tens to hundreds of rows), 10-19 the
// anchored packed kernel (rows in spatial order, anchor-relative separations; 13 and 14 with
// row tiles of 128 and 64; 15-19 staging the neighbour hits).
// Last column: 0 = scalar (static shared memory), 1 = packed (x2_smem_bytes), 2 = anchored
// (anchored_smem_bytes; needs the row order A.perm), 3 = anchored with the neighbour hits staged
// in shared memory and written as whole sectors (15, 16, 18, 19: 8 hits a group with four rows
// a thread, 16 with two), 4 = the same with 16 hits a group (17).
#define NB_MIXED_TILED_VARIANTS(X)                       \
    X(0, k_force_mixed_tiled, 4, 128, 256, 3, 0)         \
    X(1, k_force_mixed_tiled, 2, 128, 256, 4, 0)         \
    X(2, k_force_mixed_tiled, 1, 128, 256, 4, 0)         \
    X(3, k_force_mixed_tiled, 4, 256, 256, 1, 0)         \
    X(4, k_force_mixed_tiled_x2, 4, 128, 256, 3, 1)      \
    X(5, k_force_mixed_tiled_x2, 2, 128, 256, 4, 1)      \
    X(6, k_force_mixed_tiled_x2, 4, 128, 128, 4, 1)      \
    X(7, k_force_mixed_tiled_x2, 2, 256, 256, 2, 1)      \
    X(8, k_force_mixed_tiled_x2, 2, 64, 128, 8, 1)       \
    X(9, k_force_mixed_tiled_x2, 2, 32, 128, 12, 1)      \
    X(10, k_force_mixed_anchored_x2, 4, 128, 128, 3, 2)  \
    X(11, k_force_mixed_anchored_x2, 2, 128, 128, 4, 2)  \
    X(12, k_force_mixed_anchored_x2, 4, 128, 256, 2, 2)  \
    X(13, k_force_mixed_anchored_x2, 2, 64, 64, 8, 2)    \
    X(14, k_force_mixed_anchored_x2, 2, 32, 64, 12, 2)   \
    X(15, k_force_mixed_staged_x2, 4, 128, 64, 3, 3)     \
    X(16, k_force_mixed_staged_x2, 2, 128, 64, 4, 3)     \
    X(17, k_force_mixed_staged16_x2, 4, 128, 64, 2, 4)   \
    X(18, k_force_mixed_staged_x2, 4, 128, 128, 3, 3)    \
    X(19, k_force_mixed_staged_x2, 4, 128, 256, 2, 3)

struct TiledVariant {
    int ni, block, tj, smem, kind;
};
#define NB_TV_ROW(id, K, NI, B, TJ, MB, KIND)                                                         \
    {NI, B, TJ,                                                                                      \
     KIND == 1 ? x2_smem_bytes<NI, B, TJ>()                                                          \
               : (KIND >= 2 ? anchored_smem_bytes<NI, B, TJ, KIND == 4 ? 16 : (KIND == 3 ? (NI >= 4 ? 8 : 16) : 0)>() : 0), \
     KIND},
static const TiledVariant kTiled[] = {NB_MIXED_TILED_VARIANTS(NB_TV_ROW)};
#undef NB_TV_ROW

int mixed_tiled_dyn_smem(int v) { return kTiled[v].smem; }
int mixed_tiled_anchored(int v) { return v >= 0 && v < (int)(sizeof(kTiled) / sizeof(kTiled[0])) && kTiled[v].kind >= 2; }

// Raise the dynamic shared-memory limit of the packed kernels (needed above 48 KB); called
// once per context before occupancy queries and launches.
void mixed_tiled_configure()
{
#define NB_TV_CFG(id, K, NI, B, TJ, MB, KIND)                                                        \
    if (KIND)                                                                                        \
        cudaFuncSetAttribute((const void *)K<NI, B, TJ, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             kTiled[id].smem);
    NB_MIXED_TILED_VARIANTS(NB_TV_CFG)
#undef NB_TV_CFG
    cudaGetLastError();
}

int mixed_tiled_variants() { return (int)(sizeof(kTiled) / sizeof(kTiled[0])); }

void *mixed_tiled_fn(int v)
{
    switch (v) {
#define NB_TV_FN(id, K, NI, B, TJ, MB, KIND) \
    case id: return (void *)K<NI, B, TJ, MB>;
        NB_MIXED_TILED_VARIANTS(NB_TV_FN)
#undef NB_TV_FN
    default: return nullptr;
    }
}
int mixed_tiled_i_per_cta(int v) { return kTiled[v].ni * kTiled[v].block; }
int mixed_tiled_block(int v) { return kTiled[v].block; }
int mixed_tiled_tj(int v) { return kTiled[v].tj; }
int mixed_jstream_ib(int v) { return v == 0 ? 1 : (v == 1 ? 4 : (v == 2 ? 8 : 2)); }
constexpr int kJstreamBlock = 256;
int jstream_warps() { return kJstreamBlock / 32; }

void launch_force_mixed(cudaStream_t st, int kernel, int variant, int64_t ctas_x, int S, ForceArgs a)
{
    dim3 grid((unsigned)ctas_x, (unsigned)S);
    if (kernel == 1) {
        switch (variant) {
#define NB_TV_LAUNCH(id, K, NI, B, TJ, MB, KIND) \
    case id: K<NI, B, TJ, MB><<<grid, B, kTiled[id].smem, st>>>(a); break;
            NB_MIXED_TILED_VARIANTS(NB_TV_LAUNCH)
#undef NB_TV_LAUNCH
        default: break;
        }
    } else {
        switch (variant) {
        case 0: k_force_mixed_jstream<1, kJstreamBlock><<<grid, kJstreamBlock, 0, st>>>(a); break;
        case 1: k_force_mixed_jstream_x2<4, kJstreamBlock, 2><<<grid, kJstreamBlock, 0, st>>>(a); break;
        case 2: k_force_mixed_jstream_x2<8, kJstreamBlock, 1><<<grid, kJstreamBlock, 0, st>>>(a); break;
        case 3: k_force_mixed_jstream_x2<2, kJstreamBlock, 3><<<grid, kJstreamBlock, 0, st>>>(a); break;
        default: break;
        }
    }
}

}  // namespace nbgpu
