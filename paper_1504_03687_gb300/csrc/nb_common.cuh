// nb_common.cuh — device helpers shared by the sm_103a kernels of the regular-force library.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace nbgpu {

// 32-byte aligned four-double vector (the FP64 j-record half)
using dvec4 = double4_32a;
__host__ __device__ __forceinline__ dvec4 make_dvec4(double x, double y, double z, double w)
{
    return make_double4_32a(x, y, z, w);
}

// Deferred status bits, OR-ed into ctx->d_status[0] by kernels and read by nb_sync.
enum : unsigned {
    ST_NB_TRUNCATED = 1u,   // some active particle had more than nb_cap neighbours
    ST_CSR_FULL = 2u,       // the caller's CSR buffer was too small
    ST_BAD_INDEX = 4u,      // an active index was outside [0, n)
    ST_TIMEOUT = 8u,        // a bounded device wait expired
    ST_DEVICE = 16u,        // a device-side consistency check failed
    ST_DUP_INDEX = 32u      // an active index appeared twice (backward pass only)
};

// Slots of the device status array.
enum { SS_FLAGS = 0, SS_OVERFLOW_COUNT = 1, SS_QUEUE = 2, SS_WORDS = 8 };

constexpr float kPadPos = 1.0e18f;    // far-away position of the padding j-records (mass 0)

// ---- programmatic dependent launch ------------------------------------------------------
// A chain of short dependent kernels (the device-driven block steps) launches each kernel
// with programmatic stream serialisation: its CTAs are scheduled while the kernel before it
// still runs, and wait in pdl_wait() (griddepcontrol.wait: until the grids it depends on have
// completed and their writes are visible) before they touch anything those grids wrote.
// pdl_trigger() lets the next kernel's launch begin.  In a kernel launched the ordinary way
// both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                              Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ---- cp.async (LDGSTS) staging of j-tiles into shared memory ---------------------------
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// L2 policy that keeps a line past streaming traffic (evict_last), and a cp.async carrying it:
// for data every CTA re-reads (the j-records) while a kernel streams its outputs through L2.
__device__ __forceinline__ uint64_t l2_keep_policy()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}
__device__ __forceinline__ void cp_async16_keep(void *smem, const void *gmem, uint64_t policy)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "l"(policy)
                 : "memory");
}

// ---- the neighbour-test distances ------------------------------------------------------
// Both are written with explicit round-to-nearest intrinsics so that every kernel that
// decides "j is a neighbour of i" (the scalar and packed force kernels, and the packed
// kernels' replay of a chunk's hits) obtains bit-identical r^2 values.

// Mixed precision: double-single coordinate difference (hi - hi) + (lo - lo).  The hi
// difference is exact when the particles are close (Sterbenz), so close pairs keep the
// FP64 position's accuracy.
__device__ __forceinline__ float ds_diff(float jh, float jl, float ih, float il)
{
    return __fadd_rn(__fsub_rn(jh, ih), __fsub_rn(jl, il));
}
__device__ __forceinline__ float r2_f32(float dx, float dy, float dz)
{
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// FP64: ((rx*rx + ry*ry) + rz*rz) without contraction.
__device__ __forceinline__ double r2_f64(double rx, double ry, double rz)
{
    return __dadd_rn(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry)), __dmul_rn(rz, rz));
}

// ---- the Hermite predictor -----------------------------------------------------------------
// The Taylor polynomial to the jerk term (Sec. 3.3.3) in Horner form with fused multiply-adds
// (FP64 is a scarce pipe on GB300, so the divisions of the term-by-term form become constant
// factors of dt):
//   x_p = x + dt (v + dt/2 (a + dt/3 jerk)),   v_p = v + dt (a + dt/2 jerk)
// Every kernel that predicts calls this one function, so a particle predicted by the
// all-particle predictor and one predicted on load by the irregular force are bit-identical.
__device__ __forceinline__ void hermite_taylor(double x, double v, double a, double j, double dt, double &xp,
                                               double &vp)
{
    // five FMAs a component; dt/2 and dt/3 are shared by the three components of a particle
    const double h = dt * 0.5, d3 = dt * (1.0 / 3.0);
    xp = __fma_rn(dt, __fma_rn(h, __fma_rn(d3, j, a), v), x);
    vp = __fma_rn(dt, __fma_rn(h, j, a), v);
}

// ---- the Hermite corrector -----------------------------------------------------------------
// Fourth-order Hermite corrector of one component over a step h (Sec. 2, after Makino 1991):
// from the predicted xp, vp and the force and jerk a0, j0 at the start of the step and a1, j1
// at its end, the second and third derivatives of the force at the start,
//   a2 = (-6 (a0 - a1) - h (4 j0 + 2 j1)) / h^2,   a3 = (12 (a0 - a1) + 6 h (j0 + j1)) / h^3,
// and the corrected x1 = xp + h^4/24 a2 + h^5/120 a3, v1 = vp + h^3/6 a2 + h^4/24 a3.  Written
// operation by operation in the order of that definition; the units that call it are compiled
// without FMA contraction, so an FP64 run follows the plain definition to rounding.
__device__ __forceinline__ void hermite_correct(double xp, double vp, double a0, double j0, double a1, double j1,
                                                double h, double &x1, double &v1, double &a2, double &a3)
{
    const double da = a0 - a1;
    a2 = (-6.0 * da - h * (4.0 * j0 + 2.0 * j1)) / (h * h);
    a3 = (12.0 * da + 6.0 * h * (j0 + j1)) / (h * h * h);
    x1 = xp + h * h * h * h / 24.0 * a2 + h * h * h * h * h / 120.0 * a3;
    v1 = vp + h * h * h / 6.0 * a2 + h * h * h * h / 24.0 * a3;
}

// The same corrector for a step h that is a power of two (every block step of the integrator),
// given ih = 1/h (exact): the divisions by h^2 and h^3 become products with ih^2 and ih^3, and
// h^4/24, h^5/120, h^3/6 products with the rounded constants.  Scaling by a power of two
// commutes with rounding, so every result is bit-identical to hermite_correct's, with no FP64
// division (a few dozen instructions on GB300's narrow FP64 pipe).
__device__ __forceinline__ void hermite_correct_pow2(double xp, double vp, double a0, double j0, double a1, double j1,
                                                     double h, double ih, double &x1, double &v1, double &a2,
                                                     double &a3)
{
    const double da = a0 - a1;
    a2 = (-6.0 * da - h * (4.0 * j0 + 2.0 * j1)) * (ih * ih);
    a3 = (12.0 * da + 6.0 * h * (j0 + j1)) * (ih * ih * ih);
    x1 = xp + h * h * h * h * (1.0 / 24.0) * a2 + h * h * h * h * h * (1.0 / 120.0) * a3;
    v1 = vp + h * h * h * (1.0 / 6.0) * a2 + h * h * h * h * (1.0 / 24.0) * a3;
}

// 2^e, exactly, for e in [-1022, 1023].
__device__ __forceinline__ double pow2i(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// 1/h: for h a positive normal power of two (with a normal reciprocal) the exact reciprocal
// from the exponent bits, which is what the division gives; the division otherwise.
__device__ __forceinline__ double recip_pow2(double h)
{
    const long long b = __double_as_longlong(h);
    const long long ex = b >> 52;  // sign 0 and biased exponent
    if ((b & 0x000FFFFFFFFFFFFFLL) == 0 && ex >= 1 && ex <= 2045)
        return __longlong_as_double(0x7FE0000000000000LL - b);
    return 1.0 / h;
}

// ---- state records of the predict-on-load irregular force ---------------------------------
//   FP64 : 4 dvec4  {x, y, z, t_last} {vx, vy, vz, m} {ax, ay, az, 0} {jx, jy, jz, 0}
//   mixed: 5 float4 {xh, yh, zh, m} {xl, yl, zl, t_hi} {vx, vy, vz, t_lo} {ax, ay, az, 0}
//                   {jx, jy, jz, 0}
// (positions and t_last as hi/lo pairs of floats). Written for all particles by the packing
// kernel, and for the particles it corrects by the integrator's corrector.
__device__ __forceinline__ void pack_state_one(int64_t i, const double *X, const double *V, const double *A,
                                               const double *J, double t_last, double m, dvec4 *s64, float4 *s32)
{
    if (s64) {
        s64[4 * i] = make_dvec4(X[0], X[1], X[2], t_last);
        s64[4 * i + 1] = make_dvec4(V[0], V[1], V[2], m);
        s64[4 * i + 2] = make_dvec4(A[0], A[1], A[2], 0.0);
        s64[4 * i + 3] = make_dvec4(J[0], J[1], J[2], 0.0);
    } else {
        float h[3], l[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            h[c] = __double2float_rn(X[c]);
            l[c] = __double2float_rn(__dsub_rn(X[c], (double)h[c]));
        }
        const float th = __double2float_rn(t_last);
        const float tlo = __double2float_rn(__dsub_rn(t_last, (double)th));
        s32[5 * i] = make_float4(h[0], h[1], h[2], __double2float_rn(m));
        s32[5 * i + 1] = make_float4(l[0], l[1], l[2], th);
        s32[5 * i + 2] = make_float4(__double2float_rn(V[0]), __double2float_rn(V[1]), __double2float_rn(V[2]), tlo);
        s32[5 * i + 3] = make_float4(__double2float_rn(A[0]), __double2float_rn(A[1]), __double2float_rn(A[2]), 0.f);
        s32[5 * i + 4] = make_float4(__double2float_rn(J[0]), __double2float_rn(J[1]), __double2float_rn(J[2]), 0.f);
    }
}

// ---- one FP64 pair --------------------------------------------------------------------------
// p0 = {x_j, m_j}, p1 = {v_j, -} (predicted), xi, vi the predicted active particle:
// acc[0..2] += m r/|r|^3 ; acc[3..5] += m (w - 3 (r.w) r/|r|^2)/|r|^3 ; acc[6] -= m/|r|
__device__ __forceinline__ double pair_f64(const dvec4 &p0, const dvec4 &p1, const double (&xi)[3],
                                           const double (&vi)[3], bool self, double *acc)
{
    const double rx = __dsub_rn(p0.x, xi[0]), ry = __dsub_rn(p0.y, xi[1]), rz = __dsub_rn(p0.z, xi[2]);
    const double r2 = r2_f64(rx, ry, rz);
    const double rinv = self ? 0.0 : rsqrt(r2);
    const double wx = p1.x - vi[0], wy = p1.y - vi[1], wz = p1.z - vi[2];
    const double rw = rx * wx + ry * wy + rz * wz;
    const double rinv2 = rinv * rinv;
    const double mr = p0.w * rinv;
    const double mr3 = mr * rinv2;
    const double beta = -3.0 * rw * rinv2;
    acc[0] += mr3 * rx;
    acc[1] += mr3 * ry;
    acc[2] += mr3 * rz;
    acc[3] += mr3 * (wx + beta * rx);
    acc[4] += mr3 * (wy + beta * ry);
    acc[5] += mr3 * (wz + beta * rz);
    acc[6] -= mr;
    return r2;
}

// ---- warp reductions ---------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace nbgpu
