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

// ---- cp.async (LDGSTS) staging of j-tiles into shared memory ---------------------------
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ---- the neighbour-test distances ------------------------------------------------------
// Both are written with explicit round-to-nearest intrinsics so that every kernel that
// decides "j is a neighbour of i" (the force kernels and the ordered recompute of
// over-full lists) obtains bit-identical r^2 values.

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

// ---- warp reductions ---------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace nbgpu
