// predict.cu — K1: FP64 Hermite predictor of all particles and the packing of the
// j-records the force kernels stream (paper Sec. 3.3.3; the predictor is the Taylor
// series to the jerk term of the fourth-order Hermite scheme, Sec. 2).
//
// 112 B read (x, v, a, jerk: 4 x 24 B; t_last, m: 16 B) and 48 B (predicted x_p, v_p) +
// 64 B or 48 B (j-record) written per particle.  On GB300 the FP64 pipe (1/64 of the FP32
// rate), not HBM, bounds the kernel: 18 FP64 operations of Taylor terms and, for the mixed
// record, 10 more for the hi/lo split and the conversions.
#include "nb_common.cuh"
#include "nb_kernels.cuh"

namespace nbgpu {

// The predictor is hermite_taylor (nb_common.cuh).  Its operation order is fixed, so every
// replica of the state predicts bit-identically; against a term-by-term evaluation the
// results agree to a few units in the last place.

// Double-single split x = hi + lo for the mixed j-record.  hi is x with its 29 low mantissa
// bits cleared, so x - hi is exact in FP64 and hi is exactly a float: its bits are assembled
// with integer operations (exponent rebiased from 1023 to 127, top 23 mantissa bits) and only
// lo takes an FP64 subtraction and one rounding to FP32 (|x - (hi + lo)| <= 2^-48 |x|).  On
// GB300 the FP64 pipe, not HBM, bounds the predictor, and this split takes two FP64
// operations a coordinate instead of four.  Zero and values outside the normal float range
// take the conversion itself.
__device__ __forceinline__ void split_ds(double x, float &hi, float &lo)
{
    const long long b = __double_as_longlong(x);
    const double xh = __longlong_as_double(b & ~0x1FFFFFFFLL);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e >= 897 && e <= 1150)
        hi = __uint_as_float((unsigned)((b >> 32) & 0x80000000LL) | ((unsigned)(e - 896) << 23) |
                             (unsigned)((b >> 29) & 0x7FFFFF));
    else
        hi = __double2float_rn(xh);
    lo = __double2float_rn(__dsub_rn(x, xh));
}

__device__ __forceinline__ void write_records(int64_t i, double x, double y, double z, double vx,
                                              double vy, double vz, double m, dvec4 *rec64,
                                              float4 *rec32)
{
    if (rec64) {
        rec64[2 * i] = make_dvec4(x, y, z, m);
        rec64[2 * i + 1] = make_dvec4(vx, vy, vz, 0.0);
    }
    if (rec32) {
        float xh, yh, zh, xl, yl, zl;
        split_ds(x, xh, xl);
        split_ds(y, yh, yl);
        split_ds(z, zh, zl);
        rec32[3 * i] = make_float4(xh, yh, zh, __double2float_rn(m));
        rec32[3 * i + 1] = make_float4(xl, yl, zl, 0.f);
        rec32[3 * i + 2] = make_float4(__double2float_rn(vx), __double2float_rn(vy),
                                       __double2float_rn(vz), 0.f);
    }
}

__device__ __forceinline__ void write_pad(int64_t i, dvec4 *rec64, float4 *rec32)
{
    if (rec64) {
        rec64[2 * i] = make_dvec4(kPadPos, kPadPos, kPadPos, 0.0);
        rec64[2 * i + 1] = make_dvec4(0.0, 0.0, 0.0, 0.0);
    }
    if (rec32) {
        rec32[3 * i] = make_float4(kPadPos, kPadPos, kPadPos, 0.f);
        rec32[3 * i + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        rec32[3 * i + 2] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__global__ void k_predict(int64_t n, int64_t n_pad, double t, const double *__restrict__ x,
                          const double *__restrict__ v, const double *__restrict__ a,
                          const double *__restrict__ jk, const double *__restrict__ tl,
                          const double *__restrict__ m, double *__restrict__ xp,
                          double *__restrict__ vp, dvec4 *__restrict__ rec64,
                          float4 *__restrict__ rec32)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_pad;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i >= n) {
            write_pad(i, rec64, rec32);
            continue;
        }
        const double dt = __dsub_rn(t, tl[i]);
        double p[3], q[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) hermite_taylor(x[3 * i + c], v[3 * i + c], a[3 * i + c], jk[3 * i + c], dt, p[c], q[c]);
        if (xp) {  // null when only the records are wanted
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xp[3 * i + c] = p[c];
                vp[3 * i + c] = q[c];
            }
        }
        write_records(i, p[0], p[1], p[2], q[0], q[1], q[2], m[i], rec64, rec32);
    }
}

__global__ void k_pack(int64_t n, int64_t n_pad, const double *__restrict__ xp,
                       const double *__restrict__ vp, const double *__restrict__ m,
                       dvec4 *__restrict__ rec64, float4 *__restrict__ rec32)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_pad;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i >= n) {
            write_pad(i, rec64, rec32);
            continue;
        }
        write_records(i, xp[3 * i], xp[3 * i + 1], xp[3 * i + 2], vp[3 * i], vp[3 * i + 1],
                      vp[3 * i + 2], m[i], rec64, rec32);
    }
}

static int grid_for(int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    if (g > 152 * 32) g = 152 * 32;
    return g < 1 ? 1 : (int)g;
}

void launch_predict(cudaStream_t st, int64_t n, int64_t n_pad, double t, const double *x,
                    const double *v, const double *a, const double *jk, const double *tl,
                    const double *m, double *xp, double *vp, void *rec64, void *rec32)
{
    k_predict<<<grid_for(n_pad, 256), 256, 0, st>>>(n, n_pad, t, x, v, a, jk, tl, m, xp, vp,
                                                    (dvec4 *)rec64, (float4 *)rec32);
}

void launch_pack_predicted(cudaStream_t st, int64_t n, int64_t n_pad, const double *xp,
                           const double *vp, const double *m, void *rec64, void *rec32)
{
    k_pack<<<grid_for(n_pad, 256), 256, 0, st>>>(n, n_pad, xp, vp, m, (dvec4 *)rec64,
                                                 (float4 *)rec32);
}

}  // namespace nbgpu
