// predict.cu — K1: FP64 Hermite predictor of all particles and the packing of the
// j-records the force kernels stream (paper Sec. 3.3.3; the predictor is the Taylor
// series to the jerk term of the fourth-order Hermite scheme, Sec. 2).
//
// 112 B read (x, v, a, jerk: 4 x 24 B; t_last, m: 16 B) and 48 B (predicted x_p, v_p) +
// 64 B or 48 B (j-record) written per particle.  On GB300 the FP64 pipe (1/64 of the FP32
// rate), not HBM, bounds the kernel: its 18 FP64 operations are the Taylor terms; the mixed
// record's hi/lo split and every FP64 -> FP32 rounding in it are done with integer
// operations (split_ds, f64_to_f32_rn), off the FP64 pipe.
#include "nb_common.cuh"
#include "nb_kernels.cuh"

namespace nbgpu {

// The predictor is hermite_taylor (nb_common.cuh).  Its operation order is fixed, so every
// replica of the state predicts bit-identically; against a term-by-term evaluation the
// results agree to a few units in the last place.

// FP64 -> FP32 rounding to nearest, ties to even, with integer operations.  For a value whose
// float exponent is normal (FP64 biased exponent 897..1150) the 29 discarded mantissa bits
// are rounded into the kept 23 by one 64-bit add (2^28 - 1 plus the kept last bit: a carry
// out of the discarded bits happens exactly when they exceed half an ulp, or equal it with an
// odd last bit); a carry that runs into the exponent is the correct result too, unless it
// overflows the float range.  Signed zero is assembled directly; everything else (float
// subnormals, overflow, infinities, NaN) takes the conversion instruction.  The result is
// the bits of __double2float_rn(x) for every input.
__device__ __forceinline__ float f64_to_f32_rn(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const unsigned long long r = b + (0x0FFFFFFFull + ((b >> 29) & 1ull));
    const int e = (int)((b >> 52) & 0x7FF), er = (int)((r >> 52) & 0x7FF);
    if (e >= 897 && e <= 1150 && er <= 1150)
        return __uint_as_float(sign | ((unsigned)(er - 896) << 23) | ((unsigned)(r >> 29) & 0x7FFFFFu));
    if ((b << 1) == 0) return __uint_as_float(sign);
    return __double2float_rn(x);
}

// Double-single split x = hi + lo for the mixed j-record, with integer operations only for a
// value whose float exponent is normal (FP64 biased exponent 897..1150).  hi is x with its 29
// low mantissa bits cleared, so hi is exactly a float (exponent rebiased from 1023 to 127, top
// 23 mantissa bits) and x - hi = L 2^(e-1075) exactly, L being those 29 bits: lo is L rounded
// to 24 significant bits (to nearest, ties to even), its exponent from the leading bit of L,
// and the sign of x (+0 when L = 0, as the FP64 subtraction gives); a rounding carry to
// 2^24 steps the exponent by the add that assembles the bits.  |x - (hi + lo)| <= 2^-48 |x|.
// The bits are those of hi = (float)(x with the low bits cleared), lo = (float)(x - hi).
// Zero, values outside that range and a lo below the normal float range take the FP64
// subtraction and conversions.
__device__ __forceinline__ void split_ds(double x, float &hi, float &lo)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const unsigned L = (unsigned)b & 0x1FFFFFFFu;
    const int p = 31 - __clz(L);  // leading bit of L (-1 when L = 0)
    const int fe = e - 948 + p;   // biased float exponent of lo
    if (e >= 897 && e <= 1150 && (L == 0 || fe >= 1)) {
        hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | ((unsigned)(b >> 29) & 0x7FFFFFu));
        if (L == 0) {
            lo = 0.f;
        } else {
            unsigned q;
            if (p <= 23) {
                q = L << (23 - p);
            } else {
                const int sh = p - 23;
                q = (L + ((1u << (sh - 1)) - 1u) + ((L >> sh) & 1u)) >> sh;
            }
            lo = __uint_as_float(sign + ((unsigned)(fe - 1) << 23) + q);
        }
    } else {
        const double xh = __longlong_as_double((long long)(b & ~0x1FFFFFFFull));
        hi = __double2float_rn(xh);
        lo = __double2float_rn(__dsub_rn(x, xh));
    }
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
        rec32[3 * i] = make_float4(xh, yh, zh, f64_to_f32_rn(m));
        rec32[3 * i + 1] = make_float4(xl, yl, zl, 0.f);
        rec32[3 * i + 2] = make_float4(f64_to_f32_rn(vx), f64_to_f32_rn(vy), f64_to_f32_rn(vz), 0.f);
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
