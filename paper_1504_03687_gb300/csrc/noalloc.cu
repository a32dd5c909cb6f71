// noalloc.cu — nb_regular_force_noalloc: the regular force, jerk and potential of a small
// active block computed without allocating any device memory.
//
// Some callers cannot allocate device memory while they integrate: a host code whose own
// memory manager owns the whole device, or a time-step loop that must never reach
// cudaMalloc/cudaFree (they can synchronise the device and stall every stream).  This
// entry point needs no context: the caller passes the predicted state, the active list and
// the output buffers, all in device memory, and the only scratch it uses — the per-split
// partial sums — lives in a fixed file-scope device array that every GPU loading the
// library keeps until the process exits.
//
// Work decomposition: the FP64 j-streamed kernel (every CTA owns a contiguous chunk of the
// n sources for a batch of up to IB active rows; every warp walks 32 consecutive sources
// per step) reading the caller's FP64 arrays directly, followed by the fixed-order
// reduction of the partial sums.  Neighbour lists are not produced here.
// Layout: the caller's arrays are interleaved row-major (n,3) positions and velocities and
// (n) masses, read as they are (no repacking, which would need scratch): lane j loads the
// three components of particle j at a 24-byte stride, so a warp's loads of one component
// touch 768 contiguous bytes shared by the three component loads (about 3x the sectors of
// a component-major layout per instruction; the kernel is FP64-pipe bound, not load bound).
#include <mutex>

#include "nbgpu.h"
#include "nb_common.cuh"
#include "nb_kernels.cuh"

namespace nbgpu {

// 4 MiB of partial sums: [splits][7][n_i] doubles, so 7 * splits * n_i <= kNoallocDoubles.
constexpr int64_t kNoallocDoubles = int64_t(1) << 19;
constexpr int64_t kNoallocMaxRows = 65536;
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoallocDoubles];

// Device address of g_noalloc_partials per device, looked up with that device current and
// kept once the lookup has succeeded (a failed lookup is retried by the next call).
static double *g_scratch_ptr[kNoallocMaxDevices];
static std::mutex g_scratch_mutex;

template <int IB, int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    k_force_fp64_aos_jstream(int64_t n, const double *__restrict__ xp, const double *__restrict__ vp,
                             const double *__restrict__ m, const int32_t *__restrict__ idx, int64_t n_i, int S,
                             double *__restrict__ part)
{
    constexpr int W = BLOCK / 32;
    __shared__ double red[W][IB][7];
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int s = blockIdx.y;
    const int64_t k0 = (int64_t)blockIdx.x * IB;
    const int64_t j0 = (n * s) / S, j1 = (n * (s + 1)) / S;
    const int64_t w0 = j0 + ((j1 - j0) * w) / W, w1 = j0 + ((j1 - j0) * (w + 1)) / W;
    double xi[IB][3], vi[IB][3];
    int64_t gi[IB];
#pragma unroll
    for (int q = 0; q < IB; ++q) {
        int64_t g = -1;
        if (k0 + q < n_i) {
            g = idx[k0 + q];
            if (g < 0 || g >= n) g = -1;  // out-of-range rows come out as zeros
        }
        gi[q] = g;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xi[q][c] = g >= 0 ? xp[3 * g + c] : 0.0;
            vi[q][c] = g >= 0 ? vp[3 * g + c] : 0.0;
        }
    }
    double acc[IB][7];
#pragma unroll
    for (int q = 0; q < IB; ++q)
#pragma unroll
        for (int c = 0; c < 7; ++c) acc[q][c] = 0.0;
    for (int64_t j = w0 + lane; j < w1; j += 32) {
        const double xj = xp[3 * j], yj = xp[3 * j + 1], zj = xp[3 * j + 2];
        const double ux = vp[3 * j], uy = vp[3 * j + 1], uz = vp[3 * j + 2];
        const double mj = m[j];
#pragma unroll
        for (int q = 0; q < IB; ++q) {
            const double rx = xj - xi[q][0], ry = yj - xi[q][1], rz = zj - xi[q][2];
            const double r2 = r2_f64(rx, ry, rz);
            const double rinv = (j == gi[q]) ? 0.0 : rsqrt(r2);
            const double wx = ux - vi[q][0], wy = uy - vi[q][1], wz = uz - vi[q][2];
            const double rw = rx * wx + ry * wy + rz * wz;
            const double rinv2 = rinv * rinv;
            const double mr = mj * rinv;
            const double mr3 = mr * rinv2;
            const double beta = -3.0 * rw * rinv2;
            acc[q][0] += mr3 * rx;
            acc[q][1] += mr3 * ry;
            acc[q][2] += mr3 * rz;
            acc[q][3] += mr3 * (wx + beta * rx);
            acc[q][4] += mr3 * (wy + beta * ry);
            acc[q][5] += mr3 * (wz + beta * rz);
            acc[q][6] -= mr;
        }
    }
#pragma unroll
    for (int q = 0; q < IB; ++q)
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            const double v = warp_sum(acc[q][c]);
            if (lane == 0) red[w][q][c] = v;
        }
    __syncthreads();
    for (int e = tid; e < IB * 7; e += BLOCK) {
        const int q = e / 7, c = e % 7;
        if (k0 + q < n_i) {
            double sum = 0.0;
#pragma unroll
            for (int ww = 0; ww < W; ++ww) sum += red[ww][q][c];
            part[((int64_t)s * 7 + c) * n_i + k0 + q] = gi[q] >= 0 ? sum : 0.0;
        }
    }
}

static void set_msg(char *err, int32_t err_len, const char *msg)
{
    if (!err || err_len <= 0) return;
    int32_t q = 0;
    for (; q < err_len - 1 && msg[q]; ++q) err[q] = msg[q];
    err[q] = 0;
}

}  // namespace nbgpu

using namespace nbgpu;

extern "C" nb_status nb_regular_force_noalloc(int64_t n, const double *xp, const double *vp, const double *m,
                                              int64_t n_i, const int32_t *idx, double *acc, double *jerk,
                                              double *pot, void *stream, char *err, int32_t err_len)
{
    set_msg(err, err_len, "");
    if (n < 1 || n > (int64_t)INT32_MAX || n_i < 0) {
        set_msg(err, err_len, "nb_regular_force_noalloc: n must be in [1, 2^31-1] and n_i >= 0");
        return NB_ERR_ARG;
    }
    if (n_i > kNoallocMaxRows) {
        set_msg(err, err_len, "nb_regular_force_noalloc: n_i exceeds the 65536 active rows its fixed 4 MiB "
                              "scratch holds; use nb_regular_force for larger blocks");
        return NB_ERR_ARG;
    }
    if (n_i == 0) return NB_OK;
    if (!xp || !vp || !m || !idx || !acc || !jerk || !pot) {
        set_msg(err, err_len, "nb_regular_force_noalloc: null array");
        return NB_ERR_ARG;
    }
    // an error left pending by earlier work on this thread is reported as such and left in
    // place for its owner (cudaGetLastError below must only see this call's launches)
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        set_msg(err, err_len, "nb_regular_force_noalloc: a CUDA error was pending before the call (nothing run)");
        return NB_ERR_CUDA;
    }
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) {
        set_msg(err, err_len, "nb_regular_force_noalloc: no usable current CUDA device");
        return NB_ERR_CUDA;
    }
    // set-up on this device (the device is current): the scratch array's address, looked up
    // by the first call that succeeds in doing so and kept from then on
    double *part = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_partials);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();  // clear the lookup's own error; the next call retries
                set_msg(err, err_len, "nb_regular_force_noalloc: cudaGetSymbolAddress of the scratch array failed");
                return NB_ERR_CUDA;
            }
            g_scratch_ptr[dev] = static_cast<double *>(p);
        }
        part = g_scratch_ptr[dev];
    }
    int sms = 152;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 152;
    constexpr int IB = 4, BLOCK = 256;
    const int64_t batches = (n_i + IB - 1) / IB;
    int64_t S = (4 * (int64_t)sms + batches - 1) / batches;
    const int64_t s_mem = kNoallocDoubles / (7 * n_i);
    const int64_t s_len = n / 1024 > 1 ? n / 1024 : 1;
    if (S > s_mem) S = s_mem;
    if (S > s_len) S = s_len;
    if (S < 1) S = 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // every partial slot the reduction reads is written by this launch: nothing in the
    // shared scratch has to start at zero
    k_force_fp64_aos_jstream<IB, BLOCK><<<dim3((unsigned)batches, (unsigned)S), BLOCK, 0, st>>>(
        n, xp, vp, m, idx, n_i, (int)S, part);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_msg(err, err_len, cudaGetErrorString(e));
        return NB_ERR_CUDA;
    }
    launch_reduce(st, part, (int)S, n_i, acc, jerk, pot);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_msg(err, err_len, cudaGetErrorString(e));
        return NB_ERR_CUDA;
    }
    return NB_OK;
}
