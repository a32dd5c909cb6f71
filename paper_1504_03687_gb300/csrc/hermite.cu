// hermite.cu — the Hermite predictor and corrector over caller arrays, and their
// vector-Jacobian products (paper Sec. 2: the fourth-order Hermite scheme, after Makino 1991;
// Sec. 3.3.3: prediction).  They serve the differentiable block-step integration: a chain of
// block steps is predictor -> regular force -> corrector, and its gradient runs the three VJPs
// in reverse.  Every array is a device array; every kernel is one elementwise pass.
//
//   predictor : dt = t - t_last;  xp = x + dt (v + dt/2 (a + dt/3 j)),  vp = v + dt (a + dt/2 j)
//               (hermite_taylor: the same function and operation order as nb_predict)
//   its VJP   : g_x = g_xp,  g_v = dt g_xp + g_vp,  g_a = dt^2/2 g_xp + dt g_vp,
//               g_j = dt^3/6 g_xp + dt^2/2 g_vp   (t and t_last are not differentiated)
//   corrector : h = t - t_last;  hermite_correct per component
//   its VJP   : the corrector is linear in (xp, vp, a0, j0, a1, j1):
//               x1 = xp - 3h^2/20 a0 - 7h^3/60 j0 + 3h^2/20 a1 - h^3/30 j1
//               v1 = vp - h/2 a0 - 5h^2/12 j0 + h/2 a1 - h^2/12 j1
//               so g_xp = g_x1, g_vp = g_v1, g_a0 = -3h^2/20 g_x1 - h/2 g_v1,
//               g_j0 = -7h^3/60 g_x1 - 5h^2/12 g_v1, g_a1 = -g_a0, g_j1 = -h^3/30 g_x1 - h^2/12 g_v1.
// Compiled without FMA contraction (the corrector follows the plain definition's order).
#include "nb_common.cuh"
#include "nb_kernels.cuh"

namespace nbgpu {

__global__ void k_hermite_predict(int64_t n, double t, const double *__restrict__ x, const double *__restrict__ v,
                                  const double *__restrict__ a, const double *__restrict__ j,
                                  const double *__restrict__ tl, double *__restrict__ xp, double *__restrict__ vp)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < 3 * n; q += (int64_t)gridDim.x * blockDim.x) {
        const double dt = t - tl[q / 3];
        hermite_taylor(x[q], v[q], a[q], j[q], dt, xp[q], vp[q]);
    }
}

__global__ void k_hermite_predict_vjp(int64_t n, double t, const double *__restrict__ tl,
                                      const double *__restrict__ gxp, const double *__restrict__ gvp,
                                      double *__restrict__ gx, double *__restrict__ gv, double *__restrict__ ga,
                                      double *__restrict__ gj)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < 3 * n; q += (int64_t)gridDim.x * blockDim.x) {
        const double dt = t - tl[q / 3];
        const double h2 = dt * dt / 2.0, h3 = dt * dt * dt / 6.0;
        const double X = gxp[q], V = gvp[q];
        gx[q] = X;
        gv[q] = dt * X + V;
        ga[q] = h2 * X + dt * V;
        gj[q] = h3 * X + h2 * V;
    }
}

__global__ void k_hermite_correct(int64_t n, double t, const double *__restrict__ tl, const double *__restrict__ xp,
                                  const double *__restrict__ vp, const double *__restrict__ a0,
                                  const double *__restrict__ j0, const double *__restrict__ a1,
                                  const double *__restrict__ j1, double *__restrict__ x1, double *__restrict__ v1)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < 3 * n; q += (int64_t)gridDim.x * blockDim.x) {
        const double h = t - tl[q / 3];
        double a2, a3;
        hermite_correct(xp[q], vp[q], a0[q], j0[q], a1[q], j1[q], h, x1[q], v1[q], a2, a3);
    }
}

__global__ void k_hermite_correct_vjp(int64_t n, double t, const double *__restrict__ tl,
                                      const double *__restrict__ gx1, const double *__restrict__ gv1,
                                      double *__restrict__ gxp, double *__restrict__ gvp, double *__restrict__ ga0,
                                      double *__restrict__ gj0, double *__restrict__ ga1, double *__restrict__ gj1)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < 3 * n; q += (int64_t)gridDim.x * blockDim.x) {
        const double h = t - tl[q / 3];
        const double X = gx1[q], V = gv1[q];
        const double h2 = h * h, h3 = h2 * h;
        const double da0 = -3.0 * h2 / 20.0 * X - h / 2.0 * V;
        gxp[q] = X;
        gvp[q] = V;
        ga0[q] = da0;
        gj0[q] = -7.0 * h3 / 60.0 * X - 5.0 * h2 / 12.0 * V;
        ga1[q] = -da0;
        gj1[q] = -h3 / 30.0 * X - h2 / 12.0 * V;
    }
}

static unsigned hermite_grid(int64_t n)
{
    int64_t g = (3 * n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    return (unsigned)(g > 0 ? g : 1);
}

void launch_hermite_predict(cudaStream_t st, int64_t n, double t, const double *x, const double *v, const double *a,
                            const double *j, const double *tl, double *xp, double *vp)
{
    k_hermite_predict<<<hermite_grid(n), 256, 0, st>>>(n, t, x, v, a, j, tl, xp, vp);
}

void launch_hermite_predict_vjp(cudaStream_t st, int64_t n, double t, const double *tl, const double *gxp,
                                const double *gvp, double *gx, double *gv, double *ga, double *gj)
{
    k_hermite_predict_vjp<<<hermite_grid(n), 256, 0, st>>>(n, t, tl, gxp, gvp, gx, gv, ga, gj);
}

void launch_hermite_correct(cudaStream_t st, int64_t n, double t, const double *tl, const double *xp, const double *vp,
                            const double *a0, const double *j0, const double *a1, const double *j1, double *x1,
                            double *v1)
{
    k_hermite_correct<<<hermite_grid(n), 256, 0, st>>>(n, t, tl, xp, vp, a0, j0, a1, j1, x1, v1);
}

void launch_hermite_correct_vjp(cudaStream_t st, int64_t n, double t, const double *tl, const double *gx1,
                                const double *gv1, double *gxp, double *gvp, double *ga0, double *gj0, double *ga1,
                                double *gj1)
{
    k_hermite_correct_vjp<<<hermite_grid(n), 256, 0, st>>>(n, t, tl, gx1, gv1, gxp, gvp, ga0, gj0, ga1, gj1);
}

}  // namespace nbgpu
