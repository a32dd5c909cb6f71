/*
 * nb_oracle.c — plain FP64 CPU oracle for the regular-force step of NBODY6++GPU
 * (Wang et al. 2015, MNRAS 450, 4070).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * loads this file; only the tests, the package smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or helper with the
 * CUDA path.
 *
 * What it computes, and where the paper defines it:
 *  - Position/velocity prediction of all particles to the block time
 *    (Sec. 3.3.3 "Position and velocity prediction"; the Taylor form itself is
 *    not printed in the paper — it is the standard Hermite predictor the paper
 *    cites in Sec. 2, Makino 1991).
 *  - The regular force: for every active particle i, acceleration, its time
 *    derivative (jerk) and potential summed over all other particles, plus the
 *    list of neighbours inside r_s (Sec. 2, Ahmad-Cohen scheme; Sec. 3.2.1,
 *    "Regular force and potential (GPU)"; Table 2 gives the O(N_i N) cost).
 *    The sums here run over ALL j != i: the split into inside/outside r_s is a
 *    subtraction by the consumer (the paper names the regular force as the part
 *    from outside r_s; the all-j sum is what Newton's third law pins).
 *  - Its vector-Jacobian product (adjoint), obtained by differentiating the sums.
 *  - A fourth-order Hermite integrator with hierarchical power-of-two block
 *    steps (Sec. 2; the corrector and the Aarseth step criterion are the
 *    textbook forms of Makino 1991 / Makino & Aarseth 1992, which the paper
 *    cites but does not print).
 *  - Kinetic and potential energy (Sec. 3.3.2 needs W for N-body scaling).
 *  - The irregular force: the same sums over each active particle's neighbour list,
 *    with i and its neighbours predicted from their Hermite state (Sec. 2, Ahmad-Cohen;
 *    Sec. 3.2.2 and Sec. 3.3.3, neighbour-only prediction).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no ISA intrinsics).
 * Loops over j run in ascending index order; OpenMP only splits the outer loop
 * over independent outputs, so every result is bitwise reproducible.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Hermite predictor (Taylor series to the jerk term) for all n particles:
 *   dt  = t - t_last
 *   x_p = x + v dt + a dt^2/2 + jerk dt^3/6
 *   v_p = v + a dt + jerk dt^2/2
 * Arrays are row-major (n,3); t_last is (n). */
void orc_predict(int64_t n, double t, const double *x, const double *v, const double *a,
                 const double *jk, const double *t_last, double *xp, double *vp)
{
    for (int64_t i = 0; i < n; ++i) {
        const double dt = t - t_last[i];
        for (int c = 0; c < 3; ++c) {
            const int64_t q = 3 * i + c;
            xp[q] = x[q] + v[q] * dt + a[q] * dt * dt / 2.0 + jk[q] * dt * dt * dt / 6.0;
            vp[q] = v[q] + a[q] * dt + jk[q] * dt * dt / 2.0;
        }
    }
}

/* Regular force, jerk and potential of the active particles idx[0..n_i) from all
 * n predicted particles, with neighbour lists.
 *
 * For active i and every j != i (j ascending):
 *   r = x_j - x_i,  w = v_j - v_i,  r2 = r.r
 *   acc_i  += m_j r / |r|^3
 *   jerk_i += m_j [ w / |r|^3 - 3 (r.w) r / |r|^5 ]
 *   pot_i  -= m_j / |r|
 *   j is a neighbour of i iff r2 < rs2_i.
 * Output row k belongs to idx[k].  nb_list is (n_i, cap): the first cap
 * neighbours in ascending j; nb_count[k] is the true count (may exceed cap).
 * rs2 is (n_i) or, with rs2_scalar != 0, a single value.  nb_list may be NULL
 * (counts only).  Returns 0, or -1 on an index outside [0, n). */
int orc_regular_force(int64_t n, const double *xp, const double *vp, const double *m,
                      int64_t n_i, const int32_t *idx, const double *rs2, int rs2_scalar,
                      double *acc, double *jerk, double *pot,
                      int32_t *nb_count, int32_t *nb_list, int32_t cap)
{
    for (int64_t k = 0; k < n_i; ++k)
        if (idx[k] < 0 || idx[k] >= n) return -1;

#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < n_i; ++k) {
        const int64_t i = idx[k];
        const double rs2_i = rs2_scalar ? rs2[0] : rs2[k];
        double ax = 0, ay = 0, az = 0, jx = 0, jy = 0, jz = 0, ph = 0;
        int32_t cnt = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            const double rx = xp[3 * j + 0] - xp[3 * i + 0];
            const double ry = xp[3 * j + 1] - xp[3 * i + 1];
            const double rz = xp[3 * j + 2] - xp[3 * i + 2];
            const double wx = vp[3 * j + 0] - vp[3 * i + 0];
            const double wy = vp[3 * j + 1] - vp[3 * i + 1];
            const double wz = vp[3 * j + 2] - vp[3 * i + 2];
            const double r2 = rx * rx + ry * ry + rz * rz;
            const double rinv = 1.0 / sqrt(r2);
            const double rinv2 = rinv * rinv;
            const double mr3 = m[j] * rinv * rinv2;
            const double rw = rx * wx + ry * wy + rz * wz;
            ax += mr3 * rx;
            ay += mr3 * ry;
            az += mr3 * rz;
            jx += mr3 * (wx - 3.0 * rw * rinv2 * rx);
            jy += mr3 * (wy - 3.0 * rw * rinv2 * ry);
            jz += mr3 * (wz - 3.0 * rw * rinv2 * rz);
            ph -= m[j] * rinv;
            if (r2 < rs2_i) {
                if (nb_list && cnt < cap) nb_list[k * (int64_t)cap + cnt] = (int32_t)j;
                ++cnt;
            }
        }
        acc[3 * k + 0] = ax;  acc[3 * k + 1] = ay;  acc[3 * k + 2] = az;
        jerk[3 * k + 0] = jx; jerk[3 * k + 1] = jy; jerk[3 * k + 2] = jz;
        pot[k] = ph;
        if (nb_count) nb_count[k] = cnt;
    }
    return 0;
}

/* Per-pair adjoint terms.  For the loss contribution of pair (i, j),
 *   L_ij = m_j [ g_a.r/|r|^3 + g_j.w/|r|^3 - 3 (r.w)(g_j.r)/|r|^5 - g_p/|r| ],
 * with cotangents (g_a, g_j, g_p) of (acc_i, jerk_i, pot_i), this returns
 *   dr = dL_ij/dr,  dw = dL_ij/dw,  dm = dL_ij/dm_j. */
static void pair_adjoint(double rx, double ry, double rz, double wx, double wy, double wz, double mj,
                         const double *ga, const double *gj, double gp,
                         double *dr, double *dw, double *dm)
{
    const double r2 = rx * rx + ry * ry + rz * rz;
    const double rinv = 1.0 / sqrt(r2);
    const double rinv2 = rinv * rinv;
    const double rinv3 = rinv * rinv2;
    const double rinv5 = rinv3 * rinv2;
    const double rinv7 = rinv5 * rinv2;
    const double q = rx * wx + ry * wy + rz * wz;        /* r.w   */
    const double ar = ga[0] * rx + ga[1] * ry + ga[2] * rz; /* g_a.r */
    const double jr = gj[0] * rx + gj[1] * ry + gj[2] * rz; /* g_j.r */
    const double jw = gj[0] * wx + gj[1] * wy + gj[2] * wz; /* g_j.w */
    const double r[3] = {rx, ry, rz}, w[3] = {wx, wy, wz};
    for (int c = 0; c < 3; ++c) {
        /* d/dr of each term of L_ij */
        const double d_acc = ga[c] * rinv3 - 3.0 * ar * r[c] * rinv5;
        const double d_jw = -3.0 * jw * r[c] * rinv5;
        const double d_qjr = -3.0 * (w[c] * jr + q * gj[c]) * rinv5 + 15.0 * q * jr * r[c] * rinv7;
        const double d_pot = gp * r[c] * rinv3;
        dr[c] = mj * (d_acc + d_jw + d_qjr + d_pot);
        dw[c] = mj * (gj[c] * rinv3 - 3.0 * jr * r[c] * rinv5);
    }
    *dm = ar * rinv3 + jw * rinv3 - 3.0 * q * jr * rinv5 - gp * rinv;
}

/* Vector-Jacobian product of (acc, jerk, pot) over the active set w.r.t. the
 * predicted positions, velocities and masses of all n particles:
 *   L = sum_k g_acc[k].acc_k + g_jerk[k].jerk_k + g_pot[k] pot_k.
 * Since r = x_j - x_i and w = v_j - v_i:
 *   g_x[j] += dL_ij/dr,  g_x[i] -= dL_ij/dr   (same for v),  g_m[j] += dL_ij/dm_j.
 * The j-side sum (over active i) and the i-side sum (over all j) are two loops
 * over disjoint outputs.  g_x, g_v (n,3) and g_m (n) are overwritten. */
int orc_regular_force_vjp(int64_t n, const double *xp, const double *vp, const double *m,
                          int64_t n_i, const int32_t *idx,
                          const double *g_acc, const double *g_jerk, const double *g_pot,
                          double *g_x, double *g_v, double *g_m)
{
    for (int64_t k = 0; k < n_i; ++k)
        if (idx[k] < 0 || idx[k] >= n) return -1;
    /* j-side: particle j as the source of every active i's sums */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < n; ++j) {
        double gx[3] = {0, 0, 0}, gv[3] = {0, 0, 0}, gm = 0;
        for (int64_t k = 0; k < n_i; ++k) {
            const int64_t i = idx[k];
            if (i == j) continue;
            double dr[3], dw[3], dm;
            pair_adjoint(xp[3 * j] - xp[3 * i], xp[3 * j + 1] - xp[3 * i + 1], xp[3 * j + 2] - xp[3 * i + 2],
                         vp[3 * j] - vp[3 * i], vp[3 * j + 1] - vp[3 * i + 1], vp[3 * j + 2] - vp[3 * i + 2],
                         m[j], g_acc + 3 * k, g_jerk + 3 * k, g_pot[k], dr, dw, &dm);
            for (int c = 0; c < 3; ++c) { gx[c] += dr[c]; gv[c] += dw[c]; }
            gm += dm;
        }
        for (int c = 0; c < 3; ++c) { g_x[3 * j + c] = gx[c]; g_v[3 * j + c] = gv[c]; }
        g_m[j] = gm;
    }
    /* i-side: the active particle as the receiver */
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < n_i; ++k) {
        const int64_t i = idx[k];
        double gx[3] = {0, 0, 0}, gv[3] = {0, 0, 0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dr[3], dw[3], dm;
            pair_adjoint(xp[3 * j] - xp[3 * i], xp[3 * j + 1] - xp[3 * i + 1], xp[3 * j + 2] - xp[3 * i + 2],
                         vp[3 * j] - vp[3 * i], vp[3 * j + 1] - vp[3 * i + 1], vp[3 * j + 2] - vp[3 * i + 2],
                         m[j], g_acc + 3 * k, g_jerk + 3 * k, g_pot[k], dr, dw, &dm);
            for (int c = 0; c < 3; ++c) { gx[c] += dr[c]; gv[c] += dw[c]; }
        }
        for (int c = 0; c < 3; ++c) { g_x[3 * i + c] -= gx[c]; g_v[3 * i + c] -= gv[c]; }
    }
    return 0;
}

/* Kinetic and potential energy: K = 1/2 sum m v^2, W = -sum_{i<j} m_i m_j / r_ij. */
void orc_energy(int64_t n, const double *m, const double *x, const double *v, double *K, double *W)
{
    double k = 0.0, w = 0.0;
    for (int64_t i = 0; i < n; ++i)
        k += 0.5 * m[i] * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]);
#pragma omp parallel for reduction(+ : w) schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double wi = 0.0;
        for (int64_t j = i + 1; j < n; ++j) {
            const double rx = x[3 * j] - x[3 * i], ry = x[3 * j + 1] - x[3 * i + 1], rz = x[3 * j + 2] - x[3 * i + 2];
            wi -= m[i] * m[j] / sqrt(rx * rx + ry * ry + rz * rz);
        }
        w += wi;
    }
    *K = k;
    *W = w;
}

static double norm3(const double *a) { return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

/* Largest power of two (2^-k) not above dt_crit and not above dt_max. */
static double quantise_step(double dt_crit, double dt_max)
{
    double dt = dt_max;
    while (dt > dt_crit && dt > 1e-30) dt *= 0.5;
    return dt;
}

/* Fourth-order Hermite integration with hierarchical block time steps.
 *
 * Start: force and jerk of all particles at t = 0; dt_i = the largest power of
 * two below eta_s |a|/|jerk| (capped at dt_max).  Each block step: t_next =
 * min_i(t_i + dt_i); the active block is every i with t_i + dt_i == t_next; all
 * particles are predicted to t_next; the active ones get their new force and
 * jerk (a1, j1) from the predicted state and are corrected with
 *   a2 = [-6 (a0 - a1) - dt (4 j0 + 2 j1)] / dt^2,
 *   a3 = [12 (a0 - a1) + 6 dt (j0 + j1)] / dt^3,
 *   x1 = x_p + dt^4/24 a2 + dt^5/120 a3,   v1 = v_p + dt^3/6 a2 + dt^4/24 a3.
 * New step from the Aarseth criterion with the end-of-step derivatives
 * (a2' = a2 + dt a3):
 *   dt_crit = sqrt(eta (|a1||a2'| + |j1|^2) / (|j1||a3| + |a2'|^2)),
 * halved until not above dt_crit, or doubled when dt_crit >= 2 dt, t_next is a
 * multiple of 2 dt and 2 dt <= dt_max (block rule: steps are powers of 0.5).
 * With dt_fixed > 0 every particle takes that one step (shared time step).
 * x, v are advanced in place to t_end (all particles synchronised there).
 * stats (optional, 4 doubles): block steps, particle steps, pair evaluations, 0.
 * Returns 0, or -2 if max_blocks was reached. */
/* Optional schedule record / replay of hermite_core:
 *  record: t_next[b] and the active set act_idx[act_off[b] .. act_off[b+1]) of every block
 *          step b are stored (capacities cap_blocks, cap_act; -3 is returned when full);
 *  replay: the block times and active sets are taken from the arrays instead of the step
 *          criterion (a frozen schedule; the corrector still uses h = t_next - t_i). */
typedef struct {
    double *t_next;
    int64_t *act_off;
    int32_t *act_idx;
    int64_t cap_blocks, cap_act, n_blocks;
} orc_schedule;

static int hermite_core(int64_t n, const double *m, double *x, double *v, double t_end, double eta,
                        double eta_s, double dt_max, double dt_fixed, int64_t max_blocks, double *stats,
                        orc_schedule *record, const orc_schedule *replay);

int orc_hermite_run(int64_t n, const double *m, double *x, double *v, double t_end, double eta,
                    double eta_s, double dt_max, double dt_fixed, int64_t max_blocks, double *stats)
{
    return hermite_core(n, m, x, v, t_end, eta, eta_s, dt_max, dt_fixed, max_blocks, stats, NULL, NULL);
}

/* As orc_hermite_run, recording the schedule (see orc_schedule); *n_blocks receives its length. */
int orc_hermite_record(int64_t n, const double *m, double *x, double *v, double t_end, double eta,
                       double eta_s, double dt_max, int64_t max_blocks, double *t_next, int64_t *act_off,
                       int32_t *act_idx, int64_t cap_blocks, int64_t cap_act, int64_t *n_blocks)
{
    orc_schedule s = {t_next, act_off, act_idx, cap_blocks, cap_act, 0};
    const int rc = hermite_core(n, m, x, v, t_end, eta, eta_s, dt_max, 0.0, max_blocks, NULL, &s, NULL);
    *n_blocks = s.n_blocks;
    return rc;
}

/* Replay n_blocks recorded block steps from the state (x, v) at t = 0. */
int orc_hermite_replay(int64_t n, const double *m, double *x, double *v, int64_t n_blocks, const double *t_next,
                       const int64_t *act_off, const int32_t *act_idx)
{
    orc_schedule s = {(double *)t_next, (int64_t *)act_off, (int32_t *)act_idx, n_blocks, act_off[n_blocks],
                      n_blocks};
    return hermite_core(n, m, x, v, INFINITY, 0.0, 0.0, 1.0, 0.0, 0, NULL, NULL, &s);
}

static int hermite_core(int64_t n, const double *m, double *x, double *v, double t_end, double eta,
                        double eta_s, double dt_max, double dt_fixed, int64_t max_blocks, double *stats,
                        orc_schedule *record, const orc_schedule *replay)
{
    double *a = calloc(3 * n, sizeof(double)), *jk = calloc(3 * n, sizeof(double));
    double *xp = malloc(3 * n * sizeof(double)), *vp = malloc(3 * n * sizeof(double));
    double *t = calloc(n, sizeof(double)), *dt = malloc(n * sizeof(double));
    double *a1 = malloc(3 * n * sizeof(double)), *j1 = malloc(3 * n * sizeof(double));
    double *pot = malloc(n * sizeof(double));
    int32_t *act = malloc(n * sizeof(int32_t));
    const double zero = 0.0;
    int rc = 0;
    double nblocks = 0, nsteps = 0, npairs = 0;

    for (int64_t i = 0; i < n; ++i) act[i] = (int32_t)i;
    orc_regular_force(n, x, v, m, n, act, &zero, 1, a, jk, pot, NULL, NULL, 0);
    npairs += (double)n * (double)(n - 1);
    for (int64_t i = 0; i < n; ++i) {
        if (dt_fixed > 0) dt[i] = dt_fixed;
        else dt[i] = quantise_step(eta_s * norm3(a + 3 * i) / norm3(jk + 3 * i), dt_max);
    }

    for (;;) {
        double t_next = INFINITY;
        int64_t n_act = 0;
        if (replay) {
            const int64_t b = (int64_t)nblocks;
            if (b >= replay->n_blocks) break;
            t_next = replay->t_next[b];
            for (int64_t q = replay->act_off[b]; q < replay->act_off[b + 1]; ++q) act[n_act++] = replay->act_idx[q];
        } else {
            for (int64_t i = 0; i < n; ++i)
                if (t[i] + dt[i] < t_next) t_next = t[i] + dt[i];
            if (t_next > t_end) break;
            if (max_blocks > 0 && nblocks >= (double)max_blocks) { rc = -2; break; }
            for (int64_t i = 0; i < n; ++i)
                if (t[i] + dt[i] == t_next) act[n_act++] = (int32_t)i;
        }
        if (record) {
            const int64_t b = record->n_blocks;
            const int64_t o = b == 0 ? 0 : record->act_off[b];
            if (b >= record->cap_blocks || o + n_act > record->cap_act) { rc = -3; break; }
            if (b == 0) record->act_off[0] = 0;
            record->t_next[b] = t_next;
            for (int64_t k = 0; k < n_act; ++k) record->act_idx[o + k] = act[k];
            record->act_off[b + 1] = o + n_act;
            record->n_blocks = b + 1;
        }
        /* predict everybody to the block time */
        orc_predict(n, t_next, x, v, a, jk, t, xp, vp);
        orc_regular_force(n, xp, vp, m, n_act, act, &zero, 1, a1, j1, pot, NULL, NULL, 0);
        npairs += (double)n_act * (double)(n - 1);
        for (int64_t k = 0; k < n_act; ++k) {
            const int64_t i = act[k];
            const double h = t_next - t[i]; /* = dt[i] exactly (dyadic times) unless replaying */
            double a2[3], a3[3], a2e[3];
            for (int c = 0; c < 3; ++c) {
                const double da = a[3 * i + c] - a1[3 * k + c];
                a2[c] = (-6.0 * da - h * (4.0 * jk[3 * i + c] + 2.0 * j1[3 * k + c])) / (h * h);
                a3[c] = (12.0 * da + 6.0 * h * (jk[3 * i + c] + j1[3 * k + c])) / (h * h * h);
                x[3 * i + c] = xp[3 * i + c] + h * h * h * h / 24.0 * a2[c] + h * h * h * h * h / 120.0 * a3[c];
                v[3 * i + c] = vp[3 * i + c] + h * h * h / 6.0 * a2[c] + h * h * h * h / 24.0 * a3[c];
                a[3 * i + c] = a1[3 * k + c];
                jk[3 * i + c] = j1[3 * k + c];
                a2e[c] = a2[c] + h * a3[c];
            }
            t[i] = t_next;
            if (dt_fixed <= 0 && !replay) {
                const double na = norm3(a + 3 * i), nj = norm3(jk + 3 * i);
                const double n2 = norm3(a2e), n3 = norm3(a3);
                const double crit = sqrt(eta * (na * n2 + nj * nj) / (nj * n3 + n2 * n2));
                double hn = h;
                if (crit < hn) {
                    while (hn > crit && hn > 1e-30) hn *= 0.5;
                } else if (crit >= 2.0 * h && 2.0 * h <= dt_max && fmod(t_next, 2.0 * h) == 0.0) {
                    hn = 2.0 * h;
                }
                dt[i] = hn;
            }
        }
        nblocks += 1;
        nsteps += (double)n_act;
    }
    if (stats) { stats[0] = nblocks; stats[1] = nsteps; stats[2] = npairs; stats[3] = 0; }
    free(a); free(jk); free(xp); free(vp); free(t); free(dt); free(a1); free(j1); free(pot); free(act);
    return rc;
}

/* Regular-force sums of the active rows idx over a subset jdx of the sources only:
 *   acc_k = sum_{j in jdx, j != idx[k]} m_j r/|r|^3   (same for jerk and pot),
 * the definition above with the j-loop restricted (used for O(N) finite differences:
 * perturbing one particle p changes only row p and the column j = p of every row). */
int orc_pair_sums(int64_t n, const double *xp, const double *vp, const double *m, int64_t n_i, const int32_t *idx,
                  int64_t n_j, const int32_t *jdx, double *acc, double *jerk, double *pot)
{
    for (int64_t k = 0; k < n_i; ++k)
        if (idx[k] < 0 || idx[k] >= n) return -1;
    for (int64_t q = 0; q < n_j; ++q)
        if (jdx[q] < 0 || jdx[q] >= n) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n_i; ++k) {
        const int64_t i = idx[k];
        double ax = 0, ay = 0, az = 0, jx = 0, jy = 0, jz = 0, ph = 0;
        for (int64_t q = 0; q < n_j; ++q) {
            const int64_t j = jdx[q];
            if (j == i) continue;
            const double rx = xp[3 * j + 0] - xp[3 * i + 0];
            const double ry = xp[3 * j + 1] - xp[3 * i + 1];
            const double rz = xp[3 * j + 2] - xp[3 * i + 2];
            const double wx = vp[3 * j + 0] - vp[3 * i + 0];
            const double wy = vp[3 * j + 1] - vp[3 * i + 1];
            const double wz = vp[3 * j + 2] - vp[3 * i + 2];
            const double r2 = rx * rx + ry * ry + rz * rz;
            const double rinv = 1.0 / sqrt(r2);
            const double rinv2 = rinv * rinv;
            const double mr3 = m[j] * rinv * rinv2;
            const double rw = rx * wx + ry * wy + rz * wz;
            ax += mr3 * rx;
            ay += mr3 * ry;
            az += mr3 * rz;
            jx += mr3 * (wx - 3.0 * rw * rinv2 * rx);
            jy += mr3 * (wy - 3.0 * rw * rinv2 * ry);
            jz += mr3 * (wz - 3.0 * rw * rinv2 * rz);
            ph -= m[j] * rinv;
        }
        acc[3 * k + 0] = ax;  acc[3 * k + 1] = ay;  acc[3 * k + 2] = az;
        jerk[3 * k + 0] = jx; jerk[3 * k + 1] = jy; jerk[3 * k + 2] = jz;
        pot[k] = ph;
    }
    return 0;
}

/* Irregular force of the Ahmad-Cohen scheme (Sec. 2; Sec. 3.2.2 "Prediction and irregular
 * force"): for every active i = idx[k], the acceleration, jerk and potential summed over its
 * neighbour list only, j in nb_idx[nb_off[k] .. nb_off[k+1]), in list order.  The particles
 * come as their Hermite state (x, v, a, jerk at t_last) and only i and its neighbours are
 * predicted to time t (neighbour-only prediction, Sec. 3.3.3), with the same Taylor form as
 * orc_predict.  A listed j equal to i is skipped.  Returns 0, or -1 on an index outside
 * [0, n) or decreasing offsets. */
static void predict_one(int64_t p, double t, const double *x, const double *v, const double *a,
                        const double *jk, const double *t_last, double *xp, double *vp)
{
    const double dt = t - t_last[p];
    for (int c = 0; c < 3; ++c) {
        const int64_t q = 3 * p + c;
        xp[c] = x[q] + v[q] * dt + a[q] * dt * dt / 2.0 + jk[q] * dt * dt * dt / 6.0;
        vp[c] = v[q] + a[q] * dt + jk[q] * dt * dt / 2.0;
    }
}

int orc_irregular_force(int64_t n, const double *x, const double *v, const double *a, const double *jk,
                        const double *t_last, const double *m, double t, int64_t n_i, const int32_t *idx,
                        const int64_t *nb_off, const int32_t *nb_idx, double *acc, double *jerk, double *pot)
{
    for (int64_t k = 0; k < n_i; ++k) {
        if (idx[k] < 0 || idx[k] >= n || nb_off[k + 1] < nb_off[k] || nb_off[k] < 0) return -1;
        for (int64_t e = nb_off[k]; e < nb_off[k + 1]; ++e)
            if (nb_idx[e] < 0 || nb_idx[e] >= n) return -1;
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < n_i; ++k) {
        const int64_t i = idx[k];
        double xi[3], vi[3], xj[3], vj[3];
        predict_one(i, t, x, v, a, jk, t_last, xi, vi);
        double ax = 0, ay = 0, az = 0, jx = 0, jy = 0, jz = 0, ph = 0;
        for (int64_t e = nb_off[k]; e < nb_off[k + 1]; ++e) {
            const int64_t j = nb_idx[e];
            if (j == i) continue;
            predict_one(j, t, x, v, a, jk, t_last, xj, vj);
            const double rx = xj[0] - xi[0], ry = xj[1] - xi[1], rz = xj[2] - xi[2];
            const double wx = vj[0] - vi[0], wy = vj[1] - vi[1], wz = vj[2] - vi[2];
            const double r2 = rx * rx + ry * ry + rz * rz;
            const double rinv = 1.0 / sqrt(r2);
            const double rinv2 = rinv * rinv;
            const double mr3 = m[j] * rinv * rinv2;
            const double rw = rx * wx + ry * wy + rz * wz;
            ax += mr3 * rx;
            ay += mr3 * ry;
            az += mr3 * rz;
            jx += mr3 * (wx - 3.0 * rw * rinv2 * rx);
            jy += mr3 * (wy - 3.0 * rw * rinv2 * ry);
            jz += mr3 * (wz - 3.0 * rw * rinv2 * rz);
            ph -= m[j] * rinv;
        }
        acc[3 * k + 0] = ax;  acc[3 * k + 1] = ay;  acc[3 * k + 2] = az;
        jerk[3 * k + 0] = jx; jerk[3 * k + 1] = jy; jerk[3 * k + 2] = jz;
        pot[k] = ph;
    }
    return 0;
}

/* ---------------------------------------------------------------------------------------
 * Ahmad-Cohen (AC) Hermite integration with hierarchical block steps (Sec. 2: the force
 * on a particle is split into the irregular part from the neighbours inside r_s, computed
 * at every (short) irregular step, and the regular part from all other particles,
 * computed only at the (long) regular steps and extrapolated in between with its
 * derivatives; NBODY6++ adjusts r_s towards a target neighbour number NNBOPT, App. A).
 * The paper prints no formulas; this is the scheme as read here (every choice is listed in
 * the design notes):
 *
 * State of particle i: x, v at its last time t_i; total force a and jerk j there (used by
 * the predictor); irregular step dt_i, regular step DT_i (powers of 0.5, dt_i <= DT_i), the
 * time T_i of its last regular step; the regular force Fr, its derivative Jr and its higher
 * derivatives D2, D3 at T_i; the neighbour list L_i (ascending j, at most cap entries) and
 * r_s^2.
 *
 * Block step: t_next = min_i (t_i + dt_i); the active set is every i with t_i + dt_i =
 * t_next; all particles are predicted to t_next (Taylor to the jerk).  For active i,
 * with F_o, J_o the sums over the current list L_i:
 *  - irregular only (t_next is not a multiple of DT_i): the regular part is extrapolated,
 *    tau = t_next - T_i,  F_r = Fr + Jr tau + D2 tau^2/2 + D3 tau^3/6,
 *    J_r = Jr + D2 tau + D3 tau^2/2, and the new total is a1 = F_o + F_r, j1 = J_o + J_r;
 *  - regular step as well: the sums over all particles give a1, j1 exactly and the new
 *    list (r^2 < r_s^2); the regular force with the old list, a1 - F_o, and its derivative
 *    close the Hermite interpolation from (Fr, Jr) at T_i over DT = t_next - T_i, giving
 *    D2' = D2R + DT D3R and D3' = D3R at t_next; then Fr = a1 - F_n, Jr = j1 - J_n with the
 *    sums F_n, J_n over the new list, T_i = t_next, and r_s^2 is scaled by
 *    (nb_opt / max(N_b, 1))^(2/3), the factor clamped to [1/2, 2] (nb_opt <= 0: fixed r_s).
 *  - corrector on the total force (as in hermite_core) with a0, j0 at t_i and a1, j1, the
 *    irregular step from the Aarseth criterion on the total force (eta_irr) and, on a
 *    regular step, the regular step from the criterion on the old-list regular force and
 *    D2', D3' (eta_reg; an undefined criterion, e.g. no regular force, allows doubling);
 *    both follow the block rule of hermite_core.  On a regular step the regular step is
 *    raised to the new irregular step if it came out shorter (a regular step shorter than
 *    the irregular one gains nothing: the all-j sums would be taken every step anyway, and
 *    a regular force that is only rounding noise must not shrink the steps); otherwise the
 *    irregular step is capped at the regular one.
 * Start: all forces at t = 0, lists, Fr = a - F_L, Jr = j - J_L, D2 = D3 = 0, dt_i and DT_i
 * the largest powers of two below eta_s |a|/|j| and eta_s |Fr|/|Jr| (capped at dt_max; an
 * undefined ratio gives dt_max), DT_i raised to dt_i if shorter.
 * With r_s covering every particle and nb_opt <= 0 the regular force is exactly zero and
 * this reduces to hermite_core.
 * rs2 (n) is used and updated in place.  Optional outputs (n entries, or n*cap for the
 * lists): t_i, dt_i, DT_i, T_i, list lengths and lists; (n,3) each: the total acceleration and
 * jerk each particle holds after its last step (a1, j1 of that step), and the predicted state of
 * the last block step (the state those forces were evaluated on, for the particles of that
 * block; a synchronised end time makes it every particle).  stats (6 doubles): block steps,
 * irregular particle steps, regular particle steps, neighbour pair evaluations, all-j pair
 * evaluations, 0.  Returns 0, or -2 when max_blocks was reached. */
static void ac_list_sum(int64_t i, const int32_t *list, int32_t cnt, const double *xp, const double *vp,
                        const double *m, double *acc, double *jerk)
{
    double ax = 0, ay = 0, az = 0, jx = 0, jy = 0, jz = 0;
    for (int32_t q = 0; q < cnt; ++q) {
        const int64_t j = list[q];
        if (j == i) continue;
        const double rx = xp[3 * j + 0] - xp[3 * i + 0];
        const double ry = xp[3 * j + 1] - xp[3 * i + 1];
        const double rz = xp[3 * j + 2] - xp[3 * i + 2];
        const double wx = vp[3 * j + 0] - vp[3 * i + 0];
        const double wy = vp[3 * j + 1] - vp[3 * i + 1];
        const double wz = vp[3 * j + 2] - vp[3 * i + 2];
        const double r2 = rx * rx + ry * ry + rz * rz;
        const double rinv = 1.0 / sqrt(r2);
        const double rinv2 = rinv * rinv;
        const double mr3 = m[j] * rinv * rinv2;
        const double rw = rx * wx + ry * wy + rz * wz;
        ax += mr3 * rx;
        ay += mr3 * ry;
        az += mr3 * rz;
        jx += mr3 * (wx - 3.0 * rw * rinv2 * rx);
        jy += mr3 * (wy - 3.0 * rw * rinv2 * ry);
        jz += mr3 * (wz - 3.0 * rw * rinv2 * rz);
    }
    acc[0] = ax; acc[1] = ay; acc[2] = az;
    jerk[0] = jx; jerk[1] = jy; jerk[2] = jz;
}

/* The step rule of hermite_core: halve until not above crit, or double when crit >= 2 h,
 * 2 h <= dt_max and t is a multiple of 2 h. */
static double ac_step_rule(double h, double crit, double t, double dt_max)
{
    double hn = h;
    if (crit < hn) {
        while (hn > crit && hn > 1e-30) hn *= 0.5;
    } else if (crit >= 2.0 * h && 2.0 * h <= dt_max && fmod(t, 2.0 * h) == 0.0) {
        hn = 2.0 * h;
    }
    return hn;
}

/* sqrt(eta (|a||a2| + |j|^2) / (|j||a3| + |a2|^2)); +inf where the ratio is undefined. */
static double ac_criterion(double eta, const double *a, const double *j, const double *a2, const double *a3)
{
    const double na = norm3(a), nj = norm3(j), n2 = norm3(a2), n3 = norm3(a3);
    const double num = na * n2 + nj * nj, den = nj * n3 + n2 * n2;
    if (!(den > 0.0) || !(num > 0.0)) return INFINITY;
    return sqrt(eta * num / den);
}

int orc_ac_run(int64_t n, const double *m, double *x, double *v, double *rs2, double t_end, double eta_irr,
               double eta_reg, double eta_s, double dt_max, int32_t nb_opt, int32_t cap, int64_t max_blocks,
               double *stats, double *t_out, double *dt_out, double *DT_out, double *T_out, int32_t *nbc_out,
               int32_t *nbl_out, double *a_out, double *j_out, double *xp_out, double *vp_out)
{
    double *a = malloc(3 * n * sizeof(double)), *jk = malloc(3 * n * sizeof(double));
    double *xp = malloc(3 * n * sizeof(double)), *vp = malloc(3 * n * sizeof(double));
    double *t = calloc(n, sizeof(double)), *dt = malloc(n * sizeof(double));
    double *T = calloc(n, sizeof(double)), *DT = malloc(n * sizeof(double));
    double *Fr = malloc(3 * n * sizeof(double)), *Jr = malloc(3 * n * sizeof(double));
    double *D2 = calloc(3 * n, sizeof(double)), *D3 = calloc(3 * n, sizeof(double));
    double *a1 = malloc(3 * n * sizeof(double)), *j1 = malloc(3 * n * sizeof(double));
    double *pot = malloc(n * sizeof(double));
    int32_t *nbl = malloc((size_t)n * cap * sizeof(int32_t)), *nbc = malloc(n * sizeof(int32_t));
    int32_t *act = malloc(n * sizeof(int32_t)), *newl = malloc((size_t)cap * sizeof(int32_t));
    char *regk = malloc(n);
    int rc = 0;
    double nblocks = 0, nirr = 0, nreg = 0, npair_nb = 0, npair_all = 0;

    for (int64_t i = 0; i < n; ++i) act[i] = (int32_t)i;
    orc_regular_force(n, x, v, m, n, act, rs2, 0, a, jk, pot, nbc, nbl, cap);
    npair_all += (double)n * (double)(n - 1);
    for (int64_t i = 0; i < n; ++i) {
        double Fl[3], Jl[3];
        const int32_t cnt = nbc[i] < cap ? nbc[i] : cap;
        nbc[i] = cnt;
        ac_list_sum(i, nbl + i * (int64_t)cap, cnt, x, v, m, Fl, Jl);
        for (int c = 0; c < 3; ++c) {
            Fr[3 * i + c] = a[3 * i + c] - Fl[c];
            Jr[3 * i + c] = jk[3 * i + c] - Jl[c];
        }
        const double ni = norm3(a + 3 * i), nji = norm3(jk + 3 * i);
        const double nr = norm3(Fr + 3 * i), njr = norm3(Jr + 3 * i);
        dt[i] = nji > 0.0 ? quantise_step(eta_s * ni / nji, dt_max) : dt_max;
        DT[i] = njr > 0.0 ? quantise_step(eta_s * nr / njr, dt_max) : dt_max;
        if (DT[i] < dt[i]) DT[i] = dt[i];
    }

    for (;;) {
        double t_next = INFINITY;
        int64_t n_act = 0;
        for (int64_t i = 0; i < n; ++i)
            if (t[i] + dt[i] < t_next) t_next = t[i] + dt[i];
        if (t_next > t_end) break;
        if (max_blocks > 0 && nblocks >= (double)max_blocks) { rc = -2; break; }
        for (int64_t i = 0; i < n; ++i)
            if (t[i] + dt[i] == t_next) act[n_act++] = (int32_t)i;
        orc_predict(n, t_next, x, v, a, jk, t, xp, vp);
        /* forces first (all from the same predicted snapshot), then the corrections */
        for (int64_t k = 0; k < n_act; ++k) {
            const int64_t i = act[k];
            double Fo[3], Jo[3];
            ac_list_sum(i, nbl + i * (int64_t)cap, nbc[i], xp, vp, m, Fo, Jo);
            npair_nb += (double)nbc[i];
            const int reg = fmod(t_next, DT[i]) == 0.0;
            regk[k] = (char)reg;
            if (!reg) {
                const double tau = t_next - T[i];
                for (int c = 0; c < 3; ++c) {
                    const int64_t q = 3 * i + c;
                    const double Fx = Fr[q] + Jr[q] * tau + D2[q] * tau * tau / 2.0 + D3[q] * tau * tau * tau / 6.0;
                    const double Jx = Jr[q] + D2[q] * tau + D3[q] * tau * tau / 2.0;
                    a1[3 * k + c] = Fo[c] + Fx;
                    j1[3 * k + c] = Jo[c] + Jx;
                }
                continue;
            }
            /* regular step: all-j sums with the new list */
            int32_t cnt_true = 0;
            const int32_t one = (int32_t)i;
            double pk;
            orc_regular_force(n, xp, vp, m, 1, &one, rs2 + i, 1, a1 + 3 * k, j1 + 3 * k, &pk, &cnt_true, newl, cap);
            npair_all += (double)(n - 1);
            nreg += 1;
            const int32_t cnt = cnt_true < cap ? cnt_true : cap;
            double Fn[3], Jn[3], Fold[3], Jold[3], a2r[3], a3r[3];
            ac_list_sum(i, newl, cnt, xp, vp, m, Fn, Jn);
            const double H = t_next - T[i];
            for (int c = 0; c < 3; ++c) {
                const int64_t q = 3 * i + c;
                Fold[c] = a1[3 * k + c] - Fo[c];
                Jold[c] = j1[3 * k + c] - Jo[c];
                const double df = Fr[q] - Fold[c];
                const double a2 = (-6.0 * df - H * (4.0 * Jr[q] + 2.0 * Jold[c])) / (H * H);
                const double a3 = (12.0 * df + 6.0 * H * (Jr[q] + Jold[c])) / (H * H * H);
                a2r[c] = a2 + H * a3;
                a3r[c] = a3;
            }
            const double critR = ac_criterion(eta_reg, Fold, Jold, a2r, a3r);
            double DTn = ac_step_rule(DT[i], critR, t_next, dt_max);
            for (int c = 0; c < 3; ++c) {
                const int64_t q = 3 * i + c;
                Fr[q] = a1[3 * k + c] - Fn[c];
                Jr[q] = j1[3 * k + c] - Jn[c];
                D2[q] = a2r[c];
                D3[q] = a3r[c];
            }
            T[i] = t_next;
            DT[i] = DTn;  /* provisional; dt is capped against it below */
            memcpy(nbl + i * (int64_t)cap, newl, (size_t)cnt * sizeof(int32_t));
            nbc[i] = cnt;
            if (nb_opt > 0) {
                double f = pow((double)nb_opt / (double)(cnt_true > 0 ? cnt_true : 1), 2.0 / 3.0);
                f = f < 0.5 ? 0.5 : (f > 2.0 ? 2.0 : f);
                rs2[i] *= f;
            }
        }
        for (int64_t k = 0; k < n_act; ++k) {
            const int64_t i = act[k];
            const double h = t_next - t[i];
            double a2[3], a3[3], a2e[3];
            for (int c = 0; c < 3; ++c) {
                const double da = a[3 * i + c] - a1[3 * k + c];
                a2[c] = (-6.0 * da - h * (4.0 * jk[3 * i + c] + 2.0 * j1[3 * k + c])) / (h * h);
                a3[c] = (12.0 * da + 6.0 * h * (jk[3 * i + c] + j1[3 * k + c])) / (h * h * h);
                x[3 * i + c] = xp[3 * i + c] + h * h * h * h / 24.0 * a2[c] + h * h * h * h * h / 120.0 * a3[c];
                v[3 * i + c] = vp[3 * i + c] + h * h * h / 6.0 * a2[c] + h * h * h * h / 24.0 * a3[c];
                a[3 * i + c] = a1[3 * k + c];
                jk[3 * i + c] = j1[3 * k + c];
                a2e[c] = a2[c] + h * a3[c];
            }
            t[i] = t_next;
            const double crit = ac_criterion(eta_irr, a + 3 * i, jk + 3 * i, a2e, a3);
            double hn = ac_step_rule(h, crit, t_next, dt_max);
            if (regk[k]) {
                if (DT[i] < hn) DT[i] = hn;
            } else if (hn > DT[i]) {
                hn = DT[i];
            }
            dt[i] = hn;
        }
        nblocks += 1;
        nirr += (double)n_act;
    }
    if (stats) { stats[0] = nblocks; stats[1] = nirr; stats[2] = nreg; stats[3] = npair_nb; stats[4] = npair_all; stats[5] = 0; }
    for (int64_t i = 0; i < n; ++i) {
        if (t_out) t_out[i] = t[i];
        if (dt_out) dt_out[i] = dt[i];
        if (DT_out) DT_out[i] = DT[i];
        if (T_out) T_out[i] = T[i];
        if (nbc_out) nbc_out[i] = nbc[i];
    }
    if (nbl_out) memcpy(nbl_out, nbl, (size_t)n * cap * sizeof(int32_t));
    if (a_out) memcpy(a_out, a, 3 * (size_t)n * sizeof(double));
    if (j_out) memcpy(j_out, jk, 3 * (size_t)n * sizeof(double));
    if (xp_out) memcpy(xp_out, xp, 3 * (size_t)n * sizeof(double));
    if (vp_out) memcpy(vp_out, vp, 3 * (size_t)n * sizeof(double));
    free(a); free(jk); free(xp); free(vp); free(t); free(dt); free(T); free(DT); free(Fr); free(Jr);
    free(D2); free(D3); free(a1); free(j1); free(pot); free(nbl); free(nbc); free(act); free(newl); free(regk);
    return rc;
}
