/* A plain C consumer of the library (no Python): it loads a Hermite state, predicts it to
 * time t and runs the regular force on an active block with host buffers, then writes the
 * results.  Used by tests/test_c_abi.py, which compiles it with -std=c11 against
 * include/nbgpu.h and links it to libnbgpu.so.
 *
 * Input file (native byte order): int64 n; x, v, a, jerk as n*3 doubles each; m, t_last as
 * n doubles each; int64 n_i; idx as n_i int32; double rs2; double t; int32 precision; int32 cap.
 * Output file: acc, jerk (n_i*3 doubles each), pot (n_i doubles), nb_off (n_i+1 int64),
 * nb_count (n_i int32), then the nb_off[n_i] neighbour indices (int32). */
#include <stdio.h>
#include <stdlib.h>

#include "nbgpu.h"

static int get(FILE *f, void *p, size_t size, size_t count) { return fread(p, size, count, f) == count; }

static void *alloc(size_t bytes) { return malloc(bytes ? bytes : 1); }

int main(int argc, char **argv)
{
    if (argc != 3) {
        fprintf(stderr, "usage: %s input output\n", argv[0]);
        return 2;
    }
    FILE *in = fopen(argv[1], "rb");
    if (!in) return 2;
    int64_t n = 0, n_i = 0;
    int32_t precision = 0, cap = 0;
    double rs2 = 0.0, t = 0.0;
    if (!get(in, &n, sizeof n, 1) || n < 1) return 2;
    double *x = alloc(24 * n), *v = alloc(24 * n), *a = alloc(24 * n), *j = alloc(24 * n);
    double *m = alloc(8 * n), *tl = alloc(8 * n);
    int ok = get(in, x, 8, 3 * n) && get(in, v, 8, 3 * n) && get(in, a, 8, 3 * n) && get(in, j, 8, 3 * n) &&
             get(in, m, 8, n) && get(in, tl, 8, n) && get(in, &n_i, sizeof n_i, 1);
    if (!ok || n_i < 0) return 2;
    int32_t *idx = alloc(4 * n_i);
    ok = get(in, idx, 4, n_i) && get(in, &rs2, 8, 1) && get(in, &t, 8, 1) && get(in, &precision, 4, 1) &&
         get(in, &cap, 4, 1);
    fclose(in);
    if (!ok) return 2;

    nb_config cfg = {n, precision, cap, 0, 0, NULL};
    nb_ctx *ctx = NULL;
    nb_status s = nb_init(&ctx, &cfg);
    if (s != NB_OK) {
        fprintf(stderr, "nb_init: status %d\n", (int)s);
        return 1;
    }
    double *acc = alloc(24 * n_i), *jerk = alloc(24 * n_i), *pot = alloc(8 * n_i);
    int64_t *off = alloc(8 * (n_i + 1));
    int32_t *cnt = alloc(4 * n_i), *lists = alloc(4 * (size_t)n_i * cap);
    s = nb_set_particles(ctx, n, x, v, a, j, m, tl, 0);
    if (s == NB_OK) s = nb_predict(ctx, t);
    if (s == NB_OK)
        s = nb_regular_force(ctx, n_i, idx, &rs2, 1, acc, jerk, pot, off, lists, (int64_t)n_i * cap, cnt, 0);
    if (s != NB_OK && s != NB_ERR_NB_OVERFLOW) {
        fprintf(stderr, "status %d: %s\n", (int)s, nb_last_error(ctx));
        nb_free(ctx);
        return 1;
    }
    FILE *out = fopen(argv[2], "wb");
    if (!out) return 2;
    fwrite(acc, 8, 3 * n_i, out);
    fwrite(jerk, 8, 3 * n_i, out);
    fwrite(pot, 8, n_i, out);
    fwrite(off, 8, n_i + 1, out);
    fwrite(cnt, 4, n_i, out);
    fwrite(lists, 4, off[n_i], out);
    fclose(out);
    nb_free(ctx);
    printf("ok %d\n", (int)s);
    return 0;
}
