/* A C program using libnbody through include/nbody.h only: checks that the
 * header is valid C11 and that the library works without Python.  It computes
 * the force on a small system from host arrays, and compares two bodies'
 * accelerations with a direct double-precision sum written here. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "nbody.h"

int main(void) {
    enum { N = 300 };
    static double pos[N][3];
    static float mass[N], acc[N][3], pot[N];
    unsigned long long s = 12345;
    for (int i = 0; i < N; ++i) {
        for (int c = 0; c < 3; ++c) {
            s = s * 6364136223846793005ull + 1442695040888963407ull;
            pos[i][c] = (double)(s >> 11) / 9007199254740992.0 - 0.5;
        }
        mass[i] = 1.0f / N;
    }
    const double eps = 0.01;
    nbody_opts o;
    nbody_opts_default(&o);
    int rc = nbody_accel(N, &pos[0][0], mass, eps, &acc[0][0], pot, &o);
    if (rc != NBODY_OK) {
        fprintf(stderr, "nbody_accel: %s\n", nbody_strerror(rc));
        return 1;
    }
    for (int i = 0; i < N; i += N - 1) {
        double a[3] = {0, 0, 0}, p = 0;
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            double d[3], r2 = eps * eps;
            for (int c = 0; c < 3; ++c) {
                d[c] = pos[j][c] - pos[i][c];
                r2 += d[c] * d[c];
            }
            const double r = sqrt(r2);
            for (int c = 0; c < 3; ++c) a[c] += mass[j] * d[c] / (r2 * r);
            p -= mass[j] / r;
        }
        const double na = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        double err = 0;
        for (int c = 0; c < 3; ++c) err += (acc[i][c] - a[c]) * (acc[i][c] - a[c]);
        err = sqrt(err) / na;
        if (!(err < 1e-5) || !(fabs(pot[i] - p) < 1e-5 * fabs(p))) {
            fprintf(stderr, "body %d: relative error %g\n", i, err);
            return 1;
        }
    }
    if (nbody_accel(-1, NULL, NULL, eps, NULL, NULL, NULL) != NBODY_EINVAL) return 1;
    printf("c abi ok: version %d, %d kernel shapes\n", nbody_version(), nbody_num_configs());
    nbody_finalize();
    return 0;
}
