/*
 * oracle.c -- plain FP64 CPU oracle for the all-pairs softened N-body force.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity reference for the CUDA
 * library and the timed CPU baseline; the library never links, loads or calls
 * it, and it includes nothing from the library.  Only the tests, the smoke
 * check and the benchmark's CPU leg use it.
 *
 * What it computes (Miki & Hanawa, "Unified schemes for directive-based GPU
 * offloading", Sec. III.A):
 *
 *   Eq. 1 with G = 1 (Henon units):
 *       a_i   =  sum_{j != i} m_j (r_j - r_i) / (|r_j - r_i|^2 + eps^2)^{3/2}
 *   the potential accumulated under CALCULATE_POTENTIAL in Listing 4, read as
 *   the physical (negative) potential with the self term removed:
 *       phi_i = -sum_{j != i} m_j / (|r_j - r_i|^2 + eps^2)^{1/2}
 *
 * Everything is double precision, summed over j in index order, with 1/sqrt
 * taken as 1.0 / sqrt(s).  OpenMP parallelises over i only, so the result does
 * not depend on the thread count.  Build with -ffp-contract=off so that no
 * multiply-add is fused and x86 and Arm give the same bits.
 *
 * The integrator, the energy and the adjoint are not in the paper; they follow
 * the kick-drift-kick leapfrog the library implements:
 *       v <- v + (dt/2) a(x);  x <- x + dt v;  v <- v + (dt/2) a(x)
 *
 * Adjoint (reverse-mode derivative) of the force and of the leapfrog: the
 * chain rule applied to every pair term of Eq. 1.  A term
 *       m_j f(d),  f(d) = d s^{-3/2},  d = r_j - r_i,  s = |d|^2 + eps^2
 * has Jacobian  T(d) = s^{-3/2} I - 3 s^{-5/2} d d^T  with respect to d, so
 * it moves with r_j through +m_j T(d), with r_i through -m_j T(d), and with
 * m_j through f(d).  The potential term -m_j s^{-1/2} has gradient
 * m_j s^{-3/2} d with respect to r_j (minus that for r_i) and -s^{-1/2} for m_j.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int nt) {
#ifdef _OPENMP
    if (nt > 0) omp_set_num_threads(nt);
#else
    (void)nt;
#endif
}

/* Force and potential on body i from every j != i (Eq. 1, G = 1). */
static void body_sum(int64_t i, int64_t n, const double* pos, const double* mass, double eps2,
                     double* a3, double* phi) {
    const double xi = pos[3 * i + 0], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
    double ax = 0.0, ay = 0.0, az = 0.0, p = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        const double dx = pos[3 * j + 0] - xi;
        const double dy = pos[3 * j + 1] - yi;
        const double dz = pos[3 * j + 2] - zi;
        const double s = dx * dx + dy * dy + dz * dz + eps2;
        const double rinv = 1.0 / sqrt(s);
        const double w = mass[j] * rinv * rinv * rinv; /* m_j s^{-3/2} */
        ax += w * dx;
        ay += w * dy;
        az += w * dz;
        p -= mass[j] * rinv; /* -m_j s^{-1/2} */
    }
    a3[0] = ax;
    a3[1] = ay;
    a3[2] = az;
    if (phi) *phi = p;
}

/* acc (n,3) and pot (n, may be NULL) for all n bodies. */
void oracle_accel(int64_t n, const double* pos, const double* mass, double eps, double* acc,
                  double* pot) {
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) body_sum(i, n, pos, mass, eps2, acc + 3 * i, pot ? pot + i : NULL);
}

/* The same sums for the ns bodies listed in idx (each against all n bodies,
 * itself excluded): acc (ns,3), pot (ns) or NULL. */
void oracle_accel_subset(int64_t n, const double* pos, const double* mass, double eps, int64_t ns,
                         const int64_t* idx, double* acc, double* pot) {
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < ns; ++k) body_sum(idx[k], n, pos, mass, eps2, acc + 3 * k, pot ? pot + k : NULL);
}

/* Separate sinks and sources (Listing 4's calc_acc form): every pair of the
 * ni sinks with the nj sources is included. */
void oracle_accel_ij(int64_t ni, const double* ipos, int64_t nj, const double* jpos, const double* jmass,
                     double eps, double* acc, double* pot) {
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < ni; ++i) {
        double ax = 0.0, ay = 0.0, az = 0.0, p = 0.0;
        for (int64_t j = 0; j < nj; ++j) {
            const double dx = jpos[3 * j + 0] - ipos[3 * i + 0];
            const double dy = jpos[3 * j + 1] - ipos[3 * i + 1];
            const double dz = jpos[3 * j + 2] - ipos[3 * i + 2];
            const double s = dx * dx + dy * dy + dz * dz + eps2;
            const double rinv = 1.0 / sqrt(s);
            const double w = jmass[j] * rinv * rinv * rinv;
            ax += w * dx;
            ay += w * dy;
            az += w * dz;
            p -= jmass[j] * rinv;
        }
        acc[3 * i + 0] = ax;
        acc[3 * i + 1] = ay;
        acc[3 * i + 2] = az;
        if (pot) pot[i] = p;
    }
}

/* Kick-drift-kick leapfrog, in place, steps >= 0.  The force at the end of a
 * step is reused for the first kick of the next, so steps + 1 evaluations.
 * acc_out (n,3), optional: the force at the final positions. */
void oracle_leapfrog(int64_t n, double* pos, double* vel, const double* mass, double eps, double dt,
                     int64_t steps, double* acc_out) {
    double* a = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    oracle_accel(n, pos, mass, eps, a, NULL);
    const double h = 0.5 * dt;
    for (int64_t s = 0; s < steps; ++s) {
        for (int64_t k = 0; k < 3 * n; ++k) vel[k] += h * a[k];
        for (int64_t k = 0; k < 3 * n; ++k) pos[k] += dt * vel[k];
        oracle_accel(n, pos, mass, eps, a, NULL);
        for (int64_t k = 0; k < 3 * n; ++k) vel[k] += h * a[k];
    }
    if (acc_out) memcpy(acc_out, a, sizeof(double) * 3 * (size_t)n);
    free(a);
}

/* Diagnostics: out[0] = kinetic T = sum m|v|^2/2, out[1] = potential
 * W = (1/2) sum m_i phi_i, out[2] = E = T + W, out[3..5] = momentum sum m v,
 * out[6..8] = net force sum m a (zero by Newton's third law). */
void oracle_energy(int64_t n, const double* pos, const double* vel, const double* mass, double eps,
                   double* out) {
    double* a = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double* phi = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    oracle_accel(n, pos, mass, eps, a, phi);
    double t = 0, w = 0, px = 0, py = 0, pz = 0, fx = 0, fy = 0, fz = 0;
    for (int64_t i = 0; i < n; ++i) {
        const double vx = vel[3 * i], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
        t += 0.5 * mass[i] * (vx * vx + vy * vy + vz * vz);
        w += 0.5 * mass[i] * phi[i];
        px += mass[i] * vx;
        py += mass[i] * vy;
        pz += mass[i] * vz;
        fx += mass[i] * a[3 * i];
        fy += mass[i] * a[3 * i + 1];
        fz += mass[i] * a[3 * i + 2];
    }
    out[0] = t;
    out[1] = w;
    out[2] = t + w;
    out[3] = px;
    out[4] = py;
    out[5] = pz;
    out[6] = fx;
    out[7] = fy;
    out[8] = fz;
    free(a);
    free(phi);
}

/* T(d) = s^{-3/2} I - 3 s^{-5/2} d d^T for d with softening eps2. */
static void pair_jacobian(const double d[3], double eps2, double T[3][3], double* s_m32, double* s_m12) {
    const double s = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps2;
    const double r = 1.0 / sqrt(s);
    const double s32 = r * r * r;
    const double s52 = s32 * r * r;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) T[a][b] = (a == b ? s32 : 0.0) - 3.0 * s52 * d[a] * d[b];
    *s_m32 = s32;
    *s_m12 = r;
}

/* Cotangents lam (n,3) of the accelerations and mu (n, or NULL) of the
 * potentials: g_pos[k] = d(sum_i lam_i.a_i + mu_i phi_i)/d r_k and
 * g_mass[k] = the same derivative with respect to m_k.  Gathered per k:
 * body k enters the sums as the source of every pair (i, k), i != k, and as the
 * sink of every pair (k, i). */
void oracle_accel_vjp(int64_t n, const double* pos, const double* mass, double eps, const double* lam,
                      const double* mu, double* g_pos, double* g_mass) {
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t k = 0; k < n; ++k) {
        double g[3] = {0.0, 0.0, 0.0}, gm = 0.0;
        const double* lk = lam + 3 * k;
        for (int64_t i = 0; i < n; ++i) {
            if (i == k) continue;
            const double* li = lam + 3 * i;
            /* as the source of sink i: the term m_k f(r_k - r_i) of a_i */
            const double d[3] = {pos[3 * k] - pos[3 * i], pos[3 * k + 1] - pos[3 * i + 1],
                                 pos[3 * k + 2] - pos[3 * i + 2]};
            double T[3][3], s32, s12;
            pair_jacobian(d, eps2, T, &s32, &s12);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) g[a] += mass[k] * T[a][b] * li[b];
            gm += (li[0] * d[0] + li[1] * d[1] + li[2] * d[2]) * s32;
            /* as the sink of source i: the term m_i f(r_i - r_k) of a_k, T(-d) = T(d) */
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) g[a] -= mass[i] * T[a][b] * lk[b];
            if (mu) {
                /* -m_k s^{-1/2} in phi_i and -m_i s^{-1/2} in phi_k */
                for (int a = 0; a < 3; ++a) g[a] += s32 * d[a] * (mu[i] * mass[k] + mu[k] * mass[i]);
                gm -= mu[i] * s12;
            }
        }
        g_pos[3 * k + 0] = g[0];
        g_pos[3 * k + 1] = g[1];
        g_pos[3 * k + 2] = g[2];
        g_mass[k] = gm;
    }
}

/* Reverse mode of oracle_leapfrog: given gx_T = dL/dx(T) and gv_T = dL/dv(T),
 * returns dL/dx(0), dL/dv(0) and the dynamics' part of dL/dm (a loss that also
 * depends on m directly adds its own term).  The forward trajectory is kept in
 * full and every half kick is undone by its own force adjoint. */
void oracle_leapfrog_vjp(int64_t n, const double* pos0, const double* vel0, const double* mass, double eps,
                         double dt, int64_t steps, const double* gx_T, const double* gv_T, double* gx0,
                         double* gv0, double* gm) {
    const size_t n3 = 3 * (size_t)(n > 0 ? n : 1);
    double* X = (double*)malloc(sizeof(double) * n3 * (size_t)(steps + 1));
    double* x = (double*)malloc(sizeof(double) * n3);
    double* v = (double*)malloc(sizeof(double) * n3);
    double* a = (double*)malloc(sizeof(double) * n3);
    double* lv = (double*)malloc(sizeof(double) * n3);
    double* gxk = (double*)malloc(sizeof(double) * n3);
    double* gmk = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    const double h = 0.5 * dt;
    memcpy(x, pos0, sizeof(double) * 3 * (size_t)n);
    memcpy(v, vel0, sizeof(double) * 3 * (size_t)n);
    memcpy(X, x, sizeof(double) * 3 * (size_t)n);
    oracle_accel(n, x, mass, eps, a, NULL);
    for (int64_t s = 0; s < steps; ++s) {
        for (int64_t k = 0; k < 3 * n; ++k) v[k] += h * a[k];
        for (int64_t k = 0; k < 3 * n; ++k) x[k] += dt * v[k];
        oracle_accel(n, x, mass, eps, a, NULL);
        for (int64_t k = 0; k < 3 * n; ++k) v[k] += h * a[k];
        memcpy(X + n3 * (size_t)(s + 1), x, sizeof(double) * 3 * (size_t)n);
    }
    /* reverse sweep: (gx0, lv) hold dL/dx and dL/dv of the current state */
    memcpy(gx0, gx_T, sizeof(double) * 3 * (size_t)n);
    memcpy(lv, gv_T, sizeof(double) * 3 * (size_t)n);
    for (int64_t i = 0; i < n; ++i) gm[i] = 0.0;
    for (int64_t s = steps - 1; s >= 0; --s) {
        const double* x1 = X + n3 * (size_t)(s + 1);
        const double* x0 = X + n3 * (size_t)s;
        /* v_{s+1} = v_half + h a(x_{s+1}) */
        for (int64_t k = 0; k < 3 * n; ++k) a[k] = h * lv[k];
        oracle_accel_vjp(n, x1, mass, eps, a, NULL, gxk, gmk);
        for (int64_t k = 0; k < 3 * n; ++k) gx0[k] += gxk[k];
        for (int64_t i = 0; i < n; ++i) gm[i] += gmk[i];
        /* x_{s+1} = x_s + dt v_half */
        for (int64_t k = 0; k < 3 * n; ++k) lv[k] += dt * gx0[k];
        /* v_half = v_s + h a(x_s) */
        for (int64_t k = 0; k < 3 * n; ++k) a[k] = h * lv[k];
        oracle_accel_vjp(n, x0, mass, eps, a, NULL, gxk, gmk);
        for (int64_t k = 0; k < 3 * n; ++k) gx0[k] += gxk[k];
        for (int64_t i = 0; i < n; ++i) gm[i] += gmk[i];
    }
    memcpy(gv0, lv, sizeof(double) * 3 * (size_t)n);
    free(X);
    free(x);
    free(v);
    free(a);
    free(lv);
    free(gxk);
    free(gmk);
}

/*
 * Single-precision restatement of Listing 4 (Sec. III.A): a second, CPU
 * reference that evaluates the listing's own FP32 arithmetic with every
 * operation correctly rounded (IEEE binary32, no approximate reciprocal
 * square root, no flush-to-zero), in the listing's order:
 *   d = r_j - r_i                              three FP32 subtractions
 *   r2 = fma(dz, dz, fma(dy, dy, fma(dx, dx, eps^2)))   eps^2 = eps * eps in FP32
 *   w = 1 / sqrt(r2)                           correctly rounded sqrt, then division
 *   w = w * (w * w);  w = w * m_j
 *   a += fma(d, w, a) per component, p = fma(r2, w, p)   one FP32 running sum in j order
 * p accumulates m_j / r as the listing does; it is returned negated (the
 * physical potential).  The sinks are the sources here, so the pair j == i is
 * skipped (Eq. 1; the listing has no such test, which for eps > 0 changes
 * only the potential, by +m_i/eps).  This is the error an exactly rounded
 * FP32 evaluation of the listing has; the GPU kernels differ from it by the
 * hardware reciprocal-square-root approximation and their summation order.
 */
static void body_sum_listing_f32(int64_t i, int64_t n, const float* pos, const float* mass, float eps2,
                                 float* a3, float* phi) {
    const float xi = pos[3 * i + 0], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
    float ax = 0.0f, ay = 0.0f, az = 0.0f, p = 0.0f;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        const float dx = pos[3 * j + 0] - xi;
        const float dy = pos[3 * j + 1] - yi;
        const float dz = pos[3 * j + 2] - zi;
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
        float w = 1.0f / sqrtf(r2);
        w = w * (w * w);
        w = w * mass[j];
        ax = fmaf(dx, w, ax);
        ay = fmaf(dy, w, ay);
        az = fmaf(dz, w, az);
        p = fmaf(r2, w, p);
    }
    a3[0] = ax;
    a3[1] = ay;
    a3[2] = az;
    if (phi) *phi = -p;
}

/* acc (n,3) and pot (n, may be NULL) in FP32 for all n bodies. */
void oracle_accel_listing_f32(int64_t n, const float* pos, const float* mass, float eps, float* acc, float* pot) {
    const float eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) body_sum_listing_f32(i, n, pos, mass, eps2, acc + 3 * i, pot ? pot + i : NULL);
}

/* The same for the ns bodies listed in idx, each against all n bodies. */
void oracle_accel_listing_f32_subset(int64_t n, const float* pos, const float* mass, float eps, int64_t ns,
                                     const int64_t* idx, float* acc, float* pot) {
    const float eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < ns; ++k)
        body_sum_listing_f32(idx[k], n, pos, mass, eps2, acc + 3 * k, pot ? pot + k : NULL);
}
