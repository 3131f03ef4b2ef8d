/*
 * FP64 CPU oracle for the all-pairs N-body step of Milla & Rucci,
 * "Performance Comparison of Python Translators for a Multi-threaded
 * CPU-bound Application" (arXiv 2203.08263).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the independent, slow, plain
 * definition that the CUDA library is checked against. Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it. It shares no
 * code, header, table or constant with the CUDA path.
 *
 * Everything is IEEE double, compiled without fast-math and without FMA
 * contraction, parallelised over the output index with an OpenMP static
 * schedule (the loop structure of the paper's Cython prange, Section 3.3.5).
 *
 * Readings of the paper taken here (the paper prints no constants):
 *   - SOFT = eps^2 is added to |x_j - x_i|^2 (Figures python_numpy_broadcasting,
 *     numba_parallel, cython_parallel).
 *   - The force G m_i m_j d / s^1.5 is divided by m_i right after the sum
 *     (Section 3.2.4 figure); the two m_i factors cancel, so the oracle sums
 *     G m_j d / s^1.5 directly. This is also defined for m_i = 0.
 *   - The j-loop runs over every body, j = i included, exactly as printed;
 *     that term has d = 0 and contributes exactly 0 when eps > 0.
 *   - The update is the printed one: all accelerations from the positions at
 *     the start of the step, then v += a*dt/2 (a half kick), then
 *     x += v*dt with the new v, positions moved only after every body has
 *     been kicked (Section 2.3's two data dependencies).
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

void oracle_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/*
 * Acceleration of body i (Section 2.3; the force loop of the Section 3.2.4 and
 * 3.3.5 figures):  a_i = G * sum_j m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^(3/2).
 * j runs in ascending order over all n bodies.
 */
static void accel_one(int64_t n, const double *x, const double *m, double G,
                      double eps, int64_t i, double *ai) {
    const double soft = eps * eps;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double dx = x[3 * j + 0] - x[3 * i + 0];
        double dy = x[3 * j + 1] - x[3 * i + 1];
        double dz = x[3 * j + 2] - x[3 * i + 2];
        double s = dx * dx + dy * dy + dz * dz + soft;
        double r3 = s * sqrt(s);             /* s^(3/2) */
        double w = m[j] / r3;
        fx += w * dx;
        fy += w * dy;
        fz += w * dz;
    }
    ai[0] = G * fx;
    ai[1] = G * fy;
    ai[2] = G * fz;
}

/* a[k] for i = idx[k] (k < ni); idx == NULL means i = k for k < n. */
void oracle_accel(int64_t n, const double *x, const double *m, double G,
                  double eps, int64_t ni, const int64_t *idx, double *a) {
    if (idx == NULL) ni = n;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < ni; ++k) {
        int64_t i = idx ? idx[k] : k;
        accel_one(n, x, m, G, eps, i, a + 3 * k);
    }
}

/*
 * One step of the paper's update (Section 3.1.2 figure, split into the two
 * loops of Sections 3.2.3 / 3.3.5):
 *   loop 1, every i:  a_i from the old positions;
 *                     v_i <- v_i + a_i * dt / 2;
 *                     dp_i = v_i * dt          (the new v_i)
 *   loop 2, every i:  x_i <- x_i + dp_i
 * 'work' holds 3n doubles for dp.
 */
static void step_paper(int64_t n, double *x, double *v, const double *m,
                       double G, double eps, double dt, double *dp) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double a[3];
        accel_one(n, x, m, G, eps, i, a);
        for (int c = 0; c < 3; ++c) {
            v[3 * i + c] += a[c] * dt / 2.0;
            dp[3 * i + c] = v[3 * i + c] * dt;
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) x[3 * i + c] += dp[3 * i + c];
}

int oracle_step(int64_t n, double *x, double *v, const double *m, double G,
                double eps, double dt) {
    double *dp = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!dp) return -1;
    step_paper(n, x, v, m, G, eps, dt, dp);
    free(dp);
    return 0;
}

int oracle_run(int64_t n, double *x, double *v, const double *m, double G,
               double eps, double dt, int steps) {
    double *dp = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!dp) return -1;
    for (int t = 0; t < steps; ++t) step_paper(n, x, v, m, G, eps, dt, dp);
    free(dp);
    return 0;
}

/*
 * Velocity Verlet (kick-drift-kick), the integrator the paper names in
 * Sections 3.2.3 and 3.3.7 but does not print:
 *   v <- v + a(x) dt/2;  x <- x + v dt;  v <- v + a(x_new) dt/2.
 */
int oracle_run_kdk(int64_t n, double *x, double *v, const double *m, double G,
                   double eps, double dt, int steps) {
    double *a = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!a) return -1;
    for (int t = 0; t < steps; ++t) {
        oracle_accel(n, x, m, G, eps, n, NULL, a);
        for (int64_t k = 0; k < 3 * n; ++k) v[k] += a[k] * dt / 2.0;
        for (int64_t k = 0; k < 3 * n; ++k) x[k] += v[k] * dt;
        oracle_accel(n, x, m, G, eps, n, NULL, a);
        for (int64_t k = 0; k < 3 * n; ++k) v[k] += a[k] * dt / 2.0;
    }
    free(a);
    return 0;
}

/*
 * Diagnostics: out[0..2] = P = sum m v; out[3] = KE = 1/2 sum m |v|^2;
 * out[4] = Phi = -G sum_{i<j} m_i m_j / sqrt(|x_j - x_i|^2 + eps^2);
 * out[5] = H' = KE + Phi/2, the quantity the paper's half-kick update
 * conserves as dt -> 0 (its continuous limit is Newtonian motion under
 * half the pair force).
 */
void oracle_energy(int64_t n, const double *x, const double *v, const double *m,
                   double G, double eps, double *out) {
    double px = 0, py = 0, pz = 0, ke = 0, phi = 0;
    const double soft = eps * eps;
    for (int64_t i = 0; i < n; ++i) {
        px += m[i] * v[3 * i + 0];
        py += m[i] * v[3 * i + 1];
        pz += m[i] * v[3 * i + 2];
        ke += 0.5 * m[i] * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] +
                            v[3 * i + 2] * v[3 * i + 2]);
    }
#pragma omp parallel for schedule(static) reduction(+ : phi)
    for (int64_t i = 0; i < n; ++i) {
        double pi = 0.0;
        for (int64_t j = i + 1; j < n; ++j) {
            double dx = x[3 * j + 0] - x[3 * i + 0];
            double dy = x[3 * j + 1] - x[3 * i + 1];
            double dz = x[3 * j + 2] - x[3 * i + 2];
            pi += m[j] / sqrt(dx * dx + dy * dy + dz * dz + soft);
        }
        phi += m[i] * pi;
    }
    phi *= -G;
    out[0] = px;
    out[1] = py;
    out[2] = pz;
    out[3] = ke;
    out[4] = phi;
    out[5] = ke + 0.5 * phi;
}

/*
 * Jacobian blocks of the acceleration, written out from the chain rule.
 * With d = x_j - x_i and s = |d|^2 + eps^2:
 *   d a_i / d x_j = G m_j K(d)            (j != i)
 *   d a_i / d x_i = -sum_{j != i} G m_j K(d_ij)
 *   d a_i / d m_j = G d / s^(3/2)
 * where K(d) = s^(-3/2) I - 3 s^(-5/2) d d^T (symmetric).
 */
static void kblock(const double *d, double soft, double K[3][3], double *f) {
    double s = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + soft;
    double s32 = s * sqrt(s);
    double s52 = s32 * s;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            K[r][c] = (r == c ? 1.0 / s32 : 0.0) - 3.0 * d[r] * d[c] / s52;
    *f = 1.0 / s32;
}

/*
 * Vector-Jacobian product of a(x, m) with cotangent abar (row vector), summed
 * into xbar (n x 3) and mbar (n):
 *   xbar_k += sum_i (d a_i / d x_k)^T abar_i,   mbar_k += sum_i abar_i . d a_i / d m_k.
 * Parallel over the output index k; every Jacobian block is formed explicitly.
 */
void oracle_vjp(int64_t n, const double *x, const double *m, double G,
                double eps, const double *abar, double *xbar, double *mbar) {
    const double soft = eps * eps;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        double gx[3] = {0, 0, 0};
        double self[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        double gm = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            if (i == k) continue;
            double d[3], K[3][3], f;
            /* block d a_i / d x_k: d = x_k - x_i, weight G m_k */
            for (int c = 0; c < 3; ++c) d[c] = x[3 * k + c] - x[3 * i + c];
            kblock(d, soft, K, &f);
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c)
                    gx[r] += G * m[k] * K[c][r] * abar[3 * i + c];
            /* d a_i / d m_k = G d f with the same d */
            for (int c = 0; c < 3; ++c) gm += abar[3 * i + c] * G * d[c] * f;
            /* block d a_k / d x_k collects -G m_i K(x_i - x_k); K is even in d */
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) self[r][c] -= G * m[i] * K[r][c];
        }
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) gx[r] += self[c][r] * abar[3 * k + c];
        for (int c = 0; c < 3; ++c) xbar[3 * k + c] += gx[c];
        mbar[k] += gm;
    }
}

/*
 * Reverse-mode sweep of `steps` paper steps from (x0, v0) with masses m.
 * Forward: v' = v + dt/2 a(x), x' = x + dt v'. Given (xbar_T, vbar_T), each
 * reverse step (t = steps-1 ... 0) is
 *   vbar' = vbar + dt xbar;  abar = dt/2 vbar';
 *   xbar <- xbar + VJP_x(abar; x_t);  mbar += VJP_m(abar; x_t);  vbar <- vbar'.
 * The full position trajectory is stored (no checkpointing; small n only).
 * Outputs xbar0, vbar0 (n x 3) and mbar (n) are overwritten.
 */
int oracle_adjoint(int64_t n, const double *x0, const double *v0, const double *m,
                   double G, double eps, double dt, int steps,
                   const double *xbarT, const double *vbarT, double *xbar0,
                   double *vbar0, double *mbar) {
    size_t sz = 3 * (size_t)(n > 0 ? n : 1);
    double *traj = (double *)malloc(sizeof(double) * sz * (size_t)(steps > 0 ? steps : 1));
    double *x = (double *)malloc(sizeof(double) * sz);
    double *v = (double *)malloc(sizeof(double) * sz);
    double *dp = (double *)malloc(sizeof(double) * sz);
    double *ab = (double *)malloc(sizeof(double) * sz);
    if (!traj || !x || !v || !dp || !ab) {
        free(traj); free(x); free(v); free(dp); free(ab);
        return -1;
    }
    memcpy(x, x0, sizeof(double) * 3 * n);
    memcpy(v, v0, sizeof(double) * 3 * n);
    for (int t = 0; t < steps; ++t) {
        memcpy(traj + (size_t)t * sz, x, sizeof(double) * 3 * n);
        step_paper(n, x, v, m, G, eps, dt, dp);
    }
    memcpy(xbar0, xbarT, sizeof(double) * 3 * n);
    memcpy(vbar0, vbarT, sizeof(double) * 3 * n);
    for (int64_t k = 0; k < n; ++k) mbar[k] = 0.0;
    for (int t = steps - 1; t >= 0; --t) {
        for (int64_t k = 0; k < 3 * n; ++k) {
            vbar0[k] = vbar0[k] + dt * xbar0[k];
            ab[k] = dt / 2.0 * vbar0[k];
        }
        oracle_vjp(n, traj + (size_t)t * sz, m, G, eps, ab, xbar0, mbar);
    }
    free(traj); free(x); free(v); free(dp); free(ab);
    return 0;
}
