/*
 * rr_oracle.c -- plain FP64 CPU oracle of the radar ray-tracing hot path of
 * "A Realistic Radar Ray Tracing Simulator for Hand Pose Imaging"
 * (arXiv 2307.15412).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg load this library.  It shares no code,
 * header, table or constant generator with the CUDA library; it is written
 * to be read against the paper, not to be fast: brute-force ray-triangle
 * tests against every triangle, a direct sum over hits, direct DFTs.  All
 * arithmetic is IEEE double, compiled without FMA contraction so the x86
 * and Arm hosts give the same bits.  OpenMP only splits independent output
 * elements across threads; it changes no arithmetic.
 *
 * Conventions (shared with the library through its public header, not code):
 *   ray id       = i_el * n_az + i_az
 *   hit arrays   = [n_rx][K] per channel
 *   complex data = interleaved (re, im) doubles
 *   IF cube      = [n_rx][n_chirps][n_samples]
 *   RD cube      = [n_rx][doppler (fft-shifted)][range]
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define RRO_C 299792458.0

/* ------------------------------------------------------------------------
 * Ray generation.  The paper launches many rays from each Tx antenna
 * (Sec. III-A); the build's rays are the cell centres of a uniform
 * azimuth/elevation grid over +-half angles, expressed in the radar frame
 * (boresight +z) and rotated into the world by the row-major matrix R.
 * Each ray carries the solid angle of its cell, cos(el) d_az d_el.
 * ---------------------------------------------------------------------- */
void rro_ray_dirs(int n_az, int n_el, double half_az, double half_el,
                  const double *R, double *dirs, double *omega)
{
    const double daz = 2.0 * half_az / n_az, del = 2.0 * half_el / n_el;
    for (int j = 0; j < n_el; ++j) {
        const double el = -half_el + del * (j + 0.5);
        for (int i = 0; i < n_az; ++i) {
            const double az = -half_az + daz * (i + 0.5);
            const double u[3] = {cos(el) * sin(az), sin(el), cos(el) * cos(az)};
            double *o = dirs + 3 * ((int64_t)j * n_az + i);
            for (int r = 0; r < 3; ++r)
                o[r] = R[3 * r + 0] * u[0] + R[3 * r + 1] * u[1] + R[3 * r + 2] * u[2];
            omega[(int64_t)j * n_az + i] = cos(el) * daz * del;
        }
    }
}

/* ------------------------------------------------------------------------
 * Ray-triangle test, watertight form of Woop, Benthin and Wald (JCGT 2013),
 * in double.  Returns 1 and the ray parameter t (> 0) on a hit.  Faces are
 * two-sided.  A ray through an edge shared by two triangles sees the same
 * edge function with opposite sign from both, so it cannot slip through.
 * ---------------------------------------------------------------------- */
static int rro_tri_hit(const double o[3], const double d[3], const double v0[3],
                       const double v1[3], const double v2[3], double *t_out)
{
    int kz = 0;
    if (fabs(d[1]) > fabs(d[kz])) kz = 1;
    if (fabs(d[2]) > fabs(d[kz])) kz = 2;
    int kx = (kz + 1) % 3, ky = (kx + 1) % 3;
    if (d[kz] < 0.0) { int tmp = kx; kx = ky; ky = tmp; }
    const double Sx = d[kx] / d[kz], Sy = d[ky] / d[kz], Sz = 1.0 / d[kz];

    double A[3], B[3], C[3];
    for (int r = 0; r < 3; ++r) { A[r] = v0[r] - o[r]; B[r] = v1[r] - o[r]; C[r] = v2[r] - o[r]; }
    const double Ax = A[kx] - Sx * A[kz], Ay = A[ky] - Sy * A[kz];
    const double Bx = B[kx] - Sx * B[kz], By = B[ky] - Sy * B[kz];
    const double Cx = C[kx] - Sx * C[kz], Cy = C[ky] - Sy * C[kz];

    const double U = Cx * By - Cy * Bx;
    const double V = Ax * Cy - Ay * Cx;
    const double W = Bx * Ay - By * Ax;
    if ((U < 0.0 || V < 0.0 || W < 0.0) && (U > 0.0 || V > 0.0 || W > 0.0)) return 0;
    const double det = U + V + W;
    if (det == 0.0) return 0;
    const double T = U * (Sz * A[kz]) + V * (Sz * B[kz]) + W * (Sz * C[kz]);
    const double t = T / det;
    if (!(t > 0.0)) return 0;
    *t_out = t;
    return 1;
}

/* ------------------------------------------------------------------------
 * Closest hit of every ray against every triangle of the mesh (Sec. III:
 * the scene is a triangle mesh and rays are traced into it).  Brute force:
 * no acceleration structure.  Equal t keeps the lowest triangle id (the
 * loop runs in id order and only a strictly smaller t replaces the best).
 * Miss: tri = -1, t = 0.
 * ---------------------------------------------------------------------- */
void rro_trace(const float *V, int64_t nv, const int32_t *F, int64_t nt,
               const double *origin, const double *dirs, int64_t n_rays,
               int32_t *hit_tri, double *hit_t)
{
    (void)nv;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < n_rays; ++r) {
        const double *d = dirs + 3 * r;
        double best_t = INFINITY;
        int32_t best = -1;
        for (int64_t f = 0; f < nt; ++f) {
            double v[3][3];
            for (int c = 0; c < 3; ++c)
                for (int x = 0; x < 3; ++x) v[c][x] = (double)V[3 * (int64_t)F[3 * f + c] + x];
            double t;
            if (rro_tri_hit(origin, d, v[0], v[1], v[2], &t) && t < best_t) {
                best_t = t;
                best = (int32_t)f;
            }
        }
        hit_tri[r] = best;
        hit_t[r] = best < 0 ? 0.0 : best_t;
    }
}

/* ------------------------------------------------------------------------
 * Echo of one hit seen by each receive antenna (single bounce).
 *
 * Material model, Sec. III-A: the outgoing direction mixes a diffuse
 * direction n + r (Eq. 1, r uniform on the unit sphere) and the mirror
 * direction given by the law of reflection (Eq. 2, read as
 * t_o,m = t_i - 2 (t_i . n) n), with weight alpha (Eq. 3).  The hot path
 * uses the deterministic amplitude each lobe sends toward an antenna:
 *   specular lobe  s = max(0, t_o,m . w)^m_s,  w the unit vector hit -> Rx
 *   diffuse lobe   l = c_i * c_o  (the expected Lambertian return)
 *   g = (1 - alpha) s + alpha l  (Eq. 3's mixture applied to the lobes)
 * with c_i, c_o the cosines of the incident and outgoing directions against
 * the face normal turned toward the ray (two-sided faces).  No return when
 * the antenna lies behind the face.  Amplitude a = Omega g / (t r), t and r
 * the two legs; amp_mode 1 selects Eq. 4's unit amplitude per received ray.
 * Path length d = t + r (Sec. III-B: total path length per received ray),
 * path rate d-dot = v . (u + u_rx) for a rigid velocity v.
 * ---------------------------------------------------------------------- */
void rro_echo(int64_t K, const double *origin, const double *dirs, const double *t,
              const int32_t *tri, const double *omega, const float *V, const int32_t *F,
              int n_rx, const double *rx, const double *vel, double alpha, double spec_exp,
              int amp_mode, double *d_out, double *a_out, double *ddot_out)
{
    for (int64_t k = 0; k < K; ++k) {
        const double *u = dirs + 3 * k;
        double v[3][3];
        for (int c = 0; c < 3; ++c)
            for (int x = 0; x < 3; ++x) v[c][x] = (double)V[3 * (int64_t)F[3 * (int64_t)tri[k] + c] + x];
        const double e1[3] = {v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2]};
        const double e2[3] = {v[2][0] - v[0][0], v[2][1] - v[0][1], v[2][2] - v[0][2]};
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                       e1[0] * e2[1] - e1[1] * e2[0]};
        const double nl = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int x = 0; x < 3; ++x) n[x] /= nl;
        const double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
        if (un > 0.0)
            for (int x = 0; x < 3; ++x) n[x] = -n[x];
        const double ci = -(u[0] * n[0] + u[1] * n[1] + u[2] * n[2]);
        /* Eq. 2 mirror direction */
        const double un_f = -ci;
        const double m[3] = {u[0] - 2.0 * un_f * n[0], u[1] - 2.0 * un_f * n[1], u[2] - 2.0 * un_f * n[2]};
        const double p[3] = {origin[0] + t[k] * u[0], origin[1] + t[k] * u[1], origin[2] + t[k] * u[2]};
        for (int j = 0; j < n_rx; ++j) {
            const double w[3] = {p[0] - rx[3 * j], p[1] - rx[3 * j + 1], p[2] - rx[3 * j + 2]};
            const double r = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
            const double ur[3] = {w[0] / r, w[1] / r, w[2] / r};  /* Rx -> hit */
            const double co = -(ur[0] * n[0] + ur[1] * n[1] + ur[2] * n[2]);
            double g = 0.0;
            if (co > 0.0) {
                const double sdot = -(m[0] * ur[0] + m[1] * ur[1] + m[2] * ur[2]);
                const double s = sdot > 0.0 ? pow(sdot, spec_exp) : 0.0;
                const double l = ci * co;
                g = (1.0 - alpha) * s + alpha * l;
            }
            const int64_t o = (int64_t)j * K + k;
            d_out[o] = t[k] + r;
            a_out[o] = amp_mode == 1 ? 1.0 : omega[k] * g / (t[k] * r);
            ddot_out[o] = vel[0] * (u[0] + ur[0]) + vel[1] * (u[1] + ur[1]) + vel[2] * (u[2] + ur[2]);
        }
    }
}

/* ------------------------------------------------------------------------
 * IF synthesis, Eq. 4 (Sec. III-B): the baseband value of each frequency
 * step is the coherent sum over received rays of exp(-j 2 pi f d_i / c).
 * FMCW form: sample n of chirp m sees f = f0 + S t_n, t_n = n dt, and each
 * path moves with its rate (stop-and-hop): d(m) = d + d-dot m T_rep.  Each
 * hit carries its amplitude a.
 *   s[j][m][n] = sum_k a_kj exp(-j 2 pi (f0 + S t_n) (d_kj + ddot_kj m T_rep) / c)
 * Inputs are [n_rx][K] doubles; out is [n_rx][M][N] interleaved complex.
 * ---------------------------------------------------------------------- */
void rro_synth(int64_t K, int n_rx, const double *d, const double *a, const double *ddot,
               double f0, double slope, double dt, double t_rep, int M, int N, double *out)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int j = 0; j < n_rx; ++j) {
        for (int m = 0; m < M; ++m) {
            for (int n = 0; n < N; ++n) {
                const double f = f0 + slope * (n * dt);
                double re = 0.0, im = 0.0;
                for (int64_t k = 0; k < K; ++k) {
                    const int64_t o = (int64_t)j * K + k;
                    const double dm = d[o] + ddot[o] * (m * t_rep);
                    const double ph = 2.0 * M_PI * f * dm / RRO_C;
                    re += a[o] * cos(ph);
                    im -= a[o] * sin(ph);
                }
                double *y = out + 2 * (((int64_t)j * M + m) * N + n);
                y[0] = re;
                y[1] = im;
            }
        }
    }
}

static double rro_window(int kind, int i, int L)
{
    if (kind == 1 && L > 1) return 0.5 - 0.5 * cos(2.0 * M_PI * i / (L - 1));
    return 1.0;
}

/* ------------------------------------------------------------------------
 * Range-Doppler map: 2-D DFT with the + kernel over samples (range) and
 * chirps (Doppler) of the windowed IF cube, Doppler axis fft-shifted.
 *   X[j][q][k] = sum_m sum_n w_M(m) w_N(n) s[j][m][n] exp(+j 2 pi (k n / N + q m / M))
 *   out[j][(q + M/2) mod M][k] = X[j][q][k]
 * With exp(-j 2 pi f d / c) in the IF, a path d lands in range bin B d / c and
 * a path rate d-dot in Doppler bin f0 d-dot T_rep M / c.  window: 0
 * rectangular, 1 symmetric Hann.  Written as the two nested direct sums.
 * ---------------------------------------------------------------------- */
void rro_range_doppler(int n_rx, int M, int N, const double *in, int window, double *out)
{
    double *Y = (double *)malloc(sizeof(double) * 2 * (size_t)n_rx * M * N);
#pragma omp parallel for collapse(2) schedule(static)
    for (int j = 0; j < n_rx; ++j)
        for (int m = 0; m < M; ++m)
            for (int k = 0; k < N; ++k) {
                double re = 0.0, im = 0.0;
                for (int n = 0; n < N; ++n) {
                    const double *x = in + 2 * (((int64_t)j * M + m) * N + n);
                    const double w = rro_window(window, n, N);
                    const double ang = 2.0 * M_PI * (double)(((int64_t)k * n) % N) / N;
                    const double c = cos(ang), s = sin(ang);
                    re += w * (x[0] * c - x[1] * s);
                    im += w * (x[0] * s + x[1] * c);
                }
                double *y = Y + 2 * (((int64_t)j * M + m) * N + k);
                y[0] = re;
                y[1] = im;
            }
#pragma omp parallel for collapse(2) schedule(static)
    for (int j = 0; j < n_rx; ++j)
        for (int q = 0; q < M; ++q)
            for (int k = 0; k < N; ++k) {
                double re = 0.0, im = 0.0;
                for (int m = 0; m < M; ++m) {
                    const double *x = Y + 2 * (((int64_t)j * M + m) * N + k);
                    const double w = rro_window(window, m, M);
                    const double ang = 2.0 * M_PI * (double)(((int64_t)q * m) % M) / M;
                    const double c = cos(ang), s = sin(ang);
                    re += w * (x[0] * c - x[1] * s);
                    im += w * (x[0] * s + x[1] * c);
                }
                const int qs = (q + M / 2) % M;
                double *y = out + 2 * (((int64_t)j * M + qs) * N + k);
                y[0] = re;
                y[1] = im;
            }
    free(Y);
}

int rro_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
