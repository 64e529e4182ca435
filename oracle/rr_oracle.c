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

/* ------------------------------------------------------------------------
 * Counter-based random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC 2011), written from
 * its published definition.  Ten rounds; a round multiplies the even words
 * of the counter by 0xD2511F53 and 0xCD9E8D57 (64-bit products split into
 * high and low halves), XORs the high halves with the odd words and the
 * two key words, and swaps; the key advances by the Weyl constants
 * 0x9E3779B9 and 0xBB67AE85 between rounds.
 * ---------------------------------------------------------------------- */
void rro_philox4x32(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    for (int i = 0; i < 4; ++i) out[i] = c[i];
}

/* closest hit of one ray against every triangle, t in (0, tmax); -1: none */
static int32_t rro_closest(const float *V, const int32_t *F, int64_t nt, const double o[3], const double d[3],
                           double tmax, double *t_out)
{
    double best_t = tmax;
    int32_t best = -1;
    for (int64_t f = 0; f < nt; ++f) {
        double v[3][3];
        for (int c = 0; c < 3; ++c)
            for (int x = 0; x < 3; ++x) v[c][x] = (double)V[3 * (int64_t)F[3 * f + c] + x];
        double t;
        if (rro_tri_hit(o, d, v[0], v[1], v[2], &t) && t < best_t) {
            best_t = t;
            best = (int32_t)f;
        }
    }
    *t_out = best_t;
    return best;
}

/* ------------------------------------------------------------------------
 * Stochastic material model exactly as Eq. 1-3 (Sec. III-A), with
 * multiple bounces.  For every grid ray r (direction dirs[r], solid angle
 * omega[r]) from the TX, at bounce b = 0 .. B-1:
 *   closest hit p of the current ray (none: the ray leaves the scene);
 *   n_f = unit face normal turned toward the incoming direction u;
 *   Philox4x32-10 with counter (r, b, 0, 0) and key (seed, frame) gives
 *   words x0, x1; u1 = (x0 + 1/2) / 2^32, u2 = (x1 + 1/2) / 2^32; the random
 *   unit vector (Eq. 1's r) is (s cos phi, s sin phi, z), z = 1 - 2 u1,
 *   phi = 2 pi u2, s = sqrt(1 - z^2);
 *   diffuse t_o,d = (n_f + r) / |n_f + r| (Eq. 1), mirror t_o,m = u - 2
 *   (u . n_f) n_f (Eq. 2), t_o,c = (alpha t_o,d + (1 - alpha) t_o,m)
 *   normalised (Eq. 3);
 *   Rx j receives when the angle between t_o,c and the direction w_j from p
 *   to rx_j is at most theta_r, rx_j lies in front of the face (w_j . n_f >
 *   0) and no triangle lies between (the return leg from p + eps n_f);
 *   every bounce with at least one receiving antenna is one entry: path
 *   length d_j = (legs so far) + |rx_j - p|, amplitude a_j = omega[r] /
 *   (2 pi (1 - cos theta_r)) when received, else 0 (amp_mode 1: 1 when
 *   received), path rate d-dot_j = v . (u_0 - w_j) for a rigid velocity v
 *   (the first leg lengthens by v . u_0, the last shortens by v . w_j);
 *   the ray goes on from p + eps n_f along t_o,c.
 * Entries are written in (ray, bounce) order: ray_out, bounce_out,
 * tri_out [cap], d / a / dd [n_rx][cap].  Returns the number of entries
 * (more than cap: the rest were dropped).
 * ---------------------------------------------------------------------- */
int64_t rro_stochastic(const float *V, int64_t nv, const int32_t *F, int64_t nt, const double *tx,
                       int n_rx, const double *rx, const double *vel, const double *dirs, const double *omega,
                       int64_t n_rays, double alpha, double theta_r, int bounces, uint32_t seed, uint32_t frame,
                       double eps, int amp_mode, int64_t cap, int32_t *ray_out, int32_t *bounce_out,
                       int32_t *tri_out, double *d, double *a, double *dd)
{
    (void)nv;
    const double cos_r = cos(theta_r);
    const double cone = 2.0 * M_PI * (1.0 - cos_r);
    int64_t count = 0;
    /* sequential over rays so that entries come out in (ray, bounce) order */
    for (int64_t r = 0; r < n_rays; ++r) {
        double o[3] = {tx[0], tx[1], tx[2]};
        double u[3] = {dirs[3 * r], dirs[3 * r + 1], dirs[3 * r + 2]};
        const double u0[3] = {u[0], u[1], u[2]};
        double legs = 0.0;
        for (int b = 0; b < bounces; ++b) {
            double t;
            const int32_t f = rro_closest(V, F, nt, o, u, INFINITY, &t);
            if (f < 0) break;
            const double p[3] = {o[0] + t * u[0], o[1] + t * u[1], o[2] + t * u[2]};
            legs += t;
            double v[3][3];
            for (int c = 0; c < 3; ++c)
                for (int x = 0; x < 3; ++x) v[c][x] = (double)V[3 * (int64_t)F[3 * f + c] + x];
            double e1[3], e2[3], nn[3];
            for (int x = 0; x < 3; ++x) { e1[x] = v[1][x] - v[0][x]; e2[x] = v[2][x] - v[0][x]; }
            nn[0] = e1[1] * e2[2] - e1[2] * e2[1];
            nn[1] = e1[2] * e2[0] - e1[0] * e2[2];
            nn[2] = e1[0] * e2[1] - e1[1] * e2[0];
            const double nl = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
            const double un = u[0] * nn[0] + u[1] * nn[1] + u[2] * nn[2];
            const double sg = un > 0.0 ? -1.0 / nl : 1.0 / nl;
            const double n_f[3] = {nn[0] * sg, nn[1] * sg, nn[2] * sg};
            /* Eq. 1: random point on the unit sphere */
            const uint32_t ctr[4] = {(uint32_t)r, (uint32_t)b, 0u, 0u}, key[2] = {seed, frame};
            uint32_t x[4];
            rro_philox4x32(ctr, key, x);
            const double u1 = ((double)x[0] + 0.5) / 4294967296.0, u2 = ((double)x[1] + 0.5) / 4294967296.0;
            const double z = 1.0 - 2.0 * u1, phi = 2.0 * M_PI * u2, s = sqrt(fmax(0.0, 1.0 - z * z));
            double td[3] = {n_f[0] + s * cos(phi), n_f[1] + s * sin(phi), n_f[2] + z};
            double l = sqrt(td[0] * td[0] + td[1] * td[1] + td[2] * td[2]);
            for (int xx = 0; xx < 3; ++xx) td[xx] = l > 0.0 ? td[xx] / l : n_f[xx];
            /* Eq. 2: mirror direction */
            const double c2 = 2.0 * (u[0] * n_f[0] + u[1] * n_f[1] + u[2] * n_f[2]);
            const double tm[3] = {u[0] - c2 * n_f[0], u[1] - c2 * n_f[1], u[2] - c2 * n_f[2]};
            /* Eq. 3: mixture, normalised */
            double tc[3] = {alpha * td[0] + (1.0 - alpha) * tm[0], alpha * td[1] + (1.0 - alpha) * tm[1],
                            alpha * td[2] + (1.0 - alpha) * tm[2]};
            l = sqrt(tc[0] * tc[0] + tc[1] * tc[1] + tc[2] * tc[2]);
            for (int xx = 0; xx < 3; ++xx) tc[xx] = l > 0.0 ? tc[xx] / l : n_f[xx];
            const double q[3] = {p[0] + eps * n_f[0], p[1] + eps * n_f[1], p[2] + eps * n_f[2]};
            int any = 0;
            double dj[8], aj[8], ddj[8];
            for (int j = 0; j < n_rx; ++j) {
                const double w[3] = {rx[3 * j] - p[0], rx[3 * j + 1] - p[1], rx[3 * j + 2] - p[2]};
                const double L = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
                const double wu[3] = {w[0] / L, w[1] / L, w[2] / L};
                dj[j] = legs + L;
                ddj[j] = vel[0] * (u0[0] - wu[0]) + vel[1] * (u0[1] - wu[1]) + vel[2] * (u0[2] - wu[2]);
                aj[j] = 0.0;
                const double cosang = tc[0] * wu[0] + tc[1] * wu[1] + tc[2] * wu[2];
                const double front = wu[0] * n_f[0] + wu[1] * n_f[1] + wu[2] * n_f[2];
                if (cosang >= cos_r && front > 0.0) {
                    const double ws[3] = {rx[3 * j] - q[0], rx[3 * j + 1] - q[1], rx[3 * j + 2] - q[2]};
                    const double Ls = sqrt(ws[0] * ws[0] + ws[1] * ws[1] + ws[2] * ws[2]);
                    const double wsu[3] = {ws[0] / Ls, ws[1] / Ls, ws[2] / Ls};
                    double ts;
                    if (rro_closest(V, F, nt, q, wsu, Ls, &ts) < 0) {
                        aj[j] = amp_mode == 1 ? 1.0 : omega[r] / cone;
                        any = 1;
                    }
                }
            }
            if (any) {
                if (count < cap) {
                    ray_out[count] = (int32_t)r;
                    bounce_out[count] = b;
                    tri_out[count] = f;
                    for (int j = 0; j < n_rx; ++j) {
                        d[(int64_t)j * cap + count] = dj[j];
                        a[(int64_t)j * cap + count] = aj[j];
                        dd[(int64_t)j * cap + count] = ddj[j];
                    }
                }
                ++count;
            }
            for (int xx = 0; xx < 3; ++xx) { o[xx] = q[xx]; u[xx] = tc[xx]; }
        }
    }
    return count;
}
