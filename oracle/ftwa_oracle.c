/*
 * Plain FP64 CPU oracle for the fermionic truncated Wigner approximation
 * (fTWA) of the Fermi-Hubbard model, after Rousse, Eriksson and Ogren,
 * "Correlated quantum dynamics of graphene" (arXiv:2212.04352).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA library is checked against.  It shares no code,
 * header, table or helper with the CUDA library; only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.
 *
 * State layout (oracle-private): rho[s][i][j] complex, s = 0 (up), 1 (down),
 * full N x N matrix per spin, C99 double complex.
 *
 * What is computed, in the paper's order:
 *   1. Hamiltonian of Eq. 1 (FHeq1) with j_ij = t_b on bond b (both orders)
 *      and u_ij = U delta_ij (Sec. II).
 *   2. Initial Gaussian Wigner sample of Eq. 7 (ic_fTWA): rho_ii = n_i - 1/2,
 *      rho_ij = xi_ij sqrt((n_i + n_j - 2 n_i n_j)/2) for i < j, rho_ji =
 *      conj(rho_ij), with xi complex normal, E|xi|^2 = 1 (the covariance of
 *      App. A.3, Eqs. A11-A12).
 *   3. Equation of motion Eq. 6 (drho), integrated with classical RK4 (the
 *      paper states no integrator; RK4 with dt = 0.01 is the reading used).
 *   4. Estimators of Eq. 5 (fTWA_moments) and Eq. 10 (g2_fTWA) as sample
 *      means, plus the connected correlator as a two-pass covariance.
 *   5. The classical energy H_W of Eq. A10 (ftwa_h), conserved per trajectory.
 *
 * Random numbers (the paper names no generator): Philox4x32-10 from its
 * published definition (Salmon, Moraes, Dror, Shaw, SC'11), key = (seed_lo,
 * seed_hi), counter = (m_lo, m_hi, spin, pair index p(i,j) = i N - i(i+1)/2 +
 * j - i - 1 for i < j), then Box-Muller on two 53-bit uniforms in (0, 1).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 4.2).                     */
/* ------------------------------------------------------------------ */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;   /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;   /* Weyl key increments */
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(M0, c0, &hi0, &lo0);
        mulhilo32(M1, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Raw generator output for `count` consecutive pair indices, for the
 * bit-exact comparison of the integer stage. */
void orc_philox_block(uint64_t seed, int64_t m, int32_t spin, int64_t p0, int64_t count, uint32_t *out)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t q = 0; q < count; ++q) {
        uint64_t p = (uint64_t)(p0 + q);
        uint32_t ctr[4] = {(uint32_t)m, (uint32_t)((uint64_t)m >> 32), (uint32_t)spin, (uint32_t)p};
        orc_philox4x32_10(ctr, key, out + 4 * q);
    }
}

/* Standard complex normal xi = (a + i b)/sqrt(2), a, b ~ N(0, 1) i.i.d.,
 * from the four Philox words by Box-Muller. */
static cplx complex_normal(uint64_t seed, int64_t m, int spin, uint32_t p)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)m, (uint32_t)((uint64_t)m >> 32), (uint32_t)spin, p};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    uint64_t b1 = ((uint64_t)w[1] << 32) | w[0];
    uint64_t b2 = ((uint64_t)w[3] << 32) | w[2];
    double u1 = (double)(b1 >> 11) * 0x1p-53 + 0x1p-54;
    double u2 = (double)(b2 >> 11) * 0x1p-53 + 0x1p-54;
    double r = sqrt(-2.0 * log(u1));
    double a = r * cos(2.0 * M_PI * u2);
    double b = r * sin(2.0 * M_PI * u2);
    return (a + I * b) / sqrt(2.0);
}

void orc_normals(int32_t N, uint64_t seed, int64_t m, double *xi /* [2][N][N] complex, upper only */)
{
    cplx *x = (cplx *)xi;
    memset(x, 0, sizeof(cplx) * 2 * (size_t)N * N);
    for (int s = 0; s < 2; ++s)
        for (int i = 0; i < N; ++i)
            for (int j = i + 1; j < N; ++j) {
                uint32_t p = (uint32_t)(i * N - i * (i + 1) / 2 + (j - i - 1));
                x[((size_t)s * N + i) * N + j] = complex_normal(seed, m, s, p);
            }
}

/* Eq. 7: one Gaussian Wigner sample of the diagonal state n (per spin). */
void orc_sample(int32_t N, const double *n_up, const double *n_dn, uint64_t seed, int64_t m,
                double *rho_out)
{
    cplx *rho = (cplx *)rho_out;
    for (int s = 0; s < 2; ++s) {
        const double *n = s == 0 ? n_up : n_dn;
        cplx *r = rho + (size_t)s * N * N;
        for (int i = 0; i < N; ++i) {
            r[(size_t)i * N + i] = n[i] - 0.5;
            for (int j = i + 1; j < N; ++j) {
                uint32_t p = (uint32_t)(i * N - i * (i + 1) / 2 + (j - i - 1));
                double var = (n[i] + n[j] - 2.0 * n[i] * n[j]) / 2.0;
                double sd = sqrt(var > 0.0 ? var : 0.0);
                cplx xi = complex_normal(seed, m, s, p);
                r[(size_t)i * N + j] = xi * sd;
                r[(size_t)j * N + i] = conj(xi) * sd;
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Lattice: neighbour lists j_ik of Eq. 1 built from the bond list.    */
/* ------------------------------------------------------------------ */
typedef struct {
    int N;
    int *start;     /* [N+1] */
    int *nbr;       /* [2B] */
    double *hop;    /* [2B] j_ik for k = nbr[.] */
} adjacency;

static adjacency build_adjacency(int N, int B, const int32_t *bonds, const double *t_bond)
{
    adjacency a;
    a.N = N;
    a.start = calloc((size_t)N + 1, sizeof(int));
    a.nbr = malloc(sizeof(int) * (size_t)(2 * B + 1));
    a.hop = malloc(sizeof(double) * (size_t)(2 * B + 1));
    int *fill = calloc((size_t)N, sizeof(int));
    for (int b = 0; b < B; ++b) {
        a.start[bonds[2 * b] + 1]++;
        a.start[bonds[2 * b + 1] + 1]++;
    }
    for (int i = 0; i < N; ++i) a.start[i + 1] += a.start[i];
    /* bonds are visited in list order, so each site's neighbours appear in
     * bond order */
    for (int b = 0; b < B; ++b) {
        int i = bonds[2 * b], j = bonds[2 * b + 1];
        a.nbr[a.start[i] + fill[i]] = j; a.hop[a.start[i] + fill[i]] = t_bond[b]; fill[i]++;
        a.nbr[a.start[j] + fill[j]] = i; a.hop[a.start[j] + fill[j]] = t_bond[b]; fill[j]++;
    }
    free(fill);
    return a;
}

static void free_adjacency(adjacency *a)
{
    free(a->start); free(a->nbr); free(a->hop);
}

/* Eq. 6 (drho), for both spins:
 *   d/dt rho_ij,s = i sum_k ( j_jk rho_ik,s - j_ki rho_kj,s
 *                            + (u_ki - u_kj)(rho_kk,sbar + 1/2) rho_ij,s )
 * With u_ij = U delta_ij the k-sum of the interaction term reduces to
 * U [(rho_ii,sbar + 1/2) - (rho_jj,sbar + 1/2)]. */
static void rhs(const adjacency *a, double U, double hs, const cplx *rho, cplx *f)
{
    const int N = a->N;
    for (int s = 0; s < 2; ++s) {
        const cplx *r = rho + (size_t)s * N * N;
        const cplx *rb = rho + (size_t)(1 - s) * N * N;
        cplx *o = f + (size_t)s * N * N;
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                cplx acc = 0.0;
                for (int e = a->start[j]; e < a->start[j + 1]; ++e)       /* j_jk rho_ik */
                    acc += a->hop[e] * r[(size_t)i * N + a->nbr[e]];
                for (int e = a->start[i]; e < a->start[i + 1]; ++e)       /* j_ki rho_kj */
                    acc -= a->hop[e] * r[(size_t)a->nbr[e] * N + j];
                acc *= hs;                                                /* hopping scale m(t) */
                cplx ui = U * (rb[(size_t)i * N + i] + 0.5);
                cplx uj = U * (rb[(size_t)j * N + j] + 0.5);
                acc += (ui - uj) * r[(size_t)i * N + j];
                o[(size_t)i * N + j] = I * acc;
            }
    }
}

/* Time-dependent on-site potential (the time-dependent Hamiltonians of
 * Sec. III, written as h_ii(t) += v_i,s(t)): v_i,s(t) = amp[s][i] f(t) with
 * the pulse f(t) = exp(-(t - t0)^2 / (2 sigma^2)) cos(omega (t - t0) + phase)
 * (sigma <= 0: no envelope).  It adds i (v_i,s - v_j,s) rho_ij,s to Eq. 6,
 * the same form as the U term. */
typedef struct {
    const double *amp;   /* [2][N] or NULL */
    double t0, sigma, omega, phase;
    /* hopping modulation j_ij(t) = j_ij m(t), m(t) = 1 + eps g(t) with g the
     * same pulse shape and its own parameters (eps = 0: none) */
    double hop_eps, hop_t0, hop_sigma, hop_omega, hop_phase;
} drive;

static double pulse(double t, double t0, double sigma, double omega, double phase)
{
    const double env = sigma > 0.0 ? exp(-(t - t0) * (t - t0) / (2.0 * sigma * sigma)) : 1.0;
    return env * cos(omega * (t - t0) + phase);
}

static double drive_f(const drive *d, double t) { return pulse(t, d->t0, d->sigma, d->omega, d->phase); }

static double hop_scale(const drive *d, double t)
{
    if (!d || d->hop_eps == 0.0) return 1.0;
    return 1.0 + d->hop_eps * pulse(t, d->hop_t0, d->hop_sigma, d->hop_omega, d->hop_phase);
}

static void add_drive(int N, const drive *d, double t, const cplx *rho, cplx *f)
{
    if (!d || !d->amp) return;
    const double ft = drive_f(d, t);
    for (int s = 0; s < 2; ++s)
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                const size_t e = ((size_t)s * N + i) * N + j;
                f[e] += I * ft * (d->amp[s * N + i] - d->amp[s * N + j]) * rho[e];
            }
}

/* Eq. 6 with a general (symmetric) interaction matrix u_ij of Eq. 1:
 *   d/dt rho_ij,s = i sum_k ( j_jk rho_ik,s - j_ki rho_kj,s
 *                            + (u_ki - u_kj)(rho_kk,sbar + 1/2) rho_ij,s ),
 * the interaction sum taken literally over k. */
static void rhs_longrange(const adjacency *a, const double *u, const cplx *rho, cplx *f)
{
    const int N = a->N;
    for (int s = 0; s < 2; ++s) {
        const cplx *r = rho + (size_t)s * N * N;
        const cplx *rb = rho + (size_t)(1 - s) * N * N;
        cplx *o = f + (size_t)s * N * N;
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                cplx acc = 0.0;
                for (int e = a->start[j]; e < a->start[j + 1]; ++e)
                    acc += a->hop[e] * r[(size_t)i * N + a->nbr[e]];
                for (int e = a->start[i]; e < a->start[i + 1]; ++e)
                    acc -= a->hop[e] * r[(size_t)a->nbr[e] * N + j];
                cplx w = 0.0;
                for (int k = 0; k < N; ++k)
                    w += (u[(size_t)k * N + i] - u[(size_t)k * N + j]) * (rb[(size_t)k * N + k] + 0.5);
                acc += w * r[(size_t)i * N + j];
                o[(size_t)i * N + j] = I * acc;
            }
    }
}

/* RK4 integration of one state under rhs_longrange (snapshots as orc_evolve). */
void orc_evolve_longrange(int32_t N, int32_t B, const int32_t *bonds, const double *t_bond, const double *u,
                          double dt, int64_t n_steps, int64_t out_every, double *rho_in, double *snap)
{
    adjacency a = build_adjacency(N, B, bonds, t_bond);
    const size_t n = 2 * (size_t)N * N;
    cplx *y = (cplx *)rho_in;
    cplx *k = malloc(sizeof(cplx) * n), *ys = malloc(sizeof(cplx) * n), *acc = malloc(sizeof(cplx) * n);
    int64_t row = 0;
    for (int64_t step = 0; step <= n_steps; ++step) {
        if (snap && out_every > 0 && step % out_every == 0) {
            for (int s = 0; s < 2; ++s)
                for (int i = 0; i < N; ++i) snap[row * 2 * N + s * N + i] = creal(y[((size_t)s * N + i) * N + i]);
            row++;
        }
        if (step == n_steps) break;
        rhs_longrange(&a, u, y, k);
        for (size_t e = 0; e < n; ++e) { acc[e] = k[e]; ys[e] = y[e] + 0.5 * dt * k[e]; }
        rhs_longrange(&a, u, ys, k);
        for (size_t e = 0; e < n; ++e) { acc[e] += 2.0 * k[e]; ys[e] = y[e] + 0.5 * dt * k[e]; }
        rhs_longrange(&a, u, ys, k);
        for (size_t e = 0; e < n; ++e) { acc[e] += 2.0 * k[e]; ys[e] = y[e] + dt * k[e]; }
        rhs_longrange(&a, u, ys, k);
        for (size_t e = 0; e < n; ++e) y[e] += dt / 6.0 * (acc[e] + k[e]);
    }
    free(k); free(ys); free(acc);
    free_adjacency(&a);
}

void orc_rhs(int32_t N, int32_t B, const int32_t *bonds, const double *t_bond, double U,
             const double *rho, double *f)
{
    adjacency a = build_adjacency(N, B, bonds, t_bond);
    rhs(&a, U, 1.0, (const cplx *)rho, (cplx *)f);
    free_adjacency(&a);
}

/* Classical fourth-order Runge-Kutta step of Eq. 6, both spins together,
 * from time t (stage times t, t + dt/2, t + dt/2, t + dt for the drive). */
static void rk4_step(const adjacency *a, double U, double dt, cplx *y, cplx *k, cplx *ys, cplx *acc,
                     const drive *d, double t)
{
    const size_t n = 2 * (size_t)a->N * a->N;
    rhs(a, U, hop_scale(d, t), y, k);                        /* k1 = f(t, y) */
    add_drive(a->N, d, t, y, k);
    for (size_t e = 0; e < n; ++e) { acc[e] = k[e]; ys[e] = y[e] + 0.5 * dt * k[e]; }
    rhs(a, U, hop_scale(d, t + 0.5 * dt), ys, k);            /* k2 = f(t + dt/2, y + dt/2 k1) */
    add_drive(a->N, d, t + 0.5 * dt, ys, k);
    for (size_t e = 0; e < n; ++e) { acc[e] += 2.0 * k[e]; ys[e] = y[e] + 0.5 * dt * k[e]; }
    rhs(a, U, hop_scale(d, t + 0.5 * dt), ys, k);            /* k3 = f(t + dt/2, y + dt/2 k2) */
    add_drive(a->N, d, t + 0.5 * dt, ys, k);
    for (size_t e = 0; e < n; ++e) { acc[e] += 2.0 * k[e]; ys[e] = y[e] + dt * k[e]; }
    rhs(a, U, hop_scale(d, t + dt), ys, k);                  /* k4 = f(t + dt, y + dt k3) */
    add_drive(a->N, d, t + dt, ys, k);
    for (size_t e = 0; e < n; ++e) y[e] += dt / 6.0 * (acc[e] + k[e]);
}

/* Integrate one trajectory for n_steps steps from time t_start.  snap
 * (optional) receives Re rho_ii,s at steps 0, out_every, 2 out_every, ... as
 * [n_out][2N] (s-major: index s*N + i). */
static void evolve_one(const adjacency *a, double U, double dt, int64_t n_steps, int64_t out_every,
                       cplx *y, double *snap, int64_t snap_stride, const drive *d, double t_start)
{
    const int N = a->N;
    const size_t n = 2 * (size_t)N * N;
    cplx *k = malloc(sizeof(cplx) * n), *ys = malloc(sizeof(cplx) * n), *acc = malloc(sizeof(cplx) * n);
    int64_t row = 0;
    for (int64_t step = 0; step <= n_steps; ++step) {
        if (snap && out_every > 0 && step % out_every == 0) {
            for (int s = 0; s < 2; ++s)
                for (int i = 0; i < N; ++i)
                    snap[row * snap_stride + s * N + i] = creal(y[((size_t)s * N + i) * N + i]);
            row++;
        }
        if (step < n_steps) rk4_step(a, U, dt, y, k, ys, acc, d, t_start + (double)step * dt);
    }
    free(k); free(ys); free(acc);
}

void orc_evolve(int32_t N, int32_t B, const int32_t *bonds, const double *t_bond, double U, double dt,
                int64_t n_steps, int64_t out_every, double *rho, double *snap)
{
    adjacency a = build_adjacency(N, B, bonds, t_bond);
    evolve_one(&a, U, dt, n_steps, out_every, (cplx *)rho, snap, 2 * N, NULL, 0.0);
    free_adjacency(&a);
}

/* orc_evolve with the time-dependent on-site drive, from time t_start. */
void orc_evolve_drive(int32_t N, int32_t B, const int32_t *bonds, const double *t_bond, double U, double dt,
                      int64_t n_steps, int64_t out_every, double *rho, double *snap, const double *amp,
                      double t_start, double t0, double sigma, double omega, double phase, double hop_eps,
                      double hop_t0, double hop_sigma, double hop_omega, double hop_phase)
{
    adjacency a = build_adjacency(N, B, bonds, t_bond);
    drive d = {amp, t0, sigma, omega, phase, hop_eps, hop_t0, hop_sigma, hop_omega, hop_phase};
    evolve_one(&a, U, dt, n_steps, out_every, (cplx *)rho, snap, 2 * N, &d, t_start);
    free_adjacency(&a);
}

/* Sample and integrate trajectories m0 .. m0+M-1 (OpenMP over samples).
 * snap: [n_out][M][2N] with n_out = n_steps/out_every + 1 (may be NULL).
 * rho_final: [M][2][N][N] complex (may be NULL). */
int orc_run(int32_t N, int32_t B, const int32_t *bonds, const double *t_bond, double U,
            const double *n_up, const double *n_dn, uint64_t seed, int64_t m0, int64_t M,
            double dt, int64_t n_steps, int64_t out_every, double *snap, double *rho_final,
            int32_t n_threads)
{
    adjacency a = build_adjacency(N, B, bonds, t_bond);
    const int64_t n_out = out_every > 0 ? n_steps / out_every + 1 : 0;
    const size_t n = 2 * (size_t)N * N;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t mm = 0; mm < M; ++mm) {
        cplx *y = malloc(sizeof(cplx) * n);
        double *sn = snap ? malloc(sizeof(double) * (size_t)n_out * 2 * N) : NULL;
        orc_sample(N, n_up, n_dn, seed, m0 + mm, (double *)y);
        evolve_one(&a, U, dt, n_steps, out_every, y, sn, 2 * N, NULL, 0.0);
        if (sn) {
            for (int64_t r = 0; r < n_out; ++r)
                memcpy(snap + ((size_t)r * M + mm) * 2 * N, sn + (size_t)r * 2 * N, sizeof(double) * 2 * N);
            free(sn);
        }
        if (rho_final) memcpy(rho_final + (size_t)mm * 2 * n, y, sizeof(cplx) * n);
        free(y);
    }
    free_adjacency(&a);
    return 0;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Eq. A10 (ftwa_h): H_W = - sum_{ij s} j_ij rho_ij,s
 *                        + sum_{i>=j} u_ij (rho_ii,up + 1/2)(rho_jj,dn + 1/2),
 * with u_ij = U delta_ij.  Returned as a complex pair (re, im). */
void orc_energy(int32_t N, int32_t B, const int32_t *bonds, const double *t_bond, double U,
                const double *rho_in, double *out)
{
    const cplx *rho = (const cplx *)rho_in;
    cplx h = 0.0;
    for (int s = 0; s < 2; ++s)
        for (int b = 0; b < B; ++b) {
            int i = bonds[2 * b], j = bonds[2 * b + 1];
            h -= t_bond[b] * (rho[((size_t)s * N + i) * N + j] + rho[((size_t)s * N + j) * N + i]);
        }
    for (int i = 0; i < N; ++i)
        h += U * (rho[(size_t)i * N + i] + 0.5) * (rho[((size_t)N + i) * N + i] + 0.5);
    out[0] = creal(h);
    out[1] = cimag(h);
}

/* Estimators, two passes in FP64 over X[t][m][k] = Re rho_kk (k = s*N + i):
 *   occ[t][k]      = mean_m X + 1/2                         (Eq. 5, first line)
 *   conn[t][k][l]  = (1/M) sum_m (X_k - mu_k)(X_l - mu_l)     (connected <n n>)
 *   g2[t][k][l]    = mean((X_k + 1/2)(X_l + 1/2)) / (occ_k occ_l)   (Eq. 10)
 * g2 may be NULL. */
void orc_moments(int64_t T, int64_t M, int64_t K, const double *X, double *occ, double *conn, double *g2)
{
    for (int64_t t = 0; t < T; ++t) {
        const double *x = X + (size_t)t * M * K;
        double *mu = calloc((size_t)K, sizeof(double));
        for (int64_t m = 0; m < M; ++m)
            for (int64_t k = 0; k < K; ++k) mu[k] += x[m * K + k];
        for (int64_t k = 0; k < K; ++k) {
            mu[k] /= (double)M;
            occ[t * K + k] = mu[k] + 0.5;
        }
        /* entries are independent: one thread per row k (same sums, same order) */
#pragma omp parallel for schedule(dynamic)
        for (int64_t k = 0; k < K; ++k)
            for (int64_t l = 0; l < K; ++l) {
                double c = 0.0, g = 0.0;
                for (int64_t m = 0; m < M; ++m) {
                    c += (x[m * K + k] - mu[k]) * (x[m * K + l] - mu[l]);
                    g += (x[m * K + k] + 0.5) * (x[m * K + l] + 0.5);
                }
                conn[((size_t)t * K + k) * K + l] = c / (double)M;
                if (g2) g2[((size_t)t * K + k) * K + l] = (g / (double)M) / ((mu[k] + 0.5) * (mu[l] + 0.5));
            }
        free(mu);
    }
}
