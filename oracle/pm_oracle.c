/*
 * pm_oracle.c -- plain, slow, FP64 CPU oracle of one relativistic
 * particle-mesh step (gevolution 2.0, arxiv 2607.17929, Sec. 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Everything is written the obvious way: full complex 3D DFTs (own
 * recursive mixed-radix FFT), sequential sums, one loop per equation.
 * Loops whose iterations are independent (the lines of an FFT pass, mesh
 * cells, particles of the kick and drift) carry OpenMP pragmas: there are no
 * parallel reductions, so every result is bit-identical for any thread
 * count (or_set_threads; built without OpenMP the pragmas are ignored).
 * Mesh arrays are [z][y][x] with x fastest; positions are absolute box
 * coordinates in [0,1) (box length L = 1, c = 1).
 *
 * Readings of the paper used here (the paper prints continuum equations only):
 *  - units: 4 pi G = 3/2 H0^2 (critical density today = 1), particle mass
 *    m = Omega_m / N_p, per-mass momentum u = q/m, E = sqrt(a^2 + u^2);
 *  - CIC on a vertex-centred mesh, cell i = floor(x N), weights (1-f, f);
 *  - gradients: centred differences, then CIC interpolation (Sec. 4.4
 *    "second-order gradients for force interpolation");
 *  - the Laplacian eigenvalue ktilde^2 = sum_i (2N sin(pi n_i/N))^2 and
 *    ktilde_i = 2N sin(pi n_i/N) for the projection operators;
 *  - quadratic terms in phi, psi are taken from the previous step, with no
 *    predictor-corrector iterations (Sec. 3.1);
 *  - Nyquist modes (any |n_i| = N/2) are removed from chi, B and h.
 *  Two variants of the solve, each off by default:
 *  - full Hamiltonian constraint (Eq. fullHc): the terms of Eq. fullHc that
 *    are not linear in phi, psi move into the source of the linear solve,
 *    evaluated once on the previous step's phi, psi and phi' (the paper's
 *    predictor with no corrector iterations, Sec. 3.1);
 *  - B_i from the trace-free space-space equation (Eq. spacespace): its
 *    spin-1 part (d_tau + 2 Hc) B_j = W_j, integrated as d(a^2 B)/dtau = a^2 W
 *    with W at the new time (backward Euler); the first step takes B from
 *    the momentum constraint to start the integration.
 */
#include <complex.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------ */
/* Background: conformal Hubble rate and conformal time (Eq. fullHc defines  */
/* Hc = d ln a / d tau; flat LCDM, no radiation).                            */
/* ------------------------------------------------------------------------ */

double or_conformal_hubble(double a, double omega_m, double h0)
{
    return a * h0 * sqrt(omega_m / (a * a * a) + (1.0 - omega_m));
}

/* dtau/da = 1 / (a Hc(a)) */
static double dtau_da(double a, double omega_m, double h0)
{
    return 1.0 / (a * or_conformal_hubble(a, omega_m, h0));
}

/* 64-point Gauss-Legendre nodes and weights on [-1,1], found by Newton's
 * method on the Legendre polynomial P_64 (three-term recurrence). */
static double gl_x[64], gl_w[64];
static int gl_ready = 0;

static void gl_init(void)
{
    const int n = 64;
    for (int i = 0; i < n; i++) {
        double x = cos(PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) {
                /* recompute derivative at the converged node for the weight */
                p0 = 1.0; p1 = x;
                for (int k = 2; k <= n; k++) {
                    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                dp = n * (x * p1 - p0) / (x * x - 1.0);
                gl_x[i] = x;
                gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
                break;
            }
        }
    }
    gl_ready = 1;
}

/* tau(a1) - tau(a0) = int_{a0}^{a1} da / (a Hc(a)), 64-point Gauss-Legendre */
double or_tau_between(double a0, double a1, double omega_m, double h0)
{
    if (!gl_ready) gl_init();
    double mid = 0.5 * (a0 + a1), half = 0.5 * (a1 - a0), s = 0.0;
    for (int i = 0; i < 64; i++) s += gl_w[i] * dtau_da(mid + half * gl_x[i], omega_m, h0);
    return s * half;
}

/* a such that tau(a) - tau(a0) = dtau, by Newton's method on the integral */
double or_a_after(double a0, double dtau, double omega_m, double h0)
{
    double a = a0 * exp(dtau * or_conformal_hubble(a0, omega_m, h0));
    for (int it = 0; it < 60; it++) {
        double g = or_tau_between(a0, a, omega_m, h0) - dtau;
        double da = g / dtau_da(a, omega_m, h0);
        a -= da;
        if (fabs(da) <= 1e-17 * a) break;
    }
    return a;
}

/* Step schedule: a_n = a_i (a_f/a_i)^(n/nsteps), dtau_n = tau(a_{n+1}) - tau(a_n),
 * a_half_n = a(tau_n + dtau_n/2).  Arrays: a_n[nsteps+1], dtau[nsteps], a_half[nsteps]. */
void or_schedule(int nsteps, double a_i, double a_f, double omega_m, double h0,
                 double *a_n, double *dtau, double *a_half)
{
    for (int n = 0; n <= nsteps; n++) a_n[n] = a_i * pow(a_f / a_i, (double)n / nsteps);
    for (int n = 0; n < nsteps; n++) {
        dtau[n] = or_tau_between(a_n[n], a_n[n + 1], omega_m, h0);
        a_half[n] = or_a_after(a_n[n], 0.5 * dtau[n], omega_m, h0);
    }
}

/* ------------------------------------------------------------------------ */
/* FFT: recursive decimation in time over the smallest prime factor, with a  */
/* direct sum for the butterflies.  sign = -1 forward, +1 inverse; no         */
/* normalisation.                                                            */
/* ------------------------------------------------------------------------ */

static void fft_rec(cplx *x, long n, long tw_step, const cplx *tw, long ntw)
{
    if (n == 1) return;
    long p = 2;
    while (n % p) p++;
    long m = n / p;
    cplx *sub = malloc(sizeof(cplx) * n);
    for (long r = 0; r < p; r++)
        for (long j = 0; j < m; j++) sub[r * m + j] = x[j * p + r];
    for (long r = 0; r < p; r++) fft_rec(sub + r * m, m, tw_step * p, tw, ntw);
    /* X[k + q m] = sum_r exp(sign 2 pi i r (k + q m) / n) Y_r[k] */
    for (long k = 0; k < m; k++)
        for (long q = 0; q < p; q++) {
            cplx acc = 0.0;
            for (long r = 0; r < p; r++) {
                long e = (r * (k + q * m)) % n;
                acc += tw[(e * tw_step) % ntw] * sub[r * m + k];
            }
            x[k + q * m] = acc;
        }
    free(sub);
}

/* In-place 1D DFT of n points spaced `stride` apart. */
void or_fft1d(cplx *data, long n, long stride, int sign)
{
    cplx *tw = calloc((size_t)n, sizeof(cplx));
    cplx *buf = calloc((size_t)n, sizeof(cplx));
    for (long k = 0; k < n; k++) tw[k] = cexp(sign * 2.0 * PI * I * (double)k / (double)n);
    for (long j = 0; j < n; j++) buf[j] = data[j * stride];
    fft_rec(buf, n, 1, tw, n);
    for (long j = 0; j < n; j++) data[j * stride] = buf[j];
    free(buf);
    free(tw);
}

/* In-place 3D DFT of an N^3 complex array ([z][y][x]). */
void or_fft3d(cplx *data, int n, int sign)
{
    long N = n;
#pragma omp parallel for schedule(static) if (N >= 32)
    for (long z = 0; z < N; z++)
        for (long y = 0; y < N; y++) or_fft1d(data + (z * N + y) * N, N, 1, sign);
#pragma omp parallel for schedule(static) if (N >= 32)
    for (long z = 0; z < N; z++)
        for (long x = 0; x < N; x++) or_fft1d(data + z * N * N + x, N, N, sign);
#pragma omp parallel for schedule(static) if (N >= 32)
    for (long y = 0; y < N; y++)
        for (long x = 0; x < N; x++) or_fft1d(data + y * N + x, N, N * N, sign);
}

/* Threads of the OpenMP loops (n <= 0: all cores); returns the count in use, 1 without OpenMP. */
int or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    else omp_set_num_threads(omp_get_num_procs());
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Python-friendly wrapper: interleaved (re, im) doubles. */
void or_fft3d_interleaved(double *data, int n, int sign)
{
    or_fft3d((cplx *)data, n, sign);
}

/* ------------------------------------------------------------------------ */
/* Mesh helpers                                                              */
/* ------------------------------------------------------------------------ */

static inline long wrap(long i, long n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

static inline long idx3(long x, long y, long z, long n)
{
    return (wrap(z, n) * n + wrap(y, n)) * n + wrap(x, n);
}

/* signed mode number of DFT index i */
static inline long mode_of(long i, long n) { return i <= n / 2 ? i : i - n; }

/* CIC cell and offset of one coordinate (vertex-centred mesh) */
static inline void cic_axis(double x, int n, long *i, double *f)
{
    double s = x * n;
    double fl = floor(s);
    *f = s - fl;
    *i = wrap((long)fl, n);
}

/* Value of a vertex field at position p by trilinear (CIC) interpolation. */
double or_cic_value(const double *field, int n, const double *p)
{
    long i[3];
    double f[3];
    for (int d = 0; d < 3; d++) cic_axis(p[d], n, &i[d], &f[d]);
    double v = 0.0;
    for (int dz = 0; dz < 2; dz++)
        for (int dy = 0; dy < 2; dy++)
            for (int dx = 0; dx < 2; dx++) {
                double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
                v += w * field[idx3(i[0] + dx, i[1] + dy, i[2] + dz, n)];
            }
    return v;
}

void or_cic_interp(const double *field, int n, const double *pos, long np, double *out)
{
    for (long p = 0; p < np; p++) out[p] = or_cic_value(field, n, pos + 3 * p);
}

/* Add q * dx^-3 * W(vertex - x_p) to the vertex field (CIC assignment). */
static void cic_add(double *field, int n, const double *p, double q)
{
    long i[3];
    double f[3];
    for (int d = 0; d < 3; d++) cic_axis(p[d], n, &i[d], &f[d]);
    double vol = (double)n * n * n;
    for (int dz = 0; dz < 2; dz++)
        for (int dy = 0; dy < 2; dy++)
            for (int dx = 0; dx < 2; dx++) {
                double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
                field[idx3(i[0] + dx, i[1] + dy, i[2] + dz, n)] += q * w * vol;
            }
}

/* Plain CIC mass density rho(x) = dx^-3 sum_p m W (for P(k) and mass checks). */
void or_deposit_mass(int n, const double *pos, long np, double mass, double *rho)
{
    memset(rho, 0, sizeof(double) * (size_t)n * n * n);
    for (long p = 0; p < np; p++) cic_add(rho, n, pos + 3 * p, mass);
}

/* Centred-difference gradient (f(x+e_d) - f(x-e_d)) / (2 dx) along axis d. */
void or_gradient(const double *f, int n, int d, double *g)
{
    long N = n;
#pragma omp parallel for schedule(static) if (N >= 32)
    for (long z = 0; z < N; z++)
        for (long y = 0; y < N; y++)
            for (long x = 0; x < N; x++) {
                long xp = x + (d == 0), yp = y + (d == 1), zp = z + (d == 2);
                long xm = x - (d == 0), ym = y - (d == 1), zm = z - (d == 2);
                g[(z * N + y) * N + x] = (f[idx3(xp, yp, zp, N)] - f[idx3(xm, ym, zm, N)]) * 0.5 * N;
            }
}

/* ------------------------------------------------------------------------ */
/* Stress-energy projection, Eqs. (matterstress), expanded to first order in */
/* phi and psi = phi - chi with the momentum kept exact (Sec. 3.1):           */
/*   4piG a^4 e^{2psi} T^00 = 4piG a^-2 S00,  S00 = sum W m E (1 + 3phi + phi u^2/E^2) */
/*   4piG a^2 e^{2psi} T^0_i = 4piG a^-2 S0i, S0i = sum W m u_i (1 + 4phi - chi)       */
/*   T_ij = a^-2 Sij,                          Sij = sum W m u_i u_j (1 + 3phi - phi u^2/E^2) / E */
/* phi and chi at the particle come from the previous solve.  With           */
/* newtonian != 0 only the mass density is projected (Sec. 3.2).             */
/* sij order: xx, xy, xz, yy, yz, zz.                                        */
/* ------------------------------------------------------------------------ */
void or_project(int n, const double *pos, const double *mom, long np, double mass, double a,
                const double *phi_prev, const double *chi_prev, int newtonian,
                double *s00, double *s0i /* 3 N^3 */, double *sij /* 6 N^3 */)
{
    size_t nc = (size_t)n * n * n;
    memset(s00, 0, sizeof(double) * nc);
    if (!newtonian) {
        memset(s0i, 0, sizeof(double) * 3 * nc);
        memset(sij, 0, sizeof(double) * 6 * nc);
    }
    for (long p = 0; p < np; p++) {
        const double *x = pos + 3 * p, *u = mom + 3 * p;
        if (newtonian) {
            cic_add(s00, n, x, mass);
            continue;
        }
        double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        double E = sqrt(a * a + u2);
        double phi_p = or_cic_value(phi_prev, n, x);
        double chi_p = or_cic_value(chi_prev, n, x);
        cic_add(s00, n, x, mass * E * (1.0 + 3.0 * phi_p + phi_p * u2 / (E * E)));
        for (int i = 0; i < 3; i++)
            cic_add(s0i + i * nc, n, x, mass * u[i] * (1.0 + 4.0 * phi_p - chi_p));
        const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
        for (int c = 0; c < 6; c++)
            cic_add(sij + c * nc, n, x,
                    mass * u[ii[c]] * u[jj[c]] * (1.0 + 3.0 * phi_p - phi_p * u2 / (E * E)) / E);
    }
}

/* The same projection evaluated at one vertex v from a list of particles
 * (those whose cells touch v), with phi_p, chi_p given per particle:
 * out = [S00, S0x, S0y, S0z, Sxx, Sxy, Sxz, Syy, Syz, Szz] at v. */
void or_project_vertex(int n, const long v[3], const double *pos, const double *mom, long np, double mass, double a,
                       const double *phi_p, const double *chi_p, double *out)
{
    for (int c = 0; c < 10; c++) out[c] = 0.0;
    double vol = (double)n * n * n;
    for (long p = 0; p < np; p++) {
        const double *x = pos + 3 * p, *u = mom + 3 * p;
        long i[3];
        double f[3], w = 1.0;
        for (int d = 0; d < 3; d++) {
            cic_axis(x[d], n, &i[d], &f[d]);
            long off = wrap(v[d] - i[d], n);
            if (off == 0) w *= 1.0 - f[d];
            else if (off == 1) w *= f[d];
            else w = 0.0;
        }
        if (w == 0.0) continue;
        double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        double E = sqrt(a * a + u2);
        double ph = phi_p[p], ch = chi_p[p];
        out[0] += vol * w * mass * E * (1.0 + 3.0 * ph + ph * u2 / (E * E));
        for (int d = 0; d < 3; d++) out[1 + d] += vol * w * mass * u[d] * (1.0 + 4.0 * ph - ch);
        const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
        for (int c = 0; c < 6; c++)
            out[4 + c] += vol * w * mass * u[ii[c]] * u[jj[c]] * (1.0 + 3.0 * ph - ph * u2 / (E * E)) / E;
    }
}

/* ------------------------------------------------------------------------ */
/* Field equations.                                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    double a, hc;          /* a_n and Hc(a_n) */
    double dtau_prev;      /* tau_n - tau_{n-1}: backward difference of phi */
    double dtau_prev2;     /* tau_{n-1} - tau_{n-2}: phi' in the vector source */
    double dtau;           /* tau_{n+1} - tau_n: tensor integration step */
    double hc_half;        /* Hc(a_{n+1/2}) for the tensor equation */
    double four_pi_g;
    double omega_m;
    int newtonian;
    int bootstrap;         /* quasi-static phi only (first solve) */
    int full_hc;           /* nonlinear remainder of Eq. fullHc in the phi source */
    int b_space;           /* B_i from Eq. spacespace (integrated) instead of the momentum constraint */
    int b_seed;            /* with b_space: take this step's B from the momentum constraint */
    double b_decay;        /* with b_space: (a_{n-1} / a_n)^2 */
} or_solve_params;

/* 7-point Laplacian (sum of the six neighbours - 6 f) / dx^2. */
void or_laplacian7(const double *f, int n, double *out)
{
    long N = n;
#pragma omp parallel for schedule(static) if (N >= 32)
    for (long z = 0; z < N; z++)
        for (long y = 0; y < N; y++)
            for (long x = 0; x < N; x++) {
                double s = f[idx3(x + 1, y, z, N)] + f[idx3(x - 1, y, z, N)] + f[idx3(x, y + 1, z, N)] +
                           f[idx3(x, y - 1, z, N)] + f[idx3(x, y, z + 1, N)] + f[idx3(x, y, z - 1, N)];
                out[(z * N + y) * N + x] = (s - 6.0 * f[(z * N + y) * N + x]) * (double)N * (double)N;
            }
}

/*
 * Nonlinear remainder of the Hamiltonian constraint, Eq. fullHc.  With the
 * background (3/2) Hc^2 = 4piG a^2 rho_bar removed, Eq. fullHc reads
 *   lin + Nl = 4piG a^-2 (S00 - a Omega_m),  lin = Lap phi - 3 Hc phi' - 3 Hc^2 psi,
 *   Nl = (e^{2phi} - 1) Lap phi - 1/2 e^{2phi} |grad phi|^2
 *        + 3/2 [(Hc - phi')^2 e^{-2psi} - Hc^2 + 2 Hc phi' + 2 Hc^2 psi].
 * The bracket is regrouped exactly as Hc^2 (e^x - 1 - x) - 2 Hc phi' (e^x - 1)
 * + phi'^2 e^x with x = -2 psi, so that nothing of size Hc^2 cancels.
 * Evaluated on phi = phi_{n-1}, psi = phi_{n-1} - chi_{n-1} and
 * phi' = (phi_{n-1} - phi_{n-2}) / dtau_prev2; Lap is the 7-point Laplacian
 * and grad the centred difference.
 */
void or_hc_remainder(int n, double hc, double dtau_prev2, const double *phi, const double *chi,
                     const double *phi_prev2, double *out)
{
    size_t nc = (size_t)n * n * n;
    double *lap = malloc(sizeof(double) * nc), *g = malloc(sizeof(double) * 3 * nc);
    or_laplacian7(phi, n, lap);
    for (int d = 0; d < 3; d++) or_gradient(phi, n, d, g + d * nc);
    for (size_t c = 0; c < nc; c++) {
        double psi = phi[c] - chi[c];
        double dphi = (phi[c] - phi_prev2[c]) / dtau_prev2;
        double g2 = g[c] * g[c] + g[nc + c] * g[nc + c] + g[2 * nc + c] * g[2 * nc + c];
        double x = -2.0 * psi;
        out[c] = expm1(2.0 * phi[c]) * lap[c] - 0.5 * exp(2.0 * phi[c]) * g2 +
                 1.5 * (hc * hc * (expm1(x) - x) - 2.0 * hc * dphi * expm1(x) + dphi * dphi * exp(x));
    }
    free(lap);
    free(g);
}

/* ktilde_i = 2N sin(pi n_i / N): with it sum_i ktilde_i^2 is the eigenvalue of
 * minus the 7-point Laplacian. */
static inline double ktilde(long nmode, int n) { return 2.0 * n * sin(PI * (double)nmode / n); }

/* Polarisation tensors e+ and ex for the mode (nx, ny, nz): e1 is the unit
 * vector perpendicular to khat obtained from the axis with the smallest
 * |n_i| (ties to the lowest axis), e2 = khat x e1,
 * e+ = (e1 e1 - e2 e2)/sqrt2, ex = (e1 e2 + e2 e1)/sqrt2. */
void or_polarisations(const long nv[3], const double kt[3], double ep[3][3], double ex[3][3])
{
    double kn = sqrt(kt[0] * kt[0] + kt[1] * kt[1] + kt[2] * kt[2]);
    double kh[3] = {kt[0] / kn, kt[1] / kn, kt[2] / kn};
    int m = 0;
    for (int d = 1; d < 3; d++)
        if (labs(nv[d]) < labs(nv[m])) m = d;
    double e1[3] = {0, 0, 0};
    e1[m] = 1.0;
    for (int d = 0; d < 3; d++) e1[d] -= kh[m] * kh[d];
    double l = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int d = 0; d < 3; d++) e1[d] /= l;
    double e2[3] = {kh[1] * e1[2] - kh[2] * e1[1], kh[2] * e1[0] - kh[0] * e1[2], kh[0] * e1[1] - kh[1] * e1[0]};
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            ep[i][j] = (e1[i] * e1[j] - e2[i] * e2[j]) / sqrt(2.0);
            ex[i][j] = (e1[i] * e2[j] + e2[i] * e1[j]) / sqrt(2.0);
        }
}

/* One implicit-midpoint (Crank-Nicolson) step of h'' + 2 Hc h' + k^2 h = s:
 * (I - dt/2 A) y' = (I + dt/2 A) y + dt (0, s),  A = [[0, 1], [-k^2, -2 Hc]]. */
void or_tensor_step(double complex *h, double complex *v, double k2, double hc, double dt, double complex s)
{
    double m11 = 1.0, m12 = -0.5 * dt, m21 = 0.5 * dt * k2, m22 = 1.0 + dt * hc;
    double p11 = 1.0, p12 = 0.5 * dt, p21 = -0.5 * dt * k2, p22 = 1.0 - dt * hc;
    double complex r1 = p11 * (*h) + p12 * (*v);
    double complex r2 = p21 * (*h) + p22 * (*v) + dt * s;
    double det = m11 * m22 - m12 * m21;
    *h = (m22 * r1 - m12 * r2) / det;
    *v = (-m21 * r1 + m11 * r2) / det;
}

void or_tensor_step_ri(double *h, double *v, double k2, double hc, double dt, double s_re, double s_im)
{
    or_tensor_step((double complex *)h, (double complex *)v, k2, hc, dt, s_re + I * s_im);
}

/*
 * Configuration-space sources of the field equations.
 *  R     = 4piG a^-2 (S00 - a Omega_m) - (3 Hc / dtau_prev) phi_{n-1} - 3 Hc^2 chi_{n-1}
 *          (Eq. NewtonHc with the backward difference of phi and psi = phi - chi;
 *           Newtonian mode: R = 4piG a^-1 (rho - Omega_m)),
 *  F_i   = 4piG a^-2 S0i - phi' d_i psi   (Eq. momentumcontraint, non-gradient part),
 *  Sig_ij = 16piG a^-2 (Sij - delta_ij S_kk/3) - 2 TF[2 d_i phi d_j phi
 *          - (d_i phi + d_i psi)(d_j phi + d_j psi)]   (Eq. spacespace),
 * with phi, psi, phi' from the previous step(s).  Bootstrap: R only, with
 * the (3 Hc/dtau) term dropped.  full_hc: R -= Nl (or_hc_remainder).
 */
void or_sources(int n, const or_solve_params *sp, const double *s00, const double *s0i, const double *sij,
                const double *phi_prev, const double *chi_prev, const double *phi_prev2,
                double *R, double *F /* 3 N^3 */, double *Sig /* 6 N^3 */)
{
    size_t nc = (size_t)n * n * n;
    double a = sp->a, hc = sp->hc, g4 = sp->four_pi_g;
    for (size_t c = 0; c < nc; c++) {
        if (sp->newtonian)
            R[c] = g4 / a * (s00[c] - sp->omega_m);
        else if (sp->bootstrap)
            R[c] = g4 / (a * a) * (s00[c] - a * sp->omega_m) - 3.0 * hc * hc * chi_prev[c];
        else
            R[c] = g4 / (a * a) * (s00[c] - a * sp->omega_m) - 3.0 * hc / sp->dtau_prev * phi_prev[c]
                   - 3.0 * hc * hc * chi_prev[c];
    }
    if (sp->newtonian || sp->bootstrap) return;
    if (sp->full_hc) {
        double *nl = malloc(sizeof(double) * nc);
        or_hc_remainder(n, hc, sp->dtau_prev2, phi_prev, chi_prev, phi_prev2, nl);
        for (size_t c = 0; c < nc; c++) R[c] -= nl[c];
        free(nl);
    }
    double *psi = malloc(sizeof(double) * nc);
    double *gphi = malloc(sizeof(double) * 3 * nc), *gpsi = malloc(sizeof(double) * 3 * nc);
    for (size_t c = 0; c < nc; c++) psi[c] = phi_prev[c] - chi_prev[c];
    for (int d = 0; d < 3; d++) {
        or_gradient(phi_prev, n, d, gphi + d * nc);
        or_gradient(psi, n, d, gpsi + d * nc);
    }
    const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
#pragma omp parallel for schedule(static) if (n >= 32)
    for (size_t c = 0; c < nc; c++) {
        double dphi_dtau = (phi_prev[c] - phi_prev2[c]) / sp->dtau_prev2;
        for (int i = 0; i < 3; i++) F[i * nc + c] = g4 / (a * a) * s0i[i * nc + c] - dphi_dtau * gpsi[i * nc + c];
        double Q[3][3], S[3][3];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double gi = gphi[i * nc + c], gj = gphi[j * nc + c];
                Q[i][j] = 2.0 * gi * gj - (gi + gpsi[i * nc + c]) * (gj + gpsi[j * nc + c]);
            }
        for (int k = 0; k < 6; k++) {
            S[ii[k]][jj[k]] = sij[k * nc + c];
            S[jj[k]][ii[k]] = sij[k * nc + c];
        }
        double trS = S[0][0] + S[1][1] + S[2][2], trQ = Q[0][0] + Q[1][1] + Q[2][2];
        for (int k = 0; k < 6; k++) {
            int i = ii[k], j = jj[k];
            double d = (i == j) ? 1.0 : 0.0;
            Sig[k * nc + c] = 4.0 * g4 / (a * a) * (S[i][j] - d * trS / 3.0) - 2.0 * (Q[i][j] - d * trQ / 3.0);
        }
    }
    free(psi);
    free(gphi);
    free(gpsi);
}

/*
 * Fourier-space solutions, on full complex DFT arrays:
 *  phi_k = -R_k / (kt^2 + 3 Hc/dtau_prev + 3 Hc^2)          (k = 0 included)
 *  chi_k = -3/(4 kt^4) kt_i kt_j Sig_ij,k                   (scalar part of Eq. spacespace)
 *  B_i,k = 4 (delta_ij - kt_i kt_j / kt^2) F_j,k / kt^2     (spin-1 part of Eq. momentumcontraint)
 *  h_A:   s_A = e^A_ij Sig_ij,k, one Crank-Nicolson step    (spin-2 part of Eq. spacespace)
 * chi_0 = B_0 = h_0 = 0, and chi, B, h vanish on Nyquist modes.
 * b_space (B from Eq. spacespace): with d_i -> i kt_i, the vector part of
 * Sig is i (kt_i V_j + kt_j V_i) with kt.V = 0 and V = (d_tau + 2 Hc) B, so
 * kt_i Sig_ij has the transverse part i kt^2 V_j; hence
 *  W_j = -i (delta_jl - kt_j kt_l / kt^2) kt_i Sig_il,k / kt^2,
 *  B_j,k = b_decay B_j,k(previous) + dtau_prev W_j      (bs holds B_k between steps).
 * Newtonian mode: phi_k = -R_k / kt^2, phi_0 = 0, chi = B = 0.
 */
void or_fourier_solve(int n, const or_solve_params *sp, cplx *Rk /* in: R, out: phi */,
                      cplx *Fk /* 3 N^3: in F, out B */, cplx *Sk /* 6 N^3: in Sig; [0] out chi */,
                      cplx *hp, cplx *hx, cplx *vp, cplx *vx, cplx *bs /* 3 N^3 B_k state, b_space only */)
{
    long N = n;
    size_t nc = (size_t)n * n * n;
    double cphi;
    if (sp->newtonian)
        cphi = 0.0;
    else if (sp->bootstrap)
        cphi = 3.0 * sp->hc * sp->hc;
    else
        cphi = 3.0 * sp->hc / sp->dtau_prev + 3.0 * sp->hc * sp->hc;
    const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
#pragma omp parallel for schedule(static) if (N >= 32)
    for (long z = 0; z < N; z++)
        for (long y = 0; y < N; y++)
            for (long x = 0; x < N; x++) {
                size_t c = (size_t)((z * N + y) * N + x);
                long nv[3] = {mode_of(x, N), mode_of(y, N), mode_of(z, N)};
                double kt[3] = {ktilde(nv[0], n), ktilde(nv[1], n), ktilde(nv[2], n)};
                double k2 = kt[0] * kt[0] + kt[1] * kt[1] + kt[2] * kt[2];
                int zero = (nv[0] == 0 && nv[1] == 0 && nv[2] == 0);
                int nyq = (labs(nv[0]) * 2 == N) || (labs(nv[1]) * 2 == N) || (labs(nv[2]) * 2 == N);
                /* scalar potential phi */
                if (sp->newtonian && zero)
                    Rk[c] = 0.0;
                else
                    Rk[c] = -Rk[c] / (k2 + cphi);
                if (sp->newtonian || sp->bootstrap) continue;
                if (zero || nyq) {
                    Sk[c] = 0.0;
                    for (int i = 0; i < 3; i++) Fk[i * nc + c] = 0.0;
                    if (sp->b_space)
                        for (int i = 0; i < 3; i++) bs[i * nc + c] = 0.0;
                    hp[c] = hx[c] = vp[c] = vx[c] = 0.0;
                    continue;
                }
                /* Sig as a full symmetric matrix */
                cplx S[3][3];
                for (int k = 0; k < 6; k++) {
                    S[ii[k]][jj[k]] = Sk[k * nc + c];
                    S[jj[k]][ii[k]] = Sk[k * nc + c];
                }
                /* tensor sector first (needs Sig before chi overwrites Sk[0]) */
                double ep[3][3], ex[3][3];
                or_polarisations(nv, kt, ep, ex);
                cplx sp_ = 0.0, sx_ = 0.0;
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) {
                        sp_ += ep[i][j] * S[i][j];
                        sx_ += ex[i][j] * S[i][j];
                    }
                or_tensor_step(&hp[c], &vp[c], k2, sp->hc_half, sp->dtau, sp_);
                or_tensor_step(&hx[c], &vx[c], k2, sp->hc_half, sp->dtau, sx_);
                /* scalar slip chi */
                cplx kks = 0.0;
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) kks += kt[i] * kt[j] * S[i][j];
                Sk[c] = -3.0 / (4.0 * k2 * k2) * kks;
                /* frame dragging B */
                if (sp->b_space && !sp->b_seed) {
                    cplx v[3];
                    for (int l = 0; l < 3; l++) v[l] = kt[0] * S[0][l] + kt[1] * S[1][l] + kt[2] * S[2][l];
                    cplx kv = kt[0] * v[0] + kt[1] * v[1] + kt[2] * v[2];
                    for (int j = 0; j < 3; j++) {
                        cplx W = -I * (v[j] - kt[j] * kv / k2) / k2;
                        Fk[j * nc + c] = sp->b_decay * bs[j * nc + c] + sp->dtau_prev * W;
                    }
                } else {
                    cplx F[3] = {Fk[c], Fk[nc + c], Fk[2 * nc + c]};
                    cplx kF = kt[0] * F[0] + kt[1] * F[1] + kt[2] * F[2];
                    for (int i = 0; i < 3; i++) Fk[i * nc + c] = 4.0 * (F[i] - kt[i] * kF / k2) / k2;
                }
                if (sp->b_space)
                    for (int i = 0; i < 3; i++) bs[i * nc + c] = Fk[i * nc + c];
            }
}

/* Real field -> complex DFT and back. */
static cplx *to_spectrum(const double *f, int n)
{
    size_t nc = (size_t)n * n * n;
    cplx *c = malloc(sizeof(cplx) * nc);
    for (size_t i = 0; i < nc; i++) c[i] = f[i];
    or_fft3d(c, n, -1);
    return c;
}

static void to_real(cplx *c, int n, double *f)
{
    size_t nc = (size_t)n * n * n;
    or_fft3d(c, n, +1);
    for (size_t i = 0; i < nc; i++) f[i] = creal(c[i]) / (double)nc;
}

/* ------------------------------------------------------------------------ */
/* Particle update: Eqs. (drift) and (kick) of the Hamiltonian (1pclH) with   */
/* alpha = a e^psi, gamma_ij = a^2 e^{-2phi} delta_ij, beta^i = -B_i, to first */
/* order in phi, psi, B (h neglected, Sec. 3.1):                             */
/*   du_i/dtau = -E d_i psi - (u^2/E) d_i phi - u_j d_i B_j      (E at a_n)  */
/*   dx^i/dtau = (u_i/E)(1 + 3phi - chi - phi u^2/E^2) + B_i     (E at a_n+1/2) */
/* Newtonian mode (Sec. 3.2): du/dtau = -a d psi, dx/dtau = u/a.             */
/* Kick with dtau_kick = (dtau_{n-1} + dtau_n)/2, then drift with dtau_n.    */
/* ------------------------------------------------------------------------ */
void or_kick_drift(int n, double *pos, double *mom, long np, double a_kick, double a_drift,
                   double dtau_kick, double dtau_drift, int newtonian,
                   const double *phi, const double *chi, const double *B /* 3 N^3 or NULL */)
{
    size_t nc = (size_t)n * n * n;
    double *psi = malloc(sizeof(double) * nc);
    for (size_t c = 0; c < nc; c++) psi[c] = phi[c] - (newtonian ? 0.0 : chi[c]);
    double *gphi = malloc(sizeof(double) * 3 * nc), *gpsi = malloc(sizeof(double) * 3 * nc);
    double *gB = newtonian ? NULL : malloc(sizeof(double) * 9 * nc);
    for (int d = 0; d < 3; d++) {
        or_gradient(phi, n, d, gphi + d * nc);
        or_gradient(psi, n, d, gpsi + d * nc);
        if (!newtonian)
            for (int j = 0; j < 3; j++) or_gradient(B + j * nc, n, d, gB + (d * 3 + j) * nc); /* d_d B_j */
    }
#pragma omp parallel for schedule(static) if (np >= 4096)
    for (long p = 0; p < np; p++) {
        double *x = pos + 3 * p, *u = mom + 3 * p;
        double K[3];
        if (newtonian) {
            for (int i = 0; i < 3; i++) K[i] = -a_kick * or_cic_value(gpsi + i * nc, n, x);
            for (int i = 0; i < 3; i++) u[i] += dtau_kick * K[i];
            for (int i = 0; i < 3; i++) x[i] += dtau_drift * u[i] / a_drift;
        } else {
            double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            double E = sqrt(a_kick * a_kick + u2);
            for (int i = 0; i < 3; i++) {
                double dB = 0.0;
                for (int j = 0; j < 3; j++) dB += u[j] * or_cic_value(gB + (i * 3 + j) * nc, n, x);
                K[i] = -E * or_cic_value(gpsi + i * nc, n, x) - u2 / E * or_cic_value(gphi + i * nc, n, x) - dB;
            }
            for (int i = 0; i < 3; i++) u[i] += dtau_kick * K[i];
            double phi_p = or_cic_value(phi, n, x), chi_p = or_cic_value(chi, n, x);
            double Bp[3];
            for (int i = 0; i < 3; i++) Bp[i] = or_cic_value(B + i * nc, n, x);
            double v2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            double Ed = sqrt(a_drift * a_drift + v2);
            for (int i = 0; i < 3; i++)
                x[i] += dtau_drift * ((u[i] / Ed) * (1.0 + 3.0 * phi_p - chi_p - phi_p * v2 / (Ed * Ed)) + Bp[i]);
        }
        for (int i = 0; i < 3; i++) {
            x[i] -= floor(x[i]);
            if (x[i] >= 1.0) x[i] = 0.0;
        }
    }
    free(psi);
    free(gphi);
    free(gpsi);
    free(gB);
}

/* ------------------------------------------------------------------------ */
/* Power spectrum of the CIC mass density contrast delta = rho/Omega_m - 1:  */
/* P(k_b) = < |delta_k|^2 > / N^6 over modes with round(|n|) = b, b >= 1.    */
/* ------------------------------------------------------------------------ */
void or_power_spectrum(int n, const double *rho, double omega_m, int nbins,
                       double *kmean, double *pk, int64_t *nmodes)
{
    long N = n;
    size_t nc = (size_t)n * n * n;
    cplx *d = malloc(sizeof(cplx) * nc);
    for (size_t c = 0; c < nc; c++) d[c] = rho[c] / omega_m - 1.0;
    or_fft3d(d, n, -1);
    for (int b = 0; b < nbins; b++) kmean[b] = pk[b] = 0.0, nmodes[b] = 0;
    for (long z = 0; z < N; z++)
        for (long y = 0; y < N; y++)
            for (long x = 0; x < N; x++) {
                double kn = sqrt((double)(mode_of(x, N) * mode_of(x, N) + mode_of(y, N) * mode_of(y, N) +
                                          mode_of(z, N) * mode_of(z, N)));
                long b = lround(kn);
                if (b < 1 || b >= nbins) continue;
                cplx v = d[(z * N + y) * N + x];
                pk[b] += creal(v * conj(v)) / ((double)nc * (double)nc);
                kmean[b] += 2.0 * PI * kn;
                nmodes[b] += 1;
            }
    for (int b = 0; b < nbins; b++)
        if (nmodes[b]) pk[b] /= nmodes[b], kmean[b] /= nmodes[b];
    free(d);
}

/* ------------------------------------------------------------------------ */
/* Simulation driver: one full PM step = project -> solve -> kick/drift.     */
/* ------------------------------------------------------------------------ */
/* flags: 1 Newtonian limit, 2 full Hamiltonian constraint, 4 B from Eq. spacespace */
typedef struct {
    int n, nsteps, newtonian, full_hc, b_space, step;
    long np;
    double omega_m, h0, four_pi_g, mass;
    double *a_n, *dtau, *a_half;
    double *pos, *mom;
    double *phi_prev, *chi_prev, *phi_prev2; /* phi_{n-1}, chi_{n-1}, phi_{n-2} */
    double *phi, *chi, *B;                   /* latest solution: phi_n, chi_n, B_n (3 N^3) */
    double *src;                             /* last sources: R, F(3), Sig(6) */
    cplx *hp, *hx, *vp, *vx;                 /* tensor state (full DFT arrays) */
    cplx *bs;                                /* B_k between steps (b_space) */
} or_sim;

or_sim *or_sim_create(int n, long np, double omega_m, double box_mpch, double z_init, double z_final,
                      int nsteps, int flags)
{
    or_sim *s = calloc(1, sizeof(or_sim));
    size_t nc = (size_t)n * n * n;
    s->n = n;
    s->np = np;
    s->nsteps = nsteps;
    s->newtonian = flags & 1;
    s->full_hc = !s->newtonian && (flags & 2);
    s->b_space = !s->newtonian && (flags & 4);
    s->omega_m = omega_m;
    s->h0 = box_mpch / 2997.92458;
    s->four_pi_g = 1.5 * s->h0 * s->h0;
    s->mass = omega_m / (double)np;
    s->a_n = malloc(sizeof(double) * (nsteps + 1));
    s->dtau = malloc(sizeof(double) * nsteps);
    s->a_half = malloc(sizeof(double) * nsteps);
    or_schedule(nsteps, 1.0 / (1.0 + z_init), 1.0 / (1.0 + z_final), omega_m, s->h0, s->a_n, s->dtau, s->a_half);
    s->pos = malloc(sizeof(double) * 3 * np);
    s->mom = malloc(sizeof(double) * 3 * np);
    s->phi_prev = calloc(nc, sizeof(double));
    s->chi_prev = calloc(nc, sizeof(double));
    s->phi_prev2 = calloc(nc, sizeof(double));
    s->phi = calloc(nc, sizeof(double));
    s->chi = calloc(nc, sizeof(double));
    s->B = calloc(3 * nc, sizeof(double));
    s->src = calloc(10 * nc, sizeof(double));
    s->hp = calloc(nc, sizeof(cplx));
    s->hx = calloc(nc, sizeof(cplx));
    s->vp = calloc(nc, sizeof(cplx));
    s->vx = calloc(nc, sizeof(cplx));
    s->bs = calloc(3 * nc, sizeof(cplx));
    return s;
}

void or_sim_destroy(or_sim *s)
{
    if (!s) return;
    free(s->a_n); free(s->dtau); free(s->a_half); free(s->pos); free(s->mom);
    free(s->phi_prev); free(s->chi_prev); free(s->phi_prev2); free(s->phi); free(s->chi); free(s->B);
    free(s->src); free(s->hp); free(s->hx); free(s->vp); free(s->vx); free(s->bs);
    free(s);
}

void or_sim_schedule(const or_sim *s, double *a_n, double *dtau, double *a_half)
{
    memcpy(a_n, s->a_n, sizeof(double) * (s->nsteps + 1));
    memcpy(dtau, s->dtau, sizeof(double) * s->nsteps);
    memcpy(a_half, s->a_half, sizeof(double) * s->nsteps);
}

/* Solve the field equations for given configuration-space sources R, F (3),
 * Sig (6): forward DFTs, Fourier solve, inverse DFTs.  Outputs phi, chi,
 * B (3 N^3); the tensor state (4 interleaved complex N^3 arrays: h+, hx,
 * h+', hx') is advanced in place. */
void or_solve_sources(int n, const or_solve_params *sp, const double *R, const double *F, const double *Sig,
                      double *phi, double *chi, double *B, double *tensor, double *bstate)
{
    size_t nc = (size_t)n * n * n;
    cplx *Rk = to_spectrum(R, n);
    cplx *Fk = calloc(3 * nc, sizeof(cplx)), *Sk = calloc(6 * nc, sizeof(cplx));
    int full = !(sp->newtonian || sp->bootstrap);
    if (full) {
        for (int i = 0; i < 3; i++) {
            cplx *t = to_spectrum(F + i * nc, n);
            memcpy(Fk + i * nc, t, sizeof(cplx) * nc);
            free(t);
        }
        for (int i = 0; i < 6; i++) {
            cplx *t = to_spectrum(Sig + i * nc, n);
            memcpy(Sk + i * nc, t, sizeof(cplx) * nc);
            free(t);
        }
    }
    cplx *ts = (cplx *)tensor;
    or_fourier_solve(n, sp, Rk, Fk, Sk, ts, ts + nc, ts + 2 * nc, ts + 3 * nc, (cplx *)bstate);
    to_real(Rk, n, phi);
    if (full) {
        to_real(Sk, n, chi);
        for (int i = 0; i < 3; i++) to_real(Fk + i * nc, n, B + i * nc);
    } else {
        memset(chi, 0, sizeof(double) * nc);
        memset(B, 0, sizeof(double) * 3 * nc);
    }
    free(Rk);
    free(Fk);
    free(Sk);
}

/* Flat-argument form of or_solve_sources for foreign callers. */
void or_solve_sources_flat(int n, double a, double hc, double dtau_prev, double dtau_prev2, double dtau,
                           double hc_half, double four_pi_g, double omega_m, int newtonian, int bootstrap,
                           const double *R, const double *F, const double *Sig, double *phi, double *chi,
                           double *B, double *tensor, int b_space, int b_seed, double b_decay, double *bstate)
{
    or_solve_params sp = {a, hc, dtau_prev, dtau_prev2, dtau, hc_half, four_pi_g, omega_m, newtonian, bootstrap,
                          0, b_space, b_seed, b_decay};
    or_solve_sources(n, &sp, R, F, Sig, phi, chi, B, tensor, bstate);
}

void or_sources_flat(int n, double a, double hc, double dtau_prev, double dtau_prev2, double four_pi_g,
                     double omega_m, int newtonian, int bootstrap, const double *s00, const double *s0i,
                     const double *sij, const double *phi_prev, const double *chi_prev, const double *phi_prev2,
                     double *R, double *F, double *Sig, int full_hc)
{
    or_solve_params sp = {a, hc, dtau_prev, dtau_prev2, 0.0, 0.0, four_pi_g, omega_m, newtonian, bootstrap,
                          full_hc, 0, 0, 1.0};
    or_sources(n, &sp, s00, s0i, sij, phi_prev, chi_prev, phi_prev2, R, F, Sig);
}

/* project + solve at step index `k` (a = a_n[k]); writes phi, chi, B, src. */
static void sim_project_solve(or_sim *s, int k, int bootstrap)
{
    int n = s->n;
    size_t nc = (size_t)n * n * n;
    double *s00 = malloc(sizeof(double) * nc), *s0i = malloc(sizeof(double) * 3 * nc),
           *sij = malloc(sizeof(double) * 6 * nc);
    double a = s->a_n[k];
    int kk = k < s->nsteps ? k : s->nsteps - 1;
    or_solve_params sp;
    sp.a = a;
    sp.hc = or_conformal_hubble(a, s->omega_m, s->h0);
    sp.dtau_prev = (k >= 1) ? s->dtau[k - 1] : s->dtau[0];
    sp.dtau_prev2 = (k >= 2) ? s->dtau[k - 2] : s->dtau[0];
    sp.dtau = s->dtau[kk];
    sp.hc_half = or_conformal_hubble(s->a_half[kk], s->omega_m, s->h0);
    sp.four_pi_g = s->four_pi_g;
    sp.omega_m = s->omega_m;
    sp.newtonian = s->newtonian;
    sp.bootstrap = bootstrap;
    sp.full_hc = s->full_hc;
    sp.b_space = s->b_space;
    sp.b_seed = (k == 0);
    sp.b_decay = (k >= 1) ? (s->a_n[k - 1] / a) * (s->a_n[k - 1] / a) : 1.0;
    /* at the bootstrap phi_prev = chi_prev = 0, so the weights carry no potential */
    or_project(n, s->pos, s->mom, s->np, s->mass, a, s->phi_prev, s->chi_prev, s->newtonian, s00, s0i, sij);
    double *R = s->src, *F = s->src + nc, *Sig = s->src + 4 * nc;
    or_sources(n, &sp, s00, s0i, sij, s->phi_prev, s->chi_prev, s->phi_prev2, R, F, Sig);
    double *tensor = malloc(sizeof(cplx) * 4 * nc);
    memcpy(tensor, s->hp, sizeof(cplx) * nc);
    memcpy(tensor + 2 * nc, s->hx, sizeof(cplx) * nc);
    memcpy(tensor + 4 * nc, s->vp, sizeof(cplx) * nc);
    memcpy(tensor + 6 * nc, s->vx, sizeof(cplx) * nc);
    or_solve_sources(n, &sp, R, F, Sig, s->phi, s->chi, s->B, tensor, (double *)s->bs);
    memcpy(s->hp, tensor, sizeof(cplx) * nc);
    memcpy(s->hx, tensor + 2 * nc, sizeof(cplx) * nc);
    memcpy(s->vp, tensor + 4 * nc, sizeof(cplx) * nc);
    memcpy(s->vx, tensor + 6 * nc, sizeof(cplx) * nc);
    free(tensor);
    free(s00); free(s0i); free(sij);
}

/* Load particles and run the quasi-static bootstrap solve for phi_{-1}
 * (phi_{-1} = chi_{-1} = 0 in the source weights, 3Hc/dtau term dropped). */
void or_sim_set_particles(or_sim *s, const double *pos, const double *mom)
{
    size_t nc = (size_t)s->n * s->n * s->n;
    memcpy(s->pos, pos, sizeof(double) * 3 * s->np);
    memcpy(s->mom, mom, sizeof(double) * 3 * s->np);
    memset(s->phi_prev, 0, sizeof(double) * nc);
    memset(s->chi_prev, 0, sizeof(double) * nc);
    memset(s->hp, 0, sizeof(cplx) * nc); memset(s->hx, 0, sizeof(cplx) * nc);
    memset(s->vp, 0, sizeof(cplx) * nc); memset(s->vx, 0, sizeof(cplx) * nc);
    memset(s->bs, 0, sizeof(cplx) * 3 * nc);
    s->step = 0;
    sim_project_solve(s, 0, 1);
    memcpy(s->phi_prev, s->phi, sizeof(double) * nc);
    memcpy(s->phi_prev2, s->phi, sizeof(double) * nc);
    memset(s->chi_prev, 0, sizeof(double) * nc);
}

/* First half of step n: project at x_n and solve for phi_n, chi_n, B_n, h. */
int or_sim_solve(or_sim *s)
{
    int k = s->step;
    if (k >= s->nsteps) return -1;
    sim_project_solve(s, k, 0);
    return k;
}

/* Second half of step n: kick and drift, then rotate the potentials.  With
 * corr != NULL (3 N^3, components x, y, z of an additive force correction c
 * on the mesh), every particle first receives the extra kick
 *   u += dtau_kick * f * c(x_p)   (CIC value; f = a_n in the Newtonian mode,
 *                                  f = E = sqrt(a_n^2 + u^2) otherwise),
 * i.e. c corrects the force -grad psi of the kick.  Returns the new step index. */
int or_sim_update(or_sim *s, const double *corr)
{
    int k = s->step;
    if (k >= s->nsteps) return -1;
    size_t nc = (size_t)s->n * s->n * s->n;
    double dtau_kick = 0.5 * ((k >= 1 ? s->dtau[k - 1] : s->dtau[0]) + s->dtau[k]);
    if (corr) {
        double a = s->a_n[k];
        for (long p = 0; p < s->np; p++) {
            double *u = s->mom + 3 * p;
            double f = s->newtonian ? a : sqrt(a * a + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            double c[3];
            for (int i = 0; i < 3; i++) c[i] = or_cic_value(corr + i * nc, s->n, s->pos + 3 * p);
            for (int i = 0; i < 3; i++) u[i] += dtau_kick * f * c[i];
        }
    }
    or_kick_drift(s->n, s->pos, s->mom, s->np, s->a_n[k], s->a_half[k], dtau_kick, s->dtau[k], s->newtonian,
                  s->phi, s->chi, s->B);
    memcpy(s->phi_prev2, s->phi_prev, sizeof(double) * nc);
    memcpy(s->phi_prev, s->phi, sizeof(double) * nc);
    memcpy(s->chi_prev, s->chi, sizeof(double) * nc);
    s->step = k + 1;
    return s->step;
}

/* One full step n: or_sim_solve then or_sim_update without correction.
 * Returns the new step index, or -1 past the end of the schedule. */
int or_sim_step(or_sim *s)
{
    if (or_sim_solve(s) < 0) return -1;
    return or_sim_update(s, NULL);
}

/* Field ids: 0 phi, 1 chi, 2..4 B_x..B_z, 5 R, 6..8 F, 9..14 Sig (xx,xy,xz,yy,yz,zz) */
void or_sim_get_field(const or_sim *s, int id, double *out)
{
    size_t nc = (size_t)s->n * s->n * s->n;
    const double *src = NULL;
    if (id == 0) src = s->phi;
    else if (id == 1) src = s->chi;
    else if (id >= 2 && id <= 4) src = s->B + (id - 2) * nc;
    else if (id >= 5 && id <= 14) src = s->src + (id - 5) * nc;
    if (src) memcpy(out, src, sizeof(double) * nc);
}

/* Tensor state 0 h+, 1 hx, 2 h+', 3 hx' as interleaved complex N^3 arrays. */
void or_sim_get_tensor(const or_sim *s, int id, double *out)
{
    size_t nc = (size_t)s->n * s->n * s->n;
    const cplx *src = id == 0 ? s->hp : id == 1 ? s->hx : id == 2 ? s->vp : s->vx;
    memcpy(out, src, sizeof(cplx) * nc);
}

void or_sim_get_particles(const or_sim *s, double *pos, double *mom)
{
    memcpy(pos, s->pos, sizeof(double) * 3 * s->np);
    memcpy(mom, s->mom, sizeof(double) * 3 * s->np);
}

int or_sim_step_index(const or_sim *s) { return s->step; }
