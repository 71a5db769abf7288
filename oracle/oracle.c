/*
 * FP64 CPU oracle for explicit iterative stencil time stepping.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may link,
 * load or call this file: only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header or constant generator
 * with the CUDA path.
 *
 * What it computes, and where that is defined:
 *
 *  - The method of the paper ("Kernel Batching with CUDA Graphs", Sec. III-A,
 *    Listings 1-3 and Fig. 1) groups the per-iteration kernel launches of an
 *    iterative solver into iteration batches and replays them as CUDA graphs.
 *    Batching does not change what is computed: the result of I_k iterations
 *    is the result of I_k plain time steps.  The oracle is therefore the plain
 *    time stepping, one step after another, in double precision.
 *
 *  - Thermal stencils (the paper's Hotspot / Hotspot3D workloads, Sec. III-C
 *    and Fig. 7; the paper does not print their update).  The explicit update
 *    used throughout this library is
 *        T' = T + k*(P + cy*(T_N + T_S - 2T) + cx*(T_E + T_W - 2T)
 *                   + cz*(t_amb - T) [+ cz2*(T_U + T_D - 2T) in 3D])
 *    with N/S = y-1/y+1 (rows), W/E = x-1/x+1 (columns), D/U = z-1/z+1.
 *    Boundary "clamp": a neighbour outside the grid reads the cell's own
 *    value (zero flux).  Boundary "Dirichlet-0": it reads 0.
 *    In 3D the power map P is a single x-y plane that acts on layer z = 0
 *    only; every other layer has no source.
 *
 *  - FDTD (the paper's Maxwell solver, Sec. III-C: one H-field kernel and one
 *    E-field kernel per step).  The paper does not print the scheme; this is
 *    the textbook Yee leapfrog in normalised units (eps = mu = c = 1,
 *    dx = dy = dz = 1, dt = courant number s), PEC walls on a cube of N cells:
 *        H^{n+1/2} = H^{n-1/2} - s * curl_forward(E^n)
 *        E^{n+1}   = E^n       + s * curl_backward(H^{n+1/2})  (interior only)
 *    followed by a soft source Ez[src] += amp*exp(-((n - delay)/width)^2).
 *    Staggering: Ex(i+1/2,j,k), Ey(i,j+1/2,k), Ez(i,j,k+1/2),
 *    Hx(i,j+1/2,k+1/2), Hy(i+1/2,j,k+1/2), Hz(i+1/2,j+1/2,k); every
 *    component is stored in a dense (N+1)^3 array indexed [k][j][i].
 *
 *  - The same scheme in linear, possibly lossy media with a per-cell
 *    material map (or_fdtd_run_media; the paper's solver models a vacuum
 *    cavity, this is the general-medium form of the same Yee update).
 *
 * All arrays here are dense (no pitch), x fastest.  Floating point
 * contraction is disabled at build time (-ffp-contract=off) so that results
 * are the same on x86-64 and aarch64 hosts.  The OpenMP pragmas only split
 * the outer loop of a Jacobi-type update across threads; every cell is still
 * computed from the previous state by the same expression.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_BC_CLAMP 0
#define OR_BC_DIRICHLET0 1

typedef struct {
    double k, cx, cy, cz, cz2, t_amb;
} or_heat_coeffs;

/* Neighbour read with the boundary rule: inside -> the value, outside ->
 * the centre value (clamp) or 0 (Dirichlet-0). */
static double nb(int inside, double v_inside, double centre, int bc)
{
    if (inside) return v_inside;
    return bc == OR_BC_CLAMP ? centre : 0.0;
}

/* One explicit 2D thermal step (5-point).  T, Tn: ny*nx; P: ny*nx. */
void or_heat2d_step(int64_t nx, int64_t ny, const double *T, const double *P,
                    double *Tn, const or_heat_coeffs *c, int bc)
{
    int64_t y;
#pragma omp parallel for schedule(static)
    for (y = 0; y < ny; ++y) {
        for (int64_t x = 0; x < nx; ++x) {
            const int64_t i = y * nx + x;
            const double t = T[i];
            const double tn = nb(y > 0, y > 0 ? T[i - nx] : 0.0, t, bc);
            const double ts = nb(y < ny - 1, y < ny - 1 ? T[i + nx] : 0.0, t, bc);
            const double tw = nb(x > 0, x > 0 ? T[i - 1] : 0.0, t, bc);
            const double te = nb(x < nx - 1, x < nx - 1 ? T[i + 1] : 0.0, t, bc);
            Tn[i] = t + c->k * (P[i] + c->cy * (tn + ts - 2.0 * t)
                                + c->cx * (te + tw - 2.0 * t)
                                + c->cz * (c->t_amb - t));
        }
    }
}

/* One explicit 3D thermal step (7-point).  T, Tn: nz*ny*nx; P: ny*nx plane
 * acting on layer 0 only. */
void or_heat3d_step(int64_t nx, int64_t ny, int64_t nz, const double *T,
                    const double *P, double *Tn, const or_heat_coeffs *c, int bc)
{
    const int64_t plane = nx * ny;
    int64_t z;
#pragma omp parallel for schedule(static)
    for (z = 0; z < nz; ++z) {
        for (int64_t y = 0; y < ny; ++y) {
            for (int64_t x = 0; x < nx; ++x) {
                const int64_t i = z * plane + y * nx + x;
                const double t = T[i];
                const double tn = nb(y > 0, y > 0 ? T[i - nx] : 0.0, t, bc);
                const double ts = nb(y < ny - 1, y < ny - 1 ? T[i + nx] : 0.0, t, bc);
                const double tw = nb(x > 0, x > 0 ? T[i - 1] : 0.0, t, bc);
                const double te = nb(x < nx - 1, x < nx - 1 ? T[i + 1] : 0.0, t, bc);
                const double td = nb(z > 0, z > 0 ? T[i - plane] : 0.0, t, bc);
                const double tu = nb(z < nz - 1, z < nz - 1 ? T[i + plane] : 0.0, t, bc);
                const double p = (z == 0) ? P[y * nx + x] : 0.0;
                Tn[i] = t + c->k * (p + c->cy * (tn + ts - 2.0 * t)
                                    + c->cx * (te + tw - 2.0 * t)
                                    + c->cz * (c->t_amb - t)
                                    + c->cz2 * (tu + td - 2.0 * t));
            }
        }
    }
}

/* n_steps thermal steps in place on T (nz == 1 selects the 2D stencil).
 * Returns 0, or -1 if the scratch buffer cannot be allocated. */
int or_heat_run(int64_t nx, int64_t ny, int64_t nz, int64_t n_steps, double *T,
                const double *P, const or_heat_coeffs *c, int bc)
{
    const int64_t n = nx * ny * nz;
    double *tmp = (double *)malloc((size_t)n * sizeof(double));
    if (!tmp) return -1;
    double *a = T, *b = tmp;
    for (int64_t s = 0; s < n_steps; ++s) {
        if (nz == 1)
            or_heat2d_step(nx, ny, a, P, b, c, bc);
        else
            or_heat3d_step(nx, ny, nz, a, P, b, c, bc);
        double *sw = a; a = b; b = sw;
    }
    if (a != T) memcpy(T, a, (size_t)n * sizeof(double));
    free(tmp);
    return 0;
}

/* ---------------------------------------------------------------- FDTD --- */

/* Index of (i, j, k) in a dense (N+1)^3 component array. */
static inline int64_t yee(int64_t N, int64_t i, int64_t j, int64_t k)
{
    const int64_t m = N + 1;
    return (k * m + j) * m + i;
}

/* H^{n+1/2} = H^{n-1/2} - s*curl(E^n), forward differences.  Every H value
 * whose stencil lies in the (N+1)^3 box is updated; H on PEC faces sees only
 * tangential E, which is zero, and so keeps its value. */
void or_fdtd_h(int64_t N, double s, const double *Ex, const double *Ey,
               const double *Ez, double *Hx, double *Hy, double *Hz)
{
    int64_t k;
#pragma omp parallel for schedule(static)
    for (k = 0; k <= N; ++k) {
        for (int64_t j = 0; j <= N; ++j) {
            for (int64_t i = 0; i <= N; ++i) {
                const int64_t c = yee(N, i, j, k);
                if (j < N && k < N) /* Hx(i, j+1/2, k+1/2) */
                    Hx[c] -= s * ((Ez[yee(N, i, j + 1, k)] - Ez[c])
                                  - (Ey[yee(N, i, j, k + 1)] - Ey[c]));
                if (i < N && k < N) /* Hy(i+1/2, j, k+1/2) */
                    Hy[c] -= s * ((Ex[yee(N, i, j, k + 1)] - Ex[c])
                                  - (Ez[yee(N, i + 1, j, k)] - Ez[c]));
                if (i < N && j < N) /* Hz(i+1/2, j+1/2, k) */
                    Hz[c] -= s * ((Ey[yee(N, i + 1, j, k)] - Ey[c])
                                  - (Ex[yee(N, i, j + 1, k)] - Ex[c]));
            }
        }
    }
}

/* E^{n+1} = E^n + s*curl(H^{n+1/2}), backward differences, on the interior
 * unknowns only: tangential E on the PEC walls is never written (it stays 0
 * when it starts at 0). */
void or_fdtd_e(int64_t N, double s, double *Ex, double *Ey, double *Ez,
               const double *Hx, const double *Hy, const double *Hz)
{
    int64_t k;
#pragma omp parallel for schedule(static)
    for (k = 0; k <= N; ++k) {
        for (int64_t j = 0; j <= N; ++j) {
            for (int64_t i = 0; i <= N; ++i) {
                const int64_t c = yee(N, i, j, k);
                if (i < N && j >= 1 && j <= N - 1 && k >= 1 && k <= N - 1) /* Ex */
                    Ex[c] += s * ((Hz[c] - Hz[yee(N, i, j - 1, k)])
                                  - (Hy[c] - Hy[yee(N, i, j, k - 1)]));
                if (j < N && i >= 1 && i <= N - 1 && k >= 1 && k <= N - 1) /* Ey */
                    Ey[c] += s * ((Hx[c] - Hx[yee(N, i, j, k - 1)])
                                  - (Hz[c] - Hz[yee(N, i - 1, j, k)]));
                if (k < N && i >= 1 && i <= N - 1 && j >= 1 && j <= N - 1) /* Ez */
                    Ez[c] += s * ((Hy[c] - Hy[yee(N, i - 1, j, k)])
                                  - (Hx[c] - Hx[yee(N, i, j - 1, k)]));
            }
        }
    }
}

/* Soft Gaussian point source: amplitude of step n. */
double or_fdtd_source(double n, double amp, double delay, double width)
{
    const double u = (n - delay) / width;
    return amp * exp(-u * u);
}

/* Steps n0 .. n0+n_steps-1 of the leapfrog: H update, E update, then (if
 * src_on) Ez[src] += source(n). */
void or_fdtd_run(int64_t N, int64_t n0, int64_t n_steps, double s, double *Ex,
                 double *Ey, double *Ez, double *Hx, double *Hy, double *Hz,
                 int src_on, int64_t si, int64_t sj, int64_t sk, double amp,
                 double delay, double width)
{
    for (int64_t n = n0; n < n0 + n_steps; ++n) {
        or_fdtd_h(N, s, Ex, Ey, Ez, Hx, Hy, Hz);
        or_fdtd_e(N, s, Ex, Ey, Ez, Hx, Hy, Hz);
        if (src_on)
            Ez[yee(N, si, sj, sk)] += or_fdtd_source((double)n, amp, delay, width);
    }
}

/* ---------------------------------------------------------------------
 * Yee leapfrog in linear, possibly lossy media (the textbook lossy-medium
 * update with the conduction term averaged over the two time levels,
 * Taflove & Hagness, Computational Electrodynamics, Ch. 3), normalised as
 * above (eps0 = mu0 = c = 1, dx = 1, dt = s).  Material m has relative
 * permittivity eps_r, conductivity sigma, relative permeability mu_r and
 * magnetic conductivity sigma_m; with
 *   a_e = sigma s / (2 eps_r),   a_h = sigma_m s / (2 mu_r):
 *   E^{n+1}   = ca E^n       + cb curl H^{n+1/2},
 *               ca = (1 - a_e)/(1 + a_e),  cb = (s/eps_r)/(1 + a_e);
 *   H^{n+1/2} = da H^{n-1/2} - db curl E^n,
 *               da = (1 - a_h)/(1 + a_h),  db = (s/mu_r)/(1 + a_h).
 * Every component at array index c = [k][j][i] takes the material mat[c]
 * (the cell whose lower corner is (i, j, k)); ids >= n_mat are vacuum.
 * ------------------------------------------------------------------- */
typedef struct {
    double ca, cb, da, db;
} or_medium;

static or_medium or_medium_of(double s, double eps_r, double sigma, double mu_r, double sigma_m)
{
    or_medium m;
    const double ae = sigma * s / (2.0 * eps_r);
    const double ah = sigma_m * s / (2.0 * mu_r);
    m.ca = (1.0 - ae) / (1.0 + ae);
    m.cb = (s / eps_r) / (1.0 + ae);
    m.da = (1.0 - ah) / (1.0 + ah);
    m.db = (s / mu_r) / (1.0 + ah);
    return m;
}

static void or_fdtd_h_media(int64_t N, const or_medium *tab, const uint8_t *mat,
                            const double *Ex, const double *Ey, const double *Ez,
                            double *Hx, double *Hy, double *Hz)
{
    int64_t k;
#pragma omp parallel for schedule(static)
    for (k = 0; k <= N; ++k) {
        for (int64_t j = 0; j <= N; ++j) {
            for (int64_t i = 0; i <= N; ++i) {
                const int64_t c = yee(N, i, j, k);
                const or_medium m = tab[mat[c]];
                if (j < N && k < N)
                    Hx[c] = m.da * Hx[c] - m.db * ((Ez[yee(N, i, j + 1, k)] - Ez[c])
                                                   - (Ey[yee(N, i, j, k + 1)] - Ey[c]));
                if (i < N && k < N)
                    Hy[c] = m.da * Hy[c] - m.db * ((Ex[yee(N, i, j, k + 1)] - Ex[c])
                                                   - (Ez[yee(N, i + 1, j, k)] - Ez[c]));
                if (i < N && j < N)
                    Hz[c] = m.da * Hz[c] - m.db * ((Ey[yee(N, i + 1, j, k)] - Ey[c])
                                                   - (Ex[yee(N, i, j + 1, k)] - Ex[c]));
            }
        }
    }
}

static void or_fdtd_e_media(int64_t N, const or_medium *tab, const uint8_t *mat,
                            double *Ex, double *Ey, double *Ez,
                            const double *Hx, const double *Hy, const double *Hz)
{
    int64_t k;
#pragma omp parallel for schedule(static)
    for (k = 0; k <= N; ++k) {
        for (int64_t j = 0; j <= N; ++j) {
            for (int64_t i = 0; i <= N; ++i) {
                const int64_t c = yee(N, i, j, k);
                const or_medium m = tab[mat[c]];
                if (i < N && j >= 1 && j <= N - 1 && k >= 1 && k <= N - 1)
                    Ex[c] = m.ca * Ex[c] + m.cb * ((Hz[c] - Hz[yee(N, i, j - 1, k)])
                                                   - (Hy[c] - Hy[yee(N, i, j, k - 1)]));
                if (j < N && i >= 1 && i <= N - 1 && k >= 1 && k <= N - 1)
                    Ey[c] = m.ca * Ey[c] + m.cb * ((Hx[c] - Hx[yee(N, i, j, k - 1)])
                                                   - (Hz[c] - Hz[yee(N, i - 1, j, k)]));
                if (k < N && i >= 1 && i <= N - 1 && j >= 1 && j <= N - 1)
                    Ez[c] = m.ca * Ez[c] + m.cb * ((Hy[c] - Hy[yee(N, i - 1, j, k)])
                                                   - (Hx[c] - Hx[yee(N, i, j - 1, k)]));
            }
        }
    }
}

/* or_fdtd_run in media: mat is an (N+1)^3 array of material ids; the
 * material table has n_mat (<= 256) rows given as four arrays. */
int or_fdtd_run_media(int64_t N, int64_t n0, int64_t n_steps, double s, double *Ex,
                      double *Ey, double *Ez, double *Hx, double *Hy, double *Hz,
                      const uint8_t *mat, int n_mat, const double *eps_r,
                      const double *sigma, const double *mu_r, const double *sigma_m,
                      int src_on, int64_t si, int64_t sj, int64_t sk, double amp,
                      double delay, double width)
{
    or_medium tab[256];
    if (n_mat < 0 || n_mat > 256)
        return 1;
    for (int m = 0; m < 256; ++m)
        tab[m] = (m < n_mat) ? or_medium_of(s, eps_r[m], sigma[m], mu_r[m], sigma_m[m])
                             : or_medium_of(s, 1.0, 0.0, 1.0, 0.0);
    for (int64_t n = n0; n < n0 + n_steps; ++n) {
        or_fdtd_h_media(N, tab, mat, Ex, Ey, Ez, Hx, Hy, Hz);
        or_fdtd_e_media(N, tab, mat, Ex, Ey, Ez, Hx, Hy, Hz);
        if (src_on)
            Ez[yee(N, si, sj, sk)] += or_fdtd_source((double)n, amp, delay, width);
    }
    return 0;
}

/* Number of OpenMP threads the oracle uses (1 when built without OpenMP). */
int or_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Set the OpenMP thread count of the calling thread's later loops (n >= 1);
   returns the count now in effect (1 when built without OpenMP). */
int or_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(n >= 1 ? n : 1);
#else
    (void)n;
#endif
    return or_num_threads();
}
