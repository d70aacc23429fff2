/*
 * Plain FP64 CPU oracle for the wave lattice Boltzmann (LB) computation of the
 * acoustic radiation force on a density-matched compressible object
 * (Castro-Avila, Malgaretti, Harting, Munoz, "A lattice Boltzmann approach for
 * acoustic manipulation").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct statement
 * of what the GPU library computes.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the library never does, and it
 * shares no source, header, table or constant with the library.
 *
 * It follows the paper's steps in the paper's order, one full lattice pass per
 * step, with no fusion:
 *   sound speed     c(r)             Sec. VI, Eq. (79) (sign reading: cp inside)
 *   initial state   f = f^eq(rho1,0) Sec. V, Eq. (72) ("imposing fields")
 *   per time step   rho1, J1, p1     Sec. V, Eq. (62)
 *                   sample surface   Sec. VI, Eqs. (80)-(82), time average Sec. VII
 *                   BGK, tau = 1/2   Sec. V, Eqs. (63), (71)
 *                   advection        Sec. V, Eq. (64) (push form)
 *   force           King's integral  Sec. II, Eq. (14) (= Eq. (77) in LB variables)
 *
 * Pins (tests/test_oracle_*.py): collision conserves sum f and sum v f; a
 * uniform medium evolves a standing wave as the closed-form lattice mode
 * sin^2(w/2) = c^2 sum_a sin^2(k_a/2); kernel partition of unity, zero first
 * moment and constant square sum; divergence-theorem values of the force
 * functional; exact p_a^2 scaling; mirror symmetry at the node; Gor'kov (3D) and
 * Wei (2D) forces at small kR.  Surface-point generation is pinned against
 * libm sin/cos and the unit-sphere invariant.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (oracle/build.py).
 * FMA contraction is off so that the surface points follow the written
 * sequence of IEEE operations exactly.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int dim;               /* 2 (D2Q5) or 3 (D3Q7)                               */
    int n[3];              /* lattice extents along x, y, z; n[2] = 1 in 2D       */
    int wave_axis;         /* axis of the standing wave (0, 1 or 2)              */
    double c0;             /* fluid sound speed (lattice units)                  */
    double cp;             /* object sound speed                                 */
    double rho0;           /* mean density                                       */
    double p_a;            /* pressure amplitude of the standing wave            */
    double wavelength;     /* lambda in cells                                    */
    double antinode;       /* coordinate of a pressure antinode along wave_axis  */
    double center[3];      /* object centre r0                                   */
    double radius;         /* R_p                                                */
    double interface_d;    /* "square thickness" d of Eq. (79)                   */
    double surface_radius; /* radius of the integration surface                  */
    int n_surface;         /* number of surface elements N                       */
    long n_steps;          /* total LB steps                                     */
    long n_window;         /* the last n_window steps are averaged               */
    int driven;            /* 0: periodic box with the standing wave as initial
                              state; 1: driven walls along wave_axis (Sec. VII) */
    double wall_damping;   /* Phi of Eq. (73)                                    */
    double source_amplitude; /* rho_a of the source sheet                        */
} orc_problem;

enum { ORC_FLUID = 0, ORC_OBJECT = 1, ORC_BAND = 2, ORC_WALL_LO = 3, ORC_WALL_HI = 4, ORC_SOURCE = 5 };

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int orc_Q(int dim) { return 2 * dim + 1; }

size_t orc_cells(const orc_problem *P)
{
    return (size_t)P->n[0] * (size_t)P->n[1] * (size_t)P->n[2];
}

/* Velocity set of Fig. 8: v_0 = 0, then +e_a, -e_a for each axis a.  The moment
 * conditions of Eqs. (69)-(70) hold with w_0 = 1/3, w_i = 1/6, c_s^2 = 1/3 (D2Q5)
 * and w_0 = 1/4, w_i = 1/8, c_s^2 = 1/4 (D3Q7). */
static void velocity(int i, int v[3])
{
    v[0] = v[1] = v[2] = 0;
    if (i == 0) return;
    int a = (i - 1) / 2;
    v[a] = ((i - 1) % 2 == 0) ? 1 : -1;
}

static double weight(int dim, int i)
{
    if (dim == 2) return i == 0 ? 1.0 / 3.0 : 1.0 / 6.0;
    return i == 0 ? 1.0 / 4.0 : 1.0 / 8.0;
}

static double cs2(int dim) { return dim == 2 ? 1.0 / 3.0 : 1.0 / 4.0; }

static size_t cell_index(const orc_problem *P, int x, int y, int z)
{
    return ((size_t)z * P->n[1] + (size_t)y) * P->n[0] + (size_t)x;
}

static int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }

/* Periodic minimum-image displacement; exact for the quantised centres used. */
static double min_image(double d, int n)
{
    if (d >= 0.5 * n) return d - n;
    if (d < -0.5 * n) return d + n;
    return d;
}

static double dist2(const orc_problem *P, int x, int y, int z)
{
    int c[3] = {x, y, z};
    double s = 0.0;
    for (int a = 0; a < P->dim; ++a) {
        double d = min_image((double)c[a] - P->center[a], P->n[a]);
        s = s + d * d;
    }
    return s;
}

/* Eq. (79): smooth sound-speed profile of the object.  As printed, the profile
 * gives c_p far away and c_0 at the centre, which contradicts the text around
 * it (c_p is the object's speed); the oracle reads it as
 *     c(r) = c_p + (c_0 - c_p)/2 * (1 + tanh((|r - r0|^2 - R_p^2)/d)),
 * i.e. c_0 in the fluid, c_p inside the object, (c_0 + c_p)/2 on |r - r0| = R_p. */
double orc_sound_speed(const orc_problem *P, int x, int y, int z)
{
    double q = dist2(P, x, y, z) - P->radius * P->radius;
    return P->cp + 0.5 * (P->c0 - P->cp) * (1.0 + tanh(q / P->interface_d));
}

void orc_sound_speed_sq_field(const orc_problem *P, double *c2)
{
    for (int z = 0; z < P->n[2]; ++z)
        for (int y = 0; y < P->n[1]; ++y)
            for (int x = 0; x < P->n[0]; ++x) {
                double c = orc_sound_speed(P, x, y, z);
                c2[cell_index(P, x, y, z)] = c * c;
            }
}

/* Cell classes: the tanh of Eq. (79) rounds to exactly +-1 in double precision
 * when |(|r - r0|^2 - R^2)/d| >= 20; cells beyond that are pure fluid or pure
 * object, the rest form the interface band.  Decided on the exact value of
 * |r - r0|^2. */
void orc_mask(const orc_problem *P, unsigned char *mask)
{
    double half = 20.0 * P->interface_d;
    double R2 = P->radius * P->radius;
    for (int z = 0; z < P->n[2]; ++z)
        for (int y = 0; y < P->n[1]; ++y)
            for (int x = 0; x < P->n[0]; ++x) {
                double q = dist2(P, x, y, z) - R2;
                unsigned char c = ORC_BAND;
                if (q >= half) c = ORC_FLUID;
                else if (q <= -half) c = ORC_OBJECT;
                if (P->driven) {
                    int cc[3] = {x, y, z};
                    int sa = cc[P->wave_axis], ns = P->n[P->wave_axis];
                    if (sa == 0) c = ORC_WALL_LO;
                    else if (sa == ns - 1) c = ORC_WALL_HI;
                    else if (sa == 1) c = ORC_SOURCE;
                }
                mask[cell_index(P, x, y, z)] = c;
            }
}

/* ---------------------------------------------------------------------------
 * Surface elements (Sec. VI): centre R_k, unit normal n_k, element size dS_k.
 * 2D: N equal arcs, angle 2 pi (k + 1/2)/N.  3D: Fibonacci lattice,
 * z_k = 1 - (2k+1)/N, azimuth k * pi (3 - sqrt 5).  Angles are carried in turns
 * and sin/cos come from the truncated Taylor series (terms up to x^21) evaluated
 * on [-pi/4, pi/4] after an exact quadrant reduction, using only correctly
 * rounded +, -, *, /, sqrt, so the result is one fixed sequence of IEEE
 * operations.
 * ------------------------------------------------------------------------- */
static double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f = f * (double)i;   /* exact for n <= 22 */
    return f;
}

/* sin and cos of 2*pi*t for t in [0, 1). */
void orc_sincos_turns(double t, double *s, double *c)
{
    const double half_pi = 1.5707963267948966192313216916398;
    double u = t * 4.0;                 /* exact */
    int q = (int)floor(u);
    double r = u - (double)q;           /* exact, in [0, 1) */
    if (r > 0.5) { r = r - 1.0; q = q + 1; }
    double th = r * half_pi;            /* |th| <= pi/4 */
    double th2 = th * th;
    /* sin: th * sum_{m=0..10} (-1)^m th^(2m) / (2m+1)! , Horner from the top */
    double ps = 0.0;
    for (int m = 10; m >= 0; --m) {
        double coef = 1.0 / factorial(2 * m + 1);
        if (m % 2) coef = -coef;
        ps = ps * th2 + coef;
    }
    double sv = th * ps;
    /* cos: sum_{m=0..10} (-1)^m th^(2m) / (2m)! */
    double pc = 0.0;
    for (int m = 10; m >= 0; --m) {
        double coef = 1.0 / factorial(2 * m);
        if (m % 2) coef = -coef;
        pc = pc * th2 + coef;
    }
    double cv = pc;
    switch (q & 3) {
    case 0: *s = sv;  *c = cv;  break;
    case 1: *s = cv;  *c = -sv; break;
    case 2: *s = -sv; *c = -cv; break;
    default: *s = -cv; *c = sv; break;
    }
}

/* pts: N rows of (x, y, z, nx, ny, nz, dS). */
void orc_surface_points(const orc_problem *P, double *pts)
{
    const double pi = 3.14159265358979323846264338327950288;
    const double golden_turn = 0.3819660112501051517954131656;  /* (3 - sqrt 5)/2 */
    int N = P->n_surface;
    double Rs = P->surface_radius;
    for (int k = 0; k < N; ++k) {
        double n[3] = {0.0, 0.0, 0.0};
        double dS;
        if (P->dim == 2) {
            double t = (double)(2 * k + 1) / (double)(2 * N);
            orc_sincos_turns(t, &n[1], &n[0]);
            dS = (2.0 * pi * Rs) / (double)N;
        } else {
            double z = 1.0 - (double)(2 * k + 1) / (double)N;
            double rho = sqrt(1.0 - z * z);
            double a = (double)k * golden_turn;
            double t = a - floor(a);
            double sp, cp;
            orc_sincos_turns(t, &sp, &cp);
            n[0] = rho * cp;
            n[1] = rho * sp;
            n[2] = z;
            dS = (4.0 * pi * (Rs * Rs)) / (double)N;
        }
        double *row = pts + 7 * (size_t)k;
        for (int a = 0; a < 3; ++a) {
            row[a] = (a < P->dim) ? P->center[a] + Rs * n[a] : 0.0;
            row[3 + a] = n[a];
        }
        row[6] = dS;
    }
}

/* Eq. (82): three-point kernel of Roma et al., applied per axis (tensor product). */
double orc_kernel(double r)
{
    double a = fabs(r);
    if (a <= 0.5) return (1.0 + sqrt(1.0 - 3.0 * r * r)) / 3.0;
    if (a <= 1.5) return (5.0 - 3.0 * a - sqrt(1.0 - 3.0 * (1.0 - a) * (1.0 - a))) / 6.0;
    return 0.0;
}

/* Eq. (71): wave equilibrium, written with the weights and c_s^2 of Eqs. (69)-(70). */
static void equilibrium(int dim, double c2, double rho, const double J[3], double *feq)
{
    int Q = orc_Q(dim);
    double s2 = cs2(dim);
    feq[0] = rho * (1.0 + (1.0 / s2) * c2 * (weight(dim, 0) - 1.0));
    for (int i = 1; i < Q; ++i) {
        int v[3];
        velocity(i, v);
        double vJ = v[0] * J[0] + v[1] * J[1] + v[2] * J[2];
        feq[i] = (1.0 / s2) * weight(dim, i) * (c2 * rho + vJ);
    }
}

/* Standing-wave pressure at t = 0, Eq. (38) with s measured from an antinode. */
static double incident_pressure(const orc_problem *P, int x, int y, int z)
{
    const double pi = 3.14159265358979323846264338327950288;
    int c[3] = {x, y, z};
    double s = (double)c[P->wave_axis] - P->antinode;
    return P->p_a * cos(2.0 * pi * s / P->wavelength);
}

/* Eq. (72), used for the initial condition: f = f^eq(rho1 = p1/c^2, J1 = 0).
 * Layout f[i][z][y][x]. */
void orc_initial_populations(const orc_problem *P, const double *c2, double *f)
{
    size_t cells = orc_cells(P);
    int Q = orc_Q(P->dim);
    double J0[3] = {0.0, 0.0, 0.0};
    for (int z = 0; z < P->n[2]; ++z)
        for (int y = 0; y < P->n[1]; ++y)
            for (int x = 0; x < P->n[0]; ++x) {
                size_t id = cell_index(P, x, y, z);
                double rho = P->driven ? 0.0 : incident_pressure(P, x, y, z) / c2[id];
                double feq[7];
                equilibrium(P->dim, c2[id], rho, J0, feq);
                for (int i = 0; i < Q; ++i) f[(size_t)i * cells + id] = feq[i];
            }
}

/* Eq. (62): rho1 = sum_i f_i, J1 = sum_i v_i f_i.  J has dim components per cell,
 * stored as J[a][cell]. */
void orc_macroscopic(const orc_problem *P, const double *f, double *rho, double *J)
{
    size_t cells = orc_cells(P);
    int Q = orc_Q(P->dim);
    int dim = P->dim;
#pragma omp parallel for schedule(static)
    for (long id = 0; id < (long)cells; ++id) {
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; ++i) {
            int v[3];
            velocity(i, v);
            double fi = f[(size_t)i * cells + id];
            r += fi;
            for (int a = 0; a < dim; ++a) j[a] += v[a] * fi;
        }
        rho[id] = r;
        for (int a = 0; a < dim; ++a) J[(size_t)a * cells + id] = j[a];
    }
}

/* Eq. (63) with tau = 1/2 and dt = 1, written as printed:
 *   f_new = (1 - dt/tau) f + (dt/tau) f^eq. */
void orc_collide(const orc_problem *P, const double *c2, const double *f, double *fnew)
{
    size_t cells = orc_cells(P);
    int Q = orc_Q(P->dim);
    int dim = P->dim;
    const double dt = 1.0, tau = 0.5;
#pragma omp parallel for schedule(static)
    for (long id = 0; id < (long)cells; ++id) {
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; ++i) {
            int v[3];
            velocity(i, v);
            double fi = f[(size_t)i * cells + id];
            r += fi;
            for (int a = 0; a < dim; ++a) j[a] += v[a] * fi;
        }
        double feq[7];
        equilibrium(dim, c2[id], r, j, feq);
        for (int i = 0; i < Q; ++i) {
            size_t k = (size_t)i * cells + id;
            fnew[k] = (1.0 - dt / tau) * f[k] + (dt / tau) * feq[i];
        }
    }
}

/* Driven-wall geometry of Sec. VII, applied to the post-collision values of
 * step t (whose pre-collision populations are f):
 *  - the two end planes along wave_axis are partially absorbing walls, where
 *    a bounce-back step replaces the collision (Eq. 73): f_i^new = Phi f_j
 *    with v_j = -v_i; the value that would leave the domain is dropped;
 *  - the plane next to the low wall is the source sheet, where fields are
 *    imposed after the collision (Eq. 72): f^new = f^eq(rho_a sin(w t), J1)
 *    with J1 from Eq. (62) and w = 2 pi / T, T = lambda / c0 (t taken modulo T). */
void orc_apply_boundaries(const orc_problem *P, const double *c2, const double *f, double *fnew, long t)
{
    if (!P->driven) return;
    const double pi = 3.14159265358979323846264338327950288;
    size_t cells = orc_cells(P);
    int Q = orc_Q(P->dim), a = P->wave_axis, ns = P->n[a];
    long T = (long)(P->wavelength / P->c0 + 0.5);
    double rho_src = P->source_amplitude * sin(2.0 * pi * (double)(t % T) / (double)T);
    for (int z = 0; z < P->n[2]; ++z)
        for (int y = 0; y < P->n[1]; ++y)
            for (int x = 0; x < P->n[0]; ++x) {
                int cc[3] = {x, y, z};
                int sa = cc[a];
                if (sa != 0 && sa != 1 && sa != ns - 1) continue;
                size_t id = cell_index(P, x, y, z);
                double fi[7];
                for (int i = 0; i < Q; ++i) fi[i] = f[(size_t)i * cells + id];
                if (sa == 1) {
                    double J[3] = {0.0, 0.0, 0.0};
                    for (int i = 1; i < Q; ++i) {
                        int v[3];
                        velocity(i, v);
                        for (int b = 0; b < P->dim; ++b) J[b] += v[b] * fi[i];
                    }
                    double feq[7];
                    equilibrium(P->dim, c2[id], rho_src, J, feq);
                    for (int i = 0; i < Q; ++i) fnew[(size_t)i * cells + id] = feq[i];
                } else {
                    for (int i = 0; i < Q; ++i) {
                        int opp = i == 0 ? 0 : (((i - 1) % 2 == 0) ? i + 1 : i - 1);
                        fnew[(size_t)i * cells + id] = P->wall_damping * fi[opp];
                    }
                    /* outward direction: -a at the low wall, +a at the high wall */
                    int out = sa == 0 ? 2 + 2 * a : 1 + 2 * a;
                    fnew[(size_t)out * cells + id] = 0.0;
                }
            }
}

/* Eq. (64): f_i(x + v_i) = f_i^new(x), periodic on every axis. */
void orc_advect(const orc_problem *P, const double *fnew, double *f)
{
    size_t cells = orc_cells(P);
    int Q = orc_Q(P->dim);
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < P->n[2]; ++z)
        for (int y = 0; y < P->n[1]; ++y)
            for (int x = 0; x < P->n[0]; ++x) {
                size_t from = cell_index(P, x, y, z);
                for (int i = 0; i < Q; ++i) {
                    int v[3];
                    velocity(i, v);
                    size_t to = cell_index(P, wrap(x + v[0], P->n[0]),
                                           wrap(y + v[1], P->n[1]),
                                           wrap(z + v[2], P->n[2]));
                    f[(size_t)i * cells + to] = fnew[(size_t)i * cells + from];
                }
            }
}

/* Eqs. (80)-(82): p1 = c^2 rho1 (Eq. 62) and u1 = J1/rho0 interpolated to every
 * surface point with the tensor-product kernel over the 3^dim nearest cells.
 * P_out[k], U_out[3k + a]. */
void orc_interpolate(const orc_problem *P, const double *pts, const double *c2,
                     const double *rho, const double *J, double *P_out, double *U_out)
{
    size_t cells = orc_cells(P);
    int dim = P->dim;
    for (int k = 0; k < P->n_surface; ++k) {
        const double *X = pts + 7 * (size_t)k;
        int base[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) base[a] = (int)floor(X[a] + 0.5);
        double p = 0.0, u[3] = {0.0, 0.0, 0.0};
        int lz = dim == 3 ? 1 : 0;
        for (int dz = -lz; dz <= lz; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int c[3] = {base[0] + dx, base[1] + dy, base[2] + dz};
                    double w = 1.0;
                    for (int a = 0; a < dim; ++a) w *= orc_kernel((double)c[a] - X[a]);
                    size_t id = cell_index(P, wrap(c[0], P->n[0]), wrap(c[1], P->n[1]),
                                           dim == 3 ? wrap(c[2], P->n[2]) : 0);
                    p += w * c2[id] * rho[id];
                    for (int a = 0; a < dim; ++a) u[a] += w * J[(size_t)a * cells + id] / P->rho0;
                }
        P_out[k] = p;
        for (int a = 0; a < 3; ++a) U_out[3 * (size_t)k + a] = u[a];
    }
}

/* Eq. (14) (King), evaluated on the N surface elements with time averages
 * <p1^2> = Spp/n_window, <u1.u1> = Suu/n_window, <u1 (u1.n)> = Snu/n_window:
 *   F_i = - sum_k dS_k [ (<p1^2>/(2 rho0 c0^2) - rho0 <u1^2>/2) n_ki
 *                        + rho0 <u1_i (u1 . n_k)> ].                      */
void orc_force(int dim, int N, const double *pts, const double *Spp, const double *Suu,
               const double *Snu, double n_window, double rho0, double c0, double F[3])
{
    F[0] = F[1] = F[2] = 0.0;
    for (int k = 0; k < N; ++k) {
        const double *row = pts + 7 * (size_t)k;
        double pp = Spp[k] / n_window, uu = Suu[k] / n_window;
        double iso = pp / (2.0 * rho0 * c0 * c0) - 0.5 * rho0 * uu;
        for (int i = 0; i < dim; ++i) {
            double nu_i = Snu[3 * (size_t)k + i] / n_window;
            F[i] -= row[6] * (iso * row[3 + i] + rho0 * nu_i);
        }
    }
}

/* Whole protocol.  Optional outputs (NULL to skip):
 *   p1_out[cell], u1_out[a][cell]  fields at t = n_steps
 *   f_out[i][cell]                 populations at t = n_steps (pre-collision)
 *   sums_out[k][0..4]              Spp, Suu, Snu_x, Snu_y, Snu_z
 *   pts_out[k][7]                  surface elements
 * Returns 0 on success, -1 on allocation failure. */
int orc_run(const orc_problem *P, double F[3], double *p1_out, double *u1_out,
            double *f_out, double *sums_out, double *pts_out)
{
    size_t cells = orc_cells(P);
    int Q = orc_Q(P->dim), dim = P->dim, N = P->n_surface;
    double *c2 = malloc(cells * sizeof(double));
    double *f = malloc((size_t)Q * cells * sizeof(double));
    double *fnew = malloc((size_t)Q * cells * sizeof(double));
    double *rho = malloc(cells * sizeof(double));
    double *J = malloc((size_t)dim * cells * sizeof(double));
    double *pts = malloc((size_t)(N > 0 ? N : 1) * 7 * sizeof(double));
    double *Pk = malloc((size_t)(N > 0 ? N : 1) * sizeof(double));
    double *Uk = malloc((size_t)(N > 0 ? N : 1) * 3 * sizeof(double));
    double *Spp = calloc((size_t)(N > 0 ? N : 1), sizeof(double));
    double *Suu = calloc((size_t)(N > 0 ? N : 1), sizeof(double));
    double *Snu = calloc((size_t)(N > 0 ? N : 1) * 3, sizeof(double));
    int rc = 0;
    if (!c2 || !f || !fnew || !rho || !J || !pts || !Pk || !Uk || !Spp || !Suu || !Snu) {
        rc = -1;
        goto done;
    }
    orc_sound_speed_sq_field(P, c2);
    orc_surface_points(P, pts);
    orc_initial_populations(P, c2, f);
    for (long t = 0; t < P->n_steps; ++t) {
        if (t >= P->n_steps - P->n_window && N > 0) {
            orc_macroscopic(P, f, rho, J);
            orc_interpolate(P, pts, c2, rho, J, Pk, Uk);
            for (int k = 0; k < N; ++k) {
                const double *nk = pts + 7 * (size_t)k + 3;
                double *U = Uk + 3 * (size_t)k;
                double un = U[0] * nk[0] + U[1] * nk[1] + U[2] * nk[2];
                Spp[k] += Pk[k] * Pk[k];
                Suu[k] += U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
                for (int a = 0; a < 3; ++a) Snu[3 * (size_t)k + a] += U[a] * un;
            }
        }
        orc_collide(P, c2, f, fnew);
        orc_apply_boundaries(P, c2, f, fnew, t);
        orc_advect(P, fnew, f);
    }
    if (P->n_window > 0)
        orc_force(dim, N, pts, Spp, Suu, Snu, (double)P->n_window, P->rho0, P->c0, F);
    else
        F[0] = F[1] = F[2] = 0.0;
    if (p1_out || u1_out) {
        orc_macroscopic(P, f, rho, J);
        for (size_t id = 0; id < cells; ++id) {
            if (p1_out) p1_out[id] = c2[id] * rho[id];
            if (u1_out)
                for (int a = 0; a < dim; ++a)
                    u1_out[(size_t)a * cells + id] = J[(size_t)a * cells + id] / P->rho0;
        }
    }
    if (f_out) memcpy(f_out, f, (size_t)Q * cells * sizeof(double));
    if (sums_out)
        for (int k = 0; k < N; ++k) {
            sums_out[5 * (size_t)k + 0] = Spp[k];
            sums_out[5 * (size_t)k + 1] = Suu[k];
            for (int a = 0; a < 3; ++a) sums_out[5 * (size_t)k + 2 + a] = Snu[3 * (size_t)k + a];
        }
    if (pts_out) memcpy(pts_out, pts, (size_t)N * 7 * sizeof(double));
done:
    free(c2); free(f); free(fnew); free(rho); free(J); free(pts);
    free(Pk); free(Uk); free(Spp); free(Suu); free(Snu);
    return rc;
}
