// Setup kernels: cell classes and sound-speed field (Sec. VI, Eq. 79), the
// standing-wave initial condition imposed through the equilibrium (Sec. V,
// Eqs. 71-72), surface elements (Sec. VI) and the interpolation stencils with
// the three-point kernel of Eq. (82).
#include <cuda_fp16.h>

#include "wlb_internal.cuh"

namespace wlb {
namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double kHalfPi = 1.5707963267948966192313216916398;
constexpr double kGoldenTurn = 0.3819660112501051517954131656;  // (3 - sqrt 5) / 2

__device__ __forceinline__ int wrap_index(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Minimum-image displacement along a periodic axis of length n.
__device__ __forceinline__ double min_image(double d, int n) {
    if (d >= 0.5 * n) return d - n;
    if (d < -0.5 * n) return d + n;
    return d;
}

// |x - r0|^2 - R^2, exact for centres on a 2^-10 grid.
__device__ double excess_r2(const Geometry &g, int x, int y, int z) {
    const int c[3] = {x, y, z};
    double s = 0.0;
    for (int a = 0; a < g.dim; ++a) {
        double d = min_image(__dadd_rn((double)c[a], -g.center[a]), g.n[a]);
        s = __dadd_rn(s, __dmul_rn(d, d));
    }
    return __dadd_rn(s, -__dmul_rn(g.radius, g.radius));
}

__device__ uint8_t cell_class(const Geometry &g, double q) {
    if (q >= g.band_half) return CELL_FLUID;
    if (q <= -g.band_half) return CELL_OBJECT;
    return CELL_BAND;
}

// Sound speed squared as the update kernel uses it: c0^2 for fluid cells,
// cp^2 for object cells, Eq. (79) (c0 outside, cp inside) in the band.
__device__ double sound_speed_sq(const Geometry &g, int x, int y, int z) {
    double q = excess_r2(g, x, y, z);
    uint8_t k = cell_class(g, q);
    if (k == CELL_FLUID) return g.c0 * g.c0;
    if (k == CELL_OBJECT) return g.cp * g.cp;
    double c = g.cp + 0.5 * (g.c0 - g.cp) * (1.0 + tanh(q / g.interface_d));
    return c * c;
}

// Standing-wave pressure at t = 0 (Eq. 38, s measured from an antinode), one
// value per coordinate along the wave axis.
__global__ void incident_table(Geometry g, double *__restrict__ ptab) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n[g.wave_axis]) return;
    ptab[s] = g.p_a * cos(2.0 * kPi * ((double)s - g.antinode) / g.wavelength);
}

// Conversion of an FP64 value to the storage type (round to nearest).
template <typename S> __device__ __forceinline__ S to_store(double v) { return (S)v; }
template <> __device__ __forceinline__ __half to_store<__half>(double v) { return __double2half(v); }

// Populations are stored post-collision and pulled by the next update, so the
// stored value of direction i at cell x is the value that arrives at x + v_i:
// the equilibrium (Eq. 71 with rho1 = p1/c^2, J1 = 0) of the cell x + v_i,
// times the storage scale.
template <typename S, typename T>
__global__ void setup_cells(Geometry g, S *__restrict__ pop, uint8_t *__restrict__ cls, uint8_t *__restrict__ band_rows,
                            T *__restrict__ c2f, const double *__restrict__ ptab) {
    long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= g.ncell) return;
    int x = (int)(id % g.n[0]);
    long long r = id / g.n[0];
    int y = (int)(r % g.n[1]);
    int z = (int)(r / g.n[1]);
    double q = excess_r2(g, x, y, z);
    const int cc[3] = {x, y, z};
    const int ax = g.wave_axis;
    uint8_t k = cell_class(g, q);
    if (g.driven) {
        const int sa = cc[ax], ns = g.n[ax];
        if (sa == 0) k = CELL_WALL_LO;
        else if (sa == ns - 1) k = CELL_WALL_HI;
        else if (sa == 1) k = CELL_SOURCE;
    }
    cls[id] = k;
    if (k == CELL_BAND) band_rows[r] = 1;  // r = z * ny + y; every writer stores the same value
    double c2 = sound_speed_sq(g, x, y, z);  // walls and source sheet lie in the fluid
    c2f[id] = (T)c2;
    double p = g.driven ? 0.0 : ptab[cc[ax]];  // the driven cavity starts from rest
    pop[id] = to_store<S>((p / c2) * (1.0 - g.dim * c2) * g.pop_scale);  // f_0^eq = rho1 (1 - D c^2)
    for (int i = 1; i < g.q; ++i) {
        int a = (i - 1) >> 1;
        int v = ((i - 1) & 1) ? -1 : 1;
        int c[3] = {x, y, z};
        c[a] = wrap_index(c[a] + v, g.n[a]);
        double pn = g.driven ? 0.0 : ptab[c[ax]];
        pop[(long long)i * g.ncell + id] = to_store<S>(0.5 * pn * g.pop_scale);  // f_i^eq = c^2 rho1 / 2
    }
}

// sin and cos of 2 pi t, t in [0, 1): exact quadrant reduction, then the Taylor
// series to x^21 (Horner in x^2, coefficients 1/n! from exact factorials) on
// [-pi/4, pi/4].  Only correctly rounded operations, no contraction, so the
// sequence of IEEE operations is fixed.
__device__ void sincos_turns(double t, double *s, double *c) {
    double u = __dmul_rn(t, 4.0);
    int q = (int)floor(u);
    double r = __dadd_rn(u, -(double)q);
    if (r > 0.5) { r = __dadd_rn(r, -1.0); q += 1; }
    double th = __dmul_rn(r, kHalfPi);
    double th2 = __dmul_rn(th, th);
    double fact[22];
    fact[0] = 1.0;
    for (int i = 1; i < 22; ++i) fact[i] = __dmul_rn(fact[i - 1], (double)i);
    double ps = 0.0, pc = 0.0;
    for (int m = 10; m >= 0; --m) {
        double cs = __ddiv_rn(1.0, fact[2 * m + 1]);
        double cc = __ddiv_rn(1.0, fact[2 * m]);
        if (m & 1) { cs = -cs; cc = -cc; }
        ps = __dadd_rn(__dmul_rn(ps, th2), cs);
        pc = __dadd_rn(__dmul_rn(pc, th2), cc);
    }
    double sv = __dmul_rn(th, ps), cv = pc;
    switch (q & 3) {
        case 0: *s = sv; *c = cv; break;
        case 1: *s = cv; *c = -sv; break;
        case 2: *s = -sv; *c = -cv; break;
        default: *s = -cv; *c = sv; break;
    }
}

// Eq. (82): three-point kernel, one axis.
__device__ double kernel3(double r) {
    double a = fabs(r);
    if (a <= 0.5) return (1.0 + sqrt(1.0 - 3.0 * r * r)) / 3.0;
    if (a <= 1.5) return (5.0 - 3.0 * a - sqrt(1.0 - 3.0 * (1.0 - a) * (1.0 - a))) / 6.0;
    return 0.0;
}

// One thread per surface element: centre, normal and size (Sec. VI), then the
// 3^dim stencil of Eqs. (80)-(81) with tensor-product weights.
template <typename T>
__global__ void setup_surface(Geometry g, double *__restrict__ pts, T *__restrict__ nrm,
                              int4 *__restrict__ st_xyz, T *__restrict__ st_w) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.n_surface) return;
    const double Rs = g.surface_radius;
    const int N = g.n_surface;
    double n[3] = {0.0, 0.0, 0.0};
    double dS;
    if (g.dim == 2) {
        double t = __ddiv_rn((double)(2 * k + 1), (double)(2 * N));
        sincos_turns(t, &n[1], &n[0]);
        dS = __ddiv_rn(__dmul_rn(__dmul_rn(2.0, kPi), Rs), (double)N);
    } else {
        double zk = __dadd_rn(1.0, -__ddiv_rn((double)(2 * k + 1), (double)N));
        double rho = __dsqrt_rn(__dadd_rn(1.0, -__dmul_rn(zk, zk)));
        double a = __dmul_rn((double)k, kGoldenTurn);
        double t = __dadd_rn(a, -floor(a));
        double sp, cp;
        sincos_turns(t, &sp, &cp);
        n[0] = __dmul_rn(rho, cp);
        n[1] = __dmul_rn(rho, sp);
        n[2] = zk;
        dS = __ddiv_rn(__dmul_rn(__dmul_rn(4.0, kPi), __dmul_rn(Rs, Rs)), (double)N);
    }
    double X[3];
    for (int a = 0; a < 3; ++a) {
        X[a] = (a < g.dim) ? __dadd_rn(g.center[a], __dmul_rn(Rs, n[a])) : 0.0;
        pts[7 * (long long)k + a] = X[a];
        pts[7 * (long long)k + 3 + a] = n[a];
        nrm[4 * (long long)k + a] = (T)n[a];
    }
    nrm[4 * (long long)k + 3] = (T)0;
    pts[7 * (long long)k + 6] = dS;

    int base[3] = {0, 0, 0};
    for (int a = 0; a < g.dim; ++a) base[a] = (int)floor(X[a] + 0.5);
    int slot = 0;
    const int lz = g.dim == 3 ? 1 : 0;
    for (int dz = -lz; dz <= lz; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int c[3] = {base[0] + dx, base[1] + dy, base[2] + dz};
                double w = 1.0;
                for (int a = 0; a < g.dim; ++a) w *= kernel3((double)c[a] - X[a]);
                int cx = wrap_index(c[0], g.n[0]);
                int cy = wrap_index(c[1], g.n[1]);
                int cz = g.dim == 3 ? wrap_index(c[2], g.n[2]) : 0;
                long long o = (long long)k * g.stencil + slot;
                st_xyz[o] = make_int4(cx, cy, cz, 0);
                st_w[2 * o] = (T)(w * sound_speed_sq(g, cx, cy, cz));
                st_w[2 * o + 1] = (T)(w / g.rho0);
                ++slot;
            }
}

template <typename S, typename T>
cudaError_t setup_impl(const Geometry &g, const Buffers &b, cudaStream_t s) {
    const int tb = 256;
    long long blocks = (g.ncell + tb - 1) / tb;
    const int ns = g.n[g.wave_axis];
    incident_table<<<(ns + 127) / 128, 128, 0, s>>>(g, b.ptab);
    cudaError_t e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return e0;
    cudaError_t e = cudaMemsetAsync(b.band_rows, 0, (size_t)g.n[1] * g.n[2], s);
    if (e != cudaSuccess) return e;
    setup_cells<S, T><<<(unsigned)blocks, tb, 0, s>>>(g, (S *)b.pop[0], b.cls, b.band_rows, (T *)b.c2, b.ptab);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (g.n_surface > 0) {
        setup_surface<T><<<(g.n_surface + 127) / 128, 128, 0, s>>>(
            g, b.pts, (T *)b.nrm, b.st_xyz, (T *)b.st_w);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(b.acc, 0, sizeof(T) * 5 * (size_t)g.n_surface, s);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(b.acc64, 0, sizeof(double) * 5 * (size_t)g.n_surface, s);
        if (e != cudaSuccess) return e;
    }
    e = cudaMemsetAsync(b.force, 0, 4 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(b.err, 0, sizeof(int), s);
}

}  // namespace

cudaError_t launch_setup(const Geometry &g, const Buffers &b, Prec p, cudaStream_t s) {
    switch (p) {
        case Prec::F64: return setup_impl<double, double>(g, b, s);
        case Prec::F16: return setup_impl<__half, float>(g, b, s);
        default: return setup_impl<float, float>(g, b, s);
    }
}

}  // namespace wlb
