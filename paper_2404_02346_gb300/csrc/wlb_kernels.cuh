// Device-side building blocks shared by the single-lattice and batched kernels:
// storage traits of the populations and the pull-sum of the moments.
#pragma once
#include <cuda_fp16.h>

#include "wlb_internal.cuh"

namespace wlb {

constexpr unsigned kFull = 0xffffffffu;

// Storage traits: R is the arithmetic type, W the values per 16-byte vector.
// Vector accesses use streaming cache hints: every population is read once and
// written once per step.
template <typename S> struct Store;

template <> struct Store<float> {
    using R = float;
    static constexpr int W = 4;
    __device__ static void load(const float *p, float (&v)[4]) {
        const float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    __device__ static void store(float *p, const float (&v)[4]) {
        __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
    }
    __device__ static void store_keep(float *p, const float (&v)[4]) {  // normal L2 priority
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
    __device__ static void load_cg(const float *p, float (&v)[4]) {  // L2 only (data written in this launch)
        const float4 t = __ldcg(reinterpret_cast<const float4 *>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    __device__ static float get(const float *p) { return *p; }
    __device__ static void put(float *p, float v) { *p = v; }
};

template <> struct Store<double> {
    using R = double;
    static constexpr int W = 2;
    __device__ static void load(const double *p, double (&v)[2]) {
        const double2 t = __ldcs(reinterpret_cast<const double2 *>(p));
        v[0] = t.x; v[1] = t.y;
    }
    __device__ static void store(double *p, const double (&v)[2]) {
        __stcs(reinterpret_cast<double2 *>(p), make_double2(v[0], v[1]));
    }
    __device__ static void store_keep(double *p, const double (&v)[2]) {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    }
    __device__ static void load_cg(const double *p, double (&v)[2]) {
        const double2 t = __ldcg(reinterpret_cast<const double2 *>(p));
        v[0] = t.x; v[1] = t.y;
    }
    __device__ static double get(const double *p) { return *p; }
    __device__ static void put(double *p, double v) { *p = v; }
};

template <> struct Store<__half> {
    using R = float;
    static constexpr int W = 8;
    __device__ static void load(const __half *p, float (&v)[8]) {
        const uint4 t = __ldcs(reinterpret_cast<const uint4 *>(p));
        const unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __half2 h;
            memcpy(&h, &w[i], 4);
            const float2 f = __half22float2(h);
            v[2 * i] = f.x;
            v[2 * i + 1] = f.y;
        }
    }
    __device__ static void store(__half *p, const float (&v)[8]) {
        unsigned w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __half2 h = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
            memcpy(&w[i], &h, 4);
        }
        __stcs(reinterpret_cast<uint4 *>(p), make_uint4(w[0], w[1], w[2], w[3]));
    }
    __device__ static void store_keep(__half *p, const float (&v)[8]) {
        unsigned w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __half2 h = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
            memcpy(&w[i], &h, 4);
        }
        *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    __device__ static void load_cg(const __half *p, float (&v)[8]) {
        const uint4 t = __ldcg(reinterpret_cast<const uint4 *>(p));
        const unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __half2 h;
            memcpy(&h, &w[i], 4);
            const float2 f = __half22float2(h);
            v[2 * i] = f.x;
            v[2 * i + 1] = f.y;
        }
    }
    __device__ static float get(const __half *p) { return __half2float(*p); }
    __device__ static void put(__half *p, float v) { *p = __float2half_rn(v); }
};

// Correctly rounded arithmetic that the compiler never fuses into FMAs: every
// kernel that applies the collision or adds the sampling sums gets the same
// bits, whatever code surrounds it (one-step, two-step and recomputed paths).
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// tau = 1/2 collision of one cell (Eq. 71 with the moments of Eq. 62): with
// f^eq_0 = rho1 (1 - D c^2) and f^eq_{+-a} = (c^2 rho1 +- J_a) / 2, f* = 2 f^eq - f
// gives f*_0 = 2 (rho1 - D c^2 rho1) - f_0 and f*_{+-a} = c^2 rho1 - f_{-+a}.
// f: the pulled populations in velocity order (0, +x, -x, +y, -y, +z, -z).
template <typename R, int D>
__device__ __forceinline__ void collide_half(R c2, const R (&f)[2 * D + 1], R (&o)[2 * D + 1]) {
    R rho = add_rn(add_rn(add_rn(add_rn(f[0], f[1]), f[2]), f[3]), f[4]);
    if constexpr (D == 3) rho = add_rn(rho, add_rn(f[5], f[6]));
    const R eq = mul_rn(c2, rho);
    o[0] = sub_rn(mul_rn(R(2), sub_rn(rho, mul_rn(R(D), eq))), f[0]);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        o[1 + 2 * a] = sub_rn(eq, f[2 + 2 * a]);
        o[2 + 2 * a] = sub_rn(eq, f[1 + 2 * a]);
    }
}

template <int W>
__device__ __forceinline__ unsigned long long load_classes(const uint8_t *p) {
    if constexpr (W == 8) return *reinterpret_cast<const unsigned long long *>(p);
    else if constexpr (W == 4) return *reinterpret_cast<const uint32_t *>(p);
    else return *reinterpret_cast<const uint16_t *>(p);
}

// rho1 and J1 at cell (x, y, z) at the current time (in stored units): the
// pull-sum of the stored post-collision populations (Eq. 62 applied after the
// advection of Eq. 64).
template <typename S>
__device__ __forceinline__ void pulled_moments(const Geometry &g, const S *__restrict__ src, int x, int y,
                                               int z, typename Store<S>::R &rho,
                                               typename Store<S>::R (&J)[3]) {
    using R = typename Store<S>::R;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long long nc = g.ncell;
    const long long id = ((long long)z * ny + y) * nx + x;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const R f0 = Store<S>::get(src + id);
    const R fpx = Store<S>::get(src + nc + id - x + xm);
    const R fmx = Store<S>::get(src + 2 * nc + id - x + xp);
    const R fpy = Store<S>::get(src + 3 * nc + ((long long)z * ny + ym) * nx + x);
    const R fmy = Store<S>::get(src + 4 * nc + ((long long)z * ny + yp) * nx + x);
    rho = f0 + fpx + fmx + fpy + fmy;
    J[0] = fpx - fmx;
    J[1] = fpy - fmy;
    J[2] = R(0);
    if (g.dim == 3) {
        const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
        const R fpz = Store<S>::get(src + 5 * nc + ((long long)zm * ny + y) * nx + x);
        const R fmz = Store<S>::get(src + 6 * nc + ((long long)zp * ny + y) * nx + x);
        rho += fpz + fmz;
        J[2] = fpz - fmz;
    }
}

// Surface sampling.  One warp per surface element; lane l < 3^dim handles
// stencil cell l.  P = sum_l delta_l c_l^2 rho1_l and U = sum_l delta_l J1_l /
// rho0 (Eqs. 80-81), then acc += (P^2, U.U, U_x (U.n), U_y (U.n), U_z (U.n))
// in stored units.  `moments(x, y, z, rho, J)` gives rho1 and J1 of a cell at
// the sampled time.
template <typename S>
struct SampleArgs {
    Geometry g;
    const int4 *st_xyz;
    const typename Store<S>::R *st_w, *nrm;
    typename Store<S>::R *acc;
};

template <typename S>
inline SampleArgs<S> sample_args(const Geometry &g, const Buffers &b) {
    using R = typename Store<S>::R;
    SampleArgs<S> a;
    a.g = g;
    a.st_xyz = b.st_xyz;
    a.st_w = (const R *)b.st_w;
    a.nrm = (const R *)b.nrm;
    a.acc = (R *)b.acc;
    return a;
}

// End-of-period fold of one running sum into its FP64 total (scale converts
// stored units back), explicit rounding: acc64 + acc * scale as one FMA.
__device__ __forceinline__ double fold_value(double acc64, double acc, double scale) {
    return fma_rn(acc, scale, acc64);
}

// acc += (P^2, U.U, U_x (U.n), U_y (U.n), U_z (U.n)), explicit rounding.
template <typename R>
__device__ __forceinline__ void accumulate_point(R *acc, R p, const R (&u)[3], const R *n) {
    const R un = fma_rn(u[2], n[2], fma_rn(u[1], n[1], mul_rn(u[0], n[0])));
    acc[0] = fma_rn(p, p, acc[0]);
    acc[1] = add_rn(acc[1], fma_rn(u[2], u[2], fma_rn(u[1], u[1], mul_rn(u[0], u[0]))));
    acc[2] = fma_rn(u[0], un, acc[2]);
    acc[3] = fma_rn(u[1], un, acc[3]);
    acc[4] = fma_rn(u[2], un, acc[4]);
}

template <typename R, typename M>
__device__ __forceinline__ void sample_point_with(const Geometry &g, const int4 *__restrict__ st_xyz,
                                                  const R *__restrict__ st_w, const R *__restrict__ nrm, R *acc, int k,
                                                  int lane, M moments) {
    R p = R(0), u[3] = {R(0), R(0), R(0)};
    if (lane < g.stencil) {
        const long long o = (long long)k * g.stencil + lane;
        const int4 c = st_xyz[o];
        R rho, J[3];
        moments(c.x, c.y, c.z, rho, J);
        const R wp = st_w[2 * o], wu = st_w[2 * o + 1];
        p = mul_rn(wp, rho);
        u[0] = mul_rn(wu, J[0]);
        u[1] = mul_rn(wu, J[1]);
        u[2] = mul_rn(wu, J[2]);
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        p = add_rn(p, __shfl_xor_sync(kFull, p, m));
        u[0] = add_rn(u[0], __shfl_xor_sync(kFull, u[0], m));
        u[1] = add_rn(u[1], __shfl_xor_sync(kFull, u[1], m));
        u[2] = add_rn(u[2], __shfl_xor_sync(kFull, u[2], m));
    }
    if (lane == 0) accumulate_point(acc + 5 * (long long)k, p, u, nrm + 4 * (long long)k);
}

// The same for a 2D point (3 x 3 stencil) by one thread: the nine terms are
// summed in the order the xor-butterfly above sums lanes 0..8 (the other
// lanes add exact zeros): [((v0 + v8) + v4) + (v2 + v6)] + [(v1 + v5) + (v3 + v7)],
// so both forms give the same bits.
template <typename R, typename M>
__device__ __forceinline__ void sample_point_2d_thread(const Geometry &g, const int4 *__restrict__ st_xyz,
                                                       const R *__restrict__ st_w, const R *__restrict__ nrm, R *acc,
                                                       int k, M moments) {
    struct T {
        R p, u[3];
    };
    auto term = [&](int l) {  // stencil cell l: (delta c^2 rho1, delta J1 / rho0)
        const long long o = (long long)k * 9 + l;
        const int4 c = st_xyz[o];
        R rho, J[3];
        moments(c.x, c.y, c.z, rho, J);
        const R wp = st_w[2 * o], wu = st_w[2 * o + 1];
        T v;
        v.p = mul_rn(wp, rho);
#pragma unroll
        for (int a = 0; a < 3; ++a) v.u[a] = mul_rn(wu, J[a]);
        return v;
    };
    auto add = [](const T &x, const T &y) {
        T v;
        v.p = add_rn(x.p, y.p);
#pragma unroll
        for (int a = 0; a < 3; ++a) v.u[a] = add_rn(x.u[a], y.u[a]);
        return v;
    };
    // evaluated in tree order, so that few partial sums are live at a time
    T s = add(term(0), term(8));
    s = add(s, term(4));
    s = add(s, add(term(2), term(6)));
    T r = add(term(1), term(5));
    r = add(r, add(term(3), term(7)));
    s = add(s, r);
    accumulate_point(acc + 5 * (long long)k, s.p, s.u, nrm + 4 * (long long)k);
}

template <typename S, typename M>
__device__ __forceinline__ void sample_point_with(const SampleArgs<S> &a, int k, int lane, M moments) {
    sample_point_with(a.g, a.st_xyz, a.st_w, a.nrm, a.acc, k, lane, moments);
}

// Driven-cavity parameters of one step (Sec. VII).
template <typename R>
struct Drive {
    R rho_src;  // imposed rho1 on the source sheet at this step
    R phi;      // wall damping
    int axis;   // wave axis
};

// Wall and source cells (classes >= CELL_WALL_LO) replace the collision:
//   walls, Eq. (73): f*_i = Phi f_j, v_j = -v_i; the outward value is dropped;
//   source, Eq. (72): f* = f^eq(rho_src, J1), J1 from the arrived populations.
// fin / fout in velocity order (0, +x, -x, +y, -y, +z, -z).
template <typename R, int Q>
__device__ __forceinline__ void boundary_cell(unsigned k, const R (&fin)[Q], R c2, const Drive<R> &d,
                                              R (&fout)[Q]) {
    constexpr int D = (Q - 1) / 2;
    if (k == CELL_SOURCE) {
        const R eq = c2 * d.rho_src;
        fout[0] = d.rho_src * (R(1) - R(D) * c2);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const R J = fin[1 + 2 * a] - fin[2 + 2 * a];
            fout[1 + 2 * a] = R(0.5) * (eq + J);
            fout[2 + 2 * a] = R(0.5) * (eq - J);
        }
    } else {
        const int out = k == CELL_WALL_LO ? 2 + 2 * d.axis : 1 + 2 * d.axis;
        fout[0] = d.phi * fin[0];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            fout[1 + 2 * a] = 1 + 2 * a == out ? R(0) : d.phi * fin[2 + 2 * a];
            fout[2 + 2 * a] = 2 + 2 * a == out ? R(0) : d.phi * fin[1 + 2 * a];
        }
    }
}

}  // namespace wlb
