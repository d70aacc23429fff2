// Per-step kernels of the wave lattice Boltzmann force computation.
//
//   update   fused advection + BGK collision with tau = 1/2 (Sec. V, Eqs. 62-64,
//            71), pull form: the populations that reach cell x are read from
//            x - v_i and the post-collision values are written at x.
//   sample   kernel interpolation of p1 and u1 onto the surface elements
//            (Sec. VI, Eqs. 80-82) and running sums of p1^2, u1.u1, (n.u1) u1.
//   fold     once per period: running sums -> FP64 totals.
//   force    King's surface integral, Eq. (14), in FP64.
//   fields   p1 = c^2 rho1 and u1 = J1 / rho0 (Eq. 62) for read-back.
//
// With tau = 1/2 the collision f* = 2 f^eq - f becomes, with the equilibrium of
// Eq. (71) (w_i / c_s^2 = 1/2 for both D2Q5 and D3Q7),
//     f*_0  = 2 rho1 (1 - D c^2) - f_0,
//     f*_+a = c^2 rho1 + J_a - f_+a = c^2 rho1 - f_-a,
//     f*_-a = c^2 rho1 - J_a - f_-a = c^2 rho1 - f_+a.
// The update is linear in f, so populations may be stored scaled (FP16 stores
// f / p_a); the scale only enters the setup, the fold and the read-back.
#include <cmath>

#include "wlb_kernels.cuh"

namespace wlb {
namespace {

template <typename S>
__device__ __forceinline__ void sample_point(const SampleArgs<S> &a, const S *__restrict__ src, int k, int lane) {
    sample_point_with(a, k, lane, [&](int x, int y, int z, typename Store<S>::R &rho, typename Store<S>::R(&J)[3]) {
        pulled_moments(a.g, src, x, y, z, rho, J);
    });
}

template <typename S>
__global__ void __launch_bounds__(256) sample_points(SampleArgs<S> a, const S *__restrict__ src) {
    const int lane = threadIdx.x & 31;
    const int k = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (k >= a.g.n_surface) return;  // uniform per warp
    sample_point(a, src, k, lane);
}

// Row-vectorised update.  One warp owns one lattice row (fixed y, z) of
// nx = 32 * W * CH cells; lane L holds cells (c*32 + L)*W .. +W-1 of chunk c.
// Every population row is read with aligned 16-byte loads: the +-y and +-z
// neighbours are whole rows, and the +-x shift (including the periodic wrap at
// the row ends) is done with warp shuffles, so no element is loaded twice.
//
// Blocks at or beyond row_blocks sample the surface instead (one warp per
// point): they read the same input buffer and write only the running sums, so
// the sampled step is one launch.  Launched with programmatic dependent
// launch: every block lets the next launch start, then waits for the previous
// one to finish before reading.
template <typename S, int D, int CH, bool DRIVEN>
__global__ void __launch_bounds__(256) update_rows(const S *__restrict__ src, S *__restrict__ dst,
                                                   const uint8_t *__restrict__ cls,
                                                   const typename Store<S>::R *__restrict__ c2f, int nx,
                                                   int ny, int nz, long long ncell,
                                                   typename Store<S>::R c0sq, typename Store<S>::R cpsq,
                                                   long long row_blocks, SampleArgs<S> sa,
                                                   Drive<typename Store<S>::R> drv) {
    using R = typename Store<S>::R;
    constexpr int W = Store<S>::W;
    constexpr int Q = 2 * D + 1;
    asm volatile("griddepcontrol.launch_dependents;");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int lane = threadIdx.x & 31;
    if ((long long)blockIdx.x >= row_blocks) {
        const int k = (int)((((long long)blockIdx.x - row_blocks) * blockDim.x + threadIdx.x) >> 5);
        if (k < sa.g.n_surface) sample_point(sa, src, k, lane);
        return;
    }
    const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= (long long)ny * nz) return;  // uniform per warp
    const int y = (int)(row % ny);
    const int z = (int)(row / ny);
    const int ym = y == 0 ? ny - 1 : y - 1;
    const int yp = y == ny - 1 ? 0 : y + 1;
    const long long r0 = row * nx;
    const long long rym = ((long long)z * ny + ym) * nx;
    const long long ryp = ((long long)z * ny + yp) * nx;
    long long rzm = 0, rzp = 0;
    if (D == 3) {
        const int zm = z == 0 ? nz - 1 : z - 1;
        const int zp = z == nz - 1 ? 0 : z + 1;
        rzm = ((long long)zm * ny + y) * nx;
        rzp = ((long long)zp * ny + y) * nx;
    }

    R f[Q][CH][W];
    unsigned long long cl[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const int x0 = (c * 32 + lane) * W;
        Store<S>::load(src + r0 + x0, f[0][c]);
        Store<S>::load(src + ncell + r0 + x0, f[1][c]);
        Store<S>::load(src + 2 * ncell + r0 + x0, f[2][c]);
        Store<S>::load(src + 3 * ncell + rym + x0, f[3][c]);
        Store<S>::load(src + 4 * ncell + ryp + x0, f[4][c]);
        if (D == 3) {
            Store<S>::load(src + 5 * ncell + rzm + x0, f[5][c]);
            Store<S>::load(src + 6 * ncell + rzp + x0, f[6][c]);
        }
        cl[c] = load_classes<W>(cls + r0 + x0);
    }

    // The +x population arriving at x left x-1; the -x one left x+1.
    R up[CH], dn[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        up[c] = __shfl_sync(kFull, f[1][c][W - 1], (lane + 31) & 31);
        dn[c] = __shfl_sync(kFull, f[2][c][0], (lane + 1) & 31);
    }

#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const int x0 = (c * 32 + lane) * W;
        R fpx[W], fmx[W];
        fpx[0] = lane == 0 ? up[(c + CH - 1) % CH] : up[c];
#pragma unroll
        for (int e = 1; e < W; ++e) fpx[e] = f[1][c][e - 1];
#pragma unroll
        for (int e = 0; e < W - 1; ++e) fmx[e] = f[2][c][e + 1];
        fmx[W - 1] = lane == 31 ? dn[(c + 1) % CH] : dn[c];

        R o[Q][W];
#pragma unroll
        for (int e = 0; e < W; ++e) {
            const unsigned k = (unsigned)(cl[c] >> (8 * e)) & 0xffu;
            const R c2 = k == CELL_FLUID ? c0sq : (k == CELL_OBJECT ? cpsq : c2f[r0 + x0 + e]);
            R fin[Q], fo[Q];
            fin[0] = f[0][c][e];
            fin[1] = fpx[e];
            fin[2] = fmx[e];
#pragma unroll
            for (int i = 3; i < Q; ++i) fin[i] = f[i][c][e];
            collide_half<R, D>(c2, fin, fo);
            if (DRIVEN && k >= CELL_WALL_LO) boundary_cell<R, Q>(k, fin, c2, drv, fo);  // driven cavity only
#pragma unroll
            for (int i = 0; i < Q; ++i) o[i][e] = fo[i];
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) Store<S>::store(dst + i * ncell + r0 + x0, o[i]);
    }
}

// Any lattice shape: one thread per cell, scalar accesses.
template <typename S, int D, bool DRIVEN>
__global__ void __launch_bounds__(256) update_cells(const S *__restrict__ src, S *__restrict__ dst,
                                                    const uint8_t *__restrict__ cls,
                                                    const typename Store<S>::R *__restrict__ c2f, int nx,
                                                    int ny, int nz, long long ncell,
                                                    typename Store<S>::R c0sq, typename Store<S>::R cpsq,
                                                    Drive<typename Store<S>::R> drv) {
    using R = typename Store<S>::R;
    constexpr int Q = 2 * D + 1;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= ncell) return;
    const int x = (int)(id % nx);
    const long long r = id / nx;
    const int y = (int)(r % ny);
    const int z = (int)(r / ny);
    const long long row = id - x;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const R f0 = Store<S>::get(src + id);
    const R fpx = Store<S>::get(src + ncell + row + xm);
    const R fmx = Store<S>::get(src + 2 * ncell + row + xp);
    const R fpy = Store<S>::get(src + 3 * ncell + ((long long)z * ny + ym) * nx + x);
    const R fmy = Store<S>::get(src + 4 * ncell + ((long long)z * ny + yp) * nx + x);
    R fpz = 0, fmz = 0;
    if (D == 3) {
        const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
        fpz = Store<S>::get(src + 5 * ncell + ((long long)zm * ny + y) * nx + x);
        fmz = Store<S>::get(src + 6 * ncell + ((long long)zp * ny + y) * nx + x);
    }
    const uint8_t k = cls[id];
    const R c2 = k == CELL_FLUID ? c0sq : (k == CELL_OBJECT ? cpsq : c2f[id]);
    const R all[7] = {f0, fpx, fmx, fpy, fmy, fpz, fmz};
    R fin[Q], o[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fin[i] = all[i];
    collide_half<R, D>(c2, fin, o);
    if (DRIVEN && k >= CELL_WALL_LO) boundary_cell<R, Q>(k, fin, c2, drv, o);  // driven cavity only
#pragma unroll
    for (int i = 0; i < Q; ++i) Store<S>::put(dst + i * ncell + id, o[i]);
}

// acc64 += acc * scale (scale = 1 / pop_scale^2 converts stored units back).
template <typename R>
__global__ void fold_sums(int n, R *__restrict__ acc, double *__restrict__ acc64, double scale,
                          int *__restrict__ err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = fold_value(acc64[i], (double)acc[i], scale);
    acc64[i] = v;
    acc[i] = R(0);
    if (!isfinite(v)) atomicExch(err, 1);
}

// Eq. (14) on the surface elements; one block, fixed reduction order.
__global__ void __launch_bounds__(256) surface_force(Geometry g, const double *__restrict__ pts,
                                                     const double *__restrict__ acc64, double inv_nw,
                                                     double *__restrict__ force, int *__restrict__ err) {
    __shared__ double red[3][256];
    const int t = threadIdx.x;
    double F[3] = {0.0, 0.0, 0.0};
    const double rho0 = g.rho0;
    const double inv_2rc2 = 1.0 / (2.0 * rho0 * g.c0 * g.c0);
    for (int k = t; k < g.n_surface; k += blockDim.x) {
        const double *row = pts + 7 * (long long)k;
        const double *a = acc64 + 5 * (long long)k;
        const double iso = a[0] * inv_nw * inv_2rc2 - 0.5 * rho0 * (a[1] * inv_nw);
        for (int i = 0; i < 3; ++i) F[i] -= row[6] * (iso * row[3 + i] + rho0 * (a[2 + i] * inv_nw));
    }
    for (int i = 0; i < 3; ++i) red[i][t] = F[i];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s)
            for (int i = 0; i < 3; ++i) red[i][t] += red[i][t + s];
        __syncthreads();
    }
    if (t == 0) {
        for (int i = 0; i < 3; ++i) {
            const double v = i < g.dim ? red[i][0] : 0.0;
            force[i] = v;
            if (!isfinite(v)) atomicExch(err, 1);
        }
        force[3] = 0.0;
    }
}

template <typename S>
__global__ void read_fields(Geometry g, const S *__restrict__ src, const uint8_t *__restrict__ cls,
                            const typename Store<S>::R *__restrict__ c2f, long long first, long long count,
                            double *__restrict__ stage) {
    using R = typename Store<S>::R;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    const long long id = first + j;
    const int x = (int)(id % g.n[0]);
    const long long r = id / g.n[0];
    const int y = (int)(r % g.n[1]);
    const int z = (int)(r / g.n[1]);
    R rho, J[3];
    pulled_moments(g, src, x, y, z, rho, J);
    const uint8_t k = cls[id];
    const double c2 = k == CELL_FLUID ? (double)(R)(g.c0 * g.c0)
                                      : (k == CELL_OBJECT ? (double)(R)(g.cp * g.cp) : (double)c2f[id]);
    const double unscale = 1.0 / g.pop_scale;
    stage[j] = c2 * (double)rho * unscale;
    for (int a = 0; a < g.dim; ++a) stage[(long long)(1 + a) * count + j] = (double)J[a] * unscale / g.rho0;
}


// Update launch (rows, plus sampling blocks when sample is set) with the
// programmatic-serialization attribute.
template <typename R>
Drive<R> drive_of(const Geometry &g, long long t_mod) {
    Drive<R> d;
    const double two_pi = 6.283185307179586476925286766559;
    d.rho_src = (R)(g.driven ? g.source_amplitude * std::sin(two_pi * (double)t_mod / (double)g.period) * g.pop_scale
                             : 0.0);
    d.phi = (R)g.wall_damping;
    d.axis = g.wave_axis;
    return d;
}

template <typename S, int D, int CH>
cudaError_t run_rows(const Geometry &g, const Buffers &b, int src, bool sample, long long t_mod, cudaStream_t s) {
    using R = typename Store<S>::R;
    const long long rows = (long long)g.n[1] * g.n[2];
    const long long row_blocks = (rows * 32 + 255) / 256;
    const long long sample_blocks = sample && g.n_surface > 0 ? (g.n_surface + 7) / 8 : 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(row_blocks + sample_blocks));
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    auto kern = g.driven ? update_rows<S, D, CH, true> : update_rows<S, D, CH, false>;
    return cudaLaunchKernelEx(&cfg, kern, (const S *)b.pop[src], (S *)b.pop[src ^ 1],
                              (const uint8_t *)b.cls, (const R *)b.c2, g.n[0], g.n[1], g.n[2], g.ncell,
                              (R)(g.c0 * g.c0), (R)(g.cp * g.cp), row_blocks, sample_args<S>(g, b),
                              drive_of<R>(g, t_mod));
}

template <typename S>
int row_chunks(const Geometry &g) {
    constexpr int W = Store<S>::W;
    if (g.n[0] % (32 * W) != 0) return 0;
    const int ch = g.n[0] / (32 * W);
    return ch <= 4 ? ch : 0;
}

template <typename S, int D>
cudaError_t run_update(const Geometry &g, const Buffers &b, int src, bool sample, long long t_mod, cudaStream_t s,
                       bool *vec) {
    using R = typename Store<S>::R;
    const int ch = row_chunks<S>(g);
    *vec = ch > 0;
    switch (ch) {
        case 1: return run_rows<S, D, 1>(g, b, src, sample, t_mod, s);
        case 2: return run_rows<S, D, 2>(g, b, src, sample, t_mod, s);
        case 3: return run_rows<S, D, 3>(g, b, src, sample, t_mod, s);
        case 4: return run_rows<S, D, 4>(g, b, src, sample, t_mod, s);
        default: break;
    }
    const long long blocks = (g.ncell + 255) / 256;
    auto kern = g.driven ? update_cells<S, D, true> : update_cells<S, D, false>;
    kern<<<(unsigned)blocks, 256, 0, s>>>(
        (const S *)b.pop[src], (S *)b.pop[src ^ 1], b.cls, (const R *)b.c2, g.n[0], g.n[1], g.n[2],
        g.ncell, (R)(g.c0 * g.c0), (R)(g.cp * g.cp), drive_of<R>(g, t_mod));
    return cudaGetLastError();
}

template <typename S>
cudaError_t update_for(const Geometry &g, const Buffers &b, int src, bool sample, long long t_mod, cudaStream_t s,
                       bool *vec) {
    return g.dim == 3 ? run_update<S, 3>(g, b, src, sample, t_mod, s, vec)
                      : run_update<S, 2>(g, b, src, sample, t_mod, s, vec);
}

template <typename S>
cudaError_t sample_for(const Geometry &g, const Buffers &b, int src, cudaStream_t s) {
    const unsigned blocks = (unsigned)((g.n_surface + 7) / 8);
    sample_points<S><<<blocks, 256, 0, s>>>(sample_args<S>(g, b), (const S *)b.pop[src]);
    return cudaGetLastError();
}

template <typename S>
cudaError_t fields_for(const Geometry &g, const Buffers &b, int src, long long first, long long count,
                       cudaStream_t s) {
    using R = typename Store<S>::R;
    const unsigned blocks = (unsigned)((count + 255) / 256);
    read_fields<S><<<blocks, 256, 0, s>>>(g, (const S *)b.pop[src], b.cls, (const R *)b.c2, first, count,
                                          b.stage);
    return cudaGetLastError();
}

}  // namespace

bool update_is_vectorised(const Geometry &g, Prec p) {
    switch (p) {
        case Prec::F64: return row_chunks<double>(g) > 0;
        case Prec::F16: return row_chunks<__half>(g) > 0;
        default: return row_chunks<float>(g) > 0;
    }
}

cudaError_t launch_update(const Geometry &g, const Buffers &b, Prec p, int src, long long t_mod, cudaStream_t s,
                          bool *vector_path) {
    bool vec = false;
    cudaError_t e;
    switch (p) {
        case Prec::F64: e = update_for<double>(g, b, src, false, t_mod, s, &vec); break;
        case Prec::F16: e = update_for<__half>(g, b, src, false, t_mod, s, &vec); break;
        default: e = update_for<float>(g, b, src, false, t_mod, s, &vec); break;
    }
    if (vector_path) *vector_path = vec;
    return e;
}

cudaError_t launch_step(const Geometry &g, const Buffers &b, Prec p, int src, bool sample, long long t_mod,
                        cudaStream_t s) {
    if (!sample || g.n_surface == 0 || !update_is_vectorised(g, p)) {
        cudaError_t e = sample && g.n_surface > 0 ? launch_sample(g, b, p, src, s) : cudaSuccess;
        return e == cudaSuccess ? launch_update(g, b, p, src, t_mod, s, nullptr) : e;
    }
    bool vec = false;
    switch (p) {
        case Prec::F64: return update_for<double>(g, b, src, true, t_mod, s, &vec);
        case Prec::F16: return update_for<__half>(g, b, src, true, t_mod, s, &vec);
        default: return update_for<float>(g, b, src, true, t_mod, s, &vec);
    }
}

cudaError_t launch_sample(const Geometry &g, const Buffers &b, Prec p, int src, cudaStream_t s) {
    if (g.n_surface == 0) return cudaSuccess;
    switch (p) {
        case Prec::F64: return sample_for<double>(g, b, src, s);
        case Prec::F16: return sample_for<__half>(g, b, src, s);
        default: return sample_for<float>(g, b, src, s);
    }
}

cudaError_t launch_fold(const Geometry &g, const Buffers &b, Prec p, cudaStream_t s) {
    if (g.n_surface == 0) return cudaSuccess;
    const int n = 5 * g.n_surface;
    const double scale = 1.0 / (g.pop_scale * g.pop_scale);
    if (p == Prec::F64)
        fold_sums<double><<<(n + 255) / 256, 256, 0, s>>>(n, (double *)b.acc, b.acc64, scale, b.err);
    else
        fold_sums<float><<<(n + 255) / 256, 256, 0, s>>>(n, (float *)b.acc, b.acc64, scale, b.err);
    return cudaGetLastError();
}

cudaError_t launch_force(const Geometry &g, const Buffers &b, double n_window, cudaStream_t s) {
    surface_force<<<1, 256, 0, s>>>(g, b.pts, b.acc64, 1.0 / n_window, b.force, b.err);
    return cudaGetLastError();
}

cudaError_t launch_fields(const Geometry &g, const Buffers &b, Prec p, int src, long long first,
                          long long count, cudaStream_t s) {
    switch (p) {
        case Prec::F64: return fields_for<double>(g, b, src, first, count, s);
        case Prec::F16: return fields_for<__half>(g, b, src, first, count, s);
        default: return fields_for<float>(g, b, src, first, count, s);
    }
}

}  // namespace wlb
