// Batched ensembles: many independent lattices of uneven size stepped together.
//
// Each lattice runs the same protocol as a single handle (setup, unsampled and
// sampled periods, FP64 force; Secs. V-VII, Eqs. 14, 62-64, 71-72, 79-82), but
// one launch of `batch_update` advances every row of every active lattice, and
// one launch of `batch_sample` samples every surface point of every lattice in
// its averaging window.  The step index lives in device memory and is advanced
// by the last block of each update launch, so a chunk of steps is one CUDA
// graph replayed without host work.  Lattices with fewer steps than the longest
// one stop at their own n_steps (their rows are skipped).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "wlb_handle.cuh"
#include "wlb_kernels.cuh"

namespace wlb {
namespace {

// What the update of one row needs, in 64 bytes.
struct __align__(16) LatHot {
    const void *pop0, *pop1;
    const uint8_t *cls;
    const void *c2;
    long long ncell, n_steps;
    double c0sq, cpsq;
    int nx, ny, nz, pad;
};

constexpr int kMaxChunks = 4;    // rows up to 32 * W * 4 cells
constexpr int kGraphSteps = 64;  // steps per captured graph

// One warp updates one row of nx = nv * W cells, nv <= 32 * CH (lanes past the
// row end idle).  The +-x neighbours and the periodic wrap come from shuffles.
template <typename S, int D, int CH>
__device__ __forceinline__ void update_row(const S *__restrict__ src, S *__restrict__ dst,
                                           const uint8_t *__restrict__ cls,
                                           const typename Store<S>::R *__restrict__ c2f, int nx, int ny,
                                           int nz, long long ncell, int y, int z, typename Store<S>::R c0sq,
                                           typename Store<S>::R cpsq, int lane) {
    using R = typename Store<S>::R;
    constexpr int W = Store<S>::W;
    constexpr int Q = 2 * D + 1;
    const int nv = nx / W;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const long long r0 = ((long long)z * ny + y) * nx;
    const long long rym = ((long long)z * ny + ym) * nx, ryp = ((long long)z * ny + yp) * nx;
    long long rzm = 0, rzp = 0;
    if (D == 3) {
        const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
        rzm = ((long long)zm * ny + y) * nx;
        rzp = ((long long)zp * ny + y) * nx;
    }
    R f[Q][CH][W];
    unsigned long long cl[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const int v = c * 32 + lane;
        if (v < nv) {
            const int x0 = v * W;
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
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i)
#pragma unroll
                for (int e = 0; e < W; ++e) f[i][c][e] = R(0);
            cl[c] = 0;
        }
    }
    R up[CH], dn[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        up[c] = __shfl_sync(kFull, f[1][c][W - 1], (lane + 31) & 31);
        dn[c] = __shfl_sync(kFull, f[2][c][0], (lane + 1) & 31);
    }
    // wrap: +x at x = 0 comes from x = nx - 1, -x at x = nx - 1 from x = 0
    const int last_chunk = (nv - 1) >> 5, last_lane = (nv - 1) & 31;
    R lastv = f[1][0][W - 1];
#pragma unroll
    for (int c = 1; c < CH; ++c)
        if (c == last_chunk) lastv = f[1][c][W - 1];
    const R wrap_left = __shfl_sync(kFull, lastv, last_lane);
    const R wrap_right = __shfl_sync(kFull, f[2][0][0], 0);
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const int v = c * 32 + lane;
        if (v >= nv) continue;
        const int x0 = v * W;
        R fpx[W], fmx[W];
        fpx[0] = v == 0 ? wrap_left : (lane == 0 ? up[(c + CH - 1) % CH] : up[c]);
#pragma unroll
        for (int e = 1; e < W; ++e) fpx[e] = f[1][c][e - 1];
#pragma unroll
        for (int e = 0; e < W - 1; ++e) fmx[e] = f[2][c][e + 1];
        fmx[W - 1] = v == nv - 1 ? wrap_right : (lane == 31 ? dn[(c + 1) % CH] : dn[c]);
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
#pragma unroll
            for (int i = 0; i < Q; ++i) o[i][e] = fo[i];
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) Store<S>::store(dst + i * ncell + r0 + x0, o[i]);
    }
}

// Grid-stride over the rows of the lattices of one row-chunk class; row_lat
// maps a row to its lattice and row_begin gives the lattice's first row.  The
// last block of the launch that advances the step moves the counter on.
template <typename S, int D, int CH>
__global__ void __launch_bounds__(256) batch_update(const LatHot *__restrict__ lats,
                                                    const int *__restrict__ row_lat,
                                                    const long long *__restrict__ row_begin,
                                                    long long total_rows, long long *step, unsigned *done,
                                                    int advance) {
    using R = typename Store<S>::R;
    const long long t = *step;
    const int lane = threadIdx.x & 31;
    const int s = (int)(t & 1);
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < total_rows;
         row += warps) {
        const int i = row_lat[row];
        const LatHot L = lats[i];
        if (t >= L.n_steps) continue;  // uniform per warp
        const long long local = row - row_begin[i];
        const int y = (int)(local % L.ny), z = (int)(local / L.ny);
        update_row<S, D, CH>((const S *)(s ? L.pop1 : L.pop0), (S *)(s ? L.pop0 : L.pop1), L.cls,
                             (const R *)L.c2, L.nx, L.ny, L.nz, L.ncell, y, z, (R)L.c0sq, (R)L.cpsq, lane);
    }
    if (!advance) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned ticket = atomicAdd(done, 1u);
        if (ticket == gridDim.x - 1) {
            *done = 0;
            *step = t + 1;
            __threadfence();
        }
    }
}

// Grid-stride over all surface points; warps of lattices outside their
// averaging window skip.  The per-period FP32 -> FP64 fold is done here by the
// point's own lane 0 at the last step of each period.
template <typename S>
__global__ void __launch_bounds__(256) batch_sample(const BatchLat *__restrict__ lats,
                                                    const int *__restrict__ pt_lat,
                                                    const long long *__restrict__ pt_begin,
                                                    long long total_points, const long long *step) {
    using R = typename Store<S>::R;
    const long long t = *step;
    const int lane = threadIdx.x & 31;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long p = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < total_points; p += warps) {
        const int i = pt_lat[p];
        const BatchLat &L = lats[i];
        if (t < L.window_begin || t >= L.n_steps) continue;  // uniform per warp
        const int k = (int)(p - pt_begin[i]);
        const S *src = (const S *)L.b.pop[t & 1];
        R *acc = (R *)L.b.acc;
        sample_point_with(L.g, L.b.st_xyz, (const R *)L.b.st_w, (const R *)L.b.nrm, acc, k, lane,
                          [&](int x, int y, int z, R &rho, R(&J)[3]) { pulled_moments(L.g, src, x, y, z, rho, J); });
        if (lane == 0) {
            R *a = acc + 5 * (long long)k;
            if ((t - L.window_begin + 1) % L.period == 0) {
                const double scale = 1.0 / (L.g.pop_scale * L.g.pop_scale);
                double *a64 = L.b.acc64 + 5 * (long long)k;
                bool bad = false;
                for (int j = 0; j < 5; ++j) {
                    const double v = fold_value(a64[j], (double)a[j], scale);
                    a64[j] = v;
                    a[j] = R(0);
                    bad |= !isfinite(v);
                }
                if (bad) atomicExch(L.b.err, 1);
            }
        }
    }
}

// 2D lattices: one thread per point (the 3 x 3 stencil in registers) instead
// of a warp, same sums (sample_point_2d_thread); grid-stride over all points,
// fold at period ends as in batch_sample.
template <typename S>
__global__ void __launch_bounds__(256) batch_sample_2d(const BatchLat *__restrict__ lats,
                                                       const int *__restrict__ pt_lat,
                                                       const long long *__restrict__ pt_begin,
                                                       long long total_points, const long long *step) {
    using R = typename Store<S>::R;
    const long long t = *step;
    const long long threads = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < total_points; p += threads) {
        const int i = pt_lat[p];
        const BatchLat &L = lats[i];
        if (t < L.window_begin || t >= L.n_steps) continue;
        const int k = (int)(p - pt_begin[i]);
        const S *src = (const S *)L.b.pop[t & 1];
        R *a = (R *)L.b.acc;
        sample_point_2d_thread(L.g, L.b.st_xyz, (const R *)L.b.st_w, (const R *)L.b.nrm, a, k,
                               [&](int x, int y, int z, R &rho, R(&J)[3]) {
                                   pulled_moments(L.g, src, x, y, z, rho, J);
                               });
        if ((t - L.window_begin + 1) % L.period == 0) {
            const double scale = 1.0 / (L.g.pop_scale * L.g.pop_scale);
            R *ak = a + 5 * (long long)k;
            double *a64 = L.b.acc64 + 5 * (long long)k;
            bool bad = false;
            for (int j = 0; j < 5; ++j) {
                const double v = fold_value(a64[j], (double)ak[j], scale);
                a64[j] = v;
                ak[j] = R(0);
                bad |= !isfinite(v);
            }
            if (bad) atomicExch(L.b.err, 1);
        }
    }
}

template <typename S, int D>
cudaError_t launch_batch_update(int ch, const LatHot *lats, const int *row_lat, const long long *row_begin,
                                long long rows, long long *step, unsigned *done, int advance, int grid,
                                int threads, cudaStream_t s) {
    switch (ch) {
        case 1: batch_update<S, D, 1><<<grid, threads, 0, s>>>(lats, row_lat, row_begin, rows, step, done, advance); break;
        case 2: batch_update<S, D, 2><<<grid, threads, 0, s>>>(lats, row_lat, row_begin, rows, step, done, advance); break;
        case 3: batch_update<S, D, 3><<<grid, threads, 0, s>>>(lats, row_lat, row_begin, rows, step, done, advance); break;
        default: batch_update<S, D, 4><<<grid, threads, 0, s>>>(lats, row_lat, row_begin, rows, step, done, advance); break;
    }
    return cudaGetLastError();
}

__global__ void batch_advance_step(long long *step) { *step += 2; }

}  // namespace

cudaError_t launch_batch_advance(long long *step, cudaStream_t s) {
    batch_advance_step<<<1, 1, 0, s>>>(step);
    return cudaGetLastError();
}

}  // namespace wlb

using wlb::BatchLat;
using wlb::LatHot;

struct wlb_batch {
    int count = 0;
    wlb::Prec prec = wlb::Prec::F32;
    int dim = 3, chunks = 1, device = 0, n_sm = 1;
    std::vector<wlb_params> p;
    std::vector<BatchLat> lat;
    BatchLat *d_lats = nullptr;
    long long *d_row_begin = nullptr, *d_pt_begin = nullptr, *d_step = nullptr;
    unsigned *d_done = nullptr;
    // update launches, one per row-chunk class (lattices whose rows need the
    // same number of 32-lane chunks), so short rows do not pay for long ones
    int n_classes = 0;
    int class_chunks[wlb::kMaxChunks] = {0};
    int class_count[wlb::kMaxChunks] = {0};
    wlb::LatHot *d_class_lats[wlb::kMaxChunks] = {nullptr};
    long long *d_class_rows[wlb::kMaxChunks] = {nullptr};
    int *d_class_row_lat[wlb::kMaxChunks] = {nullptr};
    int *d_pt_lat = nullptr;  // point -> lattice
    long long class_total_rows[wlb::kMaxChunks] = {0};
    long long total_rows = 0, total_points = 0, max_steps = 0, lattice_updates = 0;
    cudaStream_t stream = nullptr, capture = nullptr;
    wlb::SideStream side;     // 3D two-step groups run side by side on stream (or capture) and side.stream
    void *owned = nullptr;
    double *host_out = nullptr;  // count * 5 doubles (force[4] + flag)
    int threads = 256, blocks_per_sm = 4;
    cudaGraphExec_t graph = nullptr;
    int graph_threads = 0, graph_bps = 0, graph_two = -1;
    // two steps per launch (all lattices 3D periodic FP32/FP16 with even step
    // counts): one launch of the slab kernel over every lattice's CTAs
    bool two_ok = false, two = false;
    int two_threads = 0, total_ctas = 0;  // 2D: total_ctas counts warps (row chunks)
    wlb::BatchTwoGroup groups[2];         // 3D: lane-layout groups, one launch each
    int ngroups = 0;
    int two_ch = 1;                       // 2D: chunks per lane of the widest row
    int two_nx = 0;                       // 2D: widest row (staging slot size)
    int *d_cta_lat = nullptr, *d_cta_first = nullptr;
    wlb::BatchTwoKnobs knobs;             // 3D: the plan's choices (wlb_batch_autotune)
    int plan_gen = 0, graph_plan_gen = -1;  // the captured graph's plan
    char err[512] = {0};
};

namespace {

wlb_status bfail(wlb_batch *b, wlb_status s, const char *what, cudaError_t e = cudaSuccess) {
    if (b) {
        if (e != cudaSuccess)
            snprintf(b->err, sizeof(b->err), "%s: %s", what, cudaGetErrorString(e));
        else
            snprintf(b->err, sizeof(b->err), "%s", what);
    }
    return s;
}

#define BATCH_CUDA(b, call, what)                                           \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return bfail((b), WLB_ERR_CUDA, (what), e_); \
    } while (0)

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

int vec_width(wlb::Prec p) { return p == wlb::Prec::F64 ? 2 : (p == wlb::Prec::F16 ? 8 : 4); }

// Per-lattice layouts, then the batch tables.
size_t batch_layout(const wlb_params *ps, int count, char *base, std::vector<BatchLat> *lat,
                    size_t *tables_off) {
    size_t off = 0;
    for (int i = 0; i < count; ++i) {
        wlb::Geometry g = wlb::make_geometry(&ps[i]);
        wlb::Buffers b{};
        const size_t sz = wlb::layout(g, wlb::prec_of(&ps[i]), base ? base + off : nullptr, &b);
        if (lat) {
            BatchLat L{};
            L.g = g;
            L.b = b;
            lat->push_back(L);
        }
        off += align256(sz);
    }
    *tables_off = off;
    off += align256(sizeof(BatchLat) * count);
    off += 2 * align256(sizeof(long long) * (count + 1));
    off += align256(sizeof(long long)) + align256(sizeof(unsigned));
    long long total_rows = 0;
    for (int i = 0; i < count; ++i) total_rows += (long long)ps[i].ny * ps[i].nz;
    off += wlb::kMaxChunks * (align256(sizeof(LatHot) * count) + align256(sizeof(long long) * (count + 1)));
    off += align256(sizeof(int) * total_rows);  // row -> lattice, all classes back to back
    long long total_points = 0;
    for (int i = 0; i < count; ++i)
        if (ps[i].n_avg_periods > 0) total_points += ps[i].n_surface;
    off += align256(sizeof(int) * (total_points > 0 ? total_points : 1));  // point -> lattice
    // two-step CTA -> lattice (at most one CTA per row) and each lattice's first CTA
    off += align256(sizeof(int) * total_rows) + align256(sizeof(int) * (count + 1));
    return off;
}

wlb_status batch_validate(const wlb_params *ps, int count) {
    if (!ps || count < 1) return WLB_ERR_ARG;
    for (int i = 0; i < count; ++i) {
        if (wlb_validate(&ps[i]) != WLB_OK) return WLB_ERR_ARG;
        if (ps[i].lattice != ps[0].lattice || ps[i].precision != ps[0].precision) return WLB_ERR_ARG;
        if (ps[i].boundary != WLB_BOUNDARY_PERIODIC) return WLB_ERR_ARG;
        const int W = vec_width(wlb::prec_of(&ps[i]));
        if (ps[i].nx % W != 0 || ps[i].nx > 32 * W * wlb::kMaxChunks) return WLB_ERR_ARG;
    }
    return WLB_OK;
}

cudaError_t issue_steps(wlb_batch *b, int nsteps, int threads, int bps, cudaStream_t s) {
    const int grid = b->n_sm * bps;
    if (b->two) {  // step counts are even in this mode
        if (nsteps % 2) return cudaErrorInvalidValue;
        for (int k = 0; k < nsteps; k += 2) {
            cudaError_t e =
                b->dim == 3
                    ? wlb::launch_batch_two_steps(b->prec, b->groups, b->ngroups, b->d_lats, b->d_cta_lat,
                                                  b->d_cta_first, b->d_pt_lat, b->d_pt_begin, b->total_points,
                                                  b->d_step, b->d_done, grid, s, b->side)
                    : wlb::launch_batch2d_two_steps(b->prec, b->two_ch, b->two_nx, b->d_lats, b->d_cta_lat, b->d_cta_first,
                                                    b->total_ctas, b->d_pt_lat, b->d_pt_begin, b->total_points,
                                                    b->d_step, b->d_done, grid, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    for (int k = 0; k < nsteps; ++k) {
        cudaError_t e;
        if (b->total_points > 0 && b->dim == 2) {
            const long long need = (b->total_points + threads - 1) / threads;
            const int g2 = (int)(need < grid ? need : grid);
            switch (b->prec) {
                case wlb::Prec::F64:
                    wlb::batch_sample_2d<double><<<g2, threads, 0, s>>>(b->d_lats, b->d_pt_lat, b->d_pt_begin,
                                                                       b->total_points, b->d_step);
                    break;
                case wlb::Prec::F16:
                    wlb::batch_sample_2d<__half><<<g2, threads, 0, s>>>(b->d_lats, b->d_pt_lat, b->d_pt_begin,
                                                                       b->total_points, b->d_step);
                    break;
                default:
                    wlb::batch_sample_2d<float><<<g2, threads, 0, s>>>(b->d_lats, b->d_pt_lat, b->d_pt_begin,
                                                                      b->total_points, b->d_step);
                    break;
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        } else if (b->total_points > 0) {
            switch (b->prec) {
                case wlb::Prec::F64:
                    wlb::batch_sample<double><<<grid, threads, 0, s>>>(b->d_lats, b->d_pt_lat, b->d_pt_begin,
                                                   b->total_points, b->d_step);
                    break;
                case wlb::Prec::F16:
                    wlb::batch_sample<__half><<<grid, threads, 0, s>>>(b->d_lats, b->d_pt_lat, b->d_pt_begin,
                                                   b->total_points, b->d_step);
                    break;
                default:
                    wlb::batch_sample<float><<<grid, threads, 0, s>>>(b->d_lats, b->d_pt_lat, b->d_pt_begin,
                                                   b->total_points, b->d_step);
                    break;
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        // one launch per row-chunk class; the last one advances the step
        for (int k = 0; k < b->n_classes; ++k) {
            const int ch = b->class_chunks[k], adv = k == b->n_classes - 1;
            const LatHot *L = b->d_class_lats[k];
            const int *n = b->d_class_row_lat[k];
            const long long *R = b->d_class_rows[k];
            const long long rows = b->class_total_rows[k];
            if (b->dim == 3) {
                switch (b->prec) {
                    case wlb::Prec::F64:
                        e = wlb::launch_batch_update<double, 3>(ch, L, n, R, rows, b->d_step, b->d_done, adv, grid, threads, s);
                        break;
                    case wlb::Prec::F16:
                        e = wlb::launch_batch_update<__half, 3>(ch, L, n, R, rows, b->d_step, b->d_done, adv, grid, threads, s);
                        break;
                    default:
                        e = wlb::launch_batch_update<float, 3>(ch, L, n, R, rows, b->d_step, b->d_done, adv, grid, threads, s);
                        break;
                }
            } else {
                switch (b->prec) {
                    case wlb::Prec::F64:
                        e = wlb::launch_batch_update<double, 2>(ch, L, n, R, rows, b->d_step, b->d_done, adv, grid, threads, s);
                        break;
                    case wlb::Prec::F16:
                        e = wlb::launch_batch_update<__half, 2>(ch, L, n, R, rows, b->d_step, b->d_done, adv, grid, threads, s);
                        break;
                    default:
                        e = wlb::launch_batch_update<float, 2>(ch, L, n, R, rows, b->d_step, b->d_done, adv, grid, threads, s);
                        break;
                }
            }
            if (e != cudaSuccess) return e;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Plan two steps per launch for every lattice with the knobs (3D; 2D has
// one plan) and write the CTA (3D) or warp (2D) -> lattice table, each
// lattice's first entry and, with upload_lats, the lattice descriptors that
// carry the plans.  On failure nothing the launches read has changed.
cudaError_t plan_two(wlb_batch *b, const wlb::BatchTwoKnobs &kn, bool upload_lats) {
    const int count = b->count;
    std::vector<BatchLat> lat = b->lat;
    wlb::BatchTwoGroup groups[2];
    int ngroups = 0, tasks2d = 0, two_ch = b->two_ch, two_nx = b->two_nx;
    const bool planned = b->dim == 3 ? wlb::plan_batch_two_steps(b->prec, lat.data(), count, kn, groups, &ngroups)
                                     : wlb::plan_batch2d_two_steps(b->prec, lat.data(), count, kn.rows_2d, &tasks2d,
                                                                   &two_ch, &two_nx);
    if (!planned) return cudaErrorInvalidValue;
    // CTA (3D) or warp (2D) -> lattice table, the lattices of each 3D
    // lane-layout group together; first[i] = lattice i's first entry
    std::vector<int> first(count + 1, 0), owner;
    const int ngr = b->dim == 3 ? ngroups : 1;
    int two_threads = 0;
    for (int k = 0; k < ngr; ++k) {
        const int begin = (int)owner.size();
        for (int i = 0; i < count; ++i) {
            if (b->dim == 3 && lat[i].plan.chunks_per_lane != groups[k].ch) continue;
            const int n = lat[i].plan.nslab * lat[i].plan.chunks;
            first[i] = (int)owner.size();
            owner.insert(owner.end(), (size_t)n, i);
        }
        if (b->dim == 3) {
            groups[k].cta_begin = begin;
            groups[k].ctas = (int)owner.size() - begin;
            two_threads = std::max(two_threads, groups[k].threads);
        }
    }
    if (b->dim == 2) two_threads = lat[0].plan.threads;  // warps of a block
    first[count] = (int)owner.size();
    if ((long long)owner.size() > b->total_rows) return cudaErrorInvalidValue;  // table capacity
    cudaError_t e = cudaMemcpy(b->d_cta_lat, owner.data(), sizeof(int) * owner.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_cta_first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && upload_lats)
        e = cudaMemcpy(b->d_lats, lat.data(), sizeof(BatchLat) * count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    b->lat = lat;
    for (int k = 0; k < 2; ++k) b->groups[k] = groups[k];
    b->ngroups = ngroups;
    b->two_ch = two_ch;
    b->two_nx = two_nx;
    b->two_threads = two_threads;
    b->total_ctas = (int)owner.size();
    b->knobs = kn;
    ++b->plan_gen;
    return cudaSuccess;
}

wlb_status batch_setup(wlb_batch *b) {
    for (int i = 0; i < b->count; ++i)
        BATCH_CUDA(b, wlb::launch_setup(b->lat[i].g, b->lat[i].b, b->prec, b->stream), "setup kernels");
    BATCH_CUDA(b, cudaMemsetAsync(b->d_step, 0, sizeof(long long), b->stream), "reset step");
    BATCH_CUDA(b, cudaMemsetAsync(b->d_done, 0, sizeof(unsigned), b->stream), "reset counter");
    return WLB_OK;
}

}  // namespace

extern "C" {

wlb_status wlb_batch_workspace_bytes(const wlb_params *ps, int count, size_t *bytes) {
    if (!bytes) return WLB_ERR_ARG;
    wlb_status s = batch_validate(ps, count);
    if (s != WLB_OK) return s;
    size_t toff;
    *bytes = batch_layout(ps, count, nullptr, nullptr, &toff);
    return WLB_OK;
}

wlb_status wlb_batch_create(const wlb_params *ps, int count, void *ws, size_t ws_bytes, void *stream,
                            wlb_batch **out) {
    if (!out) return WLB_ERR_ARG;
    wlb_status st = batch_validate(ps, count);
    if (st != WLB_OK) return st;
    if (ws && ((uintptr_t)ws & 255u)) return WLB_ERR_ARG;
    size_t toff;
    const size_t need = batch_layout(ps, count, nullptr, nullptr, &toff);
    if (ws && ws_bytes < need) return WLB_ERR_OOM;
    wlb_batch *b = new (std::nothrow) wlb_batch();
    if (!b) return WLB_ERR_OOM;
    b->count = count;
    b->prec = wlb::prec_of(&ps[0]);
    b->dim = ps[0].lattice == WLB_D2Q5 ? 2 : 3;
    b->p.assign(ps, ps + count);
    b->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) {
        delete b;
        return WLB_ERR_CUDA;
    }
    char *base = (char *)ws;
    if (!base) {
        if (cudaMalloc(&b->owned, need) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return WLB_ERR_OOM;
        }
        base = (char *)b->owned;
    }
    b->lat.reserve(count);
    batch_layout(ps, count, base, &b->lat, &toff);
    char *tb = base + toff;
    b->d_lats = (BatchLat *)tb;
    tb += align256(sizeof(BatchLat) * count);
    b->d_row_begin = (long long *)tb;
    tb += align256(sizeof(long long) * (count + 1));
    b->d_pt_begin = (long long *)tb;
    tb += align256(sizeof(long long) * (count + 1));
    b->d_step = (long long *)tb;
    tb += align256(sizeof(long long));
    b->d_done = (unsigned *)tb;
    tb += align256(sizeof(unsigned));
    for (int c = 0; c < wlb::kMaxChunks; ++c) {
        b->d_class_lats[c] = (LatHot *)tb;
        tb += align256(sizeof(LatHot) * count);
        b->d_class_rows[c] = (long long *)tb;
        tb += align256(sizeof(long long) * (count + 1));
    }
    int *row_lat_base = (int *)tb;
    {
        long long tr = 0, tp = 0;
        for (int i = 0; i < count; ++i) tr += (long long)ps[i].ny * ps[i].nz;
        for (int i = 0; i < count; ++i)
            if (ps[i].n_avg_periods > 0) tp += ps[i].n_surface;
        b->d_pt_lat = (int *)(tb + align256(sizeof(int) * tr));
        b->d_cta_lat = (int *)((char *)b->d_pt_lat + align256(sizeof(int) * (tp > 0 ? tp : 1)));
        b->d_cta_first = (int *)((char *)b->d_cta_lat + align256(sizeof(int) * tr));
    }
    std::vector<long long> rows(count + 1), pts(count + 1);
    int maxv = 1;
    for (int i = 0; i < count; ++i) {
        BatchLat &L = b->lat[i];
        const long long T = (long long)std::nearbyint(ps[i].wavelength / ps[i].c0);
        L.period = T;
        L.n_steps = T * ps[i].n_periods;
        L.window_begin = L.n_steps - T * ps[i].n_avg_periods;
        rows[i] = b->total_rows;
        b->total_rows += (long long)L.g.n[1] * L.g.n[2];
        if (ps[i].n_avg_periods > 0) b->total_points += L.g.n_surface;  // no window: never sampled
        if (L.n_steps > b->max_steps) b->max_steps = L.n_steps;
        b->lattice_updates += L.g.ncell * L.n_steps;
        const int nv = L.g.n[0] / vec_width(b->prec);
        if (nv > maxv) maxv = nv;
    }
    rows[count] = b->total_rows;
    pts[count] = b->total_points;
    // point ranges of the lattices that are sampled (lattices without an
    // averaging window own an empty range) and the point -> lattice table
    std::vector<int> pl((size_t)(b->total_points > 0 ? b->total_points : 1), 0);
    for (int i = 0, acc = 0; i < count; ++i) {
        pts[i] = acc;
        if (ps[i].n_avg_periods > 0) {
            for (int k = 0; k < b->lat[i].g.n_surface; ++k) pl[(size_t)acc + k] = i;
            acc += b->lat[i].g.n_surface;
        }
    }
    b->chunks = (maxv + 31) / 32;
    // row-chunk classes
    std::vector<LatHot> cl_lats[wlb::kMaxChunks];
    for (int i = 0; i < count; ++i) {
        const BatchLat &L = b->lat[i];
        const int ch = (L.g.n[0] / vec_width(b->prec) + 31) / 32;
        LatHot h{};
        h.pop0 = L.b.pop[0];
        h.pop1 = L.b.pop[1];
        h.cls = L.b.cls;
        h.c2 = L.b.c2;
        h.ncell = L.g.ncell;
        h.n_steps = L.n_steps;
        h.c0sq = L.g.c0 * L.g.c0;
        h.cpsq = L.g.cp * L.g.cp;
        h.nx = L.g.n[0];
        h.ny = L.g.n[1];
        h.nz = L.g.n[2];
        cl_lats[ch - 1].push_back(h);
    }
    e = cudaSuccess;
    for (int c = 0; c < wlb::kMaxChunks; ++c) {
        if (cl_lats[c].empty()) continue;
        std::vector<long long> begin(cl_lats[c].size() + 1, 0);
        for (size_t j = 0; j < cl_lats[c].size(); ++j)
            begin[j + 1] = begin[j] + (long long)cl_lats[c][j].ny * cl_lats[c][j].nz;
        std::vector<int> rl((size_t)begin.back());
        for (size_t j = 0; j < cl_lats[c].size(); ++j)
            for (long long r = begin[j]; r < begin[j + 1]; ++r) rl[(size_t)r] = (int)j;
        const int k = b->n_classes++;
        b->class_chunks[k] = c + 1;
        b->class_count[k] = (int)cl_lats[c].size();
        b->class_total_rows[k] = begin.back();
        b->d_class_row_lat[k] = row_lat_base;
        row_lat_base += begin.back();
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_class_lats[k], cl_lats[c].data(), sizeof(LatHot) * cl_lats[c].size(),
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_class_rows[k], begin.data(), sizeof(long long) * begin.size(),
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_class_row_lat[k], rl.data(), sizeof(int) * rl.size(), cudaMemcpyHostToDevice);
    }
    // two steps per launch where every lattice takes it (plans land in b->lat)
    bool even = true;
    for (int i = 0; i < count && even; ++i)
        even = b->lat[i].n_steps % 2 == 0 && b->lat[i].window_begin % 2 == 0 && b->lat[i].period % 2 == 0;
    if (e == cudaSuccess && even && plan_two(b, b->knobs, false) == cudaSuccess) b->two_ok = b->two = true;
    cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(b->d_lats, b->lat.data(), sizeof(BatchLat) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_pt_lat, pl.data(), sizeof(int) * pl.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_row_begin, rows.data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_pt_begin, pts.data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->side.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->side.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->side.join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&b->host_out, sizeof(double) * 5 * count, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        wlb_batch_destroy(b);
        return WLB_ERR_CUDA;
    }
    *out = b;
    return WLB_OK;
}

wlb_status wlb_batch_autotune(wlb_batch *b, int steps_per_trial, wlb_batch_tuning *best) {
    if (!b || steps_per_trial < 1) return WLB_ERR_ARG;
    wlb_status st = batch_setup(b);
    if (st != WLB_OK) return st;
    cudaEvent_t e0, e1;
    BATCH_CUDA(b, cudaEventCreate(&e0), "event");
    BATCH_CUDA(b, cudaEventCreate(&e1), "event");
    if (b->two) {
        // time one plan: a warm-up pair of steps, then steps from step 0 (all
        // lattices active)
        const int steps = 2 * ((steps_per_trial + 1) / 2);
        auto trial = [&](float *ms) -> cudaError_t {
            cudaError_t e = cudaMemsetAsync(b->d_step, 0, sizeof(long long), b->stream);
            if (e == cudaSuccess) e = issue_steps(b, 2, b->threads, b->blocks_per_sm, b->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(b->d_step, 0, sizeof(long long), b->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
            if (e == cudaSuccess) e = issue_steps(b, steps, b->threads, b->blocks_per_sm, b->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
            return e;
        };
        float best_ms = 1e30f;
        wlb::BatchTwoKnobs best_kn = b->knobs;
        int tried = 0;
        cudaError_t e = cudaSuccess;
        if (b->dim == 3) {
            // 3D: every plan of z-chunk length x slab-height cap x lane layout
            // that fits, on the actual batch
            const int zcs[] = {16, 24, 32, 48, 64, 96, 1 << 20};
            const int caps[] = {0, 8, 5};
            for (int sw = 0; sw < 2 && e == cudaSuccess; ++sw)
            for (int oc = 0; oc < 2 && e == cudaSuccess; ++oc)
                for (int zc : zcs)
                    for (int cap : caps) {
                        wlb::BatchTwoKnobs kn;
                        kn.zc_target = zc;
                        kn.h_cap = cap;
                        kn.one_chunk = oc;
                        kn.staging_warp = sw;
                        if (plan_two(b, kn, true) != cudaSuccess) {
                            cudaGetLastError();
                            continue;
                        }
                        float ms = 0;
                        if ((e = trial(&ms)) != cudaSuccess) break;
                        ++tried;
                        if (ms < best_ms) {
                            best_ms = ms;
                            best_kn = kn;
                        }
                    }
            if (e == cudaSuccess && (e = plan_two(b, best_kn, true)) != cudaSuccess) cudaGetLastError();
        } else {
            // 2D: chunk heights around the wave-filling one
            const int rows[] = {0, 32, 24, 20, 16};
            for (int r : rows) {
                wlb::BatchTwoKnobs kn = b->knobs;
                kn.rows_2d = r;
                if (plan_two(b, kn, true) != cudaSuccess) {
                    cudaGetLastError();
                    continue;
                }
                float ms = 0;
                if ((e = trial(&ms)) != cudaSuccess) break;
                ++tried;
                if (ms < best_ms) {
                    best_ms = ms;
                    best_kn = kn;
                }
            }
            if (e == cudaSuccess && (e = plan_two(b, best_kn, true)) != cudaSuccess) cudaGetLastError();
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (e != cudaSuccess) return bfail(b, WLB_ERR_CUDA, "autotune trial", e);
        if (!tried) return bfail(b, WLB_ERR_CUDA, "autotune: no plan fits");
        if (best) {
            best->threads_per_block = b->two_threads;
            best->blocks_per_sm = 1;
            best->ms_per_step = best_ms / steps;
            best->z_chunk = b->dim == 3 ? best_kn.zc_target : b->lat[0].plan.zc;
            best->slab_rows_cap = b->dim == 3 ? best_kn.h_cap : 0;
            best->one_chunk_per_lane = b->dim == 3 ? best_kn.one_chunk : 0;
            best->staging_warp = b->dim == 3 ? best_kn.staging_warp : 0;
            best->plans_tried = tried;
        }
        return WLB_OK;
    }
    const int threads_c[] = {128, 256};
    const int bps_c[] = {2, 4, 8, 16};
    float best_ms = 1e30f;
    int bt = b->threads, bb = b->blocks_per_sm;
    cudaError_t e = issue_steps(b, 2, 256, 4, b->stream);  // warm up
    for (int ti = 0; ti < 2 && e == cudaSuccess; ++ti)
        for (int bi = 0; bi < 4 && e == cudaSuccess; ++bi) {
            // every trial starts at step 0 so that all lattices are active
            e = cudaMemsetAsync(b->d_step, 0, sizeof(long long), b->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
            if (e == cudaSuccess) e = issue_steps(b, steps_per_trial, threads_c[ti], bps_c[bi], b->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && ms < best_ms) {
                best_ms = ms;
                bt = threads_c[ti];
                bb = bps_c[bi];
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return bfail(b, WLB_ERR_CUDA, "autotune trial", e);
    b->threads = bt;
    b->blocks_per_sm = bb;
    if (best) {
        best->threads_per_block = bt;
        best->blocks_per_sm = bb;
        best->ms_per_step = best_ms / steps_per_trial;
        best->z_chunk = best->slab_rows_cap = best->one_chunk_per_lane = best->staging_warp = 0;
        best->plans_tried = 8;
    }
    return WLB_OK;
}

wlb_status wlb_batch_run(wlb_batch *b, double *forces_out) {
    if (!b || !forces_out) return WLB_ERR_ARG;
    wlb_status st = batch_setup(b);
    if (st != WLB_OK) return st;
    if (!b->graph || b->graph_threads != b->threads || b->graph_bps != b->blocks_per_sm ||
        b->graph_two != (int)b->two || b->graph_plan_gen != b->plan_gen) {
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        BATCH_CUDA(b, cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t e = issue_steps(b, wlb::kGraphSteps, b->threads, b->blocks_per_sm, b->capture);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b->capture, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return bfail(b, WLB_ERR_CUDA, "capture steps", e != cudaSuccess ? e : e2);
        }
        e = cudaGraphInstantiate(&b->graph, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->graph = nullptr;
            return bfail(b, WLB_ERR_CUDA, "instantiate", e);
        }
        b->graph_threads = b->threads;
        b->graph_bps = b->blocks_per_sm;
        b->graph_two = (int)b->two;
        b->graph_plan_gen = b->plan_gen;
    }
    const long long full = b->max_steps / wlb::kGraphSteps, rest = b->max_steps % wlb::kGraphSteps;
    for (long long k = 0; k < full; ++k) BATCH_CUDA(b, cudaGraphLaunch(b->graph, b->stream), "graph launch");
    BATCH_CUDA(b, issue_steps(b, (int)rest, b->threads, b->blocks_per_sm, b->stream), "step kernels");
    for (int i = 0; i < b->count; ++i) {
        const BatchLat &L = b->lat[i];
        const long long nw = L.n_steps - L.window_begin;
        if (nw > 0 && L.g.n_surface > 0) {
            BATCH_CUDA(b, wlb::launch_force(L.g, L.b, (double)nw, b->stream), "force kernel");
        } else {
            BATCH_CUDA(b, cudaMemsetAsync(L.b.force, 0, 4 * sizeof(double), b->stream), "zero force");
        }
        BATCH_CUDA(b, cudaMemcpyAsync(b->host_out + 5 * i, L.b.force, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                                      b->stream), "force copy");
        BATCH_CUDA(b, cudaMemcpyAsync(b->host_out + 5 * i + 4, L.b.err, sizeof(int), cudaMemcpyDeviceToHost,
                                      b->stream), "flag copy");
    }
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream), "synchronize");
    bool bad = false;
    for (int i = 0; i < b->count; ++i) {
        int flag;
        memcpy(&flag, b->host_out + 5 * i + 4, sizeof(int));
        bad |= flag != 0;
        for (int a = 0; a < 3; ++a) forces_out[3 * i + a] = b->host_out[5 * i + a];
    }
    if (bad) return bfail(b, WLB_ERR_UNSTABLE, "non-finite accumulators in a lattice");
    return WLB_OK;
}

wlb_status wlb_batch_get_info(const wlb_batch *b, wlb_batch_info *out) {
    if (!b || !out) return WLB_ERR_ARG;
    out->count = b->count;
    out->total_rows = b->total_rows;
    out->total_points = b->total_points;
    out->max_steps = b->max_steps;
    out->lattice_updates = b->lattice_updates;
    out->threads_per_block = b->threads;
    out->blocks_per_sm = b->blocks_per_sm;
    out->row_chunks = b->chunks;
    out->steps_per_launch = b->two ? 2 : 1;
    out->total_ctas = b->two ? b->total_ctas : 0;
    return WLB_OK;
}

wlb_status wlb_batch_set_two_step(wlb_batch *b, int enable) {
    if (!b) return WLB_ERR_ARG;
    if (enable && !b->two_ok) return bfail(b, WLB_ERR_ARG, "two steps per launch not available for this batch");
    b->two = enable != 0;
    return WLB_OK;
}

const char *wlb_batch_last_error(const wlb_batch *b) { return b ? b->err : ""; }

wlb_status wlb_batch_destroy(wlb_batch *b) {
    if (!b) return WLB_ERR_ARG;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->capture) cudaStreamDestroy(b->capture);
    if (b->side.stream) cudaStreamDestroy(b->side.stream);
    if (b->side.fork) cudaEventDestroy(b->side.fork);
    if (b->side.join) cudaEventDestroy(b->side.join);
    if (b->host_out) cudaFreeHost(b->host_out);
    if (b->owned) cudaFree(b->owned);
    delete b;
    return WLB_OK;
}

}  // extern "C"
