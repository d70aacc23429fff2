// Two lattice steps per launch for batches of 2D lattices (D2Q5, periodic).
//
// The update is the fused advection + tau = 1/2 collision (Sec. V, Eqs.
// 62-64, 71) applied twice: S1 takes state t (buffer A) to t+1, S2 takes t+1
// to t+2 (buffer B).  In 2D a lattice row needs no neighbour row of the same
// time level besides those above and below it, so each warp sweeps a chunk of
// rows ya .. yb-1 on its own: for p = ya-1 .. yb it computes S1 on row p from
// A (rows p-1, p, p+1, staged in the warp's shared-memory ring three rows
// ahead by per-thread asynchronous copies), then S2 on row p-1 from its
// registers:
//   rest, +x, -x   from S1 of row p-1 (x shift by shuffles, periodic wrap),
//   +y             from S1 of row p-2,
//   -y             from S1 of row p.
// No barrier, no warp waits for another (each lane reads back only what it
// copied); the rows just outside a chunk are computed by both warps that need
// them.  The t+1 values
// are rounded to the storage type as a stored state would be, so results are
// bit-identical to two single steps.
#include "wlb_handle.cuh"
#include "wlb_kernels.cuh"

namespace wlb {
namespace {

constexpr int kRowsPerWarp = 32;   // row chunk of one warp (two halo rows per chunk), at most
constexpr int kMinRowsPerWarp = 8;  // batches: shortest chunk the planner considers
constexpr int kWarpsPerBlock = 2;  // small blocks: as many warps per SM as registers allow
constexpr int kDepth = 3;          // rows staged ahead per warp (shared memory)

// The value a stored state holds for v (storage rounding).
template <typename S> __device__ __forceinline__ typename Store<S>::R as_stored(typename Store<S>::R v) { return v; }
template <> __device__ __forceinline__ float as_stored<__half>(float v) { return __half2float(__float2half_rn(v)); }

// +x / -x pulls of a row held as CH chunks of W values per lane in slots
// j = c * 32 + lane (x = j * W + e), the first V slots being cells: the value
// from x - 1 and from x + 1, periodic in x.
template <typename R, int CH, int W>
__device__ __forceinline__ void row_shift(const R (&px)[CH][W], const R (&mx)[CH][W], int lane, int V,
                                          R (&fpx)[CH][W], R (&fmx)[CH][W]) {
    R up[CH], dn[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        up[c] = __shfl_sync(kFull, px[c][W - 1], (lane + 31) & 31);
        dn[c] = __shfl_sync(kFull, mx[c][0], (lane + 1) & 31);
    }
    // wrap: +x at x = 0 is the last cell's value, -x at the last cell is x = 0's
    R lastv = px[0][W - 1];
#pragma unroll
    for (int c = 1; c < CH; ++c)
        if (c == (V - 1) >> 5) lastv = px[c][W - 1];
    const R left = __shfl_sync(kFull, lastv, (V - 1) & 31);
    const R right = __shfl_sync(kFull, mx[0][0], 0);
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        fpx[c][0] = lane == 0 ? (c == 0 ? left : up[c - 1]) : up[c];
#pragma unroll
        for (int e = 1; e < W; ++e) fpx[c][e] = px[c][e - 1];
#pragma unroll
        for (int e = 0; e < W - 1; ++e) fmx[c][e] = mx[c][e + 1];
        const R next = lane == 31 ? (c == CH - 1 ? right : dn[c + 1]) : dn[c];
        fmx[c][W - 1] = c * 32 + lane == V - 1 ? right : next;
    }
}

// Plain 16-byte shared-memory reads of W values of the storage type.
template <typename S> struct StageVec;
template <> struct StageVec<float> {
    __device__ static void ld(const float *p, float (&v)[4]) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
};
template <> struct StageVec<double> {
    __device__ static void ld(const double *p, double (&v)[2]) {
        const double2 t = *reinterpret_cast<const double2 *>(p);
        v[0] = t.x; v[1] = t.y;
    }
};
template <> struct StageVec<__half> {
    __device__ static void ld(const __half *p, float (&v)[8]) {
        const uint4 t = *reinterpret_cast<const uint4 *>(p);
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
};

// Per-thread asynchronous 16-byte copies global -> shared (each lane copies
// exactly the vectors it reads back later, so waiting on its own groups is all
// the synchronisation needed).
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// One 2D lattice as a row sweep sees it.
template <typename S>
struct Rows2D {
    const S *A;  // state t
    S *B;        // state t + 2
    const uint8_t *cls;
    const typename Store<S>::R *c2f;
    int nx, ny;
    long long ncell;
    typename Store<S>::R c0sq, cpsq;
    int yc;  // rows per warp chunk
};

template <typename S>
__host__ __device__ inline Rows2D<S> rows2d(const Geometry &g, const Buffers &b, int src, int yc) {
    using R = typename Store<S>::R;
    Rows2D<S> P;
    P.A = (const S *)b.pop[src];
    P.B = (S *)b.pop[src ^ 1];
    P.cls = b.cls;
    P.c2f = (const R *)b.c2;
    P.nx = g.n[0];
    P.ny = g.n[1];
    P.ncell = g.ncell;
    P.c0sq = (R)(g.c0 * g.c0);
    P.cpsq = (R)(g.cp * g.cp);
    P.yc = yc;
    return P;
}

// The sweep of one row chunk of one lattice by one warp (warp-uniform flow).
// `ring`: this warp's kDepth staging slots of the five rows S1 of a row pulls
// (nxs values each).
template <typename S, int CH>
__device__ __forceinline__ void sweep_rows(const Rows2D<S> &P, int chunk, int lane, S *ring, int nxs) {
    using R = typename Store<S>::R;
    constexpr int W = Store<S>::W;
    const int nx = P.nx, ny = P.ny;
    const long long nc = P.ncell;
    const int V = nx / W, yc = P.yc;
    const int ya = chunk * yc, yb = min(ny, ya + yc);
    const S *__restrict__ A = P.A;
    S *__restrict__ B = P.B;
    const uint8_t *__restrict__ cls = P.cls;
    const R *__restrict__ c2f = P.c2f;
    const R c0sq = P.c0sq, cpsq = P.cpsq;
    bool act[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) act[c] = c * 32 + lane < V;
    R n0[CH][W], n1[CH][W], n2[CH][W], cq[CH][W];  // S1 of row p-1: rest, +x, -x; its c^2
    R py0[CH][W], py1[CH][W];                      // +y of S1 rows p-2, p-1
    // Stage the five rows S1 of row p pulls into slot (p - ya + 1) % kDepth;
    // one commit group per row (empty past the chunk).
    auto stage_row = [&](int p) {
        if (p <= yb) {
            const int y = (p + ny) % ny, ym = (y + ny - 1) % ny, yp = (y + 1) % ny;
            const long long r0 = (long long)y * nx;
            S *dst = ring + (size_t)((p - ya + 1) % kDepth) * 5 * nxs;
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                if (!act[c]) continue;
                const int x0 = (c * 32 + lane) * W;
                cp_async16(dst + x0, A + r0 + x0);
                cp_async16(dst + nxs + x0, A + nc + r0 + x0);
                cp_async16(dst + 2 * nxs + x0, A + 2 * nc + r0 + x0);
                cp_async16(dst + 3 * nxs + x0, A + 3 * nc + (long long)ym * nx + x0);
                cp_async16(dst + 4 * nxs + x0, A + 4 * nc + (long long)yp * nx + x0);
            }
        }
        cp_async_commit();
    };
    // class bytes of row p, one row ahead in registers
    auto load_cls = [&](int p, unsigned long long (&gc)[CH]) {
        const long long r0 = (long long)((p + ny) % ny) * nx;
#pragma unroll
        for (int c = 0; c < CH; ++c) gc[c] = act[c] ? load_classes<W>(cls + r0 + (c * 32 + lane) * W) : 0ull;
    };
#pragma unroll
    for (int d = 0; d < kDepth; ++d) stage_row(ya - 1 + d);
    unsigned long long cl[CH];
    load_cls(ya - 1, cl);
    for (int k = 0, p = ya - 1; p <= yb; ++k, ++p) {
        const int y = (p + ny) % ny;
        const long long r0 = (long long)y * nx;
        unsigned long long cln[CH];
        if (p < yb) load_cls(p + 1, cln);
        cp_async_wait<kDepth - 1>();  // this lane's copies of row p have landed
        const S *st = ring + (size_t)(k % kDepth) * 5 * nxs;
        R f[5][CH][W];
        R cs[CH][W];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int x0 = (c * 32 + lane) * W;
            if (act[c]) {
#pragma unroll
                for (int i = 0; i < 5; ++i) StageVec<S>::ld(st + (size_t)i * nxs + x0, f[i][c]);
            } else {
#pragma unroll
                for (int i = 0; i < 5; ++i)
#pragma unroll
                    for (int e = 0; e < W; ++e) f[i][c][e] = R(0);
            }
#pragma unroll
            for (int e = 0; e < W; ++e) {  // the c^2 of the one-step kernels
                const unsigned kc = (unsigned)(cl[c] >> (8 * e)) & 0xffu;
                cs[c][e] = kc == CELL_FLUID ? c0sq : (kc == CELL_OBJECT ? cpsq : (act[c] ? c2f[r0 + x0 + e] : c0sq));
            }
        }
        R fpx[CH][W], fmx[CH][W];
        row_shift<R, CH, W>(f[1], f[2], lane, V, fpx, fmx);
        R o[5][CH][W];  // S1 of row p in storage precision
#pragma unroll
        for (int c = 0; c < CH; ++c)
#pragma unroll
            for (int e = 0; e < W; ++e) {
                const R fin[5] = {f[0][c][e], fpx[c][e], fmx[c][e], f[3][c][e], f[4][c][e]};
                R t5[5];
                collide_half<R, 2>(cs[c][e], fin, t5);
#pragma unroll
                for (int i = 0; i < 5; ++i) o[i][c][e] = as_stored<S>(t5[i]);
            }
        if (k >= 2) {  // S2 on row q = p - 1
            const int q = (y + ny - 1) % ny;
            const long long rq = (long long)q * nx;
            R gpx[CH][W], gmx[CH][W];
            row_shift<R, CH, W>(n1, n2, lane, V, gpx, gmx);
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                if (!act[c]) continue;
                const int x0 = (c * 32 + lane) * W;
                R out[5][W];
#pragma unroll
                for (int e = 0; e < W; ++e) {
                    const R fin[5] = {n0[c][e], gpx[c][e], gmx[c][e], py0[c][e], o[4][c][e]};
                    R t5[5];
                    collide_half<R, 2>(cq[c][e], fin, t5);
#pragma unroll
                    for (int i = 0; i < 5; ++i) out[i][e] = t5[i];
                }
#pragma unroll
                for (int i = 0; i < 5; ++i) Store<S>::store(B + i * nc + rq + x0, out[i]);
            }
        }
        stage_row(p + kDepth);  // refill the slot just read (its values are in registers)
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            if (p < yb) cl[c] = cln[c];
#pragma unroll
            for (int e = 0; e < W; ++e) {
                py0[c][e] = py1[c][e];
                py1[c][e] = o[3][c][e];
                n0[c][e] = o[0][c][e];
                n1[c][e] = o[1][c][e];
                n2[c][e] = o[2][c][e];
                cq[c][e] = cs[c][e];
            }
        }
    }
    cp_async_wait<0>();
}

// One launch: warp w sweeps chunk w - task_first[i] of lattice i = task_lat[w]
// (lattices past their n_steps skip).  The state at step t is in buffer
// (t / 2) & 1; the last block to finish advances the step by two (every block
// has read it by then).
template <typename S, int CH>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) batch2d_update2(const BatchLat *__restrict__ lats,
                                                                       const int *__restrict__ task_lat,
                                                                       const int *__restrict__ task_first,
                                                                       int total_tasks, int nxs,
                                                                       long long *step, unsigned *done) {
    extern __shared__ __align__(16) unsigned char smem2d[];
    const long long t = *step;
    const int lane = threadIdx.x & 31;
    const int task = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (task < total_tasks) {
        const int i = task_lat[task];
        const BatchLat &L = lats[i];
        S *ring = reinterpret_cast<S *>(smem2d) + (size_t)(threadIdx.x >> 5) * kDepth * 5 * nxs;
        if (t < L.n_steps)  // warp-uniform
            sweep_rows<S, CH>(rows2d<S>(L.g, L.b, (int)((t >> 1) & 1), L.plan.zc), task - task_first[i], lane, ring,
                              nxs);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned ticket = atomicAdd(done, 1u);
        if (ticket == gridDim.x - 1) {
            *done = 0;
            *step = t + 2;
            __threadfence();
        }
    }
}

// rho1 and J1 of cell (x, y) at t+1 from the populations A of time t: each of
// the five values the cell pulls is the t+1 value of the neighbour it comes
// from, recomputed from A with the update's arithmetic and storage rounding,
// then summed in the order of pulled_moments.
template <typename S>
__device__ __forceinline__ void moments_next_2d(const Geometry &g, const S *__restrict__ A,
                                                const typename Store<S>::R *__restrict__ c2f, int x, int y,
                                                typename Store<S>::R &rho, typename Store<S>::R (&J)[3]) {
    using R = typename Store<S>::R;
    const int nx = g.n[0], ny = g.n[1];
    const long long nc = g.ncell;
    auto dn = [](int v, int n) { return v == 0 ? n - 1 : v - 1; };
    auto up = [](int v, int n) { return v == n - 1 ? 0 : v + 1; };
    auto post = [&](int i, int cx, int cy) -> R {  // f*_i(cx, cy) at t+1
        const long long row = (long long)cy * nx;
        const R fin[5] = {Store<S>::get(A + row + cx), Store<S>::get(A + nc + row + dn(cx, nx)),
                          Store<S>::get(A + 2 * nc + row + up(cx, nx)),
                          Store<S>::get(A + 3 * nc + (long long)dn(cy, ny) * nx + cx),
                          Store<S>::get(A + 4 * nc + (long long)up(cy, ny) * nx + cx)};
        R o[5];
        collide_half<R, 2>(c2f[row + cx], fin, o);
        return as_stored<S>(o[i]);
    };
    const R f0 = post(0, x, y);
    const R fpx = post(1, dn(x, nx), y);
    const R fmx = post(2, up(x, nx), y);
    const R fpy = post(3, x, dn(y, ny));
    const R fmy = post(4, x, up(y, ny));
    rho = f0 + fpx + fmx + fpy + fmy;
    J[0] = fpx - fmx;
    J[1] = fpy - fmy;
    J[2] = R(0);
}

// Sampling of both steps of a launch, one thread per point: sums of t (the
// stored state) and t+1 (recomputed) in that order, then the period fold when
// t+1 closes a period (periods and windows are even).
template <typename S>
__global__ void __launch_bounds__(256) batch2d_sample_two(const BatchLat *__restrict__ lats,
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
        const S *A = (const S *)L.b.pop[(t >> 1) & 1];
        const R *st_w = (const R *)L.b.st_w, *nrm = (const R *)L.b.nrm;
        R *acc = (R *)L.b.acc;
        sample_point_2d_thread(L.g, L.b.st_xyz, st_w, nrm, acc, k, [&](int x, int y, int z, R &rho, R(&J)[3]) {
            pulled_moments(L.g, A, x, y, z, rho, J);
        });
        sample_point_2d_thread(L.g, L.b.st_xyz, st_w, nrm, acc, k, [&](int x, int y, int, R &rho, R(&J)[3]) {
            moments_next_2d(L.g, A, (const R *)L.b.c2, x, y, rho, J);
        });
        if ((t + 2 - L.window_begin) % L.period == 0) {
            const double scale = 1.0 / (L.g.pop_scale * L.g.pop_scale);
            R *a = acc + 5 * (long long)k;
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

// A single 2D lattice (a handle): warp w sweeps row chunk w.
template <typename S, int CH>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) update2_rows2d(Rows2D<S> P, int chunks, int nxs) {
    extern __shared__ __align__(16) unsigned char smem2d[];
    const int lane = threadIdx.x & 31;
    const int task = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (task >= chunks) return;  // whole warp; the sweep has no block barrier
    S *ring = reinterpret_cast<S *>(smem2d) + (size_t)(threadIdx.x >> 5) * kDepth * 5 * nxs;
    sweep_rows<S, CH>(P, task, lane, ring, nxs);
}

// Its sampling of both steps of a launch, one thread per point, in the order
// of two single steps (the handle folds at period ends).
template <typename S>
__global__ void __launch_bounds__(256) sample_two_2d(Geometry g, const int4 *__restrict__ st_xyz,
                                                     const typename Store<S>::R *__restrict__ st_w,
                                                     const typename Store<S>::R *__restrict__ nrm,
                                                     typename Store<S>::R *acc, const S *__restrict__ A,
                                                     const typename Store<S>::R *__restrict__ c2f) {
    using R = typename Store<S>::R;
    const int k = (int)((long long)blockIdx.x * blockDim.x + threadIdx.x);
    if (k >= g.n_surface) return;
    sample_point_2d_thread(g, st_xyz, st_w, nrm, acc, k, [&](int x, int y, int z, R &rho, R(&J)[3]) {
        pulled_moments(g, A, x, y, z, rho, J);
    });
    sample_point_2d_thread(g, st_xyz, st_w, nrm, acc, k, [&](int x, int y, int, R &rho, R(&J)[3]) {
        moments_next_2d(g, A, c2f, x, y, rho, J);
    });
}

// ---------------------------------------------------------------- host side: plans and launches

// Chunks per lane for a 2D row of nx cells: 0 if it is not a whole number of
// 16-byte vectors or needs more than two chunks / eight values per lane.
template <typename S>
int chunks_2d(int nx) {
    constexpr int W = Store<S>::W;
    if (nx % W) return 0;
    const int c = (nx / W + 31) / 32;
    return (c <= 2 && W * c <= 8) ? c : 0;
}

template <typename S>
cudaError_t launch_single(const Geometry &g, const Buffers &b, const TwoStepPlan &pl, int src, bool sample,
                          cudaStream_t s) {
    using R = typename Store<S>::R;
    if (sample && g.n_surface > 0) {
        sample_two_2d<S><<<(g.n_surface + 255) / 256, 256, 0, s>>>(g, b.st_xyz, (const R *)b.st_w, (const R *)b.nrm,
                                                                   (R *)b.acc, (const S *)b.pop[src],
                                                                   (const R *)b.c2);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const Rows2D<S> P = rows2d<S>(g, b, src, pl.zc);
    const int blocks = (pl.chunks + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (pl.chunks_per_lane == 1)
        update2_rows2d<S, 1><<<blocks, pl.threads, pl.smem, s>>>(P, pl.chunks, g.n[0]);
    else if constexpr (Store<S>::W * 2 <= 8)
        update2_rows2d<S, 2><<<blocks, pl.threads, pl.smem, s>>>(P, pl.chunks, g.n[0]);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <typename S>
bool plan_for(BatchLat *lats, int count, int rows_fixed, int *tasks, int *chunks_per_lane, int *nx_max) {
    constexpr int W = Store<S>::W;
    int ch = 1, total = 0, wide = 0;
    for (int i = 0; i < count; ++i) {
        const Geometry &g = lats[i].g;
        if (g.dim != 2 || g.driven || g.n[0] % W) return false;
        const int V = g.n[0] / W;
        const int c = (V + 31) / 32;
        if (c > 2 || W * c > 8) return false;  // at most 8 values per lane
        ch = c > ch ? c : ch;
        wide = g.n[0] > wide ? g.n[0] : wide;
    }
    // Rows per warp chunk, the same for every lattice: the chunks should fill
    // whole waves of the warps an SM holds (time ~ waves x (rows + 2), the two
    // halo rows recomputed per chunk).  512 lattices of 192 rows: 32-row chunks
    // are 3072 warps in 1.68 waves of 1824, 28-row chunks 3584 in 1.96.
    int slots = 0;
    {
        int dev = 0, sms = 0, bps = 0;
        const size_t smem = (size_t)kWarpsPerBlock * kDepth * 5 * wide * sizeof(S);
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            (ch == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, batch2d_update2<S, 1>, 32 * kWarpsPerBlock,
                                                                     smem)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, batch2d_update2<S, 2>, 32 * kWarpsPerBlock,
                                                                     smem)) == cudaSuccess)
            slots = sms * bps * kWarpsPerBlock;
        cudaGetLastError();
    }
    int rows = rows_fixed > 0 ? rows_fixed : kRowsPerWarp;
    if (slots > 0 && rows_fixed <= 0) {
        long long best = -1;
        for (int zc = kRowsPerWarp; zc >= kMinRowsPerWarp; --zc) {
            long long n = 0;
            for (int i = 0; i < count; ++i) {
                const int z = lats[i].g.n[1] < zc ? lats[i].g.n[1] : zc;
                n += (lats[i].g.n[1] + z - 1) / z;
            }
            const long long cost = (n + slots - 1) / slots * (zc + 2);
            if (best < 0 || cost < best) {
                best = cost;
                rows = zc;
            }
        }
    }
    for (int i = 0; i < count; ++i) {
        const Geometry &g = lats[i].g;
        TwoStepPlan pl;
        pl.zc = g.n[1] < rows ? g.n[1] : rows;
        pl.chunks = (g.n[1] + pl.zc - 1) / pl.zc;
        pl.nslab = 1;
        pl.nseg = 1;
        pl.H = 1;
        pl.chunks_per_lane = (g.n[0] / W + 31) / 32;
        pl.threads = 32 * kWarpsPerBlock;
        lats[i].plan = pl;
        total += pl.chunks;
    }
    *tasks = total;
    *chunks_per_lane = ch;
    *nx_max = wide;
    return true;
}

template <typename S>
cudaError_t launch_for(int ch, int nx_max, const BatchLat *lats, const int *task_lat, const int *task_first,
                       int total_tasks, const int *pt_lat, const long long *pt_begin, long long total_points,
                       long long *step, unsigned *done, int sample_grid, cudaStream_t s) {
    if (total_points > 0) {
        const long long need = (total_points + 255) / 256;
        const int g = (int)(need < sample_grid ? need : sample_grid);
        batch2d_sample_two<S><<<g, 256, 0, s>>>(lats, pt_lat, pt_begin, total_points, step);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int blocks = (total_tasks + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const int threads = 32 * kWarpsPerBlock;
    // per warp: kDepth slots of five rows of the widest lattice (<= 30 KB a block)
    const size_t smem = (size_t)kWarpsPerBlock * kDepth * 5 * nx_max * sizeof(S);
    if (ch == 1)
        batch2d_update2<S, 1><<<blocks, threads, smem, s>>>(lats, task_lat, task_first, total_tasks, nx_max, step,
                                                             done);
    else if constexpr (Store<S>::W * 2 <= 8)
        batch2d_update2<S, 2><<<blocks, threads, smem, s>>>(lats, task_lat, task_first, total_tasks, nx_max, step,
                                                             done);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace

bool plan_batch2d_two_steps(Prec p, BatchLat *lats, int count, int rows, int *tasks, int *chunks_per_lane,
                            int *nx_max) {
    switch (p) {
        case Prec::F16: return plan_for<__half>(lats, count, rows, tasks, chunks_per_lane, nx_max);
        case Prec::F64: return plan_for<double>(lats, count, rows, tasks, chunks_per_lane, nx_max);
        default: return plan_for<float>(lats, count, rows, tasks, chunks_per_lane, nx_max);
    }
}

cudaError_t launch_batch2d_two_steps(Prec p, int chunks_per_lane, int nx_max, const BatchLat *lats, const int *task_lat,
                                     const int *task_first, int total_tasks, const int *pt_lat,
                                     const long long *pt_begin, long long total_points, long long *step,
                                     unsigned *done, int sample_grid, cudaStream_t s) {
    switch (p) {
        case Prec::F16:
            return launch_for<__half>(chunks_per_lane, nx_max, lats, task_lat, task_first, total_tasks, pt_lat, pt_begin,
                                      total_points, step, done, sample_grid, s);
        case Prec::F64:
            return launch_for<double>(chunks_per_lane, nx_max, lats, task_lat, task_first, total_tasks, pt_lat, pt_begin,
                                      total_points, step, done, sample_grid, s);
        default:
            return launch_for<float>(chunks_per_lane, nx_max, lats, task_lat, task_first, total_tasks, pt_lat, pt_begin,
                                     total_points, step, done, sample_grid, s);
    }
}

bool two_step_2d_supported(const Geometry &g, Prec p) {
    if (g.dim != 2 || g.driven) return false;
    switch (p) {
        case Prec::F16: return chunks_2d<__half>(g.n[0]) > 0;
        case Prec::F64: return chunks_2d<double>(g.n[0]) > 0;
        default: return chunks_2d<float>(g.n[0]) > 0;
    }
}

cudaError_t plan_two_steps_2d(const Geometry &g, Prec p, TwoStepPlan *out) {
    if (!two_step_2d_supported(g, p)) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const size_t bytes = p == Prec::F16 ? 2 : (p == Prec::F64 ? 8 : 4);
    TwoStepPlan pl;
    pl.chunks_per_lane = p == Prec::F16 ? chunks_2d<__half>(g.n[0])
                                        : (p == Prec::F64 ? chunks_2d<double>(g.n[0]) : chunks_2d<float>(g.n[0]));
    // rows per warp: up to kRowsPerWarp, fewer on short lattices so that
    // every SM gets work (at least 4: two of the rows are halo)
    const int per_sm = g.n[1] / (sms > 0 ? sms : 1);
    pl.zc = per_sm < 4 ? 4 : (per_sm > kRowsPerWarp ? kRowsPerWarp : per_sm);
    if (pl.zc > g.n[1]) pl.zc = g.n[1];
    pl.chunks = (g.n[1] + pl.zc - 1) / pl.zc;
    pl.H = pl.zc;
    pl.nslab = 1;
    pl.nseg = 1;
    pl.threads = 32 * kWarpsPerBlock;
    pl.smem = (size_t)kWarpsPerBlock * kDepth * 5 * g.n[0] * bytes;
    *out = pl;
    return cudaSuccess;
}

cudaError_t launch_two_steps_2d(const Geometry &g, const Buffers &b, Prec p, const TwoStepPlan &pl, int src,
                                bool sample, cudaStream_t s) {
    switch (p) {
        case Prec::F16: return launch_single<__half>(g, b, pl, src, sample, s);
        case Prec::F64: return launch_single<double>(g, b, pl, src, sample, s);
        default: return launch_single<float>(g, b, pl, src, sample, s);
    }
}

}  // namespace wlb
