// Two lattice steps per launch (3D, periodic): temporal blocking in y-slabs
// with recomputed halo rows; in sampled steps a sampling kernel beside it adds
// the surface sums of both steps.
//
// The update is the fused advection + tau = 1/2 collision of update_rows
// (Sec. V, Eqs. 62-64, 71) applied twice: S1 takes state t (buffer A) to t+1,
// S2 takes t+1 to t+2 (buffer B).  State t+1 never leaves the SM.
//
// A CTA owns the H rows y0 .. y0+H-1 of the planes za .. zb-1 and sweeps z.
// For each plane p = za-1 .. zb it computes S1 on the H + 2 rows y0-1 .. y0+H
// (one halo row on either side, also computed by the neighbouring slab), then
// S2 on plane p-1.  Warp w computes S1 on row y0-1+w and, for w = 1 .. H, S2 on
// the same row, so S2 pulls
//   rest, +x, -x   from the warp's registers of plane p-1 (x shift by shuffles),
//   +z             from its registers of plane p-2,
//   -z             from its registers of plane p,
//   +y, -y         from rows w-1, w+1 of plane p-1, exchanged in shared memory
//                  (a ring of three planes: one barrier per plane).
// The A rows that S1 of a plane pulls from (seven populations x (H+2) rows),
// their class bytes and, for rows holding interface-band cells (a per-row
// flag from setup, read one plane ahead), their c^2 rows are staged in shared
// memory by 1-D bulk (TMA) copies issued two planes ahead and completing on an
// mbarrier (two stages), so no warp waits on a global load of its own.  No CTA
// waits for another CTA: one launch reads A and writes B once, about half the
// HBM traffic of two single steps, plus the halo rows, which neighbouring
// slabs read at the same time (L2 hits).  Results are bit-identical to two single steps: the same
// per-cell arithmetic, and the t+1 values are rounded to the storage type as
// a single step would store them.
//
// Wide rows (x-tiles).  Shared memory bounds the slab height by the row
// length (512-cell FP32 rows leave room for 3-row slabs, so 5 S1 rows are
// computed per 3 output rows).  A plan may instead split each row into
// ntile tiles of tx cells, one warp per tile row (slab_body_tiled): a CTA
// owns one tile of its slab and stages the tile plus one 16-byte vector of
// every array on either side (wrapped around x at the row's ends), and
// computes S1 also on the two halo cells x = xa - 1 and x = xb, whose +x and
// -x values are the ones S2 pulls across the tile's ends.  The tile's rows
// are not contiguous in memory, so instead of bulk copies every warp stages
// its own row with per-thread 16-byte cp.async copies.  That staging costs
// the compute warps instructions that the bulk copies do not, so the
// automatic plan splits only rows too long for any whole-row slab.
#include <algorithm>
#include <cmath>
#include <vector>

#include "wlb_handle.cuh"
#include "wlb_kernels.cuh"

namespace wlb {
namespace {

constexpr long long kWaitLimit = 1LL << 22;  // mbarrier polls before giving up
constexpr int kMaxRows = 16;                 // S1 rows (warps) per CTA
constexpr int kRingPlanes = 3;               // +-y exchange ring
constexpr int kStages = 2;                   // staged A planes (three: 5-row slabs on 256^3, slower)

// Threads per CTA: a warp per S1 row; rows with eight values per lane keep
// enough registers (about 165) with at most twelve warps.
template <typename S, int CH>
constexpr int two_step_threads() {
    return Store<S>::W * CH <= 4 ? 32 * kMaxRows : 32 * 12;
}

// Dynamic shared memory of a whole-row slab of H rows (H + 2 S1 rows) in
// nseg segments: two staged planes of the seven populations (storage type),
// of the class bytes and, with c2_staged, of c^2 (arithmetic type; copied
// only for rows holding interface-band cells); the three-plane +-y exchange
// ring, H rows per population (+y of S1 rows 0 .. H-1 and -y of rows
// 2 .. H+1: the only ones step 2 pulls); the segment-end ring, the stage
// barriers and the staged rows' band flags.
template <typename S>
size_t whole_row_smem(int nx, int nseg, int H, bool c2_staged) {
    using R = typename Store<S>::R;
    const size_t rmax = (size_t)H + 2, n = (size_t)nx;
    return (size_t)kStages * rmax * (7 * n * sizeof(S) + (c2_staged ? n * sizeof(R) : 0) + n) +
           (size_t)kRingPlanes * 2 * (size_t)H * n * sizeof(S) + (size_t)kRingPlanes * rmax * nseg * 2 * sizeof(R) +
           (size_t)kStages * sizeof(uint64_t) + (size_t)kStages * rmax;
}

// Halo cells staged on either side of an x-tile: 16 bytes of each array.
template <typename S> constexpr int halo_pop() { return 16 / (int)sizeof(S); }
template <typename S> constexpr int halo_c2() { return 16 / (int)sizeof(typename Store<S>::R); }
constexpr int kHaloCls = 16;

// Shared memory per S1 row of a tiled plan (tiles of tx cells, one warp
// per tile row): two staged planes of tx + 2 halo cells of every array and
// the three-plane exchange ring of tx cells.
template <typename S>
constexpr size_t smem_per_tile_row(int tx) {
    using R = typename Store<S>::R;
    return (size_t)kStages * (7 * (size_t)(tx + 2 * halo_pop<S>()) * sizeof(S) +
                              (size_t)(tx + 2 * halo_c2<S>()) * sizeof(R) + (size_t)(tx + 2 * kHaloCls)) +
           (size_t)kRingPlanes * 2 * (size_t)tx * sizeof(S);
}

template <typename S> struct Vec;  // plain 16-byte shared-memory accesses

template <> struct Vec<float> {
    __device__ static void ld(const float *p, float (&v)[4]) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    __device__ static void st(float *p, const float (&v)[4]) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
    __device__ static float rounded(float v) { return v; }
    __device__ static void rounded(const float (&in)[4], float (&out)[4]) {
#pragma unroll
        for (int e = 0; e < 4; ++e) out[e] = in[e];
    }
    __device__ static float get(const float *p) { return *p; }
};

template <> struct Vec<__half> {
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
    __device__ static void st(__half *p, const float (&v)[8]) {
        unsigned w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __half2 h = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
            memcpy(&w[i], &h, 4);
        }
        *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    // the value a single step would store and the next step read back
    __device__ static float rounded(float v) { return __half2float(__float2half_rn(v)); }
    __device__ static void rounded(const float (&in)[8], float (&out)[8]) {  // pairwise, same rounding
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            const float2 f = __half22float2(__floats2half2_rn(in[e], in[e + 1]));
            out[e] = f.x;
            out[e + 1] = f.y;
        }
    }
    __device__ static float get(const __half *p) { return __half2float(*p); }
};

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bar)) : "memory");
}

__device__ __forceinline__ void bar_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool bar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P;\n\t}\n"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for a stage: false if it did not complete within the limit.
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity) {
    for (long long i = 0; i < kWaitLimit; ++i)
        if (bar_try(bar, parity)) return true;
    return false;
}

// 1-D bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(saddr(dst)),
        "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(saddr(bar))
        : "memory");
}

// Prefetch `bytes` at `src` into L2 (16-byte aligned, a multiple of 16 bytes).
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(src)), "r"(bytes)
                 : "memory");
}

// W consecutive FP32 values at p (16-byte aligned; shared or global memory).
template <int W>
__device__ __forceinline__ void load_row_vec(const float *p, float (&v)[W]) {
    static_assert(W % 4 == 0, "whole 16-byte vectors");
#pragma unroll
    for (int j = 0; j < W / 4; ++j) {
        const float4 t = *reinterpret_cast<const float4 *>(p + 4 * j);
        v[4 * j] = t.x;
        v[4 * j + 1] = t.y;
        v[4 * j + 2] = t.z;
        v[4 * j + 3] = t.w;
    }
}

// The collision of the one-step kernels (collide_half), pulled populations
// (0, +x, -x, +y, -y, +z, -z) passed one by one.
template <typename R>
__device__ __forceinline__ void collide7(R c2, R f0, R fpx, R fmx, R fpy, R fmy, R fpz, R fmz, R (&o)[7]) {
    const R f[7] = {f0, fpx, fmx, fpy, fmy, fpz, fmz};
    collide_half<R, 3>(c2, f, o);
}

// +x / -x pulls of a warp's segment of a row, held as CH chunks of W values
// per lane in slots j = c * 32 + lane (x = xs + j * W + e), of which the first
// vg are cells: the value from x - 1 and from x + 1.  Inside the segment they
// come by shuffles; at its ends from `left` (the +x value at xs - 1, used by
// slot 0) and `right` (the -x value at the first cell past the segment, used
// by slot vg - 1), both periodic in x.  With `whole` (one full segment is the
// whole row) the ends wrap around by shuffles and left / right are not read.
template <typename R, int CH, int W>
__device__ __forceinline__ void shift_x(const R (&px)[CH][W], const R (&mx)[CH][W], int lane, int vg, bool whole,
                                        R left, R right, R (&fpx)[CH][W], R (&fmx)[CH][W]) {
    R up[CH], dn[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        up[c] = __shfl_sync(kFull, px[c][W - 1], (lane + 31) & 31);
        dn[c] = __shfl_sync(kFull, mx[c][0], (lane + 1) & 31);
    }
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        fpx[c][0] = lane == 0 ? (c == 0 ? (whole ? up[CH - 1] : left) : up[c - 1]) : up[c];
#pragma unroll
        for (int e = 1; e < W; ++e) fpx[c][e] = px[c][e - 1];
#pragma unroll
        for (int e = 0; e < W - 1; ++e) fmx[c][e] = mx[c][e + 1];
        const R next = lane == 31 ? (c == CH - 1 ? (whole ? dn[0] : right) : dn[c + 1]) : dn[c];
        fmx[c][W - 1] = (!whole && c * 32 + lane == vg - 1) ? right : next;
    }
}

// rho1 and J1 of cell (x, y, z) at t+1 from the populations A of time t.
// Each of the seven values the cell pulls is the t+1 post-collision value of
// the neighbour it comes from, recomputed from A with the arithmetic of the
// update and rounded to the storage type as a single step stores it; they are
// then summed in the order of pulled_moments, so sampling t+1 here gives the
// same bits as sampling the stored state t+1.
template <typename S>
__device__ __forceinline__ void moments_next(const Geometry &g, const S *__restrict__ A,
                                             const typename Store<S>::R *__restrict__ c2f, int x, int y, int z,
                                             typename Store<S>::R &rho, typename Store<S>::R (&J)[3]) {
    using R = typename Store<S>::R;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const long long nc = g.ncell;
    auto dn = [](int v, int n) { return v == 0 ? n - 1 : v - 1; };
    auto up = [](int v, int n) { return v == n - 1 ? 0 : v + 1; };
    auto post = [&](int i, int cx, int cy, int cz) -> R {  // f*_i(cx, cy, cz) at t+1
        const long long row = ((long long)cz * ny + cy) * nx;
        const R f0 = Store<S>::get(A + row + cx);
        const R fpx = Store<S>::get(A + nc + row + dn(cx, nx));
        const R fmx = Store<S>::get(A + 2 * nc + row + up(cx, nx));
        const R fpy = Store<S>::get(A + 3 * nc + ((long long)cz * ny + dn(cy, ny)) * nx + cx);
        const R fmy = Store<S>::get(A + 4 * nc + ((long long)cz * ny + up(cy, ny)) * nx + cx);
        const R fpz = Store<S>::get(A + 5 * nc + ((long long)dn(cz, nz) * ny + cy) * nx + cx);
        const R fmz = Store<S>::get(A + 6 * nc + ((long long)up(cz, nz) * ny + cy) * nx + cx);
        R o[7];
        collide7(c2f[row + cx], f0, fpx, fmx, fpy, fmy, fpz, fmz, o);
        return Vec<S>::rounded(o[i]);
    };
    const R f0 = post(0, x, y, z);
    const R fpx = post(1, dn(x, nx), y, z);
    const R fmx = post(2, up(x, nx), y, z);
    const R fpy = post(3, x, dn(y, ny), z);
    const R fmy = post(4, x, up(y, ny), z);
    const R fpz = post(5, x, y, dn(z, nz));
    const R fmz = post(6, x, y, up(z, nz));
    rho = f0 + fpx + fmx + fpy + fmy;
    J[0] = fpx - fmx;
    J[1] = fpy - fmy;
    rho += fpz + fmz;
    J[2] = fpz - fmz;
}

// Surface sums of the two steps of a launch (times t and t+1), in the order
// two single steps add them; reads only A, before the two-step kernel runs.
template <typename S>
__global__ void __launch_bounds__(256) sample_two(SampleArgs<S> a, const S *__restrict__ A,
                                                  const typename Store<S>::R *__restrict__ c2f) {
    using R = typename Store<S>::R;
    const int lane = threadIdx.x & 31;
    const int k = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (k >= a.g.n_surface) return;  // uniform per warp
    sample_point_with(a, k, lane, [&](int x, int y, int z, R &rho, R(&J)[3]) {
        pulled_moments(a.g, A, x, y, z, rho, J);
    });
    sample_point_with(a, k, lane, [&](int x, int y, int z, R &rho, R(&J)[3]) {
        moments_next(a.g, A, c2f, x, y, z, rho, J);
    });
}

// One lattice as a two-step CTA sees it.
template <typename S>
struct SlabParams {
    const S *A;  // state t
    S *B;        // state t + 2
    const uint8_t *cls, *band_rows;
    const typename Store<S>::R *c2f;
    int nx, ny, nz;
    long long ncell;
    typename Store<S>::R c0sq, cpsq;
    int H, nslab, zc, nseg;  // plan
    int ntile, tx;           // x-tiles per row and their width in cells (ntile = 1: whole rows)
    int producer;            // whole rows: 1 = warp nseg * (H + 2) only stages planes, 0 = warp 0 also computes
    int c2_staged;           // whole rows, kernels with C2 = 0: 1 = band rows' c^2 staged in shared memory,
                             // 0 = read from global memory (prefetched into L2 with the plane's copies)
    int *err;
};

// The sweep of CTA `cta` of a lattice (slab cta % nslab, z-chunk cta / nslab)
// in the dynamic shared memory `smem`.  Block-uniform control flow.  C2 = 1:
// band rows' c^2 staged in shared memory (fixed at compile time); C2 = 0:
// P.c2_staged chooses at run time between that and S1 reading c^2 from
// global memory, where the staging warp prefetched it into L2 two planes
// ahead.  The plans that read from L2 launch the C2 = 0 form: at 512^3 FP32
// (4-row slabs) it took 1174 us per launch against 1202 us for a form
// compiled for L2 reads only (same registers; the compiler schedules the
// sweep differently).
template <typename S, int CH, bool FULL, int C2>
__device__ __forceinline__ void slab_body(const SlabParams<S> &P, int cta, unsigned char *smem) {
    // rows of nx = V * W cells, V 16-byte vectors, split into nseg segments
    // of up to 32 * CH vectors (the last one may be shorter; FULL: none is)
    using R = typename Store<S>::R;
    constexpr int W = Store<S>::W;
    const S *__restrict__ A = P.A;
    S *__restrict__ B = P.B;
    const uint8_t *__restrict__ cls = P.cls;
    const uint8_t *__restrict__ band_rows = P.band_rows;
    const R *__restrict__ c2f = P.c2f;
    const int nx = P.nx, ny = P.ny, nz = P.nz, H = P.H, nslab = P.nslab, zc = P.zc, nseg = P.nseg;
    const long long ncell = P.ncell;
    const R c0sq = P.c0sq, cpsq = P.cpsq;
    int *err = P.err;
    const int rmax = H + 2;
    const size_t rowel = (size_t)nx;
    const bool c2_staged = C2 == 1 || P.c2_staged != 0;
    // the layout of whole_row_smem
    S *stage = reinterpret_cast<S *>(smem);                                          // [kStages][7][rmax][nx]
    R *c2s = reinterpret_cast<R *>(stage + (size_t)kStages * 7 * rmax * rowel);      // [kStages][rmax][nx] or none
    uint8_t *clss = reinterpret_cast<uint8_t *>(c2s + (c2_staged ? (size_t)kStages * rmax * rowel : 0));
    S *ring = reinterpret_cast<S *>(clss + (size_t)kStages * rmax * rowel);         // [kRingPlanes][2][H][nx]
    R *edge = reinterpret_cast<R *>(ring + (size_t)kRingPlanes * 2 * H * rowel);     // [kRingPlanes][rmax][nseg][2]
    uint64_t *bar = reinterpret_cast<uint64_t *>(edge + (size_t)kRingPlanes * rmax * nseg * 2);  // [kStages]
    uint8_t *rowflag = reinterpret_cast<uint8_t *>(bar + kStages);  // [kStages][rmax]: row holds band cells

    const int slab = cta % nslab, chunk = cta / nslab;
    const int y0 = slab * H;
    const int hs = min(H, ny - y0);  // rows of this slab
    const int rs = hs + 2;           // S1 rows
    const int za = chunk * zc, zb = min(nz, za + zc);
    if (za >= zb) return;            // whole block: empty chunk
    const int L = zb - za + 2;       // S1 planes za-1 .. zb
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int issuer = P.producer ? nseg * rmax : 0;  // the warp that stages planes (a dedicated one computes nothing)
    const uint32_t row_bytes = (uint32_t)(nx * sizeof(S)), c2_bytes = (uint32_t)(nx * sizeof(R));

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) bar_init(&bar[s]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // Band flag of S1 row `lane` of plane index k (warp 0): whether its c^2
    // row must be staged.  Loaded one plane before it is needed.
    auto band_flag = [&](int k) -> int {
        if (lane >= rs) return 0;
        const int p = (za - 1 + k + nz) % nz;
        return band_rows[(long long)p * ny + (y0 - 1 + lane + ny) % ny];
    };
    // Stage the rows of S1 plane index k (plane za-1+k) into stage k % 2:
    // lane i < 8 of the issuing warp copies population i (i = 7: the class bytes) for
    // the rs rows, one bulk copy per run of rows that is contiguous in memory
    // (two where the slab's halo wraps around y); lane 8 + r copies the c^2 row
    // of S1 row r when that row holds band cells (flag), or without c^2
    // staging prefetches it into L2 for S1's own loads two planes later.
    auto issue = [&](int k, int flag) {
        const unsigned band = __ballot_sync(kFull, flag != 0);
        const int p = (za - 1 + k + nz) % nz;
        const int buf = k % kStages;
        if (lane < rs) rowflag[buf * rmax + lane] = flag != 0;  // read by S1 after a barrier
        if (lane == 0)
            bar_expect(&bar[buf], (uint32_t)rs * (7u * row_bytes + (uint32_t)nx) +
                                      (c2_staged ? (uint32_t)__popc(band) * c2_bytes : 0u));
        __syncwarp();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier reads of the stage
        if (lane < 8) {
            const int i = lane;
            const int dy = i == 3 ? -1 : (i == 4 ? 1 : 0);       // +y pulls from y-1, -y from y+1
            const int pp = i == 5 ? (p + nz - 1) % nz : (i == 6 ? (p + 1) % nz : p);
            const int ys = ((y0 - 1 + dy) % ny + ny) % ny;        // source row of S1 row 0
            for (int r = 0; r < rs;) {
                const int yr = (ys + r) % ny;
                const int len = min(rs - r, ny - yr);
                const long long row0 = (long long)pp * ny + yr;
                if (i == 7)
                    bulk_load(clss + ((size_t)buf * rmax + r) * rowel, cls + row0 * nx, (uint32_t)len * nx, &bar[buf]);
                else
                    bulk_load(stage + ((size_t)(buf * 7 + i) * rmax + r) * rowel, A + (long long)i * ncell + row0 * nx,
                              (uint32_t)len * row_bytes, &bar[buf]);
                r += len;
            }
        } else if (lane - 8 < rs && ((band >> (lane - 8)) & 1u)) {
            const int r = lane - 8;
            const long long row0 = (long long)p * ny + (y0 - 1 + r + ny) % ny;
            if (c2_staged)
                bulk_load(c2s + ((size_t)buf * rmax + r) * rowel, c2f + row0 * nx, c2_bytes, &bar[buf]);
            else
                bulk_prefetch_l2(c2f + row0 * nx, c2_bytes);
        }
    };
    int flag_next = 0;  // issuing warp: band flag of plane index k + kStages, for the issue in iteration k
    if (warp == issuer) {
        for (int j = 0; j < kStages && j < L; ++j) issue(j, band_flag(j));
        flag_next = band_flag(kStages);
    }
    __syncthreads();  // row flags of the first stages

    // warp -> S1 row `row` of the slab (y0-1+row) and segment `seg` of it
    // (cells xs .. xs + 32*W*CH - 1); a dedicated staging warp gets row rmax
    // and computes nothing
    const int row = warp / nseg, seg = warp % nseg;
    const int xs = seg * 32 * W * CH;
    const int vg = FULL ? 32 * CH : min(32 * CH, nx / W - seg * 32 * CH);  // vectors of this segment
    const bool whole = nseg == 1 && vg == 32 * CH;  // one full warp per row: x wraps by shuffles
    bool act[CH];                                   // slot holds cells
#pragma unroll
    for (int c = 0; c < CH; ++c) act[c] = FULL || c * 32 + lane < vg;
    const bool s1_row = row < rs;
    const bool s2_row = row >= 1 && row <= hs;
    const int y = (y0 - 1 + row + ny) % ny;
    // registers carried between planes (S1 results in storage precision)
    R n0[CH][W], n1[CH][W], n2[CH][W];  // rest, +x, -x of plane p-1
    R pz0[CH][W], pz1[CH][W];           // +z of planes p-2, p-1
    R cq[CH][W];                        // c^2 of plane p-1
    int failed = 0;
    int k = 0;
    for (; k < L; ++k) {
        const int p = (za - 1 + k + nz) % nz;
        const int buf = k % kStages;
        const bool ok = bar_wait(&bar[buf], (uint32_t)((k / kStages) & 1));
        R c0v[CH][W], c1v[CH][W], c2v[CH][W], c5v[CH][W], c6v[CH][W];
        R cs[CH][W];
        if (s1_row) {
            const S *st = stage + ((size_t)buf * 7 * rmax + row) * rowel;
            // c^2 row of band rows: staged, or in global memory (L2)
            const R *cst = c2_staged ? c2s + ((size_t)buf * rmax + row) * rowel : c2f + ((long long)p * ny + y) * nx;
            const uint8_t *clt = clss + ((size_t)buf * rmax + row) * rowel;
            const bool band_row = rowflag[buf * rmax + row] != 0;  // warp-uniform
            R f[7][CH][W];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int x0 = xs + (c * 32 + lane) * W;
                if (act[c]) {
#pragma unroll
                    for (int i = 0; i < 7; ++i) Vec<S>::ld(st + (size_t)i * rmax * rowel + x0, f[i][c]);
                } else {
#pragma unroll
                    for (int i = 0; i < 7; ++i)
#pragma unroll
                        for (int e = 0; e < W; ++e) f[i][c][e] = R(0);
                }
                // the c^2 the one-step kernels use for the class; a row without
                // interface-band cells holds only fluid and object cells
                const unsigned long long cl = act[c] ? load_classes<W>(clt + x0) : 0ull;
                if (band_row) {
                    R cv[W];
                    if constexpr (C2 == 1) {
#pragma unroll
                        for (int e = 0; e < W; ++e) cv[e] = act[c] ? cst[x0 + e] : c0sq;
                    } else {
                        if (act[c]) load_row_vec<W>(cst + x0, cv);
                    }
#pragma unroll
                    for (int e = 0; e < W; ++e) {
                        const unsigned kc = (unsigned)(cl >> (8 * e)) & 0xffu;
                        cs[c][e] = kc == CELL_FLUID ? c0sq : (kc == CELL_OBJECT ? cpsq : (act[c] ? cv[e] : c0sq));
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < W; ++e)
                        cs[c][e] = ((unsigned)(cl >> (8 * e)) & 0xffu) == CELL_FLUID ? c0sq : cpsq;
                }
            }
            // ends of the segment from the staged row (periodic in x)
            R left = R(0), right = R(0);
            if (!whole) {
                left = Vec<S>::get(st + (size_t)1 * rmax * rowel + (xs + nx - 1) % nx);
                right = Vec<S>::get(st + (size_t)2 * rmax * rowel + (xs + vg * W) % nx);
            }
            R fpx[CH][W], fmx[CH][W];
            shift_x<R, CH, W>(f[1], f[2], lane, vg, whole, left, right, fpx, fmx);
            // ring plane k: +y of rows 0 .. H-1, then -y of rows 2 .. H+1
            S *ry = ring + (size_t)(k % kRingPlanes) * 2 * H * rowel;
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int x0 = xs + (c * 32 + lane) * W;
                R o[7][W];
#pragma unroll
                for (int e = 0; e < W; ++e) {
                    R t[7];
                    collide7(cs[c][e], f[0][c][e], fpx[c][e], fmx[c][e], f[3][c][e], f[4][c][e], f[5][c][e],
                             f[6][c][e], t);
#pragma unroll
                    for (int i = 0; i < 7; ++i) o[i][e] = t[i];
                }
                Vec<S>::rounded(o[0], c0v[c]);
                Vec<S>::rounded(o[1], c1v[c]);
                Vec<S>::rounded(o[2], c2v[c]);
                Vec<S>::rounded(o[5], c5v[c]);
                Vec<S>::rounded(o[6], c6v[c]);
                const R (&oy)[W] = o[3];
                const R (&omy)[W] = o[4];
                if (act[c]) {
                    if (row < hs) Vec<S>::st(ry + (size_t)row * rowel + x0, oy);                // +y, S2 of row + 1
                    if (row >= 2) Vec<S>::st(ry + (size_t)(H + row - 2) * rowel + x0, omy);  // -y, S2 of row - 1
                }
            }
            // the segment's end values for the neighbouring segments' S2
            if (!whole) {
                R *ed = edge + ((size_t)(k % kRingPlanes) * rmax + row) * nseg * 2 + seg * 2;
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    if (c * 32 + lane == vg - 1) ed[0] = c1v[c][W - 1];  // +x at the last cell
                if (lane == 0) ed[1] = c2v[0][0];                        // -x at the first cell
            }
        }
        // stage `buf` consumed, ring plane k written; any failed wait ends the sweep
        if (__syncthreads_or(!ok)) {
            failed = 1;
            break;
        }
        if (warp == issuer && k + kStages < L) {
            issue(k + kStages, flag_next);
            flag_next = band_flag(k + kStages + 1);  // used in the next iteration
        }
        if (k >= 2 && s2_row) {
            const int q = (p + nz - 1) % nz;
            const long long r0 = ((long long)q * ny + y) * nx;
            const S *ry = ring + (size_t)((k - 1) % kRingPlanes) * 2 * H * rowel;
            R left = R(0), right = R(0);
            if (!whole) {
                const R *ed = edge + ((size_t)((k - 1) % kRingPlanes) * rmax + row) * nseg * 2;
                left = ed[((seg + nseg - 1) % nseg) * 2];  // +x at the previous segment's last cell
                right = ed[((seg + 1) % nseg) * 2 + 1];    // -x at the next segment's first cell
            }
            R fpx[CH][W], fmx[CH][W];
            shift_x<R, CH, W>(n1, n2, lane, vg, whole, left, right, fpx, fmx);
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                if (!act[c]) continue;
                const int x0 = xs + (c * 32 + lane) * W;
                R fpy[W], fmy[W];
                Vec<S>::ld(ry + (size_t)(row - 1) * rowel + x0, fpy);      // +y of row w-1
                Vec<S>::ld(ry + (size_t)(H + row - 1) * rowel + x0, fmy);  // -y of row w+1
                R o[7][W];
#pragma unroll
                for (int e = 0; e < W; ++e) {
                    R t[7];
                    collide7(cq[c][e], n0[c][e], fpx[c][e], fmx[c][e], fpy[e], fmy[e], pz0[c][e], c6v[c][e], t);
#pragma unroll
                    for (int i = 0; i < 7; ++i) o[i][e] = t[i];
                }
#pragma unroll
                for (int i = 0; i < 7; ++i) Store<S>::store(B + i * ncell + r0 + x0, o[i]);
            }
        }
        if (s1_row) {
#pragma unroll
            for (int c = 0; c < CH; ++c) {
#pragma unroll
                for (int e = 0; e < W; ++e) {
                    cq[c][e] = cs[c][e];
                    n0[c][e] = c0v[c][e];
                    n1[c][e] = c1v[c][e];
                    n2[c][e] = c2v[c][e];
                    pz0[c][e] = pz1[c][e];
                    pz1[c][e] = c5v[c][e];
                }
            }
        }
    }
    if (failed && threadIdx.x == 0) {
        atomicExch(err, 2);  // reported as WLB_ERR_TIMEOUT
        // let the copies still in flight (stages k .. k + kStages - 1) land before exit
        for (int j = k; j < k + kStages && j < L; ++j) bar_wait(&bar[j % kStages], (uint32_t)((j / kStages) & 1));
    }
}

// 16-byte asynchronous copy global -> shared by one thread (both 16-byte
// aligned), its commit and the wait for all but the newest N groups.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr(dst)), "l"(__cvta_generic_to_global(src))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The x-tiled sweep of CTA `cta`: x-tile cta % ntile (cells xa .. xa+tw-1 of
// every row), slab c % nslab and z-chunk c / nslab of c = cta / ntile.  One
// warp per S1 row (a tile row is at most 32 * CH vectors), so a warp reads
// only the staged row it stages itself: each lane copies its 16-byte vectors
// of the row, the tile plus one vector of populations (and of c^2, and 16
// class bytes) on either side, wrapped around x at the row's ends, with
// cp.async two planes ahead (one commit group per plane), and waits for its
// own groups.  The block barrier per plane is the +-y exchange's.  S1 also
// runs on the halo cells x = xa - 1 (lane 0; its +x value is S2's pull into
// xa) and x = xb (the lane holding the row's last vector; its -x value is
// S2's pull into xb - 1), kept in those lanes' registers until S2 of the
// plane.  Arithmetic as in slab_body, so results are bit-identical.
template <typename S, int CH, bool FULL>
__device__ __forceinline__ void slab_body_tiled(const SlabParams<S> &P, int cta, unsigned char *smem) {
    using R = typename Store<S>::R;
    constexpr int W = Store<S>::W;
    constexpr int HP = halo_pop<S>();  // halo cells per side: populations (one vector),
    constexpr int HQ = halo_c2<S>();   // c^2 (one vector),
    constexpr int HC = kHaloCls;       // class bytes (one vector)
    static_assert(HP == W && HQ == 16 / (int)sizeof(R), "one 16-byte vector on either side");
    constexpr int QW = 16 / (int)sizeof(R);                // c^2 values per 16-byte vector
    constexpr int NJ = (32 * CH + 2 + 31) / 32;            // population vectors per lane and row, at most
    constexpr int NQ = (32 * CH * W / QW + 2 + 31) / 32;   // c^2 vectors per lane and row, at most
    const S *__restrict__ A = P.A;
    S *__restrict__ B = P.B;
    const uint8_t *__restrict__ cls = P.cls;
    const uint8_t *__restrict__ band_rows = P.band_rows;
    const R *__restrict__ c2f = P.c2f;
    const int nx = P.nx, ny = P.ny, nz = P.nz, H = P.H, nslab = P.nslab, zc = P.zc, ntile = P.ntile, tx = P.tx;
    const long long ncell = P.ncell;
    const R c0sq = P.c0sq, cpsq = P.cpsq;
    const int rmax = H + 2;
    const int tile = cta % ntile, ct = cta / ntile;
    const int slab = ct % nslab, chunk = ct / nslab;
    const int xa = tile * tx, tw = min(tx, nx - xa);
    const size_t pit_s = (size_t)tx + 2 * HP, pit_q = (size_t)tx + 2 * HQ, pit_c = (size_t)tx + 2 * HC;
    S *stage = reinterpret_cast<S *>(smem);                                          // [kStages][7][rmax][pit_s]
    R *c2s = reinterpret_cast<R *>(stage + (size_t)kStages * 7 * rmax * pit_s);      // [kStages][rmax][pit_q]
    uint8_t *clss = reinterpret_cast<uint8_t *>(c2s + (size_t)kStages * rmax * pit_q);  // [kStages][rmax][pit_c]
    S *ring = reinterpret_cast<S *>(clss + (size_t)kStages * rmax * pit_c);         // [kRingPlanes][2][rmax][tx]

    const int y0 = slab * H;
    const int hs = min(H, ny - y0);  // rows of this slab
    const int rs = hs + 2;           // S1 rows
    const int za = chunk * zc, zb = min(nz, za + zc);
    if (za >= zb) return;            // whole block: empty chunk
    const int L = zb - za + 2;       // S1 planes za-1 .. zb
    const int row = threadIdx.x >> 5, lane = threadIdx.x & 31;  // warp = S1 row y0-1+row
    const bool s1_row = row < rs;
    const bool s2_row = row >= 1 && row <= hs;
    const int y = (y0 - 1 + row + ny) % ny;
    const int vg = FULL ? 32 * CH : min(32 * CH, tw / W);  // vectors of the tile row
    const int rl = (vg - 1) & 31;                          // lane holding its last vector
    bool act[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) act[c] = FULL || c * 32 + lane < vg;

    // this lane's staging vectors: v = lane + 32 j of the row (v = 0 and the
    // last one are the halo vectors), as wrapped global x of their first cell
    auto wrapx = [&](int x) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); };
    const int nv_s = tw / W + 2, nv_q = tw / QW + 2, nv_c = tw / 16 + 2;
    int gs[NJ], gq[NQ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int v = lane + 32 * j;
        gs[j] = v < nv_s ? wrapx(xa - HP + v * W) : -1;
    }
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
        const int v = lane + 32 * j;
        gq[j] = v < nv_q ? wrapx(xa - HQ + v * QW) : -1;
    }
    const int gc = lane < nv_c ? wrapx(xa - HC + lane * 16) : -1;
    auto band_flag = [&](int k) -> int {
        if (k >= L) return 0;
        return band_rows[(long long)((za - 1 + k + nz) % nz) * ny + y];
    };
    // stage this warp's S1 row of plane index k (plane za-1+k) into stage k % 2
    auto stage_row = [&](int k, int flag) {
        const int p = (za - 1 + k + nz) % nz;
        const int buf = k % kStages;
        S *dst0 = stage + ((size_t)buf * 7 * rmax + row) * pit_s;
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            const int dy = i == 3 ? -1 : (i == 4 ? 1 : 0);  // +y pulls from y-1, -y from y+1
            const int pp = i == 5 ? (p + nz - 1) % nz : (i == 6 ? (p + 1) % nz : p);
            const S *src = A + (long long)i * ncell + ((long long)pp * ny + (y + dy + ny) % ny) * nx;
            S *dst = dst0 + (size_t)i * rmax * pit_s;
#pragma unroll
            for (int j = 0; j < NJ; ++j)
                if (gs[j] >= 0) cp_async16(dst + (size_t)(lane + 32 * j) * W, src + gs[j]);
        }
        const long long rowp = ((long long)p * ny + y) * nx;
        if (gc >= 0) cp_async16(clss + ((size_t)buf * rmax + row) * pit_c + (size_t)lane * 16, cls + rowp + gc);
        if (flag) {
            R *dq = c2s + ((size_t)buf * rmax + row) * pit_q;
#pragma unroll
            for (int j = 0; j < NQ; ++j)
                if (gq[j] >= 0) cp_async16(dq + (size_t)(lane + 32 * j) * QW, c2f + rowp + gq[j]);
        }
        cp_async_commit();
    };

    // band flags of the staged planes k, k + 1 and of plane k + 2 (next issue)
    int f0 = 0, f1 = 0, fn = 0;
    if (s1_row) {
        f0 = band_flag(0);
        f1 = band_flag(1);
        stage_row(0, f0);
        stage_row(1, f1);  // L >= 3
        fn = band_flag(2);
    }
    // registers carried between planes (S1 results in storage precision)
    R n0[CH][W], n1[CH][W], n2[CH][W];  // rest, +x, -x of plane p-1
    R pz0[CH][W], pz1[CH][W];           // +z of planes p-2, p-1
    R cq[CH][W];                        // c^2 of plane p-1
    R hl = R(0), hr = R(0);             // +x at xa - 1 (lane 0), -x at xb (lane rl) of plane p-1
    for (int k = 0; k < L; ++k) {
        const int p = (za - 1 + k + nz) % nz;
        const int buf = k % kStages;
        R c0v[CH][W], c1v[CH][W], c2v[CH][W], c5v[CH][W], c6v[CH][W];
        R cs[CH][W];
        R hl_new = R(0), hr_new = R(0);
        if (s1_row) {
            cp_async_wait<1>();  // this lane's copies of stage k (the newest group is stage k + 1)
            __syncwarp();        // and the other lanes'
            // staged row of population 0 (population i at + i * pst), indexed
            // by tile cell (halo cells at -HP .. -1 and tw .. tw+HP-1)
            const S *st = stage + ((size_t)buf * 7 * rmax + row) * pit_s + HP;
            const R *cst = c2s + ((size_t)buf * rmax + row) * pit_q + HQ;
            const uint8_t *clt = clss + ((size_t)buf * rmax + row) * pit_c + HC;
            const size_t pst = (size_t)rmax * pit_s;
            const bool band_row = f0 != 0;  // warp-uniform
            R f[7][CH][W];
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int x0 = (c * 32 + lane) * W;
                if (act[c]) {
#pragma unroll
                    for (int i = 0; i < 7; ++i) Vec<S>::ld(st + (size_t)i * pst + x0, f[i][c]);
                } else {
#pragma unroll
                    for (int i = 0; i < 7; ++i)
#pragma unroll
                        for (int e = 0; e < W; ++e) f[i][c][e] = R(0);
                }
                const unsigned long long cl = act[c] ? load_classes<W>(clt + x0) : 0ull;
                if (band_row) {
#pragma unroll
                    for (int e = 0; e < W; ++e) {
                        const unsigned kc = (unsigned)(cl >> (8 * e)) & 0xffu;
                        cs[c][e] = kc == CELL_FLUID ? c0sq : (kc == CELL_OBJECT ? cpsq : (act[c] ? cst[x0 + e] : c0sq));
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < W; ++e)
                        cs[c][e] = ((unsigned)(cl >> (8 * e)) & 0xffu) == CELL_FLUID ? c0sq : cpsq;
                }
            }
            // the tile's ends pull from the staged halo cells
            const R left = Vec<S>::get(st + pst - 1);        // +x at xa - 1
            const R right = Vec<S>::get(st + 2 * pst + tw);  // -x at xb
            R fpx[CH][W], fmx[CH][W];
            shift_x<R, CH, W>(f[1], f[2], lane, vg, false, left, right, fpx, fmx);
            S *ry = ring + ((size_t)(k % kRingPlanes) * 2 * rmax + row) * tx;
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int x0 = (c * 32 + lane) * W;
                R o[7][W];
#pragma unroll
                for (int e = 0; e < W; ++e) {
                    R t[7];
                    collide7(cs[c][e], f[0][c][e], fpx[c][e], fmx[c][e], f[3][c][e], f[4][c][e], f[5][c][e],
                             f[6][c][e], t);
#pragma unroll
                    for (int i = 0; i < 7; ++i) o[i][e] = t[i];
                }
                Vec<S>::rounded(o[0], c0v[c]);
                Vec<S>::rounded(o[1], c1v[c]);
                Vec<S>::rounded(o[2], c2v[c]);
                Vec<S>::rounded(o[5], c5v[c]);
                Vec<S>::rounded(o[6], c6v[c]);
                const R (&oy)[W] = o[3];
                const R (&omy)[W] = o[4];
                if (act[c]) {
                    Vec<S>::st(ry + x0, oy);                          // +y of row w
                    Vec<S>::st(ry + (size_t)rmax * tx + x0, omy);     // -y of row w
                }
            }
            // S1 on the halo cells x = -1 and x = tw
            auto halo = [&](int x, int out) -> R {
                const unsigned kc = clt[x];
                const R c2h = kc == CELL_FLUID ? c0sq : (kc == CELL_OBJECT ? cpsq : cst[x]);
                R t[7];
                collide7(c2h, Vec<S>::get(st + x), Vec<S>::get(st + pst + x - 1), Vec<S>::get(st + 2 * pst + x + 1),
                         Vec<S>::get(st + 3 * pst + x), Vec<S>::get(st + 4 * pst + x), Vec<S>::get(st + 5 * pst + x),
                         Vec<S>::get(st + 6 * pst + x), t);
                return Vec<S>::rounded(t[out]);
            };
            if (lane == 0) hl_new = halo(-1, 1);
            if (lane == rl) hr_new = halo(tw, 2);
            __syncwarp();  // every lane is done with stage k before it is refilled
            if (k + 2 < L)
                stage_row(k + 2, fn);
            else
                cp_async_commit();  // an empty group keeps one group per plane
            f0 = f1;
            f1 = fn;
            fn = band_flag(k + 3);
        }
        __syncthreads();  // ring plane k written
        if (k >= 2 && s2_row) {
            const int q = (p + nz - 1) % nz;
            const long long r0 = ((long long)q * ny + y) * nx + xa;
            const S *ry = ring + (size_t)((k - 1) % kRingPlanes) * 2 * rmax * tx;
            R fpx[CH][W], fmx[CH][W];
            shift_x<R, CH, W>(n1, n2, lane, vg, false, hl, hr, fpx, fmx);
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                if (!act[c]) continue;
                const int x0 = (c * 32 + lane) * W;
                R fpy[W], fmy[W];
                Vec<S>::ld(ry + (size_t)(row - 1) * tx + x0, fpy);             // +y of row w-1
                Vec<S>::ld(ry + (size_t)(rmax + row + 1) * tx + x0, fmy);      // -y of row w+1
                R o[7][W];
#pragma unroll
                for (int e = 0; e < W; ++e) {
                    R t[7];
                    collide7(cq[c][e], n0[c][e], fpx[c][e], fmx[c][e], fpy[e], fmy[e], pz0[c][e], c6v[c][e], t);
#pragma unroll
                    for (int i = 0; i < 7; ++i) o[i][e] = t[i];
                }
#pragma unroll
                for (int i = 0; i < 7; ++i) Store<S>::store(B + i * ncell + r0 + x0, o[i]);
            }
        }
        if (s1_row) {
#pragma unroll
            for (int c = 0; c < CH; ++c) {
#pragma unroll
                for (int e = 0; e < W; ++e) {
                    cq[c][e] = cs[c][e];
                    n0[c][e] = c0v[c][e];
                    n1[c][e] = c1v[c][e];
                    n2[c][e] = c2v[c][e];
                    pz0[c][e] = pz1[c][e];
                    pz1[c][e] = c5v[c][e];
                }
            }
            hl = hl_new;
            hr = hr_new;
        }
    }
    cp_async_wait<0>();
}

template <typename S, int CH, bool FULL, bool TILED, int C2>
__global__ void __launch_bounds__(two_step_threads<S, CH>(), 1) update2_slab(SlabParams<S> P) {
    extern __shared__ __align__(128) unsigned char smem[];
    if constexpr (TILED)
        slab_body_tiled<S, CH, FULL>(P, blockIdx.x, smem);  // stages c^2 itself
    else
        slab_body<S, CH, FULL, C2>(P, blockIdx.x, smem);
}

// Batched ensembles: CTA j sweeps CTA j - cta_first[i] of lattice
// i = cta_lat[j] (each lattice with its own plan), skipping lattices past
// their n_steps; j = cta_base + blockIdx.x (one launch per lane-layout group).
// Every launch is two steps, so the state at step t is in buffer (t / 2) & 1.
// In the last group's launch (advance) the last CTA to finish advances the
// step: every CTA of every group has read it by then.
template <typename S, int CH, bool FULL>
__global__ void __launch_bounds__(two_step_threads<S, CH>(), 1)
    batch_update2(const BatchLat *__restrict__ lats, const int *__restrict__ cta_lat,
                  const int *__restrict__ cta_first, int cta_base, int advance, long long *step, unsigned *done) {
    using R = typename Store<S>::R;
    extern __shared__ __align__(128) unsigned char smem[];
    const long long t = *step;
    const int j = cta_base + (int)blockIdx.x;
    const int i = cta_lat[j];
    const BatchLat &L = lats[i];
    if (t < L.n_steps) {  // block-uniform
        const int src = (int)((t >> 1) & 1);
        SlabParams<S> P;
        P.A = (const S *)L.b.pop[src];
        P.B = (S *)L.b.pop[src ^ 1];
        P.cls = L.b.cls;
        P.band_rows = L.b.band_rows;
        P.c2f = (const R *)L.b.c2;
        P.nx = L.g.n[0];
        P.ny = L.g.n[1];
        P.nz = L.g.n[2];
        P.ncell = L.g.ncell;
        P.c0sq = (R)(L.g.c0 * L.g.c0);
        P.cpsq = (R)(L.g.cp * L.g.cp);
        P.H = L.plan.H;
        P.nslab = L.plan.nslab;
        P.zc = L.plan.zc;
        P.nseg = L.plan.nseg;
        P.ntile = 1;
        P.tx = P.nx;
        P.producer = L.plan.producer;
        P.c2_staged = 1;
        P.err = L.b.err;
        slab_body<S, CH, FULL, 1>(P, j - cta_first[i], smem);
    }
    if (!advance) return;
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

// Batched sampling of both steps of a launch: grid-stride over all points;
// warps of lattices outside their window skip.  Sums of t (stored state) and
// t+1 (recomputed, moments_next) in that order, then the period fold by the
// point's lane 0 when t+1 closes a period (periods and windows are even).
template <typename S>
__global__ void __launch_bounds__(256) batch_sample_two(const BatchLat *__restrict__ lats,
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
        const S *A = (const S *)L.b.pop[(t >> 1) & 1];
        const R *st_w = (const R *)L.b.st_w, *nrm = (const R *)L.b.nrm;
        R *accs = (R *)L.b.acc;
        sample_point_with(L.g, L.b.st_xyz, st_w, nrm, accs, k, lane, [&](int x, int y, int z, R &rho, R(&J)[3]) {
            pulled_moments(L.g, A, x, y, z, rho, J);
        });
        sample_point_with(L.g, L.b.st_xyz, st_w, nrm, accs, k, lane, [&](int x, int y, int z, R &rho, R(&J)[3]) {
            moments_next(L.g, A, (const R *)L.b.c2, x, y, z, rho, J);
        });
        if (lane == 0 && (t + 2 - L.window_begin) % L.period == 0) {
            const double scale = 1.0 / (L.g.pop_scale * L.g.pop_scale);
            R *acc = accs + 5 * (long long)k;
            double *a64 = L.b.acc64 + 5 * (long long)k;
            bool bad = false;
            for (int j = 0; j < 5; ++j) {
                const double v = fold_value(a64[j], (double)acc[j], scale);
                a64[j] = v;
                acc[j] = R(0);
                bad |= !isfinite(v);
            }
            if (bad) atomicExch(L.b.err, 1);
        }
    }
}

// ---------------------------------------------------------------- host side: plans and launches

// 16-byte vectors in a row, or 0 if a row is not a whole number of them or
// its class bytes are not a whole number of 16-byte units (bulk copies).
template <typename S>
int row_vectors(const Geometry &g) {
    constexpr int W = Store<S>::W;
    return (g.n[0] % W || g.n[0] % 16) ? 0 : g.n[0] / W;
}

// Chunks per lane for a row of V vectors: two where whole warps of two fill
// the row and fit the registers (mode 3 asks for two), else one (mode 2).
template <typename S>
int chunks_for(int V, int mode) {
    const bool two_fit = Store<S>::W * 2 <= 8 && V % 64 == 0;
    if (mode == 2) return 1;
    if (mode == 3) return Store<S>::W * 2 <= 8 ? 2 : 0;
    return two_fit ? 2 : 1;
}

// Tile width for ntile x-tiles of a row of nx cells (multiple of 16 cells,
// the last tile possibly narrower; ntile = 1: the whole row).
inline int tile_width(int nx, int ntile) { return ntile <= 1 ? nx : ((nx + ntile - 1) / ntile + 15) / 16 * 16; }

// The kernel of a plan: x-tiles or whole rows, full warps or not, and for
// whole rows c^2 staged (C2 = 1) or read from L2 (C2 = 0, P.c2_staged = 0).
template <typename S, int CH>
void (*slab_kernel(const TwoStepPlan &pl))(SlabParams<S>) {
    if (pl.ntile > 1) return pl.full ? update2_slab<S, CH, true, true, 1> : update2_slab<S, CH, false, true, 1>;
    if (pl.c2_staged) return pl.full ? update2_slab<S, CH, true, false, 1> : update2_slab<S, CH, false, false, 1>;
    return pl.full ? update2_slab<S, CH, true, false, 0> : update2_slab<S, CH, false, false, 0>;
}

// Whether a whole-row slab of H rows fits `smem_max` bytes, and with c^2
// staged or not: c2 = 0 stages it where it fits, 1 always, 2 never.
// Returns 1 (staged), 0 (not staged) or -1 (does not fit).
template <typename S>
int whole_row_fit(int nx, int nseg, int H, int c2, int smem_max) {
    if (c2 != 2 && whole_row_smem<S>(nx, nseg, H, true) <= (size_t)smem_max) return 1;
    if (c2 != 1 && whole_row_smem<S>(nx, nseg, H, false) <= (size_t)smem_max) return 0;
    return -1;
}

// Slab height H (rows <= smem and thread limits; `want` > 0 asks for one)
// and the z-chunk count minimising the estimated time, one CTA per SM, for
// rows split into `ntile` x-tiles (1: whole rows).  FP32: waves x planes per
// CTA x cells moved per plane (H + 2 staged rows read with their halo, H
// written); FP16 storage, whose planes cost a CTA mostly a fixed latency:
// waves x planes.  Among heights within 5 % of the best estimate the tallest
// is taken.  *cost gets the estimate of the chosen plan, *hmax the tallest
// slab that fits (either may be null).  c2: c^2 staging of whole rows
// (whole_row_fit).
template <typename S, int CH>
cudaError_t plan_ch(const Geometry &g, int want, int ntile, int staging, int c2, TwoStepPlan *pl, double *cost,
                    int *hmax) {
    using R = typename Store<S>::R;
    constexpr int W = Store<S>::W;
    int dev = 0, sms = 0, smem_max = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const bool tiled = ntile > 1;
    const int tx = tile_width(nx, ntile);
    const int tiles = (nx + tx - 1) / tx;
    if (tiled && (tiles < 2 || tx < 16)) return cudaErrorInvalidValue;
    const int nseg = (tx / W + 32 * CH - 1) / (32 * CH);
    if (tiled && nseg != 1) return cudaErrorInvalidValue;  // a tile row is one warp
    // whole rows: a dedicated staging warp on request (tiles stage per warp)
    const int producer = !tiled && staging == 2 ? 1 : 0;
    const size_t per_tile_row = tiled ? smem_per_tile_row<S>(tx) : 0;
    const size_t fixed = kStages * sizeof(uint64_t) + kStages * (size_t)kMaxRows + 16;
    int rows = std::min((two_step_threads<S, CH>() / 32 - producer) / nseg, kMaxRows);
    if (tiled)
        rows = std::min(rows, (int)(((size_t)smem_max - fixed) / per_tile_row));
    else
        while (rows >= 3 && whole_row_fit<S>(nx, nseg, rows - 2, c2, smem_max) < 0) --rows;
    if (rows < 3) return cudaErrorInvalidValue;
    if (hmax) *hmax = rows - 2;
    const int h_lo = want > 0 ? want : 1, h_hi = want > 0 ? want : rows - 2;
    if (h_hi > rows - 2) return cudaErrorInvalidValue;
    const int hp = tiled ? halo_pop<S>() : 0;
    TwoStepPlan per_h[kMaxRows];
    double cost_h[kMaxRows], best = -1;
    for (int H = h_lo; H <= h_hi; ++H) {
        const int nslab = (ny + H - 1) / H;
        cost_h[H] = -1;
        for (int C = 1; C <= nz; ++C) {
            const int zc = (nz + C - 1) / C;
            const int used = (nz + zc - 1) / zc;
            const long long waves = ((long long)tiles * nslab * used + sms - 1) / sms;
            // FP32: time follows the cells moved per plane; FP16 storage halves
            // the bytes and a plane's fixed latency dominates: count planes
            const double moved = (double)(H + 2) * (tx + 2 * hp) + (double)H * tx;
            const double c = sizeof(S) == 2 ? (double)waves * (zc + 2) : (double)waves * (zc + 2) * moved;
            if (cost_h[H] < 0 || c < cost_h[H]) {
                cost_h[H] = c;
                per_h[H].H = H;
                per_h[H].nslab = nslab;
                per_h[H].chunks = used;
                per_h[H].zc = zc;
            }
        }
        if (best < 0 || cost_h[H] < best) best = cost_h[H];
    }
    for (int H = h_hi; H >= h_lo; --H)
        if (cost_h[H] <= best * 1.05) {
            *pl = per_h[H];
            if (cost) *cost = cost_h[H];
            break;
        }
    pl->nseg = nseg;
    pl->chunks_per_lane = CH;
    pl->ntile = tiles;
    pl->tx = tx;
    pl->producer = producer;
    pl->threads = 32 * (nseg * (pl->H + 2) + producer);
    if (tiled) {
        pl->c2_staged = 1;
        pl->smem = per_tile_row * (pl->H + 2) + fixed;
    } else {
        pl->c2_staged = whole_row_fit<S>(nx, nseg, pl->H, c2, smem_max);
        pl->smem = whole_row_smem<S>(nx, nseg, pl->H, pl->c2_staged != 0);
    }
    const int last = nx - (tiles - 1) * tx;  // cells of the last tile
    pl->full = (tx / W) % (32 * CH) == 0 && (last / W) % (32 * CH) == 0;
    // the attribute belongs to the kernel, shared by every handle: allow the
    // device's whole opt-in shared memory, not just this plan's
    return cudaFuncSetAttribute(slab_kernel<S, CH>(*pl), cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
}

// Chunks per lane and segments per row for `mode` (1: automatic, 2: one
// chunk, 3: two) and x-tiles (0: automatic, 1: whole rows, n: n tiles), then
// the slab plan.  Automatic tiles: whole rows wherever a whole-row slab fits
// the shared memory (they are faster: at 512^3 FP32, 3-row whole-row slabs
// take 1254 us per launch against 1410 us for 4 tiles of 14-row slabs);
// rows too long for that take the cheapest estimate of 2 .. 16 tiles.
template <typename S>
cudaError_t plan_for(const Geometry &g, int want, int mode, int tiles, int staging, int c2, TwoStepPlan *pl) {
    constexpr int W = Store<S>::W;
    if (!row_vectors<S>(g)) return cudaErrorInvalidValue;
    auto one_c2 = [&](int nt, int c2v, TwoStepPlan *out, double *cost) -> cudaError_t {
        const int tx = tile_width(g.n[0], nt);
        if (nt > 1 && (g.n[0] + tx - 1) / tx < 2) return cudaErrorInvalidValue;
        // a tile row is one warp: two chunks per lane where one does not cover it
        const int ch = (nt > 1 && mode == 1 && tx / W > 32) ? (Store<S>::W * 2 <= 8 ? 2 : 0) : chunks_for<S>(tx / W, mode);
        if (!ch) return cudaErrorInvalidValue;
        if (ch == 1) return plan_ch<S, 1>(g, want, nt, staging, c2v, out, cost, nullptr);
        if constexpr (Store<S>::W * 2 <= 8) return plan_ch<S, 2>(g, want, nt, staging, c2v, out, cost, nullptr);
        return cudaErrorInvalidValue;
    };
    // Automatic c^2 staging of whole rows: staged, unless reading it from L2
    // lets a slab of lower estimated cost fit (512-cell FP32 rows: 4-row slabs
    // against 3, 1170 against 1238 us per launch).  Where the staged plan is
    // as cheap, a taller unstaged one is not taken (256^3 FP32: 7-row staged
    // slabs 150 us, 9-row unstaged 190 us).
    auto one = [&](int nt, TwoStepPlan *out, double *cost) -> cudaError_t {
        if (nt > 1 || c2 != 0) return one_c2(nt, c2, out, cost);
        TwoStepPlan ps, pa;
        double cs = 0, ca = 0;
        const cudaError_t es = one_c2(nt, 1, &ps, &cs);
        const cudaError_t ea = one_c2(nt, 0, &pa, &ca);
        if (es != cudaSuccess && ea != cudaSuccess) return ea;
        const bool staged = es == cudaSuccess && (ea != cudaSuccess || cs <= ca);
        *out = staged ? ps : pa;
        if (cost) *cost = staged ? cs : ca;
        return cudaSuccess;
    };
    if (tiles >= 1 && staging != 0) return one(tiles, pl, nullptr);
    if (tiles > 1) return one(tiles, pl, nullptr);
    // whole rows; a dedicated staging warp unless the thread limit then costs
    // slab height worth more than 3 % of the recomputed halo rows (measured:
    // 256^3 FP32 7 rows either way, 153.8 -> 149.7 us; 256^3 FP16 10 -> 9
    // rows, 114.2 -> 104.9 us; 512^3 FP16 4 -> 3 rows, 953.6 -> 1027.6 us)
    TwoStepPlan p0, p1;
    cudaError_t e_whole = one(1, &p0, nullptr);
    if (e_whole == cudaSuccess && staging == 0) {
        staging = 2;
        if (one(1, &p1, nullptr) == cudaSuccess &&
            (double)(p1.H + 2) / p1.H <= 1.03 * (double)(p0.H + 2) / p0.H)
            p0 = p1;
        staging = 0;
    }
    if (e_whole == cudaSuccess) {
        *pl = p0;
        return e_whole;
    }
    if (tiles == 1) return e_whole;
    TwoStepPlan best;
    double best_cost = -1;
    for (int nt : {2, 4, 8, 16}) {
        TwoStepPlan c;
        double cost = 0;
        if (one(nt, &c, &cost) != cudaSuccess) continue;
        if (best_cost < 0 || cost < best_cost) {
            best = c;
            best_cost = cost;
        }
    }
    if (best_cost < 0) return e_whole;
    *pl = best;
    return cudaSuccess;
}

// The sampling kernel runs in 128-thread blocks so that one fits on an SM
// beside a two-step CTA (registers), and on the SMs the grid leaves free.
template <typename S>
SlabParams<S> slab_params(const Geometry &g, const Buffers &b, const TwoStepPlan &pl, int src, int *err) {
    using R = typename Store<S>::R;
    SlabParams<S> P;
    P.A = (const S *)b.pop[src];
    P.B = (S *)b.pop[src ^ 1];
    P.cls = b.cls;
    P.band_rows = b.band_rows;
    P.c2f = (const R *)b.c2;
    P.nx = g.n[0];
    P.ny = g.n[1];
    P.nz = g.n[2];
    P.ncell = g.ncell;
    P.c0sq = (R)(g.c0 * g.c0);
    P.cpsq = (R)(g.cp * g.cp);
    P.H = pl.H;
    P.nslab = pl.nslab;
    P.zc = pl.zc;
    P.nseg = pl.nseg;
    P.ntile = pl.ntile;
    P.tx = pl.tx;
    P.producer = pl.producer;
    P.c2_staged = pl.c2_staged;
    P.err = err;
    return P;
}

template <typename S, int CH>
cudaError_t launch_ch(const Geometry &g, const Buffers &b, const TwoStepPlan &pl, int src, bool sample, int *err,
                      cudaStream_t s, const SideStream &side) {
    using R = typename Store<S>::R;
    const bool fork = sample && g.n_surface > 0 && side.stream;
    cudaError_t e = cudaSuccess;
    if (fork) {
        e = cudaEventRecord(side.fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side.stream, side.fork, 0);
        if (e != cudaSuccess) return e;
    }
    if (sample && g.n_surface > 0) {
        const long long blocks = ((long long)g.n_surface * 32 + 127) / 128;
        sample_two<S><<<(unsigned)blocks, 128, 0, fork ? side.stream : s>>>(sample_args<S>(g, b),
                                                                            (const S *)b.pop[src], (const R *)b.c2);
        e = cudaGetLastError();
        if (e == cudaSuccess && fork) e = cudaEventRecord(side.join, side.stream);
        if (e != cudaSuccess) return e;
    }
    slab_kernel<S, CH>(pl)<<<pl.ntile * pl.nslab * pl.chunks, pl.threads, pl.smem, s>>>(
        slab_params<S>(g, b, pl, src, err));
    e = cudaGetLastError();
    if (e == cudaSuccess && fork) e = cudaStreamWaitEvent(s, side.join, 0);  // the next launch overwrites src
    return e;
}

template <typename S>
cudaError_t launch_for(const Geometry &g, const Buffers &b, const TwoStepPlan &pl, int src, bool sample, int *err,
                       cudaStream_t s, const SideStream &side) {
    if (pl.chunks_per_lane == 1) return launch_ch<S, 1>(g, b, pl, src, sample, err, s, side);
    if constexpr (Store<S>::W * 2 <= 8)
        if (pl.chunks_per_lane == 2) return launch_ch<S, 2>(g, b, pl, src, sample, err, s, side);
    return cudaErrorInvalidValue;
}

}  // namespace

bool two_step_supported(const Geometry &g, Prec p) {
    if (g.dim != 3 || g.driven) return false;
    TwoStepPlan probe;
    switch (p) {
        case Prec::F16: return row_vectors<__half>(g) > 0 && plan_for<__half>(g, 0, 1, 0, 0, 0, &probe) == cudaSuccess;
        case Prec::F32: return row_vectors<float>(g) > 0 && plan_for<float>(g, 0, 1, 0, 0, 0, &probe) == cudaSuccess;
        default: return false;
    }
}

cudaError_t plan_two_steps(const Geometry &g, Prec p, int slab_rows, int mode, int tiles, int staging, int c2,
                           TwoStepPlan *out) {
    TwoStepPlan pl;
    if (g.dim != 3 || g.driven || (p != Prec::F16 && p != Prec::F32)) return cudaErrorInvalidValue;
    cudaError_t e = p == Prec::F16 ? plan_for<__half>(g, slab_rows, mode, tiles, staging, c2, &pl)
                                   : plan_for<float>(g, slab_rows, mode, tiles, staging, c2, &pl);
    if (e == cudaSuccess) *out = pl;
    return e;
}

// Two steps from buffer src into src ^ 1, sampling both when asked.
cudaError_t launch_two_steps(const Geometry &g, const Buffers &b, Prec p, const TwoStepPlan &pl, int src, bool sample,
                             int *err, cudaStream_t s, const SideStream &side) {
    if (!pl.H) return cudaErrorInvalidValue;
    switch (p) {
        case Prec::F16: return launch_for<__half>(g, b, pl, src, sample, err, s, side);
        case Prec::F32: return launch_for<float>(g, b, pl, src, sample, err, s, side);
        default: return cudaErrorInvalidValue;
    }
}

namespace {

// Each lattice's lane layout: one 16-byte chunk per lane for rows of up to
// 32 vectors, two (FP32) for wider rows, so that a row of up to 64 vectors is
// one warp and the slab can be taller; lattices are grouped by it.
template <typename S, int CH>
bool plan_group(BatchLat *lats, const std::vector<int> &members, int smem_max, const BatchTwoKnobs &kn,
                BatchTwoGroup *grp) {
    int t_max = 0;
    size_t s_max = 0;
    bool all_full = true;
    for (int i : members) {
        const Geometry &g = lats[i].g;
        const int V = row_vectors<S>(g);
        const int nseg = (V + 32 * CH - 1) / (32 * CH);
        TwoStepPlan pl;
        pl.producer = kn.staging_warp ? 1 : 0;
        int rows = std::min((two_step_threads<S, CH>() / 32 - pl.producer) / nseg, kMaxRows);
        // batches stage c^2 (batch_update2 has no other variant)
        while (rows >= 3 && whole_row_fit<S>(g.n[0], nseg, rows - 2, 1, smem_max) < 0) --rows;
        if (rows < 3) return false;
        pl.H = std::min(rows - 2, g.n[1]);
        if (kn.h_cap > 0) pl.H = std::min(pl.H, kn.h_cap);
        pl.nslab = (g.n[1] + pl.H - 1) / pl.H;
        // z-chunks of about zc_target planes: many CTAs of similar work across lattices
        const int zt = std::max(1, kn.zc_target);
        pl.chunks = (g.n[2] + zt - 1) / zt;
        pl.zc = (g.n[2] + pl.chunks - 1) / pl.chunks;
        pl.chunks = (g.n[2] + pl.zc - 1) / pl.zc;
        pl.nseg = nseg;
        pl.chunks_per_lane = CH;
        pl.threads = 32 * (nseg * (pl.H + 2) + pl.producer);
        pl.c2_staged = 1;
        pl.smem = whole_row_smem<S>(g.n[0], nseg, pl.H, true);
        pl.full = V % (32 * CH) == 0;
        lats[i].plan = pl;
        t_max = std::max(t_max, pl.threads);
        s_max = std::max(s_max, pl.smem);
        all_full = all_full && pl.full;
    }
    // shared by every batch: the device's whole opt-in shared memory
    cudaError_t e = all_full ? cudaFuncSetAttribute(batch_update2<S, CH, true>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max)
                             : cudaFuncSetAttribute(batch_update2<S, CH, false>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    if (e != cudaSuccess) return false;
    grp->ch = CH;
    grp->threads = t_max;
    grp->smem = s_max;
    grp->full = all_full;
    return true;
}

template <typename S>
bool plan_batch_for(BatchLat *lats, int count, const BatchTwoKnobs &kn, BatchTwoGroup *groups, int *ngroups) {
    int dev = 0, smem_max = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return false;
    std::vector<int> one, two;
    for (int i = 0; i < count; ++i) {
        const Geometry &g = lats[i].g;
        const int V = row_vectors<S>(g);
        if (g.dim != 3 || g.driven || !V) return false;
        if (Store<S>::W * 2 <= 8 && V > 32 && !kn.one_chunk) two.push_back(i);
        else one.push_back(i);
    }
    int n = 0;
    if (!one.empty()) {
        if (!plan_group<S, 1>(lats, one, smem_max, kn, &groups[n])) return false;
        ++n;
    }
    if constexpr (Store<S>::W * 2 <= 8)
        if (!two.empty()) {
            if (!plan_group<S, 2>(lats, two, smem_max, kn, &groups[n])) return false;
            ++n;
        }
    *ngroups = n;
    return true;
}

// The groups' launches after the sampling launch: one after the other on s,
// the last one advancing the step; or, with a side stream and two groups,
// side by side (the second on the side stream, forked and joined by events),
// neither advancing it, and then a one-thread launch on s advances it once
// every CTA of both has read it.
template <typename S>
cudaError_t launch_batch_for(const BatchTwoGroup *groups, int ngroups, const BatchLat *lats, const int *cta_lat,
                             const int *cta_first, const int *pt_lat, const long long *pt_begin,
                             long long total_points, long long *step, unsigned *done, int sample_grid,
                             cudaStream_t s, const SideStream &side) {
    cudaError_t e = cudaSuccess;
    if (total_points > 0) {
        batch_sample_two<S><<<sample_grid, 256, 0, s>>>(lats, pt_lat, pt_begin, total_points, step);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const bool fork = ngroups > 1 && side.stream;
    if (fork) {
        if ((e = cudaEventRecord(side.fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side.stream, side.fork, 0)) != cudaSuccess) return e;
    }
    for (int k = 0; k < ngroups; ++k) {
        const BatchTwoGroup &G = groups[k];
        const int adv = !fork && k == ngroups - 1;
        cudaStream_t sk = fork && k > 0 ? side.stream : s;
        if (G.ch == 1) {
            auto kernel = G.full ? batch_update2<S, 1, true> : batch_update2<S, 1, false>;
            kernel<<<G.ctas, G.threads, G.smem, sk>>>(lats, cta_lat, cta_first, G.cta_begin, adv, step, done);
        } else if constexpr (Store<S>::W * 2 <= 8) {
            auto kernel = G.full ? batch_update2<S, 2, true> : batch_update2<S, 2, false>;
            kernel<<<G.ctas, G.threads, G.smem, sk>>>(lats, cta_lat, cta_first, G.cta_begin, adv, step, done);
        } else {
            return cudaErrorInvalidValue;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (fork) {
        if ((e = cudaEventRecord(side.join, side.stream)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(s, side.join, 0)) != cudaSuccess) return e;
        e = launch_batch_advance(step, s);
    }
    return e;
}

}  // namespace

bool plan_batch_two_steps(Prec p, BatchLat *lats, int count, const BatchTwoKnobs &kn, BatchTwoGroup *groups,
                          int *ngroups) {
    switch (p) {
        case Prec::F16: return plan_batch_for<__half>(lats, count, kn, groups, ngroups);
        case Prec::F32: return plan_batch_for<float>(lats, count, kn, groups, ngroups);
        default: return false;
    }
}

cudaError_t launch_batch_two_steps(Prec p, const BatchTwoGroup *groups, int ngroups, const BatchLat *lats,
                                   const int *cta_lat, const int *cta_first, const int *pt_lat,
                                   const long long *pt_begin, long long total_points, long long *step,
                                   unsigned *done, int sample_grid, cudaStream_t s, const SideStream &side) {
    switch (p) {
        case Prec::F16:
            return launch_batch_for<__half>(groups, ngroups, lats, cta_lat, cta_first, pt_lat, pt_begin,
                                            total_points, step, done, sample_grid, s, side);
        case Prec::F32:
            return launch_batch_for<float>(groups, ngroups, lats, cta_lat, cta_first, pt_lat, pt_begin,
                                           total_points, step, done, sample_grid, s, side);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace wlb
