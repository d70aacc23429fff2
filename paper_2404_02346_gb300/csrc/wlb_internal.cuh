// Internal declarations shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace wlb {

// Cell classes (the byte field read by the update kernel).
enum : uint8_t { CELL_FLUID = 0, CELL_OBJECT = 1, CELL_BAND = 2, CELL_WALL_LO = 3, CELL_WALL_HI = 4, CELL_SOURCE = 5 };

// Population storage: FP32, FP64, or FP16 of f / p_a with FP32 arithmetic.
enum class Prec { F32, F64, F16 };

// Bytes of one stored population value and of one "real" value (sound speed,
// weights, running sums) for a storage precision.
inline size_t pop_bytes(Prec p) { return p == Prec::F64 ? 8 : (p == Prec::F32 ? 4 : 2); }
inline size_t real_bytes(Prec p) { return p == Prec::F64 ? 8 : 4; }

// Problem description as the kernels see it (passed by value).
struct Geometry {
    int dim, q;            // 2 or 3; 5 or 7
    int n[3];              // nx, ny, nz
    long long ncell;       // nx*ny*nz
    int wave_axis;
    double c0, cp, rho0;
    double p_a, wavelength, antinode;
    double center[3];
    double radius, interface_d, surface_radius;
    double band_half;      // class threshold on |x-r0|^2 - R^2 (20 d)
    double pop_scale;      // stored populations are f * pop_scale (1, or 1/p_a for FP16)
    int driven;            // 1: driven walls along wave_axis (Sec. VII)
    double wall_damping, source_amplitude;
    long long period;      // T = lambda / c0 steps
    int n_periods;         // run length in periods (sizes the force history)
    int n_surface;
    int stencil;           // 3^dim
};

// Device buffers carved from one workspace.
struct Buffers {
    void *pop[2];          // populations, q * ncell stored values each
    uint8_t *cls;          // ncell
    uint8_t *band_rows;    // ny * nz: 1 where row (y, z) holds an interface-band cell
    void *c2;              // ncell reals: sound speed squared (read for band cells)
    double *pts;           // n_surface * 7
    int4 *st_xyz;          // n_surface * stencil: wrapped cell coordinates
    void *st_w;            // n_surface * stencil * 2 reals: (delta c^2, delta / rho0)
    void *nrm;             // n_surface * 4 reals: normal (x, y, z, 0)
    void *acc;             // n_surface * 5 reals: running sums within a period
    double *acc64;         // n_surface * 5: folded sums
    double *force;         // 4 doubles
    double *hist;          // history_capacity x 4: after each fold, the force numerator of the sums
                           // folded so far (Eq. 14 with 1 / N_w = 1) and the samples that fold added
    double *hist_tmp;      // 4 doubles: the entry being recorded
    unsigned long long *hist_n;  // entries recorded (may exceed the capacity; the excess is dropped)
    int *err;              // 1 int: non-finite accumulator seen
    double *ptab;          // n[wave_axis]: incident pressure along the wave axis (setup)
    double *stage;         // stage_cells * (1 + dim): field read-back staging
    long long stage_cells;
};

// Launchers (each TU owns its kernels).  All return cudaGetLastError().
cudaError_t launch_setup(const Geometry &g, const Buffers &b, Prec p, cudaStream_t s);
// t_mod: step index modulo the period (phase of the driven source).
cudaError_t launch_update(const Geometry &g, const Buffers &b, Prec p, int src, long long t_mod, cudaStream_t s,
                          bool *vector_path);
cudaError_t launch_sample(const Geometry &g, const Buffers &b, Prec p, int src, cudaStream_t s);
// One whole step: the update, plus the surface sampling of the same input when
// sample is set (fused into the update launch on the row-vectorised path).
cudaError_t launch_step(const Geometry &g, const Buffers &b, Prec p, int src, bool sample, long long t_mod,
                        cudaStream_t s);
cudaError_t launch_fold(const Geometry &g, const Buffers &b, Prec p, cudaStream_t s);
cudaError_t launch_force(const Geometry &g, const Buffers &b, double n_window, cudaStream_t s);
// After a fold that added `samples` samples: append the force numerator of the
// folded sums and that count to the history (wlb_history.cu).
cudaError_t launch_record_fold(const Geometry &g, const Buffers &b, long long samples, cudaStream_t s);
// History entries kept: every full period of the run plus one partial fold.
inline long long history_capacity(const Geometry &g) { return (g.n_periods > 1 ? g.n_periods : 1) + 1; }
cudaError_t launch_fields(const Geometry &g, const Buffers &b, Prec p, int src,
                          long long first_cell, long long count, cudaStream_t s);
bool update_is_vectorised(const Geometry &g, Prec p);

// Two steps per launch (wlb_two_step.cu): 3D, periodic, FP32 or FP16 rows
// that are whole numbers of warp-wide 16-byte vectors, split into nseg
// segments of one warp each.  Slab height H, slabs and z-chunks of the grid,
// segments per row (per x-tile when rows are split into ntile tiles of tx
// cells), chunks per lane, block size and dynamic shared memory.
struct TwoStepPlan {
    int H = 0, nslab = 0, chunks = 0, zc = 0, nseg = 0, chunks_per_lane = 0, threads = 0;
    int ntile = 1, tx = 0;  // x-tiles per row and their width (1: whole rows)
    int producer = 0;       // whole rows: 1 = a dedicated warp stages the planes
    int c2_staged = 1;      // whole rows: 1 = band rows' c^2 staged in shared memory, 0 = read from L2
    bool full = false;      // every segment a full warp (no idle lanes)
    size_t smem = 0;
};
bool two_step_supported(const Geometry &g, Prec p);
// slab_rows: 0 picks H; otherwise that H.  mode: 1 automatic, 2 one 16-byte
// chunk per lane, 3 two.  tiles: 0 automatic, 1 whole rows, n >= 2 n x-tiles
// per row.  staging: 0 automatic, 1 warp 0 stages planes besides computing,
// 2 a dedicated staging warp.  c2 (whole rows): 0 stages band rows' c^2 in
// shared memory where the slab still fits, 1 always, 2 never (S1 reads it
// from global memory, prefetched into L2).  Also opts the kernel into the
// shared memory it needs on the current device.
cudaError_t plan_two_steps(const Geometry &g, Prec p, int slab_rows, int mode, int tiles, int staging, int c2,
                           TwoStepPlan *out);
// Side stream and events that let the sampling kernel of a sampled two-step
// launch run beside the update (fork before, join after).
struct SideStream {
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
// From buffer src into src ^ 1; with sample, the surface sums of both steps
// are accumulated too by a sampling kernel that reads only src, forked onto
// side.stream and joined back into s after the update is enqueued (on s
// itself when side.stream is null).
cudaError_t launch_two_steps(const Geometry &g, const Buffers &b, Prec p, const TwoStepPlan &pl, int src, bool sample,
                             int *err, cudaStream_t s, const SideStream &side);

// One lattice of a batched ensemble (wlb_batch.cu): geometry, buffers, its
// protocol lengths and, when the batch runs two steps per launch, its plan.
struct BatchLat {
    Geometry g;
    Buffers b;
    long long n_steps, window_begin, period;
    TwoStepPlan plan;
};

// Batched two steps per launch (3D): lattices are grouped by lane layout
// (chunks per lane), one launch of the slab kernel per group.
struct BatchTwoGroup {
    int ch = 1;              // 16-byte chunks per lane
    bool full = false;       // every row of the group made of full warps
    int threads = 0;         // block size of the group's launch
    size_t smem = 0;         // its dynamic shared memory
    int cta_begin = 0, ctas = 0;  // its range of the CTA -> lattice table
};
// Choices of a batched two-step plan (the autotuner tries several):
// z-chunks of about zc_target planes, slab heights capped at h_cap (0: the
// tallest that fits), one_chunk: one 16-byte chunk per lane for every lattice
// (rows over 32 vectors then take several warps) instead of two for wide rows;
// staging_warp: a dedicated warp per CTA stages the planes.
struct BatchTwoKnobs {
    int zc_target = 32, h_cap = 0, one_chunk = 0, staging_warp = 0;
    int rows_2d = 0;  // 2D: rows per warp chunk (0: chosen to fill whole waves)
};
// Plans every lattice (its plan lands in lats[i].plan) and fills up to two
// groups (cta_begin / ctas are left to the caller); false if some lattice
// cannot take two steps per launch.
bool plan_batch_two_steps(Prec p, BatchLat *lats, int count, const BatchTwoKnobs &kn, BatchTwoGroup *groups,
                          int *ngroups);
// One launch of two steps for every active lattice: CTA j of the table works
// on lattice cta_lat[j] (its CTA j - cta_first[lattice]); with points, a
// sampling launch before it adds the sums of both steps.  The state at step t
// is in buffer (t / 2) & 1; the last CTA of all groups to finish advances
// *step by 2.  With two groups and side.stream set, the second group runs on
// side.stream beside the first (forked after the sampling launch, joined back
// into s), so each group's partly filled last wave overlaps the other group.
cudaError_t launch_batch_two_steps(Prec p, const BatchTwoGroup *groups, int ngroups, const BatchLat *lats,
                                   const int *cta_lat, const int *cta_first, const int *pt_lat,
                                   const long long *pt_begin, long long total_points, long long *step,
                                   unsigned *done, int sample_grid, cudaStream_t s, const SideStream &side);
// *step += 2 by one thread on s (wlb_batch.cu): the batched step's advance
// when its groups ran side by side.
cudaError_t launch_batch_advance(long long *step, cudaStream_t s);

// Two steps per launch for a single 2D lattice (wlb_two_step_2d.cu): periodic,
// rows of at most two 16-byte chunks (8 values) per lane; each warp sweeps a
// chunk of plan.zc rows (plan.chunks chunks).  From buffer src into src ^ 1;
// with sample, a sampling kernel before the update adds both steps' sums.
bool two_step_2d_supported(const Geometry &g, Prec p);
cudaError_t plan_two_steps_2d(const Geometry &g, Prec p, TwoStepPlan *out);
cudaError_t launch_two_steps_2d(const Geometry &g, const Buffers &b, Prec p, const TwoStepPlan &pl, int src,
                                bool sample, cudaStream_t s);

// The same for batches of 2D lattices (wlb_two_step_2d.cu): a warp sweeps a
// chunk of rows of one lattice.  Plans every lattice (plan.zc rows per chunk,
// plan.chunks chunks; rows > 0 fixes plan.zc, else it is chosen to fill whole
// waves), returns the number of warps, the chunks per lane and the length of
// the widest row; false if some lattice cannot take it.
bool plan_batch2d_two_steps(Prec p, BatchLat *lats, int count, int rows, int *tasks, int *chunks_per_lane,
                            int *nx_max);
cudaError_t launch_batch2d_two_steps(Prec p, int chunks_per_lane, int nx_max, const BatchLat *lats, const int *task_lat,
                                     const int *task_first, int total_tasks, const int *pt_lat,
                                     const long long *pt_begin, long long total_points, long long *step,
                                     unsigned *done, int sample_grid, cudaStream_t s);

}  // namespace wlb
