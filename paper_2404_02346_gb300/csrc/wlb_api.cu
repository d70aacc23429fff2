// Host side of the C ABI declared in include/wlb.h: parameter validation,
// workspace layout, the step loop (per-period CUDA graphs) and read-back.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <thread>

#include "../../include/wlb.h"
#include "wlb_internal.cuh"
#include "wlb_handle.cuh"

using wlb::Buffers;
using wlb::Geometry;

namespace {

constexpr long long kStageCells = 1LL << 20;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

wlb_status fail(wlb_handle *h, wlb_status s, const char *what, cudaError_t e = cudaSuccess) {
    if (h) {
        if (e != cudaSuccess)
            snprintf(h->err, sizeof(h->err), "%s: %s", what, cudaGetErrorString(e));
        else
            snprintf(h->err, sizeof(h->err), "%s", what);
    }
    return s;
}

#define WLB_CUDA(h, call, what)                                   \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return fail((h), WLB_ERR_CUDA, (what), e_); \
    } while (0)

int dim_of(const wlb_params *p) { return p->lattice == WLB_D2Q5 ? 2 : 3; }

bool whole(double v) { return std::isfinite(v) && v > 0 && std::fabs(v - std::nearbyint(v)) < 1e-9 * std::fmax(1.0, v); }

}  // namespace

namespace wlb {

Geometry make_geometry(const wlb_params *p) {
    Geometry g{};
    g.dim = dim_of(p);
    g.q = 2 * g.dim + 1;
    g.n[0] = p->nx;
    g.n[1] = p->ny;
    g.n[2] = p->nz;
    g.ncell = (long long)p->nx * p->ny * p->nz;
    g.wave_axis = p->wave_axis;
    g.c0 = p->c0;
    g.cp = p->cp;
    g.rho0 = p->rho0;
    g.p_a = p->p_a;
    g.wavelength = p->wavelength;
    g.antinode = p->antinode;
    for (int a = 0; a < 3; ++a) g.center[a] = a < g.dim ? p->center[a] : 0.0;
    g.radius = p->radius;
    g.interface_d = p->interface_d;
    g.surface_radius = p->surface_radius;
    g.band_half = 20.0 * p->interface_d;
    g.pop_scale = p->precision == WLB_POP_F16 ? 1.0 / p->p_a : 1.0;
    g.driven = p->boundary == WLB_BOUNDARY_DRIVEN ? 1 : 0;
    g.wall_damping = p->wall_damping;
    g.source_amplitude = p->source_amplitude;
    g.period = (long long)std::nearbyint(p->wavelength / p->c0);
    g.n_periods = p->n_periods;
    g.n_surface = p->n_surface;
    g.stencil = g.dim == 3 ? 27 : 9;
    return g;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

Prec prec_of(const wlb_params *p) {
    return p->precision == WLB_POP_F64 ? wlb::Prec::F64
                                       : (p->precision == WLB_POP_F16 ? wlb::Prec::F16 : wlb::Prec::F32);
}

// Carve the workspace; with base == nullptr only the size is computed.
size_t layout(const Geometry &g, Prec prec, char *base, Buffers *b) {
    const size_t P = wlb::pop_bytes(prec), T = wlb::real_bytes(prec);
    const size_t nc = (size_t)g.ncell, N = (size_t)g.n_surface, S = (size_t)g.stencil;
    size_t off = 0;
    auto take = [&](size_t bytes) -> void * {
        void *ptr = base ? base + off : nullptr;
        off += align256(bytes ? bytes : 1);
        return ptr;
    };
    Buffers t{};
    t.pop[0] = take(g.q * nc * P);
    t.pop[1] = take(g.q * nc * P);
    t.cls = (uint8_t *)take(nc);
    t.band_rows = (uint8_t *)take((size_t)g.n[1] * g.n[2]);
    t.c2 = take(nc * T);
    t.pts = (double *)take(N * 7 * sizeof(double));
    t.st_xyz = (int4 *)take(N * S * sizeof(int4));
    t.st_w = take(N * S * 2 * T);
    t.nrm = take(N * 4 * T);
    t.acc = take(N * 5 * T);
    t.acc64 = (double *)take(N * 5 * sizeof(double));
    t.force = (double *)take(4 * sizeof(double));
    t.hist = (double *)take((size_t)history_capacity(g) * 4 * sizeof(double));
    t.hist_tmp = (double *)take(4 * sizeof(double));
    t.hist_n = (unsigned long long *)take(sizeof(unsigned long long));
    t.err = (int *)take(sizeof(int));
    t.ptab = (double *)take(sizeof(double) * g.n[g.wave_axis]);
    t.stage_cells = g.ncell < kStageCells ? g.ncell : kStageCells;
    t.stage = (double *)take((size_t)t.stage_cells * (1 + g.dim) * sizeof(double));
    if (b) *b = t;
    return off;
}

}  // namespace wlb

namespace {

using wlb::layout;
using wlb::make_geometry;
using wlb::prec_of;

void destroy_graphs(wlb_handle *h) {
    for (int i = 0; i < 2; ++i) {
        if (h->graph_free[i]) cudaGraphExecDestroy(h->graph_free[i]);
        if (h->graph_sampled[i]) cudaGraphExecDestroy(h->graph_sampled[i]);
        h->graph_free[i] = h->graph_sampled[i] = nullptr;
    }
}

// One launch of two steps from buffer src (3D slab kernel or 2D row sweep).
cudaError_t two_steps(wlb_handle *h, int src, bool sampled, cudaStream_t s) {
    if (h->g.dim == 2) return wlb::launch_two_steps_2d(h->g, h->b, h->prec, h->two_plan, src, sampled, s);
    return wlb::launch_two_steps(h->g, h->b, h->prec, h->two_plan, src, sampled, h->b.err, s, h->side);
}

// Whether, and with which plan, a handle can take two steps per launch.
bool two_step_plan(const wlb_handle *h, int slab_rows, int mode, int tiles, int staging, int c2,
                   wlb::TwoStepPlan *plan, cudaError_t *err) {
    if (h->g.dim == 2) {
        if (!wlb::two_step_2d_supported(h->g, h->prec) || slab_rows != 0 || tiles > 1 || staging == 2 || c2 != 0)
            return false;
        *err = wlb::plan_two_steps_2d(h->g, h->prec, plan);
        return true;
    }
    if (!wlb::two_step_supported(h->g, h->prec)) return false;
    *err = wlb::plan_two_steps(h->g, h->prec, slab_rows, mode, tiles, staging, c2, plan);
    return true;
}

// Update launches in one period: each flips the population buffer.
long long period_launches(const wlb_handle *h, bool) {
    return h->two_step ? h->period / 2 + h->period % 2 : h->period;
}

// Issue one period of steps starting from buffer `start` on stream s.
cudaError_t issue_period(wlb_handle *h, int start, bool sampled, cudaStream_t s) {
    int cur = start;
    long long t = 0;
    if (h->two_step)
        for (; t + 1 < h->period; t += 2) {  // two steps per launch
            cudaError_t e = two_steps(h, cur, sampled, s);
            if (e != cudaSuccess) return e;
            cur ^= 1;
        }
    for (; t < h->period; ++t) {  // graphs start on a period boundary
        cudaError_t e = wlb::launch_step(h->g, h->b, h->prec, cur, sampled, t, s);
        if (e != cudaSuccess) return e;
        cur ^= 1;
    }
    if (sampled) {
        cudaError_t e = wlb::launch_fold(h->g, h->b, h->prec, s);
        return e != cudaSuccess ? e : wlb::launch_record_fold(h->g, h->b, h->period, s);
    }
    return cudaSuccess;
}

wlb_status period_graph(wlb_handle *h, int start, bool sampled, cudaGraphExec_t *out) {
    if (*out) return WLB_OK;
    WLB_CUDA(h, cudaStreamBeginCapture(h->capture, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = issue_period(h, start, sampled, h->capture);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->capture, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(h, WLB_ERR_CUDA, "capture period", e != cudaSuccess ? e : e2);
    }
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        *out = nullptr;
        return fail(h, WLB_ERR_CUDA, "instantiate period graph", e);
    }
    return WLB_OK;
}

}  // namespace

extern "C" {

const char *wlb_status_str(wlb_status s) {
    switch (s) {
        case WLB_OK: return "ok";
        case WLB_ERR_ARG: return "invalid argument";
        case WLB_ERR_UNSTABLE: return "non-finite time averages (unstable run)";
        case WLB_ERR_CUDA: return "CUDA error";
        case WLB_ERR_OOM: return "out of memory or workspace too small";
        case WLB_ERR_STATE: return "call out of order";
        case WLB_ERR_TIMEOUT: return "device wait limit reached";
    }
    return "unknown status";
}

const char *wlb_last_error(const wlb_handle *h) { return h ? h->err : ""; }

wlb_status wlb_validate(const wlb_params *p) {
    if (!p) return WLB_ERR_ARG;
    if (p->lattice != WLB_D2Q5 && p->lattice != WLB_D3Q7) return WLB_ERR_ARG;
    if (p->precision != WLB_POP_F32 && p->precision != WLB_POP_F64 && p->precision != WLB_POP_F16)
        return WLB_ERR_ARG;
    const int D = dim_of(p);
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return WLB_ERR_ARG;
    if (D == 2 && p->nz != 1) return WLB_ERR_ARG;
    if ((long long)p->nx * p->ny * p->nz > (1LL << 40)) return WLB_ERR_ARG;
    if (p->wave_axis < 0 || p->wave_axis >= D) return WLB_ERR_ARG;
    if (!(p->c0 > 0) || !(p->cp > 0) || !(p->rho0 > 0)) return WLB_ERR_ARG;
    if (!(D * p->c0 * p->c0 < 1.0) || !(D * p->cp * p->cp < 1.0)) return WLB_ERR_ARG;
    if (!std::isfinite(p->p_a) || !std::isfinite(p->antinode)) return WLB_ERR_ARG;
    if (p->precision == WLB_POP_F16 && !(p->p_a != 0.0)) return WLB_ERR_ARG;  // storage scale 1/p_a
    if (!(p->wavelength > 0) || !whole(p->wavelength / p->c0)) return WLB_ERR_ARG;
    const int n[3] = {p->nx, p->ny, p->nz};
    if (p->boundary != WLB_BOUNDARY_PERIODIC && p->boundary != WLB_BOUNDARY_DRIVEN) return WLB_ERR_ARG;
    const bool driven = p->boundary == WLB_BOUNDARY_DRIVEN;
    if (!driven && !whole(n[p->wave_axis] / p->wavelength)) return WLB_ERR_ARG;
    if (driven) {
        if (n[p->wave_axis] < 5) return WLB_ERR_ARG;
        if (!(p->wall_damping >= 0.0 && p->wall_damping <= 1.0)) return WLB_ERR_ARG;
        if (!std::isfinite(p->source_amplitude)) return WLB_ERR_ARG;
    }
    if (!(p->radius > 0) || !(p->interface_d > 0) || !(p->surface_radius > 0)) return WLB_ERR_ARG;
    if (p->n_surface < 0 || p->n_periods < 1) return WLB_ERR_ARG;
    if (p->n_avg_periods < 0 || p->n_avg_periods > p->n_periods) return WLB_ERR_ARG;
    // Object, interface band and interpolation stencil inside half the box.
    const double band_r = std::sqrt(p->radius * p->radius + 20.0 * p->interface_d);
    const double reach = std::fmax(band_r, p->surface_radius + 1.5) + 1.0;
    for (int a = 0; a < D; ++a) {
        if (!std::isfinite(p->center[a])) return WLB_ERR_ARG;
        if (2.0 * reach > n[a]) return WLB_ERR_ARG;
    }
    // driven cavity: object, band and stencil clear of the walls and the source sheet
    if (driven && (p->center[p->wave_axis] - reach < 2.0 || p->center[p->wave_axis] + reach > n[p->wave_axis] - 2.0))
        return WLB_ERR_ARG;
    const double T = p->wavelength / p->c0;
    if ((double)p->n_periods * T > 9.0e15) return WLB_ERR_ARG;
    return WLB_OK;
}

wlb_status wlb_workspace_bytes(const wlb_params *p, size_t *bytes) {
    if (!bytes) return WLB_ERR_ARG;
    wlb_status s = wlb_validate(p);
    if (s != WLB_OK) return s;
    *bytes = layout(make_geometry(p), prec_of(p), nullptr, nullptr);
    return WLB_OK;
}

wlb_status wlb_create(const wlb_params *p, void *device_workspace, size_t workspace_bytes, void *stream,
                      wlb_handle **out) {
    if (!out) return WLB_ERR_ARG;
    wlb_status s = wlb_validate(p);
    if (s != WLB_OK) return s;
    if (device_workspace && ((uintptr_t)device_workspace & 255u)) return WLB_ERR_ARG;
    wlb_handle *h = new (std::nothrow) wlb_handle();
    if (!h) return WLB_ERR_OOM;
    h->p = *p;
    h->g = make_geometry(p);
    h->prec = prec_of(p);
    h->stream = (cudaStream_t)stream;
    h->period = (long long)std::nearbyint(p->wavelength / p->c0);
    h->n_steps = h->period * p->n_periods;
    h->n_window = h->period * p->n_avg_periods;
    h->vector_path = wlb::update_is_vectorised(h->g, h->prec);
    const size_t need = layout(h->g, h->prec, nullptr, nullptr);
    char *base = (char *)device_workspace;
    if (base && workspace_bytes < need) {  // checked before any CUDA call
        delete h;
        return WLB_ERR_OOM;
    }
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return WLB_ERR_CUDA;
    }
    if (!base) {
        e = cudaMalloc(&h->owned, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return WLB_ERR_OOM;
        }
        base = (char *)h->owned;
    }
    layout(h->g, h->prec, base, &h->b);
    e = cudaStreamCreateWithFlags(&h->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->side.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->side.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->side.join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&h->host_out, 8 * sizeof(double), cudaHostAllocDefault);
    if (e != cudaSuccess) {
        wlb_destroy(h);
        return WLB_ERR_CUDA;
    }
    // steps two per launch by default on 3D lattices where the kernel applies
    // (bit-identical); a single 2D lattice has too few row chunks to fill the
    // SMs, and one step per launch is faster there
    if (h->g.dim == 3) {
        cudaError_t pe = cudaSuccess;
        if (two_step_plan(h, 0, 1, 0, 0, 0, &h->two_plan, &pe) && pe == cudaSuccess) {
            h->two_step = true;
            h->two_mode = 1;
        }
    }
    cudaGetLastError();
    *out = h;
    return WLB_OK;
}

wlb_status wlb_init(wlb_handle *h) {
    if (!h) return WLB_ERR_ARG;
    DeviceGuard dg(h->device);
    WLB_CUDA(h, wlb::launch_setup(h->g, h->b, h->prec, h->stream), "setup kernels");
    WLB_CUDA(h, cudaMemsetAsync(h->b.hist_n, 0, sizeof(unsigned long long), h->stream), "history reset");
    h->src = 0;
    h->steps_done = h->samples_done = h->samples_in_period = 0;
    h->initialised = true;
    return WLB_OK;
}

wlb_status wlb_step(wlb_handle *h, long long n, int sample) {
    if (!h || n < 0) return WLB_ERR_ARG;
    if (!h->initialised) return fail(h, WLB_ERR_STATE, "wlb_step before wlb_init");
    DeviceGuard dg(h->device);
    const bool sampled = sample != 0 && h->g.n_surface > 0;
    while (n > 0) {
        const bool aligned = !h->g.driven || h->steps_done % h->period == 0;  // source phase
        if (n >= h->period && aligned && (!sampled || h->samples_in_period == 0)) {
            cudaGraphExec_t *slot = sampled ? &h->graph_sampled[h->src] : &h->graph_free[h->src];
            wlb_status st = period_graph(h, h->src, sampled, slot);
            if (st != WLB_OK) return st;
            WLB_CUDA(h, cudaGraphLaunch(*slot, h->stream), "graph launch");
            if (period_launches(h, sampled) & 1) h->src ^= 1;
            h->steps_done += h->period;
            if (sampled) h->samples_done += h->period;
            n -= h->period;
            continue;
        }
        if (h->two_step && n >= 2 && (!sampled || h->samples_in_period + 2 <= h->period)) {
            WLB_CUDA(h, two_steps(h, h->src, sampled, h->stream),
                     "two-step kernels");
            h->src ^= 1;
            h->steps_done += 2;
            n -= 2;
            if (sampled) {
                h->samples_done += 2;
                h->samples_in_period += 2;
                if (h->samples_in_period == h->period) {
                    WLB_CUDA(h, wlb::launch_fold(h->g, h->b, h->prec, h->stream), "fold kernel");
                    WLB_CUDA(h, wlb::launch_record_fold(h->g, h->b, h->period, h->stream), "history kernels");
                    h->samples_in_period = 0;
                }
            }
            continue;
        }
        WLB_CUDA(h, wlb::launch_step(h->g, h->b, h->prec, h->src, sampled, h->steps_done % h->period, h->stream),
                 "step kernels");
        h->src ^= 1;
        h->steps_done += 1;
        if (sampled) {
            h->samples_done += 1;
            if (++h->samples_in_period == h->period) {
                WLB_CUDA(h, wlb::launch_fold(h->g, h->b, h->prec, h->stream), "fold kernel");
                WLB_CUDA(h, wlb::launch_record_fold(h->g, h->b, h->period, h->stream), "history kernels");
                h->samples_in_period = 0;
            }
        }
        n -= 1;
    }
    return WLB_OK;
}

wlb_status wlb_force(wlb_handle *h, double force_out[3]) {
    if (!h || !force_out) return WLB_ERR_ARG;
    if (!h->initialised) return fail(h, WLB_ERR_STATE, "wlb_force before wlb_init");
    DeviceGuard dg(h->device);
    if (h->samples_done == 0 || h->g.n_surface == 0) {
        force_out[0] = force_out[1] = force_out[2] = 0.0;
        WLB_CUDA(h, cudaStreamSynchronize(h->stream), "synchronize");
        return WLB_OK;
    }
    if (h->samples_in_period > 0) {
        WLB_CUDA(h, wlb::launch_fold(h->g, h->b, h->prec, h->stream), "fold kernel");
        WLB_CUDA(h, wlb::launch_record_fold(h->g, h->b, h->samples_in_period, h->stream), "history kernels");
        h->samples_in_period = 0;
    }
    WLB_CUDA(h, wlb::launch_force(h->g, h->b, (double)h->samples_done, h->stream), "force kernel");
    WLB_CUDA(h, cudaMemcpyAsync(h->host_out, h->b.force, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
             "force copy");
    WLB_CUDA(h, cudaMemcpyAsync(h->host_out + 4, h->b.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream),
             "flag copy");
    WLB_CUDA(h, cudaStreamSynchronize(h->stream), "synchronize");
    int flag;
    memcpy(&flag, h->host_out + 4, sizeof(int));
    for (int i = 0; i < 3; ++i) force_out[i] = h->host_out[i];
    if (flag == 2) return fail(h, WLB_ERR_TIMEOUT, "two-step staging wait limit reached");
    if (flag) return fail(h, WLB_ERR_UNSTABLE, "non-finite accumulators");
    return WLB_OK;
}

// Steps of a deadline run: one period per call, at most two periods queued;
// between them the host polls the older period's marker against its clock.
static wlb_status steps_within(wlb_handle *h, long long n, int sample, std::chrono::steady_clock::time_point t0,
                               long long *issued) {
    using clk = std::chrono::steady_clock;
    auto late = [&] { return std::chrono::duration<double>(clk::now() - t0).count() > h->deadline_s; };
    while (n > 0) {
        const long long chunk = n < h->period ? n : h->period;
        wlb_status st = wlb_step(h, chunk, sample);
        if (st != WLB_OK) return st;
        cudaEvent_t mine = h->marks[*issued & 1], older = h->marks[(*issued + 1) & 1];
        WLB_CUDA(h, cudaEventRecord(mine, h->stream), "period marker");
        if (*issued > 0) {
            cudaError_t q;
            while ((q = cudaEventQuery(older)) == cudaErrorNotReady && !late())
                std::this_thread::sleep_for(std::chrono::microseconds(50));
            if (q != cudaSuccess && q != cudaErrorNotReady) return fail(h, WLB_ERR_CUDA, "period marker", q);
        }
        ++*issued;
        n -= chunk;
        if (late()) {
            // what is queued still completes: drain it, keep the handle consistent
            WLB_CUDA(h, cudaStreamSynchronize(h->stream), "synchronize");
            return fail(h, WLB_ERR_TIMEOUT, "wlb_run deadline reached");
        }
    }
    return WLB_OK;
}

wlb_status wlb_run(wlb_handle *h, double force_out[3]) {
    if (!h || !force_out) return WLB_ERR_ARG;
    wlb_status s = wlb_init(h);
    if (h->deadline_s > 0.0) {
        const auto t0 = std::chrono::steady_clock::now();
        long long issued = 0;
        if (s == WLB_OK) s = steps_within(h, h->n_steps - h->n_window, 0, t0, &issued);
        if (s == WLB_OK) s = steps_within(h, h->n_window, 1, t0, &issued);
    } else {
        if (s == WLB_OK) s = wlb_step(h, h->n_steps - h->n_window, 0);
        if (s == WLB_OK) s = wlb_step(h, h->n_window, 1);
    }
    if (s == WLB_OK) s = wlb_force(h, force_out);
    return s;
}

wlb_status wlb_set_deadline(wlb_handle *h, double seconds) {
    if (!h || !(seconds >= 0.0) || !std::isfinite(seconds)) return WLB_ERR_ARG;
    DeviceGuard dg(h->device);
    for (int i = 0; i < 2 && seconds > 0.0; ++i)
        if (!h->marks[i]) WLB_CUDA(h, cudaEventCreateWithFlags(&h->marks[i], cudaEventDisableTiming), "marker event");
    h->deadline_s = seconds;
    return WLB_OK;
}

wlb_status wlb_fields(wlb_handle *h, double *p1_out, double *u1_out) {
    if (!h) return WLB_ERR_ARG;
    if (!h->initialised) return fail(h, WLB_ERR_STATE, "wlb_fields before wlb_init");
    DeviceGuard dg(h->device);
    const long long nc = h->g.ncell, chunk = h->b.stage_cells;
    for (long long first = 0; first < nc; first += chunk) {
        const long long count = nc - first < chunk ? nc - first : chunk;
        WLB_CUDA(h, wlb::launch_fields(h->g, h->b, h->prec, h->src, first, count, h->stream), "fields kernel");
        if (p1_out)
            WLB_CUDA(h, cudaMemcpyAsync(p1_out + first, h->b.stage, count * sizeof(double),
                                        cudaMemcpyDeviceToHost, h->stream), "p1 copy");
        if (u1_out)
            for (int a = 0; a < h->g.dim; ++a)
                WLB_CUDA(h, cudaMemcpyAsync(u1_out + (long long)a * nc + first, h->b.stage + (1 + a) * count,
                                            count * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                         "u1 copy");
        // the next chunk overwrites the staging buffer
        WLB_CUDA(h, cudaStreamSynchronize(h->stream), "synchronize");
    }
    return WLB_OK;
}

wlb_status wlb_surface(wlb_handle *h, double *pts_out) {
    if (!h || (!pts_out && h->g.n_surface > 0)) return WLB_ERR_ARG;
    if (!h->initialised) return fail(h, WLB_ERR_STATE, "wlb_surface before wlb_init");
    DeviceGuard dg(h->device);
    if (h->g.n_surface > 0)
        WLB_CUDA(h, cudaMemcpyAsync(pts_out, h->b.pts, (size_t)h->g.n_surface * 7 * sizeof(double),
                                    cudaMemcpyDeviceToHost, h->stream), "points copy");
    WLB_CUDA(h, cudaStreamSynchronize(h->stream), "synchronize");
    return WLB_OK;
}

wlb_status wlb_mask(wlb_handle *h, unsigned char *mask_out) {
    if (!h || !mask_out) return WLB_ERR_ARG;
    if (!h->initialised) return fail(h, WLB_ERR_STATE, "wlb_mask before wlb_init");
    DeviceGuard dg(h->device);
    WLB_CUDA(h, cudaMemcpyAsync(mask_out, h->b.cls, (size_t)h->g.ncell, cudaMemcpyDeviceToHost, h->stream),
             "mask copy");
    WLB_CUDA(h, cudaStreamSynchronize(h->stream), "synchronize");
    return WLB_OK;
}

namespace {

// Plan two steps per launch with the handle's settings and switch to it.
wlb_status replan_two_step(wlb_handle *h, int enable, int slab_rows, int tiles, int staging, int c2) {
    wlb::TwoStepPlan plan;
    if (enable) {
        cudaError_t e = cudaSuccess;
        if (!two_step_plan(h, slab_rows, enable, tiles, staging, c2, &plan, &e))
            return fail(h, WLB_ERR_ARG,
                        "two steps per launch need a periodic lattice: 3D FP32/FP16 rows of 16-cell multiples, or 2D "
                        "rows of at most 8 values per lane (no slab height, no x-tiles)");
        if (e != cudaSuccess) return fail(h, WLB_ERR_ARG, "slab height, x-tiles or lane layout do not fit", e);
    }
    const bool same = (enable != 0) == h->two_step && plan.H == h->two_plan.H && plan.zc == h->two_plan.zc &&
                      plan.nseg == h->two_plan.nseg && plan.chunks_per_lane == h->two_plan.chunks_per_lane &&
                      plan.ntile == h->two_plan.ntile && plan.tx == h->two_plan.tx &&
                      plan.producer == h->two_plan.producer && plan.c2_staged == h->two_plan.c2_staged;
    if (!same) {
        destroy_graphs(h);  // unsampled period graphs change shape
        h->two_step = enable != 0;
        h->two_plan = plan;
    }
    h->two_mode = enable;
    h->two_rows = slab_rows;
    h->two_tiles = tiles;
    h->two_staging = staging;
    h->two_c2 = c2;
    return WLB_OK;
}

}  // namespace

wlb_status wlb_set_two_step(wlb_handle *h, int enable, int slab_rows) {
    if (!h || slab_rows < 0 || enable < 0 || enable > 3) return WLB_ERR_ARG;
    DeviceGuard dg(h->device);
    return replan_two_step(h, enable, slab_rows, h->two_tiles, h->two_staging, h->two_c2);
}

wlb_status wlb_set_two_step_tiles(wlb_handle *h, int tiles) {
    if (!h || tiles < 0) return WLB_ERR_ARG;
    DeviceGuard dg(h->device);
    if (!h->two_mode) return fail(h, WLB_ERR_STATE, "x-tiles apply to two steps per launch, which is off");
    return replan_two_step(h, h->two_mode, h->two_rows, tiles, h->two_staging, h->two_c2);
}

wlb_status wlb_set_two_step_staging(wlb_handle *h, int staging) {
    if (!h || staging < 0 || staging > 2) return WLB_ERR_ARG;
    DeviceGuard dg(h->device);
    if (!h->two_mode) return fail(h, WLB_ERR_STATE, "the staging warp applies to two steps per launch, which is off");
    return replan_two_step(h, h->two_mode, h->two_rows, h->two_tiles, staging, h->two_c2);
}

wlb_status wlb_set_two_step_c2(wlb_handle *h, int c2) {
    if (!h || c2 < 0 || c2 > 2) return WLB_ERR_ARG;
    DeviceGuard dg(h->device);
    if (!h->two_mode) return fail(h, WLB_ERR_STATE, "c^2 staging applies to two steps per launch, which is off");
    return replan_two_step(h, h->two_mode, h->two_rows, h->two_tiles, h->two_staging, c2);
}

wlb_status wlb_get_info(const wlb_handle *h, wlb_info *out) {
    if (!h || !out) return WLB_ERR_ARG;
    out->dim = h->g.dim;
    out->q = h->g.q;
    out->cells = h->g.ncell;
    out->period = h->period;
    out->n_steps = h->n_steps;
    out->n_window = h->n_window;
    out->steps_done = h->steps_done;
    out->samples_done = h->samples_done;
    out->bytes_per_update = 2.0 * h->g.q * (double)wlb::pop_bytes(h->prec) + 1.0;
    out->vector_path = h->vector_path ? 1 : 0;
    out->steps_per_launch = h->two_step ? 2 : 1;
    out->two_step_rows = h->two_step ? h->two_plan.H : 0;
    out->two_step_segments = h->two_step ? h->two_plan.nseg : 0;
    out->two_step_tiles = h->two_step ? h->two_plan.ntile : 0;
    out->two_step_staging_warp = h->two_step ? h->two_plan.producer : 0;
    out->two_step_c2_staged = h->two_step && h->g.dim == 3 ? h->two_plan.c2_staged : 0;
    return WLB_OK;
}

wlb_status wlb_destroy(wlb_handle *h) {
    if (!h) return WLB_ERR_ARG;
    DeviceGuard dg(h->device);
    destroy_graphs(h);
    if (h->capture) cudaStreamDestroy(h->capture);
    if (h->side.stream) cudaStreamDestroy(h->side.stream);
    if (h->side.fork) cudaEventDestroy(h->side.fork);
    if (h->side.join) cudaEventDestroy(h->side.join);
    for (cudaEvent_t m : h->marks)
        if (m) cudaEventDestroy(m);
    if (h->host_out) cudaFreeHost(h->host_out);
    if (h->owned) cudaFree(h->owned);
    delete h;
    return WLB_OK;
}

}  // extern "C"
