// Checkpoint and resume of a handle's dynamic state (C ABI, include/wlb.h).
// Not part of the paper's method: a long run can stop and continue.  After
// wlb_init and any steps the state is the current population buffer, the
// running surface sums of the current period, the folded FP64 sums, the force
// history, the error flag and the step counters.  Everything else (classes,
// c^2, surface points, stencils) is a function of the parameters and is
// rebuilt by the setup.
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "wlb_handle.cuh"

namespace {

constexpr char kMagic[8] = {'W', 'L', 'B', 'S', 'T', 'A', 'T', 'E'};
constexpr uint32_t kVersion = 1;
constexpr int kParamWords = 24;

// Fixed-size header in front of the arrays.  The parameters are kept as
// doubles (every int of wlb_params is exact in a double) so that a state is
// matched field by field, never through struct padding.
struct Header {
    char magic[8];
    uint32_t version, header_bytes;
    double params[kParamWords];
    long long steps_done, samples_done, samples_in_period;
    unsigned long long pop_bytes, acc_bytes, acc64_bytes, hist_bytes;
};

void canonical(const wlb_params &p, double (&w)[kParamWords]) {
    const double v[kParamWords] = {(double)p.lattice, (double)p.nx, (double)p.ny, (double)p.nz,
                                   (double)p.wave_axis, p.c0, p.cp, p.rho0, p.p_a, p.wavelength, p.antinode,
                                   p.center[0], p.center[1], p.center[2], p.radius, p.interface_d,
                                   p.surface_radius, (double)p.n_surface, (double)p.n_periods,
                                   (double)p.n_avg_periods, (double)p.precision, (double)p.boundary,
                                   p.wall_damping, p.source_amplitude};
    for (int i = 0; i < kParamWords; ++i) w[i] = v[i];
}

struct Sizes {
    size_t pop, acc, acc64, hist, total;
};

// Array sizes and the offsets that follow from them (each 8-byte aligned).
Sizes sizes_of(const wlb_handle *h) {
    const size_t nc = (size_t)h->g.ncell, N = (size_t)h->g.n_surface;
    Sizes s;
    s.pop = (size_t)h->g.q * nc * wlb::pop_bytes(h->prec);
    s.acc = N * 5 * wlb::real_bytes(h->prec);
    s.acc64 = N * 5 * sizeof(double);
    s.hist = (size_t)wlb::history_capacity(h->g) * 4 * sizeof(double);
    auto up8 = [](size_t v) { return (v + 7) & ~(size_t)7; };
    s.total = sizeof(Header) + up8(s.pop) + up8(s.acc) + s.acc64 + s.hist + 8 + 8;  // + count, error flag
    return s;
}

struct Guard {
    int prev = -1;
    explicit Guard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~Guard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

wlb_status sfail(wlb_handle *h, wlb_status s, const char *what, cudaError_t e = cudaSuccess) {
    if (e != cudaSuccess)
        snprintf(h->err, sizeof(h->err), "%s: %s", what, cudaGetErrorString(e));
    else
        snprintf(h->err, sizeof(h->err), "%s", what);
    return s;
}

}  // namespace

extern "C" {

wlb_status wlb_state_bytes(const wlb_handle *h, size_t *bytes) {
    if (!h || !bytes) return WLB_ERR_ARG;
    *bytes = sizes_of(h).total;
    return WLB_OK;
}

wlb_status wlb_save_state(wlb_handle *h, void *host, size_t bytes) {
    if (!h || !host) return WLB_ERR_ARG;
    const Sizes s = sizes_of(h);
    if (bytes < s.total) return sfail(h, WLB_ERR_ARG, "state buffer smaller than wlb_state_bytes");
    if (!h->initialised) return sfail(h, WLB_ERR_STATE, "wlb_save_state before wlb_init");
    Guard dg(h->device);
    Header hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, kMagic, sizeof(kMagic));
    hd.version = kVersion;
    hd.header_bytes = sizeof(Header);
    canonical(h->p, hd.params);
    hd.steps_done = h->steps_done;
    hd.samples_done = h->samples_done;
    hd.samples_in_period = h->samples_in_period;
    hd.pop_bytes = s.pop;
    hd.acc_bytes = s.acc;
    hd.acc64_bytes = s.acc64;
    hd.hist_bytes = s.hist;
    char *out = static_cast<char *>(host);
    memcpy(out, &hd, sizeof(hd));
    size_t off = sizeof(Header);
    struct Part {
        const void *src;
        size_t n;
    } parts[6] = {{h->b.pop[h->src], s.pop}, {h->b.acc, s.acc},           {h->b.acc64, s.acc64},
                  {h->b.hist, s.hist},         {h->b.hist_n, 8},           {h->b.err, sizeof(int)}};
    for (const Part &p : parts) {
        if (p.n) {
            cudaError_t e = cudaMemcpyAsync(out + off, p.src, p.n, cudaMemcpyDeviceToHost, h->stream);
            if (e != cudaSuccess) return sfail(h, WLB_ERR_CUDA, "state copy", e);
        }
        off += (p.n + 7) & ~(size_t)7;
    }
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return sfail(h, WLB_ERR_CUDA, "synchronize", e);
    return WLB_OK;
}

wlb_status wlb_load_state(wlb_handle *h, const void *host, size_t bytes) {
    if (!h || !host) return WLB_ERR_ARG;
    const Sizes s = sizes_of(h);
    if (bytes < s.total) return sfail(h, WLB_ERR_ARG, "state buffer smaller than wlb_state_bytes");
    Header hd;
    memcpy(&hd, host, sizeof(hd));
    if (memcmp(hd.magic, kMagic, sizeof(kMagic)) != 0 || hd.version != kVersion || hd.header_bytes != sizeof(Header))
        return sfail(h, WLB_ERR_ARG, "not a state written by wlb_save_state");
    double mine[kParamWords];
    canonical(h->p, mine);
    if (memcmp(mine, hd.params, sizeof(mine)) != 0 || hd.pop_bytes != s.pop || hd.acc_bytes != s.acc ||
        hd.acc64_bytes != s.acc64 || hd.hist_bytes != s.hist)
        return sfail(h, WLB_ERR_ARG, "state was saved for other parameters");
    if (hd.steps_done < 0 || hd.samples_done < 0 || hd.samples_in_period < 0 ||
        hd.samples_in_period >= h->period)
        return sfail(h, WLB_ERR_ARG, "state counters out of range");
    Guard dg(h->device);
    if (!h->initialised) {
        const wlb_status st = wlb_init(h);  // the parameter-derived arrays
        if (st != WLB_OK) return st;
    }
    const char *in = static_cast<const char *>(host);
    size_t off = sizeof(Header);
    struct Part {
        void *dst;
        size_t n;
    } parts[6] = {{h->b.pop[0], s.pop}, {h->b.acc, s.acc},      {h->b.acc64, s.acc64},
                  {h->b.hist, s.hist},  {h->b.hist_n, 8},       {h->b.err, sizeof(int)}};
    for (const Part &p : parts) {
        if (p.n) {
            cudaError_t e = cudaMemcpyAsync(p.dst, in + off, p.n, cudaMemcpyHostToDevice, h->stream);
            if (e != cudaSuccess) return sfail(h, WLB_ERR_CUDA, "state copy", e);
        }
        off += (p.n + 7) & ~(size_t)7;
    }
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return sfail(h, WLB_ERR_CUDA, "synchronize", e);
    h->src = 0;
    h->steps_done = hd.steps_done;
    h->samples_done = hd.samples_done;
    h->samples_in_period = hd.samples_in_period;
    return WLB_OK;
}

}  // extern "C"
