// Force history of a run (C ABI, include/wlb.h): the paper follows the force
// over time to see it settle (Sec. VII).  After the fold of every full sampled
// period, the force numerator of the FP64 sums folded so far (Eq. 14 with
// 1 / N_w = 1) is appended to a device array; the index lives in device memory,
// so replayed period graphs append too.  The force of period k is then
// (G_k - G_{k-1}) / T on the host: Eq. 14 is linear in the sums.
#include <cstdio>
#include <vector>

#include "wlb_handle.cuh"

namespace {

__global__ void push_history(const double *__restrict__ entry, double *__restrict__ hist,
                             unsigned long long *__restrict__ count, unsigned long long cap) {
    const unsigned long long k = *count;
    if (k < cap)
        for (int i = 0; i < 4; ++i) hist[4 * k + i] = entry[i];
    *count = k + 1;
}

unsigned long long capacity(const wlb::Geometry &g) {
    return (unsigned long long)(g.n_periods > 1 ? g.n_periods : 1);
}

}  // namespace

namespace wlb {

cudaError_t launch_record_period(const Geometry &g, const Buffers &b, cudaStream_t s) {
    if (g.n_surface == 0) return cudaSuccess;
    Buffers t = b;
    t.force = b.hist_tmp;  // the force kernel's reduction, into the entry
    cudaError_t e = launch_force(g, t, 1.0, s);
    if (e != cudaSuccess) return e;
    push_history<<<1, 1, 0, s>>>(b.hist_tmp, b.hist, b.hist_n, capacity(g));
    return cudaGetLastError();
}

}  // namespace wlb

extern "C" wlb_status wlb_force_history(wlb_handle *h, double *out, int max_periods, int *count) {
    if (!h || !count || max_periods < 0 || (max_periods > 0 && !out)) return WLB_ERR_ARG;
    if (!h->initialised) {
        snprintf(h->err, sizeof(h->err), "wlb_force_history before wlb_init");
        return WLB_ERR_STATE;
    }
    int prev = -1;
    if (cudaGetDevice(&prev) == cudaSuccess && prev != h->device) cudaSetDevice(h->device);
    else prev = -1;
    wlb_status st = WLB_OK;
    unsigned long long n = 0;
    cudaError_t e = cudaSuccess;
    if (h->g.n_surface > 0)
        e = cudaMemcpyAsync(&n, h->b.hist_n, sizeof(n), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    const unsigned long long cap = capacity(h->g);
    const unsigned long long have = n < cap ? n : cap;
    const unsigned long long want = have < (unsigned long long)max_periods ? have : (unsigned long long)max_periods;
    std::vector<double> G(4 * (size_t)want);
    if (e == cudaSuccess && want > 0)
        e = cudaMemcpy(G.data(), h->b.hist, G.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        snprintf(h->err, sizeof(h->err), "history copy: %s", cudaGetErrorString(e));
        st = WLB_ERR_CUDA;
    } else {
        const double T = (double)h->period;
        for (unsigned long long k = 0; k < want; ++k)
            for (int i = 0; i < 3; ++i)
                out[3 * k + i] = (G[4 * k + i] - (k > 0 ? G[4 * (k - 1) + i] : 0.0)) / T;
        *count = (int)(n < 0x7fffffffULL ? n : 0x7fffffffULL);
    }
    if (prev >= 0) cudaSetDevice(prev);
    return st;
}
