// Force history of a run (C ABI, include/wlb.h): the paper follows the force
// over time to see it settle (Sec. VII).  After every fold of the running sums
// (each full sampled period, and the partial one wlb_force folds) the force
// numerator of the FP64 sums folded so far (Eq. 14 with 1 / N_w = 1) and the
// number of samples the fold added are appended to a device array; the index
// lives in device memory, so replayed period graphs append too.  The force of
// entry k is then (G_k - G_{k-1}) / n_k on the host: Eq. 14 is linear in the
// sums.
#include <cstdio>
#include <vector>

#include "wlb_handle.cuh"

namespace {

__global__ void push_history(const double *__restrict__ entry, double *__restrict__ hist,
                             unsigned long long *__restrict__ count, unsigned long long cap, double samples) {
    const unsigned long long k = *count;
    if (k < cap) {
        for (int i = 0; i < 3; ++i) hist[4 * k + i] = entry[i];
        hist[4 * k + 3] = samples;
    }
    *count = k + 1;
}

unsigned long long capacity(const wlb::Geometry &g) { return wlb::history_capacity(g); }

}  // namespace

namespace wlb {

cudaError_t launch_record_fold(const Geometry &g, const Buffers &b, long long samples, cudaStream_t s) {
    if (g.n_surface == 0 || samples <= 0) return cudaSuccess;
    Buffers t = b;
    t.force = b.hist_tmp;  // the force kernel's reduction, into the entry
    cudaError_t e = launch_force(g, t, 1.0, s);
    if (e != cudaSuccess) return e;
    push_history<<<1, 1, 0, s>>>(b.hist_tmp, b.hist, b.hist_n, capacity(g), (double)samples);
    return cudaGetLastError();
}

}  // namespace wlb

extern "C" wlb_status wlb_force_history(wlb_handle *h, double *out, long long *samples_out, int max_entries,
                                        int *count) {
    if (!h || !count || max_entries < 0 || (max_entries > 0 && !out)) return WLB_ERR_ARG;
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
    const unsigned long long want = have < (unsigned long long)max_entries ? have : (unsigned long long)max_entries;
    std::vector<double> G(4 * (size_t)want);
    if (e == cudaSuccess && want > 0)
        e = cudaMemcpy(G.data(), h->b.hist, G.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        snprintf(h->err, sizeof(h->err), "history copy: %s", cudaGetErrorString(e));
        st = WLB_ERR_CUDA;
    } else {
        for (unsigned long long k = 0; k < want; ++k) {
            const double nk = G[4 * k + 3];
            for (int i = 0; i < 3; ++i) out[3 * k + i] = (G[4 * k + i] - (k > 0 ? G[4 * (k - 1) + i] : 0.0)) / nk;
            if (samples_out) samples_out[k] = (long long)nk;
        }
        *count = (int)(n < 0x7fffffffULL ? n : 0x7fffffffULL);
    }
    if (prev >= 0) cudaSetDevice(prev);
    return st;
}
