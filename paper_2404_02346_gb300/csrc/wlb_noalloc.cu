// wlb_average_noalloc: time averaging and force without any allocation.
//
// The paper has no counterpart of this entry point.  It exists for callers that
// cannot allocate device memory at the point where they need a force: processes
// whose device memory is a fixed pool owned by someone else (a framework's
// caching allocator that has reserved the whole budget, an arena handed to a
// plugin that is given no allocator of its own), and loops that cannot afford
// cudaMalloc / cudaFree, which may synchronise the whole device.  It runs the
// same sampling, fold and force kernels as wlb_step(sample = 1) + wlb_force,
// launched directly (instantiating a graph would allocate), with the running
// sums, their FP64 totals, the force and the error flag in one file-scope
// device array instead of the handle's workspace.
#include <cuda.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "wlb_handle.cuh"

namespace {

constexpr int kMaxSurface = WLB_NOALLOC_MAX_SURFACE;
constexpr size_t kSumBytes = (size_t)kMaxSurface * 5 * sizeof(double);  // running sums (<= FP64)
constexpr size_t kTotBytes = (size_t)kMaxSurface * 5 * sizeof(double);  // folded totals
constexpr size_t kScratchBytes = kSumBytes + kTotBytes + 256;           // + force[4] and flag

// Shared by every call on a device; held from module load until exit.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
struct ScratchAddress {
    unsigned long long context = 0;  // id of the context the address belongs to (0: none yet)
    void *addr = nullptr;
};
ScratchAddress g_scratch_addr[kMaxDevices];

// Driver calls that identify the current context, resolved through the
// runtime (no link against the driver library).
using CtxGetCurrent = CUresult(CUDAAPI *)(CUcontext *);
using CtxGetId = CUresult(CUDAAPI *)(CUcontext, unsigned long long *);
CtxGetCurrent g_ctx_get_current = nullptr;
CtxGetId g_ctx_get_id = nullptr;

cudaError_t resolve_driver_calls() {
    if (g_ctx_get_current && g_ctx_get_id) return cudaSuccess;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    void *f1 = nullptr, *f2 = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess) return e;
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
        return cudaErrorSymbolNotFound;
    g_ctx_get_current = (CtxGetCurrent)f1;
    g_ctx_get_id = (CtxGetId)f2;
    return cudaSuccess;
}

// Device address of g_scratch on `device` (which must be current).  The
// host-side symbol is not a device address.  The address is looked up once
// per device and context: the module holding the array is loaded per
// context, so after a cudaDeviceReset (a new primary context) it is looked up
// again rather than reused.
cudaError_t scratch_address(int device, void **out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    cudaError_t e = resolve_driver_calls();
    if (e != cudaSuccess) return e;
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return cudaErrorContextIsDestroyed;
    if (!ctx) {  // no context current on this thread yet: make the primary one current
        if ((e = cudaSetDevice(device)) != cudaSuccess) return e;
        if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorContextIsDestroyed;
    }
    unsigned long long id = 0;
    if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return cudaErrorContextIsDestroyed;
    ScratchAddress &slot = g_scratch_addr[device];
    if (slot.context != id || !slot.addr) {
        void *p = nullptr;
        if ((e = cudaGetSymbolAddress(&p, g_scratch)) != cudaSuccess) return e;
        slot.addr = p;
        slot.context = id;
    }
    *out = slot.addr;
    return cudaSuccess;
}

wlb_status note(wlb_handle *h, wlb_status s, const char *what, cudaError_t e = cudaSuccess) {
    if (e != cudaSuccess)
        snprintf(h->err, sizeof(h->err), "%s: %s", what, cudaGetErrorString(e));
    else
        snprintf(h->err, sizeof(h->err), "%s", what);
    return s;
}

}  // namespace

extern "C" wlb_status wlb_average_noalloc(wlb_handle *h, long long n_steps, double force_out[3]) {
    if (!h || !force_out || n_steps < 0) return WLB_ERR_ARG;
    if (!h->initialised) return note(h, WLB_ERR_STATE, "wlb_average_noalloc before wlb_init");
    if (h->g.n_surface > kMaxSurface)
        return note(h, WLB_ERR_ARG, "n_surface exceeds WLB_NOALLOC_MAX_SURFACE (8192)");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != h->device && cudaSetDevice(h->device) != cudaSuccess)
        return note(h, WLB_ERR_CUDA, "cudaSetDevice failed");
    wlb_status st = WLB_OK;
    do {
        void *base = nullptr;
        cudaError_t e = scratch_address(h->device, &base);
        if (e != cudaSuccess) { st = note(h, WLB_ERR_CUDA, "cudaGetSymbolAddress", e); break; }
        const int N = h->g.n_surface;
        const size_t tb = wlb::real_bytes(h->prec);
        wlb::Buffers b = h->b;  // populations, classes, stencils: the handle's
        b.acc = base;
        b.acc64 = (double *)((char *)base + kSumBytes);
        b.force = (double *)((char *)base + kSumBytes + kTotBytes);
        b.err = (int *)((char *)base + kSumBytes + kTotBytes + 4 * sizeof(double));
        // the array keeps the previous call's contents: clear what accumulates
        if ((e = cudaMemsetAsync(b.acc, 0, (size_t)N * 5 * tb, h->stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(b.acc64, 0, (size_t)N * 5 * sizeof(double), h->stream)) != cudaSuccess ||
            (e = cudaMemsetAsync(b.force, 0, 4 * sizeof(double) + sizeof(int), h->stream)) != cudaSuccess) {
            st = note(h, WLB_ERR_CUDA, "clear scratch", e);
            break;
        }
        long long in_period = 0;
        for (long long t = 0; t < n_steps && st == WLB_OK; ++t) {
            if ((e = wlb::launch_sample(h->g, b, h->prec, h->src, h->stream)) != cudaSuccess ||
                (e = wlb::launch_update(h->g, b, h->prec, h->src, h->steps_done % h->period, h->stream,
                                        nullptr)) != cudaSuccess) {
                st = note(h, WLB_ERR_CUDA, "step kernels", e);
                break;
            }
            h->src ^= 1;
            h->steps_done += 1;
            if (++in_period == h->period) {
                if ((e = wlb::launch_fold(h->g, b, h->prec, h->stream)) != cudaSuccess)
                    st = note(h, WLB_ERR_CUDA, "fold kernel", e);
                in_period = 0;
            }
        }
        if (st != WLB_OK) break;
        if (n_steps == 0 || N == 0) {
            if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) st = note(h, WLB_ERR_CUDA, "synchronize", e);
            force_out[0] = force_out[1] = force_out[2] = 0.0;
            break;
        }
        if (in_period > 0 && (e = wlb::launch_fold(h->g, b, h->prec, h->stream)) != cudaSuccess) {
            st = note(h, WLB_ERR_CUDA, "fold kernel", e);
            break;
        }
        if ((e = wlb::launch_force(h->g, b, (double)n_steps, h->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(h->host_out, b.force, 4 * sizeof(double) + sizeof(int),
                                 cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(h->stream)) != cudaSuccess) {
            st = note(h, WLB_ERR_CUDA, "force kernel / read-back", e);
            break;
        }
        int flag;
        memcpy(&flag, h->host_out + 4, sizeof(int));
        for (int i = 0; i < 3; ++i) force_out[i] = h->host_out[i];
        if (flag) st = note(h, WLB_ERR_UNSTABLE, "non-finite accumulators");
    } while (0);
    if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
    return st;
}
