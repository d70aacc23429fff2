// Definition of the opaque wlb_handle, shared by the C-ABI translation units.
#pragma once
#include "../../include/wlb.h"
#include "wlb_internal.cuh"

namespace wlb {
// Host helpers of the C ABI (wlb_api.cu).
Geometry make_geometry(const wlb_params *p);
Prec prec_of(const wlb_params *p);
size_t layout(const Geometry &g, Prec prec, char *base, Buffers *b);  // size only if base == nullptr
}  // namespace wlb

struct wlb_handle {
    wlb_params p;
    wlb::Geometry g;
    wlb::Buffers b;
    wlb::Prec prec = wlb::Prec::F32;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;  // private stream used only to capture graphs
    void *owned = nullptr;           // workspace allocated by the library, if any
    double *host_out = nullptr;      // pinned: force[4] + error flag
    int src = 0;                     // population buffer holding the current state
    bool initialised = false;
    long long period = 0, n_steps = 0, n_window = 0;
    long long steps_done = 0, samples_done = 0, samples_in_period = 0;
    cudaGraphExec_t graph_free[2] = {nullptr, nullptr};
    cudaGraphExec_t graph_sampled[2] = {nullptr, nullptr};
    bool vector_path = false;
    bool two_step = false;      // unsampled steps two per launch (wlb_set_two_step)
    wlb::TwoStepPlan two_plan;  // its grid, set by wlb_set_two_step
    int two_mode = 0, two_rows = 0, two_tiles = 0, two_staging = 0, two_c2 = 0;  // the settings it was planned with
    wlb::SideStream side;       // sampling beside the two-step update
    double deadline_s = 0.0;    // wlb_run's host-clock limit, 0 = none (wlb_set_deadline)
    cudaEvent_t marks[2] = {nullptr, nullptr};  // period markers of a deadline run
    char err[512] = {0};
};

