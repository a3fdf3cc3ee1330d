// The bed object behind the C ABI and the library-internal calls that the
// API translation units share (api.cu: creation, stepping, read-back;
// adjoint.cu: recording and the reverse pass).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "dem_internal.cuh"

struct AdjointState;

struct dem_bed {
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    SimParams P{};
    DevBuf B{};
    int resort_every = 20;
    int64_t steps = 0;
    bool faulted = false;
    dem_alloc_fn alloc = nullptr;
    dem_free_fn freef = nullptr;
    void* actx = nullptr;
    std::vector<void*> allocs;
    int n_geom = 0;
    std::vector<int> geom_group;     // load-driven group of each primitive, or -1
    int nbeds = 1;
    std::vector<LevelGrid> levels;   // host copy of the level table
    std::vector<int> n_active;       // particles of beds still sweeping, per sweep
    std::vector<double> z_ref;  // particle surface under each primitive at creation
    // graphs: [parity][pre, jac, post]
    cudaGraphExec_t g[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    cudaGraphExec_t g_resort = nullptr;
    int k_step = 0, k_resort = 0;
    // timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<cudaEvent_t> ev_used;   // 4 per timed step: start, Jacobi start, Jacobi end, end
    double t_step_ms = 0, t_jac_ms = 0;
    int64_t t_steps = 0;
    // reverse-mode differentiation state (adjoint.cu), created on first use
    AdjointState* adj = nullptr;
    // coloured projected Gauss-Seidel buffers (solver 1), created on first use
    PgsBuf pgs{};
    int64_t pgs_cap = 0;
    int pgs_colours = 0;        // colours of the last PGS step
    // resident-sweep buffers (layout DEM_LAYOUT_RESIDENT), created on first use
    ResBuf res{};
    // Newton impact stage buffers, created when the stage is first enabled
    ImpBuf imp{};
    int capture_err = 0;        // CUDA error of a graph call made while capturing (0: none)
    // contact-capacity growth: after an overflow the steps from the last
    // committed one are re-run with larger arrays
    bool skip_resort = false;   // the next step's re-sort already ran (in the step that overflowed)
    bool no_grow = false;       // set while a differentiation window is recorded
    int grows = 0;              // capacity growths so far
    cudaStream_t side = nullptr;   // captures the bodies of conditional graph nodes
};

// error reporting through dem_last_error(); printf-style message
dem_status dem_fail(dem_status st, const char* fmt, ...);
// device memory through the bed's allocator (or cudaMallocAsync), freed with the bed
dem_status dem_dalloc(dem_bed* b, void** p, size_t bytes);
// return one allocation made by dem_dalloc before the bed is destroyed
void dem_dfree(dem_bed* b, void* p);
// synchronise the bed's stream and report a latched device fault
dem_status dem_check_fault(dem_bed* b);
// enqueue one step through the bed's graphs (re-sort when due)
dem_status dem_launch_step(dem_bed* b);
// set the message dem_last_error() returns
void dem_set_error_message(const char* msg);
// free the differentiation state (adjoint.cu)
void dem_adjoint_release(dem_bed* b);
// free the differentiation state and every device buffer it holds (sized by
// the contact capacity, which is about to change)
void dem_adjoint_drop(dem_bed* b);

#define DEM_CK(call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return dem_fail(DEM_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                            __FILE__, __LINE__);                                              \
    } while (0)
