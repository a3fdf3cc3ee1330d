// dem_detect_contacts_noalloc: sphere-sphere contact detection that allocates
// no memory at all.
//
// Who needs it: programs that may not call cudaMalloc while they run -- a host
// simulator whose GPU memory is fully reserved by another framework's caching
// allocator, a fixed-budget or real-time co-simulation loop that forbids
// allocation after start-up, or code that enqueues work while a CUDA stream is
// being captured, where allocation calls are not allowed.  They pass their own
// input and output buffers; every intermediate array (cell histogram, cell
// offsets, particle order, counters) lives in one file-scope device array.
//
// Limits: at most DEM_NOALLOC_MAX_N particles; the scratch array takes
// sizeof(NoAllocScratch) ~ 8.4 MB on every GPU that loads the library, held
// until the process exits.  Every call reuses the same array: calls that
// overlap on the GPU (different streams, or different host threads, without
// ordering) race and corrupt each other.  Radii must be positive and finite and
// coordinates finite: otherwise no pair is written and *count receives -1.
// The pair counter is 64-bit, so a dense input (every sphere in one cell) gives
// its full pair count however large, and only the first cap pairs are written.
//
// Method: one uniform grid of cells 2 r_max wide, hashed into a fixed number of
// buckets; particles are counting-sorted into buckets; each particle tests the
// buckets of its 27 neighbour cells with the same exact FP64 predicate as the
// per-step detection (geometry.cuh).  Output order is not specified.
#include <cuda.h>

#include <mutex>

#include "dem_internal.cuh"
#include "geometry.cuh"

#define DEM_NOALLOC_MAX_N (1 << 18)
#define NA_BUCKETS (1 << 19)
#define NA_T 128

struct NoAllocScratch {
    int count[NA_BUCKETS + 1];
    int start[NA_BUCKETS + 1];
    int fill[NA_BUCKETS];
    int bucket[DEM_NOALLOC_MAX_N];
    int order[DEM_NOALLOC_MAX_N];
    int scan_tmp[3 * (NA_BUCKETS / 2048 + 2)];
    unsigned rmax_bits;   // largest radius, as the bits of a positive float
    unsigned xmax_bits;   // largest |coordinate|, likewise
    unsigned bad;         // nonzero: a radius not positive and finite, or a non-finite coordinate
    unsigned pad;
    unsigned long long npairs;   // pairs found (may exceed the caller's capacity)
};

// the per-call clear zeroes rmax_bits .. npairs as one range
static_assert(offsetof(NoAllocScratch, npairs) == offsetof(NoAllocScratch, rmax_bits) + 4 * sizeof(unsigned),
              "NoAllocScratch: the cleared header must be contiguous");

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// host-side addresses of g_noalloc_scratch, one per device, looked up once per
// CUDA context: a device reset reloads the module, and the array may move
static NoAllocScratch* g_scratch_addr[64];
static unsigned long long g_scratch_ctx[64];
static std::mutex g_scratch_mu;

// unique id of the calling thread's current context (0 if it cannot be had);
// the driver calls are reached through the runtime, so the library does not
// link the driver library itself
typedef CUresult (*PFN_ctx_current)(CUcontext*);
typedef CUresult (*PFN_ctx_id)(CUcontext, unsigned long long*);
static unsigned long long current_ctx_id() {
    static PFN_ctx_current get_cur = nullptr;
    static PFN_ctx_id get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = (PFN_ctx_current)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (PFN_ctx_id)f;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_cur && get_id && get_cur(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS) return id;
    return 0;
}

static __device__ __forceinline__ unsigned bucket_of(int cx, int cy, int cz) {
    return (((unsigned)cx * 73856093u) ^ ((unsigned)cy * 19349663u) ^ ((unsigned)cz * 83492791u)) &
           (NA_BUCKETS - 1);
}

static __device__ __forceinline__ float na_cell(const NoAllocScratch* S) {
    const float rmax = __uint_as_float(S->rmax_bits);
    const float xmax = __uint_as_float(S->xmax_bits);
    return 2.0f * rmax * 1.0001f + 2.0f * (4.0f * ldexpf(xmax, -23) + 16.0f * ldexpf(rmax, -24));
}

__global__ void __launch_bounds__(NA_T) k_na_extent(NoAllocScratch* S, int n, const double* pos,
                                                    const float* rad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float r = rad[i];
    const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
    if (!(r > 0.0f) || !isfinite(r) || !isfinite(x) || !isfinite(y) || !isfinite(z)) {
        S->bad = 1u;
        return;
    }
    // positive floats order like their bit patterns
    atomicMax(&S->rmax_bits, __float_as_uint(r));
    const float ax = fmaxf(fabsf((float)x), fmaxf(fabsf((float)y), fabsf((float)z)));
    atomicMax(&S->xmax_bits, __float_as_uint(ax));
}

// Cell coordinates clamped to +-2^30, so that neighbour offsets never overflow
// (clamping is monotone: two spheres' clamped coordinates are no further apart
// than their true ones, so no touching pair is missed).
#define NA_CLAMP (1 << 30)
static __device__ __forceinline__ int na_coord(double x, float inv) {
    const float f = (float)x * inv;
    if (!(f > -(float)NA_CLAMP)) return -NA_CLAMP;   // NaN included (only with bad input)
    if (!(f < (float)NA_CLAMP)) return NA_CLAMP;
    return __float2int_rd(f);
}

static __device__ __forceinline__ void na_coords(const NoAllocScratch* S, const double* pos, int i, int& cx,
                                                 int& cy, int& cz) {
    const float inv = 1.0f / na_cell(S);
    cx = na_coord(pos[3 * i], inv);
    cy = na_coord(pos[3 * i + 1], inv);
    cz = na_coord(pos[3 * i + 2], inv);
}

__global__ void __launch_bounds__(NA_T) k_na_count(NoAllocScratch* S, int n, const double* pos) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cx, cy, cz;
    na_coords(S, pos, i, cx, cy, cz);
    const unsigned b = bucket_of(cx, cy, cz);
    S->bucket[i] = (int)b;
    atomicAdd(&S->count[b], 1);
}

__global__ void __launch_bounds__(NA_T) k_na_fill(NoAllocScratch* S, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = S->bucket[i];
    S->order[S->start[b] + atomicAdd(&S->fill[b], 1)] = i;
}

__global__ void __launch_bounds__(NA_T) k_na_pairs(NoAllocScratch* S, int n, const double* pos, const float* rad,
                                                   long long cap, int32_t* key_a, int32_t* key_b,
                                                   float* delta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || S->bad) return;
    const float rmax = __uint_as_float(S->rmax_bits);
    const float tol = 4.0f * ldexpf(__uint_as_float(S->xmax_bits), -23) + 16.0f * ldexpf(rmax, -24);
    const double4_32a xi = make_double4_32a(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], (double)rad[i]);
    const float pxi = (float)xi.x, pyi = (float)xi.y, pzi = (float)xi.z, ri = rad[i];
    int cx, cy, cz;
    na_coords(S, pos, i, cx, cy, cz);
    unsigned seen[27];
    int nseen = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const unsigned b = bucket_of(cx + dx, cy + dy, cz + dz);
                bool dup = false;
                for (int q = 0; q < nseen; ++q) dup |= seen[q] == b;
                if (dup) continue;   // two neighbour cells sharing a bucket: scan it once
                seen[nseen++] = b;
                for (int k = S->start[b]; k < S->start[b + 1]; ++k) {
                    const int j = S->order[k];
                    if (j <= i) continue;
                    const float R = ri + rad[j] + tol;
                    const float ex = pxi - (float)pos[3 * j], ey = pyi - (float)pos[3 * j + 1],
                                ez = pzi - (float)pos[3 * j + 2];
                    if (ex * ex + ey * ey + ez * ez >= R * R) continue;
                    const double4_32a xj = make_double4_32a(pos[3 * j], pos[3 * j + 1], pos[3 * j + 2], (double)rad[j]);
                    if (!exact_pair(xi, xj)) continue;
                    // overlap as in the contact rows: (R^2 - d^2) / (R + d)
                    const double ddx = __dsub_rn(xi.x, xj.x), ddy = __dsub_rn(xi.y, xj.y), ddz = __dsub_rn(xi.z, xj.z);
                    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
                    const double Rd = __dadd_rn(xi.w, xj.w);
                    const float dl = (float)__dsub_rn(__dmul_rn(Rd, Rd), d2) / ((float)Rd + sqrtf((float)d2));
                    const unsigned long long slot = atomicAdd(&S->npairs, 1ull);
                    if (slot < (unsigned long long)cap) {
                        key_a[slot] = i;
                        key_b[slot] = j;
                        delta[slot] = dl;
                    }
                }
            }
}

__global__ void k_na_count_out(const NoAllocScratch* S, int64_t* count) {
    *count = S->bad ? (int64_t)-1 : (int64_t)S->npairs;
}

void dem_set_error_message(const char* msg);
static dem_status na_fail(dem_status st, const char* msg);

extern "C" dem_status dem_detect_contacts_noalloc(int32_t n, const double* pos, const float* radius,
                                                  int64_t cap, int32_t* key_a, int32_t* key_b,
                                                  float* delta, int64_t* count, void* stream) {
    dem_set_error_message("");
    if (n < 0 || n > DEM_NOALLOC_MAX_N) return na_fail(DEM_ERR_ARG, "n is outside [0, 262144], the limit of the static scratch array");
    if (cap < 0 || !count) return na_fail(DEM_ERR_ARG, "cap < 0 or count is NULL");
    if (n > 0 && (!pos || !radius)) return na_fail(DEM_ERR_ARG, "pos and radius are required");
    if (cap > 0 && (!key_a || !key_b || !delta)) return na_fail(DEM_ERR_ARG, "output arrays are required when cap > 0");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return na_fail(DEM_ERR_CUDA, "no current CUDA device");
    NoAllocScratch* S;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        const unsigned long long ctx = current_ctx_id();
        if (!g_scratch_addr[dev] || (ctx != 0 && ctx != g_scratch_ctx[dev])) {
            // first call on this device (or in a new context after a device
            // reset): the device address of the scratch array
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return na_fail(DEM_ERR_CUDA, cudaGetErrorString(e));
            g_scratch_addr[dev] = (NoAllocScratch*)p;
            g_scratch_ctx[dev] = current_ctx_id();
        }
        S = g_scratch_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    // clear what must start at zero: histogram, fill cursors, extents, the
    // invalid-input flag and the pair counter
    cudaMemsetAsync(S->count, 0, sizeof(S->count), s);
    cudaMemsetAsync(S->fill, 0, sizeof(S->fill), s);
    cudaMemsetAsync(&S->rmax_bits, 0, 4 * sizeof(unsigned) + sizeof(unsigned long long), s);
    const int nb = n > 0 ? (n + NA_T - 1) / NA_T : 1;
    if (n > 0) {
        k_na_extent<<<nb, NA_T, 0, s>>>(S, n, pos, radius);
        k_na_count<<<nb, NA_T, 0, s>>>(S, n, pos);
        launch_scan(S->count, S->start, NA_BUCKETS, S->scan_tmp, s);
        k_na_fill<<<nb, NA_T, 0, s>>>(S, n);
        k_na_pairs<<<nb, NA_T, 0, s>>>(S, n, pos, radius, cap, key_a, key_b, delta);
    }
    k_na_count_out<<<1, 1, 0, s>>>(S, count);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(DEM_ERR_CUDA, cudaGetErrorString(e));
    return DEM_OK;
}

// errors of this entry point are reported through dem_last_error()
static dem_status na_fail(dem_status st, const char* msg) {
    dem_set_error_message(msg);
    return st;
}
