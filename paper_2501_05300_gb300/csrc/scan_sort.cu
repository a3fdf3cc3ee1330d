// Device-wide exclusive prefix sums and a stable LSD radix sort.
//
// Scan: tiles of 2048 ints are scanned in shared memory, the tile totals are
// scanned by one block, then added back (3 kernels; 2 when one tile suffices).
// Up to three columns are scanned by the same launches.  out[n] receives the
// total, so an n-element count array yields n+1 CSR offsets.
//
// Radix sort: 8-bit digits, 4 passes over 32-bit keys.  Each pass builds
// per-tile digit histograms, scans them digit-major and scatters stably: inside
// a tile, the rank of an element among equal digits comes from warp match
// masks and per-warp digit counts, so equal keys keep their input order.
#include "dem_internal.cuh"

#define SCAN_T 256
#define SCAN_PER 8
#define SCAN_TILE (SCAN_T * SCAN_PER)

struct ScanCols {
    const int* in[3];
    const int* in2[3];  // optional second input added element-wise (NULL = none)
    int* out[3];
    const int* skip;    // optional: when *skip != 0 the scan writes nothing (NULL = always run)
};

template <int C>
__global__ void __launch_bounds__(SCAN_T) k_scan_tiles(ScanCols a, int n, int* sums, int nb) {
    if (a.skip && *a.skip) return;
    __shared__ int sm[C][SCAN_TILE];
    __shared__ int wsum[C][SCAN_T / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int base = blockIdx.x * SCAN_TILE;
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int k = 0; k < SCAN_PER; ++k) {
            int idx = base + k * SCAN_T + t;
            sm[c][k * SCAN_T + t] = idx < n ? a.in[c][idx] + (a.in2[c] ? a.in2[c][idx] : 0) : 0;
        }
    __syncthreads();
    int loc[C][SCAN_PER];
    int tot[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        int s = 0;
#pragma unroll
        for (int k = 0; k < SCAN_PER; ++k) {
            loc[c][k] = s;
            s += sm[c][t * SCAN_PER + k];
        }
        tot[c] = s;
        // inclusive warp scan of the thread totals
        int v = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) wsum[c][w] = v;
        tot[c] = v - s;  // exclusive within the warp
    }
    __syncthreads();
    if (t < 32) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            int v = t < SCAN_T / 32 ? wsum[c][t] : 0;
            int s = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(0xffffffffu, s, o);
                if (t >= o) s += u;
            }
            if (t < SCAN_T / 32) wsum[c][t] = s - v;   // exclusive warp offsets
            if (t == SCAN_T / 32 - 1) sums[c * nb + blockIdx.x] = s;
        }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < C; ++c) {
        int off = tot[c] + wsum[c][w];
#pragma unroll
        for (int k = 0; k < SCAN_PER; ++k) sm[c][t * SCAN_PER + k] = off + loc[c][k];
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int k = 0; k < SCAN_PER; ++k) {
            int idx = base + k * SCAN_T + t;
            if (idx < n) a.out[c][idx] = sm[c][k * SCAN_T + t];
        }
}

// One block: exclusive scan of the tile totals of each column in place;
// writes the grand total to out[c][n].
template <int C>
__global__ void __launch_bounds__(1024) k_scan_sums(ScanCols a, int n, int* sums, int nb) {
    if (a.skip && *a.skip) return;
    __shared__ int wsum[32];
    __shared__ int carry;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    for (int c = 0; c < C; ++c) {
        if (t == 0) carry = 0;
        __syncthreads();
        for (int base = 0; base < nb; base += 1024) {
            int idx = base + t;
            int v = idx < nb ? sums[c * nb + idx] : 0;
            int s = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += u;
            }
            if (lane == 31) wsum[w] = s;
            __syncthreads();
            if (w == 0) {
                int x = wsum[lane];
                int y = x;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int u = __shfl_up_sync(0xffffffffu, y, o);
                    if (lane >= o) y += u;
                }
                wsum[lane] = y - x;
            }
            __syncthreads();
            int excl = carry + wsum[w] + s - v;
            if (idx < nb) sums[c * nb + idx] = excl;
            __syncthreads();
            if (t == 1023) carry = excl + v;
            __syncthreads();
        }
        if (t == 0) a.out[c][n] = carry;
        __syncthreads();
    }
}

template <int C>
__global__ void __launch_bounds__(SCAN_T) k_scan_add(ScanCols a, int n, const int* sums, int nb) {
    if (a.skip && *a.skip) return;
    const int base = blockIdx.x * SCAN_TILE;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        int add = sums[c * nb + blockIdx.x];
#pragma unroll
        for (int k = 0; k < SCAN_PER; ++k) {
            int idx = base + k * SCAN_T + threadIdx.x;
            if (idx < n) a.out[c][idx] += add;
        }
    }
}

template <int C>
static int scan_impl(ScanCols a, int n, int* tmp, cudaStream_t s) {
    if (n <= 0) {
        // only the totals: zero
        for (int c = 0; c < C; ++c) cudaMemsetAsync(a.out[c], 0, sizeof(int), s);
        return 0;
    }
    int nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    k_scan_tiles<C><<<nb, SCAN_T, 0, s>>>(a, n, tmp, nb);
    k_scan_sums<C><<<1, 1024, 0, s>>>(a, n, tmp, nb);
    if (nb > 1) {
        k_scan_add<C><<<nb, SCAN_T, 0, s>>>(a, n, tmp, nb);
        return 3;
    }
    return 2;
}

int launch_scan(const int* in, int* out, int n, int* tmp, cudaStream_t s) {
    ScanCols a{};
    a.in[0] = in;
    a.out[0] = out;
    return scan_impl<1>(a, n, tmp, s);
}

int launch_scan3(const int* x, const int* y, const int* y2, const int* z, int* ox, int* oy, int* oz,
                 int n, int* tmp, cudaStream_t s, const int* skip) {
    ScanCols a{};
    a.skip = skip;
    a.in[0] = x; a.in[1] = y; a.in[2] = z;
    a.in2[1] = y2;
    a.out[0] = ox; a.out[1] = oy; a.out[2] = oz;
    return scan_impl<3>(a, n, tmp, s);
}

// ---------------------------------------------------------------------------
// radix sort of (key, value) pairs
// ---------------------------------------------------------------------------
#define RADIX_T 256
#define RADIX_PER 8
#define RADIX_TILE (RADIX_T * RADIX_PER)

int radix_blocks(int n) { return n > 0 ? (n + RADIX_TILE - 1) / RADIX_TILE : 1; }

__global__ void __launch_bounds__(RADIX_T) k_radix_hist(const unsigned* keys, int n, int shift,
                                                        int* hist, int nb) {
    __shared__ int cnt[256];
    const int t = threadIdx.x;
    cnt[t] = 0;
    __syncthreads();
    const int base = blockIdx.x * RADIX_TILE;
#pragma unroll
    for (int k = 0; k < RADIX_PER; ++k) {
        int idx = base + k * RADIX_T + t;
        if (idx < n) atomicAdd(&cnt[(keys[idx] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[t * nb + blockIdx.x] = cnt[t];
}

__global__ void __launch_bounds__(RADIX_T) k_radix_scatter(const unsigned* kin, const int* vin,
                                                           unsigned* kout, int* vout, int n,
                                                           int shift, const int* off, int nb) {
    __shared__ int running[256];
    __shared__ int wcnt[RADIX_T / 32][257];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    running[t] = off[t * nb + blockIdx.x];
    for (int q = 0; q < RADIX_T / 32; ++q) wcnt[q][t] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    const int base = blockIdx.x * RADIX_TILE;
    for (int k = 0; k < RADIX_PER; ++k) {
        int idx = base + k * RADIX_T + t;
        bool valid = idx < n;
        unsigned key = valid ? kin[idx] : 0u;
        int val = valid ? vin[idx] : 0;
        int d = valid ? (int)((key >> shift) & 255u) : 256;
        unsigned mask = __match_any_sync(0xffffffffu, d);
        int rank = __popc(mask & lt);
        if (rank == 0) wcnt[w][d] = __popc(mask);
        __syncthreads();
        if (valid) {
            int pre = 0;
            for (int q = 0; q < w; ++q) pre += wcnt[q][d];
            int pos = running[d] + pre + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        int add = 0;
        for (int q = 0; q < RADIX_T / 32; ++q) {
            add += wcnt[q][t];
            wcnt[q][t] = 0;
        }
        running[t] += add;
        if (t == 0)
            for (int q = 0; q < RADIX_T / 32; ++q) wcnt[q][256] = 0;
        __syncthreads();
    }
}

// Sorts (key_a, val_a) by key; the result ends in key_a/val_a again after the
// 4 passes.  Returns kernels launched.
int launch_radix_sort(unsigned* key_a, int* val_a, unsigned* key_b, int* val_b, int n, int* hist,
                      int* tmp, cudaStream_t s) {
    if (n <= 1) return 0;
    int nb = radix_blocks(n);
    int k = 0;
    unsigned* ki = key_a; int* vi = val_a;
    unsigned* ko = key_b; int* vo = val_b;
    for (int pass = 0; pass < 4; ++pass) {
        int shift = 8 * pass;
        k_radix_hist<<<nb, RADIX_T, 0, s>>>(ki, n, shift, hist, nb);
        k += 1 + launch_scan(hist, hist, 256 * nb, tmp, s);
        k_radix_scatter<<<nb, RADIX_T, 0, s>>>(ki, vi, ko, vo, n, shift, hist, nb);
        ++k;
        unsigned* tk = ki; ki = ko; ko = tk;
        int* tv = vi; vi = vo; vo = tv;
    }
    return k;
}
