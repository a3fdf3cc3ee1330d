// Morton re-sort of the particles: key = (level, Morton code of the cell at the
// particle's own level), stable radix sort, then every per-particle array is
// permuted.  Particles close in space end up close in memory, so the cell
// scans, contact gathers and Jacobi sweeps touch few cache lines.  The old slot
// of every new slot is kept for the warm start of the next step.
#include "dem_internal.cuh"

#define RS_T 256

// spread the low 8 bits of v to every third bit
static __device__ __forceinline__ unsigned spread3(unsigned v) {
    v &= 0xffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void __launch_bounds__(RS_T) k_morton(SimParams P, DevBuf B) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const int l = B.lvl[i];
    const LevelGrid g = B.lv[l];
    const float4 p = B.posr[i];
    unsigned cx = cell_coord(p.x, g.ox, g.inv_cell, g.nx);
    unsigned cy = cell_coord(p.y, g.oy, g.inv_cell, g.ny);
    unsigned cz = cell_coord(p.z, g.oz, g.inv_cell, g.nz);
    // keep 8 bits per axis below the level index
    int m = max(g.nx, max(g.ny, g.nz));
    int sh = 0;
    while ((m >> sh) > 256) ++sh;
    cx >>= sh; cy >>= sh; cz >>= sh;
    B.key_a[i] = ((unsigned)l << 24) | (spread3(cz) << 2) | (spread3(cy) << 1) | spread3(cx);
    B.val_a[i] = i;
}

// After a fault (a step not committed) the particles keep their order, and
// the old slots of the last re-sort stay available to the step's re-run.
__global__ void __launch_bounds__(RS_T) k_permute_gather(SimParams P, DevBuf B) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n || *B.err) return;
    const int o = B.val_a[i];
    B.t_pos[i] = B.pos[o];
    B.t_vw[i] = B.vw0[o];
    B.t_id[i] = B.id[o];
    B.t_lvl[i] = B.lvl[o];
    B.prev_of[i] = o;
    if (i == 0) *B.resorted = 1;
}

__global__ void __launch_bounds__(RS_T) k_permute_store(SimParams P, DevBuf B) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n || *B.err) return;
    const double4_32a x = B.t_pos[i];
    B.pos[i] = x;
    B.posr[i] = make_float4((float)x.x, (float)x.y, (float)x.z, (float)x.w);
    B.vw0[i] = B.t_vw[i];
    B.id[i] = B.t_id[i];
    B.lvl[i] = B.t_lvl[i];
}

int launch_resort(const SimParams& P, const DevBuf& B, cudaStream_t s) {
    if (P.n <= 1) return 0;
    const int nb = (P.n + RS_T - 1) / RS_T;
    k_morton<<<nb, RS_T, 0, s>>>(P, B);
    int k = 1 + launch_radix_sort(B.key_a, B.val_a, B.key_b, B.val_b, P.n, B.hist, B.scan_tmp, s);
    k_permute_gather<<<nb, RS_T, 0, s>>>(P, B);
    k_permute_store<<<nb, RS_T, 0, s>>>(P, B);
    return k + 2;
}
