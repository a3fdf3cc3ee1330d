// Broad and narrow phase: multi-level cell lists, sphere-sphere and
// sphere-geometry contact detection, contact and incidence lists.
//
// Levels: every particle belongs to one radius band ("level"); the cells of
// level l are 2 r_max(l) wide.  Two particles of the same level that touch lie
// in neighbouring cells; a particle looks for partners of a coarser level l'
// in the 27 cells of level l' around it, since r_a + r_b <= 2 r_max(l').
// A pair of the same level is owned by the lower stable id, a cross-level pair
// by the finer particle, so every pair is found exactly once (Sec. 2.2: the
// contact set is recomputed every time step).
//
// Contact predicate (exact): |x_a - x_b|^2 < (r_a + r_b)^2 evaluated in IEEE
// double from the double centres, as (dx^2 + dy^2) + dz^2 with every product
// and sum rounded separately (no fused multiply-add).  An FP32 pre-test with a
// tolerance tol that covers the rounding of the FP32 copies and of the FP32
// arithmetic settles all but a thin band of pairs: d_f32 >= r_a + r_b + tol
// rejects, d_f32 < r_a + r_b - tol accepts, and only the band in between is
// decided by the FP64 predicate.  tol bounds the FP32 distance's error with
// more than a factor two to spare: the copies' rounding (<= 3.5 2^-24 of the
// coordinates, moved up to 1.25x) plus a few ulps of r_a + r_b from the FP32
// arithmetic, against tol = 10 2^-24 of the coordinates + 80 2^-24 r_max; so an
// accepted pair's double distance is below r_a + r_b by far more than the
// double predicate's rounding.  The contact set is the exact predicate's.
//
// tol follows the particles: every step it is recomputed from that step's
// largest |coordinate| (the per-level boxes of k_cell_count), so the bound holds
// however far particles travel from where they were created.  It never drops
// below the creation-time tolerance the cells were sized with.  Growing it keeps
// the 27-cell search complete: inside a level's grid a coordinate is at most its
// creation extent plus the margin, where the cells' 2 tol of slack covers the
// FP32 rounding of the cell coordinates; outside it coordinates are clamped to
// the boundary cells, which only brings two particles' cells closer.  Primitives
// take their own tolerance, from the particles' and the primitives' coordinates
// (an FP32 plane test rounds both).
#include "dem_internal.cuh"

#define BP_T 128

#include "geometry.cuh"

// FP32 pre-test: can the sphere touch the primitive at all?
// (FP32 copies of the pose: on this part every FP64 instruction, a conversion
// included, costs a multiple of its FP32 counterpart)
static __device__ __forceinline__ bool geom_near(const GeomDev& g, float4 p, float tol) {
    float dx = p.x - g.fc[0], dy = p.y - g.fc[1], dz = p.z - g.fc[2];
    if (g.type == DEM_GEOM_PLANE) {
        float s = g.fn[0] * dx + g.fn[1] * dy + g.fn[2] * dz;
        return s < p.w + tol;
    }
    float reach = g.bound + p.w + tol;
    return dx * dx + dy * dy + dz * dz < reach * reach;
}

// ---------------------------------------------------------------------------
// cell lists (counting sort of particles by cell, rebuilt every step)
// ---------------------------------------------------------------------------
static __device__ __forceinline__ int cell_of(const LevelGrid& g, float4 p, int& cx, int& cy, int& cz) {
    cx = cell_coord(p.x, g.ox, g.inv_cell, g.nx);
    cy = cell_coord(p.y, g.oy, g.inv_cell, g.ny);
    cz = cell_coord(p.z, g.oz, g.inv_cell, g.nz);
    return g.offset + cx + g.nx * (cy + g.ny * cz);
}

__global__ void __launch_bounds__(BP_T) k_cell_count(SimParams P, DevBuf B) {
    __shared__ int lo[3 * DEM_MAX_LEVELS], hi[3 * DEM_MAX_LEVELS];
    for (int t = threadIdx.x; t < 3 * DEM_MAX_LEVELS; t += blockDim.x) {
        lo[t] = 0x7fffffff;
        hi[t] = (int)0x80000000;
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P.n) {
        const int l = B.lvl[i];
        const float4 p = B.posr[i];
        int cx, cy, cz;
        const int c = cell_of(B.lv[l], p, cx, cy, cz);
        B.body_cell[i] = c;
        atomicAdd(&B.cell_cnt[c], 1);
        const float q[3] = {p.x, p.y, p.z};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            atomicMin(&lo[3 * l + k], float_ord(q[k]));
            atomicMax(&hi[3 * l + k], float_ord(q[k]));
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * P.n_levels; t += blockDim.x) {
        if (lo[t] != 0x7fffffff) atomicMin(&B.lvl_lo[t], lo[t]);
        if (hi[t] != (int)0x80000000) atomicMax(&B.lvl_hi[t], hi[t]);
    }
}

// FP32 tolerance bounding the error of an FP32 distance between points whose
// coordinates are at most a in magnitude, for radii up to rmax (see the header)
static __device__ __forceinline__ float fp32_tol(float a, float rmax) {
    return 4.0f * ldexpf(1.25f * a + 8.0f * rmax, -23) + 8.0f * ldexpf(2.0f * rmax, -24);
}

__global__ void __launch_bounds__(BP_T) k_cell_fill(SimParams P, DevBuf B) {
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        // this step's tolerances, from the boxes k_cell_count has just built
        // (an empty level keeps lo > hi)
        float a = 0.0f, rmax = 0.0f;
        for (int t = threadIdx.x; t < 3 * P.n_levels; t += 32) {
            const int lo = B.lvl_lo[t], hi = B.lvl_hi[t];
            if (lo <= hi) a = fmaxf(a, fmaxf(fabsf(ord_float(lo)), fabsf(ord_float(hi))));
        }
        for (int l = threadIdx.x; l < P.n_levels; l += 32) rmax = fmaxf(rmax, B.lv[l].rmax);
        float ag = a;
        for (int g = threadIdx.x; g < P.ng; g += 32)
            ag = fmaxf(ag, fmaxf(fabsf(B.geom[g].fc[0]), fmaxf(fabsf(B.geom[g].fc[1]), fabsf(B.geom[g].fc[2]))));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
            ag = fmaxf(ag, __shfl_xor_sync(0xffffffffu, ag, o));
            rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        }
        if (threadIdx.x == 0) {
            B.tolv[0] = fmaxf(P.tol, fp32_tol(a, rmax));
            B.tolv[1] = fmaxf(P.tol, fp32_tol(ag, rmax));
        }
    }
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    int c = B.body_cell[i];
    int k = B.cell_start[c] + atomicAdd(&B.cell_fill[c], 1);
    // candidates are read in cell order, without the hop through the slot
    B.cell_body[k] = i;
    B.cell_pos[k] = B.posr[i];
    B.cell_id[k] = B.id[i];
}

// ---------------------------------------------------------------------------
// narrow phase
// ---------------------------------------------------------------------------
// PT threads per particle: the candidates of each row of cells are shared out
// across the lanes, hits are compacted into the particle's list with a ballot
// over the lanes, and lane 0 orders the list by the other particle's id.
#ifndef PT
#define PT 8
#endif
#define PT_MASK ((PT) == 32 ? 0xffffffffu : ((1u << (PT)) - 1u))
// Candidates in the FP64 band are queued per particle and decided together
// after the search, so that the FP64 predicate runs on full lanes once
// instead of on one or two lanes in every round of candidates (GB300 issues
// FP64 at 2 lanes per cycle per SM, whatever the number of active lanes).
#ifndef DEM_PAIRS_DEFER
#define DEM_PAIRS_DEFER 1
#endif
#define BAND_CAP 16
__global__ void __launch_bounds__(BP_T) k_pairs(SimParams P, DevBuf B) {
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gt / PT, lane = gt % PT;
    if (i >= P.n || *B.err) return;   // whole groups leave together
    const int grp = (threadIdx.x & 31) / PT;
    const unsigned gmask = PT_MASK << (grp * PT);
    const unsigned below = (1u << lane) - 1u;
    const float4 pi = B.posr[i];
    const double4_32a xi = B.pos[i];
    const float tol = B.tolv[0], tol_g = B.tolv[1];
    const int li = B.lvl[i];
    const int idi = B.id[i];
    int2* own = B.tmp_own + (size_t)i * P.max_own;
    int nown = 0;
    bool overflow = false;
#if DEM_PAIRS_DEFER
    __shared__ int2 band_q[BP_T / PT][BAND_CAP];
    int2* bq = band_q[threadIdx.x / PT];
    int nband = 0;
#endif
    const int lend = B.lv[li].lend, gbeg = B.lv[li].g0, gend = B.lv[li].g1;
    for (int l = li; l < lend; ++l) {
        const LevelGrid g = B.lv[l];
        if (l > li) {
            // skip a coarser level whose particles are all out of reach
            const float reach = pi.w + g.rmax + tol;
            const float q[3] = {pi.x, pi.y, pi.z};
            bool far = false;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                far |= q[k] + reach < ord_float(B.lvl_lo[3 * l + k]) || q[k] - reach > ord_float(B.lvl_hi[3 * l + k]);
            if (far) continue;
        }
        int cx, cy, cz;
        cell_of(g, pi, cx, cy, cz);
        const int x0 = max(cx - 1, 0), x1 = min(cx + 1, g.nx - 1);
        // the candidate ranges of the 3 x 3 rows of cells (z outer, y inner),
        // all loaded at once; out-of-grid rows are empty
        int st[9], pre[10];
        pre[0] = 0;
#pragma unroll
        for (int r = 0; r < 9; ++r) {
            const int z = cz + r / 3 - 1, y = cy + r % 3 - 1;
            int a = 0, b = 0;
            if (z >= 0 && z < g.nz && y >= 0 && y < g.ny) {
                const int row = g.offset + g.nx * (y + g.ny * z);
                a = B.cell_start[row + x0];
                b = B.cell_start[row + x1 + 1];
            }
            st[r] = a;
            pre[r + 1] = pre[r] + (b - a);
        }
        // the rows' candidates as one list, shared out over the lanes in order
        for (int base = 0; base < pre[9]; base += PT) {
            const int t = base + lane;
            bool hit = false, band = false;
            int j = 0, idj = 0;
            if (t < pre[9]) {
                int o = st[0];
#pragma unroll
                for (int r = 1; r < 9; ++r) o = t >= pre[r] ? st[r] - pre[r] : o;
                const int k = t + o;
                // the candidate's position, slot and id load together: a hit
                // waits on one load, not on a chain through its slot
                const float4 pj = B.cell_pos[k];
                j = B.cell_body[k];
                idj = B.cell_id[k];
                const float R = pi.w + pj.w + tol;
                const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
                const float d2 = dx * dx + dy * dy + dz * dz;
                // not itself; same level: the lower id owns the pair
                if (d2 < R * R && idj != idi && !(l == li && idj < idi)) {
                    // FP32 accept (see the header); only the band around
                    // contact takes the FP64 test
                    const float Rin = fmaxf(pi.w + pj.w - tol, 0.0f);
#if DEM_PAIRS_DEFER
                    hit = d2 < Rin * Rin;
                    band = !hit;
#else
                    hit = d2 < Rin * Rin || exact_pair(xi, B.pos[j]);
#endif
                }
            }
#if DEM_PAIRS_DEFER
            {
                // queue the band; a full queue decides the rest at once
                const unsigned bb = (__ballot_sync(gmask, band) >> (grp * PT)) & PT_MASK;
                if (band) {
                    const int q = nband + __popc(bb & below);
                    if (q < BAND_CAP) bq[q] = make_int2(j, idj);
                    else hit = exact_pair(xi, B.pos[j]);
                }
                nband = min(nband + __popc(bb), BAND_CAP);
            }
#endif
            const unsigned bal = (__ballot_sync(gmask, hit) >> (grp * PT)) & PT_MASK;
            if (hit) {
                const int q = nown + __popc(bal & below);
                if (q < P.max_own) {
                    own[q] = make_int2(j, idj);
                    atomicAdd(&B.in_cnt[j], 1);
                } else {
                    overflow = true;
                }
            }
            nown += __popc(bal);
        }
    }
#if DEM_PAIRS_DEFER
    // the queued band, all lanes of the particle at once
    __syncwarp(gmask);
    for (int base = 0; base < nband; base += PT) {
        const int t = base + lane;
        bool hit = false;
        int2 e = make_int2(0, 0);
        if (t < nband) {
            e = bq[t];
            hit = exact_pair(xi, B.pos[e.x]);
        }
        const unsigned bal = (__ballot_sync(gmask, hit) >> (grp * PT)) & PT_MASK;
        if (hit) {
            const int q = nown + __popc(bal & below);
            if (q < P.max_own) {
                own[q] = e;
                atomicAdd(&B.in_cnt[e.x], 1);
            } else {
                overflow = true;
            }
        }
        nown += __popc(bal);
    }
#endif
    int ngeo = 0;
    int* gl = B.tmp_geo + (size_t)i * P.max_geo_body;
    for (int base = gbeg; base < gend; base += PT) {
        const int gi = base + lane;
        bool hit = false;
        if (gi < gend) {
            const GeomDev& g = B.geom[gi];
            hit = geom_near(g, pi, tol_g) && geom_hit(g, xi.x, xi.y, xi.z, xi.w).hit;
        }
        const unsigned bal = (__ballot_sync(gmask, hit) >> (grp * PT)) & PT_MASK;
        if (hit) {
            const int q = ngeo + __popc(bal & below);
            if (q < P.max_geo_body) gl[q] = gi;
            else overflow = true;
        }
        ngeo += __popc(bal);
    }
    __syncwarp(gmask);
    if (lane == 0) {
        // an overflow records the size that would have held this body's lists
        if (nown > P.max_own) atomicMax(&B.need[0], nown);
        if (ngeo > P.max_geo_body) atomicMax(&B.need[1], ngeo);
        nown = min(nown, P.max_own);
        ngeo = min(ngeo, P.max_geo_body);
        // order the list by the other particle's stable id (primitives by index)
        for (int a = 1; a < nown; ++a) {
            const int2 v = own[a];
            int q = a;
            while (q > 0 && own[q - 1].y > v.y) { own[q] = own[q - 1]; --q; }
            own[q] = v;
        }
        for (int a = 1; a < ngeo; ++a) {
            const int v = gl[a];
            int q = a;
            while (q > 0 && gl[q - 1] > v) { gl[q] = gl[q - 1]; --q; }
            gl[q] = v;
        }
        B.own_cnt[i] = nown;
        B.geo_cnt[i] = ngeo;
    }
    if (overflow) set_flag(B.err, DEM_FLAG_CAPACITY);
}

// Owned lists -> contact arrays; both ends of every contact -> incidence lists.
__global__ void __launch_bounds__(BP_T) k_contacts_build(SimParams P, DevBuf B, int parity) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n || *B.err) return;
    const int os = B.own_start[parity][i];
    const int no = B.own_cnt[i];
    const int is = B.inc_start[i];
    const int2* own = B.tmp_own + (size_t)i * P.max_own;
    const long long inc_cap = 2LL * P.max_contacts;
    for (int k = 0; k < no; ++k) {
        const int c = os + k;
        if (c >= P.max_contacts) { set_flag(B.err, DEM_FLAG_CAPACITY); break; }
        const int2 e = own[k];
        B.c_other[c] = e.x;
        B.c_self[c] = i;
        B.c_key[parity][c] = e.y;
        if (is + k < inc_cap) B.inc[is + k] = make_int2(c, e.x);
        const int slot = atomicAdd(&B.in_fill[e.x], 1);
        const long long pos = (long long)B.inc_start[e.x] + B.own_cnt[e.x] + slot;
        if (pos < inc_cap) B.inc[pos] = make_int2(c | (int)0x80000000, i);
        else set_flag(B.err, DEM_FLAG_CAPACITY);
    }
    const int gs = B.geo_start[parity][i];
    const int ng = B.geo_cnt[i];
    const int* gl = B.tmp_geo + (size_t)i * P.max_geo_body;
    const int gcap = P.max_geo;
    for (int k = 0; k < ng; ++k) {
        if (gs + k >= gcap) { set_flag(B.err, DEM_FLAG_CAPACITY); break; }
        B.g_key[parity][gs + k] = gl[k];
        B.g_body[gs + k] = i;
        const int q = B.geom[gl[k]].grp;
        if (q >= 0) {   // a load-driven group: its split mass and its contact list
            atomicAdd(&B.gcnt[q], 1);
            const int slot = atomicAdd(B.gl_count, 1);
            if (slot < gcap) B.gl_list[slot] = make_int2(gs + k, i);
        }
    }
}

// Sort every incidence list by the stable id of the other body, then record
// where each contact sits in the lists of its two bodies.
__global__ void __launch_bounds__(BP_T) k_inc_sort(SimParams P, DevBuf B) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n || *B.err) return;
    const int s = B.inc_start[i], e = B.inc_start[i + 1];
    const int m = e - s;
    const int no = B.own_cnt[i];
    int2* L = B.inc + s;
    if (m - no > 0) {   // incoming entries present: the list needs sorting
        if (m <= 24) {
            int2 ent[24];
            int key[24];
            for (int k = 0; k < m; ++k) {
                int2 v = L[k];
                int q = k;
                int kv = B.id[v.y];
                while (q > 0 && key[q - 1] > kv) { ent[q] = ent[q - 1]; key[q] = key[q - 1]; --q; }
                ent[q] = v;
                key[q] = kv;
            }
            for (int k = 0; k < m; ++k) L[k] = ent[k];
        } else {
            for (int k = 1; k < m; ++k) {
                int2 v = L[k];
                int kv = B.id[v.y];
                int q = k;
                while (q > 0 && B.id[L[q - 1].y] > kv) { L[q] = L[q - 1]; --q; }
                L[q] = v;
            }
        }
    }
    for (int k = 0; k < m; ++k) {
        const int2 v = L[k];
        const int c = v.x & 0x7fffffff;
        if (v.x < 0) {          // b's entry: the other body is the owner a
            B.c_pos[c].y = s + k;
            B.c_idx[c].w = s + k;
        } else {                // the owner's entry: the other body is b
            B.c_pos[c].x = s + k;
            *reinterpret_cast<int2*>(&B.c_idx[c]) = make_int2(i, v.y);
            B.c_idx[c].z = s + k;
        }
    }
}

static inline int nblk(int n, int t) { return n > 0 ? (n + t - 1) / t : 1; }

int launch_cell_count(const SimParams& P, const DevBuf& B, cudaStream_t s) {
    k_cell_count<<<nblk(P.n, BP_T), BP_T, 0, s>>>(P, B);
    return 1;
}
int launch_cell_fill(const SimParams& P, const DevBuf& B, cudaStream_t s) {
    k_cell_fill<<<nblk(P.n, BP_T), BP_T, 0, s>>>(P, B);
    return 1;
}
int launch_pairs(const SimParams& P, const DevBuf& B, cudaStream_t s) {
    k_pairs<<<nblk(P.n * PT, BP_T), BP_T, 0, s>>>(P, B);
    return 1;
}
int launch_contacts_build(const SimParams& P, const DevBuf& B, int parity, cudaStream_t s) {
    k_contacts_build<<<nblk(P.n, BP_T), BP_T, 0, s>>>(P, B, parity);
    return 1;
}
int launch_inc_sort(const SimParams& P, const DevBuf& B, cudaStream_t s) {
    k_inc_sort<<<nblk(P.n, BP_T), BP_T, 0, s>>>(P, B);
    return 1;
}
