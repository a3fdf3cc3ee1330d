// Newton impact stage (Sec. 2.2: high-velocity impacts follow Newton's impact
// law while every other kinematic constraint is kept).
//
// Before the contact rows of a step, a contact whose normal velocity at the
// start of the step u- = n . (v_a - v_b) is below -v_imp is an impact.  In a
// bed with an impact, normal impulses p >= 0 of all its contacts are solved on
// the velocity level,
//     u+ + e_c min(u-, 0) >= 0   complementary to   p >= 0,
//     v+ = v + M^-1 sum_c n_c p_c (signs per side),
// e_c = e for impacts and 0 for the other contacts, by n_it projected Jacobi
// sweeps from p = 0 with the masses split over each body's contacts (as in the
// main solve); primitives keep their velocities.  The impulses act through the
// centres (the lever arms of a sphere contact are along n), so spins are
// unchanged.  The post-impact velocities start the SPOOK step; the impulses on
// primitives are added to the step's primitive impulse.
//
// Layout: one thread per body.  A sweep recomputes each contact's impulse at
// both of its ends from the same inputs (bit-identical) and each end keeps its
// own share, so one kernel per sweep suffices; beds without an impact return
// at once.  Inside a CUDA graph the sweeps sit in the body of a conditional
// (IF) node that the rows' count opens, so a step without any impact costs
// two small kernels.
#include <algorithm>

#include "dem_internal.cuh"
#include "geometry.cuh"

#define IM_T 128

static __device__ __forceinline__ int body_bed(const DevBuf& B, int i) { return B.lv[B.lvl[i]].bed; }

__global__ void __launch_bounds__(IM_T) k_impact_rows(SimParams P, DevBuf B, ImpBuf I, int p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n || *B.err) return;
    const double4_32a xa = B.pos[i];
    const VW sa = B.vw0[i];
    B.vw[0][i] = sa;   // iterate 0
    const float4 va = sa.v;
    const int na = (B.inc_start[i + 1] - B.inc_start[i]) + (B.geo_start[p][i + 1] - B.geo_start[p][i]);
    int hits = 0;
    // sphere-sphere contacts owned by i (a = i); the normal as the contact rows take it
    const int os = B.own_start[p][i], oe = B.own_start[p][i + 1];
    for (int c = os; c < oe; ++c) {
        const int j = B.c_other[c];
        const double4_32a xb = B.pos[j];
        const float4 vb = B.vw0[j].v;
        const int nb = (B.inc_start[j + 1] - B.inc_start[j]) + (B.geo_start[p][j + 1] - B.geo_start[p][j]);
        const double dx = __dsub_rn(xa.x, xb.x), dy = __dsub_rn(xa.y, xb.y), dz = __dsub_rn(xa.z, xb.z);
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        const float inv = 1.0f / sqrtf((float)d2);
        const float3 n = make_float3((float)dx * inv, (float)dy * inv, (float)dz * inv);
        const float u = dot(n, f3(va) - f3(vb));
        const bool hit = u < -P.v_imp;
        I.row[c] = make_float4(n.x, n.y, n.z, 1.0f / (na * va.w + nb * vb.w));
        I.tgt[c] = hit ? P.e_imp * u : 0.0f;
        I.p[0][c] = 0.0f;
        hits += hit;
    }
    // sphere-geometry contacts: the primitive's point velocity enters as n . v_point
    const int gs = B.geo_start[p][i], ge = B.geo_start[p][i + 1];
    for (int k = gs; k < ge; ++k) {
        const GeomDev& G = B.geom[B.g_key[p][k]];
        const GeoHit hh = geom_hit(G, xa.x, xa.y, xa.z, xa.w);
        const float delta = (float)hh.delta;
        const float3 n = make_float3((float)hh.n[0], (float)hh.n[1], (float)hh.n[2]);
        const float3 lever = make_float3((float)(hh.q[0] - G.c[0]) - 0.5f * delta * n.x,
                                         (float)(hh.q[1] - G.c[1]) - 0.5f * delta * n.y,
                                         (float)(hh.q[2] - G.c[2]) - 0.5f * delta * n.z);
        const float3 wg = make_float3((float)G.w[0], (float)G.w[1], (float)G.w[2]);
        const float3 vgp = make_float3((float)G.v[0], (float)G.v[1], (float)G.v[2]) + cross(wg, lever);
        const float kin = dot(n, vgp);
        const float u = dot(n, f3(va)) - kin;
        const bool hit = u < -P.v_imp;
        I.grow[k] = make_float4(n.x, n.y, n.z, 1.0f / (na * va.w));
        I.glev[k] = make_float4(lever.x, lever.y, lever.z, kin);
        I.gtgt[k] = hit ? P.e_imp * u : 0.0f;
        I.gp[0][k] = 0.0f;
        hits += hit;
    }
    if (hits) {
        atomicAdd(I.count, hits);
        I.bed[body_bed(B, i)] = 1;
    }
}

// sweep it: impulses of iterate it + 1 from the velocities of iterate it, then
// this body's velocity of iterate it + 1
__global__ void __launch_bounds__(IM_T) k_impact_sweep(SimParams P, DevBuf B, ImpBuf I, int p, int it) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n || *B.err) return;
    if (!I.bed[body_bed(B, i)] || it >= body_nit(P, B, i)) return;
    const int src = it & 1, dst = src ^ 1;
    const VW* __restrict__ vin = B.vw[src];
    const float3 vi = f3(vin[i].v);
    float3 acc = make_float3(0.f, 0.f, 0.f);
    const int e1 = B.inc_start[i + 1];
    for (int e = B.inc_start[i]; e < e1; ++e) {
        const int2 ent = B.inc[e];
        const bool sideb = ent.x < 0;
        const int c = ent.x & 0x7fffffff;
        const float3 vj = f3(vin[ent.y].v);
        const float4 r = I.row[c];
        const float3 n = f3(r);
        const float u = dot(n, sideb ? vj - vi : vi - vj);
        const float pn = fmaxf(0.0f, I.p[src][c] - r.w * (u + I.tgt[c]));
        if (!sideb) I.p[dst][c] = pn;
        acc = sideb ? acc - pn * n : acc + pn * n;
    }
    const int g1 = B.geo_start[p][i + 1];
    for (int k = B.geo_start[p][i]; k < g1; ++k) {
        const float4 r = I.grow[k];
        const float3 n = f3(r);
        const float u = dot(n, vi) - I.glev[k].w;
        const float pn = fmaxf(0.0f, I.gp[src][k] - r.w * (u + I.gtgt[k]));
        I.gp[dst][k] = pn;
        acc = acc + pn * n;
    }
    const VW s0 = B.vw0[i];
    const float3 v = f3(s0.v) + s0.v.w * acc;
    VW o;
    o.v = make_float4(v.x, v.y, v.z, s0.v.w);
    o.w = s0.w;
    B.vw[dst][i] = o;
}

// the post-impact velocities start the step; the primitives' impulses are
// added to their step impulse (fixed point, as the step's own)
__global__ void __launch_bounds__(IM_T) k_impact_final(SimParams P, DevBuf B, ImpBuf I, int p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n || *B.err) return;
    if (!I.bed[body_bed(B, i)]) return;
    const int nit = body_nit(P, B, i);
    const int last = nit & 1;
    const float4 v = B.vw[last][i].v;
    B.vw0[i].v = v;
    const int g1 = B.geo_start[p][i + 1];
    for (int k = B.geo_start[p][i]; k < g1; ++k) {
        const float pn = nit > 0 ? I.gp[last][k] : 0.0f;
        const float3 n = f3(I.grow[k]);
        const float3 Pg = make_float3(-pn * n.x, -pn * n.y, -pn * n.z);
        const float3 Tg = cross(f3(I.glev[k]), Pg);
        const float vals[6] = {Pg.x, Pg.y, Pg.z, Tg.x, Tg.y, Tg.z};
        const int g = B.g_key[p][k];
#pragma unroll
        for (int c = 0; c < 6; ++c)
            atomicAdd((unsigned long long*)&B.gacc[6 * g + c],
                      (unsigned long long)__double2ll_rn((double)vals[c] * DEM_FIX_SCALE));
    }
}

// opens the conditional body when the step has an impact (one thread: the
// condition must not be set concurrently)
__global__ void k_impact_open(ImpBuf I, cudaGraphConditionalHandle h) {
    if (blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, *I.count > 0 ? 1u : 0u);
}

static inline int nblk(int n, int t) { return n > 0 ? (n + t - 1) / t : 1; }

static void impact_sweeps(const SimParams& P, const DevBuf& B, const ImpBuf& I, int parity, cudaStream_t s) {
    const int blocks = nblk(P.n, IM_T);
    for (int it = 0; it < P.n_it; ++it) k_impact_sweep<<<blocks, IM_T, 0, s>>>(P, B, I, parity, it);
    k_impact_final<<<blocks, IM_T, 0, s>>>(P, B, I, parity);
}

// Returns the kernels launched unconditionally; a negative value is a CUDA
// error code of the graph calls (as -(int)error).
int launch_impact(const SimParams& P, const DevBuf& B, const ImpBuf& I, int parity, cudaStream_t s,
                  cudaStream_t side) {
    cudaMemsetAsync(I.bed, 0, std::max(P.n_beds, 1) * sizeof(int), s);
    cudaMemsetAsync(I.count, 0, sizeof(int), s);
    k_impact_rows<<<nblk(P.n, IM_T), IM_T, 0, s>>>(P, B, I, parity);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g);
    if (e != cudaSuccess) return -(int)e;
    if (cs != cudaStreamCaptureStatusActive) {   // eager: every sweep, beds without an impact return at once
        impact_sweeps(P, B, I, parity, s);
        return 3 + P.n_it;
    }
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess) return -(int)e;
    k_impact_open<<<1, 32, 0, s>>>(I, h);
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t nd = 0;
    if ((e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &nd)) != cudaSuccess) return -(int)e;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, deps, edges, nd, &cp)) != cudaSuccess) return -(int)e;
    // the body: the sweeps and the final update, captured on the side stream
    if ((e = cudaStreamBeginCaptureToGraph(side, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeRelaxed)) != cudaSuccess)
        return -(int)e;
    impact_sweeps(P, B, I, parity, side);
    cudaGraph_t body = nullptr;
    if ((e = cudaStreamEndCapture(side, &body)) != cudaSuccess) return -(int)e;
    // the rest of the step waits for the conditional node
    if ((e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
        cudaSuccess)
        return -(int)e;
    return 4;
}
