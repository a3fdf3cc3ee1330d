// Contact rows, projected Jacobi sweeps and integration of one SPOOK step.
//
// Per contact (Sec. 2.2): normal n from b to a, overlap delta, Hertz mapping
// g = -delta^{e_H}, eps_n = e_H / k_n with k_n = E* sqrt(d*) / 3.  The normal
// row is written for the physical normal impulse p_n: the Hertz Jacobian
// factor J = e_H max(delta, delta_floor)^{e_H - 1} is divided out, giving
//   compliance  Sigma_n = 4 eps_n Y / (dt^2 J^2),  Y = 1 / (1 + 4 tau/dt)
//   right side  b_n     = -(4/dt) Y g / J + Y n.(v_a - v_b) at the step start
// (the SPOOK stepper, Lacoursiere 2007).  Tangential (2 rows) and rolling
// (3 rows) rows have zero right side and compliance eps_reg Sigma_n.
// Each Jacobi sweep updates every contact from the velocities of the previous
// sweep: normal p_n <- max(0, p_n - D_n^{-1} w_n), tangential impulse projected
// on the disc |p_t| <= mu_t p_n (Coulomb, Eq. 6), rolling impulse on the ball
// |p_r| <= mu_r r_eff p_n (Eq. 7), where D are the diagonal blocks of
// G M~^{-1} G^T + Sigma with masses split over each body's contacts (m / n_b).
// The body pass sets v = v* + M^{-1} sum_c G_c^T p_c with v* = v + dt g.
//
// Execution, two layouts here (the resident one is in resident.cu), no atomics:
// - two-pass (k_contact_pass + k_body_pass, chained by programmatic dependent
//   launch): one thread per contact computes its update once and writes each
//   body's impulse share (the sphere-primitive contacts too; those of a
//   load-driven group in k_group_contacts); a thread per body sums its shares
//   in incidence order, then its primitive contacts' shares in list order;
// - one kernel per sweep (k_sweep<T>): T threads per body walk its incidence
//   list (ordered by the other body's stable id) and recompute each contact's
//   update from the two bodies' previous iterates -- the same arithmetic on
//   the same inputs at both ends, so both ends agree bit for bit -- write it
//   if the body owns the contact, and add their own share of the impulse.
// The contact update itself (sweep.cuh) is shared by every layout.  The rows
// and warm starts are set up one thread per contact (k_setup_pairs,
// k_setup_geo) before the sweeps.
#include <algorithm>

#include "dem_internal.cuh"
#include "geometry.cuh"
#include "sweep.cuh"

#define SV_T 128

struct RowC {
    float invDn, rhs, sig, invDt, invDr;
};

// SPOOK constants of one contact.  mlin = split 1/m_a + 1/m_b, mtan = the
// angular part of the tangential diagonal, mrot = split 1/I_a + 1/I_b.
static __device__ __forceinline__ RowC spook_row(const SimParams& P, float delta, float kn, float Gv,
                                                 float mlin, float mtan, float mrot) {
    RowC r;
    const float eps_n = P.e_H / kn;
    const float dfl = fmaxf(delta, P.delta_floor);
    const float J = P.e_H * powf(dfl, P.e_H - 1.0f);
    const float gap = -powf(delta, P.e_H);
    const float sig_scaled = 4.0f * eps_n * P.ups * (P.inv_dt * P.inv_dt);
    r.sig = sig_scaled / (J * J);
    r.rhs = (-4.0f * P.inv_dt * P.ups * gap) / J + P.ups * Gv;
    const float sig_t = P.eps_reg * r.sig;
    r.invDn = 1.0f / (mlin + r.sig);
    r.invDt = 1.0f / (mlin + mtan + sig_t);
    r.invDr = 1.0f / (mrot + sig_t);
    return r;
}

// world-frame warm start -> impulses in the basis of the new normal
static __device__ __forceinline__ void warm_project(float4 w0, float4 w1, float3 n, float4& l0, float2& l1) {
    float3 t1, t2;
    tangent_basis(n, t1, t2);
    const float3 pt = make_float3(w0.y, w0.z, w0.w);
    l0 = make_float4(w0.x, dot(pt, t1), dot(pt, t2), w1.x);
    l1 = make_float2(w1.y, w1.z);
}

// ---------------------------------------------------------------------------
// contact rows + warm start
// ---------------------------------------------------------------------------
// One thread per sphere-sphere contact (grid-stride): its rows from the two
// bodies' state, and its warm start from the previous step's impulse of the
// same pair, found among the contacts the owner held then.
__global__ void __launch_bounds__(SV_T) k_setup_pairs(SimParams P, DevBuf B, int p) {
    if (*B.err) return;
    const int q = p ^ 1;
    const int nc = min(B.own_start[p][P.n], P.max_contacts);
    const bool resorted = *B.resorted != 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        const int i = B.c_self[c], j = B.c_other[c];
        const int key = B.c_key[p][c];
        const double4_32a xa = B.pos[i], xb = B.pos[j];
        const float4 va = B.vw0[i].v, wa = B.vw0[i].w;
        const float4 vb = B.vw0[j].v, wb = B.vw0[j].w;
        const int na = (B.inc_start[i + 1] - B.inc_start[i]) + (B.geo_start[p][i + 1] - B.geo_start[p][i]);
        const int nb = (B.inc_start[j + 1] - B.inc_start[j]) + (B.geo_start[p][j + 1] - B.geo_start[p][j]);
        const int prev = resorted ? B.prev_of[i] : i;
        const int ps = B.own_start[q][prev], pe = B.own_start[q][prev + 1];
        const float ra = (float)xa.w;
        // distance in double, overlap via (R^2 - d^2) / (R + d) to avoid cancellation
        const double dx = __dsub_rn(xa.x, xb.x), dy = __dsub_rn(xa.y, xb.y), dz = __dsub_rn(xa.z, xb.z);
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        const double R = __dadd_rn(xa.w, xb.w);
        const float dist = sqrtf((float)d2);
        const float delta = (float)__dsub_rn(__dmul_rn(R, R), d2) / ((float)R + dist);
        const float inv = 1.0f / dist;
        const float3 n = make_float3((float)dx * inv, (float)dy * inv, (float)dz * inv);
        const float rb = (float)xb.w;
        const float la = ra - 0.5f * delta, lb = rb - 0.5f * delta;
        const float dstar = 2.0f * ra * rb / (ra + rb);   // (1/d_a + 1/d_b)^-1, also r_eff
        const float kn = P.kn_scale * P.Estar_ss * sqrtf(dstar) / 3.0f;
        // Jacobi splits a body's mass over its contacts; Gauss-Seidel does not
        const int sa = P.solver ? 1 : na, sb = P.solver ? 1 : nb;
        const float ima = sa * va.w, imb = sb * vb.w, iIa = sa * wa.w, iIb = sb * wb.w;
        const float Gv = dot(n, f3(va) - f3(vb));
        const RowC rc = spook_row(P, delta, kn, Gv, ima + imb, la * la * iIa + lb * lb * iIb, iIa + iIb);
        B.rec[3 * (size_t)c + 0] = make_float4(n.x, n.y, n.z, rc.invDn);
        B.rec[3 * (size_t)c + 1] = make_float4(rc.rhs, rc.sig, rc.invDt, rc.invDr);
        B.rec[3 * (size_t)c + 2] = make_float4(la, lb, P.mu_t, P.mu_r * dstar);
        B.c_delta[c] = delta;
        // warm start from the previous step's impulse of the same pair (each
        // owner's list is sorted by key)
        int kp = ps;
        while (kp < pe && B.c_key[q][kp] < key) ++kp;
        float4 l0 = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 l1 = make_float2(0.f, 0.f);
        if (kp < pe && B.c_key[q][kp] == key)
            warm_project(B.lamW[q][2 * (size_t)kp], B.lamW[q][2 * (size_t)kp + 1], n, l0, l1);
        B.lamA[0][c] = l0;
        B.lamB[0][c] = l1;
    }
}

// One thread per sphere-primitive contact (grid-stride): its rows and warm start.
__global__ void __launch_bounds__(SV_T) k_setup_geo(SimParams P, DevBuf B, int p) {
    if (*B.err) return;
    const int q = p ^ 1;
    const int ngc = min(B.geo_start[p][P.n], P.max_geo);
    const bool resorted = *B.resorted != 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ngc; k += gridDim.x * blockDim.x) {
        const int i = B.g_body[k];
        const int prev = resorted ? B.prev_of[i] : i;
        const double4_32a xa = B.pos[i];
        const float4 va = B.vw0[i].v, wa = B.vw0[i].w;
        const int na = (B.inc_start[i + 1] - B.inc_start[i]) + (B.geo_start[p][i + 1] - B.geo_start[p][i]);
        const float ra = (float)xa.w;
        const int gps = B.geo_start[q][prev], gpe = B.geo_start[q][prev + 1];
        const int g = B.g_key[p][k];
        const GeomDev& G = B.geom[g];
        // closest point, recomputed with the same routine the detection used
        const GeoHit hh = geom_hit(G, xa.x, xa.y, xa.z, xa.w);
        const double* qq = hh.q;
        const float delta = (float)hh.delta;
        const float3 n = make_float3((float)hh.n[0], (float)hh.n[1], (float)hh.n[2]);
        const float la = ra - 0.5f * delta;
        // contact point in the middle of the overlap (where the sphere's arm
        // ends: half the overlap below the surface point q, n pointing out of
        // the primitive), lever from the primitive's centre
        const float3 lever = make_float3((float)(qq[0] - G.c[0]) - 0.5f * delta * n.x,
                                         (float)(qq[1] - G.c[1]) - 0.5f * delta * n.y,
                                         (float)(qq[2] - G.c[2]) - 0.5f * delta * n.z);
        const float3 wg = make_float3((float)G.w[0], (float)G.w[1], (float)G.w[2]);
        const float3 vgp = make_float3((float)G.v[0], (float)G.v[1], (float)G.v[2]) + cross(wg, lever);
        const float dstar = 2.0f * ra;   // flat primitive: d_b -> infinity
        const float kn = P.kn_scale * G.Estar * sqrtf(dstar) / 3.0f;
        const int sa = P.solver ? 1 : na;
        const float ima = sa * va.w, iIa = sa * wa.w;
        const float Gv = dot(n, f3(va) - vgp);
        const RowC rc = spook_row(P, delta, kn, Gv, ima, la * la * iIa, iIa);
        // side b's split inverse mass: zero for kinematic geometry; a load-driven
        // group's M / n_q along its dynamic axes, which makes the tangential
        // block of D anisotropic (full 2x2 inverse: i11, i12, i22)
        float invDn = rc.invDn, i11 = rc.invDt, i12 = 0.f, i22 = rc.invDt;
        if (G.grp >= 0) {
            const GroupDev& Q = B.grp[G.grp];
            const float imq = (float)B.gcnt[G.grp] * Q.inv_mass;
            const float mx = (Q.dof & 1) ? imq : 0.f, my = (Q.dof & 2) ? imq : 0.f, mz = (Q.dof & 4) ? imq : 0.f;
            float3 t1, t2;
            tangent_basis(n, t1, t2);
            invDn = 1.0f / (ima + (mx * n.x * n.x + my * n.y * n.y + mz * n.z * n.z) + rc.sig);
            const float base = ima + la * la * iIa + P.eps_reg * rc.sig;
            const float d11 = base + (mx * t1.x * t1.x + my * t1.y * t1.y + mz * t1.z * t1.z);
            const float d22 = base + (mx * t2.x * t2.x + my * t2.y * t2.y + mz * t2.z * t2.z);
            const float d12 = mx * t1.x * t2.x + my * t1.y * t2.y + mz * t1.z * t2.z;
            const float idet = 1.0f / (d11 * d22 - d12 * d12);
            i11 = d22 * idet;
            i12 = -d12 * idet;
            i22 = d11 * idet;
        }
        float4* r = B.grec + 6 * (size_t)k;
        r[0] = make_float4(n.x, n.y, n.z, invDn);
        r[1] = make_float4(rc.rhs, rc.sig, i11, rc.invDr);
        r[2] = make_float4(la, G.mu_t, G.mu_r * ra, __int_as_float(g));
        r[3] = make_float4(vgp.x, vgp.y, vgp.z, i12);
        r[4] = make_float4(wg.x, wg.y, wg.z, i22);
        r[5] = make_float4(lever.x, lever.y, lever.z, __int_as_float(G.grp));
        B.g_delta[k] = delta;
        float4 l0 = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 l1 = make_float2(0.f, 0.f);
        for (int kk = gps; kk < gpe; ++kk)
            if (B.g_key[q][kk] == g) {
                warm_project(B.glamW[q][2 * (size_t)kk], B.glamW[q][2 * (size_t)kk + 1], n, l0, l1);
                break;
            }
        B.glamA[0][k] = l0;
        B.glamB[0][k] = l1;
    }
}


// ---------------------------------------------------------------------------
// Body pass (UPDATE = false: v^0 from the warm-start impulses) and projected
// Jacobi sweep (UPDATE = true).  T lanes share one body: lane l takes the
// body's incidence entries l, l+T, l+2T, ... and the lanes' impulse sums are
// combined by a fixed butterfly of shuffles, so the result is deterministic.
// ---------------------------------------------------------------------------
template <int T>
static __device__ __forceinline__ float sub_sum(float v) {
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

static __device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
static __device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// 32-byte records (a body's velocities VW, an impulse share Imp) move in one
// 256-bit vector access (sm_100 and later).  For the body pass's share loads,
// formerly a 128-bit and a 64-bit load, this halves the load requests and
// the L1 throttling (measured on the refined bed: 20.3 -> 19.9 us per sweep);
// elsewhere it fixes the access width.  Both types are 32-byte aligned and
// every device array starts on a 256-byte boundary (checked at allocation).
// The loads are volatile so that they stay after griddepcontrol.wait; the
// share loads stream (evict first).
#ifndef DEM_V8
#define DEM_V8 1
#endif
static __device__ __forceinline__ VW ld_vw(const VW* q) {
#if DEM_V8
    VW r;
    asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(r.v.x), "=f"(r.v.y), "=f"(r.v.z), "=f"(r.v.w), "=f"(r.w.x), "=f"(r.w.y), "=f"(r.w.z),
                   "=f"(r.w.w)
                 : "l"(q));
    return r;
#else
    return *q;
#endif
}
static __device__ __forceinline__ void st_vw(VW* q, const VW& r) {
#if DEM_V8
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(q), "f"(r.v.x), "f"(r.v.y),
                 "f"(r.v.z), "f"(r.v.w), "f"(r.w.x), "f"(r.w.y), "f"(r.w.z), "f"(r.w.w)
                 : "memory");
#else
    *q = r;
#endif
}
static __device__ __forceinline__ void share_store(Imp* q, float3 L, float3 A) {
#if DEM_V8
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %7};" ::"l"(q), "f"(L.x), "f"(L.y),
                 "f"(L.z), "f"(A.x), "f"(A.y), "f"(A.z), "f"(0.0f)
                 : "memory");
#else
    Imp v;
    v.a = make_float4(L.x, L.y, L.z, A.x);
    v.b = make_float4(A.y, A.z, 0.f, 0.f);
    *q = v;
#endif
}
static __device__ __forceinline__ void share_load_cs(const Imp* q, float3& L, float3& A) {
#if DEM_V8
    asm volatile("ld.global.cs.v8.f32 {%0, %1, %2, %3, %4, %5, _, _}, [%6];"
                 : "=f"(L.x), "=f"(L.y), "=f"(L.z), "=f"(A.x), "=f"(A.y), "=f"(A.z)
                 : "l"(q));
#else
    const float4 a = __ldcs(&q->a);
    const float2 b = __ldcs(reinterpret_cast<const float2*>(&q->b));
    L = f3(a);
    A = make_float3(a.w, b.x, b.y);
#endif
}

template <int T, bool UPDATE>
__global__ void __launch_bounds__(SV_T) k_sweep(SimParams P, DevBuf B, int p, int it) {
    if (*B.err) return;
    if (UPDATE) group_clear_ahead(P, B, it);
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gt / T, lane = gt % T;
    bool active = i < P.n;
    // sweep `it` reads iterate it&1 and writes the other; the warm-start body
    // pass (UPDATE = false) reads iterate 0 and writes velocities 0
    const int src = UPDATE ? (it & 1) : 0;
    const int dst = src ^ 1;
    const int nit = active ? body_nit(P, B, i) : 0;
    if (UPDATE) active = active && it < nit;              // this bed has finished its sweeps
    const bool last = UPDATE ? it == nit - 1 : nit == 0;  // write the final impulses
    const VW* __restrict__ vin = UPDATE ? B.vw[src] : B.vw0;
    const float4* __restrict__ lAin = B.lamA[src];
    const float2* __restrict__ lBin = B.lamB[src];
    float3 accL = make_float3(0.f, 0.f, 0.f), accA = make_float3(0.f, 0.f, 0.f);
    if (active) {
        const VW me = ld_vw(vin + i);
        const float3 vi = f3(me.v), wi = f3(me.w);
        const int e1 = B.inc_start[i + 1];
        int e = B.inc_start[i] + lane;
        int2 nxt = e < e1 ? B.inc[e] : make_int2(0, 0);
        for (; e < e1; e += T) {
            const int2 ent = nxt;
            if (e + T < e1) nxt = B.inc[e + T];   // fetch the next entry before this one's data
            const bool sideb = ent.x < 0;
            const int c = ent.x & 0x7fffffff;
            const float4 r0 = B.rec[3 * (size_t)c], r2 = B.rec[3 * (size_t)c + 2];
            const float4 l0 = lAin[c];
            const float2 l1 = lBin[c];
            const float3 n = f3(r0);
            Upd u;
            if (UPDATE) {
                const int j = ent.y;
                const float4 r1 = B.rec[3 * (size_t)c + 1];
                const VW other = ld_vw(vin + j);
                const float3 vj = f3(other.v), wj = f3(other.w);
                const float3 dv = sideb ? vj - vi : vi - vj;
                const float3 wa = sideb ? wj : wi, wb = sideb ? wi : wj;
                u = contact_update(r0, r1, r2.x, r2.y, r2.z, r2.w, l0, l1, dv, wa, wb, P.eps_reg);
                if (!sideb && !last) {
                    B.lamA[dst][c] = make_float4(u.pn, u.pt1, u.pt2, u.pr.x);
                    B.lamB[dst][c] = make_float2(u.pr.y, u.pr.z);
                }
            } else {
                tangent_basis(n, u.t1, u.t2);
                u.pn = l0.x; u.pt1 = l0.y; u.pt2 = l0.z; u.pr = make_float3(l0.w, l1.x, l1.y);
            }
            if (last && !sideb) write_world(B.lamW[p], c, n, u);
            add_impulse(n, u.t1, u.t2, sideb ? r2.y : r2.x, u.pn, u.pt1, u.pt2, u.pr, sideb, accL, accA);
        }
        const int g1 = B.geo_start[p][i + 1];
        for (int k = B.geo_start[p][i] + lane; k < g1; k += T) {
            const float4* r = B.grec + 6 * (size_t)k;
            const float4 r0 = r[0], r2 = r[2];
            const float4 l0 = B.glamA[src][k];
            const float2 l1 = B.glamB[src][k];
            const float3 n = f3(r0);
            Upd u;
            bool done = false;
            if (UPDATE) {
                u = geom_update(P, B, r, k, src, it, vi, wi, done);
                if (!last && !done) {
                    B.glamA[dst][k] = make_float4(u.pn, u.pt1, u.pt2, u.pr.x);
                    B.glamB[dst][k] = make_float2(u.pr.y, u.pr.z);
                }
            } else {
                tangent_basis(n, u.t1, u.t2);
                u.pn = l0.x; u.pt1 = l0.y; u.pt2 = l0.z; u.pr = make_float3(l0.w, l1.x, l1.y);
                const int q = __float_as_int(r[5].w);
                if (q >= 0)   // the warm start's impulse on a load-driven group: iterate 0
                    group_add(B, q, 0, (-1.0f) * (u.pn * n + lin2(u.pt1, u.t1, u.pt2, u.t2)));
            }
            if (last && !done) write_world(B.glamW[p], k, n, u);
            add_impulse(n, u.t1, u.t2, r2.x, u.pn, u.pt1, u.pt2, u.pr, false, accL, accA);
        }
    }
    if (T > 1) {
        accL = make_float3(sub_sum<T>(accL.x), sub_sum<T>(accL.y), sub_sum<T>(accL.z));
        accA = make_float3(sub_sum<T>(accA.x), sub_sum<T>(accA.y), sub_sum<T>(accA.z));
    }
    if (!active || lane != 0) return;
    const VW s0 = ld_vw(B.vw0 + i);
    const float4 v0 = s0.v, w0 = s0.w;
    const float gm = v0.w > 0.0f ? P.dt : 0.0f;
    const float3 vs = make_float3(v0.x + gm * P.gx, v0.y + gm * P.gy, v0.z + gm * P.gz);
    const float3 v = vs + v0.w * accL;
    const float3 w = f3(w0) + w0.w * accA;
    VW o;
    o.v = make_float4(v.x, v.y, v.z, v0.w);
    o.w = make_float4(w.x, w.y, w.z, w0.w);
    st_vw(B.vw[UPDATE ? dst : 0] + i, o);
}

// ---------------------------------------------------------------------------
// x += dt v (SPOOK position update), geometry forces, kinematic geometry
// ---------------------------------------------------------------------------
#define SMEM_GEOM 64   // up to this many primitives the block sums impulses in shared memory
__global__ void __launch_bounds__(SV_T) k_integrate(SimParams P, DevBuf B, int p) {
    __shared__ long long sacc[6 * SMEM_GEOM];
    const bool small = P.ng <= SMEM_GEOM;
    if (small)
        for (int t = threadIdx.x; t < 6 * P.ng; t += blockDim.x) sacc[t] = 0;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool ok = !*B.err;
    if (i < P.n && ok) {
        // the bed's final iterate (Gauss-Seidel updates one buffer in place)
        const int src = P.solver ? 0 : body_nit(P, B, i) & 1;
        const float4 v = B.vw[src][i].v, w = B.vw[src][i].w;
        if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(w.x) && isfinite(w.y) &&
              isfinite(w.z)))
            set_flag(B.err, DEM_FLAG_NONFINITE);
        B.vw0[i].v = v;
        B.vw0[i].w = w;
        double4_32a x = B.pos[i];
        const double h = (double)P.dt;
        x.x = __dadd_rn(x.x, __dmul_rn(h, (double)v.x));
        x.y = __dadd_rn(x.y, __dmul_rn(h, (double)v.y));
        x.z = __dadd_rn(x.z, __dmul_rn(h, (double)v.z));
        B.pos[i] = x;
        B.posr[i] = make_float4((float)x.x, (float)x.y, (float)x.z, (float)x.w);
    }
    if (ok) {
        // the primitives' impulses, one thread per sphere-primitive contact (full
        // lanes for the conversions to fixed point, which run on the FP64 pipe)
        const int ngc = min(B.geo_start[p][P.n], P.max_geo);
        for (int k = i; k < ngc; k += gridDim.x * blockDim.x) {
            const float4* r = B.grec + 6 * (size_t)k;
            const float4 r0 = r[0], r2 = r[2], r5 = r[5];
            const float4 W0 = B.glamW[p][2 * (size_t)k], W1 = B.glamW[p][2 * (size_t)k + 1];
            const int g = __float_as_int(r2.w);
            // impulse of the particle on the primitive: -(p_n n + p_t) at the lever, -p_r
            const float3 Pg = make_float3(-(W0.x * r0.x + W0.y), -(W0.x * r0.y + W0.z), -(W0.x * r0.z + W0.w));
            const float3 Tg = cross(f3(r5), Pg) - make_float3(W1.x, W1.y, W1.z);
            const float vals[6] = {Pg.x, Pg.y, Pg.z, Tg.x, Tg.y, Tg.z};
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const unsigned long long q = (unsigned long long)__double2ll_rn((double)vals[c] * DEM_FIX_SCALE);
                atomicAdd(small ? (unsigned long long*)&sacc[6 * g + c] : (unsigned long long*)&B.gacc[6 * g + c], q);
            }
        }
    }
    __syncthreads();
    if (small)
        for (int t = threadIdx.x; t < 6 * P.ng; t += blockDim.x)
            if (sacc[t] != 0) atomicAdd((unsigned long long*)&B.gacc[t], (unsigned long long)sacc[t]);
    // a faulted step is not committed: primitives, groups and the re-sort
    // mapping stay as they were, so the step can be re-run
    if (blockIdx.x == 0 && threadIdx.x == 0 && ok) {
        ++*B.committed;
        // load-driven groups: the solved velocity of the final iterate moves
        // the members along the dynamic axes
        for (int q = 0; q < P.n_groups; ++q) {
            double vf[3];
            group_velocity_d(P, B, q, B.grp[q].nit, vf);
            for (int ax = 0; ax < 3; ++ax) B.grp[q].v[ax] = vf[ax];
        }
        for (int g = 0; g < P.ng; ++g)
            if (B.geom[g].grp >= 0)
                for (int ax = 0; ax < 3; ++ax) B.geom[g].v[ax] = B.grp[B.geom[g].grp].v[ax];
        // kinematic primitives: translate with v, rotate with w (Rodrigues)
        const double h = (double)P.dt;
        for (int g = 0; g < P.ng; ++g) {
            GeomDev& G = B.geom[g];
            for (int c = 0; c < 3; ++c) G.c[c] = __dadd_rn(G.c[c], __dmul_rn(h, G.v[c]));
            const double wn = sqrt(G.w[0] * G.w[0] + G.w[1] * G.w[1] + G.w[2] * G.w[2]);
            if (wn > 0.0) {
                const double ax[3] = {G.w[0] / wn, G.w[1] / wn, G.w[2] / wn};
                const double th = wn * h, cs = cos(th), sn = sin(th);
                double Rot[3][3];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) Rot[a][b] = (a == b ? cs : 0.0) + (1.0 - cs) * ax[a] * ax[b];
                Rot[0][1] -= sn * ax[2]; Rot[0][2] += sn * ax[1];
                Rot[1][0] += sn * ax[2]; Rot[1][2] -= sn * ax[0];
                Rot[2][0] -= sn * ax[1]; Rot[2][1] += sn * ax[0];
                double Rn[9];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        Rn[3 * a + b] = Rot[a][0] * G.R[b] + Rot[a][1] * G.R[3 + b] + Rot[a][2] * G.R[6 + b];
                for (int k = 0; k < 9; ++k) G.R[k] = Rn[k];
            }
            for (int k = 0; k < 3; ++k) { G.fc[k] = (float)G.c[k]; G.fn[k] = (float)G.R[3 * k + 2]; }
        }
        *B.resorted = 0;
    }
}

static inline int nblk(int n, int t) { return n > 0 ? (n + t - 1) / t : 1; }

static int sm_count();

int launch_setup(const SimParams& P, const DevBuf& B, int parity, cudaStream_t s) {
    const int cblocks = std::max(1, std::min(nblk(P.max_contacts, SV_T), 16 * sm_count()));
    k_setup_pairs<<<cblocks, SV_T, 0, s>>>(P, B, parity);
    const int gblocks = std::max(1, std::min(nblk(P.max_geo, SV_T), 4 * sm_count()));
    k_setup_geo<<<gblocks, SV_T, 0, s>>>(P, B, parity);
    return 2;
}
// ---------------------------------------------------------------------------
// Two-pass sweep.  Contact pass: one thread per contact computes its update
// once from the two bodies' previous iterates, stores the new impulse and the
// impulse share of each body at the contact's position in that body's
// incidence list.  Body pass: each body adds its shares in list order (stable
// id of the other body), updates its geometry contacts, and forms
// v = v* + M^-1 sum.  Successive passes are chained with programmatic
// dependent launch: a pass may start while the previous one drains and waits
// (griddepcontrol.wait) before reading what it produced.
// ---------------------------------------------------------------------------

// Both passes read what the step produced before its sweeps (the fault flag,
// each contact's bodies and incidence positions, its rows, each body's
// incidence range and start velocity) before waiting for the previous pass, so
// those loads overlap that pass's tail; only the iterates (impulses,
// velocities, shares) are read after the wait.  None of the sweep kernels
// writes the fault flag, so reading it early sees the step's value.
//
// Launch shape and register budgets of the two passes, chosen by timing on
// the 200k refined bed (GB300): the contact pass at 64 registers (8 blocks of
// 128 threads per SM, a grid of 16 blocks per SM, the next contact's indices
// and rows prefetched), the body pass at 80 registers over one resident wave
// of 6 blocks per SM.  Tighter budgets spill and lose more than the extra
// warps gain.
#ifndef DEM_CP_BLOCKS_PER_SM
#define DEM_CP_BLOCKS_PER_SM 16
#endif
#ifndef DEM_CP_MINB
#define DEM_CP_MINB 8
#endif
#ifndef DEM_CP_PIPE
#define DEM_CP_PIPE 1
#endif
#ifndef DEM_BP_GEO_NOINLINE
#define DEM_BP_GEO_NOINLINE 0
#endif
#ifndef DEM_BP_BLOCKS_PER_SM
#define DEM_BP_BLOCKS_PER_SM 6
#endif
#ifndef DEM_BP_MINB
#define DEM_BP_MINB 6
#endif
// Sphere-primitive contacts are updated in the contact pass (those of a
// load-driven group in k_group_contacts, between the passes), which writes
// each one's impulse share (gsh); the body pass then only adds shares
// (summed in the same order, so the results are bit-identical).  Measured on
// the refined bed, its best shape is a grid-stride over one resident wave of
// 6 blocks per SM at 80 registers, each thread fetching the next body's range
// ahead (20.4 against 22.3 us per sweep with the primitive contacts in the
// body pass).
#ifndef DEM_GEO_IN_CP
#define DEM_GEO_IN_CP 1
#endif
#ifndef DEM_BP_MINB_SHARES
#define DEM_BP_MINB_SHARES 6
#endif
#ifndef DEM_BP_BLOCKS_PER_SM_SHARES
#define DEM_BP_BLOCKS_PER_SM_SHARES 6   // 0: one body per thread
#endif
__global__ void __launch_bounds__(SV_T, DEM_CP_MINB) k_contact_pass(SimParams P, DevBuf B, int p, int it, int nact) {
    const int bad = *B.err;
    // contacts are stored in owner order: those of the active prefix come first
    const int nc = min(B.own_start[p][nact], P.max_contacts);
    const int stride = gridDim.x * blockDim.x;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    bool have = c < nc;
    int4 id = make_int4(0, 0, 0, 0);
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
    if (have) {
        id = B.c_idx[c];
        r0 = B.rec[3 * (size_t)c];
        r1 = B.rec[3 * (size_t)c + 1];
        r2 = B.rec[3 * (size_t)c + 2];
    }
    pdl_wait();
    pdl_trigger();
    if (bad) return;
    group_clear_ahead(P, B, it);
    const int src = it & 1, dst = src ^ 1;
    const VW* __restrict__ vin = B.vw[src];
    while (have) {
        const int nit = body_nit(P, B, id.x);
        const bool run = it < nit;            // else this bed has finished its sweeps
        float4 l0 = make_float4(0.f, 0.f, 0.f, 0.f);
        float2 l1 = make_float2(0.f, 0.f);
        VW A, Bv;
        if (run) {
            // the previous iterate is dead after this read: stream it (evict first)
            l0 = __ldcs(&B.lamA[src][c]);
            l1 = __ldcs(&B.lamB[src][c]);
            A = ld_vw(vin + id.x);
            Bv = ld_vw(vin + id.y);
        }
#if DEM_CP_PIPE
        // the next contact's indices and rows, fetched while this one's
        // iterates are in flight
        const int cn = c + stride;
        const bool hn = cn < nc;
        int4 idn = id;
        float4 n0 = r0, n1 = r1, n2 = r2;
        if (hn) {
            idn = B.c_idx[cn];
            n0 = B.rec[3 * (size_t)cn];
            n1 = B.rec[3 * (size_t)cn + 1];
            n2 = B.rec[3 * (size_t)cn + 2];
        }
#endif
        if (run) {
            const bool last = it == nit - 1;
            const float3 va = f3(A.v), wa = f3(A.w), vb = f3(Bv.v), wb = f3(Bv.w);
            const Upd u = contact_update(r0, r1, r2.x, r2.y, r2.z, r2.w, l0, l1, va - vb, wa, wb, P.eps_reg);
            const float3 n = f3(r0);
            if (last) {
                write_world(B.lamW[p], c, n, u);
            } else {
                B.lamA[dst][c] = make_float4(u.pn, u.pt1, u.pt2, u.pr.x);
                B.lamB[dst][c] = make_float2(u.pr.y, u.pr.z);
            }
            float3 La = make_float3(0.f, 0.f, 0.f), Aa = La, Lb = La, Ab = La;
            add_impulse(n, u.t1, u.t2, r2.x, u.pn, u.pt1, u.pt2, u.pr, false, La, Aa);
            add_impulse(n, u.t1, u.t2, r2.y, u.pn, u.pt1, u.pt2, u.pr, true, Lb, Ab);
            share_store(&B.imp[id.z], La, Aa);
            share_store(&B.imp[id.w], Lb, Ab);
        }
#if DEM_CP_PIPE
        c = cn;
        have = hn;
        id = idn;
        r0 = n0; r1 = n1; r2 = n2;
#else
        c += stride;
        have = c < nc;
        if (have) {
            id = B.c_idx[c];
            r0 = B.rec[3 * (size_t)c];
            r1 = B.rec[3 * (size_t)c + 1];
            r2 = B.rec[3 * (size_t)c + 2];
        }
#endif
    }
#if DEM_GEO_IN_CP
    {
        // sphere-primitive contacts: the update geom_update makes, its impulse
        // share on the body stored for the body pass (a load-driven group's
        // contacts are left to k_group_contacts, which stores theirs)
        const int ngc = min(B.geo_start[p][nact], P.max_geo);
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ngc; k += stride) {
            const int i = B.g_body[k];
            const int nit = body_nit(P, B, i);
            if (it >= nit) continue;
            const float4* r = B.grec + 6 * (size_t)k;
            if (P.n_groups > 0 && __float_as_int(r[5].w) >= 0) continue;
            const float4 g0 = r[0], g1 = r[1], g2 = r[2], g3 = r[3], g4 = r[4];
            const float4 l0 = __ldcs(&B.glamA[src][k]);
            const float2 l1 = __ldcs(&B.glamB[src][k]);
            const VW me = ld_vw(vin + i);
            const Upd u = contact_update(g0, g1, g2.x, 0.0f, g2.y, g2.z, l0, l1, f3(me.v) - f3(g3), f3(me.w),
                                         f3(g4), P.eps_reg);
            const float3 n = f3(g0);
            if (it == nit - 1) {
                write_world(B.glamW[p], k, n, u);
            } else {
                B.glamA[dst][k] = make_float4(u.pn, u.pt1, u.pt2, u.pr.x);
                B.glamB[dst][k] = make_float2(u.pr.y, u.pr.z);
            }
            float3 La = make_float3(0.f, 0.f, 0.f), Aa = La;
            add_impulse(n, u.t1, u.t2, g2.x, u.pn, u.pt1, u.pt2, u.pr, false, La, Aa);
            share_store(&B.gsh[k], La, Aa);
        }
    }
#endif
}

// A body's sphere-geometry contacts at sweep it: updated from its iterate,
// their impulses added to (accL, accA) in list order.  Few bodies touch a
// primitive; out of line, this path does not set the register budget of the
// body pass's common path.
#if DEM_BP_GEO_NOINLINE
static __device__ __noinline__
#else
static __device__ __forceinline__
#endif
void body_geom_contacts(const SimParams& P, const DevBuf& B, int p, int it, int i, int k0, int k1, bool last,
                        float3& accL, float3& accA) {
    const int src = it & 1, dst = src ^ 1;
    const VW me = B.vw[src][i];
    const float3 vi = f3(me.v), wi = f3(me.w);
    for (int k = k0; k < k1; ++k) {
        const float4* r = B.grec + 6 * (size_t)k;
        const float4 r0 = r[0], r2 = r[2];
        const float3 n = f3(r0);
        bool done;
        const Upd u = geom_update(P, B, r, k, src, it, vi, wi, done);
        if (done) {
        } else if (last) {
            write_world(B.glamW[p], k, n, u);
        } else {
            B.glamA[dst][k] = make_float4(u.pn, u.pt1, u.pt2, u.pr.x);
            B.glamB[dst][k] = make_float2(u.pr.y, u.pr.z);
        }
        add_impulse(n, u.t1, u.t2, r2.x, u.pn, u.pt1, u.pt2, u.pr, false, accL, accA);
    }
}

// The body pass loads a body's shares DEM_BP_CHUNK at a time, all before it
// adds them, then adds them one by one in incidence order: the loads are in
// flight together, the sum keeps its fixed order (and so its rounding).
#ifndef DEM_BP_CHUNK
#define DEM_BP_CHUNK 4
#endif
// One body's sum of its impulse shares in incidence order, its geometry
// contacts, and v = v* + M^-1 sum.
template <bool GEO>
static __device__ __forceinline__ void body_update(const SimParams& P, const DevBuf& B, int p, int it, int i,
                                                   int nit, int e0, int e1, int k0, int k1, float4 v0, float4 w0) {
    const bool last = it == nit - 1;
    const int dst = (it & 1) ^ 1;
    float3 accL = make_float3(0.f, 0.f, 0.f), accA = accL;
    for (int e = e0; e < e1; e += DEM_BP_CHUNK) {
        // a share is read once, by its body: stream it
        float3 qL[DEM_BP_CHUNK], qA[DEM_BP_CHUNK];
#pragma unroll
        for (int u = 0; u < DEM_BP_CHUNK; ++u)
            if (e + u < e1) share_load_cs(&B.imp[e + u], qL[u], qA[u]);
#pragma unroll
        for (int u = 0; u < DEM_BP_CHUNK; ++u)
            if (e + u < e1) {
                accL = accL + qL[u];
                accA = accA + qA[u];
            }
    }
    if (GEO) {
        if (k0 < k1) body_geom_contacts(P, B, p, it, i, k0, k1, last, accL, accA);
    } else {
        for (int k = k0; k < k1; ++k) {   // shares of the contact pass, in list order
            float3 qL, qA;
            share_load_cs(&B.gsh[k], qL, qA);
            accL = accL + qL;
            accA = accA + qA;
        }
    }
    const float gm = v0.w > 0.0f ? P.dt : 0.0f;
    const float3 vs = make_float3(v0.x + gm * P.gx, v0.y + gm * P.gy, v0.z + gm * P.gz);
    const float3 v = vs + v0.w * accL;
    const float3 w = f3(w0) + w0.w * accA;
    VW out;
    out.v = make_float4(v.x, v.y, v.z, v0.w);
    out.w = make_float4(w.x, w.y, w.z, w0.w);
    st_vw(B.vw[dst] + i, out);
}

// GEO: the body updates its sphere-primitive contacts itself (objects with
// load-driven groups); else it adds their shares from the contact pass
template <bool GEO>
__global__ void __launch_bounds__(SV_T, GEO ? DEM_BP_MINB : DEM_BP_MINB_SHARES)
    k_body_pass(SimParams P, DevBuf B, int p, int it, int nact) {
    const int bad = *B.err;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    // the (first) body's incidence range and start velocity, before the wait
    int nit = 0, e0 = 0, e1 = 0, k0 = 0, k1 = 0;
    float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), w0 = v0;
    if (i < nact) {
        nit = body_nit(P, B, i);
        e0 = B.inc_start[i];
        e1 = B.inc_start[i + 1];
        k0 = B.geo_start[p][i];
        k1 = B.geo_start[p][i + 1];
        const VW s0 = ld_vw(B.vw0 + i);
        v0 = s0.v;
        w0 = s0.w;
    }
    pdl_wait();
    pdl_trigger();
    if (bad) return;
    if constexpr ((GEO ? DEM_BP_BLOCKS_PER_SM : DEM_BP_BLOCKS_PER_SM_SHARES) > 0) {
    // grid-stride over the bodies, the next body's range fetched ahead
    const int stride = gridDim.x * blockDim.x;
    for (; i < nact; i += stride) {
        if (it < nit) body_update<GEO>(P, B, p, it, i, nit, e0, e1, k0, k1, v0, w0);
        const int j = i + stride;
        if (j < nact) {
            nit = body_nit(P, B, j);
            e0 = B.inc_start[j];
            e1 = B.inc_start[j + 1];
            k0 = B.geo_start[p][j];
            k1 = B.geo_start[p][j + 1];
            const VW s0 = ld_vw(B.vw0 + j);
            v0 = s0.v;
            w0 = s0.w;
        }
    }
    } else {
    // one body per thread (else this bed has finished its sweeps)
    if (i < nact && it < nit) body_update<GEO>(P, B, p, it, i, nit, e0, e1, k0, k1, v0, w0);
    }
}

// Contacts of load-driven groups at sweep it, one thread each: from the body's
// iterate v^it and the group's, the new impulse (written where the sweep's
// body update reads it) and its share of the group's sum for iterate it + 1.
__global__ void __launch_bounds__(SV_T) k_group_contacts(SimParams P, DevBuf B, int p, int it) {
    if (*B.err) return;
    const int m = min(*B.gl_count, P.max_geo);
    const int src = it & 1, dst = src ^ 1;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
        const int2 e = B.gl_list[t];
        const int k = e.x, i = e.y;
        const int nit = body_nit(P, B, i);
        if (it >= nit) continue;
        const float4* r = B.grec + 6 * (size_t)k;
        const VW me = B.vw[src][i];
        const Upd u = geom_update_group(P, B, r, B.glamA[src][k], B.glamB[src][k], f3(me.v), f3(me.w),
                                        __float_as_int(r[5].w), it);
        B.glamA[dst][k] = make_float4(u.pn, u.pt1, u.pt2, u.pr.x);
        B.glamB[dst][k] = make_float2(u.pr.y, u.pr.z);
        if (it == nit - 1) write_world(B.glamW[p], k, f3(r[0]), u);
#if DEM_GEO_IN_CP
        // the impulse share on the body, for the shares-only body pass
        float3 La = make_float3(0.f, 0.f, 0.f), Aa = La;
        add_impulse(f3(r[0]), u.t1, u.t2, r[2].x, u.pn, u.pt1, u.pt2, u.pr, false, La, Aa);
        share_store(&B.gsh[k], La, Aa);
#endif
    }
}

int launch_group_contacts(const SimParams& P, const DevBuf& B, int parity, int it, cudaStream_t s) {
    if (P.n_groups == 0) return 0;
    k_group_contacts<<<64, SV_T, 0, s>>>(P, B, parity, it);
    return 1;
}

// ---------------------------------------------------------------------------
// Coloured projected Gauss-Seidel
// ---------------------------------------------------------------------------
static int sm_count();
// SplitMix64 finaliser (Steele, Lea and Flood 2014; Vigna): a contact's
// priority is the mix of its key (lower stable id, higher stable id) or
// (stable id, -(primitive + 1)); higher priority colours first.
static __device__ __forceinline__ unsigned long long pgs_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

__global__ void __launch_bounds__(SV_T) k_pgs_prepare(SimParams P, DevBuf B, PgsBuf S, int p, int nc, int ngc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < P.n)   // body of every sphere-geometry contact
        for (int k = B.geo_start[p][t]; k < B.geo_start[p][t + 1]; ++k) S.gbody[k] = t;
    if (t == 0) {
        *S.remaining = nc + ngc;
        *S.ncol = 0;
    }
    if (t < PGS_MAX_COLOURS) {
        S.colcnt[t] = 0;
        S.colfill[t] = 0;
    }
}

__global__ void __launch_bounds__(SV_T) k_pgs_keys(SimParams P, DevBuf B, PgsBuf S, int p, int nc, int ngc) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nc + ngc) return;
    unsigned long long key;
    if (u < nc) {
        const int ia = B.id[B.c_self[u]], ib = B.id[B.c_other[u]];
        const int lo = min(ia, ib), hi = max(ia, ib);
        key = ((unsigned long long)(unsigned)lo << 32) | (unsigned)hi;
    } else {
        const int k = u - nc;
        key = ((unsigned long long)(unsigned)B.id[S.gbody[k]] << 32) | (unsigned)(-(B.g_key[p][k] + 1));
    }
    S.key[u] = key;
    S.prio[u] = pgs_mix(key);
    S.col[u] = -1;
}

static __device__ __forceinline__ bool pgs_before(const PgsBuf& S, int m, int u) {
    const unsigned long long pm = S.prio[m], pu = S.prio[u];
    return pm != pu ? pm > pu : S.key[m] < S.key[u];
}

// One Jones-Plassmann round: an uncoloured contact whose higher-priority
// neighbours (contacts sharing a body) are all coloured takes the smallest
// colour none of them has -- the greedy colouring in priority order.
__global__ void __launch_bounds__(SV_T) k_pgs_round(SimParams P, DevBuf B, PgsBuf S, int p, int nc, int ngc) {
    volatile int* col = S.col;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nc + ngc; u += gridDim.x * blockDim.x) {
        if (col[u] >= 0) continue;
        int body[2];
        if (u < nc) { body[0] = B.c_self[u]; body[1] = B.c_other[u]; }
        else { body[0] = S.gbody[u - nc]; body[1] = -1; }
        unsigned long long used[2] = {0ull, 0ull};
        bool blocked = false;
        for (int s2 = 0; s2 < 2 && !blocked; ++s2) {
            const int i = body[s2];
            if (i < 0) continue;
            for (int e = B.inc_start[i]; e < B.inc_start[i + 1] && !blocked; ++e) {
                const int m = B.inc[e].x & 0x7fffffff;
                if (m == u) continue;
                const int cm = col[m];
                if (cm >= 0) used[cm >> 6] |= 1ull << (cm & 63);
                else blocked = pgs_before(S, m, u);
            }
            for (int k = B.geo_start[p][i]; k < B.geo_start[p][i + 1] && !blocked; ++k) {
                const int m = nc + k;
                if (m == u) continue;
                const int cm = col[m];
                if (cm >= 0) used[cm >> 6] |= 1ull << (cm & 63);
                else blocked = pgs_before(S, m, u);
            }
        }
        if (blocked) continue;
        const int c = ~used[0] ? __ffsll((long long)~used[0]) - 1 : (~used[1] ? 64 + __ffsll((long long)~used[1]) - 1 : -1);
        if (c < 0) {
            set_flag(B.err, DEM_FLAG_CAPACITY);   // more than PGS_MAX_COLOURS colours
            col[u] = PGS_MAX_COLOURS - 1;
        } else {
            col[u] = c;
        }
        atomicSub(S.remaining, 1);
        atomicMax(S.ncol, (c < 0 ? PGS_MAX_COLOURS - 1 : c) + 1);
    }
}

// fill = false: count per colour; true: list the contacts by colour
__global__ void __launch_bounds__(SV_T) k_pgs_bucket(PgsBuf S, int total, int fill) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= total) return;
    const int c = S.col[u];
    if (!fill) atomicAdd(&S.colcnt[c], 1);
    else S.list[S.colstart[c] + atomicAdd(&S.colfill[c], 1)] = u;
}

// Contacts of one colour: each update's impulse change goes into its bodies at
// once; no two contacts of a colour share a body.  Iterate buffer 0 in place.
__global__ void __launch_bounds__(SV_T) k_pgs_colour(SimParams P, DevBuf B, PgsBuf S, int p, int nc, int first,
                                                    int count, int last) {
    if (*B.err) return;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
        const int u = S.list[first + t];
        float3 La = make_float3(0.f, 0.f, 0.f), Aa = La, Lb = La, Ab = La;
        if (u < nc) {
            const int c = u, a = B.c_self[c], b = B.c_other[c];
            const float4 r0 = B.rec[3 * (size_t)c], r1 = B.rec[3 * (size_t)c + 1], r2 = B.rec[3 * (size_t)c + 2];
            const float4 l0 = B.lamA[0][c];
            const float2 l1 = B.lamB[0][c];
            VW A = B.vw[0][a], Bv = B.vw[0][b];
            const Upd u2 = contact_update(r0, r1, r2.x, r2.y, r2.z, r2.w, l0, l1, f3(A.v) - f3(Bv.v), f3(A.w),
                                          f3(Bv.w), P.eps_reg);
            const float3 n = f3(r0);
            const float3 dpr = u2.pr - make_float3(l0.w, l1.x, l1.y);
            add_impulse(n, u2.t1, u2.t2, r2.x, u2.pn - l0.x, u2.pt1 - l0.y, u2.pt2 - l0.z, dpr, false, La, Aa);
            add_impulse(n, u2.t1, u2.t2, r2.y, u2.pn - l0.x, u2.pt1 - l0.y, u2.pt2 - l0.z, dpr, true, Lb, Ab);
            A.v = make_float4(A.v.x + A.v.w * La.x, A.v.y + A.v.w * La.y, A.v.z + A.v.w * La.z, A.v.w);
            A.w = make_float4(A.w.x + A.w.w * Aa.x, A.w.y + A.w.w * Aa.y, A.w.z + A.w.w * Aa.z, A.w.w);
            Bv.v = make_float4(Bv.v.x + Bv.v.w * Lb.x, Bv.v.y + Bv.v.w * Lb.y, Bv.v.z + Bv.v.w * Lb.z, Bv.v.w);
            Bv.w = make_float4(Bv.w.x + Bv.w.w * Ab.x, Bv.w.y + Bv.w.w * Ab.y, Bv.w.z + Bv.w.w * Ab.z, Bv.w.w);
            B.vw[0][a] = A;
            B.vw[0][b] = Bv;
            B.lamA[0][c] = make_float4(u2.pn, u2.pt1, u2.pt2, u2.pr.x);
            B.lamB[0][c] = make_float2(u2.pr.y, u2.pr.z);
            if (last) write_world(B.lamW[p], c, n, u2);
        } else {
            const int k = u - nc, a = S.gbody[k];
            const float4* r = B.grec + 6 * (size_t)k;
            const float4 r0 = r[0], r1 = r[1], r2 = r[2], r3 = r[3], r4 = r[4];
            const float4 l0 = B.glamA[0][k];
            const float2 l1 = B.glamB[0][k];
            VW A = B.vw[0][a];
            const Upd u2 = contact_update(r0, r1, r2.x, 0.0f, r2.y, r2.z, l0, l1, f3(A.v) - f3(r3), f3(A.w), f3(r4),
                                          P.eps_reg);
            const float3 n = f3(r0);
            const float3 dpr = u2.pr - make_float3(l0.w, l1.x, l1.y);
            add_impulse(n, u2.t1, u2.t2, r2.x, u2.pn - l0.x, u2.pt1 - l0.y, u2.pt2 - l0.z, dpr, false, La, Aa);
            A.v = make_float4(A.v.x + A.v.w * La.x, A.v.y + A.v.w * La.y, A.v.z + A.v.w * La.z, A.v.w);
            A.w = make_float4(A.w.x + A.w.w * Aa.x, A.w.y + A.w.w * Aa.y, A.w.z + A.w.w * Aa.z, A.w.w);
            B.vw[0][a] = A;
            B.glamA[0][k] = make_float4(u2.pn, u2.pt1, u2.pt2, u2.pr.x);
            B.glamB[0][k] = make_float2(u2.pr.y, u2.pr.z);
            if (last) write_world(B.glamW[p], k, n, u2);
        }
    }
}

int launch_pgs_prepare(const SimParams& P, const DevBuf& B, const PgsBuf& S, int parity, int nc, int ngc,
                       cudaStream_t s) {
    k_pgs_prepare<<<nblk(std::max(P.n, PGS_MAX_COLOURS), SV_T), SV_T, 0, s>>>(P, B, S, parity, nc, ngc);
    k_pgs_keys<<<nblk(nc + ngc, SV_T), SV_T, 0, s>>>(P, B, S, parity, nc, ngc);
    return 2;
}

int launch_pgs_round(const SimParams& P, const DevBuf& B, const PgsBuf& S, int parity, int nc, int ngc,
                     cudaStream_t s) {
    k_pgs_round<<<std::max(1, std::min(nblk(nc + ngc, SV_T), 8 * sm_count())), SV_T, 0, s>>>(P, B, S, parity, nc,
                                                                                            ngc);
    return 1;
}

int launch_pgs_bucket(const PgsBuf& S, int total, bool fill, cudaStream_t s) {
    k_pgs_bucket<<<nblk(total, SV_T), SV_T, 0, s>>>(S, total, fill ? 1 : 0);
    return 1;
}

int launch_pgs_colour(const SimParams& P, const DevBuf& B, const PgsBuf& S, int parity, int nc, int first,
                      int count, bool last, cudaStream_t s) {
    k_pgs_colour<<<std::max(1, std::min(nblk(count, SV_T), 8 * sm_count())), SV_T, 0, s>>>(P, B, S, parity, nc,
                                                                                           first, count, last);
    return 1;
}

template <typename K>
static void launch_pdl(K kernel, int blocks, cudaStream_t s, const SimParams& P, const DevBuf& B, int p, int it,
                       int nact) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(SV_T);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, P, B, p, it, nact);
}

static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 152;
    }
    return n;
}

template <int T>
static void sweep_launch(const SimParams& P, const DevBuf& B, int parity, int it, int nact, bool update,
                         cudaStream_t s) {
    const int blocks = nblk(nact * T, SV_T);
    if (update) k_sweep<T, true><<<blocks, SV_T, 0, s>>>(P, B, parity, it);
    else k_sweep<T, false><<<blocks, SV_T, 0, s>>>(P, B, parity, -1);
}

static void sweep_dispatch(const SimParams& P, const DevBuf& B, int parity, int it, int nact, bool update,
                           cudaStream_t s) {
    switch (P.lanes > 0 && P.lanes <= 8 ? P.lanes : 2) {
        case 1: sweep_launch<1>(P, B, parity, it, nact, update, s); break;
        case 2: sweep_launch<2>(P, B, parity, it, nact, update, s); break;
        case 8: sweep_launch<8>(P, B, parity, it, nact, update, s); break;
        default: sweep_launch<4>(P, B, parity, it, nact, update, s); break;
    }
}

int launch_v0(const SimParams& P, const DevBuf& B, int parity, cudaStream_t s) {
    // v^0 from the warm-start impulses into velocities 0; a bed with no sweeps
    // keeps its warm start as the final impulse
    sweep_dispatch(P, B, parity, -1, P.n, false, s);
    return 1;
}

int launch_jacobi(const SimParams& P, const DevBuf& B, int parity, int it, int nact, cudaStream_t s) {
    if (P.lanes > 0 && P.lanes <= 8) {   // single-kernel sweep, T threads per body
        const int kg = launch_group_contacts(P, B, parity, it, s);
        sweep_dispatch(P, B, parity, it, nact, true, s);
        return 1 + kg;
    }
    // two-pass sweep: contacts (grid-stride) then bodies
    const int cblocks = std::max(1, std::min(nblk(nact * 8, SV_T), DEM_CP_BLOCKS_PER_SM * sm_count()));
    // bodies: one per thread, or grid-stride over a fixed number of blocks per SM
    const bool shares = DEM_GEO_IN_CP;
    const int bps = shares ? DEM_BP_BLOCKS_PER_SM_SHARES : DEM_BP_BLOCKS_PER_SM;
    const int bblocks = bps > 0 ? std::max(1, std::min(nblk(nact, SV_T), bps * sm_count())) : nblk(nact, SV_T);
    launch_pdl(k_contact_pass, cblocks, s, P, B, parity, it, nact);
    const int kg = launch_group_contacts(P, B, parity, it, s);
    if (shares) launch_pdl(k_body_pass<false>, bblocks, s, P, B, parity, it, nact);
    else launch_pdl(k_body_pass<true>, bblocks, s, P, B, parity, it, nact);
    return 2 + kg;
}

int launch_integrate(const SimParams& P, const DevBuf& B, int parity, cudaStream_t s) {
    k_integrate<<<nblk(P.n, SV_T), SV_T, 0, s>>>(P, B, parity);
    return 1;
}
