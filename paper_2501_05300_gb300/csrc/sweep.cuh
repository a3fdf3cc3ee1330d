// The canonical contact update of the projected Jacobi sweep and the impulse
// shares it gives the two bodies: shared by every sweep layout, so that all
// of them take the same arithmetic on the same inputs.
#pragma once
#include "dem_internal.cuh"

// ---------------------------------------------------------------------------
// the canonical contact update, identical at both ends of a contact
// ---------------------------------------------------------------------------
struct Upd {
    float pn, pt1, pt2;
    float3 pr, t1, t2;
};

// G2: the tangential block of D is a full 2x2 (i11 = r1.z, i12, i22), for the
// contacts of a load-driven group; otherwise it is r1.z times the identity
template <bool G2 = false>
static __device__ __forceinline__ Upd contact_update(float4 r0, float4 r1, float la, float lb, float mu_t,
                                                     float mur, float4 l0, float2 l1, float3 dv,
                                                     float3 wa, float3 wb, float eps_reg, float i12 = 0.f,
                                                     float i22 = 0.f) {
    Upd u;
    const float3 n = f3(r0);
    const float sig = r1.y, sig_t = eps_reg * r1.y;
    // normal: 0 <= p_n complementary to the SPOOK row (Eq. 5)
    const float wn = dot(n, dv) + sig * l0.x - r1.x;
    u.pn = fmaxf(0.0f, l0.x - r0.w * wn);
    // contact-point relative velocity: dv + w_a x (-l_a n) - w_b x (l_b n)
    const float3 uc = dv - cross(lin2(la, wa, lb, wb), n);
    tangent_basis(n, u.t1, u.t2);
    float pt1, pt2;
    if (G2) {
        const float w1 = dot(uc, u.t1) + sig_t * l0.y, w2 = dot(uc, u.t2) + sig_t * l0.z;
        pt1 = l0.y - fma2(r1.z, w1, i12, w2);
        pt2 = l0.z - fma2(i12, w1, i22, w2);
    } else {
        pt1 = l0.y - r1.z * (dot(uc, u.t1) + sig_t * l0.y);
        pt2 = l0.z - r1.z * (dot(uc, u.t2) + sig_t * l0.z);
    }
    const float bt = mu_t * u.pn;
    const float m2 = fma2(pt1, pt1, pt2, pt2);
    if (m2 > bt * bt) {   // Coulomb disc (Eq. 6)
        const float s = bt * rsqrtf(m2);
        pt1 *= s;
        pt2 *= s;
    }
    u.pt1 = pt1;
    u.pt2 = pt2;
    // rolling and twisting: ball |p_r| <= mu_r r_eff p_n (Eq. 7)
    const float3 pr0 = make_float3(l0.w, l1.x, l1.y);
    float3 pr = pr0 - r1.w * ((wa - wb) + sig_t * pr0);
    const float br = mur * u.pn;
    const float q2 = dot(pr, pr);
    if (q2 > br * br) pr = (br * rsqrtf(q2)) * pr;
    u.pr = pr;
    return u;
}

// A load-driven group's contact at sweep it: the group's iterate instead of
// the primitive's prescribed velocity, and the contact's impulse added to the
// group's sum for iterate it + 1 (k_group_contacts).
static __device__ __forceinline__ Upd geom_update_group(const SimParams& P, const DevBuf& B, const float4* r,
                                                        float4 l0, float2 l1, float3 vi, float3 wi, int q, int it) {
    const float4 r0 = r[0], r1 = r[1], r2 = r[2], r3 = r[3], r4 = r[4], r5 = r[5];
    const float3 vgp = group_velocity(P, B, q, it) + cross(f3(r4), f3(r5));
    const Upd u = contact_update<true>(r0, r1, r2.x, 0.0f, r2.y, r2.z, l0, l1, vi - vgp, wi, f3(r4), P.eps_reg,
                                       r3.w, r4.w);
    const float3 n = f3(r0);
    group_add(B, q, it + 1, (-1.0f) * (u.pn * n + lin2(u.pt1, u.t1, u.pt2, u.t2)));
    return u;
}

// Update of sphere-geometry contact k at sweep it from the body's iterate (vi, wi).
// A group's contact was updated by k_group_contacts: its new impulse is read.
static __device__ __forceinline__ Upd geom_update(const SimParams& P, const DevBuf& B, const float4* r, int k,
                                                  int src, int it, float3 vi, float3 wi, bool& done) {
    const float4 r0 = r[0];
    done = __float_as_int(r[5].w) >= 0;
    Upd u;
    if (done) {
        const int dst = src ^ 1;
        const float4 a = B.glamA[dst][k];
        const float2 b = B.glamB[dst][k];
        tangent_basis(f3(r0), u.t1, u.t2);
        u.pn = a.x; u.pt1 = a.y; u.pt2 = a.z; u.pr = make_float3(a.w, b.x, b.y);
        return u;
    }
    const float4 r1 = r[1], r2 = r[2], r3 = r[3], r4 = r[4];
    const float4 l0 = B.glamA[src][k];
    const float2 l1 = B.glamB[src][k];
    return contact_update(r0, r1, r2.x, 0.0f, r2.y, r2.z, l0, l1, vi - f3(r3), wi, f3(r4), P.eps_reg);
}

static __device__ __forceinline__ void write_world(float4* W, size_t c, float3 n, const Upd& u) {
    const float3 pt = lin2(u.pt1, u.t1, u.pt2, u.t2);
    W[2 * c] = make_float4(u.pn, pt.x, pt.y, pt.z);
    W[2 * c + 1] = make_float4(u.pr.x, u.pr.y, u.pr.z, 0.f);
}

// Impulse of a contact on body a with arm length l: linear P = p_n n + p_t,
// angular A = -l (n x p_t) + p_r.
static __device__ __forceinline__ void impulse_a(float3 n, float3 t1, float3 t2, float l, float pn, float pt1,
                                                 float pt2, float3 pr, float3& P, float3& A) {
    P = make_float3(__fmaf_rn(pt2, t2.x, fma2(pn, n.x, pt1, t1.x)), __fmaf_rn(pt2, t2.y, fma2(pn, n.y, pt1, t1.y)),
                    __fmaf_rn(pt2, t2.z, fma2(pn, n.z, pt1, t1.z)));
    // n x p_t = pt1 t2 - pt2 t1
    const float3 nxpt = lin2(pt1, t2, -pt2, t1);
    A = pr - l * nxpt;
}

// Impulse of a contact on the body at `side` (false = a, true = b) with arm
// length l, added to (accL, accA): linear  +-(p_n n + p_t),
// angular  -l (n x p_t) +- p_r.
static __device__ __forceinline__ void add_impulse(float3 n, float3 t1, float3 t2, float l, float pn,
                                                   float pt1, float pt2, float3 pr, bool sideb,
                                                   float3& accL, float3& accA) {
    const float3 P = make_float3(__fmaf_rn(pt2, t2.x, fma2(pn, n.x, pt1, t1.x)),
                                 __fmaf_rn(pt2, t2.y, fma2(pn, n.y, pt1, t1.y)),
                                 __fmaf_rn(pt2, t2.z, fma2(pn, n.z, pt1, t1.z)));
    // n x p_t = pt1 t2 - pt2 t1
    const float3 nxpt = lin2(pt1, t2, -pt2, t1);
    if (!sideb) {
        accL = accL + P;
        accA = accA + (pr - l * nxpt);
    } else {
        accL = accL - P;
        accA = accA - (pr + l * nxpt);
    }
}
