// Reverse-mode differentiation of the step: gradients of a linear functional
// of the per-step geometry forces with respect to the contact-stiffness scale,
// the particle friction coefficient mu_t and the rolling-resistance
// coefficient mu_r.
//
// Forward (dem_record): the ordinary step graphs, a checkpoint of the bed
// state every `every` steps and the geometry forces of every step.
// Reverse (dem_step_adjoint): segment by segment from the last, the segment's
// steps are recomputed from its checkpoint while a tape keeps what the
// reverse needs (the contact topology, the SPOOK rows of Sec. 2.2, the warm
// start and every Jacobi iterate lambda^k, v^k); then the steps are reversed
// in turn:
//   integration      x' = x + dt v^N                          (Sec. 2.2)
//   N_it sweeps       lambda^{k+1} = Pi(lambda^k - D^-1 (G v^k + Sigma lambda^k - b)),
//                     v^k = v* + M^-1 G^T lambda^k            (Eqs. 5-7)
//     each reversed with the projection Jacobians at the forward active set:
//     max(0, .) passes the normal adjoint where u_n > 0; an active Coulomb
//     disc |p_t| <= mu_t p_n (or rolling ball) scales the adjoint by
//     bound/|u| after removing its radial part, and sends the radial part to
//     the bound (p_n and mu)
//   warm start        lambda^0 = projection of the previous impulse on the
//                     new tangent plane
//   SPOOK rows        n, delta, arms, Sigma, b as functions of the positions,
//                     velocities and k_n = s_k E* sqrt(d*) / 3
// The contact set of every step is the forward's (fixed topology per step).
// Tangential impulses and their adjoints are world-frame 3-vectors, so the
// derivative of the tangent plane with the normal is exact.
//
// Geometry: planes that do not spin (their rows depend on the positions only
// through the overlap).  Determinism: every sum runs in a fixed order
// (incidence lists, fixed-grid block trees), so gradients repeat bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "bed.cuh"

#define AD_T 128
#define AD_RED_BLOCKS 296   // fixed grid of the reductions: deterministic partial sums

static inline int nblk(long long n, int t) { return n > 0 ? (int)((n + t - 1) / t) : 1; }

// Programmatic dependent launch: a kernel may start while the previous one
// drains; it waits (griddepcontrol.wait) before touching what that one wrote.
static __device__ __forceinline__ void adj_pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
static __device__ __forceinline__ void adj_pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl_adj(void (*kernel)(KArgs...), int blocks, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(AD_T);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ---------------------------------------------------------------------------
// host-side records
// ---------------------------------------------------------------------------
// What the reverse of one step reads.  Iterate arrays hold k = 0 .. n_it-1.
struct TapeStep {
    int nc = 0, ngc = 0;            // sphere-sphere / sphere-geometry contacts of the step
    int nc_prev = 0, ngc_prev = 0;  // contacts of the step before (warm-start sources)
    int resorted = 0;               // the step began with a re-sort
    int64_t step = 0;
    // bodies [n]
    VW* vw0 = nullptr;              // state at the step start (after a re-sort)
    float* rad = nullptr;
    int* cnt = nullptr;             // contacts per body (split masses)
    int* prev_of = nullptr;         // slot before the re-sort
    int* inc_start = nullptr;       // [n + 1]
    int* geo_start = nullptr;       // [n + 1]
    int2* inc = nullptr;            // [2 nc]
    // sphere-sphere contacts [nc]
    int* c_self = nullptr;
    int* c_other = nullptr;
    int2* c_pos = nullptr;
    float4* rec = nullptr;          // [3 nc]
    float* delta = nullptr;
    int* c_prev = nullptr;          // warm-start source in the previous step, or -1
    float4* c_warm = nullptr;       // [2 nc] world-frame warm-start impulse
    // sphere-geometry contacts [ngc]
    float4* grec = nullptr;         // [6 ngc]
    float* gdn = nullptr;           // [9 ngc] dn/dx of each contact's normal (world, row-major)
    float* gdelta = nullptr;
    int* g_prev = nullptr;
    float4* g_warm = nullptr;       // [2 ngc]
    // iterates
    float4* lamA = nullptr;         // [n_it * nc]
    float2* lamB = nullptr;
    float4* glamA = nullptr;        // [n_it * ngc]
    float2* glamB = nullptr;
    VW* v = nullptr;                // [n_it * n]
    void* mem = nullptr;
    size_t bytes = 0;
};

// Bed state between two steps: everything the next step reads.
struct Checkpoint {
    int64_t steps = 0;
    int nc_prev = 0, ngc_prev = 0;
    double4_32a* pos = nullptr;
    float4* posr = nullptr;
    VW* vw0 = nullptr;
    int* id = nullptr;
    int* lvl = nullptr;
    GeomDev* geom = nullptr;
    int* own_start = nullptr;   // previous step's contact lists (parity of that step)
    int* geo_start = nullptr;
    int* c_key = nullptr;
    float4* lamW = nullptr;
    int* g_key = nullptr;
    float4* glamW = nullptr;
    float* c_delta = nullptr;   // overlaps of that step (read-back)
    float* g_delta = nullptr;
    GroupDev* grp = nullptr;    // load-driven groups (velocities)
    void* mem = nullptr;
    size_t bytes = 0;
};

struct AdjointState {
    bool recorded = false;
    int64_t t0 = 0;
    int nsteps = 0, every = 0;
    SimParams P{};                  // settings the window was recorded with
    std::vector<Checkpoint> ck;     // segment starts
    Checkpoint end;                 // state after the window
    std::vector<TapeStep> tape;     // one per step of the segment being reversed
    long long* fhist = nullptr;     // [nsteps * 6 ng] fixed-point geometry impulses
    size_t fhist_n = 0;
    int* cnt_dev = nullptr;         // [2 nsteps] contacts of each recorded step (sphere, geometry)
    size_t cnt_n = 0;
    std::vector<int> counts;        // host copy of cnt_dev
    float* wts = nullptr;           // [nsteps * ng * 3] dJ/dF
    size_t wts_n = 0;
    // adjoint of the state between steps (current slot order), ping-pong
    float4* xbar[2] = {nullptr, nullptr};
    VW* sbar[2] = {nullptr, nullptr};
    // adjoints of the iterates v^k (ping-pong) and their sum over k
    VW* vb[2] = {nullptr, nullptr};
    VW* vacc = nullptr;
    // per contact: lambda-bar (2 float4) and row accumulators (2 float4)
    float4* L = nullptr;
    float4* A = nullptr;
    float4* gL = nullptr;
    float4* gA = nullptr;
    // adjoint of the final impulses of a step (its warm-start use), ping-pong
    float4* lw[2] = {nullptr, nullptr};
    float4* glw[2] = {nullptr, nullptr};
    double* part = nullptr;         // block partial sums [3 * (AD_RED_BLOCKS + body blocks)]
    double* grad = nullptr;         // [3]
};

// ---------------------------------------------------------------------------
// device: one contact's adjoint algebra
// ---------------------------------------------------------------------------
struct ARow {
    float3 n;
    float invDn, rhs, sig, invDt, invDr, la, lb, mt, mrc;
};

static __device__ __forceinline__ ARow pair_row(const float4* rec, int c) {
    const float4 r0 = rec[3 * (size_t)c], r1 = rec[3 * (size_t)c + 1], r2 = rec[3 * (size_t)c + 2];
    ARow R;
    R.n = f3(r0);
    R.invDn = r0.w; R.rhs = r1.x; R.sig = r1.y; R.invDt = r1.z; R.invDr = r1.w;
    R.la = r2.x; R.lb = r2.y; R.mt = r2.z; R.mrc = r2.w;
    return R;
}

static __device__ __forceinline__ ARow geom_row(const float4* grec, int k) {
    const float4* r = grec + 6 * (size_t)k;
    const float4 r0 = r[0], r1 = r[1], r2 = r[2];
    ARow R;
    R.n = f3(r0);
    R.invDn = r0.w; R.rhs = r1.x; R.sig = r1.y; R.invDt = r1.z; R.invDr = r1.w;
    R.la = r2.x; R.lb = 0.f; R.mt = r2.y; R.mrc = r2.z;
    return R;
}

static __device__ __forceinline__ float3 neg(float3 a) { return make_float3(-a.x, -a.y, -a.z); }

// Term of the body update v = v* + M^-1 G^T lambda in the adjoint of lambda:
// lambda-bar += G M^-1 vbar (tv, tw = M^-1 vbar at the two ends), and the
// derivative of G^T lambda with the normal and the arm lengths.
static __device__ __forceinline__ void body_term(const ARow& R, float pn, float3 pt, float3 tva, float3 twa,
                                                 float3 tvb, float3 twb, float4 L0, float4 L1, float& Ln,
                                                 float3& Lt, float3& Lr, float3& nb, float& lab, float& lbb) {
    const float3 n = R.n;
    const float3 dtv = tva - tvb;
    Ln = L0.x + dot(n, dtv);
    Lt = make_float3(L0.y, L0.z, L0.w) + dtv - R.la * cross(twa, n) - R.lb * cross(twb, n);
    Lr = make_float3(L1.x, L1.y, L1.z) + twa - twb;
    const float3 nxpt = cross(n, pt);
    nb = nb + pn * dtv - R.la * cross(pt, twa) - R.lb * cross(pt, twb);
    lab -= dot(nxpt, twa);
    lbb -= dot(nxpt, twb);
}

// Reverse of one projected Jacobi update of one contact.
//  l0, l1      lambda^k in the tangent basis of n (as the sweep stores it)
//  dv, wa, wb  v_a - v_b, w_a, w_b at iterate k
//  tv*, tw*    M^-1 vbar^{k+1} at the two ends (zero for a primitive)
//  L0, L1      in: lambda-bar^{k+1} without the body term; out: lambda-bar^k likewise
//              (L1.w carries the mu_r accumulator: sum p_n * d|p_r|-bound adjoint)
//  A0, A1      accumulators (n-bar, Sigma-bar | b-bar, l_a-bar, l_b-bar, mu_t-bar)
//  linA, angA  adjoint of (v_a, w_a) from this sweep; b takes (-linA, angB)
static __device__ __forceinline__ void adj_update(const ARow& R, float eps_reg, float4 l0, float2 l1, float3 dv,
                                                  float3 wa, float3 wb, float3 tva, float3 twa, float3 tvb,
                                                  float3 twb, float iIa, float iIb, bool pair, float4& L0,
                                                  float4& L1, float4& A0, float4& A1, float3& linA, float3& angA,
                                                  float3& angB) {
    const float3 n = R.n;
    float3 t1, t2;
    tangent_basis(n, t1, t2);
    const float sig = R.sig, sigt = eps_reg * R.sig;
    const float pn = l0.x;
    const float3 pt = l0.y * t1 + l0.z * t2;
    const float3 pr = make_float3(l0.w, l1.x, l1.y);
    // the forward update, recomputed in the sweep's operation order
    const float wn = dot(n, dv) + sig * pn - R.rhs;
    const float un = pn - R.invDn * wn;
    const float pn1 = fmaxf(0.0f, un);
    const float3 s = R.la * wa + R.lb * wb;
    const float3 uc = dv - cross(s, n);
    const float wt1 = dot(uc, t1) + sigt * l0.y, wt2 = dot(uc, t2) + sigt * l0.z;
    const float q1 = l0.y - R.invDt * wt1, q2 = l0.z - R.invDt * wt2;
    const float m2 = q1 * q1 + q2 * q2;
    const float bt = R.mt * pn1;
    const bool act_t = m2 > bt * bt;
    const float3 ut = q1 * t1 + q2 * t2;
    const float3 wt = wt1 * t1 + wt2 * t2;
    const float3 wr = (wa - wb) + sigt * pr;
    const float3 qr = pr - R.invDr * wr;
    const float q2r = dot(qr, qr);
    const float br = R.mrc * pn1;
    const bool act_r = q2r > br * br;
    const float it = act_t ? rsqrtf(m2) : 0.0f;
    const float3 pt1 = act_t ? (bt * it) * ut : ut;

    // full lambda-bar^{k+1}
    float3 nb = make_float3(A0.x, A0.y, A0.z);
    float sgb = A0.w, bb = A1.x, lab = A1.y, lbb = A1.z, mutb = A1.w, murb = L1.w;
    float Ln;
    float3 Lt, Lr;
    body_term(R, pn1, pt1, tva, twa, tvb, twb, L0, L1, Ln, Lt, Lr, nb, lab, lbb);

    // projections (Eqs. 5-7) at the forward active set
    float3 ubt = Lt;
    float btb = 0.0f;
    if (act_t) {
        const float3 qh = it * ut;
        btb = dot(qh, Lt);
        ubt = (bt * it) * (Lt - btb * qh);
    }
    float3 ubr = Lr;
    float brb = 0.0f;
    if (act_r) {
        const float ir = rsqrtf(q2r);
        const float3 rh = ir * qr;
        brb = dot(rh, Lr);
        ubr = (br * ir) * (Lr - brb * rh);
    }
    const float pnb = Ln + R.mt * btb + R.mrc * brb;
    if (pair) {
        mutb += pn1 * btb;
        murb += pn1 * brb;
    }
    const float ubn = un > 0.0f ? pnb : 0.0f;

    // lambda-bar^k through lambda^k itself
    const float fn = 1.0f - R.invDn * sig, ft = 1.0f - R.invDt * sigt, fr = 1.0f - R.invDr * sigt;
    L0 = make_float4(ubn * fn, ubt.x * ft, ubt.y * ft, ubt.z * ft);
    L1 = make_float4(ubr.x * fr, ubr.y * fr, ubr.z * fr, murb);
    // through the residual w = G v^k + Sigma lambda^k - b
    const float yn = -R.invDn * ubn;
    const float3 yt = -R.invDt * ubt, yr = -R.invDr * ubr;
    const float3 yp = yt - dot(yt, n) * n;
    const float dDn = R.invDn * R.invDn, dDr = R.invDr * R.invDr;
    const float mtan = R.invDt * R.invDt * dot(ubt, wt);   // adjoint of the angular part of D_t
    sgb += ubn * (dDn * wn - R.invDn * pn) +
           eps_reg * (mtan - R.invDt * dot(ubt, pt) + dot(ubr, dDr * wr - R.invDr * pr));
    lab += 2.0f * R.la * iIa * mtan - dot(yp, cross(wa, n));
    lbb += 2.0f * R.lb * iIb * mtan - dot(yp, cross(wb, n));
    bb += R.invDn * ubn;
    nb = nb + yn * dv - cross(yp, s) - dot(n, uc) * yt - dot(yt, n) * uc;
    A0 = make_float4(nb.x, nb.y, nb.z, sgb);
    A1 = make_float4(bb, lab, lbb, mutb);
    linA = yn * n + yp;
    const float3 nxy = cross(n, yp);
    angA = yr - R.la * nxy;
    angB = neg(yr) - R.lb * nxy;
}

// Reverse of the SPOOK row constants as functions of the overlap delta:
// J = e_H max(delta, floor)^{e_H - 1}, g = -delta^{e_H}, Sigma = 4 eps Y/(dt^2 J^2),
// b = -(4/dt) Y g / J + Y n.dv.  Returns delta-bar (arms included).
static __device__ __forceinline__ float rows_delta_bar(const SimParams& P, float delta, float sig, float sgb,
                                                       float bb, float lab, float lbb) {
    const float dfl = fmaxf(delta, P.delta_floor);
    const float J = P.e_H * powf(dfl, P.e_H - 1.0f);
    const float gap = -powf(delta, P.e_H);
    const float b1 = (-4.0f * P.inv_dt * P.ups * gap) / J;
    const float Jb = -2.0f * sig * sgb / J - bb * b1 / J;
    const float gapb = bb * (-4.0f * P.inv_dt * P.ups) / J;
    float db = gapb * (-P.e_H * powf(delta, P.e_H - 1.0f)) - 0.5f * (lab + lbb);
    if (delta > P.delta_floor) db += Jb * P.e_H * (P.e_H - 1.0f) * powf(delta, P.e_H - 2.0f);
    return db;
}

// Derivative of a sphere-primitive contact's unit normal with respect to the
// sphere centre, dn/dx (world frame, row-major), for the closest-point cases
// of geom_hit.  With e = q - cl(q) the offset of the local centre q from its
// clamped point cl and d = |e|, n_l = e / d, so dn_l/dq = (I - n_l n_l^T)
// (I - dcl/dq) / d: zero on a face or cap (the clamped axis is n_l's),
// (I - n n^T - t t^T) / d along a box edge of direction t, (I - n n^T) / d at a
// corner, (I - u u^T) / rho in the plane normal to the axis on a cylinder's
// side (u radial, rho the distance to the axis), and the general product at a
// rim.  A centre inside the primitive takes the nearest face (zero) or, in a
// cylinder's radial case, the radial direction (I - u u^T) / rho.  A plane's
// normal is fixed.  dn/dx = R (dn_l/dq) R^T.
static __device__ void geom_dn_dx(const GeomDev& g, double x0, double x1, double x2, float* out) {
    double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    if (g.type != DEM_GEOM_PLANE) {
        const double d0 = x0 - g.c[0], d1 = x1 - g.c[1], d2 = x2 - g.c[2];
        double q[3], cl[3], C[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int j = 0; j < 3; ++j) q[j] = g.R[j] * d0 + g.R[3 + j] * d1 + g.R[6 + j] * d2;
        bool inside_radial = false;
        double rho = 0.0;
        if (g.type == DEM_GEOM_BOX) {
            for (int k = 0; k < 3; ++k) {
                cl[k] = q[k] < -g.he[k] ? -g.he[k] : (q[k] > g.he[k] ? g.he[k] : q[k]);
                C[k][k] = (q[k] < -g.he[k] || q[k] > g.he[k]) ? 0.0 : 1.0;
            }
        } else {
            const double Rc = g.he[0], H = g.he[2];
            const double rho2 = q[0] * q[0] + q[1] * q[1];
            rho = sqrt(rho2);
            if (rho2 > Rc * Rc) {
                const double s = Rc / rho, ux = q[0] / rho, uy = q[1] / rho;
                cl[0] = q[0] * s; cl[1] = q[1] * s;
                C[0][0] = s * (1.0 - ux * ux); C[0][1] = -s * ux * uy;
                C[1][0] = -s * ux * uy; C[1][1] = s * (1.0 - uy * uy);
            } else {
                cl[0] = q[0]; cl[1] = q[1];
                C[0][0] = 1.0; C[1][1] = 1.0;
            }
            cl[2] = q[2] < -H ? -H : (q[2] > H ? H : q[2]);
            C[2][2] = (q[2] < -H || q[2] > H) ? 0.0 : 1.0;
            inside_radial = (H - fabs(q[2])) > (Rc - rho) && rho > 0.0;
        }
        const double e[3] = {q[0] - cl[0], q[1] - cl[1], q[2] - cl[2]};
        const double ee = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
        double Ml[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        if (ee > 0.0) {
            const double d = sqrt(ee);
            const double nl[3] = {e[0] / d, e[1] / d, e[2] / d};
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; ++k) {
                        const double P = (i == k ? 1.0 : 0.0) - nl[i] * nl[k];
                        const double Q = (k == j ? 1.0 : 0.0) - C[k][j];
                        acc += P * Q;
                    }
                    Ml[i][j] = acc / d;
                }
        } else if (g.type == DEM_GEOM_CYLINDER && inside_radial) {
            const double ux = q[0] / rho, uy = q[1] / rho;
            Ml[0][0] = (1.0 - ux * ux) / rho; Ml[0][1] = -ux * uy / rho;
            Ml[1][0] = -ux * uy / rho; Ml[1][1] = (1.0 - uy * uy) / rho;
        }
        // world: R Ml R^T (R row-major, column k = local axis k)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) acc += g.R[3 * i + a] * Ml[a][b] * g.R[3 * j + b];
                M[i][j] = acc;
            }
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) out[3 * i + j] = (float)M[i][j];
}

// ---------------------------------------------------------------------------
// tape kernels (forward recompute)
// ---------------------------------------------------------------------------
// per body: state, counts, and the warm-start source of each contact it owns
// (the same merge by key as the row set-up)
__global__ void __launch_bounds__(AD_T) k_tape_bodies(SimParams P, DevBuf B, int p, TapeStep T) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const int q = p ^ 1;
    T.vw0[i] = B.vw0[i];
    T.rad[i] = (float)B.pos[i].w;
    T.cnt[i] = (B.inc_start[i + 1] - B.inc_start[i]) + (B.geo_start[p][i + 1] - B.geo_start[p][i]);
    if (T.resorted) T.prev_of[i] = B.prev_of[i];
    const int prev = T.resorted ? B.prev_of[i] : i;
    const int os = B.own_start[p][i], oe = B.own_start[p][i + 1];
    const int ps = B.own_start[q][prev], pe = B.own_start[q][prev + 1];
    int kp = ps;
    for (int c = os; c < oe; ++c) {
        const int key = B.c_key[p][c];
        while (kp < pe && B.c_key[q][kp] < key) ++kp;
        if (kp < pe && B.c_key[q][kp] == key) {
            T.c_prev[c] = kp;
            T.c_warm[2 * (size_t)c] = B.lamW[q][2 * (size_t)kp];
            T.c_warm[2 * (size_t)c + 1] = B.lamW[q][2 * (size_t)kp + 1];
        } else {
            T.c_prev[c] = -1;
            T.c_warm[2 * (size_t)c] = make_float4(0.f, 0.f, 0.f, 0.f);
            T.c_warm[2 * (size_t)c + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    const int gs = B.geo_start[p][i], ge = B.geo_start[p][i + 1];
    const int gps = B.geo_start[q][prev], gpe = B.geo_start[q][prev + 1];
    for (int k = gs; k < ge; ++k) {
        const int g = B.g_key[p][k];
        int src = -1;
        for (int kk = gps; kk < gpe; ++kk)
            if (B.g_key[q][kk] == g) { src = kk; break; }
        T.g_prev[k] = src;
        T.g_warm[2 * (size_t)k] = src >= 0 ? B.glamW[q][2 * (size_t)src] : make_float4(0.f, 0.f, 0.f, 0.f);
        T.g_warm[2 * (size_t)k + 1] = src >= 0 ? B.glamW[q][2 * (size_t)src + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
        const double4_32a xi = B.pos[i];
        geom_dn_dx(B.geom[g], xi.x, xi.y, xi.z, T.gdn + 9 * (size_t)k);
    }
}

// iterate k of the impulses and velocities
__global__ void __launch_bounds__(AD_T) k_tape_iter(int n, int nc, int ngc, const float4* __restrict__ lA,
                                                    const float2* __restrict__ lB, const float4* __restrict__ gA,
                                                    const float2* __restrict__ gB, const VW* __restrict__ v,
                                                    float4* oA, float2* oB, float4* ogA, float2* ogB, VW* ov) {
    adj_pdl_wait();
    adj_pdl_trigger();
    const long long total = (long long)nc + ngc + n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        if (t < nc) {
            oA[t] = lA[t];
            oB[t] = lB[t];
        } else if (t < (long long)nc + ngc) {
            const long long k = t - nc;
            ogA[k] = gA[k];
            ogB[k] = gB[k];
        } else {
            const long long i = t - nc - ngc;
            ov[i] = v[i];
        }
    }
}

// ---------------------------------------------------------------------------
// reverse kernels
// ---------------------------------------------------------------------------
struct AdjBufs {
    float4* xbar_in; VW* sbar_in;     // adjoint of the state after the step
    float4* xbar_out; VW* sbar_out;   // adjoint of the state before the step (previous slot order)
    VW* vb[2];
    VW* vacc;
    float4* L; float4* A; float4* gL; float4* gA;
    float4* lw_in; float4* glw_in;    // adjoint of this step's final impulses
    float4* lw_out; float4* glw_out;  // adjoint of the previous step's final impulses
    Imp* sh;                          // per incidence entry shares
    const float* wts;                 // dJ/dF of this step [ng * 3]
    double* part;
};

// v-bar^N = vbar' + dt xbar', w-bar^N = wbar'; lambda-bar^N = warm-start adjoint
// (+ force objective for primitive contacts); accumulators zero
__global__ void __launch_bounds__(AD_T) k_adj_init(SimParams P, TapeStep T, AdjBufs Q, int slotN) {
    const long long total = (long long)P.n + T.nc + T.ngc;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        if (t < P.n) {
            const int i = (int)t;
            const VW s = Q.sbar_in[i];
            const float4 x = Q.xbar_in[i];
            VW o;
            o.v = make_float4(s.v.x + P.dt * x.x, s.v.y + P.dt * x.y, s.v.z + P.dt * x.z, 0.f);
            o.w = make_float4(s.w.x, s.w.y, s.w.z, 0.f);
            Q.vb[slotN][i] = o;
            Q.vacc[i] = o;
        } else if (t < (long long)P.n + T.nc) {
            const size_t c = (size_t)(t - P.n);
            Q.L[2 * c] = Q.lw_in[2 * c];
            Q.L[2 * c + 1] = Q.lw_in[2 * c + 1];
            Q.A[2 * c] = z;
            Q.A[2 * c + 1] = z;
        } else {
            const size_t k = (size_t)(t - P.n - T.nc);
            const float4* r = T.grec + 6 * k;
            const int g = __float_as_int(r[2].w);
            const float3 n = f3(r[0]);
            // force on primitive g: -(p_n n + p_t) / dt
            const float3 W = make_float3(Q.wts[3 * g], Q.wts[3 * g + 1], Q.wts[3 * g + 2]);
            const float4 a = Q.glw_in[2 * k];
            Q.gL[2 * k] = make_float4(a.x - dot(W, n) * P.inv_dt, a.y - W.x * P.inv_dt, a.z - W.y * P.inv_dt,
                                      a.w - W.z * P.inv_dt);
            Q.gL[2 * k + 1] = Q.glw_in[2 * k + 1];
            Q.gA[2 * k] = z;
            Q.gA[2 * k + 1] = z;
        }
    }
}

// reverse of sweep k, sphere-sphere contacts: one thread per contact
__global__ void __launch_bounds__(AD_T) k_adj_contacts(SimParams P, TapeStep T, AdjBufs Q, int k) {
    adj_pdl_wait();
    adj_pdl_trigger();
    const int src = (k + 1) & 1;
    const VW* __restrict__ vk = T.v + (size_t)k * P.n;
    const VW* __restrict__ gb = Q.vb[src];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < T.nc; c += gridDim.x * blockDim.x) {
        const int a = T.c_self[c], b = T.c_other[c];
        const ARow R = pair_row(T.rec, c);
        const float4 l0 = T.lamA[(size_t)k * T.nc + c];
        const float2 l1 = T.lamB[(size_t)k * T.nc + c];
        const VW va = vk[a], vb = vk[b];
        const VW ga = gb[a], gbb = gb[b];
        const float3 tva = va.v.w * f3(ga.v), twa = va.w.w * f3(ga.w);
        const float3 tvb = vb.v.w * f3(gbb.v), twb = vb.w.w * f3(gbb.w);
        const float iIa = T.cnt[a] * va.w.w, iIb = T.cnt[b] * vb.w.w;
        float4 L0 = Q.L[2 * (size_t)c], L1 = Q.L[2 * (size_t)c + 1];
        float4 A0 = Q.A[2 * (size_t)c], A1 = Q.A[2 * (size_t)c + 1];
        float3 linA, angA, angB;
        adj_update(R, P.eps_reg, l0, l1, f3(va.v) - f3(vb.v), f3(va.w), f3(vb.w), tva, twa, tvb, twb, iIa, iIb,
                   true, L0, L1, A0, A1, linA, angA, angB);
        Q.L[2 * (size_t)c] = L0;
        Q.L[2 * (size_t)c + 1] = L1;
        Q.A[2 * (size_t)c] = A0;
        Q.A[2 * (size_t)c + 1] = A1;
        const int2 pos = T.c_pos[c];
        Imp ia, ib;
        ia.a = make_float4(linA.x, linA.y, linA.z, angA.x);
        ia.b = make_float4(angA.y, angA.z, 0.f, 0.f);
        ib.a = make_float4(-linA.x, -linA.y, -linA.z, angB.x);
        ib.b = make_float4(angB.y, angB.z, 0.f, 0.f);
        Q.sh[pos.x] = ia;
        Q.sh[pos.y] = ib;
    }
}

// reverse of sweep k, bodies: v-bar^k = sum of the shares (incidence order)
// plus the body's primitive contacts, reversed here
__global__ void __launch_bounds__(AD_T) k_adj_bodies(SimParams P, TapeStep T, AdjBufs Q, int k) {
    adj_pdl_wait();
    adj_pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const int src = (k + 1) & 1, dst = k & 1;
    float3 lin = make_float3(0.f, 0.f, 0.f), ang = lin;
    for (int e = T.inc_start[i]; e < T.inc_start[i + 1]; ++e) {
        const Imp q = Q.sh[e];
        lin = lin + f3(q.a);
        ang = ang + make_float3(q.a.w, q.b.x, q.b.y);
    }
    const int g0 = T.geo_start[i], g1 = T.geo_start[i + 1];
    if (g0 < g1) {
        const VW vi = T.v[(size_t)k * P.n + i];
        const VW gi = Q.vb[src][i];
        const float3 tva = vi.v.w * f3(gi.v), twa = vi.w.w * f3(gi.w);
        const float3 z = make_float3(0.f, 0.f, 0.f);
        const float iIa = T.cnt[i] * vi.w.w;
        for (int kk = g0; kk < g1; ++kk) {
            const ARow R = geom_row(T.grec, kk);
            const float4* r = T.grec + 6 * (size_t)kk;
            const float4 l0 = T.glamA[(size_t)k * T.ngc + kk];
            const float2 l1 = T.glamB[(size_t)k * T.ngc + kk];
            float4 L0 = Q.gL[2 * (size_t)kk], L1 = Q.gL[2 * (size_t)kk + 1];
            float4 A0 = Q.gA[2 * (size_t)kk], A1 = Q.gA[2 * (size_t)kk + 1];
            float3 linA, angA, angB;
            adj_update(R, P.eps_reg, l0, l1, f3(vi.v) - f3(r[3]), f3(vi.w), f3(r[4]), tva, twa, z, z, iIa, 0.f,
                       false, L0, L1, A0, A1, linA, angA, angB);
            if (k == P.n_it - 1) {
                // the step's force on the primitive, -(p_n n + p_t) / dt, depends on n
                // through its normal part: n-bar += -p_n W / dt with the final p_n
                const float wn = dot(R.n, f3(vi.v) - f3(r[3])) + R.sig * l0.x - R.rhs;
                const float pn1 = fmaxf(0.0f, l0.x - R.invDn * wn);
                const int g = __float_as_int(r[2].w);
                const float s = -pn1 * P.inv_dt;
                A0 = make_float4(A0.x + s * Q.wts[3 * g], A0.y + s * Q.wts[3 * g + 1], A0.z + s * Q.wts[3 * g + 2],
                                 A0.w);
            }
            Q.gL[2 * (size_t)kk] = L0;
            Q.gL[2 * (size_t)kk + 1] = L1;
            Q.gA[2 * (size_t)kk] = A0;
            Q.gA[2 * (size_t)kk + 1] = A1;
            lin = lin + linA;
            ang = ang + angA;
        }
    }
    VW o;
    o.v = make_float4(lin.x, lin.y, lin.z, 0.f);
    o.w = make_float4(ang.x, ang.y, ang.z, 0.f);
    Q.vb[dst][i] = o;
    VW s = Q.vacc[i];
    s.v = make_float4(s.v.x + lin.x, s.v.y + lin.y, s.v.z + lin.z, 0.f);
    s.w = make_float4(s.w.x + ang.x, s.w.y + ang.y, s.w.z + ang.z, 0.f);
    Q.vacc[i] = s;
}

// fixed-order block sum of three doubles into part[3 * blockIdx.x]
static __device__ __forceinline__ void block_sum3(double a, double b, double c, double* part) {
    __shared__ double sm[3][AD_T];
    sm[0][threadIdx.x] = a;
    sm[1][threadIdx.x] = b;
    sm[2][threadIdx.x] = c;
    __syncthreads();
    for (int o = AD_T / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int q = 0; q < 3; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; ++q) part[3 * blockIdx.x + q] = sm[q][0];
}

// reverse of the warm start and of the SPOOK rows, sphere-sphere contacts
__global__ void __launch_bounds__(AD_T) k_adj_rows(SimParams P, TapeStep T, AdjBufs Q) {
    double gk = 0.0, gt = 0.0, gr = 0.0;
    const VW* __restrict__ gb = Q.vb[0];   // v-bar^0
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < T.nc; c += gridDim.x * blockDim.x) {
        const int a = T.c_self[c], b = T.c_other[c];
        const ARow R = pair_row(T.rec, c);
        const float4 l0 = T.lamA[c];   // (the rolling part of lambda^0 does not depend on the rows)
        const VW sa = T.vw0[a], sb = T.vw0[b];
        const VW ga = gb[a], gbb = gb[b];
        const float3 tva = sa.v.w * f3(ga.v), twa = sa.w.w * f3(ga.w);
        const float3 tvb = sb.v.w * f3(gbb.v), twb = sb.w.w * f3(gbb.w);
        const float4 L0 = Q.L[2 * (size_t)c], L1 = Q.L[2 * (size_t)c + 1];
        const float4 A0 = Q.A[2 * (size_t)c], A1 = Q.A[2 * (size_t)c + 1];
        float3 t1, t2;
        tangent_basis(R.n, t1, t2);
        const float3 n = R.n;
        const float3 pt = l0.y * t1 + l0.z * t2;
        float3 nb = f3(A0);
        float lab = A1.y, lbb = A1.z;
        float Ln;
        float3 Lt, Lr;
        body_term(R, l0.x, pt, tva, twa, tvb, twb, L0, L1, Ln, Lt, Lr, nb, lab, lbb);
        // warm start: lambda^0 = (p_n, P_t p_t^w, p_r^w)
        const float4 w0 = T.c_warm[2 * (size_t)c];
        const float3 ptw = make_float3(w0.y, w0.z, w0.w);
        nb = nb - dot(Lt, n) * ptw - dot(ptw, n) * Lt;
        const int pv = T.c_prev[c];
        if (pv >= 0) {
            const float3 Lp = Lt - dot(Lt, n) * n;
            Q.lw_out[2 * (size_t)pv] = make_float4(Ln, Lp.x, Lp.y, Lp.z);
            Q.lw_out[2 * (size_t)pv + 1] = make_float4(Lr.x, Lr.y, Lr.z, 0.f);
        }
        // rows
        const float sgb = A0.w, bb = A1.x;
        const float delta = T.delta[c];
        const float db = rows_delta_bar(P, delta, R.sig, sgb, bb, lab, lbb);
        nb = nb + (bb * P.ups) * (f3(sa.v) - f3(sb.v));
        const float3 vrow = (bb * P.ups) * n;
        const float ra = T.rad[a], rb = T.rad[b];
        const float dist = (ra + rb) - delta;
        const float3 dbar = (1.0f / dist) * (nb - dot(nb, n) * n) - db * n;
        const int2 pos = T.c_pos[c];
        Imp ia, ib;
        ia.a = make_float4(dbar.x, dbar.y, dbar.z, vrow.x);
        ia.b = make_float4(vrow.y, vrow.z, 0.f, 0.f);
        ib.a = make_float4(-dbar.x, -dbar.y, -dbar.z, -vrow.x);
        ib.b = make_float4(-vrow.y, -vrow.z, 0.f, 0.f);
        Q.sh[pos.x] = ia;
        Q.sh[pos.y] = ib;
        // parameters: Sigma ~ 1 / s_k, bounds mu_t p_n and mu_r d* p_n
        gk += (double)sgb * (double)(-R.sig / P.kn_scale);
        gt += (double)A1.w;
        gr += (double)L1.w * (double)(2.0f * ra * rb / (ra + rb));
    }
    block_sum3(gk, gt, gr, Q.part);
}

// per body: x-bar, v-bar, w-bar of the state before the step, with the rows
// of its primitive contacts; written in the slot order of the previous step
__global__ void __launch_bounds__(AD_T) k_adj_state(SimParams P, TapeStep T, AdjBufs Q) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double gk = 0.0;
    if (i < P.n) {
        float3 xb = f3(Q.xbar_in[i]);
        const VW acc = Q.vacc[i];
        float3 vbar = f3(acc.v);
        for (int e = T.inc_start[i]; e < T.inc_start[i + 1]; ++e) {
            const Imp q = Q.sh[e];
            xb = xb + f3(q.a);
            vbar = vbar + make_float3(q.a.w, q.b.x, q.b.y);
        }
        const int g0 = T.geo_start[i], g1 = T.geo_start[i + 1];
        if (g0 < g1) {
            const VW s = T.vw0[i];
            const VW gi = Q.vb[0][i];
            const float3 tva = s.v.w * f3(gi.v), twa = s.w.w * f3(gi.w);
            const float3 z = make_float3(0.f, 0.f, 0.f);
            for (int kk = g0; kk < g1; ++kk) {
                const ARow R = geom_row(T.grec, kk);
                const float4 l0 = T.glamA[kk];
                const float4 L0 = Q.gL[2 * (size_t)kk], L1 = Q.gL[2 * (size_t)kk + 1];
                const float4 A0 = Q.gA[2 * (size_t)kk], A1 = Q.gA[2 * (size_t)kk + 1];
                float3 t1, t2;
                tangent_basis(R.n, t1, t2);
                const float3 pt = l0.y * t1 + l0.z * t2;
                // n-bar: the sweeps' accumulations, then the body term, the warm
                // start's projection and the velocity part of the right side
                float3 nb = f3(A0);
                float lab = A1.y, lbb = 0.f;
                float Ln;
                float3 Lt, Lr;
                body_term(R, l0.x, pt, tva, twa, z, z, L0, L1, Ln, Lt, Lr, nb, lab, lbb);
                if (P.n_it == 0) {   // the step's force is the warm start's: its normal part
                    const int g = __float_as_int(T.grec[6 * (size_t)kk + 2].w);
                    const float s = -l0.x * P.inv_dt;
                    nb = nb + s * make_float3(Q.wts[3 * g], Q.wts[3 * g + 1], Q.wts[3 * g + 2]);
                }
                const float4 w0 = T.g_warm[2 * (size_t)kk];
                const float3 ptw = make_float3(w0.y, w0.z, w0.w);
                nb = nb - dot(Lt, R.n) * ptw - dot(ptw, R.n) * Lt;
                const int pv = T.g_prev[kk];
                if (pv >= 0) {
                    const float3 Lp = Lt - dot(Lt, R.n) * R.n;
                    Q.glw_out[2 * (size_t)pv] = make_float4(Ln, Lp.x, Lp.y, Lp.z);
                    Q.glw_out[2 * (size_t)pv + 1] = make_float4(Lr.x, Lr.y, Lr.z, 0.f);
                }
                const float db = rows_delta_bar(P, T.gdelta[kk], R.sig, A0.w, A1.x, lab, 0.f);
                const float3 vg = f3(T.grec[6 * (size_t)kk + 3]);   // the primitive's point velocity
                nb = nb + (A1.x * P.ups) * (f3(s.v) - vg);
                // delta = r - |x - q(x)|: d delta / dx = -n (the closest point is a
                // minimiser); n(x) through dn/dx of the contact's case (zero for
                // planes and faces)
                const float* M = T.gdn + 9 * (size_t)kk;
                xb = xb - db * R.n +
                     make_float3(M[0] * nb.x + M[3] * nb.y + M[6] * nb.z, M[1] * nb.x + M[4] * nb.y + M[7] * nb.z,
                                 M[2] * nb.x + M[5] * nb.y + M[8] * nb.z);
                vbar = vbar + (A1.x * P.ups) * R.n;
                gk += (double)A0.w * (double)(-R.sig / P.kn_scale);
            }
        }
        const int o = T.resorted ? T.prev_of[i] : i;
        Q.xbar_out[o] = make_float4(xb.x, xb.y, xb.z, 0.f);
        VW out;
        out.v = make_float4(vbar.x, vbar.y, vbar.z, 0.f);
        out.w = make_float4(acc.w.x, acc.w.y, acc.w.z, 0.f);
        Q.sbar_out[o] = out;
    }
    block_sum3(gk, 0.0, 0.0, Q.part + 3 * AD_RED_BLOCKS);
}

// grad += partial sums: thread t adds partials t, t + 256, ... in order, then a
// fixed tree; the result does not depend on timing
#define AD_RED_T 256
__global__ void __launch_bounds__(AD_RED_T) k_adj_reduce(const double* part, int nb1, int nb2, double* grad) {
    __shared__ double sm[3][AD_RED_T];
    double g[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nb1 + nb2; b += AD_RED_T) {
        const double* p = b < nb1 ? part + 3 * b : part + 3 * AD_RED_BLOCKS + 3 * (b - nb1);
        for (int q = 0; q < 3; ++q) g[q] += p[q];
    }
    for (int q = 0; q < 3; ++q) sm[q][threadIdx.x] = g[q];
    __syncthreads();
    for (int o = AD_RED_T / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int q = 0; q < 3; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; ++q) grad[q] += sm[q][0];
}

// ---------------------------------------------------------------------------
// host: memory
// ---------------------------------------------------------------------------
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// carve typed arrays out of one allocation: first pass sizes, second pass assigns
struct Carver {
    char* base;
    size_t off = 0;
    template <typename T>
    void take(T*& p, size_t count) {
        p = base ? (T*)(base + off) : nullptr;
        off += align256(std::max<size_t>(count, 1) * sizeof(T));
    }
};

template <typename F>
static dem_status carve_alloc(dem_bed* b, void*& mem, size_t& bytes, F layout) {
    Carver c0{nullptr};
    layout(c0);
    if (c0.off > bytes) {
        if (mem) dem_dfree(b, mem);
        mem = nullptr;
        bytes = 0;
        dem_status st = dem_dalloc(b, &mem, c0.off);
        if (st != DEM_OK) return st;
        bytes = c0.off;
    }
    Carver c1{(char*)mem};
    layout(c1);
    return DEM_OK;
}

static dem_status ensure_state(dem_bed* b) {
    if (b->adj) return DEM_OK;
    AdjointState* S = new AdjointState();
    b->adj = S;
    const size_t N = std::max(b->P.n, 1), C = (size_t)b->P.max_contacts, GC = (size_t)b->P.max_geo;
    dem_status st = DEM_OK;
    auto al = [&](void** p, size_t bytes) {
        if (st == DEM_OK) st = dem_dalloc(b, p, bytes);
    };
    for (int q = 0; q < 2; ++q) {
        al((void**)&S->xbar[q], N * sizeof(float4));
        al((void**)&S->sbar[q], N * sizeof(VW));
        al((void**)&S->vb[q], N * sizeof(VW));
        al((void**)&S->lw[q], 2 * C * sizeof(float4));
        al((void**)&S->glw[q], 2 * GC * sizeof(float4));
    }
    al((void**)&S->vacc, N * sizeof(VW));
    al((void**)&S->L, 2 * C * sizeof(float4));
    al((void**)&S->A, 2 * C * sizeof(float4));
    al((void**)&S->gL, 2 * GC * sizeof(float4));
    al((void**)&S->gA, 2 * GC * sizeof(float4));
    al((void**)&S->part, 3 * ((size_t)AD_RED_BLOCKS + nblk((long long)N, AD_T)) * sizeof(double));
    al((void**)&S->grad, 4 * sizeof(double));
    return st;
}

void dem_adjoint_release(dem_bed* b) {
    // the memory itself belongs to the bed's allocation list and is freed with it
    delete b->adj;
    b->adj = nullptr;
}

void dem_adjoint_drop(dem_bed* b) {
    AdjointState* S = b->adj;
    if (!S) return;
    auto fr = [&](void* p) { if (p) dem_dfree(b, p); };
    for (Checkpoint& K : S->ck) fr(K.mem);
    fr(S->end.mem);
    for (TapeStep& T : S->tape) fr(T.mem);
    fr(S->fhist); fr(S->cnt_dev); fr(S->wts);
    for (int q = 0; q < 2; ++q) {
        fr(S->xbar[q]); fr(S->sbar[q]); fr(S->vb[q]); fr(S->lw[q]); fr(S->glw[q]);
    }
    fr(S->vacc); fr(S->L); fr(S->A); fr(S->gL); fr(S->gA); fr(S->part); fr(S->grad);
    dem_adjoint_release(b);
}

// ---------------------------------------------------------------------------
// host: checkpoints
// ---------------------------------------------------------------------------
static dem_status read_counts(dem_bed* b, int parity, int* nc, int* ngc) {
    const int n = b->P.n;
    DEM_CK(cudaMemcpyAsync(nc, b->B.own_start[parity] + n, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    DEM_CK(cudaMemcpyAsync(ngc, b->B.geo_start[parity] + n, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    DEM_CK(cudaStreamSynchronize(b->stream));
    return DEM_OK;
}

static dem_status save_checkpoint(dem_bed* b, Checkpoint& K) {
    const SimParams& P = b->P;
    const DevBuf& B = b->B;
    const int n = P.n, ng = std::max(P.ng, 1);
    const int q = (int)((b->steps & 1) ^ 1);   // parity of the step before
    int nc = 0, ngc = 0;
    dem_status st = read_counts(b, q, &nc, &ngc);
    if (st != DEM_OK) return st;
    K.steps = b->steps;
    K.nc_prev = nc;
    K.ngc_prev = ngc;
    st = carve_alloc(b, K.mem, K.bytes, [&](Carver& c) {
        c.take(K.pos, n); c.take(K.posr, n); c.take(K.vw0, n); c.take(K.id, n); c.take(K.lvl, n);
        c.take(K.geom, ng); c.take(K.own_start, n + 1); c.take(K.geo_start, n + 1);
        c.take(K.c_key, nc); c.take(K.lamW, 2 * (size_t)nc); c.take(K.g_key, ngc); c.take(K.glamW, 2 * (size_t)ngc);
        c.take(K.c_delta, nc); c.take(K.g_delta, ngc); c.take(K.grp, DEM_MAX_GROUPS);
    });
    if (st != DEM_OK) return st;
    cudaStream_t s = b->stream;
    auto cp = [&](void* dst, const void* src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s) : cudaSuccess;
    };
    DEM_CK(cp(K.pos, B.pos, n * sizeof(double4_32a)));
    DEM_CK(cp(K.posr, B.posr, n * sizeof(float4)));
    DEM_CK(cp(K.vw0, B.vw0, n * sizeof(VW)));
    DEM_CK(cp(K.id, B.id, n * sizeof(int)));
    DEM_CK(cp(K.lvl, B.lvl, n * sizeof(int)));
    DEM_CK(cp(K.geom, B.geom, P.ng * sizeof(GeomDev)));
    DEM_CK(cp(K.own_start, B.own_start[q], (n + 1) * sizeof(int)));
    DEM_CK(cp(K.geo_start, B.geo_start[q], (n + 1) * sizeof(int)));
    DEM_CK(cp(K.c_key, B.c_key[q], nc * sizeof(int)));
    DEM_CK(cp(K.lamW, B.lamW[q], 2 * (size_t)nc * sizeof(float4)));
    DEM_CK(cp(K.g_key, B.g_key[q], ngc * sizeof(int)));
    DEM_CK(cp(K.glamW, B.glamW[q], 2 * (size_t)ngc * sizeof(float4)));
    DEM_CK(cp(K.c_delta, B.c_delta, nc * sizeof(float)));
    DEM_CK(cp(K.g_delta, B.g_delta, ngc * sizeof(float)));
    DEM_CK(cp(K.grp, B.grp, DEM_MAX_GROUPS * sizeof(GroupDev)));
    return DEM_OK;
}

static dem_status restore_checkpoint(dem_bed* b, const Checkpoint& K) {
    const SimParams& P = b->P;
    const DevBuf& B = b->B;
    const int n = P.n;
    b->steps = K.steps;
    const int q = (int)((b->steps & 1) ^ 1);
    cudaStream_t s = b->stream;
    // the device's count of committed steps follows the restored step number
    const long long committed = K.steps;
    DEM_CK(cudaMemcpyAsync(B.committed, &committed, sizeof committed, cudaMemcpyHostToDevice, s));
    auto cp = [&](void* dst, const void* src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s) : cudaSuccess;
    };
    DEM_CK(cp(B.pos, K.pos, n * sizeof(double4_32a)));
    DEM_CK(cp(B.posr, K.posr, n * sizeof(float4)));
    DEM_CK(cp(B.vw0, K.vw0, n * sizeof(VW)));
    DEM_CK(cp(B.id, K.id, n * sizeof(int)));
    DEM_CK(cp(B.lvl, K.lvl, n * sizeof(int)));
    DEM_CK(cp(B.geom, K.geom, P.ng * sizeof(GeomDev)));
    DEM_CK(cp(B.own_start[q], K.own_start, (n + 1) * sizeof(int)));
    DEM_CK(cp(B.geo_start[q], K.geo_start, (n + 1) * sizeof(int)));
    DEM_CK(cp(B.c_key[q], K.c_key, K.nc_prev * sizeof(int)));
    DEM_CK(cp(B.lamW[q], K.lamW, 2 * (size_t)K.nc_prev * sizeof(float4)));
    DEM_CK(cp(B.g_key[q], K.g_key, K.ngc_prev * sizeof(int)));
    DEM_CK(cp(B.glamW[q], K.glamW, 2 * (size_t)K.ngc_prev * sizeof(float4)));
    DEM_CK(cp(B.c_delta, K.c_delta, K.nc_prev * sizeof(float)));
    DEM_CK(cp(B.g_delta, K.g_delta, K.ngc_prev * sizeof(float)));
    DEM_CK(cp(B.grp, K.grp, DEM_MAX_GROUPS * sizeof(GroupDev)));
    DEM_CK(cudaMemsetAsync(B.resorted, 0, sizeof(int), s));
    return DEM_OK;
}

// ---------------------------------------------------------------------------
// host: one step recomputed with its tape
// ---------------------------------------------------------------------------
// counts: this step's and the previous step's contacts (known from dem_record,
// so that the recompute needs no synchronisation)
static dem_status tape_step(dem_bed* b, TapeStep& T, int nc, int ngc, int ncp, int ngcp) {
    const SimParams& P = b->P;
    const DevBuf& B = b->B;
    cudaStream_t s = b->stream;
    const int n = P.n, nit = P.n_it;
    const bool resort = b->g_resort && b->steps % b->resort_every == 0;
    const int p = (int)(b->steps & 1), q = p ^ 1;
    if (resort) DEM_CK(cudaGraphLaunch(b->g_resort, s));
    DEM_CK(cudaGraphLaunch(b->g[p][0], s));   // contacts, rows, warm start, v^0
    (void)q;
    T.nc = nc; T.ngc = ngc; T.nc_prev = ncp; T.ngc_prev = ngcp;
    dem_status st;
    T.resorted = resort ? 1 : 0;
    T.step = b->steps;
    const size_t it = std::max(nit, 1);
    st = carve_alloc(b, T.mem, T.bytes, [&](Carver& c) {
        c.take(T.vw0, n); c.take(T.rad, n); c.take(T.cnt, n); c.take(T.prev_of, n);
        c.take(T.inc_start, n + 1); c.take(T.geo_start, n + 1); c.take(T.inc, 2 * (size_t)nc);
        c.take(T.c_self, nc); c.take(T.c_other, nc); c.take(T.c_pos, nc); c.take(T.rec, 3 * (size_t)nc);
        c.take(T.delta, nc); c.take(T.c_prev, nc); c.take(T.c_warm, 2 * (size_t)nc);
        c.take(T.grec, 6 * (size_t)ngc); c.take(T.gdelta, ngc); c.take(T.g_prev, ngc); c.take(T.g_warm, 2 * (size_t)ngc);
        c.take(T.gdn, 9 * (size_t)ngc);
        c.take(T.lamA, it * nc); c.take(T.lamB, it * nc); c.take(T.glamA, it * ngc); c.take(T.glamB, it * ngc);
        c.take(T.v, it * n);
    });
    if (st != DEM_OK) return st;
    auto cp = [&](void* dst, const void* src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s) : cudaSuccess;
    };
    DEM_CK(cp(T.inc_start, B.inc_start, (n + 1) * sizeof(int)));
    DEM_CK(cp(T.geo_start, B.geo_start[p], (n + 1) * sizeof(int)));
    DEM_CK(cp(T.inc, B.inc, 2 * (size_t)nc * sizeof(int2)));
    DEM_CK(cp(T.c_self, B.c_self, nc * sizeof(int)));
    DEM_CK(cp(T.c_other, B.c_other, nc * sizeof(int)));
    DEM_CK(cp(T.c_pos, B.c_pos, nc * sizeof(int2)));
    DEM_CK(cp(T.rec, B.rec, 3 * (size_t)nc * sizeof(float4)));
    DEM_CK(cp(T.delta, B.c_delta, nc * sizeof(float)));
    DEM_CK(cp(T.grec, B.grec, 6 * (size_t)ngc * sizeof(float4)));
    DEM_CK(cp(T.gdelta, B.g_delta, ngc * sizeof(float)));
    k_tape_bodies<<<nblk(n, AD_T), AD_T, 0, s>>>(P, B, p, T);
    const int gi = std::min(nblk((long long)nc + ngc + n, AD_T), 8 * 152);
    auto iter = [&](int k, int from) {
        launch_pdl_adj(k_tape_iter, gi, s, n, nc, ngc, (const float4*)B.lamA[from], (const float2*)B.lamB[from],
                       (const float4*)B.glamA[from], (const float2*)B.glamB[from], (const VW*)B.vw[from],
                       T.lamA + (size_t)k * nc, T.lamB + (size_t)k * nc, T.glamA + (size_t)k * ngc,
                       T.glamB + (size_t)k * ngc, T.v + (size_t)k * n);
    };
    iter(0, 0);   // lambda^0, v^0 (with no sweeps, also the final iterate)
    for (int k = 0; k < nit; ++k) {
        launch_jacobi(P, B, p, k, b->n_active[k], s);
        if (k + 1 < nit) iter(k + 1, ((k & 1) ^ 1));
    }
    DEM_CK(cudaGetLastError());
    if (b->g[p][2]) DEM_CK(cudaGraphLaunch(b->g[p][2], s));
    b->steps++;
    return DEM_OK;
}

// reverse of one taped step; slot `cur` of the ping-pong state holds the
// adjoint of the state after it
static dem_status reverse_step(dem_bed* b, const TapeStep& T, int cur, int widx) {
    AdjointState* S = b->adj;
    const SimParams& P = b->P;
    cudaStream_t s = b->stream;
    const int n = P.n, nit = P.n_it, nx = cur ^ 1;
    AdjBufs Q;
    Q.xbar_in = S->xbar[cur]; Q.sbar_in = S->sbar[cur];
    Q.xbar_out = S->xbar[nx]; Q.sbar_out = S->sbar[nx];
    Q.vb[0] = S->vb[0]; Q.vb[1] = S->vb[1];
    Q.vacc = S->vacc;
    Q.L = S->L; Q.A = S->A; Q.gL = S->gL; Q.gA = S->gA;
    Q.lw_in = S->lw[cur]; Q.glw_in = S->glw[cur];
    Q.lw_out = S->lw[nx]; Q.glw_out = S->glw[nx];
    Q.sh = b->B.imp;
    Q.wts = S->wts + (size_t)widx * 3 * std::max(P.ng, 1);
    Q.part = S->part;
    const int gi = std::min(nblk((long long)n + T.nc + T.ngc, AD_T), 8 * 152);
    k_adj_init<<<gi, AD_T, 0, s>>>(P, T, Q, nit & 1);
    const int cb = std::max(1, std::min(nblk(T.nc, AD_T), 16 * 152));
    for (int k = nit - 1; k >= 0; --k) {
        DEM_CK(launch_pdl_adj(k_adj_contacts, cb, s, P, T, Q, k));
        DEM_CK(launch_pdl_adj(k_adj_bodies, nblk(n, AD_T), s, P, T, Q, k));
    }
    // the previous step's final impulses: only those continued here get an adjoint
    if (T.nc_prev > 0) DEM_CK(cudaMemsetAsync(Q.lw_out, 0, 2 * (size_t)T.nc_prev * sizeof(float4), s));
    if (T.ngc_prev > 0) DEM_CK(cudaMemsetAsync(Q.glw_out, 0, 2 * (size_t)T.ngc_prev * sizeof(float4), s));
    k_adj_rows<<<AD_RED_BLOCKS, AD_T, 0, s>>>(P, T, Q);
    const int sb = nblk(n, AD_T);
    k_adj_state<<<sb, AD_T, 0, s>>>(P, T, Q);
    k_adj_reduce<<<1, AD_RED_T, 0, s>>>(S->part, AD_RED_BLOCKS, sb, S->grad);
    DEM_CK(cudaGetLastError());
    return DEM_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
static dem_status check_supported(dem_bed* b) {
    const SimParams& P = b->P;
    if (!P.nit_uniform) return dem_fail(DEM_ERR_ARG, "the adjoint needs the same n_it in every bed");
    if (P.solver) return dem_fail(DEM_ERR_ARG, "the adjoint reverses the Jacobi solver only");
    if (P.v_imp > 0.f) return dem_fail(DEM_ERR_ARG, "the adjoint does not reverse the impact stage");
    std::vector<GeomDev> hg(std::max(P.ng, 1));
    if (P.ng > 0) {
        // ordered after pending velocity changes on the bed's stream
        DEM_CK(cudaMemcpyAsync(hg.data(), b->B.geom, P.ng * sizeof(GeomDev), cudaMemcpyDeviceToHost, b->stream));
        DEM_CK(cudaStreamSynchronize(b->stream));
    }
    for (int g = 0; g < P.ng; ++g) {
        if (hg[g].grp >= 0)
            return dem_fail(DEM_ERR_ARG, "the adjoint does not support load-driven primitives (primitive %d)", g);
        if (hg[g].w[0] != 0.0 || hg[g].w[1] != 0.0 || hg[g].w[2] != 0.0)
            return dem_fail(DEM_ERR_ARG, "the adjoint supports primitives that do not spin (primitive %d)", g);
    }
    return DEM_OK;
}

// ---------------------------------------------------------------------------
// whole-state checkpoints for callers (restart a window, finite differences)
// ---------------------------------------------------------------------------
struct dem_checkpoint {
    dem_bed* bed = nullptr;
    Checkpoint K;
    long long* gacc = nullptr;   // geometry impulses of the step before the snapshot
};

extern "C" dem_status dem_checkpoint_save(dem_bed* b, dem_checkpoint** out) {
    dem_set_error_message("");
    if (!b || !out) return dem_fail(DEM_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (b->faulted) return dem_fail(DEM_ERR_STATE, "the bed holds a latched device fault");
    DEM_CK(cudaSetDevice(b->dev));
    // a pending overflow is repaired (its steps re-run) before the snapshot
    dem_status st0 = dem_check_fault(b);
    if (st0 != DEM_OK) return st0;
    dem_checkpoint* c = new dem_checkpoint();
    c->bed = b;
    const size_t ng = std::max(b->P.ng, 1);
    dem_status st = save_checkpoint(b, c->K);
    if (st == DEM_OK) st = dem_dalloc(b, (void**)&c->gacc, 6 * ng * sizeof(long long));
    if (st == DEM_OK) {
        cudaError_t e = cudaMemcpyAsync(c->gacc, b->B.gacc, 6 * ng * sizeof(long long), cudaMemcpyDeviceToDevice,
                                        b->stream);
        if (e != cudaSuccess) st = dem_fail(DEM_ERR_CUDA, "%s", cudaGetErrorString(e));
    }
    if (st == DEM_OK) st = dem_check_fault(b);
    if (st != DEM_OK) {
        if (c->K.mem) dem_dfree(b, c->K.mem);
        if (c->gacc) dem_dfree(b, c->gacc);
        delete c;
        return st;
    }
    *out = c;
    return DEM_OK;
}

extern "C" dem_status dem_checkpoint_restore(dem_bed* b, const dem_checkpoint* c) {
    dem_set_error_message("");
    if (!b || !c) return dem_fail(DEM_ERR_ARG, "NULL argument");
    if (c->bed != b) return dem_fail(DEM_ERR_ARG, "the checkpoint belongs to another bed");
    if (b->faulted) return dem_fail(DEM_ERR_STATE, "the bed holds a latched device fault");
    DEM_CK(cudaSetDevice(b->dev));
    // a pending overflow is repaired before the state is replaced
    dem_status st = dem_check_fault(b);
    if (st != DEM_OK) return st;
    st = restore_checkpoint(b, c->K);
    if (st != DEM_OK) return st;
    const size_t ng = std::max(b->P.ng, 1);
    DEM_CK(cudaMemcpyAsync(b->B.gacc, c->gacc, 6 * ng * sizeof(long long), cudaMemcpyDeviceToDevice, b->stream));
    if (b->adj) b->adj->recorded = false;   // the recorded window no longer ends here
    return dem_check_fault(b);
}

extern "C" dem_status dem_checkpoint_free(dem_bed* b, dem_checkpoint* c) {
    dem_set_error_message("");
    if (!c) return DEM_OK;
    if (!b || c->bed != b) return dem_fail(DEM_ERR_ARG, "the checkpoint belongs to another bed");
    DEM_CK(cudaSetDevice(b->dev));
    if (c->K.mem) dem_dfree(b, c->K.mem);
    if (c->gacc) dem_dfree(b, c->gacc);
    delete c;
    return DEM_OK;
}

// Checkpoint interval that minimises the window's memory.  Every step is
// recomputed exactly once in the reverse pass whatever the interval, so the
// interval only trades checkpoints (nsteps / k of them) against the tapes of
// one segment (k steps): k = sqrt(nsteps * checkpoint / tape of one step),
// sizes estimated from the last step's contact count.
static int auto_interval(dem_bed* b, int nsteps) {
    int nc = 0, ngc = 0;
    if (b->steps > 0) read_counts(b, (int)((b->steps - 1) & 1), &nc, &ngc);
    const double n = std::max(b->P.n, 1), c = (double)nc + ngc;
    const double ckpt = 100.0 * n + 40.0 * c;
    const double tape = std::max(b->P.n_it, 1) * (24.0 * c + 32.0 * n) + 100.0 * c + 80.0 * n;
    const int k = (int)std::lround(std::sqrt((double)nsteps * ckpt / tape));
    return std::min(std::max(k, 1), nsteps);
}

extern "C" dem_status dem_record(dem_bed* b, int32_t nsteps, int32_t ckpt_every, double* forces) {
    dem_set_error_message("");
    if (!b) return dem_fail(DEM_ERR_ARG, "bed is NULL");
    if (nsteps < 1 || ckpt_every < 0) return dem_fail(DEM_ERR_ARG, "need nsteps >= 1 and ckpt_every >= 0");
    if (b->faulted) return dem_fail(DEM_ERR_STATE, "the bed holds a latched device fault");
    DEM_CK(cudaSetDevice(b->dev));
    dem_status st = check_supported(b);
    if (st != DEM_OK) return st;
    if (ckpt_every == 0) ckpt_every = auto_interval(b, nsteps);
    if ((st = ensure_state(b)) != DEM_OK) return st;
    AdjointState* S = b->adj;
    S->recorded = false;
    S->t0 = b->steps;
    S->nsteps = nsteps;
    S->every = ckpt_every;
    S->P = b->P;
    const int nseg = (nsteps + ckpt_every - 1) / ckpt_every;
    if ((int)S->ck.size() < nseg) S->ck.resize(nseg);
    const size_t ng = std::max(b->P.ng, 1);
    const size_t fn = (size_t)nsteps * 6 * ng;
    if (fn > S->fhist_n) {
        if (S->fhist) dem_dfree(b, S->fhist);
        S->fhist = nullptr;
        S->fhist_n = 0;
        if ((st = dem_dalloc(b, (void**)&S->fhist, fn * sizeof(long long))) != DEM_OK) return st;
        S->fhist_n = fn;
    }
    if ((size_t)(2 * nsteps) > S->cnt_n) {
        if (S->cnt_dev) dem_dfree(b, S->cnt_dev);
        S->cnt_dev = nullptr;
        S->cnt_n = 0;
        if ((st = dem_dalloc(b, (void**)&S->cnt_dev, 2 * (size_t)nsteps * sizeof(int))) != DEM_OK) return st;
        S->cnt_n = 2 * (size_t)nsteps;
    }
    // an overflow inside the window is reported, not repaired: the recorded
    // forces and counts would mix the failed and the re-run steps
    b->no_grow = true;
    struct Restore { dem_bed* b; ~Restore() { b->no_grow = false; } } restore{b};
    for (int t = 0; t < nsteps; ++t) {
        if (t % ckpt_every == 0 && (st = save_checkpoint(b, S->ck[t / ckpt_every])) != DEM_OK) return st;
        const int p = (int)(b->steps & 1);
        if ((st = dem_launch_step(b)) != DEM_OK) return st;
        DEM_CK(cudaMemcpyAsync(S->fhist + (size_t)t * 6 * ng, b->B.gacc, 6 * ng * sizeof(long long),
                               cudaMemcpyDeviceToDevice, b->stream));
        DEM_CK(cudaMemcpyAsync(S->cnt_dev + 2 * t, b->B.own_start[p] + b->P.n, sizeof(int),
                               cudaMemcpyDeviceToDevice, b->stream));
        DEM_CK(cudaMemcpyAsync(S->cnt_dev + 2 * t + 1, b->B.geo_start[p] + b->P.n, sizeof(int),
                               cudaMemcpyDeviceToDevice, b->stream));
    }
    if ((st = save_checkpoint(b, S->end)) != DEM_OK) return st;
    S->counts.assign(2 * (size_t)nsteps, 0);
    DEM_CK(cudaMemcpyAsync(S->counts.data(), S->cnt_dev, 2 * (size_t)nsteps * sizeof(int), cudaMemcpyDeviceToHost,
                           b->stream));
    if ((st = dem_check_fault(b)) != DEM_OK) return st;
    if (forces) {
        std::vector<long long> h(fn);
        DEM_CK(cudaMemcpy(h.data(), S->fhist, fn * sizeof(long long), cudaMemcpyDeviceToHost));
        std::vector<double> out((size_t)nsteps * 3 * ng);
        const double sc = 1.0 / (DEM_FIX_SCALE * (double)b->P.dt);
        for (int t = 0; t < nsteps; ++t)
            for (int g = 0; g < b->P.ng; ++g)
                for (int k = 0; k < 3; ++k)
                    out[((size_t)t * b->P.ng + g) * 3 + k] = (double)h[((size_t)t * ng + g) * 6 + k] * sc;
        if (b->P.ng > 0)
            DEM_CK(cudaMemcpy(forces, out.data(), (size_t)nsteps * 3 * b->P.ng * sizeof(double), cudaMemcpyDefault));
    }
    S->recorded = true;
    return DEM_OK;
}

extern "C" dem_status dem_step_adjoint(dem_bed* b, const double* dJ_dF, double grad[3]) {
    dem_set_error_message("");
    if (!b || !grad) return dem_fail(DEM_ERR_ARG, "NULL argument");
    if (b->faulted) return dem_fail(DEM_ERR_STATE, "the bed holds a latched device fault");
    AdjointState* S = b->adj;
    if (!S || !S->recorded) return dem_fail(DEM_ERR_STATE, "no window recorded (call dem_record first)");
    if (memcmp(&S->P, &b->P, sizeof(SimParams)) != 0)
        return dem_fail(DEM_ERR_STATE, "solver settings changed since dem_record");
    if (b->steps != S->end.steps) return dem_fail(DEM_ERR_STATE, "the bed was stepped after dem_record");
    // the reverse pass re-runs recorded steps at the recorded capacity: no growth
    b->no_grow = true;
    struct Restore { dem_bed* b; ~Restore() { b->no_grow = false; } } restore{b};
    if (S->P.ng > 0 && !dJ_dF) return dem_fail(DEM_ERR_ARG, "dJ_dF is NULL");
    DEM_CK(cudaSetDevice(b->dev));
    cudaStream_t s = b->stream;
    const SimParams& P = b->P;
    const int n = P.n, ng = P.ng, ngd = std::max(ng, 1);
    // dJ/dF on the device, as float
    const size_t wn = (size_t)S->nsteps * 3 * ngd;
    if (wn > S->wts_n) {
        if (S->wts) dem_dfree(b, S->wts);
        S->wts = nullptr;
        S->wts_n = 0;
        dem_status st = dem_dalloc(b, (void**)&S->wts, wn * sizeof(float));
        if (st != DEM_OK) return st;
        S->wts_n = wn;
    }
    {
        std::vector<double> hd((size_t)S->nsteps * 3 * ng);
        if (ng > 0) DEM_CK(cudaMemcpy(hd.data(), dJ_dF, hd.size() * sizeof(double), cudaMemcpyDefault));
        std::vector<float> hw(wn, 0.f);
        for (int t = 0; t < S->nsteps; ++t)
            for (int k = 0; k < 3 * ng; ++k) hw[(size_t)t * 3 * ngd + k] = (float)hd[(size_t)t * 3 * ng + k];
        DEM_CK(cudaMemcpy(S->wts, hw.data(), wn * sizeof(float), cudaMemcpyHostToDevice));
    }
    if (n == 0) {   // nothing depends on the parameters
        for (int k = 0; k < 3; ++k) grad[k] = 0.0;
        return DEM_OK;
    }
    // the state after the window has a zero adjoint
    const size_t N = std::max(n, 1);
    int cur = 0;
    DEM_CK(cudaMemsetAsync(S->xbar[cur], 0, N * sizeof(float4), s));
    DEM_CK(cudaMemsetAsync(S->sbar[cur], 0, N * sizeof(VW), s));
    DEM_CK(cudaMemsetAsync(S->grad, 0, 4 * sizeof(double), s));
    {
        int nc = 0, ngc = 0;
        dem_status st = read_counts(b, (int)((b->steps - 1) & 1), &nc, &ngc);
        if (st != DEM_OK) return st;
        if (nc > 0) DEM_CK(cudaMemsetAsync(S->lw[cur], 0, 2 * (size_t)nc * sizeof(float4), s));
        if (ngc > 0) DEM_CK(cudaMemsetAsync(S->glw[cur], 0, 2 * (size_t)ngc * sizeof(float4), s));
    }
    const int nseg = (S->nsteps + S->every - 1) / S->every;
    if ((int)S->tape.size() < S->every) S->tape.resize(S->every);
    dem_status st = DEM_OK;
    for (int seg = nseg - 1; seg >= 0 && st == DEM_OK; --seg) {
        const int first = seg * S->every, len = std::min(S->every, S->nsteps - first);
        if ((st = restore_checkpoint(b, S->ck[seg])) != DEM_OK) break;
        for (int j = 0; j < len && st == DEM_OK; ++j) {
            const int t = first + j;
            const int ncp = t > 0 ? S->counts[2 * (t - 1)] : S->ck[0].nc_prev;
            const int ngcp = t > 0 ? S->counts[2 * (t - 1) + 1] : S->ck[0].ngc_prev;
            st = tape_step(b, S->tape[j], S->counts[2 * t], S->counts[2 * t + 1], ncp, ngcp);
        }
        for (int j = len - 1; j >= 0 && st == DEM_OK; --j) {
            st = reverse_step(b, S->tape[j], cur, first + j);
            cur ^= 1;
        }
    }
    // back to the state after the window, with the last step's geometry impulses
    if (st == DEM_OK) st = restore_checkpoint(b, S->end);
    if (st != DEM_OK) return st;
    DEM_CK(cudaMemcpyAsync(b->B.gacc, S->fhist + (size_t)(S->nsteps - 1) * 6 * ngd, 6 * ngd * sizeof(long long),
                           cudaMemcpyDeviceToDevice, s));
    double g[4];
    DEM_CK(cudaMemcpyAsync(g, S->grad, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    if ((st = dem_check_fault(b)) != DEM_OK) return st;
    for (int k = 0; k < 3; ++k) grad[k] = g[k];
    return DEM_OK;
}
