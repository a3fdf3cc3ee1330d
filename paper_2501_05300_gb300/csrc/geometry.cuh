// Exact FP64 contact tests shared by the detection and the contact-row
// kernels.  Every product and sum is rounded on its own (explicit _rn
// intrinsics, so the compiler cannot fuse them): the predicates are defined by
// this exact sequence of IEEE double operations.
#pragma once
#include "dem_internal.cuh"

static __device__ __forceinline__ double dm(double a, double b) { return __dmul_rn(a, b); }
static __device__ __forceinline__ double da(double a, double b) { return __dadd_rn(a, b); }
static __device__ __forceinline__ double ds(double a, double b) { return __dsub_rn(a, b); }

static __device__ __forceinline__ bool exact_pair(double4_32a a, double4_32a b) {
    double dx = ds(a.x, b.x), dy = ds(a.y, b.y), dz = ds(a.z, b.z);
    double d2 = da(da(dm(dx, dx), dm(dy, dy)), dm(dz, dz));
    double R = da(a.w, b.w);
    return d2 < dm(R, R);
}

struct GeoHit {
    bool hit;
    double delta;
    double n[3];   // unit normal from the primitive to the sphere centre (world)
    double q[3];   // contact point on the primitive surface (world)
};

// Closest point of a sphere on a solid primitive; contact iff overlap > 0.
// Same operation sequence as the definition in the FP64 reference.
static __device__ GeoHit geom_hit(const GeomDev& g, double x0, double x1, double x2, double r) {
    GeoHit h;
    h.hit = false;
    if (g.type == DEM_GEOM_PLANE) {
        double n0 = g.R[2], n1 = g.R[5], n2 = g.R[8];
        double dx = ds(x0, g.c[0]), dy = ds(x1, g.c[1]), dz = ds(x2, g.c[2]);
        double s = da(da(dm(n0, dx), dm(n1, dy)), dm(n2, dz));
        if (!(s < r)) return h;
        h.hit = true;
        h.delta = ds(r, s);
        h.n[0] = n0; h.n[1] = n1; h.n[2] = n2;
        h.q[0] = ds(x0, dm(s, n0)); h.q[1] = ds(x1, dm(s, n1)); h.q[2] = ds(x2, dm(s, n2));
        return h;
    }
    double d0 = ds(x0, g.c[0]), d1 = ds(x1, g.c[1]), d2 = ds(x2, g.c[2]);
    double q[3], cl[3], nl[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) q[j] = da(da(dm(g.R[j], d0), dm(g.R[3 + j], d1)), dm(g.R[6 + j], d2));
    if (g.type == DEM_GEOM_BOX) {
#pragma unroll
        for (int k = 0; k < 3; ++k) cl[k] = q[k] < -g.he[k] ? -g.he[k] : (q[k] > g.he[k] ? g.he[k] : q[k]);
        double e0 = ds(q[0], cl[0]), e1 = ds(q[1], cl[1]), e2 = ds(q[2], cl[2]);
        double ee = da(da(dm(e0, e0), dm(e1, e1)), dm(e2, e2));
        if (ee > 0.0) {
            if (!(ee < dm(r, r))) return h;
            double d = __dsqrt_rn(ee);
            nl[0] = __ddiv_rn(e0, d); nl[1] = __ddiv_rn(e1, d); nl[2] = __ddiv_rn(e2, d);
            h.delta = ds(r, d);
        } else {
            int kb = 0;
            double best = ds(g.he[0], fabs(q[0]));
            for (int k = 1; k < 3; ++k) {
                double dk = ds(g.he[k], fabs(q[k]));
                if (dk < best) { best = dk; kb = k; }
            }
            double sg = q[kb] < 0.0 ? -1.0 : 1.0;
            nl[0] = nl[1] = nl[2] = 0.0;
            nl[kb] = sg;
            cl[0] = q[0]; cl[1] = q[1]; cl[2] = q[2];
            cl[kb] = dm(sg, g.he[kb]);
            h.delta = da(r, best);
        }
    } else {  // cylinder, axis local z
        double Rc = g.he[0], H = g.he[2];
        double rho2 = da(dm(q[0], q[0]), dm(q[1], q[1]));
        if (rho2 > dm(Rc, Rc)) {
            double rho = __dsqrt_rn(rho2);
            double s = __ddiv_rn(Rc, rho);
            cl[0] = dm(q[0], s); cl[1] = dm(q[1], s);
        } else {
            cl[0] = q[0]; cl[1] = q[1];
        }
        cl[2] = q[2] < -H ? -H : (q[2] > H ? H : q[2]);
        double e0 = ds(q[0], cl[0]), e1 = ds(q[1], cl[1]), e2 = ds(q[2], cl[2]);
        double ee = da(da(dm(e0, e0), dm(e1, e1)), dm(e2, e2));
        if (ee > 0.0) {
            if (!(ee < dm(r, r))) return h;
            double d = __dsqrt_rn(ee);
            nl[0] = __ddiv_rn(e0, d); nl[1] = __ddiv_rn(e1, d); nl[2] = __ddiv_rn(e2, d);
            h.delta = ds(r, d);
        } else {
            double rho = __dsqrt_rn(rho2);
            double dax = ds(H, fabs(q[2]));
            double drd = ds(Rc, rho);
            if (dax <= drd) {
                double sg = q[2] < 0.0 ? -1.0 : 1.0;
                nl[0] = 0.0; nl[1] = 0.0; nl[2] = sg;
                cl[0] = q[0]; cl[1] = q[1]; cl[2] = dm(sg, H);
                h.delta = da(r, dax);
            } else {
                if (rho > 0.0) { nl[0] = __ddiv_rn(q[0], rho); nl[1] = __ddiv_rn(q[1], rho); }
                else { nl[0] = 1.0; nl[1] = 0.0; }
                nl[2] = 0.0;
                cl[0] = dm(nl[0], Rc); cl[1] = dm(nl[1], Rc); cl[2] = q[2];
                h.delta = da(r, drd);
            }
        }
    }
    h.hit = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        h.n[i] = da(da(dm(g.R[3 * i], nl[0]), dm(g.R[3 * i + 1], nl[1])), dm(g.R[3 * i + 2], nl[2]));
        double w = da(da(dm(g.R[3 * i], cl[0]), dm(g.R[3 * i + 1], cl[1])), dm(g.R[3 * i + 2], cl[2]));
        h.q[i] = da(g.c[i], w);
    }
    return h;
}

