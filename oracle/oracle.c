/*
 * FP64 CPU oracle for the nonsmooth sphere DEM step of arXiv 2501.05300.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * benchmark's CPU-baseline leg; never by the library.  Shares nothing with the
 * CUDA code.  See oracle.h for the list of what it computes.
 *
 * Every floating-point value is a double.  Compile with -ffp-contract=off so
 * that no multiply-add is fused: the contact predicates below are defined by
 * the exact sequence of IEEE double operations written here.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* small vector helpers                                                       */
/* ------------------------------------------------------------------------- */
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* o) {
    double x = a[1] * b[2] - a[2] * b[1];
    double y = a[2] * b[0] - a[0] * b[2];
    double z = a[0] * b[1] - a[1] * b[0];
    o[0] = x; o[1] = y; o[2] = z;
}
static double norm3(const double* a) { return sqrt(dot3(a, a)); }

/* ------------------------------------------------------------------------- */
/* contact geometry                                                           */
/* ------------------------------------------------------------------------- */
typedef struct {
    int hit;
    double delta;   /* overlap > 0 when in contact */
    double n[3];    /* unit normal from the geometry towards the sphere centre */
    double q[3];    /* contact point on the geometry surface (world) */
} geo_hit;

/* local coordinates q = R^T (x - c), evaluated left to right */
static void to_local(const orc_geom* g, const double* x, double* q) {
    double d0 = x[0] - g->c[0], d1 = x[1] - g->c[1], d2 = x[2] - g->c[2];
    for (int j = 0; j < 3; ++j) q[j] = g->R[0 * 3 + j] * d0 + g->R[1 * 3 + j] * d1 + g->R[2 * 3 + j] * d2;
}
static void to_world_dir(const orc_geom* g, const double* l, double* o) {
    for (int i = 0; i < 3; ++i) o[i] = g->R[i * 3 + 0] * l[0] + g->R[i * 3 + 1] * l[1] + g->R[i * 3 + 2] * l[2];
}
static void to_world_pt(const orc_geom* g, const double* l, double* o) {
    double d[3];
    to_world_dir(g, l, d);
    for (int i = 0; i < 3; ++i) o[i] = g->c[i] + d[i];
}

/* Closest point of a sphere (centre x, radius r) on a solid primitive.  The
 * contact exists iff the overlap is strictly positive (Sec. 2.2: active contacts
 * have a finite overlap). */
static geo_hit sphere_geom(const orc_geom* g, const double* x, double r) {
    geo_hit h;
    memset(&h, 0, sizeof h);
    if (g->type == ORC_PLANE) {
        double nz[3] = {g->R[2], g->R[5], g->R[8]};
        double dx = x[0] - g->c[0], dy = x[1] - g->c[1], dz = x[2] - g->c[2];
        double s = nz[0] * dx + nz[1] * dy + nz[2] * dz; /* signed height above the plane */
        if (!(s < r)) return h;
        h.hit = 1;
        h.delta = r - s;
        for (int i = 0; i < 3; ++i) { h.n[i] = nz[i]; h.q[i] = x[i] - s * nz[i]; }
        return h;
    }
    double q[3], cl[3], nl[3];
    to_local(g, x, q);
    if (g->type == ORC_BOX) {
        for (int k = 0; k < 3; ++k) cl[k] = q[k] < -g->he[k] ? -g->he[k] : (q[k] > g->he[k] ? g->he[k] : q[k]);
        double e0 = q[0] - cl[0], e1 = q[1] - cl[1], e2 = q[2] - cl[2];
        double ee = e0 * e0 + e1 * e1 + e2 * e2;
        if (ee > 0.0) {
            if (!(ee < r * r)) return h;
            double d = sqrt(ee);
            nl[0] = e0 / d; nl[1] = e1 / d; nl[2] = e2 / d;
            h.delta = r - d;
        } else {
            /* centre inside: push out through the nearest face */
            int kb = 0;
            double best = g->he[0] - fabs(q[0]);
            for (int k = 1; k < 3; ++k) {
                double dk = g->he[k] - fabs(q[k]);
                if (dk < best) { best = dk; kb = k; }
            }
            double sg = q[kb] < 0.0 ? -1.0 : 1.0;
            nl[0] = nl[1] = nl[2] = 0.0;
            nl[kb] = sg;
            cl[0] = q[0]; cl[1] = q[1]; cl[2] = q[2];
            cl[kb] = sg * g->he[kb];
            h.delta = r + best;
        }
    } else { /* ORC_CYLINDER, axis = local z */
        double Rc = g->he[0], H = g->he[2];
        double rho2 = q[0] * q[0] + q[1] * q[1];
        if (rho2 > Rc * Rc) {
            double rho = sqrt(rho2);
            double s = Rc / rho;
            cl[0] = q[0] * s; cl[1] = q[1] * s;
        } else {
            cl[0] = q[0]; cl[1] = q[1];
        }
        cl[2] = q[2] < -H ? -H : (q[2] > H ? H : q[2]);
        double e0 = q[0] - cl[0], e1 = q[1] - cl[1], e2 = q[2] - cl[2];
        double ee = e0 * e0 + e1 * e1 + e2 * e2;
        if (ee > 0.0) {
            if (!(ee < r * r)) return h;
            double d = sqrt(ee);
            nl[0] = e0 / d; nl[1] = e1 / d; nl[2] = e2 / d;
            h.delta = r - d;
        } else {
            double rho = sqrt(rho2);
            double da = H - fabs(q[2]);
            double dr = Rc - rho;
            if (da <= dr) {
                double sg = q[2] < 0.0 ? -1.0 : 1.0;
                nl[0] = 0.0; nl[1] = 0.0; nl[2] = sg;
                cl[0] = q[0]; cl[1] = q[1]; cl[2] = sg * H;
                h.delta = r + da;
            } else {
                if (rho > 0.0) { nl[0] = q[0] / rho; nl[1] = q[1] / rho; }
                else { nl[0] = 1.0; nl[1] = 0.0; }
                nl[2] = 0.0;
                cl[0] = nl[0] * Rc; cl[1] = nl[1] * Rc; cl[2] = q[2];
                h.delta = r + dr;
            }
        }
    }
    h.hit = 1;
    to_world_dir(g, nl, h.n);
    to_world_pt(g, cl, h.q);
    return h;
}

/* Sphere-sphere predicate: |x_a - x_b|^2 < (r_a + r_b)^2 in IEEE double, the
 * squared distance summed as (dx^2 + dy^2) + dz^2. */
static int sphere_pair(const double* xa, double ra, const double* xb, double rb, double* d2out) {
    double dx = xa[0] - xb[0], dy = xa[1] - xb[1], dz = xa[2] - xb[2];
    double d2 = dx * dx + dy * dy + dz * dz;
    double R = ra + rb;
    *d2out = d2;
    return d2 < R * R;
}

/* ------------------------------------------------------------------------- */
/* brute-force detection                                                      */
/* ------------------------------------------------------------------------- */
typedef struct { int32_t ka, kb; int a, b; double delta; } raw_contact;

static int cmp_raw(const void* p, const void* q) {
    const raw_contact* x = (const raw_contact*)p;
    const raw_contact* y = (const raw_contact*)q;
    if (x->ka != y->ka) return x->ka < y->ka ? -1 : 1;
    if (x->kb != y->kb) return x->kb < y->kb ? -1 : 1;
    return 0;
}

typedef struct { raw_contact* v; int64_t n, cap; } raw_vec;
static void raw_push(raw_vec* r, raw_contact c) {
    if (r->n == r->cap) {
        r->cap = r->cap ? 2 * r->cap : 64;
        r->v = (raw_contact*)realloc(r->v, (size_t)r->cap * sizeof(raw_contact));
    }
    r->v[r->n++] = c;
}

/* All sphere-sphere pairs i<j are tested (O(N^2)), then every sphere against
 * every geometry.  Output sorted by key. */
static raw_vec detect_all(int32_t n, const double* x, const double* r, const int32_t* id,
                          int32_t ng, const orc_geom* g) {
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    raw_vec* part = (raw_vec*)calloc((size_t)nthr, sizeof(raw_vec));
#pragma omp parallel for schedule(dynamic, 64)
    for (int32_t i = 0; i < n; ++i) {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        for (int32_t j = i + 1; j < n; ++j) {
            double d2;
            if (sphere_pair(&x[3 * i], r[i], &x[3 * j], r[j], &d2)) {
                raw_contact c;
                int lo = id[i] < id[j] ? i : j, hi = id[i] < id[j] ? j : i;
                c.a = lo; c.b = hi; c.ka = id[lo]; c.kb = id[hi];
                c.delta = (r[i] + r[j]) - sqrt(d2);
                raw_push(&part[t], c);
            }
        }
        for (int32_t k = 0; k < ng; ++k) {
            geo_hit h = sphere_geom(&g[k], &x[3 * i], r[i]);
            if (h.hit) {
                raw_contact c;
                c.a = i; c.b = -(k + 1); c.ka = id[i]; c.kb = -(k + 1);
                c.delta = h.delta;
                raw_push(&part[t], c);
            }
        }
    }
    raw_vec all = {0, 0, 0};
    for (int t = 0; t < nthr; ++t) {
        for (int64_t k = 0; k < part[t].n; ++k) raw_push(&all, part[t].v[k]);
        free(part[t].v);
    }
    free(part);
    if (all.n > 1) qsort(all.v, (size_t)all.n, sizeof(raw_contact), cmp_raw);
    return all;
}

int64_t orc_detect(int32_t n, const double* x, const double* r, const int32_t* id,
                   int32_t ng, const orc_geom* g, int64_t cap,
                   int32_t* out_a, int32_t* out_b, double* out_delta) {
    raw_vec all = detect_all(n, x, r, id, ng, g);
    for (int64_t k = 0; k < all.n && k < cap; ++k) {
        out_a[k] = all.v[k].ka;
        out_b[k] = all.v[k].kb;
        out_delta[k] = all.v[k].delta;
    }
    int64_t m = all.n;
    free(all.v);
    return m;
}

/* ------------------------------------------------------------------------- */
/* simulation state                                                           */
/* ------------------------------------------------------------------------- */
typedef struct {
    int a, b;               /* body indices; b < 0 is geometry -(g+1) */
    int32_t ka, kb;
    double delta;
    double n[3];            /* from b to a */
    double la[3], lb[3];    /* contact points relative to the centre of a and of b */
    double t1[3], t2[3];    /* tangent basis */
    double Ga[6][6], Gb[6][6]; /* rows: normal, t1, t2, roll x, roll y, roll z; cols: linear, angular */
    double known[6];        /* G_b (v_g, w_g) for kinematic geometry */
    double known_ang[6];    /* its angular part G_b (0, w_g) */
    int grp;                /* load-driven group of the primitive, or -1 */
    double sig[6], rhs[6];
    double Dn_inv, Dt_inv[2][2], Dr_inv[3][3];
    double mu_t, mu_r_reff;
    double lam[6], lam_new[6];
} contact;

typedef struct { int32_t ka, kb; double lam7[7]; } ws_entry;

struct orc_sim {
    orc_params p;
    int32_t n, ng;
    double *x, *r, *v, *w, *inv_m, *inv_I;
    int32_t* id;
    orc_geom* g;
    contact* c;
    int64_t nc;
    ws_entry* ws;
    int64_t nws;
    double* gforce; /* 6 per geometry */
    int32_t ncol;     /* colours of the last PGS step */
    int64_t nimp;     /* impacting contacts of the last step */
    double* gimp;     /* 6 per geometry: impact-stage impulse G_b^T p of the last step */
    /* load-driven rigid groups of primitives (orc_set_load) */
    int32_t ngrp;
    int32_t* gbody;   /* per primitive: its group, or -1 (kinematic) */
    struct {
        double mass, force[3];
        int32_t dof;    /* bit k: axis k is dynamic */
        double v[3];    /* velocity of the group's primitives */
    } grp[ORC_MAX_GROUPS];
};

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static double* dup_or_zero(const double* src, size_t m) {
    double* d = (double*)calloc(m ? m : 1, sizeof(double));
    if (src) memcpy(d, src, m * sizeof(double));
    return d;
}

orc_sim* orc_create(const orc_params* p, int32_t n, const double* x, const double* r,
                    const double* v, const double* w, const int32_t* id,
                    const double* inv_m, const double* inv_I,
                    int32_t ng, const orc_geom* g) {
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->p = *p;
    s->n = n;
    s->ng = ng;
    s->x = dup_or_zero(x, 3 * (size_t)n);
    s->r = dup_or_zero(r, (size_t)n);
    s->v = dup_or_zero(v, 3 * (size_t)n);
    s->w = dup_or_zero(w, 3 * (size_t)n);
    s->id = (int32_t*)calloc(n ? n : 1, sizeof(int32_t));
    memcpy(s->id, id, (size_t)n * sizeof(int32_t));
    s->inv_m = (double*)calloc(n ? n : 1, sizeof(double));
    s->inv_I = (double*)calloc(n ? n : 1, sizeof(double));
    for (int32_t i = 0; i < n; ++i) {
        /* solid sphere: m = rho 4/3 pi r^3, I = 2/5 m r^2 */
        double m = p->rho * (4.0 / 3.0) * M_PI * r[i] * r[i] * r[i];
        double I = 0.4 * m * r[i] * r[i];
        s->inv_m[i] = inv_m ? inv_m[i] : 1.0 / m;
        s->inv_I[i] = inv_I ? inv_I[i] : 1.0 / I;
    }
    s->g = (orc_geom*)calloc(ng ? ng : 1, sizeof(orc_geom));
    if (ng) memcpy(s->g, g, (size_t)ng * sizeof(orc_geom));
    s->gforce = (double*)calloc(6 * (size_t)(ng ? ng : 1), sizeof(double));
    s->gimp = (double*)calloc(6 * (size_t)(ng ? ng : 1), sizeof(double));
    s->gbody = (int32_t*)malloc((size_t)(ng ? ng : 1) * sizeof(int32_t));
    for (int32_t k = 0; k < ng; ++k) s->gbody[k] = -1;
    return s;
}

int orc_set_load(orc_sim* s, int32_t count, const int32_t* geoms, double mass, const double force[3],
                 int32_t dof) {
    if (count < 1 || !(mass > 0.0) || dof <= 0 || dof > 7 || s->ngrp >= ORC_MAX_GROUPS) return -1;
    for (int32_t k = 0; k < count; ++k)
        if (geoms[k] < 0 || geoms[k] >= s->ng || s->gbody[geoms[k]] >= 0) return -1;
    const int32_t q = s->ngrp++;
    s->grp[q].mass = mass;
    s->grp[q].dof = dof;
    for (int a = 0; a < 3; ++a) {
        s->grp[q].force[a] = force[a];
        s->grp[q].v[a] = s->g[geoms[0]].v[a];
    }
    for (int32_t k = 0; k < count; ++k) {
        s->gbody[geoms[k]] = q;
        for (int a = 0; a < 3; ++a) s->g[geoms[k]].v[a] = s->grp[q].v[a];
    }
    return 0;
}

int orc_set_load_force(orc_sim* s, int32_t g, const double force[3]) {
    if (g < 0 || g >= s->ng || s->gbody[g] < 0) return -1;
    for (int a = 0; a < 3; ++a) s->grp[s->gbody[g]].force[a] = force[a];
    return 0;
}

void orc_destroy(orc_sim* s) {
    if (!s) return;
    free(s->x); free(s->r); free(s->v); free(s->w); free(s->inv_m); free(s->inv_I);
    free(s->id); free(s->g); free(s->c); free(s->ws); free(s->gforce); free(s->gimp); free(s->gbody);
    free(s);
}

void orc_get_state(const orc_sim* s, double* x, double* v, double* w) {
    if (x) memcpy(x, s->x, 3 * (size_t)s->n * sizeof(double));
    if (v) memcpy(v, s->v, 3 * (size_t)s->n * sizeof(double));
    if (w) memcpy(w, s->w, 3 * (size_t)s->n * sizeof(double));
}
void orc_set_state(orc_sim* s, const double* x, const double* v, const double* w) {
    if (x) memcpy(s->x, x, 3 * (size_t)s->n * sizeof(double));
    if (v) memcpy(s->v, v, 3 * (size_t)s->n * sizeof(double));
    if (w) memcpy(s->w, w, 3 * (size_t)s->n * sizeof(double));
}
void orc_set_geom_velocity(orc_sim* s, int32_t g, const double v[3], const double w[3]) {
    const int32_t q = s->gbody[g];
    if (q < 0) {
        for (int k = 0; k < 3; ++k) { s->g[g].v[k] = v[k]; s->g[g].w[k] = w[k]; }
        return;
    }
    /* a group member: the prescribed axes of the whole group */
    for (int k = 0; k < 3; ++k)
        if (!(s->grp[q].dof >> k & 1)) s->grp[q].v[k] = v[k];
    for (int32_t m = 0; m < s->ng; ++m)
        if (s->gbody[m] == q)
            for (int k = 0; k < 3; ++k) { s->g[m].v[k] = s->grp[q].v[k]; s->g[m].w[k] = w[k]; }
}
void orc_get_geom(const orc_sim* s, int32_t g, orc_geom* out) { *out = s->g[g]; }
void orc_get_geom_force(const orc_sim* s, int32_t g, double f[3], double t[3]) {
    for (int k = 0; k < 3; ++k) { f[k] = s->gforce[6 * g + k]; t[k] = s->gforce[6 * g + 3 + k]; }
}

/* tangent basis: Gram-Schmidt of the world axis least aligned with n */
static void tangent_basis(const double* n, double* t1, double* t2) {
    double e[3] = {0, 0, 0};
    double ax = fabs(n[0]), ay = fabs(n[1]), az = fabs(n[2]);
    if (ax <= ay && ax <= az) e[0] = 1; else if (ay <= az) e[1] = 1; else e[2] = 1;
    double d = dot3(e, n);
    for (int k = 0; k < 3; ++k) t1[k] = e[k] - d * n[k];
    double l = norm3(t1);
    for (int k = 0; k < 3; ++k) t1[k] /= l;
    cross3(n, t1, t2);
}

/* One Jacobian row pair for a body with contact arm l: linear part dir,
 * angular part (l x dir), so that row . (v, w) = dir . (v + w x l). */
static void row_lin(double* row, const double* dir, const double* l, double sign) {
    double lc[3];
    cross3(l, dir, lc);
    for (int k = 0; k < 3; ++k) { row[k] = sign * dir[k]; row[3 + k] = sign * lc[k]; }
}

static void inv2(double A[2][2], double out[2][2]) {
    double det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    out[0][0] = A[1][1] / det; out[1][1] = A[0][0] / det;
    out[0][1] = -A[0][1] / det; out[1][0] = -A[1][0] / det;
}
static void inv3(double A[3][3], double o[3][3]) {
    double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    double c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
    double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    double det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
    o[0][0] = c00 / det;
    o[1][0] = c01 / det;
    o[2][0] = c02 / det;
    o[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
    o[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
    o[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
    o[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
    o[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
    o[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
}

static int cmp_ws(const void* p, const void* q) {
    const ws_entry* x = (const ws_entry*)p;
    const ws_entry* y = (const ws_entry*)q;
    if (x->ka != y->ka) return x->ka < y->ka ? -1 : 1;
    if (x->kb != y->kb) return x->kb < y->kb ? -1 : 1;
    return 0;
}

static const ws_entry* ws_find(const orc_sim* s, int32_t ka, int32_t kb) {
    int64_t lo = 0, hi = s->nws - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        const ws_entry* e = &s->ws[mid];
        if (e->ka == ka && e->kb == kb) return e;
        if (e->ka < ka || (e->ka == ka && e->kb < kb)) lo = mid + 1; else hi = mid - 1;
    }
    return NULL;
}

void orc_set_warmstart(orc_sim* s, int64_t m, const int32_t* key_a, const int32_t* key_b,
                       const double* lam7) {
    free(s->ws);
    s->ws = (ws_entry*)calloc(m ? (size_t)m : 1, sizeof(ws_entry));
    s->nws = m;
    for (int64_t k = 0; k < m; ++k) {
        s->ws[k].ka = key_a[k];
        s->ws[k].kb = key_b[k];
        memcpy(s->ws[k].lam7, &lam7[7 * k], 7 * sizeof(double));
    }
    if (m > 1) qsort(s->ws, (size_t)m, sizeof(ws_entry), cmp_ws);
}

/* world-frame impulses of a contact on body a: (p_n, p_t, p_r) */
static void contact_world(const contact* c, double* lam7) {
    lam7[0] = c->lam[0];
    for (int k = 0; k < 3; ++k) {
        lam7[1 + k] = c->lam[1] * c->t1[k] + c->lam[2] * c->t2[k];
        lam7[4 + k] = c->lam[3 + k];
    }
}

/* G^T lambda for one side of the contact, added into acc (6) */
static void add_GT(double G[6][6], const double* lam, double* acc) {
    for (int col = 0; col < 6; ++col) {
        double s = 0.0;
        for (int row = 0; row < 6; ++row) s += G[row][col] * lam[row];
        acc[col] += s;
    }
}

/* ------------------------------------------------------------------------- */
/* one SPOOK step                                                             */
/* ------------------------------------------------------------------------- */
/* One projected update of contact c (Eqs. 5-7) from the body velocities
 * (vv, ww) and, for a load-driven group's primitive, the group velocity vg. */
static void project_contact(const contact* c, const double* vv, const double* ww, const double* vg,
                            double* out) {
    double wres[6];
    for (int row = 0; row < 6; ++row) {
        double gv = dot3(c->Ga[row], &vv[3 * c->a]) + dot3(&c->Ga[row][3], &ww[3 * c->a]);
        if (c->b >= 0) gv += dot3(c->Gb[row], &vv[3 * c->b]) + dot3(&c->Gb[row][3], &ww[3 * c->b]);
        else if (vg) gv += dot3(c->Gb[row], vg) + c->known_ang[row];
        else gv += c->known[row];
        wres[row] = gv + c->sig[row] * c->lam[row] - c->rhs[row];
    }
    /* normal: 0 <= lambda_n (Eq. 5) */
    double ln = c->lam[0] - c->Dn_inv * wres[0];
    if (ln < 0.0) ln = 0.0;
    /* tangential: Coulomb disc |lambda_t| <= mu_t lambda_n (Eq. 6) */
    double lt[2];
    for (int i = 0; i < 2; ++i) lt[i] = c->lam[1 + i] - (c->Dt_inv[i][0] * wres[1] + c->Dt_inv[i][1] * wres[2]);
    double ltn = sqrt(lt[0] * lt[0] + lt[1] * lt[1]);
    double bt = c->mu_t * ln;
    if (ltn > bt) { lt[0] *= bt / ltn; lt[1] *= bt / ltn; }
    /* rolling: ball |lambda_r| <= mu_r r lambda_n (Eq. 7) */
    double lr[3];
    for (int i = 0; i < 3; ++i)
        lr[i] = c->lam[3 + i] - (c->Dr_inv[i][0] * wres[3] + c->Dr_inv[i][1] * wres[4] + c->Dr_inv[i][2] * wres[5]);
    double lrn = sqrt(lr[0] * lr[0] + lr[1] * lr[1] + lr[2] * lr[2]);
    double br = c->mu_r_reff * ln;
    if (lrn > br) { for (int i = 0; i < 3; ++i) lr[i] *= br / lrn; }
    out[0] = ln;
    out[1] = lt[0]; out[2] = lt[1];
    out[3] = lr[0]; out[4] = lr[1]; out[5] = lr[2];
}

/* SplitMix64 finaliser (Steele, Lea and Flood 2014; Vigna): the priority of a
 * contact is the mix of its key (stable id of a, stable id of b or -(g+1)). */
static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static uint64_t contact_key(const contact* c) { return ((uint64_t)(uint32_t)c->ka << 32) | (uint32_t)c->kb; }

/* higher priority first; equal mixes (not expected) by key */
static int before(const contact* x, const contact* y) {
    const uint64_t kx = contact_key(x), ky = contact_key(y);
    const uint64_t px = mix64(kx), py = mix64(ky);
    return px != py ? px > py : kx < ky;
}

static const contact* g_sort_base;
static int cmp_priority(const void* pa, const void* pb) {
    const contact* x = &g_sort_base[*(const int64_t*)pa];
    const contact* y = &g_sort_base[*(const int64_t*)pb];
    return before(x, y) ? -1 : (before(y, x) ? 1 : 0);
}

/* Newton impact stage (Sec. 2.2: high-velocity impacts follow Newton's impact
 * law while every other kinematic constraint is kept).  A contact whose normal
 * velocity at the start of the step u- = G_n v is below -v_imp is an impact.
 * When the step has one, normal impulses p >= 0 of every contact are solved
 * on the velocity level,
 *     u+ + e_c min(u-, 0) >= 0   complementary to   p >= 0,
 *     u+ = G_n v+,  v+ = v + M^-1 G_n^T p,
 * with e_c = e_imp for impacts and 0 for the other contacts (no approach), by
 * N_it projected Jacobi sweeps with the masses split over each body's contacts
 * (as the main solve), from p = 0; primitives keep their velocities.  The
 * post-impact velocities then start the SPOOK step. */
static void impact_stage(orc_sim* s, const int32_t* cnt, const int64_t* start, const int64_t* inc) {
    const orc_params* P = &s->p;
    const int32_t n = s->n;
    const int64_t nc = s->nc;
    s->nimp = 0;
    memset(s->gimp, 0, 6 * (size_t)(s->ng ? s->ng : 1) * sizeof(double));
    if (!(P->v_imp > 0.0) || nc == 0) return;
    double* u0 = (double*)malloc((size_t)nc * sizeof(double));
    double* tgt = (double*)malloc((size_t)nc * sizeof(double));
    double* Dinv = (double*)malloc((size_t)nc * sizeof(double));
    double* p = (double*)calloc((size_t)nc, sizeof(double));
    double* pn = (double*)calloc((size_t)nc, sizeof(double));
    for (int64_t k = 0; k < nc; ++k) {
        const contact* c = &s->c[k];
        double u = dot3(c->Ga[0], &s->v[3 * c->a]) + dot3(&c->Ga[0][3], &s->w[3 * c->a]);
        if (c->b >= 0) u += dot3(c->Gb[0], &s->v[3 * c->b]) + dot3(&c->Gb[0][3], &s->w[3 * c->b]);
        else u += c->known[0];
        u0[k] = u;
        const int hit = u < -P->v_imp;
        tgt[k] = hit ? P->e_imp * u : 0.0;
        s->nimp += hit;
        /* D = G_n M_split^-1 G_n^T, primitives kinematic */
        const double ima = cnt[c->a] * s->inv_m[c->a], iIa = cnt[c->a] * s->inv_I[c->a];
        double D = 0.0;
        for (int q = 0; q < 3; ++q) D += c->Ga[0][q] * c->Ga[0][q] * ima + c->Ga[0][3 + q] * c->Ga[0][3 + q] * iIa;
        if (c->b >= 0) {
            const double imb = cnt[c->b] * s->inv_m[c->b], iIb = cnt[c->b] * s->inv_I[c->b];
            for (int q = 0; q < 3; ++q)
                D += c->Gb[0][q] * c->Gb[0][q] * imb + c->Gb[0][3 + q] * c->Gb[0][3 + q] * iIb;
        }
        Dinv[k] = 1.0 / D;
    }
    if (s->nimp == 0) {
        free(u0); free(tgt); free(Dinv); free(p); free(pn);
        return;
    }
    double* v0 = (double*)malloc(3 * (size_t)n * sizeof(double));
    double* w0 = (double*)malloc(3 * (size_t)n * sizeof(double));
    memcpy(v0, s->v, 3 * (size_t)n * sizeof(double));
    memcpy(w0, s->w, 3 * (size_t)n * sizeof(double));
    for (int32_t it = 0; it < P->n_it; ++it) {
        /* every contact from the bodies' current iterate */
        for (int64_t k = 0; k < nc; ++k) {
            const contact* c = &s->c[k];
            double u = dot3(c->Ga[0], &s->v[3 * c->a]) + dot3(&c->Ga[0][3], &s->w[3 * c->a]);
            if (c->b >= 0) u += dot3(c->Gb[0], &s->v[3 * c->b]) + dot3(&c->Gb[0][3], &s->w[3 * c->b]);
            else u += c->known[0];
            const double q = p[k] - Dinv[k] * (u + tgt[k]);
            pn[k] = q > 0.0 ? q : 0.0;
        }
        memcpy(p, pn, (size_t)nc * sizeof(double));
        /* every body: v+ = v + M^-1 sum_c G_n^T p_c, in contact order */
        for (int32_t i = 0; i < n; ++i) {
            double acc[6] = {0, 0, 0, 0, 0, 0};
            for (int64_t e = start[i]; e < start[i + 1]; ++e) {
                const contact* c = &s->c[inc[e] / 2];
                const double* row = (inc[e] & 1) ? c->Gb[0] : c->Ga[0];
                for (int q = 0; q < 6; ++q) acc[q] += row[q] * p[inc[e] / 2];
            }
            for (int q = 0; q < 3; ++q) {
                s->v[3 * i + q] = v0[3 * i + q] + s->inv_m[i] * acc[q];
                s->w[3 * i + q] = w0[3 * i + q] + s->inv_I[i] * acc[3 + q];
            }
        }
    }
    /* the impulse the primitives received */
    for (int64_t k = 0; k < nc; ++k) {
        const contact* c = &s->c[k];
        if (c->b >= 0) continue;
        for (int q = 0; q < 6; ++q) s->gimp[6 * (-c->b - 1) + q] += c->Gb[0][q] * p[k];
    }
    free(u0); free(tgt); free(Dinv); free(p); free(pn); free(v0); free(w0);
}

static void step_once(orc_sim* s) {
    const orc_params* P = &s->p;
    const double h = P->dt;
    const int32_t n = s->n;

    /* 1. contact detection at x_i (Sec. 2.2) */
    raw_vec raw = detect_all(n, s->x, s->r, s->id, s->ng, s->g);
    free(s->c);
    s->nc = raw.n;
    s->c = (contact*)calloc(raw.n ? (size_t)raw.n : 1, sizeof(contact));

    /* contacts per body, for the split masses m_b / n_b */
    int32_t* cnt = (int32_t*)calloc(n ? n : 1, sizeof(int32_t));
    for (int64_t k = 0; k < raw.n; ++k) {
        cnt[raw.v[k].a]++;
        if (raw.v[k].b >= 0) cnt[raw.v[k].b]++;
    }

    /* contacts per load-driven group: its split mass M / n_q */
    int32_t ncg[ORC_MAX_GROUPS] = {0};
    for (int64_t k = 0; k < raw.n; ++k)
        if (raw.v[k].b < 0 && s->gbody[-raw.v[k].b - 1] >= 0) ncg[s->gbody[-raw.v[k].b - 1]]++;

    /* SPOOK constants (Lacoursiere 2007), d = tau/dt */
    const double Ups = 1.0 / (1.0 + 4.0 * P->damp_steps);

    /* 2. contact rows */
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < raw.n; ++k) {
        contact* c = &s->c[k];
        const raw_contact* rc = &raw.v[k];
        c->a = rc->a; c->b = rc->b; c->ka = rc->ka; c->kb = rc->kb;
        const int a = c->a;
        const double* xa = &s->x[3 * a];
        const double ra = s->r[a];
        double Estar, dstar, reff, mu_t, mu_r;
        double vb_lin[3] = {0, 0, 0}, vb_ang[3] = {0, 0, 0};
        const orc_geom* geo = NULL;
        if (c->b >= 0) {
            const int b = c->b;
            const double* xb = &s->x[3 * b];
            const double rb = s->r[b];
            double d[3] = {xa[0] - xb[0], xa[1] - xb[1], xa[2] - xb[2]};
            double dist = norm3(d);
            c->delta = rc->delta;
            /* both arms end at the middle of the overlap, so the pair's
             * impulses have no net moment about any point */
            for (int q = 0; q < 3; ++q) {
                c->n[q] = d[q] / dist;
                c->la[q] = -(ra - 0.5 * c->delta) * c->n[q];
                c->lb[q] = (rb - 0.5 * c->delta) * c->n[q];
            }
            /* effective modulus and diameter of the pair (Sec. 2.2) */
            Estar = 1.0 / ((1.0 - P->nu * P->nu) / P->E + (1.0 - P->nu * P->nu) / P->E);
            dstar = 1.0 / (1.0 / (2.0 * ra) + 1.0 / (2.0 * rb));
            reff = 2.0 * ra * rb / (ra + rb);
            mu_t = P->mu_t; mu_r = P->mu_r;
        } else {
            geo = &s->g[-c->b - 1];
            geo_hit hh = sphere_geom(geo, xa, ra);
            c->delta = hh.delta;
            for (int q = 0; q < 3; ++q) {
                c->n[q] = hh.n[q];
                c->la[q] = -(ra - 0.5 * c->delta) * c->n[q];
                /* lever from the primitive's centre to the middle of the
                 * overlap, where the sphere's arm ends too: half the overlap
                 * below the surface point q (n points out of the primitive) */
                c->lb[q] = (hh.q[q] - 0.5 * c->delta * c->n[q]) - geo->c[q];
                vb_lin[q] = geo->v[q];
                vb_ang[q] = geo->w[q];
            }
            Estar = 1.0 / ((1.0 - P->nu * P->nu) / P->E + (1.0 - geo->nu * geo->nu) / geo->E);
            dstar = 2.0 * ra; /* flat geometry: d_b -> infinity */
            reff = ra;
            mu_t = geo->mu_t; mu_r = geo->mu_r;
        }
        tangent_basis(c->n, c->t1, c->t2);
        const double* dirs[3] = {c->n, c->t1, c->t2};
        for (int rrow = 0; rrow < 3; ++rrow) {
            row_lin(c->Ga[rrow], dirs[rrow], c->la, 1.0);
            row_lin(c->Gb[rrow], dirs[rrow], c->lb, -1.0);
        }
        for (int q = 0; q < 3; ++q) {
            for (int col = 0; col < 6; ++col) { c->Ga[3 + q][col] = 0.0; c->Gb[3 + q][col] = 0.0; }
            c->Ga[3 + q][3 + q] = 1.0;
            c->Gb[3 + q][3 + q] = -1.0;
        }
        c->grp = geo ? s->gbody[-c->b - 1] : -1;
        if (geo) {
            for (int rrow = 0; rrow < 6; ++rrow) {
                c->known_ang[rrow] = dot3(&c->Gb[rrow][3], vb_ang);
                c->known[rrow] = dot3(c->Gb[rrow], vb_lin) + c->known_ang[rrow];
            }
        }
        /* Hertz mapping: g = -delta^{e_H}, eps = e_H / k_n, k_n = E* sqrt(d*)/3.
         * The row is written for the physical normal impulse: the Hertz
         * Jacobian factor J = e_H delta^{e_H-1} is divided out of the row. */
        const double kn = P->kn_scale * Estar * sqrt(dstar) / 3.0;
        const double eps_n = P->e_H / kn;
        const double dfl = c->delta > P->delta_floor ? c->delta : P->delta_floor;
        const double J = P->e_H * pow(dfl, P->e_H - 1.0);
        const double gap = -pow(c->delta, P->e_H);
        const double Sig_scaled = 4.0 * eps_n * Ups / (h * h);
        c->sig[0] = Sig_scaled / (J * J);
        /* the gap part of the right side; + Ups G_n v after the impact stage */
        c->rhs[0] = (-(4.0 / h) * Ups * gap) / J;
        for (int q = 1; q < 6; ++q) { c->sig[q] = P->eps_reg * c->sig[0]; c->rhs[q] = 0.0; }
        c->mu_t = mu_t;
        c->mu_r_reff = mu_r * reff;

        /* block diagonal of G Msplit^-1 G^T + Sigma */
        double D[6][6];
        /* Jacobi splits each body's mass over its contacts (m / n_b); Gauss-Seidel
         * updates bodies between contacts and uses the masses themselves */
        const double spa = P->solver == ORC_PGS ? 1.0 : cnt[a];
        const double spb = c->b >= 0 ? (P->solver == ORC_PGS ? 1.0 : cnt[c->b]) : 0.0;
        const double ima = spa * s->inv_m[a], iIa = spa * s->inv_I[a];
        const double imb = c->b >= 0 ? spb * s->inv_m[c->b] : 0.0;
        const double iIb = c->b >= 0 ? spb * s->inv_I[c->b] : 0.0;
        /* inverse (split) mass of side b per axis: a particle's, a load-driven
         * group's along its dynamic axes, zero for kinematic geometry */
        double imb3[3] = {imb, imb, imb};
        if (c->grp >= 0)
            for (int q = 0; q < 3; ++q)
                imb3[q] = (s->grp[c->grp].dof >> q & 1) ? ncg[c->grp] / s->grp[c->grp].mass : 0.0;
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                double acc = 0.0;
                for (int q = 0; q < 3; ++q) {
                    acc += c->Ga[i][q] * c->Ga[j][q] * ima + c->Ga[i][3 + q] * c->Ga[j][3 + q] * iIa;
                    acc += c->Gb[i][q] * c->Gb[j][q] * imb3[q] + c->Gb[i][3 + q] * c->Gb[j][3 + q] * iIb;
                }
                D[i][j] = acc + (i == j ? c->sig[i] : 0.0);
            }
        c->Dn_inv = 1.0 / D[0][0];
        double Dt[2][2] = {{D[1][1], D[1][2]}, {D[2][1], D[2][2]}};
        inv2(Dt, c->Dt_inv);
        double Dr[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Dr[i][j] = D[3 + i][3 + j];
        inv3(Dr, c->Dr_inv);

        /* warm start: previous impulses of the same key, the tangential part
         * projected onto the new tangent plane */
        const ws_entry* e = ws_find(s, c->ka, c->kb);
        if (e) {
            c->lam[0] = e->lam7[0];
            c->lam[1] = dot3(&e->lam7[1], c->t1);
            c->lam[2] = dot3(&e->lam7[1], c->t2);
            c->lam[3] = e->lam7[4]; c->lam[4] = e->lam7[5]; c->lam[5] = e->lam7[6];
        } else {
            for (int q = 0; q < 6; ++q) c->lam[q] = 0.0;
        }
    }
    free(raw.v);

    /* incidence lists in contact order */
    int64_t* start = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    for (int32_t i = 0; i < n; ++i) start[i + 1] = start[i] + cnt[i];
    int64_t* inc = (int64_t*)malloc((size_t)(start[n] ? start[n] : 1) * sizeof(int64_t));
    int64_t* fill = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t k = 0; k < s->nc; ++k) {
        int a = s->c[k].a, b = s->c[k].b;
        inc[start[a] + fill[a]++] = 2 * k;          /* side a */
        if (b >= 0) inc[start[b] + fill[b]++] = 2 * k + 1; /* side b */
    }

    /* 2b. Newton impact stage, then the velocity part of the right side:
     * b_n = -(4/dt) Ups g / J + Ups G_n v with v the (post-impact) velocity at
     * the start of the step */
    impact_stage(s, cnt, start, inc);
    for (int64_t k = 0; k < s->nc; ++k) {
        contact* c = &s->c[k];
        double Gv = dot3(c->Ga[0], &s->v[3 * c->a]) + dot3(&c->Ga[0][3], &s->w[3 * c->a]);
        if (c->b >= 0) Gv += dot3(c->Gb[0], &s->v[3 * c->b]) + dot3(&c->Gb[0][3], &s->w[3 * c->b]);
        else Gv += c->known[0];
        c->rhs[0] = c->rhs[0] + Ups * Gv;
    }

    /* free velocity v* = v + dt M^-1 f_ext (gravity only) */
    double* vs = (double*)malloc(3 * (size_t)(n ? n : 1) * sizeof(double));
    double* vv = (double*)malloc(3 * (size_t)(n ? n : 1) * sizeof(double));
    double* ww = (double*)malloc(3 * (size_t)(n ? n : 1) * sizeof(double));
    for (int32_t i = 0; i < n; ++i)
        for (int q = 0; q < 3; ++q) vs[3 * i + q] = s->v[3 * i + q] + (s->inv_m[i] > 0.0 ? h * P->gravity[q] : 0.0);

    /* load-driven groups: free velocity v_q* = v_q + dt F / M along the dynamic
     * axes, current iterate vg */
    double vgs[ORC_MAX_GROUPS][3], vg[ORC_MAX_GROUPS][3];
    for (int32_t q = 0; q < s->ngrp; ++q)
        for (int a = 0; a < 3; ++a) {
            const int dyn = s->grp[q].dof >> a & 1;
            vgs[q][a] = s->grp[q].v[a] + (dyn ? h * s->grp[q].force[a] / s->grp[q].mass : 0.0);
            vg[q][a] = vgs[q][a];
        }
    /* v_q = v_q* + M^-1 sum over the group's contacts of the linear part of
     * G_b^T lambda, along the dynamic axes; summed in contact order */
    #define GROUP_UPDATE()                                                         \
    for (int32_t q = 0; q < s->ngrp; ++q) {                                        \
        double accg[3] = {0, 0, 0};                                                \
        for (int64_t k = 0; k < s->nc; ++k) {                                      \
            const contact* c = &s->c[k];                                           \
            if (c->grp != q) continue;                                             \
            double tmp[6] = {0, 0, 0, 0, 0, 0};                                    \
            add_GT((double(*)[6])c->Gb, c->lam, tmp);                              \
            for (int a = 0; a < 3; ++a) accg[a] += tmp[a];                         \
        }                                                                          \
        for (int a = 0; a < 3; ++a)                                                \
            vg[q][a] = vgs[q][a] + ((s->grp[q].dof >> a & 1) ? accg[a] / s->grp[q].mass : 0.0); \
    }

    /* v = v* + M^-1 sum_c G_c^T lambda_c */
    #define BODY_UPDATE()                                                          \
    _Pragma("omp parallel for schedule(static)")                                   \
    for (int32_t i = 0; i < n; ++i) {                                              \
        double acc[6] = {0, 0, 0, 0, 0, 0};                                        \
        for (int64_t e = start[i]; e < start[i + 1]; ++e) {                       \
            const contact* c = &s->c[inc[e] / 2];                                  \
            add_GT((double(*)[6])((inc[e] & 1) ? c->Gb : c->Ga), c->lam, acc);     \
        }                                                                          \
        for (int q = 0; q < 3; ++q) {                                              \
            vv[3 * i + q] = vs[3 * i + q] + s->inv_m[i] * acc[q];                  \
            ww[3 * i + q] = s->w[3 * i + q] + s->inv_I[i] * acc[3 + q];            \
        }                                                                          \
    }
    BODY_UPDATE();
    GROUP_UPDATE();

    /* 3. N_it projected sweeps */
    s->ncol = 0;
    if (P->solver == ORC_PGS) {
        /* Colours: contacts that share a body never share a colour.  Greedy in
         * priority order, each contact taking the smallest colour that none of
         * its already coloured neighbours has. */
        int32_t* col = (int32_t*)malloc((size_t)(s->nc ? s->nc : 1) * sizeof(int32_t));
        int64_t* order = (int64_t*)malloc((size_t)(s->nc ? s->nc : 1) * sizeof(int64_t));
        for (int64_t k = 0; k < s->nc; ++k) { col[k] = -1; order[k] = k; }
        g_sort_base = s->c;
        qsort(order, (size_t)s->nc, sizeof(int64_t), cmp_priority);
        int32_t ncol = 0;
        for (int64_t q = 0; q < s->nc; ++q) {
            const int64_t k = order[q];
            const contact* c = &s->c[k];
            unsigned char used[256];
            memset(used, 0, sizeof used);
            const int bodies[2] = {c->a, c->b};
            for (int e2 = 0; e2 < 2; ++e2) {
                const int body = bodies[e2];
                if (body < 0) continue;
                for (int64_t e = start[body]; e < start[body + 1]; ++e) {
                    const int64_t m = inc[e] / 2;
                    if (m != k && col[m] >= 0 && col[m] < 256) used[col[m]] = 1;
                }
            }
            int32_t cc = 0;
            while (cc < 255 && used[cc]) ++cc;
            col[k] = cc;
            if (cc + 1 > ncol) ncol = cc + 1;
        }
        s->ncol = ncol;
        /* sweeps: colour by colour, each contact's impulse change applied to
         * its bodies at once (no two contacts of a colour share a body) */
        for (int32_t it = 0; it < P->n_it; ++it)
            for (int32_t cc = 0; cc < ncol; ++cc)
                for (int64_t k = 0; k < s->nc; ++k) {
                    if (col[k] != cc) continue;
                    contact* c = &s->c[k];
                    double nl[6], d[6], acc[6];
                    project_contact(c, vv, ww, NULL, nl);
                    for (int q = 0; q < 6; ++q) d[q] = nl[q] - c->lam[q];
                    memset(acc, 0, sizeof acc);
                    add_GT(c->Ga, d, acc);
                    for (int q = 0; q < 3; ++q) {
                        vv[3 * c->a + q] += s->inv_m[c->a] * acc[q];
                        ww[3 * c->a + q] += s->inv_I[c->a] * acc[3 + q];
                    }
                    if (c->b >= 0) {
                        memset(acc, 0, sizeof acc);
                        add_GT(c->Gb, d, acc);
                        for (int q = 0; q < 3; ++q) {
                            vv[3 * c->b + q] += s->inv_m[c->b] * acc[q];
                            ww[3 * c->b + q] += s->inv_I[c->b] * acc[3 + q];
                        }
                    }
                    memcpy(c->lam, nl, sizeof nl);
                }
        free(col);
        free(order);
    } else {
        for (int32_t it = 0; it < P->n_it; ++it) {
#pragma omp parallel for schedule(static)
            for (int64_t k = 0; k < s->nc; ++k) {
                contact* c = &s->c[k];
                project_contact(c, vv, ww, c->grp >= 0 ? vg[c->grp] : NULL, c->lam_new);
            }
            for (int64_t k = 0; k < s->nc; ++k) memcpy(s->c[k].lam, s->c[k].lam_new, 6 * sizeof(double));
            BODY_UPDATE();
            GROUP_UPDATE();
        }
    }
    #undef BODY_UPDATE
    #undef GROUP_UPDATE
    /* the groups' new velocities move their primitives */
    for (int32_t q = 0; q < s->ngrp; ++q)
        for (int a = 0; a < 3; ++a) s->grp[q].v[a] = vg[q][a];
    for (int32_t gi = 0; gi < s->ng; ++gi)
        if (s->gbody[gi] >= 0)
            for (int a = 0; a < 3; ++a) s->g[gi].v[a] = vg[s->gbody[gi]][a];

    /* 4. SPOOK position update with the new velocity */
    for (int32_t i = 0; i < n; ++i)
        for (int q = 0; q < 3; ++q) {
            s->v[3 * i + q] = vv[3 * i + q];
            s->w[3 * i + q] = ww[3 * i + q];
            s->x[3 * i + q] += h * s->v[3 * i + q];
        }

    /* geometry force and torque about its centre: G_b^T lambda / dt */
    memset(s->gforce, 0, 6 * (size_t)(s->ng ? s->ng : 1) * sizeof(double));
    for (int64_t k = 0; k < s->nc; ++k) {
        contact* c = &s->c[k];
        if (c->b >= 0) continue;
        add_GT(c->Gb, c->lam, &s->gforce[6 * (-c->b - 1)]);
    }
    /* the impact stage's impulse on the geometry belongs to the same step */
    for (int32_t gi = 0; gi < 6 * s->ng; ++gi) s->gforce[gi] = (s->gforce[gi] + s->gimp[gi]) / h;

    /* kinematic geometry: translate with v, rotate with w (Rodrigues) */
    for (int32_t gi = 0; gi < s->ng; ++gi) {
        orc_geom* g = &s->g[gi];
        for (int q = 0; q < 3; ++q) g->c[q] += h * g->v[q];
        double wn = norm3(g->w);
        if (wn > 0.0) {
            double ax[3] = {g->w[0] / wn, g->w[1] / wn, g->w[2] / wn};
            double th = wn * h, cs = cos(th), sn = sin(th);
            double Rot[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) Rot[i][j] = (i == j ? cs : 0.0) + (1.0 - cs) * ax[i] * ax[j];
            Rot[0][1] -= sn * ax[2]; Rot[0][2] += sn * ax[1];
            Rot[1][0] += sn * ax[2]; Rot[1][2] -= sn * ax[0];
            Rot[2][0] -= sn * ax[1]; Rot[2][1] += sn * ax[0];
            double Rn[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    Rn[3 * i + j] = Rot[i][0] * g->R[0 * 3 + j] + Rot[i][1] * g->R[1 * 3 + j] + Rot[i][2] * g->R[2 * 3 + j];
            memcpy(g->R, Rn, sizeof Rn);
        }
    }

    /* warm-start store for the next step */
    free(s->ws);
    s->ws = (ws_entry*)calloc(s->nc ? (size_t)s->nc : 1, sizeof(ws_entry));
    s->nws = s->nc;
    for (int64_t k = 0; k < s->nc; ++k) {
        s->ws[k].ka = s->c[k].ka;
        s->ws[k].kb = s->c[k].kb;
        contact_world(&s->c[k], s->ws[k].lam7);
    }

    free(cnt); free(start); free(inc); free(fill); free(vs); free(vv); free(ww);
}

int32_t orc_colours(const orc_sim* s) { return s->ncol; }
int64_t orc_impacts(const orc_sim* s) { return s->nimp; }

int orc_step(orc_sim* s, int32_t nsteps) {
    if (s->p.solver == ORC_PGS && s->ngrp > 0) return -1;
    for (int32_t k = 0; k < nsteps; ++k) step_once(s);
    return 0;
}

int64_t orc_get_contacts(const orc_sim* s, int64_t cap, int32_t* key_a, int32_t* key_b,
                         double* lam7, double* delta, double* normal) {
    for (int64_t k = 0; k < s->nc && k < cap; ++k) {
        const contact* c = &s->c[k];
        if (key_a) key_a[k] = c->ka;
        if (key_b) key_b[k] = c->kb;
        if (lam7) contact_world(c, &lam7[7 * k]);
        if (delta) delta[k] = c->delta;
        if (normal) for (int q = 0; q < 3; ++q) normal[3 * k + q] = c->n[q];
    }
    return s->nc;
}
