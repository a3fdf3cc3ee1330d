// C ABI of the DEM library (include/dem.h): bed creation, the per-step graph
// of kernels, read-back and error reporting.
//
// One step (Sec. 2.2) is captured once per step parity into CUDA graphs:
//   pre:  cell lists -> contacts -> incidence -> SPOOK rows + warm start -> v^0
//   jac:  N_it projected Jacobi sweeps
//   post: integration, geometry forces, kinematic geometry
// A Morton re-sort graph runs before every `resort_every`-th step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "bed.cuh"

static thread_local std::string g_err;

static dem_status fail(dem_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

dem_status dem_fail(dem_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(DEM_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                             \
    } while (0)




// ---------------------------------------------------------------------------
// memory
// ---------------------------------------------------------------------------
static dem_status dalloc(dem_bed* b, void** p, size_t bytes) {
    bytes = std::max<size_t>(bytes, 256);
    bytes = (bytes + 255) & ~(size_t)255;
    if (b->alloc) {
        *p = b->alloc(bytes, b->actx, (void*)b->stream);
        if (!*p) return fail(DEM_ERR_CUDA, "allocator callback returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMallocAsync(p, bytes, b->stream);
        if (e != cudaSuccess)
            return fail(DEM_ERR_CUDA, "cudaMallocAsync(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    b->allocs.push_back(*p);
    // kernels move 16- and 32-byte records with vector loads and stores
    if ((uintptr_t)*p & 255) return fail(DEM_ERR_CUDA, "device allocation %p is not 256-byte aligned", *p);
    return DEM_OK;
}

dem_status dem_dalloc(dem_bed* b, void** p, size_t bytes) { return dalloc(b, p, bytes); }

void dem_dfree(dem_bed* b, void* p) {
    if (!p) return;
    for (size_t k = 0; k < b->allocs.size(); ++k)
        if (b->allocs[k] == p) {
            b->allocs[k] = b->allocs.back();
            b->allocs.pop_back();
            break;
        }
    if (b->freef) b->freef(p, b->actx, (void*)b->stream);
    else cudaFreeAsync(p, b->stream);
}

template <typename T>
static dem_status dalloc_n(dem_bed* b, T** p, size_t count) {
    return dalloc(b, (void**)p, count * sizeof(T));
}

static void release(dem_bed* b) {
    if (!b) return;
    cudaSetDevice(b->dev);
    cudaStreamSynchronize(b->stream);
    for (int p = 0; p < 2; ++p)
        for (int k = 0; k < 3; ++k)
            if (b->g[p][k]) cudaGraphExecDestroy(b->g[p][k]);
    if (b->g_resort) cudaGraphExecDestroy(b->g_resort);
    if (b->side) cudaStreamDestroy(b->side);
    dem_adjoint_release(b);
    for (cudaEvent_t e : b->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : b->ev_used) cudaEventDestroy(e);
    for (void* p : b->allocs) {
        if (b->freef) b->freef(p, b->actx, (void*)b->stream);
        else cudaFreeAsync(p, b->stream);
    }
    cudaStreamSynchronize(b->stream);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

// ---------------------------------------------------------------------------
// creation
// ---------------------------------------------------------------------------
static double estar(double E1, double nu1, double E2, double nu2) {
    return 1.0 / ((1.0 - nu1 * nu1) / E1 + (1.0 - nu2 * nu2) / E2);
}

static dem_status build_graphs(dem_bed* b);
static dem_status rebuild_graphs(dem_bed* b);

// motor velocity of a load-driven group: the prescribed axes of the group and of
// every member (the dynamic axes keep their solved velocity)
__global__ void k_group_motor(DevBuf B, int ng, int q, double vx, double vy, double vz, double wx, double wy,
                              double wz) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    GroupDev& Q = B.grp[q];
    const double v[3] = {vx, vy, vz}, w[3] = {wx, wy, wz};
    for (int ax = 0; ax < 3; ++ax)
        if (!(Q.dof >> ax & 1)) Q.v[ax] = v[ax];
    for (int g = 0; g < ng; ++g)
        if (B.geom[g].grp == q)
            for (int ax = 0; ax < 3; ++ax) {
                B.geom[g].v[ax] = Q.v[ax];
                B.geom[g].w[ax] = w[ax];
            }
}

// Height of the particle surface under each primitive: the highest top z + r
// of the particles whose centre lies inside the primitive's footprint in x, y
// (all particles if none does).  pos/rad are read with the given strides.
static void surface_refs(int n, const double* pos, int ps, const double* rad, int rs, int ng,
                         const int* type, const double* c, const double* R, const double* he,
                         std::vector<double>& out) {
    out.assign(ng, 0.0);
    double ztop_all = -1e300;
    for (int i = 0; i < n; ++i) ztop_all = std::max(ztop_all, pos[ps * i + 2] + rad[rs * i]);
    for (int g = 0; g < ng; ++g) {
        double zr = -1e300;
        for (int i = 0; i < n; ++i) {
            const double dx = pos[ps * i] - c[3 * g], dy = pos[ps * i + 1] - c[3 * g + 1];
            bool under = false;
            if (type[g] == DEM_GEOM_CYLINDER) {
                under = dx * dx + dy * dy <= he[3 * g] * he[3 * g];
            } else if (type[g] == DEM_GEOM_BOX) {
                double ex = 0, ey = 0;
                for (int k = 0; k < 3; ++k) {
                    ex += std::fabs(R[9 * g + k]) * he[3 * g + k];
                    ey += std::fabs(R[9 * g + 3 + k]) * he[3 * g + k];
                }
                under = std::fabs(dx) <= ex && std::fabs(dy) <= ey;
            }
            if (under) zr = std::max(zr, pos[ps * i + 2] + rad[rs * i]);
        }
        out[g] = zr > -1e299 ? zr : ztop_all;
    }
}

// Shared settings of all beds in one object (one SimParams).
static bool same_settings(const dem_bed_desc& a, const dem_bed_desc& b) {
    return a.E == b.E && a.nu == b.nu && a.mu_t == b.mu_t && a.mu_r == b.mu_r && a.e_H == b.e_H &&
           a.damp_steps == b.damp_steps && a.dt == b.dt && a.gravity[0] == b.gravity[0] &&
           a.gravity[1] == b.gravity[1] && a.gravity[2] == b.gravity[2] && a.kn_scale == b.kn_scale &&
           a.eps_reg == b.eps_reg && a.delta_floor == b.delta_floor && a.restitution == b.restitution &&
           a.impact_speed == b.impact_speed;
}

static dem_status check_desc(const dem_bed_desc* d, int k) {
    if (d->n < 0) return fail(DEM_ERR_ARG, "bed %d: n = %d < 0", k, d->n);
    if (d->n > 0 && (!d->pos || !d->radius)) return fail(DEM_ERR_ARG, "bed %d: pos and radius are required", k);
    if (d->n_geom < 0) return fail(DEM_ERR_ARG, "bed %d: n_geom < 0", k);
    if (d->n_geom > 0 && !d->geom) return fail(DEM_ERR_ARG, "bed %d: geom is NULL", k);
    if (!(d->dt > 0.f)) return fail(DEM_ERR_ARG, "dt must be > 0");
    if (d->n_it < 0) return fail(DEM_ERR_ARG, "bed %d: n_it < 0", k);
    if (!(d->E > 0.f) || !(d->nu > -1.f && d->nu < 0.5f)) return fail(DEM_ERR_ARG, "bad E or nu");
    if (!(d->e_H >= 1.f)) return fail(DEM_ERR_ARG, "e_H must be >= 1");
    if (!(d->rho > 0.f) && !(d->inv_mass && d->inv_inertia)) return fail(DEM_ERR_ARG, "bed %d: rho must be > 0", k);
    if (d->damp_steps < 0.f || d->mu_t < 0.f || d->mu_r < 0.f || d->eps_reg < 0.f)
        return fail(DEM_ERR_ARG, "negative damping, friction or regularisation");
    for (int g = 0; g < d->n_geom; ++g) {
        const dem_geom& G = d->geom[g];
        if (G.type < 0 || G.type > 2) return fail(DEM_ERR_ARG, "bed %d geom %d: bad type %d", k, g, G.type);
        if (!(G.E > 0.f) || G.mu_t < 0.f || G.mu_r < 0.f) return fail(DEM_ERR_ARG, "bed %d geom %d: bad material", k, g);
    }
    return DEM_OK;
}

// One object for one or many beds.  Bed k's particles get the stable ids that
// follow those of beds 0..k-1, its primitives the indices that follow theirs.
// Every bed has its own grid levels (one per radius band), so particles of
// different beds never meet even where the beds overlap in space.
static dem_status create_impl(const dem_bed_desc* descs, int nbeds, void* stream, dem_bed** out) {
    g_err.clear();
    if (!out) return fail(DEM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!descs || nbeds < 1) return fail(DEM_ERR_ARG, "desc is NULL or no beds");
    int64_t n64 = 0, ng64 = 0, cap_sum = 0;
    bool cap_default = false;   // some bed takes the default capacity (then with a pad)
    for (int k = 0; k < nbeds; ++k) {
        dem_status st = check_desc(&descs[k], k);
        if (st != DEM_OK) return st;
        if (!same_settings(descs[0], descs[k]))
            return fail(DEM_ERR_ARG, "bed %d: solver and material settings differ from bed 0", k);
        n64 += descs[k].n;
        ng64 += descs[k].n_geom;
        cap_sum += descs[k].contact_capacity > 0 ? descs[k].contact_capacity : 8LL * descs[k].n;
        cap_default |= descs[k].contact_capacity <= 0;
    }
    if (n64 > (int64_t)0x7fffffff / 8) return fail(DEM_ERR_ARG, "too many particles");
    if (ng64 > DEM_MAX_GEOM) return fail(DEM_ERR_ARG, "%lld primitives exceed %d", (long long)ng64, DEM_MAX_GEOM);
    const dem_bed_desc* d = &descs[0];
    const int n = (int)n64;

    dem_bed* b = new dem_bed();
    cudaGetDevice(&b->dev);
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return fail(DEM_ERR_CUDA, "cudaStreamCreate failed");
        }
        b->own_stream = true;
    }
    b->alloc = d->alloc;
    b->freef = d->free_fn;
    b->actx = d->alloc_ctx;
    if ((b->alloc == nullptr) != (b->freef == nullptr)) {
        release(b);
        return fail(DEM_ERR_ARG, "alloc and free_fn must be given together");
    }
    b->resort_every = d->resort_every > 0 ? d->resort_every : 20;
    b->n_geom = (int)ng64;
    b->geom_group.assign(std::max<int64_t>(ng64, 1), -1);
    b->nbeds = nbeds;

    // host copies of the inputs (they may live on the device)
    std::vector<double> pos(3 * (size_t)n);
    std::vector<float> rad(n), vel(3 * (size_t)n, 0.f), omg(3 * (size_t)n, 0.f), im(n), iI(n);
    std::vector<int> bed_of(n);
    std::vector<dem_geom> geoms;
    std::vector<int> geom_bed;
    auto fetch = [&](void* dst, const void* src, size_t bytes) -> bool {
        return cudaMemcpy(dst, src, bytes, cudaMemcpyDefault) == cudaSuccess;
    };
    {
        size_t o = 0;
        for (int k = 0; k < nbeds; ++k) {
            const dem_bed_desc& dk = descs[k];
            const size_t m = dk.n;
            bool ok = true;
            if (m > 0) {
                ok = fetch(&pos[3 * o], dk.pos, 3 * m * 8) && fetch(&rad[o], dk.radius, m * 4);
                if (dk.vel) ok = ok && fetch(&vel[3 * o], dk.vel, 3 * m * 4);
                if (dk.omega) ok = ok && fetch(&omg[3 * o], dk.omega, 3 * m * 4);
                if (dk.inv_mass) ok = ok && fetch(&im[o], dk.inv_mass, m * 4);
                if (dk.inv_inertia) ok = ok && fetch(&iI[o], dk.inv_inertia, m * 4);
            }
            if (!ok) {
                release(b);
                return fail(DEM_ERR_ARG, "bed %d: could not read the input arrays", k);
            }
            for (size_t i = 0; i < m; ++i) {
                bed_of[o + i] = k;
                if (!(rad[o + i] > 0.f) || !std::isfinite(rad[o + i])) {
                    release(b);
                    return fail(DEM_ERR_ARG, "bed %d: radius[%zu] = %g is not positive", k, i, (double)rad[o + i]);
                }
                for (int q = 0; q < 3; ++q)
                    if (!std::isfinite(pos[3 * (o + i) + q])) {
                        release(b);
                        return fail(DEM_ERR_ARG, "bed %d: pos[%zu] is not finite", k, i);
                    }
                const double r = rad[o + i];
                const double mass = (double)dk.rho * 4.0 / 3.0 * M_PI * r * r * r;
                if (!dk.inv_mass) im[o + i] = (float)(1.0 / mass);
                if (!dk.inv_inertia) iI[o + i] = (float)(1.0 / (0.4 * mass * r * r));
            }
            for (int g = 0; g < dk.n_geom; ++g) {
                geoms.push_back(dk.geom[g]);
                geom_bed.push_back(k);
            }
            o += m;
        }
    }

    SimParams& P = b->P;
    double rmin_all = 1e300, rmax_all = 0.0, absmax = 0.0;
    for (int i = 0; i < n; ++i) {
        rmin_all = std::min(rmin_all, (double)rad[i]);
        rmax_all = std::max(rmax_all, (double)rad[i]);
        for (int q = 0; q < 3; ++q) absmax = std::max(absmax, std::fabs(pos[3 * i + q]));
    }
    if (n == 0) rmin_all = rmax_all = 1e-3;
    // FP32 rounding of the copies: <= 2^-24 |x| per coordinate (margin included)
    P.tol = (float)(4.0 * std::ldexp(absmax * 1.25 + 8.0 * rmax_all, -23) + 8.0 * std::ldexp(2.0 * rmax_all, -24));

    // grid levels: per bed, one per radius band rmin_bed * ratio^k <= r < rmin_bed * ratio^(k+1)
    const double ratio = d->level_ratio > 1.f ? d->level_ratio : 2.0;
    std::vector<int> lvl(n, 0);
    std::vector<LevelGrid> levels;
    int max_nit = 0;
    int64_t total_cells = 0;
    // Levels are laid out bed by bed in decreasing n_it, and the Morton re-sort
    // orders particles by level: the particles still sweeping at sweep `it`
    // then form a prefix of the slots, and each sweep launches over that prefix.
    std::vector<int> border(nbeds);
    std::vector<size_t> poff(nbeds);
    std::vector<int> goff(nbeds);
    for (int k = 0, o = 0, g = 0; k < nbeds; ++k) {
        border[k] = k;
        poff[k] = o;
        goff[k] = g;
        o += descs[k].n;
        g += descs[k].n_geom;
    }
    std::stable_sort(border.begin(), border.end(), [&](int x, int y) { return descs[x].n_it > descs[y].n_it; });
    {
        for (int kk = 0; kk < nbeds; ++kk) {
            const int k = border[kk];
            const size_t o = poff[k];
            const int g0 = goff[k];
            const dem_bed_desc& dk = descs[k];
            const int m = dk.n;
            max_nit = std::max(max_nit, dk.n_it);
            double rmin = 1e300;
            for (int i = 0; i < m; ++i) rmin = std::min(rmin, (double)rad[o + i]);
            std::vector<int> band(m, 0);
            int bmax = 0;
            for (int i = 0; i < m; ++i) {
                int q = 0;
                double edge = rmin * ratio;
                while (q < 15 && (double)rad[o + i] >= edge) { ++q; edge *= ratio; }
                band[i] = q;
                bmax = std::max(bmax, q);
            }
            // the bed's levels: non-empty bands in increasing size
            const int first = (int)levels.size();
            std::vector<int> remap(bmax + 1, -1);
            std::vector<char> used(bmax + 1, 0);
            for (int i = 0; i < m; ++i) used[band[i]] = 1;
            if (m == 0) used[0] = 1;
            for (int q = 0; q <= bmax; ++q)
                if (used[q]) {
                    remap[q] = (int)levels.size();
                    LevelGrid g;
                    memset(&g, 0, sizeof g);
                    g.bed = k;
                    g.nit = dk.n_it;
                    levels.push_back(g);
                }
            if ((int)levels.size() > DEM_MAX_LEVELS) {
                release(b);
                return fail(DEM_ERR_ARG, "more than %d grid levels over all beds", DEM_MAX_LEVELS);
            }
            const int last = (int)levels.size();
            // bounding box and largest radius of every level
            std::vector<double> lo(3 * (last - first), 1e300), hi(3 * (last - first), -1e300), rmx(last - first, 0.0);
            for (int i = 0; i < m; ++i) {
                const int l = remap[band[i]];
                lvl[o + i] = l;
                const int j = l - first;
                rmx[j] = std::max(rmx[j], (double)rad[o + i]);
                for (int q = 0; q < 3; ++q) {
                    lo[3 * j + q] = std::min(lo[3 * j + q], pos[3 * (o + i) + q]);
                    hi[3 * j + q] = std::max(hi[3 * j + q], pos[3 * (o + i) + q]);
                }
            }
            for (int l = first; l < last; ++l) {
                LevelGrid& g = levels[l];
                const int j = l - first;
                if (m == 0) {
                    rmx[j] = 1e-3;
                    for (int q = 0; q < 3; ++q) { lo[3 * j + q] = 0; hi[3 * j + q] = 0; }
                }
                double ext = 0.0;
                for (int q = 0; q < 3; ++q) ext = std::max(ext, hi[3 * j + q] - lo[3 * j + q]);
                // the grid covers the level's particles plus a margin; particles
                // that leave it are clamped into the boundary cells (still exact)
                const double margin = std::max(8.0 * rmx[j], 0.1 * ext);
                double cell = 2.0 * rmx[j] * (1.0 + 1e-4) + 2.0 * P.tol;
                int dims[3];
                for (;;) {
                    int64_t c = 1;
                    for (int q = 0; q < 3; ++q) {
                        dims[q] = std::max(1, (int)std::ceil((hi[3 * j + q] - lo[3 * j + q] + 2 * margin) / cell));
                        c *= dims[q];
                    }
                    if (c <= (int64_t)(32 << 20)) break;
                    cell *= 1.25;   // cap the cell count; larger cells stay correct
                }
                g.ox = (float)(lo[3 * j] - margin);
                g.oy = (float)(lo[3 * j + 1] - margin);
                g.oz = (float)(lo[3 * j + 2] - margin);
                g.cell = (float)cell;
                g.inv_cell = (float)(1.0 / cell);
                g.nx = dims[0]; g.ny = dims[1]; g.nz = dims[2];
                g.offset = (int)total_cells;
                g.rmax = (float)rmx[j];
                g.lend = last;
                g.g0 = g0;
                g.g1 = g0 + dk.n_geom;
                total_cells += (int64_t)dims[0] * dims[1] * dims[2];
            }
        }
    }
    // particles still sweeping at each sweep (a prefix after the first re-sort)
    b->n_active.assign(std::max(max_nit, 1), 0);
    for (int k = 0; k < nbeds; ++k)
        for (int it = 0; it < descs[k].n_it; ++it) b->n_active[it] += descs[k].n;
    if (total_cells > (int64_t)(256 << 20)) {
        release(b);
        return fail(DEM_ERR_ARG, "broad-phase grids need %lld cells", (long long)total_cells);
    }
    const int L = (int)levels.size();
    P.n = n;
    P.ng = (int)ng64;
    P.n_levels = L;
    P.n_cells = (int)total_cells;
    P.n_it = max_nit;
    P.dt = d->dt;
    P.inv_dt = 1.0f / d->dt;
    P.e_H = d->e_H;
    P.kn_scale = d->kn_scale > 0.f ? d->kn_scale : 1.0f;
    P.eps_reg = d->eps_reg;
    P.delta_floor = d->delta_floor > 0.f ? d->delta_floor : (float)(1e-6 * 2.0 * rmin_all);
    P.ups = 1.0f / (1.0f + 4.0f * d->damp_steps);
    P.Estar_ss = (float)estar(d->E, d->nu, d->E, d->nu);
    P.mu_t = d->mu_t;
    P.mu_r = d->mu_r;
    P.gx = d->gravity[0]; P.gy = d->gravity[1]; P.gz = d->gravity[2];
    int64_t cap = cap_sum + (cap_default ? 1024 : 0);
    if (cap > (int64_t)0x3fffffff) cap = 0x3fffffff;
    P.max_contacts = (int)cap;
    P.max_geo = 2 * n + 1024;
    P.max_own = DEM_MAX_OWN;
    P.max_geo_body = DEM_MAX_GEO;
    P.lanes = d->lanes;   // 0: two-pass sweep; 1, 2, 4, 8: one kernel, that many threads per body;
                          // 16: resident sweep where the bed takes it, else two-pass
    P.solver = d->solver;
    if (P.solver != 0 && P.solver != 1) {
        release(b);
        return fail(DEM_ERR_ARG, "solver = %d is not 0 (Jacobi) or 1 (coloured Gauss-Seidel)", d->solver);
    }
    if (!(d->restitution >= 0.f && d->restitution <= 1.f) || !(d->impact_speed >= 0.f) ||
        !std::isfinite(d->impact_speed)) {
        release(b);
        return fail(DEM_ERR_ARG, "need 0 <= restitution <= 1 and a finite impact_speed >= 0");
    }
    P.e_imp = d->restitution;
    P.v_imp = d->impact_speed;
    P.n_beds = nbeds;
    P.spin_limit = DEM_SPIN_LIMIT;
    if (const char* e = std::getenv("DEM_TEST_SPIN_LIMIT")) {
        const long v = std::strtol(e, nullptr, 10);
        if (v >= 1 && v <= (long)DEM_SPIN_LIMIT) P.spin_limit = (unsigned)v;
    }
    for (int k = 1; k < nbeds && P.solver; ++k)
        if (descs[k].n_it != descs[0].n_it) {
            release(b);
            return fail(DEM_ERR_ARG, "the Gauss-Seidel solver needs the same n_it in every bed");
        }
    if (P.lanes != 0 && P.lanes != 1 && P.lanes != 2 && P.lanes != 4 && P.lanes != 8 &&
        P.lanes != DEM_LAYOUT_RESIDENT) {
        release(b);
        return fail(DEM_ERR_ARG, "lanes = %d is not 0, 1, 2, 4, 8 or 16", d->lanes);
    }
    b->levels = levels;
    P.nit_uniform = 1;
    for (int k = 1; k < nbeds; ++k) P.nit_uniform &= descs[k].n_it == descs[0].n_it;

    // sinkage references: highest particle top under each primitive's footprint (its own bed)
    {
        b->z_ref.assign(P.ng, 0.0);
        size_t o = 0;
        int g0 = 0;
        for (int k = 0; k < nbeds; ++k) {
            const dem_bed_desc& dk = descs[k];
            const int ngk = dk.n_geom;
            std::vector<int> types(ngk);
            std::vector<double> gc(3 * (size_t)ngk), gR(9 * (size_t)ngk), ghe(3 * (size_t)ngk);
            for (int g = 0; g < ngk; ++g) {
                types[g] = dk.geom[g].type;
                for (int q = 0; q < 3; ++q) { gc[3 * g + q] = dk.geom[g].c[q]; ghe[3 * g + q] = dk.geom[g].he[q]; }
                for (int q = 0; q < 9; ++q) gR[9 * g + q] = dk.geom[g].R[q];
            }
            std::vector<double> rr(rad.begin() + o, rad.begin() + o + dk.n);
            std::vector<double> zr;
            surface_refs(dk.n, pos.data() + 3 * o, 3, rr.data(), 1, ngk, types.data(), gc.data(), gR.data(),
                         ghe.data(), zr);
            for (int g = 0; g < ngk; ++g) b->z_ref[g0 + g] = zr[g];
            g0 += ngk;
            o += dk.n;
        }
    }

    // ---- device memory ----
    DevBuf& B = b->B;
    const size_t N = std::max(n, 1), C = (size_t)P.max_contacts, GC = (size_t)P.max_geo;
    const size_t NC = (size_t)P.n_cells;
    const int nbr = radix_blocks(n);
    dem_status st = DEM_OK;
#define AL(ptr, cnt) if (st == DEM_OK) st = dalloc_n(b, &(ptr), (cnt))
    AL(B.lv, (size_t)L);
    AL(B.pos, N); AL(B.posr, N); AL(B.vw0, N); AL(B.vw[0], N); AL(B.vw[1], N);
    AL(B.id, N); AL(B.lvl, N); AL(B.prev_of, N); AL(B.resorted, 1); AL(B.err, 1);
    AL(B.committed, 1); AL(B.need, 2);
    AL(B.lvl_lo, 3 * (size_t)L); AL(B.lvl_hi, 3 * (size_t)L); AL(B.tolv, 2);
    AL(B.body_cell, N); AL(B.cell_cnt, NC + 1); AL(B.cell_start, NC + 1); AL(B.cell_fill, NC + 1);
    AL(B.cell_body, N); AL(B.cell_pos, N); AL(B.cell_id, N);
    AL(B.tmp_own, N * (size_t)P.max_own); AL(B.tmp_geo, N * (size_t)P.max_geo_body);
    AL(B.own_cnt, N + 1); AL(B.in_cnt, N + 1); AL(B.geo_cnt, N + 1); AL(B.in_fill, N + 1);
    AL(B.own_start[0], N + 1); AL(B.own_start[1], N + 1); AL(B.inc_start, N + 1);
    AL(B.geo_start[0], N + 1); AL(B.geo_start[1], N + 1);
    AL(B.c_other, C); AL(B.c_key[0], C); AL(B.c_key[1], C); AL(B.rec, 3 * C); AL(B.c_delta, C);
    AL(B.lamA[0], C); AL(B.lamA[1], C); AL(B.lamB[0], C); AL(B.lamB[1], C);
    AL(B.lamW[0], 2 * C); AL(B.lamW[1], 2 * C); AL(B.inc, 2 * C);
    AL(B.c_self, C); AL(B.c_pos, C); AL(B.c_idx, C); AL(B.imp, 2 * C);
    AL(B.g_key[0], GC); AL(B.g_key[1], GC); AL(B.grec, 6 * GC); AL(B.g_delta, GC);
    AL(B.glamA[0], GC); AL(B.glamA[1], GC); AL(B.glamB[0], GC); AL(B.glamB[1], GC);
    AL(B.glamW[0], 2 * GC); AL(B.glamW[1], 2 * GC); AL(B.g_body, GC); AL(B.gsh, GC);
    AL(B.geom, (size_t)std::max(P.ng, 1)); AL(B.gacc, 6 * (size_t)std::max(P.ng, 1));
    AL(B.grp, DEM_MAX_GROUPS); AL(B.gcnt, DEM_MAX_GROUPS); AL(B.gimp, 9 * DEM_MAX_GROUPS);
    AL(B.gl_list, GC); AL(B.gl_count, 1);
    AL(B.key_a, N); AL(B.key_b, N); AL(B.val_a, N); AL(B.val_b, N);
    AL(B.hist, 256 * (size_t)nbr + 1);
    AL(B.t_pos, N); AL(B.t_vw, N); AL(B.t_id, N); AL(B.t_lvl, N);
    // scan scratch: tile totals of up to 3 columns over the largest scanned array
    const size_t scan_n = std::max({NC + 1, N + 1, 256 * (size_t)nbr + 1});
    AL(B.scan_tmp, 3 * (scan_n / 2048 + 2));
#undef AL
    if (st != DEM_OK) {
        release(b);
        return st;
    }

    // ---- upload ----
    std::vector<double4_32a> hp(N);
    std::vector<float4> hr(N);
    std::vector<VW> hv(N);
    std::vector<int> hid(N), hl(N);
    for (int i = 0; i < n; ++i) {
        hp[i] = make_double4_32a(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], (double)rad[i]);
        hr[i] = make_float4((float)pos[3 * i], (float)pos[3 * i + 1], (float)pos[3 * i + 2], rad[i]);
        hv[i].v = make_float4(vel[3 * i], vel[3 * i + 1], vel[3 * i + 2], im[i]);
        hv[i].w = make_float4(omg[3 * i], omg[3 * i + 1], omg[3 * i + 2], iI[i]);
        hid[i] = i;
        hl[i] = lvl[i];
    }
    std::vector<GeomDev> hg(std::max(P.ng, 1));
    for (int g = 0; g < P.ng; ++g) {
        const dem_geom& G = geoms[g];
        GeomDev& o = hg[g];
        memset(&o, 0, sizeof o);
        for (int k = 0; k < 3; ++k) { o.c[k] = G.c[k]; o.he[k] = G.he[k]; o.v[k] = G.v[k]; o.w[k] = G.w[k]; }
        for (int k = 0; k < 9; ++k) o.R[k] = G.R[k];
        o.type = G.type;
        o.Estar = (float)estar(d->E, d->nu, G.E, G.nu);
        o.mu_t = G.mu_t;
        o.mu_r = G.mu_r;
        o.grp = -1;
        for (int k = 0; k < 3; ++k) { o.fc[k] = (float)o.c[k]; o.fn[k] = (float)o.R[3 * k + 2]; }
        o.bound = (float)(G.type == DEM_GEOM_BOX ? std::sqrt(G.he[0] * G.he[0] + G.he[1] * G.he[1] + G.he[2] * G.he[2])
                                                 : std::sqrt(G.he[0] * G.he[0] + G.he[2] * G.he[2])) * 1.0001f;
    }
    cudaStream_t s = b->stream;
    CK(cudaMemcpyAsync(B.lv, levels.data(), L * sizeof(LevelGrid), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.pos, hp.data(), N * sizeof(double4_32a), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.posr, hr.data(), N * sizeof(float4), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.vw0, hv.data(), N * sizeof(VW), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.id, hid.data(), N * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.lvl, hl.data(), N * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(B.geom, hg.data(), hg.size() * sizeof(GeomDev), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(B.own_start[0], 0, (N + 1) * sizeof(int), s));
    CK(cudaMemsetAsync(B.own_start[1], 0, (N + 1) * sizeof(int), s));
    CK(cudaMemsetAsync(B.geo_start[0], 0, (N + 1) * sizeof(int), s));
    CK(cudaMemsetAsync(B.geo_start[1], 0, (N + 1) * sizeof(int), s));
    CK(cudaMemsetAsync(B.inc_start, 0, (N + 1) * sizeof(int), s));
    CK(cudaMemsetAsync(B.err, 0, sizeof(int), s));
    CK(cudaMemsetAsync(B.committed, 0, sizeof(long long), s));
    CK(cudaMemsetAsync(B.need, 0, 2 * sizeof(int), s));
    CK(cudaMemsetAsync(B.resorted, 0, sizeof(int), s));
    CK(cudaMemsetAsync(B.gacc, 0, 6 * std::max(P.ng, 1) * sizeof(long long), s));
    CK(cudaMemsetAsync(B.grp, 0, DEM_MAX_GROUPS * sizeof(GroupDev), s));
    CK(cudaMemsetAsync(B.gcnt, 0, DEM_MAX_GROUPS * sizeof(int), s));
    CK(cudaMemsetAsync(B.gimp, 0, 9 * DEM_MAX_GROUPS * sizeof(long long), s));
    CK(cudaMemsetAsync(B.gl_count, 0, sizeof(int), s));
    CK(cudaStreamSynchronize(s));

    st = build_graphs(b);
    if (st != DEM_OK) {
        std::string keep = g_err;
        release(b);
        g_err = keep;
        return st;
    }
    *out = b;
    return DEM_OK;
}

extern "C" dem_status dem_create_bed(const dem_bed_desc* desc, void* stream, dem_bed** out) {
    return create_impl(desc, 1, stream, out);
}

extern "C" dem_status dem_create_batch(const dem_bed_desc* descs, int32_t nbeds, void* stream, dem_bed** out) {
    return create_impl(descs, nbeds, stream, out);
}

// ---------------------------------------------------------------------------
// graphs
// ---------------------------------------------------------------------------
static dem_status capture(dem_bed* b, cudaGraphExec_t* exec, int* kernels,
                          int (*body)(dem_bed*, int), int arg) {
    cudaStream_t s = b->stream;
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    b->capture_err = 0;
    int k = body(b, arg);
    cudaError_t le = cudaGetLastError();
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (b->capture_err && e == cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(DEM_ERR_CUDA, "graph construction during capture: %s",
                    cudaGetErrorString((cudaError_t)b->capture_err));
    }
    if (le != cudaSuccess) return fail(DEM_ERR_CUDA, "kernel launch during capture: %s", cudaGetErrorString(le));
    if (e != cudaSuccess) return fail(DEM_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(DEM_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    if (kernels) *kernels += k;
    return DEM_OK;
}

static int body_pre(dem_bed* b, int p) {
    const SimParams& P = b->P;
    const DevBuf& B = b->B;
    cudaStream_t s = b->stream;
    const size_t N = std::max(P.n, 1);
    int k = 0;
    cudaMemsetAsync(B.cell_cnt, 0, ((size_t)P.n_cells + 1) * sizeof(int), s);
    cudaMemsetAsync(B.cell_fill, 0, ((size_t)P.n_cells + 1) * sizeof(int), s);
    cudaMemsetAsync(B.in_cnt, 0, (N + 1) * sizeof(int), s);
    cudaMemsetAsync(B.in_fill, 0, (N + 1) * sizeof(int), s);
    cudaMemsetAsync(B.gacc, 0, 6 * std::max(P.ng, 1) * sizeof(long long), s);
    if (P.n_groups > 0) {
        cudaMemsetAsync(B.gl_count, 0, sizeof(int), s);
        cudaMemsetAsync(B.gcnt, 0, DEM_MAX_GROUPS * sizeof(int), s);
        cudaMemsetAsync(B.gimp, 0, 9 * DEM_MAX_GROUPS * sizeof(long long), s);
    }
    // per-level boxes start empty: lo = huge (bytes 0x7f), hi = -huge (bytes 0x80)
    cudaMemsetAsync(B.lvl_lo, 0x7f, 3 * (size_t)P.n_levels * sizeof(int), s);
    cudaMemsetAsync(B.lvl_hi, 0x80, 3 * (size_t)P.n_levels * sizeof(int), s);
    if (P.n == 0) {
        cudaMemsetAsync(B.own_start[p], 0, sizeof(int), s);
        cudaMemsetAsync(B.geo_start[p], 0, sizeof(int), s);
        cudaMemsetAsync(B.inc_start, 0, sizeof(int), s);
        return 0;
    }
    k += launch_cell_count(P, B, s);
    k += launch_scan(B.cell_cnt, B.cell_start, P.n_cells, B.scan_tmp, s);
    k += launch_cell_fill(P, B, s);
    k += launch_pairs(P, B, s);
    // after a fault the scan keeps the last committed step's lists (its warm start)
    k += launch_scan3(B.own_cnt, B.own_cnt, B.in_cnt, B.geo_cnt, B.own_start[p], B.inc_start,
                      B.geo_start[p], P.n, B.scan_tmp, s, B.err);
    k += launch_contacts_build(P, B, p, s);
    k += launch_inc_sort(P, B, s);
    if (P.v_imp > 0.f && b->imp.row) {
        const int ki = launch_impact(P, B, b->imp, p, s, b->side);
        if (ki < 0) b->capture_err = -ki;
        else k += ki;
    }
    k += launch_setup(P, B, p, s);
    k += launch_v0(P, B, p, s);
    return k;
}

static int body_jac(dem_bed* b, int p) {
    int k = 0;
    if (b->P.n == 0) return 0;
    if (b->P.lanes == DEM_LAYOUT_RESIDENT && b->res.prog && resident_ok(b->P, nullptr))
        return launch_resident(b->P, b->B, b->res, p, b->stream);
    for (int it = 0; it < b->P.n_it; ++it) k += launch_jacobi(b->P, b->B, p, it, b->n_active[it], b->stream);
    return k;
}

static int body_post(dem_bed* b, int p) {
    if (b->P.n == 0) return 0;
    return launch_integrate(b->P, b->B, p, b->stream);
}

static int body_resort(dem_bed* b, int) { return launch_resort(b->P, b->B, b->stream); }

static dem_status build_graphs(dem_bed* b) {
    dem_status st;
    if (b->P.v_imp > 0.f && !b->imp.row) {
        // once: the impact stage's rows and iterates at contact capacity
        ImpBuf I{};
        const size_t C = b->P.max_contacts, G = b->P.max_geo;
        auto al = [&](void** q, size_t bytes) { if (st == DEM_OK) st = dalloc(b, q, bytes); };
        st = DEM_OK;
        al((void**)&I.row, C * sizeof(float4));
        al((void**)&I.tgt, C * sizeof(float));
        al((void**)&I.p[0], C * sizeof(float));
        al((void**)&I.p[1], C * sizeof(float));
        al((void**)&I.grow, G * sizeof(float4));
        al((void**)&I.glev, G * sizeof(float4));
        al((void**)&I.gtgt, G * sizeof(float));
        al((void**)&I.gp[0], G * sizeof(float));
        al((void**)&I.gp[1], G * sizeof(float));
        al((void**)&I.bed, std::max(b->nbeds, 1) * sizeof(int));
        al((void**)&I.count, sizeof(int));
        if (st != DEM_OK) return st;
        CK(cudaMemsetAsync(I.count, 0, sizeof(int), b->stream));
        b->imp = I;
    }
    if (b->P.v_imp > 0.f && !b->side) CK(cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking));
    int blocks = 0;
    if (b->P.lanes == DEM_LAYOUT_RESIDENT && resident_ok(b->P, &blocks) && !b->res.prog) {
        // once: the blocks' progress counters
        ResBuf R{};
        if ((st = dalloc(b, (void**)&R.prog, 2 * (size_t)blocks * sizeof(int))) != DEM_OK) return st;
        R.blocks = blocks;
        b->res = R;
    }
    for (int p = 0; p < 2; ++p) {
        int k = 0;
        if ((st = capture(b, &b->g[p][0], &k, body_pre, p)) != DEM_OK) return st;
        if (b->P.n_it > 0 && b->P.n > 0) {
            if ((st = capture(b, &b->g[p][1], &k, body_jac, p)) != DEM_OK) return st;
        }
        if (b->P.n > 0) {
            if ((st = capture(b, &b->g[p][2], &k, body_post, p)) != DEM_OK) return st;
        }
        b->k_step = k;
    }
    int kr = 0;
    if (b->P.n > 1) {
        if ((st = capture(b, &b->g_resort, &kr, body_resort, 0)) != DEM_OK) return st;
    }
    b->k_resort = kr;
    return DEM_OK;
}

// ---------------------------------------------------------------------------
// stepping and read-back
// ---------------------------------------------------------------------------
static cudaEvent_t take_event(dem_bed* b) {
    cudaEvent_t e;
    if (!b->ev_pool.empty()) {
        e = b->ev_pool.back();
        b->ev_pool.pop_back();
    } else {
        cudaEventCreate(&e);
    }
    b->ev_used.push_back(e);
    return e;
}

// fold finished timing events into the sums (call after a synchronisation)
static void collect_timing(dem_bed* b) {
    for (size_t k = 0; k + 4 <= b->ev_used.size(); k += 4) {
        float a = 0, j = 0;
        cudaEventElapsedTime(&a, b->ev_used[k], b->ev_used[k + 3]);
        cudaEventElapsedTime(&j, b->ev_used[k + 1], b->ev_used[k + 2]);
        b->t_step_ms += a;
        b->t_jac_ms += j;
        b->t_steps += 1;
    }
    for (cudaEvent_t e : b->ev_used) b->ev_pool.push_back(e);
    b->ev_used.clear();
}

static dem_status grow_and_replay(dem_bed* b);

// Synchronise and report a latched device fault.  A contact-storage overflow
// is repaired: the arrays grow and the steps from the last committed one are
// run again (grow_and_replay); other faults latch the bed.
static dem_status check_fault(dem_bed* b) {
    for (int round = 0;; ++round) {
        int err = 0;
        CK(cudaMemcpyAsync(&err, b->B.err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
        CK(cudaStreamSynchronize(b->stream));
        if (b->timing) collect_timing(b);
        if (!err) return DEM_OK;
        if (err == DEM_FLAG_CAPACITY && !b->no_grow && round < 8) {
            const dem_status st = grow_and_replay(b);
            if (st == DEM_OK) continue;
            if (st != DEM_ERR_CAPACITY) {
                b->faulted = true;
                return st;
            }
        }
        b->faulted = true;
        if (err & DEM_FLAG_TIMEOUT) return fail(DEM_ERR_TIMEOUT, "a bounded wait of the resident sweep gave up");
        if (err & DEM_FLAG_NONFINITE) return fail(DEM_ERR_NONFINITE, "non-finite velocity");
        return fail(DEM_ERR_CAPACITY, "contact storage overflowed (capacity %d contacts, %d per body)",
                    b->P.max_contacts, b->P.max_own);
    }
}

dem_status dem_check_fault(dem_bed* b) { return check_fault(b); }

// One coloured projected Gauss-Seidel solve (solver 1) between the pre and post
// graphs: colour the step's contacts, then N_it sweeps of one kernel per colour.
// The colour count is only known on the device, so this runs outside graphs.
static dem_status pgs_solve(dem_bed* b, int p) {
    const SimParams& P = b->P;
    const DevBuf& B = b->B;
    cudaStream_t s = b->stream;
    int counts[2] = {0, 0};
    CK(cudaMemcpyAsync(&counts[0], B.own_start[p] + P.n, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&counts[1], B.geo_start[p] + P.n, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int nc = std::min(counts[0], P.max_contacts), ngc = std::min(counts[1], P.max_geo);
    const int total = nc + ngc;
    PgsBuf& S = b->pgs;
    if (!S.col) {   // at capacity, once
        const size_t cap = (size_t)P.max_contacts + P.max_geo;
        dem_status st = DEM_OK;
        auto al = [&](void** q, size_t bytes) { if (st == DEM_OK) st = dalloc(b, q, bytes); };
        al((void**)&S.col, cap * sizeof(int));
        al((void**)&S.prio, cap * sizeof(unsigned long long));
        al((void**)&S.key, cap * sizeof(unsigned long long));
        al((void**)&S.gbody, (size_t)P.max_geo * sizeof(int));
        al((void**)&S.list, cap * sizeof(int));
        al((void**)&S.remaining, sizeof(int));
        al((void**)&S.ncol, sizeof(int));
        al((void**)&S.colcnt, PGS_MAX_COLOURS * sizeof(int));
        al((void**)&S.colstart, PGS_MAX_COLOURS * sizeof(int));
        al((void**)&S.colfill, PGS_MAX_COLOURS * sizeof(int));
        if (st != DEM_OK) return st;
        b->pgs_cap = (int64_t)cap;
    }
    launch_pgs_prepare(P, B, S, p, nc, ngc, s);
    // colouring rounds until every contact has a colour (bounded)
    int remaining = total, rounds = 0;
    while (remaining > 0) {
        if (rounds >= 4096) return fail(DEM_ERR_STATE, "contact colouring did not finish");
        for (int k = 0; k < 8; ++k) launch_pgs_round(P, B, S, p, nc, ngc, s);
        rounds += 8;
        CK(cudaMemcpyAsync(&remaining, S.remaining, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    int ncol = 0;
    launch_pgs_bucket(S, total, false, s);
    std::vector<int> cnt(PGS_MAX_COLOURS, 0), start(PGS_MAX_COLOURS, 0);
    CK(cudaMemcpyAsync(&ncol, S.ncol, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(cnt.data(), S.colcnt, PGS_MAX_COLOURS * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int c = 1; c < PGS_MAX_COLOURS; ++c) start[c] = start[c - 1] + cnt[c - 1];
    CK(cudaMemcpyAsync(S.colstart, start.data(), PGS_MAX_COLOURS * sizeof(int), cudaMemcpyHostToDevice, s));
    launch_pgs_bucket(S, total, true, s);
    for (int it = 0; it < P.n_it; ++it)
        for (int c = 0; c < ncol; ++c)
            if (cnt[c] > 0) launch_pgs_colour(P, B, S, p, nc, start[c], cnt[c], it == P.n_it - 1, s);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));   // the host copy of the colour starts must outlive the launches
    b->pgs_colours = ncol;
    return DEM_OK;
}

// a re-sort is due before this step (unless it already ran in the step that
// overflowed and is being re-run)
static bool resort_due(dem_bed* b) {
    const bool due = b->g_resort && b->steps % b->resort_every == 0 && !b->skip_resort;
    b->skip_resort = false;
    return due;
}

dem_status dem_launch_step(dem_bed* b) {
    const bool resort = resort_due(b);
    const int p = (int)(b->steps & 1);
    if (resort) CK(cudaGraphLaunch(b->g_resort, b->stream));
    CK(cudaGraphLaunch(b->g[p][0], b->stream));
    if (b->P.solver && b->P.n > 0 && b->P.n_it > 0) {
        dem_status st = pgs_solve(b, p);
        if (st != DEM_OK) return st;
    } else if (b->g[p][1]) CK(cudaGraphLaunch(b->g[p][1], b->stream));
    if (b->g[p][2]) CK(cudaGraphLaunch(b->g[p][2], b->stream));
    b->steps++;
    return DEM_OK;
}

extern "C" dem_status dem_step(dem_bed* b, int32_t nsteps) {
    g_err.clear();
    if (!b) return fail(DEM_ERR_ARG, "bed is NULL");
    if (nsteps < 0) return fail(DEM_ERR_ARG, "nsteps < 0");
    if (b->faulted) return fail(DEM_ERR_STATE, "the bed holds a latched device fault");
    CK(cudaSetDevice(b->dev));
    for (int k = 0; k < nsteps; ++k) {
        if (b->timing) {
            const bool resort = resort_due(b);
            const int p = (int)(b->steps & 1);
            if (b->ev_used.size() >= 4096) {
                CK(cudaStreamSynchronize(b->stream));
                collect_timing(b);
            }
            CK(cudaEventRecord(take_event(b), b->stream));
            if (resort) CK(cudaGraphLaunch(b->g_resort, b->stream));
            CK(cudaGraphLaunch(b->g[p][0], b->stream));
            CK(cudaEventRecord(take_event(b), b->stream));
            if (b->P.solver && b->P.n > 0 && b->P.n_it > 0) {
                dem_status st = pgs_solve(b, p);
                if (st != DEM_OK) return st;
            } else if (b->g[p][1]) CK(cudaGraphLaunch(b->g[p][1], b->stream));
            CK(cudaEventRecord(take_event(b), b->stream));
            if (b->g[p][2]) CK(cudaGraphLaunch(b->g[p][2], b->stream));
            CK(cudaEventRecord(take_event(b), b->stream));
            b->steps++;
        } else {
            dem_status st = dem_launch_step(b);
            if (st != DEM_OK) return st;
        }
    }
    return DEM_OK;
}

// ---------------------------------------------------------------------------
// contact-capacity growth
// ---------------------------------------------------------------------------
// A new allocation of `bytes` in place of *p, keeping its first `keep` bytes.
static dem_status regrow(dem_bed* b, void** p, size_t bytes, size_t keep) {
    void* q = nullptr;
    dem_status st = dalloc(b, &q, bytes);
    if (st != DEM_OK) return st;
    if (keep && *p) CK(cudaMemcpyAsync(q, *p, keep, cudaMemcpyDeviceToDevice, b->stream));
    if (*p) dem_dfree(b, *p);
    *p = q;
    return DEM_OK;
}

// Buffers created on first use at the old capacity: freed, made again when used.
static void drop_capacity_buffers(dem_bed* b) {
    auto fr = [&](void* p) { if (p) dem_dfree(b, p); };
    ImpBuf& I = b->imp;
    fr(I.row); fr(I.tgt); fr(I.p[0]); fr(I.p[1]); fr(I.grow); fr(I.glev); fr(I.gtgt); fr(I.gp[0]); fr(I.gp[1]);
    fr(I.bed); fr(I.count);
    b->imp = ImpBuf{};
    PgsBuf& S = b->pgs;
    fr(S.col); fr(S.prio); fr(S.key); fr(S.gbody); fr(S.list); fr(S.remaining); fr(S.ncol); fr(S.colcnt);
    fr(S.colstart); fr(S.colfill);
    b->pgs = PgsBuf{};
    b->pgs_cap = 0;
    dem_adjoint_drop(b);
}

// New capacities: C sphere-sphere and G sphere-geometry contacts, own / geob
// per body (larger or smaller; a smaller one must still hold the contacts of
// the last two steps).  The warm-start lists of both parities (keys,
// world-frame impulses, overlaps) are carried over; every other contact array
// is rebuilt by the next step.
static dem_status grow_capacity(dem_bed* b, int64_t C, int64_t G, int own, int geob) {
    SimParams& P = b->P;
    DevBuf& B = b->B;
    const size_t N = std::max(P.n, 1);
    const size_t C0 = std::min<size_t>(P.max_contacts, (size_t)C), G0 = std::min<size_t>(P.max_geo, (size_t)G);
    dem_status st = DEM_OK;
#define RE(ptr, cnt, keep) \
    if (st == DEM_OK) st = regrow(b, (void**)&(ptr), (size_t)(cnt) * sizeof(*(ptr)), (size_t)(keep) * sizeof(*(ptr)))
    if (C != P.max_contacts) {
        RE(B.c_other, C, 0); RE(B.c_key[0], C, C0); RE(B.c_key[1], C, C0); RE(B.rec, 3 * C, 0);
        RE(B.c_delta, C, C0); RE(B.lamA[0], C, 0); RE(B.lamA[1], C, 0); RE(B.lamB[0], C, 0); RE(B.lamB[1], C, 0);
        RE(B.lamW[0], 2 * C, 2 * C0); RE(B.lamW[1], 2 * C, 2 * C0); RE(B.inc, 2 * C, 0); RE(B.c_self, C, 0);
        RE(B.c_pos, C, 0); RE(B.c_idx, C, 0); RE(B.imp, 2 * C, 0);
    }
    if (G != P.max_geo) {
        RE(B.g_key[0], G, G0); RE(B.g_key[1], G, G0); RE(B.grec, 6 * G, 0); RE(B.g_delta, G, G0);
        RE(B.glamA[0], G, 0); RE(B.glamA[1], G, 0); RE(B.glamB[0], G, 0); RE(B.glamB[1], G, 0);
        RE(B.glamW[0], 2 * G, 2 * G0); RE(B.glamW[1], 2 * G, 2 * G0); RE(B.g_body, G, 0); RE(B.gsh, G, 0);
        RE(B.gl_list, G, 0);
    }
    if (own != P.max_own) RE(B.tmp_own, N * own, 0);
    if (geob != P.max_geo_body) RE(B.tmp_geo, N * geob, 0);
#undef RE
    if (st != DEM_OK) return st;
    P.max_contacts = (int)C;
    P.max_geo = (int)G;
    P.max_own = own;
    P.max_geo_body = geob;
    drop_capacity_buffers(b);
    return rebuild_graphs(b);
}

// After a contact-storage overflow: the step that overflowed and the steps
// enqueued after it did not change the bed (kernels skip their writes while
// the fault flag is set).  Read what the overflow needed, grow the arrays,
// clear the flag and enqueue those steps again from the last committed one.
// Host commands issued between them (plate velocities, loads) have already
// taken their latest values, which the re-run steps use.
static dem_status grow_and_replay(dem_bed* b) {
    const SimParams& P = b->P;
    const DevBuf& B = b->B;
    cudaStream_t s = b->stream;
    long long committed = 0;
    int need[2] = {0, 0}, resorted = 0, tot[2] = {0, 0};
    CK(cudaMemcpyAsync(&committed, B.committed, sizeof committed, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(need, B.need, sizeof need, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&resorted, B.resorted, sizeof(int), cudaMemcpyDeviceToHost, s));
    // totals of the step that overflowed (its scan ran when the overflow came
    // after it; otherwise these are an older committed step's, within capacity)
    const int pf = (int)(committed & 1);
    if (P.n > 0) {
        CK(cudaMemcpyAsync(&tot[0], B.own_start[pf] + P.n, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&tot[1], B.geo_start[pf] + P.n, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    if (committed > b->steps) return fail(DEM_ERR_STATE, "committed step count ahead of the enqueued steps");
    auto grown = [](int64_t need, int64_t have, int64_t pad) {
        return need > have ? std::max(have, need + need / 4 + pad) : have;
    };
    const int64_t C = grown(tot[0], P.max_contacts, 1024), G = grown(tot[1], P.max_geo, 1024);
    const int64_t own = grown(need[0], P.max_own, 8), geob = grown(need[1], P.max_geo_body, 4);
    if (C == P.max_contacts && G == P.max_geo && own == P.max_own && geob == P.max_geo_body)
        return fail(DEM_ERR_CAPACITY, "contact storage overflowed and no limit could be raised");
    if (C > 0x3fffffff || G > 0x3fffffff || own > 4096 || geob > 4096 ||
        (int64_t)std::max(P.n, 1) * std::max(own, geob) > (int64_t)0x7fffffff)
        return fail(DEM_ERR_CAPACITY, "contact storage overflowed beyond the largest supported capacity");
    dem_status st = grow_capacity(b, C, G, (int)own, (int)geob);
    if (st != DEM_OK) return st;
    CK(cudaMemsetAsync(B.err, 0, sizeof(int), s));
    CK(cudaMemsetAsync(B.need, 0, 2 * sizeof(int), s));
    const int64_t target = b->steps;
    b->steps = committed;
    b->skip_resort = resorted != 0;
    b->grows++;
    for (int64_t k = committed; k < target; ++k)
        if ((st = dem_launch_step(b)) != DEM_OK) return st;
    return DEM_OK;
}

extern "C" dem_status dem_apply_plate_velocity(dem_bed* b, int32_t g, const double v[3], const double w[3]) {
    g_err.clear();
    if (!b || !v || !w) return fail(DEM_ERR_ARG, "NULL argument");
    if (g < 0 || g >= b->n_geom) return fail(DEM_ERR_ARG, "geom %d out of range", g);
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(v[k]) || !std::isfinite(w[k])) return fail(DEM_ERR_ARG, "non-finite velocity");
    CK(cudaSetDevice(b->dev));
    if (b->geom_group[g] >= 0) {   // a load-driven group: its prescribed axes, all members
        k_group_motor<<<1, 32, 0, b->stream>>>(b->B, b->P.ng, b->geom_group[g], v[0], v[1], v[2], w[0], w[1], w[2]);
        CK(cudaGetLastError());
        return DEM_OK;
    }
    double vw[6] = {v[0], v[1], v[2], w[0], w[1], w[2]};
    // v and w are adjacent in GeomDev; a pageable source is staged before return
    CK(cudaMemcpyAsync(&b->B.geom[g].v[0], vw, 6 * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    return DEM_OK;
}

extern "C" dem_status dem_set_plate_load(dem_bed* b, int32_t g, const double force[3]) {
    g_err.clear();
    if (!b || !force) return fail(DEM_ERR_ARG, "NULL argument");
    if (g < 0 || g >= b->n_geom) return fail(DEM_ERR_ARG, "geom %d out of range", g);
    if (b->geom_group[g] < 0) return fail(DEM_ERR_ARG, "geom %d is in no load-driven group", g);
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(force[k])) return fail(DEM_ERR_ARG, "non-finite force");
    CK(cudaSetDevice(b->dev));
    const float f[3] = {(float)force[0], (float)force[1], (float)force[2]};
    // a pageable source is staged before the call returns
    CK(cudaMemcpyAsync(b->B.grp[b->geom_group[g]].force, f, sizeof f, cudaMemcpyHostToDevice, b->stream));
    return DEM_OK;
}

// the primitives of one group: their bed's sweep count
static int group_bed_nit(const dem_bed* b, int g) {
    for (const LevelGrid& l : b->levels)
        if (g >= l.g0 && g < l.g1) return l.nit;
    return b->P.n_it;
}

extern "C" dem_status dem_apply_plate_load(dem_bed* b, const int32_t* geoms, int32_t count, double mass,
                                           const double force[3], int32_t dof) {
    g_err.clear();
    if (!b || !geoms || !force) return fail(DEM_ERR_ARG, "NULL argument");
    if (count < 1 || !(mass > 0.0) || !std::isfinite(mass) || dof < 1 || dof > 7)
        return fail(DEM_ERR_ARG, "need count >= 1, mass > 0 and dof in 1..7");
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(force[k])) return fail(DEM_ERR_ARG, "non-finite force");
    if (b->P.n_groups >= DEM_MAX_GROUPS) return fail(DEM_ERR_ARG, "more than %d load-driven groups", DEM_MAX_GROUPS);
    if (b->P.solver) return fail(DEM_ERR_ARG, "the Gauss-Seidel solver does not take load-driven groups");
    const int bed0 = group_bed_nit(b, geoms[0]);
    for (int k = 0; k < count; ++k) {
        const int g = geoms[k];
        if (g < 0 || g >= b->n_geom) return fail(DEM_ERR_ARG, "geom %d out of range", g);
        if (b->geom_group[g] >= 0) return fail(DEM_ERR_ARG, "geom %d already belongs to a group", g);
        for (int m = 0; m < k; ++m)
            if (geoms[m] == g) return fail(DEM_ERR_ARG, "geom %d listed twice", g);
        if (group_bed_nit(b, g) != bed0) return fail(DEM_ERR_ARG, "a group's primitives must share one bed");
    }
    CK(cudaSetDevice(b->dev));
    const int q = b->P.n_groups;
    GeomDev G0;
    CK(cudaMemcpyAsync(&G0, b->B.geom + geoms[0], sizeof G0, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    GroupDev Q;
    memset(&Q, 0, sizeof Q);
    for (int k = 0; k < 3; ++k) {
        Q.v[k] = G0.v[k];
        Q.force[k] = (float)force[k];
    }
    Q.inv_mass = (float)(1.0 / mass);
    Q.dof = dof;
    Q.nit = bed0;
    CK(cudaMemcpyAsync(b->B.grp + q, &Q, sizeof Q, cudaMemcpyHostToDevice, b->stream));
    for (int k = 0; k < count; ++k) {
        const int g = geoms[k];
        // members join with the group's velocity
        CK(cudaMemcpyAsync(&b->B.geom[g].v[0], Q.v, 3 * sizeof(double), cudaMemcpyHostToDevice, b->stream));
        CK(cudaMemcpyAsync(&b->B.geom[g].grp, &q, sizeof(int), cudaMemcpyHostToDevice, b->stream));
        b->geom_group[g] = q;
    }
    CK(cudaStreamSynchronize(b->stream));
    b->P.n_groups = q + 1;
    return rebuild_graphs(b);
}

static double z_bottom(const GeomDev& G) {
    if (G.type == DEM_GEOM_BOX)
        return G.c[2] - (std::fabs(G.R[6]) * G.he[0] + std::fabs(G.R[7]) * G.he[1] + std::fabs(G.R[8]) * G.he[2]);
    if (G.type == DEM_GEOM_CYLINDER) {
        const double az = std::fabs(G.R[8]);
        return G.c[2] - (az * G.he[2] + G.he[0] * std::sqrt(std::max(0.0, 1.0 - az * az)));
    }
    return G.c[2];
}

extern "C" dem_status dem_read_forces(dem_bed* b, int32_t g, double f[3], double t[3], double* sinkage) {
    g_err.clear();
    if (!b) return fail(DEM_ERR_ARG, "bed is NULL");
    if (g < 0 || g >= b->n_geom) return fail(DEM_ERR_ARG, "geom %d out of range", g);
    CK(cudaSetDevice(b->dev));
    long long acc[6];
    GeomDev G;
    for (;;) {   // again if the check re-ran overflowed steps
        const int grows = b->grows;
        CK(cudaMemcpyAsync(acc, b->B.gacc + 6 * g, sizeof acc, cudaMemcpyDeviceToHost, b->stream));
        CK(cudaMemcpyAsync(&G, b->B.geom + g, sizeof G, cudaMemcpyDeviceToHost, b->stream));
        dem_status st = check_fault(b);
        if (st != DEM_OK) return st;
        if (b->grows == grows) break;
    }
    const double sc = 1.0 / (DEM_FIX_SCALE * (double)b->P.dt);
    for (int k = 0; k < 3; ++k) {
        if (f) f[k] = (double)acc[k] * sc;
        if (t) t[k] = (double)acc[3 + k] * sc;
    }
    if (sinkage) *sinkage = b->z_ref[g] - z_bottom(G);
    return DEM_OK;
}

extern "C" dem_status dem_read_geom(dem_bed* b, int32_t g, dem_geom* out) {
    g_err.clear();
    if (!b || !out) return fail(DEM_ERR_ARG, "NULL argument");
    if (g < 0 || g >= b->n_geom) return fail(DEM_ERR_ARG, "geom %d out of range", g);
    CK(cudaSetDevice(b->dev));
    GeomDev G;
    CK(cudaMemcpyAsync(&G, b->B.geom + g, sizeof G, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    out->type = G.type;
    for (int k = 0; k < 3; ++k) { out->c[k] = G.c[k]; out->he[k] = G.he[k]; out->v[k] = G.v[k]; out->w[k] = G.w[k]; }
    for (int k = 0; k < 9; ++k) out->R[k] = G.R[k];
    out->mu_t = G.mu_t;
    out->mu_r = G.mu_r;
    out->E = 0.f;
    out->nu = 0.f;
    return DEM_OK;
}

template <typename T>
static dem_status copy_out(void* dst, const T* src, size_t count) {
    // the caller's buffer may be host or device memory
    CK(cudaMemcpy(dst, src, count * sizeof(T), cudaMemcpyDefault));
    return DEM_OK;
}

extern "C" dem_status dem_read_state(dem_bed* b, double* pos, float* vel, float* omega, int32_t cap) {
    g_err.clear();
    if (!b) return fail(DEM_ERR_ARG, "bed is NULL");
    const int n = b->P.n;
    if (cap < n) return fail(DEM_ERR_ARG, "cap %d < n %d", cap, n);
    CK(cudaSetDevice(b->dev));
    if (n == 0) return check_fault(b);
    std::vector<double4_32a> hp(n);
    std::vector<VW> hv(n);
    std::vector<int> hid(n);
    cudaStream_t s = b->stream;
    dem_status st;
    for (;;) {   // again if the check re-ran overflowed steps
        const int grows = b->grows;
        CK(cudaMemcpyAsync(hp.data(), b->B.pos, n * sizeof(double4_32a), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(hv.data(), b->B.vw0, n * sizeof(VW), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(hid.data(), b->B.id, n * sizeof(int), cudaMemcpyDeviceToHost, s));
        st = check_fault(b);
        if (st != DEM_OK) return st;
        if (b->grows == grows) break;
    }
    std::vector<double> op(3 * (size_t)n);
    std::vector<float> ov(3 * (size_t)n), ow(3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        const int k = hid[i];
        op[3 * k] = hp[i].x; op[3 * k + 1] = hp[i].y; op[3 * k + 2] = hp[i].z;
        ov[3 * k] = hv[i].v.x; ov[3 * k + 1] = hv[i].v.y; ov[3 * k + 2] = hv[i].v.z;
        ow[3 * k] = hv[i].w.x; ow[3 * k + 1] = hv[i].w.y; ow[3 * k + 2] = hv[i].w.z;
    }
    if (pos && (st = copy_out(pos, op.data(), op.size())) != DEM_OK) return st;
    if (vel && (st = copy_out(vel, ov.data(), ov.size())) != DEM_OK) return st;
    if (omega && (st = copy_out(omega, ow.data(), ow.size())) != DEM_OK) return st;
    return DEM_OK;
}

extern "C" dem_status dem_read_contacts(dem_bed* b, int64_t cap, int32_t* key_a, int32_t* key_b,
                                        float* lam7, float* delta, int64_t* count) {
    g_err.clear();
    if (!b || !count) return fail(DEM_ERR_ARG, "NULL argument");
    if (cap < 0) return fail(DEM_ERR_ARG, "cap < 0");
    CK(cudaSetDevice(b->dev));
    *count = 0;
    const int n = b->P.n;
    // repair a pending overflow first (it re-runs steps), then read
    dem_status st0 = check_fault(b);
    if (st0 != DEM_OK || b->steps == 0 || n == 0) return st0;
    const int p = (int)((b->steps - 1) & 1);   // parity of the last step
    cudaStream_t s = b->stream;
    const DevBuf& B = b->B;
    std::vector<int> os(n + 1), gs(n + 1), hid(n);
    CK(cudaMemcpyAsync(os.data(), B.own_start[p], (n + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(gs.data(), B.geo_start[p], (n + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hid.data(), B.id, n * sizeof(int), cudaMemcpyDeviceToHost, s));
    dem_status st = check_fault(b);
    if (st != DEM_OK) return st;
    const int nc = os[n], ngc = gs[n];
    std::vector<int> key(std::max(nc, 1)), gk(std::max(ngc, 1));
    std::vector<float4> lw(2 * (size_t)std::max(nc, 1)), glw(2 * (size_t)std::max(ngc, 1));
    std::vector<float> dl(std::max(nc, 1)), gdl(std::max(ngc, 1));
    if (nc > 0) {
        CK(cudaMemcpyAsync(key.data(), B.c_key[p], nc * sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(lw.data(), B.lamW[p], 2 * (size_t)nc * sizeof(float4), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(dl.data(), B.c_delta, nc * sizeof(float), cudaMemcpyDeviceToHost, s));
    }
    if (ngc > 0) {
        CK(cudaMemcpyAsync(gk.data(), B.g_key[p], ngc * sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(glw.data(), B.glamW[p], 2 * (size_t)ngc * sizeof(float4), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(gdl.data(), B.g_delta, ngc * sizeof(float), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    const int64_t total = (int64_t)nc + ngc;
    *count = total;
    std::vector<int32_t> ka(total), kb(total);
    std::vector<float> l7(7 * (size_t)total), d7(total);
    int64_t m = 0;
    for (int i = 0; i < n; ++i) {
        for (int c = os[i]; c < os[i + 1]; ++c, ++m) {
            ka[m] = hid[i]; kb[m] = key[c]; d7[m] = dl[c];
            const float4 a = lw[2 * (size_t)c], q = lw[2 * (size_t)c + 1];
            const float v[7] = {a.x, a.y, a.z, a.w, q.x, q.y, q.z};
            memcpy(&l7[7 * m], v, sizeof v);
        }
        for (int c = gs[i]; c < gs[i + 1]; ++c, ++m) {
            ka[m] = hid[i]; kb[m] = -(gk[c] + 1); d7[m] = gdl[c];
            const float4 a = glw[2 * (size_t)c], q = glw[2 * (size_t)c + 1];
            const float v[7] = {a.x, a.y, a.z, a.w, q.x, q.y, q.z};
            memcpy(&l7[7 * m], v, sizeof v);
        }
    }
    const int64_t w = std::min<int64_t>(cap, total);
    if (w > 0) {
        if (key_a && (st = copy_out(key_a, ka.data(), w)) != DEM_OK) return st;
        if (key_b && (st = copy_out(key_b, kb.data(), w)) != DEM_OK) return st;
        if (lam7 && (st = copy_out(lam7, l7.data(), 7 * w)) != DEM_OK) return st;
        if (delta && (st = copy_out(delta, d7.data(), w)) != DEM_OK) return st;
    }
    return DEM_OK;
}

extern "C" dem_status dem_sync(dem_bed* b) {
    g_err.clear();
    if (!b) return fail(DEM_ERR_ARG, "bed is NULL");
    CK(cudaSetDevice(b->dev));
    return check_fault(b);
}

extern "C" dem_status dem_get_info(dem_bed* b, dem_info* out) {
    g_err.clear();
    if (!b || !out) return fail(DEM_ERR_ARG, "NULL argument");
    CK(cudaSetDevice(b->dev));
    {   // repair a pending overflow first (it re-runs steps and grows arrays), then read
        const dem_status st = check_fault(b);
        if (st != DEM_OK) return st;
    }
    memset(out, 0, sizeof *out);
    out->n = b->P.n;
    out->n_levels = b->P.n_levels;
    out->n_cells = b->P.n_cells;
    out->steps = b->steps;
    out->contact_capacity = b->P.max_contacts;
    out->kernels_per_step = b->k_step;
    out->kernels_per_resort = b->k_resort;
    out->n_beds = b->nbeds;
    out->lanes = b->P.lanes;
    out->resort_every = b->resort_every;
    out->solver = b->P.solver;
    out->colours = b->P.solver ? b->pgs_colours : 0;
    if (b->imp.count && b->steps > 0) {
        int m = 0;
        CK(cudaMemcpyAsync(&m, b->imp.count, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
        CK(cudaStreamSynchronize(b->stream));
        out->impacts = b->P.v_imp > 0.f ? m : 0;
    }
    if (b->steps > 0 && b->P.n > 0) {
        const int p = (int)((b->steps - 1) & 1);
        int a = 0, g = 0;
        CK(cudaMemcpyAsync(&a, b->B.own_start[p] + b->P.n, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
        CK(cudaMemcpyAsync(&g, b->B.geo_start[p] + b->P.n, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
        CK(cudaStreamSynchronize(b->stream));
        out->contacts = a;
        out->geom_contacts = g;
    }
    return check_fault(b);
}

extern "C" dem_status dem_set_timing(dem_bed* b, int32_t enable) {
    g_err.clear();
    if (!b) return fail(DEM_ERR_ARG, "bed is NULL");
    CK(cudaSetDevice(b->dev));
    CK(cudaStreamSynchronize(b->stream));
    collect_timing(b);
    b->timing = enable != 0;
    b->t_step_ms = b->t_jac_ms = 0;
    b->t_steps = 0;
    return DEM_OK;
}

extern "C" dem_status dem_read_timing(dem_bed* b, double* step_ms, double* jacobi_ms, int64_t* steps) {
    g_err.clear();
    if (!b) return fail(DEM_ERR_ARG, "bed is NULL");
    CK(cudaSetDevice(b->dev));
    CK(cudaStreamSynchronize(b->stream));
    collect_timing(b);
    if (step_ms) *step_ms = b->t_step_ms;
    if (jacobi_ms) *jacobi_ms = b->t_jac_ms;
    if (steps) *steps = b->t_steps;
    return DEM_OK;
}

// scale the impulses of the last step (the next warm start) by s
__global__ void k_rescale_warm(DevBuf B, int p, int n, float s, int cap, int gcap) {
    const int nc = min(B.own_start[p][n], cap), ng = min(B.geo_start[p][n], gcap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 2 * (nc + ng); k += gridDim.x * blockDim.x) {
        float4* q = k < 2 * nc ? &B.lamW[p][k] : &B.glamW[p][k - 2 * nc];
        float4 v = *q;
        *q = make_float4(v.x * s, v.y * s, v.z * s, v.w * s);
    }
}

extern "C" dem_status dem_set_params(dem_bed* b, const dem_bed_desc* d) {
    g_err.clear();
    if (!b || !d) return fail(DEM_ERR_ARG, "NULL argument");
    if (b->faulted) return fail(DEM_ERR_STATE, "the bed holds a latched device fault");
    if (!(d->dt > 0.f) || d->n_it < 0 || !(d->e_H >= 1.f) || d->damp_steps < 0.f || d->mu_t < 0.f ||
        d->mu_r < 0.f || d->eps_reg < 0.f)
        return fail(DEM_ERR_ARG, "invalid solver or material settings");
    const int lanes = d->lanes >= 0 ? d->lanes : b->P.lanes;
    if (lanes != 0 && lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8 && lanes != DEM_LAYOUT_RESIDENT)
        return fail(DEM_ERR_ARG, "bad lanes");
    const int solver = d->solver >= 0 ? d->solver : b->P.solver;
    if (solver != 0 && solver != 1) return fail(DEM_ERR_ARG, "bad solver");
    const float e_imp = d->restitution >= 0.f ? d->restitution : b->P.e_imp;
    const float v_imp = d->impact_speed >= 0.f ? d->impact_speed : b->P.v_imp;
    if (!(e_imp <= 1.f) || !std::isfinite(v_imp)) return fail(DEM_ERR_ARG, "bad restitution or impact_speed");
    if (solver && b->P.n_groups > 0)
        return fail(DEM_ERR_ARG, "the Gauss-Seidel solver does not take load-driven groups");
    CK(cudaSetDevice(b->dev));
    SimParams& P = b->P;
    const float scale = d->dt / P.dt;
    if (b->steps > 0 && P.n > 0 && scale != 1.0f) {
        const int p = (int)((b->steps - 1) & 1);
        k_rescale_warm<<<256, 256, 0, b->stream>>>(b->B, p, P.n, scale, P.max_contacts, P.max_geo);
        CK(cudaGetLastError());
    }
    P.n_it = d->n_it;   // every bed now takes n_it sweeps
    P.nit_uniform = 1;
    for (int q = 0; q < P.n_groups; ++q)
        CK(cudaMemcpyAsync(&b->B.grp[q].nit, &P.n_it, sizeof(int), cudaMemcpyHostToDevice, b->stream));
    for (LevelGrid& g : b->levels) g.nit = d->n_it;
    b->n_active.assign(std::max(d->n_it, 1), P.n);
    P.dt = d->dt;
    P.inv_dt = 1.0f / d->dt;
    P.e_H = d->e_H;
    P.kn_scale = d->kn_scale > 0.f ? d->kn_scale : 1.0f;
    P.eps_reg = d->eps_reg;
    P.ups = 1.0f / (1.0f + 4.0f * d->damp_steps);
    P.mu_t = d->mu_t;
    P.mu_r = d->mu_r;
    P.gx = d->gravity[0]; P.gy = d->gravity[1]; P.gz = d->gravity[2];
    P.lanes = lanes;
    P.solver = solver;
    P.e_imp = e_imp;
    P.v_imp = v_imp;
    CK(cudaMemcpyAsync(b->B.lv, b->levels.data(), b->levels.size() * sizeof(LevelGrid), cudaMemcpyHostToDevice,
                       b->stream));
    CK(cudaStreamSynchronize(b->stream));
    // the test phase starts here: re-take the surface under every primitive
    if (P.n > 0 && P.ng > 0) {
        std::vector<double4_32a> hp(P.n);
        std::vector<GeomDev> hg(P.ng);
        CK(cudaMemcpy(hp.data(), b->B.pos, P.n * sizeof(double4_32a), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(hg.data(), b->B.geom, P.ng * sizeof(GeomDev), cudaMemcpyDeviceToHost));
        std::vector<int> types(P.ng);
        std::vector<double> gc(3 * (size_t)P.ng), gR(9 * (size_t)P.ng), ghe(3 * (size_t)P.ng);
        for (int g = 0; g < P.ng; ++g) {
            types[g] = hg[g].type;
            for (int k = 0; k < 3; ++k) { gc[3 * g + k] = hg[g].c[k]; ghe[3 * g + k] = hg[g].he[k]; }
            for (int k = 0; k < 9; ++k) gR[9 * g + k] = hg[g].R[k];
        }
        surface_refs(P.n, &hp[0].x, 4, &hp[0].w, 4, P.ng, types.data(), gc.data(), gR.data(), ghe.data(),
                     b->z_ref);
    }
    for (int p = 0; p < 2; ++p)
        for (int k = 0; k < 3; ++k)
            if (b->g[p][k]) { cudaGraphExecDestroy(b->g[p][k]); b->g[p][k] = nullptr; }
    if (b->g_resort) { cudaGraphExecDestroy(b->g_resort); b->g_resort = nullptr; }
    return build_graphs(b);
}

static dem_status rebuild_graphs(dem_bed* b) {
    CK(cudaStreamSynchronize(b->stream));
    for (int p = 0; p < 2; ++p)
        for (int k = 0; k < 3; ++k)
            if (b->g[p][k]) { cudaGraphExecDestroy(b->g[p][k]); b->g[p][k] = nullptr; }
    if (b->g_resort) { cudaGraphExecDestroy(b->g_resort); b->g_resort = nullptr; }
    return build_graphs(b);
}

// time `steps` steps of the current configuration on the bed's stream [ms]
static dem_status time_steps(dem_bed* b, int steps, float* ms) {
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const bool was = b->timing;
    b->timing = false;
    CK(cudaEventRecord(e0, b->stream));
    dem_status st = dem_step(b, steps);
    CK(cudaEventRecord(e1, b->stream));
    CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->timing = was;
    return st;
}

extern "C" dem_status dem_autotune(dem_bed* b, int32_t trial_steps, int32_t* lanes_out, int32_t* resort_out) {
    g_err.clear();
    if (!b) return fail(DEM_ERR_ARG, "bed is NULL");
    if (trial_steps < 1) return fail(DEM_ERR_ARG, "trial_steps < 1");
    if (b->faulted) return fail(DEM_ERR_STATE, "the bed holds a latched device fault");
    CK(cudaSetDevice(b->dev));
    dem_status st;
    // every candidate first runs one untimed step, then trial_steps timed ones
    // (the resident layout is opt-in: measured slower than these on every bed tried)
    const int lane_opts[5] = {0, 1, 2, 4, 8};
    int best_lanes = b->P.lanes;
    float best = 1e30f;
    for (int k = 0; k < 5; ++k) {
        b->P.lanes = lane_opts[k];
        if ((st = rebuild_graphs(b)) != DEM_OK) return st;
        if ((st = dem_step(b, 1)) != DEM_OK) return st;
        float ms = 0;
        if ((st = time_steps(b, trial_steps, &ms)) != DEM_OK) return st;
        if ((st = check_fault(b)) != DEM_OK) return st;
        if (ms < best) { best = ms; best_lanes = lane_opts[k]; }
    }
    b->P.lanes = best_lanes;
    if ((st = rebuild_graphs(b)) != DEM_OK) return st;
    // re-sort period: a re-sort costs a few kernels, a stale order costs locality
    const int resort_opts[4] = {5, 10, 20, 50};
    int best_resort = b->resort_every;
    best = 1e30f;
    for (int k = 0; k < 4; ++k) {
        b->resort_every = resort_opts[k];
        const int n = std::max(trial_steps, 2 * resort_opts[k]);
        float ms = 0;
        if ((st = time_steps(b, n, &ms)) != DEM_OK) return st;
        if ((st = check_fault(b)) != DEM_OK) return st;
        if (ms / n < best) { best = ms / n; best_resort = resort_opts[k]; }
    }
    b->resort_every = best_resort;
    // contact storage: 1.5 x the contacts the trial steps needed (the arrays
    // grow again by themselves if the bed later needs more)
    if (b->P.n > 0 && !b->no_grow) {
        int nc[2] = {0, 0}, ng[2] = {0, 0};
        for (int q = 0; q < 2; ++q) {
            CK(cudaMemcpyAsync(&nc[q], b->B.own_start[q] + b->P.n, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
            CK(cudaMemcpyAsync(&ng[q], b->B.geo_start[q] + b->P.n, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
        }
        CK(cudaStreamSynchronize(b->stream));
        const int64_t mc = std::max(nc[0], nc[1]), mg = std::max(ng[0], ng[1]);
        const int64_t C = std::min<int64_t>(mc + mc / 2 + 1024, 0x3fffffff);
        const int64_t G = std::min<int64_t>(mg + mg / 2 + 1024, 0x3fffffff);
        if (C != b->P.max_contacts || G != b->P.max_geo)
            if ((st = grow_capacity(b, C, G, b->P.max_own, b->P.max_geo_body)) != DEM_OK) return st;
    }
    if (lanes_out) *lanes_out = best_lanes;
    if (resort_out) *resort_out = best_resort;
    return DEM_OK;
}

extern "C" dem_status dem_destroy_bed(dem_bed* b) {
    g_err.clear();
    release(b);
    return DEM_OK;
}

extern "C" const char* dem_last_error(void) { return g_err.c_str(); }

// lets other translation units report through dem_last_error()
void dem_set_error_message(const char* msg) { g_err = msg; }
