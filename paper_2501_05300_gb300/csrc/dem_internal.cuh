// Internal declarations of the GB300 DEM library: device data layout, launch
// wrappers and small device helpers shared by the kernels.
//
// Data layout in HBM (slot = Morton-sorted particle index; stable id = index
// in the caller's arrays):
//   bodies   pos   double4_32a (x, y, z, r)        FP64 centres, exact contact tests
//            posr  float4  (x, y, z, r)        FP32 copy for the broad phase
//            vw0   VW (v, 1/m | w, 1/I), 32 B     velocity at the start of the step
//            vw[2] VW                          Jacobi iterates v^k (ping-pong)
//   contacts one record per sphere-sphere contact, owned by one body
//            rec   3 x float4 per contact (normal, SPOOK row data, arms, cones)
//            lamA  float4 (p_n, p_t1, p_t2, p_r.x), lamB float2 (p_r.y, p_r.z)
//            lamW  2 x float4 world-frame impulses kept for the next warm start
//   incidence per body, every contact it takes part in, ordered by the stable
//            id of the other body: int2 (contact | side << 31, other slot)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dem.h"

#define DEM_MAX_LEVELS 256  // grid levels over all beds (radius bands x beds)
#define DEM_MAX_GEOM 512    // kinematic primitives over all beds
#define DEM_MAX_OWN 32   // sphere-sphere contacts one body may own per step (initial; grows on overflow)
#define DEM_MAX_GEO 8    // sphere-geometry contacts per body per step (initial; grows on overflow)
#define DEM_FIX_SCALE 17592186044416.0  // 2^44: fixed-point scale of geometry impulses [N s]
#define DEM_MAX_GROUPS 16  // load-driven rigid groups of primitives

enum { DEM_FLAG_CAPACITY = 1, DEM_FLAG_NONFINITE = 2, DEM_FLAG_TIMEOUT = 4 };

// one body's velocity record: 32 bytes, one memory sector per gather
struct __align__(32) VW {
    float4 v;   // (v.x, v.y, v.z, 1/m)
    float4 w;   // (w.x, w.y, w.z, 1/I)
};

// one incidence entry's impulse share (linear P, angular T), 32 bytes
struct __align__(32) Imp {
    float4 a;   // (P.x, P.y, P.z, T.x)
    float4 b;   // (T.y, T.z, -, -)
};

// One grid level: the particles of one radius band of one bed.
struct LevelGrid {
    float ox, oy, oz;   // origin
    float inv_cell;     // 1 / cell size
    int nx, ny, nz;     // cells per axis (coordinates are clamped into range)
    int offset;         // first global cell index of the level
    float rmax;         // largest radius of the level
    float cell;
    int bed;            // the bed the level belongs to
    int lend;           // one past the bed's last (coarsest) level
    int g0, g1;         // the bed's primitives
    int nit;            // the bed's Jacobi sweeps per step
    int pad[3];
};

struct GeomDev {
    double c[3];
    double R[9];        // row-major, column k = local axis k
    double he[3];
    double v[3];
    double w[3];
    int type;
    float Estar;        // effective modulus of the sphere-geometry pair
    float mu_t, mu_r;
    float bound;        // radius of a sphere around c holding the primitive (box, cylinder)
    int grp;            // load-driven rigid group the primitive belongs to, or -1
    float fc[3];        // c and the third column of R rounded to FP32, for the
    float fn[3];        //   FP32 pre-test (refreshed wherever c or R change)
};

// A load-driven rigid group of primitives (a plate under a normal load): it
// translates along its dynamic axes as one body of mass 1/inv_mass under a
// constant force, its velocity an unknown of the Jacobi solve; along the other
// axes it keeps its prescribed velocity.
struct GroupDev {
    double v[3];        // velocity at the start of the step (all members)
    float force[3];     // external force [N]
    float inv_mass;     // 1 / M
    int dof;            // bit k: axis k is dynamic
    int nit;            // Jacobi sweeps of the group's bed
};

struct SimParams {
    int n, ng, n_levels, n_it;
    int max_contacts;   // capacity of the sphere-sphere contact arrays
    int max_geo;        // capacity of the sphere-geometry contact arrays
    int max_own;        // sphere-sphere contacts one body may own per step
    int max_geo_body;   // sphere-geometry contacts of one body per step
    int n_cells;
    float dt, inv_dt;
    float e_H, kn_scale, eps_reg, delta_floor;
    float ups;          // SPOOK 1 / (1 + 4 tau/dt)
    float Estar_ss;     // particle-particle effective modulus
    float mu_t, mu_r;
    float gx, gy, gz;
    float tol;          // FP32 narrow-phase tolerance [m] at creation: the cells are sized with it,
                        //   and each step's tolerance (tolv) is never below it
    int lanes;          // sweep layout: 0 two-pass, else threads per body in one kernel
    int nit_uniform;    // 1 when every bed takes n_it sweeps
    int n_groups;       // load-driven groups
    int solver;         // 0 projected Jacobi (mass splitting), 1 coloured projected Gauss-Seidel
    float e_imp;        // Newton impact stage: restitution coefficient
    float v_imp;        // impact threshold [m/s]; 0: no impact stage
    int n_beds;
    unsigned spin_limit;   // polls of one neighbour counter before a resident-sweep wait gives up
};

// Polls of one neighbour counter before a wait of the resident sweep gives up
// (about a second).  The environment variable DEM_TEST_SPIN_LIMIT, read when a
// bed is created, overrides it: a test knob that makes the waits give up at
// once, to exercise the DEM_ERR_TIMEOUT path without a hung kernel.
#define DEM_SPIN_LIMIT (1u << 22)

// Device pointers of one bed.  The two warm-start generations (parity of the
// step number) are indexed [0] / [1].
struct DevBuf {
    LevelGrid* lv;      // [n_levels] grid levels (bed-major, fine to coarse)
    // bodies
    double4_32a* pos;
    float4* posr;
    VW* vw0;
    VW* vw[2];
    int* id;
    int* lvl;
    int* prev_of;       // old slot of each slot after a re-sort
    int* resorted;      // 1 during the step that follows a re-sort
    int* err;           // latched DEM_FLAG_* bits.  While it is set no kernel writes the state
                        //   that carries across steps, so the bed stays as the last
                        //   committed step left it (the step can be re-run after a grow)
    long long* committed;   // [1] steps completed without a fault
    int* need;          // [2] largest per-body counts seen in an overflow: owned contacts,
                        //   geometry contacts
    // broad phase
    int* lvl_lo;        // [3 * n_levels] per-level bounding box of the centres,
    int* lvl_hi;        //   floats as order-preserving ints, rebuilt every step
    float* tolv;        // [2] this step's FP32 narrow-phase tolerance: sphere pairs, primitives
    int* body_cell;
    int* cell_cnt;      // [n_cells + 1]
    int* cell_start;    // [n_cells + 1]
    int* cell_fill;     // [n_cells]
    int* cell_body;     // [n] slot of the particle in each cell position
    float4* cell_pos;   // [n] its FP32 centre and radius, in cell order
    int* cell_id;       // [n] its stable id, in cell order
    // per-body candidate lists of the current step
    int2* tmp_own;      // [n * max_own] (other slot, other stable id)
    int* tmp_geo;       // [n * max_geo_body] primitive index
    int* own_cnt;       // [n + 1]
    int* in_cnt;        // [n + 1]
    int* geo_cnt;       // [n + 1]
    int* in_fill;       // [n]
    // scans
    int* own_start[2];  // [n + 1] per parity
    int* inc_start;     // [n + 1]
    int* geo_start[2];  // [n + 1] per parity
    // sphere-sphere contacts
    int* c_other;       // [C] slot of body b
    int* c_key[2];      // [C] stable id of body b, per parity
    float4* rec;        // [3C]
    float* c_delta;     // [C] overlap, kept for read-back
    float4* lamA[2];    // [C] iterate ping-pong
    float2* lamB[2];
    float4* lamW[2];    // [2C] world-frame final impulses, per parity
    int2* inc;          // [2C]
    int* c_self;        // [C] slot of body a (the owner)
    int2* c_pos;        // [C] positions of the contact in a's and b's incidence lists
    int4* c_idx;        // [C] (slot of a, slot of b, c_pos.x, c_pos.y): one load in the sweep
    Imp* imp;           // [2C] per incidence entry: impulse share of its body
    // sphere-geometry contacts (one-sided)
    int* g_key[2];      // [max_geo] primitive index, per parity
    float4* grec;       // [6 * max_geo]
    float* g_delta;     // [max_geo]
    float4* glamA[2];
    float2* glamB[2];
    float4* glamW[2];   // [2 * max_geo]
    int* g_body;        // [max_geo] slot of the body of each geometry contact
    Imp* gsh;           // [max_geo] impulse share of each geometry contact on its body
    // kinematic geometry and its force accumulators
    GeomDev* geom;      // [ng]
    long long* gacc;    // [6 ng] fixed-point impulse and angular impulse
    // load-driven groups
    GroupDev* grp;      // [DEM_MAX_GROUPS]
    int* gcnt;          // [DEM_MAX_GROUPS] contacts of each group this step
    long long* gimp;    // [3][DEM_MAX_GROUPS][3] fixed-point impulse on each group, per
                        //   iterate k (buffer k % 3): read at sweep k, written at k - 1
    int2* gl_list;      // [max_geo] (contact, body) of every contact with a group's primitive
    int* gl_count;      // [1] entries of gl_list this step
    // re-sort scratch
    unsigned* key_a; unsigned* key_b;
    int* val_a; int* val_b;
    int* hist;          // radix histogram [256 * blocks]
    double4_32a* t_pos; VW* t_vw; int* t_id; int* t_lvl;
    // scan scratch
    int* scan_tmp;
};

// ----------------------------------------------------------------------------
// launch wrappers (each returns the number of kernels it enqueued)
// ----------------------------------------------------------------------------
int launch_scan(const int* in, int* out, int n, int* tmp, cudaStream_t s);
// three exclusive scans at once; column b scans b + b2 element-wise; nothing
// is written while *skip != 0 (skip may be NULL)
int launch_scan3(const int* a, const int* b, const int* b2, const int* c, int* oa, int* ob, int* oc,
                 int n, int* tmp, cudaStream_t s, const int* skip);
int launch_cell_count(const SimParams& P, const DevBuf& B, cudaStream_t s);
int launch_cell_fill(const SimParams& P, const DevBuf& B, cudaStream_t s);
int launch_pairs(const SimParams& P, const DevBuf& B, cudaStream_t s);
int launch_contacts_build(const SimParams& P, const DevBuf& B, int parity, cudaStream_t s);
int launch_inc_sort(const SimParams& P, const DevBuf& B, cudaStream_t s);
int launch_setup(const SimParams& P, const DevBuf& B, int parity, cudaStream_t s);
int launch_v0(const SimParams& P, const DevBuf& B, int parity, cudaStream_t s);
// nact: particles of the beds still sweeping at sweep `it` (a prefix of the slots)
int launch_jacobi(const SimParams& P, const DevBuf& B, int parity, int it, int nact, cudaStream_t s);
int launch_integrate(const SimParams& P, const DevBuf& B, int parity, cudaStream_t s);
// contacts of load-driven groups at sweep it (before the sweep's body updates)
int launch_group_contacts(const SimParams& P, const DevBuf& B, int parity, int it, cudaStream_t s);

// coloured projected Gauss-Seidel (solver 1): colouring and colour sweeps.
// Unified contact index u: u < nc sphere-sphere contact u, else sphere-geometry
// contact u - nc.
struct PgsBuf {
    int* col;                   // [cap] colour, -1 while uncoloured
    unsigned long long* prio;   // [cap] priority (mix of the contact key)
    unsigned long long* key;    // [cap] contact key (tie-break)
    int* gbody;                 // [max_geo] body of each sphere-geometry contact
    int* remaining;             // [1] uncoloured contacts
    int* ncol;                  // [1] colours used
    int* colcnt;                // [PGS_MAX_COLOURS] contacts per colour
    int* colstart;              // [PGS_MAX_COLOURS]
    int* colfill;               // [PGS_MAX_COLOURS]
    int* list;                  // [cap] contacts ordered by colour
};
#define PGS_MAX_COLOURS 128
int launch_pgs_prepare(const SimParams& P, const DevBuf& B, const PgsBuf& S, int parity, int nc, int ngc,
                       cudaStream_t s);
int launch_pgs_round(const SimParams& P, const DevBuf& B, const PgsBuf& S, int parity, int nc, int ngc,
                     cudaStream_t s);
int launch_pgs_bucket(const PgsBuf& S, int total, bool fill, cudaStream_t s);
int launch_pgs_colour(const SimParams& P, const DevBuf& B, const PgsBuf& S, int parity, int nc, int first,
                      int count, bool last, cudaStream_t s);

// Newton impact stage (Sec. 2.2), run before the contact rows when the
// threshold is set; its buffers are allocated when it is first enabled.
struct ImpBuf {
    float4* row;        // [C] (n, 1 / D) of each sphere-sphere contact
    float* tgt;         // [C] e u- for impacts, 0 for the other contacts
    float* p[2];        // [C] normal impulse iterates
    float4* grow;       // [G] (n, 1 / D) of each sphere-geometry contact
    float4* glev;       // [G] (lever from the primitive's centre, n . velocity of its point)
    float* gtgt;        // [G]
    float* gp[2];       // [G]
    int* bed;           // [n_beds] 1 when the bed has an impact this step
    int* count;         // [1] impacting contacts this step
};
// side: an idle stream that captures the sweeps into a conditional node's body
int launch_impact(const SimParams& P, const DevBuf& B, const ImpBuf& I, int parity, cudaStream_t s,
                  cudaStream_t side);

// Resident sweep (layout DEM_LAYOUT_RESIDENT): all sweeps of a step in one
// cooperative kernel, one block per SM, each block keeping a contiguous range
// of bodies on chip.
#define DEM_LAYOUT_RESIDENT 16
struct ResBuf {
    int* prog;          // [2 blocks] contact and body phases each block has finished this step
    int blocks;         // grid size (SM count)
};
// can the bed take the resident sweep (and with how many blocks)
bool resident_ok(const SimParams& P, int* blocks);
int launch_resident(const SimParams& P, const DevBuf& B, const ResBuf& R, int parity, cudaStream_t s);
int launch_resort(const SimParams& P, const DevBuf& B, cudaStream_t s);
int launch_radix_sort(unsigned* key_a, int* val_a, unsigned* key_b, int* val_b, int n, int* hist,
                      int* tmp, cudaStream_t s);
int radix_blocks(int n);

// ----------------------------------------------------------------------------
// device helpers
// ----------------------------------------------------------------------------
#define DEM_HD __host__ __device__ __forceinline__

static __device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
static __device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
static __device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
static __device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
// a b + c d with one fixed fusion (the compiler may fuse such a sum either
// way, and may choose differently in different kernels; every sweep layout must
// round alike)
static __device__ __forceinline__ float fma2(float a, float b, float c, float d) {
    return __fmaf_rn(c, d, __fmul_rn(a, b));
}
static __device__ __forceinline__ float dot(float3 a, float3 b) { return __fmaf_rn(a.z, b.z, fma2(a.x, b.x, a.y, b.y)); }
static __device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return make_float3(fma2(a.y, b.z, -a.z, b.y), fma2(a.z, b.x, -a.x, b.z), fma2(a.x, b.y, -a.y, b.x));
}
// a u + b v, component-wise with the same fusion
static __device__ __forceinline__ float3 lin2(float a, float3 u, float b, float3 v) {
    return make_float3(fma2(a, u.x, b, v.x), fma2(a, u.y, b, v.y), fma2(a, u.z, b, v.z));
}

// Orthonormal tangent basis (t1, t2) of a unit normal n with t2 = n x t1,
// branch-free except for the sign of n.z: Duff et al., "Building an Orthonormal
// Basis, Revisited", JCGT 6(1), 2017.
static __device__ __forceinline__ void tangent_basis(float3 n, float3& t1, float3& t2) {
    float sg = copysignf(1.0f, n.z);
    float a = -__frcp_rn(sg + n.z);
    float b = n.x * n.y * a;
    t1 = make_float3(1.0f + sg * n.x * n.x * a, sg * b, -sg * n.x);
    t2 = make_float3(b, sg + n.y * n.y * a, -n.y);
}

// cell coordinate of a position along one axis, clamped into the grid
static __device__ __forceinline__ int cell_coord(float x, float o, float inv, int nmax) {
    int c = __float2int_rd((x - o) * inv);
    return c < 0 ? 0 : (c >= nmax ? nmax - 1 : c);
}

static __device__ __forceinline__ void set_flag(int* err, int bit) { atomicOr(err, bit); }

// velocity of group q at Jacobi iterate k: v* + M^-1 (sum of the impulses of
// iterate k on it) along the dynamic axes, v* = v + dt F / M
static __device__ __forceinline__ void group_velocity_d(const SimParams& P, const DevBuf& B, int q, int k,
                                                        double v[3]) {
    const GroupDev& G = B.grp[q];
    const long long* a = B.gimp + 3 * ((k % 3) * DEM_MAX_GROUPS + q);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        v[ax] = G.v[ax];
        if (G.dof >> ax & 1)
            v[ax] += (double)P.dt * G.force[ax] * G.inv_mass + G.inv_mass * ((double)a[ax] / DEM_FIX_SCALE);
    }
}

static __device__ __forceinline__ float3 group_velocity(const SimParams& P, const DevBuf& B, int q, int k) {
    double v[3];
    group_velocity_d(P, B, q, k, v);
    return make_float3((float)v[0], (float)v[1], (float)v[2]);
}

// clear the impulse sum of iterate it + 2 before sweep it + 1 writes it (sweep
// it runs this from block 0; the sum was last read by sweep it - 1)
static __device__ __forceinline__ void group_clear_ahead(const SimParams& P, const DevBuf& B, int it) {
    if (blockIdx.x == 0 && (int)threadIdx.x < 3 * P.n_groups) {
        const int q = threadIdx.x / 3;
        if (it + 2 <= B.grp[q].nit) B.gimp[3 * (((it + 2) % 3) * DEM_MAX_GROUPS + q) + threadIdx.x % 3] = 0;
    }
}

// add the impulse Pg of one contact on group q to iterate k's sum (fixed point:
// the sum does not depend on the order of the additions)
static __device__ __forceinline__ void group_add(const DevBuf& B, int q, int k, float3 Pg) {
    unsigned long long* a = (unsigned long long*)(B.gimp + 3 * ((k % 3) * DEM_MAX_GROUPS + q));
    const int dof = B.grp[q].dof;
    if (dof & 1) atomicAdd(a, (unsigned long long)__double2ll_rn((double)Pg.x * DEM_FIX_SCALE));
    if (dof & 2) atomicAdd(a + 1, (unsigned long long)__double2ll_rn((double)Pg.y * DEM_FIX_SCALE));
    if (dof & 4) atomicAdd(a + 2, (unsigned long long)__double2ll_rn((double)Pg.z * DEM_FIX_SCALE));
}

// Jacobi sweeps per step of the bed of body i
static __device__ __forceinline__ int body_nit(const SimParams& P, const DevBuf& B, int i) {
    return P.nit_uniform ? P.n_it : B.lv[B.lvl[i]].nit;
}

// floats as ints whose order is the float order (for atomicMin / atomicMax)
static __device__ __forceinline__ int float_ord(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
static __device__ __forceinline__ float ord_float(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }
