/*
 * dem.h -- C ABI of the GB300 (sm_103a) nonsmooth sphere DEM library.
 *
 * The library advances beds of spheres with the time-implicit ("nonsmooth")
 * DEM of arXiv 2501.05300, Sec. 2.2: Newton-Euler bodies with contact
 * constraints (Eq. 2), a Hertz-mapped compliant normal constraint
 * (g_n = delta^{e_H}, eps_n = e_H/k_n, k_n = E* sqrt(d*)/3), Coulomb friction
 * and rolling resistance (Eqs. 5-7), time-integrated with the SPOOK stepper
 * and solved with a fixed number N_it (Eq. 8) of projected Jacobi sweeps,
 * warm-started from the previous step.  Beds may be locally refined: particle
 * size grows with depth (Sec. 2.1), so the broad phase keeps one cell grid per
 * radius band.
 *
 * Conventions for every call:
 *  - SI units.  Positions are double, velocities and material data float.
 *  - Array arguments are caller-owned.  Inputs are copied; they may live in
 *    host memory or in device memory of the bed's GPU (unified addressing).
 *  - Every call returns a dem_status and never throws.  dem_last_error()
 *    returns a thread-local message describing the last failure.
 *  - dem_step only enqueues work on the bed's CUDA stream and returns.  Faults
 *    found on the device are latched in a device flag, and while it is set no
 *    kernel changes the bed: the step that faulted and the steps enqueued after
 *    it are not committed.  The next synchronising call (dem_read_*, dem_sync,
 *    dem_get_info, checkpoints) handles them:
 *      - contact storage exceeded (the total, or one particle's list): the
 *        arrays grow to what the step needed and the uncommitted steps run
 *        again, with the plate velocities and loads current at that call; the
 *        results equal those of a bed created with enough capacity.  The call
 *        then succeeds.  During dem_record / dem_step_adjoint an overflow is
 *        reported instead (DEM_ERR_CAPACITY), as is one beyond 2^30 contacts;
 *      - a non-finite velocity (DEM_ERR_NONFINITE) or a resident-sweep wait
 *        that gave up (DEM_ERR_TIMEOUT) is returned, and the bed then refuses
 *        to step (DEM_ERR_STATE) until it is destroyed.
 *  - Particles are identified by their index in the arrays given to
 *    dem_create_bed ("stable id").  The library reorders particles internally
 *    (Morton order) but every read returns stable-id order.
 */
#ifndef DEM_H
#define DEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dem_status {
    DEM_OK = 0,
    DEM_ERR_ARG = 1,        /* invalid argument; nothing was changed */
    DEM_ERR_CUDA = 2,       /* a CUDA runtime call failed */
    DEM_ERR_CAPACITY = 3,   /* contact storage overflowed during a step */
    DEM_ERR_TIMEOUT = 4,    /* a bounded device wait gave up */
    DEM_ERR_NONFINITE = 5,  /* a non-finite velocity appeared */
    DEM_ERR_STATE = 6       /* the bed holds a latched device fault */
} dem_status;

typedef enum dem_geom_type {
    DEM_GEOM_PLANE = 0,     /* c: point on the plane; normal = local z; solid behind */
    DEM_GEOM_BOX = 1,       /* c: centre; he: half extents (oriented box) */
    DEM_GEOM_CYLINDER = 2   /* c: centre; axis local z; he[0] radius, he[2] half height */
} dem_geom_type;

/* A rigid kinematic primitive: bin walls, plates, grousers (Sec. 3.3).  Its
 * velocity is prescribed (a velocity motor, Sec. 2.2: G_j v = u_j(t)). */
typedef struct dem_geom {
    int32_t type;           /* dem_geom_type */
    double c[3];            /* reference point / centre [m] */
    double R[9];            /* row-major rotation; column k = local axis k in world */
    double he[3];           /* box half extents; cylinder (radius, unused, half height) [m] */
    double v[3];            /* velocity of c [m/s] */
    double w[3];            /* angular velocity about c [rad/s] */
    float E, nu;            /* Young's modulus [Pa] and Poisson ratio of the geometry */
    float mu_t, mu_r;       /* sphere-geometry friction and rolling resistance (Eqs. 6-7) */
} dem_geom;

/* Optional device allocator; when NULL the library uses cudaMallocAsync on the
 * bed's stream.  `stream` is the bed's cudaStream_t.  It must return memory
 * aligned to 256 bytes (as cudaMalloc and PyTorch's caching allocator do); a
 * bed given anything else fails to create with DEM_ERR_CUDA. */
typedef void* (*dem_alloc_fn)(size_t bytes, void* ctx, void* stream);
typedef void (*dem_free_fn)(void* ptr, void* ctx, void* stream);

typedef struct dem_bed_desc {
    int32_t n;                  /* particles, >= 0 */
    const double* pos;          /* [3n] centres (x,y,z) [m], required if n > 0 */
    const float* radius;        /* [n] radii [m] > 0, required if n > 0 */
    const float* vel;           /* [3n] initial velocities [m/s], NULL = 0 */
    const float* omega;         /* [3n] initial angular velocities [rad/s], NULL = 0 */
    const float* inv_mass;      /* [n] override of 1/m, NULL = solid spheres of density rho */
    const float* inv_inertia;   /* [n] override of 1/I, NULL = 1/(2/5 m r^2) */
    float rho;                  /* particle density [kg/m^3] (Sec. 3.1) */
    float E, nu;                /* particle Young's modulus [Pa], Poisson ratio (Sec. 3.1) */
    float mu_t, mu_r;           /* particle-particle friction / rolling resistance (Eqs. 6-7) */
    float e_H;                  /* gap exponent: 1.25 Hertz, 1.0 linear (Sec. 2.2) */
    float damp_steps;           /* damping time tau in steps, tau/dt (Sec. 2.2: 4.5) */
    float dt;                   /* time step [s] (Eq. 9) */
    int32_t n_it;               /* Jacobi sweeps per step (Eq. 8), >= 0 */
    float gravity[3];           /* [m/s^2] */
    float kn_scale;             /* factor on k_n; 1 = the paper's k_n */
    float eps_reg;              /* tangential/rolling compliance, relative to the normal one */
    float delta_floor;          /* overlap floor in the Hertz Jacobian [m]; 0 = 1e-6 * d_min */
    int32_t n_geom;             /* number of primitives, >= 0 */
    const dem_geom* geom;       /* [n_geom], host memory */
    int64_t contact_capacity;   /* sphere-sphere contacts held at first (0 = 8 n + 1024); the
                                   arrays grow when a step overflows them (see Conventions) */
    int32_t resort_every;       /* Morton re-sort period in steps; 0 = 20 */
    float level_ratio;          /* radius ratio per grid level; 0 = 2 */
    int32_t lanes;              /* Jacobi sweep layout: 0 = contact pass + body pass (default);
                                   1, 2, 4, 8 = one kernel with that many threads per particle;
                                   16 = resident: all sweeps of a step in one cooperative kernel,
                                   one block per SM holding a range of bodies on chip (beds of one
                                   n_it, Jacobi, no load-driven groups, up to ~3,500 particles per
                                   SM; other beds take the two-pass layout) */
    dem_alloc_fn alloc;         /* optional allocator (see above) */
    dem_free_fn free_fn;
    void* alloc_ctx;
    int32_t solver;             /* 0 = projected Jacobi with mass splitting (default);
                                   1 = coloured projected Gauss-Seidel (the paper's PGS, Sec. 2.2):
                                   contacts coloured so that no two of a colour share a body, swept
                                   colour by colour with the bodies updated in between, unsplit
                                   masses.  PGS runs outside CUDA graphs (a study mode), needs the
                                   same n_it in every bed, no load-driven groups, no adjoint. */
    float restitution;          /* Newton impact law (Sec. 2.2): restitution coefficient e in
                                   [0, 1] of impacting contacts */
    float impact_speed;         /* impact threshold [m/s]; 0 = no impact stage (default).  When a
                                   bed has a contact whose normal velocity at the start of the step
                                   is below -impact_speed, a velocity-level stage before the SPOOK
                                   solve gives every contact of that bed a normal impulse p >= 0
                                   with u+ >= -e u- for the impacts and u+ >= 0 for the others
                                   (n_it projected Jacobi sweeps, masses split over each body's
                                   contacts, primitives kinematic).  Its impulse on primitives is
                                   part of the step's primitive force.  No adjoint. */
} dem_bed_desc;

typedef struct dem_bed dem_bed;   /* opaque, library-owned */

typedef struct dem_info {
    int32_t n;                  /* particles */
    int32_t n_levels;           /* broad-phase grid levels */
    int64_t n_cells;            /* total cells over all levels */
    int64_t contacts;           /* sphere-sphere contacts of the last step */
    int64_t geom_contacts;      /* sphere-geometry contacts of the last step */
    int64_t steps;              /* steps taken */
    int64_t contact_capacity;
    int32_t kernels_per_step;   /* kernel launches of one plain (non-resort) step */
    int32_t kernels_per_resort; /* extra launches of a re-sort */
    int32_t n_beds;             /* beds advanced together (dem_create_batch) */
    int32_t lanes;              /* current sweep layout (see dem_bed_desc.lanes) */
    int32_t resort_every;       /* current Morton re-sort period */
    int32_t solver;             /* current solver (see dem_bed_desc.solver) */
    int32_t colours;            /* colours of the last PGS step, 0 for Jacobi */
    int64_t impacts;            /* impacting contacts of the last step (impact stage) */
} dem_info;

/* Create a bed from particles, materials and geometry.
 * stream: a cudaStream_t (NULL = the library creates a non-blocking stream).
 * Synchronous: returns when the bed is ready.  On failure *out is NULL. */
dem_status dem_create_bed(const dem_bed_desc* desc, void* stream, dem_bed** out);

/* Create one object advancing nbeds independent beds together, every step in
 * one graph launch: many small beds, like the paper's 36 refinement variants
 * (Sec. 3.3, Table 2), fill the GPU together where one alone would not.
 * descs[k] describes bed k exactly as for dem_create_bed; the solver and
 * material settings (dt, e_H, damp_steps, E, nu, mu_t, mu_r, gravity, kn_scale,
 * eps_reg, delta_floor, restitution, impact_speed) must be equal across beds,
 * n_it (Eq. 8) may differ.
 * Particles of bed k get the stable ids after those of beds 0..k-1, and its
 * primitives the indices after theirs (all dem_read_* calls use these global
 * numbers).  Beds never interact, even where they overlap in space.  Allocator,
 * re-sort period, level ratio and lanes are taken from descs[0]. */
dem_status dem_create_batch(const dem_bed_desc* descs, int32_t nbeds, void* stream, dem_bed** out);

/* Autotuner: times trial_steps steps (after one untimed step) of every sweep
 * layout (lanes 0, 1, 2, 4, 8; the resident layout 16 is opt-in), keeps the
 * fastest, then times re-sort periods 5, 10, 20, 50 and keeps the fastest.
 * Last, it sizes the contact storage to 1.5 times the contacts the trial
 * steps needed (plus 1024; larger or smaller than before), which later
 * overflows grow as usual.  The bed advances by those steps: call it in place
 * of warm-up steps.  Choices are returned through lanes_out and
 * resort_out (either may be NULL) and stay in effect.  Synchronises. */
dem_status dem_autotune(dem_bed* bed, int32_t trial_steps, int32_t* lanes_out, int32_t* resort_out);

/* Enqueue nsteps time steps (detection, SPOOK rows, N_it Jacobi sweeps,
 * integration; Sec. 2.2) on the bed's stream.  Asynchronous. */
dem_status dem_step(dem_bed* bed, int32_t nsteps);

/* Prescribe the velocity of primitive `geom_id` from the next step on
 * (motor constraint, Sec. 2.2).  v [m/s], w [rad/s] host arrays of 3. */
dem_status dem_apply_plate_velocity(dem_bed* bed, int32_t geom_id, const double v[3],
                                    const double w[3]);

/* Contact force f [N] and torque t [N m] about the primitive's centre exerted
 * by the particles during the last step (impulse / dt), and the sinkage [m]:
 * the height of the particle surface under the primitive at creation minus the
 * current lowest point of the primitive (Sec. 3.3).  Synchronises the stream.
 * Any of f, t, sinkage may be NULL. */
dem_status dem_read_forces(dem_bed* bed, int32_t geom_id, double f[3], double t[3],
                           double* sinkage);

/* Copy the state in stable-id order: pos [3n] double, vel [3n], omega [3n]
 * float; any may be NULL.  cap = capacity in particles (>= n).  Synchronises. */
dem_status dem_read_state(dem_bed* bed, double* pos, float* vel, float* omega, int32_t cap);

/* Copy the contacts of the last step, in no particular order.  For contact k:
 * key_a[k] = stable id of body a; key_b[k] = stable id of body b, or -(g+1)
 * for primitive g; lam7[7k..7k+6] = impulse on a in world frame
 * (p_n, p_t.x, p_t.y, p_t.z, p_r.x, p_r.y, p_r.z) with the normal pointing from
 * b to a; delta[k] = overlap [m].  Any output may be NULL.  Writes at most cap
 * contacts and returns the total in *count.  Synchronises. */
dem_status dem_read_contacts(dem_bed* bed, int64_t cap, int32_t* key_a, int32_t* key_b,
                             float* lam7, float* delta, int64_t* count);

/* Current pose and velocity of primitive geom_id.  Synchronises. */
dem_status dem_read_geom(dem_bed* bed, int32_t geom_id, dem_geom* out);

/* Wait for the bed's stream; returns a latched device fault if any. */
dem_status dem_sync(dem_bed* bed);

/* Sizes and counters (synchronises). */
dem_status dem_get_info(dem_bed* bed, dem_info* out);

/* Record CUDA events around the Jacobi sweeps of every step (enable != 0).
 * dem_read_timing returns, for the steps enqueued since timing was enabled,
 * the summed milliseconds of the whole steps and of their Jacobi sweeps and
 * the number of steps.  Synchronises. */
dem_status dem_set_timing(dem_bed* bed, int32_t enable);
dem_status dem_read_timing(dem_bed* bed, double* step_ms, double* jacobi_ms, int64_t* steps);

/* Change the solver and material settings of an existing bed between steps,
 * as between the generation and the test phases of Sec. 3.1 / 3.3 (reduced
 * friction while settling).  Taken from `desc`: dt, n_it, damp_steps, e_H,
 * mu_t, mu_r, gravity, kn_scale, eps_reg and lanes, and solver, restitution
 * and impact_speed unless negative (negative keeps the current value); every
 * other field is ignored.  The warm-start impulses of the last step are rescaled by
 * dt_new / dt_old so that they stand for the same forces, and the sinkage
 * reference of every primitive is re-taken from the current particle surface
 * (the test phase starts here).  Synchronises; the per-step graphs are rebuilt. */
dem_status dem_set_params(dem_bed* bed, const dem_bed_desc* desc);

/* Load-driven plate (Sec. 3.3: the plate under a normal load F_N).  The listed
 * primitives (count of them, one bed) become one rigid group that translates
 * along the axes whose bit is set in dof (bit 0 x, 1 y, 2 z) as a body of the
 * given mass [kg] under the constant external force [N] (gravity is not added:
 * include M g in force if wanted).  Its velocity along those axes is an unknown
 * of every step's Jacobi solve, with split mass M / (contacts of the group);
 * along the other axes the group keeps the motor velocity of dem_apply_plate_velocity
 * (which, on a member, sets the whole group's motor axes).  The group starts
 * with the velocity of geoms[0]; it does not rotate dynamically.  Up to 16
 * groups per object.  DEM_ERR_ARG for bad arguments or a primitive already in a
 * group.  Synchronises. */
dem_status dem_apply_plate_load(dem_bed* bed, const int32_t* geoms, int32_t count, double mass,
                                const double force[3], int32_t dof);

/* Change the external force [N] of the load-driven group that primitive geom
 * belongs to, from the next step on (a load applied gradually, as at the start
 * of the pressure-sinkage test of Sec. 3.3).  Stream-ordered, no
 * synchronisation.  DEM_ERR_ARG if geom is in no group or force is not finite. */
dem_status dem_set_plate_load(dem_bed* bed, int32_t geom, const double force[3]);

/* ---- differentiation (reverse mode) -------------------------------------
 * Gradients of J = sum_t sum_g dJ_dF[t][g] . F_t,g, a linear functional of
 * the force on every primitive in every step, with respect to the scale s_k of
 * the normal stiffness k_n = s_k E* sqrt(d*) / 3 (Sec. 2.2, all contacts), the
 * particle-particle friction coefficient mu_t (Eq. 6) and the particle-particle
 * rolling-resistance coefficient mu_r (Eq. 7).  The derivative is taken along
 * the contact set of every recorded step (fixed topology per step); contacts
 * that open or close inside the window are not differentiated.
 *
 * dem_record: advance the bed nsteps steps (as dem_step) and keep a checkpoint
 * of its state every ckpt_every steps (0: the interval that minimises the
 * memory of checkpoints plus one segment's tapes, about
 * sqrt(nsteps * checkpoint / tape of one step); the reverse pass recomputes
 * each step once whatever the interval).  forces (may be NULL): host or device
 * buffer of nsteps * n_geom * 3 doubles, the force on each primitive in each
 * step [N], the same numbers dem_read_forces returns after that step.
 * Synchronises.  Requirements: no primitive spins (planes, oriented boxes and
 * cylinders that translate are differentiated, the normal's dependence on the
 * contact's place on a box edge or corner, a cylinder side or rim included), no
 * load-driven group, every bed of the object takes the same n_it, the Jacobi
 * solver, no impact stage; else DEM_ERR_ARG.  Memory:
 * one checkpoint (positions, velocities, warm start: about 100 B per particle
 * and 40 B per contact) per ckpt_every steps.
 *
 * dem_step_adjoint: the gradient for the last recorded window.  dJ_dF: host or
 * device buffer shaped like `forces`.  grad[3] (host) receives dJ/ds_k,
 * dJ/dmu_t, dJ/dmu_r.  Each segment of ckpt_every steps is recomputed from its
 * checkpoint with a tape of every Jacobi iterate (24 B per contact and 32 B
 * per particle per sweep, for the ckpt_every steps of one segment), then
 * reversed.  The bed is left in the state after the window, so stepping may
 * continue, and the call may be repeated with other dJ_dF.  DEM_ERR_STATE if
 * nothing was recorded, the bed was stepped since, or settings changed.
 * Synchronises.  No counterpart in the paper, which does not differentiate its
 * simulations; the step it reverses is the paper's. */
dem_status dem_record(dem_bed* bed, int32_t nsteps, int32_t ckpt_every, double* forces);
dem_status dem_step_adjoint(dem_bed* bed, const double* dJ_dF, double grad[3]);

/* ---- whole-state checkpoints -----------------------------------------------
 * dem_checkpoint_save: a device copy of everything the next step reads
 * (positions, velocities, slot order, primitive poses and velocities, the last
 * step's impulses that warm-start the next) plus the last step's geometry
 * forces.  dem_checkpoint_restore puts the bed back into that state; stepping
 * from it repeats the original steps bit for bit (under the same settings;
 * settings changed with dem_set_params since the save stay in force).  A
 * restore ends a window recorded with dem_record.  Checkpoints belong to their
 * bed (DEM_ERR_ARG for another bed); free them with dem_checkpoint_free before
 * dem_destroy_bed.  Memory: about 100 B per particle and 40 B per contact, from
 * the bed's allocator.  Synchronise.  No counterpart in the paper. */
typedef struct dem_checkpoint dem_checkpoint;
dem_status dem_checkpoint_save(dem_bed* bed, dem_checkpoint** out);
dem_status dem_checkpoint_restore(dem_bed* bed, const dem_checkpoint* ckpt);
dem_status dem_checkpoint_free(dem_bed* bed, dem_checkpoint* ckpt);

/* Release all device memory of the bed.  NULL is accepted. */
dem_status dem_destroy_bed(dem_bed* bed);

/* Sphere-sphere contacts of n spheres, for callers that may not allocate GPU
 * memory: a host program whose device memory is held by another framework's
 * caching allocator, a real-time loop that forbids allocation after start-up,
 * or code enqueuing work while a stream is being captured.  The paper has no
 * counterpart: it is a service entry point of this library.
 *   pos [3n] double, radius [n] float: device memory, read only.
 *   key_a, key_b [cap] int32, delta [cap] float: device memory; contact k is the
 *     pair (key_a[k] < key_b[k]) of input indices with overlap delta[k] > 0, found
 *     with the same exact predicate as dem_step; order unspecified.
 *   count: device int64, receives the number of contacts (a 64-bit count: it may
 *     exceed cap, and only the first cap contacts are written), or -1 when a
 *     radius is not positive and finite or a coordinate is not finite (nothing
 *     is written then).
 *   stream: cudaStream_t (NULL = legacy default stream).  Asynchronous.
 * Allocates nothing: every intermediate array lives in one static device array
 * of about 8.4 MB, present on every GPU that loads the library until the process
 * exits.  n must be <= 262144 (DEM_ERR_ARG otherwise).  The first call on a
 * device, and the first call after a device reset, looks up that array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls share the array, so calls that overlap on the GPU race:
 * order them on one stream. */
dem_status dem_detect_contacts_noalloc(int32_t n, const double* pos, const float* radius, int64_t cap,
                                       int32_t* key_a, int32_t* key_b, float* delta, int64_t* count,
                                       void* stream);

/* Thread-local description of the last error ("" if none). */
const char* dem_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DEM_H */
