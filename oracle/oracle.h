/*
 * FP64 CPU oracle for the nonsmooth sphere DEM time step of
 * "Local particle refinement in terramechanical simulations" (arXiv 2501.05300).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA library against
 * an obviously correct, slow restatement of the paper's method.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * What it computes, per time step (Sec. 2.2, Eqs. 2-9):
 *   1. O(N^2) brute-force contact detection (every pair tested; Sec. 2.2: the
 *      contact set is recomputed every step), plus closed-form sphere-geometry
 *      tests (plane, oriented box, cylinder).
 *   2. The SPOOK discretisation of the Hertz-mapped compliant normal constraint
 *      (g_n = delta^{e_H}, eps_n = e_H/k_n, k_n = E* sqrt(d*)/3, Sec. 2.2) with
 *      damping time tau = 4.5 dt, Coulomb friction |lambda_t| <= mu_t lambda_n
 *      and rolling resistance |lambda_r| <= mu_r r lambda_n (Eqs. 5-7).
 *   3. A fixed number N_it of projected Jacobi sweeps (the paper's PGS replaced
 *      by a Jacobi-style sweep with mass splitting), warm-started from the
 *      previous step's multipliers matched by contact key (Sec. 2.2, "warm-
 *      starting").
 *   4. The SPOOK position update x += dt v, geometry forces and kinematic
 *      geometry motion.
 * Explicit Jacobian matrices and block inverses are used on purpose: the code
 * is written for readability against the paper, not speed.
 */
#ifndef DEM_ORACLE_H
#define DEM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_PLANE = 0, ORC_BOX = 1, ORC_CYLINDER = 2 };
enum { ORC_MAX_GROUPS = 16 };

typedef struct orc_params {
    double rho;          /* particle density [kg/m^3] (Sec. 3.1) */
    double E, nu;        /* particle Young's modulus [Pa], Poisson ratio (Sec. 3.1) */
    double mu_t, mu_r;   /* particle-particle friction and rolling resistance (Eqs. 6-7) */
    double e_H;          /* gap exponent: 5/4 Hertz, 1 linear (Sec. 2.2) */
    double damp_steps;   /* SPOOK damping time in steps, tau/dt (Sec. 2.2: 4.5) */
    double dt;           /* time step [s] */
    int32_t n_it;        /* Jacobi sweeps per step (Eq. 8) */
    double gravity[3];   /* [m/s^2] */
    double kn_scale;     /* multiplies k_n (1 = paper) */
    double eps_reg;      /* tangential/rolling compliance relative to the normal one */
    double delta_floor;  /* floor on the overlap inside the Hertz Jacobian factor [m] */
    int32_t solver;      /* ORC_JACOBI (Jacobi with mass splitting) or ORC_PGS (coloured
                            projected Gauss-Seidel, the paper's PGS ordered by contact colours) */
    double e_imp;        /* Newton restitution coefficient of the impact stage (Sec. 2.2) */
    double v_imp;        /* impact threshold: contacts approaching faster than this [m/s] are
                            impacts; 0 = no impact stage */
} orc_params;

enum { ORC_JACOBI = 0, ORC_PGS = 1 };

typedef struct orc_geom {
    int32_t type;        /* ORC_PLANE, ORC_BOX, ORC_CYLINDER */
    double c[3];         /* plane: a point on it; box/cylinder: centre */
    double R[9];         /* row-major rotation; column k = local axis k in world.
                            plane normal = local z; cylinder axis = local z */
    double he[3];        /* box: half extents; cylinder: he[0] radius, he[2] half height */
    double v[3], w[3];   /* kinematic velocity of c and angular velocity */
    double E, nu;        /* material of the geometry */
    double mu_t, mu_r;   /* sphere-geometry friction and rolling resistance */
} orc_geom;

typedef struct orc_sim orc_sim;

/* Brute-force detection at the given positions.  Writes up to `cap` contacts as
 * (key_a, key_b, delta): spheres key_a = lower id, key_b = higher id; geometry
 * key_a = sphere id, key_b = -(g+1).  Sorted by (key_a, key_b).  Returns the
 * total number of contacts (may exceed cap). */
int64_t orc_detect(int32_t n, const double* x, const double* r, const int32_t* id,
                   int32_t ng, const orc_geom* g, int64_t cap,
                   int32_t* out_a, int32_t* out_b, double* out_delta);

/* inv_m / inv_I may be NULL (computed from rho and r). */
orc_sim* orc_create(const orc_params* p, int32_t n, const double* x, const double* r,
                    const double* v, const double* w, const int32_t* id,
                    const double* inv_m, const double* inv_I,
                    int32_t ng, const orc_geom* g);
void orc_destroy(orc_sim* s);
/* Load-driven rigid group: the listed primitives translate together as one
 * body of the given mass under a constant external force [N] along the axes
 * whose bit is set in dof (bit 0 x, 1 y, 2 z); along the other axes they keep
 * their prescribed velocity; they do not rotate dynamically.  The group's
 * velocity is an unknown of every step's solve like a particle's (a dynamic
 * motor-free plate, the paper's plate under a normal load F_N, Sec. 3.3).
 * The group starts with the velocity of its first member.  Returns 0, or -1
 * for bad arguments or a primitive already in a group. */
int orc_set_load(orc_sim* s, int32_t count, const int32_t* geoms, double mass, const double force[3],
                 int32_t dof);
/* New external force of the group that primitive g belongs to, from the next
 * step on.  Returns 0, or -1 if g is in no group. */
int orc_set_load_force(orc_sim* s, int32_t g, const double force[3]);
/* Returns 0, or -1 (nothing done) for the PGS solver with load-driven groups. */
int orc_step(orc_sim* s, int32_t nsteps);
/* Colours used by the last step's PGS sweeps (0 for Jacobi). */
int32_t orc_colours(const orc_sim* s);
/* Impacting contacts of the last step (0: no impact stage ran). */
int64_t orc_impacts(const orc_sim* s);
void orc_get_state(const orc_sim* s, double* x, double* v, double* w);
void orc_set_state(orc_sim* s, const double* x, const double* v, const double* w);
void orc_set_geom_velocity(orc_sim* s, int32_t g, const double v[3], const double w[3]);
void orc_get_geom(const orc_sim* s, int32_t g, orc_geom* out);
/* Force and torque (about the geometry centre) of the last step, impulse/dt. */
void orc_get_geom_force(const orc_sim* s, int32_t g, double f[3], double t[3]);
/* Contacts of the last step, sorted by key.  lam7 = world-frame impulses of the
 * contact on body a: (p_n, p_t.x, p_t.y, p_t.z, p_r.x, p_r.y, p_r.z), with the
 * normal pointing from b to a.  Also the overlap.  Returns the count. */
int64_t orc_get_contacts(const orc_sim* s, int64_t cap, int32_t* key_a, int32_t* key_b,
                         double* lam7, double* delta, double* normal);
/* Replace the warm-start store (keys sorted by (a,b)); lam7 as above. */
void orc_set_warmstart(orc_sim* s, int64_t m, const int32_t* key_a, const int32_t* key_b,
                       const double* lam7);
int orc_threads(void);

#ifdef __cplusplus
}
#endif
#endif
