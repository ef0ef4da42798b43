/*
 * hlbm_oracle.h -- plain, slow FP64 CPU oracle of one HLBM time step.
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA path; it is
 * never part of the product path.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library: every formula here is written out
 * again from the paper (Marquardt, Hafen, Krause, "A novel particle
 * decomposition scheme to improve parallel performance of fully resolved
 * particulate flow simulations", arXiv:2312.14172).
 *
 * What it computes (one time step, Algorithm 1 of Sec. 4.2.5 without its two
 * communication rows):
 *   1. momentum exchange (MEA, Eq. hlbm:mea) summed over the cells whose centre
 *      lies inside each particle (Eqs. hydrodynamicforce, hydrodynamictorque);
 *   2. external force: weight minus buoyancy (Sec. 5.1);
 *   3. Newton-Euler update (Eqs. particlemotiontrans, motionrot);
 *   4. particle -> fluid coupling: smooth indicator B (Eq. B), velocity
 *      difference (Eq. hlbm:du), exact-difference source (Eq. kupershtokh);
 *   5. BGK collision (Eqs. collide, bgk, maxbolt) and streaming (Eq. stream)
 *      with two lattices (push into a second array), periodic axes or
 *      half-way bounce-back walls.
 *
 * Readings of passages where the paper is silent or garbled are documented
 * where they are used in hlbm_oracle.c.
 *
 * Parity-pinned functions: every exported function below is checked by the
 * CPU test-suite against closed forms, invariants or brute force (see the
 * comment of each function for its pin).  Nothing here is "parity unpinned"
 * except the whole-model comparison with the paper's experiments, for which
 * the paper prints no numbers.
 *
 * Layout conventions (shared with the C-ABI as an interface, not as code):
 *   populations f[i][z][y][x], x fastest, i in the D3Q19 order listed in
 *   hlbm_oracle.c; lattice units, dx = dt = 1, rho_f = 1; cell centre
 *   (i, j, k) sits at the point (i, j, k).
 */
#ifndef HLBM_ORACLE_H
#define HLBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_Q 19

/* shape codes */
#define ORACLE_SPHERE 0
#define ORACLE_ELLIPSOID 1
#define ORACLE_CUBOID 2
#define ORACLE_CAPSULE 3 /* radius a[0], half-length a[2] of its axis segment (body z) */
#define ORACLE_GRID 4    /* a registered signed-distance grid, its id in a[0] */
#define ORACLE_MAX_GRIDS 64

/* boundary flag bits: a set bit makes that axis bounded by two half-way
 * bounce-back walls; a clear bit makes it periodic. */
#define ORACLE_WALL_X 1
#define ORACLE_WALL_Y 2
#define ORACLE_WALL_Z 4

typedef struct oracle_sim oracle_sim;

/* --- velocity set and equilibrium (Sec. 3.1) --- */
void oracle_velocity_set(int c[ORACLE_Q][3], double w[ORACLE_Q], int opp[ORACLE_Q]);
void oracle_equilibrium(double rho, const double u[3], double feq[ORACLE_Q]);

/* --- geometry (Sec. 3.2) --- */
double oracle_indicator(double d, double eps);
/* signed distance of the body-frame offset r_body from the surface */
double oracle_sdf_body(int shape, const double a[3], const double r_body[3]);
/* rotation matrix (body -> world), row-major, from a unit quaternion (w,x,y,z) */
void oracle_rotation(const double q[4], double R[9]);
/* the inside test of Eq. hydrodynamicforce, taken in FP32 (see .c) */
int oracle_inside_fp32(int shape, const double a[3], const double q[4], const double X[3],
                       const int cell[3], const int n[3], int bc_flags);

/* --- simulation --- */
oracle_sim* oracle_create(int nx, int ny, int nz, double tau, double eps, int bc_flags,
                          const double gravity[3], const double fluid_force[3]);
void oracle_destroy(oracle_sim* s);
/* returns 0 or a negative error (bad argument) */
int oracle_add_particles(oracle_sim* s, int n, const int* shape, const double* a,
                         const double* X, const double* U, const double* omega,
                         const double* quat, const double* rho_p);
int oracle_set_particle_state(oracle_sim* s, const double* X, const double* U,
                              const double* omega, const double* quat);
void oracle_particle_state(const oracle_sim* s, double* X, double* U, double* omega,
                           double* quat, double* F, double* T);
void oracle_get_populations(const oracle_sim* s, double* f);
void oracle_set_populations(oracle_sim* s, const double* f);
void oracle_step(oracle_sim* s, int nsteps);
long oracle_steps_done(const oracle_sim* s);
int oracle_num_particles(const oracle_sim* s);

/* --- single pieces of a step, exposed for the pins --- */
/* MEA force and torque of particle p on the current populations, Eqs.
 * hlbm:mea, hydrodynamicforce, hydrodynamictorque; returns interior cell count */
long oracle_mea(const oracle_sim* s, int p, double F[3], double T[3]);
/* per-cell printed MEA sum at cell x with local particle velocity up */
void oracle_mea_printed_cell(const oracle_sim* s, const int x[3], const double up[3], double Fh[3]);
/* indicator field B(x) = max_p B_p and the winning particle (or -1) */
void oracle_indicator_field(const oracle_sim* s, double* B, int* pid);
/* one collision (no streaming) of the whole lattice into post[19][ncell] */
void oracle_collide_only(const oracle_sim* s, double* post);
/* stream a post-collision field into the lattice (replaces populations) */
void oracle_stream_only(oracle_sim* s, const double* post);
/* Newton-Euler with given total forces and torques (no MEA), for pins */
void oracle_integrate_only(oracle_sim* s, const double* F, const double* T);
/* threads the loops of a step use: omp_get_max_threads() in the -fopenmp
 * build, else 1 */
int oracle_threads(void);

/* --- signed-distance grids (the paper's outlook on other shapes, Sec. 6) ---
 * oracle_add_grid registers n0 x n1 x n2 FP32 samples of a signed distance
 * (x fastest) with spacing h on a body-frame grid centred at the origin, the
 * body's centre of mass, with its principal axes along the grid's.  Returns
 * the grid id (>= 0), or -1 (bad sizes, a non-finite sample, no negative
 * sample, or a boundary sample below eps/2: the indicator must vanish at the
 * grid's faces), or -2 (centroid off the origin by more than h/100, or
 * products of inertia above 1e-3 of the largest moment).  Particles of
 * shape ORACLE_GRID name the id in their first size parameter. */
int oracle_add_grid(oracle_sim* s, int n0, int n1, int n2, double h, const float* values);
/* the grid's distance at a body-frame point (FP64 trilinear; +inf outside) */
double oracle_grid_sdf(const oracle_sim* s, int grid, const double r_body[3]);
/* volume and principal moments per unit density of a registered grid, and
 * its circumscribed and influence radii (V, I0, I1, I2, rc, rinf) */
void oracle_grid_properties(const oracle_sim* s, int grid, double out[6]);
/* the FP32 inside test of a grid particle at a cell (as oracle_inside_fp32) */
int oracle_inside_grid_fp32(const oracle_sim* s, int grid, const double q[4], const double X[3],
                            const int cell[3]);

/* --- contact (an extension: the paper refers to a contact model without
 * stating one, Secs. 2.2 and 3.2; see hlbm_oracle.c) --- */
/* stiffness k (force units) and range zeta (cells) of the repulsion between
 * the enclosing capsules of two particles and between a capsule and a wall;
 * k = 0 switches it off (the default).  Returns 0 or -1 (bad argument). */
int oracle_set_contact(oracle_sim* s, double k, double zeta);
/* contact force and torque on every particle at the current state */
void oracle_contact_forces(const oracle_sim* s, double* F, double* T);

#ifdef __cplusplus
}
#endif
#endif
