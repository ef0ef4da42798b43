/*
 * hlbm.h -- C-ABI of the GB300 HLBM library (libhlbm.so).
 *
 * One time step of the homogenized lattice Boltzmann method (HLBM) for fully
 * resolved particulate flow, as stated in Marquardt, Hafen, Krause,
 * arXiv:2312.14172:
 *   Sec. 3.1  D3Q19 BGK collision (Eqs. collide, bgk, maxbolt, relaxation)
 *             and streaming (Eq. stream);
 *   Sec. 3.2  particle -> fluid coupling through the smooth indicator B
 *             (Eq. B), the velocity difference (Eq. hlbm:du) and the exact
 *             difference source (Eq. kupershtokh); fluid -> particle coupling
 *             through the momentum exchange (Eq. hlbm:mea) summed over the
 *             cells inside each particle (Eqs. hydrodynamicforce,
 *             hydrodynamictorque);
 *   Sec. 2.2  Newton-Euler motion (Eqs. particlemotiontrans, motionrot);
 *   Sec. 4.2.5 the order of one step (Algorithm 1).
 *
 * Conventions for every call:
 *   - Lattice units, dx = dt = 1, reference fluid density 1.  Cell (i, j, k)
 *     has its centre at the point (i, j, k).  An axis is periodic, or bounded
 *     by two half-way bounce-back walls at -1/2 and n - 1/2.
 *   - Populations are exchanged as FP64 values f_i(x) of the post-streaming
 *     state, laid out f[i][z][y][x] (x fastest), with the D3Q19 order
 *       i:  0  1  2  3  4  5  6  7  8  9 10 11 12 13 14 15 16 17 18
 *       cx: 0  1 -1  0  0  0  0  1 -1  1 -1  1 -1  1 -1  0  0  0  0
 *       cy: 0  0  0  1 -1  0  0  1 -1 -1  1  0  0  0  0  1 -1  1 -1
 *       cz: 0  0  0  0  0  1 -1  0  0  0  0  1 -1 -1  1  1 -1 -1  1
 *     and weights 1/3, 1/18 (|c| = 1), 1/36 (|c|^2 = 2).
 *   - Host arrays passed in are read during the call and may be reused when
 *     it returns; host arrays passed out are written before it returns.
 *   - Device memory is owned by the handle.  If the caller passes its own
 *     device buffer to an init call, the library carves all its arrays from
 *     it, never frees it, and the caller must keep it alive until
 *     hlbm_destroy.
 *   - All GPU work is queued on the CUDA stream given at init.  Calls that
 *     return data to the host synchronise that stream.
 *   - Return codes: HLBM_OK (0) or a negative HLBM_ERR_*; hlbm_last_error()
 *     gives a one-line reason.  A failed call leaves the handle usable unless
 *     it returned HLBM_ERR_CUDA.
 *   - Not thread-safe: one host thread at a time per handle.
 */
#ifndef HLBM_H
#define HLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HLBM_OK 0
#define HLBM_ERR_ARG (-1)      /* invalid argument */
#define HLBM_ERR_CUDA (-2)     /* a CUDA call failed */
#define HLBM_ERR_UNSTABLE (-3) /* a non-finite or non-positive density or particle state */
#define HLBM_ERR_CAPACITY (-4) /* a fixed-size work list overflowed: a tile's particle list
                                  (bin_capacity), three particles overlapping at one cell, or
                                  the list of interior cells; hlbm_last_error says which */
#define HLBM_ERR_STATE (-5)    /* call not allowed in the current state */

/* storage of the populations: the deviation f_i - w_i from the weights */
#define HLBM_FP32 0 /* as float */
#define HLBM_FP16 1 /* as half, scaled by 2^fp16_scale_log2 */

/* particle shapes; shape_params holds three numbers per particle */
#define HLBM_SPHERE 0    /* radius r (the other two entries are ignored) */
#define HLBM_ELLIPSOID 1 /* semi-axes a, b, c along the body axes */
#define HLBM_CUBOID 2    /* half-extents a, b, c along the body axes */
#define HLBM_CAPSULE 3   /* radius r, ignored, half-length h of the axis segment
                            along the body z axis: the points within r of it */
#define HLBM_GRID 4      /* a signed-distance grid registered by hlbm_add_grid:
                            its id, ignored, ignored */
#define HLBM_MAX_GRIDS 64

/* boundary flags: a set bit bounds that axis with two bounce-back walls */
#define HLBM_WALL_X 1
#define HLBM_WALL_Y 2
#define HLBM_WALL_Z 4
/* together with HLBM_WALL_Z: the box is one z slab of a larger lattice (see
 * "Sub-domains" below): its z faces bound the lattice like walls, particle
 * centres may lie beyond them, and only the owned planes enter the momentum
 * exchange */
#define HLBM_CUT_Z 8

typedef struct hlbm_ctx* hlbm_handle;

/* one lattice box of a batch */
typedef struct {
  int nx, ny, nz; /* cells per axis, each >= 1 */
  int bc_flags;   /* HLBM_WALL_* bits; clear bits are periodic axes */
} hlbm_box;

/* parameters shared by all boxes of a handle */
typedef struct {
  double tau;             /* BGK relaxation time, Eq. relaxation: tau = 3 nu + 1/2; > 1/2 */
  double eps;             /* width of the smooth boundary of Eq. B (lattice units), > 0 */
  double gravity[3];      /* acceleration g; particle force (rho_p - 1) V g, Sec. 5.1 */
  double fluid_force[3];  /* uniform force density on the fluid (0 for the paper's setups) */
  int precision;          /* HLBM_FP32 or HLBM_FP16 */
  int fp16_scale_log2;    /* HLBM_FP16 only: stored value (f_i - w_i) * 2^s, s in [0, 16] */
  int max_particles;      /* capacity of the particle table over all boxes, >= 0 */
  int bin_capacity;       /* particles per 32x8x8 cell tile seen by the collision; 0 = 64 */
  long long grid_floats;  /* capacity for the samples of signed-distance grids, >= 0 */
} hlbm_params;

/* Fills p with the defaults: tau 0.6, eps 0.5 (Sec. 3.2), no forces, FP32,
 * s = 14, max_particles 0, bin_capacity 0, grid_floats 0. */
void hlbm_default_params(hlbm_params* p);

/* Device bytes that an init call with the same arguments needs; 0 if the
 * arguments are invalid. */
size_t hlbm_required_bytes(int nboxes, const hlbm_box* boxes, const hlbm_params* prm);

/* Creates a handle for one box.  The fluid starts at rest with density 1
 * (f_i = w_i, Sec. 3.1).  cuda_stream: a cudaStream_t (NULL = legacy default
 * stream).  device_buf: NULL to let the library allocate, or a device buffer
 * of at least hlbm_required_bytes() bytes, 256-byte aligned. */
int hlbm_init_lattice(hlbm_handle* out, int nx, int ny, int nz, int bc_flags,
                      const hlbm_params* prm, void* cuda_stream, void* device_buf,
                      size_t device_buf_bytes);

/* Creates a handle for a batch of independent boxes advanced together: one
 * launch per kernel per step covers all boxes.  Same rules as
 * hlbm_init_lattice. */
int hlbm_init_batch(hlbm_handle* out, int nboxes, const hlbm_box* boxes, const hlbm_params* prm,
                    void* cuda_stream, void* device_buf, size_t device_buf_bytes);

/* Registers a signed-distance grid, the voxelised form of the paper's
 * outlook on particle shapes beyond spheres (Sec. 6): values[(k ny + j) nx
 * + i] (FP32, host) is the signed distance (negative inside) at the
 * body-frame point ((i - (nx - 1)/2) h, (j - (ny - 1)/2) h, (k - (nz - 1)/2) h),
 * nx, ny, nz >= 2, spacing h > 0.  Between samples the distance is the
 * trilinear blend of the eight corners of the grid cell holding the point,
 * and a cell centre is inside a grid particle when the FP32 blend (operation
 * order as the library's inside test states) is negative.  The body frame
 * must be the principal frame about the centre of mass: volume and second
 * moments are summed over 4 x 4 x 4 sub-cells of every grid cell (midpoint
 * rule on the blend), and a centroid off the origin by more than h/100 or
 * products of inertia above 1e-3 of the largest moment are refused.  The
 * samples on the grid's faces must be >= eps/2 (the indicator of Eq. B must
 * vanish there), at least one must be negative, and the body's circumscribed
 * radius (the farthest corner of the grid cells with a negative corner) may
 * be at most 30 cells.  The samples are copied (the handle's grid_floats
 * bounds their total).  Writes the grid id (0, 1, ...) to *grid_id.
 * HLBM_ERR_ARG for refused grids, HLBM_ERR_CAPACITY when grid_floats or
 * HLBM_MAX_GRIDS is exceeded. */
int hlbm_add_grid(hlbm_handle h, int nx, int ny, int nz, double spacing, const float* values, int* grid_id);

/* Adds n particles (Sec. 2.2), allowed only before the first step
 * (HLBM_ERR_STATE afterwards).  Arrays (host, row-major):
 *   box_id[n]      box of each particle (NULL = box 0)
 *   shape[n]       HLBM_SPHERE / HLBM_ELLIPSOID / HLBM_CUBOID / HLBM_CAPSULE /
 *                  HLBM_GRID (shape_params: the grid id, then two ignored)
 *   shape_params[3n], X[3n] centre of mass, U[3n] velocity (NULL = 0),
 *   omega[3n] angular velocity (NULL = 0), quat[4n] orientation (w,x,y,z,
 *   body -> world, normalised here; NULL = identity), rho_p[n] density.
 * Mass and inertia follow from the analytic volume and rho_p.  Rejected
 * (HLBM_ERR_ARG): non-finite or non-positive sizes or densities, a centre
 * outside the box on a wall axis, or a particle whose influence sphere (the
 * radius beyond which B of Eq. B vanishes, plus 2 cells) spans half a
 * periodic axis or more.  The influence radius is r + eps/2 for spheres, the
 * circumscribed radius + eps/2 for cuboids and a_max (1 + eps / (2 a_min))
 * for ellipsoids, h + r + eps/2 for capsules, and for grids the farthest
 * corner of the grid cells with a corner below eps/2.  The circumscribed
 * radius may be at most 30 cells. */
int hlbm_add_particles(hlbm_handle h, int n, const int* box_id, const int* shape,
                       const double* shape_params, const double* X, const double* U,
                       const double* omega, const double* quat, const double* rho_p);

/* Overwrites the motion state of all particles (any of the pointers may be
 * NULL to keep that field).  Arrays as in hlbm_add_particles.  The values are
 * checked and staged on the host, the upload is queued on the stream and the
 * call returns without waiting for it: the arrays may be reused at once.
 * A new position or orientation changes the cells inside the particles, so
 * the next step takes the bounding-box momentum exchange; positions (and the
 * orientations of non-spheres) that are not given, or that equal bit for bit
 * the state hlbm_particle_state returned after the current step, keep the
 * momentum exchange from the recorded moments.  HLBM_ERR_ARG (nothing
 * changed) for a non-finite position or a zero or non-finite quaternion. */
int hlbm_set_particle_state(hlbm_handle h, const double* X, const double* U, const double* omega,
                            const double* quat);

/* Replaces the uniform body-force density on the fluid (hlbm_params
 * fluid_force, f[3] in lattice units) from the next step on, e.g. to hold a
 * periodic suspension at zero net flow while it settles.  Waits for the
 * stream when the force changes.  HLBM_ERR_ARG for a NULL or non-finite f
 * (nothing changed). */
int hlbm_set_fluid_force(hlbm_handle h, const double f[3]);

/* Contact between particles (an extension; the paper counts contact among
 * the acting forces of Sec. 2.2 without stating a model, and its own runs
 * have none, Sec. 3.2).  Each particle is enclosed by a capsule: a sphere and
 * a capsule by themselves, an ellipsoid by the capsule along its longest
 * semi-axis a_k with radius the larger other semi-axis r and half-length
 * a_k - r, a cuboid by the capsule along its longest half-extent h_k with
 * radius |(h_i, h_j)| and half-length h_k, a grid particle by the sphere of
 * its circumscribed radius.  Two capsules of one box whose
 * axis segments come closest at p_i, p_j (minimum image) with surface gap
 * delta = |p_i - p_j| - r_i - r_j < zeta repel each other along p_i - p_j
 * with the force k ((zeta - delta) / zeta)^2, particle i taking the torque
 * (p_i - X_i) x F_i; a wall pushes the segment end nearest to it the same
 * way (delta its distance to the wall minus r).  The forces enter the
 * Newton-Euler update with the hydrodynamic force and the weight; the F and
 * T that hlbm_particle_state reports stay the hydrodynamic ones.  k >= 0 in
 * lattice force units (0, the default, switches contact off), zeta > 0
 * cells; from the next step on (waits for the stream when they change).
 * Each particle is tested against every other particle of the handle (one
 * warp per particle): meant for boxes of up to a few thousand particles.
 * HLBM_ERR_ARG for a negative or non-finite k or a zeta <= 0. */
int hlbm_set_contact(hlbm_handle h, double k, double zeta);

/* Queues nsteps >= 0 time steps (Algorithm 1: momentum exchange, external
 * force, Newton-Euler update, particle work lists, EDM coupling, collision
 * and streaming) on the stream and returns without waiting.  Errors found by
 * the GPU are reported by the next call that synchronises. */
int hlbm_step(hlbm_handle h, int nsteps);

/* Waits for the stream and returns HLBM_OK or the error the GPU flagged
 * (HLBM_ERR_UNSTABLE, HLBM_ERR_CAPACITY); the flags are then cleared. */
int hlbm_sync(hlbm_handle h);

/* Copies the particle state after the last step to host arrays (any may be
 * NULL): X, U, omega [3n], quat [4n], and the hydrodynamic force F and
 * torque T [3n] of Eqs. hydrodynamicforce / hydrodynamictorque measured in the
 * last step (weight and buoyancy not included).  Synchronises; returns like
 * hlbm_sync. */
int hlbm_particle_state(hlbm_handle h, double* X, double* U, double* omega, double* quat,
                        double* F, double* T);

/* Copies the post-streaming populations f_i(x) of box `box` to / from a host
 * array of 19 * nx * ny * nz doubles (layout above).  Set converts to the
 * storage precision.  Both synchronise. */
int hlbm_get_populations(hlbm_handle h, int box, double* host_f);
int hlbm_set_populations(hlbm_handle h, int box, const double* host_f);

/* Total mass deviation and momentum of box `box`, the moments of Sec. 3.1
 * summed over its cells: out[0] = sum_x (rho(x) - 1), out[1..3] =
 * sum_x sum_i c_i f_i(x), from the post-streaming populations as stored,
 * summed in FP64 in a fixed order.  Synchronises.  HLBM_ERR_ARG for a bad
 * box or a NULL out. */
int hlbm_fluid_momentum(hlbm_handle h, int box, double out[4]);

int hlbm_num_particles(hlbm_handle h);
long long hlbm_steps_done(hlbm_handle h);

/* Launch shape of the collision kernel: each thread block covers a brick of
 * 32 x tile_y x tile_z cells, tile_y and tile_z in {1, 2, 4, 8}, with
 * cells_x = 1 or 2 x-adjacent cells per thread (32 x tile_y or 16 x tile_y
 * threads); cells_x = 2 is the default.  Both compute the same step; their
 * results differ by FP32 rounding order only. */
int hlbm_set_launch(hlbm_handle h, int tile_y, int tile_z, int cells_x);
int hlbm_get_launch(hlbm_handle h, int* tile_y, int* tile_z, int* cells_x);

/* How the momentum exchange (Eq. hlbm:mea) of a step is computed:
 *   HLBM_MEA_KERNEL   from the populations alone, by a kernel that walks the
 *                     bounding box of each particle (default);
 *   HLBM_MEA_MOMENTS  the collision of the previous step lists the cells
 *                     inside particles with the mass and momentum their
 *                     post-collision populations carry away; the momentum
 *                     exchange is then, per listed cell, the momentum gained
 *                     minus u_p times the mass gained, from the arrivals alone.
 *                     The bounding-box kernel still runs on the first step
 *                     after any change of state.  Needs max_particles > 0; the
 *                     list is split into 64 stripes that the collision's
 *                     blocks fill in turn, each holding 1/64 of half the
 *                     lattice's cells (at least 4096 entries);
 *                     HLBM_ERR_CAPACITY when one overflows.
 * Both give the same force and torque up to FP32 summation order. */
#define HLBM_MEA_KERNEL 0
#define HLBM_MEA_MOMENTS 1
int hlbm_set_mea_mode(hlbm_handle h, int mode);
int hlbm_get_mea_mode(hlbm_handle h);

/* Times every momentum-exchange mode and launch shape (tile_y, tile_z,
 * cells_x; cells_x = 2 only with tile_y >= 2) on about 20 ms of steps
 * (nsteps to 4 nsteps) from the current state, times the three fastest once
 * more and keeps the fastest; writes the chosen shape and its time per step
 * in ms (any pointer may be NULL).  The run is left where it was: the
 * handle's whole device state is copied to a temporary device buffer (of
 * the handle's size; allocated and freed by this call) before the timed
 * steps and copied back after them.  The choice is kept for the life of the
 * process per (GPU model and SM count, boxes, precision, particle count,
 * grids, contact on or off): a later call with the same key applies it
 * without timing. */
int hlbm_autotune(hlbm_handle h, int nsteps, int* tile_y, int* tile_z, int* cells_x, float* ms_per_step);

/* Runs nsteps steps with each kernel launched on its own, bracketed by CUDA
 * events on the handle's stream, and writes the mean time per launch in ms:
 * ms[0] momentum exchange, ms[1] contact (when on), Newton-Euler and work
 * lists, ms[2] collision and streaming.  Synchronises. */
int hlbm_kernel_times(hlbm_handle h, int nsteps, float ms[3]);

/* Writes to *n the number of (cell, particle) pairs whose cell centre lies
 * inside the particle (Sec. 3.2, the cells the sums of Eqs.
 * hydrodynamicforce and hydrodynamictorque run over) at the current
 * particle state: the entries the last collision listed in the moments
 * mode, i.e. the work of the next step's momentum exchange.  A cell inside
 * two particles counts twice.  Synchronises.  HLBM_ERR_STATE outside the
 * moments mode or before the first step after a change of state. */
int hlbm_interior_cells(hlbm_handle h, long long* n);

/* Snapshots (checkpoint and restart; not part of the paper's method).
 *
 * A snapshot holds the whole state the next step reads: the registered
 * distance grids, the populations as
 * stored (the handle's block layout and precision, bit for bit), the FP64
 * particle table with shapes and box ids, the step count (hence the AA
 * parity), the fluid force, the momentum-exchange mode and, when the next
 * step takes its momentum exchange from the recorded moments, the list of
 * interior cells the last collision wrote.  Launch shape and tuning are not
 * part of it.  The layout is host byte order with fixed-width fields; it is
 * meant for the same library on machines of the same byte order.
 *
 * hlbm_checkpoint_bytes: *bytes = the size of a snapshot of the current
 * state.  Synchronises; returns the error the GPU flagged, if any (no
 * snapshot of a failed state).
 *
 * hlbm_save: writes the snapshot into the caller's host buffer buf of
 * `bytes` >= hlbm_checkpoint_bytes (pageable or pinned memory; the library
 * keeps no reference).  Synchronises.  HLBM_ERR_ARG for a NULL or too small
 * buffer.
 *
 * The contact parameters (hlbm_set_contact) travel with the snapshot.
 *
 * hlbm_load: restores a snapshot into a handle created with the same boxes,
 * precision, fp16 scale, tau, eps and gravity and max_particles at least the
 * snapshot's particle count, before its first step and before any particle
 * is added (HLBM_ERR_STATE otherwise).  The next hlbm_step continues the
 * saved run exactly as the saving handle would.  HLBM_ERR_ARG (nothing
 * queued) for a NULL, truncated or foreign buffer or one that does not fit
 * the handle; the particles go through hlbm_add_particles' checks.
 * Synchronises. */
int hlbm_checkpoint_bytes(hlbm_handle h, size_t* bytes);
int hlbm_save(hlbm_handle h, void* buf, size_t bytes);
int hlbm_load(hlbm_handle h, const void* buf, size_t bytes);

/* Momentum exchange without device allocation.
 *
 * The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory -- a particle code running inside another
 * framework's memory pool or arena, or one whose device memory is all handed
 * to it by its host application -- and still want the force and torque of
 * Eqs. hlbm:mea / hydrodynamicforce / hydrodynamictorque on populations they
 * own.  It computes what the momentum-exchange kernel of hlbm_step computes
 * (bounding-box form, FP32 cell sums, FP64 partials added in plane order) for
 * one lattice box, without a handle.
 *
 * Every intermediate lives in one file-scope device array of about 3.3 MB
 * that every GPU loading the library holds until the process exits; the
 * call allocates nothing (no cudaMalloc, no library allocator).  The first
 * call on a device (and the first in each new CUDA context on it, e.g.
 * after cudaDeviceReset) looks up that array's device address, so make it
 * before any stream capture.  All calls on a device share the array: calls
 * whose GPU work overlaps (other streams, other host threads) race; order
 * them on one stream.  The array keeps the last call's contents; the call
 * clears what must start at zero.
 *
 *   f            device: 19 planes of `plane` elements, FP32 (f - w) or FP16
 *                (f - w) * 2^fp16_scale_log2, cell (x, y, z) of plane i at
 *                i * plane + (z ny + y) nx + x, in the AA layout of `parity`
 *                (0: slot i of x holds f_i(x); 1: slot ibar of x - c_i)
 *   nx, ny, nz, bc_flags   the box as in hlbm_box
 *   n            particles, 0 <= n <= HLBM_NOALLOC_MAX_PARTICLES
 *   shape, shape_params, X, U, omega, quat   device arrays laid out as in
 *                hlbm_add_particles (U, omega, quat may be NULL)
 *   F, T         device outputs [3n]: hydrodynamic force and torque.  A
 *                particle is checked as hlbm_add_particles checks it and gets
 *                NaN force and torque when its shape code is unknown or
 *                HLBM_GRID (grids belong to a handle), a size
 *                is non-finite or <= 0, its quaternion is zero or non-finite,
 *                a centre or velocity component is non-finite, its
 *                circumscribed radius r_c exceeds 30 cells, its centre lies
 *                outside (-1/2, n - 1/2) on a wall axis, or 2 (r_c + 2) >= n
 *                on a periodic axis.  On a periodic axis any finite centre is
 *                taken modulo n (the torque arm is the minimum image).
 *   cuda_stream  the stream all work is queued on; the call does not wait
 * Returns HLBM_OK, HLBM_ERR_ARG (n out of range, bad lattice arguments, NULL
 * pointer) or HLBM_ERR_CUDA. */
#define HLBM_NOALLOC_MAX_PARTICLES 1024
int hlbm_mea_noalloc(const void* f, long long plane, int nx, int ny, int nz, int bc_flags,
                     int precision, int fp16_scale_log2, int parity, int n, const int* shape,
                     const double* shape_params, const double* X, const double* U,
                     const double* omega, const double* quat, double* F, double* T,
                     void* cuda_stream);

/* Sub-domains: z slabs of one lattice on several handles (one GPU each, or
 * several on one GPU), the single-GPU building blocks of the paper's domain
 * decomposition with its particle decomposition (Secs. 4.2.2-4.2.4).
 *
 * A slab of planes [z0, z1) of a global lattice is a box of z1 - z0 + 2
 * planes with HLBM_WALL_Z | HLBM_CUT_Z: local plane 0 and the last plane are
 * ghost copies of the neighbours' boundary planes, hlbm_set_owned_planes(h,
 * box, 1, z1 - z0 + 1) marks the rest as owned (a slab on a wall of the
 * lattice has no ghost plane on that side: its box's z wall is the wall).  Each slab holds copies of
 * the particles whose influence reaches it (positions in its local frame,
 * the periodic image nearest to it).  A step of the whole lattice is then:
 *   1. before an odd step (steps done is odd), every ghost plane receives
 *      the neighbour's boundary plane's slots that cross the face
 *      (hlbm_plane_slots: the lower ghost the slots with c_z = -1 of the
 *      lower neighbour's top owned plane, the upper ghost the slots with
 *      c_z = +1 of the upper neighbour's bottom owned plane);
 *   2. hlbm_step_forces on every slab: its partial momentum exchange
 *      (Eq. hlbm:mea over its owned cells only) per particle copy;
 *   3. the partial forces and torques of a particle are summed (in the paper
 *      by the particle's owner, from the slabs its circumscribed sphere
 *      reaches) and the totals are handed back to every slab holding it;
 *   4. hlbm_step_with_forces on every slab: external force, Newton-Euler
 *      update with those totals, coupling, collision and streaming;
 *   5. after an odd step, every owned boundary plane takes back the slots
 *      the neighbour's cells wrote into their ghost copy of it (the bottom
 *      owned plane the slots with c_z = +1 of the lower neighbour's upper
 *      ghost, the top owned plane the slots with c_z = -1 of the upper
 *      neighbour's lower ghost).
 * Every copy of a particle integrates the same totals, so the copies stay
 * identical and the lattice evolves as one box would. */

/* Owned planes [z_lo, z_hi) of a box with HLBM_CUT_Z; the other planes are
 * ghosts whose cells the momentum exchange leaves out.  Synchronises.
 * HLBM_ERR_ARG for a box without HLBM_CUT_Z or an empty or out-of-box
 * range. */
int hlbm_set_owned_planes(hlbm_handle h, int box, int z_lo, int z_hi);

/* Copies the five stored slots {i : c_z of i = dir} (dir = +1 or -1; in
 * increasing i) of every cell of plane z of box `box`, as stored (storage
 * precision, FP32 or FP16 deviations), to (put = 0) or from (put = 1) the
 * host buffer of 5 * nx * ny values laid out [slot][y][x].  These are the
 * populations that cross a z face in the in-place (AA) storage.
 * Synchronises.  HLBM_ERR_ARG for bad arguments. */
int hlbm_plane_slots(hlbm_handle h, int box, int z, int dir, void* host, int put);

/* A step split at the momentum exchange (Algorithm 1's "communicate surface
 * forces" row).  hlbm_step_forces runs the momentum exchange of the next
 * step and writes each particle's hydrodynamic force and torque [3n] (host)
 * over the cells this handle owns; synchronises.  hlbm_step_with_forces
 * takes the totals F, T [3n] (host) in their place and runs the rest of the
 * step (contact when on, external force, Newton-Euler update, work lists,
 * coupling, collision and streaming); synchronises.  hlbm_step refuses
 * while a split step is open (HLBM_ERR_STATE), and so does a second
 * hlbm_step_forces. */
int hlbm_step_forces(hlbm_handle h, double* F, double* T);
int hlbm_step_with_forces(hlbm_handle h, const double* F, const double* T);

/* One-line description of the last error on this handle (or of the last
 * failed init when h is NULL). */
const char* hlbm_last_error(hlbm_handle h);

/* Frees the handle and the device memory it allocated. */
void hlbm_destroy(hlbm_handle h);

#ifdef __cplusplus
}
#endif
#endif
