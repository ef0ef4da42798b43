// hlbm_internal.cuh -- device data layout and kernel launchers of libhlbm.
//
// HBM layout of one handle (all arrays carved from one device buffer):
//   populations   blocked structure of arrays: the cells of every row are
//                 grouped in blocks of VB = 32 consecutive x (the last block
//                 of a row padded), and block B holds its Q slots one after
//                 the other, VB values each: slot i of cell x of block B is
//                 element B * Q * VB + i * VB + (x & 31).  Blocks run x-block
//                 fastest, then y, then z, box after box (box b from block
//                 box.blk_off).  All 19 slots of 32 cells are one contiguous
//                 run of 19 * 32 values, and every slot of a cell is an
//                 immediate offset from the cell's slot 0.  Storage is the
//                 deviation f_i - w_i (times 2^s for half).  In-place AA
//                 pattern: after an even number of steps slot i of cell x
//                 holds f_i(x); after an odd number slot ibar of cell x - c_i
//                 holds f_i(x) (or slot i of x when x - c_i lies beyond a wall).
//   particles     FP64 structure of arrays, field-major (PF_* below).
//   records       one 128-byte FP32 record per particle (Rec), rebuilt after
//                 every Newton-Euler update, read by the collision and the
//                 momentum exchange.
//   bins          two alternating sets of per-tile particle lists (tile =
//                 32 x 8 x 8 cells): count[tile] and ids[tile * cap + k].
//   status        one int of error flags (ST_*).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace hlbm {

constexpr int Q = 19;
constexpr int TILE_X = 32, TILE_Y = 8, TILE_Z = 8;  // particle-bin tile

// D3Q19 (Sec. 3.1) in this library's order; opposite of i >= 1 is i +- 1
__host__ __device__ constexpr int cx(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr double wq(int i) {
  return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Division of an unsigned 32-bit n by a divisor d >= 1 fixed at set-up, with
// one high multiply (Granlund and Montgomery 1994, the unsigned case of
// their Fig. 4.1): with l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1
// and t = mulhi(m, n), n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0),
// exact for every n.
struct FastDiv {
  unsigned m;
  int s1, s2;
};
inline FastDiv make_fastdiv(unsigned d) {
  int l = 0;
  while ((1ull << l) < d) ++l;
  FastDiv f;
  f.m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 1 ? l - 1 : 0;
  return f;
}
__device__ __forceinline__ unsigned fast_div(unsigned n, const FastDiv& f) {
  const unsigned t = __umulhi(f.m, n);
  return (t + ((n - t) >> f.s1)) >> f.s2;
}

struct BoxDesc {
  int nx, ny, nz, bc;        // bc: bit a set = walls on axis a; BC_CUT_Z: see below
  int ntx, nty, ntz;         // bin tiles per axis (ntx = storage blocks per row)
  int own_lo, own_hi;        // owned z planes [own_lo, own_hi) of a BC_CUT_Z box
  FastDiv div_x, div_y;      // division by nx and by ny
  long long cell_off;        // first cell of the box in the global cell numbering
  long long tile_off;        // first bin tile of the box
  long long blk_off;         // first storage block of the box
};

// coordinates of cell c (c < nx ny nz) of a box
__device__ __forceinline__ void cell_coords(const BoxDesc& bd, unsigned c, int& x, int& y, int& z) {
  const unsigned r = fast_div(c, bd.div_x);
  const unsigned q = fast_div(r, bd.div_y);
  x = (int)(c - r * (unsigned)bd.nx);
  y = (int)(r - q * (unsigned)bd.ny);
  z = (int)q;
}

// A box with BC_CUT_Z (set together with the z-wall bit) is one z slab of a
// larger lattice: its z faces bound the lattice as walls do (only its ghost
// planes meet them), particle centres may lie beyond them, and only the
// cells of the owned planes [own_lo, own_hi) enter the momentum exchange.
constexpr int BC_CUT_Z = 8;

// resident blocks per SM of the bounding-box momentum exchange (64
// registers): the walk is latency-bound, and more resident blocks beat the
// spills this costs
#ifndef HLBM_MEA_MINBLOCKS
#define HLBM_MEA_MINBLOCKS 8
#endif
constexpr int MEA_MINBLOCKS = HLBM_MEA_MINBLOCKS;
__host__ __device__ __forceinline__ bool owned_plane(const BoxDesc& bd, int z) {
  return !(bd.bc & BC_CUT_Z) || (z >= bd.own_lo && z < bd.own_hi);
}

// blocked population storage (layout above)
constexpr int VB = 32;       // cells per storage block (= TILE_X)
constexpr int QVB = Q * VB;  // values per storage block

// storage block of cell (x, y, z) of a box, and the element of its slot 0
__host__ __device__ __forceinline__ long long block_of(const BoxDesc& bd, int x, int y, int z) {
  return bd.blk_off + ((long long)z * bd.ny + y) * bd.ntx + (x >> 5);
}
__host__ __device__ __forceinline__ long long elem_of(const BoxDesc& bd, int x, int y, int z) {
  return block_of(bd, x, y, z) * QVB + (x & 31);
}

// FP64 particle table fields (each an array of `cap` doubles).  PF_IM and
// PF_II hold 1/m and 1/I, PF_IA holds fp32(1/a_j) (exact in a double);
// PF_FC and PF_TC the contact force and torque of the step (when contact is
// on).
enum {
  PF_X = 0, PF_U = 3, PF_W = 6, PF_Q = 9, PF_F = 13, PF_T = 16,
  PF_M = 19, PF_V = 20, PF_I = 21, PF_RHO = 24, PF_A = 25, PF_RC = 28, PF_RINF = 29,
  PF_IM = 30, PF_II = 31, PF_IA = 34, PF_FC = 37, PF_TC = 40,
  PF_COUNT = 43
};

// the momentum-exchange kernel gives every z-plane of a particle's bounding
// box its own thread block; a particle spans at most this many planes
// (circumscribed radius <= 30 cells)
constexpr int MAX_PLANES = 64;

// stripes of the list of interior cells (a power of two)
constexpr int ILIST_STRIPES = 64;

// Signed-distance grids (shape 4): FP32 samples of a body-frame signed
// distance, point (i, j, k) at ((i - half_0) h, (j - half_1) h, (k - half_2) h)
// with half_j = (n_j - 1) / 2, x fastest, starting at element `off` of the
// handle's grid array.
constexpr int MAX_GRIDS = 64;
struct GridDesc {
  int n[3];
  float ih;       // fp32(1 / h)
  float half[3];  // fp32((n_j - 1) / 2)
  // a capsule about the body z axis (half-length in_h, squared radius in_r2;
  // in_r2 < 0: none) every grid cell of which has all its corners below
  // -(eps/2 + 1e-3): there B = 1 and the centre is inside, and the coupling
  // takes the distance in_d (below -(eps/2 + 1e-3)) without blending
  float in_h, in_r2, in_d;
  long long off;
};
struct GridSet {
  const GridDesc* desc;  // MAX_GRIDS entries
  const float* vals;
};

// The blend of the grid at body offset b, every operation rounded on its own
// in this order (the FP32 inside test; the oracle rounds the same steps):
//   x_j = b_j * ih + half_j; outside [0, n_j - 1]: +inf
//   i_j = min(floor(x_j), n_j - 2), t_j = x_j - i_j
//   lerp(a, b, t) = a + t * (b - a) along x (four), then y (two), then z.
__device__ __forceinline__ float grid_blend_rn(const GridDesc& g, const float* v, const float b[3]) {
  float t[3];
  int i0[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float x = __fadd_rn(__fmul_rn(b[j], g.ih), g.half[j]);
    if (!(x >= 0.0f && x <= (float)(g.n[j] - 1))) return __int_as_float(0x7f800000);
    const int i = min((int)floorf(x), g.n[j] - 2);
    i0[j] = i;
    t[j] = __fsub_rn(x, (float)i);
  }
  const float* c = v + g.off + ((long long)i0[2] * g.n[1] + i0[1]) * g.n[0] + i0[0];
  const long long sy = g.n[0], sz = (long long)g.n[0] * g.n[1];
  auto lerp = [](float a, float b_, float tt) { return __fadd_rn(a, __fmul_rn(tt, __fsub_rn(b_, a))); };
  const float e00 = lerp(c[0], c[1], t[0]);
  const float e01 = lerp(c[sy], c[sy + 1], t[0]);
  const float e10 = lerp(c[sz], c[sz + 1], t[0]);
  const float e11 = lerp(c[sz + sy], c[sz + sy + 1], t[0]);
  const float f0 = lerp(e00, e01, t[1]);
  const float f1 = lerp(e10, e11, t[1]);
  return lerp(f0, f1, t[2]);
}

// FP32 coupling record of one particle (128 bytes)
struct __align__(16) Rec {
  float xh[3], xl[3];  // centre as float pair: X = xh + xl
  float u[3], w[3];    // velocity, angular velocity
  float M[9];          // rotation body -> world, row-major; a sphere's
                       // first four: its collision bounds (SPH_* below)
  float a[3];          // radius / semi-axes / half-extents / capsule (r, r, h);
                       // a grid's circumscribed radius
  float ia[3];         // fp32(1 / a_j) (ellipsoid inside test)
  float rinf2;         // square of a radius beyond which B = 0
  float in2;           // fp32(r * r) (sphere and capsule inside tests); a
                       // grid particle: its grid id (int bits)
  int shape;
  int box;
  int pid;
};
static_assert(sizeof(Rec) == 128, "record size");
// a sphere's record: in2 * 0.99999 and in2 * 1.00001 (below / above them the
// centre-inside decision needs no exact test), (a - eps/2)^2 (-1 when
// a <= eps/2) and (a + eps/2)^2 (B is 1 within, 0 beyond), all FP32
enum { SPH_IN_LO = 0, SPH_IN_HI = 1, SPH_R2_IN = 2, SPH_R2_OUT = 3 };

// The moments-mode momentum exchange adds its per-cell FP32 terms as 64-bit
// integers in units of 2^-ACC_FRAC_BITS: integer sums do not depend on the
// order in which the cells arrive, so a run is reproducible bit for bit.  A
// term is rounded by at most 2^-45 and a particle's sum must stay below 2^19
// in magnitude (forces and torques of lattice flows are many orders smaller).
constexpr int ACC_FRAC_BITS = 44;

// status flags: ST_CAPACITY a tile's particle list is full; ST_OVERLAP three
// particles hold one cell (the list of interior cells takes two per cell);
// ST_LIST_FULL a stripe of the list of interior cells is full
enum { ST_UNSTABLE = 1, ST_CAPACITY = 2, ST_LEFT_DOMAIN = 4, ST_INTERNAL = 8, ST_OVERLAP = 16, ST_LIST_FULL = 32 };

// neighbour index helper: per-axis neighbour offsets; -1 marks a node beyond
// a wall (only possible when WALLS)
template <bool WALLS>
struct Nbr {
  int xm, xp, ym, yp, zm, zp;  // neighbour coordinates (x) or row/plane offsets (y, z)
  int x, y, z;                 // own coordinate and row/plane offsets
  __device__ __forceinline__ int at(int dx, int dy, int dz) const {
    const int a = dx < 0 ? xm : (dx > 0 ? xp : x);
    const int b = dy < 0 ? ym : (dy > 0 ? yp : y);
    const int c = dz < 0 ? zm : (dz > 0 ? zp : z);
    if (WALLS && (a < 0 || b < 0 || c < 0)) return -1;
    return a + b + c;
  }
};

template <bool WALLS>
__device__ __forceinline__ Nbr<WALLS> make_nbr(const BoxDesc& bd, int x, int y, int z);

// neighbours in the blocked storage: at() returns the element of slot 0 of
// the neighbour (slot i is VB * i further), or -1 beyond a wall
struct NbrB {
  long long xm, xp, x;  // x terms: (x >> 5) * QVB + (x & 31)
  long long ym, yp, y;  // y terms: y * ntx * QVB
  long long zm, zp, z;  // z terms incl. the box's first block
  __device__ __forceinline__ long long at(int dx, int dy, int dz) const {
    const long long a = dx < 0 ? xm : (dx > 0 ? xp : x);
    const long long b = dy < 0 ? ym : (dy > 0 ? yp : y);
    const long long c = dz < 0 ? zm : (dz > 0 ? zp : z);
    if (a < 0 || b < 0 || c < 0) return -1;
    return a + b + c;
  }
};

__device__ __forceinline__ NbrB make_nbr_blocked(const BoxDesc& bd, int x, int y, int z) {
  NbrB n;
  const int nx = bd.nx, ny = bd.ny, nz = bd.nz;
  const bool wx = bd.bc & 1, wy = bd.bc & 2, wz = bd.bc & 4;
  const long long row = (long long)bd.ntx * QVB, pln = row * ny, base = bd.blk_off * QVB;
  auto xt = [](int v) { return (long long)(v >> 5) * QVB + (v & 31); };
  n.x = xt(x);
  n.xm = x > 0 ? xt(x - 1) : (wx ? -1 : xt(nx - 1));
  n.xp = x < nx - 1 ? xt(x + 1) : (wx ? -1 : xt(0));
  n.y = y * row;
  n.ym = y > 0 ? (y - 1) * row : (wy ? -1 : (ny - 1) * row);
  n.yp = y < ny - 1 ? (y + 1) * row : (wy ? -1 : 0);
  n.z = base + z * pln;
  n.zm = z > 0 ? base + (z - 1) * pln : (wz ? -1 : base + (nz - 1) * pln);
  n.zp = z < nz - 1 ? base + (z + 1) * pln : (wz ? -1 : base);
  return n;
}

// neighbour offsets in global cell indices (the box's first cell added):
// at() returns the global index, or a negative value beyond a wall
template <bool WALLS>
__device__ __forceinline__ Nbr<WALLS> make_nbr_global(const BoxDesc& bd, int x, int y, int z) {
  Nbr<WALLS> n = make_nbr<WALLS>(bd, x, y, z);
  const int off = (int)bd.cell_off;
  n.z += off;
  n.zm = n.zm < 0 ? n.zm : n.zm + off;
  n.zp = n.zp < 0 ? n.zp : n.zp + off;
  return n;
}

template <bool WALLS>
__device__ __forceinline__ Nbr<WALLS> make_nbr(const BoxDesc& bd, int x, int y, int z) {
  Nbr<WALLS> n;
  const int nx = bd.nx, ny = bd.ny, nz = bd.nz, nxy = nx * ny;
  const bool wx = WALLS && (bd.bc & 1), wy = WALLS && (bd.bc & 2), wz = WALLS && (bd.bc & 4);
  n.x = x;
  n.y = y * nx;
  n.z = z * nxy;
  n.xm = x > 0 ? x - 1 : (wx ? -1 : nx - 1);
  n.xp = x < nx - 1 ? x + 1 : (wx ? -1 : 0);
  n.ym = y > 0 ? (y - 1) * nx : (wy ? -1 : (ny - 1) * nx);
  n.yp = y < ny - 1 ? (y + 1) * nx : (wy ? -1 : 0);
  n.zm = z > 0 ? (z - 1) * nxy : (wz ? -1 : (nz - 1) * nxy);
  n.zp = z < nz - 1 ? (z + 1) * nxy : (wz ? -1 : 0);
  return n;
}


// Programmatic dependent launch: a step's kernels, captured in one graph,
// are launched so that the next one is scheduled while the current one
// runs; each waits for its predecessor's results before reading them.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            bool pdl, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? attr : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

struct LbmArgs {
  int pdl;                  // launch with programmatic dependent launch (host side only)
  int nsm;                  // SMs of the device (host side only)
  // blocks at the end of the grid (about its last wave) that let the next
  // kernel launch as soon as they start; every earlier block does so when it
  // ends, so that the next kernel's blocks, which wait for this grid to
  // finish, take no SM room this grid's remaining blocks still need
  long long pdl_tail;
  void* f;                  // populations, blocked layout (float* or __half*)
  long long ncell;          // cells of all boxes (global cell numbering)
  const BoxDesc* boxes;
  int nboxes;
  int sub_y, sub_z;         // brick per block: 32 x sub_y x sub_z cells
  int cells_x;              // cells per thread along x: 1, or 2 (every box has an even nx)
  int nsub;                 // bricks per bin tile = (8/sub_y)*(8/sub_z)
  long long nbricks;        // total bricks (grid size)
  // bricks taken in reverse order (odd steps): a step then starts on the
  // bricks the step before ended with, whose populations L2 still holds
  int reverse;
  float omega;              // 1 / tau
  float ff[3];              // fluid force density
  float eps, inv_eps;
  float scale, inv_scale;   // half storage scale 2^s and 2^-s
  const int* bin_count;     // bins of this step
  const int* bin_ids;
  int bin_cap;
  const Rec* rec;
  // list of the cells inside particles, appended by the collision for the
  // next step's momentum exchange (nullptr: not recorded):
  //   ilist_idx[k] = (global cell index, particle), ilist_mom[k] = mass and
  //   momentum of the cell's post-collision deviations as stored.
  // It is split into ILIST_STRIPES stripes of ilist_cap entries, stripe s at
  // [s * ilist_cap, (s + 1) * ilist_cap) with its own count ilist_count[s];
  // a collision block appends to stripe (block index mod ILIST_STRIPES), so
  // the appends of the whole grid do not contend for one counter.
  int* ilist_count;
  int2* ilist_idx;
  float4* ilist_mom;
  long long ilist_cap;
  int np;                   // particles (list entries name 0 .. np-1)
  long long* acc;           // [cap][6] momentum exchange of a particle, fixed point
  GridSet grids;            // signed-distance grids of shape-4 particles
  int* status;
};

struct PartArgs {
  int pdl;                  // launch with programmatic dependent launch (host side only)
  double* P;                // FP64 table, field-major with stride cap
  int cap, np;
  const int* shape;         // [np]
  const int* box;           // [np]
  Rec* rec;
  const BoxDesc* boxes;
  double g[3];
  double eps;
  // momentum exchange input
  const void* f;            // populations, blocked layout
  float scale, inv_scale;
  // momentum-exchange kernel: one block per (particle, bounding-box plane)
  const int* chunk_p;       // [chunks] particle of the block
  const int* chunk_q;       // [chunks] plane of the block
  const int* p_chunk0;      // [cap] first block of a particle
  const int* p_nchunk;      // [cap] blocks of a particle
  int nchunks;
  int mea_planes;           // bounding-box planes per momentum-exchange block
  double* partial;          // [chunks][6] FP64 partial force/torque sums
  int* done;                // [cap] blocks finished per particle (reset to 0)
  // the same sums added up by the moments-mode momentum exchange from the
  // moments the previous collision recorded
  long long* acc;           // [cap][6] momentum exchange, fixed point (ACC_FRAC_BITS)
  int from_acc;             // 1: the update takes acc, 0: the table's F and T
  // contact between the particles' enclosing capsules and with the walls
  // (an extension; off when contact_k == 0): stiffness and range
  double contact_k, contact_zeta;
  GridSet grids;            // signed-distance grids of shape-4 particles
  int nsm;                  // SMs of the GPU (update grid size)
  int ppb;                  // particles per update block (set by the launcher)
  int* ilist_count;         // [ILIST_STRIPES], reset by the update for the next collision
  // bins written by the update (this step) and cleared (other parity)
  int* bin_count;
  int* bin_ids;
  int* bin_count_clear;
  long long ntiles;
  int bin_cap;
  int* status;
};

// "Centre inside the particle" (Sec. 3.2, above Eq. hydrodynamicforce) in
// FP32, every operation rounded on its own so that each kernel (and the
// oracle) takes the same decision:
//   r = (fp32(cell) - xh, minimum image) - xl
//   sphere:    (r0 r0 + r1 r1) + r2 r2 < fp32(a^2)
//   ellipsoid: e = (M^T r) * fp32(1/a) componentwise, (e0 e0 + e1 e1) + e2 e2 < 1
//   cuboid:    |M^T r| < a componentwise
//   capsule:   b = M^T r, t = b2 - clamp(b2, -a2, a2), (b0 b0 + b1 b1) + t t < fp32(a0^2)
// where (M^T r)_j = (M_0j r0 + M_1j r1) + M_2j r2.
__device__ __forceinline__ float offset_fp32(int cell, int n, bool wall, float xh, float xl) {
  float r0 = __fsub_rn((float)cell, xh);
  if (!wall) {
    const float L = (float)n;
    const float half = __fmul_rn(0.5f, L);
    if (r0 > half) r0 = __fsub_rn(r0, L);
    else if (r0 < -half) r0 = __fadd_rn(r0, L);
  }
  return __fsub_rn(r0, xl);
}

__device__ __forceinline__ bool inside_from_offset(const Rec& R, const float r[3], GridSet gs = GridSet{}) {
  if (R.shape == 0) {
    float s = __fmul_rn(r[0], r[0]);
    s = __fadd_rn(s, __fmul_rn(r[1], r[1]));
    s = __fadd_rn(s, __fmul_rn(r[2], r[2]));
    return s < R.in2;
  }
  float b[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    float t = __fmul_rn(R.M[0 * 3 + j], r[0]);
    t = __fadd_rn(t, __fmul_rn(R.M[1 * 3 + j], r[1]));
    t = __fadd_rn(t, __fmul_rn(R.M[2 * 3 + j], r[2]));
    b[j] = t;
  }
  if (R.shape == 1) {
    const float e0 = __fmul_rn(b[0], R.ia[0]);
    const float e1 = __fmul_rn(b[1], R.ia[1]);
    const float e2 = __fmul_rn(b[2], R.ia[2]);
    float s = __fmul_rn(e0, e0);
    s = __fadd_rn(s, __fmul_rn(e1, e1));
    s = __fadd_rn(s, __fmul_rn(e2, e2));
    return s < 1.0f;
  }
  if (R.shape == 4) {
    if (!gs.desc) return false;
    return grid_blend_rn(gs.desc[__float_as_int(R.in2)], gs.vals, b) < 0.0f;
  }
  if (R.shape == 3) {
    const float c = b[2] < -R.a[2] ? -R.a[2] : (b[2] > R.a[2] ? R.a[2] : b[2]);
    const float t = __fsub_rn(b[2], c);
    float s = __fmul_rn(b[0], b[0]);
    s = __fadd_rn(s, __fmul_rn(b[1], b[1]));
    s = __fadd_rn(s, __fmul_rn(t, t));
    return s < R.in2;
  }
  return fabsf(b[0]) < R.a[0] && fabsf(b[1]) < R.a[1] && fabsf(b[2]) < R.a[2];
}

__device__ __forceinline__ bool inside_fp32(const Rec& R, const BoxDesc& bd, int x, int y, int z,
                                            float r[3], GridSet gs = GridSet{}) {
  r[0] = offset_fp32(x, bd.nx, bd.bc & 1, R.xh[0], R.xl[0]);
  r[1] = offset_fp32(y, bd.ny, bd.bc & 2, R.xh[1], R.xl[1]);
  r[2] = offset_fp32(z, bd.nz, bd.bc & 4, R.xh[2], R.xl[2]);
  return inside_from_offset(R, r, gs);
}

// launchers (stream-ordered, no synchronisation)
cudaError_t launch_collide(const LbmArgs& a, int precision, int parity, bool walls, bool couple,
                           cudaStream_t s);
// the collision with two x-adjacent cells per thread (a.cells_x == 2)
cudaError_t launch_collide_pair(const LbmArgs& a, int precision, int parity, bool walls, bool couple,
                                cudaStream_t s);
// momentum exchange from the arrivals and the moments recorded in the list of
// interior cells (a.rec must describe the particle state of this step)
cudaError_t launch_mea_moments(const LbmArgs& a, int precision, int parity, bool walls, int nsm,
                               cudaStream_t s);
cudaError_t launch_mea(const PartArgs& a, int precision, int parity, cudaStream_t s);
cudaError_t launch_update(const PartArgs& a, cudaStream_t s);
// contact force and torque of every particle into PF_FC / PF_TC (only when
// a.contact_k > 0)
cudaError_t launch_contact(const PartArgs& a, cudaStream_t s);
cudaError_t launch_records(const PartArgs& a, cudaStream_t s);
// logical populations f_i - w_i of cells [c0, c0 + n) of one box, as float,
// into/out of stage[i * n + k]
cudaError_t launch_gather(const LbmArgs& a, int precision, int parity, int box, long long c0,
                          long long n, float* stage, cudaStream_t s);
cudaError_t launch_scatter(const LbmArgs& a, int precision, int parity, int box, long long c0,
                           long long n, const float* stage, cudaStream_t s);
// the five stored slots with c_z = dir of the cells of plane z of one box
// (ncell = nx ny of the box), to (put = 0) or from (put = 1) stage
cudaError_t launch_plane_slots(const LbmArgs& a, int precision, int box, int z, int dir, int ncell, void* stage,
                               int put, cudaStream_t s);
// FP64 mass deviation and momentum of one box: `blocks` partial sums of 4
// values into out[4 * blocks]
cudaError_t launch_fluid_moments(const LbmArgs& a, int precision, int parity, int box, int blocks,
                                 double* out, cudaStream_t s);

}  // namespace hlbm
