// particle_kernels.cu -- fluid -> particle coupling and particle motion.
//
//   mea_kernel      momentum exchange (Eq. hlbm:mea) summed over the cells
//                   whose centre lies inside each particle (Eqs.
//                   hydrodynamicforce, hydrodynamictorque); MEA_CHUNKS thread
//                   blocks per particle each walk a slab of z-planes of the
//                   particle's bounding box; per-cell sums in FP32, warp
//                   shuffles in FP32, block sums in FP64, written as partials
//                   that the update adds in a fixed order (deterministic).
//   update_kernel   weight minus buoyancy (Sec. 5.1), Newton-Euler update
//                   (Eqs. particlemotiontrans, motionrot) in FP64, the FP32
//                   coupling record of the new state, and the per-tile particle
//                   lists (the single-GPU form of the paper's particle
//                   assignment, Sec. 4.2.3) that the collision kernel reads.
//   records_kernel  coupling records only (after particles are added or set).
#include "mea_common.cuh"

namespace hlbm {

__device__ __forceinline__ double pget(const double* P, int cap, int field, int p) {
  return P[(long long)field * cap + p];
}
__device__ __forceinline__ void pset(double* P, int cap, int field, int p, double v) {
  P[(long long)field * cap + p] = v;
}

// FP32 coupling record of a particle state (X, U, W, q; semi-axes A, their
// FP32 inverses iA, radius r_inf beyond which B = 0; interface width eps)
__device__ __forceinline__ void make_record(const double X[3], const double U[3], const double W[3],
                                            const double q[4], const double A[3], const double iA[3],
                                            double rinf, float eps, int p, int shape, int box, Rec& R) {
  double Rm[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};  // a sphere needs no orientation
  if (shape != 0) rotation_rn(q, Rm);
  for (int j = 0; j < 3; ++j) {
    const float xh = __double2float_rn(X[j]);
    R.xh[j] = xh;
    R.xl[j] = __double2float_rn(X[j] - (double)xh);
    R.u[j] = (float)U[j];
    R.w[j] = (float)W[j];
    R.a[j] = __double2float_rn(A[j]);
    R.ia[j] = (float)iA[j];
  }
  for (int k = 0; k < 9; ++k) R.M[k] = __double2float_rn(Rm[k]);
  R.in2 = __double2float_rn(A[0] * A[0]);
  if (shape == 4) R.in2 = __int_as_float((int)iA[0]);  // a grid particle: its grid id
  if (shape == 0) {
    // a sphere needs no rotation: its slots hold the FP32 bounds of the
    // collision's per-cell tests (the same roundings as computed there)
    const float a_in = __fsub_rn(R.a[0], __fmul_rn(0.5f, eps));
    const float a_out = __fadd_rn(R.a[0], __fmul_rn(0.5f, eps));
    R.M[SPH_IN_LO] = __fmul_rn(R.in2, 0.99999f);
    R.M[SPH_IN_HI] = __fmul_rn(R.in2, 1.00001f);
    R.M[SPH_R2_IN] = a_in > 0.0f ? __fmul_rn(a_in, a_in) : -1.0f;
    R.M[SPH_R2_OUT] = __fmul_rn(a_out, a_out);
  }
  // B vanishes beyond r_inf; a slightly larger FP32 bound keeps the test safe
  const double rb = rinf + 0.01;
  R.rinf2 = (float)(rb * rb);
  R.shape = shape;
  R.box = box;
  R.pid = p;
}

__device__ void build_record(const double* P, int cap, int p, int shape, int box, float eps, Rec& R) {
  double X[3], U[3], W[3], q[4], A[3], iA[3];
  for (int j = 0; j < 3; ++j) {
    X[j] = pget(P, cap, PF_X + j, p);
    U[j] = pget(P, cap, PF_U + j, p);
    W[j] = pget(P, cap, PF_W + j, p);
    A[j] = pget(P, cap, PF_A + j, p);
    iA[j] = pget(P, cap, PF_IA + j, p);
  }
  for (int j = 0; j < 4; ++j) q[j] = pget(P, cap, PF_Q + j, p);
  make_record(X, U, W, q, A, iA, pget(P, cap, PF_RINF, p), eps, p, shape, box, R);
}

// MEA_MINBLOCKS resident blocks per SM; a block walks a.mea_planes
// bounding-box planes of one particle
#ifndef HLBM_MEA_THREADS
#define HLBM_MEA_THREADS 128
#endif
constexpr int MEA_THREADS = HLBM_MEA_THREADS;

template <typename S, int PAR, bool GRIDS>
__global__ void __launch_bounds__(MEA_THREADS, MEA_MINBLOCKS * 128 / MEA_THREADS) mea_kernel(PartArgs a) {
  pdl_trigger();
  pdl_wait();
  const int chunk = blockIdx.x;
  const int p = a.chunk_p[chunk], iz0 = a.chunk_q[chunk];
  __shared__ Rec R;
  __shared__ double wsum[MEA_THREADS / 32][6];
  __shared__ int s_start[MAX_PLANES + 1], s_xa[MAX_PLANES];
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < 32) reinterpret_cast<int*>(&R)[tid] = reinterpret_cast<const int*>(&a.rec[p])[tid];
  __syncthreads();
  double* out = a.partial + (long long)chunk * 6;
  const BoxDesc bd = a.boxes[R.box];
  const double rc = pget(a.P, a.cap, PF_RC, p);
  double X[3];
  // a particle whose centre is not finite or far outside the box has no
  // interior cells (the update flags it); this also bounds the loops below
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    X[j] = pget(a.P, a.cap, PF_X + j, p);
    ok = ok && (X[j] > -1.0e6 && X[j] < 1.0e6);
  }
  float sums[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (ok) {
    // planes iz0 .. iz0 + mea_planes - 1 (those past the box's extent add nothing)
    for (int iz = iz0; iz < iz0 + a.mea_planes; ++iz) {
      float ps[6];
      mea_plane_sums<S, PAR, true>(R, bd, X, rc, iz, reinterpret_cast<const S*>(a.f), 0, a.inv_scale, s_start,
                                   s_xa, ps, GRIDS ? a.grids : GridSet{});
      for (int k = 0; k < 6; ++k) sums[k] += ps[k];
      __syncthreads();  // s_start, s_xa are rewritten by the next plane
    }
  } else if (tid == 0) {
    atomicOr(a.status, ST_UNSTABLE);
  }
  float v[6] = {sums[0], sums[1], sums[2], sums[3], sums[4], sums[5]};
#pragma unroll
  for (int k = 0; k < 6; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if (lane == 0)
    for (int k = 0; k < 6; ++k) wsum[warp][k] = (double)v[k];
  __syncthreads();
  if (tid < 6) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += wsum[w][tid];
    out[tid] = s;
  }
  // the last block of a particle adds its planes' partials in plane order
  // (deterministic) and writes the particle's force and torque
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(&a.done[p], 1) == a.p_nchunk[p] - 1);
  __syncthreads();
  if (s_last) {
    __threadfence();
    if (tid < 6) {
      const int c0 = a.p_chunk0[p], nc = a.p_nchunk[p];
      double s = 0.0;
      for (int k = 0; k < nc; ++k) s += __ldcg(a.partial + (long long)(c0 + k) * 6 + tid);
      pset(a.P, a.cap, (tid < 3 ? PF_F : PF_T - 3) + tid, p, s);
    }
    if (tid == 0) a.done[p] = 0;
  }
}

// the bin tiles along one axis touched by cells [lo, hi]: one range
// [a0, a1], plus a second range [b0, b1] (empty when b1 < b0) where the cell
// range wraps around a periodic axis
struct AxisTiles {
  int a0, a1, b0, b1;
  __device__ __forceinline__ int count() const { return (a1 - a0 + 1) + max(b1 - b0 + 1, 0); }
  __device__ __forceinline__ int at(int t) const {
    const int na = a1 - a0 + 1;
    return t < na ? a0 + t : b0 + (t - na);
  }
};

__device__ AxisTiles axis_tiles(int lo, int hi, int n, int T, bool wall) {
  AxisTiles r{0, -1, 0, -1};
  if (wall) {
    lo = max(lo, 0);
    hi = min(hi, n - 1);
    if (lo <= hi) { r.a0 = lo / T; r.a1 = hi / T; }
    return r;
  }
  if (hi - lo + 1 >= n) {  // the whole periodic axis
    r.a0 = 0; r.a1 = (n - 1) / T;
    return r;
  }
  if (lo < 0) {            // [lo + n, n - 1] and [0, hi]
    r.a0 = (lo + n) / T; r.a1 = (n - 1) / T;
    r.b0 = 0; r.b1 = hi / T;
  } else if (hi >= n) {    // [lo, n - 1] and [0, hi - n]
    r.a0 = lo / T; r.a1 = (n - 1) / T;
    r.b0 = 0; r.b1 = (hi - n) / T;
  } else {
    r.a0 = lo / T; r.a1 = hi / T;
  }
  // both ends in the same tiles (an axis of one or two tiles): merge
  if (r.b1 >= r.b0 && r.b1 >= r.a0) {
    r.a0 = 0; r.a1 = max(r.a1, r.b1);
    r.b0 = 0; r.b1 = -1;
  }
  return r;
}

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// Newton-Euler step (Eqs. particlemotiontrans, motionrot), symplectic Euler:
// U += F / m with F = F_h + (rho_p - rho_f) V g, X += U; spheres:
// omega += T / I; other shapes: body-frame Euler equations
// omega_b += (T_b - omega_b x (I omega_b)) / I with the rotation of the old
// quaternion; q += q (x) (0, omega_b) / 2, normalised (for a sphere in the
// equal form (0, omega) (x) q / 2, which needs no rotation).  GB300's FP64
// pipe is narrow: a warp's FP64 instruction takes it for many cycles however
// few lanes are active, so the translation and the rotation of a block's
// particles run on two warps (two SM sub-partitions) at once, each lane one
// particle, and meet in shared memory for the record and the binning.

// Tiles of one particle's bin range, kept in shared memory between the
// Newton-Euler step and the binning.
struct BinRange {
  AxisTiles at[3];
  long long tile_off;
  int ntx, nty;
  int count;  // tiles; 0 when the particle is not binned
};

// force of the momentum exchange (row base PF_F) or torque (PF_T) of particle
// p: written into the table by the bounding-box kernel, or accumulated from
// the recorded moments (that accumulator is cleared for the next step); the
// table keeps it, and the contact force or torque joins it as an acting one
__device__ __forceinline__ void exchange_force(const PartArgs& a, int p, int row, int crow, int k0, double Fo[3]) {
  long long* acc = a.acc + (long long)p * 6 + k0;
  const double unit = 1.0 / (double)(1LL << ACC_FRAC_BITS);  // fixed point -> force and torque
  for (int j = 0; j < 3; ++j) Fo[j] = a.from_acc ? (double)acc[j] * unit : pget(a.P, a.cap, row + j, p);
  if (a.from_acc)
    for (int j = 0; j < 3; ++j) acc[j] = 0;
  for (int j = 0; j < 3; ++j) pset(a.P, a.cap, row + j, p, Fo[j]);
  if (a.contact_k > 0.0)
    for (int j = 0; j < 3; ++j) Fo[j] += pget(a.P, a.cap, crow + j, p);
}

// translation of particle p: force, U, X (wrapped on periodic axes), the
// record's position and velocity, and the tiles its bins cover
__device__ __forceinline__ void translate_particle(const PartArgs& a, int p, Rec& R, BinRange& br) {
  const double* __restrict__ P = a.P;
  const int cap = a.cap;
  const BoxDesc bd = a.boxes[a.box[p]];
  double X[3], U[3], Fh[3];
  for (int j = 0; j < 3; ++j) {
    X[j] = pget(P, cap, PF_X + j, p);
    U[j] = pget(P, cap, PF_U + j, p);
  }
  const double im = pget(P, cap, PF_IM, p), V = pget(P, cap, PF_V, p), rho = pget(P, cap, PF_RHO, p);
  const double rinf = pget(P, cap, PF_RINF, p), rc = pget(P, cap, PF_RC, p);
  exchange_force(a, p, PF_F, PF_FC, 0, Fh);
  bool ok = true;
  for (int j = 0; j < 3; ++j) {
    const double F = Fh[j] + (rho - 1.0) * V * a.g[j];  // Fh: hydrodynamic (and contact) force
    U[j] += F * im;
    X[j] += U[j];
    ok = ok && isfinite(X[j]) && isfinite(U[j]);
  }
  if (!ok) atomicOr(a.status, ST_UNSTABLE);
  const int n[3] = {bd.nx, bd.ny, bd.nz};
  for (int j = 0; j < 3; ++j) {
    if ((bd.bc >> j) & 1) {
      // a slab's cut z faces are not walls: centres may lie beyond them
      const bool cut = j == 2 && (bd.bc & BC_CUT_Z);
      if (!cut && !(X[j] > -0.5 && X[j] < n[j] - 0.5)) atomicOr(a.status, ST_LEFT_DOMAIN);
    } else {
      // a particle moves far less than a box length per step
      const double L = (double)n[j];
      if (X[j] >= L) X[j] -= L;
      else if (X[j] < 0.0) X[j] += L;
    }
  }
  for (int j = 0; j < 3; ++j) {
    pset(a.P, cap, PF_X + j, p, X[j]);
    pset(a.P, cap, PF_U + j, p, U[j]);
    const float xh = __double2float_rn(X[j]);
    R.xh[j] = xh;
    R.xl[j] = __double2float_rn(X[j] - (double)xh);
    R.u[j] = (float)U[j];
  }
  // bin tiles touched by the influence sphere, widened so that the cells next
  // to the particle's interior (which feed its momentum exchange) see it too;
  // the cell range is rounded outwards in FP32
  br.tile_off = bd.tile_off;
  br.ntx = bd.ntx;
  br.nty = bd.nty;
  br.count = 0;
  const float rb = __double2float_ru(fmax(rinf, rc + 1.5));
  const int T[3] = {TILE_X, TILE_Y, TILE_Z};
  for (int j = 0; j < 3; ++j) {
    if (!(X[j] > -1.0e6 && X[j] < 1.0e6)) return;  // flagged above; not binned
    const int lo = (int)floorf(__fsub_rd(__double2float_rd(X[j]), rb)) - 1;
    const int hi = (int)ceilf(__fadd_ru(__double2float_ru(X[j]), rb)) + 1;
    br.at[j] = axis_tiles(lo, hi, n[j], T[j], (bd.bc >> j) & 1);
  }
  br.count = br.at[0].count() * br.at[1].count() * br.at[2].count();
}

// rotation of particle p: torque, omega, quaternion, the record's angular
// velocity and orientation; the record's fixed fields (shape, box, id, sizes
// and the bounds derived from them) come from its previous record
__device__ __forceinline__ void rotate_particle(const PartArgs& a, int p, Rec& R) {
  const double* __restrict__ P = a.P;
  const int cap = a.cap;
  const int shape = a.shape[p];
  double W[3], q[4], I[3], iI[3], Th[3];
  for (int j = 0; j < 3; ++j) {
    W[j] = pget(P, cap, PF_W + j, p);
    iI[j] = pget(P, cap, PF_II + j, p);
    I[j] = shape == 0 ? 0.0 : pget(P, cap, PF_I + j, p);
  }
  for (int j = 0; j < 4; ++j) q[j] = pget(P, cap, PF_Q + j, p);
  const Rec& old = a.rec[p];
  for (int j = 0; j < 3; ++j) {
    R.a[j] = old.a[j];
    R.ia[j] = old.ia[j];
  }
  R.in2 = old.in2;
  R.rinf2 = old.rinf2;
  R.shape = old.shape;
  R.box = old.box;
  R.pid = old.pid;
  if (shape == 0)
    for (int k = 0; k < 9; ++k) R.M[k] = old.M[k];  // a sphere's collision bounds
  exchange_force(a, p, PF_T, PF_TC, 3, Th);
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  double dq[4];
  if (shape == 0) {
    // q (x) (0, omega_b) equals (0, omega) (x) q: no rotation needed
    for (int j = 0; j < 3; ++j) W[j] += Th[j] * iI[j];
    dq[0] = -0.5 * (W[0] * x + W[1] * y + W[2] * z);
    dq[1] = 0.5 * (w * W[0] + W[1] * z - W[2] * y);
    dq[2] = 0.5 * (w * W[1] + W[2] * x - W[0] * z);
    dq[3] = 0.5 * (w * W[2] + W[0] * y - W[1] * x);
  } else {
    double Rm[9], wb[3], Tb[3], Lb[3], gy[3];
    rotation_rn(q, Rm);
    for (int j = 0; j < 3; ++j) {
      wb[j] = Rm[0 * 3 + j] * W[0] + Rm[1 * 3 + j] * W[1] + Rm[2 * 3 + j] * W[2];
      Tb[j] = Rm[0 * 3 + j] * Th[0] + Rm[1 * 3 + j] * Th[1] + Rm[2 * 3 + j] * Th[2];
    }
    for (int j = 0; j < 3; ++j) Lb[j] = I[j] * wb[j];
    cross3(wb, Lb, gy);
    for (int j = 0; j < 3; ++j) wb[j] += (Tb[j] - gy[j]) * iI[j];
    for (int j = 0; j < 3; ++j) W[j] = Rm[j * 3 + 0] * wb[0] + Rm[j * 3 + 1] * wb[1] + Rm[j * 3 + 2] * wb[2];
    dq[0] = 0.5 * (-x * wb[0] - y * wb[1] - z * wb[2]);
    dq[1] = 0.5 * (w * wb[0] + y * wb[2] - z * wb[1]);
    dq[2] = 0.5 * (w * wb[1] + z * wb[0] - x * wb[2]);
    dq[3] = 0.5 * (w * wb[2] + x * wb[1] - y * wb[0]);
  }
  double nq = 0.0;
  for (int j = 0; j < 4; ++j) {
    q[j] += dq[j];
    nq += q[j] * q[j];
  }
  const double inq = rsqrt(nq);
  for (int j = 0; j < 4; ++j) q[j] *= inq;
  if (!(isfinite(W[0]) && isfinite(W[1]) && isfinite(W[2]))) atomicOr(a.status, ST_UNSTABLE);
  for (int j = 0; j < 3; ++j) {
    pset(a.P, cap, PF_W + j, p, W[j]);
    R.w[j] = (float)W[j];
  }
  for (int j = 0; j < 4; ++j) pset(a.P, cap, PF_Q + j, p, q[j]);
  if (shape != 0) {
    double Rn[9];
    rotation_rn(q, Rn);
    for (int k = 0; k < 9; ++k) R.M[k] = __double2float_rn(Rn[k]);
  }
}

// a.ppb particles per block of UPD_T threads (ppb a power of two up to
// UPD_P): lane k of warp 0 moves particle k of the block, lane k of warp 1
// turns it; then all threads store the records and add the block's
// particles to the per-tile lists, UPD_T / ppb threads per particle taking
// its tiles in turn.  Few particles get small groups, so that the blocks
// spread over the GPU and each particle's tiles take one round of atomics.
constexpr int UPD_P = 32, UPD_T = 256;

__global__ void __launch_bounds__(UPD_T) update_kernel(PartArgs a) {
  __shared__ BinRange s_br[UPD_P];
  __shared__ Rec s_rec[UPD_P];
  pdl_trigger();
  pdl_wait();
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nthr = (long long)gridDim.x * blockDim.x;
  for (long long t = tid; t < a.ntiles; t += nthr) a.bin_count_clear[t] = 0;
  if (tid < ILIST_STRIPES && a.ilist_count) a.ilist_count[tid] = 0;  // the collision appends anew
  const int ppb = a.ppb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (long long base = blockIdx.x * (long long)ppb; base < a.np; base += (long long)gridDim.x * ppb) {
    if (warp < 2 && lane < ppb) {
      const long long p = base + lane;
      if (p < a.np) {
        if (warp == 0) translate_particle(a, (int)p, s_rec[lane], s_br[lane]);
        else rotate_particle(a, (int)p, s_rec[lane]);
      } else if (warp == 0) {
        s_br[lane].count = 0;
      }
    }
    __syncthreads();
    const long long nrec = min((long long)ppb, a.np - base);
    for (int e = threadIdx.x; e < nrec * 32; e += UPD_T)
      reinterpret_cast<int*>(&a.rec[base + (e >> 5)])[e & 31] = reinterpret_cast<const int*>(&s_rec[e >> 5])[e & 31];
    const int k = threadIdx.x % ppb, sub = threadIdx.x / ppb;
    const BinRange& br = s_br[k];
    const int cx_ = br.at[0].count(), cy_ = br.at[1].count();
    const int p = (int)(base + k);
    for (int t = sub; t < br.count; t += UPD_T / ppb) {
      const int ix = t % cx_, r = t / cx_, iy = r % cy_, iz = r / cy_;
      const long long tile = br.tile_off + ((long long)br.at[2].at(iz) * br.nty + br.at[1].at(iy)) * br.ntx +
                             br.at[0].at(ix);
      const int slot = atomicAdd(&a.bin_count[tile], 1);
      if (slot < a.bin_cap) a.bin_ids[tile * a.bin_cap + slot] = p;
      else atomicOr(a.status, ST_CAPACITY);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- contact
// Contact between particles (an extension: the paper counts contact among
// the acting forces of Sec. 2.2 without stating a model, and its runs have
// none).  Each particle is enclosed by a capsule, the points within r_c of
// the segment X +- h_c e: a sphere by itself (h_c = 0), a capsule by itself,
// an ellipsoid by the capsule along its longest semi-axis a_k with r_c the
// larger other semi-axis and h_c = a_k - r_c, a cuboid by the capsule along
// its longest half-extent h_k with r_c = |(h_i, h_j)| and h_c = h_k.  Two
// capsules whose segments come closest at p_i, p_j (minimum image) with gap
// delta = |p_i - p_j| - r_i - r_j < zeta repel along n = (p_i - p_j) / |.|
// with k ((zeta - delta) / zeta)^2, and particle i takes the torque
// (p_i - X_i) x F_i; a wall pushes the segment end nearest to it the same
// way.  All in FP64 from the particle table at the state before the update.

// enclosing capsule of particle p: unit axis e, half-length h, radius r
__device__ __forceinline__ void contact_capsule(const double* P, int cap, int p, int shape, double e[3],
                                                double& h, double& r) {
  double A[3], q[4];
  for (int j = 0; j < 3; ++j) A[j] = pget(P, cap, PF_A + j, p);
  for (int j = 0; j < 4; ++j) q[j] = pget(P, cap, PF_Q + j, p);
  int k = 2;
  if (shape == 0 || shape == 4) {  // a grid particle: the sphere of its circumscribed radius
    h = 0.0;
    r = A[0];
  } else if (shape == 3) {
    h = A[2];
    r = A[0];
  } else {
    k = A[1] > A[0] ? 1 : 0;
    if (A[2] > A[k]) k = 2;
    const int i = (k + 1) % 3, j = (k + 2) % 3;
    if (shape == 1) {
      r = fmax(A[i], A[j]);
      h = A[k] - r;
    } else {
      r = sqrt(A[i] * A[i] + A[j] * A[j]);
      h = A[k];
    }
  }
  if (shape == 0 || shape == 4) {
    e[0] = 0.0; e[1] = 0.0; e[2] = 1.0;
    return;
  }
  double R[9];
  rotation_rn(q, R);
  for (int j = 0; j < 3; ++j) e[j] = R[j * 3 + k];
}

// FP32 bound on the reach of a particle's contact capsule from its centre
__device__ __forceinline__ float contact_reach(const Rec& R) {
  if (R.shape == 0 || R.shape == 4) return R.a[0];
  if (R.shape == 3) return R.a[0] + R.a[2];
  const float amax = fmaxf(R.a[0], fmaxf(R.a[1], R.a[2]));
  if (R.shape == 1) return amax;
  return sqrtf(R.a[0] * R.a[0] + R.a[1] * R.a[1] + R.a[2] * R.a[2]) + amax;  // >= h_k + |(h_i, h_j)|
}

// closest points P + s u, Q + t v of two segments (|s| <= hu, |t| <= hv,
// unit u, v): the points of closest approach of the two lines, s clamped,
// t taken from s and clamped, s taken again from t and clamped
__device__ __forceinline__ void segment_closest(const double P[3], const double u[3], double hu,
                                                const double Q[3], const double v[3], double hv,
                                                double& s, double& t) {
  double b = 0.0, d = 0.0, f = 0.0;
  for (int j = 0; j < 3; ++j) {
    const double w = P[j] - Q[j];
    b += u[j] * v[j];
    d += u[j] * w;
    f += v[j] * w;
  }
  const double den = 1.0 - b * b;
  s = den > 1e-12 ? fmin(fmax((b * f - d) / den, -hu), hu) : 0.0;
  t = fmin(fmax(b * s + f, -hv), hv);
  s = fmin(fmax(b * t - d, -hu), hu);
}

__device__ __forceinline__ double contact_ramp(double k, double zeta, double gap) {
  const double x = (zeta - gap) / zeta;
  return k * x * x;
}

// one warp per particle: the lanes take the other particles of its box in
// turn (an FP32 test of the centre distance against the capsules' reach
// first), lane 0 the walls; the warp's FP64 sums are added in a fixed order
__global__ void __launch_bounds__(256) contact_kernel(PartArgs a) {
  pdl_trigger();
  pdl_wait();
  const int i = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= a.np) return;  // whole warps
  const double* P = a.P;
  const int cap = a.cap;
  const Rec& Ri = a.rec[i];
  const int si = a.shape[i], box = a.box[i];
  const BoxDesc bd = a.boxes[box];
  const int n[3] = {bd.nx, bd.ny, bd.nz};
  double Xi[3], ei[3], hi, ri;
  for (int j = 0; j < 3; ++j) Xi[j] = pget(P, cap, PF_X + j, i);
  contact_capsule(P, cap, i, si, ei, hi, ri);
  const float reach_i = contact_reach(Ri);
  const double k = a.contact_k, zeta = a.contact_zeta;
  double F[3] = {0.0, 0.0, 0.0}, T[3] = {0.0, 0.0, 0.0};
  auto add = [&](const double pt[3], const double f[3]) {
    const double arm[3] = {pt[0] - Xi[0], pt[1] - Xi[1], pt[2] - Xi[2]};
    double tq[3];
    cross3(arm, f, tq);
    for (int c = 0; c < 3; ++c) {
      F[c] += f[c];
      T[c] += tq[c];
    }
  };
  for (int j = lane; j < a.np; j += 32) {
    if (j == i || a.box[j] != box) continue;
    const Rec& Rj = a.rec[j];
    float d2 = 0.0f;
    for (int c = 0; c < 3; ++c) {
      float dc = Rj.xh[c] - Ri.xh[c];
      if (!((bd.bc >> c) & 1)) {
        const float L = (float)n[c];
        if (dc > 0.5f * L) dc -= L;
        else if (dc < -0.5f * L) dc += L;
      }
      d2 += dc * dc;
    }
    const float lim = reach_i + contact_reach(Rj) + (float)zeta + 0.05f;
    if (d2 >= lim * lim) continue;
    double Xj[3], ej[3], hj, rj;
    for (int c = 0; c < 3; ++c) {
      double dc = pget(P, cap, PF_X + c, j) - Xi[c];
      if (!((bd.bc >> c) & 1)) {
        const double L = (double)n[c];
        if (dc > L / 2.0) dc -= L;
        else if (dc < -L / 2.0) dc += L;
      }
      Xj[c] = Xi[c] + dc;
    }
    contact_capsule(P, cap, j, a.shape[j], ej, hj, rj);
    double s, t;
    segment_closest(Xi, ei, hi, Xj, ej, hj, s, t);
    double pi[3], dv[3], dist = 0.0;
    for (int c = 0; c < 3; ++c) {
      pi[c] = Xi[c] + s * ei[c];
      dv[c] = pi[c] - (Xj[c] + t * ej[c]);
      dist += dv[c] * dv[c];
    }
    dist = sqrt(dist);
    const double gap = dist - ri - rj;
    if (gap >= zeta || !(dist > 0.0)) continue;
    const double fm = contact_ramp(k, zeta, gap);
    const double f[3] = {fm * dv[0] / dist, fm * dv[1] / dist, fm * dv[2] / dist};
    add(pi, f);
  }
  if (lane == 0) {
    for (int c = 0; c < 3; ++c) {
      if (!((bd.bc >> c) & 1) || (c == 2 && (bd.bc & BC_CUT_Z))) continue;
      for (int side = 0; side < 2; ++side) {
        const double dir = side == 0 ? -1.0 : 1.0;
        const double t = ei[c] * dir > 0.0 ? hi : (ei[c] * dir < 0.0 ? -hi : 0.0);
        const double pt[3] = {Xi[0] + t * ei[0], Xi[1] + t * ei[1], Xi[2] + t * ei[2]};
        const double gap = (side == 0 ? pt[c] + 0.5 : (n[c] - 0.5) - pt[c]) - ri;
        if (gap >= zeta) continue;
        double f[3] = {0.0, 0.0, 0.0};
        f[c] = -dir * contact_ramp(k, zeta, gap);
        add(pt, f);
      }
    }
  }
  for (int c = 0; c < 3; ++c)
    for (int o = 16; o > 0; o >>= 1) {
      F[c] += __shfl_xor_sync(0xffffffffu, F[c], o);
      T[c] += __shfl_xor_sync(0xffffffffu, T[c], o);
    }
  if (lane == 0)
    for (int c = 0; c < 3; ++c) {
      pset(a.P, cap, PF_FC + c, i, F[c]);
      pset(a.P, cap, PF_TC + c, i, T[c]);
    }
}

__global__ void records_kernel(PartArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.np) return;
  Rec R;
  build_record(a.P, a.cap, p, a.shape[p], a.box[p], (float)a.eps, R);
  a.rec[p] = R;
}

cudaError_t launch_mea(const PartArgs& a, int precision, int parity, cudaStream_t s) {
  if (a.np <= 0 || a.nchunks <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)a.nchunks;
  const bool pdl = a.pdl != 0;
  const bool g = a.grids.desc != nullptr;
  auto go = [&](auto kern) { return launch_k(kern, dim3(grid), dim3(MEA_THREADS), 0, s, pdl, a); };
  if (precision == 0) {
    if (parity == 0) return g ? go(mea_kernel<float, 0, true>) : go(mea_kernel<float, 0, false>);
    return g ? go(mea_kernel<float, 1, true>) : go(mea_kernel<float, 1, false>);
  }
  if (parity == 0) return g ? go(mea_kernel<__half, 0, true>) : go(mea_kernel<__half, 0, false>);
  return g ? go(mea_kernel<__half, 1, true>) : go(mea_kernel<__half, 1, false>);
}

cudaError_t launch_update(const PartArgs& a_in, cudaStream_t s) {
  PartArgs a = a_in;
  // particles per block: the smallest power of two that keeps the blocks
  // within about one per SM, at most UPD_P
  const long long target = a.nsm > 0 ? a.nsm : 152;
  a.ppb = 1;
  while (a.ppb < UPD_P && (long long)a.ppb * target < a.np) a.ppb *= 2;
  long long blocks = (a.np + a.ppb - 1) / a.ppb;
  long long clear_blocks = (a.ntiles + UPD_T - 1) / UPD_T;
  if (clear_blocks > blocks) blocks = clear_blocks;
  if (blocks > 65535) blocks = 65535;
  if (blocks < 1) blocks = 1;
  return launch_k(update_kernel, dim3((unsigned)blocks), dim3(UPD_T), 0, s, a.pdl != 0, a);
}

cudaError_t launch_contact(const PartArgs& a, cudaStream_t s) {
  if (a.np <= 0 || !(a.contact_k > 0.0)) return cudaSuccess;
  const long long threads = (long long)a.np * 32;
  return launch_k(contact_kernel, dim3((unsigned)((threads + 255) / 256)), dim3(256), 0, s, a.pdl != 0, a);
}

cudaError_t launch_records(const PartArgs& a, cudaStream_t s) {
  if (a.np <= 0) return cudaSuccess;
  records_kernel<<<(a.np + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace hlbm
