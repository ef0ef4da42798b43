// lbm_common.cuh -- device pieces shared by the collision kernels (one cell
// per thread in lbm_kernels.cu, two x-adjacent cells per thread in
// lbm_pair_kernels.cu): storage access, the indicator of Eq. B, the signed
// distances of the four shapes, the per-tile particle candidates and the
// per-cell coupling of Eq. hlbm:du (Sec. 3.2), and the list of cells inside
// particles that the collision appends for the next momentum exchange.
#pragma once
#include "hlbm_internal.cuh"

namespace hlbm {

constexpr int MAX_CAND = 64;  // particle records staged per block

template <typename S> struct Pop;
template <> struct Pop<float> {
  static constexpr bool SCALED = false;
  static __device__ __forceinline__ float ld(const float* p, float) { return *p; }
  static __device__ __forceinline__ void st(float* p, float v, float) { *p = v; }
  static __device__ __forceinline__ float ld_raw(const float* p) { return *p; }
  static __device__ __forceinline__ void st_raw(float* p, float v) { *p = v; }
  // two adjacent cells (8-byte aligned)
  static __device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
  static __device__ __forceinline__ void st2(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
};
template <> struct Pop<__half> {
  static __device__ __forceinline__ float ld(const __half* p, float inv_s) {
    return __half2float(*p) * inv_s;
  }
  static __device__ __forceinline__ void st(__half* p, float v, float s) { *p = __float2half_rn(v * s); }
  // the stored (scaled) value itself: the collision works in scaled units
  static constexpr bool SCALED = true;
  static __device__ __forceinline__ float ld_raw(const __half* p) { return __half2float(*p); }
  static __device__ __forceinline__ void st_raw(__half* p, float v) { *p = __float2half_rn(v); }
  // two adjacent cells (4-byte aligned)
  static __device__ __forceinline__ float2 ld2(const __half* p) {
    return __half22float2(*reinterpret_cast<const __half2*>(p));
  }
  static __device__ __forceinline__ void st2(__half* p, float2 v) {
    *reinterpret_cast<__half2*>(p) = __float22half2_rn(v);
  }
};
// the value a store of v leaves in memory, read back as a deviation
template <typename S>
__device__ __forceinline__ float stored_value(float v, float s, float inv_s) {
  if (sizeof(S) == 4) return v;
  return __half2float(__float2half_rn(v * s)) * inv_s;
}

// Addressing of a thread's cells x .. x + n - 1 (one row, one storage block)
// for the collide-and-stream: the rows y - 1, y, y + 1 as block offsets, and
// the x neighbours left of the first and right of the last cell as element
// offsets from the first cell in the same row (periodic wrap), with flags
// for an x wall there.
struct RowBlocks {
  int yb[3];   // (y + dy - 1) * ntx, or -1 beyond a y wall
  int xb, xin; // x-block of the cells and x & 31 of the first
  int dl, dr;  // element of x - 1 and of x + n, minus the element of x
  bool wl, wr; // x - 1 / x + n lies beyond an x wall
};

__device__ __forceinline__ int x_term(int x) { return (x >> 5) * QVB + (x & 31); }

template <bool WALLS>
__device__ __forceinline__ RowBlocks row_blocks(const BoxDesc& bd, int x, int y, int n) {
  RowBlocks r;
  const int nx = bd.nx, ny = bd.ny, ntx = bd.ntx;
  const bool wx = WALLS && (bd.bc & 1), wy = WALLS && (bd.bc & 2);
  r.yb[1] = y * ntx;
  r.yb[0] = y > 0 ? (y - 1) * ntx : (wy ? -1 : (ny - 1) * ntx);
  r.yb[2] = y < ny - 1 ? (y + 1) * ntx : (wy ? -1 : 0);
  r.xb = x >> 5;
  r.xin = x & 31;
  const int xl = x > 0 ? x - 1 : nx - 1, xr = x + n < nx ? x + n : x + n - nx;
  r.dl = x_term(xl) - x_term(x);
  r.dr = x_term(xr) - x_term(x);
  r.wl = wx && x == 0;
  r.wr = wx && x + n == nx;
  return r;
}

// first block of slice z + dz - 1 of the box, or -1 beyond a z wall
template <bool WALLS>
__device__ __forceinline__ void slice_blocks(const BoxDesc& bd, int z, int zb[3]) {
  const int nz = bd.nz, sl = bd.ny * bd.ntx, b0 = (int)bd.blk_off;
  const bool wz = WALLS && (bd.bc & 4);
  zb[1] = b0 + z * sl;
  zb[0] = z > 0 ? b0 + (z - 1) * sl : (wz ? -1 : b0 + (nz - 1) * sl);
  zb[2] = z < nz - 1 ? b0 + (z + 1) * sl : (wz ? -1 : b0);
}

// element of slot 0 of the first cell in storage block B
template <typename S>
__device__ __forceinline__ S* cell_ptr(S* f, int B, int xin) { return f + ((long long)B * QVB + xin); }

// sin(pi t) for |t| <= 1/2: the Taylor series of sin truncated after the
// t^11 term, in Horner form in t^2; the remainder is below
// (pi/2)^13 / 13! < 6e-8, and FP32 rounding keeps the total below 2e-7
__device__ __forceinline__ float sinpi_ramp(float t) {
  const float t2 = t * t;
  float p = -7.3704309457143508e-3f;    // -pi^11 / 11!
  p = fmaf(p, t2, 8.2145886611128229e-2f);  // pi^9 / 9!
  p = fmaf(p, t2, -5.9926452932079208e-1f); // -pi^7 / 7!
  p = fmaf(p, t2, 2.5501640398773455f);     // pi^5 / 5!
  p = fmaf(p, t2, -5.1677127800499703f);    // -pi^3 / 3!
  p = fmaf(p, t2, 3.1415926535897932f);     // pi
  return p * t;
}

// indicator of Eq. B written as (1 - sin(pi d / eps)) / 2 on the ramp, which
// equals cos^2((pi/2)(d/eps + 1/2))
__device__ __forceinline__ float indicator(float d, float eps, float inv_eps) {
  if (d <= -0.5f * eps) return 1.0f;
  if (d >= 0.5f * eps) return 0.0f;
  return 0.5f - 0.5f * sinpi_ramp(d * inv_eps);
}

// trilinear blend of a distance grid at body offset b (FP32, contracted;
// +inf outside the grid: no coupling there)
__device__ __forceinline__ float grid_blend(const GridDesc& g, const float* v, float b0, float b1, float b2) {
  const float x = fmaf(b0, g.ih, g.half[0]), y = fmaf(b1, g.ih, g.half[1]), z = fmaf(b2, g.ih, g.half[2]);
  if (!(x >= 0.0f && x <= (float)(g.n[0] - 1) && y >= 0.0f && y <= (float)(g.n[1] - 1) && z >= 0.0f &&
        z <= (float)(g.n[2] - 1)))
    return __int_as_float(0x7f800000);
  const int ix = min((int)x, g.n[0] - 2), iy = min((int)y, g.n[1] - 2), iz = min((int)z, g.n[2] - 2);
  const float tx = x - (float)ix, ty = y - (float)iy, tz = z - (float)iz;
  const float* c = v + g.off + ((long long)iz * g.n[1] + iy) * g.n[0] + ix;
  const long long sy = g.n[0], sz = (long long)g.n[0] * g.n[1];
  const float e00 = fmaf(tx, c[1] - c[0], c[0]), e01 = fmaf(tx, c[sy + 1] - c[sy], c[sy]);
  const float e10 = fmaf(tx, c[sz + 1] - c[sz], c[sz]), e11 = fmaf(tx, c[sz + sy + 1] - c[sz + sy], c[sz + sy]);
  const float f0 = fmaf(ty, e01 - e00, e00), f1 = fmaf(ty, e11 - e10, e10);
  return fmaf(tz, f1 - f0, f0);
}

// signed distance of a particle at offset r (world frame), FP32
__device__ __forceinline__ float sdf(const Rec& R, float rx, float ry, float rz, float r2, GridSet gs = GridSet{}) {
  if (R.shape == 0) return (r2 > 0.0f ? r2 * rsqrtf(r2) : 0.0f) - R.a[0];
  // body frame b = M^T r
  const float b0 = R.M[0] * rx + R.M[3] * ry + R.M[6] * rz;
  const float b1 = R.M[1] * rx + R.M[4] * ry + R.M[7] * rz;
  const float b2 = R.M[2] * rx + R.M[5] * ry + R.M[8] * rz;
  if (R.shape == 4) {
    if (!gs.desc) return __int_as_float(0x7f800000);
    const GridDesc& g = gs.desc[__float_as_int(R.in2)];
    const float t = b2 - fminf(fmaxf(b2, -g.in_h), g.in_h);
    if (b0 * b0 + b1 * b1 + t * t < g.in_r2) return g.in_d;  // deep inside: B = 1, inside
    return grid_blend(g, gs.vals, b0, b1, b2);
  }
  if (R.shape == 3) {
    const float t = b2 - fminf(fmaxf(b2, -R.a[2]), R.a[2]);
    return sqrtf(b0 * b0 + b1 * b1 + t * t) - R.a[0];
  }
  if (R.shape == 1) {
    const float e0 = b0 * R.ia[0], e1 = b1 * R.ia[1], e2 = b2 * R.ia[2];
    const float k2 = e0 * e0 + e1 * e1 + e2 * e2;
    const float g0 = e0 * R.ia[0], g1 = e1 * R.ia[1], g2v = e2 * R.ia[2];
    const float g2 = g0 * g0 + g1 * g1 + g2v * g2v;
    if (g2 == 0.0f) return -fminf(R.a[0], fminf(R.a[1], R.a[2]));
    const float k = sqrtf(k2);
    return (k - 1.0f) * k * rsqrtf(g2);
  }
  const float q0 = fabsf(b0) - R.a[0], q1 = fabsf(b1) - R.a[1], q2 = fabsf(b2) - R.a[2];
  const float o0 = fmaxf(q0, 0.0f), o1 = fmaxf(q1, 0.0f), o2 = fmaxf(q2, 0.0f);
  return sqrtf(o0 * o0 + o1 * o1 + o2 * o2) + fminf(fmaxf(q0, fmaxf(q1, q2)), 0.0f);
}

__device__ __forceinline__ int find_box(const BoxDesc* boxes, int nboxes, long long tile) {
  int lo = 0, hi = nboxes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (boxes[mid].tile_off <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// the brick of this block: 32 x sub_y x sub_z cells of one bin tile
struct Brick {
  BoxDesc bd;
  long long tile;
  int x0, y0, z0;  // first cell of the brick in its box
};

__device__ __forceinline__ Brick brick_of(const LbmArgs& a) {
  Brick k;
  const long long brick = a.reverse ? (long long)gridDim.x - 1 - blockIdx.x : (long long)blockIdx.x;
  k.tile = brick / a.nsub;
  const int sub = (int)(brick - k.tile * a.nsub);
  const int b = a.nboxes > 1 ? find_box(a.boxes, a.nboxes, k.tile) : 0;
  k.bd = a.boxes[b];
  const long long lt = k.tile - k.bd.tile_off;
  const int tx = (int)(lt % k.bd.ntx);
  const long long t2 = lt / k.bd.ntx;
  const int ty = (int)(t2 % k.bd.nty);
  const int tz = (int)(t2 / k.bd.nty);
  const int nsy = TILE_Y / a.sub_y;
  k.x0 = tx * TILE_X;
  k.y0 = ty * TILE_Y + (sub % nsy) * a.sub_y;
  k.z0 = tz * TILE_Z + (sub / nsy) * a.sub_z;
  return k;
}

// A capsule (the points within sqrt(r2) of the segment c +- h u, u a unit
// vector) that holds every cell a particle couples to (B > 0) and every cell
// inside it, used to skip cells and rows far from elongated particles.
//   sphere     radius a + eps/2, no segment
//   ellipsoid  B > 0 only where |x / a| < s = 1 + eps / (2 a_min) (there the
//              distance of Eq. B, (k - 1) k / |grad|, is at least (k - 1) a_min);
//              the ellipsoid scaled by s lies in the capsule along its longest
//              semi-axis a_k of radius s a_r and half-length s (a_k - a_r),
//              a_r the larger of the two others
//   cuboid     the box grown by eps/2 lies in the capsule along its longest
//              half-extent h_k of radius |(h_i, h_j)| + eps/2 and half-length h_k
//   capsule    itself grown by eps/2: radius a0 + eps/2 about its body-z segment
//   grid       the capsule about its body z axis that holds every grid cell
//              with a corner below eps/2 (computed when the grid is added)
// The radius carries a margin of 1e-3 relative + 0.01 cells over FP32 rounding.
struct Capsule {
  float u[3], h, r2;
};

__device__ __forceinline__ Capsule capsule_of(const Rec& R, float eps) {
  Capsule c;
  if (R.shape == 0) {
    c.u[0] = 1.0f; c.u[1] = c.u[2] = 0.0f;
    c.h = 0.0f;
    const float r = R.a[0] + 0.5f * eps;
    c.r2 = (r * 1.001f + 0.01f) * (r * 1.001f + 0.01f);
    return c;
  }
  if (R.shape == 4) {
    // the capsule about body z that holds every grid cell with a corner
    // below eps/2 (half-length and radius in the record's ia[1], ia[2])
    c.u[0] = R.M[2]; c.u[1] = R.M[5]; c.u[2] = R.M[8];
    c.h = R.ia[1];
    const float r = R.ia[2] * 1.001f + 0.01f;
    c.r2 = r * r;
    return c;
  }
  if (R.shape == 3) {
    c.u[0] = R.M[2]; c.u[1] = R.M[5]; c.u[2] = R.M[8];
    c.h = R.a[2];
    const float r = (R.a[0] + 0.5f * eps) * 1.001f + 0.01f;
    c.r2 = r * r;
    return c;
  }
  const int k = R.a[0] >= R.a[1] ? (R.a[0] >= R.a[2] ? 0 : 2) : (R.a[1] >= R.a[2] ? 1 : 2);
  const int i = k == 0 ? 1 : 0, j = k == 2 ? 1 : 2;
  // body axis k in world coordinates: column k of the body -> world rotation
  c.u[0] = R.M[k]; c.u[1] = R.M[3 + k]; c.u[2] = R.M[6 + k];
  float r;
  if (R.shape == 1) {
    const float s = 1.0f + 0.5f * eps / fminf(R.a[0], fminf(R.a[1], R.a[2]));
    const float ar = fmaxf(R.a[i], R.a[j]);
    r = s * ar;
    c.h = s * (R.a[k] - ar);
  } else {
    r = sqrtf(R.a[i] * R.a[i] + R.a[j] * R.a[j]) + 0.5f * eps;
    c.h = R.a[k];
  }
  r = r * 1.001f + 0.01f;
  c.r2 = r * r;
  return c;
}

// squared distance of offset r from the capsule's segment
__device__ __forceinline__ float capsule_dist2(const Capsule& c, float rx, float ry, float rz) {
  const float t = fminf(fmaxf(rx * c.u[0] + ry * c.u[1] + rz * c.u[2], -c.h), c.h);
  const float qx = rx - t * c.u[0], qy = ry - t * c.u[1], qz = rz - t * c.u[2];
  return qx * qx + qy * qy + qz * qz;
}

// squared distance of the x-parallel line through offset (., ry, rz) from
// the capsule's segment
__device__ __forceinline__ float capsule_row_dist2(const Capsule& c, float ry, float rz) {
  const float uu = c.u[1] * c.u[1] + c.u[2] * c.u[2];
  const float t = uu > 0.0f ? fminf(fmaxf((ry * c.u[1] + rz * c.u[2]) / uu, -c.h), c.h) : 0.0f;
  const float qy = ry - t * c.u[1], qz = rz - t * c.u[2];
  return qy * qy + qz * qz;
}

// Stage the particle candidates of the brick's tile in shared memory and
// mark, for each row (local y + sub_y * local z) of the brick, the
// candidates whose influence sphere meets the row.  Called by every thread
// of the block.
__device__ __forceinline__ void load_candidates(const LbmArgs& a, const Brick& k, Rec* srec,
                                                unsigned long long* s_rowmask) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nth = blockDim.x * blockDim.y;
  const int* ids = a.bin_ids + k.tile * (long long)a.bin_cap;
  // the tile's first 64 ids are read together with its count: one round
  // trip to L2 instead of two
  const int lane = tid & 31;
  const int id0 = lane < a.bin_cap ? ids[lane] : 0;
  const int id1 = 32 + lane < a.bin_cap ? ids[32 + lane] : 0;
  const int cnt = min(min(a.bin_count[k.tile], a.bin_cap), MAX_CAND);
  if (nth % 32 == 0) {
    // whole warps: a record is one word per lane; each warp copies up to
    // four records with their loads in flight before the stores
    const int wid = tid >> 5, nw = nth >> 5;
    for (int j0 = wid; j0 < cnt; j0 += 4 * nw) {
      int v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = j0 + u * nw;
        const int id = __shfl_sync(0xffffffffu, j < 32 ? id0 : id1, j & 31);
        v[u] = j < cnt ? reinterpret_cast<const int*>(&a.rec[id])[lane] : 0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = j0 + u * nw;
        if (j < cnt) reinterpret_cast<int*>(&srec[j])[lane] = v[u];
      }
    }
  } else {
    for (int e = tid; e < cnt * 32; e += nth) {
      const int j = e >> 5, w = e & 31;
      reinterpret_cast<int*>(&srec[j])[w] = reinterpret_cast<const int*>(&a.rec[ids[j]])[w];
    }
  }
  const int nrows = a.sub_y * a.sub_z;
  for (int r = tid; r < nrows; r += nth) s_rowmask[r] = 0ull;
  __syncthreads();
  // one (row, candidate) pair per thread: rows vary fastest, so a warp reads
  // one record and sets bits of distinct rows
  const BoxDesc& bd = k.bd;
  const float Ly = (float)bd.ny, Lz = (float)bd.nz;
  const int lr = __ffs(nrows) - 1, ly = __ffs(a.sub_y) - 1;  // sub_y, sub_z are powers of two
  for (int e = tid; e < (cnt << lr); e += nth) {
    const int r = e & (nrows - 1), j = e >> lr;
    const int yy = k.y0 + (r & (a.sub_y - 1));
    const int zz = k.z0 + (r >> ly);
    const Rec& R = srec[j];
    float r0y = (float)yy - R.xh[1], r0z = (float)zz - R.xh[2];
    if (!(bd.bc & 2)) { if (r0y > 0.5f * Ly) r0y -= Ly; else if (r0y < -0.5f * Ly) r0y += Ly; }
    if (!(bd.bc & 4)) { if (r0z > 0.5f * Lz) r0z -= Lz; else if (r0z < -0.5f * Lz) r0z += Lz; }
    const float ry = __fsub_rn(r0y, R.xl[1]), rz = __fsub_rn(r0z, R.xl[2]);
    if (ry * ry + rz * rz < R.rinf2) {
      bool hit = true;
      if (R.shape != 0) {
        const Capsule c = capsule_of(R, a.eps);
        hit = capsule_row_dist2(c, ry, rz) < c.r2;
      }
      if (hit) atomicOr(&s_rowmask[r], 1ull << j);
    }
  }
  __syncthreads();
}

// Coupling of N consecutive cells x, x+1, .. of one row with the candidates
// in rm: the largest indicator B (ties to the lowest particle id) with its
// particle velocity u_p(x) = U + w x (x - X) (Eq. hlbm:du), and up to two
// particles whose inside holds the cell's centre.
template <int N>
struct RowCoupling {
  float B[N], upx[N], upy[N], upz[N];
  int bestp[N], ip0[N], ip1[N];
};

template <int N, bool GRIDS>
__device__ __forceinline__ void couple_row(const Rec* srec, unsigned long long rm, const BoxDesc& bd,
                                           int x, int y, int z, float eps, float inv_eps, int* status,
                                           RowCoupling<N>& cc, GridSet grids) {
  // without grid particles the grid branches fold away (null grid set)
  const GridSet gs = GRIDS ? grids : GridSet{};
#pragma unroll
  for (int j = 0; j < N; ++j) {
    cc.B[j] = 0.0f;
    cc.upx[j] = cc.upy[j] = cc.upz[j] = 0.0f;
    cc.bestp[j] = 0x7fffffff;
    cc.ip0[j] = cc.ip1[j] = -1;
  }
  const float Lx = (float)bd.nx, Ly = (float)bd.ny, Lz = (float)bd.nz;
  while (rm) {
    const int k = __ffsll((long long)rm) - 1;
    rm &= rm - 1;
    const Rec& R = srec[k];
    float r0y = (float)y - R.xh[1], r0z = (float)z - R.xh[2];
    if (!(bd.bc & 2)) { if (r0y > 0.5f * Ly) r0y -= Ly; else if (r0y < -0.5f * Ly) r0y += Ly; }
    if (!(bd.bc & 4)) { if (r0z > 0.5f * Lz) r0z -= Lz; else if (r0z < -0.5f * Lz) r0z += Lz; }
    const float ry = __fsub_rn(r0y, R.xl[1]), rz = __fsub_rn(r0z, R.xl[2]);
    const float d2 = ry * ry + rz * rz;
    // the cell's coupling to R: the particle id if its centre is inside, and
    // the indicator with the particle velocity there when it is the largest
    auto take = [&](int j, float rx, bool in, float B) {
      if (in) {
        if (cc.ip0[j] < 0) cc.ip0[j] = R.pid;
        else if (cc.ip1[j] < 0) cc.ip1[j] = R.pid;
        else atomicOr(status, ST_OVERLAP);  // three overlapping particles
      }
      if (B > cc.B[j] || (B == cc.B[j] && B > 0.0f && R.pid < cc.bestp[j])) {
        cc.B[j] = B;
        cc.bestp[j] = R.pid;
        cc.upx[j] = R.u[0] + (R.w[1] * rz - R.w[2] * ry);
        cc.upy[j] = R.u[1] + (R.w[2] * rx - R.w[0] * rz);
        cc.upz[j] = R.u[2] + (R.w[0] * ry - R.w[1] * rx);
      }
    };
    auto arm_x = [&](int j) {
      float r0x = (float)(x + j) - R.xh[0];
      if (!(bd.bc & 1)) { if (r0x > 0.5f * Lx) r0x -= Lx; else if (r0x < -0.5f * Lx) r0x += Lx; }
      return __fsub_rn(r0x, R.xl[0]);
    };
    // The inside decision is the exactly rounded test of inside_from_offset;
    // away from the surface the distance evaluated here (contracted
    // arithmetic) has the same sign, and only cells within a margin far above
    // the rounding difference of the two take the exact test (sphere: 1e-5
    // relative in r^2; other shapes: 1e-3 cells).
    if (R.shape == 0) {
      // a sphere's indicator is 1 within r <= a - eps/2 and 0 beyond a + eps/2:
      // only cells in that shell need the distance and the ramp (bounds
      // precomputed in the record)
      const float in_lo = R.M[SPH_IN_LO], in_hi = R.M[SPH_IN_HI];
      const float r2_in = R.M[SPH_R2_IN], r2_out = R.M[SPH_R2_OUT];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const float rx = arm_x(j);
        const float r2 = rx * rx + d2;
        if (r2 < R.rinf2) {
          bool in;
          if (r2 < in_lo) in = true;
          else if (r2 > in_hi) in = false;
          else { const float rr[3] = {rx, ry, rz}; in = inside_from_offset(R, rr); }
          const float B = r2 <= r2_in ? 1.0f : (r2 >= r2_out ? 0.0f : indicator(sdf(R, rx, ry, rz, r2), eps, inv_eps));
          take(j, rx, in, B);
        }
      }
    } else {
      // elongated shapes: cells outside the enclosing capsule neither couple
      // nor lie inside
      const Capsule cap = capsule_of(R, eps);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const float rx = arm_x(j);
        const float r2 = rx * rx + d2;
        if (r2 < R.rinf2 && capsule_dist2(cap, rx, ry, rz) < cap.r2) {
          const float d = sdf(R, rx, ry, rz, r2, gs);
          bool in;
          if (d < -1e-3f) in = true;
          else if (d > 1e-3f) in = false;
          else { const float rr[3] = {rx, ry, rz}; in = inside_from_offset(R, rr, gs); }
          take(j, rx, in, indicator(d, eps, inv_eps));
        }
      }
    }
  }
}

__device__ __forceinline__ unsigned lane_id() {
  unsigned l;
  asm("mov.u32 %0, %%laneid;" : "=r"(l));
  return l;
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Warp-aggregated append of the cells g, g+1, .. g+N-1 that lie inside a
// particle to the list of interior cells: one entry (cell, particle) per
// particle holding the cell, with the mass and momentum of the cell's
// post-collision deviations as stored.  Called by all active lanes, which
// may be any subset of the warp: a lane's offset among the warp's entries
// is taken bit by bit of its entry count (one ballot per bit), so no lane
// depends on a value passed through another.
template <int N>
__device__ __forceinline__ void append_interior(const LbmArgs& a, unsigned g, const RowCoupling<N>& cc,
                                                const float4 (&mom)[N]) {
  int nent = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) nent += (cc.ip0[j] >= 0) + (cc.ip1[j] >= 0);
  const unsigned act = __activemask();
  if (!__ballot_sync(act, nent > 0)) return;
  const unsigned lt = lanemask_lt();
  int before = 0, total = 0;
#pragma unroll
  for (int b = 0; (1 << b) <= 2 * N; ++b) {
    const unsigned m = __ballot_sync(act, (nent >> b) & 1);
    before += __popc(m & lt) << b;
    total += __popc(m) << b;
  }
  const int leader = __ffs(act) - 1;
  const int stripe = (int)(blockIdx.x & (ILIST_STRIPES - 1));
  int base = 0;
  if ((int)lane_id() == leader) base = atomicAdd(&a.ilist_count[stripe], total);
  base = __shfl_sync(act, base, leader);
  long long k = (long long)base + before;  // within the stripe
  const long long k0 = (long long)stripe * a.ilist_cap;
#pragma unroll
  for (int j = 0; j < N; ++j) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int p = e == 0 ? cc.ip0[j] : cc.ip1[j];
      if (p >= 0) {
        if (k < a.ilist_cap) {
          a.ilist_idx[k0 + k] = make_int2((int)(g + j), p);
          a.ilist_mom[k0 + k] = mom[j];
        } else {
          atomicOr(a.status, ST_LIST_FULL);
        }
        ++k;
      }
    }
  }
}

}  // namespace hlbm
