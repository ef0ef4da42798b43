// lbm_kernels.cu -- fused D3Q19 collide-and-stream with HLBM coupling.
//
// One kernel per step does, for every cell (arXiv:2312.14172):
//   rho = sum_i f_i, rho u = sum_i c_i f_i                       (Sec. 3.1)
//   B = max_p B_p(d_s,p(x)), u_p(x) = U + omega x (x - X)        (Eq. B, Sec. 3.2)
//   Delta u = B (u_p - u) + F_f / rho                            (Eq. hlbm:du)
//   f*_i = f_i - (f_i - f^eq_i(rho, u)) / tau
//          + f^eq_i(rho, u + Delta u) - f^eq_i(rho, u)           (Eqs. collide, bgk, kupershtokh)
//   f_i(x + c_i, t + 1) = f*_i(x, t), half-way bounce-back at walls (Eq. stream)
// in the in-place AA pattern: even steps read and write only the cell's own
// slots (the post-collision value of direction i goes to slot ibar), odd
// steps read from and write to the neighbours.  Populations are stored as
// deviations d_i = f_i - w_i (float, or half scaled by 2^s); all arithmetic
// is FP32 on deviations, which keeps the small non-equilibrium parts exact to
// FP32 rounding instead of to the rounding of f ~ w_i.
#include "hlbm_internal.cuh"

namespace hlbm {

constexpr int MAX_CAND = 64;  // particle records staged per block
#ifndef HLBM_CS_MINBLOCKS
#define HLBM_CS_MINBLOCKS 3
#endif

template <typename S> struct Pop;
template <> struct Pop<float> {
  static __device__ __forceinline__ float ld(const float* p, float) { return *p; }
  static __device__ __forceinline__ void st(float* p, float v, float) { *p = v; }
};
template <> struct Pop<__half> {
  static __device__ __forceinline__ float ld(const __half* p, float inv_s) {
    return __half2float(*p) * inv_s;
  }
  static __device__ __forceinline__ void st(__half* p, float v, float s) { *p = __float2half_rn(v * s); }
};
// the value a store of v leaves in memory, read back as a deviation
template <typename S>
__device__ __forceinline__ float stored_value(float v, float s, float inv_s) {
  if (sizeof(S) == 4) return v;
  return __half2float(__float2half_rn(v * s)) * inv_s;
}

// indicator of Eq. B written as (1 - sin(pi d / eps)) / 2 on the ramp, which
// equals cos^2((pi/2)(d/eps + 1/2))
__device__ __forceinline__ float indicator(float d, float eps, float inv_eps) {
  if (d <= -0.5f * eps) return 1.0f;
  if (d >= 0.5f * eps) return 0.0f;
  return 0.5f - 0.5f * sinpif(d * inv_eps);
}

// signed distance of a particle at offset r (world frame), FP32
__device__ __forceinline__ float sdf(const Rec& R, float rx, float ry, float rz, float r2) {
  if (R.shape == 0) return sqrtf(r2) - R.a[0];
  // body frame b = M^T r
  const float b0 = R.M[0] * rx + R.M[3] * ry + R.M[6] * rz;
  const float b1 = R.M[1] * rx + R.M[4] * ry + R.M[7] * rz;
  const float b2 = R.M[2] * rx + R.M[5] * ry + R.M[8] * rz;
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

// ---------------------------------------------------------------------------
// Momentum exchange of the next step, fused into this collision.
//
// The force of Eq. hlbm:mea on particle p at step k + 1 is, over the cells x
// inside p (the used sign, see the momentum-exchange kernel),
//   F = sum_x sum_i (c_i - u_p(x)) f_i(x) + (c_i + u_p(x)) f_ibar(x - c_i)
// on the post-streaming populations of step k + 1.  Those are this step's
// post-collision values: f_i(x) = f*_i(x - c_i) and f_ibar(x - c_i) = f*_ibar(x).
// Re-indexed by the cell z whose thread holds f*_j(z) (g_j = f*_j - w_j):
//   arrival   z + c_j inside:  (c_j - u_p(z + c_j)) g_j, arm r(z) + c_j
//   departure z inside:        (-c_j + u_p(z)) g_j,     arm r(z)
// With u_p(z + c_j) = u_p(z) + w x c_j, and the masked sums over arrivals
// S0 = sum g_j, S1 = sum c_j g_j, S2 = sum |c_j|^2 g_j, M = sum g_j c_j c_j^T:
//   F_arr = S1 - u_p S0 - w x S1
//   T_arr = r x F_arr - S1 x u_p - (w S2 - M w)
//   F_dep = -S1' + u_p S0' + sum_(links into a wall) 2 c_j w_j,  T_dep = r x F_dep
// (primed sums over the links that do not end beyond a wall).  The weights'
// share cancels pairwise on every link whose both halves are counted.
// The inside decisions reuse the exact FP32 recipe of the inside test for the
// cell and its 18 neighbours, so both paths select the same cells.

struct AxisOff {
  float v[3];  // r - X component for the neighbour offsets -1, 0, +1
  bool ok[3];  // the neighbour exists (not beyond a wall)
};

__device__ __forceinline__ AxisOff axis_offsets(int x, int n, bool wall, float xh, float xl) {
  AxisOff a;
  const float r0 = __fsub_rn((float)x, xh);
  const float L = (float)n, half = __fmul_rn(0.5f, L);
#pragma unroll
  for (int d = -1; d <= 1; ++d) {
    float t = __fadd_rn(r0, (float)d);
    if (!wall) {
      if (t > half) t = __fsub_rn(t, L);
      else if (t < -half) t = __fadd_rn(t, L);
    }
    a.v[d + 1] = __fsub_rn(t, xl);
    a.ok[d + 1] = !wall || (x + d >= 0 && x + d < n);
  }
  return a;
}

// bit i set: the cell at offset c_i (i = 0: the cell itself) is inside
__device__ __forceinline__ unsigned inside_mask(const Rec& R, const AxisOff& X, const AxisOff& Y,
                                                const AxisOff& Z) {
  unsigned m = 0;
  if (R.shape == 0) {
    float sx[3], sy[3], sz[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      sx[d] = __fmul_rn(X.v[d], X.v[d]);
      sy[d] = __fmul_rn(Y.v[d], Y.v[d]);
      sz[d] = __fmul_rn(Z.v[d], Z.v[d]);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const float s2 = __fadd_rn(__fadd_rn(sx[cx(i) + 1], sy[cy(i) + 1]), sz[cz(i) + 1]);
      m |= (s2 < R.in2 ? 1u : 0u) << i;
    }
    return m;
  }
  float px[3][3], py[3][3], pz[3][3];  // [body component][offset]
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      px[j][d] = __fmul_rn(R.M[0 * 3 + j], X.v[d]);
      py[j][d] = __fmul_rn(R.M[1 * 3 + j], Y.v[d]);
      pz[j][d] = __fmul_rn(R.M[2 * 3 + j], Z.v[d]);
    }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    float b[3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
      b[j] = __fadd_rn(__fadd_rn(px[j][cx(i) + 1], py[j][cy(i) + 1]), pz[j][cz(i) + 1]);
    bool in;
    if (R.shape == 1) {
      const float e0 = __fmul_rn(b[0], R.ia[0]), e1 = __fmul_rn(b[1], R.ia[1]), e2 = __fmul_rn(b[2], R.ia[2]);
      const float s2 = __fadd_rn(__fadd_rn(__fmul_rn(e0, e0), __fmul_rn(e1, e1)), __fmul_rn(e2, e2));
      in = s2 < 1.0f;
    } else {
      in = fabsf(b[0]) < R.a[0] && fabsf(b[1]) < R.a[1] && fabsf(b[2]) < R.a[2];
    }
    m |= (in ? 1u : 0u) << i;
  }
  return m;
}

// force and torque of one cell's post-collision deviations g on a particle
__device__ __forceinline__ void mea_contribution(const Rec& R, const float g[Q], unsigned inm,
                                                 unsigned okm, float rx, float ry, float rz,
                                                 float F[3], float T[3]) {
  float S0 = 0.f, S1x = 0.f, S1y = 0.f, S1z = 0.f, S2 = 0.f;
  float Mxx = 0.f, Myy = 0.f, Mzz = 0.f, Mxy = 0.f, Mxz = 0.f, Myz = 0.f;
  float B0 = 0.f, B1x = 0.f, B1y = 0.f, B1z = 0.f, cwx = 0.f, cwy = 0.f, cwz = 0.f;
  const unsigned arr = inm & okm;
#pragma unroll
  for (int j = 1; j < Q; ++j) {
    const float gj = ((arr >> j) & 1u) ? g[j] : 0.0f;
    S0 += gj;
    if (cx(j)) { S1x += (float)cx(j) * gj; Mxx += gj; }
    if (cy(j)) { S1y += (float)cy(j) * gj; Myy += gj; }
    if (cz(j)) { S1z += (float)cz(j) * gj; Mzz += gj; }
    S2 += (float)(cx(j) * cx(j) + cy(j) * cy(j) + cz(j) * cz(j)) * gj;
    if (cx(j) && cy(j)) Mxy += (float)(cx(j) * cy(j)) * gj;
    if (cx(j) && cz(j)) Mxz += (float)(cx(j) * cz(j)) * gj;
    if (cy(j) && cz(j)) Myz += (float)(cy(j) * cz(j)) * gj;
    const bool ok = (okm >> j) & 1u;
    const float gb = ok ? g[j] : 0.0f;
    B0 += gb;
    if (cx(j)) B1x += (float)cx(j) * gb;
    if (cy(j)) B1y += (float)cy(j) * gb;
    if (cz(j)) B1z += (float)cz(j) * gb;
    if (!ok) {
      const float w2 = 2.0f * (float)wq(j);
      cwx += (float)cx(j) * w2;
      cwy += (float)cy(j) * w2;
      cwz += (float)cz(j) * w2;
    }
  }
  const float wx = R.w[0], wy = R.w[1], wz = R.w[2];
  const float upx = R.u[0] + (wy * rz - wz * ry);
  const float upy = R.u[1] + (wz * rx - wx * rz);
  const float upz = R.u[2] + (wx * ry - wy * rx);
  // arrivals
  float Fx = S1x - upx * S0 - (wy * S1z - wz * S1y);
  float Fy = S1y - upy * S0 - (wz * S1x - wx * S1z);
  float Fz = S1z - upz * S0 - (wx * S1y - wy * S1x);
  const float Mwx = Mxx * wx + Mxy * wy + Mxz * wz;
  const float Mwy = Mxy * wx + Myy * wy + Myz * wz;
  const float Mwz = Mxz * wx + Myz * wy + Mzz * wz;
  float Tx = (ry * Fz - rz * Fy) - (S1y * upz - S1z * upy) - (wx * S2 - Mwx);
  float Ty = (rz * Fx - rx * Fz) - (S1z * upx - S1x * upz) - (wy * S2 - Mwy);
  float Tz = (rx * Fy - ry * Fx) - (S1x * upy - S1y * upx) - (wz * S2 - Mwz);
  // departures, when the cell itself is inside
  if (inm & 1u) {
    const float Gx = -B1x + upx * B0 + cwx, Gy = -B1y + upy * B0 + cwy, Gz = -B1z + upz * B0 + cwz;
    Fx += Gx;
    Fy += Gy;
    Fz += Gz;
    Tx += ry * Gz - rz * Gy;
    Ty += rz * Gx - rx * Gz;
    Tz += rx * Gy - ry * Gx;
  }
  F[0] = Fx; F[1] = Fy; F[2] = Fz;
  T[0] = Tx; T[1] = Ty; T[2] = Tz;
}

template <typename S, int PAR, bool WALLS, bool COUPLE>
__global__ void __launch_bounds__(256, HLBM_CS_MINBLOCKS) collide_stream_kernel(LbmArgs a) {
  constexpr int NW = 8;  // at most 8 warps per block (32 x sub_y threads)
  __shared__ Rec srec[COUPLE ? MAX_CAND : 1];
  __shared__ float s_rout2[COUPLE ? MAX_CAND : 1], s_rfull2[COUPLE ? MAX_CAND : 1];
  __shared__ float s_rrow2[COUPLE ? MAX_CAND : 1];
  __shared__ float s_acc[COUPLE ? NW : 1][COUPLE ? MAX_CAND : 1][6];
  const long long brick = blockIdx.x;
  const long long tile = brick / a.nsub;
  const int sub = (int)(brick - tile * a.nsub);
  const int b = a.nboxes > 1 ? find_box(a.boxes, a.nboxes, tile) : 0;
  const BoxDesc bd = a.boxes[b];
  const long long lt = tile - bd.tile_off;
  const int tx = (int)(lt % bd.ntx);
  const long long t2 = lt / bd.ntx;
  const int ty = (int)(t2 % bd.nty);
  const int tz = (int)(t2 / bd.nty);
  const int nsy = TILE_Y / a.sub_y;
  const int sy = sub % nsy, sz = sub / nsy;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nth = blockDim.x * blockDim.y;
  const int lane = threadIdx.x, warp = threadIdx.y;

  int cnt = 0;
  if (COUPLE) {
    cnt = min(min(a.bin_count[tile], a.bin_cap), MAX_CAND);
    const int* ids = a.bin_ids + tile * (long long)a.bin_cap;
    for (int k = tid; k < cnt * 32; k += nth) {
      const int j = k >> 5, e = k & 31;
      reinterpret_cast<int*>(&srec[j])[e] = reinterpret_cast<const int*>(&a.rec[ids[j]])[e];
    }
    for (int k = tid; k < NW * cnt * 6; k += nth) (&s_acc[0][0][0])[(k / (cnt * 6)) * MAX_CAND * 6 + k % (cnt * 6)] = 0.0f;
    __syncthreads();
    for (int k = tid; k < cnt; k += nth) {
      const Rec& R = srec[k];
      const float amin = fminf(R.a[0], fminf(R.a[1], R.a[2]));
      const float amax = fmaxf(R.a[0], fmaxf(R.a[1], R.a[2]));
      const float rcirc = R.shape == 2 ? sqrtf(R.a[0] * R.a[0] + R.a[1] * R.a[1] + R.a[2] * R.a[2]) : amax;
      // beyond r_c + 1.5 no neighbour is inside; within r_in - 1.5 all are
      s_rout2[k] = (rcirc + 1.5f) * (rcirc + 1.5f);
      const float rf = fmaxf(amin - 1.5f, 0.0f);
      s_rfull2[k] = rf * rf;
      s_rrow2[k] = fmaxf(R.rinf2, s_rout2[k]);
    }
    __syncthreads();
  }

  const int x = tx * TILE_X + threadIdx.x;
  const int y = ty * TILE_Y + sy * a.sub_y + threadIdx.y;
  const bool valid = x < bd.nx && y < bd.ny;
  if (!COUPLE && !valid) return;
  const int z0 = tz * TILE_Z + sz * a.sub_z;
  const int z1 = min(z0 + a.sub_z, bd.nz);
  S* __restrict__ f = reinterpret_cast<S*>(a.f) + bd.cell_off;
  const long long P = a.plane;
  const float Lx = (float)bd.nx, Ly = (float)bd.ny, Lz = (float)bd.nz;

  for (int z = z0; z < z1; ++z) {
    float o[Q];
    unsigned long long nearm = 0;  // candidates whose momentum exchange this cell feeds
    if (valid) {
      const int c = (z * bd.ny + y) * bd.nx + x;
      Nbr<WALLS> nb;
      if (PAR == 1) nb = make_nbr<WALLS>(bd, x, y, z);
      float d[Q];
      // load the post-streaming deviations f_i(x) - w_i
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if (PAR == 0) {
          d[i] = Pop<S>::ld(f + i * P + c, a.inv_scale);
        } else {
          const int src = (i == 0) ? c : nb.at(-cx(i), -cy(i), -cz(i));
          d[i] = (src >= 0) ? Pop<S>::ld(f + opp(i) * P + src, a.inv_scale)
                            : Pop<S>::ld(f + i * P + c, a.inv_scale);
        }
      }
      float drho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        drho += d[i];
        if (cx(i)) jx += (float)cx(i) * d[i];
        if (cy(i)) jy += (float)cy(i) * d[i];
        if (cz(i)) jz += (float)cz(i) * d[i];
      }
      const float rho = 1.0f + drho;
      if (!(rho > 0.0f && rho < 1e30f)) atomicOr(a.status, ST_UNSTABLE);
      const float irho = 1.0f / rho;
      const float ux = jx * irho, uy = jy * irho, uz = jz * irho;
      float dux = a.ff[0] * irho, duy = a.ff[1] * irho, duz = a.ff[2] * irho;
      if (COUPLE) {
        float bestB = 0.0f, upx = 0.0f, upy = 0.0f, upz = 0.0f;
        int bestp = 0x7fffffff;
        for (int k = 0; k < cnt; ++k) {
          const Rec& R = srec[k];
          // y and z offsets are the same for the whole warp (one row of x):
          // most candidates miss the row and are rejected without divergence
          float r0y = (float)y - R.xh[1], r0z = (float)z - R.xh[2];
          if (!(bd.bc & 2)) { if (r0y > 0.5f * Ly) r0y -= Ly; else if (r0y < -0.5f * Ly) r0y += Ly; }
          if (!(bd.bc & 4)) { if (r0z > 0.5f * Lz) r0z -= Lz; else if (r0z < -0.5f * Lz) r0z += Lz; }
          const float ry = r0y - R.xl[1], rz = r0z - R.xl[2];
          const float d2 = ry * ry + rz * rz;
          if (d2 >= s_rrow2[k]) continue;
          float r0x = (float)x - R.xh[0];
          if (!(bd.bc & 1)) { if (r0x > 0.5f * Lx) r0x -= Lx; else if (r0x < -0.5f * Lx) r0x += Lx; }
          const float rx = r0x - R.xl[0];
          const float r2 = rx * rx + d2;
          if (r2 < s_rout2[k]) nearm |= 1ull << k;
          if (r2 < R.rinf2) {
            const float B = indicator(sdf(R, rx, ry, rz, r2), a.eps, a.inv_eps);
            if (B > bestB || (B == bestB && B > 0.0f && R.pid < bestp)) {
              bestB = B;
              bestp = R.pid;
              upx = R.u[0] + (R.w[1] * rz - R.w[2] * ry);
              upy = R.u[1] + (R.w[2] * rx - R.w[0] * rz);
              upz = R.u[2] + (R.w[0] * ry - R.w[1] * rx);
            }
          }
        }
        if (bestB > 0.0f) {
          dux += bestB * (upx - ux);
          duy += bestB * (upy - uy);
          duz += bestB * (upz - uz);
        }
      }
      // f*_i - w_i = (1 - 1/tau) (d_i - E_i(u)) + E_i(u + Delta u), E = f^eq - w.
      // Opposite directions share the even part of E and flip the odd part:
      // E_i = w drho + w rho (4.5 (c.u)^2 - 1.5 u.u) +- 3 w rho (c.u)
      const float om1 = 1.0f - a.omega;
      const float vx = ux + dux, vy = uy + duy, vz = uz + duz;
      const float usq = 1.5f * (ux * ux + uy * uy + uz * uz);
      const float vsq = 1.5f * (vx * vx + vy * vy + vz * vz);
      {
        constexpr float w0 = 1.0f / 3.0f;
        const float eu = w0 * drho - w0 * rho * usq, ev = w0 * drho - w0 * rho * vsq;
        o[0] = om1 * d[0] + (ev - om1 * eu);
      }
      const float wr1 = rho * (1.0f / 18.0f), wd1 = drho * (1.0f / 18.0f);
      const float wr2 = rho * (1.0f / 36.0f), wd2 = drho * (1.0f / 36.0f);
#define HLBM_PAIR(I, WR, WD, CU, CV)                                          \
      {                                                                       \
        const float cu_ = (CU), cv_ = (CV);                                   \
        const float eu = WD + WR * (4.5f * cu_ * cu_ - usq);                  \
        const float ev = WD + WR * (4.5f * cv_ * cv_ - vsq);                  \
        const float C = ev - om1 * eu;                                        \
        const float A = 3.0f * WR * (cv_ - om1 * cu_);                        \
        o[I] = om1 * d[I] + C + A;                                            \
        o[I + 1] = om1 * d[I + 1] + C - A;                                    \
      }
      HLBM_PAIR(1, wr1, wd1, ux, vx)
      HLBM_PAIR(3, wr1, wd1, uy, vy)
      HLBM_PAIR(5, wr1, wd1, uz, vz)
      HLBM_PAIR(7, wr2, wd2, ux + uy, vx + vy)
      HLBM_PAIR(9, wr2, wd2, ux - uy, vx - vy)
      HLBM_PAIR(11, wr2, wd2, ux + uz, vx + vz)
      HLBM_PAIR(13, wr2, wd2, ux - uz, vx - vz)
      HLBM_PAIR(15, wr2, wd2, uy + uz, vy + vz)
      HLBM_PAIR(17, wr2, wd2, uy - uz, vy - vz)
#undef HLBM_PAIR
      // store the post-collision deviations, streamed (AA pattern)
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if (PAR == 0) {
          Pop<S>::st(f + opp(i) * P + c, o[i], a.scale);
        } else {
          const int dst = (i == 0) ? c : nb.at(cx(i), cy(i), cz(i));
          if (dst >= 0) Pop<S>::st(f + i * P + dst, o[i], a.scale);
          else Pop<S>::st(f + opp(i) * P + c, o[i], a.scale);
        }
      }
    }
    if (COUPLE) {
      // momentum exchange of the next step from this cell's outgoing values,
      // for the candidates some lane of the warp is near
      unsigned long long wm = (unsigned long long)__reduce_or_sync(0xffffffffu, (unsigned)nearm) |
                              ((unsigned long long)__reduce_or_sync(0xffffffffu, (unsigned)(nearm >> 32)) << 32);
      while (wm) {
        const int k = __ffsll((long long)wm) - 1;
        wm &= wm - 1;
        const Rec& R = srec[k];
        float F[3] = {0.f, 0.f, 0.f}, T[3] = {0.f, 0.f, 0.f};
        if ((nearm >> k) & 1ull) {
          const AxisOff AX = axis_offsets(x, bd.nx, bd.bc & 1, R.xh[0], R.xl[0]);
          const AxisOff AY = axis_offsets(y, bd.ny, bd.bc & 2, R.xh[1], R.xl[1]);
          const AxisOff AZ = axis_offsets(z, bd.nz, bd.bc & 4, R.xh[2], R.xl[2]);
          const float rx = AX.v[1], ry = AY.v[1], rz = AZ.v[1];
          const float d2 = rx * rx + ry * ry + rz * rz;
          const unsigned inm = d2 < s_rfull2[k] ? 0x7ffffu : inside_mask(R, AX, AY, AZ);
          if (inm) {
            unsigned okm = 0x7ffffu;
            if (WALLS) {
              okm = 0;
#pragma unroll
              for (int i = 0; i < Q; ++i)
                okm |= (AX.ok[cx(i) + 1] && AY.ok[cy(i) + 1] && AZ.ok[cz(i) + 1] ? 1u : 0u) << i;
            }
            float g[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) g[i] = stored_value<S>(o[i], a.scale, a.inv_scale);
            mea_contribution(R, g, inm, okm, rx, ry, rz, F, T);
          }
        }
        float v[6] = {F[0], F[1], F[2], T[0], T[1], T[2]};
#pragma unroll
        for (int q = 0; q < 6; ++q)
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
        if (lane == 0)
#pragma unroll
          for (int q = 0; q < 6; ++q) s_acc[warp][k][q] += v[q];
      }
    }
  }
  if (COUPLE) {
    __syncthreads();
    const int nw = blockDim.y;
    for (int t = tid; t < cnt * 6; t += nth) {
      const int k = t / 6, q = t - k * 6;
      float sum = 0.0f;
      for (int w = 0; w < nw; ++w) sum += s_acc[w][k][q];
      if (sum != 0.0f) atomicAdd(&a.acc[(long long)srec[k].pid * 6 + q], (double)sum);
    }
  }
}

// logical populations of a range of cells of one box
template <typename S, int PAR, bool GATHER>
__global__ void gather_scatter_kernel(LbmArgs a, int box, long long c0, long long n, float* stage) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const BoxDesc bd = a.boxes[box];
  const long long cl = c0 + k;
  const int x = (int)(cl % bd.nx);
  const long long t = cl / bd.nx;
  const int y = (int)(t % bd.ny);
  const int z = (int)(t / bd.ny);
  const int c = (int)cl;
  S* f = reinterpret_cast<S*>(a.f) + bd.cell_off;
  const long long P = a.plane;
  const Nbr<true> nb = make_nbr<true>(bd, x, y, z);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    S* slot;
    if (PAR == 0 || i == 0) {
      slot = f + i * P + c;
    } else {
      const int src = nb.at(-cx(i), -cy(i), -cz(i));
      slot = (src >= 0) ? f + opp(i) * P + src : f + i * P + c;
    }
    if (GATHER) stage[i * n + k] = Pop<S>::ld(slot, a.inv_scale);
    else Pop<S>::st(slot, stage[i * n + k], a.scale);
  }
}

template <typename S, int PAR, bool W, bool C>
static cudaError_t launch_cs(const LbmArgs& a, cudaStream_t s) {
  dim3 block(TILE_X, a.sub_y);
  collide_stream_kernel<S, PAR, W, C><<<(unsigned)a.nbricks, block, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename S>
static cudaError_t launch_cs_prec(const LbmArgs& a, int parity, bool walls, bool couple,
                                  cudaStream_t s) {
  if (parity == 0) {
    // even steps never touch a neighbour: walls need no special case
    return couple ? launch_cs<S, 0, false, true>(a, s) : launch_cs<S, 0, false, false>(a, s);
  }
  if (walls) return couple ? launch_cs<S, 1, true, true>(a, s) : launch_cs<S, 1, true, false>(a, s);
  return couple ? launch_cs<S, 1, false, true>(a, s) : launch_cs<S, 1, false, false>(a, s);
}

cudaError_t launch_collide(const LbmArgs& a, int precision, int parity, bool walls, bool couple,
                           cudaStream_t s) {
  if (a.nbricks <= 0) return cudaSuccess;
  return precision == 0 ? launch_cs_prec<float>(a, parity, walls, couple, s)
                        : launch_cs_prec<__half>(a, parity, walls, couple, s);
}

template <typename S, bool G>
static cudaError_t launch_gs(const LbmArgs& a, int parity, int box, long long c0, long long n,
                             float* stage, cudaStream_t s) {
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (parity == 0) gather_scatter_kernel<S, 0, G><<<blocks, 256, 0, s>>>(a, box, c0, n, stage);
  else gather_scatter_kernel<S, 1, G><<<blocks, 256, 0, s>>>(a, box, c0, n, stage);
  return cudaGetLastError();
}

cudaError_t launch_gather(const LbmArgs& a, int precision, int parity, int box, long long c0,
                          long long n, float* stage, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  return precision == 0 ? launch_gs<float, true>(a, parity, box, c0, n, stage, s)
                        : launch_gs<__half, true>(a, parity, box, c0, n, stage, s);
}

cudaError_t launch_scatter(const LbmArgs& a, int precision, int parity, int box, long long c0,
                           long long n, const float* stage, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  float* st = const_cast<float*>(stage);
  return precision == 0 ? launch_gs<float, false>(a, parity, box, c0, n, st, s)
                        : launch_gs<__half, false>(a, parity, box, c0, n, st, s);
}

}  // namespace hlbm
