// lbm_pair_kernels.cu -- the fused collide-and-stream of lbm_kernels.cu
// (Eqs. collide, bgk, maxbolt, kupershtokh, stream; coupling of Eqs. B and
// hlbm:du) with two x-adjacent cells (x0, x0 + 1), x0 even, per thread.
//
// The two cells share every y/z offset, so a thread issues one 8-byte
// (float) or 4-byte (half) access for both cells wherever their two slots
// are adjacent in memory: all 19 loads and stores of an even step, and the 9
// directions with c_x = 0 of an odd step.  The 10 directions with c_x != 0
// of an odd step reach x0 - 1 .. x0 + 2 and take one access per cell.  All
// FP32 arithmetic of the collision runs on float2 with the packed FP32x2
// instructions of sm_100 and later (__ffma2_rn, __fadd2_rn, __fmul2_rn),
// one instruction for both cells.  A block is 16 x sub_y threads over the
// same 32 x sub_y x sub_z brick as the one-cell kernel.
#include <type_traits>

#include "lbm_common.cuh"

namespace hlbm {

#ifndef HLBM_CP_MINBLOCKS_F32
#define HLBM_CP_MINBLOCKS_F32 4
#endif
#ifndef HLBM_CP_MINBLOCKS_F16
#define HLBM_CP_MINBLOCKS_F16 5
#endif

namespace {

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b, rounded once: b * (-1) is exact
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// The two cells' values of one slot as held in registers between load and
// store: float2 for float storage; for half storage the packed __half2
// itself (one register), widened to float2 where the arithmetic reads it.
template <typename S> struct Two;
template <> struct Two<float> {
  using raw = float2;
  static __device__ __forceinline__ float lo(raw v) { return v.x; }
  static __device__ __forceinline__ void st1(float* p, float v) { *p = v; }
  static __device__ __forceinline__ raw ld(const float* p) { return *reinterpret_cast<const float2*>(p); }
  static __device__ __forceinline__ raw ld(const float* pa, const float* pb) { return make_float2(*pa, *pb); }
  static __device__ __forceinline__ float2 val(raw v) { return v; }
  static __device__ __forceinline__ raw pack(float2 v) { return v; }
  static __device__ __forceinline__ void st(float* p, raw v) { *reinterpret_cast<float2*>(p) = v; }
  static __device__ __forceinline__ void st(float* pa, float* pb, raw v) { *pa = v.x; *pb = v.y; }
};
template <> struct Two<__half> {
  using raw = __half2;
  static __device__ __forceinline__ __half lo(raw v) { return __low2half(v); }
  static __device__ __forceinline__ void st1(__half* p, __half v) { *p = v; }
  static __device__ __forceinline__ raw ld(const __half* p) { return *reinterpret_cast<const __half2*>(p); }
  static __device__ __forceinline__ raw ld(const __half* pa, const __half* pb) { return __halves2half2(*pa, *pb); }
  static __device__ __forceinline__ float2 val(raw v) { return __half22float2(v); }
  static __device__ __forceinline__ raw pack(float2 v) { return __float22half2_rn(v); }
  static __device__ __forceinline__ void st(__half* p, raw v) { *reinterpret_cast<__half2*>(p) = v; }
  static __device__ __forceinline__ void st(__half* pa, __half* pb, raw v) {
    *pa = __low2half(v);
    *pb = __high2half(v);
  }
};

// mass and momentum of the two cells' values v_i (opposite directions taken
// together: s = v_i + v_ibar, m = v_i - v_ibar)
template <typename T>
__device__ __forceinline__ void moments2(const typename T::raw (&d)[Q], float2& m0, float2& jx, float2& jy,
                                         float2& jz) {
  float2 m[Q];
  m0 = T::val(d[0]);
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const float2 di = T::val(d[i]), dj = T::val(d[i + 1]);
    m0 = add2(m0, add2(di, dj));
    m[i] = sub2(di, dj);
  }
  jx = add2(add2(add2(m[1], m[7]), add2(m[9], m[11])), m[13]);
  jy = add2(add2(sub2(add2(m[3], m[7]), m[9]), m[15]), m[17]);
  jz = sub2(add2(sub2(add2(m[5], m[11]), m[13]), m[15]), m[17]);
}

}  // namespace

// registers: the float kernel holds 38 FP32 arrivals and runs best at 128
// registers (4 blocks of 128 threads per SM); the half kernel holds 19
// packed pairs and runs best at 96 (5 blocks per SM; 80 spills)
template <typename S>
struct PairBlocks { static constexpr int value = sizeof(S) == 4 ? HLBM_CP_MINBLOCKS_F32 : HLBM_CP_MINBLOCKS_F16; };

// C: 0 no particles, 1 particles of the analytic shapes, 2 with distance
// grids among them
template <typename S, int PAR, bool WALLS, int C>
__global__ void __launch_bounds__(128, PairBlocks<S>::value) collide_pair_kernel(LbmArgs a) {
  constexpr bool COUPLE = C > 0;
  using T = Two<S>;
  __shared__ Rec srec[COUPLE ? MAX_CAND : 1];
  __shared__ unsigned long long s_rowmask[COUPLE ? TILE_Y * TILE_Z : 1];
  const bool early = (long long)blockIdx.x + a.pdl_tail >= (long long)gridDim.x;
  if (early) pdl_trigger();
  pdl_wait();
  const Brick k = brick_of(a);
  const BoxDesc& bd = k.bd;
  if (COUPLE) load_candidates(a, k, srec, s_rowmask);

  const int x0 = k.x0 + 2 * threadIdx.x;
  const int y = k.y0 + threadIdx.y;
  if (x0 >= bd.nx || y >= bd.ny) return;
  // an odd nx leaves one cell in a row's last pair: its second slot is the
  // row's padding, computed but never stored, and the cell's right
  // neighbour is x0 + 1 wrapped (rb.dr, rb.wr refer to x0 + 1 there)
  const bool single = x0 + 1 == bd.nx;
  const int z0 = k.z0;
  const int z1 = min(z0 + a.sub_z, bd.nz);
  const RowBlocks rb = row_blocks<WALLS>(bd, x0, y, single ? 1 : 2);
  S* const f = reinterpret_cast<S*>(a.f);
  const float sc = Pop<S>::SCALED ? a.scale : 1.0f, isc = Pop<S>::SCALED ? a.inv_scale : 1.0f;

  // Walls need selects in every direction, but only the slices and rows next
  // to a wall and the lanes at an x wall meet one; everything else runs the
  // slice without them.
  const bool row_free = !WALLS || (!((bd.bc & 2) && (y == 0 || y == bd.ny - 1)) && !rb.wl && !rb.wr);
  auto slice = [&](auto wtag, int z) {
    constexpr bool W = decltype(wtag)::value;
    int zb[3];
    slice_blocks<W>(bd, z, zb);
    S* const own = cell_ptr(f, zb[1] + rb.yb[1] + rb.xb, rb.xin);  // slot 0 of cell x0
    // arrivals (stored units), both cells
    typename T::raw d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (PAR == 0 || i == 0) {
        d[i] = T::ld(own + i * VB);
      } else {
        // slot ibar of x - c_i, or slot i of x when x - c_i lies beyond a wall
        const int by = rb.yb[1 - cy(i)], bz = zb[1 - cz(i)];
        const bool wall = W && (by < 0 || bz < 0);
        const S* src = cell_ptr(f, wall ? 0 : bz + by + rb.xb, rb.xin) + opp(i) * VB;  // x0 of the source row
        const S* mine = own + i * VB;
        if (cx(i) == 0) {
          d[i] = T::ld(wall ? mine : src);
        } else if (cx(i) > 0) {  // sources x0 - 1, x0
          const S* pa = (wall || rb.wl) ? mine : src + rb.dl;
          const S* pb = wall ? mine + 1 : src;
          d[i] = T::ld(pa, pb);
        } else {  // sources x0 + 1, x0 + 2 (a single cell: x0 + 1 wrapped)
          const S* pa = wall ? mine : (single ? (rb.wr ? mine : src + rb.dr) : src + 1);
          const S* pb = (wall || rb.wr || single) ? mine + 1 : src + rb.dr;
          d[i] = T::ld(pa, pb);
        }
      }
    }
    // coupling of both cells; it needs positions only and runs while the
    // loads above are in flight
    RowCoupling<2> cc;
    if (COUPLE) {
      couple_row<2, (C > 1)>(srec, s_rowmask[threadIdx.y + a.sub_y * (z - z0)], bd, x0, y, z, a.eps,
                             a.inv_eps, a.status, cc, a.grids);
      if (single) cc.ip0[1] = cc.ip1[1] = -1;
    }
    // mass and momentum of the arrivals
    float2 drho, jx, jy, jz;
    moments2<T>(d, drho, jx, jy, jz);
    if (Pop<S>::SCALED) {
      drho = mul2(drho, f2(isc));
      jx = mul2(jx, f2(isc));
      jy = mul2(jy, f2(isc));
      jz = mul2(jz, f2(isc));
    }
    const float2 rho = add2(f2(1.0f), drho);
    if (!(rho.x > 0.0f && rho.x < 1e30f && (single || (rho.y > 0.0f && rho.y < 1e30f))))
      atomicOr(a.status, ST_UNSTABLE);
    const float2 irho = make_float2(__fdividef(1.0f, rho.x), __fdividef(1.0f, rho.y));
    const float2 ux = mul2(jx, irho), uy = mul2(jy, irho), uz = mul2(jz, irho);
    float2 dux = mul2(f2(a.ff[0]), irho), duy = mul2(f2(a.ff[1]), irho), duz = mul2(f2(a.ff[2]), irho);
    if (COUPLE) {
      if (cc.B[0] > 0.0f) {
        dux.x += cc.B[0] * (cc.upx[0] - ux.x);
        duy.x += cc.B[0] * (cc.upy[0] - uy.x);
        duz.x += cc.B[0] * (cc.upz[0] - uz.x);
      }
      if (cc.B[1] > 0.0f) {
        dux.y += cc.B[1] * (cc.upx[1] - ux.y);
        duy.y += cc.B[1] * (cc.upy[1] - uy.y);
        duz.y += cc.B[1] * (cc.upz[1] - uz.y);
      }
    }
    // f*_i - w_i = (1 - 1/tau) (d_i - E_i(u)) + E_i(u + Delta u), E = f^eq - w;
    // E_i = w drho + w rho (4.5 (c.u)^2 - 1.5 u.u) +- 3 w rho (c.u).  With
    // v = u + Delta u and o = 1 - 1/tau, a pair +-c_i takes
    //   f*_+- = o d_+- + C +- A,  A = 3 w rho (c.v - o c.u),
    //   C = 4.5 w rho ((c.v)^2 - o (c.u)^2) + w rho K + w drho / tau,
    // K = -1.5 (v.v - o u.u) shared by all directions.
    const float2 vx = add2(ux, dux), vy = add2(uy, duy), vz = add2(uz, duz);
    const float2 nusq = mul2(fma2(uz, uz, fma2(uy, uy, mul2(ux, ux))), f2(-1.5f));
    const float2 nvsq = mul2(fma2(vz, vz, fma2(vy, vy, mul2(vx, vx))), f2(-1.5f));
    const float om1s = 1.0f - a.omega;
    const float2 om1 = f2(om1s), nom1 = f2(-om1s), omg = f2(a.omega);
    const float2 K = fma2(nom1, nusq, nvsq);
    const float2 rs = mul2(rho, f2(sc)), dso = mul2(mul2(drho, f2(sc)), omg);
    {
      const float2 C0 = fma2(mul2(rs, f2(1.0f / 3.0f)), K, mul2(dso, f2(1.0f / 3.0f)));
      d[0] = T::pack(fma2(om1, T::val(d[0]), C0));
    }
    const float2 wr1 = mul2(rs, f2(1.0f / 18.0f)), wr2 = mul2(rs, f2(1.0f / 36.0f));
    const float2 q1 = fma2(wr1, K, mul2(dso, f2(1.0f / 18.0f)));
    const float2 q2 = fma2(wr2, K, mul2(dso, f2(1.0f / 36.0f)));
    const float2 h1 = mul2(wr1, f2(4.5f)), h2 = mul2(wr2, f2(4.5f));
    const float2 w3r1 = mul2(rs, f2(1.0f / 6.0f)), w3r2 = mul2(rs, f2(1.0f / 12.0f));
    auto pair = [&](int I, float2 H, float2 Qc, float2 W3, float2 cu, float2 cv) {
      const float2 p = mul2(nom1, cu);               // -o c.u
      const float2 A = mul2(W3, add2(cv, p));
      const float2 C = fma2(H, fma2(p, cu, mul2(cv, cv)), Qc);
      d[I] = T::pack(fma2(om1, T::val(d[I]), add2(C, A)));
      d[I + 1] = T::pack(fma2(om1, T::val(d[I + 1]), sub2(C, A)));
    };
    pair(1, h1, q1, w3r1, ux, vx);
    pair(3, h1, q1, w3r1, uy, vy);
    pair(5, h1, q1, w3r1, uz, vz);
    pair(7, h2, q2, w3r2, add2(ux, uy), add2(vx, vy));
    pair(9, h2, q2, w3r2, sub2(ux, uy), sub2(vx, vy));
    pair(11, h2, q2, w3r2, add2(ux, uz), add2(vx, vz));
    pair(13, h2, q2, w3r2, sub2(ux, uz), sub2(vx, vz));
    pair(15, h2, q2, w3r2, add2(uy, uz), add2(vy, vz));
    pair(17, h2, q2, w3r2, sub2(uy, uz), sub2(vy, vz));
    // cells inside a particle record the mass and momentum they send out, as
    // stored, for the next step's momentum exchange (taken before the stores,
    // so that the values need not stay in registers through them)
    float4 mom[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
    if (COUPLE && a.ilist_idx && (cc.ip0[0] >= 0 || cc.ip0[1] >= 0)) {
      float2 ms, mx, my, mz;  // of the values as stored
      moments2<T>(d, ms, mx, my, mz);
      if (Pop<S>::SCALED) {
        ms = mul2(ms, f2(isc));
        mx = mul2(mx, f2(isc));
        my = mul2(my, f2(isc));
        mz = mul2(mz, f2(isc));
      }
      mom[0] = make_float4(ms.x, mx.x, my.x, mz.x);
      mom[1] = make_float4(ms.y, mx.y, my.y, mz.y);
    }
    // store the post-collision deviations (now in d), streamed (AA pattern):
    // slot i of x + c_i, or slot ibar of x when x + c_i lies beyond a wall
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (PAR == 0 || i == 0) {
        T::st(own + opp(i) * VB, d[i]);
      } else {
        const int by = rb.yb[1 + cy(i)], bz = zb[1 + cz(i)];
        const bool wall = W && (by < 0 || bz < 0);
        S* dst = cell_ptr(f, wall ? 0 : bz + by + rb.xb, rb.xin) + i * VB;  // x0 of the destination row
        S* mine = own + opp(i) * VB;
        if (cx(i) == 0) {
          T::st(wall ? mine : dst, d[i]);
        } else if (cx(i) > 0) {  // destinations x0 + 1, x0 + 2 (a single cell: x0 + 1 wrapped)
          if (single) {
            Two<S>::st1(wall || rb.wr ? mine : dst + rb.dr, Two<S>::lo(d[i]));
          } else {
            S* pa = wall ? mine : dst + 1;
            S* pb = (wall || rb.wr) ? mine + 1 : dst + rb.dr;
            T::st(pa, pb, d[i]);
          }
        } else {  // destinations x0 - 1, x0 (a single cell: x0 - 1 only)
          S* pa = (wall || rb.wl) ? mine : dst + rb.dl;
          if (single) {
            Two<S>::st1(pa, Two<S>::lo(d[i]));
          } else {
            S* pb = wall ? mine + 1 : dst;
            T::st(pa, pb, d[i]);
          }
        }
      }
    }
    if (COUPLE && a.ilist_idx && owned_plane(bd, z))
      append_interior<2>(a, (unsigned)(bd.cell_off + (z * bd.ny + y) * bd.nx + x0), cc, mom);
  };
  // one z slice at a time: an unrolled loop would hold two slices' arrivals
#pragma unroll 1
  for (int z = z0; z < z1; ++z) {
    if (WALLS && !(row_free && !((bd.bc & 4) && (z == 0 || z == bd.nz - 1))))
      slice(std::integral_constant<bool, WALLS>{}, z);
    else
      slice(std::integral_constant<bool, false>{}, z);
  }
  if (!early) pdl_trigger();
}

template <typename S, int PAR, bool W, int C>
static cudaError_t launch_cp(const LbmArgs& a, cudaStream_t s) {
  dim3 block(TILE_X / 2, a.sub_y);
  LbmArgs b = a;
  // resident blocks per SM as the launch bounds provide for (registers)
  b.pdl_tail = a.nsm > 0 ? (long long)a.nsm * (PairBlocks<S>::value * 128 / (int)(block.x * block.y))
                         : a.nbricks;
  return launch_k(collide_pair_kernel<S, PAR, W, C>, dim3((unsigned)a.nbricks), block, 0, s, a.pdl != 0, b);
}

template <typename S, int C>
static cudaError_t launch_cp_c(const LbmArgs& a, int parity, bool walls, cudaStream_t s) {
  if (parity == 0) return launch_cp<S, 0, false, C>(a, s);
  return walls ? launch_cp<S, 1, true, C>(a, s) : launch_cp<S, 1, false, C>(a, s);
}

template <typename S>
static cudaError_t launch_cp_prec(const LbmArgs& a, int parity, bool walls, bool couple,
                                  cudaStream_t s) {
  if (!couple) return launch_cp_c<S, 0>(a, parity, walls, s);
  return a.grids.desc ? launch_cp_c<S, 2>(a, parity, walls, s) : launch_cp_c<S, 1>(a, parity, walls, s);
}

cudaError_t launch_collide_pair(const LbmArgs& a, int precision, int parity, bool walls, bool couple,
                                cudaStream_t s) {
  if (a.nbricks <= 0) return cudaSuccess;
  return precision == 0 ? launch_cp_prec<float>(a, parity, walls, couple, s)
                        : launch_cp_prec<__half>(a, parity, walls, couple, s);
}

}  // namespace hlbm
