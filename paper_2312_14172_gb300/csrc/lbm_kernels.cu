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
#include <type_traits>

#include "lbm_common.cuh"

namespace hlbm {

#ifndef HLBM_CS_MINBLOCKS
#define HLBM_CS_MINBLOCKS 4
#endif

// C: 0 no particles, 1 particles of the analytic shapes, 2 with distance
// grids among them
template <typename S, int PAR, bool WALLS, int C>
__global__ void __launch_bounds__(256, HLBM_CS_MINBLOCKS) collide_stream_kernel(LbmArgs a) {
  constexpr bool COUPLE = C > 0;
  __shared__ Rec srec[COUPLE ? MAX_CAND : 1];
  // per row of the brick (local y + sub_y * local z): the candidates whose
  // influence sphere meets the row
  __shared__ unsigned long long s_rowmask[COUPLE ? TILE_Y * TILE_Z : 1];
  const bool early = (long long)blockIdx.x + a.pdl_tail >= (long long)gridDim.x;
  if (early) pdl_trigger();
  pdl_wait();
  const Brick k = brick_of(a);
  const BoxDesc& bd = k.bd;
  if (COUPLE) load_candidates(a, k, srec, s_rowmask);

  const int x = k.x0 + threadIdx.x;
  const int y = k.y0 + threadIdx.y;
  if (x >= bd.nx || y >= bd.ny) return;
  const int z0 = k.z0;
  const int z1 = min(z0 + a.sub_z, bd.nz);
  const RowBlocks rb = row_blocks<WALLS>(bd, x, y, 1);
  S* const f = reinterpret_cast<S*>(a.f);
  // storage scale: the collision runs on the stored (scaled) deviations
  const float sc = Pop<S>::SCALED ? a.scale : 1.0f, isc = Pop<S>::SCALED ? a.inv_scale : 1.0f;

#pragma unroll 1
  for (int z = z0; z < z1; ++z) {
    const unsigned g = (unsigned)(bd.cell_off + (z * bd.ny + y) * bd.nx + x);  // global cell index
    int zb[3];
    slice_blocks<WALLS>(bd, z, zb);
    S* const own = cell_ptr(f, zb[1] + rb.yb[1] + rb.xb, rb.xin);
    float d[Q];  // stored deviations (times the storage scale)
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (PAR == 0 || i == 0) {
        d[i] = Pop<S>::ld_raw(own + i * VB);
      } else {
        // slot ibar of x - c_i, or slot i of x when x - c_i lies beyond a wall
        const int by = rb.yb[1 - cy(i)], bz = zb[1 - cz(i)];
        const bool wall = WALLS && (by < 0 || bz < 0 || (cx(i) > 0 && rb.wl) || (cx(i) < 0 && rb.wr));
        const int dx = cx(i) > 0 ? rb.dl : (cx(i) < 0 ? rb.dr : 0);
        const S* p = wall ? own + i * VB : cell_ptr(f, bz + by + rb.xb, rb.xin) + (dx + opp(i) * VB);
        d[i] = Pop<S>::ld_raw(p);
      }
    }
    // indicator, particle velocity and particles holding the cell, from the
    // candidates that meet this row (uniform over the warp); it needs
    // positions only and runs while the loads above are in flight
    RowCoupling<1> cc;
    if (COUPLE)
      couple_row<1, (C > 1)>(srec, s_rowmask[threadIdx.y + a.sub_y * (z - z0)], bd, x, y, z, a.eps,
                             a.inv_eps, a.status, cc, a.grids);
    float drho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      drho += d[i];
      if (cx(i)) jx += (float)cx(i) * d[i];
      if (cy(i)) jy += (float)cy(i) * d[i];
      if (cz(i)) jz += (float)cz(i) * d[i];
    }
    if (Pop<S>::SCALED) {
      drho *= isc;
      jx *= isc;
      jy *= isc;
      jz *= isc;
    }
    const float rho = 1.0f + drho;
    if (!(rho > 0.0f && rho < 1e30f)) atomicOr(a.status, ST_UNSTABLE);
    const float irho = 1.0f / rho;
    const float ux = jx * irho, uy = jy * irho, uz = jz * irho;
    float dux = a.ff[0] * irho, duy = a.ff[1] * irho, duz = a.ff[2] * irho;
    if (COUPLE) {
      if (cc.B[0] > 0.0f) {
        dux += cc.B[0] * (cc.upx[0] - ux);
        duy += cc.B[0] * (cc.upy[0] - uy);
        duz += cc.B[0] * (cc.upz[0] - uz);
      }
    }
    // f*_i - w_i = (1 - 1/tau) (d_i - E_i(u)) + E_i(u + Delta u), E = f^eq - w.
    // Opposite directions share the even part of E and flip the odd part:
    // E_i = w drho + w rho (4.5 (c.u)^2 - 1.5 u.u) +- 3 w rho (c.u)
    const float om1 = 1.0f - a.omega;
    const float vx = ux + dux, vy = uy + duy, vz = uz + duz;
    const float usq = 1.5f * (ux * ux + uy * uy + uz * uz);
    const float vsq = 1.5f * (vx * vx + vy * vy + vz * vz);
    float o[Q];  // post-collision deviations (times the storage scale)
    {
      const float w0 = sc * (1.0f / 3.0f);
      const float eu = w0 * drho - w0 * rho * usq, ev = w0 * drho - w0 * rho * vsq;
      o[0] = om1 * d[0] + (ev - om1 * eu);
    }
    const float rs = rho * sc, ds = drho * sc;
    const float wr1 = rs * (1.0f / 18.0f), wd1 = ds * (1.0f / 18.0f);
    const float wr2 = rs * (1.0f / 36.0f), wd2 = ds * (1.0f / 36.0f);
#define HLBM_PAIR(I, WR, WD, CU, CV)                                          \
    {                                                                         \
      const float cu_ = (CU), cv_ = (CV);                                     \
      const float eu = WD + WR * (4.5f * cu_ * cu_ - usq);                    \
      const float ev = WD + WR * (4.5f * cv_ * cv_ - vsq);                    \
      const float C = ev - om1 * eu;                                          \
      const float A = 3.0f * WR * (cv_ - om1 * cu_);                          \
      o[I] = om1 * d[I] + C + A;                                              \
      o[I + 1] = om1 * d[I + 1] + C - A;                                      \
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
    // store the post-collision deviations, streamed (AA pattern): slot i of
    // x + c_i, or slot ibar of x when x + c_i lies beyond a wall
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (PAR == 0 || i == 0) {
        Pop<S>::st_raw(own + opp(i) * VB, o[i]);
      } else {
        const int by = rb.yb[1 + cy(i)], bz = zb[1 + cz(i)];
        const bool wall = WALLS && (by < 0 || bz < 0 || (cx(i) > 0 && rb.wr) || (cx(i) < 0 && rb.wl));
        const int dx = cx(i) > 0 ? rb.dr : (cx(i) < 0 ? rb.dl : 0);
        S* p = wall ? own + opp(i) * VB : cell_ptr(f, bz + by + rb.xb, rb.xin) + (dx + i * VB);
        Pop<S>::st_raw(p, o[i]);
      }
    }
    // cells inside a particle record the mass and momentum they send out, as
    // stored, for the next step's momentum exchange (one entry per particle)
    if (COUPLE && a.ilist_idx) {
      float4 mom[1] = {make_float4(0.f, 0.f, 0.f, 0.f)};
      if (cc.ip0[0] >= 0) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const float v = stored_value<S>(o[i], 1.0f, isc);
          mom[0].x += v;
          if (cx(i)) mom[0].y += (float)cx(i) * v;
          if (cy(i)) mom[0].z += (float)cy(i) * v;
          if (cz(i)) mom[0].w += (float)cz(i) * v;
        }
      }
      if (owned_plane(bd, z)) append_interior<1>(a, g, cc, mom);
    }
  }
  if (!early) pdl_trigger();
}

// ---------------------------------------------------------------------------
// Momentum exchange (Eq. hlbm:mea, summed by Eqs. hydrodynamicforce and
// hydrodynamictorque) from moments.  Per interior cell x the used-sign sum
//   F(x) = sum_i (c_i - u_p) f_i(x) + (c_i + u_p) f_ibar(x - c_i)
// is the momentum the cell gained by the last streaming, minus u_p times the
// mass it gained: the arrivals f_i(x) give j(x) and rho(x); the departures
// f_ibar(x - c_i) = f*_ibar(x) are the cell's own post-collision values, whose
// moments the previous collision recorded in the list of interior cells:
//   F(x) = (j - j*) - u_p(x) (rho - rho*)  [links into a wall: - 2 c_i f_i(x)]
// A persistent grid walks the list (one entry per thread, all 19 loads of a
// cell in flight together); each cell's terms are rounded to fixed point
// (ACC_FRAC_BITS), and the lanes of a warp that belong to the same particle
// are summed as integers before one 64-bit integer atomic per particle,
// component and warp: the sums do not depend on the list's order.

// Exact warp sum of the 64-bit values of the lanes in mask (the others give
// 0), from three limbs with single-instruction warp reductions: v =
// a 2^42 + b 2^21 + c with c, b in [0, 2^21) and a = v >> 42 in [-2^21,
// 2^21), so 32 lanes' limb sums stay within 32 bits.
__device__ __forceinline__ long long warp_sum_i64(long long v) {
  const unsigned c = (unsigned)v & 0x1fffffu;
  const unsigned b = (unsigned)(v >> 21) & 0x1fffffu;
  const int hi = (int)(v >> 42);
  const unsigned sc = __reduce_add_sync(0xffffffffu, c);
  const unsigned sb = __reduce_add_sync(0xffffffffu, b);
  const int sa = __reduce_add_sync(0xffffffffu, hi);
  return (long long)(((unsigned long long)(long long)sa << 42) + ((unsigned long long)sb << 21) + sc);
}

// resident blocks per SM: four with walls (64 registers), five without
#ifndef HLBM_ML_MINBLOCKS_W
#define HLBM_ML_MINBLOCKS_W 4
#endif
#ifndef HLBM_ML_MINBLOCKS
#define HLBM_ML_MINBLOCKS 5
#endif
template <typename S, int PAR, bool WALLS>
__global__ void __launch_bounds__(256, WALLS ? HLBM_ML_MINBLOCKS_W : HLBM_ML_MINBLOCKS) mea_list_kernel(LbmArgs a) {
  pdl_trigger();
  pdl_wait();
  // The list is walked in chunks of 32 entries, the stripes taken in turn
  // and each stripe from its end: the first wave reads the arrivals the
  // collision wrote last, which L2 still holds.  Chunk q covers entries
  // [c_s - 32 (j + 1), c_s - 32 j) of stripe s = q mod 64, j = q / 64, c_s the
  // stripe's count; the lanes take them in ascending order, so that a run of
  // cells the collision appended together stays in one warp.
  __shared__ int s_cnt[ILIST_STRIPES];
  __shared__ int s_chunks;  // chunks per stripe
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const int c0 = (int)min((long long)a.ilist_count[lane], a.ilist_cap);
    const int c1 = (int)min((long long)a.ilist_count[lane + 32], a.ilist_cap);
    s_cnt[lane] = c0;
    s_cnt[lane + 32] = c1;
    int m = max(c0, c1);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) s_chunks = (m + 31) / 32;
  }
  __syncthreads();
  const long long nq = (long long)ILIST_STRIPES * s_chunks;
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  const S* fbase = reinterpret_cast<const S*>(a.f);
  // position of this lane's entry in chunk q (negative: none), its index in
  // the striped list, and the entry with its recorded moments; loaded one
  // chunk ahead, so that the next entry is on its way while this one's
  // arrivals are read
  auto fetch = [&](long long q, int& pos, int2& e, float4& m) {
    pos = -1;
    e = make_int2(0, -1);
    m = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q < nq) {
      const int st = (int)(q & (ILIST_STRIPES - 1)), j = (int)(q / ILIST_STRIPES);
      pos = s_cnt[st] - 32 * (j + 1) + lane;
      if (pos >= 0) {
        const long long k = (long long)st * a.ilist_cap + pos;
        e = a.ilist_idx[k];
        m = a.ilist_mom[k];
      }
    }
  };
  long long q = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
  int pos_next;
  int2 e_next;
  float4 m_next;
  fetch(q, pos_next, e_next, m_next);
  for (; q < nq; q += nwarps) {
    bool valid = pos_next >= 0;
    const bool listed = valid;
    int pid = -1;
    float F[3] = {0.f, 0.f, 0.f}, T[3] = {0.f, 0.f, 0.f};
    const int2 e = e_next;
    const float4 sd = m_next;
    fetch(q + nwarps, pos_next, e_next, m_next);
    // an entry names a particle and a cell of that particle's box; anything
    // else was never written by the collision and is skipped with a flag
    if (valid && (e.y < 0 || e.y >= a.np)) valid = false;
    // one box: its descriptor does not wait for the particle's record
    const BoxDesc bd = a.boxes[a.nboxes == 1 || !valid ? 0 : a.rec[e.y].box];
    const long long cl = (long long)e.x - bd.cell_off;
    if (valid && (cl < 0 || cl >= (long long)bd.nx * bd.ny * bd.nz)) valid = false;
    if (listed && !valid) atomicOr(a.status, ST_INTERNAL);
    int x = 0, y = 0, z = 0;
    if (valid) cell_coords(bd, (unsigned)cl, x, y, z);
    // cells next to a wall take the wall selects; a warp without any runs
    // the plain neighbour arithmetic (the same for cells off the walls)
    bool edge = false;
    if (WALLS && valid)
      edge = ((bd.bc & 1) && (x == 0 || x == bd.nx - 1)) || ((bd.bc & 2) && (y == 0 || y == bd.ny - 1)) ||
             ((bd.bc & 4) && (z == 0 || z == bd.nz - 1));
    auto cell_terms = [&](auto wtag) {
      constexpr bool W = decltype(wtag)::value;
      const Rec& R = a.rec[pid];
      float r[3];
      r[0] = offset_fp32(x, bd.nx, bd.bc & 1, R.xh[0], R.xl[0]);
      r[1] = offset_fp32(y, bd.ny, bd.bc & 2, R.xh[1], R.xl[1]);
      r[2] = offset_fp32(z, bd.nz, bd.bc & 4, R.xh[2], R.xl[2]);
      // arrivals f_i(x) (AA accessor): slot i of x (even parity), slot ibar of
      // x - c_i (odd parity), or slot i of x when x - c_i lies beyond a wall
      const RowBlocks rb = row_blocks<W>(bd, x, y, 1);
      int zb[3];
      slice_blocks<W>(bd, z, zb);
      const S* own = cell_ptr(fbase, zb[1] + rb.yb[1] + rb.xb, rb.xin);
      float d[Q];
      unsigned walls = 0;  // bit i: x - c_i lies beyond a wall
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const int by = rb.yb[1 - cy(i)], bz = zb[1 - cz(i)];
        const bool wall = W && i > 0 && (by < 0 || bz < 0 || (cx(i) > 0 && rb.wl) || (cx(i) < 0 && rb.wr));
        if (wall) walls |= 1u << i;
        if (PAR == 0 || i == 0) {
          d[i] = Pop<S>::ld(own + i * VB, a.inv_scale);
        } else {
          const int dx = cx(i) > 0 ? rb.dl : (cx(i) < 0 ? rb.dr : 0);
          const S* src = wall ? own + i * VB : cell_ptr(fbase, bz + by + rb.xb, rb.xin) + (dx + opp(i) * VB);
          d[i] = Pop<S>::ld(src, a.inv_scale);
        }
      }
      float ms = 0.f, px = 0.f, py = 0.f, pz = 0.f;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        ms += d[i];
        if (cx(i)) px += (float)cx(i) * d[i];
        if (cy(i)) py += (float)cy(i) * d[i];
        if (cz(i)) pz += (float)cz(i) * d[i];
      }
      const float upx = R.u[0] + (R.w[1] * r[2] - R.w[2] * r[1]);
      const float upy = R.u[1] + (R.w[2] * r[0] - R.w[0] * r[2]);
      const float upz = R.u[2] + (R.w[0] * r[1] - R.w[1] * r[0]);
      const float dm = ms - sd.x;
      F[0] = (px - sd.y) - upx * dm;
      F[1] = (py - sd.z) - upy * dm;
      F[2] = (pz - sd.w) - upz * dm;
      if (W) {
#pragma unroll
        for (int i = 1; i < Q; ++i)
          if ((walls >> i) & 1u) {
            const float v = 2.0f * ((float)wq(i) + d[i]);
            if (cx(i)) F[0] -= (float)cx(i) * v;
            if (cy(i)) F[1] -= (float)cy(i) * v;
            if (cz(i)) F[2] -= (float)cz(i) * v;
          }
      }
      T[0] = r[1] * F[2] - r[2] * F[1];
      T[1] = r[2] * F[0] - r[0] * F[2];
      T[2] = r[0] * F[1] - r[1] * F[0];
    };
    if (valid) pid = e.y;
    if (WALLS && __any_sync(0xffffffffu, edge)) {
      if (valid) cell_terms(std::integral_constant<bool, WALLS>{});
    } else if (valid) {
      cell_terms(std::integral_constant<bool, false>{});
    }
    // sum the lanes of each particle present in the warp
    unsigned todo = __ballot_sync(0xffffffffu, valid);
    while (todo) {
      const int leader = __ffs(todo) - 1;
      const int p = __shfl_sync(0xffffffffu, pid, leader);
      const bool mine = valid && pid == p;
      todo &= ~__ballot_sync(0xffffffffu, mine);
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const float t = c < 3 ? F[c] : T[c - 3];
        const long long v = warp_sum_i64(mine ? __float2ll_rn(__fmul_rn(t, (float)(1LL << ACC_FRAC_BITS))) : 0LL);
        if (lane == leader)
          atomicAdd(reinterpret_cast<unsigned long long*>(&a.acc[(long long)p * 6 + c]), (unsigned long long)v);
      }
    }
  }
}

template <typename S, int PAR, bool W, int C>
static cudaError_t launch_cs(const LbmArgs& a, cudaStream_t s) {
  dim3 block(TILE_X, a.sub_y);
  LbmArgs b = a;
  // resident blocks per SM as the launch bounds provide for (registers)
  b.pdl_tail = a.nsm > 0 ? (long long)a.nsm * (HLBM_CS_MINBLOCKS * 256 / (int)(block.x * block.y)) : a.nbricks;
  return launch_k(collide_stream_kernel<S, PAR, W, C>, dim3((unsigned)a.nbricks), block, 0, s, a.pdl != 0, b);
}

template <typename S, int C>
static cudaError_t launch_cs_c(const LbmArgs& a, int parity, bool walls, cudaStream_t s) {
  // even steps never touch a neighbour: walls need no special case
  if (parity == 0) return launch_cs<S, 0, false, C>(a, s);
  return walls ? launch_cs<S, 1, true, C>(a, s) : launch_cs<S, 1, false, C>(a, s);
}

template <typename S>
static cudaError_t launch_cs_prec(const LbmArgs& a, int parity, bool walls, bool couple,
                                  cudaStream_t s) {
  if (!couple) return launch_cs_c<S, 0>(a, parity, walls, s);
  return a.grids.desc ? launch_cs_c<S, 2>(a, parity, walls, s) : launch_cs_c<S, 1>(a, parity, walls, s);
}

cudaError_t launch_collide(const LbmArgs& a, int precision, int parity, bool walls, bool couple,
                           cudaStream_t s) {
  if (a.nbricks <= 0) return cudaSuccess;
  if (a.cells_x == 2) return launch_collide_pair(a, precision, parity, walls, couple, s);
  return precision == 0 ? launch_cs_prec<float>(a, parity, walls, couple, s)
                        : launch_cs_prec<__half>(a, parity, walls, couple, s);
}

// one wave of resident blocks walks the whole list
template <typename S, int PAR, bool W>
static unsigned ml_blocks(int nsm) {
  static int per_sm = 0;  // the same on every GPU of this architecture
  if (per_sm == 0) {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, mea_list_kernel<S, PAR, W>, 256, 0) != cudaSuccess || v < 1)
      v = 1;
    per_sm = v;
  }
  return (unsigned)((nsm > 0 ? nsm : 152) * per_sm);
}

template <typename S, int PAR>
static cudaError_t launch_ml(const LbmArgs& a, bool walls, int nsm, cudaStream_t s) {
  if (walls) return launch_k(mea_list_kernel<S, PAR, true>, dim3(ml_blocks<S, PAR, true>(nsm)), dim3(256), 0, s,
                            a.pdl != 0, a);
  return launch_k(mea_list_kernel<S, PAR, false>, dim3(ml_blocks<S, PAR, false>(nsm)), dim3(256), 0, s, a.pdl != 0, a);
}

cudaError_t launch_mea_moments(const LbmArgs& a, int precision, int parity, bool walls, int nsm,
                               cudaStream_t s) {
  if (precision == 0) return parity == 0 ? launch_ml<float, 0>(a, walls, nsm, s) : launch_ml<float, 1>(a, walls, nsm, s);
  return parity == 0 ? launch_ml<__half, 0>(a, walls, nsm, s) : launch_ml<__half, 1>(a, walls, nsm, s);
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
  S* f = reinterpret_cast<S*>(a.f);
  const NbrB nb = make_nbr_blocked(bd, x, y, z);
  const long long e = elem_of(bd, x, y, z);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    S* slot;
    if (PAR == 0 || i == 0) {
      slot = f + e + i * VB;
    } else {
      const long long src = nb.at(-cx(i), -cy(i), -cz(i));
      slot = (src >= 0) ? f + src + opp(i) * VB : f + e + i * VB;
    }
    if (GATHER) stage[i * n + k] = Pop<S>::ld(slot, a.inv_scale);
    else Pop<S>::st(slot, stage[i * n + k], a.scale);
  }
}

// mass deviation and momentum of one box, sum over its cells of the logical
// f_i - w_i and c_i (f_i - w_i) (Sec. 3.1 moments; the weights carry no net
// momentum), in FP64: each block writes its four sums (added in a fixed
// order over its threads) to out[4 * blockIdx.x]
template <typename S, int PAR>
__global__ void __launch_bounds__(256) fluid_moments_kernel(LbmArgs a, int box, double* out) {
  const BoxDesc bd = a.boxes[box];
  const long long n = (long long)bd.nx * bd.ny * bd.nz;
  const S* f = reinterpret_cast<const S*>(a.f);
  double m[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long cl = blockIdx.x * (long long)blockDim.x + threadIdx.x; cl < n;
       cl += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(cl % bd.nx);
    const long long t = cl / bd.nx;
    const int y = (int)(t % bd.ny);
    const int z = (int)(t / bd.ny);
    const NbrB nb = make_nbr_blocked(bd, x, y, z);
    const long long e = elem_of(bd, x, y, z);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const S* slot;
      if (PAR == 0 || i == 0) {
        slot = f + e + i * VB;
      } else {
        const long long src = nb.at(-cx(i), -cy(i), -cz(i));
        slot = (src >= 0) ? f + src + opp(i) * VB : f + e + i * VB;
      }
      const double d = (double)Pop<S>::ld(slot, a.inv_scale);
      m[0] += d;
      if (cx(i)) m[1] += cx(i) * d;
      if (cy(i)) m[2] += cy(i) * d;
      if (cz(i)) m[3] += cz(i) * d;
    }
  }
  __shared__ double sm[4][256];
  for (int k = 0; k < 4; ++k) sm[k][threadIdx.x] = m[k];
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < 4; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) out[4 * blockIdx.x + threadIdx.x] = sm[threadIdx.x][0];
}

cudaError_t launch_fluid_moments(const LbmArgs& a, int precision, int parity, int box, int blocks,
                                 double* out, cudaStream_t s) {
  if (blocks < 1) return cudaErrorInvalidValue;
  if (precision == 0) {
    if (parity == 0) fluid_moments_kernel<float, 0><<<blocks, 256, 0, s>>>(a, box, out);
    else fluid_moments_kernel<float, 1><<<blocks, 256, 0, s>>>(a, box, out);
  } else {
    if (parity == 0) fluid_moments_kernel<__half, 0><<<blocks, 256, 0, s>>>(a, box, out);
    else fluid_moments_kernel<__half, 1><<<blocks, 256, 0, s>>>(a, box, out);
  }
  return cudaGetLastError();
}

// the five slots {i : c_iz = dir} of every cell of plane z of one box, as
// stored, to or from stage[(k ny + y) nx + x] (k the slot's rank in the set)
template <typename S>
__global__ void plane_slots_kernel(LbmArgs a, int box, int z, int dir, S* stage, int put) {
  const BoxDesc bd = a.boxes[box];
  const long long n = (long long)bd.nx * bd.ny;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= 5 * n) return;
  const int k = (int)(t / n);
  const long long c = t - k * n;
  const int y = (int)(c / bd.nx), x = (int)(c - (long long)y * bd.nx);
  // slots with c_z = +1: 5, 11, 14, 15, 18; with c_z = -1 their opposites
  const int plus[5] = {5, 11, 14, 15, 18};
  const int i = dir > 0 ? plus[k] : opp(plus[k]);
  S* f = reinterpret_cast<S*>(a.f) + elem_of(bd, x, y, z) + i * VB;
  if (put) *f = stage[t];
  else stage[t] = *f;
}

cudaError_t launch_plane_slots(const LbmArgs& a, int precision, int box, int z, int dir, int ncell, void* stage,
                               int put, cudaStream_t s) {
  const unsigned blocks = (unsigned)((5LL * ncell + 255) / 256);
  if (precision == 0)
    plane_slots_kernel<float><<<blocks, 256, 0, s>>>(a, box, z, dir, reinterpret_cast<float*>(stage), put);
  else
    plane_slots_kernel<__half><<<blocks, 256, 0, s>>>(a, box, z, dir, reinterpret_cast<__half*>(stage), put);
  return cudaGetLastError();
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
