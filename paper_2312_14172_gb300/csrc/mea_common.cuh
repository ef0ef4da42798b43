// mea_common.cuh -- device pieces of the bounding-box momentum exchange
// shared by the kernels that compute Eq. hlbm:mea (Sec. 3.2) from the
// populations alone.
#pragma once
#include "hlbm_internal.cuh"

namespace hlbm {

template <typename S> struct PopR;
template <> struct PopR<float> {
  static __device__ __forceinline__ float ld(const float* p, float) { return *p; }
};
template <> struct PopR<__half> {
  static __device__ __forceinline__ float ld(const __half* p, float inv_s) {
    return __half2float(*p) * inv_s;
  }
};

// rotation body -> world of a unit quaternion, every operation rounded on its
// own (no contraction) so that the FP32 copy matches other FP64 evaluations of
// the same formula bit for bit
__device__ __forceinline__ void rotation_rn(const double q[4], double R[9]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(__dmul_rn(y, y), __dmul_rn(z, z))));
  R[1] = __dmul_rn(2.0, __dsub_rn(__dmul_rn(x, y), __dmul_rn(w, z)));
  R[2] = __dmul_rn(2.0, __dadd_rn(__dmul_rn(x, z), __dmul_rn(w, y)));
  R[3] = __dmul_rn(2.0, __dadd_rn(__dmul_rn(x, y), __dmul_rn(w, z)));
  R[4] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(__dmul_rn(x, x), __dmul_rn(z, z))));
  R[5] = __dmul_rn(2.0, __dsub_rn(__dmul_rn(y, z), __dmul_rn(w, x)));
  R[6] = __dmul_rn(2.0, __dsub_rn(__dmul_rn(x, z), __dmul_rn(w, y)));
  R[7] = __dmul_rn(2.0, __dadd_rn(__dmul_rn(y, z), __dmul_rn(w, x)));
  R[8] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y))));
}

// force on the particle from cell x (used form of Eq. hlbm:mea):
//   sum_i (c_i - u_p) f_i(x) + (c_i + u_p) f_ibar(x - c_i)
// = sum_i c_i (in_i + out_i) - u_p sum_i (in_i - out_i), with in_i = f_i(x)
// (arrived from x - c_i) and out_i = f_ibar(x - c_i) (left x towards x - c_i).
// This is the printed per-cell sum with the opposite sign: on post-streaming
// populations the printed sum is what the cell hands to the fluid, and the
// particle feels the reverse.  Links to a node beyond a wall carry no fluid
// and are left out; on deviations d = f - w that leaves -2 c_i w_i per
// omitted link, because the weights of all 18 links sum to zero.  In both AA
// parities the pair of slots is {slot i of x, slot ibar of x - c_i}; only
// which of the two is the arrival differs.  Slot i of the cell whose slot 0
// is element e lies at f + i * P + e: P is the plane stride of a plain
// structure of arrays, or VB in the blocked layout (nb from make_nbr_blocked).
template <typename S, int PAR, typename NB>
__device__ __forceinline__ void mea_cell(const S* f, long long P, const NB& nb, long long c,
                                         float inv_s, float F[3], float& mgain) {
  F[0] = F[1] = F[2] = 0.0f;
  mgain = 0.0f;
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const long long s = nb.at(-cx(i), -cy(i), -cz(i));
    if (s < 0) {
      const float w2 = 2.0f * (float)wq(i);
      if (cx(i)) F[0] -= (float)cx(i) * w2;
      if (cy(i)) F[1] -= (float)cy(i) * w2;
      if (cz(i)) F[2] -= (float)cz(i) * w2;
      continue;
    }
    const float va = PopR<S>::ld(f + i * P + c, inv_s);       // slot i of x
    const float vb = PopR<S>::ld(f + opp(i) * P + s, inv_s);  // slot ibar of x - c_i
    const float in = PAR == 0 ? va : vb;
    const float out = PAR == 0 ? vb : va;
    const float sum = in + out;
    if (cx(i)) F[0] += (float)cx(i) * sum;
    if (cy(i)) F[1] += (float)cy(i) * sum;
    if (cz(i)) F[2] += (float)cz(i) * sum;
    mgain += in - out;
  }
}

// x-range of the cells of bounding-box row iy (plane offset dz) that can lie
// inside the circumscribed sphere (+-1 cell of margin); empty when the row
// misses it
__device__ __forceinline__ void row_range(int iy, int ext1, int lo0, int ext0, int lo1,
                                          const double X[3], float dz, float rc2, int& xa, int& len) {
  len = 0;
  xa = 0;
  if (iy >= ext1) return;
  const float dy = (float)((double)(lo1 + iy) - X[1]);
  const float d2 = dy * dy + dz * dz;
  if (d2 >= rc2) return;
  const float s = sqrtf(rc2 - d2);
  xa = max(lo0, (int)floorf((float)X[0] - s) - 1);
  const int xb = min(lo0 + ext0 - 1, (int)ceilf((float)X[0] + s) + 1);
  len = max(xb - xa + 1, 0);
}

// Per-thread sums (F, T) over the cells of plane iz of the bounding box
// [floor(X - r_c), ceil(X + r_c)] of one particle whose centre is finite.
// All threads of the block call it (it synchronises); s_start holds
// MAX_PLANES + 1 ints, s_xa MAX_PLANES.  BLOCKED: f is the library's
// blocked storage (plane unused); otherwise f holds the box alone as a plain
// structure of arrays with `plane` values per slot, cell (x, y, z) at
// (z * ny + y) * nx + x.
template <typename S, int PAR, bool BLOCKED>
__device__ __forceinline__ void mea_plane_sums(const Rec& R, const BoxDesc& bd, const double X[3],
                                               double rc, int iz, const S* f, long long plane,
                                               float inv_scale, int* s_start, int* s_xa,
                                               float out[6], GridSet gs = GridSet{}) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n[3] = {bd.nx, bd.ny, bd.nz};
  // cells that can be inside: [floor(X - r_c), ceil(X + r_c)] per axis
  int lo[3] = {0, 0, 0}, ext[3] = {0, 0, 0};
  {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      int l = (int)floor(X[j] - rc), h = (int)ceil(X[j] + rc);
      if ((bd.bc >> j) & 1) {
        const bool cut = j == 2 && (bd.bc & BC_CUT_Z);  // owned planes only
        l = max(l, cut ? bd.own_lo : 0);
        h = min(h, cut ? bd.own_hi - 1 : n[j] - 1);
      }
      lo[j] = l;
      ext[j] = min(max(h - l + 1, 0), MAX_PLANES);
    }
  }
  float Fx = 0.f, Fy = 0.f, Fz = 0.f, Tx = 0.f, Ty = 0.f, Tz = 0.f;
  if (iz < ext[2]) {  // uniform over the block
    const int zu = lo[2] + iz;
    const int z = zu < 0 ? zu + n[2] : (zu >= n[2] ? zu - n[2] : zu);
    const float dz = (float)((double)zu - X[2]);
    const float rc2 = (float)(rc * rc) * 1.0001f + 1e-3f;
    // rows of this plane that meet the circumscribed sphere, flattened
    if (warp == 0) {
      int xa0, len0, xa1, len1;
      row_range(lane, ext[1], lo[0], ext[0], lo[1], X, dz, rc2, xa0, len0);
      row_range(lane + 32, ext[1], lo[0], ext[0], lo[1], X, dz, rc2, xa1, len1);
      int s0 = len0, s1 = len1;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int t0 = __shfl_up_sync(0xffffffffu, s0, off);
        const int t1 = __shfl_up_sync(0xffffffffu, s1, off);
        if (lane >= off) { s0 += t0; s1 += t1; }
      }
      const int tot0 = __shfl_sync(0xffffffffu, s0, 31);
      s1 += tot0;
      s_start[lane] = s0 - len0;
      s_start[lane + 32] = s1 - len1;
      s_xa[lane] = xa0;
      s_xa[lane + 32] = xa1;
      if (lane == 31) s_start[MAX_PLANES] = s1;
    }
    __syncthreads();
    const int total = s_start[MAX_PLANES];
    for (int q = tid; q < total; q += blockDim.x) {
      // the row holding flat index q: the last row starting at or before q
      int r = 0;
#pragma unroll
      for (int step = 32; step > 0; step >>= 1)
        if (r + step < MAX_PLANES && s_start[r + step] <= q) r += step;
      const int xu = s_xa[r] + (q - s_start[r]);
      const int yu = lo[1] + r;
      const int x = xu < 0 ? xu + n[0] : (xu >= n[0] ? xu - n[0] : xu);
      const int y = yu < 0 ? yu + n[1] : (yu >= n[1] ? yu - n[1] : yu);
      float rr[3];
      if (!inside_fp32(R, bd, x, y, z, rr, gs)) continue;
      float Fc[3], mg;
      if constexpr (BLOCKED) {
        mea_cell<S, PAR>(f, (long long)VB, make_nbr_blocked(bd, x, y, z), elem_of(bd, x, y, z), inv_scale,
                         Fc, mg);
      } else {
        mea_cell<S, PAR>(f, plane, make_nbr<true>(bd, x, y, z), (long long)((z * bd.ny + y) * bd.nx + x),
                         inv_scale, Fc, mg);
      }
      const float upx = R.u[0] + (R.w[1] * rr[2] - R.w[2] * rr[1]);
      const float upy = R.u[1] + (R.w[2] * rr[0] - R.w[0] * rr[2]);
      const float upz = R.u[2] + (R.w[0] * rr[1] - R.w[1] * rr[0]);
      Fc[0] -= upx * mg;
      Fc[1] -= upy * mg;
      Fc[2] -= upz * mg;
      Fx += Fc[0];
      Fy += Fc[1];
      Fz += Fc[2];
      Tx += rr[1] * Fc[2] - rr[2] * Fc[1];
      Ty += rr[2] * Fc[0] - rr[0] * Fc[2];
      Tz += rr[0] * Fc[1] - rr[1] * Fc[0];
    }
  }
  out[0] = Fx; out[1] = Fy; out[2] = Fz;
  out[3] = Tx; out[4] = Ty; out[5] = Tz;
}

}  // namespace hlbm
