// noalloc.cu -- momentum exchange that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a particle code that runs inside
// another framework's memory arena or pool, code whose only device memory is
// what its host application hands it, or a process whose device memory is
// already fully reserved.  For them hlbm_mea_noalloc computes the momentum
// exchange force and torque of a set of particles on populations the caller
// owns, with every intermediate held in one file-scope device array of fixed
// size, declared below.  Every GPU that loads the library holds that array
// until the process exits.
#include <cuda.h>

#include <mutex>

#include "../../include/hlbm.h"
#include "mea_common.cuh"

namespace hlbm {
namespace {

constexpr int NA_MAX = HLBM_NOALLOC_MAX_PARTICLES;

// scratch layout (bytes): particle records, circumscribed radii, checked
// centres (wrapped into the box on periodic axes), planes per particle,
// finished-block counters, per-(particle, plane) FP64 partials
constexpr size_t NA_REC = 0;
constexpr size_t NA_RC = NA_REC + sizeof(Rec) * NA_MAX;
constexpr size_t NA_X = NA_RC + sizeof(double) * NA_MAX;
constexpr size_t NA_NPL = NA_X + sizeof(double) * 3 * NA_MAX;
constexpr size_t NA_DONE = NA_NPL + sizeof(int) * NA_MAX;
constexpr size_t NA_PART = NA_DONE + sizeof(int) * NA_MAX;
constexpr size_t NA_BYTES = NA_PART + sizeof(double) * 6 * MAX_PLANES * NA_MAX;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

struct NoAllocArgs {
  unsigned char* scratch;  // device address of g_noalloc_scratch
  const void* f;
  long long plane;
  BoxDesc bd;
  float inv_scale;
  int n;
  const int* shape;
  const double* params;
  const double* X;
  const double* U;
  const double* W;
  const double* Q;
  double* F;
  double* T;
};

__device__ __forceinline__ Rec* na_rec(const NoAllocArgs& a) { return reinterpret_cast<Rec*>(a.scratch + NA_REC); }
__device__ __forceinline__ double* na_rc(const NoAllocArgs& a) { return reinterpret_cast<double*>(a.scratch + NA_RC); }
__device__ __forceinline__ double* na_x(const NoAllocArgs& a) { return reinterpret_cast<double*>(a.scratch + NA_X); }
__device__ __forceinline__ int* na_npl(const NoAllocArgs& a) { return reinterpret_cast<int*>(a.scratch + NA_NPL); }
__device__ __forceinline__ int* na_done(const NoAllocArgs& a) { return reinterpret_cast<int*>(a.scratch + NA_DONE); }
__device__ __forceinline__ double* na_part(const NoAllocArgs& a) { return reinterpret_cast<double*>(a.scratch + NA_PART); }

// records of the caller's particles; clears the counters.  The checks are
// those of hlbm_add_particles: a centre outside (-1/2, n - 1/2) on a wall
// axis, or a particle whose circumscribed sphere plus two cells spans half a
// periodic axis or more, is invalid, and so are non-finite or non-positive
// sizes, a zero or non-finite quaternion and non-finite velocities.  On a
// periodic axis the centre is wrapped into [0, n) and kept in the scratch
// array, so that the exchange kernel walks a bounding box whose cells lie at
// most one period outside the box.  An invalid particle gets no planes and
// NaN force and torque.
__global__ void noalloc_setup_kernel(NoAllocArgs a) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.n) return;
  const int shape = a.shape[p];
  const int nn[3] = {a.bd.nx, a.bd.ny, a.bd.nz};
  double s[3], X[3], U[3], W[3], q[4], nq = 0.0;
  bool ok = shape >= 0 && shape <= 3;
  for (int j = 0; j < 3; ++j) {
    s[j] = ok ? a.params[3 * p + ((shape == 0 || (shape == 3 && j == 1)) ? 0 : j)] : 1.0;
    X[j] = a.X[3 * p + j];
    U[j] = a.U ? a.U[3 * p + j] : 0.0;
    W[j] = a.W ? a.W[3 * p + j] : 0.0;
    ok = ok && s[j] > 0.0 && isfinite(s[j]) && isfinite(X[j]) && isfinite(U[j]) && isfinite(W[j]);
  }
  for (int j = 0; j < 4; ++j) {
    q[j] = a.Q ? a.Q[4 * p + j] : (j == 0 ? 1.0 : 0.0);
    nq += q[j] * q[j];
  }
  ok = ok && nq > 0.0 && isfinite(nq);
  double rc = s[0];
  if (shape == 1) rc = fmax(s[0], fmax(s[1], s[2]));
  if (shape == 2) rc = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
  if (shape == 3) rc = s[0] + s[2];
  ok = ok && rc <= 30.0;
  for (int j = 0; j < 3 && ok; ++j) {
    if ((a.bd.bc >> j) & 1) {
      ok = X[j] > -0.5 && X[j] < nn[j] - 0.5;
    } else {
      const double L = (double)nn[j];
      ok = 2.0 * (rc + 2.0) < L;
      X[j] -= L * floor(X[j] / L);
      if (X[j] >= L) X[j] -= L;
    }
  }
  na_done(a)[p] = 0;
  if (!ok) {
    na_npl(a)[p] = 0;
    for (int j = 0; j < 3; ++j) {
      a.F[3 * p + j] = __longlong_as_double(0x7ff8000000000000LL);
      a.T[3 * p + j] = __longlong_as_double(0x7ff8000000000000LL);
    }
    return;
  }
  nq = sqrt(nq);
  for (int j = 0; j < 4; ++j) q[j] /= nq;
  Rec R;
  double M[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  if (shape != 0) rotation_rn(q, M);
  for (int j = 0; j < 3; ++j) {
    const float xh = __double2float_rn(X[j]);
    R.xh[j] = xh;
    R.xl[j] = __double2float_rn(X[j] - (double)xh);
    R.u[j] = (float)U[j];
    R.w[j] = (float)W[j];
    R.a[j] = __double2float_rn(s[j]);
    R.ia[j] = __double2float_rn(1.0 / s[j]);
    na_x(a)[3 * p + j] = X[j];
  }
  for (int k = 0; k < 9; ++k) R.M[k] = __double2float_rn(M[k]);
  R.in2 = __double2float_rn(s[0] * s[0]);
  R.rinf2 = 0.0f;
  R.shape = shape;
  R.box = 0;
  R.pid = p;
  na_rec(a)[p] = R;
  na_rc(a)[p] = rc;
  na_npl(a)[p] = (int)ceil(2.0 * rc) + 2;
}

// the bounding-box momentum exchange, one block per (particle, plane); the
// last block of a particle adds the planes' FP64 partials in plane order and
// writes the caller's output; eight resident blocks per SM, as the
// bounding-box momentum exchange of the library
template <typename S, int PAR>
__global__ void __launch_bounds__(128, 8) noalloc_mea_kernel(NoAllocArgs a) {
  const int p = blockIdx.x, iz = blockIdx.y;
  const int npl = na_npl(a)[p];
  if (iz >= npl) return;
  __shared__ Rec R;
  __shared__ double wsum[4][6];
  __shared__ int s_start[MAX_PLANES + 1], s_xa[MAX_PLANES];
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < 32) reinterpret_cast<int*>(&R)[tid] = reinterpret_cast<const int*>(&na_rec(a)[p])[tid];
  __syncthreads();
  // the centre the set-up checked and wrapped, not the caller's array again
  double X[3];
  for (int j = 0; j < 3; ++j) X[j] = na_x(a)[3 * p + j];
  float v[6];
  mea_plane_sums<S, PAR, false>(R, a.bd, X, na_rc(a)[p], iz, reinterpret_cast<const S*>(a.f), a.plane,
                         a.inv_scale, s_start, s_xa, v);
#pragma unroll
  for (int k = 0; k < 6; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if (lane == 0)
    for (int k = 0; k < 6; ++k) wsum[warp][k] = (double)v[k];
  __syncthreads();
  double* part = na_part(a) + ((long long)p * MAX_PLANES + iz) * 6;
  if (tid < 6) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += wsum[w][tid];
    part[tid] = s;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(&na_done(a)[p], 1) == npl - 1);
  __syncthreads();
  if (s_last) {
    __threadfence();
    if (tid < 6) {
      double s = 0.0;
      for (int k = 0; k < npl; ++k) s += __ldcg(na_part(a) + ((long long)p * MAX_PLANES + k) * 6 + tid);
      if (tid < 3) a.F[3 * p + tid] = s;
      else a.T[3 * p + tid - 3] = s;
    }
    if (tid == 0) na_done(a)[p] = 0;
  }
}

// Device address of the scratch array, looked up once per device and CUDA
// context: the address belongs to the context that loaded the module, so a
// new context on the device (after cudaDeviceReset, or a context the caller
// made current) takes a fresh look-up.  The context's identity comes from
// the driver's cuCtxGetCurrent / cuCtxGetId, reached through the runtime's
// entry-point query (the library does not link the driver library itself);
// where those are unavailable, or no context is current yet, the address is
// looked up again on that call.
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
unsigned char* g_na_ptr[NA_MAX_DEVICES] = {};
unsigned long long g_na_ctx[NA_MAX_DEVICES] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// identity of the current context, or 0 when none is current or the driver
// calls are unavailable (called with g_na_mutex held)
unsigned long long current_context_id() {
  static bool looked = false;
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!looked) {
    looked = true;
    void* f0 = nullptr;
    void* f1 = nullptr;
    cudaDriverEntryPointQueryResult q0 = cudaDriverEntryPointSymbolNotFound, q1 = q0;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        q0 == cudaDriverEntryPointSuccess && q1 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<CtxGetCurrentFn>(f0);
      get_id = reinterpret_cast<CtxGetIdFn>(f1);
    }
  }
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

}  // namespace
}  // namespace hlbm

using namespace hlbm;

extern "C" int hlbm_mea_noalloc(const void* f, long long plane, int nx, int ny, int nz, int bc_flags,
                                int precision, int fp16_scale_log2, int parity, int n,
                                const int* shape, const double* shape_params, const double* X,
                                const double* U, const double* omega, const double* quat,
                                double* F, double* T, void* cuda_stream) {
  if (n < 0 || n > NA_MAX) {
    return HLBM_ERR_ARG;
  }
  if (nx < 1 || ny < 1 || nz < 1 || (bc_flags & ~7) || (long long)nx * ny * nz >= (1LL << 31) ||
      plane < (long long)nx * ny * nz || (precision != HLBM_FP32 && precision != HLBM_FP16) ||
      fp16_scale_log2 < 0 || fp16_scale_log2 > 16 || (parity != 0 && parity != 1)) {
    return HLBM_ERR_ARG;
  }
  if (n == 0) return HLBM_OK;
  if (!f || !shape || !shape_params || !X || !F || !T) {
    return HLBM_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
    return HLBM_ERR_CUDA;
  }
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    const unsigned long long ctx = current_context_id();
    if (!g_na_ptr[dev] || ctx == 0 || ctx != g_na_ctx[dev]) {
      // set-up on this device and context (it is made current here if it
      // was not): the device address of the file-scope scratch array
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
        g_na_ptr[dev] = nullptr;
        return HLBM_ERR_CUDA;
      }
      g_na_ptr[dev] = static_cast<unsigned char*>(ptr);
      g_na_ctx[dev] = current_context_id();
    }
    scratch = g_na_ptr[dev];
  }
  NoAllocArgs a{};
  a.scratch = scratch;
  a.f = f;
  a.plane = plane;
  a.bd.nx = nx;
  a.bd.ny = ny;
  a.bd.nz = nz;
  a.bd.bc = bc_flags;
  a.bd.div_x = make_fastdiv((unsigned)nx);
  a.bd.div_y = make_fastdiv((unsigned)ny);
  a.bd.cell_off = 0;
  a.inv_scale = precision == HLBM_FP16 ? (float)(1.0 / (double)(1 << fp16_scale_log2)) : 1.0f;
  a.n = n;
  a.shape = shape;
  a.params = shape_params;
  a.X = X;
  a.U = U;
  a.W = omega;
  a.Q = quat;
  a.F = F;
  a.T = T;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  noalloc_setup_kernel<<<(n + 127) / 128, 128, 0, s>>>(a);
  const dim3 grid(n, MAX_PLANES);
  if (precision == HLBM_FP32) {
    if (parity == 0) noalloc_mea_kernel<float, 0><<<grid, 128, 0, s>>>(a);
    else noalloc_mea_kernel<float, 1><<<grid, 128, 0, s>>>(a);
  } else {
    if (parity == 0) noalloc_mea_kernel<__half, 0><<<grid, 128, 0, s>>>(a);
    else noalloc_mea_kernel<__half, 1><<<grid, 128, 0, s>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? HLBM_OK : HLBM_ERR_CUDA;
}

