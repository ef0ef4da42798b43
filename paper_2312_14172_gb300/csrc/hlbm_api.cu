// hlbm_api.cu -- the C-ABI of include/hlbm.h: handles, device memory layout,
// particle set-up, CUDA-graph capture of the time step, data exchange.
//
// One time step (Algorithm 1 of arXiv:2312.14172, Sec. 4.2.5, without its
// communication rows) is three launches on the handle's stream:
//   1. momentum exchange per particle          (mea_kernel)
//   2. contact forces, when switched on       (contact_kernel)
//      external force, Newton-Euler, records,
//      per-tile particle lists                 (update_kernel)
//   3. EDM coupling, collision and streaming   (collide_stream_kernel)
// Steps alternate between the two AA parities, so each parity is captured
// once as a CUDA graph and the graphs are launched alternately.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <array>
#include <vector>

#include "../../include/hlbm.h"
#include "hlbm_internal.cuh"

using namespace hlbm;

namespace {

constexpr size_t ALIGN = 256;
constexpr int DEFAULT_BIN_CAP = 64;
constexpr long long STAGE_CELLS = 1 << 18;
const double PI_D = 3.14159265358979323846;

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

struct Layout {
  long long nblocks = 0, ncell = 0, ntiles = 0, stage_cells = 0;
  int cap = 0, bin_cap = 0;
  size_t off_f, off_boxes, off_P, off_shape, off_box, off_rec, off_part, off_acc, off_chp, off_chq,
      off_pc0, off_pnc, off_done, off_lcnt, off_lidx, off_lmom, off_cnt[2], off_ids[2], off_status,
      off_stage, off_gdesc, off_gvals, total;
  long long grid_floats = 0;
  long long ilist_cap = 0;
};

bool make_layout(int nb, const hlbm_box* boxes, const hlbm_params* prm, Layout& L,
                 std::vector<BoxDesc>& bd, std::string& err) {
  if (nb < 1 || !boxes || !prm) { err = "need at least one box and parameters"; return false; }
  if (!(prm->tau > 0.5) || !std::isfinite(prm->tau)) { err = "tau must be finite and > 1/2"; return false; }
  if (!(prm->eps > 0.0) || !std::isfinite(prm->eps)) { err = "eps must be finite and > 0"; return false; }
  if (prm->precision != HLBM_FP32 && prm->precision != HLBM_FP16) { err = "unknown precision"; return false; }
  if (prm->fp16_scale_log2 < 0 || prm->fp16_scale_log2 > 16) { err = "fp16_scale_log2 out of [0, 16]"; return false; }
  if (prm->max_particles < 0) { err = "max_particles < 0"; return false; }
  if (prm->bin_capacity < 0 || prm->bin_capacity > 64) { err = "bin_capacity out of [0, 64]"; return false; }
  if (prm->grid_floats < 0 || prm->grid_floats > (1LL << 34)) { err = "grid_floats out of range"; return false; }
  for (int j = 0; j < 3; ++j)
    if (!std::isfinite(prm->gravity[j]) || !std::isfinite(prm->fluid_force[j])) { err = "non-finite force"; return false; }
  bd.assign(nb, BoxDesc{});
  long long cells = 0, tiles = 0, blocks = 0, maxbox = 0;
  for (int b = 0; b < nb; ++b) {
    const hlbm_box& B = boxes[b];
    if (B.nx < 1 || B.ny < 1 || B.nz < 1 || (B.bc_flags & ~15) ||
        ((B.bc_flags & HLBM_CUT_Z) && !(B.bc_flags & HLBM_WALL_Z))) {
      err = "bad box dimensions or flags (HLBM_CUT_Z needs HLBM_WALL_Z)";
      return false;
    }
    const long long n = (long long)B.nx * B.ny * B.nz;
    if (n >= (1LL << 31)) { err = "a box may hold at most 2^31 - 1 cells"; return false; }
    if (cells + n >= (1LL << 31)) { err = "all boxes together may hold at most 2^31 - 1 cells"; return false; }
    BoxDesc& d = bd[b];
    d.nx = B.nx; d.ny = B.ny; d.nz = B.nz; d.bc = B.bc_flags;
    d.div_x = make_fastdiv((unsigned)B.nx);
    d.div_y = make_fastdiv((unsigned)B.ny);
    d.own_lo = 0;
    d.own_hi = B.nz;
    d.ntx = (B.nx + TILE_X - 1) / TILE_X;
    d.nty = (B.ny + TILE_Y - 1) / TILE_Y;
    d.ntz = (B.nz + TILE_Z - 1) / TILE_Z;
    d.cell_off = cells;
    d.tile_off = tiles;
    d.blk_off = blocks;
    cells += n;
    tiles += (long long)d.ntx * d.nty * d.ntz;
    blocks += (long long)d.ntx * d.ny * d.nz;  // storage blocks: rows of 32 cells
    if (n > maxbox) maxbox = n;
  }
  L.nblocks = blocks;
  L.ncell = cells;
  L.ntiles = tiles;
  L.stage_cells = maxbox < STAGE_CELLS ? maxbox : STAGE_CELLS;
  L.cap = prm->max_particles;
  L.bin_cap = prm->bin_capacity ? prm->bin_capacity : DEFAULT_BIN_CAP;
  const size_t s = prm->precision == HLBM_FP32 ? 4 : 2;
  size_t o = 0;
  L.off_f = o; o = align_up(o + (size_t)QVB * L.nblocks * s);
  L.off_boxes = o; o = align_up(o + sizeof(BoxDesc) * nb);
  L.off_P = o; o = align_up(o + sizeof(double) * PF_COUNT * (size_t)L.cap);
  L.off_shape = o; o = align_up(o + sizeof(int) * (size_t)L.cap);
  L.off_box = o; o = align_up(o + sizeof(int) * (size_t)L.cap);
  L.off_rec = o; o = align_up(o + sizeof(Rec) * (size_t)L.cap);
  L.off_part = o; o = align_up(o + sizeof(double) * 6 * MAX_PLANES * (size_t)L.cap);
  L.off_acc = o; o = align_up(o + sizeof(double) * 6 * (size_t)L.cap);
  L.off_chp = o; o = align_up(o + sizeof(int) * MAX_PLANES * (size_t)L.cap);
  L.off_chq = o; o = align_up(o + sizeof(int) * MAX_PLANES * (size_t)L.cap);
  L.off_pc0 = o; o = align_up(o + sizeof(int) * (size_t)L.cap);
  L.off_pnc = o; o = align_up(o + sizeof(int) * (size_t)L.cap);
  L.off_done = o; o = align_up(o + sizeof(int) * (size_t)L.cap);
  // interior-cell list for the momentum exchange from moments, in
  // ILIST_STRIPES stripes: together room for half of all cells (more than
  // any packing of non-overlapping particles needs), and each stripe for two
  // entries per cell of a whole brick
  L.ilist_cap = L.cap > 0 ? std::max((L.ncell / 2 + ILIST_STRIPES - 1) / ILIST_STRIPES,
                                     (long long)2 * TILE_X * TILE_Y * TILE_Z) : 0;
  L.off_lcnt = o; o = align_up(o + sizeof(int) * ILIST_STRIPES);
  L.off_lidx = o; o = align_up(o + sizeof(int2) * (size_t)L.ilist_cap * ILIST_STRIPES);
  L.off_lmom = o; o = align_up(o + sizeof(float4) * (size_t)L.ilist_cap * ILIST_STRIPES);
  for (int k = 0; k < 2; ++k) {
    L.off_cnt[k] = o; o = align_up(o + sizeof(int) * (size_t)L.ntiles);
    L.off_ids[k] = o; o = align_up(o + sizeof(int) * (size_t)L.ntiles * L.bin_cap);
  }
  L.off_status = o; o = align_up(o + sizeof(int));
  L.off_stage = o; o = align_up(o + sizeof(float) * Q * (size_t)L.stage_cells);
  L.grid_floats = prm->grid_floats;
  L.off_gdesc = o; o = align_up(o + (L.grid_floats > 0 ? sizeof(GridDesc) * MAX_GRIDS : 0));
  L.off_gvals = o; o = align_up(o + sizeof(float) * (size_t)L.grid_floats);
  L.total = o;
  return true;
}

thread_local std::string g_init_err;

}  // namespace

struct hlbm_ctx {
  std::vector<BoxDesc> boxes;
  hlbm_params prm{};
  Layout L{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  char* buf = nullptr;
  bool owns = false;
  void* f = nullptr;
  BoxDesc* d_boxes = nullptr;
  double* P = nullptr;
  int* d_shape = nullptr;
  int* d_box = nullptr;
  Rec* rec = nullptr;
  double* partial = nullptr;
  long long* acc = nullptr;
  int* chunk_p = nullptr;
  int* chunk_q = nullptr;
  int* p_chunk0 = nullptr;
  int* p_nchunk = nullptr;
  int* done = nullptr;
  int* ilist_count = nullptr;
  int2* ilist_idx = nullptr;
  float4* ilist_mom = nullptr;
  int nsm = 0;
  // odd steps take the bricks in reverse order when the populations are
  // within twice the L2 (a step then starts on what the last one ended
  // with, still in L2); larger lattices gain nothing and keep one order
  bool reverse_odd = false;
  int nchunks = 0;
  std::vector<int> h_nchunk;  // bounding-box planes per particle
  int mea_planes = 1;         // bounding-box planes per momentum-exchange block
  int mea_mode = HLBM_MEA_KERNEL;
  int* cnt[2] = {nullptr, nullptr};
  int* ids[2] = {nullptr, nullptr};
  int* status = nullptr;
  float* stage = nullptr;
  // pinned host staging of the motion state (rows X, U, omega, q, F, T, each
  // n doubles) and of the status word; hstage_ev marks the end of the last
  // upload that reads it
  double* hstage = nullptr;
  int* hstatus = nullptr;
  cudaEvent_t hstage_ev = nullptr;
  bool walls = false;
  // contact stiffness and range (an extension; 0 = off)
  double contact_k = 0.0, contact_zeta = 1.0;
  int np = 0;
  long long steps = 0;
  int sub_y = 4, sub_z = 2;
  int cells_x = 1;       // cells per thread along x
  bool pair_ok = false;  // the two-cell kernel may run
  // [0][parity]: step with the momentum-exchange kernel (after any change of
  // state); [1][parity]: step that takes the sums the previous collision made
  cudaGraphExec_t exec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  // two steps in one graph: [m][parity] = step(parity, m) then step(1 - parity)
  cudaGraphExec_t exec2[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  // GRAPH_STEPS steps in one graph, the same way (when more than two)
  cudaGraphExec_t execk[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  bool graphs_ok = false;
  bool moments_valid = false;  // the accumulator holds this state's momentum exchange
  int split = 0;  // a split step is open: 1 after its bounding-box exchange, 2 after its moments one
  // hstage holds the device's particle rows X .. T as downloaded by
  // hlbm_particle_state after step hst_steps (until an upload reuses it)
  bool hst_valid = false;
  long long hst_steps = -1;
  std::vector<int> h_shape, h_box;  // host copies
  // registered signed-distance grids: host copies of the samples and what
  // was derived from them
  struct HostGrid {
    int n[3];
    double h;
    std::vector<float> v;
    double V, I1[3], rc, rinf;
    double cap_h, cap_r;  // enclosing capsule about body z of the cells where B can be positive
    long long off;
  };
  std::vector<HostGrid> grids;
  long long grid_used = 0;
  GridDesc* d_gdesc = nullptr;
  float* d_gvals = nullptr;
  std::string err;
};

#define CK(call)                                                              \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);            \
      return HLBM_ERR_CUDA;                                                   \
    }                                                                         \
  } while (0)

static int fail(hlbm_ctx* h, int code, const std::string& msg) {
  h->err = msg;
  return code;
}

static LbmArgs lbm_args(const hlbm_ctx* h, int parity) {
  LbmArgs a{};
  a.nsm = h->nsm;
  a.f = h->f;
  a.ncell = h->L.ncell;
  a.boxes = h->d_boxes;
  a.nboxes = (int)h->boxes.size();
  a.sub_y = h->sub_y;
  a.sub_z = h->sub_z;
  a.cells_x = h->cells_x;
  a.nsub = (TILE_Y / h->sub_y) * (TILE_Z / h->sub_z);
  a.nbricks = h->L.ntiles * a.nsub;
  a.reverse = parity && h->reverse_odd;
  a.omega = (float)(1.0 / h->prm.tau);
  for (int j = 0; j < 3; ++j) a.ff[j] = (float)h->prm.fluid_force[j];
  a.eps = (float)h->prm.eps;
  a.inv_eps = (float)(1.0 / h->prm.eps);
  const double sc = h->prm.precision == HLBM_FP16 ? std::ldexp(1.0, h->prm.fp16_scale_log2) : 1.0;
  a.scale = (float)sc;
  a.inv_scale = (float)(1.0 / sc);
  a.bin_count = h->cnt[parity];
  a.bin_ids = h->ids[parity];
  a.bin_cap = h->L.bin_cap;
  a.rec = h->rec;
  const bool rec = h->mea_mode == HLBM_MEA_MOMENTS && h->ilist_idx;
  a.ilist_count = h->ilist_count;
  a.ilist_idx = rec ? h->ilist_idx : nullptr;
  a.ilist_mom = rec ? h->ilist_mom : nullptr;
  a.ilist_cap = h->L.ilist_cap;
  a.np = h->np;
  a.acc = h->acc;
  a.grids = h->grids.empty() ? GridSet{} : GridSet{h->d_gdesc, h->d_gvals};
  a.status = h->status;
  return a;
}

static PartArgs part_args(const hlbm_ctx* h, int parity) {
  PartArgs a{};
  a.P = h->P;
  a.cap = h->L.cap;
  a.np = h->np;
  a.shape = h->d_shape;
  a.box = h->d_box;
  a.rec = h->rec;
  a.boxes = h->d_boxes;
  for (int j = 0; j < 3; ++j) a.g[j] = h->prm.gravity[j];
  a.eps = h->prm.eps;
  a.f = h->f;
  const double sc = h->prm.precision == HLBM_FP16 ? std::ldexp(1.0, h->prm.fp16_scale_log2) : 1.0;
  a.scale = (float)sc;
  a.inv_scale = (float)(1.0 / sc);
  a.chunk_p = h->chunk_p;
  a.chunk_q = h->chunk_q;
  a.p_chunk0 = h->p_chunk0;
  a.p_nchunk = h->p_nchunk;
  a.nchunks = h->nchunks;
  a.mea_planes = h->mea_planes;
  a.partial = h->partial;
  a.done = h->done;
  a.acc = h->acc;
  a.from_acc = 0;
  a.contact_k = h->contact_k;
  a.contact_zeta = h->contact_zeta;
  a.grids = h->grids.empty() ? GridSet{} : GridSet{h->d_gdesc, h->d_gvals};
  a.nsm = h->nsm;
  a.ilist_count = h->ilist_count;
  a.bin_count = h->cnt[parity];
  a.bin_ids = h->ids[parity];
  a.bin_count_clear = h->cnt[1 - parity];
  a.ntiles = h->L.ntiles;
  a.bin_cap = h->L.bin_cap;
  a.status = h->status;
  return a;
}

// moments: the collision of the previous step recorded the post-collision
// moments of the cells inside particles, and the momentum exchange of this
// step runs from them; otherwise the bounding-box kernel computes it from
// the populations alone (always on the first step after a change of state).
// Kernels captured into a step's graph use programmatic dependent launch.
// steps per captured graph for long runs (two-step and one-step graphs
// take the rest)
#ifndef HLBM_GRAPH_STEPS
#define HLBM_GRAPH_STEPS 8
#endif
constexpr int GRAPH_STEPS = HLBM_GRAPH_STEPS;

static cudaError_t enqueue_step(hlbm_ctx* h, int parity, bool moments, cudaStream_t s) {
  cudaError_t e;
  LbmArgs la = lbm_args(h, parity);
  la.pdl = 1;
  if (h->np > 0) {
    PartArgs pa = part_args(h, parity);
    pa.pdl = 1;
    pa.from_acc = moments ? 1 : 0;
    if (moments) {
      if ((e = launch_mea_moments(la, h->prm.precision, parity, h->walls, h->nsm, s)) != cudaSuccess) return e;
    } else if ((e = launch_mea(pa, h->prm.precision, parity, s)) != cudaSuccess) {
      return e;
    }
    if ((e = launch_contact(pa, s)) != cudaSuccess) return e;
    if ((e = launch_update(pa, s)) != cudaSuccess) return e;
  }
  return launch_collide(la, h->prm.precision, parity, h->walls, h->np > 0, s);
}

static void drop_graphs(hlbm_ctx* h) {
  for (int f = 0; f < 2; ++f)
    for (int k = 0; k < 2; ++k) {
      if (h->exec[f][k]) cudaGraphExecDestroy(h->exec[f][k]);
      if (h->exec2[f][k]) cudaGraphExecDestroy(h->exec2[f][k]);
      if (h->execk[f][k]) cudaGraphExecDestroy(h->execk[f][k]);
      h->exec[f][k] = nullptr;
      h->exec2[f][k] = nullptr;
      h->execk[f][k] = nullptr;
    }
  h->graphs_ok = false;
}

static int build_graphs(hlbm_ctx* h) {
  drop_graphs(h);
  const bool mom = h->mea_mode == HLBM_MEA_MOMENTS;
  for (int gi = 0; gi < 12; ++gi) {
    const int kind = gi >> 2, moments = (gi >> 1) & 1, parity = gi & 1;
    const int nst = kind == 0 ? 1 : (kind == 1 ? 2 : GRAPH_STEPS);
    if (moments && !mom) continue;
    if (kind == 2 && GRAPH_STEPS <= 2) continue;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_step(h, parity, moments != 0, h->cap_stream);
    for (int j = 1; j < nst && e == cudaSuccess; ++j) e = enqueue_step(h, (parity + j) & 1, mom, h->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return fail(h, HLBM_ERR_CUDA, std::string("graph capture: ") +
                                        cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    cudaGraphExec_t* dst = kind == 0 ? &h->exec[moments][parity]
                                     : (kind == 1 ? &h->exec2[moments][parity] : &h->execk[moments][parity]);
    e = cudaGraphInstantiate(dst, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(h, HLBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  h->graphs_ok = true;
  return HLBM_OK;
}

// the status word already copied to the host: HLBM_OK, or clears the device
// flags and returns the error they name
static int status_code(hlbm_ctx* h, int st) {
  if (st == 0) return HLBM_OK;
  CK(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (st & ST_CAPACITY)
    return fail(h, HLBM_ERR_CAPACITY, "a 32x8x8 tile was touched by more particles than bin_capacity");
  if (st & ST_OVERLAP)
    return fail(h, HLBM_ERR_CAPACITY, "three particles overlap at one cell (the list of interior cells takes two)");
  if (st & ST_LIST_FULL)
    return fail(h, HLBM_ERR_CAPACITY, "the list of interior cells is full");
  if (st & ST_INTERNAL)
    return fail(h, HLBM_ERR_STATE, "the list of cells inside particles held an invalid entry");
  if (st & ST_LEFT_DOMAIN)
    return fail(h, HLBM_ERR_UNSTABLE, "a particle centre left the fluid domain through a wall");
  return fail(h, HLBM_ERR_UNSTABLE, "non-finite or non-positive density, or non-finite particle state");
}

static int read_status(hlbm_ctx* h) {
  CK(cudaMemcpyAsync(h->hstatus, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return status_code(h, *h->hstatus);
}

extern "C" {

void hlbm_default_params(hlbm_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->tau = 0.6;
  p->eps = 0.5;
  p->precision = HLBM_FP32;
  p->fp16_scale_log2 = 14;
}

size_t hlbm_required_bytes(int nboxes, const hlbm_box* boxes, const hlbm_params* prm) {
  Layout L;
  std::vector<BoxDesc> bd;
  std::string err;
  if (!make_layout(nboxes, boxes, prm, L, bd, err)) return 0;
  return L.total;
}

int hlbm_init_batch(hlbm_handle* out, int nboxes, const hlbm_box* boxes, const hlbm_params* prm,
                    void* cuda_stream, void* device_buf, size_t device_buf_bytes) {
  if (!out) { g_init_err = "out is NULL"; return HLBM_ERR_ARG; }
  *out = nullptr;
  hlbm_ctx* h = new hlbm_ctx();
  std::string err;
  if (!make_layout(nboxes, boxes, prm, h->L, h->boxes, err)) {
    g_init_err = err;
    delete h;
    return HLBM_ERR_ARG;
  }
  h->prm = *prm;
  if (h->prm.bin_capacity == 0) h->prm.bin_capacity = DEFAULT_BIN_CAP;
  h->stream = (cudaStream_t)cuda_stream;
  h->pair_ok = true;  // any nx: an odd nx leaves one cell in a row's last pair
  for (int b = 0; b < nboxes; ++b) h->walls |= boxes[b].bc_flags != 0;
  h->cells_x = 2;
  cudaError_t e;
  if (device_buf) {
    if (((uintptr_t)device_buf % ALIGN) || device_buf_bytes < h->L.total) {
      g_init_err = "device buffer too small or not 256-byte aligned";
      delete h;
      return HLBM_ERR_ARG;
    }
    h->buf = (char*)device_buf;
  } else {
    e = cudaMalloc((void**)&h->buf, h->L.total);
    if (e != cudaSuccess) {
      g_init_err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
      delete h;
      return HLBM_ERR_CUDA;
    }
    h->owns = true;
  }
  e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    g_init_err = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
    hlbm_destroy(h);
    return HLBM_ERR_CUDA;
  }
  {
    const size_t rows = sizeof(double) * 19 * (size_t)std::max(h->L.cap, 1);
    e = cudaMallocHost((void**)&h->hstage, rows + sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->hstage_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      g_init_err = std::string("host staging: ") + cudaGetErrorString(e);
      hlbm_destroy(h);
      return HLBM_ERR_CUDA;
    }
    h->hstatus = (int*)((char*)h->hstage + rows);
  }
  h->f = h->buf + h->L.off_f;
  h->d_boxes = (BoxDesc*)(h->buf + h->L.off_boxes);
  h->P = (double*)(h->buf + h->L.off_P);
  h->d_shape = (int*)(h->buf + h->L.off_shape);
  h->d_box = (int*)(h->buf + h->L.off_box);
  h->rec = (Rec*)(h->buf + h->L.off_rec);
  h->partial = (double*)(h->buf + h->L.off_part);
  h->acc = (long long*)(h->buf + h->L.off_acc);
  h->chunk_p = (int*)(h->buf + h->L.off_chp);
  h->chunk_q = (int*)(h->buf + h->L.off_chq);
  h->p_chunk0 = (int*)(h->buf + h->L.off_pc0);
  h->p_nchunk = (int*)(h->buf + h->L.off_pnc);
  h->done = (int*)(h->buf + h->L.off_done);
  h->ilist_count = (int*)(h->buf + h->L.off_lcnt);
  h->ilist_idx = h->L.ilist_cap > 0 ? (int2*)(h->buf + h->L.off_lidx) : nullptr;
  h->ilist_mom = h->L.ilist_cap > 0 ? (float4*)(h->buf + h->L.off_lmom) : nullptr;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) h->nsm = 0;
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) l2 = 0;
    const size_t s = h->prm.precision == HLBM_FP16 ? 2 : 4;
    h->reverse_odd = l2 > 0 && (size_t)QVB * h->L.nblocks * s <= 2 * (size_t)l2;
  }
  for (int k = 0; k < 2; ++k) {
    h->cnt[k] = (int*)(h->buf + h->L.off_cnt[k]);
    h->ids[k] = (int*)(h->buf + h->L.off_ids[k]);
  }
  h->status = (int*)(h->buf + h->L.off_status);
  h->stage = (float*)(h->buf + h->L.off_stage);
  h->d_gdesc = h->L.grid_floats > 0 ? (GridDesc*)(h->buf + h->L.off_gdesc) : nullptr;
  h->d_gvals = h->L.grid_floats > 0 ? (float*)(h->buf + h->L.off_gvals) : nullptr;
  // zero deviations are the fluid at rest with density 1 (f_i = w_i); empty bins
  e = cudaMemsetAsync(h->buf, 0, h->L.total, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_boxes, h->boxes.data(), sizeof(BoxDesc) * nboxes, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    g_init_err = std::string("initialisation: ") + cudaGetErrorString(e);
    hlbm_destroy(h);
    return HLBM_ERR_CUDA;
  }
  *out = h;
  return HLBM_OK;
}

int hlbm_init_lattice(hlbm_handle* out, int nx, int ny, int nz, int bc_flags, const hlbm_params* prm,
                      void* cuda_stream, void* device_buf, size_t device_buf_bytes) {
  hlbm_box b{nx, ny, nz, bc_flags};
  return hlbm_init_batch(out, 1, &b, prm, cuda_stream, device_buf, device_buf_bytes);
}

void hlbm_destroy(hlbm_handle h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->owns && h->buf) cudaFree(h->buf);
  if (h->hstage_ev) cudaEventDestroy(h->hstage_ev);
  if (h->hstage) cudaFreeHost(h->hstage);
  delete h;
}

const char* hlbm_last_error(hlbm_handle h) { return h ? h->err.c_str() : g_init_err.c_str(); }

int hlbm_num_particles(hlbm_handle h) { return h ? h->np : 0; }
long long hlbm_steps_done(hlbm_handle h) { return h ? h->steps : 0; }

// volume, mass, principal inertia, circumscribed radius and the radius beyond
// which the indicator of Eq. B vanishes
static void mass_properties(int shape, const double a[3], double rho, double* V, double* m,
                            double I[3], double* rc, double* rinf, double eps) {
  if (shape == HLBM_SPHERE) {
    *V = 4.0 / 3.0 * PI_D * a[0] * a[0] * a[0];
    *m = rho * *V;
    for (int j = 0; j < 3; ++j) I[j] = 0.4 * *m * a[0] * a[0];
    *rc = a[0];
    *rinf = a[0] + eps / 2.0;
  } else if (shape == HLBM_ELLIPSOID) {
    *V = 4.0 / 3.0 * PI_D * a[0] * a[1] * a[2];
    *m = rho * *V;
    I[0] = *m * (a[1] * a[1] + a[2] * a[2]) / 5.0;
    I[1] = *m * (a[0] * a[0] + a[2] * a[2]) / 5.0;
    I[2] = *m * (a[0] * a[0] + a[1] * a[1]) / 5.0;
    const double amax = std::fmax(a[0], std::fmax(a[1], a[2]));
    const double amin = std::fmin(a[0], std::fmin(a[1], a[2]));
    *rc = amax;
    // algebraic distance: d >= (k - 1) a_min and |r| <= k a_max
    *rinf = amax * (1.0 + eps / (2.0 * amin));
  } else if (shape == HLBM_CAPSULE) {
    // a cylinder of radius r and length 2h with two hemispherical caps; a
    // cap's moment about a diameter of its flat face, 2/5 m r^2, moves to the
    // centre through the cap's centroid 3r/8 from that face
    const double r = a[0], hh = a[2];
    const double Vc = PI_D * r * r * 2.0 * hh, Vs = 4.0 / 3.0 * PI_D * r * r * r;
    *V = Vc + Vs;
    *m = rho * *V;
    const double mc = rho * Vc, ms = rho * Vs;
    I[0] = I[1] = mc * (r * r / 4.0 + hh * hh / 3.0) + ms * (0.4 * r * r + hh * hh + 0.75 * hh * r);
    I[2] = mc * r * r / 2.0 + ms * 0.4 * r * r;
    *rc = hh + r;
    *rinf = *rc + eps / 2.0;
  } else {
    *V = 8.0 * a[0] * a[1] * a[2];
    *m = rho * *V;
    I[0] = *m * (a[1] * a[1] + a[2] * a[2]) / 3.0;
    I[1] = *m * (a[0] * a[0] + a[2] * a[2]) / 3.0;
    I[2] = *m * (a[0] * a[0] + a[1] * a[1]) / 3.0;
    *rc = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    *rinf = *rc + eps / 2.0;
  }
}

// FP64 trilinear blend of a registered grid at body offset r (+inf outside)
static double grid_blend_host(const hlbm_ctx::HostGrid& g, const double r[3]) {
  int i0[3];
  double t[3];
  for (int j = 0; j < 3; ++j) {
    const double x = r[j] / g.h + 0.5 * (g.n[j] - 1);
    if (!(x >= 0.0 && x <= (double)(g.n[j] - 1))) return HUGE_VAL;
    i0[j] = std::min((int)std::floor(x), g.n[j] - 2);
    t[j] = x - i0[j];
  }
  auto at = [&](int dx, int dy, int dz) {
    return (double)g.v[((size_t)(i0[2] + dz) * g.n[1] + (i0[1] + dy)) * g.n[0] + (i0[0] + dx)];
  };
  double e[2][2];
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy) e[dz][dy] = at(0, dy, dz) + t[0] * (at(1, dy, dz) - at(0, dy, dz));
  const double f0 = e[0][0] + t[1] * (e[0][1] - e[0][0]);
  const double f1 = e[1][0] + t[1] * (e[1][1] - e[1][0]);
  return f0 + t[2] * (f1 - f0);
}

static void wrap_host(const BoxDesc& bd, double X[3]) {
  const int n[3] = {bd.nx, bd.ny, bd.nz};
  for (int j = 0; j < 3; ++j) {
    if ((bd.bc >> j) & 1) continue;
    const double L = (double)n[j];
    X[j] = X[j] - L * std::floor(X[j] / L);
    if (X[j] >= L) X[j] -= L;
  }
}

static int upload_fields(hlbm_ctx* h, int p0, int n, const std::vector<double>& tab) {
  // tab: PF_COUNT fields of n values each
  for (int fld = 0; fld < PF_COUNT; ++fld)
    CK(cudaMemcpyAsync(h->P + (size_t)fld * h->L.cap + p0, tab.data() + (size_t)fld * n,
                       sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
  return HLBM_OK;
}

// Two capsules about the body z axis of a grid, each the best of 65
// half-lengths.  Enclosing (g.cap_h, g.cap_r): the smallest that holds every
// grid cell with a corner below eps/2 (the blend is a convex combination of
// the corners, so B > 0 and the inside lie in those cells, and a cell whose
// corners are in the capsule is in it).  Inscribed (d.in_h, d.in_r2): the
// largest that meets only grid cells all of whose corners are below
// -(eps/2 + 1e-3), kept 1e-3 cells off the others (a cell's distance from the
// axis segment is bounded by its centre's minus its half-diagonal); there
// the blend is below -eps/2, so the coupling needs no blend.
static void grid_capsules(hlbm_ctx::HostGrid& g, double half_eps, GridDesc& d) {
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  auto val = [&](int i, int j, int k) { return (double)g.v[((size_t)k * ny + j) * nx + i]; };
  auto pos = [&](double i, double j, double k, double r[3]) {
    r[0] = (i - 0.5 * (nx - 1)) * g.h;
    r[1] = (j - 0.5 * (ny - 1)) * g.h;
    r[2] = (k - 0.5 * (nz - 1)) * g.h;
  };
  auto seg_d2 = [](const double r[3], double hh) {
    const double t = r[2] - std::min(std::max(r[2], -hh), hh);
    return r[0] * r[0] + r[1] * r[1] + t * t;
  };
  std::vector<std::array<double, 3>> hold, avoid;  // corners to hold, centres of cells to avoid
  std::vector<char> mark((size_t)nx * ny * nz, 0);
  const double deep = -(half_eps + 1e-3);
  for (int k = 0; k + 1 < nz; ++k)
    for (int j = 0; j + 1 < ny; ++j)
      for (int i = 0; i + 1 < nx; ++i) {
        double vmin = HUGE_VAL, vmax = -HUGE_VAL;
        for (int c = 0; c < 8; ++c) {
          const double v = val(i + (c & 1), j + ((c >> 1) & 1), k + (c >> 2));
          vmin = std::min(vmin, v);
          vmax = std::max(vmax, v);
        }
        if (vmin < half_eps)
          for (int c = 0; c < 8; ++c) mark[((size_t)(k + (c >> 2)) * ny + j + ((c >> 1) & 1)) * nx + i + (c & 1)] = 1;
        if (!(vmax < deep)) {
          double r[3];
          pos(i + 0.5, j + 0.5, k + 0.5, r);
          avoid.push_back({r[0], r[1], r[2]});
        }
      }
  double zmax = 0.0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        if (mark[((size_t)k * ny + j) * nx + i]) {
          double r[3];
          pos(i, j, k, r);
          hold.push_back({r[0], r[1], r[2]});
          zmax = std::max(zmax, std::fabs(r[2]));
        }
  g.cap_h = 0.0;
  g.cap_r = g.rinf;
  double best = HUGE_VAL;
  for (int t = 0; t <= 64; ++t) {
    const double hh = zmax * t / 64.0;
    double r2 = 0.0;
    for (const auto& c : hold) r2 = std::max(r2, seg_d2(c.data(), hh));
    const double r = std::sqrt(r2), vol = M_PI * r * r * 2.0 * hh + 4.0 / 3.0 * M_PI * r * r * r;
    if (vol < best) { best = vol; g.cap_h = hh; g.cap_r = r; }
  }
  const double half_diag = 0.5 * std::sqrt(3.0) * g.h;
  double in_h = 0.0, in_r = -1.0;
  best = 0.0;
  for (int t = 0; t <= 64; ++t) {
    const double hh = zmax * t / 64.0;
    double r2 = HUGE_VAL;
    for (const auto& c : avoid) r2 = std::min(r2, seg_d2(c.data(), hh));
    const double r = std::sqrt(r2) - half_diag - 1e-3;
    if (!(r > 0.0)) continue;
    const double vol = M_PI * r * r * 2.0 * hh + 4.0 / 3.0 * M_PI * r * r * r;
    if (vol > best) { best = vol; in_h = hh; in_r = r; }
  }
  d.in_h = (float)in_h;
  d.in_r2 = in_r > 0.0 ? (float)(in_r * in_r) : -1.0f;
  d.in_d = (float)(deep - 0.01);
}

int hlbm_add_grid(hlbm_handle h, int nx, int ny, int nz, double spacing, const float* values, int* grid_id) {
  if (!h) return HLBM_ERR_ARG;
  if (!values || !grid_id || nx < 2 || ny < 2 || nz < 2 || !(spacing > 0.0) || !std::isfinite(spacing))
    return fail(h, HLBM_ERR_ARG, "grid sizes must be >= 2, the spacing finite and > 0, the arrays non-NULL");
  const long long nv = (long long)nx * ny * nz;
  if ((int)h->grids.size() >= MAX_GRIDS) return fail(h, HLBM_ERR_CAPACITY, "HLBM_MAX_GRIDS grids already registered");
  if (h->grid_used + nv > h->L.grid_floats)
    return fail(h, HLBM_ERR_CAPACITY, "the grid samples exceed grid_floats of the parameters");
  hlbm_ctx::HostGrid g;
  g.n[0] = nx; g.n[1] = ny; g.n[2] = nz;
  g.h = spacing;
  g.v.assign(values, values + nv);
  bool neg = false;
  for (float v : g.v) {
    if (!std::isfinite(v)) return fail(h, HLBM_ERR_ARG, "non-finite grid sample");
    neg = neg || v < 0.0f;
  }
  if (!neg) return fail(h, HLBM_ERR_ARG, "a grid needs a negative sample");
  const double half_eps = h->prm.eps / 2.0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const bool face = i == 0 || j == 0 || k == 0 || i == nx - 1 || j == ny - 1 || k == nz - 1;
        if (face && !((double)g.v[((size_t)k * ny + j) * nx + i] >= half_eps))
          return fail(h, HLBM_ERR_ARG, "grid samples on its faces must be >= eps/2");
      }
  // radii: the farthest corner of the grid cells holding a corner below 0
  // (the body) and below eps/2 (where B of Eq. B can be positive)
  g.rc = g.rinf = 0.0;
  for (int k = 0; k + 1 < nz; ++k)
    for (int j = 0; j + 1 < ny; ++j)
      for (int i = 0; i + 1 < nx; ++i) {
        double vmin = HUGE_VAL, cmax = 0.0;
        for (int c = 0; c < 8; ++c) {
          const int ii = i + (c & 1), jj = j + ((c >> 1) & 1), kk = k + (c >> 2);
          vmin = std::min(vmin, (double)g.v[((size_t)kk * ny + jj) * nx + ii]);
          const double x = (ii - 0.5 * (nx - 1)) * spacing, y = (jj - 0.5 * (ny - 1)) * spacing,
                       z = (kk - 0.5 * (nz - 1)) * spacing;
          cmax = std::max(cmax, std::sqrt(x * x + y * y + z * z));
        }
        if (vmin < 0.0) g.rc = std::max(g.rc, cmax);
        if (vmin < half_eps) g.rinf = std::max(g.rinf, cmax);
      }
  if (!(g.rc <= 30.0)) return fail(h, HLBM_ERR_ARG, "circumscribed radius above 30 cells");
  // volume and second moments per unit density: midpoint rule over 4^3
  // sub-cells of every grid cell, a sub-cell counting where the blend < 0
  const int sub = 4;
  const double dv = (spacing / sub) * (spacing / sub) * (spacing / sub);
  double V = 0.0, c1[3] = {0.0, 0.0, 0.0}, S[3][3] = {{0.0}};
  for (int k = 0; k + 1 < nz; ++k)
    for (int j = 0; j + 1 < ny; ++j)
      for (int i = 0; i + 1 < nx; ++i)
        for (int mz = 0; mz < sub; ++mz)
          for (int my = 0; my < sub; ++my)
            for (int mx = 0; mx < sub; ++mx) {
              const double r[3] = {(i + (mx + 0.5) / sub - 0.5 * (nx - 1)) * spacing,
                                   (j + (my + 0.5) / sub - 0.5 * (ny - 1)) * spacing,
                                   (k + (mz + 0.5) / sub - 0.5 * (nz - 1)) * spacing};
              if (!(grid_blend_host(g, r) < 0.0)) continue;
              V += dv;
              for (int a = 0; a < 3; ++a) {
                c1[a] += r[a] * dv;
                for (int b = 0; b < 3; ++b) S[a][b] += r[a] * r[b] * dv;
              }
            }
  g.V = V;
  g.I1[0] = S[1][1] + S[2][2];
  g.I1[1] = S[0][0] + S[2][2];
  g.I1[2] = S[0][0] + S[1][1];
  const double imax = std::max(g.I1[0], std::max(g.I1[1], g.I1[2]));
  bool principal = V > 0.0;
  for (int a = 0; a < 3; ++a) principal = principal && std::fabs(c1[a] / V) <= spacing / 100.0;
  principal = principal && std::fabs(S[0][1]) <= 1e-3 * imax && std::fabs(S[0][2]) <= 1e-3 * imax &&
              std::fabs(S[1][2]) <= 1e-3 * imax;
  if (!principal)
    return fail(h, HLBM_ERR_ARG, "the grid's body frame must be its principal frame about the centre of mass");
  g.off = h->grid_used;
  GridDesc d{};
  d.n[0] = nx; d.n[1] = ny; d.n[2] = nz;
  d.ih = (float)(1.0 / spacing);
  for (int j = 0; j < 3; ++j) d.half[j] = (float)(0.5 * (g.n[j] - 1));
  grid_capsules(g, half_eps, d);
  d.off = g.off;
  const int id = (int)h->grids.size();
  CK(cudaMemcpyAsync(h->d_gvals + g.off, g.v.data(), sizeof(float) * nv, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->d_gdesc + id, &d, sizeof(GridDesc), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->grid_used += nv;
  h->grids.push_back(std::move(g));
  drop_graphs(h);  // the captured steps name the grids by pointer (set once grids exist)
  *grid_id = id;
  return HLBM_OK;
}

int hlbm_add_particles(hlbm_handle h, int n, const int* box_id, const int* shape,
                       const double* shape_params, const double* X, const double* U,
                       const double* omega, const double* quat, const double* rho_p) {
  if (!h) return HLBM_ERR_ARG;
  if (h->steps > 0) return fail(h, HLBM_ERR_STATE, "particles can only be added before the first step");
  if (n < 0 || (n > 0 && (!shape || !shape_params || !X || !rho_p)))
    return fail(h, HLBM_ERR_ARG, "n < 0 or a required array is NULL");
  if (h->np + n > h->L.cap) return fail(h, HLBM_ERR_CAPACITY, "more particles than max_particles");
  if (n == 0) return HLBM_OK;
  std::vector<double> tab((size_t)PF_COUNT * n, 0.0);
  std::vector<int> sh(n), bx(n), nch(n);
  auto T = [&](int fld, int k) -> double& { return tab[(size_t)fld * n + k]; };
  for (int k = 0; k < n; ++k) {
    const int b = box_id ? box_id[k] : 0;
    if (b < 0 || b >= (int)h->boxes.size()) return fail(h, HLBM_ERR_ARG, "box_id out of range");
    const BoxDesc& bd = h->boxes[b];
    const int s = shape[k];
    if (s < HLBM_SPHERE || s > HLBM_GRID) return fail(h, HLBM_ERR_ARG, "unknown shape");
    double a[3];
    int gid = -1;
    if (s == HLBM_GRID) {
      const double v = shape_params[3 * k];
      if (!(v >= 0.0 && v < (double)h->grids.size() && v == std::floor(v)))
        return fail(h, HLBM_ERR_ARG, "a grid particle must name a registered grid");
      gid = (int)v;
      for (int j = 0; j < 3; ++j) a[j] = h->grids[gid].rc;  // the record's radius
    } else {
      for (int j = 0; j < 3; ++j) {
        a[j] = (s == HLBM_SPHERE || (s == HLBM_CAPSULE && j == 1)) ? shape_params[3 * k] : shape_params[3 * k + j];
        if (!(a[j] > 0.0) || !std::isfinite(a[j])) return fail(h, HLBM_ERR_ARG, "shape sizes must be finite and > 0");
      }
    }
    const double rho = rho_p[k];
    if (!(rho > 0.0) || !std::isfinite(rho)) return fail(h, HLBM_ERR_ARG, "rho_p must be finite and > 0");
    double q[4] = {1.0, 0.0, 0.0, 0.0};
    if (quat) {
      double nq = 0.0;
      for (int j = 0; j < 4; ++j) nq += quat[4 * k + j] * quat[4 * k + j];
      if (!(nq > 0.0) || !std::isfinite(nq)) return fail(h, HLBM_ERR_ARG, "quaternion must be finite and non-zero");
      nq = std::sqrt(nq);
      for (int j = 0; j < 4; ++j) q[j] = quat[4 * k + j] / nq;
    }
    double V, m, I[3], rc, rinf;
    if (s == HLBM_GRID) {
      const auto& g = h->grids[gid];
      V = g.V;
      m = rho * V;
      for (int j = 0; j < 3; ++j) I[j] = rho * g.I1[j];
      rc = g.rc;
      rinf = g.rinf;
    } else {
      mass_properties(s, a, rho, &V, &m, I, &rc, &rinf, h->prm.eps);
    }
    if (!(rc <= 30.0)) return fail(h, HLBM_ERR_ARG, "circumscribed radius above 30 cells");
    double x[3];
    const int nn[3] = {bd.nx, bd.ny, bd.nz};
    for (int j = 0; j < 3; ++j) {
      x[j] = X[3 * k + j];
      const double u = U ? U[3 * k + j] : 0.0, w = omega ? omega[3 * k + j] : 0.0;
      if (!std::isfinite(x[j]) || !std::isfinite(u) || !std::isfinite(w))
        return fail(h, HLBM_ERR_ARG, "non-finite particle state");
      if ((bd.bc >> j) & 1) {
        const bool cut = j == 2 && (bd.bc & HLBM_CUT_Z);  // a slab's cut faces: centres may lie beyond
        if (!cut && !(x[j] > -0.5 && x[j] < nn[j] - 0.5))
          return fail(h, HLBM_ERR_ARG, "centre outside the box on a wall axis");
      } else if (!(2.0 * (rinf + 2.0) < nn[j])) {
        return fail(h, HLBM_ERR_ARG, "particle spans half a periodic axis or more");
      }
      T(PF_U + j, k) = u;
      T(PF_W + j, k) = w;
      T(PF_I + j, k) = I[j];
      T(PF_II + j, k) = 1.0 / I[j];
      T(PF_A + j, k) = a[j];
      // a grid particle keeps its grid id here (the record's inverse sizes
      // are unused for it)
      T(PF_IA + j, k) = s == HLBM_GRID ? (double)gid : (double)(float)(1.0 / a[j]);
    }
    if (s == HLBM_GRID) {
      // the record's ia[1], ia[2] hold the grid's enclosing capsule
      T(PF_IA + 1, k) = h->grids[gid].cap_h;
      T(PF_IA + 2, k) = h->grids[gid].cap_r;
    }
    wrap_host(bd, x);
    for (int j = 0; j < 3; ++j) T(PF_X + j, k) = x[j];
    for (int j = 0; j < 4; ++j) T(PF_Q + j, k) = q[j];
    T(PF_M, k) = m;
    T(PF_IM, k) = 1.0 / m;
    T(PF_V, k) = V;
    T(PF_RHO, k) = rho;
    T(PF_RC, k) = rc;
    T(PF_RINF, k) = rinf;
    sh[k] = s;
    bx[k] = b;
    nch[k] = (int)std::ceil(2.0 * rc) + 2;  // bounding-box planes, at most MAX_PLANES
  }
  const int p0 = h->np;
  int rc = upload_fields(h, p0, n, tab);
  if (rc != HLBM_OK) return rc;
  CK(cudaMemcpyAsync(h->d_shape + p0, sh.data(), sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->d_box + p0, bx.data(), sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
  h->np += n;
  h->hst_valid = false;
  h->h_shape.insert(h->h_shape.end(), sh.begin(), sh.end());
  h->h_box.insert(h->h_box.end(), bx.begin(), bx.end());
  h->h_nchunk.insert(h->h_nchunk.end(), nch.begin(), nch.end());
  {
    // one momentum-exchange block per particle and run of mea_planes
    // bounding-box planes: one plane while the blocks of one plane each fill
    // the GPU at most four times (the walk is latency-bound and a block's
    // fixed cost is then spread over few waves), up to three for many
    // particles, where each block's fixed cost counts in every wave
    long long planes = 0;
    for (int q = 0; q < h->np; ++q) planes += h->h_nchunk[q];
    const long long resident = (long long)(h->nsm > 0 ? h->nsm : 152) * MEA_MINBLOCKS;
    h->mea_planes = (int)std::min(3LL, std::max(1LL, planes / (4 * resident)));
    const int G = h->mea_planes;
    std::vector<int> cp, cq, c0(h->np), cn(h->np);
    for (int q = 0; q < h->np; ++q) {
      c0[q] = (int)cp.size();
      cn[q] = (h->h_nchunk[q] + G - 1) / G;
      for (int k = 0; k < cn[q]; ++k) {
        cp.push_back(q);
        cq.push_back(k * G);
      }
    }
    h->nchunks = (int)cp.size();
    CK(cudaMemcpyAsync(h->chunk_p, cp.data(), sizeof(int) * cp.size(), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->chunk_q, cq.data(), sizeof(int) * cq.size(), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->p_chunk0, c0.data(), sizeof(int) * c0.size(), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(h->p_nchunk, cn.data(), sizeof(int) * cn.size(), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  CK(launch_records(part_args(h, 0), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  drop_graphs(h);
  h->moments_valid = false;
  return HLBM_OK;
}

int hlbm_set_particle_state(hlbm_handle h, const double* X, const double* U, const double* omega,
                            const double* quat) {
  if (!h) return HLBM_ERR_ARG;
  const int n = h->np;
  if (n == 0) return HLBM_OK;
  for (int k = 0; X && k < n; ++k)
    for (int j = 0; j < 3; ++j)
      if (!std::isfinite(X[3 * k + j])) return fail(h, HLBM_ERR_ARG, "non-finite position");
  for (int k = 0; quat && k < n; ++k) {
    double nq = 0.0;
    for (int j = 0; j < 4; ++j) nq += quat[4 * k + j] * quat[4 * k + j];
    if (!(nq > 0.0) || !std::isfinite(nq)) return fail(h, HLBM_ERR_ARG, "quaternion must be finite and non-zero");
  }
  // the staging rows may still feed the previous upload
  CK(cudaEventSynchronize(h->hstage_ev));
  double* S = h->hstage;  // row r holds component r of the state, n doubles
  // The cells inside the particles (and so the list the last collision
  // recorded) depend on positions and, for non-spheres, orientations only:
  // when both come back as the state downloaded after this very step, bit
  // for bit, the next step may still take the momentum exchange from the
  // recorded moments.
  const bool fresh = h->hst_valid && h->hst_steps == h->steps;
  bool moved = false;
  if (X)
    for (int k = 0; k < n; ++k) {
      double x[3] = {X[3 * k], X[3 * k + 1], X[3 * k + 2]};
      wrap_host(h->boxes[h->h_box[k]], x);
      for (int j = 0; j < 3; ++j) {
        moved = moved || !fresh || x[j] != S[(size_t)(PF_X + j) * n + k];
        S[(size_t)(PF_X + j) * n + k] = x[j];
      }
    }
  auto rows = [&](int fld, int ncomp, const double* src) {
    for (int j = 0; j < ncomp; ++j)
      for (int k = 0; k < n; ++k) S[(size_t)(fld + j) * n + k] = src[(size_t)ncomp * k + j];
  };
  if (U) rows(PF_U, 3, U);
  if (omega) rows(PF_W, 3, omega);
  if (quat)
    for (int k = 0; k < n; ++k) {
      double nq = 0.0;
      for (int j = 0; j < 4; ++j) nq += quat[4 * k + j] * quat[4 * k + j];
      nq = std::sqrt(nq);
      for (int j = 0; j < 4; ++j) {
        const double v = quat[4 * k + j] / nq;
        if (h->h_shape[k] != HLBM_SPHERE) moved = moved || !fresh || v != S[(size_t)(PF_Q + j) * n + k];
        S[(size_t)(PF_Q + j) * n + k] = v;
      }
    }
  // the staging rows now hold the upload, not the downloaded state
  h->hst_valid = false;
  if (moved) h->moments_valid = false;
  // one strided copy per run of consecutive fields that were given
  const bool given[4] = {X != nullptr, U != nullptr, omega != nullptr, quat != nullptr};
  const int row0[5] = {PF_X, PF_U, PF_W, PF_Q, PF_F};
  for (int f0 = 0; f0 < 4;) {
    if (!given[f0]) { ++f0; continue; }
    int f1 = f0;
    while (f1 < 4 && given[f1]) ++f1;
    const int r0 = row0[f0], nr = row0[f1] - r0;
    CK(cudaMemcpy2DAsync(h->P + (size_t)r0 * h->L.cap, sizeof(double) * h->L.cap, S + (size_t)r0 * n,
                         sizeof(double) * n, sizeof(double) * n, nr, cudaMemcpyHostToDevice, h->stream));
    f0 = f1;
  }
  CK(cudaEventRecord(h->hstage_ev, h->stream));
  CK(launch_records(part_args(h, 0), h->stream));
  return HLBM_OK;
}

int hlbm_step(hlbm_handle h, int nsteps) {
  if (!h) return HLBM_ERR_ARG;
  if (h->split) return fail(h, HLBM_ERR_STATE, "a split step is open (finish it with hlbm_step_with_forces)");
  if (nsteps < 0) return fail(h, HLBM_ERR_ARG, "nsteps < 0");
  if (nsteps == 0) return HLBM_OK;
  if (!h->graphs_ok) {
    const int rc = build_graphs(h);
    if (rc != HLBM_OK) return rc;
  }
  for (int k = 0; k < nsteps;) {
    const int moments = (h->moments_valid && h->np > 0) ? 1 : 0;
    const int parity = (int)((h->steps + k) & 1);
    if (GRAPH_STEPS > 2 && nsteps - k >= GRAPH_STEPS) {
      CK(cudaGraphLaunch(h->execk[moments][parity], h->stream));
      k += GRAPH_STEPS;
    } else if (nsteps - k >= 2) {
      CK(cudaGraphLaunch(h->exec2[moments][parity], h->stream));
      k += 2;
    } else {
      CK(cudaGraphLaunch(h->exec[moments][parity], h->stream));
      k += 1;
    }
    h->moments_valid = h->mea_mode == HLBM_MEA_MOMENTS;
  }
  h->steps += nsteps;
  return HLBM_OK;
}

// ------------------------------------------------------- z-slab sub-domains
int hlbm_set_owned_planes(hlbm_handle h, int box, int z_lo, int z_hi) {
  if (!h) return HLBM_ERR_ARG;
  if (box < 0 || box >= (int)h->boxes.size()) return fail(h, HLBM_ERR_ARG, "bad box");
  BoxDesc& bd = h->boxes[box];
  if (!(bd.bc & HLBM_CUT_Z)) return fail(h, HLBM_ERR_ARG, "owned planes need a box with HLBM_CUT_Z");
  if (z_lo < 0 || z_hi > bd.nz || z_lo >= z_hi) return fail(h, HLBM_ERR_ARG, "owned planes out of the box");
  CK(cudaStreamSynchronize(h->stream));
  bd.own_lo = z_lo;
  bd.own_hi = z_hi;
  CK(cudaMemcpyAsync(h->d_boxes + box, &bd, sizeof(BoxDesc), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->moments_valid = false;  // the recorded interior cells may hold ghost planes
  return HLBM_OK;
}

int hlbm_plane_slots(hlbm_handle h, int box, int z, int dir, void* host, int put) {
  if (!h) return HLBM_ERR_ARG;
  if (box < 0 || box >= (int)h->boxes.size() || !host || (dir != 1 && dir != -1) || (put != 0 && put != 1))
    return fail(h, HLBM_ERR_ARG, "bad box, direction or buffer");
  const BoxDesc& bd = h->boxes[box];
  if (z < 0 || z >= bd.nz) return fail(h, HLBM_ERR_ARG, "plane out of the box");
  const long long ncell = (long long)bd.nx * bd.ny;
  const size_t bytes = 5 * (size_t)ncell * (h->prm.precision == HLBM_FP32 ? 4 : 2);
  if (bytes > sizeof(float) * Q * (size_t)h->L.stage_cells)
    return fail(h, HLBM_ERR_CAPACITY, "plane larger than the staging area");
  if (put) CK(cudaMemcpyAsync(h->stage, host, bytes, cudaMemcpyHostToDevice, h->stream));
  CK(launch_plane_slots(lbm_args(h, 0), h->prm.precision, box, z, dir, (int)ncell, h->stage, put, h->stream));
  if (!put) CK(cudaMemcpyAsync(host, h->stage, bytes, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (put) h->moments_valid = h->moments_valid && h->mea_mode == HLBM_MEA_MOMENTS;
  return HLBM_OK;
}

int hlbm_step_forces(hlbm_handle h, double* F, double* T) {
  if (!h) return HLBM_ERR_ARG;
  if (h->split) return fail(h, HLBM_ERR_STATE, "a split step is already open");
  const int n = h->np;
  if (n > 0 && (!F || !T)) return fail(h, HLBM_ERR_ARG, "NULL force or torque array");
  const int parity = (int)(h->steps & 1);
  if (n == 0) {
    h->split = 1;
    return HLBM_OK;
  }
  const bool moments = h->moments_valid;
  if (moments) {
    LbmArgs la = lbm_args(h, parity);
    CK(launch_mea_moments(la, h->prm.precision, parity, h->walls, h->nsm, h->stream));
    std::vector<long long> acc((size_t)6 * n);
    CK(cudaMemcpyAsync(acc.data(), h->acc, sizeof(long long) * acc.size(), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemsetAsync(h->acc, 0, sizeof(long long) * acc.size(), h->stream));
    const int st = read_status(h);
    if (st != HLBM_OK) return st;
    const double unit = 1.0 / (double)(1LL << ACC_FRAC_BITS);
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < 3; ++j) {
        F[3 * k + j] = (double)acc[6 * (size_t)k + j] * unit;
        T[3 * k + j] = (double)acc[6 * (size_t)k + 3 + j] * unit;
      }
  } else {
    CK(launch_mea(part_args(h, parity), h->prm.precision, parity, h->stream));
    std::vector<double> rows((size_t)6 * n);
    CK(cudaMemcpy2DAsync(rows.data(), sizeof(double) * n, h->P + (size_t)PF_F * h->L.cap, sizeof(double) * h->L.cap,
                         sizeof(double) * n, 6, cudaMemcpyDeviceToHost, h->stream));
    const int st = read_status(h);
    if (st != HLBM_OK) return st;
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < 3; ++j) {
        F[3 * k + j] = rows[(size_t)j * n + k];
        T[3 * k + j] = rows[(size_t)(3 + j) * n + k];
      }
  }
  h->split = moments ? 2 : 1;
  return HLBM_OK;
}

int hlbm_step_with_forces(hlbm_handle h, const double* F, const double* T) {
  if (!h) return HLBM_ERR_ARG;
  if (!h->split) return fail(h, HLBM_ERR_STATE, "no split step is open (call hlbm_step_forces first)");
  const int n = h->np;
  if (n > 0 && (!F || !T)) return fail(h, HLBM_ERR_ARG, "NULL force or torque array");
  for (int k = 0; k < 3 * n; ++k)
    if (!std::isfinite(F[k]) || !std::isfinite(T[k])) return fail(h, HLBM_ERR_ARG, "non-finite force or torque");
  const int parity = (int)(h->steps & 1);
  if (n > 0) {
    std::vector<double> rows((size_t)6 * n);
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < 3; ++j) {
        rows[(size_t)j * n + k] = F[3 * k + j];
        rows[(size_t)(3 + j) * n + k] = T[3 * k + j];
      }
    CK(cudaMemcpy2DAsync(h->P + (size_t)PF_F * h->L.cap, sizeof(double) * h->L.cap, rows.data(), sizeof(double) * n,
                         sizeof(double) * n, 6, cudaMemcpyHostToDevice, h->stream));
    PartArgs pa = part_args(h, parity);
    pa.from_acc = 0;
    CK(launch_contact(pa, h->stream));
    CK(launch_update(pa, h->stream));
  }
  CK(launch_collide(lbm_args(h, parity), h->prm.precision, parity, h->walls, n > 0, h->stream));
  CK(cudaStreamSynchronize(h->stream));  // the host rows above are released
  h->split = 0;
  h->steps += 1;
  h->moments_valid = h->mea_mode == HLBM_MEA_MOMENTS;
  h->hst_valid = false;
  return HLBM_OK;
}

int hlbm_sync(hlbm_handle h) {
  if (!h) return HLBM_ERR_ARG;
  return read_status(h);
}

int hlbm_particle_state(hlbm_handle h, double* X, double* U, double* omega, double* quat, double* F,
                        double* T) {
  if (!h) return HLBM_ERR_ARG;
  const int n = h->np;
  if (n == 0) return read_status(h);
  // rows X, U, omega, q, F, T (19 components) in one strided copy, then the status word
  double* S = h->hstage;
  CK(cudaMemcpy2DAsync(S, sizeof(double) * n, h->P + (size_t)PF_X * h->L.cap, sizeof(double) * h->L.cap,
                       sizeof(double) * n, PF_T + 3 - PF_X, cudaMemcpyDeviceToHost, h->stream));
  const int st = read_status(h);
  if (st == HLBM_ERR_CUDA) return st;
  h->hst_valid = true;
  h->hst_steps = h->steps;
  auto get = [&](int fld, int ncomp, double* dst) {
    if (!dst) return;
    for (int j = 0; j < ncomp; ++j)
      for (int k = 0; k < n; ++k) dst[(size_t)ncomp * k + j] = S[(size_t)(fld + j) * n + k];
  };
  get(PF_X, 3, X);
  get(PF_U, 3, U);
  get(PF_W, 3, omega);
  get(PF_Q, 4, quat);
  get(PF_F, 3, F);
  get(PF_T, 3, T);
  return st;
}

int hlbm_get_populations(hlbm_handle h, int box, double* host_f) {
  if (!h) return HLBM_ERR_ARG;
  if (box < 0 || box >= (int)h->boxes.size() || !host_f) return fail(h, HLBM_ERR_ARG, "bad box or NULL array");
  const BoxDesc& bd = h->boxes[box];
  const long long N = (long long)bd.nx * bd.ny * bd.nz;
  const LbmArgs la = lbm_args(h, 0);
  const int parity = (int)(h->steps & 1);
  std::vector<float> st((size_t)Q * h->L.stage_cells);
  for (long long c0 = 0; c0 < N; c0 += h->L.stage_cells) {
    const long long n = (N - c0 < h->L.stage_cells) ? N - c0 : h->L.stage_cells;
    CK(launch_gather(la, h->prm.precision, parity, box, c0, n, h->stage, h->stream));
    CK(cudaMemcpyAsync(st.data(), h->stage, sizeof(float) * Q * n, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < Q; ++i) {
      const double w = wq(i);
      for (long long k = 0; k < n; ++k) host_f[(size_t)i * N + c0 + k] = w + (double)st[(size_t)i * n + k];
    }
  }
  return HLBM_OK;
}

int hlbm_set_populations(hlbm_handle h, int box, const double* host_f) {
  if (!h) return HLBM_ERR_ARG;
  if (box < 0 || box >= (int)h->boxes.size() || !host_f) return fail(h, HLBM_ERR_ARG, "bad box or NULL array");
  const BoxDesc& bd = h->boxes[box];
  const long long N = (long long)bd.nx * bd.ny * bd.nz;
  const LbmArgs la = lbm_args(h, 0);
  const int parity = (int)(h->steps & 1);
  std::vector<float> st((size_t)Q * h->L.stage_cells);
  for (long long c0 = 0; c0 < N; c0 += h->L.stage_cells) {
    const long long n = (N - c0 < h->L.stage_cells) ? N - c0 : h->L.stage_cells;
    for (int i = 0; i < Q; ++i) {
      const double w = wq(i);
      for (long long k = 0; k < n; ++k) st[(size_t)i * n + k] = (float)(host_f[(size_t)i * N + c0 + k] - w);
    }
    CK(cudaMemcpyAsync(h->stage, st.data(), sizeof(float) * Q * n, cudaMemcpyHostToDevice, h->stream));
    CK(launch_scatter(la, h->prm.precision, parity, box, c0, n, h->stage, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  h->moments_valid = false;
  return HLBM_OK;
}

int hlbm_fluid_momentum(hlbm_handle h, int box, double out[4]) {
  if (!h) return HLBM_ERR_ARG;
  if (box < 0 || box >= (int)h->boxes.size() || !out) return fail(h, HLBM_ERR_ARG, "bad box or NULL array");
  const BoxDesc& bd = h->boxes[box];
  const long long N = (long long)bd.nx * bd.ny * bd.nz;
  // partial sums in the staging area (Q * stage_cells floats), four doubles per block
  const long long room = (long long)Q * h->L.stage_cells / 8;
  long long blocks = std::min<long long>(std::max(2 * h->nsm, 1), (N + 255) / 256);
  blocks = std::max<long long>(1, std::min(blocks, room));
  double* part = reinterpret_cast<double*>(h->stage);
  CK(launch_fluid_moments(lbm_args(h, 0), h->prm.precision, (int)(h->steps & 1), box, (int)blocks, part, h->stream));
  std::vector<double> hp(4 * (size_t)blocks);
  CK(cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int k = 0; k < 4; ++k) out[k] = 0.0;
  for (long long b = 0; b < blocks; ++b)
    for (int k = 0; k < 4; ++k) out[k] += hp[4 * b + k];
  return HLBM_OK;
}

int hlbm_set_launch(hlbm_handle h, int tile_y, int tile_z, int cells_x) {
  if (!h) return HLBM_ERR_ARG;
  auto ok = [](int v) { return v == 1 || v == 2 || v == 4 || v == 8; };
  if (!ok(tile_y) || !ok(tile_z)) return fail(h, HLBM_ERR_ARG, "tile_y and tile_z must be 1, 2, 4 or 8");
  if (cells_x != 1 && cells_x != 2) return fail(h, HLBM_ERR_ARG, "cells_x must be 1 or 2");
  if (cells_x == 2 && !h->pair_ok) return fail(h, HLBM_ERR_ARG, "cells_x = 2 is not available");
  if (tile_y != h->sub_y || tile_z != h->sub_z || cells_x != h->cells_x) {
    h->sub_y = tile_y;
    h->sub_z = tile_z;
    h->cells_x = cells_x;
    drop_graphs(h);
  }
  return HLBM_OK;
}

int hlbm_set_fluid_force(hlbm_handle h, const double f[3]) {
  if (!h || !f) return HLBM_ERR_ARG;
  for (int j = 0; j < 3; ++j)
    if (!std::isfinite(f[j])) return fail(h, HLBM_ERR_ARG, "non-finite fluid force");
  if (f[0] != h->prm.fluid_force[0] || f[1] != h->prm.fluid_force[1] || f[2] != h->prm.fluid_force[2]) {
    CK(cudaStreamSynchronize(h->stream));
    for (int j = 0; j < 3; ++j) h->prm.fluid_force[j] = f[j];
    drop_graphs(h);  // the captured steps hold the force by value
  }
  return HLBM_OK;
}

int hlbm_set_contact(hlbm_handle h, double k, double zeta) {
  if (!h) return HLBM_ERR_ARG;
  if (!(k >= 0.0) || !std::isfinite(k) || !(zeta > 0.0) || !std::isfinite(zeta))
    return fail(h, HLBM_ERR_ARG, "contact stiffness must be finite and >= 0, its range finite and > 0");
  if (k != h->contact_k || zeta != h->contact_zeta) {
    CK(cudaStreamSynchronize(h->stream));
    h->contact_k = k;
    h->contact_zeta = zeta;
    drop_graphs(h);  // the captured steps hold the parameters by value
  }
  return HLBM_OK;
}

int hlbm_set_mea_mode(hlbm_handle h, int mode) {
  if (!h) return HLBM_ERR_ARG;
  if (mode != HLBM_MEA_KERNEL && mode != HLBM_MEA_MOMENTS) return fail(h, HLBM_ERR_ARG, "unknown momentum-exchange mode");
  if (mode == HLBM_MEA_MOMENTS && !h->ilist_idx) return fail(h, HLBM_ERR_STATE, "no particle capacity");
  if (mode != h->mea_mode) {
    CK(cudaStreamSynchronize(h->stream));
    h->mea_mode = mode;
    h->moments_valid = false;
    drop_graphs(h);
  }
  return HLBM_OK;
}

int hlbm_get_mea_mode(hlbm_handle h) { return h ? h->mea_mode : HLBM_ERR_ARG; }

int hlbm_get_launch(hlbm_handle h, int* tile_y, int* tile_z, int* cells_x) {
  if (!h) return HLBM_ERR_ARG;
  if (tile_y) *tile_y = h->sub_y;
  if (tile_z) *tile_z = h->sub_z;
  if (cells_x) *cells_x = h->cells_x;
  return HLBM_OK;
}

}  // extern "C"

namespace {
// choices of hlbm_autotune per (device, boxes, precision, particle count),
// kept for the life of the process
struct TuneChoice { int ty, tz, cx, mode; float ms; };
std::mutex g_tune_mutex;
std::map<std::string, TuneChoice> g_tune_cache;

std::string tune_key(const hlbm_ctx* h) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  std::string name = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? prop.name : "?";
  std::string k = name + "|" + std::to_string(h->nsm) + "|p" + std::to_string(h->prm.precision) + "|n" +
                  std::to_string(h->np) + "|g" + std::to_string(h->grids.size()) + "|c" +
                  std::to_string(h->contact_k > 0.0);
  for (const BoxDesc& b : h->boxes)
    k += "|" + std::to_string(b.nx) + "x" + std::to_string(b.ny) + "x" + std::to_string(b.nz) + "b" +
         std::to_string(b.bc);
  return k;
}
}  // namespace

extern "C" {

int hlbm_autotune(hlbm_handle h, int nsteps, int* tile_y, int* tile_z, int* cells_x, float* ms_per_step) {
  if (!h) return HLBM_ERR_ARG;
  if (nsteps < 1) return fail(h, HLBM_ERR_ARG, "nsteps < 1");
  if (h->split) return fail(h, HLBM_ERR_STATE, "a split step is open");
  const std::string key = tune_key(h);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      const TuneChoice c = it->second;
      int r = hlbm_set_mea_mode(h, c.mode);
      if (r == HLBM_OK) r = hlbm_set_launch(h, c.ty, c.tz, c.cx);
      if (r != HLBM_OK) return r;
      if (tile_y) *tile_y = c.ty;
      if (tile_z) *tile_z = c.tz;
      if (cells_x) *cells_x = c.cx;
      if (ms_per_step) *ms_per_step = c.ms;
      return HLBM_OK;
    }
  }
  // the timed steps run on the handle itself; its whole device state (one
  // buffer) and the host-side step state are copied aside first and put
  // back afterwards, so tuning leaves the run where it was
  CK(cudaStreamSynchronize(h->stream));
  char* backup = nullptr;
  CK(cudaMalloc((void**)&backup, h->L.total));
  {
    const cudaError_t e = cudaMemcpyAsync(backup, h->buf, h->L.total, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) {
      cudaFree(backup);
      return fail(h, HLBM_ERR_CUDA, std::string("autotune backup: ") + cudaGetErrorString(e));
    }
  }
  const long long steps0 = h->steps;
  const bool moments0 = h->moments_valid, hst0 = h->hst_valid;
  const long long hst_steps0 = h->hst_steps;
  auto restore = [&]() -> int {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->buf, backup, h->L.total, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(backup);
    h->steps = steps0;
    h->moments_valid = moments0;
    h->hst_valid = hst0;
    h->hst_steps = hst_steps0;
    if (e != cudaSuccess) return fail(h, HLBM_ERR_CUDA, std::string("autotune restore: ") + cudaGetErrorString(e));
    return HLBM_OK;
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    restore();
    return fail(h, HLBM_ERR_CUDA, "autotune: cudaEventCreate failed");
  }
  struct Cand { int ty, tz, cx, mode; float ms; };
  std::vector<Cand> cand;
  const int vals[4] = {1, 2, 4, 8};
  const int nmodes = h->np > 0 ? 2 : 1;
  const int nkinds = h->pair_ok ? 2 : 1;
  for (int im = 0; im < nkinds * nmodes * 16; ++im) {
    const int kind = im / (nmodes * 16), mode = (im / 16) % nmodes, iy = (im / 4) % 4, iz = im % 4;
    if (kind == 1 && vals[iy] == 1) continue;  // 16-thread blocks leave half of each warp idle
    cand.push_back({vals[iy], vals[iz], kind + 1, mode, 0.f});
  }
  int rc = HLBM_OK;
  // steps per timing: about 20 ms, between nsteps and 4 nsteps (tuning
  // advances the state; long runs would let particles settle and overlap)
  int n = nsteps;
  auto time_one = [&](Cand& c) -> int {
    int r = hlbm_set_mea_mode(h, c.mode);
    if (r == HLBM_OK) r = hlbm_set_launch(h, c.ty, c.tz, c.cx);
    if (r == HLBM_OK) r = hlbm_step(h, 2);  // warm-up and graph build
    if (r != HLBM_OK) return r;
    cudaEventRecord(e0, h->stream);
    r = hlbm_step(h, n);
    cudaEventRecord(e1, h->stream);
    if (r != HLBM_OK) return r;
    if (cudaEventSynchronize(e1) != cudaSuccess) return fail(h, HLBM_ERR_CUDA, "autotune timing failed");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    c.ms = ms / n;
    return HLBM_OK;
  };
  for (size_t k = 0; k < cand.size() && rc == HLBM_OK; ++k) {
    rc = time_one(cand[k]);
    if (rc == HLBM_OK && k == 0) {
      n = std::min(4 * nsteps, std::max(nsteps, (int)std::ceil(20.0 / std::max(cand[0].ms, 1e-3f))));
      rc = time_one(cand[0]);
    }
  }
  if (rc == HLBM_OK) {
    // time the three fastest once more and keep the faster of the two timings
    std::vector<Cand> top = cand;
    std::sort(top.begin(), top.end(), [](const Cand& x, const Cand& y) { return x.ms < y.ms; });
    top.resize(std::min<size_t>(3, top.size()));
    for (auto& c : top) {
      const float first = c.ms;
      if ((rc = time_one(c)) != HLBM_OK) break;
      c.ms = std::min(first, c.ms);
    }
    cand = top;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == HLBM_OK) rc = read_status(h);
  const int rrc = restore();
  if (rc != HLBM_OK) return rc;
  if (rrc != HLBM_OK) return rrc;
  const Cand best = *std::min_element(cand.begin(), cand.end(),
                                      [](const Cand& x, const Cand& y) { return x.ms < y.ms; });
  rc = hlbm_set_mea_mode(h, best.mode);
  if (rc == HLBM_OK) rc = hlbm_set_launch(h, best.ty, best.tz, best.cx);
  if (tile_y) *tile_y = best.ty;
  if (tile_z) *tile_z = best.tz;
  if (cells_x) *cells_x = best.cx;
  if (ms_per_step) *ms_per_step = best.ms;
  if (rc != HLBM_OK) return rc;
  // the restored state is the one before tuning: its recorded interior
  // cells are valid for the mode in use then
  h->moments_valid = moments0 && best.mode == HLBM_MEA_MOMENTS && h->mea_mode == HLBM_MEA_MOMENTS;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = TuneChoice{best.ty, best.tz, best.cx, best.mode, best.ms};
  }
  return HLBM_OK;
}

int hlbm_kernel_times(hlbm_handle h, int nsteps, float ms[3]) {
  if (!h || !ms) return HLBM_ERR_ARG;
  if (nsteps < 1) return fail(h, HLBM_ERR_ARG, "nsteps < 1");
  cudaEvent_t ev[4];
  for (int k = 0; k < 4; ++k) CK(cudaEventCreate(&ev[k]));
  double acc[3] = {0, 0, 0};
  int rc = HLBM_OK;
  for (int s = 0; s < nsteps; ++s) {
    const int parity = (int)(h->steps & 1);
    PartArgs pa = part_args(h, parity);
    const bool fused = h->moments_valid && h->np > 0;
    pa.from_acc = fused ? 1 : 0;
    cudaEventRecord(ev[0], h->stream);
    if (h->np > 0 && !fused) launch_mea(pa, h->prm.precision, parity, h->stream);
    if (h->np > 0 && fused) launch_mea_moments(lbm_args(h, parity), h->prm.precision, parity, h->walls, h->nsm, h->stream);
    cudaEventRecord(ev[1], h->stream);
    if (h->np > 0) launch_contact(pa, h->stream);
    if (h->np > 0) launch_update(pa, h->stream);
    cudaEventRecord(ev[2], h->stream);
    launch_collide(lbm_args(h, parity), h->prm.precision, parity, h->walls, h->np > 0, h->stream);
    cudaEventRecord(ev[3], h->stream);
    const cudaError_t e = cudaEventSynchronize(ev[3]);
    if (e != cudaSuccess) { rc = fail(h, HLBM_ERR_CUDA, std::string("kernel timing: ") + cudaGetErrorString(e)); break; }
    for (int k = 0; k < 3; ++k) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      acc[k] += t;
    }
    h->steps += 1;
    h->moments_valid = h->mea_mode == HLBM_MEA_MOMENTS;
  }
  for (int k = 0; k < 4; ++k) cudaEventDestroy(ev[k]);
  if (rc != HLBM_OK) return rc;
  for (int k = 0; k < 3; ++k) ms[k] = (float)(acc[k] / nsteps);
  return read_status(h);
}

int hlbm_interior_cells(hlbm_handle h, long long* n) {
  if (!h || !n) return HLBM_ERR_ARG;
  *n = 0;
  if (h->np == 0) return HLBM_OK;
  if (h->mea_mode != HLBM_MEA_MOMENTS || !h->moments_valid || !h->ilist_idx)
    return fail(h, HLBM_ERR_STATE, "interior cells are counted by a collision in the moments mode");
  int cnt[ILIST_STRIPES];
  CK(cudaMemcpyAsync(cnt, h->ilist_count, sizeof(cnt), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  long long t = 0;
  for (int k = 0; k < ILIST_STRIPES; ++k) t += std::min((long long)cnt[k], h->L.ilist_cap);
  *n = t;
  return read_status(h);
}

}  // extern "C"
// ---------------------------------------------------------------- snapshots
// Layout (host byte order, no padding): the header below; per box nx, ny,
// nz, bc (int64); per distance grid nx, ny, nz (int64), the spacing and the
// samples (FP32); shape and box id per particle (int32); the particle
// table, PF_COUNT rows of np doubles; the interior-cell list when the next
// step takes its momentum exchange from it (ILIST_STRIPES int32 counts,
// then per stripe its int2 entries and its float4 moments); the populations
// as stored (the handle's own block layout and precision).
namespace {

constexpr char CK_MAGIC[8] = {'H', 'L', 'B', 'M', 'C', 'K', 'P', '3'};

struct CkHeader {
  char magic[8];
  int64_t nboxes, precision, fp16_scale_log2, np, pf_count, steps, mea_mode, has_list, pop_bytes, ngrids;
  double tau, eps, gravity[3], fluid_force[3], contact_k, contact_zeta;
};

size_t pop_bytes(const hlbm_ctx* h) {
  return (size_t)QVB * h->L.nblocks * (h->prm.precision == HLBM_FP32 ? 4 : 2);
}

// the snapshot's size, with the interior-list counts it will hold (read
// from the device when the next step uses the list)
int snapshot_plan(hlbm_ctx* h, size_t* total, bool* has_list, int cnt[ILIST_STRIPES]) {
  const int st = read_status(h);
  if (st != HLBM_OK) return st;
  *has_list = h->np > 0 && h->moments_valid && h->mea_mode == HLBM_MEA_MOMENTS && h->ilist_idx;
  size_t t = sizeof(CkHeader) + sizeof(int64_t) * 4 * h->boxes.size() + sizeof(int32_t) * 2 * (size_t)h->np +
             sizeof(double) * PF_COUNT * (size_t)h->np;
  for (const auto& g : h->grids) t += sizeof(int64_t) * 3 + sizeof(double) + sizeof(float) * g.v.size();
  if (*has_list) {
    CK(cudaMemcpyAsync(cnt, h->ilist_count, sizeof(int) * ILIST_STRIPES, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    t += sizeof(int32_t) * ILIST_STRIPES;
    for (int k = 0; k < ILIST_STRIPES; ++k) {
      if (cnt[k] < 0 || cnt[k] > h->L.ilist_cap) return fail(h, HLBM_ERR_STATE, "interior-cell list count out of range");
      t += (sizeof(int2) + sizeof(float4)) * (size_t)cnt[k];
    }
  }
  *total = t + pop_bytes(h);
  return HLBM_OK;
}

}  // namespace

extern "C" {

int hlbm_checkpoint_bytes(hlbm_handle h, size_t* bytes) {
  if (!h || !bytes) return HLBM_ERR_ARG;
  *bytes = 0;
  bool has_list = false;
  int cnt[ILIST_STRIPES];
  return snapshot_plan(h, bytes, &has_list, cnt);
}

int hlbm_save(hlbm_handle h, void* buf, size_t bytes) {
  if (!h) return HLBM_ERR_ARG;
  if (!buf) return fail(h, HLBM_ERR_ARG, "NULL buffer");
  size_t total = 0;
  bool has_list = false;
  int cnt[ILIST_STRIPES];
  int rc = snapshot_plan(h, &total, &has_list, cnt);
  if (rc != HLBM_OK) return rc;
  if (bytes < total) return fail(h, HLBM_ERR_ARG, "buffer smaller than hlbm_checkpoint_bytes");
  char* o = (char*)buf;
  auto put = [&](const void* src, size_t n) { std::memcpy(o, src, n); o += n; };
  CkHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, CK_MAGIC, 8);
  hd.nboxes = (int64_t)h->boxes.size();
  hd.precision = h->prm.precision;
  hd.fp16_scale_log2 = h->prm.fp16_scale_log2;
  hd.np = h->np;
  hd.pf_count = PF_COUNT;
  hd.steps = h->steps;
  hd.mea_mode = h->mea_mode;
  hd.has_list = has_list ? 1 : 0;
  hd.pop_bytes = (int64_t)pop_bytes(h);
  hd.tau = h->prm.tau;
  hd.eps = h->prm.eps;
  hd.contact_k = h->contact_k;
  hd.contact_zeta = h->contact_zeta;
  hd.ngrids = (int64_t)h->grids.size();
  for (int j = 0; j < 3; ++j) {
    hd.gravity[j] = h->prm.gravity[j];
    hd.fluid_force[j] = h->prm.fluid_force[j];
  }
  put(&hd, sizeof(hd));
  for (const BoxDesc& b : h->boxes) {
    const int64_t d[4] = {b.nx, b.ny, b.nz, b.bc};
    put(d, sizeof(d));
  }
  for (const auto& g : h->grids) {
    const int64_t d[3] = {g.n[0], g.n[1], g.n[2]};
    put(d, sizeof(d));
    put(&g.h, sizeof(double));
    put(g.v.data(), sizeof(float) * g.v.size());
  }
  const size_t np = (size_t)h->np;
  for (size_t k = 0; k < np; ++k) { const int32_t v = h->h_shape[k]; put(&v, sizeof(v)); }
  for (size_t k = 0; k < np; ++k) { const int32_t v = h->h_box[k]; put(&v, sizeof(v)); }
  if (np > 0) {
    CK(cudaMemcpy2DAsync(o, sizeof(double) * np, h->P, sizeof(double) * h->L.cap, sizeof(double) * np, PF_COUNT,
                         cudaMemcpyDeviceToHost, h->stream));
    o += sizeof(double) * PF_COUNT * np;
  }
  if (has_list) {
    put(cnt, sizeof(int32_t) * ILIST_STRIPES);
    for (int k = 0; k < ILIST_STRIPES; ++k) {
      if (cnt[k] == 0) continue;
      const size_t k0 = (size_t)k * h->L.ilist_cap;
      CK(cudaMemcpyAsync(o, h->ilist_idx + k0, sizeof(int2) * cnt[k], cudaMemcpyDeviceToHost, h->stream));
      o += sizeof(int2) * cnt[k];
      CK(cudaMemcpyAsync(o, h->ilist_mom + k0, sizeof(float4) * cnt[k], cudaMemcpyDeviceToHost, h->stream));
      o += sizeof(float4) * cnt[k];
    }
  }
  CK(cudaMemcpyAsync(o, h->f, pop_bytes(h), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return HLBM_OK;
}

int hlbm_load(hlbm_handle h, const void* buf, size_t bytes) {
  if (!h) return HLBM_ERR_ARG;
  if (!buf) return fail(h, HLBM_ERR_ARG, "NULL buffer");
  if (h->steps != 0 || h->np != 0 || !h->grids.empty())
    return fail(h, HLBM_ERR_STATE,
                "a snapshot loads into a new handle (no step taken, no particles or grids added)");
  const char* i = (const char*)buf;
  const char* end = i + bytes;
  auto get = [&](void* dst, size_t n) -> bool {
    if ((size_t)(end - i) < n) return false;
    std::memcpy(dst, i, n);
    i += n;
    return true;
  };
  CkHeader hd;
  if (!get(&hd, sizeof(hd)) || std::memcmp(hd.magic, CK_MAGIC, 8) != 0)
    return fail(h, HLBM_ERR_ARG, "not a snapshot of this library");
  if (hd.pf_count != PF_COUNT) return fail(h, HLBM_ERR_ARG, "snapshot of another particle table layout");
  if (hd.nboxes != (int64_t)h->boxes.size() || hd.precision != h->prm.precision ||
      hd.fp16_scale_log2 != h->prm.fp16_scale_log2 || hd.pop_bytes != (int64_t)pop_bytes(h))
    return fail(h, HLBM_ERR_ARG, "snapshot of other boxes or another storage precision");
  bool same = hd.tau == h->prm.tau && hd.eps == h->prm.eps;
  for (int j = 0; j < 3; ++j) same = same && hd.gravity[j] == h->prm.gravity[j];
  if (!same) return fail(h, HLBM_ERR_ARG, "snapshot taken with another tau, eps or gravity");
  if (hd.np < 0 || hd.np > h->L.cap) return fail(h, HLBM_ERR_ARG, "snapshot holds more particles than max_particles");
  bool finite_force = true;
  for (int j = 0; j < 3; ++j) finite_force = finite_force && std::isfinite(hd.fluid_force[j]);
  if (hd.steps < 0 || hd.ngrids < 0 || hd.ngrids > MAX_GRIDS ||
      (hd.mea_mode != HLBM_MEA_KERNEL && hd.mea_mode != HLBM_MEA_MOMENTS) || !finite_force ||
      !(hd.contact_k >= 0.0) || !std::isfinite(hd.contact_k) || !(hd.contact_zeta > 0.0) ||
      !std::isfinite(hd.contact_zeta))
    return fail(h, HLBM_ERR_ARG, "corrupt snapshot header");
  for (size_t b = 0; b < h->boxes.size(); ++b) {
    int64_t d[4];
    if (!get(d, sizeof(d))) return fail(h, HLBM_ERR_ARG, "truncated snapshot");
    const BoxDesc& B = h->boxes[b];
    if (d[0] != B.nx || d[1] != B.ny || d[2] != B.nz || d[3] != B.bc)
      return fail(h, HLBM_ERR_ARG, "snapshot of other boxes or another storage precision");
  }
  // the distance grids, registered again (checks and derived properties)
  for (int64_t k = 0; k < hd.ngrids; ++k) {
    int64_t d[3];
    double sp;
    if (!get(d, sizeof(d)) || !get(&sp, sizeof(sp))) return fail(h, HLBM_ERR_ARG, "truncated snapshot");
    if (d[0] < 2 || d[1] < 2 || d[2] < 2 || d[0] > (1 << 20) || d[1] > (1 << 20) || d[2] > (1 << 20))
      return fail(h, HLBM_ERR_ARG, "corrupt grid in snapshot");
    const size_t nv = (size_t)(d[0] * d[1] * d[2]);
    if ((size_t)(end - i) < sizeof(float) * nv) return fail(h, HLBM_ERR_ARG, "truncated snapshot");
    std::vector<float> v(nv);
    std::memcpy(v.data(), i, sizeof(float) * nv);
    i += sizeof(float) * nv;
    int id = -1;
    const int rc = hlbm_add_grid(h, (int)d[0], (int)d[1], (int)d[2], sp, v.data(), &id);
    if (rc != HLBM_OK) return rc;
  }
  const int n = (int)hd.np;
  std::vector<int32_t> shp(n), bx(n);
  std::vector<double> tab((size_t)PF_COUNT * n);
  if (!get(shp.data(), sizeof(int32_t) * n) || !get(bx.data(), sizeof(int32_t) * n) ||
      !get(tab.data(), sizeof(double) * tab.size()))
    return fail(h, HLBM_ERR_ARG, "truncated snapshot");
  int cnt[ILIST_STRIPES] = {0};
  std::vector<const char*> lst(ILIST_STRIPES, nullptr);
  if (hd.has_list) {
    if (!get(cnt, sizeof(cnt))) return fail(h, HLBM_ERR_ARG, "truncated snapshot");
    for (int k = 0; k < ILIST_STRIPES; ++k) {
      if (cnt[k] < 0 || cnt[k] > h->L.ilist_cap || !h->ilist_idx)
        return fail(h, HLBM_ERR_ARG, "snapshot's interior-cell list does not fit this handle");
      const size_t nb = (sizeof(int2) + sizeof(float4)) * (size_t)cnt[k];
      if ((size_t)(end - i) < nb) return fail(h, HLBM_ERR_ARG, "truncated snapshot");
      lst[k] = i;
      i += nb;
    }
  }
  if ((size_t)(end - i) < pop_bytes(h)) return fail(h, HLBM_ERR_ARG, "truncated snapshot");
  const char* pops = i;
  // the particles through the regular path (validation, derived tables),
  // then the table exactly as saved
  if (n > 0) {
    std::vector<double> a(3 * (size_t)n), X(3 * (size_t)n), U(3 * (size_t)n), W(3 * (size_t)n),
        q(4 * (size_t)n), rho(n);
    auto row = [&](int fld, int k) { return tab[(size_t)fld * n + k]; };
    for (int k = 0; k < n; ++k) {
      for (int j = 0; j < 3; ++j) {
        // a grid particle names its grid (kept in PF_IA), the others their sizes
        a[3 * k + j] = shp[k] == HLBM_GRID ? row(PF_IA + j, k) : row(PF_A + j, k);
        X[3 * k + j] = row(PF_X + j, k);
        U[3 * k + j] = row(PF_U + j, k);
        W[3 * k + j] = row(PF_W + j, k);
      }
      for (int j = 0; j < 4; ++j) q[4 * k + j] = row(PF_Q + j, k);
      rho[k] = row(PF_RHO, k);
    }
    const int rc = hlbm_add_particles(h, n, bx.data(), shp.data(), a.data(), X.data(), U.data(), W.data(),
                                      q.data(), rho.data());
    if (rc != HLBM_OK) return rc;
    CK(cudaMemcpy2DAsync(h->P, sizeof(double) * h->L.cap, tab.data(), sizeof(double) * n, sizeof(double) * n,
                         PF_COUNT, cudaMemcpyHostToDevice, h->stream));
    CK(launch_records(part_args(h, 0), h->stream));
  }
  CK(cudaMemsetAsync(h->ilist_count, 0, sizeof(int) * ILIST_STRIPES, h->stream));
  if (hd.has_list) {
    CK(cudaMemcpyAsync(h->ilist_count, cnt, sizeof(cnt), cudaMemcpyHostToDevice, h->stream));
    for (int k = 0; k < ILIST_STRIPES; ++k) {
      if (cnt[k] == 0) continue;
      const size_t k0 = (size_t)k * h->L.ilist_cap;
      CK(cudaMemcpyAsync(h->ilist_idx + k0, lst[k], sizeof(int2) * cnt[k], cudaMemcpyHostToDevice, h->stream));
      CK(cudaMemcpyAsync(h->ilist_mom + k0, lst[k] + sizeof(int2) * cnt[k], sizeof(float4) * cnt[k],
                         cudaMemcpyHostToDevice, h->stream));
    }
  }
  for (int k = 0; k < 2; ++k) CK(cudaMemsetAsync(h->cnt[k], 0, sizeof(int) * (size_t)h->L.ntiles, h->stream));
  CK(cudaMemcpyAsync(h->f, pops, pop_bytes(h), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int j = 0; j < 3; ++j) h->prm.fluid_force[j] = hd.fluid_force[j];
  h->contact_k = hd.contact_k;
  h->contact_zeta = hd.contact_zeta;
  // the saver's momentum-exchange mode, where this handle can hold its list
  if (hd.mea_mode == HLBM_MEA_KERNEL || h->ilist_idx) h->mea_mode = (int)hd.mea_mode;
  h->steps = hd.steps;
  h->moments_valid = hd.has_list != 0 && h->mea_mode == HLBM_MEA_MOMENTS;
  drop_graphs(h);
  return read_status(h);
}

}  // extern "C"
