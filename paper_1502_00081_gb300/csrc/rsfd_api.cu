// C ABI entry points, the handle, and the host-side column scheduler of the shifted COCG solve.
//
// The scheduler keeps W right-hand sides ("slots") in flight.  Each device iteration is one
// fused pass (seed SpMV + seed update + dots + FP64 scalar step) and one shift update over all
// slots; a chunk of iterations is captured once in a CUDA graph and replayed.  Between replays
// the host reads the slot states (a few hundred bytes), records the columns that finished and
// loads new columns into the freed slots, so slots never wait for the slowest column of a block.

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <exception>
#include <new>
#include <map>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "rsfd_internal.cuh"

namespace rsfd {

static thread_local std::string g_last_error = "no error";

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Handle {
  int nx = 0, ny = 0, nz = 0;
  int nxp = 0;          // padded row length of the internal vectors
  long long N = 0;
  double h = 0;
  int fd_order = 2, R = 1, nface = 1, nb = 0;
  int prec = RSFD_FP64;
  cudaStream_t user_stream = nullptr;
  cudaStream_t work = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int device = 0;
  std::vector<int64_t> brow;
  std::vector<int> track;      // tracked interior planes (rows recorded after b)
  int nr = 0;                  // recorded rows: nb + track.size() * Nx * Ny
  void* dV = nullptr;
  void* dVs = nullptr;         // double-float handles: s V for the block-floating-point split pass
  double uscale = 1.0;         // s = 24 h^2 (4th order) or 2 h^2 (2nd order)
  int64_t* dbrow = nullptr;
  // nonlocal projectors: atom-major and point-major CSR of the same entries on the device
  int n_atoms = 0, n_supp = 0;
  long long nnz = 0;
  int *d_aptr = nullptr, *d_tptr = nullptr, *d_tatom = nullptr;
  long long *d_aidx = nullptr, *d_tpidx = nullptr;
  void *d_aval = nullptr, *d_tval = nullptr;
  double* d_aE = nullptr;
  double* d_pmax = nullptr;    // per atom: the largest |projector value| (the block-floating-point bound)
  int proj_overlap = 0;        // largest number of atoms sharing a support point
  uint64_t in_hash = 0;        // hash of the operator's inputs (grid, h, order, faces, precision, V, projectors)
  DevBuf sweep;                // one column block of G0_bb for rsfd_shifted_cocg_sweep
  rsfd_solve_opts opts;
  rsfd_stats stats;
  std::string err = "no error";
  // solver workspace
  DevBuf rbuf, xbuf, pbuf, rhist, coef, eflag, slots, shifts, partials, tickets, Z, init_list, init_grid, counters;
  DevBuf pw, pcorr, pdots, ptickets;   // projector term of the solve
  DevBuf cw, ce;                       // collapse weights and factors of the shift update
  CUtensorMap tmR, tmV, tmVs;
  // dyson / transmission workspace
  DevBuf dy[8];
};

static bool is_split(int kind) { return kind == RSFD_PASS_SPLIT || kind == RSFD_PASS_SPLIT_BFP; }

rsfd_status fail(Handle* h, rsfd_status s, const std::string& msg) {
  if (h) h->err = msg;
  g_last_error = msg;
  return s;
}

#define RSFD_CK(h, call)                                                                              \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) {                                                                          \
      return fail((h), RSFD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));            \
    }                                                                                                 \
  } while (0)

static rsfd_status ensure(Handle* h, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return RSFD_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, RSFD_ERR_ALLOC, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
  }
  b.bytes = bytes;
  return RSFD_OK;
}

rsfd_status handle_ensure(Handle* h, int idx, size_t bytes, void** out) {
  rsfd_status s = ensure(h, h->dy[idx], bytes);
  if (s != RSFD_OK) return s;
  *out = h->dy[idx].p;
  return RSFD_OK;
}

cudaStream_t handle_stream(Handle* h) { return h->work; }
int handle_prec(Handle* h) { return h->prec; }
int handle_nb(Handle* h) { return h->nb; }
int handle_nx(Handle* h) { return h->nx; }
int handle_ny(Handle* h) { return h->ny; }
int handle_fd_order(Handle* h) { return h->fd_order; }
double handle_h(Handle* h) { return h->h; }
int handle_dyson_kind(Handle* h) {
  if (h->opts.dyson_kind != RSFD_DYSON_AUTO) return h->opts.dyson_kind;
  return h->prec == RSFD_FP64 ? RSFD_DYSON_FP64 : RSFD_DYSON_TC;
}
int handle_dyson_cols(Handle* h) { return h->opts.dyson_cols; }
int handle_dyson_refine(Handle* h) {
  if (h->opts.dyson_refine > 0) return h->opts.dyson_refine;
  return h->prec == RSFD_FP64 ? 2 : 1;
}
rsfd_status handle_fail(Handle* h, rsfd_status s, const std::string& m) { return fail(h, s, m); }

// order the internal stream after the caller's stream
rsfd_status handle_begin(Handle* h) {
  RSFD_CK(h, cudaSetDevice(h->device));
  RSFD_CK(h, cudaEventRecord(h->ev_in, h->user_stream));
  RSFD_CK(h, cudaStreamWaitEvent(h->work, h->ev_in, 0));
  return RSFD_OK;
}
// order the caller's stream after the internal stream
rsfd_status handle_end(Handle* h) {
  RSFD_CK(h, cudaEventRecord(h->ev_out, h->work));
  RSFD_CK(h, cudaStreamWaitEvent(h->user_stream, h->ev_out, 0));
  return RSFD_OK;
}

static void free_all(Handle* h) {
  DevBuf* bufs[] = {&h->rbuf,  &h->xbuf,      &h->pbuf,      &h->rhist,    &h->coef,
                    &h->eflag, &h->slots,     &h->shifts,    &h->partials, &h->tickets,
                    &h->Z,     &h->init_list, &h->init_grid, &h->counters, &h->pw,
                    &h->pcorr, &h->pdots,     &h->ptickets,  &h->sweep, &h->cw, &h->ce};
  for (DevBuf* b : bufs) {
    if (b->p) cudaFree(b->p);
    b->p = nullptr;
    b->bytes = 0;
  }
  for (auto& b : h->dy) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  if (h->dV) cudaFree(h->dV);
  if (h->dVs) cudaFree(h->dVs);
  if (h->dbrow) cudaFree(h->dbrow);
  void* pj[] = {h->d_aptr, h->d_tptr, h->d_tatom, h->d_aidx, h->d_tpidx, h->d_aval, h->d_tval, h->d_aE, h->d_pmax};
  for (void* q : pj)
    if (q) cudaFree(q);
  h->d_aptr = h->d_tptr = h->d_tatom = nullptr;
  h->d_aidx = h->d_tpidx = nullptr;
  h->d_aval = h->d_tval = nullptr;
  h->d_aE = nullptr;
  h->d_pmax = nullptr;
  h->dV = nullptr;
  h->dVs = nullptr;
  h->dbrow = nullptr;
}

static StencilCoef stencil_coef(int fd_order, double hh) {
  // -1/2 d^2/dx^2 with central coefficients (1,-2,1)/h^2 or (-1/12,4/3,-5/2,4/3,-1/12)/h^2 per axis
  StencilCoef c;
  const double ih2 = 1.0 / (hh * hh);
  if (fd_order == 2) {
    c.hd = 3.0 * (-0.5 * -2.0) * ih2;
    c.hk[0] = -0.5 * 1.0 * ih2;
    c.hk[1] = 0.0;
  } else {
    c.hd = 3.0 * (-0.5 * -2.5) * ih2;
    c.hk[0] = -0.5 * (4.0 / 3.0) * ih2;
    c.hk[1] = -0.5 * (-1.0 / 12.0) * ih2;
  }
  c.hk[2] = 0.0;
  return c;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
  }
  return fn;
}

// TMA descriptors of the Krylov vectors [nvec W][Nz][Ny][Nxp] and of the potential [Nz][Ny][Nxp].
// Rows are padded to Nxp (a multiple of 4) so every stride is a multiple of 16 bytes; the x extent
// is the true Nx, so reads past the last column (and outside the grid) come back as zeros.
// Boxes: fused pass 40 x (tile_y + 4R) for both; stored-product pass 36 x (tile_y + 2R) for the
// vectors and the 32 x tile_y tile for the potential.
static rsfd_status make_maps(Handle* h, int W, int tile_y, int kind, int tile_x) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return fail(h, RSFD_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const bool f64 = h->prec == RSFD_FP64;
  const CUtensorMapDataType dt = f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const cuuint64_t es = f64 ? 8 : 4;
  const cuuint64_t mR = h->prec == RSFD_DF64 ? 4 : 2, mV = h->prec == RSFD_DF64 ? 2 : 1;
  const bool stored = kind == RSFD_PASS_STORED || is_split(kind);
  const cuuint64_t nvec = stored ? 5 : 3;
  const cuuint32_t EY = (cuuint32_t)(tile_y + (stored ? 2 : 4) * h->R);
  const cuuint32_t BX = (cuuint32_t)(stored ? passu_box_x(tile_x) : pass_box_x());
  const cuuint32_t VBX = (cuuint32_t)(stored ? tile_x : pass_box_x());
  const cuuint32_t VBY = stored ? (cuuint32_t)tile_y : EY;
  {
    cuuint64_t dims[4] = {mR * h->nx, (cuuint64_t)h->ny, (cuuint64_t)h->nz, nvec * W};
    cuuint64_t strides[3] = {mR * h->nxp * es, mR * h->nxp * es * h->ny, mR * h->nxp * es * h->ny * h->nz};
    cuuint32_t box[4] = {(cuuint32_t)(mR * BX), EY, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(&h->tmR, dt, 4, h->rbuf.p, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, RSFD_ERR_CUDA, "cuTensorMapEncodeTiled (vectors) failed: " + std::to_string((int)r));
  }
  {
    cuuint64_t dims[3] = {mV * h->nx, (cuuint64_t)h->ny, (cuuint64_t)h->nz};
    cuuint64_t strides[2] = {mV * h->nxp * es, mV * h->nxp * es * h->ny};
    cuuint32_t box[3] = {(cuuint32_t)(mV * VBX), VBY, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(&h->tmV, dt, 3, h->dV, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(h, RSFD_ERR_CUDA, "cuTensorMapEncodeTiled (potential) failed: " + std::to_string((int)r));
    if (h->dVs) {   // the scaled potential s V: same layout, box and element type
      r = enc(&h->tmVs, dt, 3, h->dVs, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS)
        return fail(h, RSFD_ERR_CUDA, "cuTensorMapEncodeTiled (scaled potential) failed: " + std::to_string((int)r));
    }
  }
  return RSFD_OK;
}

// the block-floating-point split pass serves double-float handles; the others run the plain split pass
static int resolve_kind(int prec, int opt) {
  if (opt == RSFD_PASS_SPLIT_BFP) return prec == RSFD_DF64 ? opt : RSFD_PASS_SPLIT;
  if (opt == RSFD_PASS_RECOMPUTE || opt == RSFD_PASS_STORED || opt == RSFD_PASS_SPLIT) return opt;
  return RSFD_PASS_STORED;
}

static size_t kind_smem(int prec, int R, int tile_y, int depth, int kind, int tile_x = 32) {
  if (is_split(kind)) return split_smem(prec, R, tile_y, depth);
  return kind == RSFD_PASS_STORED ? passu_smem(prec, R, tile_y, depth, tile_x) : pass_smem(prec, R, tile_y, depth);
}

static int resolve_rows(int opt) {
  if (opt == 1 || opt == 2 || opt == 4) return opt;
  return 1;
}

static bool tile_ok(int prec, int R, int tile_y, int kind, int rows, int budget = 0, int tile_x = 32) {
  if (tile_y < 1) return false;
  if (is_split(kind)) {
    // one row per thread, 32-wide tiles, at most 16 rows (512 threads)
    if (tile_x != 32 || rows != 1 || tile_y > 16) return false;
    return split_smem(prec, R, tile_y, 1) <= (size_t)(216 * 1024);
  }
  if (tile_x != 32) {
    // the 16-wide tile: one-row double-float stored pass with the default register budget only
    if (tile_x != 16 || kind != RSFD_PASS_STORED || prec != RSFD_DF64 || rows != 1 || budget != 0) return false;
    if (tile_y % 2 != 0) return false;
  }
  if (kind == RSFD_PASS_STORED) {
    if (tile_y % rows != 0) return false;
    const int b = (prec == RSFD_DF64 && rows == 1) ? budget : 0;
    if (passu_threads(rows, R, tile_y, tile_x) > passu_max_threads(rows, b)) return false;
  } else {
    if (pass_threads(R, tile_y) > pass_max_threads(prec)) return false;
  }
  if (tile_y + 4 * R > 256) return false;
  return kind_smem(prec, R, tile_y, 1, kind, tile_x) <= (size_t)(216 * 1024);
}

// Fused pass: the tile height that minimises the rows computed per column of tiles,
// (tile_y + 2R) * ceil(Ny / tile_y), among the heights the CTA size and shared memory allow (ties to
// the taller tile).  Stored-product pass: 8 rows (measured fastest on the 64 x 64 x 128 workload for
// both precisions: more CTAs per SM outweigh the larger frame), fewer on smaller grids.
static int default_tile_y(int prec, int R, int ny, int kind, int rows) {
  if (is_split(kind)) return std::max(1, std::min(8, ny));
  if (kind == RSFD_PASS_STORED) {
    const int ty = std::max(rows, std::min(8, (ny + rows - 1) / rows * rows));
    if (tile_ok(prec, R, ty, kind, rows)) return ty;
  }
  int best = 0;
  long long best_rows = 0;
  for (int ty = 4; ty <= 64; ty += 4) {
    if (!tile_ok(prec, R, ty, kind, rows)) continue;
    const long long rows = (long long)(ty + 2 * R) * ((ny + ty - 1) / ty);
    if (best == 0 || rows <= best_rows) {
      best = ty;
      best_rows = rows;
    }
    if (ty >= ny) break;
  }
  return best > 0 ? best : 4;
}

}  // namespace rsfd

using namespace rsfd;

struct rsfd_handle_s : public rsfd::Handle {};

// FNV-1a, 64 bit: identifies the inputs a checkpointed column block was computed from
static uint64_t fnv1a(uint64_t hv, const void* p, size_t n) {
  const unsigned char* b = (const unsigned char*)p;
  for (size_t i = 0; i < n; ++i) {
    hv ^= b[i];
    hv *= 1099511628211ull;
  }
  return hv;
}

extern "C" {

static rsfd_status rsfd_create_impl(rsfd_handle* out, const int32_t grid[3], double hh, int32_t fd_order, int32_t n_face,
                        const double* V_loc, const rsfd_projectors* proj, int32_t precision, void* stream) {
  if (!out) return fail(nullptr, RSFD_ERR_ARG, "rsfd_create: out is NULL");
  *out = nullptr;
  if (!grid || !V_loc) return fail(nullptr, RSFD_ERR_ARG, "rsfd_create: grid and V_loc must be non-NULL");
  if (grid[0] < 1 || grid[1] < 1 || grid[2] < 2) return fail(nullptr, RSFD_ERR_ARG, "rsfd_create: grid sizes must be >= 1 (Nz >= 2)");
  if (!(hh > 0) || !isfinite(hh)) return fail(nullptr, RSFD_ERR_ARG, "rsfd_create: h must be positive");
  if (fd_order != 2 && fd_order != 4) return fail(nullptr, RSFD_ERR_ARG, "rsfd_create: fd_order must be 2 or 4");
  if (precision != RSFD_FP64 && precision != RSFD_MIXED && precision != RSFD_DF64)
    return fail(nullptr, RSFD_ERR_ARG, "rsfd_create: bad precision");
  const int R = fd_order / 2;
  if (n_face == 0) n_face = R;
  if (n_face < 1 || 2 * n_face > grid[2]) return fail(nullptr, RSFD_ERR_ARG, "rsfd_create: n_face must satisfy 1 <= n_face <= Nz/2");
  const long long N = (long long)grid[0] * grid[1] * grid[2];
  if (N > (1ll << 31) - 1) return fail(nullptr, RSFD_ERR_ARG, "rsfd_create: grid too large (N >= 2^31)");
  if (proj && proj->n_atoms > 0) {
    if (!proj->ptr || !proj->idx || !proj->val || !proj->E)
      return fail(nullptr, RSFD_ERR_ARG, "rsfd_create: projector arrays must be non-NULL");
    if (proj->ptr[0] != 0) return fail(nullptr, RSFD_ERR_ARG, "rsfd_create: projector ptr[0] must be 0");
    for (int a = 0; a < proj->n_atoms; ++a) {
      if (proj->ptr[a + 1] < proj->ptr[a]) return fail(nullptr, RSFD_ERR_ARG, "rsfd_create: projector ptr not monotone");
      if (!isfinite(proj->E[a])) return fail(nullptr, RSFD_ERR_ARG, "rsfd_create: non-finite projector energy");
    }
    const long long nnz = proj->ptr[proj->n_atoms];
    if (nnz > (1ll << 31) - 1) return fail(nullptr, RSFD_ERR_ARG, "rsfd_create: too many projector entries");
    for (long long e = 0; e < nnz; ++e) {
      if (proj->idx[e] < 0 || proj->idx[e] >= N) return fail(nullptr, RSFD_ERR_ARG, "rsfd_create: projector index out of range");
      if (!isfinite(proj->val[e])) return fail(nullptr, RSFD_ERR_ARG, "rsfd_create: non-finite projector value");
    }
  } else if (proj && proj->n_atoms < 0) {
    return fail(nullptr, RSFD_ERR_ARG, "rsfd_create: negative n_atoms");
  }
  for (long long i = 0; i < N; ++i) {
    if (!isfinite(V_loc[i])) return fail(nullptr, RSFD_ERR_ARG, "rsfd_create: V_loc has a non-finite entry");
  }
  rsfd_handle_s* h = new (std::nothrow) rsfd_handle_s();
  if (!h) return fail(nullptr, RSFD_ERR_ALLOC, "rsfd_create: host allocation failed");
  h->nx = grid[0];
  h->ny = grid[1];
  h->nz = grid[2];
  h->nxp = (grid[0] + 3) / 4 * 4;
  h->N = N;
  h->h = hh;
  h->fd_order = fd_order;
  h->R = R;
  h->nface = n_face;
  h->prec = precision;
  h->user_stream = reinterpret_cast<cudaStream_t>(stream);
  memset(&h->opts, 0, sizeof(h->opts));
  memset(&h->stats, 0, sizeof(h->stats));
  const long long nxy = (long long)h->nx * h->ny;
  h->nb = (int)(2 * n_face * nxy);
  h->nr = h->nb;
  h->brow.resize(h->nb);
  for (int pl = 0; pl < 2 * n_face; ++pl) {
    const long long z = pl < n_face ? pl : (h->nz - 2 * n_face + pl);
    for (long long o = 0; o < nxy; ++o) h->brow[pl * nxy + o] = z * nxy + o;
  }
  auto bail = [&](rsfd_status s, const std::string& m) {
    free_all(h);
    if (h->work) cudaStreamDestroy(h->work);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    delete h;
    return fail(nullptr, s, m);
  };
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->work, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = kernels_init();
  if (e != cudaSuccess) return bail(RSFD_ERR_CUDA, std::string("rsfd_create: ") + cudaGetErrorString(e));
  // potential in the padded layout of the internal vectors: float (mixed), double (fp64),
  // (hi, lo) float pairs (double-float)
  const long long npad = (long long)h->nxp * h->ny * h->nz;
  const size_t vsz = pot_elem_bytes(precision);
  e = cudaMalloc(&h->dV, npad * vsz);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->dbrow, h->nb * sizeof(int64_t));
  if (e != cudaSuccess) return bail(RSFD_ERR_ALLOC, std::string("rsfd_create: ") + cudaGetErrorString(e));
  {
    std::vector<unsigned char> vh(npad * vsz, 0);
    for (long long z = 0; z < h->nz; ++z)
      for (long long y = 0; y < h->ny; ++y)
        for (long long x = 0; x < h->nx; ++x) {
          const double v = V_loc[(z * h->ny + y) * h->nx + x];
          const long long q = (z * h->ny + y) * h->nxp + x;
          if (precision == RSFD_FP64) {
            ((double*)vh.data())[q] = v;
          } else if (precision == RSFD_MIXED) {
            ((float*)vh.data())[q] = (float)v;
          } else {
            const float hi = (float)v;
            ((float*)vh.data())[2 * q] = hi;
            ((float*)vh.data())[2 * q + 1] = (float)(v - (double)hi);
          }
        }
    e = cudaMemcpy(h->dV, vh.data(), npad * vsz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && precision == RSFD_DF64) {
      // s V for the block-floating-point split pass: s = 1 / H's coupling at distance R, which makes
      // the neighbour weights of s H the integers -16, 1 (4th order) or -1 (2nd order)
      h->uscale = (fd_order == 4 ? 24.0 : 2.0) * hh * hh;
      std::vector<unsigned char> vs(npad * vsz, 0);
      for (long long z = 0; z < h->nz; ++z)
        for (long long y = 0; y < h->ny; ++y)
          for (long long x = 0; x < h->nx; ++x) {
            const double v = h->uscale * V_loc[(z * h->ny + y) * h->nx + x];
            const long long q = (z * h->ny + y) * h->nxp + x;
            const float hi = (float)v;
            ((float*)vs.data())[2 * q] = hi;
            ((float*)vs.data())[2 * q + 1] = (float)(v - (double)hi);
          }
      e = cudaMalloc(&h->dVs, npad * vsz);
      if (e == cudaSuccess) e = cudaMemcpy(h->dVs, vs.data(), npad * vsz, cudaMemcpyHostToDevice);
    }
  }
  if (e == cudaSuccess) e = cudaMemcpy(h->dbrow, h->brow.data(), h->nb * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bail(RSFD_ERR_CUDA, std::string("rsfd_create: ") + cudaGetErrorString(e));
  {
    uint64_t hv = 1469598103934665603ull;
    const int32_t meta[6] = {grid[0], grid[1], grid[2], fd_order, n_face, precision};
    hv = fnv1a(hv, meta, sizeof(meta));
    hv = fnv1a(hv, &hh, sizeof(hh));
    hv = fnv1a(hv, V_loc, (size_t)N * sizeof(double));
    if (proj && proj->n_atoms > 0) {
      const long long nnz = proj->ptr[proj->n_atoms];
      hv = fnv1a(hv, proj->ptr, (size_t)(proj->n_atoms + 1) * sizeof(int64_t));
      hv = fnv1a(hv, proj->idx, (size_t)nnz * sizeof(int64_t));
      hv = fnv1a(hv, proj->val, (size_t)nnz * sizeof(double));
      hv = fnv1a(hv, proj->E, (size_t)proj->n_atoms * sizeof(double));
    }
    h->in_hash = hv;
  }
  if (proj && proj->n_atoms > 0) {
    // atom-major entries (padded vector indices, values in the potential's element type) and the
    // point-major transpose of the same entries (support points in ascending order, atoms ascending)
    const int na = proj->n_atoms;
    const long long nnz = proj->ptr[na];
    auto pad = [&](long long j) {
      const long long z = j / nxy, r = j - z * nxy, y = r / h->nx, x = r - y * h->nx;
      return (z * h->ny + y) * h->nxp + x;
    };
    auto put = [&](std::vector<unsigned char>& buf, long long q, double v) {
      if (precision == RSFD_FP64) {
        ((double*)buf.data())[q] = v;
      } else if (precision == RSFD_MIXED) {
        ((float*)buf.data())[q] = (float)v;
      } else {
        const float hi = (float)v;
        ((float*)buf.data())[2 * q] = hi;
        ((float*)buf.data())[2 * q + 1] = (float)(v - (double)hi);
      }
    };
    std::vector<int> aptr(na + 1);
    std::vector<long long> aidx(nnz);
    std::vector<unsigned char> aval(nnz * vsz + 16);
    std::vector<std::pair<long long, int>> ent(nnz);   // (grid index, atom) of every entry
    for (int a = 0; a <= na; ++a) aptr[a] = (int)proj->ptr[a];
    for (int a = 0; a < na; ++a)
      for (long long e2 = proj->ptr[a]; e2 < proj->ptr[a + 1]; ++e2) {
        aidx[e2] = pad(proj->idx[e2]);
        put(aval, e2, proj->val[e2]);
        ent[e2] = std::make_pair(proj->idx[e2], a);
      }
    std::vector<long long> order(nnz);
    for (long long e2 = 0; e2 < nnz; ++e2) order[e2] = e2;
    std::stable_sort(order.begin(), order.end(), [&](long long u, long long v) { return ent[u] < ent[v]; });
    std::vector<int> tptr, tatom(nnz);
    std::vector<long long> tpidx;
    std::vector<unsigned char> tval(nnz * vsz + 16);
    for (long long k = 0; k < nnz; ++k) {
      const long long e2 = order[k];
      if (k == 0 || ent[e2].first != ent[order[k - 1]].first) {
        tptr.push_back((int)k);
        tpidx.push_back(pad(ent[e2].first));
      }
      tatom[k] = ent[e2].second;
      put(tval, k, proj->val[e2]);
    }
    tptr.push_back((int)nnz);
    std::vector<double> pmax(na, 0.0);
    for (int a = 0; a < na; ++a)
      for (long long e2 = proj->ptr[a]; e2 < proj->ptr[a + 1]; ++e2) pmax[a] = std::max(pmax[a], std::fabs(proj->val[e2]));
    h->proj_overlap = 0;
    for (size_t k = 0; k + 1 < tptr.size(); ++k) h->proj_overlap = std::max(h->proj_overlap, tptr[k + 1] - tptr[k]);
    h->n_atoms = na;
    h->nnz = nnz;
    h->n_supp = (int)tpidx.size();
    e = cudaMalloc((void**)&h->d_aptr, (na + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_aidx, (nnz + 1) * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_aval, nnz * vsz + 16);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_aE, na * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_tptr, tptr.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_tpidx, (tpidx.size() + 1) * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_tatom, (nnz + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_tval, nnz * vsz + 16);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_pmax, na * sizeof(double));
    if (e != cudaSuccess) return bail(RSFD_ERR_ALLOC, std::string("rsfd_create: ") + cudaGetErrorString(e));
    e = cudaMemcpy(h->d_aptr, aptr.data(), (na + 1) * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_aidx, aidx.data(), nnz * sizeof(long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_aval, aval.data(), nnz * vsz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_aE, proj->E, na * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_tptr, tptr.data(), tptr.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(h->d_tpidx, tpidx.data(), tpidx.size() * sizeof(long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_tatom, tatom.data(), nnz * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_tval, tval.data(), nnz * vsz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_pmax, pmax.data(), na * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(RSFD_ERR_CUDA, std::string("rsfd_create: ") + cudaGetErrorString(e));
  }
  *out = h;
  return RSFD_OK;
}

static rsfd_status rsfd_boundary_rows_impl(rsfd_handle h, int32_t* nb, int64_t* rows) {
  if (!h || !nb) return fail(h, RSFD_ERR_ARG, "rsfd_boundary_rows: NULL argument");
  *nb = h->nb;
  if (rows) memcpy(rows, h->brow.data(), h->nb * sizeof(int64_t));
  return RSFD_OK;
}

static rsfd_status rsfd_set_tracked_planes_impl(rsfd_handle h, int32_t n, const int32_t* z) {
  if (!h) return fail(h, RSFD_ERR_ARG, "rsfd_set_tracked_planes: NULL handle");
  if (n < 0 || n > RSFD_MAX_TRACKED_PLANES || (n > 0 && !z))
    return fail(h, RSFD_ERR_ARG, "rsfd_set_tracked_planes: need 0 <= n <= " + std::to_string(RSFD_MAX_TRACKED_PLANES));
  std::vector<int> t(z, z + n);
  for (int i = 0; i < n; ++i) {
    if (t[i] < h->nface || t[i] >= h->nz - h->nface)
      return fail(h, RSFD_ERR_ARG, "rsfd_set_tracked_planes: plane " + std::to_string(t[i]) + " is not an interior plane");
    for (int j = 0; j < i; ++j)
      if (t[j] == t[i]) return fail(h, RSFD_ERR_ARG, "rsfd_set_tracked_planes: repeated plane");
  }
  const long long nxy = (long long)h->nx * h->ny;
  const long long nr = h->nb + (long long)n * nxy;
  if (nr > (1ll << 30)) return fail(h, RSFD_ERR_ARG, "rsfd_set_tracked_planes: too many recorded rows");
  h->track = t;
  h->nr = (int)nr;
  return RSFD_OK;
}

static rsfd_status rsfd_tracked_rows_impl(rsfd_handle h, int32_t* nr, int64_t* rows) {
  if (!h || !nr) return fail(h, RSFD_ERR_ARG, "rsfd_tracked_rows: NULL argument");
  *nr = h->nr;
  if (rows) {
    memcpy(rows, h->brow.data(), h->nb * sizeof(int64_t));
    const long long nxy = (long long)h->nx * h->ny;
    for (size_t e = 0; e < h->track.size(); ++e)
      for (long long o = 0; o < nxy; ++o) rows[h->nb + e * nxy + o] = (long long)h->track[e] * nxy + o;
  }
  return RSFD_OK;
}

static rsfd_status rsfd_set_solve_options_impl(rsfd_handle h, const rsfd_solve_opts* o) {
  if (!h) return fail(h, RSFD_ERR_ARG, "rsfd_set_solve_options: NULL handle");
  if (!o) {
    memset(&h->opts, 0, sizeof(h->opts));
    return RSFD_OK;
  }
  if (o->slots < 0 || o->iters_per_sync < 0 || o->tile_y < 0 || o->z_chunk < 0 || o->prefetch < 0)
    return fail(h, RSFD_ERR_ARG, "rsfd_set_solve_options: negative option");
  if (o->pass_kind < 0 || o->pass_kind > RSFD_PASS_SPLIT_BFP)
    return fail(h, RSFD_ERR_ARG, "rsfd_set_solve_options: bad pass_kind");
  if (o->pass_kind == RSFD_PASS_RECOMPUTE && h->n_atoms > 0)
    return fail(h, RSFD_ERR_ARG, "rsfd_set_solve_options: the recompute pass has no projector term; use the stored pass");
  if (o->rows_per_thread != 0 && o->rows_per_thread != 1 && o->rows_per_thread != 2 && o->rows_per_thread != 4)
    return fail(h, RSFD_ERR_ARG, "rsfd_set_solve_options: rows_per_thread must be 0, 1, 2 or 4");
  const int rows = resolve_rows(o->rows_per_thread);
  if (o->prefetch > pass_max_depth())
    return fail(h, RSFD_ERR_ARG, "rsfd_set_solve_options: prefetch must be <= " + std::to_string(pass_max_depth()));
  const int kind = resolve_kind(h->prec, o->pass_kind);
  if (o->reg_budget < 0 || o->reg_budget > 1)
    return fail(h, RSFD_ERR_ARG, "rsfd_set_solve_options: reg_budget must be 0 or 1");
  if (o->tile_x != 0 && o->tile_x != 16 && o->tile_x != 32)
    return fail(h, RSFD_ERR_ARG, "rsfd_set_solve_options: tile_x must be 0, 16 or 32");
  const int txo = o->tile_x == 16 ? 16 : 32;
  if (!tile_ok(h->prec, h->R, o->tile_y > 0 ? o->tile_y : default_tile_y(h->prec, h->R, h->ny, kind, rows), kind, rows,
               o->reg_budget, txo))
    return fail(h, RSFD_ERR_ARG, "rsfd_set_solve_options: the tile does not fit this pass, precision, register budget "
                                 "or tile width");
  if (o->tile_y > 0 && !tile_ok(h->prec, h->R, o->tile_y, kind, rows))
    return fail(h, RSFD_ERR_ARG, "rsfd_set_solve_options: tile_y not allowed for this precision, stencil order and pass");
  if (o->prefetch > 0 && kind_smem(h->prec, h->R,
                                   o->tile_y > 0 ? o->tile_y : default_tile_y(h->prec, h->R, h->ny, kind, rows),
                                   o->prefetch, kind) > (size_t)(216 * 1024))
    return fail(h, RSFD_ERR_ARG, "rsfd_set_solve_options: prefetch depth does not fit in shared memory");
  if (o->dyson_kind < 0 || o->dyson_kind > RSFD_DYSON_TC)
    return fail(h, RSFD_ERR_ARG, "rsfd_set_solve_options: bad dyson_kind");
  if (o->dyson_refine < 0 || o->dyson_refine > 8)
    return fail(h, RSFD_ERR_ARG, "rsfd_set_solve_options: dyson_refine must be 0 .. 8");
  if (o->iters_per_sync > kMaxHist)
    return fail(h, RSFD_ERR_ARG, "rsfd_set_solve_options: iters_per_sync must be <= " + std::to_string(kMaxHist));
  if (o->wait_cap < -1) return fail(h, RSFD_ERR_ARG, "rsfd_set_solve_options: wait_cap must be >= -1");
  if (o->dyson_cols < 0 || o->dyson_cols > 1) return fail(h, RSFD_ERR_ARG, "rsfd_set_solve_options: dyson_cols must be 0 or 1");
  if (!(o->breakdown_tol >= 0.0) || !isfinite(o->breakdown_tol))
    return fail(h, RSFD_ERR_ARG, "rsfd_set_solve_options: breakdown_tol must be finite and >= 0");
  h->opts = *o;
  return RSFD_OK;
}

static rsfd_status rsfd_get_stats_impl(rsfd_handle h, rsfd_stats* out) {
  if (!h || !out) return fail(h, RSFD_ERR_ARG, "rsfd_get_stats: NULL argument");
  *out = h->stats;
  return RSFD_OK;
}

static rsfd_status rsfd_shifted_cocg_impl(rsfd_handle h, const int64_t* cols, int32_t ncols, const double* energies,
                              int32_t Kout, const double* aux_energies, int32_t n_aux, double eta, double tol,
                              int32_t maxit, int32_t seed_kind, int32_t seed_index, void* G0_bb, rsfd_col_info* info,
                              double* final_res) {
  if (!h) return fail(nullptr, RSFD_ERR_ARG, "rsfd_shifted_cocg: NULL handle");
  if (!cols || ncols < 1) return fail(h, RSFD_ERR_ARG, "rsfd_shifted_cocg: need ncols >= 1 columns");
  if (!energies || Kout < 1) return fail(h, RSFD_ERR_ARG, "rsfd_shifted_cocg: need K >= 1 energies");
  if (n_aux < 0 || (n_aux > 0 && !aux_energies)) return fail(h, RSFD_ERR_ARG, "rsfd_shifted_cocg: bad auxiliary energies");
  for (int k = 0; k < n_aux; ++k)
    if (!isfinite(aux_energies[k])) return fail(h, RSFD_ERR_ARG, "rsfd_shifted_cocg: non-finite auxiliary energy");
  // the shifts the scalar recurrences carry: the K energies of the set, then the auxiliary ones
  // (seed candidates only: no output, not needed for termination)
  const int K = Kout + n_aux;
  if (!(eta > 0) || !isfinite(eta)) return fail(h, RSFD_ERR_ARG, "rsfd_shifted_cocg: eta must be positive");
  if (!(tol > 0) || !(tol < 1)) return fail(h, RSFD_ERR_ARG, "rsfd_shifted_cocg: tol must lie in (0, 1)");
  if (maxit < 1) return fail(h, RSFD_ERR_ARG, "rsfd_shifted_cocg: maxit must be >= 1");
  if (!G0_bb) return fail(h, RSFD_ERR_ARG, "rsfd_shifted_cocg: G0_bb is NULL");
  for (int k = 0; k < Kout; ++k)
    if (!isfinite(energies[k])) return fail(h, RSFD_ERR_ARG, "rsfd_shifted_cocg: non-finite energy");
  for (int c = 0; c < ncols; ++c)
    if (cols[c] < 0 || cols[c] >= h->N) return fail(h, RSFD_ERR_ARG, "rsfd_shifted_cocg: column index out of range");
  int seed0 = 0;
  if (seed_kind == RSFD_SEED_MID) seed0 = Kout / 2;
  else if (seed_kind == RSFD_SEED_FIRST) seed0 = 0;
  else if (seed_kind == RSFD_SEED_INDEX) {
    if (seed_index < 0 || seed_index >= Kout) return fail(h, RSFD_ERR_ARG, "rsfd_shifted_cocg: seed_index out of range");
    seed0 = seed_index;
  } else if (seed_kind == RSFD_SEED_AUX) {
    if (seed_index < 0 || seed_index >= n_aux)
      return fail(h, RSFD_ERR_ARG, "rsfd_shifted_cocg: seed_index out of range of the auxiliary energies");
    seed0 = Kout + seed_index;
  } else {
    return fail(h, RSFD_ERR_ARG, "rsfd_shifted_cocg: bad seed_kind");
  }
  const int prec = h->prec;
  const size_t vsz = vec_elem_bytes(prec), hsz = hist_elem_bytes(prec);

  // ---- launch shape
  SolveDims d;
  memset(&d, 0, sizeof(d));
  d.nx = h->nx;
  d.ny = h->ny;
  d.nz = h->nz;
  d.nxp = h->nxp;
  d.N = h->N;
  d.R = h->R;
  d.nface = h->nface;
  d.nb = h->nr;
  d.ntrack = (int)h->track.size();
  for (int e = 0; e < d.ntrack; ++e) d.track[e] = h->track[e];
  d.K = K;
  d.kreq = Kout;
  d.ncols = ncols;
  d.kind = resolve_kind(prec, h->opts.pass_kind);
  // the projector term follows a pass that stores A r (stored-product or split)
  if (h->n_atoms > 0 && d.kind == RSFD_PASS_RECOMPUTE) d.kind = RSFD_PASS_STORED;
  d.nvec = d.kind == RSFD_PASS_RECOMPUTE ? 3 : 5;
  d.rows = is_split(d.kind) ? 1 : resolve_rows(h->opts.rows_per_thread);
  d.tile_y = h->opts.tile_y > 0 ? h->opts.tile_y : default_tile_y(prec, h->R, h->ny, d.kind, d.rows);
  d.regs = (prec == RSFD_DF64 && d.rows == 1 && (d.kind == RSFD_PASS_STORED || d.kind == RSFD_PASS_SPLIT_BFP))
               ? h->opts.reg_budget
               : 0;
  d.tile_x = (h->opts.tile_x == 16 && d.kind == RSFD_PASS_STORED) ? 16 : 32;
  d.wait_cap = h->opts.wait_cap;
  d.brk_tol = h->opts.breakdown_tol > 0.0 ? h->opts.breakdown_tol : 1e-28;
  if (!tile_ok(prec, h->R, d.tile_y, d.kind, d.rows, d.regs, d.tile_x))
    return fail(h, RSFD_ERR_ARG, "rsfd_shifted_cocg: invalid tile_y / tile_x");
  // TMA prefetch depth: the option, else the deepest that fits in shared memory (fused pass: a CTA
  // alone on its SM) or 3 (stored-product pass: bundles are three times larger)
  if (h->opts.prefetch > 0) {
    d.depth = h->opts.prefetch;
  } else {
    d.depth = 1;
    const int dmax = d.kind == RSFD_PASS_STORED ? 3 : (is_split(d.kind) ? 4 : pass_max_depth());
    for (int dp = dmax; dp >= 1; --dp)
      if (kind_smem(prec, h->R, d.tile_y, dp, d.kind, d.tile_x) <= (size_t)(216 * 1024)) {
        d.depth = dp;
        break;
      }
  }
  if (kind_smem(prec, h->R, d.tile_y, d.depth, d.kind, d.tile_x) > (size_t)(216 * 1024))
    return fail(h, RSFD_ERR_ARG, "rsfd_shifted_cocg: prefetch depth does not fit in shared memory");
  {
    const int tw = d.kind == RSFD_PASS_RECOMPUTE ? pass_tile_x(h->R) : d.tile_x;
    d.tiles_x = (h->nx + tw - 1) / tw;
  }
  d.tiles_y = (h->ny + d.tile_y - 1) / d.tile_y;
  int W0 = h->opts.slots > 0 ? h->opts.slots : 256;
  W0 = std::min(W0, ncols);
  if (h->opts.z_chunk > 0) {
    d.zchunk = h->opts.z_chunk;
  } else {
    // whole z-columns per CTA (no pipeline refill) unless that leaves fewer than ~4 CTAs per SM
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    d.zchunk = h->nz;
    while (d.zchunk > 16 && (long long)d.tiles_x * d.tiles_y * ((h->nz + d.zchunk - 1) / d.zchunk) * W0 < 4LL * sms)
      d.zchunk = (d.zchunk + 1) / 2;
  }
  d.nzchunks = (h->nz + d.zchunk - 1) / d.zchunk;
  d.ctas_per_slot = d.tiles_x * d.tiles_y * d.nzchunks;
  d.ctas_c = 0;
  const int C = h->opts.iters_per_sync > 0 ? h->opts.iters_per_sync : 32;
  if (C > kMaxHist) return fail(h, RSFD_ERR_ARG, "rsfd_shifted_cocg: iters_per_sync too large");
  const long long vec = (long long)h->nxp * h->ny * h->nz;
  int W = W0;
  {
    size_t freeb = 0, totb = 0;
    RSFD_CK(h, cudaMemGetInfo(&freeb, &totb));
    const size_t per_slot = (size_t)d.nvec * vec * vsz + 2 * (size_t)K * h->nr * vsz + (size_t)C * h->nr * hsz +
                            (size_t)K * C * sizeof(ShiftCoef) + (size_t)K * sizeof(ShiftState) +
                            (size_t)(d.ctas_per_slot + 64) * 64 + 256;
    const size_t have = h->rbuf.bytes + h->xbuf.bytes + h->pbuf.bytes + h->rhist.bytes + h->coef.bytes;
    const size_t budget = (size_t)(0.6 * (double)(freeb + have));
    if (h->opts.slots <= 0) {
      while (W > 1 && per_slot * W > budget) W /= 2;
    }
  }
  d.W = W;
  if (is_split(d.kind)) {
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    d.ctas_c = split_combine_ctas(h->nz, W, sms);
  }
  d.npart = d.ctas_per_slot + d.ctas_c;
  const bool use_graphs = h->opts.use_graphs >= 0;

  // ---- workspace
  rsfd_status s;
  if ((s = ensure(h, h->rbuf, (size_t)W * d.nvec * vec * vsz)) != RSFD_OK) return s;
  if ((s = ensure(h, h->xbuf, (size_t)W * K * h->nr * vsz)) != RSFD_OK) return s;
  if ((s = ensure(h, h->pbuf, (size_t)W * K * h->nr * vsz)) != RSFD_OK) return s;
  if ((s = ensure(h, h->rhist, (size_t)W * C * h->nr * hsz)) != RSFD_OK) return s;
  if ((s = ensure(h, h->coef, (size_t)W * K * C * sizeof(ShiftCoef))) != RSFD_OK) return s;
  if ((s = ensure(h, h->cw, (size_t)W * K * 2 * C * hsz)) != RSFD_OK) return s;
  if ((s = ensure(h, h->ce, (size_t)W * K * 2 * sizeof(double2))) != RSFD_OK) return s;
  if ((s = ensure(h, h->eflag, 16)) != RSFD_OK) return s;
  if ((s = ensure(h, h->slots, (size_t)W * sizeof(SlotState))) != RSFD_OK) return s;
  if ((s = ensure(h, h->shifts, (size_t)W * K * sizeof(ShiftState))) != RSFD_OK) return s;
  if ((s = ensure(h, h->partials, (size_t)W * d.npart * 8 * sizeof(double))) != RSFD_OK) return s;
  if ((s = ensure(h, h->tickets, (size_t)W * sizeof(unsigned int))) != RSFD_OK) return s;
  if ((s = ensure(h, h->Z, (size_t)K * sizeof(double2))) != RSFD_OK) return s;
  if ((s = ensure(h, h->init_list, (size_t)W * 2 * sizeof(int))) != RSFD_OK) return s;
  if ((s = ensure(h, h->init_grid, (size_t)W * sizeof(long long))) != RSFD_OK) return s;
  if ((s = ensure(h, h->counters, 4 * sizeof(unsigned long long))) != RSFD_OK) return s;
  if ((s = make_maps(h, W, d.tile_y, d.kind, d.tile_x)) != RSFD_OK) return s;
  SolverBuffers b;
  memset(&b, 0, sizeof(b));
  b.rbuf = h->rbuf.p;
  b.xbuf = h->xbuf.p;
  b.pbuf = h->pbuf.p;
  b.rhist = h->rhist.p;
  b.coef = (ShiftCoef*)h->coef.p;
  b.cwbuf = h->cw.p;
  b.cebuf = (double2*)h->ce.p;
  b.error_flag = (int*)h->eflag.p;
  b.tmR = &h->tmR;
  b.tmV = &h->tmV;
  b.V = h->dV;
  b.tmVs = &h->tmVs;
  b.Vs = h->dVs;
  b.uscale = h->uscale;
  b.slots = (SlotState*)h->slots.p;
  b.shifts = (ShiftState*)h->shifts.p;
  b.partials = (double*)h->partials.p;
  b.tickets = (unsigned int*)h->tickets.p;
  b.Z = (double2*)h->Z.p;
  b.brow = h->dbrow;
  b.G0 = G0_bb;
  b.init_list = (int*)h->init_list.p;
  b.init_grid = (long long*)h->init_grid.p;
  b.counters = (unsigned long long*)h->counters.p;
  if (h->n_atoms > 0) {
    if ((s = ensure(h, h->pw, (size_t)W * h->n_atoms * sizeof(double2))) != RSFD_OK) return s;
    if ((s = ensure(h, h->pcorr, (size_t)W * h->n_atoms * sizeof(double2))) != RSFD_OK) return s;
    if ((s = ensure(h, h->pdots, (size_t)W * 8 * sizeof(double))) != RSFD_OK) return s;
    if ((s = ensure(h, h->ptickets, (size_t)W * sizeof(unsigned int))) != RSFD_OK) return s;
    b.n_atoms = h->n_atoms;
    b.n_supp = h->n_supp;
    b.a_ptr = h->d_aptr;
    b.a_idx = h->d_aidx;
    b.a_val = h->d_aval;
    b.a_E = h->d_aE;
    b.t_ptr = h->d_tptr;
    b.a_pmax = h->d_pmax;
    b.proj_overlap = h->proj_overlap;
    b.t_pidx = h->d_tpidx;
    b.t_atom = h->d_tatom;
    b.t_val = h->d_tval;
    b.h3 = h->h * h->h * h->h;
    b.pw = (double2*)h->pw.p;
    b.pcorr = (double2*)h->pcorr.p;
    b.pdots = (double*)h->pdots.p;
    b.ptickets = (unsigned int*)h->ptickets.p;
  }
  const StencilCoef coef = stencil_coef(h->fd_order, h->h);

  if ((s = handle_begin(h)) != RSFD_OK) return s;
  cudaStream_t st = h->work;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  RSFD_CK(h, cudaEventCreate(&t0));
  RSFD_CK(h, cudaEventCreate(&t1));
  RSFD_CK(h, cudaEventRecord(t0, st));

  std::vector<double2> Zh(K);
  for (int k = 0; k < K; ++k) Zh[k] = make_double2(k < Kout ? energies[k] : aux_energies[k - Kout], eta);
  RSFD_CK(h, cudaMemcpyAsync(b.Z, Zh.data(), K * sizeof(double2), cudaMemcpyHostToDevice, st));
  RSFD_CK(h, cudaMemsetAsync(b.tickets, 0, W * sizeof(unsigned int), st));
  if (b.n_atoms > 0) RSFD_CK(h, cudaMemsetAsync(b.ptickets, 0, W * sizeof(unsigned int), st));
  RSFD_CK(h, cudaMemsetAsync(b.counters, 0, 4 * sizeof(unsigned long long), st));
  RSFD_CK(h, cudaMemsetAsync(b.error_flag, 0, sizeof(int), st));
  std::vector<SlotState> hs(W);
  for (int w = 0; w < W; ++w) {
    memset(&hs[w], 0, sizeof(SlotState));
    hs[w].col = -1;
    hs[w].status = SLOT_EMPTY;
    hs[w].k4_n = -1;
  }
  RSFD_CK(h, cudaMemcpyAsync(b.slots, hs.data(), W * sizeof(SlotState), cudaMemcpyHostToDevice, st));

  memset(&h->stats, 0, sizeof(h->stats));
  h->stats.slots = W;
  h->stats.iters_per_sync = C;
  // Pinned host staging, double-buffered by chunk parity: the slot states copied after a chunk,
  // the error flag, the lists of finished and new columns, and the finished columns' residuals.
  struct Pinned {
    void* p = nullptr;
    ~Pinned() { if (p) cudaFreeHost(p); }
  };
  Pinned pin_states, pin_lists, pin_res;
  RSFD_CK(h, cudaMallocHost(&pin_states.p, 2 * (W * sizeof(SlotState) + 64)));
  RSFD_CK(h, cudaMallocHost(&pin_lists.p, 2 * (4 * W * sizeof(int) + W * sizeof(long long) + 64)));
  if (final_res) RSFD_CK(h, cudaMallocHost(&pin_res.p, (size_t)ncols * K * sizeof(double) + 64));
  auto states_of = [&](int par) -> SlotState* {
    return (SlotState*)((char*)pin_states.p + par * (W * sizeof(SlotState) + 64));
  };
  auto err_of = [&](int par) -> int* { return (int*)(states_of(par) + W); };
  auto lists_of = [&](int par) -> int* {
    return (int*)((char*)pin_lists.p + par * (4 * W * sizeof(int) + W * sizeof(long long) + 64));
  };
  auto grid_of = [&](int par) -> long long* { return (long long*)(lists_of(par) + 4 * W); };
  double* res_host = (double*)pin_res.p;

  std::vector<int> slot_col(W, -1);
  std::vector<long long> valid_from(W, 0);   // first chunk whose copied state reflects the slot's column
  int next = 0;
  rsfd_status worst = RSFD_OK;

  // load new columns into the given free slots (enqueued; the lists come from pinned staging set par)
  auto assign = [&](const std::vector<int>& free_slots, int par, long long first_valid) -> rsfd_status {
    int n_init = 0;
    int* list = lists_of(par) + 2 * W;
    long long* init_grid = grid_of(par);
    for (int w : free_slots) {
      if (next >= ncols) break;
      list[2 * n_init] = w;
      list[2 * n_init + 1] = next;
      init_grid[n_init] = cols[next];
      slot_col[w] = next;
      valid_from[w] = first_valid;
      ++next;
      ++n_init;
    }
    if (n_init == 0) return RSFD_OK;
    RSFD_CK(h, cudaMemcpyAsync(b.init_list, list, 2 * n_init * sizeof(int), cudaMemcpyHostToDevice, st));
    RSFD_CK(h, cudaMemcpyAsync(b.init_grid, init_grid, n_init * sizeof(long long), cudaMemcpyHostToDevice, st));
    RSFD_CK(h, launch_slot_init(prec, d, b, n_init, seed0, st));
    h->stats.n_other += 1;
    return RSFD_OK;
  };

  {
    std::vector<int> all(W);
    for (int w = 0; w < W; ++w) all[w] = w;
    if ((s = assign(all, 0, 0)) != RSFD_OK) return s;
    RSFD_CK(h, cudaStreamSynchronize(st));   // the pinned lists of set 0 are reused below
  }

  // One chunk: C passes, then the collapsed shift update of the C recorded steps.  Two graphs (and two
  // sets of profiling events) alternate, so that chunk k + 1 can be enqueued before the host reads
  // the events and slot states of chunk k.
  struct Graphs {
    cudaGraph_t g[2] = {nullptr, nullptr};
    cudaGraphExec_t x[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> ev[2];
    ~Graphs() {
      for (int i = 0; i < 2; ++i) {
        if (x[i]) cudaGraphExecDestroy(x[i]);
        if (g[i]) cudaGraphDestroy(g[i]);
        for (auto e : ev[i]) cudaEventDestroy(e);
      }
    }
  } gr;
  const bool split_ev = h->opts.profile && is_split(d.kind);
  if (h->opts.profile) {
    for (int i = 0; i < 2; ++i) {
      gr.ev[i].resize(C + 2 + (split_ev ? C : 0));   // [C + 2 + t]: between the split pass's two launches
      for (auto& e : gr.ev[i]) RSFD_CK(h, cudaEventCreate(&e));
    }
  }
  auto rec = [&](cudaEvent_t e) -> cudaError_t {
    return use_graphs ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal) : cudaEventRecord(e, st);
  };
  auto issue_chunk = [&](int par) -> rsfd_status {
    std::vector<cudaEvent_t>& pev = gr.ev[par];
    for (int t = 0; t < C; ++t) {
      if (h->opts.profile) RSFD_CK(h, rec(pev[t]));
      RSFD_CK(h, launch_pass(prec, d, b, coef, tol, maxit, C, st, split_ev ? pev[C + 2 + t] : nullptr, use_graphs));
      if (b.n_atoms > 0) RSFD_CK(h, launch_proj(prec, d, b, coef, tol, maxit, C, st));
    }
    if (h->opts.profile) RSFD_CK(h, rec(pev[C]));
    RSFD_CK(h, launch_chunk(prec, d, b, C, st));
    if (h->opts.profile) RSFD_CK(h, rec(pev[C + 1]));
    return RSFD_OK;
  };
  if (use_graphs) {
    for (int i = 0; i < 2; ++i) {
      RSFD_CK(h, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      rsfd_status cs = issue_chunk(i);
      cudaError_t ce = cudaStreamEndCapture(st, &gr.g[i]);
      if (cs != RSFD_OK) return cs;
      RSFD_CK(h, ce);
      RSFD_CK(h, cudaGraphInstantiate(&gr.x[i], gr.g[i], 0));
    }
  }
  // chunk k, followed by the copy of the slot states and the error flag into staging set k % 2
  cudaEvent_t copied[2] = {nullptr, nullptr};
  struct EvPair {
    cudaEvent_t* e;
    ~EvPair() { for (int i = 0; i < 2; ++i) if (e[i]) cudaEventDestroy(e[i]); }
  } evp{copied};
  for (int i = 0; i < 2; ++i) RSFD_CK(h, cudaEventCreateWithFlags(&copied[i], cudaEventDisableTiming));
  auto launch_chunk_k = [&](long long k) -> rsfd_status {
    const int par = (int)(k & 1);
    if (use_graphs) {
      RSFD_CK(h, cudaGraphLaunch(gr.x[par], st));
    } else {
      rsfd_status cs = issue_chunk(par);
      if (cs != RSFD_OK) return cs;
    }
    h->stats.n_pass += (int64_t)C * (is_split(d.kind) ? 2 : 1);   // the split passes launch twice per iteration
    h->stats.n_shift += 1;
    h->stats.n_other += 2 + (b.n_atoms > 0 ? 2 * C : 0);   // collapse coefficients, history reset, projectors
    RSFD_CK(h, cudaMemcpyAsync(states_of(par), b.slots, W * sizeof(SlotState), cudaMemcpyDeviceToHost, st));
    RSFD_CK(h, cudaMemcpyAsync(err_of(par), b.error_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    RSFD_CK(h, cudaEventRecord(copied[par], st));
    return RSFD_OK;
  };

  int64_t iter_sum = 0;
  if ((s = launch_chunk_k(0)) != RSFD_OK) return s;
  for (long long k = 0;; ++k) {
    // enqueue chunk k + 1 before reading chunk k's states; a slot that finished in chunk k is idle in
    // chunk k + 1 (its kernels return at once), so its x_b is still final when it is written out
    if ((s = launch_chunk_k(k + 1)) != RSFD_OK) return s;
    const int par = (int)(k & 1);
    RSFD_CK(h, cudaEventSynchronize(copied[par]));
    if (*err_of(par)) {
      worst = RSFD_ERR_TIMEOUT;
      break;
    }
    if (h->opts.profile) {
      std::vector<cudaEvent_t>& pev = gr.ev[par];
      for (int t = 0; t < C; ++t) {
        float a = 0;
        RSFD_CK(h, cudaEventElapsedTime(&a, pev[t], pev[t + 1]));
        h->stats.ms_pass += a;
        if (split_ev) {
          RSFD_CK(h, cudaEventElapsedTime(&a, pev[t], pev[C + 2 + t]));
          h->stats.ms_combine += a;
        }
      }
      float c2 = 0;
      RSFD_CK(h, cudaEventElapsedTime(&c2, pev[C], pev[C + 1]));
      h->stats.ms_shift += c2;
    }
    const SlotState* hs = states_of(par);
    // finished columns: write x_b into G0_bb (enqueued after chunk k + 1), record the outcome, free the slot
    std::vector<int> freed;
    int* list = lists_of(par);
    int n_out = 0;
    for (int w = 0; w < W; ++w) {
      if (slot_col[w] < 0 || k < valid_from[w] || hs[w].status == SLOT_RUNNING) continue;
      list[2 * n_out] = w;
      list[2 * n_out + 1] = slot_col[w];
      ++n_out;
    }
    if (n_out > 0) {
      RSFD_CK(h, cudaMemcpyAsync(b.init_list, list, 2 * n_out * sizeof(int), cudaMemcpyHostToDevice, st));
      RSFD_CK(h, launch_writeout(prec, d, b, G0_bb, n_out, st));
      h->stats.n_other += 1;
    }
    for (int q = 0; q < n_out; ++q) {
      const int w = list[2 * q], c = list[2 * q + 1];
      rsfd_status cs = RSFD_OK;
      if (hs[w].status == SLOT_MAXIT) cs = RSFD_ERR_NOT_CONVERGED;
      if (hs[w].status == SLOT_BREAKDOWN) cs = RSFD_ERR_BREAKDOWN;
      if (cs != RSFD_OK && (worst == RSFD_OK || cs == RSFD_ERR_BREAKDOWN)) worst = cs;
      iter_sum += hs[w].iters;
      if (info) {
        info[c].iters = hs[w].iters;
        info[c].switches = hs[w].switches;
        info[c].status = cs;
        info[c].final_seed = hs[w].seed;
      }
      if (final_res) {   // the residuals of the set's energies, read back before the slot is reused
        RSFD_CK(h, cudaMemcpy2DAsync(res_host + (size_t)c * Kout, sizeof(double),
                                     (const char*)(b.shifts + (size_t)w * K) + offsetof(ShiftState, res),
                                     sizeof(ShiftState), sizeof(double), Kout, cudaMemcpyDeviceToHost, st));
      }
      slot_col[w] = -1;
      freed.push_back(w);
    }
    if (!freed.empty() && next < ncols) {
      if ((s = assign(freed, par, k + 2)) != RSFD_OK) return s;
    }
    bool any = false;
    for (int w = 0; w < W; ++w) any |= slot_col[w] >= 0;
    if (!any && next >= ncols) break;
  }
  RSFD_CK(h, cudaStreamSynchronize(st));
  if (final_res && worst != RSFD_ERR_TIMEOUT) memcpy(final_res, res_host, (size_t)ncols * Kout * sizeof(double));
  RSFD_CK(h, cudaEventRecord(t1, st));
  RSFD_CK(h, cudaEventSynchronize(t1));
  float ms = 0;
  RSFD_CK(h, cudaEventElapsedTime(&ms, t0, t1));
  h->stats.ms_total = ms;
  unsigned long long cnt[4];
  RSFD_CK(h, cudaMemcpy(cnt, b.counters, sizeof(cnt), cudaMemcpyDeviceToHost));
  h->stats.shift_updates = (int64_t)cnt[0];
  h->stats.shift_slot_chunks = (int64_t)cnt[2];
  h->stats.slot_iterations = iter_sum;
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if ((s = handle_end(h)) != RSFD_OK) return s;
  if (worst == RSFD_ERR_TIMEOUT) {
    h->err = "rsfd_shifted_cocg: a bounded wait for a TMA transfer expired; the solve was abandoned";
  } else if (worst != RSFD_OK) {
    h->err = worst == RSFD_ERR_BREAKDOWN ? "rsfd_shifted_cocg: breakdown in at least one column"
                                         : "rsfd_shifted_cocg: at least one column reached maxit";
  }
  return worst;
}

static rsfd_status rsfd_dyson_boundary_impl(rsfd_handle h, const void* G0_bb, const void* Sigma_L, const void* Sigma_R,
                                int32_t K, void* G_bb, double* refine_residual) {
  if (!h) return fail(nullptr, RSFD_ERR_ARG, "rsfd_dyson_boundary: NULL handle");
  if (!G0_bb || !Sigma_L || !Sigma_R || !G_bb || K < 1) return fail(h, RSFD_ERR_ARG, "rsfd_dyson_boundary: bad arguments");
  if (G0_bb == G_bb) return fail(h, RSFD_ERR_ARG, "rsfd_dyson_boundary: G_bb may not alias G0_bb");
  return dyson_run(h, G0_bb, Sigma_L, Sigma_R, K, G_bb, refine_residual);
}

static rsfd_status rsfd_dyson_tracked_impl(rsfd_handle h, const void* G0, const void* Sigma_L, const void* Sigma_R, int32_t K,
                               void* G, double* refine_residual) {
  if (!h) return fail(nullptr, RSFD_ERR_ARG, "rsfd_dyson_tracked: NULL handle");
  if (!G0 || !Sigma_L || !Sigma_R || !G || K < 1) return fail(h, RSFD_ERR_ARG, "rsfd_dyson_tracked: bad arguments");
  if (G0 == G) return fail(h, RSFD_ERR_ARG, "rsfd_dyson_tracked: G may not alias G0");
  return dyson_tracked_run(h, h->nr, G0, Sigma_L, Sigma_R, K, G, refine_residual);
}

static rsfd_status rsfd_transmission_impl(rsfd_handle h, const void* G_bb, const void* Sigma_L, const void* Sigma_R, int32_t K,
                              double* T) {
  if (!h) return fail(nullptr, RSFD_ERR_ARG, "rsfd_transmission: NULL handle");
  if (!G_bb || !Sigma_L || !Sigma_R || !T || K < 1) return fail(h, RSFD_ERR_ARG, "rsfd_transmission: bad arguments");
  return transmission_run(h, G_bb, Sigma_L, Sigma_R, K, T);
}

static rsfd_status rsfd_lead_sigma_uniform_impl(int32_t Nx, int32_t Ny, double hh, int32_t fd_order, const double* energies,
                                    double eta, int32_t K, double* Sigma_L, double* Sigma_R) {
  if (Nx < 1 || Ny < 1 || !(hh > 0) || (fd_order != 2 && fd_order != 4) || !energies || K < 1 || !Sigma_L ||
      !Sigma_R || !(eta > 0))
    return fail(nullptr, RSFD_ERR_ARG, "rsfd_lead_sigma_uniform: bad arguments");
  std::string err;
  rsfd_status s = lead_sigma_uniform(Nx, Ny, hh, fd_order, energies, eta, K, Sigma_L, Sigma_R, &err);
  if (s != RSFD_OK) return fail(nullptr, s, err);
  return RSFD_OK;
}

const char* rsfd_last_error(rsfd_handle h) {
  if (h) return h->err.c_str();
  return g_last_error.c_str();
}

void rsfd_destroy(rsfd_handle h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->work) cudaStreamSynchronize(h->work);
  free_all(h);
  if (h->work) cudaStreamDestroy(h->work);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  delete h;
}


// Launch-option autotuner: short solves (iters seed iterations, profile events on) of the handle's
// first boundary columns at the caller's energies for every candidate (pass form, tile height, rows
// per thread, z-chunk), keeping the least device time per slot-iteration.  Results are cached per
// process by (grid, order, precision, projectors, K, slots).
struct TuneKey {
  int nx, ny, nz, fd, prec, proj, K, slots;
  bool operator<(const TuneKey& o) const {
    const int a[8] = {nx, ny, nz, fd, prec, proj, K, slots};
    const int b[8] = {o.nx, o.ny, o.nz, o.fd, o.prec, o.proj, o.K, o.slots};
    return std::lexicographical_compare(a, a + 8, b, b + 8);
  }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, std::pair<rsfd_solve_opts, double>> g_tune_cache;

static rsfd_status rsfd_autotune_impl(rsfd_handle h, const double* energies, int32_t K, double eta, int32_t slots, int32_t iters,
                          rsfd_solve_opts* best, double* us_per_slot_iteration) {
  if (!h || !energies || K < 1 || !(eta > 0) || slots < 1 || iters < 1)
    return fail(h, RSFD_ERR_ARG, "rsfd_autotune: bad argument");
  const int ncols = std::min<long long>(slots, (long long)h->brow.size());
  const TuneKey key{h->nx, h->ny, h->nz, h->fd_order, h->prec, h->n_atoms > 0 ? 1 : 0, (int)K, ncols};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      rsfd_solve_opts o = it->second.first;
      o.profile = h->opts.profile;
      o.dyson_kind = h->opts.dyson_kind;
      o.dyson_refine = h->opts.dyson_refine;
      h->opts = o;
      if (best) *best = o;
      if (us_per_slot_iteration) *us_per_slot_iteration = it->second.second;
      return RSFD_OK;
    }
  }
  const rsfd_solve_opts keep = h->opts;
  const int C = keep.iters_per_sync > 0 ? keep.iters_per_sync : 32;
  const int maxit = std::max<int>(iters, 2 * C);
  std::vector<int64_t> cols(h->brow.begin(), h->brow.begin() + ncols);
  void* G0 = nullptr;
  const size_t gbytes = (size_t)K * ncols * h->nr * (h->prec == RSFD_MIXED ? 8 : 16);
  if (cudaMalloc(&G0, gbytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, RSFD_ERR_ALLOC, "rsfd_autotune: cudaMalloc of the trial output failed");
  }
  std::vector<rsfd_col_info> info(ncols);
  std::vector<double> res((size_t)ncols * K);
  std::vector<rsfd_solve_opts> cand;
  const int kinds[4] = {RSFD_PASS_STORED, RSFD_PASS_RECOMPUTE, RSFD_PASS_SPLIT, RSFD_PASS_SPLIT_BFP};
  const int zcs[3] = {0, h->nz, (h->nz + 1) / 2};
  for (int kind : kinds) {
    if (kind == RSFD_PASS_SPLIT_BFP && resolve_kind(h->prec, kind) != kind) continue;
    if (is_split(kind)) {
      // the split pass: tile height and z-chunk
      const int tys[3] = {8, 4, 16};
      const int pfs[2] = {0, 3};
      for (int ty : tys) {
        if (ty > h->ny && ty != 4) continue;
        if (!tile_ok(h->prec, h->R, ty, kind, 1)) continue;
        for (int zc : zcs)
        for (int pf : pfs)
        for (int rb = 0; rb < (kind == RSFD_PASS_SPLIT_BFP ? 2 : 1); ++rb) {
          if (zc > 0 && zc < 8) continue;
          rsfd_solve_opts o = keep;
          o.pass_kind = kind;
          o.rows_per_thread = 0;
          o.tile_y = ty;
          o.z_chunk = zc;
          o.reg_budget = rb;
          o.tile_x = 0;
          o.slots = ncols;
          o.iters_per_sync = C;
          o.profile = 1;
          o.use_graphs = 0;
          o.prefetch = pf;
          cand.push_back(o);
        }
      }
      continue;
    }
    if (kind == RSFD_PASS_RECOMPUTE && h->n_atoms > 0) continue;
    const int rows_c[2] = {1, 2};
    for (int rows : rows_c) {
      if (kind == RSFD_PASS_RECOMPUTE && rows != 1) continue;
      const int tys[4] = {0, 8, 12, 16};
      for (int ty : tys) {
        if (kind == RSFD_PASS_RECOMPUTE && ty != 0) continue;
        const int tyv = ty > 0 ? ty : default_tile_y(h->prec, h->R, h->ny, kind, rows);
        if (ty > 0 && (ty == default_tile_y(h->prec, h->R, h->ny, kind, rows) || tyv > h->ny)) continue;
        const bool df1 = h->prec == RSFD_DF64 && kind == RSFD_PASS_STORED && rows == 1;
        // (register budget, tile width): 96 or 128 registers at width 32, and the 16-wide tile
        const int variants[3][2] = {{0, 32}, {1, 32}, {0, 16}};
        for (int vi = 0; vi < (df1 ? 3 : 1); ++vi) {
          const int budget = variants[vi][0], twx = variants[vi][1];
          if (twx == 16 && h->nx % 32 == 0) continue;   // the 16-wide tile only helps ragged widths
          if (!tile_ok(h->prec, h->R, tyv, kind, rows, budget, twx)) continue;
          for (int zc : zcs) {
            if (zc > 0 && zc < 8) continue;
            rsfd_solve_opts o = keep;
            o.pass_kind = kind;
            o.rows_per_thread = kind == RSFD_PASS_STORED ? rows : 0;
            o.tile_y = ty;
            o.z_chunk = zc;
            o.reg_budget = budget;
            o.tile_x = twx == 16 ? 16 : 0;
            o.slots = ncols;
            o.iters_per_sync = C;
            o.profile = 1;
            o.use_graphs = 0;
            o.prefetch = 0;
            cand.push_back(o);
          }
        }
      }
    }
  }
  double best_us = -1.0;
  rsfd_solve_opts best_o = keep;
  for (const rsfd_solve_opts& o : cand) {
    if (rsfd_set_solve_options(h, &o) != RSFD_OK) continue;
    const rsfd_status st = rsfd_shifted_cocg(h, cols.data(), ncols, energies, K, eta, 1e-30, maxit, RSFD_SEED_MID, 0,
                                             G0, info.data(), res.data());
    if (st != RSFD_OK && st != RSFD_ERR_NOT_CONVERGED) continue;
    const double its = (double)h->stats.slot_iterations;
    if (its <= 0) continue;
    const double us = (h->stats.ms_pass + h->stats.ms_shift) * 1e3 / its;
    if (best_us < 0 || us < best_us) {
      best_us = us;
      best_o = o;
    }
  }
  cudaFree(G0);
  if (best_us < 0) {
    h->opts = keep;
    return fail(h, RSFD_ERR_CUDA, "rsfd_autotune: no candidate ran");
  }
  best_o.profile = keep.profile;
  best_o.use_graphs = keep.use_graphs;
  if (!is_split(best_o.pass_kind)) best_o.prefetch = keep.prefetch;   // the split pass tunes its depth
  h->opts = best_o;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = std::make_pair(best_o, best_us);
  }
  if (best) *best = best_o;
  if (us_per_slot_iteration) *us_per_slot_iteration = best_us;
  return RSFD_OK;
}


// Several transition regions (each its own handle and stream) solved in one call: one host thread per
// region drives that region's iteration chunks (CUDA graphs) on the handle's own stream, so the
// regions' kernels run concurrently on the device and small regions fill the SMs that large ones
// leave idle.  The worst status is returned; each job's own status is stored in the job.
static rsfd_status rsfd_shifted_cocg_regions_impl(int32_t n, rsfd_region_solve* jobs) {
  if (n < 0 || (n > 0 && !jobs)) return fail(nullptr, RSFD_ERR_ARG, "rsfd_shifted_cocg_regions: bad job list");
  for (int i = 0; i < n; ++i) {
    if (!jobs[i].h) return fail(nullptr, RSFD_ERR_ARG, "rsfd_shifted_cocg_regions: NULL handle in job " + std::to_string(i));
    for (int j = 0; j < i; ++j)
      if (jobs[j].h == jobs[i].h)
        return fail(nullptr, RSFD_ERR_ARG, "rsfd_shifted_cocg_regions: a handle appears in two jobs");
  }
  auto run = [](rsfd_region_solve* q) {
    q->status = rsfd_shifted_cocg(q->h, q->cols, q->ncols, q->energies, q->K, q->eta, q->tol, q->maxit, q->seed_kind,
                                  q->seed_index, q->G0_bb, q->info, q->final_res);
  };
  std::vector<std::thread> th;
  th.reserve(n > 0 ? n - 1 : 0);
  try {
    for (int i = 1; i < n; ++i) th.emplace_back(run, &jobs[i]);
  } catch (...) {
    for (auto& t : th) t.join();
    return fail(nullptr, RSFD_ERR_ALLOC, "rsfd_shifted_cocg_regions: could not start a host thread");
  }
  if (n > 0) run(&jobs[0]);
  for (auto& t : th) t.join();
  rsfd_status worst = RSFD_OK;
  auto rank = [](rsfd_status st) {
    if (st == RSFD_OK) return 0;
    if (st == RSFD_ERR_NOT_CONVERGED) return 1;
    if (st == RSFD_ERR_BREAKDOWN) return 2;
    return 3;
  };
  for (int i = 0; i < n; ++i)
    if (rank(jobs[i].status) > rank(worst)) worst = jobs[i].status;
  if (rank(worst) == 3) {
    for (int i = 0; i < n; ++i)
      if (jobs[i].status == worst) {
        g_last_error = "region " + std::to_string(i) + ": " + jobs[i].h->err;
        break;
      }
  }
  return worst;
}

// Column sweep with checkpoints: blocks of `block` columns are solved one after another; each
// finished block's slice of G0_bb and its column outcomes go to <dir>/g0_block_<b>.bin (written to a
// temporary name, then renamed), and a block whose file exists and was computed from the same inputs
// is read back instead of solved.
struct SweepHeader {
  char magic[8];
  uint32_t version;
  int32_t K, nb, ncols, elem_bytes, reserved;
  uint64_t hash;
};

static uint64_t sweep_block_hash(const Handle* h, const int64_t* cols, int B, const double* energies, int K, double eta,
                                 double tol, int maxit, int seed_kind, int seed_index, int nb, size_t es) {
  uint64_t hv = h->in_hash;
  hv = fnv1a(hv, cols, (size_t)B * sizeof(int64_t));
  hv = fnv1a(hv, energies, (size_t)K * sizeof(double));
  const double dv[2] = {eta, tol};
  const int32_t iv[5] = {maxit, seed_kind, seed_index, nb, (int32_t)es};
  hv = fnv1a(hv, dv, sizeof(dv));
  hv = fnv1a(hv, iv, sizeof(iv));
  return hv;
}

static rsfd_status rsfd_shifted_cocg_sweep_impl(rsfd_handle h, const int64_t* cols, int32_t ncols, const double* energies,
                                    int32_t K, double eta, double tol, int32_t maxit, int32_t seed_kind,
                                    int32_t seed_index, int32_t block, const char* dir, void* G0_bb,
                                    rsfd_col_info* info, int32_t* blocks_resumed) {
  if (!h) return fail(nullptr, RSFD_ERR_ARG, "rsfd_shifted_cocg_sweep: NULL handle");
  if (!cols || ncols < 1 || !energies || K < 1 || block < 1 || !dir || !dir[0] || !info)
    return fail(h, RSFD_ERR_ARG, "rsfd_shifted_cocg_sweep: bad arguments");
  const size_t es = h->prec == RSFD_MIXED ? 8 : 16;
  const int nb = h->nr;
  const int nblk = (ncols + block - 1) / block;
  const int B0 = std::min(block, ncols);
  rsfd_status s;
  if ((s = ensure(h, h->sweep, (size_t)K * B0 * nb * es)) != RSFD_OK) return s;
  if (blocks_resumed) *blocks_resumed = 0;
  std::vector<unsigned char> host((size_t)K * B0 * nb * es);
  rsfd_status worst = RSFD_OK;
  for (int bi = 0; bi < nblk; ++bi) {
    const int c0 = bi * block, B = std::min(block, ncols - c0);
    const uint64_t hv = sweep_block_hash(h, cols + c0, B, energies, K, eta, tol, maxit, seed_kind, seed_index, nb, es);
    char name[64];
    snprintf(name, sizeof(name), "/g0_block_%06d.bin", bi);
    const std::string path = std::string(dir) + name;
    const size_t bytes = (size_t)K * B * nb * es;
    bool loaded = false;
    if (FILE* f = fopen(path.c_str(), "rb")) {
      SweepHeader hd;
      if (fread(&hd, sizeof(hd), 1, f) == 1 && memcmp(hd.magic, "RSFDG0BK", 8) == 0 && hd.version == 1 &&
          hd.K == K && hd.nb == nb && hd.ncols == B && hd.elem_bytes == (int32_t)es && hd.hash == hv &&
          fread(info + c0, sizeof(rsfd_col_info), B, f) == (size_t)B && fread(host.data(), 1, bytes, f) == bytes)
        loaded = true;
      fclose(f);
    }
    if (loaded) {
      if (G0_bb)
        RSFD_CK(h, cudaMemcpy2D((unsigned char*)G0_bb + (size_t)c0 * nb * es, (size_t)ncols * nb * es, host.data(),
                                (size_t)B * nb * es, (size_t)B * nb * es, K, cudaMemcpyHostToDevice));
      if (blocks_resumed) ++*blocks_resumed;
    } else {
      const rsfd_status st = rsfd_shifted_cocg(h, cols + c0, B, energies, K, eta, tol, maxit, seed_kind, seed_index,
                                               h->sweep.p, info + c0, nullptr);
      if (st != RSFD_OK && st != RSFD_ERR_NOT_CONVERGED && st != RSFD_ERR_BREAKDOWN) return st;
      if (G0_bb)
        RSFD_CK(h, cudaMemcpy2D((unsigned char*)G0_bb + (size_t)c0 * nb * es, (size_t)ncols * nb * es, h->sweep.p,
                                (size_t)B * nb * es, (size_t)B * nb * es, K, cudaMemcpyDeviceToDevice));
      RSFD_CK(h, cudaMemcpy(host.data(), h->sweep.p, bytes, cudaMemcpyDeviceToHost));
      SweepHeader hd;
      memset(&hd, 0, sizeof(hd));
      memcpy(hd.magic, "RSFDG0BK", 8);
      hd.version = 1;
      hd.K = K;
      hd.nb = nb;
      hd.ncols = B;
      hd.elem_bytes = (int32_t)es;
      hd.hash = hv;
      const std::string tmp = path + ".tmp";
      FILE* f = fopen(tmp.c_str(), "wb");
      if (!f) return fail(h, RSFD_ERR_ARG, "rsfd_shifted_cocg_sweep: cannot write " + tmp);
      const bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1 &&
                      fwrite(info + c0, sizeof(rsfd_col_info), B, f) == (size_t)B &&
                      fwrite(host.data(), 1, bytes, f) == bytes;
      if (fclose(f) != 0 || !ok || rename(tmp.c_str(), path.c_str()) != 0)
        return fail(h, RSFD_ERR_ARG, "rsfd_shifted_cocg_sweep: cannot write " + path);
    }
    for (int c = c0; c < c0 + B; ++c) {
      const rsfd_status cs = (rsfd_status)info[c].status;
      if (cs == RSFD_ERR_BREAKDOWN) worst = RSFD_ERR_BREAKDOWN;
      else if (cs == RSFD_ERR_NOT_CONVERGED && worst == RSFD_OK) worst = RSFD_ERR_NOT_CONVERGED;
    }
  }
  return worst;
}

static rsfd_status rsfd_lead_sigma_decimation_impl(rsfd_handle h, const double* V_left, const double* V_right,
                                       const double* energies, int32_t K, double eta, int32_t maxit, void* Sigma_L,
                                       void* Sigma_R, int32_t* iterations) {
  if (!h) return fail(nullptr, RSFD_ERR_ARG, "rsfd_lead_sigma_decimation: NULL handle");
  if (!energies || K < 1 || !(eta > 0) || maxit < 1 || !Sigma_L || !Sigma_R)
    return fail(h, RSFD_ERR_ARG, "rsfd_lead_sigma_decimation: bad arguments");
  if (h->nface != h->R)
    return fail(h, RSFD_ERR_ARG, "rsfd_lead_sigma_decimation: the handle's boundary slab must have fd_order/2 planes");
  const long long nl = (long long)h->R * h->nx * h->ny;
  for (const double* V : {V_left, V_right})
    if (V)
      for (long long i = 0; i < nl; ++i)
        if (!isfinite(V[i])) return fail(h, RSFD_ERR_ARG, "rsfd_lead_sigma_decimation: non-finite lead potential");
  int it = 0;
  rsfd_status s = lead_decimation_run(h, V_left, V_right, energies, K, eta, maxit, Sigma_L, Sigma_R, &it);
  if (iterations) *iterations = it;
  return s;
}

// Energies k0 .. k0 + kcount - 1 of a completed checkpointed sweep, all columns, read from the block
// files into a device buffer [kcount][ncols][nb]: the energy-chunked G0_bb of a sweep whose whole
// G0_bb does not fit in device memory.
static rsfd_status rsfd_sweep_load_energies_impl(rsfd_handle h, const int64_t* cols, int32_t ncols, const double* energies,
                                     int32_t K, double eta, double tol, int32_t maxit, int32_t seed_kind,
                                     int32_t seed_index, int32_t block, const char* dir, int32_t k0, int32_t kcount,
                                     void* G0_part) {
  if (!h) return fail(nullptr, RSFD_ERR_ARG, "rsfd_sweep_load_energies: NULL handle");
  if (!cols || ncols < 1 || !energies || K < 1 || block < 1 || !dir || !dir[0] || !G0_part || k0 < 0 || kcount < 1 ||
      k0 + kcount > K)
    return fail(h, RSFD_ERR_ARG, "rsfd_sweep_load_energies: bad arguments");
  const size_t es = h->prec == RSFD_MIXED ? 8 : 16;
  const int nb = h->nr;
  const int nblk = (ncols + block - 1) / block;
  std::vector<unsigned char> host((size_t)std::min(block, ncols) * nb * es);
  for (int bi = 0; bi < nblk; ++bi) {
    const int c0 = bi * block, B = std::min(block, ncols - c0);
    const uint64_t hv = sweep_block_hash(h, cols + c0, B, energies, K, eta, tol, maxit, seed_kind, seed_index, nb, es);
    char name[64];
    snprintf(name, sizeof(name), "/g0_block_%06d.bin", bi);
    const std::string path = std::string(dir) + name;
    FILE* f = fopen(path.c_str(), "rb");
    if (!f) return fail(h, RSFD_ERR_ARG, "rsfd_sweep_load_energies: missing " + path);
    SweepHeader hd;
    const bool ok = fread(&hd, sizeof(hd), 1, f) == 1 && memcmp(hd.magic, "RSFDG0BK", 8) == 0 && hd.version == 1 &&
                    hd.K == K && hd.nb == nb && hd.ncols == B && hd.elem_bytes == (int32_t)es && hd.hash == hv;
    if (!ok) {
      fclose(f);
      return fail(h, RSFD_ERR_ARG, "rsfd_sweep_load_energies: " + path + " was computed from other inputs");
    }
    const size_t slice = (size_t)B * nb * es;
    const long base = (long)sizeof(SweepHeader) + (long)B * (long)sizeof(rsfd_col_info);
    for (int k = k0; k < k0 + kcount; ++k) {
      if (fseek(f, base + (long)k * (long)slice, SEEK_SET) != 0 || fread(host.data(), 1, slice, f) != slice) {
        fclose(f);
        return fail(h, RSFD_ERR_ARG, "rsfd_sweep_load_energies: short read of " + path);
      }
      RSFD_CK(h, cudaMemcpy((unsigned char*)G0_part + ((size_t)(k - k0) * ncols + c0) * nb * es, host.data(), slice,
                            cudaMemcpyHostToDevice));
    }
    fclose(f);
  }
  return RSFD_OK;
}

// Entry points: the implementations above, behind a guard that turns a host-side C++ exception (a
// failed host allocation, above all) into a status code, so that none crosses the C ABI, and inside
// an NVTX range named after the entry point (setup, solve, Dyson, transmission, ... in a profile).
#define RSFD_GUARD(h, call)                                                              \
  rsfd::NvtxRange nvtx_range_(__func__);                                                 \
  try {                                                                                  \
    return call;                                                                         \
  } catch (const std::bad_alloc&) {                                                      \
    return fail((h), RSFD_ERR_ALLOC, "host allocation failed");                         \
  } catch (const std::exception& ex_) {                                                  \
    return fail((h), RSFD_ERR_CUDA, std::string("internal error: ") + ex_.what());       \
  } catch (...) {                                                                        \
    return fail((h), RSFD_ERR_CUDA, "internal error");                                   \
  }

rsfd_status rsfd_create(rsfd_handle* out, const int32_t grid[3], double hh, int32_t fd_order, int32_t n_face,
                        const double* V_loc, const rsfd_projectors* proj, int32_t precision, void* stream) {
  RSFD_GUARD(nullptr, rsfd_create_impl(out, grid, hh, fd_order, n_face, V_loc, proj, precision, stream));
}

rsfd_status rsfd_boundary_rows(rsfd_handle h, int32_t* nb, int64_t* rows) {
  RSFD_GUARD(h, rsfd_boundary_rows_impl(h, nb, rows));
}

rsfd_status rsfd_set_tracked_planes(rsfd_handle h, int32_t n, const int32_t* z) {
  RSFD_GUARD(h, rsfd_set_tracked_planes_impl(h, n, z));
}

rsfd_status rsfd_tracked_rows(rsfd_handle h, int32_t* nr, int64_t* rows) {
  RSFD_GUARD(h, rsfd_tracked_rows_impl(h, nr, rows));
}

rsfd_status rsfd_set_solve_options(rsfd_handle h, const rsfd_solve_opts* o) {
  RSFD_GUARD(h, rsfd_set_solve_options_impl(h, o));
}

rsfd_status rsfd_get_stats(rsfd_handle h, rsfd_stats* out) {
  RSFD_GUARD(h, rsfd_get_stats_impl(h, out));
}

rsfd_status rsfd_shifted_cocg(rsfd_handle h, const int64_t* cols, int32_t ncols, const double* energies, int32_t K,
                              double eta, double tol, int32_t maxit, int32_t seed_kind, int32_t seed_index,
                              void* G0_bb, rsfd_col_info* info, double* final_res) {
  RSFD_GUARD(h, rsfd_shifted_cocg_impl(h, cols, ncols, energies, K, nullptr, 0, eta, tol, maxit, seed_kind, seed_index, G0_bb, info, final_res));
}

rsfd_status rsfd_shifted_cocg_aux(rsfd_handle h, const int64_t* cols, int32_t ncols, const double* energies, int32_t K,
                                  const double* aux_energies, int32_t n_aux, double eta, double tol, int32_t maxit,
                                  int32_t seed_kind, int32_t seed_index, void* G0_bb, rsfd_col_info* info,
                                  double* final_res) {
  RSFD_GUARD(h, rsfd_shifted_cocg_impl(h, cols, ncols, energies, K, aux_energies, n_aux, eta, tol, maxit, seed_kind, seed_index, G0_bb, info, final_res));
}

rsfd_status rsfd_dyson_boundary(rsfd_handle h, const void* G0_bb, const void* Sigma_L, const void* Sigma_R,
                                int32_t K, void* G_bb, double* refine_residual) {
  RSFD_GUARD(h, rsfd_dyson_boundary_impl(h, G0_bb, Sigma_L, Sigma_R, K, G_bb, refine_residual));
}

rsfd_status rsfd_dyson_tracked(rsfd_handle h, const void* G0, const void* Sigma_L, const void* Sigma_R, int32_t K,
                               void* G, double* refine_residual) {
  RSFD_GUARD(h, rsfd_dyson_tracked_impl(h, G0, Sigma_L, Sigma_R, K, G, refine_residual));
}

rsfd_status rsfd_transmission(rsfd_handle h, const void* G_bb, const void* Sigma_L, const void* Sigma_R, int32_t K,
                              double* T) {
  RSFD_GUARD(h, rsfd_transmission_impl(h, G_bb, Sigma_L, Sigma_R, K, T));
}

rsfd_status rsfd_lead_sigma_uniform(int32_t Nx, int32_t Ny, double hh, int32_t fd_order, const double* energies,
                                    double eta, int32_t K, double* Sigma_L, double* Sigma_R) {
  RSFD_GUARD(nullptr, rsfd_lead_sigma_uniform_impl(Nx, Ny, hh, fd_order, energies, eta, K, Sigma_L, Sigma_R));
}

rsfd_status rsfd_autotune(rsfd_handle h, const double* energies, int32_t K, double eta, int32_t slots, int32_t iters,
                          rsfd_solve_opts* best, double* us_per_slot_iteration) {
  RSFD_GUARD(h, rsfd_autotune_impl(h, energies, K, eta, slots, iters, best, us_per_slot_iteration));
}

rsfd_status rsfd_shifted_cocg_regions(int32_t n, rsfd_region_solve* jobs) {
  RSFD_GUARD(nullptr, rsfd_shifted_cocg_regions_impl(n, jobs));
}

rsfd_status rsfd_shifted_cocg_sweep(rsfd_handle h, const int64_t* cols, int32_t ncols, const double* energies,
                                    int32_t K, double eta, double tol, int32_t maxit, int32_t seed_kind,
                                    int32_t seed_index, int32_t block, const char* dir, void* G0_bb,
                                    rsfd_col_info* info, int32_t* blocks_resumed) {
  RSFD_GUARD(h, rsfd_shifted_cocg_sweep_impl(h, cols, ncols, energies, K, eta, tol, maxit, seed_kind, seed_index, block, dir, G0_bb, info, blocks_resumed));
}

rsfd_status rsfd_lead_sigma_decimation(rsfd_handle h, const double* V_left, const double* V_right,
                                       const double* energies, int32_t K, double eta, int32_t maxit, void* Sigma_L,
                                       void* Sigma_R, int32_t* iterations) {
  RSFD_GUARD(h, rsfd_lead_sigma_decimation_impl(h, V_left, V_right, energies, K, eta, maxit, Sigma_L, Sigma_R, iterations));
}

rsfd_status rsfd_sweep_load_energies(rsfd_handle h, const int64_t* cols, int32_t ncols, const double* energies,
                                     int32_t K, double eta, double tol, int32_t maxit, int32_t seed_kind,
                                     int32_t seed_index, int32_t block, const char* dir, int32_t k0, int32_t kcount,
                                     void* G0_part) {
  RSFD_GUARD(h, rsfd_sweep_load_energies_impl(h, cols, ncols, energies, K, eta, tol, maxit, seed_kind, seed_index, block, dir, k0, kcount, G0_part));
}

rsfd_status rsfd_dyson_boundary_noalloc(int32_t nb, int32_t K, const void* G0_bb, const void* Sigma_L,
                                        const void* Sigma_R, void* G_bb, double* refine_residual, void* stream) {
  RSFD_GUARD(nullptr, rsfd::dyson_noalloc_run(nb, K, G0_bb, Sigma_L, Sigma_R, G_bb, refine_residual, stream));
}
}  // extern "C"
