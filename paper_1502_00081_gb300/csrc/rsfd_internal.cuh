// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/rsfd.h"

namespace rsfd {

// NVTX range over a scope (a named interval in an attached profiler's timeline; no effect otherwise)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------------------------------------
// complex helpers: float2 / double2 with interleaved (re, im)
// ---------------------------------------------------------------------------------------------
template <typename T> struct cplx_of;
template <> struct cplx_of<float> { typedef float2 type; };
template <> struct cplx_of<double> { typedef double2 type; };

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  // Smith's algorithm for a / b
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, d = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  } else {
    double r = b.x / b.y, d = b.y + b.x * r;
    return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
  }
}

// ---------------------------------------------------------------------------------------------
// solver state in device memory
// ---------------------------------------------------------------------------------------------
enum SlotStatus : int32_t {
  SLOT_EMPTY = -1,
  SLOT_RUNNING = 0,
  SLOT_DONE = 1,      // every energy converged
  SLOT_MAXIT = 2,
  SLOT_BREAKDOWN = 3,
};

// One in-flight right-hand side (a "slot").  Written by the scalar step of the pass kernel,
// read by every CTA of the next pass and by the shift-update kernel.
struct __align__(16) SlotState {
  int32_t col;        // output column index c (G0_bb[:, :, c]); -1 when empty
  int32_t n;          // index of the residual the next pass produces (r_n)
  int32_t seed;       // current seed energy index s
  int32_t status;     // SlotStatus
  int32_t switches;   // seed switches so far
  int32_t k4_n;       // iteration whose shift update is pending (-1 = none)
  int32_t iters;      // seed iterations at exit
  int32_t hcnt;       // entries recorded in the shift-update history since the last collapse
  double2 a1;         // next pass: r_n = a1 r_{n-1} + a2 r_{n-2} + aA (A r_{n-1})
  double2 a2;
  double2 aA;
  double2 Zs;         // seed energy used by the next pass (A = Zs - H)
  double2 alpha_prev; // alpha_{n-1}
  double2 rr_prev;    // (r_{n-1}, r_{n-1}) in the current seed's normalisation
  double2 carry;      // factor that brings the stored r_{n-1} to the current seed's normalisation
  // block-floating-point split pass (RSFD_PASS_SPLIT_BFP): the next combine rounds the leading
  // parts of r_n to multiples of q; mr_prev is the largest leading-part component of the stored
  // r_{n-1} (the r_{n-2} of the next combine)
  double q;
  double mr_prev;
};

// Per (slot, energy) scalars (FP64).
struct __align__(16) ShiftState {
  double2 pi_n;       // pi_n^(s,i)
  double2 pi_nm1;     // pi_{n-1}^(s,i)
  double2 alpha_prev; // alpha_{n-1}^(i)
  double2 cr;         // shift update coefficients of the pending iteration:
  double2 cb;         //   p <- cr * r_n + cb * p ;  x <- x + ca * p
  double2 ca;
  double res;         // last residual ||r_n|| / |pi_n|
  int32_t active;     // 1 while not converged
  int32_t conv_iter;  // iteration at which it converged (-1 = not yet)
};

// Coefficients of one iteration of the shifted update of one energy:
//   p <- cr r_n + cb p ;  x <- x + ca p
struct ShiftCoef {
  double2 cr, cb, ca;
};

constexpr int kMaxHist = 64;   // longest shift-update history (iterations per collapse)

struct SolveDims {
  int nx, ny, nz;
  int nxp;            // padded row length of the internal vectors (multiple of 4)
  long long N;
  int R;              // stencil reach (fd_order / 2)
  int nface;          // boundary planes per side
  int nb;             // recorded rows per column: the boundary rows, then the tracked planes
  int K;              // shifts carried by the scalar recurrences: the energies, then auxiliary seed energies
  int kreq;           // energies of the set (written out, required for convergence): the first kreq
  int W;              // slots
  int tile_y;         // stencil tile height (y); the tile width in x is fixed by the kernel
  int depth;          // TMA prefetch depth of the pass kernel
  int tiles_x, tiles_y, zchunk, nzchunks, ctas_per_slot;
  int ctas_c;         // split pass: CTAs per slot of the combine kernel (0 for the other forms)
  int npart;          // partial-sum entries per slot: ctas_per_slot + ctas_c
  int ncols;
  int ntrack;         // interior planes recorded after the boundary planes
  int track[16];      // their z indices (rows 2 nface Nx Ny + e Nx Ny ...)
  int kind;           // RSFD_PASS_RECOMPUTE, RSFD_PASS_STORED, RSFD_PASS_SPLIT or RSFD_PASS_SPLIT_BFP
  int nvec;           // Krylov vectors per slot in rbuf: 3 (r ring) or 5 (r ring + A r pair)
  int rows;           // stored-product pass: tile rows per thread (1, 2 or 4)
  int regs;           // register budget of the one-row double-float pass (0, 1)
  int tile_x;         // stored-product pass tile width in x: 32, or 16 (one-row double-float pass)
  int wait_cap;       // attempts of the passes' first TMA waits: 0 = default, < 0 = none (test)
  double brk_tol;     // quasi-null threshold of (r, r) relative to ||r||^2
};

struct Handle;   // defined in rsfd_api.cu

// Kernel launchers implemented in cocg_kernels.cu.
struct SolverBuffers {
  void* rbuf;             // [W][nvec][Nz][Ny][Nxp] vector elements
  const void* V;          // [Nz][Ny][Nxp] potential
  void* xbuf;             // [W][K][nb] boundary rows of x^(i)
  void* pbuf;             // [W][K][nb] boundary rows of p^(i)
  void* rhist;            // [W][hist_len][nb] boundary rows of r_n (hi parts)
  ShiftCoef* coef;        // [W][K][hist_len]
  void* cwbuf;            // [W][K][2][hist_len] collapse weights W_x, W_p (H type)
  double2* cebuf;         // [W][K][2] collapse factors e_x, e_p
  int* error_flag;        // set by a kernel whose bounded wait expired
  const CUtensorMap* tmR; // TMA map of rbuf
  const CUtensorMap* tmV; // TMA map of the potential
  const CUtensorMap* tmVs;// TMA map of the scaled potential s V (double-float handles)
  const void* Vs;         // [Nz][Ny][Nxp] s V as (hi, lo) floats (double-float handles)
  double uscale;          // s: the block-floating-point split pass stores s A r (integer neighbour weights)
  SlotState* slots;       // [W]
  ShiftState* shifts;     // [W][K]
  double* partials;       // [W][ctas_per_slot][8]
  unsigned int* tickets;  // [W]
  double2* Z;             // [K] complex energies
  int64_t* brow;          // [nb] boundary rows
  void* G0;               // output base
  int* init_list;         // [W][2]: slot, column c
  long long* init_grid;   // [W]: grid index j of the new column
  unsigned long long* counters;  // [0] active (slot, energy) updates, [1] slot iterations
  // nonlocal projectors (n_atoms == 0: none), V_nl r = sum_a E_a c_a p_a with c_a = h^3 p_a^T r
  int n_atoms;
  int n_supp;             // grid points in the union of the projector supports
  const int* a_ptr;       // [n_atoms + 1] atom-major CSR
  const long long* a_idx; // [nnz] padded vector index of each entry
  const void* a_val;      // [nnz] projector values (potential element type)
  const double* a_E;      // [n_atoms] projector energies
  const int* t_ptr;       // [n_supp + 1] point-major CSR of the same entries
  const long long* t_pidx;// [n_supp] padded vector index of each support point
  const int* t_atom;      // [nnz] atom of each point-major entry
  const void* t_val;      // [nnz] its projector value
  const double* a_pmax;   // [n_atoms] largest |projector value| of each atom
  int proj_overlap;       // largest number of atoms at one support point
  double h3;
  double2* pw;            // [W][n_atoms] -E_a c_a of the last pass (double-float handles: as a (hi, lo) float pair)
  double2* pcorr;         // [W][n_atoms] E_a c_a^2 / h^3
  double* pdots;          // [W][8] (r,r), (r, u_loc), ||r||^2 of the last pass
  unsigned int* ptickets; // [W]
};

struct StencilCoef {
  double hd;        // diagonal kinetic coefficient of H
  double hk[3];     // H couplings to neighbours at distance 1..R along each axis
};

struct PassConfig {
  int tile_x, tile_y;
};

// Launch one pass (stencil + seed update + dots + scalar step) over all slots; for the split pass
// an optional event is recorded between its combine and stencil launches (profiling).
cudaError_t launch_pass(int prec, const SolveDims& d, const SolverBuffers& b, const StencilCoef& c, double tol,
                        int maxit, int hist_len, cudaStream_t st, cudaEvent_t mid = nullptr, bool mid_external = false);
// Nonlocal projector term after a pass (stored-product form only): projections c_a = h^3 p_a^T r_n,
// the corrected (r_n, A r_n) and the FP64 scalar step, then u_n -= sum_a E_a c_a p_a.
cudaError_t launch_proj(int prec, const SolveDims& d, const SolverBuffers& b, const StencilCoef& c, double tol,
                        int maxit, int hist_len, cudaStream_t st);
// Apply the collapsed shift update of the recorded history of every slot, then clear the history.
cudaError_t launch_chunk(int prec, const SolveDims& d, const SolverBuffers& b, int hist_len, cudaStream_t st);
// Initialise n_init slots listed in b.init_list / b.init_grid.
cudaError_t launch_slot_init(int prec, const SolveDims& d, const SolverBuffers& b, int n_init, int seed0,
                             cudaStream_t st);
// Copy x_b of the n_out (slot, column) pairs listed in b.init_list into G0_bb.
cudaError_t launch_writeout(int prec, const SolveDims& d, const SolverBuffers& b, void* G0, int n_out,
                            cudaStream_t st);
size_t vec_elem_bytes(int prec);
size_t pot_elem_bytes(int prec);
size_t hist_elem_bytes(int prec);
size_t pass_smem(int prec, int R, int tile_y, int depth);
size_t passu_smem(int prec, int R, int tile_y, int depth, int tile_x);
int passu_threads(int rows, int R, int tile_y, int tile_x);
int passu_max_threads(int rows, int budget);
int passu_box_x(int tile_x);
int passu_box_off();
int pass_max_depth();
int split_threads(int tile_y);
size_t split_smem(int prec, int R, int tile_y, int depth);
int split_combine_ctas(int nz, int W, int sms);
int pass_box_x();
int pass_box_off();
int pass_max_threads(int prec);
int pass_tile_x(int R);
cudaError_t kernels_init();
// the pass kernel's warp-shuffle reductions need whole warps: (32 + 4R) * (tile_y + 4R) % 32 == 0
int pass_threads(int R, int tile_y);

// Handle services used by other translation units (rsfd_api.cu).
rsfd_status handle_ensure(Handle* h, int idx, size_t bytes, void** out);   // workspace slot idx < 8
cudaStream_t handle_stream(Handle* h);
int handle_prec(Handle* h);
int handle_nb(Handle* h);
rsfd_status handle_fail(Handle* h, rsfd_status s, const std::string& msg);
rsfd_status handle_begin(Handle* h);
rsfd_status handle_end(Handle* h);

int handle_nx(Handle* h);
int handle_ny(Handle* h);
int handle_fd_order(Handle* h);
double handle_h(Handle* h);
int handle_dyson_kind(Handle* h);     // resolved: RSFD_DYSON_FP64 or RSFD_DYSON_TC
int handle_dyson_refine(Handle* h);   // FP64 refinement steps of the Dyson solve
int handle_dyson_cols(Handle* h);     // 0: every column of G_bb; 1: the left slab's columns only

// Tensor-core building blocks of the Dyson step (tc_gemm.cu).  err: device flag set when a bounded
// wait of the GEMM kernel expires.
cudaError_t cgemm_tf32x3(cudaStream_t st, int batch, int m, int n, int k, float2 alpha, const float2* A, int lda,
                         long long sA, const float2* B, int ldb, long long sB, float beta, float2* C, int ldc,
                         long long sC, int* err);
cudaError_t getrf_f32_tc(cudaStream_t st, float2* M, int nb, int K, int* piv, int* info, int* err);
cudaError_t getrs_f32_tc(cudaStream_t st, const float2* LU, const int* piv, int nb, int K, const double2* B, int nrhs,
                         float2* X, int* perm, int* err);
cudaError_t getrs_f32_tc(cudaStream_t st, const float2* LU, const int* piv, int nb, int K, const float2* B, int nrhs,
                         float2* X, int* perm, int* err);
int tc_panel();

// Dyson / transmission launchers (dyson.cu).
rsfd_status dyson_run(Handle* h, const void* G0, const void* SL, const void* SR, int K, void* G, double* refres);
rsfd_status dyson_tracked_run(Handle* h, int nr, const void* G0, const void* SL, const void* SR, int K, void* G,
                              double* refres);
rsfd_status transmission_run(Handle* h, const void* G, const void* SL, const void* SR, int K, double* T);
rsfd_status lead_decimation_run(Handle* h, const double* VL, const double* VR, const double* E, int K, double eta,
                                int maxit, void* SL, void* SR, int* iters);
rsfd_status dyson_noalloc_run(int32_t nb, int32_t K, const void* G0_bb, const void* Sigma_L, const void* Sigma_R,
                              void* G_bb, double* refine_residual, void* stream);

// Host lead self-energy (lead_sigma.cpp).
rsfd_status lead_sigma_uniform(int nx, int ny, double h, int fd_order, const double* E, double eta, int K,
                               double* SL, double* SR, std::string* err);

}  // namespace rsfd
