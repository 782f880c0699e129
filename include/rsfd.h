/*
 * rsfd.h -- C ABI of the GB300 shifted-COCG / Dyson transport library.
 *
 * The library computes, for a transition region discretised on a real-space
 * finite-difference (RSFD) grid,
 *
 *   1. the unperturbed boundary Green's function  G0_bb(Z_k) = [(Z_k - H_T)^{-1}]_{b,cols}
 *      for every complex energy Z_k = E_k + i*eta and every right-hand side e_j,
 *      by the shifted COCG method with seed switching (paper: Sec. III B, Eq. GF4,
 *      Appendix Eqs. Eq ... seedswitch);
 *   2. the perturbed boundary Green's function G_bb from G0_bb and the lead
 *      self-energies through the exact OBM/Dyson relation (Eq. sec3-01a,
 *      Eqs. sec3-02 ... sec3-06);
 *   3. the Fisher-Lee transmission T(E) (Eq. TF);
 *   4. the lead self-energies those steps take (Eqs. self-energy, surface green's function):
 *      closed form for uniform leads on the host, decimation for leads with a layer potential
 *      on the GPU.
 * Around them: a launch-option autotuner, several regions in one call, checkpointed column
 * sweeps with energy-chunked read-back, interior diagonal blocks (DOS), the Dyson step's
 * tensor-core GEMM, and an allocation-free Dyson entry point.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid: Nx x Ny x Nz points, spacing h (bohr), z = transport direction.  A point
 *   (x, y, z) has linear index (z*Ny + y)*Nx + x.  H_T = -1/2 nabla^2 + V_loc
 *   (+ nonlocal projectors) with central finite differences of order 2 (7-point)
 *   or 4 (13-point) and zero ghosts outside the box on all six faces (the leads
 *   enter only through the self-energies).  Hartree atomic units.
 * Boundary row set b: the n_face outermost z-planes on each side, in increasing
 *   z, each plane x fastest; nb = 2*n_face*Nx*Ny.  The first half of b is the
 *   left slab, the second half the right slab; ns = nb/2.
 * Complex numbers: interleaved (re, im).  "c64" = 2 x float, "c128" = 2 x double.
 *   The handle's precision picks the element type of G0_bb / G_bb: c128 for
 *   RSFD_FP64 and RSFD_DF64, c64 for RSFD_MIXED.
 * Matrices: column-major per energy.  G0_bb is [K][ncols][nb]: element
 *   (k, row r, column c) sits at k*nb*ncols + c*nb + r.  Self-energies are
 *   [K][ns][ns] c128 with element (k, a, c) at k*ns*ns + c*ns + a.
 * Memory ownership: the caller owns every input and output buffer; "device"
 *   buffers must be device memory of the current CUDA device, "host" buffers
 *   host memory.  The handle owns its internal work buffers (allocated lazily,
 *   grown on demand, freed by rsfd_destroy).
 * Streams: every device operation is issued on the stream given to rsfd_create
 *   (a cudaStream_t passed as void*; NULL = legacy default stream).  Calls that
 *   return host results synchronise that stream before returning.
 * Errors: no C++ exception crosses this ABI.  Each call returns an rsfd_status;
 *   the message of the last failure is available from rsfd_last_error().  A
 *   CUDA error inside a call returns RSFD_ERR_CUDA.  Per-column solver outcomes
 *   (not converged, breakdown) are reported in rsfd_col_info and the call
 *   returns the worst of them.
 * Thread safety: a handle may be used by one host thread at a time.
 */
#ifndef RSFD_H
#define RSFD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rsfd_handle_s* rsfd_handle;

typedef enum {
  RSFD_OK = 0,
  RSFD_ERR_ARG = 1,           /* invalid argument (message says which) */
  RSFD_ERR_ALLOC = 2,         /* device or host allocation failed */
  RSFD_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  RSFD_ERR_NOT_CONVERGED = 4, /* some column hit maxit before every energy converged */
  RSFD_ERR_BREAKDOWN = 5,     /* COCG breakdown: (r, r) quasi-null while r != 0 */
  RSFD_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
  RSFD_ERR_UNSUPPORTED = 7    /* valid request that this build does not implement */
} rsfd_status;

/* Arithmetic of the shifted COCG:
 *   RSFD_FP64  complex128 Krylov vectors and FP64 arithmetic throughout.
 *   RSFD_MIXED complex64 Krylov vectors and SpMV (FP32 arithmetic), FP64 scalar recurrences and
 *              FP64 reductions (per-thread partial sums Kahan-compensated in FP32).
 *   RSFD_DF64  "double-float" Krylov vectors (each component an unevaluated sum of two floats,
 *              about 48 significant bits) with error-free FP32 arithmetic in the SpMV and the
 *              seed update, FP64 scalars.  Accuracy close to RSFD_FP64 at FP32-pipe speed. */
typedef enum { RSFD_FP64 = 0, RSFD_MIXED = 1, RSFD_DF64 = 2 } rsfd_precision;

/* Initial seed of the shifted COCG (Appendix; Sec. III C starts from the Fermi energy). */
typedef enum {
  RSFD_SEED_MID = 0,   /* energy index K/2 */
  RSFD_SEED_FIRST = 1, /* energy index 0 */
  RSFD_SEED_INDEX = 2, /* energy index seed_index */
  RSFD_SEED_AUX = 3    /* auxiliary energy seed_index of rsfd_shifted_cocg_aux (outside the set) */
} rsfd_seed_kind;

/* Separable nonlocal projectors, one per atom (Sec. II A mentions nonlocal
 * pseudopotentials as an extension): V_nl psi = sum_a E_a p_a (p_a^T psi) h^3.
 * CSR over atoms; all arrays are host memory, copied by rsfd_create. */
typedef struct {
  int32_t n_atoms;
  const int64_t* ptr; /* [n_atoms + 1] */
  const int64_t* idx; /* [nnz] linear grid indices */
  const double* val;  /* [nnz] projector values p_a(r_j) */
  const double* E;    /* [n_atoms] projector energies (Hartree) */
} rsfd_projectors;

/* Outcome of one right-hand side column of rsfd_shifted_cocg. */
typedef struct {
  int32_t iters;      /* seed iterations = applications of H_T */
  int32_t switches;   /* seed switches (Eq. seedswitch) */
  int32_t status;     /* RSFD_OK, RSFD_ERR_NOT_CONVERGED or RSFD_ERR_BREAKDOWN */
  int32_t final_seed; /* energy index of the seed when the column finished */
} rsfd_col_info;

/* Form of the seed iteration's pass (rsfd_solve_opts.pass_kind). */
typedef enum {
  RSFD_PASS_AUTO = 0,      /* RSFD_PASS_STORED when the options are not tuned; rsfd_autotune times every form
                              (on the 64^2 x 128 workload it picks RSFD_PASS_SPLIT_BFP for double-float) */
  RSFD_PASS_RECOMPUTE = 1, /* three vectors per iteration (r_{n-1}, r_{n-2} in, r_n out); A r_{n-1} is
                              recomputed on the tile plus halo and A r_n again for the dot products */
  RSFD_PASS_STORED = 2,    /* five vectors per iteration (r_{n-1}, r_{n-2}, A r_{n-1} in; r_n, A r_n out);
                              one stencil application per grid point */
  RSFD_PASS_SPLIT = 3,     /* the stored-product iteration as two launches: a pointwise combine (r_n from
                              r_{n-1}, r_{n-2}, A r_{n-1}; four vectors) and a stencil (A r_n from r_n; two
                              vectors plus its halo); one row per thread, tile width 32, tile_y <= 16 */
  RSFD_PASS_SPLIT_BFP = 4  /* double-float handles: RSFD_PASS_SPLIT with the leading
                              parts of r_n rounded to a per-column, per-iteration quantum q (block floating
                              point, q chosen from a bound on |r_n| so that every leading part is at most
                              2^21 q) and the product stored as s A r
                              with s = 24 h^2 (4th order) or 2 h^2 (2nd order), which makes the neighbour
                              weights the integers 16, -1 (or 1): the stencil's neighbour sums of leading
                              parts are then exact FP32 additions.  The iterates agree with RSFD_PASS_SPLIT
                              to double-float rounding (about 2^-45 of the bound on |r_n|).  With
                              projectors the bound adds (atoms per support point) x max_a |s E_a c_a|
                              max|p_a| for the projector term.  FP64 and complex64 handles run
                              RSFD_PASS_SPLIT */
} rsfd_pass_kind;

/* Form of the Dyson solve (rsfd_solve_opts.dyson_kind). */
typedef enum {
  RSFD_DYSON_AUTO = 0, /* RSFD_DYSON_TC for double-float and complex64 handles, RSFD_DYSON_FP64 for FP64 handles */
  RSFD_DYSON_FP64 = 1, /* LU, triangular solves and refinement in FP64 on the CUDA cores */
  RSFD_DYSON_TC = 2    /* LU and triangular solves in FP32 with their O(nb^3) updates on the tensor cores
                          (3xTF32, rsfd_cgemm_tf32x3), FP64 residuals and corrections (iterative refinement) */
} rsfd_dyson_kind;

/* Launch options of the solver; zero fields mean "choose automatically". */
typedef struct {
  int32_t slots;          /* columns iterated together (RHS block width) */
  int32_t iters_per_sync; /* iterations per CUDA-graph replay between host checks; also the number of
                             iterations collapsed into one shift update (<= 64) */
  int32_t tile_y;         /* stencil tile height in y; RSFD_ERR_ARG when the pass's CTA would exceed its
                             thread limit or 216 KB of shared memory */
  int32_t z_chunk;        /* planes per CTA along z */
  int32_t use_graphs;     /* 1 = capture iteration chunks in CUDA graphs (default), -1 = plain launches */
  int32_t profile;        /* 1 = time every kernel launch with CUDA events on the launching stream
                             (event nodes inside the CUDA graph); results in rsfd_get_stats */
  int32_t pass_kind;      /* rsfd_pass_kind */
  int32_t prefetch;       /* z-planes of input the pass keeps in flight (TMA), 1..7 */
  int32_t rows_per_thread;/* RSFD_PASS_STORED: tile rows per thread, 1, 2 or 4 (tile_y must be a multiple) */
  int32_t dyson_kind;     /* rsfd_dyson_kind of rsfd_dyson_boundary */
  int32_t dyson_refine;   /* FP64 refinement steps of rsfd_dyson_boundary (0 = 2 for FP64 handles, 1 for
                             double-float and complex64 handles; at most 8) */
  int32_t reg_budget;     /* RSFD_PASS_STORED, double-float, one row per thread: registers per thread of
                             the pass, 0 = at most 96 (CTAs of <= 640 threads; two CTAs of <= 320 threads
                             per SM), 1 = at most 128 (CTAs of <= 512 threads, tile_y <= 14, one CTA per
                             SM, no register spills); RSFD_PASS_SPLIT_BFP: the stencil launch keeps 0 = at
                             most 128 / 85 registers (one 512-thread or three 256-thread CTAs per SM) or
                             1 = at most 64 (two 512-thread or four 256-thread CTAs per SM); other passes
                             ignore it */
  int32_t tile_x;         /* RSFD_PASS_STORED, double-float, one row per thread: tile width in x, 0 or 32
                             (one tile row per warp) or 16 (two tile rows per warp; less idle work when Nx
                             is an odd multiple of 16, e.g. 48 or 80); tile_y must be even */
  int32_t wait_cap;       /* attempts of a pass's bounded wait for its TMA transfers before the wait is
                             declared lost (each attempt sleeps up to 1 ms): 0 = 4096; -1 = none, so every
                             CTA's first wait expires at once (a test of the RSFD_ERR_TIMEOUT path: the CTA
                             still drains its issued transfers with the full cap before it returns) */
  int32_t dyson_cols;     /* columns of G_bb rsfd_dyson_boundary solves: 0 = all nb; 1 = the left slab's nb/2
                             only (solve, refinement and residual on half the right-hand sides), the
                             block rsfd_transmission reads (G_RL); the other columns are set to zero */
  double breakdown_tol;   /* quasi-null test of the seed's (r_n, r_n): breakdown when |(r,r)| <= this times
                             ||r||^2 (or <= 1e-300); 0 = 1e-28.  A large value makes every column report
                             RSFD_ERR_BREAKDOWN (a test of that path) */
} rsfd_solve_opts;

/* Counters of the last rsfd_shifted_cocg call. */
typedef struct {
  double ms_total;            /* wall time of the call on the device stream (events) */
  double ms_pass;             /* summed duration of stencil/seed-update launches (profile = 1) */
  double ms_shift;            /* summed duration of the collapsed shift-update launches (profile = 1) */
  int64_t n_pass;             /* stencil/seed-update launches (two per iteration for the split passes) */
  int64_t n_shift;            /* collapsed shift-update launches (the apply kernel) */
  int64_t n_other;            /* other kernel launches (collapse coefficients, history reset, projector
                                 terms, slot set-up, write-out) */
  int64_t slot_iterations;    /* sum over columns of seed iterations */
  int64_t shift_updates;      /* recorded (column, energy, iteration) updates applied */
  int64_t shift_slot_chunks;  /* (column, collapse) pairs: each reads and writes x_b, p_b of K energies once */
  int32_t slots;              /* columns in flight that were used */
  int32_t iters_per_sync;
  double ms_combine;          /* split passes with profile = 1: the combine launches' part of ms_pass */
} rsfd_stats;

/* Create a handle for one transition region (Sec. II A, Eq. sabun1).
 *   grid[3]   = {Nx, Ny, Nz}, each >= 1 (host).
 *   h         > 0, grid spacing.
 *   fd_order  = 2 or 4.
 *   n_face    = planes per side in the boundary row set b, 1 <= n_face <= Nz/2;
 *               0 selects fd_order/2 (the planes the lead couples to).
 *   V_loc     = host [N] local potential, linear grid order.
 *   proj      = NULL or the nonlocal projectors (host arrays, copied; entries of one atom at distinct
 *               grid points).  With projectors the solver uses a pass that stores A r (the
 *               stored-product pass or a split pass; RSFD_PASS_RECOMPUTE becomes RSFD_PASS_STORED):
 *               after each pass a projection kernel forms c_a = h^3 p_a^T r_n, corrects (r_n, A r_n)
 *               and runs the scalar step, and a scatter kernel adds -sum_a E_a c_a p_a to A r_n.
 *   precision = RSFD_FP64, RSFD_MIXED or RSFD_DF64.
 *   stream    = cudaStream_t for every device operation of this handle.
 * Returns RSFD_ERR_ARG on invalid sizes, RSFD_ERR_ALLOC / RSFD_ERR_CUDA on
 * device failures; *out is NULL unless RSFD_OK. */
rsfd_status rsfd_create(rsfd_handle* out, const int32_t grid[3], double h, int32_t fd_order, int32_t n_face,
                        const double* V_loc, const rsfd_projectors* proj, int32_t precision, void* stream);

/* The boundary row set b (linear grid indices).  *nb receives its size; rows may
 * be NULL (size query) or a host array of at least *nb entries. */
rsfd_status rsfd_boundary_rows(rsfd_handle h, int32_t* nb, int64_t* rows);

/* Interior planes whose rows the solver records next to b, for the diagonal blocks G_T(z_l, z_l)
 * that the density of states needs (Sec. III B, discussion after Eq. sec3-06).  After this call
 * rsfd_shifted_cocg writes, for every column, the nr = nb + n*Nx*Ny recorded rows: b first, then
 * plane z[0], ..., plane z[n-1] (each plane in x-fastest order; rsfd_tracked_rows lists them).
 *   n  0 <= n <= RSFD_MAX_TRACKED_PLANES (0 restores nr = nb).
 *   z  host [n] distinct interior planes, n_face <= z[i] < Nz - n_face.
 * RSFD_ERR_ARG otherwise (the previous setting is kept). */
#define RSFD_MAX_TRACKED_PLANES 16
rsfd_status rsfd_set_tracked_planes(rsfd_handle h, int32_t n, const int32_t* z);

/* The recorded row set (b, then the tracked planes); *nr receives its size, rows may be NULL
 * (size query) or a host array of at least *nr entries. */
rsfd_status rsfd_tracked_rows(rsfd_handle h, int32_t* nr, int64_t* rows);

/* Set launch options for later solves (NULL restores the defaults). */
rsfd_status rsfd_set_solve_options(rsfd_handle h, const rsfd_solve_opts* opts);

/* Shifted COCG with seed switching (Sec. III B; Appendix):
 *   (Z_k - H_T) x^(k) = e_j  for k < K and every column j in cols,
 * keeping only the rows b of every x^(k):  G0_bb[k][:, c] = x^(k)_b for j = cols[c].
 *   cols       host [ncols] linear grid indices of the unit right-hand sides.
 *   energies   host [K] real parts E_k; Z_k = E_k + i*eta, eta > 0.
 *   tol        convergence threshold on ||r^(k)||_2 / ||e_j||_2 for every k.
 *   maxit      iteration cap per column (>= 1).
 *   seed_kind  rsfd_seed_kind; seed_index used with RSFD_SEED_INDEX.
 *   G0_bb      device output [K][ncols][nr], c64 or c128 per the handle's precision; nr = nb unless
 *              interior planes are tracked (rsfd_set_tracked_planes).
 *   info       host output [ncols] (nullable).
 *   final_res  host output [ncols][K] residual of each energy at exit (nullable).
 * Synchronises the handle's stream.  Returns RSFD_OK when every column
 * converged, else the worst per-column status. */
rsfd_status rsfd_shifted_cocg(rsfd_handle h, const int64_t* cols, int32_t ncols, const double* energies, int32_t K,
                              double eta, double tol, int32_t maxit, int32_t seed_kind, int32_t seed_index,
                              void* G0_bb, rsfd_col_info* info, double* final_res);

/* Shifted COCG with seed switching to energies outside the set (Appendix: the extension of Eq.
 * seedswitch to an arbitrary energy point, which the paper cites from its Ref. ss).  As
 * rsfd_shifted_cocg, plus n_aux auxiliary energies (host [n_aux], Z_a = aux_energies[a] + i*eta)
 * that are carried as shifts of their own through the scalar recurrences (Eqs. spi, salpha,
 * sbeta) so that Eq. seedswitch applies to them unchanged: one of them can be the first seed
 * (seed_kind RSFD_SEED_AUX, seed_index < n_aux), and at every seed switch they are candidates
 * like the unconverged energies of the set (largest residual wins; the set comes first on ties).
 * Nothing of their solutions is output and a column stops when the K energies of the set have
 * converged.  G0_bb, info and final_res cover the K energies only; info.final_seed >= K names
 * auxiliary energy final_seed - K.  n_aux = 0 is rsfd_shifted_cocg. */
rsfd_status rsfd_shifted_cocg_aux(rsfd_handle h, const int64_t* cols, int32_t ncols, const double* energies, int32_t K,
                                  const double* aux_energies, int32_t n_aux, double eta, double tol, int32_t maxit,
                                  int32_t seed_kind, int32_t seed_index, void* G0_bb, rsfd_col_info* info,
                                  double* final_res);

/* Launch-option autotuner for rsfd_shifted_cocg (the seed iteration and shift update of Sec. III B and
 * the Appendix; the paper has no launch shapes, so the tuned quantities are this library's own):
 * times short solves of `iters` seed iterations (at least two collapse lengths) of the handle's first
 * `slots` boundary columns at the given energies for every candidate pass form, tile height, rows per
 * thread and z-chunk, at the RHS block width `slots` and the handle's collapse length, and keeps the
 * candidate with the least device time per (column, iteration).  The result is applied to the handle
 * (rsfd_set_solve_options) and cached for the process by (grid, order, precision, projectors, K,
 * slots); the Dyson options and the profile flag are kept.
 *   energies host [K];  eta > 0;  slots >= 1 (at most the number of boundary rows is used);
 *   best (nullable) receives the options;  us_per_slot_iteration (nullable) the measured time.
 * The trial solves allocate their own output buffer.  RSFD_ERR_ARG on bad arguments,
 * RSFD_ERR_ALLOC / RSFD_ERR_CUDA when no candidate could run. */
rsfd_status rsfd_autotune(rsfd_handle h, const double* energies, int32_t K, double eta, int32_t slots, int32_t iters,
                          rsfd_solve_opts* best, double* us_per_slot_iteration);

/* Shifted COCG (Sec. III B; Appendix) over a long column list with checkpoints, so that a sweep that
 * stops (a lost job, a reboot) resumes where it stopped.  The columns are solved in blocks of `block`
 * with rsfd_shifted_cocg; after each block its slice of G0_bb and its rsfd_col_info entries are written
 * to <dir>/g0_block_<b>.bin (b = block index, six digits; written under a temporary name, then
 * renamed).  A block whose file exists and records the same inputs (operator: grid, h, order, faces,
 * precision, V_loc, projectors; solve: the block's columns, energies, eta, tol, maxit, seed policy;
 * checked by a 64-bit hash) is read back instead of solved.
 *   dir      existing, writable directory (host string);  block >= 1.
 *   G0_bb    device [K][ncols][nb] as in rsfd_shifted_cocg, or NULL to keep the results in the files only
 *            (read back by energy with rsfd_sweep_load_energies);  info host [ncols] (required).
 *   blocks_resumed (nullable) receives the number of blocks read from their files.
 * Status as rsfd_shifted_cocg (worst column outcome); RSFD_ERR_ARG when a file cannot be written. */
rsfd_status rsfd_shifted_cocg_sweep(rsfd_handle h, const int64_t* cols, int32_t ncols, const double* energies,
                                    int32_t K, double eta, double tol, int32_t maxit, int32_t seed_kind,
                                    int32_t seed_index, int32_t block, const char* dir, void* G0_bb,
                                    rsfd_col_info* info, int32_t* blocks_resumed);

/* Energies k0 .. k0 + kcount - 1 of a completed rsfd_shifted_cocg_sweep (same handle inputs and the
 * same cols, energies, eta, tol, maxit, seed policy, block and dir), every column, read from its block
 * files: G0_part device [kcount][ncols][nb], the layout of rsfd_shifted_cocg's G0_bb for those energies,
 * ready for rsfd_dyson_boundary on that energy chunk (the energy-chunked G0_bb of Sec. III B's boundary
 * blocks when all K energies do not fit in device memory).  RSFD_ERR_ARG when a block file is missing,
 * short, or was computed from other inputs. */
rsfd_status rsfd_sweep_load_energies(rsfd_handle h, const int64_t* cols, int32_t ncols, const double* energies,
                                     int32_t K, double eta, double tol, int32_t maxit, int32_t seed_kind,
                                     int32_t seed_index, int32_t block, const char* dir, int32_t k0, int32_t kcount,
                                     void* G0_part);

/* One transition region's shifted-COCG solve (the arguments of rsfd_shifted_cocg) for
 * rsfd_shifted_cocg_regions; status is written by the call. */
typedef struct {
  rsfd_handle h;
  const int64_t* cols;
  int32_t ncols;
  const double* energies;
  int32_t K;
  double eta, tol;
  int32_t maxit, seed_kind, seed_index;
  void* G0_bb;
  rsfd_col_info* info;
  double* final_res;
  rsfd_status status;
} rsfd_region_solve;

/* Shifted COCG (Sec. III B; Appendix) for several transition regions of different sizes in one call:
 * every job runs rsfd_shifted_cocg on its own handle and stream, driven by its own host thread, so the
 * regions' kernels overlap on the device.  Each handle may appear in one job only.  Returns the worst
 * job status (an error before RSFD_ERR_BREAKDOWN before RSFD_ERR_NOT_CONVERGED before RSFD_OK);
 * rsfd_last_error(NULL) names the failing region.  Results equal n separate calls. */
rsfd_status rsfd_shifted_cocg_regions(int32_t n, rsfd_region_solve* jobs);

/* Counters and timings of the last rsfd_shifted_cocg call on this handle. */
rsfd_status rsfd_get_stats(rsfd_handle h, rsfd_stats* out);

/* Dyson / OBM boundary step (Eq. sec3-01a restricted to b):
 *   (I - G0_bb(k) Sigma_bb(k)) G_bb(k) = G0_bb(k),  Sigma_bb = diag(Sigma_L, Sigma_R),
 * for every k < K.  G0_bb must hold all boundary columns in b order
 * (ncols = nb).  The solve is an LU with partial pivoting followed by FP64
 * iterative refinement of the residual G0 - (I - G0 Sigma) G.  Form (rsfd_solve_opts.dyson_kind):
 * FP64 LU on the CUDA cores (FP64 handles by default), or FP32 LU and triangular solves whose
 * updates run on the tensor cores (3xTF32) with FP64 residuals (double-float and complex64 handles
 * by default); energies are processed in chunks that fit the free device memory.
 *   G0_bb    device [K][nb][nb] (handle precision).
 *   Sigma_L, Sigma_R  device [K][ns][ns] c128.
 *   G_bb     device output, same layout and type as G0_bb (may not alias G0_bb).
 *   refine_residual  host [K] (nullable): ||G0 - M G||_F / ||G0||_F after refinement. */
rsfd_status rsfd_dyson_boundary(rsfd_handle h, const void* G0_bb, const void* Sigma_L, const void* Sigma_R,
                                int32_t K, void* G_bb, double* refine_residual);

/* Batched complex GEMM on the tensor cores: the building block of the Dyson solve's LU and triangular
 * solves (Eq. sec3-01a; see rsfd_dyson_boundary), exposed for direct use and testing.
 *   C[b] = alpha A[b] B[b] + beta C[b],  b < batch,
 * complex FP32 (interleaved re, im floats), column-major.  Every product is taken in 3xTF32 form
 * (hi*hi + hi*lo + lo*hi of the TF32 splits) with FP32 accumulation: FP32-class accuracy.
 *   A  device m x k, leading dimension lda >= m, batch stride sA (complex elements);
 *   B  device k x n, ldb >= k, stride sB;  C device m x n, ldc >= m, stride sC (may not overlap A, B);
 *   alpha host [2] (re, im);  beta 0 or 1;  stream cudaStream_t (NULL = legacy default stream).
 * The call synchronises the stream.  RSFD_ERR_ARG for bad sizes or beta, RSFD_ERR_CUDA for a launch
 * failure, RSFD_ERR_TIMEOUT when the kernel's bounded wait on its tensor-core operations expired. */
rsfd_status rsfd_cgemm_tf32x3(int32_t batch, int32_t m, int32_t n, int32_t k, const double* alpha, const void* A,
                              int32_t lda, int64_t sA, const void* B, int32_t ldb, int64_t sB, double beta, void* C,
                              int32_t ldc, int64_t sC, void* stream);

/* Dyson step on the recorded row set (Eq. sec3-01a with Sigma supported on b; the interior blocks
 * G_T(z_0, z_l), G_T(z_l, z_l) of Sec. III B):
 *   G(k) = G0(k) + G0(k)[:, b] Sigma_bb(k) (I - G0_bb(k) Sigma_bb(k))^{-1} G0(k)[b, :].
 * G0 must come from a solve whose columns are the recorded rows in rsfd_tracked_rows order
 * (ncols = nr).  G[b, b] equals rsfd_dyson_boundary's G_bb; G[l, l] is the perturbed diagonal block of
 * tracked plane l, whose -Im trace / pi gives the plane's density of states.  LU with partial pivoting
 * and two FP64 refinement steps, as rsfd_dyson_boundary.
 *   G0       device [K][nr][nr] (handle precision), column-major per energy.
 *   Sigma_L, Sigma_R  device [K][ns][ns] c128.
 *   G        device output, same layout and type as G0 (may not alias G0).
 *   refine_residual  host [K] (nullable): ||G0_b: - M G_b:||_F / ||G0_b:||_F on the boundary rows. */
rsfd_status rsfd_dyson_tracked(rsfd_handle h, const void* G0, const void* Sigma_L, const void* Sigma_R, int32_t K,
                               void* G, double* refine_residual);

/* Fisher-Lee transmission (Eq. TF; Gamma = i(Sigma - Sigma^dag)):
 *   T(k) = Tr[Gamma_L G_RL^dag Gamma_R G_RL],  G_RL = G_bb(k)[right slab, left slab].
 *   G_bb  device [K][nb][nb] (handle precision);  Sigma_L, Sigma_R device [K][ns][ns] c128;
 *   T     host output [K]. */
rsfd_status rsfd_transmission(rsfd_handle h, const void* G_bb, const void* Sigma_L, const void* Sigma_R, int32_t K,
                              double* T);

/* Self-energies of uniform V=0 leads that continue the grid (same Nx, Ny, h,
 * fd_order, Dirichlet walls) on both sides (Eqs. self-energy, sec2-01, sec2-02),
 * computed on the host in FP64 from the outgoing Bloch roots of each
 * transverse mode.  ns = (fd_order/2)*Nx*Ny.
 *   energies host [K];  Sigma_L, Sigma_R host outputs [K][ns][ns] c128 (interleaved doubles). */
rsfd_status rsfd_lead_sigma_uniform(int32_t Nx, int32_t Ny, double h, int32_t fd_order, const double* energies,
                                    double eta, int32_t K, double* Sigma_L, double* Sigma_R);

/* Self-energies of leads that repeat one principal layer of R = fd_order/2 planes with its own local
 * potential (Eq. self-energy: Sigma_L = B^dag g_L B, Sigma_R = B g_R B^dag, with the surface Green's
 * function of Eq. surface green's function of each semi-infinite lead), computed on the GPU in FP64 by
 * the Lopez Sancho-Rubio decimation, batched over energies.  The leads continue the handle's grid (same
 * Nx, Ny, h, order and Dirichlet walls); the handle's boundary slab must have R planes per side.
 *   V_left, V_right  host [R][Ny][Nx] (nullable = 0): one principal layer of each lead, planes in
 *                    increasing z, x fastest.
 *   energies host [K];  eta > 0 (Z = E + i eta);  maxit >= 1 decimation steps (each doubles the
 *   decimated length; about log2 of (lead decay length / layer) are needed, e.g. 20-40 at eta = 1e-3).
 *   Sigma_L, Sigma_R device outputs [K][ns][ns] c128, ns = R Nx Ny, as rsfd_dyson_boundary takes them.
 *   iterations (nullable) receives the largest number of steps used.
 * RSFD_ERR_NOT_CONVERGED after maxit steps, RSFD_ERR_BREAKDOWN for a singular Z - eps. */
rsfd_status rsfd_lead_sigma_decimation(rsfd_handle h, const double* V_left, const double* V_right,
                                       const double* energies, int32_t K, double eta, int32_t maxit, void* Sigma_L,
                                       void* Sigma_R, int32_t* iterations);

/* Size of the file-scope device array that rsfd_dyson_boundary_noalloc uses as scratch. */
#define RSFD_NOALLOC_SCRATCH_BYTES (32u << 20)

/* Allocation-free Dyson step.  The paper has no counterpart: this entry point exists for callers
 * that cannot allocate device memory when they need the step, e.g. a service or framework that has
 * handed its whole device-memory budget to its own caching allocator up front, or a plug-in whose
 * host application forbids it to change the device's allocation state.
 *
 * It computes the same result as rsfd_dyson_boundary for FP64 data, without a handle:
 *   (I - G0_bb(k) Sigma_bb(k)) G_bb(k) = G0_bb(k),  k < K,  with two FP64 refinement steps.
 *   nb      even, the number of boundary rows (ns = nb/2 per slab).
 *   K       1 .. 65535 energies.
 *   G0_bb   device [K][nb][nb] c128, column-major per energy (same layout as rsfd_dyson_boundary).
 *   Sigma_L, Sigma_R  device [K][ns][ns] c128.
 *   G_bb    device output [K][nb][nb] c128 (may not alias G0_bb).
 *   refine_residual  host [K] (nullable): ||G0 - M G||_F / ||G0||_F.
 *   stream  cudaStream_t (NULL = legacy default stream).  The call ends by copying its status word
 *           and the residuals to the host and synchronising this stream.
 * Scratch: a static __device__ array of RSFD_NOALLOC_SCRATCH_BYTES (32 MiB) held by every GPU that
 * loads the library until the process exits.  The call needs 3*nb*nb*K*16 bytes plus pivots and
 * returns RSFD_ERR_ARG (with a message naming the limit) when that exceeds the array; for nb = 128
 * that allows K <= 42.  Nothing is allocated: no cudaMalloc, cudaFree or allocating library call.
 * Set-up: the first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * Sharing: every call, on any stream, uses the same array and it keeps the previous call's
 * contents (the call clears what must start at zero); calls that overlap on the GPU race with
 * each other, so serialise them.
 * Returns RSFD_OK, RSFD_ERR_ARG, RSFD_ERR_CUDA, or RSFD_ERR_BREAKDOWN (singular I - G0 Sigma; the
 * message names the first such energy, as rsfd_dyson_boundary's does). */
rsfd_status rsfd_dyson_boundary_noalloc(int32_t nb, int32_t K, const void* G0_bb, const void* Sigma_L,
                                        const void* Sigma_R, void* G_bb, double* refine_residual, void* stream);

/* Message of the last failure on this handle (h = NULL: last failure of a call
 * without a handle, e.g. rsfd_create).  Never NULL. */
const char* rsfd_last_error(rsfd_handle h);

/* Free the handle and its device buffers (synchronises its stream).  NULL is a no-op. */
void rsfd_destroy(rsfd_handle h);

#ifdef __cplusplus
}
#endif

#endif /* RSFD_H */
