// Shifted COCG kernels for sm_103a.
//
// One iteration of the seed system (Appendix, Eqs. rvec, alpha, beta) is a single fused pass
// per right-hand side ("slot"):
//
//   r_n = a1 r_{n-1} + a2 r_{n-2} + aA (A r_{n-1}),       A = Z_s - H_T,
//   (r_n, r_n), (r_n, A r_n) (unconjugated) and ||r_n||^2,
//
// computed on a 2.5D tile that marches along z.  Each CTA owns an x-y tile of one slot and a
// range of z-planes; it loads r_{n-1} on the tile plus a 2R-wide halo, r_{n-2} on the tile plus
// an R-wide halo, evaluates A r_{n-1} and r_n on the tile plus R, then A r_n on the tile.  The
// halo work is recomputed rather than stored, so an iteration moves three vectors through HBM
// (read r_{n-1}, read r_{n-2}, write r_n) instead of the four or five of a stencil-then-update
// split.  The last CTA of a slot to finish (atomic ticket, no waiting) reduces the per-CTA dot
// products in a fixed order and runs the FP64 scalar step: convergence of every energy, seed
// switching (Eq. seedswitch), alpha_n, beta_{n-1}, and the shifted recurrences pi_{n+1},
// alpha_n^(i), beta_{n-1}^(i) (Eqs. spi, salpha, sbeta).  A second kernel applies the vector
// part of the shifted update (Eq. endcollinear and the x^(i) update) on the boundary rows only,
// with r_n^(i) = r_n / pi_n^(s,i) (Eq. collinear).
//
// No kernel waits on another CTA: there are no spin loops anywhere in this file.

#include <cuda_runtime.h>
#include <math.h>

#include "rsfd_internal.cuh"

namespace rsfd {
namespace {

constexpr int kTileX = 32;

// ------------------------------------------------------------------------------------------------
// vector arithmetic on interleaved complex numbers in the precision of the Krylov vectors
// ------------------------------------------------------------------------------------------------
template <typename T> struct VOps;

template <> struct VOps<float> {
  typedef float2 C;
  static __device__ __forceinline__ C zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ C add(C a, C b) { return __fadd2_rn(a, b); }
  // c + s * a, s real (packed FP32x2 FMA)
  static __device__ __forceinline__ C fmar(float s, C a, C c) { return __ffma2_rn(make_float2(s, s), a, c); }
  // c + z * a, z complex
  static __device__ __forceinline__ C fmac(C z, C a, C c) {
    c = __ffma2_rn(make_float2(z.x, z.x), a, c);
    return __ffma2_rn(make_float2(-z.y, z.y), make_float2(a.y, a.x), c);
  }
  static __device__ __forceinline__ C from(double2 z) { return make_float2((float)z.x, (float)z.y); }
};

template <> struct VOps<double> {
  typedef double2 C;
  static __device__ __forceinline__ C zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ C add(C a, C b) { return make_double2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ C fmar(double s, C a, C c) { return make_double2(fma(s, a.x, c.x), fma(s, a.y, c.y)); }
  static __device__ __forceinline__ C fmac(C z, C a, C c) {
    return make_double2(fma(z.x, a.x, fma(-z.y, a.y, c.x)), fma(z.x, a.y, fma(z.y, a.x, c.y)));
  }
  static __device__ __forceinline__ C from(double2 z) { return z; }
};

// Per-thread dot-product accumulators: (r,r), (r,Ar) unconjugated and ||r||^2.
template <typename T> struct Acc;

template <> struct Acc<double> {
  double rr_x = 0, rr_y = 0, ra_x = 0, ra_y = 0, nn = 0;
  __device__ __forceinline__ void add(double2 r, double2 v) {
    rr_x = fma(r.x, r.x, fma(-r.y, r.y, rr_x));
    rr_y = fma(2.0 * r.x, r.y, rr_y);
    ra_x = fma(r.x, v.x, fma(-r.y, v.y, ra_x));
    ra_y = fma(r.x, v.y, fma(r.y, v.x, ra_y));
    nn = fma(r.x, r.x, fma(r.y, r.y, nn));
  }
  __device__ __forceinline__ void get(double* o) const { o[0] = rr_x; o[1] = rr_y; o[2] = ra_x; o[3] = ra_y; o[4] = nn; }
};

template <> struct Acc<float> {
  float2 rr = make_float2(0.f, 0.f), rr_c = make_float2(0.f, 0.f);   // Kahan sum and compensation
  float2 ra = make_float2(0.f, 0.f), ra_c = make_float2(0.f, 0.f);
  float nn = 0.f;
  static __device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
  static __device__ __forceinline__ void kahan(float2& s, float2& c, float2 term) {
    const float2 y = sub2(term, c);
    const float2 t = __fadd2_rn(s, y);
    c = sub2(sub2(t, s), y);
    s = t;
  }
  __device__ __forceinline__ void add(float2 r, float2 v) {
    // r*r = (x^2 - y^2, 2xy);  r*v = (x vx - y vy, x vy + y vx)
    const float2 trr = make_float2(__fmaf_rn(r.x, r.x, -r.y * r.y), 2.f * r.x * r.y);
    const float2 tra = make_float2(__fmaf_rn(r.x, v.x, -r.y * v.y), __fmaf_rn(r.x, v.y, r.y * v.x));
    kahan(rr, rr_c, trr);
    kahan(ra, ra_c, tra);
    nn = __fmaf_rn(r.x, r.x, __fmaf_rn(r.y, r.y, nn));
  }
  __device__ __forceinline__ void get(double* o) const {
    o[0] = (double)rr.x - (double)rr_c.x;
    o[1] = (double)rr.y - (double)rr_c.y;
    o[2] = (double)ra.x - (double)ra_c.x;
    o[3] = (double)ra.y - (double)ra_c.y;
    o[4] = (double)nn;
  }
};

struct PassParams {
  SolveDims d;
  void* rbuf;
  const void* V;
  SlotState* slots;
  ShiftState* shifts;
  double* partials;
  unsigned int* tickets;
  const double2* Z;
  unsigned long long* counters;
  double hd;
  double hk1, hk2;
  double tol;
  int maxit;
};

// ------------------------------------------------------------------------------------------------
// block reductions (FP64)
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum NV doubles over the block; result valid in thread 0.  s_red must hold 32*NV doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* s_red) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nthr = blockDim.x * blockDim.y;
  const int lane = tid & 31, wid = tid >> 5, nw = (nthr + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) s_red[wid * NV + k] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = (lane < nw) ? s_red[lane * NV + k] : 0.0;
      v[k] = warp_sum(t);
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------------------------
// FP64 scalar step of one slot (run by the last CTA of the slot)
// ------------------------------------------------------------------------------------------------
struct ScalarShared {
  double2 rr, rAr;
  double nrm2;
  double2 beta, alpha, c, scale_n, scale_nm1, fn, fnm1, Zs;
  int stop;      // 1 = slot finished in this step
  int do_switch;
  int seed;
  int n;
  double red[32 * 5];
  int ired[32 * 2];
};

__device__ void scalar_step(const PassParams& p, int slot, ScalarShared& S) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nthr = blockDim.x * blockDim.y;
  const int K = p.d.K;
  SlotState* st = p.slots + slot;
  ShiftState* sh = p.shifts + (size_t)slot * K;
  const int n = st->n;
  const double rnorm = sqrt(S.nrm2);

  // Phase A: convergence of every active energy, ||r_n^(i)|| = ||r_n|| / |pi_n^(s,i)| (Eq. collinear)
  int cnt = 0, bad = 0;
  double best = -1.0;
  int best_i = K;
  for (int i = tid; i < K; i += nthr) {
    ShiftState& q = sh[i];
    if (!q.active) continue;
    const double res = rnorm / sqrt(cabs2(q.pi_n));
    q.res = res;
    if (!(res == res)) {
      bad = 1;
      continue;
    }
    if (res < p.tol) {
      q.active = 0;
      q.conv_iter = n;
    } else {
      ++cnt;
      if (res > best) { best = res; best_i = i; }
    }
  }
  // block reductions: count, NaN flag, argmax (ties -> lowest index)
  {
    const int lane = tid & 31, wid = tid >> 5, nw = (nthr + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) {
      cnt += __shfl_down_sync(0xffffffffu, cnt, o);
      bad |= __shfl_down_sync(0xffffffffu, bad, o);
      const double ob = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, best_i, o);
      if (ob > best || (ob == best && oi < best_i)) { best = ob; best_i = oi; }
    }
    if (lane == 0) {
      S.red[wid] = best;
      S.ired[wid] = best_i;
      S.ired[32 + wid] = cnt | (bad << 30);
    }
    __syncthreads();
    if (tid == 0) {
      int c_all = 0, b_all = 0;
      double bb = -1.0;
      int bi = K;
      for (int w = 0; w < nw; ++w) {
        const int v = S.ired[32 + w];
        c_all += v & ((1 << 30) - 1);
        b_all |= v >> 30;
        if (S.red[w] > bb || (S.red[w] == bb && S.ired[w] < bi)) { bb = S.red[w]; bi = S.ired[w]; }
      }
      // decide what this step does
      int seed = st->seed;
      S.stop = 0;
      S.do_switch = 0;
      double2 beta = make_double2(0.0, 0.0);
      double2 rr = S.rr, rAr = S.rAr;
      double2 alpha_prev = st->alpha_prev;
      // stored vectors: r_n is in the current normalisation, r_{n-1} needs the factor carried
      // over from a switch in the previous step (collinear rescaling, Eq. seedswitch)
      double2 scale_n = make_double2(1.0, 0.0), scale_nm1 = st->carry;
      if (n > 0) beta = cdiv(rr, st->rr_prev);                                   // Eq. beta
      if (b_all) {
        st->status = SLOT_BREAKDOWN;
        S.stop = 1;
      } else if (c_all == 0) {
        st->status = SLOT_DONE;
        S.stop = 1;
      } else if (n >= p.maxit) {
        st->status = SLOT_MAXIT;
        S.stop = 1;
      } else {
        if (!sh[seed].active) {
          // seed switching (Eq. seedswitch): the unconverged energy with the largest residual
          const int s2 = bi;
          const double2 fn = sh[s2].pi_n, fnm1 = sh[s2].pi_nm1;
          const double2 q = cdiv(fnm1, fn);
          beta = cmul(beta, cmul(q, q));                                         // beta_{n-1}^(s~) (Eq. sbeta)
          alpha_prev = sh[s2].alpha_prev;                                        // alpha_{n-1}^(s~)
          const double2 f2 = cmul(fn, fn);
          rAr = cdiv(cadd(rAr, cmul(csub(p.Z[s2], p.Z[seed]), rr)), f2);         // (r~, (Z_s~ - H) r~)
          rr = cdiv(rr, f2);
          scale_n = cdiv(make_double2(1.0, 0.0), fn);
          scale_nm1 = cdiv(scale_nm1, fnm1);
          S.fn = fn;
          S.fnm1 = fnm1;
          S.do_switch = 1;
          seed = s2;
          st->switches += 1;
        }
        const double rabs = sqrt(cabs2(rr));
        const double nrm2s = S.nrm2 * cabs2(scale_n);
        if (!(rabs > 1e-300) || rabs <= 1e-28 * nrm2s) {
          st->status = SLOT_BREAKDOWN;
          S.stop = 1;
        } else {
          // Eq. alpha (alpha_n), and the three-term coefficient beta_{n-1} alpha_n / alpha_{n-1}
          const double2 alpha = cdiv(rr, csub(rAr, cmul(cdiv(beta, alpha_prev), rr)));
          const double2 c = cdiv(cmul(beta, alpha), alpha_prev);
          if (!(alpha.x == alpha.x) || !(alpha.y == alpha.y) || !(c.x == c.x) || !(c.y == c.y)) {
            st->status = SLOT_BREAKDOWN;
            S.stop = 1;
          }
          S.alpha = alpha;
          S.c = c;
        }
      }
      if (S.stop) {
        st->iters = n;
        st->k4_n = -1;
      }
      S.beta = beta;
      S.rr = rr;
      S.scale_n = scale_n;
      S.scale_nm1 = scale_nm1;
      S.seed = seed;
      S.Zs = p.Z[seed];
      S.n = n;
    }
    __syncthreads();
  }
  if (S.stop) return;

  // Phase C: shifted recurrences for every active energy (Eqs. spi, salpha, sbeta) and the
  // coefficients of the vector update p_n^(i) = r_n / pi_n + beta_{n-1}^(i) p_{n-1}^(i),
  // x_{n+1}^(i) = x_n^(i) + alpha_n^(i) p_n^(i).
  const double2 one = make_double2(1.0, 0.0);
  for (int i = tid; i < K; i += nthr) {
    ShiftState& q = sh[i];
    if (!q.active) continue;
    double2 pin = q.pi_n, pinm1 = q.pi_nm1;
    if (S.do_switch) {
      pin = cdiv(pin, S.fn);
      pinm1 = cdiv(pinm1, S.fnm1);
    }
    const double2 sigma = csub(p.Z[i], S.Zs);
    const double2 ratio = cdiv(pinm1, pin);
    const double2 beta_i = cmul(cmul(ratio, ratio), S.beta);
    const double2 pinp1 = csub(cmul(cadd(cadd(one, S.c), cmul(S.alpha, sigma)), pin), cmul(S.c, pinm1));
    const double2 alpha_i = cmul(cdiv(pin, pinp1), S.alpha);
    q.cr = cdiv(S.scale_n, pin);
    q.cb = beta_i;
    q.ca = alpha_i;
    q.alpha_prev = alpha_i;
    q.pi_nm1 = pin;
    q.pi_n = pinp1;
  }
  if (tid == 0) {
    const double2 c = S.c;
    st->a1 = cmul(cadd(one, c), S.scale_n);
    st->a2 = cmul(make_double2(-c.x, -c.y), S.scale_nm1);
    st->aA = cmul(make_double2(-S.alpha.x, -S.alpha.y), S.scale_n);
    st->Zs = S.Zs;
    st->seed = S.seed;
    st->alpha_prev = S.alpha;
    st->rr_prev = S.rr;
    st->carry = S.scale_n;   // r_n becomes the next step's r_{n-1}
    st->k4_n = S.n;
    st->n = S.n + 1;
    atomicAdd(&p.counters[1], 1ull);
  }
}

// ------------------------------------------------------------------------------------------------
// the fused pass
// ------------------------------------------------------------------------------------------------
template <typename T, int R>
__global__ void __launch_bounds__(640) pass_kernel(PassParams p) {
  typedef VOps<T> O;
  typedef typename VOps<T>::C C;
  constexpr int EX = kTileX + 4 * R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ ScalarShared S;
  __shared__ int s_last;

  const int slot = blockIdx.y;
  SlotState* st = p.slots + slot;
  if (st->status != SLOT_RUNNING) return;

  const SolveDims& d = p.d;
  const int EY = blockDim.y;
  const int TY = EY - 4 * R;
  const int ex = threadIdx.x, ey = threadIdx.y;
  const int cta = blockIdx.x;
  const int tz = cta % d.nzchunks;
  const int txy = cta / d.nzchunks;
  const int tx = txy % d.tiles_x, ty = txy / d.tiles_x;
  const int z0 = tz * d.zchunk;
  const int z1 = min(z0 + d.zchunk, d.nz);
  const int gx = tx * kTileX - 2 * R + ex;
  const int gy = ty * TY - 2 * R + ey;
  const bool inside = (gx >= 0) && (gx < d.nx) && (gy >= 0) && (gy < d.ny);
  const bool is_mid = (ex >= R) && (ex < EX - R) && (ey >= R) && (ey < EY - R);
  const bool is_int = (ex >= 2 * R) && (ex < EX - 2 * R) && (ey >= 2 * R) && (ey < EY - 2 * R);
  const long long nxy = (long long)d.nx * d.ny;
  const long long coff = inside ? ((long long)gy * d.nx + gx) : 0;

  const int n = st->n;
  const C* rm1 = reinterpret_cast<const C*>(p.rbuf) + ((size_t)slot * 3 + (n + 2) % 3) * d.N;
  const C* rm2 = reinterpret_cast<const C*>(p.rbuf) + ((size_t)slot * 3 + (n + 1) % 3) * d.N;
  C* rout = reinterpret_cast<C*>(p.rbuf) + ((size_t)slot * 3 + n % 3) * d.N;
  const T* V = reinterpret_cast<const T*>(p.V);
  const C a1 = O::from(st->a1), a2 = O::from(st->a2), aA = O::from(st->aA);
  const double2 Zs = st->Zs;
  const T zre = (T)(Zs.x - p.hd), zim = (T)Zs.y;   // diagonal of A without V: Z_s - hd
  const T mh1 = (T)(-p.hk1), mh2 = (T)(-p.hk2);

  C* sA = reinterpret_cast<C*>(smem_raw);          // [2][EY][EX]  r_{n-1} on the current plane
  C* sB = sA + 2 * EY * EX;                        // [2][EY][EX]  r_n on the output plane

  C qa[2 * R + 1], qb[2 * R + 1];
  T vq[R + 1];
#pragma unroll
  for (int k = 0; k <= 2 * R; ++k) { qa[k] = O::zero(); qb[k] = O::zero(); }
#pragma unroll
  for (int k = 0; k <= R; ++k) vq[k] = (T)0;
#pragma unroll
  for (int k = 1; k <= 2 * R; ++k) {
    const int z = z0 - 2 * R + k - 1;
    if (inside && z >= 0 && z < d.nz) qa[k] = rm1[z * nxy + coff];
  }
  // Per-thread partial sums of (r,r) and (r,Ar).  The unconjugated forms cancel, so in FP32 they
  // are accumulated with Kahan compensation (plain FP32 accumulation of FP32 products makes some
  // columns stagnate); ||r||^2 has no cancellation and is summed plainly.
  Acc<T> acc;
  int buf = 0;

  for (int pz = z0 - R; pz < z1 + R; ++pz) {
    const bool pz_in = (pz >= 0) && (pz < d.nz);
#pragma unroll
    for (int k = 0; k < 2 * R; ++k) qa[k] = qa[k + 1];
    {
      const int z = pz + R;
      qa[2 * R] = (inside && z >= 0 && z < d.nz) ? rm1[z * nxy + coff] : O::zero();
    }
    C r2 = O::zero();
#pragma unroll
    for (int k = 0; k < R; ++k) vq[k] = vq[k + 1];
    vq[R] = (T)0;
    if (is_mid && inside && pz_in) {
      r2 = rm2[pz * nxy + coff];
      vq[R] = V[pz * nxy + coff];
    }
    C* A = sA + buf * EY * EX;
    C* B = sB + buf * EY * EX;
    A[ey * EX + ex] = qa[R];
    __syncthreads();
    if (is_mid) {
      C rn = O::zero();
      if (inside && pz_in) {
        // u = A r_{n-1} = (Z_s - V - hd) r_{n-1} - sum_k hk_k (neighbours at distance k)
        C s1 = O::add(O::add(qa[R - 1], qa[R + 1]),
                      O::add(O::add(A[ey * EX + ex - 1], A[ey * EX + ex + 1]),
                             O::add(A[(ey - 1) * EX + ex], A[(ey + 1) * EX + ex])));
        C u = O::fmar(mh1, s1, O::zero());
        if (R == 2) {
          C s2 = O::add(O::add(qa[0], qa[4]),
                        O::add(O::add(A[ey * EX + ex - 2], A[ey * EX + ex + 2]),
                               O::add(A[(ey - 2) * EX + ex], A[(ey + 2) * EX + ex])));
          u = O::fmar(mh2, s2, u);
        }
        C dg;
        dg.x = zre - vq[R];
        dg.y = zim;
        u = O::fmac(dg, qa[R], u);
        // r_n = a1 r_{n-1} + a2 r_{n-2} + aA u   (Eq. rvec)
        rn = O::fmac(aA, u, O::fmac(a2, r2, O::fmac(a1, qa[R], O::zero())));
      }
#pragma unroll
      for (int k = 0; k < 2 * R; ++k) qb[k] = qb[k + 1];
      qb[2 * R] = rn;
      B[ey * EX + ex] = qb[R];
    }
    __syncthreads();
    const int zo = pz - R;
    if (is_int && inside && zo >= z0 && zo < z1) {
      // v = A r_n on the output plane, then the three dot products
      const C r = qb[R];
      C s1 = O::add(O::add(qb[R - 1], qb[R + 1]),
                    O::add(O::add(B[ey * EX + ex - 1], B[ey * EX + ex + 1]),
                           O::add(B[(ey - 1) * EX + ex], B[(ey + 1) * EX + ex])));
      C v = O::fmar(mh1, s1, O::zero());
      if (R == 2) {
        C s2 = O::add(O::add(qb[0], qb[4]),
                      O::add(O::add(B[ey * EX + ex - 2], B[ey * EX + ex + 2]),
                             O::add(B[(ey - 2) * EX + ex], B[(ey + 2) * EX + ex])));
        v = O::fmar(mh2, s2, v);
      }
      C dg;
      dg.x = zre - vq[0];
      dg.y = zim;
      v = O::fmac(dg, r, v);
      acc.add(r, v);
      rout[zo * nxy + coff] = r;
    }
    buf ^= 1;
  }

  // per-CTA partial sums, promoted to FP64 for the tree
  double v5[5];
  acc.get(v5);
  block_sum<5>(v5, S.red);
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  if (tid == 0) {
    double* dst = p.partials + ((size_t)slot * d.ctas_per_slot + cta) * 8;
#pragma unroll
    for (int k = 0; k < 5; ++k) dst[k] = v5[k];
    __threadfence();
    const unsigned int t = atomicAdd(p.tickets + slot, 1u);
    s_last = (t == (unsigned int)(d.ctas_per_slot - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();

  // last CTA of the slot: fixed-order reduction of the partials, then the scalar step
  {
    const int nthr = blockDim.x * blockDim.y;
    double w5[5] = {0, 0, 0, 0, 0};
    const double* src = p.partials + (size_t)slot * d.ctas_per_slot * 8;
    for (int c = tid; c < d.ctas_per_slot; c += nthr) {
#pragma unroll
      for (int k = 0; k < 5; ++k) w5[k] += __ldcg(src + (size_t)c * 8 + k);
    }
    block_sum<5>(w5, S.red);
    if (tid == 0) {
      S.rr = make_double2(w5[0], w5[1]);
      S.rAr = make_double2(w5[2], w5[3]);
      S.nrm2 = w5[4];
      p.tickets[slot] = 0u;
    }
    __syncthreads();
  }
  scalar_step(p, slot, S);
}

// ------------------------------------------------------------------------------------------------
// shift update on the boundary rows: p <- cr r_n + cb p ; x <- x + ca p
// ------------------------------------------------------------------------------------------------
struct ShiftParams {
  SolveDims d;
  const void* rbuf;
  void* pbuf;
  void* G0;
  const SlotState* slots;
  const ShiftState* shifts;
  unsigned long long* counters;
};

template <typename T>
__global__ void __launch_bounds__(256) shift_kernel(ShiftParams p) {
  typedef VOps<T> O;
  typedef typename VOps<T>::C C;
  const int i = blockIdx.x;
  const int slot = blockIdx.y;
  const SlotState& st = p.slots[slot];
  if (st.status != SLOT_RUNNING || st.k4_n < 0) return;
  const ShiftState& q = p.shifts[(size_t)slot * p.d.K + i];
  if (!q.active) return;
  if (threadIdx.x == 0) atomicAdd(&p.counters[0], 1ull);
  const SolveDims& d = p.d;
  const long long nxy = (long long)d.nx * d.ny;
  const C* r = reinterpret_cast<const C*>(p.rbuf) + ((size_t)slot * 3 + st.k4_n % 3) * d.N;
  C* pp = reinterpret_cast<C*>(p.pbuf) + ((size_t)slot * d.K + i) * d.nb;
  C* x = reinterpret_cast<C*>(p.G0) + ((size_t)i * d.ncols + st.col) * d.nb;
  const C cr = O::from(q.cr), cb = O::from(q.cb), ca = O::from(q.ca);
  const int nplanes = 2 * d.nface;
  for (int pl = 0; pl < nplanes; ++pl) {
    const int z = (pl < d.nface) ? pl : (d.nz - nplanes + pl);
    const C* rz = r + (long long)z * nxy;
    C* pz = pp + (long long)pl * nxy;
    C* xz = x + (long long)pl * nxy;
    for (long long o = threadIdx.x; o < nxy; o += blockDim.x) {
      const C pv = O::fmac(cb, pz[o], O::fmac(cr, rz[o], O::zero()));
      pz[o] = pv;
      xz[o] = O::fmac(ca, pv, xz[o]);
    }
  }
}

// ------------------------------------------------------------------------------------------------
// slot initialisation: r_{-1} = e_j, r_{-2} = 0, p = 0, x = 0, pi = 1
// ------------------------------------------------------------------------------------------------
struct InitParams {
  SolveDims d;
  void* rbuf;
  void* pbuf;
  void* G0;
  SlotState* slots;
  ShiftState* shifts;
  const double2* Z;
  const int* init_list;
  const long long* init_grid;
  int seed0;
};

template <typename T>
__global__ void __launch_bounds__(256) init_kernel(InitParams p) {
  typedef VOps<T> O;
  typedef typename VOps<T>::C C;
  const int e = blockIdx.y;
  const int slot = p.init_list[2 * e], col = p.init_list[2 * e + 1];
  const long long j = p.init_grid[e];
  const SolveDims& d = p.d;
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gs = (long long)gridDim.x * blockDim.x;
  C* r1 = reinterpret_cast<C*>(p.rbuf) + ((size_t)slot * 3 + 1) * d.N;   // r_{-2}
  C* r2 = reinterpret_cast<C*>(p.rbuf) + ((size_t)slot * 3 + 2) * d.N;   // r_{-1}
  for (long long t = gt; t < d.N; t += gs) {
    r1[t] = O::zero();
    C v = O::zero();
    if (t == j) v.x = (T)1;
    r2[t] = v;
  }
  C* pp = reinterpret_cast<C*>(p.pbuf) + (size_t)slot * d.K * d.nb;
  const long long knb = (long long)d.K * d.nb;
  for (long long t = gt; t < knb; t += gs) {
    pp[t] = O::zero();
    const long long k = t / d.nb, row = t - k * d.nb;
    reinterpret_cast<C*>(p.G0)[((size_t)k * d.ncols + col) * d.nb + row] = O::zero();
  }
  ShiftState* sh = p.shifts + (size_t)slot * d.K;
  for (long long t = gt; t < d.K; t += gs) {
    ShiftState q;
    q.pi_n = make_double2(1.0, 0.0);
    q.pi_nm1 = make_double2(1.0, 0.0);
    q.alpha_prev = make_double2(1.0, 0.0);
    q.cr = q.cb = q.ca = make_double2(0.0, 0.0);
    q.res = 1.0;
    q.active = 1;
    q.conv_iter = -1;
    sh[t] = q;
  }
  if (gt == 0) {
    SlotState s;
    s.col = col;
    s.n = 0;
    s.seed = p.seed0;
    s.status = SLOT_RUNNING;
    s.switches = 0;
    s.k4_n = -1;
    s.iters = 0;
    s.pad0 = 0;
    s.a1 = make_double2(1.0, 0.0);       // the first pass produces r_0 = r_{-1} = e_j
    s.a2 = make_double2(0.0, 0.0);
    s.aA = make_double2(0.0, 0.0);
    s.Zs = p.Z[p.seed0];
    s.alpha_prev = make_double2(1.0, 0.0);   // alpha_{-1} = 1
    s.rr_prev = make_double2(1.0, 0.0);
    s.carry = make_double2(1.0, 0.0);
    p.slots[slot] = s;
  }
}

template <typename T, int R>
cudaError_t launch_pass_t(const SolveDims& d, const SolverBuffers& b, const StencilCoef& c, double tol, int maxit,
                          cudaStream_t st) {
  typedef typename VOps<T>::C C;
  PassParams p;
  p.d = d;
  p.rbuf = b.rbuf;
  p.V = b.V;
  p.slots = b.slots;
  p.shifts = b.shifts;
  p.partials = b.partials;
  p.tickets = b.tickets;
  p.Z = b.Z;
  p.counters = b.counters;
  p.hd = c.hd;
  p.hk1 = c.hk[0];
  p.hk2 = (R == 2) ? c.hk[1] : 0.0;
  p.tol = tol;
  p.maxit = maxit;
  const int EX = kTileX + 4 * R;
  const int EY = d.tile_y + 4 * R;
  const size_t smem = (size_t)4 * EX * EY * sizeof(C);
  dim3 grid(d.ctas_per_slot, d.W), block(EX, EY);
  pass_kernel<T, R><<<grid, block, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace

int pass_tile_x(int) { return kTileX; }

cudaError_t kernels_init() {
  // the pass kernel's dynamic shared memory (4 planes of the extended tile) can exceed 48 KB
  // in FP64 with tall tiles; raise the limit once, outside any stream capture
  cudaError_t e = cudaFuncSetAttribute(pass_kernel<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_kernel<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_kernel<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_kernel<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
  return e;
}
int pass_threads(int R, int tile_y) { return (kTileX + 4 * R) * (tile_y + 4 * R); }

cudaError_t launch_pass(bool fp64, const SolveDims& d, const SolverBuffers& b, const StencilCoef& c, double tol,
                        int maxit, cudaStream_t st) {
  if (fp64) {
    return d.R == 1 ? launch_pass_t<double, 1>(d, b, c, tol, maxit, st) : launch_pass_t<double, 2>(d, b, c, tol, maxit, st);
  }
  return d.R == 1 ? launch_pass_t<float, 1>(d, b, c, tol, maxit, st) : launch_pass_t<float, 2>(d, b, c, tol, maxit, st);
}

cudaError_t launch_shift(bool fp64, const SolveDims& d, const SolverBuffers& b, cudaStream_t st) {
  ShiftParams p;
  p.d = d;
  p.rbuf = b.rbuf;
  p.pbuf = b.pbuf;
  p.G0 = b.G0;
  p.slots = b.slots;
  p.shifts = b.shifts;
  p.counters = b.counters;
  dim3 grid(d.K, d.W), block(256);
  if (fp64) shift_kernel<double><<<grid, block, 0, st>>>(p);
  else shift_kernel<float><<<grid, block, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_slot_init(bool fp64, const SolveDims& d, const SolverBuffers& b, int n_init, int seed0,
                             cudaStream_t st) {
  if (n_init <= 0) return cudaSuccess;
  InitParams p;
  p.d = d;
  p.rbuf = b.rbuf;
  p.pbuf = b.pbuf;
  p.G0 = b.G0;
  p.slots = b.slots;
  p.shifts = b.shifts;
  p.Z = b.Z;
  p.init_list = b.init_list;
  p.init_grid = b.init_grid;
  p.seed0 = seed0;
  long long work = d.N > (long long)d.K * d.nb ? d.N : (long long)d.K * d.nb;
  int gx = (int)((work + 255) / 256);
  if (gx > 256) gx = 256;
  dim3 grid(gx, n_init), block(256);
  if (fp64) init_kernel<double><<<grid, block, 0, st>>>(p);
  else init_kernel<float><<<grid, block, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace rsfd
