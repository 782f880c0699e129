// Shifted COCG kernels for sm_103a.
//
// Seed iteration (Appendix, Eqs. rvec, alpha, beta).  One fused pass per iteration and right-hand
// side ("slot") computes
//
//   r_n = a1 r_{n-1} + a2 r_{n-2} + aA (A r_{n-1}),     A = Z_s - H_T,
//   (r_n, r_n), (r_n, A r_n) (unconjugated bilinear form) and ||r_n||^2,
//
// on a 2.5D tile that marches along z.  Each CTA owns a 32-wide x-y tile of one slot and a range
// of z-planes.  A single thread streams every plane it needs with TMA (cp.async.bulk.tensor) into a
// shared-memory ring guarded by mbarriers, up to 7 planes ahead of the consumers: r_{n-1} on the tile
// plus a 2R halo, r_{n-2} and V_loc on the same box.  TMA's zero fill outside the tensor gives the
// Dirichlet walls and the zero ghosts in z for free.  The threads keep each grid column's
// z-neighbours in registers, evaluate A r_{n-1} and r_n on the tile plus R (the halo is recomputed
// instead of stored), then A r_n on the tile for the dot products, so an iteration moves three
// vectors through HBM.  The last CTA of a slot to finish (atomic ticket; nothing waits on another
// CTA) reduces the per-CTA partial sums in a fixed order and runs the FP64 scalar step: convergence
// of every energy, seed switching (Eq. seedswitch), alpha_n, beta_{n-1} and the shifted recurrences
// pi_{n+1}, alpha_n^(i), beta_{n-1}^(i) (Eqs. spi, salpha, sbeta).
//
// Shift update (Eq. endcollinear and the x^(i) update) on the boundary rows only, with
// r_n^(i) = r_n / pi_n^(s,i) (Eq. collinear).  The recurrences p <- cr_t r_t + cb_t p,
// x <- x + ca_t p are linear in the residuals r_t, so C consecutive steps collapse into
//   x <- x + e_x p + sum_t W_x[t] r_t,   p <- e_p p + sum_t W_p[t] r_t,
// with O(C) FP64 coefficients per energy.  The pass kernel records the boundary rows of r_n and the
// scalar step records (cr, cb, ca) per energy; every C iterations one kernel applies the collapsed
// update, which reads and writes x_b and p_b once per C iterations instead of every iteration.
//
// Precisions (template MODE):
//   RSFD_FP64  complex128 vectors, FP64 arithmetic.
//   RSFD_MIXED complex64 vectors, FP32 arithmetic (packed FFMA2), FP64 scalars and reductions.
//   RSFD_DF64  complex double-float vectors (hi + lo FP32 pairs, ~48-bit significands) with
//              error-free FP32 arithmetic and FP64 scalars; the recorded r_b history (input of the
//              collapsed shift update) keeps the hi parts.
//
// Every wait in this file is an mbarrier try_wait with an iteration cap; on expiry the CTA raises an
// error flag that the host turns into RSFD_ERR_TIMEOUT.  No CTA waits on another CTA.

#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>

#include "rsfd_internal.cuh"

namespace rsfd {
size_t pass_smem(int prec, int R, int tile_y, int depth);
int pass_threads(int R, int tile_y);
namespace {

constexpr int kTileX = 32;       // interior tile width in x
constexpr int kBoxX = 40;        // TMA box width in grid points (x0 - 4 ... x0 + 35)
constexpr int kBoxOff = 4;       // the box starts kBoxOff points left of the tile
constexpr int kMaxDepth = 7;     // bundles (one plane of each input) in flight ahead of the consumers
constexpr int kMaxStages = kMaxDepth + 1;
// threads per CTA of the pass kernel (fewer for double-float, which needs more registers per thread)
template <int MODE> struct MaxThreads { static constexpr int value = 512; };
template <> struct MaxThreads<RSFD_DF64> { static constexpr int value = 384; };
template <> struct MaxThreads<RSFD_FP64> { static constexpr int value = 384; };
constexpr long long kWaitCap = 1ll << 12;   // try_wait attempts before a wait is declared lost
constexpr uint32_t kWaitHintNs = 1000000;    // suspend-time hint of one attempt (1 ms): cap ~ 4 s

// ------------------------------------------------------------------------------------------------
// packed FP32x2 helpers
// ------------------------------------------------------------------------------------------------
// Packed adds and subtracts are written as FFMA2 with a +-1 multiplier held in constant memory:
// one issued instruction with the single rounding of an add.  (A packed add, or an FFMA2 whose
// multiplier the compiler can see is 1, costs two issue slots.)
__constant__ float2 c_one2 = {1.f, 1.f};
__constant__ float2 c_mone2 = {-1.f, -1.f};
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __ffma2_rn(a, c_one2, b); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __ffma2_rn(b, c_mone2, a); }
__device__ __forceinline__ float2 f2neg(float2 a) { return __fmul2_rn(a, c_mone2); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 bc(float a) { return make_float2(a, a); }

// complex double-float: value = h + l, component-wise (h = (re_hi, im_hi), l = (re_lo, im_lo))
struct __align__(16) dfc {
  float2 h, l;
};
struct dfr {   // real double-float coefficient
  float h, l;
};
struct dfz {   // complex double-float coefficient
  dfr re, im;
};

__host__ __device__ __forceinline__ dfr to_dfr(double v) {
  dfr r;
  r.h = (float)v;
  r.l = (float)(v - (double)r.h);
  return r;
}

// Knuth's TwoSum and Dekker's FastTwoSum on packed pairs (error-free transformations)
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = f2add(a, b);
  const float2 bb = f2sub(s, a);
  e = f2add(f2sub(a, f2sub(s, bb)), f2sub(b, bb));
}
__device__ __forceinline__ void fast_two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = f2add(a, b);
  e = f2sub(b, f2sub(s, a));
}
__device__ __forceinline__ dfc df_add(dfc x, dfc y) {
  float2 s, e;
  two_sum2(x.h, y.h, s, e);
  e = f2add(e, f2add(x.l, y.l));
  dfc r;
  fast_two_sum2(s, e, r.h, r.l);
  return r;
}
// acc + c * x for a real double-float c applied to both components (exact product via FMA)
__device__ __forceinline__ dfc df_mar(dfr c, dfc x, dfc acc) {
  const float2 ch = bc(c.h);
  const float2 p = f2mul(ch, x.h);
  float2 e = f2fma(ch, x.h, f2neg(p));
  e = f2fma(bc(c.l), x.h, e);
  e = f2fma(ch, x.l, e);
  dfc prod;
  fast_two_sum2(p, e, prod.h, prod.l);
  return df_add(prod, acc);
}
__device__ __forceinline__ dfc df_swapneg(dfc x) {   // i * x
  dfc r;
  r.h = make_float2(-x.h.y, x.h.x);
  r.l = make_float2(-x.l.y, x.l.x);
  return r;
}
__device__ __forceinline__ dfr dfr_sub(dfr a, float vh, float vl) {   // a - (vh + vl), scalar
  const float s = a.h - vh;
  const float bb = s - a.h;
  float e = (a.h - (s - bb)) + (-vh - bb);
  e += a.l - vl;
  dfr r;
  r.h = s + e;
  r.l = e - (r.h - s);
  return r;
}

// ------------------------------------------------------------------------------------------------
// precision policies
// ------------------------------------------------------------------------------------------------
template <int MODE> struct Ops;

template <> struct Ops<RSFD_MIXED> {
  typedef float2 C;     // Krylov vector element
  typedef float VT;     // potential element
  typedef float2 H;     // element of A r_n in the dot products and of the r_b history
  typedef float HR;     // scalar type of H
  typedef float Real;
  typedef float2 Cplx;
  static __device__ __forceinline__ C zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ C unit() { return make_float2(1.f, 0.f); }
  static __device__ __forceinline__ C add(C a, C b) { return f2add(a, b); }
  static __device__ __forceinline__ C mar(Real c, C x, C acc) { return f2fma(bc(c), x, acc); }
  static __device__ __forceinline__ C mac(Cplx z, C x, C acc) {
    acc = f2fma(bc(z.x), x, acc);
    return f2fma(make_float2(-z.y, z.y), make_float2(x.y, x.x), acc);
  }
  // acc + (zre - v + i zim) x
  static __device__ __forceinline__ C diag(Real zre, Real zim, VT v, C x, C acc) {
    return mac(make_float2(zre - v, zim), x, acc);
  }
  static __device__ __forceinline__ H hi(C x) { return x; }
  static __device__ __forceinline__ HR vhi(VT v) { return v; }
  static __host__ __device__ __forceinline__ Real real(double v) { return (float)v; }
  static __host__ __device__ __forceinline__ Cplx cplx(double2 z) { return make_float2((float)z.x, (float)z.y); }
};

template <> struct Ops<RSFD_FP64> {
  typedef double2 C;
  typedef double VT;
  typedef double2 H;
  typedef double HR;
  typedef double Real;
  typedef double2 Cplx;
  static __device__ __forceinline__ C zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ C unit() { return make_double2(1.0, 0.0); }
  static __device__ __forceinline__ C add(C a, C b) { return make_double2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ C mar(Real c, C x, C acc) { return make_double2(fma(c, x.x, acc.x), fma(c, x.y, acc.y)); }
  static __device__ __forceinline__ C mac(Cplx z, C x, C acc) {
    return make_double2(fma(z.x, x.x, fma(-z.y, x.y, acc.x)), fma(z.x, x.y, fma(z.y, x.x, acc.y)));
  }
  static __device__ __forceinline__ C diag(Real zre, Real zim, VT v, C x, C acc) {
    return mac(make_double2(zre - v, zim), x, acc);
  }
  static __device__ __forceinline__ H hi(C x) { return x; }
  static __device__ __forceinline__ HR vhi(VT v) { return v; }
  static __host__ __device__ __forceinline__ Real real(double v) { return v; }
  static __host__ __device__ __forceinline__ Cplx cplx(double2 z) { return z; }
};

template <> struct Ops<RSFD_DF64> {
  typedef dfc C;
  typedef float2 VT;    // (hi, lo) of V
  typedef float2 H;
  typedef float HR;
  typedef dfr Real;
  typedef dfz Cplx;
  static __device__ __forceinline__ C zero() {
    dfc r;
    r.h = make_float2(0.f, 0.f);
    r.l = r.h;
    return r;
  }
  static __device__ __forceinline__ C unit() {
    dfc r;
    r.h = make_float2(1.f, 0.f);
    r.l = make_float2(0.f, 0.f);
    return r;
  }
  static __device__ __forceinline__ C add(C a, C b) { return df_add(a, b); }
  static __device__ __forceinline__ C mar(Real c, C x, C acc) { return df_mar(c, x, acc); }
  static __device__ __forceinline__ C mac(Cplx z, C x, C acc) {
    return df_mar(z.re, x, df_mar(z.im, df_swapneg(x), acc));
  }
  static __device__ __forceinline__ C diag(Real zre, Real zim, VT v, C x, C acc) {
    return df_mar(dfr_sub(zre, v.x, v.y), x, df_mar(zim, df_swapneg(x), acc));
  }
  static __device__ __forceinline__ H hi(C x) { return x.h; }
  static __device__ __forceinline__ HR vhi(VT v) { return v.x; }
  static __host__ __device__ __forceinline__ Real real(double v) { return to_dfr(v); }
  static __host__ __device__ __forceinline__ Cplx cplx(double2 z) {
    dfz r;
    r.re = to_dfr(z.x);
    r.im = to_dfr(z.y);
    return r;
  }
};


// Unnormalised double-float accumulator: value = s + lo.  Adding a double-float or an exact
// product costs one TwoSum on the leading parts plus plain additions of the error terms; the pair
// is renormalised once (FastTwoSum) when the sum is complete.
struct DFAcc {
  float2 s, lo;
};
__device__ __forceinline__ DFAcc dfacc_zero() {
  DFAcc a;
  a.s = make_float2(0.f, 0.f);
  a.lo = a.s;
  return a;
}
__device__ __forceinline__ DFAcc dfacc_from(const dfc& x) {
  DFAcc a;
  a.s = x.h;
  a.lo = x.l;
  return a;
}
__device__ __forceinline__ void dfacc_add(DFAcc& a, const dfc& x) {
  float2 t, e;
  two_sum2(a.s, x.h, t, e);
  a.s = t;
  a.lo = f2add(a.lo, f2add(e, x.l));
}
// a += c x for a real double-float c (both components), exact leading product via FMA
__device__ __forceinline__ void dfacc_mul(DFAcc& a, dfr c, const dfc& x) {
  // ne = p - c x (exact leading part, then the low-order terms), accumulated with the opposite sign
  const float2 nch = bc(-c.h);
  const float2 p = f2mul(bc(c.h), x.h);
  float2 ne = f2fma(nch, x.h, p);
  ne = f2fma(nch, x.l, ne);
  ne = f2fma(bc(-c.l), x.h, ne);
  float2 t, te;
  two_sum2(a.s, p, t, te);
  a.s = t;
  a.lo = f2add(a.lo, f2sub(te, ne));
}
// a fresh accumulator holding c x (the exact leading product and its low-order terms)
__device__ __forceinline__ DFAcc dfacc_prod(dfr c, const dfc& x) {
  const float2 nch = bc(-c.h);
  const float2 p = f2mul(bc(c.h), x.h);
  float2 ne = f2fma(nch, x.h, p);
  ne = f2fma(nch, x.l, ne);
  ne = f2fma(bc(-c.l), x.h, ne);
  DFAcc a;
  a.s = p;
  a.lo = f2neg(ne);
  return a;
}
__device__ __forceinline__ dfc dfacc_get(const DFAcc& a) {
  dfc r;
  fast_two_sum2(a.s, a.lo, r.h, r.l);
  return r;
}

// A x at one point: (zre - v + i zim) x - hk1 (sum of the 6 neighbours at distance 1)
//                                       - hk2 (sum of the 6 neighbours at distance 2)
// and the seed-residual combination a1 r1 + a2 r2 + aA u, per precision.
template <int MODE, int R> struct Stencil;

template <int R> struct Stencil<RSFD_MIXED, R> {
  typedef Ops<RSFD_MIXED> O;
  static __device__ __forceinline__ float2 sum6(const float2 (&n)[6]) {
    return f2add(f2add(f2add(n[0], n[1]), f2add(n[2], n[3])), f2add(n[4], n[5]));
  }
  static __device__ __forceinline__ float2 applyA(float2 c, const float2 (&n1)[6], const float2 (&n2)[6], float v,
                                                  float zre, float zim, float mh1, float mh2) {
    float2 u = f2mul(bc(mh1), sum6(n1));
    if (R == 2) u = f2fma(bc(mh2), sum6(n2), u);
    return O::diag(zre, zim, v, c, u);
  }
  static __device__ __forceinline__ float2 combine(float2 a1, float2 r1, float2 a2, float2 r2, float2 aA, float2 u) {
    return O::mac(aA, u, O::mac(a2, r2, O::mac(a1, r1, O::zero())));
  }
};

template <int R> struct Stencil<RSFD_FP64, R> {
  typedef Ops<RSFD_FP64> O;
  static __device__ __forceinline__ double2 sum6(const double2 (&n)[6]) {
    return O::add(O::add(O::add(n[0], n[1]), O::add(n[2], n[3])), O::add(n[4], n[5]));
  }
  static __device__ __forceinline__ double2 applyA(double2 c, const double2 (&n1)[6], const double2 (&n2)[6],
                                                   double v, double zre, double zim, double mh1, double mh2) {
    double2 u = O::mar(mh1, sum6(n1), O::zero());
    if (R == 2) u = O::mar(mh2, sum6(n2), u);
    return O::diag(zre, zim, v, c, u);
  }
  static __device__ __forceinline__ double2 combine(double2 a1, double2 r1, double2 a2, double2 r2, double2 aA,
                                                    double2 u) {
    return O::mac(aA, u, O::mac(a2, r2, O::mac(a1, r1, O::zero())));
  }
};

template <int R> struct Stencil<RSFD_DF64, R> {
  static __device__ __forceinline__ dfc sum6(const dfc (&n)[6]) {
    DFAcc a = dfacc_from(n[0]);
#pragma unroll
    for (int k = 1; k < 6; ++k) dfacc_add(a, n[k]);
    return dfacc_get(a);
  }
  static __device__ __forceinline__ dfc applyA(const dfc& c, const dfc (&n1)[6], const dfc (&n2)[6], float2 v,
                                               dfr zre, dfr zim, dfr mh1, dfr mh2) {
    DFAcc a = dfacc_prod(mh1, sum6(n1));
    if (R == 2) dfacc_mul(a, mh2, sum6(n2));
    dfacc_mul(a, dfr_sub(zre, v.x, v.y), c);
    dfacc_mul(a, zim, df_swapneg(c));
    return dfacc_get(a);
  }
  static __device__ __forceinline__ dfc combine(const dfz& a1, const dfc& r1, const dfz& a2, const dfc& r2,
                                                const dfz& aA, const dfc& u) {
    DFAcc a = dfacc_prod(a1.re, r1);
    dfacc_mul(a, a1.im, df_swapneg(r1));
    dfacc_mul(a, a2.re, r2);
    dfacc_mul(a, a2.im, df_swapneg(r2));
    dfacc_mul(a, aA.re, u);
    dfacc_mul(a, aA.im, df_swapneg(u));
    return dfacc_get(a);
  }
};

// s A x at one point for the block-floating-point split pass (double-float vectors whose leading
// parts are multiples of one quantum q, each at most 2^21 q), with s = 24 h^2 (R = 2) or 2 h^2 (R = 1):
//   s A x = 16 S1 - S2 + d x  (R = 2),   S1 + d x  (R = 1),   d = s (Z_s - hd - V) (complex),
// S1, S2 the sums of the six neighbours at distance 1 and 2.  The neighbour sums of the leading parts
// are exact FP32 additions (every partial sum is a multiple of q below 6 * 2^21 q < 2^24 q), 16 S1h
// is exact and one TwoSum forms 16 S1h - S2h; the trailing parts are summed plainly; d x takes exact
// products (FMA) and two more TwoSums join the terms.
template <int R> struct StencilBFP {
  static __device__ __forceinline__ float2 sum6h(const dfc (&n)[6]) {
    return f2add(f2add(f2add(n[0].h, n[1].h), f2add(n[2].h, n[3].h)), f2add(n[4].h, n[5].h));
  }
  static __device__ __forceinline__ float2 sum6l(const dfc (&n)[6]) {
    return f2add(f2add(f2add(n[0].l, n[1].l), f2add(n[2].l, n[3].l)), f2add(n[4].l, n[5].l));
  }
  // zre = s (Re Z_s - hd), zim = s Im Z_s (double-float scalars), vs = s V at the point
  static __device__ __forceinline__ dfc applyA(const dfc& c, const dfc (&n1)[6], const dfc (&n2)[6], float2 vs,
                                               dfr zre, float2 zim_h, float2 zim_l) {
    // L = 16 S1 - S2 (R = 2) or S1 (R = 1) as a leading part Lh and a trailing part Ll
    float2 Lh, Ll;
    if (R == 2) {
      float2 le;
      two_sum2(f2mul(bc(16.f), sum6h(n1)), f2neg(sum6h(n2)), Lh, le);
      Ll = f2sub(f2fma(bc(16.f), sum6l(n1), le), sum6l(n2));
    } else {
      Lh = sum6h(n1);
      Ll = sum6l(n1);
    }
    // P1 = dre x, dre = zre - vs (real double-float): p1 - ne1 exactly (up to the lo*lo term)
    const dfr dre = dfr_sub(zre, vs.x, vs.y);
    const float2 dh = bc(dre.h), ndh = bc(-dre.h);
    const float2 p1 = f2mul(dh, c.h);
    float2 ne1 = f2fma(ndh, c.h, p1);
    ne1 = f2fma(ndh, c.l, ne1);
    ne1 = f2fma(bc(-dre.l), c.h, ne1);
    // P2 = i zim x = zim (-x.im, x.re): zim_h = (-zim.h, zim.h), zim_l = (-zim.l, zim.l)
    const float2 sh = make_float2(c.h.y, c.h.x), sl = make_float2(c.l.y, c.l.x);
    const float2 p2 = f2mul(zim_h, sh);
    float2 ne2 = f2fma(f2neg(zim_h), sh, p2);
    ne2 = f2fma(f2neg(zim_h), sl, ne2);
    ne2 = f2fma(f2neg(zim_l), sh, ne2);
    // u = p1 + p2 +- Lh + (lo terms)
    float2 s1, t1, s2, t2;
    two_sum2(p1, p2, s1, t1);
    two_sum2(s1, Lh, s2, t2);
    float2 lo = f2add(t1, t2);
    lo = f2sub(lo, ne1);
    lo = f2sub(lo, ne2);
    lo = f2add(lo, Ll);
    dfc u;
    fast_two_sum2(s2, lo, u.h, u.l);
    return u;
  }
};

template <class T> struct Pair {
  T a, b;
};

// arithmetic on the "hi" element H (A r_n for the dot products, history, collapsed update)
template <typename HR> struct HOps;
template <> struct HOps<float> {
  typedef float2 H;
  static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ float2 add(float2 a, float2 b) { return f2add(a, b); }
  static __device__ __forceinline__ float2 mar(float c, float2 x, float2 acc) { return f2fma(bc(c), x, acc); }
  static __device__ __forceinline__ float2 mac(float2 z, float2 x, float2 acc) {
    acc = f2fma(bc(z.x), x, acc);
    return f2fma(make_float2(-z.y, z.y), make_float2(x.y, x.x), acc);
  }
  static __device__ __forceinline__ float2 diag(float zre, float zim, float v, float2 x, float2 acc) {
    return mac(make_float2(zre - v, zim), x, acc);
  }
  static __device__ __forceinline__ float2 from(double2 z) { return make_float2((float)z.x, (float)z.y); }
};
template <> struct HOps<double> {
  typedef double2 H;
  static __device__ __forceinline__ double2 zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ double2 mar(double c, double2 x, double2 acc) {
    return make_double2(fma(c, x.x, acc.x), fma(c, x.y, acc.y));
  }
  static __device__ __forceinline__ double2 mac(double2 z, double2 x, double2 acc) {
    return make_double2(fma(z.x, x.x, fma(-z.y, x.y, acc.x)), fma(z.x, x.y, fma(z.y, x.x, acc.y)));
  }
  static __device__ __forceinline__ double2 diag(double zre, double zim, double v, double2 x, double2 acc) {
    return mac(make_double2(zre - v, zim), x, acc);
  }
  static __device__ __forceinline__ double2 from(double2 z) { return z; }
};

// Per-thread dot-product accumulators: (r,r), (r,Ar) unconjugated and ||r||^2.
template <typename HR> struct Acc;

template <> struct Acc<double> {
  double rr_x = 0, rr_y = 0, ra_x = 0, ra_y = 0, nn = 0;
  __device__ __forceinline__ void add(double2 r, double2 v) {
    rr_x = fma(r.x, r.x, fma(-r.y, r.y, rr_x));
    rr_y = fma(2.0 * r.x, r.y, rr_y);
    ra_x = fma(r.x, v.x, fma(-r.y, v.y, ra_x));
    ra_y = fma(r.x, v.y, fma(r.y, v.x, ra_y));
    nn = fma(r.x, r.x, fma(r.y, r.y, nn));
  }
  // the split pass forms (r,r) and ||r||^2 where r_n is produced and (r,Ar) where A r_n is
  __device__ __forceinline__ void add_r(double2 r) {
    rr_x = fma(r.x, r.x, fma(-r.y, r.y, rr_x));
    rr_y = fma(2.0 * r.x, r.y, rr_y);
    nn = fma(r.x, r.x, fma(r.y, r.y, nn));
  }
  __device__ __forceinline__ void add_ra(double2 r, double2 v) {
    ra_x = fma(r.x, v.x, fma(-r.y, v.y, ra_x));
    ra_y = fma(r.x, v.y, fma(r.y, v.x, ra_y));
  }
  // warp sums (whole warps only); lane 0 returns them, the other lanes zeros
  __device__ __forceinline__ void get(double* o) const {
    double t[5] = {rr_x, rr_y, ra_x, ra_y, nn};
    const bool lead = (threadIdx.x & 31) == 0;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      for (int off = 16; off > 0; off >>= 1) t[k] += __shfl_down_sync(0xffffffffu, t[k], off);
      o[k] = lead ? t[k] : 0.0;
    }
  }
};

// FP32-based accumulators (complex64 and double-float vectors).  The unconjugated forms cancel
// heavily and the COCG scalars are sensitive to them (FP32-rounded products double the iteration
// count at eta = 1e-3), so every product is formed exactly with an FMA (plus the cross terms of the
// low parts) and summed into a double-float accumulator with TwoSum.  ||r||^2 has no cancellation
// and is summed plainly from the leading parts.
struct AccDF {
  float2 rr_s = make_float2(0.f, 0.f), rr_l = make_float2(0.f, 0.f);
  float2 ra_s = make_float2(0.f, 0.f), ra_l = make_float2(0.f, 0.f);
  float nn = 0.f;
  // (s, l) += (a + al) * (b + bl), component-wise, without the al*bl term
  static __device__ __forceinline__ void addprod(float2& s, float2& l, float2 a, float2 al, float2 b, float2 bl) {
    const float2 na = f2neg(a);
    const float2 p = f2mul(a, b);
    float2 ne = f2fma(na, b, p);          // p - a b, exact
    ne = f2fma(na, bl, ne);
    ne = f2fma(f2neg(al), b, ne);
    float2 t, te;
    two_sum2(s, p, t, te);
    s = t;
    l = f2add(l, f2sub(te, ne));
  }
  // r*r = (x x - y y, x y + y x);  r*v = (x a - y b, x b + y a)
  __device__ __forceinline__ void add2(float2 rh, float2 rl, float2 vh, float2 vl) {
    const float2 xh = bc(rh.x), xl = bc(rl.x);
    const float2 ny = make_float2(-rh.y, rh.y), nyl = make_float2(-rl.y, rl.y);
    addprod(rr_s, rr_l, xh, xl, rh, rl);
    addprod(rr_s, rr_l, ny, nyl, make_float2(rh.y, rh.x), make_float2(rl.y, rl.x));
    addprod(ra_s, ra_l, xh, xl, vh, vl);
    addprod(ra_s, ra_l, ny, nyl, make_float2(vh.y, vh.x), make_float2(vl.y, vl.x));
    nn = __fmaf_rn(rh.x, rh.x, __fmaf_rn(rh.y, rh.y, nn));
  }
  __device__ __forceinline__ void add(const dfc& r, const dfc& v) { add2(r.h, r.l, v.h, v.l); }
  __device__ __forceinline__ void add_r(const dfc& r) {
    const float2 rh = r.h, rl = r.l;
    addprod(rr_s, rr_l, bc(rh.x), bc(rl.x), rh, rl);
    addprod(rr_s, rr_l, make_float2(-rh.y, rh.y), make_float2(-rl.y, rl.y), make_float2(rh.y, rh.x),
            make_float2(rl.y, rl.x));
    nn = __fmaf_rn(rh.x, rh.x, __fmaf_rn(rh.y, rh.y, nn));
  }
  __device__ __forceinline__ void add_ra(const dfc& r, const dfc& v) {
    const float2 rh = r.h, rl = r.l;
    addprod(ra_s, ra_l, bc(rh.x), bc(rl.x), v.h, v.l);
    addprod(ra_s, ra_l, make_float2(-rh.y, rh.y), make_float2(-rl.y, rl.y), make_float2(v.h.y, v.h.x),
            make_float2(v.l.y, v.l.x));
  }
  static __device__ __forceinline__ float2 shfl2(float2 v, int o) {
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, o), __shfl_down_sync(0xffffffffu, v.y, o));
  }
  static __device__ __forceinline__ void merge(float2& s, float2& l, float2 os, float2 ol) {
    float2 t, te;
    two_sum2(s, os, t, te);
    s = t;
    l = f2add(l, f2add(te, ol));
  }
  // Reduce over the warp in double-float (whole warps only), then convert once per warp: lane 0
  // returns the warp's sums in FP64, the other lanes zeros.
  __device__ __forceinline__ void get(double* o) {
    for (int off = 16; off > 0; off >>= 1) {
      const float2 a = shfl2(rr_s, off), b = shfl2(rr_l, off), c = shfl2(ra_s, off), d = shfl2(ra_l, off);
      merge(rr_s, rr_l, a, b);
      merge(ra_s, ra_l, c, d);
    }
    for (int off = 16; off > 0; off >>= 1) nn += __shfl_down_sync(0xffffffffu, nn, off);
    const double nnd = (double)nn;
    const bool lead = (threadIdx.x & 31) == 0;
    o[0] = lead ? (double)rr_s.x + (double)rr_l.x : 0.0;
    o[1] = lead ? (double)rr_s.y + (double)rr_l.y : 0.0;
    o[2] = lead ? (double)ra_s.x + (double)ra_l.x : 0.0;
    o[3] = lead ? (double)ra_s.y + (double)ra_l.y : 0.0;
    o[4] = lead ? nnd : 0.0;
  }
};

// complex64 vectors: rounded FP32 products with Kahan-compensated sums.  This mode is meant for the
// regime where eps_32 * kappa is small (its SpMV error floor is eps_32 * kappa); there the rounded
// products do not slow convergence, and they cost a fifth of the exact-product form.
struct AccK {
  float2 rr = make_float2(0.f, 0.f), rr_c = make_float2(0.f, 0.f);
  float2 ra = make_float2(0.f, 0.f), ra_c = make_float2(0.f, 0.f);
  float nn = 0.f;
  static __device__ __forceinline__ void kahan(float2& s, float2& c, float2 term) {
    const float2 y = f2sub(term, c);
    const float2 t = f2add(s, y);
    c = f2sub(f2sub(t, s), y);
    s = t;
  }
  __device__ __forceinline__ void add(float2 r, float2 v) {
    const float2 trr = make_float2(__fmaf_rn(r.x, r.x, -r.y * r.y), 2.f * r.x * r.y);
    const float2 tra = make_float2(__fmaf_rn(r.x, v.x, -r.y * v.y), __fmaf_rn(r.x, v.y, r.y * v.x));
    kahan(rr, rr_c, trr);
    kahan(ra, ra_c, tra);
    nn = __fmaf_rn(r.x, r.x, __fmaf_rn(r.y, r.y, nn));
  }
  __device__ __forceinline__ void add_r(float2 r) {
    kahan(rr, rr_c, make_float2(__fmaf_rn(r.x, r.x, -r.y * r.y), 2.f * r.x * r.y));
    nn = __fmaf_rn(r.x, r.x, __fmaf_rn(r.y, r.y, nn));
  }
  __device__ __forceinline__ void add_ra(float2 r, float2 v) {
    kahan(ra, ra_c, make_float2(__fmaf_rn(r.x, v.x, -r.y * v.y), __fmaf_rn(r.x, v.y, r.y * v.x)));
  }
  // The Kahan pairs (s, -c) are double-float values: reduce them over the warp with TwoSum merges
  // (whole warps only) and convert once; lane 0 returns the warp's sums, the other lanes zeros.
  __device__ __forceinline__ void get(double* o) {
    float2 rl = f2neg(rr_c), al = f2neg(ra_c);
    for (int off = 16; off > 0; off >>= 1) {
      const float2 a = AccDF::shfl2(rr, off), b = AccDF::shfl2(rl, off), c = AccDF::shfl2(ra, off),
                   e = AccDF::shfl2(al, off);
      AccDF::merge(rr, rl, a, b);
      AccDF::merge(ra, al, c, e);
      nn += __shfl_down_sync(0xffffffffu, nn, off);
    }
    const bool lead = (threadIdx.x & 31) == 0;
    o[0] = lead ? (double)rr.x + (double)rl.x : 0.0;
    o[1] = lead ? (double)rr.y + (double)rl.y : 0.0;
    o[2] = lead ? (double)ra.x + (double)al.x : 0.0;
    o[3] = lead ? (double)ra.y + (double)al.y : 0.0;
    o[4] = lead ? (double)nn : 0.0;
  }
};

template <int MODE> struct AccOf { typedef AccDF type; };
template <> struct AccOf<RSFD_MIXED> { typedef AccK type; };
template <> struct AccOf<RSFD_FP64> { typedef Acc<double> type; };

// index of plane z among the recorded planes (boundary planes, then the tracked interior planes),
// -1 when its rows are not recorded
__device__ __forceinline__ int recorded_plane(const SolveDims& d, int z) {
  if (z < d.nface) return z;
  if (z >= d.nz - d.nface) return z - d.nz + 2 * d.nface;
  int pl = -1;
#pragma unroll 4
  for (int e = 0; e < d.ntrack; ++e)
    if (d.track[e] == z) pl = 2 * d.nface + e;
  return pl;
}

// ------------------------------------------------------------------------------------------------
// mbarrier / TMA primitives (inline PTX)
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Bounded wait for the phase with the given parity; false when the cap is reached (cap attempts).  Each try_wait
// carries a suspend-time hint, so a waiting thread sleeps until the phase completes (or the hint
// expires) instead of spinning through issue slots.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long cap = kWaitCap) {
  for (long long i = 0; i < cap; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(kWaitHintNs)
        : "memory");
    if (ok) return true;
  }
  return false;
}
// attempts of a pass's first wait on each bundle (the solve's wait_cap option; drains keep kWaitCap)
__device__ __forceinline__ long long first_wait_cap(const SolveDims& d) {
  return d.wait_cap == 0 ? kWaitCap : (d.wait_cap < 0 ? 0ll : (long long)d.wait_cap);
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// ------------------------------------------------------------------------------------------------
// reductions (FP64)
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
// Sum over the block of per-warp values held by lane 0 of each warp (the accumulators' get() leaves
// the warp sums there); fixed order over the warps.  The sums are valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum_lane0(double (&v)[NV], double* s_red) {
  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) s_red[wid * NV + k] = v[k];
  }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += s_red[w * NV + k];
      v[k] = t;
    }
  }
  __syncthreads();
}
// Largest of a non-negative per-thread value over the block, valid in thread 0 (order-free).
__device__ __forceinline__ float block_max0(float v, float* s_red) {
  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) s_red[wid] = v;
  __syncthreads();
  if (tid == 0)
    for (int w = 0; w < nw; ++w) v = fmaxf(v, s_red[w]);
  __syncthreads();
  return v;
}

struct PassParams {
  SolveDims d;
  void* rbuf;                // [W][nvec][Nz][Ny][Nxp] C
  const void* V;             // [Nz][Ny][Nxp] potential (VT)
  void* rhist;               // [W][hist_len][nb] H
  SlotState* slots;
  ShiftState* shifts;
  ShiftCoef* coef;           // [W][K][hist_len]
  double* partials;
  unsigned int* tickets;
  const double2* Z;
  unsigned long long* counters;
  int* error_flag;
  double hd;
  double hk1, hk2;
  double tol;
  int maxit;
  int hist_len;
  int depth;                 // TMA bundles in flight ahead of the consumers (1 .. kMaxDepth)
  int stored_u;              // 1: the pass reads the stored A r_{n-1} (seed switches fold the energy
                             //    shift of the stored product into a1)
  int has_proj;              // 1: nonlocal projectors; the pass leaves its dots in pdots and the
                             //    projector kernel finishes A r_n, the dots and the scalar step
  double* pdots;
  // block-floating-point split pass: the stencil stores u = s A r; the combine multiplies it by
  // aA / s (aA is stored so) and rounds the leading parts of r_n to the slot's quantum q; partial
  // entries 5 and 6 carry the largest leading-part components of r_n and of u_n
  int bfp;
  int kb;                    // leading parts are at most 2^kb q (21)
  double uscale;             // s (1 for the other forms)
  const void* Vs;            // s V, (hi, lo) floats
};

// Quantum of the block-floating-point leading parts for a bound B on every component of the next
// r_n: the power of two q with B < 2^kb q (clamped to a normal FP32 range).
__device__ __forceinline__ double bfp_quantum(double B, int kb) {
  if (!(B > 0.0) || !(B < 1e300)) return ldexp(1.0, -100);
  int e;
  frexp(B * (1.0 + 0x1p-20), &e);   // B (1 + 2^-20) < 2^e
  int ex = e - kb;
  if (ex < -100) ex = -100;
  if (ex > 100) ex = 100;
  return ldexp(1.0, ex);
}

// ------------------------------------------------------------------------------------------------
// FP64 scalar step of one slot (run by the last CTA of the slot)
// ------------------------------------------------------------------------------------------------
struct ScalarShared {
  double2 rr, rAr;
  double nrm2;
  double2 beta, alpha, c, scale_n, scale_nm1, fn, fnm1, Zs;
  double maxr, maxu;   // block-floating-point split pass: largest leading-part components of r_n, s A r_n
  int stop;
  int do_switch;
  int seed;
  int n;
  int hc;
  double red[32 * 5];
  int ired[32 * 2];
};

__device__ void scalar_step(const PassParams& p, int slot, ScalarShared& S) {
  const int tid = threadIdx.x;
  const int nthr = blockDim.x;
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
      if (i < p.d.kreq) ++cnt;   // auxiliary seed energies do not keep the column running
      if (res > best) { best = res; best_i = i; }
    }
  }
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
        if (!(rabs > 1e-300) || rabs <= p.d.brk_tol * nrm2s) {
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
      S.hc = st->hcnt;
    }
    __syncthreads();
  }
  if (S.stop) return;

  // Phase C: shifted recurrences for every active energy (Eqs. spi, salpha, sbeta) and the
  // coefficients of p_n^(i) = r_n / pi_n + beta_{n-1}^(i) p_{n-1}^(i), x_{n+1}^(i) = x_n^(i) +
  // alpha_n^(i) p_n^(i), recorded for the collapsed shift update (zero for converged energies).
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  ShiftCoef* cf = p.coef + (size_t)slot * K * p.hist_len;
  for (int i = tid; i < K; i += nthr) {
    ShiftState& q = sh[i];
    ShiftCoef e;
    if (!q.active) {
      e.cr = e.cb = e.ca = zero;
      cf[(size_t)i * p.hist_len + S.hc] = e;
      continue;
    }
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
    e.cr = cdiv(S.scale_n, pin);
    e.cb = beta_i;
    e.ca = alpha_i;
    cf[(size_t)i * p.hist_len + S.hc] = e;
    q.alpha_prev = alpha_i;
    q.pi_nm1 = pin;
    q.pi_n = pinp1;
  }
  if (tid == 0) {
    const double2 c = S.c;
    double2 a1 = cmul(cadd(one, c), S.scale_n);
    if (p.stored_u && S.do_switch) {
      // the stored product is A r_n with the previous seed's energy: A~ r_n = A r_n + (Z_s~ - Z_s) r_n
      a1 = csub(a1, cmul(cmul(S.alpha, S.scale_n), csub(S.Zs, st->Zs)));
    }
    st->a1 = a1;
    st->a2 = cmul(make_double2(-c.x, -c.y), S.scale_nm1);
    st->aA = cscale(1.0 / p.uscale, cmul(make_double2(-S.alpha.x, -S.alpha.y), S.scale_n));
    if (p.bfp) {
      // bound on every component of the next r_n = a1 r_n + a2 r_{n-1} + aA (s A r_n) from the
      // largest components of the stored vectors (|Re(a x)|, |Im(a x)| <= (|a.x| + |a.y|) max)
      const double2 a2 = st->a2, aA = st->aA;
      const double B = (fabs(a1.x) + fabs(a1.y)) * S.maxr + (fabs(a2.x) + fabs(a2.y)) * st->mr_prev +
                       (fabs(aA.x) + fabs(aA.y)) * S.maxu;
      st->mr_prev = S.maxr;
      st->q = bfp_quantum(B, p.kb);
    }
    st->Zs = S.Zs;
    st->seed = S.seed;
    st->alpha_prev = S.alpha;
    st->rr_prev = S.rr;
    st->carry = S.scale_n;   // r_n becomes the next step's r_{n-1}
    st->k4_n = S.n;
    st->hcnt = S.hc + 1;
    st->n = S.n + 1;
    atomicAdd(&p.counters[1], 1ull);
  }
}

// Per-CTA partial sums (lane 0 of each warp holds its warp's sums) -> the slot's partial array ->
// atomic ticket; the last of the slot's ctas_per_slot CTAs sums all npart partials of the slot in
// order (warp 0, fixed tree; the split pass's combine kernel has left its partials in entries
// ctas_per_slot ...) and returns true with (r,r), (r,Ar), ||r||^2 in S.  No CTA waits on another.
__device__ bool pass_finish(const PassParams& p, int slot, int cta, double (&v5)[5], ScalarShared& S, int& s_last,
                            float mxu = 0.f) {
  const int tid = threadIdx.x;
  block_sum_lane0<5>(v5, S.red);
  if (p.bfp) mxu = block_max0(mxu, reinterpret_cast<float*>(S.red));
  if (tid == 0) {
    double* dst = p.partials + ((size_t)slot * p.d.npart + cta) * 8;
#pragma unroll
    for (int k = 0; k < 5; ++k) dst[k] = v5[k];
    if (p.bfp) {
      dst[5] = 0.0;
      dst[6] = (double)mxu;
    }
    __threadfence();
    const unsigned int t = atomicAdd(p.tickets + slot, 1u);
    s_last = (t == (unsigned int)(p.d.ctas_per_slot - 1));
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  if (tid < 32) {
    double w5[5] = {0, 0, 0, 0, 0};
    const double* src = p.partials + (size_t)slot * p.d.npart * 8;
    for (int k = tid; k < p.d.npart; k += 32) {
#pragma unroll
      for (int j = 0; j < 5; ++j) w5[j] += __ldcg(src + (size_t)k * 8 + j);
    }
#pragma unroll
    for (int j = 0; j < 5; ++j) w5[j] = warp_sum(w5[j]);
    double mr = 0.0, mu = 0.0;
    if (p.bfp) {
      for (int k = tid; k < p.d.npart; k += 32) {
        mr = fmax(mr, __ldcg(src + (size_t)k * 8 + 5));
        mu = fmax(mu, __ldcg(src + (size_t)k * 8 + 6));
      }
      for (int o = 16; o > 0; o >>= 1) {
        mr = fmax(mr, __shfl_xor_sync(0xffffffffu, mr, o));
        mu = fmax(mu, __shfl_xor_sync(0xffffffffu, mu, o));
      }
    }
    if (tid == 0) {
      S.rr = make_double2(w5[0], w5[1]);
      // the block-floating-point split pass sums (r, s A r)
      S.rAr = p.uscale != 1.0 ? cscale(1.0 / p.uscale, make_double2(w5[2], w5[3])) : make_double2(w5[2], w5[3]);
      S.nrm2 = w5[4];
      S.maxr = mr;
      S.maxu = mu;
      p.tickets[slot] = 0u;
    }
  }
  __syncthreads();
  return true;
}

// ------------------------------------------------------------------------------------------------
// the fused pass
// ------------------------------------------------------------------------------------------------
template <int MODE, int R>
__global__ void __launch_bounds__(MaxThreads<MODE>::value) pass_kernel(PassParams p, const __grid_constant__ CUtensorMap tmR,
                                                           const __grid_constant__ CUtensorMap tmV) {
  typedef Ops<MODE> O;
  typedef Stencil<MODE, R> ST;
  typedef typename O::C C;
  typedef typename O::VT VT;
  typedef typename O::H H;
  typedef Pair<C> PC;
  typedef Pair<VT> PV;
  extern __shared__ unsigned char smem_raw[];
  __shared__ ScalarShared S;
  __shared__ int s_last, s_abort[2];   // abort flags indexed by step parity (set before, read after a barrier)
  __shared__ __align__(8) unsigned long long bars[kMaxStages];

  const int slot = blockIdx.y;
  SlotState* st = p.slots + slot;
  if (st->status != SLOT_RUNNING) return;
  const int kDepth = p.depth;
  const int kStages = kDepth + 1;

  // Each thread owns two x-adjacent grid points ("a pair").  Pairs of the middle region cover
  // x in [x0 - 2, x0 + 34) (18 pairs) and y in [y0 - R, y0 + TY + R); the tile proper is pairs
  // 1..16 and rows R..MY-R-1.
  const SolveDims& d = p.d;
  const int TY = d.tile_y;
  const int EY = TY + 4 * R;
  constexpr int MXP = 18;              // pairs per middle row
  constexpr int BXP = kBoxX / 2;       // pairs per box row (20)
  const int MY = TY + 2 * R;
  const int tid = threadIdx.x;
  const int cta = blockIdx.x;
  const int tz = cta % d.nzchunks;
  const int txy = cta / d.nzchunks;
  const int tx = txy % d.tiles_x, ty = txy / d.tiles_x;
  const int z0 = tz * d.zchunk;
  const int z1 = min(z0 + d.zchunk, d.nz);
  const int x0 = tx * kTileX, y0 = ty * TY;
  const bool act = tid < MXP * MY;
  const int px = tid % MXP, my = tid / MXP;
  const int gxa = x0 - 2 + 2 * px, gy = y0 - R + my;
  const bool yin = act && gy >= 0 && gy < d.ny;
  const bool ina = yin && gxa >= 0 && gxa < d.nx;
  const bool inb = yin && gxa + 1 >= 0 && gxa + 1 < d.nx;
  const bool is_int = act && px >= 1 && px < MXP - 1 && my >= R && my < MY - R;
  const int sidx = (my + R) * BXP + (px + 1);
  const long long plane_elems = (long long)d.nxp * d.ny;

  // shared-memory rings (128-byte aligned planes): RA r_{n-1}, RB r_{n-2}, VV V_loc, SB r_n
  const int NA = R + 1 + kDepth;
  const int NSB = R + 2;
  const size_t PCb = (size_t)kBoxX * EY * sizeof(C);          // bytes of one box (TMA transaction size)
  const size_t PVb = (size_t)kBoxX * EY * sizeof(VT);
  const int PEC = (int)(((PCb + 127) & ~(size_t)127) / sizeof(PC));    // plane stride in pairs
  const int PEV = (int)(((PVb + 127) & ~(size_t)127) / sizeof(PV));
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  PC* RA = (PC*)base;
  PC* RB = RA + (size_t)NA * PEC;
  PV* VV = (PV*)(RB + (size_t)kStages * PEC);
  PC* SB = (PC*)(VV + (size_t)kStages * PEV);

  // pass coefficients in the working precision, converted once per CTA (FP64 is slow on this GPU)
  struct Coefs {
    typename O::Cplx a1, a2, aA;
    typename O::Real zre, zim, mh1, mh2;
    int n, hc;
  };
  __shared__ Coefs sc;
  if (threadIdx.x == 0) {
    sc.a1 = O::cplx(st->a1);
    sc.a2 = O::cplx(st->a2);
    sc.aA = O::cplx(st->aA);
    const double2 Zs0 = st->Zs;
    sc.zre = O::real(Zs0.x - p.hd);
    sc.zim = O::real(Zs0.y);
    sc.mh1 = O::real(-p.hk1);
    sc.mh2 = O::real(-p.hk2);
    sc.n = st->n;
    sc.hc = st->hcnt;
  }
  __syncthreads();
  const int n = sc.n;
  const int b1 = (n + 2) % 3, b2 = (n + 1) % 3, bo = n % 3;
  C* rout = reinterpret_cast<C*>(p.rbuf) + ((size_t)slot * 3 + bo) * d.nz * plane_elems;   // nvec = 3
  const typename O::Cplx a1 = sc.a1, a2 = sc.a2, aA = sc.aA;
  const typename O::Real zre = sc.zre, zim = sc.zim, mh1 = sc.mh1, mh2 = sc.mh2;
  const int hc = sc.hc;
  H* hist = reinterpret_cast<H*>(p.rhist) + ((size_t)slot * p.hist_len + hc) * d.nb;
  const long long nxy = (long long)d.nx * d.ny;

  // TMA geometry: tensor-map elements per grid point along x
  constexpr int mR = (MODE == RSFD_DF64) ? 4 : 2;   // floats (doubles for FP64) per r element
  constexpr int mV = (MODE == RSFD_DF64) ? 2 : 1;
  const int xr = mR * (x0 - kBoxOff), xv = mV * (x0 - kBoxOff), yb = y0 - 2 * R;
  const uint32_t bundle_bytes = (uint32_t)(2 * PCb + PVb);
  const int nsteps = (z1 - z0) + 4 * R;
  const int rbuf1 = slot * 3 + b1, rbuf2 = slot * 3 + b2;

  auto issue = [&](int bnd) {
    const int q = z0 - 2 * R + bnd, c = q - R;
    const uint32_t bar = smem_u32(&bars[bnd % kStages]);
    mbar_expect_tx(bar, bundle_bytes);
    tma_load_4d(smem_u32(RA + (size_t)(bnd % NA) * PEC), &tmR, xr, yb, q, rbuf1, bar);
    tma_load_4d(smem_u32(RB + (size_t)(bnd % kStages) * PEC), &tmR, xr, yb, c, rbuf2, bar);
    tma_load_3d(smem_u32(VV + (size_t)(bnd % kStages) * PEV), &tmV, xv, yb, c, bar);
  };

  if (tid == 0) {
    for (int k = 0; k < kStages; ++k) mbar_init(smem_u32(&bars[k]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    s_abort[0] = s_abort[1] = 0;
  }
  __syncthreads();
  int issued = 0, s_fail = 0;
  if (tid == 0) {
    for (int bnd = 0; bnd < kDepth && bnd < nsteps; ++bnd) issue(bnd);
    issued = min(kDepth, nsteps);
  }

  // z-queues of this thread's pair: r_{n-1} on planes c-R..c+R, r_n on planes c-2R..c, V on c-2R..c
  PC qa[2 * R + 1], qb[2 * R + 1];
  PV vq[2 * R + 1];
  const C zc = O::zero();
#pragma unroll
  for (int k = 0; k <= 2 * R; ++k) {
    qa[k].a = zc; qa[k].b = zc;
    qb[k].a = zc; qb[k].b = zc;
    vq[k].a = VT(); vq[k].b = VT();
  }
  typename AccOf<MODE>::type acc;
  // ring positions, advanced incrementally: ia = s % NA, ic = (s - R) % NA, ist = s % kStages,
  // par = (s / kStages) & 1, isb = c % NSB, isv = (c - R) % NSB
  int ia = 0, ic = NA - R, ist = 0, par = 0;
  int isb = (((z0 - 3 * R) % NSB) + NSB) % NSB;
  int isv = (((z0 - 4 * R) % NSB) + NSB) % NSB;

  for (int s = 0; s < nsteps; ++s) {
    if (tid == 0 && s + kDepth < nsteps) {
      issue(s + kDepth);
      issued = s + kDepth + 1;
    }
    if (!mbar_wait(smem_u32(&bars[ist]), (uint32_t)par, first_wait_cap(p.d))) {
      s_abort[s & 1] = 1;
      atomicExch(p.error_flag, 1);
    }
    s_fail = s;
    const int c = z0 - 3 * R + s;          // centre plane of A r_{n-1} and r_n in this step
#pragma unroll
    for (int k = 0; k < 2 * R; ++k) { qa[k] = qa[k + 1]; vq[k] = vq[k + 1]; }
    if (act) {
      qa[2 * R] = RA[(size_t)ia * PEC + sidx];
      vq[2 * R] = VV[(size_t)ist * PEV + sidx];
    }
    if (s >= 2 * R && act) {
      const PC* A = RA + (size_t)ic * PEC;
      const PC L = A[sidx - 1], Rt = A[sidx + 1], U1 = A[sidx - BXP], D1 = A[sidx + BXP];
      PC U2, D2;
      if (R == 2) { U2 = A[sidx - 2 * BXP]; D2 = A[sidx + 2 * BXP]; } else { U2.a = U2.b = D2.a = D2.b = zc; }
      const PC r2 = RB[(size_t)ist * PEC + sidx];
      const PC cq = qa[R];
      // u = A r_{n-1} at both points of the pair
      const C n1a[6] = {qa[R - 1].a, qa[R + 1].a, L.b, cq.b, U1.a, D1.a};
      const C n1b[6] = {qa[R - 1].b, qa[R + 1].b, cq.a, Rt.a, U1.b, D1.b};
      C n2a[6], n2b[6];
      if (R == 2) {
        n2a[0] = qa[0].a; n2a[1] = qa[2 * R].a; n2a[2] = L.a; n2a[3] = Rt.a; n2a[4] = U2.a; n2a[5] = D2.a;
        n2b[0] = qa[0].b; n2b[1] = qa[2 * R].b; n2b[2] = L.b; n2b[3] = Rt.b; n2b[4] = U2.b; n2b[5] = D2.b;
      } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) { n2a[k] = zc; n2b[k] = zc; }
      }
      const bool cin = c >= 0 && c < d.nz;
      PC rn;
      rn.a = zc;
      rn.b = zc;
      if (cin && ina) {
        const C u = ST::applyA(cq.a, n1a, n2a, vq[2 * R].a, zre, zim, mh1, mh2);
        rn.a = ST::combine(a1, cq.a, a2, r2.a, aA, u);          // Eq. rvec
      }
      if (cin && inb) {
        const C u = ST::applyA(cq.b, n1b, n2b, vq[2 * R].b, zre, zim, mh1, mh2);
        rn.b = ST::combine(a1, cq.b, a2, r2.b, aA, u);
      }
#pragma unroll
      for (int k = 0; k < 2 * R; ++k) qb[k] = qb[k + 1];
      qb[2 * R] = rn;
      SB[(size_t)isb * PEC + sidx] = rn;
    }
    __syncthreads();
    if (s_abort[s & 1]) break;
    const int zo = c - R;
    if (s >= 3 * R && is_int && yin && zo >= z0 && zo < z1 && ina) {
      // A r_n on the output plane, then the three dot products
      const PC* B = SB + (size_t)isv * PEC;
      const PC L = B[sidx - 1], Rt = B[sidx + 1], U1 = B[sidx - BXP], D1 = B[sidx + BXP];
      PC U2, D2;
      if (R == 2) { U2 = B[sidx - 2 * BXP]; D2 = B[sidx + 2 * BXP]; } else { U2.a = U2.b = D2.a = D2.b = zc; }
      const PC cq = qb[R];
      const C n1a[6] = {qb[R - 1].a, qb[R + 1].a, L.b, cq.b, U1.a, D1.a};
      const C n1b[6] = {qb[R - 1].b, qb[R + 1].b, cq.a, Rt.a, U1.b, D1.b};
      C n2a[6], n2b[6];
      if (R == 2) {
        n2a[0] = qb[0].a; n2a[1] = qb[2 * R].a; n2a[2] = L.a; n2a[3] = Rt.a; n2a[4] = U2.a; n2a[5] = D2.a;
        n2b[0] = qb[0].b; n2b[1] = qb[2 * R].b; n2b[2] = L.b; n2b[3] = Rt.b; n2b[4] = U2.b; n2b[5] = D2.b;
      } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) { n2a[k] = zc; n2b[k] = zc; }
      }
      const C va = ST::applyA(cq.a, n1a, n2a, vq[R].a, zre, zim, mh1, mh2);
      acc.add(cq.a, va);
      C* dst = rout + (size_t)zo * plane_elems + (size_t)gy * d.nxp + gxa;
      const int pl = recorded_plane(d, zo);
      H* hrow = hist + (size_t)pl * nxy + (size_t)gy * d.nx + gxa;
      if (inb) {
        const C vb = ST::applyA(cq.b, n1b, n2b, vq[R].b, zre, zim, mh1, mh2);
        acc.add(cq.b, vb);
        *reinterpret_cast<PC*>(dst) = cq;
        if (pl >= 0) { hrow[0] = O::hi(cq.a); hrow[1] = O::hi(cq.b); }
      } else {
        dst[0] = cq.a;
        if (pl >= 0) hrow[0] = O::hi(cq.a);
      }
    }
    ia = (ia + 1 == NA) ? 0 : ia + 1;
    ic = (ic + 1 == NA) ? 0 : ic + 1;
    if (++ist == kStages) { ist = 0; par ^= 1; }
    isb = (isb + 1 == NSB) ? 0 : isb + 1;
    isv = (isv + 1 == NSB) ? 0 : isv + 1;
  }
  if (s_abort[s_fail & 1]) {
    // drain the bundles still in flight (the one whose wait expired and those issued after it)
    // before the CTA's shared memory is released
    if (tid == 0) {
      for (int bnd = s_fail; bnd < issued; ++bnd)
        mbar_wait(smem_u32(&bars[bnd % kStages]), (uint32_t)((bnd / kStages) & 1));
    }
    return;
  }

  double v5[5];
  acc.get(v5);
  if (pass_finish(p, slot, cta, v5, S, s_last)) {
    if (p.has_proj) {
      if (threadIdx.x == 0) {
        double* o = p.pdots + (size_t)slot * 8;
        o[0] = S.rr.x;
        o[1] = S.rr.y;
        o[2] = S.rAr.x;
        o[3] = S.rAr.y;
        o[4] = S.nrm2;
        o[5] = S.maxr;   // block-floating-point bounds (zero for the other forms)
        o[6] = S.maxu;
      }
    } else {
      scalar_step(p, slot, S);
    }
  }
}

// ------------------------------------------------------------------------------------------------
// the stored-product pass
// ------------------------------------------------------------------------------------------------
// One seed iteration that keeps u = A r in HBM next to r:
//
//   r_n = a1 r_{n-1} + a2 r_{n-2} + aA u_{n-1}     (pointwise, Eq. rvec with u_{n-1} = A r_{n-1})
//   u_n = A r_n                                     (one stencil application per grid point)
//
// It moves five vectors per iteration (reads r_{n-1}, r_{n-2}, u_{n-1}; writes r_n, u_n) against
// three for the fused pass, but applies the stencil once per point instead of on the tile plus halo
// and again for the dots; in double-float arithmetic the stencil dominates, so this is the faster
// form there.
//
// CTA: a 32 x TY tile of one slot and a z-range.  Each tile thread owns one x column and P
// consecutive rows, and keeps its r_n values of the last 2R + 1 planes in registers (the ring is
// rotated by unrolling the z loop, so no register moves); frame warps evaluate r_n on the R-wide
// frame the stencil needs, three points per thread.  Per z-plane one TMA bundle brings the
// 36 x (TY + 2R) boxes of r_{n-1}, r_{n-2}, u_{n-1} (plane q); a step evaluates r_n on plane q, stores
// it in a shared-memory ring of R + 1 planes, and evaluates A r_n on plane q - R, whose x and y
// neighbours were stored in earlier steps (rows inside the thread's own P come from registers).  One
// barrier per plane.
constexpr int kUBoxOff = 2;
constexpr int kFramePts = 3;        // frame points per frame thread
// launch bound per rows-per-thread P (one point per thread needs the most threads)
template <int P> struct MaxThreadsU { static constexpr int value = 384; };
template <> struct MaxThreadsU<1> { static constexpr int value = 640; };
// register-budget variants of the one-row-per-thread double-float pass: the launch bound caps the
// registers a thread may use (65536 / bound), so a smaller bound trades CTAs per SM for fewer spills
//   budget 0: bound 640 (96 registers; two CTAs of up to 320 threads per SM)
//   budget 1: bound 512 (128 registers; one CTA per SM, tiles up to 14 rows)
__host__ __device__ constexpr int passu_budget_threads(int budget) { return budget == 1 ? 512 : MaxThreadsU<1>::value; }

// tile width TX in x: 32 (one tile row per warp) or 16 (two tile rows per warp, for grids whose Nx is
// an odd multiple of 16); the box adds a 2-point frame on each side
__host__ __device__ __forceinline__ int passu_frame_warps(int R, int tile_y, int TX = kTileX) {
  const int nframe = 2 * R * tile_y + 2 * R * TX;
  return (nframe + 32 * kFramePts - 1) / (32 * kFramePts);
}
__host__ __device__ constexpr int passu_box_w(int TX) { return TX + 2 * kUBoxOff; }
// box coordinates of frame point h (R columns left and right of every tile row, then R rows below
// and above the tile); cx = -1 past the last one
template <int R, int TX = kTileX>
__device__ __forceinline__ void frame_point(int h, int TY, int nframe, int& cx, int& cy) {
  cx = -1;
  cy = 0;
  if (h >= nframe) return;
  if (h < 2 * R * TY) {
    const int side = h / (R * TY), k = h - side * R * TY;
    cy = k / R + R;
    cx = side == 0 ? kUBoxOff - R + k % R : kUBoxOff + TX + k % R;
  } else {
    const int k2 = h - 2 * R * TY;
    const int side = k2 / (R * TX), k = k2 - side * R * TX;
    cx = kUBoxOff + k % TX;
    cy = side == 0 ? k / TX : TY + R + k / TX;
  }
}

template <typename VT> __device__ __forceinline__ VT zero_v() { return VT(); }
template <> __device__ __forceinline__ float2 zero_v<float2>() { return make_float2(0.f, 0.f); }

template <int MODE, int R, int P, int NT = MaxThreadsU<P>::value, int TX = kTileX>
__global__ void __launch_bounds__(NT) passu_kernel(PassParams p, const __grid_constant__ CUtensorMap tmR) {
  typedef Ops<MODE> O;
  typedef Stencil<MODE, R> ST;
  typedef typename O::C C;
  typedef typename O::VT VT;
  typedef typename O::H H;
  constexpr int Q = 2 * R + 1;
  extern __shared__ unsigned char smem_raw[];
  __shared__ ScalarShared S;
  __shared__ int s_last, s_abort[2];   // abort flags indexed by step parity (set before, read after a barrier)
  __shared__ __align__(8) unsigned long long bars[kMaxStages];

  const int slot = blockIdx.y;
  SlotState* st = p.slots + slot;
  if (st->status != SLOT_RUNNING) return;
  const int kDepth = p.depth;
  const int kStages = kDepth + 1;
  const SolveDims& d = p.d;
  const int TY = d.tile_y;
  const int EY = TY + 2 * R;
  constexpr int BW = passu_box_w(TX);
  constexpr int HW = 32 / TX;                // tile rows per warp (1 or 2): lanes split into HW x-runs
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int xl = lane % TX;                  // x of the thread inside the tile
  const int cta = blockIdx.x;
  const int tz = cta % d.nzchunks;
  const int txy = cta / d.nzchunks;
  const int tx = txy % d.tiles_x, ty = txy / d.tiles_x;
  const int z0 = tz * d.zchunk;
  const int z1 = min(z0 + d.zchunk, d.nz);
  const int x0 = tx * TX, y0 = ty * TY;
  const int NWI = TY / (P * HW);
  const bool interior = warp < NWI;
  const int row0 = (warp * HW + lane / TX) * P;   // first tile row of a tile thread
  const int gx = x0 + xl;
  const long long plane_elems = (long long)d.nxp * d.ny;

  // shared memory: per stage the boxes of r_{n-1}, r_{n-2}, u_{n-1}; a ring of R + 1 planes of r_n
  const size_t PBb = (size_t)BW * EY * sizeof(C);
  const int PE = (int)(((PBb + 127) & ~(size_t)127) / sizeof(C));
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  C* RA = (C*)base;
  C* RB = RA + (size_t)kStages * PE;
  C* UA = RB + (size_t)kStages * PE;
  C* SB = UA + (size_t)kStages * PE;

  struct Coefs {
    typename O::Cplx a1, a2, aA;
    typename O::Real zre, zim, mh1, mh2;
    int n, hc;
  };
  __shared__ Coefs sc;
  if (threadIdx.x == 0) {
    sc.a1 = O::cplx(st->a1);
    sc.a2 = O::cplx(st->a2);
    sc.aA = O::cplx(st->aA);
    const double2 Zs0 = st->Zs;
    sc.zre = O::real(Zs0.x - p.hd);
    sc.zim = O::real(Zs0.y);
    sc.mh1 = O::real(-p.hk1);
    sc.mh2 = O::real(-p.hk2);
    sc.n = st->n;
    sc.hc = st->hcnt;
  }
  __syncthreads();
  const int n = sc.n;
  const int i1 = (n + 2) % 3, i2 = (n + 1) % 3, io = n % 3;
  const int iu1 = 3 + (n + 1) % 2, iuo = 3 + n % 2;
  const long long vec = (long long)d.nz * plane_elems;
  C* rout = reinterpret_cast<C*>(p.rbuf) + ((size_t)slot * 5 + io) * vec;
  C* uout = reinterpret_cast<C*>(p.rbuf) + ((size_t)slot * 5 + iuo) * vec;
  const VT* Vg = reinterpret_cast<const VT*>(p.V);
  const typename O::Cplx a1 = sc.a1, a2 = sc.a2, aA = sc.aA;
  const typename O::Real zre = sc.zre, zim = sc.zim, mh1 = sc.mh1, mh2 = sc.mh2;
  H* hist = reinterpret_cast<H*>(p.rhist) + ((size_t)slot * p.hist_len + sc.hc) * d.nb;
  const long long nxy = (long long)d.nx * d.ny;

  constexpr int mR = (MODE == RSFD_DF64) ? 4 : 2;
  const int xr = mR * (x0 - kUBoxOff), yb = y0 - R;
  const uint32_t bundle_bytes = (uint32_t)(3 * PBb);
  const int nsteps = (z1 - z0) + 2 * R;
  const int w1 = slot * 5 + i1, w2 = slot * 5 + i2, wu = slot * 5 + iu1;

  auto issue = [&](int bnd) {
    const int q = z0 - R + bnd;
    const int k = bnd % kStages;
    const uint32_t bar = smem_u32(&bars[k]);
    mbar_expect_tx(bar, bundle_bytes);
    tma_load_4d(smem_u32(RA + (size_t)k * PE), &tmR, xr, yb, q, w1, bar);
    tma_load_4d(smem_u32(RB + (size_t)k * PE), &tmR, xr, yb, q, w2, bar);
    tma_load_4d(smem_u32(UA + (size_t)k * PE), &tmR, xr, yb, q, wu, bar);
  };

  if (tid == 0) {
    for (int k = 0; k < kStages; ++k) mbar_init(smem_u32(&bars[k]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    s_abort[0] = s_abort[1] = 0;
  }
  __syncthreads();
  int issued = 0, s_fail = 0;
  if (tid == 0) {
    for (int bnd = 0; bnd < kDepth && bnd < nsteps; ++bnd) issue(bnd);
    issued = min(kDepth, nsteps);
  }

  typename AccOf<MODE>::type acc;
  // Step s: r_n on plane q = z0 - R + s (TMA stage ist, shared ring slot s % (R + 1)) and, from step
  // 2R on, A r_n on plane c = q - R (ring slot (s - R) % (R + 1) = (s + 1) % (R + 1)).
  int ist = 0, par = 0, isw = 0, s = 0;
  auto begin_step = [&]() {
    if (tid == 0 && s + kDepth < nsteps) {
      issue(s + kDepth);
      issued = s + kDepth + 1;
    }
    if (!mbar_wait(smem_u32(&bars[ist]), (uint32_t)par, first_wait_cap(p.d))) {
      s_abort[s & 1] = 1;
      atomicExch(p.error_flag, 1);
    }
    s_fail = s;
  };
  auto end_step = [&]() -> bool {
    __syncthreads();
    if (s_abort[s & 1]) return false;
    if (++ist == kStages) { ist = 0; par ^= 1; }
    isw = (isw == R) ? 0 : isw + 1;
    ++s;
    return true;
  };
  bool ok = true;
  if (interior) {
    C zq[P][Q];   // zq[k][t % Q]: r_n of row row0 + k on the plane combined in step t
#pragma unroll
    for (int k = 0; k < P; ++k)
#pragma unroll
      for (int t = 0; t < Q; ++t) zq[k][t] = O::zero();
    bool own[P];
    int gyk[P];
#pragma unroll
    for (int k = 0; k < P; ++k) {
      gyk[k] = y0 + row0 + k;
      own[k] = gx < d.nx && gyk[k] < d.ny;
    }
    // the combine of plane q for the P rows; the result enters ring slot isw and zq[.][PH]
    auto combine_rows = [&](auto ph_c) {
      constexpr int PH = decltype(ph_c)::value;
      C* sw = SB + (size_t)isw * PE;
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const int o = (row0 + k + R) * BW + xl + kUBoxOff;
        const size_t os = (size_t)ist * PE + o;
        const C rq = ST::combine(a1, RA[os], a2, RB[os], aA, UA[os]);   // Eq. rvec
        sw[o] = rq;
        zq[k][PH] = rq;
      }
    };
    // prologue: planes z0 - R .. z0 + R - 1, the combine only
#pragma unroll
    for (int t = 0; t < 2 * R; ++t) {
      if (ok && s < nsteps) {
        begin_step();
        if (t == 0) combine_rows(std::integral_constant<int, 0>());
        if (t == 1) combine_rows(std::integral_constant<int, 1 % Q>());
        if (t == 2) combine_rows(std::integral_constant<int, 2 % Q>());
        if (t == 3) combine_rows(std::integral_constant<int, 3 % Q>());
        ok = end_step();
      }
    }
    // steady state: step s = 2R + g Q + j has ring phase (2R + j) % Q
    auto steady = [&](auto j_c) {
      constexpr int PH = (2 * R + decltype(j_c)::value) % Q;       // slot of plane q
      constexpr int CC = (PH + Q - R) % Q;                         // slot of plane c = q - R
      begin_step();
      combine_rows(std::integral_constant<int, PH>());
      const int c = z0 - 2 * R + s;
      const C* P0 = SB + (size_t)((isw + 1 == R + 1) ? 0 : isw + 1) * PE;
#pragma unroll
      for (int k = 0; k < P; ++k) {
        const int o = (row0 + k + R) * BW + xl + kUBoxOff;
        const C rc = zq[k][CC];
        C n1[6], n2[6];
        n1[0] = zq[k][(CC + Q - 1) % Q];
        n1[1] = zq[k][(CC + 1) % Q];
        n1[2] = P0[o - 1];
        n1[3] = P0[o + 1];
        n1[4] = (k >= 1) ? zq[k - 1 >= 0 ? k - 1 : 0][CC] : P0[o - BW];
        n1[5] = (k + 1 < P) ? zq[k + 1 < P ? k + 1 : 0][CC] : P0[o + BW];
        if (R == 2) {
          n2[0] = zq[k][(CC + Q - 2) % Q];
          n2[1] = zq[k][(CC + 2) % Q];
          n2[2] = P0[o - 2];
          n2[3] = P0[o + 2];
          n2[4] = (k >= 2) ? zq[k - 2 >= 0 ? k - 2 : 0][CC] : P0[o - 2 * BW];
          n2[5] = (k + 2 < P) ? zq[k + 2 < P ? k + 2 : 0][CC] : P0[o + 2 * BW];
        } else {
#pragma unroll
          for (int m = 0; m < 6; ++m) n2[m] = O::zero();
        }
        const long long gidx = (long long)c * plane_elems + (long long)gyk[k] * d.nxp + gx;
        const VT v = own[k] ? Vg[gidx] : zero_v<VT>();
        const C u = ST::applyA(rc, n1, n2, v, zre, zim, mh1, mh2);
        if (own[k]) {
          acc.add(rc, u);
          rout[gidx] = rc;
          uout[gidx] = u;
          const int pl = recorded_plane(d, c);
          if (pl >= 0) hist[(size_t)pl * nxy + (size_t)gyk[k] * d.nx + gx] = O::hi(rc);
        }
      }
      ok = end_step();
    };
    while (ok && s < nsteps) {
      steady(std::integral_constant<int, 0>());
      if (ok && s < nsteps) steady(std::integral_constant<int, 1>());
      if (ok && s < nsteps) steady(std::integral_constant<int, 2>());
      if (R == 2) {
        if (ok && s < nsteps) steady(std::integral_constant<int, 3>());
        if (ok && s < nsteps) steady(std::integral_constant<int, 4>());
      }
    }
  } else {
    const int nframe = 2 * R * TY + 2 * R * TX;
    const int FT = passu_frame_warps(R, TY, TX) * 32;
    int fo[kFramePts];
    bool fv[kFramePts];
#pragma unroll
    for (int j = 0; j < kFramePts; ++j) {
      int cx, cy;
      frame_point<R, TX>((warp - NWI) * 32 + lane + j * FT, TY, nframe, cx, cy);
      fv[j] = cx >= 0;
      fo[j] = fv[j] ? cy * BW + cx : 0;
    }
    while (ok && s < nsteps) {
      begin_step();
      C* sw = SB + (size_t)isw * PE;
#pragma unroll
      for (int j = 0; j < kFramePts; ++j) {
        const size_t os = (size_t)ist * PE + fo[j];
        const C r = ST::combine(a1, RA[os], a2, RB[os], aA, UA[os]);
        if (fv[j]) sw[fo[j]] = r;
      }
      ok = end_step();
    }
  }
  if (!ok) {
    // drain the bundles still in flight (the one whose wait expired and those issued after it)
    // before the CTA's shared memory is released
    if (tid == 0) {
      for (int bnd = s_fail; bnd < issued; ++bnd)
        mbar_wait(smem_u32(&bars[bnd % kStages]), (uint32_t)((bnd / kStages) & 1));
    }
    return;
  }
  double v5[5];
  acc.get(v5);
  if (pass_finish(p, slot, cta, v5, S, s_last)) {
    if (p.has_proj) {
      if (threadIdx.x == 0) {
        double* o = p.pdots + (size_t)slot * 8;
        o[0] = S.rr.x;
        o[1] = S.rr.y;
        o[2] = S.rAr.x;
        o[3] = S.rAr.y;
        o[4] = S.nrm2;
        o[5] = S.maxr;   // block-floating-point bounds (zero for the other forms)
        o[6] = S.maxu;
      }
    } else {
      scalar_step(p, slot, S);
    }
  }
}

// ------------------------------------------------------------------------------------------------
// the split pass: a pointwise combine kernel, then a stencil kernel
// ------------------------------------------------------------------------------------------------
// The stored-product iteration (five vectors) as two launches per iteration:
//
//   combine_kernel:  r_n = a1 r_{n-1} + a2 r_{n-2} + aA u_{n-1}   (pointwise, Eq. rvec), the boundary
//                    rows of r_n for the shift update, and the partial sums of (r_n, r_n), ||r_n||^2;
//   stencil_kernel:  u_n = A r_n (one stencil application per point) and the partial sums of
//                    (r_n, A r_n); the last CTA of a slot reduces both kernels' partials in a fixed
//                    order and runs the FP64 scalar step.
//
// The combine moves four vectors and is bound by HBM bandwidth; the stencil moves two (plus its
// halo from L2) and carries the stencil's arithmetic without the combine's registers, so neither
// half limits the other's occupancy.  Per iteration the pair moves six vectors against the stored
// pass's five, in exchange for every grid point's stencil and combine being computed once (no frame
// recomputation).

// Combine: CTA = 256 threads over a range of z-planes of one slot; each thread walks the plane's
// padded elements with stride 256 (x, y tracked by a running counter) and handles two elements per
// step so that six 16-byte loads are in flight.
constexpr int kCombThreads = 256;

// Block-floating-point rounding of the leading parts (BFP): with Cq = 1.5 2^23 q, fl(h + Cq) - Cq is h
// rounded to a multiple of q (exact while |h| < 2^22 q: h + Cq stays in Cq's binade, whose spacing
// is q), and h - hq is exact; the remainder joins the trailing part.
template <bool BFP, typename C> struct Requant {
  static __device__ __forceinline__ C apply(const C& x, float2) { return x; }
  static __device__ __forceinline__ float amax(const C&) { return 0.f; }
};
template <> struct Requant<true, dfc> {
  static __device__ __forceinline__ dfc apply(const dfc& x, float2 cq) {
    dfc r;
    r.h = f2sub(f2add(x.h, cq), cq);
    r.l = f2add(x.l, f2sub(x.h, r.h));
    return r;
  }
  static __device__ __forceinline__ float amax(const dfc& x) { return fmaxf(fabsf(x.h.x), fabsf(x.h.y)); }
};

// one combine CTA: block cblk (of d.ctas_c, a range of z-planes) of slot `slot`; any block size
template <int MODE, bool BFP>
__device__ __forceinline__ void combine_body(const PassParams& p, const int slot, const int cblk) {
  typedef Ops<MODE> O;
  typedef Stencil<MODE, 1> ST;   // combine() does not depend on the stencil reach
  typedef typename O::C C;
  typedef typename O::H H;
  typedef Requant<BFP, C> RQ;
  __shared__ double s_red[32 * 5];
  __shared__ typename O::Cplx s_a[3];
  __shared__ int s_n, s_hc;
  __shared__ float s_cq;
  const SlotState* st = p.slots + slot;
  if (st->status != SLOT_RUNNING) return;
  const SolveDims& d = p.d;
  if (threadIdx.x == 0) {
    s_a[0] = O::cplx(st->a1);
    s_a[1] = O::cplx(st->a2);
    s_a[2] = O::cplx(st->aA);
    s_n = st->n;
    s_hc = st->hcnt;
    s_cq = BFP ? (float)(1.5 * 8388608.0 * st->q) : 0.f;
  }
  __syncthreads();
  const typename O::Cplx a1 = s_a[0], a2 = s_a[1], aA = s_a[2];
  const float2 cq = make_float2(s_cq, s_cq);
  float mxr = 0.f;
  const int n = s_n;
  const int i1 = (n + 2) % 3, i2 = (n + 1) % 3, io = n % 3, iu1 = 3 + (n + 1) % 2;
  const long long pe = (long long)d.nxp * d.ny;   // padded elements per plane
  const long long vec = (long long)d.nz * pe;
  const C* R1 = reinterpret_cast<const C*>(p.rbuf) + ((size_t)slot * 5 + i1) * vec;
  const C* R2 = reinterpret_cast<const C*>(p.rbuf) + ((size_t)slot * 5 + i2) * vec;
  const C* U1 = reinterpret_cast<const C*>(p.rbuf) + ((size_t)slot * 5 + iu1) * vec;
  C* RO = reinterpret_cast<C*>(p.rbuf) + ((size_t)slot * 5 + io) * vec;
  H* hist = reinterpret_cast<H*>(p.rhist) + ((size_t)slot * p.hist_len + s_hc) * d.nb;
  const long long nxy = (long long)d.nx * d.ny;
  const int za = (int)((long long)cblk * d.nz / d.ctas_c);
  const int zb = (int)((long long)(cblk + 1) * d.nz / d.ctas_c);
  const int tid = threadIdx.x;
  const int nthr = blockDim.x;
  const int dx = nthr % d.nxp, dy = nthr / d.nxp;
  typename AccOf<MODE>::type acc;
  for (int z = za; z < zb; ++z) {
    const long long zo = (long long)z * pe;
    const int pl = recorded_plane(d, z);
    int x = tid % d.nxp, y = tid / d.nxp;
    for (long long e = tid; e < pe; e += 2 * nthr) {
      // two elements: e and e + nthr (the second may lie past the plane)
      const long long e2 = e + nthr;
      int x2 = x + dx, y2 = y + dy;
      if (x2 >= d.nxp) { x2 -= d.nxp; ++y2; }
      const bool has2 = e2 < pe;
      const C r1a = R1[zo + e], r2a = R2[zo + e], ua = U1[zo + e];
      C r1b = O::zero(), r2b = O::zero(), ub = O::zero();
      if (has2) { r1b = R1[zo + e2]; r2b = R2[zo + e2]; ub = U1[zo + e2]; }
      const C ra = ST::combine(a1, r1a, a2, r2a, aA, ua);   // Eq. rvec
      const C qa = RQ::apply(ra, cq);
      RO[zo + e] = qa;
      if (x < d.nx) {
        acc.add_r(ra);
        if (BFP) mxr = fmaxf(mxr, RQ::amax(qa));
        if (pl >= 0) hist[(size_t)pl * nxy + (size_t)y * d.nx + x] = O::hi(ra);
      }
      if (has2) {
        const C rb = ST::combine(a1, r1b, a2, r2b, aA, ub);
        const C qb = RQ::apply(rb, cq);
        RO[zo + e2] = qb;
        if (x2 < d.nx) {
          acc.add_r(rb);
          if (BFP) mxr = fmaxf(mxr, RQ::amax(qb));
          if (pl >= 0) hist[(size_t)pl * nxy + (size_t)y2 * d.nx + x2] = O::hi(rb);
        }
      }
      x = x2 + dx;
      y = y2 + dy;
      if (x >= d.nxp) { x -= d.nxp; ++y; }
    }
  }
  double v5[5];
  acc.get(v5);
  block_sum_lane0<5>(v5, s_red);
  if (BFP) mxr = block_max0(mxr, reinterpret_cast<float*>(s_red));
  if (tid == 0) {
    double* dst = p.partials + ((size_t)slot * d.npart + d.ctas_per_slot + cblk) * 8;
#pragma unroll
    for (int k = 0; k < 5; ++k) dst[k] = v5[k];
    if (BFP) {
      dst[5] = (double)mxr;
      dst[6] = 0.0;
    }
  }
}

// At most 64 registers: four CTAs (32 warps) per SM keep enough loads in flight for HBM.
template <int MODE, bool BFP>
__global__ void __launch_bounds__(kCombThreads, 4) combine_kernel(PassParams p) {
  combine_body<MODE, BFP>(p, blockIdx.y, blockIdx.x);
}

// Stencil: CTA = a 32 x TY tile of one slot and a z-range, one thread per tile point (one warp per
// tile row).  Per z-plane one TMA transfer brings the (32 + 4) x (TY + 2R) box of r_n into a ring of
// depth + R + 1 shared-memory stages; each thread keeps its own column's r_n on the last 2R + 1
// planes in registers (ring rotated by unrolling, no moves) and takes its x and y neighbours from
// the stage of the plane it evaluates.  One barrier per plane.
constexpr int kMaxStagesS = kMaxDepth + 3;

// The potential of the plane being evaluated arrives by TMA with the plane of r_n.  There is no
// CTA-wide barrier per plane: every stage has a "full" mbarrier (the TMA transaction count) and an
// "empty" one on which each warp arrives once it is done with the stage; thread 0 waits for a stage
// to be empty before it refills it, so warps run up to the prefetch depth apart.
// BFP (double-float handles): the r_n it reads has block-floating-point leading parts, tmV maps s V,
// and it stores u_n = s A r_n (StencilBFP) with the largest leading-part component of u_n.
// one stencil CTA: tile cta (of d.ctas_per_slot) of slot `slot`; blockDim = 32 x tile_y
template <int MODE, int R, bool BFP>
__device__ __forceinline__ void stencil_body(const PassParams& p, const CUtensorMap& tmR, const CUtensorMap& tmV,
                                             const int slot, const int cta) {
  static_assert(!BFP || MODE == RSFD_DF64, "the block-floating-point pass is double-float only");
  typedef Ops<MODE> O;
  typedef typename O::C C;
  typedef typename O::VT VT;
  constexpr int Q = 2 * R + 1;
  constexpr int BW = kTileX + 2 * kUBoxOff;
  extern __shared__ unsigned char smem_raw[];
  __shared__ ScalarShared S;
  __shared__ int s_last;
  __shared__ volatile int s_abort;
  __shared__ __align__(8) unsigned long long bars[kMaxStagesS];     // full: TMA bytes landed
  __shared__ __align__(8) unsigned long long ebars[kMaxStagesS];    // empty: every warp done with it

  SlotState* st = p.slots + slot;
  if (st->status != SLOT_RUNNING) return;
  const SolveDims& d = p.d;
  const int kDepth = p.depth;
  const int NS = kDepth + R + 1;   // the stage of plane c is read R steps after its arrival
  const int TY = d.tile_y;
  const int EY = TY + 2 * R;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tz = cta % d.nzchunks;
  const int txy = cta / d.nzchunks;
  const int tx = txy % d.tiles_x, ty = txy / d.tiles_x;
  const int z0 = tz * d.zchunk;
  const int z1 = min(z0 + d.zchunk, d.nz);
  const int x0 = tx * kTileX, y0 = ty * TY;
  const int gx = x0 + lane, gy = y0 + warp;
  const bool own = gx < d.nx && gy < d.ny;
  const long long plane_elems = (long long)d.nxp * d.ny;

  // shared memory: per stage the box of r_n (plane q) and the tile of V (plane q - R)
  const size_t PBb = (size_t)BW * EY * sizeof(C);
  const int PE = (int)(((PBb + 127) & ~(size_t)127) / sizeof(C));
  const size_t PVb = (size_t)kTileX * TY * sizeof(VT);
  const int PV = (int)(((PVb + 127) & ~(size_t)127) / sizeof(VT));
  C* ring = (C*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  VT* vring = (VT*)(ring + (size_t)NS * PE);

  struct Coefs {
    typename O::Real zre, zim, mh1, mh2;
    int n;
  };
  __shared__ Coefs sc;
  if (tid == 0) {
    const double2 Zs0 = st->Zs;
    // BFP: the diagonal of s A is s (Z_s - hd) - s V
    const double sd = BFP ? p.uscale : 1.0;
    sc.zre = O::real(sd * (Zs0.x - p.hd));
    sc.zim = O::real(sd * Zs0.y);
    sc.mh1 = O::real(-p.hk1);
    sc.mh2 = O::real(-p.hk2);
    sc.n = st->n;
  }
  __syncthreads();
  const int n = sc.n;
  const int io = n % 3, iuo = 3 + n % 2;
  const long long vec = (long long)d.nz * plane_elems;
  C* uout = reinterpret_cast<C*>(p.rbuf) + ((size_t)slot * 5 + iuo) * vec;
  const typename O::Real zre = sc.zre, zim = sc.zim, mh1 = sc.mh1, mh2 = sc.mh2;
  float mxu = 0.f;

  constexpr int mR = (MODE == RSFD_DF64) ? 4 : 2;
  constexpr int mV = (MODE == RSFD_DF64) ? 2 : 1;
  const int xr = mR * (x0 - kUBoxOff), yb = y0 - R, xv = mV * x0;
  const int nsteps = (z1 - z0) + 2 * R;
  const int wr = slot * 5 + io;
  auto issue = [&](int bnd) {
    const int k = bnd % NS;
    const uint32_t bar = smem_u32(&bars[k]);
    mbar_expect_tx(bar, (uint32_t)(PBb + PVb));
    tma_load_4d(smem_u32(ring + (size_t)k * PE), &tmR, xr, yb, z0 - R + bnd, wr, bar);
    tma_load_3d(smem_u32(vring + (size_t)k * PV), &tmV, xv, y0, z0 - 2 * R + bnd, bar);
  };
  const int nwarps = blockDim.x >> 5;
  if (tid == 0) {
    for (int k = 0; k < NS; ++k) {
      mbar_init(smem_u32(&bars[k]), 1);
      mbar_init(smem_u32(&ebars[k]), (uint32_t)nwarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    s_abort = 0;
  }
  __syncthreads();
  int issued = 0;
  if (tid == 0) {
    for (int bnd = 0; bnd < kDepth && bnd < nsteps; ++bnd) issue(bnd);
    issued = min(kDepth, nsteps);
  }
  typename AccOf<MODE>::type acc;
  // step s: plane q = z0 - R + s and the potential of plane c = q - R arrive in stage s % NS; from
  // step 2R on, A r_n on plane c, whose r_n box is in stage (s - R) % NS.  A stage is released after
  // its plane served as plane c (R steps after it arrived).
  int ist = 0, par = 0, ic = NS - R, s = 0;
  const int oc = (warp + R) * BW + lane + kUBoxOff;   // this thread's point in a stage
  const int ov = warp * kTileX + lane;                // and in the potential's tile
  auto fail_now = [&]() {
    s_abort = 1;
    atomicExch(p.error_flag, 1);
  };
  auto begin_step = [&]() -> bool {
    if (tid == 0 && s + kDepth < nsteps && !s_abort) {
      const int b = s + kDepth;
      // the stage's previous bundle (b - NS) must have been released by every warp
      if (b >= NS && !mbar_wait(smem_u32(&ebars[b % NS]), (uint32_t)(((b / NS) - 1) & 1), first_wait_cap(d))) {
        fail_now();
      } else {
        issue(b);
        issued = b + 1;
      }
    }
    if (s_abort) return false;
    if (!mbar_wait(smem_u32(&bars[ist]), (uint32_t)par, first_wait_cap(d))) {
      fail_now();
      return false;
    }
    return true;
  };
  auto end_step = [&]() -> bool {
    __syncwarp();
    if (s >= R && lane == 0) mbar_arrive(smem_u32(&ebars[ic]));   // stage of bundle s - R
    if (s_abort) return false;
    if (++ist == NS) { ist = 0; par ^= 1; }
    if (++ic == NS) ic = 0;
    ++s;
    return true;
  };
  bool ok = true;
  C zq[Q];
#pragma unroll
  for (int t = 0; t < Q; ++t) zq[t] = O::zero();
#pragma unroll
  for (int t = 0; t < 2 * R; ++t) {
    if (ok && s < nsteps) {
      ok = begin_step();
      if (!ok) break;
      const C own_v = ring[(size_t)ist * PE + oc];
      if (t == 0) zq[0] = own_v;
      if (t == 1) zq[1 % Q] = own_v;
      if (t == 2) zq[2 % Q] = own_v;
      if (t == 3) zq[3 % Q] = own_v;
      ok = end_step();
    }
  }
  auto steady = [&](auto j_c) {
    constexpr int PH = (2 * R + decltype(j_c)::value) % Q;   // ring slot of plane q
    constexpr int CC = (PH + Q - R) % Q;                     // ring slot of plane c = q - R
    if (!begin_step()) {
      ok = false;
      return;
    }
    zq[PH] = ring[(size_t)ist * PE + oc];
    const int c = z0 - 2 * R + s;
    const C* P0 = ring + (size_t)ic * PE;
    C n1[6], n2[6];
    n1[0] = zq[(CC + Q - 1) % Q];
    n1[1] = zq[(CC + 1) % Q];
    n1[2] = P0[oc - 1];
    n1[3] = P0[oc + 1];
    n1[4] = P0[oc - BW];
    n1[5] = P0[oc + BW];
    if (R == 2) {
      n2[0] = zq[(CC + Q - 2) % Q];
      n2[1] = zq[(CC + 2) % Q];
      n2[2] = P0[oc - 2];
      n2[3] = P0[oc + 2];
      n2[4] = P0[oc - 2 * BW];
      n2[5] = P0[oc + 2 * BW];
    } else {
#pragma unroll
      for (int m = 0; m < 6; ++m) n2[m] = O::zero();
    }
    if (own) {
      const C rc = zq[CC];
      const VT v = vring[(size_t)ist * PV + ov];
      if constexpr (BFP) {
        const float2 zh = make_float2(-zim.h, zim.h), zl = make_float2(-zim.l, zim.l);
        const dfc u = StencilBFP<R>::applyA(rc, n1, n2, v, zre, zh, zl);
        dfc rn;   // normalised r_n for the exact products of the dot
        fast_two_sum2(rc.h, rc.l, rn.h, rn.l);
        acc.add_ra(rn, u);
        mxu = fmaxf(mxu, fmaxf(fabsf(u.h.x), fabsf(u.h.y)));
        uout[(long long)c * plane_elems + (long long)gy * d.nxp + gx] = u;
      } else {
        const C u = Stencil<MODE, R>::applyA(rc, n1, n2, v, zre, zim, mh1, mh2);
        acc.add_ra(rc, u);
        uout[(long long)c * plane_elems + (long long)gy * d.nxp + gx] = u;
      }
    }
    ok = end_step();
  };
  while (ok && s < nsteps) {
    steady(std::integral_constant<int, 0>());
    if (ok && s < nsteps) steady(std::integral_constant<int, 1>());
    if (ok && s < nsteps) steady(std::integral_constant<int, 2>());
    if (R == 2) {
      if (ok && s < nsteps) steady(std::integral_constant<int, 3>());
      if (ok && s < nsteps) steady(std::integral_constant<int, 4>());
    }
  }
  (void)ok;
  __syncthreads();   // every thread, finished or stopped by an expired wait
  if (s_abort) {
    // drain the transfers still in flight: per stage, the last bundle thread 0 issued into it (the
    // earlier ones on that stage completed before it was refilled)
    if (tid == 0) {
      for (int bnd = max(0, issued - NS); bnd < issued; ++bnd)
        mbar_wait(smem_u32(&bars[bnd % NS]), (uint32_t)((bnd / NS) & 1));
    }
    return;
  }
  double v5[5];
  acc.get(v5);
  if (pass_finish(p, slot, cta, v5, S, s_last, mxu)) {
    if (p.has_proj) {
      if (tid == 0) {
        double* o = p.pdots + (size_t)slot * 8;
        o[0] = S.rr.x;
        o[1] = S.rr.y;
        o[2] = S.rAr.x;
        o[3] = S.rAr.y;
        o[4] = S.nrm2;
        o[5] = S.maxr;   // block-floating-point bounds (zero for the other forms)
        o[6] = S.maxu;
      }
    } else {
      scalar_step(p, slot, S);
    }
  }
}

template <int MODE, int R, int NT, int MINB, bool BFP = false>
__global__ void __launch_bounds__(NT, MINB) stencil_kernel(PassParams p, const __grid_constant__ CUtensorMap tmR,
                                                             const __grid_constant__ CUtensorMap tmV) {
  stencil_body<MODE, R, BFP>(p, tmR, tmV, blockIdx.y, blockIdx.x);
}

// ------------------------------------------------------------------------------------------------
// nonlocal projector term (separable Kleinman-Bylander form, Sec. II A):
//   V_nl r = sum_a E_a c_a p_a,   c_a = h^3 p_a^T r,
// so with u_loc = (Z_s - H_loc) r from the pass,
//   A r = u_loc - sum_a E_a c_a p_a,   (r, A r) = (r, u_loc) - sum_a E_a c_a^2 / h^3.
// proj_kernel: one block per (atom, slot) forms c_a (a gather-GEMV over the atom's support, exact
// products in double-float or FP64), stores -E_a c_a and the dot correction; the last block of a
// slot (atomic ticket) sums the corrections in atom order and runs the FP64 scalar step.
// pscatter_kernel: u_n -= sum_a E_a c_a p_a over the union of the supports, one thread per support
// point gathering its atoms (point-major CSR), so no atomics and a fixed summation order.
// ------------------------------------------------------------------------------------------------
struct ProjParams {
  PassParams pp;
  int n_atoms, n_supp;
  const int* a_ptr;
  const long long* a_idx;
  const void* a_val;
  const double* a_E;
  const int* t_ptr;
  const long long* t_pidx;
  const int* t_atom;
  const void* t_val;
  double h3;
  double2* pw;
  double2* pcorr;
  unsigned int* ptickets;
  const double* pmax;        // per atom: largest |projector value|
  int overlap;               // largest number of atoms at one support point
};

// per-thread FP64 sum of p_j r_j, per precision
template <int MODE> struct ProjAcc;
template <> struct ProjAcc<RSFD_FP64> {
  double2 s = make_double2(0.0, 0.0);
  __device__ __forceinline__ void add(double pv, double2 r) {
    s.x = fma(pv, r.x, s.x);
    s.y = fma(pv, r.y, s.y);
  }
  __device__ __forceinline__ double2 get() const { return s; }
};
template <> struct ProjAcc<RSFD_MIXED> {
  double2 s = make_double2(0.0, 0.0);
  __device__ __forceinline__ void add(float pv, float2 r) {
    s.x = fma((double)pv, (double)r.x, s.x);
    s.y = fma((double)pv, (double)r.y, s.y);
  }
  __device__ __forceinline__ double2 get() const { return s; }
};
template <> struct ProjAcc<RSFD_DF64> {
  DFAcc a = dfacc_zero();
  __device__ __forceinline__ void add(float2 pv, const dfc& r) {
    dfr c;
    c.h = pv.x;
    c.l = pv.y;
    dfacc_mul(a, c, r);
  }
  __device__ __forceinline__ double2 get() const {
    return make_double2((double)a.s.x + (double)a.lo.x, (double)a.s.y + (double)a.lo.y);
  }
};

// one block per (atom, slot); an atom has ~10^3 support points, so a small block keeps the per-block
// reduction and ticket cheap against the gather
constexpr int kProjThreads = 128;
template <int MODE>
__global__ void __launch_bounds__(kProjThreads) proj_kernel(ProjParams q) {
  typedef typename Ops<MODE>::C C;
  typedef typename Ops<MODE>::VT VT;
  __shared__ ScalarShared S;
  __shared__ int s_last;
  const PassParams& p = q.pp;
  const int a = blockIdx.x, slot = blockIdx.y, tid = threadIdx.x;
  SlotState* st = p.slots + slot;
  if (st->status != SLOT_RUNNING) return;
  const int n = st->n;   // the pass of this iteration wrote r_n to ring entry n % 3
  const long long vec = (long long)p.d.nz * p.d.ny * p.d.nxp;
  const C* r = reinterpret_cast<const C*>(p.rbuf) + ((size_t)slot * p.d.nvec + n % 3) * vec;
  const VT* pv = reinterpret_cast<const VT*>(q.a_val);
  ProjAcc<MODE> acc;
  for (int e = q.a_ptr[a] + tid; e < q.a_ptr[a + 1]; e += blockDim.x) acc.add(pv[e], r[q.a_idx[e]]);
  const double2 t = acc.get();
  double v2[2] = {warp_sum(t.x), warp_sum(t.y)};
  block_sum_lane0<2>(v2, S.red);
  if (tid == 0) {
    const double2 c = make_double2(v2[0] * q.h3, v2[1] * q.h3);
    const double E = q.a_E[a];
    const double us = p.uscale;   // the block-floating-point pass stores s A r
    const double2 wv = make_double2(-E * us * c.x, -E * us * c.y);
    if (MODE == RSFD_DF64) {
      // stored as a double-float pair (16 bytes, the same slot): the scatter applies it to every
      // support point of the atom without converting it again
      dfc wc;
      wc.h = make_float2((float)wv.x, (float)wv.y);
      wc.l = make_float2((float)(wv.x - (double)wc.h.x), (float)(wv.y - (double)wc.h.y));
      *reinterpret_cast<dfc*>(q.pw + (size_t)slot * q.n_atoms + a) = wc;
    } else {
      q.pw[(size_t)slot * q.n_atoms + a] = wv;
    }
    const double2 c2 = cmul(c, c);
    q.pcorr[(size_t)slot * q.n_atoms + a] = make_double2(E * c2.x / q.h3, E * c2.y / q.h3);
    __threadfence();
    const unsigned int tk = atomicAdd(q.ptickets + slot, 1u);
    s_last = (tk == (unsigned int)(q.n_atoms - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (tid < 32) {
    double cx = 0.0, cy = 0.0;
    const double2* src = q.pcorr + (size_t)slot * q.n_atoms;
    for (int k = tid; k < q.n_atoms; k += 32) {
      const double2 v = __ldcg(src + k);
      cx += v.x;
      cy += v.y;
    }
    cx = warp_sum(cx);
    cy = warp_sum(cy);
    // block-floating-point bound: |components of sum_a w_a p_a| at any point is at most (atoms at a
    // support point) x max_a (|Re w_a| + |Im w_a|) max|p_a|
    double wm = 0.0;
    if (MODE == RSFD_DF64 && p.bfp) {
      const dfc* wd = reinterpret_cast<const dfc*>(q.pw + (size_t)slot * q.n_atoms);
      for (int k = tid; k < q.n_atoms; k += 32) {
        const float2 wh = __ldcg(&wd[k].h);
        wm = fmax(wm, ((double)fabsf(wh.x) + (double)fabsf(wh.y)) * q.pmax[k]);
      }
      for (int o = 16; o > 0; o >>= 1) wm = fmax(wm, __shfl_xor_sync(0xffffffffu, wm, o));
    }
    if (tid == 0) {
      const double* dd = p.pdots + (size_t)slot * 8;
      S.rr = make_double2(__ldcg(dd + 0), __ldcg(dd + 1));
      S.rAr = make_double2(__ldcg(dd + 2) - cx, __ldcg(dd + 3) - cy);
      S.nrm2 = __ldcg(dd + 4);
      S.maxr = __ldcg(dd + 5);
      S.maxu = __ldcg(dd + 6) + (double)q.overlap * wm;
      q.ptickets[slot] = 0u;
    }
  }
  __syncthreads();
  scalar_step(p, slot, S);
}

// u (vector element) += pv * w for a real projector value pv and a complex FP64 coefficient w
__device__ __forceinline__ void scat_add(double2& u, double pv, double2 w) {
  u.x = fma(pv, w.x, u.x);
  u.y = fma(pv, w.y, u.y);
}

template <int MODE>
__global__ void __launch_bounds__(256) pscatter_kernel(ProjParams q) {
  typedef typename Ops<MODE>::C C;
  typedef typename Ops<MODE>::VT VT;
  const PassParams& p = q.pp;
  const int slot = blockIdx.y;
  SlotState* st = p.slots + slot;
  if (st->status != SLOT_RUNNING) return;
  const int n = st->n - 1;   // the scalar step of this iteration advanced n
  const long long vec = (long long)p.d.nz * p.d.ny * p.d.nxp;
  C* u = reinterpret_cast<C*>(p.rbuf) + ((size_t)slot * p.d.nvec + 3 + n % 2) * vec;
  const VT* tv = reinterpret_cast<const VT*>(q.t_val);
  const double2* w = q.pw + (size_t)slot * q.n_atoms;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < q.n_supp; s += gridDim.x * blockDim.x) {
    const long long gi = q.t_pidx[s];
    if (MODE == RSFD_DF64) {
      const dfc u0 = *reinterpret_cast<const dfc*>(&u[gi]);
      DFAcc acc = dfacc_from(u0);
      const dfc* wd = reinterpret_cast<const dfc*>(w);   // -E_a c_a as double-float pairs (proj_kernel)
      for (int e = q.t_ptr[s]; e < q.t_ptr[s + 1]; ++e) {
        const dfc wc = wd[q.t_atom[e]];
        const float2 pf = *reinterpret_cast<const float2*>(&tv[e]);
        dfr c;
        c.h = pf.x;
        c.l = pf.y;
        dfacc_mul(acc, c, wc);
      }
      *reinterpret_cast<dfc*>(&u[gi]) = dfacc_get(acc);
    } else {
      double2 uu;
      if (MODE == RSFD_FP64) {
        uu = *reinterpret_cast<const double2*>(&u[gi]);
      } else {
        const float2 uf = *reinterpret_cast<const float2*>(&u[gi]);
        uu = make_double2((double)uf.x, (double)uf.y);
      }
      for (int e = q.t_ptr[s]; e < q.t_ptr[s + 1]; ++e) {
        const double pd = (MODE == RSFD_FP64) ? (double)*reinterpret_cast<const double*>(&tv[e])
                                              : (double)*reinterpret_cast<const float*>(&tv[e]);
        scat_add(uu, pd, w[q.t_atom[e]]);
      }
      if (MODE == RSFD_FP64) *reinterpret_cast<double2*>(&u[gi]) = uu;
      else *reinterpret_cast<float2*>(&u[gi]) = make_float2((float)uu.x, (float)uu.y);
    }
  }
}

// ------------------------------------------------------------------------------------------------
// collapsed shift update over the recorded history (hcnt steps) of every (slot, energy)
// ------------------------------------------------------------------------------------------------
struct ChunkParams {
  SolveDims d;
  const void* rhist;
  void* xbuf;
  void* pbuf;
  const SlotState* slots;
  const ShiftCoef* coef;
  void* wbuf;                // [W][K][2][hist_len] H: W_x, W_p of the collapse
  double2* ebuf;             // [W][K][2]: e_x, e_p
  unsigned long long* counters;
  int hist_len;
};

// x / p element arithmetic per precision: upd(x, e, p, s) = x + e p + s
template <int MODE> struct XUpd;
template <> struct XUpd<RSFD_MIXED> {
  typedef float2 X;
  static __device__ __forceinline__ X updc(X x, float2 e, X p, float2 s) {
    return Ops<RSFD_MIXED>::mac(e, p, f2add(x, s));
  }
};
template <> struct XUpd<RSFD_FP64> {
  typedef double2 X;
  static __device__ __forceinline__ X updc(X x, double2 e, X p, double2 s) {
    return Ops<RSFD_FP64>::mac(e, p, make_double2(x.x + s.x, x.y + s.y));
  }
};
template <> struct XUpd<RSFD_DF64> {
  typedef dfc X;
  static __device__ __forceinline__ X updc(X x, const dfz& e, X p, float2 s) {
    dfc sd;
    sd.h = s;
    sd.l = make_float2(0.f, 0.f);
    return Ops<RSFD_DF64>::mac(e, p, df_add(x, sd));
  }
};

// Collapse coefficients of every (slot, energy), one thread each: backward recurrences
//   A_l = ca_l + cb_{l+1} A_{l+1},  B_l = cb_{l+1} B_{l+1}  (A_{hc-1} = ca_{hc-1}, B_{hc-1} = 1),
//   W_x[l] = A_l cr_l, W_p[l] = B_l cr_l, e_x = cb_0 A_0, e_p = cb_0 B_0   (FP64, rounded to H for W).
template <int MODE>
__global__ void __launch_bounds__(256) chunk_coef_kernel(ChunkParams p) {
  typedef typename Ops<MODE>::HR HR;
  typedef HOps<HR> HO;
  typedef typename HO::H H;
  const SolveDims& d = p.d;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d.W * d.K) return;
  const int slot = t / d.K, i = t - slot * d.K;
  const int hc = p.slots[slot].hcnt;
  if (hc <= 0) return;
  const ShiftCoef* cf = p.coef + ((size_t)slot * d.K + i) * p.hist_len;
  H* Wx = reinterpret_cast<H*>(p.wbuf) + ((size_t)slot * d.K + i) * 2 * p.hist_len;
  H* Wp = Wx + p.hist_len;
  double2 A = cf[hc - 1].ca, B = make_double2(1.0, 0.0);
  Wx[hc - 1] = HO::from(cmul(A, cf[hc - 1].cr));
  Wp[hc - 1] = HO::from(cmul(B, cf[hc - 1].cr));
  for (int l = hc - 2; l >= 0; --l) {
    A = cadd(cf[l].ca, cmul(cf[l + 1].cb, A));
    B = cmul(cf[l + 1].cb, B);
    Wx[l] = HO::from(cmul(A, cf[l].cr));
    Wp[l] = HO::from(cmul(B, cf[l].cr));
  }
  p.ebuf[((size_t)slot * d.K + i) * 2] = cmul(cf[0].cb, A);
  p.ebuf[((size_t)slot * d.K + i) * 2 + 1] = cmul(cf[0].cb, B);
  atomicAdd(&p.counters[0], (unsigned long long)hc);
  if (i == 0) atomicAdd(&p.counters[2], 1ull);
}

// Apply the collapsed update: a block owns kChunkRows boundary rows of one slot, stages those rows'
// residual history once in shared memory (each thread its own row) and sweeps every energy,
//   x <- x + e_x p + sum_l W_x[l] r_l,   p <- e_p p + sum_l W_p[l] r_l,
// in the same summation order as a per-energy sweep.  The weights and factors of kChunkE energies at
// a time are staged in shared memory (every thread reads the same weight: a broadcast), the factors
// already converted to the vector element's coefficient type.
constexpr int kChunkRows = 128;
constexpr int kChunkE = 16;
template <int MODE>
__global__ void __launch_bounds__(kChunkRows) chunk_apply_kernel(ChunkParams p) {
  typedef typename XUpd<MODE>::X X;
  typedef typename Ops<MODE>::HR HR;
  typedef typename Ops<MODE>::Cplx Cplx;
  typedef HOps<HR> HO;
  typedef typename HO::H H;
  extern __shared__ unsigned char chunk_smem[];
  const SolveDims& d = p.d;
  const int slot = blockIdx.y;
  const int hc = p.slots[slot].hcnt;
  if (hc <= 0) return;   // uniform over the block
  const int tid = threadIdx.x, row = blockIdx.x * kChunkRows + tid;
  const bool act = row < d.nb;
  H* hs = reinterpret_cast<H*>(chunk_smem);                    // [hist_len][kChunkRows]
  H* ws = hs + (size_t)p.hist_len * kChunkRows;                // [kChunkE][2][hist_len]
  Cplx* es = reinterpret_cast<Cplx*>(ws + (size_t)kChunkE * 2 * p.hist_len);   // [kChunkE][2]
  const H* h = reinterpret_cast<const H*>(p.rhist) + (size_t)slot * p.hist_len * d.nb;
  if (act)
    for (int l = 0; l < hc; ++l) hs[l * kChunkRows + tid] = h[(size_t)l * d.nb + row];
  const H* W = reinterpret_cast<const H*>(p.wbuf) + (size_t)slot * d.K * 2 * p.hist_len;
  const double2* E = p.ebuf + (size_t)slot * d.K * 2;
  X* x = reinterpret_cast<X*>(p.xbuf) + (size_t)slot * d.K * d.nb + row;
  X* pp = reinterpret_cast<X*>(p.pbuf) + (size_t)slot * d.K * d.nb + row;
  for (int i0 = 0; i0 < d.K; i0 += kChunkE) {
    const int ne = min(kChunkE, d.K - i0);
    __syncthreads();   // the previous batch's weights are no longer read
    for (int t = tid; t < ne * 2 * hc; t += kChunkRows) {
      const int ii = t / (2 * hc), rem = t - ii * 2 * hc;
      const int which = rem / hc, l = rem - which * hc;
      ws[(ii * 2 + which) * p.hist_len + l] = W[((size_t)(i0 + ii) * 2 + which) * p.hist_len + l];
    }
    for (int t = tid; t < ne * 2; t += kChunkRows) es[t] = Ops<MODE>::cplx(E[2 * i0 + t]);
    __syncthreads();
    if (!act) continue;
    for (int ii = 0; ii < ne; ++ii) {
      const H* Wx = ws + (size_t)ii * 2 * p.hist_len;
      const H* Wp = Wx + p.hist_len;
      H sx = HO::zero(), sp = HO::zero();
      for (int l = 0; l < hc; ++l) {
        const H r = hs[l * kChunkRows + tid];
        sx = HO::mac(Wx[l], r, sx);
        sp = HO::mac(Wp[l], r, sp);
      }
      const size_t o = (size_t)(i0 + ii) * d.nb;
      const X xo = x[o], po = pp[o];
      x[o] = XUpd<MODE>::updc(xo, es[2 * ii], po, sx);
      pp[o] = XUpd<MODE>::updc(X(), es[2 * ii + 1], po, sp);
    }
  }
}

__global__ void reset_hist_kernel(SlotState* slots, int W) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w < W) slots[w].hcnt = 0;
}

// ------------------------------------------------------------------------------------------------
// slot initialisation: r_{-1} = e_j, r_{-2} = 0, p = 0, x = 0, pi = 1
// ------------------------------------------------------------------------------------------------
struct InitParams {
  SolveDims d;
  void* rbuf;
  void* xbuf;
  void* pbuf;
  SlotState* slots;
  ShiftState* shifts;
  const double2* Z;
  const int* init_list;
  const long long* init_grid;
  int seed0;
  int kb;   // block-floating-point bound exponent of the pass (21)
};

template <int MODE>
__global__ void __launch_bounds__(256) init_kernel(InitParams p) {
  typedef typename Ops<MODE>::C C;
  typedef typename XUpd<MODE>::X X;
  const int e = blockIdx.y;
  const int slot = p.init_list[2 * e], col = p.init_list[2 * e + 1];
  const long long j = p.init_grid[e];
  const SolveDims& d = p.d;
  const long long nxy = (long long)d.nx * d.ny;
  const long long jz = j / nxy, jy = (j - jz * nxy) / d.nx, jx = j - jz * nxy - jy * d.nx;
  const long long vec = (long long)d.nz * d.ny * d.nxp;
  const long long jp = (jz * d.ny + jy) * d.nxp + jx;
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gs = (long long)gridDim.x * blockDim.x;
  C* r1 = reinterpret_cast<C*>(p.rbuf) + ((size_t)slot * d.nvec + 1) * vec;   // r_{-2}
  C* r2 = reinterpret_cast<C*>(p.rbuf) + ((size_t)slot * d.nvec + 2) * vec;   // r_{-1}
  for (long long t = gt; t < vec; t += gs) {
    r1[t] = Ops<MODE>::zero();
    r2[t] = (t == jp) ? Ops<MODE>::unit() : Ops<MODE>::zero();
  }
  if (d.nvec == 5) {   // stored products A r: the first pass multiplies u_{-1} by aA = 0
    C* u0 = reinterpret_cast<C*>(p.rbuf) + ((size_t)slot * 5 + 3) * vec;
    C* u1 = reinterpret_cast<C*>(p.rbuf) + ((size_t)slot * 5 + 4) * vec;
    for (long long t = gt; t < vec; t += gs) {
      u0[t] = Ops<MODE>::zero();
      u1[t] = Ops<MODE>::zero();
    }
  }
  X* xx = reinterpret_cast<X*>(p.xbuf) + (size_t)slot * d.K * d.nb;
  X* pp = reinterpret_cast<X*>(p.pbuf) + (size_t)slot * d.K * d.nb;
  const long long knb = (long long)d.K * d.nb;
  for (long long t = gt; t < knb; t += gs) {
    xx[t] = X();
    pp[t] = X();
  }
  (void)col;
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
    s.hcnt = 0;
    s.a1 = make_double2(1.0, 0.0);       // the first pass produces r_0 = r_{-1} = e_j
    s.a2 = make_double2(0.0, 0.0);
    s.aA = make_double2(0.0, 0.0);
    s.Zs = p.Z[p.seed0];
    s.alpha_prev = make_double2(1.0, 0.0);   // alpha_{-1} = 1
    s.rr_prev = make_double2(1.0, 0.0);
    s.carry = make_double2(1.0, 0.0);
    s.q = bfp_quantum(1.0, p.kb);   // r_0 = e_j: every component at most 1
    s.mr_prev = 1.0;
    p.slots[slot] = s;
  }
}

// ------------------------------------------------------------------------------------------------
// write-out of finished columns: G0_bb[k][:, col] = x^(k)_b
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ float2 convx(float2 x, float2*) { return x; }
__device__ __forceinline__ double2 convx(double2 x, double2*) { return x; }
__device__ __forceinline__ double2 convx(dfc x, double2*) {
  return make_double2((double)x.h.x + (double)x.l.x, (double)x.h.y + (double)x.l.y);
}

template <typename X, typename G>
__global__ void writeout_kernel(SolveDims d, const void* xbuf, void* G0, const int* list) {
  const int slot = list[2 * blockIdx.y], col = list[2 * blockIdx.y + 1];
  const long long knb = (long long)d.K * d.nb;
  const long long onb = (long long)d.kreq * d.nb;   // the set's energies come first in x_b
  const X* x = reinterpret_cast<const X*>(xbuf) + (size_t)slot * knb;
  G* g = reinterpret_cast<G*>(G0);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < onb; t += (long long)gridDim.x * blockDim.x) {
    const long long k = t / d.nb, row = t - k * d.nb;
    g[((size_t)k * d.ncols + col) * d.nb + row] = convx(x[t], (G*)nullptr);
  }
}

template <int MODE, int R>
PassParams pass_params(const SolveDims& d, const SolverBuffers& b, const StencilCoef& c, double tol, int maxit,
                       int hist_len) {
  PassParams p;
  p.d = d;
  p.rbuf = b.rbuf;
  p.V = b.V;
  p.rhist = b.rhist;
  p.slots = b.slots;
  p.shifts = b.shifts;
  p.coef = b.coef;
  p.partials = b.partials;
  p.tickets = b.tickets;
  p.Z = b.Z;
  p.counters = b.counters;
  p.error_flag = b.error_flag;
  p.hd = c.hd;
  p.hk1 = c.hk[0];
  p.hk2 = (R == 2) ? c.hk[1] : 0.0;
  p.tol = tol;
  p.maxit = maxit;
  p.hist_len = hist_len;
  p.depth = d.depth;
  p.stored_u = d.kind == RSFD_PASS_STORED || d.kind == RSFD_PASS_SPLIT || d.kind == RSFD_PASS_SPLIT_BFP;
  p.has_proj = b.n_atoms > 0;
  p.pdots = b.pdots;
  const bool bfp = MODE == RSFD_DF64 && d.kind == RSFD_PASS_SPLIT_BFP;
  p.bfp = bfp ? 1 : 0;
  p.kb = 21;
  p.uscale = bfp ? b.uscale : 1.0;
  p.Vs = b.Vs;
  return p;
}

template <int MODE, int R>
cudaError_t launch_pass_t(const SolveDims& d, const SolverBuffers& b, const StencilCoef& c, double tol, int maxit,
                          int hist_len, cudaStream_t st, cudaEvent_t mid, bool mid_external) {
  PassParams p = pass_params<MODE, R>(d, b, c, tol, maxit, hist_len);
  const bool bfp = p.bfp != 0;
  dim3 grid(d.ctas_per_slot, d.W);
  if (d.kind == RSFD_PASS_SPLIT || d.kind == RSFD_PASS_SPLIT_BFP) {
    if constexpr (MODE == RSFD_DF64) {
      if (bfp) combine_kernel<MODE, true><<<dim3(d.ctas_c, d.W), kCombThreads, 0, st>>>(p);
      else combine_kernel<MODE, false><<<dim3(d.ctas_c, d.W), kCombThreads, 0, st>>>(p);
    } else {
      combine_kernel<MODE, false><<<dim3(d.ctas_c, d.W), kCombThreads, 0, st>>>(p);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (mid) {   // profiling: the boundary between the combine and the stencil launch
      e = mid_external ? cudaEventRecordWithFlags(mid, st, cudaEventRecordExternal) : cudaEventRecord(mid, st);
      if (e != cudaSuccess) return e;
    }
    const size_t smem = split_smem(MODE, R, d.tile_y, d.depth);
    const int thr = split_threads(d.tile_y);
    if constexpr (MODE == RSFD_DF64) {
      if (bfp) {
        // register budget 1: at most 64 registers, two 512-thread (four 256-thread) CTAs per SM
        if (d.regs == 1) {
          if (thr <= 256) stencil_kernel<MODE, R, 256, 4, true><<<grid, thr, smem, st>>>(p, *b.tmR, *b.tmVs);
          else stencil_kernel<MODE, R, 512, 2, true><<<grid, thr, smem, st>>>(p, *b.tmR, *b.tmVs);
        } else {
          if (thr <= 256) stencil_kernel<MODE, R, 256, 3, true><<<grid, thr, smem, st>>>(p, *b.tmR, *b.tmVs);
          else stencil_kernel<MODE, R, 512, 1, true><<<grid, thr, smem, st>>>(p, *b.tmR, *b.tmVs);
        }
        return cudaGetLastError();
      }
    }
    if (thr <= 256) stencil_kernel<MODE, R, 256, 3><<<grid, thr, smem, st>>>(p, *b.tmR, *b.tmV);
    else stencil_kernel<MODE, R, 512, 1><<<grid, thr, smem, st>>>(p, *b.tmR, *b.tmV);
    return cudaGetLastError();
  }
  if (d.kind == RSFD_PASS_STORED) {
    const size_t smem = passu_smem(MODE, R, d.tile_y, d.depth, d.tile_x);
    const int thr = passu_threads(d.rows, R, d.tile_y, d.tile_x);
    if (d.rows == 1 && MODE == RSFD_DF64 && d.tile_x == 16)
      passu_kernel<MODE, R, 1, passu_budget_threads(0), 16><<<grid, thr, smem, st>>>(p, *b.tmR);
    else if (d.rows == 1 && MODE == RSFD_DF64 && d.regs == 1)
      passu_kernel<MODE, R, 1, passu_budget_threads(1)><<<grid, thr, smem, st>>>(p, *b.tmR);
    else if (d.rows == 1) passu_kernel<MODE, R, 1><<<grid, thr, smem, st>>>(p, *b.tmR);
    else if (d.rows == 2) passu_kernel<MODE, R, 2><<<grid, thr, smem, st>>>(p, *b.tmR);
    else passu_kernel<MODE, R, 4><<<grid, thr, smem, st>>>(p, *b.tmR);
  } else {
    const size_t smem = pass_smem(MODE, R, d.tile_y, d.depth);
    pass_kernel<MODE, R><<<grid, pass_threads(R, d.tile_y), smem, st>>>(p, *b.tmR, *b.tmV);
  }
  return cudaGetLastError();
}

}  // namespace

int pass_tile_x(int) { return kTileX; }
int pass_box_x() { return kBoxX; }
int pass_box_off() { return kBoxOff; }
int pass_threads(int R, int tile_y) { return (18 * (tile_y + 2 * R) + 31) / 32 * 32; }
size_t pass_smem(int prec, int R, int tile_y, int depth) {
  const size_t es = prec == RSFD_MIXED ? 8 : 16, vs = prec == RSFD_MIXED ? 4 : 8;
  const size_t EY = (size_t)tile_y + 4 * R;
  const size_t pc = (kBoxX * EY * es + 127) & ~(size_t)127, pv = (kBoxX * EY * vs + 127) & ~(size_t)127;
  const size_t stages = (size_t)depth + 1;
  return (size_t)(R + 1 + depth + stages + R + 2) * pc + stages * pv + 128;
}
int pass_max_depth() { return kMaxDepth; }
int split_threads(int tile_y) { return 32 * tile_y; }
size_t split_smem(int prec, int R, int tile_y, int depth) {
  const size_t es = prec == RSFD_MIXED ? 8 : 16;
  const size_t pb = ((size_t)(kTileX + 2 * kUBoxOff) * (tile_y + 2 * R) * es + 127) & ~(size_t)127;
  // per TMA stage the box of r_n and the tile of the potential
  const size_t vs = prec == RSFD_MIXED ? 4 : 8;
  const size_t pv = ((size_t)kTileX * tile_y * vs + 127) & ~(size_t)127;
  return (size_t)(depth + R + 1) * (pb + pv) + 128;
}
int split_combine_ctas(int nz, int W, int sms) {
  // about eight 256-thread CTAs per SM over all slots, at least one plane each
  int c = (8 * sms + W - 1) / W;
  if (c > nz) c = nz;
  if (c > 256) c = 256;
  return c < 1 ? 1 : c;
}
int passu_box_x(int tile_x) { return passu_box_w(tile_x); }
int passu_box_off() { return kUBoxOff; }
// tile threads (one x column and P rows each) plus the frame warps
int passu_threads(int rows, int R, int tile_y, int tile_x) {
  return 32 * (tile_y / rows) / (32 / tile_x) + 32 * passu_frame_warps(R, tile_y, tile_x);
}
int passu_max_threads(int rows, int budget) {
  if (rows == 1) return passu_budget_threads(budget);
  return rows == 2 ? MaxThreadsU<2>::value : MaxThreadsU<4>::value;
}
size_t passu_smem(int prec, int R, int tile_y, int depth, int tile_x) {
  const size_t es = prec == RSFD_MIXED ? 8 : 16;
  const size_t pb = ((size_t)passu_box_w(tile_x) * (tile_y + 2 * R) * es + 127) & ~(size_t)127;
  const size_t stages = (size_t)depth + 1;
  return stages * 3 * pb + (size_t)(R + 1) * pb + 128;
}
int pass_max_threads(int prec) {
  if (prec == RSFD_DF64) return MaxThreads<RSFD_DF64>::value;
  if (prec == RSFD_FP64) return MaxThreads<RSFD_FP64>::value;
  return MaxThreads<RSFD_MIXED>::value;
}

cudaError_t kernels_init() {
  const int lim = 216 * 1024;
  cudaError_t e = cudaSuccess;
#define RSFD_ATTR(M, R)                                                                                  \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(pass_kernel<M, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(passu_kernel<M, R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(passu_kernel<M, R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(passu_kernel<M, R, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  RSFD_ATTR(RSFD_FP64, 1)
  RSFD_ATTR(RSFD_FP64, 2)
  RSFD_ATTR(RSFD_MIXED, 1)
  RSFD_ATTR(RSFD_MIXED, 2)
  RSFD_ATTR(RSFD_DF64, 1)
  RSFD_ATTR(RSFD_DF64, 2)
#undef RSFD_ATTR
#define RSFD_ATTR_S(M, R)                                                                                \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_kernel<M, R, 256, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_kernel<M, R, 512, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  RSFD_ATTR_S(RSFD_FP64, 1)
  RSFD_ATTR_S(RSFD_FP64, 2)
  RSFD_ATTR_S(RSFD_MIXED, 1)
  RSFD_ATTR_S(RSFD_MIXED, 2)
  RSFD_ATTR_S(RSFD_DF64, 1)
  RSFD_ATTR_S(RSFD_DF64, 2)
#undef RSFD_ATTR_S
  if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_kernel<RSFD_DF64, 1, 256, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_kernel<RSFD_DF64, 1, 512, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_kernel<RSFD_DF64, 2, 256, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_kernel<RSFD_DF64, 2, 512, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_kernel<RSFD_DF64, 1, 256, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_kernel<RSFD_DF64, 1, 512, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_kernel<RSFD_DF64, 2, 256, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_kernel<RSFD_DF64, 2, 512, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(chunk_apply_kernel<RSFD_FP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(chunk_apply_kernel<RSFD_MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(chunk_apply_kernel<RSFD_DF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
#define RSFD_ATTR_B(R, B)                                                                                \
  if (e == cudaSuccess)                                                                                 \
    e = cudaFuncSetAttribute(passu_kernel<RSFD_DF64, R, 1, passu_budget_threads(B)>,                    \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  RSFD_ATTR_B(1, 1)
  RSFD_ATTR_B(2, 1)
#undef RSFD_ATTR_B
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(passu_kernel<RSFD_DF64, 1, 1, passu_budget_threads(0), 16>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(passu_kernel<RSFD_DF64, 2, 1, passu_budget_threads(0), 16>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  return e;
}

cudaError_t launch_pass(int prec, const SolveDims& d, const SolverBuffers& b, const StencilCoef& c, double tol,
                        int maxit, int hist_len, cudaStream_t st, cudaEvent_t mid, bool mid_external) {
  if (prec == RSFD_FP64)
    return d.R == 1 ? launch_pass_t<RSFD_FP64, 1>(d, b, c, tol, maxit, hist_len, st, mid, mid_external)
                    : launch_pass_t<RSFD_FP64, 2>(d, b, c, tol, maxit, hist_len, st, mid, mid_external);
  if (prec == RSFD_MIXED)
    return d.R == 1 ? launch_pass_t<RSFD_MIXED, 1>(d, b, c, tol, maxit, hist_len, st, mid, mid_external)
                    : launch_pass_t<RSFD_MIXED, 2>(d, b, c, tol, maxit, hist_len, st, mid, mid_external);
  return d.R == 1 ? launch_pass_t<RSFD_DF64, 1>(d, b, c, tol, maxit, hist_len, st, mid, mid_external)
                  : launch_pass_t<RSFD_DF64, 2>(d, b, c, tol, maxit, hist_len, st, mid, mid_external);
}

template <int MODE, int R>
cudaError_t launch_proj_t(const SolveDims& d, const SolverBuffers& b, const StencilCoef& c, double tol, int maxit,
                          int hist_len, cudaStream_t st) {
  ProjParams q;
  PassParams& p = q.pp;
  p.d = d;
  p.rbuf = b.rbuf;
  p.V = b.V;
  p.rhist = b.rhist;
  p.slots = b.slots;
  p.shifts = b.shifts;
  p.coef = b.coef;
  p.partials = b.partials;
  p.tickets = b.tickets;
  p.Z = b.Z;
  p.counters = b.counters;
  p.error_flag = b.error_flag;
  p.hd = c.hd;
  p.hk1 = c.hk[0];
  p.hk2 = (R == 2) ? c.hk[1] : 0.0;
  p.tol = tol;
  p.maxit = maxit;
  p.hist_len = hist_len;
  p.depth = d.depth;
  p.stored_u = 1;
  p.has_proj = 1;
  p.bfp = (MODE == RSFD_DF64 && d.kind == RSFD_PASS_SPLIT_BFP) ? 1 : 0;
  p.kb = 21;
  p.uscale = p.bfp ? b.uscale : 1.0;
  p.Vs = b.Vs;
  p.pdots = b.pdots;
  q.n_atoms = b.n_atoms;
  q.n_supp = b.n_supp;
  q.a_ptr = b.a_ptr;
  q.a_idx = b.a_idx;
  q.a_val = b.a_val;
  q.a_E = b.a_E;
  q.t_ptr = b.t_ptr;
  q.t_pidx = b.t_pidx;
  q.t_atom = b.t_atom;
  q.t_val = b.t_val;
  q.h3 = b.h3;
  q.pw = b.pw;
  q.pcorr = b.pcorr;
  q.ptickets = b.ptickets;
  q.pmax = b.a_pmax;
  q.overlap = b.proj_overlap;
  proj_kernel<MODE><<<dim3(b.n_atoms, d.W), kProjThreads, 0, st>>>(q);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int gx = (b.n_supp + 255) / 256;
  pscatter_kernel<MODE><<<dim3(gx < 1 ? 1 : gx, d.W), 256, 0, st>>>(q);
  return cudaGetLastError();
}

cudaError_t launch_proj(int prec, const SolveDims& d, const SolverBuffers& b, const StencilCoef& c, double tol,
                        int maxit, int hist_len, cudaStream_t st) {
  if (b.n_atoms <= 0) return cudaSuccess;
  if (prec == RSFD_FP64)
    return d.R == 1 ? launch_proj_t<RSFD_FP64, 1>(d, b, c, tol, maxit, hist_len, st)
                    : launch_proj_t<RSFD_FP64, 2>(d, b, c, tol, maxit, hist_len, st);
  if (prec == RSFD_MIXED)
    return d.R == 1 ? launch_proj_t<RSFD_MIXED, 1>(d, b, c, tol, maxit, hist_len, st)
                    : launch_proj_t<RSFD_MIXED, 2>(d, b, c, tol, maxit, hist_len, st);
  return d.R == 1 ? launch_proj_t<RSFD_DF64, 1>(d, b, c, tol, maxit, hist_len, st)
                  : launch_proj_t<RSFD_DF64, 2>(d, b, c, tol, maxit, hist_len, st);
}

cudaError_t launch_chunk(int prec, const SolveDims& d, const SolverBuffers& b, int hist_len, cudaStream_t st) {
  ChunkParams p;
  p.d = d;
  p.rhist = b.rhist;
  p.xbuf = b.xbuf;
  p.pbuf = b.pbuf;
  p.slots = b.slots;
  p.coef = b.coef;
  p.counters = b.counters;
  p.hist_len = hist_len;
  p.wbuf = b.cwbuf;
  p.ebuf = b.cebuf;
  const int nct = (d.W * d.K + 255) / 256;
  dim3 grid((d.nb + kChunkRows - 1) / kChunkRows, d.W);
  const size_t hsz = prec == RSFD_FP64 ? 16 : 8;            // history / weight element
  const size_t csz = prec == RSFD_MIXED ? 8 : 16;           // converted factor (float2, double2, dfz)
  const size_t smem = (size_t)hist_len * kChunkRows * hsz + (size_t)kChunkE * 2 * hist_len * hsz + kChunkE * 2 * csz;
  if (prec == RSFD_FP64) {
    chunk_coef_kernel<RSFD_FP64><<<nct, 256, 0, st>>>(p);
    chunk_apply_kernel<RSFD_FP64><<<grid, kChunkRows, smem, st>>>(p);
  } else if (prec == RSFD_MIXED) {
    chunk_coef_kernel<RSFD_MIXED><<<nct, 256, 0, st>>>(p);
    chunk_apply_kernel<RSFD_MIXED><<<grid, kChunkRows, smem, st>>>(p);
  } else {
    chunk_coef_kernel<RSFD_DF64><<<nct, 256, 0, st>>>(p);
    chunk_apply_kernel<RSFD_DF64><<<grid, kChunkRows, smem, st>>>(p);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reset_hist_kernel<<<(d.W + 255) / 256, 256, 0, st>>>(b.slots, d.W);
  return cudaGetLastError();
}

cudaError_t launch_slot_init(int prec, const SolveDims& d, const SolverBuffers& b, int n_init, int seed0,
                             cudaStream_t st) {
  if (n_init <= 0) return cudaSuccess;
  InitParams p;
  p.d = d;
  p.rbuf = b.rbuf;
  p.xbuf = b.xbuf;
  p.pbuf = b.pbuf;
  p.slots = b.slots;
  p.shifts = b.shifts;
  p.Z = b.Z;
  p.init_list = b.init_list;
  p.init_grid = b.init_grid;
  p.seed0 = seed0;
  p.kb = 21;
  const long long vec = (long long)d.nz * d.ny * d.nxp;
  long long work = vec > (long long)d.K * d.nb ? vec : (long long)d.K * d.nb;
  int gx = (int)((work + 255) / 256);
  if (gx > 512) gx = 512;
  dim3 grid(gx, n_init), block(256);
  if (prec == RSFD_FP64) init_kernel<RSFD_FP64><<<grid, block, 0, st>>>(p);
  else if (prec == RSFD_MIXED) init_kernel<RSFD_MIXED><<<grid, block, 0, st>>>(p);
  else init_kernel<RSFD_DF64><<<grid, block, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_writeout(int prec, const SolveDims& d, const SolverBuffers& b, void* G0, int n_out,
                            cudaStream_t st) {
  if (n_out <= 0) return cudaSuccess;
  const long long knb = (long long)d.K * d.nb;
  int gx = (int)((knb + 255) / 256);
  if (gx > 1024) gx = 1024;
  dim3 grid(gx, n_out), block(256);
  if (prec == RSFD_FP64) writeout_kernel<double2, double2><<<grid, block, 0, st>>>(d, b.xbuf, G0, b.init_list);
  else if (prec == RSFD_MIXED) writeout_kernel<float2, float2><<<grid, block, 0, st>>>(d, b.xbuf, G0, b.init_list);
  else writeout_kernel<dfc, double2><<<grid, block, 0, st>>>(d, b.xbuf, G0, b.init_list);
  return cudaGetLastError();
}

size_t vec_elem_bytes(int prec) { return prec == RSFD_MIXED ? 8 : 16; }
size_t pot_elem_bytes(int prec) { return prec == RSFD_MIXED ? 4 : 8; }
size_t hist_elem_bytes(int prec) { return prec == RSFD_FP64 ? 16 : 8; }

}  // namespace rsfd
