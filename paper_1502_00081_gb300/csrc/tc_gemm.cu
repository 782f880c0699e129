// Tensor-core pieces of the Dyson step (Eq. sec3-01a on the boundary rows): a batched complex
// FP32 GEMM on the 5th-generation tensor cores (tcgen05, kind::tf32) with the 3xTF32 split, and the
// FP32 blocked LU / triangular solves whose O(nb^3) updates it carries.
//
// 3xTF32: every FP32 operand x is split into hi = x with the 13 low mantissa bits cleared (exactly a
// TF32 number) and lo = x - hi (exact in FP32).  A product a*b is taken as
// a_hi*b_hi + a_hi*b_lo + a_lo*b_hi with FP32 accumulation in tensor memory; the dropped a_lo*b_lo
// and the TF32 rounding of lo are ~2^-21 relative, so the GEMM carries FP32-class accuracy.
// Complex C = A B takes four real products: Re = Ar Br - Ai Bi, Im = Ar Bi + Ai Br; the minus sign
// is the instruction descriptor's negate-A bit.  So one K-step of 8 issues 12 MMAs of 128 x BN x 8.
//
// Data path: column-major complex (interleaved re/im) operands are read from global memory by all
// 128 threads, split, and stored into eight shared-memory planes (re_hi, re_lo, im_hi, im_lo of A
// and of B) in the K-major, no-swizzle core-matrix layout of the tensor core (8 rows x 16 bytes per
// core matrix); thread 0 issues the MMAs for a stage and commits them to that stage's mbarrier, so
// the loads of stage s+1 overlap the MMAs of stage s.  The two accumulators (Re, Im: 128 lanes x BN
// FP32 columns each) live in tensor memory and are read back by tcgen05.ld for the epilogue
// C = alpha (Re + i Im) + beta C.

#include <cuda_runtime.h>
#include <stdint.h>

#include "rsfd_internal.cuh"

namespace rsfd {
namespace {

constexpr int TC_BM = 128;        // rows of C per CTA (MMA M)
constexpr int TC_BN = 128;        // columns of C per CTA (MMA N)
constexpr int TC_KC = 16;         // complex K elements per shared-memory stage (two MMA K-steps)
constexpr int TC_THREADS = 128;
constexpr int TC_PLANE_A = TC_BM * TC_KC * 4;   // bytes of one operand plane (8 KB)
constexpr int TC_PLANE_B = TC_BN * TC_KC * 4;
constexpr int TC_STAGE = 4 * TC_PLANE_A + 4 * TC_PLANE_B;
constexpr int TC_NSTAGE = 3;
constexpr int TC_SMEM = TC_NSTAGE * TC_STAGE + 1024;
constexpr int TC_TMEM_COLS = 2 * TC_BN;         // Re and Im accumulators
// core-matrix strides of a plane: 8-row groups are adjacent (128 B apart, the "stride" offset
// along M/N); groups of 4 K-elements are one plane-height apart (the "leading" offset along K)
constexpr uint32_t TC_SBO = 128;
constexpr uint32_t TC_LBO_A = (TC_BM / 8) * 128;
constexpr uint32_t TC_LBO_B = (TC_BN / 8) * 128;
constexpr long long kTcWaitCap = 1ll << 22;
constexpr int kTcPanel = 64;     // LU panel width = K of the trailing-update GEMMs

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of the 5th-generation tensor core
  return d;                 // base offset 0, absolute LBO mode off, layout SWIZZLE_NONE
}

// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N, int negA) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)negA << 13) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < kTcWaitCap; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void split3(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}

// byte offset of element (row, k) inside one plane of `rows` rows (K-major core matrices)
__device__ __forceinline__ uint32_t plane_off(int row, int kgrp, int rows) {
  return (uint32_t)((kgrp * (rows / 8) + (row >> 3)) * 128 + (row & 7) * 16);
}

// C[b] = alpha * A[b] * B[b] + beta * C[b]   (A m x k, B k x n, C m x n, column-major complex FP32)
__global__ void __launch_bounds__(TC_THREADS, 1)
cgemm_tf32x3_kernel(int m, int n, int k, float2 alpha, const float2* __restrict__ A, int lda, long long sA,
                    const float2* __restrict__ B, int ldb, long long sB, float beta, float2* C, int ldc,
                    long long sC, int* err, int vecB) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  __shared__ __align__(8) uint64_t bars[TC_NSTAGE];
  __shared__ uint32_t tmem_base_s;
  unsigned char* smem = (unsigned char*)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * TC_BN;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base_s)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < TC_NSTAGE; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_s;
  const uint32_t tm_re = tmem, tm_im = tmem + TC_BN;

  const int nchunks = (k + TC_KC - 1) / TC_KC;
  const uint32_t id_pos = idesc_tf32(TC_BM, TC_BN, 0), id_neg = idesc_tf32(TC_BM, TC_BN, 1);
  // raw operands of one K-chunk, loaded into registers one chunk ahead of the shared-memory stores:
  // thread tid holds row m0 + tid of A and column n0 + tid of B
  float2 ra[TC_KC], rb[TC_KC];
  auto load_chunk = [&](int kc) {
    const int k0 = kc * TC_KC;
    const int gi = m0 + tid, gj = n0 + tid;
#pragma unroll
    for (int q = 0; q < TC_KC; ++q) {
      const int kk = k0 + q;
      ra[q] = (gi < m && kk < k) ? A[(long long)kk * lda + gi] : make_float2(0.f, 0.f);
    }
    if (vecB && gj < n && k0 + TC_KC <= k) {
      const float4* src = reinterpret_cast<const float4*>(B + (long long)gj * ldb + k0);
#pragma unroll
      for (int q = 0; q < TC_KC / 2; ++q) {
        const float4 v = src[q];
        rb[2 * q] = make_float2(v.x, v.y);
        rb[2 * q + 1] = make_float2(v.z, v.w);
      }
    } else {
#pragma unroll
      for (int q = 0; q < TC_KC; ++q) {
        const int kk = k0 + q;
        rb[q] = (gj < n && kk < k) ? B[(long long)gj * ldb + kk] : make_float2(0.f, 0.f);
      }
    }
  };
  // split into TF32 hi / lo planes in the core-matrix layout of stage st
  auto store_chunk = [&](unsigned char* st) {
    unsigned char* sb = st + 4 * TC_PLANE_A;
#pragma unroll
    for (int g = 0; g < TC_KC / 4; ++g) {
      float rh[4], rl[4], ih[4], il[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        split3(ra[4 * g + q].x, rh[q], rl[q]);
        split3(ra[4 * g + q].y, ih[q], il[q]);
      }
      const uint32_t o = plane_off(tid, g, TC_BM);
      *(float4*)(st + 0 * TC_PLANE_A + o) = make_float4(rh[0], rh[1], rh[2], rh[3]);
      *(float4*)(st + 1 * TC_PLANE_A + o) = make_float4(rl[0], rl[1], rl[2], rl[3]);
      *(float4*)(st + 2 * TC_PLANE_A + o) = make_float4(ih[0], ih[1], ih[2], ih[3]);
      *(float4*)(st + 3 * TC_PLANE_A + o) = make_float4(il[0], il[1], il[2], il[3]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        split3(rb[4 * g + q].x, rh[q], rl[q]);
        split3(rb[4 * g + q].y, ih[q], il[q]);
      }
      const uint32_t ob = plane_off(tid, g, TC_BN);
      *(float4*)(sb + 0 * TC_PLANE_B + ob) = make_float4(rh[0], rh[1], rh[2], rh[3]);
      *(float4*)(sb + 1 * TC_PLANE_B + ob) = make_float4(rl[0], rl[1], rl[2], rl[3]);
      *(float4*)(sb + 2 * TC_PLANE_B + ob) = make_float4(ih[0], ih[1], ih[2], ih[3]);
      *(float4*)(sb + 3 * TC_PLANE_B + ob) = make_float4(il[0], il[1], il[2], il[3]);
    }
  };
  bool ok = true;
  if (nchunks > 0) load_chunk(0);
  for (int kc = 0; kc < nchunks && ok; ++kc) {
    const int s = kc % TC_NSTAGE;
    unsigned char* st = smem + s * TC_STAGE;
    // the stage is free once the MMAs of chunk kc - TC_NSTAGE (its previous user) have completed
    if (kc >= TC_NSTAGE) ok = bar_wait(smem_addr(&bars[s]), (uint32_t)(((kc - TC_NSTAGE) / TC_NSTAGE) & 1));
    store_chunk(st);
    if (kc + 1 < nchunks) load_chunk(kc + 1);   // in flight while this chunk's MMAs are issued
    // make the generic-proxy stores visible to the tensor core, then issue from one thread
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    ok = __syncthreads_and(ok) != 0;   // uniform: a CTA whose wait expired stops as a whole
    if (!ok) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_addr(st), b0 = smem_addr(st + 4 * TC_PLANE_A);
#pragma unroll
      for (int t = 0; t < TC_KC / 8; ++t) {
        const uint32_t ka = (uint32_t)(2 * t) * TC_LBO_A, kb = (uint32_t)(2 * t) * TC_LBO_B;
        const uint64_t arh = sdesc(a0 + 0 * TC_PLANE_A + ka, TC_LBO_A, TC_SBO);
        const uint64_t arl = sdesc(a0 + 1 * TC_PLANE_A + ka, TC_LBO_A, TC_SBO);
        const uint64_t aih = sdesc(a0 + 2 * TC_PLANE_A + ka, TC_LBO_A, TC_SBO);
        const uint64_t ail = sdesc(a0 + 3 * TC_PLANE_A + ka, TC_LBO_A, TC_SBO);
        const uint64_t brh = sdesc(b0 + 0 * TC_PLANE_B + kb, TC_LBO_B, TC_SBO);
        const uint64_t brl = sdesc(b0 + 1 * TC_PLANE_B + kb, TC_LBO_B, TC_SBO);
        const uint64_t bih = sdesc(b0 + 2 * TC_PLANE_B + kb, TC_LBO_B, TC_SBO);
        const uint64_t bil = sdesc(b0 + 3 * TC_PLANE_B + kb, TC_LBO_B, TC_SBO);
        const uint32_t acc0 = (kc > 0 || t > 0) ? 1u : 0u;
        // Re += Ar Br - Ai Bi   (small terms first)
        mma_tf32(tm_re, arl, brh, id_pos, acc0);
        mma_tf32(tm_re, arh, brl, id_pos, 1u);
        mma_tf32(tm_re, ail, bih, id_neg, 1u);
        mma_tf32(tm_re, aih, bil, id_neg, 1u);
        mma_tf32(tm_re, arh, brh, id_pos, 1u);
        mma_tf32(tm_re, aih, bih, id_neg, 1u);
        // Im += Ar Bi + Ai Br
        mma_tf32(tm_im, arl, bih, id_pos, acc0);
        mma_tf32(tm_im, arh, bil, id_pos, 1u);
        mma_tf32(tm_im, ail, brh, id_pos, 1u);
        mma_tf32(tm_im, aih, brl, id_pos, 1u);
        mma_tf32(tm_im, arh, bih, id_pos, 1u);
        mma_tf32(tm_im, aih, brh, id_pos, 1u);
      }
      mma_commit(smem_addr(&bars[s]));
    }
  }
  // the last commit covers every MMA issued before it
  if (ok && nchunks > 0)
    ok = bar_wait(smem_addr(&bars[(nchunks - 1) % TC_NSTAGE]), (uint32_t)(((nchunks - 1) / TC_NSTAGE) & 1));
  ok = __syncthreads_and(ok) != 0;
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok && nchunks > 0) {
    const int i = m0 + warp * 32 + lane;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
    for (int c0 = 0; c0 < TC_BN; c0 += 16) {
      if (n0 + c0 >= n) break;   // uniform across the CTA
      float re[16], im[16];
      tmem_ld16(tm_re + lane_off + c0, re);
      tmem_ld16(tm_im + lane_off + c0, im);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (i < m) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int j = n0 + c0 + q;
          if (j < n) {
            float2* c = C + (long long)j * ldc + i;
            float2 out = make_float2(alpha.x * re[q] - alpha.y * im[q], alpha.x * im[q] + alpha.y * re[q]);
            if (beta != 0.f) {
              const float2 old = *c;
              out.x += beta * old.x;
              out.y += beta * old.y;
            }
            *c = out;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
}

// ------------------------------------------------------------------------------------------------
// FP32 blocked LU with partial pivoting and the blocked triangular solves
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ float2 fmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 fsubc(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 frecip(float2 d) {
  // 1 / d by Smith's algorithm
  if (fabsf(d.x) >= fabsf(d.y)) {
    const float r = d.y / d.x, den = d.x + d.y * r;
    return make_float2(1.f / den, -r / den);
  }
  const float r = d.x / d.y, den = d.y + d.x * r;
  return make_float2(r / den, -1.f / den);
}

// Factorise columns j0 .. j0+jb-1 of every matrix (one CTA per matrix), LAPACK getrf order:
// piv[j] is the row exchanged with row j at step j; info[b] = first zero pivot (1-based).
__global__ void __launch_bounds__(256) panel_getrf_f32(float2* M, int nb, int j0, int jb, int* piv, int* info) {
  const int b = blockIdx.x;
  float2* A = M + (long long)b * nb * nb;
  int* pv = piv + (long long)b * nb;
  __shared__ float s_val[256];
  __shared__ int s_idx[256];
  __shared__ int s_p;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int j = j0; j < j0 + jb; ++j) {
    float best = -1.f;
    int bi = j;
    for (int i = j + tid; i < nb; i += nt) {
      const float2 a = A[(long long)j * nb + i];
      const float v = fabsf(a.x) + fabsf(a.y);
      if (v > best) { best = v; bi = i; }
    }
    s_val[tid] = best;
    s_idx[tid] = bi;
    __syncthreads();
    for (int s2 = nt / 2; s2 > 0; s2 >>= 1) {
      if (tid < s2) {
        if (s_val[tid + s2] > s_val[tid] || (s_val[tid + s2] == s_val[tid] && s_idx[tid + s2] < s_idx[tid])) {
          s_val[tid] = s_val[tid + s2];
          s_idx[tid] = s_idx[tid + s2];
        }
      }
      __syncthreads();
    }
    if (tid == 0) {
      s_p = s_idx[0];
      pv[j] = s_p;
      if (!(s_val[0] > 0.f) && info[b] == 0) info[b] = j + 1;
    }
    __syncthreads();
    const int p = s_p;
    if (p != j) {
      for (int c = j0 + tid; c < j0 + jb; c += nt) {
        const float2 t = A[(long long)c * nb + j];
        A[(long long)c * nb + j] = A[(long long)c * nb + p];
        A[(long long)c * nb + p] = t;
      }
    }
    __syncthreads();
    const float2 d = A[(long long)j * nb + j];
    const float2 inv = (d.x != 0.f || d.y != 0.f) ? frecip(d) : make_float2(0.f, 0.f);
    for (int i = j + 1 + tid; i < nb; i += nt) A[(long long)j * nb + i] = fmulc(A[(long long)j * nb + i], inv);
    __syncthreads();
    const int rem_r = nb - j - 1, rem_c = j0 + jb - j - 1;
    if (rem_c > 0) {
      for (int i = j + 1 + tid; i < nb; i += nt) {
        const float2 l = A[(long long)j * nb + i];
        for (int c = j + 1; c < j0 + jb; ++c) {
          float2& a = A[(long long)c * nb + i];
          a = fsubc(a, fmulc(l, A[(long long)c * nb + j]));
        }
      }
    }
    (void)rem_r;
    __syncthreads();
  }
}

// apply the exchanges of rows j0 .. j0+jb-1 (in order) to every column outside the panel
__global__ void laswp_f32(float2* M, int nb, int j0, int jb, const int* piv, int batch) {
  const int ncol = nb - jb;
  const long long tot = (long long)ncol * batch;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / ncol);
    int c = (int)(t - (long long)b * ncol);
    if (c >= j0) c += jb;
    float2* col = M + (long long)b * nb * nb + (long long)c * nb;
    const int* pv = piv + (long long)b * nb;
    for (int j = j0; j < j0 + jb; ++j) {
      const int p = pv[j];
      if (p != j) {
        const float2 x = col[j];
        col[j] = col[p];
        col[p] = x;
      }
    }
  }
}

// X[0:ib, c] = T^{-1} X[0:ib, c] for the ib x ib diagonal block T at (r0, r0) of each matrix;
// lower = 1: unit lower triangle, lower = 0: upper triangle with its diagonal.  T is staged in
// shared memory; one thread per right-hand-side column.  X has leading dimension ldx and batch
// stride sX; the factor has leading dimension nb and batch stride nb*nb.
template <int IB>
__global__ void __launch_bounds__(128) trsm_diag_f32(const float2* LU, int nb, int r0, int ib, float2* X, int ldx,
                                                    long long sX, int nrhs, int lower) {
  __shared__ float2 T[IB][IB + 1];
  const int b = blockIdx.y;
  const float2* F = LU + (long long)b * nb * nb;
  for (int t = threadIdx.x; t < ib * ib; t += blockDim.x) {
    const int c = t / ib, r = t - c * ib;
    T[r][c] = F[(long long)(r0 + c) * nb + r0 + r];
  }
  __syncthreads();
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= nrhs) return;
  float2* x = X + b * sX + (long long)col * ldx + r0;
  float2 v[IB];
#pragma unroll
  for (int i = 0; i < IB; ++i) v[i] = i < ib ? x[i] : make_float2(0.f, 0.f);
  if (lower) {
#pragma unroll
    for (int i = 1; i < IB; ++i) {
      float2 s = v[i];
#pragma unroll
      for (int q = 0; q < i; ++q) s = fsubc(s, fmulc(T[i][q], v[q]));
      v[i] = s;
    }
  } else {
#pragma unroll
    for (int i = IB - 1; i >= 0; --i) {
      if (i < ib) {
        float2 s = v[i];
#pragma unroll
        for (int q = i + 1; q < IB; ++q)
          if (q < ib) s = fsubc(s, fmulc(T[i][q], v[q]));
        v[i] = fmulc(s, frecip(T[i][i]));
      }
    }
  }
#pragma unroll
  for (int i = 0; i < IB; ++i)
    if (i < ib) x[i] = v[i];
}

// the row permutation of P^T: perm[i] = source row of row i after the exchanges piv[0 .. nb-1]
__global__ void perm_from_piv(const int* piv, int nb, int batch, int* perm) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const int* pv = piv + (long long)b * nb;
  int* pm = perm + (long long)b * nb;
  for (int i = 0; i < nb; ++i) pm[i] = i;
  for (int j = 0; j < nb; ++j) {
    const int p = pv[j];
    if (p != j) {
      const int t = pm[j];
      pm[j] = pm[p];
      pm[p] = t;
    }
  }
}

// dst[b][:, c][i] = src[b][:, c][perm[b][i]]  for nrhs columns of nb rows (FP64 -> FP32 or FP32 -> FP32)
template <typename S>
__global__ void gather_rows_f32(const S* src, int nb, int nrhs, const int* perm, float2* dst, int batch) {
  const long long per = (long long)nb * nrhs;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < per * batch;
       t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / per, e = t - b * per;
    const long long c = e / nb, i = e - c * nb;
    const S v = src[b * per + c * nb + perm[b * nb + i]];
    dst[t] = make_float2((float)v.x, (float)v.y);
  }
}

int grid_1d(long long n) {
  long long g = (n + 255) / 256;
  return (int)(g < 8192 ? (g < 1 ? 1 : g) : 8192);
}

bool g_tc_attr_set[16] = {false};

}  // namespace

cudaError_t cgemm_tf32x3(cudaStream_t st, int batch, int m, int n, int k, float2 alpha, const float2* A, int lda,
                         long long sA, const float2* B, int ldb, long long sB, float beta, float2* C, int ldc,
                         long long sC, int* err) {
  if (batch <= 0 || m <= 0 || n <= 0) return cudaSuccess;
  if (k <= 0) return cudaErrorInvalidValue;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 16 && !g_tc_attr_set[dev]) {
    e = cudaFuncSetAttribute(cgemm_tf32x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    g_tc_attr_set[dev] = true;
  }
  dim3 grid((n + TC_BN - 1) / TC_BN, (m + TC_BM - 1) / TC_BM, batch);
  // 16-byte loads of B columns when every column start (B + j ldb + k0, k0 a multiple of 16) is aligned
  const int vecB = ((uintptr_t)B % 16 == 0) && (ldb % 2 == 0) && (sB % 2 == 0);
  cgemm_tf32x3_kernel<<<grid, TC_THREADS, TC_SMEM, st>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC,
                                                         err, vecB);
  return cudaGetLastError();
}

int tc_panel() { return kTcPanel; }

// Batched blocked LU of K matrices nb x nb (FP32 complex, column-major, contiguous), in place.
cudaError_t getrf_f32_tc(cudaStream_t st, float2* M, int nb, int K, int* piv, int* info, int* err) {
  const long long n2 = (long long)nb * nb;
  const float2 m1 = make_float2(-1.f, 0.f);
  for (int j0 = 0; j0 < nb; j0 += kTcPanel) {
    const int jb = nb - j0 < kTcPanel ? nb - j0 : kTcPanel;
    panel_getrf_f32<<<K, 256, 0, st>>>(M, nb, j0, jb, piv, info);
    if (nb > jb) laswp_f32<<<grid_1d((long long)(nb - jb) * K), 256, 0, st>>>(M, nb, j0, jb, piv, K);
    const int rest = nb - j0 - jb;
    if (rest > 0) {
      // U12 = L11^{-1} A12: the panel's unit lower diagonal block applied to the columns right of it
      dim3 g((rest + 127) / 128, K);
      trsm_diag_f32<kTcPanel><<<g, 128, 0, st>>>(M, nb, j0, jb, M + (long long)(j0 + jb) * nb, nb, n2, rest, 1);
      // A22 -= L21 U12
      cudaError_t e = cgemm_tf32x3(st, K, rest, rest, jb, m1, M + (long long)j0 * nb + j0 + jb, nb, n2,
                                   M + (long long)(j0 + jb) * nb + j0, nb, n2, 1.f,
                                   M + (long long)(j0 + jb) * nb + j0 + jb, nb, n2, err);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

// X = U^{-1} L^{-1} P B for nrhs columns per matrix.  B (FP64 or FP32 complex, [K][nrhs][nb]) is
// permuted into X (FP32) first; perm is [K][nb] scratch.
template <typename S>
cudaError_t getrs_f32_tc_impl(cudaStream_t st, const float2* LU, const int* piv, int nb, int K, const S* B, int nrhs,
                              float2* X, int* perm, int* err) {
  const long long n2 = (long long)nb * nb, sx = (long long)nb * nrhs;
  const float2 m1 = make_float2(-1.f, 0.f);
  perm_from_piv<<<(K + 127) / 128, 128, 0, st>>>(piv, nb, K, perm);
  gather_rows_f32<S><<<grid_1d(sx * K), 256, 0, st>>>(B, nb, nrhs, perm, X, K);
  const int nblk = (nb + kTcPanel - 1) / kTcPanel;
  dim3 g((nrhs + 127) / 128, K);
  for (int bi = 0; bi < nblk; ++bi) {   // forward: unit lower L
    const int r0 = bi * kTcPanel, ib = nb - r0 < kTcPanel ? nb - r0 : kTcPanel;
    trsm_diag_f32<kTcPanel><<<g, 128, 0, st>>>(LU, nb, r0, ib, X, nb, sx, nrhs, 1);
    const int rest = nb - r0 - ib;
    if (rest > 0) {
      cudaError_t e = cgemm_tf32x3(st, K, rest, nrhs, ib, m1, LU + (long long)r0 * nb + r0 + ib, nb, n2, X + r0, nb,
                                   sx, 1.f, X + r0 + ib, nb, sx, err);
      if (e != cudaSuccess) return e;
    }
  }
  for (int bi = nblk - 1; bi >= 0; --bi) {   // backward: upper U
    const int r0 = bi * kTcPanel, ib = nb - r0 < kTcPanel ? nb - r0 : kTcPanel;
    trsm_diag_f32<kTcPanel><<<g, 128, 0, st>>>(LU, nb, r0, ib, X, nb, sx, nrhs, 0);
    if (r0 > 0) {
      cudaError_t e = cgemm_tf32x3(st, K, r0, nrhs, ib, m1, LU + (long long)r0 * nb, nb, n2, X + r0, nb, sx, 1.f, X,
                                   nb, sx, err);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

cudaError_t getrs_f32_tc(cudaStream_t st, const float2* LU, const int* piv, int nb, int K, const double2* B, int nrhs,
                         float2* X, int* perm, int* err) {
  return getrs_f32_tc_impl<double2>(st, LU, piv, nb, K, B, nrhs, X, perm, err);
}
cudaError_t getrs_f32_tc(cudaStream_t st, const float2* LU, const int* piv, int nb, int K, const float2* B, int nrhs,
                         float2* X, int* perm, int* err) {
  return getrs_f32_tc_impl<float2>(st, LU, piv, nb, K, B, nrhs, X, perm, err);
}

}  // namespace rsfd

// ------------------------------------------------------------------------------------------------
// C ABI: rsfd_cgemm_tf32x3
// ------------------------------------------------------------------------------------------------
namespace {
__device__ int g_cgemm_err;   // bounded-wait flag of rsfd_cgemm_tf32x3 calls
}

extern "C" rsfd_status rsfd_cgemm_tf32x3(int32_t batch, int32_t m, int32_t n, int32_t k, const double* alpha,
                                         const void* A, int32_t lda, int64_t sA, const void* B, int32_t ldb,
                                         int64_t sB, double beta, void* C, int32_t ldc, int64_t sC, void* stream) {
  if (batch < 0 || m < 0 || n < 0 || k < 1 || !alpha || (beta != 0.0 && beta != 1.0)) return RSFD_ERR_ARG;
  if (batch == 0 || m == 0 || n == 0) return RSFD_OK;
  if (!A || !B || !C || lda < m || ldb < k || ldc < m || sA < 0 || sB < 0 || sC < 0) return RSFD_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int* err = nullptr;
  if (cudaGetSymbolAddress((void**)&err, g_cgemm_err) != cudaSuccess) return RSFD_ERR_CUDA;
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return RSFD_ERR_CUDA;
  const float2 al = make_float2((float)alpha[0], (float)alpha[1]);
  if (rsfd::cgemm_tf32x3(st, batch, m, n, k, al, (const float2*)A, lda, sA, (const float2*)B, ldb, sB, (float)beta,
                         (float2*)C, ldc, sC, err) != cudaSuccess)
    return RSFD_ERR_CUDA;
  int herr = 0;
  if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return RSFD_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return RSFD_ERR_CUDA;
  return herr ? RSFD_ERR_TIMEOUT : RSFD_OK;
}
