// Dyson / OBM boundary step and Fisher-Lee transmission.
//
// G0_bb -> G_bb: the exact relation of Eq. sec3-01a restricted to the boundary rows is the
// linear system (I - G0_bb Sigma_bb) G_bb = G0_bb with Sigma_bb = diag(Sigma_L, Sigma_R)
// (equivalent to the block formulas Eqs. sec3-02 ... sec3-06).  Every energy is an independent
// dense complex solve of size nb; the batch is processed with:
//   1. M = I - G0 Sigma           (batched complex GEMM, FP64)
//   2. M = P L U                  (batched blocked right-looking LU with partial pivoting, FP64;
//                                  panels of 32 columns, trailing updates by the batched GEMM)
//   3. G = U^{-1} L^{-1} P G0     (batched triangular solves)
//   4. FP64 iterative refinement: R = G0 - M G, G += M^{-1} R (twice), reporting ||R||/||G0||.
// T(E) = Tr[Gamma_L G_RL^H Gamma_R G_RL] (Eq. TF) with Gamma = i (Sigma - Sigma^H) is two
// GEMMs and a trace per energy.  All matrices are column-major per energy.

#include <cuda_runtime.h>
#include <math.h>

#include <cmath>
#include <cstdlib>

#include <string>
#include <vector>

#include "rsfd_internal.cuh"

namespace rsfd {
namespace {

constexpr int GT = 16;   // GEMM tile

// C[b] = alpha * op(A[b]) * B[b] + beta * C[b];  op = N or H (conjugate transpose).
// A: if opA == 0, m x k (lda); if opA == 1, k x m stored, used as its conjugate transpose.
__global__ void zgemm_batched(int m, int n, int k, double2 alpha, const double2* A, int lda, long long sA, int opA,
                              const double2* B, int ldb, long long sB, double2 beta, double2* C, int ldc,
                              long long sC) {
  __shared__ double2 As[GT][GT + 1];
  __shared__ double2 Bs[GT][GT + 1];
  const int bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int row = blockIdx.y * GT + ty;   // i in C
  const int col = blockIdx.x * GT + tx;   // j in C
  double2 acc = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < k; k0 += GT) {
    // A tile: rows blockIdx.y*GT + ty, cols k0 + tx
    {
      const int i = blockIdx.y * GT + ty, kk = k0 + tx;
      double2 v = make_double2(0.0, 0.0);
      if (i < m && kk < k) {
        if (opA == 0) v = A[(long long)kk * lda + i];
        else {
          v = A[(long long)i * lda + kk];
          v.y = -v.y;
        }
      }
      As[ty][tx] = v;
    }
    {
      const int kk = k0 + ty, j = blockIdx.x * GT + tx;
      Bs[ty][tx] = (kk < k && j < n) ? B[(long long)j * ldb + kk] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < GT; ++t) {
      const double2 a = As[ty][t], b = Bs[t][tx];
      acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
      acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
    }
    __syncthreads();
  }
  if (row < m && col < n) {
    double2* c = C + (long long)col * ldc + row;
    double2 old = (beta.x != 0.0 || beta.y != 0.0) ? *c : make_double2(0.0, 0.0);
    *c = cadd(cmul(alpha, acc), cmul(beta, old));
  }
}

void zgemm(cudaStream_t st, int batch, int m, int n, int k, double2 alpha, const double2* A, int lda, long long sA,
           int opA, const double2* B, int ldb, long long sB, double2 beta, double2* C, int ldc, long long sC) {
  dim3 grid((n + GT - 1) / GT, (m + GT - 1) / GT, batch), block(GT, GT);
  zgemm_batched<<<grid, block, 0, st>>>(m, n, k, alpha, A, lda, sA, opA, B, ldb, sB, beta, C, ldc, sC);
}

template <typename T>
__global__ void to_c128(const T* src, double2* dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = make_double2((double)src[i].x, (double)src[i].y);
}
__global__ void from_c128_f(const double2* src, float2* dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}
__global__ void copy_c128(const double2* src, double2* dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}
__device__ __forceinline__ void cvt(double2 a, double2& b) { b = a; }
__device__ __forceinline__ void cvt(double2 a, float2& b) { b = make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ void cvt(float2 a, double2& b) { b = make_double2((double)a.x, (double)a.y); }
// dst[b ds + i] = src[b ss + i] for i < n, b < batch (a block of leading columns of each energy's
// matrix, with a type conversion where the types differ)
template <typename S, typename D>
__global__ void copy_batched(const S* src, long long ss, D* dst, long long ds, long long n, int batch) {
  const long long tot = n * batch;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / n, i = t - b * n;
    cvt(src[b * ss + i], dst[b * ds + i]);
  }
}
// dst[b ds + off + i] = 0 for i < n, b < batch
template <typename D>
__global__ void zero_batched(D* dst, long long ds, long long off, long long n, int batch) {
  const long long tot = n * batch;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / n, i = t - b * n;
    D z;
    z.x = 0;
    z.y = 0;
    dst[b * ds + off + i] = z;
  }
}

// M = I - G0 * blockdiag(SL, SR) is formed by two GEMMs after M = I.
__global__ void set_identity(double2* M, int nb, int batch) {
  const long long n2 = (long long)nb * nb;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n2 * batch;
       t += (long long)gridDim.x * blockDim.x) {
    const long long e = t % n2;
    const long long c = e / nb, r = e - c * nb;
    M[t] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
}

// Blocked right-looking LU with partial pivoting (LAPACK getrf order: piv[j] is the row exchanged
// with row j at step j).  Panels of kPanel columns are factorised by one CTA per matrix; the row
// exchanges are then applied to the other columns, U12 = L11^{-1} A12 is solved, and the trailing
// block is updated by the batched GEMM, which spreads the O(nb^3) work over every SM.
constexpr int kPanel = 32;

__global__ void __launch_bounds__(256) panel_getrf(double2* M, int nb, int j0, int jb, int* piv, int* info) {
  const int b = blockIdx.x;
  double2* A = M + (long long)b * nb * nb;
  int* pv = piv + (long long)b * nb;
  __shared__ double s_val[256];
  __shared__ int s_idx[256];
  __shared__ int s_p;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int j = j0; j < j0 + jb; ++j) {
    double best = -1.0;
    int bi = j;
    for (int i = j + tid; i < nb; i += nt) {
      const double v = cabs2(A[(long long)j * nb + i]);
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
      if (!(s_val[0] > 0.0) && info[b] == 0) info[b] = j + 1;
    }
    __syncthreads();
    const int p = s_p;
    if (p != j) {   // exchange rows j and p inside the panel
      for (int c = j0 + tid; c < j0 + jb; c += nt) {
        const double2 t = A[(long long)c * nb + j];
        A[(long long)c * nb + j] = A[(long long)c * nb + p];
        A[(long long)c * nb + p] = t;
      }
    }
    __syncthreads();
    const double2 d = A[(long long)j * nb + j];
    const double2 inv = (d.x != 0.0 || d.y != 0.0) ? cdiv(make_double2(1.0, 0.0), d) : make_double2(0.0, 0.0);
    for (int i = j + 1 + tid; i < nb; i += nt) A[(long long)j * nb + i] = cmul(A[(long long)j * nb + i], inv);
    __syncthreads();
    const int rem_r = nb - j - 1, rem_c = j0 + jb - j - 1;
    const long long tot = (long long)rem_r * rem_c;
    for (long long t = tid; t < tot; t += nt) {
      const int c = j + 1 + (int)(t / rem_r), i = j + 1 + (int)(t % rem_r);
      const double2 l = A[(long long)j * nb + i], u = A[(long long)c * nb + j];
      double2& a = A[(long long)c * nb + i];
      a = csub(a, cmul(l, u));
    }
    __syncthreads();
  }
}

// apply the exchanges of rows j0 .. j0 + jb - 1 (in order) to every column outside the panel
__global__ void panel_laswp(double2* M, int nb, int j0, int jb, const int* piv, int batch) {
  const int ncol = nb - jb;
  const long long tot = (long long)ncol * batch;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / ncol);
    int c = (int)(t - (long long)b * ncol);
    if (c >= j0) c += jb;
    double2* col = M + (long long)b * nb * nb + (long long)c * nb;
    const int* pv = piv + (long long)b * nb;
    for (int j = j0; j < j0 + jb; ++j) {
      const int p = pv[j];
      if (p != j) {
        const double2 x = col[j];
        col[j] = col[p];
        col[p] = x;
      }
    }
  }
}

// U12 = L11^{-1} A12 (L11 unit lower jb x jb), one thread per column right of the panel
__global__ void panel_trsm(double2* M, int nb, int j0, int jb, int batch) {
  const int ncol = nb - j0 - jb;
  const long long tot = (long long)ncol * batch;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / ncol);
    const int c = j0 + jb + (int)(t - (long long)b * ncol);
    double2* A = M + (long long)b * nb * nb;
    double2* col = A + (long long)c * nb;
    for (int i = j0 + 1; i < j0 + jb; ++i) {
      double2 s = col[i];
      for (int k = j0; k < i; ++k) s = csub(s, cmul(A[(long long)k * nb + i], col[k]));
      col[i] = s;
    }
  }
}

// Solve (P L U) X = B in place for nrhs columns; one thread per right-hand side column.
__global__ void zgetrs_batched(const double2* LU, const int* piv, double2* B, int nb, int nrhs) {
  const int b = blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nrhs) return;
  const double2* A = LU + (long long)b * nb * nb;
  const int* pv = piv + (long long)b * nb;
  double2* x = B + ((long long)b * nrhs + c) * nb;
  for (int j = 0; j < nb; ++j) {
    const int p = pv[j];
    if (p != j) {
      const double2 t = x[j];
      x[j] = x[p];
      x[p] = t;
    }
  }
  for (int i = 0; i < nb; ++i) {       // unit lower
    double2 s = x[i];
    for (int k = 0; k < i; ++k) s = csub(s, cmul(A[(long long)k * nb + i], x[k]));
    x[i] = s;
  }
  for (int i = nb - 1; i >= 0; --i) {  // upper
    double2 s = x[i];
    for (int k = i + 1; k < nb; ++k) s = csub(s, cmul(A[(long long)k * nb + i], x[k]));
    x[i] = cdiv(s, A[(long long)i * nb + i]);
  }
}

__global__ void axpy_c128(double2* y, const double2* x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = cadd(y[i], x[i]);
}

// out[b] = sum |A[b]|^2 over n2 entries (FP64, block per batch entry)
__global__ void frob2_batched(const double2* A, long long n2, double* out) {
  const int b = blockIdx.x;
  const double2* a = A + (long long)b * n2;
  double s = 0.0;
  for (long long i = threadIdx.x; i < n2; i += blockDim.x) s += cabs2(a[i]);
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[b] = red[0];
}

// Gamma = i (S - S^H) for a batch of ns x ns matrices
__global__ void gamma_batched(const double2* S, double2* G, int ns, int batch) {
  const long long n2 = (long long)ns * ns;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n2 * batch;
       t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / n2, e = t - b * n2;
    const int c = (int)(e / ns), r = (int)(e - (long long)c * ns);
    const double2 a = S[t], bt = S[b * n2 + (long long)r * ns + c];   // S[c, r]
    // S - S^H at (r, c) = a - conj(S[c, r]);  times i
    const double2 d = make_double2(a.x - bt.x, a.y + bt.y);
    G[t] = make_double2(-d.y, d.x);
  }
}

// T[b] = Re sum_{a,c} GL[a,c] * W[c,a]
__global__ void trace_prod_batched(const double2* GL, const double2* W, int ns, double* T, double* Ti) {
  const int b = blockIdx.x;
  const long long n2 = (long long)ns * ns;
  const double2* g = GL + (long long)b * n2;
  const double2* w = W + (long long)b * n2;
  double sr = 0.0, si = 0.0;
  for (long long t = threadIdx.x; t < n2; t += blockDim.x) {
    const int c = (int)(t / ns), a = (int)(t - (long long)c * ns);
    const double2 x = g[t], y = w[(long long)a * ns + c];   // GL[a,c], W[c,a]
    sr += x.x * y.x - x.y * y.y;
    si += x.x * y.y + x.y * y.x;
  }
  __shared__ double r1[256], r2[256];
  r1[threadIdx.x] = sr;
  r2[threadIdx.x] = si;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      r1[threadIdx.x] += r1[threadIdx.x + k];
      r2[threadIdx.x] += r2[threadIdx.x + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    T[b] = r1[0];
    Ti[b] = r2[0];
  }
}

// dst[b][c][0:nrow] = src[b][c][0:nrow] for ncol columns: the leading rows of a column-major block
__global__ void copy_rows_c128(const double2* src, int lds, double2* dst, int ldd, int nrow, int ncol, int batch) {
  const long long per = (long long)nrow * ncol;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < per * batch;
       t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / per, e = t - b * per;
    const long long c = e / nrow, i = e - c * nrow;
    dst[(b * ncol + c) * ldd + i] = src[(b * ncol + c) * lds + i];
  }
}

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)(g < 4096 ? (g < 1 ? 1 : g) : 4096);
}

// batched blocked LU of K matrices nb x nb (column-major, contiguous), in place
void getrf_blocked(cudaStream_t st, double2* M, int nb, int K, int* piv, int* info) {
  const double2 m1 = make_double2(-1.0, 0.0), one = make_double2(1.0, 0.0);
  const long long n2 = (long long)nb * nb;
  for (int j0 = 0; j0 < nb; j0 += kPanel) {
    const int jb = nb - j0 < kPanel ? nb - j0 : kPanel;
    panel_getrf<<<K, 256, 0, st>>>(M, nb, j0, jb, piv, info);
    if (nb > jb) panel_laswp<<<grid_for((long long)(nb - jb) * K), 256, 0, st>>>(M, nb, j0, jb, piv, K);
    const int rest = nb - j0 - jb;
    if (rest > 0) {
      panel_trsm<<<grid_for((long long)rest * K), 256, 0, st>>>(M, nb, j0, jb, K);
      // A22 -= L21 U12
      zgemm(st, K, rest, rest, jb, m1, M + (long long)j0 * nb + j0 + jb, nb, n2, 0, M + (long long)(j0 + jb) * nb + j0,
            nb, n2, one, M + (long long)(j0 + jb) * nb + j0 + jb, nb, n2);
    }
  }
}

}  // namespace

#define DY_CK(h, call)                                                                                  \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) return handle_fail((h), RSFD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

__global__ void to_f32_c(const double2* src, float2* dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}
__global__ void add_f32_to_c128(double2* y, const float2* x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = make_double2(y[i].x + (double)x[i].x, y[i].y + (double)x[i].y);
}
__global__ void set_f32_to_c128(double2* y, const float2* x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = make_double2((double)x[i].x, (double)x[i].y);
}

// Tensor-core form of the Dyson step, energies processed in chunks that fit the device:
//   M = I - G0 Sigma                       FP64 (CUDA cores)
//   F = P L U of M in FP32                 panels on the CUDA cores, trailing updates 3xTF32 (tcgen05)
//   X = F^{-1} G0                          blocked triangular solves, updates 3xTF32 (tcgen05)
//   nref times: R = G0 - M X (FP64), X += F^{-1} R
// Reported residual ||G0 - M X|| / ||G0|| is the FP64 one after the last correction.
rsfd_status dyson_tc_run(Handle* h, const void* G0, const void* SL, const void* SR, int K, void* G, double* refres) {
  const int nb = handle_nb(h);
  const int ns = nb / 2;
  const long long n2 = (long long)nb * nb, s2 = (long long)ns * ns;
  const bool fp64in = handle_prec(h) != RSFD_MIXED;
  const int nref = handle_dyson_refine(h);
  // columns solved: all nb, or the left slab's ns (the block of G_bb the transmission uses)
  const int nc = handle_dyson_cols(h) == 1 ? ns : nb;
  const long long sx = (long long)nb * nc;
  // per energy: M (c128), X, R and the compact right-hand side (c128, nb x nc), the G0 copy when the
  // input is complex64, F (c64) and the FP32 solve (c64, nb x nc)
  const long long per = n2 * (16 + (fp64in ? 0 : 16) + 8) + sx * (3 * 16 + 8) + (long long)nb * 8 + 64;
  size_t free_b = 0, tot_b = 0;
  DY_CK(h, cudaMemGetInfo(&free_b, &tot_b));
  long long kc = (long long)(0.6 * (double)free_b) / per;
  if (kc > K) kc = K;
  if (kc < 1) kc = 1;
  const int Kc = (int)kc;
  rsfd_status s;
  void *pM, *pX, *pR, *pF, *pPiv, *pRed, *pG0, *pB;
  if ((s = handle_ensure(h, 1, n2 * Kc * sizeof(double2), &pM)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 3, sx * Kc * sizeof(double2), &pX)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 4, sx * Kc * sizeof(double2), &pR)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 2, (n2 + sx) * Kc * sizeof(float2), &pF)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 5, ((long long)Kc * (2 * nb + 1) + 1) * sizeof(int), &pPiv)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 6, (long long)2 * K * sizeof(double), &pRed)) != RSFD_OK) return s;
  if (!fp64in && (s = handle_ensure(h, 0, n2 * Kc * sizeof(double2), &pG0)) != RSFD_OK) return s;
  if (nc < nb && (s = handle_ensure(h, 7, sx * Kc * sizeof(double2), &pB)) != RSFD_OK) return s;
  if ((s = handle_begin(h)) != RSFD_OK) return s;
  cudaStream_t st = handle_stream(h);
  double2* dM = (double2*)pM;
  double2* dX = (double2*)pX;
  double2* dR = (double2*)pR;
  float2* dF = (float2*)pF;
  float2* dXf = dF + n2 * Kc;
  int* piv = (int*)pPiv;
  int* perm = piv + (long long)Kc * nb;
  int* info = perm + (long long)Kc * nb;
  int* err = info + Kc;
  double* red = (double*)pRed;
  const double2 m1 = make_double2(-1.0, 0.0), one = make_double2(1.0, 0.0);
  DY_CK(h, cudaMemsetAsync(err, 0, sizeof(int), st));
  std::vector<int> hinfo(K, 0);
  for (int k0 = 0; k0 < K; k0 += Kc) {
    const int kb = K - k0 < Kc ? K - k0 : Kc;
    const long long tot = n2 * kb, totx = sx * kb;
    const double2* g0;
    if (fp64in) {
      g0 = (const double2*)G0 + n2 * k0;
    } else {
      to_c128<float2><<<grid_for(tot), 256, 0, st>>>((const float2*)G0 + n2 * k0, (double2*)pG0, tot);
      g0 = (const double2*)pG0;
    }
    // right-hand sides: G0's first nc columns of every energy, compact (stride sx)
    const double2* b0 = g0;
    if (nc < nb) {
      copy_batched<double2, double2><<<grid_for(totx), 256, 0, st>>>(g0, n2, (double2*)pB, sx, sx, kb);
      b0 = (const double2*)pB;
    }
    const double2* sl = (const double2*)SL + s2 * k0;
    const double2* sr = (const double2*)SR + s2 * k0;
    set_identity<<<grid_for(tot), 256, 0, st>>>(dM, nb, kb);
    zgemm(st, kb, nb, ns, ns, m1, g0, nb, n2, 0, sl, ns, s2, one, dM, nb, n2);
    zgemm(st, kb, nb, ns, ns, m1, g0 + (long long)ns * nb, nb, n2, 0, sr, ns, s2, one, dM + (long long)ns * nb, nb, n2);
    to_f32_c<<<grid_for(tot), 256, 0, st>>>(dM, dF, tot);
    DY_CK(h, cudaMemsetAsync(info, 0, kb * sizeof(int), st));
    DY_CK(h, getrf_f32_tc(st, dF, nb, kb, piv, info, err));
    DY_CK(h, getrs_f32_tc(st, dF, piv, nb, kb, b0, nc, dXf, perm, err));
    set_f32_to_c128<<<grid_for(totx), 256, 0, st>>>(dX, dXf, totx);
    for (int it = 0; it < nref; ++it) {
      copy_c128<<<grid_for(totx), 256, 0, st>>>(b0, dR, totx);
      zgemm(st, kb, nb, nc, nb, m1, dM, nb, n2, 0, dX, nb, sx, one, dR, nb, sx);
      DY_CK(h, getrs_f32_tc(st, dF, piv, nb, kb, (const double2*)dR, nc, dXf, perm, err));
      add_f32_to_c128<<<grid_for(totx), 256, 0, st>>>(dX, dXf, totx);
    }
    if (refres) {
      copy_c128<<<grid_for(totx), 256, 0, st>>>(b0, dR, totx);
      zgemm(st, kb, nb, nc, nb, m1, dM, nb, n2, 0, dX, nb, sx, one, dR, nb, sx);
      frob2_batched<<<kb, 256, 0, st>>>(dR, sx, red + k0);
      frob2_batched<<<kb, 256, 0, st>>>(b0, sx, red + K + k0);
    }
    if (fp64in) {
      copy_batched<double2, double2><<<grid_for(totx), 256, 0, st>>>(dX, sx, (double2*)G + n2 * k0, n2, sx, kb);
      if (nc < nb) zero_batched<double2><<<grid_for(tot - totx), 256, 0, st>>>((double2*)G + n2 * k0, n2, sx, n2 - sx, kb);
    } else {
      copy_batched<double2, float2><<<grid_for(totx), 256, 0, st>>>(dX, sx, (float2*)G + n2 * k0, n2, sx, kb);
      if (nc < nb) zero_batched<float2><<<grid_for(tot - totx), 256, 0, st>>>((float2*)G + n2 * k0, n2, sx, n2 - sx, kb);
    }
    DY_CK(h, cudaGetLastError());
    DY_CK(h, cudaMemcpyAsync(hinfo.data() + k0, info, kb * sizeof(int), cudaMemcpyDeviceToHost, st));
  }
  int herr = 0;
  DY_CK(h, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  std::vector<double> hred(2 * K);
  if (refres) DY_CK(h, cudaMemcpyAsync(hred.data(), red, 2 * K * sizeof(double), cudaMemcpyDeviceToHost, st));
  DY_CK(h, cudaStreamSynchronize(st));
  if ((s = handle_end(h)) != RSFD_OK) return s;
  if (herr) return handle_fail(h, RSFD_ERR_TIMEOUT, "rsfd_dyson_boundary: tensor-core GEMM wait expired");
  if (refres)
    for (int k = 0; k < K; ++k) refres[k] = sqrt(hred[k]) / sqrt(hred[K + k] > 0 ? hred[K + k] : 1.0);
  for (int k = 0; k < K; ++k)
    if (hinfo[k] != 0)
      return handle_fail(h, RSFD_ERR_BREAKDOWN, "rsfd_dyson_boundary: singular I - G0 Sigma at energy " + std::to_string(k));
  return RSFD_OK;
}

rsfd_status dyson_run(Handle* h, const void* G0, const void* SL, const void* SR, int K, void* G, double* refres) {
  if (handle_dyson_kind(h) == RSFD_DYSON_TC) return dyson_tc_run(h, G0, SL, SR, K, G, refres);
  const int nb = handle_nb(h);
  const int ns = nb / 2;
  const long long n2 = (long long)nb * nb;
  const bool fp64 = handle_prec(h) != RSFD_MIXED;   // FP64 and double-float handles hold c128 data
  rsfd_status s;
  void *pG0, *pM, *pLU, *pX, *pR, *pPiv, *pRed;
  if ((s = handle_ensure(h, 0, n2 * K * sizeof(double2), &pG0)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 1, n2 * K * sizeof(double2), &pM)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 2, n2 * K * sizeof(double2), &pLU)) != RSFD_OK) return s;
  // columns solved: all nb, or the left slab's ns (the block of G_bb the transmission uses)
  const int nc = handle_dyson_cols(h) == 1 ? ns : nb;
  const long long sx = (long long)nb * nc, totx = sx * K;
  if ((s = handle_ensure(h, 3, sx * K * sizeof(double2), &pX)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 4, sx * K * sizeof(double2), &pR)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 5, (long long)K * (nb + 1) * sizeof(int), &pPiv)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 6, (long long)2 * K * sizeof(double), &pRed)) != RSFD_OK) return s;
  if ((s = handle_begin(h)) != RSFD_OK) return s;
  cudaStream_t st = handle_stream(h);
  double2* dG0 = (double2*)pG0;
  double2* dM = (double2*)pM;
  double2* dLU = (double2*)pLU;
  double2* dX = (double2*)pX;
  double2* dR = (double2*)pR;
  int* piv = (int*)pPiv;
  int* info = piv + (long long)K * nb;
  double* red = (double*)pRed;
  const long long tot = n2 * K;
  if (fp64) copy_c128<<<grid_for(tot), 256, 0, st>>>((const double2*)G0, dG0, tot);
  else to_c128<float2><<<grid_for(tot), 256, 0, st>>>((const float2*)G0, dG0, tot);
  set_identity<<<grid_for(tot), 256, 0, st>>>(dM, nb, K);
  const double2 m1 = make_double2(-1.0, 0.0), one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  // M[:, :ns] -= G0[:, :ns] SL ;  M[:, ns:] -= G0[:, ns:] SR
  zgemm(st, K, nb, ns, ns, m1, dG0, nb, n2, 0, (const double2*)SL, ns, (long long)ns * ns, one, dM, nb, n2);
  zgemm(st, K, nb, ns, ns, m1, dG0 + (long long)ns * nb, nb, n2, 0, (const double2*)SR, ns, (long long)ns * ns, one,
        dM + (long long)ns * nb, nb, n2);
  copy_c128<<<grid_for(tot), 256, 0, st>>>(dM, dLU, tot);
  DY_CK(h, cudaMemsetAsync(info, 0, K * sizeof(int), st));
  getrf_blocked(st, dLU, nb, K, piv, info);
  // right-hand sides: the first nc columns of every energy, compact (stride sx)
  const double2* b0 = dG0;
  if (nc < nb) {
    void* pB = nullptr;
    if ((s = handle_ensure(h, 7, sx * K * sizeof(double2), &pB)) != RSFD_OK) return s;
    copy_batched<double2, double2><<<grid_for(totx), 256, 0, st>>>(dG0, n2, (double2*)pB, sx, sx, K);
    b0 = (const double2*)pB;
  }
  copy_c128<<<grid_for(totx), 256, 0, st>>>(b0, dX, totx);
  {
    dim3 g((nc + 127) / 128, K);
    zgetrs_batched<<<g, 128, 0, st>>>(dLU, piv, dX, nb, nc);
  }
  // iterative refinement in FP64
  for (int it = 0; it < 2; ++it) {
    copy_c128<<<grid_for(totx), 256, 0, st>>>(b0, dR, totx);
    zgemm(st, K, nb, nc, nb, m1, dM, nb, n2, 0, dX, nb, sx, one, dR, nb, sx);
    dim3 g((nc + 127) / 128, K);
    zgetrs_batched<<<g, 128, 0, st>>>(dLU, piv, dR, nb, nc);
    axpy_c128<<<grid_for(totx), 256, 0, st>>>(dX, dR, totx);
  }
  if (refres) {
    copy_c128<<<grid_for(totx), 256, 0, st>>>(b0, dR, totx);
    zgemm(st, K, nb, nc, nb, m1, dM, nb, n2, 0, dX, nb, sx, one, dR, nb, sx);
    frob2_batched<<<K, 256, 0, st>>>(dR, sx, red);
    frob2_batched<<<K, 256, 0, st>>>(b0, sx, red + K);
  }
  if (fp64) {
    copy_batched<double2, double2><<<grid_for(totx), 256, 0, st>>>(dX, sx, (double2*)G, n2, sx, K);
    if (nc < nb) zero_batched<double2><<<grid_for(tot - totx), 256, 0, st>>>((double2*)G, n2, sx, n2 - sx, K);
  } else {
    copy_batched<double2, float2><<<grid_for(totx), 256, 0, st>>>(dX, sx, (float2*)G, n2, sx, K);
    if (nc < nb) zero_batched<float2><<<grid_for(tot - totx), 256, 0, st>>>((float2*)G, n2, sx, n2 - sx, K);
  }
  DY_CK(h, cudaGetLastError());
  std::vector<int> hinfo(K);
  DY_CK(h, cudaMemcpyAsync(hinfo.data(), info, K * sizeof(int), cudaMemcpyDeviceToHost, st));
  std::vector<double> hred(2 * K);
  if (refres) DY_CK(h, cudaMemcpyAsync(hred.data(), red, 2 * K * sizeof(double), cudaMemcpyDeviceToHost, st));
  DY_CK(h, cudaStreamSynchronize(st));
  if ((s = handle_end(h)) != RSFD_OK) return s;
  if (refres)
    for (int k = 0; k < K; ++k) refres[k] = sqrt(hred[k]) / sqrt(hred[K + k] > 0 ? hred[K + k] : 1.0);
  for (int k = 0; k < K; ++k)
    if (hinfo[k] != 0)
      return handle_fail(h, RSFD_ERR_BREAKDOWN, "rsfd_dyson_boundary: singular I - G0 Sigma at energy " + std::to_string(k));
  (void)zero;
  return RSFD_OK;
}

// Dyson step on the recorded rows: G = G0 + G0[:, b] Sigma Y with Y = (I - G0_bb Sigma)^{-1} G0[b, :]
// (the boundary rows of G), all nr x nr per energy, column-major.
rsfd_status dyson_tracked_run(Handle* h, int nr, const void* G0, const void* SL, const void* SR, int K, void* G,
                              double* refres) {
  const int nb = handle_nb(h);
  const int ns = nb / 2;
  const long long r2 = (long long)nr * nr, b2 = (long long)nb * nb, bn = (long long)nb * nr;
  const bool fp64 = handle_prec(h) != RSFD_MIXED;
  rsfd_status s;
  void *pG0, *pM, *pLU, *pY, *pR, *pPiv, *pRed, *pW;
  if ((s = handle_ensure(h, 0, r2 * K * sizeof(double2), &pG0)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 1, b2 * K * sizeof(double2), &pM)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 2, b2 * K * sizeof(double2), &pLU)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 3, bn * K * sizeof(double2), &pY)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 4, bn * K * sizeof(double2), &pR)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 5, (long long)K * (nb + 1) * sizeof(int), &pPiv)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 6, (long long)2 * K * sizeof(double), &pRed)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 7, (2 * bn + r2) * K * sizeof(double2), &pW)) != RSFD_OK) return s;
  if ((s = handle_begin(h)) != RSFD_OK) return s;
  cudaStream_t st = handle_stream(h);
  double2* dG0 = (double2*)pG0;
  double2* dM = (double2*)pM;
  double2* dLU = (double2*)pLU;
  double2* dY = (double2*)pY;
  double2* dR = (double2*)pR;
  double2* dRHS = (double2*)pW;
  double2* dW = dRHS + bn * K;
  double2* dX = dW + bn * K;
  int* piv = (int*)pPiv;
  int* info = piv + (long long)K * nb;
  double* red = (double*)pRed;
  const long long rtot = r2 * K, btot = b2 * K, ntot = bn * K;
  if (fp64) copy_c128<<<grid_for(rtot), 256, 0, st>>>((const double2*)G0, dG0, rtot);
  else to_c128<float2><<<grid_for(rtot), 256, 0, st>>>((const float2*)G0, dG0, rtot);
  const double2 m1 = make_double2(-1.0, 0.0), one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  // M = I - G0_bb Sigma (G0_bb: the leading nb x nb block of G0, leading dimension nr)
  set_identity<<<grid_for(btot), 256, 0, st>>>(dM, nb, K);
  zgemm(st, K, nb, ns, ns, m1, dG0, nr, r2, 0, (const double2*)SL, ns, (long long)ns * ns, one, dM, nb, b2);
  zgemm(st, K, nb, ns, ns, m1, dG0 + (long long)ns * nr, nr, r2, 0, (const double2*)SR, ns, (long long)ns * ns, one,
        dM + (long long)ns * nb, nb, b2);
  copy_c128<<<grid_for(btot), 256, 0, st>>>(dM, dLU, btot);
  DY_CK(h, cudaMemsetAsync(info, 0, K * sizeof(int), st));
  getrf_blocked(st, dLU, nb, K, piv, info);
  // Y = M^{-1} G0[b, :] with two FP64 refinement steps
  copy_rows_c128<<<grid_for(ntot), 256, 0, st>>>(dG0, nr, dRHS, nb, nb, nr, K);
  copy_c128<<<grid_for(ntot), 256, 0, st>>>(dRHS, dY, ntot);
  dim3 g((nr + 127) / 128, K);
  zgetrs_batched<<<g, 128, 0, st>>>(dLU, piv, dY, nb, nr);
  for (int it = 0; it < 2; ++it) {
    copy_c128<<<grid_for(ntot), 256, 0, st>>>(dRHS, dR, ntot);
    zgemm(st, K, nb, nr, nb, m1, dM, nb, b2, 0, dY, nb, bn, one, dR, nb, bn);
    zgetrs_batched<<<g, 128, 0, st>>>(dLU, piv, dR, nb, nr);
    axpy_c128<<<grid_for(ntot), 256, 0, st>>>(dY, dR, ntot);
  }
  if (refres) {
    copy_c128<<<grid_for(ntot), 256, 0, st>>>(dRHS, dR, ntot);
    zgemm(st, K, nb, nr, nb, m1, dM, nb, b2, 0, dY, nb, bn, one, dR, nb, bn);
    frob2_batched<<<K, 256, 0, st>>>(dR, bn, red);
    frob2_batched<<<K, 256, 0, st>>>(dRHS, bn, red + K);
  }
  // W = Sigma Y (block-diagonal Sigma), then G = G0 + G0[:, b] W
  zgemm(st, K, ns, nr, ns, one, (const double2*)SL, ns, (long long)ns * ns, 0, dY, nb, bn, zero, dW, nb, bn);
  zgemm(st, K, ns, nr, ns, one, (const double2*)SR, ns, (long long)ns * ns, 0, dY + ns, nb, bn, zero, dW + ns, nb, bn);
  copy_c128<<<grid_for(rtot), 256, 0, st>>>(dG0, dX, rtot);
  zgemm(st, K, nr, nr, nb, one, dG0, nr, r2, 0, dW, nb, bn, one, dX, nr, r2);
  if (fp64) copy_c128<<<grid_for(rtot), 256, 0, st>>>(dX, (double2*)G, rtot);
  else from_c128_f<<<grid_for(rtot), 256, 0, st>>>(dX, (float2*)G, rtot);
  DY_CK(h, cudaGetLastError());
  std::vector<int> hinfo(K);
  DY_CK(h, cudaMemcpyAsync(hinfo.data(), info, K * sizeof(int), cudaMemcpyDeviceToHost, st));
  std::vector<double> hred(2 * K);
  if (refres) DY_CK(h, cudaMemcpyAsync(hred.data(), red, 2 * K * sizeof(double), cudaMemcpyDeviceToHost, st));
  DY_CK(h, cudaStreamSynchronize(st));
  if ((s = handle_end(h)) != RSFD_OK) return s;
  if (refres)
    for (int k = 0; k < K; ++k) refres[k] = sqrt(hred[k]) / sqrt(hred[K + k] > 0 ? hred[K + k] : 1.0);
  for (int k = 0; k < K; ++k)
    if (hinfo[k] != 0)
      return handle_fail(h, RSFD_ERR_BREAKDOWN, "rsfd_dyson_tracked: singular I - G0 Sigma at energy " + std::to_string(k));
  return RSFD_OK;
}

// ------------------------------------------------------------------------------------------------
// Lead self-energies by decimation (Eq. self-energy with the surface Green's function of Eq. surface
// green's function), for leads that repeat one principal layer of R planes with its own potential.
// Principal-layer blocks: H00 (in-plane kinetic + z couplings inside the layer + V), H01 (layer j to
// j+1).  The right lead runs to +z (alpha_0 = H01, beta_0 = H01^T), the left lead to -z (alpha_0 =
// H01^T, beta_0 = H01).  Lopez Sancho-Rubio iteration, batched over energies, all in FP64:
//   g = (Z - eps)^{-1};  eps_s += alpha g beta;  eps += alpha g beta + beta g alpha;
//   alpha = alpha g alpha;  beta = beta g beta;
// until max |alpha|, |beta| fall below 1e-15 max |H01| for every energy; then g_s = (Z - eps_s)^{-1} and
// Sigma_R = H01 g_s H01^T, Sigma_L = H01^T g_s H01.
// ------------------------------------------------------------------------------------------------
__global__ void zi_minus(double2* A, const double2* E, const double2* Z, int n, int batch) {
  const long long n2 = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n2 * batch;
       t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / n2, e = t - b * n2;
    const long long c = e / n, r = e - c * n;
    const double2 v = E[t];
    A[t] = r == c ? make_double2(Z[b].x - v.x, Z[b].y - v.y) : make_double2(-v.x, -v.y);
  }
}
// out[b] = max |re| + |im| over n2 entries of X[b] and of Y[b]
__global__ void maxabs2_batched(const double2* X, const double2* Y, long long n2, double* out) {
  const int b = blockIdx.x;
  double m = 0.0;
  for (long long i = threadIdx.x; i < n2; i += blockDim.x) {
    const double2 x = X[(long long)b * n2 + i], y = Y[(long long)b * n2 + i];
    m = fmax(m, fmax(fabs(x.x) + fabs(x.y), fabs(y.x) + fabs(y.y)));
  }
  __shared__ double red[256];
  red[threadIdx.x] = m;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + k]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[b] = red[0];
}
// dst[b] = src (one n x n matrix broadcast to the batch)
__global__ void bcast_c128(const double2* src, double2* dst, long long n2, int batch) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n2 * batch;
       t += (long long)gridDim.x * blockDim.x)
    dst[t] = src[t % n2];
}
// rhs[b] = [X[b] | Y[b]]  (n x 2n, column-major)
__global__ void concat_cols(const double2* X, const double2* Y, double2* rhs, long long n2, int batch) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 2 * n2 * batch;
       t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / (2 * n2), e = t - b * 2 * n2;
    rhs[t] = e < n2 ? X[b * n2 + e] : Y[b * n2 + e - n2];
  }
}

static void layer_blocks(int nx, int ny, double hh, int fd_order, const double* V, std::vector<double2>& H00,
                         std::vector<double2>& H01) {
  const int R = fd_order / 2, nxy = nx * ny, n = R * nxy;
  const double c2[2] = {-2.0, 1.0}, c4[3] = {-2.5, 4.0 / 3.0, -1.0 / 12.0};
  const double* c = fd_order == 2 ? c2 : c4;
  double d[3] = {0, 0, 0};
  for (int k = 0; k <= R; ++k) d[k] = -0.5 * c[k] / (hh * hh);
  H00.assign((size_t)n * n, make_double2(0, 0));
  H01.assign((size_t)n * n, make_double2(0, 0));
  auto at = [&](std::vector<double2>& M, int r, int col) -> double2& { return M[(size_t)col * n + r]; };
  for (int a = 0; a < R; ++a)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int i = a * nxy + y * nx + x;
        at(H00, i, i).x += 3.0 * d[0] + (V ? V[i] : 0.0);   // x, y, z diagonal parts and the potential
        for (int k = 1; k <= R; ++k) {
          if (x + k < nx) { at(H00, i, i + k).x += d[k]; at(H00, i + k, i).x += d[k]; }
          if (y + k < ny) { at(H00, i, i + k * nx).x += d[k]; at(H00, i + k * nx, i).x += d[k]; }
        }
        for (int cpl = 0; cpl < R; ++cpl) {
          const int j = cpl * nxy + y * nx + x;
          if (cpl != a && std::abs(a - cpl) <= R) at(H00, i, j).x += d[std::abs(a - cpl)];
          const int dist = R + cpl - a;   // plane a of layer j to plane cpl of layer j + 1
          if (dist <= R) at(H01, i, j).x += d[dist];
        }
      }
}

rsfd_status lead_decimation_run(Handle* h, const double* VL, const double* VR, const double* E, int K, double eta,
                                int maxit, void* SLo, void* SRo, int* iters_out) {
  const int nxy = handle_nx(h) * handle_ny(h);
  const int R = handle_fd_order(h) / 2, n = R * nxy;
  const long long n2 = (long long)n * n;
  std::vector<double2> H00L, H00R, H01;
  layer_blocks(handle_nx(h), handle_ny(h), handle_h(h), handle_fd_order(h), VL, H00L, H01);
  layer_blocks(handle_nx(h), handle_ny(h), handle_h(h), handle_fd_order(h), VR, H00R, H01);
  double hmax = 0.0;
  for (const double2& v : H01) hmax = fmax(hmax, fabs(v.x));
  const double tol = 1e-15 * fmax(1.0, hmax);
  std::vector<double2> H01T((size_t)n2);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) H01T[(size_t)c * n + r] = H01[(size_t)r * n + c];
  // per energy: eps_s, eps, alpha, beta, A (LU), Y (n x 2n), rhs (n x 2n), 2 products
  const long long per = n2 * 11 * (long long)sizeof(double2) + (n + 64) * (long long)sizeof(int) + 64;
  size_t free_b = 0, tot_b = 0;
  DY_CK(h, cudaMemGetInfo(&free_b, &tot_b));
  long long kc = (long long)(0.5 * (double)free_b) / per;
  if (kc > K) kc = K;
  if (kc < 1) kc = 1;
  const int Kc = (int)kc;
  rsfd_status s;
  void *pW, *pC, *pPiv, *pZ;
  if ((s = handle_ensure(h, 1, (size_t)n2 * 11 * Kc * sizeof(double2), &pW)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 2, (size_t)n2 * 3 * sizeof(double2), &pC)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 5, ((size_t)Kc * (n + 1) + 64) * sizeof(int), &pPiv)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 6, (size_t)Kc * (sizeof(double2) + sizeof(double)), &pZ)) != RSFD_OK) return s;
  if ((s = handle_begin(h)) != RSFD_OK) return s;
  cudaStream_t st = handle_stream(h);
  double2* W = (double2*)pW;
  double2 *eps_s = W, *eps = W + n2 * Kc, *al = W + 2 * n2 * Kc, *be = W + 3 * n2 * Kc, *A = W + 4 * n2 * Kc;
  double2 *Y = W + 5 * n2 * Kc, *rhs = W + 7 * n2 * Kc, *P1 = W + 9 * n2 * Kc, *P2 = W + 10 * n2 * Kc;
  double2 *dH00 = (double2*)pC, *dH01 = dH00 + n2, *dH01T = dH00 + 2 * n2;
  int* piv = (int*)pPiv;
  int* info = piv + (long long)Kc * n;
  double2* dZ = (double2*)pZ;
  double* dmax = (double*)(dZ + Kc);
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  DY_CK(h, cudaMemcpyAsync(dH01, H01.data(), n2 * sizeof(double2), cudaMemcpyHostToDevice, st));
  DY_CK(h, cudaMemcpyAsync(dH01T, H01T.data(), n2 * sizeof(double2), cudaMemcpyHostToDevice, st));
  int it_max = 0;
  for (int lead = 0; lead < 2; ++lead) {
    const std::vector<double2>& H00 = lead == 0 ? H00R : H00L;
    double2* out = (double2*)(lead == 0 ? SRo : SLo);
    const double2* a0 = lead == 0 ? dH01 : dH01T;
    const double2* b0 = lead == 0 ? dH01T : dH01;
    DY_CK(h, cudaMemcpyAsync(dH00, H00.data(), n2 * sizeof(double2), cudaMemcpyHostToDevice, st));
    for (int k0 = 0; k0 < K; k0 += Kc) {
      const int kb = K - k0 < Kc ? K - k0 : Kc;
      const long long tot = n2 * kb;
      std::vector<double2> Zh(kb);
      for (int k = 0; k < kb; ++k) Zh[k] = make_double2(E[k0 + k], eta);
      DY_CK(h, cudaMemcpyAsync(dZ, Zh.data(), kb * sizeof(double2), cudaMemcpyHostToDevice, st));
      bcast_c128<<<grid_for(tot), 256, 0, st>>>(dH00, eps_s, n2, kb);
      bcast_c128<<<grid_for(tot), 256, 0, st>>>(dH00, eps, n2, kb);
      bcast_c128<<<grid_for(tot), 256, 0, st>>>(a0, al, n2, kb);
      bcast_c128<<<grid_for(tot), 256, 0, st>>>(b0, be, n2, kb);
      int it = 0;
      for (; it < maxit; ++it) {
        maxabs2_batched<<<kb, 256, 0, st>>>(al, be, n2, dmax);
        std::vector<double> hm(kb);
        DY_CK(h, cudaMemcpyAsync(hm.data(), dmax, kb * sizeof(double), cudaMemcpyDeviceToHost, st));
        DY_CK(h, cudaStreamSynchronize(st));
        bool done = true;
        for (int k = 0; k < kb; ++k) done &= hm[k] < tol;
        if (done) break;
        // g [alpha | beta] by LU of Z - eps
        zi_minus<<<grid_for(tot), 256, 0, st>>>(A, eps, dZ, n, kb);
        DY_CK(h, cudaMemsetAsync(info, 0, kb * sizeof(int), st));
        getrf_blocked(st, A, n, kb, piv, info);
        concat_cols<<<grid_for(2 * tot), 256, 0, st>>>(al, be, rhs, n2, kb);
        copy_c128<<<grid_for(2 * tot), 256, 0, st>>>(rhs, Y, 2 * tot);
        {
          dim3 g((2 * n + 127) / 128, kb);
          zgetrs_batched<<<g, 128, 0, st>>>(A, piv, Y, n, 2 * n);
        }
        const double2* ga = Y;        // g alpha, per energy stride 2 n2
        const double2* gb = Y + n2;   // g beta
        // P1 = alpha g beta, P2 = beta g alpha
        zgemm(st, kb, n, n, n, one, al, n, n2, 0, gb, n, 2 * n2, zero, P1, n, n2);
        zgemm(st, kb, n, n, n, one, be, n, n2, 0, ga, n, 2 * n2, zero, P2, n, n2);
        axpy_c128<<<grid_for(tot), 256, 0, st>>>(eps_s, P1, tot);
        axpy_c128<<<grid_for(tot), 256, 0, st>>>(eps, P1, tot);
        axpy_c128<<<grid_for(tot), 256, 0, st>>>(eps, P2, tot);
        // alpha <- alpha g alpha, beta <- beta g beta (through the product buffers)
        zgemm(st, kb, n, n, n, one, al, n, n2, 0, ga, n, 2 * n2, zero, P1, n, n2);
        zgemm(st, kb, n, n, n, one, be, n, n2, 0, gb, n, 2 * n2, zero, P2, n, n2);
        copy_c128<<<grid_for(tot), 256, 0, st>>>(P1, al, tot);
        copy_c128<<<grid_for(tot), 256, 0, st>>>(P2, be, tot);
      }
      it_max = it > it_max ? it : it_max;
      // Sigma = b0 g_s a0 with g_s = (Z - eps_s)^{-1}:  X = g_s a0, Sigma = b0 X
      //   right lead: b0 = H01, a0 = H01^T... the coupling into the lead and back out:
      //   Sigma_R = H01 g_s H01^T, Sigma_L = H01^T g_s H01
      zi_minus<<<grid_for(tot), 256, 0, st>>>(A, eps_s, dZ, n, kb);
      DY_CK(h, cudaMemsetAsync(info, 0, kb * sizeof(int), st));
      getrf_blocked(st, A, n, kb, piv, info);
      bcast_c128<<<grid_for(tot), 256, 0, st>>>(lead == 0 ? dH01T : dH01, Y, n2, kb);
      {
        dim3 g((n + 127) / 128, kb);
        zgetrs_batched<<<g, 128, 0, st>>>(A, piv, Y, n, n);
      }
      zgemm(st, kb, n, n, n, one, lead == 0 ? dH01 : dH01T, n, 0, 0, Y, n, n2, zero, out + n2 * k0, n, n2);
      std::vector<int> hinfo(kb);
      DY_CK(h, cudaMemcpyAsync(hinfo.data(), info, kb * sizeof(int), cudaMemcpyDeviceToHost, st));
      DY_CK(h, cudaStreamSynchronize(st));
      for (int k = 0; k < kb; ++k)
        if (hinfo[k] != 0)
          return handle_fail(h, RSFD_ERR_BREAKDOWN, "rsfd_lead_sigma_decimation: singular Z - eps at energy " +
                                                        std::to_string(k0 + k));
      if (it >= maxit)
        return handle_fail(h, RSFD_ERR_NOT_CONVERGED, "rsfd_lead_sigma_decimation: no convergence in maxit steps");
    }
  }
  DY_CK(h, cudaGetLastError());
  if ((s = handle_end(h)) != RSFD_OK) return s;
  if (iters_out) *iters_out = it_max;
  return RSFD_OK;
}

rsfd_status transmission_run(Handle* h, const void* G, const void* SL, const void* SR, int K, double* T) {
  const int nb = handle_nb(h);
  const int ns = nb / 2;
  const long long n2 = (long long)nb * nb, s2 = (long long)ns * ns;
  const bool fp64 = handle_prec(h) != RSFD_MIXED;   // FP64 and double-float handles hold c128 data
  rsfd_status s;
  void *pG, *pGL, *pGR, *pW1, *pW2, *pT;
  if ((s = handle_ensure(h, 0, n2 * K * sizeof(double2), &pG)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 1, s2 * K * sizeof(double2), &pGL)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 2, s2 * K * sizeof(double2), &pGR)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 3, s2 * K * sizeof(double2), &pW1)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 4, s2 * K * sizeof(double2), &pW2)) != RSFD_OK) return s;
  if ((s = handle_ensure(h, 6, (long long)2 * K * sizeof(double), &pT)) != RSFD_OK) return s;
  if ((s = handle_begin(h)) != RSFD_OK) return s;
  cudaStream_t st = handle_stream(h);
  double2* dG = (double2*)pG;
  const long long tot = n2 * K;
  if (fp64) copy_c128<<<grid_for(tot), 256, 0, st>>>((const double2*)G, dG, tot);
  else to_c128<float2><<<grid_for(tot), 256, 0, st>>>((const float2*)G, dG, tot);
  gamma_batched<<<grid_for(s2 * K), 256, 0, st>>>((const double2*)SL, (double2*)pGL, ns, K);
  gamma_batched<<<grid_for(s2 * K), 256, 0, st>>>((const double2*)SR, (double2*)pGR, ns, K);
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  const double2* GRL = dG + ns;   // rows ns.., cols 0..ns-1, leading dimension nb
  // W1 = Gamma_R G_RL ; W2 = G_RL^H W1
  zgemm(st, K, ns, ns, ns, one, (const double2*)pGR, ns, s2, 0, GRL, nb, n2, zero, (double2*)pW1, ns, s2);
  zgemm(st, K, ns, ns, ns, one, GRL, nb, n2, 1, (const double2*)pW1, ns, s2, zero, (double2*)pW2, ns, s2);
  double* dT = (double*)pT;
  trace_prod_batched<<<K, 256, 0, st>>>((const double2*)pGL, (const double2*)pW2, ns, dT, dT + K);
  DY_CK(h, cudaGetLastError());
  std::vector<double> hT(2 * K);
  DY_CK(h, cudaMemcpyAsync(hT.data(), dT, 2 * K * sizeof(double), cudaMemcpyDeviceToHost, st));
  DY_CK(h, cudaStreamSynchronize(st));
  if ((s = handle_end(h)) != RSFD_OK) return s;
  for (int k = 0; k < K; ++k) T[k] = hT[k];
  return RSFD_OK;
}

}  // namespace rsfd

// ------------------------------------------------------------------------------------------------
// Allocation-free variant of the Dyson step.
//
// Some callers cannot allocate device memory at the point where they need the Dyson step: a
// service or framework that has handed its whole device-memory budget to its own caching allocator
// up front (a cudaMalloc then fails, or would take memory that allocator counts on), or a plug-in
// that a host application forbids to change the device's allocation state.  For them,
// rsfd_dyson_boundary_noalloc keeps its scratch (the matrices I - G0 Sigma and their LU factors,
// the refinement residual, the pivots) in the file-scope device array below, which exists for as
// long as the library is loaded on every GPU that loaded it.  The caller passes the inputs and the
// output; nothing is allocated by the call.
// ------------------------------------------------------------------------------------------------
namespace rsfd {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)RSFD_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// device address of g_noalloc_scratch, looked up once per device (host code must not use the
// symbol itself: on the host it is only a stand-in)
constexpr int kMaxDevices = 64;
static void* g_scratch_ptr[kMaxDevices] = {nullptr};

// first singular energy: *bad starts at K (none) and takes the smallest k with a zero pivot, so the
// message names the same energy as rsfd_dyson_boundary's
__global__ void noalloc_finish(const int* info, const double* red, int K, int* bad, double* ratio) {
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    if (info[k] != 0) atomicMin(bad, k);
    const double g = red[K + k] > 0 ? red[K + k] : 1.0;
    ratio[k] = sqrt(red[k]) / sqrt(g);
  }
}

__global__ void fill_int(int* p, int v) { *p = v; }

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// Body of rsfd_dyson_boundary_noalloc (the C entry point in rsfd_api.cu wraps it in the ABI's
// exception guard).
rsfd_status dyson_noalloc_run(int32_t nb, int32_t K, const void* G0_bb, const void* Sigma_L, const void* Sigma_R,
                              void* G_bb, double* refine_residual, void* stream) {
  if (nb < 2 || (nb % 2) != 0 || K < 1 || !G0_bb || !Sigma_L || !Sigma_R || !G_bb || G0_bb == G_bb)
    return handle_fail(nullptr, RSFD_ERR_ARG, "rsfd_dyson_boundary_noalloc: bad arguments");
  // the batched kernels put the energy on gridDim.y / gridDim.z
  if (K > 65535)
    return handle_fail(nullptr, RSFD_ERR_ARG,
                       "rsfd_dyson_boundary_noalloc: K = " + std::to_string(K) + " exceeds the limit of 65535 energies per call");
  const long long n2 = (long long)nb * nb;
  const size_t need = 3 * align256((size_t)n2 * K * sizeof(double2)) + align256((size_t)K * (nb + 1) * sizeof(int)) +
                      align256((size_t)3 * K * sizeof(double)) + align256(sizeof(int));
  if (need > kNoAllocScratchBytes)
    return handle_fail(nullptr, RSFD_ERR_ARG,
                       "rsfd_dyson_boundary_noalloc: 3*nb*nb*K*16 bytes plus pivots exceed the " +
                           std::to_string(kNoAllocScratchBytes) + "-byte static scratch (nb=" + std::to_string(nb) +
                           ", K=" + std::to_string(K) + ")");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return handle_fail(nullptr, RSFD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return handle_fail(nullptr, RSFD_ERR_ARG, "rsfd_dyson_boundary_noalloc: device index too large");
  if (!g_scratch_ptr[dev]) {   // one-time set-up on this device (the current device)
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return handle_fail(nullptr, RSFD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  unsigned char* base = (unsigned char*)g_scratch_ptr[dev];
  double2* dM = (double2*)base;
  base += align256((size_t)n2 * K * sizeof(double2));
  double2* dLU = (double2*)base;
  base += align256((size_t)n2 * K * sizeof(double2));
  double2* dR = (double2*)base;
  base += align256((size_t)n2 * K * sizeof(double2));
  int* piv = (int*)base;
  int* info = piv + (size_t)K * nb;
  base += align256((size_t)K * (nb + 1) * sizeof(int));
  double* red = (double*)base;   // [2K] squared norms, [K] ratios
  base += align256((size_t)3 * K * sizeof(double));
  int* bad = (int*)base;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const double2* G0 = (const double2*)G0_bb;
  double2* dX = (double2*)G_bb;
  const long long tot = n2 * K;
  const double2 m1 = make_double2(-1.0, 0.0), one = make_double2(1.0, 0.0);
  // the scratch keeps the previous call's contents: clear the flags that must start at zero
  e = cudaMemsetAsync(info, 0, K * sizeof(int), st);
  if (e != cudaSuccess) return handle_fail(nullptr, RSFD_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  fill_int<<<1, 1, 0, st>>>(bad, K);
  set_identity<<<grid_for(tot), 256, 0, st>>>(dM, nb, K);
  const int ns = nb / 2;
  zgemm(st, K, nb, ns, ns, m1, G0, nb, n2, 0, (const double2*)Sigma_L, ns, (long long)ns * ns, one, dM, nb, n2);
  zgemm(st, K, nb, ns, ns, m1, G0 + (long long)ns * nb, nb, n2, 0, (const double2*)Sigma_R, ns, (long long)ns * ns, one,
        dM + (long long)ns * nb, nb, n2);
  copy_c128<<<grid_for(tot), 256, 0, st>>>(dM, dLU, tot);
  getrf_blocked(st, dLU, nb, K, piv, info);
  copy_c128<<<grid_for(tot), 256, 0, st>>>(G0, dX, tot);
  dim3 g((nb + 127) / 128, K);
  zgetrs_batched<<<g, 128, 0, st>>>(dLU, piv, dX, nb, nb);
  for (int it = 0; it < 2; ++it) {
    copy_c128<<<grid_for(tot), 256, 0, st>>>(G0, dR, tot);
    zgemm(st, K, nb, nb, nb, m1, dM, nb, n2, 0, dX, nb, n2, one, dR, nb, n2);
    zgetrs_batched<<<g, 128, 0, st>>>(dLU, piv, dR, nb, nb);
    axpy_c128<<<grid_for(tot), 256, 0, st>>>(dX, dR, tot);
  }
  copy_c128<<<grid_for(tot), 256, 0, st>>>(G0, dR, tot);
  zgemm(st, K, nb, nb, nb, m1, dM, nb, n2, 0, dX, nb, n2, one, dR, nb, n2);
  frob2_batched<<<K, 256, 0, st>>>(dR, n2, red);
  frob2_batched<<<K, 256, 0, st>>>(G0, n2, red + K);
  noalloc_finish<<<1, 256, 0, st>>>(info, red, K, bad, red + 2 * K);
  e = cudaGetLastError();
  int hbad = K;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && refine_residual)
    e = cudaMemcpyAsync(refine_residual, red + 2 * K, K * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return handle_fail(nullptr, RSFD_ERR_CUDA, std::string("rsfd_dyson_boundary_noalloc: ") + cudaGetErrorString(e));
  if (hbad < K)
    return handle_fail(nullptr, RSFD_ERR_BREAKDOWN,
                       "rsfd_dyson_boundary_noalloc: singular I - G0 Sigma at energy " + std::to_string(hbad));
  return RSFD_OK;
}

}  // namespace rsfd
