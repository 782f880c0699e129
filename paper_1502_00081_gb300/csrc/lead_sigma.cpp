// Self-energies of uniform V=0 finite-difference leads, computed on the host in FP64.
//
// The paper defines Sigma_L = B^dag g_L B and Sigma_R = B g_R B^dag from the surface Green's
// functions of the semi-infinite electrodes (Eqs. self-energy, surface green's function,
// sec2-01, sec2-02) but leaves their computation to the OBM method.  For a lead that continues
// the transition region's grid with V = 0, the same Dirichlet walls and the same stencil, every
// transverse mode m (eigenpair of the in-plane operator) decouples into a 1D chain along z:
//
//   2nd order:  t1 lambda^2 + (d0 + eps_m - Z) lambda + t1 = 0,         Sigma_m = t1 lambda
//   4th order:  t2 l^4 + t1 l^3 + (d0 + eps_m - Z) l^2 + t1 l + t2 = 0,   Sigma_m = H01 Phi diag(l^2) Phi^-1
//
// with the outgoing (|lambda| < 1) roots, H01 the coupling of the last two planes of the region
// to the first two planes of the lead and Phi = [[1, 1], [l1, l2]].  The palindromic quartic is
// solved in closed form through mu = l + 1/l, which turns it into the quadratic
// t2 mu^2 + t1 mu + (d0 + eps - Z - 2 t2) = 0 followed by l^2 - mu l + 1 = 0.
// The modes of the in-plane operator come from a cyclic Jacobi eigensolver of each 1D axis
// operator (the 2D modes are their tensor products).

#include <math.h>

#include <algorithm>
#include <complex>
#include <string>
#include <thread>
#include <vector>

#include "rsfd_internal.cuh"

namespace rsfd {
namespace {

typedef std::complex<double> zc;

// -1/2 d^2/dx^2 on n points with zero ghosts, dense row-major
std::vector<double> kinetic_1d(int n, double h, int fd_order) {
  std::vector<double> A((size_t)n * n, 0.0);
  const double ih2 = 1.0 / (h * h);
  const double c0 = fd_order == 2 ? -2.0 : -2.5;
  const double c1 = fd_order == 2 ? 1.0 : 4.0 / 3.0;
  const double c2 = fd_order == 2 ? 0.0 : -1.0 / 12.0;
  for (int i = 0; i < n; ++i) {
    A[(size_t)i * n + i] = -0.5 * c0 * ih2;
    if (i + 1 < n) A[(size_t)i * n + i + 1] = A[(size_t)(i + 1) * n + i] = -0.5 * c1 * ih2;
    if (i + 2 < n && c2 != 0.0) A[(size_t)i * n + i + 2] = A[(size_t)(i + 2) * n + i] = -0.5 * c2 * ih2;
  }
  return A;
}

// Cyclic Jacobi: A (n x n symmetric, row-major) -> eigenvalues w, eigenvectors as columns of V.
void jacobi_eigh(std::vector<double> A, int n, std::vector<double>& w, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double a = A[(size_t)i * n + j];
        tot += a * a;
        if (i != j) off += a * a;
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {   // rotate columns p, q
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {   // rotate rows p, q
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

zc small_root(zc a, zc b, zc c) {
  // roots of a x^2 + b x + c with product c/a; return the one of smaller modulus
  const zc s = std::sqrt(b * b - 4.0 * a * c);
  const zc q = (std::real(std::conj(b) * s) >= 0.0) ? -0.5 * (b + s) : -0.5 * (b - s);
  const zc x1 = q / a, x2 = c / q;
  return std::abs(x1) < std::abs(x2) ? x1 : x2;
}

}  // namespace

rsfd_status lead_sigma_uniform(int nx, int ny, double h, int fd_order, const double* E, double eta, int K,
                               double* SLout, double* SRout, std::string* err) {
  const int R = fd_order / 2;
  const int nxy = nx * ny;
  const long long ns = (long long)R * nxy;
  const double ih2 = 1.0 / (h * h);
  const double d0 = fd_order == 2 ? ih2 : 1.25 * ih2;                  // z part of H's diagonal
  const double t1 = fd_order == 2 ? -0.5 * ih2 : -2.0 / 3.0 * ih2;     // coupling to planes +-1
  const double t2 = fd_order == 2 ? 0.0 : 1.0 / 24.0 * ih2;            // coupling to planes +-2
  std::vector<double> wx, wy, Ux, Uy;
  jacobi_eigh(kinetic_1d(nx, h, fd_order), nx, wx, Ux);
  jacobi_eigh(kinetic_1d(ny, h, fd_order), ny, wy, Uy);
  // energies are independent: host threads take interleaved energies, each with its own scratch
  const int nthr = std::max(1, std::min<int>(K, (int)std::min(64u, std::max(1u, std::thread::hardware_concurrency()))));
  auto work = [&](int t0) {
  std::vector<zc> sig((size_t)nxy * R * R);      // per mode (j*nx + i), R x R block (a, c)
  std::vector<zc> T1((size_t)ny * nx * nx);       // [j][x][x']
  std::vector<zc> blk((size_t)nxy * nxy);
  for (int k = t0; k < K; k += nthr) {
    const zc Z(E[k], eta);
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const double eps = wy[j] + wx[i];
        zc* s = &sig[((size_t)j * nx + i) * R * R];
        if (R == 1) {
          const zc lam = small_root(zc(t1), zc(d0 + eps) - Z, zc(t1));
          s[0] = t1 * lam;
        } else {
          // t2 mu^2 + t1 mu + (d0 + eps - Z - 2 t2) = 0
          const zc a(t2), b(t1), c = zc(d0 + eps - 2.0 * t2) - Z;
          const zc sq = std::sqrt(b * b - 4.0 * a * c);
          const zc mu1 = (-b + sq) / (2.0 * a), mu2 = (-b - sq) / (2.0 * a);
          const zc l1 = small_root(zc(1.0), -mu1, zc(1.0));
          const zc l2 = small_root(zc(1.0), -mu2, zc(1.0));
          // M = Phi diag(l^2) Phi^-1 with Phi = [[1,1],[l1,l2]]
          const zc det = l2 - l1;
          const zc M00 = (l1 * l1 * l2 - l2 * l2 * l1) / det;
          const zc M01 = (l2 * l2 - l1 * l1) / det;
          const zc M10 = (l1 * l1 * l1 * l2 - l2 * l2 * l2 * l1) / det;
          const zc M11 = (l2 * l2 * l2 - l1 * l1 * l1) / det;
          // H01 = [[t2, 0], [t1, t2]]
          s[0] = t2 * M00;
          s[1] = t2 * M01;
          s[2] = t1 * M00 + t2 * M10;
          s[3] = t1 * M01 + t2 * M11;
        }
      }
    for (int a = 0; a < R; ++a)
      for (int c = 0; c < R; ++c) {
        // T1[j][x][x'] = sum_i Ux[x,i] sig_ij[a,c] Ux[x',i]
        for (int j = 0; j < ny; ++j)
          for (int x = 0; x < nx; ++x)
            for (int xp = 0; xp < nx; ++xp) {
              zc acc(0.0);
              for (int i = 0; i < nx; ++i)
                acc += Ux[(size_t)x * nx + i] * sig[((size_t)j * nx + i) * R * R + a * R + c] * Ux[(size_t)xp * nx + i];
              T1[((size_t)j * nx + x) * nx + xp] = acc;
            }
        // blk[(y,x),(y',x')] = sum_j Uy[y,j] Uy[y',j] T1[j][x][x']
        for (int y = 0; y < ny; ++y)
          for (int yp = 0; yp < ny; ++yp)
            for (int x = 0; x < nx; ++x)
              for (int xp = 0; xp < nx; ++xp) {
                zc acc(0.0);
                for (int j = 0; j < ny; ++j)
                  acc += Uy[(size_t)y * ny + j] * Uy[(size_t)yp * ny + j] * T1[((size_t)j * nx + x) * nx + xp];
                blk[((size_t)y * nx + x) * nxy + (size_t)yp * nx + xp] = acc;
              }
        // write Sigma_R block (a, c) and its mirror into Sigma_L block (R-1-a, R-1-c); column-major
        const int aL = R - 1 - a, cL = R - 1 - c;
        for (long long r = 0; r < nxy; ++r)
          for (long long q = 0; q < nxy; ++q) {
            const zc v = blk[(size_t)r * nxy + q];
            const long long rowR = a * nxy + r, colR = c * nxy + q;
            const long long rowL = aL * nxy + r, colL = cL * nxy + q;
            double* pr = SRout + 2 * ((size_t)k * ns * ns + (size_t)colR * ns + rowR);
            double* pl = SLout + 2 * ((size_t)k * ns * ns + (size_t)colL * ns + rowL);
            pr[0] = v.real();
            pr[1] = v.imag();
            pl[0] = v.real();
            pl[1] = v.imag();
          }
      }
  }
  };
  if (nthr == 1) {
    work(0);
  } else {
    std::vector<std::thread> pool;
    for (int t = 0; t < nthr; ++t) pool.emplace_back(work, t);
    for (auto& th : pool) th.join();
  }
  (void)err;
  return RSFD_OK;
}

}  // namespace rsfd
