// Host-side 1D C-FEM builder: the stiffness band and nodal weights of one dimension.
//
// Shape functions (Section 3.2 Eq. CFEM, App. C Eq. CFEM-1D): on element e = [x_e, x_e+1]
// with natural coordinate xi in [-1, 1], N~_k(xi) = sum_{i in {e, e+1}} N_i(xi) W_{i,k}(xi),
// N_e = (1 - xi)/2, N_e+1 = (1 + xi)/2, and W_i the radial basis patch interpolant of node i
// (App. B): W(xi) = Psi_a(xi) K + p(xi) L, L = (P^T R0^-1 P)^-1 P^T R0^-1,
// K = R0^-1 (I - P L), R0_jl = Psi_a(|xi_j - xi_l| / a), P_jq = xi_j^q.
// Node j of the mesh sits at xi_j = -1 + 2 (j - e) in the element's coordinate; node i's
// patch is {max(0, i-s) .. min(n-1, i+s)} (truncated at the ends of the domain).
//
// Stiffness K_dd = int B~^T B~ dx (Eq. KxxMxx) per element with 5-point Gauss-Legendre,
// dx = (h/2) dxi, d/dx = (2/h) d/dxi.  Exact when every break point of the kernel lies on
// an element end (true for a = 12 with s <= 3).  Nodal weights: trapezoid rule.
//
// Gauss-point rule (build_cfem_gauss_1d): q points per element, the shape function values
// there and the mass Phi^T diag(omega) Phi, which is the exact consistent mass of Eq. KxxMxx
// for q >= 5 (N~ is a polynomial of degree <= 4 on each element under the same condition).
#include <cmath>
#include <cstring>
#include <vector>

#include "cfem_host.h"

namespace ctd {
namespace {

double kernel(double z) {
  z = std::fabs(z);
  if (z <= 0.5) return 2.0 / 3.0 - 4.0 * z * z + 4.0 * z * z * z;
  if (z <= 1.0) return 4.0 / 3.0 - 4.0 * z + 4.0 * z * z - (4.0 / 3.0) * z * z * z;
  return 0.0;
}

double kernel_dz(double z) {
  z = std::fabs(z);
  if (z <= 0.5) return -8.0 * z + 12.0 * z * z;
  if (z <= 1.0) return -4.0 + 8.0 * z - 4.0 * z * z;
  return 0.0;
}

// In-place inverse of a small dense matrix (Gauss-Jordan, partial pivoting).
bool invert(std::vector<double>& A, int n) {
  std::vector<double> I(n * n, 0.0);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return false;
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(A[c * n + k], A[piv * n + k]);
        std::swap(I[c * n + k], I[piv * n + k]);
      }
    const double d = 1.0 / A[c * n + c];
    for (int k = 0; k < n; ++k) { A[c * n + k] *= d; I[c * n + k] *= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) { A[r * n + k] -= f * A[c * n + k]; I[r * n + k] -= f * I[c * n + k]; }
    }
  }
  A = I;
  return true;
}

std::vector<double> matmul(const std::vector<double>& A, const std::vector<double>& B,
                           int m, int k, int n) {
  std::vector<double> C(m * n, 0.0);
  for (int i = 0; i < m; ++i)
    for (int l = 0; l < k; ++l) {
      const double a = A[i * k + l];
      for (int j = 0; j < n; ++j) C[i * n + j] += a * B[l * n + j];
    }
  return C;
}

// Patch interpolant of App. B for patch nodes at natural coordinates xs (np nodes):
// outputs Kc (np x np) and Lc ((p+1) x np), row-major.
bool patch_coefficients(const std::vector<double>& xs, double a, int p,
                        std::vector<double>& Kc, std::vector<double>& Lc) {
  const int np = static_cast<int>(xs.size()), nq = p + 1;
  std::vector<double> R(np * np), P(np * nq), Pt(nq * np);
  for (int j = 0; j < np; ++j)
    for (int l = 0; l < np; ++l) R[j * np + l] = kernel(std::fabs(xs[j] - xs[l]) / a);
  for (int j = 0; j < np; ++j) {
    double v = 1.0;
    for (int q = 0; q < nq; ++q) { P[j * nq + q] = v; Pt[q * np + j] = v; v *= xs[j]; }
  }
  if (!invert(R, np)) return false;                          // R <- R0^-1
  std::vector<double> PtR = matmul(Pt, R, nq, np, np);       // P^T R0^-1
  std::vector<double> S = matmul(PtR, P, nq, np, nq);        // P^T R0^-1 P
  if (!invert(S, nq)) return false;
  Lc = matmul(S, PtR, nq, nq, np);                           // L
  std::vector<double> PL = matmul(P, Lc, np, nq, np);
  for (int j = 0; j < np; ++j)
    for (int l = 0; l < np; ++l) PL[j * np + l] = (j == l ? 1.0 : 0.0) - PL[j * np + l];
  Kc = matmul(R, PL, np, np, np);                            // R0^-1 (I - P L)
  return true;
}

// q-point Gauss-Legendre rule on [-1, 1], ascending: the roots of the Legendre polynomial
// P_q by Newton's method (P_q and P_q-1 from the three-term recurrence
// (k + 1) P_k+1 = (2k + 1) x P_k - k P_k-1, P_q' = q (x P_q - P_q-1) / (x^2 - 1)), started
// from the asymptotic guess cos(pi (i + 3/4) / (q + 1/2)); weights 2 / ((1 - x^2) P_q'(x)^2).
bool gauss_legendre(int q, double* xs, double* ws) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < (q + 1) / 2; ++i) {
    double x = std::cos(pi * (i + 0.75) / (q + 0.5)), dp = 1.0;   // p0, p1 end as P_q-1, P_q
    bool done = false;
    for (int it = 0; it < 100 && !done; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 1; k < q; ++k) {
        const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = q * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      done = std::fabs(dx) <= 4e-16;
    }
    if (!done) return false;
    // recompute the derivative at the converged root for the weight
    double p0 = 1.0, p1 = x;
    for (int k = 1; k < q; ++k) {
      const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
      p0 = p1;
      p1 = p2;
    }
    dp = q * (x * p1 - p0) / (x * x - 1.0);
    const double w = 2.0 / ((1.0 - x * x) * dp * dp);
    xs[q - 1 - i] = x;        // largest root first from the guess: fill from the top
    ws[q - 1 - i] = w;
    xs[i] = -x;
    ws[i] = w;
  }
  if (q % 2 == 1) xs[q / 2] = 0.0;
  return true;
}

// Values N~_k(xi) at natural points xi[0..nx) of element e for every supporting node
// k = s0 .. s1 (s0 = max(0, e - s), s1 = min(n - 1, e + 1 + s)): N[g * ns + k - s0].
bool element_values(int e, int n, int s, int p, double a, const double* xi, int nx, std::vector<double>& N) {
  const int s0 = std::max(0, e - s), s1 = std::min(n - 1, e + 1 + s), ns = s1 - s0 + 1;
  N.assign(static_cast<size_t>(nx) * ns, 0.0);
  for (int end = 0; end < 2; ++end) {
    const int i = e + end;
    const int p0 = std::max(0, i - s), p1 = std::min(n - 1, i + s), np = p1 - p0 + 1;
    std::vector<double> xs(np);
    for (int j = 0; j < np; ++j) xs[j] = -1.0 + 2.0 * (p0 + j - e);
    std::vector<double> Kc, Lc;
    if (!patch_coefficients(xs, a, p, Kc, Lc)) return false;
    for (int g = 0; g < nx; ++g) {
      const double Ni = end == 0 ? 0.5 * (1.0 - xi[g]) : 0.5 * (1.0 + xi[g]);
      for (int j = 0; j < np; ++j) {
        double W = 0.0;
        for (int l = 0; l < np; ++l) W += kernel(std::fabs(xi[g] - xs[l]) / a) * Kc[l * np + j];
        double pv = 1.0;
        for (int qq = 0; qq <= p; ++qq) {
          W += pv * Lc[qq * np + j];
          pv *= xi[g];
        }
        N[static_cast<size_t>(g) * ns + (p0 + j - s0)] += Ni * W;
      }
    }
  }
  return true;
}

// True if the symmetric band A (n x (2b+1), entry (i, j-i+b) = A[i][j]) is positive definite:
// banded Cholesky without pivoting succeeds with positive pivots (Sylvester's criterion).  A
// pivot must exceed 1e-12 of its diagonal entry, so that a matrix singular up to rounding
// fails; in the bisections below this only widens the bounds.
bool band_is_spd(const std::vector<double>& A, int n, int b) {
  const int w = 2 * b + 1;
  std::vector<double> L(static_cast<size_t>(n) * (b + 1), 0.0);   // L[i][k] = L(i, i - b + k)
  for (int i = 0; i < n; ++i) {
    for (int j = std::max(0, i - b); j <= i; ++j) {
      double acc = A[static_cast<size_t>(i) * w + (j - i + b)];
      for (int k = std::max(0, i - b); k < j; ++k)
        acc -= L[static_cast<size_t>(i) * (b + 1) + (k - i + b)] * L[static_cast<size_t>(j) * (b + 1) + (k - j + b)];
      if (j == i) {
        if (!(acc > 1e-12 * std::fabs(A[static_cast<size_t>(i) * w + b]))) return false;
        L[static_cast<size_t>(i) * (b + 1) + b] = std::sqrt(acc);
      } else {
        L[static_cast<size_t>(i) * (b + 1) + (j - i + b)] = acc / L[static_cast<size_t>(j) * (b + 1) + b];
      }
    }
  }
  return true;
}

// Bounds [lo, hi] of the spectrum of diag(M)^-1 M for the SPD band M: lo is the largest c found
// by bisection with M - c diag(M) positive definite, hi the smallest with c diag(M) - M
// positive definite (both tested by banded Cholesky), each moved outward by a relative 1e-6.
void mass_spectrum_bounds(const std::vector<double>& M, int n, int b, double* lo, double* hi) {
  const int w = 2 * b + 1;
  double gersh = 0.0;            // Gershgorin: every eigenvalue is below max_i sum_j |M_ij| / M_ii
  for (int i = 0; i < n; ++i) {
    double r = 0.0;
    for (int k = 0; k < w; ++k) r += std::fabs(M[static_cast<size_t>(i) * w + k]);
    gersh = std::max(gersh, r / M[static_cast<size_t>(i) * w + b]);
  }
  std::vector<double> T(M.size());
  auto shifted = [&](double c, double sign) {   // sign (M - c diag(M)), diagonal shift only
    for (size_t e = 0; e < M.size(); ++e) T[e] = sign * M[e];
    for (int i = 0; i < n; ++i) T[static_cast<size_t>(i) * w + b] -= sign * c * M[static_cast<size_t>(i) * w + b];
    return band_is_spd(T, n, b);
  };
  double a0 = 0.0, a1 = 1.0;     // M - 0 D is SPD; M - 1 D is not (its diagonal is zero)
  for (int it = 0; it < 60; ++it) {
    const double c = 0.5 * (a0 + a1);
    (shifted(c, 1.0) ? a0 : a1) = c;
  }
  double b0 = 1.0, b1 = gersh * (1.0 + 1e-12) + 1e-12;   // c D - M: not SPD at 1, SPD above Gershgorin
  for (int it = 0; it < 60; ++it) {
    const double c = 0.5 * (b0 + b1);
    (shifted(c, -1.0) ? b1 : b0) = c;
  }
  *lo = a0 * (1.0 - 1e-6);
  *hi = b1 * (1.0 + 1e-6);
}

}  // namespace

int build_cfem_gauss_1d(int n, double length, int s, int p, double a, int q, double* x_q, double* omega_q,
                        double* phi, int* phi_col0, double* mband, double* mass_bounds) {
  if (n < 2 || s < 1 || p < 0 || p > s || !(a > 0.0) || !(length > 0.0) || q < 1 || q > kMaxGaussPoints)
    return -1;
  double gx[kMaxGaussPoints], gw[kMaxGaussPoints];
  if (!gauss_legendre(q, gx, gw)) return -2;
  const int b = 2 * s + 1, w = 2 * b + 1, wphi = 2 * s + 2;
  const double h = length / (n - 1);
  if (mband) std::memset(mband, 0, sizeof(double) * static_cast<size_t>(n) * w);
  std::vector<double> N, Mown;
  if (!mband && mass_bounds) {   // the bounds need the band: assemble into a private copy
    Mown.assign(static_cast<size_t>(n) * w, 0.0);
    mband = Mown.data();
  }
  for (int e = 0; e < n - 1; ++e) {
    const int s0 = std::max(0, e - s), s1 = std::min(n - 1, e + 1 + s), ns = s1 - s0 + 1;
    if (!element_values(e, n, s, p, a, gx, q, N)) return -2;
    for (int g = 0; g < q; ++g) {
      const size_t r = static_cast<size_t>(e) * q + g;
      const double om = gw[g] * (0.5 * h);
      if (x_q) x_q[r] = e * h + (1.0 + gx[g]) * (0.5 * h);
      if (omega_q) omega_q[r] = om;
      if (phi_col0) phi_col0[r] = s0;
      if (phi)
        for (int k = 0; k < wphi; ++k) phi[r * wphi + k] = k < ns ? N[static_cast<size_t>(g) * ns + k] : 0.0;
      if (mband)
        for (int k = 0; k < ns; ++k)
          for (int l = 0; l < ns; ++l) {
            const int row = s0 + k, col = s0 + l;
            mband[static_cast<size_t>(row) * w + (col - row + b)] +=
                om * N[static_cast<size_t>(g) * ns + k] * N[static_cast<size_t>(g) * ns + l];
          }
    }
  }
  if (mass_bounds) {
    const std::vector<double> M(mband, mband + static_cast<size_t>(n) * w);
    for (int i = 0; i < n; ++i)
      if (!(M[static_cast<size_t>(i) * w + b] > 0.0)) return -2;
    if (!band_is_spd(M, n, b)) return -2;
    mass_spectrum_bounds(M, n, b, &mass_bounds[0], &mass_bounds[1]);
  }
  return 0;
}

int build_cfem_1d(int n, double length, int s, int p, double a, double* omega, double* kband) {
  if (n < 2 || s < 1 || p < 0 || p > s || !(a > 0.0) || !(length > 0.0)) return -1;
  const int b = 2 * s + 1, w = 2 * b + 1;
  const double h = length / (n - 1);
  if (omega) {
    for (int i = 0; i < n; ++i) omega[i] = h;
    omega[0] = omega[n - 1] = 0.5 * h;
  }
  if (!kband) return 0;
  std::memset(kband, 0, sizeof(double) * static_cast<size_t>(n) * w);
  static const double gx[5] = {-0.9061798459386640, -0.5384693101056831, 0.0,
                               0.5384693101056831, 0.9061798459386640};
  static const double gw[5] = {0.2369268850561891, 0.4786286704993665, 0.5688888888888889,
                               0.4786286704993665, 0.2369268850561891};
  for (int e = 0; e < n - 1; ++e) {
    const int s0 = std::max(0, e - s), s1 = std::min(n - 1, e + 1 + s);
    const int ns = s1 - s0 + 1;
    // dN~/dxi at the Gauss points for every supporting node: dN[g][k]
    std::vector<double> dN(5 * ns, 0.0);
    for (int end = 0; end < 2; ++end) {
      const int i = e + end;
      const int p0 = std::max(0, i - s), p1 = std::min(n - 1, i + s), np = p1 - p0 + 1;
      std::vector<double> xs(np);
      for (int j = 0; j < np; ++j) xs[j] = -1.0 + 2.0 * (p0 + j - e);
      std::vector<double> Kc, Lc;
      if (!patch_coefficients(xs, a, p, Kc, Lc)) return -2;
      for (int g = 0; g < 5; ++g) {
        const double xi = gx[g];
        const double Ni = end == 0 ? 0.5 * (1.0 - xi) : 0.5 * (1.0 + xi);
        const double dNi = end == 0 ? -0.5 : 0.5;
        // W(xi) and dW/dxi over the patch nodes
        std::vector<double> psi(np), dpsi(np);
        for (int l = 0; l < np; ++l) {
          const double d = xi - xs[l];
          psi[l] = kernel(std::fabs(d) / a);
          dpsi[l] = kernel_dz(std::fabs(d) / a) * (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / a;
        }
        for (int j = 0; j < np; ++j) {
          double W = 0.0, dW = 0.0;
          for (int l = 0; l < np; ++l) { W += psi[l] * Kc[l * np + j]; dW += dpsi[l] * Kc[l * np + j]; }
          double pv = 1.0, dpv = 0.0;
          for (int q = 0; q <= p; ++q) {
            W += pv * Lc[q * np + j];
            dW += dpv * Lc[q * np + j];
            dpv = (q + 1) * pv;   // d/dxi xi^(q+1) = (q+1) xi^q
            pv *= xi;
          }
          dN[g * ns + (p0 + j - s0)] += dNi * W + Ni * dW;
        }
      }
    }
    for (int k = 0; k < ns; ++k)
      for (int l = 0; l < ns; ++l) {
        double acc = 0.0;
        for (int g = 0; g < 5; ++g) acc += gw[g] * dN[g * ns + k] * dN[g * ns + l];
        const int row = s0 + k, col = s0 + l;
        kband[static_cast<size_t>(row) * w + (col - row + b)] += (2.0 / h) * acc;
      }
  }
  return 0;
}

}  // namespace ctd
