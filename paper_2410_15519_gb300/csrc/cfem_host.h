#pragma once
#include <algorithm>

namespace ctd {
// Nodal weights omega[n] and stiffness band kband[n][2b+1] (b = 2s+1; entry (i, j-i+b) is
// K[i][j]) of the 1D C-FEM on [0, length] with n nodes.  Either output may be null.
// Returns 0, or < 0 for invalid parameters / a singular patch system.
int build_cfem_1d(int n, double length, int s, int p, double a, double* omega, double* kband);

// Gauss-point rule with q points per element (1 <= q <= kMaxGaussPoints), n_q = q (n - 1)
// points ordered element by element: points x_q[n_q], weights omega_q[n_q], shape function
// values phi[n_q][2s + 2] (phi[r][k] = N~_{phi_col0[r] + k}(x_r), zero past the element's
// support) with phi_col0[n_q], and the mass band mband[n][2b+1] of Phi^T diag(omega) Phi in
// the layout of kband, and mass_bounds[2]: bounds lo <= lambda <= hi of the spectrum of
// diag(M)^-1 M (for a Chebyshev solve preconditioned by diag(M)).  Any output may be null.
// Returns 0, or < 0 as build_cfem_1d (also when the mass is not positive definite).
constexpr int kMaxGaussPoints = 16;
int build_cfem_gauss_1d(int n, double length, int s, int p, double a, int q, double* x_q, double* omega_q,
                        double* phi, int* phi_col0, double* mband, double* mass_bounds);
}  // namespace ctd
