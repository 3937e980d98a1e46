#pragma once
#include <algorithm>

namespace ctd {
// Nodal weights omega[n] and stiffness band kband[n][2b+1] (b = 2s+1; entry (i, j-i+b) is
// K[i][j]) of the 1D C-FEM on [0, length] with n nodes.  Either output may be null.
// Returns 0, or < 0 for invalid parameters / a singular patch system.
int build_cfem_1d(int n, double length, int s, int p, double a, double* omega, double* kband);
}  // namespace ctd
