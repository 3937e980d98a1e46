// Adaptive CTD (Section 3.3, "Adaptivity"): the full-grid C-FEM step that replaces a time step
// whose greedy loop would need more than M_c modes, solved by fast diagonalisation, and the
// full-grid field it leaves.  Host-side orchestration of the kernels in ctd_actd.cu.
#pragma once
#include <cstddef>

#include "ctd_kernels.h"

namespace ctd {

struct ActdState {
  void* blas = nullptr;      // cublasHandle_t
  void* dense = nullptr;     // cusolverDnHandle_t
  double* V[kMaxDim] = {};   // [n][n] column-major: generalised eigenvectors, V^T M V = I
  double* lam[kMaxDim] = {}; // [n] eigenvalues, ascending
  double* Y = nullptr;       // [N] full-grid scratch
  double* work = nullptr;    // eigensolver scratch
  size_t work_len = 0;       // doubles
  int* info = nullptr;       // eigensolver status
};

// Doubles of eigensolver scratch reserved for dimensions of up to n nodes.
size_t actd_work_doubles(int n);

// Create the library handles on `stream` and compute every dimension's eigenpairs
// (K_d V = diag(omega_d) V Lambda).  Returns 0, or a negative code with a message in *msg.
int actd_setup(ActdState& a, const StepParams& P, const double* const* kband_host, const double* const* omega_host,
               cudaStream_t stream, const char** msg);
void actd_release(ActdState& a);

// The full-grid step from the current u^k (factors in bank `bank` with Mk modes, or the grid
// array P.U when from_grid): u^{k+1} on the full grid, written to P.U.
int actd_cfe_step(ActdState& a, const StepParams& P, int from_grid, int bank, int Mk, cudaStream_t stream,
                  const char** msg);

// Full-grid nodal values of the factors of bank `bank` (Mk modes) into out (device, N doubles).
cudaError_t launch_field_from_modes(const StepParams& P, int bank, int Mk, double* out, cudaStream_t s);
// Energy parts of a full-grid field: part[g] per CTA, bulk and gradient terms summed.
cudaError_t launch_energy_grid(const StepParams& P, const double* U, double* part, int grid, cudaStream_t s);

}  // namespace ctd
