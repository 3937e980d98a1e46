// Adaptive CTD (Section 3.3, "Adaptivity"): the full-grid C-FEM step of Eq.
// AC-discrete-semi-stable-K on the tensor-product space, solved by fast diagonalisation.
//
// With the generalised eigenpairs K_d V_d = M_d V_d Lambda_d, V_d^T M_d V_d = I of every
// dimension (M_d = diag(omega_d) under the nodal rule), the full-grid operator
// c_t (x)M_d + c_k sum_d M .. K_d .. M is diagonal in the basis (x)V_d with entries
// c_t + c_k sum_d lambda_d,i_d.  The step is therefore
//   Q = (x)omega_d (c_t u^k - L w(u^k))       (right-hand side at the nodes),
//   Y = (x)V_d^T Q,  Y /= c_t + c_k sum_d lambda,  u^{k+1} = (x)V_d Y,
// each (x)V application one FP64 GEMM per axis (cuBLAS).  The eigenpairs come from the
// symmetric eigenproblem of diag(omega)^-1/2 K diag(omega)^-1/2 (cuSOLVER), once at create.
#include <algorithm>
#include <cmath>
#include <vector>

#include <cublas_v2.h>
#include <cusolverDn.h>

#include "ctd_actd.h"

namespace ctd {

namespace {

__device__ __forceinline__ void grid_index(long long p, int n1, int n2, int& i, int& j, int& l) {
  l = static_cast<int>(p % n2);
  const long long ij = p / n2;
  j = static_cast<int>(ij % n1);
  i = static_cast<int>(ij / n1);
}

__device__ __forceinline__ double field_value(const StepParams& P, int bank, int Mk, int i, int j, int l) {
  double u = 0.0;
  for (int m = 0; m < Mk; ++m) {
    double t = f2_to_double(P.d[0].bank[bank][static_cast<size_t>(m) * P.d[0].n + i]) *
               f2_to_double(P.d[1].bank[bank][static_cast<size_t>(m) * P.d[1].n + j]);
    if (P.dim == 3) t *= f2_to_double(P.d[2].bank[bank][static_cast<size_t>(m) * P.d[2].n + l]);
    u += t;
  }
  return u;
}

// Q = (x)omega (c_t u^k - L w(u^k)) at the nodes, u^k from the factors or the grid array
__global__ void actd_rhs_kernel(const StepParams P, int from_grid, int bank, int Mk, double* Q) {
  const int n1 = P.d[1].n, n2 = P.dim == 3 ? P.d[2].n : 1;
  const long long N = static_cast<long long>(P.d[0].n) * n1 * n2;
  for (long long p = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; p < N;
       p += static_cast<long long>(gridDim.x) * blockDim.x) {
    int i, j, l;
    grid_index(p, n1, n2, i, j, l);
    const double u = from_grid ? P.U[p] : field_value(P, bank, Mk, i, j, l);
    double om = P.d[0].omega[i] * P.d[1].omega[j];
    if (P.dim == 3) om *= P.d[2].omega[l];
    Q[p] = om * (P.c_t * u - P.L * 4.0 * P.a0 * (u * u * u - u));
  }
}

// Y /= c_t + c_k sum_d lambda_d
__global__ void actd_scale_kernel(const StepParams P, const double* lam0, const double* lam1, const double* lam2,
                                  double* Y) {
  const int n1 = P.d[1].n, n2 = P.dim == 3 ? P.d[2].n : 1;
  const long long N = static_cast<long long>(P.d[0].n) * n1 * n2;
  for (long long p = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; p < N;
       p += static_cast<long long>(gridDim.x) * blockDim.x) {
    int i, j, l;
    grid_index(p, n1, n2, i, j, l);
    double s = lam0[i] + lam1[j];
    if (P.dim == 3) s += lam2[l];
    Y[p] /= P.c_t + P.c_k * s;
  }
}

// V[:, k] /= sqrt(omega): eigenvectors of diag(omega)^-1/2 K diag(omega)^-1/2 to those of (K, M)
__global__ void actd_unscale_kernel(double* V, const double* omega, int n) {
  const long long total = static_cast<long long>(n) * n;
  for (long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(t % n);
    V[t] /= sqrt(omega[i]);
  }
}

__global__ void field_kernel(const StepParams P, int bank, int Mk, double* out) {
  const int n1 = P.d[1].n, n2 = P.dim == 3 ? P.d[2].n : 1;
  const long long N = static_cast<long long>(P.d[0].n) * n1 * n2;
  for (long long p = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; p < N;
       p += static_cast<long long>(gridDim.x) * blockDim.x) {
    int i, j, l;
    grid_index(p, n1, n2, i, j, l);
    out[p] = field_value(P, bank, Mk, i, j, l);
  }
}

// Discrete energy of a full-grid field (nodal rule): sum omega a0 (u^2 - 1)^2 plus
// 1/2 kappa sum_d u . (K_d along d, omega along the others) u; per-CTA partial sums.
__global__ void energy_grid_kernel(const StepParams P, double kappa, const double* U, double* part) {
  const int D = P.dim;
  const int nd[3] = {P.d[0].n, P.d[1].n, D == 3 ? P.d[2].n : 1};
  const long long N = static_cast<long long>(nd[0]) * nd[1] * nd[2];
  const long long st[3] = {static_cast<long long>(nd[1]) * nd[2], nd[2], 1};
  double acc = 0.0;
  for (long long p = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; p < N;
       p += static_cast<long long>(gridDim.x) * blockDim.x) {
    int idx[3];
    grid_index(p, nd[1], nd[2], idx[0], idx[1], idx[2]);
    const double u = U[p];
    double om[3];
    for (int d = 0; d < 3; ++d) om[d] = d < D ? P.d[d].omega[idx[d]] : 1.0;
    const double t = u * u - 1.0;
    double e = om[0] * om[1] * om[2] * P.a0 * t * t;
    for (int d = 0; d < D; ++d) {
      const Dim& dd = P.d[d];
      const int w = 2 * dd.b + 1, i = idx[d];
      double ku = 0.0;
      for (int jj = max(0, i - dd.b); jj <= min(dd.n - 1, i + dd.b); ++jj)
        ku = fma(dd.kband[static_cast<size_t>(i) * w + (jj - i + dd.b)], U[p + (jj - i) * st[d]], ku);
      double ow = 1.0;
      for (int e2 = 0; e2 < D; ++e2)
        if (e2 != d) ow *= om[e2];
      e = fma(0.5 * kappa * ow * u, ku, e);
    }
    acc += e;
  }
  acc = warp_sum(acc);
  __shared__ double s[kWarps];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += s[w];
    part[blockIdx.x] = t;
  }
}

}  // namespace

size_t actd_work_doubles(int n) {
  // the symmetric eigensolver with vectors needs about 1 + 6 n + 2 n^2 doubles, and a blocked
  // implementation more for small n: a floor of 4 Mi doubles (32 MiB)
  return 2 * static_cast<size_t>(n) * n + 64 * static_cast<size_t>(n) + (static_cast<size_t>(1) << 22);
}

int actd_setup(ActdState& a, const StepParams& P, const double* const* kband_host, const double* const* omega_host,
               cudaStream_t stream, const char** msg) {
  cublasHandle_t blas = nullptr;
  cusolverDnHandle_t dense = nullptr;
  if (cublasCreate(&blas) != CUBLAS_STATUS_SUCCESS) { *msg = "cublasCreate failed"; return -3; }
  a.blas = blas;
  if (cusolverDnCreate(&dense) != CUSOLVER_STATUS_SUCCESS) { *msg = "cusolverDnCreate failed"; return -3; }
  a.dense = dense;
  cublasSetStream(blas, stream);
  cusolverDnSetStream(dense, stream);
  cublasSetMathMode(blas, CUBLAS_DEFAULT_MATH);   // plain FP64 arithmetic, no emulation
  for (int d = 0; d < P.dim; ++d) {
    const int n = P.d[d].n, b = P.d[d].b, w = 2 * b + 1;
    // S = diag(omega)^-1/2 K diag(omega)^-1/2 (dense, symmetric)
    std::vector<double> S(static_cast<size_t>(n) * n, 0.0);
    for (int i = 0; i < n; ++i)
      for (int j = std::max(0, i - b); j <= std::min(n - 1, i + b); ++j)
        S[static_cast<size_t>(j) * n + i] =
            kband_host[d][static_cast<size_t>(i) * w + (j - i + b)] / std::sqrt(omega_host[d][i] * omega_host[d][j]);
    if (cudaMemcpyAsync(a.V[d], S.data(), sizeof(double) * S.size(), cudaMemcpyHostToDevice, stream) != cudaSuccess) {
      *msg = "eigenproblem upload failed";
      return -3;
    }
    int lwork = 0;
    if (cusolverDnDsyevd_bufferSize(dense, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, a.V[d], n, a.lam[d],
                                    &lwork) != CUSOLVER_STATUS_SUCCESS) {
      *msg = "cusolverDnDsyevd_bufferSize failed";
      return -3;
    }
    if (static_cast<size_t>(lwork) > a.work_len) { *msg = "eigensolver scratch exceeds its reserve"; return -7; }
    if (cusolverDnDsyevd(dense, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, a.V[d], n, a.lam[d], a.work,
                         lwork, a.info) != CUSOLVER_STATUS_SUCCESS) {
      *msg = "cusolverDnDsyevd failed";
      return -3;
    }
    int info = 0;
    cudaMemcpyAsync(&info, a.info, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (cudaStreamSynchronize(stream) != cudaSuccess || info != 0) { *msg = "eigensolver did not converge"; return -4; }
    actd_unscale_kernel<<<256, kThreads, 0, stream>>>(a.V[d], P.d[d].omega, n);
    if (cudaGetLastError() != cudaSuccess) { *msg = "eigenvector scaling failed"; return -3; }
  }
  return 0;
}

void actd_release(ActdState& a) {
  if (a.blas) cublasDestroy(static_cast<cublasHandle_t>(a.blas));
  if (a.dense) cusolverDnDestroy(static_cast<cusolverDnHandle_t>(a.dense));
  a.blas = nullptr;
  a.dense = nullptr;
}

namespace {
// out = Mat (or Mat^T) applied along axis d of the row-major array `in` of dims nd[]
// (out[.., i, ..] = sum_k Mat[i][k] in[.., k, ..]); Mat column-major n_d x n_d.
bool apply_axis(cublasHandle_t h, const double* Mat, bool transpose, const double* in, double* out, const int* nd,
                int D, int d) {
  long long A = 1, B = 1;
  for (int e = 0; e < d; ++e) A *= nd[e];
  for (int e = d + 1; e < D; ++e) B *= nd[e];
  const int n = nd[d];
  const double one = 1.0, zero = 0.0;
  if (B == 1) {
    // column-major view: in^c is n x A; out^c = op(Mat) in^c
    return cublasDgemm(h, transpose ? CUBLAS_OP_T : CUBLAS_OP_N, CUBLAS_OP_N, n, static_cast<int>(A), n, &one, Mat,
                       n, in, n, &zero, out, n) == CUBLAS_STATUS_SUCCESS;
  }
  // per leading index a: in_a^c is B x n; out_a^c = in_a^c op(Mat)^T
  return cublasDgemmStridedBatched(h, CUBLAS_OP_N, transpose ? CUBLAS_OP_N : CUBLAS_OP_T, static_cast<int>(B), n, n,
                                   &one, in, static_cast<int>(B), static_cast<long long>(n) * B, Mat, n, 0, &zero, out,
                                   static_cast<int>(B), static_cast<long long>(n) * B,
                                   static_cast<int>(A)) == CUBLAS_STATUS_SUCCESS;
}
}  // namespace

int actd_cfe_step(ActdState& a, const StepParams& P, int from_grid, int bank, int Mk, cudaStream_t stream,
                  const char** msg) {
  cublasHandle_t h = static_cast<cublasHandle_t>(a.blas);
  const int D = P.dim;
  int nd[3] = {P.d[0].n, P.d[1].n, D == 3 ? P.d[2].n : 1};
  const long long N = static_cast<long long>(nd[0]) * nd[1] * nd[2];
  actd_rhs_kernel<<<1024, kThreads, 0, stream>>>(P, from_grid, bank, Mk, a.Y);
  if (cudaGetLastError() != cudaSuccess) { *msg = "right-hand side launch failed"; return -3; }
  double* cur = a.Y;
  double* oth = P.U;   // free once the right-hand side is formed
  for (int d = 0; d < D; ++d) {
    if (!apply_axis(h, a.V[d], true, cur, oth, nd, D, d)) { *msg = "cublas transform failed"; return -3; }
    std::swap(cur, oth);
  }
  actd_scale_kernel<<<1024, kThreads, 0, stream>>>(P, a.lam[0], a.lam[1], D == 3 ? a.lam[2] : a.lam[1], cur);
  if (cudaGetLastError() != cudaSuccess) { *msg = "diagonal solve launch failed"; return -3; }
  for (int d = 0; d < D; ++d) {
    if (!apply_axis(h, a.V[d], false, cur, oth, nd, D, d)) { *msg = "cublas transform failed"; return -3; }
    std::swap(cur, oth);
  }
  if (cur != P.U &&
      cudaMemcpyAsync(P.U, cur, sizeof(double) * N, cudaMemcpyDeviceToDevice, stream) != cudaSuccess) {
    *msg = "field copy failed";
    return -3;
  }
  return 0;
}

cudaError_t launch_field_from_modes(const StepParams& P, int bank, int Mk, double* out, cudaStream_t s) {
  field_kernel<<<1024, kThreads, 0, s>>>(P, bank, Mk, out);
  return cudaGetLastError();
}

cudaError_t launch_energy_grid(const StepParams& P, const double* U, double* part, int grid, cudaStream_t s) {
  // kappa = c_k / L
  energy_grid_kernel<<<grid, kThreads, 0, s>>>(P, P.c_k / P.L, U, part);
  return cudaGetLastError();
}

}  // namespace ctd
