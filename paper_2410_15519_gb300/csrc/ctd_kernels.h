// Host-callable launch wrappers of the CTD kernels.
#pragma once
#include "ctd_step.cuh"

namespace ctd {
// One instance of a batched launch (global memory).
struct __align__(128) BatchEntry {
  StepParams P;
  Extra X;
};
size_t step_smem_fixed_bytes();
size_t step_arena_bytes(int n_max, size_t solver_floats, int mode);
cudaError_t launch_step(const StepParams& P, const Extra& X, int grid, cudaStream_t s);
cudaError_t launch_step_sep(const StepParams& P, const Extra& X, int grid, cudaStream_t s);
cudaError_t launch_batch_step(const BatchEntry* entries, const int* order, int count, int kstep, size_t smem,
                              cudaStream_t s);
cudaError_t launch_probe_contract(const StepParams& P, const Extra& X, int grid, int x,
                                  float* dump, cudaStream_t s);
cudaError_t launch_probe_solve(const StepParams& P, const Extra& X, int x, double a1, double a2,
                               cudaStream_t s);
cudaError_t launch_convert_modes(const StepParams& P, const Extra& X, int bank, int Mk, cudaStream_t s);
cudaError_t launch_energy_bulk(const StepParams& P, const Extra& X, int Mk, double* part, int grid,
                               cudaStream_t s);
cudaError_t launch_energy_gram(const StepParams& P, const Extra& X, int Mk, double* out, cudaStream_t s);
cudaError_t launch_modes_from_fp64(float2* dst, const double* src, long long count, cudaStream_t s);
cudaError_t launch_modes_to_fp64(double* dst, const float2* src, long long count, cudaStream_t s);
}  // namespace ctd
