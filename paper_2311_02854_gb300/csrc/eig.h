// Block Jacobi symmetric eigensolver for the reduced density matrices of the
// decimation step (Sec. 2.1): many CTAs per matrix, all matrices of a
// decimation in one batch.
#pragma once

#include <functional>
#include <vector>

#include "engine.h"

namespace dmrg {

// Diagonalises every job's A (n x n, row-major, leading dimension lda; read
// only): eigenvalues to w[n], eigenvectors to the columns of V (ld lda).
// Works on private padded copies allocated through alloc_f / free_f
// (element counts).  Stops when every matrix has off(A)/|A| <= tol or after
// max_sweeps sweeps; returns the number of FP64 sweeps run.  Batches whose
// largest matrix has 256 rows or more are first swept in FP32 (count to
// *sweeps32), then the FP32 eigenvectors are made orthonormal in FP64 (two
// Newton-Schulz steps) and A is transformed to that basis (V^T A V, FP64)
// before the FP64 sweeps.  hist (optional) receives max over matrices of
// off(A)/|A| before every sweep of both stages and at the end.  tol32 > 0
// replaces the FP32 stage's target off(A)/|A| (default 1e-5).  df_rot: the
// rotations of the FP64 sweeps that follow an FP32 stage are applied in
// double-float arithmetic (~48 significant bits on the FP32 units) instead of
// FP64.
int block_jacobi_eigh(const std::vector<EigJob>& jobs, int max_sweeps, double tol, cudaStream_t st,
                      const std::function<double*(int64_t)>& alloc_f,
                      const std::function<void(double*, int64_t)>& free_f, std::vector<double>* hist = nullptr,
                      int* sweeps32 = nullptr, double tol32 = 0.0, bool df_rot = true);

}  // namespace dmrg
