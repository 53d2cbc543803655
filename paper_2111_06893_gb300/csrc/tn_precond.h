// Column-line block preconditioner (precond.cu).
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "tn_internal.h"

size_t tn_zline_block_bytes(const DevMesh &m);   // FP64 set-up blocks
size_t tn_zline_factor_bytes(const DevMesh &m);  // FP32 factors kept for the solve
size_t tn_zline_factor_entries(const DevMesh &m);  // entries per precision (padded blocks)
int tn_zline_partials(const DevMesh &m);         // partial sums written by one solve
cudaError_t tn_zline_setup(const DevMesh &m, double *blk, float *fac, double *fac64, int *status,
                           cudaStream_t st);
cudaError_t tn_zline_solve(const DevMesh &m, int prec, const void *fac, const void *r, void *z, double *part,
                           const int *done, cudaStream_t st);
cudaError_t tn_upload_lgl_precond(const LglTables *t);
// batch: warp w of block b solves line work[4 b + w] = (instance, line); factors of
// instance i at fac + fac_off[i] (elements of the factor type), vectors at dof_off[i]
cudaError_t tn_zline_solve_batch(int N, int prec, const DevMesh *meshes, const int2 *work, int nwork,
                                 const long long *fac_off, const long long *dof_off, const void *fac,
                                 const void *r, void *z, double *part, const int *done, cudaStream_t st);
