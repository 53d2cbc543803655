// Krylov solver internals (solver.cu) used by the C ABI layer.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "tn_internal.h"
#include "tn_precond.h"


// the operator and preconditioner of a solve: one mesh, or a batch of meshes
// grouped by polynomial degree (one launch per group)
struct OpSys {
  const DevMesh *m = nullptr;  // single mesh (host copy of the struct)
  const DevMesh *meshes = nullptr;  // batch: device array of the instances' meshes
  int ngroups = 0;
  int gN[8] = {0};
  const int2 *gwork[8] = {nullptr};  // (instance, element) per CTA of the apply
  int gcount[8] = {0};
  int gpart_off[8] = {0};
  const int2 *gline[8] = {nullptr};  // (instance, line) per warp of the z-line solve
  int glines[8] = {0};
  int grz_off[8] = {0};
  const long long *dof_off = nullptr, *fac_off = nullptr;
  int mvar = 0;           // occupancy variant of the FP32 operator kernel (single mesh)
  int gvar[8] = {0};      // the same per degree group of a batch
  int n_apply_parts = 0;  // partial sums written by one apply
  int n_rz_parts = 0;     // partial sums of r.z written by one z-line solve (r.r: as many, after them)
  TnWait *zerr = nullptr; // wait limit of the line solves; flag set by one whose staging wait ran out
  unsigned *fold_cnt = nullptr;  // grouped lines: 2 counters of the alpha / beta steps folded into
                                 // the apply and the line solve (nullptr: separate scalar kernels)
  bool grouped = false;   // grouped lines (zg) instead of single lines
  ZGroupDev zg;
  cudaError_t apply(int prec, const void *u, void *y, double *part, cudaStream_t st,
                    const PcgFold *fold = nullptr) const;
  // z = M^{-1} r; q != nullptr: first r <- r - (*alpha) q.  part: n_rz_parts
  // partial r.z, then n_rz_parts partial r.r
  cudaError_t zsolve(int prec, const void *fac, void *r, const void *q, void *z, const double *alpha,
                     double *part, const int *done, cudaStream_t st, const PcgFold *fold = nullptr) const;
};

// vectors of one PCG run, all of the run's precision
struct PcgVectors {
  void *x, *r, *z, *p, *q;
  const void *b, *dinv;
  const void *zfac = nullptr;   // z-line factors of the run's precision (nullptr: Jacobi)
  double *part_rz = nullptr;    // partial r.z and r.r of the z-line solve (2 n_rz_parts)
};

cudaError_t tn_jacobi_apply(size_t n, int prec, const double *diag, const void *r, void *z, cudaStream_t st);

// called on the host after every replayed chunk; returns true to stop the run
struct ChunkHook {
  bool (*fn)(void *user) = nullptr;
  void *user = nullptr;
};

namespace tn {
// kernel launches issued on behalf of the current solve (host counter)
extern thread_local long long g_launches;
// set by a PCG run that stopped because a line solve's bounded wait ran out
extern thread_local bool g_timed_out;
cudaError_t pcg_setup_dinv(size_t n, const double *diag, void *dinv, int prec, cudaStream_t st);
cudaError_t pcg_f64(const OpSys &sys, size_t n, PcgVectors &v, bool x0_zero, double rtol, int max_iters,
                    int chunk, tn_pcg_scalars *s_dev, tn_pcg_scalars *s_host, double *part_elem,
                    double *part_red, cudaStream_t st, int *applies, ChunkHook hook = ChunkHook());
cudaError_t pcg_f32(const OpSys &sys, size_t n, PcgVectors &v, bool x0_zero, double rtol, int max_iters,
                    int chunk, tn_pcg_scalars *s_dev, tn_pcg_scalars *s_host, double *part_elem,
                    double *part_red, cudaStream_t st, int *applies);
cudaError_t residual_f64(const OpSys &sys, size_t n, const double *b, const double *x, double *Ax, double *r,
                         double *part_red, double *sum_dev, double *rr_host, cudaStream_t st);
cudaError_t norm2_f64(size_t n, const double *v, double *part_red, double *sum_dev, double *out_host,
                      cudaStream_t st);
// per-segment squared norms: out[i] = |v[off[i] .. off[i + 1])|^2 (device and host copies; synchronises)
cudaError_t segnorm2_f64(int nseg, const long long *off, const double *v, double *out_dev, double *out_host,
                         cudaStream_t st);
cudaError_t cast_scaled(size_t n, const double *r64, double scale, float *r32, float *d32, cudaStream_t st);
cudaError_t refine_update(size_t n, double *x, const float *d, double scale, cudaStream_t st);
cudaError_t fill_f64(size_t n, double *v, double val, cudaStream_t st);
int reduction_blocks();
cudaError_t multidot(size_t n, const double *a, const double *const *B_dev, int nb, double *part, double *host_tmp,
                     double *out, cudaStream_t st);
cudaError_t fcg_orth(size_t n, const double *z, const double *q, const double *const *P, const double *const *AP,
                     const double *beta, int nb, double *p, double *Ap, cudaStream_t st);
cudaError_t fcg_step(size_t n, double alpha, const double *p, const double *Ap, double *x, double *r,
                     cudaStream_t st);
cudaError_t upcast(size_t n, const float *d, double scale, double *z, cudaStream_t st);
}  // namespace tn
