// Krylov solve of A u = b (Sec. 2.3, Eq. (matrix_eqn)) on one GPU.
//
// The paper solves with GMRES; the weak-form DG operator built here is
// symmetric positive definite, so the solver is preconditioned conjugate
// gradients.  With the Jacobi preconditioner an iteration is five launches:
// the fused operator apply (which also returns p.Ap per element), a
// one-block reduction for alpha, a fused vector update (x, r, z = D^-1 r,
// partial r.z and r.r), a one-block reduction for beta and the direction
// update.  With the single-line preconditioner the residual update r -= alpha
// q runs inside the line solve (which also returns partial r.z and r.r);
// with grouped lines it is a launch of its own ahead of the solve (measured
// faster than fused there), and alpha and beta fold into the apply and the
// solve, four launches per iteration.  The solution update x += alpha p runs
// inside the direction update.  A chunk of
// iterations is recorded once in a CUDA graph and replayed.  Krylov scalars
// live on the device; once converged every kernel returns immediately, so a
// replayed chunk never runs past convergence.  The host reads a small status
// block after each chunk.  Reductions use a fixed partition and a fixed
// order, so results are bitwise reproducible.
//
// Mixed precision: a flexible CG in FP64 (residual, update, directions)
// preconditioned by a fixed number of FP32 PCG iterations (vectors,
// operator, line factors), scalars in FP64.
#include <cmath>
#include <cstring>

#include "tn_internal.h"
#include "tn_precond.h"
#include "tn_solver.h"

namespace {

// fixed partition of the vector reductions: 8 blocks per SM of the device
int red_blocks() { return 8 * tn_sm_count(); }
constexpr int kRedThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block sum of two values; result valid in thread 0
__device__ __forceinline__ void block_sum2(double &a, double &b) {
  __shared__ double ra[32], rb[32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { ra[w] = a; rb[w] = b; }
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    a = l < nw ? ra[l] : 0.0;
    b = l < nw ? rb[l] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
}

// sum of n doubles in a fixed order (one block)
__device__ double block_sum_array(const double *v, int n) {
  double acc = 0.0, dummy = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) acc += v[t];
  block_sum2(acc, dummy);
  return acc;
}

__global__ void k_alpha(tn_pcg_scalars *s, const double *partial, int n) {
  if (s->done) {
    if (threadIdx.x == 0) s->active = 0;
    return;
  }
  const double pq = block_sum_array(partial, n);
  if (threadIdx.x == 0) {
    s->active = 1;
    s->pq = pq;
    if (!(pq > 0.0) || !isfinite(pq)) {
      s->breakdown = 1;
      s->done = 1;
      s->alpha = 0.0;
    } else {
      s->alpha = s->rz / pq;
    }
  }
}

// per-thread accumulation in the vector precision (GB300's FP64 pipe is too
// narrow for per-element conversions), FP64 across threads in a fixed order
template <typename T>
__global__ void k_update(tn_pcg_scalars *s, size_t n, T *__restrict__ x, T *__restrict__ r,
                         T *__restrict__ z, const T *__restrict__ p, const T *__restrict__ q,
                         const T *__restrict__ dinv, double *part) {
  if (s->done) return;
  const T alpha = (T)s->alpha;
  T rzt = T(0), rrt = T(0);
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const T xv = x[t] + alpha * p[t];
    const T rv = r[t] - alpha * q[t];
    const T zv = dinv[t] * rv;
    x[t] = xv;
    r[t] = rv;
    z[t] = zv;
    rzt += rv * zv;
    rrt += rv * rv;
  }
  double rz = (double)rzt, rr = (double)rrt;
  block_sum2(rz, rr);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = rz;
    part[2 * blockIdx.x + 1] = rr;
  }
}

__global__ void k_beta(tn_pcg_scalars *s, const double *part, int nb) {
  if (s->done) return;
  double rz = 0.0, rr = 0.0;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) {
    rz += part[2 * t];
    rr += part[2 * t + 1];
  }
  block_sum2(rz, rr);
  if (threadIdx.x == 0) {
    s->iters += 1;
    s->rr = rr;
    if (!isfinite(rr) || !isfinite(rz)) {
      s->breakdown = 1;
      s->done = 1;
      return;
    }
    s->beta = rz / s->rz;
    s->rz = rz;
    if (rr <= s->tol2 || s->iters >= s->max_iters) s->done = 1;
  }
}

template <typename T>
__global__ void k_pupdate(const tn_pcg_scalars *s, size_t n, T *__restrict__ p, const T *__restrict__ z) {
  if (s->done) return;
  const T beta = (T)s->beta;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    p[t] = z[t] + beta * p[t];
}

// r = b - Ax, z = dinv r, p = z; partial r.z, r.r
template <typename T>
__global__ void k_init(size_t n, const T *__restrict__ b, const T *__restrict__ Ax, T *__restrict__ r,
                       T *__restrict__ z, T *__restrict__ p, const T *__restrict__ dinv, double *part) {
  double rz = 0.0, rr = 0.0;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const T rv = Ax ? b[t] - Ax[t] : b[t];
    const T zv = dinv[t] * rv;
    r[t] = rv;
    z[t] = zv;
    p[t] = zv;
    rz += (double)rv * (double)zv;
    rr += (double)rv * (double)rv;
  }
  block_sum2(rz, rr);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = rz;
    part[2 * blockIdx.x + 1] = rr;
  }
}

__global__ void k_init_scalars(tn_pcg_scalars *s, const double *part, int nb, double tol2_rel, int max_iters) {
  double rz = 0.0, rr = 0.0;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) {
    rz += part[2 * t];
    rr += part[2 * t + 1];
  }
  block_sum2(rz, rr);
  if (threadIdx.x == 0) {
    s->rz = rz;
    s->rr = rr;
    s->rr0 = rr;
    s->tol2 = tol2_rel * rr;
    s->iters = 0;
    s->max_iters = max_iters;
    s->breakdown = 0;
    s->done = (rr == 0.0 || rr <= s->tol2) ? 1 : 0;
    s->active = 0;
    s->alpha = s->beta = s->pq = 0.0;
  }
}

// sum of squares of a vector, fixed partition
template <typename T>
__global__ void k_sumsq(size_t n, const T *__restrict__ v, double *part) {
  double a = 0.0, dummy = 0.0;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    a += (double)v[t] * (double)v[t];
  block_sum2(a, dummy);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = a; part[2 * blockIdx.x + 1] = 0.0; }
}

__global__ void k_finish_sum(const double *part, int nb, double *out) {
  double a = 0.0, b = 0.0;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) { a += part[2 * t]; b += part[2 * t + 1]; }
  block_sum2(a, b);
  if (threadIdx.x == 0) { out[0] = a; out[1] = b; }
}

// r64 = b - Ax (FP64), partial r.r
__global__ void k_residual(size_t n, const double *__restrict__ b, const double *__restrict__ Ax,
                           double *__restrict__ r, double *part) {
  double a = 0.0, dummy = 0.0;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const double v = b[t] - Ax[t];
    r[t] = v;
    a += v * v;
  }
  block_sum2(a, dummy);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = a; part[2 * blockIdx.x + 1] = 0.0; }
}

// r32 = r64 * scale (rounded), d32 = 0
__global__ void k_cast_scaled(size_t n, const double *__restrict__ r64, double scale, float *__restrict__ r32,
                              float *__restrict__ d32) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    r32[t] = (float)(r64[t] * scale);
    d32[t] = 0.0f;
  }
}

// x64 += scale * d32
__global__ void k_refine(size_t n, double *__restrict__ x, const float *__restrict__ d, double scale) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    x[t] += scale * (double)d[t];
}

// dinv = 1 / diag, in T
template <typename T>
__global__ void k_invert(size_t n, const double *__restrict__ d, T *__restrict__ dinv) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    dinv[t] = (T)(1.0 / d[t]);
}

template <typename T>
__global__ void k_jacobi(size_t n, const double *__restrict__ d, const T *__restrict__ r, T *__restrict__ z) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    z[t] = (T)((double)r[t] / d[t]);
}

template <typename T>
__global__ void k_fill(size_t n, T *__restrict__ v, T val) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    v[t] = val;
}


// out[i] = sum of squares of v over segment i = [off[i], off[i + 1]) (one
// block per segment, fixed order; off has nseg + 1 entries, off[nseg] = n)
__global__ void k_segsumsq(const long long *__restrict__ off, const double *__restrict__ v,
                           double *__restrict__ out) {
  const long long a = off[blockIdx.x], b = off[blockIdx.x + 1];
  double acc = 0.0, dummy = 0.0;
  for (long long t = a + threadIdx.x; t < b; t += blockDim.x) acc += v[t] * v[t];
  block_sum2(acc, dummy);
  if (threadIdx.x == 0) out[blockIdx.x] = acc;
}

// ---- flexible CG (FP64 outer of the mixed-precision solve)
// dots[j] partials: a . B_j for up to 16 vectors B_j, fixed partition
__global__ void k_multidot(size_t n, const double *__restrict__ a, const double *const *__restrict__ B, int nb,
                           double *part) {
  __shared__ double red[16][8];
  double acc[16];
  for (int j = 0; j < nb; ++j) acc[j] = 0.0;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const double av = a[t];
    for (int j = 0; j < nb; ++j) acc[j] += av * B[j][t];
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int j = 0; j < nb; ++j) {
    double v = warp_sum(acc[j]);
    if (l == 0) red[j][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < nb) {
    double v = 0.0;
    for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) v += red[threadIdx.x][ww];
    part[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = v;
  }
}

// p = z - sum_j beta_j P_j,  Ap = q - sum_j beta_j AP_j
__global__ void k_fcg_orth(size_t n, const double *__restrict__ z, const double *__restrict__ q,
                           const double *const *__restrict__ P, const double *const *__restrict__ AP,
                           const double *__restrict__ beta, int nb, double *__restrict__ p, double *__restrict__ Ap) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    double pv = z[t], av = q[t];
    for (int j = 0; j < nb; ++j) {
      pv -= beta[j] * P[j][t];
      av -= beta[j] * AP[j][t];
    }
    p[t] = pv;
    Ap[t] = av;
  }
}

// x += alpha p, r -= alpha Ap
__global__ void k_fcg_step(size_t n, double alpha, const double *__restrict__ p, const double *__restrict__ Ap,
                           double *__restrict__ x, double *__restrict__ r) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    x[t] += alpha * p[t];
    r[t] -= alpha * Ap[t];
  }
}

// z64 = scale * d32
__global__ void k_upcast(size_t n, const float *__restrict__ d, double scale, double *__restrict__ z) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    z[t] = scale * (double)d[t];
}

// ---- variants for a preconditioner applied by a separate kernel (z-line)

__global__ void k_beta_split(tn_pcg_scalars *s, const double *rzp, int nrz, const double *rrp, int nrr) {
  if (s->done) return;
  double rz = 0.0, rr = 0.0;
  for (int t = threadIdx.x; t < nrz; t += blockDim.x) rz += rzp[t];
  for (int t = threadIdx.x; t < nrr; t += blockDim.x) rr += rrp[t];
  block_sum2(rz, rr);
  if (threadIdx.x == 0) pcg_finish_beta(s, rz, rr);
}

// x += alpha p (the iteration's solution update, deferred to here so that
// the residual update can run inside the line solve), then p = z + beta p
// unless the run has just finished
template <typename T>
__global__ void k_pupdate_x(const tn_pcg_scalars *s, size_t n, T *__restrict__ x, T *__restrict__ p,
                            const T *__restrict__ z) {
  if (!s->active) return;
  const T alpha = (T)s->alpha, beta = (T)s->beta;
  const bool more = !s->done;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const T pv = p[t];
    x[t] += alpha * pv;
    if (more) p[t] = z[t] + beta * pv;
  }
}

// r = b - Ax (or b), partial r.r
template <typename T>
__global__ void k_init_r(size_t n, const T *__restrict__ b, const T *__restrict__ Ax, T *__restrict__ r,
                         double *part) {
  double rr = 0.0, dummy = 0.0;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const T rv = Ax ? b[t] - Ax[t] : b[t];
    r[t] = rv;
    rr += (double)rv * (double)rv;
  }
  block_sum2(rr, dummy);
  if (threadIdx.x == 0) part[blockIdx.x] = rr;
}

template <typename T>
__global__ void k_copy(size_t n, T *__restrict__ dst, const T *__restrict__ src) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    dst[t] = src[t];
}

__global__ void k_init_scalars_split(tn_pcg_scalars *s, const double *rzp, int nrz, const double *rrp, int nrr,
                                     double tol2_rel, int max_iters) {
  double rz = 0.0, rr = 0.0;
  for (int t = threadIdx.x; t < nrz; t += blockDim.x) rz += rzp[t];
  for (int t = threadIdx.x; t < nrr; t += blockDim.x) rr += rrp[t];
  block_sum2(rz, rr);
  if (threadIdx.x == 0) {
    s->rz = rz;
    s->rr = rr;
    s->rr0 = rr;
    s->tol2 = tol2_rel * rr;
    s->iters = 0;
    s->max_iters = max_iters;
    s->breakdown = 0;
    s->done = (rr == 0.0 || rr <= s->tol2) ? 1 : 0;
    s->active = 0;
    s->alpha = s->beta = s->pq = 0.0;
  }
}

}  // namespace

// ------------------------------------------------------------------ host

namespace tn {

thread_local long long g_launches = 0;
thread_local bool g_timed_out = false;

#define TN_CU(call)                                   \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return e_;                 \
  } while (0)

cudaError_t pcg_setup_dinv(size_t n, const double *diag, void *dinv, int prec, cudaStream_t st) {
  g_launches += 1;
  if (prec == TN_F64) k_invert<double><<<red_blocks(), kRedThreads, 0, st>>>(n, diag, (double *)dinv);
  else k_invert<float><<<red_blocks(), kRedThreads, 0, st>>>(n, diag, (float *)dinv);
  return cudaGetLastError();
}

// one PCG iteration (five launches), all on stream st
template <typename T>
static cudaError_t pcg_iteration(const OpSys &sys, int prec, size_t n, PcgVectors &v, tn_pcg_scalars *s,
                                 double *part_elem, double *part_red, cudaStream_t st) {
  TN_CU(sys.apply(prec, v.p, v.q, part_elem, st));
  k_alpha<<<1, 1024, 0, st>>>(s, part_elem, sys.n_apply_parts);
  TN_CU(cudaGetLastError());
  k_update<T><<<red_blocks(), kRedThreads, 0, st>>>(s, n, (T *)v.x, (T *)v.r, (T *)v.z, (const T *)v.p,
                                                  (const T *)v.q, (const T *)v.dinv, part_red);
  TN_CU(cudaGetLastError());
  k_beta<<<1, 1024, 0, st>>>(s, part_red, red_blocks());
  TN_CU(cudaGetLastError());
  k_pupdate<T><<<red_blocks(), kRedThreads, 0, st>>>(s, n, (T *)v.p, (const T *)v.z);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t pcg_iteration_zline(const OpSys &sys, int prec, size_t n, PcgVectors &v, tn_pcg_scalars *s,
                                       double *part_elem, double *part_red, cudaStream_t st) {
  if (sys.grouped && sys.fold_cnt) {
    // four launches: the apply with the alpha step, the residual update,
    // the grouped-line solve with the beta step, the direction update
    PcgFold fa;
    fa.s = s;
    fa.cnt = sys.fold_cnt;
    fa.total = sys.n_apply_parts;  // one CTA per element
    fa.nparts = sys.n_apply_parts;
    fa.part = part_elem;
    TN_CU(sys.apply(prec, v.p, v.q, part_elem, st, &fa));
    PcgFold fb;
    fb.s = s;
    fb.cnt = sys.fold_cnt + 1;
    TN_CU(sys.zsolve(prec, v.zfac, v.r, v.q, v.z, &s->alpha, v.part_rz, &s->done, st, &fb));
    k_pupdate_x<T><<<red_blocks(), kRedThreads, 0, st>>>(s, n, (T *)v.x, (T *)v.p, (const T *)v.z);
    return cudaGetLastError();
  }
  TN_CU(sys.apply(prec, v.p, v.q, part_elem, st));
  k_alpha<<<1, 1024, 0, st>>>(s, part_elem, sys.n_apply_parts);
  TN_CU(cudaGetLastError());
  // r -= alpha q fused into the line solve (partials r.z and r.r)
  TN_CU(sys.zsolve(prec, v.zfac, v.r, v.q, v.z, &s->alpha, v.part_rz, &s->done, st));
  k_beta_split<<<1, 1024, 0, st>>>(s, v.part_rz, sys.n_rz_parts, v.part_rz + sys.n_rz_parts, sys.n_rz_parts);
  TN_CU(cudaGetLastError());
  k_pupdate_x<T><<<red_blocks(), kRedThreads, 0, st>>>(s, n, (T *)v.x, (T *)v.p, (const T *)v.z);
  return cudaGetLastError();
}

// PCG on A x = b in precision T; x holds the initial guess (x0_zero: x = 0).
// Records `chunk` iterations in a graph and replays it until done.
template <typename T>
static cudaError_t pcg_run(const OpSys &sys, int prec, size_t n, PcgVectors &v, bool x0_zero, double rtol,
                           int max_iters, int chunk, tn_pcg_scalars *s_dev, tn_pcg_scalars *s_host,
                           double *part_elem, double *part_red, cudaStream_t st, int *applies,
                           ChunkHook hook = ChunkHook()) {
  const bool zl = v.zfac != nullptr;
  g_launches += zl ? 5 : 3;
  if (x0_zero) {
    k_fill<T><<<red_blocks(), kRedThreads, 0, st>>>(n, (T *)v.x, T(0));
    TN_CU(cudaGetLastError());
  } else {
    TN_CU(sys.apply(prec, v.x, v.q, nullptr, st));
    *applies += 1;
  }
  const T *Ax = x0_zero ? nullptr : (const T *)v.q;
  if (zl) {
    k_init_r<T><<<red_blocks(), kRedThreads, 0, st>>>(n, (const T *)v.b, Ax, (T *)v.r, part_red);
    TN_CU(cudaGetLastError());
    TN_CU(sys.zsolve(prec, v.zfac, v.r, nullptr, v.z, nullptr, v.part_rz, nullptr, st));
    k_copy<T><<<red_blocks(), kRedThreads, 0, st>>>(n, (T *)v.p, (const T *)v.z);
    TN_CU(cudaGetLastError());
    k_init_scalars_split<<<1, 256, 0, st>>>(s_dev, v.part_rz, sys.n_rz_parts, v.part_rz + sys.n_rz_parts,
                                            sys.n_rz_parts, rtol * rtol, max_iters);
  } else {
    k_init<T><<<red_blocks(), kRedThreads, 0, st>>>(n, (const T *)v.b, Ax, (T *)v.r, (T *)v.z, (T *)v.p,
                                                  (const T *)v.dinv, part_red);
    TN_CU(cudaGetLastError());
    k_init_scalars<<<1, 256, 0, st>>>(s_dev, part_red, red_blocks(), rtol * rtol, max_iters);
  }
  TN_CU(cudaGetLastError());
  TN_CU(cudaMemcpyAsync(s_host, s_dev, sizeof(tn_pcg_scalars), cudaMemcpyDeviceToHost, st));
  TN_CU(cudaStreamSynchronize(st));
  if (s_host->done) return cudaSuccess;
  if (zl && sys.grouped && sys.fold_cnt) TN_CU(cudaMemsetAsync(sys.fold_cnt, 0, 2 * sizeof(unsigned), st));

  // one graph of `chunk` iterations, cached while the run's buffers are unchanged
  struct Key {
    const void *x, *r, *z, *p, *q, *b, *dinv, *zfac;
    const double *part_rz, *pe, *pr;
    const void *s;
    size_t n;
    int chunk, prec, E;
    const void *geo;
    DevMesh dm;  // baked into the captured kernel parameters
    OpSys sys;
    bool operator==(const Key &o) const { return std::memcmp(this, &o, sizeof(Key)) == 0; }
  };
  Key key;
  std::memset(static_cast<void *>(&key), 0, sizeof(key));
  key.x = v.x; key.r = v.r; key.z = v.z; key.p = v.p; key.q = v.q; key.b = v.b; key.dinv = v.dinv;
  key.zfac = v.zfac; key.part_rz = v.part_rz; key.pe = part_elem; key.pr = part_red; key.s = s_dev;
  key.n = n; key.chunk = chunk; key.prec = prec; key.E = sys.n_apply_parts;
  key.geo = sys.m ? (const void *)sys.m->colgeo : (const void *)sys.meshes;
  if (sys.m) std::memcpy(static_cast<void *>(&key.dm), sys.m, sizeof(DevMesh));
  std::memcpy(static_cast<void *>(&key.sys), &sys, sizeof(OpSys));
  key.sys.m = nullptr;
  static thread_local Key cached_key[2];
  static thread_local cudaGraphExec_t cached_exec[2] = {nullptr, nullptr};
  const int slot = prec == TN_F64 ? 0 : 1;
  cudaGraphExec_t exec = nullptr;
  cudaError_t err = cudaSuccess;
  if (cached_exec[slot] && cached_key[slot] == key) {
    exec = cached_exec[slot];
  } else {
    if (cached_exec[slot]) { cudaGraphExecDestroy(cached_exec[slot]); cached_exec[slot] = nullptr; }
    cudaGraph_t graph = nullptr;
    TN_CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaError_t cap = cudaSuccess;
    for (int it = 0; it < chunk && cap == cudaSuccess; ++it)
      cap = zl ? pcg_iteration_zline<T>(sys, prec, n, v, s_dev, part_elem, part_red, st)
               : pcg_iteration<T>(sys, prec, n, v, s_dev, part_elem, part_red, st);
    cudaError_t endc = cudaStreamEndCapture(st, &graph);
    if (cap != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return cap; }
    TN_CU(endc);
    err = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    TN_CU(err);
    cached_exec[slot] = exec;
    cached_key[slot] = key;
  }
  double best = INFINITY;
  int stall = 0;
  for (;;) {
    g_launches += (zl && sys.grouped && sys.fold_cnt ? 4LL : (zl && sys.grouped ? 6LL : 5LL)) * chunk;
    err = cudaGraphLaunch(exec, st);
    if (err != cudaSuccess) break;
    err = cudaMemcpyAsync(s_host, s_dev, sizeof(tn_pcg_scalars), cudaMemcpyDeviceToHost, st);
    if (err != cudaSuccess) break;
    int waitflag = 0;
    if (sys.zerr) err = cudaMemcpyAsync(&waitflag, &sys.zerr->flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (err != cudaSuccess) break;
    err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) break;
    if (waitflag) {  // a line solve gave up on its staged factors: the run is void
      g_timed_out = true;
      break;
    }
    if (s_host->done) break;
    if (hook.fn && hook.fn(hook.user)) break;
    // stagnation: the recursive residual has not halved for 40 chunks
    if (s_host->rr < 0.5 * best) { best = s_host->rr; stall = 0; }
    else if (++stall >= 40) break;
  }
  *applies += s_host->iters;
  return err;
}

cudaError_t pcg_f64(const OpSys &sys, size_t n, PcgVectors &v, bool x0_zero, double rtol, int max_iters,
                    int chunk, tn_pcg_scalars *s_dev, tn_pcg_scalars *s_host, double *part_elem,
                    double *part_red, cudaStream_t st, int *applies, ChunkHook hook) {
  return pcg_run<double>(sys, TN_F64, n, v, x0_zero, rtol, max_iters, chunk, s_dev, s_host, part_elem,
                         part_red, st, applies, hook);
}

cudaError_t pcg_f32(const OpSys &sys, size_t n, PcgVectors &v, bool x0_zero, double rtol, int max_iters,
                    int chunk, tn_pcg_scalars *s_dev, tn_pcg_scalars *s_host, double *part_elem,
                    double *part_red, cudaStream_t st, int *applies) {
  return pcg_run<float>(sys, TN_F32, n, v, x0_zero, rtol, max_iters, chunk, s_dev, s_host, part_elem,
                        part_red, st, applies);
}

// r = b - A x in FP64; returns ||r||^2 in *rr_host (synchronises)
cudaError_t residual_f64(const OpSys &sys, size_t n, const double *b, const double *x, double *Ax, double *r,
                         double *part_red, double *sum_dev, double *rr_host, cudaStream_t st) {
  g_launches += 3;
  TN_CU(sys.apply(TN_F64, x, Ax, nullptr, st));
  k_residual<<<red_blocks(), kRedThreads, 0, st>>>(n, b, Ax, r, part_red);
  TN_CU(cudaGetLastError());
  k_finish_sum<<<1, 256, 0, st>>>(part_red, red_blocks(), sum_dev);
  TN_CU(cudaGetLastError());
  double tmp[2];
  TN_CU(cudaMemcpyAsync(tmp, sum_dev, sizeof(tmp), cudaMemcpyDeviceToHost, st));
  TN_CU(cudaStreamSynchronize(st));
  *rr_host = tmp[0];
  return cudaSuccess;
}

cudaError_t norm2_f64(size_t n, const double *v, double *part_red, double *sum_dev, double *out_host,
                      cudaStream_t st) {
  g_launches += 2;
  k_sumsq<double><<<red_blocks(), kRedThreads, 0, st>>>(n, v, part_red);
  TN_CU(cudaGetLastError());
  k_finish_sum<<<1, 256, 0, st>>>(part_red, red_blocks(), sum_dev);
  TN_CU(cudaGetLastError());
  double tmp[2];
  TN_CU(cudaMemcpyAsync(tmp, sum_dev, sizeof(tmp), cudaMemcpyDeviceToHost, st));
  TN_CU(cudaStreamSynchronize(st));
  *out_host = tmp[0];
  return cudaSuccess;
}

cudaError_t segnorm2_f64(int nseg, const long long *off, const double *v, double *out_dev, double *out_host,
                         cudaStream_t st) {
  g_launches += 1;
  k_segsumsq<<<nseg, 256, 0, st>>>(off, v, out_dev);
  TN_CU(cudaGetLastError());
  TN_CU(cudaMemcpyAsync(out_host, out_dev, sizeof(double) * nseg, cudaMemcpyDeviceToHost, st));
  return cudaStreamSynchronize(st);
}

cudaError_t cast_scaled(size_t n, const double *r64, double scale, float *r32, float *d32, cudaStream_t st) {
  g_launches += 1;
  k_cast_scaled<<<red_blocks(), kRedThreads, 0, st>>>(n, r64, scale, r32, d32);
  return cudaGetLastError();
}

cudaError_t refine_update(size_t n, double *x, const float *d, double scale, cudaStream_t st) {
  g_launches += 1;
  k_refine<<<red_blocks(), kRedThreads, 0, st>>>(n, x, d, scale);
  return cudaGetLastError();
}

cudaError_t fill_f64(size_t n, double *v, double val, cudaStream_t st) {
  g_launches += 1;
  k_fill<double><<<red_blocks(), kRedThreads, 0, st>>>(n, v, val);
  return cudaGetLastError();
}

int reduction_blocks() { return red_blocks(); }

}  // namespace tn

cudaError_t OpSys::apply(int prec, const void *u, void *y, double *part, cudaStream_t st,
                         const PcgFold *fold) const {
  if (m) return tn_launch_apply(*m, prec, u, y, part, mvar, st, fold);
  for (int g = 0; g < ngroups; ++g) {
    cudaError_t e = tn_launch_apply_batch(gN[g], prec, meshes, gwork[g], gcount[g], dof_off, u, y,
                                          part ? part + gpart_off[g] : nullptr, gvar[g], st, fold);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t OpSys::zsolve(int prec, const void *fac, void *r, const void *q, void *z, const double *alpha,
                          double *part, const int *done, cudaStream_t st, const PcgFold *fold) const {
  double *prr = part ? part + n_rz_parts : nullptr;
  if (grouped) return tn_zgroup_solve(m, zg, prec, fac, r, q, z, alpha, part, prr, done, zerr, st, fold);
  if (m) return tn_zline_solve(*m, prec, fac, r, q, z, alpha, part, prr, done, zerr, st);
  for (int g = 0; g < ngroups; ++g) {
    cudaError_t e = tn_zline_solve_batch(gN[g], prec, meshes, gline[g], glines[g], fac_off, dof_off, fac, r, q, z,
                                         alpha, part ? part + grz_off[g] : nullptr,
                                         prr ? prr + grz_off[g] : nullptr, done, zerr, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

namespace tn {

// dots a . B_j (j < nb <= 16) summed in a fixed order on the host
cudaError_t multidot(size_t n, const double *a, const double *const *B_dev, int nb, double *part, double *host_tmp,
                     double *out, cudaStream_t st) {
  g_launches += 1;
  k_multidot<<<red_blocks(), kRedThreads, 0, st>>>(n, a, B_dev, nb, part);
  TN_CU(cudaGetLastError());
  TN_CU(cudaMemcpyAsync(host_tmp, part, sizeof(double) * nb * red_blocks(), cudaMemcpyDeviceToHost, st));
  TN_CU(cudaStreamSynchronize(st));
  for (int j = 0; j < nb; ++j) {
    double s = 0.0;
    for (int b = 0; b < red_blocks(); ++b) s += host_tmp[(size_t)j * red_blocks() + b];
    out[j] = s;
  }
  return cudaSuccess;
}

cudaError_t fcg_orth(size_t n, const double *z, const double *q, const double *const *P, const double *const *AP,
                     const double *beta, int nb, double *p, double *Ap, cudaStream_t st) {
  g_launches += 1;
  k_fcg_orth<<<red_blocks(), kRedThreads, 0, st>>>(n, z, q, P, AP, beta, nb, p, Ap);
  return cudaGetLastError();
}

cudaError_t fcg_step(size_t n, double alpha, const double *p, const double *Ap, double *x, double *r,
                     cudaStream_t st) {
  g_launches += 1;
  k_fcg_step<<<red_blocks(), kRedThreads, 0, st>>>(n, alpha, p, Ap, x, r);
  return cudaGetLastError();
}

cudaError_t upcast(size_t n, const float *d, double scale, double *z, cudaStream_t st) {
  g_launches += 1;
  k_upcast<<<red_blocks(), kRedThreads, 0, st>>>(n, d, scale, z);
  return cudaGetLastError();
}

}  // namespace tn

cudaError_t tn_jacobi_apply(size_t n, int prec, const double *diag, const void *r, void *z, cudaStream_t st) {
  if (prec == TN_F64) k_jacobi<double><<<red_blocks(), kRedThreads, 0, st>>>(n, diag, (const double *)r, (double *)z);
  else k_jacobi<float><<<red_blocks(), kRedThreads, 0, st>>>(n, diag, (const float *)r, (float *)z);
  return cudaGetLastError();
}

namespace tn {

}  // namespace tn
