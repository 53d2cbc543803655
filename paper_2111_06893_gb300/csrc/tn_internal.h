// Internal structures shared by the host code and the kernels of the
// thermonoise library.  Geometry is stored factorised: every element map of
// the box and cylinder meshes is x(xi, eta, zeta) = (X(xi, eta), Y(xi, eta),
// Z(zeta)) -- a cross-section map of the element's column times a vertical
// map of its slab -- so the Jacobian is block diagonal and the per-node
// geometry of Sec. 2.2.1 (J, det J, J^-1) is the product of a 2-D column
// table and a 1-D slab table.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/thermonoise.h"

#define TN_MAX_N 9
#define TN_MIN_N 3

// column geometry, per column and per cross-section node q = j * N + i
enum {
  CG_IXX = 0,  // dxi/dx
  CG_IXY = 1,  // dxi/dy
  CG_IEX = 2,  // deta/dx
  CG_IEY = 3,  // deta/dy
  CG_DET = 4,  // det of d(X, Y)/d(xi, eta)
  CG_X = 5,    // X
  CG_Y = 6,    // Y
  CG_NF = 7
};
// slab geometry, per slab and per node k along zeta
enum { SG_DZ = 0, SG_Z = 1, SG_NF = 2 };

struct DevMesh {
  int N;          // LGL points per dimension
  int p;          // degree
  int E;          // elements
  int ncol;       // columns
  int nslab;      // slabs
  int n_layers;
  int bc_side;    // TN_BC_*
  int bc_bottom;
  double penC;    // penalty constant C
  const double *colgeo;   // [ncol][CG_NF][N*N]
  const double *slabgeo;  // [nslab][SG_NF][N]
  const int *colnb;       // [ncol][4]: neighbour column across faces xi-, xi+, eta-, eta+ (-1: side)
  const int *colnbf;      // [ncol][4]: neighbour face (0..3) | (flip << 2)
  const int *slab_layer;  // [nslab]
  const double *layer_c;  // [n_layers][3]: c11, c12, c44 (isotropic: lambda+2mu, lambda, mu)
  // FP32 copies of the tables for the FP32 kernels (GB300's FP64 pipe is
  // too narrow for per-node double -> float conversions)
  const float *colgeo32 = nullptr;
  const float *slabgeo32 = nullptr;
  const float *layer_c32 = nullptr;
  float penC32 = 0.0f;
  // forward-mode seeds for derivative kernels (nullptr: no dependence)
  const double *d_slabdz = nullptr;  // [nslab][N]: d(dz/dzeta)/dtheta at each node
  const double *d_layer_c = nullptr;  // [n_layers][3]: d(c11, c12, c44)/dtheta
};

// bounded device waits (the staging waits of the line solves): the kernels
// read limit_ns and give up a wait after that many nanoseconds of
// %globaltimer, set flag = 1, wait (bounded again) for their copies still in
// flight and return; the host reports TN_ETIMEOUT.  Lives in device memory.
struct TnWait {
  unsigned long long limit_ns;
  int flag;
  int pad;
};
constexpr unsigned long long kDefaultWaitNs = 1000000000ull;  // 1 s

// device-resident Krylov scalars of one PCG run
struct tn_pcg_scalars {
  double rz, rr, rr0, pq, alpha, beta, tol2;
  int iters, max_iters, done, breakdown;
  int active;  // the current iteration ran (set by the alpha step)
};

// A PCG scalar step folded into the kernel that produces its partial sums:
// every CTA of the step's launches counts itself on cnt once its partial is
// written; the last one reduces the nparts partials in a fixed order,
// updates the scalars and resets cnt.  s == nullptr: no fold.
struct PcgFold {
  tn_pcg_scalars *s = nullptr;
  unsigned *cnt = nullptr;
  int total = 0;              // CTAs of all launches of the step
  int nparts = 0;             // partial sums to reduce
  const double *part = nullptr;   // the first of them (the second sum's follow at part2)
  const double *part2 = nullptr;
};

#ifdef __CUDACC__
// the beta step of a PCG iteration from the new r.z and r.r: beta, the
// stopping test (rr <= tol2 or the iteration limit), breakdown if either
// sum is not finite
__device__ inline void pcg_finish_beta(tn_pcg_scalars *s, double rz, double rr) {
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
#endif

// forward-mode dual number (value, derivative along one direction)
struct Dual {
  double v, d;
  Dual() = default;
  __host__ __device__ constexpr Dual(double a) : v(a), d(0.0) {}
  __host__ __device__ constexpr Dual(double a, double b) : v(a), d(b) {}
};
__host__ __device__ inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__host__ __device__ inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__host__ __device__ inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__host__ __device__ inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__host__ __device__ inline Dual operator/(Dual a, Dual b) {
  const double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
__host__ __device__ inline Dual &operator+=(Dual &a, Dual b) { a = a + b; return a; }
__host__ __device__ inline Dual &operator-=(Dual &a, Dual b) { a = a - b; return a; }
__host__ __device__ inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
__device__ inline Dual sqrt(Dual a) {
  const double r = ::sqrt(a.v);
  return Dual(r, 0.5 * a.d / r);
}

// LGL tables in constant memory, indexed by N (filled at context creation)
struct LglTables {
  double x[TN_MAX_N + 1][TN_MAX_N];
  double w[TN_MAX_N + 1][TN_MAX_N];
  double D[TN_MAX_N + 1][TN_MAX_N * TN_MAX_N];  // D[a*N+b] = l_b'(x_a)
};

// host-side helpers (mesh.cpp)
namespace tn {
void lgl(int N, double *x, double *w, double *D);
struct HostMesh {
  int N = 0, p = 0, E = 0, ncol = 0, nslab = 0, n_layers = 0;
  int bc_side = 0, bc_bottom = 0;
  double penC = 0;
  double *colgeo = nullptr;
  double *slabgeo = nullptr;
  int *colnb = nullptr, *colnbf = nullptr, *slab_layer = nullptr;
};
// fills host arrays (malloc'ed) from a description; returns TN_OK or TN_EINVAL with msg
tn_status build_host_mesh(const tn_mesh_desc *d, HostMesh *out, char *msg, int msglen);
void free_host_mesh(HostMesh *m);
}  // namespace tn

// streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount)
int tn_sm_count();

// kernels (kernels.cu) -- launchers return cudaError_t of the launch
cudaError_t tn_upload_lgl(const LglTables *t);
// derivative kernels: over the elements of slabs [s0, s1),
//   part[e - s0*ncol] = lam_e . (dA/dtheta u)_e        (seeds in m.d_*)
//   epart[e - s0*ncol] = w[layer(e)] dU_e/dtheta|_u
cudaError_t tn_launch_apply_dual(const DevMesh &m, int s0, int s1, const double *u, const double *lam,
                                 double *part, cudaStream_t st);
cudaError_t tn_launch_energy_dual(const DevMesh &m, int s0, int s1, const double *u, const double *w,
                                  double *epart, cudaStream_t st);
// the same for many parameters in one launch each: CTA b contracts element
// work[b].y along parameter work[b].x, seeded by pseed[2 p] (d_slabdz) and
// pseed[2 p + 1] (d_layer_c), device arrays; part[b] / epart[b]
cudaError_t tn_launch_apply_dual_work(const DevMesh &m, const int2 *work, int nwork, const double *const *pseed,
                                      const double *u, const double *lam, double *part, cudaStream_t st);
cudaError_t tn_launch_energy_dual_work(const DevMesh &m, const int2 *work, int nwork, const double *const *pseed,
                                       const double *u, const double *w, double *epart, cudaStream_t st);
// g = sum_i w_i K_i u (the derivative of sum_i w_i U_i with respect to u)
cudaError_t tn_launch_energy_source(const DevMesh &m, const double *u, const double *w, double *g,
                                    cudaStream_t st);
// part[b] = partial sums of lam . db/dr0 (beam width derivative of the load)
cudaError_t tn_launch_rhs_dr0(const DevMesh &m, double r0, double F0, const double *lam, double *part,
                              int nparts, cudaStream_t st);
// batches: one launch per polynomial degree; work[b] = (instance, element).
// var: occupancy variant of the FP32 kernel (0 or 1, same results)
cudaError_t tn_launch_apply_batch(int N, int precision, const DevMesh *meshes, const int2 *work, int nwork,
                                  const long long *dof_off, const void *u, void *y, double *partial,
                                  int var, cudaStream_t st, const PcgFold *fold = nullptr);
// us[v]: time per launch of FP32 variant v on one mesh (m1) or on one degree
// group of a batch (m1 = nullptr); y is overwritten
cudaError_t tn_tune_apply(const DevMesh *m1, int N, const DevMesh *meshes, const int2 *work, int nwork,
                          const long long *dof_off, const float *u, float *y, cudaStream_t st, float us[2]);
cudaError_t tn_launch_energy_batch(int N, const DevMesh *meshes, const int2 *work, int nwork,
                                   const long long *dof_off, const double *u, double *out, cudaStream_t st);
// fold (optional): the alpha step of a PCG iteration (partial = p . Ap per CTA)
cudaError_t tn_launch_apply(const DevMesh &m, int precision, const void *u, void *y,
                            double *partial, int var, cudaStream_t st, const PcgFold *fold = nullptr);
// CTAs one apply launches (one mesh, or one degree group of a batch)
int tn_apply_ctas(const DevMesh *m, int nwork);
cudaError_t tn_launch_rhs(const DevMesh &m, double r0, double F0, double *b, cudaStream_t st);
cudaError_t tn_launch_diag(const DevMesh &m, double *d, cudaStream_t st);
cudaError_t tn_launch_energy(const DevMesh &m, const double *u, double *elem_energy,
                             double *layer_energy, cudaStream_t st);
// parts[3 e + j]: the dilatational, tetragonal and shear parts of element e's
// energy (one mesh, FP64)
cudaError_t tn_launch_energy_parts(const DevMesh &m, const double *u, double *parts, cudaStream_t st);
