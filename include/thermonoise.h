/*
 * thermonoise.h -- C ABI of the GB300 (sm_103a) library for the discontinuous
 * Galerkin model of Brownian coating thermal noise (arXiv 2111.06893).
 *
 * The library applies the matrix-free internal-penalty DG operator of static
 * linear elasticity (Sec. 2.2), solves it for the Gaussian-beam load
 * (Sec. 2.1, Eq. (laserbeam); Sec. 2.3, Eq. (matrix_eqn)), reduces the
 * solution to per-layer elastic energies (Sec. 2.1, potential energy and its
 * decomposition by layer) and evaluates the noise PSD (Eq. (thermalnoise)).
 *
 * Conventions shared by every entry point
 *   - Every function returns tn_status; TN_OK == 0, errors are negative.
 *     No exception crosses the ABI.  tn_last_error() returns a thread-local,
 *     NUL-terminated description of the last failure on the calling thread.
 *   - Arguments are validated before any GPU work (TN_EINVAL).
 *   - Pointers named *_dev are device pointers owned by the caller (for
 *     example a torch tensor's data_ptr); pointers named *_host are host
 *     memory owned by the caller.  The context owns the mesh, geometry and
 *     solver workspace it allocates and frees them in tn_destroy().
 *   - Work is queued on the context's CUDA stream (given to tn_create) and is
 *     asynchronous, except where a function returns host data (then it
 *     synchronises that stream before returning).
 *   - One context per host thread at a time.
 *
 * Field layout (all device vectors): element-major, component-blocked,
 *   u[(e * 3 + c) * N^3 + (k * N + j) * N + i],  N = degree + 1,
 * with (i, j, k) the LGL node indices along the element's logical axes
 * (xi, eta, zeta), c the Cartesian component (x, y, z).  Elements are
 * numbered e = s * n_columns + col: slab s counted from the top surface z = 0
 * downwards, col the cross-section column (box: col = jy * nx + ix;
 * cylinder: nine blocks [square, inner wedges at 0/90/180/270 degrees, outer
 * wedges at 0/90/180/270 degrees], col = block * k^2 + b * k + a inside a
 * block split k x k).
 */
#ifndef THERMONOISE_H
#define THERMONOISE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TN_OK = 0,
  TN_EINVAL = -1,     /* invalid argument; nothing was launched            */
  TN_ENOMEM = -2,     /* device or host allocation failed                  */
  TN_ECUDA = -3,      /* a CUDA call failed (text in tn_last_error)        */
  TN_ENOTCONV = -4,   /* iteration limit reached; best iterate returned    */
  TN_EBREAKDOWN = -5, /* Krylov breakdown (p.Ap <= 0 or not finite)        */
  TN_ETIMEOUT = -6,   /* a bounded device wait gave up                     */
  TN_ESTATE = -7      /* call out of order (e.g. no mesh built yet)        */
} tn_status;

enum { TN_MESH_BOX = 0, TN_MESH_CYLINDER = 1 };
enum { TN_BC_FREE = 0, TN_BC_FIXED = 1 };
enum { TN_F64 = 0, TN_F32 = 1 };
enum { TN_ISO = 0, TN_CUBIC = 1 };
enum { TN_SOLVE_F64 = 0, TN_SOLVE_MIXED_F32 = 1 };
enum { TN_PC_JACOBI = 0, TN_PC_ZLINE = 1, TN_PC_ZGROUP = 2 };

typedef struct tn_ctx tn_ctx;

/* Create a context on CUDA device `device`; all work goes to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * context.  Uploads the LGL tables to the device.  Returns TN_ECUDA if the
 * device cannot be used. */
tn_status tn_create(tn_ctx **out, int device, void *cuda_stream);
/* Free everything the context owns.  NULL is accepted. */
void tn_destroy(tn_ctx *ctx);
/* Text of the last failure on this thread ("" if none). */
const char *tn_last_error(void);

/* Mesh description (Sec. 2.2.1, Fig. 1).  The cross-section is a box split
 * along x and y, or a disk of radius R made of a central square [-a, a]^2,
 * four wedges from the square to the circle of radius R1 and four outer
 * wedges to R, each of the nine blocks split k x k.  Vertically the domain is
 * cut into n_slabs slabs listed from the top (slab_z[0] = 0) downwards; slab s
 * spans slab_z[s+1] < z < slab_z[s], belongs to layer slab_layer[s] and uses a
 * logarithmic map in depth -z if slab_log[s] != 0 (then slab_z[s] < 0).
 * Layer interfaces therefore coincide with element boundaries (Sec. 4).
 * The top z = 0 carries the beam pressure (Neumann, Eq. (bc)); the sides /
 * mantle and the bottom are TN_BC_FIXED (u = 0, Eq. (BCfixed)) or
 * TN_BC_FREE (zero traction, Eq. (BCfree)).  The penalty is
 * sigma = penalty_C (degree + 1)^2 / h (Eq. (penalty)).  degree in 2..8. */
typedef struct {
  int kind;                 /* TN_MESH_BOX or TN_MESH_CYLINDER             */
  int degree;               /* polynomial degree p; N = p + 1 LGL points   */
  int nx, ny;               /* box: elements along x and y                 */
  const double *x_breaks;   /* box: nx + 1 increasing x values (host)      */
  const double *y_breaks;   /* box: ny + 1 increasing y values (host)      */
  double R, a, R1;          /* cylinder radii, 0 < a < R1 < R              */
  int k;                    /* cylinder: k x k split of each block         */
  int n_slabs;              /* >= 1                                        */
  const double *slab_z;     /* n_slabs + 1 decreasing z values, [0] == 0   */
  const int *slab_layer;    /* n_slabs layer ids in [0, n_layers)          */
  const int *slab_log;      /* n_slabs flags                               */
  int n_layers;             /* coating layers + substrate                  */
  double penalty_C;         /* > 0                                         */
  int bc_side, bc_bottom;   /* TN_BC_FREE or TN_BC_FIXED                   */
} tn_mesh_desc;

/* Build the mesh and its geometry (FP64) on the device; replaces any earlier
 * mesh of the context.  Host arrays are copied; the caller keeps ownership. */
tn_status tn_build_mesh(tn_ctx *ctx, const tn_mesh_desc *desc);

/* Number of unknowns N_DOF = 3 * N^3 * n_elements (Sec. 2.3). */
tn_status tn_ndof(const tn_ctx *ctx, int64_t *ndof);

/* Material of each layer (Sec. 2.1): TN_ISO from Young's modulus Y and
 * Poisson ratio nu (Eq. (constrel_iso) and its footnote), or TN_CUBIC with
 * c11, c12, c44 and crystal axes along x, y, z (Eq. (constrel_cryst)).
 * n must equal the mesh's n_layers; layer n-1 is the substrate. */
typedef struct {
  int kind;
  double Y, nu;
  double c11, c12, c44;
} tn_material;
tn_status tn_set_materials(tn_ctx *ctx, int n, const tn_material *m);

/* The stiffness entries an isotropic material gets in tn_set_materials and
 * in the gradients of tn_energy_grad: c_host[3] = (c11, c12, c44) =
 * (lambda + 2 mu, lambda, mu) from Young's modulus Y and Poisson ratio nu
 * (the footnote to Eq. (constrel_iso), inverted), and, if dc_host is not
 * NULL, dc_host[2 q + 0] = d c_q / dY, dc_host[2 q + 1] = d c_q / dnu, so that
 * dJ/dY = sum_q dJ/dc_q dc_host[2 q].  Host only; TN_EINVAL unless Y > 0 and
 * -1 < nu < 1/2. */
tn_status tn_iso_moduli(double Y, double nu, double *c_host, double *dc_host);

/* Gaussian beam p(r) = F0 exp(-r^2/r0^2) / (pi r0^2) (Eq. (laserbeam)),
 * centred on the z axis. r0 > 0. */
tn_status tn_set_beam(tn_ctx *ctx, double r0, double F0);

/* y = A u: one application of the DG operator of Eq. (dg_residuals) (weak
 * form, homogeneous boundary data).  precision TN_F64: u, y are double;
 * TN_F32: float (geometry is kept in FP64 and rounded per node).  u and y
 * are caller-owned device buffers of tn_ndof() elements, must not overlap,
 * and must be 16-byte aligned. */
tn_status tn_apply_operator(tn_ctx *ctx, int precision, const void *u_dev, void *y_dev);

/* Autotuning of the FP32 operator kernel (the element-wise apply of
 * Eq. (dg_residuals)).  Two builds of it differ only in the resident CTAs
 * per SM asked of the register allocator: variant 0 gives every thread the
 * registers the code needs, variant 1 one CTA more per SM with fewer
 * registers per thread.  They execute the same arithmetic in the same
 * order, so results are bit-identical.  The first tn_apply_operator
 * (TN_F32) or mixed-mode tn_solve after a mesh or batch is built times both
 * for every degree present (3 + 10 launches of each, CUDA events on the
 * stream of the call, not while it is being captured; the call's y, or the
 * solver's FP32 workspace, is overwritten meanwhile) and keeps variant 1
 * only when it is faster by more than 2 %.
 * tn_apply_tuning: variant[p - 2] for p = 2..8 is 0 or 1 once settled, -1
 * before; us (may be NULL) receives 14 doubles, the time per launch in
 * microseconds of variants 0 and 1 for each degree (0 where not timed).
 * tn_set_apply_variant fixes the variant of one degree (0 or 1; the
 * autotuner then leaves it alone) or, with -1, lets it be timed again.
 * Building a mesh or batch resets both.  variant and us are caller-owned host
 * arrays; neither call touches the GPU.  TN_EINVAL for a null context or
 * variant array, a degree outside 2..8 or a variant outside -1..1. */
tn_status tn_apply_tuning(const tn_ctx *ctx, int *variant, double *us);
tn_status tn_set_apply_variant(tn_ctx *ctx, int degree, int variant);

/* b of A u = b (Eq. (matrix_eqn)) for the beam load: b = -sum over top-face
 * nodes of w^S J^S p(r) e_z (Neumann data of Eq. (bc)).  FP64, ndof values. */
tn_status tn_rhs(tn_ctx *ctx, double *b_dev);

/* diag(A) in FP64 (the Jacobi preconditioner). ndof values. */
tn_status tn_diagonal(tn_ctx *ctx, double *d_dev);

/* z = M^-1 r for a preconditioner of the Krylov solve (Sec. 2.3 accelerates
 * its solver; these preconditioners replace its multigrid/Schwarz):
 * TN_PC_JACOBI: M = diag(A).  TN_PC_ZLINE: M = the exact principal
 * sub-matrix of A on every vertical line of nodes (one cross-section node of
 * one column, all slabs, all nodes along zeta, three components), block
 * tridiagonal over the slabs, factorised by block Cholesky (FP64) and stored
 * in FP32 -- it captures the coupling across thin layers, whose elements
 * have aspect ratios up to ~1e4.  TN_PC_ZGROUP (one mesh or a batch): the
 * same with the lines that meet at one point of the cross-section (matching
 * nodes of the lateral faces of 2 to 4 neighbouring columns) taken together:
 * the exact principal sub-matrix of A on each such group of lines, which adds
 * the interior-penalty and flux coupling across the vertical element faces
 * (Eqs. (numflux), (penalty)) that single lines leave out; TN_EINVAL if a
 * node is shared by more than 4 columns.  The first call after
 * tn_build_mesh / tn_set_materials builds the factors (FP64 set-up, about
 * (3 g N)^2 / 2 + 3 g N (8 + 6 g) FP32 and FP64 entries per group of g
 * lines and slab).
 * precision TN_F64 / TN_F32 selects double / float vectors r, z
 * (caller-owned device buffers of tn_ndof() values, 16-byte aligned, not
 * overlapping). */
tn_status tn_precond_apply(tn_ctx *ctx, int precond, int precision, const void *r_dev, void *z_dev);
/* (tn_precond_apply is asynchronous: its staging waits use the 1 s default
 * of tn_solve_opts.device_wait_limit_s, and a wait that ran out leaves z
 * incomplete without an error code; tn_solve reports timeouts.) */

/* Bytes of FP32 factors one FP32 application of `precond` must read at
 * least (building the factors first if needed), for bandwidth accounting:
 * TN_PC_ZLINE the line records; TN_PC_ZGROUP the compact factors, S_s^-1
 * (packed symmetric) and the factored couplings O_s (the records' backward
 * couplings W_s, which derive from them, are not counted); TN_PC_JACOBI the
 * inverse diagonal.  *bytes: host. */
tn_status tn_precond_factor_bytes(tn_ctx *ctx, int precond, long long *bytes);

/* Krylov solve of A u = b for the beam load (Sec. 2.3).
 * precond: TN_PC_JACOBI, TN_PC_ZLINE or TN_PC_ZGROUP (see tn_precond_apply).
 * mode TN_SOLVE_F64: preconditioned CG in FP64, restarted from the current
 * iterate (true residual) if the recursive residual drifted.
 * mode TN_SOLVE_MIXED_F32: flexible CG in FP64 (residual, update and a window
 * of fcg_window previous directions kept A-orthogonal) preconditioned by an
 * inner PCG entirely in FP32 (vectors, operator, preconditioner), run to
 * inner_rtol or inner_max iterations on the normalised FP64 residual;
 * max_outer bounds the FP64 steps.
 * Stops when ||b - A u||_2 <= rtol ||b||_2 (FP64 residual), or by the energy
 * test of energy_rtol, or when the FP64 residual stagnates (thin layers put
 * its rounding floor near eps64 * cond(A)); u_dev holds the
 * initial guess on entry if use_x0 != 0 (else it starts from 0) and the FP64
 * solution on exit.  Returns TN_ENOTCONV with the best iterate if max_iter
 * (total inner iterations) is reached. */
typedef struct {
  int mode;
  int precond;
  double rtol;
  double inner_rtol;
  int max_iter;
  int max_outer;
  int use_x0;
  int check_every;          /* iterations between host convergence checks */
  int inner_max;            /* mixed: FP32 PCG iterations per outer step (0: 40 with TN_PC_ZGROUP, else 300) */
  int fcg_window;           /* mixed: directions kept by the flexible CG (0 or max: 16) */
  double energy_rtol;       /* > 0: also stop once every layer energy U_i
                               changes by <= energy_rtol (relative) between
                               two checks (refinement steps, or check_every
                               FP64 iterations); 0: residual test only     */
  double device_wait_limit_s; /* bound on every device-side wait of the line
                               solves (a staged factor copy landing in shared
                               memory), in seconds of the GPU's global timer;
                               0: 1 s.  A wait that runs out ends its kernel
                               (after a bounded wait for its copies still in
                               flight), the solve stops at the next check and
                               returns TN_ETIMEOUT, which outranks every other
                               outcome; the context stays usable.  [0, 3600] */
} tn_solve_opts;
typedef struct {
  int status;
  int outer_iters;
  int inner_iters;
  int applies_f64;
  int applies_f32;
  int64_t launches;         /* kernel launches issued by this call         */
  double rel_residual;
  double energy_change;     /* last max_i |dU_i / U_i| (energy test only)  */
  double seconds;
} tn_solve_report;
tn_status tn_solve(tn_ctx *ctx, const tn_solve_opts *opts, double *u_dev, tn_solve_report *rep);

/* Per-layer elastic energy U_i = 1/2 sum_{e in layer i} sum_p w_p detJ_p
 * S_p : Y : S_p with S = sym grad u at the element's own nodes (Sec. 2.1,
 * U = -1/2 int S_ij T^ij dV, T = -Y S).  u_dev: FP64 field; U_host receives
 * n_layers doubles (coating layers top-down, substrate last).  Synchronises. */
tn_status tn_layer_energies(tn_ctx *ctx, const double *u_dev, double *U_host);

/* The layer energies of tn_layer_energies split by elastic modulus, for a
 * noise PSD with a separate loss angle per modulus (Sec. 2.1: a material can
 * carry different loss angles for its independent moduli; the split is this
 * library's reading).  The energy density 1/2 S : Y : S of the cubic-aligned
 * stiffness separates along its eigen-modes (T = tr S, D = sum_i S_ii^2,
 * O = S_xy^2 + S_xz^2 + S_yz^2):
 *   parts[3 L + 0]  dilatational  1/2 (c11 + 2 c12) / 3 T^2   (bulk modulus)
 *   parts[3 L + 1]  tetragonal    1/2 (c11 - c12) (D - T^2 / 3)
 *   parts[3 L + 2]  shear         1/2 4 c44 O
 * each integrated like tn_layer_energies (element LGL nodes, unlifted
 * strain); the three sum to U_L.  Isotropic layers: part 0 is the bulk
 * energy K/2 int T^2, parts 1 + 2 the shear energy mu int S_dev : S_dev.
 * One mesh or a batch (layers concatenated mirror by mirror).  u_dev: FP64
 * field; parts_host: 3 * n_layers doubles.  Allocates a scratch of
 * 3 * n_elements doubles for the call.  Synchronises. */
tn_status tn_layer_energy_parts(tn_ctx *ctx, const double *u_dev, double *parts_host);

/* Adjoint gradient of J = sum_i w_i U_i (energies of tn_layer_energies) for
 * the solution u of A u = b (caller-owned FP64 device buffer, e.g. from
 * tn_solve).  Because the weak-form operator is symmetric the adjoint
 * A lambda = g, g = dJ/du = sum_i w_i K_i u (K_i the energy matrix of layer
 * i), is solved with the same operator, preconditioner and solver (opts;
 * energy_rtol is ignored).  Then, for every parameter theta,
 *   dJ/dtheta = 1/2 u^T (sum_i w_i dK_i/dtheta) u + lambda^T (db/dtheta - dA/dtheta u),
 * with dA/dtheta u and dK_i/dtheta formed exactly by forward-mode (dual
 * number) versions of the operator and energy kernels.  Parameters:
 *   dJ_dslab_z[n_slabs + 1]  slab boundary positions slab_z[s] (the top,
 *                            s = 0, is held at z = 0 and returns 0);
 *                            layer thicknesses follow by the chain rule
 *   dJ_dr0[1]                beam width r0 (only b depends on it)
 *   dJ_dmat[3 n_layers]      c11, c12, c44 of every layer (isotropic layers:
 *                            c11 = lambda + 2 mu, c12 = lambda, c44 = mu)
 * w_host: n_layers weights (host).  lambda_dev: optional ndof FP64 device
 * buffer receiving the adjoint solution (NULL: internal).  All outputs are
 * host arrays.  Returns the adjoint solve's status (TN_ENOTCONV keeps the
 * gradients of the best adjoint iterate).  Synchronises. */
tn_status tn_energy_grad(tn_ctx *ctx, const tn_solve_opts *opts, const double *u_dev, const double *w_host,
                         double *lambda_dev, double *dJ_dslab_z, double *dJ_dr0, double *dJ_dmat,
                         tn_solve_report *rep);

/* Batches (a design sweep): many independent mirrors of uneven polynomial
 * degree and element count held by one context.  tn_batch_create(n) replaces
 * any mesh of the context by n empty slots; tn_batch_set fills slot i with a
 * mesh (as tn_build_mesh), its materials (as tn_set_materials) and its beam
 * (as tn_set_beam).  Once every slot is set the context holds the batch:
 *   - unknowns are concatenated mirror by mirror (each in the field layout
 *     above); tn_batch_offsets gives the first unknown and the first layer of
 *     every mirror (n + 1 entries each) and tn_ndof the total;
 *   - tn_apply_operator applies the block-diagonal operator of all mirrors:
 *     one launch per polynomial degree present, each CTA working on one
 *     element of one mirror;
 *   - tn_precond_apply (TN_PC_ZLINE, TN_PC_ZGROUP) and tn_solve solve all mirrors at
 *     once (one Krylov iteration serves every mirror; the energy test covers
 *     every layer of every mirror);
 *   - tn_layer_energies returns the energies of all layers of all mirrors.
 * tn_diagonal and TN_PC_JACOBI need a single mesh; gradients of a batch
 * come from tn_batch_energy_grad. */
tn_status tn_batch_create(tn_ctx *ctx, int n_instances);
tn_status tn_batch_set(tn_ctx *ctx, int instance, const tn_mesh_desc *desc, int n_materials,
                       const tn_material *m, double r0, double F0);
tn_status tn_batch_offsets(const tn_ctx *ctx, int64_t *dof_off, int *layer_off);
/* tn_energy_grad for every mirror of a batch at once: one batched adjoint
 * solve, then the per-mirror contractions.  w_host: weights of all layers
 * (concatenated like the energies); outputs concatenated mirror by mirror:
 * dJ_dslab_z[sum_i (n_slabs_i + 1)], dJ_dr0[n], dJ_dmat[3 * all layers]. */
tn_status tn_batch_energy_grad(tn_ctx *ctx, const tn_solve_opts *opts, const double *u_dev, const double *w_host,
                               double *lambda_dev, double *dJ_dslab_z, double *dJ_dr0, double *dJ_dmat,
                               tn_solve_report *rep);

/* tn_layer_energies for callers that cannot allocate device memory at the
 * time of the call (a process that reserves its HBM budget up front, or one
 * that must avoid the device-wide synchronisation an allocation or a free can
 * cause).  The paper has no counterpart: this is a library convenience.  It
 * allocates nothing: its scratch (per-element energies and per-layer sums) is
 * a fixed array in the library's device image, which every GPU that loads
 * the library holds until exit.  Limits: a single mesh of at most 65536
 * elements and 1024 layers (TN_EINVAL otherwise).  Its first call on a device
 * looks up the array's device address (cudaGetSymbolAddress); make that first
 * call before any stream capture.  All calls share the array: calls that
 * overlap on the GPU race.  Each call writes every scratch entry it reads, so
 * no clearing is needed.  u_dev: FP64 field; U_host: n_layers doubles.
 * Synchronises the context's stream. */
tn_status tn_layer_energies_noalloc(tn_ctx *ctx, const double *u_dev, double *U_host);

/* The approximate coating thermal noise of a thin isotropic coating on a
 * semi-infinite isotropic mirror, Eq. (approx_analytic) (coating
 * contribution; valid for d << r0, r0 << R): the reference of the
 * finite-size study (Sec. 3.2), to which the solved
 * S_q = 4 kB_T phi_c U_coat / (pi f F0^2) (tn_noise_psd) is compared.
 *   S = kB_T / (pi^2 f) (1 - nus^2) / (r0 Ys) (d / r0)
 *       phi_c / (Ys Yc (1 - nuc^2)(1 - nus^2))
 *       [Yc^2 (1 + nus)^2 (1 - 2 nus)^2 + Ys^2 (1 + nuc)^2 (1 - 2 nuc)]
 * Substrate (Ys, nus), coating (Yc, nuc), thickness d, beam width r0, loss
 * angle phi_c.  Host only; TN_EINVAL for non-positive scales or
 * nu outside (-1, 1/2). */
tn_status tn_thin_coating_psd(double kB_T, double f, double r0, double d, double Ys, double nus, double Yc,
                              double nuc, double phi_c, double *S_out);

/* Measured fused-multiply-add peak of the CUDA cores of `device` in
 * precision TN_F32 or TN_F64 (flop/s, an FMA counted as 2): the roofline
 * denominator of the operator apply, which is bound by arithmetic, not HBM
 * (no counterpart in the paper).  Independent FMA chains in registers on
 * 4 CTAs of 512 threads per SM, CUDA events around 5 launches after a
 * warm-up, at whatever clocks the GPU runs (none are set).  Takes ~0.1 s.
 * *flops_per_s: host.  TN_EINVAL for a bad device or precision. */
tn_status tn_fma_peak(int device, int precision, double *flops_per_s);

/* Brownian noise PSD from the energies (Eq. (thermalnoise) with Eq. (wdiss)
 * per layer, dissipated power 2 pi f sum_i phi_i U_i):
 *   S_out = 4 kB_T sum_i phi_i U_i / (pi f F0^2).  Host only. */
tn_status tn_noise_psd(const double *U_host, const double *phi_host, int n, double kB_T,
                       double f, double F0, double *S_out);

#ifdef __cplusplus
}
#endif
#endif /* THERMONOISE_H */
