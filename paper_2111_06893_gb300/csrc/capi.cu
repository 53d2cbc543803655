// C ABI of the thermonoise library (declared in include/thermonoise.h):
// context and workspace management, argument validation, and the host-side
// orchestration of the solve, energies and PSD.
#include <chrono>
#include <cmath>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <algorithm>
#include <vector>

#include "tn_internal.h"
#include "tn_precond.h"
#include "tn_solver.h"

namespace {
thread_local char g_err[512] = "";

tn_status fail(tn_status st, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

tn_status cuda_fail(cudaError_t e, const char *where) {
  return fail(TN_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CU_TRY(call, where)                          \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

template <typename T>
void dfree(T *&p) {
  if (p) cudaFree((void *)p);
  p = nullptr;
}
}  // namespace

// one mirror of a batch: its own mesh tables and material table on the device
struct BatchInst {
  tn::HostMesh hm;
  DevMesh dm{};
  double *colgeo = nullptr, *slabgeo = nullptr, *layer_c = nullptr;
  float *colgeo32 = nullptr, *slabgeo32 = nullptr, *layer_c32 = nullptr;
  int *colnb = nullptr, *colnbf = nullptr, *slab_layer = nullptr;
  double r0 = 1.0, F0 = 1.0;
  long long dof_off = 0, fac_off = 0;
  int layer_off = 0;
  bool set = false;
  std::vector<double> slab_z;
  std::vector<int> slab_log;
};

struct Batch {
  int n = 0;
  BatchInst *inst = nullptr;
  bool ready = false;
  long long ndof = 0, nfac = 0;
  int n_layers = 0, n_elems = 0;
  DevMesh *d_meshes = nullptr;
  long long *d_dof_off = nullptr, *d_fac_off = nullptr;
  int2 *d_work = nullptr, *d_lines = nullptr;
  OpSys sys;
  int2 *h_work = nullptr;  // (instance, element) in the order of the apply partials
};

struct tn_ctx {
  int device = 0;
  Batch *batch = nullptr;
  cudaStream_t stream = nullptr;   // the caller's stream
  cudaStream_t sstream = nullptr;  // internal stream used for graph capture
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  tn::HostMesh hm;
  bool have_mesh = false, have_mat = false, have_beam = false;
  DevMesh dm{};
  double *d_colgeo = nullptr, *d_slabgeo = nullptr, *d_layer_c = nullptr;
  int *d_colnb = nullptr, *d_colnbf = nullptr, *d_slab_layer = nullptr;
  float *d_colgeo32 = nullptr, *d_slabgeo32 = nullptr, *d_layer_c32 = nullptr;
  double *slab_z_host = nullptr;
  int *slab_log_host = nullptr;
  double r0 = 1.0, F0 = 1.0;
  size_t ndof = 0;
  // workspace
  size_t ws_ndof = 0;
  double *b64 = nullptr, *diag64 = nullptr, *dinv64 = nullptr, *r64 = nullptr, *z64 = nullptr,
         *p64 = nullptr, *q64 = nullptr;
  float *dinv32 = nullptr, *b32 = nullptr, *r32 = nullptr, *z32 = nullptr, *p32 = nullptr,
        *q32 = nullptr, *d32 = nullptr;
  double *part_elem = nullptr, *part_red = nullptr, *sum_dev = nullptr;
  tn_pcg_scalars *scal = nullptr, *scal_host = nullptr;
  double *elem_energy = nullptr, *layer_energy = nullptr;
  // flexible-CG window (mixed mode)
  double *fcg = nullptr;
  const double **fcg_ptrs = nullptr;   // device: [16] P, [16] AP, [2] pair
  double *fcg_beta = nullptr;
  double *fcg_part = nullptr;
  double *fcg_host = nullptr;          // host tmp for partial sums
  int fcg_m = 0;
  size_t ws_E = 0;
  int ws_layers = 0;
  // z-line preconditioner (valid while mesh and materials are unchanged)
  float *zfac = nullptr;
  double *zfac64 = nullptr;
  double *zpart = nullptr;
  int *zstatus = nullptr;
  bool zready = false;
  // grouped-line preconditioner (same validity)
  ZGroupPlan gplan;
  ZGroupDev zgd;
  int4 *d_glines = nullptr;
  long long *d_gfac_off = nullptr;
  int *d_ginst = nullptr;
  int4 *d_gpacks = nullptr;
  int *d_gqueue = nullptr;
  float *gfac = nullptr;
  double *gfac64 = nullptr;
  double *gpart = nullptr;
  int *gstatus = nullptr;
  bool gready = false;
  // FP32 operator kernel, per LGL count N (index N): the occupancy variant in
  // use, whether it is settled (timed, or fixed by the caller), and the time
  // per launch measured for variants 0 and 1; reset with the mesh
  int apply_var[10] = {0};
  bool apply_set[10] = {false};
  float apply_us[10][2] = {};
  // bounded device waits of the line solves (limit and timeout flag)
  TnWait *wctl = nullptr;
  // counters of the PCG scalar steps folded into the grouped-line iteration
  unsigned *fold_cnt = nullptr;
};

static void free_zline(tn_ctx *c) {
  dfree(c->zfac);
  dfree(c->zfac64);
  dfree(c->zpart);
  dfree(c->zstatus);
  c->zready = false;
}

static void free_zgroup(tn_ctx *c) {
  dfree(c->d_glines);
  dfree(c->d_gfac_off);
  dfree(c->d_ginst);
  dfree(c->d_gpacks);
  dfree(c->d_gqueue);
  dfree(c->gfac);
  dfree(c->gfac64);
  dfree(c->gpart);
  dfree(c->gstatus);
  for (int g = 0; g < kZgSide; ++g) {
    if (c->zgd.side[g]) cudaStreamDestroy(c->zgd.side[g]);
    if (c->zgd.join[g]) cudaEventDestroy(c->zgd.join[g]);
  }
  if (c->zgd.fork) cudaEventDestroy(c->zgd.fork);
  c->zgd = ZGroupDev();
  c->gready = false;
}

static void free_precond(tn_ctx *c) {
  free_zline(c);
  free_zgroup(c);
}

static OpSys make_sys(const tn_ctx *c);
static int total_layers(const tn_ctx *c);
static int apply_parts(const tn_ctx *c);
static bool is_batch(const tn_ctx *c);

static void reset_tuning(tn_ctx *c) {
  for (int N = 0; N < 10; ++N) {
    c->apply_var[N] = 0;
    c->apply_set[N] = false;
    c->apply_us[N][0] = c->apply_us[N][1] = 0.0f;
  }
}

static void free_mesh(tn_ctx *c) {
  free_precond(c);
  reset_tuning(c);
  dfree(c->d_colgeo);
  dfree(c->d_slabgeo);
  dfree(c->d_colnb);
  dfree(c->d_colnbf);
  dfree(c->d_slab_layer);
  dfree(c->d_colgeo32);
  dfree(c->d_slabgeo32);
  tn::free_host_mesh(&c->hm);
  std::free(c->slab_z_host);
  std::free(c->slab_log_host);
  c->slab_z_host = nullptr;
  c->slab_log_host = nullptr;
  c->have_mesh = false;
}

static void free_ws(tn_ctx *c) {
  dfree(c->b64); dfree(c->diag64); dfree(c->dinv64); dfree(c->r64); dfree(c->z64); dfree(c->p64);
  dfree(c->q64); dfree(c->dinv32); dfree(c->b32); dfree(c->r32); dfree(c->z32); dfree(c->p32);
  dfree(c->q32); dfree(c->d32);
  dfree(c->part_elem); dfree(c->part_red); dfree(c->sum_dev); dfree(c->scal);
  dfree(c->elem_energy); dfree(c->layer_energy);
  dfree(c->fcg); dfree(c->fcg_ptrs); dfree(c->fcg_beta); dfree(c->fcg_part);
  std::free(c->fcg_host);
  c->fcg_host = nullptr;
  c->fcg_m = 0;
  if (c->scal_host) cudaFreeHost(c->scal_host);
  c->scal_host = nullptr;
  c->ws_ndof = 0;
  c->ws_E = 0;
  c->ws_layers = 0;
}

static tn_status ensure_ws(tn_ctx *c) {
  const int E = apply_parts(c), NL = total_layers(c);
  if (c->ws_ndof == c->ndof && c->ws_E == (size_t)E && c->ws_layers == NL) return TN_OK;
  free_ws(c);
  const size_t n = c->ndof;
  const size_t d8 = n * sizeof(double), f4 = n * sizeof(float);
  cudaError_t e = cudaSuccess;
  auto A = [&](void **p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
  A((void **)&c->b64, d8); A((void **)&c->diag64, d8); A((void **)&c->dinv64, d8);
  A((void **)&c->r64, d8); A((void **)&c->z64, d8); A((void **)&c->p64, d8); A((void **)&c->q64, d8);
  A((void **)&c->dinv32, f4); A((void **)&c->b32, f4); A((void **)&c->r32, f4); A((void **)&c->z32, f4);
  A((void **)&c->p32, f4); A((void **)&c->q32, f4); A((void **)&c->d32, f4);
  A((void **)&c->part_elem, sizeof(double) * E);
  A((void **)&c->part_red, sizeof(double) * 2 * tn::reduction_blocks());
  A((void **)&c->sum_dev, sizeof(double) * 2);
  A((void **)&c->scal, sizeof(tn_pcg_scalars));
  A((void **)&c->elem_energy, sizeof(double) * E);
  A((void **)&c->layer_energy, sizeof(double) * NL);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&c->scal_host, sizeof(tn_pcg_scalars));
  if (e != cudaSuccess) {
    free_ws(c);
    cudaGetLastError();
    return fail(TN_ENOMEM, "workspace allocation of %zu DOF failed: %s", n, cudaGetErrorString(e));
  }
  c->ws_ndof = n;
  c->ws_E = E;
  c->ws_layers = NL;
  return TN_OK;
}

static tn_status ensure_fcg(tn_ctx *c, int m) {
  if (c->fcg_m == m) return TN_OK;
  dfree(c->fcg); dfree(c->fcg_ptrs); dfree(c->fcg_beta); dfree(c->fcg_part);
  std::free(c->fcg_host);
  c->fcg_host = nullptr;
  c->fcg_m = 0;
  const size_t n = c->ndof;
  const int nb = tn::reduction_blocks();
  cudaError_t e = cudaMalloc((void **)&c->fcg, sizeof(double) * n * 2 * m);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->fcg_ptrs, sizeof(double *) * 34);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->fcg_beta, sizeof(double) * 16);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->fcg_part, sizeof(double) * 16 * nb);
  c->fcg_host = (double *)std::malloc(sizeof(double) * 16 * nb);
  if (e != cudaSuccess || !c->fcg_host) {
    cudaGetLastError();
    return fail(TN_ENOMEM, "flexible CG window of %d directions", m);
  }
  const double *ptrs[32];
  for (int j = 0; j < m; ++j) {
    ptrs[j] = c->fcg + (size_t)j * n;            // P_j
    ptrs[16 + j] = c->fcg + (size_t)(m + j) * n;  // AP_j
  }
  e = cudaMemcpy(c->fcg_ptrs, ptrs, sizeof(ptrs), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "fcg pointers");
  c->fcg_m = m;
  return TN_OK;
}

// builds the z-line factors on stream st (temporary FP64 blocks freed after)
static tn_status ensure_zline(tn_ctx *c, cudaStream_t st) {
  if (c->zready) return TN_OK;
  free_zline(c);
  size_t bb = 0, fb = 0;
  int nparts = 0;
  if (is_batch(c)) {
    for (int i = 0; i < c->batch->n; ++i) {
      const size_t b1 = tn_zline_block_bytes(c->batch->inst[i].dm);
      bb = b1 > bb ? b1 : bb;
    }
    fb = (size_t)c->batch->nfac * sizeof(float);
    nparts = c->batch->sys.n_rz_parts;
  } else {
    bb = tn_zline_block_bytes(c->dm);
    fb = tn_zline_factor_bytes(c->dm);
    nparts = tn_zline_partials(c->dm);
  }
  double *blk = nullptr;
  cudaError_t e = cudaMalloc((void **)&blk, bb);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->zfac, fb);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->zfac64, 2 * fb);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->zpart, sizeof(double) * 2 * nparts);  // r.z, r.r
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->zstatus, 2 * sizeof(int));  // factor status, solve timeout
  if (e != cudaSuccess) {
    if (blk) cudaFree(blk);
    free_precond(c);
    cudaGetLastError();
    return fail(TN_ENOMEM, "z-line preconditioner needs %.2f GB: %s", (bb + 3 * fb) / 1e9, cudaGetErrorString(e));
  }
  int status = 0;
  e = cudaMemsetAsync(c->zstatus, 0, 2 * sizeof(int), st);
  if (!is_batch(c)) {
    if (e == cudaSuccess) e = tn_zline_setup(c->dm, blk, c->zfac, c->zfac64, c->zstatus, st);
  } else {
    for (int i = 0; i < c->batch->n && e == cudaSuccess; ++i) {
      const BatchInst &q = c->batch->inst[i];
      e = tn_zline_setup(q.dm, blk, c->zfac + q.fac_off, c->zfac64 + q.fac_off, c->zstatus, st);
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, c->zstatus, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(blk);
  if (e != cudaSuccess) return cuda_fail(e, "z-line set-up");
  if (status) return fail(TN_EBREAKDOWN, "z-line block not positive definite");
  c->zready = true;
  return TN_OK;
}

// builds the grouped-line factors (one mesh, or every mirror of a batch) on
// stream st; the FP64 set-up blocks and scratch are freed after
static tn_status ensure_zgroup(tn_ctx *c, cudaStream_t st) {
  if (c->gready) return TN_OK;
  free_zgroup(c);
  const int n = is_batch(c) ? c->batch->n : 1;
  std::vector<const tn::HostMesh *> hms(n);
  std::vector<DevMesh> dms(n);
  for (int i = 0; i < n; ++i) {
    hms[i] = is_batch(c) ? &c->batch->inst[i].hm : &c->hm;
    dms[i] = is_batch(c) ? c->batch->inst[i].dm : c->dm;
  }
  char msg[160];
  if (!tn_zgroup_plan(hms.data(), n, &c->gplan, msg, sizeof(msg))) return fail(TN_EINVAL, "%s", msg);
  const ZGroupPlan &p = c->gplan;
  size_t bb = 0, xb = 0, wb = 0;
  for (int i = 0; i < n; ++i) {
    const size_t b1 = tn_zline_block_bytes(dms[i]), x1 = tn_zgroup_cross_bytes(dms[i]),
                 w1 = tn_zgroup_work_bytes(dms[i], p, i);
    bb = b1 > bb ? b1 : bb;
    xb = x1 > xb ? x1 : xb;
    wb = w1 > wb ? w1 : wb;
  }
  const size_t fb = (size_t)p.nfac * sizeof(float);
  double *blk = nullptr, *xblk = nullptr, *work = nullptr;
  cudaError_t e = cudaMalloc((void **)&blk, bb);
  if (e == cudaSuccess) e = cudaMalloc((void **)&xblk, xb);
  if (e == cudaSuccess) e = cudaMalloc((void **)&work, wb);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->gfac, fb);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->gfac64, 2 * fb);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->gpart, sizeof(double) * 2 * p.ngroups);  // r.z, r.r
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->gstatus, 2 * sizeof(int));  // factor status, solve timeout
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_glines, sizeof(int4) * p.ngroups);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_gfac_off, sizeof(long long) * p.ngroups);
  if (e == cudaSuccess && is_batch(c)) e = cudaMalloc((void **)&c->d_ginst, sizeof(int) * p.ngroups);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_gpacks, sizeof(int4) * p.packs.size());
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_gqueue, sizeof(int) * 2 * kZgMaxPk);
  if (e != cudaSuccess) {
    dfree(blk); dfree(xblk); dfree(work);
    free_zgroup(c);
    cudaGetLastError();
    return fail(TN_ENOMEM, "grouped-line preconditioner needs %.2f GB: %s", (bb + xb + wb + 3 * fb) / 1e9,
                cudaGetErrorString(e));
  }
  ZGroupDev &g = c->zgd;
  for (int k = 0; k < kZgSide && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&g.side[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.join[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.fork, cudaEventDisableTiming);
  g.lines = c->d_glines;
  g.fac_off = c->d_gfac_off;
  g.inst = is_batch(c) ? c->d_ginst : nullptr;
  g.meshes = is_batch(c) ? c->batch->d_meshes : nullptr;
  g.dof_off = is_batch(c) ? c->batch->d_dof_off : nullptr;
  g.ndof = (long long)c->ndof;
  g.ngroups = p.ngroups;
  g.ncls = p.ncls;
  for (int k = 0; k < p.ncls; ++k) {
    g.cls_N[k] = p.cls_N[k]; g.cls_G[k] = p.cls_G[k]; g.cls_start[k] = p.cls_start[k]; g.cls_n[k] = p.cls_n[k];
  }
  g.packs = c->d_gpacks;
  g.queue = c->d_gqueue;
  g.npk = p.npk;
  for (int k = 0; k < p.npk; ++k) { g.pk_N[k] = p.pk_N[k]; g.pk_start[k] = p.pk_start[k]; g.pk_n[k] = p.pk_n[k]; }
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_gpacks, p.packs.data(), sizeof(int4) * p.packs.size(),
                                            cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_gqueue, 0, sizeof(int) * 2 * kZgMaxPk, st);
  int status = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_glines, p.lines.data(), sizeof(int4) * p.ngroups,
                                            cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_gfac_off, p.fac_off.data(), sizeof(long long) * p.ngroups,
                                            cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && is_batch(c))
    e = cudaMemcpyAsync(c->d_ginst, p.inst.data(), sizeof(int) * p.ngroups, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->gstatus, 0, 2 * sizeof(int), st);
  for (int i = 0; i < n && e == cudaSuccess; ++i)  // one mirror after another (shared set-up scratch)
    e = tn_zgroup_setup(dms[i], p, c->zgd, i, c->d_glines, c->d_gfac_off, blk, xblk, work, c->gfac, c->gfac64,
                        c->gstatus, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, c->gstatus, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dfree(blk); dfree(xblk); dfree(work);
  if (e != cudaSuccess) { free_zgroup(c); return cuda_fail(e, "grouped-line set-up"); }
  if (status) { free_zgroup(c); return fail(TN_EBREAKDOWN, "grouped-line block not positive definite"); }
  c->gready = true;
  return TN_OK;
}

// the operator system with the grouped-line solve in place of the single lines
static OpSys with_groups(OpSys s, const tn_ctx *c) {
  s.grouped = true;
  s.fold_cnt = c->fold_cnt;
  s.zg = c->zgd;
  s.n_rz_parts = c->zgd.ngroups;
  s.zerr = c->wctl;
  return s;
}

// per-layer energies of u (all mirrors of a batch, concatenated) into host out
static cudaError_t energies_host(tn_ctx *c, const double *u, double *out, cudaStream_t st) {
  if (!is_batch(c)) {
    cudaError_t e = tn_launch_energy(c->dm, u, c->elem_energy, c->layer_energy, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out, c->layer_energy, sizeof(double) * c->dm.n_layers, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
  }
  Batch *b = c->batch;
  const OpSys &s = b->sys;
  cudaError_t e = cudaSuccess;
  for (int g = 0; g < s.ngroups && e == cudaSuccess; ++g)
    e = tn_launch_energy_batch(s.gN[g], b->d_meshes, s.gwork[g], s.gcount[g], b->d_dof_off, u,
                               c->elem_energy + s.gpart_off[g], st);
  double *tmp = (double *)std::malloc(sizeof(double) * b->n_elems);
  if (!tmp) return cudaErrorMemoryAllocation;
  if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, c->elem_energy, sizeof(double) * b->n_elems, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) {
    for (int l = 0; l < b->n_layers; ++l) out[l] = 0.0;
    // fixed order: the order of the work list
    for (int w = 0; w < b->n_elems; ++w) {
      const int2 it = b->h_work[w];
      const BatchInst &q = b->inst[it.x];
      out[q.layer_off + q.hm.slab_layer[it.y / q.hm.ncol]] += tmp[w];
    }
  }
  std::free(tmp);
  return e;
}

// energies of the current iterate and their largest relative change since the
// previous call (for the energy stopping test)
struct EnergyTrack {
  tn_ctx *c;
  const double *u;
  cudaStream_t st;
  double tol;
  std::vector<double> prev = std::vector<double>(65536), cur = std::vector<double>(65536);
  bool have_prev = false;
  double change = INFINITY;
  cudaError_t err = cudaSuccess;
  bool step() {
    const int nl = total_layers(c);
    err = energies_host(c, u, cur.data(), st);
    if (err != cudaSuccess) return true;
    bool ok = have_prev;
    double ch = 0.0;
    for (int i = 0; i < nl && have_prev; ++i) {
      const double d = std::fabs(cur[i] - prev[i]) / std::fabs(cur[i]);
      ch = d > ch ? d : ch;
    }
    if (have_prev) change = ch;
    for (int i = 0; i < nl; ++i) prev[i] = cur[i];
    have_prev = true;
    return ok && change <= tol;
  }
  static bool hook(void *self) { return static_cast<EnergyTrack *>(self)->step(); }
};

static void free_batch(tn_ctx *c) {
  Batch *b = c->batch;
  if (!b) return;
  for (int i = 0; i < b->n; ++i) {
    BatchInst &q = b->inst[i];
    dfree(q.colgeo); dfree(q.slabgeo); dfree(q.layer_c); dfree(q.colgeo32); dfree(q.slabgeo32);
    dfree(q.layer_c32); dfree(q.colnb); dfree(q.colnbf); dfree(q.slab_layer);
    tn::free_host_mesh(&q.hm);
  }
  delete[] b->inst;
  dfree(b->d_meshes); dfree(b->d_dof_off); dfree(b->d_fac_off); dfree(b->d_work); dfree(b->d_lines);
  delete[] b->h_work;
  delete b;
  c->batch = nullptr;
}

static bool is_batch(const tn_ctx *c) { return c->batch != nullptr; }

static OpSys make_sys(const tn_ctx *c) {
  OpSys s;
  if (is_batch(c)) {
    s = c->batch->sys;
    for (int g = 0; g < s.ngroups; ++g) s.gvar[g] = c->apply_var[s.gN[g]];
  } else {
    s.m = &c->dm;
    s.mvar = c->apply_var[c->dm.N];
    s.n_apply_parts = c->dm.E;
    s.n_rz_parts = tn_zline_partials(c->dm);
  }
  s.zerr = c->wctl;
  return s;
}

// Autotuner of the FP32 operator kernel: for every LGL count of the context
// (the mesh, or each degree group of a batch) not yet settled, times both
// occupancy variants on the vectors u -> y (y is overwritten) and keeps
// variant 1 only when it is faster by more than 2 %.  Nothing is timed while
// st is being captured into a graph.
static tn_status ensure_tuned(tn_ctx *c, const float *u, float *y, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CU_TRY(cudaStreamIsCapturing(st, &cs), "capture status");
  if (cs != cudaStreamCaptureStatusNone) return TN_OK;
  const bool batch = is_batch(c);
  const OpSys s = make_sys(c);
  const int ng = batch ? s.ngroups : 1;
  for (int g = 0; g < ng; ++g) {
    const int N = batch ? s.gN[g] : c->dm.N;
    if (N < 3 || N > 9 || c->apply_set[N]) continue;
    float us[2] = {0.0f, 0.0f};
    if (batch)
      CU_TRY(tn_tune_apply(nullptr, N, s.meshes, s.gwork[g], s.gcount[g], s.dof_off, u, y, st, us), "tuning");
    else
      CU_TRY(tn_tune_apply(&c->dm, N, nullptr, nullptr, 0, nullptr, u, y, st, us), "tuning");
    c->apply_us[N][0] = us[0];
    c->apply_us[N][1] = us[1];
    c->apply_var[N] = us[1] < 0.98f * us[0] ? 1 : 0;
    c->apply_set[N] = true;
  }
  return TN_OK;
}

static int total_layers(const tn_ctx *c) { return is_batch(c) ? c->batch->n_layers : c->dm.n_layers; }
static int apply_parts(const tn_ctx *c) { return is_batch(c) ? c->batch->n_elems : c->dm.E; }

// b of every mirror (beam load)
static cudaError_t make_rhs(const tn_ctx *c, double *b, cudaStream_t st) {
  if (!is_batch(c)) return tn_launch_rhs(c->dm, c->r0, c->F0, b, st);
  for (int i = 0; i < c->batch->n; ++i) {
    const BatchInst &q = c->batch->inst[i];
    cudaError_t e = tn_launch_rhs(q.dm, q.r0, q.F0, b + q.dof_off, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static tn_status need_ready(const tn_ctx *c, bool beam) {
  if (!c) return fail(TN_EINVAL, "null context");
  if (c->batch) {
    if (!c->batch->ready) return fail(TN_ESTATE, "batch not finalised: set every instance first");
    return TN_OK;
  }
  if (!c->have_mesh) return fail(TN_ESTATE, "no mesh: call tn_build_mesh first");
  if (!c->have_mat) return fail(TN_ESTATE, "no materials: call tn_set_materials after tn_build_mesh");
  if (beam && !c->have_beam) return fail(TN_ESTATE, "no beam: call tn_set_beam first");
  return TN_OK;
}

extern "C" {

const char *tn_last_error(void) { return g_err; }

tn_status tn_create(tn_ctx **out, int device, void *cuda_stream) {
  if (!out) return fail(TN_EINVAL, "out is null");
  *out = nullptr;
  int count = 0;
  CU_TRY(cudaGetDeviceCount(&count), "cudaGetDeviceCount");
  if (device < 0 || device >= count) return fail(TN_EINVAL, "device %d out of range (%d devices)", device, count);
  CU_TRY(cudaSetDevice(device), "cudaSetDevice");
  tn_ctx *c = new (std::nothrow) tn_ctx();
  if (!c) return fail(TN_ENOMEM, "host allocation failed");
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaStreamCreateWithFlags(&c->sstream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->wctl, sizeof(TnWait));
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->fold_cnt, 2 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(c->fold_cnt, 0, 2 * sizeof(unsigned));
  if (e == cudaSuccess) {
    const TnWait w0{kDefaultWaitNs, 0, 0};
    e = cudaMemcpy(c->wctl, &w0, sizeof(w0), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) {
    static LglTables tabs;
    std::memset(&tabs, 0, sizeof(tabs));
    for (int N = 2; N <= TN_MAX_N; ++N) {
      double D[TN_MAX_N * TN_MAX_N];
      tn::lgl(N, tabs.x[N], tabs.w[N], D);
      std::memcpy(tabs.D[N], D, sizeof(double) * N * N);
    }
    e = tn_upload_lgl(&tabs);
    if (e == cudaSuccess) e = tn_upload_lgl_precond(&tabs);
  }
  if (e != cudaSuccess) {
    tn_destroy(c);
    return cuda_fail(e, "tn_create");
  }
  *out = c;
  return TN_OK;
}

void tn_destroy(tn_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  free_ws(c);
  free_mesh(c);
  free_batch(c);
  dfree(c->d_layer_c);
  dfree(c->d_layer_c32);
  dfree(c->wctl);
  dfree(c->fold_cnt);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->sstream) cudaStreamDestroy(c->sstream);
  delete c;
}

tn_status tn_build_mesh(tn_ctx *c, const tn_mesh_desc *d) {
  if (!c || !d) return fail(TN_EINVAL, "null argument");
  tn::HostMesh hm;
  char msg[256] = "";
  tn_status st = tn::build_host_mesh(d, &hm, msg, sizeof(msg));
  if (st != TN_OK) return fail(st, "tn_build_mesh: %s", msg);
  CU_TRY(cudaSetDevice(c->device), "cudaSetDevice");
  CU_TRY(cudaStreamSynchronize(c->stream), "sync before rebuilding the mesh");
  free_mesh(c);
  free_batch(c);
  free_ws(c);
  dfree(c->d_layer_c);
  dfree(c->d_layer_c32);
  c->have_mat = false;
  c->hm = hm;
  const int N2 = hm.N * hm.N;
  cudaError_t e = cudaSuccess;
  auto up = [&](void **dst, const void *src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(dst, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  };
  up((void **)&c->d_colgeo, hm.colgeo, sizeof(double) * (size_t)hm.ncol * CG_NF * N2);
  up((void **)&c->d_slabgeo, hm.slabgeo, sizeof(double) * (size_t)hm.nslab * SG_NF * hm.N);
  up((void **)&c->d_colnb, hm.colnb, sizeof(int) * 4 * hm.ncol);
  up((void **)&c->d_colnbf, hm.colnbf, sizeof(int) * 4 * hm.ncol);
  up((void **)&c->d_slab_layer, hm.slab_layer, sizeof(int) * hm.nslab);
  {
    const size_t ncg = (size_t)hm.ncol * CG_NF * N2, nsg = (size_t)hm.nslab * SG_NF * hm.N;
    float *f32 = (float *)std::malloc(sizeof(float) * (ncg > nsg ? ncg : nsg));
    if (!f32) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess) {
      for (size_t q = 0; q < ncg; ++q) f32[q] = (float)hm.colgeo[q];
      up((void **)&c->d_colgeo32, f32, sizeof(float) * ncg);
    }
    if (e == cudaSuccess) {
      for (size_t q = 0; q < nsg; ++q) f32[q] = (float)hm.slabgeo[q];
      up((void **)&c->d_slabgeo32, f32, sizeof(float) * nsg);
    }
    std::free(f32);
  }
  if (e != cudaSuccess) {
    free_mesh(c);
    return cuda_fail(e, "uploading the mesh");
  }
  c->slab_z_host = (double *)std::malloc(sizeof(double) * (hm.nslab + 1));
  c->slab_log_host = (int *)std::malloc(sizeof(int) * hm.nslab);
  if (!c->slab_z_host || !c->slab_log_host) {
    free_mesh(c);
    return fail(TN_ENOMEM, "host allocation failed");
  }
  std::memcpy(c->slab_z_host, d->slab_z, sizeof(double) * (hm.nslab + 1));
  std::memcpy(c->slab_log_host, d->slab_log, sizeof(int) * hm.nslab);
  DevMesh &m = c->dm;
  m.N = hm.N; m.p = hm.p; m.E = hm.E; m.ncol = hm.ncol; m.nslab = hm.nslab; m.n_layers = hm.n_layers;
  m.bc_side = hm.bc_side; m.bc_bottom = hm.bc_bottom; m.penC = hm.penC;
  m.colgeo = c->d_colgeo; m.slabgeo = c->d_slabgeo; m.colnb = c->d_colnb; m.colnbf = c->d_colnbf;
  m.slab_layer = c->d_slab_layer; m.layer_c = nullptr;
  m.colgeo32 = c->d_colgeo32; m.slabgeo32 = c->d_slabgeo32; m.layer_c32 = nullptr;
  m.penC32 = (float)hm.penC;
  c->ndof = (size_t)3 * hm.N * hm.N * hm.N * hm.E;
  c->have_mesh = true;
  return TN_OK;
}

tn_status tn_ndof(const tn_ctx *c, int64_t *ndof) {
  if (!c || !ndof) return fail(TN_EINVAL, "null argument");
  if (c->batch ? !c->batch->ready : !c->have_mesh) return fail(TN_ESTATE, "no mesh");
  *ndof = (int64_t)c->ndof;
  return TN_OK;
}

// (c11, c12, c44) = (lambda + 2 mu, lambda, mu) of an isotropic material and
// their derivatives d/dY, d/dnu (footnote to Eq. (constrel_iso) inverted:
// mu = Y / (2 (1 + nu)), lambda = Y nu / ((1 + nu)(1 - 2 nu)))
static void iso_moduli(double Y, double nu, double c[3], double dc[6]) {
  const double mu = Y / (2.0 * (1.0 + nu));
  const double g = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), lam = Y * g;
  c[0] = lam + 2.0 * mu; c[1] = lam; c[2] = mu;
  if (!dc) return;
  const double dmu_dY = 1.0 / (2.0 * (1.0 + nu)), dmu_dnu = -Y / (2.0 * (1.0 + nu) * (1.0 + nu));
  const double q = (1.0 + nu) * (1.0 - 2.0 * nu);
  const double dlam_dY = g, dlam_dnu = Y * (1.0 + 2.0 * nu * nu) / (q * q);
  dc[0] = dlam_dY + 2.0 * dmu_dY; dc[1] = dlam_dnu + 2.0 * dmu_dnu;
  dc[2] = dlam_dY;                dc[3] = dlam_dnu;
  dc[4] = dmu_dY;                 dc[5] = dmu_dnu;
}

// (c11, c12, c44) per layer from the ABI materials; false + message on error
static bool material_table(int n, const tn_material *mats, double *h, char *msg, int len) {
  for (int i = 0; i < n; ++i) {
    const tn_material &m = mats[i];
    if (m.kind == TN_ISO) {
      if (!(m.Y > 0.0) || !(m.nu > -1.0 && m.nu < 0.5)) {
        std::snprintf(msg, len, "material %d: need Y > 0 and -1 < nu < 1/2", i);
        return false;
      }
      iso_moduli(m.Y, m.nu, h + 3 * i, nullptr);
    } else if (m.kind == TN_CUBIC) {
      if (!(m.c44 > 0.0) || !(m.c11 > std::fabs(m.c12)) || !(m.c11 + 2.0 * m.c12 > 0.0)) {
        std::snprintf(msg, len, "material %d: cubic stiffness not positive definite", i);
        return false;
      }
      h[3 * i] = m.c11; h[3 * i + 1] = m.c12; h[3 * i + 2] = m.c44;
    } else {
      std::snprintf(msg, len, "material %d: unknown kind %d", i, m.kind);
      return false;
    }
  }
  return true;
}

tn_status tn_set_materials(tn_ctx *c, int n, const tn_material *mats) {
  if (!c || !mats) return fail(TN_EINVAL, "null argument");
  if (c->batch) return fail(TN_ESTATE, "the context holds a batch: use tn_batch_set");
  if (!c->have_mesh) return fail(TN_ESTATE, "no mesh: call tn_build_mesh first");
  if (n != c->hm.n_layers) return fail(TN_EINVAL, "got %d materials for %d layers", n, c->hm.n_layers);
  double *h = (double *)std::malloc(sizeof(double) * 3 * n);
  if (!h) return fail(TN_ENOMEM, "host allocation failed");
  char msg[160];
  if (!material_table(n, mats, h, msg, sizeof(msg))) {  // the same table as a batch mirror gets
    std::free(h);
    return fail(TN_EINVAL, "%s", msg);
  }
  CU_TRY(cudaSetDevice(c->device), "cudaSetDevice");
  CU_TRY(cudaStreamSynchronize(c->stream), "sync before replacing materials");
  dfree(c->d_layer_c);
  dfree(c->d_layer_c32);
  float h32[3 * 4096];
  if (n > 4096) { std::free(h); return fail(TN_EINVAL, "at most 4096 layers"); }
  for (int i = 0; i < 3 * n; ++i) h32[i] = (float)h[i];
  cudaError_t e = cudaMalloc((void **)&c->d_layer_c, sizeof(double) * 3 * n);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_layer_c, h, sizeof(double) * 3 * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_layer_c32, sizeof(float) * 3 * n);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_layer_c32, h32, sizeof(float) * 3 * n, cudaMemcpyHostToDevice);
  std::free(h);
  if (e != cudaSuccess) return cuda_fail(e, "uploading materials");
  c->dm.layer_c = c->d_layer_c;
  c->dm.layer_c32 = c->d_layer_c32;
  c->have_mat = true;
  free_precond(c);
  return TN_OK;
}

tn_status tn_set_beam(tn_ctx *c, double r0, double F0) {
  if (!c) return fail(TN_EINVAL, "null context");
  if (!(r0 > 0.0) || !std::isfinite(F0)) return fail(TN_EINVAL, "need r0 > 0 and finite F0");
  c->r0 = r0;
  c->F0 = F0;
  c->have_beam = true;
  return TN_OK;
}

// ---------------------------------------------------------------- batches

static tn_status batch_finalize(tn_ctx *c) {
  Batch *b = c->batch;
  long long dof = 0, fac = 0;
  int lay = 0, elems = 0;
  for (int i = 0; i < b->n; ++i) {
    BatchInst &q = b->inst[i];
    q.dof_off = dof;
    q.fac_off = fac;
    q.layer_off = lay;
    const long long M = 3LL * q.hm.N;
    dof += 3LL * q.hm.N * q.hm.N * q.hm.N * q.hm.E;
    fac += (long long)tn_zline_factor_entries(q.dm);
    (void)M;
    lay += q.hm.n_layers;
    elems += q.hm.E;
  }
  b->ndof = dof; b->nfac = fac; b->n_layers = lay; b->n_elems = elems;
  std::vector<int2> work, lines;
  OpSys &s = b->sys;
  s = OpSys();
  int rz = 0;
  for (int N = TN_MIN_N; N <= TN_MAX_N; ++N) {
    const int w0 = (int)work.size(), l0 = (int)lines.size();
    for (int i = 0; i < b->n; ++i) {
      const BatchInst &q = b->inst[i];
      if (q.hm.N != N) continue;
      for (int e = 0; e < q.hm.E; ++e) work.push_back(make_int2(i, e));
      for (int l = 0; l < q.hm.ncol * N * N; ++l) lines.push_back(make_int2(i, l));
    }
    if ((int)work.size() == w0) continue;
    const int g = s.ngroups++;
    s.gN[g] = N;
    s.gcount[g] = (int)work.size() - w0;
    s.gpart_off[g] = w0;
    s.glines[g] = (int)lines.size() - l0;
    s.grz_off[g] = rz;
    rz += (s.glines[g] + 3) / 4;
    s.gwork[g] = reinterpret_cast<const int2 *>((size_t)w0);   // offsets, fixed below
    s.gline[g] = reinterpret_cast<const int2 *>((size_t)l0);
  }
  std::vector<DevMesh> dms(b->n);
  std::vector<long long> doff(b->n + 1), foff(b->n);
  for (int i = 0; i < b->n; ++i) { dms[i] = b->inst[i].dm; doff[i] = b->inst[i].dof_off; foff[i] = b->inst[i].fac_off; }
  doff[b->n] = b->ndof;  // the last entry closes the last mirror (per-mirror norms)
  cudaError_t e = cudaSuccess;
  auto up = [&](void **dst, const void *src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(dst, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  };
  up((void **)&b->d_meshes, dms.data(), sizeof(DevMesh) * b->n);
  up((void **)&b->d_dof_off, doff.data(), sizeof(long long) * (b->n + 1));
  up((void **)&b->d_fac_off, foff.data(), sizeof(long long) * b->n);
  up((void **)&b->d_work, work.data(), sizeof(int2) * work.size());
  up((void **)&b->d_lines, lines.data(), sizeof(int2) * lines.size());
  if (e != cudaSuccess) return cuda_fail(e, "uploading the batch");
  for (int g = 0; g < s.ngroups; ++g) {
    s.gwork[g] = b->d_work + (size_t)s.gwork[g];
    s.gline[g] = b->d_lines + (size_t)s.gline[g];
  }
  s.meshes = b->d_meshes;
  s.dof_off = b->d_dof_off;
  s.fac_off = b->d_fac_off;
  s.n_apply_parts = elems;
  s.n_rz_parts = rz;
  b->h_work = new (std::nothrow) int2[work.size()];
  if (!b->h_work) return fail(TN_ENOMEM, "host allocation failed");
  std::memcpy(b->h_work, work.data(), sizeof(int2) * work.size());
  c->ndof = (size_t)dof;
  b->ready = true;
  return TN_OK;
}

extern "C" {

tn_status tn_batch_create(tn_ctx *c, int n) {
  if (!c) return fail(TN_EINVAL, "null context");
  if (n < 1 || n > 65536) return fail(TN_EINVAL, "need 1 <= n <= 65536 instances");
  CU_TRY(cudaSetDevice(c->device), "cudaSetDevice");
  CU_TRY(cudaStreamSynchronize(c->stream), "sync before replacing the mesh");
  free_mesh(c);
  free_batch(c);
  free_ws(c);
  dfree(c->d_layer_c);
  dfree(c->d_layer_c32);
  c->have_mat = false;
  Batch *b = new (std::nothrow) Batch();
  if (b) b->inst = new (std::nothrow) BatchInst[n];
  if (!b || !b->inst) { delete b; return fail(TN_ENOMEM, "host allocation failed"); }
  b->n = n;
  c->batch = b;
  c->ndof = 0;
  return TN_OK;
}

tn_status tn_batch_set(tn_ctx *c, int i, const tn_mesh_desc *d, int n_mat, const tn_material *mats, double r0,
                       double F0) {
  if (!c || !d || !mats) return fail(TN_EINVAL, "null argument");
  if (!c->batch) return fail(TN_ESTATE, "no batch: call tn_batch_create first");
  Batch *b = c->batch;
  if (i < 0 || i >= b->n) return fail(TN_EINVAL, "instance %d out of range", i);
  if (b->inst[i].set) return fail(TN_ESTATE, "instance %d already set", i);
  if (!(r0 > 0.0) || !std::isfinite(F0)) return fail(TN_EINVAL, "need r0 > 0 and finite F0");
  tn::HostMesh hm;
  char msg[256] = "";
  tn_status st = tn::build_host_mesh(d, &hm, msg, sizeof(msg));
  if (st != TN_OK) return fail(st, "instance %d: %s", i, msg);
  if (n_mat != hm.n_layers) { tn::free_host_mesh(&hm); return fail(TN_EINVAL, "instance %d: %d materials for %d layers", i, n_mat, hm.n_layers); }
  std::vector<double> h(3 * n_mat);
  if (!material_table(n_mat, mats, h.data(), msg, sizeof(msg))) { tn::free_host_mesh(&hm); return fail(TN_EINVAL, "instance %d: %s", i, msg); }
  std::vector<float> h32(h.begin(), h.end());
  CU_TRY(cudaSetDevice(c->device), "cudaSetDevice");
  BatchInst &q = b->inst[i];
  q.hm = hm;
  const int N2 = hm.N * hm.N;
  const size_t ncg = (size_t)hm.ncol * CG_NF * N2, nsg = (size_t)hm.nslab * SG_NF * hm.N;
  std::vector<float> cg32(hm.colgeo, hm.colgeo + ncg), sg32(hm.slabgeo, hm.slabgeo + nsg);
  cudaError_t e = cudaSuccess;
  auto up = [&](void **dst, const void *src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(dst, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  };
  up((void **)&q.colgeo, hm.colgeo, sizeof(double) * ncg);
  up((void **)&q.slabgeo, hm.slabgeo, sizeof(double) * nsg);
  up((void **)&q.colgeo32, cg32.data(), sizeof(float) * ncg);
  up((void **)&q.slabgeo32, sg32.data(), sizeof(float) * nsg);
  up((void **)&q.colnb, hm.colnb, sizeof(int) * 4 * hm.ncol);
  up((void **)&q.colnbf, hm.colnbf, sizeof(int) * 4 * hm.ncol);
  up((void **)&q.slab_layer, hm.slab_layer, sizeof(int) * hm.nslab);
  up((void **)&q.layer_c, h.data(), sizeof(double) * h.size());
  up((void **)&q.layer_c32, h32.data(), sizeof(float) * h32.size());
  if (e != cudaSuccess) return cuda_fail(e, "uploading a batch instance");
  DevMesh &m = q.dm;
  m.N = hm.N; m.p = hm.p; m.E = hm.E; m.ncol = hm.ncol; m.nslab = hm.nslab; m.n_layers = hm.n_layers;
  m.bc_side = hm.bc_side; m.bc_bottom = hm.bc_bottom; m.penC = hm.penC; m.penC32 = (float)hm.penC;
  m.colgeo = q.colgeo; m.slabgeo = q.slabgeo; m.colnb = q.colnb; m.colnbf = q.colnbf; m.slab_layer = q.slab_layer;
  m.layer_c = q.layer_c; m.colgeo32 = q.colgeo32; m.slabgeo32 = q.slabgeo32; m.layer_c32 = q.layer_c32;
  q.r0 = r0;
  q.F0 = F0;
  q.slab_z.assign(d->slab_z, d->slab_z + hm.nslab + 1);
  q.slab_log.assign(d->slab_log, d->slab_log + hm.nslab);
  q.set = true;
  for (int k = 0; k < b->n; ++k)
    if (!b->inst[k].set) return TN_OK;
  return batch_finalize(c);
}

tn_status tn_batch_offsets(const tn_ctx *c, int64_t *dof_off, int *layer_off) {
  if (!c || !dof_off || !layer_off) return fail(TN_EINVAL, "null argument");
  if (!c->batch || !c->batch->ready) return fail(TN_ESTATE, "no finalised batch");
  const Batch *b = c->batch;
  for (int i = 0; i < b->n; ++i) { dof_off[i] = b->inst[i].dof_off; layer_off[i] = b->inst[i].layer_off; }
  dof_off[b->n] = b->ndof;
  layer_off[b->n] = b->n_layers;
  return TN_OK;
}

}  // extern "C"

static tn_status check_buf(const tn_ctx *c, const void *p, size_t elem, const char *name) {
  if (!p) return fail(TN_EINVAL, "%s is null", name);
  if (((uintptr_t)p) % 16) return fail(TN_EINVAL, "%s must be 16-byte aligned", name);
  (void)c; (void)elem;
  return TN_OK;
}

tn_status tn_apply_operator(tn_ctx *c, int precision, const void *u, void *y) {
  tn_status st = need_ready(c, false);
  if (st) return st;
  if (precision != TN_F64 && precision != TN_F32) return fail(TN_EINVAL, "precision must be TN_F64 or TN_F32");
  const size_t es = precision == TN_F64 ? 8 : 4;
  if ((st = check_buf(c, u, es, "u"))) return st;
  if ((st = check_buf(c, y, es, "y"))) return st;
  const char *a = (const char *)u, *b = (const char *)y;
  const size_t bytes = c->ndof * es;
  if (a < b + bytes && b < a + bytes) return fail(TN_EINVAL, "u and y overlap");
  if (precision == TN_F32 && (st = ensure_tuned(c, (const float *)u, (float *)y, c->stream))) return st;
  CU_TRY(make_sys(c).apply(precision, u, y, nullptr, c->stream), "apply launch");
  return TN_OK;
}

tn_status tn_apply_tuning(const tn_ctx *c, int *variant, double *us) {
  if (!c || !variant) return fail(TN_EINVAL, "null argument");
  for (int p = 2; p <= 8; ++p) {
    const int N = p + 1;
    variant[p - 2] = c->apply_set[N] ? c->apply_var[N] : -1;
    if (us) {
      us[2 * (p - 2)] = c->apply_us[N][0];
      us[2 * (p - 2) + 1] = c->apply_us[N][1];
    }
  }
  return TN_OK;
}

tn_status tn_set_apply_variant(tn_ctx *c, int degree, int variant) {
  if (!c) return fail(TN_EINVAL, "null context");
  if (degree < 2 || degree > 8) return fail(TN_EINVAL, "degree must be in 2..8");
  if (variant < -1 || variant > 1) return fail(TN_EINVAL, "variant must be -1, 0 or 1");
  const int N = degree + 1;
  c->apply_var[N] = variant < 0 ? 0 : variant;
  c->apply_set[N] = variant >= 0;
  c->apply_us[N][0] = c->apply_us[N][1] = 0.0f;
  return TN_OK;
}

tn_status tn_rhs(tn_ctx *c, double *b) {
  tn_status st = need_ready(c, true);
  if (st) return st;
  if ((st = check_buf(c, b, 8, "b"))) return st;
  CU_TRY(make_rhs(c, b, c->stream), "rhs launch");
  return TN_OK;
}

tn_status tn_diagonal(tn_ctx *c, double *d) {
  tn_status st = need_ready(c, false);
  if (st) return st;
  if (is_batch(c)) return fail(TN_EINVAL, "tn_diagonal works on a single mesh");
  if ((st = check_buf(c, d, 8, "d"))) return st;
  CU_TRY(tn_launch_diag(c->dm, d, c->stream), "diag launch");
  return TN_OK;
}

static tn_status solve_impl(tn_ctx *c, const tn_solve_opts *o, const double *rhs, double *u,
                            tn_solve_report *rep);

tn_status tn_solve(tn_ctx *c, const tn_solve_opts *o, double *u, tn_solve_report *rep) {
  tn_status st = need_ready(c, true);
  if (st) return st;
  return solve_impl(c, o, nullptr, u, rep);
}

// A u = rhs (rhs == nullptr: the beam load); u, rhs device FP64
static tn_status solve_impl(tn_ctx *c, const tn_solve_opts *o, const double *rhs, double *u,
                            tn_solve_report *rep) {
  tn_status st = TN_OK;
  if (!o) return fail(TN_EINVAL, "opts is null");
  if ((st = check_buf(c, u, 8, "u"))) return st;
  if (o->mode != TN_SOLVE_F64 && o->mode != TN_SOLVE_MIXED_F32) return fail(TN_EINVAL, "unknown solve mode");
  if (o->precond != TN_PC_JACOBI && o->precond != TN_PC_ZLINE && o->precond != TN_PC_ZGROUP)
    return fail(TN_EINVAL, "unknown preconditioner");
  if (is_batch(c) && o->precond == TN_PC_JACOBI) return fail(TN_EINVAL, "a batch is solved with line blocks");
  if (!(o->rtol > 0.0) || !(o->rtol < 1.0)) return fail(TN_EINVAL, "rtol must be in (0, 1)");
  if (o->max_iter < 1) return fail(TN_EINVAL, "max_iter must be >= 1");
  if (!(o->energy_rtol >= 0.0)) return fail(TN_EINVAL, "energy_rtol must be >= 0");
  if (!(o->device_wait_limit_s >= 0.0) || !(o->device_wait_limit_s <= 3600.0))
    return fail(TN_EINVAL, "device_wait_limit_s must be in [0, 3600]");
  if (total_layers(c) > 65536) return fail(TN_EINVAL, "at most 65536 layers in all");
  if (o->mode == TN_SOLVE_MIXED_F32 && (!(o->inner_rtol > 0.0) || !(o->inner_rtol < 1.0) || o->max_outer < 1))
    return fail(TN_EINVAL, "mixed mode needs 0 < inner_rtol < 1 and max_outer >= 1");
  CU_TRY(cudaSetDevice(c->device), "cudaSetDevice");
  if ((st = ensure_ws(c))) return st;
  const int chunk = o->check_every > 0 ? o->check_every : 25;
  const auto t0 = std::chrono::steady_clock::now();
  tn::g_launches = 2;  // rhs and diagonal below
  tn::g_timed_out = false;
  cudaStream_t s = c->sstream;
  CU_TRY(cudaEventRecord(c->ev_in, c->stream), "event");
  CU_TRY(cudaStreamWaitEvent(s, c->ev_in, 0), "event wait");
  const size_t n = c->ndof;
  if (rhs) CU_TRY(cudaMemcpyAsync(c->b64, rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, s), "rhs copy");
  else CU_TRY(make_rhs(c, c->b64, s), "rhs");
  if (!is_batch(c)) CU_TRY(tn_launch_diag(c->dm, c->diag64, s), "diag");
  double bb = 0.0;
  CU_TRY(tn::norm2_f64(n, c->b64, c->part_red, c->sum_dev, &bb, s), "norm b");
  // a batch is converged when every mirror is: the relative residual is the
  // largest over the mirrors of |r_i| / |b_i| (mirrors with b_i = 0 aside)
  std::vector<double> bbi, rri;
  double *seg_dev = nullptr;
  struct SegFree {
    double *&p;
    ~SegFree() { if (p) cudaFree(p); }
  } seg_free{seg_dev};
  if (is_batch(c)) {
    const int nb = c->batch->n;
    bbi.resize(nb);
    rri.resize(nb);
    CU_TRY(cudaMalloc((void **)&seg_dev, sizeof(double) * nb), "per-mirror norms");
    CU_TRY(tn::segnorm2_f64(nb, c->batch->d_dof_off, c->b64, seg_dev, bbi.data(), s), "norm b per mirror");
  }
  // relative residual of r64 (|r|^2 = rr overall)
  auto rel_res = [&](double rr, cudaError_t *err) {
    *err = cudaSuccess;
    if (bbi.empty()) return std::sqrt(rr / bb);
    *err = tn::segnorm2_f64((int)bbi.size(), c->batch->d_dof_off, c->r64, seg_dev, rri.data(), s);
    double mx = 0.0;
    for (size_t i = 0; i < bbi.size(); ++i)
      if (bbi[i] > 0.0) mx = std::max(mx, std::sqrt(rri[i] / bbi[i]));
    return std::isfinite(rr) ? mx : rr;
  };
  cudaError_t rerr = cudaSuccess;
  const bool zg = o->precond == TN_PC_ZGROUP;
  const bool zl = o->precond == TN_PC_ZLINE || zg;  // a line-type solve (single or grouped lines)
  if (zg) {
    tn_status zs = ensure_zgroup(c, s);
    if (zs != TN_OK) return zs;
  } else if (zl) {
    tn_status zs = ensure_zline(c, s);
    if (zs != TN_OK) return zs;
  }
  // this solve's wait limit, timeout flag cleared (pageable source: copied
  // before the call returns)
  const TnWait wset{o->device_wait_limit_s > 0.0 ? (unsigned long long)(o->device_wait_limit_s * 1e9 + 0.5)
                                                 : kDefaultWaitNs, 0, 0};
  CU_TRY(cudaMemcpyAsync(c->wctl, &wset, sizeof(wset), cudaMemcpyHostToDevice, s), "wait limit");
  const OpSys sys = zg ? with_groups(make_sys(c), c) : make_sys(c);
  float *const lfac = zg ? c->gfac : c->zfac;
  double *const lfac64 = zg ? c->gfac64 : c->zfac64;
  double *const lpart = zg ? c->gpart : c->zpart;
  tn_solve_report r{};
  tn_status result = TN_OK;
  if (bb == 0.0) {
    CU_TRY(tn::fill_f64(n, u, 0.0, s), "zero");
  } else if (o->mode == TN_SOLVE_F64) {
    if (!is_batch(c)) CU_TRY(tn::pcg_setup_dinv(n, c->diag64, c->dinv64, TN_F64, s), "dinv");
    PcgVectors v{u, c->r64, c->z64, c->p64, c->q64, c->b64, c->dinv64};
    if (zl) { v.zfac = lfac64; v.part_rz = lpart; }
    // FP64 PCG; restarted from the current iterate (true residual) if the
    // recursively updated residual drifted away from b - A x
    bool x0_zero = o->use_x0 == 0;
    EnergyTrack et{c, u, s, o->energy_rtol};
    ChunkHook hook;
    if (o->energy_rtol > 0.0) { hook.fn = &EnergyTrack::hook; hook.user = &et; }
    bool energy_done = false;
    for (int restart = 0; restart < 4 && !energy_done; ++restart) {
      int applies = 0;
      CU_TRY(tn::pcg_f64(sys, n, v, x0_zero, o->rtol, o->max_iter - r.inner_iters, chunk, c->scal,
                         c->scal_host, c->part_elem, c->part_red, s, &applies, hook), "pcg f64");
      CU_TRY(et.err, "energy check");
      energy_done = o->energy_rtol > 0.0 && et.have_prev && et.change <= o->energy_rtol;
      r.energy_change = et.change;
      r.inner_iters += c->scal_host->iters;
      r.outer_iters += 1;
      r.applies_f64 += applies;
      if (tn::g_timed_out) break;
      if (c->scal_host->breakdown) {
        result = fail(TN_EBREAKDOWN, "CG breakdown after %d iterations", r.inner_iters);
        break;
      }
      double rr = 0.0;
      CU_TRY(tn::residual_f64(sys, n, c->b64, u, c->q64, c->r64, c->part_red, c->sum_dev, &rr, s), "residual");
      r.applies_f64 += 1;
      double rel = rel_res(rr, &rerr);
      CU_TRY(rerr, "norm r per mirror");
      if (energy_done || rel <= o->rtol || r.inner_iters >= o->max_iter) break;
      x0_zero = false;
    }
    r.status = energy_done ? 1 : 0;
  } else {
    if ((st = ensure_tuned(c, c->p32, c->q32, s))) return st;
    if (!is_batch(c)) CU_TRY(tn::pcg_setup_dinv(n, c->diag64, c->dinv32, TN_F32, s), "dinv32");
    const int m = o->fcg_window > 0 ? (o->fcg_window > 16 ? 16 : o->fcg_window) : 16;
    // default inner length: grouped lines reach the energy test fastest with
    // short inner runs (the flexible CG keeps the directions across them)
    const int kin = o->inner_max > 0 ? o->inner_max : (o->precond == TN_PC_ZGROUP ? 40 : 300);
    if ((st = ensure_fcg(c, m))) return st;
    double *P0 = c->fcg, *AP0 = c->fcg + (size_t)m * n;
    // r = b - A x
    if (!o->use_x0) {
      CU_TRY(tn::fill_f64(n, u, 0.0, s), "zero");
      CU_TRY(cudaMemcpyAsync(c->r64, c->b64, n * sizeof(double), cudaMemcpyDeviceToDevice, s), "r = b");
    } else {
      double rr0;
      CU_TRY(tn::residual_f64(sys, n, c->b64, u, c->q64, c->r64, c->part_red, c->sum_dev, &rr0, s), "residual");
      r.applies_f64 += 1;
    }
    int total_inner = 0;
    EnergyTrack et{c, u, s, o->energy_rtol};
    double best = INFINITY, pAp[16];
    int stall = 0, replaced = 0;
    bool energy_done = false;
    for (int k = 0; k < o->max_outer; ++k) {
      double rr = 0.0;
      CU_TRY(tn::norm2_f64(n, c->r64, c->part_red, c->sum_dev, &rr, s), "norm r");
      r.rel_residual = rel_res(rr, &rerr);
      CU_TRY(rerr, "norm r per mirror");
      if (!std::isfinite(rr)) { result = fail(TN_EBREAKDOWN, "non-finite residual"); break; }
      if (r.rel_residual <= o->rtol) {
        // the updated residual drifts from b - A u; confirm on the true one
        // and carry on from it (a few times at most) while it is above rtol
        CU_TRY(tn::residual_f64(sys, n, c->b64, u, c->q64, c->r64, c->part_red, c->sum_dev, &rr, s),
               "residual");
        r.applies_f64 += 1;
        r.rel_residual = rel_res(rr, &rerr);
        CU_TRY(rerr, "norm r per mirror");
        if (r.rel_residual <= o->rtol || ++replaced > 3) break;
        best = r.rel_residual;
        stall = 0;
      }
      if (o->energy_rtol > 0.0 && k > 0) {
        energy_done = et.step();
        CU_TRY(et.err, "energy check");
        r.energy_change = et.change;
        if (energy_done) break;
      }
      if (r.rel_residual < 0.5 * best) { best = r.rel_residual; stall = 0; }
      else if (++stall >= 30) break;  // FP64 rounding floor reached
      if (total_inner >= o->max_iter) break;
      // inner FP32 PCG on A d = r / |r|
      const double rn = std::sqrt(rr);
      CU_TRY(tn::cast_scaled(n, c->r64, 1.0 / rn, c->b32, c->d32, s), "cast");
      PcgVectors v{c->d32, c->r32, c->z32, c->p32, c->q32, c->b32, c->dinv32};
      if (zl) { v.zfac = lfac; v.part_rz = lpart; }
      int applies = 0;
      CU_TRY(tn::pcg_f32(sys, n, v, true, o->inner_rtol, kin, kin, c->scal, c->scal_host, c->part_elem,
                         c->part_red, s, &applies), "pcg f32");
      total_inner += c->scal_host->iters;
      r.applies_f32 += applies;
      if (tn::g_timed_out) break;
      r.outer_iters += 1;
      // z = |r| d (FP64), q = A z
      CU_TRY(tn::upcast(n, c->d32, rn, c->z64, s), "upcast");
      CU_TRY(sys.apply(TN_F64, c->z64, c->q64, nullptr, s), "apply f64");
      tn::g_launches += 1;
      r.applies_f64 += 1;
      // keep the new direction A-orthogonal to the last nb ones
      const int nb = k < m ? k : m, slot = k % m;
      double beta[16];
      if (nb > 0) {
        double zAp[16];
        CU_TRY(tn::multidot(n, c->z64, c->fcg_ptrs + 16, nb, c->fcg_part, c->fcg_host, zAp, s), "dots");
        for (int j = 0; j < nb; ++j) beta[j] = zAp[j] / pAp[j];
        CU_TRY(cudaMemcpyAsync(c->fcg_beta, beta, sizeof(double) * nb, cudaMemcpyHostToDevice, s), "beta");
      }
      CU_TRY(tn::fcg_orth(n, c->z64, c->q64, c->fcg_ptrs, c->fcg_ptrs + 16, c->fcg_beta, nb,
                          P0 + (size_t)slot * n, AP0 + (size_t)slot * n, s), "orth");
      const double *pair[2] = {c->r64, AP0 + (size_t)slot * n};
      CU_TRY(cudaMemcpyAsync(c->fcg_ptrs + 32, pair, sizeof(pair), cudaMemcpyHostToDevice, s), "pair");
      double d2[2];
      CU_TRY(tn::multidot(n, P0 + (size_t)slot * n, c->fcg_ptrs + 32, 2, c->fcg_part, c->fcg_host, d2, s), "dots");
      if (!(d2[1] > 0.0)) { result = fail(TN_EBREAKDOWN, "flexible CG breakdown (p.Ap = %g)", d2[1]); break; }
      pAp[slot] = d2[1];
      CU_TRY(tn::fcg_step(n, d2[0] / d2[1], P0 + (size_t)slot * n, AP0 + (size_t)slot * n, u, c->r64, s), "step");
    }
    r.inner_iters = total_inner;
    r.status = energy_done ? 1 : 0;
  }
  // true FP64 residual of the returned iterate
  const bool energy_ok = r.status == 1;
  r.status = 0;
  if (bb != 0.0 && result == TN_OK && !tn::g_timed_out) {
    double rr = 0.0;
    CU_TRY(tn::residual_f64(sys, n, c->b64, u, c->q64, c->r64, c->part_red, c->sum_dev, &rr, s), "residual");
    r.applies_f64 += 1;
    r.rel_residual = rel_res(rr, &rerr);
    CU_TRY(rerr, "norm r per mirror");
    if (!(r.rel_residual <= o->rtol) && !energy_ok)
      result = fail(TN_ENOTCONV, "not converged: relative residual %.3e > %.3e after %d iterations",
                    r.rel_residual, o->rtol, r.inner_iters);
  }
  TnWait wout{};
  CU_TRY(cudaMemcpyAsync(&wout, c->wctl, sizeof(wout), cudaMemcpyDeviceToHost, s), "status");
  const TnWait wdef{kDefaultWaitNs, 0, 0};  // later calls (tn_precond_apply) wait with the default limit
  CU_TRY(cudaMemcpyAsync(c->wctl, &wdef, sizeof(wdef), cudaMemcpyHostToDevice, s), "wait limit");
  CU_TRY(cudaEventRecord(c->ev_out, s), "event");
  CU_TRY(cudaStreamWaitEvent(c->stream, c->ev_out, 0), "event wait");
  CU_TRY(cudaStreamSynchronize(s), "sync");
  if (zl && wout.flag)  // the iterate is not trustworthy: the timeout outranks every other outcome
    result = fail(TN_ETIMEOUT, "a line solve gave up waiting for its staged factors (limit %.3g s)",
                  (double)wset.limit_ns * 1e-9);
  r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  r.status = result;
  r.launches = tn::g_launches;
  if (rep) *rep = r;
  return result;
}

tn_status tn_precond_factor_bytes(tn_ctx *c, int precond, long long *bytes) {
  tn_status st = need_ready(c, false);
  if (st) return st;
  if (!bytes) return fail(TN_EINVAL, "bytes is null");
  CU_TRY(cudaSetDevice(c->device), "cudaSetDevice");
  if ((st = ensure_ws(c))) return st;
  if (precond == TN_PC_ZGROUP) {
    if ((st = ensure_zgroup(c, c->stream))) return st;
    *bytes = c->gplan.ncompact * (long long)sizeof(float);
    return TN_OK;
  }
  if (precond == TN_PC_ZLINE) {
    if ((st = ensure_zline(c, c->stream))) return st;
    *bytes = is_batch(c) ? c->batch->nfac * (long long)sizeof(float) : (long long)tn_zline_factor_bytes(c->dm);
    return TN_OK;
  }
  if (precond == TN_PC_JACOBI) {
    *bytes = (long long)c->ndof * (long long)sizeof(float);
    return TN_OK;
  }
  return fail(TN_EINVAL, "unknown preconditioner");
}

tn_status tn_precond_apply(tn_ctx *c, int precond, int precision, const void *r, void *z) {
  tn_status st = need_ready(c, false);
  if (st) return st;
  if (precision != TN_F64 && precision != TN_F32) return fail(TN_EINVAL, "precision must be TN_F64 or TN_F32");
  if (precond != TN_PC_JACOBI && precond != TN_PC_ZLINE && precond != TN_PC_ZGROUP)
    return fail(TN_EINVAL, "unknown preconditioner");
  const size_t es = precision == TN_F64 ? 8 : 4;
  if ((st = check_buf(c, r, es, "r"))) return st;
  if ((st = check_buf(c, z, es, "z"))) return st;
  const char *a = (const char *)r, *b = (const char *)z;
  if (a < b + c->ndof * es && b < a + c->ndof * es) return fail(TN_EINVAL, "r and z overlap");
  CU_TRY(cudaSetDevice(c->device), "cudaSetDevice");
  if ((st = ensure_ws(c))) return st;
  if (precond == TN_PC_ZGROUP) {
    if ((st = ensure_zgroup(c, c->stream))) return st;
    CU_TRY(with_groups(make_sys(c), c)
               .zsolve(precision, precision == TN_F64 ? (const void *)c->gfac64 : (const void *)c->gfac,
                       const_cast<void *>(r), nullptr, z, nullptr, c->gpart, nullptr, c->stream),
           "grouped-line solve");
    return TN_OK;
  }
  if (precond == TN_PC_ZLINE) {
    if ((st = ensure_zline(c, c->stream))) return st;
    CU_TRY(make_sys(c).zsolve(precision, precision == TN_F64 ? (const void *)c->zfac64 : (const void *)c->zfac,
                              const_cast<void *>(r), nullptr, z, nullptr, c->zpart, nullptr, c->stream),
           "z-line solve");
    return TN_OK;
  }
  if (is_batch(c)) return fail(TN_EINVAL, "Jacobi needs a single mesh");
  CU_TRY(tn_launch_diag(c->dm, c->diag64, c->stream), "diag");
  CU_TRY(tn_jacobi_apply(c->ndof, precision, c->diag64, r, z, c->stream), "jacobi");
  return TN_OK;
}


// d(dz/dzeta)/d(z_s) at every node of slab q, for the slab boundary s
// (slab q = s - 1 has z_bot = z_s, slab q = s has z_top = z_s)
static void slab_seed(const tn::HostMesh &hm, const double *slab_z, const int *slab_log, int s, double *seed) {
  const int N = hm.N;
  double x[TN_MAX_N], w[TN_MAX_N], D[TN_MAX_N * TN_MAX_N];
  tn::lgl(N, x, w, D);
  for (int q = 0; q < hm.nslab * N; ++q) seed[q] = 0.0;
  for (int q = s - 1; q <= s; ++q) {
    if (q < 0 || q >= hm.nslab) continue;
    const bool top = (q == s);  // z_s is the top of slab q
    const double zt = slab_z[q], zb = slab_z[q + 1];
    for (int k = 0; k < N; ++k) {
      double d;
      if (slab_log[q]) {
        const double dt = -zt, db = -zb, a = 0.5 * (1 + x[k]), b = 0.5 * (1 - x[k]);
        const double S = std::exp(a * std::log(dt) + b * std::log(db)), L = std::log(db) - std::log(dt);
        // dz/dzeta = S L / 2;  d/dz = -d/d(depth)
        d = top ? -0.5 * (S * a / dt * L - S / dt) : -0.5 * (S * b / db * L + S / db);
      } else {
        d = top ? 0.5 : -0.5;
      }
      seed[(size_t)q * N + k] = d;
    }
  }
}

// dJ/dtheta for every parameter of one mirror, given u, lambda and the layer
// weights on the device: the dual-number operator contractions of every
// parameter (over the slabs it touches) in one launch and the energy
// contractions in another (work lists of (parameter, element) pairs), one
// partial per CTA, then one copy to the host and fixed-order sums there.
// seed_dev: n_slabs x (n_slabs N) doubles (the slab seeds of every boundary);
// matseed: an identity of row stride mat_ld >= 3 n_layers (row 3 L + q
// seeds modulus q of layer L); part and work_dev: grad_parts(hm) entries;
// pseed_dev: 2 per parameter; tmp: host scratch of grad_parts(hm) doubles.
static size_t grad_parts(const tn::HostMesh &hm) {
  const int S = hm.nslab;
  size_t n = 256;  // r0
  for (int b = 1; b <= S; ++b) {
    const int a0 = b - 2 < 0 ? 0 : b - 2, a1 = b + 2 > S ? S : b + 2;
    const int k0 = b - 1 < 0 ? 0 : b - 1, k1 = b + 1 > S ? S : b + 1;
    n += (size_t)(a1 - a0 + k1 - k0) * hm.ncol;
  }
  for (int L = 0; L < hm.n_layers; ++L) {
    int lo = S, hi = -1;
    for (int q = 0; q < S; ++q)
      if (hm.slab_layer[q] == L) { lo = q < lo ? q : lo; hi = q > hi ? q : hi; }
    if (hi < 0) continue;
    const int a0 = lo - 1 < 0 ? 0 : lo - 1, a1 = hi + 2 > S ? S : hi + 2;
    n += 3 * (size_t)(a1 - a0 + hi + 1 - lo) * hm.ncol;
  }
  return n;
}

static cudaError_t grad_contractions(const tn::HostMesh &hm, const DevMesh &dm, const double *slab_z,
                                     const int *slab_log, const double *u, const double *lam, const double *wdev,
                                     double r0, double F0, double *dJ_dslab_z, double *dJ_dr0, double *dJ_dmat,
                                     double *part, double *tmp, double *seed_dev, const double *matseed, int mat_ld,
                                     int2 *work_dev, const double **pseed_dev, cudaStream_t s) {
  const int S = hm.nslab, nl = hm.n_layers, N = hm.N, nc = hm.ncol;
  std::vector<double> seed((size_t)S * S * N);
  for (int b = 1; b <= S; ++b) slab_seed(hm, slab_z, slab_log, b, seed.data() + (size_t)(b - 1) * S * N);
  // parameters: slab boundaries b = 1..S, then (layer L, modulus q) of the
  // layers that own slabs; per parameter the slabs of its operator and
  // energy contractions
  struct Param { int a0, a1, k0, k1; const double *ss, *ms; };
  std::vector<Param> prm;
  for (int b = 1; b <= S; ++b)
    prm.push_back({b - 2 < 0 ? 0 : b - 2, b + 2 > S ? S : b + 2, b - 1 < 0 ? 0 : b - 1, b + 1 > S ? S : b + 1,
                   seed_dev + (size_t)(b - 1) * S * N, nullptr});
  std::vector<int> mat_param(3 * nl, -1);
  for (int L = 0; L < nl; ++L) {
    int lo = S, hi = -1;
    for (int q = 0; q < S; ++q)
      if (hm.slab_layer[q] == L) { lo = q < lo ? q : lo; hi = q > hi ? q : hi; }
    if (hi < 0) continue;
    for (int q = 0; q < 3; ++q) {
      mat_param[3 * L + q] = (int)prm.size();
      prm.push_back({lo - 1 < 0 ? 0 : lo - 1, hi + 2 > S ? S : hi + 2, lo, hi + 1, nullptr,
                     matseed + (size_t)(3 * L + q) * mat_ld});
    }
  }
  // work lists (parameter, element), the operator's first, then the energy's
  std::vector<int2> work;
  std::vector<size_t> aoff(prm.size() + 1), eoff(prm.size() + 1);
  std::vector<const double *> ps(2 * prm.size());
  for (size_t p = 0; p < prm.size(); ++p) {
    aoff[p] = work.size();
    for (int e = prm[p].a0 * nc; e < prm[p].a1 * nc; ++e) work.push_back(make_int2((int)p, e));
    ps[2 * p] = prm[p].ss;
    ps[2 * p + 1] = prm[p].ms;
  }
  aoff[prm.size()] = work.size();
  const size_t na = work.size();
  for (size_t p = 0; p < prm.size(); ++p) {
    eoff[p] = work.size() - na;
    for (int e = prm[p].k0 * nc; e < prm[p].k1 * nc; ++e) work.push_back(make_int2((int)p, e));
  }
  eoff[prm.size()] = work.size() - na;
  const size_t ne = work.size() - na;
  cudaError_t e = cudaMemcpyAsync(seed_dev, seed.data(), sizeof(double) * seed.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(work_dev, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pseed_dev, ps.data(), sizeof(double *) * ps.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = tn_launch_apply_dual_work(dm, work_dev, (int)na, pseed_dev, u, lam, part, s);
  if (e == cudaSuccess) e = tn_launch_energy_dual_work(dm, work_dev + na, (int)ne, pseed_dev, u, wdev, part + na, s);
  if (e == cudaSuccess) e = tn_launch_rhs_dr0(dm, r0, F0, lam, part + na + ne, 256, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, part, sizeof(double) * (na + ne + 256), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // also keeps the host arrays alive until copied
  if (e != cudaSuccess) return e;
  auto sum = [&](size_t a, size_t b) {
    double acc = 0.0;
    for (size_t i = a; i < b; ++i) acc += tmp[i];
    return acc;
  };
  auto dJ = [&](size_t p) {  // dK - dA u
    return sum(na + eoff[p], na + eoff[p + 1]) - sum(aoff[p], aoff[p + 1]);
  };
  dJ_dslab_z[0] = 0.0;
  for (int b = 1; b <= S; ++b) dJ_dslab_z[b] = dJ(b - 1);
  for (int t = 0; t < 3 * nl; ++t) dJ_dmat[t] = mat_param[t] >= 0 ? dJ(mat_param[t]) : 0.0;
  *dJ_dr0 = sum(na + ne, na + ne + 256);
  return cudaSuccess;
}

// the adjoint gradient of the context's mirror or batch (see the header)
static tn_status grad_impl(tn_ctx *c, const tn_solve_opts *o, const double *u, const double *w_host,
                           double *lambda, double *dJ_dslab_z, double *dJ_dr0, double *dJ_dmat,
                           tn_solve_report *rep) {
  tn_status st = need_ready(c, true);
  if (st) return st;
  if (!o || !w_host || !dJ_dslab_z || !dJ_dr0 || !dJ_dmat) return fail(TN_EINVAL, "null argument");
  if ((st = check_buf(c, u, 8, "u"))) return st;
  if (lambda && (st = check_buf(c, lambda, 8, "lambda"))) return st;
  CU_TRY(cudaSetDevice(c->device), "cudaSetDevice");
  if ((st = ensure_ws(c))) return st;
  const int nl = total_layers(c);
  const size_t n = c->ndof;
  size_t Pmax = 0, SSNmax = 0;
  int NLmax = 0;
  const int ninst = is_batch(c) ? c->batch->n : 1;
  for (int i = 0; i < ninst; ++i) {
    const tn::HostMesh &hm = is_batch(c) ? c->batch->inst[i].hm : c->hm;
    Pmax = std::max(Pmax, grad_parts(hm));
    SSNmax = std::max(SSNmax, (size_t)hm.nslab * hm.nslab * hm.N);
    NLmax = std::max(NLmax, hm.n_layers);
  }
  double *wdev = nullptr, *g = nullptr, *lam = lambda, *part = nullptr, *seed_dev = nullptr, *matseed = nullptr;
  int2 *work_dev = nullptr;
  const double **pseed_dev = nullptr;
  std::vector<double> tmp(Pmax);
  cudaError_t e = cudaMalloc((void **)&wdev, sizeof(double) * nl);
  if (e == cudaSuccess) e = cudaMalloc((void **)&g, sizeof(double) * n);
  if (e == cudaSuccess && !lam) e = cudaMalloc((void **)&lam, sizeof(double) * n);
  if (e == cudaSuccess) e = cudaMalloc((void **)&part, sizeof(double) * Pmax);
  if (e == cudaSuccess) e = cudaMalloc((void **)&seed_dev, sizeof(double) * SSNmax);
  if (e == cudaSuccess) e = cudaMalloc((void **)&matseed, sizeof(double) * 9 * NLmax * NLmax);
  if (e == cudaSuccess) e = cudaMalloc((void **)&work_dev, sizeof(int2) * Pmax);
  if (e == cudaSuccess) e = cudaMalloc((void **)&pseed_dev, sizeof(double *) * 2 * (SSNmax + 3 * (size_t)NLmax));
  if (e == cudaSuccess) {  // the moduli seeds: identity of 3 NLmax (row 3L + q seeds modulus q of layer L)
    std::vector<double> eye((size_t)9 * NLmax * NLmax, 0.0);
    for (int t = 0; t < 3 * NLmax; ++t) eye[(size_t)t * 3 * NLmax + t] = 1.0;
    e = cudaMemcpy(matseed, eye.data(), sizeof(double) * eye.size(), cudaMemcpyHostToDevice);
  }
  tn_solve_report r{};
  cudaStream_t s = c->stream;
  auto cleanup = [&]() {
    if (wdev) cudaFree(wdev);
    if (g) cudaFree(g);
    if (lam && lam != lambda) cudaFree(lam);
    if (part) cudaFree(part);
    if (seed_dev) cudaFree(seed_dev);
    if (matseed) cudaFree(matseed);
    if (work_dev) cudaFree(work_dev);
    if (pseed_dev) cudaFree(pseed_dev);
  };
  if (e != cudaSuccess) { cleanup(); cudaGetLastError(); return fail(TN_ENOMEM, "gradient workspace"); }
  // adjoint source g = sum_i w_i K_i u per mirror
  e = cudaMemcpyAsync(wdev, w_host, sizeof(double) * nl, cudaMemcpyHostToDevice, s);
  if (!is_batch(c)) {
    if (e == cudaSuccess) e = tn_launch_energy_source(c->dm, u, wdev, g, s);
  } else {
    for (int i = 0; i < c->batch->n && e == cudaSuccess; ++i) {
      const BatchInst &q = c->batch->inst[i];
      e = tn_launch_energy_source(q.dm, u + q.dof_off, wdev + q.layer_off, g + q.dof_off, s);
    }
  }
  if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "adjoint source"); }
  tn_solve_opts ao = *o;
  ao.energy_rtol = 0.0;
  st = solve_impl(c, &ao, g, lam, &r);
  if (st != TN_OK && st != TN_ENOTCONV) { cleanup(); return st; }
  tn_status result = st;
  if (!is_batch(c)) {
    e = grad_contractions(c->hm, c->dm, c->slab_z_host, c->slab_log_host, u, lam, wdev, c->r0, c->F0, dJ_dslab_z,
                          dJ_dr0, dJ_dmat, part, tmp.data(), seed_dev, matseed, 3 * NLmax, work_dev, pseed_dev, s);
  } else {
    size_t zoff = 0;
    for (int i = 0; i < c->batch->n && e == cudaSuccess; ++i) {
      const BatchInst &q = c->batch->inst[i];
      e = grad_contractions(q.hm, q.dm, q.slab_z.data(), q.slab_log.data(), u + q.dof_off, lam + q.dof_off,
                            wdev + q.layer_off, q.r0, q.F0, dJ_dslab_z + zoff, dJ_dr0 + i,
                            dJ_dmat + 3 * (size_t)q.layer_off, part, tmp.data(), seed_dev, matseed, 3 * NLmax,
                            work_dev, pseed_dev, s);
      zoff += q.hm.nslab + 1;
    }
  }
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, "gradient contractions");
  if (rep) *rep = r;
  return result;
}

tn_status tn_energy_grad(tn_ctx *c, const tn_solve_opts *o, const double *u, const double *w_host,
                         double *lambda, double *dJ_dslab_z, double *dJ_dr0, double *dJ_dmat,
                         tn_solve_report *rep) {
  if (c && is_batch(c)) return fail(TN_EINVAL, "tn_energy_grad works on a single mesh; use tn_batch_energy_grad");
  return grad_impl(c, o, u, w_host, lambda, dJ_dslab_z, dJ_dr0, dJ_dmat, rep);
}

tn_status tn_batch_energy_grad(tn_ctx *c, const tn_solve_opts *o, const double *u, const double *w_host,
                               double *lambda, double *dJ_dslab_z, double *dJ_dr0, double *dJ_dmat,
                               tn_solve_report *rep) {
  if (c && !is_batch(c)) return fail(TN_EINVAL, "tn_batch_energy_grad needs a batch");
  return grad_impl(c, o, u, w_host, lambda, dJ_dslab_z, dJ_dr0, dJ_dmat, rep);
}

tn_status tn_layer_energies(tn_ctx *c, const double *u, double *U_host) {
  tn_status st = need_ready(c, false);
  if (st) return st;
  if ((st = check_buf(c, u, 8, "u"))) return st;
  if (!U_host) return fail(TN_EINVAL, "U_host is null");
  CU_TRY(cudaSetDevice(c->device), "cudaSetDevice");
  if ((st = ensure_ws(c))) return st;
  CU_TRY(energies_host(c, u, U_host, c->stream), "energies");
  return TN_OK;
}

tn_status tn_layer_energy_parts(tn_ctx *c, const double *u, double *parts_host) {
  tn_status st = need_ready(c, false);
  if (st) return st;
  if ((st = check_buf(c, u, 8, "u"))) return st;
  if (!parts_host) return fail(TN_EINVAL, "parts_host is null");
  CU_TRY(cudaSetDevice(c->device), "cudaSetDevice");
  const int n = is_batch(c) ? c->batch->n : 1;
  size_t E = 0;
  for (int i = 0; i < n; ++i) E += is_batch(c) ? (size_t)c->batch->inst[i].hm.E : (size_t)c->hm.E;
  double *dev = nullptr;
  CU_TRY(cudaMalloc((void **)&dev, sizeof(double) * 3 * E), "energy-parts scratch");
  std::vector<double> h(3 * E);
  cudaError_t e = cudaSuccess;
  size_t eo = 0;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    const DevMesh &dm = is_batch(c) ? c->batch->inst[i].dm : c->dm;
    const long long off = is_batch(c) ? c->batch->inst[i].dof_off : 0;
    e = tn_launch_energy_parts(dm, u + off, dev + 3 * eo, c->stream);
    eo += dm.E;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), dev, sizeof(double) * 3 * E, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(dev);
  if (e != cudaSuccess) return cuda_fail(e, "energy parts");
  // per layer, slab by slab and column by column (fixed order)
  const int nl = total_layers(c);
  for (int l = 0; l < 3 * nl; ++l) parts_host[l] = 0.0;
  eo = 0;
  for (int i = 0; i < n; ++i) {
    const tn::HostMesh &hm = is_batch(c) ? c->batch->inst[i].hm : c->hm;
    const int lo = is_batch(c) ? c->batch->inst[i].layer_off : 0;
    for (int el = 0; el < hm.E; ++el) {
      const int L = lo + hm.slab_layer[el / hm.ncol];
      for (int j = 0; j < 3; ++j) parts_host[3 * L + j] += h[3 * (eo + el) + j];
    }
    eo += hm.E;
  }
  return TN_OK;
}

tn_status tn_thin_coating_psd(double kB_T, double f, double r0, double d, double Ys, double nus, double Yc,
                              double nuc, double phi_c, double *S_out) {
  if (!S_out) return fail(TN_EINVAL, "S_out is null");
  if (!(kB_T > 0.0) || !(f > 0.0) || !(r0 > 0.0) || !(d > 0.0) || !(Ys > 0.0) || !(Yc > 0.0) ||
      !(nus > -1.0 && nus < 0.5) || !(nuc > -1.0 && nuc < 0.5))
    return fail(TN_EINVAL, "need kB_T, f, r0, d, Ys, Yc > 0 and -1 < nu < 1/2");
  const double a = (1.0 + nus) * (1.0 - 2.0 * nus), b = (1.0 + nuc);
  const double bracket = Yc * Yc * a * a + Ys * Ys * b * b * (1.0 - 2.0 * nuc);
  *S_out = kB_T / (M_PI * M_PI * f) * (1.0 - nus * nus) / (r0 * Ys) * (d / r0) * phi_c /
           (Ys * Yc * (1.0 - nuc * nuc) * (1.0 - nus * nus)) * bracket;
  return TN_OK;
}

tn_status tn_iso_moduli(double Y, double nu, double *c, double *dc) {
  if (!c) return fail(TN_EINVAL, "c is null");
  if (!(Y > 0.0) || !(nu > -1.0 && nu < 0.5)) return fail(TN_EINVAL, "need Y > 0 and -1 < nu < 1/2");
  iso_moduli(Y, nu, c, dc);
  return TN_OK;
}

tn_status tn_noise_psd(const double *U, const double *phi, int n, double kB_T, double f, double F0,
                       double *S_out) {
  if (!U || !phi || !S_out || n < 1) return fail(TN_EINVAL, "null argument or n < 1");
  if (!(kB_T > 0.0) || !(f > 0.0) || !(F0 != 0.0)) return fail(TN_EINVAL, "need kB_T > 0, f > 0, F0 != 0");
  double w = 0.0;
  for (int i = 0; i < n; ++i) w += phi[i] * U[i];
  *S_out = 4.0 * kB_T * w / (M_PI * f * F0 * F0);
  return TN_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------
// Per-layer energies without any allocation.
//
// Some callers cannot allocate device memory when they ask for energies: a
// process that reserves its whole HBM budget up front (a serving pool that
// hands out fixed buffers), or one that must not trigger the device-wide
// synchronisation that cudaMalloc / cudaFree can imply while other streams
// are busy.  tn_layer_energies allocates its scratch on first use; this
// variant instead uses a fixed scratch array that lives in the library's
// device image: every GPU that loads the library holds it (532 KB) until the
// process exits.  It bounds the mesh to kNoAllocMaxElements elements and
// kNoAllocMaxLayers layers.  Every call shares the array, so calls that
// overlap on the GPU (other streams, other threads) race; each call writes
// every entry it later reads, so nothing has to be cleared between calls.
namespace {
constexpr int kNoAllocMaxElements = 65536;
constexpr int kNoAllocMaxLayers = 1024;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxElements + kNoAllocMaxLayers];

constexpr int kNoAllocMaxDevices = 64;
double *g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};
std::mutex g_noalloc_mutex;

// device address of the scratch array on the current device (set up once per
// device; in host code the symbol itself is only a host-side stand-in)
cudaError_t noalloc_scratch(int device, double **out) {
  if (device < 0 || device >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[device] = static_cast<double *>(p);
  }
  *out = g_noalloc_ptr[device];
  return cudaSuccess;
}
}  // namespace

extern "C" tn_status tn_layer_energies_noalloc(tn_ctx *c, const double *u, double *U_host) {
  tn_status st = need_ready(c, false);
  if (st) return st;
  if (is_batch(c)) return fail(TN_EINVAL, "tn_layer_energies_noalloc works on a single mesh");
  if ((st = check_buf(c, u, 8, "u"))) return st;
  if (!U_host) return fail(TN_EINVAL, "U_host is null");
  if (c->dm.E > kNoAllocMaxElements || c->dm.n_layers > kNoAllocMaxLayers)
    return fail(TN_EINVAL, "tn_layer_energies_noalloc: mesh has %d elements and %d layers; the fixed scratch "
                "holds at most %d elements and %d layers (use tn_layer_energies)",
                c->dm.E, c->dm.n_layers, kNoAllocMaxElements, kNoAllocMaxLayers);
  CU_TRY(cudaSetDevice(c->device), "cudaSetDevice");
  double *scratch = nullptr;
  CU_TRY(noalloc_scratch(c->device, &scratch), "cudaGetSymbolAddress of the fixed scratch");
  double *elem = scratch, *layer = scratch + kNoAllocMaxElements;
  CU_TRY(tn_launch_energy(c->dm, u, elem, layer, c->stream), "energy launch");
  CU_TRY(cudaMemcpyAsync(U_host, layer, sizeof(double) * c->dm.n_layers, cudaMemcpyDeviceToHost, c->stream),
         "energy copy");
  CU_TRY(cudaStreamSynchronize(c->stream), "energy sync");
  return TN_OK;
}
