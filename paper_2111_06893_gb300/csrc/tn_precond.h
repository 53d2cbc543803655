// Column-line block preconditioner (precond.cu).
#pragma once

#include <cstddef>
#include <vector>
#include <cuda_runtime.h>

#include "tn_internal.h"

size_t tn_zline_block_bytes(const DevMesh &m);   // FP64 set-up blocks
size_t tn_zline_factor_bytes(const DevMesh &m);  // FP32 factors kept for the solve
size_t tn_zline_factor_entries(const DevMesh &m);  // entries per precision (padded records)
int tn_zline_partials(const DevMesh &m);         // partial sums of r.z (and of r.r) written by one solve
cudaError_t tn_zline_setup(const DevMesh &m, double *blk, float *fac, double *fac64, int *status,
                           cudaStream_t st);
// z = M^{-1} r with M the column-line blocks; q != nullptr: first
// r <- r - (*alpha) q (written back).  Per block of four lines: part_rz[b] =
// partial r.z, part_rr[b] = partial r.r (either may be nullptr).  *done != 0:
// returns at once.  A staging wait that runs out sets *zerr = 1.
cudaError_t tn_zline_solve(const DevMesh &m, int prec, const void *fac, void *r, const void *q, void *z,
                           const double *alpha, double *part_rz, double *part_rr, const int *done, TnWait *zerr,
                           cudaStream_t st);
cudaError_t tn_upload_lgl_precond(const LglTables *t);
// batch: warp w of block b solves line work[4 b + w] = (instance, line); factors of
// instance i at fac + fac_off[i] (elements of the factor type), vectors at dof_off[i]
cudaError_t tn_zline_solve_batch(int N, int prec, const DevMesh *meshes, const int2 *work, int nwork,
                                 const long long *fac_off, const long long *dof_off, const void *fac, void *r,
                                 const void *q, void *z, const double *alpha, double *part_rz, double *part_rr,
                                 const int *done, TnWait *zerr, cudaStream_t st);

// ---- line groups: lines joined by matching nodes of lateral faces
constexpr int kZgMaxCls = 28;  // classes: (group size 1..4) x (N = 3..9)
constexpr int kZgMaxPk = 7;    // pack lists: one per degree (N = 3..9), one launch each
constexpr int kZgSide = 6;     // side streams the launches of a batch run on
// the groups of one mesh or of every mirror of a batch, ordered by class
// (group size, largest first; then N; then mirror)
struct ZGroupPlan {
  int ngroups = 0;
  std::vector<int4> lines;          // per group: line ids col * N^2 + j * N + i of its mirror (-1: unused)
  std::vector<int> inst;            // per group: mirror
  std::vector<long long> fac_off;   // per group: first factor entry
  long long nfac = 0;               // factor entries in all
  long long ncompact = 0;           // of which Linv_s and the O factors (the rest: W_s)
  int ncls = 0;
  int cls_N[kZgMaxCls] = {0}, cls_G[kZgMaxCls] = {0}, cls_start[kZgMaxCls] = {0}, cls_n[kZgMaxCls] = {0};
  std::vector<int> inst_start, inst_n;  // [mirror * 5 + g]: first group and count of size g (set-up)
  // packs: up to four groups filling the four warps of a CTA (-1: none),
  // per degree, largest first
  std::vector<int4> packs;
  int npk = 0;
  int pk_N[kZgMaxPk] = {0}, pk_start[kZgMaxPk] = {0}, pk_n[kZgMaxPk] = {0};
};
// device view of a plan and the streams the classes run on
struct ZGroupDev {
  const int4 *lines = nullptr;
  const long long *fac_off = nullptr;
  const int *inst = nullptr;           // batch: mirror of every group (nullptr: one mesh)
  const DevMesh *meshes = nullptr;     // batch: meshes of the mirrors (device)
  const long long *dof_off = nullptr;  // batch: first unknown of every mirror (device)
  long long ndof = 0;                  // unknowns of the mesh or of the whole batch
  int ngroups = 0, ncls = 0;
  int cls_N[kZgMaxCls] = {0}, cls_G[kZgMaxCls] = {0}, cls_start[kZgMaxCls] = {0}, cls_n[kZgMaxCls] = {0};
  const int4 *packs = nullptr;         // the plan's packs (device)
  int *queue = nullptr;                // per degree: next pack, CTAs finished (device, zero between launches)
  int npk = 0;
  int pk_N[kZgMaxPk] = {0}, pk_start[kZgMaxPk] = {0}, pk_n[kZgMaxPk] = {0};
  cudaStream_t side[kZgSide] = {nullptr};
  cudaEvent_t fork = nullptr, join[kZgSide] = {nullptr};
};
bool tn_zgroup_plan(const tn::HostMesh *const *hms, int n, ZGroupPlan *plan, char *msg, int msglen);
size_t tn_zgroup_cross_bytes(const DevMesh &m);                                // FP64 cross-line blocks (set-up)
size_t tn_zgroup_work_bytes(const DevMesh &m, const ZGroupPlan &p, int inst);  // FP64 scratch (set-up)
// factors of mirror `inst` (its mesh m); blk: tn_zline_block_bytes(m);
// fac / fac64: plan.nfac entries; *status = 1 on a non-positive pivot.  The
// group sizes factor at once on st and gd's first three side streams
// (forked from and joined back into st with gd's events).
cudaError_t tn_zgroup_setup(const DevMesh &m, const ZGroupPlan &p, const ZGroupDev &gd, int inst,
                            const int4 *lines, const long long *fac_off, double *blk, double *xblk, double *work,
                            float *fac, double *fac64, int *status, cudaStream_t st);
// as tn_zline_solve, over the groups (m: the mesh, nullptr for a batch);
// partial sums: one per group.  q != nullptr: r -= alpha q first, as a
// launch of its own over all gd.ndof unknowns
// fold (optional): the beta step of a PCG iteration (s and cnt; the rest is
// filled in here)
cudaError_t tn_zgroup_solve(const DevMesh *m, const ZGroupDev &gd, int prec, const void *fac, void *r,
                            const void *q, void *z, const double *alpha, double *part_rz, double *part_rr,
                            const int *done, TnWait *zerr, cudaStream_t st, const PcgFold *fold = nullptr);
