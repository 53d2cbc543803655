// Column-line and grouped-line block preconditioners for thin layers.
//
// The paper accelerates its Krylov solver with multigrid and an additive
// Schwarz smoother (Sec. 2.3).  The dominant difficulty of thin coating layers
// is the strong coupling across the layers: elements with aspect ratios up
// to ~1e4 and penalties sigma ~ 1/h_z on the layer interfaces (Eq. (penalty)).
// This preconditioner takes, for every vertical line of nodes (column col,
// cross-section node (i, j), all slabs, all N nodes along zeta, three
// components), the exact principal sub-matrix A_LL of the DG operator on that
// line and inverts it: A_LL is block tridiagonal over the slabs (3N x 3N
// blocks: D_s inside slab s, O_s coupling slab s to the slab below through
// the face terms of Eq. (numflux)).  Set-up: the blocks are formed from the
// same weak-form terms as the operator (FP64), factorised by block Cholesky
// along the line (one thread per line) and stored in FP32.  Application:
// one warp per line, the 3N unknowns of a slab on the lanes, forward and
// backward block substitution.  The grouped variant (further below) takes
// the lines through one cross-section point of neighbouring columns
// together, adding the lateral-face coupling between them.
#include <cstdio>
#include <type_traits>
#include <vector>

#include "tn_internal.h"
#include "tn_precond.h"

// device constants are per translation unit (no relocatable device code):
// this file keeps its own copy of the LGL tables
__constant__ LglTables c_lgl_pc;

cudaError_t tn_upload_lgl_precond(const LglTables *t) {
  return cudaMemcpyToSymbol(c_lgl_pc, t, sizeof(LglTables));
}

namespace {

// Factor record of one line and slab s: [Linv_s | Z_s].
//  Linv_s: inverse of the lower Cholesky factor of the slab's Schur
//          complement, lower triangular, packed column by column (column c
//          holds rows c..M-1 at zcol(M, c) + (row - c)), M (M + 1) / 2 entries;
//  Z_s:    L_{s-1}^{-1} O_{s-1}, row-major with an odd row stride zld(M) so
//          that lanes reading one entry per row hit distinct banks.
// Both parts are padded to a multiple of 4 entries (16-byte cp.async chunks
// for float and double records).
__host__ __device__ constexpr int pad4(int v) { return ((v + 3) / 4) * 4; }
__host__ __device__ constexpr int zlp(int M) { return pad4(M * (M + 1) / 2); }
__host__ __device__ constexpr int zld(int M) { return M | 1; }
__host__ __device__ constexpr int zzp(int M) { return pad4(M * zld(M)); }
__host__ __device__ constexpr int zrec(int M) { return zlp(M) + zzp(M); }
__host__ __device__ constexpr int zcol(int M, int c) { return c * M - c * (c - 1) / 2; }

#define LD(a, b) c_lgl_pc.D[N][(a) * N + (b)]
#define LW(a) c_lgl_pc.w[N][(a)]

// Q_ab(g, h) = sum_{alpha beta} g_alpha Y^{alpha a beta b} h_beta for a
// cubic-aligned stiffness (isotropic: c11 = l + 2m, c12 = l, c44 = m)
__device__ __forceinline__ double Qab(int a, int b, const double g[3], const double h[3], double c11,
                                      double c12, double c44) {
  if (a == b) {
    double s = c11 * g[a] * h[a];
    for (int al = 0; al < 3; ++al)
      if (al != a) s += c44 * g[al] * h[al];
    return s;
  }
  return c12 * g[a] * h[b] + c44 * g[b] * h[a];
}

// physical gradient of a basis function from its logical gradient lg
__device__ __forceinline__ void phys(const double lg[3], double ixx, double ixy, double iex, double iey,
                                     double dz, double g[3]) {
  g[0] = ixx * lg[0] + iex * lg[1];
  g[1] = ixy * lg[0] + iey * lg[1];
  g[2] = lg[2] / dz;
}

// D_s and O_s of every line through element e: one thread per line (i, j)
template <int N>
__global__ void zline_blocks_kernel(const DevMesh m, double *__restrict__ blk) {
  constexpr int M = 3 * N, N2 = N * N;
  const int e = blockIdx.x, t = threadIdx.x;
  if (t >= N2) return;
  const int s = e / m.ncol, c = e - s * m.ncol;
  const int i = t % N, j = t / N;
  const size_t line = (size_t)c * N2 + t;
  double *Dm = blk + ((line * m.nslab + s) * 2 + 0) * M * M;
  double *Om = blk + ((line * m.nslab + s) * 2 + 1) * M * M;
  for (int q = 0; q < M * M; ++q) { Dm[q] = 0.0; Om[q] = 0.0; }
  const double *cg = m.colgeo + (size_t)c * CG_NF * N2;
  const double *sg = m.slabgeo + (size_t)s * SG_NF * N;
  const int qq = j * N + i;
  const double ixx = cg[CG_IXX * N2 + qq], ixy = cg[CG_IXY * N2 + qq];
  const double iex = cg[CG_IEX * N2 + qq], iey = cg[CG_IEY * N2 + qq];
  const double det2 = cg[CG_DET * N2 + qq];
  double dz[N];
  for (int k = 0; k < N; ++k) dz[k] = sg[SG_DZ * N + k];
  const int L = m.slab_layer[s];
  const double c11 = m.layer_c[3 * L], c12 = m.layer_c[3 * L + 1], c44 = m.layer_c[3 * L + 2];
  const double Dii = LD(i, i), Djj = LD(j, j);

  // ---- volume: r on the z-line
  for (int kk = 0; kk < N; ++kk) {
    const double wJ = LW(i) * LW(j) * LW(kk) * det2 * dz[kk];
    for (int k = 0; k < N; ++k) {
      double lk[3] = {k == kk ? Dii : 0.0, k == kk ? Djj : 0.0, LD(kk, k)}, gk[3];
      phys(lk, ixx, ixy, iex, iey, dz[kk], gk);
      for (int k2 = 0; k2 < N; ++k2) {
        double l2[3] = {k2 == kk ? Dii : 0.0, k2 == kk ? Djj : 0.0, LD(kk, k2)}, g2[3];
        phys(l2, ixx, ixy, iex, iey, dz[kk], g2);
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) Dm[(a * N + k) * M + b * N + k2] += wJ * Qab(a, b, gk, g2, c11, c12, c44);
      }
    }
  }
  // r on the xi- and eta-lines through the node (diagonal in k)
  for (int k = 0; k < N; ++k) {
    for (int r = 0; r < N; ++r) {
      if (r != i) {
        const int q2 = j * N + r;
        const double wJ = LW(r) * LW(j) * LW(k) * cg[CG_DET * N2 + q2] * dz[k];
        const double d = LD(r, i);
        const double g[3] = {cg[CG_IXX * N2 + q2] * d, cg[CG_IXY * N2 + q2] * d, 0.0};
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) Dm[(a * N + k) * M + b * N + k] += wJ * Qab(a, b, g, g, c11, c12, c44);
      }
      if (r != j) {
        const int q2 = r * N + i;
        const double wJ = LW(i) * LW(r) * LW(k) * cg[CG_DET * N2 + q2] * dz[k];
        const double d = LD(r, j);
        const double g[3] = {cg[CG_IEX * N2 + q2] * d, cg[CG_IEY * N2 + q2] * d, 0.0};
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) Dm[(a * N + k) * M + b * N + k] += wJ * Qab(a, b, g, g, c11, c12, c44);
      }
    }
  }

  const double sp1 = (double)((m.p + 1) * (m.p + 1)) * m.penC;
  // ---- faces of the element that contain line nodes
  for (int f = 0; f < 6; ++f) {
    const int d = f >> 1, sd = f & 1;
    const int idx = d == 0 ? i : (d == 1 ? j : -1);
    if (d < 2 && idx != (sd ? N - 1 : 0)) continue;
    // kind and neighbour
    int kind;  // 0 interior, 1 dirichlet, 2 neumann
    double h2 = 0.0, n11 = c11, n12 = c12, n44 = c44;
    if (d < 2) {
      const int nbc = m.colnb[4 * c + f];
      if (nbc >= 0) {
        kind = 0;
        const int code = m.colnbf[4 * c + f];
        const int f2 = code & 3, d2 = f2 >> 1, end2 = (f2 & 1) ? N - 1 : 0;
        const int t1 = d == 0 ? j : i;
        const int a2 = (code >> 2) ? N - 1 - t1 : t1;
        const int i2 = d2 == 0 ? end2 : a2, j2 = d2 == 0 ? a2 : end2;
        const double *g2 = m.colgeo + (size_t)nbc * CG_NF * N2;
        const double rx = g2[(d2 == 0 ? CG_IXX : CG_IEX) * N2 + j2 * N + i2];
        const double ry = g2[(d2 == 0 ? CG_IXY : CG_IEY) * N2 + j2 * N + i2];
        h2 = 2.0 / sqrt(rx * rx + ry * ry);
      } else {
        kind = m.bc_side == TN_BC_FIXED ? 1 : 2;
      }
    } else if (f == 4) {
      if (s + 1 < m.nslab) {
        kind = 0;
        h2 = 2.0 * m.slabgeo[((size_t)(s + 1) * SG_NF + SG_DZ) * N + N - 1];
        const int L2 = m.slab_layer[s + 1];
        n11 = m.layer_c[3 * L2]; n12 = m.layer_c[3 * L2 + 1]; n44 = m.layer_c[3 * L2 + 2];
      } else {
        kind = m.bc_bottom == TN_BC_FIXED ? 1 : 2;
      }
    } else {
      if (s > 0) {
        kind = 0;
        h2 = 2.0 * m.slabgeo[((size_t)(s - 1) * SG_NF + SG_DZ) * N + 0];
        const int L2 = m.slab_layer[s - 1];
        n11 = m.layer_c[3 * L2]; n12 = m.layer_c[3 * L2 + 1]; n44 = m.layer_c[3 * L2 + 2];
      } else {
        kind = 2;  // top: beam pressure (Neumann)
      }
    }
    if (kind == 2) continue;
    double n[3], mag = 1.0;
    if (d == 2) { n[0] = 0.0; n[1] = 0.0; n[2] = sd ? 1.0 : -1.0; }
    else {
      const double rx = d == 0 ? ixx : iex, ry = d == 0 ? ixy : iey;
      mag = sqrt(rx * rx + ry * ry);
      n[0] = (sd ? 1.0 : -1.0) * rx / mag; n[1] = (sd ? 1.0 : -1.0) * ry / mag; n[2] = 0.0;
    }
    const double cT = kind == 0 ? -0.5 : -1.0, cP = kind == 0 ? 1.0 : 2.0;
    const double s11 = kind == 0 ? 0.5 * (c11 + n11) : c11, s12 = kind == 0 ? 0.5 * (c12 + n12) : c12,
                 s44 = kind == 0 ? 0.5 * (c44 + n44) : c44;
    const int kend = sd ? N - 1 : 0;
    for (int k = 0; k < N; ++k) {
      if (d == 2 && k != kend) continue;  // line node on the face
      double W, h;
      if (d == 2) { W = LW(i) * LW(j) * det2; h = 2.0 * dz[k]; }
      else { W = (d == 0 ? LW(j) : LW(i)) * LW(k) * det2 * dz[k] * mag; h = 2.0 / mag; }
      // T1[(a,k),(b,k2)] = W Q_ab(n, grad psi_k2 at node k); added with its transpose
      for (int k2 = 0; k2 < N; ++k2) {
        double l2[3] = {k2 == k ? Dii : 0.0, k2 == k ? Djj : 0.0, LD(k, k2)}, g2[3];
        phys(l2, ixx, ixy, iex, iey, dz[k], g2);
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            const double v = cT * W * Qab(a, b, n, g2, c11, c12, c44);
            Dm[(a * N + k) * M + b * N + k2] += v;
            Dm[(b * N + k2) * M + a * N + k] += v;
          }
      }
      const double sig = sp1 / (kind == 0 ? (h < h2 ? h : h2) : h);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Dm[(a * N + k) * M + b * N + k] += cP * W * sig * Qab(a, b, n, n, s11, s12, s44);
    }
    // ---- coupling to the slab below (face zeta = -1, k = 0, neighbour's k = N-1)
    if (f == 4 && kind == 0) {
      const double W = LW(i) * LW(j) * det2;
      const double dz2 = m.slabgeo[((size_t)(s + 1) * SG_NF + SG_DZ) * N + N - 1];
      const double sig = sp1 / (2.0 * dz[0] < 2.0 * dz2 ? 2.0 * dz[0] : 2.0 * dz2);
      for (int k = 0; k < N; ++k)
        for (int k2 = 0; k2 < N; ++k2) {
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
              double v = 0.0;
              if (k == 0) {  // -1/2 V^T W Tr_ext: neighbour basis gradient at its node N-1
                double l2[3] = {k2 == N - 1 ? Dii : 0.0, k2 == N - 1 ? Djj : 0.0, LD(N - 1, k2)}, g2[3];
                phys(l2, ixx, ixy, iex, iey, dz2, g2);
                v += -0.5 * W * Qab(a, b, n, g2, n11, n12, n44);
              }
              if (k2 == N - 1) {  // +1/2 Tr^T W V_ext: own basis gradient at node 0
                double l1[3] = {k == 0 ? Dii : 0.0, k == 0 ? Djj : 0.0, LD(0, k)}, g1[3];
                phys(l1, ixx, ixy, iex, iey, dz[0], g1);
                v += 0.5 * W * Qab(b, a, n, g1, c11, c12, c44);
              }
              if (k == 0 && k2 == N - 1) v -= W * sig * Qab(a, b, n, n, s11, s12, s44);
              Om[(a * N + k) * M + b * N + k2] += v;
            }
        }
    }
  }
}

// block Cholesky along each line (FP64, in place), then FP32 factors:
// L_s column-major with inverted diagonal, Z_s = L_{s-1}^{-1} O_{s-1} row-major
template <int N>
__global__ void zline_factor_kernel(int nlines, int S, double *__restrict__ blk, float *__restrict__ fac,
                                    double *__restrict__ fac64, int *__restrict__ status) {
  constexpr int M = 3 * N;
  const int line = blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= nlines) return;
  for (int s = 0; s < S; ++s) {
    double *Dm = blk + (((size_t)line * S + s) * 2 + 0) * M * M;
    if (s > 0) {
      const double *Lp = blk + (((size_t)line * S + s - 1) * 2 + 0) * M * M;
      double *Z = blk + (((size_t)line * S + s - 1) * 2 + 1) * M * M;  // O_{s-1} -> Z_s in place
      for (int col = 0; col < M; ++col)
        for (int r = 0; r < M; ++r) {
          double v = Z[r * M + col];
          for (int q = 0; q < r; ++q) v -= Lp[r * M + q] * Z[q * M + col];
          Z[r * M + col] = v / Lp[r * M + r];
        }
      for (int r = 0; r < M; ++r)
        for (int c2 = 0; c2 <= r; ++c2) {
          double v = 0.0;
          for (int q = 0; q < M; ++q) v += Z[q * M + r] * Z[q * M + c2];
          Dm[r * M + c2] -= v;
        }
    }
    for (int col = 0; col < M; ++col) {
      double v = Dm[col * M + col];
      for (int q = 0; q < col; ++q) v -= Dm[col * M + q] * Dm[col * M + q];
      if (!(v > 0.0)) {
        atomicExch(status, 1);
        v = 1e-300;
      }
      const double dgl = sqrt(v);
      Dm[col * M + col] = dgl;
      for (int r = col + 1; r < M; ++r) {
        double w = Dm[r * M + col];
        for (int q = 0; q < col; ++q) w -= Dm[r * M + q] * Dm[col * M + q];
        Dm[r * M + col] = w / dgl;
      }
    }
    // inverse of the lower-triangular factor (forward substitution on the
    // identity), packed by columns; Z_s with row stride zld(M)
    constexpr int LP = zlp(M), LDZ = zld(M), RS = zrec(M);
    float *Lf = fac + ((size_t)line * S + s) * RS;
    double *Ld = fac64 + ((size_t)line * S + s) * RS;
    for (int col = 0; col < M; ++col) {
      const int pc = zcol(M, col);
      for (int r = col; r < M; ++r) {
        double v;
        if (r == col) {
          v = 1.0 / Dm[r * M + r];
        } else {
          double acc = 0.0;
          for (int q = col; q < r; ++q) acc += Dm[r * M + q] * Ld[pc + (q - col)];
          v = -acc / Dm[r * M + r];
        }
        Ld[pc + (r - col)] = v;
        Lf[pc + (r - col)] = (float)v;
      }
    }
    for (int q = M * (M + 1) / 2; q < LP; ++q) { Lf[q] = 0.0f; Ld[q] = 0.0; }
    float *Zf = Lf + LP;
    double *Zd = Ld + LP;
    const double *Z = s > 0 ? blk + (((size_t)line * S + s - 1) * 2 + 1) * M * M : nullptr;
    for (int q = 0; q < zzp(M); ++q) {
      const int r = q / LDZ, col = q - r * LDZ;
      const double v = (Z && r < M && col < M) ? Z[r * M + col] : 0.0;
      Zf[q] = (float)v;
      Zd[q] = v;
    }
  }
}

// ---- bulk (TMA) copies global -> shared, completion counted on an mbarrier
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// one lane: announce `bytes` on bar, then start the copies that deliver them
__device__ __forceinline__ void mbar_expect(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// hint: bring `bytes` at src into L2 (no completion to wait for)
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// wait for the phase with parity `par` of bar to complete; false once
// limit_ns nanoseconds have passed without it (the copy never landed).
// try_wait may suspend the thread inside the hardware until the phase
// completes, which suits the usual limits; limits under kPollNs poll with the
// non-blocking test_wait so that the limit itself is honoured.
constexpr unsigned long long kPollNs = 100000ull;
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned par, unsigned long long limit_ns) {
  const bool poll = limit_ns < kPollNs;
  unsigned long long t0 = 0;
  for (bool first = true;; first = false) {
    unsigned ok;
    if (poll)
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(ok)
          : "r"(smem_u32(bar)), "r"(par)
          : "memory");
    else
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(ok)
          : "r"(smem_u32(bar)), "r"(par)
          : "memory");
    if (ok) return true;
    if (first) t0 = global_ns();
    else if (global_ns() - t0 > limit_ns) return false;
  }
}
// after a timed-out wait: the bound given to the copies still in flight
constexpr unsigned long long kDrainNs = 2000000000ull;
__device__ __forceinline__ unsigned long long wait_limit(const TnWait *w) {
  return w ? w->limit_ns : kDefaultWaitNs;
}

// shared memory of one warp: two stages of one factor record, two
// broadcast vectors of 32 entries, two mbarriers
template <int N, typename F>
__host__ __device__ constexpr int zline_warp_bytes() {
  return 2 * zrec(3 * N) * (int)sizeof(F) + 2 * 32 * (int)sizeof(F) + 16;
}
template <int N, typename F>
constexpr size_t zline_smem() { return (size_t)4 * zline_warp_bytes<N, F>(); }

// 16-byte broadcast read of entries c4 .. c4 + 16/sizeof(T) - 1 of a vector
// that every lane of the warp reads at once
template <typename T> struct Vec16;
template <> struct Vec16<float> {
  static constexpr int W = 4;
  __device__ static void load(const float *p, float *v) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
};
template <> struct Vec16<double> {
  static constexpr int W = 2;
  __device__ static void load(const double *p, double *v) {
    const double2 t = *reinterpret_cast<const double2 *>(p);
    v[0] = t.x; v[1] = t.y;
  }
};

// sum_cc A(cc) x_cc over cc < M with x read from the broadcast vector xv and
// A(cc) given by `ent` (three partial sums to shorten the dependent chain)
template <int M, typename T, typename Ent>
__device__ __forceinline__ T bcast_dot(const T *xv, Ent ent) {
  constexpr int W = Vec16<T>::W;
  T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int c4 = 0; c4 < M; c4 += W) {
    T v[W];
    Vec16<T>::load(xv + c4, v);
#pragma unroll
    for (int u = 0; u < W; ++u)
      if (c4 + u < M) acc[(c4 + u) % 3] += ent(c4 + u) * v[u];
  }
  return (acc[0] + acc[1]) + acc[2];
}

// z = A_LL^{-1} r on one line (one warp; lane l = a * N + k holds one unknown
// of a slab), with A_LL = L L^T block-bidiagonal:
//   forward   y_s = Linv_s (r_s - Z_s^T y_{s-1})      (y = L^{-1} r, kept in z)
//   backward  x_s = Linv_s^T (y_s - Z_{s+1} x_{s+1})  (x = L^{-T} y)
// Every product is a broadcast matrix-vector product.  The factor record of
// the next slab is brought into shared memory by one bulk copy while the
// current slab is worked on (two stages); this lane's r, q and y entries are
// loaded two slabs ahead into registers.  UPD: first r <- r - alpha q (the
// PCG residual update, written back).  Adds this lane's r.z (= |y|^2, since
// r.z = r^T L^-T L^-1 r) and r.r to rz, rr.  A staging wait that runs out
// sets *err and ends the line.
template <int N, typename T, typename F, bool UPD>
__device__ __forceinline__ void zline_line(const DevMesh &m, const F *__restrict__ fac, T *__restrict__ r,
                                           const T *__restrict__ q, T *__restrict__ z, T alpha, int line,
                                           int lane, unsigned char *smem, TnWait *err, T &rz, T &rr) {
  static_assert(sizeof(T) == sizeof(F), "vectors and factors share one precision");
  constexpr int M = 3 * N, N2 = N * N, n = N * N * N;
  constexpr int LP = zlp(M), LDZ = zld(M), RS = zrec(M);
  const int S = m.nslab;
  const int c = line / N2, qn = line - c * N2, i = qn % N, j = qn / N;
  const int a = lane / N, k = lane - (lane / N) * N;
  const bool act = lane < M;
  const int ll = act ? lane : 0;
  const size_t off = (size_t)k * N2 + j * N + i;
  const size_t ncol = m.ncol;
  const F *base = fac + (size_t)line * S * RS;
  F *const stg0 = reinterpret_cast<F *>(smem);
  T *const vb = reinterpret_cast<T *>(smem + 2 * RS * sizeof(F));  // b_s / y_s (broadcast)
  T *const vx = vb + 32;                                            // y_{s-1} / x_{s+1} (broadcast)
  unsigned long long *const bar =
      reinterpret_cast<unsigned long long *>(smem + 2 * RS * sizeof(F) + 64 * sizeof(F));
  unsigned ph = 0u, pend = 0u;  // bit b: phase parity / copy in flight of stage b
  auto stg = [&](int b) { return stg0 + b * RS; };
  auto gidx = [&](int s) { return ((size_t)(s * ncol + c) * 3 + (act ? a : 0)) * n + off; };
  auto issue = [&](int b, const F *src0, int cnt0, const F *src1, int cnt1) {
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_expect(bar + b, (unsigned)((cnt0 + cnt1) * sizeof(F)));
      bulk_g2s(stg(b), src0, (unsigned)(cnt0 * sizeof(F)), bar + b);
      if (cnt1) bulk_g2s(stg(b) + LP, src1, (unsigned)(cnt1 * sizeof(F)), bar + b);
    }
    pend |= 1u << b;
  };
  const unsigned long long lim = wait_limit(err);
  // the warp agrees on the outcome; a stage counts as landed only if every
  // lane saw it land, so that the lanes keep one view of the stages
  auto wait = [&](int b) {
    const bool ok = __all_sync(0xffffffffu, mbar_wait(bar + b, (ph >> b) & 1u, lim));
    if (ok) {
      ph ^= 1u << b;
      pend &= ~(1u << b);
    }
    return ok;
  };
  auto drain = [&]() {  // after a timeout: a bounded wait for every copy still in flight
    if (pend & 1u) mbar_wait(bar, ph & 1u, kDrainNs);
    if (pend & 2u) mbar_wait(bar + 1, (ph >> 1) & 1u, kDrainNs);
    if (lane == 0 && err) atomicExch(&err->flag, 1);
  };
  if (lane == 0) {
    mbar_init(bar);
    mbar_init(bar + 1);
    mbar_init_fence();
  }
  __syncwarp();
  // forward sweep
  issue(0, base, RS, nullptr, 0);
  T r0 = act ? r[gidx(0)] : T(0), q0 = (UPD && act) ? q[gidx(0)] : T(0);
  T r1 = (act && S > 1) ? r[gidx(1)] : T(0), q1 = (UPD && act && S > 1) ? q[gidx(1)] : T(0);
  T yprev = T(0);
  if (lane == 0 && S > 1) bulk_prefetch_l2(base + RS, RS * sizeof(F));
  for (int s = 0; s < S; ++s) {
    const int b = s & 1;
    // the record two slabs ahead goes to L2 now, so that its bulk copy (issued
    // at the next step) is served from L2
    if (lane == 0 && s + 2 < S) bulk_prefetch_l2(base + (size_t)(s + 2) * RS, RS * sizeof(F));
    if (s + 1 < S) issue(b ^ 1, base + (size_t)(s + 1) * RS, RS, nullptr, 0);
    if (!wait(b)) { drain(); return; }
    const F *Li = stg(b), *Zs = stg(b) + LP;
    const size_t idx = gidx(s);
    T rv = r0;
    if (UPD) {
      rv -= alpha * q0;
      if (act) r[idx] = rv;
    }
    // entries two slabs ahead
    r0 = r1;
    q0 = q1;
    if (act && s + 2 < S) {
      r1 = r[gidx(s + 2)];
      if (UPD) q1 = q[gidx(s + 2)];
    }
    rr += rv * rv;
    T bv = rv;
    if (s > 0) bv -= bcast_dot<M, T>(vx, [&](int cc) { return (T)Zs[cc * LDZ + ll]; });  // Z_s^T y_{s-1}
    vb[lane] = act ? bv : T(0);
    __syncwarp();
    T y = bcast_dot<M, T>(vb, [&](int cc) { return cc <= ll ? (T)Li[zcol(M, cc) + ll - cc] : T(0); });
    if (!act) y = T(0);
    rz += y * y;
    if (act) z[idx] = y;
    yprev = y;
    __syncwarp();  // every lane is done with vx, vb and stage b
    vx[lane] = y;
    __syncwarp();
  }
  // backward sweep: slab s needs Linv_s and Z_{s+1}
  auto issue_bwd = [&](int s, int b) {
    issue(b, base + (size_t)s * RS, LP, base + (size_t)(s + 1) * RS + LP, s + 1 < S ? RS - LP : 0);
  };
  const int pl = zcol(M, ll) - ll;
  int bb = S & 1;  // the stage the forward sweep did not end on
  issue_bwd(S - 1, bb);
  T y0 = yprev;  // y_{S-1}
  T y1 = (act && S > 1) ? z[gidx(S - 2)] : T(0);
  T y2 = (act && S > 2) ? z[gidx(S - 3)] : T(0);
  if (lane == 0 && S > 1) bulk_prefetch_l2(base + (size_t)(S - 2) * RS, RS * sizeof(F));
  for (int s = S - 1; s >= 0; --s, bb ^= 1) {
    if (lane == 0 && s >= 2) bulk_prefetch_l2(base + (size_t)(s - 2) * RS, RS * sizeof(F));
    if (s > 0) issue_bwd(s - 1, bb ^ 1);
    if (!wait(bb)) { drain(); return; }
    const F *Li = stg(bb), *Zn = stg(bb) + LP;
    T yv = y0;
    y0 = y1;
    y1 = y2;
    if (act && s >= 3) y2 = z[gidx(s - 3)];
    if (s + 1 < S) yv -= bcast_dot<M, T>(vx, [&](int cc) { return (T)Zn[ll * LDZ + cc]; });  // Z_{s+1} x_{s+1}
    vb[lane] = act ? yv : T(0);
    __syncwarp();
    T x = bcast_dot<M, T>(vb, [&](int cc) { return cc >= ll ? (T)Li[pl + cc] : T(0); });
    if (!act) x = T(0);
    if (act) z[gidx(s)] = x;
    __syncwarp();  // every lane is done with vx, vb and stage bb
    vx[lane] = x;
    __syncwarp();
  }
}

// four lines (warps) per block; per-block partial sums of r.z and r.r
__device__ __forceinline__ void block_partial2(double rz, double rr, double *part_rz, double *part_rr) {
  __shared__ double red[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rz += __shfl_xor_sync(0xffffffffu, rz, o);
    rr += __shfl_xor_sync(0xffffffffu, rr, o);
  }
  if (lane == 0) { red[warp] = rz; red[4 + warp] = rr; }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (part_rz) part_rz[blockIdx.x] = red[0] + red[1] + red[2] + red[3];
    if (part_rr) part_rr[blockIdx.x] = red[4] + red[5] + red[6] + red[7];
  }
}

template <int N, typename T, typename F, bool UPD>
__global__ void __launch_bounds__(128)
zline_solve_kernel(const DevMesh m, const F *__restrict__ fac, T *__restrict__ r, const T *__restrict__ q,
                   T *__restrict__ z, const double *__restrict__ alpha, double *__restrict__ part_rz,
                   double *__restrict__ part_rr, const int *__restrict__ done, TnWait *__restrict__ err) {
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char zsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int line = blockIdx.x * 4 + warp;
  const T al = UPD ? (T)*alpha : T(0);
  T rz = T(0), rr = T(0);
  if (line < m.ncol * N * N)
    zline_line<N, T, F, UPD>(m, fac, r, q, z, al, line, lane, zsm + warp * zline_warp_bytes<N, F>(), err, rz,
                             rr);
  block_partial2((double)rz, (double)rr, part_rz, part_rr);
}

// a batch: warp w of block b handles line work[4 b + w] = (instance, line)
template <int N, typename T, typename F, bool UPD>
__global__ void __launch_bounds__(128)
zline_solve_batch_kernel(const DevMesh *__restrict__ meshes, const int2 *__restrict__ work, int nwork,
                         const long long *__restrict__ fac_off, const long long *__restrict__ dof_off,
                         const F *__restrict__ fac, T *__restrict__ r, const T *__restrict__ q,
                         T *__restrict__ z, const double *__restrict__ alpha, double *__restrict__ part_rz,
                         double *__restrict__ part_rr, const int *__restrict__ done, TnWait *__restrict__ err) {
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char zsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wi = blockIdx.x * 4 + warp;
  const T al = UPD ? (T)*alpha : T(0);
  T rz = T(0), rr = T(0);
  if (wi < nwork) {
    const int2 w = work[wi];
    const long long off = dof_off[w.x];
    zline_line<N, T, F, UPD>(meshes[w.x], fac + fac_off[w.x], r + off, UPD ? q + off : nullptr, z + off, al,
                             w.y, lane, zsm + warp * zline_warp_bytes<N, F>(), err, rz, rr);
  }
  block_partial2((double)rz, (double)rr, part_rz, part_rr);
}

// ---------------------------------------------------------------- line groups
// The lines through the matching nodes of two columns that share a lateral
// face are coupled by that face's interior-penalty and flux terms (Eqs.
// (numflux), (penalty)), which the single-line blocks leave out; with the
// penalty ~ C (p + 1)^2 / h these are the stiffest couplings left.  A group
// is a set of lines joined by such face matches (1 to 4 lines: a node inside
// a column face, on a column edge or at a corner where up to four columns
// meet); its block is the exact principal sub-matrix of A on all its lines,
// again block tridiagonal over the slabs, with 3 g N unknowns per slab and
// the cross-line face terms in the diagonal blocks.

// Cross-line block of element e = (s, c), lateral face f and face position t:
// rows = the line through the face node (this element), columns = the line
// through the matching node of the neighbour column (same slab):
//   -1/2 V^T W Tr_ext + 1/2 Tr^T W V_ext - V^T W Pen V_ext
// restricted to the two lines (the neighbour's traction and this element's
// test traction reduce to the zeta derivative and the diagonal xi / eta
// derivative entries on a line).  Zero where f has no neighbour.
template <int N>
__global__ void zgroup_cross_kernel(const DevMesh m, double *__restrict__ xblk) {
  constexpr int M = 3 * N, N2 = N * N;
  const int e = blockIdx.x, t = threadIdx.x % N, f = threadIdx.x / N;
  if (f >= 4) return;
  const int s = e / m.ncol, c = e - s * m.ncol;
  double *X = xblk + (((size_t)e * 4 + f) * N + t) * M * M;
  for (int q = 0; q < M * M; ++q) X[q] = 0.0;
  const int nbc = m.colnb[4 * c + f];
  if (nbc < 0) return;
  const int d = f >> 1, sd = f & 1, end = sd ? N - 1 : 0;
  const int i = d == 0 ? end : t, j = d == 0 ? t : end;
  const int code = m.colnbf[4 * c + f];
  const int f2 = code & 3, d2 = f2 >> 1, end2 = (f2 & 1) ? N - 1 : 0;
  const int a2 = (code >> 2) ? N - 1 - t : t;
  const int i2 = d2 == 0 ? end2 : a2, j2 = d2 == 0 ? a2 : end2;
  const double *cg = m.colgeo + (size_t)c * CG_NF * N2;
  const double *cg2 = m.colgeo + (size_t)nbc * CG_NF * N2;
  const int q1 = j * N + i, q2 = j2 * N + i2;
  const double ixx = cg[CG_IXX * N2 + q1], ixy = cg[CG_IXY * N2 + q1];
  const double iex = cg[CG_IEX * N2 + q1], iey = cg[CG_IEY * N2 + q1], det2 = cg[CG_DET * N2 + q1];
  const double jxx = cg2[CG_IXX * N2 + q2], jxy = cg2[CG_IXY * N2 + q2];
  const double jex = cg2[CG_IEX * N2 + q2], jey = cg2[CG_IEY * N2 + q2];
  const double *sg = m.slabgeo + (size_t)s * SG_NF * N;
  double dz[N];
  for (int k = 0; k < N; ++k) dz[k] = sg[SG_DZ * N + k];
  const int L = m.slab_layer[s];  // both sides lie in slab s: one material
  const double c11 = m.layer_c[3 * L], c12 = m.layer_c[3 * L + 1], c44 = m.layer_c[3 * L + 2];
  const double rx = d == 0 ? ixx : iex, ry = d == 0 ? ixy : iey;
  const double mag = sqrt(rx * rx + ry * ry);
  const double n[3] = {(sd ? 1.0 : -1.0) * rx / mag, (sd ? 1.0 : -1.0) * ry / mag, 0.0};
  const double sx = d2 == 0 ? jxx : jex, sy = d2 == 0 ? jxy : jey;
  const double h = 2.0 / mag, h2 = 2.0 / sqrt(sx * sx + sy * sy);
  const double sig = (double)((m.p + 1) * (m.p + 1)) * m.penC / (h < h2 ? h : h2);
  const double Dii = LD(i, i), Djj = LD(j, j), Dii2 = LD(i2, i2), Djj2 = LD(j2, j2);
  const double wt = d == 0 ? LW(j) : LW(i);
  for (int k = 0; k < N; ++k) {
    const double Wk = wt * LW(k) * det2 * dz[k] * mag;
    for (int k2 = 0; k2 < N; ++k2) {
      const double Wk2 = wt * LW(k2) * det2 * dz[k2] * mag;
      // neighbour basis (i2, j2, k2) at its node (i2, j2, k); own basis (i, j, k) at (i, j, k2)
      const double l2[3] = {k2 == k ? Dii2 : 0.0, k2 == k ? Djj2 : 0.0, LD(k, k2)};
      const double l1[3] = {k == k2 ? Dii : 0.0, k == k2 ? Djj : 0.0, LD(k2, k)};
      double g2[3], g1[3];
      phys(l2, jxx, jxy, jex, jey, dz[k], g2);
      phys(l1, ixx, ixy, iex, iey, dz[k2], g1);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double v = -0.5 * Wk * Qab(a, b, n, g2, c11, c12, c44) + 0.5 * Wk2 * Qab(b, a, n, g1, c11, c12, c44);
          if (k == k2) v -= Wk * sig * Qab(a, b, n, n, c11, c12, c44);
          X[(a * N + k) * M + b * N + k2] = v;
        }
    }
  }
}

// Group record of slab s: [S_s^{-1} packed by columns (lower triangle,
// zlp(MG)) | O_{s-1} in factored form (8 MG) | W_s], S_s = L_s L_s^T the
// slab's Schur complement of the block Cholesky (S_s^{-1} = Linv_s^T
// Linv_s).  The coupling block O_{s-1} (rows: slab s - 1,
// columns: slab s, block diagonal over the lines) is nonzero only in the
// rows of the bottom-face nodes (k = 0) and the columns of the top-face
// nodes (k2 = N - 1) of each line (Eqs. (numflux), (penalty) on the zeta
// face), so O = E_0 X^T + Y E_{N-1}^T with per row t: X[t][a] = O[(a, 0), t]
// and Y[t][b] = O[t, (b, N - 1)] (Y zero on k = 0 rows).  Row t stores
// X[t][0..2], 0, Y[t][0..2], 0.  The solve applies the coupling through
// these factors instead of storing Z_s = Linv_{s-1} O_{s-1} densely.
// The record ends with the backward sweep's coupling W_s = S_s^{-1} [Y_s | E_0]
// (MG x 6G, rows padded to zg_ws(G)), S_s = L_s L_s^T the slab's Schur
// complement and Y_s, E_0 of O_s (the coupling to slab s + 1): per line l,
// column 6 l + b holds Y of component b and column 6 l + 3 + a the unit
// vector of row (a, k = 0); zero for the last slab.  With it the backward
// step x_s = Linv_s^T (y_s - Linv_s O_s x_{s+1}) = w_s - W_s v, v the six
// numbers per line x_{s+1}(b, N - 1) and X^T x_{s+1}.
__host__ __device__ constexpr int zg_ws(int G) { return pad4(6 * G); }
__host__ __device__ constexpr int zg_rec(int MG, int G) { return zlp(MG) + 8 * MG + MG * zg_ws(G); }

// block Cholesky along the slabs of one group (one CTA; FP64 working
// matrices G and Linv of (3 g N)^2 entries each and the (6 g)^2 C in
// `work`), then FP32 and FP64 records [S_s^{-1} packed | O_{s-1} factors |
// W_s]
template <int N>
__global__ void __launch_bounds__(128)
zgroup_factor_kernel(const DevMesh m, const int4 *__restrict__ glines, const long long *__restrict__ gfac,
                     int gbase, int g, const double *__restrict__ blk, const double *__restrict__ xblk,
                     double *__restrict__ work, float *__restrict__ fac, double *__restrict__ fac64,
                     int *__restrict__ status) {
  constexpr int M = 3 * N, N2 = N * N;
  const int grp = gbase + blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  const int MG = g * M, S = m.nslab;
  const int LP = zlp(MG), RS = zg_rec(MG, g), WS = zg_ws(g);
  double *Gm = work + (size_t)blockIdx.x * 3 * MG * MG, *Li = Gm + MG * MG, *Cm = Li + MG * MG;
  __shared__ int lid[4], xof[4][4];
  if (tid < 4) {
    const int4 L4 = glines[grp];
    lid[tid] = tid == 0 ? L4.x : (tid == 1 ? L4.y : (tid == 2 ? L4.z : L4.w));
  }
  __syncthreads();
  if (tid < 16) {  // which face block couples line t1 (rows) to line t2 (columns)
    const int t1 = tid >> 2, t2 = tid & 3;
    int x = -1;
    if (t1 < g && t2 < g && t1 != t2) {
      const int c1 = lid[t1] / N2, qq = lid[t1] - c1 * N2, i1 = qq % N, j1 = qq / N;
      for (int f = 0; f < 4; ++f) {
        const int nbc = m.colnb[4 * c1 + f];
        const int d = f >> 1, end = (f & 1) ? N - 1 : 0;
        if (nbc < 0 || (d == 0 ? i1 : j1) != end) continue;
        const int tp = d == 0 ? j1 : i1;
        const int code = m.colnbf[4 * c1 + f], f2 = code & 3, d2 = f2 >> 1, end2 = (f2 & 1) ? N - 1 : 0;
        const int a2 = (code >> 2) ? N - 1 - tp : tp;
        const int i2 = d2 == 0 ? end2 : a2, j2 = d2 == 0 ? a2 : end2;
        if (nbc * N2 + j2 * N + i2 == lid[t2]) x = f * N + tp;
      }
    }
    xof[t1][t2] = x;
  }
  __syncthreads();
  const long long rec0 = gfac[grp];
  for (int s = 0; s < S; ++s) {
    // Schur complement of slab s: the diagonal block (line blocks, cross-line
    // face blocks) minus O_{s-1}^T S_{s-1}^{-1} O_{s-1}.  With O_{s-1} = U V^T,
    // U = [Y | E_0] (slab s - 1) and V = [E_{N-1} | X] (slab s), columns
    // paired as in W_{s-1} = S_{s-1}^{-1} U, that is V C V^T with the 6g x 6g
    // C = U^T W_{s-1}; a row of V has at most four nonzeros
    const int G6 = 6 * g;
    if (s > 0) {
      const double *Wp = fac64 + rec0 + (long long)(s - 1) * RS + LP + 8 * MG;
      for (int q = tid; q < G6 * G6; q += nth) {
        const int i = q / G6, j = q - i * G6, l = i / 6, ii = i - l * 6;
        double acc = 0.0;
        if (ii < 3) {  // Y of component b = ii: O_{s-1}[p, (b, N - 1)] on the rows p of line l with k != 0
          const double *O = blk + (((size_t)lid[l] * S + (s - 1)) * 2 + 1) * M * M;
          for (int pl = 0; pl < M; ++pl)
            if (pl % N != 0) acc += O[pl * M + ii * N + (N - 1)] * Wp[(size_t)(l * M + pl) * WS + j];
        } else {  // E_0: row (a, k = 0) of line l
          acc = Wp[(size_t)(l * M + (ii - 3) * N) * WS + j];
        }
        Cm[q] = acc;
      }
      __syncthreads();
    }
    for (int q = tid; q < MG * MG; q += nth) {
      const int r = q / MG, cc = q - r * MG, t1 = r / M, t2 = cc / M, rr = r - t1 * M, c2 = cc - t2 * M;
      double v = 0.0;
      if (t1 == t2) {
        v = blk[(((size_t)lid[t1] * S + s) * 2 + 0) * M * M + rr * M + c2];
      } else if (xof[t1][t2] >= 0) {
        const size_t e = (size_t)s * m.ncol + lid[t1] / N2;
        v = xblk[(e * 4 * N + xof[t1][t2]) * M * M + rr * M + c2];
      }
      if (s > 0) {  // the nonzeros of V's rows r and cc: (column, value)
        int ir[4], ic[4];
        double vr[4], vc[4];
        int nr = 0, nc = 0;
        const double *Or = blk + (((size_t)lid[t1] * S + (s - 1)) * 2 + 1) * M * M;
        const double *Oc = blk + (((size_t)lid[t2] * S + (s - 1)) * 2 + 1) * M * M;
        if (rr % N == N - 1) { ir[nr] = 6 * t1 + rr / N; vr[nr++] = 1.0; }
        if (c2 % N == N - 1) { ic[nc] = 6 * t2 + c2 / N; vc[nc++] = 1.0; }
        for (int a = 0; a < 3; ++a) {
          ir[nr] = 6 * t1 + 3 + a; vr[nr++] = Or[(a * N) * M + rr];  // X[r][a] = O_{s-1}[(a, 0), r]
          ic[nc] = 6 * t2 + 3 + a; vc[nc++] = Oc[(a * N) * M + c2];
        }
        double sum = 0.0;
        for (int x = 0; x < nr; ++x) {
          double row = 0.0;
          for (int y = 0; y < nc; ++y) row += Cm[ir[x] * G6 + ic[y]] * vc[y];
          sum += vr[x] * row;
        }
        v -= sum;
      }
      Gm[q] = v;
    }
    __syncthreads();
    // Cholesky, lower triangle in place
    for (int col = 0; col < MG; ++col) {
      if (tid == 0) {
        double dv = Gm[col * MG + col];
        if (!(dv > 0.0)) {
          atomicExch(status, 1);
          dv = 1e-300;
        }
        Gm[col * MG + col] = sqrt(dv);
      }
      __syncthreads();
      const double piv = Gm[col * MG + col];
      for (int r = col + 1 + tid; r < MG; r += nth) Gm[r * MG + col] /= piv;
      __syncthreads();
      const int w = MG - col - 1;
      for (int q = tid; q < w * w; q += nth) {
        const int r = col + 1 + q / w, c2 = col + 1 + q % w;
        if (c2 <= r) Gm[r * MG + c2] -= Gm[r * MG + col] * Gm[c2 * MG + col];
      }
      __syncthreads();
    }
    // Linv = L^{-1}, one column per thread (forward substitution on the
    // identity); its upper triangle is zero (read by the products below)
    for (int cc = tid; cc < MG; cc += nth) {
      for (int r = 0; r < cc; ++r) Li[r * MG + cc] = 0.0;
      for (int r = cc; r < MG; ++r) {
        double acc = r == cc ? 1.0 : 0.0;
        for (int p = cc; p < r; ++p) acc -= Gm[r * MG + p] * Li[p * MG + cc];
        Li[r * MG + cc] = acc / Gm[r * MG + r];
      }
    }
    __syncthreads();
    float *Lf = fac + rec0 + (long long)s * RS;
    double *Ld = fac64 + rec0 + (long long)s * RS;
    for (int q = tid; q < MG * MG; q += nth) {  // S^{-1} = Linv^T Linv, lower triangle
      const int r = q / MG, cc = q - r * MG;
      if (r >= cc) {
        double acc = 0.0;
        for (int p = r; p < MG; ++p) acc += Li[p * MG + r] * Li[p * MG + cc];
        const int pi = zcol(MG, cc) + r - cc;
        Ld[pi] = acc;
        Lf[pi] = (float)acc;
      }
    }
    for (int q = MG * (MG + 1) / 2 + tid; q < LP; q += nth) { Lf[q] = 0.0f; Ld[q] = 0.0; }
    for (int q = tid; q < 8 * MG; q += nth) {  // factors of O_{s-1}
      const int t = q >> 3, j = q & 7, l = t / M, tl = t - l * M, tk = tl % N;
      double v = 0.0;
      if (s > 0 && (j & 3) < 3) {
        const double *O = blk + (((size_t)lid[l] * S + (s - 1)) * 2 + 1) * M * M;
        if (j < 4) v = O[(j * N) * M + tl];                        // X[t][a] = O[(a, 0), t]
        else if (tk != 0) v = O[tl * M + (j - 4) * N + (N - 1)];  // Y[t][b] = O[t, (b, N - 1)]
      }
      Lf[LP + q] = (float)v;
      Ld[LP + q] = v;
    }
    __syncthreads();
    // W_s = Linv_s^T (Linv_s [Y_s | E_0]); L (in Gm) is no longer needed
    double *T1 = Gm;  // MG x 6g
    if (s + 1 < S) {
      for (int q = tid; q < MG * 6 * g; q += nth) {
        const int r = q / (6 * g), j = q - r * (6 * g), l = j / 6, jj = j - l * 6;
        double acc = 0.0;
        if (jj < 3) {  // Y of O_s, component b = jj: O_s[p, (b, N - 1)] on the rows p of line l with k != 0
          const double *O = blk + (((size_t)lid[l] * S + s) * 2 + 1) * M * M;
          for (int pl = 0; pl < M; ++pl)
            if (pl % N != 0) acc += Li[r * MG + l * M + pl] * O[pl * M + jj * N + (N - 1)];
        } else {  // E_0 of row (a, k = 0) of line l: a column of Linv
          acc = Li[r * MG + l * M + (jj - 3) * N];
        }
        T1[q] = acc;
      }
      __syncthreads();
    }
    for (int q = tid; q < MG * WS; q += nth) {
      const int t = q / WS, j = q - t * WS;
      double acc = 0.0;
      if (s + 1 < S && j < 6 * g)
        for (int r = t; r < MG; ++r) acc += Li[r * MG + t] * T1[r * 6 * g + j];
      Lf[LP + 8 * MG + q] = (float)acc;
      Ld[LP + 8 * MG + q] = acc;
    }
    __syncthreads();
  }
}

// ---- the grouped-line solve: packed slots, one launch per degree
// A group of G lines (3 G N rows per slab) is solved by a slot of G warps,
// one row per thread.  A CTA of four warps takes one pack at a time from a
// queue: one group of 4 lines, 3 + 1, 2 + 2, 2 + 1 + 1 or 1 + 1 + 1 + 1
// lines, largest packs first.  Each slot syncs with its own named barrier
// (a warp with __syncwarp) and streams its factor records through a ring of
// P stages in shared memory (bulk copies completing on one mbarrier per
// stage), so that up to P - 1 copies are in flight while one stage is used:
// small groups, whose per-slab work is short, get the deepest rings.
constexpr int kZgThreads = 128;  // four warps per CTA
constexpr int kZgMaxStages = 8;

// floats / doubles of staging per warp: two records of the largest group
// (4 lines) across the four warps of a CTA, so that six CTAs (FP32, N = 7)
// share an SM; smaller groups fit more stages in the same room
// stage buffer of a group of G lines: the larger of the forward stage
// (S_s^{-1} and the O factors of record s) and the backward stage (W_s and
// the O factors of record s + 1)
template <int N, int G>
__host__ __device__ constexpr int zg_stage() {
  return (zlp(3 * G * N) > 3 * G * N * zg_ws(G) ? zlp(3 * G * N) : 3 * G * N * zg_ws(G)) + 8 * 3 * G * N;
}
template <int N, typename T>
__host__ __device__ constexpr int zg_stage_per_warp() {
  return pad4((zg_stage<N, 4>() * 2 + 3) / 4);
}
template <int N, typename T>
constexpr size_t zg_smem() {
  return (4 * (size_t)zg_stage_per_warp<N, T>() + 4 * kZgThreads) * sizeof(T) + 4 * kZgMaxStages * 8;
}

__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}
// true if p holds on any of the nthreads threads of named barrier id (and a sync)
__device__ __forceinline__ bool named_any(int id, int nthreads, bool p) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred q, o;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred o, %2, %3, q;\n selp.u32 %0, 1, 0, o;\n}\n"
      : "=r"(r)
      : "r"((unsigned)p), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void mbar_inval(unsigned long long *bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// three warp-wide sums at once: the three butterflies interleaved level by
// level, so that their shuffles overlap instead of running one sum after
// the other (every lane gets the three sums)
template <typename T>
__device__ __forceinline__ void warp_allsum3(T &a, T &b, T &c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T a2 = __shfl_xor_sync(0xffffffffu, a, o);
    const T b2 = __shfl_xor_sync(0xffffffffu, b, o);
    const T c2 = __shfl_xor_sync(0xffffffffu, c, o);
    a += a2;
    b += b2;
    c += c2;
  }
}

// z = A_GG^{-1} r on group grp by the slot of G warps starting at warp w0;
// line li of the group is warp w0 + li, its rows (a, k) lanes a N + k < 3N:
//   forward   y_s = Linv_s (r_s - O_{s-1}^T w_{s-1}),  w_s = Linv_s^T y_s
//   backward  x_s = Linv_s^T (y_s - Linv_s O_s x_{s+1}) = w_s - W_s v_{s+1}
// (v: six numbers per line, x_{s+1}(b, N - 1) and X^T x_{s+1}).  The forward
// step forms w_s = S_s^{-1} b_s, b_s = r_s - O_{s-1}^T w_{s-1}, in one
// symmetric product, and r.z = sum_s |y_s|^2 = sum_s b_s . w_s.  O in its
// factored form acts line by line (it is block diagonal over the lines), so
// its products are warp shuffles and warp sums; S_s^{-1} b_s and W_s v cross
// lines, through broadcast vectors in shared memory (double-buffered by step
// parity).  Stage u < S: S_u^{-1} and the O factors of record u; stage u >= S:
// W_s of record s and the O factors of record s + 1, s = 2S - 2 - u.  Stage u
// uses ring buffer u % P and mbarrier u % P with phase parity (u / P) & 1.
// Writes the group's partial r.z (= |y|^2) and r.r.  A wait that runs
// out sets err->flag and ends the slot after bounded waits for the copies in
// flight.
template <int N, int G, typename T>
__device__ __forceinline__ void zg_slot(int grp, int w0, int mncol, int S, const T *__restrict__ r,
                                        T *__restrict__ z, const int4 *__restrict__ glines,
                                        const long long *__restrict__ gfac, const T *__restrict__ fac,
                                        T *__restrict__ stage, int cap, T *__restrict__ vecs,
                                        unsigned long long *__restrict__ bars, double *__restrict__ psum,
                                        unsigned long long lim, TnWait *__restrict__ err, double *__restrict__ part_rz,
                                        double *__restrict__ part_rr) {
  constexpr int M = 3 * N, N2 = N * N, n = N * N * N, MG = G * M, NT = 32 * G;
  constexpr int LP = zlp(MG), RS = zg_rec(MG, G), WS = zg_ws(G), RSS = zg_stage<N, G>();
  constexpr int LPX = LP + 8 * MG;  // forward stage: S_s^{-1} and the O factors of record s
  constexpr int BW = MG * WS;       // backward stage: W_s, then the O factors of record s + 1
  const int lt = threadIdx.x - 32 * w0, bid = 1 + w0;
  auto sync = [&]() {
    if (G == 1) __syncwarp();
    else named_sync(bid, NT);
  };
  auto any = [&](bool p) { return G == 1 ? __any_sync(0xffffffffu, p) : named_any(bid, NT, p); };
  const int li = lt >> 5, lane = lt & 31;
  const bool act = lane < M;
  const int t = li * M + (act ? lane : 0);  // row of the group's blocks
  const int a = (act ? lane : 0) / N, k = (act ? lane : 0) - a * N;
  // broadcast vectors hold line lj's M entries at 32 lj (16-byte aligned)
  T *const vbuf = vecs + 4 * 32 * w0;  // [2 parities][vb][32 G] (room for 2 x 2 x 32 G)
  auto vb = [&](int par) { return vbuf + par * 2 * NT; };
  const int4 L4 = glines[grp];
  const int lid = li == 0 ? L4.x : (li == 1 ? L4.y : (li == 2 ? L4.z : L4.w));
  const int c = lid / N2, qn = lid - c * N2;
  // vector entry of this row in slab s: g0 + s * gs
  const size_t gs = (size_t)mncol * 3 * n, g0 = ((size_t)c * 3 + a) * n + (size_t)k * N2 + qn;
  auto gidx = [&](int s) { return g0 + (size_t)s * gs; };
  const T *base = fac + gfac[grp];
  const int total = 2 * S;
  int P = cap / RSS;
  P = P > kZgMaxStages ? kZgMaxStages : P;
  P = P > total ? total : P;
  // stage sources: forward stage u = S_u^{-1} and O factors of record u;
  // backward stage u (slab s = 2S - 2 - u < S - 1) = W_s of record s and the
  // O factors of record s + 1 (the last slab, s = S - 1, needs no stage)
  const int total_st = 2 * S - 1;
  int issued = 0, ib = 0;  // stages issued so far and the ring buffer of the next (same in every thread)
  const T *src = base;     // lane 0: the next stage's (first) source
  auto issue_next = [&]() {
    if (issued >= total_st) return;
    const int u = issued++, b = ib;
    ib = ib + 1 == P ? 0 : ib + 1;
    if (lt == 0) {
      T *dst = stage + (size_t)b * RSS;
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      if (u < S) {
        mbar_expect(bars + b, (unsigned)(LPX * sizeof(T)));
        bulk_g2s(dst, src, (unsigned)(LPX * sizeof(T)), bars + b);
        src = u + 1 < S ? src + RS : src - RS;  // then the backward stages from record S - 2 down
      } else {
        mbar_expect(bars + b, (unsigned)((BW + 8 * MG) * sizeof(T)));
        bulk_g2s(dst, src + LPX, (unsigned)(BW * sizeof(T)), bars + b);
        bulk_g2s(dst + BW, src + RS + LP, (unsigned)(8 * MG * sizeof(T)), bars + b);
        src -= RS;
      }
    }
  };
  // the slot agrees on the outcome (a barrier of the slot): a stage counts
  // as landed only if every thread saw it land.  wb / wpar: ring buffer and
  // phase parity of the stage waited for next (stage u: u % P, (u / P) & 1)
  int wb = 0;
  unsigned wpar = 0u;
  auto wait = [&]() {
    const bool ok = !any(!mbar_wait(bars + wb, wpar, lim));
    if (G == 1) __syncwarp();  // memory order across the warp, as the named barrier gives
    return ok;
  };
  auto wait_done = [&]() {  // advance to the next stage
    if (++wb == P) {
      wb = 0;
      wpar ^= 1u;
    }
  };
  if (lt == 0) {
    for (int b = 0; b < P; ++b) mbar_init(bars + b);
    mbar_init_fence();
  }
  sync();
  for (int u = 0; u + 1 < P; ++u) issue_next();
  T rz = T(0), rr = T(0);
  bool bad = false;
  int at = 0;  // the stage being waited for
  const int pl = zcol(MG, t) - t;
  // w = S^{-1} v, line block by line block, the block index a compile-time
  // constant so that every packed offset folds: row t of the symmetric
  // S^{-1} is the stored lower triangle's row t (blocks before this thread's
  // line, and its own block up to the diagonal) followed by its column t
  // (its own block below the diagonal, and the blocks after it)
  const int tl = act ? lane : 0;  // row within the line
  auto lblock = [&](const T *Ls, const T *v, auto LJ) {
    constexpr int c0 = decltype(LJ)::value * M;
    return bcast_dot<M, T>(v + 32 * decltype(LJ)::value,
                           [&](int cc) { return Ls[zcol(MG, c0 + cc) + t - c0 - cc]; });
  };
  auto ublock = [&](const T *Ls, const T *v, auto LJ) {
    constexpr int c0 = decltype(LJ)::value * M;
    return bcast_dot<M, T>(v + 32 * decltype(LJ)::value, [&](int cc) { return Ls[pl + c0 + cc]; });
  };
  auto dblock = [&](const T *Ls, const T *v, auto LJ) {
    constexpr int c0 = decltype(LJ)::value * M;
    return bcast_dot<M, T>(v + 32 * decltype(LJ)::value, [&](int cc) {
      return cc <= tl ? Ls[zcol(MG, c0 + cc) + t - c0 - cc] : Ls[pl + c0 + cc];
    });
  };
  auto symrow = [&](const T *Ls, const T *v) {
    T acc = T(0);
    auto part = [&](auto LJ) {
      constexpr int J = decltype(LJ)::value;
      if (J >= G) return;
      if (J < li) acc += lblock(Ls, v, LJ);
      else if (J == li) acc += dblock(Ls, v, LJ);
      else acc += ublock(Ls, v, LJ);
    };
    part(std::integral_constant<int, 0>{});
    part(std::integral_constant<int, 1>{});
    part(std::integral_constant<int, 2>{});
    part(std::integral_constant<int, 3>{});
    return acc;
  };
  // forward sweep
  T r0 = act ? r[gidx(0)] : T(0);
  T r1 = (act && S > 1) ? r[gidx(1)] : T(0);
  T w = T(0);
  for (int s = 0; s < S; ++s, ++at) {
    if (!wait()) { bad = true; break; }
    const T *Ls = stage + (size_t)wb * RSS, *XY = Ls + LP + 8 * t;
    wait_done();
    issue_next();  // every thread is past step s - 1: its buffer is free
    const int par = s & 1;
    const T rv = r0;
    r0 = r1;
    if (act && s + 2 < S) r1 = r[gidx(s + 2)];
    rr += rv * rv;
    T bv = rv;
    if (s > 0) {  // bv -= (O_{s-1}^T w_{s-1})_t, line by line
      const T x0 = XY[0], x1 = XY[1], x2 = XY[2];
      T s0 = act ? XY[4] * w : T(0), s1 = act ? XY[5] * w : T(0), s2 = act ? XY[6] * w : T(0);
      warp_allsum3(s0, s1, s2);
      T o = x0 * __shfl_sync(0xffffffffu, w, 0) + x1 * __shfl_sync(0xffffffffu, w, N) +
            x2 * __shfl_sync(0xffffffffu, w, 2 * N);
      if (k == N - 1) o += a == 0 ? s0 : (a == 1 ? s1 : s2);
      bv -= o;
    }
    if (act) vb(par)[lt] = bv;
    sync();
    w = symrow(Ls, vb(par));  // w_s = S_s^{-1} bv = Linv_s^T y_s
    if (!act) w = T(0);
    rz += bv * w;             // |y_s|^2
    if (act) z[gidx(s)] = w;  // read back by the backward sweep
  }
  // backward sweep: x_{S-1} = w_{S-1} (already in z), then
  // x_s = w_s - W_s v_{s+1}, v per line: x_{s+1}(b, N - 1) and X^T x_{s+1}
  if (!bad) {
    T x = w;
    T w1 = (act && S > 1) ? z[gidx(S - 2)] : T(0);
    T w2 = (act && S > 2) ? z[gidx(S - 3)] : T(0);
    for (int s = S - 2; s >= 0; --s, ++at) {
      if (!wait()) { bad = true; break; }
      const T *Ws = stage + (size_t)wb * RSS, *XY = Ws + BW + 8 * t;
      wait_done();
      issue_next();
      const int par = s & 1;
      const T wv = w1;
      w1 = w2;
      if (act && s >= 2) w2 = z[gidx(s - 2)];
      const T e0 = __shfl_sync(0xffffffffu, x, N - 1);
      const T e1 = __shfl_sync(0xffffffffu, x, 2 * N - 1);
      const T e2 = __shfl_sync(0xffffffffu, x, 3 * N - 1);
      T c0 = act ? XY[0] * x : T(0), c1 = act ? XY[1] * x : T(0), c2 = act ? XY[2] * x : T(0);
      warp_allsum3(c0, c1, c2);
      if (lane < 6) vb(par)[32 * li + lane] = lane < 3 ? (lane == 0 ? e0 : (lane == 1 ? e1 : e2))
                                                      : (lane == 3 ? c0 : (lane == 4 ? c1 : c2));
      sync();
      const T *Wr = Ws + t * WS;
      T acc = T(0);
#pragma unroll
      for (int l = 0; l < G; ++l) {
        const T *vl = vb(par) + 32 * l;
        acc += (Wr[6 * l] * vl[0] + Wr[6 * l + 1] * vl[1] + Wr[6 * l + 2] * vl[2]) +
               (Wr[6 * l + 3] * vl[3] + Wr[6 * l + 4] * vl[4] + Wr[6 * l + 5] * vl[5]);
      }
      x = act ? wv - acc : T(0);
      if (act) z[gidx(s)] = x;
    }
  }
  if (bad) {  // a copy never landed: bounded waits for every copy in flight, then report
    for (int u = at; u < issued; ++u) {
      mbar_wait(bars + wb, wpar, kDrainNs);
      wait_done();
    }
    if (lt == 0 && err) atomicExch(&err->flag, 1);
  }
  // the group's partial sums, in a fixed order
  double vrz = (double)rz, vrr = (double)rr;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    vrz += __shfl_xor_sync(0xffffffffu, vrz, o);
    vrr += __shfl_xor_sync(0xffffffffu, vrr, o);
  }
  if (lane == 0) {
    psum[(w0 + li) * 2] = vrz;
    psum[(w0 + li) * 2 + 1] = vrr;
  }
  sync();
  if (lt == 0) {
    double srz = 0.0, srr = 0.0;
    for (int ww = 0; ww < G; ++ww) {
      srz += psum[(w0 + ww) * 2];
      srr += psum[(w0 + ww) * 2 + 1];
    }
    if (part_rz) part_rz[grp] = srz;
    if (part_rr) part_rr[grp] = srr;
    for (int b = 0; b < P; ++b) mbar_inval(bars + b);  // every phase issued has completed
  }
}

// The beta step of a PCG iteration folded into the grouped-line solve: once
// every CTA of all the step's launches has written its groups' r.z and r.r
// partials, the last reduces them in a fixed order (group 0 .. ngroups - 1)
// and updates beta and the stopping test.
__device__ void fold_beta(const PcgFold &f) {
  __shared__ int last;
  __shared__ double red[2][kZgThreads / 32];
  __syncthreads();  // every slot of this CTA has written its partials
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(f.cnt, 1u) == (unsigned)(f.total - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double rz = 0.0, rr = 0.0;
  for (int t = threadIdx.x; t < f.nparts; t += blockDim.x) {
    rz += __ldcg(f.part + t);
    rr += __ldcg(f.part2 + t);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rz += __shfl_xor_sync(0xffffffffu, rz, o);
    rr += __shfl_xor_sync(0xffffffffu, rr, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = rz;
    red[1][threadIdx.x >> 5] = rr;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kZgThreads / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    pcg_finish_beta(f.s, a, b);
    *f.cnt = 0u;
    __threadfence();
  }
}

// packs [pk0, pk0 + npk) of one degree; CTAs take packs from queue[0]
// (largest first); the last CTA to finish resets queue[0..1] for the next
// launch.  One mesh (ginst == nullptr) or a batch (per group: its mirror's
// mesh and first unknown).
template <int N, typename T>
__global__ void __launch_bounds__(kZgThreads, 4)
zgroup_packed_kernel(const DevMesh m1, const int *__restrict__ ginst, const DevMesh *__restrict__ meshes,
                     const long long *__restrict__ dof_off, const int4 *__restrict__ glines,
                     const long long *__restrict__ gfac, const int4 *__restrict__ packs, int pk0, int npk,
                     int *__restrict__ queue, const T *__restrict__ fac, const T *__restrict__ r,
                     T *__restrict__ z, double *__restrict__ part_rz, double *__restrict__ part_rr, const int *__restrict__ done,
                     TnWait *__restrict__ err, const PcgFold fold) {
  if (done && *done) return;
  constexpr int SW = zg_stage_per_warp<N, T>();
  extern __shared__ __align__(16) unsigned char zsm[];
  T *const stage0 = reinterpret_cast<T *>(zsm);
  T *const vecs = stage0 + 4 * SW;
  unsigned long long *const bars = reinterpret_cast<unsigned long long *>(vecs + 4 * kZgThreads);
  __shared__ int s_pk;
  __shared__ double psum[8];
  const int warp = threadIdx.x >> 5;
  const unsigned long long lim = wait_limit(err);
  for (;;) {
    if (threadIdx.x == 0) s_pk = atomicAdd(queue, 1);
    __syncthreads();
    const int pk = s_pk;
    __syncthreads();
    if (pk >= npk) break;
    const int4 P4 = packs[pk0 + pk];
    const int ent[4] = {P4.x, P4.y, P4.z, P4.w};
    int w0 = 0, grp = -1, G = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int g = ent[i];
      if (g < 0 || grp >= 0) continue;
      const int4 L = glines[g];
      const int gs = 1 + (L.y >= 0) + (L.z >= 0) + (L.w >= 0);
      if (warp >= w0 && warp < w0 + gs) {
        grp = g;
        G = gs;
      } else {
        w0 += gs;
      }
    }
    if (grp >= 0) {
      int mncol = m1.ncol, mslab = m1.nslab;
      const T *rg = r;
      T *zg = z;
      if (ginst) {
        const int in = ginst[grp];
        mncol = meshes[in].ncol;
        mslab = meshes[in].nslab;
        const long long o = dof_off[in];
        rg += o;
        zg += o;
      }
      T *stg = stage0 + (size_t)w0 * SW;
      unsigned long long *sb = bars + kZgMaxStages * w0;
      const int cap = G * SW;
      switch (G) {
        case 1:
          zg_slot<N, 1, T>(grp, w0, mncol, mslab, rg, zg, glines, gfac, fac, stg, cap, vecs, sb, psum,
                                lim, err, part_rz, part_rr);
          break;
        case 2:
          zg_slot<N, 2, T>(grp, w0, mncol, mslab, rg, zg, glines, gfac, fac, stg, cap, vecs, sb, psum,
                                lim, err, part_rz, part_rr);
          break;
        case 3:
          zg_slot<N, 3, T>(grp, w0, mncol, mslab, rg, zg, glines, gfac, fac, stg, cap, vecs, sb, psum,
                                lim, err, part_rz, part_rr);
          break;
        default:
          zg_slot<N, 4, T>(grp, w0, mncol, mslab, rg, zg, glines, gfac, fac, stg, cap, vecs, sb, psum,
                                lim, err, part_rz, part_rr);
          break;
      }
    }
    __syncthreads();  // every slot of the pack is done with shared memory
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(queue + 1, 1) == (int)gridDim.x - 1) {
      queue[0] = 0;
      queue[1] = 0;
      __threadfence();
    }
  }
  if (fold.s) fold_beta(fold);
}

template <int N>
cudaError_t setup_n(const DevMesh &m, double *blk, float *fac, double *fac64, int *status, cudaStream_t st) {
  zline_blocks_kernel<N><<<m.E, ((N * N + 31) / 32) * 32, 0, st>>>(m, blk);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const int nlines = m.ncol * N * N;
  zline_factor_kernel<N><<<(nlines + 63) / 64, 64, 0, st>>>(nlines, m.nslab, blk, fac, fac64, status);
  return cudaGetLastError();
}

// opt in to more than 48 KB of dynamic shared memory (FP64, large N)
template <typename K>
cudaError_t zline_smem_optin(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int N, typename T, bool UPD>
cudaError_t solve_nt(const DevMesh &m, const void *fac, void *r, const void *q, void *z, const double *alpha,
                     double *part_rz, double *part_rr, const int *done, TnWait *zerr, cudaStream_t st) {
  const int blocks = (m.ncol * N * N + 3) / 4;
  constexpr size_t sm = zline_smem<N, T>();
  cudaError_t err = zline_smem_optin(zline_solve_kernel<N, T, T, UPD>, sm);
  if (err != cudaSuccess) return err;
  zline_solve_kernel<N, T, T, UPD><<<blocks, 128, sm, st>>>(m, (const T *)fac, (T *)r, (const T *)q, (T *)z,
                                                             alpha, part_rz, part_rr, done, zerr);
  return cudaGetLastError();
}

template <int N>
cudaError_t solve_n(const DevMesh &m, int prec, const void *fac, void *r, const void *q, void *z,
                    const double *alpha, double *part_rz, double *part_rr, const int *done, TnWait *zerr,
                    cudaStream_t st) {
  if (prec == TN_F64)
    return q ? solve_nt<N, double, true>(m, fac, r, q, z, alpha, part_rz, part_rr, done, zerr, st)
             : solve_nt<N, double, false>(m, fac, r, q, z, alpha, part_rz, part_rr, done, zerr, st);
  return q ? solve_nt<N, float, true>(m, fac, r, q, z, alpha, part_rz, part_rr, done, zerr, st)
           : solve_nt<N, float, false>(m, fac, r, q, z, alpha, part_rz, part_rr, done, zerr, st);
}

template <int N, typename T, bool UPD>
cudaError_t solve_batch_nt(const DevMesh *meshes, const int2 *work, int nwork, const long long *fac_off,
                           const long long *dof_off, const void *fac, void *r, const void *q, void *z,
                           const double *alpha, double *part_rz, double *part_rr, const int *done, TnWait *zerr,
                           cudaStream_t st) {
  constexpr size_t sm = zline_smem<N, T>();
  cudaError_t err = zline_smem_optin(zline_solve_batch_kernel<N, T, T, UPD>, sm);
  if (err != cudaSuccess) return err;
  zline_solve_batch_kernel<N, T, T, UPD><<<(nwork + 3) / 4, 128, sm, st>>>(
      meshes, work, nwork, fac_off, dof_off, (const T *)fac, (T *)r, (const T *)q, (T *)z, alpha, part_rz,
      part_rr, done, zerr);
  return cudaGetLastError();
}

template <int N>
cudaError_t solve_batch_n(int prec, const DevMesh *meshes, const int2 *work, int nwork, const long long *fac_off,
                          const long long *dof_off, const void *fac, void *r, const void *q, void *z,
                          const double *alpha, double *part_rz, double *part_rr, const int *done, TnWait *zerr,
                          cudaStream_t st) {
  if (prec == TN_F64)
    return q ? solve_batch_nt<N, double, true>(meshes, work, nwork, fac_off, dof_off, fac, r, q, z, alpha,
                                               part_rz, part_rr, done, zerr, st)
             : solve_batch_nt<N, double, false>(meshes, work, nwork, fac_off, dof_off, fac, r, q, z, alpha,
                                                part_rz, part_rr, done, zerr, st);
  return q ? solve_batch_nt<N, float, true>(meshes, work, nwork, fac_off, dof_off, fac, r, q, z, alpha, part_rz,
                                            part_rr, done, zerr, st)
           : solve_batch_nt<N, float, false>(meshes, work, nwork, fac_off, dof_off, fac, r, q, z, alpha,
                                             part_rz, part_rr, done, zerr, st);
}

template <int N>
cudaError_t zgroup_setup_n(const DevMesh &m, const ZGroupPlan &p, const ZGroupDev &gd, int inst,
                           const int4 *lines, const long long *fac_off, double *blk, double *xblk, double *work,
                           float *fac, double *fac64, int *status, cudaStream_t st) {
  zline_blocks_kernel<N><<<m.E, ((N * N + 31) / 32) * 32, 0, st>>>(m, blk);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  zgroup_cross_kernel<N><<<m.E, ((4 * N + 31) / 32) * 32, 0, st>>>(m, xblk);
  err = cudaGetLastError();
  // the four group sizes at once, each with its own scratch: the 4-line
  // groups (few, long) on st, the others on side streams forked from it
  if (err == cudaSuccess) err = cudaEventRecord(gd.fork, st);
  size_t off = 0;
  bool used[3] = {false, false, false};
  for (int g = 1; g <= 4 && err == cudaSuccess; ++g) {
    const int cnt = p.inst_n[(size_t)inst * 5 + g];
    if (!cnt) continue;
    cudaStream_t sg = st;
    if (g < 4) {
      sg = gd.side[g - 1];
      err = cudaStreamWaitEvent(sg, gd.fork, 0);
      used[g - 1] = true;
      if (err != cudaSuccess) break;
    }
    zgroup_factor_kernel<N><<<cnt, 128, 0, sg>>>(m, lines, fac_off, p.inst_start[(size_t)inst * 5 + g], g, blk,
                                                 xblk, work + off, fac, fac64, status);
    err = cudaGetLastError();
    const size_t MG = (size_t)g * 3 * N;
    off += (size_t)cnt * 3 * MG * MG;
  }
  for (int k = 0; k < 3 && err == cudaSuccess; ++k) {
    if (!used[k]) continue;
    err = cudaEventRecord(gd.join[k], gd.side[k]);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(st, gd.join[k], 0);
  }
  return err;
}

// persistent: as many CTAs as fit at once, never more than packs.  grid == 0:
// only compute the grid into *grid_out; else launch with it.
template <int N, typename T>
cudaError_t zgroup_launch_t(const DevMesh &m, const ZGroupDev &gd, int k, const void *fac, const void *r, void *z,
                            double *prz, double *prr, const int *done, TnWait *zerr, cudaStream_t st,
                            const PcgFold &fold, int *grid_out) {
  constexpr size_t sm = zg_smem<N, T>();
  auto kern = zgroup_packed_kernel<N, T>;
  cudaError_t err = zline_smem_optin(kern, sm);
  if (err != cudaSuccess) return err;
  static int per_sm[64] = {0};
  int dev = 0;
  err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!per_sm[dev]) {
    // shared memory before L1: the CTAs per SM are limited by the staging rings
    err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (err != cudaSuccess) return err;
    int b = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kZgThreads, sm);
    if (err != cudaSuccess) return err;
    per_sm[dev] = b > 0 ? b : 1;
  }
  int grid = per_sm[dev] * tn_sm_count();
  grid = grid < gd.pk_n[k] ? grid : gd.pk_n[k];
  if (grid_out) {
    *grid_out = grid;
    return cudaSuccess;
  }
  kern<<<grid, kZgThreads, sm, st>>>(m, gd.inst, gd.meshes, gd.dof_off, gd.lines, gd.fac_off, gd.packs,
                                     gd.pk_start[k], gd.pk_n[k], gd.queue + 2 * k, (const T *)fac, (const T *)r,
                                     (T *)z, prz, prr, done, zerr, fold);
  return cudaGetLastError();
}

template <int N>
cudaError_t zgroup_launch_n(const DevMesh &m, const ZGroupDev &gd, int k, int prec, const void *fac, const void *r,
                            void *z, double *prz, double *prr, const int *done, TnWait *zerr, cudaStream_t st,
                            const PcgFold &fold, int *grid_out) {
  if (prec == TN_F64)
    return zgroup_launch_t<N, double>(m, gd, k, fac, r, z, prz, prr, done, zerr, st, fold, grid_out);
  return zgroup_launch_t<N, float>(m, gd, k, fac, r, z, prz, prr, done, zerr, st, fold, grid_out);
}

// r -= alpha q ahead of the grouped-line solve (the PCG residual update; a
// separate pass measured faster than the update fused into the line walk)
template <typename T>
__global__ void zgroup_rupdate_kernel(long long n, T *__restrict__ r, const T *__restrict__ q,
                                      const double *__restrict__ alpha, const int *__restrict__ done) {
  if (done && *done) return;
  const T al = (T)*alpha;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    r[i] -= al * q[i];
}

}  // namespace

// union-find over face matches of the lines (col * N^2 + j * N + i)
static int uf_find(std::vector<int> &p, int x) {
  while (p[x] != x) {
    p[x] = p[p[x]];
    x = p[x];
  }
  return x;
}

// the groups of one mesh (members ascending), or false if a node is shared
// by more than 4 columns
static bool mesh_groups(const tn::HostMesh &hm, std::vector<std::vector<int>> &out, char *msg, int msglen) {
  const int N = hm.N, N2 = N * N, nl = hm.ncol * N2;
  std::vector<int> par(nl);
  for (int x = 0; x < nl; ++x) par[x] = x;
  for (int c = 0; c < hm.ncol; ++c)
    for (int f = 0; f < 4; ++f) {
      const int nbc = hm.colnb[4 * c + f];
      if (nbc < 0) continue;
      const int d = f >> 1, end = (f & 1) ? N - 1 : 0;
      const int code = hm.colnbf[4 * c + f], f2 = code & 3, d2 = f2 >> 1, end2 = (f2 & 1) ? N - 1 : 0;
      for (int t = 0; t < N; ++t) {
        const int i = d == 0 ? end : t, j = d == 0 ? t : end;
        const int a2 = (code >> 2) ? N - 1 - t : t;
        const int i2 = d2 == 0 ? end2 : a2, j2 = d2 == 0 ? a2 : end2;
        const int ra = uf_find(par, c * N2 + j * N + i), rb = uf_find(par, nbc * N2 + j2 * N + i2);
        if (ra != rb) par[ra < rb ? rb : ra] = ra < rb ? ra : rb;
      }
    }
  std::vector<std::vector<int>> comp(nl);
  for (int x = 0; x < nl; ++x) comp[uf_find(par, x)].push_back(x);
  out.clear();
  for (int x = 0; x < nl; ++x) {
    if (comp[x].empty()) continue;
    if (comp[x].size() > 4) {
      std::snprintf(msg, msglen, "a cross-section node is shared by %d columns (line groups hold at most 4)",
                    (int)comp[x].size());
      return false;
    }
    out.push_back(comp[x]);
  }
  return true;
}

bool tn_zgroup_plan(const tn::HostMesh *const *hms, int n, ZGroupPlan *p, char *msg, int msglen) {
  std::vector<std::vector<std::vector<int>>> per(n);
  for (int i = 0; i < n; ++i)
    if (!mesh_groups(*hms[i], per[i], msg, msglen)) return false;
  *p = ZGroupPlan();
  p->inst_start.assign((size_t)n * 5, 0);
  p->inst_n.assign((size_t)n * 5, 0);
  // order: group size (largest first), degree, mirror -- one class per (size, degree)
  for (int g = 4; g >= 1; --g)
    for (int N = TN_MIN_N; N <= TN_MAX_N; ++N) {
      const int start = p->ngroups;
      for (int i = 0; i < n; ++i) {
        if (hms[i]->N != N) continue;
        const long long rec = zg_rec(g * 3 * N, g);
        p->inst_start[(size_t)i * 5 + g] = p->ngroups;
        for (const auto &mm : per[i]) {
          if ((int)mm.size() != g) continue;
          p->lines.push_back(make_int4(mm[0], g > 1 ? mm[1] : -1, g > 2 ? mm[2] : -1, g > 3 ? mm[3] : -1));
          p->inst.push_back(i);
          p->fac_off.push_back(p->nfac);
          p->nfac += (long long)hms[i]->nslab * rec;
          p->ncompact += (long long)hms[i]->nslab * (zlp(g * 3 * N) + 8 * g * 3 * N);
          ++p->inst_n[(size_t)i * 5 + g];
          ++p->ngroups;
        }
      }
      if (p->ngroups == start) continue;
      if (p->ncls >= kZgMaxCls) {
        std::snprintf(msg, msglen, "too many line-group classes");
        return false;
      }
      p->cls_N[p->ncls] = N;
      p->cls_G[p->ncls] = g;
      p->cls_start[p->ncls] = start;
      p->cls_n[p->ncls] = p->ngroups - start;
      ++p->ncls;
    }
  // packs of groups filling the four warps of a CTA, per degree, largest
  // first: 4, 3 + 1, 2 + 2, 2 + 1 + 1, 1 + 1 + 1 + 1 lines
  for (int N = TN_MIN_N; N <= TN_MAX_N; ++N) {
    std::vector<int> by[5];
    for (int k = 0; k < p->ncls; ++k)
      if (p->cls_N[k] == N)
        for (int i = 0; i < p->cls_n[k]; ++i) by[p->cls_G[k]].push_back(p->cls_start[k] + i);
    if (by[1].empty() && by[2].empty() && by[3].empty() && by[4].empty()) continue;
    const int start = (int)p->packs.size();
    size_t i1 = 0;
    auto one = [&]() { return i1 < by[1].size() ? by[1][i1++] : -1; };
    for (int g4 : by[4]) p->packs.push_back(make_int4(g4, -1, -1, -1));
    for (int g3 : by[3]) p->packs.push_back(make_int4(g3, one(), -1, -1));
    for (size_t i = 0; i < by[2].size(); i += 2) {
      if (i + 1 < by[2].size()) {
        p->packs.push_back(make_int4(by[2][i], by[2][i + 1], -1, -1));
      } else {
        const int a = one();
        const int b = a >= 0 ? one() : -1;
        p->packs.push_back(make_int4(by[2][i], a, b, -1));
      }
    }
    while (i1 < by[1].size()) {
      const int a = one(), b = one(), c = one(), d = one();
      p->packs.push_back(make_int4(a, b, c, d));
    }
    if (p->npk >= kZgMaxPk) {
      std::snprintf(msg, msglen, "too many degrees for the grouped-line solve");
      return false;
    }
    p->pk_N[p->npk] = N;
    p->pk_start[p->npk] = start;
    p->pk_n[p->npk] = (int)p->packs.size() - start;
    ++p->npk;
  }
  return true;
}

size_t tn_zgroup_cross_bytes(const DevMesh &m) {
  const size_t M = 3 * m.N;
  return (size_t)m.E * 4 * m.N * M * M * sizeof(double);
}

size_t tn_zgroup_work_bytes(const DevMesh &m, const ZGroupPlan &p, int inst) {
  size_t sum = 0;
  for (int g = 1; g <= 4; ++g) {
    const size_t MG = (size_t)g * 3 * m.N;
    sum += (size_t)p.inst_n[(size_t)inst * 5 + g] * 3 * MG * MG * sizeof(double);
  }
  return sum;
}

cudaError_t tn_zgroup_setup(const DevMesh &m, const ZGroupPlan &p, const ZGroupDev &gd, int inst,
                            const int4 *lines, const long long *fac_off, double *blk, double *xblk, double *work,
                            float *fac, double *fac64, int *status, cudaStream_t st) {
  switch (m.N) {
#define TN_CASE(NN) \
    case NN: return zgroup_setup_n<NN>(m, p, gd, inst, lines, fac_off, blk, xblk, work, fac, fac64, status, st);
    TN_CASE(3) TN_CASE(4) TN_CASE(5) TN_CASE(6) TN_CASE(7) TN_CASE(8) TN_CASE(9)
#undef TN_CASE
    default: return cudaErrorInvalidValue;
  }
}

// one launch per degree present (one for a single mesh): the first on st,
// the others on side streams forked from and joined back into st (also
// inside a capture)
cudaError_t tn_zgroup_solve(const DevMesh *m, const ZGroupDev &gd, int prec, const void *fac, void *r,
                            const void *q, void *z, const double *alpha, double *part_rz, double *part_rr,
                            const int *done, TnWait *zerr, cudaStream_t st, const PcgFold *fold_in) {
  const DevMesh one = m ? *m : DevMesh{};
  cudaError_t err = cudaSuccess;
  PcgFold fold = fold_in ? *fold_in : PcgFold();
  if (fold.s) {  // the grids of every launch, for the last-CTA count
    fold.total = 0;
    fold.nparts = gd.ngroups;
    fold.part = part_rz;
    fold.part2 = part_rr;
    for (int k = 0; k < gd.npk && err == cudaSuccess; ++k) {
      int g = 0;
      switch (gd.pk_N[k]) {
#define TN_CASE(NN)                                                                                              \
        case NN:                                                                                                \
          err = zgroup_launch_n<NN>(one, gd, k, prec, fac, r, z, part_rz, part_rr, done, zerr, st, fold, &g); \
          break;
        TN_CASE(3) TN_CASE(4) TN_CASE(5) TN_CASE(6) TN_CASE(7) TN_CASE(8) TN_CASE(9)
#undef TN_CASE
        default: err = cudaErrorInvalidValue;
      }
      fold.total += g;
    }
    if (err != cudaSuccess) return err;
  }
  if (q) {  // the residual update, before every degree class reads r
    const int blocks = 4 * tn_sm_count();
    if (prec == TN_F64)
      zgroup_rupdate_kernel<double><<<blocks, 256, 0, st>>>(gd.ndof, (double *)r, (const double *)q, alpha, done);
    else
      zgroup_rupdate_kernel<float><<<blocks, 256, 0, st>>>(gd.ndof, (float *)r, (const float *)q, alpha, done);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  if (gd.npk > 1) err = cudaEventRecord(gd.fork, st);
  bool used[kZgSide] = {false};
  for (int k = 0; k < gd.npk && err == cudaSuccess; ++k) {
    cudaStream_t sk = st;
    if (k > 0) {
      const int sd = (k - 1) % kZgSide;
      sk = gd.side[sd];
      if (!used[sd]) {
        err = cudaStreamWaitEvent(sk, gd.fork, 0);
        used[sd] = true;
        if (err != cudaSuccess) break;
      }
    }
    switch (gd.pk_N[k]) {
#define TN_CASE(NN)                                                                                        \
      case NN:                                                                                            \
        err = zgroup_launch_n<NN>(one, gd, k, prec, fac, r, z, part_rz, part_rr, done, zerr, sk, fold, nullptr); \
        break;
      TN_CASE(3) TN_CASE(4) TN_CASE(5) TN_CASE(6) TN_CASE(7) TN_CASE(8) TN_CASE(9)
#undef TN_CASE
      default: err = cudaErrorInvalidValue;
    }
  }
  for (int sd = 0; sd < kZgSide && err == cudaSuccess; ++sd) {
    if (!used[sd]) continue;
    err = cudaEventRecord(gd.join[sd], gd.side[sd]);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(st, gd.join[sd], 0);
  }
  return err;
}

size_t tn_zline_block_bytes(const DevMesh &m) {
  const size_t M = 3 * m.N;
  return (size_t)m.ncol * m.N * m.N * m.nslab * 2 * M * M * sizeof(double);
}

size_t tn_zline_factor_entries(const DevMesh &m) {
  return (size_t)m.ncol * m.N * m.N * m.nslab * zrec(3 * m.N);
}

size_t tn_zline_factor_bytes(const DevMesh &m) { return tn_zline_factor_entries(m) * sizeof(float); }

int tn_zline_partials(const DevMesh &m) { return (m.ncol * m.N * m.N + 3) / 4; }

cudaError_t tn_zline_setup(const DevMesh &m, double *blk, float *fac, double *fac64, int *status,
                           cudaStream_t st) {
  switch (m.N) {
    case 3: return setup_n<3>(m, blk, fac, fac64, status, st);
    case 4: return setup_n<4>(m, blk, fac, fac64, status, st);
    case 5: return setup_n<5>(m, blk, fac, fac64, status, st);
    case 6: return setup_n<6>(m, blk, fac, fac64, status, st);
    case 7: return setup_n<7>(m, blk, fac, fac64, status, st);
    case 8: return setup_n<8>(m, blk, fac, fac64, status, st);
    case 9: return setup_n<9>(m, blk, fac, fac64, status, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t tn_zline_solve(const DevMesh &m, int prec, const void *fac, void *r, const void *q, void *z,
                           const double *alpha, double *part_rz, double *part_rr, const int *done, TnWait *zerr,
                           cudaStream_t st) {
  switch (m.N) {
#define TN_CASE(NN) \
    case NN: return solve_n<NN>(m, prec, fac, r, q, z, alpha, part_rz, part_rr, done, zerr, st);
    TN_CASE(3) TN_CASE(4) TN_CASE(5) TN_CASE(6) TN_CASE(7) TN_CASE(8) TN_CASE(9)
#undef TN_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t tn_zline_solve_batch(int N, int prec, const DevMesh *meshes, const int2 *work, int nwork,
                                 const long long *fac_off, const long long *dof_off, const void *fac, void *r,
                                 const void *q, void *z, const double *alpha, double *part_rz, double *part_rr,
                                 const int *done, TnWait *zerr, cudaStream_t st) {
  if (nwork <= 0) return cudaSuccess;
  switch (N) {
#define TN_CASE(NN)                                                                                   \
    case NN:                                                                                         \
      return solve_batch_n<NN>(prec, meshes, work, nwork, fac_off, dof_off, fac, r, q, z, alpha, part_rz, \
                               part_rr, done, zerr, st);
    TN_CASE(3) TN_CASE(4) TN_CASE(5) TN_CASE(6) TN_CASE(7) TN_CASE(8) TN_CASE(9)
#undef TN_CASE
    default: return cudaErrorInvalidValue;
  }
}
