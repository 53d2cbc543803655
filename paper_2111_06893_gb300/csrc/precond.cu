// Column-line block preconditioner for thin layers.
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
// backward block substitution.
#include <cstdio>

#include "tn_internal.h"
#include "tn_precond.h"

// device constants are per translation unit (no relocatable device code):
// this file keeps its own copy of the LGL tables
__constant__ LglTables c_lgl_pc;

cudaError_t tn_upload_lgl_precond(const LglTables *t) {
  return cudaMemcpyToSymbol(c_lgl_pc, t, sizeof(LglTables));
}

namespace {

// factor blocks are padded to a multiple of 4 entries (16-byte aligned for
// cp.async of float and double blocks)
__host__ __device__ constexpr int zpad(int M) { return ((M * M + 3) / 4) * 4; }

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
    // identity), stored column-major; Z_s row-major; blocks padded to MP
    constexpr int MP = zpad(M);
    float *Lf = fac + (((size_t)line * S + s) * 2 + 0) * MP;
    double *Ld = fac64 + (((size_t)line * S + s) * 2 + 0) * MP;
    for (int col = 0; col < M; ++col) {
      for (int r = 0; r < M; ++r) {
        double v;
        if (r < col) v = 0.0;
        else if (r == col) v = 1.0 / Dm[r * M + r];
        else {
          double acc = 0.0;
          for (int q = col; q < r; ++q) acc += Dm[r * M + q] * Ld[col * M + q];
          v = -acc / Dm[r * M + r];
        }
        Ld[col * M + r] = v;
        Lf[col * M + r] = (float)v;
      }
    }
    float *Zf = fac + (((size_t)line * S + s) * 2 + 1) * MP;
    double *Zd = fac64 + (((size_t)line * S + s) * 2 + 1) * MP;
    if (s > 0) {
      const double *Z = blk + (((size_t)line * S + s - 1) * 2 + 1) * M * M;
      for (int q = 0; q < M * M; ++q) { Zf[q] = (float)Z[q]; Zd[q] = Z[q]; }
    } else {
      for (int q = 0; q < M * M; ++q) { Zf[q] = 0.0f; Zd[q] = 0.0; }
    }
  }
}

// cp.async of one padded block pair (2 MP entries) into shared memory by a warp
template <typename F, int MP>
__device__ __forceinline__ void stage_pair(F *dst, const F *src, int lane) {
  constexpr int CH = (2 * MP * (int)sizeof(F)) / 16;  // 16-byte chunks
  const unsigned sdst = (unsigned)__cvta_generic_to_shared(dst);
  for (int t = lane; t < CH; t += 32)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sdst + 16 * t), "l"(src + t * (16 / (int)sizeof(F))));
  asm volatile("cp.async.commit_group;\n" ::);
}
__device__ __forceinline__ void wait_staged_all_but_one() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void wait_staged_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// z = A_LL^{-1} r on one line (one warp; lane l = a * N + k holds one unknown
// of a slab).  Forward:  y_s = Linv_s (r_s - Z_s^T y_{s-1});
// backward:  x_s = Linv_s^T (y_s - Z_{s+1} x_{s+1}).  Every product is a
// broadcast matrix-vector product (no dependent substitution chain); the
// slab's blocks are staged in shared memory (two buffers, cp.async) so that
// global reads are contiguous.  Returns this lane's share of r . z.
template <int N, typename T, typename F>
__device__ __forceinline__ T zline_line(const DevMesh &m, const F *__restrict__ fac, const T *__restrict__ r,
                                        T *__restrict__ z, int line, int lane, F *buf) {
  constexpr int M = 3 * N, N2 = N * N, n = N * N * N, MP = zpad(M);
  const int S = m.nslab;
  T rzt = T(0);
  const int c = line / N2, q = line - c * N2, i = q % N, j = q / N;
  const int a = lane / N, k = lane - (lane / N) * N;
  const bool act = lane < M;
  const int ll = act ? lane : 0;
  const size_t off = (size_t)k * N2 + j * N + i;
  const F *base = fac + (size_t)line * S * 2 * MP;  // slab s: [Linv_s | Z_s]
  // forward sweep
  stage_pair<F, MP>(buf, base, lane);
  T yprev = T(0);
  for (int s = 0; s < S; ++s) {
    F *cur = buf + (s & 1) * 2 * MP;
    if (s + 1 < S) {
      stage_pair<F, MP>(buf + ((s + 1) & 1) * 2 * MP, base + (size_t)(s + 1) * 2 * MP, lane);
      wait_staged_all_but_one();
    } else {
      wait_staged_all();
    }
    __syncwarp();
    const F *Li = cur, *Zs = cur + MP;
    const size_t e = (size_t)s * m.ncol + c;
    const size_t idx = (e * 3 + (act ? a : 0)) * n + off;
    T b = act ? r[idx] : T(0);
    if (s > 0) {
#pragma unroll
      for (int cc = 0; cc < M; ++cc) b -= (T)Zs[cc * M + ll] * __shfl_sync(0xffffffffu, yprev, cc);
    }
    T y = T(0);
#pragma unroll
    for (int cc = 0; cc < M; ++cc) y += (T)Li[cc * M + ll] * __shfl_sync(0xffffffffu, b, cc);
    if (!act) y = T(0);
    if (act) z[idx] = y;
    yprev = y;
    __syncwarp();  // buffer (s & 1) is restaged two slabs later
  }
  // backward sweep: slab s needs Linv_s and Z_{s+1}
  T xn = T(0);
  for (int s = S - 1; s >= 0; --s) {
    const F *Li = base + (size_t)s * 2 * MP;
    F *cur = buf;
    // stage Linv_s (first half of pair s) and Z_{s+1} (second half of pair s+1)
    {
      constexpr int CH = (MP * (int)sizeof(F)) / 16;
      const unsigned d0 = (unsigned)__cvta_generic_to_shared(cur);
      const unsigned d1 = (unsigned)__cvta_generic_to_shared(cur + MP);
      for (int t = lane; t < CH; t += 32)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d0 + 16 * t), "l"(Li + t * (16 / (int)sizeof(F))));
      if (s + 1 < S) {
        const F *Zn = base + (size_t)(s + 1) * 2 * MP + MP;
        for (int t = lane; t < CH; t += 32)
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d1 + 16 * t), "l"(Zn + t * (16 / (int)sizeof(F))));
      }
      asm volatile("cp.async.commit_group;\n" ::);
      wait_staged_all();
    }
    __syncwarp();
    const size_t e = (size_t)s * m.ncol + c;
    const size_t idx = (e * 3 + (act ? a : 0)) * n + off;
    T yv = act ? z[idx] : T(0);
    if (s < S - 1) {
      const F *Zs = cur + MP;
#pragma unroll
      for (int cc = 0; cc < M; ++cc) yv -= (T)Zs[ll * M + cc] * __shfl_sync(0xffffffffu, xn, cc);
    }
    T x = T(0);
#pragma unroll
    for (int cc = 0; cc < M; ++cc) x += (T)cur[ll * M + cc] * __shfl_sync(0xffffffffu, yv, cc);
    if (!act) x = T(0);
    if (act) {
      z[idx] = x;
      rzt += r[idx] * x;
    }
    xn = x;
    __syncwarp();
  }
  return rzt;
}

// four lines (warps) per block; partial sums of r . z per block
__device__ __forceinline__ void block_partial_rz(double rz, double *part) {
  __shared__ double red[4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rz += __shfl_xor_sync(0xffffffffu, rz, o);
  if (lane == 0) red[warp] = rz;
  __syncthreads();
  if (threadIdx.x == 0 && part) part[blockIdx.x] = red[0] + red[1] + red[2] + red[3];
}

template <int N, typename F>
constexpr size_t zline_smem() { return sizeof(F) * 4 * 2 * 2 * zpad(3 * N); }

template <int N, typename T, typename F>
__global__ void __launch_bounds__(128)
zline_solve_kernel(const DevMesh m, const F *__restrict__ fac, const T *__restrict__ r, T *__restrict__ z,
                   double *__restrict__ part, const int *__restrict__ done) {
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char zsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  F *buf = reinterpret_cast<F *>(zsm) + warp * 4 * zpad(3 * N);
  const int line = blockIdx.x * 4 + warp;
  T rzt = T(0);
  if (line < m.ncol * N * N) rzt = zline_line<N, T, F>(m, fac, r, z, line, lane, buf);
  block_partial_rz((double)rzt, part);
}

// a batch: warp w of block b handles line work[4 b + w] = (instance, line)
template <int N, typename T, typename F>
__global__ void __launch_bounds__(128)
zline_solve_batch_kernel(const DevMesh *__restrict__ meshes, const int2 *__restrict__ work, int nwork,
                         const long long *__restrict__ fac_off, const long long *__restrict__ dof_off,
                         const F *__restrict__ fac, const T *__restrict__ r, T *__restrict__ z,
                         double *__restrict__ part, const int *__restrict__ done) {
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char zsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  F *buf = reinterpret_cast<F *>(zsm) + warp * 4 * zpad(3 * N);
  const int wi = blockIdx.x * 4 + warp;
  T rzt = T(0);
  if (wi < nwork) {
    const int2 w = work[wi];
    const long long off = dof_off[w.x];
    rzt = zline_line<N, T, F>(meshes[w.x], fac + fac_off[w.x], r + off, z + off, w.y, lane, buf);
  }
  block_partial_rz((double)rzt, part);
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

template <int N>
cudaError_t solve_n(const DevMesh &m, int prec, const void *fac, const void *r, void *z, double *part,
                    const int *done, cudaStream_t st) {
  const int nlines = m.ncol * N * N;
  const int blocks = (nlines + 3) / 4;
  cudaError_t err = prec == TN_F64
                        ? zline_smem_optin(zline_solve_kernel<N, double, double>, zline_smem<N, double>())
                        : zline_smem_optin(zline_solve_kernel<N, float, float>, zline_smem<N, float>());
  if (err != cudaSuccess) return err;
  if (prec == TN_F64)
    zline_solve_kernel<N, double, double><<<blocks, 128, zline_smem<N, double>(), st>>>(
        m, (const double *)fac, (const double *)r, (double *)z, part, done);
  else
    zline_solve_kernel<N, float, float><<<blocks, 128, zline_smem<N, float>(), st>>>(
        m, (const float *)fac, (const float *)r, (float *)z, part, done);
  return cudaGetLastError();
}

}  // namespace

size_t tn_zline_block_bytes(const DevMesh &m) {
  const size_t M = 3 * m.N;
  return (size_t)m.ncol * m.N * m.N * m.nslab * 2 * M * M * sizeof(double);
}

size_t tn_zline_factor_entries(const DevMesh &m) {
  return (size_t)m.ncol * m.N * m.N * m.nslab * 2 * zpad(3 * m.N);
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

cudaError_t tn_zline_solve(const DevMesh &m, int prec, const void *fac, const void *r, void *z, double *part,
                           const int *done, cudaStream_t st) {
  switch (m.N) {
    case 3: return solve_n<3>(m, prec, fac, r, z, part, done, st);
    case 4: return solve_n<4>(m, prec, fac, r, z, part, done, st);
    case 5: return solve_n<5>(m, prec, fac, r, z, part, done, st);
    case 6: return solve_n<6>(m, prec, fac, r, z, part, done, st);
    case 7: return solve_n<7>(m, prec, fac, r, z, part, done, st);
    case 8: return solve_n<8>(m, prec, fac, r, z, part, done, st);
    case 9: return solve_n<9>(m, prec, fac, r, z, part, done, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t tn_zline_solve_batch(int N, int prec, const DevMesh *meshes, const int2 *work, int nwork,
                                 const long long *fac_off, const long long *dof_off, const void *fac,
                                 const void *r, void *z, double *part, const int *done, cudaStream_t st) {
  if (nwork <= 0) return cudaSuccess;
  const int blocks = (nwork + 3) / 4;
  switch (N) {
#define TN_CASE(NN)                                                                                       \
  case NN:                                                                                               \
    {                                                                                                    \
      cudaError_t oe = prec == TN_F64                                                                    \
          ? zline_smem_optin(zline_solve_batch_kernel<NN, double, double>, zline_smem<NN, double>())     \
          : zline_smem_optin(zline_solve_batch_kernel<NN, float, float>, zline_smem<NN, float>());       \
      if (oe != cudaSuccess) return oe;                                                                  \
    }                                                                                                    \
    if (prec == TN_F64)                                                                                  \
      zline_solve_batch_kernel<NN, double, double><<<blocks, 128, zline_smem<NN, double>(), st>>>(      \
          meshes, work, nwork, fac_off, dof_off, (const double *)fac, (const double *)r, (double *)z, part, done); \
    else                                                                                                 \
      zline_solve_batch_kernel<NN, float, float><<<blocks, 128, zline_smem<NN, float>(), st>>>(          \
          meshes, work, nwork, fac_off, dof_off, (const float *)fac, (const float *)r, (float *)z, part, done);    \
    return cudaGetLastError();
    TN_CASE(3) TN_CASE(4) TN_CASE(5) TN_CASE(6) TN_CASE(7) TN_CASE(8) TN_CASE(9)
#undef TN_CASE
    default: return cudaErrorInvalidValue;
  }
}
