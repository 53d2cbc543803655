// sm_103a kernels of the DG elasticity operator (Sec. 2.2), its right-hand
// side, diagonal and per-layer energies.
//
// Operator (weak form of Eq. (dg_residuals), LGL quadrature, M = w detJ):
//   y = sum_m D_m^T F^m  -  sum_faces W ( 1/2 (T + T_ext) - sigma P[[u]] )
//   F^m_j = J^-1[m][a] (Y : S_eff)^{aj},  S_eff = w detJ sym(grad u) + L,
//   L = sum_faces W (-1/2) sym(n (x) [[u]])          (lifted auxiliary strain)
// with W = w^S J^S at face nodes, T = n . Y grad u (unlifted, as in
// Eq. (numfluxprimal)), [[u]] = u - u_ext, P[[u]] = n . Y_* : sym(n (x) [[u]])
// (Eq. (constrel_avg)), sigma = C (p+1)^2 / min(h, h_ext) (Eq. (penalty)).
// Dirichlet faces (Eq. (bc), u_b = 0): u_ext = -u, T_ext = T, Y_* = Y.
// Neumann faces: no term.
//
// One CTA per element, one thread per node.  The element's own field is
// staged in shared memory; for each interior face the neighbour's face values
// and its logical normal derivative are gathered (neighbour data are L2
// hits), then the neighbour traction is formed at the face nodes, then every
// node forms its strain, stress, face terms and fluxes, and finally the
// transposed derivative contractions give y.  The FP32 kernel is built in two
// occupancy variants (registers per thread against CTAs per SM) with
// identical arithmetic; tn_tune_apply times both on the mesh at hand.
#include <cstdio>
#include <type_traits>

#include "tn_internal.h"

__constant__ LglTables c_lgl;
__constant__ float c_Df[TN_MAX_N + 1][TN_MAX_N * TN_MAX_N];
__constant__ float c_wf[TN_MAX_N + 1][TN_MAX_N];

cudaError_t tn_upload_lgl(const LglTables *t) {
  cudaError_t err = cudaMemcpyToSymbol(c_lgl, t, sizeof(LglTables));
  if (err != cudaSuccess) return err;
  static float Df[TN_MAX_N + 1][TN_MAX_N * TN_MAX_N];
  static float wf[TN_MAX_N + 1][TN_MAX_N];
  for (int N = 0; N <= TN_MAX_N; ++N) {
    for (int a = 0; a < TN_MAX_N * TN_MAX_N; ++a) Df[N][a] = (float)t->D[N][a];
    for (int a = 0; a < TN_MAX_N; ++a) wf[N][a] = (float)t->w[N][a];
  }
  err = cudaMemcpyToSymbol(c_Df, Df, sizeof(Df));
  if (err != cudaSuccess) return err;
  return cudaMemcpyToSymbol(c_wf, wf, sizeof(wf));
}

namespace {

template <typename T> struct Tab;
template <> struct Tab<double> {
  static __device__ __forceinline__ double D(int N, int a, int b) { return c_lgl.D[N][a * N + b]; }
  static __device__ __forceinline__ double w(int N, int a) { return c_lgl.w[N][a]; }
};
template <> struct Tab<Dual> {
  static __device__ __forceinline__ double D(int N, int a, int b) { return c_lgl.D[N][a * N + b]; }
  static __device__ __forceinline__ double w(int N, int a) { return c_lgl.w[N][a]; }
};
template <> struct Tab<float> {
  static __device__ __forceinline__ float D(int N, int a, int b) { return c_Df[N][a * N + b]; }
  static __device__ __forceinline__ float w(int N, int a) { return c_wf[N][a]; }
};

// geometry / material accessors: plain types round the FP64 tables, the dual
// type also carries the derivative seed of the current direction
template <typename T>
__device__ __forceinline__ T slab_dz(const DevMesh &m, int s, int k) {
  return (T)m.slabgeo[((size_t)s * SG_NF + SG_DZ) * m.N + k];
}
template <>
__device__ __forceinline__ float slab_dz<float>(const DevMesh &m, int s, int k) {
  return m.slabgeo32[((size_t)s * SG_NF + SG_DZ) * m.N + k];
}
template <>
__device__ __forceinline__ Dual slab_dz<Dual>(const DevMesh &m, int s, int k) {
  return Dual(m.slabgeo[((size_t)s * SG_NF + SG_DZ) * m.N + k], m.d_slabdz ? m.d_slabdz[(size_t)s * m.N + k] : 0.0);
}
template <typename T>
__device__ __forceinline__ T layer_coef(const DevMesh &m, int L, int q) {
  return (T)m.layer_c[3 * L + q];
}
template <>
__device__ __forceinline__ float layer_coef<float>(const DevMesh &m, int L, int q) {
  return m.layer_c32[3 * L + q];
}
// column geometry table in the kernel's precision
template <typename T> struct ColGeo { using type = double; };
template <> struct ColGeo<float> { using type = float; };
template <typename T>
__device__ __forceinline__ const typename ColGeo<T>::type *col_table(const DevMesh &m) {
  if constexpr (std::is_same<T, float>::value) return m.colgeo32;
  else return m.colgeo;
}
template <typename T>
__device__ __forceinline__ T pen_const(const DevMesh &m) {
  if constexpr (std::is_same<T, float>::value) return m.penC32;
  else return T(m.penC);
}
template <>
__device__ __forceinline__ Dual layer_coef<Dual>(const DevMesh &m, int L, int q) {
  return Dual(m.layer_c[3 * L + q], m.d_layer_c ? m.d_layer_c[3 * L + q] : 0.0);
}

// min(h, h_ext) of Eq. (penalty).  Sides whose h agree to 1e-12 relative
// are a tie (equal layer thicknesses, computed from slab positions with
// rounding): the dual number keeps the smaller value and takes the smaller
// derivative -- the one-sided derivative for an increasing parameter, the
// same from both elements of the face (so dA/dtheta stays symmetric)
template <typename T>
__device__ __forceinline__ T hmin(T a, T b) { return a < b ? a : b; }
template <>
__device__ __forceinline__ Dual hmin<Dual>(Dual a, Dual b) {
  if (fabs(a.v - b.v) <= 1e-12 * fmax(fabs(a.v), fabs(b.v)))
    return Dual(a.v < b.v ? a.v : b.v, a.d < b.d ? a.d : b.d);
  return a.v < b.v ? a : b;
}

// symmetric tensors as (xx, yy, zz, xy, xz, yz)
template <typename T> struct Sym { T xx, yy, zz, xy, xz, yz; };

// stress of a strain for a cubic-aligned stiffness (isotropic: c11 = l + 2m,
// c12 = l, c44 = m): s_ii = (c11 - c12) S_ii + c12 tr S, s_ij = 2 c44 S_ij
template <typename T>
__device__ __forceinline__ Sym<T> stress(const Sym<T> &S, T c11, T c12, T c44) {
  const T tr = S.xx + S.yy + S.zz, d = c11 - c12, two44 = c44 + c44;
  return {d * S.xx + c12 * tr, d * S.yy + c12 * tr, d * S.zz + c12 * tr,
          two44 * S.xy, two44 * S.xz, two44 * S.yz};
}

template <typename T>
__device__ __forceinline__ void contract_n(const Sym<T> &s, const T n[3], T out[3]) {
  out[0] = n[0] * s.xx + n[1] * s.xy + n[2] * s.xz;
  out[1] = n[0] * s.xy + n[1] * s.yy + n[2] * s.yz;
  out[2] = n[0] * s.xz + n[1] * s.yz + n[2] * s.zz;
}

template <typename T>
__device__ __forceinline__ Sym<T> sym_outer(const T n[3], const T v[3]) {
  const T h = T(0.5);
  return {n[0] * v[0], n[1] * v[1], n[2] * v[2], h * (n[0] * v[1] + n[1] * v[0]),
          h * (n[0] * v[2] + n[2] * v[0]), h * (n[1] * v[2] + n[2] * v[1])};
}

// physical gradient G[a][l] = sum_m Jinv[m][a] d_m u_l for the block-diagonal
// J^-1 = [[ixx, ixy, 0], [iex, iey, 0], [0, 0, 1/dz]]; returns sym(G)
template <typename T>
__device__ __forceinline__ Sym<T> strain(const T dxi[3], const T deta[3], const T dzeta[3], T ixx,
                                         T ixy, T iex, T iey, T idz) {
  T G[3][3];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    G[0][l] = ixx * dxi[l] + iex * deta[l];
    G[1][l] = ixy * dxi[l] + iey * deta[l];
    G[2][l] = idz * dzeta[l];
  }
  const T h = T(0.5);
  return {G[0][0], G[1][1], G[2][2], h * (G[0][1] + G[1][0]), h * (G[0][2] + G[2][0]),
          h * (G[1][2] + G[2][1])};
}

enum { FK_INTERIOR = 0, FK_DIRICHLET = 1, FK_NEUMANN = 2 };

struct FaceInfo {
  int kind[6];
  int nb[6];      // neighbour element
  int nbface[6];  // neighbour face 0..5
  int flip[6];
  int nbslab[6];
  int nbcol[6];
};

// face kinds and neighbours of element (s, c)
__device__ void face_info(const DevMesh &m, int s, int c, FaceInfo &fi, int f) {
  if (f < 4) {
    const int nbc = m.colnb[4 * c + f];
    if (nbc >= 0) {
      const int code = m.colnbf[4 * c + f];
      fi.kind[f] = FK_INTERIOR;
      fi.nb[f] = s * m.ncol + nbc;
      fi.nbface[f] = code & 3;
      fi.flip[f] = code >> 2;
      fi.nbslab[f] = s;
      fi.nbcol[f] = nbc;
    } else {
      fi.kind[f] = m.bc_side == TN_BC_FIXED ? FK_DIRICHLET : FK_NEUMANN;
      fi.nb[f] = -1; fi.nbface[f] = 0; fi.flip[f] = 0; fi.nbslab[f] = s; fi.nbcol[f] = c;
    }
  } else if (f == 4) {  // zeta = -1: the slab below
    if (s + 1 < m.nslab) {
      fi.kind[f] = FK_INTERIOR; fi.nb[f] = (s + 1) * m.ncol + c; fi.nbface[f] = 5;
      fi.flip[f] = 0; fi.nbslab[f] = s + 1; fi.nbcol[f] = c;
    } else {
      fi.kind[f] = m.bc_bottom == TN_BC_FIXED ? FK_DIRICHLET : FK_NEUMANN;
      fi.nb[f] = -1; fi.nbface[f] = 0; fi.flip[f] = 0; fi.nbslab[f] = s; fi.nbcol[f] = c;
    }
  } else {  // zeta = +1: the slab above, or the top surface (beam, Neumann)
    if (s > 0) {
      fi.kind[f] = FK_INTERIOR; fi.nb[f] = (s - 1) * m.ncol + c; fi.nbface[f] = 4;
      fi.flip[f] = 0; fi.nbslab[f] = s - 1; fi.nbcol[f] = c;
    } else {
      fi.kind[f] = FK_NEUMANN;
      fi.nb[f] = -1; fi.nbface[f] = 0; fi.flip[f] = 0; fi.nbslab[f] = s; fi.nbcol[f] = c;
    }
  }
}

// node indices (i, j, k) of face node (t1, t2) on face f, end index set
template <int N>
__device__ __forceinline__ void face_node(int f, int t1, int t2, int &i, int &j, int &k) {
  const int d = f >> 1, end = (f & 1) ? N - 1 : 0;
  if (d == 0) { i = end; j = t1; k = t2; }
  else if (d == 1) { i = t1; j = end; k = t2; }
  else { i = t1; j = t2; k = end; }
}

// outward normal, W = w^S J^S and h = 2 detJ / J^S at a face node of face f,
// from the column's 2x2 inverse map, its determinant and the slab's dz/dzeta;
// wt is the product of the two tangential LGL weights of the node
template <typename T>
__device__ __forceinline__ void face_geom_w(int f, T wt, T ixx, T ixy, T iex, T iey, T det2, T dz,
                                            T n[3], T &W, T &h) {
  const int d = f >> 1;
  const T sgn = (f & 1) ? T(1) : T(-1);
  if (d == 2) {
    n[0] = T(0); n[1] = T(0); n[2] = sgn;
    W = wt * det2;
    h = T(2) * dz;
    return;
  }
  const T rx = d == 0 ? ixx : iex, ry = d == 0 ? ixy : iey;
  const T mag = sqrt(rx * rx + ry * ry);
  const T inv = T(1) / mag;
  n[0] = sgn * rx * inv; n[1] = sgn * ry * inv; n[2] = T(0);
  W = wt * det2 * dz * mag;
  h = T(2) * inv;
}

template <typename T, int N>
__device__ __forceinline__ void face_geom(int f, int i, int j, int k, T ixx, T ixy, T iex, T iey,
                                          T det2, T dz, T n[3], T &W, T &h) {
  const int d = f >> 1;
  const T wt = d == 0 ? Tab<T>::w(N, j) * Tab<T>::w(N, k)
                      : (d == 1 ? Tab<T>::w(N, i) * Tab<T>::w(N, k) : Tab<T>::w(N, i) * Tab<T>::w(N, j));
  face_geom_w<T>(f, wt, ixx, ixy, iex, iey, det2, dz, n, W, h);
}

template <int N> __host__ __device__ constexpr int nthreads() { return ((N * N * N + 31) / 32) * 32; }

template <int N, typename T>
constexpr size_t apply_smem() {
  return sizeof(T) * (12 * N * N * N + 42 * N * N);
}

// T = double / float: y = A u (and optionally partial[e] = u_e . y_e).
// T = Dual: derivative of A u along the seeded direction; partial[e] = lam_e . (dA u)_e, y unused.
// work (optional, derivatives): CTA b contracts element work[b].y along
// parameter work[b].x, whose seeds are pseed[2 work[b].x] (d(dz/dzeta) per
// slab node) and pseed[2 work[b].x + 1] (d(c11, c12, c44) per layer),
// either may be nullptr; partial[b] as before.
template <int N, typename T, typename TIO>
__global__ void __launch_bounds__(nthreads<N>())
apply_kernel(const DevMesh m0, int e0, const TIO *__restrict__ u, TIO *__restrict__ y, double *__restrict__ partial,
             const double *__restrict__ lam, const int2 *__restrict__ work = nullptr,
             const double *const *__restrict__ pseed = nullptr) {
  DevMesh m = m0;
  int ework = -1;
  if (work) {
    const int2 wk = work[blockIdx.x];
    ework = wk.y;
    m.d_slabdz = pseed[2 * wk.x];
    m.d_layer_c = pseed[2 * wk.x + 1];
  }
  constexpr int n = N * N * N, N2 = N * N, NT = nthreads<N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *su = reinterpret_cast<T *>(smem_raw);  // [3][n]
  T *sF = su + 3 * n;                        // [3][3][n]
  T *nbv = sF + 9 * n;                       // [6][3][N2]
  T *nbt = nbv + 18 * N2;                    // [6][3][N2] normal derivative, then traction
  T *nbh = nbt + 18 * N2;                    // [6][N2]
  __shared__ FaceInfo fi;
  __shared__ T nbc[6][3];
  __shared__ double red[NT / 32];

  const int e = work ? ework : e0 + blockIdx.x, tid = threadIdx.x;
  const int s = e / m.ncol, c = e - s * m.ncol;
  const TIO *ue = u + (size_t)e * 3 * n;
  for (int t = tid; t < 3 * n; t += NT) su[t] = T(ue[t]);
  if (tid < 6) {
    face_info(m, s, c, fi, tid);
    const int L = m.slab_layer[fi.nbslab[tid]];
    nbc[tid][0] = layer_coef<T>(m, L, 0);
    nbc[tid][1] = layer_coef<T>(m, L, 1);
    nbc[tid][2] = layer_coef<T>(m, L, 2);
  }
  __syncthreads();

  // ---- gather neighbour face values and logical normal derivatives
  for (int t = tid; t < 6 * N2; t += NT) {
    const int f = t / N2, q = t - f * N2;
    if (fi.kind[f] != FK_INTERIOR) continue;
    const int t1 = q % N, t2 = q / N;
    const int f2 = fi.nbface[f], d2 = f2 >> 1, end = (f2 & 1) ? N - 1 : 0;
    int i2, j2, k2;
    if ((f >> 1) == 2) { i2 = t1; j2 = t2; k2 = end; }
    else {
      const int a = fi.flip[f] ? N - 1 - t1 : t1;
      k2 = t2;
      if (d2 == 0) { i2 = end; j2 = a; } else { i2 = a; j2 = end; }
    }
    const TIO *u2 = u + (size_t)fi.nb[f] * 3 * n;
    const int stride = d2 == 0 ? 1 : (d2 == 1 ? N : N2);
    const int base = (k2 * N + j2) * N + i2 - end * stride;
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      T line[N];
#pragma unroll
      for (int mm = 0; mm < N; ++mm) line[mm] = T(u2[cc * n + base + mm * stride]);
      T dn = T(0);
#pragma unroll
      for (int mm = 0; mm < N; ++mm) dn += Tab<T>::D(N, end, mm) * line[mm];
      nbv[(f * 3 + cc) * N2 + q] = line[end];
      nbt[(f * 3 + cc) * N2 + q] = dn;
    }
    T h2;
    if (d2 == 2) {
      h2 = T(2) * slab_dz<T>(m, fi.nbslab[f], end);
    } else {
      const auto *g2 = col_table<T>(m) + (size_t)fi.nbcol[f] * CG_NF * N2;
      const int q2 = j2 * N + i2;
      const T rx = (T)g2[(d2 == 0 ? CG_IXX : CG_IEX) * N2 + q2];
      const T ry = (T)g2[(d2 == 0 ? CG_IXY : CG_IEY) * N2 + q2];
      h2 = T(2) / sqrt(rx * rx + ry * ry);
    }
    nbh[f * N2 + q] = h2;
  }
  __syncthreads();

  const auto *cg = col_table<T>(m) + (size_t)c * CG_NF * N2;
  const int Lown = m.slab_layer[s];
  const T c11 = layer_coef<T>(m, Lown, 0), c12 = layer_coef<T>(m, Lown, 1), c44 = layer_coef<T>(m, Lown, 2);

  // ---- neighbour traction n . Y_ext grad u_ext at the face nodes
  for (int t = tid; t < 6 * N2; t += NT) {
    const int f = t / N2, q = t - f * N2;
    if (fi.kind[f] != FK_INTERIOR) continue;
    const int t1 = q % N, t2 = q / N, d = f >> 1;
    const int f2 = fi.nbface[f], d2 = f2 >> 1, end2 = (f2 & 1) ? N - 1 : 0;
    T dt1[3], dt2[3], dn[3];
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      const T *v = nbv + (f * 3 + cc) * N2;
      T a1 = T(0), a2 = T(0);
#pragma unroll
      for (int mm = 0; mm < N; ++mm) {
        a1 += Tab<T>::D(N, t1, mm) * v[t2 * N + mm];
        a2 += Tab<T>::D(N, t2, mm) * v[mm * N + t1];
      }
      dt1[cc] = a1; dt2[cc] = a2;
      dn[cc] = nbt[(f * 3 + cc) * N2 + q];
    }
    // neighbour logical derivatives in its own frame and its J^-1 there
    T dxi[3], deta[3], dzeta[3];
    T jxx, jxy, jex, jey, jdz;
    int i, j, k;
    face_node<N>(f, t1, t2, i, j, k);
    if (d == 2) {
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) { dxi[cc] = dt1[cc]; deta[cc] = dt2[cc]; dzeta[cc] = dn[cc]; }
      const int qq = j * N + i;
      jxx = (T)cg[CG_IXX * N2 + qq]; jxy = (T)cg[CG_IXY * N2 + qq];
      jex = (T)cg[CG_IEX * N2 + qq]; jey = (T)cg[CG_IEY * N2 + qq];
      jdz = T(1) / slab_dz<T>(m, fi.nbslab[f], end2);
    } else {
      const T sg1 = fi.flip[f] ? T(-1) : T(1);
      const int a = fi.flip[f] ? N - 1 - t1 : t1;
      int i2, j2;
      if (d2 == 0) {
        i2 = end2; j2 = a;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) { dxi[cc] = dn[cc]; deta[cc] = sg1 * dt1[cc]; dzeta[cc] = dt2[cc]; }
      } else {
        i2 = a; j2 = end2;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) { deta[cc] = dn[cc]; dxi[cc] = sg1 * dt1[cc]; dzeta[cc] = dt2[cc]; }
      }
      const auto *g2 = col_table<T>(m) + (size_t)fi.nbcol[f] * CG_NF * N2;
      const int q2 = j2 * N + i2;
      jxx = (T)g2[CG_IXX * N2 + q2]; jxy = (T)g2[CG_IXY * N2 + q2];
      jex = (T)g2[CG_IEX * N2 + q2]; jey = (T)g2[CG_IEY * N2 + q2];
      jdz = T(1) / slab_dz<T>(m, s, t2);
    }
    const Sym<T> S2 = strain(dxi, deta, dzeta, jxx, jxy, jex, jey, jdz);
    const Sym<T> s2 = stress(S2, nbc[f][0], nbc[f][1], nbc[f][2]);
    // our outward normal at this face node
    const int qq = j * N + i;
    T nrm[3], W, h;
    face_geom<T, N>(f, i, j, k, (T)cg[CG_IXX * N2 + qq], (T)cg[CG_IXY * N2 + qq],
                    (T)cg[CG_IEX * N2 + qq], (T)cg[CG_IEY * N2 + qq], (T)cg[CG_DET * N2 + qq],
                    slab_dz<T>(m, s, k), nrm, W, h);
    T tr[3];
    contract_n(s2, nrm, tr);
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) nbt[(f * 3 + cc) * N2 + q] = tr[cc];
  }

  __syncthreads();

  // ---- per node: strain, stress, face terms, fluxes
  T ysurf[3] = {T(0), T(0), T(0)};
  const int p = tid;
  const bool active = p < n;
  const int i = p % N, j = (p / N) % N, k = p / N2;
  if (active) {
    T dxi[3], deta[3], dzeta[3];
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      const T *v = su + cc * n;
      T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll
      for (int mm = 0; mm < N; ++mm) {
        a0 += Tab<T>::D(N, i, mm) * v[(k * N + j) * N + mm];
        a1 += Tab<T>::D(N, j, mm) * v[(k * N + mm) * N + i];
        a2 += Tab<T>::D(N, k, mm) * v[(mm * N + j) * N + i];
      }
      dxi[cc] = a0; deta[cc] = a1; dzeta[cc] = a2;
    }
    const int qq = j * N + i;
    const T ixx = (T)cg[CG_IXX * N2 + qq], ixy = (T)cg[CG_IXY * N2 + qq];
    const T iex = (T)cg[CG_IEX * N2 + qq], iey = (T)cg[CG_IEY * N2 + qq];
    const T det2 = (T)cg[CG_DET * N2 + qq], dz = slab_dz<T>(m, s, k);
    const T idz = T(1) / dz;
    const Sym<T> S = strain(dxi, deta, dzeta, ixx, ixy, iex, iey, idz);
    const T wJ = Tab<T>::w(N, i) * Tab<T>::w(N, j) * Tab<T>::w(N, k) * det2 * dz;
    Sym<T> Se = {wJ * S.xx, wJ * S.yy, wJ * S.zz, wJ * S.xy, wJ * S.xz, wJ * S.yz};
    const bool onface = i == 0 || i == N - 1 || j == 0 || j == N - 1 || k == 0 || k == N - 1;
    if (onface) {
      const Sym<T> sig = stress(S, c11, c12, c44);
      const T sp1 = T((float)((m.p + 1) * (m.p + 1))) * pen_const<T>(m);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int idx = d == 0 ? i : (d == 1 ? j : k);
        if (idx != 0 && idx != N - 1) continue;
        const int f = 2 * d + (idx == N - 1 ? 1 : 0);
        const int kind = fi.kind[f];
        if (kind == FK_NEUMANN) continue;
        T nrm[3], W, h;
        face_geom<T, N>(f, i, j, k, ixx, ixy, iex, iey, det2, dz, nrm, W, h);
        T tr[3];
        contract_n(sig, nrm, tr);
        const int t1 = d == 0 ? j : i, t2 = d == 2 ? j : k;
        const int q = t2 * N + t1;
        const T uo[3] = {su[p], su[n + p], su[2 * n + p]};
        T jump[3], tr2[3], h2, y11, y12, y44;
        if (kind == FK_INTERIOR) {
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) {
            jump[cc] = uo[cc] - nbv[(f * 3 + cc) * N2 + q];
            tr2[cc] = nbt[(f * 3 + cc) * N2 + q];
          }
          h2 = nbh[f * N2 + q];
          y11 = T(0.5) * (c11 + nbc[f][0]);
          y12 = T(0.5) * (c12 + nbc[f][1]);
          y44 = T(0.5) * (c44 + nbc[f][2]);
        } else {
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) { jump[cc] = uo[cc] + uo[cc]; tr2[cc] = tr[cc]; }
          h2 = h; y11 = c11; y12 = c12; y44 = c44;
        }
        const T sigma = sp1 / hmin<T>(h, h2);
        const Sym<T> Ej = sym_outer(nrm, jump);
        const Sym<T> Sj = stress(Ej, y11, y12, y44);
        T pen[3];
        contract_n(Sj, nrm, pen);
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) ysurf[cc] -= W * (T(0.5) * (tr[cc] + tr2[cc]) - sigma * pen[cc]);
        const T hw = T(-0.5) * W;
        Se.xx += hw * Ej.xx; Se.yy += hw * Ej.yy; Se.zz += hw * Ej.zz;
        Se.xy += hw * Ej.xy; Se.xz += hw * Ej.xz; Se.yz += hw * Ej.yz;
      }
    }
    const Sym<T> se = stress(Se, c11, c12, c44);
    // F^m_j = Jinv[m][a] sigma^{aj}
    sF[(0 * 3 + 0) * n + p] = ixx * se.xx + ixy * se.xy;
    sF[(0 * 3 + 1) * n + p] = ixx * se.xy + ixy * se.yy;
    sF[(0 * 3 + 2) * n + p] = ixx * se.xz + ixy * se.yz;
    sF[(1 * 3 + 0) * n + p] = iex * se.xx + iey * se.xy;
    sF[(1 * 3 + 1) * n + p] = iex * se.xy + iey * se.yy;
    sF[(1 * 3 + 2) * n + p] = iex * se.xz + iey * se.yz;
    sF[(2 * 3 + 0) * n + p] = idz * se.xz;
    sF[(2 * 3 + 1) * n + p] = idz * se.yz;
    sF[(2 * 3 + 2) * n + p] = idz * se.zz;
  }
  __syncthreads();

  // ---- weak divergence: y = sum_m D_m^T F^m
  double dot = 0.0;
  T dott = T(0);
  if (active) {
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      const T *F0 = sF + (0 * 3 + cc) * n, *F1 = sF + (1 * 3 + cc) * n, *F2 = sF + (2 * 3 + cc) * n;
      T acc = ysurf[cc];
#pragma unroll
      for (int mm = 0; mm < N; ++mm) {
        acc += Tab<T>::D(N, mm, i) * F0[(k * N + j) * N + mm];
        acc += Tab<T>::D(N, mm, j) * F1[(k * N + mm) * N + i];
        acc += Tab<T>::D(N, mm, k) * F2[(mm * N + j) * N + i];
      }
      if constexpr (std::is_same<T, Dual>::value) {
        dot += acc.d * lam[(size_t)e * 3 * n + cc * n + p];
      } else {
        y[(size_t)e * 3 * n + cc * n + p] = acc;
        dott += acc * su[cc * n + p];
      }
    }
  }
  if constexpr (!std::is_same<T, Dual>::value) dot = (double)dott;
  if (partial) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    if ((tid & 31) == 0) red[tid >> 5] = dot;
    __syncthreads();
    if (tid == 0) {
      double sum = 0.0;
      for (int w = 0; w < NT / 32; ++w) sum += red[w];
      partial[blockIdx.x] = sum;
    }
  }
}

// ---------------------------------------------------------------------------
// Second form of the operator kernel for T = float / double.  Same arithmetic
// as apply_kernel, reorganised so that every sum-factorised contraction is a
// "line task": one thread owns a whole line of N nodes along one logical
// direction, keeps it in registers and produces all N outputs with the
// derivative matrix as compile-time (warp-uniform) constant operands.  This
// removes the per-thread-indexed constant loads and cuts shared-memory traffic
// about threefold.  Phases (one CTA per element, one thread per node):
//   1  gather neighbour face values / normal derivatives  +  gradient lines
//   2  neighbour tangential derivative lines on the face planes
//   3  neighbour traction at the face nodes
//   4  per node: strain, stress, face terms, lifted strain, fluxes
//   5  weak-divergence lines (one partial sum per direction)
//   6  per node: sum the three directions and the face terms, store y
template <int N, typename T>
constexpr size_t apply2_smem() {
  return sizeof(T) * (3 * N * N * N + 9 * N * N * N + 9 * N * N * N + 18 * N * N * 4 + 6 * N * N);
}

// out[a'] = sum_a D[a'][a] v[a]   (derivative along the line)
template <int N, typename T>
__device__ __forceinline__ void line_diff(const T v[N], T out[N]) {
#pragma unroll
  for (int a2 = 0; a2 < N; ++a2) {
    T acc = T(0);
#pragma unroll
    for (int a = 0; a < N; ++a) acc += Tab<T>::D(N, a2, a) * v[a];
    out[a2] = acc;
  }
}
// out[a'] = sum_a D[a][a'] v[a]   (transposed: weak divergence along the line)
template <int N, typename T>
__device__ __forceinline__ void line_difft(const T v[N], T out[N]) {
#pragma unroll
  for (int a2 = 0; a2 < N; ++a2) {
    T acc = T(0);
#pragma unroll
    for (int a = 0; a < N; ++a) acc += Tab<T>::D(N, a, a2) * v[a];
    out[a2] = acc;
  }
}

// node index of position a on line l of direction d (l enumerates the N^2 lines)
template <int N>
__device__ __forceinline__ int line_node(int d, int l, int a) {
  const int hi = l / N, lo = l - hi * N;
  if (d == 0) return (hi * N + lo) * N + a;   // (k, j) fixed, i = a
  if (d == 1) return (hi * N + a) * N + lo;   // (k, i) fixed, j = a
  return (a * N + hi) * N + lo;               // (j, i) fixed, k = a
}

// u, y: the element's instance vectors; partial: this CTA's slot or nullptr
template <int N, typename T>
__device__ __forceinline__ void apply2_body(const DevMesh &m, const int e, const T *__restrict__ u,
                                            T *__restrict__ y, double *__restrict__ partial,
                                            unsigned char *smem_raw) {
  constexpr int n = N * N * N, N2 = N * N, NT = nthreads<N>();
  T *su = reinterpret_cast<T *>(smem_raw);  // [3][n]
  T *sG = su + 3 * n;                        // [3 dir][3 comp][n] logical gradient, then fluxes F^m_j
  T *sY = sG + 9 * n;                        // [3 dir][3 comp][n] divergence partial sums
  T *nbv = sY + 9 * n;                       // [6][3][N2] neighbour face values
  T *nbt = nbv + 18 * N2;                    // [6][3][N2] normal derivative, then traction
  T *nbd = nbt + 18 * N2;                    // [2][6][3][N2] tangential derivatives
  T *nbh = nbd + 36 * N2;                    // [6][N2]
  __shared__ FaceInfo fi;
  __shared__ T nbc[6][3];
  __shared__ double red[NT / 32];

  const int tid = threadIdx.x;
  const int s = e / m.ncol, c = e - s * m.ncol;
  const T *ue = u + (size_t)e * 3 * n;
  for (int t = tid; t < 3 * n; t += NT) su[t] = ue[t];
  if (tid < 6) {
    face_info(m, s, c, fi, tid);
    const int L = m.slab_layer[fi.nbslab[tid]];
    nbc[tid][0] = layer_coef<T>(m, L, 0);
    nbc[tid][1] = layer_coef<T>(m, L, 1);
    nbc[tid][2] = layer_coef<T>(m, L, 2);
  }
  __syncthreads();

  // ---- phase 1: neighbour gather tasks [0, 6 N2) and gradient line tasks [6 N2, 6 N2 + 9 N2)
  for (int t = tid; t < 15 * N2; t += NT) {
    if (t < 6 * N2) {
      const int f = t / N2, q = t - f * N2;
      if (fi.kind[f] != FK_INTERIOR) continue;
      const int t1 = q % N, t2 = q / N;
      const int f2 = fi.nbface[f], d2 = f2 >> 1, end = (f2 & 1) ? N - 1 : 0;
      int i2, j2, k2;
      if ((f >> 1) == 2) { i2 = t1; j2 = t2; k2 = end; }
      else {
        const int a = fi.flip[f] ? N - 1 - t1 : t1;
        k2 = t2;
        if (d2 == 0) { i2 = end; j2 = a; } else { i2 = a; j2 = end; }
      }
      const T *u2 = u + (size_t)fi.nb[f] * 3 * n;
      const int stride = d2 == 0 ? 1 : (d2 == 1 ? N : N2);
      const int base = (k2 * N + j2) * N + i2 - end * stride;
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        T line[N];
#pragma unroll
        for (int mm = 0; mm < N; ++mm) line[mm] = u2[cc * n + base + mm * stride];
        T dn = T(0);
        if (end == 0) {
#pragma unroll
          for (int mm = 0; mm < N; ++mm) dn += Tab<T>::D(N, 0, mm) * line[mm];
          nbv[(f * 3 + cc) * N2 + q] = line[0];
        } else {
#pragma unroll
          for (int mm = 0; mm < N; ++mm) dn += Tab<T>::D(N, N - 1, mm) * line[mm];
          nbv[(f * 3 + cc) * N2 + q] = line[N - 1];
        }
        nbt[(f * 3 + cc) * N2 + q] = dn;
      }
      T h2;
      if (d2 == 2) {
        h2 = T(2) * slab_dz<T>(m, fi.nbslab[f], end);
      } else {
        const auto *g2 = col_table<T>(m) + (size_t)fi.nbcol[f] * CG_NF * N2;
        const int q2 = j2 * N + i2;
        const T rx = (T)g2[(d2 == 0 ? CG_IXX : CG_IEX) * N2 + q2];
        const T ry = (T)g2[(d2 == 0 ? CG_IXY : CG_IEY) * N2 + q2];
        h2 = T(2) / sqrt(rx * rx + ry * ry);
      }
      nbh[f * N2 + q] = h2;
    } else {
      const int tt = t - 6 * N2, d = tt / (3 * N2), rem = tt - d * 3 * N2, cc = rem / N2, l = rem - cc * N2;
      const T *v = su + cc * n;
      T in[N], out[N];
#pragma unroll
      for (int a = 0; a < N; ++a) in[a] = v[line_node<N>(d, l, a)];
      line_diff<N, T>(in, out);
      T *g = sG + (d * 3 + cc) * n;
#pragma unroll
      for (int a = 0; a < N; ++a) g[line_node<N>(d, l, a)] = out[a];
    }
  }
  __syncthreads();

  // ---- phase 2: tangential derivatives of the neighbour face values
  for (int t = tid; t < 36 * N; t += NT) {
    const int f = t / (6 * N), rem = t - f * 6 * N, cc = rem / (2 * N), r2 = rem - cc * 2 * N;
    const int dir = r2 / N, l = r2 - dir * N;
    if (fi.kind[f] != FK_INTERIOR) continue;
    const T *v = nbv + (f * 3 + cc) * N2;
    T in[N], out[N];
    if (dir == 0) {  // along t1, fixed t2 = l
#pragma unroll
      for (int a = 0; a < N; ++a) in[a] = v[l * N + a];
    } else {         // along t2, fixed t1 = l
#pragma unroll
      for (int a = 0; a < N; ++a) in[a] = v[a * N + l];
    }
    line_diff<N, T>(in, out);
    T *o = nbd + ((dir * 6 + f) * 3 + cc) * N2;
    if (dir == 0) {
#pragma unroll
      for (int a = 0; a < N; ++a) o[l * N + a] = out[a];
    } else {
#pragma unroll
      for (int a = 0; a < N; ++a) o[a * N + l] = out[a];
    }
  }
  __syncthreads();

  const auto *cg = col_table<T>(m) + (size_t)c * CG_NF * N2;
  const int Lown = m.slab_layer[s];
  const T c11 = layer_coef<T>(m, Lown, 0), c12 = layer_coef<T>(m, Lown, 1), c44 = layer_coef<T>(m, Lown, 2);

  // ---- phase 3: neighbour traction n . Y_ext grad u_ext at the face nodes
  for (int t = tid; t < 6 * N2; t += NT) {
    const int f = t / N2, q = t - f * N2;
    if (fi.kind[f] != FK_INTERIOR) continue;
    const int t1 = q % N, t2 = q / N, d = f >> 1;
    const int f2 = fi.nbface[f], d2 = f2 >> 1, end2 = (f2 & 1) ? N - 1 : 0;
    T dt1[3], dt2[3], dn[3];
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      dt1[cc] = nbd[((0 * 6 + f) * 3 + cc) * N2 + q];
      dt2[cc] = nbd[((1 * 6 + f) * 3 + cc) * N2 + q];
      dn[cc] = nbt[(f * 3 + cc) * N2 + q];
    }
    T dxi[3], deta[3], dzeta[3];
    T jxx, jxy, jex, jey, jdz;
    int i, j, k;
    face_node<N>(f, t1, t2, i, j, k);
    if (d == 2) {
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) { dxi[cc] = dt1[cc]; deta[cc] = dt2[cc]; dzeta[cc] = dn[cc]; }
      const int qq = j * N + i;
      jxx = (T)cg[CG_IXX * N2 + qq]; jxy = (T)cg[CG_IXY * N2 + qq];
      jex = (T)cg[CG_IEX * N2 + qq]; jey = (T)cg[CG_IEY * N2 + qq];
      jdz = T(1) / slab_dz<T>(m, fi.nbslab[f], end2);
    } else {
      const T sg1 = fi.flip[f] ? T(-1) : T(1);
      const int a = fi.flip[f] ? N - 1 - t1 : t1;
      int i2, j2;
      if (d2 == 0) {
        i2 = end2; j2 = a;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) { dxi[cc] = dn[cc]; deta[cc] = sg1 * dt1[cc]; dzeta[cc] = dt2[cc]; }
      } else {
        i2 = a; j2 = end2;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) { deta[cc] = dn[cc]; dxi[cc] = sg1 * dt1[cc]; dzeta[cc] = dt2[cc]; }
      }
      const auto *g2 = col_table<T>(m) + (size_t)fi.nbcol[f] * CG_NF * N2;
      const int q2 = j2 * N + i2;
      jxx = (T)g2[CG_IXX * N2 + q2]; jxy = (T)g2[CG_IXY * N2 + q2];
      jex = (T)g2[CG_IEX * N2 + q2]; jey = (T)g2[CG_IEY * N2 + q2];
      jdz = T(1) / slab_dz<T>(m, s, t2);
    }
    const Sym<T> S2 = strain(dxi, deta, dzeta, jxx, jxy, jex, jey, jdz);
    const Sym<T> s2 = stress(S2, nbc[f][0], nbc[f][1], nbc[f][2]);
    const int qq = j * N + i;
    T nrm[3], W, h;
    face_geom<T, N>(f, i, j, k, (T)cg[CG_IXX * N2 + qq], (T)cg[CG_IXY * N2 + qq],
                    (T)cg[CG_IEX * N2 + qq], (T)cg[CG_IEY * N2 + qq], (T)cg[CG_DET * N2 + qq],
                    slab_dz<T>(m, s, k), nrm, W, h);
    T tr[3];
    contract_n(s2, nrm, tr);
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) nbt[(f * 3 + cc) * N2 + q] = tr[cc];
  }
  __syncthreads();

  // ---- phase 4: per node
  T ysurf[3] = {T(0), T(0), T(0)};
  T uown[3] = {T(0), T(0), T(0)};
  const int p = tid;
  const bool active = p < n;
  const int i = p % N, j = (p / N) % N, k = p / N2;
  if (active) {
    T dxi[3], deta[3], dzeta[3];
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      dxi[cc] = sG[(0 * 3 + cc) * n + p];
      deta[cc] = sG[(1 * 3 + cc) * n + p];
      dzeta[cc] = sG[(2 * 3 + cc) * n + p];
      uown[cc] = su[cc * n + p];
    }
    const int qq = j * N + i;
    const T ixx = (T)cg[CG_IXX * N2 + qq], ixy = (T)cg[CG_IXY * N2 + qq];
    const T iex = (T)cg[CG_IEX * N2 + qq], iey = (T)cg[CG_IEY * N2 + qq];
    const T det2 = (T)cg[CG_DET * N2 + qq], dz = slab_dz<T>(m, s, k);
    const T idz = T(1) / dz;
    const Sym<T> S = strain(dxi, deta, dzeta, ixx, ixy, iex, iey, idz);
    const T wJ = Tab<T>::w(N, i) * Tab<T>::w(N, j) * Tab<T>::w(N, k) * det2 * dz;
    Sym<T> Se = {wJ * S.xx, wJ * S.yy, wJ * S.zz, wJ * S.xy, wJ * S.xz, wJ * S.yz};
    const bool onface = i == 0 || i == N - 1 || j == 0 || j == N - 1 || k == 0 || k == N - 1;
    if (onface) {
      const Sym<T> sig = stress(S, c11, c12, c44);
      const T sp1 = T((float)((m.p + 1) * (m.p + 1))) * pen_const<T>(m);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int idx = d == 0 ? i : (d == 1 ? j : k);
        if (idx != 0 && idx != N - 1) continue;
        const int f = 2 * d + (idx == N - 1 ? 1 : 0);
        const int kind = fi.kind[f];
        if (kind == FK_NEUMANN) continue;
        T nrm[3], W, h;
        face_geom<T, N>(f, i, j, k, ixx, ixy, iex, iey, det2, dz, nrm, W, h);
        T tr[3];
        contract_n(sig, nrm, tr);
        const int t1 = d == 0 ? j : i, t2 = d == 2 ? j : k;
        const int q = t2 * N + t1;
        T jump[3], tr2[3], h2, y11, y12, y44;
        if (kind == FK_INTERIOR) {
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) {
            jump[cc] = uown[cc] - nbv[(f * 3 + cc) * N2 + q];
            tr2[cc] = nbt[(f * 3 + cc) * N2 + q];
          }
          h2 = nbh[f * N2 + q];
          y11 = T(0.5) * (c11 + nbc[f][0]);
          y12 = T(0.5) * (c12 + nbc[f][1]);
          y44 = T(0.5) * (c44 + nbc[f][2]);
        } else {
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) { jump[cc] = uown[cc] + uown[cc]; tr2[cc] = tr[cc]; }
          h2 = h; y11 = c11; y12 = c12; y44 = c44;
        }
        const T sigma = sp1 / hmin<T>(h, h2);
        const Sym<T> Ej = sym_outer(nrm, jump);
        const Sym<T> Sj = stress(Ej, y11, y12, y44);
        T pen[3];
        contract_n(Sj, nrm, pen);
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) ysurf[cc] -= W * (T(0.5) * (tr[cc] + tr2[cc]) - sigma * pen[cc]);
        const T hw = T(-0.5) * W;
        Se.xx += hw * Ej.xx; Se.yy += hw * Ej.yy; Se.zz += hw * Ej.zz;
        Se.xy += hw * Ej.xy; Se.xz += hw * Ej.xz; Se.yz += hw * Ej.yz;
      }
    }
    const Sym<T> se = stress(Se, c11, c12, c44);
    // fluxes F^m_j overwrite the gradient at this node (read above by this thread only)
    sG[(0 * 3 + 0) * n + p] = ixx * se.xx + ixy * se.xy;
    sG[(0 * 3 + 1) * n + p] = ixx * se.xy + ixy * se.yy;
    sG[(0 * 3 + 2) * n + p] = ixx * se.xz + ixy * se.yz;
    sG[(1 * 3 + 0) * n + p] = iex * se.xx + iey * se.xy;
    sG[(1 * 3 + 1) * n + p] = iex * se.xy + iey * se.yy;
    sG[(1 * 3 + 2) * n + p] = iex * se.xz + iey * se.yz;
    sG[(2 * 3 + 0) * n + p] = idz * se.xz;
    sG[(2 * 3 + 1) * n + p] = idz * se.yz;
    sG[(2 * 3 + 2) * n + p] = idz * se.zz;
  }
  __syncthreads();

  // ---- phase 5: weak-divergence lines
  for (int t = tid; t < 9 * N2; t += NT) {
    const int d = t / (3 * N2), rem = t - d * 3 * N2, cc = rem / N2, l = rem - cc * N2;
    const T *F = sG + (d * 3 + cc) * n;
    T in[N], out[N];
#pragma unroll
    for (int a = 0; a < N; ++a) in[a] = F[line_node<N>(d, l, a)];
    line_difft<N, T>(in, out);
    T *o = sY + (d * 3 + cc) * n;
#pragma unroll
    for (int a = 0; a < N; ++a) o[line_node<N>(d, l, a)] = out[a];
  }
  __syncthreads();

  // ---- phase 6: y = sum of the three directions + face terms
  T dott = T(0);
  if (active) {
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      const T acc = ysurf[cc] + sY[(0 * 3 + cc) * n + p] + sY[(1 * 3 + cc) * n + p] + sY[(2 * 3 + cc) * n + p];
      y[(size_t)e * 3 * n + cc * n + p] = acc;
      dott += acc * uown[cc];
    }
  }
  if (partial) {
    double dot = (double)dott;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    if ((tid & 31) == 0) red[tid >> 5] = dot;
    __syncthreads();
    if (tid == 0) {
      double sum = 0.0;
      for (int w = 0; w < NT / 32; ++w) sum += red[w];
      *partial = sum;
    }
  }
}

// resident CTAs per SM requested from the register allocator for the
// line-task kernel.  Variant 0: FP32, the CTAs per SM that fit ~60 registers
// per thread (N = 7: three CTAs of 352 threads); FP64: one.  Variant 1
// (FP32 only): one CTA more per SM than the registers of variant 0 allow,
// within the shared-memory limit (N = 3: 32, 4: 16, 5: 8, 6: 5, 7: 4, 8: 3,
// 9: 2), paid for with fewer registers per thread.  The two variants run the
// same instructions in the same order, so their results are bit-identical;
// the autotuner below times both on the mesh at hand.
template <int N, typename T, int V>
__host__ __device__ constexpr int apply2_min_blocks() {
  if (sizeof(T) != 4) return 1;
  if (V == 0) return N <= 4 ? 8 : (N == 5 ? 6 : (N == 6 ? 4 : (N == 7 ? 3 : (N == 8 ? 2 : 1))));
  return N == 3 ? 32 : (N == 4 ? 16 : (N == 5 ? 8 : (N == 6 ? 5 : (N == 7 ? 4 : (N == 8 ? 3 : 2)))));
}

// The alpha step of a PCG iteration folded into the operator apply: once
// every CTA of the step has written its p . Ap partial, the last reduces
// all partials in a fixed order (0 .. nparts - 1) and sets alpha = rz / pAp
// (breakdown if pAp <= 0 or not finite).  A run that has finished skips the
// apply and marks the iteration inactive.
__device__ __forceinline__ bool fold_skip(const PcgFold &f) {
  if (!f.s || !f.s->done) return false;
  if (blockIdx.x == 0 && threadIdx.x == 0) f.s->active = 0;
  return true;
}
__device__ void fold_alpha(const PcgFold &f) {
  const double *__restrict__ part = f.part;
  __shared__ int last;
  __shared__ double red[32];
  __syncthreads();  // this CTA's partial is written
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(f.cnt, 1u) == (unsigned)(f.total - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double acc = 0.0;
  for (int t = threadIdx.x; t < f.nparts; t += blockDim.x) acc += __ldcg(part + t);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double pq = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) pq += red[w];
    tn_pcg_scalars *s = f.s;
    s->active = 1;
    s->pq = pq;
    if (!(pq > 0.0) || !isfinite(pq)) {
      s->breakdown = 1;
      s->done = 1;
      s->alpha = 0.0;
    } else {
      s->alpha = s->rz / pq;
    }
    *f.cnt = 0u;
    __threadfence();
  }
}

template <int N, typename T, int V>
__global__ void __launch_bounds__(nthreads<N>(), (apply2_min_blocks<N, T, V>()))
apply2_kernel(const DevMesh m, int e0, const T *__restrict__ u, T *__restrict__ y, double *__restrict__ partial,
              const PcgFold fold) {
  if (fold_skip(fold)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  apply2_body<N, T>(m, e0 + blockIdx.x, u, y, partial ? partial + blockIdx.x : nullptr, smem_raw);
  if (fold.s) fold_alpha(fold);
}

// a batch of meshes: CTA b works on element work[b].y of instance work[b].x
template <int N, typename T, int V>
__global__ void __launch_bounds__(nthreads<N>(), (apply2_min_blocks<N, T, V>()))
apply2_batch_kernel(const DevMesh *__restrict__ meshes, const int2 *__restrict__ work,
                    const long long *__restrict__ dof_off, const T *__restrict__ u, T *__restrict__ y,
                    double *__restrict__ partial, const PcgFold fold) {
  if (fold_skip(fold)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) unsigned char sm_raw[sizeof(DevMesh)];
  DevMesh &sm = *reinterpret_cast<DevMesh *>(sm_raw);
  const int2 w = work[blockIdx.x];
  if (threadIdx.x == 0) memcpy(sm_raw, &meshes[w.x], sizeof(DevMesh));
  __syncthreads();
  const long long off = dof_off[w.x];
  apply2_body<N, T>(sm, w.y, u + off, y + off, partial ? partial + blockIdx.x : nullptr, smem_raw);
  if (fold.s) fold_alpha(fold);
}

// the dynamic shared-memory opt-in of a kernel, once per device
template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes, int &configured_device) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_device == dev) return cudaSuccess;
  cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (err == cudaSuccess) configured_device = dev;
  return err;
}

// fold / fold_part: the alpha step (fold_part: the partials of all the
// step's launches, of which this launch writes `partial` onwards)
template <int N, typename T, int V>
cudaError_t launch_apply2_batch_v(const DevMesh *meshes, const int2 *work, int nwork, const long long *dof_off,
                                  const T *u, T *y, double *partial, cudaStream_t st, const PcgFold &fold) {
  constexpr size_t sm = apply2_smem<N, T>();
  static int configured_device = -1;
  cudaError_t err = allow_smem(apply2_batch_kernel<N, T, V>, sm, configured_device);
  if (err != cudaSuccess) return err;
  if (nwork <= 0) return cudaSuccess;
  apply2_batch_kernel<N, T, V><<<nwork, nthreads<N>(), sm, st>>>(meshes, work, dof_off, u, y, partial, fold);
  return cudaGetLastError();
}

template <int N, typename T, int V>
cudaError_t launch_apply2_v(const DevMesh &m, const T *u, T *y, double *partial, cudaStream_t st,
                            const PcgFold &fold) {
  constexpr size_t sm = apply2_smem<N, T>();
  static int configured_device = -1;
  cudaError_t err = allow_smem(apply2_kernel<N, T, V>, sm, configured_device);
  if (err != cudaSuccess) return err;
  apply2_kernel<N, T, V><<<m.E, nthreads<N>(), sm, st>>>(m, 0, u, y, partial, fold);
  return cudaGetLastError();
}

// variant 1 exists for FP32 only
template <int N, typename T>
cudaError_t launch_apply2_batch(const DevMesh *meshes, const int2 *work, int nwork, const long long *dof_off,
                                const T *u, T *y, double *partial, cudaStream_t st, int var,
                                const PcgFold &fold = PcgFold()) {
  if constexpr (sizeof(T) == 4) {
    if (var == 1) return launch_apply2_batch_v<N, T, 1>(meshes, work, nwork, dof_off, u, y, partial, st, fold);
  }
  return launch_apply2_batch_v<N, T, 0>(meshes, work, nwork, dof_off, u, y, partial, st, fold);
}

template <int N, typename T>
cudaError_t launch_apply2(const DevMesh &m, const T *u, T *y, double *partial, cudaStream_t st, int var,
                          const PcgFold &fold = PcgFold()) {
  if constexpr (sizeof(T) == 4) {
    if (var == 1) return launch_apply2_v<N, T, 1>(m, u, y, partial, st, fold);
  }
  return launch_apply2_v<N, T, 0>(m, u, y, partial, st, fold);
}

// time per launch (us) of both FP32 variants on one mesh (m1) or one degree
// group of a batch: 3 untimed launches, then 10 between CUDA events on st
template <int N>
cudaError_t tune_apply2(const DevMesh *m1, const DevMesh *meshes, const int2 *work, int nwork,
                        const long long *dof_off, const float *u, float *y, cudaStream_t st, float us[2]) {
  cudaEvent_t ev[2];
  cudaError_t err = cudaEventCreate(&ev[0]);
  if (err != cudaSuccess) return err;
  err = cudaEventCreate(&ev[1]);
  if (err != cudaSuccess) {
    cudaEventDestroy(ev[0]);
    return err;
  }
  for (int v = 0; v < 2 && err == cudaSuccess; ++v) {
    for (int i = 0; i < 13 && err == cudaSuccess; ++i) {
      if (i == 3) err = cudaEventRecord(ev[0], st);
      if (err != cudaSuccess) break;
      err = m1 ? launch_apply2<N, float>(*m1, u, y, nullptr, st, v)
               : launch_apply2_batch<N, float>(meshes, work, nwork, dof_off, u, y, nullptr, st, v);
    }
    if (err == cudaSuccess) err = cudaEventRecord(ev[1], st);
    if (err == cudaSuccess) err = cudaEventSynchronize(ev[1]);
    float ms = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    us[v] = ms * 100.0f;  // 10 launches: ms / 10 * 1000
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  return err;
}

template <int N, typename T, typename TIO>
cudaError_t launch_apply_range(const DevMesh &m, int s0, int s1, const TIO *u, TIO *y, double *partial,
                               const double *lam, cudaStream_t st) {
  constexpr size_t sm = apply_smem<N, T>();
  static int configured_device = -1;  // the attribute is per function and device
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_device != dev) {
    cudaError_t err = cudaFuncSetAttribute(apply_kernel<N, T, TIO>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    configured_device = dev;
  }
  const int nblk = (s1 - s0) * m.ncol;
  if (nblk <= 0) return cudaSuccess;
  apply_kernel<N, T, TIO><<<nblk, nthreads<N>(), sm, st>>>(m, s0 * m.ncol, u, y, partial, lam);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply_t(const DevMesh &m, const T *u, T *y, double *partial, cudaStream_t st, int var,
                           const PcgFold &fold) {
  switch (m.N) {
    case 3: return launch_apply2<3, T>(m, u, y, partial, st, var, fold);
    case 4: return launch_apply2<4, T>(m, u, y, partial, st, var, fold);
    case 5: return launch_apply2<5, T>(m, u, y, partial, st, var, fold);
    case 6: return launch_apply2<6, T>(m, u, y, partial, st, var, fold);
    case 7: return launch_apply2<7, T>(m, u, y, partial, st, var, fold);
    case 8: return launch_apply2<8, T>(m, u, y, partial, st, var, fold);
    case 9: return launch_apply2<9, T>(m, u, y, partial, st, var, fold);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------- RHS
// b = -sum_top W p(r) e_z at the top-surface nodes (Neumann beam data)
__global__ void rhs_kernel(const DevMesh m, double r0, double F0, double *__restrict__ b) {
  const int N = m.N, n = N * N * N, N2 = N * N;
  const size_t total = (size_t)m.E * 3 * n;
  const double norm = F0 / (M_PI * r0 * r0), ir2 = 1.0 / (r0 * r0);
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(t % n);
    const size_t ec = t / n;
    const int cc = (int)(ec % 3);
    const int e = (int)(ec / 3);
    double v = 0.0;
    if (cc == 2 && e < m.ncol && p / N2 == N - 1) {  // top slab, k = N-1, z component
      const int q = p % N2, i = q % N, j = q / N;
      const double *g = m.colgeo + (size_t)e * CG_NF * N2;
      const double X = g[CG_X * N2 + q], Y = g[CG_Y * N2 + q];
      const double W = c_lgl.w[N][i] * c_lgl.w[N][j] * g[CG_DET * N2 + q];
      v = -W * norm * exp(-(X * X + Y * Y) * ir2);
    }
    b[t] = v;
  }
}

// ------------------------------------------------------------ diagonal
// diag(A) at (e, comp c, node p):
//   volume: sum over the three lines through p of w detJ (c11 g_c^2 + c44 sum_{a!=c} g_a^2)
//           with g the physical gradient of the basis function at the node
//   face f containing p (non-Neumann): -2 W Q + 2 W sigma (c11* n_c^2 + c44* (1 - n_c^2)) x s
//           with Q = c11 n_c g_c + c44 sum_{a != c} n_a g_a, interior: factor 1/2 on both.
__global__ void diag_kernel(const DevMesh m, double *__restrict__ dg) {
  const int N = m.N, n = N * N * N, N2 = N * N;
  const int e = blockIdx.x;
  const int s = e / m.ncol, c = e - s * m.ncol;
  __shared__ FaceInfo fi;
  __shared__ double nbc[6][3];
  if (threadIdx.x < 6) {
    face_info(m, s, c, fi, threadIdx.x);
    const int L = m.slab_layer[fi.nbslab[threadIdx.x]];
    for (int a = 0; a < 3; ++a) nbc[threadIdx.x][a] = m.layer_c[3 * L + a];
  }
  __syncthreads();
  const double *cg = m.colgeo + (size_t)c * CG_NF * N2;
  const double *sg = m.slabgeo + (size_t)s * SG_NF * N;
  const int L = m.slab_layer[s];
  const double c11 = m.layer_c[3 * L], c12 = m.layer_c[3 * L + 1], c44 = m.layer_c[3 * L + 2];
  (void)c12;
#define DD(a, b) c_lgl.D[N][(a) * N + (b)]
#define WW(a) c_lgl.w[N][(a)]
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    const int i = p % N, j = (p / N) % N, k = p / N2;
    double out[3] = {0.0, 0.0, 0.0};
    // volume: nodes r on the three lines through p
    for (int line = 0; line < 3; ++line) {
      for (int r = 0; r < N; ++r) {
        int ri = i, rj = j, rk = k;
        if (line == 0) ri = r; else if (line == 1) rj = r; else rk = r;
        const bool self = (ri == i && rj == j && rk == k);
        if (self && line > 0) continue;  // count r = p once
        const int q = rj * N + ri;
        double lg[3];
        if (self) { lg[0] = DD(i, i); lg[1] = DD(j, j); lg[2] = DD(k, k); }
        else {
          lg[0] = line == 0 ? DD(ri, i) : 0.0;
          lg[1] = line == 1 ? DD(rj, j) : 0.0;
          lg[2] = line == 2 ? DD(rk, k) : 0.0;
        }
        const double ixx = cg[CG_IXX * N2 + q], ixy = cg[CG_IXY * N2 + q];
        const double iex = cg[CG_IEX * N2 + q], iey = cg[CG_IEY * N2 + q];
        const double dz = sg[SG_DZ * N + rk];
        const double g[3] = {ixx * lg[0] + iex * lg[1], ixy * lg[0] + iey * lg[1], lg[2] / dz};
        const double wJ = WW(ri) * WW(rj) * WW(rk) * cg[CG_DET * N2 + q] * dz;
        const double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
        for (int cc = 0; cc < 3; ++cc) out[cc] += wJ * (c11 * g[cc] * g[cc] + c44 * (g2 - g[cc] * g[cc]));
      }
    }
    // faces
    const int q = j * N + i;
    const double ixx = cg[CG_IXX * N2 + q], ixy = cg[CG_IXY * N2 + q];
    const double iex = cg[CG_IEX * N2 + q], iey = cg[CG_IEY * N2 + q];
    const double det2 = cg[CG_DET * N2 + q], dz = sg[SG_DZ * N + k];
    const double lg[3] = {DD(i, i), DD(j, j), DD(k, k)};
    const double g[3] = {ixx * lg[0] + iex * lg[1], ixy * lg[0] + iey * lg[1], lg[2] / dz};
    const double sp1 = (double)((m.p + 1) * (m.p + 1)) * m.penC;
    for (int d = 0; d < 3; ++d) {
      const int idx = d == 0 ? i : (d == 1 ? j : k);
      if (idx != 0 && idx != N - 1) continue;
      const int f = 2 * d + (idx == N - 1 ? 1 : 0);
      if (fi.kind[f] == FK_NEUMANN) continue;
      double nrm[3], W, h;
      const double wt = d == 0 ? WW(j) * WW(k) : (d == 1 ? WW(i) * WW(k) : WW(i) * WW(j));
      face_geom_w<double>(f, wt, ixx, ixy, iex, iey, det2, dz, nrm, W, h);
      double h2, y11, y44, fac;
      if (fi.kind[f] == FK_INTERIOR) {
        // neighbour h at the matching node
        const int t1 = d == 0 ? j : i, t2 = d == 2 ? j : k;
        const int f2 = fi.nbface[f], d2 = f2 >> 1, end2 = (f2 & 1) ? N - 1 : 0;
        if (d == 2) {
          h2 = 2.0 * m.slabgeo[((size_t)fi.nbslab[f] * SG_NF + SG_DZ) * N + end2];
        } else {
          const int a = fi.flip[f] ? N - 1 - t1 : t1;
          const int i2 = d2 == 0 ? end2 : a, j2 = d2 == 0 ? a : end2;
          const double *g2 = m.colgeo + (size_t)fi.nbcol[f] * CG_NF * N2;
          const double rx = g2[(d2 == 0 ? CG_IXX : CG_IEX) * N2 + j2 * N + i2];
          const double ry = g2[(d2 == 0 ? CG_IXY : CG_IEY) * N2 + j2 * N + i2];
          h2 = 2.0 / sqrt(rx * rx + ry * ry);
        }
        (void)t2;
        y11 = 0.5 * (c11 + nbc[f][0]);
        y44 = 0.5 * (c44 + nbc[f][2]);
        fac = 0.5;
      } else {
        h2 = h; y11 = c11; y44 = c44; fac = 1.0;
      }
      const double sigma = sp1 / hmin<double>(h, h2);
      for (int cc = 0; cc < 3; ++cc) {
        double Qc = 0.0;
        for (int a = 0; a < 3; ++a) Qc += (a == cc ? c11 : c44) * nrm[a] * g[a];
        const double pn = y11 * nrm[cc] * nrm[cc] + y44 * (1.0 - nrm[cc] * nrm[cc]);
        out[cc] += -2.0 * fac * W * Qc + (fac == 0.5 ? 1.0 : 2.0) * W * sigma * pn;
      }
    }
    for (int cc = 0; cc < 3; ++cc) dg[((size_t)e * 3 + cc) * n + p] = out[cc];
  }
#undef DD
#undef WW
}

// ------------------------------------------------------------- energies
// elem[blockIdx.x] = 1/2 sum_p w_p detJ_p S_p : Y : S_p, S = sym grad u
// (unlifted), for the elements e0 + blockIdx.x; T = Dual gives the derivative
// along the seeded direction instead; scaled by w[layer] if w is given.
template <int N, typename T>
__global__ void __launch_bounds__(nthreads<N>())
energy_kernel(const DevMesh m0, int e0, const double *__restrict__ u, const double *__restrict__ w,
              double *__restrict__ elem, const int2 *__restrict__ work = nullptr,
              const double *const *__restrict__ pseed = nullptr) {
  DevMesh m = m0;  // work: as for apply_kernel
  int ework = -1;
  if (work) {
    const int2 wk = work[blockIdx.x];
    ework = wk.y;
    m.d_slabdz = pseed[2 * wk.x];
    m.d_layer_c = pseed[2 * wk.x + 1];
  }
  constexpr int n = N * N * N, N2 = N * N, NT = nthreads<N>();
  __shared__ double su[3 * n];
  __shared__ double red[NT / 32];
  const int e = work ? ework : e0 + blockIdx.x, tid = threadIdx.x;
  const int s = e / m.ncol, c = e - s * m.ncol;
  for (int t = tid; t < 3 * n; t += NT) su[t] = u[(size_t)e * 3 * n + t];
  __syncthreads();
  const double *cg = m.colgeo + (size_t)c * CG_NF * N2;
  const int L = m.slab_layer[s];
  const T c11 = layer_coef<T>(m, L, 0), c12 = layer_coef<T>(m, L, 1), c44 = layer_coef<T>(m, L, 2);
  double en = 0.0;
  if (tid < n) {
    const int p = tid, i = p % N, j = (p / N) % N, k = p / N2;
    T dxi[3], deta[3], dzeta[3];
    for (int cc = 0; cc < 3; ++cc) {
      const double *v = su + cc * n;
      double a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
      for (int mm = 0; mm < N; ++mm) {
        a0 += Tab<double>::D(N, i, mm) * v[(k * N + j) * N + mm];
        a1 += Tab<double>::D(N, j, mm) * v[(k * N + mm) * N + i];
        a2 += Tab<double>::D(N, k, mm) * v[(mm * N + j) * N + i];
      }
      dxi[cc] = T(a0); deta[cc] = T(a1); dzeta[cc] = T(a2);
    }
    const int q = j * N + i;
    const T dz = slab_dz<T>(m, s, k);
    const Sym<T> S = strain<T>(dxi, deta, dzeta, T(cg[CG_IXX * N2 + q]), T(cg[CG_IXY * N2 + q]),
                               T(cg[CG_IEX * N2 + q]), T(cg[CG_IEY * N2 + q]), T(1.0) / dz);
    const Sym<T> sg2 = stress(S, c11, c12, c44);
    const T dens = S.xx * sg2.xx + S.yy * sg2.yy + S.zz * sg2.zz +
                   T(2.0) * (S.xy * sg2.xy + S.xz * sg2.xz + S.yz * sg2.yz);
    const T val = T(0.5 * Tab<double>::w(N, i) * Tab<double>::w(N, j) * Tab<double>::w(N, k) *
                    cg[CG_DET * N2 + q]) * dz * dens;
    if constexpr (std::is_same<T, Dual>::value) en = val.d;
    else en = val;
    if (w) en *= w[L];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) en += __shfl_xor_sync(0xffffffffu, en, o);
  if ((tid & 31) == 0) red[tid >> 5] = en;
  __syncthreads();
  if (tid == 0) {
    double sum = 0.0;
    for (int ww = 0; ww < NT / 32; ++ww) sum += red[ww];
    elem[blockIdx.x] = sum;
  }
}

// The layer energy split along the eigen-modes of the (cubic-aligned)
// stiffness, for separate loss angles per modulus (Sec. 2.1): with
// T = tr S, D = sum_i S_ii^2, O = S_xy^2 + S_xz^2 + S_yz^2,
//   dilatational   1/2 (c11 + 2 c12) / 3 T^2
//   tetragonal     1/2 (c11 - c12) (D - T^2 / 3)
//   shear          1/2 4 c44 O
// (they sum to 1/2 S : Y : S; isotropic: bulk K T^2 / 2 and shear
// mu S_dev : S_dev = tetragonal + shear).  parts[3 e + j], element e.
template <int N>
__global__ void __launch_bounds__(nthreads<N>())
energy_parts_kernel(const DevMesh m, const double *__restrict__ u, double *__restrict__ parts) {
  constexpr int n = N * N * N, N2 = N * N, NT = nthreads<N>();
  __shared__ double su[3 * n];
  __shared__ double red[3][NT / 32];
  const int e = blockIdx.x, tid = threadIdx.x;
  const int s = e / m.ncol, c = e - s * m.ncol;
  for (int t = tid; t < 3 * n; t += NT) su[t] = u[(size_t)e * 3 * n + t];
  __syncthreads();
  const double *cg = m.colgeo + (size_t)c * CG_NF * N2;
  const int L = m.slab_layer[s];
  const double c11 = m.layer_c[3 * L], c12 = m.layer_c[3 * L + 1], c44 = m.layer_c[3 * L + 2];
  double pe[3] = {0.0, 0.0, 0.0};
  if (tid < n) {
    const int p = tid, i = p % N, j = (p / N) % N, k = p / N2;
    double dxi[3], deta[3], dzeta[3];
    for (int cc = 0; cc < 3; ++cc) {
      const double *v = su + cc * n;
      double a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
      for (int mm = 0; mm < N; ++mm) {
        a0 += Tab<double>::D(N, i, mm) * v[(k * N + j) * N + mm];
        a1 += Tab<double>::D(N, j, mm) * v[(k * N + mm) * N + i];
        a2 += Tab<double>::D(N, k, mm) * v[(mm * N + j) * N + i];
      }
      dxi[cc] = a0; deta[cc] = a1; dzeta[cc] = a2;
    }
    const int q = j * N + i;
    const double dz = slab_dz<double>(m, s, k);
    const Sym<double> S = strain<double>(dxi, deta, dzeta, cg[CG_IXX * N2 + q], cg[CG_IXY * N2 + q],
                                         cg[CG_IEX * N2 + q], cg[CG_IEY * N2 + q], 1.0 / dz);
    const double wJ = 0.5 * Tab<double>::w(N, i) * Tab<double>::w(N, j) * Tab<double>::w(N, k) *
                      cg[CG_DET * N2 + q] * dz;
    const double T = S.xx + S.yy + S.zz, D = S.xx * S.xx + S.yy * S.yy + S.zz * S.zz;
    const double O = S.xy * S.xy + S.xz * S.xz + S.yz * S.yz;
    pe[0] = wJ * (c11 + 2.0 * c12) / 3.0 * T * T;
    pe[1] = wJ * (c11 - c12) * (D - T * T / 3.0);
    pe[2] = wJ * 4.0 * c44 * O;
  }
#pragma unroll
  for (int jj = 0; jj < 3; ++jj) {
    double v = pe[jj];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[jj][tid >> 5] = v;
  }
  __syncthreads();
  if (tid < 3) {
    double sum = 0.0;
    for (int ww = 0; ww < NT / 32; ++ww) sum += red[tid][ww];
    parts[(size_t)e * 3 + tid] = sum;
  }
}

// element energies of a batch: out[b] = energy of element work[b].y of
// instance work[b].x (FP64)
template <int N>
__global__ void __launch_bounds__(nthreads<N>())
energy_batch_kernel(const DevMesh *__restrict__ meshes, const int2 *__restrict__ work,
                    const long long *__restrict__ dof_off, const double *__restrict__ u, double *__restrict__ out) {
  constexpr int n = N * N * N, N2 = N * N, NT = nthreads<N>();
  __shared__ double su[3 * n];
  __shared__ double red[NT / 32];
  __shared__ __align__(16) unsigned char m_raw[sizeof(DevMesh)];
  DevMesh &m = *reinterpret_cast<DevMesh *>(m_raw);
  const int2 w = work[blockIdx.x];
  const int tid = threadIdx.x;
  if (tid == 0) memcpy(m_raw, &meshes[w.x], sizeof(DevMesh));
  __syncthreads();
  const int e = w.y;
  const int s = e / m.ncol, c = e - s * m.ncol;
  const double *ue = u + dof_off[w.x] + (size_t)e * 3 * n;
  for (int t = tid; t < 3 * n; t += NT) su[t] = ue[t];
  __syncthreads();
  const double *cg = m.colgeo + (size_t)c * CG_NF * N2;
  const int L = m.slab_layer[s];
  const double c11 = m.layer_c[3 * L], c12 = m.layer_c[3 * L + 1], c44 = m.layer_c[3 * L + 2];
  double en = 0.0;
  if (tid < n) {
    const int p = tid, i = p % N, j = (p / N) % N, k = p / N2;
    double dxi[3], deta[3], dzeta[3];
    for (int cc = 0; cc < 3; ++cc) {
      const double *v = su + cc * n;
      double a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
      for (int mm = 0; mm < N; ++mm) {
        a0 += Tab<double>::D(N, i, mm) * v[(k * N + j) * N + mm];
        a1 += Tab<double>::D(N, j, mm) * v[(k * N + mm) * N + i];
        a2 += Tab<double>::D(N, k, mm) * v[(mm * N + j) * N + i];
      }
      dxi[cc] = a0; deta[cc] = a1; dzeta[cc] = a2;
    }
    const int q = j * N + i;
    const double dz = m.slabgeo[((size_t)s * SG_NF + SG_DZ) * N + k];
    const Sym<double> S = strain<double>(dxi, deta, dzeta, cg[CG_IXX * N2 + q], cg[CG_IXY * N2 + q],
                                         cg[CG_IEX * N2 + q], cg[CG_IEY * N2 + q], 1.0 / dz);
    const Sym<double> sg2 = stress(S, c11, c12, c44);
    const double dens = S.xx * sg2.xx + S.yy * sg2.yy + S.zz * sg2.zz +
                        2.0 * (S.xy * sg2.xy + S.xz * sg2.xz + S.yz * sg2.yz);
    en = 0.5 * Tab<double>::w(N, i) * Tab<double>::w(N, j) * Tab<double>::w(N, k) * cg[CG_DET * N2 + q] * dz * dens;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) en += __shfl_xor_sync(0xffffffffu, en, o);
  if ((tid & 31) == 0) red[tid >> 5] = en;
  __syncthreads();
  if (tid == 0) {
    double sum = 0.0;
    for (int ww = 0; ww < NT / 32; ++ww) sum += red[ww];
    out[blockIdx.x] = sum;
  }
}

// g_e = w[layer(e)] K_e u: the weak divergence of w detJ Y : sym grad u
// (the volume part of the operator, no faces) -- d(sum_i w_i U_i)/du
template <int N>
__global__ void __launch_bounds__(nthreads<N>())
energy_source_kernel(const DevMesh m, const double *__restrict__ u, const double *__restrict__ w,
                     double *__restrict__ g) {
  constexpr int n = N * N * N, N2 = N * N, NT = nthreads<N>();
  __shared__ double su[3 * n];
  __shared__ double sF[9 * n];
  const int e = blockIdx.x, tid = threadIdx.x;
  const int s = e / m.ncol, c = e - s * m.ncol;
  for (int t = tid; t < 3 * n; t += NT) su[t] = u[(size_t)e * 3 * n + t];
  __syncthreads();
  const double *cg = m.colgeo + (size_t)c * CG_NF * N2;
  const int L = m.slab_layer[s];
  const double c11 = m.layer_c[3 * L], c12 = m.layer_c[3 * L + 1], c44 = m.layer_c[3 * L + 2];
  const double wl = w[L];
  const int p = tid, i = p % N, j = (p / N) % N, k = p / N2;
  if (tid < n) {
    double dxi[3], deta[3], dzeta[3];
    for (int cc = 0; cc < 3; ++cc) {
      const double *v = su + cc * n;
      double a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
      for (int mm = 0; mm < N; ++mm) {
        a0 += Tab<double>::D(N, i, mm) * v[(k * N + j) * N + mm];
        a1 += Tab<double>::D(N, j, mm) * v[(k * N + mm) * N + i];
        a2 += Tab<double>::D(N, k, mm) * v[(mm * N + j) * N + i];
      }
      dxi[cc] = a0; deta[cc] = a1; dzeta[cc] = a2;
    }
    const int q = j * N + i;
    const double ixx = cg[CG_IXX * N2 + q], ixy = cg[CG_IXY * N2 + q];
    const double iex = cg[CG_IEX * N2 + q], iey = cg[CG_IEY * N2 + q];
    const double dz = m.slabgeo[((size_t)s * SG_NF + SG_DZ) * N + k], idz = 1.0 / dz;
    const Sym<double> S = strain<double>(dxi, deta, dzeta, ixx, ixy, iex, iey, idz);
    const double wJ = wl * Tab<double>::w(N, i) * Tab<double>::w(N, j) * Tab<double>::w(N, k) *
                      cg[CG_DET * N2 + q] * dz;
    const Sym<double> Se = {wJ * S.xx, wJ * S.yy, wJ * S.zz, wJ * S.xy, wJ * S.xz, wJ * S.yz};
    const Sym<double> se = stress(Se, c11, c12, c44);
    sF[0 * n + p] = ixx * se.xx + ixy * se.xy;
    sF[1 * n + p] = ixx * se.xy + ixy * se.yy;
    sF[2 * n + p] = ixx * se.xz + ixy * se.yz;
    sF[3 * n + p] = iex * se.xx + iey * se.xy;
    sF[4 * n + p] = iex * se.xy + iey * se.yy;
    sF[5 * n + p] = iex * se.xz + iey * se.yz;
    sF[6 * n + p] = idz * se.xz;
    sF[7 * n + p] = idz * se.yz;
    sF[8 * n + p] = idz * se.zz;
  }
  __syncthreads();
  if (tid < n) {
    for (int cc = 0; cc < 3; ++cc) {
      const double *F0 = sF + cc * n, *F1 = sF + (3 + cc) * n, *F2 = sF + (6 + cc) * n;
      double acc = 0.0;
#pragma unroll
      for (int mm = 0; mm < N; ++mm) {
        acc += Tab<double>::D(N, mm, i) * F0[(k * N + j) * N + mm];
        acc += Tab<double>::D(N, mm, j) * F1[(k * N + mm) * N + i];
        acc += Tab<double>::D(N, mm, k) * F2[(mm * N + j) * N + i];
      }
      g[(size_t)e * 3 * n + cc * n + p] = acc;
    }
  }
}

// partial sums of lam . db/dr0 over the top-surface nodes:
// b_z = -W F0 exp(-r^2/r0^2) / (pi r0^2),  db_z/dr0 = b_z (2 r^2 / r0^3 - 2 / r0)
__global__ void rhs_dr0_kernel(const DevMesh m, double r0, double F0, const double *__restrict__ lam,
                               double *__restrict__ part) {
  const int N = m.N, n = N * N * N, N2 = N * N;
  const size_t total = (size_t)m.ncol * N2;  // top-surface nodes
  const double norm = F0 / (M_PI * r0 * r0), ir2 = 1.0 / (r0 * r0);
  double acc = 0.0;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int e = (int)(t / N2), q = (int)(t % N2), i = q % N, j = q / N;
    const double *g = m.colgeo + (size_t)e * CG_NF * N2;
    const double X = g[CG_X * N2 + q], Y = g[CG_Y * N2 + q], r2 = X * X + Y * Y;
    const double W = c_lgl.w[N][i] * c_lgl.w[N][j] * g[CG_DET * N2 + q];
    const double bz = -W * norm * exp(-r2 * ir2);
    const double dbz = bz * (2.0 * r2 * ir2 / r0 - 2.0 / r0);
    acc += lam[((size_t)e * 3 + 2) * n + (N - 1) * N2 + q] * dbz;
  }
  __shared__ double red[8];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

// one block: per layer, sum the element energies slab by slab in a fixed order
__global__ void layer_sum_kernel(const DevMesh m, const double *__restrict__ elem, double *__restrict__ out) {
  __shared__ double red[32];
  for (int L = 0; L < m.n_layers; ++L) {
    double acc = 0.0;
    for (int s = 0; s < m.nslab; ++s) {
      if (m.slab_layer[s] != L) continue;
      for (int c = threadIdx.x; c < m.ncol; c += blockDim.x) acc += elem[(size_t)s * m.ncol + c];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
      out[L] = sum;
    }
    __syncthreads();
  }
}

template <int N>
cudaError_t launch_energy_n(const DevMesh &m, const double *u, double *elem, cudaStream_t st) {
  energy_kernel<N, double><<<m.E, nthreads<N>(), 0, st>>>(m, 0, u, nullptr, elem);
  return cudaGetLastError();
}

template <int N>
cudaError_t launch_energy_dual_n(const DevMesh &m, int s0, int s1, const double *u, const double *w,
                                 double *epart, cudaStream_t st) {
  const int nblk = (s1 - s0) * m.ncol;
  if (nblk <= 0) return cudaSuccess;
  energy_kernel<N, Dual><<<nblk, nthreads<N>(), 0, st>>>(m, s0 * m.ncol, u, w, epart);
  return cudaGetLastError();
}

}  // namespace

cudaError_t tn_launch_apply(const DevMesh &m, int precision, const void *u, void *y,
                            double *partial, int var, cudaStream_t st, const PcgFold *fold) {
  const PcgFold f = fold ? *fold : PcgFold();
  if (precision == TN_F64)
    return launch_apply_t<double>(m, (const double *)u, (double *)y, partial, st, 0, f);
  return launch_apply_t<float>(m, (const float *)u, (float *)y, partial, st, var, f);
}

int tn_apply_ctas(const DevMesh *m, int nwork) { return m ? m->E : nwork; }

cudaError_t tn_tune_apply(const DevMesh *m1, int N, const DevMesh *meshes, const int2 *work, int nwork,
                          const long long *dof_off, const float *u, float *y, cudaStream_t st, float us[2]) {
  switch (N) {
    case 3: return tune_apply2<3>(m1, meshes, work, nwork, dof_off, u, y, st, us);
    case 4: return tune_apply2<4>(m1, meshes, work, nwork, dof_off, u, y, st, us);
    case 5: return tune_apply2<5>(m1, meshes, work, nwork, dof_off, u, y, st, us);
    case 6: return tune_apply2<6>(m1, meshes, work, nwork, dof_off, u, y, st, us);
    case 7: return tune_apply2<7>(m1, meshes, work, nwork, dof_off, u, y, st, us);
    case 8: return tune_apply2<8>(m1, meshes, work, nwork, dof_off, u, y, st, us);
    case 9: return tune_apply2<9>(m1, meshes, work, nwork, dof_off, u, y, st, us);
    default: return cudaErrorInvalidValue;
  }
}

int tn_sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (!cache[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 152;
    cache[dev] = n;
  }
  return cache[dev];
}

cudaError_t tn_launch_rhs(const DevMesh &m, double r0, double F0, double *b, cudaStream_t st) {
  rhs_kernel<<<4 * tn_sm_count(), 256, 0, st>>>(m, r0, F0, b);
  return cudaGetLastError();
}

cudaError_t tn_launch_diag(const DevMesh &m, double *d, cudaStream_t st) {
  diag_kernel<<<m.E, 128, 0, st>>>(m, d);
  return cudaGetLastError();
}

cudaError_t tn_launch_energy(const DevMesh &m, const double *u, double *elem, double *layer,
                             cudaStream_t st) {
  cudaError_t err;
  switch (m.N) {
    case 3: err = launch_energy_n<3>(m, u, elem, st); break;
    case 4: err = launch_energy_n<4>(m, u, elem, st); break;
    case 5: err = launch_energy_n<5>(m, u, elem, st); break;
    case 6: err = launch_energy_n<6>(m, u, elem, st); break;
    case 7: err = launch_energy_n<7>(m, u, elem, st); break;
    case 8: err = launch_energy_n<8>(m, u, elem, st); break;
    case 9: err = launch_energy_n<9>(m, u, elem, st); break;
    default: return cudaErrorInvalidValue;
  }
  if (err != cudaSuccess) return err;
  layer_sum_kernel<<<1, 256, 0, st>>>(m, elem, layer);
  return cudaGetLastError();
}

cudaError_t tn_launch_energy_parts(const DevMesh &m, const double *u, double *parts, cudaStream_t st) {
  switch (m.N) {
#define TN_CASE(NN) \
    case NN: energy_parts_kernel<NN><<<m.E, nthreads<NN>(), 0, st>>>(m, u, parts); return cudaGetLastError();
    TN_CASE(3) TN_CASE(4) TN_CASE(5) TN_CASE(6) TN_CASE(7) TN_CASE(8) TN_CASE(9)
#undef TN_CASE
    default: return cudaErrorInvalidValue;
  }
}

#define TN_DISPATCH_N(...)                  \
  switch (m.N) {                            \
    case 3: { constexpr int NN = 3; __VA_ARGS__; } \
    case 4: { constexpr int NN = 4; __VA_ARGS__; } \
    case 5: { constexpr int NN = 5; __VA_ARGS__; } \
    case 6: { constexpr int NN = 6; __VA_ARGS__; } \
    case 7: { constexpr int NN = 7; __VA_ARGS__; } \
    case 8: { constexpr int NN = 8; __VA_ARGS__; } \
    case 9: { constexpr int NN = 9; __VA_ARGS__; } \
    default: return cudaErrorInvalidValue;  \
  }

cudaError_t tn_launch_apply_dual(const DevMesh &m, int s0, int s1, const double *u, const double *lam,
                                 double *part, cudaStream_t st) {
  TN_DISPATCH_N(return launch_apply_range<NN, Dual, double>(m, s0, s1, u, nullptr, part, lam, st))
}

cudaError_t tn_launch_energy_dual(const DevMesh &m, int s0, int s1, const double *u, const double *w,
                                  double *epart, cudaStream_t st) {
  TN_DISPATCH_N(return launch_energy_dual_n<NN>(m, s0, s1, u, w, epart, st))
}

cudaError_t tn_launch_apply_dual_work(const DevMesh &m, const int2 *work, int nwork, const double *const *pseed,
                                      const double *u, const double *lam, double *part, cudaStream_t st) {
  if (nwork <= 0) return cudaSuccess;
  TN_DISPATCH_N({
    constexpr size_t sm = apply_smem<NN, Dual>();
    static int configured_device = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_device != dev) {
      cudaError_t err = cudaFuncSetAttribute(apply_kernel<NN, Dual, double>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (err != cudaSuccess) return err;
      configured_device = dev;
    }
    apply_kernel<NN, Dual, double><<<nwork, nthreads<NN>(), sm, st>>>(m, 0, u, nullptr, part, lam, work, pseed);
    return cudaGetLastError();
  })
}

cudaError_t tn_launch_energy_dual_work(const DevMesh &m, const int2 *work, int nwork, const double *const *pseed,
                                       const double *u, const double *w, double *epart, cudaStream_t st) {
  if (nwork <= 0) return cudaSuccess;
  TN_DISPATCH_N({
    energy_kernel<NN, Dual><<<nwork, nthreads<NN>(), 0, st>>>(m, 0, u, w, epart, work, pseed);
    return cudaGetLastError();
  })
}

cudaError_t tn_launch_energy_source(const DevMesh &m, const double *u, const double *w, double *g,
                                    cudaStream_t st) {
  TN_DISPATCH_N(energy_source_kernel<NN><<<m.E, nthreads<NN>(), 0, st>>>(m, u, w, g); return cudaGetLastError())
}

cudaError_t tn_launch_rhs_dr0(const DevMesh &m, double r0, double F0, const double *lam, double *part,
                              int nparts, cudaStream_t st) {
  rhs_dr0_kernel<<<nparts, 256, 0, st>>>(m, r0, F0, lam, part);
  return cudaGetLastError();
}

cudaError_t tn_launch_apply_batch(int N, int precision, const DevMesh *meshes, const int2 *work, int nwork,
                                  const long long *dof_off, const void *u, void *y, double *partial,
                                  int var, cudaStream_t st, const PcgFold *fold) {
  const PcgFold f = fold ? *fold : PcgFold();
  switch (N) {
#define TN_CASE(NN)                                                                                    \
  case NN:                                                                                            \
    return precision == TN_F64                                                                        \
               ? launch_apply2_batch<NN, double>(meshes, work, nwork, dof_off, (const double *)u,    \
                                                 (double *)y, partial, st, 0, f)                      \
               : launch_apply2_batch<NN, float>(meshes, work, nwork, dof_off, (const float *)u,      \
                                                (float *)y, partial, st, var, f);
    TN_CASE(3) TN_CASE(4) TN_CASE(5) TN_CASE(6) TN_CASE(7) TN_CASE(8) TN_CASE(9)
#undef TN_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t tn_launch_energy_batch(int N, const DevMesh *meshes, const int2 *work, int nwork,
                                   const long long *dof_off, const double *u, double *out, cudaStream_t st) {
  if (nwork <= 0) return cudaSuccess;
  switch (N) {
#define TN_CASE(NN)                                                                                    \
  case NN:                                                                                            \
    energy_batch_kernel<NN><<<nwork, nthreads<NN>(), 0, st>>>(meshes, work, dof_off, u, out);          \
    return cudaGetLastError();
    TN_CASE(3) TN_CASE(4) TN_CASE(5) TN_CASE(6) TN_CASE(7) TN_CASE(8) TN_CASE(9)
#undef TN_CASE
    default: return cudaErrorInvalidValue;
  }
}
