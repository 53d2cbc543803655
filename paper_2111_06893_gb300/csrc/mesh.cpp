// Host-side mesh construction: LGL tables, the factorised element geometry
// (column cross-section maps x slab vertical maps) and the face-neighbour
// tables of the box and cylinder decompositions of Sec. 2.2.1 / Fig. 1.
//
// Geometry is evaluated from closed-form derivatives of the maps in FP64:
//   square block   (X, Y) = a (xi, eta)
//   inner wedge    (X, Y) = (1-xi)/2 (a, a eta) + (1+xi)/2 R1 (cos t, sin t)
//   outer wedge    (X, Y) = ((1-xi)/2 R1 + (1+xi)/2 R) (cos t, sin t)
//   with t = pi eta / 4, rotated by 90 degree steps for the other wedges;
//   slabs: z linear in zeta, or log-linear in depth -z (substrate slabs).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "tn_internal.h"

namespace tn {

// LGL nodes by Newton's method on P'_{N-1} (Legendre recurrence), weights
// 2 / (N (N-1) P_{N-1}^2), derivative matrix from barycentric weights.
static void legendre_pd(int n, double x, double *P, double *dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int m = 1; m < n; ++m) {
    double p2 = ((2.0 * m + 1.0) * x * p1 - m * p0) / (m + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  *dP = n * (p0 - x * p1) / (1.0 - x * x);
}

void lgl(int N, double *x, double *w, double *D) {
  const int n = N - 1;
  for (int a = 0; a < N; ++a) x[a] = -std::cos(M_PI * a / n);
  for (int a = 1; a < n; ++a) {
    for (int it = 0; it < 200; ++it) {
      double P, dP;
      legendre_pd(n, x[a], &P, &dP);
      double d2P = (2.0 * x[a] * dP - n * (n + 1.0) * P) / (1.0 - x[a] * x[a]);
      double dx = dP / d2P;
      x[a] -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
  }
  x[0] = -1.0;
  x[n] = 1.0;
  // symmetrise the nodes exactly
  for (int a = 0; a < N / 2; ++a) {
    double s = 0.5 * (x[n - a] - x[a]);
    x[a] = -s;
    x[n - a] = s;
  }
  if (N % 2) x[N / 2] = 0.0;
  for (int a = 0; a < N; ++a) {
    double p0 = 1.0, p1 = x[a];
    for (int m = 1; m < n; ++m) {
      double p2 = ((2.0 * m + 1.0) * x[a] * p1 - m * p0) / (m + 1.0);
      p0 = p1;
      p1 = p2;
    }
    w[a] = 2.0 / (N * n * p1 * p1);
  }
  std::vector<double> lam(N);
  for (int b = 0; b < N; ++b) {
    double prod = 1.0;
    for (int m = 0; m < N; ++m)
      if (m != b) prod *= (x[b] - x[m]);
    lam[b] = 1.0 / prod;
  }
  for (int a = 0; a < N; ++a) {
    double diag = 0.0;
    for (int b = 0; b < N; ++b) {
      if (a == b) continue;
      double v = (lam[b] / lam[a]) / (x[a] - x[b]);
      D[a * N + b] = v;
      diag -= v;
    }
    D[a * N + a] = diag;
  }
}

static void set_err(char *msg, int len, const char *s) {
  if (msg && len > 0) std::snprintf(msg, len, "%s", s);
}

// 2x2 Jacobian of a cross-section map at block coordinates (xb, eb):
// J[0] = dX/dxi, J[1] = dX/deta, J[2] = dY/dxi, J[3] = dY/deta
static void rotate(int r, double *X, double *Y) {
  double x = *X, y = *Y;
  switch (r & 3) {
    case 0: break;
    case 1: *X = -y; *Y = x; break;
    case 2: *X = -x; *Y = -y; break;
    default: *X = y; *Y = -x; break;
  }
}

static void cyl_block_map(int blk, double xb, double eb, double a, double R1, double R,
                          double *X, double *Y, double J[4]) {
  if (blk == 0) {
    *X = a * xb;
    *Y = a * eb;
    J[0] = a; J[1] = 0.0; J[2] = 0.0; J[3] = a;
    return;
  }
  const double t = M_PI * eb / 4.0, ct = std::cos(t), st = std::sin(t), dt = M_PI / 4.0;
  double X0, Y0, j0, j1, j2, j3;
  if (blk <= 4) {
    X0 = 0.5 * (1 - xb) * a + 0.5 * (1 + xb) * R1 * ct;
    Y0 = 0.5 * (1 - xb) * a * eb + 0.5 * (1 + xb) * R1 * st;
    j0 = -0.5 * a + 0.5 * R1 * ct;
    j1 = -0.5 * (1 + xb) * R1 * st * dt;
    j2 = -0.5 * a * eb + 0.5 * R1 * st;
    j3 = 0.5 * (1 - xb) * a + 0.5 * (1 + xb) * R1 * ct * dt;
  } else {
    const double rho = 0.5 * (1 - xb) * R1 + 0.5 * (1 + xb) * R;
    X0 = rho * ct;
    Y0 = rho * st;
    j0 = 0.5 * (R - R1) * ct;
    j1 = -rho * st * dt;
    j2 = 0.5 * (R - R1) * st;
    j3 = rho * ct * dt;
  }
  const int r = (blk - 1) % 4;
  double cx = j0, cy = j2;  // column dxi of (X0, Y0)
  double ex = j1, ey = j3;  // column deta
  rotate(r, &X0, &Y0);
  rotate(r, &cx, &cy);
  rotate(r, &ex, &ey);
  *X = X0;
  *Y = Y0;
  J[0] = cx; J[1] = ex; J[2] = cy; J[3] = ey;
}

tn_status build_host_mesh(const tn_mesh_desc *d, HostMesh *out, char *msg, int msglen) {
  if (!d || !out) { set_err(msg, msglen, "null argument"); return TN_EINVAL; }
  const int p = d->degree, N = p + 1;
  if (N < TN_MIN_N || N > TN_MAX_N) { set_err(msg, msglen, "degree must be in 2..8"); return TN_EINVAL; }
  if (d->n_slabs < 1 || !d->slab_z || !d->slab_layer || !d->slab_log) {
    set_err(msg, msglen, "need n_slabs >= 1 and slab arrays"); return TN_EINVAL;
  }
  if (d->n_layers < 1) { set_err(msg, msglen, "n_layers must be >= 1"); return TN_EINVAL; }
  if (!(d->penalty_C > 0.0)) { set_err(msg, msglen, "penalty_C must be > 0"); return TN_EINVAL; }
  if ((d->bc_side != TN_BC_FREE && d->bc_side != TN_BC_FIXED) ||
      (d->bc_bottom != TN_BC_FREE && d->bc_bottom != TN_BC_FIXED)) {
    set_err(msg, msglen, "bc must be TN_BC_FREE or TN_BC_FIXED"); return TN_EINVAL;
  }
  if (d->slab_z[0] != 0.0) { set_err(msg, msglen, "slab_z[0] must be 0 (top surface)"); return TN_EINVAL; }
  for (int s = 0; s < d->n_slabs; ++s) {
    if (!(d->slab_z[s + 1] < d->slab_z[s])) { set_err(msg, msglen, "slab_z must decrease"); return TN_EINVAL; }
    if (d->slab_layer[s] < 0 || d->slab_layer[s] >= d->n_layers) {
      set_err(msg, msglen, "slab_layer out of range"); return TN_EINVAL;
    }
    if (d->slab_log[s] && !(d->slab_z[s] < 0.0)) {
      set_err(msg, msglen, "a logarithmic slab must start below z = 0"); return TN_EINVAL;
    }
  }
  int ncol = 0;
  if (d->kind == TN_MESH_BOX) {
    if (d->nx < 1 || d->ny < 1 || !d->x_breaks || !d->y_breaks) {
      set_err(msg, msglen, "box needs nx, ny >= 1 and break arrays"); return TN_EINVAL;
    }
    for (int i = 0; i < d->nx; ++i)
      if (!(d->x_breaks[i + 1] > d->x_breaks[i])) { set_err(msg, msglen, "x_breaks must increase"); return TN_EINVAL; }
    for (int j = 0; j < d->ny; ++j)
      if (!(d->y_breaks[j + 1] > d->y_breaks[j])) { set_err(msg, msglen, "y_breaks must increase"); return TN_EINVAL; }
    ncol = d->nx * d->ny;
  } else if (d->kind == TN_MESH_CYLINDER) {
    if (d->k < 1 || !(d->a > 0.0) || !(d->R1 > d->a * std::sqrt(2.0)) || !(d->R > d->R1)) {
      set_err(msg, msglen, "cylinder needs k >= 1 and 0 < a*sqrt(2) < R1 < R"); return TN_EINVAL;
    }
    ncol = 9 * d->k * d->k;
  } else {
    set_err(msg, msglen, "unknown mesh kind"); return TN_EINVAL;
  }
  const long long E = (long long)ncol * d->n_slabs;
  if (E <= 0 || E * 3LL * N * N * N > (1LL << 40)) { set_err(msg, msglen, "mesh too large"); return TN_EINVAL; }

  HostMesh m;
  m.N = N; m.p = p; m.ncol = ncol; m.nslab = d->n_slabs; m.E = (int)E;
  m.n_layers = d->n_layers; m.bc_side = d->bc_side; m.bc_bottom = d->bc_bottom;
  m.penC = d->penalty_C;
  double x[TN_MAX_N], w[TN_MAX_N], D[TN_MAX_N * TN_MAX_N];
  lgl(N, x, w, D);
  const int N2 = N * N;
  m.colgeo = (double *)std::calloc((size_t)ncol * CG_NF * N2, sizeof(double));
  m.slabgeo = (double *)std::calloc((size_t)m.nslab * SG_NF * N, sizeof(double));
  m.colnb = (int *)std::malloc(sizeof(int) * ncol * 4);
  m.colnbf = (int *)std::malloc(sizeof(int) * ncol * 4);
  m.slab_layer = (int *)std::malloc(sizeof(int) * m.nslab);
  if (!m.colgeo || !m.slabgeo || !m.colnb || !m.colnbf || !m.slab_layer) {
    free_host_mesh(&m);
    set_err(msg, msglen, "host allocation failed");
    return TN_ENOMEM;
  }
  // ---- columns: geometry and neighbours
  for (int c = 0; c < ncol; ++c) {
    double *g = m.colgeo + (size_t)c * CG_NF * N2;
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) {
        double X, Y, J[4];
        if (d->kind == TN_MESH_BOX) {
          const int ix = c % d->nx, jy = c / d->nx;
          const double x0 = d->x_breaks[ix], x1 = d->x_breaks[ix + 1];
          const double y0 = d->y_breaks[jy], y1 = d->y_breaks[jy + 1];
          X = x0 + 0.5 * (1 + x[i]) * (x1 - x0);
          Y = y0 + 0.5 * (1 + x[j]) * (y1 - y0);
          J[0] = 0.5 * (x1 - x0); J[1] = 0.0; J[2] = 0.0; J[3] = 0.5 * (y1 - y0);
        } else {
          const int k = d->k, blk = c / (k * k), cl = c % (k * k), bi = cl / k, ai = cl % k;
          const double xb = -1.0 + (2.0 * ai + 1.0 + x[i]) / k;
          const double eb = -1.0 + (2.0 * bi + 1.0 + x[j]) / k;
          cyl_block_map(blk, xb, eb, d->a, d->R1, d->R, &X, &Y, J);
          for (int t = 0; t < 4; ++t) J[t] /= k;
        }
        const double det = J[0] * J[3] - J[1] * J[2];
        if (!(det > 0.0)) {
          free_host_mesh(&m);
          set_err(msg, msglen, "non-positive cross-section Jacobian");
          return TN_EINVAL;
        }
        const int q = j * N + i;
        g[CG_IXX * N2 + q] = J[3] / det;   // dxi/dx
        g[CG_IXY * N2 + q] = -J[1] / det;  // dxi/dy
        g[CG_IEX * N2 + q] = -J[2] / det;  // deta/dx
        g[CG_IEY * N2 + q] = J[0] / det;   // deta/dy
        g[CG_DET * N2 + q] = det;
        g[CG_X * N2 + q] = X;
        g[CG_Y * N2 + q] = Y;
      }
    int *nb = m.colnb + 4 * c, *nf = m.colnbf + 4 * c;
    if (d->kind == TN_MESH_BOX) {
      const int ix = c % d->nx, jy = c / d->nx;
      nb[0] = ix > 0 ? c - 1 : -1;              nf[0] = 1;
      nb[1] = ix < d->nx - 1 ? c + 1 : -1;      nf[1] = 0;
      nb[2] = jy > 0 ? c - d->nx : -1;          nf[2] = 3;
      nb[3] = jy < d->ny - 1 ? c + d->nx : -1;  nf[3] = 2;
    } else {
      const int k = d->k, kk = k * k, blk = c / kk, cl = c % kk, bi = cl / k, ai = cl % k;
      auto col = [&](int b, int a_, int b_) { return b * kk + b_ * k + a_; };
      // inside a block
      nb[0] = ai > 0 ? col(blk, ai - 1, bi) : -2;          nf[0] = 1;
      nb[1] = ai < k - 1 ? col(blk, ai + 1, bi) : -2;      nf[1] = 0;
      nb[2] = bi > 0 ? col(blk, ai, bi - 1) : -2;          nf[2] = 3;
      nb[3] = bi < k - 1 ? col(blk, ai, bi + 1) : -2;      nf[3] = 2;
      if (blk == 0) {  // square: faces to the inner wedges
        if (nb[1] == -2) { nb[1] = col(1, 0, bi); nf[1] = 0; }                 // x = +a, aligned
        if (nb[3] == -2) { nb[3] = col(2, 0, k - 1 - ai); nf[3] = 0 | 4; }     // y = +a, reversed
        if (nb[0] == -2) { nb[0] = col(3, 0, k - 1 - bi); nf[0] = 0 | 4; }     // x = -a, reversed
        if (nb[2] == -2) { nb[2] = col(4, 0, ai); nf[2] = 0; }                 // y = -a, aligned
      } else if (blk <= 4) {
        const int r = blk - 1;
        if (nb[0] == -2) {  // to the square
          switch (r) {
            case 0: nb[0] = col(0, k - 1, bi); nf[0] = 1; break;
            case 1: nb[0] = col(0, k - 1 - bi, k - 1); nf[0] = 3 | 4; break;
            case 2: nb[0] = col(0, 0, k - 1 - bi); nf[0] = 0 | 4; break;
            default: nb[0] = col(0, bi, 0); nf[0] = 2; break;
          }
        }
        if (nb[1] == -2) { nb[1] = col(5 + r, 0, bi); nf[1] = 0; }
        if (nb[3] == -2) { nb[3] = col(1 + (r + 1) % 4, ai, 0); nf[3] = 2; }
        if (nb[2] == -2) { nb[2] = col(1 + (r + 3) % 4, ai, k - 1); nf[2] = 3; }
      } else {
        const int r = blk - 5;
        if (nb[0] == -2) { nb[0] = col(1 + r, k - 1, bi); nf[0] = 1; }
        if (nb[1] == -2) { nb[1] = -1; nf[1] = 0; }  // mantle
        if (nb[3] == -2) { nb[3] = col(5 + (r + 1) % 4, ai, 0); nf[3] = 2; }
        if (nb[2] == -2) { nb[2] = col(5 + (r + 3) % 4, ai, k - 1); nf[2] = 3; }
      }
    }
  }
  // ---- slabs
  for (int s = 0; s < m.nslab; ++s) {
    double *g = m.slabgeo + (size_t)s * SG_NF * N;
    const double zt = d->slab_z[s], zb = d->slab_z[s + 1];
    for (int k = 0; k < N; ++k) {
      double z, dz;
      if (d->slab_log[s]) {
        const double lt = std::log(-zt), lb = std::log(-zb);
        const double depth = std::exp(0.5 * (1 + x[k]) * lt + 0.5 * (1 - x[k]) * lb);
        z = -depth;
        dz = 0.5 * depth * (lb - lt);
      } else {
        z = 0.5 * (1 + x[k]) * zt + 0.5 * (1 - x[k]) * zb;
        dz = 0.5 * (zt - zb);
      }
      g[SG_DZ * N + k] = dz;
      g[SG_Z * N + k] = z;
    }
    m.slab_layer[s] = d->slab_layer[s];
  }
  *out = m;
  return TN_OK;
}

void free_host_mesh(HostMesh *m) {
  std::free(m->colgeo);
  std::free(m->slabgeo);
  std::free(m->colnb);
  std::free(m->colnbf);
  std::free(m->slab_layer);
  m->colgeo = m->slabgeo = nullptr;
  m->colnb = m->colnbf = m->slab_layer = nullptr;
}

}  // namespace tn
