/*
 * Oracle: Q1 finite-element discretisation in space (Sec. 3.2, Eq. semi-disc),
 * lumped mass, cell-constant anisotropic conductivity, stimulus initial state.
 * TEST INFRASTRUCTURE ONLY -- see oracle.h.
 *
 * The element matrices are integrated by the 2-point Gauss rule per axis, which
 * is exact for the products of Q1 basis functions and their gradients:
 *   K^e_ab = int_e (D grad phi_a) . grad phi_b,    m_a = sum_b int_e phi_a phi_b.
 * The conductivity (Sec. 2.1, fiber tensor of the workloads) is constant per
 * cell:  D = s_t I + (s_l - s_t) f f^T,  s_l = s_l0 exp(Z(centroid)),
 *        f = (cos th, sin th, 0),  th = theta0 (2D) or linear in z (3D).
 * Nodes and cells are numbered with x fastest; the stiffness of node A is
 * stored as its couplings to the 3^dim offsets {-1,0,1}^dim, x fastest.
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

int or_nodes(const or_level* lv) {
  int n = 1;
  for (int d = 0; d < lv->dim; ++d) n *= lv->n[d] + 1;
  return n;
}

int or_cells(const or_level* lv) {
  int n = 1;
  for (int d = 0; d < lv->dim; ++d) n *= lv->n[d];
  return n;
}

/* couplings per node: the 3^dim offsets in {-1,0,1}^dim, x fastest */
int or_n_offsets(int dim) { return dim == 3 ? 27 : (dim == 2 ? 9 : 3); }
static int n_off(int dim) { return or_n_offsets(dim); }

void or_assemble(const or_level* lv, const double* Z, double* mass, double* Kst) {
  const double pi = 3.14159265358979323846;
  int dim = lv->dim;
  int nx = lv->n[0], ny = dim >= 2 ? lv->n[1] : 1, nz = dim == 3 ? lv->n[2] : 1;
  int Nx = nx + 1, Ny = dim >= 2 ? ny + 1 : 1;
  int nodes = or_nodes(lv), no = n_off(dim), nloc = 1 << dim;
  double h[3] = {lv->L[0] / nx, dim >= 2 ? lv->L[1] / ny : 1.0, dim == 3 ? lv->L[2] / nz : 1.0};
  double vol = h[0] * h[1] * h[2];
  memset(mass, 0, sizeof(double) * nodes);
  memset(Kst, 0, sizeof(double) * (size_t)nodes * no);
  const double gp[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
  int ngauss = 1 << dim;
  for (int kz = 0; kz < nz; ++kz)
    for (int jy = 0; jy < ny; ++jy)
      for (int ix = 0; ix < nx; ++ix) {
        int cell = (kz * ny + jy) * nx + ix;
        double th = lv->theta0;
        if (dim == 3) th = lv->theta0 + (lv->theta1 - lv->theta0) * ((kz + 0.5) * h[2]) / lv->L[2];
        th = th * pi / 180.0;
        double f[3] = {cos(th), sin(th), 0.0};
        double D[3][3];
        if (lv->cond_kind == 1) {   /* the paper's isotropic G = G0 (1 + Z) */
          double g = lv->s_l0 * (1.0 + Z[cell]);
          for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) D[p][q] = p == q ? g : 0.0;
        } else {
          double sl = lv->s_l0 * exp(Z[cell]);
          for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) D[p][q] = (p == q ? lv->s_t : 0.0) + (sl - lv->s_t) * f[p] * f[q];
        }
        double Ke[8][8]; double me[8];
        memset(Ke, 0, sizeof(Ke)); memset(me, 0, sizeof(me));
        for (int g = 0; g < ngauss; ++g) {
          double xi[3] = {gp[g & 1], dim >= 2 ? gp[(g >> 1) & 1] : 0.0, dim == 3 ? gp[(g >> 2) & 1] : 0.0};
          double w = vol / (double)ngauss; /* Gauss weights 1/2 per axis times |J| */
          double phi[8], grad[8][3];
          for (int a = 0; a < nloc; ++a) {
            double fac[3], dfac[3];
            for (int d = 0; d < dim; ++d) {
              int bit = (a >> d) & 1;
              fac[d] = bit ? xi[d] : 1.0 - xi[d];
              dfac[d] = (bit ? 1.0 : -1.0) / h[d];
            }
            phi[a] = 1.0;
            for (int d = 0; d < dim; ++d) phi[a] *= fac[d];
            for (int d = 0; d < dim; ++d) {
              double gd = dfac[d];
              for (int e = 0; e < dim; ++e) if (e != d) gd *= fac[e];
              grad[a][d] = gd;
            }
          }
          for (int a = 0; a < nloc; ++a) {
            for (int b = 0; b < nloc; ++b) {
              double s = 0.0;
              for (int p = 0; p < dim; ++p)
                for (int q = 0; q < dim; ++q) s += D[p][q] * grad[b][q] * grad[a][p];
              Ke[a][b] += w * s;
              me[a] += w * phi[a] * phi[b];
            }
          }
        }
        for (int a = 0; a < nloc; ++a) {
          int ai = ix + (a & 1), aj = jy + ((a >> 1) & 1), ak = kz + ((a >> 2) & 1);
          int A = (ak * Ny + aj) * Nx + ai;
          mass[A] += me[a];
          for (int b = 0; b < nloc; ++b) {
            int di = (b & 1) - (a & 1), dj = ((b >> 1) & 1) - ((a >> 1) & 1);
            int dk = ((b >> 2) & 1) - ((a >> 2) & 1);
            int o = (di + 1) + (dim >= 2 ? 3 * (dj + 1) : 0) + (dim == 3 ? 9 * (dk + 1) : 0);
            Kst[(size_t)A * no + o] += Ke[a][b];
          }
        }
      }
}

void or_stiff_apply(const or_level* lv, const double* Kst, const double* v, double* y) {
  int dim = lv->dim;
  int Nx = lv->n[0] + 1, Ny = dim >= 2 ? lv->n[1] + 1 : 1, Nz = dim == 3 ? lv->n[2] + 1 : 1;
  int no = n_off(dim);
  for (int k = 0; k < Nz; ++k)
    for (int j = 0; j < Ny; ++j)
      for (int i = 0; i < Nx; ++i) {
        int A = (k * Ny + j) * Nx + i;
        double s = 0.0;
        for (int o = 0; o < no; ++o) {
          int di = o % 3 - 1, dj = dim >= 2 ? (o / 3) % 3 - 1 : 0, dk = dim == 3 ? o / 9 - 1 : 0;
          int ii = i + di, jj = j + dj, kk = k + dk;
          if (ii < 0 || ii >= Nx || jj < 0 || jj >= Ny || kk < 0 || kk >= Nz) continue;
          s += Kst[(size_t)A * no + o] * v[(kk * Ny + jj) * Nx + ii];
        }
        y[A] = s;
      }
}

void or_initial(const or_level* lv, double* u0) {
  int dim = lv->dim;
  if (lv->stim_kind == 1) {   /* the applied current starts from rest */
    int n = or_nodes(lv);
    for (int i = 0; i < n; ++i) u0[i] = 0.0;
    return;
  }
  int Nx = lv->n[0] + 1, Ny = dim >= 2 ? lv->n[1] + 1 : 1, Nz = dim == 3 ? lv->n[2] + 1 : 1;
  double h[3] = {lv->L[0] / lv->n[0], dim >= 2 ? lv->L[1] / lv->n[1] : 0.0,
                 dim == 3 ? lv->L[2] / lv->n[2] : 0.0};
  for (int k = 0; k < Nz; ++k)
    for (int j = 0; j < Ny; ++j)
      for (int i = 0; i < Nx; ++i) {
        double x[3] = {i * h[0], j * h[1], k * h[2]};
        double r2 = 0.0;
        for (int d = 0; d < dim; ++d) r2 += (x[d] - lv->stim_c[d]) * (x[d] - lv->stim_c[d]);
        u0[(k * Ny + j) * Nx + i] = r2 < lv->stim_r * lv->stim_r ? 1.0 : 0.0;
      }
}

/* Applied current of the paper's set-up (Sec. 4): I_app(x, t) =
 * stim_amp exp(-|x - x0|^2 / sigma^2) for 0 <= t < t1, averaged over step k:
 * the time integral over [t_{k-1}, t_k] (the overlap with [0, t1)) over dt. */
void or_stimulus_step(const or_level* lv, int k, double* s) {
  int dim = lv->dim, n = or_nodes(lv);
  if (lv->stim_kind != 1) {
    for (int i = 0; i < n; ++i) s[i] = 0.0;
    return;
  }
  double dt = lv->T / lv->m;
  double a = (k - 1) * dt, b = k * dt;
  double overlap = fmin(b, lv->stim_t1) - a;
  if (overlap < 0.0) overlap = 0.0;
  int Nx = lv->n[0] + 1, Ny = dim >= 2 ? lv->n[1] + 1 : 1, Nz = dim == 3 ? lv->n[2] + 1 : 1;
  double h[3] = {lv->L[0] / lv->n[0], dim >= 2 ? lv->L[1] / lv->n[1] : 0.0,
                 dim == 3 ? lv->L[2] / lv->n[2] : 0.0};
  for (int kk = 0; kk < Nz; ++kk)
    for (int j = 0; j < Ny; ++j)
      for (int i = 0; i < Nx; ++i) {
        double x[3] = {i * h[0], j * h[1], kk * h[2]};
        double r2 = 0.0;
        for (int d = 0; d < dim; ++d) r2 += (x[d] - lv->stim_c[d]) * (x[d] - lv->stim_c[d]);
        s[(kk * Ny + j) * Nx + i] =
            overlap > 0.0 ? lv->stim_amp * exp(-r2 / (lv->stim_sigma * lv->stim_sigma)) * overlap / dt : 0.0;
      }
}
