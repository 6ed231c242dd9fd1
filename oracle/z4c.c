/*
 * Oracle (test infrastructure only): BSSN-Z4c right-hand side (Sec. II.B.1,
 * Eq. bssn and Eq. moving_puncture), cartoon y-derivatives (Sec. II.B.2,
 * Eq. cartoon_bnd), Kreiss-Oliger dissipation, matter terms and the
 * constraint diagnostics (Sec. II.F.1) of Lam & Shibata (arXiv:2502.03223).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "orc.h"

static const int S6[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};

/* ---------------- parities (reading: rotation by pi about the z axis, equatorial mirror) ---------------- */

/* x -> -x parity of the y = 0 plane is the rotation by pi about the z axis:
   x and y components of vectors and the xz, yz tensor components flip sign. */
int orc_field_parity_x(int f) {
  switch (f) {
    case O_GX: case O_GY: case O_BX: case O_BY: case O_BBX: case O_BBY:
    case O_HXZ: case O_HYZ: case O_AXZ: case O_AYZ:
      return -1;
    default:
      return 1;
  }
}

/* z -> -z mirror: z components of vectors and the xz, yz tensor components flip sign. */
int orc_field_parity_z(int f) {
  switch (f) {
    case O_GZ: case O_BZ: case O_BBZ:
    case O_HXZ: case O_HYZ: case O_AXZ: case O_AYZ:
      return -1;
    default:
      return 1;
  }
}

int orc_prim_parity_x(int f) { return (f == O_UX || f == O_UY) ? -1 : 1; }
int orc_prim_parity_z(int f) { return (f == O_UZ) ? -1 : 1; }

/* fields whose d_y, d_xy, d_yz are set to zero (Sec. II.B.2): scalars, z
   components of vectors, zz components of tensors */
static int y_zero(int f) {
  switch (f) {
    case O_W: case O_KH: case O_TH: case O_AL:
    case O_GZ: case O_BZ: case O_BBZ: case O_HZZ: case O_AZZ:
      return 1;
    default:
      return 0;
  }
}

/* ---------------- cartoon planes, Sec. II.B.2 ---------------- */

static void rotate_vec(double c, double s, const double *in, double *out, int ix, int iy, int iz) {
  out[ix] = c * in[ix] - s * in[iy];
  out[iy] = s * in[ix] + c * in[iy];
  out[iz] = in[iz];
}

/* tensor components at offsets xx,xy,xz,yy,yz,zz from base */
static void rotate_ten(double c, double s, const double *in, double *out, int b) {
  double txx = in[b], txy = in[b + 1], txz = in[b + 2], tyy = in[b + 3], tyz = in[b + 4], tzz = in[b + 5];
  out[b] = c * c * txx - 2.0 * c * s * txy + s * s * tyy;
  out[b + 1] = c * s * txx + (c * c - s * s) * txy - c * s * tyy;
  out[b + 2] = c * txz - s * tyz;
  out[b + 3] = s * s * txx + 2.0 * c * s * txy + c * c * tyy;
  out[b + 4] = s * txz + c * tyz;
  out[b + 5] = tzz;
}

/* Interpolation weights of the cartoon planes (Sec. II.B.2): for x_j and the
   plane m dy (dy = dx), the nine Lagrange weights on x_{j-4..j+4} at
   varpi = sqrt(x_j^2 + (m dy)^2) and cos, sin of the azimuth phi of the point;
   level independent, computed once for j in [1, jmax]. */
typedef struct { double w[9], cs, sn; } cartoon_coef;

static cartoon_coef *cartoon_table(int jmax) {
  cartoon_coef *t = (cartoon_coef *)calloc((size_t)(jmax + 1) * 3, sizeof(cartoon_coef));
  double nodes[9];
  for (int n = 0; n < 9; ++n) nodes[n] = n - 4;
  for (int j = 1; j <= jmax; ++j)
    for (int m = 1; m <= 3; ++m) {
      cartoon_coef *e = &t[j * 3 + (m - 1)];
      double x = j - 0.5, y = m;
      double vp = sqrt(x * x + y * y);
      orc_lagrange(9, nodes, vp - x, e->w);
      e->cs = x / vp;
      e->sn = y / vp;
    }
  return t;
}

/* Values of the metric fields on the planes y = +m dy and y = -m dy at
   (x_j, z_k), m in 1..3: Lagrange interpolation with x_{j-4..j+4} at varpi
   (the same for both planes), rotated by +phi and -phi.  For j <= 0 the
   values are the rotation by pi of the points (x_{1-j}, -+m dy). */
static void cartoon_planes(const orc_ctx *c, int l, double **U, const cartoon_coef *tab, int j, int k, int m,
                           double plus[O_NMET], double minus[O_NMET], const int *need) {
  const orc_level *L = &c->lv[l];
  if (j <= 0) {
    cartoon_planes(c, l, U, tab, 1 - j, k, m, minus, plus, need);
    for (int f = 0; f < O_NMET; ++f) {
      plus[f] *= orc_field_parity_x(f);
      minus[f] *= orc_field_parity_x(f);
    }
    return;
  }
  const cartoon_coef *e = &tab[j * 3 + (m - 1)];
  double base[O_NMET];
  for (int f = 0; f < O_NMET; ++f) {
    base[f] = 0.0;
    if (need && !need[f]) continue;
    /* sum_n w_n Q_n written as Q_j + sum_n w_n (Q_n - Q_j) (the weights sum to 1) */
    double q0 = U[f][oidx(L, j, k)], s = 0.0;
    for (int n = 0; n < 9; ++n) s += e->w[n] * (U[f][oidx(L, j - 4 + n, k)] - q0);
    base[f] = q0 + s;
  }
  for (int sgn = 0; sgn < 2; ++sgn) {
    double *out = sgn == 0 ? plus : minus;
    double sn = sgn == 0 ? e->sn : -e->sn;
    out[O_W] = base[O_W]; out[O_KH] = base[O_KH]; out[O_TH] = base[O_TH]; out[O_AL] = base[O_AL];
    rotate_vec(e->cs, sn, base, out, O_GX, O_GY, O_GZ);
    rotate_vec(e->cs, sn, base, out, O_BX, O_BY, O_BZ);
    rotate_vec(e->cs, sn, base, out, O_BBX, O_BBY, O_BBZ);
    rotate_ten(e->cs, sn, base, out, O_HXX);
    rotate_ten(e->cs, sn, base, out, O_AXX);
  }
}

/* d_y Q and d_yy Q from the planes by 6th-order central differences (dy = dx),
   on j in [-2, nx+4], k in [-2, nz+7]; entries outside stay zero. */
void orc_cartoon_dy(const orc_ctx *c, int l, double **U, double **dy, double **dyy) {
  orc_cartoon_dy_mask(c, l, U, dy, dyy, NULL);
}

/* as orc_cartoon_dy, for the fields with need[f] != 0 only (need = NULL: all);
   the op counter uses it to count the planes the right-hand side needs */
void orc_cartoon_dy_mask(const orc_ctx *c, int l, double **U, double **dy, double **dyy, const int *need) {
  const orc_level *L = &c->lv[l];
  size_t n = (size_t)L->px * L->pz;
  for (int f = 0; f < O_NMET; ++f) { memset(dy[f], 0, n * sizeof(double)); memset(dyy[f], 0, n * sizeof(double)); }
  cartoon_coef *tab = cartoon_table(L->nx + 4);
#pragma omp parallel for schedule(static)
  for (int k = -2; k <= L->nz + 7; ++k)
    for (int j = -2; j <= L->nx + 4; ++j) {
      double pl[7][O_NMET];
      int id = oidx(L, j, k);
      for (int f = 0; f < O_NMET; ++f) pl[3][f] = U[f][id];
      for (int m = 1; m <= 3; ++m) cartoon_planes(c, l, U, tab, j, k, m, pl[3 + m], pl[3 - m], need);
      for (int f = 0; f < O_NMET; ++f) {
        if (need && !need[f]) continue;
        /* difference form: the weights of a derivative sum to zero */
        double s1 = 0.0, s2 = 0.0;
        for (int m = 0; m < 7; ++m) {
          s1 += orc_c1[m] * (pl[m][f] - pl[3][f]);
          s2 += orc_c2[m] * (pl[m][f] - pl[3][f]);
        }
        dy[f][id] = y_zero(f) ? 0.0 : s1 / L->dx;
        dyy[f][id] = s2 / (L->dx * L->dx);
      }
    }
  free(tab);
}

/* ---------------- derivatives at one cell ---------------- */

/* Eq. cartoon_bnd: d_xy of x/y vector and tensor components from d_x, for
   cells beyond the level edge where the planes are not available. */
static void cartoon_edge_xy(const double Q[O_NMET], const double dQ[O_NMET][3], double x, double ddQ[O_NMET][6]) {
  const int vx[3] = {O_GX, O_BX, O_BBX};
  for (int v = 0; v < 3; ++v) {
    int fx = vx[v], fy = vx[v] + 1;
    ddQ[fx][1] = Q[fy] / (x * x) - dQ[fy][0] / x;
    ddQ[fy][1] = -Q[fx] / (x * x) + dQ[fx][0] / x;
  }
  const int tb[2] = {O_HXX, O_AXX};
  for (int t = 0; t < 2; ++t) {
    int b = tb[t];
    int xx = b, xy = b + 1, xz = b + 2, yy = b + 3, yz = b + 4;
    ddQ[xz][1] = Q[yz] / (x * x) - dQ[yz][0] / x;
    ddQ[yz][1] = -Q[xz] / (x * x) + dQ[xz][0] / x;
    ddQ[xx][1] = 2.0 * (Q[xy] / (x * x) - dQ[xy][0] / x);
    ddQ[yy][1] = -2.0 * (Q[xy] / (x * x) - dQ[xy][0] / x);
    /* tensor yy - xx: the flat part of gt cancels, so h may be used directly */
    ddQ[xy][1] = (Q[yy] - Q[xx]) / (x * x) + (dQ[xx][0] - dQ[yy][0]) / x;
  }
}

/* All first (central), second derivatives and the advection term beta^k d_k Q
   of every metric field at cell (j,k).  dy/dyy: from orc_cartoon_dy (NULL in
   planar geometry, where d_y = 0). */
void orc_derivs_cell(const orc_ctx *c, int l, double **U, double **dy, double **dyy, int j, int k,
                     double Q[O_NMET], double dQ[O_NMET][3], double ddQ[O_NMET][6], double adv[O_NMET]) {
  orc_derivs_cell_mask(c, l, U, dy, dyy, j, k, NULL, NULL, Q, dQ, ddQ, adv);
}

/* as orc_derivs_cell, computing first derivatives only where need1[f] and
   second derivatives only where need2[f] (NULL: all; others left zero); the
   op counter uses it to count the derivatives the right-hand side needs */
void orc_derivs_cell_mask(const orc_ctx *c, int l, double **U, double **dy, double **dyy, int j, int k,
                          const int *need1, const int *need2, double Q[O_NMET], double dQ[O_NMET][3],
                          double ddQ[O_NMET][6], double adv[O_NMET]) {
  const orc_level *L = &c->lv[l];
  double dx = L->dx, dz = L->dz;
  int id = oidx(L, j, k);
  for (int f = 0; f < O_NMET; ++f) {
    const double *u = U[f];
    double u0 = u[id];
    Q[f] = u0;
    for (int a = 0; a < 3; ++a) dQ[f][a] = 0.0;
    for (int a = 0; a < 6; ++a) ddQ[f][a] = 0.0;
    int n1 = !need1 || need1[f], n2 = !need2 || need2[f];
    /* all stencils in difference form sum_n c_n (u_n - u_0): exact zero on constants */
    if (n1) {
      double sx = 0, sz = 0;
      for (int n = -3; n <= 3; ++n) {
        sx += orc_c1[n + 3] * (u[oidx(L, j + n, k)] - u0);
        sz += orc_c1[n + 3] * (u[oidx(L, j, k + n)] - u0);
      }
      dQ[f][0] = sx / dx;
      dQ[f][2] = sz / dz;
    }
    if (n2) {
      double sxx = 0, szz = 0, sxz = 0;
      for (int n = -3; n <= 3; ++n) {
        sxx += orc_c2[n + 3] * (u[oidx(L, j + n, k)] - u0);
        szz += orc_c2[n + 3] * (u[oidx(L, j, k + n)] - u0);
        for (int m = -3; m <= 3; ++m) sxz += orc_c1[n + 3] * orc_c1[m + 3] * (u[oidx(L, j + n, k + m)] - u0);
      }
      ddQ[f][0] = sxx / (dx * dx);
      ddQ[f][5] = szz / (dz * dz);
      ddQ[f][2] = sxz / (dx * dz);
    }
    if (dy) {
      dQ[f][1] = dy[f][id];
      if (n2) {
        ddQ[f][3] = dyy[f][id];
        double sxy = 0, syz = 0, d0 = dy[f][id];
        if (!y_zero(f))
          for (int n = -3; n <= 3; ++n) {
            sxy += orc_c1[n + 3] * (dy[f][oidx(L, j + n, k)] - d0);
            syz += orc_c1[n + 3] * (dy[f][oidx(L, j, k + n)] - d0);
          }
        ddQ[f][1] = y_zero(f) ? 0.0 : sxy / dx;
        ddQ[f][4] = y_zero(f) ? 0.0 : syz / dz;
      }
    }
  }
  if (dy && j > L->nx) {
    /* the edge formula needs d_x of the tensor/vector components */
    double ddQe[O_NMET][6];
    memcpy(ddQe, ddQ, sizeof(ddQe));
    cartoon_edge_xy(Q, dQ, (j - 0.5) * dx, ddQe);
    for (int f = 0; f < O_NMET; ++f)
      if (!need2 || need2[f]) ddQ[f][1] = ddQe[f][1];
  }

  /* advection: 6th-order lopsided in x and z, upwind with the sign of beta;
     central (from the planes) in y */
  double bx = Q[O_BX], by = Q[O_BY], bz = Q[O_BZ];
  for (int f = 0; f < O_NMET; ++f) {
    const double *u = U[f];
    double u0 = u[id];
    double ax = 0.0, az = 0.0;
    if (bx > 0.0) { for (int n = -2; n <= 4; ++n) ax += orc_lop[n + 2] * (u[oidx(L, j + n, k)] - u0); ax /= dx; }
    else if (bx < 0.0) { for (int n = -2; n <= 4; ++n) ax -= orc_lop[n + 2] * (u[oidx(L, j - n, k)] - u0); ax /= dx; }
    if (bz > 0.0) { for (int n = -2; n <= 4; ++n) az += orc_lop[n + 2] * (u[oidx(L, j, k + n)] - u0); az /= dz; }
    else if (bz < 0.0) { for (int n = -2; n <= 4; ++n) az -= orc_lop[n + 2] * (u[oidx(L, j, k - n)] - u0); az /= dz; }
    adv[f] = bx * ax + bz * az + by * dQ[f][1];
  }
}

/* 8th-order Kreiss-Oliger term -(eps/256)(dx^7 D^8_x + dz^7 D^8_z) Q (sign and
   power chosen so that it dissipates; Sec. II.B.1). */
void orc_ko_cell(const orc_ctx *c, int l, double **U, int j, int k, double ko[O_NMET]) {
  const orc_level *L = &c->lv[l];
  for (int f = 0; f < O_NMET; ++f) {
    double sx = 0.0, sz = 0.0, u0 = U[f][oidx(L, j, k)];
    for (int n = -4; n <= 4; ++n) {
      sx += orc_ko[n + 4] * (U[f][oidx(L, j + n, k)] - u0);
      sz += orc_ko[n + 4] * (U[f][oidx(L, j, k + n)] - u0);
    }
    ko[f] = -(c->p.eps_ko / 256.0) * (sx / L->dx + sz / L->dz);
  }
}

/* ---------------- matter terms ---------------- */

/* E = rho h w^2 - P, S_i = rho h w u_i, S_ij = rho h u_i u_j + P gamma_ij */
void orc_matter_point(const orc_params *p, const double pr[O_NPRIM], double W, const double h[6],
                      double *E, double Si[3], double Sij[6]) {
  (void)p;
  double g[6] = {1.0 + h[0], h[1], h[2], 1.0 + h[3], h[4], 1.0 + h[5]}, gi[6];
  orc_inv3(g, gi, 0);
  double u[3] = {pr[O_UX], pr[O_UY], pr[O_UZ]};
  double uu = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) uu += gi[S6[a][b]] * u[a] * u[b];
  double w = sqrt(1.0 + W * W * uu);
  double rho = pr[O_RHO], P = pr[O_P];
  double rh = rho * (1.0 + pr[O_EPS] + P / rho);
  *E = rh * w * w - P;
  for (int a = 0; a < 3; ++a) Si[a] = rh * w * u[a];
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b) Sij[S6[a][b]] = rh * u[a] * u[b] + P * g[S6[a][b]] / (W * W);
}

/* ---------------- geometry helpers ---------------- */

typedef struct {
  double W, al, Kh, Th;
  double g[3][3], gi[3][3], A[3][3];
  double dg[3][3][3];          /* d_k gt_ij  -> dg[k][i][j] */
  double ddg[3][3][3][3];      /* d_k d_l gt_ij -> ddg[k][l][i][j] */
  double Gl[3][3][3];          /* Gt_{k,ij} */
  double G2[3][3][3];          /* Gt^k_ij */
  double Gd[3];                /* gt^jk Gt^i_jk */
  double dW[3], ddW[3][3], dal[3], ddal[3][3];
  double R[3][3];              /* physical Ricci tensor */
  double Rs;                   /* physical Ricci scalar */
} geom;

static void geom_fill(const double Q[O_NMET], const double dQ[O_NMET][3], const double ddQ[O_NMET][6], geom *G) {
  G->W = Q[O_W]; G->al = Q[O_AL]; G->Kh = Q[O_KH]; G->Th = Q[O_TH];
  double gs[6], gis[6];
  for (int a = 0; a < 6; ++a) gs[a] = Q[O_HXX + a];
  gs[0] += 1.0; gs[3] += 1.0; gs[5] += 1.0;
  orc_inv3(gs, gis, 0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      G->g[i][j] = gs[S6[i][j]];
      G->gi[i][j] = gis[S6[i][j]];
      G->A[i][j] = Q[O_AXX + S6[i][j]];
      for (int k = 0; k < 3; ++k) {
        G->dg[k][i][j] = dQ[O_HXX + S6[i][j]][k];
        for (int l = 0; l < 3; ++l) G->ddg[k][l][i][j] = ddQ[O_HXX + S6[i][j]][S6[k][l]];
      }
    }
  for (int k = 0; k < 3; ++k) {
    G->dW[k] = dQ[O_W][k];
    G->dal[k] = dQ[O_AL][k];
    for (int l = 0; l < 3; ++l) { G->ddW[k][l] = ddQ[O_W][S6[k][l]]; G->ddal[k][l] = ddQ[O_AL][S6[k][l]]; }
  }
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        G->Gl[k][i][j] = 0.5 * (G->dg[i][k][j] + G->dg[j][k][i] - G->dg[k][i][j]);
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int l = 0; l < 3; ++l) s += G->gi[k][l] * G->Gl[l][i][j];
        G->G2[k][i][j] = s;
      }
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) s += G->gi[j][k] * G->G2[i][j][k];
    G->Gd[i] = s;
  }
}

/* Ricci tensor of gamma_ij = gt_ij / W^2 split as Rt_ij + R^W_ij (the
   conformal decomposition used with Eq. bssn); the d_j Gt^k term uses the
   evolved Gt^k, the quadratic term the computed Gt_d^k. */
static void geom_ricci(const double dQ[O_NMET][3], geom *G) {
  double dGt[3][3];  /* dGt[j][k] = d_j Gt^k */
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 3; ++k) dGt[j][k] = dQ[O_GX + k][j];
  double DDW[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = G->ddW[i][j];
      for (int k = 0; k < 3; ++k) s -= G->G2[k][i][j] * G->dW[k];
      DDW[i][j] = s;
    }
  double trDDW = 0.0, dW2 = 0.0;
  for (int l = 0; l < 3; ++l)
    for (int m = 0; m < 3; ++m) { trDDW += G->gi[l][m] * DDW[l][m]; dW2 += G->gi[l][m] * G->dW[l] * G->dW[m]; }
  double W = G->W;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double r = 0.0;
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) r += -0.5 * G->gi[l][m] * G->ddg[l][m][i][j];
      for (int k = 0; k < 3; ++k) r += 0.5 * (G->g[k][i] * dGt[j][k] + G->g[k][j] * dGt[i][k]);
      for (int k = 0; k < 3; ++k) r += 0.5 * G->Gd[k] * (G->Gl[i][j][k] + G->Gl[j][i][k]);
      for (int l = 0; l < 3; ++l)
        for (int m = 0; m < 3; ++m) {
          double s = 0.0;
          for (int k = 0; k < 3; ++k)
            s += G->G2[k][l][i] * G->Gl[j][k][m] + G->G2[k][l][j] * G->Gl[i][k][m] + G->G2[k][i][m] * G->Gl[k][l][j];
          r += G->gi[l][m] * s;
        }
      double rw = (DDW[i][j] + G->g[i][j] * trDDW) / W - 2.0 * G->g[i][j] * dW2 / (W * W);
      G->R[i][j] = r + rw;
    }
  double rs = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) rs += G->gi[i][j] * G->R[i][j];
  G->Rs = W * W * rs;
}

void orc_ricci_point(const double Q[O_NMET], const double dQ[O_NMET][3], const double ddQ[O_NMET][6], double Rij[6]) {
  geom G;
  geom_fill(Q, dQ, ddQ, &G);
  geom_ricci(dQ, &G);
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) Rij[S6[i][j]] = G.R[i][j];
}

/* ---------------- Z4c right-hand side, Eq. bssn + Eq. moving_puncture ---------------- */

void orc_z4c_point(const orc_params *p, const double Q[O_NMET], const double dQ[O_NMET][3],
                   const double ddQ[O_NMET][6], const double adv[O_NMET], double E,
                   const double Si[3], const double Sij6[6], double fz, double rhs[O_NMET]) {
  geom G;
  geom_fill(Q, dQ, ddQ, &G);
  geom_ricci(dQ, &G);
  const double PI = 3.14159265358979323846;
  double W = G.W, al = G.al, Kh = G.Kh, Th = G.Th;
  double K = Kh + 2.0 * Th;
  double kap = p->bssn ? 0.0 : p->kappa * fz;   /* Z4 damping radius factor exp(-r^2/r_Z4^2) on kappa; none in BSSN */

  double beta[3] = {Q[O_BX], Q[O_BY], Q[O_BZ]};
  double Bv[3] = {Q[O_BBX], Q[O_BBY], Q[O_BBZ]};
  double Gt[3] = {Q[O_GX], Q[O_GY], Q[O_GZ]};
  double db[3][3], ddb[3][3][3];  /* db[k][i] = d_k beta^i, ddb[k][l][i] */
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) {
      db[k][i] = dQ[O_BX + i][k];
      for (int l = 0; l < 3; ++l) ddb[k][l][i] = ddQ[O_BX + i][S6[k][l]];
    }
  (void)beta;
  double dKh[3], dTh[3];
  for (int k = 0; k < 3; ++k) { dKh[k] = dQ[O_KH][k]; dTh[k] = dQ[O_TH][k]; }
  double Sij[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Sij[i][j] = Sij6[S6[i][j]];

  /* D_i D_j alpha of the physical metric */
  double DDa[3][3];
  double daW = 0.0;
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) daW += G.gi[k][l] * G.dal[k] * G.dW[l];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = G.ddal[i][j];
      for (int k = 0; k < 3; ++k) s -= G.G2[k][i][j] * G.dal[k];
      s += (G.dal[i] * G.dW[j] + G.dal[j] * G.dW[i] - G.g[i][j] * daW) / W;
      DDa[i][j] = s;
    }
  double D2a = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) D2a += G.gi[i][j] * DDa[i][j];
  D2a *= W * W;

  double Aup[3][3], AA = 0.0, AikAkj[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) s += G.gi[i][a] * G.gi[j][b] * G.A[a][b];
      Aup[i][j] = s;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      AA += G.A[i][j] * Aup[i][j];
      double s = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) s += G.A[i][k] * G.gi[k][l] * G.A[l][j];
      AikAkj[i][j] = s;
    }
  double divb = db[0][0] + db[1][1] + db[2][2];
  double Str = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Str += G.gi[i][j] * Sij[i][j];
  Str *= W * W;

  /* W */
  rhs[O_W] = adv[O_W] + W / 3.0 * (al * K - divb);
  /* gt_ij (evolved as h_ij) */
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      double s = -2.0 * al * G.A[i][j] - 2.0 / 3.0 * G.g[i][j] * divb;
      for (int k = 0; k < 3; ++k) s += G.g[i][k] * db[j][k] + G.g[j][k] * db[i][k];
      rhs[O_HXX + S6[i][j]] = adv[O_HXX + S6[i][j]] + s;
    }
  /* At_ij */
  double X[3][3], trX = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) X[i][j] = al * G.R[i][j] - DDa[i][j] - 8.0 * PI * al * Sij[i][j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) trX += G.gi[i][j] * X[i][j];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      double s = W * W * (X[i][j] - G.g[i][j] * trX / 3.0);
      s += al * (K * G.A[i][j] - 2.0 * AikAkj[i][j]);
      for (int k = 0; k < 3; ++k) s += G.A[k][j] * db[i][k] + G.A[k][i] * db[j][k];
      s -= 2.0 / 3.0 * G.A[i][j] * divb;
      rhs[O_AXX + S6[i][j]] = adv[O_AXX + S6[i][j]] + s;
    }
  /* Khat, Eq. K */
  rhs[O_KH] = adv[O_KH] - D2a + al * (AA + K * K / 3.0) + 4.0 * PI * al * (Str + E) + al * kap * Th;
  /* Gt^i */
  double gsrc[3];
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j) s -= 2.0 * Aup[i][j] * G.dal[j];
    double inner = 0.0;
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) inner += G.G2[i][j][k] * Aup[j][k];
    for (int j = 0; j < 3; ++j) {
      inner -= G.gi[i][j] * (2.0 * dKh[j] + dTh[j]) / 3.0;
      inner -= 3.0 / W * Aup[i][j] * G.dW[j];
      inner -= 8.0 * PI * G.gi[i][j] * Si[j];
    }
    s += 2.0 * al * inner;
    s += 2.0 / 3.0 * G.Gd[i] * divb;
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) s += G.gi[j][k] * ddb[j][k][i];
    for (int j = 0; j < 3; ++j) {
      double dd = 0.0;
      for (int k = 0; k < 3; ++k) dd += ddb[j][k][k];
      s += G.gi[i][j] * dd / 3.0;
    }
    for (int j = 0; j < 3; ++j) s -= G.Gd[j] * db[j][i];
    s -= 2.0 * al * kap * (Gt[i] - G.Gd[i]);
    gsrc[i] = s;
    rhs[O_GX + i] = adv[O_GX + i] + s;
  }
  /* Theta (held at zero in BSSN) */
  rhs[O_TH] = p->bssn ? 0.0
                      : adv[O_TH] + fz * (0.5 * al * (G.Rs - AA + 2.0 / 3.0 * K * K) - 8.0 * PI * al * E)
                            - 2.0 * al * kap * Th;
  /* gauge: 1+log with Khat, Gamma-driver */
  rhs[O_AL] = adv[O_AL] - 2.0 * al * Kh;
  for (int i = 0; i < 3; ++i) {
    rhs[O_BX + i] = adv[O_BX + i] + 0.75 * Bv[i];
    rhs[O_BBX + i] = adv[O_BBX + i] + gsrc[i] - p->eta_B * Bv[i];
  }
}

/* Hamiltonian and momentum constraints (Sec. II.F.1):
   H = R + K^2 - K_ij K^ij - 16 pi E,
   M_i = D_j K^j_i - D_i K - 8 pi S_i, written with the conformal variables:
   M_i = d_j At^j_i - Gt^l_ji At^j_l - (3/W) At^l_i d_l W - (2/3) d_i K - 8 pi S_i. */
void orc_constraints_point(const double Q[O_NMET], const double dQ[O_NMET][3], const double ddQ[O_NMET][6],
                           double E, const double Si[3], double *H, double M[3]) {
  geom G;
  geom_fill(Q, dQ, ddQ, &G);
  geom_ricci(dQ, &G);
  const double PI = 3.14159265358979323846;
  double K = G.Kh + 2.0 * G.Th;
  double Aup[3][3], AA = 0.0, trA = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) s += G.gi[i][a] * G.gi[j][b] * G.A[a][b];
      Aup[i][j] = s;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) { AA += G.A[i][j] * Aup[i][j]; trA += G.gi[i][j] * G.A[i][j]; }
  double KK = AA + 2.0 / 3.0 * K * trA + K * K / 3.0;
  *H = G.Rs + K * K - KK - 16.0 * PI * E;

  double dA[3][3][3];  /* dA[k][i][j] = d_k At_ij */
  double dgi[3][3][3]; /* d_k gt^ij */
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        dA[k][i][j] = dQ[O_AXX + S6[i][j]][k];
        double s = 0.0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) s -= G.gi[i][a] * G.gi[j][b] * G.dg[k][a][b];
        dgi[k][i][j] = s;
      }
  double Amix[3][3];  /* At^j_i = gt^jk At_ki -> Amix[j][i] */
  for (int j = 0; j < 3; ++j)
    for (int i = 0; i < 3; ++i) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += G.gi[j][k] * G.A[k][i];
      Amix[j][i] = s;
    }
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) s += dgi[j][j][k] * G.A[k][i] + G.gi[j][k] * dA[j][k][i];
    for (int j = 0; j < 3; ++j)
      for (int l = 0; l < 3; ++l) s -= G.G2[l][j][i] * Amix[j][l];
    for (int l = 0; l < 3; ++l) s -= 3.0 / G.W * Amix[l][i] * G.dW[l];
    s -= 2.0 / 3.0 * (dQ[O_KH][i] + 2.0 * dQ[O_TH][i]);
    s -= 8.0 * PI * Si[i];
    M[i] = s;
  }
}
