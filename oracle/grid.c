/*
 * Oracle (test infrastructure only): the FMR level hierarchy of Sec. II.A,
 * ghost fill (axis/equator parity, outer boundary of Sec. II.B.3, buffer
 * prolongation of Sec. II.D), the finite-volume hydro update of Sec. II.C.1,
 * the RK stage, restriction and reflux (Sec. II.D) and the diagnostics of
 * Sec. II.F.1 of Lam & Shibata (arXiv:2502.03223).  Plain loops, FP64.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "orc.h"


static const double PI = 3.14159265358979323846;

static double *alloc_arr(size_t n) { return (double *)calloc(n, sizeof(double)); }

orc_ctx *orc_create(const orc_params *p) {
  orc_stencil_init();
  if (p->n_levels < 1 || p->n_levels > ORC_MAXL) return NULL;
  if (p->n_levels > 1 && (p->nx != p->nz || p->nx % 2 != 0 || p->nx < 16 || p->geometry != 1)) return NULL;
  orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
  c->p = *p;
  for (int l = 0; l < p->n_levels; ++l) {
    orc_level *L = &c->lv[l];
    L->nx = p->nx; L->nz = p->nz;
    L->px = p->nx + 2 * ORC_G; L->pz = p->nz + 2 * ORC_G;
    L->dx = p->dx0 / (double)(1 << l);
    L->dz = p->dz0 / (double)(1 << l);
    size_t n = (size_t)L->px * L->pz;
    for (int f = 0; f < O_NSTATE; ++f) {
      L->un[f] = alloc_arr(n); L->us[f] = alloc_arr(n); L->ka[f] = alloc_arr(n); L->rhs[f] = alloc_arr(n);
    }
    for (int f = 0; f < O_NPRIM; ++f) L->prim[f] = alloc_arr(n);
    L->status = (unsigned char *)calloc(n, 1);
    for (int f = 0; f < O_NCONS; ++f) {
      L->fx[f] = alloc_arr(n); L->fz[f] = alloc_arr(n);
      for (int r = 0; r < 4; ++r) L->freg[r][f] = alloc_arr((size_t)(p->nx > p->nz ? p->nx : p->nz) + 2);
    }
    for (int f = 0; f < O_NSTATE; ++f) L->uold[f] = alloc_arr(n);
    for (int f = 0; f < O_NMET; ++f) L->ut[f] = alloc_arr(n);
    for (int f = 0; f < O_NPRIM; ++f) { L->pold[f] = alloc_arr(n); L->pnow[f] = alloc_arr(n); L->pt[f] = alloc_arr(n); }
    L->wpar = 1.0;
  }
  return c;
}

void orc_destroy(orc_ctx *c) {
  if (!c) return;
  for (int l = 0; l < c->p.n_levels; ++l) {
    orc_level *L = &c->lv[l];
    for (int f = 0; f < O_NSTATE; ++f) { free(L->un[f]); free(L->us[f]); free(L->ka[f]); free(L->rhs[f]); }
    for (int f = 0; f < O_NPRIM; ++f) free(L->prim[f]);
    free(L->status);
    for (int f = 0; f < O_NCONS; ++f) {
      free(L->fx[f]); free(L->fz[f]);
      for (int r = 0; r < 4; ++r) free(L->freg[r][f]);
    }
    for (int f = 0; f < O_NSTATE; ++f) free(L->uold[f]);
    for (int f = 0; f < O_NMET; ++f) free(L->ut[f]);
    for (int f = 0; f < O_NPRIM; ++f) { free(L->pold[f]); free(L->pnow[f]); free(L->pt[f]); }
  }
  free(c);
}

static double **stage_state(orc_ctx *c, int l, int s) { return s == 0 ? c->lv[l].un : c->lv[l].us; }

static int n_stages(const orc_params *p) { return p->rk == 0 ? 4 : 3; }

/* stage time fractions c_s and the weights b_s of the final combination */
static double stage_c(const orc_params *p, int s) {
  static const double c4[4] = {0.0, 0.5, 0.5, 1.0}, c3[3] = {0.0, 1.0, 0.5};
  return p->rk == 0 ? c4[s] : c3[s];
}
static double stage_b(const orc_params *p, int s) {
  static const double b4[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0}, b3[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
  return p->rk == 0 ? b4[s] : b3[s];
}

static double xc(const orc_level *L, int j) { return (j - 0.5) * L->dx; }
static double zc(const orc_level *L, int k) { return (k - 0.5) * L->dz; }

static void cell_h(double **U, int id, double h[6]) {
  for (int a = 0; a < 6; ++a) h[a] = U[O_HXX + a][id];
}

/* update region [1, jmax] x [1, kmax] of a level at stage s (Sec. II.D:
   [1, N+4] in all but the last stage on refined levels, [1, N] otherwise) */
static void region(const orc_ctx *c, int l, int s, int *jmax, int *kmax) {
  const orc_level *L = &c->lv[l];
  int ext = (l > 0 && s < n_stages(&c->p) - 1) ? 4 : 0;
  *jmax = L->nx + ext;
  *kmax = L->nz + ext;
}

/* ---------------- ghost fill ---------------- */

static void parity_fill(orc_ctx *c, int l, double **U) {
  orc_level *L = &c->lv[l];
  for (int k = 1; k <= L->nz + ORC_G; ++k)
    for (int j = 1 - ORC_G; j <= 0; ++j) {
      int d = oidx(L, j, k), s = oidx(L, 1 - j, k);
      for (int f = 0; f < O_NMET; ++f) U[f][d] = orc_field_parity_x(f) * U[f][s];
      for (int f = 0; f < O_NPRIM; ++f) L->prim[f][d] = orc_prim_parity_x(f) * L->prim[f][s];
    }
  for (int k = 1 - ORC_G; k <= 0; ++k)
    for (int j = 1 - ORC_G; j <= L->nx + ORC_G; ++j) {
      int d = oidx(L, j, k), s = oidx(L, j, 1 - k);
      for (int f = 0; f < O_NMET; ++f) U[f][d] = orc_field_parity_z(f) * U[f][s];
      for (int f = 0; f < O_NPRIM; ++f) L->prim[f][d] = orc_prim_parity_z(f) * L->prim[f][s];
    }
}

static void outflow_fill(orc_ctx *c, int l, double **U) {
  orc_level *L = &c->lv[l];
  for (int k = 1 - ORC_G; k <= L->nz + ORC_G; ++k)
    for (int j = 1 - ORC_G; j <= L->nx + ORC_G; ++j) {
      if (j >= 1 && j <= L->nx && k >= 1 && k <= L->nz) continue;
      int jj = j < 1 ? 1 : (j > L->nx ? L->nx : j);
      int kk = k < 1 ? 1 : (k > L->nz ? L->nz : k);
      int d = oidx(L, j, k), s = oidx(L, jj, kk);
      for (int f = 0; f < O_NSTATE; ++f) U[f][d] = U[f][s];
      for (int f = 0; f < O_NPRIM; ++f) L->prim[f][d] = L->prim[f][s];
    }
}

/* Outer boundary of the coarsest level (Sec. II.B.3):
   Q(r) = Q_inf + (1 - tau/r) (Q^n - Q_inf)(r - tau), tau = c_s dt, with a
   2nd-order (3x3) Lagrange interpolation of the step-start state Q^n; the
   hydro primitives are copied from the nearest interior cell.  A frozen
   metric (Cowling runs) keeps its ghosts as given; hydro_outer = 1 keeps the
   hydro ghosts at the initial data (a known inflow solution). */
static void outer_fill(orc_ctx *c, double **U, double tau) {
  orc_level *L = &c->lv[0];
  double **Un = L->un;
  double n3[3] = {-1, 0, 1};
  for (int k = 1; k <= L->nz + ORC_G; ++k)
    for (int j = 1; j <= L->nx + ORC_G; ++j) {
      if (j <= L->nx && k <= L->nz) continue;
      int d = oidx(L, j, k);
      double x = xc(L, j), z = zc(L, k), r = sqrt(x * x + z * z);
      double fac = 1.0 - tau / r;
      double xs = x * fac, zs = z * fac;
      double xi = xs / L->dx + 0.5, ze = zs / L->dz + 0.5;
      int i0 = (int)floor(xi + 0.5), k0 = (int)floor(ze + 0.5);
      if (i0 > L->nx + ORC_G - 1) i0 = L->nx + ORC_G - 1;
      if (k0 > L->nz + ORC_G - 1) k0 = L->nz + ORC_G - 1;
      double wx[3], wz[3];
      orc_lagrange(3, n3, xi - i0, wx);
      orc_lagrange(3, n3, ze - k0, wz);
      for (int f = 0; f < (c->p.evolve_spacetime ? O_NMET : 0); ++f) {
        double qinf = (f == O_W || f == O_AL) ? 1.0 : 0.0;
        /* interpolation in difference form about the central node (weights sum to 1) */
        double q0 = Un[f][oidx(L, i0, k0)] - qinf, s = 0.0;
        for (int b = 0; b < 3; ++b)
          for (int a = 0; a < 3; ++a) s += wx[a] * wz[b] * (Un[f][oidx(L, i0 - 1 + a, k0 - 1 + b)] - qinf - q0);
        U[f][d] = qinf + fac * (q0 + s);
      }
      if (c->p.hydro_outer) continue;
      int jj = j > L->nx ? L->nx : j, kk = k > L->nz ? L->nz : k;
      int s = oidx(L, jj, kk);
      for (int f = 0; f < O_NPRIM; ++f) L->prim[f][d] = L->prim[f][s];
    }
}

static double minmod(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  return fabs(a) < fabs(b) ? a : b;
}

/* parent cell and offset (in parent cells) of child index j: child centre
   sits a quarter parent cell left (odd j) or right (even j) of parent m */
static void child_to_parent(int j, int *m, double *off) {
  if (j % 2 == 0) { *m = j / 2; *off = 0.25; }
  else { *m = (j + 1) / 2; *off = -0.25; }
}

/* 8th-order Lagrange weights over 8 parent cells for a child index: cells m-3..m+4 (offset +1/4) or m-4..m+3 (-1/4) */
static void prol_weights(int j, int *base, double w[8]) {
  int m; double off;
  child_to_parent(j, &m, &off);
  double nodes[8];
  if (off > 0) { *base = m - 3; for (int n = 0; n < 8; ++n) nodes[n] = n - 3; }
  else { *base = m - 4; for (int n = 0; n < 8; ++n) nodes[n] = n - 4; }
  orc_lagrange(8, nodes, off, w);
}

/* Prolongation into the buffer zone of level l (Sec. II.D): 8th-order
   Lagrange for the metric, minmod-limited linear for the primitives, then
   conserved variables rebuilt from the primitives. full = refill [N+1, N+8]
   (start of the step), else only [N+5, N+8]. */
static void prolong_from(orc_ctx *c, int l, double **U, double **Up, double **Pprim, int full) {
  orc_level *L = &c->lv[l], *P = &c->lv[l - 1];
  int lo = full ? L->nx + 1 : L->nx + 5;
  for (int k = 1; k <= L->nz + ORC_G; ++k)
    for (int j = 1; j <= L->nx + ORC_G; ++j) {
      if (j < lo && k < lo) continue;
      int d = oidx(L, j, k);
      int bx, bz;
      double wx[8], wz[8];
      prol_weights(j, &bx, wx);
      prol_weights(k, &bz, wz);
      int mx0, mz0; double ox0, oz0;
      child_to_parent(j, &mx0, &ox0);
      child_to_parent(k, &mz0, &oz0);
      for (int f = 0; f < O_NMET; ++f) {
        double q0 = Up[f][oidx(P, mx0, mz0)], s = 0.0;
        for (int b = 0; b < 8; ++b)
          for (int a = 0; a < 8; ++a) s += wx[a] * wz[b] * (Up[f][oidx(P, bx + a, bz + b)] - q0);
        U[f][d] = q0 + s;
      }
      int mx, mz; double ox, oz;
      child_to_parent(j, &mx, &ox);
      child_to_parent(k, &mz, &oz);
      double pr[O_NPRIM];
      for (int f = 0; f < O_NPRIM; ++f) {
        double *a = Pprim[f];
        double a0 = a[oidx(P, mx, mz)];
        double sx = minmod(a[oidx(P, mx + 1, mz)] - a0, a0 - a[oidx(P, mx - 1, mz)]);
        double sz = minmod(a[oidx(P, mx, mz + 1)] - a0, a0 - a[oidx(P, mx, mz - 1)]);
        pr[f] = a0 + ox * sx + oz * sz;
      }
      double pc = orc_eos_pcold(&c->p, pr[O_RHO]);
      if (pr[O_P] < pc || c->p.eos_adiabatic) pr[O_P] = pc;
      pr[O_EPS] = orc_eos_eps(&c->p, pr[O_RHO], pr[O_P]);
      for (int f = 0; f < O_NPRIM; ++f) L->prim[f][d] = pr[f];
      double h[6], q[O_NCONS];
      cell_h(U, d, h);
      orc_prim2cons(&c->p, pr, U[O_W][d], h, xc(L, j), q);
      for (int f = 0; f < O_NCONS; ++f) U[O_NMET + f][d] = q[f];
    }
}

static void prolong_fill(orc_ctx *c, int l, double **U, double **Up, int full) {
  prolong_from(c, l, U, Up, c->lv[l - 1].prim, full);
}

/* Parent data of a sub-cycled level at time t^n + theta (t^{n+1} - t^n) of the
   parent's step (Sec. II.D): second-order Lagrange through the parent's time
   slices t^{n-1}, t^n, t^{n+1}; for the primitives first order through
   t^n, t^{n+1} where (p^{n+1} - p^n)(p^n - p^{n-1}) < 0; first order
   everywhere while no t^{n-1} slice exists yet. */
static void time_interp(orc_ctx *c, int lp, double theta) {
  orc_level *P = &c->lv[lp];
  size_t n = (size_t)P->px * P->pz;
  double wm = 0.5 * theta * (theta - 1.0), wp = 0.5 * theta * (theta + 1.0);   /* weights of t^{n-1}, t^{n+1} */
  /* after the parent's step: un holds t^{n+1}, us holds t^n */
  for (int f = 0; f < O_NMET; ++f)
    for (size_t i = 0; i < n; ++i) {
      double q0 = P->us[f][i], q1 = P->un[f][i];
      P->ut[f][i] = P->have_old ? q0 + wm * (P->uold[f][i] - q0) + wp * (q1 - q0) : q0 + theta * (q1 - q0);
    }
  for (int f = 0; f < O_NPRIM; ++f)
    for (size_t i = 0; i < n; ++i) {
      double q0 = P->pnow[f][i], q1 = P->prim[f][i];
      int quad = P->have_old && !((q1 - q0) * (q0 - P->pold[f][i]) < 0.0);
      P->pt[f][i] = quad ? q0 + wm * (P->pold[f][i] - q0) + wp * (q1 - q0) : q0 + theta * (q1 - q0);
    }
}

void orc_fill(orc_ctx *c, int s, double dt) {
  for (int l = 0; l < c->p.n_levels; ++l) {
    double **U = stage_state(c, l, s);
    if (c->p.geometry == 0) { outflow_fill(c, l, U); continue; }
    if (l == 0) outer_fill(c, U, stage_c(&c->p, s) * dt);
    else prolong_fill(c, l, U, stage_state(c, l - 1, s), s == 0);
    parity_fill(c, l, U);
  }
}

/* ---------------- hydro right-hand side, Sec. II.C.1-2 ---------------- */

static void face_metric(const orc_level *L, double **U, int j, int k, int dir, double *alpha, double beta[3],
                        double *W, double h[6]) {
  double v[O_NMET];
  for (int f = 0; f < O_NMET; ++f) {
    double q0 = U[f][oidx(L, j, k)], s = 0.0;
    for (int n = 0; n < 6; ++n) {
      int id = dir == 0 ? oidx(L, j - 2 + n, k) : oidx(L, j, k - 2 + n);
      s += orc_face6[n] * (U[f][id] - q0);
    }
    v[f] = q0 + s;
  }
  *alpha = v[O_AL];
  beta[0] = v[O_BX]; beta[1] = v[O_BY]; beta[2] = v[O_BZ];
  *W = v[O_W];
  for (int a = 0; a < 6; ++a) h[a] = v[O_HXX + a];
}

/* reconstructed (rho, u_x, u_y, u_z, P) at the face j+1/2 (dir 0) or k+1/2 (dir 1) */
static void face_prims(const orc_level *L, int j, int k, int dir, double pl[5], double prr[5]) {
  static const int pf[5] = {O_RHO, O_UX, O_UY, O_UZ, O_P};
  for (int v = 0; v < 5; ++v) {
    double a[6];
    for (int n = 0; n < 6; ++n) {
      int id = dir == 0 ? oidx(L, j - 2 + n, k) : oidx(L, j, k - 2 + n);
      a[n] = L->prim[pf[v]][id];
    }
    orc_ppm_face(a, &pl[v], &prr[v]);
  }
  /* first order on a side whose density or pressure came out non-positive */
  int cl = dir == 0 ? oidx(L, j, k) : oidx(L, j, k);
  int cr = dir == 0 ? oidx(L, j + 1, k) : oidx(L, j, k + 1);
  if (!(pl[0] > 0.0) || !(pl[4] > 0.0))
    for (int v = 0; v < 5; ++v) pl[v] = L->prim[pf[v]][cl];
  if (!(prr[0] > 0.0) || !(prr[4] > 0.0))
    for (int v = 0; v < 5; ++v) prr[v] = L->prim[pf[v]][cr];
}

/* Hydro sources at a cell centre (Sec. II.C.1), in the conformal variables:
   s_S_k = P d_k(alpha W^-3) - W^-3 rho h w^2 [d_k alpha - v_i d_k beta^i
           + (W^2/2) alpha v_a v_b d_k gt^ab + (alpha/W) v_i v^i d_k W]   (k = x, z)
   plus alpha W^-3 (S_y vbar^y + P)/x on s_Sx when x > 0 (cylindrical),
   s_E = W^-3 (alpha K^ij S_ij - rho h w^2 v^i d_i alpha), s_D = s_Sphi = 0.
   d*[e]: derivatives in e = 0 (x), 1 (z); dh[e][ij]; db[e][i] = d_e beta^i. */
void orc_hydro_source(const orc_params *p, const double pr[O_NPRIM], double al, double betay, double W,
                      const double h[6], const double A[6], double K, const double dal[2], const double db[2][3],
                      const double dW[2], const double dh[2][6], double x, double src[O_NCONS]) {
  (void)p;
  static const int S6[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  double g[6] = {1.0 + h[0], h[1], h[2], 1.0 + h[3], h[4], 1.0 + h[5]}, gi[6];
  orc_inv3(g, gi, 0);
  double rho = pr[O_RHO], P = pr[O_P];
  double u[3] = {pr[O_UX], pr[O_UY], pr[O_UZ]};
  double uu = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) uu += gi[S6[a][b]] * u[a] * u[b];
  double w = sqrt(1.0 + W * W * uu);
  double rhw2 = rho * (1.0 + pr[O_EPS] + P / rho) * w * w;
  double vd[3] = {u[0] / w, u[1] / w, u[2] / w};    /* v_i */
  double vu[3];                                      /* v^i = W^2 gt^ij v_j */
  for (int a = 0; a < 3; ++a) {
    double sum = 0.0;
    for (int b = 0; b < 3; ++b) sum += gi[S6[a][b]] * vd[b];
    vu[a] = W * W * sum;
  }
  double vv = vd[0] * vu[0] + vd[1] * vu[1] + vd[2] * vu[2];
  double W3i = 1.0 / (W * W * W);
  double sk[2];
  for (int e = 0; e < 2; ++e) {
    /* d_e gt^ab = -gt^ac gt^bd d_e gt_cd */
    double vvdg = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double dgi = 0.0;
        for (int cc = 0; cc < 3; ++cc)
          for (int d2 = 0; d2 < 3; ++d2) dgi -= gi[S6[a][cc]] * gi[S6[b][d2]] * dh[e][S6[cc][d2]];
        vvdg += vd[a] * vd[b] * dgi;
      }
    double vdb = vd[0] * db[e][0] + vd[1] * db[e][1] + vd[2] * db[e][2];
    double dalW3 = W3i * dal[e] - 3.0 * al * W3i / W * dW[e];  /* d(alpha W^-3) */
    sk[e] = P * dalW3 - W3i * rhw2 * (dal[e] - vdb + 0.5 * W * W * al * vvdg + al / W * vv * dW[e]);
  }
  /* geometric source (f_Sphi)^phi / varpi = alpha psi^6 (S_y vbar^y + P) / x */
  double geo = 0.0;
  if (x > 0.0) {
    double vbary = vu[1] - betay / al;
    geo = al * W3i * (rhw2 * vd[1] * vbary + P) / x;
  }
  /* K^ij S_ij = rho h w^2 K_ij v^i v^j + P gamma^ij K_ij, K_ij = (At_ij + gt_ij K/3) / W^2 */
  double Kd[3][3], vKv = 0.0, trK = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) Kd[a][b] = (A[S6[a][b]] + g[S6[a][b]] * K / 3.0) / (W * W);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      vKv += vu[a] * vu[b] * Kd[a][b];
      trK += W * W * gi[S6[a][b]] * Kd[a][b];
    }
  double KS = rhw2 * vKv + P * trK;
  src[O_QD] = 0.0;
  src[O_QSX] = sk[0] + geo;
  src[O_QSY] = 0.0;
  src[O_QSZ] = sk[1];
  src[O_QE] = W3i * (al * KS - rhw2 * (vu[0] * dal[0] + vu[2] * dal[1]));
}

static void hydro_rhs(orc_ctx *c, int l, int s, double **U, int jmax, int kmax) {
  orc_level *L = &c->lv[l];
  const orc_params *p = &c->p;
  int cyl = p->geometry == 1;
  double wb = stage_b(p, s);
  int has_child = l < p->n_levels - 1, has_parent = l > 0;
  /* x-faces j+1/2, j in [0, jmax], rows [1, kmax] (rows in parallel: each
     flux-register entry belongs to one row) */
  int nfb = 0;
#pragma omp parallel for schedule(static) reduction(+ : nfb)
  for (int k = 1; k <= kmax; ++k)
    for (int j = 0; j <= jmax; ++j) {
      double pl[5], prr[5], al, be[3], W, h[6], f[O_NCONS];
      face_prims(L, j, k, 0, pl, prr);
      face_metric(L, U, j, k, 0, &al, be, &W, h);
      nfb += orc_riemann_flux(p, 0, pl, prr, al, be, W, h, f);
      double xf = j * L->dx;  /* x_{j+1/2} */
      double area = cyl ? xf * L->dz : L->dz;
      int id = oidx(L, j, k);
      for (int v = 0; v < O_NCONS; ++v) L->fx[v][id] = area * f[v];
      if (cyl) L->fx[O_QSY][id] *= xf;
      if (has_child && j == L->nx / 2 && k <= L->nz / 2)
        for (int v = 0; v < O_NCONS; ++v) L->freg[0][v][k] += wb * L->fx[v][id];
      if (has_parent && j == L->nx && k <= L->nz)
        for (int v = 0; v < O_NCONS; ++v) L->freg[1][v][k] += wb * L->wpar * L->fx[v][id];
    }
  /* z-faces k+1/2 (the register rows k = nz/2, nz are each one iteration) */
#pragma omp parallel for schedule(static) reduction(+ : nfb)
  for (int k = 0; k <= kmax; ++k)
    for (int j = 1; j <= jmax; ++j) {
      double pl[5], prr[5], al, be[3], W, h[6], f[O_NCONS];
      face_prims(L, j, k, 1, pl, prr);
      face_metric(L, U, j, k, 1, &al, be, &W, h);
      nfb += orc_riemann_flux(p, 1, pl, prr, al, be, W, h, f);
      /* equatorial mirror face: D, S_x, S_phi and E are even in z, so their
         z-fluxes vanish on the symmetry plane (only the pressure term of the
         S_z flux remains); the solver reproduces this only up to rounding */
      if (cyl && k == 0) f[O_QD] = f[O_QSX] = f[O_QSY] = f[O_QE] = 0.0;
      double x = xc(L, j);
      double area = cyl ? x * L->dx : L->dx;
      int id = oidx(L, j, k);
      for (int v = 0; v < O_NCONS; ++v) L->fz[v][id] = area * f[v];
      if (cyl) L->fz[O_QSY][id] *= x;
      if (has_child && k == L->nz / 2 && j <= L->nx / 2)
        for (int v = 0; v < O_NCONS; ++v) L->freg[2][v][j] += wb * L->fz[v][id];
      if (has_parent && k == L->nz && j <= L->nx)
        for (int v = 0; v < O_NCONS; ++v) L->freg[3][v][j] += wb * L->wpar * L->fz[v][id];
    }
  c->n_fallback += nfb;
  /* divergence and sources */
#pragma omp parallel for schedule(static)
  for (int k = 1; k <= kmax; ++k)
    for (int j = 1; j <= jmax; ++j) {
      int id = oidx(L, j, k);
      double x = xc(L, j);
      double vol = cyl ? x * L->dx * L->dz : L->dx * L->dz;
      double div[O_NCONS];
      for (int v = 0; v < O_NCONS; ++v)
        div[v] = (L->fx[v][id] - L->fx[v][oidx(L, j - 1, k)] + L->fz[v][id] - L->fz[v][oidx(L, j, k - 1)]) / vol;

      /* metric and its central 6th-order derivatives at the cell centre */
      double al = U[O_AL][id], W = U[O_W][id];
      double h[6];
      cell_h(U, id, h);
      double g[6] = {1.0 + h[0], h[1], h[2], 1.0 + h[3], h[4], 1.0 + h[5]}, gi[6];
      orc_inv3(g, gi, 0);
      static const int S6[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
      double dal[2] = {0, 0}, dW[2] = {0, 0}, db[2][3] = {{0}}, dh[2][6] = {{0}};
      for (int n = -3; n <= 3; ++n) {   /* difference form, exact zero on constants */
        int ix = oidx(L, j + n, k), iz = oidx(L, j, k + n);
        double cc = orc_c1[n + 3];
        dal[0] += cc * (U[O_AL][ix] - U[O_AL][id]); dal[1] += cc * (U[O_AL][iz] - U[O_AL][id]);
        dW[0] += cc * (U[O_W][ix] - U[O_W][id]); dW[1] += cc * (U[O_W][iz] - U[O_W][id]);
        for (int a = 0; a < 3; ++a) {
          db[0][a] += cc * (U[O_BX + a][ix] - U[O_BX + a][id]);
          db[1][a] += cc * (U[O_BX + a][iz] - U[O_BX + a][id]);
        }
        for (int a = 0; a < 6; ++a) {
          dh[0][a] += cc * (U[O_HXX + a][ix] - U[O_HXX + a][id]);
          dh[1][a] += cc * (U[O_HXX + a][iz] - U[O_HXX + a][id]);
        }
      }
      double dd[2] = {L->dx, L->dz};
      for (int e = 0; e < 2; ++e) {
        dal[e] /= dd[e]; dW[e] /= dd[e];
        for (int a = 0; a < 3; ++a) db[e][a] /= dd[e];
        for (int a = 0; a < 6; ++a) dh[e][a] /= dd[e];
      }
      double pr[O_NPRIM];
      for (int f = 0; f < O_NPRIM; ++f) pr[f] = L->prim[f][id];
      double A[6];
      for (int a = 0; a < 6; ++a) A[a] = U[O_AXX + a][id];
      double K = U[O_KH][id] + 2.0 * U[O_TH][id];
      double src[O_NCONS];
      orc_hydro_source(p, pr, al, U[O_BY][id], W, h, A, K, dal, db, dW, dh, cyl ? x : 0.0, src);
      for (int v = 0; v < O_NCONS; ++v) L->rhs[O_NMET + v][id] = src[v] - div[v];
    }
}

/* ---------------- Z4c right-hand side on a level ---------------- */

static void z4c_rhs(orc_ctx *c, int l, double **U, int jmax, int kmax) {
  orc_level *L = &c->lv[l];
  size_t n = (size_t)L->px * L->pz;
  double *dy[O_NMET], *dyy[O_NMET];
  int cyl = c->p.geometry == 1;
  if (cyl) {
    for (int f = 0; f < O_NMET; ++f) { dy[f] = alloc_arr(n); dyy[f] = alloc_arr(n); }
    orc_cartoon_dy(c, l, U, dy, dyy);
  }
#pragma omp parallel for schedule(static)
  for (int k = 1; k <= kmax; ++k)
    for (int j = 1; j <= jmax; ++j) {
      int id = oidx(L, j, k);
      double Q[O_NMET], dQ[O_NMET][3], ddQ[O_NMET][6], adv[O_NMET], ko[O_NMET], r[O_NMET];
      orc_derivs_cell(c, l, U, cyl ? dy : NULL, cyl ? dyy : NULL, j, k, Q, dQ, ddQ, adv);
      orc_ko_cell(c, l, U, j, k, ko);
      double pr[O_NPRIM], E, Si[3], Sij[6], h[6];
      for (int f = 0; f < O_NPRIM; ++f) pr[f] = L->prim[f][id];
      cell_h(U, id, h);
      orc_matter_point(&c->p, pr, Q[O_W], h, &E, Si, Sij);
      double x = xc(L, j), z = zc(L, k);
      double fz = exp(-(x * x + z * z) / (c->p.r_z4 * c->p.r_z4));
      orc_z4c_point(&c->p, Q, dQ, ddQ, adv, E, Si, Sij, fz, r);
      for (int f = 0; f < O_NMET; ++f) L->rhs[f][id] = r[f] + ko[f];
    }
  if (cyl)
    for (int f = 0; f < O_NMET; ++f) { free(dy[f]); free(dyy[f]); }
}

/* ---------------- algebraic constraints, Sec. II.B.1 ---------------- */

static void enforce(double **U, int id) {
  double g[6], gi[6], d;
  for (int a = 0; a < 6; ++a) g[a] = U[O_HXX + a][id];
  g[0] += 1.0; g[3] += 1.0; g[5] += 1.0;
  orc_inv3(g, gi, &d);
  static const int S6[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  double trA = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) trA += gi[S6[a][b]] * U[O_AXX + S6[a][b]][id];
  double f13 = pow(d, -1.0 / 3.0), f16 = pow(d, -1.0 / 6.0);
  for (int a = 0; a < 6; ++a) {
    double At = U[O_AXX + a][id] - g[a] * trA / 3.0;
    U[O_AXX + a][id] = f13 * At;
    double gn = f13 * g[a];
    U[O_HXX + a][id] = (a == 0 || a == 3 || a == 5) ? gn - 1.0 : gn;
  }
  U[O_W][id] *= f16;
  U[O_KH][id] += trA;
}

/* cell (j, k) of level l inside the excised inner boundary x^2 + z^2 < r_hold^2 */
static int held(const orc_ctx *c, int l, int j, int k) {
  if (!(c->p.r_hold > 0.0)) return 0;
  double x = xc(&c->lv[l], j), z = zc(&c->lv[l], k);
  return x * x + z * z < c->p.r_hold * c->p.r_hold;
}

/* ---------------- primitive recovery over a region ---------------- */

/* skip_held: leave the cells of the excised inner boundary alone (stage updates) */
static void c2p_region_h(orc_ctx *c, int l, double **U, int j0, int j1, int k0, int k1, int skip_held) {
  orc_level *L = &c->lv[l];
#pragma omp parallel for schedule(static)
  for (int k = k0; k <= k1; ++k)
    for (int j = j0; j <= j1; ++j) {
      if (skip_held && held(c, l, j, k)) continue;
      int id = oidx(L, j, k);
      double q[O_NCONS], pr[O_NPRIM], h[6];
      for (int f = 0; f < O_NCONS; ++f) q[f] = U[O_NMET + f][id];
      cell_h(U, id, h);
      int it;
      int st = orc_con2prim(&c->p, q, U[O_W][id], h, xc(L, j), pr, &it);
      for (int f = 0; f < O_NCONS; ++f) U[O_NMET + f][id] = q[f];
      for (int f = 0; f < O_NPRIM; ++f) L->prim[f][id] = pr[f];
      L->status[id] = (unsigned char)st;
    }
}

static void c2p_region(orc_ctx *c, int l, double **U, int j0, int j1, int k0, int k1) {
  c2p_region_h(c, l, U, j0, j1, k0, k1, 0);
}

/* ---------------- one RK stage on all levels ---------------- */

/* One RK stage of level l with step dt.  At stage 0 the level's flux
   registers at its own child boundary (0, 2) are cleared, those at its parent
   boundary (1, 3) when reset_parent is set (a sub-cycled level sums them over
   both of its steps inside one parent step). */
static void stage_level(orc_ctx *c, int l, int s, double dt, int reset_parent) {
  const orc_params *p = &c->p;
  orc_level *L = &c->lv[l];
  if (s == 0) {
    size_t rn = sizeof(double) * ((p->nx > p->nz ? p->nx : p->nz) + 2);
    for (int f = 0; f < O_NCONS; ++f) {
      memset(L->freg[0][f], 0, rn);
      memset(L->freg[2][f], 0, rn);
      if (reset_parent) { memset(L->freg[1][f], 0, rn); memset(L->freg[3][f], 0, rn); }
    }
  }
  double **U = stage_state(c, l, s);
  int jmax, kmax;
  region(c, l, s, &jmax, &kmax);
  hydro_rhs(c, l, s, U, jmax, kmax);
  if (p->evolve_spacetime) z4c_rhs(c, l, U, jmax, kmax);
#pragma omp parallel for schedule(static)
  for (int k = 1; k <= kmax; ++k)
    for (int j = 1; j <= jmax; ++j) {
      int id = oidx(L, j, k);
      int hold = held(c, l, j, k);
      for (int f = 0; f < O_NSTATE; ++f) {
        if (f < O_NMET && !p->evolve_spacetime) continue;
        if (f >= O_NMET && hold) { L->us[f][id] = L->un[f][id]; continue; }   /* excised: U^n kept */
        double un = L->un[f][id], us = U[f][id], kk = L->rhs[f][id];
        double out;
        if (p->rk == 0) {
          static const double a4[3] = {0.5, 0.5, 1.0};
          if (s < 3) {
            L->ka[f][id] = (s == 0 ? 0.0 : L->ka[f][id]) + stage_b(p, s) * kk;
            out = un + a4[s] * dt * kk;
          } else {
            out = un + dt * (L->ka[f][id] + kk / 6.0);
          }
        } else {
          if (s == 0) out = un + dt * kk;
          else if (s == 1) out = 0.75 * un + 0.25 * us + 0.25 * dt * kk;
          else out = un / 3.0 + 2.0 / 3.0 * us + 2.0 / 3.0 * dt * kk;
        }
        L->us[f][id] = out;
      }
      if (p->evolve_spacetime) enforce(L->us, id);
    }
  c2p_region_h(c, l, L->us, 1, jmax, 1, kmax, 1);
}

static void swap_level(orc_ctx *c, int l) {
  for (int f = 0; f < O_NSTATE; ++f) {
    double *t = c->lv[l].un[f]; c->lv[l].un[f] = c->lv[l].us[f]; c->lv[l].us[f] = t;
  }
}

void orc_stage(orc_ctx *c, int s, double dt) {
  const orc_params *p = &c->p;
  int S = n_stages(p);
  if (s == 0) c->dt_step = dt;
  for (int l = 0; l < p->n_levels; ++l) stage_level(c, l, s, dt, 1);
  if (s == S - 1) {
    if (p->geometry == 1) outer_fill(c, c->lv[0].us, dt);
    for (int l = 0; l < p->n_levels; ++l) swap_level(c, l);
  }
}

/* ---------------- restriction and reflux, Sec. II.D ---------------- */

/* Lagrange weights at the parent centre (child index 2j - 1/2) from 8 child
   cells: centred on 2j-4..2j+3, shifted inward so that no node passes N. */
static void rest_weights(int j, int N, int *base, double w[8]) {
  int b = 2 * j - 4;
  if (b + 7 > N) b = N - 7;
  double nodes[8];
  for (int n = 0; n < 8; ++n) nodes[n] = b + n;
  orc_lagrange(8, nodes, 2.0 * j - 0.5, w);
  *base = b;
}

/* Restriction of level l onto its parent, reflux of the parent cells next to
   the refinement boundary with the parent's step dt, recovery there, and the
   parent's axis/equator ghosts. */
static void restrict_pair(orc_ctx *c, int l, double dt) {
  {
    orc_level *C = &c->lv[l], *P = &c->lv[l - 1];
    double **Uc = C->un, **Up = P->un;
    /* the child's axis/equator ghosts mirror its final (already restricted) interior */
    parity_fill(c, l, Uc);
    int Nh = P->nx / 2;
    for (int k = 1; k <= Nh; ++k)
      for (int j = 1; j <= Nh; ++j) {
        int d = oidx(P, j, k);
        /* conservative volume average (cylindrical volumes ~ x) */
        double vp = xc(P, j) * P->dx * P->dz;
        for (int f = 0; f < O_NCONS; ++f) {
          double s = 0.0;
          for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
              int jj = 2 * j - 1 + a, kk = 2 * k - 1 + b;
              s += Uc[O_NMET + f][oidx(C, jj, kk)] * xc(C, jj) * C->dx * C->dz;
            }
          Up[O_NMET + f][d] = s / vp;
        }
        /* metric: 8th-order Lagrange, tensor product */
        int bx, bz;
        double wx[8], wz[8];
        rest_weights(j, C->nx, &bx, wx);
        rest_weights(k, C->nz, &bz, wz);
        for (int f = 0; f < O_NMET; ++f) {
          double q0 = Uc[f][oidx(C, 2 * j, 2 * k)], s = 0.0;
          for (int b = 0; b < 8; ++b)
            for (int a = 0; a < 8; ++a) s += wx[a] * wz[b] * (Uc[f][oidx(C, bx + a, bz + b)] - q0);
          Up[f][d] = q0 + s;
        }
      }
    /* reflux on the parent cells just outside the child: replace the coarse
       face flux by the sum of the fine face fluxes (RK-weighted over the step;
       a sub-cycled child's registers carry dt_child / dt over its two steps) */
    for (int k = 1; k <= Nh; ++k) {
      int d = oidx(P, Nh + 1, k);
      double vp = xc(P, Nh + 1) * P->dx * P->dz;
      for (int f = 0; f < O_NCONS; ++f) {
        double fine = C->freg[1][f][2 * k - 1] + C->freg[1][f][2 * k];
        Up[O_NMET + f][d] += dt * (fine - P->freg[0][f][k]) / vp;
      }
    }
    for (int j = 1; j <= Nh; ++j) {
      int d = oidx(P, j, Nh + 1);
      double vp = xc(P, j) * P->dx * P->dz;
      for (int f = 0; f < O_NCONS; ++f) {
        double fine = C->freg[3][f][2 * j - 1] + C->freg[3][f][2 * j];
        Up[O_NMET + f][d] += dt * (fine - P->freg[2][f][j]) / vp;
      }
    }
    c2p_region(c, l - 1, Up, 1, Nh, 1, Nh);
    c2p_region(c, l - 1, Up, Nh + 1, Nh + 1, 1, Nh);
    c2p_region(c, l - 1, Up, 1, Nh, Nh + 1, Nh + 1);
    /* ghosts of the parent mirror its restricted interior */
    parity_fill(c, l - 1, Up);
  }
}

void orc_restrict_reflux(orc_ctx *c) {
  for (int l = c->p.n_levels - 1; l >= 1; --l) restrict_pair(c, l, c->dt_step);
}

/* ---------------- diagnostics, Sec. II.F.1 ---------------- */

/* out: [||H||_2, ||M_x||_2, ||M_y||_2, ||M_z||_2, M_b, J, rho_max, n_status_flags]
   over the cells of each level not covered by a finer one; volume element
   2 pi x dx dz (cylindrical) or dx dz (planar), integrals over the
   computational domain. */
void orc_diag(orc_ctx *c, double *out) {
  const orc_params *p = &c->p;
  orc_fill(c, 0, 0.0);
  int cyl = p->geometry == 1;
  double sH = 0, sM[3] = {0, 0, 0}, sV = 0, Mb = 0, J = 0, rmax = 0, nflag = 0;
  for (int l = 0; l < p->n_levels; ++l) {
    orc_level *L = &c->lv[l];
    double **U = L->un;
    size_t n = (size_t)L->px * L->pz;
    double *dy[O_NMET], *dyy[O_NMET];
    if (cyl && p->evolve_spacetime) {
      for (int f = 0; f < O_NMET; ++f) { dy[f] = alloc_arr(n); dyy[f] = alloc_arr(n); }
      orc_cartoon_dy(c, l, U, dy, dyy);
    }
    for (int k = 1; k <= L->nz; ++k)
      for (int j = 1; j <= L->nx; ++j) {
        if (l < p->n_levels - 1 && j <= L->nx / 2 && k <= L->nz / 2) continue;
        int id = oidx(L, j, k);
        double x = xc(L, j);
        double vol = cyl ? 2.0 * PI * x * L->dx * L->dz : L->dx * L->dz;
        Mb += U[O_NMET + O_QD][id] * vol;
        J += U[O_NMET + O_QSY][id] * vol;
        if (L->prim[O_RHO][id] > rmax) rmax = L->prim[O_RHO][id];
        if (L->status[id] & (O_ST_NOCONV | O_ST_BAD)) nflag += 1;
        sV += vol;
        if (p->evolve_spacetime) {
          double Q[O_NMET], dQ[O_NMET][3], ddQ[O_NMET][6], adv[O_NMET], pr[O_NPRIM], E, Si[3], Sij[6], h[6];
          orc_derivs_cell(c, l, U, cyl ? dy : NULL, cyl ? dyy : NULL, j, k, Q, dQ, ddQ, adv);
          for (int f = 0; f < O_NPRIM; ++f) pr[f] = L->prim[f][id];
          cell_h(U, id, h);
          orc_matter_point(p, pr, Q[O_W], h, &E, Si, Sij);
          double H, M[3];
          orc_constraints_point(Q, dQ, ddQ, E, Si, &H, M);
          sH += H * H * vol;
          for (int a = 0; a < 3; ++a) sM[a] += M[a] * M[a] * vol;
        }
      }
    if (cyl && p->evolve_spacetime)
      for (int f = 0; f < O_NMET; ++f) { free(dy[f]); free(dyy[f]); }
  }
  out[0] = sqrt(sH / sV);
  for (int a = 0; a < 3; ++a) out[1 + a] = sqrt(sM[a] / sV);
  out[4] = Mb; out[5] = J; out[6] = rmax; out[7] = nflag;
}

/* ---------------- data in / out ---------------- */

/* kind 0: 25 metric + (rho, u_x, u_y, u_z, P) padded planes; eps from the
   EOS, conserved variables from Eq. cons_var on every cell.
   kind 1: 30 state planes (metric + conserved); primitives recovered. */
int orc_set_level(orc_ctx *c, int l, int kind, const double *data) {
  if (l < 0 || l >= c->p.n_levels) return -1;
  orc_level *L = &c->lv[l];
  size_t n = (size_t)L->px * L->pz;
  if (kind == 0) {
    for (int f = 0; f < O_NMET; ++f) memcpy(L->un[f], data + f * n, n * sizeof(double));
    for (int k = 1 - ORC_G; k <= L->nz + ORC_G; ++k)
      for (int j = 1 - ORC_G; j <= L->nx + ORC_G; ++j) {
        int id = oidx(L, j, k);
        double pr[O_NPRIM];
        for (int v = 0; v < 4; ++v) pr[v] = data[(O_NMET + v) * n + id];
        pr[O_P] = data[(O_NMET + 4) * n + id];
        if (c->p.eos_adiabatic) pr[O_P] = orc_eos_pcold(&c->p, pr[O_RHO]);   /* zero temperature */
        pr[O_EPS] = orc_eos_eps(&c->p, pr[O_RHO], pr[O_P]);
        for (int f = 0; f < O_NPRIM; ++f) L->prim[f][id] = pr[f];
        double h[6], q[O_NCONS];
        cell_h(L->un, id, h);
        orc_prim2cons(&c->p, pr, L->un[O_W][id], h, xc(L, j), q);
        for (int f = 0; f < O_NCONS; ++f) L->un[O_NMET + f][id] = q[f];
      }
  } else {
    for (int f = 0; f < O_NSTATE; ++f) memcpy(L->un[f], data + f * n, n * sizeof(double));
    c2p_region(c, l, L->un, 1 - ORC_G, L->nx + ORC_G, 1 - ORC_G, L->nz + ORC_G);
  }
  for (int f = 0; f < O_NSTATE; ++f) memcpy(L->us[f], L->un[f], n * sizeof(double));
  return 0;
}

/* which: 0 step-start state, 1 stage state, 2 primitives, 3 rhs, 4 status */
int orc_read(orc_ctx *c, int l, int which, int field, double *out) {
  if (l < 0 || l >= c->p.n_levels) return -1;
  orc_level *L = &c->lv[l];
  size_t n = (size_t)L->px * L->pz;
  const double *src = NULL;
  if (which == 0) src = L->un[field];
  else if (which == 1) src = L->us[field];
  else if (which == 2) src = L->prim[field];
  else if (which == 3) src = L->rhs[field];
  else {
    for (size_t i = 0; i < n; ++i) out[i] = L->status[i];
    return 0;
  }
  memcpy(out, src, n * sizeof(double));
  return 0;
}

/* ---------------- Berger-Oliger sub-cycling, Sec. II.D ---------------- */

/* levels [0, G) share the coarse step; levels >= G take half their parent's step */
static int lockstep_levels(const orc_params *p) {
  int K = p->subcycle_from;
  return (K <= 0 || K >= p->n_levels) ? p->n_levels : K;
}

static void save_now(orc_ctx *c, int l) {
  orc_level *L = &c->lv[l];
  size_t n = (size_t)L->px * L->pz;
  for (int f = 0; f < O_NPRIM; ++f) memcpy(L->pnow[f], L->prim[f], n * sizeof(double));
}

/* after a parent step and its children's: t^n becomes t^{n-1} (a copy: the
   stage register keeps fields a frozen-metric run never rewrites) */
static void rotate_slices(orc_ctx *c, int l) {
  orc_level *L = &c->lv[l];
  size_t n = (size_t)L->px * L->pz;
  for (int f = 0; f < O_NSTATE; ++f) memcpy(L->uold[f], L->us[f], n * sizeof(double));
  for (int f = 0; f < O_NPRIM; ++f) { double *t = L->pold[f]; L->pold[f] = L->pnow[f]; L->pnow[f] = t; }
  L->have_old = 1;
}

/* two steps of dtl of sub-cycled level l inside one step of its parent */
static void advance_sub(orc_ctx *c, int l, double dtl) {
  const orc_params *p = &c->p;
  int S = n_stages(p), L = p->n_levels;
  c->lv[l].wpar = 0.5;
  for (int m = 0; m < 2; ++m) {
    for (int s = 0; s < S; ++s) {
      double **U = stage_state(c, l, s);
      time_interp(c, l - 1, 0.5 * (m + stage_c(p, s)));
      prolong_from(c, l, U, c->lv[l - 1].ut, c->lv[l - 1].pt, s == 0);
      parity_fill(c, l, U);
      if (s == 0 && l + 1 < L) save_now(c, l);
      stage_level(c, l, s, dtl, m == 0);
    }
    swap_level(c, l);
    if (l + 1 < L) {
      parity_fill(c, l, c->lv[l].un);
      advance_sub(c, l + 1, 0.5 * dtl);
      restrict_pair(c, l + 1, dtl);
      rotate_slices(c, l);
    }
  }
}

/* nsteps steps of the coarse step dt: levels below subcycle_from in lockstep,
   then each deeper level twice per step of its parent, restriction and
   reflux whenever a child has caught up with its parent */
void orc_step(orc_ctx *c, double dt, int nsteps) {
  const orc_params *p = &c->p;
  int S = n_stages(p), L = p->n_levels, G = lockstep_levels(p);
  for (int it = 0; it < nsteps; ++it) {
    if (G == L) {
      for (int s = 0; s < S; ++s) {
        orc_fill(c, s, dt);
        orc_stage(c, s, dt);
      }
      orc_restrict_reflux(c);
      continue;
    }
    c->dt_step = dt;
    for (int s = 0; s < S; ++s) {
      for (int l = 0; l < G; ++l) {
        double **U = stage_state(c, l, s);
        if (l == 0) outer_fill(c, U, stage_c(p, s) * dt);
        else prolong_fill(c, l, U, stage_state(c, l - 1, s), s == 0);
        parity_fill(c, l, U);
      }
      if (s == 0) save_now(c, G - 1);
      for (int l = 0; l < G; ++l) stage_level(c, l, s, dt, 1);
    }
    outer_fill(c, c->lv[0].us, dt);
    for (int l = 0; l < G; ++l) swap_level(c, l);
    parity_fill(c, G - 1, c->lv[G - 1].un);
    advance_sub(c, G, 0.5 * dt);
    restrict_pair(c, G, dt);
    rotate_slices(c, G - 1);
    for (int l = G - 1; l >= 1; --l) restrict_pair(c, l, dt);
  }
}

int orc_fallbacks(const orc_ctx *c) { return c->n_fallback; }

/* Worker threads of the parallel loops (OpenMP builds; the per-cell
   arithmetic, hence every result, is the same for any count). */
#ifdef _OPENMP
#include <omp.h>
void orc_set_threads(int n) { omp_set_num_threads(n > 0 ? n : omp_get_num_procs()); }
int orc_get_threads(void) { return omp_get_max_threads(); }
#else
void orc_set_threads(int n) { (void)n; }
int orc_get_threads(void) { return 1; }
#endif

/* Derivatives (central first, second, advection) of every metric field of the
   step-start state at n cells, with the cartoon y-derivatives; for tests. */
void orc_derivs_batch(orc_ctx *c, int l, int n, const int *js, const int *ks, double *dQo, double *ddQo, double *advo) {
  orc_level *L = &c->lv[l];
  size_t np = (size_t)L->px * L->pz;
  int cyl = c->p.geometry == 1;
  double *dy[O_NMET], *dyy[O_NMET];
  if (cyl) {
    for (int f = 0; f < O_NMET; ++f) { dy[f] = alloc_arr(np); dyy[f] = alloc_arr(np); }
    orc_cartoon_dy(c, l, L->un, dy, dyy);
  }
  for (int i = 0; i < n; ++i) {
    double Q[O_NMET], dQ[O_NMET][3], ddQ[O_NMET][6], adv[O_NMET];
    orc_derivs_cell(c, l, L->un, cyl ? dy : NULL, cyl ? dyy : NULL, js[i], ks[i], Q, dQ, ddQ, adv);
    memcpy(dQo + (size_t)i * O_NMET * 3, dQ, sizeof(dQ));
    memcpy(ddQo + (size_t)i * O_NMET * 6, ddQ, sizeof(ddQ));
    memcpy(advo + (size_t)i * O_NMET, adv, sizeof(adv));
  }
  if (cyl)
    for (int f = 0; f < O_NMET; ++f) { free(dy[f]); free(dyy[f]); }
}

/* The parent data a sub-cycled child sees at time t^n + theta (t^{n+1} - t^n)
   (time_interp), for tests: slices packs the level's padded planes in the
   order 25 metric at t^{n-1}, t^n, t^{n+1}, then 6 primitives at t^{n-1},
   t^n, t^{n+1}; out receives the 25 interpolated metric planes and the 6
   interpolated primitive planes.  have_old = 0: no t^{n-1} slice yet. */
void orc_time_interp_probe(orc_ctx *c, int l, double theta, int have_old, const double *slices, double *out) {
  orc_level *P = &c->lv[l];
  size_t n = (size_t)P->px * P->pz;
  const double *s = slices;
  for (int f = 0; f < O_NMET; ++f) memcpy(P->uold[f], s + (size_t)f * n, n * sizeof(double));
  s += (size_t)O_NMET * n;
  for (int f = 0; f < O_NMET; ++f) memcpy(P->us[f], s + (size_t)f * n, n * sizeof(double));
  s += (size_t)O_NMET * n;
  for (int f = 0; f < O_NMET; ++f) memcpy(P->un[f], s + (size_t)f * n, n * sizeof(double));
  s += (size_t)O_NMET * n;
  for (int f = 0; f < O_NPRIM; ++f) memcpy(P->pold[f], s + (size_t)f * n, n * sizeof(double));
  s += (size_t)O_NPRIM * n;
  for (int f = 0; f < O_NPRIM; ++f) memcpy(P->pnow[f], s + (size_t)f * n, n * sizeof(double));
  s += (size_t)O_NPRIM * n;
  for (int f = 0; f < O_NPRIM; ++f) memcpy(P->prim[f], s + (size_t)f * n, n * sizeof(double));
  P->have_old = have_old;
  time_interp(c, l, theta);
  for (int f = 0; f < O_NMET; ++f) memcpy(out + (size_t)f * n, P->ut[f], n * sizeof(double));
  for (int f = 0; f < O_NPRIM; ++f) memcpy(out + (size_t)(O_NMET + f) * n, P->pt[f], n * sizeof(double));
}
