/*
 * Oracle (test infrastructure only): equation of state, primitive -> conserved
 * map and the primitive recovery of Sec. II.C.3-4 of Lam & Shibata
 * (arXiv:2502.03223).  Plain FP64, written for reading, not speed.
 */
#include <math.h>
#include "orc.h"

/* Hybrid EOS, Sec. II.C.3: a piecewise polytropic cold part,
     P_c = K_i rho^Gamma_i,  eps_c = K_i rho^(Gamma_i - 1) / (Gamma_i - 1) + Delta eps_i
   on rho_(i-1) <= rho < rho_i (rho_0 = 0), with K_1 = K, Gamma_1 = Gamma,
   Delta eps_1 = 0 and, going up through the transitions, K_(i+1) from the
   continuity of P_c and Delta eps_(i+1) from that of eps_c; plus the thermal
   Gamma-law P_th = rho (Gamma_th - 1) eps_th. */
static void cold_piece(const orc_params *p, double rho, double *K, double *G, double *de) {
  double k = p->K, g = p->Gamma, d = 0.0;
  for (int i = 0; i + 1 < p->n_pieces; ++i) {
    double rt = p->pwp_rho[i];
    if (rho < rt) break;
    double g2 = p->pwp_Gamma[i];
    double k2 = k * pow(rt, g - g2);                                   /* K_i rho_i^G_i = K_(i+1) rho_i^G_(i+1) */
    d = d + k * pow(rt, g - 1.0) / (g - 1.0) - k2 * pow(rt, g2 - 1.0) / (g2 - 1.0);
    k = k2;
    g = g2;
  }
  *K = k; *G = g; *de = d;
}

double orc_eos_pcold(const orc_params *p, double rho) {
  if (p->K == 0.0) return 0.0;
  double K, G, de;
  cold_piece(p, rho, &K, &G, &de);
  return K * pow(rho, G);
}

double orc_eos_ecold(const orc_params *p, double rho) {
  if (p->K == 0.0) return 0.0;
  double K, G, de;
  cold_piece(p, rho, &K, &G, &de);
  return K * pow(rho, G - 1.0) / (G - 1.0) + de;
}

/* Gamma_i of the piece holding rho (d ln P_c / d ln rho) */
double orc_eos_gamma_cold(const orc_params *p, double rho) {
  double K, G, de;
  cold_piece(p, rho, &K, &G, &de);
  return G;
}

/* P = P_cold + P_th with eps_th = eps - eps_cold (Sec. II.C.3). */
double orc_eos_press(const orc_params *p, double rho, double eps) {
  double eth = eps - orc_eos_ecold(p, rho);
  return orc_eos_pcold(p, rho) + (p->Gamma_th - 1.0) * rho * eth;
}

/* Inverse of the above in eps. */
double orc_eos_eps(const orc_params *p, double rho, double press) {
  return orc_eos_ecold(p, rho) + (press - orc_eos_pcold(p, rho)) / ((p->Gamma_th - 1.0) * rho);
}

/* Sound speed squared of the hybrid EOS:
   c_s^2 h rho = dP/drho|_eps rho + P dP/deps|_rho / rho = Gamma P_cold + Gamma_th P_th,
   clamped to [0, 1). */
double orc_eos_cs2(const orc_params *p, double rho, double eps, double press) {
  double pc = orc_eos_pcold(p, rho);
  double h = 1.0 + eps + press / rho;
  double cs2 = (orc_eos_gamma_cold(p, rho) * pc + p->Gamma_th * (press - pc)) / (rho * h);
  if (!(cs2 > 0.0)) cs2 = 0.0;
  if (cs2 >= 1.0) cs2 = 1.0 - 1e-15;
  return cs2;
}

/* Inverse of a symmetric 3x3 matrix stored (xx,xy,xz,yy,yz,zz), by cofactors. */
void orc_inv3(const double g[6], double gi[6], double *det) {
  double xx = g[0], xy = g[1], xz = g[2], yy = g[3], yz = g[4], zz = g[5];
  double cxx = yy * zz - yz * yz;
  double cxy = xz * yz - xy * zz;
  double cxz = xy * yz - xz * yy;
  double cyy = xx * zz - xz * xz;
  double cyz = xy * xz - xx * yz;
  double czz = xx * yy - xy * xy;
  double d = xx * cxx + xy * cxy + xz * cxz;
  gi[0] = cxx / d; gi[1] = cxy / d; gi[2] = cxz / d;
  gi[3] = cyy / d; gi[4] = cyz / d; gi[5] = czz / d;
  if (det) *det = d;
}

static void conf_metric(const double h[6], double gt[6]) {
  gt[0] = 1.0 + h[0]; gt[1] = h[1]; gt[2] = h[2];
  gt[3] = 1.0 + h[3]; gt[4] = h[4]; gt[5] = 1.0 + h[5];
}

/* gamma^{ij} a_i a_j with gamma^{ij} = W^2 gt^{ij} */
static double up_norm2(const double gti[6], double W, const double a[3]) {
  double s = gti[0] * a[0] * a[0] + gti[3] * a[1] * a[1] + gti[5] * a[2] * a[2]
           + 2.0 * (gti[1] * a[0] * a[1] + gti[2] * a[0] * a[2] + gti[4] * a[1] * a[2]);
  return W * W * s;
}

/* Eq. cons_var: q = psi^6 (rho w, rho h w u_i, rho h w^2 - P), psi^6 = W^-3.
   In cylindrical geometry the evolved azimuthal momentum is q_Sphi = x q_Sy
   (u_phi = x u_y, Sec. II.C.1). */
void orc_prim2cons(const orc_params *p, const double pr[O_NPRIM], double W, const double h[6], double x,
                   double q[O_NCONS]) {
  double gt[6], gti[6];
  conf_metric(h, gt);
  orc_inv3(gt, gti, 0);
  double u[3] = {pr[O_UX], pr[O_UY], pr[O_UZ]};
  double w = sqrt(1.0 + up_norm2(gti, W, u));
  double rho = pr[O_RHO], P = pr[O_P], eps = pr[O_EPS];
  double hh = 1.0 + eps + P / rho;
  double psi6 = 1.0 / (W * W * W);
  q[O_QD] = psi6 * rho * w;
  q[O_QSX] = psi6 * rho * hh * w * u[0];
  q[O_QSY] = psi6 * rho * hh * w * u[1];
  q[O_QSZ] = psi6 * rho * hh * w * u[2];
  q[O_QE] = psi6 * (rho * hh * w * w - P);
  if (p->geometry == 1) q[O_QSY] *= x;
}

/* ---------------- primitive recovery, Sec. II.C.4 (Galeazzi et al. 2013, App. C) ---------------- */

typedef struct {
  const orc_params *p;
  double D, qq, r;  /* D, q = E/D - 1, r = |S|/D */
} c2p_data;

/* master function f(z) = z - r / h(z), Eq. c2p_fn.  The thermal EOS is
   evaluated with eps clamped to the cold minimum (reading documented with the
   oracle), so the bracket stays valid; the unclamped eps decides afterwards
   whether the cold recovery is needed. */
static double c2p_master(double z, const c2p_data *d) {
  double w = sqrt(1.0 + z * z);
  double rho = d->D / w;
  double eps = w * d->qq - z * d->r + z * z / (1.0 + w);
  double emin = orc_eos_ecold(d->p, rho);
  if (eps < emin) eps = emin;
  double P = orc_eos_press(d->p, rho, eps);
  double a = P / (rho * (1.0 + eps));
  double h = (1.0 + eps) * (1.0 + a);
  return z - d->r / h;
}

/* cold master function z - r / h_cold(rho(z)) */
static double c2p_cold_master(double z, const c2p_data *d) {
  double w = sqrt(1.0 + z * z);
  double rho = d->D / w;
  double hc = 1.0 + orc_eos_ecold(d->p, rho) + orc_eos_pcold(d->p, rho) / rho;
  return z - d->r / hc;
}

/* Illinois variant of regula falsi on [a, b].  Returns the root estimate;
   *ok = 0 if the iteration cap was reached or the bracket had no sign change. */
static double illinois(double (*f)(double, const c2p_data *), const c2p_data *d, double a, double b,
                       double tol, int maxit, int *iters, int *ok) {
  double fa = f(a, d), fb = f(b, d);
  *iters = 0;
  *ok = 1;
  if (fa == 0.0) return a;
  if (fb == 0.0) return b;
  if (fa * fb > 0.0) {
    *ok = 0;
    return fabs(fa) < fabs(fb) ? a : b;
  }
  int side = 0;
  double c = a;
  for (int it = 1; it <= maxit; ++it) {
    *iters = it;
    c = (a * fb - b * fa) / (fb - fa);
    double fc = f(c, d);
    if (fc == 0.0) return c;
    if (fc * fb > 0.0) {           /* root in [a, c]: c replaces b */
      b = c; fb = fc;
      if (side == -1) fa *= 0.5;   /* a kept twice in a row */
      side = -1;
    } else {                       /* root in [c, b]: c replaces a */
      a = c; fa = fc;
      if (side == +1) fb *= 0.5;
      side = +1;
    }
    double scale = fabs(c) > 1e-30 ? fabs(c) : 1e-30;
    if (fabs(b - a) <= tol * scale) return c;
  }
  *ok = 0;
  return c;
}

static void set_atmosphere(const orc_params *p, double pr[O_NPRIM]) {
  pr[O_RHO] = p->rho_atm;
  pr[O_UX] = pr[O_UY] = pr[O_UZ] = 0.0;
  pr[O_EPS] = orc_eos_ecold(p, p->rho_atm);
  pr[O_P] = orc_eos_pcold(p, p->rho_atm);
}

/* Conserved -> primitive for one cell.  q is updated in place when the
   recovery had to change the state (S rescale, cold branch, atmosphere).
   Returns the status bits. */
int orc_con2prim(const orc_params *p, double q[O_NCONS], double W, const double h[6], double x,
                 double pr[O_NPRIM], int *iters) {
  double gt[6], gti[6];
  conf_metric(h, gt);
  orc_inv3(gt, gti, 0);
  double W3 = W * W * W;
  double D = q[O_QD] * W3;
  double S[3] = {q[O_QSX] * W3, q[O_QSY] * W3, q[O_QSZ] * W3};
  if (p->geometry == 1) S[1] /= x;
  double E = q[O_QE] * W3;
  int st = 0;
  *iters = 0;

  if (!(D > 0.0) || !isfinite(D) || !isfinite(E) || !isfinite(S[0]) || !isfinite(S[1]) || !isfinite(S[2])
      || !(E > 0.0)) {
    set_atmosphere(p, pr);
    orc_prim2cons(p, pr, W, h, x, q);
    return O_ST_ATM | O_ST_BAD;
  }
  /* rho = D / w <= D for any root (w >= 1), so D < rho_atm always ends in the
     atmosphere reset (Sec. II.C.4): the recovery's result would be discarded */
  if (D < p->rho_atm) {
    set_atmosphere(p, pr);
    orc_prim2cons(p, pr, W, h, x, q);
    return O_ST_ATM;
  }

  double r = sqrt(up_norm2(gti, W, S)) / D;
  if (p->eos_adiabatic) {
    /* "adiabatic" EOS (Sec. III): zero temperature, the energy equation is
       discarded: the cold recovery from D and S_i alone, the Lorentz factor
       capped at w_max through r (z = r / h_c <= r), then E rebuilt */
    double zmax = sqrt(p->w_max * p->w_max - 1.0);
    if (r > zmax) {
      double s = zmax / r;
      S[0] *= s; S[1] *= s; S[2] *= s;
      r = zmax;
      st |= O_ST_KRESCALE;
    }
    c2p_data dc = {p, D, 0.0, r};
    int ok = 1;
    double z = illinois(c2p_cold_master, &dc, 0.0, r, p->c2p_tol, p->c2p_maxit, iters, &ok);
    if (!ok) st |= O_ST_NOCONV;
    double w = sqrt(1.0 + z * z);
    double rho = D / w;
    double eps = orc_eos_ecold(p, rho);
    double P = orc_eos_pcold(p, rho);
    double hh = 1.0 + eps + P / rho;
    pr[O_RHO] = rho;
    pr[O_EPS] = eps;
    pr[O_P] = P;
    pr[O_UX] = S[0] / (D * hh);
    pr[O_UY] = S[1] / (D * hh);
    pr[O_UZ] = S[2] / (D * hh);
    if (rho < p->rho_atm) {
      set_atmosphere(p, pr);
      st |= O_ST_ATM;
    }
    orc_prim2cons(p, pr, W, h, x, q);
    return st;
  }
  double qq = E / D - 1.0;
  double k = r / (1.0 + qq);
  double vmax = sqrt(1.0 - 1.0 / (p->w_max * p->w_max));
  double kmax = 2.0 * vmax / (1.0 + vmax * vmax);
  if (k > kmax) {
    double s = kmax / k;
    S[0] *= s; S[1] *= s; S[2] *= s;
    r *= s;
    k = kmax;
    st |= O_ST_KRESCALE;
  }

  c2p_data d = {p, D, qq, r};
  double zm = 0.5 * k / sqrt(1.0 - 0.25 * k * k);
  double zp = k / sqrt(1.0 - k * k);
  int ok = 1;
  double z = illinois(c2p_master, &d, zm, zp, p->c2p_tol, p->c2p_maxit, iters, &ok);
  if (!ok) st |= O_ST_NOCONV;

  double w = sqrt(1.0 + z * z);
  double rho = D / w;
  double eps = w * qq - z * r + z * z / (1.0 + w);
  double P;
  if (eps < orc_eos_ecold(p, rho)) {
    /* cold recovery from (D, S_i) alone, then E is reset */
    int it2 = 0, ok2 = 1;
    z = illinois(c2p_cold_master, &d, 0.0, r, p->c2p_tol, p->c2p_maxit, &it2, &ok2);
    *iters += it2;
    if (!ok2) st |= O_ST_NOCONV;
    w = sqrt(1.0 + z * z);
    rho = D / w;
    eps = orc_eos_ecold(p, rho);
    P = orc_eos_pcold(p, rho);
    st |= O_ST_COLD;
  } else {
    P = orc_eos_press(p, rho, eps);
  }
  double hh = 1.0 + eps + P / rho;
  pr[O_RHO] = rho;
  pr[O_EPS] = eps;
  pr[O_P] = P;
  pr[O_UX] = S[0] / (D * hh);
  pr[O_UY] = S[1] / (D * hh);
  pr[O_UZ] = S[2] / (D * hh);

  if (rho < p->rho_atm) {
    set_atmosphere(p, pr);
    st |= O_ST_ATM;
  }
  if (st & (O_ST_ATM | O_ST_COLD | O_ST_KRESCALE)) orc_prim2cons(p, pr, W, h, x, q);
  return st;
}
