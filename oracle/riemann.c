/*
 * Oracle (test infrastructure only): PPM reconstruction and the tetrad-frame
 * HLLC / TVDLF numerical flux of Sec. II.C.2 of Lam & Shibata (arXiv:2502.03223).
 */
#include <math.h>
#include "orc.h"

/* ---------------- PPM (Colella & Woodward 1984), Sec. II.C.2 ---------------- */

static double sgn(double v) { return v > 0.0 ? 1.0 : (v < 0.0 ? -1.0 : 0.0); }

/* monotonised-central limited slope, CW84 Eqs. (1.7)-(1.8) */
static double ppm_slope(double am, double a0, double ap) {
  double dl = a0 - am, dr = ap - a0;
  if (dl * dr <= 0.0) return 0.0;
  double dc = 0.5 * (ap - am);
  double m = fabs(dc);
  if (2.0 * fabs(dl) < m) m = 2.0 * fabs(dl);
  if (2.0 * fabs(dr) < m) m = 2.0 * fabs(dr);
  return sgn(dc) * m;
}

/* parabola monotonicity constraints, CW84 Eq. (1.10) */
static void ppm_mono(double a0, double *aL, double *aR) {
  if ((*aR - a0) * (a0 - *aL) <= 0.0) {
    *aL = a0;
    *aR = a0;
    return;
  }
  double d = *aR - *aL;
  double a6 = 6.0 * (a0 - 0.5 * (*aL + *aR));
  if (d * a6 > d * d) *aL = 3.0 * a0 - 2.0 * (*aR);
  else if (-d * d > d * a6) *aR = 3.0 * a0 - 2.0 * (*aL);
}

/* Face j+1/2 from the cells a[0..5] = j-2..j+3: returns the state on the left
   (from the parabola of cell j) and on the right (from cell j+1). */
void orc_ppm_face(const double a[6], double *left, double *right) {
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int i = 1; i <= 4; ++i) s[i] = ppm_slope(a[i - 1], a[i], a[i + 1]);
  double I[5];  /* I[i] = value at face between a[i] and a[i+1] */
  for (int i = 1; i <= 3; ++i) I[i] = a[i] + 0.5 * (a[i + 1] - a[i]) - (s[i + 1] - s[i]) / 6.0;
  double aL = I[1], aR = I[2];
  ppm_mono(a[2], &aL, &aR);
  *left = aR;
  double bL = I[2], bR = I[3];
  ppm_mono(a[3], &bL, &bR);
  *right = bL;
}

/* ---------------- tetrad-frame Riemann solver, Sec. II.C.2 ---------------- */

typedef struct { double D, S[3], E, P, vx, lm, lp; } sr_state;

/* tetrad-frame state from the tetrad 4-velocity components */
static void sr_fill(const orc_params *p, double rho, double P, const double ut[3], sr_state *s) {
  if (p->eos_adiabatic) P = orc_eos_pcold(p, rho);   /* zero temperature at the face too */
  double w = sqrt(1.0 + ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
  double v[3] = {ut[0] / w, ut[1] / w, ut[2] / w};
  double eps = orc_eos_eps(p, rho, P);
  double hh = 1.0 + eps + P / rho;
  double cs2 = orc_eos_cs2(p, rho, eps, P);
  s->D = rho * w;
  for (int a = 0; a < 3; ++a) s->S[a] = rho * hh * w * w * v[a];
  s->E = rho * hh * w * w - P;
  s->P = P;
  s->vx = v[0];
  double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  double disc = cs2 * (1.0 - v2) * (1.0 - v2 * cs2 - v[0] * v[0] * (1.0 - cs2));
  if (disc < 0.0) disc = 0.0;
  double den = 1.0 - v2 * cs2;
  s->lm = (v[0] * (1.0 - cs2) - sqrt(disc)) / den;
  s->lp = (v[0] * (1.0 - cs2) + sqrt(disc)) / den;
}

static void sr_flux(const sr_state *s, double f[5]) {
  f[0] = s->D * s->vx;
  f[1] = s->S[0] * s->vx + s->P;
  f[2] = s->S[1] * s->vx;
  f[3] = s->S[2] * s->vx;
  f[4] = (s->E + s->P) * s->vx;
}

static void sr_cons(const sr_state *s, double q[5]) {
  q[0] = s->D; q[1] = s->S[0]; q[2] = s->S[1]; q[3] = s->S[2]; q[4] = s->E;
}

/* Numerical flux through a coordinate face normal to dir (0: x, 1: z).
   pl/prr: (rho, u_x, u_y, u_z, P) on the two sides (covariant u_i).
   Metric at the face: alpha, beta^i, W, h_ij (gt_ij = delta_ij + h_ij).
   f: conservative flux alpha psi^6 (D vbar, S_j vbar + P delta, ...) with
   Cartesian momentum components.  Returns 1 if HLLC fell back to TVDLF. */
int orc_riemann_flux(const orc_params *p, int dir, const double pl[5], const double prr[5],
                     double alpha, const double beta[3], double W, const double h[6], double f[O_NCONS]) {
  /* relabel so that the face normal is the first axis: x-face (x,y,z); z-face (z,x,y) */
  int perm[3];
  if (dir == 0) { perm[0] = 0; perm[1] = 1; perm[2] = 2; }
  else { perm[0] = 2; perm[1] = 0; perm[2] = 1; }
  double g[3][3], gf[3][3];
  g[0][0] = 1.0 + h[0]; g[0][1] = g[1][0] = h[1]; g[0][2] = g[2][0] = h[2];
  g[1][1] = 1.0 + h[3]; g[1][2] = g[2][1] = h[4]; g[2][2] = 1.0 + h[5];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) gf[a][b] = g[perm[a]][perm[b]];
  double gs[6] = {gf[0][0], gf[0][1], gf[0][2], gf[1][1], gf[1][2], gf[2][2]}, gi[6];
  orc_inv3(gs, gi, 0);
  double gixx = gi[0], gixy = gi[1], gixz = gi[2];
  double bx = beta[perm[0]];
  double uL[3], uR[3];
  for (int a = 0; a < 3; ++a) { uL[a] = pl[1 + perm[a]]; uR[a] = prr[1 + perm[a]]; }

  /* tetrad legs (x-face form of Sec. II.C.2) */
  double Bh = 1.0 / sqrt(gixx), Ch = 1.0 / sqrt(gf[2][2]), Dh = Bh * Ch;
  double eu[3][3] = {  /* contravariant spatial components e_(a)^i */
      {W * Bh * gixx, W * Bh * gixy, W * Bh * gixz},
      {0.0, W * Dh * gf[2][2], -W * Dh * gf[1][2]},
      {0.0, 0.0, W * Ch}};
  /* covariant spatial components e_(a)_i = gamma_ij e_(a)^j.  For the second
     leg this gives (D/W)(-gt^xy, gt^xx, 0): the inverse-metric components
     (the printed covariant form carries gt_xy, gt_xx, which is not the
     lowered contravariant leg). */
  double ed[3][3] = {
      {Bh / W, 0.0, 0.0},
      {-Dh * gixy / W, Dh * gixx / W, 0.0},
      {Ch * gf[0][2] / W, Ch * gf[1][2] / W, Ch * gf[2][2] / W}};
  double utL[3], utR[3];
  for (int a = 0; a < 3; ++a) {
    utL[a] = eu[a][0] * uL[0] + eu[a][1] * uL[1] + eu[a][2] * uL[2];
    utR[a] = eu[a][0] * uR[0] + eu[a][1] * uR[1] + eu[a][2] * uR[2];
  }
  sr_state L, R;
  sr_fill(p, pl[0], pl[4], utL, &L);
  sr_fill(p, prr[0], prr[4], utR, &R);
  double qL[5], qR[5], fL[5], fR[5];
  sr_cons(&L, qL); sr_cons(&R, qR);
  sr_flux(&L, fL); sr_flux(&R, fR);

  double lamL = L.lm < R.lm ? L.lm : R.lm;
  double lamR = L.lp > R.lp ? L.lp : R.lp;
  double sqgxx = W * sqrt(gixx);           /* sqrt(gamma^xx), gamma^ij = W^2 gt^ij */
  double vint = bx / (alpha * sqgxx);      /* interface velocity */

  double F[5];
  int fallback = 0;
  if (p->solver == 0) {
    double qs[5], fs[5];
    if (lamL >= vint) {
      for (int n = 0; n < 5; ++n) { qs[n] = qL[n]; fs[n] = fL[n]; }
    } else if (lamR <= vint) {
      for (int n = 0; n < 5; ++n) { qs[n] = qR[n]; fs[n] = fR[n]; }
    } else {
      double dl = lamR - lamL;
      double qh[5], fh[5];
      for (int n = 0; n < 5; ++n) {
        qh[n] = (lamR * qR[n] - lamL * qL[n] + fL[n] - fR[n]) / dl;
        fh[n] = (lamR * fL[n] - lamL * fR[n] + lamR * lamL * (qR[n] - qL[n])) / dl;
      }
      /* F_E lam^2 - (E + F_Sx) lam + S_x = 0, the root with the minus sign,
         written as 2 S_x / ((E + F_Sx) + sqrt(disc)) */
      double bb = qh[4] + fh[1];
      double disc = bb * bb - 4.0 * fh[4] * qh[1];
      double lamc = 0.0, Pc = 0.0;
      int bad = 0;
      if (!(disc >= 0.0)) bad = 1;
      else {
        lamc = 2.0 * qh[1] / (bb + sqrt(disc));
        Pc = -lamc * fh[4] + fh[1];
        if (!(lamc >= lamL && lamc <= lamR) || !(Pc > 0.0)) bad = 1;
      }
      if (!bad) {
        const sr_state *K = (vint <= lamc) ? &L : &R;
        const double *qK = (vint <= lamc) ? qL : qR;
        const double *fK = (vint <= lamc) ? fL : fR;
        double lamK = (vint <= lamc) ? lamL : lamR;
        double den = lamK - lamc;
        double fac = lamK - K->vx;
        qs[0] = K->D * fac / den;
        qs[1] = (K->S[0] * fac + Pc - K->P) / den;
        qs[2] = K->S[1] * fac / den;
        qs[3] = K->S[2] * fac / den;
        qs[4] = (K->E * fac + Pc * lamc - K->P * K->vx) / den;
        for (int n = 0; n < 5; ++n) {
          fs[n] = fK[n] + lamK * (qs[n] - qK[n]);
          if (!isfinite(fs[n]) || !isfinite(qs[n])) bad = 1;
        }
      }
      if (bad) fallback = 1;
    }
    if (!fallback)
      for (int n = 0; n < 5; ++n) F[n] = fs[n] - vint * qs[n];
  }
  if (p->solver == 1 || fallback) {
    double a1 = fabs(lamL - vint), a2 = fabs(lamR - vint);
    double cmax = a1 > a2 ? a1 : a2;
    for (int n = 0; n < 5; ++n)
      F[n] = 0.5 * ((fL[n] - vint * qL[n]) + (fR[n] - vint * qR[n])) - 0.5 * cmax * (qR[n] - qL[n]);
  }

  /* back to the Eulerian frame, times alpha psi^6 */
  double pre = alpha / (W * W * W) * sqgxx;
  double Sf[3];
  for (int i = 0; i < 3; ++i) Sf[i] = ed[0][i] * F[1] + ed[1][i] * F[2] + ed[2][i] * F[3];
  f[O_QD] = pre * F[0];
  f[O_QE] = pre * F[4];
  double Sc[3];
  for (int a = 0; a < 3; ++a) Sc[perm[a]] = pre * Sf[a];
  f[O_QSX] = Sc[0];
  f[O_QSY] = Sc[1];
  f[O_QSZ] = Sc[2];
  return fallback;
}
