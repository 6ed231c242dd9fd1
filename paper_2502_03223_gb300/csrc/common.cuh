// Device-side building blocks of the SACRA-2D hot path on sm_103a:
// level views, the hybrid EOS, the primitive recovery, PPM and the
// tetrad-frame HLLC/TVDLF flux (Lam & Shibata, arXiv:2502.03223, Sec. II.C).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sacra2d.h"

namespace sacra {

constexpr int GH = 8;          // padding on every side ((4+4) buffer, Sec. II.A)
constexpr int NMET = 25;
constexpr int NCONS = 5;
constexpr int NST = 30;
constexpr int NPRIM = 6;

// state field numbers (see include/sacra2d.h)
enum : int {
  fW = 0, fHXX, fHXY, fHXZ, fHYY, fHYZ, fHZZ, fAXX, fAXY, fAXZ, fAYY, fAYZ, fAZZ,
  fKH, fGX, fGY, fGZ, fTH, fAL, fBX, fBY, fBZ, fBBX, fBBY, fBBZ,
  fQD, fQSX, fQSY, fQSZ, fQE
};
enum : int { pRHO = 0, pUX, pUY, pUZ, pP, pEPS };

// recovery status bits
constexpr int ST_NOCONV = 1, ST_COLD = 2, ST_ATM = 4, ST_KRESCALE = 8, ST_BAD = 16;

struct DevParams {
  int geometry, evolve, solver, rk, c2p_maxit, n_levels;
  double K, Gamma, Gamma_th, rho_atm, w_max, c2p_tol;
  double kappa, eta_B, eps_ko, r_z4;
};

// One refinement level as seen by a kernel: planes of P = px * pz doubles.
struct Lev {
  int nx, nz, px, pz, rw;
  double dx, dz;
  size_t P;
  double *un, *us, *ka, *rhs;   // NST planes each
  double *prim;                 // NPRIM planes
  int *status;
  double *fx, *fz;              // NCONS planes of face fluxes (area-weighted)
  double *freg;                 // 4 x NCONS x rw flux registers
  double *dy, *dyy;             // NMET planes of cartoon d_y, d_yy
  unsigned long long *nfb;      // HLLC -> TVDLF fallback counter
};

__host__ __device__ inline int cid(const Lev &L, int j, int k) { return (k + GH - 1) * L.px + (j + GH - 1); }

// ------------------------------------------------------------------ small tensor helpers

struct Sym3 {
  double xx, xy, xz, yy, yz, zz;
};

__device__ inline double s3get(const Sym3 &m, int i, int j) {
  const int t = i * 3 + j;
  switch (t) {
    case 0: return m.xx;
    case 1: case 3: return m.xy;
    case 2: case 6: return m.xz;
    case 4: return m.yy;
    case 5: case 7: return m.yz;
    default: return m.zz;
  }
}

__device__ inline Sym3 s3inv(const Sym3 &g, double *detp) {
  const double cxx = g.yy * g.zz - g.yz * g.yz;
  const double cxy = g.xz * g.yz - g.xy * g.zz;
  const double cxz = g.xy * g.yz - g.xz * g.yy;
  const double det = g.xx * cxx + g.xy * cxy + g.xz * cxz;
  const double id = 1.0 / det;
  Sym3 r;
  r.xx = cxx * id; r.xy = cxy * id; r.xz = cxz * id;
  r.yy = (g.xx * g.zz - g.xz * g.xz) * id;
  r.yz = (g.xy * g.xz - g.xx * g.yz) * id;
  r.zz = (g.xx * g.yy - g.xy * g.xy) * id;
  if (detp) *detp = det;
  return r;
}

// a^i b^j m_ij for symmetric m
__device__ inline double s3quad(const Sym3 &m, const double a[3], const double b[3]) {
  return m.xx * a[0] * b[0] + m.yy * a[1] * b[1] + m.zz * a[2] * b[2]
       + m.xy * (a[0] * b[1] + a[1] * b[0]) + m.xz * (a[0] * b[2] + a[2] * b[0]) + m.yz * (a[1] * b[2] + a[2] * b[1]);
}

__device__ inline void s3vec(const Sym3 &m, const double a[3], double o[3]) {
  o[0] = m.xx * a[0] + m.xy * a[1] + m.xz * a[2];
  o[1] = m.xy * a[0] + m.yy * a[1] + m.yz * a[2];
  o[2] = m.xz * a[0] + m.yz * a[1] + m.zz * a[2];
}

__device__ inline Sym3 conf_metric(const double *U, size_t P, int id) {
  Sym3 g;
  g.xx = 1.0 + U[(size_t)fHXX * P + id];
  g.xy = U[(size_t)fHXY * P + id];
  g.xz = U[(size_t)fHXZ * P + id];
  g.yy = 1.0 + U[(size_t)fHYY * P + id];
  g.yz = U[(size_t)fHYZ * P + id];
  g.zz = 1.0 + U[(size_t)fHZZ * P + id];
  return g;
}

// ------------------------------------------------------------------ EOS (Sec. II.C.3)

// The FP64 pow is a long instruction sequence on this part; Gamma = 2 (all
// the neutron-star workloads) takes the exact product instead, rounded the
// same way as K * pow(rho, 2).
__device__ inline double eos_pc(const DevParams &p, double rho) {
  if (p.K == 0.0) return 0.0;
  return p.Gamma == 2.0 ? p.K * (rho * rho) : p.K * pow(rho, p.Gamma);
}
__device__ inline double eos_ec(const DevParams &p, double rho) {
  if (p.K == 0.0) return 0.0;
  return p.Gamma == 2.0 ? p.K * rho : p.K * pow(rho, p.Gamma - 1.0) / (p.Gamma - 1.0);
}
__device__ inline double eos_p(const DevParams &p, double rho, double eps) {
  return eos_pc(p, rho) + (p.Gamma_th - 1.0) * rho * (eps - eos_ec(p, rho));
}
__device__ inline double eos_eps(const DevParams &p, double rho, double P) {
  return eos_ec(p, rho) + (P - eos_pc(p, rho)) / ((p.Gamma_th - 1.0) * rho);
}
// c_s^2 rho h = Gamma P_cold + Gamma_th P_th, clamped to [0, 1)
__device__ inline double eos_cs2(const DevParams &p, double rho, double eps, double P) {
  const double pc = eos_pc(p, rho);
  const double h = 1.0 + eps + P / rho;
  double c2 = (p.Gamma * pc + p.Gamma_th * (P - pc)) / (rho * h);
  if (!(c2 > 0.0)) c2 = 0.0;
  if (c2 >= 1.0) c2 = 1.0 - 1e-15;
  return c2;
}

// ------------------------------------------------------------------ primitive <-> conserved (Eq. cons_var)

// pr: rho, u_x, u_y, u_z, P, eps; q: psi^6 (D, S_x, S_y or x S_y, S_z, E)
__device__ inline void prim_to_cons(const DevParams &p, const double pr[NPRIM], double W, const Sym3 &gt, double x,
                                    double q[NCONS]) {
  const Sym3 gi = s3inv(gt, nullptr);
  const double u[3] = {pr[pUX], pr[pUY], pr[pUZ]};
  const double w = sqrt(1.0 + W * W * s3quad(gi, u, u));
  const double rho = pr[pRHO], P = pr[pP];
  const double rhw = rho * (1.0 + pr[pEPS] + P / rho) * w;
  const double psi6 = 1.0 / (W * W * W);
  q[0] = psi6 * rho * w;
  q[1] = psi6 * rhw * u[0];
  q[2] = psi6 * rhw * u[1] * (p.geometry == SACRA_CYLINDRICAL ? x : 1.0);
  q[3] = psi6 * rhw * u[2];
  q[4] = psi6 * (rhw * w - P);
}

// Master functions of the recovery (Sec. II.C.4, Eq. c2p_fn); COLD selects
// z - r / h_cold(rho(z)).  The thermal EOS sees eps clamped to the cold curve.
template <bool COLD>
__device__ inline double c2p_fun(const DevParams &p, double z, double D, double qq, double r) {
  const double w = sqrt(1.0 + z * z);
  const double rho = D / w;
  if (COLD) {
    const double hc = 1.0 + eos_ec(p, rho) + eos_pc(p, rho) / rho;
    return z - r / hc;
  }
  double eps = w * qq - z * r + z * z / (1.0 + w);
  const double emin = eos_ec(p, rho);
  if (eps < emin) eps = emin;
  const double P = eos_p(p, rho, eps);
  const double a = P / (rho * (1.0 + eps));
  return z - r / ((1.0 + eps) * (1.0 + a));
}

// Illinois bracketing iteration on [a, b]; *ok = 0 on no sign change or cap
template <bool COLD>
__device__ double illinois(const DevParams &p, double a, double b, double D, double qq, double r, int *its, int *ok) {
  double fa = c2p_fun<COLD>(p, a, D, qq, r), fb = c2p_fun<COLD>(p, b, D, qq, r);
  *its = 0;
  *ok = 1;
  if (fa == 0.0) return a;
  if (fb == 0.0) return b;
  if (fa * fb > 0.0) {
    *ok = 0;
    return fabs(fa) < fabs(fb) ? a : b;
  }
  int last = 0;  // -1: the upper end moved last, +1: the lower end moved last
  double c = a;
  for (int it = 1; it <= p.c2p_maxit; ++it) {
    *its = it;
    c = (a * fb - b * fa) / (fb - fa);
    const double fc = c2p_fun<COLD>(p, c, D, qq, r);
    if (fc == 0.0) return c;
    if (fc * fb > 0.0) {
      b = c; fb = fc;
      if (last == -1) fa *= 0.5;
      last = -1;
    } else {
      a = c; fa = fc;
      if (last == +1) fb *= 0.5;
      last = +1;
    }
    if (fabs(b - a) <= p.c2p_tol * fmax(fabs(c), 1e-30)) return c;
  }
  *ok = 0;
  return c;
}

__device__ inline void atmosphere(const DevParams &p, double pr[NPRIM]) {
  pr[pRHO] = p.rho_atm;
  pr[pUX] = pr[pUY] = pr[pUZ] = 0.0;
  pr[pEPS] = eos_ec(p, p.rho_atm);
  pr[pP] = eos_pc(p, p.rho_atm);
}

// Conserved -> primitive for one cell (Galeazzi et al. 2013, App. C; cold
// fallback and atmosphere of Sec. II.C.4).  q is rewritten when the state
// had to change.  Returns the status bits.
__device__ inline int cons_to_prim(const DevParams &p, double q[NCONS], double W, const Sym3 &gt, double x,
                                   double pr[NPRIM]) {
  const Sym3 gi = s3inv(gt, nullptr);
  const double W3 = W * W * W;
  const double D = q[0] * W3;
  double S[3] = {q[1] * W3, q[2] * W3, q[3] * W3};
  if (p.geometry == SACRA_CYLINDRICAL) S[1] /= x;
  const double E = q[4] * W3;
  if (!(D > 0.0) || !(E > 0.0) || !isfinite(D) || !isfinite(E) || !isfinite(S[0]) || !isfinite(S[1]) ||
      !isfinite(S[2])) {
    atmosphere(p, pr);
    prim_to_cons(p, pr, W, gt, x, q);
    return ST_ATM | ST_BAD;
  }
  int st = 0;
  double r = sqrt(W * W * s3quad(gi, S, S)) / D;
  const double qq = E / D - 1.0;
  double k = r / (1.0 + qq);
  const double vmax = sqrt(1.0 - 1.0 / (p.w_max * p.w_max));
  const double kmax = 2.0 * vmax / (1.0 + vmax * vmax);
  if (k > kmax) {
    const double s = kmax / k;
    S[0] *= s; S[1] *= s; S[2] *= s;
    r *= s;
    k = kmax;
    st |= ST_KRESCALE;
  }
  const double zlo = 0.5 * k / sqrt(1.0 - 0.25 * k * k);
  const double zhi = k / sqrt(1.0 - k * k);
  int its, ok;
  double z = illinois<false>(p, zlo, zhi, D, qq, r, &its, &ok);
  if (!ok) st |= ST_NOCONV;
  double w = sqrt(1.0 + z * z);
  double rho = D / w;
  double eps = w * qq - z * r + z * z / (1.0 + w);
  double P;
  if (eps < eos_ec(p, rho)) {
    z = illinois<true>(p, 0.0, r, D, qq, r, &its, &ok);
    if (!ok) st |= ST_NOCONV;
    w = sqrt(1.0 + z * z);
    rho = D / w;
    eps = eos_ec(p, rho);
    P = eos_pc(p, rho);
    st |= ST_COLD;
  } else {
    P = eos_p(p, rho, eps);
  }
  const double Dh = D * (1.0 + eps + P / rho);
  pr[pRHO] = rho;
  pr[pEPS] = eps;
  pr[pP] = P;
  pr[pUX] = S[0] / Dh;
  pr[pUY] = S[1] / Dh;
  pr[pUZ] = S[2] / Dh;
  if (rho < p.rho_atm) {
    atmosphere(p, pr);
    st |= ST_ATM;
  }
  if (st & (ST_ATM | ST_COLD | ST_KRESCALE)) prim_to_cons(p, pr, W, gt, x, q);
  return st;
}

// ------------------------------------------------------------------ PPM (Colella & Woodward 1984)

__device__ inline double mc_slope(double am, double a0, double ap) {
  const double dl = a0 - am, dr = ap - a0;
  if (dl * dr <= 0.0) return 0.0;
  const double dc = 0.5 * (ap - am);
  const double lim = fmin(fabs(dc), fmin(2.0 * fabs(dl), 2.0 * fabs(dr)));
  return dc > 0.0 ? lim : -lim;
}

__device__ inline void ppm_limit(double a0, double &aL, double &aR) {
  if ((aR - a0) * (a0 - aL) <= 0.0) {
    aL = a0;
    aR = a0;
    return;
  }
  const double d = aR - aL;
  const double a6 = 6.0 * (a0 - 0.5 * (aL + aR));
  if (d * a6 > d * d) aL = 3.0 * a0 - 2.0 * aR;
  else if (-d * d > d * a6) aR = 3.0 * a0 - 2.0 * aL;
}

// face between c[2] and c[3] of the six cells c[0..5]
__device__ inline void ppm_pair(const double c[6], double &left, double &right) {
  const double s1 = mc_slope(c[0], c[1], c[2]);
  const double s2 = mc_slope(c[1], c[2], c[3]);
  const double s3 = mc_slope(c[2], c[3], c[4]);
  const double s4 = mc_slope(c[3], c[4], c[5]);
  const double im = c[1] + 0.5 * (c[2] - c[1]) - (s2 - s1) / 6.0;   // face j-1/2
  const double i0 = c[2] + 0.5 * (c[3] - c[2]) - (s3 - s2) / 6.0;   // face j+1/2
  const double ip = c[3] + 0.5 * (c[4] - c[3]) - (s4 - s3) / 6.0;   // face j+3/2
  double aL = im, aR = i0;
  ppm_limit(c[2], aL, aR);
  left = aR;
  double bL = i0, bR = ip;
  ppm_limit(c[3], bL, bR);
  right = bL;
}

// ------------------------------------------------------------------ tetrad-frame Riemann solver (Sec. II.C.2)

struct SRState {
  double D, S0, S1, S2, E, P, vx, lm, lp;
};

__device__ inline void sr_state(const DevParams &p, double rho, double P, double u0, double u1, double u2, SRState &s) {
  const double w = sqrt(1.0 + u0 * u0 + u1 * u1 + u2 * u2);
  const double eps = eos_eps(p, rho, P);
  const double h = 1.0 + eps + P / rho;
  const double c2 = eos_cs2(p, rho, eps, P);
  const double rhw = rho * h * w;          // rho h w^2 v = rho h w u
  s.D = rho * w;
  s.S0 = rhw * u0; s.S1 = rhw * u1; s.S2 = rhw * u2;
  s.E = rhw * w - P;
  s.P = P;
  const double v0 = u0 / w, v1 = u1 / w, v2 = u2 / w;
  s.vx = v0;
  const double vv = v0 * v0 + v1 * v1 + v2 * v2;
  double disc = c2 * (1.0 - vv) * (1.0 - vv * c2 - v0 * v0 * (1.0 - c2));
  disc = disc < 0.0 ? 0.0 : sqrt(disc);
  const double den = 1.0 / (1.0 - vv * c2);
  s.lm = (v0 * (1.0 - c2) - disc) * den;
  s.lp = (v0 * (1.0 - c2) + disc) * den;
}

__device__ inline void sr_qf(const SRState &s, double q[5], double f[5]) {
  q[0] = s.D; q[1] = s.S0; q[2] = s.S1; q[3] = s.S2; q[4] = s.E;
  f[0] = s.D * s.vx;
  f[1] = s.S0 * s.vx + s.P;
  f[2] = s.S1 * s.vx;
  f[3] = s.S2 * s.vx;
  f[4] = s.S0;            // (E + P) v^x = S_x
}

// Flux through a face normal to dir (0 = x, 1 = z).  pl/pr: rho, u_x, u_y,
// u_z, P; face metric alpha, beta^i, W, gt_ij.  out: alpha psi^6 times the
// Eulerian flux with Cartesian momentum components.  Returns 1 on a
// HLLC -> TVDLF fallback.
__device__ inline int face_flux(const DevParams &p, int dir, const double pl[5], const double pr[5], double alpha,
                                const double beta[3], double W, const Sym3 &g, double out[5]) {
  // work in a frame whose first axis is the face normal: (x,y,z) or (z,x,y)
  Sym3 m;
  double bn, uL[3], uR[3];
  if (dir == 0) {
    m = g;
    bn = beta[0];
    uL[0] = pl[1]; uL[1] = pl[2]; uL[2] = pl[3];
    uR[0] = pr[1]; uR[1] = pr[2]; uR[2] = pr[3];
  } else {
    m.xx = g.zz; m.xy = g.xz; m.xz = g.yz; m.yy = g.xx; m.yz = g.xy; m.zz = g.yy;
    bn = beta[2];
    uL[0] = pl[3]; uL[1] = pl[1]; uL[2] = pl[2];
    uR[0] = pr[3]; uR[1] = pr[1]; uR[2] = pr[2];
  }
  const Sym3 mi = s3inv(m, nullptr);
  const double Bh = rsqrt(mi.xx);                 // 1/sqrt(gt^xx)
  const double Ch = rsqrt(m.zz);                  // 1/sqrt(gt_zz)
  const double Dh = Bh * Ch;
  // tetrad components of u: e_(a)^i u_i with the contravariant legs
  //   e_x = W B (gt^xx, gt^xy, gt^xz), e_y = W D (0, gt_zz, -gt_yz), e_z = W C (0, 0, 1)
  const double tL0 = W * Bh * (mi.xx * uL[0] + mi.xy * uL[1] + mi.xz * uL[2]);
  const double tL1 = W * Dh * (m.zz * uL[1] - m.yz * uL[2]);
  const double tL2 = W * Ch * uL[2];
  const double tR0 = W * Bh * (mi.xx * uR[0] + mi.xy * uR[1] + mi.xz * uR[2]);
  const double tR1 = W * Dh * (m.zz * uR[1] - m.yz * uR[2]);
  const double tR2 = W * Ch * uR[2];
  SRState L, R;
  sr_state(p, pl[0], pl[4], tL0, tL1, tL2, L);
  sr_state(p, pr[0], pr[4], tR0, tR1, tR2, R);
  double qL[5], fL[5], qR[5], fR[5];
  sr_qf(L, qL, fL);
  sr_qf(R, qR, fR);
  const double lamL = fmin(L.lm, R.lm);
  const double lamR = fmax(L.lp, R.lp);
  const double sgxx = W * sqrt(mi.xx);
  const double vint = bn / (alpha * sgxx);

  double F[5];
  int fb = 0;
  if (p.solver == SACRA_HLLC) {
    if (lamL >= vint) {
      for (int n = 0; n < 5; ++n) F[n] = fL[n] - vint * qL[n];
    } else if (lamR <= vint) {
      for (int n = 0; n < 5; ++n) F[n] = fR[n] - vint * qR[n];
    } else {
      const double idl = 1.0 / (lamR - lamL);
      // HLL state and flux, only the components the contact speed needs
      const double Eh = (lamR * qR[4] - lamL * qL[4] + fL[4] - fR[4]) * idl;
      const double Sh = (lamR * qR[1] - lamL * qL[1] + fL[1] - fR[1]) * idl;
      const double FEh = (lamR * fL[4] - lamL * fR[4] + lamR * lamL * (qR[4] - qL[4])) * idl;
      const double FSh = (lamR * fL[1] - lamL * fR[1] + lamR * lamL * (qR[1] - qL[1])) * idl;
      const double bb = Eh + FSh;
      const double disc = bb * bb - 4.0 * FEh * Sh;
      bool bad = !(disc >= 0.0);
      double lamc = 0.0, Pc = 0.0;
      if (!bad) {
        lamc = 2.0 * Sh / (bb + sqrt(disc));     // minus root, cancellation free
        Pc = FSh - lamc * FEh;
        bad = !(lamc >= lamL && lamc <= lamR) || !(Pc > 0.0);
      }
      if (!bad) {
        const bool left = vint <= lamc;
        const SRState &K = left ? L : R;
        const double *qK = left ? qL : qR;
        const double *fK = left ? fL : fR;
        const double lamK = left ? lamL : lamR;
        const double fac = lamK - K.vx;
        const double iden = 1.0 / (lamK - lamc);
        double qs[5];
        qs[0] = K.D * fac * iden;
        qs[1] = (K.S0 * fac + Pc - K.P) * iden;
        qs[2] = K.S1 * fac * iden;
        qs[3] = K.S2 * fac * iden;
        qs[4] = (K.E * fac + Pc * lamc - K.P * K.vx) * iden;
        for (int n = 0; n < 5; ++n) {
          const double fs = fK[n] + lamK * (qs[n] - qK[n]);
          F[n] = fs - vint * qs[n];
          if (!isfinite(F[n])) bad = true;
        }
      }
      fb = bad ? 1 : 0;
    }
  }
  if (p.solver != SACRA_HLLC || fb) {
    const double cmax = fmax(fabs(lamL - vint), fabs(lamR - vint));
    for (int n = 0; n < 5; ++n)
      F[n] = 0.5 * ((fL[n] - vint * qL[n]) + (fR[n] - vint * qR[n])) - 0.5 * cmax * (qR[n] - qL[n]);
  }
  // back to the Eulerian frame with the covariant legs e_(a)_i:
  //   e_x = (B/W)(1,0,0), e_y = (D/W)(-gt^xy, gt^xx, 0), e_z = (C/W)(gt_xz, gt_yz, gt_zz)
  const double pre = alpha / (W * W * W) * sgxx;
  const double iW = 1.0 / W;
  const double S0 = iW * (Bh * F[1] - Dh * mi.xy * F[2] + Ch * m.xz * F[3]);
  const double S1 = iW * (Dh * mi.xx * F[2] + Ch * m.yz * F[3]);
  const double S2 = iW * (Ch * m.zz * F[3]);
  out[0] = pre * F[0];
  out[4] = pre * F[4];
  if (dir == 0) {
    out[1] = pre * S0; out[2] = pre * S1; out[3] = pre * S2;
  } else {  // frame axes (z, x, y)
    out[3] = pre * S0; out[1] = pre * S1; out[2] = pre * S2;
  }
  return fb;
}

}  // namespace sacra
