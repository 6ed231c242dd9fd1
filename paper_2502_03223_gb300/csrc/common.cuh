// Device-side building blocks of the SACRA-2D hot path on sm_103a:
// level views, the hybrid EOS, the primitive recovery, PPM and the
// tetrad-frame HLLC/TVDLF flux (Lam & Shibata, arXiv:2502.03223, Sec. II.C).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

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

struct MlpNet;

// Cold polytropic pieces of one star beyond the first (Sec. II.C.3), in
// device memory: piece i (0-based) holds rho in [rho[i-1], rho[i]).
constexpr int kMaxPieces = 8;
struct PwpTable {
  double rho[kMaxPieces - 1], K[kMaxPieces], G[kMaxPieces], gm1[kMaxPieces], de[kMaxPieces];
  float frho[kMaxPieces - 1], fK[kMaxPieces], fG[kMaxPieces], fgm1[kMaxPieces], fde[kMaxPieces];
};

struct DevParams {
  int geometry, evolve, solver, rk, c2p_maxit, n_levels;
  int mixed;             // SACRA_MIXED_* bits: parts whose arithmetic runs in FP32 (FP64 differences and updates)
  int K_zero, gamma2;    // K == 0 (pure Gamma-law), Gamma == 2
  int hydro_outer;       // 1: level 0's outer hydro ghosts stay at the initial data
  int adiabatic;         // 1: zero temperature, P = P_cold, eps = eps_cold, energy equation discarded
  int n_pieces;          // cold pieces (1: K, Gamma; more: the table pwp)
  int bssn;              // 1: BSSN (Theta held at zero, kappa = 0)
  const PwpTable *pwp;   // device copy of the pieces when n_pieces > 1
  double c2p_zmax;       // sqrt(w_max^2 - 1): Lorentz-factor cap of the adiabatic recovery
  double ith1;           // 1 / (Gamma_th - 1)
  float fith1;
  double r_hold2;        // > 0: hydro held at U^n where x^2 + z^2 < r_hold2 (excised inner boundary)
  double K, Gamma, Gamma_th, rho_atm, w_max, c2p_tol;
  double kappa, eta_B, eps_ko, r_z4;
  double c2p_kmax;       // 2 v_max / (1 + v_max^2), v_max = sqrt(1 - 1 / w_max^2)
  // FP32 copies for the mixed-precision kernels (no conversions on the device)
  float fK, fGamma, fGm1, fGamma_th, fGth1, fkappa, feta_B, firz2, fko;
  double ko;             // -eps_KO / 256
  // learned seed of the primitive recovery (null: plain bracket) and its counters
  // [Illinois evaluations, recoveries with a seed tried, seeded brackets that held, recoveries]
  const MlpNet *mlp;
  unsigned long long *c2p_stats;
};

// a parameter in arithmetic T: the FP64 value, or its FP32 copy
template <typename T>
__host__ __device__ __forceinline__ T pv(double d, float f) {
  if constexpr (sizeof(T) == 4) return f;
  else return d;
}

// fills every field from the public parameters (host)
inline void fill_dev_params(const sacra_params *p, DevParams *d) {
  *d = DevParams{};
  d->geometry = p->geometry; d->evolve = p->evolve_spacetime; d->solver = p->solver; d->rk = p->rk;
  d->c2p_maxit = p->c2p_maxit; d->n_levels = p->n_levels; d->mixed = p->precision & SACRA_MIXED;
  d->K_zero = p->K == 0.0; d->gamma2 = p->Gamma == 2.0;
  d->K = p->K; d->Gamma = p->Gamma; d->Gamma_th = p->Gamma_th; d->rho_atm = p->rho_atm; d->w_max = p->w_max;
  d->c2p_tol = p->c2p_tol; d->kappa = p->kappa; d->eta_B = p->eta_B; d->eps_ko = p->eps_ko; d->r_z4 = p->r_z4;
  d->fK = (float)p->K; d->fGamma = (float)p->Gamma; d->fGm1 = (float)(p->Gamma - 1.0);
  d->fGamma_th = (float)p->Gamma_th; d->fGth1 = (float)(p->Gamma_th - 1.0);
  d->fkappa = (float)p->kappa; d->feta_B = (float)p->eta_B;
  d->firz2 = (float)(1.0 / (p->r_z4 * p->r_z4));
  d->fko = (float)(-p->eps_ko / 256.0);
  d->ko = -p->eps_ko / 256.0;
  const double vmax = sqrt(1.0 - 1.0 / (p->w_max * p->w_max));
  d->c2p_kmax = 2.0 * vmax / (1.0 + vmax * vmax);
  d->hydro_outer = p->hydro_outer != 0;
  d->r_hold2 = p->r_hold > 0.0 ? p->r_hold * p->r_hold : 0.0;
  d->adiabatic = p->eos_adiabatic != 0;
  d->bssn = p->bssn != 0;
  if (d->bssn) { d->kappa = 0.0; d->fkappa = 0.0f; }
  d->n_pieces = p->n_pieces > 1 ? p->n_pieces : 1;
  d->pwp = nullptr;      // set by the owner of the device copy
  d->c2p_zmax = sqrt(p->w_max * p->w_max - 1.0);
  d->ith1 = 1.0 / (p->Gamma_th - 1.0);
  d->fith1 = (float)d->ith1;
}

// The pieces' constants (host): K_(i+1) from continuity of P_cold at rho_i,
// Delta eps_(i+1) from continuity of eps_cold there, Delta eps_1 = 0.
inline void fill_pwp_table(const sacra_params *p, PwpTable *t) {
  memset(t, 0, sizeof(*t));
  const int n = p->n_pieces > 1 ? p->n_pieces : 1;
  t->K[0] = p->K; t->G[0] = p->Gamma; t->gm1[0] = p->Gamma - 1.0; t->de[0] = 0.0;
  for (int i = 1; i < n; ++i) {
    const double rt = p->pwp_rho[i - 1], g = t->G[i - 1], g2 = p->pwp_Gamma[i - 1], k = t->K[i - 1];
    t->rho[i - 1] = rt;
    t->G[i] = g2;
    t->gm1[i] = g2 - 1.0;
    t->K[i] = k * pow(rt, g - g2);
    t->de[i] = t->de[i - 1] + k * pow(rt, g - 1.0) / (g - 1.0) - t->K[i] * pow(rt, g2 - 1.0) / (g2 - 1.0);
  }
  for (int i = 0; i < kMaxPieces; ++i) {
    if (i < kMaxPieces - 1) t->frho[i] = (float)t->rho[i];
    t->fK[i] = (float)t->K[i]; t->fG[i] = (float)t->G[i]; t->fgm1[i] = (float)t->gm1[i]; t->fde[i] = (float)t->de[i];
  }
}

// One refinement level as seen by a kernel: planes of P = px * pz doubles.
struct LevF {                   // FP32 copies of the spacing constants
  float dx, dz, idx, idz, i60x, i60z, i180x, i180z, ixz;
};

struct Lev {
  int nx, nz, px, pz, rw;
  double dx, dz;
  double i60x, i60z, i180x;     // 1 / (60 dx), 1 / (60 dz), 1 / (180 dx^2)
  double i180z, ixz, idx, idz;  // 1 / (180 dz^2), 1 / (3600 dx dz), 1 / dx, 1 / dz
  LevF f;
  size_t P;
  double *un, *us, *ka, *rhs;   // NST planes each
  double *rhsq;                 // NCONS planes of the hydro right-hand side (d_t q_D .. d_t q_E)
  double *prim;                 // NPRIM planes
  int *status;
  double *fx, *fz;              // NCONS planes of face fluxes (area-weighted)
  double *freg;                 // 4 x NCONS x rw flux registers
  double *dy, *dyy;             // NMET planes of cartoon d_y, d_yy
  unsigned long long *nfb;      // HLLC -> TVDLF fallback counter
};

__host__ __device__ inline int cid(const Lev &L, int j, int k) { return (k + GH - 1) * L.px + (j + GH - 1); }

// spacing and the constants derived from it (host)
inline void set_spacing(Lev &L, double dx, double dz) {
  L.dx = dx; L.dz = dz;
  L.i60x = 1.0 / (60.0 * dx); L.i60z = 1.0 / (60.0 * dz); L.i180x = 1.0 / (180.0 * dx * dx);
  L.i180z = 1.0 / (180.0 * dz * dz); L.ixz = 1.0 / (3600.0 * dx * dz); L.idx = 1.0 / dx; L.idz = 1.0 / dz;
  L.f.dx = (float)dx; L.f.dz = (float)dz; L.f.idx = (float)(1.0 / dx); L.f.idz = (float)(1.0 / dz);
  L.f.i60x = (float)L.i60x; L.f.i60z = (float)L.i60z;
  L.f.i180x = (float)(1.0 / (180.0 * dx * dx)); L.f.i180z = (float)(1.0 / (180.0 * dz * dz));
  L.f.ixz = (float)(1.0 / (3600.0 * dx * dz));
}

// ------------------------------------------------------------------ FP64 <-> FP32 without the FP64 pipe
//
// On this part conversions between double and float issue at the FP64 rate
// (about 2 per clock per SM, like a DADD), while integer and FP32 operations
// issue some 30-60x faster.  The mixed-precision kernels therefore take FP32
// views of FP64 data with integer bit operations:
//   split_f64(u) = (hi, lo): hi = u truncated to 24 significant bits, lo = the
//   next 23 bits (u - hi - lo < 2^-46 |u|).  A difference of two nearby FP64
//   values is then (hi_a - hi_b) + (lo_a - lo_b): the hi part is exact when
//   the two are within a factor 2 (Sterbenz), so the FP32 result carries one
//   rounding, the same as rounding the exact FP64 difference.
//   f32_of(u) = hi + lo, u rounded to FP32.  f64_of(f): exact widening.
// |u| below 2^-126 flushes to zero, above 2^128 (or NaN) gives +-inf; lo
// flushes to zero below 2^-103 |u| scale.
struct F2 {
  float hi, lo;
};

__device__ __forceinline__ F2 split_f64(double u) {
  const unsigned hw = (unsigned)__double2hiint(u), lw = (unsigned)__double2loint(u);
  const unsigned sg = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7FFu);
  const int E = e - 896, Fe = e - 919;                   // FP32 exponent fields of hi and of lo's scale
  const unsigned mh = ((hw & 0xFFFFFu) << 3) | (lw >> 29);   // top 23 mantissa bits
  const unsigned ml = (lw & 0x1FFFFFFFu) >> 6;               // next 23 bits
  F2 r;
  r.hi = E <= 0 ? 0.0f : (E >= 255 ? __uint_as_float(sg | 0x7F800000u) : __uint_as_float(sg | ((unsigned)E << 23) | mh));
  // 1.ml x 2^k minus 2^k = 0.ml x 2^k: exact in FP32, normalises lo
  const unsigned lb = sg | ((unsigned)(Fe > 0 ? Fe : 1) << 23);
  r.lo = (Fe > 0 && E < 255) ? __uint_as_float(lb | ml) - __uint_as_float(lb) : 0.0f;
  return r;
}

__device__ __forceinline__ float f32_of(double u) {
  const F2 s = split_f64(u);
  return s.hi + s.lo;
}

__device__ __forceinline__ float f32_diff(const F2 &a, const F2 &b) { return (a.hi - b.hi) + (a.lo - b.lo); }

__device__ __forceinline__ double f64_of(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xFFu, sg = b & 0x80000000u, m = b & 0x7FFFFFu;
  unsigned hw, lw = m << 29;
  if (e == 0) { hw = sg; lw = 0; }                                   // zero (subnormals flushed)
  else if (e == 255) hw = sg | 0x7FF00000u | (m >> 3) | (m ? 0x80000u : 0u);
  else hw = sg | ((e + 896u) << 20) | (m >> 3);
  return __hiloint2double((int)hw, (int)lw);
}

// loads and stores of FP64 data in arithmetic T
template <typename T>
__device__ __forceinline__ T ld_as(double u) {
  if constexpr (sizeof(T) == 4) return f32_of(u);
  else return u;
}
template <typename T>
__device__ __forceinline__ double to_f64(T v) {
  if constexpr (sizeof(T) == 4) return f64_of(v);
  else return v;
}

// ------------------------------------------------------------------ small tensor helpers

template <typename T>
struct Sym3T {
  T xx, xy, xz, yy, yz, zz;
};
using Sym3 = Sym3T<double>;

template <typename T>
__device__ inline Sym3T<T> s3inv(const Sym3T<T> &g, T *detp) {
  const T cxx = g.yy * g.zz - g.yz * g.yz;
  const T cxy = g.xz * g.yz - g.xy * g.zz;
  const T cxz = g.xy * g.yz - g.xz * g.yy;
  const T det = g.xx * cxx + g.xy * cxy + g.xz * cxz;
  const T id = T(1) / det;
  Sym3T<T> r;
  r.xx = cxx * id; r.xy = cxy * id; r.xz = cxz * id;
  r.yy = (g.xx * g.zz - g.xz * g.xz) * id;
  r.yz = (g.xy * g.xz - g.xx * g.yz) * id;
  r.zz = (g.xx * g.yy - g.xy * g.xy) * id;
  if (detp) *detp = det;
  return r;
}

// a^i b^j m_ij for symmetric m
template <typename T>
__device__ inline T s3quad(const Sym3T<T> &m, const T a[3], const T b[3]) {
  return m.xx * a[0] * b[0] + m.yy * a[1] * b[1] + m.zz * a[2] * b[2]
       + m.xy * (a[0] * b[1] + a[1] * b[0]) + m.xz * (a[0] * b[2] + a[2] * b[0]) + m.yz * (a[1] * b[2] + a[2] * b[1]);
}

template <typename T>
__device__ inline void s3vec(const Sym3T<T> &m, const T a[3], T o[3]) {
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
// same way as K * pow(rho, 2).  Templated on the arithmetic type T (double,
// or float in the mixed-precision hydro); every constant goes through T(...).
// More than one cold piece: the piece holding rho from the star's table.
template <typename T>
__device__ __forceinline__ int eos_piece(const DevParams &p, T rho) {
  int i = 0;
  while (i < p.n_pieces - 1 && rho >= pv<T>(p.pwp->rho[i], p.pwp->frho[i])) ++i;
  return i;
}
template <typename T>
__device__ inline T eos_pc(const DevParams &p, T rho) {
  if (p.K_zero) return T(0);
  if (p.n_pieces > 1) {
    const int i = eos_piece(p, rho);
    return pv<T>(p.pwp->K[i], p.pwp->fK[i]) * pow(rho, pv<T>(p.pwp->G[i], p.pwp->fG[i]));
  }
  const T K = pv<T>(p.K, p.fK);
  return p.gamma2 ? K * (rho * rho) : K * pow(rho, pv<T>(p.Gamma, p.fGamma));
}
template <typename T>
__device__ inline T eos_ec(const DevParams &p, T rho) {
  if (p.K_zero) return T(0);
  if (p.n_pieces > 1) {
    const int i = eos_piece(p, rho);
    const T gm1 = pv<T>(p.pwp->gm1[i], p.pwp->fgm1[i]);
    return pv<T>(p.pwp->K[i], p.pwp->fK[i]) * pow(rho, gm1) / gm1 + pv<T>(p.pwp->de[i], p.pwp->fde[i]);
  }
  const T K = pv<T>(p.K, p.fK);
  const T gm1 = pv<T>(p.Gamma - 1.0, p.fGm1);
  return p.gamma2 ? K * rho : K * pow(rho, gm1) / gm1;
}
// Gamma of the piece holding rho
template <typename T>
__device__ inline T eos_gc(const DevParams &p, T rho) {
  if (p.n_pieces > 1) {
    const int i = eos_piece(p, rho);
    return pv<T>(p.pwp->G[i], p.pwp->fG[i]);
  }
  return pv<T>(p.Gamma, p.fGamma);
}
template <typename T>
__device__ inline T eos_p(const DevParams &p, T rho, T eps) {
  return eos_pc(p, rho) + pv<T>(p.Gamma_th - 1.0, p.fGth1) * rho * (eps - eos_ec(p, rho));
}
template <typename T>
__device__ inline T eos_eps(const DevParams &p, T rho, T P) {
  return eos_ec(p, rho) + (P - eos_pc(p, rho)) / (pv<T>(p.Gamma_th - 1.0, p.fGth1) * rho);
}
// c_s^2 rho h = Gamma P_cold + Gamma_th P_th, clamped to [0, 1)
template <typename T>
__device__ inline T eos_cs2(const DevParams &p, T rho, T eps, T P) {
  const T pc = eos_pc(p, rho);
  const T h = T(1) + eps + P / rho;
  T c2 = (eos_gc(p, rho) * pc + pv<T>(p.Gamma_th, p.fGamma_th) * (P - pc)) / (rho * h);
  if (!(c2 > T(0))) c2 = T(0);
  const T cmax = sizeof(T) == 8 ? T(1.0 - 1e-15) : T(1.0f - 1e-6f);
  if (c2 >= T(1)) c2 = cmax;
  return c2;
}

}  // namespace sacra
#include "mlp.cuh"
namespace sacra {

// ------------------------------------------------------------------ primitive <-> conserved (Eq. cons_var)

// pr: rho, u_x, u_y, u_z, P, eps; q: psi^6 (D, S_x, S_y or x S_y, S_z, E)
__device__ inline void prim_to_cons(const DevParams &p, const double pr[NPRIM], double W, const Sym3 &gt, double x,
                                    double q[NCONS]) {
  const double u[3] = {pr[pUX], pr[pUY], pr[pUZ]};
  // matter at rest (the atmosphere): w = 1 exactly, no inverse metric needed
  double w = 1.0;
  if (u[0] != 0.0 || u[1] != 0.0 || u[2] != 0.0) {
    const Sym3 gi = s3inv(gt, (double *)nullptr);
    w = sqrt(1.0 + W * W * s3quad(gi, u, u));
  }
  const double rho = pr[pRHO], P = pr[pP];
  const double rhw = rho * (1.0 + pr[pEPS] + P / rho) * w;
  const double psi6 = 1.0 / (W * W * W);
  q[0] = psi6 * rho * w;
  q[1] = psi6 * rhw * u[0];
  q[2] = psi6 * rhw * u[1] * (p.geometry == SACRA_CYLINDRICAL ? x : 1.0);
  q[3] = psi6 * rhw * u[2];
  q[4] = psi6 * (rhw * w - P);
}

// D and its reciprocal (1 / rho = w / D inside the master function)
struct C2pD {
  double v, inv;
};

// Master functions of the recovery (Sec. II.C.4, Eq. c2p_fn); COLD selects
// z - r / h_cold(rho(z)).  The thermal EOS sees eps clamped to the cold curve.
// h = (1 + eps)(1 + a), a = P / (rho (1 + eps)), is formed as 1 + eps + P / rho.
template <bool COLD>
__device__ inline double c2p_fun(const DevParams &p, double z, C2pD D, double qq, double r) {
  const double w2 = 1.0 + z * z, iw = rsqrt(w2);   // 1 / w: rho = D / w without a division
  const double w = w2 * iw;
  const double rho = D.v * iw, irho = w * D.inv;
  if (COLD) {
    const double hc = 1.0 + eos_ec(p, rho) + eos_pc(p, rho) * irho;
    return z - r / hc;
  }
  double eps = w * qq - z * r + z * z / (1.0 + w);
  const double emin = eos_ec(p, rho);
  if (eps < emin) eps = emin;
  const double P = eos_p(p, rho, eps);
  return z - r / (1.0 + eps + P * irho);
}

// Illinois bracketing iteration from the bracket [a, b] with the master
// function's values fa, fb there; *ok = 0 on no sign change or at the cap
template <bool COLD>
__device__ double illinois_from(const DevParams &p, double a, double fa, double b, double fb, C2pD D, double qq,
                                double r, int *its, int *ok) {
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

// Illinois bracketing iteration on [a, b]
template <bool COLD>
__device__ double illinois(const DevParams &p, double a, double b, C2pD D, double qq, double r, int *its, int *ok) {
  const double fa = c2p_fun<COLD>(p, a, D, qq, r), fb = c2p_fun<COLD>(p, b, D, qq, r);
  return illinois_from<COLD>(p, a, fa, b, fb, D, qq, r, its, ok);
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
// SEED: the learned seed is compiled in (and used when net is not null)
template <bool SEED = false>
__device__ inline int cons_to_prim(const DevParams &p, double q[NCONS], double W, const Sym3 &gt, double x,
                                   double pr[NPRIM], const MlpNet *net = nullptr, const Sym3 *gi_known = nullptr) {
  const Sym3 gi = gi_known ? *gi_known : s3inv(gt, (double *)nullptr);   // the caller may hold gt^-1
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
  // the recovery returns rho = D / w <= D (w >= 1, either branch), so D < rho_atm
  // ends in the atmosphere reset of Sec. II.C.4 whatever the solve gives: skip it
  if (D < p.rho_atm) {
    atmosphere(p, pr);
    prim_to_cons(p, pr, W, gt, x, q);
    return ST_ATM;
  }
  int st = 0;
  double r = sqrt(W * W * s3quad(gi, S, S)) / D;
  if (p.adiabatic) {
    // "adiabatic" EOS (Sec. III): zero temperature, the energy equation is
    // discarded: the cold recovery from D and S_i alone, the Lorentz factor
    // capped at w_max through r (z = r / h_c <= r), then E rebuilt
    if (r > p.c2p_zmax) {
      const double s = p.c2p_zmax / r;
      S[0] *= s; S[1] *= s; S[2] *= s;
      r = p.c2p_zmax;
      st |= ST_KRESCALE;
    }
    int its, ok;
    const double z = illinois<true>(p, 0.0, r, C2pD{D, 1.0 / D}, 0.0, r, &its, &ok);
    if (!ok) st |= ST_NOCONV;
    const double w = sqrt(1.0 + z * z);
    const double rho = D / w;
    const double eps = eos_ec(p, rho), P = eos_pc(p, rho);
    const double iDh = 1.0 / (D * (1.0 + eps + P / rho));
    pr[pRHO] = rho;
    pr[pEPS] = eps;
    pr[pP] = P;
    pr[pUX] = S[0] * iDh;
    pr[pUY] = S[1] * iDh;
    pr[pUZ] = S[2] * iDh;
    if (rho < p.rho_atm) {
      atmosphere(p, pr);
      st |= ST_ATM;
    }
    prim_to_cons(p, pr, W, gt, x, q);
    return st;
  }
  const C2pD Dd{D, 1.0 / D};
  const double qq = E / D - 1.0;
  double k = r / (1.0 + qq);
  const double kmax = p.c2p_kmax;
  if (k > kmax) {
    const double s = kmax / k;
    S[0] *= s; S[1] *= s; S[2] *= s;
    r *= s;
    k = kmax;
    st |= ST_KRESCALE;
  }
  const double zlo = 0.5 * k * rsqrt(1.0 - 0.25 * k * k);
  const double zhi = k * rsqrt(1.0 - k * k);
  int its, ok;
  double z = 0.0;
  bool solved = false;
  unsigned long long ev = 0, tried = 0, held = 0;
  if (SEED && net && r > 0.0 && k >= net->kmin) {
    // learned seed: P / D -> v = r / (1 + q + P / D) -> z0 = v / sqrt(1 - v^2) (FP32).  The master
    // function at z0 tells the side of the root; the bracket is [z0, z0 (1 + delta)] or
    // [z0 (1 - delta), z0] inside [zlo, zhi], and the Illinois iteration itself is unchanged
    float x[MLP_IN];
    c2p_features(p, D, qq, r, k, W, gt, gi, x);
    const float pd = exp10f(mlp_forward(net, x));
    const float v = f32_of(r) / (1.0f + f32_of(qq) + pd);
    tried = 1;
    if (v > 0.0f && v < 1.0f) {
      const float z0 = v * rsqrtf(1.0f - v * v), dl = net->delta;
      const double zs = fmin(fmax(f64_of(z0), zlo), zhi);
      const double f0 = c2p_fun<false>(p, zs, Dd, qq, r);
      double a, fa, b, fb;
      if (f0 < 0.0) {
        a = zs; fa = f0;
        b = fmin(zhi, f64_of(z0 * (1.0f + dl)));
        fb = c2p_fun<false>(p, b, Dd, qq, r);
      } else {
        b = zs; fb = f0;
        a = fmax(zlo, f64_of(z0 * (1.0f - dl)));
        fa = c2p_fun<false>(p, a, Dd, qq, r);
      }
      ev += 2;
      if (a <= b) {
        z = illinois_from<false>(p, a, fa, b, fb, Dd, qq, r, &its, &ok);
        ev += its;
        solved = ok != 0;
        held = solved ? 1 : 0;
      }
    }
  }
  if (!solved) {
    z = illinois<false>(p, zlo, zhi, Dd, qq, r, &its, &ok);
    ev += its + 2;
  }
  if (p.c2p_stats) {
    atomicAdd(p.c2p_stats + 0, ev);
    if (tried) atomicAdd(p.c2p_stats + 1, tried);
    if (held) atomicAdd(p.c2p_stats + 2, held);
    atomicAdd(p.c2p_stats + 3, 1ull);
  }
  if (!ok) st |= ST_NOCONV;
  double w = sqrt(1.0 + z * z);
  double rho = D / w;
  double eps = w * qq - z * r + z * z / (1.0 + w);
  double P;
  if (eps < eos_ec(p, rho)) {
    z = illinois<true>(p, 0.0, r, Dd, qq, r, &its, &ok);
    if (!ok) st |= ST_NOCONV;
    w = sqrt(1.0 + z * z);
    rho = D / w;
    eps = eos_ec(p, rho);
    P = eos_pc(p, rho);
    st |= ST_COLD;
  } else {
    P = eos_p(p, rho, eps);
  }
  const double iDh = 1.0 / (D * (1.0 + eps + P / rho));
  pr[pRHO] = rho;
  pr[pEPS] = eps;
  pr[pP] = P;
  pr[pUX] = S[0] * iDh;
  pr[pUY] = S[1] * iDh;
  pr[pUZ] = S[2] * iDh;
  if (rho < p.rho_atm) {
    atmosphere(p, pr);
    st |= ST_ATM;
  }
  if (st & (ST_ATM | ST_COLD | ST_KRESCALE)) prim_to_cons(p, pr, W, gt, x, q);
  return st;
}

// ------------------------------------------------------------------ PPM (Colella & Woodward 1984)

// The reconstruction is written with explicitly rounded operations (no fused
// multiply-add chosen by the compiler), so that the per-face form and the
// shared-memory staged form of the flux kernels give the same values.
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }

template <typename T>
__device__ inline T mc_slope(T am, T a0, T ap) {
  const T dl = rn_sub(a0, am), dr = rn_sub(ap, a0);
  if (rn_mul(dl, dr) <= T(0)) return T(0);
  const T dc = rn_mul(T(0.5), rn_sub(ap, am));
  const T lim = fmin(fabs(dc), fmin(T(2) * fabs(dl), T(2) * fabs(dr)));
  return dc > T(0) ? lim : -lim;
}

template <typename T>
__device__ inline void ppm_limit(T a0, T &aL, T &aR) {
  if (rn_mul(rn_sub(aR, a0), rn_sub(a0, aL)) <= T(0)) {
    aL = a0;
    aR = a0;
    return;
  }
  const T d = rn_sub(aR, aL);
  const T a6 = rn_mul(T(6), rn_sub(a0, rn_mul(T(0.5), rn_add(aL, aR))));
  const T dd = rn_mul(d, d), da6 = rn_mul(d, a6);
  if (da6 > dd) aL = rn_sub(rn_mul(T(3), a0), T(2) * aR);
  else if (-dd > da6) aR = rn_sub(rn_mul(T(3), a0), T(2) * aL);
}

// interface value between cells a (slope sa) and b (slope sb), 4th order
template <typename T>
__device__ __forceinline__ T ppm_iface(T a, T b, T sa, T sb) {
  return rn_sub(rn_add(a, rn_mul(T(0.5), rn_sub(b, a))), rn_mul(rn_sub(sb, sa), T(1.0 / 6.0)));
}

// face between c[2] and c[3] of the six cells c[0..5]
template <typename T>
__device__ inline void ppm_pair(const T c[6], T &left, T &right) {
  const T s1 = mc_slope(c[0], c[1], c[2]);
  const T s2 = mc_slope(c[1], c[2], c[3]);
  const T s3 = mc_slope(c[2], c[3], c[4]);
  const T s4 = mc_slope(c[3], c[4], c[5]);
  const T im = ppm_iface(c[1], c[2], s1, s2);   // face j-1/2
  const T i0 = ppm_iface(c[2], c[3], s2, s3);   // face j+1/2
  const T ip = ppm_iface(c[3], c[4], s3, s4);   // face j+3/2
  T aL = im, aR = i0;
  ppm_limit(c[2], aL, aR);
  left = aR;
  T bL = i0, bR = ip;
  ppm_limit(c[3], bL, bR);
  right = bL;
}

// ------------------------------------------------------------------ tetrad-frame Riemann solver (Sec. II.C.2)

template <typename T>
struct SRState {
  T D, S0, S1, S2, E, P, vx, lm, lp;
};

// State of one side in the tetrad frame.  P is the pressure, Poff the value
// carried in the fluxes: P itself, or P minus a face reference pressure in
// the mixed-precision form (see face_flux).
template <typename T>
__device__ inline void sr_state(const DevParams &p, T rho, T P, T Poff, T u0, T u1, T u2, SRState<T> &s) {
  if (p.adiabatic) {            // zero temperature at the face too
    const T Pc = eos_pc(p, rho);
    Poff += Pc - P;
    P = Pc;
  }
  // the EOS quantities of eos_eps and eos_cs2 with one reciprocal of rho and of w
  const T w = sqrt(T(1) + u0 * u0 + u1 * u1 + u2 * u2);
  const T iw = T(1) / w, irho = T(1) / rho;
  const T pc = eos_pc(p, rho);
  const T eps = eos_ec(p, rho) + (P - pc) * irho * pv<T>(p.ith1, p.fith1);
  const T h = T(1) + eps + P * irho;
  T c2 = (eos_gc(p, rho) * pc + pv<T>(p.Gamma_th, p.fGamma_th) * (P - pc)) * irho / h;
  if (!(c2 > T(0))) c2 = T(0);
  if (c2 >= T(1)) c2 = sizeof(T) == 8 ? T(1.0 - 1e-15) : T(1.0f - 1e-6f);
  const T rhw = rho * h * w;          // rho h w^2 v = rho h w u
  s.D = rho * w;
  s.S0 = rhw * u0; s.S1 = rhw * u1; s.S2 = rhw * u2;
  s.E = rhw * w - P;
  s.P = Poff;
  const T v0 = u0 * iw, v1 = u1 * iw, v2 = u2 * iw;
  s.vx = v0;
  const T vv = v0 * v0 + v1 * v1 + v2 * v2;
  T disc = c2 * (T(1) - vv) * (T(1) - vv * c2 - v0 * v0 * (T(1) - c2));
  disc = disc < T(0) ? T(0) : sqrt(disc);
  const T den = T(1) / (T(1) - vv * c2);
  s.lm = (v0 * (T(1) - c2) - disc) * den;
  s.lp = (v0 * (T(1) - c2) + disc) * den;
}

template <typename T>
__device__ inline void sr_qf(const SRState<T> &s, T q[5], T f[5]) {
  q[0] = s.D; q[1] = s.S0; q[2] = s.S1; q[3] = s.S2; q[4] = s.E;
  f[0] = s.D * s.vx;
  f[1] = s.S0 * s.vx + s.P;
  f[2] = s.S1 * s.vx;
  f[3] = s.S2 * s.vx;
  f[4] = s.S0;            // (E + P) v^x = S_x
}

// Flux through a face normal to dir (0 = x, 1 = z) in arithmetic T.  pl/pr:
// rho, u_x, u_y, u_z, P - pref; face metric alpha, beta^i, W, gt_ij.  out:
// alpha psi^6 times the Eulerian flux with Cartesian momentum components,
// except that the normal momentum flux lacks alpha W^-3 pref.  Returns 1 on a
// HLLC -> TVDLF fallback.
//
// FP64 (pref = 0): the solver as written in Sec. II.C.2.  FP32 (mixed
// precision): the same algebra arranged so that rounding scales with what is
// small in a nearly static flow, not with rho or P: the pressure is carried as
// an offset from a face reference pref (which the caller adds back in FP64),
// and the HLLC star states enter as increments q* - q_K, formed from
// (lambda_c - v_K) and (P_c - P_K) instead of by subtracting two O(rho)
// numbers.
template <typename T>
__device__ inline int face_flux(const DevParams &p, int dir, const T pl[5], const T pr[5], T alpha, const T beta[3],
                                T W, const Sym3T<T> &g, T out[5], T pref = T(0)) {
  constexpr bool kDelta = sizeof(T) == 4;
  // work in a frame whose first axis is the face normal: (x,y,z) or (z,x,y)
  Sym3T<T> m;
  T bn, uL[3], uR[3];
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
  const Sym3T<T> mi = s3inv(m, (T *)nullptr);
  const T Bh = rsqrt(mi.xx);                 // 1/sqrt(gt^xx)
  const T Ch = rsqrt(m.zz);                  // 1/sqrt(gt_zz)
  const T Dh = Bh * Ch;
  // tetrad components of u: e_(a)^i u_i with the contravariant legs
  //   e_x = W B (gt^xx, gt^xy, gt^xz), e_y = W D (0, gt_zz, -gt_yz), e_z = W C (0, 0, 1)
  const T tL0 = W * Bh * (mi.xx * uL[0] + mi.xy * uL[1] + mi.xz * uL[2]);
  const T tL1 = W * Dh * (m.zz * uL[1] - m.yz * uL[2]);
  const T tL2 = W * Ch * uL[2];
  // equal states on both sides (uniform matter, the atmosphere): the Riemann
  // fan is the state itself for any solver, so the flux is f - v_int q
  const bool same = pl[0] == pr[0] && pl[1] == pr[1] && pl[2] == pr[2] && pl[3] == pr[3] && pl[4] == pr[4];
  SRState<T> L, R;
  sr_state(p, pl[0], kDelta ? pl[4] + pref : pl[4], pl[4], tL0, tL1, tL2, L);
  T qL[5], fL[5], qR[5], fR[5];
  sr_qf(L, qL, fL);
  if (same) {
    R = L;
    for (int n = 0; n < 5; ++n) { qR[n] = qL[n]; fR[n] = fL[n]; }
  } else {
    const T tR0 = W * Bh * (mi.xx * uR[0] + mi.xy * uR[1] + mi.xz * uR[2]);
    const T tR1 = W * Dh * (m.zz * uR[1] - m.yz * uR[2]);
    const T tR2 = W * Ch * uR[2];
    sr_state(p, pr[0], kDelta ? pr[4] + pref : pr[4], pr[4], tR0, tR1, tR2, R);
    sr_qf(R, qR, fR);
  }
  const T lamL = fmin(L.lm, R.lm);
  const T lamR = fmax(L.lp, R.lp);
  const T sgxx = W * (mi.xx * Bh);           // W sqrt(gt^xx)
  const T vint = bn / (alpha * sgxx);

  T F[5];
  int fb = 0;
  if (same) {
    for (int n = 0; n < 5; ++n) F[n] = fL[n] - vint * qL[n];
  } else if (p.solver == SACRA_HLLC) {
    if (lamL >= vint) {
      for (int n = 0; n < 5; ++n) F[n] = fL[n] - vint * qL[n];
    } else if (lamR <= vint) {
      for (int n = 0; n < 5; ++n) F[n] = fR[n] - vint * qR[n];
    } else {
      const T idl = T(1) / (lamR - lamL);
      // HLL state and flux, only the components the contact speed needs
      const T Eh = (lamR * qR[4] - lamL * qL[4] + fL[4] - fR[4]) * idl;
      const T Sh = (lamR * qR[1] - lamL * qL[1] + fL[1] - fR[1]) * idl;
      const T FEh = (lamR * fL[4] - lamL * fR[4] + lamR * lamL * (qR[4] - qL[4])) * idl;
      const T FSh = (lamR * fL[1] - lamL * fR[1] + lamR * lamL * (qR[1] - qL[1])) * idl;
      const T bb = Eh + (kDelta ? FSh + pref : FSh);   // FSh (and Pc) are offset by pref in the FP32 form
      const T disc = bb * bb - T(4) * FEh * Sh;
      bool bad = !(disc >= T(0));
      T lamc = T(0), Pc = T(0);
      if (!bad) {
        lamc = T(2) * Sh / (bb + sqrt(disc));     // minus root, cancellation free
        Pc = FSh - lamc * FEh;
        bad = !(lamc >= lamL && lamc <= lamR) || !((kDelta ? Pc + pref : Pc) > T(0));
      }
      if (!bad) {
        const bool left = vint <= lamc;
        const SRState<T> &K = left ? L : R;
        const T *qK = left ? qL : qR;
        const T *fK = left ? fL : fR;
        const T lamK = left ? lamL : lamR;
        const T iden = T(1) / (lamK - lamc);
        if constexpr (kDelta) {
          // q* - q_K = [(lambda_c - v_K) q_K + (P_c - P_K) (0, 1, 0, 0, lambda_c)
          //             + P_K (lambda_c - v_K) (0, 0, 0, 0, 1)] / (lambda_K - lambda_c)
          const T dv = (lamc - K.vx) * iden;
          const T dP = (Pc - K.P) * iden;
          T dq[5];
          dq[0] = K.D * dv;
          dq[1] = K.S0 * dv + dP;
          dq[2] = K.S1 * dv;
          dq[3] = K.S2 * dv;
          dq[4] = (K.E + (K.P + pref)) * dv + dP * lamc;
          for (int n = 0; n < 5; ++n) {
            F[n] = fK[n] + lamK * dq[n] - vint * (qK[n] + dq[n]);
            if (!isfinite(F[n])) bad = true;
          }
        } else {
          const T fac = lamK - K.vx;
          T qs[5];
          qs[0] = K.D * fac * iden;
          qs[1] = (K.S0 * fac + Pc - K.P) * iden;
          qs[2] = K.S1 * fac * iden;
          qs[3] = K.S2 * fac * iden;
          qs[4] = (K.E * fac + Pc * lamc - K.P * K.vx) * iden;
          for (int n = 0; n < 5; ++n) {
            const T fs = fK[n] + lamK * (qs[n] - qK[n]);
            F[n] = fs - vint * qs[n];
            if (!isfinite(F[n])) bad = true;
          }
        }
      }
      fb = bad ? 1 : 0;
    }
  }
  if (!same && (p.solver != SACRA_HLLC || fb)) {
    const T cmax = fmax(fabs(lamL - vint), fabs(lamR - vint));
    for (int n = 0; n < 5; ++n)
      F[n] = T(0.5) * ((fL[n] - vint * qL[n]) + (fR[n] - vint * qR[n])) - T(0.5) * cmax * (qR[n] - qL[n]);
  }
  // back to the Eulerian frame with the covariant legs e_(a)_i:
  //   e_x = (B/W)(1,0,0), e_y = (D/W)(-gt^xy, gt^xx, 0), e_z = (C/W)(gt_xz, gt_yz, gt_zz)
  const T iW = T(1) / W;
  const T pre = alpha * (iW * iW * iW) * sgxx;
  const T S0 = iW * (Bh * F[1] - Dh * mi.xy * F[2] + Ch * m.xz * F[3]);
  const T S1 = iW * (Dh * mi.xx * F[2] + Ch * m.yz * F[3]);
  const T S2 = iW * (Ch * m.zz * F[3]);
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
