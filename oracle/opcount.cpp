// Op-counting build of the oracle (test infrastructure only).
//
// The oracle's own C sources are compiled here as C++ with `double` replaced
// by a scalar that counts floating-point operations (add/sub, mul, div, sqrt
// and transcendental calls each count 1; comparisons and fabs count 0).  A
// small TOV hierarchy is set up and one RK stage is taken phase by phase, so
// that the count of each phase per cell (or face) is the operation count of
// the plain restatement of the method (its loops as written, zero-weight taps
// included).  Output: one JSON object.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

namespace oc {
struct Counts {
  long long add = 0, mul = 0, div = 0, sqr = 0, fn = 0;
  long long total() const { return add + mul + div + sqr + fn; }
};
static Counts g;

struct Real {
  double v;
  Real() : v(0.0) {}
  Real(double x) : v(x) {}
  explicit operator int() const { return (int)v; }
  explicit operator unsigned char() const { return (unsigned char)v; }
  Real operator-() const { return Real(-v); }
  Real &operator+=(const Real &o) { ++g.add; v += o.v; return *this; }
  Real &operator-=(const Real &o) { ++g.add; v -= o.v; return *this; }
  Real &operator*=(const Real &o) { ++g.mul; v *= o.v; return *this; }
  Real &operator/=(const Real &o) { ++g.div; v /= o.v; return *this; }
};
inline Real operator+(const Real &a, const Real &b) { ++g.add; return Real(a.v + b.v); }
inline Real operator-(const Real &a, const Real &b) { ++g.add; return Real(a.v - b.v); }
inline Real operator*(const Real &a, const Real &b) { ++g.mul; return Real(a.v * b.v); }
inline Real operator/(const Real &a, const Real &b) { ++g.div; return Real(a.v / b.v); }
inline bool operator<(const Real &a, const Real &b) { return a.v < b.v; }
inline bool operator>(const Real &a, const Real &b) { return a.v > b.v; }
inline bool operator<=(const Real &a, const Real &b) { return a.v <= b.v; }
inline bool operator>=(const Real &a, const Real &b) { return a.v >= b.v; }
inline bool operator==(const Real &a, const Real &b) { return a.v == b.v; }
inline bool operator!=(const Real &a, const Real &b) { return a.v != b.v; }
inline Real sqrt(const Real &a) { ++g.sqr; return Real(std::sqrt(a.v)); }
inline Real pow(const Real &a, const Real &b) { ++g.fn; return Real(std::pow(a.v, b.v)); }
inline Real exp(const Real &a) { ++g.fn; return Real(std::exp(a.v)); }
inline Real fabs(const Real &a) { return Real(std::fabs(a.v)); }
inline Real floor(const Real &a) { return Real(std::floor(a.v)); }
inline bool isfinite(const Real &a) { return std::isfinite(a.v); }
}  // namespace oc

using oc::Real;
using oc::sqrt;
using oc::pow;
using oc::exp;
using oc::fabs;
using oc::floor;
using oc::isfinite;

#define double Real
#include "eos_c2p.c"
#include "stencil.c"
#include "riemann.c"
#include "z4c.c"
#include "grid.c"
#undef double

// ------------------------------------------------------------------ driver

static Real *load_planes(const char *path, size_t n) {
  FILE *f = fopen(path, "rb");
  if (!f) return nullptr;
  Real *a = (Real *)calloc(n, sizeof(Real));
  for (size_t i = 0; i < n; ++i) {
    double v;
    if (fread(&v, sizeof(double), 1, f) != 1) { fclose(f); free(a); return nullptr; }
    a[i] = Real(v);
  }
  fclose(f);
  return a;
}

// argv: n_levels N dx0 K Gamma Gamma_th rho_atm kappa eta_B r_z4 file_level0 [file_level1 ...]
int main(int argc, char **argv) {
  if (argc < 12) { fprintf(stderr, "usage\n"); return 2; }
  orc_params p;
  memset(&p, 0, sizeof(p));
  p.n_levels = atoi(argv[1]);
  p.nx = p.nz = atoi(argv[2]);
  p.geometry = 1; p.evolve_spacetime = 1; p.solver = 0; p.rk = 0; p.c2p_maxit = 100;
  p.dx0 = p.dz0 = Real(atof(argv[3]));
  p.K = Real(atof(argv[4])); p.Gamma = Real(atof(argv[5])); p.Gamma_th = Real(atof(argv[6]));
  p.rho_atm = Real(atof(argv[7])); p.kappa = Real(atof(argv[8])); p.eta_B = Real(atof(argv[9]));
  p.r_z4 = Real(atof(argv[10])); p.eps_ko = Real(0.5); p.w_max = Real(100.0); p.c2p_tol = Real(1e-12);
  orc_ctx *c = orc_create(&p);
  const size_t np = (size_t)(p.nx + 16) * (p.nz + 16);
  for (int l = 0; l < p.n_levels; ++l) {
    Real *d = load_planes(argv[11 + l], 30 * np);
    if (!d) { fprintf(stderr, "bad data file\n"); return 2; }
    orc_set_level(c, l, 0, d);
    free(d);
  }
  orc_fill(c, 0, Real(0.1));
  // one refined level is counted (level 1 if present): region [1, N] x [1, N]
  const int l = p.n_levels > 1 ? 1 : 0;
  orc_level *L = &c->lv[l];
  Real **U = L->un;
  const int N = p.nx;
  const long long cells = (long long)N * N;
  oc::Counts base;

  // hydro faces: PPM + face metric + tetrad HLLC/TVDLF, per x-face
  oc::g = base;
  long long nfaces = 0;
  for (int k = 1; k <= N; ++k)
    for (int j = 0; j <= N; ++j) {
      Real pl[5], prr[5], al, be[3], W, h[6], f[O_NCONS];
      face_prims(L, j, k, 0, pl, prr);
      face_metric(L, U, j, k, 0, &al, be, &W, h);
      orc_riemann_flux(&c->p, 0, pl, prr, al, be, W, h, f);
      ++nfaces;
    }
  const double face_flops = (double)oc::g.total() / nfaces;
  // hydro divergence + sources, per cell (faces precomputed by hydro_rhs)
  hydro_rhs(c, l, 0, U, N, N);
  oc::g = base;
  {
    // re-run only the cell loop: the face loops are counted above, so count
    // the whole hydro_rhs and subtract the face part of both directions
    hydro_rhs(c, l, 0, U, N, N);
  }
  const double hydro_all = (double)oc::g.total();
  long long nzf = (long long)N * (N + 1);
  const double div_flops = (hydro_all - face_flops * (nfaces + nzf)) / cells;
  // the derivatives the right-hand side needs: first derivatives of W, h_ij,
  // Khat, Gt^i, Theta, alpha, beta^i; second derivatives of W, h_ij, alpha,
  // beta^i; planes of every field whose d_y or d_yy enters (all but the
  // scalars Khat and Theta, whose y-derivatives vanish)
  int need1[O_NMET] = {0}, need2[O_NMET] = {0}, needp[O_NMET];
  const int f1[] = {O_W, O_HXX, O_HXY, O_HXZ, O_HYY, O_HYZ, O_HZZ, O_KH, O_GX, O_GY, O_GZ, O_TH, O_AL, O_BX, O_BY, O_BZ};
  const int f2[] = {O_W, O_HXX, O_HXY, O_HXZ, O_HYY, O_HYZ, O_HZZ, O_AL, O_BX, O_BY, O_BZ};
  for (int f : f1) need1[f] = 1;
  for (int f : f2) need2[f] = 1;
  for (int f = 0; f < O_NMET; ++f) needp[f] = (f == O_KH || f == O_TH) ? 0 : 1;
  // cartoon planes (d_y, d_yy), per cell of the computed patch
  size_t n = np;
  Real *dy[O_NMET], *dyy[O_NMET];
  for (int f = 0; f < O_NMET; ++f) { dy[f] = (Real *)calloc(n, sizeof(Real)); dyy[f] = (Real *)calloc(n, sizeof(Real)); }
  oc::g = base;
  orc_cartoon_dy_mask(c, l, U, dy, dyy, needp);
  const long long cart_cells = (long long)(N + 7) * (N + 10);
  const double cart_flops = (double)oc::g.total() / cart_cells;
  // derivatives + advection + KO, per cell
  oc::g = base;
  for (int k = 1; k <= N; ++k)
    for (int j = 1; j <= N; ++j) {
      Real Q[O_NMET], dQ[O_NMET][3], ddQ[O_NMET][6], adv[O_NMET], ko[O_NMET];
      orc_derivs_cell_mask(c, l, U, dy, dyy, j, k, need1, need2, Q, dQ, ddQ, adv);
      orc_ko_cell(c, l, U, j, k, ko);
    }
  const double deriv_flops = (double)oc::g.total() / cells;
  // pointwise Z4c (matter, damping factor, RHS), per cell
  oc::g = base;
  for (int k = 1; k <= N; ++k)
    for (int j = 1; j <= N; ++j) {
      int id = oidx(L, j, k);
      Real Q[O_NMET], dQ[O_NMET][3], ddQ[O_NMET][6], adv[O_NMET], r[O_NMET];
      oc::Counts save = oc::g;
      orc_derivs_cell(c, l, U, dy, dyy, j, k, Q, dQ, ddQ, adv);
      oc::g = save;
      Real pr[O_NPRIM], E, Si[3], Sij[6], h[6];
      for (int f = 0; f < O_NPRIM; ++f) pr[f] = L->prim[f][id];
      cell_h(U, id, h);
      orc_matter_point(&c->p, pr, Q[O_W], h, &E, Si, Sij);
      Real x = xc(L, j), z = zc(L, k);
      Real fz = exp(-(x * x + z * z) / (c->p.r_z4 * c->p.r_z4));
      orc_z4c_point(&c->p, Q, dQ, ddQ, adv, E, Si, Sij, fz, r);
    }
  const double point_flops = (double)oc::g.total() / cells;
  // RK combination (RK4 stage 0: 2 ops per field), algebraic constraints, recovery, per cell
  oc::g = base;
  long long c2p_iters = 0;
  for (int k = 1; k <= N; ++k)
    for (int j = 1; j <= N; ++j) {
      int id = oidx(L, j, k);
      for (int f = 0; f < O_NSTATE; ++f) {
        Real kk = L->rhs[f][id];
        L->ka[f][id] = Real(1.0 / 6.0) * kk;
        L->us[f][id] = L->un[f][id] + Real(0.5) * Real(0.1) * kk;
      }
      enforce(L->us, id);
      Real q[O_NCONS], pr[O_NPRIM], h[6];
      for (int f = 0; f < O_NCONS; ++f) q[f] = L->us[O_NMET + f][id];
      cell_h(L->us, id, h);
      int it;
      orc_con2prim(&c->p, q, L->us[O_W][id], h, xc(L, j), pr, &it);
      c2p_iters += it;
    }
  const double update_flops = (double)oc::g.total() / cells;
  printf("{\"level\": %d, \"N\": %d, \"flux_face\": %.1f, \"hydro_div_cell\": %.1f, \"cartoon_cell\": %.1f, "
         "\"z4c_derivs_cell\": %.1f, \"z4c_point_cell\": %.1f, \"rk_update_cell\": %.1f, \"c2p_iters_mean\": %.3f}\n",
         l, N, face_flops, div_flops, cart_flops, deriv_flops, point_flops, update_flops,
         (double)c2p_iters / cells);
  return 0;
}
