/*
 * Oracle (test infrastructure only): finite-difference, Kreiss-Oliger and
 * Lagrange weights, derived at start-up from their definitions (a Vandermonde
 * solve for derivatives, the Lagrange product formula for interpolation)
 * rather than typed in.  Sec. II.B.1 (6th-order central and lopsided
 * differences, 8th-order KO), Sec. II.B.2 (9-point cartoon interpolation),
 * Sec. II.C.2 (metric to faces), Sec. II.D (8th-order prolongation and
 * restriction).
 */
#include <math.h>
#include <string.h>
#include "orc.h"

double orc_c1[7], orc_c2[7], orc_lop[7], orc_ko[9], orc_face6[6];
double orc_prol8[8], orc_rest8[8];

/* Weights w_n on nodes s_n so that sum_n w_n f(s_n) = f^(deriv)(x) exactly for
   polynomials of degree < npts: sum_n w_n (s_n - x)^m = m! delta_{m,deriv}. */
void orc_fd_weights(int npts, const double *nodes, double x, int deriv, double *w) {
  double A[16][17];
  for (int m = 0; m < npts; ++m) {
    for (int n = 0; n < npts; ++n) A[m][n] = pow(nodes[n] - x, (double)m);
    double fact = 1.0;
    for (int i = 2; i <= m; ++i) fact *= i;
    A[m][npts] = (m == deriv) ? fact : 0.0;
  }
  /* Gaussian elimination with partial pivoting */
  for (int c = 0; c < npts; ++c) {
    int piv = c;
    for (int r = c + 1; r < npts; ++r)
      if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
    if (piv != c)
      for (int q = 0; q <= npts; ++q) { double t = A[c][q]; A[c][q] = A[piv][q]; A[piv][q] = t; }
    for (int r = 0; r < npts; ++r) {
      if (r == c) continue;
      double fct = A[r][c] / A[c][c];
      for (int q = c; q <= npts; ++q) A[r][q] -= fct * A[c][q];
    }
  }
  for (int n = 0; n < npts; ++n) w[n] = A[n][npts] / A[n][n];
}

/* Lagrange interpolation weights: w_n = prod_{m != n} (x - s_m)/(s_n - s_m). */
void orc_lagrange(int npts, const double *nodes, double x, double *w) {
  for (int n = 0; n < npts; ++n) {
    double v = 1.0;
    for (int m = 0; m < npts; ++m)
      if (m != n) v *= (x - nodes[m]) / (nodes[n] - nodes[m]);
    w[n] = v;
  }
}

static int inited = 0;

void orc_stencil_init(void) {
  if (inited) return;
  double s7[7] = {-3, -2, -1, 0, 1, 2, 3};
  orc_fd_weights(7, s7, 0.0, 1, orc_c1);     /* 6th-order central first derivative */
  orc_fd_weights(7, s7, 0.0, 2, orc_c2);     /* 6th-order central second derivative */
  double sl[7] = {-2, -1, 0, 1, 2, 3, 4};
  orc_fd_weights(7, sl, 0.0, 1, orc_lop);    /* lopsided, shifted one point toward +x */
  double s9[9] = {-4, -3, -2, -1, 0, 1, 2, 3, 4};
  orc_fd_weights(9, s9, 0.0, 8, orc_ko);     /* 8th difference (Delta^8 d^8) */
  double s6[6] = {-2, -1, 0, 1, 2, 3};
  orc_lagrange(6, s6, 0.5, orc_face6);       /* cell centres j-2..j+3 -> face j+1/2 */
  double s8[8] = {-3, -2, -1, 0, 1, 2, 3, 4};
  orc_lagrange(8, s8, 0.25, orc_prol8);      /* parent cells m-3..m+4 -> m + 1/4 */
  orc_lagrange(8, s8, 0.5, orc_rest8);       /* child cells 2j-4..2j+3 -> parent centre */
  inited = 1;
}
