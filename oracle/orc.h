/*
 * SACRA-2D reference oracle: internal declarations.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, FP64 CPU restatement of
 * the method of Lam & Shibata, "SACRA-2D" (arXiv:2502.03223).  It shares no
 * code, header, table or constant with the CUDA library under
 * paper_2502_03223_gb300/; only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may call it.
 *
 * Conventions (the oracle's own):
 *   level arrays are padded, G = 8 ghost/buffer cells on every side,
 *   cell (j,k) with j in [-7, nx+8] (paper's index, interior [1, nx]) is stored
 *   at (k + 7) * px + (j + 7), px = nx + 16, pz = nz + 16.
 */
#ifndef SACRA_ORACLE_H
#define SACRA_ORACLE_H

#include <stddef.h>

#define ORC_G 8
#define ORC_MAXL 12

/* metric fields (Sec. II.B.1): W, h_ij, At_ij, Khat, Gt^i, Theta, alpha, beta^i, B^i */
enum {
  O_W = 0, O_HXX, O_HXY, O_HXZ, O_HYY, O_HYZ, O_HZZ,
  O_AXX, O_AXY, O_AXZ, O_AYY, O_AYZ, O_AZZ,
  O_KH, O_GX, O_GY, O_GZ, O_TH, O_AL, O_BX, O_BY, O_BZ, O_BBX, O_BBY, O_BBZ,
  O_NMET
};
/* conserved fields (Eq. cons_var): q_D, q_Sx, q_Sy (q_Sphi = x q_Sy in cylindrical geometry), q_Sz, q_E */
enum { O_QD = 0, O_QSX, O_QSY, O_QSZ, O_QE, O_NCONS };
#define O_NSTATE (O_NMET + O_NCONS)
/* primitive fields: rho, u_x, u_y, u_z (covariant), P, eps */
enum { O_RHO = 0, O_UX, O_UY, O_UZ, O_P, O_EPS, O_NPRIM };

/* status bits of the primitive recovery (per cell) */
#define O_ST_NOCONV  1
#define O_ST_COLD    2
#define O_ST_ATM     4
#define O_ST_KRESCALE 8
#define O_ST_BAD     16

typedef struct {
  int n_levels;          /* L */
  int nx, nz;            /* cells per level in x and z (N x N for FMR) */
  int geometry;          /* 0: planar slab (Cartesian FV), 1: cylindrical (x = varpi) with cartoon */
  int evolve_spacetime;  /* 0: metric frozen (Cowling / flat) */
  int solver;            /* 0: HLLC with TVDLF fallback, 1: TVDLF */
  int rk;                /* 0: classical RK4, 1: SSP-RK3 */
  int c2p_maxit;
  int subcycle_from;     /* 0: all levels share one dt (lockstep); K >= 1: levels >= K take dt / 2 of their parent */
  int hydro_outer;       /* hydro at the outer boundary: 0 zero-gradient copy, 1 held at the initial data */
  int eos_adiabatic;     /* 1: zero temperature, P = P_cold, eps = eps_cold, energy equation discarded */
  int n_pieces;          /* cold polytropic pieces (0 or 1: the single piece K, Gamma) */
  int bssn;              /* 1: BSSN (Theta held at zero, kappa = 0) instead of Z4c */
  double dx0, dz0;       /* spacing of level 0 */
  double kappa, eta_B, eps_ko, r_z4;
  double K, Gamma, Gamma_th;
  double rho_atm, w_max, c2p_tol;
  double r_hold;         /* > 0: hydro held at U^n inside x^2 + z^2 < r_hold^2 (excised inner boundary) */
  double pwp_rho[7];     /* transition densities rho_1 < ... < rho_(n-1) */
  double pwp_Gamma[7];   /* Gamma_2 .. Gamma_n (piece 1: K, Gamma) */
} orc_params;

typedef struct {
  int nx, nz, px, pz;
  double dx, dz;
  double *un[O_NSTATE];   /* state at the start of the step */
  double *us[O_NSTATE];   /* stage state */
  double *ka[O_NSTATE];   /* RK4 accumulator */
  double *rhs[O_NSTATE];  /* right-hand side of the current stage */
  double *prim[O_NPRIM];
  unsigned char *status;
  double *fx[O_NCONS];    /* x-face fluxes, face j+1/2 stored at cell j */
  double *fz[O_NCONS];    /* z-face fluxes, face k+1/2 stored at cell k */
  /* flux registers, RK-weighted sums over the stages of one step:
     0: x-face nx/2+1/2, 1: x-face nx+1/2 (indexed by k), 2: z-face nz/2+1/2, 3: z-face nz+1/2 (indexed by j) */
  double *freg[4][O_NCONS];
  /* Berger-Oliger sub-cycling (Sec. II.D): this level's state and primitives at
     t^{n-1} and its primitives at t^n (time slices for a sub-cycled child), and
     its data interpolated to a stage time of its sub-cycled child */
  double *uold[O_NSTATE];
  double *pold[O_NPRIM], *pnow[O_NPRIM];
  double *ut[O_NMET], *pt[O_NPRIM];
  int have_old;
  double wpar;            /* weight of this level's parent-boundary flux registers: dt_l / dt_(l-1) */
} orc_level;

typedef struct {
  orc_params p;
  orc_level lv[ORC_MAXL];
  double dt_step;
  int n_fallback;         /* HLLC -> TVDLF fallbacks counted since creation */
} orc_ctx;

static inline int oidx(const orc_level *L, int j, int k) { return (k + ORC_G - 1) * L->px + (j + ORC_G - 1); }

/* ---- eos_c2p.c ---- */
double orc_eos_pcold(const orc_params *p, double rho);
double orc_eos_ecold(const orc_params *p, double rho);
double orc_eos_press(const orc_params *p, double rho, double eps);
double orc_eos_eps(const orc_params *p, double rho, double press);
double orc_eos_cs2(const orc_params *p, double rho, double eps, double press);
double orc_eos_gamma_cold(const orc_params *p, double rho);
void orc_inv3(const double g[6], double gi[6], double *det);
void orc_prim2cons(const orc_params *p, const double pr[O_NPRIM], double W, const double h[6], double x, double q[O_NCONS]);
int orc_con2prim(const orc_params *p, double q[O_NCONS], double W, const double h[6], double x, double pr[O_NPRIM], int *iters);

/* ---- riemann.c ---- */
void orc_ppm_face(const double a[6], double *left, double *right);
int orc_riemann_flux(const orc_params *p, int dir, const double pl[5], const double prr[5],
                     double alpha, const double beta[3], double W, const double h[6], double f[O_NCONS]);

/* ---- stencil.c ---- */
void orc_fd_weights(int npts, const double *nodes, double x, int deriv, double *w);
void orc_lagrange(int npts, const double *nodes, double x, double *w);
extern double orc_c1[7], orc_c2[7], orc_lop[7], orc_ko[9], orc_face6[6];
extern double orc_prol8[8], orc_rest8[8];
void orc_stencil_init(void);

/* ---- z4c.c ---- */
void orc_z4c_point(const orc_params *p, const double Q[O_NMET], const double dQ[O_NMET][3],
                   const double ddQ[O_NMET][6], const double adv[O_NMET], double E,
                   const double Si[3], const double Sij[6], double fz, double rhs[O_NMET]);
void orc_constraints_point(const double Q[O_NMET], const double dQ[O_NMET][3], const double ddQ[O_NMET][6],
                           double E, const double Si[3], double *H, double M[3]);
void orc_ricci_point(const double Q[O_NMET], const double dQ[O_NMET][3], const double ddQ[O_NMET][6], double Rij[6]);
void orc_cartoon_dy(const orc_ctx *c, int l, double **U, double **dy, double **dyy);
void orc_cartoon_dy_mask(const orc_ctx *c, int l, double **U, double **dy, double **dyy, const int *need);
void orc_derivs_cell(const orc_ctx *c, int l, double **U, double **dy, double **dyy, int j, int k,
                     double Q[O_NMET], double dQ[O_NMET][3], double ddQ[O_NMET][6], double adv[O_NMET]);
void orc_derivs_cell_mask(const orc_ctx *c, int l, double **U, double **dy, double **dyy, int j, int k,
                          const int *need1, const int *need2, double Q[O_NMET], double dQ[O_NMET][3],
                          double ddQ[O_NMET][6], double adv[O_NMET]);
void orc_ko_cell(const orc_ctx *c, int l, double **U, int j, int k, double ko[O_NMET]);
void orc_matter_point(const orc_params *p, const double pr[O_NPRIM], double W, const double h[6],
                      double *E, double Si[3], double Sij[6]);
int orc_field_parity_x(int f);
int orc_field_parity_z(int f);
int orc_prim_parity_x(int f);
int orc_prim_parity_z(int f);

/* ---- grid.c ---- */
void orc_hydro_source(const orc_params *p, const double pr[O_NPRIM], double al, double betay, double W,
                      const double h[6], const double A[6], double K, const double dal[2], const double db[2][3],
                      const double dW[2], const double dh[2][6], double x, double src[O_NCONS]);
orc_ctx *orc_create(const orc_params *p);
void orc_destroy(orc_ctx *c);

#endif
