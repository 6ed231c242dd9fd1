// Host-side launchers of the sm_103a kernels (one stream, no allocation).
#pragma once

#include "common.cuh"

namespace sacra {

// interpolation weights computed on the host and kept in constant memory
struct GridWeights {
  double prol[8];        // 8 parent cells m-3..m+4 -> child at m + 1/4 (reverse for m - 1/4)
  double rest_c[8];      // 8 child cells 2j-4..2j+3 -> parent centre (child index 2j - 1/2)
  double rest_s1[8];     // 8 child cells N-7..N -> child index N - 5/2 (parent j = N/2 - 1)
  double rest_s0[8];     // 8 child cells N-7..N -> child index N - 1/2 (parent j = N/2)
};
void set_grid_weights(const GridWeights &w);

void launch_flux_x(const Lev &L, const DevParams &p, const double *U, int jmax, int kmax, double wb, int has_child,
                   int has_parent, cudaStream_t s);
void launch_flux_z(const Lev &L, const DevParams &p, const double *U, int jmax, int kmax, double wb, int has_child,
                   int has_parent, cudaStream_t s);
void launch_hydro_div(const Lev &L, const DevParams &p, const double *U, int jmax, int kmax, cudaStream_t s);
void launch_prim2cons_all(const Lev &L, const DevParams &p, double *U, cudaStream_t s);
void launch_c2p_region(const Lev &L, const DevParams &p, double *U, int j0, int j1, int k0, int k1, cudaStream_t s,
                       int skip_corner = 0);

void launch_cartoon(const Lev &L, const DevParams &p, const double *U, const double *tab, int tab_stride, cudaStream_t s);
void launch_z4c_derivs(const Lev &L, const DevParams &p, const double *U, double *DS, int jmax, int kmax, cudaStream_t s);
void launch_z4c_point(const Lev &L, const DevParams &p, const double *U, const double *DS, int jmax, int kmax,
                      cudaStream_t s);
int z4c_scratch_planes();

void launch_parity_x(const Lev &L, double *U, cudaStream_t s);
void launch_parity_z(const Lev &L, double *U, cudaStream_t s);
void launch_outflow(const Lev &L, double *U, cudaStream_t s);
void launch_outer(const Lev &L, const double *Un, double *U, double tau, cudaStream_t s);
// two launches: the metric (one thread per buffer cell and field), then the hydro
void launch_prolong(const Lev &L, const Lev &Pa, const DevParams &p, double *U, const double *Up, int full,
                    cudaStream_t s);
int prolong_cells(const Lev &L, int full);
void launch_rk_update(const Lev &L, const DevParams &p, double *Ust, int stage, double dt, int jmax, int kmax,
                      cudaStream_t s);
void launch_restrict(const Lev &C, const Lev &Pa, cudaStream_t s);
void launch_reflux(const Lev &C, const Lev &Pa, double dt, cudaStream_t s);
void launch_diag(const Lev &L, const DevParams &p, const double *DS, int covered, int evolve, double *partials,
                 int slot, cudaStream_t s);
int diag_blocks(const Lev &L);
void launch_diag_final(const double *partials, int n, double *out, cudaStream_t s);

}  // namespace sacra
