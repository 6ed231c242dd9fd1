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

// ---- batched launches: one persistent launch per kernel kind and stage over
// the tiles of all levels of all stars of a batch (see capi.cu)
struct BL {                 // one level of one star as a stage sees it
  Lev L;
  DevParams P;              // the star's parameters (EOS, gauge, atmosphere, ...)
  const double *U;          // stage state read (Un at stage 0, Us after)
  void *DS;                 // this level's derivative scratch (FP64 or FP32 planes)
  int jmax, kmax;           // update region [1, jmax] x [1, kmax]
  int has_child, has_parent;
  double wb;                // RK weight of this stage's fluxes in the child-boundary flux registers
  double wbp;               // ... in the parent-boundary registers (wb dt_level / dt_parent)
};
struct Tile {               // one block's worth of cells of one level
  int bl, j0, k0, pad;
};
struct Batch {
  const BL *bl;             // device array
  const Tile *tiles;        // device array
  int ntiles;
  int grid;                 // persistent blocks
  dim3 block;               // tile shape = block shape
  int *ctr;                 // tiles handed out past the first gridDim.x (zero at the launch)
};
// Walk over the tiles of a batched launch.  DYN: block b starts with tile b,
// then takes the next tile not yet handed out from the launch's counter, so
// that a block on cheap tiles (atmosphere) takes more of them than one on
// costly tiles (matter under recovery); otherwise a grid stride (the kernels
// whose tiles cost the same, where the counter only adds register pressure).
// The block copies the tile's level view into shared memory (so that every
// thread reads the level and its parameters from there) and calls f(view,
// tile) with all threads.  Tiles are independent, so which block handles a
// tile changes no value.
template <bool DYN = true, class F>
__device__ __forceinline__ void for_tiles(const Batch &b, F &&f) {
  __shared__ BL sb;
  const int nth = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
  if constexpr (DYN) {
    __shared__ int next;
    int t = blockIdx.x;
    while (t < b.ntiles) {
      const Tile tl = b.tiles[t];
      const int *src = reinterpret_cast<const int *>(b.bl + tl.bl);
      int *dst = reinterpret_cast<int *>(&sb);
      for (int i = tid; i < (int)(sizeof(BL) / sizeof(int)); i += nth) dst[i] = src[i];
      __syncthreads();
      f(sb, tl);
      if (tid == 0) next = (int)gridDim.x + atomicAdd(b.ctr, 1);
      __syncthreads();
      t = next;
    }
  } else {
    for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
      const Tile tl = b.tiles[t];
      const int *src = reinterpret_cast<const int *>(b.bl + tl.bl);
      int *dst = reinterpret_cast<int *>(&sb);
      for (int i = tid; i < (int)(sizeof(BL) / sizeof(int)); i += nth) dst[i] = src[i];
      __syncthreads();
      f(sb, tl);
      __syncthreads();
    }
  }
}
static_assert(sizeof(BL) % sizeof(int) == 0, "BL is copied as ints");

enum BKind { B_FLUX_X = 0, B_FLUX_Z, B_HYDRO, B_CARTOON, B_DERIVS, B_POINT, B_RK, B_NKIND };

// ---- level lists: one launch of a per-level operation (ghost fill,
// prolongation, restriction, reflux, recovery) over several levels, e.g. the
// same depth of every star of a batch; item i is handled by the blocks of
// grid slice blockIdx.z / (the operation's planes) == i
struct LItem {
  Lev L, Pa;                // the level and its parent (restriction: the child and the parent)
  DevParams P;              // the star's parameters
  const double *A;          // input state: the parent's stage state (prolongation), U^n (outer boundary)
  double *B;                // output state: the level's stage state (ghost fill), its U^n (restriction)
};
void launch_l_parity_x(const LItem *items, int n, int max_nx, cudaStream_t s);
void launch_l_parity_z(const LItem *items, int n, int max_nx, cudaStream_t s);        // after the x parity
void launch_l_outer(const LItem *items, int n, int max_nx, double tau, int metric, int prims, cudaStream_t s);
void launch_l_prolong(const LItem *items, int n, int max_nx, int full, cudaStream_t s); // metric, then hydro
void launch_l_restrict(const LItem *items, int n, int max_nx, cudaStream_t s);        // metric, then conserved
void launch_l_reflux(const LItem *items, int n, int max_nx, double dt, cudaStream_t s);
void launch_l_c2p_restricted(const LItem *items, int n, int max_nx, cudaStream_t s);
void launch_b_flux_x(const Batch &b, const DevParams &p, cudaStream_t s);
void launch_b_flux_z(const Batch &b, const DevParams &p, cudaStream_t s);
void launch_b_hydro_div(const Batch &b, const DevParams &p, cudaStream_t s);
// FP64 cartoon kernel: per column j, the weights of each d_y / d_yy output on the nine
// values x_{j-4..j+4} (interpolation at varpi_m, rotation by +-phi_m and the 6th-order
// differences over the planes m = -3..3 folded together), dimensionless:
//   [0, 9) Sd, [9, 18) D1, [18, 27) E1, [27, 36) C2, [36, 45) F, [45, 54) G, [54, 63) H, 63 K2, 64 Kb
constexpr int kCartoonW = 68;
void launch_b_cartoon(const Batch &b, const DevParams &p, const double *tab, int tab_stride, const double *tabw,
                      cudaStream_t s);
void launch_b_z4c_derivs(const Batch &b, const DevParams &p, cudaStream_t s);
// store_rs: the pass also writes the Ricci scalar it forms (FP64, or the FP32
// value widened) into the FP64 scratch plane z4c_ricci_plane()
void launch_b_z4c_point(const Batch &b, const DevParams &p, cudaStream_t s, int store_rs = 0);
void launch_b_rk_update(const Batch &b, const DevParams &p, int stage, double dt, cudaStream_t s);
// the derivative passes have fixed tile shapes (their shared-memory staging)
dim3 z4c_derivs_f32_block();
dim3 z4c_derivs_f64_block();

void launch_flux_x(const Lev &L, const DevParams &p, const double *U, int jmax, int kmax, double wb, int has_child,
                   int has_parent, cudaStream_t s);
void launch_flux_z(const Lev &L, const DevParams &p, const double *U, int jmax, int kmax, double wb, int has_child,
                   int has_parent, cudaStream_t s);
void launch_hydro_div(const Lev &L, const DevParams &p, const double *U, int jmax, int kmax, cudaStream_t s);
void launch_prim2cons_all(const Lev &L, const DevParams &p, double *U, cudaStream_t s);
void launch_c2p_region(const Lev &L, const DevParams &p, double *U, int j0, int j1, int k0, int k1, cudaStream_t s,
                       int skip_corner = 0);

void launch_cartoon(const Lev &L, const DevParams &p, const double *U, const double *tab, int tab_stride,
                    const double *tabw, cudaStream_t s);
void launch_z4c_derivs(const Lev &L, const DevParams &p, const double *U, double *DS, int jmax, int kmax, cudaStream_t s);
void launch_z4c_point(const Lev &L, const DevParams &p, const double *U, const double *DS, int jmax, int kmax,
                      cudaStream_t s);
int z4c_scratch_planes();
int z4c_ricci_plane();

void launch_parity_x(const Lev &L, double *U, cudaStream_t s);
void launch_parity_z(const Lev &L, double *U, cudaStream_t s);
void launch_outflow(const Lev &L, double *U, cudaStream_t s);
void launch_outer(const Lev &L, const DevParams &p, const double *Un, double *U, double tau, cudaStream_t s);
// two launches: the metric (one thread per buffer cell and field), then the hydro
void launch_prolong(const Lev &L, const Lev &Pa, const DevParams &p, double *U, const double *Up, int full,
                    cudaStream_t s);
int prolong_cells(const Lev &L, int full);
void launch_rk_update(const Lev &L, const DevParams &p, double *Ust, int stage, double dt, int jmax, int kmax,
                      cudaStream_t s);
void launch_restrict(const Lev &C, const Lev &Pa, cudaStream_t s);
// parent data at time t^n + theta (t^{n+1} - t^n) for a sub-cycled child (Sec. II.D)
void launch_time_interp(const Lev &P, const double *uold, const double *pold, const double *pnow, double *ut,
                        double *pt, double theta, int have_old, cudaStream_t s);
void launch_reflux(const Lev &C, const Lev &Pa, double dt, cudaStream_t s);
// RS: NULL, or the Ricci scalar of this state per cell, which then replaces
// the second derivatives and the Ricci tensor
void launch_diag(const Lev &L, const DevParams &p, const double *DS, int covered, int evolve, double *partials,
                 int slot, cudaStream_t s, const double *RS = nullptr);
int diag_blocks(const Lev &L);
void launch_diag_final(const double *partials, int n, double *out, cudaStream_t s);

// learned seed of the primitive recovery (mlp.cu): tuples from a level's state,
// training (forward, backward, Adam) and the full-batch gradient
size_t mlp_collect_scratch_bytes(const Lev &L);
// tuples of one level appended in cell order at *count; scratch: mlp_collect_scratch_bytes(L) device bytes
void launch_mlp_collect(const Lev &L, const DevParams &p, float *out, long long cap, unsigned long long *count,
                        void *scratch, cudaStream_t s);
int mlp_train(const float *samples, long long n, int steps, int batch_blocks, float lr, unsigned long long seed,
              float kmin, MlpNet *dev_net, float *host_loss, float *host_report, cudaStream_t s);
int mlp_grad(const float *samples, long long n, const MlpNet *dev_net, float *host_grad, float *host_loss,
             cudaStream_t s);

}  // namespace sacra
