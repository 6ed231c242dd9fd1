// FMR grid kernels on sm_103a (Lam & Shibata, arXiv:2502.03223, Sec. II.A,
// II.B.3, II.D, II.F.1): symmetry and outer-boundary ghost fill, buffer-zone
// prolongation, the RK stage update with the algebraic constraints and the
// primitive recovery, restriction, reflux and deterministic diagnostics.
#include "kernels.h"
#include "z4c.cuh"

namespace sacra {

__constant__ GridWeights cW;

void set_grid_weights(const GridWeights &w) { cudaMemcpyToSymbol(cW, &w, sizeof(GridWeights)); }

// x -> -x parity (rotation by pi about z) and z -> -z parity of every field
__device__ __forceinline__ double sgn_x(int f) {
  switch (f) {
    case fGX: case fGY: case fBX: case fBY: case fBBX: case fBBY:
    case fHXZ: case fHYZ: case fAXZ: case fAYZ:
      return -1.0;
    default:
      return 1.0;
  }
}
__device__ __forceinline__ double sgn_z(int f) {
  switch (f) {
    case fGZ: case fBZ: case fBBZ: case fHXZ: case fHYZ: case fAXZ: case fAYZ:
      return -1.0;
    default:
      return 1.0;
  }
}

// axis ghosts j in [-7, 0] for rows [1, nz+8]; blockIdx.z: plane (25 metric
// fields, then the 6 primitives)
__device__ __forceinline__ void parity_x_body(const Lev &L, double *__restrict__ U, int bx, int by, int f) {
  const int j = -7 + (int)(bx * blockDim.x + threadIdx.x);
  const int k = 1 + (int)(by * blockDim.y + threadIdx.y);
  if (j > 0 || k > L.nz + GH) return;
  const int d = cid(L, j, k), s = cid(L, 1 - j, k);
  if (f < NMET) {
    double *u = U + (size_t)f * L.P;
    u[d] = sgn_x(f) * u[s];
  } else {
    const int q = f - NMET;
    double *u = L.prim + (size_t)q * L.P;
    u[d] = ((q == pUX || q == pUY) ? -1.0 : 1.0) * u[s];
  }
}

__global__ void k_parity_x(Lev L, double *__restrict__ U) { parity_x_body(L, U, blockIdx.x, blockIdx.y, blockIdx.z); }

// equator ghosts k in [-7, 0] for all columns; blockIdx.z as above
__device__ __forceinline__ void parity_z_body(const Lev &L, double *__restrict__ U, int bx, int by, int f) {
  const int j = -7 + (int)(bx * blockDim.x + threadIdx.x);
  const int k = -7 + (int)(by * blockDim.y + threadIdx.y);
  if (j > L.nx + GH || k > 0) return;
  const int d = cid(L, j, k), s = cid(L, j, 1 - k);
  if (f < NMET) {
    double *u = U + (size_t)f * L.P;
    u[d] = sgn_z(f) * u[s];
  } else {
    const int q = f - NMET;
    double *u = L.prim + (size_t)q * L.P;
    u[d] = (q == pUZ ? -1.0 : 1.0) * u[s];
  }
}

__global__ void k_parity_z(Lev L, double *__restrict__ U) { parity_z_body(L, U, blockIdx.x, blockIdx.y, blockIdx.z); }

// planar slab: zero-gradient copy into every ghost cell
__global__ void k_outflow(Lev L, double *__restrict__ U) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.px * L.pz) return;
  const int j = i % L.px - GH + 1, k = i / L.px - GH + 1;
  if (j >= 1 && j <= L.nx && k >= 1 && k <= L.nz) return;
  const int jj = min(max(j, 1), L.nx), kk = min(max(k, 1), L.nz);
  const int s = cid(L, jj, kk);
  const size_t P = L.P;
  for (int f = 0; f < NST; ++f) U[(size_t)f * P + i] = U[(size_t)f * P + s];
#pragma unroll
  for (int f = 0; f < NPRIM; ++f) L.prim[(size_t)f * P + i] = L.prim[(size_t)f * P + s];
}

// Outer boundary of the coarsest level (Sec. II.B.3): Q = Q_inf + (1 - tau/r)
// (Q^n - Q_inf)(r - tau), quadratic (3x3) Lagrange interpolation of the step-
// start state Un; hydro primitives copied from the nearest interior cell.
// Threads: the L-shaped strip {j > nx or k > nz} of [1, nx+8] x [1, nz+8],
// indexed compactly (rows k > nz first), times kOuterGroups groups of fields
// (blockIdx.y) that share the interpolation weights.
constexpr int kOuterGroups = 5;

__device__ __forceinline__ void outer_body(const Lev &L, const double *__restrict__ Un, double *__restrict__ U,
                                           double tau, int metric, int prims, int bx, int group) {
  int i = bx * blockDim.x + threadIdx.x;
  const int w = L.nx + GH, top = GH * w;
  int j, k;
  if (i < top) {
    j = 1 + i % w;
    k = L.nz + 1 + i / w;
  } else {
    i -= top;
    if (i >= GH * L.nz) return;
    j = L.nx + 1 + i % GH;
    k = 1 + i / GH;
  }
  const size_t P = L.P;
  const double x = (j - 0.5) * L.dx, z = (k - 0.5) * L.dz;
  const double r = sqrt(x * x + z * z);
  const double fac = 1.0 - tau / r;
  const double xi = x * fac / L.dx + 0.5, ze = z * fac / L.dz + 0.5;
  const int i0 = min((int)floor(xi + 0.5), L.nx + GH - 1), k0 = min((int)floor(ze + 0.5), L.nz + GH - 1);
  const double tx = xi - i0, tz = ze - k0;
  const double wx[3] = {0.5 * tx * (tx - 1.0), (1.0 - tx) * (1.0 + tx), 0.5 * tx * (tx + 1.0)};
  const double wz[3] = {0.5 * tz * (tz - 1.0), (1.0 - tz) * (1.0 + tz), 0.5 * tz * (tz + 1.0)};
  const int d = cid(L, j, k), c0 = cid(L, i0, k0);
  for (int f = group; metric && f < NMET; f += kOuterGroups) {
    const double qinf = (f == fW || f == fAL) ? 1.0 : 0.0;
    const double *u = Un + (size_t)f * P + c0;
    const double u0 = u[0] - qinf;
    double s = 0.0;
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) s += wx[a] * wz[b] * (u[(b - 1) * L.px + (a - 1)] - qinf - u0);
    U[(size_t)f * P + d] = qinf + fac * (u0 + s);
  }
  if (group == 0 && prims) {
    const int sc = cid(L, min(j, L.nx), min(k, L.nz));
#pragma unroll
    for (int f = 0; f < NPRIM; ++f) L.prim[(size_t)f * P + d] = L.prim[(size_t)f * P + sc];
  }
}

__global__ void k_outer(Lev L, const double *__restrict__ Un, double *__restrict__ U, double tau, int metric,
                        int prims) {
  outer_body(L, Un, U, tau, metric, prims, blockIdx.x, blockIdx.y);
}

__device__ __forceinline__ double minmod(double a, double b) {
  return a * b <= 0.0 ? 0.0 : (fabs(a) < fabs(b) ? a : b);
}

// Buffer cells of a level: the L-shaped strip {j >= lo or k >= lo} of
// [1, N+8]^2 (lo = N+1 at the start of a step, N+5 afterwards), indexed
// compactly: first the rows k >= lo, then the columns j >= lo below them.
__device__ __forceinline__ bool buffer_cell(const Lev &L, int lo, int i, int &j, int &k) {
  const int w = L.nx + GH;                 // cells 1..N+8 in x
  const int rows = (L.nz + GH) - lo + 1;   // rows lo..N+8
  const int top = rows * w;
  if (i < top) {
    j = 1 + i % w;
    k = lo + i / w;
    return true;
  }
  i -= top;
  const int cols = w - lo + 1;             // columns lo..N+8
  if (i >= cols * (lo - 1)) return false;
  j = lo + i % cols;
  k = 1 + i / cols;
  return true;
}

// Buffer-zone prolongation of the metric (Sec. II.D): 8th-order Lagrange,
// tensor product over 8x8 parent cells, one thread per (buffer cell, field).
__device__ __forceinline__ void prolong_metric_body(const Lev &L, const Lev &Pa, double *__restrict__ U,
                                                    const double *__restrict__ Up, int lo, int blk, int f) {
  int j, k;
  if (!buffer_cell(L, lo, blk * blockDim.x + threadIdx.x, j, k)) return;
  const bool ex = (j & 1) == 0, ez = (k & 1) == 0;
  const int mx = ex ? j / 2 : (j + 1) / 2, mz = ez ? k / 2 : (k + 1) / 2;
  const int bx = ex ? mx - 3 : mx - 4, bz = ez ? mz - 3 : mz - 4;
  const double *u = Up + (size_t)f * Pa.P;
  const double u0 = u[cid(Pa, mx, mz)];
  const int pb = cid(Pa, bx, bz);
  double s = 0.0;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    double r = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) r += (ex ? cW.prol[a] : cW.prol[7 - a]) * (u[pb + b * Pa.px + a] - u0);
    s += (ez ? cW.prol[b] : cW.prol[7 - b]) * r;
  }
  U[(size_t)f * L.P + cid(L, j, k)] = u0 + s;
}

// Pairs of buffer cells (j, k), (j, k + 1) with k odd: lo is odd and N even
// on refined levels, so the rows of both parts of the strip pair up.
__device__ __forceinline__ bool buffer_pair(const Lev &L, int lo, int i, int &j, int &k) {
  const int w = L.nx + GH;
  const int prow = ((L.nz + GH) - lo + 1) / 2;   // row pairs (lo, lo+1) .. (N+7, N+8)
  const int top = prow * w;
  if (i < top) {
    j = 1 + i % w;
    k = lo + 2 * (i / w);
    return true;
  }
  i -= top;
  const int cols = w - lo + 1;
  if (i >= cols * ((lo - 1) / 2)) return false;
  j = lo + i % cols;
  k = 1 + 2 * (i / cols);
  return true;
}

// The metric prolongation of a pair of buffer cells one above the other: the
// two children share their parent cell (same u0) and seven of their eight
// parent rows, so the x-interpolations of the nine rows are formed once.
// Each child's sums are those of prolong_metric_body, in the same order.
__device__ __forceinline__ void prolong_metric_pair_body(const Lev &L, const Lev &Pa, double *__restrict__ U,
                                                         const double *__restrict__ Up, int lo, int blk, int f) {
  int j, k;
  if (!buffer_pair(L, lo, blk * blockDim.x + threadIdx.x, j, k)) return;
  const bool ex = (j & 1) == 0;
  const int mx = ex ? j / 2 : (j + 1) / 2, mz = (k + 1) / 2;   // k odd: both children in parent row mz
  const int bx = ex ? mx - 3 : mx - 4, bz = mz - 4;
  const double *u = Up + (size_t)f * Pa.P;
  const double u0 = u[cid(Pa, mx, mz)];
  const int pb = cid(Pa, bx, bz);
  double r[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    double q = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) q += (ex ? cW.prol[a] : cW.prol[7 - a]) * (u[pb + t * Pa.px + a] - u0);
    r[t] = q;
  }
  double so = 0.0, se = 0.0;   // child k (odd: rows bz..bz+7), child k+1 (even: rows bz+1..bz+8)
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    so += cW.prol[7 - b] * r[b];
    se += cW.prol[b] * r[b + 1];
  }
  U[(size_t)f * L.P + cid(L, j, k)] = u0 + so;
  U[(size_t)f * L.P + cid(L, j, k + 1)] = u0 + se;
}

__global__ void k_prolong_metric(Lev L, Lev Pa, double *__restrict__ U, const double *__restrict__ Up, int lo) {
  prolong_metric_body(L, Pa, U, Up, lo, blockIdx.x, blockIdx.y);
}

// Buffer-zone primitives by minmod-limited linear prolongation, then the
// conserved variables from them with the prolongated metric.
__device__ __forceinline__ void prolong_hydro_body(const Lev &L, const Lev &Pa, const DevParams &p,
                                                   double *__restrict__ U, int lo, int bx) {
  int j, k;
  if (!buffer_cell(L, lo, bx * blockDim.x + threadIdx.x, j, k)) return;
  const size_t P = L.P, PP = Pa.P;
  const bool ex = (j & 1) == 0, ez = (k & 1) == 0;
  const int mx = ex ? j / 2 : (j + 1) / 2, mz = ez ? k / 2 : (k + 1) / 2;
  const int pc = cid(Pa, mx, mz);
  const int d = cid(L, j, k);
  const double ox = ex ? 0.25 : -0.25, oz = ez ? 0.25 : -0.25;
  double pr[NPRIM];
#pragma unroll
  for (int f = 0; f < NPRIM; ++f) {
    const double *a = Pa.prim + (size_t)f * PP + pc;
    const double a0 = a[0];
    pr[f] = a0 + ox * minmod(a[1] - a0, a0 - a[-1]) + oz * minmod(a[Pa.px] - a0, a0 - a[-Pa.px]);
  }
  const double pc0 = eos_pc(p, pr[pRHO]);
  if (pr[pP] < pc0 || p.adiabatic) pr[pP] = pc0;
  pr[pEPS] = eos_eps(p, pr[pRHO], pr[pP]);
#pragma unroll
  for (int f = 0; f < NPRIM; ++f) L.prim[(size_t)f * P + d] = pr[f];
  const Sym3 g = conf_metric(U, P, d);
  double q[NCONS];
  prim_to_cons(p, pr, U[(size_t)fW * P + d], g, (j - 0.5) * L.dx, q);
#pragma unroll
  for (int v = 0; v < NCONS; ++v) U[(size_t)(fQD + v) * P + d] = q[v];
}

__global__ void k_prolong_hydro(Lev L, Lev Pa, DevParams p, double *__restrict__ U, int lo) {
  prolong_hydro_body(L, Pa, p, U, lo, blockIdx.x);
}

// det gt = 1 and tr At = 0 after every stage (Sec. II.B.1):
// gt <- d^(-1/3) gt, W <- d^(-1/6) W, At <- d^(-1/3)(At - gt tr/3), Khat += tr
// gi_out: the inverse of the normalised conformal metric, gt^-1 / c13 with
// 1 / c13 = det c13^2
__device__ inline void enforce_algebraic(double m[NST], Sym3 *gi_out) {
  Sym3 g;
  g.xx = 1.0 + m[fHXX]; g.xy = m[fHXY]; g.xz = m[fHXZ]; g.yy = 1.0 + m[fHYY]; g.yz = m[fHYZ]; g.zz = 1.0 + m[fHZZ];
  double det;
  const Sym3 gi = s3inv(g, &det);
  const double tr = gi.xx * m[fAXX] + gi.yy * m[fAYY] + gi.zz * m[fAZZ]
                  + 2.0 * (gi.xy * m[fAXY] + gi.xz * m[fAXZ] + gi.yz * m[fAYZ]);
  const double c13 = rcbrt(det), c16 = sqrt(c13), tr3 = tr / 3.0;
  const double gv[6] = {g.xx, g.xy, g.xz, g.yy, g.yz, g.zz};
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    m[fAXX + a] = c13 * (m[fAXX + a] - gv[a] * tr3);
    const double gn = c13 * gv[a];
    m[fHXX + a] = (a == 0 || a == 3 || a == 5) ? gn - 1.0 : gn;
  }
  m[fW] *= c16;
  m[fKH] += tr;
  const double s = det * c13 * c13;
  gi_out->xx = gi.xx * s; gi_out->xy = gi.xy * s; gi_out->xz = gi.xz * s;
  gi_out->yy = gi.yy * s; gi_out->yz = gi.yz * s; gi_out->zz = gi.zz * s;
}

// RK stage combination on [1, jmax] x [1, kmax], then algebraic constraints
// and primitive recovery.  Ust = stage state read (Un at stage 0, Us after);
// the result is written to Us.
template <bool SEED = false>
__device__ __forceinline__ void rk_update_cell(const Lev &L, const DevParams &p, const double *__restrict__ Ust, int stage, double dt,
                                                   int jmax, int kmax, int j, int k, const MlpNet *net = nullptr) {
  if (j > jmax || k > kmax) return;
  const size_t P = L.P;
  const int id = cid(L, j, k);
  double m[NST];
  const int f0 = p.evolve ? 0 : NMET;
  bool held = false;   // excised inner boundary: the hydro keeps U^n and is not recovered
  if (p.r_hold2 > 0.0) {
    const double x = (j - 0.5) * L.dx, z = (k - 0.5) * L.dz;
    held = x * x + z * z < p.r_hold2;
  }
  for (int f = 0; f < NST; ++f) {
    const size_t o = (size_t)f * P + id;
    if (f < f0) { m[f] = L.us[o]; continue; }
    if (f >= NMET && held) { m[f] = L.un[o]; continue; }
    const double un = L.un[o], kk = L.rhs[o];
    double out;
    if (p.rk == SACRA_RK4) {
      if (stage < 3) {
        const double bw = stage == 0 ? 1.0 / 6.0 : 1.0 / 3.0;
        L.ka[o] = (stage == 0 ? 0.0 : L.ka[o]) + bw * kk;
        out = un + (stage == 2 ? 1.0 : 0.5) * dt * kk;
      } else {
        out = un + dt * (L.ka[o] + kk * (1.0 / 6.0));
      }
    } else {
      if (stage == 0) out = un + dt * kk;
      else if (stage == 1) out = 0.75 * un + 0.25 * Ust[o] + 0.25 * dt * kk;
      else out = un * (1.0 / 3.0) + (2.0 / 3.0) * Ust[o] + (2.0 / 3.0) * dt * kk;
    }
    m[f] = out;
  }
  Sym3 gin;
  if (p.evolve) enforce_algebraic(m, &gin);
  if (held) {
    for (int f = f0; f < NST; ++f) L.us[(size_t)f * P + id] = m[f];
    return;
  }
  Sym3 g;
  g.xx = 1.0 + m[fHXX]; g.xy = m[fHXY]; g.xz = m[fHXZ]; g.yy = 1.0 + m[fHYY]; g.yz = m[fHYZ]; g.zz = 1.0 + m[fHZZ];
  double pr[NPRIM];
  const int st = cons_to_prim<SEED>(p, m + fQD, m[fW], g, (j - 0.5) * L.dx, pr, net, p.evolve ? &gin : nullptr);
  for (int f = f0; f < NST; ++f) L.us[(size_t)f * P + id] = m[f];
#pragma unroll
  for (int f = 0; f < NPRIM; ++f) L.prim[(size_t)f * P + id] = pr[f];
  L.status[id] = st;
}

__global__ void __launch_bounds__(128) k_rk_update(Lev L, DevParams p, const double *__restrict__ Ust, int stage, double dt,
                                                   int jmax, int kmax) {
  rk_update_cell(L, p, Ust, stage, dt, jmax, kmax, 1 + (int)(blockIdx.x * blockDim.x + threadIdx.x), 1 + (int)(blockIdx.y * blockDim.y + threadIdx.y));
}

template <bool SEED>
__global__ void __launch_bounds__(128) kb_rk_update(Batch b, DevParams p, int stage, double dt) {
  if constexpr (SEED) {
    // the learned recovery seed (one network for the batch) staged in shared memory
    __shared__ MlpNet snet;
    const uint4 *src = reinterpret_cast<const uint4 *>(p.mlp);
    uint4 *dst = reinterpret_cast<uint4 *>(&snet);
    const int nth = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int i = tid; i < (int)(sizeof(MlpNet) / sizeof(uint4)); i += nth) dst[i] = src[i];
    __syncthreads();
    for_tiles(b, [&](const BL &q, const Tile &tl) {
      rk_update_cell<true>(q.L, q.P, q.U, stage, dt, q.jmax, q.kmax, tl.j0 + threadIdx.x, tl.k0 + threadIdx.y, &snet);
    });
  } else {
    for_tiles(b, [&](const BL &q, const Tile &tl) {
      rk_update_cell<false>(q.L, q.P, q.U, stage, dt, q.jmax, q.kmax, tl.j0 + threadIdx.x, tl.k0 + threadIdx.y);
    });
  }
}

void launch_b_rk_update(const Batch &b, const DevParams &p, int stage, double dt, cudaStream_t s) {
  if (b.ntiles <= 0) return;
  if (p.mlp) kb_rk_update<true><<<b.grid, b.block, 0, s>>>(b, p, stage, dt);
  else kb_rk_update<false><<<b.grid, b.block, 0, s>>>(b, p, stage, dt);
}

// Parent data of a sub-cycled child at time t^n + theta (t^{n+1} - t^n)
// (Sec. II.D): second-order Lagrange through the parent's slices t^{n-1}
// (uold, pold), t^n (us, pnow), t^{n+1} (un, prim) in difference form about
// t^n; first order through t^n, t^{n+1} for a primitive where
// (p^{n+1} - p^n)(p^n - p^{n-1}) < 0, and everywhere while have_old = 0.
// One thread per padded cell and plane (25 metric planes, then 6 primitives).
__global__ void k_time_interp(Lev P, const double *__restrict__ uold, const double *__restrict__ pold,
                              const double *__restrict__ pnow, double *__restrict__ ut, double *__restrict__ pt,
                              double theta, int have_old) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.px * P.pz) return;
  const int f = blockIdx.y;
  const double wm = 0.5 * theta * (theta - 1.0), wp = 0.5 * theta * (theta + 1.0);
  if (f < NMET) {
    const size_t o = (size_t)f * P.P + i;
    const double q0 = P.us[o], q1 = P.un[o];
    ut[o] = have_old ? q0 + wm * (uold[o] - q0) + wp * (q1 - q0) : q0 + theta * (q1 - q0);
  } else {
    const size_t o = (size_t)(f - NMET) * P.P + i;
    const double q0 = pnow[o], q1 = P.prim[o];
    const bool quad = have_old && !((q1 - q0) * (q0 - pold[o]) < 0.0);
    pt[o] = quad ? q0 + wm * (pold[o] - q0) + wp * (q1 - q0) : q0 + theta * (q1 - q0);
  }
}

void launch_time_interp(const Lev &P, const double *uold, const double *pold, const double *pnow, double *ut,
                        double *pt, double theta, int have_old, cudaStream_t s) {
  const int n = P.px * P.pz;
  k_time_interp<<<dim3((n + 255) / 256, NMET + NPRIM), 256, 0, s>>>(P, uold, pold, pnow, ut, pt, theta, have_old);
}

// Restriction of child level C onto parent cells [1, N/2]^2 (Sec. II.D):
// q as the volume-weighted average of the 2x2 children, the metric by 8th-
// order Lagrange (nodes shifted inward so that none passes the child edge N).
// blockIdx.z + f0: the field (metric 0..24, conserved 25..29).
__device__ __forceinline__ void restrict_body(const Lev &C, const Lev &Pa, int f0, int blkx, int blky, int plane) {
  const int j = 1 + (int)(blkx * blockDim.x + threadIdx.x);
  const int k = 1 + (int)(blky * blockDim.y + threadIdx.y);
  const int nh = Pa.nx / 2;
  if (j > nh || k > nh) return;
  const int f = f0 + plane;
  const size_t P = C.P, PP = Pa.P;
  const int d = cid(Pa, j, k);
  const int c00 = cid(C, 2 * j - 1, 2 * k - 1);
  if (f >= NMET) {
    const double xp = (j - 0.5) * Pa.dx;
    const double xa = (2 * j - 1.5) * C.dx, xb = (2 * j - 0.5) * C.dx;
    const double *q = C.un + (size_t)f * P + c00;
    // (x-weighted sum of 4 children) * dxc dzc / (x_p dxp dzp); dxp dzp = 4 dxc dzc
    const double s = xa * (q[0] + q[C.px]) + xb * (q[1] + q[C.px + 1]);
    Pa.un[(size_t)f * PP + d] = s / (4.0 * xp);
    return;
  }
  const double *wx, *wz;
  int bx, bz;
  const int N = C.nx;
  if (j <= nh - 2) { wx = cW.rest_c; bx = 2 * j - 4; } else { wx = (j == nh) ? cW.rest_s0 : cW.rest_s1; bx = N - 7; }
  if (k <= nh - 2) { wz = cW.rest_c; bz = 2 * k - 4; } else { wz = (k == nh) ? cW.rest_s0 : cW.rest_s1; bz = N - 7; }
  const int cb = cid(C, bx, bz);
  const double *u = C.un + (size_t)f * P;
  const double u0 = u[c00];
  double s = 0.0;
  for (int b = 0; b < 8; ++b) {
    double r = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) r += wx[a] * (u[cb + b * C.px + a] - u0);
    s += wz[b] * r;
  }
  Pa.un[(size_t)f * PP + d] = u0 + s;
}

__global__ void k_restrict(Lev C, Lev Pa, int f0) { restrict_body(C, Pa, f0, blockIdx.x, blockIdx.y, blockIdx.z); }

// The metric part of the restriction as two passes through shared memory: the
// x-interpolation of every child row a tile of parent cells needs (each row
// serves four parent rows), then the z-interpolation of those row values;
// the same 8 x 8 weights as k_restrict, applied as separable sums.  Block:
// RX x RZ parent cells of one field (blockIdx.z).
constexpr int RX = 32, RZ = 8, RROWS = 2 * RZ + 6;
__device__ __forceinline__ void restrict_metric_body(const Lev &C, const Lev &Pa, int bx, int by, int f) {
  __shared__ double row[RROWS][RX];
  const int nh = Pa.nx / 2, N = C.nx;
  const int j0 = 1 + bx * RX, k0 = 1 + by * RZ;
  const double *u = C.un + (size_t)f * C.P;
  // pass 1: child rows rs .. rs + RROWS - 1 interpolated in x at each parent
  // column; rs = 2 k0 - 4, or N - 7 when the tile holds only the last two rows
  const int rs = min(2 * k0 - 4, N - 7);
  const int tid = threadIdx.y * RX + threadIdx.x;
  for (int e = tid; e < RROWS * RX; e += RX * RZ) {
    const int rr = e / RX, jj = e % RX;
    const int j = j0 + jj, kc = rs + rr;
    double v = 0.0;
    if (j <= nh && kc <= N) {
      const double *wx;
      int bx;
      if (j <= nh - 2) { wx = cW.rest_c; bx = 2 * j - 4; } else { wx = (j == nh) ? cW.rest_s0 : cW.rest_s1; bx = N - 7; }
      const double *q = u + cid(C, bx, kc);
#pragma unroll
      for (int a = 0; a < 8; ++a) v += wx[a] * q[a];
    }
    row[rr][jj] = v;
  }
  __syncthreads();
  // pass 2: z-interpolation of the rows
  const int j = j0 + (int)threadIdx.x, k = k0 + (int)threadIdx.y;
  if (j > nh || k > nh) return;
  const double *wz;
  int bz;
  if (k <= nh - 2) { wz = cW.rest_c; bz = 2 * k - 4; } else { wz = (k == nh) ? cW.rest_s0 : cW.rest_s1; bz = N - 7; }
  const int r0 = bz - rs;
  double s = 0.0;
#pragma unroll
  for (int b = 0; b < 8; ++b) s += wz[b] * row[r0 + b][threadIdx.x];
  Pa.un[(size_t)f * Pa.P + cid(Pa, j, k)] = s;
}

__global__ void __launch_bounds__(RX * RZ) k_restrict_metric(Lev C, Lev Pa) {
  restrict_metric_body(C, Pa, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Reflux (Sec. II.D): parent cells next to the child's outer faces get the
// sum of the fine fluxes (RK-weighted) instead of the coarse flux.
__device__ __forceinline__ void reflux_body(const Lev &C, const Lev &Pa, double dt, int bx) {
  const int i = bx * blockDim.x + threadIdx.x;
  const int nh = Pa.nx / 2;
  if (i >= 2 * nh) return;
  const bool xface = i < nh;
  const int t = (xface ? i : i - nh) + 1;            // k (x-face) or j (z-face) in [1, N/2]
  const int j = xface ? nh + 1 : t, k = xface ? t : nh + 1;
  const int d = cid(Pa, j, k);
  const double vol = (j - 0.5) * Pa.dx * Pa.dx * Pa.dz;
  const int rc = xface ? 0 : 2, rf = xface ? 1 : 3;
  for (int v = 0; v < NCONS; ++v) {
    const double fine = C.freg[(size_t)(rf * NCONS + v) * C.rw + 2 * t - 1] + C.freg[(size_t)(rf * NCONS + v) * C.rw + 2 * t];
    const double coarse = Pa.freg[(size_t)(rc * NCONS + v) * Pa.rw + t];
    Pa.un[(size_t)(fQD + v) * Pa.P + d] += dt * (fine - coarse) / vol;
  }
}

__global__ void k_reflux(Lev C, Lev Pa, double dt) { reflux_body(C, Pa, dt, blockIdx.x); }

// ---------------------------------------------------------------- diagnostics

constexpr int DIAG_Q = 9;   // H^2 dV, Mx^2 dV, My^2 dV, Mz^2 dV, dV, qD dV, qSphi dV, rho_max, n_fail
constexpr int DIAG_T = 128;

// Block reduction of the diagnostic sums (slot 7: maximum) in a fixed order, so
// the result is the same on every run: a shuffle tree inside each warp, then
// warp 0 combines the per-warp values the same way.  The block total ends in
// acc of thread 0.
__device__ __forceinline__ void diag_block_reduce(double acc[DIAG_Q], double (*sh)[DIAG_T / 32], int t) {
  const int lane = t & 31, w = t >> 5;
#pragma unroll
  for (int q = 0; q < DIAG_Q; ++q) {
    double v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double u = __shfl_down_sync(0xffffffffu, v, o);
      v = (q == 7) ? fmax(v, u) : v + u;
    }
    if (lane == 0) sh[q][w] = v;
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int q = 0; q < DIAG_Q; ++q) {
      double v = lane < DIAG_T / 32 ? sh[q][lane] : (q == 7 ? -1e300 : 0.0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double u = __shfl_down_sync(0xffffffffu, v, o);
        v = (q == 7) ? fmax(v, u) : v + u;
      }
      acc[q] = v;
    }
  }
}

// S: storage type of the derivative scratch and the cartoon planes (FP32 in
// the mixed-precision Z4c form); the constraint algebra is FP64 either way.
// RSK: the Ricci scalar comes from RS (formed by the pointwise pass of the
// same stage); otherwise the kernel forms the Ricci tensor itself.
template <typename S, bool RSK>
__global__ void __launch_bounds__(DIAG_T) k_diag(Lev L, DevParams p, const S *__restrict__ DS,
                                                 const double *__restrict__ RS, int covered, int evolve,
                                                 double *__restrict__ partials) {
  __shared__ double sh[DIAG_Q][DIAG_T / 32];
  const int t = threadIdx.x;
  const int n = L.nx * L.nz;
  const int i = blockIdx.x * DIAG_T + t;
  double acc[DIAG_Q];
#pragma unroll
  for (int q = 0; q < DIAG_Q; ++q) acc[q] = 0.0;
  if (i < n) {
    const int j = 1 + i % L.nx, k = 1 + i / L.nx;
    const bool skip = covered && j <= L.nx / 2 && k <= L.nz / 2;
    if (!skip) {
      constexpr double PI = 3.14159265358979323846;
      const size_t P = L.P;
      const int id = cid(L, j, k);
      const bool cyl = p.geometry == SACRA_CYLINDRICAL;
      const double x = (j - 0.5) * L.dx;
      const double vol = cyl ? 2.0 * PI * x * L.dx * L.dz : L.dx * L.dz;
      const double *U = L.un;
      acc[4] = vol;
      acc[5] = U[(size_t)fQD * P + id] * vol;
      acc[6] = U[(size_t)fQSY * P + id] * vol;
      acc[7] = L.prim[(size_t)pRHO * P + id];
      acc[8] = (L.status[id] & (ST_NOCONV | ST_BAD)) ? 1.0 : 0.0;
      if (evolve) {
        // DS holds the derivative scratch of the Z4c pass for this level
        constexpr int D1 = 0, D2 = 48;
        Z4cIn<double> z;
        // the fields the constraints take (lapse, shift, Gt^i and B^i enter
        // neither); every loop below is unrolled so that all indices are
        // compile-time constants and the arrays stay in registers
        z.W = U[(size_t)fW * P + id];
        z.Kh = U[(size_t)fKH * P + id]; z.Th = U[(size_t)fTH * P + id];
#pragma unroll
        for (int a = 0; a < 6; ++a) { z.h[a] = U[(size_t)(fHXX + a) * P + id]; z.A[a] = U[(size_t)(fAXX + a) * P + id]; }
        // the first derivatives the constraints take: W, gt_ij, Khat, Theta
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          z.dW[c] = DS[(size_t)(D1 + c) * P + id];
#pragma unroll
          for (int a = 0; a < 6; ++a) z.dh[a][c] = DS[(size_t)(D1 + 3 * (1 + a) + c) * P + id];
          z.dKh[c] = DS[(size_t)(D1 + 21 + c) * P + id];
          z.dTh[c] = DS[(size_t)(D1 + 33 + c) * P + id];
        }
        Geo<double> G;
        if constexpr (RSK) {
          // the pointwise pass of the same stage has formed the Ricci scalar:
          // only the metric and its inverse are needed here
          G.g.xx = 1.0 + z.h[0]; G.g.xy = z.h[1]; G.g.xz = z.h[2];
          G.g.yy = 1.0 + z.h[3]; G.g.yz = z.h[4]; G.g.zz = 1.0 + z.h[5];
          G.gi = s3inv(G.g, (double *)nullptr);
          G.Rs = RS[id];
        } else {
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int a = 0; a < 3; ++a) z.dGt[a][c] = DS[(size_t)(D1 + 3 * (8 + a) + c) * P + id];
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            z.ddW[q] = DS[(size_t)(D2 + q) * P + id];
#pragma unroll
            for (int a = 0; a < 6; ++a) z.ddh[a][q] = DS[(size_t)(D2 + 6 * (1 + a) + q) * P + id];
          }
          geo_fill(z, G);
          geo_ricci(z, G);
        }
        double pr[NPRIM];
#pragma unroll
        for (int f = 0; f < NPRIM; ++f) pr[f] = L.prim[(size_t)f * P + id];
        double E, Si[3], Sij[6];
        matter(pr, z.W, G.g, G.gi, E, Si, Sij);
        const double K = z.Kh + 2.0 * z.Th;
        const Sym3 &gi = G.gi;
        const double gim[3][3] = {{gi.xx, gi.xy, gi.xz}, {gi.xy, gi.yy, gi.yz}, {gi.xz, gi.yz, gi.zz}};
        double Am[3][3];   // At^j_i -> Am[j][i]
#pragma unroll
        for (int jj = 0; jj < 3; ++jj)
#pragma unroll
          for (int ii = 0; ii < 3; ++ii)
            Am[jj][ii] = gim[jj][0] * z.A[sp(0, ii)] + gim[jj][1] * z.A[sp(1, ii)] + gim[jj][2] * z.A[sp(2, ii)];
        double AA = 0.0, trA = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          trA += Am[a][a];
#pragma unroll
          for (int b = 0; b < 3; ++b) AA += Am[a][b] * Am[b][a];
        }
        const double H = G.Rs + K * K - (AA + (2.0 / 3.0) * K * trA + K * K / 3.0) - 16.0 * PI * E;
        // d_k At_ij: x, z by central differences, y from the cartoon planes
        double dA[6][3];
        const double i60x = 1.0 / (60.0 * L.dx), i60z = 1.0 / (60.0 * L.dz);
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          const double *u = U + (size_t)(fAXX + a) * P + id;
          dA[a][0] = (45.0 * (u[1] - u[-1]) - 9.0 * (u[2] - u[-2]) + (u[3] - u[-3])) * i60x;
          dA[a][2] = (45.0 * (u[L.px] - u[-L.px]) - 9.0 * (u[2 * L.px] - u[-2 * L.px]) + (u[3 * L.px] - u[-3 * L.px])) * i60z;
          dA[a][1] = (cyl && a != 5) ? (double)reinterpret_cast<const S *>(L.dy)[(size_t)(fAXX + a) * P + id] : 0.0;
        }
        // v^k = d_j gt^jk = -gt^ja gt^kb d_j gt_ab = -gt^kb w_b, w_b = gt^ja d_j gt_ab
        double wv[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          double t = 0.0;
#pragma unroll
          for (int jj = 0; jj < 3; ++jj)
#pragma unroll
            for (int a = 0; a < 3; ++a) t += gim[jj][a] * z.dh[sp(a, b)][jj];
          wv[b] = t;
        }
        double v[3];
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) v[kk] = -(gim[kk][0] * wv[0] + gim[kk][1] * wv[1] + gim[kk][2] * wv[2]);
        // Gt^l_ji At^j_l = Gt_{m,ji} At^jm = (1/2) At^jm d_i gt_jm: of the three
        // derivative terms of Gt_{m,ji} the two with d_j and d_m cancel against
        // the symmetric At^jm
        double Au[6];      // At^jm
#pragma unroll
        for (int jj = 0; jj < 3; ++jj)
#pragma unroll
          for (int m = jj; m < 3; ++m) Au[sp(jj, m)] = Am[jj][0] * gim[0][m] + Am[jj][1] * gim[1][m] + Am[jj][2] * gim[2][m];
        const double i3W = 3.0 / z.W;
        double M[3];
#pragma unroll
        for (int ii = 0; ii < 3; ++ii) {
          double s = 0.0;
#pragma unroll
          for (int kk = 0; kk < 3; ++kk) {
            s += v[kk] * z.A[sp(kk, ii)];
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) s += gim[jj][kk] * dA[sp(kk, ii)][jj];
          }
          s -= 0.5 * (Au[0] * z.dh[0][ii] + Au[3] * z.dh[3][ii] + Au[5] * z.dh[5][ii]
                      + 2.0 * (Au[1] * z.dh[1][ii] + Au[2] * z.dh[2][ii] + Au[4] * z.dh[4][ii]));
#pragma unroll
          for (int l = 0; l < 3; ++l) s -= i3W * Am[l][ii] * z.dW[l];
          s -= (2.0 / 3.0) * (z.dKh[ii] + 2.0 * z.dTh[ii]) + 8.0 * PI * Si[ii];
          M[ii] = s;
        }
        acc[0] = H * H * vol;
        acc[1] = M[0] * M[0] * vol; acc[2] = M[1] * M[1] * vol; acc[3] = M[2] * M[2] * vol;
      }
    }
  }
  diag_block_reduce(acc, sh, t);
  if (t == 0)
#pragma unroll
    for (int q = 0; q < DIAG_Q; ++q) partials[(size_t)blockIdx.x * DIAG_Q + q] = acc[q];
}

// fixed-order sum of the block partials (deterministic)
__global__ void k_diag_final(const double *__restrict__ partials, int n, double *__restrict__ out) {
  __shared__ double sh[DIAG_Q][DIAG_T / 32];
  const int t = threadIdx.x;
  double acc[DIAG_Q];
#pragma unroll
  for (int q = 0; q < DIAG_Q; ++q) acc[q] = 0.0;
  for (int b = t; b < n; b += DIAG_T)
#pragma unroll
    for (int q = 0; q < DIAG_Q; ++q)
      acc[q] = (q == 7) ? fmax(acc[q], partials[(size_t)b * DIAG_Q + q]) : acc[q] + partials[(size_t)b * DIAG_Q + q];
  diag_block_reduce(acc, sh, t);
  if (t == 0)
#pragma unroll
    for (int q = 0; q < DIAG_Q; ++q) out[q] = acc[q];
}

// ---------------------------------------------------------------- level-list kernels
//
// The same bodies over the items of a level list (all levels of one depth of
// a batch's stars, say): one launch instead of one per level.  The grid is
// sized for the largest item; blocks beyond an item's extent do nothing.
constexpr int kParityPlanes = NMET + NPRIM;

__global__ void kl_parity_x(const LItem *__restrict__ items) {
  const LItem &it = items[blockIdx.z / kParityPlanes];
  parity_x_body(it.L, it.B, blockIdx.x, blockIdx.y, blockIdx.z % kParityPlanes);
}
__global__ void kl_parity_z(const LItem *__restrict__ items) {
  const LItem &it = items[blockIdx.z / kParityPlanes];
  parity_z_body(it.L, it.B, blockIdx.x, blockIdx.y, blockIdx.z % kParityPlanes);
}
__global__ void kl_outer(const LItem *__restrict__ items, double tau, int metric, int prims) {
  const LItem &it = items[blockIdx.z];
  outer_body(it.L, it.A, it.B, tau, metric, prims, blockIdx.x, blockIdx.y);
}
__global__ void kl_prolong_metric(const LItem *__restrict__ items, int full) {
  const LItem &it = items[blockIdx.z];
  prolong_metric_pair_body(it.L, it.Pa, it.B, it.A, full ? it.L.nx + 1 : it.L.nx + 5, blockIdx.x, blockIdx.y);
}
__global__ void kl_prolong_hydro(const LItem *__restrict__ items, int full) {
  const LItem &it = items[blockIdx.z];
  prolong_hydro_body(it.L, it.Pa, it.P, it.B, full ? it.L.nx + 1 : it.L.nx + 5, blockIdx.x);
}
__global__ void __launch_bounds__(RX * RZ) kl_restrict_metric(const LItem *__restrict__ items) {
  const LItem &it = items[blockIdx.z / NMET];
  restrict_metric_body(it.L, it.Pa, blockIdx.x, blockIdx.y, blockIdx.z % NMET);
}
__global__ void kl_restrict(const LItem *__restrict__ items) {
  const LItem &it = items[blockIdx.z / NCONS];
  restrict_body(it.L, it.Pa, NMET, blockIdx.x, blockIdx.y, blockIdx.z % NCONS);
}
__global__ void kl_reflux(const LItem *__restrict__ items, double dt) {
  const LItem &it = items[blockIdx.z];
  reflux_body(it.L, it.Pa, dt, blockIdx.x);
}

void launch_l_parity_x(const LItem *items, int n, int max_nx, cudaStream_t s) {
  if (n <= 0) return;
  kl_parity_x<<<dim3(1, (max_nx + GH + 15) / 16, n * kParityPlanes), dim3(8, 16), 0, s>>>(items);
}

void launch_l_parity_z(const LItem *items, int n, int max_nx, cudaStream_t s) {
  if (n <= 0) return;
  kl_parity_z<<<dim3((max_nx + 2 * GH + 31) / 32, 1, n * kParityPlanes), dim3(32, 8), 0, s>>>(items);
}

void launch_l_outer(const LItem *items, int n, int max_nx, double tau, int metric, int prims, cudaStream_t s) {
  if (n <= 0) return;
  const int cells = GH * (max_nx + GH) + GH * max_nx;
  kl_outer<<<dim3((cells + 127) / 128, kOuterGroups, n), 128, 0, s>>>(items, tau, metric, prims);
}

void launch_l_prolong(const LItem *items, int n, int max_nx, int full, cudaStream_t s) {
  if (n <= 0) return;
  const int lo = full ? max_nx + 1 : max_nx + 5, w = max_nx + GH;
  const int cells = ((max_nx + GH) - lo + 1) * w + (w - lo + 1) * (lo - 1);
  kl_prolong_metric<<<dim3((cells / 2 + 127) / 128, NMET, n), 128, 0, s>>>(items, full);
  kl_prolong_hydro<<<dim3((cells + 127) / 128, 1, n), 128, 0, s>>>(items, full);
}

void launch_l_restrict(const LItem *items, int n, int max_nx, cudaStream_t s) {
  if (n <= 0) return;
  const int nh = max_nx / 2;
  kl_restrict_metric<<<dim3((nh + RX - 1) / RX, (nh + RZ - 1) / RZ, n * NMET), dim3(RX, RZ), 0, s>>>(items);
  kl_restrict<<<dim3((nh + 31) / 32, (nh + 3) / 4, n * NCONS), dim3(32, 4), 0, s>>>(items);
}

void launch_l_reflux(const LItem *items, int n, int max_nx, double dt, cudaStream_t s) {
  if (n <= 0) return;
  kl_reflux<<<dim3((max_nx + 127) / 128, 1, n), 128, 0, s>>>(items, dt);
}

// ---------------------------------------------------------------- host launchers

void launch_parity_x(const Lev &L, double *U, cudaStream_t s) {
  k_parity_x<<<dim3(1, (L.nz + GH + 15) / 16, NMET + NPRIM), dim3(8, 16), 0, s>>>(L, U);
}

void launch_parity_z(const Lev &L, double *U, cudaStream_t s) {
  k_parity_z<<<dim3((L.nx + 2 * GH + 31) / 32, 1, NMET + NPRIM), dim3(32, 8), 0, s>>>(L, U);
}

void launch_outflow(const Lev &L, double *U, cudaStream_t s) {
  k_outflow<<<(unsigned)((L.P + 255) / 256), 256, 0, s>>>(L, U);
}

void launch_outer(const Lev &L, const DevParams &p, const double *Un, double *U, double tau, cudaStream_t s) {
  const int n = GH * (L.nx + GH) + GH * L.nz;
  k_outer<<<dim3((n + 127) / 128, kOuterGroups), 128, 0, s>>>(L, Un, U, tau, p.evolve, !p.hydro_outer);
}

int prolong_cells(const Lev &L, int full) {
  const int lo = full ? L.nx + 1 : L.nx + 5;
  const int w = L.nx + GH;
  return ((L.nz + GH) - lo + 1) * w + (w - lo + 1) * (lo - 1);
}

void launch_prolong(const Lev &L, const Lev &Pa, const DevParams &p, double *U, const double *Up, int full,
                    cudaStream_t s) {
  const int lo = full ? L.nx + 1 : L.nx + 5;
  const int n = prolong_cells(L, full);
  k_prolong_metric<<<dim3((n + 127) / 128, NMET), 128, 0, s>>>(L, Pa, U, Up, lo);
  k_prolong_hydro<<<(n + 127) / 128, 128, 0, s>>>(L, Pa, p, U, lo);
}

void launch_rk_update(const Lev &L, const DevParams &p, double *Ust, int stage, double dt, int jmax, int kmax,
                      cudaStream_t s) {
  dim3 b(32, 4), g((jmax + 31) / 32, (kmax + 3) / 4);
  k_rk_update<<<g, b, 0, s>>>(L, p, Ust, stage, dt, jmax, kmax);
}

void launch_restrict(const Lev &C, const Lev &Pa, cudaStream_t s) {
  const int nh = Pa.nx / 2;
  k_restrict_metric<<<dim3((nh + RX - 1) / RX, (nh + RZ - 1) / RZ, NMET), dim3(RX, RZ), 0, s>>>(C, Pa);
  dim3 b(32, 4), g((nh + 31) / 32, (nh + 3) / 4, NCONS);
  k_restrict<<<g, b, 0, s>>>(C, Pa, NMET);
}

void launch_reflux(const Lev &C, const Lev &Pa, double dt, cudaStream_t s) {
  const int n = Pa.nx;  // 2 * N/2 cells
  k_reflux<<<(n + 127) / 128, 128, 0, s>>>(C, Pa, dt);
}

int diag_blocks(const Lev &L) { return (L.nx * L.nz + DIAG_T - 1) / DIAG_T; }

void launch_diag(const Lev &L, const DevParams &p, const double *DS, int covered, int evolve, double *partials, int slot,
                 cudaStream_t s, const double *RS) {
  double *out = partials + (size_t)slot * DIAG_Q;
  const float *DSf = reinterpret_cast<const float *>(DS);
  if (p.mixed & SACRA_MIXED_Z4C) {
    if (RS) k_diag<float, true><<<diag_blocks(L), DIAG_T, 0, s>>>(L, p, DSf, RS, covered, evolve, out);
    else k_diag<float, false><<<diag_blocks(L), DIAG_T, 0, s>>>(L, p, DSf, RS, covered, evolve, out);
  } else {
    if (RS) k_diag<double, true><<<diag_blocks(L), DIAG_T, 0, s>>>(L, p, DS, RS, covered, evolve, out);
    else k_diag<double, false><<<diag_blocks(L), DIAG_T, 0, s>>>(L, p, DS, RS, covered, evolve, out);
  }
}

void launch_diag_final(const double *partials, int n, double *out, cudaStream_t s) {
  k_diag_final<<<1, DIAG_T, 0, s>>>(partials, n, out);
}

}  // namespace sacra
