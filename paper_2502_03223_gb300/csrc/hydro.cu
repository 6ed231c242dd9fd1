// GRHD kernels on sm_103a (Lam & Shibata, arXiv:2502.03223, Sec. II.C):
// per-face PPM reconstruction + metric interpolation + tetrad HLLC/TVDLF flux,
// per-cell flux divergence with cylindrical areas/volumes and the geometric and
// gravitational sources, primitive recovery, initial conserved variables.
#include "fixed.cuh"
#include "kernels.h"
#include "z4c.cuh"

namespace sacra {

// 6-point (6th-order) interpolation of a metric field to the face between
// u[0] and u[s]: (3,-25,150,150,-25,3)/256.  FP64 form: difference form about
// u[0] (exact on constants).
__device__ __forceinline__ double face6_fp64(const double *u, int s) {
  const double u0 = u[0];
  return u0 + (3.0 * (u[-2 * s] - u0) - 25.0 * (u[-s] - u0) + 150.0 * (u[s] - u0) - 25.0 * (u[2 * s] - u0)
               + 3.0 * (u[3 * s] - u0)) * (1.0 / 256.0);
}
// The same interpolant as an exact integer sum: the six values on the
// fixed-point grid of their largest exponent (fixed.cuh; one guard bit, |v| <
// 2^54, so the weighted sum, weight sum 356, stays below 2^63), one
// conversion and an exact power-of-two scale: the interpolant rounded once,
// in two FP64 operations instead of twelve.  Non-finite values and values
// near the bottom of the normal range take the FP64 form.
__device__ __forceinline__ double face6(const double *u, int s) {
  long long b[6];
#pragma unroll
  for (int n = 0; n < 6; ++n) b[n] = fx::bits(u[(n - 2) * s]);
  int E = 0;
#pragma unroll
  for (int n = 0; n < 6; ++n) E = max(E, fx::expo(b[n]));
  if (E < 64 || E == 2047) return face6_fp64(u, s);
  long long v[6];
#pragma unroll
  for (int n = 0; n < 6; ++n) v[n] = fx::fix(b[n], E);
  const long long S = 3 * (v[0] + v[5]) - 25 * (v[1] + v[4]) + 150 * (v[2] + v[3]);
  return (double)S * fx::unit(1.0 / 256.0, E);
}

// Face j+1/2 (dir 0, stride 1) or k+1/2 (dir 1, stride px) of cell (j, k):
// reconstruction, metric at the face and the flux, FP64.
// The flux of the face from its reconstructed states pl (cell side), pr
// (neighbour side): a side whose density or pressure is not positive drops
// to first order, then the metric at the face and the Riemann solver.
template <int DIR>
__device__ inline void flux_states_f64(const Lev &L, const DevParams &p, const double *__restrict__ U, int j, int k,
                                       double pl[5], double pr[5], double out[NCONS], int *fb) {
  const size_t P = L.P;
  const int s = DIR == 0 ? 1 : L.px;
  const int id = cid(L, j, k);
  const int pf[5] = {pRHO, pUX, pUY, pUZ, pP};
  if (!(pl[0] > 0.0) || !(pl[4] > 0.0))
#pragma unroll
    for (int v = 0; v < 5; ++v) pl[v] = L.prim[(size_t)pf[v] * P + id];
  if (!(pr[0] > 0.0) || !(pr[4] > 0.0))
#pragma unroll
    for (int v = 0; v < 5; ++v) pr[v] = L.prim[(size_t)pf[v] * P + id + s];
  const double alpha = face6(U + (size_t)fAL * P + id, s);
  const double W = face6(U + (size_t)fW * P + id, s);
  double beta[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) beta[i] = face6(U + (size_t)(fBX + i) * P + id, s);
  Sym3 g;
  g.xx = 1.0 + face6(U + (size_t)fHXX * P + id, s);
  g.xy = face6(U + (size_t)fHXY * P + id, s);
  g.xz = face6(U + (size_t)fHXZ * P + id, s);
  g.yy = 1.0 + face6(U + (size_t)fHYY * P + id, s);
  g.yz = face6(U + (size_t)fHYZ * P + id, s);
  g.zz = 1.0 + face6(U + (size_t)fHZZ * P + id, s);
  *fb = face_flux<double>(p, DIR, pl, pr, alpha, beta, W, g, out);
}

template <int DIR>
__device__ inline void flux_at_f64(const Lev &L, const DevParams &p, const double *__restrict__ U, int j, int k,
                                   double out[NCONS], int *fb) {
  const size_t P = L.P;
  const int s = DIR == 0 ? 1 : L.px;
  const int id = cid(L, j, k);
  const int pf[5] = {pRHO, pUX, pUY, pUZ, pP};
  double pl[5], pr[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    const double *a = L.prim + (size_t)pf[v] * P + id;
    const double c[6] = {a[-2 * s], a[-s], a[0], a[s], a[2 * s], a[3 * s]};
    ppm_pair(c, pl[v], pr[v]);
  }
  flux_states_f64<DIR>(L, p, U, j, k, pl, pr, out, fb);
}

// PPM of the lines of a tile through shared memory (FP64).  The per-face form
// forms each MC slope for four faces and each interface value for three; here
// a block forms every slope, interface value and limited parabola of its
// tile's lines once, with the same formulas (the same values), and each face
// reads its two states.  Lines run along the face normal: rows for x-faces
// (DIR 0), columns for z-faces (DIR 1); a tile holds nli lines of nal faces
// starting at along-index a0 and line l0.  Shared memory (kernels' dynamic
// buffer): per variable and line, the slopes of cells a0-1 .. a0+nal+1 (then
// the left parabola values of cells a0 .. a0+nal), the interfaces between
// cells a0-1+t and a0+t, t < nal+2, and the right parabola values of cells
// a0 .. a0+nal.  Only cells that faces of the region use are formed.
__host__ __device__ constexpr int ppm_tile_doubles(int nal, int nli) { return 5 * nli * ((nal + 3) + (nal + 2) + (nal + 1)); }

template <int DIR>
__device__ __forceinline__ void ppm_tile(const Lev &L, int j0, int k0, int jmax, int kmax, double *sm) {
  const int nal = DIR == 0 ? (int)blockDim.x : (int)blockDim.y, nli = DIR == 0 ? (int)blockDim.y : (int)blockDim.x;
  const int nth = (int)(blockDim.x * blockDim.y), tid = (int)(threadIdx.y * blockDim.x + threadIdx.x);
  const int sS = nal + 3, sI = nal + 2, sR = nal + 1;
  double *S = sm, *I = S + 5 * nli * sS, *RR = I + 5 * nli * sI;
  const int s = DIR == 0 ? 1 : L.px;
  const int a0 = DIR == 0 ? j0 : k0, l0 = DIR == 0 ? k0 : j0;
  const int amax = DIR == 0 ? jmax : kmax, lmax = DIR == 0 ? kmax : jmax;
  auto at = [&](int v, int line, int along) {
    const int pf = v == 0 ? pRHO : (v == 1 ? pUX : (v == 2 ? pUY : (v == 3 ? pUZ : pP)));
    const int j = DIR == 0 ? along : line, k = DIR == 0 ? line : along;
    return L.prim + (size_t)pf * L.P + cid(L, j, k);
  };
  for (int it = tid; it < 5 * nli * sS; it += nth) {          // slopes of cells a0 - 1 + t
    const int t = it % sS, r = it / sS, line = r % nli, v = r / nli, c = a0 - 1 + t;
    if (l0 + line > lmax || c > amax + 2) continue;
    const double *a = at(v, l0 + line, c);
    S[it] = mc_slope(a[-s], a[0], a[s]);
  }
  __syncthreads();
  for (int it = tid; it < 5 * nli * sI; it += nth) {          // interface between cells c and c + 1
    const int t = it % sI, r = it / sI, line = r % nli, v = r / nli, c = a0 - 1 + t;
    if (l0 + line > lmax || c > amax + 1) continue;
    const double *a = at(v, l0 + line, c);
    const double *sl = S + (size_t)r * sS + t;
    I[it] = ppm_iface(a[0], a[s], sl[0], sl[1]);
  }
  __syncthreads();
  for (int it = tid; it < 5 * nli * sR; it += nth) {          // limited parabola of cell a0 + t
    const int t = it % sR, r = it / sR, line = r % nli, v = r / nli, c = a0 + t;
    if (l0 + line > lmax || c > amax + 1) continue;
    double aL = I[(size_t)r * sI + t], aR = I[(size_t)r * sI + t + 1];
    ppm_limit(*at(v, l0 + line, c), aL, aR);
    S[(size_t)r * sS + t] = aL;
    RR[it] = aR;
  }
  __syncthreads();
}

// the two states of face (a0 + t) of line `line` of the staged tile
template <int DIR>
__device__ __forceinline__ void ppm_tile_states(const double *sm, int t, int line, double pl[5], double pr[5]) {
  const int nal = DIR == 0 ? (int)blockDim.x : (int)blockDim.y, nli = DIR == 0 ? (int)blockDim.y : (int)blockDim.x;
  const int sS = nal + 3, sI = nal + 2, sR = nal + 1;
  const double *S = sm, *RR = sm + 5 * nli * (sS + sI);
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    pl[v] = RR[(size_t)(v * nli + line) * sR + t];
    pr[v] = S[(size_t)(v * nli + line) * sS + t + 1];
  }
}

// The same face in FP32 (mixed precision), arranged so that rounding scales
// with what varies across the face, not with rho or P:
//  * the pressure is reconstructed as the offset P - P_j (PPM commutes with a
//    constant shift) from exact differences, and the HLLC solver carries it
//    as that offset (face_flux with pref = P_j);
//  * the metric at the face is the cell value plus an FP32 increment formed
//    from exact differences (integer splits, no FP64 instruction);
//  * the normal momentum flux then lacks g_f P_j, g = alpha W^-3 at the face;
//    it is split as g_j P_j (cell j, FP64: the large part, which cancels
//    between the faces of a cell in FP64) plus (g_f - g_j) P_j in FP32 from
//    the face increments of alpha and W, in a form without cancellation:
//      g_f / g_j - 1 = [x - 3y - 3y^2 - y^3] / (1 + y)^3,
//      x = dalpha / alpha_j, y = dW / W_j.
// The only FP64 instructions are the 5 of g_j P_j and the final addition.
//
// The FP32 form hands a face to the FP64 solver where FP32 rounding could
// change a discrete branch: a stencil with a strong density or pressure
// contrast (a stellar surface, the atmosphere: reconstructed values of order
// eps_32 * max decide the positivity fallback there, and the contact pressure
// of a near-vacuum Riemann problem is of that order too), and every face where
// the FP32 HLLC fails.  Elsewhere the branches have wide margins.
constexpr float kMixedContrast = 1e-3f;

// The FP32 inputs of a face come from a source with two views of cell j + n,
// n = -2..3 along the face normal: pair(q, n), the split (hi, lo) of slot q
// (0 rho, 1 P, 2 alpha, 3 W, 4-6 beta^i, 7-12 h_ij), and single(v, n), u_i
// rounded to FP32 (v = 0, 1, 2).  Both sources give the same values.
constexpr int kF32Pair = 13, kF32Single = 3, kF32Slots = 2 * kF32Pair + kF32Single;
__device__ __forceinline__ int f32_pair_field(int q) {
  return q == 0 ? -1 - pRHO : (q == 1 ? -1 - pP : (q == 2 ? fAL : (q == 3 ? fW : (q < 7 ? fBX + q - 4 : fHXX + q - 7))));
}

// per-face loads from the level's arrays
struct F32Global {
  const double *prim, *U;
  size_t P;
  int id, s;
  __device__ __forceinline__ F2 pair(int q, int n) const {
    const int f = f32_pair_field(q);
    return split_f64(f < 0 ? prim[(size_t)(-1 - f) * P + id + n * s] : U[(size_t)f * P + id + n * s]);
  }
  __device__ __forceinline__ float single(int v, int n) const { return f32_of(prim[(size_t)(pUX + v) * P + id + n * s]); }
};

// the staged tile (f32_tile): slot-major, then line, then cell along the normal
struct F32Staged {
  const float *sm;
  int nli, nc, line, c0;     // c0: the tile index of cell j
  __device__ __forceinline__ F2 pair(int q, int n) const {
    const float *a = sm + (size_t)((2 * q) * nli + line) * nc + c0 + n;
    return F2{a[0], a[(size_t)nli * nc]};
  }
  __device__ __forceinline__ float single(int v, int n) const {
    return sm[(size_t)((2 * kF32Pair + v) * nli + line) * nc + c0 + n];
  }
};

// face interpolation (3,-25,150,150,-25,3)/256 of slot q as an increment over
// the cell value, from exact differences; c: the cell's split
template <class Src>
__device__ __forceinline__ float face6_delta(const Src &src, int q, F2 &c) {
  c = src.pair(q, 0);
  return (3.0f * f32_diff(src.pair(q, -2), c) - 25.0f * f32_diff(src.pair(q, -1), c)
          + 150.0f * f32_diff(src.pair(q, 1), c) - 25.0f * f32_diff(src.pair(q, 2), c)
          + 3.0f * f32_diff(src.pair(q, 3), c)) * (1.0f / 256.0f);
}

// The FP32 flux of face (j, k) from src; false where the face goes to the
// FP64 solver (a contrast in the stencil, or a failed FP32 HLLC: *fb set)
template <int DIR, class Src>
__device__ inline bool flux_f32(const Lev &L, const DevParams &p, const double *__restrict__ U, int j, int k,
                                const Src &src, double out[NCONS], int *fb) {
  float rmin = src.pair(0, -2).hi, rmax = rmin, qmin = src.pair(1, -2).hi, qmax = qmin;
#pragma unroll
  for (int n = -1; n <= 3; ++n) {
    const float rv = src.pair(0, n).hi, qv = src.pair(1, n).hi;
    rmin = fminf(rmin, rv); rmax = fmaxf(rmax, rv);
    qmin = fminf(qmin, qv); qmax = fmaxf(qmax, qv);
  }
  if (!(rmin > kMixedContrast * rmax && qmin > kMixedContrast * qmax)) return false;
  float pl[5], pr[5];
  {
    float c[6];
#pragma unroll
    for (int n = -2; n <= 3; ++n) {
      const F2 r = src.pair(0, n);
      c[n + 2] = r.hi + r.lo;
    }
    ppm_pair(c, pl[0], pr[0]);
  }
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    float c[6];
#pragma unroll
    for (int n = -2; n <= 3; ++n) c[n + 2] = src.single(v, n);
    ppm_pair(c, pl[v + 1], pr[v + 1]);
  }
  const F2 Ps = src.pair(1, 0);
  const float pref = Ps.hi + Ps.lo;
  {
    const float c[6] = {f32_diff(src.pair(1, -2), Ps), f32_diff(src.pair(1, -1), Ps), 0.0f,
                        f32_diff(src.pair(1, 1), Ps), f32_diff(src.pair(1, 2), Ps), f32_diff(src.pair(1, 3), Ps)};
    ppm_pair(c, pl[4], pr[4]);
    if (!(pl[0] > 0.0f) || !(pl[4] + pref > 0.0f)) {
      const F2 r = src.pair(0, 0);
      pl[0] = r.hi + r.lo;
#pragma unroll
      for (int v = 0; v < 3; ++v) pl[v + 1] = src.single(v, 0);
      pl[4] = 0.0f;
    }
    if (!(pr[0] > 0.0f) || !(pr[4] + pref > 0.0f)) {
      const F2 r = src.pair(0, 1);
      pr[0] = r.hi + r.lo;
#pragma unroll
      for (int v = 0; v < 3; ++v) pr[v + 1] = src.single(v, 1);
      pr[4] = c[3];
    }
  }
  F2 ca, cw, cb;
  const float da = face6_delta(src, 2, ca);
  const float dW = face6_delta(src, 3, cw);
  const float aj = ca.hi + ca.lo, Wj = cw.hi + cw.lo;
  const float alpha = aj + da, W = Wj + dW;
  float beta[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float d = face6_delta(src, 4 + i, cb);
    beta[i] = (cb.hi + cb.lo) + d;
  }
  Sym3T<float> g;
  float gv[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    const float d = face6_delta(src, 7 + a, cb);
    gv[a] = (cb.hi + cb.lo) + d;
  }
  g.xx = 1.0f + gv[0]; g.xy = gv[1]; g.xz = gv[2]; g.yy = 1.0f + gv[3]; g.yz = gv[4]; g.zz = 1.0f + gv[5];
  float o[5];
  *fb = face_flux<float>(p, DIR, pl, pr, alpha, beta, W, g, o, pref);
  if (*fb) return false;
  // (g_f - g_j) P_j in FP32
  const float x = da / aj, y = dW / Wj, y1 = 1.0f + y;
  const float rel = (x - y * (3.0f + y * (3.0f + y))) / (y1 * y1 * y1);
  const float gj32 = aj / (Wj * Wj * Wj);
  constexpr int n = DIR == 0 ? 1 : 3;
  o[n] += gj32 * rel * pref;
#pragma unroll
  for (int v = 0; v < NCONS; ++v) out[v] = f64_of(o[v]);
  // g_j P_j in FP64
  const size_t P = L.P;
  const int id = cid(L, j, k);
  const double aj64 = U[(size_t)fAL * P + id], Wj64 = U[(size_t)fW * P + id], Pj = L.prim[(size_t)pP * P + id];
  out[n] += aj64 * Pj / (Wj64 * Wj64 * Wj64);
  return true;
}

// the FP64 solver for the faces the FP32 form hands over (few): out of line,
// so that its registers do not weigh on the FP32 path
template <int DIR>
__device__ __noinline__ void flux_at_f64_call(const Lev &L, const DevParams &p, const double *__restrict__ U, int j,
                                              int k, double out[NCONS], int *fb) {
  flux_at_f64<DIR>(L, p, U, j, k, out, fb);
}

// The flux of one face in arithmetic T (FP32: from src, else the FP64 solver).
template <typename T, int DIR, class Src>
__device__ inline void flux_face(const Lev &L, const DevParams &p, const double *__restrict__ U, int j, int k,
                                 const Src &src, double out[NCONS], int *fb) {
  if constexpr (sizeof(T) == 4) {
    if (flux_f32<DIR>(L, p, U, j, k, src, out, fb)) return;
    flux_at_f64_call<DIR>(L, p, U, j, k, out, fb);
  } else {
    flux_at_f64<DIR>(L, p, U, j, k, out, fb);
  }
}

// The FP32 inputs of a tile's faces staged through shared memory: every cell
// of the tile's lines that a face of the region uses (cells a0-2 .. a0+nal+2
// along the normal) split once, instead of once per face that reads it (six).
// Layout and views as F32Staged; kF32Slots * nli * (nal + 5) floats.
__host__ __device__ constexpr int f32_tile_floats(int nal, int nli) { return kF32Slots * nli * (nal + 5); }

template <int DIR>
__device__ __forceinline__ void f32_tile(const Lev &L, const double *__restrict__ U, int j0, int k0, int jmax,
                                         int kmax, float *sm) {
  const int nal = DIR == 0 ? (int)blockDim.x : (int)blockDim.y, nli = DIR == 0 ? (int)blockDim.y : (int)blockDim.x;
  const int nth = (int)(blockDim.x * blockDim.y), tid = (int)(threadIdx.y * blockDim.x + threadIdx.x);
  const int nc = nal + 5;
  const int a0 = DIR == 0 ? j0 : k0, l0 = DIR == 0 ? k0 : j0;
  const int amax = DIR == 0 ? jmax : kmax, lmax = DIR == 0 ? kmax : jmax;
  const int per = nli * nc;
  // one cell per thread and pass, its sixteen loads issued together; cells
  // contiguous in memory go to neighbouring threads (along x for x-faces,
  // across the lines (columns j) for z-faces)
  for (int cell = tid; cell < per; cell += nth) {
    const int c = DIR == 0 ? cell % nc : cell / nli, line = DIR == 0 ? cell / nc : cell % nli;
    const int along = a0 - 2 + c;
    if (l0 + line > lmax || along > amax + 3) continue;
    const int j = DIR == 0 ? along : l0 + line, k = DIR == 0 ? l0 + line : along;
    const int id = cid(L, j, k);
    float *o = sm + (size_t)line * nc + c;
    double u[kF32Pair + kF32Single];
#pragma unroll
    for (int q = 0; q < kF32Pair; ++q) {
      const int f = f32_pair_field(q);
      u[q] = f < 0 ? L.prim[(size_t)(-1 - f) * L.P + id] : U[(size_t)f * L.P + id];
    }
#pragma unroll
    for (int v = 0; v < kF32Single; ++v) u[kF32Pair + v] = L.prim[(size_t)(pUX + v) * L.P + id];
#pragma unroll
    for (int q = 0; q < kF32Pair; ++q) {
      const F2 v = split_f64(u[q]);
      o[(size_t)(2 * q) * per] = v.hi;
      o[(size_t)(2 * q + 1) * per] = v.lo;
    }
#pragma unroll
    for (int v = 0; v < kF32Single; ++v) o[(size_t)(2 * kF32Pair + v) * per] = f32_of(u[kF32Pair + v]);
  }
  __syncthreads();
}

// x-faces j+1/2 for j in [0, jmax], rows [1, kmax].  Stores area-weighted
// fluxes (cylindrical: area x_{j+1/2} dz, and one more factor x for S_phi)
// and accumulates the flux registers of the refinement boundaries.
template <typename T>
__device__ __forceinline__ void flux_x_cell(const Lev &L, const DevParams &p, const double *__restrict__ U, int jmax, int kmax,
                                                 double wb, int has_child, int has_parent, int j, int k, double wbp,
                                                 const double *stage_sm = nullptr, const float *stage32 = nullptr) {
  if (j > jmax || k > kmax) return;
  double f[NCONS];
  int fb;
  if (stage_sm) {
    double pl[5], pr[5];
    ppm_tile_states<0>(stage_sm, threadIdx.x, threadIdx.y, pl, pr);
    flux_states_f64<0>(L, p, U, j, k, pl, pr, f, &fb);
  } else if (stage32) {
    const int nal = 0 == 0 ? (int)blockDim.x : (int)blockDim.y, nli = 0 == 0 ? (int)blockDim.y : (int)blockDim.x;
    const F32Staged src{stage32, nli, nal + 5, (int)threadIdx.y, (int)threadIdx.x + 2};
    flux_face<float, 0>(L, p, U, j, k, src, f, &fb);
  } else {
    const F32Global src{L.prim, U, L.P, cid(L, j, k), 1};
    flux_face<T, 0>(L, p, U, j, k, src, f, &fb);
  }
  const bool cyl = p.geometry == SACRA_CYLINDRICAL;
  const double xf = j * L.dx;
  const double area = cyl ? xf * L.dz : L.dz;
#pragma unroll
  for (int v = 0; v < NCONS; ++v) f[v] *= area;
  if (cyl) f[2] *= xf;
  const int id = cid(L, j, k);
#pragma unroll
  for (int v = 0; v < NCONS; ++v) L.fx[(size_t)v * L.P + id] = f[v];
  if (has_child && j == L.nx / 2 && k <= L.nz / 2)
#pragma unroll
    for (int v = 0; v < NCONS; ++v) L.freg[(size_t)(0 * NCONS + v) * L.rw + k] += wb * f[v];
  if (has_parent && j == L.nx && k <= L.nz)
#pragma unroll
    for (int v = 0; v < NCONS; ++v) L.freg[(size_t)(1 * NCONS + v) * L.rw + k] += wbp * f[v];
  if (fb) atomicAdd(L.nfb, 1ull);
}

template <typename T>
__global__ void __launch_bounds__(128) k_flux_x(Lev L, DevParams p, const double *__restrict__ U, int jmax, int kmax,
                                                 double wb, int has_child, int has_parent) {
  flux_x_cell<T>(L, p, U, jmax, kmax, wb, has_child, has_parent, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y + 1, wb);
}

template <typename T>
__device__ __forceinline__ void flux_z_cell(const Lev &L, const DevParams &p, const double *__restrict__ U, int jmax, int kmax,
                                                 double wb, int has_child, int has_parent, int j, int k, double wbp,
                                                 const double *stage_sm = nullptr, const float *stage32 = nullptr) {
  if (j > jmax || k > kmax) return;
  double f[NCONS];
  int fb;
  if (stage_sm) {
    double pl[5], pr[5];
    ppm_tile_states<1>(stage_sm, threadIdx.y, threadIdx.x, pl, pr);
    flux_states_f64<1>(L, p, U, j, k, pl, pr, f, &fb);
  } else if (stage32) {
    const int nal = 1 == 0 ? (int)blockDim.x : (int)blockDim.y, nli = 1 == 0 ? (int)blockDim.y : (int)blockDim.x;
    const F32Staged src{stage32, nli, nal + 5, (int)threadIdx.x, (int)threadIdx.y + 2};
    flux_face<float, 1>(L, p, U, j, k, src, f, &fb);
  } else {
    const F32Global src{L.prim, U, L.P, cid(L, j, k), L.px};
    flux_face<T, 1>(L, p, U, j, k, src, f, &fb);
  }
  const bool cyl = p.geometry == SACRA_CYLINDRICAL;
  // equatorial mirror plane: D, S_x, S_phi, E are even in z, their z-fluxes vanish there
  if (cyl && k == 0) f[0] = f[1] = f[2] = f[4] = 0.0;
  const double x = (j - 0.5) * L.dx;
  const double area = cyl ? x * L.dx : L.dx;
#pragma unroll
  for (int v = 0; v < NCONS; ++v) f[v] *= area;
  if (cyl) f[2] *= x;
  const int id = cid(L, j, k);
#pragma unroll
  for (int v = 0; v < NCONS; ++v) L.fz[(size_t)v * L.P + id] = f[v];
  if (has_child && k == L.nz / 2 && j <= L.nx / 2)
#pragma unroll
    for (int v = 0; v < NCONS; ++v) L.freg[(size_t)(2 * NCONS + v) * L.rw + j] += wb * f[v];
  if (has_parent && k == L.nz && j <= L.nx)
#pragma unroll
    for (int v = 0; v < NCONS; ++v) L.freg[(size_t)(3 * NCONS + v) * L.rw + j] += wbp * f[v];
  if (fb) atomicAdd(L.nfb, 1ull);
}

template <typename T>
__global__ void __launch_bounds__(128) k_flux_z(Lev L, DevParams p, const double *__restrict__ U, int jmax, int kmax,
                                                 double wb, int has_child, int has_parent) {
  flux_z_cell<T>(L, p, U, jmax, kmax, wb, has_child, has_parent, blockIdx.x * blockDim.x + threadIdx.x + 1, blockIdx.y * blockDim.y + threadIdx.y, wb);
}

// 6th-order central first derivative: exact differences (FP64, or FP32 from
// integer splits), weighted sum in T
template <typename T>
__device__ __forceinline__ T cd1(const double *u, int s, T idx) {
  if constexpr (sizeof(T) == 4) {
    return (45.0f * f32_diff(split_f64(u[s]), split_f64(u[-s])) - 9.0f * f32_diff(split_f64(u[2 * s]), split_f64(u[-2 * s]))
            + f32_diff(split_f64(u[3 * s]), split_f64(u[-3 * s]))) * idx;
  } else {
    return (45.0 * (u[s] - u[-s]) - 9.0 * (u[2 * s] - u[-2 * s]) + (u[3 * s] - u[-3 * s])) * idx;
  }
}

// d_t q = <s> - (1/dV) sum (area-weighted fluxes), Sec. II.C.1.  The flux
// divergence is FP64; the sources are evaluated in arithmetic T:
//   s_Sk = P d_k(alpha W^-3) - W^-3 rho h w^2 [d_k alpha - v_i d_k beta^i
//          + (W^2/2) alpha v_a v_b d_k gt^ab + (alpha/W) v_i v^i d_k W]
//        (+ alpha W^-3 (S_y vbar^y + P)/x for k = x, cylindrical),
//   s_E  = W^-3 (alpha K^ij S_ij - rho h w^2 v^i d_i alpha), s_D = s_Sphi = 0.
// DS: the level's derivative scratch of the same stage (the derivative pass
// has run), whose first derivatives of alpha, W, beta^i and gt_ij replace the
// six-point differences here in the FP64 form; nullptr: the differences are
// formed here.
template <typename T>
__device__ __forceinline__ void hydro_rhs_cell(const Lev &L, const DevParams &p, const double *__restrict__ U, int jmax,
                                               int kmax, int j, int k, const void *DS = nullptr) {
  if (j > jmax || k > kmax) return;
  const size_t P = L.P;
  const int id = cid(L, j, k);
  const int sz = L.px;
  const bool cyl = p.geometry == SACRA_CYLINDRICAL;
  const double xd = (j - 0.5) * L.dx;
  const double ivol = 1.0 / (cyl ? xd * L.dx * L.dz : L.dx * L.dz);
  double div[NCONS];
#pragma unroll
  for (int v = 0; v < NCONS; ++v) {
    const double *fx = L.fx + (size_t)v * P + id;
    const double *fz = L.fz + (size_t)v * P + id;
    div[v] = (fx[0] - fx[-1] + fz[0] - fz[-sz]) * ivol;
  }
  auto ld = [&](int f) { return ld_as<T>(U[(size_t)f * P + id]); };
  const T x = sizeof(T) == 4 ? T(((float)j - 0.5f) * f32_of(L.dx)) : T(xd);
  const T W = ld(fW), al = ld(fAL);
  Sym3T<T> g;
  if constexpr (sizeof(T) == 4) {
    g.xx = 1.0f + ld(fHXX); g.yy = 1.0f + ld(fHYY); g.zz = 1.0f + ld(fHZZ);
  } else {
    g.xx = 1.0 + U[(size_t)fHXX * P + id]; g.yy = 1.0 + U[(size_t)fHYY * P + id]; g.zz = 1.0 + U[(size_t)fHZZ * P + id];
  }
  g.xy = ld(fHXY); g.xz = ld(fHXZ); g.yz = ld(fHYZ);
  const Sym3T<T> gi = s3inv(g, (T *)nullptr);
  const T i60[2] = {ld_as<T>(L.i60x), ld_as<T>(L.i60z)};
  const int st[2] = {1, sz};
  T pr[NPRIM];
#pragma unroll
  for (int f = 0; f < NPRIM; ++f) pr[f] = ld_as<T>(L.prim[(size_t)f * P + id]);
  const T rho = pr[pRHO], Pp = pr[pP];
  const T u[3] = {pr[pUX], pr[pUY], pr[pUZ]};
  const T w = sqrt(T(1) + W * W * s3quad(gi, u, u));
  const T iw = T(1) / w;
  const T rhw2 = rho * (T(1) + pr[pEPS] + Pp / rho) * w * w;
  const T vd[3] = {u[0] * iw, u[1] * iw, u[2] * iw};
  T vu[3];
  s3vec(gi, vd, vu);
  vu[0] *= W * W; vu[1] *= W * W; vu[2] *= W * W;
  const T vv = vd[0] * vu[0] + vd[1] * vu[1] + vd[2] * vu[2];
  const T iW = T(1) / W, iW3 = iW * iW * iW;
  // gt^ac v_c, used in v_a v_b d gt^ab = -(gt^ac v_c)(gt^bd v_d) d gt_cd
  T gv[3];
  s3vec(gi, vd, gv);
  // The sources take the first derivatives the stage's derivative pass has
  // written when that pass ran in the same arithmetic (FP64 sources with the
  // FP64 pass; FP32 sources with the FP32 pass, whose stencil sums of exact
  // differences are the ones cd1 forms), else form their own
  const bool use_ds = DS != nullptr && (sizeof(T) == 8) == !(p.mixed & SACRA_MIXED_Z4C);
  // d_x (e = 0) or d_z (e = 1) of metric field f
  auto d1 = [&](int f, int e) -> T {
    if (use_ds) return reinterpret_cast<const T *>(DS)[(size_t)(DS_D1 + 3 * d1_of(f) + (e == 0 ? 0 : 2)) * P + id];
    return cd1<T>(U + (size_t)f * P + id, st[e], i60[e]);
  };
  T src[2], dal[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    dal[e] = d1(fAL, e);
    const T dW = d1(fW, e);
    T vdb = T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) vdb += vd[i] * d1(fBX + i, e);
    Sym3T<T> dg;
    dg.xx = d1(fHXX, e);
    dg.xy = d1(fHXY, e);
    dg.xz = d1(fHXZ, e);
    dg.yy = d1(fHYY, e);
    dg.yz = d1(fHYZ, e);
    dg.zz = d1(fHZZ, e);
    const T vvdgi = -s3quad(dg, gv, gv);
    const T dalW3 = iW3 * dal[e] - T(3) * al * iW3 * iW * dW;
    src[e] = Pp * dalW3 - iW3 * rhw2 * (dal[e] - vdb + T(0.5) * W * W * al * vvdgi + al * iW * vv * dW);
  }
  T geo = T(0);
  if (cyl) {
    const T vbary = vu[1] - ld(fBY) / al;
    geo = al * iW3 * (rhw2 * vd[1] * vbary + Pp) / x;
  }
  // K^ij S_ij = rho h w^2 K_ij v^i v^j + P gamma^ij K_ij, K_ij = (At_ij + gt_ij K/3) / W^2
  T K;
  if constexpr (sizeof(T) == 4) K = ld(fKH) + 2.0f * ld(fTH);
  else K = U[(size_t)fKH * P + id] + 2.0 * U[(size_t)fTH * P + id];
  Sym3T<T> Kd;
  const T K3 = K * T(1.0 / 3.0), iW2 = iW * iW;
  Kd.xx = (ld(fAXX) + g.xx * K3) * iW2;
  Kd.xy = (ld(fAXY) + g.xy * K3) * iW2;
  Kd.xz = (ld(fAXZ) + g.xz * K3) * iW2;
  Kd.yy = (ld(fAYY) + g.yy * K3) * iW2;
  Kd.yz = (ld(fAYZ) + g.yz * K3) * iW2;
  Kd.zz = (ld(fAZZ) + g.zz * K3) * iW2;
  // gamma^ij K_ij = W^2 gt^ij K_ij (equal to K when At is trace-free)
  const T trK = W * W * (gi.xx * Kd.xx + gi.yy * Kd.yy + gi.zz * Kd.zz
                         + T(2) * (gi.xy * Kd.xy + gi.xz * Kd.xz + gi.yz * Kd.yz));
  const T KS = rhw2 * s3quad(Kd, vu, vu) + Pp * trK;
  const T sE = iW3 * (al * KS - rhw2 * (vu[0] * dal[0] + vu[2] * dal[1]));
  double *rq = L.rhsq + id;     // planes d_t q_D, q_Sx, q_Sy, q_Sz, q_E
  rq[0] = -div[0];
  rq[P] = to_f64<T>(src[0] + geo) - div[1];
  rq[2 * P] = -div[2];
  rq[3 * P] = to_f64<T>(src[1]) - div[3];
  rq[4 * P] = to_f64<T>(sE) - div[4];
}

template <typename T>
__global__ void __launch_bounds__(128) k_hydro_rhs(Lev L, DevParams p, const double *__restrict__ U, int jmax, int kmax) {
  hydro_rhs_cell<T>(L, p, U, jmax, kmax, blockIdx.x * blockDim.x + threadIdx.x + 1, blockIdx.y * blockDim.y + threadIdx.y + 1);
}

// eps from the EOS and conserved variables on every padded cell (initial data)
__global__ void k_prim2cons_all(Lev L, DevParams p, double *__restrict__ U) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.px * L.pz) return;
  const size_t P = L.P;
  double pr[NPRIM];
#pragma unroll
  for (int f = 0; f < NPRIM; ++f) pr[f] = L.prim[(size_t)f * P + i];
  if (p.adiabatic) {                    // zero temperature
    pr[pP] = eos_pc(p, pr[pRHO]);
    L.prim[(size_t)pP * P + i] = pr[pP];
  }
  pr[pEPS] = eos_eps(p, pr[pRHO], pr[pP]);
  L.prim[(size_t)pEPS * P + i] = pr[pEPS];
  const int j = i % L.px - GH + 1;
  const double x = (j - 0.5) * L.dx;
  const Sym3 g = conf_metric(U, P, i);
  double q[NCONS];
  prim_to_cons(p, pr, U[(size_t)fW * P + i], g, x, q);
#pragma unroll
  for (int v = 0; v < NCONS; ++v) U[(size_t)(fQD + v) * P + i] = q[v];
}

// primitive recovery on [j0, j1] x [k0, k1] of state U
__device__ __forceinline__ void c2p_region_body(const Lev &L, const DevParams &p, double *__restrict__ U, int j0, int j1,
                                                int k0, int k1, int skip_corner, int bx, int by) {
  const int j = j0 + (int)(bx * blockDim.x + threadIdx.x);
  const int k = k0 + (int)(by * blockDim.y + threadIdx.y);
  if (j > j1 || k > k1 || (skip_corner && j == j1 && k == k1)) return;
  const size_t P = L.P;
  const int id = cid(L, j, k);
  double q[NCONS], pr[NPRIM];
#pragma unroll
  for (int v = 0; v < NCONS; ++v) q[v] = U[(size_t)(fQD + v) * P + id];
  const Sym3 g = conf_metric(U, P, id);
  const int st = cons_to_prim(p, q, U[(size_t)fW * P + id], g, (j - 0.5) * L.dx, pr);
#pragma unroll
  for (int f = 0; f < NPRIM; ++f) L.prim[(size_t)f * P + id] = pr[f];
  if ((st & (ST_ATM | ST_COLD | ST_KRESCALE)) || p.adiabatic)   // the adiabatic recovery always rebuilds E
#pragma unroll
    for (int v = 0; v < NCONS; ++v) U[(size_t)(fQD + v) * P + id] = q[v];
  L.status[id] = st;
}

__global__ void k_c2p_region(Lev L, DevParams p, double *__restrict__ U, int j0, int j1, int k0, int k1, int skip_corner) {
  c2p_region_body(L, p, U, j0, j1, k0, k1, skip_corner, blockIdx.x, blockIdx.y);
}

// primitive recovery on the parent cells a restriction and reflux changed,
// [1, N/2 + 1]^2 without the corner, of every item of a level list
__global__ void kl_c2p_restricted(const LItem *__restrict__ items) {
  const LItem &it = items[blockIdx.z];
  const int nh = it.Pa.nx / 2;
  c2p_region_body(it.Pa, it.P, it.Pa.un, 1, nh + 1, 1, nh + 1, 1, blockIdx.x, blockIdx.y);
}

void launch_l_c2p_restricted(const LItem *items, int n, int max_nx, cudaStream_t s) {
  if (n <= 0) return;
  const int nh = max_nx / 2;                  // the largest parent's N/2
  dim3 b(32, 4), g((nh + 1 + 31) / 32, (nh + 1 + 3) / 4, n);
  kl_c2p_restricted<<<g, b, 0, s>>>(items);
}

// ---------------------------------------------------------------- batched persistent kernels
//
// One launch covers the tiles of every level of every star in a batch: each
// block walks the tile list with a grid stride; a tile is one block's worth of
// cells of one level (origin j0, k0; extent = the block shape).
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 0) kb_flux_x(Batch b, DevParams p) {
  for_tiles(b, [&](const BL &q, const Tile &tl) {
    flux_x_cell<T>(q.L, q.P, q.U, q.jmax, q.kmax, q.wb, q.has_child, q.has_parent, tl.j0 + threadIdx.x, tl.k0 + threadIdx.y, q.wbp);
  });
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 0) kb_flux_z(Batch b, DevParams p) {
  for_tiles(b, [&](const BL &q, const Tile &tl) {
    flux_z_cell<T>(q.L, q.P, q.U, q.jmax, q.kmax, q.wb, q.has_child, q.has_parent, tl.j0 + threadIdx.x, tl.k0 + threadIdx.y, q.wbp);
  });
}

// FP64 faces with the PPM staged through shared memory (dynamic buffer of
// ppm_tile_doubles(...) doubles)
__global__ void __launch_bounds__(256, 2) kb_flux_x_st(Batch b, DevParams p) {
  extern __shared__ double ppm_sm[];
  for_tiles(b, [&](const BL &q, const Tile &tl) {
    ppm_tile<0>(q.L, tl.j0, tl.k0, q.jmax, q.kmax, ppm_sm);
    flux_x_cell<double>(q.L, q.P, q.U, q.jmax, q.kmax, q.wb, q.has_child, q.has_parent, tl.j0 + threadIdx.x,
                        tl.k0 + threadIdx.y, q.wbp, ppm_sm);
  });
}

__global__ void __launch_bounds__(256, 2) kb_flux_z_st(Batch b, DevParams p) {
  extern __shared__ double ppm_sm[];
  for_tiles(b, [&](const BL &q, const Tile &tl) {
    ppm_tile<1>(q.L, tl.j0, tl.k0, q.jmax, q.kmax, ppm_sm);
    flux_z_cell<double>(q.L, q.P, q.U, q.jmax, q.kmax, q.wb, q.has_child, q.has_parent, tl.j0 + threadIdx.x,
                        tl.k0 + threadIdx.y, q.wbp, ppm_sm);
  });
}

// FP32 faces with their inputs staged through shared memory (dynamic buffer
// of f32_tile_floats(...) floats)
__global__ void __launch_bounds__(256, 2) kb_flux_x_st32(Batch b, DevParams p) {
  extern __shared__ float f32_sm[];
  for_tiles(b, [&](const BL &q, const Tile &tl) {
    f32_tile<0>(q.L, q.U, tl.j0, tl.k0, q.jmax, q.kmax, f32_sm);
    flux_x_cell<float>(q.L, q.P, q.U, q.jmax, q.kmax, q.wb, q.has_child, q.has_parent, tl.j0 + threadIdx.x,
                       tl.k0 + threadIdx.y, q.wbp, nullptr, f32_sm);
  });
}

__global__ void __launch_bounds__(256, 2) kb_flux_z_st32(Batch b, DevParams p) {
  extern __shared__ float f32_sm[];
  for_tiles(b, [&](const BL &q, const Tile &tl) {
    f32_tile<1>(q.L, q.U, tl.j0, tl.k0, q.jmax, q.kmax, f32_sm);
    flux_z_cell<float>(q.L, q.P, q.U, q.jmax, q.kmax, q.wb, q.has_child, q.has_parent, tl.j0 + threadIdx.x,
                       tl.k0 + threadIdx.y, q.wbp, nullptr, f32_sm);
  });
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 0) kb_hydro_rhs(Batch b, DevParams p) {
  for_tiles(b, [&](const BL &q, const Tile &tl) {
    hydro_rhs_cell<T>(q.L, q.P, q.U, q.jmax, q.kmax, tl.j0 + threadIdx.x, tl.k0 + threadIdx.y,
                      q.P.evolve ? q.DS : nullptr);
  });
}

// The FP64 faces always stage their PPM (one kernel per direction, so every
// tile shape gives the same values), the FP32 faces their split inputs (the
// staged and per-face forms give the same values); a shape whose buffer would
// pass the 48 KB a launch may take without opting in keeps the per-face form.
constexpr size_t kPpmSmemMax = 48 * 1024;

void launch_b_flux_x(const Batch &b, const DevParams &p, cudaStream_t s) {
  if (b.ntiles <= 0) return;
  if (p.mixed & SACRA_MIXED_FLUX) {
    const size_t sm = f32_tile_floats(b.block.x, b.block.y) * sizeof(float);
    if (sm <= kPpmSmemMax) kb_flux_x_st32<<<b.grid, b.block, sm, s>>>(b, p);
    else kb_flux_x<float><<<b.grid, b.block, 0, s>>>(b, p);
    return;
  }
  const size_t sm = ppm_tile_doubles(b.block.x, b.block.y) * sizeof(double);
  if (sm <= kPpmSmemMax) kb_flux_x_st<<<b.grid, b.block, sm, s>>>(b, p);
  else kb_flux_x<double><<<b.grid, b.block, 0, s>>>(b, p);
}

void launch_b_flux_z(const Batch &b, const DevParams &p, cudaStream_t s) {
  if (b.ntiles <= 0) return;
  if (p.mixed & SACRA_MIXED_FLUX) {
    const size_t sm = f32_tile_floats(b.block.y, b.block.x) * sizeof(float);
    if (sm <= kPpmSmemMax) kb_flux_z_st32<<<b.grid, b.block, sm, s>>>(b, p);
    else kb_flux_z<float><<<b.grid, b.block, 0, s>>>(b, p);
    return;
  }
  const size_t sm = ppm_tile_doubles(b.block.y, b.block.x) * sizeof(double);
  if (sm <= kPpmSmemMax) kb_flux_z_st<<<b.grid, b.block, sm, s>>>(b, p);
  else kb_flux_z<double><<<b.grid, b.block, 0, s>>>(b, p);
}

void launch_b_hydro_div(const Batch &b, const DevParams &p, cudaStream_t s) {
  if (b.ntiles <= 0) return;
  if (p.mixed & SACRA_MIXED_SOURCES) kb_hydro_rhs<float><<<b.grid, b.block, 0, s>>>(b, p);
  else kb_hydro_rhs<double><<<b.grid, b.block, 0, s>>>(b, p);
}

// ---------------------------------------------------------------- host launchers

void launch_flux_x(const Lev &L, const DevParams &p, const double *U, int jmax, int kmax, double wb, int has_child,
                   int has_parent, cudaStream_t s) {
  const dim3 g((jmax + 1 + 31) / 32, (kmax + 3) / 4), b(32, 4);
  if (p.mixed & SACRA_MIXED_FLUX) k_flux_x<float><<<g, b, 0, s>>>(L, p, U, jmax, kmax, wb, has_child, has_parent);
  else k_flux_x<double><<<g, b, 0, s>>>(L, p, U, jmax, kmax, wb, has_child, has_parent);
}

void launch_flux_z(const Lev &L, const DevParams &p, const double *U, int jmax, int kmax, double wb, int has_child,
                   int has_parent, cudaStream_t s) {
  const dim3 g((jmax + 31) / 32, (kmax + 1 + 3) / 4), b(32, 4);
  if (p.mixed & SACRA_MIXED_FLUX) k_flux_z<float><<<g, b, 0, s>>>(L, p, U, jmax, kmax, wb, has_child, has_parent);
  else k_flux_z<double><<<g, b, 0, s>>>(L, p, U, jmax, kmax, wb, has_child, has_parent);
}

void launch_hydro_div(const Lev &L, const DevParams &p, const double *U, int jmax, int kmax, cudaStream_t s) {
  const dim3 g((jmax + 31) / 32, (kmax + 3) / 4), b(32, 4);
  if (p.mixed & SACRA_MIXED_SOURCES) k_hydro_rhs<float><<<g, b, 0, s>>>(L, p, U, jmax, kmax);
  else k_hydro_rhs<double><<<g, b, 0, s>>>(L, p, U, jmax, kmax);
}

void launch_prim2cons_all(const Lev &L, const DevParams &p, double *U, cudaStream_t s) {
  k_prim2cons_all<<<(unsigned)((L.P + 255) / 256), 256, 0, s>>>(L, p, U);
}

void launch_c2p_region(const Lev &L, const DevParams &p, double *U, int j0, int j1, int k0, int k1, cudaStream_t s,
                       int skip_corner) {
  dim3 b(32, 4), g((j1 - j0 + 1 + 31) / 32, (k1 - k0 + 1 + 3) / 4);
  k_c2p_region<<<g, b, 0, s>>>(L, p, U, j0, j1, k0, k1, skip_corner);
}

}  // namespace sacra
