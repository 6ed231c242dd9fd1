// Z4c right-hand side kernels on sm_103a (Lam & Shibata, arXiv:2502.03223,
// Sec. II.B): cartoon y-derivatives (Sec. II.B.2), 6th-order central,
// lopsided and mixed differences, 8th-order Kreiss-Oliger dissipation, and the
// pointwise right-hand side.  Three passes per level and stage:
//   k_cartoon:    interpolate-and-rotate planes y = +-m dy -> d_y, d_yy scratch
//   k_z4c_derivs: all x/z/mixed derivatives, advection + KO -> derivative scratch
//   k_z4c_point:  pointwise Z4c algebra -> rhs
#include <type_traits>

#include "kernels.h"
#include "z4c.cuh"
#include "fixed.cuh"

namespace sacra {

// fields that are interpolated onto the cartoon planes
__constant__ int kCartoonFields[20] = {fW,   fAL,  fHXX, fHXY, fHXZ, fHYY, fHYZ, fHZZ, fAXX, fAXY,
                                       fAXZ, fAYY, fAYZ, fBX,  fBY,  fBZ,  fGX,  fGY,  fBBX, fBBY};

__device__ __forceinline__ double par_x(int f) {
  switch (f) {
    case fGX: case fGY: case fBX: case fBY: case fBBX: case fBBY:
    case fHXZ: case fHYZ: case fAXZ: case fAYZ:
      return -1.0;
    default:
      return 1.0;
  }
}

// x-parity of the cartoon fields in kCartoonFields order (compile-time form)
__host__ __device__ constexpr float par_x_slot(int a) {
  return (a == 4 || a == 6 || a == 10 || a == 12 || a == 13 || a == 14 || a == 16 || a == 17 || a == 18 || a == 19)
             ? -1.0f : 1.0f;
}

// d_y and d_yy at (x_j, z_k) by the cartoon method (Sec. II.B.2): the planes
// y = +-m dy (m = 1..3, dy = dx) hold the 9-point Lagrange interpolant in x at
// varpi_m = sqrt(x_j^2 + (m dy)^2), rotated by +-phi_m, and d_y, d_yy are the
// 6th-order central differences over the seven planes.  All three steps are
// linear in the nine values u(x_{j-4..j+4}), so each output is one 9-point
// sum with per-column weights (kernels.h, built on the host from the same
// interpolation weights): a scalar's d_yy; a vector's d_y from its other
// component and its d_yy; a symmetric tensor's d_y from the rotated
// components and its d_yy from the pairs (xx, yy), xy, xz, yz.  Second
// derivatives are taken on u_n - u_0 (exact zero on constants).  Columns
// j <= 0 are the rotation by pi of column 1 - j: d_y there is -parity times
// the value at 1 - j, d_yy parity times it.
__device__ __forceinline__ void cartoon_f64_cell(const Lev &L, const double *__restrict__ U,
                                                 const double *__restrict__ tabw, int j, int k) {
  if (j > L.nx + 4 || k > L.nz + 7) return;
  const bool flip = j <= 0;
  const int jj = flip ? 1 - j : j;
  const size_t P = L.P;
  const int c0 = cid(L, jj, k) - 4;
  const int o = cid(L, j, k);
  const double *Wt = tabw + (size_t)jj * kCartoonW;
  const double *Sd = Wt, *D1 = Wt + 9, *E1 = Wt + 18, *C2 = Wt + 27, *F = Wt + 36, *G = Wt + 45, *H = Wt + 54;
  const double K2 = Wt[63], Kb = Wt[64];
  const double i1 = L.i60x, i2 = L.i180x;
  auto ld = [&](int f, int n) { return U[(size_t)f * P + c0 + n]; };
  auto st1 = [&](int f, double v) { L.dy[(size_t)f * P + o] = (flip ? -par_x(f) * v : v) * i1; };
  auto st2 = [&](int f, double v) { L.dyy[(size_t)f * P + o] = (flip ? par_x(f) * v : v) * i2; };
  // scalars under the rotation: W, alpha, h_zz, beta^z (d_y = 0)
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int f = q == 0 ? fW : (q == 1 ? fAL : (q == 2 ? fHZZ : fBZ));
    const double u0 = ld(f, 4);
    double s = 0.0;
#pragma unroll
    for (int n = 0; n < 9; ++n)
      if (n != 4) s += Sd[n] * (ld(f, n) - u0);
    st2(f, s);
  }
  // vectors (x, y components): beta (d_y, d_yy), Gt and B (d_y)
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int fx_ = q == 0 ? fBX : (q == 1 ? fGX : fBBX), fy_ = fx_ + 1;
    double sx = 0.0, sy = 0.0;
#pragma unroll
    for (int n = 0; n < 9; ++n) {
      sx += D1[n] * ld(fy_, n);
      sy += D1[n] * ld(fx_, n);
    }
    st1(fx_, sx);
    st1(fy_, -sy);
    if (q == 0) {
      const double x0 = ld(fx_, 4), y0 = ld(fy_, 4);
      double ax = K2 * x0, ay = K2 * y0;
#pragma unroll
      for (int n = 0; n < 9; ++n)
        if (n != 4) {
          ax += C2[n] * (ld(fx_, n) - x0);
          ay += C2[n] * (ld(fy_, n) - y0);
        }
      st2(fx_, ax);
      st2(fy_, ay);
    }
  }
  // symmetric tensors h_ij (d_y, d_yy) and At_ij (d_y): components xx, xy, xz, yy, yz
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int f0 = q == 0 ? fHXX : fAXX;
    double exy = 0.0, exxyy = 0.0, dxz = 0.0, dyz = 0.0;
#pragma unroll
    for (int n = 0; n < 9; ++n) {
      exy += E1[n] * ld(f0 + 1, n);
      exxyy += E1[n] * (ld(f0, n) - ld(f0 + 3, n));
      dxz += D1[n] * ld(f0 + 4, n);
      dyz += D1[n] * ld(f0 + 2, n);
    }
    st1(f0, exy);
    st1(f0 + 3, -exy);
    st1(f0 + 1, -0.5 * exxyy);
    st1(f0 + 2, dxz);
    st1(f0 + 4, -dyz);
    if (q == 0) {
      const double xx0 = ld(f0, 4), xy0 = ld(f0 + 1, 4), xz0 = ld(f0 + 2, 4), yy0 = ld(f0 + 3, 4), yz0 = ld(f0 + 4, 4);
      double axx = Kb * (yy0 - xx0), ayy = Kb * (xx0 - yy0), axy = -2.0 * Kb * xy0, axz = K2 * xz0, ayz = K2 * yz0;
#pragma unroll
      for (int n = 0; n < 9; ++n)
        if (n != 4) {
          const double dxx = ld(f0, n) - xx0, dyy = ld(f0 + 3, n) - yy0;
          axx += F[n] * dxx + G[n] * dyy;
          ayy += G[n] * dxx + F[n] * dyy;
          axy += H[n] * (ld(f0 + 1, n) - xy0);
          axz += C2[n] * (ld(f0 + 2, n) - xz0);
          ayz += C2[n] * (ld(f0 + 4, n) - yz0);
        }
      st2(f0, axx);
      st2(f0 + 1, axy);
      st2(f0 + 2, axz);
      st2(f0 + 3, ayy);
      st2(f0 + 4, ayz);
    }
  }
}

__global__ void __launch_bounds__(128) k_cartoon_f64(Lev L, const double *__restrict__ U, const double *__restrict__ tabw) {
  cartoon_f64_cell(L, U, tabw, blockIdx.x * blockDim.x + threadIdx.x - 2, blockIdx.y * blockDim.y + threadIdx.y - 2);
}

// Mixed precision: the same planes in FP32, formed as differences from the
// centre value so that their small variations keep FP32 relative precision:
// the interpolation sums FP64 differences u_n - u_j with FP32 weights, and the
// rotation is applied to (base - centre) analytically.
__device__ __forceinline__ void deltas_vec(float c1, float sn, float ux, float uy, float sx, float sy, float &dxp,
                                           float &dyp) {
  // (R(u + s))_x - u_x, (R(u + s))_y - u_y with c1 = cos phi - 1
  dxp = c1 * ux - sn * uy + (c1 + 1.0f) * sx - sn * sy;
  dyp = sn * ux + c1 * uy + sn * sx + (c1 + 1.0f) * sy;
}

// tensor components xx,xy,xz,yy,yz(,zz) of u (centre) and s (interpolated - centre)
__device__ __forceinline__ void deltas_ten(float c1, float sn, const float u[5], const float s[5], float d[5]) {
  const float c = c1 + 1.0f, s2 = sn * sn, cs = c * sn;
  // R u R^T - u (uses c^2 - 1 = -sn^2) plus R s R^T
  d[0] = s2 * (u[3] - u[0]) - 2.0f * cs * u[1] + (c * c * s[0] - 2.0f * cs * s[1] + s2 * s[3]);
  d[1] = cs * (u[0] - u[3]) - 2.0f * s2 * u[1] + (cs * (s[0] - s[3]) + (c * c - s2) * s[1]);
  d[2] = c1 * u[2] - sn * u[4] + (c * s[2] - sn * s[4]);
  d[3] = s2 * (u[0] - u[3]) + 2.0f * cs * u[1] + (s2 * s[0] + 2.0f * cs * s[1] + c * c * s[3]);
  d[4] = sn * u[2] + c1 * u[4] + (sn * s[2] + c * s[4]);
}

// The nine x-neighbours u(x_{jj-4+n}, z_k), n = 0..8, of a cell's stencil as
// FP32 splits: read and split per cell (Cartoon32Global) or from a tile's
// row staged in shared memory (Cartoon32Staged); both give the same values.
struct Cartoon32Global {
  const double *U;
  size_t P;
  int c0;                  // cid(jj - 4, k)
  __device__ __forceinline__ F2 at(int a, int n) const { return split_f64(U[(size_t)kCartoonFields[a] * P + c0 + n]); }
};
struct Cartoon32Staged {
  const float *sm;         // [2 a (+1 for lo)][row][column], columns from the tile's base column
  int per, nc, row, c0;    // per = rows * nc; c0: the column of jj - 4
  __device__ __forceinline__ F2 at(int a, int n) const {
    const float *h = sm + (size_t)(2 * a) * per + (size_t)row * nc + c0 + n;
    return F2{h[0], h[per]};
  }
};

// the tile's stencil columns, base = (smallest jj of the tile) - 4 .. base + bx + 7
__host__ __device__ constexpr int cartoon32_tile_floats(int bx, int by) { return 2 * 20 * by * (bx + 8); }
__device__ __forceinline__ int cartoon32_base(int j0) { return (j0 >= 1 ? j0 : 1) - 4; }

__device__ __forceinline__ void cartoon32_tile(const Lev &L, const double *__restrict__ U, int j0, int k0, float *sm) {
  const int bx = (int)blockDim.x, by = (int)blockDim.y, nc = bx + 8, per = by * nc;
  const int nth = bx * by, tid = (int)(threadIdx.y * blockDim.x + threadIdx.x);
  const int base = cartoon32_base(j0);
  const size_t P = L.P;
  for (int e = tid; e < per; e += nth) {              // one stencil point per thread and pass, its 20 fields together
    const int c = e % nc, row = e / nc;
    const int j = base + c, k = k0 + row;
    if (j > L.nx + GH || k > L.nz + 7) continue;      // past every stencil of the region's cells
    const int id = cid(L, j, k);
    double u[20];
#pragma unroll
    for (int a = 0; a < 20; ++a) u[a] = U[(size_t)kCartoonFields[a] * P + id];
#pragma unroll
    for (int a = 0; a < 20; ++a) {
      const F2 v = split_f64(u[a]);
      sm[(size_t)(2 * a) * per + e] = v.hi;
      sm[(size_t)(2 * a + 1) * per + e] = v.lo;
    }
  }
  __syncthreads();
}

template <class Src>
__device__ __forceinline__ void cartoon_f32_cell(const Lev &L, const Src &src, const double *__restrict__ tab,
                                                 int tab_stride, int j, int k) {
  if (j > L.nx + 4 || k > L.nz + 7) return;
  const bool flip = j <= 0;
  const int jj = flip ? 1 - j : j;
  const size_t P = L.P;
  float w[3][9], cm1[3], sn[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const double *t = tab + (size_t)(jj * 3 + m) * tab_stride;   // 9 weights, cos, sin, cos - 1
#pragma unroll
    for (int n = 0; n < 9; ++n) w[m][n] = f32_of(t[n]);
    sn[m] = f32_of(t[10]);
    cm1[m] = f32_of(t[11]);
  }
  // interpolated minus centre value on the three planes, from exact FP64 differences
  float u0[20], sv[3][20];
#pragma unroll
  for (int a = 0; a < 20; ++a) {
    const F2 c = src.at(a, 4);
    u0[a] = c.hi + c.lo;
    float dn[9];
#pragma unroll
    for (int n = 0; n < 9; ++n) dn[n] = n == 4 ? 0.0f : f32_diff(src.at(a, n), c);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      float acc = 0.0f;
#pragma unroll
      for (int n = 0; n < 9; ++n) acc += w[m][n] * dn[n];
      sv[m][a] = acc;
    }
  }
  float d1[20], d2[20];
#pragma unroll
  for (int a = 0; a < 20; ++a) { d1[a] = 0.0f; d2[a] = 0.0f; }
  const float c1w[3] = {45.0f, -9.0f, 1.0f}, c2w[3] = {270.0f, -27.0f, 2.0f};
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const float c1 = cm1[m], s1 = sn[m];
    const float *v = sv[m];
    float dp[20], dm[20];   // plane (+m), plane (-m) minus centre, at jj
    dp[0] = dm[0] = v[0];
    dp[1] = dm[1] = v[1];
    deltas_ten(c1, s1, u0 + 2, v + 2, dp + 2);
    deltas_ten(c1, -s1, u0 + 2, v + 2, dm + 2);
    dp[7] = dm[7] = v[7];                 // h_zz
    deltas_ten(c1, s1, u0 + 8, v + 8, dp + 8);
    deltas_ten(c1, -s1, u0 + 8, v + 8, dm + 8);
    deltas_vec(c1, s1, u0[13], u0[14], v[13], v[14], dp[13], dp[14]);
    deltas_vec(c1, -s1, u0[13], u0[14], v[13], v[14], dm[13], dm[14]);
    dp[15] = dm[15] = v[15];              // beta^z
    deltas_vec(c1, s1, u0[16], u0[17], v[16], v[17], dp[16], dp[17]);
    deltas_vec(c1, -s1, u0[16], u0[17], v[16], v[17], dm[16], dm[17]);
    deltas_vec(c1, s1, u0[18], u0[19], v[18], v[19], dp[18], dp[19]);
    deltas_vec(c1, -s1, u0[18], u0[19], v[18], v[19], dm[18], dm[19]);
    const float w1 = c1w[m], w2 = c2w[m];
#pragma unroll
    for (int a = 0; a < 20; ++a) {
      // at flipped points the +m plane is par * (-m plane of jj) and vice versa
      const float pr = par_x_slot(a);
      const float plus = flip ? pr * dm[a] : dp[a];
      const float minus = flip ? pr * dp[a] : dm[a];
      d1[a] += w1 * (plus - minus);
      d2[a] += w2 * (plus + minus);
    }
  }
  // FP32 planes (same plane stride as the FP64 layout)
  float *dyf = reinterpret_cast<float *>(L.dy);
  float *dyyf = reinterpret_cast<float *>(L.dyy);
  const int o = cid(L, j, k);
  const float i1 = (float)(1.0 / (60.0 * L.dx)), i2 = (float)(1.0 / (180.0 * L.dx * L.dx));
#pragma unroll
  for (int a = 2; a < 20; ++a) {
    const int f = kCartoonFields[a];
    if (f == fHZZ || f == fBZ) continue;
    dyf[(size_t)f * P + o] = d1[a] * i1;
  }
  const int sec[11] = {0, 1, 2, 3, 4, 5, 6, 7, 13, 14, 15};
#pragma unroll
  for (int b = 0; b < 11; ++b) dyyf[(size_t)kCartoonFields[sec[b]] * P + o] = d2[sec[b]] * i2;
}

__global__ void __launch_bounds__(128) k_cartoon_f32(Lev L, const double *__restrict__ U, const double *__restrict__ tab,
                                                     int tab_stride) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x - 2, k = blockIdx.y * blockDim.y + threadIdx.y - 2;
  if (j > L.nx + 4 || k > L.nz + 7) return;
  const Cartoon32Global src{U, L.P, cid(L, j <= 0 ? 1 - j : j, k) - 4};
  cartoon_f32_cell(L, src, tab, tab_stride, j, k);
}

// ---------------------------------------------------------------- derivative pass

// derivative scratch layout (planes): D1 first derivatives of the 16 fields
// below (3 planes each), D2 second derivatives of 11 fields (6 planes each),
// AK advection + KO of all 25 fields.
__constant__ int kD1Fields[16] = {fW, fHXX, fHXY, fHXZ, fHYY, fHYZ, fHZZ, fKH, fGX, fGY, fGZ, fTH, fAL, fBX, fBY, fBZ};
__constant__ int kD2Fields[11] = {fW, fHXX, fHXY, fHXZ, fHYY, fHYZ, fHZZ, fAL, fBX, fBY, fBZ};

__device__ __forceinline__ bool y_zero(int f) {
  return f == fW || f == fKH || f == fTH || f == fAL || f == fGZ || f == fBZ || f == fBBZ || f == fHZZ || f == fAZZ;
}

// Stencils: the differences of the FP64 data are always taken in FP64; the
// weighted sums run in arithmetic T (FP64, or FP32 in the mixed form).
template <typename T>
__device__ __forceinline__ T fd1(const double *u, int s, T idx) {
  return (T(45) * T(u[s] - u[-s]) - T(9) * T(u[2 * s] - u[-2 * s]) + T(u[3 * s] - u[-3 * s])) * idx;
}
template <typename T>
__device__ __forceinline__ T fd2(const double *u, int s, T idx2) {
  const double u0 = u[0];
  return (T(270) * (T(u[s] - u0) + T(u[-s] - u0)) - T(27) * (T(u[2 * s] - u0) + T(u[-2 * s] - u0))
          + T(2) * (T(u[3 * s] - u0) + T(u[-3 * s] - u0))) * idx2;
}
// upwind-biased 6th-order derivative in the direction of the advecting velocity
template <typename T>
__device__ __forceinline__ T fdlop(const double *u, int s, T v, T idx) {
  if (v == T(0)) return T(0);
  const int t = v > T(0) ? s : -s;
  const double u0 = u[0];
  const T r = T(2) * T(u[-2 * t] - u0) - T(24) * T(u[-t] - u0) + T(80) * T(u[t] - u0) - T(30) * T(u[2 * t] - u0)
            + T(8) * T(u[3 * t] - u0) - T(u[4 * t] - u0);
  return (v > T(0) ? r : -r) * idx;
}
template <typename T>
__device__ __forceinline__ T fdko(const double *u, int s) {
  const double u0 = u[0];
  return (T(u[4 * s] - u0) + T(u[-4 * s] - u0)) - T(8) * (T(u[3 * s] - u0) + T(u[-3 * s] - u0))
       + T(28) * (T(u[2 * s] - u0) + T(u[-2 * s] - u0)) - T(56) * (T(u[s] - u0) + T(u[-s] - u0));
}


// Mixed-precision derivative pass.  The block stages each field's tile with
// a 4-cell halo in shared memory as FP32 (hi, lo) splits (integer bit
// operations, no FP64 instruction), so every stencil difference is one
// rounding of the exact FP64 difference, and the weighted sums run in FP32.
// Outputs (the derivative scratch, same plane layout as the FP64 pass) are
// FP32; the cartoon planes it reads are FP32 as well.
constexpr int DTX = 32, DTZ = 8, DHX = DTX + 8, DHZ = DTZ + 8;

// calls fn(std::integral_constant<int, F>) for F = F0 .. NMET - 1 (compile-time field loop)
template <int F0>
struct FieldLoop {
  template <class Fn>
  __device__ __forceinline__ static void run(Fn &&fn) {
    fn(std::integral_constant<int, F0>{});
    FieldLoop<F0 + 1>::run(fn);
  }
};
template <>
struct FieldLoop<NMET> {
  template <class Fn>
  __device__ __forceinline__ static void run(Fn &&) {}
};

__host__ __device__ constexpr bool y_zero_c(int f) {
  return f == fW || f == fKH || f == fTH || f == fAL || f == fGZ || f == fBZ || f == fBBZ || f == fHZZ || f == fAZZ;
}

// one block = one tile of DTX x DTZ cells with origin (j0, k0)
// The field loop is double-buffered: the loads of field f + 1 are issued
// before field f's stencils run from the other buffer, and one barrier per
// field separates a buffer's last reads from its next writes.
constexpr int kStagePer = (DHX * DHZ + DTX * DTZ - 1) / (DTX * DTZ);   // staged points per thread and field
__device__ __forceinline__ void z4c_derivs_f32_tile(const Lev &L, const DevParams &p, const double *__restrict__ U,
                                                    float *__restrict__ DS, int jmax, int kmax, int cyl, int j0, int k0,
                                                    float2 (*tiles)[DHZ][DHX]) {
  const int tx = threadIdx.x, tz = threadIdx.y, tid = tz * DTX + tx;
  const int j = j0 + tx, k = k0 + tz;
  const bool live = j <= jmax && k <= kmax;
  const size_t P = L.P;
  const int id = cid(L, live ? j : 1, live ? k : 1);
  const int jlim = L.nx + GH, klim = L.nz + GH;
  const float *dyf = reinterpret_cast<const float *>(L.dy);
  const float *dyyf = reinterpret_cast<const float *>(L.dyy);
  const float i60x = L.f.i60x, i60z = L.f.i60z, i180x = L.f.i180x, i180z = L.f.i180z, ixz = L.f.ixz;
  const float ko = p.fko;
  const float ikx = L.f.idx, ikz = L.f.idz;
  const bool edge = cyl && j > L.nx;
  const float bx = f32_of(U[(size_t)fBX * P + id]), by = f32_of(U[(size_t)fBY * P + id]),
              bz = f32_of(U[(size_t)fBZ * P + id]);
  float ev[7], ed[7];   // edge formula: values and d_x of h_xx, h_xy, h_xz, h_yy, h_yz, beta^x, beta^y
#pragma unroll
  for (int q = 0; q < 7; ++q) ev[q] = ed[q] = 0.0f;

  // the tile points this thread stages (the same for every field): their
  // offsets in a field's plane, -1 past the tile or the padded level
  int soff[kStagePer];
#pragma unroll
  for (int r = 0; r < kStagePer; ++r) {
    const int e = tid + r * DTX * DTZ;
    const int gj = j0 - 4 + e % DHX, gk = k0 - 4 + e / DHX;
    soff[r] = (e < DHX * DHZ && gj <= jlim && gk <= klim) ? cid(L, gj, gk) : -1;
  }
  double pre[kStagePer];
  auto fetch = [&](int f) {
#pragma unroll
    for (int r = 0; r < kStagePer; ++r) pre[r] = soff[r] >= 0 ? U[(size_t)f * P + soff[r]] : 0.0;
  };
  auto stage = [&](float2 (*t)[DHX]) {
#pragma unroll
    for (int r = 0; r < kStagePer; ++r) {
      const int e = tid + r * DTX * DTZ;
      if (e < DHX * DHZ) {
        const F2 v = soff[r] >= 0 ? split_f64(pre[r]) : F2{0.0f, 0.0f};
        t[e / DHX][e % DHX] = make_float2(v.hi, v.lo);
      }
    }
  };
  fetch(0);
  stage(tiles[0]);
  __syncthreads();

  FieldLoop<0>::run([&](auto fc) {
    constexpr int f = decltype(fc)::value;
    float2 (*tile)[DHX] = tiles[f & 1];
    if constexpr (f + 1 < NMET) fetch(f + 1);
    if (live) {
      const int cx = tx + 4, cz = tz + 4;
      const float2 c = tile[cz][cx];
      auto at = [&](int dx, int dz) { return tile[cz + dz][cx + dx]; };
      auto df = [&](float2 a, float2 b) { return (a.x - b.x) + (a.y - b.y); };
      float Dx[9], Dz[9];   // u(n) - u(0), n = -4..4
#pragma unroll
      for (int n = -4; n <= 4; ++n) {
        Dx[n + 4] = n == 0 ? 0.0f : df(at(n, 0), c);
        Dz[n + 4] = n == 0 ? 0.0f : df(at(0, n), c);
      }
      constexpr int a1 = d1_of(f), a2 = d2_of(f);
      float d1x = 0.0f;
      if constexpr (a1 >= 0) {
        d1x = (45.0f * df(at(1, 0), at(-1, 0)) - 9.0f * df(at(2, 0), at(-2, 0)) + df(at(3, 0), at(-3, 0))) * i60x;
        const float d1z = (45.0f * df(at(0, 1), at(0, -1)) - 9.0f * df(at(0, 2), at(0, -2)) + df(at(0, 3), at(0, -3))) * i60z;
        DS[(size_t)(DS_D1 + 3 * a1 + 0) * P + id] = d1x;
        DS[(size_t)(DS_D1 + 3 * a1 + 2) * P + id] = d1z;
        DS[(size_t)(DS_D1 + 3 * a1 + 1) * P + id] = (cyl && !y_zero_c(f)) ? dyf[(size_t)f * P + id] : 0.0f;
      }
      if constexpr (a2 >= 0) {
        float dxz = 0.0f;
#pragma unroll
        for (int n = 1; n <= 3; ++n) {
          const float w = n == 1 ? 45.0f : (n == 2 ? -9.0f : 1.0f);
          const float zp = 45.0f * df(at(n, 1), at(n, -1)) - 9.0f * df(at(n, 2), at(n, -2)) + df(at(n, 3), at(n, -3));
          const float zm = 45.0f * df(at(-n, 1), at(-n, -1)) - 9.0f * df(at(-n, 2), at(-n, -2)) + df(at(-n, 3), at(-n, -3));
          dxz += w * (zp - zm);
        }
        float dxy = 0.0f, dyz = 0.0f, dyy = 0.0f;
        if (cyl) {
          dyy = dyyf[(size_t)f * P + id];
          if (!y_zero_c(f)) {
            const float *q = dyf + (size_t)f * P + id;
            const int sz = L.px;
            dyz = (45.0f * (q[sz] - q[-sz]) - 9.0f * (q[2 * sz] - q[-2 * sz]) + (q[3 * sz] - q[-3 * sz])) * i60z;
            if (!edge) dxy = (45.0f * (q[1] - q[-1]) - 9.0f * (q[2] - q[-2]) + (q[3] - q[-3])) * i60x;
          }
        }
        float *o = DS + (size_t)(DS_D2 + 6 * a2) * P + id;
        o[0] = (270.0f * (Dx[5] + Dx[3]) - 27.0f * (Dx[6] + Dx[2]) + 2.0f * (Dx[7] + Dx[1])) * i180x;
        o[P] = dxy;
        o[2 * P] = dxz * ixz;
        o[3 * P] = dyy;
        o[4 * P] = dyz;
        o[5 * P] = (270.0f * (Dz[5] + Dz[3]) - 27.0f * (Dz[6] + Dz[2]) + 2.0f * (Dz[7] + Dz[1])) * i180z;
      }
      // advection: lopsided in x and z (upwind side of the shift), central in y from the planes; KO
      float adv = 0.0f;
      auto lop = [](const float *D, float v) {   // upwind-biased stencil, side of sign(v)
        if (v > 0.0f) return 2.0f * D[2] - 24.0f * D[3] + 80.0f * D[5] - 30.0f * D[6] + 8.0f * D[7] - D[8];
        if (v < 0.0f) return -(2.0f * D[6] - 24.0f * D[5] + 80.0f * D[3] - 30.0f * D[2] + 8.0f * D[1] - D[0]);
        return 0.0f;
      };
      adv += bx * lop(Dx, bx) * i60x + bz * lop(Dz, bz) * i60z;
      if (cyl && !y_zero_c(f)) adv += by * dyf[(size_t)f * P + id];
      const float kx = (Dx[8] + Dx[0]) - 8.0f * (Dx[7] + Dx[1]) + 28.0f * (Dx[6] + Dx[2]) - 56.0f * (Dx[5] + Dx[3]);
      const float kz = (Dz[8] + Dz[0]) - 8.0f * (Dz[7] + Dz[1]) + 28.0f * (Dz[6] + Dz[2]) - 56.0f * (Dz[5] + Dz[3]);
      adv += ko * (kx * ikx + kz * ikz);
      DS[(size_t)(DS_AK + f) * P + id] = adv;
      constexpr int eq = f == fHXX ? 0 : f == fHXY ? 1 : f == fHXZ ? 2 : f == fHYY ? 3 : f == fHYZ ? 4 : f == fBX ? 5 : f == fBY ? 6 : -1;
      if constexpr (eq >= 0) {
        ev[eq] = c.x + c.y;
        ed[eq] = d1x;
      }
    }
    if constexpr (f + 1 < NMET) stage(tiles[(f + 1) & 1]);
    __syncthreads();
  });
  if (live && edge) {
    // Eq. cartoon_bnd for cells beyond the level edge: d_xy from d_x and values
    const float x = ((float)j - 0.5f) * L.f.dx;
    const float ix = 1.0f / x, ix2 = ix * ix;
    auto put = [&](int a, float v) { DS[(size_t)(DS_D2 + 6 * a + 1) * P + id] = v; };
    put(8, ev[6] * ix2 - ed[6] * ix);
    put(9, -ev[5] * ix2 + ed[5] * ix);
    put(3, ev[4] * ix2 - ed[4] * ix);
    put(5, -ev[2] * ix2 + ed[2] * ix);
    const float txy = ev[1] * ix2 - ed[1] * ix;
    put(1, 2.0f * txy);
    put(4, -2.0f * txy);
    put(2, (ev[3] - ev[0]) * ix2 + (ed[0] - ed[3]) * ix);
  }
}

// FP64 derivative pass, one thread per cell.  Per field the seventeen stencil
// values (nine along x, nine along z) go onto one fixed-point grid (fixed.cuh)
// and every integer-weight sum is formed exactly in 64-bit integers: the
// central first and second derivatives, the lopsided advection stencil (as
// its odd and even parts A + sign(beta) B, both from the symmetric pairs), the
// Kreiss-Oliger sum and the z-difference numerator that the neighbouring
// columns use for d_xz.  Each result is converted and scaled once in FP64.
// A field falls back to the FP64 difference form (u(n) - u(0), exact zero on
// constants) where the fixed-point form does not apply: non-finite values,
// values below 2^-895 (grid below the normal range), or a second-derivative
// sum that could pass 2^63.
__constant__ signed char kD1Of[NMET] = {0, 1, 2, 3, 4, 5, 6, -1, -1, -1, -1, -1, -1, 7, 8, 9, 10, 11, 12, 13, 14, 15, -1, -1, -1};
__constant__ signed char kD2Of[NMET] = {0, 1, 2, 3, 4, 5, 6, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 7, 8, 9, 10, -1, -1, -1};

// the (unscaled) 6th-order z-difference numerator at column c in FP64
__device__ __forceinline__ double zdiff_num(const double *c, int sz) {
  return 45.0 * (c[sz] - c[-sz]) - 9.0 * (c[2 * sz] - c[-2 * sz]) + (c[3 * sz] - c[-3 * sz]);
}

// Staged form (tb given; block FDX x FDZ, tile origin j0, k0): each field's
// tile with a 4-cell halo is held in shared memory as the values' bit
// patterns, double-buffered: the loads of field f + 1 are issued before field
// f's stencils run from the other buffer, and one barrier per field closes
// it.  The stencils read the same values as from global memory.
constexpr int FDX = 16, FDZ = 8, FHX = FDX + 8, FHZ = FDZ + 8;
constexpr int kF64Per = FHX * FHZ / (FDX * FDZ);      // staged points per thread and field
static_assert(FHX * FHZ == kF64Per * FDX * FDZ, "the halo tile splits evenly over the block");

template <typename T>
__device__ __forceinline__ void z4c_derivs_cell(const Lev &L, const DevParams &p, const double *__restrict__ U,
                                                double *__restrict__ DS, int jmax, int kmax, int cyl, int j, int k,
                                                long long *sdn = nullptr, int *sde = nullptr, int j0 = 0,
                                                long long (*tb)[FHZ][FHX] = nullptr, int k0 = 0) {
  static_assert(sizeof(T) == 8, "the FP32 form is z4c_derivs_f32_tile");
  // Staged form (tb, sdn, sde given): the mixed derivative d_xz is the
  // x-difference of the z-difference numerators of the neighbouring columns,
  // exact integers on each column's own grid (numerator, exponent), which the
  // block exchanges through shared memory (row of blockDim.x + 6 columns per
  // thread row: each thread its own column, the three threads at either end of
  // a row one halo column each); every thread of the block runs the field loop
  // (it has barriers).  Per-cell form (none given): d_xz in FP64 from the
  // column differences.
  const bool xch = tb != nullptr;
  const bool active = j <= jmax && k <= kmax;
  if (!xch && !active) return;
  const int bw = (int)blockDim.x + 6, tx = (int)threadIdx.x;
  long long *rown = xch ? sdn + (size_t)threadIdx.y * bw : nullptr;
  int *rowe = xch ? sde + (size_t)threadIdx.y * bw : nullptr;
  const size_t P = L.P;
  const int id = cid(L, j, k);
  const int sz = L.px;
  const double i60x = L.i60x, i60z = L.i60z, i180x = L.i180x, i180z = L.i180z, ixz = L.ixz;
  const bool edge = cyl && j > L.nx;
  const bool own_col = k <= kmax && j <= jmax + 3;          // a column some cell of the row differentiates
  double bx = 0.0, by = 0.0, bz = 0.0;
  if (active) {
    bx = U[(size_t)fBX * P + id]; by = U[(size_t)fBY * P + id]; bz = U[(size_t)fBZ * P + id];
  }
  // per-cell factors: the integer lopsided sums are doubled, the KO sums share one grid
  const double ax = bx * (0.5 * i60x), az = bz * (0.5 * i60z);
  const bool bxpos = fx::bits(bx) > 0, bzpos = fx::bits(bz) > 0;   // beta > 0 (a zero beta has ax = 0)
  const double ko = p.ko, ikx = L.idx, ikz = L.idz;
  const double kfx = ko * ikx, kfz = ko * ikz;
  const bool same_d = ikx == ikz;
  // staged form: this thread's points of the halo tile (offset in a field's
  // plane, -1 past the padded level) and the loads in flight
  const int tid = (int)(threadIdx.y * blockDim.x + threadIdx.x), tz = (int)threadIdx.y;
  int soff[kF64Per];
  long long pre[kF64Per];
  if (tb) {
#pragma unroll
    for (int r = 0; r < kF64Per; ++r) {
      const int e = tid + r * FDX * FDZ;
      const int gj = j0 - 4 + e % FHX, gk = k0 - 4 + e / FHX;
      soff[r] = (gj <= L.nx + GH && gk <= L.nz + GH) ? cid(L, gj, gk) : -1;
    }
  }
  auto fetch = [&](int f) {
#pragma unroll
    for (int r = 0; r < kF64Per; ++r) pre[r] = soff[r] >= 0 ? fx::bits(U[(size_t)f * P + soff[r]]) : 0ll;
  };
  auto stage = [&](long long (*t)[FHX]) {
#pragma unroll
    for (int r = 0; r < kF64Per; ++r) {
      const int e = tid + r * FDX * FDZ;
      t[e / FHX][e % FHX] = pre[r];
    }
  };
  if (tb) {
    fetch(0);
    stage(tb[0]);
    __syncthreads();
  }
#pragma unroll 1
  for (int f = 0; f < NMET; ++f) {
    const int a1 = kD1Of[f], a2 = kD2Of[f];
    const bool yz = y_zero(f);
    const double *u = U + (size_t)f * P + id;
    long long (*tile)[FHX] = tb ? tb[f & 1] : nullptr;
    if (tb && f + 1 < NMET) fetch(f + 1);
    long long cn = 0;                  // z-difference numerator of this thread's column ...
    int ce = 1;                        // ... on the grid 2^(ce - kGrid); -1: not finite
    if (active) {
      long long X[9], Z[9];
      if (tile) {
#pragma unroll
        for (int n = 0; n < 9; ++n) {
          X[n] = tile[tz + 4][tx + n];
          Z[n] = n == 4 ? X[4] : tile[tz + n][tx + 4];
        }
      } else {
#pragma unroll
        for (int n = 0; n < 9; ++n) {
          X[n] = fx::bits(u[n - 4]);
          Z[n] = n == 4 ? X[4] : fx::bits(u[(n - 4) * sz]);
        }
      }
      int E = 0;
#pragma unroll
      for (int n = 0; n < 9; ++n) E = max(E, max(fx::expo(X[n]), fx::expo(Z[n])));
      bool fast = E < 2047, zero = false;
      long long d1xn = 0, d1zn = 0, d2xn = 0, d2zn = 0, kxn = 0, kzn = 0, lxn = 0, lzn = 0;
      if (E == 0) {                                   // zeros (or subnormals: FP64 form)
        long long o = 0;
#pragma unroll
        for (int n = 0; n < 9; ++n) o |= (X[n] | Z[n]) & ~(1ll << 63);
        zero = o == 0;
        fast = false;
      }
      if (fast) {
#pragma unroll
        for (int n = 0; n < 9; ++n) {
          X[n] = fx::fix(X[n], E);
          Z[n] = n == 4 ? X[4] : fx::fix(Z[n], E);
        }
        const long long c2 = 2 * X[4];
        const long long ox1 = X[5] - X[3], ox2 = X[6] - X[2], ox3 = X[7] - X[1], ox4 = X[8] - X[0];
        const long long ex1 = X[5] + X[3] - c2, ex2 = X[6] + X[2] - c2, ex3 = X[7] + X[1] - c2, ex4 = X[8] + X[0] - c2;
        const long long oz1 = Z[5] - Z[3], oz2 = Z[6] - Z[2], oz3 = Z[7] - Z[1], oz4 = Z[8] - Z[0];
        const long long ez1 = Z[5] + Z[3] - c2, ez2 = Z[6] + Z[2] - c2, ez3 = Z[7] + Z[1] - c2, ez4 = Z[8] + Z[0] - c2;
        // |values| < 2^54 on the grid: the first-derivative, lopsided (doubled) and KO sums stay
        // below 2^63 by their weight sums (110, 360, 256); the second derivative (weight sum 1088
        // on the values) is checked on its pair sums
        d1xn = 45 * ox1 - 9 * ox2 + ox3;
        d1zn = 45 * oz1 - 9 * oz2 + oz3;
        if (a2 >= 0) {
          // the sums wrap (unsigned) where the check fails; the FP64 form then replaces them
          typedef unsigned long long u64;
          const long long m = fx::mag(ex1) | fx::mag(ex2) | fx::mag(ex3) | fx::mag(ez1) | fx::mag(ez2) | fx::mag(ez3);
          fast = (m >> 54) == 0;
          d2xn = (long long)(270ull * (u64)ex1 - 27ull * (u64)ex2 + 2ull * (u64)ex3);
          d2zn = (long long)(270ull * (u64)ez1 - 27ull * (u64)ez2 + 2ull * (u64)ez3);
        }
        kxn = ex4 - 8 * ex3 + 28 * ex2 - 56 * ex1;      // each below 2^62, so their sum fits as well
        kzn = ez4 - 8 * ez3 + 28 * ez2 - 56 * ez1;
        const long long Ax = 104 * ox1 - 32 * ox2 + 8 * ox3 - ox4, Bx = 56 * ex1 - 28 * ex2 + 8 * ex3 - ex4;
        const long long Az = 104 * oz1 - 32 * oz2 + 8 * oz3 - oz4, Bz = 56 * ez1 - 28 * ez2 + 8 * ez3 - ez4;
        lxn = bxpos ? Ax + Bx : Ax - Bx;
        lzn = bzpos ? Az + Bz : Az - Bz;
      }
      double dxy = 0.0, dyz = 0.0, dyy = 0.0, dy1 = 0.0;
      if (cyl && !yz) dy1 = L.dy[(size_t)f * P + id];
      if (a2 >= 0 && cyl) {
        dyy = L.dyy[(size_t)f * P + id];
        if (!yz) {
          const double *q = L.dy + (size_t)f * P + id;
          dyz = (45.0 * (q[sz] - q[-sz]) - 9.0 * (q[2 * sz] - q[-2 * sz]) + (q[3 * sz] - q[-3 * sz])) * i60z;
          if (!edge) dxy = (45.0 * (q[1] - q[-1]) - 9.0 * (q[2] - q[-2]) + (q[3] - q[-3])) * i60x;
        }
      }
      double adv = by * dy1;
      if (fast || zero) {
        if (fast) {
          if (a1 >= 0) {
            DS[(size_t)(DS_D1 + 3 * a1 + 0) * P + id] = (double)d1xn * fx::unit(i60x, E);
            DS[(size_t)(DS_D1 + 3 * a1 + 2) * P + id] = (double)d1zn * fx::unit(i60z, E);
          }
          if (a2 >= 0) {
            DS[(size_t)(DS_D2 + 6 * a2 + 0) * P + id] = (double)d2xn * fx::unit(i180x, E);
            DS[(size_t)(DS_D2 + 6 * a2 + 5) * P + id] = (double)d2zn * fx::unit(i180z, E);
          }
          adv += (double)lxn * fx::unit(ax, E);
          adv += (double)lzn * fx::unit(az, E);
          if (same_d) adv += (double)(kxn + kzn) * fx::unit(kfx, E);
          else adv += (double)kxn * fx::unit(kfx, E) + (double)kzn * fx::unit(kfz, E);
        } else {
          if (a1 >= 0) {
            DS[(size_t)(DS_D1 + 3 * a1 + 0) * P + id] = 0.0;
            DS[(size_t)(DS_D1 + 3 * a1 + 2) * P + id] = 0.0;
          }
          if (a2 >= 0) {
            DS[(size_t)(DS_D2 + 6 * a2 + 0) * P + id] = 0.0;
            DS[(size_t)(DS_D2 + 6 * a2 + 5) * P + id] = 0.0;
          }
        }
      } else {
        // FP64 difference form
        const double u0 = u[0];
        double Dx[9], Dz[9];
#pragma unroll
        for (int n = -4; n <= 4; ++n) {
          Dx[n + 4] = n == 0 ? 0.0 : u[n] - u0;
          Dz[n + 4] = n == 0 ? 0.0 : u[n * sz] - u0;
        }
        if (a1 >= 0) {
          DS[(size_t)(DS_D1 + 3 * a1 + 0) * P + id] = (45.0 * (Dx[5] - Dx[3]) - 9.0 * (Dx[6] - Dx[2]) + (Dx[7] - Dx[1])) * i60x;
          DS[(size_t)(DS_D1 + 3 * a1 + 2) * P + id] = (45.0 * (Dz[5] - Dz[3]) - 9.0 * (Dz[6] - Dz[2]) + (Dz[7] - Dz[1])) * i60z;
        }
        if (a2 >= 0) {
          DS[(size_t)(DS_D2 + 6 * a2 + 0) * P + id] = (270.0 * (Dx[5] + Dx[3]) - 27.0 * (Dx[6] + Dx[2]) + 2.0 * (Dx[7] + Dx[1])) * i180x;
          DS[(size_t)(DS_D2 + 6 * a2 + 5) * P + id] = (270.0 * (Dz[5] + Dz[3]) - 27.0 * (Dz[6] + Dz[2]) + 2.0 * (Dz[7] + Dz[1])) * i180z;
        }
        auto lop = [](const double *D, double v) {
          if (v > 0.0) return 2.0 * D[2] - 24.0 * D[3] + 80.0 * D[5] - 30.0 * D[6] + 8.0 * D[7] - D[8];
          if (v < 0.0) return -(2.0 * D[6] - 24.0 * D[5] + 80.0 * D[3] - 30.0 * D[2] + 8.0 * D[1] - D[0]);
          return 0.0;
        };
        adv += bx * (lop(Dx, bx) * i60x) + bz * (lop(Dz, bz) * i60z);
        const double kx = (Dx[8] + Dx[0]) - 8.0 * (Dx[7] + Dx[1]) + 28.0 * (Dx[6] + Dx[2]) - 56.0 * (Dx[5] + Dx[3]);
        const double kz = (Dz[8] + Dz[0]) - 8.0 * (Dz[7] + Dz[1]) + 28.0 * (Dz[6] + Dz[2]) - 56.0 * (Dz[5] + Dz[3]);
        adv += ko * (kx * ikx + kz * ikz);
      }
      if (a1 >= 0) DS[(size_t)(DS_D1 + 3 * a1 + 1) * P + id] = dy1;
      if (a2 >= 0) {
        double *o = DS + (size_t)(DS_D2 + 6 * a2) * P + id;
        o[P] = dxy;
        o[3 * P] = dyy;
        o[4 * P] = dyz;
      }
      DS[(size_t)(DS_AK + f) * P + id] = adv;
    }
    if (xch && a2 >= 0 && own_col) {
      // every column's numerator from its own six z-values on their own grid
      // (the halo columns' form), so d_xz does not depend on where the tile
      // edges fall; this includes the columns right of the region that cells
      // of the region use
      fx::diff6_bits(&tile[tz + 4][tx + 4], FHX, cn, ce);
    }
    if (a2 >= 0) {
      double dxz = 0.0;
      bool fp64 = !xch;
      if (xch) {
        // (the previous field's row reads end before the field's closing barrier)
        rown[tx + 3] = own_col ? cn : 0;
        rowe[tx + 3] = own_col ? ce : 1;
        if (tx < 3 || tx >= (int)blockDim.x - 3) {
          const int e = tx < 3 ? tx : tx + 6;            // halo slot: columns j0 - 3 .. j0 - 1, j0 + bx .. + 2
          const int jc = j0 - 3 + e;
          long long hn = 0;
          int he = 1;
          if (k <= kmax && jc <= jmax + 3) fx::diff6_bits(&tile[tz + 4][jc - j0 + 4], FHX, hn, he);
          rown[e] = hn;
          rowe[e] = he;
        }
        __syncthreads();
        if (active) {
          // the six neighbouring numerators on one grid, 54 bits below the
          // largest of them (the weighted sum then stays below 2^62): exact for
          // numerators within 2^54 of the largest, combined exactly
          const long long *rn = rown + tx + 3;
          const int *re = rowe + tx + 3;
          int top = -100000;
          bool fin = true;
#pragma unroll
          for (int n = -3; n <= 3; ++n)
            if (n != 0) {
              fin = fin && re[n] >= 0;
              if (rn[n] != 0) top = max(top, re[n] + 64 - __clzll(fx::mag(rn[n])));
            }
          if (!fin) {
            fp64 = true;
          } else if (top > -100000) {
            const int G = top - 54;
            long long v[7];
#pragma unroll
            for (int n = -3; n <= 3; ++n)
              if (n != 0) {
                const int sh = re[n] - G;
                v[n + 3] = sh >= 0 ? (long long)((unsigned long long)rn[n] << sh) : fx::shr(rn[n], -sh);
              }
            const long long c = 45 * (v[4] - v[2]) - 9 * (v[5] - v[1]) + (v[6] - v[0]);
            dxz = (double)c * fx::unit(ixz, G);
          }
        }
      }
      if (active && fp64) {
        dxz = 0.0;
#pragma unroll
        for (int n = 1; n <= 3; ++n) {
          const double w = n == 1 ? 45.0 : (n == 2 ? -9.0 : 1.0);
          dxz += w * (zdiff_num(u + n, sz) - zdiff_num(u - n, sz));
        }
        dxz *= ixz;
      }
      if (active) DS[(size_t)(DS_D2 + 6 * a2 + 2) * P + id] = dxz;
    }
    if (tb) {
      if (f + 1 < NMET) stage(tb[(f + 1) & 1]);
      __syncthreads();
    }
  }
  if (!active) return;
  if (edge) {
    // Eq. cartoon_bnd for cells beyond the level edge: d_xy from d_x and values
    const double x = (j - 0.5) * L.dx;
    const double ix = 1.0 / x, ix2 = ix * ix;
    auto val = [&](int f) { return U[(size_t)f * P + id]; };
    auto ddx = [&](int f) { return DS[(size_t)(DS_D1 + 3 * kD1Of[f]) * P + id]; };
    auto put = [&](int a, double v) { DS[(size_t)(DS_D2 + 6 * a + 1) * P + id] = v; };
    put(8, val(fBY) * ix2 - ddx(fBY) * ix);
    put(9, -val(fBX) * ix2 + ddx(fBX) * ix);
    put(3, val(fHYZ) * ix2 - ddx(fHYZ) * ix);
    put(5, -val(fHXZ) * ix2 + ddx(fHXZ) * ix);
    const double txy = val(fHXY) * ix2 - ddx(fHXY) * ix;
    put(1, 2.0 * txy);
    put(4, -2.0 * txy);
    put(2, (val(fHYY) - val(fHXX)) * ix2 + (ddx(fHXX) - ddx(fHYY)) * ix);
  }
}

template <typename T>
__global__ void __launch_bounds__(128) k_z4c_derivs(Lev L, DevParams p, const double *__restrict__ U,
                                                     double *__restrict__ DS, int jmax, int kmax, int cyl) {
  __shared__ long long sdn[(32 + 6) * 4];   // the launch shape is 32 x 4
  __shared__ int sde[(32 + 6) * 4];
  const int j0 = blockIdx.x * blockDim.x + 1;
  const bool xch = blockDim.x == 32 && blockDim.y == 4;
  z4c_derivs_cell<T>(L, p, U, DS, jmax, kmax, cyl, j0 + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y + 1,
                     xch ? sdn : nullptr, xch ? sde : nullptr, j0);
}

__global__ void __launch_bounds__(DTX * DTZ, 3) k_z4c_derivs_f32(Lev L, DevParams p, const double *__restrict__ U,
                                                              float *__restrict__ DS, int jmax, int kmax, int cyl) {
  __shared__ float2 tiles[2][DHZ][DHX];
  z4c_derivs_f32_tile(L, p, U, DS, jmax, kmax, cyl, blockIdx.x * DTX + 1, blockIdx.y * DTZ + 1, tiles);
}

__global__ void __launch_bounds__(DTX * DTZ, 4) kb_z4c_derivs_f32(Batch b, DevParams p) {
  __shared__ float2 tiles[2][DHZ][DHX];
  const int cyl = p.geometry == SACRA_CYLINDRICAL;
  for_tiles<false>(b, [&](const BL &q, const Tile &tl) {
    z4c_derivs_f32_tile(q.L, q.P, q.U, reinterpret_cast<float *>(q.DS), q.jmax, q.kmax, cyl, tl.j0, tl.k0, tiles);
  });
}

// ---------------------------------------------------------------- pointwise pass

template <typename T>
__device__ inline void load_z4c_in(const Lev &L, const double *__restrict__ U, const T *__restrict__ DS, int id,
                                   Z4cIn<T> &z) {
  const size_t P = L.P;
  z.W = ld_as<T>(U[(size_t)fW * P + id]);
  z.al = ld_as<T>(U[(size_t)fAL * P + id]);
  z.Kh = ld_as<T>(U[(size_t)fKH * P + id]);
  z.Th = ld_as<T>(U[(size_t)fTH * P + id]);
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    z.h[a] = ld_as<T>(U[(size_t)(fHXX + a) * P + id]);
    z.A[a] = ld_as<T>(U[(size_t)(fAXX + a) * P + id]);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    z.Gt[i] = ld_as<T>(U[(size_t)(fGX + i) * P + id]);
    z.beta[i] = ld_as<T>(U[(size_t)(fBX + i) * P + id]);
    z.B[i] = ld_as<T>(U[(size_t)(fBBX + i) * P + id]);
  }
  auto d1 = [&](int a, int k) { return DS[(size_t)(DS_D1 + 3 * a + k) * P + id]; };
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    z.dW[k] = d1(0, k);
#pragma unroll
    for (int a = 0; a < 6; ++a) z.dh[a][k] = d1(1 + a, k);
    z.dKh[k] = d1(7, k);
#pragma unroll
    for (int i = 0; i < 3; ++i) z.dGt[i][k] = d1(8 + i, k);
    z.dTh[k] = d1(11, k);
    z.dal[k] = d1(12, k);
#pragma unroll
    for (int i = 0; i < 3; ++i) z.db[i][k] = d1(13 + i, k);
  }
  auto d2 = [&](int a, int q) { return DS[(size_t)(DS_D2 + 6 * a + q) * P + id]; };
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    z.ddW[q] = d2(0, q);
#pragma unroll
    for (int a = 0; a < 6; ++a) z.ddh[a][q] = d2(1 + a, q);
    z.ddal[q] = d2(7, q);
#pragma unroll
    for (int i = 0; i < 3; ++i) z.ddb[i][q] = d2(8 + i, q);
  }
}

template <typename T>
__device__ __forceinline__ void z4c_point_cell(const Lev &L, const DevParams &p, const double *__restrict__ U,
                                                    const T *__restrict__ DS, int jmax, int kmax, int j, int k,
                                                    double *__restrict__ rs_out = nullptr) {
  if (j > jmax || k > kmax) return;
  const size_t P = L.P;
  const int id = cid(L, j, k);
  Z4cIn<T> z;
  load_z4c_in(L, U, DS, id, z);
  Geo<T> G;
  geo_fill(z, G);
  geo_ricci(z, G);
  if (rs_out) rs_out[id] = to_f64<T>(G.Rs);
  T pr[NPRIM];
#pragma unroll
  for (int f = 0; f < NPRIM; ++f) pr[f] = ld_as<T>(L.prim[(size_t)f * P + id]);
  T E, Si[3], Sij[6];
  matter(pr, z.W, G.g, G.gi, E, Si, Sij);
  T fz;
  if constexpr (sizeof(T) == 4) {
    const float x = ((float)j - 0.5f) * f32_of(L.dx), zc = ((float)k - 0.5f) * f32_of(L.dz);
    fz = expf(-(x * x + zc * zc) * p.firz2);
  } else {
    const double x = (j - 0.5) * L.dx, zc = (k - 0.5) * L.dz;
    fz = exp(-(x * x + zc * zc) / (p.r_z4 * p.r_z4));
  }
  T src[NMET];
  z4c_source(p, z, G, E, Si, Sij, fz, src);
#pragma unroll
  // FP64: source + advection/KO in FP64; FP32: their FP32 sum, widened exactly
#pragma unroll
  for (int f = 0; f < NMET; ++f) L.rhs[(size_t)f * P + id] = to_f64<T>(src[f] + DS[(size_t)(DS_AK + f) * P + id]);
}

template <typename T>
__global__ void __launch_bounds__(128) k_z4c_point(Lev L, DevParams p, const double *__restrict__ U,
                                                    const T *__restrict__ DS, int jmax, int kmax) {
  z4c_point_cell<T>(L, p, U, DS, jmax, kmax, blockIdx.x * blockDim.x + threadIdx.x + 1, blockIdx.y * blockDim.y + threadIdx.y + 1);
}

// ---------------------------------------------------------------- host launchers

void launch_z4c_point(const Lev &L, const DevParams &p, const double *U, const double *DS, int jmax, int kmax,
                      cudaStream_t s) {
  dim3 b(32, 4), g((jmax + 31) / 32, (kmax + 3) / 4);
  if (p.mixed & SACRA_MIXED_Z4C) k_z4c_point<float><<<g, b, 0, s>>>(L, p, U, reinterpret_cast<const float *>(DS), jmax, kmax);
  else k_z4c_point<double><<<g, b, 0, s>>>(L, p, U, DS, jmax, kmax);
}

void launch_cartoon(const Lev &L, const DevParams &p, const double *U, const double *tab, int tab_stride,
                    const double *tabw, cudaStream_t s) {
  dim3 b(32, 4), g((L.nx + 7 + 31) / 32, (L.nz + 10 + 3) / 4);
  if (p.mixed & SACRA_MIXED_Z4C) k_cartoon_f32<<<g, b, 0, s>>>(L, U, tab, tab_stride);
  else k_cartoon_f64<<<g, b, 0, s>>>(L, U, tabw);
}

void launch_z4c_derivs(const Lev &L, const DevParams &p, const double *U, double *DS, int jmax, int kmax, cudaStream_t s) {
  if (p.mixed & SACRA_MIXED_Z4C) {
    dim3 b(DTX, DTZ), g((jmax + DTX - 1) / DTX, (kmax + DTZ - 1) / DTZ);
    k_z4c_derivs_f32<<<g, b, 0, s>>>(L, p, U, reinterpret_cast<float *>(DS), jmax, kmax, p.geometry == SACRA_CYLINDRICAL);
  } else {
    dim3 b(32, 4), g((jmax + 31) / 32, (kmax + 3) / 4);
    k_z4c_derivs<double><<<g, b, 0, s>>>(L, p, U, DS, jmax, kmax, p.geometry == SACRA_CYLINDRICAL);
  }
}

// ---------------------------------------------------------------- batched persistent kernels

__global__ void __launch_bounds__(128) kb_cartoon_f64(Batch b, const double *__restrict__ tabw) {
  for_tiles(b, [&](const BL &q, const Tile &tl) {
    cartoon_f64_cell(q.L, q.U, tabw, tl.j0 + threadIdx.x, tl.k0 + threadIdx.y);
  });
}

// FP32 cartoon planes, every tile's stencil rows split once into shared
// memory (dynamic buffer of cartoon32_tile_floats(...) floats)
__global__ void __launch_bounds__(128, 3) kb_cartoon_f32(Batch b, const double *__restrict__ tab, int tab_stride) {
  extern __shared__ float c32_sm[];
  for_tiles(b, [&](const BL &q, const Tile &tl) {
    cartoon32_tile(q.L, q.U, tl.j0, tl.k0, c32_sm);
    const int j = tl.j0 + threadIdx.x, jj = j <= 0 ? 1 - j : j;
    const int nc = (int)blockDim.x + 8;
    const Cartoon32Staged src{c32_sm, (int)blockDim.y * nc, nc, (int)threadIdx.y, jj - 4 - cartoon32_base(tl.j0)};
    cartoon_f32_cell(q.L, src, tab, tab_stride, j, tl.k0 + threadIdx.y);
  });
}

// the FP64 derivative pass on FDX x FDZ tiles, staged and double-buffered
constexpr int kDxzRow = (FDX + 6) * FDZ;
__global__ void __launch_bounds__(FDX * FDZ, 4) kb_z4c_derivs(Batch b, DevParams p) {
  __shared__ long long sdn[kDxzRow];
  __shared__ int sde[kDxzRow];
  __shared__ long long tb[2][FHZ][FHX];
  const int cyl = p.geometry == SACRA_CYLINDRICAL;
  for_tiles(b, [&](const BL &q, const Tile &tl) {
    z4c_derivs_cell<double>(q.L, q.P, q.U, reinterpret_cast<double *>(q.DS), q.jmax, q.kmax, cyl, tl.j0 + threadIdx.x,
                            tl.k0 + threadIdx.y, sdn, sde, tl.j0, tb, tl.k0);
  });
}

template <typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 0) kb_z4c_point(Batch b, DevParams p, int store_rs) {
  for_tiles<false>(b, [&](const BL &q, const Tile &tl) {
    double *rs = store_rs ? reinterpret_cast<double *>(q.DS) + (size_t)DS_RS * q.L.P : nullptr;
    z4c_point_cell<T>(q.L, q.P, q.U, reinterpret_cast<const T *>(q.DS), q.jmax, q.kmax, tl.j0 + threadIdx.x,
                      tl.k0 + threadIdx.y, rs);
  });
}

void launch_b_cartoon(const Batch &b, const DevParams &p, const double *tab, int tab_stride, const double *tabw,
                      cudaStream_t s) {
  if (b.ntiles <= 0) return;
  if (p.mixed & SACRA_MIXED_Z4C)
    kb_cartoon_f32<<<b.grid, b.block, cartoon32_tile_floats(b.block.x, b.block.y) * sizeof(float), s>>>(b, tab, tab_stride);
  else kb_cartoon_f64<<<b.grid, b.block, 0, s>>>(b, tabw);
}

void launch_b_z4c_derivs(const Batch &b, const DevParams &p, cudaStream_t s) {
  if (b.ntiles <= 0) return;
  if (p.mixed & SACRA_MIXED_Z4C) kb_z4c_derivs_f32<<<b.grid, dim3(DTX, DTZ), 0, s>>>(b, p);
  else kb_z4c_derivs<<<b.grid, dim3(FDX, FDZ), 0, s>>>(b, p);
}

void launch_b_z4c_point(const Batch &b, const DevParams &p, cudaStream_t s, int store_rs) {
  if (b.ntiles <= 0) return;
  if (p.mixed & SACRA_MIXED_Z4C) kb_z4c_point<float><<<b.grid, b.block, 0, s>>>(b, p, store_rs);
  else kb_z4c_point<double><<<b.grid, b.block, 0, s>>>(b, p, store_rs);
}

dim3 z4c_derivs_f32_block() { return dim3(DTX, DTZ); }
dim3 z4c_derivs_f64_block() { return dim3(FDX, FDZ); }

int z4c_scratch_planes() { return DS_N; }
int z4c_ricci_plane() { return DS_RS; }

}  // namespace sacra
