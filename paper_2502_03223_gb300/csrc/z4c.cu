// Z4c right-hand side kernels on sm_103a (Lam & Shibata, arXiv:2502.03223,
// Sec. II.B): cartoon y-derivatives (Sec. II.B.2), 6th-order central,
// lopsided and mixed differences, 8th-order Kreiss-Oliger dissipation, and the
// pointwise right-hand side.  Three passes per level and stage:
//   k_cartoon:    interpolate-and-rotate planes y = +-m dy -> d_y, d_yy scratch
//   k_z4c_derivs: all x/z/mixed derivatives, advection + KO -> derivative scratch
//   k_z4c_point:  pointwise Z4c algebra -> rhs
#include "kernels.h"
#include "z4c.cuh"

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

// rotate interpolated base values v[20] (ordered as kCartoonFields) by phi
__device__ __forceinline__ void rotate20(const double v[20], double c, double s, double o[20]) {
  o[0] = v[0]; o[1] = v[1];
  // tensor h: xx,xy,xz,yy,yz,zz at 2..7
  o[2] = c * c * v[2] - 2.0 * c * s * v[3] + s * s * v[5];
  o[3] = c * s * (v[2] - v[5]) + (c * c - s * s) * v[3];
  o[4] = c * v[4] - s * v[6];
  o[5] = s * s * v[2] + 2.0 * c * s * v[3] + c * c * v[5];
  o[6] = s * v[4] + c * v[6];
  o[7] = v[7];
  // tensor At: xx,xy,xz,yy,yz at 8..12
  o[8] = c * c * v[8] - 2.0 * c * s * v[9] + s * s * v[11];
  o[9] = c * s * (v[8] - v[11]) + (c * c - s * s) * v[9];
  o[10] = c * v[10] - s * v[12];
  o[11] = s * s * v[8] + 2.0 * c * s * v[9] + c * c * v[11];
  o[12] = s * v[10] + c * v[12];
  // vectors beta (13..15), Gt (16,17), B (18,19)
  o[13] = c * v[13] - s * v[14];
  o[14] = s * v[13] + c * v[14];
  o[15] = v[15];
  o[16] = c * v[16] - s * v[17];
  o[17] = s * v[16] + c * v[17];
  o[18] = c * v[18] - s * v[19];
  o[19] = s * v[18] + c * v[19];
}

// Planes y = +-m dy at (x_j, z_k): 9-point Lagrange in x at varpi, rotated by
// +-phi (Sec. II.B.2); j <= 0 from the rotation by pi of (x_{1-j}, -+m dy).
// d_y and d_yy by 6th-order central differences over m = -3..3 (dy = dx).
__global__ void k_cartoon_f64(Lev L, const double *__restrict__ U, const double *__restrict__ tab, int tab_stride) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x - 2;
  const int k = blockIdx.y * blockDim.y + threadIdx.y - 2;
  if (j > L.nx + 4 || k > L.nz + 7) return;
  const bool flip = j <= 0;
  const int jj = flip ? 1 - j : j;
  const size_t P = L.P;
  const int c0 = cid(L, jj, k);
  double base0[20];
#pragma unroll
  for (int a = 0; a < 20; ++a) base0[a] = U[(size_t)kCartoonFields[a] * P + c0];
  double d1[20], d2[20];
#pragma unroll
  for (int a = 0; a < 20; ++a) { d1[a] = 0.0; d2[a] = 0.0; }
  const double c1w[3] = {45.0, -9.0, 1.0}, c2w[3] = {270.0, -27.0, 2.0};
  for (int m = 1; m <= 3; ++m) {
    const double *t = tab + (size_t)(jj * 3 + (m - 1)) * tab_stride;   // 9 weights, cos, sin
    double v[20];
#pragma unroll
    for (int a = 0; a < 20; ++a) {
      const double *u = U + (size_t)kCartoonFields[a] * P + c0 - 4;
      double s = 0.0;
#pragma unroll
      for (int n = 0; n < 9; ++n) s += t[n] * (u[n] - base0[a]);
      v[a] = base0[a] + s;
    }
    double pp[20], pm[20];
    rotate20(v, t[9], t[10], pp);
    rotate20(v, t[9], -t[10], pm);
    const double w1 = c1w[m - 1], w2 = c2w[m - 1];
#pragma unroll
    for (int a = 0; a < 20; ++a) {
      // at flipped points the +m plane is par * (-m plane of jj) and vice versa
      const double plus = flip ? par_x(kCartoonFields[a]) * pm[a] : pp[a];
      const double minus = flip ? par_x(kCartoonFields[a]) * pp[a] : pm[a];
      const double centre = flip ? par_x(kCartoonFields[a]) * base0[a] : base0[a];
      d1[a] += w1 * (plus - minus);
      d2[a] += w2 * ((plus - centre) + (minus - centre));
    }
  }
  const int o = cid(L, j, k);
  const double i1 = 1.0 / (60.0 * L.dx), i2 = 1.0 / (180.0 * L.dx * L.dx);
  // d_y of the fields whose y-derivative is not forced to zero
#pragma unroll
  for (int a = 2; a < 20; ++a) {
    const int f = kCartoonFields[a];
    if (f == fHZZ || f == fBZ) continue;
    L.dy[(size_t)f * P + o] = d1[a] * i1;
  }
  // d_yy of W, h_ij, alpha, beta^i
  const int sec[11] = {0, 1, 2, 3, 4, 5, 6, 7, 13, 14, 15};
#pragma unroll
  for (int b = 0; b < 11; ++b) L.dyy[(size_t)kCartoonFields[sec[b]] * P + o] = d2[sec[b]] * i2;
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

__global__ void k_cartoon_f32(Lev L, const double *__restrict__ U, const double *__restrict__ tab, int tab_stride) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x - 2;
  const int k = blockIdx.y * blockDim.y + threadIdx.y - 2;
  if (j > L.nx + 4 || k > L.nz + 7) return;
  const bool flip = j <= 0;
  const int jj = flip ? 1 - j : j;
  const size_t P = L.P;
  const int c0 = cid(L, jj, k);
  double base0[20];
  float u0[20];
#pragma unroll
  for (int a = 0; a < 20; ++a) {
    base0[a] = U[(size_t)kCartoonFields[a] * P + c0];
    u0[a] = (float)base0[a];
  }
  float d1[20], d2[20];
#pragma unroll
  for (int a = 0; a < 20; ++a) { d1[a] = 0.0f; d2[a] = 0.0f; }
  const float c1w[3] = {45.0f, -9.0f, 1.0f}, c2w[3] = {270.0f, -27.0f, 2.0f};
  for (int m = 1; m <= 3; ++m) {
    const double *t = tab + (size_t)(jj * 3 + (m - 1)) * tab_stride;   // 9 weights, cos, sin
    float w[9];
#pragma unroll
    for (int n = 0; n < 9; ++n) w[n] = (float)t[n];
    float sv[20];
#pragma unroll
    for (int a = 0; a < 20; ++a) {
      const double *u = U + (size_t)kCartoonFields[a] * P + c0 - 4;
      float acc = 0.0f;
#pragma unroll
      for (int n = 0; n < 9; ++n) acc += w[n] * (float)(u[n] - base0[a]);
      sv[a] = acc;
    }
    const float c1 = (float)(t[9] - 1.0), sn = (float)t[10];
    float dp[20], dm[20];   // plane (+m), plane (-m) minus centre, at jj
    dp[0] = dm[0] = sv[0];
    dp[1] = dm[1] = sv[1];
    deltas_ten(c1, sn, u0 + 2, sv + 2, dp + 2);
    deltas_ten(c1, -sn, u0 + 2, sv + 2, dm + 2);
    dp[7] = dm[7] = sv[7];                 // h_zz
    deltas_ten(c1, sn, u0 + 8, sv + 8, dp + 8);
    deltas_ten(c1, -sn, u0 + 8, sv + 8, dm + 8);
    deltas_vec(c1, sn, u0[13], u0[14], sv[13], sv[14], dp[13], dp[14]);
    deltas_vec(c1, -sn, u0[13], u0[14], sv[13], sv[14], dm[13], dm[14]);
    dp[15] = dm[15] = sv[15];              // beta^z
    deltas_vec(c1, sn, u0[16], u0[17], sv[16], sv[17], dp[16], dp[17]);
    deltas_vec(c1, -sn, u0[16], u0[17], sv[16], sv[17], dm[16], dm[17]);
    deltas_vec(c1, sn, u0[18], u0[19], sv[18], sv[19], dp[18], dp[19]);
    deltas_vec(c1, -sn, u0[18], u0[19], sv[18], sv[19], dm[18], dm[19]);
    const float w1 = c1w[m - 1], w2 = c2w[m - 1];
#pragma unroll
    for (int a = 0; a < 20; ++a) {
      // at flipped points the +m plane is par * (-m plane of jj) and vice versa
      const float pr = (float)par_x(kCartoonFields[a]);
      const float plus = flip ? pr * dm[a] : dp[a];
      const float minus = flip ? pr * dp[a] : dm[a];
      d1[a] += w1 * (plus - minus);
      d2[a] += w2 * (plus + minus);
    }
  }
  const int o = cid(L, j, k);
  const float i1 = (float)(1.0 / (60.0 * L.dx)), i2 = (float)(1.0 / (180.0 * L.dx * L.dx));
#pragma unroll
  for (int a = 2; a < 20; ++a) {
    const int f = kCartoonFields[a];
    if (f == fHZZ || f == fBZ) continue;
    L.dy[(size_t)f * P + o] = (double)(d1[a] * i1);
  }
  const int sec[11] = {0, 1, 2, 3, 4, 5, 6, 7, 13, 14, 15};
#pragma unroll
  for (int b = 0; b < 11; ++b) L.dyy[(size_t)kCartoonFields[sec[b]] * P + o] = (double)(d2[sec[b]] * i2);
}

// ---------------------------------------------------------------- derivative pass

// derivative scratch layout (planes): D1 first derivatives of the 16 fields
// below (3 planes each), D2 second derivatives of 11 fields (6 planes each),
// AK advection + KO of all 25 fields.
__constant__ int kD1Fields[16] = {fW, fHXX, fHXY, fHXZ, fHYY, fHYZ, fHZZ, fKH, fGX, fGY, fGZ, fTH, fAL, fBX, fBY, fBZ};
__constant__ int kD2Fields[11] = {fW, fHXX, fHXY, fHXZ, fHYY, fHYZ, fHZZ, fAL, fBX, fBY, fBZ};
constexpr int DS_D1 = 0, DS_D2 = 48, DS_AK = 114, DS_N = 139;

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

template <typename T>
__global__ void __launch_bounds__(128) k_z4c_derivs(Lev L, DevParams p, const double *__restrict__ U,
                                                     double *__restrict__ DS, int jmax, int kmax, int cyl) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int k = blockIdx.y * blockDim.y + threadIdx.y + 1;
  if (j > jmax || k > kmax) return;
  const size_t P = L.P;
  const int id = cid(L, j, k);
  const int sz = L.px;
  const T i60x = T(1.0 / (60.0 * L.dx)), i60z = T(1.0 / (60.0 * L.dz));
  const T i180x = T(1.0 / (180.0 * L.dx * L.dx)), i180z = T(1.0 / (180.0 * L.dz * L.dz));
  const T ixz = T(1.0 / (3600.0 * L.dx * L.dz));
  const bool edge = cyl && j > L.nx;
  const T x = T((j - 0.5) * L.dx);

  // first derivatives
  for (int a = 0; a < 16; ++a) {
    const int f = kD1Fields[a];
    const double *u = U + (size_t)f * P + id;
    DS[(size_t)(DS_D1 + 3 * a + 0) * P + id] = (double)fd1<T>(u, 1, i60x);
    DS[(size_t)(DS_D1 + 3 * a + 2) * P + id] = (double)fd1<T>(u, sz, i60z);
    DS[(size_t)(DS_D1 + 3 * a + 1) * P + id] = (cyl && !y_zero(f)) ? L.dy[(size_t)f * P + id] : 0.0;
  }
  // second derivatives: xx, xy, xz, yy, yz, zz
  for (int a = 0; a < 11; ++a) {
    const int f = kD2Fields[a];
    const double *u = U + (size_t)f * P + id;
    T dxz = T(0);
#pragma unroll
    for (int n = 1; n <= 3; ++n) {
      const T w = n == 1 ? T(45) : (n == 2 ? T(-9) : T(1));
      // d_z at j+n minus d_z at j-n (pair form in both directions, FP64 differences)
      const T zp = T(45) * T(u[n + sz] - u[n - sz]) - T(9) * T(u[n + 2 * sz] - u[n - 2 * sz]) + T(u[n + 3 * sz] - u[n - 3 * sz]);
      const T zm = T(45) * T(u[-n + sz] - u[-n - sz]) - T(9) * T(u[-n + 2 * sz] - u[-n - 2 * sz]) + T(u[-n + 3 * sz] - u[-n - 3 * sz]);
      dxz += w * (zp - zm);
    }
    T dxy = T(0), dyz = T(0), dyy = T(0);
    if (cyl) {
      dyy = T(L.dyy[(size_t)f * P + id]);
      if (!y_zero(f) && !edge) {
        const double *dyf = L.dy + (size_t)f * P + id;
        dxy = fd1<T>(dyf, 1, i60x);
        dyz = fd1<T>(dyf, sz, i60z);
      } else if (!y_zero(f)) {
        dyz = fd1<T>(L.dy + (size_t)f * P + id, sz, i60z);
      }
    }
    double *o = DS + (size_t)(DS_D2 + 6 * a) * P + id;
    o[0] = (double)fd2<T>(u, 1, i180x);
    o[P] = (double)dxy;
    o[2 * P] = (double)(dxz * ixz);
    o[3 * P] = (double)dyy;
    o[4 * P] = (double)dyz;
    o[5 * P] = (double)fd2<T>(u, sz, i180z);
  }
  if (edge) {
    // Eq. cartoon_bnd for cells beyond the level edge: d_xy from d_x and values
    const T ix = T(1) / x, ix2 = ix * ix;
    auto val = [&](int f) { return T(U[(size_t)f * P + id]); };
    auto ddx = [&](int f) { return fd1<T>(U + (size_t)f * P + id, 1, i60x); };
    auto put = [&](int a, T v) { DS[(size_t)(DS_D2 + 6 * a + 1) * P + id] = (double)v; };
    // beta^x, beta^y are D2 entries 8, 9; h_ij entries 1..6 (xx,xy,xz,yy,yz,zz)
    put(8, val(fBY) * ix2 - ddx(fBY) * ix);
    put(9, -val(fBX) * ix2 + ddx(fBX) * ix);
    put(3, val(fHYZ) * ix2 - ddx(fHYZ) * ix);
    put(5, -val(fHXZ) * ix2 + ddx(fHXZ) * ix);
    const T txy = val(fHXY) * ix2 - ddx(fHXY) * ix;
    put(1, T(2) * txy);
    put(4, T(-2) * txy);
    put(2, (val(fHYY) - val(fHXX)) * ix2 + (ddx(fHXX) - ddx(fHYY)) * ix);
  }
  // advection (lopsided in x, z; central in y from the planes) + KO
  const T bx = T(U[(size_t)fBX * P + id]), by = T(U[(size_t)fBY * P + id]), bz = T(U[(size_t)fBZ * P + id]);
  const T ko = T(-p.eps_ko / 256.0);
  const T ikx = T(1.0 / L.dx), ikz = T(1.0 / L.dz);
  for (int f = 0; f < NMET; ++f) {
    const double *u = U + (size_t)f * P + id;
    T adv = bx * fdlop<T>(u, 1, bx, i60x) + bz * fdlop<T>(u, sz, bz, i60z);
    if (cyl && !y_zero(f)) adv += by * T(L.dy[(size_t)f * P + id]);
    adv += ko * (fdko<T>(u, 1) * ikx + fdko<T>(u, sz) * ikz);
    DS[(size_t)(DS_AK + f) * P + id] = (double)adv;
  }
}

// ---------------------------------------------------------------- pointwise pass

template <typename T>
__device__ inline void load_z4c_in(const Lev &L, const double *__restrict__ U, const double *__restrict__ DS, int id,
                                   Z4cIn<T> &z) {
  const size_t P = L.P;
  z.W = T(U[(size_t)fW * P + id]);
  z.al = T(U[(size_t)fAL * P + id]);
  z.Kh = T(U[(size_t)fKH * P + id]);
  z.Th = T(U[(size_t)fTH * P + id]);
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    z.h[a] = T(U[(size_t)(fHXX + a) * P + id]);
    z.A[a] = T(U[(size_t)(fAXX + a) * P + id]);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    z.Gt[i] = T(U[(size_t)(fGX + i) * P + id]);
    z.beta[i] = T(U[(size_t)(fBX + i) * P + id]);
    z.B[i] = T(U[(size_t)(fBBX + i) * P + id]);
  }
  auto d1 = [&](int a, int k) { return T(DS[(size_t)(DS_D1 + 3 * a + k) * P + id]); };
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
  auto d2 = [&](int a, int q) { return T(DS[(size_t)(DS_D2 + 6 * a + q) * P + id]); };
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
__global__ void __launch_bounds__(128) k_z4c_point(Lev L, DevParams p, const double *__restrict__ U,
                                                    const double *__restrict__ DS, int jmax, int kmax) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int k = blockIdx.y * blockDim.y + threadIdx.y + 1;
  if (j > jmax || k > kmax) return;
  const size_t P = L.P;
  const int id = cid(L, j, k);
  Z4cIn<T> z;
  load_z4c_in(L, U, DS, id, z);
  Geo<T> G;
  geo_fill(z, G);
  geo_ricci(z, G);
  T pr[NPRIM];
#pragma unroll
  for (int f = 0; f < NPRIM; ++f) pr[f] = T(L.prim[(size_t)f * P + id]);
  T E, Si[3], Sij[6];
  matter(pr, z.W, G.g, G.gi, E, Si, Sij);
  const double x = (j - 0.5) * L.dx, zc = (k - 0.5) * L.dz;
  const T fz = T(exp(-(x * x + zc * zc) / (p.r_z4 * p.r_z4)));
  T src[NMET];
  z4c_source(p, z, G, E, Si, Sij, fz, src);
#pragma unroll
  for (int f = 0; f < NMET; ++f) L.rhs[(size_t)f * P + id] = (double)src[f] + DS[(size_t)(DS_AK + f) * P + id];
}

// ---------------------------------------------------------------- host launchers

void launch_z4c_point(const Lev &L, const DevParams &p, const double *U, const double *DS, int jmax, int kmax,
                      cudaStream_t s) {
  dim3 b(32, 4), g((jmax + 31) / 32, (kmax + 3) / 4);
  if (p.mixed & SACRA_MIXED_Z4C) k_z4c_point<float><<<g, b, 0, s>>>(L, p, U, DS, jmax, kmax);
  else k_z4c_point<double><<<g, b, 0, s>>>(L, p, U, DS, jmax, kmax);
}

void launch_cartoon(const Lev &L, const DevParams &p, const double *U, const double *tab, int tab_stride, cudaStream_t s) {
  dim3 b(32, 4), g((L.nx + 7 + 31) / 32, (L.nz + 10 + 3) / 4);
  if (p.mixed & SACRA_MIXED_Z4C) k_cartoon_f32<<<g, b, 0, s>>>(L, U, tab, tab_stride);
  else k_cartoon_f64<<<g, b, 0, s>>>(L, U, tab, tab_stride);
}

void launch_z4c_derivs(const Lev &L, const DevParams &p, const double *U, double *DS, int jmax, int kmax, cudaStream_t s) {
  dim3 b(32, 4), g((jmax + 31) / 32, (kmax + 3) / 4);
  if (p.mixed & SACRA_MIXED_Z4C) k_z4c_derivs<float><<<g, b, 0, s>>>(L, p, U, DS, jmax, kmax, p.geometry == SACRA_CYLINDRICAL);
  else k_z4c_derivs<double><<<g, b, 0, s>>>(L, p, U, DS, jmax, kmax, p.geometry == SACRA_CYLINDRICAL);
}

int z4c_scratch_planes() { return DS_N; }

}  // namespace sacra
