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
__global__ void k_cartoon(Lev L, const double *__restrict__ U, const double *__restrict__ tab, int tab_stride) {
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

__device__ __forceinline__ double fd1(const double *u, int s, double idx) {
  return (45.0 * (u[s] - u[-s]) - 9.0 * (u[2 * s] - u[-2 * s]) + (u[3 * s] - u[-3 * s])) * idx;
}
__device__ __forceinline__ double fd2(const double *u, int s, double idx2) {
  const double u0 = u[0];
  return (270.0 * ((u[s] - u0) + (u[-s] - u0)) - 27.0 * ((u[2 * s] - u0) + (u[-2 * s] - u0))
          + 2.0 * ((u[3 * s] - u0) + (u[-3 * s] - u0))) * idx2;
}
// upwind-biased 6th-order derivative in the direction of the advecting velocity
__device__ __forceinline__ double fdlop(const double *u, int s, double v, double idx) {
  if (v == 0.0) return 0.0;
  const int t = v > 0.0 ? s : -s;
  const double u0 = u[0];
  const double r = 2.0 * (u[-2 * t] - u0) - 24.0 * (u[-t] - u0) + 80.0 * (u[t] - u0) - 30.0 * (u[2 * t] - u0)
                 + 8.0 * (u[3 * t] - u0) - (u[4 * t] - u0);
  return (v > 0.0 ? r : -r) * idx;
}
__device__ __forceinline__ double fdko(const double *u, int s) {
  const double u0 = u[0];
  return ((u[4 * s] - u0) + (u[-4 * s] - u0)) - 8.0 * ((u[3 * s] - u0) + (u[-3 * s] - u0))
       + 28.0 * ((u[2 * s] - u0) + (u[-2 * s] - u0)) - 56.0 * ((u[s] - u0) + (u[-s] - u0));
}

__global__ void __launch_bounds__(128) k_z4c_derivs(Lev L, DevParams p, const double *__restrict__ U,
                                                     double *__restrict__ DS, int jmax, int kmax, int cyl) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int k = blockIdx.y * blockDim.y + threadIdx.y + 1;
  if (j > jmax || k > kmax) return;
  const size_t P = L.P;
  const int id = cid(L, j, k);
  const int sz = L.px;
  const double i60x = 1.0 / (60.0 * L.dx), i60z = 1.0 / (60.0 * L.dz);
  const double i180x = 1.0 / (180.0 * L.dx * L.dx), i180z = 1.0 / (180.0 * L.dz * L.dz);
  const double ixz = 1.0 / (3600.0 * L.dx * L.dz);
  const bool edge = cyl && j > L.nx;
  const double x = (j - 0.5) * L.dx;

  // first derivatives
  for (int a = 0; a < 16; ++a) {
    const int f = kD1Fields[a];
    const double *u = U + (size_t)f * P + id;
    DS[(size_t)(DS_D1 + 3 * a + 0) * P + id] = fd1(u, 1, i60x);
    DS[(size_t)(DS_D1 + 3 * a + 2) * P + id] = fd1(u, sz, i60z);
    DS[(size_t)(DS_D1 + 3 * a + 1) * P + id] = (cyl && !y_zero(f)) ? L.dy[(size_t)f * P + id] : 0.0;
  }
  // second derivatives: xx, xy, xz, yy, yz, zz
  for (int a = 0; a < 11; ++a) {
    const int f = kD2Fields[a];
    const double *u = U + (size_t)f * P + id;
    double dxz = 0.0;
#pragma unroll
    for (int n = 1; n <= 3; ++n) {
      const double w = n == 1 ? 45.0 : (n == 2 ? -9.0 : 1.0);
      // d_z at j+n minus d_z at j-n (pair form in both directions)
      const double zp = 45.0 * (u[n + sz] - u[n - sz]) - 9.0 * (u[n + 2 * sz] - u[n - 2 * sz]) + (u[n + 3 * sz] - u[n - 3 * sz]);
      const double zm = 45.0 * (u[-n + sz] - u[-n - sz]) - 9.0 * (u[-n + 2 * sz] - u[-n - 2 * sz]) + (u[-n + 3 * sz] - u[-n - 3 * sz]);
      dxz += w * (zp - zm);
    }
    double dxy = 0.0, dyz = 0.0, dyy = 0.0;
    if (cyl) {
      dyy = L.dyy[(size_t)f * P + id];
      if (!y_zero(f) && !edge) {
        const double *dyf = L.dy + (size_t)f * P + id;
        dxy = fd1(dyf, 1, i60x);
        dyz = fd1(dyf, sz, i60z);
      } else if (!y_zero(f)) {
        dyz = fd1(L.dy + (size_t)f * P + id, sz, i60z);
      }
    }
    double *o = DS + (size_t)(DS_D2 + 6 * a) * P + id;
    o[0] = fd2(u, 1, i180x);
    o[P] = dxy;
    o[2 * P] = dxz * ixz;
    o[3 * P] = dyy;
    o[4 * P] = dyz;
    o[5 * P] = fd2(u, sz, i180z);
  }
  if (edge) {
    // Eq. cartoon_bnd for cells beyond the level edge: d_xy from d_x and values
    const double ix = 1.0 / x, ix2 = ix * ix;
    auto val = [&](int f) { return U[(size_t)f * P + id]; };
    auto ddx = [&](int f) { return fd1(U + (size_t)f * P + id, 1, i60x); };
    auto put = [&](int a, double v) { DS[(size_t)(DS_D2 + 6 * a + 1) * P + id] = v; };
    // beta^x, beta^y are D2 entries 8, 9; h_ij entries 1..6 (xx,xy,xz,yy,yz,zz)
    put(8, val(fBY) * ix2 - ddx(fBY) * ix);
    put(9, -val(fBX) * ix2 + ddx(fBX) * ix);
    put(3, val(fHYZ) * ix2 - ddx(fHYZ) * ix);
    put(5, -val(fHXZ) * ix2 + ddx(fHXZ) * ix);
    const double txy = val(fHXY) * ix2 - ddx(fHXY) * ix;
    put(1, 2.0 * txy);
    put(4, -2.0 * txy);
    put(2, (val(fHYY) - val(fHXX)) * ix2 + (ddx(fHXX) - ddx(fHYY)) * ix);
  }
  // advection (lopsided in x, z; central in y from the planes) + KO
  const double bx = U[(size_t)fBX * P + id], by = U[(size_t)fBY * P + id], bz = U[(size_t)fBZ * P + id];
  const double ko = -p.eps_ko / 256.0;
  const double ikx = 1.0 / L.dx, ikz = 1.0 / L.dz;
  for (int f = 0; f < NMET; ++f) {
    const double *u = U + (size_t)f * P + id;
    double adv = bx * fdlop(u, 1, bx, i60x) + bz * fdlop(u, sz, bz, i60z);
    if (cyl && !y_zero(f)) adv += by * L.dy[(size_t)f * P + id];
    adv += ko * (fdko(u, 1) * ikx + fdko(u, sz) * ikz);
    DS[(size_t)(DS_AK + f) * P + id] = adv;
  }
}

// ---------------------------------------------------------------- pointwise pass

__device__ inline void load_z4c_in(const Lev &L, const double *__restrict__ U, const double *__restrict__ DS, int id,
                                   Z4cIn &z) {
  const size_t P = L.P;
  z.W = U[(size_t)fW * P + id];
  z.al = U[(size_t)fAL * P + id];
  z.Kh = U[(size_t)fKH * P + id];
  z.Th = U[(size_t)fTH * P + id];
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    z.h[a] = U[(size_t)(fHXX + a) * P + id];
    z.A[a] = U[(size_t)(fAXX + a) * P + id];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    z.Gt[i] = U[(size_t)(fGX + i) * P + id];
    z.beta[i] = U[(size_t)(fBX + i) * P + id];
    z.B[i] = U[(size_t)(fBBX + i) * P + id];
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

__global__ void __launch_bounds__(128) k_z4c_point(Lev L, DevParams p, const double *__restrict__ U,
                                                    const double *__restrict__ DS, int jmax, int kmax) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int k = blockIdx.y * blockDim.y + threadIdx.y + 1;
  if (j > jmax || k > kmax) return;
  const size_t P = L.P;
  const int id = cid(L, j, k);
  Z4cIn z;
  load_z4c_in(L, U, DS, id, z);
  Geo G;
  geo_fill(z, G);
  geo_ricci(z, G);
  double pr[NPRIM];
#pragma unroll
  for (int f = 0; f < NPRIM; ++f) pr[f] = L.prim[(size_t)f * P + id];
  double E, Si[3], Sij[6];
  matter(pr, z.W, G.g, G.gi, E, Si, Sij);
  const double x = (j - 0.5) * L.dx, zc = (k - 0.5) * L.dz;
  const double fz = exp(-(x * x + zc * zc) / (p.r_z4 * p.r_z4));
  double src[NMET];
  z4c_source(p, z, G, E, Si, Sij, fz, src);
#pragma unroll
  for (int f = 0; f < NMET; ++f) L.rhs[(size_t)f * P + id] = src[f] + DS[(size_t)(DS_AK + f) * P + id];
}

// ---------------------------------------------------------------- host launchers

void launch_z4c_point(const Lev &L, const DevParams &p, const double *U, const double *DS, int jmax, int kmax,
                      cudaStream_t s) {
  dim3 b(32, 4), g((jmax + 31) / 32, (kmax + 3) / 4);
  k_z4c_point<<<g, b, 0, s>>>(L, p, U, DS, jmax, kmax);
}

void launch_cartoon(const Lev &L, const double *U, const double *tab, int tab_stride, cudaStream_t s) {
  dim3 b(32, 4), g((L.nx + 7 + 31) / 32, (L.nz + 10 + 3) / 4);
  k_cartoon<<<g, b, 0, s>>>(L, U, tab, tab_stride);
}

void launch_z4c_derivs(const Lev &L, const DevParams &p, const double *U, double *DS, int jmax, int kmax, cudaStream_t s) {
  dim3 b(32, 4), g((jmax + 31) / 32, (kmax + 3) / 4);
  k_z4c_derivs<<<g, b, 0, s>>>(L, p, U, DS, jmax, kmax, p.geometry == SACRA_CYLINDRICAL);
}

int z4c_scratch_planes() { return DS_N; }

}  // namespace sacra
