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

// field of cartoon slot a (kCartoonFields, compile-time form)
__host__ __device__ constexpr int cartoon_field(int a) {
  constexpr int f[20] = {fW, fAL, fHXX, fHXY, fHXZ, fHYY, fHYZ, fHZZ, fAXX, fAXY,
                         fAXZ, fAYY, fAYZ, fBX, fBY, fBZ, fGX, fGY, fBBX, fBBY};
  return f[a];
}

// x-parity of the cartoon fields in kCartoonFields order (compile-time form)
__host__ __device__ constexpr float par_x_slot(int a) {
  return (a == 4 || a == 6 || a == 10 || a == 12 || a == 13 || a == 14 || a == 16 || a == 17 || a == 18 || a == 19)
             ? -1.0f : 1.0f;
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
// The fields are taken group by group (scalars, the h and At tensors, the
// beta, Gt and B vectors): each group's three planes come from one pass over
// its 9-point stencils, and only the group's components are live at a time.
struct CartoonOut {
  double *dy, *dyy;
  size_t P;
  int o;
  double i1, i2;
};

// accumulate the d_y / d_yy sums of slot a from its +m / -m plane values
__device__ __forceinline__ void cartoon_acc(int a, bool flip, double w1, double w2, double pp, double pm, double base,
                                            double &d1, double &d2) {
  const double pr = par_x_slot(a);
  const double plus = flip ? pr * pm : pp;
  const double minus = flip ? pr * pp : pm;
  const double centre = flip ? pr * base : base;
  d1 += w1 * (plus - minus);
  d2 += w2 * ((plus - centre) + (minus - centre));
}

__device__ __forceinline__ void cartoon_store(const CartoonOut &c, int a, double d1, double d2) {
  const int f = cartoon_field(a);
  if (f != fHZZ && f != fBZ && a >= 2) c.dy[(size_t)f * c.P + c.o] = d1 * c.i1;
  if (a <= 7 || (a >= 13 && a <= 15)) c.dyy[(size_t)f * c.P + c.o] = d2 * c.i2;
}

__device__ __forceinline__ void cartoon_f64_cell(const Lev &L, const double *__restrict__ U, const double *__restrict__ tab,
                                                     int tab_stride, int j, int k) {
  if (j > L.nx + 4 || k > L.nz + 7) return;
  const bool flip = j <= 0;
  const int jj = flip ? 1 - j : j;
  const size_t P = L.P;
  const int c0 = cid(L, jj, k);
  const double *t0 = tab + (size_t)(jj * 3) * tab_stride;   // per m: 9 weights, cos, sin
  CartoonOut co{L.dy, L.dyy, P, cid(L, j, k), L.i60x, L.i180x};
  const double c1w[3] = {45.0, -9.0, 1.0}, c2w[3] = {270.0, -27.0, 2.0};
  // the three planes of slot a: v[m] = base + sum_n t_m[n] (u[n] - base)
  auto planes = [&](int a, double &base, double v[3]) {
    const double *u = U + (size_t)cartoon_field(a) * P + c0 - 4;
    base = u[4];
    double s[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int n = 0; n < 9; ++n) {
      const double d = u[n] - base;
#pragma unroll
      for (int m = 0; m < 3; ++m) s[m] += t0[m * tab_stride + n] * d;
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) v[m] = base + s[m];
  };
  // scalars under the rotation: W, alpha, h_zz, beta^z
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int a = q == 0 ? 0 : (q == 1 ? 1 : (q == 2 ? 7 : 15));
    double base, v[3], d1 = 0.0, d2 = 0.0;
    planes(a, base, v);
#pragma unroll
    for (int m = 0; m < 3; ++m) cartoon_acc(a, flip, c1w[m], c2w[m], v[m], v[m], base, d1, d2);
    cartoon_store(co, a, d1, d2);
  }
  // vectors (x, y components): beta, Gt, B
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const int a = q == 0 ? 13 : (q == 1 ? 16 : 18);
    double bx, by, vx[3], vy[3];
    planes(a, bx, vx);
    planes(a + 1, by, vy);
    double d1x = 0.0, d2x = 0.0, d1y = 0.0, d2y = 0.0;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const double c = t0[m * tab_stride + 9], sn = t0[m * tab_stride + 10];
      const double px = c * vx[m] - sn * vy[m], py = sn * vx[m] + c * vy[m];
      const double mx = c * vx[m] - (-sn) * vy[m], my = (-sn) * vx[m] + c * vy[m];
      cartoon_acc(a, flip, c1w[m], c2w[m], px, mx, bx, d1x, d2x);
      cartoon_acc(a + 1, flip, c1w[m], c2w[m], py, my, by, d1y, d2y);
    }
    cartoon_store(co, a, d1x, d2x);
    cartoon_store(co, a + 1, d1y, d2y);
  }
  // symmetric tensors h_ij (slots 2..6) and At_ij (8..12): xx, xy, xz, yy, yz
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int a0 = q == 0 ? 2 : 8;
    double b[5], v[5][3];
#pragma unroll
    for (int i = 0; i < 5; ++i) planes(a0 + i, b[i], v[i]);
    double d1[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, d2[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const double c = t0[m * tab_stride + 9];
      double pp[5], pm[5];
#pragma unroll
      for (int sg = 0; sg < 2; ++sg) {
        const double sn = sg == 0 ? t0[m * tab_stride + 10] : -t0[m * tab_stride + 10];
        double *r = sg == 0 ? pp : pm;
        r[0] = c * c * v[0][m] - 2.0 * c * sn * v[1][m] + sn * sn * v[3][m];
        r[1] = c * sn * (v[0][m] - v[3][m]) + (c * c - sn * sn) * v[1][m];
        r[2] = c * v[2][m] - sn * v[4][m];
        r[3] = sn * sn * v[0][m] + 2.0 * c * sn * v[1][m] + c * c * v[3][m];
        r[4] = sn * v[2][m] + c * v[4][m];
      }
#pragma unroll
      for (int i = 0; i < 5; ++i) cartoon_acc(a0 + i, flip, c1w[m], c2w[m], pp[i], pm[i], b[i], d1[i], d2[i]);
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) cartoon_store(co, a0 + i, d1[i], d2[i]);
  }
}

__global__ void __launch_bounds__(128) k_cartoon_f64(Lev L, const double *__restrict__ U, const double *__restrict__ tab,
                                                     int tab_stride) {
  cartoon_f64_cell(L, U, tab, tab_stride, blockIdx.x * blockDim.x + threadIdx.x - 2, blockIdx.y * blockDim.y + threadIdx.y - 2);
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

__device__ __forceinline__ void cartoon_f32_cell(const Lev &L, const double *__restrict__ U, const double *__restrict__ tab,
                                                     int tab_stride, int j, int k) {
  if (j > L.nx + 4 || k > L.nz + 7) return;
  const bool flip = j <= 0;
  const int jj = flip ? 1 - j : j;
  const size_t P = L.P;
  const int c0 = cid(L, jj, k);
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
    const double *u = U + (size_t)kCartoonFields[a] * P + c0 - 4;
    const F2 c = split_f64(u[4]);
    u0[a] = c.hi + c.lo;
    float dn[9];
#pragma unroll
    for (int n = 0; n < 9; ++n) dn[n] = n == 4 ? 0.0f : f32_diff(split_f64(u[n]), c);
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
  cartoon_f32_cell(L, U, tab, tab_stride, blockIdx.x * blockDim.x + threadIdx.x - 2, blockIdx.y * blockDim.y + threadIdx.y - 2);
}

// ---------------------------------------------------------------- derivative pass

// derivative scratch layout (planes): D1 first derivatives of the 16 fields
// below (3 planes each), D2 second derivatives of 11 fields (6 planes each),
// AK advection + KO of all 25 fields.
__constant__ int kD1Fields[16] = {fW, fHXX, fHXY, fHXZ, fHYY, fHYZ, fHZZ, fKH, fGX, fGY, fGZ, fTH, fAL, fBX, fBY, fBZ};
__constant__ int kD2Fields[11] = {fW, fHXX, fHXY, fHXZ, fHYY, fHYZ, fHZZ, fAL, fBX, fBY, fBZ};
// DS_RS: the Ricci scalar of the pointwise pass, written when the diagnostics
// of the step's starting state are formed in the same stage.  The plane index
// counts FP64 planes in both forms: in the FP32 form it lies past the FP32
// planes of the same allocation (DS_N FP64 planes).
constexpr int DS_D1 = 0, DS_D2 = 48, DS_AK = 114, DS_RS = 139, DS_N = 140;

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

__host__ __device__ constexpr int d1_of(int f) {
  return f <= fHZZ ? f : (f == fKH ? 7 : (f >= fGX && f <= fGZ ? 8 + f - fGX : (f == fTH ? 11 : (f == fAL ? 12 : (f >= fBX && f <= fBZ ? 13 + f - fBX : -1)))));
}
__host__ __device__ constexpr int d2_of(int f) {
  return f <= fHZZ ? f : (f == fAL ? 7 : (f >= fBX && f <= fBZ ? 8 + f - fBX : -1));
}
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
__device__ __forceinline__ void z4c_derivs_f32_tile(const Lev &L, const DevParams &p, const double *__restrict__ U,
                                                    float *__restrict__ DS, int jmax, int kmax, int cyl, int j0, int k0,
                                                    float2 (*tile)[DHX]) {
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

  FieldLoop<0>::run([&](auto fc) {
    constexpr int f = decltype(fc)::value;
    const double *Uf = U + (size_t)f * P;
    for (int e = tid; e < DHX * DHZ; e += DTX * DTZ) {
      const int ex = e % DHX, ez = e / DHX;
      const int gj = j0 - 4 + ex, gk = k0 - 4 + ez;
      F2 v = {0.0f, 0.0f};
      if (gj <= jlim && gk <= klim) v = split_f64(Uf[cid(L, gj, gk)]);
      tile[ez][ex] = make_float2(v.hi, v.lo);
    }
    __syncthreads();
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

// FP64 derivative pass, one thread per cell: per field the differences
// u(n) - u(0), n = -4..4, along x and z are formed once and shared by the
// first and second derivatives, the lopsided advection and the Kreiss-Oliger
// term (difference form: exact zero on constants).
__constant__ signed char kD1Of[NMET] = {0, 1, 2, 3, 4, 5, 6, -1, -1, -1, -1, -1, -1, 7, 8, 9, 10, 11, 12, 13, 14, 15, -1, -1, -1};
__constant__ signed char kD2Of[NMET] = {0, 1, 2, 3, 4, 5, 6, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 7, 8, 9, 10, -1, -1, -1};

template <typename T>
__device__ __forceinline__ void z4c_derivs_cell(const Lev &L, const DevParams &p, const double *__restrict__ U,
                                                double *__restrict__ DS, int jmax, int kmax, int cyl, int j, int k,
                                                double *sdz = nullptr, int j0 = 0) {
  static_assert(sizeof(T) == 8, "the FP32 form is z4c_derivs_f32_tile");
  // XCH (sdz given): the mixed derivative d_xz is the x-difference of the
  // z-differences of the neighbouring columns, which the block exchanges
  // through shared memory (row of blockDim.x + 6 columns per thread row);
  // every thread of the block then runs the field loop (it has barriers)
  const bool xch = sdz != nullptr;
  const bool active = j <= jmax && k <= kmax;
  if (!xch && !active) return;
  const int bw = (int)blockDim.x + 6;
  double *srow = xch ? sdz + (size_t)threadIdx.y * bw : nullptr;
  const size_t P = L.P;
  const int id = cid(L, j, k);
  const int sz = L.px;
  const double i60x = L.i60x, i60z = L.i60z, i180x = L.i180x, i180z = L.i180z, ixz = L.ixz;
  const bool edge = cyl && j > L.nx;
  const double bx = U[(size_t)fBX * P + id], by = U[(size_t)fBY * P + id], bz = U[(size_t)fBZ * P + id];
  const double ko = p.ko, ikx = L.idx, ikz = L.idz;
#pragma unroll 1
  for (int f = 0; f < NMET; ++f) {
    if (xch && kD2Of[f] >= 0) {
      __syncthreads();                                   // the previous field's row is read
      for (int e = threadIdx.x; e < bw; e += blockDim.x) {
        const int jc = j0 - 3 + e;
        double v = 0.0;
        if (k <= kmax && jc <= jmax + 3) {
          const double *c = U + (size_t)f * P + cid(L, jc, k);
          v = 45.0 * (c[sz] - c[-sz]) - 9.0 * (c[2 * sz] - c[-2 * sz]) + (c[3 * sz] - c[-3 * sz]);
        }
        srow[e] = v;
      }
      __syncthreads();
    }
    if (!active) continue;
    const double *u = U + (size_t)f * P + id;
    const double u0 = u[0];
    double Dx[9], Dz[9];
#pragma unroll
    for (int n = -4; n <= 4; ++n) {
      Dx[n + 4] = n == 0 ? 0.0 : u[n] - u0;
      Dz[n + 4] = n == 0 ? 0.0 : u[n * sz] - u0;
    }
    const int a1 = kD1Of[f], a2 = kD2Of[f];
    const bool yz = y_zero(f);
    if (a1 >= 0) {
      DS[(size_t)(DS_D1 + 3 * a1 + 0) * P + id] = (45.0 * (Dx[5] - Dx[3]) - 9.0 * (Dx[6] - Dx[2]) + (Dx[7] - Dx[1])) * i60x;
      DS[(size_t)(DS_D1 + 3 * a1 + 2) * P + id] = (45.0 * (Dz[5] - Dz[3]) - 9.0 * (Dz[6] - Dz[2]) + (Dz[7] - Dz[1])) * i60z;
      DS[(size_t)(DS_D1 + 3 * a1 + 1) * P + id] = (cyl && !yz) ? L.dy[(size_t)f * P + id] : 0.0;
    }
    if (a2 >= 0) {
      double dxz = 0.0;
      if (xch) {
        const double *r = srow + threadIdx.x + 3;        // r[n]: z-difference at column j + n
        dxz = 45.0 * (r[1] - r[-1]) - 9.0 * (r[2] - r[-2]) + (r[3] - r[-3]);
      } else {
#pragma unroll
        for (int n = 1; n <= 3; ++n) {
          const double w = n == 1 ? 45.0 : (n == 2 ? -9.0 : 1.0);
          // d_z at j+n minus d_z at j-n (pair form in both directions)
          const double zp = 45.0 * (u[n + sz] - u[n - sz]) - 9.0 * (u[n + 2 * sz] - u[n - 2 * sz]) + (u[n + 3 * sz] - u[n - 3 * sz]);
          const double zm = 45.0 * (u[-n + sz] - u[-n - sz]) - 9.0 * (u[-n + 2 * sz] - u[-n - 2 * sz]) + (u[-n + 3 * sz] - u[-n - 3 * sz]);
          dxz += w * (zp - zm);
        }
      }
      double dxy = 0.0, dyz = 0.0, dyy = 0.0;
      if (cyl) {
        dyy = L.dyy[(size_t)f * P + id];
        if (!yz) {
          const double *q = L.dy + (size_t)f * P + id;
          dyz = (45.0 * (q[sz] - q[-sz]) - 9.0 * (q[2 * sz] - q[-2 * sz]) + (q[3 * sz] - q[-3 * sz])) * i60z;
          if (!edge) dxy = (45.0 * (q[1] - q[-1]) - 9.0 * (q[2] - q[-2]) + (q[3] - q[-3])) * i60x;
        }
      }
      double *o = DS + (size_t)(DS_D2 + 6 * a2) * P + id;
      o[0] = (270.0 * (Dx[5] + Dx[3]) - 27.0 * (Dx[6] + Dx[2]) + 2.0 * (Dx[7] + Dx[1])) * i180x;
      o[P] = dxy;
      o[2 * P] = dxz * ixz;
      o[3 * P] = dyy;
      o[4 * P] = dyz;
      o[5 * P] = (270.0 * (Dz[5] + Dz[3]) - 27.0 * (Dz[6] + Dz[2]) + 2.0 * (Dz[7] + Dz[1])) * i180z;
    }
    // advection: lopsided in x and z (upwind side of the shift), central in y; KO
    auto lop = [](const double *D, double v) {
      if (v > 0.0) return 2.0 * D[2] - 24.0 * D[3] + 80.0 * D[5] - 30.0 * D[6] + 8.0 * D[7] - D[8];
      if (v < 0.0) return -(2.0 * D[6] - 24.0 * D[5] + 80.0 * D[3] - 30.0 * D[2] + 8.0 * D[1] - D[0]);
      return 0.0;
    };
    double adv = bx * (lop(Dx, bx) * i60x) + bz * (lop(Dz, bz) * i60z);
    if (cyl && !yz) adv += by * L.dy[(size_t)f * P + id];
    const double kx = (Dx[8] + Dx[0]) - 8.0 * (Dx[7] + Dx[1]) + 28.0 * (Dx[6] + Dx[2]) - 56.0 * (Dx[5] + Dx[3]);
    const double kz = (Dz[8] + Dz[0]) - 8.0 * (Dz[7] + Dz[1]) + 28.0 * (Dz[6] + Dz[2]) - 56.0 * (Dz[5] + Dz[3]);
    adv += ko * (kx * ikx + kz * ikz);
    DS[(size_t)(DS_AK + f) * P + id] = adv;
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
  __shared__ double sdz[(32 + 6) * 4];   // the launch shape is 32 x 4
  const int j0 = blockIdx.x * blockDim.x + 1;
  const bool xch = blockDim.x == 32 && blockDim.y == 4;
  z4c_derivs_cell<T>(L, p, U, DS, jmax, kmax, cyl, j0 + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y + 1,
                     xch ? sdz : nullptr, j0);
}

__global__ void __launch_bounds__(DTX * DTZ, 3) k_z4c_derivs_f32(Lev L, DevParams p, const double *__restrict__ U,
                                                              float *__restrict__ DS, int jmax, int kmax, int cyl) {
  __shared__ float2 tile[DHZ][DHX];
  z4c_derivs_f32_tile(L, p, U, DS, jmax, kmax, cyl, blockIdx.x * DTX + 1, blockIdx.y * DTZ + 1, tile);
}

__global__ void __launch_bounds__(DTX * DTZ, 4) kb_z4c_derivs_f32(Batch b, DevParams p) {
  __shared__ float2 tile[DHZ][DHX];
  const int cyl = p.geometry == SACRA_CYLINDRICAL;
  for_tiles(b, [&](const BL &q, const Tile &tl) {
    z4c_derivs_f32_tile(q.L, q.P, q.U, reinterpret_cast<float *>(q.DS), q.jmax, q.kmax, cyl, tl.j0, tl.k0, tile);
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

void launch_cartoon(const Lev &L, const DevParams &p, const double *U, const double *tab, int tab_stride, cudaStream_t s) {
  dim3 b(32, 4), g((L.nx + 7 + 31) / 32, (L.nz + 10 + 3) / 4);
  if (p.mixed & SACRA_MIXED_Z4C) k_cartoon_f32<<<g, b, 0, s>>>(L, U, tab, tab_stride);
  else k_cartoon_f64<<<g, b, 0, s>>>(L, U, tab, tab_stride);
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

__global__ void __launch_bounds__(128) kb_cartoon_f64(Batch b, const double *__restrict__ tab, int tab_stride) {
  for_tiles(b, [&](const BL &q, const Tile &tl) {
    cartoon_f64_cell(q.L, q.U, tab, tab_stride, tl.j0 + threadIdx.x, tl.k0 + threadIdx.y);
  });
}

__global__ void __launch_bounds__(128, 3) kb_cartoon_f32(Batch b, const double *__restrict__ tab, int tab_stride) {
  for_tiles(b, [&](const BL &q, const Tile &tl) {
    cartoon_f32_cell(q.L, q.U, tab, tab_stride, tl.j0 + threadIdx.x, tl.k0 + threadIdx.y);
  });
}

constexpr int kDxzRow = 304;   // (blockDim.x + 6) * blockDim.y for every tuned shape up to 256 threads
__global__ void __launch_bounds__(256) kb_z4c_derivs(Batch b, DevParams p) {
  __shared__ double sdz[kDxzRow];
  const int cyl = p.geometry == SACRA_CYLINDRICAL;
  const bool xch = ((int)blockDim.x + 6) * (int)blockDim.y <= kDxzRow;
  for_tiles(b, [&](const BL &q, const Tile &tl) {
    z4c_derivs_cell<double>(q.L, q.P, q.U, reinterpret_cast<double *>(q.DS), q.jmax, q.kmax, cyl, tl.j0 + threadIdx.x,
                            tl.k0 + threadIdx.y, xch ? sdz : nullptr, tl.j0);
  });
}

template <typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 0) kb_z4c_point(Batch b, DevParams p, int store_rs) {
  for_tiles(b, [&](const BL &q, const Tile &tl) {
    double *rs = store_rs ? reinterpret_cast<double *>(q.DS) + (size_t)DS_RS * q.L.P : nullptr;
    z4c_point_cell<T>(q.L, q.P, q.U, reinterpret_cast<const T *>(q.DS), q.jmax, q.kmax, tl.j0 + threadIdx.x,
                      tl.k0 + threadIdx.y, rs);
  });
}

void launch_b_cartoon(const Batch &b, const DevParams &p, const double *tab, int tab_stride, cudaStream_t s) {
  if (b.ntiles <= 0) return;
  if (p.mixed & SACRA_MIXED_Z4C) kb_cartoon_f32<<<b.grid, b.block, 0, s>>>(b, tab, tab_stride);
  else kb_cartoon_f64<<<b.grid, b.block, 0, s>>>(b, tab, tab_stride);
}

void launch_b_z4c_derivs(const Batch &b, const DevParams &p, cudaStream_t s) {
  if (b.ntiles <= 0) return;
  if (p.mixed & SACRA_MIXED_Z4C) kb_z4c_derivs_f32<<<b.grid, dim3(DTX, DTZ), 0, s>>>(b, p);
  else kb_z4c_derivs<<<b.grid, b.block, 0, s>>>(b, p);
}

void launch_b_z4c_point(const Batch &b, const DevParams &p, cudaStream_t s, int store_rs) {
  if (b.ntiles <= 0) return;
  if (p.mixed & SACRA_MIXED_Z4C) kb_z4c_point<float><<<b.grid, b.block, 0, s>>>(b, p, store_rs);
  else kb_z4c_point<double><<<b.grid, b.block, 0, s>>>(b, p, store_rs);
}

dim3 z4c_derivs_f32_block() { return dim3(DTX, DTZ); }

int z4c_scratch_planes() { return DS_N; }
int z4c_ricci_plane() { return DS_RS; }

}  // namespace sacra
