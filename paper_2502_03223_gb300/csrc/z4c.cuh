// Pointwise BSSN-Z4c algebra on the device (Lam & Shibata, arXiv:2502.03223,
// Sec. II.B.1, Eq. bssn, Eq. K, Eq. moving_puncture): conformal Christoffel
// symbols, Ricci tensor of gamma_ij = gt_ij / W^2, the right-hand side and
// the Hamiltonian / momentum constraints (Sec. II.F.1).
#pragma once

#include "common.cuh"

namespace sacra {

// Derivative scratch of a level (planes of stride P): DS_D1 + 3 a + k the
// first derivative d_k (x, y, z) of field slot a = d1_of(f) (16 fields),
// DS_D2 + 6 a + q the second derivatives (pair order xx, xy, xz, yy, yz, zz)
// of slot a = d2_of(f) (11 fields), DS_AK + f advection plus Kreiss-Oliger of
// all 25 fields.  DS_RS: the Ricci scalar of the pointwise pass, written when
// the diagnostics of the step's starting state are formed in the same stage;
// the plane index counts FP64 planes in both forms (in the FP32 form it lies
// past the FP32 planes of the same allocation of DS_N FP64 planes).
constexpr int DS_D1 = 0, DS_D2 = 48, DS_AK = 114, DS_RS = 139, DS_N = 140;

__host__ __device__ constexpr int d1_of(int f) {
  return f <= fHZZ ? f : (f == fKH ? 7 : (f >= fGX && f <= fGZ ? 8 + f - fGX : (f == fTH ? 11 : (f == fAL ? 12 : (f >= fBX && f <= fBZ ? 13 + f - fBX : -1)))));
}
__host__ __device__ constexpr int d2_of(int f) {
  return f <= fHZZ ? f : (f == fAL ? 7 : (f >= fBX && f <= fBZ ? 8 + f - fBX : -1));
}

// symmetric-pair index of (i, j)
__device__ __forceinline__ int sp(int i, int j) {
  return (i == j) ? (i == 0 ? 0 : (i == 1 ? 3 : 5)) : (i + j == 1 ? 1 : (i + j == 2 ? 2 : 4));
}

// Inputs of the pointwise right-hand side.  First derivatives d[k] of the
// fields that enter undifferentiated-by-advection terms, second derivatives
// in the pair order xx,xy,xz,yy,yz,zz.
template <typename T>
struct Z4cIn {
  T W, al, Kh, Th;
  T h[6], A[6], Gt[3], beta[3], B[3];
  T dW[3], dKh[3], dTh[3], dal[3];
  T dh[6][3];       // d_k h_ij  -> dh[ij][k]
  T dGt[3][3];      // d_k Gt^i  -> dGt[i][k]
  T db[3][3];       // d_k beta^i -> db[i][k]
  T ddW[6], ddal[6];
  T ddh[6][6];      // d_kl h_ij -> ddh[ij][kl]
  T ddb[3][6];      // d_kl beta^i
};

template <typename T>
struct Geo {
  Sym3T<T> g, gi;
  T Gl[3][6];       // Gt_{k,ij}
  T G2[3][6];       // Gt^k_ij
  T Gd[3];          // gt^jk Gt^i_jk
  T R[6];           // physical Ricci tensor
  T Rs;             // physical Ricci scalar
};

template <typename T>
__device__ inline void geo_fill(const Z4cIn<T> &z, Geo<T> &G) {
  G.g.xx = T(1.0) + z.h[0]; G.g.xy = z.h[1]; G.g.xz = z.h[2];
  G.g.yy = T(1.0) + z.h[3]; G.g.yz = z.h[4]; G.g.zz = T(1.0) + z.h[5];
  G.gi = s3inv(G.g, (T *)nullptr);
  // Gt_{k,ij} = (d_i gt_kj + d_j gt_ki - d_k gt_ij) / 2
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j)
        G.Gl[k][sp(i, j)] = T(0.5) * (z.dh[sp(k, j)][i] + z.dh[sp(k, i)][j] - z.dh[sp(i, j)][k]);
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    G.G2[0][a] = G.gi.xx * G.Gl[0][a] + G.gi.xy * G.Gl[1][a] + G.gi.xz * G.Gl[2][a];
    G.G2[1][a] = G.gi.xy * G.Gl[0][a] + G.gi.yy * G.Gl[1][a] + G.gi.yz * G.Gl[2][a];
    G.G2[2][a] = G.gi.xz * G.Gl[0][a] + G.gi.yz * G.Gl[1][a] + G.gi.zz * G.Gl[2][a];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
    G.Gd[i] = G.gi.xx * G.G2[i][0] + G.gi.yy * G.G2[i][3] + G.gi.zz * G.G2[i][5]
            + T(2.0) * (G.gi.xy * G.G2[i][1] + G.gi.xz * G.G2[i][2] + G.gi.yz * G.G2[i][4]);
}

// Ricci tensor of gamma = gt / W^2: Rt_ij (conformal part with d_j Gt^k from
// the evolved Gt, quadratic term with the computed Gt_d) plus the part from W.
template <typename T>
__device__ inline void geo_ricci(const Z4cIn<T> &z, Geo<T> &G) {
  const Sym3T<T> &gi = G.gi;
  const T gim[3][3] = {{gi.xx, gi.xy, gi.xz}, {gi.xy, gi.yy, gi.yz}, {gi.xz, gi.yz, gi.zz}};
  const T gm[3][3] = {{G.g.xx, G.g.xy, G.g.xz}, {G.g.xy, G.g.yy, G.g.yz}, {G.g.xz, G.g.yz, G.g.zz}};
  // D~_i D~_j W and the traces
  T DDW[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) DDW[a] = z.ddW[a] - (G.G2[0][a] * z.dW[0] + G.G2[1][a] * z.dW[1] + G.G2[2][a] * z.dW[2]);
  const T trDDW = gi.xx * DDW[0] + gi.yy * DDW[3] + gi.zz * DDW[5] + T(2.0) * (gi.xy * DDW[1] + gi.xz * DDW[2] + gi.yz * DDW[4]);
  const T dW2 = s3quad(gi, z.dW, z.dW);
  const T iW = T(1.0) / z.W;
  // gt^lm (Gt^k_li Gt_{j,km} + Gt^k_lj Gt_{i,km} + Gt^k_im Gt_{k,lj}) with the last
  // index of Gt_{j,km} raised once, M[j][k][l] = gt^lm Gt_{j,km}: the first two
  // terms are Q_ij + Q_ji with Q_ij = Gt^k_li M[j][k][l], the third Gt^k_im M[k][j][m]
  T M[3][3][3];
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = 0; l < 3; ++l)
        M[j][k][l] = gim[l][0] * G.Gl[j][sp(k, 0)] + gim[l][1] * G.Gl[j][sp(k, 1)] + gim[l][2] * G.Gl[j][sp(k, 2)];
  T Q[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      T q = T(0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) q += G.G2[k][sp(l, i)] * M[j][k][l];
      Q[i][j] = q;
    }
  T Rsum = T(0.0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int ij = sp(i, j);
      T r = T(0.0);
      // -1/2 gt^lm d_l d_m gt_ij
      r -= T(0.5) * (gi.xx * z.ddh[ij][0] + gi.yy * z.ddh[ij][3] + gi.zz * z.ddh[ij][5]
                  + T(2.0) * (gi.xy * z.ddh[ij][1] + gi.xz * z.ddh[ij][2] + gi.yz * z.ddh[ij][4]));
      // gt_k(i d_j) Gt^k
#pragma unroll
      for (int k = 0; k < 3; ++k) r += T(0.5) * (gm[k][i] * z.dGt[k][j] + gm[k][j] * z.dGt[k][i]);
      // Gt_d^k Gt_(ij)k
#pragma unroll
      for (int k = 0; k < 3; ++k) r += T(0.5) * G.Gd[k] * (G.Gl[i][sp(j, k)] + G.Gl[j][sp(i, k)]);
      // the quadratic Christoffel terms (above)
      T s3 = Q[i][j] + Q[j][i];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int m = 0; m < 3; ++m) s3 += G.G2[k][sp(i, m)] * M[k][j][m];
      r += s3;
      r += (DDW[ij] + gm[i][j] * trDDW) * iW - T(2.0) * gm[i][j] * dW2 * iW * iW;
      G.R[ij] = r;
      Rsum += (i == j ? T(1.0) : T(2.0)) * gim[i][j] * r;
    }
  G.Rs = z.W * z.W * Rsum;
}

// Matter terms E, S_i, S_ij from the primitives (rho, u_i, P, eps)
template <typename T>
__device__ inline void matter(const T pr[NPRIM], T W, const Sym3T<T> &g, const Sym3T<T> &gi, T &E, T S[3], T Sij[6]) {
  const T u[3] = {pr[pUX], pr[pUY], pr[pUZ]};
  const T w = sqrt(T(1.0) + W * W * s3quad(gi, u, u));
  const T rho = pr[pRHO], P = pr[pP];
  const T rh = rho * (T(1.0) + pr[pEPS] + P / rho);
  E = rh * w * w - P;
  S[0] = rh * w * u[0]; S[1] = rh * w * u[1]; S[2] = rh * w * u[2];
  const T iW2 = T(1.0) / (W * W);
  Sij[0] = rh * u[0] * u[0] + P * g.xx * iW2;
  Sij[1] = rh * u[0] * u[1] + P * g.xy * iW2;
  Sij[2] = rh * u[0] * u[2] + P * g.xz * iW2;
  Sij[3] = rh * u[1] * u[1] + P * g.yy * iW2;
  Sij[4] = rh * u[1] * u[2] + P * g.yz * iW2;
  Sij[5] = rh * u[2] * u[2] + P * g.zz * iW2;
}

// Source part of the Z4c right-hand side (everything but advection and KO).
// fz = exp(-r^2/r_Z4^2) multiplies kappa and the Theta source.
// out[25]; the B^i entries contain only their own source (Gt source - eta B).
template <typename T>
__device__ inline void z4c_source(const DevParams &p, const Z4cIn<T> &z, const Geo<T> &G, T E, const T Si[3],
                                  const T Sij[6], T fz, T out[NMET]) {
  const T PI = T(3.14159265358979323846);
  const Sym3T<T> &gi = G.gi;
  const T gim[3][3] = {{gi.xx, gi.xy, gi.xz}, {gi.xy, gi.yy, gi.yz}, {gi.xz, gi.yz, gi.zz}};
  const T gm[3][3] = {{G.g.xx, G.g.xy, G.g.xz}, {G.g.xy, G.g.yy, G.g.yz}, {G.g.xz, G.g.yz, G.g.zz}};
  const T W = z.W, al = z.al;
  const T K = z.Kh + T(2.0) * z.Th;
  const T kap = pv<T>(p.kappa, p.fkappa) * fz;
  const T divb = z.db[0][0] + z.db[1][1] + z.db[2][2];
  const T iW = T(1.0) / W;

  // physical D_i D_j alpha
  const T daW = s3quad(gi, z.dal, z.dW);
  T DDa[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int ij = sp(i, j);
      DDa[ij] = z.ddal[ij] - (G.G2[0][ij] * z.dal[0] + G.G2[1][ij] * z.dal[1] + G.G2[2][ij] * z.dal[2])
              + (z.dal[i] * z.dW[j] + z.dal[j] * z.dW[i] - gm[i][j] * daW) * iW;
    }
  const T D2a = W * W * (gi.xx * DDa[0] + gi.yy * DDa[3] + gi.zz * DDa[5]
                              + T(2.0) * (gi.xy * DDa[1] + gi.xz * DDa[2] + gi.yz * DDa[4]));
  // At with mixed and raised indices
  T Am[3][3];   // At_i^k = At_il gt^lk  -> Am[i][k]
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      Am[i][k] = z.A[sp(i, 0)] * gim[0][k] + z.A[sp(i, 1)] * gim[1][k] + z.A[sp(i, 2)] * gim[2][k];
  T Au[6];      // At^ij
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) Au[sp(i, j)] = gim[i][0] * Am[0][j] + gim[i][1] * Am[1][j] + gim[i][2] * Am[2][j];
  T AA = T(0.0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) AA += Am[i][k] * Am[k][i];
  const T Str = W * W * (gi.xx * Sij[0] + gi.yy * Sij[3] + gi.zz * Sij[5]
                              + T(2.0) * (gi.xy * Sij[1] + gi.xz * Sij[2] + gi.yz * Sij[4]));

  out[fW] = W * (al * K - divb) * T(1.0 / 3.0);

  // X_ij = alpha R_ij - D_i D_j alpha - 8 pi alpha S_ij and its gt-trace
  T X[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) X[a] = al * G.R[a] - DDa[a] - T(8.0) * PI * al * Sij[a];
  const T trX = gi.xx * X[0] + gi.yy * X[3] + gi.zz * X[5] + T(2.0) * (gi.xy * X[1] + gi.xz * X[2] + gi.yz * X[4]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int ij = sp(i, j);
      T sh = -T(2.0) * al * z.A[ij] - (T(2.0) / T(3.0)) * gm[i][j] * divb;
      T sa = W * W * (X[ij] - gm[i][j] * (trX * T(1.0 / 3.0)))
                + al * (K * z.A[ij] - T(2.0) * (Am[i][0] * z.A[sp(0, j)] + Am[i][1] * z.A[sp(1, j)] + Am[i][2] * z.A[sp(2, j)]))
                - (T(2.0) / T(3.0)) * z.A[ij] * divb;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        sh += gm[i][k] * z.db[k][j] + gm[j][k] * z.db[k][i];
        sa += z.A[sp(k, j)] * z.db[k][i] + z.A[sp(k, i)] * z.db[k][j];
      }
      out[fHXX + ij] = sh;
      out[fAXX + ij] = sa;
    }

  out[fKH] = -D2a + al * (AA + K * K * T(1.0 / 3.0)) + T(4.0) * PI * al * (Str + E) + al * kap * z.Th;

#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T in = T(0.0), s = T(0.0), lap = T(0.0), grad = T(0.0);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      s -= T(2.0) * Au[sp(i, j)] * z.dal[j];
      in -= gim[i][j] * (T(2.0) * z.dKh[j] + z.dTh[j]) * T(1.0 / 3.0) + T(3.0) * iW * Au[sp(i, j)] * z.dW[j]
          + T(8.0) * PI * gim[i][j] * Si[j];
      grad += gim[i][j] * (z.ddb[0][sp(j, 0)] + z.ddb[1][sp(j, 1)] + z.ddb[2][sp(j, 2)]);
      s -= G.Gd[j] * z.db[i][j];
    }
#pragma unroll
    for (int a = 0; a < 6; ++a) in += (a == 0 || a == 3 || a == 5 ? T(1.0) : T(2.0)) * G.G2[i][a] * Au[a];
    lap = gi.xx * z.ddb[i][0] + gi.yy * z.ddb[i][3] + gi.zz * z.ddb[i][5]
        + T(2.0) * (gi.xy * z.ddb[i][1] + gi.xz * z.ddb[i][2] + gi.yz * z.ddb[i][4]);
    s += T(2.0) * al * in + (T(2.0) / T(3.0)) * G.Gd[i] * divb + lap + grad * T(1.0 / 3.0) - T(2.0) * al * kap * (z.Gt[i] - G.Gd[i]);
    out[fGX + i] = s;
    out[fBBX + i] = s - pv<T>(p.eta_B, p.feta_B) * z.B[i];
  }

  out[fTH] = p.bssn ? T(0)
                    : fz * (T(0.5) * al * (G.Rs - AA + (T(2.0) / T(3.0)) * K * K) - T(8.0) * PI * al * E) - T(2.0) * al * kap * z.Th;
  out[fAL] = -T(2.0) * al * z.Kh;
#pragma unroll
  for (int i = 0; i < 3; ++i) out[fBX + i] = T(0.75) * z.B[i];
}

}  // namespace sacra
