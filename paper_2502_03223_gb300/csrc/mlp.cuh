// Learned seed of the primitive recovery (no counterpart in the paper): a
// 9 -> 64 -> 64 -> 1 tanh network with BF16 weights and FP32 arithmetic that
// predicts log10(P / D) from the conserved variables and metric invariants.
// The predicted pressure gives a first value of the recovery's unknown z (the
// paper's root variable of Eq. c2p_fn); the FP64 Illinois iteration then runs
// on a narrow bracket around it, and on the full bracket whenever the narrow
// one does not enclose the root, so the converged primitives are those of the
// plain solve to its tolerance.
#pragma once

#include <stdint.h>
#include <string.h>

// included from common.cuh after DevParams, Sym3, the FP32 views and the EOS

namespace sacra {

constexpr int MLP_IN = 9, MLP_H = 64;
constexpr int MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;

// the packed network as the kernels read it (one device copy per context)
struct alignas(16) MlpNet {
  uint16_t w1[MLP_H * MLP_IN];   // BF16, row-major (hidden unit, input)
  uint16_t w2[MLP_H * MLP_H];    // BF16, row-major (out, in)
  uint16_t w3[MLP_H];            // BF16
  uint16_t pad_[4];
  float b1[MLP_H], b2[MLP_H], b3;
  float in_mu[MLP_IN], in_sd[MLP_IN], out_mu, out_sd;
  float delta;                   // relative half-width of the seeded bracket
  float kmin;                    // the seed is tried where k = r / (1 + q) >= kmin
};

__host__ __device__ inline float bf16_to_f32(uint16_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float((unsigned)b << 16);
#else
  unsigned u = (unsigned)b << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}

// round to nearest, ties to even (finite inputs)
__host__ __device__ inline uint16_t f32_to_bf16(float f) {
#ifdef __CUDA_ARCH__
  const unsigned u = __float_as_uint(f);
#else
  unsigned u;
  memcpy(&u, &f, 4);
#endif
  return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

// The 9 inputs, from the recovery's own quantities: D, q = E/D - 1, r = |S|/D
// (Eq. c2p_fn), k = r / (1 + q), the conformal factor W and invariants of the
// conformal metric (tr gt - 3, tr gt^-1 - 3, h_ij h_ij), and the cold-curve
// scale log10(P_cold(D) / D).
__device__ __forceinline__ void c2p_features(const DevParams &p, double D, double qq, double r, double k, double W,
                                             const Sym3 &gt, const Sym3 &gi, float x[MLP_IN]) {
  const float Df = f32_of(D);
  x[0] = log10f(Df);
  x[1] = log10f(1.0f + f32_of(qq));
  x[2] = f32_of(r);
  x[3] = f32_of(k);
  x[4] = log10f(f32_of(W));
  x[5] = (f32_of(gt.xx) - 1.0f) + (f32_of(gt.yy) - 1.0f) + (f32_of(gt.zz) - 1.0f);
  x[6] = (f32_of(gi.xx) - 1.0f) + (f32_of(gi.yy) - 1.0f) + (f32_of(gi.zz) - 1.0f);
  const float hxx = f32_of(gt.xx) - 1.0f, hyy = f32_of(gt.yy) - 1.0f, hzz = f32_of(gt.zz) - 1.0f;
  const float hxy = f32_of(gt.xy), hxz = f32_of(gt.xz), hyz = f32_of(gt.yz);
  x[7] = hxx * hxx + hyy * hyy + hzz * hzz + 2.0f * (hxy * hxy + hxz * hxz + hyz * hyz);
  x[8] = p.K_zero ? 0.0f : log10f(eos_pc<float>(p, Df) / Df);
}

// two BF16 values packed in a 32-bit word -> floats (low half first)
__device__ __forceinline__ void bf16x2(unsigned u, float &lo, float &hi) {
  lo = __uint_as_float(u << 16);
  hi = __uint_as_float(u & 0xFFFF0000u);
}

// y = log10(P / D) predicted (FP32 accumulation over BF16 weights, read 8 at a time)
__device__ inline float mlp_forward(const MlpNet *__restrict__ net, const float x[MLP_IN]) {
  float xh[MLP_IN];
#pragma unroll
  for (int i = 0; i < MLP_IN; ++i) xh[i] = (x[i] - net->in_mu[i]) / net->in_sd[i];
  float h1[MLP_H];
  const unsigned *w1 = reinterpret_cast<const unsigned *>(net->w1);   // 9 inputs per row: pairs span rows
#pragma unroll
  for (int j = 0; j < MLP_H; ++j) h1[j] = net->b1[j];
#pragma unroll
  for (int q = 0; q < MLP_H * MLP_IN / 2; ++q) {
    float lo, hi;
    bf16x2(w1[q], lo, hi);
    const int e0 = 2 * q, e1 = 2 * q + 1;
    h1[e0 / MLP_IN] += lo * xh[e0 % MLP_IN];
    h1[e1 / MLP_IN] += hi * xh[e1 % MLP_IN];
  }
#pragma unroll
  for (int j = 0; j < MLP_H; ++j) h1[j] = tanhf(h1[j]);
  float y = net->b3;
  const uint4 *w2 = reinterpret_cast<const uint4 *>(net->w2);
  const unsigned *w3 = reinterpret_cast<const unsigned *>(net->w3);
  for (int j = 0; j < MLP_H; j += 2) {
    float a0 = net->b2[j], a1 = net->b2[j + 1];
#pragma unroll
    for (int c = 0; c < MLP_H / 8; ++c) {
      const uint4 u = w2[j * (MLP_H / 8) + c], v = w2[(j + 1) * (MLP_H / 8) + c];
      float l, h;
      bf16x2(u.x, l, h); a0 += l * h1[8 * c + 0] + h * h1[8 * c + 1];
      bf16x2(u.y, l, h); a0 += l * h1[8 * c + 2] + h * h1[8 * c + 3];
      bf16x2(u.z, l, h); a0 += l * h1[8 * c + 4] + h * h1[8 * c + 5];
      bf16x2(u.w, l, h); a0 += l * h1[8 * c + 6] + h * h1[8 * c + 7];
      bf16x2(v.x, l, h); a1 += l * h1[8 * c + 0] + h * h1[8 * c + 1];
      bf16x2(v.y, l, h); a1 += l * h1[8 * c + 2] + h * h1[8 * c + 3];
      bf16x2(v.z, l, h); a1 += l * h1[8 * c + 4] + h * h1[8 * c + 5];
      bf16x2(v.w, l, h); a1 += l * h1[8 * c + 6] + h * h1[8 * c + 7];
    }
    float o0, o1;
    bf16x2(w3[j / 2], o0, o1);
    y += o0 * tanhf(a0) + o1 * tanhf(a1);
  }
  return net->out_mu + net->out_sd * y;
}

}  // namespace sacra
