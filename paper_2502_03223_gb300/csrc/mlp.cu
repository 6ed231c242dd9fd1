// Learned seed of the primitive recovery: the tuples the solver generates,
// and the network's training on the GPU (forward, backward and Adam in this
// file's kernels).  Inference runs inside the recovery (common.cuh).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "kernels.h"

namespace sacra {

constexpr int MLP_TUPLE = MLP_IN + 1;   // 9 features, target log10(P / D)
constexpr int MLP_S = 128;              // samples per block in training

// ---------------------------------------------------------------- tuples from the solver's state

// One tuple per interior cell of the level whose recovery is non-trivial (moving
// fluid, above the atmosphere, no cold or atmosphere branch): the inputs the
// recovery computes from (q, W, gt) and the converged log10(P / D).  Cell i of
// the level (row-major over the interior) gives the tuple; false if none.
__device__ inline bool collect_cell(const Lev &L, const DevParams &p, int i, float x[MLP_IN], float *y) {
  if (i >= L.nx * L.nz) return false;
  const int j = 1 + i % L.nx, k = 1 + i / L.nx;
  const size_t P = L.P;
  const int id = cid(L, j, k);
  if (L.status[id] & (ST_ATM | ST_COLD | ST_BAD | ST_NOCONV)) return false;
  const double rho = L.prim[(size_t)pRHO * P + id], Pr = L.prim[(size_t)pP * P + id];
  if (!(rho > 10.0 * p.rho_atm) || !(Pr > 0.0)) return false;
  const Sym3 gt = conf_metric(L.un, P, id);
  const Sym3 gi = s3inv(gt, (double *)nullptr);
  const double W = L.un[(size_t)fW * P + id];
  const double W3 = W * W * W;
  const double D = L.un[(size_t)fQD * P + id] * W3;
  double S[3] = {L.un[(size_t)fQSX * P + id] * W3, L.un[(size_t)fQSY * P + id] * W3, L.un[(size_t)fQSZ * P + id] * W3};
  if (p.geometry == SACRA_CYLINDRICAL) S[1] /= (j - 0.5) * L.dx;
  const double E = L.un[(size_t)fQE * P + id] * W3;
  const double r = sqrt(W * W * s3quad(gi, S, S)) / D;
  if (!(r > 0.0) || !(D > 0.0)) return false;
  const double qq = E / D - 1.0;
  const double kk = fmin(r / (1.0 + qq), p.c2p_kmax);
  c2p_features(p, D, qq, r, kk, W, gt, gi, x);
  *y = log10f(f32_of(Pr / D));
  return true;
}

// The tuples are written in cell order (levels in call order), so that the
// training set, its held-out split and the trained network do not depend on
// the order in which threads ran: a count per block of MC_B cells, a scan of
// those counts (from the running total of earlier calls), then each cell's
// slot = its block's offset + its rank among the block's tuples.
constexpr int MC_B = 256;

__global__ void __launch_bounds__(MC_B) k_mlp_count(Lev L, DevParams p, int *__restrict__ bcount) {
  float x[MLP_IN], y;
  const bool v = collect_cell(L, p, blockIdx.x * MC_B + threadIdx.x, x, &y);
  const int c = __syncthreads_count(v);
  if (threadIdx.x == 0) bcount[blockIdx.x] = c;
}

__global__ void k_mlp_scan(const int *__restrict__ bcount, int nb, unsigned long long *__restrict__ count,
                           unsigned long long *__restrict__ boff) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned long long base = *count;
  for (int b = 0; b < nb; ++b) {
    boff[b] = base;
    base += (unsigned long long)bcount[b];
  }
  *count = base;
}

__global__ void __launch_bounds__(MC_B) k_mlp_write(Lev L, DevParams p, const unsigned long long *__restrict__ boff,
                                                    float *__restrict__ out, long long cap) {
  __shared__ int wsum[MC_B / 32];
  float x[MLP_IN], y = 0.0f;
  const bool v = collect_cell(L, p, blockIdx.x * MC_B + threadIdx.x, x, &y);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned m = __ballot_sync(0xffffffffu, v);
  if (lane == 0) wsum[w] = __popc(m);
  __syncthreads();
  int before = __popc(m & ((1u << lane) - 1u));
  for (int q = 0; q < w; ++q) before += wsum[q];
  if (!v) return;
  const unsigned long long slot = boff[blockIdx.x] + (unsigned long long)before;
  if ((long long)slot >= cap) return;
  float *o = out + slot * MLP_TUPLE;
#pragma unroll
  for (int a = 0; a < MLP_IN; ++a) o[a] = x[a];
  o[MLP_IN] = y;
}

// ---------------------------------------------------------------- training

// counter-based index of training sample `slot` of step `step` (splitmix64 mix)
__host__ __device__ inline unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Samples with index % 5 == 4 are held out; training draws from the others.
__device__ inline long long train_index(unsigned long long seed, int step, int slot, long long n) {
  const long long groups = n / 5;
  const unsigned long long h = mix64(seed ^ mix64(((unsigned long long)step << 32) | (unsigned)slot));
  return 5 * (long long)(h % (unsigned long long)groups) + (long long)((h >> 40) % 4);
}

struct MlpStats {
  float in_mu[MLP_IN], in_sd[MLP_IN], out_mu, out_sd;
};

// One block: MLP_S samples (a minibatch slice, or consecutive samples when
// steps < 0) forward and backward with the BF16 weights of `net`; writes
// the block's partial gradient of L = (1/norm) sum (yh - th)^2 (flat order:
// w1, b1, w2, b2, w3, b3) and its partial loss.
__global__ void __launch_bounds__(MLP_S) k_mlp_grad(const float *__restrict__ samples, long long n, const MlpNet *net,
                                                    unsigned long long seed, int step, float norm,
                                                    float *__restrict__ partial, float *__restrict__ partial_loss) {
  extern __shared__ float sm[];
  float *w1 = sm;                                 // 64 x 9
  float *w2 = w1 + MLP_H * MLP_IN;                // 64 x 64
  float *w3 = w2 + MLP_H * MLP_H;                 // 64
  float *xs = w3 + MLP_H;                         // S x 9
  float *h1 = xs + MLP_S * MLP_IN;                // S x 64
  float *h2 = h1 + MLP_S * MLP_H;
  float *d1 = h2 + MLP_S * MLP_H;
  float *d2 = d1 + MLP_S * MLP_H;
  float *es = d2 + MLP_S * MLP_H;                 // S
  const int t = threadIdx.x;
  for (int q = t; q < MLP_H * MLP_IN; q += MLP_S) w1[q] = bf16_to_f32(net->w1[q]);
  for (int q = t; q < MLP_H * MLP_H; q += MLP_S) w2[q] = bf16_to_f32(net->w2[q]);
  for (int q = t; q < MLP_H; q += MLP_S) w3[q] = bf16_to_f32(net->w3[q]);
  __syncthreads();
  // this thread's sample
  long long idx;
  bool live;
  if (step >= 0) {
    idx = train_index(seed, step, blockIdx.x * MLP_S + t, n);
    live = true;
  } else {
    idx = (long long)blockIdx.x * MLP_S + t;
    live = idx < n;
  }
  float *x = xs + t * MLP_IN, *a1 = h1 + t * MLP_H, *a2 = h2 + t * MLP_H;
  float e = 0.0f;
  if (live) {
    const float *s = samples + idx * MLP_TUPLE;
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) x[i] = (s[i] - net->in_mu[i]) / net->in_sd[i];
    const float th = (s[MLP_IN] - net->out_mu) / net->out_sd;
    for (int jj = 0; jj < MLP_H; ++jj) {
      float a = net->b1[jj];
#pragma unroll
      for (int i = 0; i < MLP_IN; ++i) a += w1[jj * MLP_IN + i] * x[i];
      a1[jj] = tanhf(a);
    }
    float yh = net->b3;
    for (int jj = 0; jj < MLP_H; ++jj) {
      float a = net->b2[jj];
      for (int i = 0; i < MLP_H; ++i) a += w2[jj * MLP_H + i] * a1[i];
      a2[jj] = tanhf(a);
      yh += w3[jj] * a2[jj];
    }
    e = 2.0f * (yh - th) / norm;
    float *g2 = d2 + t * MLP_H, *g1 = d1 + t * MLP_H;
    for (int jj = 0; jj < MLP_H; ++jj) g2[jj] = e * w3[jj] * (1.0f - a2[jj] * a2[jj]);
    for (int i = 0; i < MLP_H; ++i) {
      float s2 = 0.0f;
      for (int jj = 0; jj < MLP_H; ++jj) s2 += w2[jj * MLP_H + i] * g2[jj];
      g1[i] = s2 * (1.0f - a1[i] * a1[i]);
    }
    partial_loss[(size_t)blockIdx.x * MLP_S + t] = (yh - th) * (yh - th) / norm;
  } else {
    for (int i = 0; i < MLP_IN; ++i) x[i] = 0.0f;
    for (int jj = 0; jj < MLP_H; ++jj) { a1[jj] = a2[jj] = 0.0f; d1[t * MLP_H + jj] = d2[t * MLP_H + jj] = 0.0f; }
    partial_loss[(size_t)blockIdx.x * MLP_S + t] = 0.0f;
  }
  es[t] = e;
  __syncthreads();
  // block sums over its samples, one parameter per thread at a time (fixed order)
  float *g = partial + (size_t)blockIdx.x * MLP_NPARAM;
  for (int q = t; q < MLP_NPARAM; q += MLP_S) {
    float acc = 0.0f;
    int o = q;
    if (o < MLP_H * MLP_IN) {                       // w1[i][k]
      const int i = o / MLP_IN, kk = o % MLP_IN;
      for (int s = 0; s < MLP_S; ++s) acc += d1[s * MLP_H + i] * xs[s * MLP_IN + kk];
    } else if ((o -= MLP_H * MLP_IN) < MLP_H) {     // b1[i]
      for (int s = 0; s < MLP_S; ++s) acc += d1[s * MLP_H + o];
    } else if ((o -= MLP_H) < MLP_H * MLP_H) {      // w2[j][i]
      const int jj = o / MLP_H, i = o % MLP_H;
      for (int s = 0; s < MLP_S; ++s) acc += d2[s * MLP_H + jj] * h1[s * MLP_H + i];
    } else if ((o -= MLP_H * MLP_H) < MLP_H) {      // b2[j]
      for (int s = 0; s < MLP_S; ++s) acc += d2[s * MLP_H + o];
    } else if ((o -= MLP_H) < MLP_H) {              // w3[j]
      for (int s = 0; s < MLP_S; ++s) acc += es[s] * h2[s * MLP_H + o];
    } else {                                        // b3
      for (int s = 0; s < MLP_S; ++s) acc += es[s];
    }
    g[q] = acc;
  }
}

// sum of the block partials (fixed order), then Adam on the FP32 master weights
// and the BF16 / FP32 copies the network uses
__global__ void k_mlp_adam(const float *__restrict__ partial, int nblocks, float *__restrict__ theta,
                           float *__restrict__ m, float *__restrict__ v, MlpNet *net, float lr, float b1t, float b2t) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= MLP_NPARAM) return;
  float g = 0.0f;
  for (int b = 0; b < nblocks; ++b) g += partial[(size_t)b * MLP_NPARAM + q];
  const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  const float mq = beta1 * m[q] + (1.0f - beta1) * g;
  const float vq = beta2 * v[q] + (1.0f - beta2) * g * g;
  m[q] = mq;
  v[q] = vq;
  const float th = theta[q] - lr * (mq / b1t) / (sqrtf(vq / b2t) + eps);
  theta[q] = th;
  int o = q;
  if (o < MLP_H * MLP_IN) { net->w1[o] = f32_to_bf16(th); return; }
  if ((o -= MLP_H * MLP_IN) < MLP_H) { net->b1[o] = th; return; }
  if ((o -= MLP_H) < MLP_H * MLP_H) { net->w2[o] = f32_to_bf16(th); return; }
  if ((o -= MLP_H * MLP_H) < MLP_H) { net->b2[o] = th; return; }
  if ((o -= MLP_H) < MLP_H) { net->w3[o] = f32_to_bf16(th); return; }
  net->b3 = th;
}

__global__ void k_mlp_sum(const float *__restrict__ partial, int nblocks, float *__restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= MLP_NPARAM) return;
  float g = 0.0f;
  for (int b = 0; b < nblocks; ++b) g += partial[(size_t)b * MLP_NPARAM + q];
  out[q] = g;
}

// feature and target moments over the training samples: per block sums of x and x^2
__global__ void k_mlp_moments(const float *__restrict__ samples, long long n, double *__restrict__ partial) {
  __shared__ double sh[2 * MLP_TUPLE][128];
  const int t = threadIdx.x;
  double acc[2 * MLP_TUPLE];
#pragma unroll
  for (int a = 0; a < 2 * MLP_TUPLE; ++a) acc[a] = 0.0;
  for (long long i = (long long)blockIdx.x * 128 + t; i < n; i += (long long)gridDim.x * 128) {
    if (i % 5 == 4) continue;
#pragma unroll
    for (int a = 0; a < MLP_TUPLE; ++a) {
      const double s = samples[i * MLP_TUPLE + a];
      acc[a] += s;
      acc[MLP_TUPLE + a] += s * s;
    }
  }
#pragma unroll
  for (int a = 0; a < 2 * MLP_TUPLE; ++a) sh[a][t] = acc[a];
  __syncthreads();
  if (t < 2 * MLP_TUPLE) {
    double s = 0.0;
    for (int q = 0; q < 128; ++q) s += sh[t][q];
    partial[(size_t)blockIdx.x * 2 * MLP_TUPLE + t] = s;
  }
}

// relative error of the seed z0 on held-out samples: |z(pred) / z(true) - 1|
__global__ void k_mlp_eval(const float *__restrict__ samples, long long n, const MlpNet *net, float *__restrict__ zerr,
                           float *__restrict__ yerr) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long i = 5 * g + 4;
  if (i >= n) return;
  const float *s = samples + i * MLP_TUPLE;
  float x[MLP_IN];
#pragma unroll
  for (int a = 0; a < MLP_IN; ++a) x[a] = s[a];
  const float y = mlp_forward(net, x);
  const float q1 = exp10f(x[1]), r = x[2];   // 1 + q, r
  auto zof = [&](float yy) {
    const float v = r / (q1 + exp10f(yy));
    return v * rsqrtf(fmaxf(1.0f - v * v, 1e-30f));
  };
  zerr[g] = fabsf(zof(y) / zof(s[MLP_IN]) - 1.0f);
  yerr[g] = fabsf(y - s[MLP_IN]);
}

size_t mlp_grad_smem() {
  return sizeof(float) * (MLP_H * MLP_IN + MLP_H * MLP_H + MLP_H + MLP_S * MLP_IN + 4 * MLP_S * MLP_H + MLP_S);
}

// ---------------------------------------------------------------- host side

size_t mlp_collect_scratch_bytes(const Lev &L) {
  const size_t nb = (size_t)(L.nx * L.nz + MC_B - 1) / MC_B;
  return nb * sizeof(unsigned long long) + nb * sizeof(int);
}

void launch_mlp_collect(const Lev &L, const DevParams &p, float *out, long long cap, unsigned long long *count,
                        void *scratch, cudaStream_t s) {
  const int nb = (L.nx * L.nz + MC_B - 1) / MC_B;
  unsigned long long *boff = reinterpret_cast<unsigned long long *>(scratch);
  int *bcount = reinterpret_cast<int *>(boff + nb);
  k_mlp_count<<<nb, MC_B, 0, s>>>(L, p, bcount);
  k_mlp_scan<<<1, 32, 0, s>>>(bcount, nb, count, boff);
  k_mlp_write<<<nb, MC_B, 0, s>>>(L, p, boff, out, cap);
}

namespace {

struct DevBuf {
  void *p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  bool alloc(size_t bytes) { return cudaMalloc(&p, bytes) == cudaSuccess; }
};

// Glorot-uniform initial weights from a splitmix64 stream, zero biases
void init_theta(unsigned long long seed, std::vector<float> &theta) {
  theta.assign(MLP_NPARAM, 0.0f);
  unsigned long long st = seed;
  auto uni = [&]() { st = mix64(st); return (double)(st >> 11) * (1.0 / 9007199254740992.0); };
  size_t o = 0;
  const double a1 = sqrt(6.0 / (MLP_IN + MLP_H)), a2 = sqrt(6.0 / (MLP_H + MLP_H)), a3 = sqrt(6.0 / (MLP_H + 1));
  for (int q = 0; q < MLP_H * MLP_IN; ++q) theta[o++] = (float)((2.0 * uni() - 1.0) * a1);
  o += MLP_H;
  for (int q = 0; q < MLP_H * MLP_H; ++q) theta[o++] = (float)((2.0 * uni() - 1.0) * a2);
  o += MLP_H;
  for (int q = 0; q < MLP_H; ++q) theta[o++] = (float)((2.0 * uni() - 1.0) * a3);
}

void pack(const std::vector<float> &theta, MlpNet &net) {
  size_t o = 0;
  for (int q = 0; q < MLP_H * MLP_IN; ++q) net.w1[q] = f32_to_bf16(theta[o++]);
  for (int q = 0; q < MLP_H; ++q) net.b1[q] = theta[o++];
  for (int q = 0; q < MLP_H * MLP_H; ++q) net.w2[q] = f32_to_bf16(theta[o++]);
  for (int q = 0; q < MLP_H; ++q) net.b2[q] = theta[o++];
  for (int q = 0; q < MLP_H; ++q) net.w3[q] = f32_to_bf16(theta[o++]);
  net.b3 = theta[o++];
}

}  // namespace

int mlp_train(const float *samples, long long n, int steps, int batch_blocks, float lr, unsigned long long seed,
              float kmin, MlpNet *dev_net, float *host_loss, float *host_report, cudaStream_t s) {
  if (!samples || n < 50 || steps < 0 || batch_blocks < 1 || !dev_net || !(lr > 0)) return -1;
  // moments of the training samples -> normalisation
  const int mb = 256;
  DevBuf mom;
  if (!mom.alloc(sizeof(double) * mb * 2 * MLP_TUPLE)) return -3;
  k_mlp_moments<<<mb, 128, 0, s>>>(samples, n, (double *)mom.p);
  std::vector<double> hm((size_t)mb * 2 * MLP_TUPLE);
  cudaMemcpyAsync(hm.data(), mom.p, hm.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return -2;
  long long ntr = 0;
  for (long long i = 0; i < n; ++i) ntr += (i % 5 != 4);
  MlpNet net;
  memset(&net, 0, sizeof(net));
  for (int a = 0; a < MLP_TUPLE; ++a) {
    double sx = 0.0, sxx = 0.0;
    for (int b = 0; b < mb; ++b) {
      sx += hm[(size_t)b * 2 * MLP_TUPLE + a];
      sxx += hm[(size_t)b * 2 * MLP_TUPLE + MLP_TUPLE + a];
    }
    const double mu = sx / ntr, var = std::max(sxx / ntr - mu * mu, 0.0);
    const double sd = var > 1e-24 ? sqrt(var) : 1.0;
    if (a < MLP_IN) { net.in_mu[a] = (float)mu; net.in_sd[a] = (float)sd; }
    else { net.out_mu = (float)mu; net.out_sd = (float)sd; }
  }
  std::vector<float> theta;
  init_theta(seed, theta);
  pack(theta, net);
  net.delta = 0.05f;
  net.kmin = kmin;
  cudaMemcpyAsync(dev_net, &net, sizeof(net), cudaMemcpyHostToDevice, s);
  DevBuf th, m, v, part, ploss;
  const size_t P = MLP_NPARAM;
  if (!th.alloc(P * 4) || !m.alloc(P * 4) || !v.alloc(P * 4) || !part.alloc((size_t)batch_blocks * P * 4) ||
      !ploss.alloc((size_t)batch_blocks * MLP_S * 4))
    return -3;
  cudaMemcpyAsync(th.p, theta.data(), P * 4, cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(m.p, 0, P * 4, s);
  cudaMemsetAsync(v.p, 0, P * 4, s);
  const size_t smem = mlp_grad_smem();
  cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const float norm = (float)batch_blocks * MLP_S;
  std::vector<float> lossbuf((size_t)batch_blocks * MLP_S);
  double b1t = 1.0, b2t = 1.0;
  for (int it = 0; it < steps; ++it) {
    k_mlp_grad<<<batch_blocks, MLP_S, smem, s>>>(samples, n, dev_net, seed, it, norm, (float *)part.p, (float *)ploss.p);
    b1t *= 0.9;
    b2t *= 0.999;
    // cosine decay from lr to lr / 100
    const double lr_t = lr * (0.01 + 0.99 * 0.5 * (1.0 + cos(M_PI * it / std::max(steps, 1))));
    k_mlp_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>((const float *)part.p, batch_blocks, (float *)th.p,
                                                         (float *)m.p, (float *)v.p, dev_net, (float)lr_t,
                                                         (float)(1.0 - b1t), (float)(1.0 - b2t));
    if (host_loss) {
      cudaMemcpyAsync(lossbuf.data(), ploss.p, lossbuf.size() * 4, cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) return -2;
      double l = 0.0;
      for (float x : lossbuf) l += x;
      host_loss[it] = (float)l;
    }
  }
  // held-out error of the seed -> the bracket half-width
  const long long nval = n / 5;
  DevBuf ze, ye;
  if (nval < 1 || !ze.alloc(nval * 4) || !ye.alloc(nval * 4)) return -3;
  k_mlp_eval<<<(unsigned)((nval + 127) / 128), 128, 0, s>>>(samples, n, dev_net, (float *)ze.p, (float *)ye.p);
  std::vector<float> hz(nval), hy(nval);
  cudaMemcpyAsync(hz.data(), ze.p, nval * 4, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(hy.data(), ye.p, nval * 4, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return -2;
  std::vector<float> sz = hz;
  const size_t q = std::min<size_t>(sz.size() - 1, (size_t)(0.999 * sz.size()));
  std::nth_element(sz.begin(), sz.begin() + q, sz.end());
  const float zq = sz[q];
  const float delta = std::min(0.05f, std::max(1e-5f, 2.0f * zq));   // twice the 99.9th percentile
  cudaMemcpyAsync(&dev_net->delta, &delta, sizeof(float), cudaMemcpyHostToDevice, s);
  if (host_report) {
    double sy = 0.0;
    for (float x : hy) sy += (double)x * x;
    host_report[0] = (float)sqrt(sy / hy.size());   // held-out RMS error of log10(P / D)
    host_report[1] = zq;                             // 99.9th percentile of the seed's relative z error
    host_report[2] = delta;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return -2;
  return 0;
}

int mlp_grad(const float *samples, long long n, const MlpNet *dev_net, float *host_grad, float *host_loss,
             cudaStream_t s) {
  if (!samples || n < 1 || !dev_net || !host_grad) return -1;
  const int nb = (int)((n + MLP_S - 1) / MLP_S);
  DevBuf part, ploss, out;
  if (!part.alloc((size_t)nb * MLP_NPARAM * 4) || !ploss.alloc((size_t)nb * MLP_S * 4) || !out.alloc(MLP_NPARAM * 4))
    return -3;
  const size_t smem = mlp_grad_smem();
  cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_mlp_grad<<<nb, MLP_S, smem, s>>>(samples, n, dev_net, 0ull, -1, (float)n, (float *)part.p, (float *)ploss.p);
  k_mlp_sum<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>((const float *)part.p, nb, (float *)out.p);
  cudaMemcpyAsync(host_grad, out.p, MLP_NPARAM * 4, cudaMemcpyDeviceToHost, s);
  std::vector<float> lb((size_t)nb * MLP_S);
  cudaMemcpyAsync(lb.data(), ploss.p, lb.size() * 4, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return -2;
  if (host_loss) {
    double l = 0.0;
    for (float x : lb) l += x;
    *host_loss = (float)l;
  }
  return 0;
}

}  // namespace sacra
