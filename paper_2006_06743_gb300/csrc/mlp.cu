// mlp.cu -- the core-point surrogate: a d -> 128 -> 128 -> 1 perceptron with
// exact (erf) GELU, trained and evaluated by this file's kernels.
//
// The paper has no learned component.  The surrogate predicts, from a point's
// coordinates, whether Algorithm 1 would make it a core point (step 3), so
// that confidently classified points can skip most of their sampled queries
// (step 2).  Weights are stored as an FP32 master vector; every kernel rounds
// them to FP16 when it stages them in shared memory and accumulates in FP32.
//
// Parameter vector (FP32, device), d = input features, H = 128:
//   [W1 (H x d) | b1 (H) | W2 (H x H) | b2 (H) | w3 (H) | b3 (1) | mean (d) | std (d)]
// The first H*d + H*H + 3H + 1 entries are trained; mean/std standardise the
// inputs (u = (x - mean) / std) and come from sng_mlp_standardize.
//
// Forward (per point):   a1 = W1 u + b1, h1 = gelu(a1), a2 = W2 h1 + b2,
//                        h2 = gelu(a2), z = w3 . h2 + b3, p = sigmoid(z)
// Loss: mean binary cross-entropy on the logit z.  Backward: the chain rule,
// gelu'(t) = Phi(t) + t phi(t).  Optimiser: Adam with bias correction.
#include <cmath>
#include <cuda_fp16.h>

#include "api_common.cuh"
#include "graph.cuh"

namespace sng {

constexpr int kH = 128;
constexpr int32_t kDegUnit = 16;  // degree units per draw when reweighting

struct MlpOff {
  int64_t w1, b1, w2, b2, w3, b3, train, mean, std, total;
};

__host__ __device__ inline MlpOff mlp_off(int d) {
  MlpOff o;
  o.w1 = 0;
  o.b1 = (int64_t)kH * d;
  o.w2 = o.b1 + kH;
  o.b2 = o.w2 + (int64_t)kH * kH;
  o.w3 = o.b2 + kH;
  o.b3 = o.w3 + kH;
  o.train = o.b3 + 1;
  o.mean = o.train;
  o.std = o.mean + d;
  o.total = o.std + d;
  return o;
}

__device__ __forceinline__ float h16(float v) { return __half2float(__float2half_rn(v)); }

__device__ __forceinline__ float gelu_f(float a) {
  return 0.5f * a * (1.f + erff(a * 0.70710678118654752f));
}

__device__ __forceinline__ float gelu_grad_f(float a) {
  return 0.5f * (1.f + erff(a * 0.70710678118654752f)) +
         a * 0.39894228040143268f * expf(-0.5f * a * a);
}

// Shared-memory image of the network for DMAX input features:
//   W1 [H][DMAX] | b1 [H] | W2T [H][H] (W2T[j][t] = W2[t][j]) | b2 [H] | w3 [H]
//   | b3 | mean [DMAX] | istd [DMAX]
template <int DMAX>
struct Smem {
  static constexpr int w1 = 0;
  static constexpr int b1 = w1 + kH * DMAX;
  static constexpr int w2t = b1 + kH;
  static constexpr int b2 = w2t + kH * kH;
  static constexpr int w3 = b2 + kH;
  static constexpr int b3 = w3 + kH;
  static constexpr int mean = b3 + 4;
  static constexpr int istd = mean + DMAX;
  static constexpr int total = istd + DMAX;
  static constexpr size_t bytes = sizeof(float) * total;
};

template <int DMAX>
__device__ void stage_weights(const float *P, int d, float *s) {
  const MlpOff o = mlp_off(d);
  for (int t = threadIdx.x; t < kH * DMAX; t += blockDim.x) {
    const int j = t / DMAX, k = t % DMAX;
    s[Smem<DMAX>::w1 + t] = k < d ? h16(P[o.w1 + (int64_t)j * d + k]) : 0.f;
  }
  for (int t = threadIdx.x; t < kH * kH; t += blockDim.x) {
    const int j = t / kH, tt = t % kH;  // W2T[j][tt] = W2[tt][j]
    s[Smem<DMAX>::w2t + t] = h16(P[o.w2 + (int64_t)tt * kH + j]);
  }
  for (int t = threadIdx.x; t < kH; t += blockDim.x) {
    s[Smem<DMAX>::b1 + t] = h16(P[o.b1 + t]);
    s[Smem<DMAX>::b2 + t] = h16(P[o.b2 + t]);
    s[Smem<DMAX>::w3 + t] = h16(P[o.w3 + t]);
  }
  for (int k = threadIdx.x; k < DMAX; k += blockDim.x) {
    s[Smem<DMAX>::mean + k] = k < d ? P[o.mean + k] : 0.f;
    s[Smem<DMAX>::istd + k] = k < d ? 1.f / P[o.std + k] : 0.f;
  }
  if (threadIdx.x == 0) s[Smem<DMAX>::b3] = h16(P[o.b3]);
  __syncthreads();
}

// One point through the network.  Optionally records u, a1, a2 (training).
template <int DMAX>
__device__ __forceinline__ float forward_point(const float *s, const float *xrow, int d,
                                               float *u_out, float *a1_out, float *a2_out) {
  float u[DMAX];
#pragma unroll
  for (int k = 0; k < DMAX; ++k) {
    u[k] = k < d ? (xrow[k] - s[Smem<DMAX>::mean + k]) * s[Smem<DMAX>::istd + k] : 0.f;
    if (u_out && k < d) u_out[k] = u[k];
  }
  float a2[kH];
#pragma unroll
  for (int t = 0; t < kH; ++t) a2[t] = s[Smem<DMAX>::b2 + t];
#pragma unroll 1
  for (int j = 0; j < kH; ++j) {
    const float *w1r = s + Smem<DMAX>::w1 + j * DMAX;
    float a = s[Smem<DMAX>::b1 + j];
#pragma unroll
    for (int k = 0; k < DMAX; ++k) a = fmaf(w1r[k], u[k], a);
    if (a1_out) a1_out[j] = a;
    const float h = gelu_f(a);
    const float *w2r = s + Smem<DMAX>::w2t + j * kH;
#pragma unroll
    for (int t = 0; t < kH; ++t) a2[t] = fmaf(w2r[t], h, a2[t]);
  }
  float z = s[Smem<DMAX>::b3];
#pragma unroll
  for (int t = 0; t < kH; ++t) {
    if (a2_out) a2_out[t] = a2[t];
    z = fmaf(s[Smem<DMAX>::w3 + t], gelu_f(a2[t]), z);
  }
  return z;
}

// --------------------------------------------------------------- inference

struct GateArgs {
  int32_t fp32_activations;   // 0: mma.sync, 1: CUDA cores with FP32 activations, 2: tcgen05
  const float *x;
  int64_t ld;
  int64_t n;
  int32_t d;
  const float *P;
  float *prob;          // nullable
  float p_noise, p_core;
  int32_t m, m_core, m_noise;  // draws for uncertain / confident-core / -noise points
  int32_t w_full, w_core, w_noise;  // degree weight per kept draw of each class
  uint8_t *forced;      // nullable: 2 noise, 1 core, 0 uncertain
  int32_t by_degree;    // 1: gated points keep the degree test (forced stays 0)
  int32_t *m_row;       // nullable
  int32_t *w_row;       // nullable
  unsigned long long *counters;  // nullable: [0] queries [1] core [2] noise
};

template <int DMAX>
__global__ void __launch_bounds__(128, 1) mlp_gate_kernel(GateArgs a) {
  extern __shared__ float smem_w[];
  stage_weights<DMAX>(a.P, a.d, smem_w);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long q = 0, nc = 0, nn = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    const float z = forward_point<DMAX>(smem_w, a.x + i * a.ld, a.d, nullptr, nullptr, nullptr);
    const float p = 1.f / (1.f + expf(-z));
    if (a.prob) a.prob[i] = p;
    if (a.forced) {
      uint8_t f = 0;
      int32_t mi = a.m, wi = a.w_full;
      if (p < a.p_noise) {
        f = 2;
        mi = a.m_noise;
        wi = a.w_noise;
        ++nn;
      } else if (p > a.p_core) {
        f = 1;
        mi = a.m_core;
        wi = a.w_core;
        ++nc;
      }
      a.forced[i] = a.by_degree ? 0 : f;
      a.m_row[i] = mi;
      if (a.w_row) a.w_row[i] = wi;
      q += (unsigned long long)mi;
    }
  }
  if (a.counters) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      q += __shfl_xor_sync(kFullMask, q, o);
      nc += __shfl_xor_sync(kFullMask, nc, o);
      nn += __shfl_xor_sync(kFullMask, nn, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(a.counters + 0, q);
      atomicAdd(a.counters + 1, nc);
      atomicAdd(a.counters + 2, nn);
    }
  }
}

// ------------------------------------------------ inference on tensor cores
//
// The gate's two dense layers run on the tensor cores with warp-level
// mma.sync.m16n8k16 (FP16 operands, FP32 accumulation): one warp pushes 16
// points through the network.  Layer-1 accumulators (16 x 128) become,
// after bias + GELU and rounding to FP16, exactly the A fragments of layer 2
// in registers (the m16n8 accumulator layout of two adjacent n-tiles is the
// m16k16 A layout), so hidden activations never touch memory.  Weights are
// staged once per block in shared memory as FP16, rows padded so the
// fragment loads are free of bank conflicts.  Activations are FP16 at the MMA
// inputs (standardised inputs and layer-1 outputs).
//
// Fragment layouts (PTX ISA, mma.m16n8k16, g = lane / 4, q = lane % 4):
//   A (16x16, row): a0 = (g, 2q..2q+1), a1 = (g+8, 2q..), a2 = (g, 2q+8..),
//                   a3 = (g+8, 2q+8..)
//   B (16x8, col):  b0 = (k = 2q..2q+1, n = g), b1 = (k = 2q+8.., n = g)
//   C (16x8):       c0,c1 = (g, 2q..2q+1), c2,c3 = (g+8, 2q..2q+1)

constexpr int kW1Pad = 8;                 // halves of padding per W1 row
constexpr int kW2Stride = kH + 8;         // halves per W2 row (136)

template <int KT1>
struct MmaSmem {
  static constexpr int k1 = 16 * KT1;                    // padded input width
  static constexpr int w1_stride = k1 + kW1Pad;          // halves per W1 row
  static constexpr size_t w1 = 0;                        // half [H][w1_stride]
  static constexpr size_t w2 = w1 + sizeof(__half) * kH * w1_stride;   // half [H][136]
  static constexpr size_t fp = w2 + sizeof(__half) * kH * kW2Stride;   // float params
  // float params: b1[H] b2[H] w3[H] b3 pad[3] mean[k1] istd[k1]
  static constexpr size_t fp_count = 3 * kH + 4 + 2 * k1;
  static constexpr size_t xs = fp + sizeof(float) * fp_count;          // float [warps][16][k1]
  static constexpr size_t bytes(int warps) { return xs + sizeof(float) * warps * 16 * k1; }
};

__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, "
      "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int KT1>
__global__ void __launch_bounds__(128) mlp_gate_mma_kernel(GateArgs a) {
  using L = MmaSmem<KT1>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __half *w1s = reinterpret_cast<__half *>(smem_raw + L::w1);
  __half *w2s = reinterpret_cast<__half *>(smem_raw + L::w2);
  float *fp = reinterpret_cast<float *>(smem_raw + L::fp);
  float *b1s = fp, *b2s = fp + kH, *w3s = fp + 2 * kH, *b3s = fp + 3 * kH;
  float *means = fp + 3 * kH + 4, *istd = means + L::k1;
  const int d = a.d;
  const MlpOff o = mlp_off(d);
  for (int t = threadIdx.x; t < kH * L::w1_stride; t += blockDim.x) {
    const int j = t / L::w1_stride, k = t % L::w1_stride;
    w1s[t] = __float2half_rn(k < d ? a.P[o.w1 + (int64_t)j * d + k] : 0.f);
  }
  for (int t = threadIdx.x; t < kH * kW2Stride; t += blockDim.x) {
    const int j = t / kW2Stride, k = t % kW2Stride;   // W2s[j][k] = W2[j][k]
    w2s[t] = __float2half_rn(k < kH ? a.P[o.w2 + (int64_t)j * kH + k] : 0.f);
  }
  for (int t = threadIdx.x; t < kH; t += blockDim.x) {
    b1s[t] = h16(a.P[o.b1 + t]);
    b2s[t] = h16(a.P[o.b2 + t]);
    w3s[t] = h16(a.P[o.w3 + t]);
  }
  for (int k = threadIdx.x; k < L::k1; k += blockDim.x) {
    means[k] = k < d ? a.P[o.mean + k] : 0.f;
    istd[k] = k < d ? 1.f / a.P[o.std + k] : 0.f;
  }
  if (threadIdx.x == 0) b3s[0] = h16(a.P[o.b3]);
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, q = lane & 3;
  float *xs = reinterpret_cast<float *>(smem_raw + L::xs) + warp * 16 * L::k1;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned long long nq = 0, nc = 0, nn = 0;
  for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * 16; base < a.n;
       base += warps_total * 16) {
    // stage 16 standardised rows (zero past n and past d)
    for (int t = lane; t < 16 * L::k1; t += 32) {
      const int r = t / L::k1, k = t % L::k1;
      const int64_t i = base + r;
      xs[t] = (i < a.n && k < d) ? (a.x[i * a.ld + k] - means[k]) * istd[k] : 0.f;
    }
    __syncwarp();
    // layer 1: acc1[nt] = U (16 x k1) * W1^T (k1 x 128)
    float acc1[kH / 8][4];
#pragma unroll
    for (int nt = 0; nt < kH / 8; ++nt) acc1[nt][0] = acc1[nt][1] = acc1[nt][2] = acc1[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < KT1; ++kt) {
      uint32_t af[4];
      const float *r0 = xs + g * L::k1 + kt * 16 + 2 * q;
      const float *r1 = xs + (g + 8) * L::k1 + kt * 16 + 2 * q;
      af[0] = pack_h2(r0[0], r0[1]);
      af[1] = pack_h2(r1[0], r1[1]);
      af[2] = pack_h2(r0[8], r0[9]);
      af[3] = pack_h2(r1[8], r1[9]);
#pragma unroll
      for (int nt = 0; nt < kH / 8; ++nt) {
        const __half *wr = w1s + (nt * 8 + g) * L::w1_stride + kt * 16 + 2 * q;
        mma16816(acc1[nt], af, *reinterpret_cast<const uint32_t *>(wr),
                 *reinterpret_cast<const uint32_t *>(wr + 8));
      }
    }
    __syncwarp();
    // bias + GELU -> FP16 A fragments of layer 2 (k-tile kt2 = n-tiles 2kt2, 2kt2+1)
    uint32_t hf[kH / 16][4];
#pragma unroll
    for (int kt2 = 0; kt2 < kH / 16; ++kt2) {
      const int c0 = kt2 * 16 + 2 * q, c1 = c0 + 8;
      const float *lo = acc1[2 * kt2], *hi = acc1[2 * kt2 + 1];
      hf[kt2][0] = pack_h2(gelu_f(lo[0] + b1s[c0]), gelu_f(lo[1] + b1s[c0 + 1]));
      hf[kt2][1] = pack_h2(gelu_f(lo[2] + b1s[c0]), gelu_f(lo[3] + b1s[c0 + 1]));
      hf[kt2][2] = pack_h2(gelu_f(hi[0] + b1s[c1]), gelu_f(hi[1] + b1s[c1 + 1]));
      hf[kt2][3] = pack_h2(gelu_f(hi[2] + b1s[c1]), gelu_f(hi[3] + b1s[c1 + 1]));
    }
    // layer 2 and the output unit, one n-tile of hidden units at a time
    float z0 = 0.f, z1 = 0.f;   // rows g and g + 8
#pragma unroll 2
    for (int nt = 0; nt < kH / 8; ++nt) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kt2 = 0; kt2 < kH / 16; ++kt2) {
        const __half *wr = w2s + (nt * 8 + g) * kW2Stride + kt2 * 16 + 2 * q;
        mma16816(c, hf[kt2], *reinterpret_cast<const uint32_t *>(wr),
                 *reinterpret_cast<const uint32_t *>(wr + 8));
      }
      const int col = nt * 8 + 2 * q;
      z0 = fmaf(w3s[col], gelu_f(c[0] + b2s[col]), z0);
      z0 = fmaf(w3s[col + 1], gelu_f(c[1] + b2s[col + 1]), z0);
      z1 = fmaf(w3s[col], gelu_f(c[2] + b2s[col]), z1);
      z1 = fmaf(w3s[col + 1], gelu_f(c[3] + b2s[col + 1]), z1);
    }
    z0 += __shfl_xor_sync(kFullMask, z0, 1);
    z0 += __shfl_xor_sync(kFullMask, z0, 2);
    z1 += __shfl_xor_sync(kFullMask, z1, 1);
    z1 += __shfl_xor_sync(kFullMask, z1, 2);
    if (q < 2) {
      const int64_t i = base + g + 8 * q;
      const float z = (q == 0 ? z0 : z1) + b3s[0];
      if (i < a.n) {
        const float p = 1.f / (1.f + expf(-z));
        if (a.prob) a.prob[i] = p;
        if (a.forced) {
          uint8_t f = 0;
          int32_t mi = a.m, wi = a.w_full;
          if (p < a.p_noise) {
            f = 2;
            mi = a.m_noise;
            wi = a.w_noise;
            ++nn;
          } else if (p > a.p_core) {
            f = 1;
            mi = a.m_core;
            wi = a.w_core;
            ++nc;
          }
          a.forced[i] = a.by_degree ? 0 : f;
          a.m_row[i] = mi;
          if (a.w_row) a.w_row[i] = wi;
          nq += (unsigned long long)mi;
        }
      }
    }
    __syncwarp();
  }
  if (a.counters) {
#pragma unroll
    for (int o2 = 16; o2 >= 1; o2 >>= 1) {
      nq += __shfl_xor_sync(kFullMask, nq, o2);
      nc += __shfl_xor_sync(kFullMask, nc, o2);
      nn += __shfl_xor_sync(kFullMask, nn, o2);
    }
    if (lane == 0) {
      atomicAdd(a.counters + 0, nq);
      atomicAdd(a.counters + 1, nc);
      atomicAdd(a.counters + 2, nn);
    }
  }
}

// ---------------------------------------------------------------- training

struct TrainWs {
  int32_t B;           // batch rows
  float *u;            // B x d
  float *a1;           // B x H
  float *a2;           // B x H
  float *dz;           // B
  float *da1;          // B x H
  float *da2;          // B x H
  float *grad;         // train-part gradient
  double *loss;        // per-step loss sums
};

struct FwdArgs {
  const float *x;
  const uint8_t *y;
  int64_t n;
  int32_t d;
  const float *P;
  TrainWs ws;
  int32_t sample;      // 1: hash-sampled batch; 0: rows 0..B-1; 2: rows (step*B+b) mod n
  uint64_t seed;
  int64_t step;
  FastMod fm_n;        // remainder constants for n (batch sampling)
  int32_t loss_slot;
};

__device__ __forceinline__ int64_t batch_row(const FwdArgs &a, int b) {
  if (!a.sample) return b;
  if (a.sample == 2) return (int64_t)(((uint64_t)a.step * (uint64_t)a.ws.B + (uint64_t)b) %
                                      (uint64_t)a.n);
  const uint64_t k = mix64(a.seed ^ mix64((uint64_t)a.step));
  return (int64_t)fast_mod(mix64(k ^ (uint64_t)b), a.fm_n);
}

template <int DMAX>
__global__ void __launch_bounds__(128, 1) mlp_train_fwd(FwdArgs a) {
  extern __shared__ float smem_w[];
  stage_weights<DMAX>(a.P, a.d, smem_w);
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (b < a.ws.B) {
    const int64_t i = batch_row(a, b);
    const float z = forward_point<DMAX>(smem_w, a.x + i * a.d, a.d, a.ws.u + (int64_t)b * a.d,
                                        a.ws.a1 + (int64_t)b * kH, a.ws.a2 + (int64_t)b * kH);
    const float y = a.y[i] ? 1.f : 0.f;
    const float sig = 1.f / (1.f + expf(-z));
    a.ws.dz[b] = (sig - y) / (float)a.ws.B;
    l = (double)(fmaxf(z, 0.f) - z * y + log1pf(expf(-fabsf(z))));
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) l += __shfl_xor_sync(kFullMask, l, o);
  if ((threadIdx.x & 31) == 0 && a.ws.loss) atomicAdd(a.ws.loss + a.loss_slot, l);
}

// da2 = dz * w3 * gelu'(a2);  dh1 = W2^T da2;  da1 = dh1 * gelu'(a1)
constexpr size_t kBwdSmem = sizeof(float) * (kH * kH + kH);

__global__ void __launch_bounds__(128, 1) mlp_train_bwd(const float *P, int d, TrainWs ws) {
  extern __shared__ float smem_b[];
  float *w2t = smem_b;
  float *w3s = smem_b + kH * kH;
  const MlpOff o = mlp_off(d);
  for (int t = threadIdx.x; t < kH * kH; t += blockDim.x) {
    const int j = t / kH, tt = t % kH;
    w2t[t] = h16(P[o.w2 + (int64_t)tt * kH + j]);
  }
  for (int t = threadIdx.x; t < kH; t += blockDim.x) w3s[t] = h16(P[o.w3 + t]);
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= ws.B) return;
  const float dz = ws.dz[b];
  float da2[kH];
  const float *a2 = ws.a2 + (int64_t)b * kH;
#pragma unroll
  for (int t = 0; t < kH; ++t) {
    da2[t] = dz * w3s[t] * gelu_grad_f(a2[t]);
    ws.da2[(int64_t)b * kH + t] = da2[t];
  }
#pragma unroll 1
  for (int j = 0; j < kH; ++j) {
    const float *wr = w2t + j * kH;
    float s = 0.f;
#pragma unroll
    for (int t = 0; t < kH; ++t) s = fmaf(wr[t], da2[t], s);
    ws.da1[(int64_t)b * kH + j] = s * gelu_grad_f(ws.a1[(int64_t)b * kH + j]);
  }
}

// out[m][c] += sum_b A[b][m] * f(Bm[b][c]) over a slice of the batch
// (A: B x M, Bm: B x N, both row-major; f = identity or gelu).  32x32 output
// tile per block, 8 x 32 threads, batch staged through shared memory.
__global__ void __launch_bounds__(256) outer_sum_kernel(const float *A, int lda, int M,
                                                        const float *Bm, int ldb, int N,
                                                        int apply_gelu, int B, int chunk,
                                                        float *out, int ldo) {
  __shared__ float As[32][33];
  __shared__ float Bs[32][33];
  const int m0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int b_begin = blockIdx.z * chunk, b_end = min(B, b_begin + chunk);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // ty 0..7
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int b0 = b_begin; b0 < b_end; b0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const int b = b0 + r;
      As[r][tx] = (b < b_end && m0 + tx < M) ? A[(int64_t)b * lda + m0 + tx] : 0.f;
      float v = (b < b_end && c0 + tx < N) ? Bm[(int64_t)b * ldb + c0 + tx] : 0.f;
      Bs[r][tx] = apply_gelu ? gelu_f(v) : v;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
      const float bv = Bs[r][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(As[r][ty + 8 * q], bv, acc[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int mm = m0 + ty + 8 * q, cc = c0 + tx;
    if (mm < M && cc < N) atomicAdd(out + (int64_t)mm * ldo + cc, acc[q]);
  }
}

// out[c] += sum_b f(Bm[b][c]) * (A ? A[b] : 1)
__global__ void col_sum_kernel(const float *Bm, int ldb, int N, const float *A, int B,
                               float *out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += Bm[(int64_t)b * ldb + c] * (A ? A[b] : 1.f);
  atomicAdd(out + c, s);
}

__global__ void adam_kernel(float *P, const float *g, float *m, float *v, int64_t count,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// column mean / std of x (n x d) in FP64 partial sums
__global__ void col_moments_kernel(const float *x, int64_t n, int d, double *acc) {
  const int k = threadIdx.x;
  if (k >= d) return;
  double s = 0.0, s2 = 0.0;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const double v = x[i * d + k];
    s += v;
    s2 += v * v;
  }
  atomicAdd(acc + k, s);
  atomicAdd(acc + d + k, s2);
}

__global__ void col_finish_kernel(const double *acc, int64_t n, int d, float *mean, float *stdv) {
  const int k = threadIdx.x;
  if (k >= d) return;
  const double mu = acc[k] / (double)n;
  double var = acc[d + k] / (double)n - mu * mu;
  if (var < 0) var = 0;
  double sd = sqrt(var);
  if (!(sd > 1e-12)) sd = 1.0;
  mean[k] = (float)mu;
  stdv[k] = (float)sd;
}

// ------------------------------------------ inference on tcgen05 tensor cores
//
// The same two dense layers with the fifth-generation tensor-core
// instructions: a CTA of 8 warps pushes 128 points at a time through the
// network.  One thread issues tcgen05.mma (M = 128 points, N = 128 hidden
// units, K = 16 per instruction, FP16 operands from shared memory, FP32
// accumulators in tensor memory); the layer-1 accumulators are read back with
// tcgen05.ld (warps w and w + 4 own TMEM lanes 32 (w % 4) .. + 31, i.e. those
// points, and split the columns), take bias + GELU,
// are rounded to FP16 and written to shared memory as layer 2's A operand;
// layer 2's accumulators take bias + GELU and the output unit in registers.
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// the matrix is tiled by "core matrices" of 8 rows x 8 FP16 values (16
// bytes per row, 128 bytes each), stored [row group][k group][8 rows][16 B],
// so the descriptor's leading byte offset (between core matrices adjacent
// along K) is 128 and its stride byte offset (between 8-row groups) is
// (K / 8) * 128.  A k-step of 16 values advances the start address by two
// core matrices (256 bytes).
//
// Instruction descriptor (kind::f16): D format F32 (bit 4), A and B FP16
// (format 0, K-major), N >> 3 in bits 17-22, M >> 4 in bits 24-28.  Shared
// memory descriptor: start address >> 4 in bits 0-13, leading byte offset >>
// 4 in bits 16-29, stride byte offset >> 4 in bits 32-45, version 1 in bits
// 46-47, no swizzle (bits 61-63 zero).
//
// Every wait is bounded: a tensor-core completion that does not arrive in
// time sets an error bit in counters[3] (the caller reports it), and the
// kernel still frees its tensor memory before returning.

constexpr int kTcM = 128;            // points per tile
constexpr int kTcCols = 256;         // TMEM columns: layer 1 [0, 128), layer 2 [128, 256)
constexpr uint32_t kTcIdesc = (1u << 4) | ((uint32_t)(kH >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
constexpr uint32_t kTcWaitLimit = 1u << 26;

template <int KT1>
struct TcSmem {
  static constexpr int k1 = 16 * KT1;
  static constexpr size_t xa = 0;                                  // half [128][k1]
  static constexpr size_t w1 = xa + 2 * kTcM * k1;                 // half [128][k1]
  static constexpr size_t h1 = w1 + 2 * kH * k1;                   // half [128][128]
  static constexpr size_t w2 = h1 + 2 * kTcM * kH;                 // half [128][128]
  static constexpr size_t fp = w2 + 2 * kH * kH;                   // float params
  static constexpr size_t fp_count = 3 * kH + 4 + 2 * k1;          // b1 b2 w3 b3 pad mean istd
  static constexpr size_t zp = (fp + 4 * fp_count + 15) / 16 * 16;   // float [128] partial sums
  static constexpr size_t bar = zp + 4 * kTcM;                     // mbarrier (8 B)
  static constexpr size_t taddr = bar + 8;                         // TMEM base (4 B)
  static constexpr size_t bytes = taddr + 8 + 1024;                // + alignment slack
};

// Byte offset of element (r, k) in the canonical K-major no-swizzle layout of
// a matrix with K columns.
__device__ __forceinline__ uint32_t kmajor_off(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// Waits for the barrier's phase `parity` to complete; false after the bound.
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < kTcWaitLimit; ++it) {
    uint32_t done = 0;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (one lane each).
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

template <int KT1>
__global__ void __launch_bounds__(256, 2) mlp_gate_tc05_kernel(GateArgs a) {
  using L = TcSmem<KT1>;
  constexpr int K1 = L::k1;
  extern __shared__ unsigned char smem_dyn[];
  // 1024-byte aligned base for the operand tiles
  unsigned char *sm = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  float *fp = reinterpret_cast<float *>(sm + L::fp);
  float *b1s = fp, *b2s = fp + kH, *w3s = fp + 2 * kH, *b3s = fp + 3 * kH;
  float *means = fp + 3 * kH + 4, *istd = means + K1;
  const uint32_t bar = smem_u32(sm + L::bar);
  uint32_t *taddr_slot = reinterpret_cast<uint32_t *>(sm + L::taddr);
  const int d = a.d;
  const MlpOff o = mlp_off(d);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // weights, FP16-rounded, in the canonical layout (B operands: rows = units)
  for (int t = threadIdx.x; t < kH * K1; t += blockDim.x) {
    const int j = t / K1, k = t % K1;
    const float w = k < d ? a.P[o.w1 + (int64_t)j * d + k] : 0.f;
    *reinterpret_cast<__half *>(sm + L::w1 + kmajor_off(j, k, K1)) = __float2half_rn(w);
  }
  for (int t = threadIdx.x; t < kH * kH; t += blockDim.x) {
    const int j = t / kH, k = t % kH;
    *reinterpret_cast<__half *>(sm + L::w2 + kmajor_off(j, k, kH)) =
        __float2half_rn(a.P[o.w2 + (int64_t)j * kH + k]);
  }
  for (int t = threadIdx.x; t < kH; t += blockDim.x) {
    b1s[t] = h16(a.P[o.b1 + t]);
    b2s[t] = h16(a.P[o.b2 + t]);
    w3s[t] = h16(a.P[o.w3 + t]);
  }
  for (int k = threadIdx.x; k < K1; k += blockDim.x) {
    means[k] = k < d ? a.P[o.mean + k] : 0.f;
    istd[k] = k < d ? 1.f / a.P[o.std + k] : 0.f;
  }
  if (threadIdx.x == 0) {
    b3s[0] = h16(a.P[o.b3]);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(taddr_slot)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *taddr_slot;
  // warps w and w + 4 share TMEM lanes 32 (w % 4) .. + 31 (points) and split
  // the 128 columns of each layer between them
  const int quarter = warp & 3, half = warp >> 2;
  const uint32_t t_lanes = (uint32_t)(quarter * 32) << 16;
  float *zpart = reinterpret_cast<float *>(sm + L::zp);
  const uint32_t sx = smem_u32(sm + L::xa), sw1 = smem_u32(sm + L::w1);
  const uint32_t sh1 = smem_u32(sm + L::h1), sw2 = smem_u32(sm + L::w2);
  uint32_t parity = 0;
  bool ok = true;
  unsigned long long nq = 0, nc = 0, nn = 0;

  for (int64_t base = (int64_t)blockIdx.x * kTcM; base < a.n && ok; base += (int64_t)gridDim.x * kTcM) {
    // standardised inputs of 128 points, FP16 (zero past n and past d)
    for (int t = threadIdx.x; t < kTcM * K1; t += blockDim.x) {
      const int r = t / K1, k = t % K1;
      const int64_t i = base + r;
      const float v = (i < a.n && k < d) ? (a.x[i * a.ld + k] - means[k]) * istd[k] : 0.f;
      *reinterpret_cast<__half *>(sm + L::xa + kmajor_off(r, k, K1)) = __float2half_rn(v);
    }
    // make the generic-proxy writes visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x == 0) {
#pragma unroll
      for (int ks = 0; ks < KT1; ++ks)
        tc_mma(tbase, smem_desc(sx + 256 * ks, 128, (K1 / 8) * 128),
               smem_desc(sw1 + 256 * ks, 128, (K1 / 8) * 128), ks > 0);
      tc_commit(bar);
    }
    ok = __syncthreads_and(tc_wait(bar, parity) ? 1 : 0) != 0;   // uniform in the block
    parity ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      // layer 1: bias + GELU -> FP16 hidden activations (A operand of layer 2)
      const int r = quarter * 32 + lane;
#pragma unroll 1
      for (int c = 2 * half; c < 2 * half + 2; ++c) {
        float v[32];
        tc_ld32(tbase + t_lanes + (uint32_t)(32 * c), v);
#pragma unroll
        for (int g8 = 0; g8 < 4; ++g8) {
          __align__(16) __half hv[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int col = 32 * c + 8 * g8 + e;
            hv[e] = __float2half_rn(gelu_f(v[8 * g8 + e] + b1s[col]));
          }
          *reinterpret_cast<uint4 *>(sm + L::h1 + kmajor_off(r, 32 * c + 8 * g8, kH)) =
              *reinterpret_cast<const uint4 *>(hv);
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ok = __syncthreads_and(ok ? 1 : 0) != 0;   // every thread takes the same branch
    if (!ok) break;
    if (threadIdx.x == 0) {
#pragma unroll
      for (int ks = 0; ks < kH / 16; ++ks)
        tc_mma(tbase + kH, smem_desc(sh1 + 256 * ks, 128, (kH / 8) * 128),
               smem_desc(sw2 + 256 * ks, 128, (kH / 8) * 128), ks > 0);
      tc_commit(bar);
    }
    ok = __syncthreads_and(tc_wait(bar, parity) ? 1 : 0) != 0;
    parity ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float z = 0.f;
    if (ok) {
      // layer 2: bias + GELU, then the output unit (each half of the columns
      // in one warp; the two partial sums meet in shared memory)
#pragma unroll 1
      for (int c = 2 * half; c < 2 * half + 2; ++c) {
        float v[32];
        tc_ld32(tbase + t_lanes + (uint32_t)(kH + 32 * c), v);
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          const int col = 32 * c + e;
          z = fmaf(w3s[col], gelu_f(v[e] + b2s[col]), z);
        }
      }
      if (half == 1) zpart[quarter * 32 + lane] = z;
    }
    __syncthreads();
    if (ok && half == 0) {
      z += zpart[quarter * 32 + lane];
      const int64_t i = base + quarter * 32 + lane;
      if (i < a.n) {
        const float p = 1.f / (1.f + expf(-(z + b3s[0])));
        if (a.prob) a.prob[i] = p;
        if (a.forced) {
          uint8_t f = 0;
          int32_t mi = a.m, wi = a.w_full;
          if (p < a.p_noise) {
            f = 2;
            mi = a.m_noise;
            wi = a.w_noise;
            ++nn;
          } else if (p > a.p_core) {
            f = 1;
            mi = a.m_core;
            wi = a.w_core;
            ++nc;
          }
          a.forced[i] = a.by_degree ? 0 : f;
          a.m_row[i] = mi;
          if (a.w_row) a.w_row[i] = wi;
          nq += (unsigned long long)mi;
        }
      }
    }
    // the next tile overwrites the operands and the accumulators
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
  }
  if (a.counters) {
#pragma unroll
    for (int o2 = 16; o2 >= 1; o2 >>= 1) {
      nq += __shfl_xor_sync(kFullMask, nq, o2);
      nc += __shfl_xor_sync(kFullMask, nc, o2);
      nn += __shfl_xor_sync(kFullMask, nn, o2);
    }
    if (lane == 0) {
      atomicAdd(a.counters + 0, nq);
      atomicAdd(a.counters + 1, nc);
      atomicAdd(a.counters + 2, nn);
    }
    if (!ok && threadIdx.x == 0) atomicOr(a.counters + 3, 1ull);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kTcCols)
                 : "memory");
}

template <int KT1>
static cudaError_t launch_gate_tc05(const GateArgs &a, cudaStream_t st) {
  const size_t smem = TcSmem<KT1>::bytes;
  cudaError_t e = cudaFuncSetAttribute((const void *)mlp_gate_tc05_kernel<KT1>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // two CTAs per SM: each holds 256 of the SM's 512 TMEM columns (shared
  // memory, about 100 KB each, admits no third)
  const int64_t need = (a.n + kTcM - 1) / kTcM;
  const int grid = (int)std::min<int64_t>(need, 2 * (int64_t)device_sms());
  mlp_gate_tc05_kernel<KT1><<<grid, 256, smem, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------- dispatch

template <int DMAX>
static cudaError_t smem_optin(const void *fn) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Smem<DMAX>::bytes);
}

static int dmax_for(int d) { return d <= 8 ? 8 : d <= 32 ? 32 : 64; }

template <int KT1>
static cudaError_t launch_gate_mma(const GateArgs &a, cudaStream_t st) {
  const size_t smem = MmaSmem<KT1>::bytes(4);
  cudaError_t e = cudaFuncSetAttribute((const void *)mlp_gate_mma_kernel<KT1>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mlp_gate_mma_kernel<KT1>, 128, smem);
  const int64_t need = (a.n + 63) / 64;
  const int grid = (int)std::min<int64_t>(need, (int64_t)device_sms() * (occ > 0 ? occ : 1));
  mlp_gate_mma_kernel<KT1><<<grid, 128, smem, st>>>(a);
  note_launch();
  return cudaGetLastError();
}

static cudaError_t launch_gate_simt(const GateArgs &a, cudaStream_t st);

// Gate / prediction: tensor-core kernel (FP16 activations at the MMA inputs)
// unless FP32 activations are asked for.
static cudaError_t launch_gate(const GateArgs &a, cudaStream_t st) {
  if (a.fp32_activations == 1) return launch_gate_simt(a, st);
  if (a.fp32_activations == 2) {
    switch ((a.d + 15) / 16) {
      case 1: return launch_gate_tc05<1>(a, st);
      case 2: return launch_gate_tc05<2>(a, st);
      case 3: return launch_gate_tc05<3>(a, st);
      default: return launch_gate_tc05<4>(a, st);
    }
  }
  switch ((a.d + 15) / 16) {
    case 1: return launch_gate_mma<1>(a, st);
    case 2: return launch_gate_mma<2>(a, st);
    case 3: return launch_gate_mma<3>(a, st);
    default: return launch_gate_mma<4>(a, st);
  }
}

// FP32-activation reference path on CUDA cores (kept for checking).
static cudaError_t launch_gate_simt(const GateArgs &a, cudaStream_t st) {
  const int sms = device_sms();
  const int64_t need = (a.n + 127) / 128;
  const int grid = (int)std::min<int64_t>(need, (int64_t)sms * 2);
  switch (dmax_for(a.d)) {
    case 8:
      smem_optin<8>((const void *)mlp_gate_kernel<8>);
      mlp_gate_kernel<8><<<grid, 128, Smem<8>::bytes, st>>>(a);
      break;
    case 32:
      smem_optin<32>((const void *)mlp_gate_kernel<32>);
      mlp_gate_kernel<32><<<grid, 128, Smem<32>::bytes, st>>>(a);
      break;
    default:
      smem_optin<64>((const void *)mlp_gate_kernel<64>);
      mlp_gate_kernel<64><<<grid, 128, Smem<64>::bytes, st>>>(a);
      break;
  }
  note_launch();
  return cudaGetLastError();
}

static cudaError_t launch_train_fwd(const FwdArgs &a, cudaStream_t st) {
  const int grid = (a.ws.B + 127) / 128;
  switch (dmax_for(a.d)) {
    case 8:
      smem_optin<8>((const void *)mlp_train_fwd<8>);
      mlp_train_fwd<8><<<grid, 128, Smem<8>::bytes, st>>>(a);
      break;
    case 32:
      smem_optin<32>((const void *)mlp_train_fwd<32>);
      mlp_train_fwd<32><<<grid, 128, Smem<32>::bytes, st>>>(a);
      break;
    default:
      smem_optin<64>((const void *)mlp_train_fwd<64>);
      mlp_train_fwd<64><<<grid, 128, Smem<64>::bytes, st>>>(a);
      break;
  }
  note_launch();
  return cudaGetLastError();
}

// Gradient of the batch loss into ws.grad (zeroed here).
static cudaError_t launch_loss_grad(const FwdArgs &a, cudaStream_t st) {
  const MlpOff o = mlp_off(a.d);
  const TrainWs &w = a.ws;
  cudaMemsetAsync(w.grad, 0, sizeof(float) * o.train, st);
  cudaError_t e = launch_train_fwd(a, st);
  if (e != cudaSuccess) return e;
  cudaFuncSetAttribute((const void *)mlp_train_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)kBwdSmem);
  mlp_train_bwd<<<(w.B + 127) / 128, 128, kBwdSmem, st>>>(a.P, a.d, w);
  const int chunk = 256;
  const int splits = (w.B + chunk - 1) / chunk;
  // dW2[t][j] = sum_b da2[b][t] gelu(a1[b][j])
  outer_sum_kernel<<<dim3(kH / 32, kH / 32, splits), 256, 0, st>>>(
      w.da2, kH, kH, w.a1, kH, kH, 1, w.B, chunk, w.grad + o.w2, kH);
  // dW1[j][k] = sum_b da1[b][j] u[b][k]
  outer_sum_kernel<<<dim3(kH / 32, (a.d + 31) / 32, splits), 256, 0, st>>>(
      w.da1, kH, kH, w.u, a.d, a.d, 0, w.B, chunk, w.grad + o.w1, a.d);
  // dw3[t] = sum_b dz[b] gelu(a2[b][t])
  outer_sum_kernel<<<dim3(1, kH / 32, splits), 256, 0, st>>>(
      w.dz, 1, 1, w.a2, kH, kH, 1, w.B, chunk, w.grad + o.w3, kH);
  col_sum_kernel<<<1, kH, 0, st>>>(w.da1, kH, kH, nullptr, w.B, w.grad + o.b1);
  col_sum_kernel<<<1, kH, 0, st>>>(w.da2, kH, kH, nullptr, w.B, w.grad + o.b2);
  col_sum_kernel<<<1, 32, 0, st>>>(w.dz, 1, 1, nullptr, w.B, w.grad + o.b3);
  note_launch(7);
  return cudaGetLastError();
}

static sng_status alloc_ws(Scratch &s, int B, int d, int steps, TrainWs *w) {
  const MlpOff o = mlp_off(d);
  sng_status rc;
  w->B = B;
  if ((rc = s.alloc((void **)&w->u, sizeof(float) * B * d, "mlp u")) ||
      (rc = s.alloc((void **)&w->a1, sizeof(float) * B * kH, "mlp a1")) ||
      (rc = s.alloc((void **)&w->a2, sizeof(float) * B * kH, "mlp a2")) ||
      (rc = s.alloc((void **)&w->dz, sizeof(float) * B, "mlp dz")) ||
      (rc = s.alloc((void **)&w->da1, sizeof(float) * B * kH, "mlp da1")) ||
      (rc = s.alloc((void **)&w->da2, sizeof(float) * B * kH, "mlp da2")) ||
      (rc = s.alloc((void **)&w->grad, sizeof(float) * o.train, "mlp grad")) ||
      (rc = s.alloc((void **)&w->loss, sizeof(double) * (steps > 0 ? steps : 1), "mlp loss")))
    return rc;
  cudaMemsetAsync(w->loss, 0, sizeof(double) * (steps > 0 ? steps : 1), s.stream);
  return SNG_OK;
}

static sng_status check_cfg(const sng_mlp_config *c) {
  if (!c) return fail(SNG_EINVAL, "mlp config is NULL");
  if (c->d < 1 || c->d > 64) return fail(SNG_EINVAL, "mlp d must be in [1, 64]");
  if (c->hidden != kH) return fail(SNG_EINVAL, "mlp hidden width must be %d", kH);
  if (c->fp32_activations < 0 || c->fp32_activations > 2)
    return fail(SNG_EINVAL, "fp32_activations must be 0, 1 or 2");
  return SNG_OK;
}

__global__ void loss_to_float(const double *l, int steps, int B, float *out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < steps) out[s] = (float)(l[s] / (double)B);
}

}  // namespace sng

using namespace sng;

extern "C" {

int64_t sng_mlp_param_count(int32_t d, int32_t hidden) {
  if (d < 1 || d > 64 || hidden != kH) return -1;
  return mlp_off(d).total;
}

sng_status sng_mlp_standardize(const float *x, int64_t n, int32_t d, float *params,
                               void *stream) {
  if (!x || !params) return fail(SNG_EINVAL, "NULL argument");
  if (n < 1 || d < 1 || d > 64) return fail(SNG_EINVAL, "bad n or d");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch s(st);
  double *acc;
  sng_status rc = s.alloc((void **)&acc, sizeof(double) * 2 * d, "moments");
  if (rc) return rc;
  cudaMemsetAsync(acc, 0, sizeof(double) * 2 * d, st);
  const MlpOff o = mlp_off(d);
  col_moments_kernel<<<device_sms() * 4, 64, 0, st>>>(x, n, d, acc);
  col_finish_kernel<<<1, 64, 0, st>>>(acc, n, d, params + o.mean, params + o.std);
  note_launch(2);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SNG_OK : cuda_fail(e, "standardize");
}

sng_status sng_mlp_loss_grad(const float *x, const uint8_t *y, int64_t n,
                             const sng_mlp_config *cfg, const float *params, float *grad,
                             double *loss, void *stream) {
  sng_status rc = check_cfg(cfg);
  if (rc) return rc;
  if (!x || !y || !params || !grad) return fail(SNG_EINVAL, "NULL argument");
  if (n < 1 || n > (1 << 24)) return fail(SNG_EINVAL, "n must be in [1, 2^24]");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch s(st);
  TrainWs w;
  if ((rc = alloc_ws(s, (int)n, cfg->d, 1, &w))) return rc;
  FwdArgs a{x, y, n, cfg->d, params, w, 0, 0, 0, make_fastmod(n + 1), 0};
  cudaError_t e = launch_loss_grad(a, st);
  if (e != cudaSuccess) return cuda_fail(e, "loss_grad");
  const MlpOff o = mlp_off(cfg->d);
  cudaMemcpyAsync(grad, w.grad, sizeof(float) * o.train, cudaMemcpyDeviceToDevice, st);
  double l = 0;
  e = cudaMemcpyAsync(&l, w.loss, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "loss_grad read-back");
  if (loss) *loss = l / (double)n;
  return SNG_OK;
}

sng_status sng_mlp_train(const float *x, const uint8_t *y, int64_t n, const sng_mlp_config *cfg,
                         float *params, float *adam_m, float *adam_v, int64_t step0,
                         int64_t steps, float *loss_trace, void *stream) {
  NvtxRange nvtx_range("sng_mlp_train");
  sng_status rc = check_cfg(cfg);
  if (rc) return rc;
  if (!x || !y || !params || !adam_m || !adam_v) return fail(SNG_EINVAL, "NULL argument");
  if (n < 1 || n > 0x7fffffffLL) return fail(SNG_EINVAL, "n out of range");
  if (cfg->batch < 1 || cfg->batch > (1 << 20)) return fail(SNG_EINVAL, "bad batch size");
  if (steps < 0 || steps > (1 << 24) || step0 < 0) return fail(SNG_EINVAL, "bad step range");
  if (!(cfg->lr > 0.f) || !(cfg->beta1 >= 0.f && cfg->beta1 < 1.f) ||
      !(cfg->beta2 >= 0.f && cfg->beta2 < 1.f) || !(cfg->adam_eps > 0.f))
    return fail(SNG_EINVAL, "bad optimiser settings");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch s(st);
  TrainWs w;
  if ((rc = alloc_ws(s, cfg->batch, cfg->d, (int)steps, &w))) return rc;
  const MlpOff o = mlp_off(cfg->d);
  const FastMod fm = make_fastmod(n + 1);  // divisor n
  for (int64_t k = 0; k < steps; ++k) {
    const int64_t t = step0 + k + 1;  // Adam step count
    FwdArgs a{x, y, n, cfg->d, params, w, cfg->sequential ? 2 : 1, cfg->seed, step0 + k, fm,
              (int32_t)k};
    cudaError_t e = launch_loss_grad(a, st);
    if (e != cudaSuccess) return cuda_fail(e, "train step");
    const float c1 = (float)(1.0 - std::pow((double)cfg->beta1, (double)t));
    const float c2 = (float)(1.0 - std::pow((double)cfg->beta2, (double)t));
    adam_kernel<<<64, 256, 0, st>>>(params, w.grad, adam_m, adam_v, o.train, cfg->lr,
                                    cfg->beta1, cfg->beta2, cfg->adam_eps, c1, c2);
    note_launch();
  }
  if (loss_trace && steps > 0) {
    loss_to_float<<<(int)((steps + 255) / 256), 256, 0, st>>>(w.loss, (int)steps, cfg->batch,
                                                                loss_trace);
    note_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "train");
  return SNG_OK;
}

sng_status sng_mlp_predict(const float *x, int64_t n, const sng_mlp_config *cfg,
                           const float *params, float *prob, void *stream) {
  NvtxRange nvtx_range("sng_mlp_predict");
  sng_status rc = check_cfg(cfg);
  if (rc) return rc;
  if (!x || !params || !prob) return fail(SNG_EINVAL, "NULL argument");
  if (n < 1) return fail(SNG_EINVAL, "n must be >= 1");
  GateArgs a{cfg->fp32_activations,
             x,
             cfg->d,
             n,
             cfg->d,
             params,
             prob,
             0.f,
             1.f,
             0,
             0,
             0,
             1,
             1,
             1,
             nullptr,
             0,
             nullptr,
             nullptr,
             nullptr};
  cudaError_t e = launch_gate(a, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? SNG_OK : cuda_fail(e, "predict");
}

sng_status sng_cluster_surrogate(const void *x, const sng_params *params,
                                 const sng_mlp_config *cfg, const float *mlp_params,
                                 const sng_gate *gate, int32_t *labels, uint8_t *core,
                                 sng_stats *stats, void *stream) {
  NvtxRange nvtx_range("sng_cluster_surrogate");
  Resolved r;
  sng_status rc = validate(x, params, &r);
  if (rc) return rc;
  if ((rc = check_cfg(cfg))) return rc;
  if (!labels || !mlp_params || !gate) return fail(SNG_EINVAL, "NULL argument");
  if (params->dtype != SNG_F32) return fail(SNG_EINVAL, "surrogate form takes FP32 points");
  if (r.row_begin != 0 || r.row_end != r.n)
    return fail(SNG_EINVAL, "a source-row range is for sng_build_graph only");
  if (params->sample_mode != SNG_SAMPLE_HASH)
    return fail(SNG_EINVAL, "surrogate form needs hashed draws");
  if (cfg->d != params->d) return fail(SNG_EINVAL, "mlp d differs from the points' d");
  const float pn = gate->p_noise, pc = gate->p_core;
  if (!(pn >= 0.f && pn <= pc && pc <= 1.f))
    return fail(SNG_EINVAL, "need 0 <= p_noise <= p_core <= 1");
  if (!(gate->core_draw_frac > 0.f && gate->core_draw_frac <= 1.f))
    return fail(SNG_EINVAL, "core_draw_frac must be in (0, 1]");
  if (!(gate->noise_draw_frac >= 0.f && gate->noise_draw_frac <= 1.f))
    return fail(SNG_EINVAL, "noise_draw_frac must be in [0, 1]");
  if (gate->reweight != 0 && gate->reweight != 1) return fail(SNG_EINVAL, "reweight is 0 or 1");
  if (gate->by_degree != 0 && gate->by_degree != 1) return fail(SNG_EINVAL, "by_degree is 0 or 1");
  if (params->flags & SNG_FLAG_NO_SYNC)
    return fail(SNG_EINVAL, "SNG_FLAG_NO_SYNC is for sng_cluster only");
  if (params->metric != SNG_METRIC_L2)
    return fail(SNG_EINVAL, "the surrogate form uses the Euclidean ball (metric 0)");
  if (gate->reweight && params->degree_mode == SNG_DEG_SIMPLE)
    return fail(SNG_EINVAL, "reweighted degrees are multigraph counts; not with simple-graph degree");
  device_sms();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scratch s(st);
  Timer tm((params->flags & SNG_FLAG_TIMING) != 0);
  uint8_t *forced;
  int32_t *m_row, *w_row = nullptr;
  unsigned long long *gcnt;
  if ((rc = s.alloc((void **)&forced, (size_t)r.n, "forced")) ||
      (rc = s.alloc((void **)&m_row, (size_t)r.n * 4, "draws per row")) ||
      (rc = s.alloc((void **)&gcnt, 4 * 8, "gate counters")))
    return rc;
  if (gate->reweight && (rc = s.alloc((void **)&w_row, (size_t)r.n * 4, "degree weights")))
    return rc;
  cudaMemsetAsync(gcnt, 0, 4 * 8, st);
  const int32_t m_core = (int32_t)std::ceil((double)gate->core_draw_frac * (double)r.m);
  const int32_t m_noise = (int32_t)std::ceil((double)gate->noise_draw_frac * (double)r.m);
  // reweighting: a kept draw of a point that drew m_i of m partners counts
  // m / m_i (in units of 1/16), an unbiased estimate of its plain count
  const int32_t unit = gate->reweight ? kDegUnit : 1;
  auto weight = [&](int32_t mi) {
    if (!gate->reweight) return 1;
    if (mi <= 0) return kDegUnit;
    return (int32_t)std::lround((double)kDegUnit * (double)r.m / (double)mi);
  };
  GateArgs ga{cfg->fp32_activations,
              static_cast<const float *>(x),
              params->ld,
              r.n,
              params->d,
              mlp_params,
              nullptr,
              pn,
              pc,
              (int32_t)r.m,
              m_core,
              m_noise,
              weight((int32_t)r.m),
              weight(m_core),
              weight(m_noise),
              forced,
              gate->by_degree,
              m_row,
              w_row,
              gcnt};
  tm.mark(st, 9);
  cudaError_t e = launch_gate(ga, st);
  if (e != cudaSuccess) return cuda_fail(e, "surrogate gate");
  GraphBufs gb;
  gb.want_src = true;
  if ((rc = run_graph(x, params, r, s, &gb, m_row, &tm, w_row))) return rc;
  uint8_t *core_buf = core;
  int32_t *parent = nullptr;
  if (!core_buf && (rc = s.alloc((void **)&core_buf, (size_t)r.n, "core"))) return rc;
  if ((rc = s.alloc((void **)&parent, (size_t)r.n * 4, "parent"))) return rc;
  const int sms = device_sms();
  CoreArgs ca{r.n, params->min_pts * unit, gb.deg, forced, core_buf, parent, labels};
  launch_core_init(ca, sms, st);
  tm.mark(st, 4);
  UnionArgs ua{r.n,      gb.row_ptr, gb.col,      gb.src,      gb.num_edges,
               core_buf, parent,     labels,      gb.counters, loop_limit()};
  launch_union(ua, sms, st);
  tm.mark(st, 5);
  launch_label(ua, sms, st);
  tm.mark(st, 6);
  FinalizeArgs fa{r.n, core_buf, gb.band_flag, labels, gb.counters, parent, loop_limit()};
  launch_finalize(fa, sms, st);
  tm.mark(st, 7);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "surrogate cluster launches");
  rc = read_stats(gb.counters, r, stats, st, &tm);
  note_mapping(gb, stats);
  if (stats && rc == SNG_OK) {
    unsigned long long g[4];
    e = cudaMemcpyAsync(g, gcnt, sizeof(g), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "gate counters");
    stats->queries = (int64_t)g[0];
    stats->surrogate_core = (int64_t)g[1];
    stats->surrogate_noise = (int64_t)g[2];
  }
  s.release();
  return rc;
}

}  // extern "C"
