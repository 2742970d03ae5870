// The learned initial guess (the paper has no counterpart): a four-layer 3x3 convolutional
// network on the tensor cores (BF16 operands staged in shared memory, fed to mma.sync
// m16n8k16 by ldmatrix, FP32 accumulation), its training (MSE loss, backward pass, AdamW on
// FP32 master weights), and the kernels that turn solver fields into network features and the
// network's output back into a solver state (the 13-moment Grad state).
#include "nrmg.h"
#include "nrmg_internal.h"
#include "nrmg_net.h"

#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

using namespace nrmg;

namespace {

constexpr int kLayers = 4;
constexpr int kTaps = 9;
typedef __nv_bfloat16 bf16;

// ------------------------------------------------------------------ tensor-core helpers
__device__ __forceinline__ uint32_t sm_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Four 8x8 b16 matrices; lane l gives the row address of row (l & 7) of matrix (l >> 3).
__device__ __forceinline__ void ldsm4(uint32_t a, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldsm4t(uint32_t a, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
// d += A B with A 16x16 (row-major fragment), B 16x8 (column-major fragment), BF16 inputs.
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}

// ------------------------------------------------------------------ convolution
// out[p][co] = sum_{t, ci} in[p + off_t][ci] W[t][co][ci]: an implicit GEMM with the pixels
// as rows, the 9*CI (tap, channel) pairs as the reduction and CO as columns.  A CTA owns an
// 8 x 32 output tile (one image row of 32 pixels per warp, as two 16-pixel MMA row blocks that
// share every weight fragment), keeps all 9 taps of the layer's weights in shared memory and
// walks the tiles persistently.  Shared-memory rows are padded by 8 elements so that the
// eight rows one ldmatrix phase reads fall in distinct bank groups.
enum ConvMode { kRelu = 0, kLinear = 1, kMask = 2 };
constexpr int kTH = 8, kTW = 32, kConvThreads = 256;

template <int CI, int CO>
struct ConvSmem {
  static constexpr int RS = CI + 8;
  static constexpr int kW = kTaps * CO * RS;
  static constexpr int kIn = (kTH + 2) * (kTW + 2) * RS;
  static constexpr size_t bytes = (size_t)(kW + kIn) * sizeof(bf16) + CO * sizeof(float);
};

// MODE kRelu: out16 = bf16(relu(conv + bias)); kLinear: out32 = conv + bias (FP32);
// kMask: out16 = bf16(conv * [mask > 0]) (the backward pass through a ReLU).
template <int CI, int CO, int MODE>
__global__ void __launch_bounds__(kConvThreads, 1)
    conv3x3_kernel(const bf16 *__restrict__ in, const bf16 *__restrict__ wt, const float *__restrict__ bias,
                   const bf16 *__restrict__ mask, int B, int H, int W, bf16 *__restrict__ out16,
                   float *__restrict__ out32) {
  using S = ConvSmem<CI, CO>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bf16 *sw = reinterpret_cast<bf16 *>(smem_raw);
  bf16 *sin = sw + S::kW;
  float *sb = reinterpret_cast<float *>(sin + S::kIn);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int q = tid; q < kTaps * CO * (CI / 8); q += kConvThreads) {
    const int row = q / (CI / 8), c8 = q - row * (CI / 8);
    *reinterpret_cast<uint4 *>(sw + row * S::RS + c8 * 8) =
        *reinterpret_cast<const uint4 *>(wt + (size_t)row * CI + c8 * 8);
  }
  if (tid < CO) sb[tid] = bias ? bias[tid] : 0.f;
  const int tiles_w = (W + kTW - 1) / kTW, tiles_h = (H + kTH - 1) / kTH;
  const long long ntiles = (long long)B * tiles_h * tiles_w;
  const uint32_t in_base = sm_addr(sin), w_base = sm_addr(sw);
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int tw = (int)(tile % tiles_w);
    const long long rest = tile / tiles_w;
    const int th = (int)(rest % tiles_h), b = (int)(rest / tiles_h);
    const int h0 = th * kTH, w0 = tw * kTW;
    __syncthreads();  // the previous tile's fragments are read (and the weights stored)
    for (int q = tid; q < (kTH + 2) * (kTW + 2) * (CI / 8); q += kConvThreads) {
      const int pix = q / (CI / 8), c8 = q - pix * (CI / 8);
      const int hh = pix / (kTW + 2), ww = pix - hh * (kTW + 2);
      const int h = h0 - 1 + hh, w = w0 - 1 + ww;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (h >= 0 && h < H && w >= 0 && w < W)
        v = *reinterpret_cast<const uint4 *>(in + (((size_t)b * H + h) * W + w) * CI + c8 * 8);
      *reinterpret_cast<uint4 *>(sin + pix * S::RS + c8 * 8) = v;
    }
    __syncthreads();
    const int h = h0 + warp;
    if (h >= H) continue;
    float acc[2][CO / 8][4];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int n = 0; n < CO / 8; ++n)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[s][n][k] = 0.f;
#pragma unroll 1
    for (int t = 0; t < kTaps; ++t) {
      const int dy = t / 3 - 1, dx = t % 3 - 1;
      uint32_t a_addr[2];
#pragma unroll
      for (int s = 0; s < 2; ++s)
        a_addr[s] = in_base +
                    (((warp + 1 + dy) * (kTW + 2) + (16 * s + (lane & 15) + 1 + dx)) * S::RS + (lane >> 4) * 8) *
                        (uint32_t)sizeof(bf16);
      const uint32_t b_addr =
          w_base + ((t * CO + (lane >> 4) * 8 + (lane & 7)) * S::RS + ((lane >> 3) & 1) * 8) * (uint32_t)sizeof(bf16);
#pragma unroll
      for (int kc = 0; kc < CI / 16; ++kc) {
        uint32_t a0[4], a1[4];
        ldsm4(a_addr[0] + kc * 32, a0);
        ldsm4(a_addr[1] + kc * 32, a1);
#pragma unroll
        for (int np = 0; np < CO / 16; ++np) {
          uint32_t bf[4];
          ldsm4(b_addr + (np * 16 * S::RS + kc * 16) * (uint32_t)sizeof(bf16), bf);
          mma16816(acc[0][2 * np], a0, bf[0], bf[1]);
          mma16816(acc[0][2 * np + 1], a0, bf[2], bf[3]);
          mma16816(acc[1][2 * np], a1, bf[0], bf[1]);
          mma16816(acc[1][2 * np + 1], a1, bf[2], bf[3]);
        }
      }
    }
    const int g = lane >> 2, tg = lane & 3;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int w = w0 + 16 * s + g + 8 * half;
        if (w >= W) continue;
        const size_t pix = ((size_t)b * H + h) * W + w;
#pragma unroll
        for (int n = 0; n < CO / 8; ++n) {
          const int co = n * 8 + 2 * tg;
          float v0 = acc[s][n][2 * half], v1 = acc[s][n][2 * half + 1];
          if (MODE == kRelu) {
            v0 = fmaxf(v0 + sb[co], 0.f);
            v1 = fmaxf(v1 + sb[co + 1], 0.f);
            *reinterpret_cast<uint32_t *>(out16 + pix * CO + co) = pack_bf16(v0, v1);
          } else if (MODE == kLinear) {
            *reinterpret_cast<float2 *>(out32 + pix * CO + co) = make_float2(v0 + sb[co], v1 + sb[co + 1]);
          } else {
            const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162 *>(mask + pix * CO + co);
            if (!(__bfloat162float(m.x) > 0.f)) v0 = 0.f;
            if (!(__bfloat162float(m.y) > 0.f)) v1 = 0.f;
            *reinterpret_cast<uint32_t *>(out16 + pix * CO + co) = pack_bf16(v0, v1);
          }
        }
      }
  }
}

// ------------------------------------------------------------------ weight gradient
// dW[t][co][ci] = sum_p G[p][co] a[p + off_t][ci] and db[co] = sum_p G[p][co]: a GEMM whose
// reduction runs over the pixels.  A CTA owns a 4 x 32 pixel tile at a time (persistent);
// each of its 16 warps owns one 16 (co) x 16 (ci) block for a subset of the taps, reads G^T
// and the shifted activations with transposing ldmatrix, and keeps its accumulators in
// registers across tiles.  Every CTA writes its own partial sums; a second kernel adds them in
// a fixed order, so the gradient is deterministic.
constexpr int kGH = 4, kGW = 32, kGradThreads = 512, kMaxGradCTAs = 320;

template <int CI, int CO>
struct GradSmem {
  static constexpr int RA = CI + 8, RG = CO + 8;
  static constexpr int kA = (kGH + 2) * (kGW + 2) * RA;
  static constexpr int kG = kGH * kGW * RG;
  static constexpr size_t bytes = (size_t)(kA + kG) * sizeof(bf16);
  static constexpr int kPairs = (CO / 16) * (CI / 16);
  static constexpr int kTG = (kGradThreads / 32) / kPairs;
  static constexpr int kTPW = (kTaps + kTG - 1) / kTG;
  static_assert((kGradThreads / 32) % kPairs == 0, "warps must tile the (co, ci) blocks");
};

template <int CI, int CO>
__global__ void __launch_bounds__(kGradThreads, 1)
    wgrad_kernel(const bf16 *__restrict__ a, const bf16 *__restrict__ G, int B, int H, int W,
                 float *__restrict__ partials) {
  using S = GradSmem<CI, CO>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bf16 *sa = reinterpret_cast<bf16 *>(smem_raw);
  bf16 *sg = sa + S::kA;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int pair = warp % S::kPairs, tgrp = warp / S::kPairs;
  const int mt = pair / (CI / 16), np = pair % (CI / 16);
  float acc[S::kTPW][2][4];
#pragma unroll
  for (int j = 0; j < S::kTPW; ++j)
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[j][n][k] = 0.f;
  float bsum = 0.f;
  const int tiles_w = (W + kGW - 1) / kGW, tiles_h = (H + kGH - 1) / kGH;
  const long long ntiles = (long long)B * tiles_h * tiles_w;
  const uint32_t a_base = sm_addr(sa), g_base = sm_addr(sg);
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int tw = (int)(tile % tiles_w);
    const long long rest = tile / tiles_w;
    const int th = (int)(rest % tiles_h), b = (int)(rest / tiles_h);
    const int h0 = th * kGH, w0 = tw * kGW;
    __syncthreads();
    for (int q = tid; q < (kGH + 2) * (kGW + 2) * (CI / 8); q += kGradThreads) {
      const int pix = q / (CI / 8), c8 = q - pix * (CI / 8);
      const int hh = pix / (kGW + 2), ww = pix - hh * (kGW + 2);
      const int h = h0 - 1 + hh, w = w0 - 1 + ww;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (h >= 0 && h < H && w >= 0 && w < W)
        v = *reinterpret_cast<const uint4 *>(a + (((size_t)b * H + h) * W + w) * CI + c8 * 8);
      *reinterpret_cast<uint4 *>(sa + pix * S::RA + c8 * 8) = v;
    }
    for (int q = tid; q < kGH * kGW * (CO / 8); q += kGradThreads) {
      const int pix = q / (CO / 8), c8 = q - pix * (CO / 8);
      const int hh = pix / kGW, ww = pix - hh * kGW;
      const int h = h0 + hh, w = w0 + ww;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (h < H && w < W) v = *reinterpret_cast<const uint4 *>(G + (((size_t)b * H + h) * W + w) * CO + c8 * 8);
      *reinterpret_cast<uint4 *>(sg + pix * S::RG + c8 * 8) = v;
    }
    __syncthreads();
    if (tid < CO)
      for (int p = 0; p < kGH * kGW; ++p) bsum += __bfloat162float(sg[p * S::RG + tid]);
#pragma unroll 1
    for (int r = 0; r < kGH; ++r)
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        uint32_t af[4];
        const int gp = r * kGW + 16 * s + (lane & 7) + (lane >> 4) * 8;
        ldsm4t(g_base + (gp * S::RG + mt * 16 + ((lane >> 3) & 1) * 8) * (uint32_t)sizeof(bf16), af);
        const int bp = 16 * s + (lane & 7) + ((lane >> 3) & 1) * 8;
        const int bc = np * 16 + (lane >> 4) * 8;
#pragma unroll
        for (int j = 0; j < S::kTPW; ++j) {
          const int t = tgrp + S::kTG * j;
          if (t < kTaps) {
            const int dy = t / 3 - 1, dx = t % 3 - 1;
            uint32_t bfr[4];
            ldsm4t(a_base + (((r + 1 + dy) * (kGW + 2) + bp + 1 + dx) * S::RA + bc) * (uint32_t)sizeof(bf16), bfr);
            mma16816(acc[j][0], af, bfr[0], bfr[1]);
            mma16816(acc[j][1], af, bfr[2], bfr[3]);
          }
        }
      }
  }
  float *out = partials + (size_t)blockIdx.x * (kTaps * CO * CI + CO);
  const int g = lane >> 2, tg = lane & 3;
#pragma unroll
  for (int j = 0; j < S::kTPW; ++j) {
    const int t = tgrp + S::kTG * j;
    if (t >= kTaps) continue;
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int co = mt * 16 + g + 8 * half, ci = np * 16 + n * 8 + 2 * tg;
        *reinterpret_cast<float2 *>(out + ((size_t)t * CO + co) * CI + ci) =
            make_float2(acc[j][n][2 * half], acc[j][n][2 * half + 1]);
      }
  }
  if (tid < CO) out[kTaps * CO * CI + tid] = bsum;
}

__global__ void sum_partials_kernel(const float *__restrict__ partials, int nparts, int len, float *__restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < nparts; ++b) s += partials[(size_t)b * len + i];
    out[i] = s;
  }
}

// ------------------------------------------------------------------ small kernels
__global__ void pack_input_kernel(const float *__restrict__ x, int cin, long long P, int CI, bf16 *__restrict__ a0) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < P * CI; q += (long long)gridDim.x * blockDim.x) {
    const long long p = q / CI;
    const int c = (int)(q - p * CI);
    a0[q] = __float2bfloat16_rn(c < cin ? x[p * cin + c] : 0.f);
  }
}

__global__ void unpad_output_kernel(const float *__restrict__ y32, int CO, long long P, int cout, float *__restrict__ y) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < P * cout; q += (long long)gridDim.x * blockDim.x) {
    const long long p = q / cout;
    y[q] = y32[p * CO + (int)(q - p * cout)];
  }
}

// Squared error of the real output channels and G = bf16(fp32(2 (y - t) / n)) (zero on
// padded channels); per-block partial sums of the squared error in FP64.
constexpr int kRedThreads = 256, kLossBlocks = 512;
__global__ void mse_kernel(const float *__restrict__ y32, int CO, const float *__restrict__ tgt, int cout, long long P,
                           double inv_n, bf16 *__restrict__ G, double *__restrict__ partials) {
  __shared__ double red[kRedThreads];
  double acc = 0.0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < P * CO; q += (long long)gridDim.x * blockDim.x) {
    const long long p = q / CO;
    const int c = (int)(q - p * CO);
    float gv = 0.f;
    if (c < cout) {
      const double d = (double)y32[q] - (double)tgt[p * cout + c];
      acc += d * d;
      gv = (float)(2.0 * d * inv_n);
    }
    G[q] = __float2bfloat16_rn(gv);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void final_sum_kernel(const double *__restrict__ partials, int n, double scale, double *__restrict__ out) {
  __shared__ double red[kRedThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += kRedThreads) acc += partials[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] * scale;
}

struct NetShape {
  int ci[kLayers], co[kLayers];
  long long woff[kLayers], boff[kLayers];  // offsets of weights and biases in the flat array
  long long wbf[kLayers];                  // offsets of a layer's BF16 weights
  long long n, nw;
};

// AdamW with bias-corrected moments; weight decay on weights only.
__global__ void adamw_kernel(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                             const float *__restrict__ g, NetShape S, float lr, float wd, float b1, float b2, float eps,
                             float bc1, float bc2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < S.n; i += (long long)gridDim.x * blockDim.x) {
    bool is_bias = false;
#pragma unroll
    for (int l = 0; l < kLayers; ++l) is_bias |= (i >= S.boff[l] && i < S.boff[l] + S.co[l]);
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float pi = p[i];
    if (!is_bias) pi -= lr * wd * pi;
    pi -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    p[i] = pi;
  }
}

// BF16 copies of every layer's weights: forward [t][co][ci] and, for the backward pass, the
// tap-flipped transpose [8 - t][ci][co].
__global__ void convert_weights_kernel(const float *__restrict__ p, NetShape S, bf16 *__restrict__ wf,
                                       bf16 *__restrict__ wt) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < S.nw; i += (long long)gridDim.x * blockDim.x) {
    int l = 0;
    while (l + 1 < kLayers && i >= S.wbf[l + 1]) ++l;
    const long long j = i - S.wbf[l];
    const int CI = S.ci[l], CO = S.co[l];
    const int t = (int)(j / ((long long)CO * CI));
    const int r = (int)(j - (long long)t * CO * CI);
    const int co = r / CI, ci = r - co * CI;
    const bf16 b = __float2bfloat16_rn(p[S.woff[l] + j]);
    wf[i] = b;
    wt[S.wbf[l] + ((long long)(kTaps - 1 - t) * CI + ci) * CO + co] = b;
  }
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Uniform weights in +-scale_l on real channels, zero on padded ones and on the biases.
__global__ void init_params_kernel(float *__restrict__ p, NetShape S, int cin, int hidden, int cout,
                                   unsigned long long seed) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < S.n; i += (long long)gridDim.x * blockDim.x) {
    float val = 0.f;
    for (int l = 0; l < kLayers; ++l) {
      if (i >= S.woff[l] && i < S.boff[l]) {
        const long long j = i - S.woff[l];
        const int CI = S.ci[l], CO = S.co[l];
        const int r = (int)(j % ((long long)CO * CI));
        const int co = r / CI, ci = r - co * CI;
        const int rci = l == 0 ? cin : hidden, rco = l == kLayers - 1 ? cout : hidden;
        if (ci < rci && co < rco) {
          const double scale = sqrt((l == kLayers - 1 ? 3.0 : 6.0) / (9.0 * rci));
          const uint64_t h = splitmix64(seed ^ splitmix64((uint64_t)i));
          const double u = (double)(h >> 11) * (1.0 / 9007199254740992.0);  // [0, 1)
          val = (float)((2.0 * u - 1.0) * scale);
        }
      }
    }
    p[i] = val;
  }
}

// ------------------------------------------------------------------ field-level glue
__constant__ int c_learn_idx[NRMG_LEARN_COUT] = {0, 1, 2, 4, 5, 6, 8, 10, 11, 12};
constexpr double kFeatScale = NRMG_LEARN_FEATURE_SCALE, kTargetScale = NRMG_LEARN_TARGET_SCALE;
__constant__ double c_learn_rest[NRMG_LEARN_COUT] = {1.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};

__global__ void features_kernel(const double *__restrict__ cf, int Hc, int Wc, double lx, double ly, double Kn,
                                double U, double *__restrict__ pro, float *__restrict__ x) {
  const int H = 2 * Hc, W = 2 * Wc;
  const double inv_u = kFeatScale / U;
  const float lkn = (float)log10(Kn), lkw = (float)log10(Kn * W / lx);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < H * W; c += gridDim.x * blockDim.x) {
    const int I = c / W, J = c - I * W;
    const int i = I >> 1, j = J >> 1;
    const int in = (I & 1) ? min(i + 1, Hc - 1) : max(i - 1, 0);
    const int jn = (J & 1) ? min(j + 1, Wc - 1) : max(j - 1, 0);
    const double *f00 = cf + (size_t)(i * Wc + j) * 14, *f01 = cf + (size_t)(i * Wc + jn) * 14;
    const double *f10 = cf + (size_t)(in * Wc + j) * 14, *f11 = cf + (size_t)(in * Wc + jn) * 14;
    double *o = pro + (size_t)c * 14;
    for (int k = 0; k < 14; ++k)
      o[k] = 0.5625 * f00[k] + 0.1875 * (f01[k] + f10[k]) + 0.0625 * f11[k];
    float *xc = x + (size_t)c * NRMG_LEARN_CIN;
    for (int k = 0; k < NRMG_LEARN_COUT; ++k) xc[k] = (float)((o[c_learn_idx[k]] - c_learn_rest[k]) * inv_u);
    xc[10] = lkn;
    xc[11] = lkw;
    xc[12] = (float)U;
    xc[13] = (float)((J + 0.5) / W);
    xc[14] = (float)((I + 0.5) / H);
    xc[15] = I == 0 ? 1.f : 0.f;
    xc[16] = J == W - 1 ? 1.f : 0.f;
    xc[17] = I == H - 1 ? 1.f : 0.f;
    xc[18] = J == 0 ? 1.f : 0.f;
  }
}

__global__ void targets_kernel(const double *__restrict__ pro, const double *__restrict__ fine, int cells, double U,
                               float *__restrict__ t) {
  const double inv_u = kTargetScale / U;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < cells * NRMG_LEARN_COUT; q += gridDim.x * blockDim.x) {
    const int c = q / NRMG_LEARN_COUT, k = q - c * NRMG_LEARN_COUT;
    t[q] = (float)((fine[(size_t)c * 14 + c_learn_idx[k]] - pro[(size_t)c * 14 + c_learn_idx[k]]) * inv_u);
  }
}

__global__ void combine_kernel(const double *__restrict__ pro, const float *__restrict__ y, int cells, double U,
                               double *__restrict__ out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += gridDim.x * blockDim.x) {
    const double *p = pro + (size_t)c * 14;
    double *o = out + (size_t)c * 14;
    for (int k = 0; k < 14; ++k) o[k] = p[k];
    for (int k = 0; k < NRMG_LEARN_COUT; ++k)
      o[c_learn_idx[k]] += (U / kTargetScale) * (double)y[(size_t)c * NRMG_LEARN_COUT + k];
    o[3] = 0.0;
    o[7] = 0.0;
    o[9] = 0.0;
    o[13] = 0.0;
  }
}

// ---- learned coarse-level correction: scale of the coarse change, network input, targets
constexpr double kCorrScale = NRMG_CORR_FIELD_SCALE;

// s = max over coarse cells and learned fields of |after - before| kCorrScale / U (one block;
// at least 1e-300 so that dividing by it stays finite)
__global__ void corr_scale_kernel(const double *__restrict__ cb, const double *__restrict__ ca, int cells, double U,
                                  double *__restrict__ s) {
  __shared__ double red[1024];
  double m = 0.0;
  for (int q = threadIdx.x; q < cells * NRMG_LEARN_COUT; q += blockDim.x) {
    const int c = q / NRMG_LEARN_COUT, k = q - c * NRMG_LEARN_COUT;
    const size_t o = (size_t)c * 14 + c_learn_idx[k];
    m = fmax(m, fabs(ca[o] - cb[o]));
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) s[0] = fmax(red[0] * kCorrScale / U, 1e-300);
}

__global__ void corr_features_kernel(const double *__restrict__ cb, const double *__restrict__ ca, int Hc, int Wc,
                                     const double *__restrict__ fine, double lx, double ly, double Kn, double U,
                                     const double *__restrict__ sdev, float *__restrict__ x) {
  const int H = 2 * Hc, W = 2 * Wc;
  const double inv_u = kCorrScale / U, inv_us = kCorrScale / (U * sdev[0]);
  const float lkn = (float)log10(Kn), lkw = (float)log10(Kn * W / lx);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < H * W; c += gridDim.x * blockDim.x) {
    const int I = c / W, J = c - I * W;
    const int i = I >> 1, j = J >> 1;
    const int in = (I & 1) ? min(i + 1, Hc - 1) : max(i - 1, 0);
    const int jn = (J & 1) ? min(j + 1, Wc - 1) : max(j - 1, 0);
    const size_t c00 = (size_t)(i * Wc + j) * 14, c01 = (size_t)(i * Wc + jn) * 14;
    const size_t c10 = (size_t)(in * Wc + j) * 14, c11 = (size_t)(in * Wc + jn) * 14;
    float *xc = x + (size_t)c * NRMG_CORR_CIN;
    for (int k = 0; k < NRMG_LEARN_COUT; ++k) {
      const int f = c_learn_idx[k];
      const double d = 0.5625 * (ca[c00 + f] - cb[c00 + f]) + 0.1875 * ((ca[c01 + f] - cb[c01 + f]) +
                                                                        (ca[c10 + f] - cb[c10 + f])) +
                       0.0625 * (ca[c11 + f] - cb[c11 + f]);
      xc[k] = (float)(d * inv_us);
      xc[10 + k] = (float)((fine[(size_t)c * 14 + f] - c_learn_rest[k]) * inv_u);
    }
    xc[20] = lkn;
    xc[21] = lkw;
    xc[22] = (float)U;
    xc[23] = (float)((J + 0.5) / W);
    xc[24] = (float)((I + 0.5) / H);
    xc[25] = I == 0 ? 1.f : 0.f;
    xc[26] = J == W - 1 ? 1.f : 0.f;
    xc[27] = I == H - 1 ? 1.f : 0.f;
    xc[28] = J == 0 ? 1.f : 0.f;
  }
}

__global__ void corr_targets_kernel(const double *__restrict__ fine, const double *__restrict__ conv, int cells,
                                    double U, double scale, float *__restrict__ t) {
  const double f = kCorrScale / (U * scale);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < cells * NRMG_LEARN_COUT; q += gridDim.x * blockDim.x) {
    const int c = q / NRMG_LEARN_COUT, k = q - c * NRMG_LEARN_COUT;
    t[q] = (float)((conv[(size_t)c * 14 + c_learn_idx[k]] - fine[(size_t)c * 14 + c_learn_idx[k]]) * f);
  }
}

// Graded positions of the Grad-13 coefficients (-1 when the degree exceeds M).
struct GradIdx {
  int s[3][3];     // e_i + e_j
  int q[3][3];     // q[i][d]: e_i + 2 e_d (d == i: 3 e_i)
};

__global__ void grad13_kernel(const double *__restrict__ fields, int ncell, int NP, GradIdx gi, double *__restrict__ P,
                              double *__restrict__ F) {
  const long long tot = (long long)ncell * NP;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (long long)gridDim.x * blockDim.x) {
    const long long c = q / NP;
    const int o = (int)(q - c * NP);
    const double *fc = fields + c * 14;
    double val = 0.0;
    if (o == 0) val = fc[0];
    const double tr3 = (fc[5] + fc[8] + fc[10]) / 3.0;
    const double sig[3][3] = {{fc[5] - tr3, fc[6], fc[7]}, {fc[6], fc[8] - tr3, fc[9]}, {fc[7], fc[9], fc[10] - tr3}};
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j)
        if (o == gi.s[i][j]) val = i == j ? 0.5 * sig[i][j] : sig[i][j];
    for (int i = 0; i < 3; ++i)
      for (int d = 0; d < 3; ++d)
        if (o == gi.q[i][d]) val = 0.2 * fc[11 + i];
    F[q] = val;
    if (o == 0) {
      double *pc = P + c * 4;
      pc[0] = fc[1];
      pc[1] = fc[2];
      pc[2] = 0.0;
      pc[3] = fc[4];
    }
  }
}

int graded_index(int M, int a1, int a2, int a3) {
  const int deg = a1 + a2 + a3;
  if (deg > M) return -1;
  return deg * (deg + 1) * (deg + 2) / 6 + (deg - a1) * (deg - a1 + 1) / 2 + (deg - a1 - a2);
}

int grid_1d(long long work, int cap = 4096) {
  long long g = (work + 255) / 256;
  return (int)std::max<long long>(1, std::min<long long>(g, cap));
}

}  // namespace

namespace nrmg {
cudaError_t launch_corr_inputs(const double *cb, const double *ca, int Hc, int Wc, const double *fine, double lx,
                               double ly, double Kn, double U, double *s_dev, float *x, cudaStream_t st) {
  corr_scale_kernel<<<1, 1024, 0, st>>>(cb, ca, Hc * Wc, U, s_dev);
  corr_features_kernel<<<grid_1d(4ll * Hc * Wc), 256, 0, st>>>(cb, ca, Hc, Wc, fine, lx, ly, Kn, U, s_dev, x);
  return cudaGetLastError();
}

cudaError_t launch_grad13(const double *fields, int ncell, int M, int NP, double *P, double *F, cudaStream_t st) {
  GradIdx gi;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      int e[3] = {0, 0, 0};
      e[i] += 1;
      e[j] += 1;
      gi.s[i][j] = graded_index(M, e[0], e[1], e[2]);
      int f[3] = {0, 0, 0};
      f[i] += 1;
      f[j] += 2;
      gi.q[i][j] = graded_index(M, f[0], f[1], f[2]);
    }
  grad13_kernel<<<grid_1d((long long)ncell * NP, 8192), 256, 0, st>>>(fields, ncell, NP, gi, P, F);
  return cudaGetLastError();
}
}  // namespace nrmg

// ------------------------------------------------------------------ host side of the network
struct nrmg_net {
  int cin, hidden, cout, CI0, CO3;
  long long max_pixels;
  cudaStream_t stream;
  int nsm;
  NetShape S;
  long long step;
  float *params, *m, *v, *grad;
  bf16 *wf, *wt;
  bf16 *act[kLayers];   // a_0 .. a_3 (inputs of the layers)
  float *y32;
  bf16 *g3, *gx, *gy;
  float *wpart;
  double *lpart, *loss;
  double *hloss;        // pinned host scalar
};

namespace {

int pad_in(int c) { return c <= 16 ? 16 : (c <= 32 ? 32 : 64); }

bool valid_sizes(int cin, int hidden, int cout, long long max_pixels) {
  return cin >= 1 && cin <= 64 && (hidden == 32 || hidden == 64) && cout >= 1 && cout <= 16 && max_pixels >= 1 &&
         max_pixels <= (1ll << 31);
}

NetShape make_shape(int cin, int hidden, int cout) {
  NetShape S;
  const int ci[kLayers] = {pad_in(cin), hidden, hidden, hidden};
  const int co[kLayers] = {hidden, hidden, hidden, 16};
  (void)cout;
  long long off = 0, wb = 0;
  for (int l = 0; l < kLayers; ++l) {
    S.ci[l] = ci[l];
    S.co[l] = co[l];
    S.woff[l] = off;
    off += (long long)kTaps * co[l] * ci[l];
    S.boff[l] = off;
    off += co[l];
    S.wbf[l] = wb;
    wb += (long long)kTaps * co[l] * ci[l];
  }
  S.n = off;
  S.nw = wb;
  return S;
}

struct Carve {
  size_t off = 0;
  char *base = nullptr;
  template <typename T>
  T *take(long long count) {
    off = (off + 255) & ~size_t(255);
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += (size_t)count * sizeof(T);
    return p;
  }
};

size_t carve(nrmg_net *n, char *base, int cin, int hidden, int cout, long long P) {
  NetShape S = make_shape(cin, hidden, cout);
  Carve c;
  c.base = base;
  float *params = c.take<float>(S.n), *m = c.take<float>(S.n), *v = c.take<float>(S.n), *grad = c.take<float>(S.n);
  bf16 *wf = c.take<bf16>(S.nw), *wt = c.take<bf16>(S.nw);
  bf16 *act[kLayers];
  act[0] = c.take<bf16>(P * S.ci[0]);
  for (int l = 1; l < kLayers; ++l) act[l] = c.take<bf16>(P * hidden);
  float *y32 = c.take<float>(P * 16);
  bf16 *g3 = c.take<bf16>(P * 16), *gx = c.take<bf16>(P * hidden), *gy = c.take<bf16>(P * hidden);
  float *wpart = c.take<float>((long long)kMaxGradCTAs * (kTaps * 64 * 64 + 64));
  double *lpart = c.take<double>(kLossBlocks), *loss = c.take<double>(1);
  if (n) {
    n->S = S;
    n->params = params;
    n->m = m;
    n->v = v;
    n->grad = grad;
    n->wf = wf;
    n->wt = wt;
    for (int l = 0; l < kLayers; ++l) n->act[l] = act[l];
    n->y32 = y32;
    n->g3 = g3;
    n->gx = gx;
    n->gy = gy;
    n->wpart = wpart;
    n->lpart = lpart;
    n->loss = loss;
  }
  return c.off + 256;
}

template <typename Kern>
int persistent_grid(Kern k, int threads, size_t smem, int nsm, long long ntiles) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, smem) != cudaSuccess || occ < 1) occ = 1;
  return (int)std::max<long long>(1, std::min<long long>(ntiles, (long long)occ * nsm));
}

template <int CI, int CO, int MODE>
cudaError_t conv_launch(const nrmg_net *n, const bf16 *in, const bf16 *w, const float *bias, const bf16 *mask, int B,
                        int H, int W, bf16 *out16, float *out32) {
  const size_t smem = ConvSmem<CI, CO>::bytes;
  auto k = conv3x3_kernel<CI, CO, MODE>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long ntiles = (long long)B * ((H + kTH - 1) / kTH) * ((W + kTW - 1) / kTW);
  const int grid = persistent_grid(k, kConvThreads, smem, n->nsm, ntiles);
  k<<<grid, kConvThreads, smem, n->stream>>>(in, w, bias, mask, B, H, W, out16, out32);
  return cudaGetLastError();
}

template <int CI, int CO>
cudaError_t wgrad_launch(const nrmg_net *n, const bf16 *a, const bf16 *G, int B, int H, int W, float *grad_out) {
  const size_t smem = GradSmem<CI, CO>::bytes;
  auto k = wgrad_kernel<CI, CO>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long ntiles = (long long)B * ((H + kGH - 1) / kGH) * ((W + kGW - 1) / kGW);
  const int grid = std::min(kMaxGradCTAs, persistent_grid(k, kGradThreads, smem, n->nsm, ntiles));
  k<<<grid, kGradThreads, smem, n->stream>>>(a, G, B, H, W, n->wpart);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int len = kTaps * CO * CI + CO;
  sum_partials_kernel<<<grid_1d(len, 1024), 256, 0, n->stream>>>(n->wpart, grid, len, grad_out);
  return cudaGetLastError();
}

// Dispatch on the padded channel counts: the forward layers are (ci_0, hidden), (hidden,
// hidden) with ReLU and (hidden, 16) linear; the backward-data passes (16, hidden) and
// (hidden, hidden) with the ReLU mask.
cudaError_t conv(const nrmg_net *n, int CI, int CO, int mode, const bf16 *in, const bf16 *w, const float *bias,
                 const bf16 *mask, int B, int H, int W, bf16 *out16, float *out32) {
#define NRMG_CONV(CI_, CO_, MODE_)                     \
  if (CI == CI_ && CO == CO_ && mode == MODE_)         \
    return conv_launch<CI_, CO_, MODE_>(n, in, w, bias, mask, B, H, W, out16, out32);
  NRMG_CONV(16, 32, kRelu)
  NRMG_CONV(16, 64, kRelu)
  NRMG_CONV(32, 32, kRelu)
  NRMG_CONV(32, 64, kRelu)
  NRMG_CONV(64, 32, kRelu)
  NRMG_CONV(64, 64, kRelu)
  NRMG_CONV(32, 16, kLinear)
  NRMG_CONV(64, 16, kLinear)
  NRMG_CONV(16, 32, kMask)
  NRMG_CONV(16, 64, kMask)
  NRMG_CONV(32, 32, kMask)
  NRMG_CONV(64, 64, kMask)
#undef NRMG_CONV
  return cudaErrorInvalidValue;
}

cudaError_t wgrad(const nrmg_net *n, int CI, int CO, const bf16 *a, const bf16 *G, int B, int H, int W, float *out) {
  if (CI == 16 && CO == 32) return wgrad_launch<16, 32>(n, a, G, B, H, W, out);
  if (CI == 16 && CO == 64) return wgrad_launch<16, 64>(n, a, G, B, H, W, out);
  if (CI == 32 && CO == 32) return wgrad_launch<32, 32>(n, a, G, B, H, W, out);
  if (CI == 32 && CO == 64) return wgrad_launch<32, 64>(n, a, G, B, H, W, out);
  if (CI == 64 && CO == 32) return wgrad_launch<64, 32>(n, a, G, B, H, W, out);
  if (CI == 64 && CO == 64) return wgrad_launch<64, 64>(n, a, G, B, H, W, out);
  if (CI == 32 && CO == 16) return wgrad_launch<32, 16>(n, a, G, B, H, W, out);
  if (CI == 64 && CO == 16) return wgrad_launch<64, 16>(n, a, G, B, H, W, out);
  return cudaErrorInvalidValue;
}

#define NCK(expr)                                   \
  do {                                              \
    if ((expr) != cudaSuccess) return NRMG_ERR_CUDA; \
  } while (0)

nrmg_status forward_internal(nrmg_net *n, const float *x, int B, int H, int W) {
  const long long P = (long long)B * H * W;
  const NetShape &S = n->S;
  pack_input_kernel<<<grid_1d(P * S.ci[0], 8192), 256, 0, n->stream>>>(x, n->cin, P, S.ci[0], n->act[0]);
  NCK(cudaGetLastError());
  for (int l = 0; l < kLayers; ++l) {
    const bool last = l == kLayers - 1;
    NCK(conv(n, S.ci[l], S.co[l], last ? kLinear : kRelu, n->act[l], n->wf + S.wbf[l], n->params + S.boff[l], nullptr,
             B, H, W, last ? nullptr : n->act[l + 1], last ? n->y32 : nullptr));
  }
  return NRMG_OK;
}

bool call_ok(const nrmg_net *n, const void *x, int B, int H, int W) {
  return n && x && B >= 1 && H >= 1 && W >= 1 && (long long)B * H * W <= n->max_pixels;
}

nrmg_status gradients_internal(nrmg_net *n, const float *x, const float *t, int B, int H, int W, float *grad) {
  nrmg_status s = forward_internal(n, x, B, H, W);
  if (s != NRMG_OK) return s;
  const long long P = (long long)B * H * W;
  const NetShape &S = n->S;
  mse_kernel<<<kLossBlocks, kRedThreads, 0, n->stream>>>(n->y32, S.co[3], t, n->cout, P, 1.0 / ((double)P * n->cout),
                                                          n->g3, n->lpart);
  NCK(cudaGetLastError());
  final_sum_kernel<<<1, kRedThreads, 0, n->stream>>>(n->lpart, kLossBlocks, 1.0 / ((double)P * n->cout), n->loss);
  NCK(cudaGetLastError());
  // layer l: dW_l from (a_l, G_l); G_{l-1} = bf16(convT(G_l, W_l) * [a_l > 0])
  const bf16 *Gl = n->g3;
  bf16 *bufs[2] = {n->gx, n->gy};
  for (int l = kLayers - 1; l >= 0; --l) {
    NCK(wgrad(n, S.ci[l], S.co[l], n->act[l], Gl, B, H, W, grad + S.woff[l]));
    if (l == 0) break;
    bf16 *Gn = bufs[l & 1];
    NCK(conv(n, S.co[l], S.ci[l], kMask, Gl, n->wt + S.wbf[l], nullptr, n->act[l], B, H, W, Gn, nullptr));
    Gl = Gn;
  }
  return NRMG_OK;
}

nrmg_status read_loss(nrmg_net *n, double *loss_out) {
  if (!loss_out) return NRMG_OK;
  NCK(cudaMemcpyAsync(n->hloss, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
  NCK(cudaStreamSynchronize(n->stream));
  *loss_out = *n->hloss;
  return NRMG_OK;
}

nrmg_status refresh_bf16(nrmg_net *n) {
  convert_weights_kernel<<<grid_1d(n->S.nw, 2048), 256, 0, n->stream>>>(n->params, n->S, n->wf, n->wt);
  NCK(cudaGetLastError());
  return NRMG_OK;
}

}  // namespace

namespace nrmg {
bool net_fits(const ::nrmg_net *n, int cin, int cout, long long pixels, cudaStream_t st) {
  return n && n->cin == cin && n->cout == cout && pixels <= n->max_pixels && n->stream == st;
}
}  // namespace nrmg

extern "C" {

size_t nrmg_net_workspace_bytes(int cin, int hidden, int cout, long long max_pixels) {
  if (!valid_sizes(cin, hidden, cout, max_pixels)) return 0;
  return carve(nullptr, nullptr, cin, hidden, cout, max_pixels);
}

nrmg_status nrmg_net_create(int cin, int hidden, int cout, long long max_pixels, unsigned long long seed,
                            void *ws, size_t ws_bytes, void *cuda_stream, nrmg_net **out) {
  if (!out || !ws || ((uintptr_t)ws & 255) || !valid_sizes(cin, hidden, cout, max_pixels)) return NRMG_ERR_ARG;
  *out = nullptr;
  if (ws_bytes < nrmg_net_workspace_bytes(cin, hidden, cout, max_pixels)) return NRMG_ERR_ARG;
  nrmg_net *n = new nrmg_net();
  n->cin = cin;
  n->hidden = hidden;
  n->cout = cout;
  n->max_pixels = max_pixels;
  n->stream = (cudaStream_t)cuda_stream;
  carve(n, (char *)ws, cin, hidden, cout, max_pixels);
  n->CI0 = n->S.ci[0];
  n->CO3 = n->S.co[3];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaMallocHost(&n->hloss, sizeof(double)) != cudaSuccess) {
    delete n;
    return NRMG_ERR_CUDA;
  }
  init_params_kernel<<<grid_1d(n->S.n, 2048), 256, 0, n->stream>>>(n->params, n->S, cin, hidden, cout, seed);
  cudaMemsetAsync(n->m, 0, sizeof(float) * n->S.n, n->stream);
  cudaMemsetAsync(n->v, 0, sizeof(float) * n->S.n, n->stream);
  if (cudaGetLastError() != cudaSuccess || refresh_bf16(n) != NRMG_OK) {
    cudaFreeHost(n->hloss);
    delete n;
    return NRMG_ERR_CUDA;
  }
  *out = n;
  return NRMG_OK;
}

nrmg_status nrmg_net_destroy(nrmg_net *n) {
  if (!n) return NRMG_ERR_ARG;
  cudaStreamSynchronize(n->stream);
  cudaFreeHost(n->hloss);
  delete n;
  return NRMG_OK;
}

long long nrmg_net_param_count(const nrmg_net *n) { return n ? n->S.n : 0; }

nrmg_status nrmg_net_get_params(nrmg_net *n, float *dev_params) {
  if (!n || !dev_params) return NRMG_ERR_ARG;
  NCK(cudaMemcpyAsync(dev_params, n->params, sizeof(float) * n->S.n, cudaMemcpyDeviceToDevice, n->stream));
  return NRMG_OK;
}

nrmg_status nrmg_net_set_params(nrmg_net *n, const float *dev_params) {
  if (!n || !dev_params) return NRMG_ERR_ARG;
  NCK(cudaMemcpyAsync(n->params, dev_params, sizeof(float) * n->S.n, cudaMemcpyDeviceToDevice, n->stream));
  NCK(cudaMemsetAsync(n->m, 0, sizeof(float) * n->S.n, n->stream));
  NCK(cudaMemsetAsync(n->v, 0, sizeof(float) * n->S.n, n->stream));
  n->step = 0;
  return refresh_bf16(n);
}

nrmg_status nrmg_net_forward(nrmg_net *n, const float *x, int B, int H, int W, float *y) {
  if (!call_ok(n, x, B, H, W) || !y) return NRMG_ERR_ARG;
  nrmg_status s = forward_internal(n, x, B, H, W);
  if (s != NRMG_OK) return s;
  const long long P = (long long)B * H * W;
  unpad_output_kernel<<<grid_1d(P * n->cout, 8192), 256, 0, n->stream>>>(n->y32, n->CO3, P, n->cout, y);
  NCK(cudaGetLastError());
  return NRMG_OK;
}

nrmg_status nrmg_net_gradients(nrmg_net *n, const float *x, const float *t, int B, int H, int W, float *grad,
                               double *loss_out) {
  if (!call_ok(n, x, B, H, W) || !t || !grad) return NRMG_ERR_ARG;
  nrmg_status s = gradients_internal(n, x, t, B, H, W, grad);
  if (s != NRMG_OK) return s;
  return read_loss(n, loss_out);
}

nrmg_status nrmg_net_train_step(nrmg_net *n, const float *x, const float *t, int B, int H, int W, float lr, float wd,
                                double *loss_out) {
  if (!call_ok(n, x, B, H, W) || !t || !(lr >= 0.f) || !(wd >= 0.f)) return NRMG_ERR_ARG;
  nrmg_status s = gradients_internal(n, x, t, B, H, W, n->grad);
  if (s != NRMG_OK) return s;
  n->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = (float)(1.0 - pow((double)b1, (double)n->step));
  const float bc2 = (float)(1.0 - pow((double)b2, (double)n->step));
  adamw_kernel<<<grid_1d(n->S.n, 2048), 256, 0, n->stream>>>(n->params, n->m, n->v, n->grad, n->S, lr, wd, b1, b2,
                                                              1e-8f, bc1, bc2);
  NCK(cudaGetLastError());
  if ((s = refresh_bf16(n)) != NRMG_OK) return s;
  return read_loss(n, loss_out);
}

nrmg_status nrmg_learned_features(const double *cf, int Hc, int Wc, double lx, double ly, double Kn, double U,
                                  double *pro, float *x, void *stream) {
  if (!cf || !pro || !x || Hc < 1 || Wc < 1 || (long long)Hc * Wc * 4 > (1ll << 30) || !(lx > 0.0) || !(ly > 0.0) ||
      !(Kn > 0.0) || !(U > 0.0))
    return NRMG_ERR_ARG;
  features_kernel<<<grid_1d(4ll * Hc * Wc), 256, 0, (cudaStream_t)stream>>>(cf, Hc, Wc, lx, ly, Kn, U, pro, x);
  NCK(cudaGetLastError());
  return NRMG_OK;
}

nrmg_status nrmg_learned_targets(const double *pro, const double *fine, int cells, double U, float *t, void *stream) {
  if (!pro || !fine || !t || cells < 1 || cells > (1 << 26) || !(U > 0.0)) return NRMG_ERR_ARG;
  targets_kernel<<<grid_1d((long long)cells * NRMG_LEARN_COUT), 256, 0, (cudaStream_t)stream>>>(pro, fine, cells, U, t);
  NCK(cudaGetLastError());
  return NRMG_OK;
}

nrmg_status nrmg_learned_correction_targets(const double *fine, const double *conv, int cells, double U,
                                            double scale, float *t, void *stream) {
  if (!fine || !conv || !t || cells < 1 || cells > (1 << 26) || !(U > 0.0) || !(scale > 0.0)) return NRMG_ERR_ARG;
  corr_targets_kernel<<<grid_1d((long long)cells * NRMG_LEARN_COUT), 256, 0, (cudaStream_t)stream>>>(fine, conv, cells,
                                                                                                    U, scale, t);
  NCK(cudaGetLastError());
  return NRMG_OK;
}

nrmg_status nrmg_learned_combine(const double *pro, const float *y, int cells, double U, double *out, void *stream) {
  if (!pro || !y || !out || cells < 1 || !(U > 0.0)) return NRMG_ERR_ARG;
  combine_kernel<<<grid_1d(cells), 256, 0, (cudaStream_t)stream>>>(pro, y, cells, U, out);
  NCK(cudaGetLastError());
  return NRMG_OK;
}

}  // extern "C"
