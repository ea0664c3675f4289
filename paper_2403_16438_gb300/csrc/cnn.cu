// Learned shift proposal: a 6-layer CNN on a 128x128 centre crop of the frame
// and of the template, regressing the frame's rigid shift, with hand-written
// forward, backward and optimizer kernels for sm_103a.
//
// Network (weights used in BF16, accumulation in FP32; master weights FP32):
//   input  [2][128][128]: frame crop and template crop, each normalised by its
//          own mean and standard deviation
//   conv1  3x3 stride 2 pad 1, 2 -> 32, ReLU        -> [32][64][64]
//   conv2..conv5 3x3 stride 2 pad 1, 32 -> 32, ReLU -> 32, 16, 8, 4
//   conv6  3x3 stride 1 pad 1, 32 -> 32, ReLU        -> [32][4][4]
//   global average pool -> 32, linear 32 -> 2 = shift / kShiftScale (dy, dx)
// Flat parameter layout: per conv layer weights [co][ci][3][3] then bias [co];
// then the linear weights [2][32] and bias [2].
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "vimg_internal.h"

namespace vimg {

namespace {

constexpr int kC = 32;
constexpr int kLayers = 6;
constexpr int kInC[kLayers] = {2, 32, 32, 32, 32, 32};
constexpr int kStride[kLayers] = {2, 2, 2, 2, 2, 1};
constexpr int kSide[kLayers + 1] = {128, 64, 32, 16, 8, 4, 4};  // input side of layer l = kSide[l]

constexpr int w_count(int l) { return kC * kInC[l] * 9; }
constexpr int w_off(int l) {
  int o = 0;
  for (int i = 0; i < l; ++i) o += w_count(i) + kC;
  return o;
}
constexpr int kLinOff = w_off(kLayers);
constexpr int kParams = kLinOff + 2 * kC + 2;

// Activation workspace layout (floats, per sample): input, then each layer's
// post-ReLU output, then the pooled vector and the network output.
constexpr int act_per_sample(int l) {  // size of buffer l (0 = input)
  return l == 0 ? 2 * 128 * 128 : kC * kSide[l] * kSide[l];
}
constexpr size_t act_off(int l, int n) {
  size_t o = 0;
  for (int i = 0; i < l; ++i) o += (size_t)act_per_sample(i) * n;
  return o;
}

constexpr int kThreads = 256;

// ---- input: centre crop, per-image normalisation ---------------------------------
__global__ void k_cnn_input(const uint16_t* __restrict__ frames, int H, int W,
                            const float* __restrict__ tmpl, long long tmpl_stride,
                            float* __restrict__ out) {
  const int b = blockIdx.x, ch = blockIdx.y;
  const int y0 = (H - kCrop) / 2, x0 = (W - kCrop) / 2;
  __shared__ float red[kThreads];
  __shared__ float stat[2];
  auto val = [&](int i) -> float {
    const int y = y0 + i / kCrop, x = x0 + i % kCrop;
    return ch == 0 ? (float)frames[(size_t)b * H * W + (size_t)y * W + x]
                   : tmpl[(size_t)b * tmpl_stride + (size_t)y * W + x];
  };
  float s = 0.f;
  for (int i = threadIdx.x; i < kCrop * kCrop; i += kThreads) s += val(i);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) stat[0] = red[0] / (kCrop * kCrop);
  __syncthreads();
  const float mean = stat[0];
  float q = 0.f;
  for (int i = threadIdx.x; i < kCrop * kCrop; i += kThreads) {
    const float d = val(i) - mean;
    q += d * d;
  }
  red[threadIdx.x] = q;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) stat[1] = 1.0f / (sqrtf(red[0] / (kCrop * kCrop)) + 1e-3f);
  __syncthreads();
  const float inv = stat[1];
  float* o = out + ((size_t)b * 2 + ch) * kCrop * kCrop;
  for (int i = threadIdx.x; i < kCrop * kCrop; i += kThreads) o[i] = (val(i) - mean) * inv;
}

// ---- conv 3x3 forward + ReLU: thread per (output pixel, group of kC / COG channels)
// The deep layers have few pixels, so they split the output channels over COG
// threads to keep enough warps in flight; the large layers give a thread PX
// adjacent output pixels of a row, which share each tap's weight loads.  Pairs
// of channels accumulate with the packed FP32 FMA (two independent
// round-to-nearest FMAs, the same results as scalar fmaf); every output sums
// its taps in the same order (input channels, rows, columns; taps outside the
// image skipped) whatever COG and PX.
template <int CIN, int S, int COG, int PX>
__global__ void __launch_bounds__(kThreads, 2)
    k_conv_fwd(const float* __restrict__ in, const __nv_bfloat16* __restrict__ w,
               const float* __restrict__ bias, float* __restrict__ out, int n, int HI, int HO) {
  constexpr int NC = kC / COG;          // output channels per thread (multiple of 4)
  constexpr int NXC = S * (PX - 1) + 3;  // input columns the PX pixels' taps read
  __shared__ __align__(16) float ws[CIN * 9][kC];
  for (int i = threadIdx.x; i < CIN * 9 * kC; i += kThreads) {
    const int co = i / (CIN * 9), r = i - co * (CIN * 9);
    ws[r][co] = __bfloat162float(w[i]);
  }
  __syncthreads();
  const int hox = HO / PX;  // pixel groups per output row
  const int npg = n * HO * hox;
  const int t = blockIdx.x * kThreads + threadIdx.x;
  if (t >= npg * COG) return;
  const int g = t / npg, pg = t - g * npg;
  const int b = pg / (HO * hox), rem = pg - b * HO * hox, oy = rem / hox;
  const int ox0 = (rem - oy * hox) * PX;
  float2 acc[PX][NC / 2];
#pragma unroll
  for (int k = 0; k < PX; ++k)
#pragma unroll
    for (int c = 0; c < NC / 2; ++c)
      acc[k][c] = make_float2(bias[g * NC + 2 * c], bias[g * NC + 2 * c + 1]);
  // the taps of the next input channel are loaded before the current channel's FMAs
  bool vy[3], vx[NXC];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int iy = oy * S + k - 1;
    vy[k] = iy >= 0 && iy < HI;
  }
#pragma unroll
  for (int j = 0; j < NXC; ++j) {
    const int ix = ox0 * S + j - 1;
    vx[j] = ix >= 0 && ix < HI;
  }
  const float* ip0 = in + (size_t)b * CIN * HI * HI + (oy * S - 1) * HI + (ox0 * S - 1);
  auto load_taps = [&](int ci, float (&v)[3][NXC]) {
    const float* ip = ip0 + (size_t)ci * HI * HI;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int j = 0; j < NXC; ++j) v[ky][j] = vy[ky] && vx[j] ? __ldg(ip + ky * HI + j) : 0.f;
  };
  // (one pixel per thread: the next channel's taps are loaded ahead; several
  // pixels per thread give the FMAs enough independent work without it)
  constexpr bool kAhead = PX == 1;
  float vin[3][NXC];
  load_taps(0, vin);
#pragma unroll(kAhead ? 2 : 1)
  for (int ci = 0; ci < CIN; ++ci) {
    float vnext[3][NXC];
    if (!kAhead && ci > 0) load_taps(ci, vin);
    if (kAhead && ci + 1 < CIN) load_taps(ci + 1, vnext);
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      if (!vy[ky]) continue;
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const float4* wr = reinterpret_cast<const float4*>(&ws[ci * 9 + ky * 3 + kx][g * NC]);
#pragma unroll
        for (int q = 0; q < NC / 4; ++q) {
          const float4 wv = wr[q];
#pragma unroll
          for (int k = 0; k < PX; ++k) {
            const int j = kx + S * k;
            if (!vx[j]) continue;
            const float2 vv = make_float2(vin[ky][j], vin[ky][j]);
            acc[k][2 * q] = __ffma2_rn(make_float2(wv.x, wv.y), vv, acc[k][2 * q]);
            acc[k][2 * q + 1] = __ffma2_rn(make_float2(wv.z, wv.w), vv, acc[k][2 * q + 1]);
          }
        }
      }
    }
    if (kAhead) {
#pragma unroll
      for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int j = 0; j < NXC; ++j) vin[ky][j] = vnext[ky][j];
    }
  }
  float* op = out + ((size_t)b * kC + g * NC) * HO * HO + oy * HO + ox0;
#pragma unroll
  for (int c = 0; c < NC / 2; ++c)
#pragma unroll
    for (int k = 0; k < PX; ++k) {
      op[(size_t)(2 * c) * HO * HO + k] = fmaxf(acc[k][c].x, 0.f);
      op[(size_t)(2 * c + 1) * HO * HO + k] = fmaxf(acc[k][c].y, 0.f);
    }
}

// ---- fused tail: conv4, conv5, conv6 (+ ReLU), global average pool, linear ---------
// One CTA per sample.  The layers' inputs stay in shared memory (the 16x16x32
// output of conv3 is read once); every output channel is the FMA chain of
// k_conv_fwd (bias, then input channels, rows, columns in order, taps outside
// the image skipped), the pool sums the 16 positions in order and scales by
// 1/16, and the linear layer sums its 32 products by a fixed butterfly.  The
// activations the backward pass reads (a4, a5, a6, the pooled vector) are
// written as well.
constexpr int kTailIn = kC * 16 * 16;  // conv4 input
constexpr size_t kTailSmem =
    sizeof(float) * ((size_t)kTailIn + kC * 9 * kC + kC * 8 * 8 + 2 * kC * 4 * 4);

template <int HI, int S>
__device__ __forceinline__ void tail_conv(const float* __restrict__ x, const float (*ws)[kC],
                                          const float* __restrict__ bias, float* __restrict__ y,
                                          float* __restrict__ yg) {
  constexpr int HO = HI / S, NPIX = HO * HO, NC = kC * NPIX / kThreads;  // channels per thread
  const int pix = threadIdx.x % NPIX, g = threadIdx.x / NPIX;
  const int oy = pix / HO, ox = pix - oy * HO;
  float acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = bias[g * NC + c];
  for (int ci = 0; ci < kC; ++ci) {
    const float* ip = x + ci * HI * HI;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const int iy = oy * S + ky - 1;
      if (iy < 0 || iy >= HI) continue;
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int ix = ox * S + kx - 1;
        if (ix < 0 || ix >= HI) continue;
        const float v = ip[iy * HI + ix];
        const float* wr = &ws[ci * 9 + ky * 3 + kx][g * NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = fmaf(wr[c], v, acc[c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const float r = fmaxf(acc[c], 0.f);
    y[(g * NC + c) * NPIX + pix] = r;
    yg[(g * NC + c) * NPIX + pix] = r;
  }
}

__device__ __forceinline__ void tail_weights(const __nv_bfloat16* __restrict__ w, float (*ws)[kC]) {
  for (int i = threadIdx.x; i < kC * 9 * kC; i += kThreads) {
    const int co = i / (kC * 9), r = i - co * (kC * 9);
    ws[r][co] = __bfloat162float(w[i]);
  }
}

__global__ void __launch_bounds__(kThreads)
    k_cnn_tail(const float* __restrict__ a3, const float* __restrict__ params,
               const __nv_bfloat16* __restrict__ wb, float* __restrict__ a4,
               float* __restrict__ a5, float* __restrict__ a6, float* __restrict__ gap,
               float* __restrict__ out) {
  extern __shared__ __align__(16) float tsm[];
  float* x = tsm;                                                  // [32][16][16]
  float(*ws)[kC] = reinterpret_cast<float(*)[kC]>(x + kTailIn);    // [288][32]
  float* y4 = x + kTailIn + kC * 9 * kC;                           // [32][8][8]
  float* y5 = y4 + kC * 8 * 8;                                     // [32][4][4]
  float* y6 = y5 + kC * 4 * 4;                                     // [32][4][4]
  const int b = blockIdx.x;
  const float4* src = reinterpret_cast<const float4*>(a3 + (size_t)b * kTailIn);
  for (int i = threadIdx.x; i < kTailIn / 4; i += kThreads)
    reinterpret_cast<float4*>(x)[i] = __ldg(src + i);
  tail_weights(wb + w_off(3), ws);
  __syncthreads();
  tail_conv<16, 2>(x, ws, params + w_off(3) + w_count(3), y4, a4 + (size_t)b * kC * 64);
  __syncthreads();
  tail_weights(wb + w_off(4), ws);
  __syncthreads();
  tail_conv<8, 2>(y4, ws, params + w_off(4) + w_count(4), y5, a5 + (size_t)b * kC * 16);
  __syncthreads();
  tail_weights(wb + w_off(5), ws);
  __syncthreads();
  tail_conv<4, 1>(y5, ws, params + w_off(5) + w_count(5), y6, a6 + (size_t)b * kC * 16);
  __syncthreads();
  if (threadIdx.x < 32) {  // pool and linear: lane = channel
    const int c = threadIdx.x;
    const float* lw = params + kLinOff;
    const float* pp = y6 + c * 16;
    float sv = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) sv += pp[i];
    sv *= (1.0f / 16.0f);
    gap[(size_t)b * kC + c] = sv;
    float o0 = lw[c] * sv, o1 = lw[kC + c] * sv;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      o0 += __shfl_xor_sync(0xffffffffu, o0, off);
      o1 += __shfl_xor_sync(0xffffffffu, o1, off);
    }
    if (c == 0) {
      out[2 * b] = o0 + params[kLinOff + 2 * kC];
      out[2 * b + 1] = o1 + params[kLinOff + 2 * kC + 1];
    }
  }
}

// ---- loss: L = (1/n) sum_b sum_j (out - target / scale)^2 -----------------------------
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ target, int n,
                      float scale, float* __restrict__ dout, float* __restrict__ loss) {
  __shared__ float red[kThreads];
  float s = 0.f;
  for (int i = threadIdx.x; i < 2 * n; i += kThreads) {
    const float d = out[i] - target[i] / scale;
    dout[i] = 2.0f * d / n;
    s += d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) *loss = red[0] / n;
}

// ---- backward of pool + linear: grads of the linear layer and of conv6's output ----
__global__ void k_gap_lin_bwd(const float* __restrict__ dout, const float* __restrict__ gap,
                              const float* __restrict__ lw, float* __restrict__ d_a6,
                              float* __restrict__ g_lw, float* __restrict__ g_lb, int n) {
  const int c = threadIdx.x;  // one warp, lanes = channels; loops over the batch
  float gw0 = 0.f, gw1 = 0.f, gb0 = 0.f, gb1 = 0.f;
  for (int b = 0; b < n; ++b) {
    const float d0 = dout[2 * b], d1 = dout[2 * b + 1];
    const float g = gap[(size_t)b * kC + c];
    gw0 += d0 * g;
    gw1 += d1 * g;
    gb0 += d0;
    gb1 += d1;
    const float dg = (d0 * lw[c] + d1 * lw[kC + c]) * (1.0f / 16.0f);
    float* p = d_a6 + ((size_t)b * kC + c) * 16;
#pragma unroll
    for (int i = 0; i < 16; ++i) p[i] = dg;
  }
  g_lw[c] += gw0;
  g_lw[kC + c] += gw1;
  if (c == 0) {
    g_lb[0] += gb0;
    g_lb[1] += gb1;
  }
}

// d <- d * (a > 0): gradient through the ReLU of a layer whose output is a.
__global__ void k_relu_bwd(float* __restrict__ d, const float* __restrict__ a, size_t count) {
  for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < count;
       i += (size_t)gridDim.x * kThreads)
    if (!(a[i] > 0.f)) d[i] = 0.f;
}

// ---- conv backward, data: thread per input pixel, all 32 input channels ------------
template <int S>
__global__ void __launch_bounds__(kThreads)
    k_conv_bwd_data(const float* __restrict__ dpre, const __nv_bfloat16* __restrict__ w,
                    float* __restrict__ din, int n, int HI, int HO) {
  __shared__ __align__(16) float wt[kC * 9][kC];  // [co*9 + k][ci]
  for (int i = threadIdx.x; i < kC * kC * 9; i += kThreads) {
    const int co = i / (kC * 9), r = i - co * (kC * 9), ci = r / 9, k = r - ci * 9;
    wt[co * 9 + k][ci] = __bfloat162float(w[i]);
  }
  __syncthreads();
  const int pix = blockIdx.x * kThreads + threadIdx.x;
  if (pix >= n * HI * HI) return;
  const int b = pix / (HI * HI), rem = pix - b * HI * HI, iy = rem / HI, ix = rem - iy * HI;
  float acc[kC];
#pragma unroll
  for (int c = 0; c < kC; ++c) acc[c] = 0.f;
#pragma unroll
  for (int ky = 0; ky < 3; ++ky) {
    const int ny = iy + 1 - ky;
    if (ny < 0 || ny % S) continue;
    const int oy = ny / S;
    if (oy >= HO) continue;
#pragma unroll
    for (int kx = 0; kx < 3; ++kx) {
      const int nx = ix + 1 - kx;
      if (nx < 0 || nx % S) continue;
      const int ox = nx / S;
      if (ox >= HO) continue;
      const float* gp = dpre + (size_t)b * kC * HO * HO + oy * HO + ox;
      for (int co = 0; co < kC; ++co) {
        const float g = __ldg(gp + (size_t)co * HO * HO);
        const float4* wr = reinterpret_cast<const float4*>(wt[co * 9 + ky * 3 + kx]);
#pragma unroll
        for (int q = 0; q < kC / 4; ++q) {
          const float4 wv = wr[q];
          acc[4 * q] = fmaf(wv.x, g, acc[4 * q]);
          acc[4 * q + 1] = fmaf(wv.y, g, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(wv.z, g, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(wv.w, g, acc[4 * q + 3]);
        }
      }
    }
  }
  float* op = din + (size_t)b * kC * HI * HI + iy * HI + ix;
#pragma unroll
  for (int c = 0; c < kC; ++c) op[(size_t)c * HI * HI] = acc[c];
}

// ---- conv backward, weights: block per (output channel, slice of pixels); each
// thread accumulates the 9 taps of kCiChunk input channels, then a block reduction
// and one atomic add per weight. -----------------------------------------------------
constexpr int kCiChunk = 8;

template <int CIN, int S>
__global__ void __launch_bounds__(kThreads)
    k_conv_bwd_w(const float* __restrict__ dpre, const float* __restrict__ in,
                 float* __restrict__ gw, float* __restrict__ gb, int n, int HI, int HO) {
  constexpr int CC = CIN < kCiChunk ? CIN : kCiChunk;
  const int co = blockIdx.x, ci0 = blockIdx.z * CC;
  const int npix = n * HO * HO;
  float acc[CC * 9];
#pragma unroll
  for (int i = 0; i < CC * 9; ++i) acc[i] = 0.f;
  float accb = 0.f;
  for (int pix = blockIdx.y * kThreads + threadIdx.x; pix < npix; pix += gridDim.y * kThreads) {
    const int b = pix / (HO * HO), rem = pix - b * HO * HO, oy = rem / HO, ox = rem - oy * HO;
    const float g = __ldg(dpre + ((size_t)b * kC + co) * HO * HO + rem);
    if (g == 0.f) continue;
    accb += g;
#pragma unroll
    for (int c = 0; c < CC; ++c) {
      const float* ip = in + ((size_t)b * CIN + ci0 + c) * HI * HI;
#pragma unroll
      for (int ky = 0; ky < 3; ++ky) {
        const int iy = oy * S + ky - 1;
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const int ix = ox * S + kx - 1;
          const float v = (iy >= 0 && iy < HI && ix >= 0 && ix < HI) ? __ldg(ip + iy * HI + ix) : 0.f;
          acc[c * 9 + ky * 3 + kx] = fmaf(g, v, acc[c * 9 + ky * 3 + kx]);
        }
      }
    }
  }
  __shared__ float red[kThreads / 32][CC * 9 + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < CC * 9; ++i) {
    float v = acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid][i] = v;
  }
  {
    float v = accb;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid][CC * 9] = v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < CC * 9 + 1; i += kThreads) {
    float v = 0.f;
    for (int q = 0; q < kThreads / 32; ++q) v += red[q][i];
    if (i < CC * 9) {
      const int c = i / 9, k = i - c * 9;
      atomicAdd(gw + ((size_t)co * CIN + ci0 + c) * 9 + k, v);
    } else if (blockIdx.z == 0) {
      atomicAdd(gb + co, v);
    }
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int count, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ q, int count) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  if (i < count) q[i] = __float2bfloat16_rn(p[i]);
}

inline int blocks(size_t count) { return (int)((count + kThreads - 1) / kThreads); }

template <int CIN, int S, int COG, int PX>
cudaError_t conv_fwd(const float* in, const __nv_bfloat16* w, const float* b, float* out, int n,
                     int HI, int HO, cudaStream_t st) {
  k_conv_fwd<CIN, S, COG, PX><<<blocks((size_t)n * HO * (HO / PX) * COG), kThreads, 0, st>>>(
      in, w, b, out, n, HI, HO);
  return cudaGetLastError();
}

}  // namespace

int cnn_param_count() { return kParams; }

size_t cnn_act_floats(int n) { return act_off(kLayers + 1, n) + (size_t)(kC + 2) * n; }

// Forward of n samples.  in: [n][2][128][128] already prepared; acts: workspace
// of cnn_act_floats(n) floats whose first part holds the input; out [n][2].
cudaError_t cnn_forward(const float* params, const __nv_bfloat16* wb, float* acts, int n,
                        float* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
    const float* in = acts + act_off(l, n);
    float* o = acts + act_off(l + 1, n);
    const __nv_bfloat16* w = wb + w_off(l);
    const float* b = params + w_off(l) + w_count(l);
    const int HI = kSide[l], HO = kSide[l + 1];
    // output channel groups per layer: more threads where there are few pixels
    if (l == 0) e = conv_fwd<2, 2, 1, 2>(in, w, b, o, n, HI, HO, st);
    else if (l == 1) e = conv_fwd<32, 2, 1, 2>(in, w, b, o, n, HI, HO, st);
    else e = conv_fwd<32, 2, 1, 2>(in, w, b, o, n, HI, HO, st);
  }
  if (e != cudaSuccess) return e;
  // conv4..conv6, pool and linear in one kernel per sample
  static unsigned char attr[kMaxDevices] = {};
  e = once_per_device(attr, [](int) {
    return cudaFuncSetAttribute(k_cnn_tail, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kTailSmem);
  });
  if (e != cudaSuccess) return e;
  k_cnn_tail<<<n, kThreads, kTailSmem, st>>>(
      acts + act_off(3, n), params, wb, acts + act_off(4, n), acts + act_off(5, n),
      acts + act_off(6, n), acts + act_off(kLayers + 1, n), out);
  return cudaGetLastError();
}

// Backward: dout [n][2] -> grads [kParams] (accumulated; the caller zeroes).
// dacts: workspace of cnn_act_floats(n) floats.
cudaError_t cnn_backward(const float* params, const __nv_bfloat16* wb, const float* acts,
                         float* dacts, int n, const float* dout, float* grads, cudaStream_t st) {
  const float* gap = acts + act_off(kLayers + 1, n);
  k_gap_lin_bwd<<<1, 32, 0, st>>>(dout, gap, params + kLinOff, dacts + act_off(kLayers, n),
                                  grads + kLinOff, grads + kLinOff + 2 * kC, n);
  cudaError_t e = cudaGetLastError();
  for (int l = kLayers - 1; l >= 0 && e == cudaSuccess; --l) {
    const int HI = kSide[l], HO = kSide[l + 1];
    float* d = dacts + act_off(l + 1, n);
    const float* a = acts + act_off(l + 1, n);
    const size_t cnt = (size_t)n * kC * HO * HO;
    k_relu_bwd<<<std::min(blocks(cnt), 4096), kThreads, 0, st>>>(d, a, cnt);
    const float* in = acts + act_off(l, n);
    float* gw = grads + w_off(l);
    float* gb = gw + w_count(l);
    const int ysl = std::max(1, std::min(64, blocks((size_t)n * HO * HO)));
    if (l == 0) {
      k_conv_bwd_w<2, 2><<<dim3(kC, ysl, 1), kThreads, 0, st>>>(d, in, gw, gb, n, HI, HO);
    } else {
      if (kStride[l] == 2)
        k_conv_bwd_w<32, 2><<<dim3(kC, ysl, 32 / kCiChunk), kThreads, 0, st>>>(d, in, gw, gb, n, HI, HO);
      else
        k_conv_bwd_w<32, 1><<<dim3(kC, ysl, 32 / kCiChunk), kThreads, 0, st>>>(d, in, gw, gb, n, HI, HO);
      e = cudaGetLastError();
      if (e != cudaSuccess) break;
      float* din = dacts + act_off(l, n);
      if (kStride[l] == 2)
        k_conv_bwd_data<2><<<blocks((size_t)n * HI * HI), kThreads, 0, st>>>(d, wb + w_off(l), din, n, HI, HO);
      else
        k_conv_bwd_data<1><<<blocks((size_t)n * HI * HI), kThreads, 0, st>>>(d, wb + w_off(l), din, n, HI, HO);
    }
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t cnn_input(const uint16_t* frames, int n, int H, int W, const float* tmpl,
                      long long tmpl_stride, float* acts, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_cnn_input<<<dim3(n, 2), kThreads, 0, st>>>(frames, H, W, tmpl, tmpl_stride, acts);
  return cudaGetLastError();
}

cudaError_t cnn_mse(const float* out, const float* target, int n, float* dout, float* loss,
                    cudaStream_t st) {
  k_mse<<<1, kThreads, 0, st>>>(out, target, n, kShiftScale, dout, loss);
  return cudaGetLastError();
}

cudaError_t cnn_adam(float* p, const float* g, float* m, float* v, float lr, float b1, float b2,
                     float eps, int step, cudaStream_t st) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<blocks(kParams), kThreads, 0, st>>>(p, g, m, v, kParams, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t cnn_to_bf16(const float* p, __nv_bfloat16* q, cudaStream_t st) {
  k_to_bf16<<<blocks(kParams), kThreads, 0, st>>>(p, q, kParams);
  return cudaGetLastError();
}

}  // namespace vimg
