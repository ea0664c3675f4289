// Motion estimation kernels for sm_103a: patch-tiled ZNCC (Sec. II of Bando et
// al., BIBM 2023), aggregation over patches, integer peak and subpixel refinement.
//
//   ZNCC_p(d) = sum_k Tc_p[k] F[k+d] / sqrt( |Tc_p|^2 * sum_k (F[k+d] - mean F)^2 )
//   C(d)      = mean_p ZNCC_p(d)
//
// Tc_p is the centred template patch (constant per template).  Its zero sum makes
// the numerator independent of the window mean, so the numerator is a plain
// correlation and the window statistics enter only through the normalisation.
// The window statistics are exact integers (sums of uint16 and their squares in
// int64), so N*sum F^2 - (sum F)^2 carries no rounding at all.  Patch values are
// summed over patches in 2^-40 fixed point with 64-bit integer atomics: the sum
// is exact and independent of the order in which CTAs finish.
#include <climits>
#include <cstdio>

#include "vimg_internal.h"

namespace vimg {

// ---------------------------------------------------------------------------
// Template preparation: per patch the mean (double), the centred patch (fp32),
// its squared norm and an integer offset near the patch mean.
__global__ void k_template_prep(const float* __restrict__ T, int W, PatchGrid g,
                                TemplateDev td) {
  const int p = blockIdx.x;
  const int ty = g.y0 + (p / g.nx) * kPatch, tx = g.x0 + (p % g.nx) * kPatch;
  __shared__ double red[64];
  double s = 0.0;
  for (int i = threadIdx.x; i < kPatchArea; i += blockDim.x)
    s += (double)T[(size_t)(ty + i / kPatch) * W + tx + i % kPatch];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 32; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double mean = red[0] / kPatchArea;
  __syncthreads();
  double q = 0.0;
  for (int i = threadIdx.x; i < kPatch * kTplStride; i += blockDim.x) {
    const int ky = i / kTplStride, kx = i % kTplStride;
    float v = 0.f;
    if (kx < kPatch) {
      const double c = (double)T[(size_t)(ty + ky) * W + tx + kx] - mean;
      v = (float)c;
      q += c * c;
    }
    td.tc[(size_t)p * kPatch * kTplStride + i] = v;
  }
  red[threadIdx.x] = q;
  __syncthreads();
  for (int o = 32; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    td.tn2[p] = (float)red[0];
    double m = mean < 0.0 ? 0.0 : (mean > 65535.0 ? 65535.0 : mean);
    td.coff[p] = (int)(m + 0.5);
  }
}

cudaError_t launch_template_prep(const float* T, int H, int W, PatchGrid g, TemplateDev td,
                                 cudaStream_t st) {
  (void)H;
  k_template_prep<<<g.ny * g.nx, 64, 0, st>>>(T, W, g, td);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Window statistics ("table-based area sums" of Sec. II, kept local): for each
// frame, patch and displacement the exact integers S1 = sum F, S2 = sum F^2 over
// the 21x21 window, and the normalisation factor
//   inv(d) = 21 / sqrt(|Tc|^2 * (441 S2 - S1^2))       (0 if either factor is 0)
// so that ZNCC = numerator * inv.  One CTA per (patch, frame); row sums slide
// along x, window sums slide along y.
constexpr int kStatThreads = 256;

__global__ void __launch_bounds__(kStatThreads)
    k_stats(const uint16_t* __restrict__ frames, int H, int W, PatchGrid g, int R,
            const float* __restrict__ tn2, float* __restrict__ inv) {
  const int p = blockIdx.x, f = blockIdx.y, np = g.ny * g.nx;
  const int w = 2 * R + 1, side = kPatch + 2 * R;
  const int ty = g.y0 + (p / g.nx) * kPatch - R, tx = g.x0 + (p % g.nx) * kPatch - R;
  __shared__ int reg[53 * 53];
  __shared__ int rs1[53 * kMaxWin];
  __shared__ long long rs2[53 * kMaxWin];
  const uint16_t* F = frames + (size_t)f * H * W;
  for (int i = threadIdx.x; i < side * side; i += blockDim.x)
    reg[i] = F[(size_t)(ty + i / side) * W + tx + i % side];
  __syncthreads();
  // Row sums: thread (r, quarter) slides over its quarter of the displacements.
  const int qlen = (w + 3) / 4;
  for (int job = threadIdx.x; job < side * 4; job += blockDim.x) {
    const int r = job >> 2, d0 = (job & 3) * qlen, d1 = min(w, d0 + qlen);
    if (d0 >= d1) continue;
    const int* row = reg + r * side;
    int s1 = 0;
    long long s2 = 0;
    for (int k = 0; k < kPatch; ++k) {
      const int v = row[d0 + k];
      s1 += v;
      s2 += (long long)v * v;
    }
    for (int d = d0; d < d1; ++d) {
      rs1[r * kMaxWin + d] = s1;
      rs2[r * kMaxWin + d] = s2;
      if (d + 1 < d1) {
        const int a = row[d + kPatch], b = row[d];
        s1 += a - b;
        s2 += (long long)a * a - (long long)b * b;
      }
    }
  }
  __syncthreads();
  const float t2 = tn2[p];
  float* out = inv + (size_t)(f * np + p) * w * kInvStride;
  for (int job = threadIdx.x; job < w * 4; job += blockDim.x) {
    const int dx = job >> 2, y0 = (job & 3) * qlen, y1 = min(w, y0 + qlen);
    if (y0 >= y1) continue;
    long long s1 = 0, s2 = 0;
    for (int k = 0; k < kPatch; ++k) {
      s1 += rs1[(y0 + k) * kMaxWin + dx];
      s2 += rs2[(y0 + k) * kMaxWin + dx];
    }
    for (int dy = y0; dy < y1; ++dy) {
      const long long sf = (long long)kPatchArea * s2 - s1 * s1;
      float v = 0.f;
      if (sf > 0 && t2 > 0.f) v = (float)kPatch * rsqrtf(t2 * (float)sf);
      out[dy * kInvStride + dx] = v;
      if (dy + 1 < y1) {
        s1 += rs1[(dy + kPatch) * kMaxWin + dx] - rs1[dy * kMaxWin + dx];
        s2 += rs2[(dy + kPatch) * kMaxWin + dx] - rs2[dy * kMaxWin + dx];
      }
    }
  }
}

cudaError_t launch_stats(const uint16_t* frames, int nf, int H, int W, PatchGrid g, int R,
                         const TemplateDev& td, float* inv, cudaStream_t st) {
  if (nf <= 0) return cudaSuccess;
  k_stats<<<dim3(g.ny * g.nx, nf), kStatThreads, 0, st>>>(frames, H, W, g, R, td.tn2, inv);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP32 correlation numerators on CUDA cores.
//
// CTA = (frame, patch row, group of up to kGroup patches).  The union of the
// group's search regions (53 rows x (21 G + 2R) cols) is staged once in shared
// memory as exact fp32 integers F - c.  Work is a list of output ROWS (patch u,
// displacement row dy), each 2R+1 displacements wide, accumulated in registers:
//   main pass u:      lane = dy in 0..31, every lane on patch u (template loads
//                     are warp-uniform broadcasts, frame rows distinct);
//   remainder pass:   lane = u, dy = 32 (only when 2R+1 = 33).
// A lane streams the 21 frame rows it needs: per row 53 shared loads feed
// 21 x 33 FMAs.  Each finished row is normalised and added to a per-CTA int64
// surface in shared memory; the CTA then adds that surface to the frame's
// global sums.
constexpr int kGroup = 15;
constexpr int kCsEntries = kMaxWin * kMaxWin + 1;  // keeps what follows 16-byte aligned
constexpr int kCorrWarps = 8;
constexpr int kCorrThreads = kCorrWarps * 32;

template <int NX>
__device__ __forceinline__ void corr_row(const float* __restrict__ rrow, int rs,
                                         const float* __restrict__ trow, float (&acc)[NX]) {
#pragma unroll
  for (int j = 0; j < NX; ++j) acc[j] = 0.f;
#pragma unroll 1
  for (int ky = 0; ky < kPatch; ++ky) {
    float fr[NX + kPatch - 1];
#pragma unroll
    for (int i = 0; i < NX + kPatch - 1; ++i) fr[i] = rrow[i];
    float t[kTplStride];
#pragma unroll
    for (int i = 0; i < kTplStride; i += 4) {
      const float4 v = *reinterpret_cast<const float4*>(trow + i);
      t[i] = v.x, t[i + 1] = v.y, t[i + 2] = v.z, t[i + 3] = v.w;
    }
#pragma unroll
    for (int kx = 0; kx < kPatch; ++kx)
#pragma unroll
      for (int j = 0; j < NX; ++j) acc[j] = fmaf(t[kx], fr[j + kx], acc[j]);
    rrow += rs;
    trow += kTplStride;
  }
}

template <int NX>
__global__ void __launch_bounds__(kCorrThreads, 2)
    k_corr_f32(const uint16_t* __restrict__ frames, int H, int W, PatchGrid g, int R,
               const float* __restrict__ tc, const int* __restrict__ coff,
               const float* __restrict__ inv, unsigned long long* __restrict__ csum) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int f = blockIdx.y, np = g.ny * g.nx, w = 2 * R + 1;
  const int groups_per_row = (g.nx + kGroup - 1) / kGroup;
  const int py = blockIdx.x / groups_per_row, gx = blockIdx.x % groups_per_row;
  const int px0 = gx * kGroup, G = min(kGroup, g.nx - px0);
  const int rows = kPatch + 2 * R, cols = G * kPatch + 2 * R;
  // Rows are allocated for the widest window (a lane always reads 53 values) and
  // given an odd stride so that lanes on different rows hit distinct banks.
  const int rs = (G * kPatch + 2 * kMaxR) | 1;
  const int ry = g.y0 + py * kPatch - R, rx = g.x0 + px0 * kPatch - R;

  unsigned long long* cs = reinterpret_cast<unsigned long long*>(smem);      // [w][w]
  float* tsm = reinterpret_cast<float*>(cs + kCsEntries);                    // [G][21][24]
  float* reg = tsm + kGroup * kPatch * kTplStride;                           // [rows][rs]

  const int p0 = py * g.nx + px0;
  const float c = (float)coff[p0];
  for (int i = threadIdx.x; i < w * w; i += blockDim.x) cs[i] = 0ull;
  for (int i = threadIdx.x * 4; i < G * kPatch * kTplStride; i += blockDim.x * 4)
    *reinterpret_cast<float4*>(tsm + i) =
        *reinterpret_cast<const float4*>(tc + (size_t)p0 * kPatch * kTplStride + i);
  const uint16_t* F = frames + (size_t)f * H * W;
  for (int i = threadIdx.x; i < rows * rs; i += blockDim.x) {
    const int r = i / rs, x = i - r * rs;
    reg[i] = x < cols ? (float)F[(size_t)(ry + r) * W + rx + x] - c : 0.f;
  }
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n_pass = G + (w > 32 ? 1 : 0);
  for (int pass = warp; pass < n_pass; pass += kCorrWarps) {
    int u, dy;
    if (pass < G) {
      u = pass;
      dy = lane;
    } else {
      u = lane;
      dy = 32;
    }
    const bool active = u < G && dy < w;
    const int uu = active ? u : 0, dd = active ? dy : 0;
    float acc[NX];
    corr_row<NX>(reg + dd * rs + uu * kPatch, rs, tsm + uu * kPatch * kTplStride, acc);
    if (active) {
      const float* iv = inv + ((size_t)(f * np + p0 + uu) * w + dd) * kInvStride;
      unsigned long long* crow = cs + dd * w;
#pragma unroll
      for (int j = 0; j < NX; ++j) {
        if (j < w) {
          const float z = acc[j] * __ldg(iv + j);
          atomicAdd(crow + j, (unsigned long long)__float2ll_rn(z * (float)kFix));
        }
      }
    }
  }
  __syncthreads();
  unsigned long long* out = csum + (size_t)f * w * w;
  for (int i = threadIdx.x; i < w * w; i += blockDim.x) atomicAdd(out + i, cs[i]);
}

static size_t corr_smem_bytes(int R) {
  const int rows = kPatch + 2 * R, rs = (kGroup * kPatch + 2 * kMaxR) | 1;
  return sizeof(unsigned long long) * kCsEntries +
         sizeof(float) * (size_t)kGroup * kPatch * kTplStride + sizeof(float) * rows * rs;
}

cudaError_t launch_corr_f32(const uint16_t* frames, int nf, int H, int W, PatchGrid g, int R,
                            const TemplateDev& td, const float* inv,
                            unsigned long long* csum, cudaStream_t st) {
  if (nf <= 0) return cudaSuccess;
  const size_t smem = corr_smem_bytes(R);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_corr_f32<kMaxWin>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)corr_smem_bytes(kMaxR));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int groups = g.ny * ((g.nx + kGroup - 1) / kGroup);
  k_corr_f32<kMaxWin><<<dim3(groups, nf), kCorrThreads, smem, st>>>(frames, H, W, g, R, td.tc,
                                                                    td.coff, inv, csum);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Integer peak with the tie-break (largest C, then smallest dy^2+dx^2, then dy,
// then dx) and the per-axis 3-point parabola.  One warp per frame.  All
// comparisons use the exact fixed-point sums.
struct Cand {
  long long v;
  int key;  // (dy^2+dx^2) << 12 | (dy+16) << 6 | (dx+16): smaller wins ties
  int idx;
};

__device__ __forceinline__ bool better(const Cand& a, const Cand& b) {
  return a.v > b.v || (a.v == b.v && a.key < b.key);
}

__device__ __forceinline__ Cand warp_best(Cand c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Cand d;
    d.v = __shfl_xor_sync(0xffffffffu, c.v, o);
    d.key = __shfl_xor_sync(0xffffffffu, c.key, o);
    d.idx = __shfl_xor_sync(0xffffffffu, c.idx, o);
    if (better(d, c)) c = d;
  }
  return c;
}

__global__ void k_peak(const unsigned long long* __restrict__ csum, int R, int np,
                       float* __restrict__ shifts, float* __restrict__ info,
                       double* __restrict__ surface) {
  const int f = blockIdx.x, lane = threadIdx.x, w = 2 * R + 1, nw = w * w;
  const long long* C = reinterpret_cast<const long long*>(csum) + (size_t)f * nw;
  const Cand none = {LLONG_MIN, 0x7fffffff, -1};
  Cand b = none;
  for (int i = lane; i < nw; i += 32) {
    const int dy = i / w - R, dx = i % w - R;
    Cand c = {C[i], ((dy * dy + dx * dx) << 12) | ((dy + 16) << 6) | (dx + 16), i};
    if (better(c, b)) b = c;
  }
  b = warp_best(b);
  Cand s2 = none;
  for (int i = lane; i < nw; i += 32) {
    if (i == b.idx) continue;
    const int dy = i / w - R, dx = i % w - R;
    Cand c = {C[i], ((dy * dy + dx * dx) << 12) | ((dy + 16) << 6) | (dx + 16), i};
    if (better(c, s2)) s2 = c;
  }
  s2 = warp_best(s2);
  if (surface) {
    for (int i = lane; i < nw; i += 32) surface[(size_t)f * nw + i] = (double)C[i] / kFix / np;
  }
  if (lane == 0) {
    const int iy = b.idx / w, ix = b.idx % w;
    float s[2] = {(float)(iy - R), (float)(ix - R)};
    for (int ax = 0; ax < 2; ++ax) {
      const int i = ax == 0 ? iy : ix;
      if (i == 0 || i == w - 1) continue;
      const int step = ax == 0 ? w : 1;
      const long long cm = C[b.idx - step], cp = C[b.idx + step], c0 = C[b.idx];
      const long long den = cm - 2 * c0 + cp;
      if (den >= 0) continue;
      float d = (float)(cm - cp) / (2.0f * (float)den);
      d = fminf(0.5f, fmaxf(-0.5f, d));
      s[ax] += d;
    }
    if (shifts) {
      shifts[2 * f] = s[0];
      shifts[2 * f + 1] = s[1];
    }
    if (info) {
      info[4 * f + 0] = (float)(iy - R);
      info[4 * f + 1] = (float)(ix - R);
      info[4 * f + 2] = (float)((double)b.v / kFix / np);
      info[4 * f + 3] = s2.idx >= 0 ? (float)((double)s2.v / kFix / np) : 0.f;
    }
  }
}

cudaError_t launch_peak(const unsigned long long* csum, int nf, int R, int np, float* shifts,
                        float* peak_info, double* surface, cudaStream_t st) {
  if (nf <= 0) return cudaSuccess;
  k_peak<<<nf, 32, 0, st>>>(csum, R, np, shifts, peak_info, surface);
  return cudaGetLastError();
}

}  // namespace vimg
