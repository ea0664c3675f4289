// Fused temporal pass for sm_103a: resampling of each frame at its shift, the
// corrected (or high-passed) output, the Gaussian pre-smoothing of Eq. 2 and the
// per-segment summaries of Sec. III-B (Bando et al., BIBM 2023):
//   S_i(x) = (1/L) sum_t V_i(x,t)                              (Eq. 1)
//   T_i(x) = max_t Vbar_i(x,t) - median_t Vbar_i(x,t)           (Eq. 2)
// with V_t(y,x) = F_t(y + s_y, x + s_x) (bilinear, clamped coordinates) and
// Vbar the Gaussian-smoothed V (radius ceil(4 sigma), mirror border).
//
// One CTA owns a 32x32 output tile for one segment slot and walks the slot's
// frames in order.  Per frame it resamples the tile plus a 12-pixel halo into
// shared memory (the halo pixels are mirrored at the image border, exactly as
// the Gaussian's boundary rule asks), writes the tile's corrected pixels, runs
// the row and column passes of the separable Gaussian in shared memory, and
// updates per-pixel running sum and max in registers and the smoothed history
// of the segment in shared memory (50 x 1024 floats).  At the end of a complete
// segment every pixel's median comes from two 25-element sorting networks and a
// merge-path selection of the 25th and 26th smallest values.
//
// The high-pass y[t] = v[t] - (1/W) sum_{k<W} v[t-k] (v[t<0] := v[0]) keeps an
// exact running sum in 2^-16 fixed point (64-bit integers); values leaving the
// window are recomputed from their frames rather than stored.
//
// Voltage traces (Sec. II, third stage: the mean of the corrected frame within
// each neuron ROI) ride on the same pass: each pixel's V_t, in 2^-20 fixed point,
// is summed over the lanes of a warp per ROI and added to a 64-bit per-frame,
// per-ROI accumulator -- integer sums, so the result does not depend on the
// order of the atomics, on the tiling or on the chunking of the stream.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cstring>

#include "tc_ptx.h"
#include "vimg_internal.h"

namespace vimg {

constexpr int kTempThreads = 512;
constexpr int kFst = 58;                 // staged frame row stride (uint16), >= 58 columns
constexpr int kFstRows = 57;             // staged frame rows (56 + 1 for the bilinear taps)
constexpr int kExt = kTile + 2 * kGaussMaxRadius;  // 56
constexpr int kTaps = 2 * kGaussMaxRadius + 1;     // 25
constexpr float kHpScale = 65536.0f;

// ---- sorting networks (Batcher's odd-even merge sort, generated at compile time)
struct CmpPair {
  unsigned char a, b;
};

template <int N, int NREAL>
struct OddEvenMergeNet {
  CmpPair pairs[N * 16];
  int n;
  constexpr OddEvenMergeNet() : pairs(), n(0) {
    for (int p = 1; p < N; p <<= 1)
      for (int k = p; k >= 1; k >>= 1)
        for (int j = k % p; j + k < N; j += 2 * k)
          for (int i = 0; i < k && i + j + k < N; ++i)
            if ((i + j) / (2 * p) == (i + j + k) / (2 * p) && i + j + k < NREAL) {
              pairs[n].a = (unsigned char)(i + j);
              pairs[n].b = (unsigned char)(i + j + k);
              ++n;
            }
  }
};

template <int N, int NREAL>
__device__ __forceinline__ void sort_net(float* v) {
  constexpr OddEvenMergeNet<N, NREAL> net{};
  constexpr int nc = net.n;
#pragma unroll
  for (int c = 0; c < nc; ++c) {
    const float x = v[net.pairs[c].a], y = v[net.pairs[c].b];
    v[net.pairs[c].a] = fminf(x, y);
    v[net.pairs[c].b] = fmaxf(x, y);
  }
}

// Median of 50 values: sort both halves, then the k-th smallest of two sorted
// runs A, B is min_i max(A[i-1], B[k-1-i]).
__device__ __forceinline__ float median50_v(const float (&h)[50], float* maxv = nullptr) {
  float a[32], b[32];
#pragma unroll
  for (int i = 0; i < 25; ++i) {
    a[i] = h[i];
    b[i] = h[25 + i];
  }
  sort_net<32, 25>(a);
  sort_net<32, 25>(b);
  float m25 = fminf(a[24], b[24]);
#pragma unroll
  for (int i = 1; i <= 24; ++i) m25 = fminf(m25, fmaxf(a[i - 1], b[24 - i]));
  float m26 = FLT_MAX;
#pragma unroll
  for (int i = 1; i <= 25; ++i) m26 = fminf(m26, fmaxf(a[i - 1], b[25 - i]));
  if (maxv) *maxv = fmaxf(a[24], b[24]);
  return 0.5f * (m25 + m26);
}

// Median of the first n <= 50 values (any n): pad to 64 with +inf, sort, pick.
__device__ __forceinline__ float median_any_v(const float (&h)[50], int n, float* maxv = nullptr) {
  float v[64];
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = (i < 50 && i < n) ? h[i] : FLT_MAX;
  sort_net<64, 64>(v);
  float lo = 0.f, hi = 0.f, top = 0.f;
  const int il = (n - 1) / 2, ih = n / 2;
#pragma unroll
  for (int i = 0; i < 64; ++i) {
    if (i == il) lo = v[i];
    if (i == ih) hi = v[i];
    if (i == n - 1) top = v[i];
  }
  if (maxv) *maxv = top;
  return 0.5f * (lo + hi);
}

__device__ __forceinline__ float median50(const float* __restrict__ h, int stride) {
  float v[50];
#pragma unroll
  for (int i = 0; i < 50; ++i) v[i] = h[i * stride];
  return median50_v(v);
}

__device__ __forceinline__ float median_any(const float* __restrict__ h, int stride, int n) {
  float v[50];
#pragma unroll
  for (int i = 0; i < 50; ++i) v[i] = i < n ? h[i * stride] : FLT_MAX;
  return median_any_v(v, n);
}

// ---- resampling ----------------------------------------------------------------
struct Split {
  int i;
  float f;
};

__device__ __forceinline__ Split split_shift(float s) {
  const float fl = floorf(s);
  return {(int)fl, s - fl};
}

// Mirror index for the Gaussian border ("d c b a | a b c d"), then clamped into
// the image: indices more than 12 past the border only feed outputs outside it.
__device__ __forceinline__ int mirror_idx(int i, int n) {
  i = i < 0 ? -i - 1 : (i >= n ? 2 * n - i - 1 : i);
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// V(y, x) = F(y + s_y, x + s_x), bilinear, coordinates clamped to the image.
// s = i + f with 0 <= f < 1 keeps every weight exact.  Global-memory form (used
// for the few high-pass samples outside the staged tile).
__device__ __forceinline__ float bilin(const uint16_t* __restrict__ F, int H, int W, int y, int x,
                                       Split sy, Split sx) {
  int r0, r1, c0, c1;
  float wy, wx;
  const int yi = y + sy.i, xi = x + sx.i;
  if (yi < 0) {
    r0 = r1 = 0;
    wy = 0.f;
  } else if (yi >= H - 1) {
    r0 = r1 = H - 1;
    wy = 0.f;
  } else {
    r0 = yi;
    r1 = yi + 1;
    wy = sy.f;
  }
  if (xi < 0) {
    c0 = c1 = 0;
    wx = 0.f;
  } else if (xi >= W - 1) {
    c0 = c1 = W - 1;
    wx = 0.f;
  } else {
    c0 = xi;
    c1 = xi + 1;
    wx = sx.f;
  }
  const float a = __ldg(F + (size_t)r0 * W + c0), b = __ldg(F + (size_t)r0 * W + c1);
  const float c = __ldg(F + (size_t)r1 * W + c0), d = __ldg(F + (size_t)r1 * W + c1);
  const float top = fmaf(wx, b - a, a), bot = fmaf(wx, d - c, c);
  return fmaf(wy, bot - top, top);
}

// Source window of the staged frame tile: the 57x57 frame pixels under the
// halo-extended tile moved by the shift's integer part, (r0, c0) = tile origin
// - 12 + floor(s).  Pixels outside the image are staged with clamped
// coordinates (replicated edges), which makes the bilinear formula on the
// staged window equal to the clamped-coordinate resampling everywhere in the
// image.  `plain` = the window lies inside the image (no clamping needed).
struct StageGeom {
  Split sy, sx;
  int r0, c0;   // window origin in the frame (may be outside the image)
  int c0e;      // first staged column (c0, or c0 rounded down to even for 2-pixel words)
  bool plain;
};

__device__ __forceinline__ StageGeom stage_geom(Split sy, Split sx, int ty0, int tx0, int H,
                                                int W, bool pairs) {
  StageGeom g;
  g.sy = sy;
  g.sx = sx;
  g.r0 = ty0 - kGaussMaxRadius + sy.i;
  g.c0 = tx0 - kGaussMaxRadius + sx.i;
  g.plain = g.r0 >= 0 && g.r0 + kFstRows - 1 <= H - 1 && g.c0 >= 0 && g.c0 + kFstRows - 1 <= W - 1;
  g.c0e = (g.plain && pairs) ? (g.c0 & ~1) : g.c0;
  return g;
}

__device__ __forceinline__ void frame_at(const FrameSource& s, long long t, const uint16_t*& F,
                                         Split& sy, Split& sx, int HW) {
  long long v = t - s.t_first;
  if (v < 0) v = 0;  // the host keeps every frame a launch can ask for; never read before it
  if (v >= (long long)s.n_carry + s.n_batch) v = (long long)s.n_carry + s.n_batch - 1;
  const float* sh;
  if (v < s.n_carry) {
    F = s.carry + (size_t)v * HW;
    sh = s.carry_shift + 2 * v;
  } else {
    F = s.batch + (size_t)(v - s.n_carry) * HW;
    sh = s.batch_shift + 2 * (v - s.n_carry);
  }
  sy = split_shift(sh[0]);
  sx = split_shift(sh[1]);
}

__device__ __forceinline__ long long hp_q(float v) { return __float2ll_rn(v * kHpScale); }

// Adds V of this warp's 64 pixels to the per-ROI sums of frame row `acc`.  ma /
// mb: the pixels' ROI ids + 1 in four 16-bit fields (0 = unused).  V in
// [0, 65535] gives q = round(V 2^20) < 2^36 per pixel.  Each pass
// takes one id still pending in some lane, so a warp does one 64-bit atomic per
// distinct ROI it covers.
__device__ __forceinline__ void roi_add(unsigned long long ma, unsigned long long mb, float v_a,
                                        float v_b, unsigned long long* __restrict__ acc) {
  const long long qa = __float2ll_rn(v_a * (float)kRoiFix), qb = __float2ll_rn(v_b * (float)kRoiFix);
  for (;;) {
    const unsigned long long m = ma ? ma : mb;
    const unsigned my = m ? (unsigned)(m >> ((__ffsll((long long)m) - 1) & ~15)) & 0xffffu : 0u;
    const unsigned any = __ballot_sync(0xffffffffu, my != 0);
    if (!any) break;
    const unsigned id = __shfl_sync(0xffffffffu, my, __ffs(any) - 1);
    long long c = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (((ma >> (16 * k)) & 0xffffu) == id) {
        c += qa;
        ma &= ~(0xffffull << (16 * k));
      }
      if (((mb >> (16 * k)) & 0xffffu) == id) {
        c += qb;
        mb &= ~(0xffffull << (16 * k));
      }
    }
    // 0 <= c < 2^37: the warp sum of its low 20 and high 17 bits fits 32 bits each
    const unsigned lo = __reduce_add_sync(0xffffffffu, (unsigned)c & 0xfffffu);
    const unsigned hi = __reduce_add_sync(0xffffffffu, (unsigned)(c >> 20));
    if ((threadIdx.x & 31) == 0)
      atomicAdd(acc + (id - 1), ((unsigned long long)hi << 20) + lo);
  }
}

// ---- the fused kernel ------------------------------------------------------------
constexpr int kPfRows = (kFstRows + 7) / 8;  // prefetch: 64 columns x 8 rows per pass
constexpr int kPf2Rows = (kFstRows + 15) / 16;  // pairs: 32 words (64 columns) x 16 rows per pass

// One CTA per (job, segment slot, tile); the job comes from the prefix counts.
__global__ void __launch_bounds__(kTempThreads, 1) k_temporal(const __grid_constant__ TemporalBatch b) {
  extern __shared__ __align__(16) float sm[];
  const int jb = job_of(b.begin, b.n, blockIdx.x);
  const TemporalArgs& a = b.a[jb];
  const int H = a.H, W = a.W, L = a.L, HW = H * W;
  float* vext = sm;                            // [56][56] resampled tile + halo
  float* hbuf = vext + kExt * kExt;            // [56][32] row-smoothed
  float* hist = hbuf + kExt * kTile;           // [L][1024] smoothed history
  float* shs = hist + (size_t)L * kTile * kTile;  // [L][2] shifts of the slot's frames
  unsigned short* fst = reinterpret_cast<unsigned short*>(shs + 2 * kMaxL);  // [57][58]
  const int ntx = (W + kTile - 1) / kTile, tiles = ntx * ((H + kTile - 1) / kTile);
  const int local = blockIdx.x - b.begin[jb];
  const int slot = local / tiles, tile = local - slot * tiles;
  const int ty0 = (tile / ntx) * kTile, tx0 = (tile % ntx) * kTile;
  const int tid = threadIdx.x, lx = tid & 31, ly0 = (tid >> 5) * 2;
  const int x = tx0 + lx, ya = ty0 + ly0, yb = ya + 1;
  const bool va = ya < H && x < W, vb = yb < H && x < W;
  const FrameSource& src = a.src;
  const long long t_end = src.t_first + src.n_carry + src.n_batch;
  const long long s0 = a.seg_base + (long long)slot * L;
  const long long s1 = s0 + L < t_end ? s0 + L : t_end;
  const int nfr = (int)(s1 - s0);
  const bool complete = s0 + L <= t_end;
  // warps holding ROI pixels (the ids themselves are re-read per frame from L1)
  const unsigned long long* roi_pa =
      a.roi_acc && va ? a.roi_members + (size_t)ya * W + x : nullptr;
  const unsigned long long* roi_pb =
      a.roi_acc && vb ? a.roi_members + (size_t)yb * W + x : nullptr;
  const bool roi_warp = __any_sync(0xffffffffu, (roi_pa && __ldg(roi_pa)) || (roi_pb && __ldg(roi_pb)));

  // halo rows / columns of the extended tile outside the image: mirrored (Eq. 2's
  // border rule) by copies after the resampling
  const bool mirror_rows = ty0 - kGaussMaxRadius < 0 || ty0 + kTile + kGaussMaxRadius > H;
  const bool mirror_cols = tx0 - kGaussMaxRadius < 0 || tx0 + kTile + kGaussMaxRadius > W;

  float w[kTaps];
#pragma unroll
  for (int i = 0; i < kTaps; ++i) w[i] = a.gw[i];

  // shifts of the slot's frames
  for (int i = tid; i < 2 * nfr; i += kTempThreads) {
    const long long v = s0 + (i >> 1) - src.t_first;
    shs[i] = v < src.n_carry ? src.carry_shift[2 * v + (i & 1)]
                             : src.batch_shift[2 * (v - src.n_carry) + (i & 1)];
  }
  __syncthreads();

  auto frame_ptr = [&](long long t) -> const uint16_t* {
    const long long v = t - src.t_first;
    return v < src.n_carry ? src.carry + (size_t)v * HW : src.batch + (size_t)(v - src.n_carry) * HW;
  };
  const bool pairs = a.pairs != 0;
  auto geom_of = [&](int fi) {
    return stage_geom(split_shift(shs[2 * fi]), split_shift(shs[2 * fi + 1]), ty0, tx0, H, W,
                      pairs);
  };
  // prefetch pattern: column pc of rows pr, pr + 8, ... (no division); with
  // pairs, 2-pixel word pc2 of rows pr2, pr2 + 16, ...
  const int pc = tid & 63, pr = tid >> 6;
  const int pc2 = tid & 31, pr2 = tid >> 5;

  float sum_a = 0.f, sum_b = 0.f, mx_a = -FLT_MAX, mx_b = -FLT_MAX;
  long long hs_a = 0, hs_b = 0;
  bool hp_init = false;
  const bool do_hp = a.out_hp && a.hp_w > 0 && a.corrected;
  const float hp_inv = 1.0f / ((float)a.hp_w * kHpScale);

  // Loads of a frame's window into registers: 2-pixel words (plain window, even
  // width) or single pixels at clamped coordinates.
  const int ncw = kFstRows + 1;  // staged columns incl. the even-rounding one (58)
  auto load_window = [&](const uint16_t* F, const StageGeom& gm, unsigned short (&pf)[kPfRows],
                         unsigned (&pf2)[kPf2Rows]) {
    if (gm.plain && pairs) {
      const unsigned* F2 = reinterpret_cast<const unsigned*>(F + (size_t)gm.r0 * W + gm.c0e);
#pragma unroll
      for (int k = 0; k < kPf2Rows; ++k) {
        const int r = pr2 + 16 * k;
        pf2[k] = (r < kFstRows && 2 * pc2 < ncw) ? __ldg(F2 + (size_t)r * (W >> 1) + pc2) : 0u;
      }
    } else {
      const int cc = min(max(gm.c0 + pc, 0), W - 1);
#pragma unroll
      for (int k = 0; k < kPfRows; ++k) {
        const int r = pr + 8 * k;
        const int rr = min(max(gm.r0 + r, 0), H - 1);
        pf[k] = (r < kFstRows && pc < kFstRows) ? __ldg(F + (size_t)rr * W + cc) : (unsigned short)0;
      }
    }
  };
  auto store_window = [&](const StageGeom& gm, const unsigned short (&pf)[kPfRows],
                          const unsigned (&pf2)[kPf2Rows]) {
    if (gm.plain && pairs) {
#pragma unroll
      for (int k = 0; k < kPf2Rows; ++k) {
        const int r = pr2 + 16 * k;
        if (r < kFstRows && 2 * pc2 < ncw) reinterpret_cast<unsigned*>(fst + r * kFst)[pc2] = pf2[k];
      }
    } else {
#pragma unroll
      for (int k = 0; k < kPfRows; ++k) {
        const int r = pr + 8 * k;
        if (r < kFstRows && pc < kFstRows) fst[r * kFst + pc] = pf[k];
      }
    }
  };

  // Stage the slot's first frame (blocking).
  StageGeom gcur = geom_of(0);
  {
    unsigned short pf0[kPfRows];
    unsigned pf20[kPf2Rows];
    load_window(frame_ptr(s0), gcur, pf0, pf20);
    store_window(gcur, pf0, pf20);
  }
  __syncthreads();

  for (int fi = 0; fi < nfr; ++fi) {
    const long long t = s0 + fi;
    // 0. issue the next frame's loads now; they land while this frame computes
    const bool more = fi + 1 < nfr;
    StageGeom gnext = gcur;
    unsigned short pf[kPfRows];
    unsigned pf2[kPf2Rows];
    if (more) {
      gnext = geom_of(fi + 1);
      load_window(frame_ptr(t + 1), gnext, pf, pf2);
    }
    // 1. resample the tile + halo from the staged frame: source (r, c) = tile
    // coordinate relative to the window origin, constant weights
    {
      const float fy = gcur.sy.f, fx = gcur.sx.f;
      const int ox = gcur.c0 - gcur.c0e;  // 0, or 1 after the even rounding
      if (tid < kExt * 8) {
        const int ry = tid >> 3, c0 = (tid & 7) * 7;
        const unsigned short* top = fst + ry * kFst + c0 + ox;
        const unsigned short* bot = top + kFst;
        float tp[8], bt[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          tp[k] = top[k];
          bt[k] = bot[k];
        }
#pragma unroll
        for (int k = 0; k < 7; ++k) {
          const float u = fmaf(fx, tp[k + 1] - tp[k], tp[k]);
          const float d = fmaf(fx, bt[k + 1] - bt[k], bt[k]);
          vext[ry * kExt + c0 + k] = fmaf(fy, d - u, u);
        }
      }
    }
    __syncthreads();
    // halo rows, then halo columns, outside the image: the value at the mirrored
    // coordinate (always an in-image row or column of the extended tile for the
    // 12 pixels that in-image outputs read; farther ones feed only outputs
    // outside the image and are left as they are)
    if (mirror_rows) {
      // ext rows [0, nt) above the image and [kExt - nb, kExt) below it
      const int nt = max(0, kGaussMaxRadius - ty0), nb = max(0, ty0 + kTile + kGaussMaxRadius - H);
      for (int i = tid; i < (nt + nb) * kExt; i += kTempThreads) {
        const int k = i / kExt, rx = i - k * kExt;
        const int ry = k < nt ? k : kExt - nb + (k - nt);
        const int rs = mirror_idx(ty0 - kGaussMaxRadius + ry, H) - (ty0 - kGaussMaxRadius);
        if (rs >= 0 && rs < kExt) vext[ry * kExt + rx] = vext[rs * kExt + rx];
      }
      __syncthreads();
    }
    if (mirror_cols) {
      const int nl = max(0, kGaussMaxRadius - tx0), nr = max(0, tx0 + kTile + kGaussMaxRadius - W);
      for (int i = tid; i < (nl + nr) * kExt; i += kTempThreads) {
        const int k = i / kExt, ry = i - k * kExt;
        const int rx = k < nl ? k : kExt - nr + (k - nl);
        const int cs = mirror_idx(tx0 - kGaussMaxRadius + rx, W) - (tx0 - kGaussMaxRadius);
        if (cs >= 0 && cs < kExt) vext[ry * kExt + rx] = vext[ry * kExt + cs];
      }
      __syncthreads();
    }
    const float v_a = vext[(ly0 + kGaussMaxRadius) * kExt + lx + kGaussMaxRadius];
    const float v_b = vext[(ly0 + 1 + kGaussMaxRadius) * kExt + lx + kGaussMaxRadius];
    // 2. corrected (or high-passed) output of frames new to this call
    if (t >= src.t_new && a.corrected) {
      float* out = a.corrected + (size_t)(t - src.t_new) * HW;
      float o_a = v_a, o_b = v_b;
      if (do_hp) {
        if (!hp_init) {
          // running sum of v[t-1] .. v[t-W+1] (v[t<0] := v[0])
          for (int k = 1; k < a.hp_w; ++k) {
            const long long u = t - k < 0 ? 0 : t - k;
            const uint16_t* Fu;
            Split uy, ux;
            frame_at(src, u, Fu, uy, ux, HW);
            if (va) hs_a += hp_q(bilin(Fu, H, W, ya, x, uy, ux));
            if (vb) hs_b += hp_q(bilin(Fu, H, W, yb, x, uy, ux));
          }
          hp_init = true;
        }
        const long long qa = hp_q(v_a), qb = hp_q(v_b);
        hs_a += qa;
        hs_b += qb;
        o_a = (float)(qa * a.hp_w - hs_a) * hp_inv;
        o_b = (float)(qb * a.hp_w - hs_b) * hp_inv;
        // drop v[t-W+1] for the next frame
        const long long u0 = t - a.hp_w + 1, u = u0 < 0 ? 0 : u0;
        const uint16_t* Fu;
        Split uy, ux;
        frame_at(src, u, Fu, uy, ux, HW);
        if (va) hs_a -= hp_q(bilin(Fu, H, W, ya, x, uy, ux));
        if (vb) hs_b -= hp_q(bilin(Fu, H, W, yb, x, uy, ux));
      }
      if (va) out[(size_t)ya * W + x] = o_a;
      if (vb) out[(size_t)yb * W + x] = o_b;
    }
    // 2b. voltage traces of frames new to this call (V, never the high-pass)
    if (roi_warp && t >= src.t_new)
      roi_add(roi_pa ? __ldg(roi_pa) : 0ull, roi_pb ? __ldg(roi_pb) : 0ull, v_a, v_b,
              a.roi_acc + (size_t)(t - src.t_new) * a.n_rois);
    // 3. row pass of the Gaussian: 56 rows x 8 groups of 4 output columns
    if (tid < kExt * 8) {
      const int r = tid >> 3, cg = tid & 7;
      const float* in = vext + r * kExt + cg * 4;
      float v[kTaps + 3];
#pragma unroll
      for (int i = 0; i < kTaps + 3; i += 4) {
        const float4 q = *reinterpret_cast<const float4*>(in + i);
        v[i] = q.x, v[i + 1] = q.y, v[i + 2] = q.z, v[i + 3] = q.w;
      }
      float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int m = 0; m < kTaps; ++m)
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = fmaf(w[m], v[j + m], o[j]);
      *reinterpret_cast<float4*>(hbuf + r * kTile + cg * 4) = make_float4(o[0], o[1], o[2], o[3]);
    }
    // 4. stage the next frame (the current one was consumed before the barrier)
    if (more) {
      store_window(gnext, pf, pf2);
      gcur = gnext;
    }
    __syncthreads();
    // 5. column pass: two output rows per thread, then the segment accumulators
    float col[kTaps + 1];
#pragma unroll
    for (int k = 0; k < kTaps + 1; ++k) col[k] = hbuf[(ly0 + k) * kTile + lx];
    // even and odd taps in separate chains (four independent FMA chains per thread)
    float b_a = 0.f, b_b = 0.f, c_a = 0.f, c_b = 0.f;
#pragma unroll
    for (int m = 0; m + 1 < kTaps; m += 2) {
      b_a = fmaf(w[m], col[m], b_a);
      b_b = fmaf(w[m], col[m + 1], b_b);
      c_a = fmaf(w[m + 1], col[m + 1], c_a);
      c_b = fmaf(w[m + 1], col[m + 2], c_b);
    }
    b_a = fmaf(w[kTaps - 1], col[kTaps - 1], b_a) + c_a;
    b_b = fmaf(w[kTaps - 1], col[kTaps], b_b) + c_b;
    sum_a += v_a;
    sum_b += v_b;
    mx_a = fmaxf(mx_a, b_a);
    mx_b = fmaxf(mx_b, b_b);
    float* hrow = hist + (size_t)fi * (kTile * kTile) + ly0 * kTile + lx;
    hrow[0] = b_a;
    hrow[kTile] = b_b;
  }
  if (!complete || !a.summary) return;
  float* S = a.summary + (size_t)slot * 2 * HW;
  float* T = S + HW;
  const float invL = 1.0f / (float)L;
  for (int q = 0; q < 2; ++q) {
    const bool ok = q == 0 ? va : vb;
    if (!ok) continue;
    const int y = q == 0 ? ya : yb;
    const float* h = hist + (ly0 + q) * kTile + lx;
    const float med = L == 50 ? median50(h, kTile * kTile) : median_any(h, kTile * kTile, L);
    S[(size_t)y * W + x] = (q == 0 ? sum_a : sum_b) * invL;
    T[(size_t)y * W + x] = (q == 0 ? mx_a : mx_b) - med;
  }
}

static size_t temporal_smem(int L) {
  return sizeof(float) * ((size_t)kExt * kExt + (size_t)kExt * kTile + (size_t)L * kTile * kTile +
                          2 * kMaxL) +
         sizeof(unsigned short) * (kFstRows * kFst);
}



// ---- the fused pass with the segment history in tensor memory -------------------
// Same arithmetic as k_temporal (corrected frames and T_i bit for bit; S_i adds
// the frames in two interleaved partial sums), for launches without the
// high-pass output, widths that are multiples of 8 and 16-byte aligned frame
// buffers.  A CTA still owns one 32x32 output tile for one segment slot, but:
//   * the segment's smoothed history (up to 50 frames x 1,024 pixels) lives in
//     the SM's tensor memory (128 lanes x 512 columns) instead of 200 KB of
//     shared memory;
//   * four groups of 4 warps take every fourth frame, each with its own
//     buffers and named barrier, so that some groups compute while others wait;
//   * each frame's 57 x 64 source window arrives as one TMA box (3-D map over
//     [frames][H][W]) in a double buffer per group, two of the group's frames
//     ahead; samples outside the image are read at clamped indices of the
//     window (the clamped coordinates of the resampling).
// Work of a group per frame: its 4 warps resample (7 rows x 2 columns per thread
// and chunk, two chunks), run the row pass (one row x 16 columns per thread) and
// the column pass (4 rows of one column per thread and job, two jobs), keep the
// smoothed history, store the corrected pixels and add the traces and segment
// sums.  Thread (w, lane) owns the 8 pixels at rows 4 w + i and 4 (w + 4) + i,
// column lane (i < 4) -- the same pixels in every group.
// Tensor memory: warp w (0..3) of a group reaches lanes 32 w .. +31; pixel q =
// 4 j + i (job j) of a thread keeps its smoothed value of segment frame t at
// column 64 q + t, whichever group smoothed that frame.  At the segment's end
// the groups share out the 8 pixels of every thread for the median and the
// maximum.
constexpr int kTmGroups = 6, kTmGroup = 128, kTmThreads = kTmGroups * kTmGroup;
constexpr int kStCols = 64, kStRows = kFstRows;       // source window of one frame (uint16)
constexpr int kStBytes = kStCols * kStRows * 2;        // 7,296 B: one TMA box
constexpr int kStStride = 7424;                        // stage buffer pitch (128-byte multiple)
constexpr int kVS = 60;   // resampled-tile row stride: 128-bit row-pass loads without conflicts
constexpr int kHS = 36;   // row-pass output row stride: 128-bit stores without conflicts
constexpr int kTmCols = 512;
constexpr size_t kTmSmemUsed = 2 * kTmGroups * (size_t)kStStride +
                               sizeof(float) * (kTmGroups * (size_t)kExt * (kVS + kHS) + 2 * kMaxL) +
                               (sizeof(float2) + 2 * sizeof(int4)) * kMaxL;
// Shared memory requested per CTA (the layout plus 128 bytes to align its start):
// more than half of the SM's, so that one CTA (which holds all of the SM's
// tensor memory) runs per SM.
constexpr size_t kTmSmem = kTmSmemUsed + 128 > 120 * 1024 ? kTmSmemUsed + 128 : 120 * 1024;
static_assert(kTmGroups * 8 * kTmGroup * sizeof(float) <= kTmGroups * sizeof(float) * kExt * kVS,
              "partial-sum exchange fits the resampled-tile buffers");
static_assert(kTmSmemUsed + 128 <= 227 * 1024, "shared memory of the tensor-memory temporal kernel");

struct TemporalMaps {
  CUtensorMap m[kMaxVideos][2];  // per job: [0] carry buffer, [1] caller's batch
};

// Gaussian taps shared by every job of a launch: a kernel parameter read at
// fixed offsets, so the FMAs take them straight from the constant bank.
struct TemporalTaps {
  float w[2 * kGaussMaxRadius + 1];
};

__device__ __forceinline__ void group_bar(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kTmGroup) : "memory");
}

// Group barrier that also returns the OR of `v` over the group's threads.
__device__ __forceinline__ bool group_bar_or(int id, bool v) {
  int r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.s32 p, %1, 0;\nbar.red.or.pred q, %2, %3, p;\nselp.s32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((int)v), "r"(id), "r"(kTmGroup)
      : "memory");
  return r != 0;
}

// 2^23 + u for one uint16 half u of a 32-bit word, exactly: the byte permute
// builds its bits.  Subtracting 2^23, or another such value, is exact.
__device__ __forceinline__ float u16m(unsigned w, unsigned sel) {
  return __uint_as_float(__byte_perm(w, 0x4B000000u, sel));
}
constexpr unsigned kSelLo = 0x7410u, kSelHi = 0x7432u;

// Source window of frame fi for a tile: rows r0 .. r0 + 56 and columns c0e ..
// c0e + 63, c0e = the window's first column rounded down to a multiple of 8
// (TMA boxes start on 16-byte boundaries), ox = the remainder.  Of the window,
// rows [top, bot) and columns [left, right) lie inside the image; a sample
// outside takes the value at the clamped position (the resampling's clamped
// coordinates), so the window is read at clamped indices and the zeros that
// the TMA writes outside the image are never used.
struct WinGeom {
  float fy, fx;
  int r0, c0e, ox, top, bot, left, right;
  bool meets;    // the window overlaps the image (TMA); else filled by plain loads
  bool rows_in;  // no row clamping needed
  bool cols_in;  // the columns the resampling reads lie inside the image
};

__device__ __forceinline__ WinGeom win_geom(const float* shs, int fi, int ty0, int tx0, int H,
                                            int W) {
  // shifts beyond +-2^20 px resample to the same edge pixels; bounding them
  // keeps the integer arithmetic in range
  const float sy = fminf(fmaxf(shs[2 * fi], -1048576.f), 1048576.f);
  const float sx = fminf(fmaxf(shs[2 * fi + 1], -1048576.f), 1048576.f);
  const Split a = split_shift(sy), b = split_shift(sx);
  WinGeom g;
  g.fy = a.f;
  g.fx = b.f;
  g.r0 = ty0 - kGaussMaxRadius + a.i;
  const int c0 = tx0 - kGaussMaxRadius + b.i;
  g.c0e = c0 & ~7;
  g.ox = c0 - g.c0e;
  g.meets = g.r0 + kStRows - 1 >= 0 && g.r0 <= H - 1 && g.c0e + kStCols - 1 >= 0 && g.c0e <= W - 1;
  g.top = min(kStRows - 1, max(0, -g.r0));
  g.bot = max(g.top + 1, min(kStRows, H - g.r0));
  g.left = min(kStCols - 1, max(0, -g.c0e));
  g.right = max(g.left + 1, min(kStCols, W - g.c0e));
  // a window that misses the image is filled at clamped coordinates already
  g.rows_in = !g.meets || (g.top == 0 && g.bot == kStRows);
  g.cols_in = !g.meets || (g.ox >= g.left && g.ox + kExt + 1 <= g.right);
  return g;
}

// Resampling of the tile + halo, one warp per 7 output rows, lane p < 28 = the
// output columns 2p, 2p + 1 (same formula and order as k_temporal: lerp along x
// on each source row, then along y).  Each source row's lerps feed two output
// rows.  kRowClamp: source rows read at clamped indices.
// Contiguous form: the two columns' three samples per row are two 32-bit words.
template <bool kRowClamp>
__device__ __forceinline__ void resample_words(const unsigned short* st16, float* vext, int kc,
                                               int p, int ox, float fy, float fx, int top,
                                               int bot) {
  const unsigned* sw = reinterpret_cast<const unsigned*>(st16) + ((2 * p + ox) >> 1);
  const bool odd = ox & 1;
  const unsigned sa = odd ? kSelHi : kSelLo, sb = odd ? kSelLo : kSelHi;
  float* vo = vext + kc * 7 * kVS + 2 * p;
  float ph0 = 0.f, ph1 = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    int r = kc * 7 + j;
    if (kRowClamp) r = min(max(r, top), bot - 1);
    const unsigned w0 = sw[r * (kStCols / 2)], w1 = sw[r * (kStCols / 2) + 1];
    // 2^23 + u of the three samples; differences of these are exact
    const float ma = u16m(w0, sa), mb = u16m(odd ? w1 : w0, sb), mc = u16m(w1, sa);
    const float va = ma - 8388608.0f, vb = mb - 8388608.0f;
    const float h0 = fmaf(fx, mb - ma, va), h1 = fmaf(fx, mc - mb, vb);
    if (j > 0)
      *reinterpret_cast<float2*>(vo + (j - 1) * kVS) =
          make_float2(fmaf(fy, h0 - ph0, ph0), fmaf(fy, h1 - ph1, ph1));
    ph0 = h0;
    ph1 = h1;
  }
}

// General form: output column 2p + e reads window columns s[e][0], s[e][1]
// (mirrored at the image border for the Gaussian's halo, clamped to the image).
template <bool kRowClamp>
__device__ __forceinline__ void resample_cols(const unsigned short* st16, float* vext, int kc,
                                              int p, const int (&s)[2][2], float fy, float fx,
                                              int top, int bot) {
  float* vo = vext + kc * 7 * kVS + 2 * p;
  float ph0 = 0.f, ph1 = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    int r = kc * 7 + j;
    if (kRowClamp) r = min(max(r, top), bot - 1);
    const unsigned short* row = st16 + r * kStCols;
    const float a0 = __uint_as_float(0x4B000000u | row[s[0][0]]) - 8388608.0f;
    const float b0 = __uint_as_float(0x4B000000u | row[s[0][1]]) - 8388608.0f;
    const float a1 = __uint_as_float(0x4B000000u | row[s[1][0]]) - 8388608.0f;
    const float b1 = __uint_as_float(0x4B000000u | row[s[1][1]]) - 8388608.0f;
    const float h0 = fmaf(fx, b0 - a0, a0), h1 = fmaf(fx, b1 - a1, a1);
    if (j > 0)
      *reinterpret_cast<float2*>(vo + (j - 1) * kVS) =
          make_float2(fmaf(fy, h0 - ph0, ph0), fmaf(fy, h1 - ph1, ph1));
    ph0 = h0;
    ph1 = h1;
  }
}

// Tile coordinate of the in-image position mirrored at the border ("d c b a |
// a b c d"); positions that only feed outputs outside the image stay in the tile.
__device__ __forceinline__ int mirror_local(int i, int o, int n) {
  return min(max(mirror_idx(o + i, n) - o, 0), kExt - 1);
}

__global__ void __launch_bounds__(kTmThreads, 1)
    k_temporal_tm(const __grid_constant__ TemporalBatch b, const __grid_constant__ TemporalMaps maps,
                  const __grid_constant__ TemporalTaps taps) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kTmGroups][2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_any;
  // TMA destinations start on 128-byte boundaries: the dynamic region is
  // aligned here (the launch requests 128 bytes more than the layout needs)
  unsigned char* smraw = smem_raw + ((128u - (tc::su32(smem_raw) & 127u)) & 127u);
  const int jb = job_of(b.begin, b.n, blockIdx.x);
  const TemporalArgs& a = b.a[jb];
  const int H = a.H, W = a.W, L = a.L, HW = H * W;
  const int ntx = (W + kTile - 1) / kTile, tiles = ntx * ((H + kTile - 1) / kTile);
  const int local = blockIdx.x - b.begin[jb];
  const int slot = local / tiles, tile = local - slot * tiles;
  const int ty0 = (tile / ntx) * kTile, tx0 = (tile % ntx) * kTile;
  const int tid = threadIdx.x, grp = tid / kTmGroup, gt = tid % kTmGroup, wg = gt >> 5;
  const int lane = tid & 31, bar_id = 1 + grp;
  unsigned char* stage = smraw + grp * 2 * kStStride;  // [2][kStStride] this group's windows
  float* fbase = reinterpret_cast<float*>(smraw + 2 * kTmGroups * kStStride);
  float* vext = fbase + grp * (kExt * kVS);                            // [56][kVS] tile + halo
  float* hbuf = fbase + kTmGroups * kExt * kVS + grp * (kExt * kHS);   // [56][kHS] row-smoothed
  float* shs = fbase + kTmGroups * kExt * (kVS + kHS);                 // [L][2] shifts of the slot
  float2* geo_f = reinterpret_cast<float2*>(shs + 2 * kMaxL);  // [L] (fy, fx)
  int4* geo_i = reinterpret_cast<int4*>(geo_f + kMaxL);         // [L] (r0, c0e, ox, flags)
  int4* geo_b = geo_i + kMaxL;                                  // [L] (top, bot, left, right)
  const FrameSource& src = a.src;
  const long long t_end = src.t_first + src.n_carry + src.n_batch;
  const long long s0 = a.seg_base + (long long)slot * L;
  const long long s1 = s0 + L < t_end ? s0 + L : t_end;
  const int nfr = (int)(s1 - s0);
  const bool complete = s0 + L <= t_end;

  if (tid < 32) tc::tmem_alloc(&tmem_slot, kTmCols);
  if (tid == 0) {
    for (int g = 0; g < kTmGroups; ++g)
      for (int k = 0; k < 2; ++k) tc::mbar_init(&full[g][k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_any = 0;
  }
  for (int i = tid; i < 2 * nfr; i += kTmThreads) {
    const long long v = s0 + (i >> 1) - src.t_first;
    shs[i] = v < src.n_carry ? src.carry_shift[2 * v + (i & 1)]
                             : src.batch_shift[2 * (v - src.n_carry) + (i & 1)];
  }
  __syncthreads();
  if (tid < nfr) {  // source-window geometry of every frame of the slot, once
    const WinGeom g = win_geom(shs, tid, ty0, tx0, H, W);
    geo_f[tid] = make_float2(g.fy, g.fx);
    geo_i[tid] = make_int4(g.r0, g.c0e, g.ox,
                           (g.meets ? 1 : 0) | (g.rows_in ? 2 : 0) | (g.cols_in ? 4 : 0));
    geo_b[tid] = make_int4(g.top, g.bot, g.left, g.right);
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tlane = tmem_slot + ((uint32_t)(32 * wg) << 16);
  const float* w = taps.w;

  // this thread's 8 pixels: rows yb + 16 j + i (job j, i < 4), column x
  const int x = tx0 + lane, yb = ty0 + 4 * wg;
  const bool xin = x < W;
  bool myroi = false;
  if (a.roi_acc && xin)
    for (int q = 0; q < 8; ++q) {
      const int y = yb + 16 * (q >> 2) + (q & 3);
      if (y < H && __ldg(a.roi_members + (size_t)y * W + x)) myroi = true;
    }
  const bool roi_warp = __any_sync(0xffffffffu, myroi);
  // the Gaussian's mirrored halo: the row pass reads mirrored rows, and the
  // resampling computes halo columns at their mirrored positions
  const bool mirror_rows = ty0 - kGaussMaxRadius < 0 || ty0 + kTile + kGaussMaxRadius > H;
  const bool mirror_cols = tx0 - kGaussMaxRadius < 0 || tx0 + kTile + kGaussMaxRadius > W;
  const int oy = ty0 - kGaussMaxRadius, oxt = tx0 - kGaussMaxRadius;
  const int rp_row = gt >> 1;  // row-pass row of this thread (gt < 112)
  const int rp_src = mirror_rows ? mirror_local(rp_row, oy, H) : rp_row;
  const int cm0 = mirror_cols ? mirror_local(2 * lane, oxt, W) : 2 * lane;
  const int cm1 = mirror_cols ? mirror_local(2 * lane + 1, oxt, W) : 2 * lane + 1;

  // frames grp, grp + 4, ... of the slot; the k-th goes to buffer k mod 2
  const int nmine = nfr > grp ? (nfr - grp + kTmGroups - 1) / kTmGroups : 0;
  // TMA of frame fi's window into buffer buf (windows that miss the image are
  // filled by plain loads when consumed); returns whether a copy was issued
  auto issue = [&](int fi, int buf) -> bool {
    const int4 gi = geo_i[fi];
    if (!(gi.w & 1)) return false;
    const long long v = s0 + fi - src.t_first;
    const int which = v < src.n_carry ? 0 : 1;
    const int z = (int)(which ? v - src.n_carry : v);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc::mbar_expect_tx(&full[grp][buf], kStBytes);
    tc::tma_load_3d(stage + buf * kStStride, &maps.m[jb][which], gi.y, gi.x, z, &full[grp][buf]);
    return true;
  };
  uint32_t pending = 0;  // (thread gt == 0) buffers with a copy in flight
  if (gt == 0)
    for (int k = 0; k < 2 && k < nmine; ++k)
      if (issue(grp + kTmGroups * k, k)) pending |= 1u << k;
  float* const obase = a.corrected ? a.corrected + (size_t)yb * W + x : nullptr;

  float sm[8];  // sums of V over this group's frames
#pragma unroll
  for (int q = 0; q < 8; ++q) sm[q] = 0.f;
  uint32_t phase = 0;  // bit k: parity of buffer k's next completion
  bool aborted = false;
  for (int k = 0; k < nmine; ++k) {
    const int fi = grp + kTmGroups * k, buf = k & 1;
    const long long t = s0 + fi;
    const float2 gf = geo_f[fi];
    const int4 gi = geo_i[fi];
    const int r0 = gi.x, c0e = gi.y, ox = gi.z;
    const bool meets = gi.w & 1, rows_in = gi.w & 2, cols_in = gi.w & 4;
    unsigned short* st16 = reinterpret_cast<unsigned short*>(stage + buf * kStStride);
    bool late = false;
    if (meets) {
      late = !tc::mbar_wait_short(&full[grp][buf], (phase >> buf) & 1);
      phase ^= 1u << buf;
      if (gt == 0 && !late) pending &= ~(1u << buf);
    }
    if (group_bar_or(bar_id, late)) {
      aborted = true;
      break;
    }
    if (!meets) {
      // the window misses the image: every sample is an edge pixel of the frame
      const long long v = t - src.t_first;
      const uint16_t* F = v < src.n_carry ? src.carry + (size_t)v * HW
                                          : src.batch + (size_t)(v - src.n_carry) * HW;
      for (int i = gt; i < kStRows * kStCols; i += kTmGroup) {
        const int r = i >> 6, c = i & 63;
        const int rr = min(max(r0 + r, 0), H - 1), cc = min(max(c0e + c, 0), W - 1);
        st16[i] = __ldg(F + (size_t)rr * W + cc);
      }
      group_bar(bar_id);
    }
    // 1. resample the tile + halo into vext: warp w takes the 7-row chunks w and
    //    w + 4, lane p < 28 the columns 2p, 2p + 1
    if (lane < 28) {
#pragma unroll 1
      for (int ch = wg; ch < 8; ch += 4) {
        if (cols_in && !mirror_cols) {
          if (rows_in)
            resample_words<false>(st16, vext, ch, lane, ox, gf.x, gf.y, 0, kStRows);
          else {
            const int4 gb = geo_b[fi];
            resample_words<true>(st16, vext, ch, lane, ox, gf.x, gf.y, gb.x, gb.y);
          }
        } else {
          const int4 gb = geo_b[fi];
          int sc[2][2];
          sc[0][0] = min(max(cm0 + ox, gb.z), gb.w - 1);
          sc[0][1] = min(max(cm0 + ox + 1, gb.z), gb.w - 1);
          sc[1][0] = min(max(cm1 + ox, gb.z), gb.w - 1);
          sc[1][1] = min(max(cm1 + ox + 1, gb.z), gb.w - 1);
          if (rows_in)
            resample_cols<false>(st16, vext, ch, lane, sc, gf.x, gf.y, 0, kStRows);
          else
            resample_cols<true>(st16, vext, ch, lane, sc, gf.x, gf.y, gb.x, gb.y);
        }
      }
    }
    group_bar(bar_id);  // window consumed, tile resampled
    if (gt == 0 && k + 2 < nmine && issue(fi + 2 * kTmGroups, buf)) pending |= 1u << buf;
    float v[8];  // V of the thread's 8 pixels
#pragma unroll
    for (int q = 0; q < 8; ++q)
      v[q] = vext[(kGaussMaxRadius + 4 * wg + 16 * (q >> 2) + (q & 3)) * kVS + kGaussMaxRadius + lane];
    // 2. row pass of the Gaussian: thread = one row x 16 output columns (halo
    //    rows outside the image read their mirrored row); each output sums its
    //    25 taps in order, as in k_temporal
    if (gt < 2 * kExt) {
      const int ch = gt & 1;
      const float* in = vext + rp_src * kVS + ch * 16;
      float xv[40];
#pragma unroll
      for (int i = 0; i < 40; i += 4) {
        const float4 q = *reinterpret_cast<const float4*>(in + i);
        xv[i] = q.x, xv[i + 1] = q.y, xv[i + 2] = q.z, xv[i + 3] = q.w;
      }
      float o[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) o[j] = 0.f;
#pragma unroll
      for (int m = 0; m < kTaps; ++m)
#pragma unroll
        for (int j = 0; j < 16; ++j) o[j] = fmaf(w[m], xv[j + m], o[j]);
      float* out = hbuf + rp_row * kHS + ch * 16;
#pragma unroll
      for (int j = 0; j < 16; j += 4)
        *reinterpret_cast<float4*>(out + j) = make_float4(o[j], o[j + 1], o[j + 2], o[j + 3]);
    }
    group_bar(bar_id);
    // 3. column pass: two jobs of 4 output rows of one column, each output in
    //    two chains (even and odd taps) as in k_temporal; the smoothed history
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      float col[kTaps + 3];
#pragma unroll
      for (int kk = 0; kk < kTaps + 3; ++kk)
        col[kk] = hbuf[(4 * wg + 16 * j + kk) * kHS + lane];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float be = 0.f, bo = 0.f;
#pragma unroll
        for (int m = 0; m + 1 < kTaps; m += 2) {
          be = fmaf(w[m], col[i + m], be);
          bo = fmaf(w[m + 1], col[i + m + 1], bo);
        }
        const float vb = fmaf(w[kTaps - 1], col[i + kTaps - 1], be) + bo;
        tc::tmem_st1(tlane + (uint32_t)(64 * (4 * j + i) + fi), vb);
      }
    }
    // 4. outputs of frames new to this call, traces, segment sums
    const bool fresh = t >= src.t_new;
    if (fresh && obase && xin) {
      float* out = obase + (size_t)(t - src.t_new) * HW;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int dy = 16 * (q >> 2) + (q & 3);
        if (yb + dy < H) out[(size_t)dy * W] = v[q];
      }
    }
    if (roi_warp && fresh) {
      unsigned long long* racc = a.roi_acc + (size_t)(t - src.t_new) * a.n_rois;
#pragma unroll
      for (int q = 0; q < 8; q += 2) {
        const int dy = 16 * (q >> 2) + (q & 3);
        const unsigned long long* mrow = a.roi_members + (size_t)(yb + dy) * W + x;
        roi_add(xin && yb + dy < H ? __ldg(mrow) : 0ull,
                xin && yb + dy + 1 < H ? __ldg(mrow + W) : 0ull, v[q], v[q + 1], racc);
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) sm[q] += v[q];
    tc::tmem_wait_st();
  }
  if (aborted) {
    if (gt == 0) {
      if (a.err) atomicExch(a.err, 1);
      abort_any = 1;
      // wait (bounded) for this group's copies still in flight
      for (int bb = 0; bb < 2; ++bb)
        if (pending & (1u << bb)) tc::mbar_wait(&full[grp][bb], (phase >> bb) & 1);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (complete && a.summary && !abort_any) {
    // each group's partial sums over its frames; the groups share out the 8
    // pixels of every thread (pixel q goes to group q mod 6) and add the
    // partial sums in group order; maximum and median come from the history
    float* xs = fbase;  // [group][pixel 0..7][128]
#pragma unroll
    for (int q = 0; q < 8; ++q) xs[(grp * 8 + q) * kTmGroup + gt] = sm[q];
    __syncthreads();
    float* S = a.summary + (size_t)slot * 2 * HW;
    float* T = S + HW;
    const float invL = 1.0f / (float)L;
    for (int q = grp; q < 8; q += kTmGroups) {
      const int y = yb + 16 * (q >> 2) + (q & 3);
      float st = 0.f;
#pragma unroll
      for (int g = 0; g < kTmGroups; ++g) st += xs[(g * 8 + q) * kTmGroup + gt];
      const uint32_t ta = tlane + (uint32_t)(64 * q);
      uint32_t r0[16], r1[16], r2[16], r3[2];
      tc::tmem_ld16_nowait(ta, r0);
      tc::tmem_ld16_nowait(ta + 16, r1);
      tc::tmem_ld16_nowait(ta + 32, r2);
      tc::tmem_ld2_nowait(ta + 48, r3);
      tc::tmem_wait_ld();
      float h[50];
#pragma unroll
      for (int z = 0; z < 16; ++z) {
        h[z] = __uint_as_float(r0[z]);
        h[16 + z] = __uint_as_float(r1[z]);
        h[32 + z] = __uint_as_float(r2[z]);
      }
      h[48] = __uint_as_float(r3[0]);
      h[49] = __uint_as_float(r3[1]);
      float mt;
      const float med = L == 50 ? median50_v(h, &mt) : median_any_v(h, L, &mt);
      if (y < H && xin) {
        S[(size_t)y * W + x] = st * invL;
        T[(size_t)y * W + x] = mt - med;
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (tid < 32) tc::tmem_dealloc(tmem_slot, kTmCols);
}

// TMA map of a uint16 frame buffer [n][H][W]: boxes of 64 columns x 57 rows x 1
// frame; coordinates outside the buffer read zeros.
static bool tm_frame_map(CUtensorMap* m, const uint16_t* base, int n, int H, int W) {
  tc::EncodeTiledFn fn = tc::encode_fn();
  if (!fn || !base) return false;
  cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)(n > 0 ? n : 1)};
  cuuint64_t strides[2] = {(cuuint64_t)W * 2, (cuuint64_t)H * W * 2};
  cuuint32_t box[3] = {(cuuint32_t)kStCols, (cuuint32_t)kStRows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<uint16_t*>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The tensor-memory kernel applies: no high-pass output, W a multiple of 8 (rows
// on 16-byte boundaries), 16-byte aligned frame buffers, an 8-byte aligned
// corrected output (pixel pairs are stored together), and not switched off.
static bool tm_applies(const TemporalArgs& a) {
  const bool hp = a.out_hp && a.hp_w > 0 && a.corrected;
  const uintptr_t bb = reinterpret_cast<uintptr_t>(a.src.batch);
  const uintptr_t cb = reinterpret_cast<uintptr_t>(a.src.carry);
  const uintptr_t ob = reinterpret_cast<uintptr_t>(a.corrected);
  return !a.smem_history && !hp && a.W % 8 == 0 && a.src.n_batch > 0 && bb && (bb & 15) == 0 &&
         (a.src.n_carry == 0 || (cb && (cb & 15) == 0)) && (ob & 7) == 0;
}

// ---- voltage-trace ROIs ----------------------------------------------------------
// One thread per pixel: the ids (+1) of the ROIs containing it, in increasing
// order, packed into four 16-bit fields; per-ROI pixel counts.
__global__ void k_roi_build(const uint8_t* __restrict__ masks, int n_rois, int HW,
                            unsigned long long* __restrict__ members, int* __restrict__ counts,
                            int* __restrict__ too_many) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
    unsigned long long m = 0;
    int k = 0;
    for (int r = 0; r < n_rois; ++r) {
      if (!masks[(size_t)r * HW + p]) continue;
      atomicAdd(counts + r, 1);
      if (k < 4)
        m |= (unsigned long long)(r + 1) << (16 * k);
      else
        atomicExch(too_many, 1);
      ++k;
    }
    members[p] = m;
  }
}

__global__ void k_roi_finalize(const unsigned long long* __restrict__ acc,
                               const int* __restrict__ counts, long long total, int n_rois,
                               float* __restrict__ traces) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = counts[i % n_rois];
    traces[i] = c > 0 ? (float)((double)(long long)acc[i] / (kRoiFix * (double)c)) : 0.0f;
  }
}

cudaError_t roi_build(const uint8_t* masks, int n_rois, int H, int W, unsigned long long* members,
                      int* counts, int* too_many, cudaStream_t st) {
  const int HW = H * W;
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)(n_rois > 0 ? n_rois : 1), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(too_many, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const int blocks = (HW + 255) / 256 < 4096 ? (HW + 255) / 256 : 4096;
  k_roi_build<<<blocks, 256, 0, st>>>(masks, n_rois, HW, members, counts, too_many);
  return cudaGetLastError();
}

cudaError_t roi_finalize(const unsigned long long* acc, const int* counts, int nf, int n_rois,
                         float* traces, cudaStream_t st) {
  const long long total = (long long)nf * n_rois;
  if (total <= 0) return cudaSuccess;
  const long long want = (total + 255) / 256;
  const int blocks = want < 4096 ? (int)want : 4096;
  k_roi_finalize<<<blocks, 256, 0, st>>>(acc, counts, total, n_rois, traces);
  return cudaGetLastError();
}

// ---- whole-video summary images -------------------------------------------------
// VolPy's temporal average and local correlation images of V (compared in Sec.
// III-A, Fig. 2).  Per pixel, over the launch's frames: sums of d, d^2 and of d
// times its E, S, SE and SW neighbours (each unordered 8-neighbour pair once),
// d = V - T (any per-pixel constant gives the same correlation; the template
// keeps d small so that FP32 sums over one launch stay accurate), then added to
// FP64 accumulators [6][H][W].  One CTA owns a 32 x 8 output tile and walks the
// frames, 8 at a time: V of the tile plus its E/S/SW halo for 8 frames is
// resampled into shared memory in one pass, so those loads overlap.
constexpr int kVsX = 32, kVsY = 8;
constexpr int kVsF = 8;  // frames resampled per shared-memory pass (loads in flight together)

__global__ void __launch_bounds__(kVsX * kVsY) k_vsum(const uint16_t* __restrict__ frames,
                                                      const float* __restrict__ shifts, int nf,
                                                      int H, int W, const float* __restrict__ ref,
                                                      double* __restrict__ acc) {
  __shared__ float vs[kVsF][kVsY + 1][kVsX + 2];  // rows y0..y0+8, columns x0-1..x0+32
  __shared__ float rt[kVsY + 1][kVsX + 2];        // template over the same window
  __shared__ int si[kVsF][2];                      // integer parts of the shifts
  __shared__ float sf[kVsF][2];                    // fractional parts
  __shared__ int inside[kVsF];                     // source window inside the image
  const int tx = threadIdx.x % kVsX, ty = threadIdx.x / kVsX;
  const int x0 = blockIdx.x * kVsX, y0 = blockIdx.y * kVsY;
  const int x = x0 + tx, y = y0 + ty;
  const bool in = x < W && y < H;
  const bool hasE = x + 1 < W, hasS = y + 1 < H, hasSW = hasS && x >= 1, hasSE = hasS && hasE;
  float s1 = 0.f, s2 = 0.f, pe = 0.f, ps = 0.f, pse = 0.f, psw = 0.f;
  constexpr int nv = (kVsY + 1) * (kVsX + 2);
  for (int j = threadIdx.x; j < nv; j += blockDim.x) {
    const int ry = j / (kVsX + 2), rx = j - ry * (kVsX + 2);
    const int yy = y0 + ry, xx = x0 - 1 + rx;
    rt[ry][rx] = (yy < H && xx >= 0 && xx < W) ? __ldg(ref + (size_t)yy * W + xx) : 0.f;
  }
  for (int f0 = 0; f0 < nf; f0 += kVsF) {
    const int nb = min(kVsF, nf - f0);
    __syncthreads();  // the previous pass's values are consumed
    if (threadIdx.x < nb) {
      const Split a = split_shift(__ldg(shifts + 2 * (f0 + threadIdx.x)));
      const Split b = split_shift(__ldg(shifts + 2 * (f0 + threadIdx.x) + 1));
      si[threadIdx.x][0] = a.i, si[threadIdx.x][1] = b.i;
      sf[threadIdx.x][0] = a.f, sf[threadIdx.x][1] = b.f;
      // rows y0 + a.i .. y0 + 9 + a.i and columns x0 - 1 + b.i .. x0 + 34 + b.i in the image
      inside[threadIdx.x] = y0 + a.i >= 0 && y0 + kVsY + 1 + a.i < H && x0 - 1 + b.i >= 0 &&
                            x0 + kVsX + 1 + b.i < W;
    }
    __syncthreads();
    // unrolled so that several values' taps are in flight at once (the loop is
    // bound by L2 latency, not by arithmetic)
#pragma unroll 5
    for (int i = threadIdx.x; i < nb * nv; i += blockDim.x) {
      const int fk = i / nv, j = i - fk * nv;
      const int ry = j / (kVsX + 2), rx = j - ry * (kVsX + 2);
      const int yy = y0 + ry, xx = x0 - 1 + rx;
      float v = 0.f;
      if (yy < H && xx >= 0 && xx < W) {
        const uint16_t* F = frames + (size_t)(f0 + fk) * H * W;
        if (inside[fk]) {  // no clamping: the four taps are (yy + iy, xx + ix) and right/below
          const uint16_t* q = F + (size_t)(yy + si[fk][0]) * W + xx + si[fk][1];
          const float a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + W), d = __ldg(q + W + 1);
          const float wx = sf[fk][1], wy = sf[fk][0];
          const float top = fmaf(wx, b - a, a), bot = fmaf(wx, d - c, c);
          v = fmaf(wy, bot - top, top);
        } else {
          v = bilin(F, H, W, yy, xx, Split{si[fk][0], sf[fk][0]}, Split{si[fk][1], sf[fk][1]});
        }
        v -= rt[ry][rx];
      }
      vs[fk][ry][rx] = v;
    }
    __syncthreads();
    for (int fk = 0; fk < nb; ++fk) {
      const float d = vs[fk][ty][tx + 1];
      s1 += d;
      s2 = fmaf(d, d, s2);
      pe = fmaf(d, vs[fk][ty][tx + 2], pe);
      ps = fmaf(d, vs[fk][ty + 1][tx + 1], ps);
      pse = fmaf(d, vs[fk][ty + 1][tx + 2], pse);
      psw = fmaf(d, vs[fk][ty + 1][tx], psw);
    }
  }
  if (!in) return;
  const size_t HW = (size_t)H * W, o = (size_t)y * W + x;
  acc[o] += s1;
  acc[HW + o] += s2;
  if (hasE) acc[2 * HW + o] += pe;
  if (hasS) acc[3 * HW + o] += ps;
  if (hasSE) acc[4 * HW + o] += pse;
  if (hasSW) acc[5 * HW + o] += psw;
}

// A(x) = T(x) + S_d / n; C(x) = mean over in-image 8-neighbours of the Pearson
// correlation (0 where either trace is constant), FP64.
__global__ void k_vsum_final(const double* __restrict__ acc, const float* __restrict__ ref,
                             long long n, int H, int W, float* __restrict__ avg,
                             float* __restrict__ corr) {
  const size_t HW = (size_t)H * W;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < HW;
       o += (size_t)gridDim.x * blockDim.x) {
    const int y = (int)(o / W), x = (int)(o % W);
    const double dn = (double)n;
    auto var = [&](size_t q) {
      const double v = acc[HW + q] - acc[q] * acc[q] / dn;
      return v > 1e-9 * acc[HW + q] ? v : 0.0;  // constant traces (up to FP32 rounding)
    };
    const double vx = var(o);
    double tot = 0.0;
    int cnt = 0;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (!dy && !dx) continue;
        const int yy = y + dy, xx = x + dx;
        if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
        ++cnt;
        const size_t q = (size_t)yy * W + xx;
        // the pair's product sum is stored at its upper (or, in a row, left)
        // pixel: slot 2 = E, 3 = S, 4 = SE, 5 = SW of that pixel
        const bool here = dy > 0 || (dy == 0 && dx > 0);
        const size_t at = here ? o : q;
        const int slot = dy == 0 ? 2 : (dx == 0 ? 3 : (dx == dy ? 4 : 5));
        const double vy = var(q);
        if (vx > 0.0 && vy > 0.0) {
          const double cov = acc[slot * HW + at] - acc[o] * acc[q] / dn;
          tot += cov / sqrt(vx * vy);
        }
      }
    if (avg) avg[o] = (float)((double)__ldg(ref + o) + acc[o] / dn);
    if (corr) corr[o] = cnt ? (float)(tot / cnt) : 0.f;
  }
}

cudaError_t launch_vsum(const uint16_t* frames, const float* shifts, int nf, int H, int W,
                        const float* ref, double* acc, cudaStream_t st) {
  if (nf <= 0) return cudaSuccess;
  dim3 grid((W + kVsX - 1) / kVsX, (H + kVsY - 1) / kVsY);
  k_vsum<<<grid, kVsX * kVsY, 0, st>>>(frames, shifts, nf, H, W, ref, acc);
  return cudaGetLastError();
}

cudaError_t launch_vsum_final(const double* acc, const float* ref, long long n, int H, int W,
                              float* avg, float* corr, cudaStream_t st) {
  const size_t HW = (size_t)H * W;
  const int blocks = (int)std::min<size_t>((HW + 255) / 256, 4096);
  k_vsum_final<<<blocks, 256, 0, st>>>(acc, ref, n, H, W, avg, corr);
  return cudaGetLastError();
}

bool temporal_batch_finalize(TemporalBatch& b) {
  if (b.n < 1 || b.n > kMaxVideos) return false;
  long long s = 0;
  b.begin[0] = 0;
  for (int i = 0; i < b.n; ++i) {
    const TemporalArgs& a = b.a[i];
    if (a.n_seg < 0 || a.L < 1 || a.L > kMaxL || a.H < 1 || a.W < 1) return false;
    s += (long long)a.n_seg * (((a.H + kTile - 1) / kTile) * ((a.W + kTile - 1) / kTile));
    if (s > INT_MAX) return false;
    b.begin[i + 1] = (int)s;
  }
  return true;
}

cudaError_t temporal_init() {
  static unsigned char done[kMaxDevices] = {};
  return once_per_device(done, [](int) {
    cudaError_t e = cudaFuncSetAttribute(k_temporal, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)temporal_smem(kMaxL));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_temporal_tm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kTmSmem);
    return e;
  });
}

// The kernel is chosen per video, so that a video gets the same arithmetic
// whether it runs alone or with others: the videos for which the tensor-memory
// kernel applies go to launches of it (one per set of Gaussian taps, which that
// kernel takes as one kernel parameter), the others to one launch of the
// general kernel.
cudaError_t launch_temporal_multi(const TemporalBatch& b, cudaStream_t st) {
  if (b.begin[b.n] <= 0) return cudaSuccess;
  cudaError_t e = temporal_init();
  if (e != cudaSuccess) return e;
  bool tm[kMaxVideos], done[kMaxVideos];
  TemporalBatch gb{};
  for (int i = 0; i < b.n; ++i) {
    CUtensorMap probe[2];
    const TemporalArgs& a = b.a[i];
    tm[i] = tm_applies(a) &&
            tm_frame_map(&probe[0], a.src.n_carry > 0 ? a.src.carry : a.src.batch,
                         a.src.n_carry > 0 ? a.src.n_carry : a.src.n_batch, a.H, a.W) &&
            tm_frame_map(&probe[1], a.src.batch, a.src.n_batch, a.H, a.W);
    done[i] = !tm[i];
    if (!tm[i]) gb.a[gb.n++] = a;
  }
  for (int lead = 0; lead < b.n; ++lead) {
    if (done[lead]) continue;
    TemporalBatch tb{};
    TemporalMaps maps;
    std::memset(&maps, 0, sizeof(maps));
    TemporalTaps taps;
    std::memcpy(taps.w, b.a[lead].gw, sizeof(taps.w));
    for (int i = lead; i < b.n; ++i) {
      const TemporalArgs& a = b.a[i];
      if (done[i] || std::memcmp(a.gw, taps.w, sizeof(taps.w)) != 0) continue;
      tm_frame_map(&maps.m[tb.n][0], a.src.n_carry > 0 ? a.src.carry : a.src.batch,
                   a.src.n_carry > 0 ? a.src.n_carry : a.src.n_batch, a.H, a.W);
      tm_frame_map(&maps.m[tb.n][1], a.src.batch, a.src.n_batch, a.H, a.W);
      tb.a[tb.n++] = a;
      done[i] = true;
    }
    if (!temporal_batch_finalize(tb)) return cudaErrorInvalidValue;
    if (tb.begin[tb.n] > 0) {
      k_temporal_tm<<<tb.begin[tb.n], kTmThreads, kTmSmem, st>>>(tb, maps, taps);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  if (gb.n > 0) {
    if (!temporal_batch_finalize(gb)) return cudaErrorInvalidValue;
    if (gb.begin[gb.n] > 0) {
      int L = 1;
      for (int i = 0; i < gb.n; ++i) L = L > gb.a[i].L ? L : gb.a[i].L;
      k_temporal<<<gb.begin[gb.n], kTempThreads, temporal_smem(L), st>>>(gb);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t launch_temporal(const TemporalArgs& a, cudaStream_t st) {
  if (a.n_seg <= 0) return cudaSuccess;
  TemporalBatch b{};
  b.n = 1;
  b.a[0] = a;
  if (!temporal_batch_finalize(b)) return cudaErrorInvalidValue;
  return launch_temporal_multi(b, st);
}

}  // namespace vimg
