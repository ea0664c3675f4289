// Spiking-pixel U-Net stage for sm_103a (Sec. III-C of Bando et al., BIBM 2023):
// a U-Net on 64x64 patches of the segment's summary pair (S_i, T_i), patches
// every 32 px (plus one flush with the far border), outputs merged into one
// probability map per segment by a tent-weighted average.
//
// Network (the layer sizes of the paper's figure are not available; this is
// the reading): per level two 3x3 convolutions (zero padding 1) + ReLU with
// 16, 32, 64, 128, 256 channels at 64, 32, 16, 8, 4 px, 2x2 max pooling between
// levels; decoder: 2x2 stride-2 up-convolution (no activation) halving the
// channels, concatenation [skip, up], two 3x3 convolutions + ReLU; output 1x1
// convolution 16 -> 1 and a sigmoid.  Inputs: S_i and T_i standardised over the
// whole image, (x - mean) / (std + 1e-3).
//
// Every 3x3 convolution and up-convolution is an implicit GEMM on the tensor
// cores (tcgen05.mma kind::f16, BF16 operands, FP32 accumulation in TMEM):
//   D[pixel][n] = sum_{tap, ci} A[pixel][(tap, ci)] * B[(tap, ci)][n]
// M = 128 consecutive pixels of the activation array, N = output channels (x 4
// quadrants for an up-convolution), K = taps x input channels in chunks.
// Activations live in 8-channel planes [C/8][guard + pixels + guard][8] (BF16),
// so the 8 channels of 8 consecutive pixels form one K-major core matrix
// (8 rows x 16 B).  On the 64, 32 and 16 px levels every image carries a
// one-pixel zero border and the planes zero guard zones that no kernel
// writes: tap (dy, dx) of a 3x3 convolution then reads pixel i + dy (s + 2) +
// dx of the same plane, so one contiguous halo per plane, fetched by one bulk
// copy, serves all nine taps through shifted shared-memory descriptors, and up
// to four 128-row subtiles share a halo (independent accumulators, interleaved
// MMAs).  The 8 and 4 px levels are stored dense and take one im2col TMA box
// per tap and plane (zero fill outside the image gives the padding).  B chunks
// are weights pre-packed in the same core-matrix layout; a layer's weights
// stay in shared memory when they fit.  Per layer, the configuration (channels
// per chunk, subtiles, stages, one or two CTAs per SM) is chosen by the
// estimated L2 -> SM bytes per output row.
//
// Warp roles (persistent CTAs, 192 threads): warp 4 producer, warp 5 MMA
// issuer, warps 0-3 epilogue (TMEM lane = pixel): + bias, ReLU, BF16 stores
// into the planes at a plane offset (which forms the concatenations in place),
// or the 2x2 scatter of an up-convolution.  Two TMEM accumulators let the
// epilogue of one tile overlap the MMAs of the next.  Every wait is bounded:
// on timeout the CTA records an error, stops issuing, drains its own copies and
// MMAs, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "tc_ptx.h"
#include "vimg_internal.h"

namespace vimg {
namespace {
using namespace tc;

constexpr int kUPatch = 64;
constexpr int kUStride = 32;
constexpr int kULevels = 4;
constexpr int kUC0 = 16;                 // channels at 64x64
constexpr double kUEps = 1e-3;           // standardisation: (x - m) / (sd + eps)
constexpr int kUMaxStages = 8;
constexpr int kUEpiWarps = 4;
constexpr int kUThreads = (kUEpiWarps + 2) * 32;  // 192
constexpr size_t kUSmemMax = 200 * 1024;

// Architecture in parameter order: kind (0 conv 3x3, 1 up 2x2, 2 output 1x1),
// input and output channels.
struct LayerDef {
  int kind, cin, cout;
};

std::vector<LayerDef> unet_defs() {
  std::vector<LayerDef> d;
  int ch[kULevels + 1];
  for (int l = 0; l <= kULevels; ++l) ch[l] = kUC0 << l;
  d.push_back({0, 2, ch[0]});
  d.push_back({0, ch[0], ch[0]});
  for (int l = 1; l <= kULevels; ++l) {
    d.push_back({0, ch[l - 1], ch[l]});
    d.push_back({0, ch[l], ch[l]});
  }
  for (int l = kULevels - 1; l >= 0; --l) {
    d.push_back({1, ch[l + 1], ch[l]});
    d.push_back({0, 2 * ch[l], ch[l]});
    d.push_back({0, ch[l], ch[l]});
  }
  d.push_back({2, ch[0], 1});
  return d;
}

size_t weight_count(const LayerDef& L) {
  const int taps = L.kind == 0 ? 9 : (L.kind == 1 ? 4 : 1);
  return (size_t)L.cin * L.cout * taps;
}

// Activations are BF16 in 8-channel planes: [C / 8][guard + pixels + guard][8],
// pixels patch-major, so that 8 channels of consecutive pixels -- one K-major
// core matrix per 8 pixels -- are contiguous.  Levels 0..kUPadLevels-1 (64, 32,
// 16 px) are stored with a one-pixel zero border (side s + 2) and zero guard
// zones around each plane, none of which any kernel writes: a 3x3 convolution
// reads pixel i + dy (s + 2) + dx of the same plane, so one contiguous halo of
// 128 + 2 (s + 2) + 2 pixels per plane, fetched by one bulk copy, serves all
// nine taps ("halo" tiles, shifted descriptors).  The 8 and 4 px levels are
// stored dense; their tiles take one TMA box per tap and plane (im2col boxes
// with zero fill at the image border): a border would add 56 % and 125 % rows
// there (measured: the 8 px level padded is 13 % slower).
constexpr int kUPadLevels = 3;
constexpr int kUGuard = 640;  // guard pixels before and after each padded plane

struct ConvParams {
  int lin;                 // 1: padded input, halo tiles (bulk copies); 0: im2col boxes (TMA)
  const __nv_bfloat16* in; // input planes (halo tiles)
  size_t in_plane;         // elements per input plane (incl. guards)
  int in_guard;            // guard pixels before the data of an input plane
  int m_px;                // M rows in use: pixels of the input layout (incl. border)
  int s_in, sp_in;         // input side, and its stored side (s_in + 2 when padded)
  int bh, bb;              // boxes: rows and images per box (bh * bb * s_in = 128)
  int hoff;                // halo: first pixel = m0 - hoff
  uint32_t plane_bytes;    // halo: one 8-channel plane in shared memory (rows x 16 B)
  int kc, nkc, taps;       // channels per K chunk, chunks per tile (x taps in box mode)
  int R;                   // 128-row subtiles per tile (halo tiles share one halo)
  int bres;                // 1: the layer's weights stay in shared memory for the whole CTA
  uint32_t bres_bytes;
  int ntile, n_ntiles, n_mtiles;
  int stages;
  uint32_t a_bytes, b_bytes;   // per stage
  const __nv_bfloat16* wpack;  // [n_ntiles][chunk][tap in chunk][kc / 8][ntile][8]
  const float* bias;           // [n_ntiles * ntile]
  __nv_bfloat16* out;
  size_t out_plane;            // elements per output plane (incl. guards)
  int out_guard, out_goff;     // guard pixels; first output plane written
  int so, spo;                 // output side, stored output side
  int up, cout, relu;
  unsigned long long div_img, div_sp;  // ceil(2^40 / (sp_in^2)), ceil(2^40 / sp_in)
  int* err;
};

// n / d for 0 <= n < 2^31 and d < 2^16 from M = ceil(2^40 / d): the estimate is
// exact or one too large.
__device__ __forceinline__ int fdiv(int n, int d, unsigned long long M) {
  int q = (int)(((unsigned long long)n * M) >> 40);
  if (q * d > n) --q;
  return q;
}

// Bounded wait with a short sleep between polls, for the epilogue warps (they
// wait long) so that they leave issue slots to the MMA thread.
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t* bar, uint32_t parity) {
  for (long long i = 0; i < kTcSpin; ++i) {
    if (mbar_wait(bar, parity, 1)) return true;
    __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// TQ: taps per stage (9 for 3x3 halo tiles, 1 for up-convolutions and im2col boxes).
template <int TQ>
__global__ void __launch_bounds__(kUThreads, 1)
    k_conv_tc(const __grid_constant__ CUtensorMap tmap, const ConvParams p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kUMaxStages], empty[kUMaxStages];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], mma_done, bres_full;
  __shared__ float sbias[4 * 256];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int S = p.stages;
  unsigned char* sBres = smem;                                   // resident weights
  unsigned char* sA = smem + p.bres_bytes;                       // [S][a_bytes]
  unsigned char* sB = sA + (size_t)S * p.a_bytes;                // [S][b_bytes] (not resident)
  const int n_tiles = p.n_mtiles * p.n_ntiles;
  const int nq = TQ == 9 ? p.nkc : p.taps * p.nkc;           // stages per tile
  const int acc_cols = p.R * p.ntile;                        // columns of one accumulator
  uint32_t tcols = 32;
  while (tcols < (uint32_t)(2 * acc_cols)) tcols <<= 1;
  const uint32_t stage_tx = p.a_bytes + (p.bres ? 0u : p.b_bytes);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&tmem_base)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  for (int i = tid; i < p.n_ntiles * p.ntile; i += blockDim.x) sbias[i] = p.bias[i];
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kUEpiWarps);
    }
    mbar_init(&mma_done, 1);
    mbar_init(&bres_full, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const int img_px = p.sp_in * p.sp_in;
  const int m_tile = 128 * p.R;

  if (warp == kUEpiWarps) {
    // ---------------- producer ----------------
    if (lane == 0) {
      if (p.bres) {  // the whole layer's weights, once
        mbar_expect_tx(&bres_full, p.bres_bytes);
        for (uint32_t o = 0; o < p.bres_bytes; o += 32768u) {
          const uint32_t n = p.bres_bytes - o < 32768u ? p.bres_bytes - o : 32768u;
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  su32(sBres + o)),
              "l"(reinterpret_cast<const unsigned char*>(p.wpack) + o), "r"(n),
              "r"(su32(&bres_full))
              : "memory");
        }
      }
      int it = 0;
      for (int tile = blockIdx.x; tile < n_tiles && !abort_flag; tile += gridDim.x) {
        const int nt = tile % p.n_ntiles, mt = tile / p.n_ntiles;
        const int m0 = mt * m_tile, b0 = m0 / img_px, h0 = (m0 - b0 * img_px) / p.sp_in;
        for (int q = 0; q < nq; ++q, ++it) {
          const int s = it % S, cyc = it / S;
          if (cyc > 0 && !mbar_wait(&empty[s], (cyc - 1) & 1)) {
            atomicExch(p.err, 1);
            abort_flag = 1;
            break;
          }
          mbar_expect_tx(&full[s], stage_tx);
          unsigned char* a_dst = sA + (size_t)s * p.a_bytes;
          if (p.lin) {
            // one contiguous halo per plane (the guards keep it inside the buffer)
            const __nv_bfloat16* src0 =
                p.in + (size_t)(p.in_guard + m0 - p.hoff) * 8 + (size_t)q * (p.kc / 8) * p.in_plane;
            for (int g = 0; g < p.kc / 8; ++g)
              asm volatile(
                  "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                      su32(a_dst + g * p.plane_bytes)),
                  "l"(src0 + (size_t)g * p.in_plane), "r"(p.plane_bytes), "r"(su32(&full[s]))
                  : "memory");
          } else {
            const int t = q / p.nkc, c = q - t * p.nkc;
            const int dy = p.taps == 9 ? t / 3 - 1 : 0, dx = p.taps == 9 ? t % 3 - 1 : 0;
            // map dims {8 s (x, channel), s (y), P, planes}: x = dx * 8 elements
            for (int g = 0; g < p.kc / 8; ++g)
              asm volatile(
                  "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(
                      su32(a_dst + g * 2048)),
                  "l"(&tmap), "r"(dx * 8), "r"(h0 + dy), "r"(b0), "r"(c * (p.kc / 8) + g),
                  "r"(su32(&full[s]))
                  : "memory");
          }
          if (!p.bres)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    su32(sB + (size_t)s * p.b_bytes)),
                "l"(p.wpack + ((size_t)nt * nq + q) * (p.b_bytes / 2)), "r"(p.b_bytes),
                "r"(su32(&full[s]))
                : "memory");
        }
      }
      // wait (bounded) for the last use of every stage: no copy outlives the CTA
      for (int s = 0; s < S && s < it; ++s) mbar_wait(&full[s], ((it - 1 - s) / S) & 1);
      if (p.bres) mbar_wait(&bres_full, 0);
    }
  } else if (warp == kUEpiWarps + 1) {
    // ---------------- MMA issuer ----------------
    // The whole warp runs the loop in step and one elected lane issues each MMA
    // and commit, so the descriptor arithmetic stays warp-uniform.
    {
      int it = 0, tl = 0;
      bool issued = false, fail = false;
      const uint32_t idesc = idesc_for(p.ntile);
      const uint32_t a_lbo = p.lin ? p.plane_bytes : 2048u;
      // descriptor steps in 16-byte units
      const uint64_t a_k = (2 * a_lbo) >> 4, b_k = (2 * p.ntile * 16) >> 4;
      const uint64_t b_t = ((uint32_t)p.ntile * p.kc * 2) >> 4;
      uint64_t a_t[TQ];  // halo tiles: tap (dy, dx) starts hoff + dy (s + 2) + dx pixels in
#pragma unroll
      for (int t = 0; t < TQ; ++t)
        a_t[t] = TQ == 9 ? (uint64_t)(p.hoff + (t / 3 - 1) * p.sp_in + (t % 3 - 1)) : 0;
      const int kk = p.kc / 16, R = p.R;
      if (p.bres && !mbar_wait_warp(&bres_full, 0)) fail = true;
      for (int tile = blockIdx.x; tile < n_tiles && !fail; tile += gridDim.x, ++tl) {
        if (__shfl_sync(0xffffffffu, abort_flag, 0)) break;
        const int buf = tl & 1, use = tl >> 1;
        if (use > 0) {
          if (!mbar_wait_warp(&acc_empty[buf], (use - 1) & 1)) {
            fail = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
        }
        const uint32_t dbase = tmem + (uint32_t)(buf * acc_cols);
        for (int q = 0; q < nq; ++q, ++it) {
          const int s = it % S;
          if (!mbar_wait_warp(&full[s], (it / S) & 1)) {
            fail = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint64_t ad0 = desc(su32(sA + (size_t)s * p.a_bytes), a_lbo, 128);
          const uint64_t bd0 =
              p.bres ? desc(su32(sBres + (size_t)q * p.b_bytes), p.ntile * 16, 128)
                     : desc(su32(sB + (size_t)s * p.b_bytes), p.ntile * 16, 128);
          // taps outer, subtiles inner: consecutive MMAs go to independent accumulators
#pragma unroll
          for (int t = 0; t < TQ; ++t) {
            for (int k = 0; k < kk; ++k) {
              const uint64_t ad = ad0 + a_t[t] + (uint64_t)k * a_k;
              const uint64_t bd = bd0 + (uint64_t)t * b_t + (uint64_t)k * b_k;
              const uint32_t acc = (q > 0 || t > 0 || k > 0) ? 1u : 0u;
#pragma unroll
              for (int r = 0; r < 4; ++r) {
                if (r < R)
                  asm volatile(
                      "{\n.reg .pred pe, pa;\nelect.sync _|pe, 0xffffffff;\nsetp.ne.b32 pa, %4, 0;\n"
                      "@pe tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n}\n" ::"r"(
                          dbase + (uint32_t)(r * p.ntile)),
                      "l"(ad + (uint64_t)(128 * r)), "l"(bd), "r"(idesc), "r"(acc));
              }
            }
          }
          issued = true;
          mma_commit_elect(&empty[s]);
        }
        if (fail) break;
        mma_commit_elect(&acc_full[buf]);
      }
      if (fail && lane == 0) {
        atomicExch(p.err, 1);
        abort_flag = 1;
      }
      // every MMA issued by this warp has completed before the CTA frees TMEM
      if (issued) {
        mma_commit_elect(&mma_done);
        mbar_wait_warp(&mma_done, 0);
      }
    }
  } else {
    // ------ epilogue: warp w owns TMEM lanes (pixels) 32 w .. 32 w + 31 of each subtile ------
    int tl = 0;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const int pad_in = p.sp_in != p.s_in, pad_out = p.spo != p.so;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++tl) {
      const int buf = tl & 1, use = tl >> 1;
      const int nt = tile % p.n_ntiles, mt = tile / p.n_ntiles;
      if (!mbar_wait_sleep(&acc_full[buf], use & 1)) {
        atomicExch(p.err, 1);
        abort_flag = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      for (int r = 0; r < p.R; ++r) {
        const int m = mt * m_tile + 128 * r + warp * 32 + lane;
        // input pixel of this row; rows on the zero border (or past the end) store nothing
        const int b = fdiv(m, img_px, p.div_img), rr = m - b * img_px;
        const int yq = fdiv(rr, p.sp_in, p.div_sp);
        const int y = yq - pad_in, x = rr - yq * p.sp_in - pad_in;
        const bool valid = m < p.m_px && y >= 0 && y < p.s_in && x >= 0 && x < p.s_in;
        const size_t row_out = (size_t)b * p.spo;
        // two 16-column TMEM loads in flight per wait
        for (int c2 = 0; c2 < p.ntile; c2 += 32) {
          uint32_t raw[2][16];
          const uint32_t ta = tmem + lane_base + (uint32_t)(buf * acc_cols + r * p.ntile + c2);
          tmem_ld16_nowait(ta, raw[0]);
          if (c2 + 16 < p.ntile) tmem_ld16_nowait(ta + 16, raw[1]);
          tmem_wait_ld();
          for (int hh = 0; hh < 2 && c2 + 16 * hh < p.ntile; ++hh) {
          const int c0 = c2 + 16 * hh;
          float v[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(raw[hh][j]);
          if (!valid) continue;
          const int ng = nt * p.ntile + c0;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            v[j] += sbias[ng + j];
            if (p.relu) v[j] = fmaxf(v[j], 0.f);
          }
          int ch, oy = y, ox = x;
          if (p.up) {
            const int qd = ng / p.cout;
            ch = ng - qd * p.cout;
            oy = 2 * y + (qd >> 1), ox = 2 * x + (qd & 1);
          } else {
            ch = ng;
          }
          const size_t opix = (row_out + oy + pad_out) * p.spo + ox + pad_out;
          uint4 lo, hi;
          lo.x = pack_bf16x2(v[0], v[1]), lo.y = pack_bf16x2(v[2], v[3]);
          lo.z = pack_bf16x2(v[4], v[5]), lo.w = pack_bf16x2(v[6], v[7]);
          hi.x = pack_bf16x2(v[8], v[9]), hi.y = pack_bf16x2(v[10], v[11]);
          hi.z = pack_bf16x2(v[12], v[13]), hi.w = pack_bf16x2(v[14], v[15]);
          // two planes of 8 channels; consecutive lanes = consecutive pixels
          __nv_bfloat16* dst = p.out + (size_t)(p.out_goff + ch / 8) * p.out_plane +
                               (size_t)(p.out_guard + opix) * 8;
          *reinterpret_cast<uint4*>(dst) = lo;
          *reinterpret_cast<uint4*>(dst + p.out_plane) = hi;
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}

// ---- small kernels ---------------------------------------------------------------
// Weights of one layer into the B-operand layout [nt][chunk][tap in chunk][g][n][8]
// (box tiles: chunk = tap x channel chunk, one tap each; halo tiles: chunk =
// channel chunk, all taps), BF16; ci = c kc + 8 g + j, column ng = nt ntile + n.
__global__ void k_pack(const float* __restrict__ w, const float* __restrict__ bias, int up,
                       int lin, int cin_real, int cout, int taps, int kc, int nkc, int ntile,
                       int n_ntiles, __nv_bfloat16* __restrict__ out, float* __restrict__ bout) {
  const int nq = lin ? nkc : taps * nkc, tq = lin ? taps : 1;
  const long long total = (long long)n_ntiles * nq * tq * kc * ntile;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long r = i;
    const int j = (int)(r % 8);
    r /= 8;
    const int n = (int)(r % ntile);
    r /= ntile;
    const int g = (int)(r % (kc / 8));
    r /= kc / 8;
    const int tt = (int)(r % tq);
    r /= tq;
    const int q = (int)(r % nq);
    const int nt = (int)(r / nq);
    const int t = lin ? tt : q / nkc, c = lin ? q : q - (q / nkc) * nkc;
    const int ci = c * kc + 8 * g + j, ng = nt * ntile + n;
    float v = 0.f;
    if (ci < cin_real) {
      if (up) {
        const int qd = ng / cout, co = ng - qd * cout;
        v = w[(((size_t)ci * cout + co) * 2 + (qd >> 1)) * 2 + (qd & 1)];
      } else {
        v = w[((size_t)ng * cin_real + ci) * 9 + t];
      }
    }
    out[i] = __float2bfloat16_rn(v);
    if (i < (long long)n_ntiles * ntile) bout[i] = bias[up ? (int)(i % cout) : (int)i];
  }
}

constexpr int kUStatBlocks = 64;  // partial-sum blocks per image

// Partial FP64 sums of x and x^2 per image (fixed order per block).
__global__ void k_ustats_part(const float* __restrict__ summary, int HW, double* __restrict__ part) {
  __shared__ double r1[256], r2[256];
  const float* img = summary + (size_t)blockIdx.y * HW;
  double s = 0.0, q = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < HW; i += gridDim.x * blockDim.x) {
    const double v = (double)img[i];
    s += v;
    q = fma(v, v, q);
  }
  r1[threadIdx.x] = s;
  r2[threadIdx.x] = q;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      r1[threadIdx.x] += r1[threadIdx.x + o];
      r2[threadIdx.x] += r2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x)] = r1[0];
    part[2 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x) + 1] = r2[0];
  }
}

// Mean and 1 / (population std + eps) per image from the partial sums.
__global__ void k_ustats_fin(const double* __restrict__ part, int n_img, int HW,
                             double* __restrict__ stats) {
  const int im = blockIdx.x * blockDim.x + threadIdx.x;
  if (im >= n_img) return;
  double s = 0.0, q = 0.0;
  for (int b = 0; b < kUStatBlocks; ++b) {
    s += part[2 * ((size_t)im * kUStatBlocks + b)];
    q += part[2 * ((size_t)im * kUStatBlocks + b) + 1];
  }
  const double mean = s / HW, var = fmax(q / HW - mean * mean, 0.0);
  stats[2 * im] = mean;
  stats[2 * im + 1] = 1.0 / (sqrt(var) + kUEps);
}

__device__ __forceinline__ int upos(int j, int n) { return min(kUStride * j, n - kUPatch); }

// Patches of the standardised pair into plane 0 of the padded level-0 input
// (66 x 66 per patch, border and plane 1 left zero): channels 0, 1 = S, T.
__global__ void k_uinput(const float* __restrict__ summary, const double* __restrict__ stats,
                         int H, int W, int npy, int npx, int n_patch_total, int guard,
                         __nv_bfloat16* __restrict__ in0) {
  const long long total = (long long)n_patch_total * kUPatch * kUPatch;
  constexpr int sp = kUPatch + 2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(i % kUPatch), u = (int)((i / kUPatch) % kUPatch);
    const int pt = (int)(i / (kUPatch * kUPatch));
    const int seg = pt / (npy * npx), pr = pt - seg * npy * npx;
    const int y = upos(pr / npx, H) + u, x = upos(pr % npx, W) + v;
    const size_t HW = (size_t)H * W;
    const float* S = summary + (size_t)seg * 2 * HW;
    const double* st = stats + 4 * seg;
    // (x - mean) / (std + eps) as one FP32 FMA with the FP64 statistics rounded once
    const float zs = fmaf(S[(size_t)y * W + x], (float)st[1], (float)(-st[0] * st[1]));
    const float zt = fmaf(S[HW + (size_t)y * W + x], (float)st[3], (float)(-st[2] * st[3]));
    uint4 a;
    a.x = pack_bf16x2(zs, zt);
    a.y = a.z = a.w = 0u;
    const size_t o = ((size_t)pt * sp + u + 1) * sp + v + 1;
    *reinterpret_cast<uint4*>(in0 + (guard + o) * 8) = a;
  }
}

// 2x2 max pooling between planar buffers: planes [0, G) of the input (stored
// side spi = 2 so or 2 so + 2) into planes [0, G) of the output (side spo).
__global__ void k_upool(const __nv_bfloat16* __restrict__ in, size_t in_plane, int in_guard,
                        int spi, __nv_bfloat16* __restrict__ out, size_t out_plane, int out_guard,
                        int spo, int P, int so, int G) {
  const int pi = spi != 2 * so, po = spo != so;
  const long long npx = (long long)P * so * so, total = npx * G;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long px = i % npx;
    const int g = (int)(i / npx);
    const int xo = (int)(px % so), yo = (int)((px / so) % so);
    const long long b = px / ((long long)so * so);
    const size_t ip = ((size_t)b * spi + 2 * yo + pi) * spi + 2 * xo + pi;
    const __nv_bfloat16* src = in + (size_t)g * in_plane + (in_guard + ip) * 8;
    const uint4 a = *reinterpret_cast<const uint4*>(src);
    const uint4 bq = *reinterpret_cast<const uint4*>(src + 8);
    const uint4 c = *reinterpret_cast<const uint4*>(src + (size_t)spi * 8);
    const uint4 d = *reinterpret_cast<const uint4*>(src + (size_t)spi * 8 + 8);
    const __nv_bfloat162* pa = reinterpret_cast<const __nv_bfloat162*>(&a);
    const __nv_bfloat162* pb = reinterpret_cast<const __nv_bfloat162*>(&bq);
    const __nv_bfloat162* pc = reinterpret_cast<const __nv_bfloat162*>(&c);
    const __nv_bfloat162* pd = reinterpret_cast<const __nv_bfloat162*>(&d);
    uint4 o;
    __nv_bfloat162* pw = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
    for (int k = 0; k < 4; ++k) pw[k] = __hmax2(__hmax2(pa[k], pb[k]), __hmax2(pc[k], pd[k]));
    const size_t op = ((size_t)b * spo + yo + po) * spo + xo + po;
    *reinterpret_cast<uint4*>(out + (size_t)g * out_plane + (out_guard + op) * 8) = o;
  }
}

// Output layer: p = sigmoid(b + sum_c w_c d0_c), FP32 weights, per patch pixel
// (d0: two planes, padded 66 x 66 per patch).
__global__ void k_uout(const __nv_bfloat16* __restrict__ d0, size_t plane, int guard,
                       const float* __restrict__ wout, long long n_px, float* __restrict__ prob) {
  constexpr int sp = kUPatch + 2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_px;
       i += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(i % kUPatch), u = (int)((i / kUPatch) % kUPatch);
    const long long pt = i / (kUPatch * kUPatch);
    const size_t o = ((size_t)pt * sp + u + 1) * sp + v + 1;
    const uint4 a = *reinterpret_cast<const uint4*>(d0 + (guard + o) * 8);
    const uint4 b = *reinterpret_cast<const uint4*>(d0 + plane + (guard + o) * 8);
    const __nv_bfloat16* ha = reinterpret_cast<const __nv_bfloat16*>(&a);
    const __nv_bfloat16* hb = reinterpret_cast<const __nv_bfloat16*>(&b);
    float s = wout[kUC0];
#pragma unroll
    for (int c = 0; c < 8; ++c) s = fmaf(wout[c], __bfloat162float(ha[c]), s);
#pragma unroll
    for (int c = 0; c < 8; ++c) s = fmaf(wout[8 + c], __bfloat162float(hb[c]), s);
    prob[i] = 1.0f / (1.0f + expf(-s));
  }
}

// Interior of planes [goff, goff + C / 8) of a planar buffer (stored side sp)
// into a dense NHWC array [P][s][s][C].
__global__ void k_ucompact(const __nv_bfloat16* __restrict__ in, size_t plane, int guard, int goff,
                           int P, int s, int sp, int C, __nv_bfloat16* __restrict__ out) {
  const int pad = sp != s;
  const long long total = (long long)P * s * s * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long px = i / C;
    const int x = (int)(px % s), y = (int)((px / s) % s);
    const long long b = px / ((long long)s * s);
    const size_t ip = ((size_t)b * sp + y + pad) * sp + x + pad;
    out[i] = in[(size_t)(goff + c / 8) * plane + (guard + ip) * 8 + (c % 8)];
  }
}

__device__ __forceinline__ float utent(int u) { return (float)min(u + 1, kUPatch - u); }

// Weighted average of the patches covering each pixel (fixed order).
__global__ void k_umerge(const float* __restrict__ pprob, int H, int W, int npy, int npx, int k,
                         float* __restrict__ out) {
  const long long total = (long long)k * H * W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int X = (int)(i % W), Y = (int)((i / W) % H), seg = (int)(i / ((long long)H * W));
    int cy[3] = {Y / kUStride - 1, Y / kUStride, npy - 1};
    int cx[3] = {X / kUStride - 1, X / kUStride, npx - 1};
    float acc = 0.f, ws = 0.f;
    for (int a = 0; a < 3; ++a) {
      const int jy = cy[a];
      if (jy < 0 || jy >= npy || (a == 2 && (jy == cy[0] || jy == cy[1]))) continue;
      const int u = Y - upos(jy, H);
      if (u < 0 || u >= kUPatch) continue;
      for (int c = 0; c < 3; ++c) {
        const int jx = cx[c];
        if (jx < 0 || jx >= npx || (c == 2 && (jx == cx[0] || jx == cx[1]))) continue;
        const int v = X - upos(jx, W);
        if (v < 0 || v >= kUPatch) continue;
        const float wt = utent(u) * utent(v);
        const size_t pt = (size_t)seg * npy * npx + (size_t)jy * npx + jx;
        acc = fmaf(wt, pprob[(pt * kUPatch + u) * kUPatch + v], acc);
        ws += wt;
      }
    }
    out[i] = acc / ws;
  }
}

int grid_for(long long n, int threads, int sms) {
  const long long want = (n + threads - 1) / threads;
  const long long cap = (long long)sms * 16;
  return (int)std::max(1LL, std::min(want, cap));
}

}  // namespace
}  // namespace vimg

using namespace vimg;

struct vimg_unet {
  int H = 0, W = 0, max_seg = 0, npy = 0, npx = 0, npatch = 0, P = 0;
  int dev = 0, sms = 0;
  cudaStream_t st = nullptr;
  std::string err;
  int sticky = 0;
  bool loaded = false;
  std::vector<LayerDef> defs;
  float* wout = nullptr;  // [17] output layer, FP32
  // activations: planar BF16 (levels < kUPadLevels with zero border and guards)
  struct Act {
    __nv_bfloat16* p = nullptr;
    int level = 0, C = 0, guard = 0;
    size_t plane = 0;  // elements per 8-channel plane
  };
  Act in0;
  Act a[kULevels + 1];     // first encoder conv of a level
  Act da[kULevels];        // first decoder conv of a level
  Act cat[kULevels];       // [skip, up] per level 0..3
  Act pool[kULevels + 1];  // pooled input of levels 1..4
  Act d[kULevels + 1];     // decoder output per level 0..3, bottleneck at 4
  float* pprob = nullptr;                 // [P][64][64]
  double* stats = nullptr;                // [max_seg][2][2]
  double* part = nullptr;                 // [max_seg][2][kUStatBlocks][2]
  int* dev_err = nullptr;
  struct Conv {
    ConvParams p;
    CUtensorMap map;
    int grid = 0;
    size_t smem = 0;
    int cin_real = 0;                     // weights' input channels (2 for the first layer)
  };
  std::vector<Conv> convs;  // execution order = parameter order
  // profiling: event pairs around the tensor-core launches and the whole run
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  int ev_used = 0;
  double conv_ms = 0.0, total_ms = 0.0;
  long long conv_launches = 0;
  int last_np = 0;  // patches of the last internal pass (for vimg_unet_activation)
  std::vector<void*> allocs;
};

namespace {

int ufail(vimg_unet* u, int code, const std::string& msg) {
  if (u) {
    u->err = msg;
    if (code == VIMG_ERR_CUDA || code == VIMG_ERR_TIMEOUT) u->sticky = code;
  }
  return code;
}

#define UCK(call, what)                                                                 \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return ufail(u, VIMG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <class T>
cudaError_t ualloc(vimg_unet* u, T*& p, size_t n) {
  cudaError_t e = cudaMalloc((void**)&p, sizeof(T) * std::max<size_t>(n, 1));
  if (e == cudaSuccess) u->allocs.push_back(p);
  return e;
}

inline int side(int l) { return kUPatch >> l; }
inline int stored(int l) { return l < kUPadLevels ? side(l) + 2 : side(l); }

// One tensor-core layer: input = all planes of `in`; output into planes
// [out_goff, out_goff + cout / 8) of `out`.
int setup_conv(vimg_unet* u, const vimg_unet::Act& in, int cin_real, int taps, int n_total, int up,
               int cout, int relu, const vimg_unet::Act& out, int out_goff) {
  vimg_unet::Conv c{};
  ConvParams& p = c.p;
  const int P = u->P, li = in.level, cin = in.C;
  p.s_in = side(li), p.sp_in = stored(li);
  p.lin = p.sp_in != p.s_in;
  p.m_px = P * p.sp_in * p.sp_in;
  p.taps = taps;
  p.ntile = std::min(n_total, 256);
  p.n_ntiles = n_total / p.ntile;
  p.n_mtiles = (p.m_px + 127) / 128;
  // Halo tiles: channels per chunk (kc), 128-row subtiles per tile (R) and stages,
  // for two CTAs per SM (shared memory <= 104 KB, 2 x 2 R ntile TMEM columns
  // <= 512) or one; all taps' weights of a chunk sit in one stage (<= 48 KB),
  // the whole layer's weights stay resident when they fit.
  struct Cfg {
    int kc, R, S, bres;
    size_t smem;
  };
  auto halo_cfg = [&](int kc, int R, size_t budget) -> Cfg {
    Cfg f{kc, R, 0, 0, 0};
    if ((size_t)taps * p.ntile * kc * 2 > 48 * 1024 || cin % kc) return f;
    const int hoff = taps == 9 ? p.sp_in + 1 : 0;
    const size_t rows = (size_t)((128 * R + 2 * hoff + 7) & ~7);
    const size_t a = (kc / 8) * rows * 16, b = (size_t)taps * p.ntile * kc * 2;
    const size_t wbytes = (size_t)(cin / kc) * b;
    f.bres = p.n_ntiles == 1 && wbytes <= 160 * 1024 && wbytes + 2 * a <= budget;
    const size_t stage = a + (f.bres ? 0 : b), fixed = f.bres ? wbytes : 0;
    if (fixed + 2 * stage > budget) return f;
    f.S = (int)std::min<size_t>(4, (budget - fixed) / stage);
    f.smem = fixed + f.S * stage;
    return f;
  };
  if (p.lin) {
    // Every feasible (budget, R, kc): estimated L2 -> shared-memory bytes per
    // output row (halos of all planes, plus the weights unless resident),
    // divided by 0.7 when only one CTA fits an SM (less latency hiding).
    Cfg best{0, 0, 0, 0, 0};
    double best_cost = 0.0;
    for (size_t budget : {(size_t)104 * 1024, kUSmemMax}) {
      const int rmax = std::max(1, std::min(4, (budget == kUSmemMax ? 256 : 128) / p.ntile));
      for (int R = rmax; R >= 1; --R)
        for (int kc : {64, 32, 16}) {
          if (kc > cin) continue;
          const Cfg f = halo_cfg(kc, R, budget);
          if (f.S < 2) continue;
          const int hoff = taps == 9 ? p.sp_in + 1 : 0;
          const double rows = (double)((128 * R + 2 * hoff + 7) & ~7);
          const double a_all = (cin / 8) * rows * 16.0;
          const double b_all = f.bres ? 0.0 : (double)taps * p.ntile * cin * 2;
          const double cost = (a_all + b_all) / (128.0 * R) / (budget == kUSmemMax ? 0.7 : 1.0);
          if (!best.S || cost < best_cost) best = f, best_cost = cost;
        }
    }
    if (!best.S) return ufail(u, VIMG_ERR_ARG, "unet: no halo configuration fits");
    p.kc = best.kc, p.R = best.R, p.stages = best.S, p.bres = best.bres;
  } else {
    p.kc = std::min(cin, 64);
    p.R = 1;
    p.bres = 0;
  }
  p.nkc = cin / p.kc;
  p.n_mtiles = (p.m_px + 128 * p.R - 1) / (128 * p.R);
  if (p.lin) {
    p.in = in.p, p.in_plane = in.plane, p.in_guard = in.guard;
    p.hoff = taps == 9 ? p.sp_in + 1 : 0;
    const int rows = (128 * p.R + 2 * p.hoff + 7) & ~7;  // 128-byte multiple
    p.plane_bytes = (uint32_t)rows * 16;
    p.a_bytes = (uint32_t)(p.kc / 8) * p.plane_bytes;
    p.b_bytes = (uint32_t)taps * p.ntile * p.kc * 2;
    if (p.hoff > in.guard || rows - p.hoff > in.guard)
      return ufail(u, VIMG_ERR_ARG, "unet: halo exceeds the guard zone");
    p.bres_bytes = p.bres ? (uint32_t)(p.nkc * p.b_bytes) : 0u;
  } else {
    p.bh = std::min(p.s_in, 128 / p.s_in);
    p.bb = std::max(1, 128 / (p.s_in * p.s_in));
    p.a_bytes = 128u * p.kc * 2u;
    p.b_bytes = (uint32_t)p.ntile * p.kc * 2u;
    p.bres_bytes = 0;
    p.stages = (int)std::min<size_t>(kUMaxStages, kUSmemMax / (p.a_bytes + p.b_bytes));
  }
  const size_t stage = (size_t)p.a_bytes + (p.bres ? 0 : p.b_bytes);
  if (p.stages < 2 || cin % 16 || p.ntile % 16 || n_total % p.ntile ||
      (!p.lin && (p.bh * p.bb * p.s_in != 128 || 8 * p.s_in > 256)))
    return ufail(u, VIMG_ERR_ARG, "unet: unsupported layer shape");
  p.bias = nullptr, p.wpack = nullptr;  // set after allocation
  p.out = out.p, p.out_plane = out.plane, p.out_guard = out.guard, p.out_goff = out_goff;
  p.so = up ? 2 * p.s_in : p.s_in;
  p.spo = stored(out.level);
  p.up = up, p.cout = cout, p.relu = relu, p.err = u->dev_err;
  c.cin_real = cin_real;
  c.smem = p.bres_bytes + (size_t)p.stages * stage;
  p.div_img = ((1ull << 40) + (unsigned long long)(p.sp_in * p.sp_in) - 1) / (p.sp_in * p.sp_in);
  p.div_sp = ((1ull << 40) + (unsigned long long)p.sp_in - 1) / p.sp_in;
  if (p.n_ntiles * p.ntile > 4 * 256) return ufail(u, VIMG_ERR_ARG, "unet: too many columns");
  if (!p.lin) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return ufail(u, VIMG_ERR_CUDA, "unet: cuTensorMapEncodeTiled unavailable");
    const int sd = p.s_in;
    cuuint64_t dims[4] = {(cuuint64_t)8 * sd, (cuuint64_t)sd, (cuuint64_t)P, (cuuint64_t)cin / 8};
    cuuint64_t strides[3] = {(cuuint64_t)sd * 16, (cuuint64_t)sd * sd * 16,
                             (cuuint64_t)in.plane * 2};
    cuuint32_t box[4] = {(cuuint32_t)(8 * sd), (cuuint32_t)p.bh, (cuuint32_t)p.bb, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = fn(&c.map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4,
                    const_cast<__nv_bfloat16*>(in.p + (size_t)in.guard * 8), dims, strides, box,
                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return ufail(u, VIMG_ERR_CUDA, "unet: tensor map encode failed");
  } else {
    std::memset(&c.map, 0, sizeof(c.map));  // unused by halo tiles
  }
  // resident CTAs per SM: shared memory (228 KB per SM, ~1 KB reserved per CTA)
  // and tensor memory (512 columns)
  int tcols = 32;
  while (tcols < 2 * p.R * p.ntile) tcols <<= 1;
  const int by_smem = (int)((228 * 1024) / (c.smem + 6 * 1024));  // + static smem
  const int occ = std::max(1, std::min({by_smem, 512 / tcols, 4}));
  c.grid = u->sms * occ;
  u->convs.push_back(c);
  return VIMG_OK;
}

size_t pack_elems(const ConvParams& p) {
  return (size_t)p.n_ntiles * p.taps * p.nkc * p.kc * p.ntile;
}

}  // namespace

extern "C" int vimg_unet_param_count(void) {
  size_t n = 0;
  for (const LayerDef& L : unet_defs()) n += weight_count(L) + L.cout;
  return (int)n;
}

extern "C" int vimg_unet_layers(int* kind, int* cin, int* cout, int cap) {
  const std::vector<LayerDef> d = unet_defs();
  for (int i = 0; i < (int)d.size() && i < cap; ++i) {
    if (kind) kind[i] = d[i].kind;
    if (cin) cin[i] = d[i].cin;
    if (cout) cout[i] = d[i].cout;
  }
  return (int)d.size();
}

extern "C" void vimg_unet_destroy(vimg_unet* u) {
  if (!u) return;
  for (void* q : u->allocs) cudaFree(q);
  for (cudaEvent_t e : u->ev) cudaEventDestroy(e);
  delete u;
}

static std::string g_unet_create_error;

extern "C" vimg_unet* vimg_unet_create(int H, int W, int max_segments, void* stream) {
  if (H < kUPatch || W < kUPatch || H > 8192 || W > 8192 || max_segments < 1 ||
      max_segments > 4096) {
    g_unet_create_error = "vimg_unet_create: need 64 <= H, W <= 8192 and 1..4096 segments";
    return nullptr;
  }
  vimg_unet* u = new vimg_unet();
  u->H = H, u->W = W, u->max_seg = max_segments;
  u->npy = (H - kUPatch + kUStride - 1) / kUStride + 1;
  u->npx = (W - kUPatch + kUStride - 1) / kUStride + 1;
  u->npatch = u->npy * u->npx;
  u->P = u->npatch * max_segments;
  u->st = static_cast<cudaStream_t>(stream);
  u->defs = unet_defs();
  auto bail = [&](const std::string& m) -> vimg_unet* {
    g_unet_create_error = m;
    vimg_unet_destroy(u);
    return nullptr;
  };
  if (cudaGetDevice(&u->dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&u->sms, cudaDevAttrMultiProcessorCount, u->dev) != cudaSuccess)
    return bail("vimg_unet_create: no CUDA device");
  static unsigned char attr[kMaxDevices] = {};
  if (once_per_device(attr, [](int) {
        cudaError_t e = cudaFuncSetAttribute(k_conv_tc<9>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kUSmemMax);
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(k_conv_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kUSmemMax);
        return e;
      }) != cudaSuccess)
    return bail("vimg_unet_create: kernel attribute");
  const size_t P = u->P;
  cudaError_t e = cudaSuccess;
  auto A = [&](auto*& ptr, size_t n) {
    if (e == cudaSuccess) e = ualloc(u, ptr, n);
  };
  // planar activations, zeroed once: borders and guards are never written
  auto Z = [&](vimg_unet::Act& act, int level, int C) {
    act.level = level, act.C = C;
    act.guard = level < kUPadLevels ? kUGuard : 0;
    act.plane = (P * (size_t)stored(level) * stored(level) + 2 * (size_t)act.guard) * 8;
    const size_t n = act.plane * (C / 8);
    A(act.p, n);
    if (e == cudaSuccess) e = cudaMemsetAsync(act.p, 0, n * sizeof(__nv_bfloat16), u->st);
  };
  A(u->dev_err, 1);
  A(u->stats, 4 * (size_t)max_segments);
  A(u->part, 4 * (size_t)max_segments * kUStatBlocks);
  A(u->pprob, P * kUPatch * kUPatch);
  Z(u->in0, 0, kUC0);
  for (int l = 0; l <= kULevels; ++l) {
    const int C = kUC0 << l;
    Z(u->a[l], l, C);
    Z(u->d[l], l, C);
    if (l < kULevels) Z(u->cat[l], l, 2 * C);
    if (l < kULevels) Z(u->da[l], l, C);
    if (l > 0) Z(u->pool[l], l, C / 2);
  }
  A(u->wout, kUC0 + 1);
  if (e == cudaSuccess) e = cudaMemsetAsync(u->dev_err, 0, sizeof(int), u->st);
  if (e != cudaSuccess) return bail(std::string("vimg_unet_create: ") + cudaGetErrorString(e));
  // layer plan (execution order = parameter order)
  int li = 0;
  auto conv = [&](const vimg_unet::Act& in, const vimg_unet::Act& out, int goff) {
    const LayerDef& L = u->defs[li++];
    return setup_conv(u, in, L.cin, 9, L.cout, 0, L.cout, 1, out, goff);
  };
  auto upc = [&](const vimg_unet::Act& in, const vimg_unet::Act& out, int goff) {
    const LayerDef& L = u->defs[li++];
    return setup_conv(u, in, L.cin, 1, 4 * L.cout, 1, L.cout, 0, out, goff);
  };
  int rc = VIMG_OK;
  // encoder: level l input = in0 (l = 0) or pool[l]; skip -> cat[l] planes [0, C / 8)
  for (int l = 0; l <= kULevels && rc == VIMG_OK; ++l) {
    const vimg_unet::Act& in = l == 0 ? u->in0 : u->pool[l];
    rc = conv(in, u->a[l], 0);
    if (rc == VIMG_OK) rc = l < kULevels ? conv(u->a[l], u->cat[l], 0) : conv(u->a[l], u->d[l], 0);
  }
  // decoder: up from d[l + 1] into cat[l] planes [C / 8, C / 4), then two convolutions -> d[l]
  for (int l = kULevels - 1; l >= 0 && rc == VIMG_OK; --l) {
    const int C = kUC0 << l;
    rc = upc(u->d[l + 1], u->cat[l], C / 8);
    if (rc == VIMG_OK) rc = conv(u->cat[l], u->da[l], 0);
    if (rc == VIMG_OK) rc = conv(u->da[l], u->d[l], 0);
  }
  if (rc != VIMG_OK) return bail(u->err);
  // packed weights and biases per tensor-core layer
  for (auto& c : u->convs) {
    __nv_bfloat16* w = nullptr;
    float* b = nullptr;
    A(w, pack_elems(c.p));
    A(b, (size_t)c.p.n_ntiles * c.p.ntile);
    c.p.wpack = w, c.p.bias = b;
  }
  // the zeroed buffers must be in place before any stream uses them
  if (e == cudaSuccess) e = cudaStreamSynchronize(u->st);
  if (e != cudaSuccess) return bail(std::string("vimg_unet_create: ") + cudaGetErrorString(e));
  return u;
}

extern "C" const char* vimg_unet_last_error(const vimg_unet* u) {
  return u ? u->err.c_str() : g_unet_create_error.c_str();
}

extern "C" int vimg_unet_load(vimg_unet* u, const float* d_params) {
  if (!u || !d_params) return ufail(u, VIMG_ERR_ARG, "vimg_unet_load: null argument");
  if (u->sticky) return u->sticky;
  size_t off = 0;
  for (size_t i = 0; i < u->defs.size(); ++i) {
    const LayerDef& L = u->defs[i];
    const size_t nw = weight_count(L);
    const float* w = d_params + off;
    const float* b = w + nw;
    off += nw + L.cout;
    if (L.kind == 2) {
      UCK(cudaMemcpyAsync(u->wout, w, sizeof(float) * (kUC0 + 1), cudaMemcpyDeviceToDevice, u->st),
          "unet output weights");
      continue;
    }
    vimg_unet::Conv& c = u->convs[i];
    const ConvParams& p = c.p;
    const long long total = (long long)pack_elems(p);
    k_pack<<<grid_for(total, 256, u->sms), 256, 0, u->st>>>(
        w, b, p.up, p.lin, c.cin_real, L.cout, p.taps, p.kc, p.nkc, p.ntile, p.n_ntiles,
        const_cast<__nv_bfloat16*>(p.wpack), const_cast<float*>(p.bias));
    UCK(cudaGetLastError(), "unet weight pack");
  }
  // synchronous, so that a handle on another stream may run the U-Net next
  UCK(cudaStreamSynchronize(u->st), "unet weight pack");
  u->loaded = true;
  return VIMG_OK;
}

namespace {

int record(vimg_unet* u, cudaStream_t st) {
  if (!u->prof) return -1;
  if (u->ev_used >= (int)u->ev.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    u->ev.push_back(e);
  }
  cudaEventRecord(u->ev[u->ev_used], st);
  return u->ev_used++;
}

// Sums the recorded intervals: pairs (conv begin, end) ..., then (run begin, end).
int prof_collect(vimg_unet* u, const std::vector<int>& conv_ev, int run0, int run1) {
  if (!u->prof) return VIMG_OK;
  UCK(cudaEventSynchronize(u->ev[run1]), "unet profile sync");
  for (size_t i = 0; i + 1 < conv_ev.size(); i += 2) {
    float ms = 0.f;
    if (conv_ev[i] >= 0 && conv_ev[i + 1] >= 0 &&
        cudaEventElapsedTime(&ms, u->ev[conv_ev[i]], u->ev[conv_ev[i + 1]]) == cudaSuccess)
      u->conv_ms += ms;
    u->conv_launches++;
  }
  float ms = 0.f;
  if (run0 >= 0 && cudaEventElapsedTime(&ms, u->ev[run0], u->ev[run1]) == cudaSuccess)
    u->total_ms += ms;
  u->ev_used = 0;
  return VIMG_OK;
}

}  // namespace

int vimg_unet_run_on(vimg_unet* u, const float* d_summary, int k, float* d_prob, cudaStream_t st) {
  if (!u) return ufail(u, VIMG_ERR_ARG, "null U-Net");
  if (u->sticky) return u->sticky;
  if (!u->loaded) return ufail(u, VIMG_ERR_ARG, "vimg_unet_load must come before vimg_unet_run");
  if (k < 0 || (k > 0 && (!d_summary || !d_prob))) return ufail(u, VIMG_ERR_ARG, "vimg_unet_run: bad arguments");
  const size_t HW = (size_t)u->H * u->W;
  std::vector<int> conv_ev;
  const int run0 = k > 0 ? record(u, st) : -1;
  for (int s0 = 0; s0 < k; s0 += u->max_seg) {
    const int ks = std::min(k - s0, u->max_seg);
    const float* summ = d_summary + (size_t)s0 * 2 * HW;
    const int np = ks * u->npatch;
    k_ustats_part<<<dim3(kUStatBlocks, 2 * ks), 256, 0, st>>>(summ, (int)HW, u->part);
    UCK(cudaGetLastError(), "unet statistics");
    k_ustats_fin<<<(2 * ks + 63) / 64, 64, 0, st>>>(u->part, 2 * ks, (int)HW, u->stats);
    UCK(cudaGetLastError(), "unet statistics");
    const long long n_in = (long long)np * kUPatch * kUPatch;
    k_uinput<<<grid_for(n_in, 256, u->sms), 256, 0, st>>>(summ, u->stats, u->H, u->W, u->npy,
                                                          u->npx, np, u->in0.guard, u->in0.p);
    UCK(cudaGetLastError(), "unet input");
    // the tensor-core layers run over the np patch slots in use
    size_t ci = 0;
    auto run_conv = [&]() -> int {
      vimg_unet::Conv& c = u->convs[ci++];
      ConvParams p = c.p;
      p.m_px = np * p.sp_in * p.sp_in;
      p.n_mtiles = (p.m_px + 128 * p.R - 1) / (128 * p.R);
      const int grid = std::min(c.grid, p.n_mtiles * p.n_ntiles);
      conv_ev.push_back(record(u, st));
      if (p.lin && p.taps == 9)
        k_conv_tc<9><<<grid, kUThreads, c.smem, st>>>(c.map, p);
      else
        k_conv_tc<1><<<grid, kUThreads, c.smem, st>>>(c.map, p);
      conv_ev.push_back(record(u, st));
      UCK(cudaGetLastError(), "unet convolution");
      return VIMG_OK;
    };
    int rc = VIMG_OK;
    for (int l = 0; l <= kULevels && rc == VIMG_OK; ++l) {
      if (l > 0) {
        const int so = side(l), G = (kUC0 << (l - 1)) / 8;
        const vimg_unet::Act &src = u->cat[l - 1], &dst = u->pool[l];
        const long long n = (long long)np * so * so * G;
        k_upool<<<grid_for(n, 256, u->sms), 256, 0, st>>>(src.p, src.plane, src.guard,
                                                          stored(l - 1), dst.p, dst.plane,
                                                          dst.guard, stored(l), np, so, G);
        UCK(cudaGetLastError(), "unet pooling");
      }
      rc = run_conv();
      if (rc == VIMG_OK) rc = run_conv();
    }
    for (int l = kULevels - 1; l >= 0 && rc == VIMG_OK; --l)
      for (int j = 0; j < 3 && rc == VIMG_OK; ++j) rc = run_conv();
    if (rc != VIMG_OK) return rc;
    const long long n_px = (long long)np * kUPatch * kUPatch;
    k_uout<<<grid_for(n_px, 256, u->sms), 256, 0, st>>>(u->d[0].p, u->d[0].plane, u->d[0].guard,
                                                        u->wout, n_px, u->pprob);
    UCK(cudaGetLastError(), "unet output layer");
    const long long n_out = (long long)ks * HW;
    k_umerge<<<grid_for(n_out, 256, u->sms), 256, 0, st>>>(u->pprob, u->H, u->W, u->npy, u->npx, ks,
                                                          d_prob + (size_t)s0 * HW);
    UCK(cudaGetLastError(), "unet merge");
    u->last_np = np;
  }
  if (k > 0) {
    const int run1 = record(u, st);
    if (run1 >= 0) return prof_collect(u, conv_ev, run0, run1);
  }
  return VIMG_OK;
}

extern "C" int vimg_unet_run(vimg_unet* u, const float* d_summary, int k, float* d_prob) {
  return vimg_unet_run_on(u, d_summary, k, d_prob, u ? u->st : nullptr);
}

extern "C" int vimg_unet_synchronize(vimg_unet* u) {
  if (!u) return ufail(u, VIMG_ERR_ARG, "null U-Net");
  if (u->sticky) return u->sticky;
  UCK(cudaStreamSynchronize(u->st), "unet synchronize");
  int flag = 0;
  UCK(cudaMemcpy(&flag, u->dev_err, sizeof(int), cudaMemcpyDeviceToHost), "unet error read");
  if (flag) return ufail(u, VIMG_ERR_TIMEOUT, "unet: a tensor-core kernel's bounded wait gave up");
  return VIMG_OK;
}

extern "C" int vimg_unet_profile(vimg_unet* u, int on) {
  if (!u) return ufail(u, VIMG_ERR_ARG, "null U-Net");
  u->prof = on != 0;
  u->ev_used = 0;
  return VIMG_OK;
}

extern "C" int vimg_unet_profile_read(vimg_unet* u, double* conv_ms, double* total_ms,
                                      long long* conv_launches, int reset) {
  if (!u) return ufail(u, VIMG_ERR_ARG, "null U-Net");
  if (conv_ms) *conv_ms = u->conv_ms;
  if (total_ms) *total_ms = u->total_ms;
  if (conv_launches) *conv_launches = u->conv_launches;
  if (reset) {
    u->conv_ms = u->total_ms = 0.0;
    u->conv_launches = 0;
  }
  return VIMG_OK;
}

int unet_dims(const vimg_unet* u, int* H, int* W) {
  if (!u) return -1;
  *H = u->H, *W = u->W;
  return 0;
}

extern "C" int vimg_unet_activation(vimg_unet* u, int i, void* d_out, int* n_patches, int* side_out,
                                    int* channels) {
  if (!u) return ufail(u, VIMG_ERR_ARG, "null U-Net");
  if (u->sticky) return u->sticky;
  const int n_tc = (int)u->convs.size();
  if (i < 0 || i > n_tc + 1) return ufail(u, VIMG_ERR_ARG, "vimg_unet_activation: bad index");
  const int np = u->last_np;
  int sd, C;
  if (i == 0) {
    sd = kUPatch, C = kUC0;
  } else if (i <= n_tc) {
    const ConvParams& p = u->convs[i - 1].p;
    sd = p.so, C = p.up ? p.cout : p.ntile * p.n_ntiles;
  } else {
    sd = kUPatch, C = 1;
  }
  if (n_patches) *n_patches = np;
  if (side_out) *side_out = sd;
  if (channels) *channels = C;
  if (!d_out || np == 0) return VIMG_OK;
  if (i == n_tc + 1) {
    UCK(cudaMemcpyAsync(d_out, u->pprob, sizeof(float) * (size_t)np * kUPatch * kUPatch,
                        cudaMemcpyDeviceToDevice, u->st),
        "unet activation copy");
    return VIMG_OK;
  }
  const __nv_bfloat16* src;
  size_t plane;
  int sp, guard, goff;
  if (i == 0) {
    src = u->in0.p, plane = u->in0.plane, guard = u->in0.guard, sp = stored(0), goff = 0;
  } else {
    const ConvParams& p = u->convs[i - 1].p;
    src = p.out, plane = p.out_plane, guard = p.out_guard, sp = p.spo, goff = p.out_goff;
  }
  const long long n = (long long)np * sd * sd * C;
  k_ucompact<<<grid_for(n, 256, u->sms), 256, 0, u->st>>>(src, plane, guard, goff, np, sd, sp, C,
                                                         static_cast<__nv_bfloat16*>(d_out));
  UCK(cudaGetLastError(), "unet activation copy");
  return VIMG_OK;
}
