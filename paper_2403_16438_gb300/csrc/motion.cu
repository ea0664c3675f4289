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
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>

#include "tc_ptx.h"
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
// Window statistics ("table-based area sums" of Sec. II).  For every window
// top-left position (y, x) of the search region, the exact integers
//   S1 = sum F,  S2 = sum F^2  over the 21x21 window,  SF = 441 S2 - S1^2,
// give isf(y, x) = 1 / sqrt(SF) (0 when SF = 0).  isf does not depend on the
// patch; the patch enters as the scalar 21 / |Tc_p|, so
//   ZNCC_p(d) = numerator_p(d) * 21 / |Tc_p| * isf(ty_p + dy, tx_p + dx).
// The map covers the top-left positions of all windows of all patches:
// rows y0 - R .. y0 + 21 (ny - 1) + R, likewise for columns.  One CTA per
// 56 x 32 block of positions per frame: row sums slide along x, window sums
// slide along y, in exact integers (32-bit squared sums for blocks of moderate
// range, 64-bit otherwise; see box_sums).
constexpr int kGroup = 11;  // patches per FP32 correlation work item (see k_corr_f32)
constexpr int kBoxRows = 56, kBoxCols = 32, kBoxThreads = 256;
constexpr int kBoxIR = kBoxRows + kPatch - 1, kBoxIC = kBoxCols + kPatch - 1;  // 76 x 52 inputs
constexpr int kBoxInStride = kBoxIC + 1;     // 53: odd, so rows fall in distinct banks
constexpr int kBoxRsStride = kBoxCols + 1;   // 33
constexpr int kBoxLoads = (kBoxIR * kBoxIC + kBoxThreads - 1) / kBoxThreads;     // 16

// Stats-map geometry for a patch grid.
__host__ __device__ inline void stats_map_dims(PatchGrid g, int R, int* oy, int* ox, int* sh,
                                               int* sw) {
  *oy = g.y0 - R;
  *ox = g.x0 - R;
  *sh = kPatch * (g.ny - 1) + 2 * R + 1;
  *sw = kPatch * (g.nx - 1) + 2 * R + 1;
}

__host__ __device__ inline int stats_tiles(PatchGrid g, int R) {
  int oy, ox, sh, sw;
  stats_map_dims(g, R, &oy, &ox, &sh, &sw);
  return ((sw + kBoxCols - 1) / kBoxCols) * ((sh + kBoxRows - 1) / kBoxRows);
}

// Pixels of a staged block are taken relative to c = the middle of their range:
// SF = 441 S2 - S1^2 does not change under a common shift, and when every
// |F - c| <= kBoxDev32 the squared sums stay below 2^32 (441 * 3100^2 < 2^32),
// so they run in unsigned 32-bit arithmetic (a slide's intermediate value is
// exact modulo 2^32 and its result is in range).  Wider blocks use 64 bits.
constexpr int kBoxDev32 = 3100;
constexpr int kBoxChunk = 11;  // row-sum positions per job: 76 rows x 3 jobs (11, 11, 10)

template <typename Acc2>
__device__ __forceinline__ Acc2 box_sq(int v) {
  return (Acc2)((long long)v * v);
}

// Row sums, then window sums and the isf outputs of one staged block.
template <typename Acc2>
__device__ __forceinline__ void box_sums(const int* __restrict__ in, int* __restrict__ rs1,
                                         Acc2* __restrict__ rs2, int c, int by, int bx, int sh,
                                         int sw, float* __restrict__ out) {
  // job = (column chunk, row) with the row fastest: the lanes of a warp take
  // consecutive rows, whose strides (53 and 33 words) put them in distinct banks
  for (int job = threadIdx.x; job < kBoxIR * 3; job += kBoxThreads) {
    const int q = job / kBoxIR, r = job - q * kBoxIR, c0 = q * kBoxChunk;
    const int n = min(kBoxChunk, kBoxCols - c0);
    const int* row = in + r * kBoxInStride + c0;
    int s1 = 0;
    Acc2 s2 = 0;
#pragma unroll
    for (int k = 0; k < kPatch; ++k) {
      const int v = row[k] - c;
      s1 += v;
      s2 += box_sq<Acc2>(v);
    }
    int* o1 = rs1 + r * kBoxRsStride + c0;
    Acc2* o2 = rs2 + r * kBoxRsStride + c0;
#pragma unroll
    for (int k = 0; k < kBoxChunk; ++k) {
      if (k < n) {
        o1[k] = s1;
        o2[k] = s2;
        if (k + 1 < n) {  // reads columns up to c0 + n - 1 + 20 <= 51
          const int a = row[k + kPatch] - c, b = row[k] - c;
          s1 += a - b;
          s2 += box_sq<Acc2>(a) - box_sq<Acc2>(b);
        }
      }
    }
  }
  __syncthreads();
  // window sums: 32 columns x 8 chunks of 7 rows
  const int col = threadIdx.x & 31, r0 = (threadIdx.x >> 5) * 7;
  int s1 = 0;  // |S1| <= 441 * 65535 < 2^31
  Acc2 s2 = 0;
#pragma unroll
  for (int k = 0; k < kPatch; ++k) {
    s1 += rs1[(r0 + k) * kBoxRsStride + col];
    s2 += rs2[(r0 + k) * kBoxRsStride + col];
  }
#pragma unroll
  for (int r = r0; r < r0 + 7; ++r) {
    const int y = by + r, x = bx + col;
    const long long sf = (long long)kPatchArea * (long long)s2 - (long long)s1 * s1;
    if (y < sh && x < sw) out[(size_t)y * sw + x] = sf > 0 ? rsqrtf((float)sf) : 0.f;
    if (r + 1 < r0 + 7) {
      s1 += rs1[(r + kPatch) * kBoxRsStride + col] - rs1[r * kBoxRsStride + col];
      s2 += rs2[(r + kPatch) * kBoxRsStride + col] - rs2[r * kBoxRsStride + col];
    }
  }
}

// One CTA per (job, frame, block of positions); the job comes from the prefix
// counts of the table.
__global__ void __launch_bounds__(kBoxThreads, 4)
    k_boxstats(const __grid_constant__ MotionBatch b, const int* __restrict__ list,
               const int* __restrict__ list_n) {
  // Without a list every CTA takes one work item.  With a frame list (fallback
  // frames of the learned proposal; one job) a small grid strides over the
  // listed frames' items, whose count is read on the device.
  int n_items = b.stats_begin[b.n];
  if (list) {
    const MotionJob& J0 = b.j[0];
    n_items = min(J0.nf, *list_n) * stats_tiles(J0.g, J0.R);
  }
  __shared__ int in[kBoxIR * kBoxInStride];
  __shared__ int rs1[kBoxIR * kBoxRsStride];
  __shared__ long long rs2[kBoxIR * kBoxRsStride];  // 32-bit sums use its first half
  __shared__ unsigned wmin[kBoxThreads / 32], wmax[kBoxThreads / 32];
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
  const int jb = list ? 0 : job_of(b.stats_begin, b.n, item);
  const MotionJob& J = b.j[jb];
  const int H = J.H, W = J.W;
  int oy, ox, sh, sw;
  stats_map_dims(J.g, J.R, &oy, &ox, &sh, &sw);
  const int ntx = (sw + kBoxCols - 1) / kBoxCols, per = ntx * ((sh + kBoxRows - 1) / kBoxRows);
  const int local = item - (list ? 0 : b.stats_begin[jb]);
  const int fi = local / per, rem = local - fi * per;
  const int f = list ? list[fi] : fi;
  const int by = (rem / ntx) * kBoxRows, bx = (rem % ntx) * kBoxCols;
  const uint16_t* F = J.frames + (size_t)f * H * W;
  {
    // all loads in flight at once, then the shared stores and the block's range
    unsigned v[kBoxLoads];
#pragma unroll
    for (int k = 0; k < kBoxLoads; ++k) {
      const int i = threadIdx.x + k * kBoxThreads;
      const int r = i / kBoxIC, c = i - r * kBoxIC;
      const int y = min(oy + by + r, H - 1), x = min(ox + bx + c, W - 1);
      v[k] = i < kBoxIR * kBoxIC ? __ldg(F + (size_t)y * W + x) : 0u;
    }
    unsigned mn = 0xffffu, mx = 0u;
#pragma unroll
    for (int k = 0; k < kBoxLoads; ++k) {
      const int i = threadIdx.x + k * kBoxThreads;
      const int r = i / kBoxIC, c = i - r * kBoxIC;
      if (i < kBoxIR * kBoxIC) {
        in[r * kBoxInStride + c] = (int)v[k];
        mn = min(mn, v[k]);
        mx = max(mx, v[k]);
      }
    }
    mn = __reduce_min_sync(0xffffffffu, mn);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0) {
      wmin[threadIdx.x >> 5] = mn;
      wmax[threadIdx.x >> 5] = mx;
    }
  }
  __syncthreads();
  unsigned mn = wmin[0], mx = wmax[0];
#pragma unroll
  for (int w = 1; w < kBoxThreads / 32; ++w) {
    mn = min(mn, wmin[w]);
    mx = max(mx, wmax[w]);
  }
  const int c = (int)((mn + mx) >> 1);
  float* out = J.isf + (size_t)f * sh * sw;
  if ((int)mx - c <= kBoxDev32)
    box_sums<unsigned>(in, rs1, reinterpret_cast<unsigned*>(rs2), c, by, bx, sh, sw, out);
  else
    box_sums<long long>(in, rs1, rs2, c, by, bx, sh, sw, out);
  __syncthreads();  // the shared buffers are reused by the next item
  }
}

// The same statistics with each block's 76 x 52 input tile staged by one 3-D TMA
// box (64 columns from the block's first input column rounded down to a multiple
// of 8, so the copy's x coordinate is 16-byte aligned) instead of 16 indexed
// 16-bit loads per thread: one pass then copies the tile into the odd-stride
// integer layout of box_sums and takes the range of the pixels that in-map
// windows read.  Coordinates outside the image read zeros (in-map windows never
// reach them).  The tile shares its space with the squared row sums, which are
// written only after the copy pass.  Outputs are those of k_boxstats bit for bit
// (exact integer sums, same SF and rsqrtf).
struct StatsMaps {
  CUtensorMap m[kMaxVideos];  // per job: the frames [nf][H][W] (uint16), boxes 64 x 76 x 1
};
constexpr int kBoxTmaW = 64;
constexpr int kBoxTmaBytes = kBoxTmaW * kBoxIR * 2;
constexpr size_t kBoxRs2Bytes = ((size_t)kBoxIR * kBoxRsStride * 8 + 127) & ~(size_t)127;
constexpr size_t kBoxTmaSmem = kBoxRs2Bytes + sizeof(int) * kBoxIR * kBoxInStride +
                               sizeof(int) * kBoxIR * kBoxRsStride + 128;
static_assert(kBoxTmaBytes <= (int)kBoxRs2Bytes, "the staged tile fits the squared row sums");
static_assert(kBoxIC + 7 <= kBoxTmaW, "the box covers the tile after the alignment shift");
static_assert(kBoxTmaSmem <= 48 * 1024, "no shared-memory attribute needed");

__global__ void __launch_bounds__(kBoxThreads, 4)
    k_boxstats_tma(const __grid_constant__ MotionBatch b, const __grid_constant__ StatsMaps maps,
                   const int* __restrict__ list, const int* __restrict__ list_n) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full;
  __shared__ unsigned wmin[kBoxThreads / 32], wmax[kBoxThreads / 32];
  // TMA destinations start on 128-byte boundaries: the dynamic region is
  // aligned here (the launch requests 128 bytes more than the layout needs)
  unsigned char* sm = smem_raw + ((128u - (tc::su32(smem_raw) & 127u)) & 127u);
  long long* rs2 = reinterpret_cast<long long*>(sm);
  const unsigned short* tin = reinterpret_cast<const unsigned short*>(sm);  // [76][64]
  int* in = reinterpret_cast<int*>(sm + kBoxRs2Bytes);
  int* rs1 = in + kBoxIR * kBoxInStride;
  int n_items = b.stats_begin[b.n];
  if (list) {
    const MotionJob& J0 = b.j[0];
    n_items = min(J0.nf, *list_n) * stats_tiles(J0.g, J0.R);
  }
  if (threadIdx.x == 0) {
    tc::mbar_init(&full, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t phase = 0;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int jb = list ? 0 : job_of(b.stats_begin, b.n, item);
    const MotionJob& J = b.j[jb];
    int oy, ox, sh, sw;
    stats_map_dims(J.g, J.R, &oy, &ox, &sh, &sw);
    const int ntx = (sw + kBoxCols - 1) / kBoxCols, per = ntx * ((sh + kBoxRows - 1) / kBoxRows);
    const int local = item - (list ? 0 : b.stats_begin[jb]);
    const int fi = local / per, rem = local - fi * per;
    const int f = list ? list[fi] : fi;
    const int by = (rem / ntx) * kBoxRows, bx = (rem % ntx) * kBoxCols;
    const int x = ox + bx, x0 = x & ~7, oxs = x - x0;  // ox >= 0
    if (threadIdx.x == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // after the last item's reads
      tc::mbar_expect_tx(&full, kBoxTmaBytes);
      tc::tma_load_3d(sm, &maps.m[jb], x0, oy + by, f, &full);
    }
    const bool late = !tc::mbar_wait(&full, phase);
    if (__syncthreads_or(late)) {  // give up on the whole block, report, drain the copy
      if (threadIdx.x == 0) {
        if (J.err) atomicExch(J.err, 1);
        tc::mbar_wait(&full, phase);
      }
      return;
    }
    phase ^= 1u;
    // tile -> odd-stride integers; range of the pixels in-map windows read
    const int ir = min(kBoxIR, sh - by + kPatch - 1), ic = min(kBoxIC, sw - bx + kPatch - 1);
    unsigned mn = 0xffffu, mx = 0u;
    {
      const int cc = threadIdx.x & 63;
      for (int r = threadIdx.x >> 6; r < kBoxIR; r += kBoxThreads / 64) {
        if (cc < kBoxIC) {
          const unsigned v = tin[r * kBoxTmaW + oxs + cc];
          in[r * kBoxInStride + cc] = (int)v;
          if (r < ir && cc < ic) {
            mn = min(mn, v);
            mx = max(mx, v);
          }
        }
      }
    }
    mn = __reduce_min_sync(0xffffffffu, mn);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0) {
      wmin[threadIdx.x >> 5] = mn;
      wmax[threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    mn = wmin[0], mx = wmax[0];
#pragma unroll
    for (int w = 1; w < kBoxThreads / 32; ++w) {
      mn = min(mn, wmin[w]);
      mx = max(mx, wmax[w]);
    }
    const int c = (int)((mn + mx) >> 1);
    float* out = J.isf + (size_t)f * sh * sw;
    if ((int)mx - c <= kBoxDev32)
      box_sums<unsigned>(in, rs1, reinterpret_cast<unsigned*>(rs2), c, by, bx, sh, sw, out);
    else
      box_sums<long long>(in, rs1, rs2, c, by, bx, sh, sw, out);
    __syncthreads();  // the tile space and the shared buffers are reused by the next item
  }
}

// 3-D TMA map of a uint16 frame buffer [n][H][W], boxes box_w x box_h x 1.
static bool frames_map_3d(CUtensorMap* m, const uint16_t* base, int n, int H, int W, int box_w,
                          int box_h) {
  tc::EncodeTiledFn fn = tc::encode_fn();
  if (!fn || !base || n < 1) return false;
  cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)n};
  cuuint64_t strides[2] = {(cuuint64_t)W * 2, (cuuint64_t)H * W * 2};
  cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<uint16_t*>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t stats_map_floats(PatchGrid g, int R) {
  int oy, ox, sh, sw;
  stats_map_dims(g, R, &oy, &ox, &sh, &sw);
  return (size_t)sh * sw;
}

static MotionJob one_job(const uint16_t* frames, int nf, int H, int W, PatchGrid g, int R,
                         const TemplateDev& td, float* isf, unsigned long long* csum) {
  MotionJob j{};
  j.frames = frames, j.nf = nf, j.H = H, j.W = W, j.g = g, j.R = R;
  j.tc = td.tc, j.tn2 = td.tn2, j.coff = td.coff, j.isf = isf, j.csum = csum;
  return j;
}

bool motion_batch_finalize(MotionBatch& b) {
  if (b.n < 1 || b.n > kMaxVideos) return false;
  long long s = 0, c = 0, p = 0;
  b.stats_begin[0] = b.corr_begin[0] = b.peak_begin[0] = 0;
  for (int i = 0; i < b.n; ++i) {
    const MotionJob& J = b.j[i];
    if (J.nf < 0 || J.R < 0 || J.R > kMaxR || J.g.ny < 1 || J.g.nx < 1) return false;
    s += (long long)J.nf * stats_tiles(J.g, J.R);
    c += (long long)J.nf * J.g.ny * ((J.g.nx + kGroup - 1) / kGroup);
    p += J.nf;
    if (s > INT_MAX || c > INT_MAX) return false;
    b.stats_begin[i + 1] = (int)s;
    b.corr_begin[i + 1] = (int)c;
    b.peak_begin[i + 1] = (int)p;
  }
  return true;
}

cudaError_t launch_stats_multi(const MotionBatch& b, cudaStream_t st, const int* list,
                               const int* list_n) {
  int blocks = b.stats_begin[b.n];
  if (blocks <= 0) return cudaSuccess;
  if (list) {  // one wave of CTAs that stride over the listed frames' items
    cudaError_t e = kernels_init();
    if (e != cudaSuccess) return e;
    blocks = std::min(blocks, 4 * sm_count());
  }
  // the TMA-staged kernel when every job can report a wait that gave up and
  // its frames allow 16-byte aligned boxes
  StatsMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  bool tma = true;
  for (int i = 0; i < b.n && tma; ++i) {
    const MotionJob& J = b.j[i];
    if (J.nf == 0) continue;
    tma = J.err != nullptr && J.W % 8 == 0 &&
          (reinterpret_cast<uintptr_t>(J.frames) & 15) == 0 &&
          frames_map_3d(&maps.m[i], J.frames, J.nf, J.H, J.W, kBoxTmaW, kBoxIR);
  }
  if (tma)
    k_boxstats_tma<<<blocks, kBoxThreads, kBoxTmaSmem, st>>>(b, maps, list, list_n);
  else
    k_boxstats<<<blocks, kBoxThreads, 0, st>>>(b, list, list_n);
  return cudaGetLastError();
}

cudaError_t launch_stats(const uint16_t* frames, int nf, int H, int W, PatchGrid g, int R,
                         const TemplateDev& td, float* isf, cudaStream_t st, const int* list,
                         const int* list_n, int* err) {
  if (nf <= 0) return cudaSuccess;
  MotionBatch b{};
  b.n = 1;
  b.j[0] = one_job(frames, nf, H, W, g, R, td, isf, nullptr);
  b.j[0].err = err;
  if (!motion_batch_finalize(b)) return cudaErrorInvalidValue;
  return launch_stats_multi(b, st, list, list_n);
}

// ---------------------------------------------------------------------------
// FP32 correlation numerators on CUDA cores.
//
// Work item = (frame, patch row, group of up to kGroup = 11 patches).  The union
// of the group's search regions (53 rows x (21 G + 2R) cols) is staged in shared
// memory as exact fp32 integers F - c, with the block of the isf map those
// windows use.  Twelve warps then each own one output-row pass:
//   pass u < G:   lane = dy in 0..31, all lanes on patch u (template loads are
//                 warp-uniform, frame rows distinct);
//   pass G:       the 33rd displacement row (dy = 32, when 2R+1 = 33) of all G
//                 patches, lane = (u, half of the columns), 17 columns per lane.
// A lane streams the 21 frame rows it needs: per row 53 shared loads feed
// 21 x 33 FMAs into 33 register accumulators (37 loads, 21 x 17 FMAs in pass G).  Each finished row is normalised
// and added in 2^-40 fixed point to the item's int64 surface in shared memory,
// which is finally added to the frame's global sums.
//
// The kernel is persistent: one CTA per SM with two 12-warp consumer groups,
// each with its own shared buffers.  Group 1 starts once group 0 has staged its
// first item, so from then on one group's staging (global-memory latency) runs
// while the other group computes, and the SM's FMA pipes stay busy.
//
// The group size GP (patches per work item, 11 by default) is a template
// parameter: a CTA holds two groups of GP + 1 warps.  A row of nx patches takes
// ceil(nx / GP) items, so GP = 11 fills every group on 22-patch rows (512 px)
// while 7 or 8 fit 35- or 47-patch rows (768 or 1,024 px) better; the per-item
// arithmetic does not depend on GP except through the offset c of the item's
// first patch (F - c is exact, so only the rounding of the FP32 sums moves).
constexpr int kCsEntries = kMaxWin * kMaxWin + 1;  // keeps what follows 16-byte aligned
constexpr int kRegionRows = kPatch + 2 * kMaxR;                     // 53
constexpr int kHalfRow = 17;  // columns per lane in the 33rd-row pass (0..16 or 16..32)
// Region row stride for a group of G patches: at least one column beyond the
// G * 21 + 32 that the windows read (a lane's last 8-byte pair may reach one
// column past its 53 values), and 2 mod 4, so that lanes on consecutive rows
// reading 8-byte pairs fall in distinct banks (rs / 2 odd).
__host__ __device__ constexpr int corr_region_stride(int G) {
  return G * kPatch + 2 * kMaxR + 1 + ((2 - (G * kPatch + 2 * kMaxR + 1) % 4) + 4) % 4;
}

static_assert(corr_region_stride(11) == 266 && corr_region_stride(10) == 246 &&
                  corr_region_stride(8) == 202 && corr_region_stride(7) == 182,
              "region strides of the patch-group sizes");

template <int GP>
struct CorrGeom {
  static_assert(GP >= 2 && GP <= 16, "the 33rd-row pass maps 16 patches x 2 column halves");
  static constexpr int kWarps = GP + 1;                            // per group
  static constexpr int kThreads = 32 * kWarps;                     // per group
  static constexpr int kCta = 2 * kThreads;                        // two groups
  static constexpr int kStride = corr_region_stride(GP);          // region row stride
  static constexpr int kIsf = (GP - 1) * kPatch + kMaxWin;         // isf columns
  static constexpr int kIsfFloats = (kMaxWin * kIsf + 3) & ~3;     // keeps the region 16-B aligned
  static constexpr size_t kSmem =                                  // per group, 16-byte multiple
      (sizeof(unsigned long long) * kCsEntries + sizeof(float) * kIsfFloats +
       sizeof(float) * kRegionRows * kStride + 15) & ~(size_t)15;
};

// floor(i / d) as a multiply-high by m = ceil(2^32 / d): exact for i < 2^32 / d,
// far above any index here (d <= 266, i < 14,100).
__device__ __forceinline__ unsigned fast_div(unsigned i, unsigned m) { return __umulhi(i, m); }

template <int N>
__device__ __forceinline__ void group_sync(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(N) : "memory");
}

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
      const float4 v = __ldg(reinterpret_cast<const float4*>(trow + i));
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

// corr_row with the frame values read as 8-byte pairs: rrow - SH is 8-byte
// aligned (SH = the parity of the row start), rs is even, and the window's
// values are the pairs' elements SH .. SH + NX + 19; the FMAs and their order
// are those of corr_row.
template <int NX, int SH>
__device__ __forceinline__ void corr_row_pairs(const float* __restrict__ rrow, int rs,
                                               const float* __restrict__ trow,
                                               float (&acc)[NX]) {
  constexpr int kPairs = (NX + kPatch - 1 + SH + 1) / 2;
#pragma unroll
  for (int j = 0; j < NX; ++j) acc[j] = 0.f;
  const float2* rp = reinterpret_cast<const float2*>(rrow - SH);
  const int rs2 = rs >> 1;
#pragma unroll 1
  for (int ky = 0; ky < kPatch; ++ky) {
    float fr[2 * kPairs];
#pragma unroll
    for (int i = 0; i < kPairs; ++i) {
      const float2 v = rp[i];
      fr[2 * i] = v.x, fr[2 * i + 1] = v.y;
    }
    float t[kTplStride];
#pragma unroll
    for (int i = 0; i < kTplStride; i += 4) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(trow + i));
      t[i] = v.x, t[i + 1] = v.y, t[i + 2] = v.z, t[i + 3] = v.w;
    }
#pragma unroll
    for (int kx = 0; kx < kPatch; ++kx)
#pragma unroll
      for (int j = 0; j < NX; ++j) acc[j] = fmaf(t[kx], fr[SH + j + kx], acc[j]);
    rp += rs2;
    trow += kTplStride;
  }
}

// kPairs: the frame values of a row are read as 8-byte pairs (rows of stride
// corr_region_stride(G)); otherwise as single words from rows of odd stride.
// Pairs save load instructions, which pays on wide frames whose groups of
// many warps compete for issue; the single-word form, with one copy of the row
// loop, is faster where the groups have few patches (latency-bound).
template <int NX, int GP, bool kPairs>
__global__ void __launch_bounds__(CorrGeom<GP>::kCta, 1)
    k_corr_f32(const __grid_constant__ MotionBatch b, const int* __restrict__ list,
               const int* __restrict__ list_n) {
  using C = CorrGeom<GP>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int grp = threadIdx.x / C::kThreads, gtid = threadIdx.x - grp * C::kThreads;
  const int lane = gtid & 31, gwarp = gtid >> 5;
  unsigned long long* cs = reinterpret_cast<unsigned long long*>(smem + grp * C::kSmem);
  float* ism = reinterpret_cast<float*>(cs + kCsEntries);  // [w][scols]
  float* reg = ism + C::kIsfFloats;                      // [rows][rs], 16-byte aligned
  // With a frame list (fallback frames of the learned proposal; one job) only the
  // listed frames are processed; their count is read from device memory.
  int n_items = b.corr_begin[b.n];
  if (list) {
    const PatchGrid g0 = b.j[0].g;
    n_items = min(b.j[0].nf, *list_n) * g0.ny * ((g0.nx + GP - 1) / GP);
  }
  const int bar = 1 + grp;  // named barrier of this group (0 is __syncthreads)

  if (grp == 1) asm volatile("bar.sync 3, %0;" ::"r"(C::kCta) : "memory");
  bool released = false;
  for (int k = grp;; k += 2) {
    const int item = blockIdx.x + k * gridDim.x;
    if (item >= n_items) break;
    const int jb = list ? 0 : job_of(b.corr_begin, b.n, item);
    const MotionJob& J = b.j[jb];
    const PatchGrid g = J.g;
    const int R = J.R, H = J.H, W = J.W;
    const int w = 2 * R + 1, rows = kPatch + 2 * R;
    const int groups_per_row = (g.nx + GP - 1) / GP;
    const int items_per_frame = g.ny * groups_per_row;
    int oy, ox, sh, sw;
    stats_map_dims(g, R, &oy, &ox, &sh, &sw);
    const int local = item - (list ? 0 : b.corr_begin[jb]);
    const int fi = local / items_per_frame, rem = local - fi * items_per_frame;
    const int f = list ? list[fi] : fi;
    const uint16_t* __restrict__ frames = J.frames;
    const float* __restrict__ tc = J.tc;
    const float* __restrict__ tn2 = J.tn2;
    const float* __restrict__ isf = J.isf;
    unsigned long long* __restrict__ csum = J.csum;
    const int py = rem / groups_per_row, gx = rem - py * groups_per_row;
    const int px0 = gx * GP, G = min(GP, g.nx - px0);
    const int cols = G * kPatch + 2 * R;
    // Rows are allocated for the widest window (a lane always reads 53 values);
    // the stride lets lanes on different rows read 8-byte pairs from distinct banks.
    const int rs = kPairs ? corr_region_stride(G) : ((G * kPatch + 2 * kMaxR) | 1);  // <= C::kStride
    const int scols = (G - 1) * kPatch + w;       // isf columns this item uses
    const int ry = g.y0 + py * kPatch - R, rx = g.x0 + px0 * kPatch - R;
    const int p0 = py * g.nx + px0;
    const float c = (float)J.coff[p0];

    // Stage: every thread first issues its global loads (one round trip per
    // batch), then converts and stores.
    for (int i = gtid; i < w * w; i += C::kThreads) cs[i] = 0ull;
    const float* isf_f = isf + (size_t)f * sh * sw + (size_t)(ry - oy) * sw + (rx - ox);
    const uint16_t* F = frames + (size_t)f * H * W + (size_t)ry * W + rx;
    {
      constexpr int kRegLoads = (kRegionRows * C::kStride + C::kThreads - 1) / C::kThreads;
      constexpr int kBatches = 3;  // batches of loads keep the registers in budget
      constexpr int kHalf = (kRegLoads + kBatches - 1) / kBatches;
      const unsigned m = 0xffffffffu / (unsigned)rs + 1u;
#pragma unroll 1
      for (int b = 0; b < kBatches; ++b) {
        unsigned short v[kHalf];
#pragma unroll
        for (int q = 0; q < kHalf; ++q) {
          const int i = gtid + (b * kHalf + q) * C::kThreads;
          const int r = (int)fast_div((unsigned)i, m), x = i - r * rs;
          v[q] = (i < rows * rs && x < cols) ? __ldg(F + (size_t)r * W + x) : (unsigned short)0;
        }
#pragma unroll
        for (int q = 0; q < kHalf; ++q) {
          const int i = gtid + (b * kHalf + q) * C::kThreads;
          const int x = i - (int)fast_div((unsigned)i, m) * rs;
          if (i < rows * rs) reg[i] = x < cols ? (float)v[q] - c : 0.f;
        }
      }
    }
    {
      constexpr int kIsfLoads = (kMaxWin * C::kIsf + C::kThreads - 1) / C::kThreads;
      constexpr int kIsfHalf = (kIsfLoads + 1) / 2;
      const unsigned m = 0xffffffffu / (unsigned)scols + 1u;
#pragma unroll 1
      for (int b = 0; b < 2; ++b) {
        float v[kIsfHalf];
#pragma unroll
        for (int q = 0; q < kIsfHalf; ++q) {
          const int i = gtid + (b * kIsfHalf + q) * C::kThreads;
          const int r = (int)fast_div((unsigned)i, m), x = i - r * scols;
          v[q] = i < w * scols ? __ldg(isf_f + (size_t)r * sw + x) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < kIsfHalf; ++q) {
          const int i = gtid + (b * kIsfHalf + q) * C::kThreads;
          if (i < w * scols) ism[i] = v[q];
        }
      }
    }
    group_sync<C::kThreads>(bar);
    if (grp == 0 && !released) {  // let group 1 start staging now
      asm volatile("bar.arrive 3, %0;" ::"r"(C::kCta) : "memory");
      released = true;
    }
    // One output-row pass per warp.
    const int n_pass = G + (w > 32 ? 1 : 0);
    for (int pass = gwarp; pass < n_pass; pass += C::kWarps) {
      if (pass < G) {
        const int u = pass, dy = lane;
        const bool active = dy < w;
        const int dd = active ? dy : 0;
        float acc[NX];
        // the row start's parity is u's (21 is odd, rs even): warp-uniform
        const float* rstart = reg + dd * rs + u * kPatch;
        const float* tp = tc + (size_t)(p0 + u) * kPatch * kTplStride;
        if constexpr (kPairs) {
          if (u & 1)
            corr_row_pairs<NX, 1>(rstart, rs, tp, acc);
          else
            corr_row_pairs<NX, 0>(rstart, rs, tp, acc);
        } else {
          corr_row<NX>(rstart, rs, tp, acc);
        }
        if (active) {
          const float t2 = __ldg(tn2 + p0 + u);
          const float pscale = t2 > 0.f ? (float)kPatch * rsqrtf(t2) : 0.f;
          const float* iv = ism + dd * scols + u * kPatch;
          unsigned long long* crow = cs + dd * w;
#pragma unroll
          for (int j = 0; j < NX; ++j) {
            if (j < w) {
              const float z = acc[j] * pscale * iv[j];
              atomicAdd(crow + j, (unsigned long long)__float2ll_rn(z * (float)kFix));
            }
          }
        }
      } else {
        // The 33rd displacement row (dy = 32; this pass exists only for 2R + 1 = 33)
        // of all G patches: lane = (u = lane & 15, columns 0..16 or 16..32), 17
        // accumulators each, column 16 kept by the first half.
        const int u = lane & 15, half = lane >> 4, dx0 = 16 * half;
        const bool active = u < G;
        const int uu = active ? u : 0;
        float acc[kHalfRow];
        corr_row<kHalfRow>(reg + 32 * rs + uu * kPatch + dx0, rs,
                           tc + (size_t)(p0 + uu) * kPatch * kTplStride, acc);
        if (active) {
          const float t2 = __ldg(tn2 + p0 + uu);
          const float pscale = t2 > 0.f ? (float)kPatch * rsqrtf(t2) : 0.f;
          const float* iv = ism + 32 * scols + uu * kPatch + dx0;
          unsigned long long* crow = cs + 32 * w + dx0;
#pragma unroll
          for (int j = 0; j < kHalfRow; ++j) {
            if (half == 0 || j > 0) {
              const float z = acc[j] * pscale * iv[j];
              atomicAdd(crow + j, (unsigned long long)__float2ll_rn(z * (float)kFix));
            }
          }
        }
      }
    }
    group_sync<C::kThreads>(bar);
    unsigned long long* out = csum + (size_t)f * w * w;
    for (int i = gtid; i < w * w; i += C::kThreads) atomicAdd(out + i, cs[i]);
    group_sync<C::kThreads>(bar);
  }
  if (grp == 0 && !released) asm volatile("bar.arrive 3, %0;" ::"r"(C::kCta) : "memory");
}

static int g_sms[kMaxDevices] = {};
static unsigned char g_sms_done[kMaxDevices] = {};
static unsigned char g_kernels_done[kMaxDevices] = {};

int sm_count() {
  const cudaError_t e = once_per_device(g_sms_done, [](int dev) {
    int sms = 0;
    const cudaError_t r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (r == cudaSuccess) g_sms[dev] = sms;
    return r;
  });
  const int dev = current_device();
  return e == cudaSuccess && dev >= 0 ? g_sms[dev] : 0;
}

template <int GP>
static cudaError_t corr_attr() {
  cudaError_t e = cudaFuncSetAttribute(k_corr_f32<kMaxWin, GP, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(2 * CorrGeom<GP>::kSmem));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_corr_f32<kMaxWin, GP, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * CorrGeom<GP>::kSmem));
  return e;
}

cudaError_t kernels_init() {
  return once_per_device(g_kernels_done, [](int) {
    if (sm_count() <= 0) return cudaErrorInvalidDevice;
    cudaError_t e = corr_attr<11>();
    if (e == cudaSuccess) e = corr_attr<10>();
    if (e == cudaSuccess) e = corr_attr<8>();
    if (e == cudaSuccess) e = corr_attr<7>();
    if (e == cudaSuccess) e = temporal_init();
    return e;
  });
}

bool corr_group_valid(int cg) { return cg == 0 || cg == 7 || cg == 8 || cg == 10 || cg == 11; }

// Pair loads for a job: at least two groups per patch row, so that the
// groups are mostly full.
static bool corr_pairs_for(const MotionJob& J, int GP) { return J.g.nx >= 2 * GP; }

// The jobs of b whose group size is GP (and whose load form is kPairs), with
// their work items counted in groups of GP patches, in one launch.
template <int GP, bool kPairs>
static cudaError_t launch_corr_group(const MotionBatch& b, cudaStream_t st, const int* list,
                                     const int* list_n) {
  MotionBatch s{};
  long long c = 0;
  for (int i = 0; i < b.n; ++i) {
    const MotionJob& J = b.j[i];
    if ((J.cg ? J.cg : kGroup) != GP || corr_pairs_for(J, GP) != kPairs) continue;
    s.j[s.n] = J;
    c += (long long)J.nf * J.g.ny * ((J.g.nx + GP - 1) / GP);
    if (c > INT_MAX) return cudaErrorInvalidValue;
    s.corr_begin[++s.n] = (int)c;
  }
  if (s.n == 0 || c == 0) return cudaSuccess;
  const int grid = std::min(sm_count(), (int)((c + 1) / 2));
  k_corr_f32<kMaxWin, GP, kPairs><<<grid, CorrGeom<GP>::kCta, 2 * CorrGeom<GP>::kSmem, st>>>(
      s, list, list_n);
  return cudaGetLastError();
}

cudaError_t launch_corr_f32_multi(const MotionBatch& b, cudaStream_t st, const int* list,
                                  const int* list_n) {
  const int items = b.corr_begin[b.n];
  if (items <= 0) return cudaSuccess;
  for (int i = 0; i < b.n; ++i)
    if (!corr_group_valid(b.j[i].cg)) return cudaErrorInvalidValue;
  cudaError_t e = kernels_init();
  if (e == cudaSuccess) e = launch_corr_group<11, true>(b, st, list, list_n);
  if (e == cudaSuccess) e = launch_corr_group<11, false>(b, st, list, list_n);
  if (e == cudaSuccess) e = launch_corr_group<10, true>(b, st, list, list_n);
  if (e == cudaSuccess) e = launch_corr_group<10, false>(b, st, list, list_n);
  if (e == cudaSuccess) e = launch_corr_group<8, true>(b, st, list, list_n);
  if (e == cudaSuccess) e = launch_corr_group<8, false>(b, st, list, list_n);
  if (e == cudaSuccess) e = launch_corr_group<7, true>(b, st, list, list_n);
  if (e == cudaSuccess) e = launch_corr_group<7, false>(b, st, list, list_n);
  return e;
}

cudaError_t launch_corr_f32(const uint16_t* frames, int nf, int H, int W, PatchGrid g, int R,
                            const TemplateDev& td, const float* isf,
                            unsigned long long* csum, cudaStream_t st, const int* list,
                            const int* list_n, int cg) {
  if (nf <= 0) return cudaSuccess;
  MotionBatch b{};
  b.n = 1;
  b.j[0] = one_job(frames, nf, H, W, g, R, td, const_cast<float*>(isf), csum);
  b.j[0].cg = cg;
  if (!motion_batch_finalize(b)) return cudaErrorInvalidValue;
  return launch_corr_f32_multi(b, st, list, list_n);
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

// Integer peak (with the tie-break) and parabola over a wy x wx surface whose
// (0,0) entry is displacement (oy, ox).  Writes the shift, the peak info and,
// for the full window, the surface.  Returns the flat index of d*.
__device__ __forceinline__ int peak_of(const long long* C, int wy, int wx, int oy, int ox, int np,
                                       int lane, Cand& best, Cand& second, float s[2]) {
  const Cand none = {LLONG_MIN, 0x7fffffff, -1};
  const int nw = wy * wx;
  Cand b = none;
  for (int i = lane; i < nw; i += 32) {
    const int dy = i / wx + oy, dx = i % wx + ox;
    Cand c = {C[i], ((dy * dy + dx * dx) << 12) | ((dy + 16) << 6) | (dx + 16), i};
    if (better(c, b)) b = c;
  }
  b = warp_best(b);
  Cand s2 = none;
  for (int i = lane; i < nw; i += 32) {
    if (i == b.idx) continue;
    const int dy = i / wx + oy, dx = i % wx + ox;
    Cand c = {C[i], ((dy * dy + dx * dx) << 12) | ((dy + 16) << 6) | (dx + 16), i};
    if (better(c, s2)) s2 = c;
  }
  s2 = warp_best(s2);
  const int iy = b.idx / wx, ix = b.idx % wx;
  s[0] = (float)(iy + oy);
  s[1] = (float)(ix + ox);
  for (int ax = 0; ax < 2; ++ax) {
    const int i = ax == 0 ? iy : ix, n = ax == 0 ? wy : wx;
    if (i == 0 || i == n - 1) continue;
    const int step = ax == 0 ? wx : 1;
    const long long cm = C[b.idx - step], cp = C[b.idx + step], c0 = C[b.idx];
    const long long den = cm - 2 * c0 + cp;
    if (den >= 0) continue;
    float d = (float)(cm - cp) / (2.0f * (float)den);
    d = fminf(0.5f, fmaxf(-0.5f, d));
    s[ax] += d;
  }
  best = b;
  second = s2;
  (void)np;
  return b.idx;
}

__global__ void k_peak(const __grid_constant__ MotionBatch mb, const int* __restrict__ list,
                       const int* __restrict__ list_n) {
  if (list && (int)blockIdx.x >= *list_n) return;
  const int jb = list ? 0 : job_of(mb.peak_begin, mb.n, blockIdx.x);
  const MotionJob& J = mb.j[jb];
  const int f = list ? list[blockIdx.x] : (int)blockIdx.x - mb.peak_begin[jb];
  const int R = J.R, np = J.g.ny * J.g.nx;
  const unsigned long long* __restrict__ csum = J.csum;
  float* __restrict__ shifts = J.shifts;
  float* __restrict__ info = J.info;
  double* __restrict__ surface = J.surface;
  const int lane = threadIdx.x, w = 2 * R + 1, nw = w * w;
  const long long* C = reinterpret_cast<const long long*>(csum) + (size_t)f * nw;
  Cand b, s2;
  float s[2];
  peak_of(C, w, w, -R, -R, np, lane, b, s2, s);
  if (surface) {
    for (int i = lane; i < nw; i += 32) surface[(size_t)f * nw + i] = (double)C[i] / kFix / np;
  }
  if (lane == 0) {
    if (shifts) {
      shifts[2 * f] = s[0];
      shifts[2 * f + 1] = s[1];
    }
    if (info) {
      info[4 * f + 0] = (float)(b.idx / w - R);
      info[4 * f + 1] = (float)(b.idx % w - R);
      info[4 * f + 2] = (float)((double)b.v / kFix / np);
      info[4 * f + 3] = s2.idx >= 0 ? (float)((double)s2.v / kFix / np) : 0.f;
    }
  }
}

cudaError_t launch_peak_multi(const MotionBatch& b, cudaStream_t st, const int* list,
                              const int* list_n) {
  const int blocks = b.peak_begin[b.n];
  if (blocks <= 0) return cudaSuccess;
  k_peak<<<blocks, 32, 0, st>>>(b, list, list_n);
  return cudaGetLastError();
}

cudaError_t launch_peak(const unsigned long long* csum, int nf, int R, int np, float* shifts,
                        float* peak_info, double* surface, cudaStream_t st, const int* list,
                        const int* list_n) {
  if (nf <= 0) return cudaSuccess;
  MotionBatch b{};
  b.n = 1;
  MotionJob& j = b.j[0];
  j.csum = const_cast<unsigned long long*>(csum);
  j.nf = nf, j.R = R, j.g = PatchGrid{1, np, 0, 0};
  j.shifts = shifts, j.info = peak_info, j.surface = surface;
  b.peak_begin[0] = 0, b.peak_begin[1] = nf;
  return launch_peak_multi(b, st, list, list_n);
}

// ---------------------------------------------------------------------------
// Narrow window around a proposed shift p_t (learned proposal): the 7x7
// displacements centred on c_t = round(p_t) (clamped so the window stays in
// [-R, R]^2), i.e. +-2 px plus a one-pixel ring for the refinement.  CTA = 24
// patches x 8 lanes (lane = displacement row), the union of the group's 27-row
// regions staged in shared memory.  Same normalisation and fixed-point sums as
// the full window.
constexpr int kNarrow = kNarrowWin;  // 7
constexpr int kNarrowGroup = 24;     // patches per CTA (one patch row, or part of it)
// staged row stride (floats): at least 24 x 21 + 6, and = 4 (mod 32) so that the
// 32 lanes of a warp (4 patches 21 words apart x 8 rows) read distinct banks
constexpr int kNarrowStride = ((kNarrowGroup * kPatch + kNarrow - 1 - 4 + 31) & ~31) + 4;
static_assert(kNarrowStride % 32 == 4 && kNarrowStride >= kNarrowGroup * kPatch + kNarrow - 1,
              "narrow region stride");

__device__ __forceinline__ void narrow_center(const float* prop, int f, int R, int& cy, int& cx) {
  // prop holds the network output (shift / kShiftScale)
  const int lim = R - kNarrow / 2;
  const float py = prop[2 * f] * kShiftScale, px = prop[2 * f + 1] * kShiftScale;
  cy = isfinite(py) ? (int)rintf(fmaxf(-64.f, fminf(64.f, py))) : 0;
  cx = isfinite(px) ? (int)rintf(fmaxf(-64.f, fminf(64.f, px))) : 0;
  cy = max(-lim, min(lim, cy));
  cx = max(-lim, min(lim, cx));
}

__global__ void __launch_bounds__(kNarrowGroup * 8, 4)
    k_corr_narrow(const uint16_t* __restrict__ frames, int H, int W, PatchGrid g, int R,
                  const float* __restrict__ tc, const float* __restrict__ tn2,
                  const float* __restrict__ isf, const float* __restrict__ prop,
                  unsigned long long* __restrict__ csum) {
  extern __shared__ __align__(16) float nreg[];  // [27][nrs] frame region - c
  __shared__ unsigned long long cs[kNarrow * kNarrow];
  // frames vary fastest over the grid, so the CTAs resident on an SM at a time
  // mostly share one patch group, whose template rows then stay in L1
  const int f = blockIdx.x;
  const int gpr = (g.nx + kNarrowGroup - 1) / kNarrowGroup;
  const int py = blockIdx.y / gpr, px0 = (blockIdx.y % gpr) * kNarrowGroup;
  const int G = min(kNarrowGroup, g.nx - px0);
  const int u = threadIdx.x >> 3, dy = threadIdx.x & 7;
  int cy, cx;
  narrow_center(prop, f, R, cy, cx);
  const int wy0 = cy - kNarrow / 2, wx0 = cx - kNarrow / 2;
  const int rows = kNarrow + kPatch - 1, cols = G * kPatch + kNarrow - 1;
  const int nrs = kNarrowStride;
  const int ty = g.y0 + py * kPatch, tx0 = g.x0 + px0 * kPatch;
  for (int i = threadIdx.x; i < kNarrow * kNarrow; i += blockDim.x) cs[i] = 0ull;
  // stage the union of the group's narrow regions: batches of independent loads
  // (coalesced along rows), then the shared stores
  const uint16_t* F = frames + (size_t)f * H * W + (size_t)(ty + wy0) * W + tx0 + wx0;
  {
    constexpr int kBatch = 12;
    const int total = rows * cols;
    const unsigned m = 0xffffffffu / (unsigned)cols + 1u;  // i / cols exact for i < 2^32 / cols
    for (int base = threadIdx.x; base < total; base += kBatch * blockDim.x) {
      unsigned short v[kBatch];
#pragma unroll
      for (int q = 0; q < kBatch; ++q) {
        const int i = base + q * blockDim.x;
        const int r = (int)fast_div((unsigned)i, m), x = i - r * cols;
        v[q] = i < total ? __ldg(F + (size_t)r * W + x) : (unsigned short)0;
      }
#pragma unroll
      for (int q = 0; q < kBatch; ++q) {
        const int i = base + q * blockDim.x;
        const int r = (int)fast_div((unsigned)i, m), x = i - r * cols;
        if (i < total) nreg[r * nrs + x] = (float)v[q];
      }
    }
  }
  __syncthreads();
  if (u < G && dy < kNarrow) {
    const int p = py * g.nx + px0 + u;
    const float* rrow = nreg + dy * nrs + u * kPatch;
    const float* trow = tc + (size_t)p * kPatch * kTplStride;
    float acc[kNarrow];
#pragma unroll
    for (int j = 0; j < kNarrow; ++j) acc[j] = 0.f;
#pragma unroll 1
    for (int ky = 0; ky < kPatch; ++ky) {
      float fr[kNarrow + kPatch - 1];
#pragma unroll
      for (int i = 0; i < kNarrow + kPatch - 1; ++i) fr[i] = rrow[i];
      float t[kTplStride];
#pragma unroll
      for (int i = 0; i < kTplStride; i += 4) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(trow + i));
        t[i] = v.x, t[i + 1] = v.y, t[i + 2] = v.z, t[i + 3] = v.w;
      }
#pragma unroll
      for (int kx = 0; kx < kPatch; ++kx)
#pragma unroll
        for (int j = 0; j < kNarrow; ++j) acc[j] = fmaf(t[kx], fr[j + kx], acc[j]);
      rrow += nrs;
      trow += kTplStride;
    }
    int oy, ox, sh, sw;
    stats_map_dims(g, R, &oy, &ox, &sh, &sw);
    const float t2 = __ldg(tn2 + p);
    const float pscale = t2 > 0.f ? (float)kPatch * rsqrtf(t2) : 0.f;
    const int txp = tx0 + u * kPatch;
    const float* iv = isf + (size_t)f * sh * sw + (size_t)(ty + wy0 + dy - oy) * sw + (txp + wx0 - ox);
#pragma unroll
    for (int j = 0; j < kNarrow; ++j) {
      const float z = acc[j] * pscale * __ldg(iv + j);
      atomicAdd(cs + dy * kNarrow + j, (unsigned long long)__float2ll_rn(z * (float)kFix));
    }
  }
  __syncthreads();
  unsigned long long* out = csum + (size_t)f * kNarrow * kNarrow;
  for (int i = threadIdx.x; i < kNarrow * kNarrow; i += blockDim.x) atomicAdd(out + i, cs[i]);
}

// Window statistics of the narrow window only: for each patch the 7x7 window
// positions around the frame's proposal (the entries of the isf map that
// k_corr_narrow reads), with the same exact integers and the same rounding as
// k_boxstats.  One warp per (frame, patch): lane c reads column c of the 27x27
// region row by row (coalesced) and slides vertically (column sums at the 7 row
// offsets); the 49 windows then sum 21 column sums each.  Frames that fall back
// to the full window get the full map afterwards.
constexpr int kNsPatches = 2;  // patches (warps) per CTA
__global__ void __launch_bounds__(32 * kNsPatches)
    k_boxstats_narrow(const uint16_t* __restrict__ frames, int nf, int H, int W, PatchGrid g,
                      int R, const float* __restrict__ prop, float* __restrict__ isf) {
  constexpr int kRegion = kNarrow + kPatch - 1;  // 27
  __shared__ int cs1[kNsPatches][kNarrow][kRegion];
  __shared__ long long cs2[kNsPatches][kNarrow][kRegion];
  const int np = g.ny * g.nx, f = blockIdx.y, wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.x * kNsPatches + wl;
  if (p >= np || f >= nf) return;
  int cy, cx;
  narrow_center(prop, f, R, cy, cx);
  const int wy0 = cy - kNarrow / 2, wx0 = cx - kNarrow / 2;
  const int ty = g.y0 + (p / g.nx) * kPatch, tx = g.x0 + (p % g.nx) * kPatch;
  if (lane < kRegion) {
    const uint16_t* col = frames + (size_t)f * H * W + (size_t)(ty + wy0) * W + tx + wx0 + lane;
    int v[kRegion];
#pragma unroll
    for (int r = 0; r < kRegion; ++r) v[r] = __ldg(col + (size_t)r * W);
    int s1 = 0;
    long long s2 = 0;
#pragma unroll
    for (int r = 0; r < kPatch; ++r) {
      s1 += v[r];
      s2 += (long long)v[r] * v[r];
    }
#pragma unroll
    for (int j = 0; j < kNarrow; ++j) {
      cs1[wl][j][lane] = s1;
      cs2[wl][j][lane] = s2;
      if (j + 1 < kNarrow) {
        const int a = v[j + kPatch], b = v[j];
        s1 += a - b;
        s2 += (long long)a * a - (long long)b * b;
      }
    }
  }
  __syncwarp();
  int oy, ox, sh, sw;
  stats_map_dims(g, R, &oy, &ox, &sh, &sw);
  float* out = isf + (size_t)f * sh * sw + (size_t)(ty + wy0 - oy) * sw + (tx + wx0 - ox);
  for (int i = lane; i < kNarrow * kNarrow; i += 32) {
    const int dy = i / kNarrow, dx = i - dy * kNarrow;
    long long s1 = 0, s2 = 0;
#pragma unroll
    for (int c = 0; c < kPatch; ++c) {
      s1 += cs1[wl][dy][dx + c];
      s2 += cs2[wl][dy][dx + c];
    }
    const long long sf = (long long)kPatchArea * s2 - s1 * s1;
    out[(size_t)dy * sw + dx] = sf > 0 ? rsqrtf((float)sf) : 0.f;
  }
}

cudaError_t launch_stats_narrow(const uint16_t* frames, int nf, int H, int W, PatchGrid g, int R,
                                const float* prop, float* isf, cudaStream_t st) {
  if (nf <= 0) return cudaSuccess;
  const int np = g.ny * g.nx;
  k_boxstats_narrow<<<dim3((np + kNsPatches - 1) / kNsPatches, nf), 32 * kNsPatches, 0, st>>>(
      frames, nf, H, W, g, R, prop, isf);
  return cudaGetLastError();
}

// Peak of the narrow window.  Falls back to the full window (frame appended to
// the device-side list) when d* lies on the 7x7 border or C(d*) < threshold.
// surface (optional): the 7x7 values at their places in the full (2R+1)^2 grid;
// prop_px (optional): the proposal in px.
__global__ void k_peak_narrow(const unsigned long long* __restrict__ csum, int R, int np,
                              const float* __restrict__ prop, float thresh,
                              float* __restrict__ shifts, float* __restrict__ info,
                              int* __restrict__ list, int* __restrict__ list_n,
                              double* __restrict__ surface, float* __restrict__ prop_px) {
  const int f = blockIdx.x, lane = threadIdx.x, nw = kNarrow * kNarrow;
  const long long* C = reinterpret_cast<const long long*>(csum) + (size_t)f * nw;
  int cy, cx;
  narrow_center(prop, f, R, cy, cx);
  Cand b, s2;
  float s[2];
  peak_of(C, kNarrow, kNarrow, cy - kNarrow / 2, cx - kNarrow / 2, np, lane, b, s2, s);
  if (surface) {
    const int w = 2 * R + 1;
    for (int i = lane; i < nw; i += 32) {
      const int y = cy - kNarrow / 2 + i / kNarrow + R, x = cx - kNarrow / 2 + i % kNarrow + R;
      surface[(size_t)f * w * w + (size_t)y * w + x] = (double)C[i] / kFix / np;
    }
  }
  if (lane != 0) return;
  if (prop_px) {
    prop_px[2 * f] = prop[2 * f] * kShiftScale;
    prop_px[2 * f + 1] = prop[2 * f + 1] * kShiftScale;
  }
  const int iy = b.idx / kNarrow, ix = b.idx % kNarrow;
  const float cpk = (float)((double)b.v / kFix / np);
  const bool edge = iy == 0 || ix == 0 || iy == kNarrow - 1 || ix == kNarrow - 1;
  if (edge || cpk < thresh) {
    list[atomicAdd(list_n, 1)] = f;
    return;
  }
  if (shifts) {
    shifts[2 * f] = s[0];
    shifts[2 * f + 1] = s[1];
  }
  if (info) {
    info[4 * f + 0] = (float)(iy + cy - kNarrow / 2);
    info[4 * f + 1] = (float)(ix + cx - kNarrow / 2);
    info[4 * f + 2] = cpk;
    info[4 * f + 3] = s2.idx >= 0 ? (float)((double)s2.v / kFix / np) : 0.f;
  }
}

cudaError_t launch_corr_narrow(const uint16_t* frames, int nf, int H, int W, PatchGrid g, int R,
                               const TemplateDev& td, const float* isf, const float* prop,
                               unsigned long long* csum, cudaStream_t st) {
  if (nf <= 0) return cudaSuccess;
  const size_t smem = sizeof(float) * (kNarrow + kPatch - 1) * kNarrowStride;
  static unsigned char attr[kMaxDevices] = {};
  cudaError_t e = once_per_device(attr, [smem](int) {
    return cudaFuncSetAttribute(k_corr_narrow, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  });
  if (e != cudaSuccess) return e;
  const int groups = g.ny * ((g.nx + kNarrowGroup - 1) / kNarrowGroup);
  k_corr_narrow<<<dim3(nf, groups), kNarrowGroup * 8, smem, st>>>(frames, H, W, g, R, td.tc, td.tn2,
                                                                   isf, prop, csum);
  return cudaGetLastError();
}

__global__ void k_count_add(const int* __restrict__ n, long long* __restrict__ total) {
  *total += *n;
}

cudaError_t launch_count_add(const int* n, long long* total, cudaStream_t st) {
  k_count_add<<<1, 1, 0, st>>>(n, total);
  return cudaGetLastError();
}

cudaError_t launch_peak_narrow(const unsigned long long* csum, int nf, int R, int np,
                               const float* prop, float thresh, float* shifts, float* info,
                               int* list, int* list_n, double* surface, float* prop_px,
                               cudaStream_t st) {
  if (nf <= 0) return cudaSuccess;
  k_peak_narrow<<<nf, 32, 0, st>>>(csum, R, np, prop, thresh, shifts, info, list, list_n, surface,
                                   prop_px);
  return cudaGetLastError();
}

}  // namespace vimg
