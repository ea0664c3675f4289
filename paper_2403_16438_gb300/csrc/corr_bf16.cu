// BF16 tensor-core (tcgen05) correlation numerators of Sec. II, FP32 accumulate.
//
// num_p(d) = sum_k Tc_p[k] F[k + d] = sum_k Tc_p[k] Fc[k + d] + B_p(d), where
//   Fc = F - round(T)                  (per pixel; small magnitude, exact in FP32)
//   B_p(d) = sum_k Tc_p[k] round(T)[k + d]   (frame independent, set per template)
// Only Fc and Tc go through BF16; B_p is exact up to FP32 rounding.
//
// Implicit GEMM per patch p and group of 16 frames (one tcgen05.mma per step):
//   D[(f, jy)][jx] += sum_{c} A[(f, jy)][(rho, c)] * Bt[(rho, c)][jx]
//   A[(f, jy)][(rho, c)] = Fc_f[y_p - R + 8 b_y + jy + rho][x_p - R - o_p + 16 b_x + c]
//   Bt[(rho, c)][jx]     = Tc_p[rho][c - jx - o_p]        (Toeplitz along x)
// so D = num_p(dy = 8 b_y + jy - R, dx = 16 b_x + jx - R).  M = 128 rows =
// 16 frames x 8 displacement rows: the displacement row comes for free from the
// 16-byte row stride of the canonical (no swizzle, K-major) core matrices, so the
// frames need no im2col; they arrive by TMA straight from the Fc images (one 3-D
// box of 8 columns x 60 rows x 16 frames per column block).  Bt is precomputed
// per patch (o_p = 8-alignment offset of the patch's window).  5 x 3 blocks of
// (8 dy x 16 dx) cover the 33 x 33 window; K = 21 rows x 48 columns.
//
// N = 32: the template is split into a BF16 high part and a BF16 remainder (16 dx
// columns each), so it enters with ~16 significant bits; only Fc is rounded.
//
// Each CTA (one per SM, persistent) walks (frame group, patch) work units.  One
// thread waits for the unit's TMA loads, issues its 945 MMAs and commits them to
// an mbarrier; as soon as they complete the next unit's loads are issued, so the
// epilogue (hi + lo + background term -> per-patch numerators in global memory)
// overlaps them.  k_zncc_reduce then forms C(d) = sum_p ZNCC_p(d) per frame in
// patch order (deterministic) as 2^-40 fixed point.  Every wait is bounded: on
// timeout the CTA records an error and stops issuing work.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>

#include "vimg_internal.h"

namespace vimg {

namespace {

constexpr int kFr = 16;           // frames per group (M = 128 = 16 x 8)
constexpr int kRowsA = 60;        // staged rows: 5 dy blocks x 8 + 20
constexpr int kColBlk = 10;       // staged column blocks of 8 (80 columns)
constexpr int kDyBlk = 5, kDxBlk = 3, kKq = 3;  // K chunks of 16 columns per template row
constexpr int kJx = 16;                       // displacement columns per block
constexpr int kN = 2 * kJx;                   // N = [template hi part | lo part]
constexpr uint32_t kAColBytes = kFr * kRowsA * 16;               // 15,360 B per column block
constexpr uint32_t kABytes = kColBlk * kAColBytes;              // 153,600 B
constexpr uint32_t kBtBytesPerRow = 6 * 4 * 128;                // 6 K-blocks x 4 N-blocks
constexpr uint32_t kBtBytes = kPatch * kBtBytesPerRow;          // 64,512 B per patch
constexpr int kThreads = 128;
constexpr int kTmemCols = 512;
constexpr long long kSpin = 1LL << 22;  // bounded waits (seconds at most)

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | ((uint64_t)1 << 46);
}

constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  for (long long s = 0; s < kSpin && !done; ++s)
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(su32(bar)), "r"(parity));
  return done != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(kThreads, 1)
    k_corr_bf16(const __grid_constant__ CUtensorMap tmap, int nf, int R, PatchGrid g,
                const __nv_bfloat16* __restrict__ bt, const float* __restrict__ bgc,
                float* __restrict__ num, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                 // [10 col blocks][16 frames][60 rows][16 B]
  unsigned char* sB = smem + kABytes;       // [21][6 K blocks][4 N blocks][8][8] bf16
  __shared__ __align__(8) uint64_t bar_load, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int np = g.ny * g.nx, w = 2 * R + 1, nw = w * w;
  const int n_groups = (nf + kFr - 1) / kFr;
  const int n_work = n_groups * np;  // (frame group, patch) pairs, patch fastest

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar_load)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar_mma)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  uint32_t ph_load = 0, ph_mma = 0;
  const int f_loc = (warp * 32 + lane) >> 3, jy = lane & 7;

  // loads of one (frame group, patch) work unit: 10 TMA boxes of Fc + the patch's Bt
  auto issue_loads = [&](int wk) {
    const int grp = wk / np, p = wk - grp * np;
    const int ty = g.y0 + (p / g.nx) * kPatch, tx = g.x0 + (p % g.nx) * kPatch;
    const int xa = (tx - R) & ~7;  // 16-byte aligned start column
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(&bar_load)),
                 "r"(kABytes + kBtBytes));
    for (int cb = 0; cb < kColBlk; ++cb)
      asm volatile(
          "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
              su32(sA + cb * kAColBytes)),
          "l"(&tmap), "r"(xa + 8 * cb), "r"(ty - R), "r"(grp * kFr), "r"(su32(&bar_load))
          : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(sB)),
        "l"(bt + (size_t)p * (kBtBytes / 2)), "r"(kBtBytes), "r"(su32(&bar_load))
        : "memory");
  };

  if (tid == 0 && (int)blockIdx.x < n_work) issue_loads(blockIdx.x);
  for (int wk = blockIdx.x; wk < n_work; wk += gridDim.x) {
    const int grp = wk / np, p = wk - grp * np;
    // 1. operands of this unit have landed -> MMAs: 5 x 3 blocks x 21 rows x 3 chunks
    if (tid == 0) {
      if (!mbar_wait(&bar_load, ph_load)) {
        atomicExch(err, 1);
        abort_flag = 1;
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = su32(sA), b0 = su32(sB);
        for (int by = 0; by < kDyBlk; ++by)
          for (int bx = 0; bx < kDxBlk; ++bx) {
            const uint32_t d = tmem + (uint32_t)((by * kDxBlk + bx) * kN);
            for (int rho = 0; rho < kPatch; ++rho)
              for (int q = 0; q < kKq; ++q) {
                const uint32_t aaddr = a0 + (uint32_t)(2 * bx + 2 * q) * kAColBytes +
                                       (uint32_t)(8 * by + rho) * 16;
                const uint64_t ad = desc(aaddr, kAColBytes, kRowsA * 16);
                const uint64_t bd = desc(b0 + (uint32_t)(rho * 6 + 2 * q) * 512, 512, 128);
                const uint32_t acc = (rho | q) ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred pa;\nsetp.ne.b32 pa, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n}\n" ::"r"(d),
                    "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
              }
          }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            su32(&bar_mma)));
      }
    }
    ph_load ^= 1;
    if (!mbar_wait(&bar_mma, ph_mma)) {
      atomicExch(err, 1);
      abort_flag = 1;
    }
    ph_mma ^= 1;
    __syncthreads();
    if (abort_flag) break;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // 2. the shared operands are free: start the next unit's loads now
    if (tid == 0 && wk + (int)gridDim.x < n_work) issue_loads(wk + gridDim.x);
    // 3. epilogue (overlaps those loads): numerator = hi + lo parts + background term
    {
      const int f = grp * kFr + f_loc;
      float* out = num + ((size_t)min(f, nf - 1) * np + p) * nw;
      const float* bg = bgc + (size_t)p * nw;
      for (int by = 0; by < kDyBlk; ++by) {
        const int dyi = 8 * by + jy;
        for (int bx = 0; bx < kDxBlk; ++bx) {
          float hv[16], lv[16];
          tmem_ld16(tmem + lane_base + (by * kDxBlk + bx) * kN, hv);
          tmem_ld16(tmem + lane_base + (by * kDxBlk + bx) * kN + kJx, lv);
          if (f < nf && dyi < w) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int dxi = 16 * bx + j;
              if (dxi < w) out[dyi * w + dxi] = hv[j] + lv[j] + __ldg(bg + dyi * w + dxi);
            }
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
  }
  // drain: a load issued for a unit this CTA will not run is impossible (it only
  // issues the next unit it owns), so nothing is in flight here.
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// ZNCC of every (frame, displacement) summed over the patches in patch order:
//   C(d) = sum_p num_p(d) * 21 / |Tc_p| * isf(window_p(d)),  stored in 2^-40 fixed point.
__global__ void k_zncc_reduce(const float* __restrict__ num, int nf, int R, PatchGrid g,
                              const float* __restrict__ tn2, const float* __restrict__ isf,
                              int sh, int sw, unsigned long long* __restrict__ csum) {
  const int f = blockIdx.y, w = 2 * R + 1, nw = w * w, np = g.ny * g.nx;
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= nw) return;
  const int dy = d / w, dx = d - dy * w;
  const float* nf_ = num + (size_t)f * np * nw + d;
  const float* is = isf + (size_t)f * sh * sw + (size_t)dy * sw + dx;
  float acc = 0.f;
  for (int p = 0; p < np; ++p) {
    const int py = p / g.nx, px = p - py * g.nx;
    const float t2 = __ldg(tn2 + p);
    const float ps = t2 > 0.f ? (float)kPatch * rsqrtf(t2) : 0.f;
    acc = fmaf(__ldg(nf_ + (size_t)p * nw) * ps, __ldg(is + (size_t)py * kPatch * sw + px * kPatch), acc);
  }
  csum[(size_t)f * nw + d] = (unsigned long long)__float2ll_rn(acc * (float)kFix);
}

// ---- per-template constants -----------------------------------------------------
// Bt_p: [rho][K block 0..5][N block 0..3][n%8][c%8] bf16, n = part * 16 + jx:
// part 0 = bf16(Tc_p[rho][c - jx - o_p]), part 1 = bf16 of the remainder, so the
// two parts carry the template to ~16 significant bits.
__global__ void k_bt_prep(const float* __restrict__ tc, PatchGrid g, int R,
                          __nv_bfloat16* __restrict__ bt) {
  const int p = blockIdx.x;
  const int tx = g.x0 + (p % g.nx) * kPatch, o = (tx - R) & 7;
  const float* t = tc + (size_t)p * kPatch * kTplStride;
  __nv_bfloat16* out = bt + (size_t)p * (kBtBytes / 2);
  for (int i = threadIdx.x; i < (int)(kBtBytes / 2); i += blockDim.x) {
    const int rho = i / (kBtBytesPerRow / 2), r = i % (kBtBytesPerRow / 2);
    const int kb = r / 256, nb = (r / 64) & 3, n = nb * 8 + ((r >> 3) & 7), c = kb * 8 + (r & 7);
    const int part = n / kJx, jx = n % kJx, kx = c - jx - o;
    const float v = kx >= 0 && kx < kPatch ? t[rho * kTplStride + kx] : 0.f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    out[i] = part == 0 ? hi : __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

// B_p(d) = sum_k Tc_p[k] * round(T)[window_p(d) + k], FP32 over exact small terms
// (Tc_p in FP32, round(T) - c_p an exact integer).
__global__ void k_bg_corr(const float* __restrict__ tc, const int* __restrict__ coff,
                          const float* __restrict__ tround, int W, PatchGrid g, int R,
                          float* __restrict__ bgc) {
  const int p = blockIdx.x, w = 2 * R + 1;
  const int ty = g.y0 + (p / g.nx) * kPatch, tx = g.x0 + (p % g.nx) * kPatch;
  const float c = (float)coff[p];
  const float* t = tc + (size_t)p * kPatch * kTplStride;
  double tsum = 0.0;  // sum of the FP32 centred values (tiny; restores the offset exactly)
  for (int k = 0; k < kPatchArea; ++k) tsum += t[(k / kPatch) * kTplStride + k % kPatch];
  for (int i = threadIdx.x; i < w * w; i += blockDim.x) {
    const int dy = i / w - R, dx = i % w - R;
    float acc = 0.f;
    for (int ky = 0; ky < kPatch; ++ky)
      for (int kx = 0; kx < kPatch; ++kx)
        acc = fmaf(t[ky * kTplStride + kx],
                   tround[(size_t)(ty + dy + ky) * W + tx + dx + kx] - c, acc);
    bgc[(size_t)p * w * w + i] = acc + (float)(c * tsum);
  }
}

__global__ void k_round_template(const float* __restrict__ T, int n, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = fminf(65535.f, fmaxf(0.f, rintf(T[i])));
}

// Fc = F - round(T) as BF16, rows padded to Wp columns.
__global__ void k_fc(const uint16_t* __restrict__ frames, int nf, int H, int W, int Wp,
                     const float* __restrict__ tround, __nv_bfloat16* __restrict__ fc) {
  const size_t total = (size_t)nf * H * Wp;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % Wp);
    const size_t r = i / Wp;
    const int y = (int)(r % H);
    const size_t f = r / H;
    float v = 0.f;
    if (x < W) v = (float)frames[(f * H + y) * W + x] - tround[(size_t)y * W + x];
    fc[i] = __float2bfloat16_rn(v);
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

}  // namespace

size_t bf16_bt_bytes(PatchGrid g) { return (size_t)g.ny * g.nx * kBtBytes; }
int bf16_row_pitch(int W) { return (W + 7) & ~7; }

cudaError_t bf16_template_prep(const float* T, int H, int W, PatchGrid g, int R,
                               const TemplateDev& td, float* tround, __nv_bfloat16* bt,
                               float* bgc, cudaStream_t st) {
  const int n = H * W;
  k_round_template<<<(n + 255) / 256, 256, 0, st>>>(T, n, tround);
  k_bt_prep<<<g.ny * g.nx, 256, 0, st>>>(td.tc, g, R, bt);
  k_bg_corr<<<g.ny * g.nx, 256, 0, st>>>(td.tc, td.coff, tround, W, g, R, bgc);
  return cudaGetLastError();
}

cudaError_t bf16_make_fc(const uint16_t* frames, int nf, int H, int W, const float* tround,
                         __nv_bfloat16* fc, cudaStream_t st) {
  if (nf <= 0) return cudaSuccess;
  const int Wp = bf16_row_pitch(W);
  const size_t total = (size_t)nf * H * Wp;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 4096);
  k_fc<<<blocks, 256, 0, st>>>(frames, nf, H, W, Wp, tround, fc);
  return cudaGetLastError();
}

// Tensor map over Fc [cap_frames][H][Wp] bf16 with 8 x 60 x 16 boxes.
int bf16_tensor_map(void* map_out, __nv_bfloat16* fc, int cap_frames, int H, int W) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return -1;
  const int Wp = bf16_row_pitch(W);
  cuuint64_t dims[3] = {(cuuint64_t)Wp, (cuuint64_t)H, (cuuint64_t)cap_frames};
  cuuint64_t strides[2] = {(cuuint64_t)Wp * 2, (cuuint64_t)Wp * H * 2};
  cuuint32_t box[3] = {8, kRowsA, kFr};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(static_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, fc,
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -2;
}

size_t bf16_tensor_map_bytes() { return sizeof(CUtensorMap); }

cudaError_t launch_corr_bf16(const void* tmap, int nf, int R, PatchGrid g,
                             const __nv_bfloat16* bt, const float* bgc, const TemplateDev& td,
                             const float* isf, float* num, unsigned long long* csum, int* err,
                             cudaStream_t st) {
  if (nf <= 0) return cudaSuccess;
  static int sms = 0;
  const size_t smem = kABytes + kBtBytes;
  if (!sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_corr_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
      sms = 0;
      return e;
    }
  }
  const int np = g.ny * g.nx, groups = (nf + kFr - 1) / kFr, w = 2 * R + 1;
  const CUtensorMap* map = static_cast<const CUtensorMap*>(tmap);
  k_corr_bf16<<<std::min(groups * np, sms), kThreads, smem, st>>>(*map, nf, R, g, bt, bgc, num,
                                                                  err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int sh = kPatch * (g.ny - 1) + 2 * R + 1, sw = kPatch * (g.nx - 1) + 2 * R + 1;
  k_zncc_reduce<<<dim3((w * w + 127) / 128, nf), 128, 0, st>>>(num, nf, R, g, td.tn2, isf, sh, sw,
                                                              csum);
  return cudaGetLastError();
}

}  // namespace vimg
