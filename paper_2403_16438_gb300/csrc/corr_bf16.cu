// BF16 tensor-core (tcgen05) correlation numerators of Sec. II, FP32 accumulate.
//
// num_p(d) = sum_k Tc_p[k] F[k + d] = sum_k Tc_p[k] Fc[k + d] + B_p(d), where
//   Fc = F - round(T)                  (per pixel; small magnitude)
//   B_p(d) = sum_k Tc_p[k] round(T)[k + d]   (frame independent, set per template)
// Only Fc and Tc go through BF16; B_p is exact up to FP32 rounding.
//
// Implicit GEMM per patch p and group of up to 128 frames (N = frames):
//   D[(xl, i)][f] += sum_{k} A[(xl, i)][k] * B[k][f]
//   B[k][f] = Fc_f[y_p - R + y][x_p - R - o_p + 16 b + k]       (frame row y, column k)
//   A[(xl, i)][k] = Tc_p[y - 8a - i][k - o_p - xl]              (Toeplitz in x and y)
// so D = num_p(dy = 8a + i - R, dx = 16b + xl - R): an M = 128 block of 8 dy x 16 dx
// displacements; a = 0..4 and b = 0..2 cover the 33 x 33 window; the K loop runs
// over the 53 frame rows y of the patch's search region and 3 chunks of 16
// columns.  A depends on (a, y) only through y - 8a and not on b at all, so one
// compact store per patch serves every MMA: S[xl][c][q][j] = Tc[27 - q][8c + j -
// o_p - xl] with template rows reversed (q = 27 - r, zero rows above and
// below), so that the 8 rows of a core matrix -- 8 consecutive dy -- are 8
// consecutive 16-byte rows of S starting at q0 = 27 - (y - 8a).
// The frames arrive by TMA from Fc images laid out [row][8-column block][frame]
// [8], so each frame row of the region is one box of 6 column blocks x 128 frames.
//
// One tcgen05.mma of M = 128, K = 16 occupies the tensor pipe for N / 2 cycles
// (64 at N = 128), so one warp must issue an MMA in less than that: the issue
// loop is kept to straight-line, warp-uniform code, and commits are grouped.
// The kernel runs N = 128 so that four accumulators fit in TMEM (512 columns):
// dy block a of pass P (P counts passes over all units) uses slot (a + P) mod 4.  Only 4 dy blocks are ever live at once
// (block 0 ends at row 27, block 4 starts at row 32), and the rotation gives
// every other hand-off between passes many rows of slack.
//
// Warp roles (one persistent CTA per SM, 320 threads):
//   warp 8  producer: per work unit the patch's A store (bulk copy, double
//           buffered across units), then 3 passes x 53 frame rows of B through
//           an 8-row ring whose rows land and are released in groups of 4;
//   warp 9  MMA issuer (the whole warp in step, one elected lane issuing): per
//           row, 3 MMAs for each dy block the row feeds; one commit per 4 rows
//           frees a ring group, one per finished dy block hands its accumulator
//           to the epilogue;
//   warps 0-7 epilogue: TMEM -> registers (warp w: lanes 32 (w mod 4) .. + 31,
//           columns 64 (w / 4) .. + 63), + B_p(d), stores of the per-patch
//           numerators, then release of the accumulator slot.
// k_zncc_reduce then forms C(d) = sum_p ZNCC_p(d) per frame in patch order
// (deterministic) as 2^-40 fixed point.  Every wait is bounded: on timeout the
// CTA records an error, stops issuing work, waits (bounded) for its own copies
// and MMAs, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>

#include "tc_ptx.h"
#include "vimg_internal.h"

namespace vimg {

namespace {
using namespace tc;

constexpr int kNF = 128;           // frames per group (N of a full group)
constexpr int kRows = 53;          // frame rows of a search region (21 + 2 R, R = 16)
constexpr int kDyBlk = 5;          // dy blocks of 8
constexpr int kSlots = 4;          // TMEM accumulators of kNF columns
constexpr int kPasses = 3;         // dx blocks of 16
constexpr int kKq = 3;             // K chunks of 16 columns per row
constexpr int kCb = 6;             // 8-column blocks per pass window (48 columns)
constexpr int kQ = 35;             // reversed template rows incl. zero padding
constexpr int kXl = 16;            // dx per block
constexpr uint32_t kASlice = kQ * 16;                  // 560 B: one (xl, c) column strip
constexpr uint32_t kAXl = kCb * kASlice;               // 3,360 B per xl
constexpr uint32_t kABytes = kXl * kAXl;               // 53,760 B per patch
constexpr uint32_t kBStage = kCb * kNF * 16;           // 12,288 B per frame row
constexpr int kStages = 8;                             // ring of frame rows
constexpr int kGroupRows = 4;                          // rows landing on one barrier, released by one commit
constexpr size_t kSmem = 2 * (size_t)kABytes + (size_t)kStages * kBStage;  // 205,824 B
constexpr int kEpiWarps = 8;
constexpr int kThreads = (kEpiWarps + 2) * 32;         // 320
constexpr int kTmemCols = 512;
constexpr int kWin = 33;
constexpr int kNWin = kWin * kWin;

// Position of displacement (dyi, dxi) (0..32 each) in the numerator buffer:
// blocks (a, b) in order b-major, within a block the accumulator row order
// m = 8 xl + i, with only the valid rows of the edge blocks (a = 4: dyi = 32;
// b = 2: dxi = 32) kept, so a warp's stores are contiguous.
__host__ __device__ __forceinline__ int dperm(int dyi, int dxi) {
  const int a = dyi >> 3, i = dyi & 7, b = dxi >> 4, xl = dxi & 15;
  const int base = b * 528;
  if (b < 2) return base + (a < 4 ? a * 128 + xl * 8 + i : 512 + xl);
  return base + (a < 4 ? a * 8 + i : 32);
}

// The three K chunks of one dy block and frame row, kind::f16 with BF16
// operands and the FP32 accumulator in TMEM at d: D (+)= sum_q A_q * B_q
// (accumulate_first = 0: the first product overwrites D, the others add).
// Called by a whole converged warp; one elected lane issues all three.
__device__ __forceinline__ void mma_bf16_x3(uint32_t d, uint64_t a0, uint64_t b0, uint32_t idesc,
                                            uint32_t accumulate_first) {
  static_assert(kKq == 3, "three K chunks of 16 columns per frame row");
  constexpr uint64_t kDa = 2 * kASlice >> 4, kDb = 2 * kNF * 16 >> 4;  // per K chunk, 16-B units
  asm volatile(
      "{\n.reg .pred pe, pa, pt;\nelect.sync _|pe, 0xffffffff;\n"
      "setp.ne.b32 pa, %7, 0;\nsetp.eq.b32 pt, %7, %7;\n"
      "@pe tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %4, %8, pa;\n"
      "@pe tcgen05.mma.cta_group::1.kind::f16 [%0], %2, %5, %8, pt;\n"
      "@pe tcgen05.mma.cta_group::1.kind::f16 [%0], %3, %6, %8, pt;\n}\n" ::"r"(d),
      "l"(a0), "l"(a0 + kDa), "l"(a0 + 2 * kDa), "l"(b0), "l"(b0 + kDb), "l"(b0 + 2 * kDb),
      "r"(accumulate_first), "r"(idesc));
}

// Last frame row of dy block a (rows beyond 52 only feed displacements past 32).
__host__ __device__ __forceinline__ int last_row(int a) { return min(8 * a + 27, kRows - 1); }

// The row segments the issue loop walks: rows [y0, y1) feed exactly dy blocks
// a0..a1.  Checked at compile time against the rule they encode (row y feeds
// block a iff 8a <= y <= last_row(a)), so that every row of a pass is issued
// once with its full block set.
struct RowSegment {
  int y0, y1, a0, a1;
};
constexpr RowSegment kRowSegments[] = {{0, 8, 0, 0},   {8, 16, 0, 1},  {16, 24, 0, 2},
                                       {24, 28, 0, 3}, {28, 32, 1, 3}, {32, 36, 1, 4},
                                       {36, 44, 2, 4}, {44, 52, 3, 4}, {52, 53, 4, 4}};
constexpr bool row_segments_match() {
  int y = 0;
  for (const RowSegment& g : kRowSegments) {
    if (g.y0 != y || g.y1 <= g.y0) return false;
    for (; y < g.y1; ++y)
      for (int a = 0; a < kDyBlk; ++a) {
        const bool fed = 8 * a <= y && y <= (8 * a + 27 < kRows - 1 ? 8 * a + 27 : kRows - 1);
        if (fed != (g.a0 <= a && a <= g.a1)) return false;
      }
  }
  return y == kRows;
}
static_assert(row_segments_match(), "row segments and dy-block sets of the issue loop");

// State of the MMA-issuing warp carried from row to row.
struct IssueState {
  uint32_t it;    // frame rows consumed (position in the ring)
  uint32_t used;  // bit s: accumulator slot s has been used before
  uint32_t par;   // bit s: parity of slot s's next release by the epilogue
};

struct IssueCtx {
  uint64_t* full;
  uint64_t* grp_empty;
  uint64_t* acc_full;
  uint64_t* acc_free;
  uint32_t tmem, idesc;
  uint64_t b_desc0;
};

// MMAs of frame rows [y0, y1) of one pass, rows that feed exactly the dy blocks
// A0..A1: with the block set fixed at compile time each row's MMAs are
// straight-line code.  Per block and row, three K chunks of 16 columns; the
// block's first row overwrites its accumulator slot (after the epilogue has
// released it) and its last row commits it to the epilogue.  False when a wait
// gave up.
template <int A0, int A1>
__device__ __forceinline__ bool issue_rows(int y0, int y1, uint32_t pass, uint64_t& ad_row,
                                           IssueState& st, const IssueCtx& c) {
  static_assert(kRows == 53 && kDyBlk == 5, "row segments assume a 53-row region, 5 dy blocks");
  for (int y = y0; y < y1; ++y, ++st.it, --ad_row) {
    const uint32_t s = st.it % kStages;
    if (s % kGroupRows == 0) {  // the first row of a ring group: all its rows have landed
      if (!mbar_wait_warp(&c.full[s / kGroupRows], (st.it / kStages) & 1)) return false;
      asm volatile("tcgen05.fence::after_thread_sync;");
    }
    const uint64_t bd0 = c.b_desc0 + (uint64_t)(s * (kBStage >> 4));
#pragma unroll
    for (int a = A0; a <= A1; ++a) {
      const uint32_t slot = (a + pass) & (kSlots - 1);
      const uint32_t d = c.tmem + slot * kNF;
      const uint64_t ad0 = ad_row + (uint64_t)(8 * a);
      if (y == 8 * a) {
        const uint32_t bit = 1u << slot;
        if (st.used & bit) {
          if (!mbar_wait_warp(&c.acc_free[slot], (st.par >> slot) & 1)) return false;
          st.par ^= bit;
          asm volatile("tcgen05.fence::after_thread_sync;");
        }
        st.used |= bit;
        mma_bf16_x3(d, ad0, bd0, c.idesc, 0u);
      } else {
        mma_bf16_x3(d, ad0, bd0, c.idesc, 1u);
      }
      if (y == last_row(a)) mma_commit_elect(&c.acc_full[slot]);
    }
    if (s % kGroupRows == kGroupRows - 1) mma_commit_elect(&c.grp_empty[s / kGroupRows]);
  }
  return true;
}

__global__ void __launch_bounds__(kThreads, 1)
    k_corr_bf16(const __grid_constant__ CUtensorMap tmap, int nf, PatchGrid g,
                const __nv_bfloat16* __restrict__ astore, const float* __restrict__ bgc,
                float* __restrict__ num, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                     // [2][kABytes]
  unsigned char* sB = smem + 2 * kABytes;       // [kStages][kBStage]
  // full[q]: the kGroupRows frame rows of ring group q have landed (one wait per group);
  // grp_empty[q]: the MMAs reading them have completed
  __shared__ __align__(8) uint64_t full[kStages / kGroupRows], grp_empty[kStages / kGroupRows];
  __shared__ __align__(8) uint64_t a_full[2], a_empty[2];
  __shared__ __align__(8) uint64_t acc_full[kSlots], acc_free[kSlots], mma_done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int np = g.ny * g.nx;
  const int n_groups = (nf + kNF - 1) / kNF;
  const int n_work = n_groups * np;  // (frame group, patch) units, patch fastest

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int q = 0; q < kStages / kGroupRows; ++q) {
      mbar_init(&full[q], kGroupRows);
      mbar_init(&grp_empty[q], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&a_full[i], 1);
      mbar_init(&a_empty[i], 1);
    }
    for (int a = 0; a < kSlots; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_free[a], kEpiWarps);
    }
    mbar_init(&mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_flag = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  if (warp == kEpiWarps) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int it = 0, u = 0, na = 0;  // B rows, units, A copies issued
      for (int wk = blockIdx.x; wk < n_work && !abort_flag; wk += gridDim.x, ++u) {
        const int grp = wk / np, p = wk - grp * np;
        const int ty = g.y0 + (p / g.nx) * kPatch, tx = g.x0 + (p % g.nx) * kPatch;
        const int cb0 = (tx - kMaxR) >> 3;  // tx - R >= 0 on the patch grid
        const int buf = u & 1;
        if (u >= 2 && !mbar_wait(&a_empty[buf], ((u >> 1) - 1) & 1)) {
          atomicExch(err, 1);
          abort_flag = 1;
          break;
        }
        mbar_expect_tx(&a_full[buf], kABytes);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                su32(sA + buf * kABytes)),
            "l"(astore + (size_t)p * (kABytes / 2)), "r"(kABytes), "r"(su32(&a_full[buf]))
            : "memory");
        ++na;
        for (int b = 0; b < kPasses && !abort_flag; ++b)
          for (int y = 0; y < kRows; ++y, ++it) {
            const int s = it % kStages, cyc = it / kStages;
            // the first row of a ring group waits until the MMAs of its previous
            // use have completed
            if (cyc > 0 && s % kGroupRows == 0 &&
                !mbar_wait(&grp_empty[s / kGroupRows], (cyc - 1) & 1)) {
              atomicExch(err, 1);
              abort_flag = 1;
              break;
            }
            uint64_t* fb = &full[s / kGroupRows];
            mbar_expect_tx(fb, kBStage);  // one of the group's kGroupRows arrivals
            asm volatile(
                "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(
                    su32(sB + s * kBStage)),
                "l"(&tmap), "r"(0), "r"(grp * (kNF / 16)), "r"(cb0 + 2 * b), "r"(ty - kMaxR + y),
                "r"(su32(fb))
                : "memory");
          }
      }
      // a last, partial ring group completes with plain arrivals in place of its
      // missing rows
      if (it % kGroupRows)
        for (int r = it % kGroupRows; r < kGroupRows; ++r) mbar_arrive(&full[(it % kStages) / kGroupRows]);
      // wait (bounded) for the copies this thread issued: the last use of every group
      const int n_grp = (it + kGroupRows - 1) / kGroupRows, ring = kStages / kGroupRows;
      for (int q = 0; q < ring && q < n_grp; ++q) mbar_wait(&full[q], ((n_grp - 1 - q) / ring) & 1);
      for (int i = 0; i < 2 && i < na; ++i) mbar_wait(&a_full[i], ((na - 1 - i) >> 1) & 1);
    }
  } else if (warp == kEpiWarps + 1) {
    // ---------------- MMA issuer ----------------
    // The whole warp runs the loop in step and one elected lane issues each MMA
    // and commit, so the descriptor arithmetic stays warp-uniform.  At N = 128
    // an MMA occupies the tensor pipe for about 64 cycles, and a single warp's
    // dependent integer work easily costs more, so the bookkeeping is kept
    // small: slot state in bit masks (no local arrays), the abort flag read once
    // per work unit, one wait per ring group, descriptors advanced by constants,
    // and the dy blocks of each row segment fixed at compile time.
    {
      uint32_t u = 0;
      IssueState st{0, 0, 0};
      bool issued = false, fail = false;
      for (int wk = blockIdx.x; wk < n_work; wk += gridDim.x, ++u) {
        if (__shfl_sync(0xffffffffu, abort_flag, 0)) break;
        const int grp = wk / np;
        const int rem = nf - grp * kNF;
        const int n_cols = rem >= kNF ? kNF : ((rem + 15) & ~15);
        const uint32_t idesc = idesc_for(n_cols);
        const uint32_t buf = u & 1;
        if (!mbar_wait_warp(&a_full[buf], (u >> 1) & 1)) {
          fail = true;
          break;
        }
        // Descriptors change only in their start-address field (bits 0-13, in
        // 16-byte units): build the constant parts once, add offsets per MMA.
        const uint64_t a_desc0 = desc(su32(sA + buf * kABytes), kASlice, kAXl);
        const uint64_t b_desc0 = desc(su32(sB), kNF * 16, 128);
        const IssueCtx c{full, grp_empty, acc_full, acc_free, tmem, idesc, b_desc0};
        for (int b = 0; b < kPasses && !fail; ++b) {
          issued = true;
          // A rows start at q0 = 27 - (y - 8 a): one 16-byte row less per frame row
          uint64_t ad_row = a_desc0 + 27;
          const uint32_t pass = u * kPasses + b;
          // row segments with a fixed set of dy blocks (a with 8a <= y <= last_row(a))
          // (kRowSegments, spelled out so that each segment's block set is a
          // template argument)
#define VIMG_SEG(i)                                                                      \
  issue_rows<kRowSegments[i].a0, kRowSegments[i].a1>(kRowSegments[i].y0, kRowSegments[i].y1, \
                                                     pass, ad_row, st, c)
          fail = !(VIMG_SEG(0) && VIMG_SEG(1) && VIMG_SEG(2) && VIMG_SEG(3) && VIMG_SEG(4) &&
                   VIMG_SEG(5) && VIMG_SEG(6) && VIMG_SEG(7) && VIMG_SEG(8));
#undef VIMG_SEG
          static_assert(sizeof(kRowSegments) / sizeof(kRowSegments[0]) == 9, "nine segments");
        }
        if (fail) break;
        mma_commit_elect(&a_empty[buf]);
      }
      if (fail && lane == 0) {
        atomicExch(err, 1);
        abort_flag = 1;
      }
      // every MMA issued by this warp has completed before the CTA frees TMEM
      if (issued) {
        mma_commit_elect(&mma_done);
        mbar_wait_warp(&mma_done, 0);
      }
    }
  } else {
    // ------ epilogue (warp w: TMEM lanes 32 (w mod 4) .. + 31, columns 64 (w / 4) .. + 63) ------
    const int quad = warp & 3, half = warp >> 2;
    const int m = quad * 32 + lane, xl = m >> 3, i = m & 7;
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    int u = 0;
    uint32_t epar = 0;  // bit s: parity of the next completion of slot s
    for (int wk = blockIdx.x; wk < n_work; wk += gridDim.x, ++u) {
      const int grp = wk / np, p = wk - grp * np;
      const int nvalid = min(kNF, nf - grp * kNF);
      const int c_lo = half * (kNF / 2), c_hi = min(nvalid, c_lo + kNF / 2);
      const float* bg = bgc + (size_t)p * kNWin;
      bool stop = false;
      for (int b = 0; b < kPasses && !stop; ++b) {
        const int pass = u * kPasses + b;
        const int dxi = 16 * b + xl;
        for (int a = 0; a < kDyBlk; ++a) {
          const int slot = (a + pass) & (kSlots - 1);
          const uint32_t k = (epar >> slot) & 1;
          epar ^= 1u << slot;
          const int dyi = 8 * a + i;
          const bool valid = dyi < kWin && dxi < kWin;
          const float bgv = valid ? __ldg(bg + dyi * kWin + dxi) : 0.f;
          const int dp = valid ? dperm(dyi, dxi) : 0;
          if (!mbar_wait(&acc_full[slot], k)) {
            atomicExch(err, 1);
            abort_flag = 1;
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          float* out = num + ((size_t)(grp * kNF) * np + p) * kNWin + dp;
          for (int c0 = c_lo; c0 < c_hi; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + lane_base + (uint32_t)(slot * kNF + c0), v);
            if (valid) {
#pragma unroll
              for (int j = 0; j < 16; ++j)
                if (c0 + j < c_hi) out[(size_t)(c0 + j) * np * kNWin] = v[j] + bgv;
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;");
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_free[slot]);
        }
      }
      if (stop || abort_flag) break;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// Displacement (dyi, dxi) stored at position t of a numerator row (inverse of dperm).
__device__ __forceinline__ void dperm_inv(int t, int& dyi, int& dxi) {
  const int b = t / 528, r = t - 528 * b;
  if (b < 2) {
    if (r < 512) {
      const int a = r >> 7, mm = r & 127;
      dyi = 8 * a + (mm & 7);
      dxi = 16 * b + (mm >> 3);
    } else {
      dyi = 32;
      dxi = 16 * b + (r - 512);
    }
  } else if (r < 32) {
    dyi = r;
    dxi = 32;
  } else {
    dyi = 32;
    dxi = 32;
  }
}

// ZNCC of every (frame, displacement) summed over the patches in patch order:
//   C(d) = sum_p num_p(d) * 21 / |Tc_p| * isf(window_p(d)),  stored in 2^-40 fixed point.
// Thread = storage position t of two consecutive frames (contiguous numerator
// reads; the patch scale is computed once for both and twice the loads are in
// flight); each frame's sum runs in patch order.
__global__ void k_zncc_reduce(const float* __restrict__ num, int nf, PatchGrid g,
                              const float* __restrict__ tn2, const float* __restrict__ isf,
                              int sh, int sw, unsigned long long* __restrict__ csum) {
  const int f0 = 2 * blockIdx.y, np = g.ny * g.nx;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kNWin || f0 >= nf) return;
  const bool two = f0 + 1 < nf;
  const int f1 = two ? f0 + 1 : f0;  // a missing second frame repeats the first (not stored)
  int dy, dx;
  dperm_inv(t, dy, dx);
  const float* n0 = num + (size_t)f0 * np * kNWin + t;
  const float* n1 = num + (size_t)f1 * np * kNWin + t;
  const float* i0 = isf + (size_t)f0 * sh * sw + (size_t)dy * sw + dx;
  const float* i1 = isf + (size_t)f1 * sh * sw + (size_t)dy * sw + dx;
  float acc0 = 0.f, acc1 = 0.f;
  int p = 0;
  for (int py = 0; py < g.ny; ++py) {
    const size_t ro = (size_t)py * kPatch * sw;
#pragma unroll 4
    for (int px = 0; px < g.nx; ++px, ++p) {
      const float t2 = __ldg(tn2 + p);
      const float ps = t2 > 0.f ? (float)kPatch * rsqrtf(t2) : 0.f;
      const size_t no = (size_t)p * kNWin, io = ro + px * kPatch;
      acc0 = fmaf(__ldg(n0 + no) * ps, __ldg(i0 + io), acc0);
      acc1 = fmaf(__ldg(n1 + no) * ps, __ldg(i1 + io), acc1);
    }
  }
  const size_t o = (size_t)dy * kWin + dx;
  csum[(size_t)f0 * kNWin + o] = (unsigned long long)__float2ll_rn(acc0 * (float)kFix);
  if (two) csum[(size_t)f1 * kNWin + o] = (unsigned long long)__float2ll_rn(acc1 * (float)kFix);
}

// ---- per-template constants -----------------------------------------------------
// A store of patch p: [xl][c][q][j] bf16 = Tc_p[27 - q][8 c + j - o_p - xl] (0 outside).
__global__ void k_a_prep(const float* __restrict__ tc, PatchGrid g,
                         __nv_bfloat16* __restrict__ as) {
  const int p = blockIdx.x;
  const int tx = g.x0 + (p % g.nx) * kPatch, o = (tx - kMaxR) & 7;
  const float* t = tc + (size_t)p * kPatch * kTplStride;
  __nv_bfloat16* out = as + (size_t)p * (kABytes / 2);
  for (int e = threadIdx.x; e < (int)(kABytes / 2); e += blockDim.x) {
    const int j = e & 7, q = (e >> 3) % kQ, c = (e / (8 * kQ)) % kCb, x = e / (8 * kQ * kCb);
    const int r = 27 - q, s = 8 * c + j - o - x;
    const float v = (r >= 0 && r < kPatch && s >= 0 && s < kPatch) ? t[r * kTplStride + s] : 0.f;
    out[e] = __float2bfloat16_rn(v);
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

// Fc = F - round(T) as BF16 in the layout [row][8-column block][frame][8] with
// fcap frame slots (columns past W are zero).  A warp takes one frame row, two
// column blocks and 16 frames (lane = block * 16 + frame): each frame's two blocks
// are one 32-byte read, and each block's 16 frames one 256-byte write.
__global__ void k_fc(const uint16_t* __restrict__ frames, int nf, int H, int W, int ncb, int fcap,
                     const float* __restrict__ tround, __nv_bfloat16* __restrict__ fc) {
  const int lane = threadIdx.x & 31, cbl = lane >> 4, fl = lane & 15;
  const int ncb2 = (ncb + 1) / 2, nf16 = (nf + 15) / 16;
  const long long items = (long long)H * ncb2 * nf16;
  const long long wstride = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long it = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < items;
       it += wstride) {
    const int f16 = (int)(it % nf16);
    const long long r = it / nf16;
    const int cb2 = (int)(r % ncb2), y = (int)(r / ncb2);
    const int f = f16 * 16 + fl, cb = 2 * cb2 + cbl;
    if (f >= nf || cb >= ncb) continue;
    const uint16_t* src = frames + ((size_t)f * H + y) * W + 8 * cb;
    const float* tr = tround + (size_t)y * W + 8 * cb;
    uint16_t px[8];
    if (8 * cb + 8 <= W && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
      const uint4 q = __ldg(reinterpret_cast<const uint4*>(src));
      px[0] = q.x & 0xFFFF, px[1] = q.x >> 16, px[2] = q.y & 0xFFFF, px[3] = q.y >> 16;
      px[4] = q.z & 0xFFFF, px[5] = q.z >> 16, px[6] = q.w & 0xFFFF, px[7] = q.w >> 16;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) px[j] = 8 * cb + j < W ? __ldg(src + j) : 0;
    }
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      v[j] = __float2bfloat16_rn(8 * cb + j < W ? (float)px[j] - __ldg(tr + j) : 0.f);
    *reinterpret_cast<uint4*>(fc + (((size_t)y * ncb + cb) * fcap + f) * 8) =
        *reinterpret_cast<const uint4*>(v);
  }
}

int fc_slots(int cap_frames) { return (cap_frames + 15) & ~15; }

}  // namespace

size_t bf16_astore_bytes(PatchGrid g) { return (size_t)g.ny * g.nx * kABytes; }
int bf16_row_pitch(int W) { return (W + 7) & ~7; }
size_t bf16_fc_elems(int cap_frames, int H, int W) {
  return (size_t)fc_slots(cap_frames) * H * bf16_row_pitch(W);
}

cudaError_t bf16_template_prep(const float* T, int H, int W, PatchGrid g, int R,
                               const TemplateDev& td, float* tround, __nv_bfloat16* as,
                               float* bgc, cudaStream_t st) {
  const int n = H * W;
  k_round_template<<<(n + 255) / 256, 256, 0, st>>>(T, n, tround);
  k_a_prep<<<g.ny * g.nx, 256, 0, st>>>(td.tc, g, as);
  k_bg_corr<<<g.ny * g.nx, 256, 0, st>>>(td.tc, td.coff, tround, W, g, R, bgc);
  return cudaGetLastError();
}

cudaError_t bf16_make_fc(const uint16_t* frames, int nf, int cap_frames, int H, int W,
                         const float* tround, __nv_bfloat16* fc, cudaStream_t st) {
  if (nf <= 0) return cudaSuccess;
  const int ncb = bf16_row_pitch(W) / 8;
  const size_t warps = (size_t)H * ((ncb + 1) / 2) * ((nf + 15) / 16);
  const int blocks = (int)std::min<size_t>((warps + 7) / 8, 8192);
  k_fc<<<blocks, 256, 0, st>>>(frames, nf, H, W, ncb, fc_slots(cap_frames), tround, fc);
  return cudaGetLastError();
}

// Tensor map over Fc [H][ncb][fcap][8] bf16 as 4-D {128 = 16 frames x 8, fcap/16, ncb, H}
// with boxes {128, 8, 6, 1}: one frame row, 6 column blocks, 128 frames.
int bf16_tensor_map(void* map_out, __nv_bfloat16* fc, int cap_frames, int H, int W) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return -1;
  const int ncb = bf16_row_pitch(W) / 8, fcap = fc_slots(cap_frames);
  cuuint64_t dims[4] = {128, (cuuint64_t)fcap / 16, (cuuint64_t)ncb, (cuuint64_t)H};
  cuuint64_t strides[3] = {256, (cuuint64_t)fcap * 16, (cuuint64_t)ncb * fcap * 16};
  cuuint32_t box[4] = {128, kNF / 16, kCb, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(static_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, fc,
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -2;
}

size_t bf16_tensor_map_bytes() { return sizeof(CUtensorMap); }

size_t bf16_num_floats(int cap_frames, PatchGrid g) {
  return (size_t)cap_frames * g.ny * g.nx * kNWin;
}

cudaError_t launch_corr_bf16(const void* tmap, int nf, int R, PatchGrid g,
                             const __nv_bfloat16* as, const float* bgc, const TemplateDev& td,
                             const float* isf, float* num, unsigned long long* csum, int* err,
                             cudaStream_t st) {
  if (nf <= 0) return cudaSuccess;
  if (R != kMaxR) return cudaErrorInvalidValue;
  static unsigned char attr[kMaxDevices] = {};
  cudaError_t ea = once_per_device(attr, [](int) {
    return cudaFuncSetAttribute(k_corr_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kSmem);
  });
  if (ea != cudaSuccess) return ea;
  const int sms = sm_count();
  if (sms <= 0) return cudaErrorInvalidDevice;
  const int np = g.ny * g.nx, groups = (nf + kNF - 1) / kNF;
  const CUtensorMap* map = static_cast<const CUtensorMap*>(tmap);
  k_corr_bf16<<<std::min(groups * np, sms), kThreads, kSmem, st>>>(*map, nf, g, as, bgc, num, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int sh = kPatch * (g.ny - 1) + 2 * R + 1, sw = kPatch * (g.nx - 1) + 2 * R + 1;
  k_zncc_reduce<<<dim3((kNWin + 127) / 128, (nf + 1) / 2), 128, 0, st>>>(num, nf, g, td.tn2,
                                                                         isf, sh, sw, csum);
  return cudaGetLastError();
}

}  // namespace vimg
