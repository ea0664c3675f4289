// Footprint reconstruction of Sec. III-D (Bando et al., BIBM 2023) on the GPU:
// per-segment probability maps p_i -> b_i = p_i > 0.5 -> 8-connected components
// -> shape cleanup (area, eccentricity, concaveness) -> b = OR_i -> components of
// b ("regions") -> NMF P ~ F A (Eq. 3) on each region.
//
// Readings (the paper gives the steps, not the constants): kept blobs have
// area in [20, 1000] px, eccentricity <= 0.95 (pixel-centre covariance) and
// concaveness 1 - area / hull area <= 0.3 (convex hull of the pixel squares);
// the region's blobs (segment order, then smallest pixel) are clustered
// greedily by overlap (a blob joins the first cluster whose first blob it
// overlaps with 2 |a & b| >= |a | b|); N = clusters; F starts as the clusters'
// union indicators, A as the mean of p_i over them (>= 1e-6); 100
// multiplicative updates (A then F, denominators + 1e-9).
//
// Connected components: union-find over all K maps at once, each union linking
// the larger root to the smaller with atomicMin (Playne & Hawick's scheme), so
// that every label is the component's smallest pixel index.  Component ids come
// from a prefix sum over the roots (ascending pixel order), pixel lists from a
// counting sort.  Shape decisions use exact integer sums and FP64 without
// contraction.  The NMF runs one CTA per region with fixed-order reductions.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "vimg_internal.h"

namespace vimg {
namespace {

constexpr float kSegThreshold = 0.5f;
constexpr int kAreaMin = 20, kAreaMax = 1000;
constexpr double kEccMax = 0.95, kConcaveMax = 0.3;
constexpr int kNmfIters = 100;
constexpr float kNmfEps = 1e-9f, kAFloor = 1e-6f;
// Capacity of the NMF kernel (not a rule of the method): a region with more
// pixels or more clusters is not factorised here and is reported through the
// per-region status (vimg_segment_status) instead.
constexpr int kMaxN = 32;          // clusters (neurons) per region
constexpr int kMaxRegion = 16000;  // pixels per region
constexpr int kShapeWarps = 1216;  // warps of the shape kernel (hull scratch each)
constexpr int kHullScratch = 12 * kAreaMax;  // corners (4 n) + chain (<= 8 n)

// ---- union-find connected components over nm maps of HW pixels ------------------
__device__ __forceinline__ int uf_find(const int* L, int x) {
  int r = x;
  while (true) {  // parents strictly decrease: ends at a root
    const int p = L[r];
    if (p == r) return r;
    r = p;
  }
}

__device__ __forceinline__ void uf_unite(int* L, int a, int b) {
  while (true) {  // every retry lowers a root index: ends
    a = uf_find(L, a);
    b = uf_find(L, b);
    if (a == b) return;
    if (a < b) {
      const int old = atomicMin(L + b, a);
      if (old == b) return;
      b = old;
    } else {
      const int old = atomicMin(L + a, b);
      if (old == a) return;
      a = old;
    }
  }
}

// L[m][p] = m HW + p for foreground pixels, -1 for background.  Mask source:
// probability maps (p > threshold) or a byte mask.
__global__ void k_cc_init(const float* __restrict__ prob, const unsigned char* __restrict__ mask,
                          long long total, int* __restrict__ L) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const bool fg = prob ? prob[i] > kSegThreshold : mask[i] != 0;
    L[i] = fg ? (int)i : -1;
  }
}

__global__ void k_cc_merge(int* __restrict__ L, long long total, int H, int W) {
  const long long HW = (long long)H * W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    if (L[i] < 0) continue;
    const int p = (int)(i % HW), y = p / W, x = p - y * W;
    // neighbours already scanned in raster order: W, NW, N, NE
    if (x > 0 && L[i - 1] >= 0) uf_unite(L, (int)i, (int)(i - 1));
    if (y > 0) {
      if (x > 0 && L[i - W - 1] >= 0) uf_unite(L, (int)i, (int)(i - W - 1));
      if (L[i - W] >= 0) uf_unite(L, (int)i, (int)(i - W));
      if (x + 1 < W && L[i - W + 1] >= 0) uf_unite(L, (int)i, (int)(i - W + 1));
    }
  }
}

__global__ void k_cc_flatten(int* __restrict__ L, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    if (L[i] >= 0) L[i] = uf_find(L, (int)i);
}

// ---- exclusive scan of int32 (three phases, 1024 elements per block) -----------
constexpr int kScanBlock = 1024;

__device__ __forceinline__ int block_exclusive_scan(int v, int* tmp, int& total) {
  const int tid = threadIdx.x;
  tmp[tid] = v;
  __syncthreads();
  for (int o = 1; o < blockDim.x; o <<= 1) {
    const int add = tid >= o ? tmp[tid - o] : 0;
    __syncthreads();
    tmp[tid] += add;
    __syncthreads();
  }
  total = tmp[blockDim.x - 1];
  const int r = tmp[tid] - v;
  __syncthreads();
  return r;
}

__global__ void k_scan_blocks(const int* __restrict__ in, long long n, int* __restrict__ out,
                              int* __restrict__ sums) {
  __shared__ int tmp[kScanBlock];
  const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
  const int v = i < n ? in[i] : 0;
  int total;
  const int r = block_exclusive_scan(v, tmp, total);
  if (i < n) out[i] = r;
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Sequential scan of the block sums by one block, in chunks (fixed order).
__global__ void k_scan_sums(int* __restrict__ sums, int nb, int* __restrict__ grand) {
  __shared__ int tmp[kScanBlock];
  int carry = 0;
  for (int base = 0; base < nb; base += kScanBlock) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? sums[i] : 0;
    int total;
    const int r = block_exclusive_scan(v, tmp, total);
    if (i < nb) sums[i] = r + carry;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *grand = carry;
}

__global__ void k_scan_add(int* __restrict__ out, long long n, const int* __restrict__ sums) {
  const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
  if (i < n) out[i] += sums[blockIdx.x];
}

// ---- component bookkeeping -----------------------------------------------------------
__global__ void k_root_flags(const int* __restrict__ L, long long total, int* __restrict__ f) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    f[i] = L[i] == (int)i ? 1 : 0;
}

// Per pixel: its component id (ids[root]); per component: pixel count.
__global__ void k_comp_count(const int* __restrict__ L, const int* __restrict__ ids, long long total,
                             int* __restrict__ cnt) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    if (L[i] >= 0) atomicAdd(cnt + ids[L[i]], 1);
}

__global__ void k_comp_scatter(const int* __restrict__ L, const int* __restrict__ ids, long long total,
                               const int* __restrict__ off, int* __restrict__ cursor,
                               int* __restrict__ list) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    if (L[i] >= 0) {
      const int c = ids[L[i]];
      list[off[c] + atomicAdd(cursor + c, 1)] = (int)i;
    }
}

// Sorts a short int list in place (one warp; odd-even transposition, bounded).
__device__ void warp_sort(int* a, int n) {
  const int lane = threadIdx.x & 31;
  for (int ph = 0; ph < n; ++ph) {
    for (int i = 2 * lane + (ph & 1); i + 1 < n; i += 64) {
      const int x = a[i], y = a[i + 1];
      if (x > y) {
        a[i] = y;
        a[i + 1] = x;
      }
    }
    __syncwarp();
  }
}

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }

// Shape test of every per-segment component (one warp each): candidates by area
// get their pixel list sorted, exact integer moments, the eccentricity and the
// hull area in FP64 without contraction (the oracle's operations), keep[c] = 1/0.
// The hull is Andrew's monotone chain over each row's extreme corners of the
// pixel squares, in the warp's scratch (kHullScratch entries: 4 n corners and a
// chain of at most 2 (4 n) entries).
__global__ void k_blob_shape(int* __restrict__ list, const int* __restrict__ off,
                             const int* __restrict__ cnt, int n_comp, int W, long long HW,
                             long long* __restrict__ scr, int* __restrict__ keep) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_comp; c += warps) {
    const int n = cnt[c];
    if (n < kAreaMin || n > kAreaMax) {
      if (lane == 0) keep[c] = 0;
      continue;
    }
    int* a = list + off[c];
    warp_sort(a, n);
    const int base = (int)((a[0] / HW) * HW);  // the map's offset, same for every pixel
    long long sy = 0, sx = 0, syy = 0, sxx = 0, sxy = 0;
    for (int i = lane; i < n; i += 32) {
      const int p = a[i] - base, y = p / W, x = p - y * W;
      sy += y, sx += x, syy += (long long)y * y, sxx += (long long)x * x, sxy += (long long)x * y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      syy += __shfl_xor_sync(0xffffffffu, syy, o);
      sxx += __shfl_xor_sync(0xffffffffu, sxx, o);
      sxy += __shfl_xor_sync(0xffffffffu, sxy, o);
    }
    if (lane) continue;
    const double dn = (double)n, my = (double)sy / dn, mx = (double)sx / dn;
    const double cyy = dsub((double)syy / dn, dmul(my, my));
    const double cxx = dsub((double)sxx / dn, dmul(mx, mx));
    const double cxy = dsub((double)sxy / dn, dmul(my, mx));
    const double tr = dadd(cyy, cxx), det = dsub(dmul(cyy, cxx), dmul(cxy, cxy));
    const double disc = sqrt(fmax(dsub(dmul(tr, tr) / 4.0, det), 0.0));
    const double l1 = dadd(tr / 2.0, disc), l2 = dsub(tr / 2.0, disc);
    const double ecc = l1 > 0.0 ? sqrt(fmax(0.0, dsub(1.0, fmax(l2, 0.0) / l1))) : 0.0;
    if (ecc > kEccMax) {
      keep[c] = 0;
      continue;
    }
    // corners (x << 32 | y) of each row's extremes: rows come in order, x ascending
    long long* pts = scr + (long long)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kHullScratch;
    long long* hull = pts + 4 * kAreaMax;
    int npt = 0;
    for (int i = 0; i < n;) {
      const int p0 = a[i] - base, y = p0 / W, lo = p0 - y * W;
      int j = i;
      while (j + 1 < n && (a[j + 1] - base) / W == y) ++j;
      const int hi = a[j] - base - y * W + 1;
      pts[npt++] = ((long long)lo << 32) | (unsigned)y;
      pts[npt++] = ((long long)lo << 32) | (unsigned)(y + 1);
      pts[npt++] = ((long long)hi << 32) | (unsigned)y;
      pts[npt++] = ((long long)hi << 32) | (unsigned)(y + 1);
      i = j + 1;
    }
    for (int i = 1; i < npt; ++i) {  // insertion sort by (x, y)
      const long long v = pts[i];
      int j = i - 1;
      while (j >= 0 && pts[j] > v) {
        pts[j + 1] = pts[j];
        --j;
      }
      pts[j + 1] = v;
    }
    int m = 0;
    for (int i = 0; i < npt; ++i)
      if (m == 0 || pts[m - 1] != pts[i]) pts[m++] = pts[i];
    auto X = [](long long v) { return v >> 32; };
    auto Y = [](long long v) { return (long long)(unsigned)(v & 0xffffffffll); };
    auto cross = [&](long long o, long long p, long long q) {
      return (X(p) - X(o)) * (Y(q) - Y(o)) - (Y(p) - Y(o)) * (X(q) - X(o));
    };
    int k = 0;
    for (int i = 0; i < m; ++i) {  // lower chain
      while (k >= 2 && cross(hull[k - 2], hull[k - 1], pts[i]) <= 0) --k;
      hull[k++] = pts[i];
    }
    for (int i = m - 2, t = k + 1; i >= 0; --i) {  // upper chain (ends on the first point)
      while (k >= t && cross(hull[k - 2], hull[k - 1], pts[i]) <= 0) --k;
      hull[k++] = pts[i];
    }
    long long s2 = 0;  // twice the signed area, exact
    for (int i = 0; i + 1 < k; ++i) s2 += X(hull[i]) * Y(hull[i + 1]) - X(hull[i + 1]) * Y(hull[i]);
    const double area = (double)(s2 < 0 ? -s2 : s2) / 2.0;
    keep[c] = dsub(1.0, dn / area) <= kConcaveMax ? 1 : 0;
  }
}

// b(x) = 1 on every kept blob's pixels (one warp per blob).
__global__ void k_or_mask(const int* __restrict__ list, const int* __restrict__ off,
                          const int* __restrict__ cnt, const int* __restrict__ keep, int n_comp,
                          long long HW, unsigned char* __restrict__ b) {
  const int lane = threadIdx.x & 31, warps = (gridDim.x * blockDim.x) >> 5;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_comp; c += warps)
    if (keep[c])
      for (int i = lane; i < cnt[c]; i += 32) b[list[off[c] + i] % HW] = 1;
}

// Region of each kept blob (by its first pixel), and per-region blob counts.
__global__ void k_blob_region(const int* __restrict__ list, const int* __restrict__ off,
                              const int* __restrict__ keep, int n_comp, long long HW,
                              const int* __restrict__ Lb, const int* __restrict__ rid,
                              int* __restrict__ breg, int* __restrict__ rcnt) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_comp; c += gridDim.x * blockDim.x) {
    int r = -1;
    if (keep[c]) {
      r = rid[Lb[list[off[c]] % HW]];
      atomicAdd(rcnt + r, 1);
    }
    breg[c] = r;
  }
}

__global__ void k_blob_scatter(const int* __restrict__ breg, int n_comp, const int* __restrict__ roff,
                               int* __restrict__ cursor, int* __restrict__ rblobs) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_comp; c += gridDim.x * blockDim.x)
    if (breg[c] >= 0) rblobs[roff[breg[c]] + atomicAdd(cursor + breg[c], 1)] = c;
}

// |a & b| of two ascending pixel lists of single maps (global indices; each
// list's map offset is removed once, not per element).
__device__ int inter_count(const int* a, int na, const int* b, int nb, long long HW) {
  const int ba = (int)((a[0] / HW) * HW), bb = (int)((b[0] / HW) * HW);
  int i = 0, j = 0, k = 0;
  while (i < na && j < nb) {
    const int x = a[i] - ba, y = b[j] - bb;
    if (x == y) ++k, ++i, ++j;
    else if (x < y) ++i;
    else ++j;
  }
  return k;
}

// Per region (one warp): sort its blobs and pixels, cluster the blobs greedily
// by overlap (the first blob of a cluster represents it), record N and each
// blob's cluster.  A region beyond the NMF kernel's capacity gets N = 0, every
// blob cluster -1 and status VIMG_REGION_TOO_LARGE (more than kMaxRegion
// pixels) or VIMG_REGION_TOO_MANY (more than kMaxN clusters); else status 0.
__global__ void k_region_cluster(int* __restrict__ rblobs, const int* __restrict__ roff,
                                 const int* __restrict__ rcnt, int* __restrict__ rpix,
                                 const int* __restrict__ poff, const int* __restrict__ pcnt,
                                 int n_reg, const int* __restrict__ list,
                                 const int* __restrict__ off, const int* __restrict__ cnt,
                                 long long HW, int* __restrict__ bclu, int* __restrict__ nreg,
                                 int* __restrict__ status) {
  const int lane = threadIdx.x & 31, warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_reg; r += warps) {
    int* bl = rblobs + roff[r];
    const int nb = rcnt[r];
    if (pcnt[r] > kMaxRegion) {  // beyond capacity: reported, not factorised
      if (lane == 0) nreg[r] = 0, status[r] = VIMG_REGION_TOO_LARGE;
      for (int q = lane; q < nb; q += 32) bclu[bl[q]] = -1;
      continue;
    }
    warp_sort(bl, nb);
    warp_sort(rpix + poff[r], pcnt[r]);
    if (lane) continue;
    int reps[kMaxN];
    int N = 0;
    bool over = false;
    for (int q = 0; q < nb && !over; ++q) {
      const int c = bl[q];
      const int* a = list + off[c];
      int j = 0;
      for (; j < N; ++j) {
        const int rc = reps[j];
        const int in = inter_count(a, cnt[c], list + off[rc], cnt[rc], HW);
        if (2 * in >= cnt[c] + cnt[rc] - in) break;
      }
      if (j == N) {
        if (N == kMaxN) {
          over = true;
          break;
        }
        reps[N++] = c;
      }
      bclu[c] = j;
    }
    if (over)
      for (int q = 0; q < nb; ++q) bclu[bl[q]] = -1;
    nreg[r] = over ? 0 : N;
    status[r] = over ? VIMG_REGION_TOO_MANY : 0;
  }
}

// Position of pixel p in a region's ascending pixel list (present by construction).
__device__ __forceinline__ int row_of(const int* pix, int m, int p) {
  int lo = 0, hi = m - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (pix[mid] < p) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// One CTA per region: gather P [M][K], F0 = cluster-union indicators, A0 = the
// mean of p_i over each union (>= 1e-6), then the multiplicative updates; the
// footprints and activities go to the outputs.
__global__ void __launch_bounds__(256) k_region_nmf(
    const float* __restrict__ prob, int K, long long HW, const int* __restrict__ rpix,
    const int* __restrict__ poff, const int* __restrict__ pcnt, const int* __restrict__ rblobs,
    const int* __restrict__ roff, const int* __restrict__ rcnt, const int* __restrict__ bclu,
    const int* __restrict__ list, const int* __restrict__ off, const int* __restrict__ cnt,
    const int* __restrict__ nreg, const long long* __restrict__ soff, const int* __restrict__ noff,
    float* __restrict__ Pw, float* __restrict__ Fw, float* __restrict__ Aw,
    float* __restrict__ Anw, float* __restrict__ foot, float* __restrict__ act, int max_neurons) {
  const int r = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int M = pcnt[r], N = nreg[r];
  if (N == 0) return;
  const int* pix = rpix + poff[r];
  float* P = Pw + soff[r] * K;   // [M][K]
  float* F = Fw + soff[r] * kMaxN;  // [M][N]
  float* A = Aw + (long long)noff[r] * K;     // [N][K]
  float* An = Anw + (long long)noff[r] * K;   // next A
  __shared__ float G[kMaxN * kMaxN], AA[kMaxN * kMaxN];
  __shared__ int ucnt[kMaxN];
  for (long long i = tid; i < (long long)M * K; i += nt) {
    const int row = (int)(i / K), seg = (int)(i - (long long)row * K);
    P[i] = prob[(long long)seg * HW + pix[row]];
  }
  for (long long i = tid; i < (long long)M * N; i += nt) F[i] = 0.f;
  __syncthreads();
  // cluster unions: every blob marks its cluster's column
  for (int q = 0; q < rcnt[r]; ++q) {
    const int c = rblobs[roff[r] + q], j = bclu[c];
    if (j < 0) continue;
    const int base = (int)((list[off[c]] / HW) * HW);
    for (int i = tid; i < cnt[c]; i += nt) F[(long long)row_of(pix, M, list[off[c] + i] - base) * N + j] = 1.f;
    __syncthreads();
  }
  if (tid < N) {
    int u = 0;
    for (int row = 0; row < M; ++row) u += F[(long long)row * N + tid] > 0.f;
    ucnt[tid] = u;
  }
  __syncthreads();
  for (int i = tid; i < N * K; i += nt) {
    const int j = i / K, seg = i - j * K;
    float s = 0.f;
    for (int row = 0; row < M; ++row)
      if (F[(long long)row * N + j] > 0.f) s += P[(long long)row * K + seg];
    A[i] = fmaxf(s / (float)ucnt[j], kAFloor);
  }
  __syncthreads();
  for (int it = 0; it < kNmfIters; ++it) {
    // G = F'F
    for (int e = tid; e < N * N; e += nt) {
      const int j = e / N, l = e - j * N;
      float s = 0.f;
      for (int row = 0; row < M; ++row) s = fmaf(F[(long long)row * N + j], F[(long long)row * N + l], s);
      G[e] = s;
    }
    __syncthreads();
    // A <- A * (F'P) / (G A + eps), into An, then copied back
    for (int i = tid; i < N * K; i += nt) {
      const int j = i / K, seg = i - j * K;
      float num = 0.f, den = 0.f;
      for (int row = 0; row < M; ++row) num = fmaf(F[(long long)row * N + j], P[(long long)row * K + seg], num);
      for (int l = 0; l < N; ++l) den = fmaf(G[j * N + l], A[l * K + seg], den);
      An[i] = A[i] * num / (den + kNmfEps);
    }
    __syncthreads();
    for (int i = tid; i < N * K; i += nt) A[i] = An[i];
    __syncthreads();
    // AA = A A'
    for (int e = tid; e < N * N; e += nt) {
      const int j = e / N, l = e - j * N;
      float s = 0.f;
      for (int seg = 0; seg < K; ++seg) s = fmaf(A[j * K + seg], A[l * K + seg], s);
      AA[e] = s;
    }
    __syncthreads();
    // F <- F * (P A') / (F AA + eps), row by row
    for (int row = tid; row < M; row += nt) {
      float fr[kMaxN], num[kMaxN];
      for (int j = 0; j < N; ++j) fr[j] = F[(long long)row * N + j], num[j] = 0.f;
      for (int seg = 0; seg < K; ++seg) {
        const float pv = P[(long long)row * K + seg];
        for (int j = 0; j < N; ++j) num[j] = fmaf(pv, A[j * K + seg], num[j]);
      }
      for (int j = 0; j < N; ++j) {
        float den = 0.f;
        for (int l = 0; l < N; ++l) den = fmaf(fr[l], AA[l * N + j], den);
        F[(long long)row * N + j] = fr[j] * num[j] / (den + kNmfEps);
      }
    }
    __syncthreads();
  }
  // outputs: neuron noff[r] + j
  for (int j = 0; j < N; ++j) {
    const int nid = noff[r] + j;
    if (nid >= max_neurons) break;
    if (foot)
      for (int row = tid; row < M; row += nt) foot[(long long)nid * HW + pix[row]] = F[(long long)row * N + j];
    if (act)
      for (int seg = tid; seg < K; seg += nt) act[(long long)nid * K + seg] = A[j * K + seg];
  }
}

// Region index of every pixel of b, -1 elsewhere.
__global__ void k_region_map(const int* __restrict__ Lb, const int* __restrict__ rid, long long HW,
                             int* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = Lb[i] >= 0 ? rid[Lb[i]] : -1;
}

int grid_of(long long n, int t) { return (int)std::max(1LL, std::min((n + t - 1) / t, 65535LL)); }

}  // namespace
}  // namespace vimg

using namespace vimg;

struct vimg_segmenter {
  int H = 0, W = 0, Kmax = 0;
  cudaStream_t st = nullptr;
  std::string err;
  std::vector<void*> allocs;
  int* L = nullptr;      // [Kmax][HW] labels, then scan temporaries
  int* flags = nullptr;  // [Kmax HW]
  int* ids = nullptr;    // [Kmax HW]
  int* sums = nullptr;   // scan block sums
  int* grand = nullptr;  // [1]
  int* list = nullptr;   // [Kmax HW] pixel lists
  long long* scr = nullptr;  // [kShapeWarps][kHullScratch] hull scratch
  unsigned char* b = nullptr;  // [HW]
  int* Lb = nullptr;           // [HW]
  int* rid = nullptr;          // [HW]
  int* rpix = nullptr;         // [HW]
  std::vector<int> status;     // per region of the last vimg_segment call
};

namespace {

int sfail(vimg_segmenter* s, int code, const std::string& m) {
  if (s) s->err = m;
  return code;
}

#define SCK(call, what)                                                                   \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return sfail(s, VIMG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// out = exclusive scan of in (n elements); returns the total (synchronises).
int scan(vimg_segmenter* s, const int* in, long long n, int* out, int* total) {
  const long long nb = (n + kScanBlock - 1) / kScanBlock;
  if (n == 0) {
    *total = 0;
    return VIMG_OK;
  }
  k_scan_blocks<<<(unsigned)nb, kScanBlock, 0, s->st>>>(in, n, out, s->sums);
  k_scan_sums<<<1, kScanBlock, 0, s->st>>>(s->sums, (int)nb, s->grand);
  k_scan_add<<<(unsigned)nb, kScanBlock, 0, s->st>>>(out, n, s->sums);
  SCK(cudaGetLastError(), "scan");
  SCK(cudaMemcpyAsync(total, s->grand, sizeof(int), cudaMemcpyDeviceToHost, s->st), "scan total");
  SCK(cudaStreamSynchronize(s->st), "scan total");
  return VIMG_OK;
}

// Connected components of nm maps (prob > threshold, or a byte mask): labels in L.
int label(vimg_segmenter* s, const float* prob, const unsigned char* mask, long long total, int* L) {
  const int g = grid_of(total, 256);
  k_cc_init<<<g, 256, 0, s->st>>>(prob, mask, total, L);
  k_cc_merge<<<g, 256, 0, s->st>>>(L, total, s->H, s->W);
  k_cc_flatten<<<g, 256, 0, s->st>>>(L, total);
  SCK(cudaGetLastError(), "labelling");
  return VIMG_OK;
}

template <class T>
T* dev_alloc(vimg_segmenter* s, std::vector<void*>& own, size_t n, cudaError_t& e) {
  T* p = nullptr;
  if (e == cudaSuccess) e = cudaMalloc((void**)&p, sizeof(T) * std::max<size_t>(n, 1));
  if (e == cudaSuccess) own.push_back(p);
  (void)s;
  return p;
}

}  // namespace

extern "C" vimg_segmenter* vimg_segmenter_create(int H, int W, int max_segments, void* stream) {
  if (H < 1 || W < 1 || (long long)H * W > (1 << 24) || max_segments < 1 ||
      (long long)max_segments * H * W >= (1LL << 31) / 8)
    return nullptr;
  vimg_segmenter* s = new vimg_segmenter();
  s->H = H, s->W = W, s->Kmax = max_segments;
  s->st = static_cast<cudaStream_t>(stream);
  const size_t HW = (size_t)H * W, tot = HW * max_segments;
  cudaError_t e = cudaSuccess;
  s->L = dev_alloc<int>(s, s->allocs, tot, e);
  s->flags = dev_alloc<int>(s, s->allocs, tot, e);
  s->ids = dev_alloc<int>(s, s->allocs, tot, e);
  s->sums = dev_alloc<int>(s, s->allocs, tot / kScanBlock + 2, e);
  s->grand = dev_alloc<int>(s, s->allocs, 1, e);
  s->list = dev_alloc<int>(s, s->allocs, tot, e);
  s->scr = dev_alloc<long long>(s, s->allocs, (size_t)kShapeWarps * kHullScratch, e);
  s->b = dev_alloc<unsigned char>(s, s->allocs, HW, e);
  s->Lb = dev_alloc<int>(s, s->allocs, HW, e);
  s->rid = dev_alloc<int>(s, s->allocs, HW, e);
  s->rpix = dev_alloc<int>(s, s->allocs, HW, e);
  if (e != cudaSuccess) {
    for (void* q : s->allocs) cudaFree(q);
    delete s;
    return nullptr;
  }
  return s;
}

extern "C" void vimg_segmenter_destroy(vimg_segmenter* s) {
  if (!s) return;
  for (void* q : s->allocs) cudaFree(q);
  delete s;
}

extern "C" const char* vimg_segmenter_last_error(const vimg_segmenter* s) {
  return s ? s->err.c_str() : "";
}

extern "C" int vimg_segment_status(const vimg_segmenter* s, int* status, int n) {
  if (!s || n < 0 || (n > 0 && !status)) return VIMG_ERR_ARG;
  const int m = (int)s->status.size();
  for (int i = 0; i < n && i < m; ++i) status[i] = s->status[i];
  return m;
}

extern "C" int vimg_segment(vimg_segmenter* s, const float* d_prob, int K, float* d_footprints,
                            float* d_activity, int max_neurons, int* d_region_map, int* n_regions) {
  if (!s) return VIMG_ERR_ARG;
  if (K < 1 || K > s->Kmax || !d_prob || max_neurons < 0)
    return sfail(s, VIMG_ERR_ARG, "vimg_segment: bad arguments");
  const long long HW = (long long)s->H * s->W, total = HW * K;
  s->status.clear();
  // 1. per-segment components, ids by ascending pixel index, pixel lists
  int rc = label(s, d_prob, nullptr, total, s->L);
  if (rc) return rc;
  k_root_flags<<<grid_of(total, 256), 256, 0, s->st>>>(s->L, total, s->flags);
  int n_comp = 0;
  if ((rc = scan(s, s->flags, total, s->ids, &n_comp))) return rc;
  std::vector<void*> tmp;
  auto cleanup = [&]() {
    for (void* q : tmp) cudaFree(q);
  };
  cudaError_t e = cudaSuccess;
  int* cnt = dev_alloc<int>(s, tmp, n_comp, e);
  int* off = dev_alloc<int>(s, tmp, n_comp, e);
  int* cursor = dev_alloc<int>(s, tmp, n_comp, e);
  int* keep = dev_alloc<int>(s, tmp, n_comp, e);
  int* breg = dev_alloc<int>(s, tmp, n_comp, e);
  int* bclu = dev_alloc<int>(s, tmp, n_comp, e);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int) * std::max(n_comp, 1), s->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, sizeof(int) * std::max(n_comp, 1), s->st);
  if (e != cudaSuccess) {
    cleanup();
    return sfail(s, VIMG_ERR_CUDA, std::string("vimg_segment: ") + cudaGetErrorString(e));
  }
  int fg = 0;
  k_comp_count<<<grid_of(total, 256), 256, 0, s->st>>>(s->L, s->ids, total, cnt);
  if ((rc = scan(s, cnt, n_comp, off, &fg))) return cleanup(), rc;
  k_comp_scatter<<<grid_of(total, 256), 256, 0, s->st>>>(s->L, s->ids, total, off, cursor, s->list);
  // 2. shape cleanup, OR mask, regions
  k_blob_shape<<<std::min(grid_of((long long)n_comp * 32, 256), kShapeWarps / 8), 256, 0, s->st>>>(
      s->list, off, cnt, n_comp, s->W, HW, s->scr, keep);
  SCK(cudaMemsetAsync(s->b, 0, HW, s->st), "mask reset");
  k_or_mask<<<grid_of((long long)n_comp * 32, 256), 256, 0, s->st>>>(s->list, off, cnt, keep,
                                                                     n_comp, HW, s->b);
  if ((rc = label(s, nullptr, s->b, HW, s->Lb))) return cleanup(), rc;
  k_root_flags<<<grid_of(HW, 256), 256, 0, s->st>>>(s->Lb, HW, s->flags);
  int n_reg = 0;
  if ((rc = scan(s, s->flags, HW, s->rid, &n_reg))) return cleanup(), rc;
  if (n_regions) *n_regions = n_reg;
  if (d_region_map) k_region_map<<<grid_of(HW, 256), 256, 0, s->st>>>(s->Lb, s->rid, HW, d_region_map);
  int* pcnt = dev_alloc<int>(s, tmp, n_reg, e);
  int* poff = dev_alloc<int>(s, tmp, n_reg, e);
  int* rcnt = dev_alloc<int>(s, tmp, n_reg, e);
  int* roff = dev_alloc<int>(s, tmp, n_reg, e);
  int* rcur = dev_alloc<int>(s, tmp, n_reg, e);
  int* nreg = dev_alloc<int>(s, tmp, n_reg, e);
  int* rstat = dev_alloc<int>(s, tmp, n_reg, e);
  int* rblobs = dev_alloc<int>(s, tmp, n_comp, e);
  for (int* z : {pcnt, rcnt, rcur})
    if (e == cudaSuccess) e = cudaMemsetAsync(z, 0, sizeof(int) * std::max(n_reg, 1), s->st);
  if (e != cudaSuccess) {
    cleanup();
    return sfail(s, VIMG_ERR_CUDA, std::string("vimg_segment: ") + cudaGetErrorString(e));
  }
  s->status.assign(n_reg, 0);
  if (n_reg == 0) {
    e = cudaStreamSynchronize(s->st);
    cleanup();
    return e == cudaSuccess ? 0 : sfail(s, VIMG_ERR_CUDA, cudaGetErrorString(e));
  }
  int npix = 0, nb = 0;
  k_comp_count<<<grid_of(HW, 256), 256, 0, s->st>>>(s->Lb, s->rid, HW, pcnt);
  if ((rc = scan(s, pcnt, n_reg, poff, &npix))) return cleanup(), rc;
  SCK(cudaMemsetAsync(rcur, 0, sizeof(int) * n_reg, s->st), "cursor reset");
  k_comp_scatter<<<grid_of(HW, 256), 256, 0, s->st>>>(s->Lb, s->rid, HW, poff, rcur, s->rpix);
  k_blob_region<<<grid_of(n_comp, 256), 256, 0, s->st>>>(s->list, off, keep, n_comp, HW, s->Lb,
                                                         s->rid, breg, rcnt);
  if ((rc = scan(s, rcnt, n_reg, roff, &nb))) return cleanup(), rc;
  SCK(cudaMemsetAsync(rcur, 0, sizeof(int) * n_reg, s->st), "cursor reset");
  k_blob_scatter<<<grid_of(n_comp, 256), 256, 0, s->st>>>(breg, n_comp, roff, rcur, rblobs);
  // 3. clustering: N per region
  k_region_cluster<<<grid_of((long long)n_reg * 32, 256), 256, 0, s->st>>>(
      rblobs, roff, rcnt, s->rpix, poff, pcnt, n_reg, s->list, off, cnt, HW, bclu, nreg, rstat);
  SCK(cudaGetLastError(), "clustering");
  std::vector<int> hN(n_reg), hM(n_reg);
  SCK(cudaMemcpyAsync(hN.data(), nreg, sizeof(int) * n_reg, cudaMemcpyDeviceToHost, s->st), "N");
  SCK(cudaMemcpyAsync(hM.data(), pcnt, sizeof(int) * n_reg, cudaMemcpyDeviceToHost, s->st), "M");
  SCK(cudaMemcpyAsync(s->status.data(), rstat, sizeof(int) * n_reg, cudaMemcpyDeviceToHost, s->st),
      "status");
  SCK(cudaStreamSynchronize(s->st), "N");
  std::vector<long long> hso(n_reg);
  std::vector<int> hno(n_reg);
  long long so = 0;
  int neurons = 0;
  for (int r = 0; r < n_reg; ++r) {
    hso[r] = so, hno[r] = neurons;
    so += hM[r];
    neurons += hN[r];
  }
  long long* soff = dev_alloc<long long>(s, tmp, n_reg, e);
  int* noff = dev_alloc<int>(s, tmp, n_reg, e);
  float* Pw = dev_alloc<float>(s, tmp, (size_t)so * K, e);
  float* Fw = dev_alloc<float>(s, tmp, (size_t)so * kMaxN, e);
  float* Aw = dev_alloc<float>(s, tmp, (size_t)std::max(neurons, 1) * K, e);
  float* Anw = dev_alloc<float>(s, tmp, (size_t)std::max(neurons, 1) * K, e);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(soff, hso.data(), sizeof(long long) * n_reg, cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(noff, hno.data(), sizeof(int) * n_reg, cudaMemcpyHostToDevice, s->st);
  const int n_out = std::min(neurons, max_neurons);
  if (e == cudaSuccess && d_footprints && n_out > 0)
    e = cudaMemsetAsync(d_footprints, 0, sizeof(float) * (size_t)n_out * HW, s->st);
  if (e != cudaSuccess) {
    cleanup();
    return sfail(s, VIMG_ERR_CUDA, std::string("vimg_segment: ") + cudaGetErrorString(e));
  }
  // 4. NMF per region
  k_region_nmf<<<n_reg, 256, 0, s->st>>>(d_prob, K, HW, s->rpix, poff, pcnt, rblobs, roff, rcnt,
                                         bclu, s->list, off, cnt, nreg, soff, noff, Pw, Fw, Aw, Anw,
                                         d_footprints, d_activity, max_neurons);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  cleanup();
  if (e != cudaSuccess) return sfail(s, VIMG_ERR_CUDA, std::string("vimg_segment: ") + cudaGetErrorString(e));
  (void)fg, (void)npix, (void)nb;
  return neurons;
}
