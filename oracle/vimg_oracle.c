/*
 * vimg_oracle.c -- plain FP64 CPU oracle for the frame-stream hot path of
 * Bando et al., "Real-time Neuron Segmentation for Voltage Imaging" (BIBM 2023).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * Everything here is the plain definition, by direct sums, in double
 * precision, in the order the paper states it:
 *   - motion correction by zero-mean normalized cross-correlation (ZNCC) of
 *     21x21 patches tiled over the image, one rigid motion vector per frame
 *     (Sec. II);
 *   - time segments of L = 50 frames (Sec. III-B);
 *   - spatial summary S_i = temporal mean of the corrected video (Eq. 1);
 *   - temporal summary T_i = max - median of the Gaussian-smoothed video,
 *     sigma = 3 px (Eq. 2);
 *   - voltage traces: the mean pixel intensity within each neuron ROI for each
 *     frame of the motion-corrected video (Sec. II, third pipeline stage).
 * Where the paper is silent (patch-grid placement, aggregation rule, tie
 * break, subpixel refinement, resampling, high-pass filter, Gaussian
 * truncation and border, median of an even count) the readings are stated at
 * each function.  Parallelism (OpenMP over patches / rows) never changes the
 * arithmetic of any single value.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_FLAG_OUT_HIGHPASS 4 /* corrected output holds the high-passed video */

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Patch grid (Sec. II: 21x21 patches tiled to cover the image).
 * Reading: non-overlapping P x P patches placed inside the region where every
 * window shifted by up to +-R stays in bounds, centred in that region:
 *   n_y = floor((H - 2R) / P),  y0 = R + floor(((H - 2R) - n_y P) / 2),
 * and the same along x.  out = {n_y, n_x, y0, x0}.  Returns 0, or -1 when no
 * patch fits. */
int orc_patch_grid(int H, int W, int R, int P, int* out) {
  if (H <= 0 || W <= 0 || R < 0 || P <= 0) return -1;
  int ny = (H - 2 * R) / P, nx = (W - 2 * R) / P;
  if (H - 2 * R < P || W - 2 * R < P || ny <= 0 || nx <= 0) return -1;
  out[0] = ny;
  out[1] = nx;
  out[2] = R + ((H - 2 * R) - ny * P) / 2;
  out[3] = R + ((W - 2 * R) - nx * P) / 2;
  return 0;
}

/* ZNCC (Sec. II) of the template patch whose top-left corner is (ty, tx) with
 * the frame window displaced by d = (dy, dx): the textbook definition
 *   sum (T - mean T)(F - mean F) / sqrt( sum (T - mean T)^2 * sum (F - mean F)^2 ).
 * Reading: the template patch is fixed and the frame window moves; raw pixel
 * values; 0 when either centred norm is 0. */
double orc_zncc(const uint16_t* F, int H, int W, const double* T, int ty, int tx, int P, int dy,
                int dx) {
  (void)H;
  double n = (double)P * P, mt = 0.0, mf = 0.0;
  for (int ky = 0; ky < P; ++ky)
    for (int kx = 0; kx < P; ++kx) {
      mt += T[(size_t)(ty + ky) * W + (tx + kx)];
      mf += F[(size_t)(ty + ky + dy) * W + (tx + kx + dx)];
    }
  mt /= n;
  mf /= n;
  double num = 0.0, st = 0.0, sf = 0.0;
  for (int ky = 0; ky < P; ++ky)
    for (int kx = 0; kx < P; ++kx) {
      double a = T[(size_t)(ty + ky) * W + (tx + kx)] - mt;
      double b = (double)F[(size_t)(ty + ky + dy) * W + (tx + kx + dx)] - mf;
      num += a * b;
      st += a * a;
      sf += b * b;
    }
  if (st == 0.0 || sf == 0.0) return 0.0;
  return num / sqrt(st * sf);
}

/* Correlation surface of one frame over the window dy in [dy0, dy0+wy),
 * dx in [dx0, dx0+wx) (all inside [-R, R]).
 * Aggregation (Sec. II: patch values are "aggregated" to pick the motion
 * vector; the rule is not given).  Reading: C(d) = arithmetic mean over all
 * patches of ZNCC_p(d).  C is [wy][wx]; Z (optional) is [n_patches][wy][wx].
 * Returns 0 or -1. */
int orc_surface(const uint16_t* F, int H, int W, const double* T, int R, int P, int dy0, int dx0,
                int wy, int wx, double* C, double* Z) {
  int g[4];
  if (orc_patch_grid(H, W, R, P, g)) return -1;
  if (dy0 < -R || dx0 < -R || dy0 + wy - 1 > R || dx0 + wx - 1 > R || wy <= 0 || wx <= 0)
    return -1;
  int np = g[0] * g[1], nw = wy * wx;
  double* z = Z ? Z : (double*)malloc(sizeof(double) * (size_t)np * nw);
  if (!z) return -1;
#pragma omp parallel for schedule(dynamic)
  for (int p = 0; p < np; ++p) {
    int ty = g[2] + (p / g[1]) * P, tx = g[3] + (p % g[1]) * P;
    for (int iy = 0; iy < wy; ++iy)
      for (int ix = 0; ix < wx; ++ix)
        z[(size_t)p * nw + iy * wx + ix] = orc_zncc(F, H, W, T, ty, tx, P, dy0 + iy, dx0 + ix);
  }
  for (int i = 0; i < nw; ++i) {
    double s = 0.0;
    for (int p = 0; p < np; ++p) s += z[(size_t)p * nw + i];
    C[i] = s / np;
  }
  if (!Z) free(z);
  return 0;
}

/* Integer peak and subpixel refinement of a surface C[wy][wx] whose (0,0)
 * entry is displacement (dy0, dx0).
 * Integer peak: d* = argmax C.  Reading for exact ties: smallest dy^2+dx^2,
 * then smallest dy, then smallest dx.
 * Subpixel (not in the paper; reading): per axis a 3-point parabola through
 * c-, c0, c+ at d*-e, d*, d*+e:  delta = (c- - c+) / (2 (c- - 2 c0 + c+)),
 * set to 0 when the curvature term is >= 0 or a neighbour lies outside the
 * window, then clamped to [-0.5, 0.5].
 * out_s = {dy* + delta_y, dx* + delta_x}; out_d = {dy*, dx*};
 * out_info = {C(d*), second-largest C value, flags}; flags bit 0/1 = d* on the
 * window border in y/x.  */
void orc_peak(const double* C, int dy0, int dx0, int wy, int wx, double* out_s, int* out_d,
              double* out_info) {
  int by = 0, bx = 0;
  double best = C[0];
  for (int iy = 0; iy < wy; ++iy)
    for (int ix = 0; ix < wx; ++ix) {
      double c = C[iy * wx + ix];
      int dy = dy0 + iy, dx = dx0 + ix, cy = dy0 + by, cx = dx0 + bx;
      int better = 0;
      if (c > best) better = 1;
      else if (c == best) {
        long r = (long)dy * dy + (long)dx * dx, rb = (long)cy * cy + (long)cx * cx;
        if (r < rb || (r == rb && (dy < cy || (dy == cy && dx < cx)))) better = 1;
      }
      if (better) {
        best = c;
        by = iy;
        bx = ix;
      }
    }
  double second = -INFINITY;
  for (int i = 0; i < wy * wx; ++i)
    if (i != by * wx + bx && C[i] > second) second = C[i];
  int flags = 0;
  double dlt[2] = {0.0, 0.0};
  for (int ax = 0; ax < 2; ++ax) {
    int i = ax == 0 ? by : bx, n = ax == 0 ? wy : wx;
    if (i == 0 || i == n - 1) {
      flags |= 1 << ax;
      continue;
    }
    double cm = ax == 0 ? C[(by - 1) * wx + bx] : C[by * wx + bx - 1];
    double cp = ax == 0 ? C[(by + 1) * wx + bx] : C[by * wx + bx + 1];
    double c0 = C[by * wx + bx];
    double den = cm - 2.0 * c0 + cp;
    if (den >= 0.0) continue;
    double d = (cm - cp) / (2.0 * den);
    if (d > 0.5) d = 0.5;
    if (d < -0.5) d = -0.5;
    dlt[ax] = d;
  }
  out_d[0] = dy0 + by;
  out_d[1] = dx0 + bx;
  out_s[0] = out_d[0] + dlt[0];
  out_s[1] = out_d[1] + dlt[1];
  out_info[0] = best;
  out_info[1] = second;
  out_info[2] = flags;
}

/* Resampling of the shifted frame (implied by Sec. II: the corrected video
 * shows stationary neurons; the method is not given).  Reading: bilinear,
 *   V(y, x) = F(y + s_y, x + s_x),
 * each coordinate clamped to [0, H-1] x [0, W-1] (replicated border). */
void orc_resample(const uint16_t* F, int H, int W, double sy, double sx, double* V) {
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      double ty = y + sy, tx = x + sx;
      if (ty < 0.0) ty = 0.0;
      if (ty > H - 1) ty = H - 1;
      if (tx < 0.0) tx = 0.0;
      if (tx > W - 1) tx = W - 1;
      int y0 = (int)floor(ty), x0 = (int)floor(tx);
      int y1 = y0 + 1 < H ? y0 + 1 : H - 1, x1 = x0 + 1 < W ? x0 + 1 : W - 1;
      double wy = ty - y0, wx = tx - x0;
      double a = F[(size_t)y0 * W + x0], b = F[(size_t)y0 * W + x1];
      double c = F[(size_t)y1 * W + x0], d = F[(size_t)y1 * W + x1];
      V[(size_t)y * W + x] = (1.0 - wy) * ((1.0 - wx) * a + wx * b) + wy * ((1.0 - wx) * c + wx * d);
    }
}

/* Mirror index for the Gaussian border ("d c b a | a b c d"): -1 -> 0, -2 -> 1,
 * n -> n-1, n+1 -> n-2.  Valid while the radius is below n. */
static int mirror(int i, int n) {
  if (i < 0) return -i - 1;
  if (i >= n) return 2 * n - i - 1;
  return i;
}

/* Gaussian spatial pre-smoothing of Eq. 2 (sigma = 3 px in the paper).
 * Reading: radius ceil(4 sigma), weights exp(-k^2 / (2 sigma^2)) normalised to
 * sum 1, separable (rows then columns), mirror border. */
int orc_gauss(const double* V, int H, int W, double sigma, double* Vbar) {
  int r = (int)ceil(4.0 * sigma);
  if (r >= H || r >= W || sigma <= 0.0) return -1;
  double* w = (double*)malloc(sizeof(double) * (2 * r + 1));
  double* tmp = (double*)malloc(sizeof(double) * (size_t)H * W);
  if (!w || !tmp) {
    free(w);
    free(tmp);
    return -1;
  }
  double s = 0.0;
  for (int k = -r; k <= r; ++k) s += (w[k + r] = exp(-(double)k * k / (2.0 * sigma * sigma)));
  for (int k = 0; k <= 2 * r; ++k) w[k] /= s;
#pragma omp parallel for
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      double a = 0.0;
      for (int k = -r; k <= r; ++k) a += w[k + r] * V[(size_t)y * W + mirror(x + k, W)];
      tmp[(size_t)y * W + x] = a;
    }
#pragma omp parallel for
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      double a = 0.0;
      for (int k = -r; k <= r; ++k) a += w[k + r] * tmp[(size_t)mirror(y + k, H) * W + x];
      Vbar[(size_t)y * W + x] = a;
    }
  free(w);
  free(tmp);
  return 0;
}

/* Voltage trace extraction (Sec. II, third stage of the pipeline): the mean
 * pixel intensity within each ROI of one motion-corrected frame V [H][W].
 * masks [n_rois][H][W]: nonzero = pixel in the ROI; ROIs may overlap.  An
 * empty ROI gives 0 (reading: the paper never has one). */
void orc_roi_means(const double* V, int H, int W, const uint8_t* masks, int n_rois, double* out) {
  size_t hw = (size_t)H * W;
  for (int r = 0; r < n_rois; ++r) {
    const uint8_t* m = masks + hw * r;
    double sum = 0.0;
    long long cnt = 0;
    for (size_t px = 0; px < hw; ++px)
      if (m[px]) {
        sum += V[px];
        cnt++;
      }
    out[r] = cnt ? sum / (double)cnt : 0.0;
  }
}

static int cmp_double(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return (x > y) - (x < y);
}

/* Median by full sort.  Reading for an even count: mean of the two middle
 * order statistics. */
double orc_median(const double* v, int n) {
  double* t = (double*)malloc(sizeof(double) * n);
  memcpy(t, v, sizeof(double) * n);
  qsort(t, n, sizeof(double), cmp_double);
  double m = (n % 2) ? t[n / 2] : 0.5 * (t[n / 2 - 1] + t[n / 2]);
  free(t);
  return m;
}

/* ------------------------------------------------------------------------ */
/* Streaming pipeline with state carried across calls.                       */

typedef struct {
  int H, W, R, P, L, hp_w, flags;
  double sigma;
  double* T;       /* template H*W */
  int have_T;
  long long t;     /* frames seen */
  double* first_V; /* V of frame 0: the high-pass takes v[t<0] := v[0] */
  double* ring;    /* last hp_w frames of V, frame t at slot t % hp_w */
  int seg_n;       /* frames in the open segment */
  double* seg_V;   /* [L][H*W] corrected frames of the open segment */
  uint8_t* masks;  /* [n_rois][H*W] ROI masks for the voltage traces, or NULL */
  int n_rois;
  double* seg_Vb;  /* [L][H*W] smoothed frames of the open segment */
} orc_t;

void orc_destroy(orc_t* o) {
  if (!o) return;
  free(o->T);
  free(o->first_V);
  free(o->ring);
  free(o->seg_V);
  free(o->seg_Vb);
  free(o->masks);
  free(o);
}

orc_t* orc_create(int H, int W, int R, int P, int L, double sigma, int hp_w, int flags) {
  int g[4];
  if (orc_patch_grid(H, W, R, P, g) || L <= 0 || hp_w < 0) return NULL;
  if ((int)ceil(4.0 * sigma) >= H || (int)ceil(4.0 * sigma) >= W || sigma <= 0.0) return NULL;
  orc_t* o = (orc_t*)calloc(1, sizeof(orc_t));
  size_t hw = (size_t)H * W;
  o->H = H, o->W = W, o->R = R, o->P = P, o->L = L, o->hp_w = hp_w, o->flags = flags;
  o->sigma = sigma;
  o->T = (double*)calloc(hw, sizeof(double));
  o->first_V = (double*)calloc(hw, sizeof(double));
  o->ring = (double*)calloc(hw * (hp_w > 0 ? hp_w : 1), sizeof(double));
  o->seg_V = (double*)calloc(hw * L, sizeof(double));
  o->seg_Vb = (double*)calloc(hw * L, sizeof(double));
  if (!o->T || !o->first_V || !o->ring || !o->seg_V || !o->seg_Vb) {
    orc_destroy(o);
    return NULL;
  }
  return o;
}

void orc_set_template(orc_t* o, const double* T) {
  memcpy(o->T, T, sizeof(double) * (size_t)o->H * o->W);
  o->have_T = 1;
}

long long orc_frames_seen(const orc_t* o) { return o->t; }

/* ROI masks [n_rois][H][W] (copied) for the traces of orc_process; n_rois = 0
 * clears them.  Returns 0 or -1. */
int orc_set_rois(orc_t* o, const uint8_t* masks, int n_rois) {
  free(o->masks);
  o->masks = NULL;
  o->n_rois = 0;
  if (n_rois <= 0) return 0;
  size_t bytes = (size_t)n_rois * o->H * o->W;
  o->masks = (uint8_t*)malloc(bytes);
  if (!o->masks) return -1;
  memcpy(o->masks, masks, bytes);
  o->n_rois = n_rois;
  return 0;
}

int orc_estimate(const orc_t* o, const uint16_t* F, double* s, int* d, double* info,
                 double* C_out);

/* Places the stream at absolute frame t_start, a multiple of L (segments are
 * the absolute ranges [iL, (i+1)L), Sec. III-B), with no open segment; the n
 * frames before it ([n][H][W], frames t_start - n .. t_start - 1) only fill the
 * high-pass history (their shifts are estimated, nothing is emitted).  With
 * n >= min(t_start, hp_w - 1), every later output equals that of one stream
 * from frame 0.  Returns 0 or -1. */
int orc_seek(orc_t* o, long long t_start, const uint16_t* frames, int n) {
  if (!o || t_start < 0 || t_start % o->L != 0 || n < 0 || n > t_start) return -1;
  if (n > 0 && !o->have_T) return -1;
  int H = o->H, W = o->W;
  size_t hw = (size_t)H * W;
  o->t = t_start - n;
  o->seg_n = 0;
  double* V = (double*)malloc(sizeof(double) * hw);
  if (!V) return -1;
  for (int i = 0; i < n; ++i) {
    const uint16_t* F = frames + hw * i;
    double s[2], inf[3];
    int d[2];
    if (orc_estimate(o, F, s, d, inf, NULL)) {
      free(V);
      return -1;
    }
    orc_resample(F, H, W, s[0], s[1], V);
    if (o->hp_w > 0) {
      if (o->t == 0) memcpy(o->first_V, V, sizeof(double) * hw);
      memcpy(o->ring + hw * (size_t)(o->t % o->hp_w), V, sizeof(double) * hw);
    }
    o->t++;
  }
  free(V);
  return 0;
}

/* Motion estimate of one frame over the full +-R window: shift, integer peak,
 * and {C(d*), second C, flags}.  C_out (optional) receives the (2R+1)^2
 * surface. */
int orc_estimate(const orc_t* o, const uint16_t* F, double* s, int* d, double* info,
                 double* C_out) {
  int w = 2 * o->R + 1;
  double* C = C_out ? C_out : (double*)malloc(sizeof(double) * w * w);
  int rc = orc_surface(F, o->H, o->W, o->T, o->R, o->P, -o->R, -o->R, w, w, C, NULL);
  if (!rc) orc_peak(C, -o->R, -o->R, w, w, s, d, info);
  if (!C_out) free(C);
  return rc;
}

/* Process n frames [n][H][W].  When `shifts_in` is given those shifts are
 * applied instead of being estimated (the temporal stage alone).
 * Outputs (each optional): shifts [n][2], dstar [n][2], info [n][3],
 * surface [n][(2R+1)^2], corrected [n][H][W] (V, or the high-passed V when
 * ORC_FLAG_OUT_HIGHPASS is set), summary [k][2][H][W] (S_i then T_i), traces
 * [n][n_rois] (orc_roi_means of each corrected frame V, never the high-pass).
 * Returns k, the number of segments completed by this call, or -1.
 *
 * Segments (Sec. III-B) are the absolute frame ranges [iL, (i+1)L); only
 * complete segments are emitted and an open segment carries over.
 *   S_i(x) = (1/L) sum_t V_i(x, t)                       (Eq. 1)
 *   T_i(x) = max_t Vbar_i(x, t) - median_t Vbar_i(x, t)   (Eq. 2)
 * High-pass (not in the paper; reading): trailing boxcar baseline
 *   y[t] = v[t] - (1/W_hp) sum_{k=0}^{W_hp-1} v[t-k],  v[t<0] := v[0],
 * applied to V over the whole stream; it never feeds S_i or T_i. */
int orc_process(orc_t* o, const uint16_t* frames, int n, const double* shifts_in, double* shifts,
                int* dstar, double* info, double* surface, double* corrected, double* summary,
                double* traces) {
  if (!o || !o->have_T || n < 0) return -1;
  int H = o->H, W = o->W, w = 2 * o->R + 1;
  size_t hw = (size_t)H * W;
  double* V = (double*)malloc(sizeof(double) * hw);
  double* Vb = (double*)malloc(sizeof(double) * hw);
  double* med = (double*)malloc(sizeof(double) * o->L);
  if (!V || !Vb || !med) {
    free(V);
    free(Vb);
    free(med);
    return -1;
  }
  int k = 0;
  for (int i = 0; i < n; ++i) {
    const uint16_t* F = frames + hw * i;
    double s[2], inf[3];
    int d[2];
    if (shifts_in) {
      s[0] = shifts_in[2 * i];
      s[1] = shifts_in[2 * i + 1];
      d[0] = (int)lround(s[0]);
      d[1] = (int)lround(s[1]);
      inf[0] = inf[1] = inf[2] = 0.0;
    } else if (orc_estimate(o, F, s, d, inf, surface ? surface + (size_t)i * w * w : NULL)) {
      free(V);
      free(Vb);
      free(med);
      return -1;
    }
    if (shifts) shifts[2 * i] = s[0], shifts[2 * i + 1] = s[1];
    if (dstar) dstar[2 * i] = d[0], dstar[2 * i + 1] = d[1];
    if (info) memcpy(info + 3 * i, inf, sizeof(inf));
    orc_resample(F, H, W, s[0], s[1], V);
    if (traces && o->n_rois > 0)
      orc_roi_means(V, H, W, o->masks, o->n_rois, traces + (size_t)i * o->n_rois);
    long long t = o->t;
    if (o->hp_w > 0) {
      if (t == 0) memcpy(o->first_V, V, sizeof(double) * hw);
      memcpy(o->ring + hw * (size_t)(t % o->hp_w), V, sizeof(double) * hw);
    }
    if (corrected) {
      double* out = corrected + hw * i;
      if ((o->flags & ORC_FLAG_OUT_HIGHPASS) && o->hp_w > 0) {
        for (size_t px = 0; px < hw; ++px) {
          double base = 0.0;
          for (int q = 0; q < o->hp_w; ++q) {
            long long u = t - q;
            base += u < 0 ? o->first_V[px] : o->ring[hw * (size_t)(u % o->hp_w) + px];
          }
          out[px] = V[px] - base / o->hp_w;
        }
      } else {
        memcpy(out, V, sizeof(double) * hw);
      }
    }
    if (orc_gauss(V, H, W, o->sigma, Vb)) {
      free(V);
      free(Vb);
      free(med);
      return -1;
    }
    memcpy(o->seg_V + hw * o->seg_n, V, sizeof(double) * hw);
    memcpy(o->seg_Vb + hw * o->seg_n, Vb, sizeof(double) * hw);
    o->seg_n++;
    o->t++;
    if (o->seg_n == o->L) {
      if (summary) {
        double* S = summary + (size_t)k * 2 * hw;
        double* Tm = S + hw;
        for (size_t px = 0; px < hw; ++px) {
          double sum = 0.0, mx = -INFINITY;
          for (int q = 0; q < o->L; ++q) {
            sum += o->seg_V[hw * q + px];
            double b = o->seg_Vb[hw * q + px];
            if (b > mx) mx = b;
            med[q] = b;
          }
          S[px] = sum / o->L;
          Tm[px] = mx - orc_median(med, o->L);
        }
      }
      k++;
      o->seg_n = 0;
    }
  }
  free(V);
  free(Vb);
  free(med);
  return k;
}
