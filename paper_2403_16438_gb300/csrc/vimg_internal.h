// Internal definitions shared by the CUDA translation units of libvimg.
// Not part of the public ABI (include/vimg.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vimg.h"

namespace vimg {

constexpr int kPatch = 21;               // patch side (Sec. II)
constexpr int kPatchArea = kPatch * kPatch;
constexpr int kMaxR = 16;                // largest search radius
constexpr int kMaxWin = 2 * kMaxR + 1;   // 33 displacements per axis
constexpr int kInvStride = 36;           // padded row of per-window factors
constexpr int kTplStride = 24;           // padded template-patch row (floats)
constexpr int kGaussMaxRadius = 12;      // ceil(4 * 3)
constexpr int kTile = 32;                // temporal-kernel output tile side
constexpr int kMaxL = 50;                // longest segment the temporal kernel holds
constexpr int kMaxHp = 64;               // longest high-pass window
constexpr double kFix = 1099511627776.0; // 2^40: fixed-point scale of C sums
constexpr int kNarrowWin = 7;            // learned proposal: +-2 px plus a refinement ring
constexpr int kCrop = 128;               // learned proposal: centre crop side
constexpr float kShiftScale = 12.0f;     // network output x 12 = shift in px

struct PatchGrid {
  int ny, nx, y0, x0;
};

// Per-handle template constants on the device.
struct TemplateDev {
  float* tc;   // [np][21][kTplStride] centred template patches
  float* tn2;  // [np] squared norms of the centred patches
  int* coff;   // [np] integer offsets ~ patch means (exactness of F - c in fp32)
};

// Where the frames of one temporal-kernel launch come from.  Virtual frame v
// (0 <= v < n_virtual) is absolute frame t_first + v; v < n_carry lives in the
// carry buffer, the rest in the caller's batch.
struct FrameSource {
  const uint16_t* carry;     // [n_carry][H][W]
  const float* carry_shift;  // [n_carry][2]
  const uint16_t* batch;     // [n_batch][H][W]
  const float* batch_shift;  // [n_batch][2]
  int n_carry, n_batch;
  long long t_first;         // absolute index of virtual frame 0
  long long t_new;           // absolute index of the first frame new to this call
};

struct TemporalArgs {
  FrameSource src;
  int H, W, L, hp_w, gauss_r;
  float gw[2 * kGaussMaxRadius + 1];  // normalised Gaussian taps
  long long seg_base;                 // absolute start of segment slot 0
  int n_seg;                          // segment slots in this launch
  int out_hp;                         // corrected output holds the high-pass
  int pairs;                          // stage frames as 2-pixel words (W even, 4-byte aligned)
  const unsigned long long* roi_members;  // [H][W] up to 4 ROI ids + 1 (16 bits each), or null
  unsigned long long* roi_acc;        // [n_batch][n_rois] fixed-point sums of V, or null
  int n_rois;
  float* corrected;                   // [n_batch][H][W] or null
  float* summary;                     // [k][2][H][W] or null (slot j -> index j)
  int* err;                           // sticky device error flag (bounded waits), or null
  int smem_history;                   // force the shared-memory-history kernel
};

// ---- several videos per launch ----------------------------------------------
// The motion and temporal kernels take a table of per-video jobs by value
// (__grid_constant__); a CTA finds its job from the prefix counts of work items.
// A single video is a table of one job.
constexpr int kMaxVideos = 8;

struct MotionJob {
  const uint16_t* frames;     // [nf][H][W]
  float* isf;                 // [nf][stats map] per-window 1/sqrt(SF)
  unsigned long long* csum;   // [nf][w*w] fixed-point C sums
  const float* tc;            // template constants (TemplateDev)
  const float* tn2;
  const int* coff;
  float* shifts;              // [nf][2] or null
  float* info;                // [nf][4] or null
  double* surface;            // [nf][w*w] or null
  int* err;                   // sticky device error flag of bounded waits, or null
  PatchGrid g;
  int nf, H, W, R;
  int cg;                     // patches per FP32 correlation item (0 = 11; 7, 8, 10, 11)
};

struct MotionBatch {
  int n;                               // jobs in use
  int stats_begin[kMaxVideos + 1];     // prefix counts of work items per kernel
  int corr_begin[kMaxVideos + 1];
  int peak_begin[kMaxVideos + 1];
  MotionJob j[kMaxVideos];
};

struct TemporalBatch {
  int n;
  int begin[kMaxVideos + 1];  // prefix counts of (tile, segment slot) items
  TemporalArgs a[kMaxVideos];
};

// Job index of work item `item` (begin[] ascending, begin[0] = 0).
__host__ __device__ __forceinline__ int job_of(const int* begin, int n, int item) {
  int j = 0;
  while (j + 1 < n && item >= begin[j + 1]) ++j;
  return j;
}

// ---- one-time set-up per device ------------------------------------------------
// Kernel attributes (cudaFuncSetAttribute) and the SM count belong to a device:
// the set-up below runs once for every device the library is used on, with that
// device current.
constexpr int kMaxDevices = 64;

// Index of the current device, or -1 (no device, or beyond kMaxDevices).
inline int current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return -1;
  return dev;
}

// Runs fn() once per device; done[] holds one flag per device.  Concurrent first
// calls may both run fn, which must therefore be idempotent.
template <class Fn>
cudaError_t once_per_device(unsigned char (&done)[kMaxDevices], Fn fn) {
  const int dev = current_device();
  if (dev < 0) return cudaErrorInvalidDevice;
  if (__atomic_load_n(&done[dev], __ATOMIC_ACQUIRE)) return cudaSuccess;
  const cudaError_t e = fn(dev);
  if (e == cudaSuccess) __atomic_store_n(&done[dev], (unsigned char)1, __ATOMIC_RELEASE);
  return e;
}

// SM count of the current device (0 if unknown); cached per device.
int sm_count();

// Fills the prefix counts; returns false if a job is malformed.
bool motion_batch_finalize(MotionBatch& b);
bool temporal_batch_finalize(TemporalBatch& b);
// One launch per stage over every job of the table.
cudaError_t launch_stats_multi(const MotionBatch& b, cudaStream_t st, const int* list = nullptr,
                               const int* list_n = nullptr);
cudaError_t launch_corr_f32_multi(const MotionBatch& b, cudaStream_t st,
                                  const int* list = nullptr, const int* list_n = nullptr);
cudaError_t launch_peak_multi(const MotionBatch& b, cudaStream_t st, const int* list = nullptr,
                              const int* list_n = nullptr);
cudaError_t launch_temporal_multi(const TemporalBatch& b, cudaStream_t st);
// Sets kernel attributes once per device (before any stream capture).
cudaError_t kernels_init();
cudaError_t temporal_init();

// ---- launchers (each enqueues on `st`; returns cudaGetLastError()) ----------
cudaError_t launch_template_prep(const float* T, int H, int W, PatchGrid g, TemplateDev td,
                                 cudaStream_t st);
size_t stats_map_floats(PatchGrid g, int R);  // per frame
// list/list_n (device): only the listed frames (count read on the device).
// err (device, may be null): the flag a bounded wait that gave up sets; without
// it the statistics run on the kernel that stages with plain loads.
cudaError_t launch_stats(const uint16_t* frames, int nf, int H, int W, PatchGrid g, int R,
                         const TemplateDev& td, float* isf, cudaStream_t st,
                         const int* list = nullptr, const int* list_n = nullptr,
                         int* err = nullptr);
// Only the isf entries of the narrow windows around the proposals.
cudaError_t launch_stats_narrow(const uint16_t* frames, int nf, int H, int W, PatchGrid g, int R,
                                const float* prop, float* isf, cudaStream_t st);
// list/list_n (device): process only the listed frames (count read on the device).
// cg: patches per work item of the FP32 correlation (0 = the default 11; 7, 8,
// 10 or 11; corr_group_valid).
bool corr_group_valid(int cg);
cudaError_t launch_corr_f32(const uint16_t* frames, int nf, int H, int W, PatchGrid g, int R,
                            const TemplateDev& td, const float* isf,
                            unsigned long long* csum, cudaStream_t st,
                            const int* list = nullptr, const int* list_n = nullptr, int cg = 0);
cudaError_t launch_peak(const unsigned long long* csum, int nf, int R, int np, float* shifts,
                        float* peak_info, double* surface, cudaStream_t st,
                        const int* list = nullptr, const int* list_n = nullptr);
cudaError_t launch_corr_narrow(const uint16_t* frames, int nf, int H, int W, PatchGrid g, int R,
                               const TemplateDev& td, const float* isf, const float* prop,
                               unsigned long long* csum, cudaStream_t st);
// surface (optional): the 7x7 values placed in the full grid; prop_px (optional):
// the proposals in px.
cudaError_t launch_peak_narrow(const unsigned long long* csum, int nf, int R, int np,
                               const float* prop, float thresh, float* shifts, float* info,
                               int* list, int* list_n, double* surface, float* prop_px,
                               cudaStream_t st);

cudaError_t launch_count_add(const int* n, long long* total, cudaStream_t st);

// BF16 tensor-core correlation (corr_bf16.cu)
size_t bf16_astore_bytes(PatchGrid g);              // per-patch Toeplitz template stores
int bf16_row_pitch(int W);
size_t bf16_fc_elems(int cap_frames, int H, int W);  // frame-offset image buffer
size_t bf16_tensor_map_bytes();
int bf16_tensor_map(void* map_out, __nv_bfloat16* fc, int cap_frames, int H, int W);
cudaError_t bf16_template_prep(const float* T, int H, int W, PatchGrid g, int R,
                               const TemplateDev& td, float* tround, __nv_bfloat16* as,
                               float* bgc, cudaStream_t st);
cudaError_t bf16_make_fc(const uint16_t* frames, int nf, int cap_frames, int H, int W,
                         const float* tround, __nv_bfloat16* fc, cudaStream_t st);
cudaError_t launch_corr_bf16(const void* tmap, int nf, int R, PatchGrid g,
                             const __nv_bfloat16* as, const float* bgc, const TemplateDev& td,
                             const float* isf, float* num, unsigned long long* csum, int* err,
                             cudaStream_t st);

// learned proposal (cnn.cu)
int cnn_param_count();
size_t cnn_act_floats(int n);
cudaError_t cnn_input(const uint16_t* frames, int n, int H, int W, const float* tmpl,
                      long long tmpl_stride, float* acts, cudaStream_t st);
cudaError_t cnn_forward(const float* params, const __nv_bfloat16* wb, float* acts, int n,
                        float* out, cudaStream_t st);
cudaError_t cnn_backward(const float* params, const __nv_bfloat16* wb, const float* acts,
                         float* dacts, int n, const float* dout, float* grads, cudaStream_t st);
cudaError_t cnn_mse(const float* out, const float* target, int n, float* dout, float* loss,
                    cudaStream_t st);
cudaError_t cnn_adam(float* p, const float* g, float* m, float* v, float lr, float b1, float b2,
                     float eps, int step, cudaStream_t st);
cudaError_t cnn_to_bf16(const float* p, __nv_bfloat16* q, cudaStream_t st);
cudaError_t launch_temporal(const TemporalArgs& a, cudaStream_t st);
// Voltage-trace ROIs: per-pixel membership (up to 4 ids + 1 packed in 16-bit
// fields) and per-ROI pixel counts from uint8 masks; *too_many set when a pixel
// lies in more than 4 ROIs.
cudaError_t roi_build(const uint8_t* masks, int n_rois, int H, int W,
                      unsigned long long* members, int* counts, int* too_many, cudaStream_t st);
// traces[f][r] = acc[f][r] / (2^20 * counts[r]) (0 for an empty ROI).
cudaError_t roi_finalize(const unsigned long long* acc, const int* counts, int nf, int n_rois,
                         float* traces, cudaStream_t st);
constexpr double kRoiFix = 1048576.0;  // 2^20: fixed-point scale of the trace sums
// Whole-video summary images: per-pixel FP64 sums [6][H][W] of d = V - T, d^2 and
// d times the E, S, SE, SW neighbours over nf frames; and the images from them.
cudaError_t launch_vsum(const uint16_t* frames, const float* shifts, int nf, int H, int W,
                        const float* ref, double* acc, cudaStream_t st);
cudaError_t launch_vsum_final(const double* acc, const float* ref, long long n, int H, int W,
                              float* avg, float* corr, cudaStream_t st);

}  // namespace vimg

// U-Net stage on a given stream (the handle's, when attached).
int vimg_unet_run_on(vimg_unet* u, const float* d_summary, int k, float* d_prob, cudaStream_t st);
int unet_dims(const vimg_unet* u, int* H, int* W);
