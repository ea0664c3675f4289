/*
 * vimg.h -- C ABI of the GB300-native frame-stream hot path for real-time
 * voltage imaging (Bando et al., "Real-time Neuron Segmentation for Voltage
 * Imaging", BIBM 2023).
 *
 * What one call computes, per uint16 frame F_t of an H x W video:
 *   1. Rigid motion estimate by zero-mean normalized cross-correlation (ZNCC)
 *      of 21x21 template patches tiled over the image, for every candidate
 *      displacement d in a (2R+1)^2 window, the patch values aggregated into
 *      one surface C_t(d) whose maximum is the frame's motion vector
 *      (Sec. II, "Motion correction").  The patch grid is the non-overlapping
 *      grid centred in the region where all shifted windows stay in bounds;
 *      C_t is the mean of the patch ZNCCs; ties go to the smallest |d|, then
 *      smallest dy, then dx; a 3-point parabola per axis refines the peak.
 *   2. Resampling: V_t(y,x) = F_t(y + s_y, x + s_x), bilinear, coordinates
 *      clamped to the image (the corrected video of Sec. II).
 *   3. Optional temporal high-pass of each pixel trace (trailing boxcar of
 *      hp_window frames, v[t<0] := v[0]).
 *   4. Time segments of L frames at absolute frame indices (Sec. III-B) and
 *      per segment the spatial summary S_i = temporal mean of V (Eq. 1) and
 *      the temporal summary T_i = max - median of the Gaussian-smoothed video
 *      (sigma 3 px, radius ceil(4 sigma), mirror border; Eq. 2).  The median
 *      of an even count is the mean of the two middle values.
 *
 * Conventions for every entry point:
 *   - Device pointers are caller-owned CUDA global-memory pointers on the
 *     handle's device; host pointers are ordinary (preferably pinned) host
 *     memory.  The library owns only its handle workspace.
 *   - All device work is enqueued on params.stream (0 = legacy default
 *     stream); the call returns without waiting for it, except the _host
 *     entry point, which synchronises before returning.  Outputs are valid
 *     once the caller has synchronised that stream.
 *   - Layouts are dense row-major: frames [n][H][W] uint16, shifts [n][2]
 *     float32 (dy, dx), corrected [n][H][W] float32, summaries [k][2][H][W]
 *     float32 with S_i before T_i.
 *   - Return value >= 0 is success (for process calls: k, the number of
 *     segments completed and written by this call).  Negative values are the
 *     VIMG_ERR_* codes; vimg_last_error() then describes the failure.  A
 *     device-side failure makes the handle's error sticky: every later call
 *     on that handle returns the same code.
 *   - A handle is not thread safe; use one handle per host thread.
 */
#ifndef VIMG_H
#define VIMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VIMG_OK 0
#define VIMG_ERR_ARG (-1)         /* invalid argument or NULL pointer            */
#define VIMG_ERR_NO_TEMPLATE (-2) /* vimg_set_template has not been called       */
#define VIMG_ERR_CUDA (-3)        /* a CUDA runtime call failed                  */
#define VIMG_ERR_TIMEOUT (-4)     /* a device-side wait gave up (sticky)         */
#define VIMG_ERR_OOM (-5)         /* device or host allocation failed            */
#define VIMG_ERR_SIZE (-6)        /* H or W below 2R + patch, or above limits    */

/* params.flags */
#define VIMG_CORR_BF16 1      /* BF16 tensor-core (tcgen05) correlation numerators:
                                 the frame minus the rounded template and the
                                 centred template go through BF16 with FP32
                                 accumulation; needs search_radius 16; not with
                                 VIMG_PROPOSAL_CNN                               */
#define VIMG_PROPOSAL_CNN 2   /* learned shift proposal + narrow window          */
#define VIMG_OUT_HIGHPASS 4   /* corrected output holds the high-passed video    */
#define VIMG_VIDEO_SUMMARY 8  /* accumulate the whole-video average and local
                                 correlation images (vimg_video_summary)          */
#define VIMG_TEMPORAL_SMEM 16 /* run the general temporal kernel (segment history
                                 in shared memory) even where the faster one
                                 (history in tensor memory, TMA-staged frames)
                                 applies; same results, for comparisons. The
                                 faster kernel needs W a multiple of 8, 16-byte
                                 aligned frame buffers and no high-pass output   */

typedef struct vimg_handle vimg_handle;

typedef struct {
  int search_radius;        /* R: displacements in [-R, R]^2; 0..16; default 16  */
  int patch;                /* patch side; the paper's 21 (Sec. II); 21 only     */
  int segment_len;          /* L; the paper's 50 (Sec. III-B); 1..50             */
  float gauss_sigma;        /* Eq. 2 smoothing sigma; the paper's 3.0; radius
                               ceil(4 sigma) must be <= 12                       */
  int hp_window;            /* boxcar high-pass length; 0 = off; <= 64           */
  int flags;                /* VIMG_* flags above                                */
  float fallback_zncc;      /* learned proposal: full search if C(d*) < this     */
  int narrow_radius;        /* learned proposal: window half-width (default 2)   */
  void* stream;             /* cudaStream_t for all work; NULL = default stream  */
  long long timeout_spins;  /* cap on any device-side wait loop                  */
  int max_chunk;            /* frames per internal batch (workspace sizing)      */
  int corr_group;           /* patches per work item of the FP32 correlation:
                               0 = 11 (fills 22-patch rows, 512 px); 7, 8, 10
                               or 11 (e.g. 7 for 35-patch rows, 768 px).  Only
                               the rounding of the FP32 sums depends on it      */
} vimg_params;

/* Fills *p with the defaults above (R = 16, patch 21, L = 50, sigma 3,
 * high-pass off, no flags, fallback 0.5, narrow radius 2, default stream,
 * max_chunk 200, corr_group 0 = 11). */
void vimg_default_params(vimg_params* p);

/* Creates a handle for H x W frames on the current CUDA device and allocates
 * its workspace.  Returns NULL on invalid parameters (see vimg_last_error(NULL)),
 * on VIMG_ERR_SIZE conditions, or when allocation fails. */
vimg_handle* vimg_create(int H, int W, const vimg_params* p);

/* Releases the handle and its workspace after draining its stream.  NULL is
 * accepted. */
void vimg_destroy(vimg_handle* h);

/* Sets the reference template T (device float32 [H][W]).  Per patch the
 * centred template T - mean(T_p) and its squared norm are precomputed on the
 * device (the constant parts of the ZNCC of Sec. II).  The template is copied;
 * the caller may reuse its buffer once the stream has passed this call.
 * Resets nothing else. */
int vimg_set_template(vimg_handle* h, const float* d_template);

/* Processes the next n >= 0 frames of the stream (device uint16 [n][H][W]).
 *   d_shifts_out    device float32 [n][2], the estimated (dy, dx) per frame;
 *                   may be NULL.
 *   d_corrected_out device float32 [n][H][W]: V_t, or the high-passed V_t when
 *                   VIMG_OUT_HIGHPASS is set; may be NULL.
 *   d_summary_out   device float32 [k][2][H][W] for the k segments completed
 *                   by this call, k = floor((frames_seen % L + n) / L); may be
 *                   NULL.
 * Frames of an unfinished segment (and the frames the high-pass still needs)
 * are kept in the handle, so any split of a stream into calls gives identical
 * results.  Returns k >= 0 or a VIMG_ERR_* code. */
int vimg_process(vimg_handle* h, const uint16_t* d_frames, int n, float* d_shifts_out,
                 float* d_corrected_out, float* d_summary_out);

/* Optional extra outputs and inputs of one process call.  Any member may be
 * NULL. */
typedef struct {
  float* shifts;          /* [n][2] estimated (dy, dx)                          */
  float* corrected;       /* [n][H][W]                                          */
  float* summary;         /* [k][2][H][W]                                       */
  float* peak_info;       /* [n][4]: dy*, dx*, C(d*), second-largest C          */
  double* surface;        /* [n][2R+1][2R+1] aggregated surface C_t, for
                             diagnostics and parity checks.  With
                             VIMG_PROPOSAL_CNN: the full surface for frames that
                             fell back to the full window; for the others only
                             the 7x7 narrow window is computed and every other
                             entry is NaN                                       */
  const float* shifts_in; /* [n][2]: apply these shifts instead of estimating
                             them (the temporal stage alone)                    */
  float* traces;          /* [n][n_rois] voltage traces: the mean of the corrected
                             frame V_t (never the high-pass) within each ROI set
                             by vimg_set_rois (Sec. II, third stage)            */
  float* prob;            /* [k][H][W] spiking-probability maps of the segments the
                             call completes (U-Net of Sec. III-C on each summary
                             pair); needs `summary` and a U-Net attached with
                             vimg_attach_unet                                   */
  float* proposal;        /* [n][2] the learned proposal (dy, dx) in px before
                             rounding (VIMG_PROPOSAL_CNN only): the narrow window
                             is centred on it, rounded to the nearest integer
                             and clamped to [-(R-3), R-3]                       */
} vimg_io;

/* Voltage-trace ROIs (Sec. II: the third stage of the pipeline takes the mean
 * pixel intensity within each detected neuron ROI for each frame of the
 * motion-corrected video).  d_masks: device uint8 [n_rois][H][W], nonzero =
 * pixel in the ROI; ROIs may overlap, up to 4 at any pixel (more returns
 * VIMG_ERR_ARG with the previous ROIs kept).  0 <= n_rois <= 65535; n_rois = 0
 * clears the ROIs.  The traces are accumulated inside the fused temporal pass
 * in 2^-20 fixed point (exact and independent of the order of the additions);
 * an empty ROI gives 0.  Synchronises the handle's stream (it checks the
 * overlap limit).  Returns VIMG_OK or an error. */
int vimg_set_rois(vimg_handle* h, const uint8_t* d_masks, int n_rois);

/* Whole-video summary images of the motion-corrected video V over every frame
 * since vimg_create / vimg_reset (handle created with VIMG_VIDEO_SUMMARY): the
 * temporal average A(x) = mean_t V(x, t) and the local correlation image C(x) =
 * mean over the in-image 8-neighbours y of the Pearson correlation over time of
 * V(x, .) and V(y, .) (0 for a constant trace) -- the two images VolPy derives
 * from a whole video, which Sec. III-A and Fig. 2 compare with the per-segment
 * summaries.  Accumulated per pixel in FP32 within a call's internal batch and in
 * FP64 across batches.  d_average, d_correlation: device float32 [H][W] (either
 * may be NULL); enqueued on the handle's stream.  VIMG_ERR_ARG without the flag
 * or before the first frame. */
int vimg_video_summary(vimg_handle* h, float* d_average, float* d_correlation);

/* Same as vimg_process with the vimg_io members.  Returns k or an error. */
int vimg_process_io(vimg_handle* h, const uint16_t* d_frames, int n, const vimg_io* io);

/* End-to-end variant with HOST buffers: h_frames host uint16 [n][H][W] is
 * streamed to the device in batches of max_chunk frames, the first a quarter of
 * that (uploads run up to two batches ahead of the compute, into a ring of
 * three device stages; only the first batch's upload is not overlapped), and the
 * shifts (host float32 [n][2]) and the summaries (host float32 [k][2][H][W])
 * are copied back on a stream of their own.  Host buffers should be pinned for
 * the copies to overlap the compute.  Either output
 * may be NULL.  d_corrected_out is an optional DEVICE buffer [n][H][W].
 * Whole-video summary sums (VIMG_VIDEO_SUMMARY) accumulate as in vimg_process;
 * voltage traces and probability maps need vimg_process_io.
 * Synchronises before returning.  Returns k or an error. */
int vimg_process_host(vimg_handle* h, const uint16_t* h_frames, int n, float* h_shifts_out,
                      float* h_summary_out, float* d_corrected_out);

/* Waits for the handle's stream and reports device-side failures: returns
 * VIMG_ERR_TIMEOUT (sticky) if a kernel's bounded wait gave up (the kernel then
 * stopped issuing work and returned), VIMG_ERR_CUDA on a CUDA error, else
 * VIMG_OK. */
int vimg_synchronize(vimg_handle* h);

/* Frames seen by the handle so far (host-side counter; no device sync). */
long long vimg_frames_seen(const vimg_handle* h);

/* Forgets the stream state (frames seen, open segment, high-pass history);
 * keeps the template. */
int vimg_reset(vimg_handle* h);

/* Starts the stream at absolute frame index t_start, a multiple of the segment
 * length L, as if the frames before it had been processed: segments then fall
 * on the absolute ranges [iL, (i+1)L) (Sec. III-B), and the shifts, corrected
 * (or high-passed) frames, segment summaries and traces of frames t >= t_start
 * equal, bit for bit, those of one stream over the whole video from frame 0.
 * This is how one video is cut into time shards that independent handles (on
 * one GPU or several) process.  d_history: device uint16 [n_history][H][W], the
 * frames t_start - n_history .. t_start - 1; the high-pass needs the last
 * min(t_start, hp_window - 1) of them (their shifts are estimated; nothing is
 * output for them, and the whole-video summary images start empty).  Resets
 * the state first, like vimg_reset.  Enqueued on the handle's stream.  Returns
 * VIMG_OK or an error (VIMG_ERR_ARG for t_start not a multiple of L or too
 * short a history). */
int vimg_seek(vimg_handle* h, long long t_start, const uint16_t* d_history, int n_history);

/* Stream-state checkpoint and restore.  What carries over from one call to the
 * next is the stream position, the frames of the open segment with their
 * shifts (which also hold the high-pass history; Sec. III-B segments span
 * calls), the whole-video summary sums (VIMG_VIDEO_SUMMARY) and the proposal
 * counters.  vimg_state_bytes: size in bytes of the current state (it grows
 * with the frames held for the open segment), or a negative VIMG_ERR_* code.
 * vimg_get_state: waits for the handle's streams and writes the state to host
 * memory `host` of `bytes` bytes (>= vimg_state_bytes; VIMG_ERR_ARG if
 * smaller).  vimg_set_state: replaces the handle's state by one that
 * vimg_get_state wrote on a handle of the same H, W, segment length,
 * high-pass window, search radius and flags (VIMG_ERR_ARG otherwise, state
 * unchanged); the template, proposal weights and ROIs are not part of it.
 * After a restore the stream continues bit for bit as the checkpointed one
 * would have.  Both return VIMG_OK or an error. */
long long vimg_state_bytes(const vimg_handle* h);
int vimg_get_state(vimg_handle* h, void* host, long long bytes);
int vimg_set_state(vimg_handle* h, const void* host, long long bytes);

/* Message for the last failure on h, or for the last failed vimg_create on
 * this host thread when h is NULL.  Never NULL. */
const char* vimg_last_error(const vimg_handle* h);

/* ---- Learned shift proposal -------------------------------------------------
 * A 6-layer CNN (3x3 convolutions, 32 channels, stride 2 in layers 1-5, ReLU,
 * global average pool, linear 32 -> 2) reads the 128x128 centre crops of the
 * frame and of the template (each normalised by its own mean and standard
 * deviation) and regresses the frame's shift.  With VIMG_PROPOSAL_CNN the
 * correlation of Sec. II then runs only on the 7x7 displacements around the
 * rounded proposal (+-2 px plus a refinement ring); a frame whose peak lies on
 * that window's border or whose C(d*) is below params.fallback_zncc is searched
 * again over the full +-R window (a device-side list, no host round trip).
 * Weights are used in BF16 with FP32 accumulation; training keeps FP32 master
 * weights.  The paper's own network is a segmentation U-Net; this proposal
 * network is an addition of this library.  All pointers are device pointers;
 * all calls enqueue on `stream` and return VIMG_OK or an error code.
 * Parameter layout (floats): per convolution weights [32][c_in][3][3] then
 * bias [32] (c_in = 2 for the first layer, 32 after), then the linear weights
 * [2][32] and bias [2].  Network output = shift / 12 px. */
int vimg_cnn_param_count(void);
/* Floats of activation workspace for a batch of n samples. */
size_t vimg_cnn_workspace_floats(int n);
/* Writes the normalised input crops of n frames [n][H][W] (H, W >= 128) into
 * the start of the workspace d_ws.  The template of sample b is d_template +
 * b * template_stride (template_stride = 0: one template [H][W] for all). */
int vimg_cnn_prepare(const uint16_t* d_frames, int n, int H, int W, const float* d_template,
                     long long template_stride, float* d_ws, void* stream);
/* BF16 copy of the parameters (d_params_bf16: vimg_cnn_param_count() bf16). */
int vimg_cnn_pack_bf16(const float* d_params, void* d_params_bf16, void* stream);
/* Forward of the prepared batch: d_out [n][2] (shift / 12), activations kept
 * in d_ws for the backward pass. */
int vimg_cnn_forward(const float* d_params, const void* d_params_bf16, float* d_ws, int n,
                     float* d_out, void* stream);
/* Mean squared error against d_target [n][2] (px): d_dout [n][2] and, if
 * d_loss is not NULL, the loss (one float). */
int vimg_cnn_loss(const float* d_out, const float* d_target, int n, float* d_dout, float* d_loss,
                  void* stream);
/* Backward pass: adds the parameter gradients to d_grads (zero it first);
 * d_dws is a second workspace of vimg_cnn_workspace_floats(n) floats. */
int vimg_cnn_backward(const float* d_params, const void* d_params_bf16, const float* d_ws,
                      float* d_dws, int n, const float* d_dout, float* d_grads, void* stream);
/* One Adam step (bias-corrected, step counts from 1) on the FP32 parameters. */
int vimg_cnn_adam(float* d_params, const float* d_grads, float* d_m, float* d_v, float lr,
                  float beta1, float beta2, float eps, int step, void* stream);
/* Copies trained FP32 parameters into the handle (kept as BF16 for inference). */
int vimg_load_proposal(vimg_handle* h, const float* d_params);
/* Frames estimated and frames that fell back to the full window since the
 * handle was created (synchronises the handle's stream). */
int vimg_proposal_stats(vimg_handle* h, long long* frames, long long* fallbacks);

/* ---- Several videos per call -------------------------------------------------
 * A serving-shaped scheduling layer over the per-video method; the paper has
 * no counterpart (it processes one recording at a time).  Each video v has its
 * own handle hs[v] (own H x W, template and stream state) and processes the
 * next ns[v] >= 0 frames of d_frames[v] (device uint16 [ns[v]][H_v][W_v]),
 * with the same outputs and the same results, bit for bit, as vimg_process on
 * that handle.  The call advances in steps: per step every video with frames
 * left takes up to `chunk` of them (shortened to end on a segment boundary),
 * and each kernel of the path (window statistics, correlation, peak, fused
 * temporal pass) is launched once for the step's videos, up to 8 videos per
 * launch (more are split into groups of 8).
 *
 * Requirements: 1 <= k <= 64 distinct handles on one device, each with its
 * template set, created without VIMG_CORR_BF16, VIMG_PROPOSAL_CNN and
 * VIMG_VIDEO_SUMMARY (the batched form runs the full-window FP32 method and
 * the outputs below; voltage traces and probability maps need vimg_process_io).  Work is enqueued on hs[0]'s
 * stream; the other handles' streams are ordered before and after the call
 * with events.  Output arrays have k entries; any entry (or the whole array)
 * may be NULL.  d_shifts_out[v] is [ns[v]][2]; d_summary_out[v] is
 * [k_v][2][H_v][W_v] as for vimg_process.  d_corrected_out[v] is
 * [ns[v]][H_v][W_v], or, with ring_chunks > 0, a ring of ring_chunks slots of
 * `chunk` frames: step s writes its frames from the start of slot
 * (s mod ring_chunks).  segments_out (k ints, may be NULL) receives k_v.
 * Returns the sum of the k_v or a VIMG_ERR_* code (the message is on hs[0]). */
typedef struct {
  int chunk;        /* frames per video per step; 0 = each handle's max_chunk;
                       must not exceed any handle's max_chunk                   */
  int ring_chunks;  /* 0: contiguous corrected output; > 0: ring slots        */
  int use_graph;    /* 1: record the call's launches into a CUDA graph once and
                       replay it for identical calls (same handles in the same
                       stream state, same pointers, sizes and options)         */
  int reserved;     /* 0 */
} vimg_batch_opts;

int vimg_process_batch(vimg_handle* const* hs, int k, const uint16_t* const* d_frames,
                       const int* ns, float* const* d_shifts_out, float* const* d_corrected_out,
                       float* const* d_summary_out, int* segments_out,
                       const vimg_batch_opts* opts);

/* Per-stage timing with CUDA events recorded around each of the library's
 * launches on params.stream (off by default).  Stages:
 *   0 window statistics, 1 correlation numerators, 2 peak + refinement,
 *   3 fused temporal pass, 4 learned proposal, 5 carry copies (not a kernel),
 *   6 downstream outputs (voltage-trace finalize, whole-video summary sums).
 * vimg_profile_read synchronises the stream, writes the summed milliseconds
 * and the launch counts of each stage into ms[VIMG_NSTAGES] and
 * launches[VIMG_NSTAGES] (either may be NULL), and clears them when reset != 0.
 * At most 65,536 launches are recorded between reads; later ones are counted
 * but not timed.  Returns VIMG_OK or an error. */
#define VIMG_NSTAGES 7
int vimg_profile_enable(vimg_handle* h, int on);
int vimg_profile_read(vimg_handle* h, double* ms, long long* launches, int reset);

/* Motion estimate with no allocation at all, for callers that cannot allocate
 * device memory when they need shifts: real-time acquisition loops that forbid
 * allocator calls (an allocation can synchronise the device or block on the
 * driver and miss the frame deadline), and hosts that have already reserved all
 * device memory for their own frame buffers.  The paper has no counterpart; it
 * is an interface of this library.
 *
 * Computes, for n frames (device uint16 [n][H][W]) against the template
 * (device float32 [H][W]), the same shifts as vimg_process's motion estimate:
 * d_shifts_out device float32 [n][2] (dy, dx); d_peak_info (optional) device
 * float32 [n][4] as in vimg_io.  No handle, no stream state.  All scratch lives
 * in one 12 MiB array in the library's static device memory, which every GPU
 * that loads the library holds until the process exits.  Frames up to
 * 1024 x 1024 (search_radius <= 16) fit; larger ones return VIMG_ERR_SIZE with
 * nothing enqueued.  The first call on a device looks up the array's device
 * address and sets the kernels' attributes with that device current: make it
 * before any stream capture.  Every
 * call shares the array (and clears what must start at zero); calls whose work
 * overlaps on the GPU race and give wrong results, so serialise them.  Work is
 * enqueued on `stream` (NULL = default stream).  Returns VIMG_OK or an error
 * code (VIMG_ERR_ARG, VIMG_ERR_SIZE, VIMG_ERR_CUDA). */
int vimg_motion_noalloc(const float* d_template, const uint16_t* d_frames, int n, int H, int W,
                        int search_radius, float* d_shifts_out, float* d_peak_info,
                        void* stream);

/* Library version string. */
const char* vimg_version(void);

/* Measures the device's FP32 FMA rate (FLOP/s, 2 per FMA) with a kernel of
 * independent FMA chains on every SM, timed on `stream` (NULL = default) after
 * a warm-up run; synchronous.  The denominator of the FP32 correlation kernel's
 * ALU roofline.  The paper has no counterpart.  Returns VIMG_OK or an error. */
int vimg_fma_rate(void* stream, double* flops_per_s);

/* ---- spiking-pixel U-Net (Sec. III-C) ---------------------------------------
 * A U-Net on 64x64 patches of a segment's summary pair (S_i, T_i) gives the
 * probability that spiking neurons lie at each pixel during the segment; the
 * patches (every 32 px along each axis plus one flush with the far border) are
 * merged into one H x W map by a weighted average with the tent weight
 * w(u) w(v), w(u) = min(u + 1, 64 - u).  Inputs are S_i and T_i standardised
 * over the whole image, (x - mean) / (std + 1e-3).
 *
 * Network (layer sizes are a reading; the paper's figure is not available):
 * levels at 64, 32, 16, 8, 4 px with 16, 32, 64, 128, 256 channels; per level
 * two 3x3 convolutions (zero padding 1) + ReLU, 2x2 max pooling between
 * levels; decoder: 2x2 stride-2 up-convolution (no activation), concatenation
 * [skip, up], two 3x3 convolutions + ReLU; output 1x1 convolution 16 -> 1 and
 * a sigmoid.  3x3 and up-convolutions run on the tensor cores with BF16
 * weights and activations and FP32 accumulation; the output layer in FP32.
 *
 * Parameters: flat float32, per layer in network order (vimg_unet_layers) the
 * weights then the bias; 3x3 weights [Cout][Cin][3][3], up-convolution weights
 * [Cin][Cout][2][2] (out[co][2y+i][2x+j] += in[ci][y][x] w[ci][co][i][j]),
 * output weights [16] and bias [1]. */
typedef struct vimg_unet vimg_unet;

/* Number of parameters (floats). */
int vimg_unet_param_count(void);

/* Architecture in parameter order: kind (0 = 3x3 convolution + ReLU, 1 = 2x2
 * up-convolution, 2 = 1x1 output + sigmoid), input and output channels of
 * the first `cap` layers (NULL arrays allowed).  Returns the layer count. */
int vimg_unet_layers(int* kind, int* cin, int* cout, int cap);

/* Workspace for H x W summary images (64 <= H, W <= 8192) and up to
 * `max_segments` segments per internal pass; all calls enqueue on `stream`
 * (a cudaStream_t, NULL = legacy default).  NULL on failure
 * (vimg_unet_last_error(NULL) says why). */
vimg_unet* vimg_unet_create(int H, int W, int max_segments, void* stream);
void vimg_unet_destroy(vimg_unet* u);
const char* vimg_unet_last_error(const vimg_unet* u);

/* Converts the parameters (device float32, vimg_unet_param_count floats) into
 * the tensor-core layout.  Synchronous: the array may be freed on return. */
int vimg_unet_load(vimg_unet* u, const float* d_params);

/* d_summary: device float32 [k][2][H][W] (S_i, T_i); d_prob: device float32
 * [k][H][W].  Any k >= 0 (processed max_segments at a time). */
int vimg_unet_run(vimg_unet* u, const float* d_summary, int k, float* d_prob);

/* Synchronises the stream; VIMG_ERR_TIMEOUT (sticky) if a tensor-core kernel's
 * bounded wait gave up. */
int vimg_unet_synchronize(vimg_unet* u);

/* CUDA-event timing of the tensor-core launches and of whole runs (ms), summed
 * until read with reset != 0.  Profiling synchronises at the end of each run. */
int vimg_unet_profile(vimg_unet* u, int on);
int vimg_unet_profile_read(vimg_unet* u, double* conv_ms, double* total_ms,
                           long long* conv_launches, int reset);

/* Inspection of the last internal pass of vimg_unet_run (its n_patches =
 * patches of up to max_segments segments, patch order segment-major, then
 * patch rows, then patch columns): i = 0 the standardised input patches
 * (BF16 [n][64][64][16], channels 0 and 1 = S, T), i = 1..22 the output of the
 * i-th 3x3 or up-convolution in execution order (BF16 NHWC [n][side][side][C];
 * execution order = parameter order), i = 23 the per-patch probabilities
 * (float32 [n][64][64]).  Reports n_patches, side and C; copies into d_out
 * (device, dense) on the stream unless it is NULL. */
int vimg_unet_activation(vimg_unet* u, int i, void* d_out, int* n_patches, int* side,
                         int* channels);

/* ---- footprint reconstruction (Sec. III-D) -------------------------------------
 * From per-segment spiking-probability maps p_i (e.g. vimg_io.prob): binary masks
 * p_i > 0.5; 8-connected components kept if 20 <= area <= 1000 px, eccentricity
 * (pixel-centre covariance) <= 0.95 and concaveness 1 - area / convex-hull area
 * (hull of the pixel squares) <= 0.3; b = OR over segments; each 8-connected
 * component of b ("region") is factorised by NMF, P ~ F A (Eq. 3; rows = the
 * region's pixels, columns = segments), with N = the number of clusters of its
 * kept blobs (a blob joins the first cluster whose first blob it overlaps with
 * IoU >= 1/2) and 100 multiplicative updates from the clusters' union masks.
 * The constants are readings: the paper names the criteria, not their values.
 * Neurons are numbered by region (smallest pixel index), then cluster.
 *
 * Capacity: the NMF kernel holds a region of at most 16,000 pixels and 32
 * clusters.  A region beyond either limit is not factorised (it contributes no
 * neuron) and is reported by vimg_segment_status; every other region's result
 * is unaffected. */
#define VIMG_REGION_TOO_LARGE 1 /* more than 16,000 pixels */
#define VIMG_REGION_TOO_MANY 2  /* more than 32 clusters */
typedef struct vimg_segmenter vimg_segmenter;

/* Workspace for H x W maps and up to max_segments of them; NULL on failure. */
vimg_segmenter* vimg_segmenter_create(int H, int W, int max_segments, void* stream);
void vimg_segmenter_destroy(vimg_segmenter* s);
const char* vimg_segmenter_last_error(const vimg_segmenter* s);

/* d_prob: device float32 [K][H][W].  Outputs (device, any may be NULL):
 * d_footprints float32 [max_neurons][H][W] (F columns, 0 outside the region),
 * d_activity float32 [max_neurons][K] (rows of A), d_region_map int32 [H][W]
 * (region of each pixel of b, -1 elsewhere); *n_regions (host) = regions.
 * Synchronous.  Returns the number of neurons found (only the first
 * max_neurons are written) or an error code. */
int vimg_segment(vimg_segmenter* s, const float* d_prob, int K, float* d_footprints,
                 float* d_activity, int max_neurons, int* d_region_map, int* n_regions);

/* Per-region status of the last vimg_segment call, in region order (host int
 * array of n entries; the first min(n, regions) are written): 0 = factorised,
 * VIMG_REGION_TOO_LARGE or VIMG_REGION_TOO_MANY = beyond the NMF kernel's
 * capacity, not factorised.  Returns the number of regions of that call (0
 * after a failed call) or VIMG_ERR_ARG. */
int vimg_segment_status(const vimg_segmenter* s, int* status, int n);

/* Attaches a U-Net of the same H x W to a handle (NULL detaches); the handle
 * does not own it.  vimg_process_io then fills vimg_io.prob on the handle's
 * stream. */
int vimg_attach_unet(vimg_handle* h, vimg_unet* u);

#ifdef __cplusplus
}
#endif

#endif /* VIMG_H */
