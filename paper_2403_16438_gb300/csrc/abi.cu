// C ABI of libvimg (include/vimg.h): handle, argument checks, device workspace,
// stream state carried across calls, and the order of kernel launches per call.
//
// Per internal batch of at most max_chunk frames (batches end on segment
// boundaries whenever possible, so the batch's raw frames are still in L2 when
// the temporal pass reads them again):
//   1. motion estimate of the whole batch: zero the fixed-point surfaces, window
//      statistics, correlation numerators, integer peak + parabola;
//   2. one fused temporal launch over every segment slot the batch touches (and,
//      with ROIs set, the voltage traces of the batch's frames);
//   3. the raw frames and shifts still needed later (the open segment and the
//      high-pass history) are copied into the handle's carry buffer.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <atomic>
#include <vector>

#include "vimg_internal.h"

using namespace vimg;

namespace {
constexpr int kProfSlots = 65536;
thread_local std::string g_create_error;

// Event pairs around launches, summed per stage when read.
struct Prof {
  bool on = false;
  cudaEvent_t* ev = nullptr;  // [kProfSlots][2]
  int* stage = nullptr;       // [kProfSlots]
  int used = 0;
  double ms[VIMG_NSTAGES] = {};
  long long launches[VIMG_NSTAGES] = {};
};
}  // namespace

constexpr int kRing = 3;  // frame stages of vimg_process_host

struct vimg_handle {
  int H = 0, W = 0;
  vimg_params p{};
  PatchGrid g{};
  int np = 0, w = 0, nwin = 0;
  int dev = 0;
  cudaStream_t st = nullptr;
  TemplateDev td{};
  bool have_template = false;
  float* tmpl = nullptr;                // [H][W] copy of the template
  // learned proposal
  bool have_proposal = false;
  float* cnn_p = nullptr;               // FP32 parameters
  __nv_bfloat16* cnn_b = nullptr;       // BF16 copy used for inference
  float* cnn_acts = nullptr;            // [cnn_act_floats(max_chunk)]
  float* prop = nullptr;                // [max_chunk][2] network output
  unsigned long long* csum_n = nullptr; // [max_chunk][49] narrow-window sums
  int* fb_list = nullptr;               // [max_chunk] frames falling back
  int* fb_n = nullptr;                  // [1]
  long long* fb_total = nullptr;        // [1] fallbacks since creation
  long long prop_frames = 0;
  // BF16 tensor-core correlation
  float* tround = nullptr;              // [H][W] rounded template
  __nv_bfloat16* as = nullptr;          // per-patch Toeplitz template stores
  float* bgc = nullptr;                 // [np][w*w] background correlation
  __nv_bfloat16* fc = nullptr;          // [max_chunk][H][Wp] frame - rounded template
  float* num = nullptr;                 // [max_chunk][np][w*w] per-patch numerators
  alignas(64) unsigned char tmap[128];  // tensor map over fc
  int* dev_err = nullptr;               // device-side wait timeouts (sticky)
  float gw[2 * kGaussMaxRadius + 1] = {};
  float* inv = nullptr;                 // [max_chunk][stats map] 1/sqrt(SF) per window
  unsigned long long* csum = nullptr;   // [max_chunk][nwin]
  float* shift_tmp = nullptr;           // [max_chunk][2]
  uint16_t* carry[2] = {nullptr, nullptr};
  float* carry_shift[2] = {nullptr, nullptr};
  int carry_cap = 0, carry_n = 0, carry_cur = 0;
  long long frames_seen = 0;
  // host-buffer path
  // vimg_process_host: a ring of kRing frame stages (uploads run up to kRing - 1
  // batches ahead of the compute), two output stages downloaded on their own stream
  uint16_t* stage[kRing] = {};
  float* stage_shift[2] = {};    // [max_chunk][2]
  float* stage_summary[2] = {};  // [max segments per batch][2][H][W]
  cudaStream_t copy_st = nullptr, dl_st = nullptr;
  cudaEvent_t ev_copied[kRing] = {};
  cudaEvent_t ev_used[kRing] = {};
  cudaEvent_t ev_out[2] = {};   // a batch's outputs are complete in the output stage
  cudaEvent_t ev_dl[2] = {};    // the output stage has been downloaded
  Prof prof;
  int sticky = 0;
  std::string err;
  long long id = 0;                     // unique per handle (graph cache keys)
  // voltage-trace ROIs
  int n_rois = 0;
  unsigned long long* roi_members = nullptr;  // [H][W] ids + 1, four 16-bit fields
  int* roi_count = nullptr;                   // [n_rois] pixels per ROI
  unsigned long long* roi_acc = nullptr;      // [max_chunk][n_rois] 2^-20 fixed-point sums
  int* roi_flag = nullptr;                    // [1] a pixel in more than 4 ROIs
  vimg_unet* unet = nullptr;                  // attached U-Net stage (not owned)
  double* vs_acc = nullptr;                   // [6][H][W] whole-video summary sums
  long long vs_frames = 0;
  // CUDA graphs of vimg_process_batch calls led by this handle
  struct GraphEntry {
    std::vector<long long> key;
    cudaGraphExec_t exec = nullptr;
    std::vector<long long> end_state;  // per video: frames_seen, carry_n, carry_cur
    std::vector<int> segs;
    int ret = 0;
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t cap_st = nullptr;        // private stream the graphs are recorded on
};

static std::atomic<long long> g_next_id{1};

// Records the start of a stage's launch; returns the slot or -1.
static int prof_begin(vimg_handle* h, int stage) {
  Prof& p = h->prof;
  if (!p.on) return -1;
  p.launches[stage]++;
  if (p.used >= kProfSlots) return -1;
  const int s = p.used++;
  p.stage[s] = stage;
  cudaEventRecord(p.ev[2 * s], h->st);
  return s;
}

static void prof_end(vimg_handle* h, int slot) {
  if (slot >= 0) cudaEventRecord(h->prof.ev[2 * slot + 1], h->st);
}

static int fail(vimg_handle* h, int code, const std::string& msg) {
  if (h) {
    h->err = msg;
    if (code == VIMG_ERR_CUDA || code == VIMG_ERR_TIMEOUT) h->sticky = code;
  } else {
    g_create_error = msg;
  }
  return code;
}

static int cuda_fail(vimg_handle* h, cudaError_t e, const char* what) {
  return fail(h, VIMG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                               \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
  } while (0)

extern "C" void vimg_default_params(vimg_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->search_radius = 16;
  p->patch = kPatch;
  p->segment_len = 50;
  p->gauss_sigma = 3.0f;
  p->hp_window = 0;
  p->flags = 0;
  p->fallback_zncc = 0.5f;
  p->narrow_radius = 2;
  p->stream = nullptr;
  p->timeout_spins = 1LL << 26;
  p->max_chunk = 200;
}

extern "C" const char* vimg_version(void) { return "vimg 0.1 (sm_103a)"; }

static bool grid_for(int H, int W, int R, PatchGrid* g) {
  if (H - 2 * R < kPatch || W - 2 * R < kPatch) return false;
  g->ny = (H - 2 * R) / kPatch;
  g->nx = (W - 2 * R) / kPatch;
  g->y0 = R + ((H - 2 * R) - g->ny * kPatch) / 2;
  g->x0 = R + ((W - 2 * R) - g->nx * kPatch) / 2;
  return true;
}

static void free_all(vimg_handle* h) {
  void* ptrs[] = {h->td.tc, h->td.tn2, h->td.coff, h->inv, h->csum, h->shift_tmp,
                  h->carry[0], h->carry[1], h->carry_shift[0], h->carry_shift[1],
                  h->stage[0], h->stage[1], h->stage[2], h->stage_shift[0], h->stage_shift[1],
                  h->stage_summary[0], h->stage_summary[1], h->tmpl,
                  h->cnn_p, h->cnn_b, h->cnn_acts, h->prop, h->csum_n, h->fb_list, h->fb_n,
                  h->fb_total, h->tround, h->as, h->bgc, h->fc, h->dev_err, h->num,
                  h->roi_members, h->roi_count, h->roi_acc, h->roi_flag, h->vs_acc};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (int i = 0; i < kRing; ++i) {
    if (h->ev_copied[i]) cudaEventDestroy(h->ev_copied[i]);
    if (h->ev_used[i]) cudaEventDestroy(h->ev_used[i]);
  }
  for (int i = 0; i < 2; ++i) {
    if (h->ev_out[i]) cudaEventDestroy(h->ev_out[i]);
    if (h->ev_dl[i]) cudaEventDestroy(h->ev_dl[i]);
  }
  if (h->copy_st) cudaStreamDestroy(h->copy_st);
  if (h->dl_st) cudaStreamDestroy(h->dl_st);
  for (auto& ge : h->graphs)
    if (ge.exec) cudaGraphExecDestroy(ge.exec);
  h->graphs.clear();
  if (h->cap_st) cudaStreamDestroy(h->cap_st);
  if (h->prof.ev) {
    for (int i = 0; i < 2 * kProfSlots; ++i)
      if (h->prof.ev[i]) cudaEventDestroy(h->prof.ev[i]);
    delete[] h->prof.ev;
    delete[] h->prof.stage;
  }
}

extern "C" vimg_handle* vimg_create(int H, int W, const vimg_params* pin) {
  vimg_params p;
  if (pin)
    p = *pin;
  else
    vimg_default_params(&p);
  if (H <= 0 || W <= 0 || H > 8192 || W > 8192) {
    fail(nullptr, VIMG_ERR_SIZE, "H and W must be in 1..8192");
    return nullptr;
  }
  if (p.search_radius < 0 || p.search_radius > kMaxR) {
    fail(nullptr, VIMG_ERR_ARG, "search_radius must be in 0..16");
    return nullptr;
  }
  if (p.patch != kPatch) {
    fail(nullptr, VIMG_ERR_ARG, "patch must be 21");
    return nullptr;
  }
  if (p.segment_len < 1 || p.segment_len > kMaxL) {
    fail(nullptr, VIMG_ERR_ARG, "segment_len must be in 1..50");
    return nullptr;
  }
  if (!(p.gauss_sigma > 0.f) || (int)std::ceil(4.0 * p.gauss_sigma) > kGaussMaxRadius) {
    fail(nullptr, VIMG_ERR_ARG, "gauss_sigma must be in (0, 3] (radius ceil(4 sigma) <= 12)");
    return nullptr;
  }
  if (p.hp_window < 0 || p.hp_window > kMaxHp) {
    fail(nullptr, VIMG_ERR_ARG, "hp_window must be in 0..64");
    return nullptr;
  }
  if (p.max_chunk < 1 || p.max_chunk > 4096) {
    fail(nullptr, VIMG_ERR_ARG, "max_chunk must be in 1..4096");
    return nullptr;
  }
  if (!corr_group_valid(p.corr_group)) {
    fail(nullptr, VIMG_ERR_ARG, "corr_group must be 0, 7, 8, 10 or 11");
    return nullptr;
  }
  if (p.flags & ~(VIMG_CORR_BF16 | VIMG_PROPOSAL_CNN | VIMG_OUT_HIGHPASS | VIMG_VIDEO_SUMMARY |
                  VIMG_TEMPORAL_SMEM)) {
    fail(nullptr, VIMG_ERR_ARG, "unknown flag bits");
    return nullptr;
  }
  if ((p.flags & VIMG_CORR_BF16) && (p.flags & VIMG_PROPOSAL_CNN)) {
    fail(nullptr, VIMG_ERR_ARG, "VIMG_CORR_BF16 and VIMG_PROPOSAL_CNN cannot be combined");
    return nullptr;
  }
  if ((p.flags & VIMG_CORR_BF16) && p.search_radius != kMaxR) {
    fail(nullptr, VIMG_ERR_ARG, "VIMG_CORR_BF16 needs search_radius 16");
    return nullptr;
  }
  if ((p.flags & VIMG_PROPOSAL_CNN) &&
      (H < kCrop || W < kCrop || p.search_radius < kNarrowWin / 2 + 1 || !(p.fallback_zncc <= 1.f))) {
    fail(nullptr, VIMG_ERR_ARG,
         "VIMG_PROPOSAL_CNN needs H, W >= 128, search_radius >= 4 and fallback_zncc <= 1");
    return nullptr;
  }
  PatchGrid g;
  if (!grid_for(H, W, p.search_radius, &g) || H <= kGaussMaxRadius || W <= kGaussMaxRadius) {
    fail(nullptr, VIMG_ERR_SIZE, "H and W must be at least 2*search_radius + 21");
    return nullptr;
  }
  vimg_handle* h = new vimg_handle();
  h->id = g_next_id++;
  h->H = H, h->W = W, h->p = p, h->g = g;
  h->np = g.ny * g.nx;
  h->w = 2 * p.search_radius + 1;
  h->nwin = h->w * h->w;
  h->st = (cudaStream_t)p.stream;
  // Gaussian taps (Eq. 2): exp(-k^2 / (2 sigma^2)) normalised, zero beyond ceil(4 sigma).
  {
    const int r = (int)std::ceil(4.0 * p.gauss_sigma);
    double wsum = 0.0, wd[2 * kGaussMaxRadius + 1] = {};
    for (int k = -r; k <= r; ++k)
      wsum += (wd[k + kGaussMaxRadius] = std::exp(-(double)k * k / (2.0 * p.gauss_sigma * p.gauss_sigma)));
    for (int k = 0; k < 2 * kGaussMaxRadius + 1; ++k) h->gw[k] = (float)(wd[k] / wsum);
  }
  const size_t HW = (size_t)H * W;
  h->carry_cap = std::max(p.segment_len - 1, p.hp_window > 0 ? p.hp_window - 1 : 0);
  cudaError_t e = cudaGetDevice(&h->dev);
  if (e == cudaSuccess) e = kernels_init();
#define ALLOC(ptr, bytes)                                                   \
  if (e == cudaSuccess && (bytes) > 0) e = cudaMalloc((void**)&(ptr), (bytes));
  ALLOC(h->td.tc, sizeof(float) * h->np * kPatch * kTplStride);
  ALLOC(h->td.tn2, sizeof(float) * h->np);
  ALLOC(h->td.coff, sizeof(int) * h->np);
  ALLOC(h->inv, sizeof(float) * (size_t)p.max_chunk * stats_map_floats(g, p.search_radius));
  ALLOC(h->csum, sizeof(unsigned long long) * (size_t)p.max_chunk * h->nwin);
  ALLOC(h->shift_tmp, sizeof(float) * 2 * (size_t)p.max_chunk);
  for (int i = 0; i < 2; ++i) {
    ALLOC(h->carry[i], sizeof(uint16_t) * HW * std::max(1, h->carry_cap));
    ALLOC(h->carry_shift[i], sizeof(float) * 2 * std::max(1, h->carry_cap));
  }
  ALLOC(h->tmpl, sizeof(float) * HW);
  ALLOC(h->dev_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->dev_err, 0, sizeof(int));
  if (p.flags & VIMG_CORR_BF16) {
    ALLOC(h->tround, sizeof(float) * HW);
    ALLOC(h->as, bf16_astore_bytes(g));
    ALLOC(h->bgc, sizeof(float) * h->np * h->nwin);
    ALLOC(h->fc, sizeof(__nv_bfloat16) * bf16_fc_elems(p.max_chunk, H, W));
    ALLOC(h->num, sizeof(float) * (size_t)p.max_chunk * h->np * h->nwin);
    if (e == cudaSuccess && bf16_tensor_map(h->tmap, h->fc, p.max_chunk, H, W) != 0)
      e = cudaErrorNotSupported;
  }
  if (p.flags & VIMG_VIDEO_SUMMARY) {
    ALLOC(h->vs_acc, sizeof(double) * 6 * HW);
    if (e == cudaSuccess) e = cudaMemset(h->vs_acc, 0, sizeof(double) * 6 * HW);
  }
  if (p.flags & VIMG_PROPOSAL_CNN) {
    ALLOC(h->cnn_p, sizeof(float) * cnn_param_count());
    ALLOC(h->cnn_b, sizeof(__nv_bfloat16) * cnn_param_count());
    ALLOC(h->cnn_acts, sizeof(float) * cnn_act_floats(p.max_chunk));
    ALLOC(h->prop, sizeof(float) * 2 * (size_t)p.max_chunk);
    ALLOC(h->csum_n, sizeof(unsigned long long) * kNarrowWin * kNarrowWin * (size_t)p.max_chunk);
    ALLOC(h->fb_list, sizeof(int) * (size_t)p.max_chunk);
    ALLOC(h->fb_n, sizeof(int));
    ALLOC(h->fb_total, sizeof(long long));
    if (e == cudaSuccess) e = cudaMemset(h->fb_total, 0, sizeof(long long));
  }
#undef ALLOC
  if (e != cudaSuccess) {
    fail(nullptr, e == cudaErrorMemoryAllocation ? VIMG_ERR_OOM : VIMG_ERR_CUDA,
         std::string("workspace allocation failed: ") + cudaGetErrorString(e));
    free_all(h);
    delete h;
    return nullptr;
  }
  return h;
}

extern "C" void vimg_destroy(vimg_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  if (h->copy_st) cudaStreamSynchronize(h->copy_st);
  if (h->dl_st) cudaStreamSynchronize(h->dl_st);
  free_all(h);
  delete h;
}

extern "C" const char* vimg_last_error(const vimg_handle* h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

extern "C" long long vimg_frames_seen(const vimg_handle* h) { return h ? h->frames_seen : -1; }

// Stream-state blob: this header, then the open segment's frames [carry_n][H][W]
// (uint16) and shifts [carry_n][2] (float), then the whole-video sums [6][H][W]
// (double) when the handle keeps them.
struct StateHeader {
  uint32_t magic, version;
  int H, W, segment_len, hp_window, search_radius, flags;
  long long frames_seen, vs_frames, prop_frames, fb_total;
  int carry_n, has_vs;
};
constexpr uint32_t kStateMagic = 0x534d4956u;  // "VIMS"

static long long state_size(const vimg_handle* h, int carry_n) {
  const long long HW = (long long)h->H * h->W;
  return (long long)sizeof(StateHeader) + carry_n * HW * 2 + carry_n * 2LL * 4 +
         (h->vs_acc ? 6 * HW * 8 : 0);
}

extern "C" long long vimg_state_bytes(const vimg_handle* h) {
  if (!h) return VIMG_ERR_ARG;
  return state_size(h, h->carry_n);
}

extern "C" int vimg_get_state(vimg_handle* h, void* host, long long bytes) {
  if (!h) return fail(h, VIMG_ERR_ARG, "null handle");
  if (h->sticky) return h->sticky;
  if (!host || bytes < state_size(h, h->carry_n))
    return fail(h, VIMG_ERR_ARG, "vimg_get_state: buffer smaller than vimg_state_bytes");
  CK(cudaStreamSynchronize(h->st), "stream sync");
  if (h->copy_st) CK(cudaStreamSynchronize(h->copy_st), "stream sync");
  if (h->dl_st) CK(cudaStreamSynchronize(h->dl_st), "stream sync");
  StateHeader hd{};
  hd.magic = kStateMagic, hd.version = 1;
  hd.H = h->H, hd.W = h->W, hd.segment_len = h->p.segment_len, hd.hp_window = h->p.hp_window;
  hd.search_radius = h->p.search_radius, hd.flags = h->p.flags;
  hd.frames_seen = h->frames_seen, hd.vs_frames = h->vs_frames, hd.prop_frames = h->prop_frames;
  hd.carry_n = h->carry_n, hd.has_vs = h->vs_acc ? 1 : 0;
  if (h->fb_total)
    CK(cudaMemcpy(&hd.fb_total, h->fb_total, sizeof(long long), cudaMemcpyDeviceToHost),
       "state copy");
  unsigned char* o = static_cast<unsigned char*>(host);
  std::memcpy(o, &hd, sizeof(hd));
  o += sizeof(hd);
  const size_t HW = (size_t)h->H * h->W;
  if (h->carry_n > 0) {
    CK(cudaMemcpy(o, h->carry[h->carry_cur], sizeof(uint16_t) * HW * h->carry_n,
                  cudaMemcpyDeviceToHost),
       "state copy");
    o += sizeof(uint16_t) * HW * h->carry_n;
    CK(cudaMemcpy(o, h->carry_shift[h->carry_cur], sizeof(float) * 2 * h->carry_n,
                  cudaMemcpyDeviceToHost),
       "state copy");
    o += sizeof(float) * 2 * h->carry_n;
  }
  if (h->vs_acc)
    CK(cudaMemcpy(o, h->vs_acc, sizeof(double) * 6 * HW, cudaMemcpyDeviceToHost), "state copy");
  return VIMG_OK;
}

extern "C" int vimg_set_state(vimg_handle* h, const void* host, long long bytes) {
  if (!h) return fail(h, VIMG_ERR_ARG, "null handle");
  if (h->sticky) return h->sticky;
  StateHeader hd{};
  if (!host || bytes < (long long)sizeof(hd))
    return fail(h, VIMG_ERR_ARG, "vimg_set_state: no state header");
  std::memcpy(&hd, host, sizeof(hd));
  if (hd.magic != kStateMagic || hd.version != 1)
    return fail(h, VIMG_ERR_ARG, "vimg_set_state: not a state written by vimg_get_state");
  if (hd.H != h->H || hd.W != h->W || hd.segment_len != h->p.segment_len ||
      hd.hp_window != h->p.hp_window || hd.search_radius != h->p.search_radius ||
      hd.flags != h->p.flags || hd.has_vs != (h->vs_acc ? 1 : 0))
    return fail(h, VIMG_ERR_ARG, "vimg_set_state: state of a handle with other parameters");
  if (hd.carry_n < 0 || hd.carry_n > h->carry_cap || hd.frames_seen < hd.carry_n ||
      bytes < state_size(h, hd.carry_n))
    return fail(h, VIMG_ERR_ARG, "vimg_set_state: inconsistent or truncated state");
  CK(cudaStreamSynchronize(h->st), "stream sync");
  if (h->copy_st) CK(cudaStreamSynchronize(h->copy_st), "stream sync");
  if (h->dl_st) CK(cudaStreamSynchronize(h->dl_st), "stream sync");
  const unsigned char* in = static_cast<const unsigned char*>(host) + sizeof(hd);
  const size_t HW = (size_t)h->H * h->W;
  if (hd.carry_n > 0) {
    CK(cudaMemcpy(h->carry[0], in, sizeof(uint16_t) * HW * hd.carry_n, cudaMemcpyHostToDevice),
       "state copy");
    in += sizeof(uint16_t) * HW * hd.carry_n;
    CK(cudaMemcpy(h->carry_shift[0], in, sizeof(float) * 2 * hd.carry_n, cudaMemcpyHostToDevice),
       "state copy");
    in += sizeof(float) * 2 * hd.carry_n;
  }
  if (h->vs_acc)
    CK(cudaMemcpy(h->vs_acc, in, sizeof(double) * 6 * HW, cudaMemcpyHostToDevice), "state copy");
  if (h->fb_total)
    CK(cudaMemcpy(h->fb_total, &hd.fb_total, sizeof(long long), cudaMemcpyHostToDevice),
       "state copy");
  h->carry_cur = 0;
  h->carry_n = hd.carry_n;
  h->frames_seen = hd.frames_seen;
  h->vs_frames = hd.vs_frames;
  h->prop_frames = hd.prop_frames;
  return VIMG_OK;
}

extern "C" int vimg_reset(vimg_handle* h) {
  if (!h) return fail(h, VIMG_ERR_ARG, "null handle");
  if (h->sticky) return h->sticky;
  h->frames_seen = 0;
  h->carry_n = 0;
  if (h->vs_acc) {
    CK(cudaMemsetAsync(h->vs_acc, 0, sizeof(double) * 6 * h->H * h->W, h->st), "summary reset");
    h->vs_frames = 0;
  }
  return VIMG_OK;
}

extern "C" int vimg_seek(vimg_handle* h, long long t_start, const uint16_t* d_history,
                         int n_history) {
  if (!h) return fail(h, VIMG_ERR_ARG, "null handle");
  if (h->sticky) return h->sticky;
  const int L = h->p.segment_len;
  const long long need_ll =
      std::min<long long>(t_start, h->p.hp_window > 0 ? h->p.hp_window - 1 : 0);
  if (t_start < 0 || t_start % L != 0 || n_history < 0 || n_history > t_start ||
      (n_history > 0 && !d_history) || n_history < need_ll)
    return fail(h, VIMG_ERR_ARG,
                "vimg_seek: t_start must be a non-negative multiple of the segment length and "
                "the history must hold the min(t_start, hp_window - 1) frames before it");
  const int need = (int)need_ll;
  if (need > 0 && !h->have_template)
    return fail(h, VIMG_ERR_NO_TEMPLATE, "vimg_set_template must come before vimg_seek");
  if (need > 0 && (h->p.flags & VIMG_PROPOSAL_CNN) && !h->have_proposal)
    return fail(h, VIMG_ERR_ARG, "vimg_load_proposal must come before vimg_seek");
  h->frames_seen = 0;
  h->carry_n = 0;
  if (h->vs_acc) {
    CK(cudaMemsetAsync(h->vs_acc, 0, sizeof(double) * 6 * h->H * h->W, h->st), "summary reset");
    h->vs_frames = 0;
  }
  if (need == 0) {
    h->frames_seen = t_start;
    return VIMG_OK;
  }
  // the last `need` history frames: their shifts are estimated and they enter
  // the carried high-pass history; nothing is output and the whole-video sums
  // do not see them
  h->frames_seen = t_start - need;
  double* vs = h->vs_acc;
  h->vs_acc = nullptr;
  vimg_io io{};
  const size_t HW = (size_t)h->H * h->W;
  const int rc = vimg_process_io(h, d_history + HW * (size_t)(n_history - need), need, &io);
  h->vs_acc = vs;
  if (rc < 0) return rc;
  return h->frames_seen == t_start ? VIMG_OK : fail(h, VIMG_ERR_ARG, "vimg_seek: stream position");
}

extern "C" int vimg_set_template(vimg_handle* h, const float* d_template) {
  if (!h || !d_template) return fail(h, VIMG_ERR_ARG, "null handle or template");
  if (h->sticky) return h->sticky;
  CK(launch_template_prep(d_template, h->H, h->W, h->g, h->td, h->st), "template prep launch");
  CK(cudaMemcpyAsync(h->tmpl, d_template, sizeof(float) * h->H * h->W, cudaMemcpyDeviceToDevice,
                     h->st),
     "template copy");
  if (h->p.flags & VIMG_CORR_BF16)
    CK(bf16_template_prep(d_template, h->H, h->W, h->g, h->p.search_radius, h->td, h->tround,
                          h->as, h->bgc, h->st),
       "tensor-core template prep");
  h->have_template = true;
  return VIMG_OK;
}

extern "C" int vimg_video_summary(vimg_handle* h, float* d_average, float* d_correlation) {
  if (!h) return fail(h, VIMG_ERR_ARG, "null handle");
  if (h->sticky) return h->sticky;
  if (!h->vs_acc) return fail(h, VIMG_ERR_ARG, "vimg_video_summary needs VIMG_VIDEO_SUMMARY");
  if (h->vs_frames < 1) return fail(h, VIMG_ERR_ARG, "vimg_video_summary: no frames yet");
  CK(launch_vsum_final(h->vs_acc, h->tmpl, h->vs_frames, h->H, h->W, d_average, d_correlation,
                       h->st),
     "video summary launch");
  return VIMG_OK;
}

extern "C" int vimg_attach_unet(vimg_handle* h, vimg_unet* u) {
  if (!h) return fail(h, VIMG_ERR_ARG, "null handle");
  if (h->sticky) return h->sticky;
  if (u) {
    int H = 0, W = 0;
    unet_dims(u, &H, &W);
    if (H != h->H || W != h->W) return fail(h, VIMG_ERR_ARG, "vimg_attach_unet: size mismatch");
  }
  h->unet = u;
  return VIMG_OK;
}

extern "C" int vimg_set_rois(vimg_handle* h, const uint8_t* d_masks, int n_rois) {
  if (!h) return fail(h, VIMG_ERR_ARG, "null handle");
  if (h->sticky) return h->sticky;
  if (n_rois < 0 || n_rois > 65535 || (n_rois > 0 && !d_masks))
    return fail(h, VIMG_ERR_ARG, "vimg_set_rois: n_rois must be in 0..65535 with a mask array");
  if (n_rois == 0) {
    h->n_rois = 0;
    return VIMG_OK;
  }
  const size_t HW = (size_t)h->H * h->W;
  unsigned long long *mem = nullptr, *acc = nullptr;
  int *cnt = nullptr, *flag = nullptr;
  auto drop = [&]() {
    if (mem) cudaFree(mem);
    if (acc) cudaFree(acc);
    if (cnt) cudaFree(cnt);
    if (flag) cudaFree(flag);
  };
  cudaError_t e = cudaMalloc((void**)&mem, sizeof(unsigned long long) * HW);
  if (e == cudaSuccess) e = cudaMalloc((void**)&cnt, sizeof(int) * (size_t)n_rois);
  if (e == cudaSuccess)
    e = cudaMalloc((void**)&acc, sizeof(unsigned long long) * (size_t)h->p.max_chunk * n_rois);
  if (e == cudaSuccess) e = cudaMalloc((void**)&flag, sizeof(int));
  if (e == cudaSuccess) e = roi_build(d_masks, n_rois, h->H, h->W, mem, cnt, flag, h->st);
  int too_many = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&too_many, flag, sizeof(int), cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) {
    drop();
    return cuda_fail(h, e, "vimg_set_rois");
  }
  if (too_many) {
    drop();
    return fail(h, VIMG_ERR_ARG, "vimg_set_rois: a pixel lies in more than 4 ROIs");
  }
  for (void* q : {(void*)h->roi_members, (void*)h->roi_count, (void*)h->roi_acc, (void*)h->roi_flag})
    if (q) cudaFree(q);
  h->roi_members = mem, h->roi_count = cnt, h->roi_acc = acc, h->roi_flag = flag;
  h->n_rois = n_rois;
  return VIMG_OK;
}

// Motion estimate of nf frames (nf <= max_chunk) into shifts[nf][2].
static int estimate(vimg_handle* h, const uint16_t* frames, int nf, float* shifts,
                    float* peak_info, double* surface, float* prop_px) {
  const int R = h->p.search_radius;
  CK(cudaMemsetAsync(h->csum, 0, sizeof(unsigned long long) * (size_t)nf * h->nwin, h->st),
     "surface reset");
  if (h->p.flags & VIMG_PROPOSAL_CNN) {
    // learned proposal -> narrow window -> full window for the listed frames
    int ps = prof_begin(h, 4);
    CK(cnn_input(frames, nf, h->H, h->W, h->tmpl, 0, h->cnn_acts, h->st), "proposal input");
    CK(cnn_forward(h->cnn_p, h->cnn_b, h->cnn_acts, nf, h->prop, h->st), "proposal forward");
    prof_end(h, ps);
    ps = prof_begin(h, 0);
    CK(launch_stats_narrow(frames, nf, h->H, h->W, h->g, R, h->prop, h->inv, h->st),
       "narrow window statistics launch");
    prof_end(h, ps);
    CK(cudaMemsetAsync(h->csum_n, 0, sizeof(unsigned long long) * kNarrowWin * kNarrowWin * nf,
                       h->st),
       "narrow surface reset");
    CK(cudaMemsetAsync(h->fb_n, 0, sizeof(int), h->st), "list reset");
    ps = prof_begin(h, 1);
    CK(launch_corr_narrow(frames, nf, h->H, h->W, h->g, R, h->td, h->inv, h->prop, h->csum_n,
                          h->st),
       "narrow correlation launch");
    prof_end(h, ps);
    ps = prof_begin(h, 2);
    if (surface)  // all-ones bytes: NaN wherever no displacement is evaluated
      CK(cudaMemsetAsync(surface, 0xff, sizeof(double) * (size_t)nf * h->nwin, h->st),
         "surface fill");
    CK(launch_peak_narrow(h->csum_n, nf, R, h->np, h->prop, h->p.fallback_zncc, shifts, peak_info,
                          h->fb_list, h->fb_n, surface, prop_px, h->st),
       "narrow peak launch");
    prof_end(h, ps);
    ps = prof_begin(h, 0);
    CK(launch_stats(frames, nf, h->H, h->W, h->g, R, h->td, h->inv, h->st, h->fb_list, h->fb_n,
                    h->dev_err),
       "fallback window statistics launch");
    prof_end(h, ps);
    ps = prof_begin(h, 1);
    CK(launch_corr_f32(frames, nf, h->H, h->W, h->g, R, h->td, h->inv, h->csum, h->st, h->fb_list,
                       h->fb_n, h->p.corr_group),
       "fallback correlation launch");
    prof_end(h, ps);
    ps = prof_begin(h, 2);
    CK(launch_peak(h->csum, nf, R, h->np, shifts, peak_info, surface, h->st, h->fb_list, h->fb_n),
       "fallback peak launch");
    prof_end(h, ps);
    CK(launch_count_add(h->fb_n, h->fb_total, h->st), "fallback count");
    h->prop_frames += nf;
    return VIMG_OK;
  }
  // One launch per stage for the whole batch: thousands of CTAs, so the last
  // partial wave costs little.
  int ps = prof_begin(h, 0);
  CK(launch_stats(frames, nf, h->H, h->W, h->g, R, h->td, h->inv, h->st, nullptr, nullptr,
                  h->dev_err),
     "window statistics launch");
  prof_end(h, ps);
  ps = prof_begin(h, 1);
  if (h->p.flags & VIMG_CORR_BF16) {
    CK(bf16_make_fc(frames, nf, h->p.max_chunk, h->H, h->W, h->tround, h->fc, h->st),
       "frame offset images");
    CK(launch_corr_bf16(h->tmap, nf, R, h->g, h->as, h->bgc, h->td, h->inv, h->num, h->csum,
                        h->dev_err, h->st),
       "tensor-core correlation launch");
  } else {
    CK(launch_corr_f32(frames, nf, h->H, h->W, h->g, R, h->td, h->inv, h->csum, h->st, nullptr,
                       nullptr, h->p.corr_group),
       "correlation launch");
  }
  prof_end(h, ps);
  ps = prof_begin(h, 2);
  CK(launch_peak(h->csum, nf, R, h->np, shifts, peak_info, surface, h->st), "peak launch");
  prof_end(h, ps);
  return VIMG_OK;
}

// Temporal-pass arguments of one internal batch of n frames (summary: where
// this batch's first completed segment goes).
static TemporalArgs temporal_args(const vimg_handle* h, const uint16_t* frames, int n,
                                  const float* shifts, float* corrected, float* summary) {
  const long long seen = h->frames_seen;
  const int L = h->p.segment_len;
  const int c = (int)(seen % L);
  TemporalArgs a{};
  a.src.carry = h->carry[h->carry_cur];
  a.src.carry_shift = h->carry_shift[h->carry_cur];
  a.src.batch = frames;
  a.src.batch_shift = shifts;
  a.src.n_carry = h->carry_n;
  a.src.n_batch = n;
  a.src.t_first = seen - h->carry_n;
  a.src.t_new = seen;
  a.H = h->H, a.W = h->W, a.L = L, a.hp_w = h->p.hp_window, a.gauss_r = kGaussMaxRadius;
  std::memcpy(a.gw, h->gw, sizeof(a.gw));
  a.seg_base = seen - c;
  a.n_seg = (c + n + L - 1) / L;
  a.out_hp = (h->p.flags & VIMG_OUT_HIGHPASS) ? 1 : 0;
  a.pairs = (h->W % 2 == 0) && ((reinterpret_cast<uintptr_t>(frames) & 3) == 0) &&
            ((reinterpret_cast<uintptr_t>(a.src.carry) & 3) == 0);
  a.corrected = corrected;
  a.summary = summary;
  a.err = h->dev_err;
  a.smem_history = (h->p.flags & VIMG_TEMPORAL_SMEM) ? 1 : 0;
  return a;
}

// After a batch of n frames: keeps the frames (and shifts) that later batches
// still need -- the open segment and the high-pass history -- in the carry
// buffer, and advances the stream state.  Returns the segments completed.
static int advance_state(vimg_handle* h, const uint16_t* frames, const float* shifts, int n,
                         cudaStream_t st) {
  const size_t HW = (size_t)h->H * h->W;
  const int L = h->p.segment_len;
  const long long seen = h->frames_seen;
  const int k = (int)((seen % L + n) / L);
  // New carry: the last K' frames of (carry ++ batch).
  const long long seen2 = seen + n;
  const int c2 = (int)(seen2 % L);
  const int hp_need = h->p.hp_window > 0 ? h->p.hp_window - 1 : 0;
  int K = std::max(c2, hp_need);
  if (K > seen2) K = (int)seen2;
  const int nv = h->carry_n + n, nxt = 1 - h->carry_cur;
  int dst = 0;
  const int pcs = K > 0 && st == h->st ? prof_begin(h, 5) : -1;
  for (int v = nv - K; v < nv;) {
    const bool in_carry = v < h->carry_n;
    const int run = in_carry ? std::min(h->carry_n - v, nv - v) : nv - v;
    const uint16_t* sf = in_carry ? h->carry[h->carry_cur] + HW * v : frames + HW * (v - h->carry_n);
    const float* ss = in_carry ? h->carry_shift[h->carry_cur] + 2 * v : shifts + 2 * (v - h->carry_n);
    CK(cudaMemcpyAsync(h->carry[nxt] + HW * dst, sf, sizeof(uint16_t) * HW * run,
                       cudaMemcpyDeviceToDevice, st),
       "carry copy");
    CK(cudaMemcpyAsync(h->carry_shift[nxt] + 2 * dst, ss, sizeof(float) * 2 * run,
                       cudaMemcpyDeviceToDevice, st),
       "carry shift copy");
    dst += run;
    v += run;
  }
  prof_end(h, pcs);
  h->carry_cur = nxt;
  h->carry_n = K;
  h->frames_seen = seen2;
  return k;
}

// One internal batch: n <= max_chunk frames.
static int process_batch(vimg_handle* h, const uint16_t* frames, int n, const vimg_io& io,
                         int k_before) {
  const size_t HW = (size_t)h->H * h->W;
  const float* shifts;
  if (io.shifts_in) {
    shifts = io.shifts_in;
  } else {
    float* out = io.shifts ? io.shifts : h->shift_tmp;
    int rc = estimate(h, frames, n, out, io.peak_info, io.surface, io.proposal);
    if (rc) return rc;
    shifts = out;
  }
  TemporalArgs a = temporal_args(h, frames, n, shifts, io.corrected,
                                 io.summary ? io.summary + (size_t)k_before * 2 * HW : nullptr);
  const bool traces = io.traces && h->n_rois > 0;
  if (traces) {
    CK(cudaMemsetAsync(h->roi_acc, 0, sizeof(unsigned long long) * (size_t)n * h->n_rois, h->st),
       "trace reset");
    a.roi_members = h->roi_members;
    a.roi_acc = h->roi_acc;
    a.n_rois = h->n_rois;
  }
  if (io.corrected || io.summary || traces) {
    const int ps = prof_begin(h, 3);
    CK(launch_temporal(a, h->st), "temporal launch");
    prof_end(h, ps);
  }
  if (traces || h->vs_acc) {
    const int ps = prof_begin(h, 6);
    if (traces)
      CK(roi_finalize(h->roi_acc, h->roi_count, n, h->n_rois, io.traces, h->st), "trace launch");
    if (h->vs_acc) {
      CK(launch_vsum(frames, shifts, n, h->H, h->W, h->tmpl, h->vs_acc, h->st),
         "video summary launch");
      h->vs_frames += n;
    }
    prof_end(h, ps);
  }
  const int k = advance_state(h, frames, shifts, n, h->st);
  if (k > 0 && io.prob) {
    const int rc = vimg_unet_run_on(h->unet, io.summary + (size_t)k_before * 2 * HW, k,
                                    io.prob + (size_t)k_before * HW, h->st);
    if (rc < 0) return fail(h, rc, std::string("U-Net: ") + vimg_unet_last_error(h->unet));
  }
  return k;
}

extern "C" int vimg_process_io(vimg_handle* h, const uint16_t* d_frames, int n, const vimg_io* io) {
  if (!h) return fail(h, VIMG_ERR_ARG, "null handle");
  if (h->sticky) return h->sticky;
  if (n < 0 || (n > 0 && !d_frames) || !io) return fail(h, VIMG_ERR_ARG, "bad frames or io");
  if (!io->shifts_in && !h->have_template)
    return fail(h, VIMG_ERR_NO_TEMPLATE, "vimg_set_template must come before vimg_process");
  if (!io->shifts_in && (h->p.flags & VIMG_PROPOSAL_CNN) && !h->have_proposal)
    return fail(h, VIMG_ERR_ARG, "vimg_load_proposal must come before vimg_process");
  if (io->prob && (!io->summary || !h->unet))
    return fail(h, VIMG_ERR_ARG, "vimg_io.prob needs summary output and an attached U-Net");
  const size_t HW = (size_t)h->H * h->W;
  const int L = h->p.segment_len, maxc = h->p.max_chunk;
  int done = 0, k_total = 0;
  while (done < n) {
    int m = std::min(n - done, maxc);
    if (m < n - done) {
      const int cut = (int)((h->frames_seen + m) % L);
      if (m - cut > 0) m -= cut;  // end the batch on a segment boundary
    }
    vimg_io sub = *io;
    if (io->shifts) sub.shifts = io->shifts + 2 * (size_t)done;
    if (io->shifts_in) sub.shifts_in = io->shifts_in + 2 * (size_t)done;
    if (io->corrected) sub.corrected = io->corrected + HW * done;
    if (io->peak_info) sub.peak_info = io->peak_info + 4 * (size_t)done;
    if (io->surface) sub.surface = io->surface + (size_t)h->nwin * done;
    if (io->proposal) sub.proposal = io->proposal + 2 * (size_t)done;
    if (io->traces) sub.traces = io->traces + (size_t)h->n_rois * done;
    int k = process_batch(h, d_frames + HW * done, m, sub, k_total);
    if (k < 0) return k;
    k_total += k;
    done += m;
  }
  return k_total;
}

extern "C" int vimg_process(vimg_handle* h, const uint16_t* d_frames, int n, float* d_shifts_out,
                            float* d_corrected_out, float* d_summary_out) {
  vimg_io io{};
  io.shifts = d_shifts_out;
  io.corrected = d_corrected_out;
  io.summary = d_summary_out;
  return vimg_process_io(h, d_frames, n, &io);
}

// ---- several videos per call ---------------------------------------------------
namespace {
constexpr int kMaxBatchVideos = 64;
constexpr size_t kMaxGraphs = 4;

struct BatchCall {
  vimg_handle* const* hs;
  int k;
  const uint16_t* const* frames;
  const int* ns;
  float* const* shifts;
  float* const* corrected;
  float* const* summary;
  int ring;
  std::vector<int> chunk;  // per video
};

template <class T>
T* entry(T* const* arr, int v) {
  return arr ? arr[v] : nullptr;
}
}  // namespace

// Enqueues the whole call on st: per step, one launch per kernel for up to
// kMaxVideos videos.  Returns the total segment count; segs[v] gets k_v.
static int batch_body(const BatchCall& c, cudaStream_t st, std::vector<int>& segs) {
  vimg_handle* h = c.hs[0];  // error messages go to the lead handle
  const int k = c.k;
  std::vector<int> done(k, 0);
  segs.assign(k, 0);
  int total = 0;
  for (int s = 0;; ++s) {
    std::vector<int> act, m(k, 0);
    for (int v = 0; v < k; ++v) {
      const int left = c.ns[v] - done[v];
      if (left <= 0) continue;
      const vimg_handle* hv = c.hs[v];
      int mv = std::min(left, c.chunk[v]);
      if (mv < left) {
        const int cut = (int)((hv->frames_seen + mv) % hv->p.segment_len);
        if (mv - cut > 0) mv -= cut;  // end the step on a segment boundary
      }
      m[v] = mv;
      act.push_back(v);
    }
    if (act.empty()) break;
    for (size_t g0 = 0; g0 < act.size(); g0 += kMaxVideos) {
      const int gn = (int)std::min<size_t>(kMaxVideos, act.size() - g0);
      MotionBatch mb{};
      mb.n = gn;
      float* sh_out[kMaxVideos];
      const uint16_t* fr[kMaxVideos];
      for (int i = 0; i < gn; ++i) {
        const int v = act[g0 + i];
        vimg_handle* hv = c.hs[v];
        const size_t HW = (size_t)hv->H * hv->W;
        float* so = entry(c.shifts, v);
        sh_out[i] = so ? so + 2 * (size_t)done[v] : hv->shift_tmp;
        fr[i] = c.frames[v] + HW * done[v];
        MotionJob& J = mb.j[i];
        J.frames = fr[i], J.nf = m[v], J.H = hv->H, J.W = hv->W, J.g = hv->g;
        J.R = hv->p.search_radius;
        J.tc = hv->td.tc, J.tn2 = hv->td.tn2, J.coff = hv->td.coff;
        J.isf = hv->inv, J.csum = hv->csum, J.shifts = sh_out[i], J.err = hv->dev_err;
        J.cg = hv->p.corr_group;
        CK(cudaMemsetAsync(hv->csum, 0, sizeof(unsigned long long) * (size_t)m[v] * hv->nwin, st),
           "surface reset");
      }
      if (!motion_batch_finalize(mb)) return fail(h, VIMG_ERR_ARG, "batch too large");
      CK(launch_stats_multi(mb, st), "batched window statistics launch");
      CK(launch_corr_f32_multi(mb, st), "batched correlation launch");
      CK(launch_peak_multi(mb, st), "batched peak launch");
      TemporalBatch tb{};
      for (int i = 0; i < gn; ++i) {
        const int v = act[g0 + i];
        vimg_handle* hv = c.hs[v];
        const size_t HW = (size_t)hv->H * hv->W;
        float* co = entry(c.corrected, v);
        float* su = entry(c.summary, v);
        if (!co && !su) continue;
        if (co)
          co += HW * (c.ring > 0 ? (size_t)(s % c.ring) * c.chunk[v] : (size_t)done[v]);
        if (su) su += (size_t)segs[v] * 2 * HW;
        tb.a[tb.n++] = temporal_args(hv, fr[i], m[v], sh_out[i], co, su);
      }
      if (tb.n > 0) {
        if (!temporal_batch_finalize(tb)) return fail(h, VIMG_ERR_ARG, "batch too large");
        CK(launch_temporal_multi(tb, st), "batched temporal launch");
      }
      for (int i = 0; i < gn; ++i) {
        const int v = act[g0 + i];
        const int kk = advance_state(c.hs[v], fr[i], sh_out[i], m[v], st);
        if (kk < 0) {
          if (c.hs[v] != h) fail(h, kk, c.hs[v]->err);
          return kk;
        }
        segs[v] += kk;
        total += kk;
        done[v] += m[v];
      }
    }
  }
  return total;
}

extern "C" int vimg_process_batch(vimg_handle* const* hs, int k, const uint16_t* const* d_frames,
                                  const int* ns, float* const* d_shifts_out,
                                  float* const* d_corrected_out, float* const* d_summary_out,
                                  int* segments_out, const vimg_batch_opts* opts) {
  if (!hs || k < 1 || k > kMaxBatchVideos || !d_frames || !ns)
    return fail(hs && k >= 1 ? hs[0] : nullptr, VIMG_ERR_ARG,
                "vimg_process_batch: need 1..64 handles, frame pointers and counts");
  vimg_handle* h = hs[0];
  if (!h) return fail(nullptr, VIMG_ERR_ARG, "vimg_process_batch: null handle");
  vimg_batch_opts o{};
  if (opts) o = *opts;
  if (o.chunk < 0 || o.ring_chunks < 0 || o.reserved != 0)
    return fail(h, VIMG_ERR_ARG, "vimg_process_batch: bad options");
  BatchCall c{hs, k, d_frames, ns, d_shifts_out, d_corrected_out, d_summary_out, o.ring_chunks, {}};
  for (int v = 0; v < k; ++v) {
    vimg_handle* hv = hs[v];
    if (!hv) return fail(h, VIMG_ERR_ARG, "vimg_process_batch: null handle");
    for (int u = 0; u < v; ++u)
      if (hs[u] == hv) return fail(h, VIMG_ERR_ARG, "vimg_process_batch: repeated handle");
    if (hv->sticky) {
      h->err = "vimg_process_batch: a handle is in an error state: " + hv->err;
      return hv->sticky;
    }
    if (hv->dev != h->dev) return fail(h, VIMG_ERR_ARG, "vimg_process_batch: handles on different devices");
    if (hv->p.flags & (VIMG_CORR_BF16 | VIMG_PROPOSAL_CNN | VIMG_VIDEO_SUMMARY))
      return fail(h, VIMG_ERR_ARG,
                  "vimg_process_batch: handles must run the full-window FP32 method "
                  "without whole-video summaries");
    if (!hv->have_template)
      return fail(h, VIMG_ERR_NO_TEMPLATE, "vimg_process_batch: a handle has no template");
    if (ns[v] < 0 || (ns[v] > 0 && !d_frames[v]))
      return fail(h, VIMG_ERR_ARG, "vimg_process_batch: bad frame count or pointer");
    if (o.chunk > hv->p.max_chunk)
      return fail(h, VIMG_ERR_ARG, "vimg_process_batch: chunk exceeds a handle's max_chunk");
    c.chunk.push_back(o.chunk > 0 ? o.chunk : hv->p.max_chunk);
  }
  cudaStream_t st = h->st;
  // Order the other handles' streams before this call.
  struct EventGuard {
    cudaEvent_t e = nullptr;
    ~EventGuard() {
      if (e) cudaEventDestroy(e);
    }
  } guard;
  cudaEvent_t& ev = guard.e;
  bool other = false;
  for (int v = 1; v < k; ++v) other = other || hs[v]->st != st;
  if (other) {
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event create");
    for (int v = 1; v < k; ++v)
      if (hs[v]->st != st) {
        CK(cudaEventRecord(ev, hs[v]->st), "event record");
        CK(cudaStreamWaitEvent(st, ev, 0), "stream wait");
      }
  }
  std::vector<int> segs;
  int ret = 0;
  if (!o.use_graph) {
    ret = batch_body(c, st, segs);
  } else {
    // key: handles and their stream state, pointers, sizes, options
    std::vector<long long> key = {k, o.chunk, o.ring_chunks};
    for (int v = 0; v < k; ++v) {
      const vimg_handle* hv = hs[v];
      key.insert(key.end(), {hv->id, hv->frames_seen, hv->carry_n, hv->carry_cur, ns[v],
                             (long long)(uintptr_t)d_frames[v],
                             (long long)(uintptr_t)entry(d_shifts_out, v),
                             (long long)(uintptr_t)entry(d_corrected_out, v),
                             (long long)(uintptr_t)entry(d_summary_out, v)});
    }
    vimg_handle::GraphEntry* hit = nullptr;
    for (auto& ge : h->graphs)
      if (ge.key == key) hit = &ge;
    if (hit) {
      CK(cudaGraphLaunch(hit->exec, st), "graph launch");
      for (int v = 0; v < k; ++v) {
        hs[v]->frames_seen = hit->end_state[3 * v];
        hs[v]->carry_n = (int)hit->end_state[3 * v + 1];
        hs[v]->carry_cur = (int)hit->end_state[3 * v + 2];
      }
      segs = hit->segs;
      ret = hit->ret;
    } else {
      std::vector<long long> saved;
      for (int v = 0; v < k; ++v)
        saved.insert(saved.end(), {hs[v]->frames_seen, hs[v]->carry_n, hs[v]->carry_cur});
      auto restore = [&]() {
        for (int v = 0; v < k; ++v) {
          hs[v]->frames_seen = saved[3 * v];
          hs[v]->carry_n = (int)saved[3 * v + 1];
          hs[v]->carry_cur = (int)saved[3 * v + 2];
        }
      };
      // Recorded on a private stream (the legacy default stream cannot be
      // captured), launched on st.
      if (!h->cap_st)
        CK(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking), "capture stream");
      CK(cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeRelaxed), "graph capture begin");
      ret = batch_body(c, h->cap_st, segs);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(h->cap_st, &graph);
      if (ret < 0 || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        restore();
        if (ret < 0) return ret;
        return cuda_fail(h, e, "graph capture end");
      }
      cudaGraphExec_t exec = nullptr;
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        restore();
        return cuda_fail(h, e, "graph instantiate");
      }
      e = cudaGraphLaunch(exec, st);
      if (e != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        restore();
        return cuda_fail(h, e, "graph launch");
      }
      vimg_handle::GraphEntry ge;
      ge.key = std::move(key);
      ge.exec = exec;
      for (int v = 0; v < k; ++v)
        ge.end_state.insert(ge.end_state.end(),
                            {hs[v]->frames_seen, hs[v]->carry_n, hs[v]->carry_cur});
      ge.segs = segs;
      ge.ret = ret;
      if (h->graphs.size() >= kMaxGraphs) {
        cudaGraphExecDestroy(h->graphs.front().exec);
        h->graphs.erase(h->graphs.begin());
      }
      h->graphs.push_back(std::move(ge));
    }
  }
  if (ev && ret >= 0) {
    CK(cudaEventRecord(ev, st), "event record");
    for (int v = 1; v < k; ++v)
      if (hs[v]->st != st) CK(cudaStreamWaitEvent(hs[v]->st, ev, 0), "stream wait");
  }
  if (ret >= 0 && segments_out)
    for (int v = 0; v < k; ++v) segments_out[v] = segs[v];
  return ret;
}

extern "C" int vimg_process_host(vimg_handle* h, const uint16_t* h_frames, int n,
                                 float* h_shifts_out, float* h_summary_out,
                                 float* d_corrected_out) {
  if (!h) return fail(h, VIMG_ERR_ARG, "null handle");
  if (h->sticky) return h->sticky;
  if (n < 0 || (n > 0 && !h_frames)) return fail(h, VIMG_ERR_ARG, "bad frames");
  if (!h->have_template) return fail(h, VIMG_ERR_NO_TEMPLATE, "no template");
  const size_t HW = (size_t)h->H * h->W;
  const int L = h->p.segment_len, maxc = h->p.max_chunk;
  const int max_seg = (L - 1 + maxc) / L;
  if (!h->stage[0]) {
    for (int i = 0; i < kRing; ++i) {
      CK(cudaMalloc((void**)&h->stage[i], sizeof(uint16_t) * HW * maxc), "stage alloc");
      CK(cudaEventCreateWithFlags(&h->ev_copied[i], cudaEventDisableTiming), "event");
      CK(cudaEventCreateWithFlags(&h->ev_used[i], cudaEventDisableTiming), "event");
      CK(cudaEventRecord(h->ev_used[i], h->st), "event record");
    }
    for (int i = 0; i < 2; ++i) {
      CK(cudaMalloc((void**)&h->stage_shift[i], sizeof(float) * 2 * maxc), "stage alloc");
      CK(cudaMalloc((void**)&h->stage_summary[i],
                    sizeof(float) * 2 * HW * std::max(1, max_seg)),
         "stage alloc");
      CK(cudaEventCreateWithFlags(&h->ev_out[i], cudaEventDisableTiming), "event");
      CK(cudaEventCreateWithFlags(&h->ev_dl[i], cudaEventDisableTiming), "event");
      CK(cudaEventRecord(h->ev_dl[i], h->st), "event record");
    }
    CK(cudaStreamCreateWithFlags(&h->copy_st, cudaStreamNonBlocking), "copy stream");
    CK(cudaStreamCreateWithFlags(&h->dl_st, cudaStreamNonBlocking), "download stream");
  }
  // Three streams: uploads (copy_st) into a ring of kRing frame stages, compute
  // (st), downloads (dl_st) from two output stages.  Only events order them, so
  // a slow copy in either direction stalls the compute only when the ring (or
  // the output pair) is exhausted.
  int done = 0, k_total = 0, buf = 0, ob = 0;
  // the first batch is a quarter of max_chunk (whole segments): its upload is
  // the only one no compute hides, and the next, full batch uploads behind it
  const int first = std::max(L, (maxc / 4) / L * L);
  while (done < n) {
    int m = std::min(n - done, done == 0 ? std::min(first, maxc) : maxc);
    if (m < n - done) {
      const int cut = (int)((h->frames_seen + m) % L);
      if (m - cut > 0) m -= cut;
    }
    // H2D into stage[buf] once the batch that last used it has finished.
    CK(cudaStreamWaitEvent(h->copy_st, h->ev_used[buf], 0), "wait");
    CK(cudaMemcpyAsync(h->stage[buf], h_frames + HW * done, sizeof(uint16_t) * HW * m,
                       cudaMemcpyHostToDevice, h->copy_st),
       "frames upload");
    CK(cudaEventRecord(h->ev_copied[buf], h->copy_st), "event record");
    CK(cudaStreamWaitEvent(h->st, h->ev_copied[buf], 0), "wait");
    // the output stage ob is free once its previous download has finished
    CK(cudaStreamWaitEvent(h->st, h->ev_dl[ob], 0), "wait");
    vimg_io io{};
    io.shifts = h->stage_shift[ob];
    io.corrected = d_corrected_out ? d_corrected_out + HW * done : nullptr;
    io.summary = h_summary_out ? h->stage_summary[ob] : nullptr;
    int k = vimg_process_io(h, h->stage[buf], m, &io);
    if (k < 0) return k;
    CK(cudaEventRecord(h->ev_used[buf], h->st), "event record");
    CK(cudaEventRecord(h->ev_out[ob], h->st), "event record");
    CK(cudaStreamWaitEvent(h->dl_st, h->ev_out[ob], 0), "wait");
    if (h_shifts_out)
      CK(cudaMemcpyAsync(h_shifts_out + 2 * (size_t)done, h->stage_shift[ob],
                         sizeof(float) * 2 * m, cudaMemcpyDeviceToHost, h->dl_st),
         "shifts download");
    if (h_summary_out && k > 0)
      CK(cudaMemcpyAsync(h_summary_out + 2 * HW * (size_t)k_total, h->stage_summary[ob],
                         sizeof(float) * 2 * HW * k, cudaMemcpyDeviceToHost, h->dl_st),
         "summary download");
    CK(cudaEventRecord(h->ev_dl[ob], h->dl_st), "event record");
    k_total += k;
    done += m;
    buf = (buf + 1) % kRing;
    ob ^= 1;
  }
  // the caller's next work on the handle's stream sees the downloads complete
  CK(cudaStreamWaitEvent(h->st, h->ev_dl[ob ^ 1], 0), "wait");
  CK(cudaStreamSynchronize(h->st), "stream sync");
  return k_total;
}

extern "C" int vimg_profile_enable(vimg_handle* h, int on) {
  if (!h) return fail(h, VIMG_ERR_ARG, "null handle");
  if (h->sticky) return h->sticky;
  Prof& p = h->prof;
  if (on && !p.ev) {
    p.ev = new cudaEvent_t[2 * kProfSlots]();
    p.stage = new int[kProfSlots]();
    for (int i = 0; i < 2 * kProfSlots; ++i) CK(cudaEventCreate(&p.ev[i]), "event create");
  }
  p.on = on != 0;
  return VIMG_OK;
}

extern "C" int vimg_profile_read(vimg_handle* h, double* ms, long long* launches, int reset) {
  if (!h) return fail(h, VIMG_ERR_ARG, "null handle");
  if (h->sticky) return h->sticky;
  Prof& p = h->prof;
  if (p.used > 0) {
    CK(cudaStreamSynchronize(h->st), "stream sync");
    for (int s = 0; s < p.used; ++s) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, p.ev[2 * s], p.ev[2 * s + 1]), "event time");
      p.ms[p.stage[s]] += t;
    }
    p.used = 0;
  }
  for (int i = 0; i < VIMG_NSTAGES; ++i) {
    if (ms) ms[i] = p.ms[i];
    if (launches) launches[i] = p.launches[i];
    if (reset) p.ms[i] = 0.0, p.launches[i] = 0;
  }
  return VIMG_OK;
}

extern "C" int vimg_cnn_param_count(void) { return cnn_param_count(); }

extern "C" size_t vimg_cnn_workspace_floats(int n) { return n > 0 ? cnn_act_floats(n) : 0; }

static int cnn_status(cudaError_t e) {
  if (e != cudaSuccess) {
    g_create_error = std::string("proposal kernel: ") + cudaGetErrorString(e);
    return VIMG_ERR_CUDA;
  }
  return VIMG_OK;
}

extern "C" int vimg_cnn_prepare(const uint16_t* d_frames, int n, int H, int W,
                                const float* d_template, long long template_stride, float* d_ws,
                                void* stream) {
  if (n < 0 || (n > 0 && (!d_frames || !d_template || !d_ws)) || H < kCrop || W < kCrop)
    return VIMG_ERR_ARG;
  return cnn_status(cnn_input(d_frames, n, H, W, d_template, template_stride, d_ws,
                              (cudaStream_t)stream));
}

extern "C" int vimg_cnn_pack_bf16(const float* d_params, void* d_params_bf16, void* stream) {
  if (!d_params || !d_params_bf16) return VIMG_ERR_ARG;
  return cnn_status(cnn_to_bf16(d_params, (__nv_bfloat16*)d_params_bf16, (cudaStream_t)stream));
}

extern "C" int vimg_cnn_forward(const float* d_params, const void* d_params_bf16, float* d_ws,
                                int n, float* d_out, void* stream) {
  if (!d_params || !d_params_bf16 || !d_ws || !d_out || n < 1) return VIMG_ERR_ARG;
  return cnn_status(cnn_forward(d_params, (const __nv_bfloat16*)d_params_bf16, d_ws, n, d_out,
                                (cudaStream_t)stream));
}

extern "C" int vimg_cnn_loss(const float* d_out, const float* d_target, int n, float* d_dout,
                             float* d_loss, void* stream) {
  if (!d_out || !d_target || !d_dout || n < 1) return VIMG_ERR_ARG;
  return cnn_status(cnn_mse(d_out, d_target, n, d_dout, d_loss, (cudaStream_t)stream));
}

extern "C" int vimg_cnn_backward(const float* d_params, const void* d_params_bf16,
                                 const float* d_ws, float* d_dws, int n, const float* d_dout,
                                 float* d_grads, void* stream) {
  if (!d_params || !d_params_bf16 || !d_ws || !d_dws || !d_dout || !d_grads || n < 1)
    return VIMG_ERR_ARG;
  return cnn_status(cnn_backward(d_params, (const __nv_bfloat16*)d_params_bf16, d_ws, d_dws, n,
                                 d_dout, d_grads, (cudaStream_t)stream));
}

extern "C" int vimg_cnn_adam(float* d_params, const float* d_grads, float* d_m, float* d_v,
                             float lr, float beta1, float beta2, float eps, int step,
                             void* stream) {
  if (!d_params || !d_grads || !d_m || !d_v || step < 1) return VIMG_ERR_ARG;
  return cnn_status(cnn_adam(d_params, d_grads, d_m, d_v, lr, beta1, beta2, eps, step,
                             (cudaStream_t)stream));
}

extern "C" int vimg_load_proposal(vimg_handle* h, const float* d_params) {
  if (!h || !d_params) return fail(h, VIMG_ERR_ARG, "null handle or parameters");
  if (h->sticky) return h->sticky;
  if (!(h->p.flags & VIMG_PROPOSAL_CNN))
    return fail(h, VIMG_ERR_ARG, "handle was created without VIMG_PROPOSAL_CNN");
  CK(cudaMemcpyAsync(h->cnn_p, d_params, sizeof(float) * cnn_param_count(),
                     cudaMemcpyDeviceToDevice, h->st),
     "proposal copy");
  CK(cnn_to_bf16(h->cnn_p, h->cnn_b, h->st), "proposal pack");
  h->have_proposal = true;
  return VIMG_OK;
}

extern "C" int vimg_proposal_stats(vimg_handle* h, long long* frames, long long* fallbacks) {
  if (!h) return fail(h, VIMG_ERR_ARG, "null handle");
  if (h->sticky) return h->sticky;
  long long fb = 0;
  if (h->fb_total) {
    CK(cudaMemcpyAsync(&fb, h->fb_total, sizeof(long long), cudaMemcpyDeviceToHost, h->st),
       "stats copy");
    CK(cudaStreamSynchronize(h->st), "stream sync");
  }
  if (frames) *frames = h->prop_frames;
  if (fallbacks) *fallbacks = fb;
  return VIMG_OK;
}

extern "C" int vimg_synchronize(vimg_handle* h) {
  if (!h) return fail(h, VIMG_ERR_ARG, "null handle");
  if (h->sticky) return h->sticky;
  int derr = 0;
  CK(cudaMemcpyAsync(&derr, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, h->st), "status copy");
  CK(cudaStreamSynchronize(h->st), "stream sync");
  if (derr)
    return fail(h, VIMG_ERR_TIMEOUT,
                "a device-side wait gave up (flag " +
                    std::to_string(derr) + ")");
  return VIMG_OK;
}
