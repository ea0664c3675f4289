// Motion estimate without any allocation: vimg_motion_noalloc.
//
// Some callers cannot allocate device memory at the moment they need shifts:
// real-time acquisition loops that forbid allocator calls (cudaMalloc can
// synchronise the device and block on the driver, which breaks the frame
// deadline), and hosts that hand the GPU to this library with every byte of
// device memory already reserved for their own frame buffers.  For them this
// entry point runs the same kernels as vimg_process's motion estimate (template
// preparation, exact window statistics, FP32 ZNCC correlation, integer peak and
// parabola) with all of its scratch in one fixed array that lives in the
// library's static device memory.
//
// Limits and rules:
//   - The array holds kNoAllocBytes (12 MiB); frames up to 1024 x 1024 with a
//     search radius up to 16 fit.  Larger frames are rejected with
//     VIMG_ERR_SIZE before any work is enqueued.  At 1024 x 1024 and R = 16 the
//     statistics maps of two frames fill the array, so frames go two per launch
//     there.
//   - Every GPU that loads the library holds the array until the process exits.
//   - The first call on a device looks up the array's device address with that
//     device current (cudaGetSymbolAddress) and sets the kernels' attributes for
//     that device.  Make that first call before any stream capture begins.
//   - Every call shares the one array and leaves its contents behind; the call
//     clears what must start at zero itself.  Calls whose work overlaps on the
//     GPU (different streams, or different host threads without ordering) race
//     on the array and give wrong results: serialise them.
#include <mutex>

#include "vimg_internal.h"

using namespace vimg;

namespace {
constexpr size_t kNoAllocBytes = 12u << 20;
}  // namespace

// The scratch array itself (host code must use its device address, see below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

constexpr int kNoAllocMaxSide = 1024;
constexpr int kNoAllocBatch = 16;  // frames per stats/correlation launch (as vimg_process)

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Device address of the scratch array on the current device (looked up once per
// device).  In host code g_noalloc_scratch names a host-side stand-in, not device
// memory: only the address returned here may be handed to a kernel.
cudaError_t noalloc_scratch(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
  return cudaSuccess;
}

}  // namespace

extern "C" int vimg_motion_noalloc(const float* d_template, const uint16_t* d_frames, int n,
                                   int H, int W, int search_radius, float* d_shifts_out,
                                   float* d_peak_info, void* stream) {
  if (!d_template || (n > 0 && (!d_frames || !d_shifts_out)) || n < 0) return VIMG_ERR_ARG;
  if (search_radius < 0 || search_radius > kMaxR) return VIMG_ERR_ARG;
  const int R = search_radius;
  if (H > kNoAllocMaxSide || W > kNoAllocMaxSide || H - 2 * R < kPatch || W - 2 * R < kPatch)
    return VIMG_ERR_SIZE;
  PatchGrid g;
  g.ny = (H - 2 * R) / kPatch;
  g.nx = (W - 2 * R) / kPatch;
  g.y0 = R + ((H - 2 * R) - g.ny * kPatch) / 2;
  g.x0 = R + ((W - 2 * R) - g.nx * kPatch) / 2;
  const int np = g.ny * g.nx, w = 2 * R + 1, nwin = w * w;
  // Scratch layout: template constants, then per-frame statistics maps and
  // fixed-point surfaces for one batch.
  const size_t b_tc = align256(sizeof(float) * (size_t)np * kPatch * kTplStride);
  const size_t b_tn2 = align256(sizeof(float) * np);
  const size_t b_coff = align256(sizeof(int) * np);
  const size_t per_frame_isf = sizeof(float) * stats_map_floats(g, R);
  const size_t per_frame_cs = sizeof(unsigned long long) * nwin;
  const size_t fixed = b_tc + b_tn2 + b_coff;
  if (fixed + align256(per_frame_isf) + align256(per_frame_cs) > kNoAllocBytes)
    return VIMG_ERR_SIZE;
  int batch = (int)((kNoAllocBytes - fixed - 512) / (per_frame_isf + per_frame_cs));
  if (batch > kNoAllocBatch) batch = kNoAllocBatch;
  if (batch < 1) return VIMG_ERR_SIZE;  // not one frame's scratch: nothing is enqueued
  if (n == 0) return VIMG_OK;

  const int dev = current_device();
  if (dev < 0) return VIMG_ERR_CUDA;
  if (kernels_init() != cudaSuccess) return VIMG_ERR_CUDA;
  unsigned char* base = nullptr;
  if (noalloc_scratch(dev, &base) != cudaSuccess) return VIMG_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  TemplateDev td;
  td.tc = reinterpret_cast<float*>(base);
  td.tn2 = reinterpret_cast<float*>(base + b_tc);
  td.coff = reinterpret_cast<int*>(base + b_tc + b_tn2);
  float* isf = reinterpret_cast<float*>(base + fixed);
  unsigned long long* csum =
      reinterpret_cast<unsigned long long*>(base + fixed + align256(per_frame_isf * batch));
  if (launch_template_prep(d_template, H, W, g, td, st) != cudaSuccess) return VIMG_ERR_CUDA;
  const size_t HW = (size_t)H * W;
  for (int f0 = 0; f0 < n; f0 += batch) {
    const int m = n - f0 < batch ? n - f0 : batch;
    if (cudaMemsetAsync(csum, 0, per_frame_cs * m, st) != cudaSuccess) return VIMG_ERR_CUDA;
    if (launch_stats(d_frames + HW * f0, m, H, W, g, R, td, isf, st) != cudaSuccess)
      return VIMG_ERR_CUDA;
    if (launch_corr_f32(d_frames + HW * f0, m, H, W, g, R, td, isf, csum, st) != cudaSuccess)
      return VIMG_ERR_CUDA;
    if (launch_peak(csum, m, R, np, d_shifts_out + 2 * (size_t)f0,
                    d_peak_info ? d_peak_info + 4 * (size_t)f0 : nullptr, nullptr, st) !=
        cudaSuccess)
      return VIMG_ERR_CUDA;
  }
  return VIMG_OK;
}
