// noalloc.cu -- hierarchical-DDA traversal that allocates nothing.
//
// hdda_traverse_hdda needs a little device scratch per call (per-CTA sample
// sums, their scan, a few counters) and a lattice table that it caches; it
// allocates both itself.  Some callers cannot allow that: a host application
// that reserves all of the GPU's memory up front and hands libraries fixed
// buffers, or a render loop that must never enter the CUDA allocator.  For
// them this file provides one more entry point whose scratch lives in a
// file-scope device array of fixed size.  The caller still passes inputs and
// outputs; the library allocates no device or host memory on this path.
//
// The array is created when the library is loaded on a device and stays
// there until the process exits.  Host code cannot use the array's name as
// a device address (it names a host-side stand-in), so the address is looked
// up once per device with cudaGetSymbolAddress while that device is current.
// The first call on each device does that lookup; make it before any stream
// capture.  Every call uses the same array: calls whose GPU work overlaps
// (on different streams, or from different host threads) race on it and
// must be serialised by the caller.  Each call clears the counters it needs
// and keeps nothing from the previous call.
#include <mutex>

#include "grid.cuh"

namespace {

constexpr int kStaticMaxCandidates = 16384;            // lattice candidates per ray
constexpr int64_t kStaticMaxTiles = 16384;             // CTAs of 128 rays: 2,097,152 rays
constexpr size_t kStaticScratchBytes = 393728;         // the documented size
// The array must hold the traversal's scratch layout at the maximum sizes; a
// change to that layout that outgrows it fails to compile here.
static_assert(hdda::traverse_scratch_bytes(kStaticMaxCandidates, kStaticMaxTiles) <=
                  kStaticScratchBytes,
              "static scratch smaller than the traversal's layout at its maximum sizes");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (looked up once).
int static_scratch(void** out) {
  int dev = 0;
  HDDA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return hdda::set_error(HDDA_ERR_INVALID_ARG, "device %d beyond %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return hdda::cuda_error(e, "cudaGetSymbolAddress(g_static_scratch)");
    if (!p) return hdda::set_error(HDDA_ERR_CUDA, "static scratch has no device address");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return HDDA_OK;
}

}  // namespace

extern "C" int hdda_traverse_hdda_noalloc(const float* rays_o, const float* rays_d,
                                          int64_t n_rays, const hdda_grid* grid,
                                          const hdda_params* params, int64_t* offsets,
                                          int32_t* ray_idx, float* t0, float* t1,
                                          int64_t capacity, int64_t* total_out,
                                          hdda_stream_t stream) {
  hdda::clear_error();
  void* scratch = nullptr;
  int st = static_scratch(&scratch);
  if (st != HDDA_OK) return st;
  return hdda::traverse_with_scratch(true, rays_o, rays_d, n_rays, grid, params, offsets,
                                     ray_idx, t0, t1, capacity, total_out, scratch,
                                     kStaticMaxCandidates, kStaticMaxTiles,
                                     (cudaStream_t)stream);
}
