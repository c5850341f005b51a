// hdda_internal.cuh -- device-side views, status helpers and the exact
// binary32 point arithmetic shared by the grid builders and the samplers.
//
// Every float operation that decides a sample goes through __fadd_rn /
// __fsub_rn / __fmul_rn, which the compiler never contracts into a fused
// multiply-add, and the translation units that use them are also compiled
// with -fmad=false.  Together with IEEE round-to-nearest on both sides this
// makes the samplers reproduce the binary32 definition exactly.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hdda.h"

namespace hdda {

constexpr int kMaxLevels = HDDA_MAX_LEVELS;
constexpr int kBlockDim = 8;     // leaf block edge (8^3 voxels)
constexpr int kNodeDim = 16;     // node edge in blocks (16^3 blocks)
constexpr int kNodeVox = kBlockDim * kNodeDim;  // 128 voxels per node edge
constexpr int kNodeWords = 4096 / 32;           // 128 mask words per node
constexpr int kLeafWords = 512 / 32;            // 16 words per leaf
// Refinement masks (set bit = the group holds some occupied voxel):
//   per node: 64 bits for its 4^3 groups of 32^3 voxels, then 512 bits for
//   its 8^3 groups of 16^3 voxels;  per leaf: 64 bits for its 4^3 cells of
//   2^3 voxels, then 8 bits for its 2^3 cells of 4^3 voxels, then 64 bits
//   for the 2^3-voxel cells that are fully occupied.
constexpr int kSuperWords = 2 + 16;
constexpr int kLeafSubWords = 5;
// Region map (built from the refined tree): one 16-bit entry per 2^3-voxel
// cell, level by level, cells in C order over C = ceil(R / 2) per axis.
// Bits 8-15: log2 of the edge of the coarsest uniform region of the refined
// tree that holds the cell (0: the cell itself is not uniform; 1: a 2^3
// cell; 2: an empty or full 4^3 cell; 3: an empty or tiled 8^3 block; 4, 5: an
// empty 16^3 or 32^3 group; 7: an empty or full 128^3 node).  Bits 0-7: the
// cell's voxels, bit ((x & 1) * 2 + (y & 1)) * 2 + (z & 1); 0x00 or 0xff
// when the region is uniform, so the occupancy of any voxel is one bit test.
constexpr int kMapNodeLog2 = 7;  // log2(kNodeVox)

// Walk variants: dense bit array, VDB tree, VDB tree with refinement masks.
// kModeVdbMap walks the refined tree's regions, found through the region map.
enum WalkMode : int { kModeDense = 0, kModeVdb = 1, kModeVdbMap = 2 };

enum NodeState : uint32_t { kNodeEmpty = 0, kNodeMixed = 1, kNodeFull = 2 };
enum BlockState : uint8_t { kBlockEmpty = 0, kBlockPartial = 1, kBlockFull = 2 };

// Status bits a kernel may raise in a device status word.
enum DeviceStatus : uint32_t {
  kDevOk = 0,
  kDevStepLimit = 1u << 0,
  kDevInternal = 1u << 1,
  kDevCapacity = 1u << 2,
  kDevTimeout = 1u << 3,
  kDevBadIndex = 1u << 4,
};

struct LevelDev {
  float lo[3];
  float hi[3];
  float s[3];  // fl32(res / fl32(hi - lo))
};

// Everything a traversal kernel needs to know about a grid, passed by value
// as a kernel parameter (it lives in the constant bank).
struct GridDev {
  int kind;
  int L, R, B, N;
  int W;                     // dense bit words per level
  LevelDev lv[kMaxLevels];
  const float* thr;          // [L][3][R+1] exact index thresholds
  const uint32_t* bits;      // dense: [L][W]
  const uint32_t* child;     // vdb: [L*N^3][128]
  const uint32_t* tile;      // vdb: [L*N^3][128]
  const uint32_t* prefix;    // vdb: [L*N^3][128] global leaf index per word
  const uint32_t* nstate;    // vdb: [L*N^3]
  const uint32_t* leaves;    // vdb: [n_leaves][16]
  const uint32_t* nsuper;    // vdb: [L*N^3][kSuperWords]
  const uint32_t* lsub;      // vdb: [n_leaves][kLeafSubWords]
  const uint16_t* rmap;      // vdb: [L][C][C][C] region map, C = ceil(R / 2)
  int check;                 // walk checks that each region holds its point
};

// Buckets of the lattice's inverse index (t -> k), over binary32 keys.
constexpr int kKidxMax = 2048;

// The lattice shared by every ray of a call: t[0..K], tm[0..K-1] (interval
// midpoints), and a bucket index kidx[0..NB+1] over the order-preserving
// keys of tm: kidx[b] = first k with key(tm_k) >= key0 + (b << shift).
// hdr = {key0, shift, NB, closed form, ks, A, -, -} lives in device memory
// next to the tables (the closed form of the index estimate: see lat_hdr).
struct LatticeDev {
  const float* t;
  const float* tm;
  const int* kidx;
  const uint32_t* hdr;
  int K;
};

// Bytes of one lattice block of capacity max_k: t, tm, kidx and hdr.
__host__ __device__ constexpr size_t lattice_block_bytes(int max_k) {
  return (sizeof(float) * (2 * (size_t)max_k + 1) + sizeof(int) * (kKidxMax + 2) + 32 + 255) &
         ~(size_t)255;
}

__device__ __forceinline__ int voxel_index(float x, float lo, float s, int R) {
  float u = __fmul_rn(__fsub_rn(x, lo), s);
  int i = (int)floorf(u);
  return min(max(i, 0), R - 1);
}

// Order-preserving map between binary32 values and uint32 keys.
__device__ __forceinline__ uint32_t float_key(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}

}  // namespace hdda

// ---------------------------------------------------------------------------
// host-side helpers (runtime.cu)
// ---------------------------------------------------------------------------
namespace hdda {
int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what);
void clear_error();

// True while the kernel timers are enabled (runtime.cu).
bool profiler_on();
// True while the work counters are enabled (runtime.cu).
bool counters_on();
// True while the walk's device-side region checks are enabled (runtime.cu).
bool region_checks_on();
// The two-pass samplers' current form, HDDA_SAMPLER_FUSED or _SEPARATE (runtime.cu).
int sampler_form();
// Blob evaluations counted by the compositor since the last call (composite.cu).
unsigned long long composite_take_blob_evals();
// The same count for the render-only path (render.cu).
unsigned long long render_take_blob_evals();

// Brackets one kernel launch with events when the profiler is enabled.
class KernelTimer {
 public:
  // allow = false makes it a no-op (paths that must not create CUDA objects).
  KernelTimer(const char* name, cudaStream_t s, bool allow = true);
  void stop();
  ~KernelTimer() { stop(); }
 private:
  const char* name_;
  cudaStream_t s_;
  cudaEvent_t a_ = nullptr;
  bool live_ = false;
};
// Traversal over scratch memory the caller provides instead of memory the
// library allocates (traverse.cu).  `scratch` is device memory of at least
// traverse_scratch_bytes(max_k, max_tiles) bytes, 256-byte aligned; nothing
// is allocated.  Rays per tile: traverse_rays_per_tile().  Layout: 256 bytes
// of lattice read-back words, one lattice block of capacity max_k, then the
// one-pass sampler's 32-byte header and one 8-byte state per tile.
constexpr size_t traverse_scratch_bytes(int max_k, int64_t max_tiles) {
  return 256 + lattice_block_bytes(max_k) + 32 + 8 * (size_t)max_tiles;
}
// Validates params and returns the cached device lattice for them (traverse.cu).
int lattice_for(const hdda_params* p, cudaStream_t s, LatticeDev* out);
int64_t traverse_rays_per_tile();
int traverse_with_scratch(bool vdb, const float* ro, const float* rd, int64_t n,
                          const struct ::hdda_grid* grid, const hdda_params* params,
                          int64_t* offsets, int32_t* ray_idx, float* t0, float* t1,
                          int64_t capacity, int64_t* total_out, void* scratch, int max_k,
                          int64_t max_tiles, cudaStream_t s);
}  // namespace hdda

#define HDDA_CUDA_TRY(expr)                                   \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) return ::hdda::cuda_error(_e, #expr); \
  } while (0)
