// traverse.cu -- the per-ray samplers: dense-grid DDA (the baseline) and
// hierarchical DDA over the VDB grid (Sec. 2.3, Sec. 3, Algorithm 1).
//
// Both samplers share one walk.  The lattice t_0 < t_1 < ... depends only on
// the call's parameters (Algorithm 1 advances t_last by Delta t whatever
// voxel it is in), so it is computed once per parameter set into a small
// device table and shared by every ray.  A ray then alternates two steps
// (Algorithm 1's analyzer and its inner loops):
//
//   locate   the lattice point x(t_k) is classified and given a REGION: an
//            axis-aligned set that holds x(t_k) and has one occupancy value
//            throughout.  For dense DDA the region is the voxel; for HDDA it
//            is the coarsest uniform node of the tree: an empty or full
//            16^3-block node, an empty or tiled 8^3 block, or a voxel of a
//            leaf.  Outside every cascade box the region is a half-space the
//            ray is leaving towards, or everything when it never comes back.
//   cross    the first later lattice point outside the region is found by a
//            galloping then bisecting search over k.  Every probe evaluates
//            the point exactly as the definition does.
//
// Why this is exact: binary32 rounding is monotone, so for a fixed ray each
// coordinate fl(o + fl(tm_k * d)) is monotone in k, and so is every voxel
// index derived from it.  The points inside an axis-aligned region therefore
// form one contiguous run of k, and only the region's exit plane on each
// axis (the one the ray moves towards) can end the run.  Region bounds are
// exact binary32 thresholds (grid.cu), so "inside" is decided exactly too.
// The result is the sample set of the definition, with dense DDA and HDDA
// bit-identical; HDDA just crosses far fewer regions.
//
// Output is produced in two passes (count, then emit) with the per-CTA
// totals scanned by the last CTA of the count pass, so emission needs no
// separate scan kernel and rays with no samples are not walked twice.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "grid.cuh"

namespace hdda {
namespace {

constexpr int kBS = 128;  // threads per CTA of the samplers
constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// lattice
// ---------------------------------------------------------------------------

__device__ __forceinline__ float lattice_next(float t, const hdda_params& p) {
  const float dt = fminf(fmaxf(__fmul_rn(t, p.cone_angle), p.step), p.max_step);
  return __fadd_rn(t, dt);
}

__global__ void lattice_count_kernel(hdda_params p, int64_t* out) {
  float t = p.near_t;
  int64_t k = 0, limit = 0;
  for (;;) {
    const float tn = lattice_next(t, p);
    if (tn > p.far_t) break;
    if (k == p.max_steps) { limit = 1; break; }
    ++k;
    t = tn;
  }
  out[0] = k;
  out[1] = limit;
}

__global__ void lattice_fill_kernel(hdda_params p, int K, float* __restrict__ t_out,
                                    float* __restrict__ tm_out) {
  float t = p.near_t;
  t_out[0] = t;
  for (int k = 0; k < K; ++k) {
    const float tn = lattice_next(t, p);
    t_out[k + 1] = tn;
    tm_out[k] = __fmul_rn(__fadd_rn(t, tn), 0.5f);
    t = tn;
  }
}

// ---------------------------------------------------------------------------
// the walk
// ---------------------------------------------------------------------------

struct Ray {
  float o[3], d[3];
  bool neg[3];  // direction component < 0 (a zero component counts as positive)
};

__device__ __forceinline__ bool load_ray(const float* __restrict__ ro,
                                         const float* __restrict__ rd, int64_t r, Ray& ray) {
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    ray.o[c] = __ldg(ro + 3 * r + c);
    ray.d[c] = __ldg(rd + 3 * r + c);
    ok &= isfinite(ray.o[c]) && isfinite(ray.d[c]);
    ray.neg[c] = ray.d[c] < 0.f;
  }
  return ok;
}

// x = o + tm * d per axis, one rounding per operation.
__device__ __forceinline__ void point_at(const Ray& r, float tm, float x[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) x[c] = __fadd_rn(r.o[c], __fmul_rn(tm, r.d[c]));
}

// A region is kept as one exit plane per axis: e[c] bounds the region on the
// side the ray moves towards (upper bound, exclusive, for d >= 0; lower
// bound, inclusive, for d < 0).
__device__ __forceinline__ bool outside(const float x[3], const float e[3], const Ray& r) {
  return ((x[0] >= e[0]) != r.neg[0]) | ((x[1] >= e[1]) != r.neg[1]) |
         ((x[2] >= e[2]) != r.neg[2]);
}

// Intersects the region with [lo, hi) along axis c.
__device__ __forceinline__ void clip(float e[3], const Ray& r, int c, float lo, float hi) {
  e[c] = r.neg[c] ? fmaxf(e[c], lo) : fminf(e[c], hi);
}

// Intersects the region with voxels [a0, a1) of axis c of one level, using
// the exact thresholds X[a] (only the bound on the exit side is loaded).
__device__ __forceinline__ void clip_cells(float e[3], const Ray& r, const float* __restrict__ thr,
                                           int R1, int c, int a0, int a1) {
  if (r.neg[c]) e[c] = fmaxf(e[c], __ldg(thr + c * R1 + a0));
  else e[c] = fminf(e[c], __ldg(thr + c * R1 + a1));
}

// Classifies x and sets e to the region holding it.  Returns its occupancy.
template <bool kVdb>
__device__ __forceinline__ bool locate(const GridDev& g, const Ray& r, const float x[3],
                                       float e[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) e[c] = r.neg[c] ? -INFINITY : INFINITY;
  int l = -1;
  for (int lv = 0; lv < g.L; ++lv) {
    const LevelDev& B = g.lv[lv];
    bool inside = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) inside &= (x[c] >= B.lo[c]) & (x[c] < B.hi[c]);
    if (inside) { l = lv; break; }
    // x lies outside this (finer) box: keep a half-space that separates the
    // ray's later points from it, preferring the one it leaves last.
    int best = -1;
    float best_t = -1.f;
    bool never = false;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (x[c] < B.lo[c]) {
        if (!(r.d[c] > 0.f)) never = true;  // coordinate never grows: never enters
        else {
          const float t = __fdividef(B.lo[c] - x[c], r.d[c]);
          if (t > best_t) { best_t = t; best = c; }
        }
      } else if (x[c] >= B.hi[c]) {
        if (!(r.d[c] < 0.f)) never = true;
        else {
          const float t = __fdividef(x[c] - B.hi[c], -r.d[c]);
          if (t > best_t) { best_t = t; best = c; }
        }
      }
    }
    if (never || best < 0) continue;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (c != best) continue;
      if (r.neg[c]) e[c] = fmaxf(e[c], B.hi[c]);  // region x >= hi
      else e[c] = fminf(e[c], B.lo[c]);           // region x < lo
    }
  }
  if (l < 0) return false;

  const LevelDev& V = g.lv[l];
  int i[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    clip(e, r, c, V.lo[c], V.hi[c]);
    i[c] = voxel_index(x[c], V.lo[c], V.s[c], g.R);
  }
  const int R1 = g.R + 1;
  const float* thr = g.thr + (int64_t)l * 3 * R1;
  if (!kVdb) {
    const int64_t lin = ((int64_t)i[0] * g.R + i[1]) * g.R + i[2];
    const uint32_t w = __ldg(g.bits + (int64_t)l * g.W + (lin >> 5));
#pragma unroll
    for (int c = 0; c < 3; ++c) clip_cells(e, r, thr, R1, c, i[c], i[c] + 1);
    return (w >> (lin & 31)) & 1u;
  }
  // node level
  const int N = g.N;
  const int64_t ng = (int64_t)l * N * N * N +
                     ((i[0] >> 7) * N + (i[1] >> 7)) * N + (i[2] >> 7);
  const uint32_t st = __ldg(g.nstate + ng);
  if (st != kNodeMixed) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int a0 = i[c] & ~(kNodeVox - 1);
      clip_cells(e, r, thr, R1, c, a0, min(a0 + kNodeVox, g.R));
    }
    return st == kNodeFull;
  }
  // block level: empty or tile
  const int cell = (((i[0] >> 3) & 15) * 16 + ((i[1] >> 3) & 15)) * 16 + ((i[2] >> 3) & 15);
  const int w = cell >> 5;
  const uint32_t bit = 1u << (cell & 31);
  const uint32_t cw = __ldg(g.child + ng * kNodeWords + w);
  if (!(cw & bit)) {
    const uint32_t tw = __ldg(g.tile + ng * kNodeWords + w);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int a0 = i[c] & ~(kBlockDim - 1);
      clip_cells(e, r, thr, R1, c, a0, min(a0 + kBlockDim, g.R));
    }
    return (tw & bit) != 0u;
  }
  // voxel of a leaf
  const uint32_t leaf = __ldg(g.prefix + ng * kNodeWords + w) + __popc(cw & (bit - 1u));
  const int v = ((i[0] & 7) * 8 + (i[1] & 7)) * 8 + (i[2] & 7);
  const uint32_t lw = __ldg(g.leaves + (int64_t)leaf * kLeafWords + (v >> 5));
#pragma unroll
  for (int c = 0; c < 3; ++c) clip_cells(e, r, thr, R1, c, i[c], i[c] + 1);
  return (lw >> (v & 31)) & 1u;
}

// First k' in (k, K] whose point is outside the region (K if none).  The
// point of k is inside.  xo receives the point of k' when k' < K.
__device__ __forceinline__ int cross(const Ray& r, const float* __restrict__ tm, int k, int K,
                                     const float e[3], float xo[3]) {
  int lo = k, hi, step = 1;
  for (;;) {
    hi = lo + step;
    if (hi >= K) { hi = K; break; }
    float xh[3];
    point_at(r, __ldg(tm + hi), xh);
    if (outside(xh, e, r)) {
      xo[0] = xh[0]; xo[1] = xh[1]; xo[2] = xh[2];
      break;
    }
    lo = hi;
    step <<= 1;
  }
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    float xm[3];
    point_at(r, __ldg(tm + mid), xm);
    if (outside(xm, e, r)) {
      hi = mid;
      xo[0] = xm[0]; xo[1] = xm[1]; xo[2] = xm[2];
    } else {
      lo = mid;
    }
  }
  return hi;
}

template <bool kVdb, bool kEmit>
__device__ __forceinline__ int64_t walk(const GridDev& g, const LatticeDev& lat, const Ray& r,
                                        int32_t rid, int64_t out, int32_t* __restrict__ ray_idx,
                                        float* __restrict__ t0, float* __restrict__ t1,
                                        unsigned* __restrict__ status) {
  const int K = lat.K;
  int64_t cnt = 0;
  if (K <= 0) return 0;
  float x[3];
  point_at(r, __ldg(lat.tm), x);
  int k = 0;
  while (k < K) {
    float e[3];
    const bool occ = locate<kVdb>(g, r, x, e);
    if (outside(x, e, r)) atomicOr(status, kDevInternal);  // region must hold its point
    const int kn = cross(r, lat.tm, k, K, e, x);
    if (occ) {
      if (kEmit) {
        float ta = __ldg(lat.t + k);
        for (int j = k; j < kn; ++j) {
          const float tb = __ldg(lat.t + j + 1);
          ray_idx[out + cnt] = rid;
          t0[out + cnt] = ta;
          t1[out + cnt] = tb;
          ta = tb;
          ++cnt;
        }
      } else {
        cnt += kn - k;
      }
    }
    k = kn;
  }
  return cnt;
}

__device__ __forceinline__ int64_t cta_exclusive_scan64(int64_t v, int64_t* total) {
  __shared__ int64_t wt[kBS / 32 + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wt[warp] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t s = 0;
    for (int w = 0; w < kBS / 32; ++w) {
      const int64_t t = wt[w];
      wt[w] = s;
      s += t;
    }
    wt[kBS / 32] = s;
  }
  __syncthreads();
  const int64_t res = wt[warp] + inc - v;
  *total = wt[kBS / 32];
  __syncthreads();
  return res;
}

// Pass 1: per-ray counts into offsets[r]; per-CTA sums; the last CTA to
// finish scans the CTA sums into tile_prefix and writes the total.
template <bool kVdb>
__global__ void __launch_bounds__(kBS) count_kernel(
    const float* __restrict__ ro, const float* __restrict__ rd, int64_t n, GridDev g,
    LatticeDev lat, int64_t* __restrict__ offsets, int64_t* __restrict__ tile_sum,
    int64_t* __restrict__ tile_prefix, unsigned* __restrict__ ticket,
    unsigned* __restrict__ status, int64_t* __restrict__ total) {
  const int64_t r = blockIdx.x * (int64_t)kBS + threadIdx.x;
  int64_t c = 0;
  if (r < n) {
    Ray ray;
    if (load_ray(ro, rd, r, ray))
      c = walk<kVdb, false>(g, lat, ray, (int32_t)r, 0, nullptr, nullptr, nullptr, status);
    offsets[r] = c;
  }
  int64_t bsum = 0;
  cta_exclusive_scan64(c, &bsum);
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
    tile_sum[blockIdx.x] = bsum;
    __threadfence();
    is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  int64_t carry = 0;
  for (int64_t c0 = 0; c0 < gridDim.x; c0 += kBS) {
    const int64_t i = c0 + threadIdx.x;
    const int64_t v = i < gridDim.x ? __ldcg(tile_sum + i) : 0;
    int64_t chunk = 0;
    const int64_t ex = cta_exclusive_scan64(v, &chunk);
    if (i < gridDim.x) tile_prefix[i] = carry + ex;
    carry += chunk;
  }
  if (threadIdx.x == 0) *total = carry;
}

// Turns the counts in offsets[] into CSR row pointers.
__device__ __forceinline__ int64_t finish_offsets(int64_t r, int64_t n, int64_t* offsets,
                                                  const int64_t* tile_prefix,
                                                  const int64_t* total, int64_t& c) {
  c = r < n ? offsets[r] : 0;
  int64_t unused = 0;
  const int64_t off = __ldg(tile_prefix + blockIdx.x) + cta_exclusive_scan64(c, &unused);
  if (r < n) offsets[r] = off;
  if (blockIdx.x == 0 && threadIdx.x == 0) offsets[n] = *total;
  return off;
}

__global__ void __launch_bounds__(kBS) offsets_kernel(int64_t n, int64_t* __restrict__ offsets,
                                                      const int64_t* __restrict__ tile_prefix,
                                                      const int64_t* __restrict__ total) {
  const int64_t r = blockIdx.x * (int64_t)kBS + threadIdx.x;
  int64_t c;
  finish_offsets(r, n, offsets, tile_prefix, total, c);
}

// Pass 2: row pointers, then every ray with samples walks again and writes them.
template <bool kVdb>
__global__ void __launch_bounds__(kBS) emit_kernel(
    const float* __restrict__ ro, const float* __restrict__ rd, int64_t n, GridDev g,
    LatticeDev lat, int64_t* __restrict__ offsets, const int64_t* __restrict__ tile_prefix,
    const int64_t* __restrict__ total, int32_t* __restrict__ ray_idx, float* __restrict__ t0,
    float* __restrict__ t1, unsigned* __restrict__ status) {
  const int64_t r = blockIdx.x * (int64_t)kBS + threadIdx.x;
  int64_t c;
  const int64_t off = finish_offsets(r, n, offsets, tile_prefix, total, c);
  if (r < n && c > 0) {
    Ray ray;
    load_ray(ro, rd, r, ray);
    walk<kVdb, true>(g, lat, ray, (int32_t)r, off, ray_idx, t0, t1, status);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct LatticeEntry {
  hdda_params key;
  int device;
  float* t;
  float* tm;
  int K;
  int status;
};

std::mutex g_lattice_mu;
std::vector<LatticeEntry> g_lattices;

bool same_params(const hdda_params& a, const hdda_params& b) {
  return std::memcmp(&a, &b, sizeof(hdda_params)) == 0;
}

int validate_params(const hdda_params* p) {
  if (!p) return set_error(HDDA_ERR_INVALID_ARG, "params is NULL");
  const float v[5] = {p->near_t, p->far_t, p->step, p->cone_angle, p->max_step};
  for (float f : v)
    if (!std::isfinite(f)) return set_error(HDDA_ERR_INVALID_ARG, "params must be finite");
  if (!(p->step > 0.f) || !(p->max_step > 0.f) || !(p->cone_angle >= 0.f))
    return set_error(HDDA_ERR_INVALID_ARG, "need step > 0, max_step > 0, cone_angle >= 0");
  if (p->max_steps < 0 || p->max_steps > (1 << 24))
    return set_error(HDDA_ERR_INVALID_ARG, "max_steps=%d outside 0..2^24", p->max_steps);
  return HDDA_OK;
}

// Pinned host words for the one read-back per call.
struct HostWords {
  int64_t* p = nullptr;
  ~HostWords() { if (p) cudaFreeHost(p); }
};
thread_local HostWords t_host;

int host_words(int64_t** out) {
  if (!t_host.p) HDDA_CUDA_TRY(cudaMallocHost(&t_host.p, 8 * sizeof(int64_t)));
  *out = t_host.p;
  return HDDA_OK;
}

// The lattice of a parameter set, computed on the device once and cached.
// The first use synchronises `s` (to size the table) and must happen outside
// stream capture.
int get_lattice(const hdda_params& p, cudaStream_t s, LatticeDev* out) {
  int dev = 0;
  HDDA_CUDA_TRY(cudaGetDevice(&dev));
  hdda_params key;
  std::memset(&key, 0, sizeof(key));
  key.near_t = p.near_t; key.far_t = p.far_t; key.step = p.step;
  key.cone_angle = p.cone_angle; key.max_step = p.max_step; key.max_steps = p.max_steps;
  std::lock_guard<std::mutex> lock(g_lattice_mu);
  for (const LatticeEntry& e : g_lattices) {
    if (e.device == dev && same_params(e.key, key)) {
      if (e.status != HDDA_OK)
        return set_error(e.status, "lattice has more than max_steps=%d candidates", p.max_steps);
      *out = LatticeDev{e.t, e.tm, e.K};
      return HDDA_OK;
    }
  }
  int64_t* hw = nullptr;
  int st = host_words(&hw);
  if (st != HDDA_OK) return st;
  int64_t* dk = nullptr;
  HDDA_CUDA_TRY(cudaMallocAsync(&dk, 2 * sizeof(int64_t), s));
  lattice_count_kernel<<<1, 1, 0, s>>>(key, dk);
  HDDA_CUDA_TRY(cudaGetLastError());
  HDDA_CUDA_TRY(cudaMemcpyAsync(hw, dk, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  HDDA_CUDA_TRY(cudaFreeAsync(dk, s));
  HDDA_CUDA_TRY(cudaStreamSynchronize(s));
  LatticeEntry e{key, dev, nullptr, nullptr, (int)hw[0], HDDA_OK};
  if (hw[1]) {
    e.status = HDDA_ERR_STEP_LIMIT;
    g_lattices.push_back(e);
    return set_error(HDDA_ERR_STEP_LIMIT, "lattice has more than max_steps=%d candidates",
                     p.max_steps);
  }
  float* buf = nullptr;
  HDDA_CUDA_TRY(cudaMalloc(&buf, sizeof(float) * (2 * (size_t)e.K + 1)));
  e.t = buf;
  e.tm = buf + e.K + 1;
  lattice_fill_kernel<<<1, 1, 0, s>>>(key, e.K, e.t, e.tm);
  HDDA_CUDA_TRY(cudaGetLastError());
  HDDA_CUDA_TRY(cudaStreamSynchronize(s));  // published to every stream from here on
  g_lattices.push_back(e);
  *out = LatticeDev{e.t, e.tm, e.K};
  return HDDA_OK;
}

int traverse(bool vdb, const float* ro, const float* rd, int64_t n, const hdda_grid* grid,
             const hdda_params* params, int64_t* offsets, int32_t* ray_idx, float* t0, float* t1,
             int64_t capacity, int64_t* total_out, cudaStream_t s) {
  clear_error();
  if (!grid) return set_error(HDDA_ERR_INVALID_ARG, "grid is NULL");
  if (grid->kind != (vdb ? HDDA_GRID_VDB : HDDA_GRID_DENSE))
    return set_error(HDDA_ERR_INVALID_ARG, vdb ? "hdda traversal needs a VDB grid"
                                               : "dense traversal needs a dense grid");
  if (n < 0 || n > INT32_MAX) return set_error(HDDA_ERR_INVALID_ARG, "n_rays=%lld", (long long)n);
  if (!offsets || !total_out) return set_error(HDDA_ERR_INVALID_ARG, "offsets/total_out NULL");
  if (n > 0 && (!ro || !rd)) return set_error(HDDA_ERR_INVALID_ARG, "rays NULL");
  if (capacity < 0) return set_error(HDDA_ERR_INVALID_ARG, "capacity < 0");
  if (capacity > 0 && (!ray_idx || !t0 || !t1))
    return set_error(HDDA_ERR_INVALID_ARG, "sample outputs NULL with capacity > 0");
  int st = validate_params(params);
  if (st != HDDA_OK) return st;
  int dev = 0;
  HDDA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != grid->device)
    return set_error(HDDA_ERR_INVALID_ARG, "grid lives on device %d, current is %d",
                     grid->device, dev);
  LatticeDev lat;
  st = get_lattice(*params, s, &lat);
  if (st != HDDA_OK) return st;
  *total_out = 0;
  if (n == 0) {
    HDDA_CUDA_TRY(cudaMemsetAsync(offsets, 0, sizeof(int64_t), s));
    return HDDA_OK;
  }
  const GridDev g = grid->view();
  const unsigned nb = (unsigned)((n + kBS - 1) / kBS);
  // scratch: [ticket u32, status u32, total i64] + tile_sum[nb] + tile_prefix[nb]
  char* scratch = nullptr;
  HDDA_CUDA_TRY(cudaMallocAsync(&scratch, 16 + 16 * (size_t)nb, s));
  unsigned* ticket = reinterpret_cast<unsigned*>(scratch);
  unsigned* status = ticket + 1;
  int64_t* total = reinterpret_cast<int64_t*>(scratch + 8);
  int64_t* tile_sum = reinterpret_cast<int64_t*>(scratch + 16);
  int64_t* tile_prefix = tile_sum + nb;
  int64_t* hw = nullptr;
  st = host_words(&hw);
  if (st == HDDA_OK) {
    cudaError_t e = cudaMemsetAsync(scratch, 0, 16, s);
    if (e == cudaSuccess) {
      KernelTimer kt(vdb ? "hdda_count" : "dense_count", s);
      if (vdb)
        count_kernel<true><<<nb, kBS, 0, s>>>(ro, rd, n, g, lat, offsets, tile_sum, tile_prefix,
                                              ticket, status, total);
      else
        count_kernel<false><<<nb, kBS, 0, s>>>(ro, rd, n, g, lat, offsets, tile_sum,
                                               tile_prefix, ticket, status, total);
      kt.stop();
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hw, scratch, 16, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_error(e, "count pass");
  }
  if (st == HDDA_OK) {
    const unsigned dev_status = reinterpret_cast<unsigned*>(hw)[1];
    const int64_t tot = hw[1];
    *total_out = tot;
    if (dev_status & kDevInternal) {
      st = set_error(HDDA_ERR_INTERNAL, "region check failed on the device");
    } else if (capacity == 0) {
      KernelTimer kt("offsets", s);
      offsets_kernel<<<nb, kBS, 0, s>>>(n, offsets, tile_prefix, total);
      kt.stop();
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) st = cuda_error(e, "offsets_kernel");
    } else if (capacity < tot) {
      st = set_error(HDDA_ERR_CAPACITY, "capacity %lld < %lld samples", (long long)capacity,
                     (long long)tot);
    } else {
      KernelTimer kt(vdb ? "hdda_emit" : "dense_emit", s);
      if (vdb)
        emit_kernel<true><<<nb, kBS, 0, s>>>(ro, rd, n, g, lat, offsets, tile_prefix, total,
                                             ray_idx, t0, t1, status);
      else
        emit_kernel<false><<<nb, kBS, 0, s>>>(ro, rd, n, g, lat, offsets, tile_prefix, total,
                                              ray_idx, t0, t1, status);
      kt.stop();
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) st = cuda_error(e, "emit_kernel");
    }
  }
  cudaError_t e = cudaFreeAsync(scratch, s);
  if (st == HDDA_OK && e != cudaSuccess) st = cuda_error(e, "cudaFreeAsync");
  return st;
}

}  // namespace

// ---------------------------------------------------------------------------
// traversal over caller-provided scratch (no allocation of any kind)
// ---------------------------------------------------------------------------
// Scratch layout: [0,256) header {ticket u32, status u32, total i64,
// lattice count i64, lattice limit flag i64}; then t[max_k + 1] and
// tm[max_k] floats; then tile_sum[max_tiles] and tile_prefix[max_tiles].

namespace {
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

size_t traverse_scratch_bytes(int max_k, int64_t max_tiles) {
  return 256 + align256(sizeof(float) * (2 * (size_t)max_k + 1)) +
         2 * sizeof(int64_t) * (size_t)max_tiles;
}

int64_t traverse_rays_per_tile() { return kBS; }

int traverse_with_scratch(bool vdb, const float* ro, const float* rd, int64_t n,
                          const hdda_grid* grid, const hdda_params* params, int64_t* offsets,
                          int32_t* ray_idx, float* t0, float* t1, int64_t capacity,
                          int64_t* total_out, void* scratch, int max_k, int64_t max_tiles,
                          cudaStream_t s) {
  clear_error();
  if (!grid) return set_error(HDDA_ERR_INVALID_ARG, "grid is NULL");
  if (grid->kind != (vdb ? HDDA_GRID_VDB : HDDA_GRID_DENSE))
    return set_error(HDDA_ERR_INVALID_ARG, vdb ? "hdda traversal needs a VDB grid"
                                               : "dense traversal needs a dense grid");
  if (n < 0 || n > INT32_MAX) return set_error(HDDA_ERR_INVALID_ARG, "n_rays=%lld", (long long)n);
  const int64_t nb = (n + kBS - 1) / kBS;
  if (nb > max_tiles)
    return set_error(HDDA_ERR_INVALID_ARG,
                     "n_rays=%lld exceeds the static scratch maximum of %lld rays",
                     (long long)n, (long long)(max_tiles * kBS));
  if (!offsets || !total_out) return set_error(HDDA_ERR_INVALID_ARG, "offsets/total_out NULL");
  if (n > 0 && (!ro || !rd)) return set_error(HDDA_ERR_INVALID_ARG, "rays NULL");
  if (capacity < 0) return set_error(HDDA_ERR_INVALID_ARG, "capacity < 0");
  if (capacity > 0 && (!ray_idx || !t0 || !t1))
    return set_error(HDDA_ERR_INVALID_ARG, "sample outputs NULL with capacity > 0");
  if (!scratch) return set_error(HDDA_ERR_INVALID_ARG, "scratch is NULL");
  int st = validate_params(params);
  if (st != HDDA_OK) return st;
  int dev = 0;
  HDDA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != grid->device)
    return set_error(HDDA_ERR_INVALID_ARG, "grid lives on device %d, current is %d",
                     grid->device, dev);
  *total_out = 0;

  char* base = static_cast<char*>(scratch);
  unsigned* ticket = reinterpret_cast<unsigned*>(base);
  unsigned* status = ticket + 1;
  int64_t* total = reinterpret_cast<int64_t*>(base + 8);
  int64_t* lat_words = reinterpret_cast<int64_t*>(base + 16);
  float* lat_t = reinterpret_cast<float*>(base + 256);
  float* lat_tm = lat_t + max_k + 1;
  int64_t* tile_sum =
      reinterpret_cast<int64_t*>(base + 256 + align256(sizeof(float) * (2 * (size_t)max_k + 1)));
  int64_t* tile_prefix = tile_sum + max_tiles;

  // The array keeps the previous call's contents: clear the counters first.
  HDDA_CUDA_TRY(cudaMemsetAsync(base, 0, 32, s));
  hdda_params key;
  std::memset(&key, 0, sizeof(key));
  key.near_t = params->near_t; key.far_t = params->far_t; key.step = params->step;
  key.cone_angle = params->cone_angle; key.max_step = params->max_step;
  key.max_steps = params->max_steps;
  lattice_count_kernel<<<1, 1, 0, s>>>(key, lat_words);
  HDDA_CUDA_TRY(cudaGetLastError());
  int64_t hw[2] = {0, 0};  // pageable host words: no host allocation either
  HDDA_CUDA_TRY(cudaMemcpyAsync(hw, lat_words, sizeof(hw), cudaMemcpyDeviceToHost, s));
  HDDA_CUDA_TRY(cudaStreamSynchronize(s));
  if (hw[1])
    return set_error(HDDA_ERR_STEP_LIMIT, "lattice has more than max_steps=%d candidates",
                     params->max_steps);
  if (hw[0] > max_k)
    return set_error(HDDA_ERR_INVALID_ARG,
                     "lattice of %lld candidates exceeds the static scratch maximum of %d",
                     (long long)hw[0], max_k);
  const LatticeDev lat{lat_t, lat_tm, (int)hw[0]};
  lattice_fill_kernel<<<1, 1, 0, s>>>(key, lat.K, lat_t, lat_tm);
  HDDA_CUDA_TRY(cudaGetLastError());
  if (n == 0) {
    HDDA_CUDA_TRY(cudaMemsetAsync(offsets, 0, sizeof(int64_t), s));
    return HDDA_OK;
  }
  const GridDev g = grid->view();
  if (vdb)
    count_kernel<true><<<(unsigned)nb, kBS, 0, s>>>(ro, rd, n, g, lat, offsets, tile_sum,
                                                    tile_prefix, ticket, status, total);
  else
    count_kernel<false><<<(unsigned)nb, kBS, 0, s>>>(ro, rd, n, g, lat, offsets, tile_sum,
                                                     tile_prefix, ticket, status, total);
  HDDA_CUDA_TRY(cudaGetLastError());
  HDDA_CUDA_TRY(cudaMemcpyAsync(hw, base, 16, cudaMemcpyDeviceToHost, s));
  HDDA_CUDA_TRY(cudaStreamSynchronize(s));
  const unsigned dev_status = reinterpret_cast<unsigned*>(hw)[1];
  const int64_t tot = hw[1];
  *total_out = tot;
  if (dev_status & kDevInternal)
    return set_error(HDDA_ERR_INTERNAL, "region check failed on the device");
  if (capacity == 0) {
    offsets_kernel<<<(unsigned)nb, kBS, 0, s>>>(n, offsets, tile_prefix, total);
    HDDA_CUDA_TRY(cudaGetLastError());
    return HDDA_OK;
  }
  if (capacity < tot)
    return set_error(HDDA_ERR_CAPACITY, "capacity %lld < %lld samples", (long long)capacity,
                     (long long)tot);
  if (vdb)
    emit_kernel<true><<<(unsigned)nb, kBS, 0, s>>>(ro, rd, n, g, lat, offsets, tile_prefix,
                                                   total, ray_idx, t0, t1, status);
  else
    emit_kernel<false><<<(unsigned)nb, kBS, 0, s>>>(ro, rd, n, g, lat, offsets, tile_prefix,
                                                    total, ray_idx, t0, t1, status);
  HDDA_CUDA_TRY(cudaGetLastError());
  return HDDA_OK;
}

}  // namespace hdda

extern "C" int hdda_traverse_dense(const float* rays_o, const float* rays_d, int64_t n_rays,
                                   const hdda_grid* grid, const hdda_params* params,
                                   int64_t* offsets, int32_t* ray_idx, float* t0, float* t1,
                                   int64_t capacity, int64_t* total_out, hdda_stream_t stream) {
  return hdda::traverse(false, rays_o, rays_d, n_rays, grid, params, offsets, ray_idx, t0, t1,
                        capacity, total_out, (cudaStream_t)stream);
}

extern "C" int hdda_traverse_hdda(const float* rays_o, const float* rays_d, int64_t n_rays,
                                  const hdda_grid* grid, const hdda_params* params,
                                  int64_t* offsets, int32_t* ray_idx, float* t0, float* t1,
                                  int64_t capacity, int64_t* total_out, hdda_stream_t stream) {
  return hdda::traverse(true, rays_o, rays_d, n_rays, grid, params, offsets, ray_idx, t0, t1,
                        capacity, total_out, (cudaStream_t)stream);
}
