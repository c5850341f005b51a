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
//            16^3-block node, an empty 32^3 or 16^3 group (refinement), an
//            empty or tiled 8^3 block, an empty or fully occupied 4^3 or 2^3
//            cell (refinement), or a voxel of a leaf; with the refinement,
//            one load from the region map (grid.cu) names it, without the
//            tree is descended per region.  Outside
//            every cascade box the region is a half-space the ray is leaving
//            towards, or everything when it never comes back.
//   cross    the first later lattice point outside the region.  The ray's
//            parameter at the region's exit plane gives an estimate through
//            a bucket index over the lattice; two exact probes confirm it
//            (a gallop and bisection take over when they do not).  Every
//            probe evaluates the point exactly as the definition does.
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
// Launch shapes.  The allocating entry points run, by default, two kernels:
// walk_kernel (persistent warps take 32-ray tiles in order from an atomic
// counter and walk them with the lattice, bucket, threshold and node tables
// staged in shared memory; each ray's sample count and merged occupied runs
// go to global memory, with no CTA barrier anywhere, plus one sum per 32-ray
// tile, also added to sums per 32 and per 1024 tiles) and emit_kernel
// (persistent warps again, one 32-ray tile at a time: the sums of the earlier
// tiles (tile_offset) plus a warp scan give each ray's offset; it writes the
// CSR offsets and expands its rays' runs into (ray, t_k, t_k+1) samples
// through a record list in shared memory, with coalesced 16-byte stores,
// four samples per lane).  With hdda_set_sampler_form(HDDA_SAMPLER_FUSED) one
// kernel, walk_emit_kernel, does the walk and the emit, the offsets coming
// from a decoupled look-back.  The allocation-free entry point runs one
// kernel, onepass_kernel, whose CTAs keep the runs in shared memory and look
// back right after walking, so its scratch stays a few hundred kilobytes.  A
// ray with more runs than are kept walks again and writes its own samples.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "walk.cuh"

namespace hdda {
namespace {

constexpr int kBS = 128;        // rays (threads) per CTA tile
constexpr unsigned kSpinLimit = 1u << 22;  // look-back polls before giving up

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

// Fills t, tm and the bucket index of a lattice block laid out as
// lattice_block_bytes(max_k): t[max_k+1], tm[max_k], kidx[kKidxMax+2], hdr[8].
// One CTA: thread 0 runs the recurrence (it is sequential by definition) and
// sizes the buckets; then every thread fills buckets, each by a binary search
// for the first k with key(tm_k) >= its lower bound (tm is non-decreasing).
constexpr int kFillThreads = 1024;

__global__ void __launch_bounds__(kFillThreads) lattice_fill_kernel(hdda_params p, int K,
                                                                     int max_k,
                                                                     char* __restrict__ block) {
  __shared__ uint32_t s_hdr[3];
  float* t_out = reinterpret_cast<float*>(block);
  float* tm_out = t_out + max_k + 1;
  int* kidx = reinterpret_cast<int*>(tm_out + max_k);
  uint32_t* hdr = reinterpret_cast<uint32_t*>(kidx + kKidxMax + 2);
  if (threadIdx.x == 0) {
    float t = p.near_t;
    t_out[0] = t;
    for (int k = 0; k < K; ++k) {
      const float tn = lattice_next(t, p);
      t_out[k + 1] = tn;
      tm_out[k] = __fmul_rn(__fadd_rn(t, tn), 0.5f);
      t = tn;
    }
    uint32_t key0 = 0, shift = 0;
    int NB = 0;
    if (K > 0) {
      key0 = float_key(tm_out[0]);
      const uint32_t range = float_key(tm_out[K - 1]) - key0;
      while ((range >> shift) >= (uint32_t)kKidxMax) ++shift;
      NB = (int)(range >> shift) + 1;
    }
    s_hdr[0] = key0;
    s_hdr[1] = shift;
    s_hdr[2] = (uint32_t)NB;
    hdr[0] = key0;
    hdr[1] = shift;
    hdr[2] = (uint32_t)NB;
    // A closed form for the walk's index estimates, used instead of the buckets
    // when it holds: form 1, the spacing is constant; form 2, it is the constant
    // step up to index ks and then grows geometrically (Delta t = t * cone, so t
    // and tm gain a factor 1 + cone per index), with the cap max_step never
    // binding.  A = 1 / log2(1 + cone).
    uint32_t form = 0;
    int ks = K;
    float A = 0.f;
    if (K > 0) {
      if (p.cone_angle == 0.f || p.max_step <= p.step) {
        form = 1;  // constant spacing throughout
      } else if (__fmul_rn(t_out[K], p.cone_angle) <= p.max_step) {
        ks = 0;
        while (ks < K && !(__fmul_rn(t_out[ks], p.cone_angle) > p.step)) ++ks;
        form = ks < K ? 2 : 1;
        A = (float)(0.69314718055994531 / log1p((double)p.cone_angle));
      }
    }
    hdr[3] = form;
    hdr[4] = (uint32_t)ks;
    hdr[5] = __float_as_uint(A);
  }
  __syncthreads();  // thread 0's table is visible to the block from here on
  if (K == 0) {
    if (threadIdx.x == 0) kidx[0] = kidx[1] = 0;
    return;
  }
  const uint32_t key0 = s_hdr[0], shift = s_hdr[1];
  const int NB = (int)s_hdr[2];
  for (int b = threadIdx.x; b <= NB; b += blockDim.x) {
    const uint64_t bound = (uint64_t)key0 + ((uint64_t)b << shift);
    int lo = 0, hi = K;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((uint64_t)float_key(tm_out[mid]) < bound) lo = mid + 1;
      else hi = mid;
    }
    kidx[b] = lo;
  }
  if (threadIdx.x == 0) kidx[NB + 1] = K;
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

// ---------------------------------------------------------------------------
// decoupled look-back over tiles
// ---------------------------------------------------------------------------

// State words: the top two bits flag the value as the tile's own sample
// total (its aggregate) or as its inclusive prefix.
constexpr unsigned long long kFlagAggregate = 1ull << 62;
constexpr unsigned long long kFlagPrefix = 2ull << 62;
constexpr unsigned long long kValueMask = (1ull << 62) - 1;


__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// True (on every lane) once some wait of the launch has run out of polls:
// checked every 1024 polls, so that after one timeout the other waits end
// at once instead of each running out in turn.
__device__ __forceinline__ bool gave_up(const unsigned* status, unsigned polls) {
  if (polls & 1023u) return false;
  unsigned v = 0;
  if ((threadIdx.x & 31) == 0) v = *reinterpret_cast<const volatile unsigned*>(status);
  return (__shfl_sync(kFull, v, 0) & kDevTimeout) != 0;
}

// Sums the aggregates of the tiles before `tile` back to the first published
// prefix, publishes the inclusive prefix (excl + agg) and returns the
// exclusive one.  Called by one whole warp, which reads 32 predecessors per
// poll, once the tile's own aggregate is published.  Every predecessor tile
// was handed out earlier and publishes its aggregate without waiting for
// any other tile, so each wait ends; the poll count is still bounded, and
// running out of it raises kDevTimeout (the host then reports
// HDDA_ERR_TIMEOUT) and publishes what it has so that later tiles finish.
__device__ int64_t lookback_prefix(unsigned long long* state, int tile, int64_t agg,
                                   unsigned* status) {
  const int lane = threadIdx.x & 31;
  if (tile == 0) {
    if (lane == 0) st_release(state, kFlagPrefix | (unsigned long long)agg);
    return 0;
  }
  int64_t excl = 0;
  int base = tile - 1;  // lane i looks at tile base - i
  unsigned polls = 0;
  for (;;) {
    const int j = base - lane;
    const unsigned long long w = j >= 0 ? ld_acquire(state + j) : kFlagPrefix;
    const unsigned long long f = w & ~kValueMask;
    const unsigned pmask = __ballot_sync(kFull, f == kFlagPrefix);
    const unsigned zmask = __ballot_sync(kFull, f == 0);
    const int first_p = pmask ? __ffs(pmask) - 1 : 32;  // nearest published prefix
    const unsigned need = first_p >= 31 ? kFull : ((2u << first_p) - 1u);
    if (zmask & need) {  // a tile this one depends on has not published yet
      if (++polls > kSpinLimit || gave_up(status, polls)) {
        if (lane == 0) atomicOr(status, kDevTimeout);
        break;
      }
      __nanosleep(64);
      continue;
    }
    int64_t v = lane <= first_p ? (int64_t)(w & kValueMask) : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    excl += v;
    if (first_p < 32) break;
    base -= 32;
  }
  if (lane == 0) st_release(state + tile, kFlagPrefix | (unsigned long long)(excl + agg));
  return excl;
}

// Publishes this tile's aggregate, then looks back (lookback_prefix).
__device__ int64_t lookback(unsigned long long* state, int tile, int64_t agg,
                            unsigned* status) {
  if (tile != 0 && (threadIdx.x & 31) == 0)
    st_release(state + tile, kFlagAggregate | (unsigned long long)agg);
  return lookback_prefix(state, tile, agg, status);
}

// Waits (bounded, as lookback_prefix) until the tile's aggregate is
// published and returns it.  Every lane acquires the word itself, so the
// tile's counts and runs, stored before the release, are visible to each.
__device__ int64_t wait_aggregate(const unsigned long long* state, int tile, unsigned* status) {
  unsigned polls = 0;
  for (;;) {
    const unsigned long long w = ld_acquire(state + tile);
    if (__all_sync(kFull, (w & ~kValueMask) != 0)) return (int64_t)(w & kValueMask);
    if (++polls > kSpinLimit || gave_up(status, polls)) {
      if ((threadIdx.x & 31) == 0) atomicOr(status, kDevTimeout);
      return 0;
    }
    __nanosleep(64);
  }
}

// ---------------------------------------------------------------------------
// one-pass sampler (bounded scratch: runs stay in shared memory)
// ---------------------------------------------------------------------------

template <int kMode>
__global__ void __launch_bounds__(kBS) onepass_kernel(
    const float* __restrict__ ro, const float* __restrict__ rd, int64_t n, GridDev g,
    LatticeDev lat, int64_t* __restrict__ offsets, int32_t* __restrict__ ray_idx,
    float* __restrict__ t0, float* __restrict__ t1, int64_t capacity,
    unsigned long long* __restrict__ tile_state, unsigned* __restrict__ tile_counter,
    unsigned* __restrict__ status, int64_t* __restrict__ total_out) {
  __shared__ uint2 s_runs[kMaxRuns * kBS];
  __shared__ int s_tile;
  __shared__ int64_t s_prefix;
  if (threadIdx.x == 0) s_tile = (int)atomicAdd(tile_counter, 1u);
  __syncthreads();
  const int tile = s_tile;
  const int64_t r = (int64_t)tile * kBS + threadIdx.x;
  const LatHdr h = lat_hdr(lat);

  Ray ray;
  bool valid = false;
  int64_t c = 0;
  int nruns = 0;
  if (r < n) {
    valid = load_ray(ro, rd, r, ray);
    if (valid)
      c = walk<kMode, false, false>(g, global_tabs(g), lat, h, ray, s_runs + threadIdx.x, kBS,
                                   nruns, 0, 0, 0, nullptr, nullptr, nullptr, status);
  }
  int64_t agg = 0;
  const int64_t local = cta_exclusive_scan64(c, &agg);
  if (threadIdx.x < 32) {
    const int64_t pre = lookback(tile_state, tile, agg, status);
    if (threadIdx.x == 0) s_prefix = pre;
  }
  __syncthreads();
  const int64_t off = s_prefix + local;
  // offsets are clamped to the sample buffer when it is too small (as in the
  // two-pass emit); the total is reported unclamped
  const int64_t cap = capacity > 0 ? capacity : INT64_MAX;
  if (r < n) offsets[r] = min(off, cap);
  if (tile == (int)gridDim.x - 1 && threadIdx.x == kBS - 1) {
    offsets[n] = min(off + c, cap);
    *total_out = off + c;
  }
  if (capacity <= 0) return;
  const int warp = threadIdx.x >> 5;
  const bool overflow = nruns > kMaxRuns;
  expand_warp<true>(off, c, overflow, s_runs + warp * 32, kBS,
                    (int32_t)((int64_t)tile * kBS + warp * 32), lat.t, capacity, ray_idx, t0, t1);
  if (overflow && valid) {
    int unused = 0;
    walk<kMode, true, false>(g, global_tabs(g), lat, h, ray, nullptr, 0, unused, (int32_t)r, off,
                            capacity, ray_idx, t0, t1, status);
  }
}

// ---------------------------------------------------------------------------
// two-pass sampler: walk (persistent warps, staged tables), then emit
// ---------------------------------------------------------------------------

constexpr int kEmitWarps = 4;

// Pass 2 for one 32-ray tile, independent of every other tile: its offset
// is the sum of the earlier tiles' samples (tile_offset, from the group sums
// the walk kept) plus a warp scan; its runs become a record list in shared
// memory (rec: kRecMax records and a sentinel) that expand_records turns into
// samples.  A ray with more runs than were kept walks again.  The last tile
// writes the total.
template <int kMode>
__device__ __forceinline__ void emit_tile(
    int64_t tile, unsigned T, uint2* rec, const float* __restrict__ ro,
    const float* __restrict__ rd, int64_t n, const GridDev& g, const LatticeDev& lat,
    const int32_t* __restrict__ counts, const uint8_t* __restrict__ nruns,
    const uint2* __restrict__ runs, const int64_t* __restrict__ tile_sum,
    const unsigned long long* __restrict__ sums32,
    const unsigned long long* __restrict__ sums1024, int64_t* __restrict__ offsets,
    int32_t* __restrict__ ray_idx, float* __restrict__ t0, float* __restrict__ t1,
    int64_t capacity, bool vec, int64_t* __restrict__ total, unsigned* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  const int64_t r = tile * 32 + lane;
  const int c = r < n ? counts[r] : 0;
  const int nr = r < n ? (int)nruns[r] : 0;
  const int64_t wbeg = tile_offset(tile, tile_sum, sums32, sums1024);
  // a tile holds at most 32 * 2^24 samples: 32-bit positions within it
  int inc = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += y;
  }
  const int q = inc - c;
  const int tot = __shfl_sync(kFull, inc, 31);
  const int64_t off = wbeg + q;
  if (tile == (int64_t)T - 1 && lane == 0) *total = wbeg + tot;
  if (capacity > 0) {
    // with too small a buffer the CSR offsets are clamped to it, so that a
    // consumer of the arrays stays in bounds; the status says what happened
    if (r < n) offsets[r] = min(off, capacity);
    if (r == n - 1) offsets[n] = min(off + c, capacity);
    if (wbeg + tot > capacity && lane == 0) atomicOr(status, kDevCapacity);
  } else {
    if (r < n) offsets[r] = off;
    if (r == n - 1) offsets[n] = off + c;
    return;
  }
  const int kept = c <= 0 ? 0 : nr > kMaxRuns ? 1 : nr;
  int kinc = kept;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, kinc, o);
    if (lane >= o) kinc += y;
  }
  const int nrec = __shfl_sync(kFull, kinc, 31);
  list_runs(rec, kinc - kept, lane, nr, c, (uint32_t)q, runs + r, n);
  if (lane == 0) rec[nrec] = make_uint2(kRecEnd, 0u);
  __syncwarp();
  const int64_t room = capacity - wbeg;
  const int lim = room <= 0 ? 0 : (int)min((int64_t)tot, room);
  expand_records(rec, nrec, lim, wbeg, (int32_t)(tile * 32), lat.t, vec, ray_idx, t0, t1);
  if (nr > kMaxRuns) {
    Ray ray;
    load_ray(ro, rd, r, ray);
    const LatHdr h = lat_hdr(lat);
    int unused = 0;
    walk<kMode, true, false>(g, global_tabs(g), lat, h, ray, nullptr, 0, unused, (int32_t)r, off,
                             capacity, ray_idx, t0, t1, status);
  }
}

// Pass 2.  Persistent: each warp takes 32-ray tiles from an atomic counter
// until none is left, so a warp that finishes early takes more tiles
// instead of idling until its CTA's slowest tile is done.  (Taking the next
// tile and loading its counts before expanding the current one measured 5-14 %
// slower: tiles held by busy warps lengthen the tail.)
template <int kMode>
__global__ void __launch_bounds__(kEmitWarps * 32, 7) emit_kernel(
    const float* __restrict__ ro, const float* __restrict__ rd, int64_t n, GridDev g,
    LatticeDev lat, const int32_t* __restrict__ counts, const uint8_t* __restrict__ nruns,
    const uint2* __restrict__ runs, const int64_t* __restrict__ tile_sum,
    const unsigned long long* __restrict__ sums32,
    const unsigned long long* __restrict__ sums1024, int64_t* __restrict__ offsets,
    int32_t* __restrict__ ray_idx, float* __restrict__ t0, float* __restrict__ t1,
    int64_t capacity, bool vec, unsigned* __restrict__ tile_counter, int64_t* __restrict__ total,
    unsigned* __restrict__ status) {
  __shared__ uint2 s_rec[kEmitWarps][kRecMax + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned T = (unsigned)((n + 31) / 32);
  for (;;) {
    unsigned tile = 0;
    if (lane == 0) tile = atomicAdd(tile_counter, 1u);
    tile = __shfl_sync(kFull, tile, 0);
    if (tile >= T) break;
    emit_tile<kMode>(tile, T, s_rec[warp], ro, rd, n, g, lat, counts, nruns, runs, tile_sum,
                     sums32, sums1024, offsets, ray_idx, t0, t1, capacity, vec, total, status);
    __syncwarp();  // the next tile reuses this warp's shared memory
  }
}

// Resident CTAs of the persistent emit: one wave, or fewer for small calls.
template <int kMode>
unsigned emit_grid(int64_t T) {
  int dev = 0, sms = 1, per_sm = 1;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, emit_kernel<kMode>,
                                                    kEmitWarps * 32, 0) != cudaSuccess ||
      per_sm <= 0)
    per_sm = 1;
  const int64_t want = (T + kEmitWarps - 1) / kEmitWarps;
  const int64_t full = (int64_t)(sms > 0 ? sms : 1) * per_sm;
  return (unsigned)(want < full ? want : full);
}

// ---------------------------------------------------------------------------
// fused sampler: the walk and the emit in one persistent kernel
// ---------------------------------------------------------------------------
//
// Phase 1: each warp walks 32-ray tiles (as walk_kernel: counts, run counts
// and runs to global memory) and publishes each tile's sample total as its
// aggregate in the decoupled look-back's state word.  Phase 2, once every
// tile has been handed out: warps take tiles to write out, in tile order.
// Writing out = waiting for the tile's aggregate, looking back for its
// exclusive prefix, writing the CSR offsets and expanding the runs through a
// per-warp record list in shared memory (expand_records).  Warps whose walks
// end early thus write out the first tiles while the last ones are still
// walked, and no scan or emit launch follows.
//
// No wait can last forever: a walk publishes its aggregate without waiting
// for anything, every tile has been handed out to a running warp before
// phase 2 begins anywhere, and the waits themselves are bounded
// (kDevTimeout).

// Shared memory of the fused kernel: the staged tables (kSm), then one
// record list (kRecMax records and the sentinel) per warp.
__host__ __device__ inline size_t walk_emit_smem(size_t stage_bytes) {
  return stage_bytes + (size_t)(kWalkBS / 32) * (kRecMax + 1) * sizeof(uint2);
}

// Writes out tile e: its CSR offsets and, below `capacity`, its samples.
template <int kMode, bool kSm>
__device__ __forceinline__ void emit_fused_tile(
    int e, uint2* rec, const float* __restrict__ ro, const float* __restrict__ rd, int64_t n,
    unsigned T, const GridDev& g, const Tabs& tb, const LatticeDev& ls, const LatHdr& h,
    const int32_t* counts, const uint8_t* nruns, const uint2* runs, unsigned long long* state,
    int64_t* __restrict__ offsets, int32_t* __restrict__ ray_idx, float* __restrict__ t0,
    float* __restrict__ t1, int64_t capacity, bool vec, int64_t* __restrict__ total,
    unsigned* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  const int64_t agg = wait_aggregate(state, e, status);
  const int64_t excl = lookback_prefix(state, e, agg, status);
  const int64_t r = (int64_t)e * 32 + lane;
  // written in this kernel by another warp: read through L2 (after the acquire)
  const int c = r < n ? __ldcg(counts + r) : 0;
  const int nr = r < n ? (int)__ldcg(nruns + r) : 0;
  // a tile holds at most 32 * 2^24 samples: 32-bit positions within it
  int inc = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += y;
  }
  const int q = inc - c;  // this ray's first position within the tile
  const int tot = __shfl_sync(kFull, inc, 31);
  const int64_t off = excl + q;
  if (capacity > 0) {
    // with too small a buffer the CSR offsets are clamped to it, so that a
    // consumer of the arrays stays in bounds; the status says what happened
    if (r < n) offsets[r] = min(off, capacity);
    if (r == n - 1) offsets[n] = min(off + c, capacity);
    if (excl + tot > capacity && lane == 0) atomicOr(status, kDevCapacity);
  } else {
    if (r < n) offsets[r] = off;
    if (r == n - 1) offsets[n] = off + c;
  }
  if (e == (int)T - 1 && lane == 0) *total = excl + tot;
  if (capacity <= 0) return;
  // the record list: an exclusive scan of the lanes' record counts
  const int kept = c <= 0 ? 0 : nr > kMaxRuns ? 1 : nr;
  int kinc = kept;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, kinc, o);
    if (lane >= o) kinc += y;
  }
  const int nrec = __shfl_sync(kFull, kinc, 31);
  list_runs(rec, kinc - kept, lane, nr, c, (uint32_t)q, runs + r, n);
  if (lane == 0) rec[nrec] = make_uint2(kRecEnd, 0u);
  __syncwarp();
  const int64_t room = capacity - excl;
  const int lim = room <= 0 ? 0 : (int)min((int64_t)tot, room);
  expand_records(rec, nrec, lim, excl, (int32_t)((int64_t)e * 32), ls.t, vec, ray_idx, t0, t1);
  __syncwarp();  // the next tile reuses rec
  if (nr > kMaxRuns) {
    Ray ray;
    load_ray(ro, rd, r, ray);
    int unused = 0;
    walk<kMode, true, kSm>(g, tb, ls, h, ray, nullptr, 0, unused, (int32_t)r, off, capacity,
                           ray_idx, t0, t1, status);
  }
}

template <int kMode, bool kSm, bool kSkip, bool kCheck>
__global__ void __launch_bounds__(kWalkBS) walk_emit_kernel(
    const float* __restrict__ ro, const float* __restrict__ rd, int64_t n, GridDev g,
    LatticeDev lat, int32_t* counts, uint8_t* nruns_out, uint2* runs,
    unsigned long long* state, unsigned* __restrict__ walk_counter,
    unsigned* __restrict__ emit_counter, int64_t* __restrict__ offsets,
    int32_t* __restrict__ ray_idx, float* __restrict__ t0, float* __restrict__ t1,
    int64_t capacity, bool vec, int64_t* __restrict__ total, unsigned* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem[];
  const LatHdr h = lat_hdr(lat);
  Tabs tb = global_tabs(g);
  LatticeDev ls = lat;
  size_t stage_bytes = 0;
  if constexpr (kSm) {
    const int64_t nodes = (int64_t)g.L * g.N * g.N * g.N;
    stage_bytes = stage_layout(lat.K, g.L, g.R, nodes, kMode).bytes;
    stage_walk_tables<kMode>(smem, g, lat, h, tb, ls);
    __syncthreads();
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint2* rec = reinterpret_cast<uint2*>(smem + stage_bytes) + warp * (kRecMax + 1);
  const unsigned T = (unsigned)((n + 31) / 32);
  for (;;) {  // phase 1: walk tiles until none is left
    unsigned tile = 0;
    if (lane == 0) tile = atomicAdd(walk_counter, 1u);
    tile = __shfl_sync(kFull, tile, 0);
    if (tile >= T) break;
    const int64_t r = (int64_t)tile * 32 + lane;
    int64_t c = 0;
    if (r < n) {
      Ray ray;
      int nr = 0;
      if (load_ray(ro, rd, r, ray))
        c = walk<kMode, false, kSm, kSkip, kCheck>(g, tb, ls, h, ray, runs + r, n, nr, 0, 0, 0,
                                                  nullptr, nullptr, nullptr, status);
      counts[r] = (int32_t)c;
      nruns_out[r] = (uint8_t)min(nr, 255);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    __syncwarp();  // orders every lane's counts and runs before lane 0's release
    if (lane == 0) st_release(state + tile, kFlagAggregate | (unsigned long long)c);
  }
  for (;;) {  // phase 2: every tile is handed out; write tiles out in order
    unsigned e = 0;
    if (lane == 0) e = atomicAdd(emit_counter, 1u);
    e = __shfl_sync(kFull, e, 0);
    if (e >= T) break;
    emit_fused_tile<kMode, kSm>((int)e, rec, ro, rd, n, T, g, tb, ls, h, counts, nruns_out, runs,
                                state, offsets, ray_idx, t0, t1, capacity, vec, total, status);
  }
}

template <int kMode, bool kSm, bool kSkip>
int launch_walk_emit(const WalkArgs& w, size_t stage, unsigned long long* state,
                     unsigned* emit_counter, int64_t* offsets, int32_t* ray_idx, float* t0,
                     float* t1, int64_t capacity, bool vec, int64_t* total, cudaStream_t s) {
  auto kern = w.g.check ? walk_emit_kernel<kMode, kSm, kSkip, true>
                        : walk_emit_kernel<kMode, kSm, kSkip, false>;
  const size_t smem = walk_emit_smem(kSm ? stage : 0);
  HDDA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
  int dev = 0, sms = 0, per_sm = 0;
  HDDA_CUDA_TRY(cudaGetDevice(&dev));
  HDDA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HDDA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWalkBS, smem));
  if (per_sm <= 0) return set_error(HDDA_ERR_INTERNAL, "fused sampler does not fit an SM");
  // as the walk: one resident wave, at most one CTA per eight 32-ray tiles
  const int64_t want = ((w.n + 31) / 32 + 7) / 8;
  const int64_t full = (int64_t)sms * per_sm;
  const unsigned grid = (unsigned)(want < full ? want : full);
  kern<<<grid, kWalkBS, smem, s>>>(w.ro, w.rd, w.n, w.g, w.lat, w.counts, w.nruns, w.runs, state,
                                   w.counter, emit_counter, offsets, ray_idx, t0, t1, capacity,
                                   vec, total, w.status);
  HDDA_CUDA_TRY(cudaGetLastError());
  return HDDA_OK;
}

template <int kMode>
int launch_walk_emit_mode(const WalkArgs& w, size_t stage, bool skip, unsigned long long* state,
                          unsigned* emit_counter, int64_t* offsets, int32_t* ray_idx, float* t0,
                          float* t1, int64_t capacity, bool vec, int64_t* total,
                          cudaStream_t s) {
  const bool sm = stage <= kMaxStageBytes;
  if (skip)
    return sm ? launch_walk_emit<kMode, true, true>(w, stage, state, emit_counter, offsets,
                                                   ray_idx, t0, t1, capacity, vec, total, s)
              : launch_walk_emit<kMode, false, true>(w, stage, state, emit_counter, offsets,
                                                    ray_idx, t0, t1, capacity, vec, total, s);
  return sm ? launch_walk_emit<kMode, true, false>(w, stage, state, emit_counter, offsets,
                                                  ray_idx, t0, t1, capacity, vec, total, s)
            : launch_walk_emit<kMode, false, false>(w, stage, state, emit_counter, offsets,
                                                   ray_idx, t0, t1, capacity, vec, total, s);
}

const char* walk_emit_name(int mode) {
  return mode == kModeDense ? "dense_walk_emit"
         : mode == kModeVdb ? "hdda_walk_emit_plain" : "hdda_walk_emit";
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct LatticeEntry {
  hdda_params key;
  int device;
  char* block;
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
  if (p->image_width < 0)
    return set_error(HDDA_ERR_INVALID_ARG, "image_width=%d < 0", p->image_width);
  return HDDA_OK;
}

hdda_params canonical(const hdda_params& p) {
  hdda_params key;
  std::memset(&key, 0, sizeof(key));
  key.near_t = p.near_t; key.far_t = p.far_t; key.step = p.step;
  key.cone_angle = p.cone_angle; key.max_step = p.max_step; key.max_steps = p.max_steps;
  return key;
}

// Pinned host words for the read-backs of the allocating path.
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
  const hdda_params key = canonical(p);
  std::lock_guard<std::mutex> lock(g_lattice_mu);
  for (const LatticeEntry& e : g_lattices) {
    if (e.device == dev && same_params(e.key, key)) {
      if (e.status != HDDA_OK)
        return set_error(e.status, "lattice has more than max_steps=%d candidates", p.max_steps);
      *out = lattice_view(e.block, e.K, e.K);
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
  LatticeEntry e{key, dev, nullptr, (int)hw[0], HDDA_OK};
  if (hw[1]) {
    e.status = HDDA_ERR_STEP_LIMIT;
    g_lattices.push_back(e);
    return set_error(HDDA_ERR_STEP_LIMIT, "lattice has more than max_steps=%d candidates",
                     p.max_steps);
  }
  HDDA_CUDA_TRY(cudaMalloc(&e.block, lattice_block_bytes(e.K)));
  lattice_fill_kernel<<<1, kFillThreads, 0, s>>>(key, e.K, e.K, e.block);
  HDDA_CUDA_TRY(cudaGetLastError());
  HDDA_CUDA_TRY(cudaStreamSynchronize(s));  // published to every stream from here on
  g_lattices.push_back(e);
  *out = lattice_view(e.block, e.K, e.K);
  return HDDA_OK;
}

int check_args(bool vdb, const float* ro, const float* rd, int64_t n, const hdda_grid* grid,
               const hdda_params* params, int64_t* offsets, int32_t* ray_idx, float* t0,
               float* t1, int64_t capacity, int64_t* total_out) {
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
  return HDDA_OK;
}

// Reads the header words {.., status, total} back and turns them into a status.
int finish(int64_t* hw, const char* header, int64_t capacity, int64_t* total_out,
           cudaStream_t s) {
  HDDA_CUDA_TRY(cudaMemcpyAsync(hw, header, 16, cudaMemcpyDeviceToHost, s));
  HDDA_CUDA_TRY(cudaStreamSynchronize(s));
  const unsigned dev_status = reinterpret_cast<unsigned*>(hw)[1];
  const int64_t tot = hw[1];
  *total_out = tot;
  if (dev_status & kDevInternal)
    return set_error(HDDA_ERR_INTERNAL, "region check failed on the device");
  if (dev_status & kDevTimeout)
    return set_error(HDDA_ERR_TIMEOUT, "tile look-back gave up waiting");
  if (capacity > 0 && capacity < tot)
    return set_error(HDDA_ERR_CAPACITY, "capacity %lld < %lld samples", (long long)capacity,
                     (long long)tot);
  return HDDA_OK;
}

// One-pass launch over scratch = [32-byte header | tile states]:
// header = {tile counter u32, status u32, total i64}.
int run_onepass(const float* ro, const float* rd, int64_t n, const hdda_grid* grid,
                const LatticeDev& lat, int64_t* offsets, int32_t* ray_idx, float* t0, float* t1,
                int64_t capacity, int64_t* total_out, char* scratch, int64_t* hw,
                cudaStream_t s) {
  const unsigned nb = (unsigned)((n + kBS - 1) / kBS);
  unsigned* counter = reinterpret_cast<unsigned*>(scratch);
  unsigned* status = counter + 1;
  int64_t* total = reinterpret_cast<int64_t*>(scratch + 8);
  unsigned long long* state = reinterpret_cast<unsigned long long*>(scratch + 32);
  HDDA_CUDA_TRY(cudaMemsetAsync(scratch, 0, 32 + 8 * (size_t)nb, s));
  const GridDev g = grid->view();
  switch (walk_mode(grid)) {
    case kModeDense:
      onepass_kernel<kModeDense><<<nb, kBS, 0, s>>>(ro, rd, n, g, lat, offsets, ray_idx, t0, t1,
                                                    capacity, state, counter, status, total);
      break;
    case kModeVdb:
      onepass_kernel<kModeVdb><<<nb, kBS, 0, s>>>(ro, rd, n, g, lat, offsets, ray_idx, t0, t1,
                                                  capacity, state, counter, status, total);
      break;
    default:
      onepass_kernel<kModeVdbMap><<<nb, kBS, 0, s>>>(ro, rd, n, g, lat, offsets, ray_idx, t0,
                                                         t1, capacity, state, counter, status,
                                                         total);
      break;
  }
  HDDA_CUDA_TRY(cudaGetLastError());
  return finish(hw, scratch, capacity, total_out, s);
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr size_t kTwopassHead = 256;

// Bytes of the two-pass scratch for n rays.
size_t twopass_scratch_bytes(int64_t n) {
  const int64_t T = (n + 31) / 32;
  return kTwopassHead + 2 * a256(8 * (size_t)T) + a256(4 * (size_t)n) + a256((size_t)n) +
         a256(sizeof(uint2) * kMaxRuns * (size_t)n);
}

const char* emit_name(int mode) {
  return mode == kModeDense ? "dense_emit" : mode == kModeVdb ? "hdda_emit_plain" : "hdda_emit";
}

// Two-pass launch.  Scratch: [0, 256) header {walk counter u32, status u32,
// total i64, emit counter u32}, then tile sums, the walk's group sums (per 32
// and per 1024 tiles), counts, run counts, runs.  The separate form (the
// default) runs the walk and the emit, which takes each tile's offset from
// the tile and group sums (no scan kernel in between); the fused form runs
// both passes in one kernel (walk_emit_kernel), whose look-back states take
// the tile sums' space.
int run_twopass(const float* ro, const float* rd, int64_t n, const hdda_grid* grid,
                const LatticeDev& lat, int32_t width, int64_t* offsets, int32_t* ray_idx,
                float* t0, float* t1, int64_t capacity, int64_t* total_out, char* scratch,
                int64_t* hw, unsigned* dev_status, cudaStream_t s) {
  const int64_t T = (n + 31) / 32;
  unsigned* walk_counter = reinterpret_cast<unsigned*>(scratch);
  unsigned* status = dev_status ? dev_status : walk_counter + 1;
  int64_t* total = reinterpret_cast<int64_t*>(scratch + 8);
  unsigned* emit_counter = reinterpret_cast<unsigned*>(scratch + 16);
  // region A (after the header): the group sums of the separate form,
  // ceil(T / 32) per 32 tiles then ceil(T / 1024) per 1024 tiles, or the
  // look-back states of the fused form; region B: the tile sums.  Both forms
  // clear the header and what they use of region A with one memset.
  char* p = scratch + kTwopassHead;
  const int64_t G32 = (T + 31) / 32, G1024 = (T + 1023) / 1024;
  unsigned long long* sums32 = reinterpret_cast<unsigned long long*>(p);
  unsigned long long* sums1024 = sums32 + G32;
  unsigned long long* state = sums32;
  p += a256(8 * (size_t)T);
  int64_t* tile_sum = reinterpret_cast<int64_t*>(p);
  p += a256(8 * (size_t)T);
  int32_t* counts = reinterpret_cast<int32_t*>(p);
  p += a256(4 * (size_t)n);
  uint8_t* nruns = reinterpret_cast<uint8_t*>(p);
  p += a256((size_t)n);
  uint2* runs = reinterpret_cast<uint2*>(p);
  const int mode = walk_mode(grid);
  WalkArgs w{ro, rd, n, grid->view(), lat, counts, nruns, runs, tile_sum, walk_counter,
             status};
  const size_t stage = stage_layout(lat.K, w.g.L, w.g.R, grid->nodes_total(), mode).bytes;
  const bool skip = grid->walk_variant == HDDA_WALK_SKIP;
  const bool vec = ((reinterpret_cast<uintptr_t>(ray_idx) | reinterpret_cast<uintptr_t>(t0) |
                     reinterpret_cast<uintptr_t>(t1)) & 15) == 0;
  if (sampler_form() == HDDA_SAMPLER_FUSED) {
    HDDA_CUDA_TRY(cudaMemsetAsync(scratch, 0, kTwopassHead + 8 * (size_t)T, s));
    KernelTimer kt(walk_emit_name(mode), s);
    const int st =
        mode == kModeDense
            ? launch_walk_emit_mode<kModeDense>(w, stage, skip, state, emit_counter, offsets,
                                                ray_idx, t0, t1, capacity, vec, total, s)
        : mode == kModeVdb
            ? launch_walk_emit_mode<kModeVdb>(w, stage, skip, state, emit_counter, offsets,
                                              ray_idx, t0, t1, capacity, vec, total, s)
            : launch_walk_emit_mode<kModeVdbMap>(w, stage, skip, state, emit_counter, offsets,
                                                 ray_idx, t0, t1, capacity, vec, total, s);
    if (st != HDDA_OK) return st;
    kt.stop();
    if (dev_status) return HDDA_OK;  // stream-ordered: nothing is read back
    return finish(hw, scratch, capacity, total_out, s);
  }
  // a walk in pixel blocks adds the tile sums up atomically: region B is
  // cleared too (it follows region A)
  w.width = (int32_t)std::min<int64_t>(width, n);
  HDDA_CUDA_TRY(cudaMemsetAsync(
      scratch, 0,
      w.width > 0 ? kTwopassHead + a256(8 * (size_t)T) + 8 * (size_t)T
                  : kTwopassHead + 8 * (size_t)(G32 + G1024),
      s));
  w.sums32 = sums32;
  w.sums1024 = sums1024;
  {
    KernelTimer kt(walk_name(mode), s);
    const int st = mode == kModeDense ? launch_walk_mode<kModeDense>(w, stage, skip, s)
                   : mode == kModeVdb ? launch_walk_mode<kModeVdb>(w, stage, skip, s)
                                      : launch_walk_mode<kModeVdbMap>(w, stage, skip, s);
    if (st != HDDA_OK) return st;
  }
  {
    KernelTimer kt(emit_name(mode), s);
    switch (mode) {
      case kModeDense:
        emit_kernel<kModeDense><<<emit_grid<kModeDense>(T), kEmitWarps * 32, 0, s>>>(
            ro, rd, n, w.g, lat, counts, nruns, runs, tile_sum, sums32, sums1024, offsets,
            ray_idx, t0, t1, capacity, vec, emit_counter, total, status);
        break;
      case kModeVdb:
        emit_kernel<kModeVdb><<<emit_grid<kModeVdb>(T), kEmitWarps * 32, 0, s>>>(
            ro, rd, n, w.g, lat, counts, nruns, runs, tile_sum, sums32, sums1024, offsets,
            ray_idx, t0, t1, capacity, vec, emit_counter, total, status);
        break;
      default:
        emit_kernel<kModeVdbMap><<<emit_grid<kModeVdbMap>(T), kEmitWarps * 32, 0, s>>>(
            ro, rd, n, w.g, lat, counts, nruns, runs, tile_sum, sums32, sums1024, offsets,
            ray_idx, t0, t1, capacity, vec, emit_counter, total, status);
        break;
    }
  }
  HDDA_CUDA_TRY(cudaGetLastError());
  if (dev_status) return HDDA_OK;  // stream-ordered: nothing is read back
  return finish(hw, scratch, capacity, total_out, s);
}

int traverse(bool vdb, const float* ro, const float* rd, int64_t n, const hdda_grid* grid,
             const hdda_params* params, int64_t* offsets, int32_t* ray_idx, float* t0, float* t1,
             int64_t capacity, int64_t* total_out, cudaStream_t s) {
  clear_error();
  int st = check_args(vdb, ro, rd, n, grid, params, offsets, ray_idx, t0, t1, capacity,
                      total_out);
  if (st != HDDA_OK) return st;
  LatticeDev lat;
  st = get_lattice(*params, s, &lat);
  if (st != HDDA_OK) return st;
  *total_out = 0;
  if (n == 0) {
    HDDA_CUDA_TRY(cudaMemsetAsync(offsets, 0, sizeof(int64_t), s));
    return HDDA_OK;
  }
  int64_t* hw = nullptr;
  st = host_words(&hw);
  if (st != HDDA_OK) return st;
  char* scratch = nullptr;
  HDDA_CUDA_TRY(cudaMallocAsync(&scratch, twopass_scratch_bytes(n), s));
  st = run_twopass(ro, rd, n, grid, lat, params->image_width, offsets, ray_idx, t0, t1, capacity,
                   total_out, scratch, hw, nullptr, s);
  cudaError_t e = cudaFreeAsync(scratch, s);
  if (st == HDDA_OK && e != cudaSuccess) st = cuda_error(e, "cudaFreeAsync");
  return st;
}

// The same two passes in stream order: no read-back and no synchronisation;
// the total stays in offsets[n] and device status bits go to dev_status.
int traverse_async(const float* ro, const float* rd, int64_t n, const hdda_grid* grid,
                   const hdda_params* params, int64_t* offsets, int32_t* ray_idx, float* t0,
                   float* t1, int64_t capacity, uint32_t* dev_status, cudaStream_t s) {
  clear_error();
  if (!dev_status) return set_error(HDDA_ERR_INVALID_ARG, "dev_status is NULL");
  if (reinterpret_cast<uintptr_t>(dev_status) % 4 != 0)
    return set_error(HDDA_ERR_INVALID_ARG, "dev_status must be 4-byte aligned");
  int64_t unused_total = 0;
  const bool vdb = grid && grid->kind == HDDA_GRID_VDB;
  int st = check_args(vdb, ro, rd, n, grid, params, offsets, ray_idx, t0, t1, capacity,
                      &unused_total);
  if (st != HDDA_OK) return st;
  LatticeDev lat;
  st = get_lattice(*params, s, &lat);
  if (st != HDDA_OK) return st;
  if (n == 0) {
    HDDA_CUDA_TRY(cudaMemsetAsync(offsets, 0, sizeof(int64_t), s));
    return HDDA_OK;
  }
  char* scratch = nullptr;
  HDDA_CUDA_TRY(cudaMallocAsync(&scratch, twopass_scratch_bytes(n), s));
  st = run_twopass(ro, rd, n, grid, lat, params->image_width, offsets, ray_idx, t0, t1,
                   capacity, &unused_total, scratch, nullptr, dev_status, s);
  cudaError_t e = cudaFreeAsync(scratch, s);
  if (st == HDDA_OK && e != cudaSuccess) st = cuda_error(e, "cudaFreeAsync");
  return st;
}

}  // namespace

int lattice_for(const hdda_params* p, cudaStream_t s, LatticeDev* out) {
  const int st = validate_params(p);
  if (st != HDDA_OK) return st;
  return get_lattice(*p, s, out);
}

// ---------------------------------------------------------------------------
// traversal over caller-provided scratch (no allocation of any kind)
// ---------------------------------------------------------------------------
// Scratch layout (traverse_scratch_bytes): [0, 256) lattice read-back words;
// then one lattice block of capacity max_k; then the sampler's 32-byte
// header and tile states.

int64_t traverse_rays_per_tile() { return kBS; }

int traverse_with_scratch(bool vdb, const float* ro, const float* rd, int64_t n,
                          const hdda_grid* grid, const hdda_params* params, int64_t* offsets,
                          int32_t* ray_idx, float* t0, float* t1, int64_t capacity,
                          int64_t* total_out, void* scratch, int max_k, int64_t max_tiles,
                          cudaStream_t s) {
  clear_error();
  int st = check_args(vdb, ro, rd, n, grid, params, offsets, ray_idx, t0, t1, capacity,
                      total_out);
  if (st != HDDA_OK) return st;
  const int64_t nb = (n + kBS - 1) / kBS;
  if (nb > max_tiles)
    return set_error(HDDA_ERR_INVALID_ARG,
                     "n_rays=%lld exceeds the static scratch maximum of %lld rays",
                     (long long)n, (long long)(max_tiles * kBS));
  if (!scratch) return set_error(HDDA_ERR_INVALID_ARG, "scratch is NULL");
  *total_out = 0;
  char* base = static_cast<char*>(scratch);
  int64_t* lat_words = reinterpret_cast<int64_t*>(base);
  char* block = base + 256;
  char* sampler_scratch = block + lattice_block_bytes(max_k);

  // The array keeps the previous call's contents: clear what is read first.
  HDDA_CUDA_TRY(cudaMemsetAsync(base, 0, 32, s));
  const hdda_params key = canonical(*params);
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
  const int K = (int)hw[0];
  lattice_fill_kernel<<<1, kFillThreads, 0, s>>>(key, K, max_k, block);
  HDDA_CUDA_TRY(cudaGetLastError());
  if (n == 0) {
    HDDA_CUDA_TRY(cudaMemsetAsync(offsets, 0, sizeof(int64_t), s));
    return HDDA_OK;
  }
  return run_onepass(ro, rd, n, grid, lattice_view(block, max_k, K), offsets, ray_idx, t0, t1,
                     capacity, total_out, sampler_scratch, hw, s);
}

}  // namespace hdda

extern "C" int hdda_traverse_dense(const float* rays_o, const float* rays_d, int64_t n_rays,
                                   const hdda_grid* grid, const hdda_params* params,
                                   int64_t* offsets, int32_t* ray_idx, float* t0, float* t1,
                                   int64_t capacity, int64_t* total_out, hdda_stream_t stream) {
  return hdda::traverse(false, rays_o, rays_d, n_rays, grid, params, offsets, ray_idx, t0, t1,
                        capacity, total_out, (cudaStream_t)stream);
}

extern "C" int hdda_traverse_async(const float* rays_o, const float* rays_d, int64_t n_rays,
                                   const hdda_grid* grid, const hdda_params* params,
                                   int64_t* offsets, int32_t* ray_idx, float* t0, float* t1,
                                   int64_t capacity, uint32_t* dev_status, hdda_stream_t stream) {
  return hdda::traverse_async(rays_o, rays_d, n_rays, grid, params, offsets, ray_idx, t0, t1,
                              capacity, dev_status, (cudaStream_t)stream);
}

extern "C" int hdda_traverse_hdda(const float* rays_o, const float* rays_d, int64_t n_rays,
                                  const hdda_grid* grid, const hdda_params* params,
                                  int64_t* offsets, int32_t* ray_idx, float* t0, float* t1,
                                  int64_t capacity, int64_t* total_out, hdda_stream_t stream) {
  return hdda::traverse(true, rays_o, rays_d, n_rays, grid, params, offsets, ray_idx, t0, t1,
                        capacity, total_out, (cudaStream_t)stream);
}
