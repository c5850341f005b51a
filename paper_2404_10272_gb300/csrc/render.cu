// render.cu -- the render-only path: the sampler and the compositor joined
// at the level of runs, so that no sample is ever written to memory (the
// fused sampler + field evaluation; Sec. 1's accumulation applied to the
// intervals Algorithm 1 keeps).
//
// Pass 1 is the samplers' walk (walk_kernel, walk.cuh): each ray's merged
// occupied runs of lattice indices [k_begin, k_end), the first kMaxRuns of
// them, and its number of runs.  Pass 2 (render_kernel) gives each warp 8
// consecutive rays (measured faster than 4 or 16).  Every
// lattice index k of a run is the sample (t_k, t_{k+1}) with midpoint tm_k,
// read from the lattice table all rays share, so a warp numbers its rays'
// samples locally (a warp scan of the run lengths), and each sample of a
// 64-sample chunk (two per lane, field.cuh) finds its ray (compares against
// the slots' first positions, kept in registers) and its run (binary search
// over that ray's runs in shared memory).  The task's rays are staged in
// shared memory.  No global scan, no sample arrays, no host read-back.
//
// A ray with more than kMaxRuns runs is finished in rounds: after the runs
// it has are composited, it walks again from the end of the last one
// (walk_from) and the next kMaxRuns runs are composited with its
// transmittance and colour carried over, so samples are still accumulated
// front to back.
//
// The same kernel with kStore also writes what the samplers' emit writes:
// the CSR offsets (each task's 32-ray tile prefix from the tile scan plus a
// warp scan of the tile's counts) and every sample at its CSR position (the
// ray's offset, plus its samples of earlier rounds, plus its position in
// this round), so one pass both stores the samples and composites them
// (hdda_traverse_composite).
#include "field.cuh"
#include "walk.cuh"

namespace hdda {
namespace {

constexpr int kRenderWarps = 4;
constexpr int kRenderRays = 8;  // rays per warp task
constexpr uint32_t kNoRun = 0x7fffffffu;

// Blob evaluations (sample x kept blob), counted only while profiling.
__device__ unsigned long long g_render_evals;

// Outputs of the storing form (kStore): the samplers' CSR arrays.
struct StoreArgs {
  const int64_t* tile_prefix;  // exclusive prefix of the 32-ray tiles' sample counts
  const int32_t* counts;       // samples per ray
  int64_t* offsets;            // [n + 1], clamped to capacity
  int32_t* ray_idx;
  float* t0;
  float* t1;
  int64_t capacity;
  unsigned* status;            // kDevCapacity when the samples do not fit
};

// Position p of a round (numbered over the warp's rays) -> its lattice index:
// the run j of slot `own` that starts at or before p.  Runs hold {first k,
// first position}; unused slots have position kNoRun.
__device__ __forceinline__ int run_k(const uint2* sr, int own, int p, int& j) {
  j = 0;
#pragma unroll
  for (int s = kMaxRuns / 2; s > 0; s >>= 1)
    if (sr[(j + s) * kRenderRays + own].y <= (uint32_t)p) j += s;
  const uint2 e = sr[j * kRenderRays + own];
  return (int)e.x + (p - (int)e.y);
}

template <int kMode, bool kStore>
__global__ void __launch_bounds__(kRenderWarps * 32, 6) render_kernel(
    const float* __restrict__ ro, const float* __restrict__ rd, int64_t n, GridDev g,
    LatticeDev lat, const uint8_t* __restrict__ nruns, const uint2* __restrict__ runs,
    const float* __restrict__ field, int G, float* __restrict__ rgba, bool count_evals,
    StoreArgs out) {
  extern __shared__ __align__(16) unsigned char smem[];  // field_smem_bytes(G, kRenderWarps)
  __shared__ float s_T[kRenderWarps][kRenderRays];
  __shared__ float4 s_C[kRenderWarps][kRenderRays];
  __shared__ uint16_t s_cand[kRenderWarps][kMaxGauss];  // the task's candidate blobs
  __shared__ float4 s_ray[kRenderWarps][kRenderRays][2];  // {o, d.x}, {d.y, d.z, 1/|d|^2, -}
  __shared__ int64_t s_gbase[kRenderWarps][kRenderRays];  // storing form: output of position 0
  // run j of ray slot i at [j * kRenderRays + i]: {first k, first position}
  __shared__ uint2 s_run[kRenderWarps][kMaxRuns * kRenderRays];
  const FieldSmem fs = stage_blobs(smem, field, G);
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t task = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (task * kRenderRays >= n) return;  // uniform per warp; no block barrier follows
  float* T_s = s_T[wib];
  float4* C_s = s_C[wib];
  float4 (*rs)[2] = s_ray[wib];
  int64_t* gb = s_gbase[wib];
  uint2* sr = s_run[wib];
  unsigned long long evals = 0;  // this warp's blob evaluations
  const LatHdr h = lat_hdr(lat);
  const int64_t r = task * kRenderRays + lane;
  const bool has_ray = lane < kRenderRays && r < n;
  bool ok = false;
  if (lane < kRenderRays) {
    // the ray stays in shared memory only; a ray that needs another round of
    // runs rebuilds its walk state from there
    float o[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 0.f};
    if (has_ray) {
      ok = true;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        o[c] = __ldg(ro + 3 * r + c);
        d[c] = __ldg(rd + 3 * r + c);
        ok &= isfinite(o[c]) && isfinite(d[c]);
      }
    }
    T_s[lane] = 1.f;
    C_s[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    const float dd = fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2]));
    rs[lane][0] = make_float4(o[0], o[1], o[2], d[0]);
    rs[lane][1] = make_float4(d[1], d[2], dd > 1e-30f ? 1.f / dd : 0.f, 0.f);
  }
  __syncwarp();
  uint16_t* cand = s_cand[wib];
  const int ncand =
      task_candidates(fs, G, rs, (int)min((int64_t)kRenderRays, n - task * kRenderRays), cand);
  const int nr_all = ok ? (int)nruns[r] : 0;  // saturated at 255
  int nr = min(nr_all, kMaxRuns);
  for (int j = 0; j < nr; ++j) sr[j * kRenderRays + lane] = __ldg(runs + (int64_t)j * n + r);
  int k_next = lat.K;  // where the ray's walk resumes
  if (nr_all > kMaxRuns) k_next = (int)sr[(kMaxRuns - 1) * kRenderRays + lane].y;
  // storing form: lane i < kRenderRays holds ray i's CSR offset, then, per
  // round, the output position of the round's position 0 of that ray
  int64_t gofs = 0;
  if constexpr (kStore) {
    constexpr int kTasksPerTile = 32 / kRenderRays;
    const int64_t tile = task / kTasksPerTile;
    const int64_t tr = tile * 32 + lane;
    const int64_t c = tr < n ? (int64_t)__ldg(out.counts + tr) : 0;
    int64_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += y;
    }
    const int64_t ex = __ldg(out.tile_prefix + tile) + inc - c;
    const int first = (int)(task % kTasksPerTile) * kRenderRays;
    gofs = __shfl_sync(kFull, ex, first + (lane & (kRenderRays - 1)));
    const int64_t mine = __shfl_sync(kFull, c, first + (lane & (kRenderRays - 1)));
    // capacity 0 counts only: offsets unclamped, no samples, no status
    const bool clamp = out.capacity > 0;
    if (has_ray) {
      out.offsets[r] = clamp ? min(gofs, out.capacity) : gofs;
      if (r == n - 1) out.offsets[n] = clamp ? min(gofs + mine, out.capacity) : gofs + mine;
    }
    if (__any_sync(kFull, clamp && has_ray && gofs + mine > out.capacity) && lane == 0)
      atomicOr(out.status, kDevCapacity);
  }
  for (;;) {
    // this round's runs: lengths, the warp's numbering, then first positions
    int cnt = 0;
    for (int j = 0; j < nr; ++j) {
      const uint2 v = sr[j * kRenderRays + lane];
      cnt += (int)(v.y - v.x);
    }
    int inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += y;
    }
    const int pos = inc - cnt;
    const int W = __shfl_sync(kFull, inc, 31);
    // every lane keeps the first positions of slots 1 .. kRenderRays - 1
    int q[kRenderRays];
#pragma unroll
    for (int i = 1; i < kRenderRays; ++i) q[i] = __shfl_sync(kFull, pos, i);
    if (lane < kRenderRays) {
      if constexpr (kStore) gb[lane] = gofs - pos;
      int qq = pos;
      for (int j = 0; j < kMaxRuns; ++j) {
        uint2& e = sr[j * kRenderRays + lane];
        if (j < nr) {
          const int len = (int)(e.y - e.x);
          e.y = (uint32_t)qq;
          qq += len;
        } else {
          e = make_uint2(0u, kNoRun);
        }
      }
    }
    __syncwarp();
    for (int base = 0; base < W; base += kChunk) {
      Elem e[2];
      int k0 = 0, j0 = 0;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int p = base + 2 * lane + hh;
        int own = 0;  // the last slot whose first position is <= p
#pragma unroll
        for (int i = 1; i < kRenderRays; ++i) own += p >= q[i];
        e[hh].own = own;
        e[hh].a0 = e[hh].a1 = e[hh].px = e[hh].py = e[hh].pz = 0.f;
        if (p < W) {
          int k;
          if (hh == 1 && own == e[0].own &&
              (j0 + 1 >= kMaxRuns || (uint32_t)p < sr[(j0 + 1) * kRenderRays + own].y)) {
            // the next lattice index of e0's run: its start is e0's end
            k = k0 + 1;
            e[1].a0 = e[0].a1;
          } else {
            int j;
            k = run_k(sr, own, p, j);
            e[hh].a0 = __ldg(lat.t + k);
            k0 = k;
            j0 = j;
          }
          e[hh].a1 = __ldg(lat.t + k + 1);
          // the midpoint as the lattice defines it: fl(fl(t_k + t_k+1) * 0.5)
          const float tm = __fmul_rn(__fadd_rn(e[hh].a0, e[hh].a1), 0.5f);
          const float4 A = rs[own][0], B = rs[own][1];
          e[hh].px = fmaf(tm, A.w, A.x);
          e[hh].py = fmaf(tm, B.x, A.y);
          e[hh].pz = fmaf(tm, B.y, A.z);
          if constexpr (kStore) {
            const int64_t qo = gb[own] + p;
            if (qo < out.capacity) {
              out.ray_idx[qo] = (int32_t)(task * kRenderRays + own);
              out.t0[qo] = e[hh].a0;
              out.t1[qo] = e[hh].a1;
            }
          }
        }
      }
      evals += composite_chunk2(fs, cand, ncand, min(kChunk, W - base), e[0], e[1], rs, T_s, C_s);
    }
    if constexpr (kStore) gofs += cnt;  // this round's samples of the lane's ray are written
    const bool more = k_next < lat.K;
    if (!__any_sync(kFull, more)) break;
    nr = 0;
    if (more) {
      Ray ray;
      const float4 A = rs[lane][0], B = rs[lane][1];
      const float o[3] = {A.x, A.y, A.z}, d[3] = {A.w, B.x, B.y};
#pragma unroll
      for (int c = 0; c < 3; ++c) {  // as load_ray (walk.cuh) sets them up
        ray.o[c] = o[c];
        ray.d[c] = d[c];
        ray.neg[c] = d[c] < 0.f;
        ray.inv[c] = d[c] != 0.f ? 1.0f / d[c] : INFINITY;
      }
      k_next = walk_from<kMode, false>(g, global_tabs(g), lat, h, ray, k_next, sr + lane,
                                       kRenderRays, nr);
    }
    __syncwarp();
  }
  if (has_ray) {
    const float4 acc = C_s[lane];
    reinterpret_cast<float4*>(rgba)[r] = make_float4(acc.x, acc.y, acc.z, 1.f - T_s[lane]);
  }
  if (count_evals && lane == 0) atomicAdd(&g_render_evals, evals);
}

const char* render_name(int mode) {
  return mode == kModeDense ? "dense_render" : mode == kModeVdb ? "hdda_render_plain"
                                                                 : "hdda_render";
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Scratch: [0, 256) header {walk counter u32, status u32}, then counts, run
// counts and runs (the render kernel needs no tile sums: the walk skips them).
size_t render_scratch_bytes(int64_t n) {
  return 256 + a256(4 * (size_t)n) + a256((size_t)n) + a256(sizeof(uint2) * kMaxRuns * (size_t)n);
}

// Pinned host word for the synchronous status read.
struct HostWord {
  unsigned* p = nullptr;
  ~HostWord() { if (p) cudaFreeHost(p); }
};
thread_local HostWord t_word;

int launch_render(const float* ro, const float* rd, int64_t n, const hdda_grid* grid,
                  const LatticeDev& lat, int32_t width, const float* field, int G, float* rgba,
                  unsigned* dev_status, char* scratch, cudaStream_t s) {
  unsigned* counter = reinterpret_cast<unsigned*>(scratch);
  unsigned* status = dev_status ? dev_status : counter + 1;
  char* p = scratch + 256;
  int32_t* counts = reinterpret_cast<int32_t*>(p);
  p += a256(4 * (size_t)n);
  uint8_t* nr = reinterpret_cast<uint8_t*>(p);
  p += a256((size_t)n);
  uint2* runs = reinterpret_cast<uint2*>(p);
  HDDA_CUDA_TRY(cudaMemsetAsync(scratch, 0, 256, s));
  const int mode = walk_mode(grid);
  WalkArgs w{ro, rd, n, grid->view(), lat, counts, nr, runs, nullptr, counter, status};
  w.width = (int32_t)(width < n ? width : n);
  const size_t stage = stage_layout(lat.K, w.g.L, w.g.R, grid->nodes_total(), mode).bytes;
  {
    KernelTimer kt(walk_name(mode), s);
    const bool skip = grid->walk_variant == HDDA_WALK_SKIP;
    const int st = mode == kModeDense ? launch_walk_mode<kModeDense>(w, stage, skip, s)
                   : mode == kModeVdb ? launch_walk_mode<kModeVdb>(w, stage, skip, s)
                                      : launch_walk_mode<kModeVdbMap>(w, stage, skip, s);
    if (st != HDDA_OK) return st;
  }
  {
    KernelTimer kt(render_name(mode), s);
    const int64_t warps = (n + kRenderRays - 1) / kRenderRays;
    const unsigned nb = (unsigned)((warps + kRenderWarps - 1) / kRenderWarps);
    const bool ev = counters_on();
    const size_t fsm = field_smem_bytes(G, kRenderWarps);
    switch (mode) {
      case kModeDense:
        render_kernel<kModeDense, false><<<nb, kRenderWarps * 32, fsm, s>>>(
            ro, rd, n, w.g, lat, nr, runs, field, G, rgba, ev, StoreArgs{});
        break;
      case kModeVdb:
        render_kernel<kModeVdb, false><<<nb, kRenderWarps * 32, fsm, s>>>(
            ro, rd, n, w.g, lat, nr, runs, field, G, rgba, ev, StoreArgs{});
        break;
      default:
        render_kernel<kModeVdbMap, false><<<nb, kRenderWarps * 32, fsm, s>>>(
            ro, rd, n, w.g, lat, nr, runs, field, G, rgba, ev, StoreArgs{});
        break;
    }
  }
  HDDA_CUDA_TRY(cudaGetLastError());
  return HDDA_OK;
}

// Scratch of the storing form: the header, tile sums and prefixes, counts,
// run counts and runs.
size_t sample_composite_scratch_bytes(int64_t n) {
  const int64_t T = (n + 31) / 32;
  return 256 + 2 * a256(8 * (size_t)T) + a256(4 * (size_t)n) + a256((size_t)n) +
         a256(sizeof(uint2) * kMaxRuns * (size_t)n);
}

const char* sample_composite_name(int mode) {
  return mode == kModeDense ? "dense_sample_composite"
         : mode == kModeVdb ? "hdda_sample_composite_plain"
                            : "hdda_sample_composite";
}

// Walk, tile scan, then the storing render kernel: the samplers' outputs and
// the frame in one pass over the samples.
int launch_sample_composite(const float* ro, const float* rd, int64_t n, const hdda_grid* grid,
                            const LatticeDev& lat, int32_t width, const float* field, int G,
                            float* rgba,
                            int64_t* offsets, int32_t* ray_idx, float* t0, float* t1,
                            int64_t capacity, unsigned* status, char* scratch, cudaStream_t s) {
  const int64_t T = (n + 31) / 32;
  unsigned* counter = reinterpret_cast<unsigned*>(scratch);
  int64_t* total = reinterpret_cast<int64_t*>(scratch + 8);
  char* p = scratch + 256;
  int64_t* tile_sum = reinterpret_cast<int64_t*>(p);
  p += a256(8 * (size_t)T);
  int64_t* tile_prefix = reinterpret_cast<int64_t*>(p);
  p += a256(8 * (size_t)T);
  int32_t* counts = reinterpret_cast<int32_t*>(p);
  p += a256(4 * (size_t)n);
  uint8_t* nr = reinterpret_cast<uint8_t*>(p);
  p += a256((size_t)n);
  uint2* runs = reinterpret_cast<uint2*>(p);
  // a walk in pixel blocks adds the tile sums up atomically: clear them too
  WalkArgs w{ro, rd, n, grid->view(), lat, counts, nr, runs, tile_sum, counter, status};
  w.width = (int32_t)(width < n ? width : n);
  HDDA_CUDA_TRY(cudaMemsetAsync(scratch, 0, w.width > 0 ? 256 + 8 * (size_t)T : 256, s));
  const int mode = walk_mode(grid);
  const size_t stage = stage_layout(lat.K, w.g.L, w.g.R, grid->nodes_total(), mode).bytes;
  {
    KernelTimer kt(walk_name(mode), s);
    const bool skip = grid->walk_variant == HDDA_WALK_SKIP;
    const int st = mode == kModeDense ? launch_walk_mode<kModeDense>(w, stage, skip, s)
                   : mode == kModeVdb ? launch_walk_mode<kModeVdb>(w, stage, skip, s)
                                      : launch_walk_mode<kModeVdbMap>(w, stage, skip, s);
    if (st != HDDA_OK) return st;
  }
  {
    KernelTimer kt("tile_scan", s);
    if (T <= (int64_t)kMaxSupers * kSuperTiles)
      tile_scan_par_kernel<<<(unsigned)((T + kSuperTiles - 1) / kSuperTiles), kSuperTiles, 0, s>>>(
          tile_sum, T, tile_prefix, total, offsets + n);
    else
      tile_scan_kernel<<<1, kScanThreads, 0, s>>>(tile_sum, T, tile_prefix, total, offsets + n);
  }
  HDDA_CUDA_TRY(cudaGetLastError());
  {
    KernelTimer kt(sample_composite_name(mode), s);
    const int64_t warps = (n + kRenderRays - 1) / kRenderRays;
    const unsigned nb = (unsigned)((warps + kRenderWarps - 1) / kRenderWarps);
    const bool ev = counters_on();
    const size_t fsm = field_smem_bytes(G, kRenderWarps);
    const StoreArgs out{tile_prefix, counts, offsets, ray_idx, t0, t1, capacity, status};
    switch (mode) {
      case kModeDense:
        render_kernel<kModeDense, true><<<nb, kRenderWarps * 32, fsm, s>>>(
            ro, rd, n, w.g, lat, nr, runs, field, G, rgba, ev, out);
        break;
      case kModeVdb:
        render_kernel<kModeVdb, true><<<nb, kRenderWarps * 32, fsm, s>>>(
            ro, rd, n, w.g, lat, nr, runs, field, G, rgba, ev, out);
        break;
      default:
        render_kernel<kModeVdbMap, true><<<nb, kRenderWarps * 32, fsm, s>>>(
            ro, rd, n, w.g, lat, nr, runs, field, G, rgba, ev, out);
        break;
    }
  }
  HDDA_CUDA_TRY(cudaGetLastError());
  return HDDA_OK;
}

}  // namespace

unsigned long long render_take_blob_evals() {
  unsigned long long v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_render_evals, sizeof(v)) != cudaSuccess) return 0;
  cudaMemcpyToSymbol(g_render_evals, &zero, sizeof(zero));
  return v;
}

}  // namespace hdda

extern "C" int hdda_render(const float* rays_o, const float* rays_d, int64_t n_rays,
                           const hdda_grid* grid, const hdda_params* params, const float* field,
                           int n_gauss, float* rgba_out, uint32_t* dev_status,
                           hdda_stream_t stream) {
  using namespace hdda;
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  if (!grid) return set_error(HDDA_ERR_INVALID_ARG, "grid is NULL");
  if (n_rays < 0 || n_rays > INT32_MAX)
    return set_error(HDDA_ERR_INVALID_ARG, "n_rays=%lld", (long long)n_rays);
  if (n_gauss < 0 || n_gauss > kMaxGauss)
    return set_error(HDDA_ERR_INVALID_ARG, "n_gauss=%d outside 0..%d", n_gauss, kMaxGauss);
  if (n_rays > 0 && (!rays_o || !rays_d || !rgba_out))
    return set_error(HDDA_ERR_INVALID_ARG, "NULL pointer");
  if (n_gauss > 0 && !field) return set_error(HDDA_ERR_INVALID_ARG, "field is NULL");
  if (reinterpret_cast<uintptr_t>(rgba_out) % 16 != 0)
    return set_error(HDDA_ERR_INVALID_ARG, "rgba_out must be 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(dev_status) % 4 != 0)
    return set_error(HDDA_ERR_INVALID_ARG, "dev_status must be 4-byte aligned");
  int dev = 0;
  HDDA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != grid->device)
    return set_error(HDDA_ERR_INVALID_ARG, "grid lives on device %d, current is %d",
                     grid->device, dev);
  LatticeDev lat;
  int st = lattice_for(params, s, &lat);
  if (st != HDDA_OK) return st;
  if (n_rays == 0) return HDDA_OK;
  unsigned* hw = nullptr;
  if (!dev_status) {
    if (!t_word.p) HDDA_CUDA_TRY(cudaMallocHost(&t_word.p, sizeof(unsigned)));
    hw = t_word.p;
  }
  char* scratch = nullptr;
  HDDA_CUDA_TRY(cudaMallocAsync(&scratch, render_scratch_bytes(n_rays), s));
  st = launch_render(rays_o, rays_d, n_rays, grid, lat, params->image_width, field, n_gauss,
                     rgba_out, dev_status, scratch, s);
  if (st == HDDA_OK && !dev_status) {
    cudaError_t e = cudaMemcpyAsync(hw, scratch + 4, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = cuda_error(e, "cudaMemcpyAsync(status)");
  }
  cudaError_t e = cudaFreeAsync(scratch, s);
  if (st == HDDA_OK && e != cudaSuccess) st = cuda_error(e, "cudaFreeAsync");
  if (st != HDDA_OK || dev_status) return st;
  HDDA_CUDA_TRY(cudaStreamSynchronize(s));
  if (*hw & kDevInternal) return set_error(HDDA_ERR_INTERNAL, "region check failed on the device");
  return HDDA_OK;
}

extern "C" int hdda_traverse_composite(const float* rays_o, const float* rays_d, int64_t n_rays,
                                       const hdda_grid* grid, const hdda_params* params,
                                       int64_t* offsets, int32_t* ray_idx, float* t0, float* t1,
                                       int64_t capacity, const float* field, int n_gauss,
                                       float* rgba_out, uint32_t* dev_status,
                                       hdda_stream_t stream) {
  using namespace hdda;
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  if (!grid) return set_error(HDDA_ERR_INVALID_ARG, "grid is NULL");
  if (!params) return set_error(HDDA_ERR_INVALID_ARG, "params is NULL");
  if (n_rays < 0 || n_rays > INT32_MAX)
    return set_error(HDDA_ERR_INVALID_ARG, "n_rays=%lld", (long long)n_rays);
  if (n_gauss < 0 || n_gauss > kMaxGauss)
    return set_error(HDDA_ERR_INVALID_ARG, "n_gauss=%d outside 0..%d", n_gauss, kMaxGauss);
  if (!offsets) return set_error(HDDA_ERR_INVALID_ARG, "offsets is NULL");
  if (capacity < 0) return set_error(HDDA_ERR_INVALID_ARG, "capacity < 0");
  if (capacity > 0 && (!ray_idx || !t0 || !t1))
    return set_error(HDDA_ERR_INVALID_ARG, "sample arrays NULL");
  if (n_rays > 0 && (!rays_o || !rays_d || !rgba_out))
    return set_error(HDDA_ERR_INVALID_ARG, "NULL pointer");
  if (n_gauss > 0 && !field) return set_error(HDDA_ERR_INVALID_ARG, "field is NULL");
  if (reinterpret_cast<uintptr_t>(rgba_out) % 16 != 0)
    return set_error(HDDA_ERR_INVALID_ARG, "rgba_out must be 16-byte aligned");
  if (!dev_status) return set_error(HDDA_ERR_INVALID_ARG, "dev_status is NULL");
  if (reinterpret_cast<uintptr_t>(dev_status) % 4 != 0)
    return set_error(HDDA_ERR_INVALID_ARG, "dev_status must be 4-byte aligned");
  int dev = 0;
  HDDA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != grid->device)
    return set_error(HDDA_ERR_INVALID_ARG, "grid lives on device %d, current is %d",
                     grid->device, dev);
  LatticeDev lat;
  int st = lattice_for(params, s, &lat);
  if (st != HDDA_OK) return st;
  if (n_rays == 0) {
    HDDA_CUDA_TRY(cudaMemsetAsync(offsets, 0, sizeof(int64_t), s));
    return HDDA_OK;
  }
  char* scratch = nullptr;
  HDDA_CUDA_TRY(cudaMallocAsync(&scratch, sample_composite_scratch_bytes(n_rays), s));
  st = launch_sample_composite(rays_o, rays_d, n_rays, grid, lat, params->image_width, field,
                               n_gauss, rgba_out, offsets, ray_idx, t0, t1, capacity, dev_status,
                               scratch, s);
  cudaError_t e = cudaFreeAsync(scratch, s);
  if (st == HDDA_OK && e != cudaSuccess) st = cuda_error(e, "cudaFreeAsync");
  return st;
}
