// batch.cu -- many sampling jobs (scenes, cameras, image sizes, cascade
// depths) in one launch sequence that can be captured once in a CUDA graph
// and replayed.
//
// A job is one traversal: its rays, its grid, its lattice parameters and its
// own output buffers.  Every job's rays are cut into 32-ray tiles numbered
// consecutively over all jobs.  batch_walk_kernel is persistent: each warp
// takes `tiles_per_fetch` tiles at a time from one atomic counter (work
// stealing), finds the job of each tile by binary search, copies that job's
// grid descriptor into its own slice of shared memory when the job changes,
// and walks the tile exactly as the single-call walk does.  One scan over all
// tiles then gives every tile its offset; a job's offsets are those minus the
// job's first prefix.  batch_emit_kernel writes each job's CSR offsets and
// samples into that job's buffers, with the capacity checked per job.  With
// these three kernels and a few memsets, a batch is one graph launch however
// many jobs it holds; the sizes (block of the walk, tiles per fetch, warps per
// emit CTA) are chosen by the autotuner in the Python package.
#include <cstring>
#include <new>
#include <vector>

#include "walk.cuh"

namespace hdda {
namespace {

constexpr int kMaxBatchJobs = 4096;
constexpr unsigned kJobCapacity = 1u;  // job status bit: outputs smaller than its samples

struct JobDev {
  GridDev g;
  LatticeDev lat;
  const float* ro;
  const float* rd;
  int64_t n;
  int64_t* offsets;
  int32_t* ray_idx;
  float* t0;
  float* t1;
  int64_t capacity;
  int64_t tile0;  // first tile of the job in the batch numbering
  int64_t tiles;
};

// Largest j with tile0[j] <= t (tile0 has J + 1 entries, tile0[J] = T).
__device__ __forceinline__ int find_job(const int64_t* __restrict__ tile0, int J, int64_t t) {
  int lo = 0, hi = J - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(tile0 + mid) <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

constexpr int kGridWords = (sizeof(GridDev) + 3) / 4;

// Copies a job's grid descriptor into a warp's shared-memory slot.
__device__ __forceinline__ void warp_copy_grid(GridDev* dst, const GridDev* src) {
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int i = threadIdx.x & 31; i < kGridWords; i += 32) d[i] = __ldg(s + i);
  __syncwarp();
}

template <int kMode, int kBlock, bool kSkip, bool kCheck>
__global__ void __launch_bounds__(kBlock) batch_walk_kernel(
    const JobDev* __restrict__ jobs, const int64_t* __restrict__ tile0, int J, int64_t T,
    int tiles_per_fetch, int32_t* __restrict__ counts, uint8_t* __restrict__ nruns_out,
    uint2* __restrict__ runs, int64_t* __restrict__ tile_sum, unsigned* __restrict__ counter,
    unsigned* __restrict__ status) {
  __shared__ __align__(16) GridDev s_grid[kBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  GridDev& g = s_grid[warp];
  const int64_t slots = T * 32;  // ray slots over the whole batch (stride of the runs)
  int cur = -1;
  LatticeDev lat{};
  LatHdr h{};
  int64_t n = 0, job_tile0 = 0;
  const float* ro = nullptr;
  const float* rd = nullptr;
  for (;;) {
    unsigned first = 0;
    if (lane == 0) first = atomicAdd(counter, (unsigned)tiles_per_fetch);
    first = __shfl_sync(kFull, first, 0);
    if ((int64_t)first >= T) break;
    const int64_t last = min((int64_t)first + tiles_per_fetch, T);
    for (int64_t t = first; t < last; ++t) {
      const int j = find_job(tile0, J, t);
      if (j != cur) {
        cur = j;
        warp_copy_grid(&g, &jobs[j].g);
        lat = jobs[j].lat;
        h = lat_hdr(lat);
        n = jobs[j].n;
        job_tile0 = jobs[j].tile0;
        ro = jobs[j].ro;
        rd = jobs[j].rd;
      }
      const int64_t lr = (t - job_tile0) * 32 + lane;
      const int64_t gr = t * 32 + lane;
      int64_t c = 0;
      if (lr < n) {
        Ray ray;
        int nr = 0;
        if (load_ray(ro, rd, lr, ray))
          c = walk<kMode, false, false, kSkip, kCheck>(g, global_tabs(g), lat, h, ray, runs + gr,
                                                       slots, nr, 0, 0, 0, nullptr, nullptr,
                                                       nullptr, status);
        counts[gr] = (int32_t)c;
        nruns_out[gr] = (uint8_t)min(nr, 255);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
      if (lane == 0) tile_sum[t] = c;
    }
  }
}

template <int kMode, int kWarps>
__global__ void __launch_bounds__(kWarps * 32) batch_emit_kernel(
    const JobDev* __restrict__ jobs, const int64_t* __restrict__ tile0, int J, int64_t T,
    const int32_t* __restrict__ counts, const uint8_t* __restrict__ nruns,
    const uint2* __restrict__ runs, const int64_t* __restrict__ tile_prefix,
    const int64_t* __restrict__ grand_total, int64_t* __restrict__ job_totals,
    unsigned* __restrict__ job_status, unsigned* __restrict__ status) {
  __shared__ uint2 s_rec[kWarps][kRecMax + 1];
  __shared__ __align__(16) GridDev s_grid[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t t = (int64_t)blockIdx.x * kWarps + warp;
  if (t >= T) return;  // uniform per warp
  const int j = find_job(tile0, J, t);
  const JobDev& jb = jobs[j];
  const int64_t jt0 = jb.tile0, n = jb.n, capacity = jb.capacity;
  const int64_t lr = (t - jt0) * 32 + lane;
  const int64_t gr = t * 32 + lane;
  const int64_t slots = T * 32;
  const int c = lr < n ? counts[gr] : 0;
  const int nr = lr < n ? (int)nruns[gr] : 0;
  // a tile holds at most 32 * 2^24 samples: 32-bit positions within it
  int inc = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += y;
  }
  const int q = inc - c;
  const int64_t base = __ldg(tile_prefix + jt0);
  const int64_t wbeg = __ldg(tile_prefix + t) - base;  // the tile's first sample in the job
  const int64_t off = wbeg + q;
  if (lr < n) jb.offsets[lr] = off;
  if (t == jt0 + jb.tiles - 1 && lane == 0) {
    const int64_t next = __ldg(tile0 + j + 1);
    const int64_t total = (next < T ? __ldg(tile_prefix + next) : *grand_total) - base;
    jb.offsets[n] = total;
    job_totals[j] = total;
    if (capacity > 0 && total > capacity) atomicOr(job_status + j, kJobCapacity);
  }
  if (capacity <= 0) return;
  // the tile's runs as a record list, expanded with 16-byte stores where the
  // job's outputs allow (expand_records, walk.cuh)
  uint2* rec = s_rec[warp];
  const int kept = c <= 0 ? 0 : nr > kMaxRuns ? 1 : nr;
  int kinc = kept;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, kinc, o);
    if (lane >= o) kinc += y;
  }
  const int nrec = __shfl_sync(kFull, kinc, 31);
  list_runs(rec, kinc - kept, lane, nr, c, (uint32_t)q, runs + gr, slots);
  if (lane == 0) rec[nrec] = make_uint2(kRecEnd, 0u);
  __syncwarp();
  const int tot = __shfl_sync(kFull, inc, 31);
  const int64_t room = capacity - wbeg;
  const int lim = room <= 0 ? 0 : (int)min((int64_t)tot, room);
  const bool vec = ((reinterpret_cast<uintptr_t>(jb.ray_idx) |
                     reinterpret_cast<uintptr_t>(jb.t0) | reinterpret_cast<uintptr_t>(jb.t1)) &
                    15) == 0;
  const bool overflow = nr > kMaxRuns;
  const LatticeDev lat = jb.lat;
  expand_records(rec, nrec, lim, wbeg, (int32_t)(lr - lane), lat.t, vec, jb.ray_idx, jb.t0,
                 jb.t1);
  if (__any_sync(kFull, overflow)) {
    warp_copy_grid(&s_grid[warp], &jb.g);  // the whole warp copies; only overflowing lanes walk
    if (overflow) {
      Ray ray;
      load_ray(jb.ro, jb.rd, lr, ray);
      const LatHdr h = lat_hdr(lat);
      int unused = 0;
      walk<kMode, true, false>(s_grid[warp], global_tabs(s_grid[warp]), lat, h, ray, nullptr, 0,
                               unused, (int32_t)lr, off, capacity, jb.ray_idx, jb.t0, jb.t1,
                               status);
    }
  }
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace hdda

struct hdda_batch {
  int n_jobs = 0;
  int mode = 0;
  int device = 0;
  int64_t T = 0;
  bool check = false;  // region checks, as set when the batch was created
  hdda_batch_config cfg{};
  hdda::JobDev* jobs = nullptr;  // device
  int64_t* tile0 = nullptr;      // device [J + 1]
  char* scratch = nullptr;
  size_t scratch_bytes = 0;
  // a batch without a graph takes its scratch from the stream-ordered allocator of
  // the stream it was created on and returns it there
  cudaStream_t alloc_stream = nullptr;
  bool async_scratch = false;
  // carved from scratch
  unsigned* counter = nullptr;
  unsigned* status = nullptr;
  int64_t* total = nullptr;
  int64_t* tile_sum = nullptr;
  int64_t* tile_prefix = nullptr;
  int32_t* counts = nullptr;
  uint8_t* nruns = nullptr;
  uint2* runs = nullptr;
  int64_t* job_totals = nullptr;
  unsigned* job_status = nullptr;
  std::vector<int64_t*> zero_offsets;  // offsets[0] of jobs without rays
  unsigned walk_grid = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace hdda {
namespace {

template <int kMode, int kBlock, bool kSkip>
int batch_walk_grid(unsigned* out) {
  int dev = 0, sms = 0, per_sm = 0;
  HDDA_CUDA_TRY(cudaGetDevice(&dev));
  HDDA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HDDA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, batch_walk_kernel<kMode, kBlock, kSkip, false>, kBlock, 0));
  *out = (unsigned)(sms * (per_sm > 0 ? per_sm : 1));
  return HDDA_OK;
}

template <int kMode, bool kSkip>
int walk_grid_for(int block, unsigned* out) {
  switch (block) {
    case 128: return batch_walk_grid<kMode, 128, kSkip>(out);
    case 256: return batch_walk_grid<kMode, 256, kSkip>(out);
    default: return batch_walk_grid<kMode, 512, kSkip>(out);
  }
}

template <int kMode>
int walk_grid_for_block(int block, bool skip, unsigned* out) {
  return skip ? walk_grid_for<kMode, true>(block, out) : walk_grid_for<kMode, false>(block, out);
}

template <int kMode, bool kSkip, bool kCheck>
void launch_batch_walk_c(const hdda_batch* b, cudaStream_t s) {
  const unsigned grid = b->walk_grid;
  const int tpf = b->cfg.rays_per_fetch / 32;
#define HDDA_BATCH_WALK(BS)                                                              \
  batch_walk_kernel<kMode, BS, kSkip, kCheck><<<grid, BS, 0, s>>>(                       \
      b->jobs, b->tile0, b->n_jobs, b->T, tpf, b->counts, b->nruns, b->runs, b->tile_sum, \
      b->counter, b->status)
  switch (b->cfg.walk_block) {
    case 128: HDDA_BATCH_WALK(128); break;
    case 256: HDDA_BATCH_WALK(256); break;
    default: HDDA_BATCH_WALK(512); break;
  }
#undef HDDA_BATCH_WALK
}

template <int kMode, bool kSkip>
void launch_batch_walk_v(const hdda_batch* b, cudaStream_t s) {
  if (b->check) launch_batch_walk_c<kMode, kSkip, true>(b, s);
  else launch_batch_walk_c<kMode, kSkip, false>(b, s);
}

template <int kMode>
void launch_batch_walk(const hdda_batch* b, cudaStream_t s) {
  if (b->cfg.walk_variant == HDDA_WALK_SKIP) launch_batch_walk_v<kMode, true>(b, s);
  else launch_batch_walk_v<kMode, false>(b, s);
}

template <int kMode>
void launch_batch_emit(const hdda_batch* b, cudaStream_t s) {
#define HDDA_BATCH_EMIT(W)                                                                    \
  batch_emit_kernel<kMode, W><<<(unsigned)((b->T + W - 1) / W), W * 32, 0, s>>>(             \
      b->jobs, b->tile0, b->n_jobs, b->T, b->counts, b->nruns, b->runs, b->tile_prefix,      \
      b->total, b->job_totals, b->job_status, b->status)
  switch (b->cfg.emit_warps) {
    case 2: HDDA_BATCH_EMIT(2); break;
    case 4: HDDA_BATCH_EMIT(4); break;
    default: HDDA_BATCH_EMIT(8); break;
  }
#undef HDDA_BATCH_EMIT
}

// Queues one execution of the batch on s (memsets, walk, scan, emit).
int enqueue(const hdda_batch* b, cudaStream_t s) {
  HDDA_CUDA_TRY(cudaMemsetAsync(b->scratch, 0, 256, s));
  HDDA_CUDA_TRY(cudaMemsetAsync(b->job_totals, 0, sizeof(int64_t) * b->n_jobs, s));
  HDDA_CUDA_TRY(cudaMemsetAsync(b->job_status, 0, sizeof(unsigned) * b->n_jobs, s));
  for (int64_t* p : b->zero_offsets) HDDA_CUDA_TRY(cudaMemsetAsync(p, 0, sizeof(int64_t), s));
  if (b->T == 0) return HDDA_OK;
  switch (b->mode) {
    case kModeDense: launch_batch_walk<kModeDense>(b, s); break;
    case kModeVdb: launch_batch_walk<kModeVdb>(b, s); break;
    default: launch_batch_walk<kModeVdbMap>(b, s); break;
  }
  HDDA_CUDA_TRY(cudaGetLastError());
  tile_scan_kernel<<<1, kScanThreads, 0, s>>>(b->tile_sum, b->T, b->tile_prefix, b->total,
                                              b->total + 1);
  HDDA_CUDA_TRY(cudaGetLastError());
  switch (b->mode) {
    case kModeDense: launch_batch_emit<kModeDense>(b, s); break;
    case kModeVdb: launch_batch_emit<kModeVdb>(b, s); break;
    default: launch_batch_emit<kModeVdbMap>(b, s); break;
  }
  HDDA_CUDA_TRY(cudaGetLastError());
  return HDDA_OK;
}

int check_config(const hdda_batch_config& c) {
  if (c.walk_block != 128 && c.walk_block != 256 && c.walk_block != 512)
    return set_error(HDDA_ERR_INVALID_ARG, "walk_block must be 128, 256 or 512");
  if (c.rays_per_fetch < 32 || c.rays_per_fetch > 1024 || c.rays_per_fetch % 32)
    return set_error(HDDA_ERR_INVALID_ARG, "rays_per_fetch must be a multiple of 32 in 32..1024");
  if (c.emit_warps != 2 && c.emit_warps != 4 && c.emit_warps != 8)
    return set_error(HDDA_ERR_INVALID_ARG, "emit_warps must be 2, 4 or 8");
  if (c.walk_variant != HDDA_WALK_BRANCH && c.walk_variant != HDDA_WALK_SKIP)
    return set_error(HDDA_ERR_INVALID_ARG, "walk_variant must be HDDA_WALK_BRANCH or _SKIP");
  return HDDA_OK;
}

int create(const hdda_job* jobs, int n_jobs, const hdda_batch_config* cfg, hdda_batch** out,
           cudaStream_t s) {
  if (!out) return set_error(HDDA_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_jobs < 1 || n_jobs > kMaxBatchJobs)
    return set_error(HDDA_ERR_INVALID_ARG, "n_jobs=%d outside 1..%d", n_jobs, kMaxBatchJobs);
  if (!jobs) return set_error(HDDA_ERR_INVALID_ARG, "jobs is NULL");
  hdda_batch_config c{256, 64, 4, 1, HDDA_WALK_BRANCH};
  if (cfg) c = *cfg;
  int st = check_config(c);
  if (st != HDDA_OK) return st;
  int dev = 0;
  HDDA_CUDA_TRY(cudaGetDevice(&dev));
  std::vector<JobDev> host(n_jobs);
  std::vector<int64_t> tile0(n_jobs + 1);
  int mode = -1;
  int64_t T = 0;
  std::vector<int64_t*> zero_offsets;
  for (int j = 0; j < n_jobs; ++j) {
    const hdda_job& jb = jobs[j];
    if (!jb.grid) return set_error(HDDA_ERR_INVALID_ARG, "job %d: grid is NULL", j);
    if (jb.grid->device != dev)
      return set_error(HDDA_ERR_INVALID_ARG, "job %d: grid lives on another device", j);
    const int m = jb.grid->kind == HDDA_GRID_DENSE
                      ? kModeDense
                      : (jb.grid->refine ? kModeVdbMap : kModeVdb);
    if (mode >= 0 && m != mode)
      return set_error(HDDA_ERR_INVALID_ARG, "job %d: all grids of a batch must be of one kind", j);
    mode = m;
    if (jb.n_rays < 0 || jb.n_rays > INT32_MAX)
      return set_error(HDDA_ERR_INVALID_ARG, "job %d: n_rays=%lld", j, (long long)jb.n_rays);
    if (!jb.offsets) return set_error(HDDA_ERR_INVALID_ARG, "job %d: offsets is NULL", j);
    if (jb.n_rays > 0 && (!jb.rays_o || !jb.rays_d))
      return set_error(HDDA_ERR_INVALID_ARG, "job %d: rays NULL", j);
    if (jb.capacity < 0) return set_error(HDDA_ERR_INVALID_ARG, "job %d: capacity < 0", j);
    if (jb.capacity > 0 && (!jb.ray_idx || !jb.t0 || !jb.t1))
      return set_error(HDDA_ERR_INVALID_ARG, "job %d: sample outputs NULL", j);
    LatticeDev lat;
    st = lattice_for(&jb.params, s, &lat);
    if (st != HDDA_OK) return st;
    JobDev& d = host[j];
    std::memset(&d, 0, sizeof(d));
    d.g = jb.grid->view();
    d.lat = lat;
    d.ro = jb.rays_o;
    d.rd = jb.rays_d;
    d.n = jb.n_rays;
    d.offsets = jb.offsets;
    d.ray_idx = jb.ray_idx;
    d.t0 = jb.t0;
    d.t1 = jb.t1;
    d.capacity = jb.capacity;
    d.tile0 = T;
    d.tiles = (jb.n_rays + 31) / 32;
    tile0[j] = T;
    T += d.tiles;
    if (jb.n_rays == 0) zero_offsets.push_back(jb.offsets);
  }
  tile0[n_jobs] = T;

  hdda_batch* b = new (std::nothrow) hdda_batch();
  if (!b) return set_error(HDDA_ERR_OOM, "host allocation failed");
  b->n_jobs = n_jobs;
  b->mode = mode;
  b->device = dev;
  b->T = T;
  b->check = region_checks_on();
  b->cfg = c;
  b->zero_offsets = zero_offsets;
  const int64_t slots = T * 32;
  b->scratch_bytes = 256 + 2 * a256(8 * (size_t)T + 8) + a256(4 * (size_t)slots) +
                     a256((size_t)slots) + a256(sizeof(uint2) * kMaxRuns * (size_t)slots) +
                     a256(8 * (size_t)n_jobs) + a256(4 * (size_t)n_jobs) +
                     a256(sizeof(JobDev) * n_jobs) + a256(8 * (size_t)(n_jobs + 1));
  // A graph keeps the addresses it was captured with, so a graph batch owns plain device
  // memory; any other batch draws from the stream-ordered pool, so that creating and freeing
  // one per request group (a server's admission tick) never synchronises the device.
  b->async_scratch = !c.use_graph;
  b->alloc_stream = s;
  cudaError_t e = b->async_scratch ? cudaMallocAsync(&b->scratch, b->scratch_bytes, s)
                                   : cudaMalloc(&b->scratch, b->scratch_bytes);
  if (e != cudaSuccess) {
    b->scratch = nullptr;
    delete b;
    return cuda_error(e, "batch scratch allocation");
  }
  char* p = b->scratch;
  b->counter = reinterpret_cast<unsigned*>(p);
  b->status = b->counter + 1;
  b->total = reinterpret_cast<int64_t*>(p + 8);  // total and a spare word
  p += 256;
  b->tile_sum = reinterpret_cast<int64_t*>(p);
  p += a256(8 * (size_t)T + 8);
  b->tile_prefix = reinterpret_cast<int64_t*>(p);
  p += a256(8 * (size_t)T + 8);
  b->counts = reinterpret_cast<int32_t*>(p);
  p += a256(4 * (size_t)slots);
  b->nruns = reinterpret_cast<uint8_t*>(p);
  p += a256((size_t)slots);
  b->runs = reinterpret_cast<uint2*>(p);
  p += a256(sizeof(uint2) * kMaxRuns * (size_t)slots);
  b->job_totals = reinterpret_cast<int64_t*>(p);
  p += a256(8 * (size_t)n_jobs);
  b->job_status = reinterpret_cast<unsigned*>(p);
  p += a256(4 * (size_t)n_jobs);
  b->jobs = reinterpret_cast<JobDev*>(p);
  p += a256(sizeof(JobDev) * n_jobs);
  b->tile0 = reinterpret_cast<int64_t*>(p);
  st = HDDA_OK;
  e = cudaMemcpyAsync(b->jobs, host.data(), sizeof(JobDev) * n_jobs, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->tile0, tile0.data(), 8 * (size_t)(n_jobs + 1), cudaMemcpyHostToDevice,
                        s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host tables may go out of scope
  if (e != cudaSuccess) st = cuda_error(e, "batch tables");
  if (st == HDDA_OK) {
    const bool skip = c.walk_variant == HDDA_WALK_SKIP;
    switch (mode) {
      case kModeDense:
        st = walk_grid_for_block<kModeDense>(c.walk_block, skip, &b->walk_grid);
        break;
      case kModeVdb:
        st = walk_grid_for_block<kModeVdb>(c.walk_block, skip, &b->walk_grid);
        break;
      default:
        st = walk_grid_for_block<kModeVdbMap>(c.walk_block, skip, &b->walk_grid);
        break;
    }
  }
  if (st == HDDA_OK && c.use_graph) {
    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const int est = enqueue(b, cs);
      cudaGraph_t graph = nullptr;
      e = cudaStreamEndCapture(cs, &graph);
      if (est != HDDA_OK) st = est;
      b->graph = graph;
    }
    if (st == HDDA_OK && e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (cs) cudaStreamDestroy(cs);
    if (st == HDDA_OK && e != cudaSuccess) st = cuda_error(e, "batch graph capture");
  }
  if (st != HDDA_OK) {
    hdda_batch_free(b);
    return st;
  }
  *out = b;
  return HDDA_OK;
}

}  // namespace
}  // namespace hdda

using namespace hdda;

extern "C" int hdda_batch_create(const hdda_job* jobs, int n_jobs, const hdda_batch_config* cfg,
                                 hdda_batch** out, hdda_stream_t stream) {
  clear_error();
  return create(jobs, n_jobs, cfg, out, (cudaStream_t)stream);
}

extern "C" int hdda_batch_launch(hdda_batch* b, hdda_stream_t stream) {
  clear_error();
  if (!b) return set_error(HDDA_ERR_INVALID_ARG, "batch is NULL");
  int dev = 0;
  HDDA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != b->device) return set_error(HDDA_ERR_INVALID_ARG, "batch lives on another device");
  KernelTimer kt("batch", (cudaStream_t)stream);
  if (b->exec) {
    HDDA_CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return HDDA_OK;
  }
  return enqueue(b, (cudaStream_t)stream);
}

extern "C" int hdda_batch_results(hdda_batch* b, int64_t* totals, uint32_t* status,
                                  hdda_stream_t stream) {
  clear_error();
  if (!b) return set_error(HDDA_ERR_INVALID_ARG, "batch is NULL");
  const cudaStream_t s = (cudaStream_t)stream;
  std::vector<int64_t> t(b->n_jobs);
  std::vector<unsigned> js(b->n_jobs);
  unsigned hdr[2] = {0, 0};
  HDDA_CUDA_TRY(cudaMemcpyAsync(t.data(), b->job_totals, 8 * (size_t)b->n_jobs,
                                cudaMemcpyDeviceToHost, s));
  HDDA_CUDA_TRY(cudaMemcpyAsync(js.data(), b->job_status, 4 * (size_t)b->n_jobs,
                                cudaMemcpyDeviceToHost, s));
  HDDA_CUDA_TRY(cudaMemcpyAsync(hdr, b->counter, sizeof(hdr), cudaMemcpyDeviceToHost, s));
  HDDA_CUDA_TRY(cudaStreamSynchronize(s));
  int worst = HDDA_OK;
  for (int j = 0; j < b->n_jobs; ++j) {
    if (totals) totals[j] = t[j];
    const int code = (js[j] & kJobCapacity) ? HDDA_ERR_CAPACITY : HDDA_OK;
    if (status) status[j] = (uint32_t)code;
    if (code != HDDA_OK) worst = code;
  }
  if (hdr[1] & kDevInternal) return set_error(HDDA_ERR_INTERNAL, "region check failed");
  if (worst != HDDA_OK) return set_error(worst, "a job's outputs are smaller than its samples");
  return HDDA_OK;
}

extern "C" void hdda_batch_free(hdda_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->scratch) {
    if (b->async_scratch) {
      cudaFreeAsync(b->scratch, b->alloc_stream);  // after the batch's work on that stream
    } else {
      cudaDeviceSynchronize();
      cudaFree(b->scratch);
    }
  }
  delete b;
}
