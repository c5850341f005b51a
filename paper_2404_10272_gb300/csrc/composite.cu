// composite.cu -- front-to-back compositing of stored samples over a
// Gaussian-blob field (Sec. 1: the sampled points' densities and colours are
// accumulated into the pixel).  The blob field, its culling and the
// per-chunk accumulation are in field.cuh.
//
// Work split: a warp owns kRaysPerWarp consecutive rays, whose samples are
// one contiguous range of the CSR arrays, and walks that range 64 samples at
// a time, two per lane (field.cuh), so every lane has work whatever the rays'
// lengths.  One warp per task and small CTAs let the hardware scheduler
// balance tasks of uneven cost; tasks of 4 rays (about 170 samples in the
// object-centric frame, 750 in the unbounded one) keep the last tasks short.
// The task's rays (origin, direction) are staged in shared memory, and
// every lane keeps the rays' first sample positions in registers, so a
// sample finds its ray by compares.
#include "field.cuh"

namespace hdda {
namespace {

constexpr int kWarpsPerCta = 4;
constexpr int kRaysPerWarp = 4;
constexpr unsigned kFull = 0xffffffffu;

// Blob evaluations (sample x kept blob), counted only while profiling.
__device__ unsigned long long g_blob_evals;

__global__ void __launch_bounds__(kWarpsPerCta * 32, 8) composite_kernel(
    const float* __restrict__ ro, const float* __restrict__ rd, int64_t n,
    const int64_t* __restrict__ offsets, const float* __restrict__ t0,
    const float* __restrict__ t1, const float* __restrict__ field, int G,
    float* __restrict__ rgba, bool count_evals) {
  extern __shared__ __align__(16) unsigned char smem[];  // field_smem_bytes(G, kWarpsPerCta)
  __shared__ float s_T[kWarpsPerCta][kRaysPerWarp];
  __shared__ float4 s_C[kWarpsPerCta][kRaysPerWarp];
  __shared__ uint16_t s_cand[kWarpsPerCta][kMaxGauss];  // the task's candidate blobs
  __shared__ float4 s_ray[kWarpsPerCta][kRaysPerWarp][2];  // {o, d.x}, {d.y, d.z, 1/|d|^2, -}
  const FieldSmem fs = stage_blobs(smem, field, G);
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* T_s = s_T[wib];
  float4* C_s = s_C[wib];
  float4(*rs)[2] = s_ray[wib];
  unsigned long long evals = 0;  // this warp's blob evaluations
  const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (wg * kRaysPerWarp >= n) return;  // uniform per warp; no block barrier follows
  const int64_t r = wg * kRaysPerWarp + lane;
  const bool has_ray = lane < kRaysPerWarp && r < n;
  const int64_t rr = has_ray ? r : min(wg * kRaysPerWarp + kRaysPerWarp, n);
  const int64_t sb = offsets[rr];
  const int64_t se = has_ray ? offsets[r + 1] : sb;
  if (lane < kRaysPerWarp) {
    float o[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 0.f};
    if (has_ray) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        o[c] = __ldg(ro + 3 * r + c);
        d[c] = __ldg(rd + 3 * r + c);
      }
    }
    const float dd = fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2]));
    rs[lane][0] = make_float4(o[0], o[1], o[2], d[0]);
    rs[lane][1] = make_float4(d[1], d[2], dd > 1e-30f ? 1.f / dd : 0.f, 0.f);
    T_s[lane] = 1.f;
    C_s[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncwarp();
  const int64_t wbeg = __shfl_sync(kFull, sb, 0);
  const int64_t wend = __shfl_sync(kFull, se, kRaysPerWarp - 1);
  // first sample of rays 1 .. kRaysPerWarp - 1 relative to the warp's first sample (a
  // task's samples fit in 32 bits)
  int sfirst[kRaysPerWarp];
#pragma unroll
  for (int i = 1; i < kRaysPerWarp; ++i) sfirst[i] = (int)(__shfl_sync(kFull, sb, i) - wbeg);
  const int total = (int)(wend - wbeg);
  // a task of more than two chunks first narrows the field to the blobs near its rays'
  // lines; a shorter one tests every blob in its chunks (the narrowing would cost more
  // than it saves)
  uint16_t* cand = s_cand[wib];
  int ncand = G;
  if (total > 2 * kChunk) {
    ncand = task_candidates(fs, G, rs, (int)min((int64_t)kRaysPerWarp, n - wg * kRaysPerWarp),
                            cand);
  } else {
    for (int q = lane; q < G; q += 32) cand[q] = (uint16_t)q;
    __syncwarp();
  }
  // the next chunk's interval ends are loaded one chunk ahead, so their
  // DRAM latency overlaps the current chunk's field evaluation
  float n0a = 0.f, n1a = 0.f, n0b = 0.f, n1b = 0.f;
  if (2 * lane < total) {
    n0a = __ldg(t0 + wbeg + 2 * lane);
    n1a = __ldg(t1 + wbeg + 2 * lane);
  }
  if (2 * lane + 1 < total) {
    n0b = __ldg(t0 + wbeg + 2 * lane + 1);
    n1b = __ldg(t1 + wbeg + 2 * lane + 1);
  }
  for (int base = 0; base < total; base += kChunk) {
    const int nlive = min(kChunk, total - base);
    Elem e[2];
    e[0].a0 = n0a; e[0].a1 = n1a; e[1].a0 = n0b; e[1].a1 = n1b;
    const int pa = base + kChunk + 2 * lane;
    if (pa < total) {
      n0a = __ldg(t0 + wbeg + pa);
      n1a = __ldg(t1 + wbeg + pa);
    }
    if (pa + 1 < total) {
      n0b = __ldg(t0 + wbeg + pa + 1);
      n1b = __ldg(t1 + wbeg + pa + 1);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int p = base + 2 * lane + h;
      int own = 0;  // the last ray starting at or before p
#pragma unroll
      for (int i = 1; i < kRaysPerWarp; ++i) own += p >= sfirst[i];
      e[h].own = own;
      e[h].px = e[h].py = e[h].pz = 0.f;
      if (p < total) {
        const float4 A = rs[own][0], B = rs[own][1];
        const float tm = 0.5f * (e[h].a0 + e[h].a1);
        e[h].px = fmaf(tm, A.w, A.x);
        e[h].py = fmaf(tm, B.x, A.y);
        e[h].pz = fmaf(tm, B.y, A.z);
      }
    }
    evals += composite_chunk2(fs, cand, ncand, nlive, e[0], e[1], rs, T_s, C_s);
  }
  if (has_ray) {
    const float4 acc = C_s[lane];
    reinterpret_cast<float4*>(rgba)[r] = make_float4(acc.x, acc.y, acc.z, 1.f - T_s[lane]);
  }
  if (count_evals && lane == 0) atomicAdd(&g_blob_evals, evals);
}

}  // namespace

unsigned long long composite_take_blob_evals() {
  unsigned long long v = 0, zero = 0;
  if (cudaMemcpyFromSymbol(&v, g_blob_evals, sizeof(v)) != cudaSuccess) return 0;
  cudaMemcpyToSymbol(g_blob_evals, &zero, sizeof(zero));
  return v;
}

}  // namespace hdda

extern "C" int hdda_composite(const float* rays_o, const float* rays_d, int64_t n_rays,
                              const int64_t* offsets, const float* t0, const float* t1,
                              const float* field, int n_gauss, float* rgba_out,
                              hdda_stream_t stream) {
  using namespace hdda;
  clear_error();
  if (n_rays < 0) return set_error(HDDA_ERR_INVALID_ARG, "n_rays < 0");
  if (n_gauss < 0 || n_gauss > kMaxGauss)
    return set_error(HDDA_ERR_INVALID_ARG, "n_gauss=%d outside 0..%d", n_gauss, kMaxGauss);
  if (n_rays == 0) return HDDA_OK;
  if (!rays_o || !rays_d || !offsets || !rgba_out || (n_gauss > 0 && !field))
    return set_error(HDDA_ERR_INVALID_ARG, "NULL pointer");
  if (reinterpret_cast<uintptr_t>(rgba_out) % 16 != 0)
    return set_error(HDDA_ERR_INVALID_ARG, "rgba_out must be 16-byte aligned");
  const int64_t warps = (n_rays + kRaysPerWarp - 1) / kRaysPerWarp;
  const int64_t blocks = (warps + kWarpsPerCta - 1) / kWarpsPerCta;
  if (blocks > INT32_MAX) return set_error(HDDA_ERR_INVALID_ARG, "too many rays");
  const unsigned grid = (unsigned)blocks;
  KernelTimer kt("composite", (cudaStream_t)stream);
  composite_kernel<<<grid, kWarpsPerCta * 32, field_smem_bytes(n_gauss, kWarpsPerCta),
                     (cudaStream_t)stream>>>(
      rays_o, rays_d, n_rays, offsets, t0, t1, field, n_gauss, rgba_out, counters_on());
  kt.stop();
  HDDA_CUDA_TRY(cudaGetLastError());
  return HDDA_OK;
}
