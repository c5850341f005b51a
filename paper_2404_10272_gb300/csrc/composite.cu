// composite.cu -- front-to-back compositing of stored samples over a
// Gaussian-blob field (Sec. 1: the sampled points' densities and colours are
// accumulated into the pixel).  The blob field, its culling and the
// per-chunk accumulation are in field.cuh.
//
// Work split: a warp owns kRaysPerWarp consecutive rays, whose samples are
// one contiguous range of the CSR arrays, and walks that range 32 samples at
// a time, one sample per lane, so every lane has work whatever the rays'
// lengths.  One warp per task and small CTAs let the hardware scheduler
// balance tasks of uneven cost; tasks of 4 rays (about 170 samples in the
// object-centric frame, 750 in the unbounded one) keep the last tasks short,
// measured faster than 8, 16 or 2.
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
  __shared__ float s_T[kWarpsPerCta][32];
  __shared__ float4 s_C[kWarpsPerCta][32];
  const FieldSmem fs = stage_blobs(smem, field, G);
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* T_s = s_T[wib];
  float4* C_s = s_C[wib];
  unsigned long long evals = 0;  // this warp's blob evaluations
  const int64_t wg = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (wg * kRaysPerWarp < n) {
    const int64_t r = wg * kRaysPerWarp + lane;
    const bool has_ray = lane < kRaysPerWarp && r < n;
    const int64_t rr = has_ray ? r : min(wg * kRaysPerWarp + kRaysPerWarp, n);
    const int64_t sb = offsets[rr];
    const int64_t se = has_ray ? offsets[r + 1] : sb;
    float o[3] = {0.f, 0.f, 0.f}, d[3] = {0.f, 0.f, 0.f};
    if (has_ray) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        o[c] = __ldg(ro + 3 * r + c);
        d[c] = __ldg(rd + 3 * r + c);
      }
    }
    T_s[lane] = 1.f;
    C_s[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();
    const int64_t wbeg = __shfl_sync(kFull, sb, 0);
    const int64_t wend = __shfl_sync(kFull, se, 31);
    const int sbr = (int)(sb - wbeg);  // a warp's samples fit in 32 bits (4 rays)
    // the next chunk's interval ends are loaded one chunk ahead, so their
    // DRAM latency overlaps the current chunk's field evaluation
    float n0 = 0.f, n1 = 0.f;
    if (wbeg + lane < wend) {
      n0 = __ldg(t0 + wbeg + lane);
      n1 = __ldg(t1 + wbeg + lane);
    }
    for (int64_t base = wbeg; base < wend; base += 32) {
      const int64_t p = base + lane;
      const bool live = p < wend;
      const float c0 = n0, c1 = n1;
      if (p + 32 < wend) {
        n0 = __ldg(t0 + p + 32);
        n1 = __ldg(t1 + p + 32);
      }
      const int pr = (int)(p - wbeg);
      int own = 0;  // the last ray slot whose first sample is <= p
#pragma unroll
      for (int s = kRaysPerWarp / 2; s > 0; s >>= 1) {
        const int v = __shfl_sync(kFull, sbr, own + s);
        if (v <= pr) own += s;
      }
      const float ox = __shfl_sync(kFull, o[0], own), oy = __shfl_sync(kFull, o[1], own),
                  oz = __shfl_sync(kFull, o[2], own);
      const float dx = __shfl_sync(kFull, d[0], own), dy = __shfl_sync(kFull, d[1], own),
                  dz = __shfl_sync(kFull, d[2], own);
      float a0 = 0.f, a1 = 0.f, px = 0.f, py = 0.f, pz = 0.f;
      if (live) {
        a0 = c0;
        a1 = c1;
        const float tm = 0.5f * (a0 + a1);
        px = fmaf(tm, dx, ox);
        py = fmaf(tm, dy, oy);
        pz = fmaf(tm, dz, oz);
      }
      evals += composite_chunk(fs, G, live, p + 1 >= wend, own, px, py, pz, a0, a1, T_s, C_s);
    }
    if (has_ray) {
      const float4 acc = C_s[lane];
      reinterpret_cast<float4*>(rgba)[r] = make_float4(acc.x, acc.y, acc.z, 1.f - T_s[lane]);
    }
    if (count_evals && lane == 0) atomicAdd(&g_blob_evals, evals);
  }
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
