// composite.cu -- front-to-back compositing of the kept intervals over a
// Gaussian-blob field (Sec. 1: the sampled points' densities and colours are
// accumulated into the pixel).  The blob field stands in for the trained
// radiance field.
//
// Work split: a warp owns kRaysPerWarp consecutive rays, whose samples are
// one contiguous range of the CSR arrays, and walks that range 32 samples at
// a time, one sample per lane, so every lane has work whatever the rays'
// lengths.  One warp per task and small CTAs let the hardware scheduler
// balance tasks of uneven cost.  Each lane evaluates the field at its
// sample's midpoint; a segmented warp scan (segments = rays) turns the
// per-sample (1 - alpha) into transmittance inside the chunk, the owning
// ray's transmittance so far is carried in shared memory from chunk to
// chunk, and a segmented sum adds each ray's colour contributions at the
// segment's last lane.  Blob parameters sit in shared memory with the
// exponent prescaled for exp2.
//
// Blob culling: before evaluating a chunk, the warp takes the bounding box
// of its 32 sample points and keeps, in a shared-memory list, only the blobs
// whose centre lies within kCullSigmas standard deviations of that box.  A
// dropped blob's weight at any of those points is below
// a * exp(-kCullSigmas^2 / 2) = a * e^-24.5, about 2e-11 of its amplitude,
// so the sums change far below the compositor's 1e-5 tolerance; in the
// object-centric scene about 20 of 64 blobs survive per chunk.  Each blob's
// weight is one exp2 of fma(d^2, -log2(e) / (2 s^2), log2(a)), so amplitudes
// must be non-negative.
#include <cmath>

#include "hdda_internal.cuh"

namespace hdda {
namespace {

constexpr int kMaxGauss = 256;
constexpr int kWarpsPerCta = 4;
constexpr int kRaysPerWarp = 16;
constexpr float kCullSigmas = 7.f;
constexpr unsigned kFull = 0xffffffffu;

// Blob evaluations (sample x kept blob), counted only while profiling.
__device__ unsigned long long g_blob_evals;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Segmented inclusive scan over the warp; `head` marks a segment's first lane.
template <typename Op>
__device__ __forceinline__ float seg_scan(float v, bool head, int lane, Op op) {
  unsigned f = head;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float y = __shfl_up_sync(kFull, v, o);
    const unsigned g = __shfl_up_sync(kFull, f, o);
    if (lane >= o) {
      if (!f) v = op(y, v);
      f |= g;
    }
  }
  return v;
}

__global__ void __launch_bounds__(kWarpsPerCta * 32) composite_kernel(
    const float* __restrict__ ro, const float* __restrict__ rd, int64_t n,
    const int64_t* __restrict__ offsets, const float* __restrict__ t0,
    const float* __restrict__ t1, const float* __restrict__ field, int G,
    float* __restrict__ rgba, bool count_evals) {
  __shared__ float4 gpos[kMaxGauss];  // mu_x, mu_y, mu_z, -log2(e) / (2 s^2)
  __shared__ float4 gcol[kMaxGauss];  // log2(a), r, g, b
  __shared__ float gcut[kMaxGauss];   // (kCullSigmas * s)^2
  __shared__ uint16_t s_list[kWarpsPerCta][kMaxGauss];  // blobs kept for the current chunk
  __shared__ float s_T[kWarpsPerCta][32];
  __shared__ float4 s_C[kWarpsPerCta][32];
  for (int i = threadIdx.x; i < G; i += blockDim.x) {
    const float* f = field + 8 * i;
    const float s = f[3];
    gpos[i] = make_float4(f[0], f[1], f[2], -1.4426950408889634f / (2.f * s * s));
    gcol[i] = make_float4(log2f(f[4]), f[5], f[6], f[7]);
    gcut[i] = (kCullSigmas * s) * (kCullSigmas * s);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* T_s = s_T[wib];
  float4* C_s = s_C[wib];
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
    for (int64_t base = wbeg; base < wend; base += 32) {
      const int64_t p = base + lane;
      const bool live = p < wend;
      int own = 0;  // the last lane whose first sample is <= p
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) {
        const int64_t v = __shfl_sync(kFull, sb, own + s);
        if (v <= p) own += s;
      }
      float alpha = 0.f, wr = 0.f, wgr = 0.f, wb = 0.f;
      {
        const float ox = __shfl_sync(kFull, o[0], own), oy = __shfl_sync(kFull, o[1], own),
                    oz = __shfl_sync(kFull, o[2], own);
        const float dx = __shfl_sync(kFull, d[0], own), dy = __shfl_sync(kFull, d[1], own),
                    dz = __shfl_sync(kFull, d[2], own);
        float a0 = 0.f, a1 = 0.f, px = 0.f, py = 0.f, pz = 0.f;
        if (live) {
          a0 = __ldg(t0 + p);
          a1 = __ldg(t1 + p);
          const float tm = 0.5f * (a0 + a1);
          px = ox + tm * dx;
          py = oy + tm * dy;
          pz = oz + tm * dz;
        }
        // bounding box of the chunk's points, then the blobs within reach of it
        float bx0 = live ? px : INFINITY, by0 = live ? py : INFINITY, bz0 = live ? pz : INFINITY;
        float bx1 = live ? px : -INFINITY, by1 = live ? py : -INFINITY, bz1 = live ? pz : -INFINITY;
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
          bx0 = fminf(bx0, __shfl_xor_sync(kFull, bx0, o2));
          by0 = fminf(by0, __shfl_xor_sync(kFull, by0, o2));
          bz0 = fminf(bz0, __shfl_xor_sync(kFull, bz0, o2));
          bx1 = fmaxf(bx1, __shfl_xor_sync(kFull, bx1, o2));
          by1 = fmaxf(by1, __shfl_xor_sync(kFull, by1, o2));
          bz1 = fmaxf(bz1, __shfl_xor_sync(kFull, bz1, o2));
        }
        uint16_t* list = s_list[wib];
        int m = 0;
        for (int q0 = 0; q0 < G; q0 += 32) {
          bool near = false;
          if (q0 + lane < G) {
            const float4 P = gpos[q0 + lane];
            const float ex = fmaxf(0.f, fmaxf(bx0 - P.x, P.x - bx1));
            const float ey = fmaxf(0.f, fmaxf(by0 - P.y, P.y - by1));
            const float ez = fmaxf(0.f, fmaxf(bz0 - P.z, P.z - bz1));
            near = ex * ex + ey * ey + ez * ez <= gcut[q0 + lane];
          }
          const unsigned ball = __ballot_sync(kFull, near);
          if (near) list[m + __popc(ball & ((1u << lane) - 1u))] = (uint16_t)(q0 + lane);
          m += __popc(ball);
        }
        if (count_evals && lane == 0)
          atomicAdd(&g_blob_evals, (unsigned long long)m * (unsigned long long)min(wend - base, (int64_t)32));
        __syncwarp();
        float sigma = 0.f, sr = 0.f, sg = 0.f, sbl = 0.f;
        for (int i = 0; i < m; ++i) {
          const int q = list[i];
          const float4 P = gpos[q];
          const float ex = px - P.x, ey = py - P.y, ez = pz - P.z;
          const float d2 = ex * ex + ey * ey + ez * ez;
          const float4 C = gcol[q];
          const float w = ex2_approx(fmaf(d2, P.w, C.x));
          sigma += w;
          sr = fmaf(w, C.y, sr);
          sg = fmaf(w, C.z, sg);
          sbl = fmaf(w, C.w, sbl);
        }
        __syncwarp();
        if (live) {
          alpha = -expm1f(-sigma * (a1 - a0));
          if (sigma > 0.f) {
            const float inv = alpha / sigma;
            wr = sr * inv;
            wgr = sg * inv;
            wb = sbl * inv;
          }
        }
      }
      const int own_prev = __shfl_up_sync(kFull, own, 1);
      const int own_next = __shfl_down_sync(kFull, own, 1);
      const bool head = lane == 0 || own_prev != own;
      const bool tail = live && (lane == 31 || own_next != own || p + 1 >= wend);
      const float keep = 1.f - alpha;
      const float incl = seg_scan(keep, head, lane, [](float a, float b) { return a * b; });
      float excl = __shfl_up_sync(kFull, incl, 1);
      if (head) excl = 1.f;
      const float Tj = T_s[own] * excl;
      const auto add = [](float a, float b) { return a + b; };
      const float cr = seg_scan(Tj * wr, head, lane, add);
      const float cg = seg_scan(Tj * wgr, head, lane, add);
      const float cb = seg_scan(Tj * wb, head, lane, add);
      const float T_end = T_s[own] * incl;
      __syncwarp();
      if (tail) {
        T_s[own] = T_end;
        float4 acc = C_s[own];
        acc.x += cr;
        acc.y += cg;
        acc.z += cb;
        C_s[own] = acc;
      }
      __syncwarp();
    }
    if (has_ray) {
      const float4 acc = C_s[lane];
      reinterpret_cast<float4*>(rgba)[r] = make_float4(acc.x, acc.y, acc.z, 1.f - T_s[lane]);
    }
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
  composite_kernel<<<grid, kWarpsPerCta * 32, 0, (cudaStream_t)stream>>>(
      rays_o, rays_d, n_rays, offsets, t0, t1, field, n_gauss, rgba_out, profiler_on());
  kt.stop();
  HDDA_CUDA_TRY(cudaGetLastError());
  return HDDA_OK;
}
