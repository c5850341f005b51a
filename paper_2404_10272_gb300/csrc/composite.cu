// composite.cu -- front-to-back compositing of the kept intervals over a
// Gaussian-blob field (Sec. 1: the sampled points' densities and colours are
// accumulated into the pixel).  The blob field stands in for the trained
// radiance field.
//
// One warp per ray.  The warp takes the ray's samples 32 at a time: each
// lane evaluates the field at its sample's midpoint, a warp product scan of
// (1 - alpha) gives every sample its transmittance inside the chunk, and the
// chunk's product carries to the next one.  Each lane keeps its own colour
// partial sums, reduced once at the end.  Blob parameters sit in shared
// memory; the exponent is prescaled so that one exp2 serves each blob.
#include <cmath>

#include "hdda_internal.cuh"

namespace hdda {
namespace {

constexpr int kMaxGauss = 256;
constexpr int kWarpsPerCta = 8;
constexpr unsigned kFull = 0xffffffffu;

__global__ void __launch_bounds__(kWarpsPerCta * 32) composite_kernel(
    const float* __restrict__ ro, const float* __restrict__ rd, int64_t n,
    const int64_t* __restrict__ offsets, const float* __restrict__ t0,
    const float* __restrict__ t1, const float* __restrict__ field, int G,
    float* __restrict__ rgba) {
  __shared__ float4 gpos[kMaxGauss];  // mu_x, mu_y, mu_z, -log2(e) / (2 s^2)
  __shared__ float4 gcol[kMaxGauss];  // a, r, g, b
  for (int i = threadIdx.x; i < G; i += blockDim.x) {
    const float* f = field + 8 * i;
    const float s = f[3];
    gpos[i] = make_float4(f[0], f[1], f[2], -1.4426950408889634f / (2.f * s * s));
    gcol[i] = make_float4(f[4], f[5], f[6], f[7]);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp0; r < n; r += nwarps) {
    const int64_t s0 = offsets[r], s1 = offsets[r + 1];
    const float ox = __ldg(ro + 3 * r), oy = __ldg(ro + 3 * r + 1), oz = __ldg(ro + 3 * r + 2);
    const float dx = __ldg(rd + 3 * r), dy = __ldg(rd + 3 * r + 1), dz = __ldg(rd + 3 * r + 2);
    float T = 1.f;
    float cr = 0.f, cg = 0.f, cb = 0.f;
    for (int64_t base = s0; base < s1; base += 32) {
      const int64_t j = base + lane;
      float alpha = 0.f, keep = 1.f, wr = 0.f, wg = 0.f, wb = 0.f;
      if (j < s1) {
        const float a0 = __ldg(t0 + j), a1 = __ldg(t1 + j);
        const float tm = 0.5f * (a0 + a1);
        const float px = ox + tm * dx, py = oy + tm * dy, pz = oz + tm * dz;
        float sigma = 0.f, sr = 0.f, sg = 0.f, sb = 0.f;
        for (int q = 0; q < G; ++q) {
          const float4 P = gpos[q];
          const float ex = px - P.x, ey = py - P.y, ez = pz - P.z;
          const float d2 = ex * ex + ey * ey + ez * ez;
          const float4 C = gcol[q];
          const float w = C.x * exp2f(d2 * P.w);
          sigma += w;
          sr += w * C.y;
          sg += w * C.z;
          sb += w * C.w;
        }
        const float od = sigma * (a1 - a0);
        alpha = -expm1f(-od);
        keep = expf(-od);
        if (sigma > 0.f) {
          const float inv = alpha / sigma;
          wr = sr * inv;
          wg = sg * inv;
          wb = sb * inv;
        }
      }
      // inclusive product scan of keep across the chunk
      float inc = keep;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc *= y;
      }
      float excl = __shfl_up_sync(kFull, inc, 1);
      if (lane == 0) excl = 1.f;
      const float Tj = T * excl;
      cr += Tj * wr;
      cg += Tj * wg;
      cb += Tj * wb;
      T *= __shfl_sync(kFull, inc, 31);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      cr += __shfl_xor_sync(kFull, cr, o);
      cg += __shfl_xor_sync(kFull, cg, o);
      cb += __shfl_xor_sync(kFull, cb, o);
    }
    if (lane == 0) {
      reinterpret_cast<float4*>(rgba)[r] = make_float4(cr, cg, cb, 1.f - T);
    }
  }
}

}  // namespace
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
  int dev = 0, sms = 0;
  HDDA_CUDA_TRY(cudaGetDevice(&dev));
  HDDA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t want = (n_rays + kWarpsPerCta - 1) / kWarpsPerCta;
  const int64_t cap = (int64_t)sms * 8;  // persistent: a few CTAs per SM
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  KernelTimer kt("composite", (cudaStream_t)stream);
  composite_kernel<<<grid, kWarpsPerCta * 32, 0, (cudaStream_t)stream>>>(
      rays_o, rays_d, n_rays, offsets, t0, t1, field, n_gauss, rgba_out);
  kt.stop();
  HDDA_CUDA_TRY(cudaGetLastError());
  return HDDA_OK;
}
