// field.cuh -- the Gaussian-blob field and the warp-cooperative front-to-back
// accumulation shared by the compositor over stored samples (composite.cu)
// and the render-only path that expands runs on the fly (render.cu).
//
// Sec. 1: the densities and colours at a ray's sampled points are
// accumulated into its pixel, front to back.  The blob field stands in for
// the trained radiance field: sigma(x) = sum_g a_g exp(-|x - mu_g|^2 /
// (2 s_g^2)), colour = the sigma-weighted mean of the blobs' colours.
//
// A warp works through its samples 32 at a time, one sample per lane, in ray
// order.  A segmented warp scan (segments = rays) turns the per-sample
// (1 - alpha) into transmittance inside the chunk; each ray's transmittance
// so far and its colour sum are carried in shared memory (T_s, C_s, indexed
// by the ray's slot in the warp) from chunk to chunk.
//
// Blob culling: before evaluating a chunk, the warp takes the bounding box
// of its 32 points and keeps, in a shared-memory list, only the blobs whose
// centre lies within kCullSigmas standard deviations of that box.  A dropped
// blob's weight at any of those points is below a * exp(-kCullSigmas^2 / 2)
// = a * e^-24.5, about 2e-11 of its amplitude, far below the compositor's
// 1e-5 tolerance.  Each kept blob costs one exp2 of fma(d^2, -log2(e) /
// (2 s^2), log2(a)), so amplitudes must be non-negative.  Every product-sum
// is written as an explicit fmaf, so the arithmetic does not depend on the
// translation unit's contraction flags.
#pragma once

#include <cmath>

#include "hdda_internal.cuh"

namespace hdda {
namespace {

constexpr int kMaxGauss = 256;
constexpr float kCullSigmas = 7.f;
constexpr unsigned kFieldFull = 0xffffffffu;

// One blob in shared memory, prescaled for exp2.
struct BlobRec {
  float4 pos;  // mu_x, mu_y, mu_z, -log2(e) / (2 s^2)
  float4 col;  // log2(a), r, g, b
};

// Dynamic shared memory of a compositing CTA with `warps` warps over G
// blobs: the field (records, then (kCullSigmas s)^2 per blob), then one
// list of kept records per warp.
__host__ __device__ inline size_t field_smem_bytes(int G, int warps) {
  return (size_t)G * sizeof(BlobRec) + (((size_t)G * sizeof(float) + 15) & ~(size_t)15) +
         (size_t)warps * G * sizeof(BlobRec);
}

struct FieldSmem {
  const BlobRec* tab;
  const float* cut;
  BlobRec* kept;  // this warp's list
};

// Block-wide copy of `G` blobs of 8 floats {mu[3], s, a, rgb[3]} into the
// dynamic shared memory `smem`; the caller synchronises the block afterwards.
__device__ __forceinline__ FieldSmem stage_blobs(unsigned char* smem, const float* __restrict__ field,
                                                 int G) {
  BlobRec* tab = reinterpret_cast<BlobRec*>(smem);
  float* cut = reinterpret_cast<float*>(smem + (size_t)G * sizeof(BlobRec));
  BlobRec* kept = reinterpret_cast<BlobRec*>(
      smem + (size_t)G * sizeof(BlobRec) + (((size_t)G * sizeof(float) + 15) & ~(size_t)15));
  for (int i = threadIdx.x; i < G; i += blockDim.x) {
    const float* f = field + 8 * i;
    const float s = f[3];
    tab[i].pos = make_float4(f[0], f[1], f[2], -1.4426950408889634f / (2.f * s * s));
    tab[i].col = make_float4(log2f(f[4]), f[5], f[6], f[7]);
    cut[i] = (kCullSigmas * s) * (kCullSigmas * s);
  }
  return FieldSmem{tab, cut, kept + (threadIdx.x >> 5) * G};
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Order-preserving float <-> uint32 keys, so that warp min/max reductions
// run on the integer reduction unit.
__device__ __forceinline__ uint32_t fkey(float f) {
  const uint32_t u = __float_as_uint(f);
  return u ^ ((uint32_t)((int32_t)u >> 31) | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
  return __uint_as_float(k ^ (((k >> 31) - 1u) | 0x80000000u));
}
__device__ __forceinline__ float warp_min(float v) {
  return fkey_inv(__reduce_min_sync(kFieldFull, fkey(v)));
}
__device__ __forceinline__ float warp_max(float v) {
  return fkey_inv(__reduce_max_sync(kFieldFull, fkey(v)));
}

// One 32-sample chunk.  Lane `lane` holds a sample when `live`: the interval
// [a0, a1) of the ray in slot `own`, evaluated at point (px, py, pz).  Live
// lanes come first and are in ray order; `last` marks the lane holding the
// warp's final sample.  Updates T_s[own] and C_s[own].  Returns the
// chunk's blob evaluations (live samples x kept blobs), the same on every
// lane.
__device__ __forceinline__ int composite_chunk(const FieldSmem& fs, int G, bool live, bool last,
                                               int own, float px, float py, float pz, float a0,
                                               float a1, float* T_s, float4* C_s) {
  const int lane = threadIdx.x & 31;
  float alpha = 0.f, wr = 0.f, wgr = 0.f, wb = 0.f;
  int nevals;
  {
    // bounding box of the chunk's points, then the blobs within reach of it
    const float bx0 = warp_min(live ? px : INFINITY), by0 = warp_min(live ? py : INFINITY),
                bz0 = warp_min(live ? pz : INFINITY);
    const float bx1 = warp_max(live ? px : -INFINITY), by1 = warp_max(live ? py : -INFINITY),
                bz1 = warp_max(live ? pz : -INFINITY);
    BlobRec* kept = fs.kept;
    int m = 0;
    for (int q0 = 0; q0 < G; q0 += 32) {
      const int q = q0 + lane;
      bool near = false;
      BlobRec b;
      if (q < G) {
        b = fs.tab[q];
        const float ex = fmaxf(0.f, fmaxf(bx0 - b.pos.x, b.pos.x - bx1));
        const float ey = fmaxf(0.f, fmaxf(by0 - b.pos.y, b.pos.y - by1));
        const float ez = fmaxf(0.f, fmaxf(bz0 - b.pos.z, b.pos.z - bz1));
        near = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= fs.cut[q];
      }
      const unsigned ball = __ballot_sync(kFieldFull, near);
      if (near) kept[m + __popc(ball & ((1u << lane) - 1u))] = b;
      m += __popc(ball);
    }
    nevals = m * __popc(__ballot_sync(kFieldFull, live));
    __syncwarp();
    float sigma = 0.f, sr = 0.f, sg = 0.f, sbl = 0.f;
#pragma unroll 4
    for (int i = 0; i < m; ++i) {
      const float4 P = kept[i].pos;
      const float ex = px - P.x, ey = py - P.y, ez = pz - P.z;
      const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
      const float4 C = kept[i].col;
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
        const float inv = __fdividef(alpha, sigma);
        wr = sr * inv;
        wgr = sg * inv;
        wb = sbl * inv;
      }
    }
  }
  // segments = rays: each lane's segment starts at the last head at or below it
  const int own_prev = __shfl_up_sync(kFieldFull, own, 1);
  const int own_next = __shfl_down_sync(kFieldFull, own, 1);
  const bool head = lane == 0 || own_prev != own;
  const bool tail = live && (lane == 31 || own_next != own || last);
  const unsigned heads = __ballot_sync(kFieldFull, head);
  const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
  bool in[5];
#pragma unroll
  for (int b = 0; b < 5; ++b) in[b] = lane - (1 << b) >= start;
  // transmittance through the segment (inclusive product of 1 - alpha)
  float incl = 1.f - alpha;
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    const float y = __shfl_up_sync(kFieldFull, incl, 1 << b);
    if (in[b]) incl *= y;
  }
  float excl = __shfl_up_sync(kFieldFull, incl, 1);
  if (head) excl = 1.f;
  const float T0 = T_s[own];
  const float Tj = T0 * excl;
  float cr = Tj * wr, cg = Tj * wgr, cb = Tj * wb;
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    const float yr = __shfl_up_sync(kFieldFull, cr, 1 << b);
    const float yg = __shfl_up_sync(kFieldFull, cg, 1 << b);
    const float yb = __shfl_up_sync(kFieldFull, cb, 1 << b);
    if (in[b]) {
      cr += yr;
      cg += yg;
      cb += yb;
    }
  }
  const float T_end = T0 * incl;
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
  return nevals;
}

}  // namespace
}  // namespace hdda
