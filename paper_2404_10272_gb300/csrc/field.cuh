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

// The field in shared memory, prescaled for exp2.
struct BlobTables {
  float4 pos[kMaxGauss];  // mu_x, mu_y, mu_z, -log2(e) / (2 s^2)
  float4 col[kMaxGauss];  // log2(a), r, g, b
  float cut[kMaxGauss];   // (kCullSigmas * s)^2
};

// Block-wide copy of `G` blobs of 8 floats {mu[3], s, a, rgb[3]}; the caller
// synchronises the block afterwards.
__device__ __forceinline__ void stage_blobs(BlobTables& bt, const float* __restrict__ field,
                                            int G) {
  for (int i = threadIdx.x; i < G; i += blockDim.x) {
    const float* f = field + 8 * i;
    const float s = f[3];
    bt.pos[i] = make_float4(f[0], f[1], f[2], -1.4426950408889634f / (2.f * s * s));
    bt.col[i] = make_float4(log2f(f[4]), f[5], f[6], f[7]);
    bt.cut[i] = (kCullSigmas * s) * (kCullSigmas * s);
  }
}

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
    const float y = __shfl_up_sync(kFieldFull, v, o);
    const unsigned g = __shfl_up_sync(kFieldFull, f, o);
    if (lane >= o) {
      if (!f) v = op(y, v);
      f |= g;
    }
  }
  return v;
}

// One 32-sample chunk.  Lane `lane` holds a sample when `live`: the interval
// [a0, a1) of the ray in slot `own`, evaluated at point (px, py, pz).  Live
// lanes come first and are in ray order; `last` marks the lane holding the
// warp's final sample.  Updates T_s[own] and C_s[own].  `evals`, when
// non-null, counts sample x kept-blob evaluations.
__device__ __forceinline__ void composite_chunk(const BlobTables& bt, int G, uint16_t* list,
                                                bool live, bool last, int own, float px,
                                                float py, float pz, float a0, float a1,
                                                float* T_s, float4* C_s,
                                                unsigned long long* evals) {
  const int lane = threadIdx.x & 31;
  float alpha = 0.f, wr = 0.f, wgr = 0.f, wb = 0.f;
  {
    // bounding box of the chunk's points, then the blobs within reach of it
    float bx0 = live ? px : INFINITY, by0 = live ? py : INFINITY, bz0 = live ? pz : INFINITY;
    float bx1 = live ? px : -INFINITY, by1 = live ? py : -INFINITY, bz1 = live ? pz : -INFINITY;
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
      bx0 = fminf(bx0, __shfl_xor_sync(kFieldFull, bx0, o2));
      by0 = fminf(by0, __shfl_xor_sync(kFieldFull, by0, o2));
      bz0 = fminf(bz0, __shfl_xor_sync(kFieldFull, bz0, o2));
      bx1 = fmaxf(bx1, __shfl_xor_sync(kFieldFull, bx1, o2));
      by1 = fmaxf(by1, __shfl_xor_sync(kFieldFull, by1, o2));
      bz1 = fmaxf(bz1, __shfl_xor_sync(kFieldFull, bz1, o2));
    }
    int m = 0;
    for (int q0 = 0; q0 < G; q0 += 32) {
      bool near = false;
      if (q0 + lane < G) {
        const float4 P = bt.pos[q0 + lane];
        const float ex = fmaxf(0.f, fmaxf(bx0 - P.x, P.x - bx1));
        const float ey = fmaxf(0.f, fmaxf(by0 - P.y, P.y - by1));
        const float ez = fmaxf(0.f, fmaxf(bz0 - P.z, P.z - bz1));
        near = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= bt.cut[q0 + lane];
      }
      const unsigned ball = __ballot_sync(kFieldFull, near);
      if (near) list[m + __popc(ball & ((1u << lane) - 1u))] = (uint16_t)(q0 + lane);
      m += __popc(ball);
    }
    if (evals) {
      const int nl = __popc(__ballot_sync(kFieldFull, live));
      if (lane == 0) atomicAdd(evals, (unsigned long long)m * (unsigned long long)nl);
    }
    __syncwarp();
    float sigma = 0.f, sr = 0.f, sg = 0.f, sbl = 0.f;
    for (int i = 0; i < m; ++i) {
      const int q = list[i];
      const float4 P = bt.pos[q];
      const float ex = px - P.x, ey = py - P.y, ez = pz - P.z;
      const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
      const float4 C = bt.col[q];
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
  const int own_prev = __shfl_up_sync(kFieldFull, own, 1);
  const int own_next = __shfl_down_sync(kFieldFull, own, 1);
  const bool head = lane == 0 || own_prev != own;
  const bool tail = live && (lane == 31 || own_next != own || last);
  const float keep = 1.f - alpha;
  const float incl = seg_scan(keep, head, lane, [](float a, float b) { return a * b; });
  float excl = __shfl_up_sync(kFieldFull, incl, 1);
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

}  // namespace
}  // namespace hdda
