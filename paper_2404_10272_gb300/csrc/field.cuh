// field.cuh -- the Gaussian-blob field and the warp-cooperative front-to-back
// accumulation shared by the compositor over stored samples (composite.cu)
// and the render-only path that expands runs on the fly (render.cu).
//
// Sec. 1: the densities and colours at a ray's sampled points are
// accumulated into its pixel, front to back.  The blob field stands in for
// the trained radiance field: sigma(x) = sum_g a_g exp(-|x - mu_g|^2 /
// (2 s_g^2)), colour = the sigma-weighted mean of the blobs' colours.
//
// A warp works through its samples 64 at a time in ray order: lane l holds
// the chunk's samples 2l and 2l + 1 ("elements" 0 and 1).  Every blob record
// the warp reads from shared memory (a broadcast) thus serves two points, and
// the two points are evaluated together with Blackwell's paired binary32
// instructions (add/mul/fma .f32x2: one issue slot for both).  The shared
// memory data path, not the arithmetic, limits a one-point-per-lane loop:
// each broadcast record costs the same wavefronts whatever the lane uses it
// for.  A segmented warp scan over the lanes' element pairs (segments = rays)
// turns the per-sample (1 - alpha) into transmittance inside the chunk; each
// ray's transmittance so far and its colour sum are carried in shared memory
// (T_s, C_s, indexed by the ray's slot in the warp) from chunk to chunk.
//
// Blob culling, in two stages.  Per warp task, the blobs within reach of the
// lines of the task's rays become its candidates (a list of indices).  Before
// evaluating a chunk, the warp keeps, in a shared-memory list, only the
// candidates whose centre lies within kCullSigmas standard deviations of the
// chunk's points: of the segments of the (one or two)
// rays the points lie on, between the smallest and largest midpoint
// parameter of each ray's samples in the chunk (single-instruction warp
// reductions over binary32, redux.sync.{min,max}.f32), or of the points'
// bounding box when the chunk spans three rays or more.  The reach carries a
// relative margin of 1e-5 for binary32 rounding, so no blob within
// kCullSigmas s of a point is dropped.  A dropped blob's weight at any of
// those points is below a * exp(-kCullSigmas^2 / 2) = a * e^-24.5, about
// 2e-11 of its amplitude, far below the compositor's 1e-5 tolerance.  Each kept blob costs one exp2 of
// fma(d^2, -log2(e) / (2 s^2), log2(a)), so amplitudes must be non-negative.
// Every product-sum is an explicit fused multiply-add, so the arithmetic
// does not depend on the translation unit's contraction flags.
#pragma once

#include <cmath>

#include "hdda_internal.cuh"

namespace hdda {
namespace {

constexpr int kMaxGauss = 256;
constexpr float kCullSigmas = 7.f;
constexpr unsigned kFieldFull = 0xffffffffu;
constexpr int kChunk = 64;  // samples per warp step: two per lane

// One blob in shared memory, prescaled for exp2; the centre is stored
// negated so that x - mu is one add.
struct BlobRec {
  float4 pos;  // -mu_x, -mu_y, -mu_z, -log2(e) / (2 s^2)
  float4 col;  // log2(a), r, g, b
};

// The culling test's view of a blob: the negated centre and its reach,
// kCullSigmas s plus a margin of 1e-5 |mu| (max norm) for binary32 rounding
// in the distance tests.
struct BlobCull {
  float4 v;  // -mu_x, -mu_y, -mu_z, reach
};

// Dynamic shared memory of a compositing CTA with `warps` warps over G
// blobs: the field records, their culling entries, then one list of kept
// records per warp.
__host__ __device__ inline size_t field_smem_bytes(int G, int warps) {
  return (size_t)G * (sizeof(BlobRec) + sizeof(BlobCull)) + (size_t)warps * G * sizeof(BlobRec);
}

struct FieldSmem {
  const BlobRec* tab;
  const BlobCull* cull;
  BlobRec* kept;  // this warp's list
};

// Block-wide copy of `G` blobs of 8 floats {mu[3], s, a, rgb[3]} into the
// dynamic shared memory `smem`; the caller synchronises the block afterwards.
__device__ __forceinline__ FieldSmem stage_blobs(unsigned char* smem, const float* __restrict__ field,
                                                 int G) {
  BlobRec* tab = reinterpret_cast<BlobRec*>(smem);
  BlobCull* cull = reinterpret_cast<BlobCull*>(smem + (size_t)G * sizeof(BlobRec));
  BlobRec* kept = reinterpret_cast<BlobRec*>(smem + (size_t)G * (sizeof(BlobRec) + sizeof(BlobCull)));
  for (int i = threadIdx.x; i < G; i += blockDim.x) {
    const float* f = field + 8 * i;
    const float s = f[3];
    tab[i].pos = make_float4(-f[0], -f[1], -f[2], -1.4426950408889634f / (2.f * s * s));
    tab[i].col = make_float4(log2f(f[4]), f[5], f[6], f[7]);
    const float mu_max = fmaxf(fabsf(f[0]), fmaxf(fabsf(f[1]), fabsf(f[2])));
    cull[i].v = make_float4(-f[0], -f[1], -f[2], kCullSigmas * s + 1e-5f * mu_max);
  }
  return FieldSmem{tab, cull, kept + (threadIdx.x >> 5) * G};
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Warp-wide minimum / maximum of binary32 values, one instruction each
// (sm_100 and later).  NaN inputs are ignored.
__device__ __forceinline__ float warp_min(float v) {
  float r;
  asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ float warp_max(float v) {
  float r;
  asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
  return r;
}

__device__ __forceinline__ float2 splat(float v) { return make_float2(v, v); }

// Opacity 1 - exp(-tau) of two intervals at once.  For |tau| < 1/2 it is the
// Taylor series of -expm1(-tau) = tau * sum_k (-tau)^k / (k+1)!, k = 0..7,
// in Horner form (the first term left out, (tau/2)^8 / 9! < 1.1e-8, is far
// below binary32 rounding), which keeps small opacities accurate to a few
// ulp; beyond, 1 - exp2(-tau log2 e), whose absolute error of a few 1e-8 is
// small against an opacity of at least 0.39.
__device__ __forceinline__ float2 opacity2(float2 tau) {
  const float2 x = make_float2(-tau.x, -tau.y);
  float2 p = splat(1.f / 40320.f);  // 1/8!
  p = __ffma2_rn(p, x, splat(1.f / 5040.f));
  p = __ffma2_rn(p, x, splat(1.f / 720.f));
  p = __ffma2_rn(p, x, splat(1.f / 120.f));
  p = __ffma2_rn(p, x, splat(1.f / 24.f));
  p = __ffma2_rn(p, x, splat(1.f / 6.f));
  p = __ffma2_rn(p, x, splat(0.5f));
  p = __ffma2_rn(p, x, splat(1.f));
  const float2 series = __fmul2_rn(tau, p);
  const float2 big = make_float2(1.f - ex2_approx(-1.4426950408889634f * tau.x),
                                 1.f - ex2_approx(-1.4426950408889634f * tau.y));
  return make_float2(fabsf(tau.x) < 0.5f ? series.x : big.x,
                     fabsf(tau.y) < 0.5f ? series.y : big.y);
}

// The part of one ray that a chunk's samples of it lie on: centre point c,
// half-length hh in the ray's parameter, direction d and 1 / |d|^2.
struct Segment {
  float cx, cy, cz, hh, dx, dy, dz, idd;
};

// Squared distance from the blob centre (given negated) to the segment.
__device__ __forceinline__ float seg_dist2(const Segment& S, const float4& nmu) {
  const float wx = S.cx + nmu.x, wy = S.cy + nmu.y, wz = S.cz + nmu.z;  // c - mu
  const float u = -fmaf(wx, S.dx, fmaf(wy, S.dy, wz * S.dz)) * S.idd;
  const float t = fminf(fmaxf(u, -S.hh), S.hh);
  const float qx = fmaf(t, S.dx, wx), qy = fmaf(t, S.dy, wy), qz = fmaf(t, S.dz, wz);
  return fmaf(qx, qx, fmaf(qy, qy, qz * qz));
}

// Segment of ray slot `slot` over the parameter range [tmin, tmax] (midpoint
// parameters of its samples in the chunk); rs[slot] = {o, d.x}, {d.y, d.z,
// 1/|d|^2, -}.  Also returns the rounding margin for distances to it.
__device__ __forceinline__ Segment make_segment(const float4 (*rs)[2], int slot, float tmin,
                                                float tmax, float& eps) {
  const float4 A = rs[slot][0], B = rs[slot][1];
  const float tmid = 0.5f * (tmin + tmax);
  Segment S;
  S.hh = 0.5f * (tmax - tmin);
  S.dx = A.w;
  S.dy = B.x;
  S.dz = B.y;
  S.idd = B.z;
  S.cx = fmaf(tmid, S.dx, A.x);
  S.cy = fmaf(tmid, S.dy, A.y);
  S.cz = fmaf(tmid, S.dz, A.z);
  const float cm = fmaxf(fabsf(S.cx), fmaxf(fabsf(S.cy), fabsf(S.cz)));
  const float dm = fmaxf(fabsf(S.dx), fmaxf(fabsf(S.dy), fabsf(S.dz)));
  eps = 1e-5f * (1.f + cm + S.hh * dm);
  return S;
}

// One sample of a chunk: the interval [a0, a1) of the ray in slot `own`,
// evaluated at point (px, py, pz).
struct Elem {
  float px, py, pz, a0, a1;
  int own;
};

// The blobs within reach of the lines of a warp task's rays, as a list of
// blob indices in `cand` (in blob order); returns their number.  Every
// sample of a ray lies on its line (up to binary32 rounding, which the
// margin covers: a sample within reach of a blob is at most reach + |mu|
// from the origin), so a chunk only has to test these candidates.  rs[slot]
// holds {o, d.x}, {d.y, d.z, 1/|d|^2, -} of the task's `nrays` rays.
__device__ __forceinline__ int task_candidates(const FieldSmem& fs, int G,
                                               const float4 (*rs)[2], int nrays,
                                               uint16_t* cand) {
  const int lane = threadIdx.x & 31;
  int n = 0;
  for (int q0 = 0; q0 < G; q0 += 32) {
    const int q = q0 + lane;
    bool near = false;
    if (q < G) {
      const float4 c = fs.cull[q].v;  // -mu, reach
      const float mu_max = fmaxf(fabsf(c.x), fmaxf(fabsf(c.y), fabsf(c.z)));
      for (int r = 0; r < nrays; ++r) {
        const float4 A = rs[r][0], B = rs[r][1];
        const float wx = A.x + c.x, wy = A.y + c.y, wz = A.z + c.z;  // o - mu
        const float u = -fmaf(wx, A.w, fmaf(wy, B.x, wz * B.y)) * B.z;
        const float qx = fmaf(u, A.w, wx), qy = fmaf(u, B.x, wy), qz = fmaf(u, B.y, wz);
        const float o_max = fmaxf(fabsf(A.x), fmaxf(fabsf(A.y), fabsf(A.z)));
        const float reach = c.w + 2e-5f * (1.f + o_max + mu_max + c.w);
        near |= fmaf(qx, qx, fmaf(qy, qy, qz * qz)) <= reach * reach;
      }
    }
    const unsigned ball = __ballot_sync(kFieldFull, near);
    if (near) cand[n + __popc(ball & ((1u << lane) - 1u))] = (uint16_t)q;
    n += __popc(ball);
  }
  __syncwarp();
  return n;
}

// One 64-sample chunk.  Lane l holds the chunk's samples 2l (e0) and
// 2l + 1 (e1); samples below `nlive` are live, the rest padding (live
// samples come first and are in ray order, so a ray's samples are
// consecutive).  Updates T_s[own] and C_s[own] of every ray the chunk
// touches.  `cand` lists the task's candidate blobs (task_candidates).
// Returns the chunk's blob evaluations (live samples x kept blobs), the same
// on every lane.
__device__ __forceinline__ int composite_chunk2(const FieldSmem& fs, const uint16_t* cand,
                                                int ncand, int nlive, const Elem& e0,
                                                const Elem& e1, const float4 (*rs)[2],
                                                float* T_s, float4* C_s) {
  const int lane = threadIdx.x & 31;
  const bool live0 = 2 * lane < nlive, live1 = 2 * lane + 1 < nlive;
  float2 sig = splat(0.f), cr = sig, cg = sig, cb = sig;
  int m = 0;
  {
    // The blobs within reach of the chunk's points.  A chunk holds the
    // samples of one or two rays (its first and last ray slot) in most
    // cases: the points of a ray lie on a segment of it, so a blob is kept
    // when it lies within reach of one of those segments.  With three rays
    // or more, the test is against the points' bounding box.
    const int s_first = __shfl_sync(kFieldFull, e0.own, 0);
    const int s_last =
        (int)__reduce_max_sync(kFieldFull, (unsigned)(live1 ? e1.own : live0 ? e0.own : 0));
    const bool segs = s_last - s_first <= 1, two = s_last != s_first;
    Segment SA, SB;
    float epsA = 0.f, epsB = 0.f;
    float bx0 = 0.f, by0 = 0.f, bz0 = 0.f, bx1 = 0.f, by1 = 0.f, bz1 = 0.f;
    if (segs) {
      const float tm0 = 0.5f * (e0.a0 + e0.a1), tm1 = 0.5f * (e1.a0 + e1.a1);
      const bool a0 = live0 && e0.own == s_first, a1 = live1 && e1.own == s_first;
      const float tA0 = warp_min(fminf(a0 ? tm0 : INFINITY, a1 ? tm1 : INFINITY));
      const float tA1 = warp_max(fmaxf(a0 ? tm0 : -INFINITY, a1 ? tm1 : -INFINITY));
      SA = make_segment(rs, s_first, tA0, tA1, epsA);
      if (two) {
        const bool b0 = live0 && e0.own == s_last, b1 = live1 && e1.own == s_last;
        const float tB0 = warp_min(fminf(b0 ? tm0 : INFINITY, b1 ? tm1 : INFINITY));
        const float tB1 = warp_max(fmaxf(b0 ? tm0 : -INFINITY, b1 ? tm1 : -INFINITY));
        SB = make_segment(rs, s_last, tB0, tB1, epsB);
      }
    } else {
      bx0 = warp_min(fminf(live0 ? e0.px : INFINITY, live1 ? e1.px : INFINITY));
      by0 = warp_min(fminf(live0 ? e0.py : INFINITY, live1 ? e1.py : INFINITY));
      bz0 = warp_min(fminf(live0 ? e0.pz : INFINITY, live1 ? e1.pz : INFINITY));
      bx1 = warp_max(fmaxf(live0 ? e0.px : -INFINITY, live1 ? e1.px : -INFINITY));
      by1 = warp_max(fmaxf(live0 ? e0.py : -INFINITY, live1 ? e1.py : -INFINITY));
      bz1 = warp_max(fmaxf(live0 ? e0.pz : -INFINITY, live1 ? e1.pz : -INFINITY));
    }
    BlobRec* kept = fs.kept;
    for (int i0 = 0; i0 < ncand; i0 += 32) {
      const int i = i0 + lane;
      bool near = false;
      int q = 0;
      if (i < ncand) {
        q = cand[i];
        const float4 c = fs.cull[q].v;  // -mu, reach
        if (segs) {
          const float ra = c.w + epsA;
          near = seg_dist2(SA, c) <= ra * ra;
          if (two) {  // warp-uniform
            const float rb = c.w + epsB;
            near |= seg_dist2(SB, c) <= rb * rb;
          }
        } else {
          const float ex = fmaxf(0.f, fmaxf(bx0 + c.x, -c.x - bx1));
          const float ey = fmaxf(0.f, fmaxf(by0 + c.y, -c.y - by1));
          const float ez = fmaxf(0.f, fmaxf(bz0 + c.z, -c.z - bz1));
          near = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= c.w * c.w;
        }
      }
      const unsigned ball = __ballot_sync(kFieldFull, near);
      if (near) kept[m + __popc(ball & ((1u << lane) - 1u))] = fs.tab[q];
      m += __popc(ball);
    }
    __syncwarp();
    // both points of the lane at once: half x is e0, half y is e1
    const float2 X = make_float2(e0.px, e1.px), Y = make_float2(e0.py, e1.py),
                 Z = make_float2(e0.pz, e1.pz);
#pragma unroll 4
    for (int i = 0; i < m; ++i) {
      const float4 P = kept[i].pos;
      const float4 C = kept[i].col;
      const float2 ex = __fadd2_rn(X, splat(P.x)), ey = __fadd2_rn(Y, splat(P.y)),
                   ez = __fadd2_rn(Z, splat(P.z));
      float2 d2 = __fmul2_rn(ez, ez);
      d2 = __ffma2_rn(ey, ey, d2);
      d2 = __ffma2_rn(ex, ex, d2);
      const float2 a = __ffma2_rn(d2, splat(P.w), splat(C.x));
      const float2 w = make_float2(ex2_approx(a.x), ex2_approx(a.y));
      sig = __fadd2_rn(sig, w);
      cr = __ffma2_rn(w, splat(C.y), cr);
      cg = __ffma2_rn(w, splat(C.z), cg);
      cb = __ffma2_rn(w, splat(C.w), cb);
    }
    __syncwarp();
  }
  // opacity and colour weight of each element
  const float2 al = opacity2(make_float2(sig.x * (e0.a1 - e0.a0), sig.y * (e1.a1 - e1.a0)));
  float alpha0 = 0.f, alpha1 = 0.f;
  float3 w0 = make_float3(0.f, 0.f, 0.f), w1 = w0;
  if (live0) {
    alpha0 = al.x;
    if (sig.x > 0.f) {
      const float inv = __fdividef(alpha0, sig.x);
      w0 = make_float3(cr.x * inv, cg.x * inv, cb.x * inv);
    }
  }
  if (live1) {
    alpha1 = al.y;
    if (sig.y > 0.f) {
      const float inv = __fdividef(alpha1, sig.y);
      w1 = make_float3(cr.y * inv, cg.y * inv, cb.y * inv);
    }
  }
  // Segments = rays.  e0 starts a segment when its ray differs from the
  // previous lane's e1 (or at lane 0), e1 when its ray differs from e0.  The
  // warp scans run over each lane's LAST segment (the one holding e1): its
  // product of (1 - alpha) and its colour sum, restarting at every lane that
  // holds a segment start.
  const int own1_prev = __shfl_up_sync(kFieldFull, e1.own, 1);
  const int own0_next = __shfl_down_sync(kFieldFull, e0.own, 1);
  const bool head0 = lane == 0 || own1_prev != e0.own;
  const bool head1 = e1.own != e0.own;
  const float f0 = 1.f - alpha0, f1 = 1.f - alpha1;
  const unsigned heads = __ballot_sync(kFieldFull, head0 || head1);
  const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
  bool in[5];
#pragma unroll
  for (int b = 0; b < 5; ++b) in[b] = lane - (1 << b) >= start;
  // transmittance: inclusive product through e1 within its segment
  float incl = head1 ? f1 : f0 * f1;
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    const float y = __shfl_up_sync(kFieldFull, incl, 1 << b);
    if (in[b]) incl *= y;
  }
  const float carry = __shfl_up_sync(kFieldFull, incl, 1);  // through the previous lane's e1
  const float x0 = head0 ? 1.f : carry;                      // before e0, within its segment
  const float x1 = head1 ? 1.f : x0 * f0;                    // before e1
  const float T0b = T_s[e1.own];  // the ray's transmittance before this chunk
  const float ta = T_s[e0.own] * x0, tb = T0b * x1;
  const float3 c0 = make_float3(ta * w0.x, ta * w0.y, ta * w0.z);
  const float3 c1 = make_float3(tb * w1.x, tb * w1.y, tb * w1.z);
  float sr = head1 ? c1.x : c0.x + c1.x, sg = head1 ? c1.y : c0.y + c1.y,
        sb = head1 ? c1.z : c0.z + c1.z;
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    const float yr = __shfl_up_sync(kFieldFull, sr, 1 << b);
    const float yg = __shfl_up_sync(kFieldFull, sg, 1 << b);
    const float yb = __shfl_up_sync(kFieldFull, sb, 1 << b);
    if (in[b]) {
      sr += yr;
      sg += yg;
      sb += yb;
    }
  }
  const float pr = __shfl_up_sync(kFieldFull, sr, 1), pg = __shfl_up_sync(kFieldFull, sg, 1),
              pb = __shfl_up_sync(kFieldFull, sb, 1);
  // e0 ends a segment when e1 is padding or starts another ray; e1 ends one
  // at the lane's end when the next element is padding or another ray
  const bool tail0 = live0 && (!live1 || head1);
  const bool tail1 = live1 && (lane == 31 || 2 * lane + 2 >= nlive || own0_next != e1.own);
  __syncwarp();
  if (tail0) {
    T_s[e0.own] = ta * f0;
    float4 acc = C_s[e0.own];
    acc.x += (head0 ? 0.f : pr) + c0.x;
    acc.y += (head0 ? 0.f : pg) + c0.y;
    acc.z += (head0 ? 0.f : pb) + c0.z;
    C_s[e0.own] = acc;
  }
  if (tail1) {
    T_s[e1.own] = T0b * incl;
    float4 acc = C_s[e1.own];
    acc.x += sr;
    acc.y += sg;
    acc.z += sb;
    C_s[e1.own] = acc;
  }
  __syncwarp();
  return m * nlive;
}

}  // namespace
}  // namespace hdda
