// walk.cuh -- the per-ray walk shared by the single-call samplers
// (traverse.cu), the render-only path (render.cu) and the batched sampler
// (batch.cu): the lattice view, its header (closed form and bucket index),
// ray loading, exact point evaluation, region location on a dense or VDB
// grid, the region crossing search, the walk itself (from the start, or
// resumed after its first runs), the warp-cooperative expansion of runs into
// samples (4-byte stores for the one-pass kernel; a per-tile record list and
// 16-byte stores for the emits), the persistent walk kernel with its staged
// tables and its launch, and the scan of per-tile sample counts.  How the walk works
// and why it is exact is explained at the top of traverse.cu.
#pragma once

#include "grid.cuh"

namespace hdda {
namespace {

constexpr int kMaxRuns = 16;    // runs per ray kept between the walk and the emit
constexpr unsigned kFull = 0xffffffffu;

// Loads from a table that lives in shared memory (kSm) or in global memory
// (read-only path).
template <bool kSm, typename T>
__device__ __forceinline__ T ld(const T* p) {
  if constexpr (kSm) return *p;
  else return __ldg(p);
}

// ---------------------------------------------------------------------------
// lattice
// ---------------------------------------------------------------------------

__device__ __forceinline__ float lattice_next(float t, const hdda_params& p) {
  const float dt = fminf(fmaxf(__fmul_rn(t, p.cone_angle), p.step), p.max_step);
  return __fadd_rn(t, dt);
}

LatticeDev lattice_view(char* block, int max_k, int K) {
  float* t = reinterpret_cast<float*>(block);
  float* tm = t + max_k + 1;
  int* kidx = reinterpret_cast<int*>(tm + max_k);
  uint32_t* hdr = reinterpret_cast<uint32_t*>(kidx + kKidxMax + 2);
  return LatticeDev{t, tm, kidx, hdr, K};
}

// The lattice header: the bucket index's {key0, shift, NB} and, when the
// lattice has the closed form (constant spacing up to index ks, geometric
// growth by 1 + cone per index from there), the values that estimate an
// index from it: tm_k = tm0 + k dt for k < ks and tm_k = tm_ks (1 + cone)^(k -
// ks) from ks on, both up to the recurrence's rounding.
struct LatHdr {
  uint32_t key0, shift;
  int NB;
  int lin;        // the closed form: 0 none (buckets), 1 constant spacing, 2 then geometric
  float tm0, inv_dt;
  float tm_s, inv_tm_s, ks, A;  // tm_ks (+inf when ks = K), 1 / tm_ks, ks, 1 / log2(1 + cone)
};

__device__ __forceinline__ LatHdr lat_hdr(const LatticeDev& lat) {
  LatHdr h{__ldg(lat.hdr), __ldg(lat.hdr + 1), (int)__ldg(lat.hdr + 2),
           (int)__ldg(lat.hdr + 3), 0.f, 0.f, INFINITY, 0.f, 0.f, 0.f};
  if (h.lin && lat.K > 0) {
    const int ks = (int)__ldg(lat.hdr + 4);
    h.tm0 = __ldg(lat.tm);
    h.inv_dt = 1.0f / (__ldg(lat.t + 1) - __ldg(lat.t));
    h.ks = (float)ks;
    h.A = __uint_as_float(__ldg(lat.hdr + 5));
    if (h.lin == 2 && ks < lat.K) {
      h.tm_s = __ldg(lat.tm + ks);
      h.inv_tm_s = 1.0f / h.tm_s;
    } else {
      h.lin = 1;
    }
  } else {
    h.lin = 0;
  }
  return h;
}

// First k with tm_k >= te (K if none), through the bucket index.
template <bool kSm>
__device__ __forceinline__ int first_k_at(const LatticeDev& lat, const LatHdr& h, float te) {
  const uint32_t key = float_key(te);
  const int b = key < h.key0 ? 0 : (int)min((key - h.key0) >> h.shift, (uint32_t)h.NB);
  int lo = ld<kSm>(lat.kidx + b);
  const int hi = ld<kSm>(lat.kidx + b + 1);
  while (lo < hi && ld<kSm>(lat.tm + lo) < te) ++lo;
  return lo;
}

// ---------------------------------------------------------------------------
// the walk
// ---------------------------------------------------------------------------

struct Ray {
  float o[3], d[3], inv[3];
  bool neg[3];  // direction component < 0 (a zero component counts as positive)
};

__device__ __forceinline__ bool load_ray(const float* __restrict__ ro,
                                         const float* __restrict__ rd, int64_t r, Ray& ray) {
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    ray.o[c] = __ldg(ro + 3 * r + c);
    ray.d[c] = __ldg(rd + 3 * r + c);
    ok &= isfinite(ray.o[c]) && isfinite(ray.d[c]);
    ray.neg[c] = ray.d[c] < 0.f;
    // estimates only; +inf for a zero component (either sign), so that the
    // crossing estimate needs no test for it (see cross)
    ray.inv[c] = ray.d[c] != 0.f ? 1.0f / ray.d[c] : INFINITY;
  }
  return ok;
}

// The grid tables the walk reads per region, in shared memory (staged) or
// global memory; the rest of the grid stays in the GridDev kernel parameter.
struct Tabs {
  const float* thr;
  const uint32_t* child;
  const uint32_t* tile;
  const uint32_t* prefix;
  const uint32_t* nstate;
};

__device__ __forceinline__ Tabs global_tabs(const GridDev& g) {
  return Tabs{g.thr, g.child, g.tile, g.prefix, g.nstate};
}

// x = o + tm * d per axis, one rounding per operation.
__device__ __forceinline__ void point_at(const Ray& r, float tm, float x[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) x[c] = __fadd_rn(r.o[c], __fmul_rn(tm, r.d[c]));
}

// A region is kept as one exit plane per axis: e[c] bounds the region on the
// side the ray moves towards (upper bound, exclusive, for d >= 0; lower
// bound, inclusive, for d < 0).
__device__ __forceinline__ bool outside(const float x[3], const float e[3], const Ray& r) {
  return ((x[0] >= e[0]) != r.neg[0]) | ((x[1] >= e[1]) != r.neg[1]) |
         ((x[2] >= e[2]) != r.neg[2]);
}

// Intersects the region with [lo, hi) along axis c.
__device__ __forceinline__ void clip(float e[3], const Ray& r, int c, float lo, float hi) {
  e[c] = r.neg[c] ? fmaxf(e[c], lo) : fminf(e[c], hi);
}

// Intersects the region with voxels [a0, a1) of axis c of one level, using
// the exact thresholds X[a] (only the bound on the exit side is loaded).
template <bool kSm>
__device__ __forceinline__ void clip_cells(float e[3], const Ray& r, const float* thr, int R1,
                                           int c, int a0, int a1) {
  if (r.neg[c]) e[c] = fmaxf(e[c], ld<kSm>(thr + c * R1 + a0));
  else e[c] = fminf(e[c], ld<kSm>(thr + c * R1 + a1));
}

// Classifies x and sets e to the region holding it.  Returns its occupancy.
// kSm: the tables in tb point into shared memory.  `gone` carries, from one
// call to the next along a ray, the levels whose box the ray has left for
// good: a point outside a box on an axis whose coordinate does not move
// back towards it stays outside (each coordinate is monotone in k), so
// those levels need no test, and no half-space, again.  Only finer levels
// are recorded (the coarsest is tested once per call anyway; measured
// faster for single-level grids).
// kOne: the grid has one level, so the level index is the constant 0 and
// the level's box, scale and tables are addressed without it.
template <int kMode, bool kSm, bool kOne>
__device__ __forceinline__ bool locate_impl(const GridDev& g, const Tabs& tb, const Ray& r,
                                            const float x[3], float e[3], unsigned& gone) {
  const int L = kOne ? 1 : g.L;
#pragma unroll
  for (int c = 0; c < 3; ++c) e[c] = r.neg[c] ? -INFINITY : INFINITY;
  int l = -1;
  for (int lv = 0; lv < L; ++lv) {
    if (lv + 1 < L && ((gone >> lv) & 1u)) continue;
    const LevelDev& B = g.lv[lv];
    bool inside = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) inside &= (x[c] >= B.lo[c]) & (x[c] < B.hi[c]);
    if (inside) { l = lv; break; }
    // x lies outside this (finer) box: keep a half-space that separates the
    // ray's later points from it, preferring the one it leaves last.
    int best = -1;
    float best_t = -1.f;
    bool never = false;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (x[c] < B.lo[c]) {
        if (!(r.d[c] > 0.f)) never = true;  // coordinate never grows: never enters
        else {
          const float t = (B.lo[c] - x[c]) * r.inv[c];
          if (t > best_t) { best_t = t; best = c; }
        }
      } else if (x[c] >= B.hi[c]) {
        if (!(r.d[c] < 0.f)) never = true;
        else {
          const float t = (B.hi[c] - x[c]) * r.inv[c];
          if (t > best_t) { best_t = t; best = c; }
        }
      }
    }
    if (never) {
      if (lv + 1 < L) gone |= 1u << lv;
      continue;
    }
    if (best < 0) continue;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (c != best) continue;
      if (r.neg[c]) e[c] = fmaxf(e[c], B.hi[c]);  // region x >= hi
      else e[c] = fminf(e[c], B.lo[c]);           // region x < lo
    }
  }
  if (l < 0) return false;
  if constexpr (kOne) l = 0;

  const LevelDev& V = g.lv[kOne ? 0 : l];
  int i[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    clip(e, r, c, V.lo[c], V.hi[c]);
    i[c] = voxel_index(x[c], V.lo[c], V.s[c], g.R);
  }
  // Descend to the coarsest uniform region holding x: an aligned cube of
  // `sz` voxels (cut off at the grid edge).  Every kind ends in the one clip
  // below, so lanes that stop at different depths share it.
  int sz = 1;
  bool occ;
  do {
    if constexpr (kMode == kModeDense) {
      // R^3 <= 2^30 and L * W <= 2^28: 32-bit offsets (5 % faster than 64-bit)
      const int lin = (i[0] * g.R + i[1]) * g.R + i[2];
      const uint32_t w = __ldg(g.bits + (l * g.W + (lin >> 5)));
      occ = (w >> (lin & 31)) & 1u;
      break;
    }
    if constexpr (kMode == kModeVdbMap) {
      // the refined tree's region, flattened: one 2-byte load.  C^3 * L <= 2^27 * 8
      // entries, so the offset fits 32 bits
      const int C = (g.R + 1) >> 1;
      const int cell = ((l * C + (i[0] >> 1)) * C + (i[1] >> 1)) * C + (i[2] >> 1);
      const uint32_t m = __ldg(g.rmap + cell);
      occ = (m >> (((i[0] & 1) << 2) | ((i[1] & 1) << 1) | (i[2] & 1))) & 1u;
      sz = 1 << (m >> 8);
      break;
    }
    // plain tree.  Node level: L * N^3 <= 8 * 8^3 nodes and L * B^3 * 16 <= 2^28 leaf
    // words, so every offset below fits 32 bits (cheaper address arithmetic than 64-bit)
    const int N = g.N;
    const int ng = l * N * N * N + ((i[0] >> 7) * N + (i[1] >> 7)) * N + (i[2] >> 7);
    const uint32_t st = ld<kSm>(tb.nstate + ng);
    if (st != kNodeMixed) {
      sz = kNodeVox;
      occ = st == kNodeFull;
      break;
    }
    // block level: empty or tile
    const int cell = (((i[0] >> 3) & 15) * 16 + ((i[1] >> 3) & 15)) * 16 + ((i[2] >> 3) & 15);
    const int w = cell >> 5;
    const uint32_t bit = 1u << (cell & 31);
    const uint32_t cw = ld<kSm>(tb.child + ng * kNodeWords + w);
    if (!(cw & bit)) {
      sz = kBlockDim;
      occ = (ld<kSm>(tb.tile + ng * kNodeWords + w) & bit) != 0u;
      break;
    }
    // voxel of a leaf
    const uint32_t leaf = ld<kSm>(tb.prefix + ng * kNodeWords + w) + __popc(cw & (bit - 1u));
    const int v = ((i[0] & 7) * 8 + (i[1] & 7)) * 8 + (i[2] & 7);
    const uint32_t lw = __ldg(g.leaves + (leaf * (uint32_t)kLeafWords + (uint32_t)(v >> 5)));
    occ = (lw >> (v & 31)) & 1u;
  } while (false);
  const int R1 = g.R + 1;
  const float* thr = tb.thr + l * 3 * R1;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int a0 = i[c] & -sz;
    clip_cells<kSm>(e, r, thr, R1, c, a0, min(a0 + sz, g.R));
  }
  return occ;
}

template <int kMode, bool kSm>
__device__ __forceinline__ bool locate(const GridDev& g, const Tabs& tb, const Ray& r,
                                       const float x[3], float e[3], unsigned& gone) {
  if (g.L == 1) return locate_impl<kMode, kSm, true>(g, tb, r, x, e, gone);  // uniform
  return locate_impl<kMode, kSm, false>(g, tb, r, x, e, gone);
}

// First k' in (k, K] whose point is outside the region (K if none).  The
// point of k is inside.  xo receives the point of k' when k' < K.
template <bool kSm>
__device__ __forceinline__ int cross(const Ray& r, const LatticeDev& lat, const LatHdr& h, int k,
                                     const float e[3], float xo[3]) {
  const int K = lat.K;
  // estimate: the ray parameter where it meets the first exit plane.  On an
  // axis the ray does not move along, inv is +inf and the region holds the
  // point, so e - o > 0 there (or e = +inf): the term is +inf (or NaN when
  // e - o = 0, which fminf ignores) and sets no bound.
  float te = INFINITY;
#pragma unroll
  for (int c = 0; c < 3; ++c) te = fminf(te, (e[c] - r.o[c]) * r.inv[c]);
  // The closed form (lat_hdr) lands on the first k with tm_k >= te, or next
  // to it, with fewer instructions than the bucket index.
  int ke;
  if (h.lin == 1) {  // uniform over the launch
    ke = (int)ceilf(fminf(fmaxf((te - h.tm0) * h.inv_dt, 0.f), (float)K));
  } else if (h.lin == 2) {
    const float fc = (te - h.tm0) * h.inv_dt;                  // constant spacing
    const float fg = fmaf(__log2f(te * h.inv_tm_s), h.A, h.ks);  // geometric growth
    ke = (int)ceilf(fminf(fmaxf(te < h.tm_s ? fc : fg, 0.f), (float)K));
  } else {
    ke = first_k_at<kSm>(lat, h, te);
  }
  ke = max(ke, k + 1);
  int lo, hi;  // invariant: point lo inside (lo >= k); point hi outside, or hi == K
  float xp[3];
  if (ke >= K) {
    if (K - 1 == k) return K;
    point_at(r, ld<kSm>(lat.tm + K - 1), xp);
    if (!outside(xp, e, r)) return K;
    lo = k;
    hi = K - 1;
    xo[0] = xp[0]; xo[1] = xp[1]; xo[2] = xp[2];
  } else {
    point_at(r, ld<kSm>(lat.tm + ke), xp);
    if (!outside(xp, e, r)) {
      // estimate too early: gallop forward
      lo = ke;
      int step = 1;
      for (;;) {
        hi = lo + step;
        if (hi >= K) { hi = K; break; }
        point_at(r, ld<kSm>(lat.tm + hi), xp);
        if (outside(xp, e, r)) {
          xo[0] = xp[0]; xo[1] = xp[1]; xo[2] = xp[2];
          break;
        }
        lo = hi;
        step <<= 1;
      }
    } else {
      xo[0] = xp[0]; xo[1] = xp[1]; xo[2] = xp[2];
      if (ke - 1 == k) return ke;
      point_at(r, ld<kSm>(lat.tm + ke - 1), xp);
      if (!outside(xp, e, r)) return ke;  // the usual case: estimate exact
      lo = k;
      hi = ke - 1;
      xo[0] = xp[0]; xo[1] = xp[1]; xo[2] = xp[2];
    }
  }
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    point_at(r, ld<kSm>(lat.tm + mid), xp);
    if (outside(xp, e, r)) {
      hi = mid;
      xo[0] = xp[0]; xo[1] = xp[1]; xo[2] = xp[2];
    } else {
      lo = mid;
    }
  }
  return hi;
}

// Walks one ray.  Counts its samples and merges occupied regions into runs
// [k_begin, k_end): the first kMaxRuns go to runs[j * stride]; nruns counts
// all.  With kEmit it instead writes the samples from `out`, below
// `capacity` (lat.t must then be a global-memory table).
// kSkip selects the control flow of Algorithm 2 ("DDA skip": cross every
// leading empty region in an inner loop, then take the occupied one)
// instead of Algorithm 1 ("DDA branch": one region per iteration, branching
// on its occupancy).  The regions crossed, and so the samples, are the same.
// kCheck tests that every region holds the point it was found from (raising
// kDevInternal otherwise); the invariant the crossing search rests on.
template <int kMode, bool kEmit, bool kSm, bool kSkip = false, bool kCheck = false>
__device__ __forceinline__ int64_t walk(const GridDev& g, const Tabs& tb, const LatticeDev& lat,
                                        const LatHdr& h, const Ray& r, uint2* runs,
                                        int64_t stride, int& nruns, int32_t rid,
                                        int64_t out, int64_t capacity,
                                        int32_t* __restrict__ ray_idx, float* __restrict__ t0,
                                        float* __restrict__ t1, unsigned* __restrict__ status) {
  const int K = lat.K;
  int64_t cnt = 0;
  nruns = 0;
  if (K <= 0) return 0;
  int rb = -1, re = -1;  // open run
  float x[3];
  point_at(r, ld<kSm>(lat.tm), x);
  int k = 0;
  unsigned gone = 0u;  // cascade levels the ray has left for good
  while (k < K) {
    bool occ;
    int kn;
    // One region; in the skip form, every leading empty region first (one
    // copy of locate and cross serves both forms).  cross advances by
    // construction; the skip form still guards its inner loop (no progress:
    // report, end the ray).  With that conditional store in the loop the
    // skip form measured 2.6x faster (object frame) than without it, while
    // the same guard costs the branch form 5 %, so only the skip form has it.
    for (;;) {
      float e[3];
      occ = locate<kMode, kSm>(g, tb, r, x, e, gone);
      if constexpr (kCheck)
        if (outside(x, e, r)) atomicOr(status, kDevInternal);
      kn = cross<kSm>(r, lat, h, k, e, x);
      if constexpr (kSkip)
        if (kn <= k) {
          atomicOr(status, kDevInternal);
          occ = false;
          kn = K;
        }
      if (!kSkip || occ || kn >= K) break;
      k = kn;
    }
    if (occ) {
      if (kEmit) {
        float ta = __ldg(lat.t + k);
        for (int j = k; j < kn; ++j) {
          const float tb = __ldg(lat.t + j + 1);
          const int64_t p = out + cnt;
          if (p < capacity) {
            ray_idx[p] = rid;
            t0[p] = ta;
            t1[p] = tb;
          }
          ta = tb;
          ++cnt;
        }
      } else {
        cnt += kn - k;
        if (k == re) {
          re = kn;  // adjacent occupied region: extend the run
        } else {
          if (rb >= 0) {
            if (nruns < kMaxRuns) runs[nruns * stride] = make_uint2(rb, re);
            ++nruns;
          }
          rb = k;
          re = kn;
        }
      }
    }
    k = kn;
  }
  if (!kEmit && rb >= 0) {
    if (nruns < kMaxRuns) runs[nruns * stride] = make_uint2(rb, re);
    ++nruns;
  }
  return cnt;
}

// Walks one ray from lattice index k0 and stops after kMaxRuns runs: writes
// them to runs[j * stride], sets nruns, and returns the index where the walk
// resumes (the first k of the next run), or K once the ray is done.  Used
// for rays with more runs than the first pass keeps; resuming at any k gives
// the same samples because every point is classified on its own.  It does
// not check its regions: the first pass crossed the same ones.
template <int kMode, bool kSm>
__device__ __forceinline__ int walk_from(const GridDev& g, const Tabs& tb, const LatticeDev& lat,
                                         const LatHdr& h, const Ray& r, int k0, uint2* runs,
                                         int stride, int& nruns) {
  const int K = lat.K;
  nruns = 0;
  if (k0 >= K) return K;
  int rb = -1, re = -1;  // open run
  float x[3];
  point_at(r, ld<kSm>(lat.tm + k0), x);
  int k = k0;
  unsigned gone = 0u;
  while (k < K) {
    float e[3];
    // the general form only: this path is rare, and one copy of the location
    // code keeps its caller's registers free
    const bool occ = locate_impl<kMode, kSm, false>(g, tb, r, x, e, gone);
    const int kn = cross<kSm>(r, lat, h, k, e, x);
    if (occ) {
      if (k == re) {
        re = kn;
      } else {
        if (rb >= 0) {
          runs[nruns * stride] = make_uint2(rb, re);
          if (++nruns == kMaxRuns) return k;
        }
        rb = k;
        re = kn;
      }
    }
    k = kn;
  }
  if (rb >= 0) runs[(nruns++) * stride] = make_uint2(rb, re);
  return K;
}

// ---------------------------------------------------------------------------
// expansion of runs into samples
// ---------------------------------------------------------------------------

// One warp writes the samples of its 32 rays.  Lane i holds ray rid0 + i
// with `c` samples from output position `off` (rays in order, so the
// warp's samples are one contiguous range); its runs are runs0[i + j *
// stride], j < kMaxRuns.  Lane j of each 32-sample chunk finds the ray that
// owns its position (binary search over the lanes' offsets) and the run
// inside it.  Rays with more runs than were kept are skipped here; they
// walk again.  Nothing at or past `capacity` is written.
template <bool kSm>
__device__ __forceinline__ void expand_warp(int64_t off, int64_t c, bool overflow,
                                            const uint2* runs0, int64_t stride, int32_t rid0,
                                            const float* __restrict__ t, int64_t capacity,
                                            int32_t* __restrict__ ray_idx,
                                            float* __restrict__ t0, float* __restrict__ t1) {
  const int lane = threadIdx.x & 31;
  const int64_t wbeg = __shfl_sync(kFull, off, 0);
  const int64_t wend = __shfl_sync(kFull, off + c, 31);
  for (int64_t base = wbeg; base < wend; base += 32) {
    const int64_t p = base + lane;
    int own = 0;  // the last lane whose offset is <= p
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      const int64_t v = __shfl_sync(kFull, off, own + s);
      if (v <= p) own += s;
    }
    const int64_t own_off = __shfl_sync(kFull, off, own);
    const int own_ovf = __shfl_sync(kFull, (int)overflow, own);
    if (p < wend && !own_ovf && p < capacity) {
      const uint2* rr = runs0 + own;
      int64_t loc = p - own_off;
      uint2 run = ld<kSm>(rr);
      int j = 0;
      while (loc >= (int64_t)(run.y - run.x)) {
        loc -= run.y - run.x;
        run = ld<kSm>(rr + (++j) * stride);
      }
      const int k = (int)run.x + (int)loc;
      ray_idx[p] = rid0 + own;
      t0[p] = __ldg(t + k);
      t1[p] = __ldg(t + k + 1);
    }
  }
}

// The expansion of the two-pass samplers' emit (separate, fused with the
// walk, or batched), with 16-byte stores.  A warp first lists its tile's
// runs, rays in order and each ray's runs in order, as records {first output
// position relative to the tile's first sample, (first k << 5) | lane}: one
// per run, or, for a ray with more runs than were kept, one record with
// kRecSkip set that covers all of that ray's samples (the ray walks again and
// writes them itself).  A sentinel record with position kRecEnd follows the
// last.  Positions are then expanded four per lane per 128-position block
// (expand_records): a lane finds the record holding its first position, and
// a record covers at least one position, so its four positions lie in at most
// four consecutive records.  A sample's k is its record's first k plus its
// distance from the record's first position.  Positions at or past `lim` (the
// tile's samples, cut off at the buffer's capacity) are not written.
constexpr int kRecMax = 32 * kMaxRuns;   // records of one 32-ray tile
constexpr uint32_t kRecSkip = 1u << 31;
constexpr uint32_t kRecEnd = 0xffffffffu;

// Lane-local part of the listing: writes this lane's records from index
// `first` (the lanes' exclusive scan of their record counts).  `c` is the
// lane's sample count and `q` its first position relative to the tile; run j
// of the lane's ray is runs_r[j * stride].  The runs are read through L2
// (ld.global.cg), not the read-only path, because the fused sampler form
// reads them in the kernel that wrote them.
__device__ __forceinline__ void list_runs(uint2* rec, int first, int lane, int nr, int64_t c,
                                          uint32_t q, const uint2* __restrict__ runs_r,
                                          int64_t stride) {
  if (c <= 0) return;
  if (nr > kMaxRuns) {
    rec[first] = make_uint2(q, kRecSkip | (uint32_t)lane);
    return;
  }
  for (int j0 = 0; j0 < nr; j0 += 4) {
    uint2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (j0 + u < nr) v[u] = __ldcg(runs_r + (int64_t)(j0 + u) * stride);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (j0 + u < nr) {
        rec[first + j0 + u] = make_uint2(q, (v[u].x << 5) | (uint32_t)lane);
        q += v[u].y - v[u].x;
      }
    }
  }
}

// One record as the expansion uses it: its sample positions q map to
// lattice index kq + q (kq = first k - first position) and to ray rid0 +
// lane; `skip` marks a ray that writes its own samples; `nxt` is the next
// record's first position.
struct RecView {
  int kq;
  int32_t rid;
  bool skip;
  uint32_t nxt;
};

__device__ __forceinline__ RecView rec_view(const uint2* rec, int u, int32_t rid0) {
  const uint2 r = rec[u];
  RecView v;
  v.kq = (int)((r.y & ~kRecSkip) >> 5) - (int)r.x;
  v.rid = rid0 + (int)(r.y & 31u);
  v.skip = (r.y & kRecSkip) != 0u;
  v.nxt = rec[u + 1].x;
  return v;
}

// The four positions q0 .. q0 + 3 of one lane, from record u on, record by
// record (any number of record changes).  Returns in ok[i] whether position
// q0 + i is written here.
__device__ __forceinline__ void expand_four_any(const uint2* rec, int& u, int q0, int lim,
                                                int32_t rid0, const float* __restrict__ t,
                                                int32_t vr[4], float va[4], float vb[4],
                                                bool ok[4]) {
  RecView v = rec_view(rec, u, rid0);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int q = q0 + i;
    ok[i] = q >= 0 && q < lim;
    vr[i] = 0;
    va[i] = vb[i] = 0.f;
    if (!ok[i]) continue;
    if ((uint32_t)q >= v.nxt) v = rec_view(rec, ++u, rid0);  // a record holds >= 1 position
    ok[i] = !v.skip;
    if (!ok[i]) continue;
    const int k = v.kq + q;
    vr[i] = v.rid;
    va[i] = __ldg(t + k);
    vb[i] = __ldg(t + k + 1);
  }
}

// Expands the records rec[0 .. nrec) (sentinel at rec[nrec]) of one tile
// whose first sample goes to output position wbeg.  vec: ray_idx, t0 and t1
// are 16-byte aligned, so whole 4-position groups take one 16-byte store
// per array.  Each 128-position block starts from `ufirst`, a record at or
// before all of its positions (the record of the previous block's last
// position): lane j reads the first position of record ufirst + j, and a
// five-step shuffle search gives each lane the last of those 32 records
// starting at or before its first position; a lane whose position lies
// beyond them (a block of more than 32 records) binary-searches the rest.
// A lane's four positions then take their lattice index, ray and skip flag
// from that record or the next one by selects; only a lane whose positions
// reach a third record steps through them one by one.
__device__ __forceinline__ void expand_records(const uint2* rec, int nrec, int lim, int64_t wbeg,
                                               int32_t rid0, const float* __restrict__ t,
                                               bool vec, int32_t* __restrict__ ray_idx,
                                               float* __restrict__ t0, float* __restrict__ t1) {
  if (nrec <= 0 || lim <= 0) return;
  const int lane = threadIdx.x & 31;
  int ufirst = 0;  // rec[0] starts at position 0
  for (int base = -(int)(wbeg & 3); base < lim; base += 128) {
    const int q0 = base + 4 * lane;
    const int qs = max(q0, 0);
    const uint32_t pj = rec[min(ufirst + lane, nrec)].x;  // the sentinel past the end
    int j = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      const uint32_t pv = __shfl_sync(kFull, pj, j + s);
      if (pv <= (uint32_t)qs) j += s;
    }
    int u = ufirst + j;
    if (j == 31 && u < nrec) {  // the record may lie further on: binary search
      int hi = nrec;  // rec[u] <= qs < rec[hi] (the sentinel)
      while (hi - u > 1) {
        const int mid = (u + hi) >> 1;
        if (rec[mid].x <= (uint32_t)qs) u = mid;
        else hi = mid;
      }
    }
    int32_t vr[4];
    float va[4], vb[4];
    bool ok[4] = {false, false, false, false};
    if (qs < lim) {
      // The lane's positions lie in record u and, past its end, in record u + 1
      // (without branches), unless they reach a third record (short runs).
      const RecView a = rec_view(rec, u, rid0);
      const RecView b = rec_view(rec, min(u + 1, nrec - 1), rid0);  // used only past a.nxt
      if ((uint32_t)(q0 + 3) >= b.nxt && a.nxt <= (uint32_t)(q0 + 3)) {
        expand_four_any(rec, u, q0, lim, rid0, t, vr, va, vb, ok);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int q = q0 + i;
          const bool in_a = (uint32_t)q < a.nxt;
          const int k = (in_a ? a.kq : b.kq) + q;
          vr[i] = in_a ? a.rid : b.rid;
          ok[i] = q >= 0 && q < lim && !(in_a ? a.skip : b.skip);
          va[i] = ok[i] ? __ldg(t + k) : 0.f;
          vb[i] = ok[i] ? __ldg(t + k + 1) : 0.f;
        }
        if (a.nxt <= (uint32_t)(q0 + 3)) ++u;  // the record of the lane's last position
      }
      const int64_t p0 = wbeg + q0;
      if (vec && (ok[0] & ok[1] & ok[2] & ok[3])) {
        *reinterpret_cast<int4*>(ray_idx + p0) = make_int4(vr[0], vr[1], vr[2], vr[3]);
        *reinterpret_cast<float4*>(t0 + p0) = make_float4(va[0], va[1], va[2], va[3]);
        *reinterpret_cast<float4*>(t1 + p0) = make_float4(vb[0], vb[1], vb[2], vb[3]);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (!ok[i]) continue;
          ray_idx[p0 + i] = vr[i];
          t0[p0 + i] = va[i];
          t1[p0 + i] = vb[i];
        }
      }
    }
    ufirst = __shfl_sync(kFull, u, 31);  // the record of this block's last position
  }
}

// ---------------------------------------------------------------------------
// pass 1 of the two-pass samplers and of the render-only path: the walk
// (persistent warps, staged tables)
// ---------------------------------------------------------------------------

// 32 warps, one CTA per SM: the tables are staged once per SM (3 % faster than
// two CTAs of 512 on the object frame, no register spills)
constexpr int kWalkBS = 1024;

// Shared-memory bytes that stage the walk's tables (0 = they do not fit).
struct StageLayout {
  size_t tm, kidx, thr, child, tile, prefix, nstate, bytes;
};

__host__ __device__ inline StageLayout stage_layout(int K, int L, int R, int64_t nodes, int mode) {
  StageLayout s{};
  size_t o = 0;
  s.tm = o; o += sizeof(float) * (size_t)K;
  s.kidx = o; o += sizeof(int) * (size_t)(kKidxMax + 2);
  s.thr = o; o += sizeof(float) * (size_t)L * 3 * (R + 1);
  s.child = s.tile = s.prefix = s.nstate = o;
  if (mode == kModeVdb) {
    s.child = o; o += 4 * (size_t)nodes * kNodeWords;
    s.tile = o; o += 4 * (size_t)nodes * kNodeWords;
    s.prefix = o; o += 4 * (size_t)nodes * kNodeWords;
    s.nstate = o; o += 4 * (size_t)nodes;
  }
  s.bytes = (o + 15) & ~(size_t)15;
  return s;
}

constexpr size_t kMaxStageBytes = 96 * 1024;

template <typename T>
__device__ __forceinline__ void stage_copy(T* dst, const T* __restrict__ src, int64_t count) {
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) dst[i] = __ldg(src + i);
}

// Copies the walk's tables into shared memory at `smem` (stage_layout) and
// points tb and ls at the copies; the caller synchronises the block before
// the first walk.
template <int kMode>
__device__ __forceinline__ void stage_walk_tables(unsigned char* smem, const GridDev& g,
                                                  const LatticeDev& lat, const LatHdr& h,
                                                  Tabs& tb, LatticeDev& ls) {
  const int64_t nodes = (int64_t)g.L * g.N * g.N * g.N;
  const StageLayout sl = stage_layout(lat.K, g.L, g.R, nodes, kMode);
  float* s_tm = reinterpret_cast<float*>(smem + sl.tm);
  int* s_kidx = reinterpret_cast<int*>(smem + sl.kidx);
  float* s_thr = reinterpret_cast<float*>(smem + sl.thr);
  stage_copy(s_tm, lat.tm, lat.K);
  stage_copy(s_kidx, lat.kidx, (int64_t)h.NB + 2);
  stage_copy(s_thr, g.thr, (int64_t)g.L * 3 * (g.R + 1));
  ls.tm = s_tm;
  ls.kidx = s_kidx;
  tb.thr = s_thr;
  if constexpr (kMode == kModeVdb) {
    uint32_t* s_child = reinterpret_cast<uint32_t*>(smem + sl.child);
    uint32_t* s_tile = reinterpret_cast<uint32_t*>(smem + sl.tile);
    uint32_t* s_prefix = reinterpret_cast<uint32_t*>(smem + sl.prefix);
    uint32_t* s_nstate = reinterpret_cast<uint32_t*>(smem + sl.nstate);
    stage_copy(s_child, g.child, nodes * kNodeWords);
    stage_copy(s_tile, g.tile, nodes * kNodeWords);
    stage_copy(s_prefix, g.prefix, nodes * kNodeWords);
    stage_copy(s_nstate, g.nstate, nodes);
    tb.child = s_child;
    tb.tile = s_tile;
    tb.prefix = s_prefix;
    tb.nstate = s_nstate;
  }
}

// Adds v samples to 32-ray tile t: its sum and, when kept, the sums of its
// groups of 32 and of 1024 tiles (all zeroed by the caller).
__device__ __forceinline__ void add_tile_sum(int64_t t, int64_t v, int64_t* tile_sum,
                                             unsigned long long* sums32,
                                             unsigned long long* sums1024) {
  atomicAdd(reinterpret_cast<unsigned long long*>(tile_sum) + t, (unsigned long long)v);
  if (sums32) {
    atomicAdd(sums32 + (t >> 5), (unsigned long long)v);
    atomicAdd(sums1024 + (t >> 10), (unsigned long long)v);
  }
}

// Pass 1.  Persistent: each warp takes work tiles in order until none is
// left, so a warp never waits for another.  A work tile is 32 consecutive
// rays, or, when the rays are the pixels of a `width`-wide image row by row
// (width > 0), a block of 8 x 4 pixels, whose rays start and end their
// regions at more similar depths.  Writes counts[r], nruns[r] (saturated at
// 255) and the first kMaxRuns runs at runs[r + j * n], and, unless tile_sum
// is null, each 32-ray tile's sample total at tile_sum[r / 32]: stored in
// index order, added atomically in block order (then zeroed by the caller).
template <int kMode, bool kSm, bool kSkip, bool kCheck>
__global__ void __launch_bounds__(kWalkBS) walk_kernel(
    const float* __restrict__ ro, const float* __restrict__ rd, int64_t n, GridDev g,
    LatticeDev lat, int32_t* __restrict__ counts, uint8_t* __restrict__ nruns_out,
    uint2* __restrict__ runs, int64_t* __restrict__ tile_sum, unsigned* __restrict__ tile_counter,
    unsigned* __restrict__ status, unsigned long long* __restrict__ sums32,
    unsigned long long* __restrict__ sums1024, int32_t width) {
  extern __shared__ __align__(16) unsigned char smem[];
  const LatHdr h = lat_hdr(lat);
  Tabs tb = global_tabs(g);
  LatticeDev ls = lat;
  if constexpr (kSm) {
    stage_walk_tables<kMode>(smem, g, lat, h, tb, ls);
    __syncthreads();
  }
  // work tiles, and block columns: 8 x 4 blocks over ceil(n / width) rows.
  // Kept in shared memory, not in registers across the walk.
  __shared__ unsigned s_tiles[2];
  if (threadIdx.x == 0) {
    const unsigned bc = width > 0 ? ((unsigned)width + 7) / 8 : 0;
    s_tiles[0] = width > 0 ? bc * (unsigned)(((n + width - 1) / width + 3) / 4)
                           : (unsigned)((n + 31) / 32);
    s_tiles[1] = bc;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned tile = 0;
    if (lane == 0) tile = atomicAdd(tile_counter, 1u);
    tile = __shfl_sync(kFull, tile, 0);
    if (tile >= s_tiles[0]) break;
    int64_t r;
    bool ok;
    if (width > 0) {
      const unsigned bcols = s_tiles[1];
      const unsigned by = tile / bcols, x = (tile - by * bcols) * 8 + (lane & 7);
      r = (int64_t)(by * 4 + (lane >> 3)) * width + x;
      ok = x < (unsigned)width && r < n;
    } else {
      r = (int64_t)tile * 32 + lane;
      ok = r < n;
    }
    int64_t c = 0;
    if (ok) {
      Ray ray;
      int nr = 0;
      if (load_ray(ro, rd, r, ray))
        c = walk<kMode, false, kSm, kSkip, kCheck>(g, tb, ls, h, ray, runs + r, n, nr, 0, 0, 0,
                                                  nullptr, nullptr, nullptr, status);
      counts[r] = (int32_t)c;
      nruns_out[r] = (uint8_t)min(nr, 255);
    }
    if (!tile_sum) continue;
    if (width > 0) {
      // the 8 lanes of a block row hold consecutive rays, so at most two
      // 32-ray tiles: the row leader's and the next.  A row whose leader is
      // out of range has no ray in range.
      const int64_t t = r >> 5, ta = __shfl_sync(kFull, t, lane & ~7);
      int64_t a = t == ta ? c : 0, b = c - a;
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        a += __shfl_xor_sync(kFull, a, o);
        b += __shfl_xor_sync(kFull, b, o);
      }
      if ((lane & 7) == 0) {
        if (a) add_tile_sum(ta, a, tile_sum, sums32, sums1024);
        if (b) add_tile_sum(ta + 1, b, tile_sum, sums32, sums1024);
      }
      continue;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if (lane == 0) {
      const int64_t t = r >> 5;  // lane 0's ray opens the tile
      tile_sum[t] = c;
      if (sums32) {  // the group sums tile_offset reads (zeroed by the caller)
        atomicAdd(sums32 + (t >> 5), (unsigned long long)c);
        atomicAdd(sums1024 + (t >> 10), (unsigned long long)c);
      }
    }
  }
}

// The first output position of tile t: the sum of every earlier tile's
// samples, from the sums the walk kept per 1024 tiles and per 32 tiles and
// the tile sums themselves (at most 31 + 31 entries of the last two, and
// t / 1024 of the first, read by the warp's lanes at once).  Called by a
// whole warp; every lane returns the offset.
__device__ __forceinline__ int64_t tile_offset(int64_t t, const int64_t* __restrict__ tile_sum,
                                               const unsigned long long* __restrict__ sums32,
                                               const unsigned long long* __restrict__ sums1024) {
  const int lane = threadIdx.x & 31;
  int64_t v = 0;
  const int64_t g2 = t >> 10;  // whole 1024-tile groups before t
  for (int64_t j = lane; j < g2; j += 32) v += (int64_t)__ldg(sums1024 + j);
  const int64_t g1 = (g2 << 5) + lane;  // 32-tile groups of t's 1024-tile group before t's
  if (g1 < (t >> 5)) v += (int64_t)__ldg(sums32 + g1);
  const int64_t j0 = ((t >> 5) << 5) + lane;  // tiles of t's 32-tile group before t
  if (j0 < t) v += __ldg(tile_sum + j0);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// host-side launch of the walk
// ---------------------------------------------------------------------------

// The walk a grid takes: dense DDA, or HDDA with or without refinement.
int walk_mode(const hdda_grid* grid) {
  if (grid->kind == HDDA_GRID_DENSE) return kModeDense;
  return grid->refine ? kModeVdbMap : kModeVdb;
}

struct WalkArgs {
  const float* ro;
  const float* rd;
  int64_t n;
  GridDev g;
  LatticeDev lat;
  int32_t* counts;
  uint8_t* nruns;
  uint2* runs;
  int64_t* tile_sum;
  unsigned* counter;
  unsigned* status;
  unsigned long long* sums32 = nullptr;    // optional group sums for tile_offset
  unsigned long long* sums1024 = nullptr;
  int32_t width = 0;                       // image width: walk in 8 x 4 pixel blocks
};

template <int kMode, bool kSm, bool kSkip>
int launch_walk(const WalkArgs& w, size_t smem, cudaStream_t s) {
  // the checked instantiation only while region checks are on
  auto kern = w.g.check ? walk_kernel<kMode, kSm, kSkip, true> : walk_kernel<kMode, kSm, kSkip, false>;
  if (smem > 48 * 1024)
    HDDA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
  int dev = 0, sms = 0, per_sm = 0;
  HDDA_CUDA_TRY(cudaGetDevice(&dev));
  HDDA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HDDA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWalkBS, smem));
  // one resident wave, but no more CTAs than one per eight 32-ray tiles: a small call
  // is still spread over several SMs (its warps take tiles from the shared counter)
  // without every SM staging the tables for warps that find no tile.  On the 96x96
  // frame (288 tiles) the walk takes 0.0745 ms this way, 0.0792 ms with a CTA per
  // tile and 0.0851 ms with a CTA per 32 tiles.
  const int64_t want = ((w.n + 31) / 32 + 7) / 8;
  const int64_t full = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  const unsigned grid = (unsigned)(want < full ? want : full);
  kern<<<grid, kWalkBS, smem, s>>>(w.ro, w.rd, w.n, w.g, w.lat, w.counts, w.nruns, w.runs,
                                   w.tile_sum, w.counter, w.status, w.sums32, w.sums1024,
                                   w.width);
  HDDA_CUDA_TRY(cudaGetLastError());
  return HDDA_OK;
}

template <int kMode>
int launch_walk_mode(const WalkArgs& w, size_t stage_bytes, bool skip, cudaStream_t s) {
  if (skip)
    return stage_bytes <= kMaxStageBytes ? launch_walk<kMode, true, true>(w, stage_bytes, s)
                                         : launch_walk<kMode, false, true>(w, 0, s);
  return stage_bytes <= kMaxStageBytes ? launch_walk<kMode, true, false>(w, stage_bytes, s)
                                       : launch_walk<kMode, false, false>(w, 0, s);
}

const char* walk_name(int mode) {
  return mode == kModeDense ? "dense_walk" : mode == kModeVdb ? "hdda_walk_plain" : "hdda_walk";
}

// ---------------------------------------------------------------------------
// scan of per-tile sample counts
// ---------------------------------------------------------------------------

// Exclusive scan of the per-tile sums by one CTA of 1024 threads.  The sums
// go through shared memory in chunks of 4096 (coalesced loads and stores);
// each thread scans 4 consecutive entries, a CTA scan joins the threads and
// a carry joins the chunks.  Writes the total and offsets[n] too.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;

__global__ void __launch_bounds__(kScanThreads) tile_scan_kernel(
    const int64_t* __restrict__ tile_sum, int64_t T, int64_t* __restrict__ tile_prefix,
    int64_t* __restrict__ total, int64_t* __restrict__ offsets_end) {
  __shared__ int64_t buf[kScanThreads * kScanPer];
  __shared__ int64_t wt[33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t carry = 0;
  for (int64_t c0 = 0; c0 < T; c0 += kScanThreads * kScanPer) {
    const int64_t m = min((int64_t)kScanThreads * kScanPer, T - c0);
    for (int i = threadIdx.x; i < kScanThreads * kScanPer; i += kScanThreads)
      buf[i] = i < m ? tile_sum[c0 + i] : 0;
    __syncthreads();
    int64_t v[kScanPer];
    int64_t sum = 0;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
      v[j] = buf[threadIdx.x * kScanPer + j];
      sum += v[j];
    }
    int64_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) wt[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      const int64_t t = wt[lane];
      int64_t ti = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, ti, o);
        if (lane >= o) ti += y;
      }
      wt[lane] = ti - t;
      if (lane == 31) wt[32] = ti;
    }
    __syncthreads();
    int64_t run = carry + wt[warp] + inc - sum;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
      buf[threadIdx.x * kScanPer + j] = run;
      run += v[j];
    }
    carry += wt[32];
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += kScanThreads) tile_prefix[c0 + i] = buf[i];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *total = carry;
    *offsets_end = carry;
  }
}


// The same scan in parallel, for at most kMaxSupers * kSuperTiles tiles:
// CTA b adds up every tile sum before its own kSuperTiles tiles (at most
// (kMaxSupers - 1) loads per thread, eight in flight) and scans its own;
// no CTA waits for another.
constexpr int kSuperTiles = 1024;
constexpr int kMaxSupers = 64;

__global__ void __launch_bounds__(kSuperTiles) tile_scan_par_kernel(
    const int64_t* __restrict__ tile_sum, int64_t T, int64_t* __restrict__ tile_prefix,
    int64_t* __restrict__ total, int64_t* __restrict__ offsets_end) {
  __shared__ int64_t wt[33];
  __shared__ int64_t ws[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int b = blockIdx.x;
  int64_t before = 0;
#pragma unroll 8
  for (int j = 0; j < b; ++j) before += tile_sum[(int64_t)j * kSuperTiles + threadIdx.x];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(kFull, before, o);
  if (lane == 0) ws[warp] = before;
  const int64_t i = (int64_t)b * kSuperTiles + threadIdx.x;
  const int64_t x = i < T ? tile_sum[i] : 0;
  int64_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wt[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int64_t t = wt[lane];
    int64_t ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(kFull, ti, o);
      if (lane >= o) ti += y;
    }
    wt[lane] = ti - t;
    if (lane == 31) wt[32] = ti;
  }
  __syncthreads();
  int64_t base = 0;
#pragma unroll 8
  for (int w = 0; w < kSuperTiles / 32; ++w) base += ws[w];
  if (i < T) tile_prefix[i] = base + wt[warp] + inc - x;
  if (b == (int)gridDim.x - 1 && threadIdx.x == 0) {
    *total = base + wt[32];
    *offsets_end = base + wt[32];
  }
}

}  // namespace
}  // namespace hdda
