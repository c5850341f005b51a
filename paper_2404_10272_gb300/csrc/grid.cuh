// grid.cuh -- host-side grid object shared by the builders and samplers.
#pragma once

#include "hdda_internal.cuh"

struct hdda_grid {
  int kind = HDDA_GRID_DENSE;
  int L = 0, R = 0, B = 0, N = 0, W = 0;
  int device = 0;
  hdda_aabb boxes[HDDA_MAX_LEVELS];
  float scale[HDDA_MAX_LEVELS][3];

  // One device allocation holds every array below.
  void* base = nullptr;
  size_t base_bytes = 0;

  float* thr = nullptr;          // [L][3][R+1]
  uint32_t* bits = nullptr;      // dense [L][W]
  uint32_t* child = nullptr;     // vdb [L*N^3][128]
  uint32_t* tile = nullptr;      // vdb [L*N^3][128]
  uint32_t* prefix = nullptr;    // vdb [L*N^3][128]
  uint32_t* nstate = nullptr;    // vdb [L*N^3]
  uint32_t* leaves = nullptr;    // vdb [L*B^3][16] capacity, compact prefix used
  uint32_t* nsuper = nullptr;    // vdb [L*N^3][kSuperWords] refinement masks
  uint32_t* lsub = nullptr;      // vdb [L*B^3][kLeafSubWords] capacity, per leaf
  uint16_t* rmap = nullptr;      // vdb [L][C^3] region map, C = ceil(R / 2)
  int refine = 1;                // HDDA walks the refined tree (through the region map)
  int walk_variant = HDDA_WALK_BRANCH;  // control flow of the two-pass walk
  // build temporaries (kept so that a rebuild allocates nothing)
  uint32_t* blk_masks = nullptr; // [L*B^3][16]
  uint8_t* blk_state = nullptr;  // [L*B^3]
  uint32_t* local_prefix = nullptr;  // [L*N^3][128]
  uint32_t* node_leaves = nullptr;   // [L*N^3]
  uint32_t* node_tiles = nullptr;    // [L*N^3]
  int64_t* totals = nullptr;         // [2]: n_leaves, n_tiles

  cudaEvent_t built = nullptr;   // recorded after the last (re)build

  int64_t nodes_total() const { return (int64_t)L * N * N * N; }
  int64_t blocks_total() const { return (int64_t)L * B * B * B; }
  int64_t thr_count() const { return (int64_t)L * 3 * (R + 1); }
  int64_t map_cells() const {
    const int64_t C = (R + 1) / 2;
    return (int64_t)L * C * C * C;
  }

  hdda::GridDev view() const {
    hdda::GridDev g{};
    g.kind = kind;
    g.L = L; g.R = R; g.B = B; g.N = N; g.W = W;
    for (int l = 0; l < L; ++l) {
      for (int c = 0; c < 3; ++c) {
        g.lv[l].lo[c] = boxes[l].lo[c];
        g.lv[l].hi[c] = boxes[l].hi[c];
        g.lv[l].s[c] = scale[l][c];
      }
    }
    g.thr = thr; g.bits = bits; g.child = child; g.tile = tile;
    g.prefix = prefix; g.nstate = nstate; g.leaves = leaves;
    g.nsuper = nsuper; g.lsub = lsub; g.rmap = rmap;
    g.check = hdda::region_checks_on() ? 1 : 0;
    return g;
  }
};
