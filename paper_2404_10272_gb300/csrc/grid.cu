// grid.cu -- dense bit-array packing (the paper's baseline grid) and the
// GPU builder of the VDB-style sparse grid (Sec. 3: the dense occupancy grid
// becomes a VDB tree whose uniform blocks are pruned into tiles).
//
// Kernels
//   thresholds_kernel   exact per-axis voxel boundaries X[a] (one thread per
//                       boundary, binary search over binary32 keys)
//   pack_dense_kernel   uint8 voxels -> uint32 bit words, one ballot per word
//   vdb_blocks_kernel   one warp per 8^3 block: 16 ballots give the 512-bit
//                       leaf mask and the block's empty/partial/full state
//   vdb_nodes_kernel    one 128-thread CTA per 16^3-block node: ballots over
//                       the block states give the child and tile masks, a
//                       CTA scan gives each mask word's leaf-count prefix
//   vdb_finalize_kernel one CTA: scan of leaf counts over all nodes, global
//                       leaf prefix per mask word, leaf and tile totals
//   vdb_scatter_kernel  16 threads per partial block copy its mask into the
//                       compact leaf pool
//   region_map_kernel   one thread per 2^3-voxel cell: the refined tree's
//                       region holding the cell, flattened into 16 bits (an
//                       update that changes no block's state recomputes only
//                       the changed blocks' cells: region_map_blocks_kernel)
// The node and scatter kernels also write the refinement masks (occupied
// 32^3 and 16^3 groups per node, occupied 4^3 and 2^3 cells per leaf) that
// let hierarchical DDA cross empty space in power-of-two steps below and
// above the 8^3 leaf, in the manner of an octree (Sec. 5 suggests finer
// subdivision).  The region map flattens the refined tree for the walk: a
// ray point's region (its size and occupancy) is one 2-byte load there
// instead of a descent through node, group, block, leaf and cell masks.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "grid.cuh"

namespace hdda {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__global__ void thresholds_kernel(GridDev g, float* __restrict__ thr) {
  const int64_t R1 = g.R + 1;
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)g.L * 3 * R1) return;
  const int a = (int)(idx % R1);
  const int lc = (int)(idx / R1);
  const int c = lc % 3, l = lc / 3;
  const float lo = g.lv[l].lo[c], hi = g.lv[l].hi[c], s = g.lv[l].s[c];
  float X;
  if (a == 0) {
    X = lo;
  } else if (a == g.R) {
    X = hi;
  } else if (voxel_index(hi, lo, s, g.R) < a) {
    X = hi;  // no point of the box reaches index a
  } else {
    // voxel_index is monotone in x, so the set {x : index >= a} is an upper
    // range of binary32 values; find its first element.
    uint32_t kl = float_key(lo);  // index(lo) = 0 < a
    uint32_t kh = float_key(hi);  // index(hi) >= a
    while (kh - kl > 1u) {
      uint32_t km = kl + (kh - kl) / 2u;
      if (voxel_index(key_float(km), lo, s, g.R) >= a) kh = km; else kl = km;
    }
    X = key_float(kh);
  }
  thr[idx] = X;
}

__global__ void pack_dense_kernel(const uint8_t* __restrict__ dense, int L, int R, int W,
                                  uint32_t* __restrict__ bits) {
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t total = (int64_t)L * W;
  const int64_t w0 = warp * 32;
  if (w0 >= total) return;  // uniform per warp
  const int64_t R3 = (int64_t)R * R * R;
  uint32_t mine = 0;
  for (int j = 0; j < 32; ++j) {
    const int64_t gw = w0 + j;
    bool on = false;
    if (gw < total) {
      const int64_t l = gw / W, w = gw % W;
      const int64_t lin = w * 32 + lane;
      if (lin < R3) on = dense[l * R3 + lin] != 0;
    }
    const uint32_t b = __ballot_sync(kFull, on);
    if (lane == j) mine = b;
  }
  if (w0 + lane < total) bits[w0 + lane] = mine;
}

// The 512 occupancy bits of the 8^3 block (bx, by, bz) of one level, voxel
// ((x%8)*8 + y%8)*8 + z%8 at bit v%32 of word v/32: lane w < 16 receives word
// w.  Every lane loads its 16 voxels first, so the loads are in flight
// together, then the warp votes word by word.  Voxels past the grid's edge
// are empty.
__device__ __forceinline__ uint32_t block_words(const uint8_t* __restrict__ lvl, int R, int bx,
                                                int by, int bz, int lane) {
  uint32_t mine = 0;
  // the 16 voxels of each lane first (loads in flight together), then the votes
  uint8_t on[16];
#pragma unroll
  for (int w = 0; w < 16; ++w) {
    const int v = w * 32 + lane;  // local voxel ((x%8)*8 + y%8)*8 + z%8
    const int x = bx * 8 + (v >> 6), y = by * 8 + ((v >> 3) & 7), z = bz * 8 + (v & 7);
    on[w] = 0;
    if (x < R && y < R && z < R) on[w] = __ldg(lvl + ((int64_t)x * R + y) * R + z);
  }
#pragma unroll
  for (int w = 0; w < 16; ++w) {
    const uint32_t bal = __ballot_sync(kFull, on[w] != 0);
    if (lane == w) mine = bal;
  }
  return mine;
}

__global__ void vdb_blocks_kernel(const uint8_t* __restrict__ dense, int L, int R, int B,
                                  uint32_t* __restrict__ blk_masks,
                                  uint8_t* __restrict__ blk_state) {
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t B3 = (int64_t)B * B * B;
  if (warp >= (int64_t)L * B3) return;  // uniform per warp
  const int l = (int)(warp / B3);
  const int64_t b = warp % B3;
  const int bx = (int)(b / ((int64_t)B * B)), by = (int)((b / B) % B), bz = (int)(b % B);
  const uint8_t* lvl = dense + (int64_t)l * R * R * R;
  const uint32_t mine = block_words(lvl, R, bx, by, bz, lane);
  const bool any = __any_sync(kFull, lane < 16 && mine != 0u);
  const bool all = __all_sync(kFull, lane >= 16 || mine == kFull);
  if (lane < 16) blk_masks[warp * 16 + lane] = mine;
  if (lane == 0) blk_state[warp] = all ? kBlockFull : (any ? kBlockPartial : kBlockEmpty);
}

// Exclusive CTA-wide scan of one uint32 per thread (blockDim.x <= 1024, multiple of 32).
__device__ uint32_t cta_exclusive_scan(uint32_t v, uint32_t* warp_tot, uint32_t* total_out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = lane < nw ? warp_tot[lane] : 0u;
    uint32_t ti = t;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(kFull, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < nw) warp_tot[lane] = ti - t;  // exclusive warp offsets
    if (lane == 31) warp_tot[32] = ti;       // CTA total
  }
  __syncthreads();
  uint32_t r = warp_tot[warp] + inc - v;
  if (total_out) *total_out = warp_tot[32];
  __syncthreads();
  return r;
}

// `gate` (null: always) lets an incremental update skip the kernel when no
// block changed between empty, partial and full; the value is the same for
// every thread of the launch.
// A cell of a node beyond the grid's edge (never stored as a block state).
constexpr uint8_t kBlockOutside = 0xff;

__global__ void vdb_nodes_kernel(int L, int B, int N, const uint8_t* __restrict__ blk_state,
                                 uint32_t* __restrict__ child, uint32_t* __restrict__ tile,
                                 uint32_t* __restrict__ local_prefix,
                                 uint32_t* __restrict__ node_leaves,
                                 uint32_t* __restrict__ node_tiles,
                                 uint32_t* __restrict__ nstate,
                                 uint32_t* __restrict__ nsuper, const unsigned* __restrict__ gate) {
  if (gate && *gate == 0u) return;
  __shared__ uint32_t warp_tot[33];
  __shared__ uint32_t s_occ[kNodeWords];  // child | tile
  __shared__ uint32_t s_g16[16];          // occupied 16^3 groups
  const int64_t N3 = (int64_t)N * N * N;
  const int64_t B3 = (int64_t)B * B * B;
  const int64_t ng = blockIdx.x;
  const int l = (int)(ng / N3);
  const int node = (int)(ng % N3);
  const int nx = node / (N * N), ny = (node / N) % N, nz = node % N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t my_child = 0, my_tile = 0, my_in = 0;
  // all 32 block states of this warp's words first (loads in flight together), then the votes
  uint8_t st[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const int cell = (warp * 32 + j) * 32 + lane;
    const int bx = nx * 16 + (cell >> 8), by = ny * 16 + ((cell >> 4) & 15),
              bz = nz * 16 + (cell & 15);
    st[j] = kBlockOutside;
    if (bx < B && by < B && bz < B)
      st[j] = __ldg(blk_state + (int64_t)l * B3 + ((int64_t)bx * B + by) * B + bz);
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const uint32_t c = __ballot_sync(kFull, st[j] == kBlockPartial);
    const uint32_t t = __ballot_sync(kFull, st[j] == kBlockFull);
    const uint32_t i = __ballot_sync(kFull, st[j] != kBlockOutside);
    if (lane == j) { my_child = c; my_tile = t; my_in = i; }
  }
  const int w = threadIdx.x;  // mask word 0..127
  child[ng * kNodeWords + w] = my_child;
  tile[ng * kNodeWords + w] = my_tile;
  uint32_t leaves = 0, tiles = 0, incells = 0;
  local_prefix[ng * kNodeWords + w] = cta_exclusive_scan(__popc(my_child), warp_tot, &leaves);
  cta_exclusive_scan(__popc(my_tile), warp_tot, &tiles);
  cta_exclusive_scan(__popc(my_in), warp_tot, &incells);
  if (threadIdx.x == 0) {
    node_leaves[ng] = leaves;
    node_tiles[ng] = tiles;
    uint32_t st = kNodeMixed;
    if (leaves == 0 && tiles == 0) st = kNodeEmpty;
    else if (leaves == 0 && tiles == incells) st = kNodeFull;
    nstate[ng] = st;
  }
  // refinement: 16^3-voxel groups are 2^3 cells, 32^3-voxel groups 2^3 of those
  s_occ[w] = my_child | my_tile;
  __syncthreads();
  for (int j = 0; j < 4; ++j) {
    const int g2 = j * kNodeWords + threadIdx.x;  // 0..511
    const int gx = g2 >> 6, gy = (g2 >> 3) & 7, gz = g2 & 7;
    bool any = false;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int cell = ((2 * gx + (a >> 2)) * 16 + (2 * gy + ((a >> 1) & 1))) * 16 + 2 * gz + (a & 1);
      any |= (s_occ[cell >> 5] >> (cell & 31)) & 1u;
    }
    const uint32_t bal = __ballot_sync(kFull, any);
    if (lane == 0) s_g16[g2 >> 5] = bal;
  }
  __syncthreads();
  if (threadIdx.x < 64) {
    const int g4 = threadIdx.x;
    const int gx = g4 >> 4, gy = (g4 >> 2) & 3, gz = g4 & 3;
    bool any = false;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int g2 = ((2 * gx + (a >> 2)) * 8 + (2 * gy + ((a >> 1) & 1))) * 8 + 2 * gz + (a & 1);
      any |= (s_g16[g2 >> 5] >> (g2 & 31)) & 1u;
    }
    const uint32_t bal = __ballot_sync(kFull, any);
    if (lane == 0) nsuper[ng * kSuperWords + warp] = bal;
  }
  if (threadIdx.x < 16) nsuper[ng * kSuperWords + 2 + threadIdx.x] = s_g16[threadIdx.x];
}

constexpr int kMaxNodesTotal = HDDA_MAX_LEVELS * (HDDA_MAX_RES / kNodeVox) *
                               (HDDA_MAX_RES / kNodeVox) * (HDDA_MAX_RES / kNodeVox);

__global__ void vdb_finalize_kernel(int64_t nodes, const uint32_t* __restrict__ node_leaves,
                                    const uint32_t* __restrict__ node_tiles,
                                    const uint32_t* __restrict__ local_prefix,
                                    uint32_t* __restrict__ prefix, int64_t* __restrict__ totals,
                                    const unsigned* __restrict__ gate) {
  if (gate && *gate == 0u) return;
  __shared__ uint32_t base[kMaxNodesTotal];
  __shared__ uint32_t warp_tot[33];
  uint32_t carry = 0, tiles = 0;
  for (int64_t c0 = 0; c0 < nodes; c0 += blockDim.x) {
    const int64_t i = c0 + threadIdx.x;
    const uint32_t v = i < nodes ? node_leaves[i] : 0u;
    uint32_t chunk = 0;
    const uint32_t ex = cta_exclusive_scan(v, warp_tot, &chunk);
    if (i < nodes) base[i] = carry + ex;
    carry += chunk;
    uint32_t tchunk = 0;
    cta_exclusive_scan(i < nodes ? node_tiles[i] : 0u, warp_tot, &tchunk);
    tiles += tchunk;
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < nodes * kNodeWords; i += blockDim.x)
    prefix[i] = base[i / kNodeWords] + local_prefix[i];
  if (threadIdx.x == 0) {
    totals[0] = carry;
    totals[1] = tiles;
  }
}

// Copies the mask of partial block `blk` into its slot of the compact leaf
// pool and writes the leaf's refinement masks (occupied 2^3 and 4^3 cells,
// fully occupied 2^3 cells).  Called by the 16 threads of one aligned
// half-warp, `part` = 0..15, all of them together.
__device__ __forceinline__ void scatter_block(int64_t blk, int part, int B, int N,
                                              const uint32_t* __restrict__ blk_masks,
                                              const uint32_t* __restrict__ child,
                                              const uint32_t* __restrict__ prefix,
                                              uint32_t* __restrict__ leaves,
                                              uint32_t* __restrict__ lsub) {
  const int64_t B3 = (int64_t)B * B * B;
  const int l = (int)(blk / B3);
  const int64_t b = blk % B3;
  const int bx = (int)(b / ((int64_t)B * B)), by = (int)((b / B) % B), bz = (int)(b % B);
  const int node = ((bx >> 4) * N + (by >> 4)) * N + (bz >> 4);
  const int64_t ng = (int64_t)l * N * N * N + node;
  const int cell = ((bx & 15) * 16 + (by & 15)) * 16 + (bz & 15);
  const int w = cell >> 5;
  const uint32_t bit = 1u << (cell & 31);
  const uint32_t leaf = prefix[ng * kNodeWords + w] + __popc(child[ng * kNodeWords + w] & (bit - 1u));
  leaves[(int64_t)leaf * kLeafWords + part] = blk_masks[blk * kLeafWords + part];
  // refinement masks: each of the 16 threads classifies 4 of the 64 2^3
  // cells; OR-reductions over the aligned half-warp join them
  const unsigned half = 0xFFFFu << (threadIdx.x & 16);
  const uint32_t* m = blk_masks + blk * kLeafWords;
  uint32_t c2 = 0, f2 = 0, c4 = 0;  // bits of this thread's word (part >> 3) of c2/f2
  for (int q = 0; q < 4; ++q) {
    const int cell = 4 * part + q;  // 2^3 cells, (cx*4 + cy)*4 + cz
    const int cx = cell >> 4, cy = (cell >> 2) & 3, cz = cell & 3;
    bool any = false, all = true;
    for (int a = 0; a < 8; ++a) {
      const int v = ((2 * cx + (a >> 2)) * 8 + (2 * cy + ((a >> 1) & 1))) * 8 + 2 * cz + (a & 1);
      const bool on = (__ldg(m + (v >> 5)) >> (v & 31)) & 1u;
      any |= on;
      all &= on;
    }
    if (any) {
      c2 |= 1u << (cell & 31);
      c4 |= 1u << (((cx >> 1) * 2 + (cy >> 1)) * 2 + (cz >> 1));
    }
    if (all) f2 |= 1u << (cell & 31);
  }
  uint32_t c2w[2] = {part < 8 ? c2 : 0u, part < 8 ? 0u : c2};
  uint32_t f2w[2] = {part < 8 ? f2 : 0u, part < 8 ? 0u : f2};
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    c2w[0] |= __shfl_xor_sync(half, c2w[0], o);
    c2w[1] |= __shfl_xor_sync(half, c2w[1], o);
    f2w[0] |= __shfl_xor_sync(half, f2w[0], o);
    f2w[1] |= __shfl_xor_sync(half, f2w[1], o);
    c4 |= __shfl_xor_sync(half, c4, o);
  }
  if (part == 0) {
    uint32_t* out = lsub + (int64_t)leaf * kLeafSubWords;
    out[0] = c2w[0];
    out[1] = c2w[1];
    out[2] = c4;
    out[3] = f2w[0];
    out[4] = f2w[1];
  }
}

__global__ void vdb_scatter_kernel(int L, int B, int N, const uint8_t* __restrict__ blk_state,
                                   const uint32_t* __restrict__ blk_masks,
                                   const uint32_t* __restrict__ child,
                                   const uint32_t* __restrict__ prefix,
                                   uint32_t* __restrict__ leaves, uint32_t* __restrict__ lsub,
                                   const unsigned* __restrict__ gate) {
  if (gate && *gate == 0u) return;
  // grid-stride, so that an update can launch a small grid that exits at once when
  // gated off; the stride is a multiple of 16, so a half-warp stays on one block
  const int64_t total = (int64_t)L * B * B * B * 16;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blk = t >> 4;
    if (blk_state[blk] != kBlockPartial) continue;
    scatter_block(blk, (int)(t & 15), B, N, blk_masks, child, prefix, leaves, lsub);
  }
}

// Incremental update, step 1: one warp per listed block (every block when
// `list` is null).  The block's mask and state are recomputed from the dense
// bytes; a mask that differs is stored and changed[i] set, and flags[0] is
// set when the block's state (empty, partial, full) changes, since the node
// masks and the leaf compaction then change too.  An index outside the grid
// is skipped and raises kDevBadIndex.
__global__ void vdb_update_blocks_kernel(const uint8_t* __restrict__ dense, int L, int R, int B,
                                         const int64_t* __restrict__ list, int64_t count,
                                         uint32_t* __restrict__ blk_masks,
                                         uint8_t* __restrict__ blk_state,
                                         uint8_t* __restrict__ changed, unsigned* __restrict__ flags,
                                         unsigned* __restrict__ status) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= count) return;  // uniform per warp
  const int64_t B3 = (int64_t)B * B * B;
  const int64_t blk = list ? list[i] : i;
  if (blk < 0 || blk >= (int64_t)L * B3) {
    if (lane == 0) {
      changed[i] = 0;
      atomicOr(status, kDevBadIndex);
    }
    return;
  }
  const int l = (int)(blk / B3);
  const int64_t b = blk % B3;
  const int bx = (int)(b / ((int64_t)B * B)), by = (int)((b / B) % B), bz = (int)(b % B);
  const uint8_t* lvl = dense + (int64_t)l * R * R * R;
  const uint32_t mine = block_words(lvl, R, bx, by, bz, lane);
  const uint32_t old = lane < 16 ? blk_masks[blk * kLeafWords + lane] : 0u;
  const bool diff = __any_sync(kFull, lane < 16 && mine != old);
  const bool any = __any_sync(kFull, lane < 16 && mine != 0u);
  const bool all = __all_sync(kFull, lane >= 16 || mine == kFull);
  const uint8_t st = all ? kBlockFull : (any ? kBlockPartial : kBlockEmpty);
  if (diff && lane < 16) blk_masks[blk * kLeafWords + lane] = mine;
  if (lane == 0) {
    changed[i] = diff ? 1 : 0;
    if (st != blk_state[blk]) {
      blk_state[blk] = st;
      flags[0] = 1u;
    }
  }
}

// Incremental update, last step when no block changed state: the changed
// partial blocks' leaves are rewritten in place (16 threads per listed
// block); the tree's structure and every other leaf stay as they are.
__global__ void vdb_rewrite_leaves_kernel(int B, int N, const int64_t* __restrict__ list,
                                          int64_t count, const uint8_t* __restrict__ changed,
                                          const unsigned* __restrict__ flags,
                                          const uint8_t* __restrict__ blk_state,
                                          const uint32_t* __restrict__ blk_masks,
                                          const uint32_t* __restrict__ child,
                                          const uint32_t* __restrict__ prefix,
                                          uint32_t* __restrict__ leaves,
                                          uint32_t* __restrict__ lsub) {
  if (*flags != 0u) return;  // the structure changed: the full scatter ran instead
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t i = t >> 4;
  if (i >= count || !changed[i]) return;
  const int64_t blk = list ? list[i] : i;
  if (blk_state[blk] != kBlockPartial) return;
  scatter_block(blk, (int)(t & 15), B, N, blk_masks, child, prefix, leaves, lsub);
}

// ---------------------------------------------------------------------------
// host side
// The region map (layout in hdda_internal.cuh), written after the tree and
// its refinement masks.  Each thread descends the refined tree from the
// cell's first voxel, exactly as a walk over the tree would: node state,
// empty 32^3 and 16^3 groups, empty or tiled 8^3 block, empty or full 4^3
// cell (full: its eight 2^3 cells are), empty or full 2^3 cell; a cell that
// is none of these keeps its 8 voxel bits.  Voxels past the grid edge (odd R) are empty in the leaves.
__device__ __forceinline__ uint16_t region_map_cell(const GridDev& g, int64_t idx) {
  const int C = (g.R + 1) >> 1;
  int64_t q = idx;
  const int a2 = (int)(q % C);
  q /= C;
  const int a1 = (int)(q % C);
  q /= C;
  const int a0 = (int)(q % C);
  const int l = (int)(q / C);
  const int i[3] = {2 * a0, 2 * a1, 2 * a2};
  const int N = g.N;
  const int ng = l * N * N * N + ((i[0] >> 7) * N + (i[1] >> 7)) * N + (i[2] >> 7);
  uint32_t lg = 0, mask = 0;
  do {
    const uint32_t st = g.nstate[ng];
    if (st != kNodeMixed) {
      lg = kMapNodeLog2;
      mask = st == kNodeFull ? 0xffu : 0u;
      break;
    }
    const uint32_t* ns = g.nsuper + ng * kSuperWords;
    const int g4 = (((i[0] >> 5) & 3) * 4 + ((i[1] >> 5) & 3)) * 4 + ((i[2] >> 5) & 3);
    if (!((ns[g4 >> 5] >> (g4 & 31)) & 1u)) { lg = 5; break; }
    const int g2 = (((i[0] >> 4) & 7) * 8 + ((i[1] >> 4) & 7)) * 8 + ((i[2] >> 4) & 7);
    if (!((ns[2 + (g2 >> 5)] >> (g2 & 31)) & 1u)) { lg = 4; break; }
    const int cell = (((i[0] >> 3) & 15) * 16 + ((i[1] >> 3) & 15)) * 16 + ((i[2] >> 3) & 15);
    const int w = cell >> 5;
    const uint32_t bit = 1u << (cell & 31);
    const uint32_t cw = g.child[ng * kNodeWords + w];
    if (!(cw & bit)) {
      lg = 3;
      mask = (g.tile[ng * kNodeWords + w] & bit) ? 0xffu : 0u;
      break;
    }
    const uint32_t leaf = g.prefix[ng * kNodeWords + w] + __popc(cw & (bit - 1u));
    const uint32_t* ls = g.lsub + leaf * (uint32_t)kLeafSubWords;
    const int c4 = (((i[0] >> 2) & 1) * 2 + ((i[1] >> 2) & 1)) * 2 + ((i[2] >> 2) & 1);
    if (!((ls[2] >> c4) & 1u)) { lg = 2; break; }
    // a 4^3 cell is full when its eight 2^3 cells are: bits base + {0, 1, 4, 5, 16, 17,
    // 20, 21} of the leaf's 64-bit full-cell mask
    const uint64_t full2 = (uint64_t)ls[3] | ((uint64_t)ls[4] << 32);
    const int base4 = 32 * ((i[0] >> 2) & 1) + 8 * ((i[1] >> 2) & 1) + 2 * ((i[2] >> 2) & 1);
    if (((full2 >> base4) & 0x330033ull) == 0x330033ull) { lg = 2; mask = 0xffu; break; }
    const int c2 = (((i[0] >> 1) & 3) * 4 + ((i[1] >> 1) & 3)) * 4 + ((i[2] >> 1) & 3);
    lg = 1;
    if (!((ls[c2 >> 5] >> (c2 & 31)) & 1u)) break;          // empty 2^3 cell
    if ((ls[3 + (c2 >> 5)] >> (c2 & 31)) & 1u) { mask = 0xffu; break; }  // full 2^3 cell
    lg = 0;
    const uint32_t* lw = g.leaves + leaf * (uint32_t)kLeafWords;
    for (int u = 0; u < 8; ++u) {
      const int x = (i[0] & 7) + (u >> 2), y = (i[1] & 7) + ((u >> 1) & 1), z = (i[2] & 7) + (u & 1);
      const int v = (x * 8 + y) * 8 + z;
      mask |= ((lw[v >> 5] >> (v & 31)) & 1u) << u;
    }
  } while (false);
  return (uint16_t)((lg << 8) | mask);
}

// The whole map, one thread per cell.  With `flags` (an update), only when
// the update changed the tree's structure.
__global__ void region_map_kernel(GridDev g, uint16_t* __restrict__ rmap,
                                  const unsigned* __restrict__ flags) {
  if (flags && *flags == 0u) return;
  const int C = (g.R + 1) >> 1;
  const int64_t cells = (int64_t)g.L * C * C * C;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < cells;
       idx += (int64_t)gridDim.x * blockDim.x)  // grid-stride, as vdb_scatter_kernel
    rmap[idx] = region_map_cell(g, idx);
}

// An update that left every block's state as it was (so every node, group
// and block region stays the same) changes the map only inside the blocks
// whose voxels changed: their 4^3 cells are recomputed, 64 threads per block.
__global__ void region_map_blocks_kernel(GridDev g, uint16_t* __restrict__ rmap,
                                         const int64_t* __restrict__ list, int64_t count,
                                         const uint8_t* __restrict__ changed,
                                         const unsigned* __restrict__ flags) {
  if (*flags != 0u) return;  // the structure changed: the whole map is recomputed
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t i = t >> 6;
  if (i >= count || !changed[i]) return;
  const int64_t blk = list ? list[i] : i;
  const int B = g.B, C = (g.R + 1) >> 1;
  const int64_t B3 = (int64_t)B * B * B;
  const int l = (int)(blk / B3);
  const int64_t b = blk % B3;
  const int bx = (int)(b / ((int64_t)B * B)), by = (int)((b / B) % B), bz = (int)(b % B);
  const int c = (int)(t & 63);
  const int cx = 4 * bx + (c >> 4), cy = 4 * by + ((c >> 2) & 3), cz = 4 * bz + (c & 3);
  if (cx >= C || cy >= C || cz >= C) return;  // past the grid edge (R not a multiple of 8)
  const int64_t idx = (((int64_t)l * C + cx) * C + cy) * C + cz;
  rmap[idx] = region_map_cell(g, idx);
}

// ---------------------------------------------------------------------------

int validate(const uint8_t* dense, int levels, int res, const hdda_aabb* aabbs) {
  if (!dense) return set_error(HDDA_ERR_INVALID_ARG, "dense is NULL");
  if (!aabbs) return set_error(HDDA_ERR_INVALID_ARG, "aabbs is NULL");
  if (levels < 1 || levels > HDDA_MAX_LEVELS)
    return set_error(HDDA_ERR_INVALID_ARG, "levels=%d outside 1..%d", levels, HDDA_MAX_LEVELS);
  if (res < 1 || res > HDDA_MAX_RES)
    return set_error(HDDA_ERR_INVALID_ARG, "res=%d outside 1..%d", res, HDDA_MAX_RES);
  for (int l = 0; l < levels; ++l) {
    for (int c = 0; c < 3; ++c) {
      const float lo = aabbs[l].lo[c], hi = aabbs[l].hi[c];
      if (!std::isfinite(lo) || !std::isfinite(hi) || !(lo < hi))
        return set_error(HDDA_ERR_INVALID_ARG, "level %d axis %d: box [%g, %g) invalid", l, c,
                         (double)lo, (double)hi);
      const float s = (float)res / (hi - lo);
      if (!std::isfinite(s))
        return set_error(HDDA_ERR_INVALID_ARG, "level %d axis %d: scale not finite", l, c);
    }
  }
  return HDDA_OK;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename T>
void carve(char* base, size_t& off, T*& ptr, int64_t count, bool take) {
  if (take) {
    ptr = reinterpret_cast<T*>(base ? base + off : nullptr);
    off = align_up(off + sizeof(T) * (size_t)count);
  } else {
    ptr = nullptr;
  }
}

size_t layout(hdda_grid* g, char* base) {
  const bool vdb = g->kind == HDDA_GRID_VDB;
  size_t off = 0;
  carve(base, off, g->thr, g->thr_count(), true);
  carve(base, off, g->bits, (int64_t)g->L * g->W, !vdb);
  const int64_t nw = g->nodes_total() * kNodeWords;
  carve(base, off, g->child, nw, vdb);
  carve(base, off, g->tile, nw, vdb);
  carve(base, off, g->prefix, nw, vdb);
  carve(base, off, g->nstate, g->nodes_total(), vdb);
  carve(base, off, g->leaves, g->blocks_total() * kLeafWords, vdb);
  carve(base, off, g->nsuper, g->nodes_total() * kSuperWords, vdb);
  carve(base, off, g->lsub, g->blocks_total() * kLeafSubWords, vdb);
  carve(base, off, g->rmap, g->map_cells(), vdb);
  carve(base, off, g->blk_masks, g->blocks_total() * kLeafWords, vdb);
  carve(base, off, g->blk_state, g->blocks_total(), vdb);
  carve(base, off, g->local_prefix, nw, vdb);
  carve(base, off, g->node_leaves, g->nodes_total(), vdb);
  carve(base, off, g->node_tiles, g->nodes_total(), vdb);
  carve(base, off, g->totals, 2, vdb);
  return off;
}

unsigned blocks_for(int64_t threads, int per) { return (unsigned)((threads + per - 1) / per); }

// CTAs of the update's gated grid-stride kernels: eight 256-thread CTAs per SM of a
// 152-SM GB300, about one resident wave
constexpr unsigned kGatedCtas = 152 * 8;

int launch_build(hdda_grid* g, const uint8_t* dense, cudaStream_t s) {
  if (g->kind == HDDA_GRID_DENSE) {
    const int64_t words = (int64_t)g->L * g->W;
    KernelTimer kt("pack_dense", s);
    pack_dense_kernel<<<blocks_for(words, 256), 256, 0, s>>>(dense, g->L, g->R, g->W, g->bits);
    kt.stop();
    HDDA_CUDA_TRY(cudaGetLastError());
  } else {
    const int64_t nblk = g->blocks_total();
    KernelTimer kt("build_vdb", s);  // the five build kernels together
    vdb_blocks_kernel<<<blocks_for(nblk * 32, 256), 256, 0, s>>>(dense, g->L, g->R, g->B,
                                                                 g->blk_masks, g->blk_state);
    HDDA_CUDA_TRY(cudaGetLastError());
    vdb_nodes_kernel<<<(unsigned)g->nodes_total(), kNodeWords, 0, s>>>(
        g->L, g->B, g->N, g->blk_state, g->child, g->tile, g->local_prefix, g->node_leaves,
        g->node_tiles, g->nstate, g->nsuper, nullptr);
    HDDA_CUDA_TRY(cudaGetLastError());
    vdb_finalize_kernel<<<1, 1024, 0, s>>>(g->nodes_total(), g->node_leaves, g->node_tiles,
                                          g->local_prefix, g->prefix, g->totals, nullptr);
    HDDA_CUDA_TRY(cudaGetLastError());
    vdb_scatter_kernel<<<blocks_for(nblk * 16, 256), 256, 0, s>>>(
        g->L, g->B, g->N, g->blk_state, g->blk_masks, g->child, g->prefix, g->leaves, g->lsub,
        nullptr);
    HDDA_CUDA_TRY(cudaGetLastError());
    region_map_kernel<<<blocks_for(g->map_cells(), 256), 256, 0, s>>>(g->view(), g->rmap,
                                                                       nullptr);
    kt.stop();
    HDDA_CUDA_TRY(cudaGetLastError());
  }
  HDDA_CUDA_TRY(cudaEventRecord(g->built, s));
  return HDDA_OK;
}

int create(int kind, const uint8_t* dense, int levels, int res, const hdda_aabb* aabbs,
           hdda_grid** out, cudaStream_t s) {
  clear_error();
  if (!out) return set_error(HDDA_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int st = validate(dense, levels, res, aabbs);
  if (st != HDDA_OK) return st;
  hdda_grid* g = new (std::nothrow) hdda_grid();
  if (!g) return set_error(HDDA_ERR_OOM, "host allocation failed");
  g->kind = kind;
  g->L = levels;
  g->R = res;
  g->B = (res + kBlockDim - 1) / kBlockDim;
  g->N = (g->B + kNodeDim - 1) / kNodeDim;
  g->W = (int)(((int64_t)res * res * res + 31) / 32);
  cudaError_t e = cudaGetDevice(&g->device);
  if (e != cudaSuccess) { delete g; return cuda_error(e, "cudaGetDevice"); }
  for (int l = 0; l < levels; ++l) {
    g->boxes[l] = aabbs[l];
    for (int c = 0; c < 3; ++c) g->scale[l][c] = (float)res / (aabbs[l].hi[c] - aabbs[l].lo[c]);
  }
  g->base_bytes = layout(g, nullptr);
  e = cudaMalloc(&g->base, g->base_bytes);
  if (e != cudaSuccess) { delete g; return cuda_error(e, "cudaMalloc(grid)"); }
  layout(g, static_cast<char*>(g->base));
  e = cudaEventCreateWithFlags(&g->built, cudaEventDisableTiming);
  if (e != cudaSuccess) { hdda_grid_free(g); return cuda_error(e, "cudaEventCreate"); }
  thresholds_kernel<<<blocks_for(g->thr_count(), 128), 128, 0, s>>>(g->view(), g->thr);
  e = cudaGetLastError();
  if (e != cudaSuccess) { hdda_grid_free(g); return cuda_error(e, "thresholds_kernel"); }
  st = launch_build(g, dense, s);
  if (st != HDDA_OK) { hdda_grid_free(g); return st; }
  *out = g;
  return HDDA_OK;
}

int64_t structure_bytes(const hdda_grid* g, int64_t n_leaves) {
  int64_t b = (int64_t)g->L * (int64_t)sizeof(LevelDev) + g->thr_count() * 4;
  if (g->kind == HDDA_GRID_DENSE) {
    b += (int64_t)g->L * g->W * 4;
  } else {
    b += g->nodes_total() * (3 * kNodeWords * 4 + 4);
    b += n_leaves * kLeafWords * 4;
    if (g->refine) b += g->nodes_total() * kSuperWords * 4 + n_leaves * kLeafSubWords * 4;
  }
  return b;
}

}  // namespace
}  // namespace hdda

using namespace hdda;

extern "C" int hdda_pack_dense(const uint8_t* dense, int levels, int res, const hdda_aabb* aabbs,
                               hdda_grid** out, hdda_stream_t stream) {
  return create(HDDA_GRID_DENSE, dense, levels, res, aabbs, out, (cudaStream_t)stream);
}

extern "C" int hdda_build_vdb(const uint8_t* dense, int levels, int res, const hdda_aabb* aabbs,
                              hdda_grid** out, size_t* bytes_out, hdda_stream_t stream) {
  int st = create(HDDA_GRID_VDB, dense, levels, res, aabbs, out, (cudaStream_t)stream);
  if (st != HDDA_OK || !bytes_out) return st;
  hdda_grid_stats gs;
  st = hdda_grid_stats_get(*out, &gs);
  if (st != HDDA_OK) return st;
  *bytes_out = (size_t)gs.bytes;
  return HDDA_OK;
}

extern "C" int hdda_grid_rebuild(hdda_grid* grid, const uint8_t* dense, hdda_stream_t stream) {
  clear_error();
  if (!grid) return set_error(HDDA_ERR_INVALID_ARG, "grid is NULL");
  if (!dense) return set_error(HDDA_ERR_INVALID_ARG, "dense is NULL");
  return launch_build(grid, dense, (cudaStream_t)stream);
}

namespace hdda {
namespace {

// Pinned host word for the synchronous status read of an update.
struct UpdateWord {
  unsigned* p = nullptr;
  ~UpdateWord() { if (p) cudaFreeHost(p); }
};
thread_local UpdateWord t_update_word;

int update_vdb(hdda_grid* g, const uint8_t* dense, const int64_t* blocks, int64_t n_blocks,
               uint32_t* dev_status, cudaStream_t s) {
  const int64_t count = blocks ? n_blocks : g->blocks_total();
  if (count == 0) return HDDA_OK;
  unsigned* hw = nullptr;
  if (!dev_status) {
    if (!t_update_word.p) HDDA_CUDA_TRY(cudaMallocHost(&t_update_word.p, sizeof(unsigned)));
    hw = t_update_word.p;
  }
  // scratch: {flags[0] = structure changed, status}, then changed[count]
  char* scratch = nullptr;
  HDDA_CUDA_TRY(cudaMallocAsync(&scratch, 16 + (size_t)count, s));
  unsigned* flags = reinterpret_cast<unsigned*>(scratch);
  unsigned* status = dev_status ? dev_status : flags + 1;
  uint8_t* changed = reinterpret_cast<uint8_t*>(scratch + 16);
  int st = HDDA_OK;
  cudaError_t e = cudaMemsetAsync(scratch, 0, 16, s);
  if (e != cudaSuccess) st = cuda_error(e, "cudaMemsetAsync");
  if (st == HDDA_OK) {
    KernelTimer kt("update_vdb", s);  // the update's seven kernels together
    vdb_update_blocks_kernel<<<blocks_for(count * 32, 256), 256, 0, s>>>(
        dense, g->L, g->R, g->B, blocks, count, g->blk_masks, g->blk_state, changed, flags,
        status);
    vdb_nodes_kernel<<<(unsigned)g->nodes_total(), kNodeWords, 0, s>>>(
        g->L, g->B, g->N, g->blk_state, g->child, g->tile, g->local_prefix, g->node_leaves,
        g->node_tiles, g->nstate, g->nsuper, flags);
    vdb_finalize_kernel<<<1, 1024, 0, s>>>(g->nodes_total(), g->node_leaves, g->node_tiles,
                                          g->local_prefix, g->prefix, g->totals, flags);
    // the gated kernels run as grid-stride loops over a grid of at most kGatedCtas CTAs,
    // so that they cost next to nothing when the update changed no block's state
    vdb_scatter_kernel<<<std::min(blocks_for(g->blocks_total() * 16, 256), kGatedCtas), 256, 0,
                         s>>>(g->L, g->B, g->N, g->blk_state, g->blk_masks, g->child, g->prefix,
                              g->leaves, g->lsub, flags);
    vdb_rewrite_leaves_kernel<<<blocks_for(count * 16, 256), 256, 0, s>>>(
        g->B, g->N, blocks, count, changed, flags, g->blk_state, g->blk_masks, g->child,
        g->prefix, g->leaves, g->lsub);
    region_map_kernel<<<std::min(blocks_for(g->map_cells(), 256), kGatedCtas), 256, 0, s>>>(
        g->view(), g->rmap, flags);
    region_map_blocks_kernel<<<blocks_for(count * 64, 256), 256, 0, s>>>(
        g->view(), g->rmap, blocks, count, changed, flags);
    kt.stop();
    e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_error(e, "update kernels");
  }
  if (st == HDDA_OK && !dev_status) {
    e = cudaMemcpyAsync(hw, flags + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = cuda_error(e, "cudaMemcpyAsync(status)");
  }
  e = cudaFreeAsync(scratch, s);
  if (st == HDDA_OK && e != cudaSuccess) st = cuda_error(e, "cudaFreeAsync");
  if (st != HDDA_OK) return st;
  HDDA_CUDA_TRY(cudaEventRecord(g->built, s));
  if (dev_status) return HDDA_OK;
  HDDA_CUDA_TRY(cudaStreamSynchronize(s));
  if (*hw & kDevBadIndex)
    return set_error(HDDA_ERR_INVALID_ARG, "a block index lies outside the grid (skipped)");
  return HDDA_OK;
}

}  // namespace
}  // namespace hdda

extern "C" int hdda_grid_update(hdda_grid* grid, const uint8_t* dense, const int64_t* blocks,
                                int64_t n_blocks, uint32_t* dev_status, hdda_stream_t stream) {
  clear_error();
  if (!grid) return set_error(HDDA_ERR_INVALID_ARG, "grid is NULL");
  if (!dense) return set_error(HDDA_ERR_INVALID_ARG, "dense is NULL");
  if (blocks && (n_blocks < 0 || n_blocks > ((int64_t)1 << 26)))
    return set_error(HDDA_ERR_INVALID_ARG, "n_blocks=%lld outside 0..2^26", (long long)n_blocks);
  if (reinterpret_cast<uintptr_t>(dev_status) % 4 != 0)
    return set_error(HDDA_ERR_INVALID_ARG, "dev_status must be 4-byte aligned");
  int dev = 0;
  HDDA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != grid->device)
    return set_error(HDDA_ERR_INVALID_ARG, "grid lives on device %d, current is %d",
                     grid->device, dev);
  cudaStream_t s = (cudaStream_t)stream;
  if (grid->kind == HDDA_GRID_DENSE) return launch_build(grid, dense, s);  // one repack
  return update_vdb(grid, dense, blocks, n_blocks, dev_status, s);
}

extern "C" int hdda_grid_stats_get(const hdda_grid* g, hdda_grid_stats* out) {
  clear_error();
  if (!g || !out) return set_error(HDDA_ERR_INVALID_ARG, "grid or out is NULL");
  std::memset(out, 0, sizeof(*out));
  out->kind = g->kind;
  out->levels = g->L;
  out->res = g->R;
  out->blocks = g->B;
  out->nodes = g->N;
  out->dense_bytes = (int64_t)g->L * g->W * 4;
  int64_t totals[2] = {0, 0};
  if (g->kind == HDDA_GRID_VDB) {
    HDDA_CUDA_TRY(cudaEventSynchronize(g->built));
    HDDA_CUDA_TRY(cudaMemcpy(totals, g->totals, sizeof(totals), cudaMemcpyDeviceToHost));
  }
  out->n_leaves = totals[0];
  out->n_tiles = totals[1];
  out->bytes = structure_bytes(g, totals[0]);
  if (g->kind == HDDA_GRID_VDB) out->map_bytes = g->map_cells() * (int64_t)sizeof(uint16_t);
  return HDDA_OK;
}

extern "C" int hdda_grid_copy_array(const hdda_grid* g, int which, void* dst, size_t bytes,
                                    size_t* needed) {
  clear_error();
  if (!g) return set_error(HDDA_ERR_INVALID_ARG, "grid is NULL");
  const bool vdb = g->kind == HDDA_GRID_VDB;
  const void* src = nullptr;
  size_t n = 0;
  const size_t nw = (size_t)g->nodes_total() * kNodeWords * 4;
  switch (which) {
    case HDDA_ARRAY_THRESHOLDS: src = g->thr; n = (size_t)g->thr_count() * 4; break;
    case HDDA_ARRAY_DENSE_BITS: if (!vdb) { src = g->bits; n = (size_t)g->L * g->W * 4; } break;
    case HDDA_ARRAY_CHILD_MASK: if (vdb) { src = g->child; n = nw; } break;
    case HDDA_ARRAY_TILE_MASK: if (vdb) { src = g->tile; n = nw; } break;
    case HDDA_ARRAY_LEAF_PREFIX: if (vdb) { src = g->prefix; n = nw; } break;
    case HDDA_ARRAY_LEAVES:
    case HDDA_ARRAY_LEAF_SUB:
      if (vdb) {
        hdda_grid_stats gs;
        int st = hdda_grid_stats_get(g, &gs);
        if (st != HDDA_OK) return st;
        const bool sub = which == HDDA_ARRAY_LEAF_SUB;
        src = sub ? g->lsub : g->leaves;
        n = (size_t)gs.n_leaves * (sub ? kLeafSubWords : kLeafWords) * 4;
      }
      break;
    case HDDA_ARRAY_NODE_SUPER:
      if (vdb) { src = g->nsuper; n = (size_t)g->nodes_total() * kSuperWords * 4; }
      break;
    case HDDA_ARRAY_REGION_MAP:
      if (vdb) { src = g->rmap; n = (size_t)g->map_cells() * sizeof(uint16_t); }
      break;
    default: break;
  }
  if (!src) return set_error(HDDA_ERR_INVALID_ARG, "array %d not held by this grid", which);
  if (needed) *needed = n;
  if (!dst) return HDDA_OK;
  if (bytes < n) return set_error(HDDA_ERR_CAPACITY, "array needs %zu bytes, got %zu", n, bytes);
  HDDA_CUDA_TRY(cudaEventSynchronize(g->built));
  if (n) HDDA_CUDA_TRY(cudaMemcpy(dst, src, n, cudaMemcpyDeviceToHost));
  return HDDA_OK;
}

extern "C" int hdda_grid_set_refine(hdda_grid* g, int on) {
  clear_error();
  if (!g) return set_error(HDDA_ERR_INVALID_ARG, "grid is NULL");
  if (g->kind != HDDA_GRID_VDB)
    return set_error(HDDA_ERR_INVALID_ARG, "refinement applies to VDB grids");
  g->refine = on ? 1 : 0;
  return HDDA_OK;
}

extern "C" int hdda_grid_set_walk(hdda_grid* g, int variant) {
  clear_error();
  if (!g) return set_error(HDDA_ERR_INVALID_ARG, "grid is NULL");
  if (variant != HDDA_WALK_BRANCH && variant != HDDA_WALK_SKIP)
    return set_error(HDDA_ERR_INVALID_ARG, "walk variant %d unknown", variant);
  g->walk_variant = variant;
  return HDDA_OK;
}

extern "C" void hdda_grid_free(hdda_grid* g) {
  if (!g) return;
  if (g->built) {
    cudaEventSynchronize(g->built);
    cudaEventDestroy(g->built);
  }
  if (g->base) {
    cudaDeviceSynchronize();
    cudaFree(g->base);
  }
  delete g;
}
