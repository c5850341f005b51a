/*
 * hdda.h -- C ABI of libhdda, a GB300 (sm_103a) occupancy-grid ray sampler
 * with VDB-style sparse grids and hierarchical DDA.
 *
 * Method: Kato & Tarashima, "Plug-and-Play Acceleration of Occupancy
 * Grid-based NeRF Rendering using VDB Grid and Hierarchical Ray Traversal"
 * (CVPR-W 2024).  A trained dense binary occupancy grid, one level or a
 * cascade of levels whose voxel size doubles (Sec. 4.1), is rebuilt into a
 * sparse tree whose uniform blocks become tiles (Sec. 3), and every camera
 * ray is walked with hierarchical DDA, which skips a whole empty node in one
 * step (Sec. 2.3, Fig. 1), keeping the lattice samples that fall in occupied
 * voxels (Algorithm 1).  The dense-grid DDA walk it replaces is exported
 * beside it.
 *
 * Conventions for every call
 *   - Pointers are DEVICE pointers owned by the caller unless a parameter
 *     says "host".  The library never frees caller memory.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     are stream-ordered and return before the GPU work finishes, except
 *     where a host value is returned (noted per call): those synchronise the
 *     stream once.
 *   - Every call returns an hdda_status; 0 is success.  On failure
 *     hdda_last_error() gives a message (thread-local).  No C++ exception
 *     crosses this boundary.  A failed call leaves outputs unspecified.
 *   - Grids are read-only while any traversal that uses them is in flight.
 *
 * Grid layout conventions
 *   - Dense occupancy input: uint8 [levels][res][res][res], C order
 *     (x slowest, z fastest), non-zero = occupied.  Level 0 is the finest.
 *   - Level boxes are half-open [lo, hi) per axis.  A point belongs to the
 *     finest level whose box holds it (Sec. 3, last paragraph).
 *   - Voxel index of a point x at level l, per axis c, in binary32 with no
 *     fused multiply-add:
 *         s_c = res / (hi_c - lo_c)
 *         i_c = clamp(floor((x_c - lo_c) * s_c), 0, res - 1)
 */
#ifndef HDDA_H
#define HDDA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; declared here so the ABI needs no CUDA header. */
typedef struct CUstream_st* hdda_stream_t;

typedef enum {
    HDDA_OK = 0,
    HDDA_ERR_INVALID_ARG = 1, /* bad pointer, size, shape or parameter      */
    HDDA_ERR_CUDA = 2,        /* a CUDA runtime call failed                 */
    HDDA_ERR_CAPACITY = 3,    /* output buffer smaller than the sample count */
    HDDA_ERR_STEP_LIMIT = 4,  /* lattice longer than params.max_steps       */
    HDDA_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up         */
    HDDA_ERR_OOM = 6,         /* device allocation failed                   */
    HDDA_ERR_INTERNAL = 7     /* a device-side consistency check failed     */
} hdda_status;

#define HDDA_MAX_LEVELS 8
#define HDDA_MAX_RES 1024

/* Half-open box [lo, hi) of one cascade level, in world units. */
typedef struct {
    float lo[3];
    float hi[3];
} hdda_aabb;

/*
 * Lattice parameters shared by every ray of a call (Sec. 3: constant step
 * for bounded scenes, linearly increasing step for unbounded ones;
 * Algorithm 1: the lattice advances independently of voxel boundaries).
 * In binary32, no fused multiply-add:
 *     t_0 = near_t
 *     t_{k+1} = t_k + min(max(t_k * cone_angle, step), max_step)
 *     candidate k exists iff t_{k+1} <= far_t
 * All values finite; step > 0, max_step > 0, cone_angle >= 0,
 * 0 <= max_steps <= 2^24.  More candidates than max_steps is
 * HDDA_ERR_STEP_LIMIT.  Directions need not be unit length: t is in units
 * of |d|.
 *
 * image_width is a hint on the order of the rays, not a lattice parameter:
 * 0, or the width W of an image whose pixels the rays are, row by row (ray r
 * is pixel (r mod W, r div W); the last row may be partial).  With W > 0 the
 * walk of hdda_traverse_hdda, hdda_traverse_dense, hdda_traverse_async,
 * hdda_render and hdda_traverse_composite takes the rays in 8 x 4 pixel
 * blocks, so that the rays a warp walks together are neighbours in both
 * image axes; every output is the same as with 0, bit for bit.  The fused
 * sampler form, the batched sampler and hdda_traverse_hdda_noalloc ignore
 * it.  Negative is HDDA_ERR_INVALID_ARG.
 */
typedef struct {
    float near_t;
    float far_t;
    float step;
    float cone_angle;
    float max_step;
    int32_t max_steps;
    int32_t image_width;
} hdda_params;

typedef struct hdda_grid hdda_grid; /* opaque, library-owned device object */

typedef enum { HDDA_GRID_DENSE = 0, HDDA_GRID_VDB = 1 } hdda_grid_kind;

typedef struct {
    int32_t kind;        /* hdda_grid_kind                                  */
    int32_t levels;
    int32_t res;
    int32_t blocks;      /* ceil(res / 8): 8^3-voxel blocks per axis        */
    int32_t nodes;       /* ceil(blocks / 16): 16^3-block nodes per axis    */
    int32_t reserved;
    int64_t n_leaves;    /* VDB: stored 8^3 leaf bitmasks (partial blocks)  */
    int64_t n_tiles;     /* VDB: fully occupied blocks stored as tile bits  */
    int64_t bytes;       /* bytes the traversal reads: level table,
                            index thresholds, masks and leaves (Table 3)    */
    int64_t dense_bytes; /* levels * ceil(res^3 / 32) * 4: the dense bit
                            array the paper starts from (Table 3 caption)   */
    int64_t map_bytes;   /* VDB: the region map HDDA reads with refinement
                            on (HDDA_ARRAY_REGION_MAP), 2 bytes per 2^3
                            cell per level; not part of `bytes`            */
} hdda_grid_stats;

/* Arrays of a grid that hdda_grid_copy_array can export. */
typedef enum {
    /* float [levels][3][res+1]: X[a] = smallest binary32 x in [lo, hi] whose
       voxel index (formula above) is >= a; X[0] = lo, X[res] = hi.  Voxel a
       along axis c is exactly [X[a], X[a+1]).                               */
    HDDA_ARRAY_THRESHOLDS = 0,
    /* uint32 [levels][ceil(res^3/32)]: voxel (x, y, z) of level l is bit
       ((x*res + y)*res + z) of level l's bit string, bit b of word w being
       voxel 32w + b (DENSE grids).                                          */
    HDDA_ARRAY_DENSE_BITS = 1,
    /* uint32 [levels][nodes^3][128]: 4096-bit child mask per node; block
       (bx, by, bz) is cell ((bx%16)*16 + by%16)*16 + bz%16 of node
       ((bx/16)*nodes + by/16)*nodes + bz/16; a bit is set when the block is
       partly occupied (VDB grids).                                          */
    HDDA_ARRAY_CHILD_MASK = 2,
    /* uint32 [levels][nodes^3][128]: tile mask, set when all 512 voxels of
       the block exist and are occupied (VDB grids).                          */
    HDDA_ARRAY_TILE_MASK = 3,
    /* uint32 [levels][nodes^3][128]: global index of the first leaf whose
       cell lies in each child-mask word (VDB grids).                         */
    HDDA_ARRAY_LEAF_PREFIX = 4,
    /* uint32 [n_leaves][16]: 512-bit leaf masks in (level, node, cell)
       order; voxel (x%8, y%8, z%8) is bit ((x%8)*8 + y%8)*8 + z%8 (VDB).    */
    HDDA_ARRAY_LEAVES = 5,
    /* uint32 [levels][nodes^3][18] refinement masks of each node (VDB): words
       0-1 = 64 bits, one per 32^3-voxel group g = (gx*4 + gy)*4 + gz with
       gc = (voxel_c % 128) / 32; words 2-17 = 512 bits, one per 16^3-voxel
       group g = (gx*8 + gy)*8 + gz with gc = (voxel_c % 128) / 16.  A bit is
       set when the group holds an occupied voxel.                           */
    HDDA_ARRAY_NODE_SUPER = 6,
    /* uint32 [n_leaves][5] refinement masks of each leaf (VDB), leaf order as
       HDDA_ARRAY_LEAVES: words 0-1 = 64 bits, one per 2^3-voxel cell
       c = (cx*4 + cy)*4 + cz with cc = (voxel_c % 8) / 2; word 2 = 8 bits,
       one per 4^3-voxel cell c = (cx*2 + cy)*2 + cz with cc = (voxel_c % 8)
       / 4 (a bit is set when the cell holds an occupied voxel); words 3-4 =
       64 bits over the 2^3-voxel cells again, set when all 8 voxels of the
       cell are occupied.                                                     */
    HDDA_ARRAY_LEAF_SUB = 7,
    /* uint16 [levels][C][C][C], C = ceil(res / 2): the region map (VDB), one
       entry per 2^3-voxel cell (voxel_c / 2 per axis).  Bits 8-15: log2 of
       the edge of the coarsest uniform region of the refined tree holding
       the cell: 7 = an empty or full 128^3 node, 5 / 4 = an empty 32^3 /
       16^3 group, 3 = an empty or tiled 8^3 block, 2 = an empty or full 4^3
       cell, 1 = an empty or full 2^3 cell, 0 = the cell is not uniform.  Bits 0-7:
       voxel (x, y, z) of the cell is bit ((x%2)*2 + y%2)*2 + z%2; all eight
       equal (0x00 or 0xff) when the region is uniform.                       */
    HDDA_ARRAY_REGION_MAP = 8
} hdda_array;

/* Version string of the library. */
const char* hdda_version(void);

/* Message of the last failed call on this host thread ("" if none). */
const char* hdda_last_error(void);

/*
 * Dense grid for the dense-DDA baseline: packs `dense` into the bit array
 * the paper starts from (Sec. 2.2: the occupancy grid is a dense binary grid;
 * Table 3: 128^3 grid = 256 KiB) and builds the per-axis index thresholds.
 *   dense   device uint8 [levels][res][res][res]
 *   levels  1..HDDA_MAX_LEVELS;  res 1..HDDA_MAX_RES
 *   aabbs   HOST array of `levels` boxes, finite, lo < hi per axis
 *   out     receives a new grid; free it with hdda_grid_free
 * Stream-ordered; `dense` may be reused once the stream has passed the call.
 */
int hdda_pack_dense(const uint8_t* dense, int levels, int res, const hdda_aabb* aabbs,
                    hdda_grid** out, hdda_stream_t stream);

/*
 * VDB-style sparse grid for hierarchical DDA (Sec. 3: the dense grid becomes
 * a VDB tree; blocks that hold one value become tiles).  Per level: 8^3 leaf
 * bitmasks for partly occupied blocks, and per 16^3-block node a child mask,
 * a tile mask and a leaf-index prefix table.  Arguments as hdda_pack_dense;
 * bytes_out (HOST, may be NULL) receives hdda_grid_stats.bytes, which makes
 * the call synchronise the stream once.
 */
int hdda_build_vdb(const uint8_t* dense, int levels, int res, const hdda_aabb* aabbs,
                   hdda_grid** out, size_t* bytes_out, hdda_stream_t stream);

/*
 * Rebuilds a grid in place from new occupancy of the same shape (levels,
 * res and boxes unchanged), e.g. after an occupancy update during training.
 * Allocates nothing and does not synchronise; traversals queued on other
 * streams must not overlap it.
 */
int hdda_grid_rebuild(hdda_grid* grid, const uint8_t* dense, hdda_stream_t stream);

/*
 * Incremental rebuild: updates a VDB grid to new occupancy when only some
 * 8^3 blocks may have changed (an occupancy update during training touches
 * part of the grid; the paper's grid is read-only on the GPU and re-pruned
 * on the CPU, Sec. 5).  The result is bit for bit the grid a full rebuild
 * from `dense` gives, provided every block outside the list is unchanged.
 *   dense        device uint8 [levels][res][res][res], the NEW occupancy
 *   blocks       device int64 [n_blocks]: indices l * B^3 + (bx * B + by) * B
 *                + bz of the 8^3 blocks that may have changed (B = ceil(res
 *                / 8), block (bx, by, bz) holds voxels 8 bx .. 8 bx + 7 on x,
 *                and so on); duplicates are allowed; NULL = every block
 *   n_blocks     0..2^26 (ignored when blocks is NULL)
 *   dev_status   NULL: the call synchronises the stream once and returns
 *                HDDA_ERR_INVALID_ARG if an index lay outside the grid (such
 *                entries are skipped).  Otherwise a DEVICE uint32 (4-byte
 *                aligned) that receives the status bits by atomic OR (bit 4 =
 *                index outside the grid); no synchronisation.
 * Work: the listed blocks are re-masked from `dense` and compared with the
 * masks kept from the last build.  When no block changes between empty,
 * partial and full, only the changed leaves are rewritten in place;
 * otherwise the node masks and the leaf pool are rebuilt from the kept block
 * masks (no dense byte outside the list is read).  Scratch of 16 + n_blocks
 * bytes comes from the stream-ordered allocator.  A dense grid is simply
 * repacked.  Like hdda_grid_rebuild, it must not overlap traversals of the
 * grid queued on other streams.
 */
int hdda_grid_update(hdda_grid* grid, const uint8_t* dense, const int64_t* blocks,
                     int64_t n_blocks, uint32_t* dev_status, hdda_stream_t stream);

/* Fills *out (HOST).  Synchronises the grid's last build stream. */
int hdda_grid_stats_get(const hdda_grid* grid, hdda_grid_stats* out);

/*
 * Copies one exported array (see hdda_array) into HOST memory `dst` of
 * `bytes` bytes; *needed (HOST, may be NULL) receives its size.  With
 * dst == NULL only the size is returned.  Synchronous.  An array the grid's
 * kind does not hold is HDDA_ERR_INVALID_ARG.
 */
int hdda_grid_copy_array(const hdda_grid* grid, int which, void* dst, size_t bytes,
                         size_t* needed);

/*
 * Chooses the hierarchy hdda_traverse_hdda walks on a VDB grid.  on = 1 (the
 * default): besides empty nodes, empty or tiled 8^3 blocks and single leaf
 * voxels, it also crosses empty 32^3 and 16^3 groups inside a node and
 * empty or full 4^3 and 2^3 cells inside a leaf in one step each, an
 * octree-style refinement of the VDB tree (Sec. 5 names finer subdivision
 * as worth studying).  The walk finds each region in the region map
 * (HDDA_ARRAY_REGION_MAP, built with the tree) by one lookup.  on = 0: the
 * plain tree of 8^3 leaves under 16^3-block nodes, descended per region.
 * Results are identical either way.  Not for dense grids.
 */
int hdda_grid_set_refine(hdda_grid* grid, int on);

/*
 * Control flow of the per-ray walk of hdda_traverse_dense / hdda_traverse_hdda
 * on this grid (supplementary material, Algorithms 1 and 2):
 *   HDDA_WALK_BRANCH (default): one region per step, branching on its
 *     occupancy ("DDA branch", Algorithm 1);
 *   HDDA_WALK_SKIP: every run of leading empty regions is crossed in an
 *     inner loop before the occupied region is taken ("DDA skip",
 *     Algorithm 2, read as t1 <- t_last and `until grid.at(ijk)`).
 * The samples are identical; only the SIMT schedule differs.  Batches and
 * hdda_traverse_hdda_noalloc always use the branch form.
 */
typedef enum { HDDA_WALK_BRANCH = 0, HDDA_WALK_SKIP = 1 } hdda_walk_variant;
int hdda_grid_set_walk(hdda_grid* grid, int variant);

/* Frees a grid (waits for the device to finish with it).  NULL is a no-op. */
void hdda_grid_free(hdda_grid* grid);

/*
 * Dense-grid DDA sampler (the baseline the paper replaces; Algorithm 1 with
 * DDA as the analyzer).  Each ray walks the voxels of the dense bit array
 * that its lattice visits, one lookup per voxel, and keeps every lattice
 * interval whose midpoint voxel is occupied at the finest level holding it.
 *   rays_o, rays_d  device float [n_rays][3]; a ray with a non-finite
 *                   component has no samples
 *   grid            a HDDA_GRID_DENSE grid
 *   params          HOST pointer
 *   offsets         device int64 [n_rays + 1]: receives CSR row pointers
 *                   (offsets[r]..offsets[r+1] are ray r's samples)
 *   ray_idx, t0, t1 device int32 / float / float [capacity]: the kept
 *                   intervals (r, t_k, t_{k+1}), rays in order, each ray's
 *                   intervals in ascending k
 *   capacity        0 = count only: offsets and *total_out are filled and
 *                   nothing else is written.  Otherwise, if capacity < total
 *                   the call returns HDDA_ERR_CAPACITY (with *total_out set),
 *                   writes no sample at or past index capacity, and clamps
 *                   the offsets to capacity (so that they describe exactly
 *                   the samples written and a consumer stays in bounds).
 *   total_out       HOST int64: number of kept intervals
 * Kernels in stream order; the call synchronises the stream once at the
 * end to read the total, so every output is complete when it returns.
 */
int hdda_traverse_dense(const float* rays_o, const float* rays_d, int64_t n_rays,
                        const hdda_grid* grid, const hdda_params* params, int64_t* offsets,
                        int32_t* ray_idx, float* t0, float* t1, int64_t capacity,
                        int64_t* total_out, hdda_stream_t stream);

/*
 * Hierarchical-DDA sampler over a VDB grid (Sec. 2.3 and Sec. 3; Algorithm 1
 * with HDDA as the analyzer).  Arguments and outputs as hdda_traverse_dense;
 * `grid` must be a HDDA_GRID_VDB grid built from the same occupancy.  Empty
 * nodes, empty blocks, tiles and single voxels are each crossed in one step;
 * the result is bit-identical to hdda_traverse_dense.
 */
int hdda_traverse_hdda(const float* rays_o, const float* rays_d, int64_t n_rays,
                       const hdda_grid* grid, const hdda_params* params, int64_t* offsets,
                       int32_t* ray_idx, float* t0, float* t1, int64_t capacity,
                       int64_t* total_out, hdda_stream_t stream);

/*
 * Either sampler in stream order: the same outputs as hdda_traverse_hdda (a
 * VDB grid) or hdda_traverse_dense (a dense grid), without the read-back of
 * the total and without any synchronisation, so that a consumer such as
 * hdda_composite can be queued right behind it.
 *   offsets         as above; the total is offsets[n_rays], on the device
 *   capacity        as above (0 = count only); a capacity below the total
 *                   raises bit 2 of *dev_status, writes no sample at or past
 *                   capacity and clamps the offsets to capacity
 *   dev_status      DEVICE uint32 (required, 4-byte aligned) that receives
 *                   status bits by atomic OR: bit 1 = internal region check
 *                   failed (only while hdda_set_region_checks is on), bit 2 =
 *                   capacity below the total
 * The first use of a parameter set synchronises once (the lattice is
 * computed then).  Scratch comes from the stream-ordered allocator.
 */
int hdda_traverse_async(const float* rays_o, const float* rays_d, int64_t n_rays,
                        const hdda_grid* grid, const hdda_params* params, int64_t* offsets,
                        int32_t* ray_idx, float* t0, float* t1, int64_t capacity,
                        uint32_t* dev_status, hdda_stream_t stream);

/*
 * Hierarchical-DDA sampler that allocates nothing, for callers that must not
 * allocate GPU memory: applications that reserve all device memory up front
 * and hand libraries fixed buffers, or loops that must never enter the CUDA
 * allocator.  The paper has no counterpart; it is a deployment variant of
 * hdda_traverse_hdda with the same arguments and the same results.
 *
 * Its per-call scratch (lattice table, per-CTA sums and counters) lives in
 * one fixed device array of 393,728 bytes inside the library, present on
 * every GPU that loads the library until the process exits; the lattice is
 * recomputed on every call instead of being cached.  Limits, rejected with
 * HDDA_ERR_INVALID_ARG and a message: n_rays <= 2,097,152 and at most
 * 16,384 lattice candidates per ray.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) and should come before any stream capture.  All
 * calls share the array: calls whose GPU work overlaps race on it and must
 * be serialised by the caller.  Every call, not only the first, synchronises
 * the stream twice (lattice length, sample total), so no call can be
 * captured into a CUDA graph; every output is complete when it returns.
 */
int hdda_traverse_hdda_noalloc(const float* rays_o, const float* rays_d, int64_t n_rays,
                               const hdda_grid* grid, const hdda_params* params,
                               int64_t* offsets, int32_t* ray_idx, float* t0, float* t1,
                               int64_t capacity, int64_t* total_out, hdda_stream_t stream);

/*
 * Batched sampling: many traversal jobs in one launch sequence.
 *
 * Each job is one traversal with its own rays, grid, lattice parameters and
 * output buffers (the fields mean what the arguments of hdda_traverse_hdda
 * mean; a job's `capacity` may be 0 to count only).  All grids of a batch
 * must be of one kind (dense, VDB, or VDB with refinement off).  The jobs'
 * rays are cut into 32-ray tiles numbered over the whole batch; persistent
 * warps take tiles from one counter (work stealing across jobs), so jobs of
 * very different sizes share the GPU without a launch per job.  A batch is
 * a plan: hdda_batch_create fixes the job table and scratch (and, with
 * use_graph, captures the launch sequence into a CUDA graph); every
 * hdda_batch_launch re-runs it, reading whatever the job buffers then hold.
 * Buffers and grids must stay alive and unchanged in shape while the batch
 * exists.  Not in the paper (its renderer draws one frame at a time); this is
 * the throughput path for many cameras and scenes.
 */
typedef struct {
    const float* rays_o;     /* device float [n_rays][3]                    */
    const float* rays_d;     /* device float [n_rays][3]                    */
    int64_t n_rays;
    const hdda_grid* grid;
    hdda_params params;
    int64_t* offsets;        /* device int64 [n_rays + 1]                  */
    int32_t* ray_idx;        /* device [capacity]                          */
    float* t0;
    float* t1;
    int64_t capacity;
} hdda_job;

typedef struct {
    int walk_block;      /* threads per CTA of the walk: 128, 256 or 512     */
    int rays_per_fetch;  /* rays a warp takes per atomic fetch: 32..1024, x32 */
    int emit_warps;      /* warps (32-ray tiles) per CTA of the emit: 2, 4, 8 */
    int use_graph;       /* capture the sequence in a CUDA graph at create    */
    int walk_variant;    /* HDDA_WALK_BRANCH or HDDA_WALK_SKIP: the control
                            flow of Algorithm 1 or of Algorithm 2; both keep
                            the same samples                                  */
} hdda_batch_config;

typedef struct hdda_batch hdda_batch;  /* opaque, library-owned */

/* Builds a batch plan for `n_jobs` jobs (HOST array, 1..4096); cfg (HOST) may
 * be NULL for {256, 64, 4, 1, HDDA_WALK_BRANCH}.  Looks up each job's lattice (synchronising
 * once per new parameter set) and synchronises the stream once.  Scratch: plain device
 * memory for a graph batch, the stream-ordered allocator of `stream` otherwise. */
int hdda_batch_create(const hdda_job* jobs, int n_jobs, const hdda_batch_config* cfg,
                      hdda_batch** out, hdda_stream_t stream);

/* Runs the batch on `stream` (one graph launch, or its kernels); async. */
int hdda_batch_launch(hdda_batch* batch, hdda_stream_t stream);

/* Waits for the stream and reads every job's sample total and status (HOST
 * arrays of n_jobs; either may be NULL).  A job whose capacity is below its
 * total gets HDDA_ERR_CAPACITY (its samples below capacity are written) and
 * the call returns that code too. */
int hdda_batch_results(hdda_batch* batch, int64_t* totals, uint32_t* status,
                       hdda_stream_t stream);

/* Frees a batch.  A batch made with use_graph = 0 returns its scratch to the
 * stream-ordered allocator on the stream it was created on, after the work
 * queued there (no synchronisation; launch such a batch only on that stream
 * or order other streams after it); a graph batch waits for the device and
 * frees plain device memory.  NULL is a no-op. */
void hdda_batch_free(hdda_batch* batch);

/*
 * Front-to-back compositing of the kept intervals over a Gaussian-blob field
 * (Sec. 1: densities and colours of the sampled points are accumulated into
 * the pixel).  For each ray, in order of its samples, with x the position at
 * the interval midpoint:
 *     sigma = sum_g a_g exp(-|x - mu_g|^2 / (2 s_g^2))
 *     c     = sum_g a_g exp(...) rgb_g / sigma      (0 when sigma == 0)
 *     alpha = 1 - exp(-sigma (t1 - t0)) ;  C += T alpha c ;  T *= 1 - alpha
 * and rgba_out[r] = (C, 1 - T): black background, no early termination.
 *   rays_o, rays_d  device float [n_rays][3]
 *   offsets         device int64 [n_rays + 1] (as written by a traversal)
 *   t0, t1          device float samples
 *   field           device float [n_gauss][8] = mu_x, mu_y, mu_z, s, a, r, g, b,
 *                   with s > 0 and a >= 0.  A blob is skipped for a group of
 *                   64 consecutive samples when it lies farther than 7 s from
 *                   every one of them (its weight there is below a * e^-24.5);
 *                   the distance tests keep a small margin for rounding, so
 *                   no blob within 7 s of a sample is skipped
 *   n_gauss         0..256
 *   rgba_out        device float [n_rays][4]
 * Stream-ordered, no synchronisation.
 */
int hdda_composite(const float* rays_o, const float* rays_d, int64_t n_rays,
                   const int64_t* offsets, const float* t0, const float* t1,
                   const float* field, int n_gauss, float* rgba_out, hdda_stream_t stream);

/*
 * Render-only path: samples and composites in one call without writing any
 * sample to memory (the sampler and the field evaluation fused).  Ray r's
 * pixel is the one hdda_composite gives for the intervals that
 * hdda_traverse_hdda (VDB grid) or hdda_traverse_dense (dense grid) keeps
 * for it, up to float summation order (both are within 1e-5 of the same
 * FP64 accumulation).  A VDB grid is walked by HDDA with its refinement and
 * walk-variant settings, a dense grid by dense DDA.
 *   rays_o, rays_d, n_rays, grid, params   as for hdda_traverse_hdda
 *   field, n_gauss, rgba_out               as for hdda_composite
 *   dev_status   NULL: the call synchronises the stream once at the end and
 *                returns HDDA_ERR_INTERNAL if a device-side region check
 *                failed (checks on, see hdda_set_region_checks).  Otherwise a DEVICE uint32 (4-byte aligned) that
 *                receives the device status bits by atomic OR (bit 1 =
 *                region check failed); the call then returns once the work
 *                is enqueued and does not synchronise, except on the first
 *                use of a parameter set (the lattice is computed then).
 * Scratch of about 134 bytes per ray comes from the stream-ordered allocator
 * and is returned in stream order.
 */
int hdda_render(const float* rays_o, const float* rays_d, int64_t n_rays,
                const hdda_grid* grid, const hdda_params* params, const float* field,
                int n_gauss, float* rgba_out, uint32_t* dev_status, hdda_stream_t stream);

/*
 * Sampling and compositing fused: the outputs of hdda_traverse_async and of
 * hdda_render from one stream-ordered call (Algorithm 1's kept intervals,
 * stored, and Sec. 1's accumulation over them).  The walk and the tile scan
 * run as in the samplers; then one kernel expands each ray's runs, writes
 * every sample at its CSR position and composites it, so the samples are
 * written once and never read back.
 *   rays_o, rays_d, n_rays, grid, params   as for hdda_traverse_async
 *   offsets, ray_idx, t0, t1, capacity      as for hdda_traverse_async: the
 *                same values bit for bit (capacity 0 writes the offsets
 *                only, unclamped); a capacity below the total raises bit 2
 *                of *dev_status, writes no sample at or past capacity and
 *                clamps the offsets to capacity
 *   field, n_gauss, rgba_out                as for hdda_render: the same
 *                frame, bit for bit
 *   dev_status   DEVICE uint32 (required, 4-byte aligned), as for
 *                hdda_traverse_async
 * Stream-ordered, no synchronisation except on the first use of a parameter
 * set.  Scratch of about 150 bytes per ray comes from the stream-ordered
 * allocator.
 */
int hdda_traverse_composite(const float* rays_o, const float* rays_d, int64_t n_rays,
                            const hdda_grid* grid, const hdda_params* params, int64_t* offsets,
                            int32_t* ray_idx, float* t0, float* t1, int64_t capacity,
                            const float* field, int n_gauss, float* rgba_out,
                            uint32_t* dev_status, hdda_stream_t stream);

/*
 * Kernel timing and work counters for measurement, off by default; the
 * paper has no counterpart (it reports frame rates only).
 *   HDDA_PROFILE_TIMERS    every kernel the library launches is bracketed
 *                          by two CUDA events recorded on its stream (one
 *                          event pair per launch)
 *   HDDA_PROFILE_COUNTERS  the compositors count blob evaluations (sample x
 *                          kept blob), one atomic add per warp task; this
 *                          is extra device work, so time with the timers
 *                          alone
 * hdda_profiler_enable(flags) sets both switches (0 turns everything off).
 * hdda_profiler_read synchronises on the recorded events, writes up to `cap`
 * per-kernel aggregates (HOST array) and clears them; *n_out (HOST)
 * receives how many entries there were.  Counters appear as entries named
 * "composite_blob_evals" and "render_blob_evals" whose `launches` field
 * holds the count and whose total_ms is 0.
 */
enum { HDDA_PROFILE_TIMERS = 1, HDDA_PROFILE_COUNTERS = 2 };

typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
} hdda_kernel_time;

int hdda_profiler_enable(int flags);
int hdda_profiler_read(hdda_kernel_time* out, int cap, int* n_out);

/*
 * Device-side region checks, off by default (an assertion, as in a debug
 * build): while on, every walk tests that each region it crosses holds the
 * lattice point that was classified to find it (the invariant the exact
 * crossing search of Sec. 3's walk rests on), and a failure raises the internal
 * status bit, so that the calls above return HDDA_ERR_INTERNAL or set bit 1
 * of their device status word.  A correct library never fails the check;
 * it costs about 5 % of the walk, so production runs leave it off.
 * The checks run in the walk pass of hdda_traverse_hdda, hdda_traverse_dense,
 * hdda_traverse_async, hdda_render and the batched sampler; the later
 * passes that re-walk a ray cross the same regions unchecked, and the
 * allocation-free entry point does not check.  The setting is process-wide
 * and is read when work is enqueued: a call (or a batch, at
 * hdda_batch_create) made after the switch sees it.
 * hdda_set_region_checks returns HDDA_OK; hdda_region_checks returns the
 * current setting (0 or 1).
 */
int hdda_set_region_checks(int on);
int hdda_region_checks(void);

/*
 * Form of the two-pass samplers (hdda_traverse_dense, hdda_traverse_hdda,
 * hdda_traverse_async); the samples are the same in both.
 *   HDDA_SAMPLER_SEPARATE (default): the walk (pass 1) and the emit (pass 2)
 *     as two kernels; the walk also keeps sample totals per 32 and per 1024
 *     tiles, from which the emit adds up each tile's output offset (the
 *     prefix sum of Algorithm 1's per-ray sample counts).
 *   HDDA_SAMPLER_FUSED: one persistent kernel; its warps walk 32-ray tiles
 *     until none is left, then write tiles out in order, each tile's offset
 *     from a decoupled look-back over the totals the walks published, so
 *     that warps done walking write out early tiles while the last ones are
 *     still walked.
 *     On full frames it measured no faster than the separate form (the
 *     write-out's memory waits slow the walks that share its SMs).
 * Not in the paper (its sampler is one thread per ray appending to a
 * buffer).  The setting is process-wide and read when a call enqueues its
 * work.  hdda_set_sampler_form returns HDDA_OK, or HDDA_ERR_INVALID_ARG for
 * any other value; hdda_sampler_form returns the current form.
 */
typedef enum { HDDA_SAMPLER_SEPARATE = 0, HDDA_SAMPLER_FUSED = 1 } hdda_sampler_form_t;
int hdda_set_sampler_form(int form);
int hdda_sampler_form(void);

#ifdef __cplusplus
}
#endif

#endif /* HDDA_H */
