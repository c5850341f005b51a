"""White-box restatement of the library's refinement-mask and region-map
layouts (not collected by pytest).

The refinement masks and the region map are this library's own acceleration
structures (an octree-style subdivision inside VDB nodes and leaves, and its
flattening into one entry per 2^3 cell), not definitions from the paper, so
they live with the tests rather than in the oracle.  The masks are derived
here with numpy from a tree built by ``oracle.build_vdb``, the map directly
from the dense occupancy, both in the layouts documented for
HDDA_ARRAY_NODE_SUPER / HDDA_ARRAY_LEAF_SUB / HDDA_ARRAY_REGION_MAP in
include/hdda.h, and compared word for word with what the library exports.
"""
import numpy as np


def vdb_refinement(v: dict) -> tuple[np.ndarray, np.ndarray]:
    """Refinement masks of a tree from build_vdb, in the library's layout.

    Per node, 18 uint32 words: 64 bits for its 4^3 groups of 32^3 voxels
    (group (gx*4 + gy)*4 + gz), then 512 bits for its 8^3 groups of 16^3
    voxels ((gx*8 + gy)*8 + gz); a bit is set when the group holds a child
    or a tile.  Per leaf, 5 words: 64 bits for its 4^3 cells of 2^3 voxels
    ((cx*4 + cy)*4 + cz), then 8 bits for its 2^3 cells of 4^3 voxels, a bit
    set when the cell holds an occupied voxel; then 64 bits for the 2^3-voxel
    cells again, a bit set when all 8 voxels of the cell are occupied.
    """
    L, N = v["levels"], v["nodes"]
    occ = (np.unpackbits(v["child"].view(np.uint8), bitorder="little")
           | np.unpackbits(v["tile"].view(np.uint8), bitorder="little")).reshape(L, N ** 3, 16, 16, 16)
    g16 = occ.reshape(L, N ** 3, 8, 2, 8, 2, 8, 2).any(axis=(3, 5, 7))
    g32 = g16.reshape(L, N ** 3, 4, 2, 4, 2, 4, 2).any(axis=(3, 5, 7))
    pack = lambda b: np.packbits(b.reshape(L, N ** 3, -1), axis=-1, bitorder="little").view("<u4")
    nsuper = np.concatenate([pack(g32), pack(g16)], axis=-1)
    leaves = v["leaves"]
    lsub = np.zeros((leaves.shape[0], 5), np.uint32)
    if leaves.shape[0]:
        bits = np.unpackbits(leaves.view(np.uint8), bitorder="little").reshape(-1, 8, 8, 8)
        c2 = bits.reshape(-1, 4, 2, 4, 2, 4, 2).any(axis=(2, 4, 6))
        c4 = c2.reshape(-1, 2, 2, 2, 2, 2, 2).any(axis=(2, 4, 6))
        f2 = bits.reshape(-1, 4, 2, 4, 2, 4, 2).all(axis=(2, 4, 6))
        lsub[:, 0:2] = np.packbits(c2.reshape(-1, 64), axis=-1, bitorder="little").view("<u4")
        lsub[:, 2] = np.packbits(c4.reshape(-1, 8), axis=-1, bitorder="little")[:, 0]
        lsub[:, 3:5] = np.packbits(f2.reshape(-1, 64), axis=-1, bitorder="little").view("<u4")
    return nsuper.astype(np.uint32), lsub




def region_map(occ: np.ndarray) -> np.ndarray:
    """Region map of an occupancy grid uint8 [L, R, R, R], in the library's layout:
    uint16 [L, C, C, C] with C = ceil(R / 2).  For each 2^3 cell, the high byte is log2 of
    the edge of the first uniform region in the order 128^3 node (empty or full), 32^3
    group (empty), 16^3 group (empty), 8^3 block (empty or full), 4^3 cell (empty or
    full), 2^3 cell (empty or full) -- aligned cubes of the grid padded with empty voxels -- and 0
    when none is; the low byte holds the cell's voxels, bit ((x%2)*2 + y%2)*2 + z%2."""
    L, R = occ.shape[0], occ.shape[1]
    P = -(-R // 128) * 128
    pad = np.zeros((L, P, P, P), bool)
    pad[:, :R, :R, :R] = occ != 0
    C = (R + 1) // 2

    def cubes(s, fn):
        n = P // s
        return fn(pad.reshape(L, n, s, n, s, n, s), axis=(2, 4, 6))

    def per_cell(a, s):
        # value of the size-s cube holding each 2^3 cell, for the first C cells per axis
        r = s // 2
        return a.repeat(r, 1).repeat(r, 2).repeat(r, 3)[:, :C, :C, :C]

    cells = pad.reshape(L, P // 2, 2, P // 2, 2, P // 2, 2).transpose(0, 1, 3, 5, 2, 4, 6)
    cells = cells.reshape(L, P // 2, P // 2, P // 2, 8)[:, :C, :C, :C]
    bits = (cells.astype(np.uint16) << np.arange(8, dtype=np.uint16)).sum(-1).astype(np.uint16)
    out = np.zeros((L, C, C, C), np.uint16)
    done = np.zeros((L, C, C, C), bool)

    def take(mask, lg, full):
        nonlocal done
        m = mask & ~done
        out[m] = (lg << 8) | (0xFF if full else 0)
        done |= m

    for s, lg, kinds in ((128, 7, (False, True)), (32, 5, (False,)), (16, 4, (False,)),
                         (8, 3, (False, True)), (4, 2, (False, True)), (2, 1, (False, True))):
        empty = per_cell(~cubes(s, np.any), s)
        full = per_cell(cubes(s, np.all), s)
        for f in kinds:
            take(full if f else empty, lg, f)
    out[~done] = bits[~done]
    return out
