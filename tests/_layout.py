"""White-box restatement of the library's refinement-mask layout (not collected
by pytest).

The refinement masks are this library's own acceleration structure (an
octree-style subdivision inside VDB nodes and leaves), not a definition from
the paper, so they live with the tests rather than in the oracle.  The masks
are derived here with numpy from a tree built by ``oracle.build_vdb`` and the
layout documented for HDDA_ARRAY_NODE_SUPER / HDDA_ARRAY_LEAF_SUB in
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


