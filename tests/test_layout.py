"""The refinement-mask restatement in tests/_layout.py, checked on a hand-worked
grid before the GPU parity test compares the library's exported masks with it."""
import numpy as np

import _layout
import oracle


def test_vdb_refinement_masks_single_voxel():
    # voxel (5, 9, 40) of a 64^3 grid: 32^3 group (0, 0, 1) -> bit 1 of word 0; 16^3 group
    # (0, 0, 2) -> bit 2 of word 2; in its leaf, local (5, 1, 0): 2^3 cell (2, 0, 0) -> bit 32,
    # i.e. bit 0 of word 1; 4^3 cell (1, 0, 0) -> bit 4 of word 2
    occ = np.zeros((1, 64, 64, 64), np.uint8)
    occ[0, 5, 9, 40] = 1
    v = oracle.build_vdb(occ)
    ns, ls = _layout.vdb_refinement(v)
    assert ns.shape == (1, 1, 18)
    assert ns[0, 0, 0] == 1 << 1 and ns[0, 0, 1] == 0
    assert ns[0, 0, 2] == 1 << 2 and not ns[0, 0, 3:].any()
    assert ls.tolist() == [[0, 1, 1 << 4, 0, 0]]
    # the whole 2^3 cell (4..5, 8..9, 40..41) occupied: the same cell is also full,
    # bit 32 of the full-cell words (bit 0 of word 4)
    occ[0, 4:6, 8:10, 40:42] = 1
    _, ls = _layout.vdb_refinement(oracle.build_vdb(occ))
    assert ls.tolist() == [[0, 1, 1 << 4, 0, 1]]
    # one voxel less: occupied but no longer full
    occ[0, 4, 8, 40] = 0
    _, ls = _layout.vdb_refinement(oracle.build_vdb(occ))
    assert ls.tolist() == [[0, 1, 1 << 4, 0, 0]]
