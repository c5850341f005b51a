"""The refinement-mask and region-map restatements in tests/_layout.py, checked on
hand-worked grids before the GPU parity tests compare the library's exported arrays
with them."""
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


def test_region_map_hand_worked():
    # one occupied voxel (5, 9, 40) of a 64^3 grid (padded to one 128^3 node):
    # its 2^3 cell (2, 4, 20) is mixed and holds bit ((5%2)*2 + 9%2)*2 + 40%2 = 6;
    # the other cells of its 4^3 cell are empty 2^3 cells; the rest of its 8^3 block
    # (0..7, 8..15, 40..47) lies in empty 4^3 cells; blocks of its 16^3 group are empty
    # 8^3 blocks; the rest of its 32^3 group (0..31, 0..31, 32..63) is empty 16^3
    # groups; everything else is an empty 32^3 group
    occ = np.zeros((1, 64, 64, 64), np.uint8)
    occ[0, 5, 9, 40] = 1
    m = _layout.region_map(occ)
    assert m.shape == (1, 32, 32, 32) and m.dtype == np.uint16
    assert m[0, 2, 4, 20] == 1 << 6
    assert m[0, 2, 4, 21] == 1 << 8 and m[0, 3, 5, 21] == 1 << 8
    assert m[0, 0, 4, 20] == 2 << 8 and m[0, 3, 7, 23] == 2 << 8
    assert m[0, 4, 4, 20] == 3 << 8 and m[0, 7, 7, 23] == 3 << 8
    assert m[0, 8, 4, 20] == 4 << 8 and m[0, 15, 15, 31] == 4 << 8
    assert m[0, 0, 0, 0] == 5 << 8 and m[0, 31, 31, 31] == 5 << 8
    counts = np.unique(m >> 8, return_counts=True)
    assert dict(zip(counts[0].tolist(), counts[1].tolist())) == {
        0: 1, 1: 8 - 1, 2: 64 - 8, 3: 512 - 64, 4: 4096 - 512, 5: 32768 - 4096}
    # a full 2^3 cell next to it: full (0xff) at size 2; a full 8^3 block: a tile
    occ[0, 0:2, 0:2, 0:2] = 1
    occ[0, 16:24, 16:24, 16:24] = 1
    m = _layout.region_map(occ)
    assert m[0, 0, 0, 0] == (1 << 8) | 0xFF and m[0, 0, 0, 1] == 1 << 8
    assert m[0, 8, 8, 8] == (3 << 8) | 0xFF and m[0, 11, 11, 11] == (3 << 8) | 0xFF
    # every voxel occupied on a 128^3 grid: one full node; none: one empty node
    assert (_layout.region_map(np.ones((1, 128, 128, 128), np.uint8)) == (7 << 8) | 0xFF).all()
    assert (_layout.region_map(np.zeros((2, 128, 128, 128), np.uint8)) == 7 << 8).all()
    # a full 64^3 grid is padded with empty voxels: never a full node, full 8^3 tiles
    assert (_layout.region_map(np.ones((1, 64, 64, 64), np.uint8)) == (3 << 8) | 0xFF).all()


def test_region_map_odd_resolution():
    # R = 5: C = 3 cells per axis; the last cell per axis holds voxel 4 and padding
    occ = np.zeros((1, 5, 5, 5), np.uint8)
    occ[0, 4, 4, 4] = 1
    m = _layout.region_map(occ)
    assert m.shape == (1, 3, 3, 3)
    assert m[0, 2, 2, 2] == 1 << 0           # voxel (4,4,4): bit ((0*2)+0)*2+0 = 0
    assert m[0, 0, 0, 0] == 2 << 8           # empty 4^3 cell (0..3)^3
    assert m[0, 2, 2, 1] == 2 << 8           # voxels (4..5, 4..5, 2..3): empty 4^3 cell
    assert (np.sort(m.reshape(-1))[1:] == 2 << 8).all()  # the other 26 cells likewise
