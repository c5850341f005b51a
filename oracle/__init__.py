"""CPU oracle for the occupancy-grid ray sampler -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never touches it, and it never touches them: the two
share no code.  Inputs for both sides come from seeded generators; the
oracle only ever receives plain numpy arrays.

Contents
--------
``lattice``   the binary32 step recurrence of one ray (Algorithm 1; Sec. 3).
``sample``    brute-force sampling over every lattice candidate, keeping an
              interval when the voxel holding its midpoint is occupied at the
              finest level that contains it (Algorithm 1; Sec. 3).
``composite`` binary64 front-to-back accumulation over a Gaussian-blob field
              (Sec. 1: densities and colours of the samples are accumulated
              into the pixel).
``pack_dense_bits``  the dense bit array, the paper's baseline representation
              (Table 3 caption: 256 KiB for one 128^3 grid).
``build_vdb`` the sparse tree the library builds from the dense bits: 8^3
              leaf bitmasks under 16^3 node child masks, with fully occupied
              8^3 blocks pruned into tiles (Sec. 3: redundant blocks become
              tiles that hold one value for many voxels).

The first three live in ``hdda_oracle.c`` (plain C, compiled with
``-O2 -ffp-contract=off -fno-fast-math``); the last two are numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hdda_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]

OK, ERR_INVALID_ARG, ERR_CAPACITY, ERR_STEP_LIMIT = 0, 1, 3, 4
_ERRORS = {
    ERR_INVALID_ARG: "invalid argument",
    ERR_CAPACITY: "output capacity below the number of samples",
    ERR_STEP_LIMIT: "more lattice candidates than max_steps",
}

_lock = threading.Lock()
_lib = None


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle status {code}: {_ERRORS.get(code, 'unknown')}")
        self.code = code


def build(force: bool = False) -> str:
    """Compiles the C oracle into oracle/_build/liboracle.so (gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_SO)) or os.path.getmtime(_SO) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.run(["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # ORACLE_SO_OVERRIDE lets the mutation test load a deliberately broken copy
        path = os.environ.get("ORACLE_SO_OVERRIDE") or build()
        lib = ctypes.CDLL(path)
        f32, i64, i32, p = ctypes.c_float, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        lib.oracle_lattice.argtypes = [f32, f32, f32, f32, f32, i64, p, i64, p]
        lib.oracle_lattice.restype = i32
        lib.oracle_sample.argtypes = [p, p, i64, p, i32, i32, p, f32, f32, f32, f32, f32, i64,
                                      p, p, p, p, i64, p]
        lib.oracle_sample.restype = i32
        lib.oracle_composite.argtypes = [p, p, i64, p, p, p, p, i32, p]
        lib.oracle_composite.restype = i32
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(code: int):
    if code != OK:
        raise OracleError(code)


def lattice(near: float, far: float, step: float, cone: float = 0.0,
            max_step: float = 1e10, max_steps: int = 1 << 22) -> np.ndarray:
    """t_0 .. t_K of the step recurrence, as float32 (K candidates)."""
    lib = _load()
    n = ctypes.c_int64(0)
    _check(lib.oracle_lattice(near, far, step, cone, max_step, max_steps, None, 0,
                              ctypes.byref(n)))
    out = np.empty(n.value + 1, np.float32)
    _check(lib.oracle_lattice(near, far, step, cone, max_step, max_steps, _ptr(out),
                              out.size, ctypes.byref(n)))
    return out


def _aabbs(aabbs, levels):
    a = np.ascontiguousarray(np.asarray(aabbs, np.float32).reshape(levels, 6))
    return a


def sample(rays_o, rays_d, occ, aabbs, near, far, step, cone=0.0, max_step=1e10,
           max_steps=1 << 22, count_only=False):
    """Brute-force sampler.

    rays_o, rays_d: float32 [n, 3]; occ: uint8 [L, R, R, R] (C order, x
    slowest); aabbs: [L, 6] = (lo_x, lo_y, lo_z, hi_x, hi_y, hi_z), level 0
    finest.  Returns (offsets int64 [n+1], ray_idx int32 [S], t0 float32 [S],
    t1 float32 [S]); with count_only only offsets are filled.
    """
    lib = _load()
    o = np.ascontiguousarray(rays_o, np.float32).reshape(-1, 3)
    d = np.ascontiguousarray(rays_d, np.float32).reshape(-1, 3)
    assert o.shape == d.shape
    occ = np.ascontiguousarray(occ, np.uint8)
    if occ.ndim == 3:
        occ = occ[None]
    L, R = occ.shape[0], occ.shape[1]
    assert occ.shape == (L, R, R, R)
    box = _aabbs(aabbs, L)
    n = o.shape[0]
    offsets = np.zeros(n + 1, np.int64)
    total = ctypes.c_int64(0)
    args = (_ptr(o), _ptr(d), n, _ptr(occ), L, R, _ptr(box), near, far, step, cone,
            max_step, max_steps, _ptr(offsets))
    _check(lib.oracle_sample(*args, None, None, None, 0, ctypes.byref(total)))
    S = total.value
    ray_idx = np.empty(S, np.int32)
    t0 = np.empty(S, np.float32)
    t1 = np.empty(S, np.float32)
    if not count_only and S > 0:
        _check(lib.oracle_sample(*args, _ptr(ray_idx), _ptr(t0), _ptr(t1), S,
                                 ctypes.byref(total)))
    return offsets, ray_idx, t0, t1


def composite(rays_o, rays_d, offsets, t0, t1, field) -> np.ndarray:
    """Binary64 front-to-back compositing; returns float64 [n, 4] RGBA."""
    lib = _load()
    o = np.ascontiguousarray(rays_o, np.float32).reshape(-1, 3)
    d = np.ascontiguousarray(rays_d, np.float32).reshape(-1, 3)
    off = np.ascontiguousarray(offsets, np.int64)
    a0 = np.ascontiguousarray(t0, np.float32)
    a1 = np.ascontiguousarray(t1, np.float32)
    fld = np.ascontiguousarray(field, np.float32).reshape(-1, 8)
    n = o.shape[0]
    assert off.shape == (n + 1,)
    out = np.zeros((n, 4), np.float64)
    _check(lib.oracle_composite(_ptr(o), _ptr(d), n, _ptr(off), _ptr(a0), _ptr(a1),
                                _ptr(fld), fld.shape[0], _ptr(out)))
    return out


# ---------------------------------------------------------------------------
# Grid structures (numpy).  The layouts are the library's documented ones;
# they are restated here from that statement, not shared with the library.
# ---------------------------------------------------------------------------

def dense_words_per_level(R: int) -> int:
    return (R * R * R + 31) // 32


def pack_dense_bits(occ) -> np.ndarray:
    """Dense bit array: voxel (l, x, y, z) is bit ((x*R + y)*R + z) of level
    l's bit string, stored as little-endian uint32 words (bit b of word w is
    voxel 32*w + b).  Returns uint32 [L, ceil(R^3/32)]."""
    occ = np.asarray(occ)
    if occ.ndim == 3:
        occ = occ[None]
    L, R = occ.shape[0], occ.shape[1]
    W = dense_words_per_level(R)
    out = np.zeros((L, W), np.uint32)
    for l in range(L):
        bits = np.zeros(W * 32, np.uint8)
        bits[: R ** 3] = (occ[l].reshape(-1) != 0)
        out[l] = np.packbits(bits, bitorder="little").view("<u4")
    return out


def build_vdb(occ) -> dict:
    """Sparse tree of one grid stack, level by level.

    Blocks are 8^3 voxels, B = ceil(R/8) per axis, voxels beyond R empty.
    Nodes are 16^3 blocks, N = ceil(B/16) per axis.  Block (bx, by, bz) is
    cell ((bx%16)*16 + by%16)*16 + bz%16 of node (bx//16, by//16, bz//16),
    nodes numbered (nx*N + ny)*N + nz.  Per node: child mask and tile mask of
    4096 bits as 128 little-endian uint32 words.  A block is a tile when all
    512 of its voxels exist and are occupied, a child (leaf) when some but not
    all are occupied.  Leaves are stored in order of (level, node, cell); each
    is 512 bits (16 uint32 words), voxel (x%8, y%8, z%8) at bit
    ((x%8)*8 + y%8)*8 + z%8.
    """
    occ = np.asarray(occ)
    if occ.ndim == 3:
        occ = occ[None]
    L, R = occ.shape[0], occ.shape[1]
    B = (R + 7) // 8
    N = (B + 15) // 16
    child = np.zeros((L, N ** 3, 4096), bool)
    tile = np.zeros((L, N ** 3, 4096), bool)
    leaves = []
    n_tiles = 0
    for l in range(L):
        g = np.zeros((B * 8,) * 3, np.uint8)
        g[:R, :R, :R] = occ[l] != 0
        blk = g.reshape(B, 8, B, 8, B, 8).transpose(0, 2, 4, 1, 3, 5)  # [bx,by,bz,x,y,z]
        cnt = blk.reshape(B, B, B, 512).sum(-1)
        for nx in range(N):
            for ny in range(N):
                for nz in range(N):
                    node = (nx * N + ny) * N + nz
                    for cx in range(16):
                        bx = nx * 16 + cx
                        if bx >= B:
                            continue
                        for cy in range(16):
                            by = ny * 16 + cy
                            if by >= B:
                                continue
                            for cz in range(16):
                                bz = nz * 16 + cz
                                if bz >= B:
                                    continue
                                cell = (cx * 16 + cy) * 16 + cz
                                c = cnt[bx, by, bz]
                                if c == 512:
                                    tile[l, node, cell] = True
                                    n_tiles += 1
                                elif c > 0:
                                    child[l, node, cell] = True
                                    bits = blk[bx, by, bz].reshape(512)
                                    leaves.append(np.packbits(bits, bitorder="little").view("<u4"))
    pack = lambda m: np.packbits(m.reshape(-1, 4096), axis=-1, bitorder="little").view("<u4").reshape(L, N ** 3, 128)
    leaf_arr = np.stack(leaves) if leaves else np.zeros((0, 16), np.uint32)
    return {
        "levels": L, "res": R, "blocks": B, "nodes": N,
        "child": pack(child), "tile": pack(tile),
        "leaves": leaf_arr.astype(np.uint32), "n_leaves": len(leaves), "n_tiles": n_tiles,
    }


def densify_vdb(v: dict) -> np.ndarray:
    """Inverse of build_vdb: the uint8 [L, R, R, R] grid the tree encodes."""
    L, R, B, N = v["levels"], v["res"], v["blocks"], v["nodes"]
    out = np.zeros((L, B * 8, B * 8, B * 8), np.uint8)
    child = np.unpackbits(v["child"].view(np.uint8), bitorder="little").reshape(L, N ** 3, 4096)
    tile = np.unpackbits(v["tile"].view(np.uint8), bitorder="little").reshape(L, N ** 3, 4096)
    leaf = 0
    for l in range(L):
        for node in range(N ** 3):
            nx, ny, nz = node // (N * N), (node // N) % N, node % N
            for cell in range(4096):
                bx = nx * 16 + cell // 256
                by = ny * 16 + (cell // 16) % 16
                bz = nz * 16 + cell % 16
                sl = (l, slice(bx * 8, bx * 8 + 8), slice(by * 8, by * 8 + 8), slice(bz * 8, bz * 8 + 8))
                if tile[l, node, cell]:
                    out[sl] = 1
                elif child[l, node, cell]:
                    bits = np.unpackbits(v["leaves"][leaf].view(np.uint8), bitorder="little")
                    out[sl] = bits.reshape(8, 8, 8)
                    leaf += 1
    return out[:, :R, :R, :R]
