"""CPU oracle for the batch SHA-3 library -- TEST INFRASTRUCTURE ONLY.

A plain, slow restatement of the paper's Section 3 (Keccak-p, the sponge and
the six SHA-3 functions, Eq. 1-18), read against FIPS 202 where the paper's
equations are garbled.  The arithmetic lives in ``keccak_ref.c`` (bit-level,
one bit per byte); this module only compiles it with gcc and marshals
arguments through ctypes.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never does, and this
package imports nothing from the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = ("keccak_ref.c", "batch.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

#: Digest sizes in bytes of the fixed-output variants; None for the XOFs.
DIGEST_BYTES = (28, 32, 48, 64, None, None)
#: Capacities c in bits (Eq. 13-18).
CAPACITY_BITS = (448, 512, 768, 1024, 256, 512)
OK, ERR_INVALID, ERR_NOMEM = 0, -1, -2


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the sources (plain C11, pthreads)."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    hdr = os.path.join(_HERE, "keccak_ref.h")
    newest = max(os.path.getmtime(p) for p in srcs + [hdr])
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=c11", "-Wall", "-Wextra", "-shared", "-fPIC", "-pthread",
           *srcs, "-o", tmp]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            for name in ("oracle_theta", "oracle_rho", "oracle_pi", "oracle_chi"):
                getattr(L, name).argtypes = [ctypes.c_int, u8p]
                getattr(L, name).restype = None
            L.oracle_iota.argtypes = [ctypes.c_int, ctypes.c_int, u8p]
            L.oracle_iota.restype = None
            L.oracle_rnd.argtypes = [ctypes.c_int, ctypes.c_int, u8p]
            L.oracle_rnd.restype = None
            L.oracle_keccak_p.argtypes = [ctypes.c_int, ctypes.c_int, u8p]
            L.oracle_keccak_p.restype = ctypes.c_int
            L.oracle_rc_bit.argtypes = [ctypes.c_long]
            L.oracle_rc_bit.restype = ctypes.c_int
            L.oracle_round_constant.argtypes = [ctypes.c_int, ctypes.c_int]
            L.oracle_round_constant.restype = ctypes.c_uint64
            L.oracle_rho_offset.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.oracle_rho_offset.restype = ctypes.c_int
            L.oracle_keccak_c.argtypes = [ctypes.c_int, u8p, ctypes.c_size_t, ctypes.c_size_t, u8p]
            L.oracle_keccak_c.restype = ctypes.c_int
            L.oracle_hash.argtypes = [ctypes.c_int, u8p, ctypes.c_size_t, u8p, ctypes.c_size_t]
            L.oracle_hash.restype = ctypes.c_int
            L.oracle_inc_size.argtypes = []
            L.oracle_inc_size.restype = ctypes.c_size_t
            L.oracle_inc_init.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.oracle_inc_init.restype = ctypes.c_int
            L.oracle_inc_absorb.argtypes = [ctypes.c_void_p, u8p, ctypes.c_size_t]
            L.oracle_inc_absorb.restype = ctypes.c_int
            L.oracle_inc_final.argtypes = [ctypes.c_void_p, u8p, ctypes.c_size_t]
            L.oracle_inc_final.restype = ctypes.c_int
            L.oracle_merkle_node_count.argtypes = [ctypes.c_uint64]
            L.oracle_merkle_node_count.restype = ctypes.c_uint64
            L.oracle_merkle_levels.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64, u8p]
            L.oracle_merkle_levels.restype = ctypes.c_int
            L.oracle_merkle_sha3_256.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64, u8p]
            L.oracle_merkle_sha3_256.restype = ctypes.c_int
            L.oracle_merkle_message.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64, u8p]
            L.oracle_merkle_message.restype = ctypes.c_int
            L.oracle_hash_batch.argtypes = [u8p, u64p, u64p, u8p, u32p, u8p, ctypes.c_uint64,
                                            ctypes.c_int]
            L.oracle_hash_batch.restype = ctypes.c_int
            L.oracle_count_images_b25.argtypes = [ctypes.c_int, ctypes.c_int]
            L.oracle_count_images_b25.restype = ctypes.c_int64
            _lib = L
    return _lib


def _p(arr: np.ndarray, ctype=ctypes.c_uint8):
    return arr.ctypes.data_as(ctypes.POINTER(ctype))


def _bytes_arr(data) -> np.ndarray:
    if isinstance(data, np.ndarray):
        return np.ascontiguousarray(data, dtype=np.uint8).reshape(-1)
    return np.frombuffer(bytes(data), dtype=np.uint8).copy()


def _bits(S) -> np.ndarray:
    a = np.ascontiguousarray(S, dtype=np.uint8).reshape(-1).copy()
    if a.size == 0 or a.max(initial=0) > 1:
        raise ValueError("a state is a string of bits with values 0/1")
    return a


# -- step mappings and the permutation (bit strings, Eq. 1 order) -----------
def step(name: str, w: int, S, ir: int = 0) -> np.ndarray:
    """Applies one step mapping ('theta', 'rho', 'pi', 'chi', 'iota', 'rnd')."""
    a = _bits(S)
    if a.size != 25 * w:
        raise ValueError("state size must be 25*w")
    fn = getattr(lib(), "oracle_" + name)
    if name in ("iota", "rnd"):
        fn(w, ir, _p(a))
    else:
        fn(w, _p(a))
    return a


def keccak_p(b: int, nr: int, S) -> np.ndarray:
    a = _bits(S)
    if a.size != b:
        raise ValueError("state size must be b")
    if lib().oracle_keccak_p(b, nr, _p(a)) != OK:
        raise ValueError("invalid width or round count")
    return a


def rc_bit(t: int) -> int:
    return int(lib().oracle_rc_bit(t))


def round_constant(l: int, ir: int) -> int:
    return int(lib().oracle_round_constant(l, ir))


def rho_offset(w: int, x: int, y: int) -> int:
    return int(lib().oracle_rho_offset(w, x, y))


def keccak_c(c: int, N_bits, d_bits: int) -> np.ndarray:
    n = np.ascontiguousarray(N_bits, dtype=np.uint8).reshape(-1).copy()
    z = np.zeros(max(d_bits, 1), dtype=np.uint8)
    if lib().oracle_keccak_c(c, _p(n), n.size, d_bits, _p(z)) != OK:
        raise ValueError("invalid capacity")
    return z[:d_bits]


# -- byte-level functions --------------------------------------------------
def hash(variant: int, msg, out_len: int | None = None) -> bytes:  # noqa: A001
    """SHA3-224/256/384/512 (variants 0-3) or SHAKE128/256 (4, 5) of msg."""
    if out_len is None:
        out_len = DIGEST_BYTES[variant]
        if out_len is None:
            raise ValueError("SHAKE needs out_len")
    m = _bytes_arr(msg)
    out = np.zeros(max(out_len, 1), dtype=np.uint8)
    rc = lib().oracle_hash(variant, _p(m), m.size, _p(out), out_len)
    if rc != OK:
        raise ValueError(f"oracle_hash failed with {rc}")
    return out[:out_len].tobytes()


class Incremental:
    """init / absorb(piece) ... / final(out_len), same result as hash()."""

    def __init__(self, variant: int):
        self._buf = ctypes.create_string_buffer(lib().oracle_inc_size())
        if lib().oracle_inc_init(self._buf, variant) != OK:
            raise ValueError("invalid variant")

    def absorb(self, piece) -> None:
        m = _bytes_arr(piece)
        if lib().oracle_inc_absorb(self._buf, _p(m), m.size) != OK:
            raise ValueError("absorb failed")

    def final(self, out_len: int) -> bytes:
        out = np.zeros(max(out_len, 1), dtype=np.uint8)
        if lib().oracle_inc_final(self._buf, _p(out), out_len) != OK:
            raise ValueError("final failed")
        return out[:out_len].tobytes()


def merkle_node_count(n_leaves: int) -> int:
    return int(lib().oracle_merkle_node_count(n_leaves))


def merkle_levels(buf, n_leaves: int, leaf_bytes: int) -> np.ndarray:
    """All nodes, level by level (leaves first), as an (n_nodes, 32) array."""
    b = _bytes_arr(buf)
    if b.size < n_leaves * leaf_bytes:
        raise ValueError("buffer too small")
    total = merkle_node_count(n_leaves)
    nodes = np.zeros((max(total, 1), 32), dtype=np.uint8)
    if lib().oracle_merkle_levels(_p(b), n_leaves, leaf_bytes, _p(nodes)) != OK:
        raise ValueError("invalid tree")
    return nodes[:total]


def merkle_root(buf, n_leaves: int, leaf_bytes: int) -> bytes:
    b = _bytes_arr(buf)
    if b.size < n_leaves * leaf_bytes:
        raise ValueError("buffer too small")
    root = np.zeros(32, dtype=np.uint8)
    if lib().oracle_merkle_sha3_256(_p(b), n_leaves, leaf_bytes, _p(root)) != OK:
        raise ValueError("invalid tree")
    return root.tobytes()


def merkle_message_root(msg, chunk_bytes: int) -> bytes:
    """Root of the tree over one message cut into chunk_bytes chunks."""
    m = _bytes_arr(msg)
    root = np.zeros(32, dtype=np.uint8)
    src = m if m.size else np.zeros(1, np.uint8)
    if lib().oracle_merkle_message(_p(src), m.size, chunk_bytes, _p(root)) != OK:
        raise ValueError("invalid chunk size")
    return root.tobytes()


def hash_batch(msgs, offsets, lens, variants, out_lens, nthreads: int | None = None) -> np.ndarray:
    """Hashes a CSR batch on host threads; returns the concatenated outputs."""
    m = _bytes_arr(msgs)
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    ln = np.ascontiguousarray(lens, dtype=np.uint64)
    var = np.ascontiguousarray(variants, dtype=np.uint8)
    ol = np.ascontiguousarray(out_lens, dtype=np.uint32)
    n = off.size
    if not (ln.size == var.size == ol.size == n):
        raise ValueError("offsets, lens, variants and out_lens must have one entry per message")
    if n and int((off + ln).max()) > m.size:
        raise ValueError("a message runs past the end of msgs")
    out = np.zeros(max(int(ol.sum(dtype=np.uint64)), 1), dtype=np.uint8)
    threads = nthreads or len(os.sched_getaffinity(0))
    rc = lib().oracle_hash_batch(_p(m if m.size else np.zeros(1, np.uint8)), _p(off, ctypes.c_uint64),
                                 _p(ln, ctypes.c_uint64), _p(var), _p(ol, ctypes.c_uint32),
                                 _p(out), n, threads)
    if rc != OK:
        raise ValueError(f"oracle_hash_batch failed with {rc}")
    return out[: int(ol.sum(dtype=np.uint64))]


def count_images_b25(nr: int, nthreads: int | None = None) -> int:
    return int(lib().oracle_count_images_b25(nr, nthreads or len(os.sched_getaffinity(0))))
