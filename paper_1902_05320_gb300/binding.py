"""ctypes binding of ``libsha3gb.so`` (the C ABI of ``include/sha3gb.h``).

Argument marshalling only: every step of the hashing path runs in the CUDA
library.  Device buffers are passed as torch CUDA tensors (or raw integer
addresses), host buffers as numpy arrays or torch CPU tensors; ``stream``
defaults to torch's current stream.  There is no CPU fallback: if the library
has not been built, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsha3gb.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "sha3gb.h")

KB_SHA3_224, KB_SHA3_256, KB_SHA3_384, KB_SHA3_512, KB_SHAKE128, KB_SHAKE256 = 0, 1, 2, 3, 4, 5
KB_OK, KB_ERR_INVALID, KB_ERR_NOMEM, KB_ERR_CUDA, KB_ERR_TIMEOUT, KB_ERR_TOO_LARGE = 0, -1, -2, -3, -4, -5
KB_NOALLOC_MAX_MESSAGES = 65536
KB_NOALLOC_SCRATCH_BYTES = 833152
KB_DEV_BAD_VARIANT, KB_DEV_BAD_OUTLEN, KB_DEV_TIMEOUT = 0x1, 0x2, 0x4
DIGEST_BYTES = (28, 32, 48, 64, None, None)
RATE_BYTES = (144, 136, 104, 72, 168, 136)
NAMES = ("SHA3-224", "SHA3-256", "SHA3-384", "SHA3-512", "SHAKE128", "SHAKE256")

_lock = threading.Lock()
_lib = None


class Sha3gbError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what} failed with status {status}")
        self.status = status


def declared_functions() -> list[str]:
    """Names of the functions declared in include/sha3gb.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("defined",)))


_SIGS = {
    "keccak_batch_uniform": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                            ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]),
    "keccak_batch": (ctypes.c_int, [ctypes.c_void_p] * 6 + [ctypes.c_uint64, ctypes.c_void_p]),
    "keccak_batch_autotune": (ctypes.c_int, [ctypes.c_void_p] * 6 + [ctypes.c_uint64, ctypes.c_void_p,
                                                                      ctypes.c_void_p, ctypes.c_void_p,
                                                                      ctypes.c_void_p]),
    "keccak_batch_noalloc": (ctypes.c_int, [ctypes.c_void_p] * 6 + [ctypes.c_uint64, ctypes.c_void_p]),
    "keccak_tuned_config": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]),
    "keccak_batch_autotune_ex": (ctypes.c_int, [ctypes.c_void_p] * 6 + [ctypes.c_uint64, ctypes.c_void_p,
                                                                         ctypes.c_void_p]),
    "keccak_tuned_config_ex": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_void_p]),
    "keccak_batch_uniform_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                                 ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint64,
                                                 ctypes.c_void_p]),
    "keccak_host_path_for": (ctypes.c_int, [ctypes.c_uint64]),
    "keccak_host_alloc": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_void_p]),
    "keccak_host_free": (ctypes.c_int, [ctypes.c_void_p]),
    "keccak_host_numa_node": (ctypes.c_int, [ctypes.c_void_p]),
    "keccak_stream_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]),
    "keccak_stream_absorb": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_uint64, ctypes.c_void_p]),
    "keccak_stream_final": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_uint64, ctypes.c_void_p]),
    "keccak_stream_init_absorb": (ctypes.c_int, [ctypes.c_void_p] * 5 + [ctypes.c_uint64, ctypes.c_void_p]),
    "keccak_stream_absorb_final": (ctypes.c_int, [ctypes.c_void_p] * 6 + [ctypes.c_uint64, ctypes.c_void_p]),
    "merkle_sha3_256": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "merkle_sha3_256_many": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                            ctypes.c_void_p, ctypes.c_void_p]),
    "merkle_sha3_256_message": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                                               ctypes.c_void_p]),
    "merkle_node_count": (ctypes.c_uint64, [ctypes.c_uint64]),
    "merkle_sha3_256_levels": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                                              ctypes.c_void_p]),
    "keccak_p_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                      ctypes.c_void_p]),
    "keccak_last_error": (ctypes.c_int, [ctypes.c_void_p]),
    "keccak_release": (None, []),
    "sha3gb_round_constants": (ctypes.c_int, [ctypes.c_void_p]),
    "sha3gb_rho_offsets": (ctypes.c_int, [ctypes.c_void_p]),
    "sha3gb_version": (ctypes.c_char_p, []),
    "keccak_tune_set": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64]),
    "keccak_tune_get": (ctypes.c_int64, [ctypes.c_int]),
    "sha3gb_int_issue_probe": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]),
    "sha3gb_wait_timeout_probe": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]),
    "sha3gb_host_link_probe": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
}


def load() -> ctypes.CDLL:
    """Loads the library (built by ``paper_1902_05320_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with `python -m paper_1902_05320_gb300.build` "
                    "(there is no CPU fallback)")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x).__name__}")


def _stream(stream) -> int | None:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(status: int, what: str) -> int:
    if status < 0:
        raise Sha3gbError(status, what)
    return status


def keccak_batch_uniform(msgs, stride: int, length: int, variant: int, out_len: int, digests, n: int,
                         stream=None) -> None:
    _check(load().keccak_batch_uniform(_ptr(msgs), stride, length, variant, out_len, _ptr(digests), n,
                                       _stream(stream)), "keccak_batch_uniform")


def keccak_batch(msgs, offsets, lens, variants, out_lens, digests, n: int, stream=None) -> None:
    _check(load().keccak_batch(_ptr(msgs), _ptr(offsets), _ptr(lens), _ptr(variants), _ptr(out_lens),
                               _ptr(digests), n, _stream(stream)), "keccak_batch")


class QueueConfig(ctypes.Structure):
    """kb_queue_config of sha3gb.h."""
    _fields_ = [("min_blocks", ctypes.c_int64), ("blocks_per_sm", ctypes.c_int64), ("staging", ctypes.c_int64),
                ("warp_messages", ctypes.c_int64), ("ms", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {"min_blocks": self.min_blocks, "blocks_per_sm": self.blocks_per_sm,
                "staging": QUEUE_STAGING_NAMES.get(self.staging, self.staging),
                "threads_per_message": "1" if self.warp_messages == 0 else
                f"32 for the {self.warp_messages} costliest, 1 for the rest",
                "warp_messages": self.warp_messages, "ms": self.ms}


def keccak_batch_autotune(msgs, offsets, lens, variants, out_lens, digests, n: int, stream=None) -> dict:
    """Runs the ragged-schedule autotuner on this batch (digests are written
    as by keccak_batch); returns the chosen configuration and its time."""
    cfg = QueueConfig()
    _check(load().keccak_batch_autotune_ex(_ptr(msgs), _ptr(offsets), _ptr(lens), _ptr(variants), _ptr(out_lens),
                                           _ptr(digests), n, _stream(stream), ctypes.addressof(cfg)),
           "keccak_batch_autotune_ex")
    return cfg.as_dict()


def keccak_tuned_config(n: int) -> dict:
    """The configuration (register budget, blocks per SM, staging, threads per
    message) keccak_batch's queue schedule would use for n messages on the
    current device."""
    cfg = QueueConfig()
    _check(load().keccak_tuned_config_ex(n, ctypes.addressof(cfg)), "keccak_tuned_config_ex")
    d = cfg.as_dict()
    d.pop("ms")
    return d


def keccak_batch_noalloc(msgs, offsets, lens, variants, out_lens, digests, n: int, stream=None) -> None:
    """keccak_batch with its scratch in a fixed device array (no device
    allocation); at most KB_NOALLOC_MAX_MESSAGES messages; calls that overlap
    on the GPU race."""
    _check(load().keccak_batch_noalloc(_ptr(msgs), _ptr(offsets), _ptr(lens), _ptr(variants), _ptr(out_lens),
                                       _ptr(digests), n, _stream(stream)), "keccak_batch_noalloc")


def keccak_batch_uniform_host(h_msgs, stride: int, length: int, variant: int, out_len: int, h_digests,
                              n: int, stream=None) -> None:
    _check(load().keccak_batch_uniform_host(_ptr(h_msgs), stride, length, variant, out_len, _ptr(h_digests),
                                            n, _stream(stream)), "keccak_batch_uniform_host")


def keccak_host_path_for(n: int) -> int:
    """KB_HOST_PATH_STAGED / _ZERO_COPY chosen for n messages, or _AUTO while undecided."""
    return _check(load().keccak_host_path_for(n), "keccak_host_path_for")


class HostBuffer:
    """Page-locked host memory on the NUMA node nearest the current device
    (keccak_host_alloc); ``array`` is a numpy uint8 view of it.  Freed by
    ``free()`` or when the object is collected."""

    def __init__(self, nbytes: int):
        p = ctypes.c_void_p()
        _check(load().keccak_host_alloc(nbytes, ctypes.addressof(p)), "keccak_host_alloc")
        self.ptr, self.nbytes = int(p.value), nbytes
        self.array = np.ctypeslib.as_array((ctypes.c_uint8 * nbytes).from_address(self.ptr))

    def data_ptr(self) -> int:
        return self.ptr

    def numa_node(self) -> int:
        return int(load().keccak_host_numa_node(self.ptr))

    def free(self) -> None:
        if self.ptr:
            self.array = None
            _check(load().keccak_host_free(self.ptr), "keccak_host_free")
            self.ptr = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


KB_STATE_BYTES = 384
KB_SERVER_LONG_LANE_PARALLEL, KB_SERVER_LONG_THREAD_PER_REQUEST = 0, 1


def keccak_stream_init(states, variants, n: int, stream=None) -> None:
    _check(load().keccak_stream_init(_ptr(states), _ptr(variants), n, _stream(stream)), "keccak_stream_init")


def keccak_stream_absorb(states, msgs, offsets, lens, n: int, stream=None) -> None:
    _check(load().keccak_stream_absorb(_ptr(states), _ptr(msgs), _ptr(offsets), _ptr(lens), n, _stream(stream)),
           "keccak_stream_absorb")


def keccak_stream_final(states, out_lens, digests, n: int, stream=None) -> None:
    _check(load().keccak_stream_final(_ptr(states), _ptr(out_lens), _ptr(digests), n, _stream(stream)),
           "keccak_stream_final")


def keccak_stream_init_absorb(states, variants, msgs, offsets, lens, n: int, stream=None) -> None:
    _check(load().keccak_stream_init_absorb(_ptr(states), _ptr(variants), _ptr(msgs), _ptr(offsets), _ptr(lens), n,
                                            _stream(stream)), "keccak_stream_init_absorb")


def keccak_stream_absorb_final(states, msgs, offsets, lens, out_lens, digests, n: int, stream=None) -> None:
    _check(load().keccak_stream_absorb_final(_ptr(states), _ptr(msgs), _ptr(offsets), _ptr(lens), _ptr(out_lens),
                                             _ptr(digests), n, _stream(stream)), "keccak_stream_absorb_final")


def merkle_sha3_256(buf, n_leaves: int, leaf_bytes: int, stream=None) -> bytes:
    root = (ctypes.c_uint8 * 32)()
    _check(load().merkle_sha3_256(_ptr(buf), n_leaves, leaf_bytes, ctypes.addressof(root), _stream(stream)),
           "merkle_sha3_256")
    return bytes(root)


def merkle_sha3_256_many(buf, n_trees: int, leaves_per_tree: int, leaf_bytes: int, roots, stream=None) -> None:
    _check(load().merkle_sha3_256_many(_ptr(buf), n_trees, leaves_per_tree, leaf_bytes, _ptr(roots),
                                       _stream(stream)), "merkle_sha3_256_many")


def merkle_sha3_256_message(msg, length: int, chunk_bytes: int, stream=None) -> bytes:
    root = (ctypes.c_uint8 * 32)()
    _check(load().merkle_sha3_256_message(_ptr(msg), length, chunk_bytes, ctypes.addressof(root), _stream(stream)),
           "merkle_sha3_256_message")
    return bytes(root)


def merkle_node_count(n_leaves: int) -> int:
    return int(load().merkle_node_count(n_leaves))


def merkle_sha3_256_levels(buf, n_leaves: int, leaf_bytes: int, nodes, stream=None) -> None:
    _check(load().merkle_sha3_256_levels(_ptr(buf), n_leaves, leaf_bytes, _ptr(nodes), _stream(stream)),
           "merkle_sha3_256_levels")


def keccak_p_batch(states, b: int, nr: int, n: int, stream=None) -> None:
    _check(load().keccak_p_batch(_ptr(states), b, nr, n, _stream(stream)), "keccak_p_batch")


def keccak_last_error(stream=None) -> int:
    return _check(load().keccak_last_error(_stream(stream)), "keccak_last_error")


def keccak_release() -> None:
    load().keccak_release()


KB_TUNE_REPRESENTATION = 0
KB_REP_PLAIN, KB_REP_INTERLEAVED = 0, 1
KB_TUNE_RAGGED_SCHEDULE, KB_TUNE_GRAPHS, KB_TUNE_AUTOTUNE = 1, 2, 3
KB_TUNE_QUEUE_MIN_BLOCKS, KB_TUNE_QUEUE_BLOCKS_PER_SM = 4, 5
KB_SCHEDULE_INPUT_ORDER, KB_SCHEDULE_QUEUE, KB_SCHEDULE_LANE_PARALLEL, KB_SCHEDULE_PER_VARIANT = 0, 1, 2, 3
KB_TUNE_HOST_PATH = 6
KB_HOST_PATH_AUTO, KB_HOST_PATH_STAGED, KB_HOST_PATH_ZERO_COPY = 0, 1, 2
KB_TUNE_STAGING = 7
KB_STAGING_DIRECT, KB_STAGING_TMA = 0, 1
KB_TUNE_QUEUE_STAGING, KB_TUNE_QUEUE_WARP_MESSAGES = 8, 9
KB_QUEUE_STAGING_DIRECT, KB_QUEUE_STAGING_DIRECT_LOOPED, KB_QUEUE_STAGING_ASYNC, KB_QUEUE_STAGING_REGS = 1, 2, 3, 4
QUEUE_STAGING_NAMES = {KB_QUEUE_STAGING_DIRECT: "direct", KB_QUEUE_STAGING_DIRECT_LOOPED: "direct_looped",
                       KB_QUEUE_STAGING_ASYNC: "async", KB_QUEUE_STAGING_REGS: "regs"}
KB_TUNE_KEYS = 10


def keccak_tune_set(key: int, value: int) -> None:
    _check(load().keccak_tune_set(key, value), "keccak_tune_set")


def keccak_tune_get(key: int) -> int:
    return int(load().keccak_tune_get(key))


def round_constants() -> list[int]:
    out = (ctypes.c_uint64 * 24)()
    _check(load().sha3gb_round_constants(ctypes.addressof(out)), "sha3gb_round_constants")
    return list(out)


def rho_offsets() -> list[int]:
    out = (ctypes.c_uint32 * 25)()
    _check(load().sha3gb_rho_offsets(ctypes.addressof(out)), "sha3gb_rho_offsets")
    return list(out)


def int_issue_probe(op: int, iters: int = 4096, stream=None) -> float:
    """Measured 32-bit integer thread-instructions per SM clock for one kind of
    instruction: 0 LOP3 (chi table), 1 SHF (register shift), 2 PRMT (register
    selector), 3 three-input add."""
    out = ctypes.c_double()
    _check(load().sha3gb_int_issue_probe(op, iters, ctypes.addressof(out), _stream(stream)), "int_issue_probe")
    return out.value


def host_link_probe(host, device, nbytes: int, mode: int, reps: int = 5, stream=None) -> float:
    """GB/s over the host link: mode 0 copy engine host->device, 1 device->host,
    2 both at once (half each way), 3 SM loads of page-locked host memory."""
    out = ctypes.c_double()
    _check(load().sha3gb_host_link_probe(_ptr(host), _ptr(device), nbytes, mode, reps, ctypes.addressof(out),
                                         _stream(stream)), "sha3gb_host_link_probe")
    return out.value


def wait_timeout_probe(limit_ns: int, arrive: bool = False, stream=None) -> None:
    """Runs the staging kernel's bounded mbarrier wait on a barrier that
    nothing completes (arrive=False: it gives up after limit_ns and sets
    KB_DEV_TIMEOUT, read with keccak_last_error) or that completes at once."""
    _check(load().sha3gb_wait_timeout_probe(limit_ns, int(bool(arrive)), _stream(stream)), "wait_timeout_probe")


def version() -> str:
    return load().sha3gb_version().decode()


# ---- convenience: Python byte strings in, digests out ---------------------------
def pack_messages(messages, variants=KB_SHA3_256, out_lens=None):
    """The ragged-batch layout of keccak_batch for a sequence of byte strings:
    (msgs uint8, offsets uint64, lens uint64, variants uint8, out_lens uint32),
    messages back to back.  `variants` is one function id or one per message;
    `out_lens` defaults to the digest size of each SHA3 function and must be
    given (one value or one per message) for SHAKE."""
    n = len(messages)
    views = [np.frombuffer(bytes(m), dtype=np.uint8) for m in messages]
    lens = np.fromiter((v.size for v in views), dtype=np.uint64, count=n)
    offsets = np.zeros(n, dtype=np.uint64)
    if n > 1:
        np.cumsum(lens[:-1], out=offsets[1:])
    msgs = np.concatenate(views) if n and int(lens.sum()) else np.zeros(1, dtype=np.uint8)
    var = np.broadcast_to(np.asarray(variants, dtype=np.int64), (n,))
    if n and (var.min() < 0 or var.max() > 5):
        raise ValueError("variants must be function ids 0..5")
    var = var.astype(np.uint8)
    if out_lens is None:
        if n and (var >= 4).any():
            raise ValueError("SHAKE messages need an out_len")
        ol = np.array([DIGEST_BYTES[v] for v in var], dtype=np.uint32)
    else:
        ol = np.broadcast_to(np.asarray(out_lens, dtype=np.int64), (n,))
        if n and (ol.min() < 0 or ol.max() > 0xFFFFFFFF):
            raise ValueError("out_lens must fit in 32 bits")
        ol = ol.astype(np.uint32)
        for v, o in zip(var, ol):
            if v < 4 and o != DIGEST_BYTES[v]:
                raise ValueError(f"{NAMES[v]} gives {DIGEST_BYTES[v]} bytes, not {o}")
    return msgs, offsets, lens, var, ol


def hash_many(messages, variants=KB_SHA3_256, out_lens=None, stream=None) -> list[bytes]:
    """Hashes a sequence of byte strings as one ragged batch on the current
    CUDA device (keccak_batch) and returns their digests, in order."""
    import torch

    n = len(messages)
    if n == 0:
        return []
    msgs, offsets, lens, var, ol = pack_messages(messages, variants, out_lens)
    as_dev = lambda a: torch.from_numpy(a.view({8: np.int64, 4: np.int32, 1: np.uint8}[a.itemsize])).cuda()  # noqa
    d = [as_dev(np.ascontiguousarray(a)) for a in (msgs, offsets, lens, var, ol)]
    total = int(ol.sum(dtype=np.uint64))
    out = torch.empty(max(total, 1), dtype=torch.uint8, device="cuda")
    keccak_batch(*d, out, n, stream)
    err = keccak_last_error(stream)
    if err:
        raise Sha3gbError(-err, f"keccak_batch device status 0x{err:x}")
    host = out.cpu().numpy()[:total].tobytes()
    ends = np.cumsum(ol.astype(np.uint64))
    starts = ends - ol
    return [host[int(a):int(b)] for a, b in zip(starts, ends)]
