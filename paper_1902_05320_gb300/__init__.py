"""Batch SHA-3 (SHA3-224/256/384/512, SHAKE128/256) and Merkle roots on GB300.

The hashing runs in the CUDA library ``libsha3gb.so`` (C ABI in
``include/sha3gb.h``); ``binding`` is its thin ctypes wrapper, ``workloads``
the seeded synthetic input generators, ``build`` the in-tree nvcc build.
"""
from .binding import (  # noqa: F401
    DIGEST_BYTES, NAMES, RATE_BYTES, Sha3gbError, keccak_batch, keccak_batch_uniform,
    keccak_batch_uniform_host, keccak_last_error, keccak_release, merkle_node_count, merkle_sha3_256,
    merkle_sha3_256_levels, rho_offsets, round_constants, version,
)
