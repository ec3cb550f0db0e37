"""Pins the oracle's tree mode against a second, recursive definition.

The paper's tree mode (Section 4) combines digests pairwise up to a root and
fixes no node format; the library's rules are leaf = SHA3-256(0x00 || leaf),
node = SHA3-256(0x01 || left || right), one level at a time, an odd last node
carried up unchanged.  Level-by-level pairing with that carry equals the
recursive split at the largest power of two below n, written here with
hashlib, independently of the oracle's loop.
"""
import hashlib

import numpy as np
import pytest


def _h(data: bytes) -> bytes:
    return hashlib.sha3_256(data).digest()


def _recursive_root(leaves):
    if len(leaves) == 1:
        return _h(b"\x00" + leaves[0])
    k = 1
    while 2 * k < len(leaves):
        k *= 2
    return _h(b"\x01" + _recursive_root(leaves[:k]) + _recursive_root(leaves[k:]))


@pytest.mark.parametrize("n_leaves", list(range(1, 34)) + [64, 65, 100])
def test_merkle_root_matches_recursive_definition(oracle_mod, n_leaves):
    rng = np.random.default_rng(n_leaves)
    leaf_bytes = 1 + n_leaves % 7 * 19
    buf = rng.integers(0, 256, size=n_leaves * leaf_bytes, dtype=np.uint8).tobytes()
    leaves = [buf[i * leaf_bytes:(i + 1) * leaf_bytes] for i in range(n_leaves)]
    assert oracle_mod.merkle_root(buf, n_leaves, leaf_bytes) == _recursive_root(leaves)


def test_odd_node_is_promoted_unchanged(oracle_mod):
    buf = bytes(range(35))
    L = [_h(b"\x00" + buf[5 * i:5 * i + 5]) for i in range(7)]
    n01, n23, n45 = (_h(b"\x01" + L[a] + L[a + 1]) for a in (0, 2, 4))
    # n = 3: the third leaf digest rises one level unchanged.
    assert oracle_mod.merkle_root(buf, 3, 5) == _h(b"\x01" + n01 + L[2])
    # n = 5: the fifth leaf digest rises two levels unchanged.
    assert oracle_mod.merkle_root(buf, 5, 5) == _h(b"\x01" + _h(b"\x01" + n01 + n23) + L[4])
    # n = 7: levels are 7 -> 4 -> 2 -> 1, with leaf 6 carried once.
    n456 = _h(b"\x01" + n45 + L[6])
    assert oracle_mod.merkle_root(buf, 7, 5) == _h(b"\x01" + _h(b"\x01" + n01 + n23) + n456)


def test_merkle_levels_layout(oracle_mod):
    buf = bytes(range(6 * 3))
    nodes = oracle_mod.merkle_levels(buf, 6, 3)
    assert nodes.shape == (6 + 3 + 2 + 1, 32)
    assert oracle_mod.merkle_node_count(6) == 12
    assert oracle_mod.merkle_node_count(1) == 1
    assert nodes[0].tobytes() == _h(b"\x00" + buf[:3])
    assert nodes[-1].tobytes() == oracle_mod.merkle_root(buf, 6, 3)
    # The odd node of level 1 (index 8 overall) is copied to level 2 unchanged.
    assert nodes[10].tobytes() == nodes[8].tobytes()


def test_merkle_rejects_empty(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.merkle_root(b"", 0, 8)
    with pytest.raises(ValueError):
        oracle_mod.merkle_root(b"abc", 1, 0)


@pytest.mark.parametrize("length,chunk", [(0, 64), (1, 64), (64, 64), (65, 64), (1000, 64), (1000, 999),
                                          (4097, 128), (777, 1), (3000, 136), (135, 136)])
def test_message_tree_matches_recursive_definition(oracle_mod, length, chunk):
    # One message cut into chunks (last one shorter; empty message = one empty
    # leaf), the same leaf/node rules, against the recursive definition.
    msg = np.random.default_rng(length + chunk).integers(0, 256, size=length, dtype=np.uint8).tobytes()
    leaves = [msg[i:i + chunk] for i in range(0, length, chunk)] or [b""]
    assert oracle_mod.merkle_message_root(msg, chunk) == _recursive_root(leaves)
