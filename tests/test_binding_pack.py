"""The binding's packing of Python byte strings into keccak_batch's ragged
layout (host-side marshalling, no GPU), and its checks."""
import numpy as np
import pytest

from paper_1902_05320_gb300 import binding as kb


def test_messages_back_to_back_with_offsets_and_lengths():
    msgs, offs, lens, var, ol = kb.pack_messages([b"abc", b"", b"hello", bytes(range(200))])
    assert msgs.dtype == np.uint8 and msgs.tobytes() == b"abc" + b"hello" + bytes(range(200))
    assert offs.tolist() == [0, 3, 3, 8] and lens.tolist() == [3, 0, 5, 200]
    assert var.tolist() == [1, 1, 1, 1] and ol.tolist() == [32, 32, 32, 32]
    assert (offs.dtype, lens.dtype, var.dtype, ol.dtype) == (np.uint64, np.uint64, np.uint8, np.uint32)


def test_per_message_variants_and_shake_lengths():
    _, _, _, var, ol = kb.pack_messages([b"a", b"b", b"c", b"d"], variants=[0, 3, 4, 5], out_lens=[28, 64, 1, 500])
    assert var.tolist() == [0, 3, 4, 5] and ol.tolist() == [28, 64, 1, 500]
    _, _, _, var, ol = kb.pack_messages([b"a", b"b"], variants=kb.KB_SHAKE128, out_lens=0)
    assert var.tolist() == [4, 4] and ol.tolist() == [0, 0]


def test_empty_batch_and_empty_messages():
    msgs, offs, lens, var, ol = kb.pack_messages([])
    assert offs.size == 0 and lens.size == 0 and msgs.size == 1
    msgs, offs, lens, _, _ = kb.pack_messages([b"", b""])
    assert lens.tolist() == [0, 0] and offs.tolist() == [0, 0] and msgs.size == 1


@pytest.mark.parametrize("kwargs", [dict(variants=6), dict(variants=-1), dict(variants=kb.KB_SHAKE256),
                                    dict(variants=kb.KB_SHA3_256, out_lens=31), dict(variants=5, out_lens=-1),
                                    dict(variants=4, out_lens=1 << 32)])
def test_bad_arguments_are_refused_on_the_host(kwargs):
    with pytest.raises(ValueError):
        kb.pack_messages([b"x", b"y"], **kwargs)
