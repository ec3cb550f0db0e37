"""Tuned queue configurations across processes: the SHA3GB_TUNE_CACHE file and
the SHA3GB_TUNE modes.  The library reads both variables once per process, so
each case runs in a fresh Python child; digests are checked against the
oracle here."""
import hashlib
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1902_05320_gb300 import workloads as W

pytestmark = pytest.mark.gpu

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N, SEED, MAX_LEN, GAP = 3000, 95, 8000, 3

CHILD = r"""
import hashlib, json, sys
import torch
from paper_1902_05320_gb300 import binding as kb, workloads as W
n, seed, max_len, gap, action = int(sys.argv[1]), int(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4]), sys.argv[5]
b = W.ragged_batch(n, seed=seed, max_len=max_len, gap=gap)
d = [torch.from_numpy(x).cuda() for x in (b.msgs, b.offsets, b.lens, b.variants, b.out_lens)]
out = torch.zeros(b.total_out(), dtype=torch.uint8, device="cuda")
res = {"before": kb.keccak_tuned_config(n)}
if action == "autotune":
    res["chosen"] = kb.keccak_batch_autotune(*d, out, n)
else:
    kb.keccak_batch(*d, out, n)
torch.cuda.synchronize()
res["after"] = kb.keccak_tuned_config(n)
res["digest"] = hashlib.sha256(out.cpu().numpy().tobytes()).hexdigest()
print(json.dumps(res))
"""


def _child(action, cache=None, mode=None):
    env = dict(os.environ)
    env.pop("SHA3GB_TUNE_CACHE", None)
    env.pop("SHA3GB_TUNE", None)
    if cache is not None:
        env["SHA3GB_TUNE_CACHE"] = str(cache)
    if mode is not None:
        env["SHA3GB_TUNE"] = mode
    r = subprocess.run([sys.executable, "-c", CHILD, str(N), str(SEED), str(MAX_LEN), str(GAP), action],
                       cwd=REPO, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.fixture(scope="module")
def want(oracle_mod):
    b = W.ragged_batch(N, seed=SEED, max_len=MAX_LEN, gap=GAP)
    out = oracle_mod.hash_batch(b.msgs, b.offsets, b.lens, b.variants, b.out_lens, os.cpu_count() or 1)
    return hashlib.sha256(np.ascontiguousarray(out).tobytes()).hexdigest()


def _lines(path):
    return [json.loads(l) for l in path.read_text().splitlines() if l]


SIZE_CLASS = N.bit_length() - 1
# The built-in configuration (no tuned entry, no knob).
DEFAULT = {"min_blocks": 2, "blocks_per_sm": 0, "staging": "regs", "threads_per_message": "1", "warp_messages": 0}
ROW_KEYS = {"gpu", "sms", "size_class", "min_blocks", "blocks_per_sm", "staging", "warp_messages"}
STAGING = {"direct": 1, "direct_looped": 2, "async": 3, "regs": 4}


def _dims(cfg):
    return {k: cfg[k] for k in DEFAULT}


def _row_dims(row):
    return (row["min_blocks"], row["blocks_per_sm"], row["staging"], row["warp_messages"])


def _cfg_dims(cfg):
    return (cfg["min_blocks"], cfg["blocks_per_sm"], STAGING[cfg["staging"]], cfg["warp_messages"])


def test_cache_file_carries_the_tuned_configuration(tmp_path, want):
    cache = tmp_path / "tune.jsonl"
    first = _child("autotune", cache)
    assert first["digest"] == want
    chosen = first["chosen"]
    assert first["after"] == _dims(chosen)
    rows = _lines(cache)
    assert len(rows) == 1 and set(rows[0]) == ROW_KEYS
    assert rows[0]["size_class"] == SIZE_CLASS and rows[0]["sms"] >= 1
    assert _row_dims(rows[0]) == _cfg_dims(chosen)
    # A new process on the same GPU starts from the file.
    second = _child("batch", cache)
    assert second["before"] == first["after"] and second["digest"] == want
    # Tuning the same size class again replaces its line.
    third = _child("autotune", cache)
    assert third["digest"] == want and len(_lines(cache)) == 1


def test_tune_off_ignores_the_cache(tmp_path, want):
    cache = tmp_path / "tune.jsonl"
    first = _child("autotune", cache)
    off = _child("batch", cache, mode="off")
    assert off["before"] == DEFAULT and off["digest"] == want
    assert first["digest"] == want


def test_tune_full_tunes_on_first_sight(tmp_path, want):
    cache = tmp_path / "tune.jsonl"
    full = _child("batch", cache, mode="full")
    assert full["before"] == DEFAULT
    assert full["after"]["min_blocks"] in (2, 3, 4, 5, 6, 8) and full["after"]["blocks_per_sm"] >= 1
    assert full["digest"] == want
    rows = _lines(cache)
    assert len(rows) == 1 and rows[0]["size_class"] == SIZE_CLASS
    assert _row_dims(rows[0]) == _cfg_dims(full["after"])


def test_malformed_and_foreign_cache_lines_are_ignored(tmp_path, want):
    cache = tmp_path / "tune.jsonl"
    # Learn this GPU's name and SM count from a file the library wrote.
    probe = tmp_path / "probe.jsonl"
    _child("autotune", probe)
    row = _lines(probe)[0]
    entry = dict(row, size_class=SIZE_CLASS)
    cache.write_text("garbage\n"
                     + json.dumps(dict(entry, gpu="Some other GPU", min_blocks=8, blocks_per_sm=1)) + "\n"
                     + json.dumps(dict(entry, sms=row["sms"] + 1, min_blocks=8, blocks_per_sm=1)) + "\n"
                     + json.dumps(dict(entry, min_blocks=7, blocks_per_sm=1)) + "\n"  # not a compiled budget
                     + json.dumps(dict(entry, min_blocks=8, blocks_per_sm=99)) + "\n"  # out of range
                     + json.dumps(dict(entry, min_blocks=8, staging=3)) + "\n"  # staging not compiled at 8
                     + json.dumps(dict(entry, min_blocks=2, staging=9)) + "\n"  # no such staging
                     + json.dumps(dict(entry, min_blocks=2, warp_messages=-5)) + "\n"
                     + '{"gpu": "", "sms": 1}\n')
    r = _child("batch", cache)
    assert r["before"] == DEFAULT and r["digest"] == want
    # The same entry with valid values is taken.
    cache.write_text(json.dumps(dict(entry, min_blocks=8, blocks_per_sm=1, staging=1, warp_messages=0)) + "\n")
    r = _child("batch", cache)
    assert r["before"] == dict(DEFAULT, min_blocks=8, blocks_per_sm=1, staging="direct") and r["digest"] == want
    cache.write_text(json.dumps(dict(entry, min_blocks=2, blocks_per_sm=1, staging=4, warp_messages=32)) + "\n")
    r = _child("batch", cache)
    assert r["before"] == dict(DEFAULT, min_blocks=2, blocks_per_sm=1, staging="regs", warp_messages=32,
                               threads_per_message="32 for the 32 costliest, 1 for the rest")
    assert r["digest"] == want
    # A line in the older form (no staging, no warp_messages) reads as direct
    # loads with one thread per message.
    old = {k: entry[k] for k in ("gpu", "sms", "size_class")}
    cache.write_text(json.dumps(dict(old, min_blocks=4, blocks_per_sm=2)) + "\n")
    r = _child("batch", cache)
    assert r["before"] == dict(DEFAULT, min_blocks=4, blocks_per_sm=2, staging="direct") and r["digest"] == want
