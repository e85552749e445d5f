"""The autotuner's optional cache file (LATTICE_TUNE_CACHE): a tuned choice
is appended as one JSON line, a later process takes a valid entry without
tuning, and an entry the lattice cannot run is ignored.  Each case runs in a
fresh process, since the cache file is read once per process."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROBE = r"""
import json, sys
import paper_1209_0296_gb300 as lt
L = int(sys.argv[1])
g = lt.Lattice(2, L, 1, lt.ISING, 1.0, 0.0, 2.3, seed=3, init=lt.INIT_RANDOM)
g.sweep(64)
g.synchronize()
k = g.get_kernel()
print(json.dumps({"kernel": k["kernel"], "tile_h": k["tile_h"]}))
"""


def _run(L, cache):
    env = dict(os.environ, LATTICE_TUNE_CACHE=str(cache), PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", PROBE, str(L)], env=env, capture_output=True, text=True,
                         timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_tuned_choice_is_written(tmp_path):
    cache = tmp_path / "tune.jsonl"
    k = _run(256, cache)
    lines = [json.loads(x) for x in cache.read_text().splitlines()]
    assert len(lines) == 1
    e = lines[0]
    assert (e["model"], e["L"]) == (0, 256)
    assert e["kernel"] == k["kernel"]


def test_cached_choice_is_taken(tmp_path):
    cache = tmp_path / "tune.jsonl"
    cache.write_text('{"model": 0, "L": 192, "kernel": 2, "tile_h": 32}\n')
    k = _run(192, cache)
    assert (k["kernel"], k["tile_h"]) == (2, 32)   # the tiled kernel, as the file says
    assert len(cache.read_text().splitlines()) == 1   # no new tuning appended


def test_unusable_entry_is_ignored(tmp_path):
    cache = tmp_path / "tune.jsonl"
    # the resident kernel cannot hold an L = 1024 lattice in one CTA
    cache.write_text('{"model": 0, "L": 1024, "kernel": 4, "tile_h": 0}\n')
    k = _run(1024, cache)
    assert k["kernel"] != 4
    assert len(cache.read_text().splitlines()) == 2   # tuned afresh and appended
