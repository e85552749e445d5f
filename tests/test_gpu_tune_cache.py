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


PROBE3 = r"""
import json, sys
import numpy as np
import paper_1209_0296_gb300 as lt
dims, L, two_S, model = (int(x) for x in sys.argv[1:5])
args = (dims, L, two_S, model, 1.0, 0.0, 2.7) if model != lt.NE else (dims, L, two_S, model, 0.0, 0.0, 0.3)
init = lt.INIT_EQUILIBRIUM if model == lt.NE else lt.INIT_RANDOM
g = lt.Lattice(*args, seed=5, init=init)
g.sweep(300)                      # tuned on these sweeps
ref = lt.Lattice(*args, seed=5, init=init)
ref.set_kernel(lt.KERNEL_WIDE, 0, 0, 3)   # fixed kernel, graph size 3 (pinned: never tuned)
ref.sweep(300)
k = g.get_kernel()
same = bool(np.array_equal(g.get_spins(), ref.get_spins())) and bool(
    np.array_equal(g.series(0, 300)["bond"], ref.series(0, 300)["bond"]))
print(json.dumps({"kernel": k["kernel"], "graph": k["sweeps_per_graph"], "same": same,
                  "ref_graph": ref.get_kernel()["sweeps_per_graph"]}))
"""


@pytest.mark.parametrize("dims,L,two_S,model", [(2, 4096, 1, 0), (2, 1000, 1, 1), (3, 64, 2, 0), (2, 256, 2, 2)])
def test_graph_size_is_tuned_and_changes_no_bits(tmp_path, dims, L, two_S, model):
    # the tuner picks the sweeps per graph replay for every model and
    # dimension (3D spin-1, Potts and North-East at L % 32 != 0 included),
    # records it, and the tuned lattice ends bit for bit where a lattice
    # with a fixed kernel and graph size ends
    cache = tmp_path / "tune.jsonl"
    env = dict(os.environ, LATTICE_TUNE_CACHE=str(cache), PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", PROBE3, str(dims), str(L), str(two_S), str(model)], env=env,
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    r = json.loads(out.stdout.strip().splitlines()[-1])
    assert r["same"] and r["ref_graph"] == 3
    lines = [json.loads(x) for x in cache.read_text().splitlines()]
    assert len(lines) == 1
    e = lines[0]
    assert (e["model"], e["dims"], e["two_S"], e["L"]) == (model, dims, two_S, L)
    assert e["graph"] > 0 and e["graph"] == r["graph"]
