"""Serving loop: continuous batching of independent requests.

Each served result must equal its lattice run alone and the CPU oracle's
run of the same request (bit for bit: spins and the final exact counters),
requests that arrive while others run must be admitted and finish before
long ones do, and admission must respect the HBM budget and the slot limit.
"""
import time

import numpy as np
import pytest

import oracle
import paper_1209_0296_gb300 as lt
from paper_1209_0296_gb300.workloads import served_mix

pytestmark = pytest.mark.gpu

REQS = [
    dict(dims=2, L=64, two_S=1, model=lt.ISING, J=1.0, h=0.0, T_or_c=2.269185, seed=1234,
         init=lt.INIT_COLD, sweeps=300),
    dict(dims=2, L=128, two_S=1, model=lt.ISING, J=1.0, h=0.0, T_or_c=2.0, seed=5,
         init=lt.INIT_RANDOM, sweeps=77),
    dict(dims=2, L=96, two_S=1, model=lt.NE, J=0.0, h=0.0, T_or_c=0.2, seed=6,
         init=lt.INIT_EQUILIBRIUM, sweeps=500),
    dict(dims=2, L=50, two_S=1, model=lt.ISING, J=1.0, h=0.2, T_or_c=2.5, seed=7,
         init=lt.INIT_RANDOM, sweeps=41),
    dict(dims=3, L=8, two_S=2, model=lt.ISING, J=1.0, h=0.0, T_or_c=3.0, seed=8,
         init=lt.INIT_RANDOM, sweeps=260),
    dict(dims=2, L=256, two_S=1, model=lt.ISING, J=1.0, h=0.0, T_or_c=3.0, seed=9,
         init=lt.INIT_RANDOM, sweeps=0),
    dict(dims=2, L=320, two_S=1, model=lt.NE, J=0.0, h=0.0, T_or_c=0.05, seed=10,
         init=lt.INIT_EQUILIBRIUM, sweeps=129),
]


def _oracle(r):
    o = oracle.Lattice(r["dims"], r["L"], r["two_S"], r["model"], r["J"], r["h"], r["T_or_c"],
                       seed=r["seed"], init=r["init"])
    ser = o.sweep(r["sweeps"]) if r["sweeps"] > 0 else None
    return o, ser


def _check_against_oracle(r, spins, res):
    o, ser = _oracle(r)
    assert np.array_equal(spins, o.spins), r
    if ser is not None:
        # the unflipped count is kept for the North-East model only
        keys = ("bond", "mag", "up", "unflipped") if r["model"] == lt.NE else ("bond", "mag", "up")
        for key in keys:
            assert res[key] == ser[key][-1], (key, r)
    else:
        # no sweep ran, so there are no per-sweep counters: compare the
        # per-site observables of the initial state
        m = o.measure()
        N = r["L"] ** r["dims"]
        assert res["M"] == pytest.approx(m["mag"] / N)
        assert res["E"] == pytest.approx(float(o.energy(m["bond"], m["mag"])) / N)


def _solo(r):
    g = lt.Lattice(r["dims"], r["L"], r["two_S"], r["model"], r["J"], r["h"], r["T_or_c"],
                   seed=r["seed"], init=r["init"])
    g.sweep(r["sweeps"])
    return g


def test_served_results_equal_solo_runs():
    srv = lt.Server(hbm_budget_bytes=1 << 30, max_slots=64, chunk_sweeps=64)
    ids = [srv.submit(**r, keep_spins=True) for r in REQS]
    srv.drain(120.0)
    for rid, r in zip(ids, REQS):
        N = r["L"] ** r["dims"]
        spins = np.empty(N, dtype=np.int8)
        res = srv.poll(rid, spins)
        assert res is not None and res["status"] == 0, res
        assert res["sweeps_done"] == r["sweeps"]
        g = _solo(r)
        assert np.array_equal(spins, g.get_spins()), r
        o = g.observables()
        assert res["E"] == pytest.approx(o["E"]) and res["M"] == pytest.approx(o["M"])
        if r["sweeps"] > 0:
            ser = g.series(r["sweeps"] - 1, 1)
            assert res["bond"] == ser["bond"][0] and res["mag"] == ser["mag"][0]
        assert res["t_submit"] <= res["t_admit"] <= res["t_done"]
        _check_against_oracle(r, spins, res)
        with pytest.raises(lt.LatticeError):
            srv.poll(rid)  # released after the first successful poll
    srv.close()


def test_served_mix_requests_match_the_oracle():
    # the first requests of the served mix (L rounded to even, so sizes the
    # fast kernels do not take are served too), sweeps scaled down so the
    # oracle finishes in seconds; submitted back to back so they share rounds
    reqs = [r for r in served_mix(n=40, seed=99, sweep_scale=0.01) if r["L"] ** 2 * r["sweeps"] <= 3e7]
    assert len(reqs) >= 20 and any(r["L"] % 32 for r in reqs)
    srv = lt.Server(hbm_budget_bytes=1 << 30, max_slots=64, chunk_sweeps=32)
    keys = ("dims", "L", "two_S", "model", "J", "h", "T_or_c", "seed", "init", "sweeps")
    ids = [srv.submit(**{k: r[k] for k in keys}, keep_spins=True) for r in reqs]
    srv.drain(300.0)
    for rid, r in zip(ids, reqs):
        spins = np.empty(r["L"] ** 2, dtype=np.int8)
        res = srv.poll(rid, spins)
        assert res is not None and res["status"] == 0, res
        assert res["sweeps_done"] == r["sweeps"]
        _check_against_oracle(r, spins, res)
    srv.close()


def test_late_short_request_overlaps_and_finishes_first():
    srv = lt.Server(hbm_budget_bytes=1 << 30, max_slots=16, chunk_sweeps=32)
    long_id = srv.submit(dims=2, L=1024, model=lt.ISING, T_or_c=2.3, seed=3, sweeps=4000)
    time.sleep(0.05)
    short_id = srv.submit(dims=2, L=64, model=lt.ISING, T_or_c=2.3, seed=4, sweeps=64)
    assert srv.poll(long_id) is None          # still running (LAT_EBUSY)
    srv.drain(300.0)
    a, b = srv.poll(long_id), srv.poll(short_id)
    assert b["t_admit"] < a["t_done"]         # admitted while the long one ran
    assert b["t_done"] < a["t_done"]          # and finished first
    srv.close()


def test_budget_and_slots_serialise_admission():
    # each L=256 Ising lattice is charged ~142 kB (two spin buffers, table,
    # counters); a 200 kB budget holds one at a time
    srv = lt.Server(hbm_budget_bytes=200_000, max_slots=8, chunk_sweeps=16)
    ids = [srv.submit(dims=2, L=256, model=lt.ISING, T_or_c=2.5, seed=s, sweeps=40)
           for s in range(4)]
    srv.drain(120.0)
    res = [srv.poll(i) for i in ids]
    assert all(r["status"] == 0 for r in res)
    for prev, nxt in zip(res, res[1:]):
        assert nxt["t_admit"] >= prev["t_done"] - 1e-6
    srv.close()
    srv = lt.Server(hbm_budget_bytes=1 << 30, max_slots=1, chunk_sweeps=16)
    ids = [srv.submit(dims=2, L=64, model=lt.ISING, T_or_c=2.5, seed=s, sweeps=20) for s in range(3)]
    srv.drain(120.0)
    res = [srv.poll(i) for i in ids]
    for prev, nxt in zip(res, res[1:]):
        assert nxt["t_admit"] >= prev["t_done"] - 1e-6
    srv.close()


def test_invalid_and_oversized_requests():
    srv = lt.Server(hbm_budget_bytes=100_000, max_slots=4, chunk_sweeps=16)
    with pytest.raises(lt.LatticeError) as e:
        srv.submit(dims=4, L=16, sweeps=1)
    assert e.value.code == -1
    with pytest.raises(lt.LatticeError) as e:
        srv.submit(dims=2, L=1024, sweeps=1)      # 2 MB > budget: can never be admitted
    assert e.value.code == -2
    with pytest.raises(lt.LatticeError) as e:
        srv.poll(12345)
    assert e.value.code == -8
    srv.close()


def test_drain_times_out_on_the_host_then_finishes():
    # a bounded wait that runs out: drain returns LAT_ETIMEOUT (the request
    # keeps running), and a later unbounded drain sees it finish
    srv = lt.Server(hbm_budget_bytes=1 << 30, max_slots=8, chunk_sweeps=256)
    rid = srv.submit(dims=2, L=2048, model=lt.ISING, T_or_c=2.3, seed=3, sweeps=60000)
    with pytest.raises(lt.LatticeError) as err:
        srv.drain(0.001)
    assert err.value.code == -4
    srv.drain(0.0)
    res = srv.poll(rid)
    assert res is not None and res["status"] == 0 and res["sweeps_done"] == 60000
    srv.close()


def test_a_failed_request_ends_alone():
    # An allocation failure injected on the host hits one request's lattice
    # creation: that request ends with LAT_ENOMEM while a long request that
    # was already running and one submitted after it finish, bit-exact.
    lib = lt.load()
    srv = lt.Server(hbm_budget_bytes=1 << 30, max_slots=16, chunk_sweeps=32)
    long_req = dict(dims=2, L=1024, two_S=1, model=lt.ISING, J=1.0, h=0.0, T_or_c=2.3, seed=3,
                    init=lt.INIT_RANDOM, sweeps=3000)
    wid = srv.submit(**long_req)
    t0 = time.time()
    while srv.stats()["rounds"] < 4 and time.time() - t0 < 60:   # its upload slots are all in use by now
        time.sleep(0.005)
    lib.lattice_test_fail_alloc(1)            # the next device allocation fails
    bad = srv.submit(dims=2, L=96, model=lt.ISING, T_or_c=2.5, seed=4, sweeps=50)
    late = dict(dims=2, L=50, two_S=1, model=lt.NE, J=0.0, h=0.0, T_or_c=0.3, seed=5,
                init=lt.INIT_EQUILIBRIUM, sweeps=80)
    res_bad = None
    try:
        t0 = time.time()
        while res_bad is None and time.time() - t0 < 60:
            res_bad = srv.poll(bad)
            time.sleep(0.002)
    finally:
        lib.lattice_test_fail_alloc(0)
    assert res_bad is not None and res_bad["status"] == -2 and res_bad["sweeps_done"] == 0
    assert srv.poll(wid) is None              # the long request is still running
    lid = srv.submit(**late, keep_spins=True)
    srv.drain(300.0)
    N = late["L"] ** 2
    spins = np.empty(N, dtype=np.int8)
    res_late = srv.poll(lid, spins)
    res_long = srv.poll(wid)
    assert res_late["status"] == 0 and res_long["status"] == 0
    assert res_long["sweeps_done"] == 3000
    _check_against_oracle(late, spins, res_late)
    srv.close()


def test_failed_request_status_is_reported():
    lib = lt.load()
    srv = lt.Server(hbm_budget_bytes=1 << 30, max_slots=4, chunk_sweeps=16)
    lib.lattice_test_fail_alloc(1)
    try:
        rid = srv.submit(dims=2, L=64, model=lt.ISING, T_or_c=2.5, seed=4, sweeps=10)
        srv.drain(60.0)
    finally:
        lib.lattice_test_fail_alloc(0)
    res = srv.poll(rid)
    assert res["status"] == -2 and res["sweeps_done"] == 0   # LAT_ENOMEM
    ok = srv.submit(dims=2, L=64, model=lt.ISING, T_or_c=2.5, seed=4, sweeps=10)
    srv.drain(60.0)
    assert srv.poll(ok)["status"] == 0
    srv.close()


def test_busy_time_is_reported():
    srv = lt.Server(hbm_budget_bytes=1 << 30, max_slots=16, chunk_sweeps=64)
    for s in range(6):
        srv.submit(dims=2, L=512, model=lt.ISING, T_or_c=2.3, seed=s, sweeps=400)
    srv.drain(120.0)
    st = srv.stats()
    assert st["rounds"] >= 7 and 0.0 < st["busy_s"] <= st["wall_s"]
    srv.close()
