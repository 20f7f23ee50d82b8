"""Serving loop: resident systems, continuous batching across worker streams,
admission by device-memory budget with eviction, per-request failures and
cancellation.  Every result must equal the same system's result computed
alone (bitwise: the kernels are deterministic and a request touches only its
own system's buffers)."""
import math
import time

import numpy as np
import pytest

import paper_1711_02976_gb300 as rp
import synth
from gpu_util import matvec

pytestmark = pytest.mark.gpu


def _systems(seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for k, n in enumerate([3000, 12000, 800, 25000, 5000]):
        pos = rng.random((n, 3)) if k % 2 == 0 else synth._sphere_surface(rng, n, 0.5, (0.5, 0.5, 0.5))
        a = 0.5 / n ** (1 / 3) * 0.3
        out.append((pos, a, 3 if k % 2 == 0 else 6, 1 if k % 2 == 0 else 0))
    return out


def test_results_in_the_mix_equal_results_alone():
    rng = np.random.default_rng(1)
    systems = _systems()
    srv = rp.rpy_server_create(slots=3)
    try:
        ids = [rp.rpy_server_add_system(srv, pos, a, d, precision=prec) for pos, a, d, prec in systems]
        jobs = []
        for r in range(30):
            k = int(rng.integers(len(systems)))
            pos, a, d, prec = systems[k]
            newpos = pos + 1e-3 * rng.standard_normal(pos.shape) if r % 3 else None
            f = rng.standard_normal(pos.shape)
            u = np.zeros_like(f)
            rid = rp.rpy_server_submit(srv, ids[k], newpos, f, 6 * math.pi * a, u)
            jobs.append((rid, k, newpos, f, u))
        last_pos = [s[0] for s in systems]
        for i, (rid, k, newpos, f, u) in enumerate(jobs):
            if i % 2:
                st, lat = rp.rpy_server_wait(srv, rid)
            else:
                st, lat, tm = rp.rpy_server_wait_times(srv, rid)
                # phase times: device time of each phase inside the worker's wall time
                assert tm["matvec_ms"] > 0 and tm["h2d_ms"] > 0 and tm["d2h_ms"] > 0
                if newpos is not None:
                    assert tm["build_ms"] > 0   # new positions: the tree is rebuilt
                assert tm["h2d_ms"] + tm["build_ms"] + tm["matvec_ms"] + tm["d2h_ms"] <= tm["run_ms"] + 1.0
                assert tm["queue_ms"] + tm["run_ms"] <= lat + 1.0
            assert st == 0 and lat > 0
            pos, a, d, prec = systems[k]
            if newpos is not None:
                last_pos[k] = newpos
            ref, _ = matvec(last_pos[k], f, a, 6 * math.pi * a, d, precision=prec)
            np.testing.assert_array_equal(u, ref)
        stats = rp.rpy_server_stats_get(srv)
        assert stats["completed"] == 30 and stats["failed"] == 0 and stats["p99_ms"] >= stats["p50_ms"] > 0
    finally:
        rp.rpy_server_destroy(srv)


def test_admission_budget_evicts_and_serves_everything():
    rng = np.random.default_rng(2)
    systems = _systems(3)
    fps = [rp.rpy_tree_footprint(len(p), d, prec) for p, a, d, prec in systems]
    budget = max(fps) + min(fps)          # never all resident at once
    srv = rp.rpy_server_create(device_budget_bytes=budget, slots=2)
    try:
        ids = [rp.rpy_server_add_system(srv, pos, a, d, precision=prec) for pos, a, d, prec in systems]
        jobs = []
        for r in range(20):
            k = r % len(systems)
            pos, a, d, prec = systems[k]
            f = rng.standard_normal(pos.shape)
            u = np.zeros_like(f)
            jobs.append((rp.rpy_server_submit(srv, ids[k], None, f, 1.0, u), k, f, u))
        for rid, k, f, u in jobs:
            assert rp.rpy_server_wait(srv, rid)[0] == 0
            pos, a, d, prec = systems[k]
            ref, _ = matvec(pos, f, a, 1.0, d, precision=prec)
            np.testing.assert_array_equal(u, ref)
        st = rp.rpy_server_stats_get(srv)
        assert st["evictions"] > 0 and st["peak_resident_bytes"] <= budget * 1.5
    finally:
        rp.rpy_server_destroy(srv)


def test_poisoned_request_fails_alone_and_cancel():
    rng = np.random.default_rng(4)
    pos, a, d, prec = _systems()[0]
    srv = rp.rpy_server_create(slots=1)
    try:
        sid = rp.rpy_server_add_system(srv, pos, a, d, precision=prec)
        bad = pos.copy()
        bad[5, 0] = np.nan
        f = rng.standard_normal(pos.shape)
        u_bad, u_ok, u_c = np.zeros_like(f), np.zeros_like(f), np.zeros_like(f)
        r_bad = rp.rpy_server_submit(srv, sid, bad, f, 1.0, u_bad)
        r_ok = rp.rpy_server_submit(srv, sid, pos, f, 1.0, u_ok)
        r_c = rp.rpy_server_submit(srv, sid, None, f, 1.0, u_c)
        cancelled = rp.rpy_server_cancel(srv, r_c) == 0
        assert rp.rpy_server_wait(srv, r_bad)[0] == -6          # non-finite positions
        assert rp.rpy_server_wait(srv, r_ok)[0] == 0             # the system recovers
        ref, _ = matvec(pos, f, a, 1.0, d, precision=prec)
        np.testing.assert_array_equal(u_ok, ref)
        st_c = rp.rpy_server_wait(srv, r_c)[0]
        assert st_c == (-7 if cancelled else 0)
    finally:
        rp.rpy_server_destroy(srv)


def test_served_results_match_the_oracle_at_serving_sizes():
    """Requests of the serving mix at realistic sizes (a 300k-bead cube in the 3-digit FP32
    form and a 200k-bead sphere at 6 digits in FP64, jittered positions and fresh forces each
    request, both resident, requests interleaved on three slots) meet their digit settings
    against the oracle on sampled targets."""
    import oracle
    rng = np.random.default_rng(9)
    n1, n2 = 300000, 200000
    cube = rng.random((n1, 3))
    sph = synth._sphere_surface(rng, n2, 0.5, (0.5, 0.5, 0.5))
    a1, a2 = 0.5 / n1 ** (1 / 3), 0.5 / n2 ** (1 / 3)
    srv = rp.rpy_server_create(slots=3)
    try:
        s1 = rp.rpy_server_add_system(srv, cube, a1, 3, precision=rp.RPY_FP32)
        s2 = rp.rpy_server_add_system(srv, sph, a2, 6, precision=rp.RPY_FP64)
        jobs = []
        for r in range(6):
            sid, base, a, tol = (s1, cube, a1, 1e-3) if r % 2 == 0 else (s2, sph, a2, 1e-6)
            pos = base + 1e-3 * rng.standard_normal(base.shape)
            f = rng.standard_normal(base.shape)
            u = np.zeros_like(f)
            jobs.append((rp.rpy_server_submit(srv, sid, pos, f, 6 * math.pi * a, u), pos, f, a, tol, u))
        for rid, pos, f, a, tol, u in jobs:
            assert rp.rpy_server_wait(srv, rid)[0] == 0
            tg = synth.sample_targets(len(pos), 200, seed=rid)
            ref = oracle.rpy_direct(pos, f, a, 6 * math.pi * a, targets=tg)
            assert oracle.rel_l2(u[tg], ref) <= tol
    finally:
        rp.rpy_server_destroy(srv)
