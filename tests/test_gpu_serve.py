"""Continuous-batching server: admission by footprint, results equal each solve alone.

Requests that arrive while others are active join the running batch (same
launches), so a solve's result must not depend on its neighbours: the server's
kinetic energy and enstrophy of every solve equal, bit for bit, those of the same
solve run alone through fd_create / fd_step / fd_diagnostics; the final states of
binary64 and mixed binary64 / double-word solves served in a mix match the FP64
oracle (relative L-inf 1e-12), and every solve's final state equals the same solve
alone over the whole state.
"""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1610_09146_gb300 as fd  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    fd.build()


REQS = [
    dict(tag=1, n=16, steps=7, Re=1600.0, Mach=0.1, dtype="f32", algorithm="recompute_all", dt=1e-3),
    dict(tag=2, n=(20, 18, 24), steps=3, Re=500.0, Mach=0.3, dtype="f64", algorithm="store_some", dt=2e-3),
    dict(tag=3, n=24, steps=5, Re=2000.0, Mach=0.2, dtype="f32", algorithm="store_some", tile_points=128, dt=1e-3),
    dict(tag=4, n=12, steps=9, Re=900.0, Mach=0.35, dtype="f64", algorithm="recompute_all", dt=1e-3),
    dict(tag=5, n=16, steps=4, Re=3000.0, Mach=0.15, dtype="f32", algorithm="recompute_all", dt=1e-3),
]


def alone(r):
    with fd.Solver(r["n"], Re=r["Re"], Mach=r["Mach"], dt=r["dt"], algorithm=r["algorithm"], dtype=r["dtype"]) as s:
        s.step(r["steps"])
        return s.diagnostics()


def test_results_in_the_mix_equal_alone():
    got = {}
    with fd.Server(1 << 30, max_active=8) as srv:
        srv.submit(REQS[0])
        srv.submit(REQS[1])
        srv.tick()
        srv.submit(REQS[2])      # joins while 1 and 2 are active
        srv.tick()
        srv.tick()
        srv.submit(REQS[3])
        srv.submit(REQS[4])
        for _ in range(40):
            srv.tick()
            for r in srv.poll():
                got[r["tag"]] = r
            if len(got) == len(REQS):
                break
    assert set(got) == {r["tag"] for r in REQS}
    for r in REQS:
        ke, en = alone(r)
        assert got[r["tag"]]["status"] == fd.FD_OK
        assert got[r["tag"]]["steps"] == r["steps"]
        assert got[r["tag"]]["ke"] == ke and got[r["tag"]]["enstrophy"] == en, r["tag"]


def test_admission_respects_the_arena():
    big = dict(tag=10, n=32, steps=2, dtype="f64", algorithm="store_some", dt=1e-3)
    with fd.Server(1 << 30, max_active=4) as probe:
        need = probe.footprint(big)
    # an arena for exactly one such solve: the second waits until the first retires
    with fd.Server(need + 4096, max_active=4) as srv:
        srv.submit(big)
        srv.submit(dict(big, tag=11))
        assert srv.tick() == 1
        assert srv.stats()["queued"] == 1
        srv.tick()                      # tag 10 finishes (2 steps) and frees its block
        done = [r["tag"] for r in srv.poll()]
        assert done == [10]
        assert srv.tick() == 1          # tag 11 admitted now
        srv.tick()
        assert [r["tag"] for r in srv.poll()] == [11]
        assert srv.stats()["arena_used"] > 0   # 11's state is kept until the next tick
        srv.tick()
        assert srv.stats()["arena_used"] == 0


def test_too_large_request_is_refused_and_cancel_works():
    with fd.Server(1 << 20, max_active=4) as srv:
        with pytest.raises(fd.FdError) as e:
            srv.submit(dict(tag=1, n=64, steps=1, dtype="f64"))
        assert e.value.code == fd.FD_EBUSY
        srv.submit(dict(tag=2, n=8, steps=50, dtype="f32"))
        srv.submit(dict(tag=3, n=8, steps=1, dtype="f32"))
        srv.cancel(3)
        srv.tick()
        srv.cancel(2)
        srv.tick()
        res = {r["tag"]: r for r in srv.poll()}
        assert res[3]["status"] == fd.FD_EBUSY and res[3]["steps"] == 0
        assert res[2]["status"] == fd.FD_EBUSY and res[2]["steps"] == 1
        with pytest.raises(fd.FdError):
            srv.cancel(99)


def test_tma_and_thread_staged_binary32_solves_share_a_tick():
    """Binary32 recompute-all solves whose x extent is a multiple of 4 are staged by
    TMA (ghost-padded fields), the others by threads; both kinds advance in the same
    ticks, join and leave at different times, and each equals its solve alone."""
    reqs = [
        dict(tag=21, n=(18, 20, 22), steps=6, Re=1600.0, Mach=0.1, dtype="f32", algorithm="recompute_all", dt=1e-3),
        dict(tag=22, n=(32, 24, 40), steps=4, Re=900.0, Mach=0.2, dtype="f32", algorithm="recompute_all", dt=1e-3),
        dict(tag=23, n=(21, 16, 16), steps=3, Re=2500.0, Mach=0.3, dtype="f32", algorithm="recompute_all", dt=2e-3),
        dict(tag=24, n=(64, 8, 72), steps=5, Re=1200.0, Mach=0.15, dtype="f32", algorithm="recompute_all", dt=1e-3),
    ]
    got = {}
    with fd.Server(1 << 30, max_active=8) as srv:
        srv.submit(reqs[0])
        srv.submit(reqs[1])
        srv.tick()
        srv.submit(reqs[2])
        srv.tick()
        srv.submit(reqs[3])
        for _ in range(40):
            srv.tick()
            for r in srv.poll():
                got[r["tag"]] = r
            if len(got) == len(reqs):
                break
    assert set(got) == {r["tag"] for r in reqs}
    for r in reqs:
        ke, en = alone(r)
        assert got[r["tag"]]["status"] == fd.FD_OK
        assert got[r["tag"]]["ke"] == ke and got[r["tag"]]["enstrophy"] == en, r["tag"]


def test_served_states_match_the_oracle_and_alone():
    """Solves join and leave a running mix; each final state is read through
    fd_server_get_state after its result is polled (before the next tick), and
    checked against the oracle's run of the same request (binary64 requests to
    1e-12 in relative L-inf, binary32 requests to 1e-5 in relative L2) and
    against the same solve run alone (bit for bit)."""
    reqs = [
        dict(tag=31, n=(12, 10, 14), steps=4, Re=800.0, Mach=0.2, dtype="f64", algorithm="store_some", dt=1e-3),
        dict(tag=32, n=16, steps=6, Re=1600.0, Mach=0.1, dtype="f64", algorithm="recompute_all", dt=1e-3),
        dict(tag=33, n=(16, 12, 20), steps=5, Re=2000.0, Mach=0.3, dtype="f32", algorithm="recompute_all", dt=1e-3),
        dict(tag=34, n=(10, 14, 12), steps=3, Re=1200.0, Mach=0.25, dtype="f32", algorithm="store_some", dt=2e-3),
        dict(tag=35, n=(20, 8, 16), steps=7, Re=3000.0, Mach=0.15, dtype="f64", algorithm="store_some", dt=1e-3),
        dict(tag=36, n=(14, 16, 12), steps=5, Re=1600.0, Mach=0.1, dtype="f64dw", algorithm="store_some", dt=1e-3),
        dict(tag=37, n=18, steps=3, Re=900.0, Mach=0.3, dtype="f64dw", algorithm="store_some", dt=2e-3),
    ]
    by_tag = {r["tag"]: r for r in reqs}
    states, results = {}, {}
    with fd.Server(1 << 30, max_active=8) as srv:
        srv.submit(reqs[0])
        srv.submit(reqs[2])
        srv.tick()
        srv.submit(reqs[1])
        srv.tick()
        srv.submit(reqs[3])
        srv.submit(reqs[4])
        srv.submit(reqs[5])
        srv.tick()
        srv.submit(reqs[6])
        for _ in range(40):
            srv.tick()
            for r in srv.poll():
                results[r["tag"]] = r
                states[r["tag"]] = srv.state(r["tag"], by_tag[r["tag"]]["n"])
            if len(results) == len(reqs):
                break
        with pytest.raises(fd.FdError) as e:
            srv.state(999, 8)
        assert e.value.code == fd.FD_EINVAL
    assert set(states) == set(by_tag)
    for tag, r in by_tag.items():
        assert results[tag]["status"] == fd.FD_OK and results[tag]["steps"] == r["steps"]
        Q = states[tag]
        n = r["n"]
        nx, ny, nz = (n, n, n) if isinstance(n, int) else n
        ref = O.run(O.tgv_ic(nx, ny, nz, 1.4, r["Mach"]), r["steps"], dt=r["dt"], Re=r["Re"], Mach=r["Mach"])
        if r["dtype"] in ("f64", "f64dw"):
            err = max(np.abs(Q[v] - ref[v]).max() / np.abs(ref[v]).max() for v in range(5))
            assert err <= 1e-12, tag
        else:  # the binary32 mode's bound: relative L2 of each variable <= 1e-5
            err = max(np.linalg.norm(Q[v] - ref[v]) / np.linalg.norm(ref[v]) for v in range(5))
            assert err <= 1e-5, tag
        with fd.Solver(r["n"], Re=r["Re"], Mach=r["Mach"], dt=r["dt"], algorithm=r["algorithm"],
                       dtype=r["dtype"]) as s:
            s.step(r["steps"])
            assert np.array_equal(s.state(), Q), tag
