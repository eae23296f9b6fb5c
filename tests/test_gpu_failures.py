"""Failure handling without faulting the GPU: failures are made on the host.

An allocator callback that returns NULL stands for an out-of-memory device; the
library must return FD_ENOMEM with a message, leave nothing allocated, and stay
usable.  Malformed arguments return FD_EINVAL before any launch.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1610_09146_gb300 as fd  # noqa: E402
from paper_1610_09146_gb300 import native  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    fd.build()


class CountingAlloc:
    """Device allocator that fails after `budget` successful calls and counts frees."""

    def __init__(self, budget):
        self.budget = budget
        self.live = {}
        self.calls = 0

        def _alloc(ctx, nbytes, stream):
            self.calls += 1
            if self.budget <= 0:
                return None
            self.budget -= 1
            p = torch.cuda.caching_allocator_alloc(int(nbytes))
            self.live[p] = nbytes
            return p

        def _free(ctx, ptr, nbytes, stream):
            assert self.live.pop(int(ptr)) == nbytes
            torch.cuda.caching_allocator_delete(int(ptr))

        self.struct = native.FdAlloc(native.ALLOC_FN(_alloc), native.FREE_FN(_free), None)


def test_create_reports_out_of_memory():
    a = CountingAlloc(0)
    with pytest.raises(fd.FdError) as e:
        native.fd_create(16, 16, 16, 1600.0, 0.1, 0.71, 1.4, 1e-3, fd.FD_STORE_SOME, fd.FD_F64, a.struct, 0)
    assert e.value.code == fd.FD_ENOMEM
    assert "allocator returned NULL" in fd.fd_last_error(None)
    assert a.calls == 1 and not a.live
    # the library is still usable afterwards
    with fd.Solver(16, dt=1e-3) as s:
        s.step(1)
        assert s.check_finite()


def test_batch_reports_out_of_memory_and_frees_everything():
    a = CountingAlloc(0)
    d = native.FdInstanceDesc(16, 16, 16, 1600.0, 0.1, 0.71, 1.4, 1e-3, fd.FD_RECOMPUTE_ALL, 0)
    with pytest.raises(fd.FdError) as e:
        native.fd_batch_create([d], fd.FD_F32_ACCDW, a.struct, 0)
    assert e.value.code == fd.FD_ENOMEM and not a.live


def test_server_arena_failure_and_table_growth_failure():
    # arena allocation fails
    a = CountingAlloc(0)
    with pytest.raises(fd.FdError) as e:
        native.fd_server_create(1 << 24, 4, a.struct, 0)
    assert e.value.code == fd.FD_ENOMEM and not a.live
    # arena and fixed buffers succeed, the instance-table buffer of the first tick does not
    a = CountingAlloc(2)
    srv = native.fd_server_create(1 << 24, 4, a.struct, 0)
    native.fd_server_submit(srv, fd.Server.request(dict(n=8, steps=1, dtype="f32", tag=7)))
    with pytest.raises(fd.FdError) as e:
        native.fd_server_tick(srv)
    assert e.value.code == fd.FD_ECUDA
    native.fd_server_destroy(srv)
    assert not a.live


def test_malformed_requests_are_rejected_before_any_launch():
    with fd.Server(1 << 24, max_active=2) as srv:
        for bad in (dict(n=4, steps=1), dict(n=8, steps=0), dict(n=8, steps=1, Re=-1.0),
                    dict(n=8, steps=1, algorithm="store_all"), dict(n=8, steps=1, tile_points=3)):
            with pytest.raises(fd.FdError) as e:
                srv.submit(bad)
            assert e.value.code == fd.FD_EINVAL
        assert srv.stats()["queued"] == 0
    with fd.Solver(8, dt=1e-3) as s:
        Q = s.state()
        with pytest.raises(fd.FdError):
            fd.fd_set_state(s.h, np.zeros(3))
        assert np.array_equal(s.state(), Q)


def test_kernel_wait_that_runs_out_is_reported_and_the_context_survives():
    """A wait inside the TMA-staged kernel that never completes (the copy of one
    plane is left out on purpose) gives up after 0.5 s, records it in the
    kernel's error word and ends the block; nothing faults or hangs, and the
    device stays usable for the next solver."""
    import os
    import time
    if os.environ.get("FDGB300_NO_TMA") == "1":
        pytest.skip("TMA staging turned off")
    t0 = time.perf_counter()
    word = native.fd_selftest_wait_timeout()
    elapsed = time.perf_counter() - t0
    assert word == 1
    assert elapsed < 30.0
    with fd.Solver(32, algorithm="recompute_all", dtype="f32") as s:
        s.step(2)
        assert s.check_finite()
        assert np.isfinite(s.diagnostics()[0])
