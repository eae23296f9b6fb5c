"""fd_residual_noalloc: the store-some residual without any allocation, checked
against fd_residual (which works through a handle) and against the oracle's
residual on the same states.

The entry point is for callers that cannot allocate device memory when they need
R(Q) (an external integrator inside a stream capture or a fixed memory budget);
its scratch is a fixed array inside the library shared by all calls.  Two calls
in a row on different states must each match fd_residual, so nothing left in
the shared scratch by one call can leak into the next.
"""
import numpy as np
import pytest

import oracle as O
from tests.inputs import rough_state, smooth_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1610_09146_gb300 as fd  # noqa: E402
from paper_1610_09146_gb300 import native  # noqa: E402

RE, MACH, PR, GAMMA = 1600.0, 0.1, 0.71, 1.4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    fd.build()


def rel_linf(a, b):
    return max(np.abs(a[v] - b[v]).max() / max(np.abs(b[v]).max(), 1e-300) for v in range(5))


def reference_residual(Q0):
    nz, ny, nx = Q0.shape[1:]
    with fd.Solver((nx, ny, nz), Re=RE, Mach=MACH, Pr=PR, gamma=GAMMA, dt=1e-3, algorithm="store_some",
                   dtype="f64") as s:
        s.set_state(Q0)
        return s.residual()


def noalloc_residual(Q0, stream):
    nz, ny, nx = Q0.shape[1:]
    Qd = torch.from_numpy(Q0).to("cuda")
    Rd = torch.full_like(Qd, float("nan"))
    rc = native.fd_residual_noalloc(Qd.data_ptr(), Rd.data_ptr(), nx, ny, nz, RE, MACH, PR, GAMMA,
                                    stream.cuda_stream)
    assert rc == fd.FD_OK
    stream.synchronize()
    return Rd.cpu().numpy()


def test_two_calls_in_a_row_match_fd_residual():
    stream = torch.cuda.current_stream()
    Qa = smooth_state((24, 20, 28), seed=31)   # nz, ny, nx: ragged sizes
    Qb = rough_state((24, 20, 28), seed=32)
    Ra_ref, Rb_ref = reference_residual(Qa), reference_residual(Qb)
    Ra = noalloc_residual(Qa, stream)
    Rb = noalloc_residual(Qb, stream)
    assert rel_linf(Ra, Ra_ref) <= 1e-12
    assert rel_linf(Rb, Rb_ref) <= 1e-12
    assert rel_linf(Ra, O.residual(Qa, Re=RE, Mach=MACH, Pr=PR, gamma=GAMMA)) <= 1e-12
    assert rel_linf(Rb, O.residual(Qb, Re=RE, Mach=MACH, Pr=PR, gamma=GAMMA)) <= 1e-12


def test_largest_allowed_grid_then_a_small_one():
    stream = torch.cuda.current_stream()
    n = 64  # 64^3 = FD_NOALLOC_MAX_POINTS
    Qa = smooth_state((n, n, n), seed=41)
    Qb = smooth_state((8, 9, 10), seed=42)
    Ra = noalloc_residual(Qa, stream)
    Rb = noalloc_residual(Qb, stream)
    assert rel_linf(Ra, reference_residual(Qa)) <= 1e-12
    assert rel_linf(Rb, reference_residual(Qb)) <= 1e-12
    assert rel_linf(Ra, O.residual(Qa, Re=RE, Mach=MACH, Pr=PR, gamma=GAMMA)) <= 1e-12
    assert rel_linf(Rb, O.residual(Qb, Re=RE, Mach=MACH, Pr=PR, gamma=GAMMA)) <= 1e-12


def test_sizes_beyond_the_scratch_are_rejected():
    Q = torch.zeros(5 * 65 * 64 * 64, dtype=torch.float64, device="cuda")
    R = torch.zeros_like(Q)
    assert native.fd_residual_noalloc(Q.data_ptr(), R.data_ptr(), 65, 64, 64, RE, MACH, PR, GAMMA, 0) == fd.FD_EINVAL
    assert native.fd_residual_noalloc(Q.data_ptr(), R.data_ptr(), 4, 64, 64, RE, MACH, PR, GAMMA, 0) == fd.FD_EINVAL
    assert native.fd_residual_noalloc(0, R.data_ptr(), 8, 8, 8, RE, MACH, PR, GAMMA, 0) == fd.FD_EINVAL
    assert native.FD_NOALLOC_MAX_POINTS == 64**3
