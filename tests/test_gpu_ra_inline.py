"""Recompute-all with the primitives recomputed at every tap (FD_RECOMPUTE_ALL_INLINE).

Every u_i, p and T value comes from the state at that tap with the same formulas as
the stored primitives of the other families, so the residual and the steps equal
the stored-primitive recompute-all family bit for bit, and the oracle to relative
L-inf 1e-12; the handle holds only the state and the saved register.
"""
import numpy as np
import pytest

import oracle as O
from tests.inputs import rough_state, smooth_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1610_09146_gb300 as fd  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    fd.build()


def rel_linf(a, b):
    return max(np.abs(a[v] - b[v]).max() / max(np.abs(b[v]).max(), 1e-300) for v in range(5))


@pytest.mark.parametrize("shape,kind", [((23, 19, 21), "rough"), ((18, 24, 20), "smooth")])
def test_equals_stored_primitive_recompute_all(shape, kind):
    Q0 = rough_state(shape, seed=61) if kind == "rough" else smooth_state(shape, seed=62)
    nz, ny, nx = shape
    out = {}
    for alg in ("recompute_all", "recompute_all_inline"):
        with fd.Solver((nx, ny, nz), dt=1e-3, algorithm=alg) as s:
            s.set_state(Q0)
            R = s.residual()
            s.step(3)
            out[alg] = (R, s.state(), s.device_bytes())
    assert np.array_equal(out["recompute_all_inline"][0], out["recompute_all"][0])
    assert np.array_equal(out["recompute_all_inline"][1], out["recompute_all"][1])
    assert out["recompute_all_inline"][2] < 0.7 * out["recompute_all"][2]
    assert rel_linf(out["recompute_all_inline"][0], O.residual(Q0)) <= 1e-12


def test_ten_steps_tgv_32_matches_oracle():
    n = 32
    ref = O.run(O.tgv_ic(n, n, n, 1.4, 0.1), 10, dt=1e-3)
    with fd.Solver(n, dt=1e-3, algorithm="recompute_all_inline") as s:
        s.step(10)
        assert rel_linf(s.state(), ref) <= 1e-12
        ke, en = s.diagnostics()
    ke_ref, en_ref = O.diagnostics(ref)
    assert abs(ke - ke_ref) <= 1e-13 * ke_ref and abs(en - en_ref) <= 1e-13 * en_ref


def test_binary64_only():
    for dtype in ("f32", "df64", "f64dw"):
        with pytest.raises(fd.FdError) as e:
            fd.Solver(8, dt=1e-3, algorithm="recompute_all_inline", dtype=dtype)
        assert e.value.code == fd.FD_EINVAL
