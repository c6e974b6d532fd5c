"""The FP64 local solve of the sweeps (FP32 estimate, one Newton step whose
residual is evaluated with error-free FP32 transformations) against the
direct FP64 closed forms of Eq. 2, on 16 M device-generated inputs that
cover the one-, two- and three-term cases."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eik():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1306_4743_gb300 import eik as e
    e.load()
    return e


@pytest.mark.parametrize("seed", [1, 2])
def test_sweep_local_solve_matches_direct_fp64(eik, seed):
    ulps, norm = eik.selftest_local_solve(count=1 << 24, seed=seed)
    # within a few units of (ulp(U) + 2^-44 s): a few ulps of U except where
    # U is not much larger than the local step s (near an exit), where the
    # FP32-pair residual of the Newton step sets the floor
    assert norm <= 4.0, (norm, ulps)
