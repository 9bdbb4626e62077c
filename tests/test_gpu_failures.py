"""Failure paths through the C ABI: argument checks of the setters and the
bounded-wait failure path of the tensor-core kernels.  Nothing here faults,
traps or hangs the GPU: the refused calls are refused on the host before any
GPU work, and the wait check waits (a bounded number of polls) on an mbarrier
that nothing arrives on, with no copy or MMA in flight."""
import numpy as np
import pytest

from paper_1507_05141_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_05141_gb300 import native
    return native


def _code(native, fn, *a):
    with pytest.raises(native.ShdError) as ei:
        fn(*a)
    return ei.value.code


def test_bad_angles_groups_grid(native):
    s = native.Solver(0, "fp32")
    # discrete orthogonality needs n_mu >= L+1 and n_phi >= 2L+1
    assert _code(native, s.set_angles, 3, 3, 16) == native.ERR_ARG
    assert _code(native, s.set_angles, 3, 8, 6) == native.ERR_ARG
    assert _code(native, s.set_angles, 10, 22, 44) == native.ERR_ARG
    assert _code(native, s.set_angles, 3, 64, 128) == native.ERR_ARG  # more than 4096 ordinates
    # groups: G >= 1, edges positive, finite and strictly ascending
    assert _code(native, s.set_groups, np.array([1.0])) == native.ERR_ARG
    assert _code(native, s.set_groups, np.array([1.0, 0.5, 2.0])) == native.ERR_ARG
    assert _code(native, s.set_groups, np.array([0.0, 1.0])) == native.ERR_ARG
    assert _code(native, s.set_groups, np.array([1.0, 1.0])) == native.ERR_ARG
    assert _code(native, s.set_groups, np.array([1.0, np.inf])) == native.ERR_ARG
    # grid: every dimension >= 2, positive finite box
    assert _code(native, s.set_grid, 1, 4, 4) == native.ERR_ARG
    assert _code(native, s.set_grid, 4, 4, 4, 1.0, -1.0, 1.0) == native.ERR_ARG
    assert _code(native, s.set_time, -1.0) == native.ERR_ARG
    # call order: stepping an unconfigured context is refused
    assert _code(native, s.step, 1) in (native.ERR_STATE, native.ERR_ARG)
    s.close()


def test_fields_before_grid_refused(native):
    s = native.Solver(0, "fp64")
    spec = inputs.ragged_mixed()
    assert _code(native, s.set_fields, spec.alpha0, spec.ne, spec.u, spec.emis0) == native.ERR_STATE
    s.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_bounded_wait_gives_up_and_reports(native, precision):
    """The wait runs out, the flag is raised, the call returns SHD_ERR_TIMEOUT
    and clears it; the context stays usable (a later step and its sums are
    bit-identical to those of a context that never ran the check)."""
    spec = inputs.ragged_mixed(grid=(12, 8, 6), G=2)
    s = native.Solver.from_spec(spec, precision=precision)
    ref = native.Solver.from_spec(spec, precision=precision)
    rc, msg = s.check_bounded_wait(1000)
    assert rc == native.ERR_TIMEOUT
    assert "bounded wait" in msg
    rc, _ = s.check_bounded_wait(1000)  # the flag was cleared: the check runs again
    assert rc == native.ERR_TIMEOUT
    I0 = inputs.random_state(spec, seed=2)
    for x in (s, ref):
        x.set_state(I0)
        x.step(2)
    assert s.sums() == ref.sums()
    assert np.array_equal(s.get_state(), ref.get_state())
    s.close()
    ref.close()


def test_bounded_wait_limits_checked(native):
    s = native.Solver(0, "fp32")
    assert s.check_bounded_wait(0)[0] == native.ERR_ARG
    assert s.check_bounded_wait((1 << 22) + 1)[0] == native.ERR_ARG
    s.close()
