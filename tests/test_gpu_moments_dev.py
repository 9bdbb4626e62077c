"""shd_get_moments_dev: the moments of the current state (Sec. 2, the
projection of stage a1) into caller-owned device memory, bit-identical to
what shd_get_moments returns to the host, on the context's stream and on a
caller's stream."""
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


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_moments_dev_equals_host_moments(native, precision):
    import torch
    spec = inputs.jet(n=12, G=3, L=3, tau_r=3.0, gmax=4.0)
    s = native.Solver.from_spec(spec, precision=precision)
    s.set_state(inputs.random_state(spec, seed=17))
    s.step(2)
    mom = torch.full((s.Nc, s.G, 10), float("nan"), dtype=torch.float64, device="cuda")
    s.moments_dev(mom)
    torch.cuda.synchronize()
    J, H, K = s.moments()
    m = mom.cpu().numpy()
    assert np.array_equal(m[..., 0], J)
    assert np.array_equal(m[..., 1:4], H)
    assert np.array_equal(m[..., 4:10], K)
    # on a caller's stream, after one more step on it
    st = torch.cuda.Stream()
    s.step(1, st.cuda_stream)
    mom2 = torch.zeros_like(mom)
    s.moments_dev(mom2, st.cuda_stream)
    st.synchronize()
    J2, _, _ = s.moments()
    assert np.array_equal(mom2.cpu().numpy()[..., 0], J2)
    assert not np.array_equal(J2, J)
    with pytest.raises(ValueError):
        s.moments_dev(mom.float())
    s.close()
