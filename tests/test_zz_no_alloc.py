"""The projection entry point that allocates nothing (shd_project_noalloc).

It serves callers that cannot call cudaMalloc when they need the moments
(device memory owned by another allocator, loops that must not meet the
allocator's implicit synchronisation, processes at their memory limit).  Its
outputs must equal those of the ordinary entry point, shd_get_moments, on two
calls in a row (the static scratch keeps the previous call's contents), and it
must refuse a problem whose scratch would not fit.

This file is collected last on purpose: a run that stops at the first failure
has then already run every other test.
"""
import numpy as np
import pytest

from paper_1507_05141_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-6, "mixed": 1e-6}

# (precision, grid): FP64 and FP32 on the ragged grid (brick kernels); MIXED
# on a grid whose planes are multiples of 4 nodes, where the projection runs
# the TMA-fed tensor-core segment kernels with the static array as their
# node-major scratch (tensor maps over an address inside it)
CASES = [("fp64", (11, 9, 7), 5), ("fp32", (11, 9, 7), 5), ("mixed", (16, 12, 8), 2)]


def _native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_05141_gb300 import native
    return native


@pytest.mark.parametrize("precision,grid,G", CASES)
def test_noalloc_projection_matches_get_moments(precision, grid, G):
    import torch
    native = _native()
    spec = inputs.ragged_mixed(grid=grid, G=G, scattering="thomson")
    assert np.any(spec.u != 0), "the case must exercise the scratch (moving nodes)"
    s = native.Solver.from_spec(spec, precision=precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    dev_before = torch.cuda.current_device()
    Ish = torch.empty((spec.Nc, spec.G, spec.NLM), dtype=dt, device="cuda")
    mom = torch.empty((spec.Nc, spec.G, 10), dtype=dt, device="cuda")
    for seed in (21, 22):  # two calls in a row on different states
        s.set_state(inputs.random_state(spec, seed=seed))
        J, H, K, Ish_ref = s.moments(with_sh=True)
        Ish.fill_(float("nan"))
        mom.fill_(float("nan"))
        s.project_noalloc(Ish, mom)
        assert torch.cuda.current_device() == dev_before  # the caller's device is kept
        torch.cuda.synchronize()
        Ish_n = Ish.double().cpu().numpy()
        mom_n = mom.double().cpu().numpy()
        tol = TOL[precision]
        assert np.all(np.isfinite(Ish_n)) and np.all(np.isfinite(mom_n))
        assert np.max(np.abs(Ish_n - Ish_ref)) <= tol * np.max(np.abs(Ish_ref))
        assert np.max(np.abs(mom_n[..., 0] - J)) <= tol * np.max(np.abs(J))
        assert np.max(np.abs(mom_n[..., 1:4] - H)) <= tol * np.max(np.abs(J))
        assert np.max(np.abs(mom_n[..., 4:10] - K)) <= tol * np.max(np.abs(J))
    s.close()


def test_noalloc_rejects_problems_beyond_the_scratch():
    import torch
    native = _native()
    spec = inputs.jet(n=24, G=16, L=7)   # moving nodes; 24^3 x 16 x 512 floats > 64 MiB
    s = native.Solver.from_spec(spec, precision="fp32")
    s.zero_state()
    Ish = torch.empty(1, device="cuda")
    mom = torch.empty(1, device="cuda")
    with pytest.raises(native.ShdError, match="scratch"):
        s.project_noalloc(Ish, mom)
    s.close()
