"""The tensor-core source stage (a2 for kernels that mix groups: the
Klein-Nishina multigroup kernel, Sec. 2.3 eq:comptoncross) in the mixed
precision against the FP64 oracle: whole steps, with the step's sums, at
group counts that fill the MMA's N and K exactly (32) and that leave padding
(21), at L = 7 (eight nodes per tile, up to 120 of 128 rows) and L = 3."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_05141_gb300 import inputs

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-4


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_05141_gb300 import native
    return native


@pytest.mark.parametrize("G,L", [(32, 7), (21, 3), (8, 7)])
def test_kn_steps_mixed_tensor_core_source(native, G, L):
    spec = inputs.ragged_mixed(grid=(12, 8, 6), G=G, L=L, scattering="kn")
    spec.edges = np.geomspace(1e-3, 1e1, G + 1)  # energies up to 10 m_e c^2: strong down-scattering
    K, so = O.kn_table(spec.edges, spec.L)
    P = O.OracleProblem(grid=spec.grid, L=spec.L, nmu=spec.nmu, nphi=spec.nphi, edges=spec.edges,
                        alpha0=spec.alpha0, ne=spec.ne, u=spec.u, emis0=spec.emis0, K=K, sigma_out=so,
                        kappa=spec.kappa, box=spec.box)
    s = native.Solver.from_spec(spec, precision="mixed")
    s.set_source_path("tensor")
    assert s.source_path()[0] == 2
    I0 = inputs.random_state(spec, seed=9)
    s.set_state(I0)
    s.step(2)
    J, H, Kt, Ish = s.moments(with_sh=True)
    e_g, p_g, r_g = s.sums()
    I_ref, _, sums = P.step(I0, 2)
    Ish_r, J_r, H_r, K_r = P.project(I_ref)
    assert float(np.max(np.abs(J - J_r) / np.abs(J_r))) < MIXED_TOL
    assert float(np.max(np.abs(Ish - Ish_r)) / np.max(np.abs(Ish_r))) < MIXED_TOL
    f, f_r = O.moments_to_eddington(J, Kt), O.moments_to_eddington(J_r, K_r)
    assert float(np.max(np.abs(f - f_r))) < MIXED_TOL
    assert abs(e_g - sums[0]) <= MIXED_TOL * abs(sums[0])
    assert abs(p_g - sums[1]) <= MIXED_TOL * abs(sums[1])
    assert abs(r_g - sums[2]) <= 1e-3 * abs(sums[2]) + 1e-7
    s.close()


def test_source_path_timed_choice(native):
    """The default times both source passes on the first step and keeps the
    faster; both give the same step to within the mixed tolerance."""
    spec = inputs.ragged_mixed(grid=(16, 8, 6), G=16, L=7, scattering="kn")
    I0 = inputs.random_state(spec, seed=4)
    out = {}
    for path in ("auto", "cuda", "tensor"):
        s = native.Solver.from_spec(spec, precision="mixed")
        s.set_source_path(path)
        s.set_state(I0)
        s.step(2)
        out[path] = s.get_state()
        p, ms_cc, ms_tc = s.source_path()
        if path == "auto":
            assert p in (1, 2) and ms_cc > 0 and ms_tc > 0
            assert p == (2 if ms_tc < ms_cc else 1)
        s.close()
    scale = np.max(np.abs(out["cuda"]))
    assert float(np.max(np.abs(out["tensor"] - out["cuda"]))) < 1e-5 * scale
    s = native.Solver.from_spec(inputs.ragged_mixed(), precision="mixed")  # Thomson: diagonal, CUDA cores only
    with pytest.raises(native.ShdError):
        s.set_source_path("tensor")
    s.close()
