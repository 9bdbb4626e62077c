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
