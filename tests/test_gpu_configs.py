"""The other workload recipes at oracle-sized resolution, element by element
against the FP64 oracle: the Klein-Nishina Compton shell, the Gamma = 30 jet
in a cocoon (FP64 Doppler factors above Gamma = 10 on the mixed path) and a
batch of independent random problems stepped as one batch."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_05141_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_TOL = 1e-4


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_05141_gb300 import native
    return native


def _oracle(spec):
    if spec.scattering == "kn":
        K, so = O.kn_table(spec.edges, spec.L)
    elif spec.scattering == "thomson":
        K, so = O.thomson_table(spec.G, spec.L)
    else:
        K, so = O.iso_table(spec.G, spec.L)
    return O.OracleProblem(grid=spec.grid, L=spec.L, nmu=spec.nmu, nphi=spec.nphi, edges=spec.edges,
                           alpha0=spec.alpha0, ne=spec.ne, u=spec.u, emis0=spec.emis0, K=K, sigma_out=so,
                           kappa=spec.kappa, box=spec.box)


def _check(s, spec, I0, nsteps, tol, oracle=None):
    P = oracle or _oracle(spec)
    I_ref, _, sums = P.step(I0, nsteps)
    _, J_r, H_r, K_r = P.project(I_ref)
    J, H, K = s.moments()
    scale = np.max(np.abs(J_r))
    assert np.max(np.abs(J - J_r) / np.maximum(np.abs(J_r), 1e-12 * scale)) < tol
    assert np.max(np.abs(H - H_r)) / np.max(np.abs(H_r)) < tol
    f = O.moments_to_eddington(J, K)
    assert np.max(np.abs(f - O.moments_to_eddington(J_r, K_r))) < tol
    e_g, p_g, _ = s.sums()
    assert abs(e_g - sums[0]) <= tol * abs(sums[0])
    assert abs(p_g - sums[1]) <= tol * abs(sums[1])


@pytest.mark.parametrize("precision,tol,nsteps", [("fp64", FP64_TOL, 2), ("mixed", MIXED_TOL, 1)])
def test_compton_shell(native, precision, tol, nsteps):
    spec = inputs.compton_shell(n=12, G=6, L=3)
    s = native.Solver.from_spec(spec, precision=precision)
    I0 = inputs.random_state(spec, seed=41)
    s.set_state(I0)
    s.step(nsteps)
    _check(s, spec, I0, nsteps, tol)


@pytest.mark.parametrize("precision,tol,nsteps", [("fp64", FP64_TOL, 2), ("mixed", MIXED_TOL, 1)])
def test_jet_cocoon_gamma30(native, precision, tol, nsteps):
    spec = inputs.jet_cocoon(n=12, G=6, L=3)
    s = native.Solver.from_spec(spec, precision=precision)
    I0 = inputs.random_state(spec, seed=42)
    s.set_state(I0)
    s.step(nsteps)
    _check(s, spec, I0, nsteps, tol)


@pytest.mark.parametrize("precision,tol", [("fp64", FP64_TOL), ("mixed", MIXED_TOL)])
def test_batch_of_random_problems(native, precision, tol):
    specs = [inputs.batch_problem(i, n_range=(8, 14), g_range=(3, 6), Ls=(3,)) for i in range(4)]
    solvers, states = [], []
    for i, spec in enumerate(specs):
        s = native.Solver.from_spec(spec, precision=precision)
        I0 = inputs.random_state(spec, seed=50 + i)
        s.set_state(I0)
        solvers.append(s)
        states.append(I0)
    b = native.Batch(solvers)
    b.step(2)
    for s, spec, I0 in zip(solvers, specs, states):
        _check(s, spec, I0, 2, tol)
    b.close()
