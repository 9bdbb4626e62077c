"""The cubic Bezier short characteristic (Sec. 2) on the GPU against the
FP64 oracle's Bezier sweep, through the C ABI: the sweep stage alone on
random inputs, whole steps in FP64 (1e-10), FP32 and MIXED, and the size
limit of the Bezier kernel."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_05141_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-5, "mixed": 1e-4}


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_05141_gb300 import native
    return native


def _oracle(spec):
    K, so = O.thomson_table(spec.G, spec.L) if spec.scattering == "thomson" else O.kn_table(spec.edges, spec.L)
    P = O.OracleProblem(grid=spec.grid, L=spec.L, nmu=spec.nmu, nphi=spec.nphi, edges=spec.edges,
                        alpha0=spec.alpha0, ne=spec.ne, u=spec.u, emis0=spec.emis0, K=K, sigma_out=so,
                        kappa=spec.kappa, box=spec.box)
    P.set_integrator("bezier")
    return P


def _rel_cols(a, b):
    return float(np.max(np.abs(a - b) / np.max(np.abs(b), axis=0, keepdims=True)))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_bezier_sweep_stage(native, precision):
    spec = inputs.ragged_mixed(scattering="thomson")
    P = _oracle(spec)
    s = native.Solver.from_spec(spec, precision=precision)
    s.set_integrator("bezier")
    rng = np.random.default_rng(17)
    I = inputs.random_state(spec, seed=3)
    eta = rng.random(I.shape) * 3.0
    chi = rng.random(I.shape) * 20.0 + 1e-3
    out = s.stage_sweep(I, eta, chi)
    ref = P.sweep(I, eta, chi)
    assert _rel_cols(out, ref) < TOL[precision]
    s.close()


@pytest.mark.parametrize("precision,kind", [("fp64", "thomson"), ("fp64", "kn"), ("fp32", "thomson"),
                                            ("mixed", "thomson")])
def test_bezier_steps(native, precision, kind):
    spec = inputs.ragged_mixed(scattering=kind) if precision != "mixed" else \
        inputs.jet(n=16, G=4, L=3, tau_r=4.0, gmax=4.0)
    P = _oracle(spec)
    s = native.Solver.from_spec(spec, precision=precision)
    s.set_integrator("bezier")
    I0 = inputs.random_state(spec, seed=5)
    s.set_state(I0)
    s.step(3)  # the second and third steps replay the captured step
    I = s.get_state()
    J, H, K = s.moments()
    I_ref, _, _ = P.step(I0, 3)
    _, J_r, H_r, K_r = P.project(I_ref)
    assert _rel_cols(I, I_ref) < TOL[precision]
    f, f_r = O.moments_to_eddington(J, K), O.moments_to_eddington(J_r, K_r)
    assert float(np.max(np.abs(f - f_r))) < TOL[precision]
    # the Bezier scheme differs from the linear one (the switch is live)
    s.set_integrator("linear")
    s.set_state(I0)
    s.step(3)
    assert float(np.max(np.abs(s.get_state() - I))) > 1e-6 * float(np.max(np.abs(I)))
    s.close()


def test_bezier_plane_limit(native):
    spec = inputs.ragged_mixed(grid=(64, 64, 4), G=1, L=1)
    s = native.Solver.from_spec(spec, precision="fp64")
    s.set_integrator("bezier")
    s.zero_state()
    with pytest.raises(native.ShdError, match="Bezier"):
        s.step(1)
    s.close()
