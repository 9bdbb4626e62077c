"""Runge-Kutta sub-stepping of the time step (App. A, eq:rk4th) and Ng
acceleration of the static Lambda iteration (Sec. 2) on the GPU against the
FP64 oracle, through the C ABI.

RK4 steps start from a zero state (the field builds up smoothly from the
emission): the printed combination amplifies components that a sub-solve
damps completely (by up to 9 per step), so a random grid-scale initial state
would magnify rounding differences step by step."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_05141_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
TOL = {"fp64": 1e-10, "fp32": 2e-5, "mixed": 1e-4}


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_05141_gb300 import native
    return native


def _oracle(spec, kind=None):
    kind = kind or spec.scattering
    K, so = {"thomson": lambda: O.thomson_table(spec.G, spec.L), "iso": lambda: O.iso_table(spec.G, spec.L),
             "kn": lambda: O.kn_table(spec.edges, spec.L)}[kind]()
    return O.OracleProblem(grid=spec.grid, L=spec.L, nmu=spec.nmu, nphi=spec.nphi, edges=spec.edges,
                           alpha0=spec.alpha0, ne=spec.ne, u=spec.u, emis0=spec.emis0, K=K, sigma_out=so,
                           kappa=spec.kappa, box=spec.box)


def _rel_elem(a, b, floor_frac=1e-12):
    b = np.asarray(b)
    den = np.maximum(np.abs(b), floor_frac * np.max(np.abs(b)))
    return float(np.max(np.abs(np.asarray(a) - b) / den))


@pytest.mark.parametrize("precision,spec_name", [("fp64", "ragged_thomson"), ("fp64", "ragged_kn"),
                                                 ("mixed", "jet16"), ("fp32", "ragged_thomson")])
def test_rk4_steps(native, precision, spec_name):
    spec = {"ragged_thomson": lambda: inputs.ragged_mixed(scattering="thomson"),
            "ragged_kn": lambda: inputs.ragged_mixed(scattering="kn"),
            "jet16": lambda: inputs.jet(n=16, G=4, L=3, tau_r=4.0, gmax=4.0)}[spec_name]()
    tol = TOL[precision]
    P = _oracle(spec)
    s = native.Solver.from_spec(spec, precision=precision)
    s.set_time_scheme("rk4")
    s.zero_state()
    s.step(3)   # the first step runs as direct launches, the next two replay the captured RK4 step
    I = s.get_state()
    J, H, K = s.moments()
    e_g, p_g, _ = s.sums()
    I2 = P.step_rk4(np.zeros((spec.Nc, spec.G, spec.N)), 2)
    I3 = P.step_rk4(I2, 1)
    _, J_r, H_r, K_r = P.project(I3)
    _, J2, _, _ = P.project(I2)
    scale = np.max(np.abs(I3), axis=0, keepdims=True)
    assert float(np.max(np.abs(I - I3) / scale)) < tol
    assert _rel_elem(J, J_r) < tol
    f, f_r = O.moments_to_eddington(J, K), O.moments_to_eddington(J_r, K_r)
    assert float(np.max(np.abs(f - f_r))) < tol
    # the step's sums: energy and photon number of the state it started from
    de = np.diff(spec.edges)
    cen = np.sqrt(spec.edges[:-1] * spec.edges[1:])
    e_r = float(np.sum(4 * np.pi * J2 * de[None, :]))
    p_r = float(np.sum(4 * np.pi * J2 * (de / cen)[None, :]))
    assert abs(e_g - e_r) <= tol * abs(e_r) and abs(p_g - p_r) <= tol * abs(p_r)
    # switching back to the Euler step on the same context
    s.set_time_scheme("euler")
    s.step(1)
    I_e, _, _ = P.step(I3, 1)
    assert float(np.max(np.abs(s.get_state() - I_e) / np.max(np.abs(I_e), axis=0, keepdims=True))) < 3 * tol
    s.close()


def test_ng_static_fp64_matches_oracle(native):
    spec = inputs.relax_box(n=12)
    P = _oracle(spec)
    s = native.Solver.from_spec(spec, precision="fp64")
    s.set_ng(4)
    s.zero_state()
    it_g, r_g = s.solve_static(1e-8, 300)
    I_ref, it_r, r_r = P.solve_static_ng(tol=1e-8, max_iter=300, period=4)
    _, it_plain, _ = P.solve_static(tol=1e-8, max_iter=300)
    assert it_g == it_r < it_plain
    assert abs(r_g - r_r) <= 1e-6 * r_r
    assert _rel_elem(s.get_state(), I_ref, 1e-13) < FP64_TOL
    s.close()


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_ng_static_single_precision(native, precision):
    """Single precision with Ng: converges to the tolerance in fewer
    iterations than without, to the same fixed point as the plain iteration
    in that precision.  The fixed point of a single-precision iteration
    differs from the FP64 one by the per-iteration rounding amplified by the
    iteration's 1/(1 - rho) (rho: its spectral radius, about 0.9 here), so
    against the oracle's static solution the bound is ten times the
    per-step tolerance."""
    spec = inputs.jet(n=12, G=3, L=3, tau_r=6.0, gmax=3.0)
    P = _oracle(spec)
    I_ref, it_r, _ = P.solve_static(tol=1e-7, max_iter=400)
    plain = native.Solver.from_spec(spec, precision=precision)
    plain.zero_state()
    it_p, _ = plain.solve_static(1e-6, 300)
    I_p = plain.get_state()
    plain.close()
    s = native.Solver.from_spec(spec, precision=precision)
    s.set_ng(4)
    s.zero_state()
    it_g, r_g = s.solve_static(1e-6, 300)
    assert r_g <= 1e-6 and it_g < it_p
    I = s.get_state()
    scale = np.max(np.abs(I_ref))
    assert float(np.max(np.abs(I - I_p)) / scale) < 2e-5
    assert float(np.max(np.abs(I - I_ref)) / scale) < 10 * TOL[precision]
    with pytest.raises(native.ShdError):
        s.set_ng(3)
    s.close()
