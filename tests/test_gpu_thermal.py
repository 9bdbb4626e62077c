"""Compton scattering off thermal electrons (the temperature field's kernel;
the paper's own is cold) on the GPU against the FP64 oracle: the 13 tables
of the temperature grid built on the device, whole steps with a node
temperature field spanning several grid brackets in FP64, FP32 and MIXED,
and the temperature field's checks."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_05141_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-5, "mixed": 1e-4}
_TABLES = {}


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_05141_gb300 import native
    return native


def _spec():
    spec = inputs.ragged_mixed(G=6, L=3, scattering="kn_thermal", theta_range=(3e-3, 0.5))
    spec.edges = np.geomspace(1e-3, 3.0, 7)
    return spec


def _tables(spec):
    key = (tuple(spec.edges), spec.L)
    if key not in _TABLES:
        _TABLES[key] = O.thermal_tables(spec.edges, spec.L)
    return _TABLES[key]


def _oracle(spec):
    Kth, soth = _tables(spec)
    th = {"theta_e": spec.extra["theta_e"], "K_th": Kth, "so_th": soth, "lg0": O.THERMAL_LG0, "dlg": O.THERMAL_DLG}
    return O.OracleProblem(grid=spec.grid, L=spec.L, nmu=spec.nmu, nphi=spec.nphi, edges=spec.edges,
                           alpha0=spec.alpha0, ne=spec.ne, u=spec.u, emis0=spec.emis0, K=Kth[0], sigma_out=soth[0],
                           kappa=spec.kappa, box=spec.box, thermal=th)


def test_thermal_tables_match_oracle(native):
    spec = _spec()
    s = native.Solver.from_spec(spec, precision="fp64")
    K, so = s.get_thermal_tables()
    Kr, sor = _tables(spec)
    assert float(np.max(np.abs(K - Kr)) / np.max(np.abs(Kr))) < 1e-10
    assert float(np.max(np.abs(so - sor) / sor)) < 1e-10
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_thermal_steps(native, precision):
    spec = _spec()
    th = spec.extra["theta_e"]
    assert len(np.unique(np.floor((np.log10(th) + 3) / 0.25))) >= 5  # several brackets of the grid
    P = _oracle(spec)
    s = native.Solver.from_spec(spec, precision=precision)
    I0 = inputs.random_state(spec, seed=5)
    s.set_state(I0)
    s.step(2)
    I = s.get_state()
    J, H, K = s.moments()
    e_g, p_g, _ = s.sums()
    I_ref, _, sums = P.step(I0, 2)
    _, J_r, H_r, K_r = P.project(I_ref)
    tol = TOL[precision]
    assert float(np.max(np.abs(I - I_ref) / np.max(np.abs(I_ref), axis=0, keepdims=True))) < tol
    assert float(np.max(np.abs(J - J_r) / np.abs(J_r))) < tol
    f, f_r = O.moments_to_eddington(J, K), O.moments_to_eddington(J_r, K_r)
    assert float(np.max(np.abs(f - f_r))) < tol
    assert abs(e_g - sums[0]) <= tol * abs(sums[0]) and abs(p_g - sums[1]) <= tol * abs(sums[1])
    s.close()


def test_thermal_needs_and_checks_temperatures(native):
    spec = _spec()
    s = native.Solver.from_spec(spec, precision="fp32")
    s.set_fields(spec.alpha0, spec.ne, spec.u, spec.emis0)  # no temperatures
    s.zero_state()
    with pytest.raises(native.ShdError) as ei:
        s.step(1)
    assert ei.value.code == native.ERR_STATE
    bad = spec.extra["theta_e"].copy()
    bad[3] = -1.0
    with pytest.raises(native.ShdError, match="theta_e"):
        s.set_fields(spec.alpha0, spec.ne, spec.u, spec.emis0, bad)
    s.set_fields(spec.alpha0, spec.ne, spec.u, spec.emis0, spec.extra["theta_e"])
    s.step(1)
    s.close()
