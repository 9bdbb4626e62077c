"""Batches of independent problems (shd_batch_*): every problem of a batch
ends bit-identical to the same problem stepped on its own, and the FP64 one
matches the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_05141_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_05141_gb300 import native
    return native


def _problems():
    return [(inputs.ragged_mixed(), "fp64"),
            (inputs.jet(n=12, G=3, L=3, tau_r=3.0, gmax=4.0), "mixed"),
            (inputs.relax_box(n=8), "fp32"),
            (inputs.ragged_mixed(grid=(12, 8, 8), G=2), "mixed")]


def test_batch_matches_single_problems_and_oracle(native):
    probs = _problems()
    batch_solvers, single_solvers = [], []
    for i, (spec, prec) in enumerate(probs):
        I0 = inputs.random_state(spec, seed=20 + i)
        for group in (batch_solvers, single_solvers):
            s = native.Solver.from_spec(spec, precision=prec)
            s.set_state(I0)
            group.append(s)
    b = native.Batch(batch_solvers)
    n0 = native.launch_count()
    b.step(3)
    assert native.launch_count() > n0
    for s in single_solvers:
        s.step(3)
    for (spec, prec), sb, ss in zip(probs, batch_solvers, single_solvers):
        Jb, Hb, Kb = sb.moments()
        Js, Hs, Ks = ss.moments()
        assert np.array_equal(Jb, Js) and np.array_equal(Hb, Hs) and np.array_equal(Kb, Ks)
        assert np.array_equal(np.array(sb.sums()), np.array(ss.sums()))
    # the FP64 problem against the oracle
    spec, _ = probs[0]
    K, so = O.thomson_table(spec.G, spec.L)
    P = O.OracleProblem(grid=spec.grid, L=spec.L, nmu=spec.nmu, nphi=spec.nphi, edges=spec.edges,
                        alpha0=spec.alpha0, ne=spec.ne, u=spec.u, emis0=spec.emis0, K=K, sigma_out=so,
                        kappa=spec.kappa, box=spec.box)
    I_ref, _, _ = P.step(inputs.random_state(spec, seed=20), 3)
    _, J_r, _, _ = P.project(I_ref)
    J, _, _ = batch_solvers[0].moments()
    assert np.max(np.abs(J - J_r)) / np.max(np.abs(J_r)) < 1e-10
    b.close()


def test_batch_after_setter_and_more_steps(native):
    """A setter on one problem between batch steps (its captured step is
    dropped and recaptured); the batch keeps matching single stepping."""
    probs = _problems()[1:3]
    bs, ss = [], []
    for i, (spec, prec) in enumerate(probs):
        I0 = inputs.random_state(spec, seed=30 + i)
        for group in (bs, ss):
            s = native.Solver.from_spec(spec, precision=prec)
            s.set_state(I0)
            group.append(s)
    b = native.Batch(bs)
    b.step(2)
    for s in ss:
        s.step(2)
    for s in (bs[0], ss[0]):
        s.set_time(probs[0][0].kappa * 0.5)
    b.step(3)
    for s in ss:
        s.step(3)
    for sb, s1 in zip(bs, ss):
        assert np.array_equal(sb.moments()[0], s1.moments()[0])
    b.close()


def test_batched_sweep_matches_single_and_per_problem_sweeps(native):
    """Sweep mode 1 (one persistent plane sweep per kernel variant over the
    batch's work list) against mode 0 (each problem sweeps alone) and single
    stepping: uneven FP32 problems of several variants (one ordinate block
    per plane, two, a ragged grid the one-CTA sweep cannot take), an RK4
    problem that keeps its own sweep, and a Bezier one; enough steps to
    replay both S_lm buffers' graphs."""
    probs = [(inputs.jet(n=16, G=3, L=3, tau_r=3.0, gmax=4.0), "mixed", "euler", "linear"),
             (inputs.relax_box(n=8), "fp32", "euler", "linear"),
             (inputs.jet(n=40, G=2, L=3, tau_r=3.0, gmax=4.0), "fp32", "euler", "linear"),
             (inputs.ragged_mixed(grid=(12, 8, 8), G=2), "mixed", "euler", "linear"),
             (inputs.ragged_mixed(grid=(11, 9, 7), G=2), "mixed", "euler", "linear"),
             (inputs.relax_box(n=12), "fp32", "rk4", "linear"),
             (inputs.jet(n=12, G=2, L=3, tau_r=3.0, gmax=4.0), "mixed", "euler", "bezier")]
    groups = {"b1": [], "b0": [], "one": []}
    for i, (spec, prec, scheme, integ) in enumerate(probs):
        I0 = inputs.random_state(spec, seed=40 + i)
        for g in groups.values():
            s = native.Solver.from_spec(spec, precision=prec)
            s.set_time_scheme(scheme)
            s.set_integrator(integ)
            s.set_state(I0)
            g.append(s)
    b1, b0 = native.Batch(groups["b1"]), native.Batch(groups["b0"])
    b1.set_sweep_mode(1)
    nsteps = 5
    b1.step(2)
    b0.step(2)
    n = native.launch_count()
    b1.step(nsteps - 2)
    n1 = native.launch_count() - n
    n = native.launch_count()
    b0.step(nsteps - 2)
    n0 = native.launch_count() - n
    # the linear Euler problems whose planes the one-CTA sweep takes share one
    # launch per kernel variant in place of one each
    assert 0 < n1 < n0, (n1, n0)
    for s in groups["one"]:
        s.step(nsteps)
    for k, (sb1, sb0, s1) in enumerate(zip(groups["b1"], groups["b0"], groups["one"])):
        for a, b, c in zip(sb1.moments(), sb0.moments(), s1.moments()):
            assert np.array_equal(a, c), k
            assert np.array_equal(b, c), k
        assert np.array_equal(np.array(sb1.sums()), np.array(s1.sums())), k
    b1.close()
    b0.close()
