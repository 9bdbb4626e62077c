"""Every schedule of the single-precision sweep against the oracle and
against each other.

A schedule splits each (ordinate, group) plane over a thread-block cluster
of C CTAs of NT threads, each CTA owning a block of rows, and reads the
neighbouring block's row through distributed shared memory.  The arithmetic
per node is the same for every schedule, so results are bit-identical to the
one-CTA-a-plane kernel; each is also checked against the FP64 oracle (Sec. 2
eq:shdom, Sec. 2.1 eq:time).  Grids:

* (60, 52, 6): ragged blocks (52 rows over 8 CTAs), and classes with fewer
  rows than CTAs (6 rows over 8: CTAs with no rows still take part in every
  cluster barrier);
* (62, 52, 6): rows of 62 nodes, so a block must hold an even number of rows
  to start on a 16-byte boundary;
* (96, 96, 32): 9216-node planes, too large for one CTA's shared memory (only
  clusters can sweep them).  The z spacing is 2.8 times the x spacing, so the
  ordinates of the outer rings (|mu| = 0.96: |n_z| / |n_x| = 3.4) cross z
  faces first and the z-class, whose planes these are, is not empty (a grid
  of 4 z-nodes would leave it empty and sweep only 384-node planes).  8 x 384
  and 4 x 768 threads hold its blocks of 1152 and 2304 nodes at exactly three
  nodes a thread.
* (21, 22, 19): a ragged grid (no plane, and not Nc, a multiple of 4), which
  only one-CTA schedules sweep: 1024, 512 and 256 threads, each plane copied
  as its 16-byte aligned cover;
* (32, 32, 8): 1024-node planes, swept by one CTA of 1024, 512 or 256
  threads as well as by clusters;
* (128, 128, 32): 16384-node planes, whose 8-CTA blocks of 2048 nodes fill
  every slot of 512 threads x 4 nodes (the 128^3 workload's schedule).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_05141_gb300 import inputs

pytestmark = pytest.mark.gpu

FP32_TOL = 2e-5
SCHEDULES = [(1, 1024), (1, 512), (1, 256), (2, 256), (2, 384), (2, 512), (2, 768), (2, 1024), (4, 256), (4, 384), (4, 512),
             (4, 768), (4, 1024), (8, 256), (8, 384), (8, 512), (8, 768), (8, 1024),
             (16, 256), (16, 384), (16, 512), (16, 1024)]


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_05141_gb300 import native
    return native


def _oracle_step(spec, I0):
    K, so = O.thomson_table(spec.G, spec.L)
    P = O.OracleProblem(grid=spec.grid, L=spec.L, nmu=spec.nmu, nphi=spec.nphi, edges=spec.edges,
                        alpha0=spec.alpha0, ne=spec.ne, u=spec.u, emis0=spec.emis0, K=K, sigma_out=so,
                        kappa=spec.kappa, box=spec.box)
    I, _, _ = P.step(I0, 1)
    return I


@pytest.mark.parametrize("grid", [(60, 52, 6), (62, 52, 6), (96, 96, 32), (21, 22, 19), (32, 32, 8),
                                  (128, 128, 32)])
def test_every_schedule(native, grid):
    spec = inputs.ragged_mixed(grid=grid, G=2, L=3)
    I0 = inputs.random_state(spec, seed=41)
    I_ref = _oracle_step(spec, I0)
    scale = np.max(np.abs(I_ref), axis=0, keepdims=True)
    ran, first = [], None
    s = native.Solver.from_spec(spec, precision="fp32")
    for C, NT in SCHEDULES:
        try:
            s.set_sweep_schedule(C, NT)
        except native.ShdError:
            continue  # does not fit this grid
        s.set_state(I0)
        s.step(1)
        I = s.get_state()
        assert s.sweep_schedule()[0] == (C, NT)
        err = float(np.max(np.abs(I - I_ref) / scale))
        assert err < FP32_TOL, ((C, NT), err)
        if first is None:
            first = ((C, NT), I)
        else:
            assert np.array_equal(I, first[1]), ((C, NT), first[0])
        ran.append((C, NT))
    s.close()
    if grid in ((21, 22, 19), (32, 32, 8)):
        assert (1, 512) in ran and (1, 256) in ran, ran
    if grid == (21, 22, 19):
        assert all(c == 1 for c, _ in ran), ran  # clusters need aligned planes
        return
    assert any(c > 1 for c, _ in ran), "no cluster schedule ran"
    if grid == (128, 128, 32):
        assert (8, 512) in ran and (1, 1024) not in ran, ran
    if grid == (96, 96, 32):
        assert (1, 1024) not in ran  # the 9216-node planes need a cluster
        assert (8, 384) in ran and (4, 768) in ran  # three nodes a thread


def test_automatic_choice_is_timed_and_kept(native):
    spec = inputs.ragged_mixed(grid=(64, 64, 6), G=2, L=3)
    s = native.Solver.from_spec(spec, precision="mixed")
    assert s.sweep_schedule()[0] == (0, 0)
    s.set_state(inputs.random_state(spec, seed=3))
    s.step(2)
    (C, NT), rows = s.sweep_schedule()
    assert (C, NT) != (0, 0)
    assert len(rows) >= 2
    times = {(c, nt): ms for c, nt, ms in rows}
    assert (C, NT) in times and times[(C, NT)] == min(times.values())
    s.step(1)
    assert s.sweep_schedule()[0] == (C, NT)  # kept
    with pytest.raises(native.ShdError):
        s.set_sweep_schedule(3, 256)
    # a second context of the same shape takes the choice without timing
    s2 = native.Solver.from_spec(spec, precision="mixed")
    s2.set_state(inputs.random_state(spec, seed=3))
    s3 = native.Solver.from_spec(spec, precision="mixed")
    s3.set_state(inputs.random_state(spec, seed=3))
    s3.set_sweep_schedule(C, NT)  # forced: the same kernels, never timed
    n0 = native.launch_count()
    s2.step(2)
    n_cached = native.launch_count() - n0
    n0 = native.launch_count()
    s3.step(2)
    n_forced = native.launch_count() - n0
    assert s2.sweep_schedule()[0] == (C, NT)
    assert n_cached == n_forced, (n_cached, n_forced)  # no timing launches
    assert np.array_equal(s2.get_state(), s3.get_state())
    s2.close()
    s3.close()
    s.close()
