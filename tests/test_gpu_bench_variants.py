"""Oracle parity of the kernel variants the benchmark itself runs.

The benchmark (the 64^3 jet, L = 7, 16 x 32 ordinates) sweeps planes of
4096 nodes, which selects the FP32 two-buffer sweep with four nodes per
thread, and runs the TMA-fed tensor-core transforms with 64 harmonics.
Smaller cases reach the same variants when one ordinate class has 4096-node
planes and every plane is a multiple of 4 nodes:

* (64, 64, 6): z-crossing ordinates sweep 64 x 64 planes;
* (8, 64, 64): x-crossing ordinates sweep 64 x 64 (y, z) planes;
* (64, 8, 64): y-crossing ordinates sweep 64 x 64 (x, z) planes;

all at L = 7 with 16 x 32 ordinates and nx, ny multiples of 4 (segment
tiling of the mixed transforms).  Two steps, element by element against the
FP64 oracle (Sec. 2 eq:shdom, Sec. 2.1 eq:time, Sec. 2.2 frame order).

The full-size case runs one step of the 64^3 jet itself (FP32 and MIXED) and
checks the new intensity of sampled (ordinate, group) pairs at every node:
the oracle computes those pairs' laboratory eta, chi node by node and
sweeps only them.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1507_05141_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 2e-5
MIXED_TOL = 1e-4
TOL = {"fp64": FP64_TOL, "fp32": FP32_TOL, "mixed": MIXED_TOL}


@pytest.fixture(scope="module")
def native():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1507_05141_gb300 import native
    return native


def _oracle(spec):
    K, so = O.thomson_table(spec.G, spec.L) if spec.scattering == "thomson" else O.kn_table(spec.edges, spec.L)
    return O.OracleProblem(grid=spec.grid, L=spec.L, nmu=spec.nmu, nphi=spec.nphi, edges=spec.edges,
                           alpha0=spec.alpha0, ne=spec.ne, u=spec.u, emis0=spec.emis0, K=K, sigma_out=so,
                           kappa=spec.kappa, box=spec.box)


def _rel_elem(a, b, floor_frac=1e-12):
    b = np.asarray(b)
    den = np.maximum(np.abs(b), floor_frac * np.max(np.abs(b)))
    return float(np.max(np.abs(np.asarray(a) - b) / den))


_ORACLE_CACHE = {}


def _oracle_two_steps(grid):
    """Two oracle steps of the ragged flow recipe at L = 7 on `grid` (shared by
    the precisions)."""
    if grid not in _ORACLE_CACHE:
        spec = inputs.ragged_mixed(grid=grid, G=2, L=7)
        I0 = inputs.random_state(spec, seed=31)
        P = _oracle(spec)
        I_ref, _, _ = P.step(I0, 2)
        Ish_r, J_r, H_r, K_r = P.project(I_ref)
        _ORACLE_CACHE[grid] = (spec, I0, I_ref, Ish_r, J_r, H_r, K_r)
    return _ORACLE_CACHE[grid]


@pytest.mark.parametrize("grid", [(64, 64, 6), (8, 64, 64), (64, 8, 64)])
@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_4096_node_planes_l7(native, grid, precision):
    spec, I0, I_ref, Ish_r, J_r, H_r, K_r = _oracle_two_steps(grid)
    tol = TOL[precision]
    s = native.Solver.from_spec(spec, precision=precision)
    s.set_state(I0)
    s.step(2)
    I = s.get_state()
    J, H, K, Ish = s.moments(with_sh=True)
    s.close()
    # the state itself: error relative to each (group, ordinate) column's scale
    scale = np.max(np.abs(I_ref), axis=0, keepdims=True)
    assert float(np.max(np.abs(I - I_ref) / scale)) < tol
    assert _rel_elem(J, J_r) < tol
    Jm = np.max(np.abs(J_r), axis=0, keepdims=True)[..., None]
    assert float(np.max(np.abs(H - H_r) / Jm)) < tol
    f, f_r = O.moments_to_eddington(J, K), O.moments_to_eddington(J_r, K_r)
    assert float(np.max(np.abs(f - f_r))) < tol
    assert float(np.max(np.abs(Ish - Ish_r)) / np.max(np.abs(Ish_r))) < tol


def test_4096_node_planes_l7_fp64(native):
    spec, I0, I_ref, _, J_r, _, K_r = _oracle_two_steps((64, 64, 6))
    s = native.Solver.from_spec(spec, precision="fp64")
    s.set_state(I0)
    s.step(2)
    I = s.get_state()
    J, H, K = s.moments()
    s.close()
    assert _rel_elem(I, I_ref, 1e-13) < FP64_TOL
    assert _rel_elem(J, J_r) < FP64_TOL
    f, f_r = O.moments_to_eddington(J, K), O.moments_to_eddington(J_r, K_r)
    assert float(np.max(np.abs(f - f_r))) < FP64_TOL


def _sample_pairs(spec):
    """(mesh ordinate, group) pairs covering the three sweep classes, a
    diagonal direction and both ends of the group range."""
    _, _, dirs, _ = O.ordinates(spec.nmu, spec.nphi)
    ax = np.argmax(np.abs(dirs), axis=1)
    ks = [int(np.argmax(np.abs(dirs[:, 2]))), int(np.nonzero(ax == 0)[0][0]), int(np.nonzero(ax == 1)[0][-1]),
          int(np.argmin(np.abs(np.abs(dirs[:, 0]) - np.abs(dirs[:, 1])) + np.abs(dirs[:, 2])))]
    gs = [0, spec.G // 2, spec.G - 1, spec.G // 3]
    return [(k, g) for k, g in zip(ks, gs)]


def _oracle_pairs_full_size(spec, seed, pairs, chunk=2048):
    """One oracle step of the full-size problem restricted to `pairs`: the
    per-node stages (project, source, sh2lab) on chunks of nodes, then the
    sweep of the sampled pairs over the whole grid."""
    n = len(pairs)
    In = np.zeros((n, spec.Nc))
    eta = np.zeros((n, spec.Nc))
    chi = np.zeros((n, spec.Nc))
    K, so = O.thomson_table(spec.G, spec.L)
    for c0 in range(0, spec.Nc, chunk):
        nodes = np.arange(c0, min(spec.Nc, c0 + chunk))
        sub = inputs.sub_spec(spec, nodes)
        Psub = O.OracleProblem(grid=sub.grid, L=sub.L, nmu=sub.nmu, nphi=sub.nphi, edges=sub.edges,
                               alpha0=sub.alpha0, ne=sub.ne, u=sub.u, emis0=sub.emis0, K=K, sigma_out=so,
                               kappa=spec.kappa, box=spec.box)
        I_sub = inputs.hash_state_numpy(spec, seed=seed, nodes=nodes)
        Ip, _, _, _ = Psub.project(I_sub)
        e, x = Psub.sh2lab(Psub.source(Ip))
        for i, (k, g) in enumerate(pairs):
            In[i, nodes] = I_sub[:, g, k]
            eta[i, nodes] = e[:, g, k]
            chi[i, nodes] = x[:, g, k]
    return _oracle(spec).sweep_pairs(pairs, In, eta, chi)


def test_jet_64_full_size_step_sampled_pairs(native):
    """One step of the benchmark workload itself (64^3, 16 groups, L = 7,
    16 x 32 ordinates) in FP32 and MIXED from a seeded state; the new
    intensity of sampled (ordinate, group) pairs at every node against the
    oracle's step restricted to those pairs."""
    import torch
    spec = inputs.jet()
    seed = 17
    pairs = _sample_pairs(spec)
    ref = _oracle_pairs_full_size(spec, seed, pairs)
    for precision in ("mixed", "fp32"):
        s = native.Solver.from_spec(spec, precision=precision)
        dev = inputs.hash_state_torch(spec, seed=seed, device="cuda")
        s.set_state_dev(dev)
        s.step(1)
        s.get_state_dev(dev)
        torch.cuda.synchronize()
        s.close()
        view = dev.view(spec.Nc, spec.G, spec.N)
        got = np.stack([view[:, g, k].cpu().numpy() for k, g in pairs])
        del dev, view
        torch.cuda.empty_cache()
        for i in range(len(pairs)):
            err = float(np.max(np.abs(got[i] - ref[i])) / np.max(np.abs(ref[i])))
            assert err < TOL[precision], (precision, pairs[i], err)
