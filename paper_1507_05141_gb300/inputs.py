"""Seeded synthetic problem generators shared by the tests, the benchmark and
the oracle checks.

This module only draws the problem: grid, groups, fluid and opacity fields,
emissivities and the initial intensity.  It holds none of the solver's own
arithmetic (no quadrature, harmonics, Lorentz transformation, scattering
kernel or transfer), so both sides of every parity test can take their inputs
from it.

Recipes (numpy ``PCG64``, seed ``20150717 + index`` unless given):

* ``relax_box``     (16^3, 1 group, L=3, 8x16 ordinates, at rest): extinction
  5 across the unit box times a mean-preserving log-normal factor
  ``exp(0.2 xi - 0.02)`` per node; absorption = scattering = chi/2
  (isotropic scattering, albedo 1/2); thermal source B = 1; vacuum faces;
  ``c dt`` = half a node spacing.
* ``jet``           (64^3, 16 log groups over 1e-3..1e1 m_e c^2, L=7, 16x32):
  a cylindrical jet along z through the box centre, Gamma = 1 + 9 s(r) with
  s = 1 for r <= 0.2 falling smoothly to 0 at r = 0.3; Thomson scattering
  with a uniform n_e sigma_T giving radial optical depth ``tau_r`` from the
  axis to r = 0.5; comoving emissivity n_e eps^-1; vacuum faces;
  ``c dt`` = half a node spacing.
* ``compton_shell`` (96^3, 32 log groups over 1e-4..1e2, L=7, 16x32): a
  Gaussian random electron-temperature field (FFT-filtered white noise,
  correlation length 0.1 box) mapped to [0.01, 0.3] m_e c^2; a radial shell
  flow 0.25 <= r <= 0.40 with Gamma rising 2 -> 5 across it and blending to
  1 over 0.05 outside; n_e sigma_T = 5 per box length; grey absorption
  n_e (1/0.95 - 1) (albedo 0.95 in the Thomson limit); thermal emission
  alpha B_g(theta_e) with B_g the group average of x^3/(exp(x/theta)-1).

* ``jet_cocoon``    (128^3, 64 log groups over 1e-4..1e2, L=7, 16x32): a jet
  core r <= 0.08 with Gamma = 30 along z inside a cocoon 0.08..0.3 with
  u = 0.6 r_hat + 0.9 z_hat, smooth blends over 0.02; Klein-Nishina with
  albedo 0.95 and thermal emission from a random electron temperature as in
  ``compton_shell``.
* ``batch_problem`` (problem i of a batch of independent problems): cubic n,
  G, L drawn per problem; a jet of radius 0.2 along a random axis with Gamma
  log-uniform in [1, 20]; box optical depth log-uniform in [0.1, 20];
  Thomson or Klein-Nishina with probability 1/2 each.
* ``ragged_mixed``  (default 11x9x7, 5 groups, L=3): a non-cubic box with a
  tilted jet, random perturbations and 30 % of nodes at rest.

Every recipe accepts reduced ``n``, ``G``, ``L`` for oracle-sized cases; the
ordinate set follows ``nmu = 2(L+1)``, ``nphi = 4(L+1)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 20150717


@dataclass
class ProblemSpec:
    name: str
    grid: tuple
    box: tuple
    L: int
    nmu: int
    nphi: int
    edges: np.ndarray
    alpha0: np.ndarray      # [Nc, G]
    ne: np.ndarray          # [Nc]
    u: np.ndarray           # [Nc, 3]
    emis0: np.ndarray       # [Nc, G]
    scattering: str         # "iso" | "thomson" | "kn"
    kappa: float            # 1/(c dt) for the time steps
    steps: int
    extra: dict = field(default_factory=dict)

    @property
    def Nc(self):
        return int(np.prod(self.grid))

    @property
    def G(self):
        return len(self.edges) - 1

    @property
    def N(self):
        return self.nmu * self.nphi

    @property
    def NLM(self):
        return (self.L + 1) ** 2

    @property
    def updates_per_step(self):
        return self.Nc * self.N * self.G


def _rng(index, seed):
    return np.random.Generator(np.random.PCG64(BASE_SEED + index if seed is None else seed))


def _coords(n, box=1.0):
    h = box / (n - 1)
    x = np.arange(n) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")  # c = (iz*ny + iy)*nx + ix
    return X.ravel(), Y.ravel(), Z.ravel(), h


def _smoothstep(t):
    t = np.clip(t, 0.0, 1.0)
    return t * t * (3.0 - 2.0 * t)


def ordinate_counts(L):
    return 2 * (L + 1), 4 * (L + 1)


def relax_box(n=16, L=3, seed=None, index=0):
    rng = _rng(index, seed)
    Nc = n ** 3
    chi = 5.0 * np.exp(0.2 * rng.standard_normal(Nc) - 0.02)
    alpha0 = (chi / 2.0)[:, None]
    ne = chi / 2.0
    nmu, nphi = ordinate_counts(L)
    h = 1.0 / (n - 1)
    return ProblemSpec("relax_box", (n, n, n), (1.0, 1.0, 1.0), L, nmu, nphi,
                       np.array([0.5, 1.5]), alpha0, ne, np.zeros((Nc, 3)),
                       alpha0 * 1.0, "iso", kappa=1.0 / (0.5 * h), steps=10,
                       extra={"static_tol": 1e-6})


def jet_lorentz_factor(r, gmax=10.0, r_core=0.2, r_edge=0.3):
    s = 1.0 - _smoothstep((r - r_core) / (r_edge - r_core))
    return 1.0 + (gmax - 1.0) * s


def jet(n=64, G=16, L=7, tau_r=10.0, gmax=10.0, seed=None, index=1, emin=1e-3, emax=1e1):
    _rng(index, seed)  # the jet problem is deterministic; keep the stream reserved
    X, Y, Z, h = _coords(n)
    r = np.hypot(X - 0.5, Y - 0.5)
    gam = jet_lorentz_factor(r, gmax)
    u = np.zeros((n ** 3, 3))
    u[:, 2] = np.sqrt(np.maximum(gam * gam - 1.0, 0.0))
    edges = np.geomspace(emin, emax, G + 1)
    centre = np.sqrt(edges[:-1] * edges[1:])
    ne = np.full(n ** 3, tau_r / 0.5)
    alpha0 = np.zeros((n ** 3, G))
    emis0 = ne[:, None] * centre[None, :] ** -1.0
    nmu, nphi = ordinate_counts(L)
    return ProblemSpec("jet", (n, n, n), (1.0, 1.0, 1.0), L, nmu, nphi, edges, alpha0, ne, u,
                       emis0, "thomson", kappa=1.0 / (0.5 * h), steps=100,
                       extra={"tau_r": tau_r, "gmax": gmax})


def gaussian_random_field(n, corr, rng):
    w = rng.standard_normal((n, n, n))
    k = np.fft.fftfreq(n, d=1.0 / (n - 1))
    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")
    filt = np.exp(-0.5 * (2 * np.pi * corr) ** 2 * (KX ** 2 + KY ** 2 + KZ ** 2))
    f = np.real(np.fft.ifftn(np.fft.fftn(w) * filt))
    return f.ravel()


def planck_group(edges, theta, nsub=8):
    """Group average of x^3/(exp(x/theta) - 1) over each group (code units)."""
    G = len(edges) - 1
    xg, wg = np.polynomial.legendre.leggauss(nsub)
    out = np.zeros((theta.size, G))
    for g in range(G):
        a, b = np.log(edges[g]), np.log(edges[g + 1])
        s = 0.5 * (b - a) * xg + 0.5 * (a + b)
        x = np.exp(s)
        wq = 0.5 * (b - a) * wg * x
        arg = x[None, :] / theta[:, None]
        val = np.where(arg < 700.0, x[None, :] ** 3 / np.expm1(np.minimum(arg, 700.0)), 0.0)
        out[:, g] = (val * wq[None, :]).sum(axis=1) / (edges[g + 1] - edges[g])
    return out


def compton_shell(n=96, G=32, L=7, seed=None, index=2, emin=1e-4, emax=1e2, albedo=0.95):
    rng = _rng(index, seed)
    X, Y, Z, h = _coords(n)
    f = gaussian_random_field(n, 0.1, rng)
    theta = 0.01 + (f - f.min()) / (f.max() - f.min()) * (0.3 - 0.01)
    dx, dy, dz = X - 0.5, Y - 0.5, Z - 0.5
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    t = np.clip((r - 0.25) / 0.15, 0.0, 1.0)
    gam_in = 2.0 + 3.0 * t
    inside = (r >= 0.25) & (r <= 0.40)
    blend = np.where(r < 0.25, 1.0 - _smoothstep((0.25 - r) / 0.05), 1.0 - _smoothstep((r - 0.40) / 0.05))
    gam = np.where(inside, gam_in, 1.0 + (np.where(r < 0.25, 2.0, 5.0) - 1.0) * blend)
    um = np.sqrt(np.maximum(gam * gam - 1.0, 0.0))
    rs = np.maximum(r, 1e-30)
    u = np.stack([um * dx / rs, um * dy / rs, um * dz / rs], axis=1)
    u[r == 0.0] = 0.0
    edges = np.geomspace(emin, emax, G + 1)
    ne = np.full(n ** 3, 5.0)
    alpha0 = np.repeat((ne * (1.0 / albedo - 1.0))[:, None], G, axis=1)
    emis0 = alpha0 * planck_group(edges, theta)
    nmu, nphi = ordinate_counts(L)
    return ProblemSpec("compton_shell", (n, n, n), (1.0, 1.0, 1.0), L, nmu, nphi, edges, alpha0, ne,
                       u, emis0, "kn", kappa=1.0 / (0.5 * h), steps=200, extra={"theta_e": theta})


def jet_cocoon(n=128, G=64, L=7, seed=None, index=5, emin=1e-4, emax=1e2, albedo=0.95, tau_box=5.0):
    """A fast jet core (r <= 0.08, Gamma = 30 along z) inside a slower
    cocoon (0.08 < r < 0.3, u = 0.6 r_hat + 0.9 z_hat, Gamma ~ 1.5), smooth
    blends over 0.02; cold Klein-Nishina scattering with albedo 0.95 in every
    group and thermal emission from a Gaussian random electron-temperature
    field mapped to [0.01, 0.3]."""
    rng = _rng(index, seed)
    X, Y, Z, h = _coords(n)
    f = gaussian_random_field(n, 0.1, rng)
    theta = 0.01 + (f - f.min()) / (f.max() - f.min()) * (0.3 - 0.01)
    dx, dy = X - 0.5, Y - 0.5
    r = np.hypot(dx, dy)
    rs = np.maximum(r, 1e-30)
    rx, ry = np.where(r > 0, dx / rs, 0.0), np.where(r > 0, dy / rs, 0.0)
    core = 1.0 - _smoothstep((r - 0.08) / 0.02)     # 1 inside the core
    cocoon = 1.0 - _smoothstep((r - 0.30) / 0.02)   # 1 inside the cocoon's outer radius
    u_core = np.stack([np.zeros_like(r), np.zeros_like(r), np.full_like(r, np.sqrt(30.0 ** 2 - 1.0))], axis=1)
    u_coc = np.stack([0.6 * rx, 0.6 * ry, np.full_like(r, 0.9)], axis=1)
    u = core[:, None] * u_core + (1.0 - core)[:, None] * cocoon[:, None] * u_coc
    u[np.all(np.abs(u) < 1e-12, axis=1)] = 0.0
    edges = np.geomspace(emin, emax, G + 1)
    ne = np.full(n ** 3, tau_box)
    alpha0 = np.repeat((ne * (1.0 / albedo - 1.0))[:, None], G, axis=1)
    emis0 = alpha0 * planck_group(edges, theta)
    nmu, nphi = ordinate_counts(L)
    return ProblemSpec("jet_cocoon", (n, n, n), (1.0, 1.0, 1.0), L, nmu, nphi, edges, alpha0, ne, u, emis0, "kn",
                       kappa=1.0 / (0.5 * h), steps=500, extra={"theta_e": theta})


def batch_problem(i, seed=None, n_range=(16, 64), g_range=(8, 32), Ls=(3, 5, 7)):
    """Problem i of the batch of independent problems: cubic grid n ~ U{n_range},
    G ~ U{g_range} log groups over 1e-3..1e1, L from Ls, a jet of radius 0.2
    along an isotropically random axis through the box centre with Gamma
    log-uniform in [1, 20], box optical depth log-uniform in [0.1, 20],
    Thomson or Klein-Nishina scattering with probability 1/2 each."""
    rng = _rng(1000 * (i + 1) + 4, seed)
    n = int(rng.integers(n_range[0], n_range[1] + 1))
    G = int(rng.integers(g_range[0], g_range[1] + 1))
    L = int(rng.choice(Ls))
    axis = rng.standard_normal(3)
    axis /= np.linalg.norm(axis)
    gmax = float(np.exp(rng.uniform(0.0, np.log(20.0))))
    tau = float(np.exp(rng.uniform(np.log(0.1), np.log(20.0))))
    kind = "kn" if rng.random() < 0.5 else "thomson"
    X, Y, Z, h = _coords(n)
    p = np.stack([X - 0.5, Y - 0.5, Z - 0.5], axis=1)
    r = np.linalg.norm(p - (p @ axis)[:, None] * axis[None, :], axis=1)
    gam = jet_lorentz_factor(r, gmax, 0.2, 0.3)
    u = np.sqrt(np.maximum(gam * gam - 1.0, 0.0))[:, None] * axis[None, :]
    u[gam <= 1.0] = 0.0
    edges = np.geomspace(1e-3, 1e1, G + 1)
    centre = np.sqrt(edges[:-1] * edges[1:])
    ne = np.full(n ** 3, tau)
    alpha0 = np.full((n ** 3, G), 0.1 * tau)
    emis0 = ne[:, None] * centre[None, :] ** -1.0
    nmu, nphi = ordinate_counts(L)
    return ProblemSpec(f"batch_{i}", (n, n, n), (1.0, 1.0, 1.0), L, nmu, nphi, edges, alpha0, ne, u, emis0, kind,
                       kappa=1.0 / (0.5 * h), steps=20, extra={"gmax": gmax, "tau": tau})


def random_state(spec: ProblemSpec, seed=12345, scale=1.0, layout="cgk"):
    """A positive seeded intensity for single-step parity checks, [c][g][k]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    I = scale * (0.5 + rng.random((spec.Nc, spec.G, spec.N)))
    return I


def ragged_mixed(grid=(11, 9, 7), G=5, L=3, gmax=3.0, seed=None, index=7, scattering="thomson", theta_range=None):
    """A small non-cubic problem with flow, absorption, emission and
    scattering, for element-by-element parity on sizes that leave ragged
    tiles.  Velocity: a tilted jet plus a weak random component.  With
    theta_range = (lo, hi) the nodes also get electron temperatures
    log-uniform in [lo, hi] (extra["theta_e"])."""
    rng = _rng(index, seed)
    nx, ny, nz = grid
    hx, hy, hz = 1.0 / (nx - 1), 1.2 / (ny - 1), 0.9 / (nz - 1)
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    X = (ix * hx).transpose(2, 1, 0).ravel()
    Y = (iy * hy).transpose(2, 1, 0).ravel()
    Z = (iz * hz).transpose(2, 1, 0).ravel()
    Nc = nx * ny * nz
    axis = np.array([0.3, -0.2, 1.0])
    axis /= np.linalg.norm(axis)
    p = np.stack([X - 0.5, Y - 0.6, Z - 0.45], axis=1)
    r = np.linalg.norm(p - (p @ axis)[:, None] * axis[None, :], axis=1)
    gam = jet_lorentz_factor(r, gmax, 0.15, 0.3)
    u = np.sqrt(np.maximum(gam ** 2 - 1.0, 0.0))[:, None] * axis[None, :]
    u += 0.05 * rng.standard_normal((Nc, 3))
    u[rng.random(Nc) < 0.3] = 0.0  # a share of nodes at rest
    edges = np.geomspace(1e-2, 3.0, G + 1)
    centre = np.sqrt(edges[:-1] * edges[1:])
    ne = 2.0 * np.exp(0.3 * rng.standard_normal(Nc))
    alpha0 = 0.5 * np.exp(0.3 * rng.standard_normal((Nc, G)))
    emis0 = (1.0 + rng.random((Nc, 1))) * centre[None, :] ** -0.5
    nmu, nphi = ordinate_counts(L)
    extra = {}
    if theta_range is not None:
        lo, hi = np.log10(theta_range[0]), np.log10(theta_range[1])
        extra["theta_e"] = 10.0 ** rng.uniform(lo, hi, Nc)
    return ProblemSpec("ragged_mixed", grid, (1.0, 1.2, 0.9), L, nmu, nphi, edges, alpha0, ne, u,
                       emis0, scattering, kappa=1.0 / (0.5 * hx), steps=3, extra=extra)


# ----------------------------------------------------------------------------
# counter-based seeded intensities, computable for any element on either side
# ----------------------------------------------------------------------------
# value(i) = 0.5 + fmix32((i + seed * 0x9E3779B9) mod 2^32) / 2^32 for the
# flat index i = (c*G + g)*N + k of the [c][g][k] layout; fmix32 is the
# MurmurHash3 32-bit finaliser.  Products are split so that every
# intermediate fits in a signed 64-bit integer (numpy and torch alike).

_M32 = 0xFFFFFFFF


def _mul32(h, c):
    lo = h & 0xFFFF
    hi = h >> 16
    return ((lo * c) + (((hi * c) & 0xFFFF) << 16)) & _M32


def _fmix32(h):
    h = h ^ (h >> 16)
    h = _mul32(h, 0x85EBCA6B)
    h = h ^ (h >> 13)
    h = _mul32(h, 0xC2B2AE35)
    h = h ^ (h >> 16)
    return h


def _hash_unit(idx, seed):
    h = _fmix32((idx + seed * 0x9E3779B9) & _M32)
    h = h.double() if hasattr(h, "double") else h.astype(np.float64)  # torch or numpy
    return 0.5 + h / 4294967296.0


def hash_state_numpy(spec: ProblemSpec, seed: int, nodes=None):
    """Seeded intensity [len(nodes)][G][N] (all nodes when nodes is None)."""
    nodes = np.arange(spec.Nc) if nodes is None else np.asarray(nodes)
    per = spec.G * spec.N
    idx = nodes.astype(np.int64)[:, None] * per + np.arange(per, dtype=np.int64)[None, :]
    return _hash_unit(idx, int(seed)).reshape(len(nodes), spec.G, spec.N)


def hash_state_torch(spec: ProblemSpec, seed: int, device="cuda", chunk=1 << 26):
    """The same seeded intensity as one flat FP64 tensor on ``device``."""
    import torch
    n = spec.Nc * spec.G * spec.N
    out = torch.empty(n, dtype=torch.float64, device=device)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        idx = torch.arange(s, e, dtype=torch.int64, device=device)
        out[s:e] = _hash_unit(idx, int(seed))
    return out


def sub_spec(spec: ProblemSpec, nodes):
    """The per-node fields of a subset of nodes as a (len, 1, 1) problem, for
    checks of the per-node stages (projection, source, transforms)."""
    nodes = np.asarray(nodes)
    return ProblemSpec(spec.name + "_sub", (len(nodes), 1, 1), spec.box, spec.L, spec.nmu, spec.nphi,
                       spec.edges, spec.alpha0[nodes], spec.ne[nodes], spec.u[nodes], spec.emis0[nodes],
                       spec.scattering, spec.kappa, spec.steps, dict(spec.extra))
