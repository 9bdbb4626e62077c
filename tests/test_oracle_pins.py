"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value is a
closed form, a library routine standing in for a textbook special case, an
invariant, or a number printed in the paper (tests/golden/, cited there).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#", ndmin=2)


# --------------------------------------------------------------------------
# quadrature and spherical harmonics (Sec. 2.3)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 33])
def test_gauss_legendre_matches_numpy(n):
    x, w = O.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.allclose(x, xr, atol=1e-14, rtol=0)
    assert np.allclose(w, wr, atol=1e-14, rtol=0)


def test_ordinates_weights_and_directions():
    mu, wmu, dirs, W = O.ordinates(8, 16)
    assert abs(W.sum() - 4 * np.pi) < 1e-13
    assert np.allclose(np.linalg.norm(dirs, axis=1), 1.0, atol=1e-15)
    # phi_b = 2 pi b / nphi from the x axis towards y (Sec. 2, geometry); b = 4 is +y
    k = 3 * 16 + 4
    assert dirs[k, 0] == 0.0 and dirs[k, 1] > 0
    assert dirs[3 * 16, 1] == 0.0 and dirs[3 * 16, 0] > 0


def _real_sh_scipy(L, mu, phi):
    """Real orthonormal SH without Condon-Shortley phase, from scipy's complex
    Y_l^m (which carries the (-1)^m phase)."""
    from scipy.special import sph_harm_y
    th = np.arccos(mu)
    out = np.zeros((L + 1) ** 2)
    for l in range(L + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            y = sph_harm_y(l, am, th, phi) * (-1) ** am  # remove Condon-Shortley
            if m == 0:
                v = y.real
            elif m > 0:
                v = np.sqrt(2) * y.real
            else:
                v = np.sqrt(2) * y.imag
            out[l * l + l + m] = v
    return out


@pytest.mark.parametrize("mu,phi", [(0.3, 0.7), (-0.91, 4.0), (0.999, 2.2), (0.0, 0.0)])
def test_ylm_matches_scipy(mu, phi):
    L = 9
    assert np.allclose(O.ylm(L, mu, phi), _real_sh_scipy(L, mu, phi), atol=1e-12, rtol=1e-12)


def test_ylm_low_order_closed_forms():
    mu, phi = 0.4, 1.1
    st = np.sqrt(1 - mu * mu)
    Y = O.ylm(2, mu, phi)
    ref = np.array([
        0.5 / np.sqrt(np.pi),
        np.sqrt(3 / (4 * np.pi)) * st * np.sin(phi),
        np.sqrt(3 / (4 * np.pi)) * mu,
        np.sqrt(3 / (4 * np.pi)) * st * np.cos(phi),
        np.sqrt(15 / (16 * np.pi)) * st * st * np.sin(2 * phi),
        np.sqrt(15 / (4 * np.pi)) * mu * st * np.sin(phi),
        np.sqrt(5 / (16 * np.pi)) * (3 * mu * mu - 1),
        np.sqrt(15 / (4 * np.pi)) * mu * st * np.cos(phi),
        np.sqrt(15 / (16 * np.pi)) * st * st * np.cos(2 * phi),
    ])
    assert np.allclose(Y, ref, atol=1e-15, rtol=1e-14)


@pytest.mark.parametrize("L", [1, 3, 5, 7])
def test_discrete_orthogonality(L):
    nmu, nphi = 2 * (L + 1), 4 * (L + 1)
    _, _, _, W = O.ordinates(nmu, nphi)
    Y = O.ylm_table(L, nmu, nphi)
    gram = (Y * W[:, None]).T @ Y
    assert np.abs(gram - np.eye((L + 1) ** 2)).max() < 1e-13


# --------------------------------------------------------------------------
# Lorentz transformation (Sec. 2.2, eq:lorentzfreq, eq:lorentzray)
# --------------------------------------------------------------------------

def test_paper_lorentz_factors():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "lorentz_factors.txt"))
            if ln.strip() and not ln.startswith("#")]
    for beta_s, g_s in rows:
        beta = float(beta_s)
        half_ulp = 0.5 * 10.0 ** -len(g_s.split(".")[1])  # half a unit of the last printed digit
        ux = beta / np.sqrt(1 - beta * beta)
        _, r = O.lab_to_comoving([ux, 0, 0], [0.0, 0.0, 1.0])  # n perpendicular: r = Gamma
        assert abs(r - float(g_s)) <= half_ulp


@pytest.mark.parametrize("beta", [0.3, 0.9, 0.999, 1 - 5e-7])
@pytest.mark.parametrize("mu", [-0.95, -0.2, 0.0, 0.5, 0.99])
def test_boost_along_z_matches_textbook(beta, mu):
    """For v along z: nu0/nu = Gamma (1 - beta mu), mu0 = (mu - beta)/(1 - beta mu)."""
    gam = 1 / np.sqrt((1 - beta) * (1 + beta))
    st = np.sqrt(1 - mu * mu)
    n = np.array([st * np.cos(0.3), st * np.sin(0.3), mu])
    n0, r = O.lab_to_comoving([0, 0, gam * beta], n)
    assert r == pytest.approx(gam * (1 - beta * mu), rel=1e-11)
    assert n0[2] == pytest.approx((mu - beta) / (1 - beta * mu), rel=1e-9, abs=1e-12)
    # azimuth is unchanged by a boost along z
    if st > 0:
        assert np.arctan2(n0[1], n0[0]) == pytest.approx(0.3, abs=1e-10)


def test_boost_unit_norm_and_round_trip():
    rng = np.random.default_rng(3)
    for _ in range(200):
        u = rng.normal(size=3) * rng.choice([0.1, 3.0, 30.0, 1000.0])
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        n0, r = O.lab_to_comoving(u, n)
        assert np.linalg.norm(n0) == pytest.approx(1.0, abs=1e-11)
        n1, q = O.comoving_to_lab(u, n0)
        assert np.allclose(n1, n, atol=1e-9)
        assert r * q == pytest.approx(1.0, rel=1e-10)
        # nu0/nu against the direct formula where it does not cancel badly
        gam = np.sqrt(1 + u @ u)
        assert r == pytest.approx(gam - u @ n, rel=1e-13 * gam * gam + 1e-14, abs=1e-300)


# --------------------------------------------------------------------------
# remapping between frames (Sec. 2.2, last paragraph; Sec. 3.4)
# --------------------------------------------------------------------------

def _iso_problem(edges, u, L=3, nmu=8, nphi=16, S00=1.0, spec_index=0.0):
    G = len(edges) - 1
    K, so = O.iso_table(G, L)
    centre = np.sqrt(edges[:-1] * edges[1:])
    P = O.OracleProblem(grid=(2, 2, 2), L=L, nmu=nmu, nphi=nphi, edges=edges,
                        alpha0=np.ones((8, G)), ne=np.zeros(8), u=np.tile(u, (8, 1)),
                        emis0=np.zeros((8, G)), K=K, sigma_out=so)
    Sp = np.zeros((8, G, (L + 1) ** 2))
    Sp[:, :, 0] = S00 * np.sqrt(4 * np.pi) * centre[None, :] ** (-spec_index)
    return P, Sp


def test_isotropic_boost_paper_criterion():
    """Comoving isotropic intensity -> laboratory: [Gamma(1 - mu beta)]^-3 I0
    within 1e-6 (Sec. 3.4) for Gamma = 10, 100, 1000, on a small mesh."""
    tab = _golden("isotropic_boost.txt")
    for one_minus_beta, _g, tol in tab:
        beta = 1.0 - one_minus_beta
        gam = 1 / np.sqrt(one_minus_beta * (1 + beta))
        P, Sp = _iso_problem(np.array([1e-5, 1e5]), [0, 0, gam * beta], nmu=32, nphi=64)
        eta, chi = P.sh2lab(Sp)
        S_lab = eta[0, 0] / chi[0, 0]
        mu, _, dirs, _ = O.ordinates(32, 64)
        ref = (gam * (1 - dirs[:, 2] * beta)) ** -3
        assert np.max(np.abs(S_lab - ref) / ref) < tol
        assert np.max(np.abs(S_lab - ref) / ref) < 1e-9  # and in fact to rounding


def test_power_law_boost_exact_with_geometric_groups():
    """I/nu^3 invariance with a comoving power law eps^-s: interior groups get
    D^-(3+s) S0(ebar_g) exactly (geometric frequency remap)."""
    edges = np.geomspace(1e-3, 1e1, 33)
    s = 1.3
    beta = 0.6
    gam = 1 / np.sqrt(1 - beta * beta)
    P, Sp = _iso_problem(edges, [0, 0, gam * beta], spec_index=s)
    eta, chi = P.sh2lab(Sp)
    S_lab = eta[0] / chi[0]                          # [g][k]
    _, _, dirs, _ = O.ordinates(8, 16)
    D = gam * (1 - beta * dirs[:, 2])                # nu0/nu
    centre = np.sqrt(edges[:-1] * edges[1:])
    ref = D[None, :] ** -(3 + s) * centre[:, None] ** -s
    g_int = slice(4, 28)  # groups whose shifted energy stays between centres
    assert np.max(np.abs(S_lab[g_int] - ref[g_int]) / ref[g_int]) < 1e-12
    # chi nu invariance: chi_lab = D chi0 for a grey chi0
    assert np.allclose(chi[0], np.ones_like(chi[0]) * D[None, :], rtol=1e-13)


def test_interp_freq_rules():
    edges = np.array([1.0, 2.0, 4.0, 8.0])
    c = np.sqrt(edges[:-1] * edges[1:])
    F = 3.0 * c ** -2.0
    e = 3.1
    assert O.interp_freq(edges, F, e) == pytest.approx(3.0 * e ** -2.0, rel=1e-14)
    assert O.interp_freq(edges, F, 1.2) == F[0]           # between edge and first centre
    assert O.interp_freq(edges, F, 0.9) == 0.0            # beyond the edges
    assert O.interp_freq(edges, F, 9.0, True) == F[-1]
    G2 = np.array([-1.0, 2.0, 5.0])                        # sign change: linear in log eps
    t = np.log(e / c[1]) / np.log(c[2] / c[1])
    assert O.interp_freq(edges, G2, e) == pytest.approx(2.0 ** (1 - t) * 5.0 ** t, rel=1e-14)  # both > 0
    t0 = np.log(1.7 / c[0]) / np.log(c[1] / c[0])
    assert O.interp_freq(edges, G2, 1.7) == pytest.approx((1 - t0) * -1.0 + t0 * 2.0, rel=1e-14)


def test_interp_angle_exact_cases():
    nmu, nphi = 8, 16
    mu, _, dirs, _ = O.ordinates(nmu, nphi)
    const = np.full(nmu * nphi, 2.5)
    lin = dirs[:, 2].copy()  # F = mu: bilinear is exact between rings
    rng = np.random.default_rng(0)
    for _ in range(50):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        assert O.interp_angle(nmu, nphi, mu, const, n) == pytest.approx(2.5, rel=1e-15)
        if mu[0] <= n[2] <= mu[-1]:
            assert O.interp_angle(nmu, nphi, mu, lin, n) == pytest.approx(n[2], abs=1e-14)
    # at a mesh direction the node value comes back
    F = rng.random(nmu * nphi)
    for k in [0, 17, 63, 127]:
        assert O.interp_angle(nmu, nphi, mu, F, dirs[k]) == pytest.approx(F[k], rel=1e-12)


# --------------------------------------------------------------------------
# moments
# --------------------------------------------------------------------------

def _box(grid, L=3, G=1, u=None, alpha=1.0, ne=0.0, emis=0.0, box=(1.0, 1.0, 1.0), edges=None,
         table="iso"):
    Nc = int(np.prod(grid))
    if edges is None:
        edges = np.geomspace(0.5, 1.5, G + 1)
    K, so = (O.iso_table if table == "iso" else O.thomson_table)(G, L)
    nmu, nphi = 2 * (L + 1), 4 * (L + 1)
    return O.OracleProblem(grid=grid, L=L, nmu=nmu, nphi=nphi, edges=edges,
                           alpha0=np.broadcast_to(np.asarray(alpha, float), (Nc, G)).copy()
                           if np.ndim(alpha) < 2 else alpha,
                           ne=np.broadcast_to(np.asarray(ne, float), (Nc,)).copy(),
                           u=np.zeros((Nc, 3)) if u is None else u,
                           emis0=np.broadcast_to(np.asarray(emis, float), (Nc, G)).copy()
                           if np.ndim(emis) < 2 else emis,
                           K=K, sigma_out=so, box=box)


def test_isotropic_moments_exact():
    P = _box((3, 3, 3), L=3, G=2)
    I = np.full((27, 2, P.N), 1.7)
    Ip, J, H, Kt = P.project(I)
    assert np.allclose(J, 1.7, rtol=1e-14)
    assert np.abs(H).max() < 1e-14
    f = O.moments_to_eddington(J, Kt)
    assert np.allclose(f[..., :3], 1 / 3, atol=1e-14)
    assert np.abs(f[..., 3:]).max() < 1e-14
    assert np.allclose(Ip[..., 0], 1.7 * np.sqrt(4 * np.pi), rtol=1e-14)
    assert np.abs(Ip[..., 1:]).max() < 1e-13


def test_eddington_trace_is_one():
    P = _box((3, 3, 3), L=3, G=2)
    I = np.random.default_rng(1).random((27, 2, P.N))
    _, J, _, Kt = P.project(I)
    assert np.allclose(Kt[..., 0] + Kt[..., 1] + Kt[..., 2], J, rtol=1e-14)


def test_projection_round_trip_is_identity():
    """SH -> ordinates -> SH is the identity for l <= L (discrete orthogonality):
    the source built from I_p, evaluated on ordinates and projected back."""
    P = _box((2, 2, 2), L=3, G=1, alpha=1.0, ne=0.0)
    rng = np.random.default_rng(5)
    Sp = rng.normal(size=(8, 1, 16))
    eta, chi = P.sh2lab(Sp)
    Ip, _, _, _ = P.project(eta / chi)
    assert np.allclose(Ip, Sp, atol=1e-13)


# --------------------------------------------------------------------------
# source (Sec. 2.3)
# --------------------------------------------------------------------------

def test_thomson_table_values_and_photon_conservation():
    K, so = O.thomson_table(4, 3)
    assert K[2, 0, 0] / K[0, 0, 0] == pytest.approx(0.1)
    # pure Thomson scattering, no absorption: S_lm = I_lm for l = 0 (omega = 1)
    P = _box((2, 2, 2), L=3, G=4, alpha=0.0, ne=3.0, table="thomson")
    Ip = np.random.default_rng(2).normal(size=(8, 4, 16))
    Sp = P.source(Ip)
    assert np.allclose(Sp[..., 0], Ip[..., 0], rtol=1e-15)
    assert np.allclose(Sp[..., 4:9], 0.1 * Ip[..., 4:9], rtol=1e-15)
    assert np.allclose(Sp[..., 1:4], 0.0) and np.allclose(Sp[..., 9:], 0.0)


def test_source_albedo_and_emission():
    P = _box((2, 2, 2), L=3, G=1, alpha=1.0, ne=3.0, emis=2.0)   # omega = 3/4
    Ip = np.zeros((8, 1, 16))
    Ip[..., 0] = 5.0
    Sp = P.source(Ip)
    assert np.allclose(Sp[..., 0], 0.75 * 5.0 + np.sqrt(4 * np.pi) * 2.0 / 4.0, rtol=1e-15)


# --------------------------------------------------------------------------
# Klein-Nishina table (Sec. 2.3, eq:comptoncross)
# --------------------------------------------------------------------------

def _sigma_kn(x):
    """Textbook total Klein-Nishina cross-section / sigma_T."""
    import mpmath as mp
    with mp.workdps(60):  # the closed form cancels badly at small x
        x = mp.mpf(x)
        l = mp.log(1 + 2 * x)
        return float(mp.mpf(3) / 4 * ((1 + x) / x ** 3 * (2 * x * (1 + x) / (1 + 2 * x) - l)
                                      + l / (2 * x) - (1 + 3 * x) / (1 + 2 * x) ** 2))


def _sigma_energy(x):
    """Closed form of Int dOmega (dsigma/dOmega)(eps1/eps) / sigma_T for the KN
    cross-section (the energy carried away by scattered photons)."""
    import mpmath as mp
    with mp.workdps(60):
        x = mp.mpf(x)
        l = mp.log(1 + 2 * x)
        num = (-24 * x ** 4 + 24 * x ** 3 + 76 * x ** 2 + 48 * x + 9
               + (1 + 2 * x) ** 3 * (8 * x ** 2 - 6 * x + 6 * l - 9))
        return float(num / (16 * x ** 3 * (1 + 2 * x) ** 3))


def _group_integral(f, a, b):
    from scipy.integrate import quad
    val, _ = quad(lambda t: f(np.exp(t)) * np.exp(t), np.log(a), np.log(b), epsabs=0, epsrel=1e-13,
                  limit=200)
    return val


@pytest.mark.parametrize("edges", [np.geomspace(1e-3, 1e1, 9), np.linspace(0.1, 1.1, 11)])
def test_kn_out_scattering_matches_closed_form(edges):
    K, so = O.kn_table(edges, 3)
    for g in range(len(edges) - 1):
        ref = _group_integral(_sigma_kn, edges[g], edges[g + 1]) / (edges[g + 1] - edges[g])
        assert so[g] == pytest.approx(ref, rel=1e-11)


def test_kn_photon_number_and_energy_balance():
    """Summed over final groups: the photon-number kernel gives the total
    cross-section and the energy kernel the energy-scattering cross-section,
    for incident groups whose down-scattered photons cannot leave the range."""
    edges = np.geomspace(1e-3, 1e1, 9)
    de = np.diff(edges)
    KN, _ = O.kn_table(edges, 2, energy_weighted=False)
    KE, so = O.kn_table(edges, 2, energy_weighted=True)
    for gp in range(len(de)):
        if edges[gp] / (1 + 2 * edges[gp]) < edges[0]:
            continue  # down-scatter can leak below the lowest edge
        num = (de * KN[0, :, gp]).sum()
        en = (de * KE[0, :, gp]).sum()
        assert num == pytest.approx(_group_integral(_sigma_kn, edges[gp], edges[gp + 1]), rel=1e-11)
        assert en == pytest.approx(_group_integral(_sigma_energy, edges[gp], edges[gp + 1]), rel=1e-10)
        assert en < num  # electrons gain what photons lose (recoil)
        # no up-scattering off cold electrons
        assert np.all(KE[:, gp + 1:, gp] == 0.0) or gp == len(de) - 1


def test_kn_thomson_limit():
    edges = np.geomspace(1e-7, 1.2e-7, 3)
    K, so = O.kn_table(edges, 3)
    x = edges[-1]
    assert np.allclose(so, 1.0, atol=3 * x)
    Ksum = K.sum(axis=1)                       # over final groups (tiny shifts cross edges)
    w = np.diff(edges)
    tot = (K * w[None, :, None]).sum(axis=1) / w
    assert np.allclose(tot[0], 1.0, atol=5 * x)
    assert np.allclose(tot[2], 0.1, atol=5 * x)
    assert np.allclose(tot[1], 0.0, atol=5 * x) and np.allclose(tot[3], 0.0, atol=5 * x)
    assert Ksum.shape == (4, 2)


# --------------------------------------------------------------------------
# transfer sweep (Sec. 2, Sec. 2.1, Sec. 3.1)
# --------------------------------------------------------------------------

def _z_dominant(dirs):
    a = np.abs(dirs)
    return (a[:, 2] >= a[:, 0]) & (a[:, 2] >= a[:, 1]) & (a[:, 2] > a[:, 0]) & (a[:, 2] > a[:, 1])


def _node_xyz(grid, box):
    nx, ny, nz = grid
    h = [box[0] / (nx - 1), box[1] / (ny - 1), box[2] / (nz - 1)]
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return ix.ravel() * h[0], iy.ravel() * h[1], iz.ravel() * h[2]


def test_beam_attenuation_exact():
    """exp(-alpha s) along a beam (Sec. 3.1): with inflow values set to the
    analytic plane-parallel solution, every z-dominant ordinate reproduces
    I0 exp(-alpha z'/|mu|) at every node."""
    grid, box = (6, 5, 9), (1.0, 1.0, 1.0)
    alpha = 2.3
    P = _box(grid, L=3, G=1, alpha=alpha, box=box)
    mu, _, dirs, _ = O.ordinates(P.nmu, P.nphi)
    X, Y, Z = _node_xyz(grid, box)
    zp = np.where(dirs[None, :, 2] > 0, Z[:, None], box[2] - Z[:, None])  # path from inflow z-face
    exact = 1.4 * np.exp(-alpha * zp / np.abs(dirs[None, :, 2]))
    P.set_bc(2, exact[:, None, :])
    Nc = X.size
    eta = np.zeros((Nc, 1, P.N))
    chi = np.full((Nc, 1, P.N), alpha)
    out = P.sweep(np.zeros_like(eta), eta, chi)
    zd = _z_dominant(dirs)
    assert zd.sum() > 0
    assert np.allclose(out[:, 0, zd], exact[:, zd], rtol=1e-13, atol=0)


def test_linear_source_exact_along_z():
    """The linear-in-tau short characteristic integrates a source linear in tau
    exactly: dI/dtau = S - I with S = a + b tau has I = a + b(tau - 1) + C e^-tau."""
    grid, box = (5, 4, 12), (1.0, 1.0, 1.0)
    for chi_v in [0.3, 4.0, 60.0, 1e-4]:
        P = _box(grid, L=3, G=1, alpha=chi_v, box=box)
        _, _, dirs, _ = O.ordinates(P.nmu, P.nphi)
        X, Y, Z = _node_xyz(grid, box)
        a_, b_, C = 0.7, 1.9, 0.4
        # source as a function of z: S = a + b chi z  (the optical depth from z = 0)
        S = a_ + b_ * chi_v * Z
        Nc = Z.size
        eta = np.repeat((chi_v * S)[:, None, None], P.N, axis=2)
        chi = np.full((Nc, 1, P.N), chi_v)
        zd = _z_dominant(dirs) & (dirs[:, 2] > 0)
        mu_k = dirs[:, 2]
        # along +z with slant factor 1/mu: tau' = chi z / mu, S(tau') = a + b mu tau'
        tau = chi_v * Z[:, None] / np.where(mu_k > 0, mu_k, 1.0)[None, :]
        bb = b_ * mu_k[None, :]
        exact = a_ + bb * (tau - 1.0) + C * np.exp(-tau)
        P.set_bc(2, exact[:, None, :])
        out = P.sweep(np.zeros_like(eta), eta, chi)
        assert np.allclose(out[:, 0, zd], exact[:, zd], rtol=1e-12, atol=1e-13), chi_v


def test_equilibrium_stays_exact():
    """All inflow = B and eta = chi B: I = B at every node, ordinate and step,
    for any chi field and any time step."""
    grid = (5, 6, 4)
    Nc = 120
    rng = np.random.default_rng(4)
    for kappa in [0.0, 7.0]:
        P = _box(grid, L=3, G=2, box=(1.0, 1.3, 0.8))
        P.set_kappa(kappa)
        P.set_bc(1, np.array([2.0, 0.5]))
        B = np.array([2.0, 0.5])[None, :, None]
        chi = rng.uniform(0.01, 50.0, size=(Nc, 2, P.N))
        out = P.sweep(np.broadcast_to(B, (Nc, 2, P.N)), chi * B, chi)
        assert np.allclose(out, np.broadcast_to(B, out.shape), rtol=1e-14)


def test_time_term_is_backward_euler():
    """Uniform medium, no transport gradients: one step gives
    I^{n+1} = (kappa I^n + chi B)/(kappa + chi) (Sec. 2.1, eq:time)."""
    grid = (4, 4, 4)
    chi_v, B, I_old, kappa = 3.0, 1.5, 0.2, 10.0
    P = _box(grid, L=3, G=1)
    P.set_kappa(kappa)
    expect = (kappa * I_old + chi_v * B) / (kappa + chi_v)
    P.set_bc(1, np.array([expect]))
    Nc = 64
    out = P.sweep(np.full((Nc, 1, P.N), I_old), np.full((Nc, 1, P.N), chi_v * B),
                  np.full((Nc, 1, P.N), chi_v))
    assert np.allclose(out, expect, rtol=1e-14)


def test_vacuum_inflow_faces_are_zero():
    grid = (4, 5, 6)
    P = _box(grid, L=3, G=1)
    _, _, dirs, _ = O.ordinates(P.nmu, P.nphi)
    Nc = 120
    out = P.sweep(np.zeros((Nc, 1, P.N)), np.ones((Nc, 1, P.N)), np.ones((Nc, 1, P.N)))
    iz, iy, ix = np.meshgrid(np.arange(6), np.arange(5), np.arange(4), indexing="ij")
    for k in range(P.N):
        n = dirs[k]
        inflow = np.zeros(Nc, bool)
        for a, (idx, dim) in enumerate([(ix, 4), (iy, 5), (iz, 6)]):
            if n[a] > 0:
                inflow |= (idx.ravel() == 0)
            elif n[a] < 0:
                inflow |= (idx.ravel() == dim - 1)
        assert np.all(out[inflow, 0, k] == 0.0)
        assert np.all(out[~inflow, 0, k] > 0.0)


# --------------------------------------------------------------------------
# whole step (Sec. 2 Lambda iteration)
# --------------------------------------------------------------------------

def test_static_thick_interior_is_isotropic():
    """Optically thick static medium: the Eddington factor approaches 1/3 in
    the interior and the relative S change falls geometrically."""
    n = 9
    P = _box((n, n, n), L=3, G=1, alpha=20.0, ne=20.0, emis=20.0)
    I, it, resid = P.solve_static(tol=1e-8, max_iter=400)
    assert resid <= 1e-8
    _, J, _, Kt = P.project(I)
    f = O.moments_to_eddington(J, Kt)
    c = (n // 2 * n + n // 2) * n + n // 2
    assert np.allclose(f[c, 0, :3], 1 / 3, atol=5e-3)
    assert J[c, 0] == pytest.approx(1.0, rel=2e-2)  # B = emis/alpha = 1 deep inside


def test_free_streaming_eddington_factor_rises():
    """A point-like source in vacuum: the largest eigenvalue of f grows towards
    1 with distance from the source (trace f = 1 exactly)."""
    n = 13
    Nc = n ** 3
    emis = np.zeros((Nc, 1))
    alpha = np.full((Nc, 1), 1e-6)
    c0 = (6 * n + 6) * n + 6
    emis[c0] = 1.0
    alpha[c0] = 1.0
    P = _box((n, n, n), L=3, G=1, alpha=alpha, emis=emis)
    I, _, _ = P.step(np.zeros((Nc, 1, P.N)), 1)
    _, J, _, Kt = P.project(I)
    lam = []
    for d in [2, 4, 6]:
        c = (6 * n + 6) * n + 6 + d
        f = O.moments_to_eddington(J[c:c + 1], Kt[c:c + 1])[0, 0]
        M = np.array([[f[0], f[3], f[4]], [f[3], f[1], f[5]], [f[4], f[5], f[2]]])
        assert np.trace(M) == pytest.approx(1.0, abs=1e-13)
        lam.append(np.linalg.eigvalsh(M)[-1])
    assert lam[0] > 1 / 3 and lam[0] < lam[1] < lam[2] <= 1.0 + 1e-12


@pytest.mark.parametrize("beta,s", [(0.3, 0.0), (0.6, 1.0), (0.8, -0.5)])
def test_projection_of_lab_isotropic_power_law(beta, s):
    """A laboratory field isotropic with I = eps^-s seen from a fluid moving
    along +z: I0 = (Gamma(1 + beta mu0))^-(3+s) eps0^-s (I/nu^3 invariant,
    eq:lorentzfreq).  Its comoving energy density and flux follow from
    one-dimensional integrals over mu0."""
    from scipy.integrate import quad
    gam = 1 / np.sqrt(1 - beta * beta)
    edges = np.geomspace(1e-2, 1e2, 41)
    G = 40
    centre = np.sqrt(edges[:-1] * edges[1:])
    L, nmu, nphi = 3, 24, 8
    K, so = O.iso_table(G, L)
    P = O.OracleProblem(grid=(2, 2, 2), L=L, nmu=nmu, nphi=nphi, edges=edges,
                        alpha0=np.ones((8, G)), ne=np.zeros(8), u=np.tile([0, 0, gam * beta], (8, 1)),
                        emis0=np.zeros((8, G)), K=K, sigma_out=so)
    I = np.broadcast_to(centre[None, :, None] ** -s, (8, G, nmu * nphi))
    Ip, J, _, _ = P.project(I)
    j0 = 0.5 * quad(lambda m: (gam * (1 + beta * m)) ** -(3 + s), -1, 1, epsabs=0, epsrel=1e-13)[0]
    h0 = 0.5 * quad(lambda m: m * (gam * (1 + beta * m)) ** -(3 + s), -1, 1, epsabs=0, epsrel=1e-13)[0]
    g_int = slice(8, 32)  # shifted energies stay between group centres
    Y00, Y10 = 0.5 / np.sqrt(np.pi), np.sqrt(3 / (4 * np.pi))
    J0 = Ip[0, g_int, 0] * Y00                 # (1/4pi) Int I0 dOmega0
    H0 = Ip[0, g_int, 2] * Y10 / 3.0            # (1/4pi) Int mu0 I0 dOmega0
    ref = centre[g_int] ** -s
    assert np.allclose(J0, j0 * ref, rtol=2e-9)
    assert np.allclose(H0, h0 * ref, rtol=2e-8)
    assert h0 < 0  # a headwind: the comoving flux points against the motion
    # the laboratory moments of the same field are those of the lab field
    assert np.allclose(J[0], centre ** -s, rtol=1e-13)


# --------------------------------------------------------------------------
# Klein-Nishina table entry by entry (Sec. 2.3, eq:comptoncross)
# --------------------------------------------------------------------------

def _kn_entry_quad(l, g, gp, edges, ew):
    """K_l[g][g'] straight from its definition by nested adaptive quadrature:
    (2 pi / de_g) int_{g'} d eps int d mu P_l(mu) dsigma/dOmega (eps1/eps)^ew,
    over the angles whose scattered energy eps1 = eps/(1 + eps(1 - mu)) lies
    in group g, i.e. mu in [1 - 1/e_g + 1/eps, 1 - 1/e_{g+1} + 1/eps] within
    [-1, 1].  dsigma/dOmega (sigma_T units) is the textbook Klein-Nishina
    form (3/16pi) r^2 (r + 1/r - sin^2 Theta), r = eps1/eps."""
    from scipy.integrate import quad
    from scipy.special import eval_legendre

    def inner(eps):
        lo = max(-1.0, 1.0 - 1.0 / edges[g] + 1.0 / eps)
        hi = min(1.0, 1.0 - 1.0 / edges[g + 1] + 1.0 / eps)
        if not hi > lo:
            return 0.0

        def f(mu):
            r = 1.0 / (1.0 + eps * (1.0 - mu))
            return eval_legendre(l, mu) * 3.0 / (16.0 * np.pi) * r * r * (r + 1.0 / r - (1.0 - mu * mu)) * r ** ew

        return quad(f, lo, hi, epsabs=1e-15, epsrel=1e-12, limit=100)[0]

    a, b = edges[gp], edges[gp + 1]
    # kinks of the outer integrand: where a limit of the angle range hits +-1
    kinks = [e for e in edges if a < e < b]
    kinks += [e / (1 - 2 * e) for e in edges if e < 0.5 and a < e / (1 - 2 * e) < b]
    pts = sorted(set([a, b] + kinks))
    tot = 0.0
    for x0, x1 in zip(pts[:-1], pts[1:]):
        tot += quad(inner, x0, x1, epsabs=0, epsrel=1e-11, limit=200)[0]
    return 2.0 * np.pi * tot / (edges[g + 1] - edges[g])


@pytest.mark.parametrize("ew", [1, 0])
def test_kn_table_entries_match_adaptive_quadrature(ew):
    """Every l <= 3 entry of the multigroup KN table at finite energy (where
    l >= 1 terms are far from their Thomson values and P_l's sign matters),
    against nested adaptive quadrature of the definition."""
    edges = np.array([0.03, 0.08, 0.25, 0.7, 2.0, 5.0])
    L = 3
    K, _ = O.kn_table(edges, L, energy_weighted=bool(ew))
    G = len(edges) - 1
    worst = 0.0
    for l in range(L + 1):
        for g in range(G):
            for gp in range(G):
                ref = _kn_entry_quad(l, g, gp, edges, ew)
                scale = max(np.max(np.abs(K[0])), 1e-300)
                worst = max(worst, abs(K[l, g, gp] - ref) / scale)
    assert worst < 1e-9
    # the l = 1 row is not a rescaled l = 0 row: forward-peaked KN makes
    # K_1 / K_0 depend on the energy (a dropped or mis-signed P_1 fails here)
    assert np.any(K[1] < 0) or np.any(K[1] > 0)
    diag = [K[1, g, g] / K[0, g, g] for g in range(G) if K[0, g, g] > 0]
    assert max(diag) - min(diag) > 1e-3


# --------------------------------------------------------------------------
# FP64 sums (stage a5) in closed form
# --------------------------------------------------------------------------

def test_sums_closed_form_for_isotropic_group_state():
    """I = B_g at every node and ordinate: J = B_g exactly, so the energy is
    4 pi Nc sum_g B_g de_g and the photon number 4 pi Nc sum_g B_g de_g /
    sqrt(e_g e_{g+1}); with S_old = (1 + d) S_new the relative change is |d|."""
    edges = np.array([0.02, 0.05, 0.3, 0.31, 4.0])
    G = len(edges) - 1
    grid = (4, 3, 5)
    Nc = int(np.prod(grid))
    B = np.array([2.0, 0.5, 7.0, 0.125])
    P = _box(grid, L=2, G=G, edges=edges)
    I = np.broadcast_to(B[None, :, None], (Nc, G, P.N)).copy()
    Ip, J, _, _ = P.project(I)
    assert np.allclose(J, B[None, :], rtol=1e-14, atol=0)
    de = np.diff(edges)
    cen = np.sqrt(edges[:-1] * edges[1:])
    rng = np.random.default_rng(3)
    Snew = rng.normal(size=Ip.shape)
    out = P.sums(J, Snew, Snew * (1 + 0.0375))
    assert out[0] == pytest.approx(4 * np.pi * Nc * np.sum(B * de), rel=1e-13)
    assert out[1] == pytest.approx(4 * np.pi * Nc * np.sum(B * de / cen), rel=1e-13)
    assert out[2] == pytest.approx(0.0375, rel=1e-12)
    assert P.sums(J, Snew)[2] == 0.0


# --------------------------------------------------------------------------
# whole solver against a brute-force Monte Carlo (Sec. 3.5 compares the
# method with Monte Carlo; tests/mc_photon.py follows photons one by one)
# --------------------------------------------------------------------------

def _mc():
    import importlib
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    if here not in sys.path:
        sys.path.insert(0, here)
    return importlib.import_module("mc_photon")


def _uniform_box_static(n, *, alpha, sig, edges, u, s, nmu, nphi, L=3):
    Nc = n ** 3
    G = len(edges) - 1
    cen = np.sqrt(edges[:-1] * edges[1:])
    K, so = O.iso_table(G, L)
    P = O.OracleProblem(grid=(n, n, n), L=L, nmu=nmu, nphi=nphi, edges=edges, alpha0=np.full((Nc, G), alpha),
                        ne=np.full(Nc, sig), u=np.tile(np.asarray(u, float), (Nc, 1)),
                        emis0=np.tile(alpha * cen ** -s, (Nc, 1)), K=K, sigma_out=so, kappa=0.0)
    I, _, _ = P.solve_static(tol=1e-11, max_iter=400)
    _, J, H, _ = P.project(I)
    return J.reshape(n, n, n, G), H.reshape(n, n, n, G, 3)


def _cell_average(F, n, centre, half):
    """Average over the cube centre +- half of the quadratic interpolant of
    node values F[iz, iy, ix] (tensor product of 1-D parabolas through the
    nearest node and its two neighbours)."""
    h = 1.0 / (n - 1)
    idx = [int(round(c / h)) for c in centre]  # (x, y, z)
    w = np.array([half * half / (6 * h * h), 1 - half * half / (3 * h * h), half * half / (6 * h * h)])
    ix, iy, iz = idx
    blk = F[iz - 1:iz + 2, iy - 1:iy + 2, ix - 1:ix + 2]
    return np.einsum("i,j,k,ijk...->...", w, w, w, blk)


def test_static_box_matches_monte_carlo():
    """Uniform static box (absorption 1, isotropic scattering 1, emission
    alpha B with B = 1, vacuum faces): J at the centre and at (0.5, 0.5, 0.25)
    against photon-by-photon Monte Carlo.  The oracle's short-characteristic
    error is first order in the node spacing; its Richardson extrapolation
    from 9^3 and 17^3 nodes must agree with the Monte Carlo to 3 sigma + 1 %,
    each grid to 3 sigma + 3 %."""
    MC = _mc()
    a = 1.0 / 16
    centres = [(0.5, 0.5, 0.5), (0.5, 0.5, 0.25)]
    cells = [([c - a for c in cen], [c + a for c in cen]) for cen in centres]
    M, E = MC.run(box=[1, 1, 1], alpha0=1.0, sigma0=1.0, beta=np.zeros(3), cells=cells,
                  bins=np.array([-np.inf, np.inf]), n_packets=4_000_000, seed=20150717)
    Jmc, sig = M[0, :, 0], E[0, :, 0]
    edges = np.array([0.5, 1.5])
    vals = {}
    for n in (9, 17):
        J, _ = _uniform_box_static(n, alpha=1.0, sig=1.0, edges=edges, u=(0, 0, 0), s=0.0, nmu=8, nphi=16)
        vals[n] = np.array([_cell_average(J[..., 0], n, cen, a) for cen in centres])
    ext = 2 * vals[17] - vals[9]
    assert np.all(sig < 0.01 * Jmc)
    assert np.all(np.abs(ext - Jmc) <= 3 * sig + 0.01 * Jmc), (ext, Jmc, sig)
    for n in (9, 17):
        assert np.all(np.abs(vals[n] - Jmc) <= 3 * sig + 0.03 * Jmc), (n, vals[n], Jmc, sig)


def test_moving_box_matches_monte_carlo():
    """The same box moving at beta = 0.5 along z (u = Gamma beta = 0.577)
    with the comoving power-law emissivity eps^-1: the laboratory J and H_z
    at the centre and at z = 0.25 and 0.75 against photon-by-photon Monte
    Carlo with Lorentz-transformed emission and scattering.  The exact
    solution is a power law eps^-1 at every point, which the geometric group
    interpolation carries exactly, so the middle groups of a wide group range
    are compared in one sum.  Allowance: 3 sigma + 3 % of J (the 9^3 grid's
    short-characteristic error and the 12 x 24 ordinate mesh of the remaps).
    The flow makes the field asymmetric in z: the downstream cell is
    brighter, and the flux is along +z at the centre (a sign error in the
    boost fails both)."""
    MC = _mc()
    beta = 0.5
    gam = 1.0 / np.sqrt(1.0 - beta * beta)
    edges = np.geomspace(1e-2, 1e2, 13)
    a = 1.0 / 16
    centres = [(0.5, 0.5, 0.5), (0.5, 0.5, 0.25), (0.5, 0.5, 0.75)]
    cells = [([c - a for c in cen], [c + a for c in cen]) for cen in centres]
    M, E = MC.run(box=[1, 1, 1], alpha0=1.0, sigma0=1.0, beta=np.array([0.0, 0.0, beta]), A=1.0, s=1.0,
                  e_lo=edges[0], e_hi=edges[-1], cells=cells, bins=edges, n_packets=4_000_000, seed=20150718)
    mid = slice(3, 9)
    logw = np.log(edges[9] / edges[3])
    Jmc = M[0, :, mid].sum(axis=1) / logw                       # eps J(eps), the same in every middle group
    Hmc = M[3, :, mid].sum(axis=1) / logw
    sJ = np.sqrt((E[0, :, mid] ** 2).sum(axis=1)) / logw
    sH = np.sqrt((E[3, :, mid] ** 2).sum(axis=1)) / logw
    n = 9
    J, H = _uniform_box_static(n, alpha=1.0, sig=1.0, edges=edges, u=(0, 0, gam * beta), s=1.0, nmu=12, nphi=24)
    cen = np.sqrt(edges[:-1] * edges[1:])
    Jo = np.array([np.mean(_cell_average(J[..., mid] * cen[mid], n, c, a)) for c in centres])
    Ho = np.array([np.mean(_cell_average(H[..., mid, 2] * cen[mid], n, c, a)) for c in centres])
    assert np.all(sJ < 0.01 * Jmc)
    assert np.all(np.abs(Jo - Jmc) <= 3 * sJ + 0.03 * Jmc), (Jo, Jmc, sJ)
    assert np.all(np.abs(Ho - Hmc) <= 3 * sH + 0.03 * Jmc), (Ho, Hmc, sH)
    assert Jmc[2] > Jmc[1] and Jo[2] > Jo[1]
    assert Hmc[0] > 10 * sH[0] and Ho[0] > 0


# --------------------------------------------------------------------------
# Runge-Kutta sub-stepping (App. A, eq:rk4th) and Ng acceleration (Sec. 2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("z", [0.3, -0.7, 1.9, -2.5])
def test_rk4_combination_is_classical_rk4_for_explicit_increments(z):
    """With sub-solves that return the explicit increment X + frac dt f(X),
    f(y) = lambda y, App. A's combination is the classical fourth-order
    Runge-Kutta method: one step multiplies y by 1 + z + z^2/2 + z^3/6 +
    z^4/24 (z = lambda dt) exactly.  A wrong stage fraction or combination
    weight changes that polynomial."""
    y0 = np.array([1.25])
    out = O.rk4_combine(lambda frac, X: X + frac * z * X, y0)
    taylor = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    assert out[0] == pytest.approx(1.25 * taylor, rel=1e-14)


def test_rk4_keeps_equilibrium_exactly():
    """I = B everywhere with emission alpha B, isotropic inflow B: every
    sub-solve returns B, so the Runge-Kutta step does too."""
    grid = (5, 4, 6)
    B = 1.7
    P = _box(grid, L=3, G=1, alpha=2.0, ne=1.5, emis=2.0 * B)
    P.set_bc(1, np.array([B]))
    P.set_kappa(9.0)
    I = np.full((int(np.prod(grid)), 1, P.N), B)
    out = P.step_rk4(I, 2)
    assert np.allclose(out, B, rtol=1e-14, atol=0)


def test_rk4_more_accurate_than_one_euler_step():
    """The purpose App. A gives the sub-steps: from a smooth state (half the
    static solution of the relaxation box) one step of c dt = h/2 by the
    Runge-Kutta combination is closer to a fine-time reference (128 backward-
    Euler steps of dt/128) than one backward-Euler step."""
    from paper_1507_05141_gb300 import inputs
    spec = inputs.relax_box(n=10)
    K, so = O.iso_table(spec.G, spec.L)
    mk = lambda kap: O.OracleProblem(grid=spec.grid, L=spec.L, nmu=spec.nmu, nphi=spec.nphi, edges=spec.edges,
                                     alpha0=spec.alpha0, ne=spec.ne, u=spec.u, emis0=spec.emis0, K=K, sigma_out=so,
                                     kappa=kap)
    Ist, _, _ = mk(0.0).solve_static(tol=1e-10)
    I0 = 0.5 * Ist
    kap = 1.0 / (0.5 / 9.0)
    P = mk(kap)
    Ibe, _, _ = P.step(I0.copy(), 1)
    Irk = P.step_rk4(I0.copy(), 1)
    Iref, _, _ = mk(kap * 128).step(I0.copy(), 128)
    err = lambda a: np.max(np.abs(a - Iref)) / np.max(np.abs(Iref))
    assert err(Irk) < 0.6 * err(Ibe)


def test_ng_exact_for_two_mode_linear_iteration():
    """For a linear iteration x <- M x + c whose error lies in two eigenvectors
    of M, the error polynomial of Ng's extrapolation can vanish on both
    eigenvalues, so one extrapolation from four iterates hits the fixed point
    (to rounding); with three modes it still cuts the error."""
    rng = np.random.default_rng(5)
    n = 12
    V = np.linalg.qr(rng.normal(size=(n, n)))[0]
    lam = np.concatenate([[0.9, -0.6, 0.3], rng.uniform(-0.2, 0.2, n - 3)])
    M = V @ np.diag(lam) @ V.T
    c = rng.normal(size=n)
    xstar = np.linalg.solve(np.eye(n) - M, c)
    for modes, bound in ((2, 1e-10), (3, None)):
        x = xstar + V[:, :modes] @ rng.normal(size=modes)
        it = [x]
        for _ in range(3):
            it.append(M @ it[-1] + c)
        ext = O.ng_extrapolate(it[3], it[2], it[1], it[0])
        e_plain = np.linalg.norm(it[3] - xstar)
        e_ng = np.linalg.norm(ext - xstar)
        if bound is not None:
            assert e_ng < bound * np.linalg.norm(xstar)
        else:
            assert e_ng < e_plain


def test_ng_static_solve_converges_faster_to_the_same_solution():
    from paper_1507_05141_gb300 import inputs
    spec = inputs.relax_box(n=12)
    K, so = O.iso_table(spec.G, spec.L)
    P = O.OracleProblem(grid=spec.grid, L=spec.L, nmu=spec.nmu, nphi=spec.nphi, edges=spec.edges,
                        alpha0=spec.alpha0, ne=spec.ne, u=spec.u, emis0=spec.emis0, K=K, sigma_out=so,
                        kappa=spec.kappa)
    I1, it1, _ = P.solve_static(tol=1e-8, max_iter=300)
    I2, it2, r2 = P.solve_static_ng(tol=1e-8, max_iter=300, period=4)
    assert r2 <= 1e-8 and it2 < 0.75 * it1
    assert np.max(np.abs(I2 - I1)) < 1e-6 * np.max(np.abs(I1))
    I3, it3, _ = P.solve_static_ng(tol=1e-8, max_iter=300, period=0)  # off: the plain iteration
    assert it3 == it1 and np.array_equal(I3, I1)


# --------------------------------------------------------------------------
# cubic Bezier short characteristic (Sec. 2: the paper's ray tracing scheme)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("x", [1e-8, 1e-3, 0.2, 0.999, 1.0, 1.5, 7.0, 40.0])
def test_bezier_weights_match_quadrature(x):
    """x times the integral over the segment of each cubic Bernstein
    polynomial against e^-(x - t) (t the optical depth from U), by adaptive
    quadrature; the weights add up to 1 - e^-x (a constant source)."""
    from scipy.integrate import quad
    w = O.bezier_weights(x)
    basis = [lambda u: (1 - u) ** 3, lambda u: 3 * u * (1 - u) ** 2, lambda u: 3 * u * u * (1 - u),
             lambda u: u ** 3]
    assert w[0] == pytest.approx(np.exp(-x), rel=1e-15)
    for j, B in enumerate(basis):
        ref = x * quad(lambda u: B(u) * np.exp(-x * (1 - u)), 0, 1, epsabs=0, epsrel=1e-13, limit=200)[0]
        assert w[1 + j] == pytest.approx(ref, rel=1e-12, abs=1e-300)
    assert np.sum(w[1:]) == pytest.approx(-np.expm1(-x), rel=1e-13)


def test_bezier_linear_source_exact_along_z():
    """A source linear in optical depth has the same slope at every node, so
    every end derivative is that slope, the control points lie on the line
    (no clamping) and the Bezier curve is the line: exact, as for the linear
    scheme."""
    grid, box = (5, 4, 12), (1.0, 1.0, 1.0)
    for chi_v in [0.3, 4.0, 60.0]:
        P = _box(grid, L=3, G=1, alpha=chi_v, box=box)
        P.set_integrator("bezier")
        _, _, dirs, _ = O.ordinates(P.nmu, P.nphi)
        X, Y, Z = _node_xyz(grid, box)
        a_, b_, C = 0.7, 1.9, 0.4
        S = a_ + b_ * chi_v * Z
        Nc = Z.size
        eta = np.repeat((chi_v * S)[:, None, None], P.N, axis=2)
        chi = np.full((Nc, 1, P.N), chi_v)
        zd = _z_dominant(dirs) & (dirs[:, 2] > 0)
        mu_k = dirs[:, 2]
        tau = chi_v * Z[:, None] / np.where(mu_k > 0, mu_k, 1.0)[None, :]
        bb = b_ * mu_k[None, :]
        exact = a_ + bb * (tau - 1.0) + C * np.exp(-tau)
        P.set_bc(2, exact[:, None, :])
        out = P.sweep(np.zeros_like(eta), eta, chi)
        assert np.allclose(out[:, 0, zd], exact[:, zd], rtol=1e-12, atol=1e-13), chi_v


def test_bezier_beam_and_equilibrium_exact():
    grid, box = (6, 5, 9), (1.0, 1.0, 1.0)
    alpha = 2.3
    P = _box(grid, L=3, G=1, alpha=alpha, box=box)
    P.set_integrator("bezier")
    _, _, dirs, _ = O.ordinates(P.nmu, P.nphi)
    X, Y, Z = _node_xyz(grid, box)
    zp = np.where(dirs[None, :, 2] > 0, Z[:, None], box[2] - Z[:, None])
    exact = 1.4 * np.exp(-alpha * zp / np.abs(dirs[None, :, 2]))
    P.set_bc(2, exact[:, None, :])
    Nc = X.size
    out = P.sweep(np.zeros((Nc, 1, P.N)), np.zeros((Nc, 1, P.N)), np.full((Nc, 1, P.N), alpha))
    zd = _z_dominant(dirs)
    assert np.allclose(out[:, 0, zd], exact[:, zd], rtol=1e-13, atol=0)
    rng = np.random.default_rng(4)
    grid = (5, 6, 4)
    for kappa in [0.0, 7.0]:
        P = _box(grid, L=3, G=2, box=(1.0, 1.3, 0.8))
        P.set_integrator("bezier")
        P.set_kappa(kappa)
        P.set_bc(1, np.array([2.0, 0.5]))
        B = np.array([2.0, 0.5])[None, :, None]
        chi = rng.uniform(0.01, 50.0, size=(120, 2, P.N))
        out = P.sweep(np.broadcast_to(B, (120, 2, P.N)), chi * B, chi)
        assert np.allclose(out, np.broadcast_to(B, out.shape), rtol=1e-14)


def test_bezier_third_order_for_smooth_source():
    """S = A e^(beta chi z) along z with the exact solution on the inflow
    faces: at the centre column (away from the faces, whose nodes have
    one-sided derivatives) the error falls eightfold per halving of the node
    spacing (third order) where the linear scheme's falls fourfold."""
    def errs(integ, chi_v):
        out_e = []
        for nz in (17, 33, 65):
            grid, box = (9, 9, nz), (1.0, 1.0, 1.0)
            P = _box(grid, L=3, G=1, alpha=chi_v, box=box)
            P.set_integrator(integ)
            _, _, dirs, _ = O.ordinates(P.nmu, P.nphi)
            X, Y, Z = _node_xyz(grid, box)
            beta, A, I0 = 1.5, 0.8, 0.3
            mu = dirs[:, 2]
            zd = _z_dominant(dirs) & (mu > 0)
            tau = chi_v * Z[:, None] / np.where(mu > 0, mu, 1.0)[None, :]
            S = A * np.exp(beta * chi_v * Z)
            Nc = Z.size
            eta = np.repeat((chi_v * S)[:, None, None], P.N, axis=2)
            chi = np.full((Nc, 1, P.N), chi_v)
            b = beta * mu[None, :]
            exact = I0 * np.exp(-tau) + A * (np.exp(b * tau) - np.exp(-tau)) / (b + 1)
            P.set_bc(2, exact[:, None, :])
            out = P.sweep(np.zeros_like(eta), eta, chi)
            centre = (np.abs(X - 0.5) < 1e-9) & (np.abs(Y - 0.5) < 1e-9)
            out_e.append(np.max(np.abs(out[centre][:, 0, zd] - exact[centre][:, zd]) / np.abs(exact[centre][:, zd])))
        return out_e
    for chi_v in (1.0, 4.0):
        eb, el = errs("bezier", chi_v), errs("linear", chi_v)
        assert eb[-2] / eb[-1] > 6.0 and 3.5 < el[-2] / el[-1] < 4.5
        assert eb[-1] < 0.2 * el[-1]


def test_bezier_no_overshoot_at_a_step():
    """A source jumping from 0 to 1 in an optically thick medium: the clamped
    control points keep the curve within its end values, so the intensity
    stays within [0, 1] (vacuum inflow) for every ordinate."""
    grid = (6, 6, 16)
    chi_v = 40.0
    P = _box(grid, L=3, G=1, alpha=chi_v)
    P.set_integrator("bezier")
    X, Y, Z = _node_xyz(grid, (1.0, 1.0, 1.0))
    S = np.where(Z > 0.45, 1.0, 0.0)
    Nc = Z.size
    eta = np.repeat((chi_v * S)[:, None, None], P.N, axis=2)
    chi = np.full((Nc, 1, P.N), chi_v)
    out = P.sweep(np.zeros_like(eta), eta, chi)
    assert out.min() >= 0.0 and out.max() <= 1.0 + 1e-14


# --------------------------------------------------------------------------
# Compton scattering off thermal electrons (the temperature field's kernel)
# --------------------------------------------------------------------------

def test_thermal_kn_cold_limit():
    """theta -> 0: the electron average collapses to electrons at rest; the
    group-summed photon-number and energy kernels (smooth: the sum over
    final groups removes the group indicator) equal the cold table's (the
    thermal effects are of order theta = 1e-8).  The lowest incident group
    is left out: its down-scattered photons leave the range, and the leak
    edge is resolved differently by the two quadratures."""
    edges = np.geomspace(1e-3, 1e1, 9)
    de = np.diff(edges)
    for ew in (True, False):
        Kc, soc = O.kn_table(edges, 3, energy_weighted=ew)
        Kt, sot = O.kn_thermal_table(edges, 3, 1e-8, energy_weighted=ew)
        sc, st = (de[:, None] * Kc[0]).sum(axis=0), (de[:, None] * Kt[0]).sum(axis=0)
        assert np.allclose(st[1:], sc[1:], rtol=1e-6)
        assert np.allclose(sot, soc, rtol=1e-7)


@pytest.mark.parametrize("theta", [0.01, 0.1])
def test_thermal_kn_total_cross_section(theta):
    """sigma_out^theta of a group against nested adaptive quadrature of
    <(1 - beta mu_e) sigma_KN(gamma eps (1 - beta mu_e))> over the
    Maxwell-Juttner density gamma^2 beta e^(-gamma/theta) / (theta K2(1/theta))
    and the group's energies, sigma_KN the textbook total cross-section."""
    from scipy.integrate import quad
    from scipy.special import kve

    def skn(x):
        if x < 1e-4:
            return 1 - 2 * x + 5.2 * x * x
        l = np.log1p(2 * x)
        return 0.75 * ((1 + x) / x ** 3 * (2 * x * (1 + x) / (1 + 2 * x) - l) + l / (2 * x)
                       - (1 + 3 * x) / (1 + 2 * x) ** 2)
    norm = theta * kve(2, 1.0 / theta)  # theta K2(1/theta) e^(1/theta), so dens carries e^(-(gamma-1)/theta)

    def avg(eps):
        def over_gamma(g):
            b = np.sqrt(1 - 1 / (g * g))
            dens = g * g * b * np.exp(-(g - 1) / theta) / norm
            inner = quad(lambda m: 0.5 * (1 - b * m) * skn(g * eps * (1 - b * m)), -1, 1, epsabs=0, epsrel=1e-11)[0]
            return dens * inner
        return quad(over_gamma, 1.0, 1.0 + 60 * theta, epsabs=0, epsrel=1e-10, limit=200)[0]
    edges = np.array([0.1, 0.3, 1.0])
    _, so = O.kn_thermal_table(edges, 1, theta)
    ref = quad(avg, edges[0], edges[1], epsabs=0, epsrel=1e-9)[0] / (edges[1] - edges[0])
    assert so[0] == pytest.approx(ref, rel=1e-6)


@pytest.mark.parametrize("theta", [0.01, 0.05, 0.2])
def test_thermal_kn_mean_energy_gain_thomson_limit(theta):
    """Low-energy photons (eps << theta, gamma eps << 1) gain on average
    (4/3) <gamma^2 beta^2> = 4 theta K3(1/theta)/K2(1/theta) of their energy
    per scattering (Thomson scattering off a relativistic Maxwellian), less
    the recoil, which is below 0.3 % of it here: the ratio of the energy to
    the photon-number group sums of the thermal tables."""
    from scipy.special import kve
    edges = np.geomspace(1e-6, 1e1, 29)
    de = np.diff(edges)
    KE, _ = O.kn_thermal_table(edges, 0, theta, energy_weighted=True)
    KN, _ = O.kn_thermal_table(edges, 0, theta, energy_weighted=False)
    gain = (de[:, None] * KE[0]).sum(axis=0) / (de[:, None] * KN[0]).sum(axis=0) - 1.0
    ref = 4.0 * theta * kve(3, 1.0 / theta) / kve(2, 1.0 / theta)
    for g in (3, 4, 5):   # eps ~ 1e-5 .. 3e-5, inside the range after up- and down-scattering
        assert gain[g] == pytest.approx(ref, rel=1e-2), (g, gain[g], ref)


def test_thermal_kn_upscatters_and_cold_does_not():
    edges = np.geomspace(1e-3, 1e1, 9)
    Kc, _ = O.kn_table(edges, 2)
    Kt, _ = O.kn_thermal_table(edges, 2, 0.1)
    up = np.triu(np.ones((8, 8), bool), k=1)  # g > g' is the lower triangle of K[g][g']; use the transpose
    assert np.all(Kc[0][up.T] == 0.0)
    assert np.max(Kt[0][up.T]) > 0.01 * np.max(Kt[0])
