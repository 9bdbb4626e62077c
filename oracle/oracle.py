"""Python entry to the plain FP64 CPU oracle (``shdom_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this module; the CUDA library never does.

The C source is compiled with gcc on first use (or by ``build()``) into
``oracle/_build/liboracle.so``.  Every function takes and returns float64
numpy arrays in the oracle's canonical layouts:

* discrete-ordinate arrays ``[c][g][k]`` (node, group, ordinate),
* spherical-harmonic arrays ``[c][g][p]`` with ``p = l*l + l + m``,
* ``c = (iz*ny + iy)*nx + ix``, ``k = a*nphi + b``.

Each wrapper names the paper passage its C function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "shdom_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


class Problem(ctypes.Structure):
    """Mirror of ``orc_problem`` (held by :class:`OracleProblem`)."""

    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
        ("L", ctypes.c_int), ("nmu", ctypes.c_int), ("nphi", ctypes.c_int),
        ("G", ctypes.c_int),
        ("edges", _dp), ("alpha0", _dp), ("ne", _dp), ("u", _dp), ("emis0", _dp),
        ("K", _dp), ("sigma_out", _dp),
        ("kappa", ctypes.c_double),
        ("bc_mode", ctypes.c_int), ("bc", _dp),
        ("integrator", ctypes.c_int),
        ("nth", ctypes.c_int), ("th_lg0", ctypes.c_double), ("th_dlg", ctypes.c_double),
        ("K_th", _dp), ("so_th", _dp), ("theta_e", _dp),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, -O2, no host-specific flags)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            for name in ("orc_project", "orc_source", "orc_sh2lab", "orc_sweep", "orc_sweep_pairs", "orc_step"):
                getattr(_lib, name).restype = ctypes.c_int
            _lib.orc_lab_to_comoving.restype = ctypes.c_double
            _lib.orc_comoving_to_lab.restype = ctypes.c_double
            _lib.orc_interp_angle.restype = ctypes.c_double
            _lib.orc_interp_angle.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_long, _dp]
            _lib.orc_interp_freq.restype = ctypes.c_double
            _lib.orc_interp_freq.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_long, ctypes.c_double, ctypes.c_int]
    return _lib


def _p(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------
# quadrature, harmonics, Lorentz (Sec. 2.2, Sec. 2.3)
# ----------------------------------------------------------------------------

def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().orc_gauss_legendre(ctypes.c_int(n), _p(x), _p(w))
    return x, w


def ordinates(nmu: int, nphi: int):
    """(mu, wmu, dirs[k][3], W[k]) of the Gauss-Legendre x uniform-phi set."""
    mu = np.zeros(nmu)
    wmu = np.zeros(nmu)
    dirs = np.zeros((nmu * nphi, 3))
    W = np.zeros(nmu * nphi)
    lib().orc_ordinates(ctypes.c_int(nmu), ctypes.c_int(nphi), _p(mu), _p(wmu), _p(dirs), _p(W))
    return mu, wmu, dirs, W


def ylm(L: int, mu: float, phi: float) -> np.ndarray:
    """Real orthonormal Y_p(mu, phi), p = l*l + l + m, l <= L (Sec. 2.3)."""
    Y = np.zeros((L + 1) ** 2)
    lib().orc_ylm(ctypes.c_int(L), ctypes.c_double(mu), ctypes.c_double(phi), _p(Y))
    return Y


def ylm_table(L: int, nmu: int, nphi: int) -> np.ndarray:
    mu, _, _, _ = ordinates(nmu, nphi)
    out = np.zeros((nmu * nphi, (L + 1) ** 2))
    for a in range(nmu):
        for b in range(nphi):
            out[a * nphi + b] = ylm(L, mu[a], 2.0 * np.pi * b / nphi)
    return out


def lab_to_comoving(u, n):
    """(n0, nu0/nu) for laboratory direction n (eq:lorentzfreq, eq:lorentzray)."""
    u = _f64(u); n = _f64(n)
    n0 = np.zeros(3)
    r = lib().orc_lab_to_comoving(_p(u), _p(n), _p(n0))
    return n0, r


def comoving_to_lab(u, n0):
    """(n, nu/nu0) for comoving direction n0 (inverse boost)."""
    u = _f64(u); n0 = _f64(n0)
    n = np.zeros(3)
    q = lib().orc_comoving_to_lab(_p(u), _p(n0), _p(n))
    return n, q


def interp_angle(nmu, nphi, mu, F, n):
    mu = _f64(mu); F = _f64(F); n = _f64(n)
    return lib().orc_interp_angle(nmu, nphi, _p(mu), _p(F), 1, _p(n))


def interp_freq(edges, F, eps, nearest_outside=False):
    edges = _f64(edges); F = _f64(F)
    return lib().orc_interp_freq(len(edges) - 1, _p(edges), _p(F), 1, float(eps), int(nearest_outside))


def bezier_weights(x: float):
    """(e^-x, wU, wCU, wCP, wP) of the cubic Bezier short characteristic
    over optical depth x (Sec. 2; the C oracle's orc_bezier_weights)."""
    w = np.zeros(5)
    lib().orc_bezier_weights(ctypes.c_double(float(x)), _p(w))
    return w


def kn_table(edges, L: int, energy_weighted: bool = True):
    """(K[l][g][g'], sigma_out[g']) of the multigroup Klein-Nishina kernel
    (Sec. 2.3, eq:comptoncross), in sigma_T units."""
    edges = _f64(edges)
    G = len(edges) - 1
    K = np.zeros((L + 1, G, G))
    so = np.zeros(G)
    lib().orc_kn_table(ctypes.c_int(G), _p(edges), ctypes.c_int(L), ctypes.c_int(int(energy_weighted)),
                       _p(K), _p(so))
    return K, so


def kn_thermal_table(edges, L: int, theta: float, energy_weighted: bool = True):
    """(K[l][g][g'], sigma_out[g']) of Compton scattering off isotropic
    Maxwell-Juttner electrons at temperature theta = kT_e/m_e c^2 (the
    reading of Sec. 2.3 for a temperature field: the cold kernel averaged
    over the electrons), in sigma_T units, by the oracle's product
    quadrature."""
    edges = _f64(edges)
    G = len(edges) - 1
    K = np.zeros((L + 1, G, G))
    so = np.zeros(G)
    lib().orc_kn_thermal_table(ctypes.c_int(G), _p(edges), ctypes.c_int(L), ctypes.c_int(int(energy_weighted)),
                               ctypes.c_double(float(theta)), _p(K), _p(so))
    return K, so


# the temperature grid of the library's thermal Compton kernel:
# theta_i = 10^(THERMAL_LG0 + i THERMAL_DLG), i < THERMAL_N
THERMAL_LG0, THERMAL_DLG, THERMAL_N = -3.0, 0.25, 13


def thermal_tables(edges, L: int, lg0=THERMAL_LG0, dlg=THERMAL_DLG, n=THERMAL_N):
    """The thermal kernels (energy form) and out-scattering cross-sections on
    the temperature grid 10^(lg0 + i dlg), i < n: ([n][L+1][G][G], [n][G])."""
    Ks, sos = [], []
    for i in range(n):
        K, so = kn_thermal_table(edges, L, 10.0 ** (lg0 + i * dlg))
        Ks.append(K)
        sos.append(so)
    return np.array(Ks), np.array(sos)


def thomson_table(G: int, L: int):
    """Thomson kernel: diagonal, K_0 = 1, K_2 = (1/2)/5 (Sec. 2.3, Thomson
    phase function 3/4(1 + cos^2) = 1 + P_2/2)."""
    K = np.zeros((L + 1, G, G))
    K[0] = np.eye(G)
    if L >= 2:
        K[2] = np.eye(G) * 0.1
    return K, np.ones(G)


def iso_table(G: int, L: int):
    """Isotropic scattering: only K_0 = 1 (chi_l = delta_l0)."""
    K = np.zeros((L + 1, G, G))
    K[0] = np.eye(G)
    return K, np.ones(G)


# ----------------------------------------------------------------------------
# the problem and the step
# ----------------------------------------------------------------------------

class OracleProblem:
    """Holds the numpy arrays behind an ``orc_problem`` so they stay alive."""

    def __init__(self, *, grid, L, nmu, nphi, edges, alpha0, ne, u, emis0, K, sigma_out,
                 kappa=0.0, bc_mode=0, bc=None, box=(1.0, 1.0, 1.0), thermal=None):
        nx, ny, nz = grid
        self.grid = (nx, ny, nz)
        self.Nc = nx * ny * nz
        self.L, self.nmu, self.nphi = L, nmu, nphi
        self.N = nmu * nphi
        self.NLM = (L + 1) ** 2
        self.edges = _f64(edges)
        self.G = len(self.edges) - 1
        self.alpha0 = _f64(alpha0).reshape(self.Nc, self.G)
        self.ne = _f64(ne).reshape(self.Nc)
        self.u = _f64(u).reshape(self.Nc, 3)
        self.emis0 = _f64(emis0).reshape(self.Nc, self.G)
        self.K = _f64(K).reshape(L + 1, self.G, self.G)
        self.sigma_out = _f64(sigma_out).reshape(self.G)
        self.bc = _f64(bc)
        self.s = Problem()
        s = self.s
        s.nx, s.ny, s.nz = nx, ny, nz
        s.lx, s.ly, s.lz = box
        s.L, s.nmu, s.nphi, s.G = L, nmu, nphi, self.G
        s.edges, s.alpha0, s.ne, s.u = _p(self.edges), _p(self.alpha0), _p(self.ne), _p(self.u)
        s.emis0, s.K, s.sigma_out = _p(self.emis0), _p(self.K), _p(self.sigma_out)
        s.kappa = float(kappa)
        s.bc_mode = int(bc_mode)
        s.bc = _p(self.bc) if self.bc is not None else None
        if thermal is not None:
            # {"theta_e": [Nc], "K_th": [nth][L+1][G][G], "so_th": [nth][G], "lg0": .., "dlg": ..}
            self.theta_e = _f64(thermal["theta_e"]).reshape(self.Nc)
            self.K_th = _f64(thermal["K_th"])
            self.so_th = _f64(thermal["so_th"])
            s.nth = int(self.so_th.shape[0])
            s.th_lg0, s.th_dlg = float(thermal["lg0"]), float(thermal["dlg"])
            s.K_th, s.so_th, s.theta_e = _p(self.K_th), _p(self.so_th), _p(self.theta_e)

    def set_integrator(self, name):
        """'linear' (linear-in-tau short characteristic) or 'bezier' (the
        cubic Bezier short characteristic the paper uses, Sec. 2)."""
        self.s.integrator = {"linear": 0, "bezier": 1}[name]

    def set_kappa(self, kappa):
        self.s.kappa = float(kappa)

    def set_bc(self, mode, data=None):
        self.bc = _f64(data)
        self.s.bc_mode = int(mode)
        self.s.bc = _p(self.bc) if self.bc is not None else None

    # -- stages --------------------------------------------------------------
    def project(self, I):
        """Stage a1: lab -> comoving remap, SH projection, lab moments (Sec. 2.2, 2.3)."""
        I = _f64(I).reshape(self.Nc, self.G, self.N)
        Ip = np.zeros((self.Nc, self.G, self.NLM))
        J = np.zeros((self.Nc, self.G))
        H = np.zeros((self.Nc, self.G, 3))
        Kt = np.zeros((self.Nc, self.G, 6))
        lib().orc_project(ctypes.byref(self.s), _p(I), _p(Ip), _p(J), _p(H), _p(Kt))
        return Ip, J, H, Kt

    def source(self, Ip):
        """Stage a2: comoving SH source (Sec. 2.3)."""
        Ip = _f64(Ip).reshape(self.Nc, self.G, self.NLM)
        Sp = np.zeros_like(Ip)
        lib().orc_source(ctypes.byref(self.s), _p(Ip), _p(Sp))
        return Sp

    def sh2lab(self, Sp):
        """Stage a3: SH -> comoving ordinates -> laboratory (eta_lab, chi_lab) (Sec. 2.2)."""
        Sp = _f64(Sp).reshape(self.Nc, self.G, self.NLM)
        eta = np.zeros((self.Nc, self.G, self.N))
        chi = np.zeros((self.Nc, self.G, self.N))
        lib().orc_sh2lab(ctypes.byref(self.s), _p(Sp), _p(eta), _p(chi))
        return eta, chi

    def sweep(self, In, eta, chi):
        """Stage a4: short-characteristic sweep with the time term (Sec. 2, 2.1)."""
        In = _f64(In).reshape(self.Nc, self.G, self.N)
        eta = _f64(eta).reshape(self.Nc, self.G, self.N)
        chi = _f64(chi).reshape(self.Nc, self.G, self.N)
        out = np.zeros_like(In)
        lib().orc_sweep(ctypes.byref(self.s), _p(In), _p(eta), _p(chi), _p(out))
        return out

    def sweep_pairs(self, pairs, In, eta, chi):
        """Stage a4 for chosen (ordinate k, group g) pairs only (Sec. 2, 2.1):
        In, eta, chi and the result are [pair][c] (a pair's column over every
        node), for problems whose full DO arrays do not fit in host memory."""
        pairs = np.asarray(pairs, dtype=np.int32).reshape(-1, 2)
        kk = np.ascontiguousarray(pairs[:, 0])
        gg = np.ascontiguousarray(pairs[:, 1])
        n = len(pairs)
        In = _f64(In).reshape(n, self.Nc)
        eta = _f64(eta).reshape(n, self.Nc)
        chi = _f64(chi).reshape(n, self.Nc)
        out = np.zeros_like(In)
        ip = ctypes.POINTER(ctypes.c_int)
        lib().orc_sweep_pairs(ctypes.byref(self.s), ctypes.c_int(n), kk.ctypes.data_as(ip), gg.ctypes.data_as(ip),
                              _p(In), _p(eta), _p(chi), _p(out))
        return out

    def sums(self, J, Snew, Sold=None):
        """Stage a5: energy, photon number, relative S change (FP64)."""
        out = np.zeros(3)
        lib().orc_sums(ctypes.byref(self.s), _p(_f64(J)), _p(_f64(Snew)), _p(_f64(Sold)), _p(out))
        return out

    def step(self, I, nsteps=1, Sprev=None):
        """``nsteps`` source iterations / time steps; returns (I, Sprev, sums)."""
        I = np.array(I, dtype=np.float64).reshape(self.Nc, self.G, self.N)
        if Sprev is None:
            Sprev = np.zeros((self.Nc, self.G, self.NLM))
        sums = np.zeros(3)
        for _ in range(nsteps):
            rc = lib().orc_step(ctypes.byref(self.s), _p(I), _p(Sprev), _p(sums))
            if rc != 0:
                raise MemoryError("oracle step failed")
        return I, Sprev, sums

    def solve(self, frac, I):
        """One source iteration of eq:time over the time step frac * dt from
        I (kappa = 1/(c dt) divided by frac): the paper's script-I."""
        kap = self.s.kappa
        self.s.kappa = kap / frac
        try:
            out, _, _ = self.step(np.array(I, dtype=np.float64), 1)
        finally:
            self.s.kappa = kap
        return out

    def step_rk4(self, I, nsteps=1):
        """``nsteps`` time steps by the Runge-Kutta sub-stepping of App. A."""
        I = np.array(I, dtype=np.float64).reshape(self.Nc, self.G, self.N)
        for _ in range(nsteps):
            I = rk4_combine(self.solve, I)
        return I

    def solve_static_ng(self, tol=1e-6, max_iter=500, period=4, I=None):
        """Lambda iteration of the static problem (kappa = 0) from I (default
        0) with Ng acceleration of the source (Sec. 2): each iteration projects
        I, forms S^n, reports the relative change against the source used in
        the previous iteration; at n >= 4 with n - (last extrapolation) >=
        period, S^n is replaced by ng_extrapolate(S^n, S^(n-1), S^(n-2),
        S^(n-3)); then S is transformed to the ordinates and swept.  Stops
        after iteration n > 1 whose relative change is <= tol.  Returns
        (I, iterations, residual)."""
        kap = self.s.kappa
        self.s.kappa = 0.0
        if I is None:
            I = np.zeros((self.Nc, self.G, self.N))
        I = np.array(I, dtype=np.float64)
        hist = {}
        Sprev = None
        last = 0
        it = 0
        resid = np.inf
        try:
            while it < max_iter:
                n = it + 1
                Ip, J, _, _ = self.project(I)
                S = self.source(Ip)
                resid = self.sums(J, S, Sprev)[2]
                if period and n >= 4 and n - last >= period:
                    x = ng_extrapolate(S, hist[n - 1], hist[n - 2], hist[n - 3])
                    if x is not None:
                        S = x
                        last = n
                hist[n] = S
                hist.pop(n - 3, None)
                eta, chi = self.sh2lab(S)
                I = self.sweep(I, eta, chi)
                Sprev = S
                it += 1
                if it > 1 and resid <= tol:
                    break
        finally:
            self.s.kappa = kap
        return I, it, resid

    def solve_static(self, tol=1e-6, max_iter=500, I=None):
        """Lambda iteration from I (default 0) with kappa = 0 until the relative
        S change is <= tol (Sec. 2)."""
        kap = self.s.kappa
        self.s.kappa = 0.0
        if I is None:
            I = np.zeros((self.Nc, self.G, self.N))
        Sprev = np.zeros((self.Nc, self.G, self.NLM))
        it = 0
        resid = np.inf
        try:
            while it < max_iter:
                I, Sprev, sums = self.step(I, 1, Sprev)
                it += 1
                resid = sums[2]
                if it > 1 and resid <= tol:
                    break
        finally:
            self.s.kappa = kap
        return I, it, resid


def rk4_combine(solve, I):
    """One time step by the Runge-Kutta sub-stepping of App. A (eq:rk4th).

    ``solve(frac, X)`` returns the solution of eq:time over the time step
    frac * dt from the intensity X (the paper's script-I(frac dt, X)).  In the
    paper's order: dI1 = I(dt/6, I) - I, I1 = I + 3 dI1; dI2 = I(dt/3, I1) -
    I1, I2 = I + 3/2 dI2; dI3 = I(dt/3, I2) - I2, I3 = I + 3 dI3; dI4 =
    I(dt/6, I3) - I3; the new intensity is I + dI1 + dI2 + dI3 + dI4."""
    d1 = solve(1.0 / 6.0, I) - I
    I1 = I + 3.0 * d1
    d2 = solve(1.0 / 3.0, I1) - I1
    I2 = I + 1.5 * d2
    d3 = solve(1.0 / 3.0, I2) - I2
    I3 = I + 3.0 * d3
    d4 = solve(1.0 / 6.0, I3) - I3
    return I + d1 + d2 + d3 + d4


def ng_extrapolate(x0, x1, x2, x3):
    """Ng's acceleration of an iteration (Sec. 2 cites it for the Lambda
    iteration; Ng 1974), from the newest iterate x0 and the three before it:
    with Q1 = x0 - 2 x1 + x2, Q2 = x0 - x1 - x2 + x3, Q3 = x0 - x1, the
    coefficients (a, b) minimise |Q3 - a Q1 - b Q2|^2 (normal equations of
    the five inner products), and the extrapolated iterate is
    (1 - a - b) x0 + a x1 + b x2.  Returns None when the 2 x 2 system is
    singular (det <= 1e-14 <Q1,Q1><Q2,Q2>)."""
    q1 = (x0 - 2.0 * x1 + x2).ravel()
    q2 = (x0 - x1 - x2 + x3).ravel()
    q3 = (x0 - x1).ravel()
    a11, a12, a22 = q1 @ q1, q1 @ q2, q2 @ q2
    b1, b2 = q1 @ q3, q2 @ q3
    det = a11 * a22 - a12 * a12
    if not (np.isfinite(det) and det > 1e-14 * a11 * a22):
        return None
    a = (b1 * a22 - b2 * a12) / det
    b = (b2 * a11 - b1 * a12) / det
    return (1.0 - a - b) * x0 + a * x1 + b * x2


def moments_to_eddington(J, Kt, floor=1e-300):
    """Eddington tensor f_ij = K_ij / J (lab frame), 0 where J <= floor."""
    J = np.asarray(J)
    f = np.zeros_like(Kt)
    ok = J > floor
    f[ok] = Kt[ok] / J[ok][..., None]
    return f
