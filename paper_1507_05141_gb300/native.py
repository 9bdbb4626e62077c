"""Thin ctypes binding of the C ABI in ``include/shdom_gb300.h``.

Argument marshalling only: every stage of the step runs in the library's CUDA
kernels.  Importing this module does not need a GPU; loading the library
(:func:`lib`) raises if it has not been built, and every call raises
:class:`ShdError` on a non-zero status.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_STATE, ERR_NAN, ERR_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
FP64, FP32, MIXED = 0, 1, 2
SCAT_ISO, SCAT_THOMSON, SCAT_KN, SCAT_TABLE, SCAT_KN_THERMAL = 1, 2, 3, 4, 5
THERMAL_N = 13  # temperature grid of the thermal kernel: 10^(-3 + i/4)
BC_VACUUM, BC_ISO, BC_FULL = 0, 1, 2
TIME_EULER, TIME_RK4 = 0, 1
SC_LINEAR, SC_BEZIER = 0, 1
PRECISIONS = {"fp64": FP64, "fp32": FP32, "mixed": MIXED}
SCATTERING = {"iso": SCAT_ISO, "thomson": SCAT_THOMSON, "kn": SCAT_KN, "table": SCAT_TABLE,
              "kn_thermal": SCAT_KN_THERMAL}
STAGES = ("project", "source", "sums", "sh2lab", "sweep")

_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p
_i = ctypes.c_int
_ll = ctypes.c_longlong

# name -> (restype, argtypes)
_SIGS = {
    "shd_create": (_i, [ctypes.POINTER(_vp), _i, _i]),
    "shd_destroy": (None, [_vp]),
    "shd_last_error": (ctypes.c_char_p, []),
    "shd_set_grid": (_i, [_vp, _i, _i, _i, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "shd_set_angles": (_i, [_vp, _i, _i, _i]),
    "shd_set_groups": (_i, [_vp, _i, _dp]),
    "shd_set_fields": (_i, [_vp, _dp, _dp, _dp, _dp, _dp]),
    "shd_get_thermal_tables": (_i, [_vp, _dp, _dp]),
    "shd_set_scattering": (_i, [_vp, _i, _dp, _dp]),
    "shd_get_scattering": (_i, [_vp, _dp, _dp]),
    "shd_set_boundary": (_i, [_vp, _i, _dp]),
    "shd_set_time": (_i, [_vp, ctypes.c_double]),
    "shd_set_state": (_i, [_vp, _dp]),
    "shd_get_state": (_i, [_vp, _dp]),
    "shd_step": (_i, [_vp, _i, _vp]),
    "shd_zero_state": (_i, [_vp]),
    "shd_solve_static": (_i, [_vp, ctypes.c_double, _i, ctypes.POINTER(_i), _dp]),
    "shd_get_moments": (_i, [_vp, _dp, _dp, _dp, _dp]),
    "shd_get_sums": (_i, [_vp, _dp, _dp, _dp]),
    "shd_stage_project": (_i, [_vp, _dp, _dp, _dp, _dp, _dp]),
    "shd_stage_source": (_i, [_vp, _dp, _dp]),
    "shd_stage_sh2lab": (_i, [_vp, _dp, _dp, _dp]),
    "shd_stage_sweep": (_i, [_vp, _dp, _dp, _dp, _dp]),
    "shd_set_state_dev": (_i, [_vp, _vp, _vp]),
    "shd_get_state_dev": (_i, [_vp, _vp, _vp]),
    "shd_get_sizes": (_i, [_vp, ctypes.POINTER(_ll), ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "shd_device_bytes": (_ll, [_vp]),
    "shd_set_timing": (_i, [_vp, _i]),
    "shd_get_timing": (_i, [_vp, _dp, ctypes.POINTER(_ll)]),
    "shd_launch_count": (ctypes.c_ulonglong, []),
    "shd_batch_create": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(_vp)]),
    "shd_batch_step": (_i, [_vp, _i, _vp]),
    "shd_get_moments_dev": (_i, [_vp, _vp, _vp]),
    "shd_batch_set_sweep_mode": (_i, [_vp, _i]),
    "shd_batch_destroy": (None, [_vp]),
    "shd_check_bounded_wait": (_i, [_vp, _ll]),
    "shd_set_ng": (_i, [_vp, _i]),
    "shd_set_integrator": (_i, [_vp, _i]),
    "shd_set_source_path": (_i, [_vp, _i]),
    "shd_get_source_path": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_float),
                                 ctypes.POINTER(ctypes.c_float)]),
    "shd_get_transform_path": (_i, [_vp, ctypes.POINTER(_i)]),
    "shd_set_time_scheme": (_i, [_vp, _i]),
    "shd_set_sweep_schedule": (_i, [_vp, _i, _i]),
    "shd_get_sweep_schedule": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                                    ctypes.POINTER(ctypes.c_float)]),
    "shd_project_noalloc": (_i, [_vp, _vp, _vp, _vp]),
    "shd_noalloc_last_error": (ctypes.c_char_p, []),
}

_lib = None


class ShdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"shd error {code}: {msg}")
        self.code = code


def library_path():
    return _build.lib_path()


def lib(build_if_missing: bool = False):
    """Load the CUDA library.  Raises if it is missing (no fallback)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
            _build.build()
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy


def torch_stream():
    """torch's current CUDA stream as a handle the library can order against
    (torch reports the legacy default stream as 0, which the C ABI reads as
    'the context's own stream')."""
    import torch
    h = torch.cuda.current_stream().cuda_stream
    return h if h else CUDA_STREAM_LEGACY


def exported_symbols():
    return list(_SIGS)


def launch_count():
    """Kernels the native library has launched in this process so far."""
    return int(lib().shd_launch_count())


def _check(rc):
    if rc != 0:
        raise ShdError(rc, lib().shd_last_error().decode())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class Solver:
    """One problem on one GPU: owns a library context."""

    def __init__(self, device: int = 0, precision: str | int = "fp64"):
        self._L = lib()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        h = _vp()
        _check(self._L.shd_create(ctypes.byref(h), int(device), prec))
        self._h = h
        self.precision = prec
        self.grid = None
        self.N = self.G = self.NLM = None

    def close(self):
        if getattr(self, "_h", None):
            self._L.shd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- set-up ---------------------------------------------------------------
    def set_grid(self, nx, ny, nz, lx=1.0, ly=1.0, lz=1.0):
        _check(self._L.shd_set_grid(self._h, nx, ny, nz, lx, ly, lz))
        self.grid = (nx, ny, nz)
        self.Nc = nx * ny * nz

    def set_angles(self, L, nmu, nphi):
        _check(self._L.shd_set_angles(self._h, L, nmu, nphi))
        self.N = nmu * nphi
        self.NLM = (L + 1) ** 2
        self.L = L

    def set_groups(self, edges):
        e = _f64(edges)
        _check(self._L.shd_set_groups(self._h, len(e) - 1, _ptr(e)))
        self.G = len(e) - 1

    def set_fields(self, alpha0, ne, u, emis0, theta_e=None):
        a, n, uu, em = _f64(alpha0), _f64(ne), _f64(u), _f64(emis0)
        th = _f64(theta_e) if theta_e is not None else None
        _check(self._L.shd_set_fields(self._h, _ptr(a), _ptr(n), _ptr(uu), _ptr(em), _ptr(th)))

    def set_scattering(self, kind, K=None, sigma_out=None):
        k = SCATTERING[kind] if isinstance(kind, str) else int(kind)
        K_, s_ = _f64(K), _f64(sigma_out)
        _check(self._L.shd_set_scattering(self._h, k, _ptr(K_), _ptr(s_)))

    def get_thermal_tables(self):
        """(K_th [13][L+1][G][G], sigma_out_th [13][G]) of the thermal kernel."""
        K = np.zeros((THERMAL_N, self.L + 1, self.G, self.G))
        s = np.zeros((THERMAL_N, self.G))
        _check(self._L.shd_get_thermal_tables(self._h, _ptr(K), _ptr(s)))
        return K, s

    def get_scattering(self):
        K = np.zeros((self.L + 1, self.G, self.G))
        s = np.zeros(self.G)
        _check(self._L.shd_get_scattering(self._h, _ptr(K), _ptr(s)))
        return K, s

    def set_boundary(self, mode, data=None):
        d = _f64(data)
        _check(self._L.shd_set_boundary(self._h, int(mode), _ptr(d)))

    def set_time(self, kappa):
        _check(self._L.shd_set_time(self._h, float(kappa)))

    def set_state(self, I):
        a = _f64(I)
        _check(self._L.shd_set_state(self._h, _ptr(a)))

    def zero_state(self):
        _check(self._L.shd_zero_state(self._h))

    def set_state_dev(self, tensor, stream=None):
        """State from a contiguous FP64 CUDA tensor in the [c][g][k] layout
        (read on ``stream``, default torch's current stream)."""
        import torch
        assert tensor.dtype == torch.float64 and tensor.is_cuda and tensor.is_contiguous()
        assert tensor.numel() == self.Nc * self.G * self.N
        st = torch_stream() if stream is None else stream
        _check(self._L.shd_set_state_dev(self._h, ctypes.c_void_p(tensor.data_ptr()), ctypes.c_void_p(st)))

    def get_state_dev(self, tensor, stream=None):
        """State into a contiguous FP64 CUDA tensor in the [c][g][k] layout
        (written on ``stream``, default torch's current stream)."""
        import torch
        assert tensor.dtype == torch.float64 and tensor.is_cuda and tensor.is_contiguous()
        assert tensor.numel() == self.Nc * self.G * self.N
        st = torch_stream() if stream is None else stream
        _check(self._L.shd_get_state_dev(self._h, ctypes.c_void_p(tensor.data_ptr()), ctypes.c_void_p(st)))

    def get_state(self):
        out = np.zeros((self.Nc, self.G, self.N))
        _check(self._L.shd_get_state(self._h, _ptr(out)))
        return out

    @classmethod
    def from_spec(cls, spec, device=0, precision="fp64", scattering=None):
        s = cls(device, precision)
        s.set_grid(*spec.grid, *spec.box)
        s.set_angles(spec.L, spec.nmu, spec.nphi)
        s.set_groups(spec.edges)
        s.set_scattering(scattering or spec.scattering)
        s.set_fields(spec.alpha0, spec.ne, spec.u, spec.emis0, spec.extra.get("theta_e"))
        s.set_time(spec.kappa)
        return s

    # -- the step -------------------------------------------------------------
    def step(self, nsteps=1, stream=None):
        """Enqueue nsteps source iterations on ``stream`` (a cudaStream_t as int,
        or None for the library's own stream)."""
        _check(self._L.shd_step(self._h, int(nsteps), stream))

    def solve_static(self, tol=1e-6, max_iter=500):
        it = _i()
        r = ctypes.c_double()
        _check(self._L.shd_solve_static(self._h, float(tol), int(max_iter), ctypes.byref(it), ctypes.byref(r)))
        return it.value, r.value

    def moments(self, with_sh=False):
        nCG = self.Nc * self.G
        J = np.zeros((self.Nc, self.G))
        H = np.zeros((self.Nc, self.G, 3))
        K = np.zeros((self.Nc, self.G, 6))
        Ish = np.zeros((self.Nc, self.G, self.NLM)) if with_sh else None
        _check(self._L.shd_get_moments(self._h, _ptr(J), _ptr(H), _ptr(K), _ptr(Ish)))
        del nCG
        return (J, H, K, Ish) if with_sh else (J, H, K)

    def moments_dev(self, mom, stream=None):
        """J, H, K of the current state into the CUDA tensor ``mom`` (float64,
        [Nc][G][10] contiguous, on this solver's device): J, H_x, H_y, H_z,
        K_xx, K_yy, K_zz, K_xy, K_xz, K_yz, as moments() returns them."""
        import torch
        if (mom.dtype != torch.float64 or not mom.is_cuda or not mom.is_contiguous()
                or mom.numel() != self.Nc * self.G * 10):
            raise ValueError("mom must be a contiguous float64 CUDA tensor of Nc*G*10 elements")
        _check(self._L.shd_get_moments_dev(self._h, mom.data_ptr(), stream))

    def sums(self):
        e, p, r = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(self._L.shd_get_sums(self._h, ctypes.byref(e), ctypes.byref(p), ctypes.byref(r)))
        return e.value, p.value, r.value

    # -- single stages ----------------------------------------------------------
    def stage_project(self, I):
        a = _f64(I)
        Ish = np.zeros((self.Nc, self.G, self.NLM))
        J = np.zeros((self.Nc, self.G))
        H = np.zeros((self.Nc, self.G, 3))
        K = np.zeros((self.Nc, self.G, 6))
        _check(self._L.shd_stage_project(self._h, _ptr(a), _ptr(Ish), _ptr(J), _ptr(H), _ptr(K)))
        return Ish, J, H, K

    def stage_source(self, Ish):
        a = _f64(Ish)
        out = np.zeros((self.Nc, self.G, self.NLM))
        _check(self._L.shd_stage_source(self._h, _ptr(a), _ptr(out)))
        return out

    def stage_sh2lab(self, Ssh):
        a = _f64(Ssh)
        eta = np.zeros((self.Nc, self.G, self.N))
        chi = np.zeros((self.Nc, self.G, self.N))
        _check(self._L.shd_stage_sh2lab(self._h, _ptr(a), _ptr(eta), _ptr(chi)))
        return eta, chi

    def stage_sweep(self, I_old, eta, chi):
        a, e, c = _f64(I_old), _f64(eta), _f64(chi)
        out = np.zeros((self.Nc, self.G, self.N))
        _check(self._L.shd_stage_sweep(self._h, _ptr(a), _ptr(e), _ptr(c), _ptr(out)))
        return out

    # -- timing -------------------------------------------------------------------
    def set_timing(self, on=True):
        _check(self._L.shd_set_timing(self._h, int(bool(on))))

    def timing(self):
        ms = np.zeros(5)
        n = _ll()
        _check(self._L.shd_get_timing(self._h, _ptr(ms), ctypes.byref(n)))
        return dict(zip(STAGES, ms)), n.value

    def project_noalloc(self, Ish, mom, stream=None):
        """Stage a1 of the current state into caller-owned CUDA tensors
        ``Ish`` [c][g][p] and ``mom`` [c][g][10] (working precision) without
        any allocation in the library."""
        rc = self._L.shd_project_noalloc(self._h, ctypes.c_void_p(Ish.data_ptr()), ctypes.c_void_p(mom.data_ptr()),
                                         None if stream is None else ctypes.c_void_p(stream))
        if rc != 0:
            raise ShdError(rc, self._L.shd_noalloc_last_error().decode() or "shd_project_noalloc failed")

    def set_integrator(self, name):
        """'linear' (linear-in-tau short characteristic) or 'bezier' (the
        paper's cubic Bezier short characteristic)."""
        code = {"linear": SC_LINEAR, "bezier": SC_BEZIER}[name] if isinstance(name, str) else int(name)
        _check(self._L.shd_set_integrator(self._h, code))

    def set_source_path(self, path):
        """Source pass of a group-mixing kernel in MIXED: 'auto' (timed),
        'cuda' (CUDA cores) or 'tensor' (tcgen05)."""
        code = {"auto": 0, "cuda": 1, "tensor": 2}[path] if isinstance(path, str) else int(path)
        _check(self._L.shd_set_source_path(self._h, code))

    def source_path(self):
        """(path in use: 0 untimed, 1 CUDA cores, 2 tensor cores; ms CUDA cores; ms tensor cores)."""
        p, a, b = _i(), ctypes.c_float(), ctypes.c_float()
        _check(self._L.shd_get_source_path(self._h, ctypes.byref(p), ctypes.byref(a), ctypes.byref(b)))
        return p.value, a.value, b.value

    def transform_path(self):
        """Kernels carrying the transforms: 0 CUDA cores, 1 tensor-core tiles,
        2 tensor-core segments through TMA, 3 the segment kernels with
        cp.async loads and direct stores (rows not multiples of 4 nodes)."""
        p = _i()
        _check(self._L.shd_get_transform_path(self._h, ctypes.byref(p)))
        return p.value

    def set_ng(self, period=4):
        """Ng acceleration of solve_static every `period` (>= 4) iterations; 0 = off."""
        _check(self._L.shd_set_ng(self._h, int(period)))

    def set_time_scheme(self, scheme):
        """'euler' (one backward-Euler source iteration per step) or 'rk4'
        (the four sub-solves of the paper's App. A)."""
        code = {"euler": TIME_EULER, "rk4": TIME_RK4}[scheme] if isinstance(scheme, str) else int(scheme)
        _check(self._L.shd_set_time_scheme(self._h, code))

    def set_sweep_schedule(self, C=0, NT=0):
        """Force the single-precision sweep's cluster split (C CTAs of NT
        threads a plane); C = 0 returns to the timed automatic choice."""
        _check(self._L.shd_set_sweep_schedule(self._h, int(C), int(NT)))

    def sweep_schedule(self):
        """((C, NT) in use, [(C, NT, ms), ...] of the last timed choice)."""
        C, NT, n = _i(), _i(), _i()
        buf = (ctypes.c_float * 48)()
        _check(self._L.shd_get_sweep_schedule(self._h, ctypes.byref(C), ctypes.byref(NT), ctypes.byref(n), buf))
        rows = [(int(buf[3 * i]), int(buf[3 * i + 1]), float(buf[3 * i + 2])) for i in range(n.value)]
        return (C.value, NT.value), rows

    def check_bounded_wait(self, polls=1000):
        """Run the bounded-wait failure path once; returns the status code
        (SHD_ERR_TIMEOUT expected) and the library's message."""
        rc = self._L.shd_check_bounded_wait(self._h, int(polls))
        return rc, self._L.shd_last_error().decode()

    def device_bytes(self):
        return int(self._L.shd_device_bytes(self._h))


class Batch:
    """Independent problems stepped together: each batch step is one CUDA
    graph launch with one time step per problem (see shd_batch_step).  The
    solvers stay usable for reading results and must outlive the batch."""

    def __init__(self, solvers):
        self._L = lib()
        self._solvers = list(solvers)
        arr = (_vp * len(self._solvers))(*[s._h for s in self._solvers])
        h = _vp()
        _check(self._L.shd_batch_create(ctypes.byref(h), len(self._solvers), arr))
        self._h = h

    def step(self, nsteps=1, stream=None):
        """Enqueue nsteps steps of every problem on ``stream`` (a cudaStream_t
        as int, or None for the first problem's own stream)."""
        _check(self._L.shd_batch_step(self._h, int(nsteps), stream))

    def set_sweep_mode(self, mode):
        """0 (default): each problem sweeps in its own launches; 1: the
        sweeps of every problem that allows it in one persistent launch per
        kernel variant."""
        _check(self._L.shd_batch_set_sweep_mode(self._h, int(mode)))

    def close(self):
        if getattr(self, "_h", None):
            self._L.shd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
