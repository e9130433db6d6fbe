"""FP64 CPU oracle of the WaterLily time step.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
cpu_baseline / reference legs are the only callers.  The product path (the CUDA
library and its binding) never imports this package.

The arithmetic lives in ``wl_oracle.cpp`` (plain double-precision loops); this
module builds it with the host compiler and wraps it with ctypes.  Each wrapper
names the routine of the paper it stands for (Section 2 and Table 2 of the
WaterLily paper); the readings where the paper is silent are listed in the C++
header comment.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wl_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.c_double
_I = ctypes.c_int
_P = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (OpenMP on).  Returns the library path."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        sig = {
            "or_create": (_P, [_I, _IP, _D, _DP, ctypes.c_uint, _I, _DP, _D, _D, _D, _I, _D]),
            "or_destroy": (None, [_P]),
            "or_nlevels": (_I, [_P]),
            "or_level_dims": (None, [_P, _I, _IP]),
            "or_get_level_L": (None, [_P, _I, _DP]),
            "or_get_mu0": (None, [_P, _DP]),
            "or_get_mu1": (None, [_P, _DP]),
            "or_set_u": (None, [_P, _DP]),
            "or_get_u": (None, [_P, _DP]),
            "or_npad": (ctypes.c_long, [_P]),
            "or_get_u_padded": (None, [_P, _DP]),
            "or_set_p": (None, [_P, _DP]),
            "or_get_p": (None, [_P, _DP]),
            "or_get_dt": (_D, [_P]),
            "or_set_dt": (None, [_P, _D]),
            "or_get_time": (_D, [_P]),
            "or_last_iters": (_I, [_P]),
            "or_last_resid": (_D, [_P]),
            "or_set_ic": (None, [_P, _I, _D]),
            "or_convdiff": (None, [_P, _DP, _DP]),
            "or_bdim_stage": (None, [_P, _I, _D, _DP, _DP, _DP]),
            "or_divergence": (None, [_P, _DP]),
            "or_poisson_apply": (None, [_P, _I, _DP, _DP]),
            "or_poisson_diag": (None, [_P, _I, _DP]),
            "or_pcg": (_I, [_P, _I, _DP, _DP, _D, _I, _DP]),
            "or_dense_solve": (_I, [_P, _I, _DP, _DP]),
            "or_vcycle": (_D, [_P, _DP, _DP, _I, _I]),
            "or_rb_sweep": (None, [_P, _I, _DP, _DP]),
            "or_project": (None, [_P, _D, _D, _D, _I, _I]),
            "or_step": (None, [_P, _I, _D, _I, _D, _I]),
            "or_cfl": (_D, [_P]),
            "or_forces": (None, [_P, _DP]),
            "or_set_body_nodes": (None, [_P, _DP]),
            "or_viscous_force": (None, [_P, _DP]),
            "or_kinetic_energy": (_D, [_P]),
            "or_K0": (_D, [_D]),
            "or_K1": (_D, [_D]),
            "or_face_value": (_D, [_D, _D, _D]),
            "or_psi": (_D, [_D]),
            "or_sdf": (_D, [_P, _DP, _DP]),
            "or_convdiff_adjoint": (None, [_P, _DP, _DP, _DP]),
            "or_stage_adjoint": (None, [_P, _I, _D, _DP, _DP, _DP, _DP, _DP, _DP, _DP]),
            "or_project_adjoint": (None, [_P, _DP, _D, _D, _D, _DP, _DP, _DP, _DP]),
            "or_force_adjoint": (None, [_P, _DP, _DP, _DP, _DP, _DP]),
            "or_moments_adjoint": (None, [_P, _DP, _DP, _DP, _DP]),
            "or_rollout_grad": (_I, [_P, _I, _D, _D, _DP, _DP, _DP]),
            "or_set_exit": (_I, [_P, _I]),
            "or_get_exit": (None, [_P, _DP]),
            "or_set_exit_plane": (None, [_P, _DP]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def K0(s: float) -> float:
    """Zeroth moment of the cosine kernel (BDIM, Section 2)."""
    return _load().or_K0(float(s))


def K1(s: float) -> float:
    """First moment of the cosine kernel over [s, 1] (BDIM, Section 2)."""
    return _load().or_K1(float(s))


def face_value(u: float, c: float, d: float) -> float:
    """Koren-limited kappa=1/3 face value from upwind u, centre c, downwind d."""
    return _load().or_face_value(float(u), float(c), float(d))


def psi(r: float) -> float:
    """Koren limiter psi(r) = max(0, min(2r, (2+r)/3, 2))."""
    return _load().or_psi(float(r))


class Oracle:
    """One simulation held by the oracle.

    dims are given x first; fields are returned as numpy arrays shaped
    (D, [nz,] ny, nx) for velocity and ([nz,] ny, nx) for scalars.
    """

    def __init__(self, dims, nu, U=None, periodic=0, body=None, eps=1.0, advect=True,
                 dt_cap=10.0):
        self.lib = _load()
        self.D = len(dims)
        self.dims = tuple(int(d) for d in dims)
        U = list(U) if U is not None else [0.0] * self.D
        U = (U + [0.0] * 3)[:3]
        kind, center, r1, r2 = 0, [0.0, 0.0, 0.0], 0.0, 0.0
        nodes = None
        if body is not None:
            kind = int(body.get("kind", 1))
            if kind == 3:  # signed distance sampled at the nodes, shape reversed(dims + 1)
                nodes = np.ascontiguousarray(body["nodes"], dtype=np.float64).reshape(-1)
                kind = 0
            else:
                center = (list(body["center"]) + [0.0] * 3)[:3]
                r1 = float(body.get("radius", 0.0))
                r2 = float(body.get("radius2", 0.0))
        d3 = (ctypes.c_int * 3)(*(list(self.dims) + [1] * (3 - self.D)))
        self.h = self.lib.or_create(self.D, d3, float(nu), (ctypes.c_double * 3)(*U),
                                    int(periodic), kind, (ctypes.c_double * 3)(*center),
                                    r1, r2, float(eps), int(bool(advect)), float(dt_cap))
        if not self.h:
            raise ValueError("oracle: bad arguments")
        if nodes is not None:
            want = int(np.prod([d + 1 for d in self.dims]))
            if nodes.size != want:
                raise ValueError(f"oracle: {want} node values expected, got {nodes.size}")
            self.lib.or_set_body_nodes(self.h, _dp(nodes))
        self.ncell = int(np.prod(self.dims))
        self.shape = tuple(reversed(self.dims))
        # body parameters the adjoint differentiates: circle/sphere (R, c_0, ..); torus (R, r, c_x, c_y, c_z)
        self.n_theta = 5 if kind == 2 else self.D + 1

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.or_destroy(h)
            self.h = None

    # ----- geometry / hierarchy
    def nlevels(self) -> int:
        return self.lib.or_nlevels(self.h)

    def level_dims(self, l):
        d = (ctypes.c_int * 3)()
        self.lib.or_level_dims(self.h, l, d)
        return tuple(d[i] for i in range(self.D))

    def level_L(self, l):
        dims = self.level_dims(l)
        n = int(np.prod(dims))
        out = np.zeros(self.D * n)
        self.lib.or_get_level_L(self.h, l, _dp(out))
        return out.reshape((self.D,) + tuple(reversed(dims)))

    def mu0(self):
        out = np.zeros(self.D * self.ncell)
        self.lib.or_get_mu0(self.h, _dp(out))
        return out.reshape((self.D,) + self.shape)

    def mu1(self):
        out = np.zeros(self.D * self.D * self.ncell)
        self.lib.or_get_mu1(self.h, _dp(out))
        return out.reshape((self.D, self.D) + self.shape)

    def sdf(self, x):
        xx = np.zeros(3)
        xx[: len(x)] = x
        n = np.zeros(3)
        d = self.lib.or_sdf(self.h, _dp(xx), _dp(n))
        return d, n[: self.D]

    # ----- state
    def set_u(self, u):
        a = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        assert a.size == self.D * self.ncell
        self.lib.or_set_u(self.h, _dp(a))

    def get_u(self):
        out = np.zeros(self.D * self.ncell)
        self.lib.or_get_u(self.h, _dp(out))
        return out.reshape((self.D,) + self.shape)

    def get_u_padded(self):
        npad = self.lib.or_npad(self.h)
        out = np.zeros(self.D * npad)
        self.lib.or_get_u_padded(self.h, _dp(out))
        pshape = tuple(n + 4 for n in reversed(self.dims))
        return out.reshape((self.D,) + pshape)

    def set_p(self, p):
        a = np.ascontiguousarray(p, dtype=np.float64).reshape(-1)
        assert a.size == self.ncell
        self.lib.or_set_p(self.h, _dp(a))

    def get_p(self):
        out = np.zeros(self.ncell)
        self.lib.or_get_p(self.h, _dp(out))
        return out.reshape(self.shape)

    @property
    def dt(self) -> float:
        return self.lib.or_get_dt(self.h)

    @dt.setter
    def dt(self, v: float):
        self.lib.or_set_dt(self.h, float(v))

    @property
    def time(self) -> float:
        return self.lib.or_get_time(self.h)

    def set_ic(self, kind=0, amp=1.0):
        """kind 0: uniform U; kind 1: Taylor-Green vortex of amplitude amp."""
        self.lib.or_set_ic(self.h, int(kind), float(amp))

    # ----- routines of the step (Table 2)
    def convdiff(self, u):
        a = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        out = np.zeros(self.D * self.ncell)
        self.lib.or_convdiff(self.h, _dp(a), _dp(out))
        return out.reshape((self.D,) + self.shape)

    def bdim_stage(self, stage, dt, u0, u1=None):
        a = np.ascontiguousarray(u0, dtype=np.float64).reshape(-1)
        b = None if u1 is None else np.ascontiguousarray(u1, dtype=np.float64).reshape(-1)
        out = np.zeros(self.D * self.ncell)
        self.lib.or_bdim_stage(self.h, int(stage), float(dt), _dp(a),
                               _dp(b) if b is not None else None, _dp(out))
        return out.reshape((self.D,) + self.shape)

    def divergence(self):
        out = np.zeros(self.ncell)
        self.lib.or_divergence(self.h, _dp(out))
        return out.reshape(self.shape)

    def poisson_apply(self, x, level=0):
        dims = self.level_dims(level)
        a = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        out = np.zeros(int(np.prod(dims)))
        self.lib.or_poisson_apply(self.h, level, _dp(a), _dp(out))
        return out.reshape(tuple(reversed(dims)))

    def poisson_diag(self, level=0):
        dims = self.level_dims(level)
        out = np.zeros(int(np.prod(dims)))
        self.lib.or_poisson_diag(self.h, level, _dp(out))
        return out.reshape(tuple(reversed(dims)))

    def pcg(self, z, x0=None, tol=1e-10, maxit=100000, level=0):
        dims = self.level_dims(level)
        n = int(np.prod(dims))
        x = np.zeros(n) if x0 is None else np.ascontiguousarray(x0, dtype=np.float64).reshape(-1).copy()
        zz = np.ascontiguousarray(z, dtype=np.float64).reshape(-1)
        res = ctypes.c_double(0.0)
        it = self.lib.or_pcg(self.h, level, _dp(x), _dp(zz), float(tol), int(maxit), ctypes.byref(res))
        return x.reshape(tuple(reversed(dims))), it, res.value

    def dense_solve(self, z, level=0):
        dims = self.level_dims(level)
        n = int(np.prod(dims))
        x = np.zeros(n)
        zz = np.ascontiguousarray(z, dtype=np.float64).reshape(-1)
        rc = self.lib.or_dense_solve(self.h, level, _dp(x), _dp(zz))
        if rc != 0:
            raise RuntimeError("dense solve failed")
        return x.reshape(tuple(reversed(dims)))

    def vcycle(self, x, z, pre=0, post=4):
        xx = np.ascontiguousarray(x, dtype=np.float64).reshape(-1).copy()
        zz = np.ascontiguousarray(z, dtype=np.float64).reshape(-1)
        r = self.lib.or_vcycle(self.h, _dp(xx), _dp(zz), int(pre), int(post))
        return xx.reshape(self.shape), r

    def rb_sweep(self, x, z, level=0):
        dims = self.level_dims(level)
        xx = np.ascontiguousarray(x, dtype=np.float64).reshape(-1).copy()
        zz = np.ascontiguousarray(z, dtype=np.float64).reshape(-1)
        self.lib.or_rb_sweep(self.h, level, _dp(xx), _dp(zz))
        return xx.reshape(tuple(reversed(dims)))

    def project(self, w, dt, tol=1e-10, maxit=100000, solver=0):
        """solver 0: Jacobi-PCG (reference); 1: multigrid V(0,4) cycles (maxit = cycles)."""
        self.lib.or_project(self.h, float(w), float(dt), float(tol), int(maxit), int(solver))
        return self.lib.or_last_iters(self.h), self.lib.or_last_resid(self.h)

    def step(self, n=1, tol=1e-10, maxit=100000, dt_fixed=0.0, solver=0):
        self.lib.or_step(self.h, int(n), float(tol), int(maxit), float(dt_fixed), int(solver))

    def cfl(self) -> float:
        return self.lib.or_cfl(self.h)

    def forces(self):
        F = np.zeros(3)
        self.lib.or_forces(self.h, _dp(F))
        return F[: self.D]

    def viscous_force(self):
        """Viscous force on the body: sum over band cells of 2 nu S n K_eps(d)."""
        F = np.zeros(3)
        self.lib.or_viscous_force(self.h, _dp(F))
        return F[: self.D]

    def kinetic_energy(self) -> float:
        return self.lib.or_kinetic_energy(self.h)

    def set_exit(self, on=True):
        """Convective exit on the upper x face (the exit face starts at U_x)."""
        if self.lib.or_set_exit(self.h, int(bool(on))) != 0:
            raise ValueError("a convective exit needs a non-periodic x direction")

    def set_exit_plane(self, e):
        a = np.ascontiguousarray(e, dtype=np.float64).reshape(-1)
        self.lib.or_set_exit_plane(self.h, _dp(a))

    def get_exit(self):
        """Normal velocity on the exit face, shape (n_2, n_1) (2-D: (n_1,))."""
        n1 = self.dims[1]
        n2 = self.dims[2] if self.D == 3 else 1
        out = np.zeros(n1 * n2)
        self.lib.or_get_exit(self.h, _dp(out))
        return out.reshape((n2, n1) if self.D == 3 else (n1,))

    # ---- reverse-mode derivative (adjoint) of the step at fixed dt; theta = (R, c_0, ..)
    def _vec(self, a, blocks):
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        assert a.size == blocks * self.ncell
        return a

    def convdiff_adjoint(self, u, rbar):
        """(d convdiff/du at u)^T rbar."""
        out = np.zeros(self.D * self.ncell)
        self.lib.or_convdiff_adjoint(self.h, _dp(self._vec(u, self.D)), _dp(self._vec(rbar, self.D)), _dp(out))
        return out.reshape((self.D,) + self.shape)

    def stage_adjoint(self, stage, dt, u0, u1, outbar):
        """Transpose of bdim_stage: returns (u0bar, u1bar, mu0bar, mu1bar[D*D])."""
        D, n = self.D, self.ncell
        u0b, u1b, m0b, m1b = (np.zeros(D * n), np.zeros(D * n), np.zeros(D * n), np.zeros(D * D * n))
        u1p = _dp(self._vec(u1, D)) if u1 is not None else None
        self.lib.or_stage_adjoint(self.h, int(stage), float(dt), _dp(self._vec(u0, D)), u1p,
                                  _dp(self._vec(outbar, D)), _dp(u0b), _dp(u1b), _dp(m0b), _dp(m1b))
        sh = (D,) + self.shape
        return u0b.reshape(sh), u1b.reshape(sh), m0b.reshape(sh), m1b.reshape((D * D,) + self.shape)

    def project_adjoint(self, v, w, dt, ubar, pbar, tol=1e-12):
        """Transpose of project! of v (weight w) for cotangents of u and p: (vbar, Lbar)."""
        D, n = self.D, self.ncell
        vb, Lb = np.zeros(D * n), np.zeros(D * n)
        self.lib.or_project_adjoint(self.h, _dp(self._vec(v, D)), float(w), float(dt), float(tol),
                                    _dp(self._vec(ubar, D)), _dp(self._vec(pbar, 1)), _dp(vb), _dp(Lb))
        sh = (D,) + self.shape
        return vb.reshape(sh), Lb.reshape(sh)

    def force_adjoint(self, p, Fbar):
        """Force of p and its adjoint: (F, pbar, theta-cotangent of the force weights)."""
        F, pb, tb = np.zeros(3), np.zeros(self.ncell), np.zeros(5)
        fb = np.zeros(3)
        fb[: self.D] = Fbar
        self.lib.or_force_adjoint(self.h, _dp(self._vec(p, 1)), _dp(fb), _dp(F), _dp(pb), _dp(tb))
        return F[: self.D], pb.reshape(self.shape), tb[: self.n_theta]

    def moments_adjoint(self, mu0bar, Lbar, mu1bar):
        tb = np.zeros(5)
        D = self.D
        self.lib.or_moments_adjoint(self.h, _dp(self._vec(mu0bar, D)), _dp(self._vec(Lbar, D)),
                                    _dp(self._vec(mu1bar, D * D)), _dp(tb))
        return tb[: self.n_theta]

    def rollout_grad(self, nsteps, dt, gF, tol=1e-12):
        """nsteps steps at fixed dt from the current state (which advances); returns the
        forces after each step (nsteps x D) and dJ/dtheta for J = sum_n gF[n] . F_n,
        theta = (R, c_0, .., c_{D-1}) of the circle/sphere or (R, r, c_x, c_y, c_z) of the
        torus."""
        D = self.D
        g = np.ascontiguousarray(gF, dtype=np.float64).reshape(-1)
        assert g.size == nsteps * D
        F, tb = np.zeros(nsteps * D), np.zeros(5)
        rc = self.lib.or_rollout_grad(self.h, int(nsteps), float(dt), float(tol), _dp(g), _dp(F), _dp(tb))
        if rc != 0:
            raise ValueError("rollout_grad needs a circle/sphere or torus body, nsteps >= 1 and dt > 0")
        return F.reshape(nsteps, D), tb[: self.n_theta]
