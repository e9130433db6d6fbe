"""ctypes binding of libwl.so (include/wl.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does nothing
but convert arguments; all of the time step runs in the library's CUDA kernels.
PyTorch supplies device memory (the sim workspace, device-side field buffers) and
the CUDA stream.  If libwl.so has not been built the import of the library fails
loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# WL_LIB=debug selects the bounds-checked build (libwl_debug.so) for the whole process
LIB_PATH = os.path.join(HERE, "libwl_debug.so" if os.environ.get("WL_LIB") == "debug" else "libwl.so")
DEBUG_LIB_PATH = os.path.join(HERE, "libwl_debug.so")

WL_OK = 0
WL_EINVAL = -1
WL_ENOMEM = -2
WL_ECUDA = -3
WL_ENONFINITE = -4
WL_ETIMEOUT = -5
WL_WNOTCONV = 1
WL_NODEBUG = 2

WL_FIELD_U = 0
WL_FIELD_P = 1
WL_FIELD_DIV = 2
WL_FIELD_MU0 = 3
WL_FIELD_Z = 4
WL_FIELD_UPRED = 5
WL_FIELD_USTAGE = 6
WL_FIELD_EXIT = 7

WL_BODY_NONE = 0
WL_BODY_SPHERE = 1
WL_BODY_TORUS = 2
WL_PATH_RESID_STAGED, WL_PATH_CLUSTER_TAIL, WL_PATH_BLOCK_TAIL, WL_PATH_TALL_TILES = 1, 2, 4, 8
WL_BODY_FIELD = 3

WL_COARSE_FP32 = 0
WL_COARSE_BF16 = 1
WL_COARSE_FP16 = 2
# storage of the multigrid levels between the fine and the coarsest one, by name
COARSE_PRECISION = {"fp32": WL_COARSE_FP32, "bf16": WL_COARSE_BF16, "fp16": WL_COARSE_FP16}

# every symbol include/wl.h declares
EXPORTS = (
    "wl_default_opts", "wl_workspace_bytes", "wl_create", "wl_set_ic", "wl_step", "wl_stage",
    "wl_project", "wl_gmg_vcycle", "wl_forces", "wl_viscous_force", "wl_get_field", "wl_set_field", "wl_get_dt",
    "wl_set_dt", "wl_get_time", "wl_status", "wl_profile_step", "wl_graph_kernels", "wl_levels", "wl_level_dims",
    "wl_destroy", "wl_last_error", "wl_forces_noalloc", "wl_wait_probe", "wl_step_batch",
    "wl_grad_workspace_bytes", "wl_grad_forward", "wl_grad_backward", "wl_level_split", "wl_kernel_paths",
    "wl_state_bytes", "wl_save", "wl_load", "wl_get_metrics",
    "wl_batch_create", "wl_batch_step", "wl_batch_destroy", "wl_batch_last_error", "wl_event_elapsed",
    "wl_debug_bounds",
)
METRIC_RING, METRIC_FIELDS = 1024, 13
METRICS = ("step", "time", "dt", "vcycles1", "vcycles2", "resid1", "resid2", "cfl", "ke", "maxdiv", "F0", "F1", "F2")
KCLASSES = ("stage", "band", "resid_fine", "restrict", "sweep_fine", "sweep_coarse", "coarsest", "correct",
            "control", "sweep_fine_uni", "sweep_fine_bandt", "resid_fine_uni", "resid_fine_bandt")


class WlBody(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("center", ctypes.c_double * 3),
                ("radius", ctypes.c_double), ("radius2", ctypes.c_double),
                ("sdf_nodes", ctypes.POINTER(ctypes.c_float))]


class WlOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_vcycles", ctypes.c_int), ("post", ctypes.c_int),
                ("eps", ctypes.c_double), ("dt_cap", ctypes.c_double), ("dt_fixed", ctypes.c_double),
                ("periodic_mask", ctypes.c_uint), ("advect", ctypes.c_int), ("precision", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("stream", ctypes.c_void_p), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("exit_bc", ctypes.c_int), ("coarse_precision", ctypes.c_int),
                ("metrics", ctypes.c_int)]


class WLError(RuntimeError):
    def __init__(self, rc, msg):
        super().__init__(f"libwl error {rc}: {msg}")
        self.rc = rc


_lib = None


def load(path: str = LIB_PATH):
    """Load libwl.so (raises if it is missing) and declare every signature."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built: run __graft_entry__.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    I, D, P = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    IP, DP = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    sig = {
        "wl_default_opts": (None, [ctypes.POINTER(WlOpts)]),
        "wl_workspace_bytes": (ctypes.c_size_t, [IP, I, ctypes.POINTER(WlOpts)]),
        "wl_create": (I, [IP, I, D, DP, ctypes.POINTER(WlBody), ctypes.POINTER(WlOpts), ctypes.POINTER(H)]),
        "wl_set_ic": (I, [H, I, D, P, I]),
        "wl_step": (I, [H, I]),
        "wl_stage": (I, [H, I]),
        "wl_project": (I, [H, D, IP, DP]),
        "wl_gmg_vcycle": (I, [H, DP]),
        "wl_forces": (I, [H, DP]),
        "wl_viscous_force": (I, [H, DP]),
        "wl_get_field": (I, [H, I, P, I]),
        "wl_set_field": (I, [H, I, P, I]),
        "wl_get_dt": (I, [H, DP]),
        "wl_set_dt": (I, [H, D]),
        "wl_get_time": (I, [H, DP, ctypes.POINTER(ctypes.c_longlong)]),
        "wl_status": (I, [H, IP, ctypes.POINTER(ctypes.c_longlong), DP]),
        "wl_profile_step": (I, [H, I, DP, ctypes.POINTER(ctypes.c_longlong)]),
        "wl_graph_kernels": (I, [H, IP, IP]),
        "wl_levels": (I, [H, IP]),
        "wl_level_dims": (I, [H, I, IP]),
        "wl_destroy": (None, [H]),
        "wl_last_error": (ctypes.c_char_p, [H]),
        "wl_forces_noalloc": (I, [IP, I, ctypes.c_uint, ctypes.POINTER(WlBody), D, P, P, P, P]),
        "wl_wait_probe": (I, [D, DP]),
        "wl_step_batch": (I, [ctypes.POINTER(H), I, I, P]),
        "wl_grad_workspace_bytes": (ctypes.c_size_t, [H, I, I]),
        "wl_grad_forward": (I, [H, I, I, P, ctypes.c_size_t, DP]),
        "wl_grad_backward": (I, [H, DP, DP]),
        "wl_level_split": (I, [H, I, IP, DP]),
        "wl_kernel_paths": (I, [H, ctypes.POINTER(ctypes.c_uint)]),
        "wl_state_bytes": (ctypes.c_size_t, [H]),
        "wl_get_metrics": (I, [H, DP, I, IP]),
        "wl_batch_create": (I, [ctypes.c_longlong, ctypes.POINTER(ctypes.c_void_p)]),
        "wl_batch_step": (I, [ctypes.c_void_p, ctypes.POINTER(H), I, P, P]),
        "wl_batch_destroy": (None, [ctypes.c_void_p]),
        "wl_batch_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
        "wl_event_elapsed": (I, [P, P, ctypes.POINTER(ctypes.c_float)]),
        "wl_debug_bounds": (I, [H, ctypes.POINTER(ctypes.c_uint)]),
        "wl_save": (I, [H, P, ctypes.c_size_t, I]),
        "wl_load": (I, [H, P, ctypes.c_size_t, I]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


# ----------------------------------------------------------------- C entry points
def wl_default_opts() -> WlOpts:
    o = WlOpts()
    load().wl_default_opts(ctypes.byref(o))
    return o


def wl_workspace_bytes(dims, opts: WlOpts | None = None) -> int:
    d = (ctypes.c_int * 3)(*(list(dims) + [1] * (3 - len(dims))))
    return load().wl_workspace_bytes(d, len(dims), ctypes.byref(opts) if opts is not None else None)


def wl_create(dims, nu, U, body: WlBody | None, opts: WlOpts | None):
    d = (ctypes.c_int * 3)(*(list(dims) + [1] * (3 - len(dims))))
    u = (ctypes.c_double * 3)(*(list(U) + [0.0] * (3 - len(U))))
    h = ctypes.c_void_p()
    rc = load().wl_create(d, len(dims), float(nu), u, ctypes.byref(body) if body is not None else None,
                          ctypes.byref(opts) if opts is not None else None, ctypes.byref(h))
    return rc, h


def wl_set_ic(h, kind, amp=1.0, src_ptr=None, src_is_device=0):
    return load().wl_set_ic(h, int(kind), float(amp), src_ptr, int(src_is_device))


def wl_step(h, nsteps=1):
    return load().wl_step(h, int(nsteps))


def wl_stage(h, stage):
    return load().wl_stage(h, int(stage))


def wl_project(h, w):
    it = ctypes.c_int(0)
    r = ctypes.c_double(0.0)
    rc = load().wl_project(h, float(w), ctypes.byref(it), ctypes.byref(r))
    return rc, it.value, r.value


def wl_gmg_vcycle(h):
    r = ctypes.c_double(0.0)
    rc = load().wl_gmg_vcycle(h, ctypes.byref(r))
    return rc, r.value


def wl_forces(h, D):
    F = (ctypes.c_double * 3)()
    rc = load().wl_forces(h, F)
    return rc, [F[i] for i in range(D)]


def wl_viscous_force(h, D):
    F = (ctypes.c_double * 3)()
    rc = load().wl_viscous_force(h, F)
    return rc, [F[i] for i in range(D)]


def wl_get_field(h, which, dst_ptr, dst_is_device):
    return load().wl_get_field(h, int(which), dst_ptr, int(dst_is_device))


def wl_set_field(h, which, src_ptr, src_is_device):
    return load().wl_set_field(h, int(which), src_ptr, int(src_is_device))


def wl_get_dt(h):
    v = ctypes.c_double(0.0)
    rc = load().wl_get_dt(h, ctypes.byref(v))
    return rc, v.value


def wl_set_dt(h, dt):
    return load().wl_set_dt(h, float(dt))


def wl_get_time(h):
    t = ctypes.c_double(0.0)
    n = ctypes.c_longlong(0)
    rc = load().wl_get_time(h, ctypes.byref(t), ctypes.byref(n))
    return rc, t.value, n.value


def wl_status(h):
    it = (ctypes.c_int * 2)()
    tot = ctypes.c_longlong(0)
    worst = ctypes.c_double(0.0)
    rc = load().wl_status(h, it, ctypes.byref(tot), ctypes.byref(worst))
    return rc, (it[0], it[1]), tot.value, worst.value


def wl_profile_step(h, nsteps):
    ms = (ctypes.c_double * len(KCLASSES))()
    n = (ctypes.c_longlong * len(KCLASSES))()
    rc = load().wl_profile_step(h, int(nsteps), ms, n)
    return rc, {k: (ms[i], n[i]) for i, k in enumerate(KCLASSES)}


def wl_graph_kernels(h):
    a, b = ctypes.c_int(0), ctypes.c_int(0)
    rc = load().wl_graph_kernels(h, ctypes.byref(a), ctypes.byref(b))
    return rc, a.value, b.value


def wl_levels(h):
    n = ctypes.c_int(0)
    rc = load().wl_levels(h, ctypes.byref(n))
    return rc, n.value


def wl_level_dims(h, l):
    d = (ctypes.c_int * 3)()
    rc = load().wl_level_dims(h, int(l), d)
    return rc, (d[0], d[1], d[2])


def wl_destroy(h):
    load().wl_destroy(h)


def wl_forces_noalloc(dims, periodic, body: WlBody, eps, p_ptr, L_ptr, F_ptr, stream=None):
    """Allocation-free pressure force on caller-owned device fields (see include/wl.h)."""
    d = (ctypes.c_int * 3)(*(list(dims) + [1] * (3 - len(dims))))
    return load().wl_forces_noalloc(d, len(dims), int(periodic), ctypes.byref(body), float(eps), p_ptr, L_ptr,
                                    F_ptr, stream)


def wl_step_batch(handles, nsteps, stream=None):
    """Advance the sims `handles` (wl_handle values) by nsteps each, together (see include/wl.h)."""
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    return load().wl_step_batch(arr, len(handles), int(nsteps), stream)


def wl_debug_bounds(h):
    """(rc, flags) of the bounds-checked build's index checks and canaries (see wl.h)."""
    f = ctypes.c_uint(0)
    rc = load().wl_debug_bounds(h, ctypes.byref(f))
    return rc, f.value


def wl_event_elapsed(start, end):
    """ms between two recorded CUDA events (raw cudaEvent_t handles)."""
    ms = ctypes.c_float(0.0)
    rc = load().wl_event_elapsed(start, end, ctypes.byref(ms))
    if rc != WL_OK:
        raise WLError(rc, "wl_event_elapsed")
    return ms.value


class Batch:
    """Batched steps of many small simulations (wl_batch_*): sims of at most max_cells
    cells (and the options the batched kernels cover) step in one graph per dimension,
    the others with their own graphs."""

    def __init__(self, max_cells):
        h = ctypes.c_void_p()
        rc = load().wl_batch_create(int(max_cells), ctypes.byref(h))
        if rc != WL_OK:
            raise WLError(rc, "wl_batch_create")
        self.h = h

    def step(self, handles, stream=None, small_done=None):
        arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
        rc = load().wl_batch_step(self.h, arr, len(handles), stream, small_done)
        if rc < 0:
            msg = load().wl_batch_last_error(self.h)
            raise WLError(rc, "wl_batch_step: " + (msg.decode() if msg else ""))
        return rc

    def close(self):
        if self.h is not None and self.h.value:
            load().wl_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wl_wait_probe(seconds):
    """Bounded-wait self-test (see include/wl.h): (rc, elapsed ms); rc is WL_ETIMEOUT."""
    ms = ctypes.c_double(0.0)
    rc = load().wl_wait_probe(float(seconds), ctypes.byref(ms))
    return rc, ms.value


def make_body(body) -> WlBody:
    """A wl_body from a dict: kind (WL_BODY_*), center, radius, radius2, or for
    WL_BODY_FIELD the node-sampled distance `nodes` (shape reversed(dims + 1)).  The
    returned struct keeps the node array alive (attribute `_nodes`) until wl_create."""
    b = WlBody()
    b.kind = int(body.get("kind", WL_BODY_SPHERE))
    c = list(body.get("center", (0.0, 0.0, 0.0))) + [0.0] * 3
    for i in range(3):
        b.center[i] = float(c[i])
    b.radius = float(body.get("radius", 0.0))
    b.radius2 = float(body.get("radius2", 0.0))
    if b.kind == WL_BODY_FIELD:
        nodes = np.ascontiguousarray(body["nodes"], dtype=np.float32).reshape(-1)
        b._nodes = nodes
        b.sdf_nodes = nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    return b


def wl_state_bytes(h) -> int:
    return int(load().wl_state_bytes(h))


def wl_save(h, dst_ptr, nbytes, dst_is_device):
    return load().wl_save(h, dst_ptr, int(nbytes), int(dst_is_device))


def wl_load(h, src_ptr, nbytes, src_is_device):
    return load().wl_load(h, src_ptr, int(nbytes), int(src_is_device))


def wl_get_metrics(h, max_records=METRIC_RING):
    out = np.zeros((max(int(max_records), 0), METRIC_FIELDS))
    n = ctypes.c_int(0)
    rc = load().wl_get_metrics(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(max_records),
                               ctypes.byref(n))
    return rc, out[: n.value]


def wl_last_error(h) -> str:
    s = load().wl_last_error(h)
    return s.decode() if s else ""


# ----------------------------------------------------------------- convenience wrapper
class Sim:
    """One simulation: workspace from torch's caching allocator, work on torch's
    current CUDA stream, fields exchanged as torch tensors or numpy arrays.
    Every method is a direct call of the C entry point of the same name."""

    def __init__(self, dims, nu, U, body=None, periodic=0, tol=1e-6, max_vcycles=32, post=4, eps=1.0,
                 dt_cap=10.0, dt_fixed=0.0, advect=True, precision=1, use_graph=True, device=None,
                 coarse_precision=0, exit_bc=False, metrics=False):
        import torch

        self.torch = torch
        self.dims = tuple(int(d) for d in dims)
        self.D = len(self.dims)
        self.ncell = int(np.prod(self.dims))
        self.shape = tuple(reversed(self.dims))
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        o = wl_default_opts()
        o.tol, o.max_vcycles, o.post, o.eps = float(tol), int(max_vcycles), int(post), float(eps)
        o.dt_cap, o.dt_fixed, o.periodic_mask = float(dt_cap), float(dt_fixed), int(periodic)
        o.advect, o.precision, o.use_graph = int(bool(advect)), int(precision), int(bool(use_graph))
        o.coarse_precision = COARSE_PRECISION.get(coarse_precision, coarse_precision)
        o.exit_bc = int(bool(exit_bc))
        o.metrics = int(bool(metrics))
        with torch.cuda.device(self.device):
            o.stream = torch.cuda.current_stream().cuda_stream
            nbytes = wl_workspace_bytes(self.dims, o)
            if nbytes == 0:
                raise WLError(WL_EINVAL, "bad dimensions")
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            o.workspace = self.workspace.data_ptr()
            o.workspace_bytes = nbytes
            b = None
            # body parameters of the gradient: circle/sphere (R, c_0, ..), torus (R, r, c_x, c_y, c_z)
            self.n_theta = 5 if body is not None and int(body.get("kind", 1)) == WL_BODY_TORUS else self.D + 1
            if body is not None:
                b = make_body(body)
                if b.kind == WL_BODY_FIELD and b._nodes.size != int(np.prod([d + 1 for d in self.dims])):
                    raise WLError(WL_EINVAL, "sdf nodes: (n0+1)(n1+1)[(n2+1)] values expected")
            rc, h = wl_create(self.dims, nu, U, b, o)
        if rc != WL_OK:
            raise WLError(rc, "wl_create failed")
        self.h = h
        self.opts = o

    def _check(self, rc, what):
        if rc < 0:
            raise WLError(rc, f"{what}: {wl_last_error(self.h)}")
        return rc

    def close(self):
        if getattr(self, "h", None):
            wl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # fields
    def _nblocks(self, which):
        return self.D if which in (WL_FIELD_U, WL_FIELD_MU0, WL_FIELD_UPRED, WL_FIELD_USTAGE) else 1

    def _field_shape(self, which):
        if which == WL_FIELD_EXIT:  # the exit plane: n_1 [x n_2] values, y fastest
            return tuple(reversed(self.dims[1:]))
        nb = self._nblocks(which)
        return ((nb,) if nb > 1 else ()) + self.shape

    def get(self, which, device=False):
        """Field as a float32 tensor on the GPU (device=True) or a numpy array."""
        shape = self._field_shape(which)
        if device:
            t = self.torch.empty(shape, dtype=self.torch.float32, device=self.device)
            self._check(wl_get_field(self.h, which, t.data_ptr(), 1), "wl_get_field")
            return t
        a = np.empty(shape, dtype=np.float32)
        self._check(wl_get_field(self.h, which, a.ctypes.data, 0), "wl_get_field")
        return a

    def set(self, which, value):
        n = int(np.prod(self._field_shape(which)))
        if isinstance(value, np.ndarray):
            a = np.ascontiguousarray(value, dtype=np.float32)
            assert a.size == n
            self._check(wl_set_field(self.h, which, a.ctypes.data, 0), "wl_set_field")
        else:
            t = value.to(device=self.device, dtype=self.torch.float32).contiguous()
            assert t.numel() == n
            self._check(wl_set_field(self.h, which, t.data_ptr(), 1), "wl_set_field")

    # routines
    def set_ic(self, kind=0, amp=1.0, u=None):
        if kind == 2:
            a = np.ascontiguousarray(u, dtype=np.float32)
            return self._check(wl_set_ic(self.h, 2, amp, a.ctypes.data, 0), "wl_set_ic")
        return self._check(wl_set_ic(self.h, kind, amp), "wl_set_ic")

    def step(self, n=1):
        return self._check(wl_step(self.h, n), "wl_step")

    def metrics(self, max_records=METRIC_RING):
        """The last per-step metric records (wl_get_metrics), oldest first, as a dict of
        numpy arrays keyed by METRICS."""
        rc, rec = wl_get_metrics(self.h, max_records)
        self._check(rc, "wl_get_metrics")
        return {k: rec[:, i] for i, k in enumerate(METRICS)}

    def save(self, device=False):
        """The sim's state (wl_save) as a uint8 numpy array, or a uint8 tensor on its
        device when device=True."""
        n = wl_state_bytes(self.h)
        if device:
            buf = self.torch.empty(n, dtype=self.torch.uint8, device=self.device)
            self._check(wl_save(self.h, buf.data_ptr(), n, 1), "wl_save")
        else:
            buf = np.empty(n, dtype=np.uint8)
            self._check(wl_save(self.h, buf.ctypes.data, n, 0), "wl_save")
        return buf

    def load(self, buf):
        """Restore a state saved by save() (host array or device tensor)."""
        if isinstance(buf, np.ndarray):
            a = np.ascontiguousarray(buf, dtype=np.uint8)
            return self._check(wl_load(self.h, a.ctypes.data, a.nbytes, 0), "wl_load")
        return self._check(wl_load(self.h, buf.data_ptr(), buf.numel() * buf.element_size(), 1), "wl_load")

    def stage(self, stage):
        return self._check(wl_stage(self.h, stage), "wl_stage")

    def project(self, w):
        rc, it, r = wl_project(self.h, w)
        self._check(rc, "wl_project")
        return rc, it, r

    def gmg_vcycle(self):
        rc, r = wl_gmg_vcycle(self.h)
        self._check(rc, "wl_gmg_vcycle")
        return r

    def forces(self):
        rc, F = wl_forces(self.h, self.D)
        self._check(rc, "wl_forces")
        return np.array(F)

    def viscous_force(self):
        """wl_viscous_force: the viscous force on the body of the current velocity."""
        rc, F = wl_viscous_force(self.h, self.D)
        self._check(rc, "wl_viscous_force")
        return np.array(F)

    @property
    def dt(self):
        rc, v = wl_get_dt(self.h)
        self._check(rc, "wl_get_dt")
        return v

    @dt.setter
    def dt(self, v):
        self._check(wl_set_dt(self.h, v), "wl_set_dt")

    def time(self):
        rc, t, n = wl_get_time(self.h)
        self._check(rc, "wl_get_time")
        return t, n

    def status(self):
        rc, last, tot, worst = wl_status(self.h)
        self._check(rc, "wl_status")
        return rc, last, tot, worst

    def graph_kernels(self):
        """wl_graph_kernels: (kernels per step outside the V-cycles, kernels per V-cycle)."""
        rc, a, b = wl_graph_kernels(self.h)
        self._check(rc, "wl_graph_kernels")
        return a, b

    def profile_step(self, nsteps=1):
        """{kernel class: (total ms, launches)} over nsteps host-driven steps."""
        rc, d = wl_profile_step(self.h, nsteps)
        self._check(rc, "wl_profile_step")
        return d

    def grad_forward(self, nsteps, every):
        """wl_grad_forward: nsteps steps recording the force after each (returned as an
        (nsteps, D) float64 array) and the checkpoints for grad_backward; the gradient
        workspace is a torch tensor kept by this object."""
        nb = load().wl_grad_workspace_bytes(self.h, int(nsteps), int(every))
        if nb == 0:
            raise WLError(WL_EINVAL, "bad gradient rollout arguments")
        self.grad_workspace = self.torch.empty(nb + 256, dtype=self.torch.uint8, device=self.device)
        base = self.grad_workspace.data_ptr()
        ptr = (base + 255) // 256 * 256
        F = np.zeros(int(nsteps) * self.D)
        rc = load().wl_grad_forward(self.h, int(nsteps), int(every), ctypes.c_void_p(ptr), nb,
                                    F.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        self._check(rc, "wl_grad_forward")
        self.grad_steps = int(nsteps)
        return F.reshape(int(nsteps), self.D)

    def grad_backward(self, gF, return_status=False):
        """wl_grad_backward: dJ/dtheta for J = sum_n gF[n] . F_n, theta = (R, c_0, ..) of a
        circle/sphere or (R, r, c_x, c_y, c_z) of a torus (and the status, WL_OK or
        WL_WNOTCONV, with return_status)."""
        g = np.ascontiguousarray(gF, dtype=np.float64).reshape(-1)
        n = getattr(self, "grad_steps", 0)
        if n and g.size != n * self.D:
            raise WLError(WL_EINVAL, f"gF must hold {n} x {self.D} values")
        tb = np.zeros(self.n_theta)
        rc = load().wl_grad_backward(self.h, g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     tb.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        self._check(rc, "wl_grad_backward")
        return (tb, rc) if return_status else tb

    def kernel_paths(self):
        """Bits of the kernel paths the step takes (wl_kernel_paths: WL_PATH_*)."""
        v = ctypes.c_uint(0)
        self._check(load().wl_kernel_paths(self.h, ctypes.byref(v)), "wl_kernel_paths")
        return v.value

    def level_split(self, l=0):
        """(split, band_fraction) of level l's staged kernels (wl_level_split)."""
        sp, fr = ctypes.c_int(0), ctypes.c_double(0.0)
        self._check(load().wl_level_split(self.h, int(l), ctypes.byref(sp), ctypes.byref(fr)), "wl_level_split")
        return bool(sp.value), fr.value

    def levels(self):
        rc, n = wl_levels(self.h)
        self._check(rc, "wl_levels")
        return [wl_level_dims(self.h, l)[1][: self.D] for l in range(n)]
