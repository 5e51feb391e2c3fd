"""Thin Python binding of the C ABI in ``include/vlb.h`` (ctypes).

The functions carry the C names and only marshal arguments: every step of the
method runs in the CUDA kernels of ``libvlb.so``.  There is no CPU fallback;
importing this module fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("VLB_LIBRARY") or os.path.join(_HERE, "libvlb.so")  # another build (the autotuner's)

VLB_ABI_VERSION = 1
VLB_OK, VLB_EINVAL, VLB_ENOMEM, VLB_ECUDA, VLB_ESTATE, VLB_EUNSTABLE, VLB_EOVERFLOW, VLB_ETIMEOUT = (
    0, -1, -2, -3, -4, -5, -6, -7)
VLB_FP64, VLB_FP32, VLB_FP16_STORE, VLB_BF16_STORE = 0, 1, 2, 3
VLB_WALL_ADIABATIC, VLB_WALL_DIRICHLET = 0, 1
VLB_FIELD_RHO, VLB_FIELD_UX, VLB_FIELD_UY, VLB_FIELD_T, VLB_FIELD_FS = 1, 2, 4, 8, 16
VLB_FIELD_ALL = 31

STATUS_NAMES = {0: "VLB_OK", -1: "VLB_EINVAL", -2: "VLB_ENOMEM", -3: "VLB_ECUDA", -4: "VLB_ESTATE",
                -5: "VLB_EUNSTABLE", -6: "VLB_EOVERFLOW", -7: "VLB_ETIMEOUT"}


class vlb_params(ctypes.Structure):
    """Mirror of ``vlb_params`` in include/vlb.h (same order and types)."""
    _fields_ = [
        ("abi_version", ctypes.c_uint32),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("periodic", ctypes.c_int32 * 2),
        ("thermal_wall", ctypes.c_int32 * 4),
        ("thermal_rates_mode", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("max_particles", ctypes.c_int32),
        ("outflow_mask", ctypes.c_int32), ("reserved1", ctypes.c_int32),
        ("tau_f", ctypes.c_double),
        ("lambda_q_flow", ctypes.c_double),
        ("s_e", ctypes.c_double),
        ("prandtl", ctypes.c_double),
        ("rho_ratio", ctypes.c_double),
        ("cv_ratio", ctypes.c_double),
        ("k_ratio_default", ctypes.c_double),
        ("gravity", ctypes.c_double * 2),
        ("beta", ctypes.c_double),
        ("T_ref", ctypes.c_double),
        ("T_fluid_init", ctypes.c_double),
        ("wall_T", ctypes.c_double * 4),
        ("contact_range", ctypes.c_double),
        ("contact_eps_p", ctypes.c_double),
        ("contact_eps_w", ctypes.c_double),
    ]


class VlbError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class vlb_serve_params(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_uint64), ("steps_per_round", ctypes.c_int32), ("max_active", ctypes.c_int32)]


VLB_CASE_QUEUED, VLB_CASE_ACTIVE, VLB_CASE_DONE, VLB_CASE_FAILED = 0, 1, 2, 3


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_2410_23802_gb300.build.build() "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    d = P(ctypes.c_double)
    h = ctypes.c_void_p
    sig = {
        "vlb_params_size": (ctypes.c_size_t, []),
        "vlb_params_default": (ctypes.c_int, [P(vlb_params)]),
        "vlb_create": (ctypes.c_int, [P(vlb_params), P(ctypes.c_void_p)]),
        "vlb_set_stream": (ctypes.c_int, [h, ctypes.c_void_p]),
        "vlb_set_fixed_temperature": (ctypes.c_int, [h, ctypes.c_int32, ctypes.c_int32, P(ctypes.c_int32)]),
        "vlb_add_particles": (ctypes.c_int, [h, ctypes.c_int32, d, d, d, d, d, d]),
        "vlb_add_ellipses": (ctypes.c_int, [h, ctypes.c_int32, d, d, d, d, d, d, d, d]),
        "vlb_step": (ctypes.c_int, [h, ctypes.c_int32]),
        "vlb_insert_particles": (ctypes.c_int, [h, ctypes.c_int32, d, d, d, d, d, d]),
        "vlb_step_batch": (ctypes.c_int, [P(ctypes.c_void_p), ctypes.c_int32, ctypes.c_int32, P(ctypes.c_int32)]),
        "vlb_debug_batch_wait": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32]),
        "vlb_set_batch_form": (ctypes.c_int, [ctypes.c_int32]),
        "vlb_get_batch_form": (ctypes.c_int32, []),
        "vlb_synchronize": (ctypes.c_int, [h]),
        "vlb_get_step": (ctypes.c_int, [h, P(ctypes.c_int64)]),
        "vlb_get_fields": (ctypes.c_int, [h, ctypes.c_uint32, d, d, d, d, d]),
        "vlb_get_particle_state": (ctypes.c_int, [h, ctypes.c_int32, d, d, d, d, d, d]),
        "vlb_get_particle_count": (ctypes.c_int, [h, P(ctypes.c_int32)]),
        "vlb_particle_state_async": (ctypes.c_int, [h, ctypes.c_int32]),
        "vlb_particle_state_wait": (ctypes.c_int, [h, ctypes.c_int32, d, d, d, d, d, d, P(ctypes.c_int64)]),
        "vlb_get_audit": (ctypes.c_int, [h, d, d, d]),
        "vlb_get_solid_fraction": (ctypes.c_int, [h, P(ctypes.c_uint8), P(ctypes.c_int32),
                                                  P(ctypes.c_uint8), d]),
        "vlb_get_solid_fraction_noalloc": (ctypes.c_int, [h, P(ctypes.c_uint8), P(ctypes.c_int32),
                                                          P(ctypes.c_uint8), d]),
        "vlb_get_contact_pairs": (ctypes.c_int, [h, ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_int32)]),
        "vlb_state_size": (ctypes.c_int, [h, P(ctypes.c_uint64)]),
        "vlb_save_state": (ctypes.c_int, [h, ctypes.c_void_p, ctypes.c_uint64]),
        "vlb_load_state": (ctypes.c_int, [h, ctypes.c_void_p, ctypes.c_uint64]),
        "vlb_profile_begin": (ctypes.c_int, [h, ctypes.c_int32]),
        "vlb_profile_end": (ctypes.c_int, [h, d, P(ctypes.c_int32), P(ctypes.c_int32)]),
        "vlb_last_error": (ctypes.c_char_p, [h]),
        "vlb_destroy": (None, [h]),
        "vlb_device_bytes": (ctypes.c_int, [P(vlb_params), ctypes.c_int32, d, P(ctypes.c_uint64)]),
        "vlb_serve_params_default": (ctypes.c_int, [P(vlb_serve_params)]),
        "vlb_serve_create": (ctypes.c_int, [P(vlb_serve_params), P(ctypes.c_void_p)]),
        "vlb_serve_submit": (ctypes.c_int, [h, P(vlb_params), ctypes.c_int32, d, d, d, d, ctypes.c_int64,
                                            P(ctypes.c_int64)]),
        "vlb_serve_poll": (ctypes.c_int, [h, P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32)]),
        "vlb_serve_case_info": (ctypes.c_int, [h, ctypes.c_int64, P(ctypes.c_int32), P(ctypes.c_int32),
                                               P(ctypes.c_int32), P(ctypes.c_int32), d]),
        "vlb_serve_take": (ctypes.c_int, [h, ctypes.c_int64, d, d, d, d, d, d]),
        "vlb_serve_last_error": (ctypes.c_char_p, [h]),
        "vlb_serve_destroy": (None, [h]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if lib.vlb_params_size() != ctypes.sizeof(vlb_params):
        raise ImportError("vlb_params layout differs between include/vlb.h and the binding")
    return lib


_lib = _load()


def _ptr(a, ctype=ctypes.c_double):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctype))


def _check(status: int, h=None):
    if status != VLB_OK:
        msg = _lib.vlb_last_error(h)
        raise VlbError(status, msg.decode() if msg else "")


def vlb_params_default(**overrides) -> vlb_params:
    """The library's defaults with overrides by field name; ``outflow`` (four
    flags, sides x-, x+, y-, y+) sets ``outflow_mask``."""
    p = vlb_params()
    _check(_lib.vlb_params_default(ctypes.byref(p)))
    for k, v in overrides.items():
        if k == "outflow":
            p.outflow_mask = sum(1 << i for i, flag in enumerate(v) if flag)
        elif not hasattr(p, k):
            raise AttributeError(f"vlb_params has no field {k}")
        elif k in ("periodic", "thermal_wall", "wall_T", "gravity"):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(p, k, v)
    return p


def vlb_create(params: vlb_params):
    h = ctypes.c_void_p()
    _check(_lib.vlb_create(ctypes.byref(params), ctypes.byref(h)))
    return h


def vlb_set_stream(h, stream_ptr: int):
    _check(_lib.vlb_set_stream(h, ctypes.c_void_p(stream_ptr)), h)


def vlb_add_particles(h, xy, radius, T0, k_ratio=None, uv=None, omega=None):
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1)
    radius = np.ascontiguousarray(radius, dtype=np.float64)
    T0 = np.ascontiguousarray(T0, dtype=np.float64)
    n = radius.shape[0]
    conv = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1)  # noqa: E731
    k_ratio, uv, omega = conv(k_ratio), conv(uv), conv(omega)
    _check(_lib.vlb_add_particles(h, n, _ptr(xy), _ptr(radius), _ptr(T0), _ptr(k_ratio), _ptr(uv), _ptr(omega)), h)


def vlb_add_ellipses(h, xy, semi_a, semi_b, theta, T0, k_ratio=None, uv=None, omega=None):
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1)
    semi_a = np.ascontiguousarray(semi_a, dtype=np.float64)
    semi_b = np.ascontiguousarray(semi_b, dtype=np.float64)
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    T0 = np.ascontiguousarray(T0, dtype=np.float64)
    n = semi_a.shape[0]
    conv = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1)  # noqa: E731
    k_ratio, uv, omega = conv(k_ratio), conv(uv), conv(omega)
    _check(_lib.vlb_add_ellipses(h, n, _ptr(xy), _ptr(semi_a), _ptr(semi_b), _ptr(theta), _ptr(T0), _ptr(k_ratio),
                                 _ptr(uv), _ptr(omega)), h)


def vlb_insert_particles(h, xy, radius, T0, k_ratio=None, uv=None, omega=None):
    """Add disks between two steps (mid-run insertion)."""
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1)
    radius = np.ascontiguousarray(radius, dtype=np.float64)
    T0 = np.ascontiguousarray(T0, dtype=np.float64)
    conv = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(-1)  # noqa: E731
    k_ratio, uv, omega = conv(k_ratio), conv(uv), conv(omega)
    _check(_lib.vlb_insert_particles(h, radius.shape[0], _ptr(xy), _ptr(radius), _ptr(T0), _ptr(k_ratio), _ptr(uv),
                                     _ptr(omega)), h)


def vlb_step(h, nsteps: int = 1):
    _check(_lib.vlb_step(h, int(nsteps)), h)


def vlb_step_batch(handles, nsteps: int = 1):
    """nsteps steps of every handle in `handles`, interleaved on their streams."""
    hs = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    failed = ctypes.c_int32(-1)
    st = _lib.vlb_step_batch(hs, len(handles), int(nsteps), ctypes.byref(failed))
    _check(st, handles[failed.value] if failed.value >= 0 else None)


VLB_BATCH_TILES, VLB_BATCH_PERSISTENT = 0, 1


def vlb_set_batch_form(form: int) -> None:
    """Form of later vlb_step_batch calls (process-wide): VLB_BATCH_TILES or VLB_BATCH_PERSISTENT."""
    _check(_lib.vlb_set_batch_form(int(form)), None)


def vlb_get_batch_form() -> int:
    return int(_lib.vlb_get_batch_form())


def vlb_debug_batch_wait(wait_ns: int = 0, stuck_handle: int = -1) -> None:
    """Test hook: the limit of vlb_step_batch's device-side waits (0: one second) and a handle position whose
    waits never end (-1: none)."""
    _check(_lib.vlb_debug_batch_wait(int(wait_ns), int(stuck_handle)), None)


def vlb_synchronize(h):
    _check(_lib.vlb_synchronize(h), h)


def vlb_get_step(h) -> int:
    n = ctypes.c_int64()
    _check(_lib.vlb_get_step(h, ctypes.byref(n)), h)
    return n.value


def vlb_get_fields(h, nx: int, ny: int, mask: int = VLB_FIELD_ALL, out: dict | None = None) -> dict:
    names = ["rho", "ux", "uy", "T", "fs"]
    res = {} if out is None else out
    arrs = []
    for k, nm in enumerate(names):
        if mask & (1 << k):
            a = res.get(nm)
            if a is None or a.shape != (ny, nx):
                a = np.empty((ny, nx), dtype=np.float64)
            res[nm] = a
            arrs.append(a)
        else:
            arrs.append(None)
    _check(_lib.vlb_get_fields(h, mask, *[_ptr(a) for a in arrs]), h)
    return res


def vlb_get_particle_count(h) -> int:
    n = ctypes.c_int32()
    _check(_lib.vlb_get_particle_count(h, ctypes.byref(n)), h)
    return n.value


def vlb_get_particle_state(h, n: int | None = None) -> dict:
    n = vlb_get_particle_count(h) if n is None else n
    xy, uv, force = np.empty((n, 2)), np.empty((n, 2)), np.empty((n, 2))
    theta, omega, torque = np.empty(n), np.empty(n), np.empty(n)
    _check(_lib.vlb_get_particle_state(h, n, _ptr(xy), _ptr(theta), _ptr(uv), _ptr(omega), _ptr(force),
                                       _ptr(torque)), h)
    return {"x": xy[:, 0].copy(), "y": xy[:, 1].copy(), "theta": theta, "ux": uv[:, 0].copy(),
            "uy": uv[:, 1].copy(), "omega": omega, "fx": force[:, 0].copy(), "fy": force[:, 1].copy(),
            "torque": torque}


def vlb_particle_state_async(h, n: int):
    """Queue a copy of the first n particles' state at the current level (no wait)."""
    _check(_lib.vlb_particle_state_async(h, int(n)), h)


def vlb_particle_state_wait(h, n: int, out: dict | None = None) -> tuple[dict, int]:
    """The oldest queued copy (as vlb_get_particle_state returns it) and its step.
    `out` (a dict of arrays from an earlier call) is filled in place when given."""
    if out is None:
        out = {"xy": np.empty((n, 2)), "uv": np.empty((n, 2)), "force": np.empty((n, 2)),
               "theta": np.empty(n), "omega": np.empty(n), "torque": np.empty(n)}
    step = ctypes.c_int64()
    _check(_lib.vlb_particle_state_wait(h, int(n), _ptr(out["xy"]), _ptr(out["theta"]), _ptr(out["uv"]),
                                        _ptr(out["omega"]), _ptr(out["force"]), _ptr(out["torque"]),
                                        ctypes.byref(step)), h)
    return out, step.value


def vlb_get_audit(h):
    m, e, g = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_lib.vlb_get_audit(h, ctypes.byref(m), ctypes.byref(e), ctypes.byref(g)), h)
    return m.value, e.value, g.value


def vlb_get_solid_fraction(h, nx: int, ny: int):
    count = np.empty((ny, nx), dtype=np.uint8)
    owner = np.empty((ny, nx, 4), dtype=np.int32)
    flag = np.empty((ny, nx, 4), dtype=np.uint8)
    fsp = np.empty((ny, nx, 4), dtype=np.float64)
    _check(_lib.vlb_get_solid_fraction(h, _ptr(count, ctypes.c_uint8), _ptr(owner, ctypes.c_int32),
                                       _ptr(flag, ctypes.c_uint8), _ptr(fsp)), h)
    return count, owner, flag, fsp


VLB_NOALLOC_MAX_CELLS = 65536


def vlb_get_solid_fraction_noalloc(h, nx: int, ny: int):
    """Same outputs as vlb_get_solid_fraction, from the library's static
    device scratch instead of per-call device allocations (see include/vlb.h
    for the limits: at most VLB_NOALLOC_MAX_CELLS cells, initialised handle,
    calls must not overlap on the GPU)."""
    count = np.empty((ny, nx), dtype=np.uint8)
    owner = np.empty((ny, nx, 4), dtype=np.int32)
    flag = np.empty((ny, nx, 4), dtype=np.uint8)
    fsp = np.empty((ny, nx, 4), dtype=np.float64)
    _check(_lib.vlb_get_solid_fraction_noalloc(h, _ptr(count, ctypes.c_uint8), _ptr(owner, ctypes.c_int32),
                                               _ptr(flag, ctypes.c_uint8), _ptr(fsp)), h)
    return count, owner, flag, fsp


def vlb_get_contact_pairs(h) -> np.ndarray:
    n = ctypes.c_int32()
    _check(_lib.vlb_get_contact_pairs(h, 0, None, ctypes.byref(n)), h)
    buf = np.empty(2 * max(n.value, 1), dtype=np.int32)
    _check(_lib.vlb_get_contact_pairs(h, n.value, _ptr(buf, ctypes.c_int32), ctypes.byref(n)), h)
    return buf[: 2 * n.value].reshape(-1, 2)


def vlb_set_fixed_temperature(h, held, first: int = 0) -> None:
    """Hold particles first .. first + len(held) - 1 at their temperature T0: held 1 (reading R11, the covered
    part of each cell), 2 (reading R11b, every owned cell whole), 0 conduct."""
    a = np.ascontiguousarray(np.asarray(held, dtype=np.int32))
    _check(_lib.vlb_set_fixed_temperature(h, int(first), int(a.size), _ptr(a, ctypes.c_int32)), h)


def vlb_state_size(h) -> int:
    n = ctypes.c_uint64()
    _check(_lib.vlb_state_size(h, ctypes.byref(n)), h)
    return n.value


def vlb_save_state(h) -> np.ndarray:
    """The handle's state image (checkpoint) as a uint8 array."""
    buf = np.empty(vlb_state_size(h), dtype=np.uint8)
    _check(_lib.vlb_save_state(h, buf.ctypes.data_as(ctypes.c_void_p), buf.nbytes), h)
    return buf


def vlb_load_state(h, image) -> None:
    """Restore a state image (from vlb_save_state, or its bytes read back from a file)."""
    buf = np.ascontiguousarray(np.frombuffer(image, dtype=np.uint8) if isinstance(image, (bytes, bytearray))
                               else image, dtype=np.uint8)
    _check(_lib.vlb_load_state(h, buf.ctypes.data_as(ctypes.c_void_p), buf.nbytes), h)


def vlb_profile_begin(h, max_steps: int):
    _check(_lib.vlb_profile_begin(h, int(max_steps)), h)


def vlb_profile_end(h):
    ms, nl, lps = ctypes.c_double(), ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.vlb_profile_end(h, ctypes.byref(ms), ctypes.byref(nl), ctypes.byref(lps)), h)
    return ms.value, nl.value, lps.value


def vlb_last_error(h=None) -> str:
    msg = _lib.vlb_last_error(h)
    return msg.decode() if msg else ""


def vlb_destroy(h):
    if h is not None and h.value:
        _lib.vlb_destroy(h)
        h.value = None


class Lattice:
    """Owning wrapper of one handle (closes it on exit)."""

    def __init__(self, params: vlb_params):
        self.params = params
        self.nx, self.ny = params.nx, params.ny
        self.h = vlb_create(params)

    def add_particles(self, *a, **k):
        vlb_add_particles(self.h, *a, **k)

    def add_ellipses(self, *a, **k):
        vlb_add_ellipses(self.h, *a, **k)

    def step(self, n: int = 1):
        vlb_step(self.h, n)

    def insert_particles(self, *a, **k):
        vlb_insert_particles(self.h, *a, **k)

    def fields(self, mask: int = VLB_FIELD_ALL) -> dict:
        return vlb_get_fields(self.h, self.nx, self.ny, mask)

    def particles(self) -> dict:
        return vlb_get_particle_state(self.h)

    def audit(self):
        return vlb_get_audit(self.h)

    def save_state(self, path=None):
        """Checkpoint: the state image, also written to `path` if given."""
        img = vlb_save_state(self.h)
        if path is not None:
            img.tofile(path)
        return img

    def load_state(self, image_or_path):
        """Resume from a state image (array, bytes or a file written by save_state)."""
        img = np.fromfile(image_or_path, dtype=np.uint8) if isinstance(image_or_path, (str, os.PathLike)) \
            else image_or_path
        vlb_load_state(self.h, img)

    def close(self):
        vlb_destroy(self.h)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def vlb_device_bytes(params: vlb_params, radius) -> int:
    """Device bytes of a handle of these parameters with particles of these radii."""
    radius = np.ascontiguousarray(radius, dtype=np.float64).reshape(-1)
    out = ctypes.c_uint64()
    _check(_lib.vlb_device_bytes(ctypes.byref(params), radius.shape[0], _ptr(radius) if radius.size else None,
                                 ctypes.byref(out)))
    return out.value


class Server:
    """Served mode (vlb_serve_*): cases are submitted as they arrive, admitted
    by HBM budget, stepped together, and their results taken when done."""

    def __init__(self, hbm_budget: int = 0, steps_per_round: int = 100, max_active: int = 0):
        sp = vlb_serve_params()
        _check(_lib.vlb_serve_params_default(ctypes.byref(sp)))
        sp.hbm_budget, sp.steps_per_round, sp.max_active = int(hbm_budget), int(steps_per_round), int(max_active)
        self.s = ctypes.c_void_p()
        st = _lib.vlb_serve_create(ctypes.byref(sp), ctypes.byref(self.s))
        if st != VLB_OK:
            raise VlbError(st, (_lib.vlb_serve_last_error(None) or b"").decode())

    def _check(self, st):
        if st != VLB_OK:
            raise VlbError(st, (_lib.vlb_serve_last_error(self.s) or b"").decode())

    def submit(self, params: vlb_params, xy, radius, T0, nsteps: int, k_ratio=None) -> int:
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1)
        radius = np.ascontiguousarray(radius, dtype=np.float64).reshape(-1)
        T0 = np.ascontiguousarray(T0, dtype=np.float64).reshape(-1)
        k = None if k_ratio is None else np.ascontiguousarray(k_ratio, dtype=np.float64).reshape(-1)
        cid = ctypes.c_int64()
        self._check(_lib.vlb_serve_submit(self.s, ctypes.byref(params), radius.shape[0], _ptr(xy), _ptr(radius),
                                          _ptr(T0), _ptr(k), int(nsteps), ctypes.byref(cid)))
        return cid.value

    def poll(self):
        """One round; returns (queued, active, finished)."""
        q, a, d = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(_lib.vlb_serve_poll(self.s, ctypes.byref(q), ctypes.byref(a), ctypes.byref(d)))
        return q.value, a.value, d.value

    def info(self, cid: int) -> dict:
        st, nx, ny, n = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        t = np.zeros(3)
        self._check(_lib.vlb_serve_case_info(self.s, int(cid), ctypes.byref(st), ctypes.byref(nx), ctypes.byref(ny),
                                             ctypes.byref(n), _ptr(t)))
        return {"state": st.value, "nx": nx.value, "ny": ny.value, "n": n.value, "t_submit": t[0],
                "t_admit": t[1], "t_done": t[2]}

    def take(self, cid: int):
        """(fields dict as Lattice.fields() gives it, particle dict) of a finished case."""
        i = self.info(cid)
        nx, ny, n = i["nx"], i["ny"], i["n"]
        f = {k: np.empty((ny, nx)) for k in ("rho", "ux", "uy", "T", "fs")}
        ps = np.empty((max(n, 1), 9))
        self._check(_lib.vlb_serve_take(self.s, int(cid), _ptr(f["rho"]), _ptr(f["ux"]), _ptr(f["uy"]), _ptr(f["T"]),
                                        _ptr(f["fs"]), _ptr(ps)))
        ps = ps[:n]
        names = ("x", "y", "theta", "ux", "uy", "omega", "fx", "fy", "torque")
        return f, {k: ps[:, j].copy() for j, k in enumerate(names)}

    def close(self):
        if self.s is not None and self.s.value:
            _lib.vlb_serve_destroy(self.s)
            self.s.value = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
