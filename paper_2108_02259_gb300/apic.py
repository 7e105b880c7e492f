"""Thin ctypes binding of libapiccontact (include/apiccontact.h).

Argument marshalling only: every step of the contact computation runs in the
library's CUDA kernels.  Device arrays are torch CUDA tensors (pointers and
the current torch stream are passed through); host arrays are numpy arrays
(the call sets APIC_HOST_PTRS and the library copies in and out).

The library must have been built (``paper_2108_02259_gb300.build.build()``);
loading fails loudly otherwise.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libapiccontact.so")
# APIC_DEBUG_BOUNDS=1 in the environment loads the bounds-checking build
# (build.build(debug=True)) instead
if os.environ.get("APIC_DEBUG_BOUNDS") == "1":
    LIB_PATH = os.path.join(_PKG, "libapiccontact_debug.so")

APIC_OK = 0
APIC_ERR_INVALID_ARG = -1
APIC_ERR_OUT_OF_MEMORY = -2
APIC_ERR_CUDA = -3
APIC_ERR_TIMEOUT = -4
APIC_ERR_ADMISSION = -5
APIC_ERR_NOT_READY = -6

APIC_FP64 = 1 << 0
APIC_HOST_PTRS = 1 << 1
APIC_VARIANT_PIC = 1 << 2
APIC_VARIANT_SEP23 = 1 << 3
APIC_DETERMINISTIC = 1 << 5
APIC_CHECK = 1 << 6
APIC_MASS_NORMALS = 1 << 7
APIC_PARTITIONED = 1 << 8  # batched scenes are partitions of one scene (grid sums shared)
APIC_AUGURY_INIT = 1 << 4

EXPORTED = [
    "apic_last_error", "apic_version", "apic_create", "apic_destroy", "apic_contact_step",
    "apic_set_profiling", "apic_get_profile", "apic_scratch_bytes", "apic_contact_step_static",
    "apic_contact_step_batched", "apic_server_create", "apic_server_destroy", "apic_sim_open", "apic_sim_submit",
    "apic_ticket_poll", "apic_ticket_wait", "apic_sim_read", "apic_sim_close", "apic_server_get_stats",
    "apic_variant_count", "apic_variant_name", "apic_set_variant", "apic_get_variant", "apic_autotune",
    "apic_set_graphs", "apic_set_overlap", "apic_set_allocator", "apic_get_tuning", "apic_set_tuning",
    "apic_server_set_policy", "apic_node_normals",
    "apic_augury_steps",
    "apic_sim_export", "apic_sim_import", "apic_mass_normals",
    "apic_place_by_budget", "apic_group_create", "apic_group_destroy", "apic_group_server", "apic_group_set_policy",
    "apic_group_open", "apic_group_get_stats", "apic_sim_server", "apic_debug_build", "apic_debug_flags",
]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_int32)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t, C.c_int32)


MAX_BODIES = 32  # bodies per scene (the width of the node body masks)


def _default_n_bodies(body, n: int) -> int:
    """n_bodies when the caller gives none: one more than the largest body
    id for host arrays; for device tensors the limit of 32, an upper bound
    that needs no device read (results do not depend on it; a per-pair
    friction table needs the true count)."""
    if n == 0:
        return 1
    if _is_torch(body):
        return MAX_BODIES
    return int(np.asarray(body).max()) + 1


class StepArgs(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("n_bodies", C.c_int32), ("n_iter", C.c_int32),
        ("body", C.c_void_p), ("x", C.c_void_p), ("v", C.c_void_p), ("C", C.c_void_p),
        ("m", C.c_void_p), ("nrm", C.c_void_p), ("v_out", C.c_void_p), ("C_out", C.c_void_p),
        ("h", C.c_double), ("mu", C.c_double), ("mu_pair", C.c_void_p), ("flags", C.c_uint32),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("P_in", C.c_double * 3), ("P_out", C.c_double * 3), ("L_in", C.c_double * 3),
        ("L_out", C.c_double * 3), ("multibody_nodes", C.c_int64), ("active_blocks", C.c_int64),
        ("work_items", C.c_int64), ("E_in", C.c_double), ("E_out", C.c_double),
    ]

    def as_dict(self):
        return dict(P_in=np.array(self.P_in[:]), P_out=np.array(self.P_out[:]), L_in=np.array(self.L_in[:]),
                    L_out=np.array(self.L_out[:]), multibody_nodes=int(self.multibody_nodes),
                    active_blocks=int(self.active_blocks), work_items=int(self.work_items),
                    E_in=float(self.E_in), E_out=float(self.E_out))


class ServerStats(C.Structure):
    _fields_ = [
        ("completed", C.c_int64), ("failed", C.c_int64), ("batches", C.c_int64), ("particle_iters", C.c_int64),
        ("latency_p50_ms", C.c_double), ("latency_p99_ms", C.c_double), ("latency_mean_ms", C.c_double),
        ("mean_batch_scenes", C.c_double), ("resident_bytes", C.c_int64), ("open_sims", C.c_int64),
    ]


class Profile(C.Structure):
    _fields_ = [
        ("steps", C.c_int64), ("iter_launches", C.c_int64), ("iter_ms", C.c_double), ("prep_ms", C.c_double),
        ("step_ms", C.c_double), ("particles", C.c_int64), ("active_nodes", C.c_int64),
        ("kernel_launches", C.c_int64), ("sort_launches", C.c_int64), ("mass_ms", C.c_double),
        ("graph_launches", C.c_int64),
    ]


_lib = None


class AuguryArgs(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("n_bodies", C.c_int32), ("n_iter", C.c_int32), ("body", C.c_void_p),
        ("x", C.c_void_p), ("v", C.c_void_p), ("C", C.c_void_p), ("av", C.c_void_p), ("aC", C.c_void_p),
        ("m", C.c_void_p), ("fixed", C.c_void_p), ("n_springs", C.c_int64), ("springs", C.c_void_p),
        ("rest", C.c_void_p), ("stiffness", C.c_void_p), ("gravity", C.c_double * 3), ("n_tri", C.c_int64),
        ("tri", C.c_void_p), ("h", C.c_double), ("mu", C.c_double), ("mu_pair", C.c_void_p), ("dt", C.c_double),
        ("tau", C.c_double), ("flags", C.c_uint32),
    ]


class AuguryStats(C.Structure):
    _fields_ = [("P", C.c_double * 3), ("L", C.c_double * 3), ("kinetic", C.c_double), ("springs", C.c_double),
                ("gravity", C.c_double)]

    def as_dict(self):
        return {"P": np.array(self.P[:]), "L": np.array(self.L[:]), "kinetic": self.kinetic,
                "springs": self.springs, "gravity": self.gravity}


class ApicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libapiccontact error {code}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    """Load the library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with paper_2108_02259_gb300.build.build()")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.apic_last_error.restype = C.c_char_p
    lib.apic_version.restype = C.c_char_p
    lib.apic_create.argtypes = [C.POINTER(P), C.c_int32, C.c_size_t]
    lib.apic_destroy.argtypes = [P]
    lib.apic_contact_step.argtypes = [P, C.POINTER(StepArgs), P, C.POINTER(Stats)]
    lib.apic_server_create.argtypes = [C.POINTER(P), C.c_int32, C.c_size_t, C.c_int32, C.c_int32]
    lib.apic_server_destroy.argtypes = [P]
    lib.apic_sim_open.argtypes = [P, C.POINTER(StepArgs), C.POINTER(P)]
    lib.apic_sim_submit.argtypes = [P, C.c_double, C.POINTER(C.c_uint64)]
    lib.apic_ticket_poll.argtypes = [P, C.c_uint64, C.POINTER(C.c_int32), C.POINTER(C.c_double)]
    lib.apic_ticket_wait.argtypes = [P, C.c_uint64, C.c_double, C.POINTER(C.c_double)]
    lib.apic_sim_read.argtypes = [P, P, P, P]
    lib.apic_sim_close.argtypes = [P]
    lib.apic_server_get_stats.argtypes = [P, C.POINTER(ServerStats), C.c_int32]
    for f in ("apic_server_create", "apic_server_destroy", "apic_sim_open", "apic_sim_submit", "apic_ticket_poll",
              "apic_ticket_wait", "apic_sim_read", "apic_sim_close", "apic_server_get_stats"):
        getattr(lib, f).restype = C.c_int32
    lib.apic_contact_step_batched.argtypes = [P, C.POINTER(StepArgs), C.c_int32, P, C.POINTER(Stats)]
    lib.apic_contact_step_batched.restype = C.c_int32
    lib.apic_debug_build.restype = C.c_int32
    lib.apic_debug_flags.argtypes = [C.POINTER(C.c_uint32), C.c_int32]
    lib.apic_debug_flags.restype = C.c_int32
    lib.apic_place_by_budget.argtypes = [P, C.c_int32, C.c_int64]
    lib.apic_place_by_budget.restype = C.c_int32
    lib.apic_group_create.argtypes = [C.POINTER(P), P, C.c_int32, C.c_size_t, C.c_int32, C.c_int32]
    lib.apic_group_destroy.argtypes = [P]
    lib.apic_group_server.argtypes = [P, C.c_int32, C.POINTER(P)]
    lib.apic_group_set_policy.argtypes = [P, C.c_int32, C.c_int32]
    lib.apic_group_open.argtypes = [P, C.POINTER(StepArgs), C.POINTER(P), C.POINTER(C.c_int32)]
    lib.apic_group_get_stats.argtypes = [P, C.POINTER(ServerStats), C.c_int32]
    lib.apic_sim_server.argtypes = [P, C.POINTER(P)]
    for f in ("apic_group_create", "apic_group_destroy", "apic_group_server", "apic_group_set_policy",
              "apic_group_open", "apic_group_get_stats", "apic_sim_server"):
        getattr(lib, f).restype = C.c_int32
    lib.apic_mass_normals.argtypes = [P, C.POINTER(StepArgs), C.c_double, P, P]
    lib.apic_mass_normals.restype = C.c_int32
    lib.apic_contact_step_static.argtypes = [C.POINTER(StepArgs), P, C.POINTER(Stats)]
    lib.apic_contact_step_static.restype = C.c_int32
    lib.apic_set_profiling.argtypes = [P, C.c_int32]
    lib.apic_get_profile.argtypes = [P, C.POINTER(Profile)]
    lib.apic_scratch_bytes.argtypes = [P, C.POINTER(C.c_size_t)]
    lib.apic_variant_count.argtypes = []
    lib.apic_variant_count.restype = C.c_int32
    lib.apic_variant_name.argtypes = [C.c_int32]
    lib.apic_variant_name.restype = C.c_char_p
    lib.apic_set_variant.argtypes = [P, C.c_int32]
    lib.apic_get_variant.argtypes = [P, C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.apic_autotune.argtypes = [P, C.POINTER(StepArgs), C.c_int32, P, C.POINTER(C.c_int32)]
    lib.apic_set_graphs.argtypes = [P, C.c_int32]
    lib.apic_set_overlap.argtypes = [P, C.c_int32]
    lib.apic_set_allocator.argtypes = [P, ALLOC_FN, FREE_FN, P]
    I32P = C.POINTER(C.c_int32)
    lib.apic_get_tuning.argtypes = [P, I32P, I32P, C.c_int32, I32P]
    lib.apic_set_tuning.argtypes = [P, I32P, I32P, C.c_int32]
    lib.apic_server_set_policy.argtypes = [P, C.c_int32, C.c_int32]
    lib.apic_node_normals.argtypes = [P, C.c_int64, P, C.c_int64, P, P, C.c_uint32, P]
    lib.apic_node_normals.restype = C.c_int32
    lib.apic_augury_steps.argtypes = [P, C.POINTER(AuguryArgs), C.c_int32, P, C.POINTER(AuguryStats)]
    lib.apic_augury_steps.restype = C.c_int32
    lib.apic_sim_export.argtypes = [P, P, C.POINTER(C.c_size_t)]
    lib.apic_sim_export.restype = C.c_int32
    lib.apic_sim_import.argtypes = [P, P, C.c_size_t, C.POINTER(P)]
    lib.apic_sim_import.restype = C.c_int32
    lib.apic_server_set_policy.restype = C.c_int32
    for f in ("apic_create", "apic_destroy", "apic_contact_step", "apic_set_profiling", "apic_get_profile",
              "apic_scratch_bytes", "apic_set_variant", "apic_get_variant", "apic_autotune", "apic_set_graphs",
              "apic_set_overlap", "apic_set_allocator", "apic_get_tuning", "apic_set_tuning"):
        getattr(lib, f).restype = C.c_int32
    _lib = lib
    return lib


def _check(code):
    if code != APIC_OK:
        raise ApicError(code, load().apic_last_error().decode())


class Context:
    """An apic_ctx on one CUDA device (scratch grows on demand)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        lib = load()
        h = C.c_void_p()
        _check(lib.apic_create(C.byref(h), int(device), int(hbm_budget_bytes)))
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            load().apic_destroy(self._h)
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

    @property
    def handle(self):
        return self._h

    def set_profiling(self, on: bool):
        _check(load().apic_set_profiling(self._h, 1 if on else 0))

    def profile(self) -> dict:
        p = Profile()
        _check(load().apic_get_profile(self._h, C.byref(p)))
        return {k: getattr(p, k) for k, _ in Profile._fields_}

    def scratch_bytes(self) -> int:
        v = C.c_size_t()
        _check(load().apic_scratch_bytes(self._h, C.byref(v)))
        return int(v.value)

    def set_variant(self, v: int):
        """Fix the transfer-kernel variant (-1: tune per size class)."""
        _check(load().apic_set_variant(self._h, int(v)))

    def variant(self, n_particles: int) -> tuple[int, bool]:
        """(variant, decided) for a call of n_particles FP32 particles."""
        v, d = C.c_int32(), C.c_int32()
        _check(load().apic_get_variant(self._h, int(n_particles), C.byref(v), C.byref(d)))
        return int(v.value), bool(d.value)

    def autotune(self, scenes, n_iter: int, flags: int = 0, stream=None) -> int:
        """Tune the size class of these BatchScene now (their outputs are
        overwritten); returns the chosen variant."""
        arr, ns, sptr, _keep = _batch_args(scenes, n_iter, flags, stream)
        v = C.c_int32()
        _check(load().apic_autotune(self._h, arr, ns, sptr, C.byref(v)))
        return int(v.value)

    def set_graphs(self, on: bool):
        """Replay the transfer passes as a CUDA graph (default) or not."""
        _check(load().apic_set_graphs(self._h, 1 if on else 0))

    def set_allocator(self, alloc, free):
        """Serve the context's scratch from alloc(nbytes, device) -> int
        device pointer (256-byte aligned, 0 on failure) and free(ptr, nbytes,
        device), e.g. torch.cuda.caching_allocator_alloc / _delete.  Before
        the first step only."""
        def a(_user, nbytes, device):
            try:
                return int(alloc(int(nbytes), int(device)))
            except Exception:
                return 0

        def f(_user, ptr, nbytes, device):
            free(int(ptr), int(nbytes), int(device))

        cbs = (ALLOC_FN(a), FREE_FN(f))
        _check(load().apic_set_allocator(self._h, cbs[0], cbs[1], None))
        self._alloc_cbs = cbs  # the library calls them until the context is destroyed

    def tuning(self) -> dict:
        """{size class: variant} for every class the autotuner has decided."""
        lib, cnt = load(), C.c_int32()
        _check(lib.apic_get_tuning(self._h, None, None, 0, C.byref(cnt)))
        n = cnt.value
        cls, var = (C.c_int32 * max(n, 1))(), (C.c_int32 * max(n, 1))()
        _check(lib.apic_get_tuning(self._h, cls, var, n, C.byref(cnt)))
        return {int(cls[i]): int(var[i]) for i in range(min(n, cnt.value))}

    def set_tuning(self, table: dict):
        """Mark size classes decided: {size class: variant}."""
        n = len(table)
        cls = (C.c_int32 * max(n, 1))(*[int(k) for k in table])
        var = (C.c_int32 * max(n, 1))(*[int(v) for v in table.values()])
        _check(load().apic_set_tuning(self._h, cls, var, n))

    def save_tuning(self, path: str):
        """Write the decided classes to a JSON file keyed by GPU model and
        the library's variant list."""
        import json

        import torch

        doc = {"gpu": torch.cuda.get_device_name(self.device), "variants": variants(),
               "classes": {str(k): v for k, v in sorted(self.tuning().items())}}
        with open(path, "w") as fh:
            json.dump(doc, fh, indent=1)

    def load_tuning(self, path: str) -> bool:
        """Apply a file from save_tuning if it was made on this GPU model with
        these variants; returns whether it was applied."""
        import json

        import torch

        doc = json.load(open(path))
        if doc.get("gpu") != torch.cuda.get_device_name(self.device) or doc.get("variants") != variants():
            return False
        self.set_tuning({int(k): int(v) for k, v in doc.get("classes", {}).items()})
        return True

    def set_overlap(self, on: bool):
        """Let each pass start while the grid before it finishes (default) or not."""
        _check(load().apic_set_overlap(self._h, 1 if on else 0))


def variants() -> list[str]:
    """Descriptions of the transfer-kernel variants, by index."""
    lib = load()
    return [lib.apic_variant_name(i).decode() for i in range(lib.apic_variant_count())]


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        return a.data_ptr()
    if a.flags.writeable and a.size:
        # (cheaper than a.ctypes.data, which builds a helper object per call)
        return C.addressof(C.c_char.from_buffer(a))
    return a.ctypes.data


@dataclass
class StepResult:
    v: object
    C: object
    stats: dict | None


def contact_step(ctx: Context, x, v, Cm, m, nrm, body, h: float, mu: float, n_iter: int, n_bodies: int | None = None,
                 mu_pair=None, flags: int = 0, v_out=None, C_out=None, stream=None, stats: bool = False) -> StepResult:
    """One contact step through the C ABI.

    Device path: x float64 [n,3], v [n,3], C [n,3,3], m [n], nrm [n,3] (all float32,
    or all float64 for the FP64 build), body int32 [n] -- torch CUDA tensors,
    contiguous.  Host path: the same as numpy arrays.  Outputs are allocated when
    not given (in place is allowed).  `stream` is a torch.cuda.Stream (default:
    the current one)."""
    lib = load()
    dev = _is_torch(x)
    n = int(x.shape[0])
    dt = v.dtype
    if dev:
        import torch

        fp64 = dt == torch.float64
        for t in (x, v, Cm, m, nrm, body):
            if t is not None and (not t.is_cuda or not t.is_contiguous()):
                raise ValueError("device path wants contiguous CUDA tensors")
        if x.dtype != torch.float64 or body.dtype != torch.int32:
            raise ValueError("x must be float64 and body int32")
        if any(t.dtype != dt for t in (Cm, m, nrm) if t is not None):
            raise ValueError("v, C, m, nrm must share one dtype")
        if v_out is None:
            v_out = torch.empty_like(v)
        if C_out is None:
            C_out = torch.empty_like(Cm)
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        sptr = stream.cuda_stream
    else:
        fp64 = dt == np.float64
        x = np.ascontiguousarray(x, np.float64)
        body = np.ascontiguousarray(body, np.int32)
        v, Cm, m = (np.ascontiguousarray(a, dt) for a in (v, Cm, m))
        nrm = None if nrm is None else np.ascontiguousarray(nrm, dt)
        if v_out is None:
            v_out = np.empty_like(v)
        if C_out is None:
            C_out = np.empty_like(Cm)
        sptr = None if stream is None else stream.cuda_stream
        flags |= APIC_HOST_PTRS
    if fp64:
        flags |= APIC_FP64
    if nrm is None:
        flags |= APIC_MASS_NORMALS  # normals from the bodies' grid mass
    if n_bodies is None:
        if mu_pair is not None:
            raise ValueError("a per-pair friction table needs n_bodies")
        n_bodies = _default_n_bodies(body, n)
    mp = None
    if mu_pair is not None:
        mp = np.ascontiguousarray(np.asarray(mu_pair, np.float64).reshape(n_bodies, n_bodies))
    a = StepArgs(n, int(n_bodies), int(n_iter), _ptr(body), _ptr(x), _ptr(v), _ptr(Cm), _ptr(m), _ptr(nrm),
                 _ptr(v_out), _ptr(C_out), float(h), float(mu), None if mp is None else mp.ctypes.data, int(flags))
    st = Stats() if stats else None
    _check(lib.apic_contact_step(ctx.handle, C.byref(a), sptr, C.byref(st) if stats else None))
    return StepResult(v_out, C_out, st.as_dict() if stats else None)


MASS_NORMAL_THRESHOLD = 0.5  # the threshold APIC_MASS_NORMALS uses


def mass_normals(ctx: Context, x, m, body, h: float, n_bodies: int | None = None,
                 threshold: float = MASS_NORMAL_THRESHOLD, out=None, stream=None, deterministic: bool = False):
    """apic_mass_normals: normals from each body's grid mass, in the
    caller's order.  x [n,3] float64, m [n] float32 (or float64 for the
    FP64 path), body [n] int32: torch CUDA tensors.  Returns out [n,3]."""
    import torch

    lib = load()
    n = int(x.shape[0])
    for t in (x, m, body):
        if not t.is_cuda or not t.is_contiguous() or t.device != x.device:
            raise ValueError("apic_mass_normals wants contiguous CUDA tensors on one device")
    flags = APIC_FP64 if m.dtype == torch.float64 else 0
    if deterministic:
        flags |= APIC_DETERMINISTIC
    if out is None:
        out = torch.empty((n, 3), dtype=m.dtype, device=x.device)
    if stream is None:
        stream = torch.cuda.current_stream(x.device)
    if n_bodies is None:
        n_bodies = _default_n_bodies(body, n)
    a = StepArgs(n, int(n_bodies), 0, _ptr(body), _ptr(x), None, None, _ptr(m), None, None, None, float(h), 0.0,
                 None, int(flags))
    _check(lib.apic_mass_normals(ctx.handle, C.byref(a), float(threshold), _ptr(out), stream.cuda_stream))
    return out


def contact_step_static(x, v, Cm, m, nrm, body, h: float, mu: float, n_iter: int, n_bodies: int | None = None,
                        mu_pair=None, flags: int = 0, v_out=None, C_out=None, stream=None,
                        stats: bool = False) -> StepResult:
    """apic_contact_step_static: the same step with no device allocation at all
    (scratch from the library's fixed static device array).  Torch CUDA
    tensors only, same layouts as contact_step."""
    import torch

    lib = load()
    n = int(x.shape[0])
    dt = v.dtype
    for t in (x, v, Cm, m, nrm, body):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("apic_contact_step_static wants contiguous CUDA tensors")
        if t.device != x.device:
            raise ValueError(f"apic_contact_step_static: tensors on {t.device} and {x.device}")
    for t in (v_out, C_out):
        if t is not None and (t.device != x.device or not t.is_contiguous()):
            raise ValueError("apic_contact_step_static: outputs must be contiguous tensors on the inputs' device")
    if stream is not None and stream.device != x.device:
        raise ValueError(f"apic_contact_step_static: stream of {stream.device}, tensors on {x.device}")
    if dt == torch.float64:
        flags |= APIC_FP64
    if v_out is None:
        v_out = torch.empty_like(v)
    if C_out is None:
        C_out = torch.empty_like(Cm)
    if stream is None:
        stream = torch.cuda.current_stream(x.device)
    if n_bodies is None:
        if mu_pair is not None:
            raise ValueError("a per-pair friction table needs n_bodies")
        n_bodies = _default_n_bodies(body, n)
    mp = None
    if mu_pair is not None:
        mp = np.ascontiguousarray(np.asarray(mu_pair, np.float64).reshape(n_bodies, n_bodies))
    a = StepArgs(n, int(n_bodies), int(n_iter), _ptr(body), _ptr(x), _ptr(v), _ptr(Cm), _ptr(m), _ptr(nrm),
                 _ptr(v_out), _ptr(C_out), float(h), float(mu), None if mp is None else mp.ctypes.data, int(flags))
    st = Stats() if stats else None
    # the library's static array belongs to the current device: make it the
    # tensors' device for the call
    with torch.cuda.device(x.device):
        _check(lib.apic_contact_step_static(C.byref(a), stream.cuda_stream, C.byref(st) if stats else None))
    return StepResult(v_out, C_out, st.as_dict() if stats else None)


def node_normals(ctx: Context, x, tri, fp64: bool = False, out=None, stream=None):
    """apic_node_normals: area-weighted unit normals of the boundary faces
    around each node (Sec. 2.3).  x [n, 3] float64 and tri [n_tri, 3] int32,
    both torch CUDA tensors (device path) or both numpy arrays (host path).
    Returns out [n, 3] (float32, or float64 with fp64)."""
    lib = load()
    n = int(x.shape[0])
    n_tri = int(tri.shape[0])
    flags = APIC_FP64 if fp64 else 0
    if _is_torch(x):
        import torch

        if out is None:
            out = torch.empty((n, 3), dtype=torch.float64 if fp64 else torch.float32, device=x.device)
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        sptr = stream.cuda_stream
    else:
        flags |= APIC_HOST_PTRS
        x = np.ascontiguousarray(x, np.float64)
        tri = np.ascontiguousarray(tri, np.int32)
        if out is None:
            out = np.empty((n, 3), np.float64 if fp64 else np.float32)
        sptr = None if stream is None else stream.cuda_stream
    _check(lib.apic_node_normals(ctx.handle, n, _ptr(x), n_tri, _ptr(tri) if n_tri else None, _ptr(out), flags,
                                 sptr))
    return out


def augury_steps(ctx: Context, x, v, Cm, av, aC, m, body, springs, rest, stiffness, tri, h: float, mu: float,
                 n_iter: int, dt: float, tau: float, n_steps: int, gravity=(0.0, 0.0, 0.0), fixed=None,
                 n_bodies: int | None = None, mu_pair=None, flags: int = 0, init: bool = False, stream=None,
                 stats: bool = False):
    """apic_augury_steps on torch CUDA tensors, advanced in place: x [n,3]
    float64; v [n,3], Cm [n,9], av [n,3], aC [n,9], m [n] float32 (or all
    float64 for the FP64 path); body int32; springs [S,2] int32; rest and
    stiffness float64; tri [T,3] int32; fixed uint8 or None.  Returns the
    final-state stats dict (or None)."""
    import torch

    lib = load()
    if v.dtype == torch.float64:
        flags |= APIC_FP64
    if init:
        flags |= APIC_AUGURY_INIT
    n = int(x.shape[0])
    if n_bodies is None:
        if mu_pair is not None:
            raise ValueError("a per-pair friction table needs n_bodies")
        n_bodies = _default_n_bodies(body, n)
    mp = None
    if mu_pair is not None:
        mp = np.ascontiguousarray(np.asarray(mu_pair, np.float64).reshape(n_bodies, n_bodies))
    a = AuguryArgs(n, int(n_bodies), int(n_iter), _ptr(body), _ptr(x), _ptr(v), _ptr(Cm), _ptr(av), _ptr(aC), _ptr(m),
                   _ptr(fixed), int(springs.shape[0]), _ptr(springs) if springs.shape[0] else None,
                   _ptr(rest) if springs.shape[0] else None, _ptr(stiffness) if springs.shape[0] else None,
                   (C.c_double * 3)(*[float(g) for g in gravity]), int(tri.shape[0]),
                   _ptr(tri) if tri.shape[0] else None, float(h), float(mu), None if mp is None else mp.ctypes.data,
                   float(dt), float(tau), int(flags))
    if stream is None:
        stream = torch.cuda.current_stream(x.device)
    st = AuguryStats()
    _check(lib.apic_augury_steps(ctx.handle, C.byref(a), int(n_steps), stream.cuda_stream,
                                 C.byref(st) if stats else None))
    return st.as_dict() if stats else None


class BatchScene:
    """One scene of a batched call: device tensors (or numpy arrays for the
    host path) in the layouts of contact_step."""

    def __init__(self, x, v, Cm, m, nrm, body, h, mu, n_bodies=None, mu_pair=None, v_out=None, C_out=None):
        self.x, self.v, self.C, self.m, self.nrm, self.body = x, v, Cm, m, nrm, body
        self.h, self.mu, self.mu_pair = float(h), float(mu), mu_pair
        n = int(x.shape[0])
        if n_bodies is None and mu_pair is not None:
            raise ValueError("a per-pair friction table needs n_bodies")
        self.n_bodies = n_bodies if n_bodies is not None else _default_n_bodies(body, n)
        if v_out is None:
            v_out = v.new_empty(v.shape) if _is_torch(v) else np.empty_like(v)
        if C_out is None:
            C_out = Cm.new_empty(Cm.shape) if _is_torch(Cm) else np.empty_like(Cm)
        self.v_out, self.C_out = v_out, C_out


def _batch_args(scenes, n_iter, flags, stream):
    ns = len(scenes)
    dev = _is_torch(scenes[0].x)
    if dev:
        import torch

        fp64 = scenes[0].v.dtype == torch.float64
        if stream is None:
            stream = torch.cuda.current_stream(scenes[0].x.device)
        sptr = stream.cuda_stream
    else:
        fp64 = scenes[0].v.dtype == np.float64
        sptr = None if stream is None else stream.cuda_stream
        flags |= APIC_HOST_PTRS
    if fp64:
        flags |= APIC_FP64
    arr = (StepArgs * ns)()
    keep = []
    for i, sc in enumerate(scenes):
        mp = None
        if sc.mu_pair is not None:
            mp = np.ascontiguousarray(np.asarray(sc.mu_pair, np.float64).reshape(sc.n_bodies, sc.n_bodies))
            keep.append(mp)
        arr[i] = StepArgs(int(sc.x.shape[0]), int(sc.n_bodies), int(n_iter), _ptr(sc.body), _ptr(sc.x), _ptr(sc.v),
                          _ptr(sc.C), _ptr(sc.m), _ptr(sc.nrm), _ptr(sc.v_out), _ptr(sc.C_out), sc.h, sc.mu,
                          None if mp is None else mp.ctypes.data, int(flags))
    return arr, ns, sptr, keep


def contact_step_batched(ctx: Context, scenes, n_iter: int, flags: int = 0, stream=None, stats: bool = False):
    """apic_contact_step_batched over a list of BatchScene (all device or all
    host arrays, one precision).  Returns the per-scene stats (or None); the
    results are in each scene's v_out / C_out."""
    arr, ns, sptr, _keep = _batch_args(scenes, n_iter, flags, stream)
    st = (Stats * ns)() if stats else None
    _check(load().apic_contact_step_batched(ctx.handle, arr, ns, sptr, st if stats else None))
    return [st[i].as_dict() for i in range(ns)] if stats else None


class Server:
    """apic_server: resident simulations stepped by worker threads that batch
    ready requests (continuous batching) under an HBM budget."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, n_workers: int = 2, max_batch_scenes: int = 64):
        lib = load()
        h = C.c_void_p()
        _check(lib.apic_server_create(C.byref(h), int(device), int(hbm_budget_bytes), int(n_workers),
                                      int(max_batch_scenes)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().apic_server_destroy(self._h)
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

    def open_sim(self, x, v, Cm, m, nrm, body, h, mu, n_iter, n_bodies=None, mu_pair=None, flags=0):
        """Admit a simulation from host numpy arrays (or CUDA tensors)."""
        return Sim(self, x, v, Cm, m, nrm, body, h, mu, n_iter, n_bodies, mu_pair, flags)

    def poll(self, ticket):
        done, lat = C.c_int32(), C.c_double()
        _check(load().apic_ticket_poll(self._h, int(ticket), C.byref(done), C.byref(lat)))
        return bool(done.value), (lat.value if done.value else None)

    def wait(self, ticket, timeout_s: float = 60.0):
        lat = C.c_double()
        _check(load().apic_ticket_wait(self._h, int(ticket), float(timeout_s), C.byref(lat)))
        return lat.value

    def import_sim(self, checkpoint: bytes):
        """apic_sim_import: a new simulation resumed from Sim.export()."""
        import struct

        h = C.c_void_p()
        _check(load().apic_sim_import(self._h, checkpoint, len(checkpoint), C.byref(h)))
        _magic, _version, flags, n = struct.unpack_from("<8sIIq", checkpoint, 0)  # validated by the library
        return Sim._adopt(self, h, int(n), np.float64 if flags & APIC_FP64 else np.float32)

    def set_policy(self, variant: int = -1, graphs: bool = True):
        """Launch policy of the worker contexts (see apic_server_set_policy)."""
        _check(load().apic_server_set_policy(self._h, int(variant), 1 if graphs else 0))

    def stats(self, reset: bool = False) -> dict:
        st = ServerStats()
        _check(load().apic_server_get_stats(self._h, C.byref(st), 1 if reset else 0))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}


def _sim_args(x, v, Cm, m, nrm, body, h, mu, n_iter, n_bodies=None, mu_pair=None, flags=0):
    """StepArgs admitting a simulation (host numpy arrays or CUDA tensors),
    with the arrays it points into kept alive in the returned tuple."""
    dev = _is_torch(x)
    if not dev:
        x = np.ascontiguousarray(x, np.float64)
        body = np.ascontiguousarray(body, np.int32)
        dt = np.asarray(v).dtype
        v, Cm, m = (np.ascontiguousarray(a, dt) for a in (v, Cm, m))
        nrm = None if nrm is None else np.ascontiguousarray(nrm, dt)
        flags |= APIC_HOST_PTRS
        fp64 = dt == np.float64
    else:
        import torch

        fp64 = v.dtype == torch.float64
    if fp64:
        flags |= APIC_FP64
    if nrm is None:
        flags |= APIC_MASS_NORMALS
    n = int(x.shape[0])
    if n_bodies is None and mu_pair is not None:
        raise ValueError("a per-pair friction table needs n_bodies")
    nb = n_bodies if n_bodies is not None else _default_n_bodies(body, n)
    mp = None
    if mu_pair is not None:
        mp = np.ascontiguousarray(np.asarray(mu_pair, np.float64).reshape(nb, nb))
    a = StepArgs(n, int(nb), int(n_iter), _ptr(body), _ptr(x), _ptr(v), _ptr(Cm), _ptr(m), _ptr(nrm), None,
                 None, float(h), float(mu), None if mp is None else mp.ctypes.data, int(flags))
    return a, n, (np.float64 if fp64 else np.float32), (x, v, Cm, m, nrm, body, mp)


class Sim:
    def __init__(self, srv, x, v, Cm, m, nrm, body, h, mu, n_iter, n_bodies=None, mu_pair=None, flags=0):
        lib = load()
        self.srv = srv
        a, self.n, self.dtype, _keep = _sim_args(x, v, Cm, m, nrm, body, h, mu, n_iter, n_bodies, mu_pair, flags)
        hsim = C.c_void_p()
        _check(lib.apic_sim_open(srv.handle, C.byref(a), C.byref(hsim)))
        self._h = hsim

    def wait(self, ticket, timeout_s: float = 60.0):
        """Wait for one of this simulation's requests (on its own server)."""
        return self.srv.wait(ticket, timeout_s)

    @classmethod
    def _adopt(cls, srv, handle, n, dtype):
        self = cls.__new__(cls)
        self.srv, self._h, self.n, self.dtype = srv, handle, n, dtype
        return self

    def export(self) -> bytes:
        """apic_sim_export: a checkpoint of the whole state, as bytes."""
        lib = load()
        size = C.c_size_t()
        _check(lib.apic_sim_export(self._h, None, C.byref(size)))
        buf = C.create_string_buffer(size.value)
        _check(lib.apic_sim_export(self._h, buf, C.byref(size)))
        return buf.raw[: size.value]

    def submit(self, dt_advect: float = 0.0) -> int:
        t = C.c_uint64()
        _check(load().apic_sim_submit(self._h, float(dt_advect), C.byref(t)))
        return t.value

    def read(self):
        x = np.empty((self.n, 3), np.float64)
        v = np.empty((self.n, 3), self.dtype)
        Cm = np.empty((self.n, 3, 3), self.dtype)
        _check(load().apic_sim_read(self._h, x.ctypes.data, v.ctypes.data, Cm.ctypes.data))
        return x, v, Cm

    def close(self):
        if getattr(self, "_h", None):
            load().apic_sim_close(self._h)
            self._h = None


class _Member(Server):
    """A server owned by a Group (not destroyed on its own)."""

    def __init__(self, handle):  # noqa: D401 - no server is created here
        self._h = handle

    def close(self):
        self._h = None


class Group:
    """apic_group: one server per device; simulations are admitted on the
    device with the most HBM budget left (apic_place_by_budget) and stay
    there.  Nothing crosses devices on the data path."""

    def __init__(self, devices, hbm_budget_per_device: int = 0, n_workers: int = 2, max_batch_scenes: int = 64):
        lib = load()
        devs = (C.c_int32 * len(devices))(*[int(d) for d in devices])
        h = C.c_void_p()
        _check(lib.apic_group_create(C.byref(h), devs, len(devices), int(hbm_budget_per_device), int(n_workers),
                                     int(max_batch_scenes)))
        self._h = h
        self.members = []
        for i in range(len(devices)):
            m = C.c_void_p()
            _check(lib.apic_group_server(self._h, i, C.byref(m)))
            self.members.append(_Member(m))

    def open_sim(self, x, v, Cm, m, nrm, body, h, mu, n_iter, n_bodies=None, mu_pair=None, flags=0):
        """Admit a simulation on the member with the most room; the returned
        Sim has .member (its index) and waits on its own server."""
        a, n, dtype, _keep = _sim_args(x, v, Cm, m, nrm, body, h, mu, n_iter, n_bodies, mu_pair, flags)
        hs, k = C.c_void_p(), C.c_int32()
        _check(load().apic_group_open(self._h, C.byref(a), C.byref(hs), C.byref(k)))
        sim = Sim._adopt(self.members[k.value], hs, n, dtype)
        sim.member = k.value
        return sim

    def set_policy(self, variant: int = -1, graphs: bool = True):
        _check(load().apic_group_set_policy(self._h, int(variant), 1 if graphs else 0))

    def stats(self, reset: bool = False) -> dict:
        st = ServerStats()
        _check(load().apic_group_get_stats(self._h, C.byref(st), 1 if reset else 0))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            load().apic_group_destroy(self._h)
            self._h = None
            for m in self.members:
                m.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def place_by_budget(free_bytes, need: int) -> int:
    """apic_place_by_budget (host only): index of the device with the most
    room that still holds `need` bytes, or -1."""
    arr = (C.c_int64 * len(free_bytes))(*[int(b) for b in free_bytes])
    return int(load().apic_place_by_budget(arr, len(free_bytes), int(need)))


def debug_flags(clear: bool = True) -> int:
    """apic_debug_flags: bounds-check bits recorded on the current device
    (always 0 in the normal build)."""
    v = C.c_uint32()
    _check(load().apic_debug_flags(C.byref(v), 1 if clear else 0))
    return int(v.value)
