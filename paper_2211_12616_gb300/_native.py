"""ctypes binding of libmptrac (include/mptrac.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module only turns
torch tensors into device pointers and status codes into exceptions.  If the
shared library is missing the import fails loudly -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmptrac.so")

MPTRAC_FP32, MPTRAC_BF16, MPTRAC_FP16 = 0, 1, 2
MAX_NZ = 256                      # MPTRAC_MAX_NZ: largest supported number of pressure levels
STATUS = {0: "OK", -1: "E_INVALID_ARG", -2: "E_OOM", -3: "E_CUDA", -4: "E_TIME_RANGE",
          -5: "E_WORKSPACE", -6: "E_TIMEOUT", -7: "E_NOT_INIT"}


class MptracError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("lon0", C.c_double), ("dlon", C.c_double), ("lat0", C.c_double), ("dlat", C.c_double),
                ("plev", C.POINTER(C.c_double)), ("storage", C.c_int), ("nvars", C.c_int)]


class ParticlesDesc(C.Structure):
    _fields_ = [("n", C.c_int64), ("lon", C.c_void_p), ("lat", C.c_void_p), ("p", C.c_void_p),
                ("id", C.c_void_p), ("release", C.c_void_p), ("up", C.c_void_p), ("vp", C.c_void_p),
                ("wp", C.c_void_p)]


class DiffParamsDesc(C.Structure):
    _fields_ = [("dx", C.c_double), ("dz", C.c_double), ("meso_f", C.c_double),
                ("scale_height", C.c_double), ("turb", C.c_int), ("meso", C.c_int)]


# exported symbol -> (restype, argtypes)
SIGNATURES = {
    "mptrac_init_grid": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(GridDesc)]),
    "mptrac_destroy": (C.c_int, [C.c_void_p]),
    "mptrac_last_error": (C.c_char_p, [C.c_void_p]),
    "mptrac_load_met": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_int, C.c_void_p]),
    "mptrac_set_releases": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "mptrac_advect": (C.c_int, [C.c_void_p, C.POINTER(ParticlesDesc), C.c_double, C.c_double, C.c_int,
                                C.c_void_p]),
    "mptrac_diffuse": (C.c_int, [C.c_void_p, C.POINTER(ParticlesDesc), C.c_double, C.c_double,
                                 C.POINTER(DiffParamsDesc), C.c_uint64, C.c_uint64, C.c_int, C.c_void_p]),
    "mptrac_step": (C.c_int, [C.c_void_p, C.POINTER(ParticlesDesc), C.c_double, C.c_double,
                              C.POINTER(DiffParamsDesc), C.c_uint64, C.c_uint64, C.c_int, C.c_void_p]),
    "mptrac_step_sort": (C.c_int, [C.c_void_p, C.POINTER(ParticlesDesc), C.c_double, C.c_double,
                                   C.POINTER(DiffParamsDesc), C.c_uint64, C.c_uint64, C.c_int, C.c_void_p,
                                   C.c_size_t, C.c_void_p]),
    "mptrac_step_handoff": (C.c_int, [C.c_void_p, C.POINTER(ParticlesDesc), C.c_double, C.c_double,
                                      C.POINTER(DiffParamsDesc), C.c_uint64, C.c_uint64, C.c_int, C.c_void_p,
                                      C.c_size_t, C.c_void_p]),
    "mptrac_sort_handoff": (C.c_int, [C.c_void_p, C.POINTER(ParticlesDesc), C.c_void_p, C.c_size_t, C.c_void_p]),
    "mptrac_sort_workspace_bytes": (C.c_size_t, [C.c_void_p, C.c_int64]),
    "mptrac_sort": (C.c_int, [C.c_void_p, C.POINTER(ParticlesDesc), C.c_void_p, C.c_size_t, C.c_void_p]),
    "mptrac_cell_keys": (C.c_int, [C.c_void_p, C.POINTER(ParticlesDesc), C.c_void_p, C.c_void_p]),
    "mptrac_interp": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mptrac_philox": (C.c_int, [C.c_void_p, C.c_int64, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mptrac_met_slot_info": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                       C.POINTER(C.c_double), C.POINTER(C.c_size_t)]),
    "mptrac_met_slot_copy": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mptrac_kernel_launches": (C.c_uint64, []),
    "mptrac_copy_probe": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int, C.c_void_p]),
    "mptrac_sort_noalloc": (C.c_int, [C.c_void_p, C.POINTER(ParticlesDesc), C.c_void_p]),
    "mptrac_sort_at": (C.c_int, [C.c_void_p, C.POINTER(ParticlesDesc), C.c_double, C.c_void_p, C.c_size_t,
                                 C.c_void_p]),
    "mptrac_set_launch": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "mptrac_sample_met": (C.c_int, [C.c_void_p, C.POINTER(ParticlesDesc), C.c_double, C.c_void_p, C.c_void_p]),
    "mptrac_sediment": (C.c_int, [C.c_void_p, C.POINTER(ParticlesDesc), C.c_void_p, C.c_void_p, C.c_double,
                                  C.c_double, C.c_int, C.c_void_p]),
    "mptrac_grid_counts": (C.c_int, [C.c_void_p, C.POINTER(ParticlesDesc), C.c_void_p, C.c_void_p]),
    "mptrac_advect_masked": (C.c_int, [C.c_void_p, C.POINTER(ParticlesDesc), C.c_void_p, C.c_double, C.c_double,
                                       C.c_int, C.c_void_p]),
    "mptrac_surr_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int64]),
    "mptrac_surr_destroy": (C.c_int, [C.c_void_p]),
    "mptrac_surr_set_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mptrac_surr_get_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mptrac_surr_get_grads": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mptrac_surr_set_norm": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mptrac_surr_features": (C.c_int, [C.c_void_p, C.POINTER(ParticlesDesc), C.c_double, C.c_void_p, C.c_void_p]),
    "mptrac_surr_targets": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p]),
    "mptrac_surr_colstats": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_double,
                                       C.c_void_p]),
    "mptrac_surr_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "mptrac_surr_grads": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "mptrac_surr_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_float, C.c_int,
                                         C.c_void_p, C.c_void_p]),
    "mptrac_surr_train_epoch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_double,
                                          C.c_double, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "mptrac_surr_advance": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(ParticlesDesc), C.c_double, C.c_double,
                                      C.c_void_p, C.c_void_p, C.c_void_p]),
    "mptrac_surr_set_kernel": (C.c_int, [C.c_void_p, C.c_int]),
    "mptrac_surr_status": (C.c_int, [C.c_void_p, C.c_void_p]),
}

_lib = None


def load() -> C.CDLL:
    """Loads libmptrac.so (built by ``__graft_entry__.build()``); raises if it is absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libmptrac.so not found at {LIB_PATH}: build it first "
                              "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype, fn.argtypes = res, args
        _lib = lib
    return _lib


def check(code: int, ctx=None):
    if code != 0:
        msg = load().mptrac_last_error(ctx)
        raise MptracError(code, msg.decode() if msg else "")


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensors passed to libmptrac must be contiguous")
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to libmptrac must be C-contiguous")
        return t.ctypes.data
    raise TypeError(f"unsupported buffer type {type(t)}")


class DiffParams:
    def __init__(self, dx=50.0, dz=0.1, meso_f=0.16, scale_height=7000.0, turb=True, meso=True):
        self.dx, self.dz, self.meso_f, self.scale_height = dx, dz, meso_f, scale_height
        self.turb, self.meso = bool(turb), bool(meso)

    def desc(self) -> DiffParamsDesc:
        return DiffParamsDesc(self.dx, self.dz, self.meso_f, self.scale_height, int(self.turb), int(self.meso))


class Particles:
    """Device structure-of-arrays particle state (torch tensors own the memory).

    lon/lat/p float64, id/release int32 tensors holding uint32 bit patterns,
    up/vp/wp float32 mesoscale perturbations.
    """
    FIELDS = ("lon", "lat", "p", "id", "release", "up", "vp", "wp")

    def __init__(self, lon, lat, p, id, release=None, up=None, vp=None, wp=None):
        self.lon, self.lat, self.p, self.id = lon, lat, p, id
        self.release, self.up, self.vp, self.wp = release, up, vp, wp

    @classmethod
    def from_numpy(cls, d: dict, device="cuda", meso=True, release=True):
        n = len(d["lon"])
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(device=device, dtype=dt)
        u32 = lambda a: torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.uint32)).view(np.int32)).to(device)
        up = vp = wp = None
        if meso:
            up = t(d.get("up", np.zeros(n)), torch.float32)
            vp = t(d.get("vp", np.zeros(n)), torch.float32)
            wp = t(d.get("wp", np.zeros(n)), torch.float32)
        rel = u32(d.get("release", np.zeros(n, np.uint32))) if release else None
        return cls(t(d["lon"], torch.float64), t(d["lat"], torch.float64), t(d["p"], torch.float64),
                   u32(d["id"]), rel, up, vp, wp)

    def to_numpy(self) -> dict:
        out = {}
        for k in self.FIELDS:
            v = getattr(self, k)
            if v is None:
                continue
            a = v.detach().cpu().numpy()
            out[k] = a.view(np.uint32) if k in ("id", "release") else a
        return out

    def clone(self) -> "Particles":
        return Particles(*[None if getattr(self, k) is None else getattr(self, k).clone() for k in self.FIELDS])

    def view(self, a: int, b: int) -> "Particles":
        """Particles [a, b) as views of the same device memory."""
        return Particles(*[None if getattr(self, k) is None else getattr(self, k)[a:b] for k in self.FIELDS])

    def copy_(self, other: "Particles"):
        for k in self.FIELDS:
            a, b = getattr(self, k), getattr(other, k)
            if a is not None and b is not None:
                a.copy_(b, non_blocking=True)
        return self

    @property
    def n(self) -> int:
        return int(self.lon.numel())

    def desc(self) -> ParticlesDesc:
        return ParticlesDesc(self.n, *[_ptr(getattr(self, k)) for k in self.FIELDS[:]])


class Context:
    """One grid + three met slots (``mptrac_init_grid``)."""

    def __init__(self, grid, storage: int = MPTRAC_FP32, nvars: int = 3):
        lib = load()
        self.grid = grid
        self.storage, self.nvars = storage, nvars
        self._plev = np.ascontiguousarray(grid.plev, dtype=np.float64)
        gd = GridDesc(grid.nx, grid.ny, grid.nz, grid.lon0, grid.dlon, grid.lat0, grid.dlat,
                      self._plev.ctypes.data_as(C.POINTER(C.c_double)), storage, nvars)
        h = C.c_void_p()
        check(lib.mptrac_init_grid(C.byref(h), C.byref(gd)))
        self.h = h
        self._keep = []

    def close(self):
        if getattr(self, "h", None):
            check(load().mptrac_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_met(self, slot, t, u, v, w, T=None, stream=None):
        on_dev = isinstance(u, torch.Tensor) and u.is_cuda
        if not on_dev:
            u, v, w = (np.ascontiguousarray(a, dtype=np.float32) for a in (u, v, w))
            T = None if T is None else np.ascontiguousarray(T, dtype=np.float32)
            self._keep = [u, v, w, T]     # host copies stay alive until the next call
        check(load().mptrac_load_met(self.h, slot, float(t), _ptr(u), _ptr(v), _ptr(w), _ptr(T),
                                     int(on_dev), _stream(stream)), self.h)

    def set_releases(self, t_start, t_end):
        ts = np.ascontiguousarray(t_start, dtype=np.float64)
        te = np.ascontiguousarray(t_end, dtype=np.float64)
        check(load().mptrac_set_releases(self.h, ts.size, ts.ctypes.data, te.ctypes.data), self.h)

    def advect(self, parts: Particles, t, dt, nsteps, stream=None):
        check(load().mptrac_advect(self.h, C.byref(parts.desc()), float(t), float(dt), int(nsteps),
                                   _stream(stream)), self.h)

    def diffuse(self, parts: Particles, t, dt, prm: DiffParams, seed, step0, nsteps, stream=None):
        check(load().mptrac_diffuse(self.h, C.byref(parts.desc()), float(t), float(dt), C.byref(prm.desc()),
                                    int(seed), int(step0), int(nsteps), _stream(stream)), self.h)

    def step(self, parts: Particles, t, dt, prm: DiffParams, seed, step0, nsteps, stream=None):
        check(load().mptrac_step(self.h, C.byref(parts.desc()), float(t), float(dt), C.byref(prm.desc()),
                                 int(seed), int(step0), int(nsteps), _stream(stream)), self.h)

    def step_sort(self, parts: Particles, t, dt, prm: DiffParams, seed, step0, nsteps,
                  workspace: torch.Tensor | None = None, stream=None):
        """``step`` then ``sort`` in one call (the step hands its results to the sort)."""
        if workspace is None:
            workspace = torch.empty(self.sort_workspace_bytes(parts.n), dtype=torch.uint8, device=parts.lon.device)
        check(load().mptrac_step_sort(self.h, C.byref(parts.desc()), float(t), float(dt), C.byref(prm.desc()),
                                      int(seed), int(step0), int(nsteps), _ptr(workspace), workspace.numel(),
                                      _stream(stream)), self.h)
        return workspace

    def step_handoff(self, parts: Particles, t, dt, prm: DiffParams, seed, step0, nsteps, workspace: torch.Tensor,
                     stream=None):
        """First half of ``step_sort``: the result stays in ``workspace`` until ``sort_handoff``."""
        check(load().mptrac_step_handoff(self.h, C.byref(parts.desc()), float(t), float(dt), C.byref(prm.desc()),
                                         int(seed), int(step0), int(nsteps), _ptr(workspace), workspace.numel(),
                                         _stream(stream)), self.h)

    def sort_handoff(self, parts: Particles, workspace: torch.Tensor, stream=None):
        """Second half of ``step_sort``."""
        check(load().mptrac_sort_handoff(self.h, C.byref(parts.desc()), _ptr(workspace), workspace.numel(),
                                         _stream(stream)), self.h)

    def sort_workspace_bytes(self, n: int) -> int:
        return int(load().mptrac_sort_workspace_bytes(self.h, int(n)))

    def sort(self, parts: Particles, workspace: torch.Tensor | None = None, stream=None):
        nbytes = self.sort_workspace_bytes(parts.n)
        if workspace is None:
            workspace = torch.empty(nbytes, dtype=torch.uint8, device=parts.lon.device)
        check(load().mptrac_sort(self.h, C.byref(parts.desc()), _ptr(workspace), workspace.numel(),
                                 _stream(stream)), self.h)
        return workspace

    def sort_at(self, parts: Particles, t, workspace: torch.Tensor | None = None, stream=None):
        nbytes = self.sort_workspace_bytes(parts.n)
        if workspace is None:
            workspace = torch.empty(nbytes, dtype=torch.uint8, device=parts.lon.device)
        check(load().mptrac_sort_at(self.h, C.byref(parts.desc()), float(t), _ptr(workspace), workspace.numel(),
                                    _stream(stream)), self.h)
        return workspace

    def sample_met(self, parts: Particles, t, stream=None) -> torch.Tensor:
        out = torch.empty(4, parts.n, dtype=torch.float32, device=parts.lon.device)
        check(load().mptrac_sample_met(self.h, C.byref(parts.desc()), float(t), _ptr(out), _stream(stream)), self.h)
        return out

    def sediment(self, parts: Particles, radius: torch.Tensor, density: torch.Tensor, t, dt, nsteps, stream=None):
        check(load().mptrac_sediment(self.h, C.byref(parts.desc()), _ptr(radius), _ptr(density), float(t), float(dt),
                                     int(nsteps), _stream(stream)), self.h)

    def grid_counts(self, parts: Particles, stream=None) -> torch.Tensor:
        g = self.grid
        out = torch.empty(g.nx * g.ny * g.nz, dtype=torch.int32, device=parts.lon.device)
        check(load().mptrac_grid_counts(self.h, C.byref(parts.desc()), _ptr(out), _stream(stream)), self.h)
        return out

    def set_launch(self, variant: int = 0, persistent: bool = False, per_thread: int = 1):
        """Launch variant and schedule of the fused step (``mptrac_set_launch``): one wave of
        persistent blocks, else ``per_thread`` particles per thread."""
        if persistent and per_thread != 1:
            raise ValueError("a persistent launch takes no particles-per-thread count")
        schedule = 1 if persistent else (int(per_thread) if per_thread > 1 else 0)
        check(load().mptrac_set_launch(self.h, int(variant), schedule), self.h)

    def cell_keys(self, parts: Particles, stream=None) -> torch.Tensor:
        keys = torch.empty(parts.n, dtype=torch.int32, device=parts.lon.device)
        check(load().mptrac_cell_keys(self.h, C.byref(parts.desc()), _ptr(keys), _stream(stream)), self.h)
        return keys

    def interp(self, lon, lat, p, t, stream=None):
        n = lon.numel()
        dev = lon.device
        u, v, w = (torch.empty(n, dtype=torch.float32, device=dev) for _ in range(3))
        var = torch.empty(3, n, dtype=torch.float32, device=dev)
        check(load().mptrac_interp(self.h, n, _ptr(lon), _ptr(lat), _ptr(p), float(t), _ptr(u), _ptr(v),
                                   _ptr(w), _ptr(var), _stream(stream)), self.h)
        return u, v, w, var

    def slot_info(self, slot):
        rec, sc, t, nb = C.c_void_p(), C.c_void_p(), C.c_double(), C.c_size_t()
        check(load().mptrac_met_slot_info(self.h, slot, C.byref(rec), C.byref(sc), C.byref(t), C.byref(nb)),
              self.h)
        return rec.value, sc.value, t.value, nb.value

    def slot_arrays(self, slot, stream=None):
        """Copies of slot `slot`'s records ([ny][nx][nz][4]) and scales ([4][nz]) as numpy arrays."""
        _, _, t, nb = self.slot_info(slot)
        g = self.grid
        rec = torch.empty(nb, dtype=torch.uint8, device="cuda")
        sc = torch.empty(4 * g.nz, dtype=torch.float32, device="cuda")
        check(load().mptrac_met_slot_copy(self.h, slot, _ptr(rec), _ptr(sc), _stream(stream)), self.h)
        torch.cuda.synchronize()
        dt = np.float32 if self.storage == MPTRAC_FP32 else np.uint16
        return rec.cpu().numpy().view(dt).reshape(g.ny, g.nx, g.nz, 4), sc.cpu().numpy().reshape(4, g.nz), t


def philox(ctr: torch.Tensor, seed: int, with_normals: bool = False, stream=None):
    """Raw Philox4x32-10 words for counters ``ctr`` (int32 tensor [4][n] of uint32 bits)."""
    n = ctr.shape[1]
    out = torch.empty(4, n, dtype=torch.int32, device=ctr.device)
    z = torch.empty(4, n, dtype=torch.float32, device=ctr.device) if with_normals else None
    check(load().mptrac_philox(_ptr(ctr), n, int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(out), _ptr(z), _stream(stream)))
    return (out, z) if with_normals else out


def copy_probe(src: torch.Tensor, dst: torch.Tensor, reps: int, stream=None):
    """``mptrac_copy_probe``: one launch copying src into dst ``reps`` times through L2."""
    nbytes = src.numel() * src.element_size()
    assert dst.numel() * dst.element_size() >= nbytes
    check(load().mptrac_copy_probe(_ptr(src), _ptr(dst), nbytes, int(reps), _stream(stream)))


# ---------------------------------------------------------------------------
# learned surrogate
# ---------------------------------------------------------------------------
SURR_NFEAT, SURR_KPAD, SURR_HIDDEN, SURR_NOUT, SURR_NPARAM = 168, 176, 128, 3, 39555
SURR_KERNEL_TCGEN05, SURR_KERNEL_MMA_SYNC, SURR_KERNEL_WAIT_TEST = 0, 1, 2


class Surrogate:
    """Handle of ``mptrac_surr``: parameters, Adam state and activation buffers on the device."""

    def __init__(self, max_batch: int = 65536):
        h = C.c_void_p()
        check(load().mptrac_surr_create(C.byref(h), int(max_batch)))
        self.h, self.max_batch = h, int(max_batch)
        self._loss = torch.zeros(1, dtype=torch.float32, device="cuda")

    def close(self):
        if getattr(self, "h", None):
            check(load().mptrac_surr_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == SURR_NPARAM
        check(load().mptrac_surr_set_params(self.h, a.ctypes.data))

    def get_params(self) -> np.ndarray:
        a = np.empty(SURR_NPARAM, dtype=np.float32)
        check(load().mptrac_surr_get_params(self.h, a.ctypes.data))
        return a

    def get_grads(self) -> np.ndarray:
        a = np.empty(SURR_NPARAM, dtype=np.float32)
        check(load().mptrac_surr_get_grads(self.h, a.ctypes.data))
        return a

    def set_norm(self, mu_x, sd_x, mu_y, sd_y):
        arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float32)) for a in (mu_x, sd_x, mu_y, sd_y)]
        check(load().mptrac_surr_set_norm(self.h, *[a.ctypes.data for a in arrs]))

    def forward(self, x: torch.Tensor, stream=None) -> torch.Tensor:
        n = x.shape[0]
        y = torch.empty(n, 8, dtype=torch.float32, device=x.device)
        check(load().mptrac_surr_forward(self.h, _ptr(x), n, _ptr(y), _stream(stream)))
        return y

    def grads(self, x: torch.Tensor, y: torch.Tensor, stream=None) -> torch.Tensor:
        self._loss.zero_()
        check(load().mptrac_surr_grads(self.h, _ptr(x), _ptr(y), x.shape[0], _ptr(self._loss), _stream(stream)))
        return self._loss

    def train_step(self, x: torch.Tensor, y: torch.Tensor, lr: float, step: int, loss: torch.Tensor,
                   stream=None):
        """One Adam step; the batch loss is added to the 1-element device tensor ``loss``."""
        check(load().mptrac_surr_train_step(self.h, _ptr(x), _ptr(y), x.shape[0], float(lr), int(step),
                                            _ptr(loss), _stream(stream)))

    def train_epoch(self, x: torch.Tensor, y: torch.Tensor, batch: int, lr_max: float, lr_min: float,
                    step0: int, total_steps: int, loss: torch.Tensor, stream=None):
        """Adam steps step0 + 1 ... on the consecutive mini-batches of (x, y) under the cosine
        learning-rate decay, in one library call (``mptrac_surr_train_epoch``)."""
        check(load().mptrac_surr_train_epoch(self.h, _ptr(x), _ptr(y), x.shape[0], int(batch), float(lr_max),
                                             float(lr_min), int(step0), int(total_steps), _ptr(loss),
                                             _stream(stream)))

    def advance(self, ctx: "Context", parts: "Particles", t, dt_seg, fallback: torch.Tensor,
                count: torch.Tensor | None = None, stream=None):
        """One surrogate segment; ``count`` (int64 device tensor, optional) accumulates the fallback particles."""
        check(load().mptrac_surr_advance(ctx.h, self.h, C.byref(parts.desc()), float(t), float(dt_seg),
                                         _ptr(fallback), _ptr(count), _stream(stream)), ctx.h)

    def set_kernel(self, kernel: int):
        """SURR_KERNEL_TCGEN05 (default) or SURR_KERNEL_MMA_SYNC for the fused inference."""
        check(load().mptrac_surr_set_kernel(self.h, int(kernel)))

    def status(self, stream=None):
        """Synchronises the stream; raises MptracError (E_TIMEOUT) if a fused inference gave up a wait."""
        check(load().mptrac_surr_status(self.h, _stream(stream)))


def surr_features(ctx: "Context", parts: "Particles", t, out: torch.Tensor | None = None, stream=None):
    if out is None:
        out = torch.empty(parts.n, SURR_KPAD, dtype=torch.float32, device=parts.lon.device)
    check(load().mptrac_surr_features(ctx.h, C.byref(parts.desc()), float(t), _ptr(out), _stream(stream)), ctx.h)
    return out


def surr_targets(p0: "Particles", p1: "Particles", out: torch.Tensor | None = None, stream=None):
    n = p0.n
    if out is None:
        out = torch.empty(n, SURR_NOUT, dtype=torch.float32, device=p0.lon.device)
    check(load().mptrac_surr_targets(n, _ptr(p0.lon), _ptr(p0.lat), _ptr(p0.p), _ptr(p1.lon), _ptr(p1.lat),
                                     _ptr(p1.p), _ptr(out), _stream(stream)))
    return out


def colstats(data: torch.Tensor, sd_min: float = 1e-12, stream=None):
    """Column mean and standard deviation of a [n][ncol] float32 device tensor (synchronises);
    a standard deviation not above sd_min comes back as 1 (``mptrac_surr_colstats``)."""
    n, ncol = data.shape
    mean = torch.empty(ncol, dtype=torch.float64, device=data.device)
    sd = torch.empty(ncol, dtype=torch.float64, device=data.device)
    check(load().mptrac_surr_colstats(_ptr(data), n, ncol, _ptr(mean), _ptr(sd), float(sd_min), _stream(stream)))
    return mean.cpu().numpy(), sd.cpu().numpy()


def advect_masked(ctx: "Context", parts: "Particles", mask: torch.Tensor, t, dt, nsteps, stream=None):
    check(load().mptrac_advect_masked(ctx.h, C.byref(parts.desc()), _ptr(mask), float(t), float(dt), int(nsteps),
                                      _stream(stream)), ctx.h)
