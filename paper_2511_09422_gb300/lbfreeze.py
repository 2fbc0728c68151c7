"""Thin ctypes binding of the C ABI in ``include/lbfreeze.h`` (``liblbfreeze.so``).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Device memory for inputs and outputs can be torch CUDA tensors
(their data pointers are passed through) and the stream a torch stream.
There is no CPU fallback: ``load()`` raises if the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

LB_OK, LB_ERR_INVALID_ARG, LB_ERR_CUDA, LB_ERR_OOM, LB_ERR_UNSTABLE = 0, 1, 2, 3, 4
LB_STORAGE_F32, LB_STORAGE_F16, LB_STORAGE_F16_H32 = 0, 1, 2  # lb_params.pop_storage
LB_LATTICE_D2Q9, LB_LATTICE_D2Q5 = 0, 1    # lb_params.lattice_fl
FIELD_NAMES = ("phi", "T", "fs", "C", "ux", "uy", "p")
REDUCE_NAMES = ("sum_phi", "sum_rhoH", "sum_C", "sum_fs", "sum_chi", "front", "Vs", "Vsl")


class LbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("lbfreeze status %d: %s" % (status, msg))
        self.status = status


class lb_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("bc_bottom", C.c_int), ("bc_top", C.c_int),
                ("T_bottom", C.c_double), ("T_top", C.c_double), ("T_bottom_amp", C.c_double),
                ("T_bottom_modes", C.c_int), ("cos_theta_bottom", C.c_double), ("cos_theta_top", C.c_double)]


_PARAM_DOUBLES = ("rho_l", "rho_s", "rho_g", "mu_l", "mu_s", "mu_g", "lam_l", "lam_s", "lam_g",
                  "cp_l", "cp_s", "cp_g", "latent", "T_sol", "T_liq", "k_p", "D_l", "D_s", "eps",
                  "mobility", "sigma0", "sigma_T", "sigma_c", "T_ref", "c_ref", "gx", "gy")
_PARAM_INTS = ("fs_modulated_st", "phase_change_on", "divu_mode", "pop_storage", "lattice_fl")


class lb_params(C.Structure):
    _fields_ = [(k, C.c_double) for k in _PARAM_DOUBLES] + [(k, C.c_int) for k in _PARAM_INTS]


_fp = C.POINTER(C.c_float)


class lb_fields(C.Structure):
    _fields_ = [("phi", _fp), ("T", _fp), ("C", _fp), ("ux", _fp), ("uy", _fp), ("on_device", C.c_int)]


_lib = None
_lock = threading.Lock()

EXPORTS = ("lb_create", "lb_set_stream", "lb_step", "lb_get_fields", "lb_set_fields", "lb_reduce", "lb_steps_taken",
           "lb_save", "lb_load", "lb_destroy", "lb_error_string", "lb_last_error", "lb_device_bytes",
           "lb_batch_create", "lb_batch_set_stream", "lb_batch_step", "lb_batch_use_graph", "lb_batch_tune",
           "lb_batch_instance", "lb_batch_size", "lb_batch_last_error", "lb_batch_destroy",
           "lb_slab_create", "lb_slab_halo_bytes", "lb_slab_pack", "lb_slab_unpack")


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load liblbfreeze.so; raises if it has not been built (``__graft_entry__.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("liblbfreeze.so is not built (%s); run __graft_entry__.build()" % path)
        L = C.CDLL(path)
        L.lb_create.restype = C.c_int
        L.lb_create.argtypes = [C.POINTER(lb_grid), C.POINTER(lb_params), C.POINTER(lb_fields), C.POINTER(C.c_void_p)]
        L.lb_set_stream.restype = C.c_int
        L.lb_set_stream.argtypes = [C.c_void_p, C.c_void_p]
        L.lb_step.restype = C.c_int
        L.lb_step.argtypes = [C.c_void_p, C.c_int]
        L.lb_get_fields.restype = C.c_int
        L.lb_get_fields.argtypes = [C.c_void_p] + [C.c_void_p] * 7 + [C.c_int]
        L.lb_set_fields.restype = C.c_int
        L.lb_set_fields.argtypes = [C.c_void_p] + [C.c_void_p] * 7 + [C.c_int]
        L.lb_reduce.restype = C.c_int
        L.lb_reduce.argtypes = [C.c_void_p, C.POINTER(C.c_double)]
        L.lb_steps_taken.restype = C.c_int
        L.lb_steps_taken.argtypes = [C.c_void_p, C.POINTER(C.c_long)]
        L.lb_save.restype = C.c_int
        L.lb_save.argtypes = [C.c_void_p, C.c_char_p]
        L.lb_load.restype = C.c_int
        L.lb_load.argtypes = [C.c_void_p, C.c_char_p]
        L.lb_destroy.restype = None
        L.lb_destroy.argtypes = [C.c_void_p]
        L.lb_error_string.restype = C.c_char_p
        L.lb_error_string.argtypes = [C.c_int]
        L.lb_last_error.restype = C.c_char_p
        L.lb_last_error.argtypes = [C.c_void_p]
        L.lb_device_bytes.restype = C.c_size_t
        L.lb_device_bytes.argtypes = [C.c_void_p]
        L.lb_batch_create.restype = C.c_int
        L.lb_batch_create.argtypes = [C.c_int, C.POINTER(lb_grid), C.POINTER(lb_params), C.POINTER(lb_fields),
                                      C.POINTER(C.c_void_p)]
        L.lb_batch_set_stream.restype = C.c_int
        L.lb_batch_set_stream.argtypes = [C.c_void_p, C.c_void_p]
        L.lb_batch_step.restype = C.c_int
        L.lb_batch_step.argtypes = [C.c_void_p, C.c_int]
        L.lb_batch_use_graph.restype = C.c_int
        L.lb_batch_use_graph.argtypes = [C.c_void_p, C.c_int]
        L.lb_batch_tune.restype = C.c_int
        L.lb_batch_tune.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int)]
        L.lb_batch_instance.restype = C.c_int
        L.lb_batch_instance.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]
        L.lb_batch_size.restype = C.c_int
        L.lb_batch_size.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_longlong)]
        L.lb_batch_last_error.restype = C.c_char_p
        L.lb_batch_last_error.argtypes = [C.c_void_p]
        L.lb_batch_destroy.restype = None
        L.lb_batch_destroy.argtypes = [C.c_void_p]
        L.lb_slab_create.restype = C.c_int
        L.lb_slab_create.argtypes = [C.POINTER(lb_grid), C.POINTER(lb_params), C.POINTER(lb_fields), C.c_int, C.c_int,
                                     C.POINTER(C.c_void_p)]
        L.lb_slab_halo_bytes.restype = C.c_size_t
        L.lb_slab_halo_bytes.argtypes = [C.c_void_p]
        L.lb_slab_pack.restype = C.c_int
        L.lb_slab_pack.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int]
        L.lb_slab_unpack.restype = C.c_int
        L.lb_slab_unpack.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int]
        _lib = L
        return _lib


def make_grid(g: dict) -> lb_grid:
    s = lb_grid()
    for k, _ in lb_grid._fields_:
        setattr(s, k, g.get(k, 0))
    return s


def make_params(p: dict) -> lb_params:
    s = lb_params()
    for k in _PARAM_DOUBLES:
        setattr(s, k, float(p[k]))
    for k in _PARAM_INTS:
        setattr(s, k, int(p.get(k, 0)))
    return s


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _is_cuda_tensor(a) -> bool:
    return _is_torch(a) and bool(a.is_cuda)


def _torch_stream(stream_obj):
    """The torch stream object of a handle's stream: the legacy default stream
    for None, the object itself for a torch stream, else an external stream
    over the raw cudaStream_t."""
    import torch
    if isinstance(stream_obj, torch.cuda.Stream):
        return stream_obj
    ptr = stream_obj if isinstance(stream_obj, int) or stream_obj is None else getattr(stream_obj, "cuda_stream",
                                                                                      stream_obj)
    return torch.cuda.ExternalStream(int(ptr)) if ptr else torch.cuda.default_stream()


def _host_array(v) -> np.ndarray:
    """A float32 numpy view of host data; a torch CPU tensor (pinned or not) is
    viewed in place, so a pinned buffer stays the one the copy reads from."""
    if _is_torch(v):
        v = v.detach().numpy()
    return np.asarray(v, dtype=np.float32)


def slab_extent(ny: int, y0: int, y1: int):
    """Local rows of the slab [y0, y1) of a lattice of ny rows: [y0 - 2, y1 + 2),
    without the two ghost rows at an end that is a wall (y0 = 0 or y1 = ny)."""
    return (y0 - 2 if y0 > 0 else 0), (y1 + 2 if y1 < ny else ny)


class Solver:
    """One lattice on the GPU.

    ``fields`` maps phi, T, C (and optionally ux, uy) to ny x nx arrays: numpy
    arrays or torch CPU tensors (host; pinned tensors copy fastest), or float32
    contiguous torch CUDA tensors (device).  ``stream``
    is a torch.cuda.Stream, a raw cudaStream_t integer, or None (legacy default
    stream)."""

    def __init__(self, grid: dict, params: dict, fields: dict, stream=None, slab=None):
        """``slab=(y0, y1)`` makes this the slab of rows [y0, y1) of the lattice
        ``grid`` (lb_slab_create): ``fields`` then hold the rows [y0 - 2, y1 + 2)
        of the lattice's initial fields, the two extra rows at an end only where
        a neighbouring slab lies (``slab_extent``), and ``ny`` is the local row
        count including those ghost rows."""
        L = load()
        self.nx = int(grid["nx"])
        self.slab = None if slab is None else (int(slab[0]), int(slab[1]))
        if self.slab is None:
            self.ny = int(grid["ny"])
        else:
            lo, hi = slab_extent(int(grid["ny"]), *self.slab)
            self.ny = hi - lo
        n = self.nx * self.ny
        self._grid, self._params = make_grid(grid), make_params(params)
        keep = {}
        on_device = any(_is_cuda_tensor(fields.get(k)) for k in ("phi", "T", "C"))
        for k in ("phi", "T", "C", "ux", "uy"):
            v = fields.get(k)
            if v is None:
                continue
            if on_device:
                if not (_is_torch(v) and v.is_cuda and v.dtype.__str__() == "torch.float32" and v.is_contiguous()):
                    raise ValueError("device fields must be contiguous float32 CUDA tensors (%s)" % k)
                if v.numel() != n:
                    raise ValueError("field %s has %d values, expected %d" % (k, v.numel(), n))
            else:
                v = np.ascontiguousarray(_host_array(v).reshape(-1))
                if v.size != n:
                    raise ValueError("field %s has %d values, expected %d" % (k, v.size, n))
            keep[k] = v
        f = lb_fields()
        for k in ("phi", "T", "C", "ux", "uy"):
            v = keep.get(k)
            if v is None:
                setattr(f, k, None)
            elif on_device:
                setattr(f, k, C.cast(C.c_void_p(v.data_ptr()), _fp))
            else:
                setattr(f, k, v.ctypes.data_as(_fp))
        f.on_device = 1 if on_device else 0
        if on_device:
            import torch
            torch.cuda.current_stream().synchronize()  # the inputs' producers have finished
        h = C.c_void_p()
        if self.slab is None:
            st = L.lb_create(C.byref(self._grid), C.byref(self._params), C.byref(f), C.byref(h))
        else:
            st = L.lb_slab_create(C.byref(self._grid), C.byref(self._params), C.byref(f), self.slab[0], self.slab[1],
                                  C.byref(h))
        if st != LB_OK:
            raise LbError(st, L.lb_last_error(None).decode())
        self._h = h
        self._stream_obj = None
        if stream is not None:
            self.set_stream(stream)

    # -- plumbing ---------------------------------------------------------------------------
    def _check(self, st: int):
        if st != LB_OK:
            raise LbError(st, load().lb_last_error(self._h).decode())

    def set_stream(self, stream):
        ptr = stream if isinstance(stream, int) else getattr(stream, "cuda_stream", stream)
        self._stream_obj = stream
        self._check(load().lb_set_stream(self._h, C.c_void_p(int(ptr) if ptr else 0)))

    @classmethod
    def _view(cls, handle: int, nx: int, ny: int, owner) -> "Solver":
        """A Solver over a handle owned elsewhere (a batch instance); close() leaves it alone."""
        s = cls.__new__(cls)
        s.nx, s.ny = nx, ny
        s._h = C.c_void_p(handle)
        s._stream_obj = getattr(owner, "_stream_obj", None)
        s._owner = owner
        return s

    def close(self):
        if getattr(self, "_owner", None) is not None:
            self._h = C.c_void_p()
            return
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lb_destroy(self._h)
            self._h = C.c_void_p()

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
    def handle(self) -> int:
        return int(self._h.value or 0)

    @property
    def device_bytes(self) -> int:
        return int(load().lb_device_bytes(self._h))

    @property
    def steps(self) -> int:
        v = C.c_long()
        self._check(load().lb_steps_taken(self._h, C.byref(v)))
        return int(v.value)

    # -- the method ---------------------------------------------------------------------------
    def step(self, n: int = 1):
        self._check(load().lb_step(self._h, int(n)))

    # -- slabs of a larger lattice ------------------------------------------------------------
    @property
    def halo_bytes(self) -> int:
        """Bytes of one face's halo message (0 for a whole lattice)."""
        return int(load().lb_slab_halo_bytes(self._h))

    def pack_halo(self, face: int, dst):
        """The two owned rows next to face 0 (low y) or 1 (high y), every
        population and lagged plane, into ``dst``: a uint8 numpy array / torch
        CPU tensor (synchronises) or a uint8 CUDA tensor (on the handle's
        stream, ordered with torch's current stream) of halo_bytes bytes."""
        self._halo_call(load().lb_slab_pack, face, dst)

    def unpack_halo(self, face: int, src):
        """A neighbour's message (see pack_halo) into the ghost rows at ``face``."""
        self._halo_call(load().lb_slab_unpack, face, src)

    def _halo_call(self, fn, face, buf):
        if _is_cuda_tensor(buf):
            import torch
            if buf.numel() * buf.element_size() != self.halo_bytes or not buf.is_contiguous():
                raise ValueError("halo buffer must be contiguous with halo_bytes bytes")
            hs, cur = _torch_stream(self._stream_obj), torch.cuda.current_stream()
            hs.wait_stream(cur)
            self._check(fn(self._h, int(face), C.c_void_p(buf.data_ptr()), 1))
            cur.wait_stream(hs)
            return
        h = buf.detach().numpy() if _is_torch(buf) else buf
        if not (isinstance(h, np.ndarray) and h.flags["C_CONTIGUOUS"] and h.nbytes == self.halo_bytes):
            raise ValueError("halo buffer must be contiguous with halo_bytes bytes")
        self._check(fn(self._h, int(face), C.c_void_p(h.ctypes.data), 0))

    def fields(self, device: bool = False, names=FIELD_NAMES, out=None):
        """Macroscopic fields of the current state as (ny, nx) arrays: numpy on
        the host, or torch CUDA tensors with ``device=True``.  ``out`` supplies
        the destinations instead (a dict of contiguous float32 arrays of nx*ny
        values: all numpy / torch CPU tensors, e.g. pinned, or all CUDA tensors)."""
        if out is not None:
            dev = [_is_cuda_tensor(v) for v in out.values()]
            if dev and any(dev) != all(dev):
                raise ValueError("fields(out=...) mixes host and device destinations")
            device = bool(dev) and all(dev)
            ptrs = []
            for k in FIELD_NAMES:
                v = out.get(k)
                if v is None:
                    ptrs.append(None)
                    continue
                if device:
                    ok = v.dtype.__str__() == "torch.float32" and v.is_contiguous() and v.numel() == self.nx * self.ny
                    ptr = v.data_ptr()
                else:
                    h = v.detach().numpy() if _is_torch(v) else v  # a view: the call writes into v
                    ok = (isinstance(h, np.ndarray) and h.dtype == np.float32 and h.flags["C_CONTIGUOUS"]
                          and h.size == self.nx * self.ny)
                    ptr = h.ctypes.data
                if not ok:
                    raise ValueError("fields(out=...): %s must be contiguous float32 with nx*ny values" % k)
                ptrs.append(C.c_void_p(ptr))
            self._get_fields(ptrs, device)
            return out
        if device:
            import torch
            out = {k: torch.empty((self.ny, self.nx), dtype=torch.float32, device="cuda") for k in names}
            ptrs = [C.c_void_p(out[k].data_ptr()) if k in out else None for k in FIELD_NAMES]
        else:
            out = {k: np.empty((self.ny, self.nx), dtype=np.float32) for k in names}
            ptrs = [C.c_void_p(out[k].ctypes.data) if k in out else None for k in FIELD_NAMES]
        self._get_fields(ptrs, device)
        return out

    def _get_fields(self, ptrs, device: bool):
        """lb_get_fields into device or host pointers.  Device outputs are
        written on the handle's stream and read by torch on its current stream,
        so the current stream waits for the handle's before and after: the
        outputs' earlier users have finished, and later ones see the values."""
        if not device:
            self._check(load().lb_get_fields(self._h, *ptrs, 0))
            return
        import torch
        hs, cur = _torch_stream(self._stream_obj), torch.cuda.current_stream()
        hs.wait_stream(cur)
        self._check(load().lb_get_fields(self._h, *ptrs, 1))
        cur.wait_stream(hs)

    def set_fields(self, fields: dict):
        """Replace the state by the equilibrium of the given fields (keys of
        FIELD_NAMES; phi, T, C required): all numpy float32 (ny, nx) arrays, or
        all contiguous float32 CUDA tensors."""
        order = ("phi", "T", "fs", "C", "ux", "uy", "p")
        vals = [fields.get(k) for k in order]
        dev = [_is_cuda_tensor(v) for v in vals if v is not None]
        if dev and any(dev) != all(dev):
            raise ValueError("set_fields mixes host and device inputs")
        device = bool(dev) and all(dev)
        keep, ptrs = [], []
        for k, v in zip(order, vals):
            if v is None:
                ptrs.append(None)
                continue
            if device:
                if not (str(v.dtype) == "torch.float32" and v.is_contiguous() and v.numel() == self.nx * self.ny):
                    raise ValueError("set_fields: %s must be contiguous float32 with nx*ny values" % k)
                ptrs.append(C.c_void_p(v.data_ptr()))
            else:
                a = np.ascontiguousarray(v, dtype=np.float32)
                if a.size != self.nx * self.ny:
                    raise ValueError("set_fields: %s must have nx*ny values" % k)
                keep.append(a)
                ptrs.append(C.c_void_p(a.ctypes.data))
        if not device:
            self._check(load().lb_set_fields(self._h, *ptrs, 0))
            return
        # device inputs: the handle's stream reads them after torch's producers,
        # and torch's later writers wait for that read
        import torch
        hs, cur = _torch_stream(self._stream_obj), torch.cuda.current_stream()
        hs.wait_stream(cur)
        self._check(load().lb_set_fields(self._h, *ptrs, 1))
        cur.wait_stream(hs)

    def reduce(self) -> np.ndarray:
        out = (C.c_double * 8)()
        self._check(load().lb_reduce(self._h, out))
        return np.array(out[:], dtype=np.float64)

    def save(self, path: str):
        self._check(load().lb_save(self._h, path.encode()))

    def load_state(self, path: str):
        self._check(load().lb_load(self._h, path.encode()))


def from_workload(w: dict, stream=None) -> Solver:
    return Solver(w["grid"], w["params"], w["fields"], stream=stream)


class Batch:
    """Independent lattices advanced together by one persistent launch per step.

    ``workloads`` is a list of dicts with ``grid``, ``params`` and ``fields``
    (host arrays, as for Solver).  ``instance(i)`` gives a Solver view of
    instance i for fields / reduce / save; the batch owns it."""

    def __init__(self, workloads, stream=None):
        L = load()
        n = len(workloads)
        if n < 1:
            raise ValueError("a batch needs at least one instance")
        grids = (lb_grid * n)()
        params = (lb_params * n)()
        fields = (lb_fields * n)()
        self._keep = []
        self.shapes = []
        for i, w in enumerate(workloads):
            g = w["grid"]
            nx, ny = int(g["nx"]), int(g["ny"])
            grids[i] = make_grid(g)
            params[i] = make_params(w["params"])
            f = lb_fields()
            for k in ("phi", "T", "C", "ux", "uy"):
                v = w["fields"].get(k)
                if v is None:
                    setattr(f, k, None)
                    continue
                v = np.ascontiguousarray(_host_array(v).reshape(-1))
                if v.size != nx * ny:
                    raise ValueError("instance %d: field %s has %d values, expected %d" % (i, k, v.size, nx * ny))
                self._keep.append(v)
                setattr(f, k, v.ctypes.data_as(_fp))
            f.on_device = 0
            fields[i] = f
            self.shapes.append((nx, ny))
        h = C.c_void_p()
        st = L.lb_batch_create(n, grids, params, fields, C.byref(h))
        if st != LB_OK:
            raise LbError(st, L.lb_batch_last_error(None).decode())
        self._keep = []
        self._h = h
        self.n = n
        self._stream_obj = None
        if stream is not None:
            self.set_stream(stream)

    def _check(self, st: int):
        if st != LB_OK:
            raise LbError(st, load().lb_batch_last_error(self._h).decode())

    def set_stream(self, stream):
        ptr = stream if isinstance(stream, int) else getattr(stream, "cuda_stream", stream)
        self._stream_obj = stream
        self._check(load().lb_batch_set_stream(self._h, C.c_void_p(int(ptr) if ptr else 0)))

    def step(self, n: int = 1):
        self._check(load().lb_batch_step(self._h, int(n)))

    def use_graph(self, on: bool):
        self._check(load().lb_batch_use_graph(self._h, 1 if on else 0))

    def tune(self, trials: int = 5):
        """Autotune the inner segment height per size class; returns the choices."""
        out = (C.c_int * 3)()
        self._check(load().lb_batch_tune(self._h, int(trials), out))
        return list(out)

    def instance(self, i: int) -> Solver:
        h = C.c_void_p()
        self._check(load().lb_batch_instance(self._h, int(i), C.byref(h)))
        nx, ny = self.shapes[i]
        return Solver._view(h.value, nx, ny, self)

    @property
    def cells(self) -> int:
        c = C.c_longlong()
        self._check(load().lb_batch_size(self._h, None, C.byref(c)))
        return int(c.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lb_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
