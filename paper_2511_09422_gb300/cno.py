"""Thin ctypes binding of the C ABI in ``include/cno.h`` (``libcno.so``): the
convolutional neural operator used as the learned surrogate of the LB step.

Argument marshalling only: the convolutions, the training step, the optimiser
and the coupling with the LB fields all run in the library's CUDA kernels.
Device memory is passed as torch CUDA tensors (their data pointers), the
stream is the current torch stream.  There is no CPU fallback: ``load()``
raises if the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

CNO_OK = 0
WIDTHS = (64, 128, 256, 256)  # channels of the four levels
CIN = 64                      # input channels (the fields, zero-padded to one 128-byte row)
COUT = 64                     # head channels (the first NF are used)
NF = 7                        # phi, T, f_s, C, u_x, u_y, p

_lib = None
_lock = threading.Lock()

EXPORTS = ("cno_error_string", "cno_read_status", "cno_wait_selftest", "cno_conv3x3_forward", "cno_conv3x3_dgrad", "cno_conv3x3_wgrad",
           "cno_weights_to_bf16", "cno_create", "cno_destroy", "cno_set_stream", "cno_num_params",
           "cno_set_params", "cno_get_params", "cno_get_grads", "cno_forward", "cno_train_step",
           "cno_last_output", "cno_pack_fields", "cno_pack_delta", "cno_apply_update", "cno_field_checks")


class CnoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("cno status %d: %s" % (status, msg))
        self.status = status


def library_path() -> str:
    return _build.CNO_LIB


def load(path: str | None = None):
    """Load libcno.so; raises if it has not been built (``__graft_entry__.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or _build.CNO_LIB
        if not os.path.exists(path):
            raise RuntimeError("libcno.so is not built (%s); run __graft_entry__.build()" % path)
        L = C.CDLL(path)
        vp, i, f, d = C.c_void_p, C.c_int, C.c_float, C.c_double
        sig = {
            "cno_error_string": (C.c_char_p, []),
            "cno_read_status": (i, [C.POINTER(C.c_uint), i]),
            "cno_wait_selftest": (i, [d, C.POINTER(C.c_int), C.POINTER(d)]),
            "cno_conv3x3_forward": (i, [vp, i, i, i, i, vp, vp, i, i, vp, i, i, i, vp]),
            "cno_conv3x3_dgrad": (i, [vp, i, i, i, i, vp, i, vp, vp, vp]),
            "cno_conv3x3_wgrad": (i, [vp, vp, i, i, i, i, i, vp, vp, vp]),
            "cno_weights_to_bf16": (i, [vp, i, i, vp, vp, vp]),
            "cno_create": (i, [i, C.POINTER(C.c_int), i, i, C.POINTER(vp)]),
            "cno_destroy": (i, [vp]),
            "cno_set_stream": (i, [vp, vp]),
            "cno_num_params": (i, [vp, C.POINTER(C.c_longlong)]),
            "cno_set_params": (i, [vp, vp]),
            "cno_get_params": (i, [vp, vp]),
            "cno_get_grads": (i, [vp, vp]),
            "cno_forward": (i, [vp, vp, i, i, i, vp, i]),
            "cno_train_step": (i, [vp, vp, vp, i, i, i, f, i, C.POINTER(d)]),
            "cno_last_output": (i, [vp, C.POINTER(vp)]),
            "cno_pack_fields": (i, [vp, i, i, i, vp, vp, vp, i, vp]),
            "cno_pack_delta": (i, [vp, vp, i, i, i, vp, vp, vp]),
            "cno_apply_update": (i, [vp, vp, i, i, i, vp, i, vp, vp, vp, f, vp]),
            "cno_field_checks": (i, [vp, vp, vp, vp, i, i, C.POINTER(d), vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return _lib


def _check(status: int):
    if status != CNO_OK:
        raise CnoError(status, load().cno_error_string().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def wait_selftest(seconds: float = 0.2):
    """(gave_up, elapsed seconds) of a bounded wait on a barrier nothing arrives at."""
    g, e = C.c_int(0), C.c_double(0.0)
    _check(load().cno_wait_selftest(float(seconds), C.byref(g), C.byref(e)))
    return bool(g.value), float(e.value)


def read_status(clear: bool = False) -> int:
    v = C.c_uint(0)
    _check(load().cno_read_status(C.byref(v), int(clear)))
    return int(v.value)


def conv3x3_forward(x, w_bf16, bias, act: bool, out_f32: bool = False, n_store: int | None = None):
    """y = conv3x3(x, W) + b (lrelu if act); x bf16 [n,h,w,cin], W bf16 [cout,9,cin], b fp32 [cout]."""
    import torch
    n, h, wd, cin = x.shape
    cout = w_bf16.shape[0]
    ns = cout if n_store is None else n_store
    y = torch.empty((n, h, wd, ns), device=x.device, dtype=torch.float32 if out_f32 else torch.bfloat16)
    _check(load().cno_conv3x3_forward(_ptr(x), n, h, wd, cin, _ptr(w_bf16), _ptr(bias), cout, int(act), _ptr(y),
                                      int(out_f32), ns, ns, _stream()))
    return y


def conv3x3_dgrad(dz, wd_bf16, slope_src=None):
    """dx = conv3x3(dz, Wd) (times lrelu'(slope_src)); Wd bf16 [cin,9,cout]."""
    import torch
    n, h, w, cout = dz.shape
    cin = wd_bf16.shape[0]
    dx = torch.empty((n, h, w, cin), device=dz.device, dtype=torch.bfloat16)
    _check(load().cno_conv3x3_dgrad(_ptr(dz), n, h, w, cout, _ptr(wd_bf16), cin, _ptr(slope_src), _ptr(dx),
                                    _stream()))
    return dx


def conv3x3_wgrad(dz, x):
    """(dW fp32 [cout,9,cin], db fp32 [cout]) of sum(dz * conv3x3(x, W))."""
    import torch
    n, h, w, cout = dz.shape
    cin = x.shape[3]
    dw = torch.empty((cout, 9, cin), device=dz.device, dtype=torch.float32)
    db = torch.empty((cout,), device=dz.device, dtype=torch.float32)
    _check(load().cno_conv3x3_wgrad(_ptr(dz), _ptr(x), n, h, w, cin, cout, _ptr(dw), _ptr(db), _stream()))
    return dw, db


def weights_to_bf16(w32):
    """(W bf16 [cout,9,cin], Wd bf16 [cin,9,cout] with taps reversed) of FP32 weights."""
    import torch
    cout, _, cin = w32.shape
    wf = torch.empty((cout, 9, cin), device=w32.device, dtype=torch.bfloat16)
    wd = torch.empty((cin, 9, cout), device=w32.device, dtype=torch.bfloat16)
    _check(load().cno_weights_to_bf16(_ptr(w32), cout, cin, _ptr(wf), _ptr(wd), _stream()))
    return wf, wd


def layer_shapes(cin=CIN, widths=WIDTHS, cout=COUT):
    """(in, out) of the twelve convolutions in the order of the flat parameter vector."""
    c0, c1, c2, c3 = widths
    return [(cin, c0), (c0, c0), (c0, c1), (c1, c1), (c1, c2), (c2, c2), (c2, c3), (c3, c3),
            (c3, c1), (c1, c0), (c0, c0), (c0, cout)]


def forward_flops(h, w, n=1, cin=CIN, widths=WIDTHS, cout=COUT):
    """Multiply-add FLOPs (2 per MAC) of the twelve convolutions of one forward
    pass over n images of h x w."""
    levels = [0, 0, 1, 1, 2, 2, 3, 3, 2, 1, 0, 0]
    return sum(2.0 * 9 * ci * co * n * (h >> lv) * (w >> lv)
               for (ci, co), lv in zip(layer_shapes(cin, widths, cout), levels))


def unflatten(flat, cin=CIN, widths=WIDTHS, cout=COUT):
    """[(W [o,9,i], b [o])] views of a flat parameter vector."""
    out, k = [], 0
    for ci, co in layer_shapes(cin, widths, cout):
        w = flat[k:k + co * 9 * ci].reshape(co, 9, ci)
        k += co * 9 * ci
        b = flat[k:k + co]
        k += co
        out.append((w, b))
    return out


def flatten(params):
    return np.concatenate([np.concatenate([np.asarray(w, np.float32).ravel(), np.asarray(b, np.float32).ravel()])
                           for w, b in params])


class Net:
    """A network on the current CUDA device (see include/cno.h)."""

    def __init__(self, cin=CIN, widths=WIDTHS, cout=COUT, nf=NF):
        L = load()
        self.cin, self.widths, self.cout, self.nf = cin, tuple(widths), cout, nf
        h = C.c_void_p()
        arr = (C.c_int * 4)(*widths)
        _check(L.cno_create(cin, arr, cout, nf, C.byref(h)))
        self._h = h
        n = C.c_longlong()
        _check(L.cno_num_params(h, C.byref(n)))
        self.nparams = int(n.value)
        _check(L.cno_set_stream(h, _stream()))

    def close(self):
        if self._h:
            load().cno_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self):
        _check(load().cno_set_stream(self._h, _stream()))

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == self.nparams
        _check(load().cno_set_params(self._h, flat.ctypes.data_as(C.c_void_p)))

    def params(self):
        out = np.empty(self.nparams, np.float32)
        _check(load().cno_get_params(self._h, out.ctypes.data_as(C.c_void_p)))
        return out

    def grads(self):
        out = np.empty(self.nparams, np.float32)
        _check(load().cno_get_grads(self._h, out.ctypes.data_as(C.c_void_p)))
        return out

    def forward(self, x, out=None):
        """x bf16 [n,h,w,cin] -> FP32 [n,h,w,nf] (device)."""
        import torch
        n, h, w, _ = x.shape
        if out is None:
            out = torch.empty((n, h, w, self.nf), device=x.device, dtype=torch.float32)
        _check(load().cno_forward(self._h, _ptr(x), n, h, w, _ptr(out), out.shape[-1]))
        return out

    def train_step(self, x, target, lr: float, update: bool = True, want_loss: bool = True):
        n, h, w, _ = x.shape
        loss = C.c_double(0.0)
        _check(load().cno_train_step(self._h, _ptr(x), _ptr(target), n, h, w, float(lr), int(update),
                                     C.byref(loss) if want_loss else None))
        return float(loss.value) if want_loss else None


def _ptr_array(ts):
    return (C.c_void_p * len(ts))(*[t.data_ptr() for t in ts])


def pack_fields(fields, offset, inv_scale, cin=CIN, out=None):
    """Network input (bf16 [1,ny,nx,cin], or the given `out` of that shape) from a
    list of device FP32 fields [ny,nx]."""
    import torch
    ny, nx = fields[0].shape
    x = torch.empty((1, ny, nx, cin), device=fields[0].device, dtype=torch.bfloat16) if out is None else out
    off = (C.c_float * len(fields))(*offset)
    isc = (C.c_float * len(fields))(*inv_scale)
    _check(load().cno_pack_fields(_ptr_array(fields), len(fields), nx, ny, off, isc, _ptr(x), cin, _stream()))
    return x


def pack_delta(cur, nxt, inv_scale, out):
    """out[y,x,f] = (nxt[f] - cur[f]) * inv_scale[f] (device FP32 [ny,nx,nfield])."""
    ny, nx = cur[0].shape
    isc = (C.c_float * len(cur))(*inv_scale)
    _check(load().cno_pack_delta(_ptr_array(cur), _ptr_array(nxt), len(cur), nx, ny, isc, _ptr(out), _stream()))
    return out


def apply_update(src, dst, out, scale, phi_band=0.0, lo=None, hi=None):
    """dst[f] = clamp(src[f] + scale[f] * out[..., f], lo[f], hi[f]) (device; dst
    may be src); with phi_band > 0, field 0 changes only where |src[0]| < phi_band."""
    ny, nx = src[0].shape
    n = len(src)
    sc = (C.c_float * n)(*scale)
    lo_a = None if lo is None else (C.c_float * n)(*lo)
    hi_a = None if hi is None else (C.c_float * n)(*hi)
    _check(load().cno_apply_update(_ptr_array(src), _ptr_array(dst), n, nx, ny, _ptr(out), out.shape[-1], sc, lo_a,
                                   hi_a, float(phi_band), _stream()))


def field_checks(phi, fs=None, T=None, hcoef=None):
    """(sum phi, sum chi, sum f_s, sum (1 - phi^2), sum |grad phi|, min T, max T,
    sum rho H) in FP64 of device fields [ny,nx]; hcoef = ((rho Cp)_l, (rho Cp)_s,
    (rho Cp)_g, rho_l L) for the enthalpy sum."""
    ny, nx = phi.shape
    out = (C.c_double * 8)()
    hc = None if hcoef is None else (C.c_float * 4)(*hcoef)
    _check(load().cno_field_checks(_ptr(phi), _ptr(fs), _ptr(T), hc, nx, ny, out, _stream()))
    return tuple(out)
