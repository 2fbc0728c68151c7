"""The C ABI library without a GPU: it builds for sm_103a, loads, exports every
symbol that include/lbfreeze.h declares, its struct layouts match the Python
binding, and argument checks reject bad input before touching a device."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2511_09422_gb300 import _build, lbfreeze
from paper_2511_09422_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbfreeze.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return lbfreeze.load()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 12
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (lb_[a-z_]+)\b", out))
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)
    assert set(lbfreeze.EXPORTS) <= set(names)


def test_struct_layout_matches_header(tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbfreeze.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(lb_grid), sizeof(lb_params),'
                    ' sizeof(lb_fields), offsetof(lb_params, fs_modulated_st), offsetof(lb_params, divu_mode),'
                    ' offsetof(lb_params, pop_storage));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(prog)], check=True)
    vals = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()))
    assert vals == [C.sizeof(lbfreeze.lb_grid), C.sizeof(lbfreeze.lb_params), C.sizeof(lbfreeze.lb_fields),
                    lbfreeze.lb_params.fs_modulated_st.offset, lbfreeze.lb_params.divu_mode.offset,
                    lbfreeze.lb_params.pop_storage.offset]


def test_error_strings(lib):
    for k in range(5):
        assert lib.lb_error_string(k)
    assert lib.lb_error_string(99) == b"unknown status"
    lib.lb_destroy(None)  # no-op


def _create(lib, grid, params, n, phi=True):
    z = np.zeros(n, dtype=np.float32)
    f = lbfreeze.lb_fields()
    ptr = z.ctypes.data_as(C.POINTER(C.c_float))
    f.phi = ptr if phi else None
    f.T, f.C, f.ux, f.uy, f.on_device = ptr, ptr, None, None, 0
    h = C.c_void_p()
    st = lib.lb_create(C.byref(lbfreeze.make_grid(grid)), C.byref(lbfreeze.make_params(params)), C.byref(f), C.byref(h))
    return st, h


@pytest.mark.parametrize("bad", [
    dict(grid=dict(nx=0)), dict(grid=dict(ny=0)), dict(grid=dict(nx=1 << 15, ny=1 << 15)),
    dict(grid=dict(nx=1, ny=1 << 26)),
    dict(params=dict(eps=0.0)), dict(params=dict(rho_g=0.0)), dict(params=dict(mu_l=0.0)),
    dict(params=dict(mobility=-1.0)), dict(params=dict(lam_s=0.0)), dict(params=dict(D_l=0.0)),
    dict(params=dict(divu_mode=2)), dict(params=dict(divu_mode=-1)), dict(params=dict(pop_storage=3)), dict(params=dict(sigma0=float("nan"))),
    dict(params=dict(lattice_fl=2)), dict(params=dict(lattice_fl=1, pop_storage=1)),
    dict(params=dict(lattice_fl=1, pop_storage=2)),
    dict(grid=dict(cos_theta_bottom=1.5)), dict(grid=dict(cos_theta_top=float("nan"))),
    dict(params=dict(T_sol=1.0, T_liq=0.0)), dict(grid=dict(bc_top=7)), dict(phi=False)])
def test_invalid_arguments_rejected_without_a_device(lib, bad):
    w = W.stefan_layer(nx=8, ny=8, h0=4)
    g = dict(w["grid"], **bad.get("grid", {}))
    p = dict(w["params"], **bad.get("params", {}))
    st, h = _create(lib, g, p, 64, phi=bad.get("phi", True))
    assert st == lbfreeze.LB_ERR_INVALID_ARG
    assert h.value is None
    assert lib.lb_last_error(None)



def test_create_error_message_is_per_thread(lib):
    """lb_last_error(NULL) is the calling thread's last lb_create failure: a
    failure in another thread neither shows nor overwrites it."""
    import threading
    w = W.stefan_layer(nx=8, ny=8, h0=4)
    st, _ = _create(lib, w["grid"], dict(w["params"], eps=0.0), 64)
    assert st == lbfreeze.LB_ERR_INVALID_ARG
    mine = lib.lb_last_error(None)
    assert b"eps" in mine
    seen = {}

    def other():
        seen["before"] = lib.lb_last_error(None)
        st2, _ = _create(lib, dict(w["grid"], nx=0), w["params"], 64)
        seen["status"] = st2
        seen["after"] = lib.lb_last_error(None)

    t = threading.Thread(target=other)
    t.start()
    t.join()
    assert seen["before"] == b""
    assert seen["status"] == lbfreeze.LB_ERR_INVALID_ARG and b"nx" in seen["after"]
    assert lib.lb_last_error(None) == mine

def test_null_arguments(lib):
    assert lib.lb_create(None, None, None, None) == lbfreeze.LB_ERR_INVALID_ARG
    assert lib.lb_step(None, 1) == lbfreeze.LB_ERR_INVALID_ARG
    assert lib.lb_reduce(None, None) == lbfreeze.LB_ERR_INVALID_ARG
    assert lib.lb_get_fields(None, *([None] * 7), 0) == lbfreeze.LB_ERR_INVALID_ARG
    assert lib.lb_slab_create(None, None, None, 0, 8, None) == lbfreeze.LB_ERR_INVALID_ARG
    assert lib.lb_slab_pack(None, 0, None, 0) == lbfreeze.LB_ERR_INVALID_ARG
    assert lib.lb_slab_unpack(None, 1, None, 1) == lbfreeze.LB_ERR_INVALID_ARG
    assert lib.lb_slab_halo_bytes(None) == 0


@pytest.mark.parametrize("y0,y1", [(0, 3), (2, 20), (20, 38), (-1, 10), (30, 41)])
def test_slab_rows_rejected_without_a_device(lib, y0, y1):
    """A slab of fewer than 4 rows, or one that leaves a neighbour fewer than
    4, or one outside the lattice, is refused before any device work."""
    import ctypes as C
    w = W.parity_droplet(nx=32, ny=40)
    f = lbfreeze.lb_fields()
    phi = np.zeros(32 * 44, dtype=np.float32)
    for k in ("phi", "T", "C"):
        setattr(f, k, phi.ctypes.data_as(C.POINTER(C.c_float)))
    h = C.c_void_p()
    st = lib.lb_slab_create(C.byref(lbfreeze.make_grid(w["grid"])), C.byref(lbfreeze.make_params(w["params"])),
                            C.byref(f), y0, y1, C.byref(h))
    assert st == lbfreeze.LB_ERR_INVALID_ARG and h.value is None
    assert b"slab" in lib.lb_last_error(None)


def test_workloads_are_seeded():
    a = W.parity_droplet(nx=32, ny=32)
    b = W.parity_droplet(nx=32, ny=32)
    for k in ("phi", "T", "C"):
        assert np.array_equal(a["fields"][k], b["fields"][k])
    c = W.parity_droplet(nx=32, ny=32, seed=1)
    assert not np.array_equal(a["fields"]["T"], c["fields"]["T"])


def test_droplet_sweep_is_seeded_and_in_range():
    a = W.droplet_sweep(n=12)
    b = W.droplet_sweep(n=12)
    for wa, wb in zip(a, b):
        assert wa["grid"] == wb["grid"] and wa["params"] == wb["params"]
        for k in wa["fields"]:
            assert np.array_equal(wa["fields"][k], wb["fields"][k])
        side = wa["grid"]["nx"]
        assert wa["grid"]["ny"] == side and 128 <= side <= 512
        assert 0.2 * side <= wa["meta"]["radius"] <= 0.35 * side
        assert 0.05 <= wa["meta"]["ste"] <= 0.5 and 0.0 <= wa["meta"]["c0"] <= 0.1
    assert len({w["grid"]["nx"] for w in a}) > 6  # uneven sizes
