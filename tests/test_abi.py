"""C ABI checks that need no GPU: the library loads, exports every declared symbol, and
rejects invalid configurations before touching the device."""
import ctypes as C
import os
import re

import pytest

import paper_2304_14074_gb300 as ch
from paper_2304_14074_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(inc, fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(ch_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = ch.load()
    decl = declared_functions()
    assert len(decl) >= 15
    missing = [n for n in decl if not hasattr(lib, n)]
    assert not missing, missing
    assert set(decl) == set(ch.EXPORTED_SYMBOLS)


def test_status_strings():
    lib = ch.load()
    for code, name in ch.STATUS.items():
        assert lib.ch_status_string(code).decode() == name


def _cfg(**kw):
    base = dict(n=64, eps=0.05, T=0.1, n_slices=4, fine_steps=10)
    base.update(kw)
    return ch.Config(**base).c()


BAD_CONFIGS = [dict(dim=2), dict(n=0), dict(n=5000), dict(eps=0.0), dict(eps=float("inf")), dict(T=-1.0),
               dict(T=float("nan")), dict(n_slices=0), dict(fine_steps=0), dict(coarse_steps=0),
               dict(max_iters=9), dict(precision=3), dict(newton_tol=0.0), dict(newton_tol=float("inf")),
               dict(variant="PA-I", newton_max=0), dict(tol=float("nan")), dict(err_tol=float("inf")),
               dict(lin_tol=1.0), dict(lin_tol=float("nan")), dict(lin_max=20000)]


@pytest.mark.parametrize("bad", BAD_CONFIGS)
def test_create_rejects_invalid_config_without_device(bad):
    lib = ch.load()
    cc = _cfg(**bad)
    h = C.c_void_p()
    assert lib.ch_parareal_create(C.byref(cc), 1, None, C.byref(h)) == 1
    assert not h.value


def test_create_rejects_bad_batch_and_null_out():
    lib = ch.load()
    cc = _cfg()
    h = C.c_void_p()
    assert lib.ch_parareal_create(C.byref(cc), 0, None, C.byref(h)) == 1
    assert lib.ch_parareal_create(C.byref(cc), 1, None, None) == 1
    assert lib.ch_parareal_create(None, 1, None, C.byref(h)) == 1


def test_propagate_rejects_invalid_arguments_without_device():
    lib = ch.load()
    cc = _cfg()
    assert lib.ch_propagate(C.byref(cc), 0, 0, 1e-3, 1, C.c_void_p(8), C.c_void_p(8), None, None) == 1
    assert lib.ch_propagate(C.byref(cc), 1, 7, 1e-3, 1, C.c_void_p(8), C.c_void_p(8), None, None) == 1
    assert lib.ch_propagate(C.byref(cc), 1, 0, 0.0, 1, C.c_void_p(8), C.c_void_p(8), None, None) == 1
    assert lib.ch_propagate(C.byref(cc), 1, 0, 1e-3, 1, None, C.c_void_p(8), None, None) == 1


def test_theory_bound_rejects_invalid_arguments_without_device():
    lib = ch.load()
    cc = _cfg()
    out = (C.c_double * 8)()
    assert lib.ch_parareal_theory_bound(None, 0.0, 2, out, 8, None) == 1
    assert lib.ch_parareal_theory_bound(C.byref(cc), 0.0, 2, None, 8, None) == 1
    assert lib.ch_parareal_theory_bound(C.byref(cc), 0.0, -1, out, 8, None) == 1
    assert lib.ch_parareal_theory_bound(C.byref(cc), 0.0, 6, out, 8, None) == 1  # needs kmax + 3
    for field, value in (("n", 0), ("eps", 0.0), ("T", -1.0), ("n_slices", 0), ("fine_steps", 0),
                         ("coarse_steps", 0), ("variant", 5), ("dim", 3)):
        bad = _cfg()
        setattr(bad, field, value)
        assert lib.ch_parareal_theory_bound(C.byref(bad), 0.0, 2, out, 8, None) == 1, field
    npa = _cfg()
    npa.variant = 3  # NPA-I needs the LTE constant
    assert lib.ch_parareal_theory_bound(C.byref(npa), 0.0, 2, out, 8, None) == 1
    assert lib.ch_parareal_theory_bound(C.byref(npa), float("nan"), 2, out, 8, None) == 1


def test_set_fine_nn_rejects_null_handle_without_device():
    lib = ch.load()
    assert lib.ch_parareal_set_fine_nn(None, 8, 0.25, 1e-10, 100) == 1


def test_destroy_accepts_null_and_last_error_on_null():
    lib = ch.load()
    lib.ch_parareal_destroy(None)
    assert lib.ch_parareal_last_error(None).decode() == "NULL handle"


def test_binding_struct_layout_matches_header(tmp_path):
    """Sizes and field offsets of the ctypes structures equal those the C compiler gives the
    header's structs."""
    import subprocess
    fields = {"ch_config": [f for f, _ in _lib._Config._fields_], "ch_stats": [f for f, _ in _lib._Stats._fields_]}
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "ch_parareal.h"', "int main(void) {"]
    for st, fs in fields.items():
        src.append(f'  printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            src.append(f'  printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    src += ["  return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for st, cls in (("ch_config", _lib._Config), ("ch_stats", _lib._Stats)):
        assert int(got[st]) == C.sizeof(cls), st
        for f in fields[st]:
            assert int(got[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)


def test_gtheta_entry_points_reject_invalid_arguments_without_device():
    lib = ch.load()
    assert lib.ch_gtheta_create(0, None, None) == 1
    lib.ch_gtheta_destroy(None)
    assert lib.ch_gtheta_last_error(None).decode() == "NULL handle"
    assert lib.ch_gtheta_set_params(None, None, 0) == 1
    assert lib.ch_gtheta_get_params(None, None, 0) == 1
    assert lib.ch_gtheta_forward(None, None, None, None, 1, 8) == 1
    assert lib.ch_gtheta_gradients(None, None, None, 1, 8, 1, None, 0, None) == 1
    assert lib.ch_gtheta_train(None, None, None, 1, 2, 8, 1, 1, 1, 1e-3, 0, None) == 1
    assert lib.ch_parareal_set_coarse_model(None, None, 0, 0) == 1
    assert lib.ch_parareal_get_reference_device(None, None, 0) == 1
    assert lib.ch_parareal_set_eps(None, None, 0) == 1
    assert lib.ch_ensemble_create(None, 1, None, None, None) == 1
    assert lib.ch_ensemble_run(None) == 1
    assert lib.ch_ensemble_groups(None) == 0
    lib.ch_ensemble_destroy(None)
    assert lib.ch_ensemble_last_error(None).decode() == "NULL handle"


def test_gtheta_parameter_layout_matches_header():
    src = open(os.path.join(ROOT, "include", "ch_parareal.h")).read()
    m = re.search(r"#define\s+CH_GTHETA_PARAMS\s+(\d+)", src)
    assert m and int(m.group(1)) == ch.CH_GTHETA_PARAMS
    c = _lib.GTHETA_CHANNELS
    assert sum(9 * c[l] * c[l + 1] + c[l + 1] for l in range(6)) == ch.CH_GTHETA_PARAMS
    import numpy as np
    p = np.arange(ch.CH_GTHETA_PARAMS, dtype=np.float32)
    W, b = ch.gtheta_unflatten(p)
    assert W[0].shape == (3, 3, 32, 1) and W[5].shape == (3, 3, 1, 32) and b[5].shape == (1,)
    assert W[1][0, 0, 0, 1] == 320 + 1 and b[0][0] == 288  # W_l[dy][dx][co][ci] then b_l
    assert np.array_equal(ch.gtheta_flatten(W, b), p)


@pytest.mark.parametrize("bad", BAD_CONFIGS + [dict(dim=2, n=31)])
def test_noalloc_rejects_invalid_config_without_device(bad):
    """The allocation-free entry point applies the same checks as ch_parareal_create (plus
    dim = 1) before it touches the device."""
    lib = ch.load()
    cc = _cfg(**bad)
    nd = cc.n ** cc.dim if cc.n > 0 else 1
    ns = max(cc.n_slices, 1)
    s = lib.ch_parareal_solve_noalloc(C.byref(cc), 1, C.c_void_p(8), C.c_void_p(8), (ns + 1) * nd, None, None)
    assert s == 1
