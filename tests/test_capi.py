"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/fzp.h declares, and rejects invalid input before it
touches the device."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fzp():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2609_01978_gb300 as m
    return m


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"FZP_API\s+[\w\s\*]+?\b(fzp_\w+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(fzp):
    names = _declared()
    assert {"fzp_plan", "fzp_propagate_roi", "fzp_metrics", "fzp_plan_destroy", "fzp_last_error"} <= names
    L = fzp.lib()
    for n in sorted(names):
        assert hasattr(L, n), n


@pytest.mark.parametrize("kw,frag", [
    (dict(D=-1.0), "positive"),
    (dict(f=0.0), "positive"),
    (dict(lam=float("nan")), "finite"),
    (dict(pitch=0.0), "positive"),
    (dict(M=100), "power of two"),
    (dict(M=32), "power of two"),
    (dict(M=2048), "power of two"),
    (dict(N=1000), "odd"),
    (dict(dx=2e-6), "Eq. 6"),
    (dict(form=7), "form"),
    (dict(precision=9), "precision"),
    (dict(centre_open=2), "centre_open"),
    (dict(centre_open=1, levels=4), "binary amplitude"),
])
def test_invalid_parameters_rejected(fzp, kw, frag):
    base = dict(D=1e-3, f=5e-3, lam=632.8e-9, M=64, pitch=0.4e-6)
    base.update(kw)
    with pytest.raises(fzp.FzpError) as ei:
        fzp.Plan(**base)
    assert ei.value.status == fzp.FZP_E_INVALID
    assert frag in str(ei.value)


def test_unsupported_combinations(fzp):
    base = dict(D=1e-3, f=5e-3, lam=632.8e-9, M=64, pitch=0.4e-6)
    with pytest.raises(fzp.FzpError) as ei:
        fzp.Plan(form=fzp.FORM_DENSE, precision=fzp.PREC_FP32, **base)
    assert ei.value.status == fzp.FZP_E_UNSUPPORTED
    with pytest.raises(fzp.FzpError) as ei:
        fzp.Plan(form=fzp.FORM_BLUESTEIN, precision=fzp.PREC_SPLIT_BF16, **base)
    assert ei.value.status == fzp.FZP_E_UNSUPPORTED


def test_roi_origin_validation(fzp):
    """Off-axis ROI (Eq. 10's A from the first ROI coordinate): x0 = y0 is
    accepted and reported by the host plan; x0 != y0 needs a second kernel
    matrix and is unsupported; a bad flag or a non-finite origin is invalid."""
    import ctypes
    L = fzp.lib()
    base = dict(D=1e-3, f=5e-3, lam=632.8e-9, M=64, pitch=0.4e-6)
    q = fzp.plan_query(x0=-3.3e-6, **base)
    assert q["x0"] == -3.3e-6
    assert fzp.plan_query(**base)["x0"] == -32 * 0.4e-6
    inf = fzp.PlanInfo()
    for kw, status in [(dict(roi_origin=1, x0=1e-6, y0=2e-6), fzp.FZP_E_UNSUPPORTED),
                       (dict(roi_origin=2), fzp.FZP_E_INVALID),
                       (dict(roi_origin=1, x0=float("inf"), y0=float("inf")), fzp.FZP_E_INVALID),
                       (dict(reserved=1), fzp.FZP_E_INVALID),
                       (dict(conv=3), fzp.FZP_E_INVALID),
                       (dict(conv=-1), fzp.FZP_E_INVALID),
                       (dict(conv=2, precision=0), fzp.FZP_E_UNSUPPORTED)]:
        p = fzp._params(**base)
        for k, v in kw.items():
            setattr(p, k, v)
        assert L.fzp_plan_query(ctypes.byref(p), ctypes.byref(inf)) == status, kw
        h = ctypes.c_void_p()
        assert L.fzp_plan(ctypes.byref(p), ctypes.byref(h)) == status and not h.value, kw


def test_null_arguments(fzp):
    import ctypes
    L = fzp.lib()
    assert L.fzp_plan(None, None) == fzp.FZP_E_INVALID
    h = ctypes.c_void_p()
    assert L.fzp_plan(None, ctypes.byref(h)) == fzp.FZP_E_INVALID and not h.value
    assert L.fzp_propagate_roi(None, 0, 1, None, 0, None) == fzp.FZP_E_INVALID
    assert L.fzp_metrics(None, None, None, None) == fzp.FZP_E_INVALID
    assert L.fzp_plan_destroy(None) == fzp.FZP_OK
    assert b"NULL" in L.fzp_last_error() or L.fzp_last_error() != b""


def test_struct_layouts_match_header(fzp, tmp_path):
    """Every ctypes mirror of a struct in include/fzp.h has the C compiler's
    size and field offsets (the binding marshals by layout, not by name)."""
    import ctypes
    pairs = [("fzp_deform", fzp.Deform), ("fzp_params", fzp.Params), ("fzp_plan_info", fzp.PlanInfo),
             ("fzp_metrics_t", fzp.Metrics), ("fzp_profile_t", fzp.Profile)]
    rename = {"lam": "lambda"}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fzp.h"', "int main(void) {"]
    for cname, cls in pairs:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            c = rename.get(fname, fname)
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {c}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        a, b, v = line.split()
        got[(a, b)] = int(v)
    for cname, cls in pairs:
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_other_entry_points_validate_before_the_device(fzp):
    """Batch, surrogate and no-allocation metric calls reject bad arguments on
    the host (these run here, with no GPU)."""
    import ctypes
    L = fzp.lib()
    h = ctypes.c_void_p()
    assert L.fzp_batch_plan(None, 1, ctypes.byref(h)) == fzp.FZP_E_INVALID
    good = fzp._params(D=1e-3, f=5e-3, lam=632.8e-9, M=64, pitch=0.4e-6)
    arr = (fzp.Params * 1)(good)
    assert L.fzp_batch_plan(arr, 0, ctypes.byref(h)) == fzp.FZP_E_INVALID and not h.value
    bad = fzp._params(D=-1.0, f=5e-3, lam=632.8e-9, M=64, pitch=0.4e-6)
    arr = (fzp.Params * 2)(bad, good)
    assert L.fzp_batch_plan(arr, 2, ctypes.byref(h)) == fzp.FZP_E_INVALID and not h.value
    assert b"positive" in L.fzp_last_error()
    for sizes in [(0, 512, 3, 4114, 256), (8, 512, 0, 4114, 256), (8, 512, 3, 4114, 0), (8, 70000, 3, 4, 4)]:
        assert L.fzp_surrogate_create(*sizes, 0, ctypes.byref(h)) == fzp.FZP_E_INVALID and not h.value
    host = (ctypes.c_double * 2)()
    for kw in (dict(M=1024), dict(M=100), dict(N=1000, M=64), dict(levels=70, M=64)):
        base = dict(D=1e-3, f=5e-3, lam=632.8e-9, pitch=0.4e-6)
        base.update(kw)
        with pytest.raises(fzp.FzpError) as e:
            fzp.metrics_noalloc(ctypes.addressof(host), **base)
        assert e.value.status == fzp.FZP_E_INVALID
    assert L.fzp_batch_destroy(None) == fzp.FZP_OK
    assert L.fzp_surrogate_destroy(None) == fzp.FZP_OK


def test_saczt_host_plan(fzp):
    """The SA-CZT form's host checks: FP32 only, binary flat plates only, exact
    radii in this form only, the padded grid (a power of two >= 1.5 N) reported
    and limited to 16384."""
    import ctypes
    L = fzp.lib()
    base = dict(D=4e-3, f=20e-3, lam=632.8e-9, M=256, pitch=0.2e-6, form=fzp.FORM_SACZT, precision=fzp.PREC_FP32)
    q = fzp.plan_query(exact_radii=1, **base)
    assert q["N"] == 5057 and q["fft_length"] == 8192
    inf = fzp.PlanInfo()
    for kw, status in [(dict(precision=fzp.PREC_FP64), fzp.FZP_E_UNSUPPORTED),
                       (dict(levels=4), fzp.FZP_E_UNSUPPORTED),
                       (dict(form=fzp.FORM_BLUESTEIN, exact_radii=1), fzp.FZP_E_UNSUPPORTED),
                       (dict(D=0.02, f=0.1), fzp.FZP_E_UNSUPPORTED),   # N = 25,285: P = 65536 > 16384
                       (dict(exact_radii=2), fzp.FZP_E_INVALID),
                       (dict(cluster=2), fzp.FZP_E_INVALID)]:
        p = fzp._params(**dict(base, **kw))
        assert L.fzp_plan_query(ctypes.byref(p), ctypes.byref(inf)) == status, kw
