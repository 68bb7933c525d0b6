"""CPU checks of the C ABI: the library builds, loads and exports every entry
point include/wlseno.h declares; calls that need no GPU behave as documented."""
import ctypes
import os
import re

import pytest

from paper_1602_02694_gb300 import wlseno as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "wlseno.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wlseno_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(W.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return W.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
        assert name in W.SIGNATURES, f"binding does not declare {name}"
    assert set(W.SIGNATURES) == set(names)


def test_status_strings(lib):
    assert lib.wlseno_status_string(0) == b"ok"
    assert lib.wlseno_status_string(-8) == b"calls made in the wrong order"
    assert lib.wlseno_status_string(-3) == b"invalid stencil"


def test_argument_errors_without_gpu(lib):
    # null arguments are rejected before any CUDA call
    assert lib.wlseno_create(None, 0, None) == -1
    assert lib.wlseno_get_info(None, None) == -1
    assert lib.wlseno_reconstruct(None, None, None, None, None) == -1
    assert lib.wlseno_rk_step(None, None, 0.0, 0.0, 1, None, None) == -1
    lib.wlseno_destroy(None)
    sch = W.wlseno_scheme()
    sch.pde, sch.n_comp, sch.eps, sch.alpha_c, sch.rank_tol = 7, 1, 1e-2, 1.5, 1e-10
    h = ctypes.c_void_p()
    assert lib.wlseno_create(ctypes.byref(h), 0, ctypes.byref(sch)) == -1  # unknown pde


def test_create_reports_missing_device(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    sch = W.wlseno_scheme()
    sch.pde, sch.n_comp, sch.eps, sch.alpha_c, sch.rank_tol = 0, 1, 1e-2, 1.5, 1e-10
    h = ctypes.c_void_p()
    assert lib.wlseno_create(ctypes.byref(h), 0, ctypes.byref(sch)) == -4


def test_balanced_option_is_validated_before_any_cuda_call(lib):
    """balanced: 0 or 1, scalar equations only, a finite margin >= 0."""
    base = dict(pde=1, n_comp=1, eps=1e-2, alpha_c=1.5, rank_tol=1e-10, balance_margin=0.02)
    bad = [dict(balanced=2), dict(balanced=1, pde=2, n_comp=4, gamma=1.4),
           dict(balanced=1, balance_margin=-1.0), dict(balanced=1, balance_margin=float("nan")),
           dict(balanced=1, balance_margin=float("inf"))]
    for change in bad:
        sch = W.wlseno_scheme()
        for k, v in {**base, **change}.items():
            setattr(sch, k, v)
        h = ctypes.c_void_p()
        assert lib.wlseno_create(ctypes.byref(h), 0, ctypes.byref(sch)) == -1, change


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the header's sizes and field
    offsets (compiled and printed by the host C compiler)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"wlseno_mesh": W.wlseno_mesh, "wlseno_stencil_opts": W.wlseno_stencil_opts,
               "wlseno_scheme": W.wlseno_scheme, "wlseno_info": W.wlseno_info,
               "wlseno_diagnostics": W.wlseno_diagnostics}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "wlseno.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        parts = line.split()
        if len(parts) == 3:
            got[(parts[0], parts[1])] = int(parts[2])
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def test_kernel_kind_and_status_tables_match_the_header():
    text = open(HEADER).read()
    n_kinds = int(re.search(r"WLSENO_N_KERNEL_KINDS\s*=\s*(\d+)", text).group(1))
    assert len(W.KERNEL_KINDS) == n_kinds
    kinds = dict((m.group(1).lower(), int(m.group(2)))
                 for m in re.finditer(r"WLSENO_KERNEL_([A-Z]+)\s*=\s*(\d+)", text))
    for k, name in enumerate(W.KERNEL_KINDS):
        assert kinds[name] == k, name
    assert int(re.search(r"WLSENO_EULER\s*=\s*(\d+)", text).group(1)) == W.EULER
    assert int(re.search(r"WLSENO_FP32_BULK\s*=\s*(\d+)", text).group(1)) == W.FP32_BULK
