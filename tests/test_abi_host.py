"""C-ABI checks that need no GPU: the library loads, exports every function the
header declares, and rejects invalid boundary specifications before touching CUDA."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_0811_4593_gb300 import build
    build.build()
    import paper_0811_4593_gb300._binding as b
    return b


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^LBM_API\s+[\w\s\*]+?\b(lbm_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("lbm_create", "lbm_step", "lbm_macros", "lbm_destroy", "lbm_residual"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    lib = C.CDLL(L.library_path())
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(L.EXPORTS)


def make_specs(b, kinds, us=None, tables=None):
    specs = (b.FaceSpec * 6)()
    keep = []
    for i in range(6):
        specs[i].kind = kinds[i]
        u = (us or [(0.0, 0.0, 0.0)] * 6)[i]
        for j in range(3):
            specs[i].u[j] = u[j]
        if tables and tables[i] is not None:
            t = np.ascontiguousarray(tables[i], np.float64)
            keep.append(t)
            specs[i].u_table = t.ctypes.data_as(C.POINTER(C.c_double))
    return specs, keep


def create(b, nx, ny, nz, tau, specs, prec=1, rho0=1.0):
    out = C.c_void_p()
    st = b.lib().lbm_create(nx, ny, nz, tau, C.cast(specs, C.c_void_p), prec, rho0, C.byref(out))
    return st, out


@pytest.mark.parametrize("case", ["small_dim", "tau", "unpaired", "normal_speed", "table_speed", "table_nan",
                                  "rho0", "precision", "too_large", "kind", "two_pressure_axes",
                                  "pressure_density", "pressure_table_nan"])
def test_invalid_specifications_are_rejected(L, case):
    b = L
    kinds = [1, 1, 0, 0, 1, 1]
    us = [(0.0, 0.0, 0.0)] * 6
    tables = None
    dims, tau, prec, rho0 = (8, 8, 8), 0.8, 1, 1.0
    if case == "small_dim":
        dims = (2, 8, 8)
    elif case == "tau":
        tau = 0.5
    elif case == "unpaired":
        kinds = [1, 0, 0, 0, 1, 1]
    elif case == "normal_speed":
        us[0] = (1.0, 0.0, 0.0)
    elif case == "table_speed":
        t = np.zeros((8, 8, 3))
        t[3, 4, 0] = -1.5
        tables = [None, t, None, None, None, None]
    elif case == "table_nan":
        t = np.zeros((8, 8, 3))
        t[0, 0, 2] = np.nan
        tables = [None, None, None, None, t, None]
    elif case == "rho0":
        rho0 = -1.0
    elif case == "precision":
        prec = 7
    elif case == "too_large":
        dims = (1024, 1024, 256)
    elif case == "kind":
        kinds = [3, 3, 0, 0, 1, 1]
    elif case == "two_pressure_axes":
        kinds = [2, 1, 0, 0, 2, 1]
    elif case == "pressure_density":
        kinds = [2, 1, 0, 0, 1, 1]
    elif case == "pressure_table_nan":
        kinds = [1, 2, 0, 0, 1, 1]
    specs, keep = make_specs(b, kinds, us, tables)
    if case == "two_pressure_axes":
        specs[0].rho = specs[4].rho = 1.0
    if case == "pressure_table_nan":
        t = np.ones((8, 8))
        t[2, 2] = np.nan
        keep.append(t)
        specs[1].rho_table = t.ctypes.data_as(C.POINTER(C.c_double))
    st, out = create(b, *dims, tau, specs, prec, rho0)
    assert st == b.LBM_ERR_ARG, (case, st, b.last_error())
    assert not out.value
    assert len(b.last_error()) > 0
    del keep


def test_unknown_scheme_is_rejected(L):
    b = L
    specs, keep = make_specs(b, [1, 1, 0, 0, 1, 1])
    out = C.c_void_p()
    st = b.lib().lbm_create_scheme(8, 8, 8, 0.8, C.cast(specs, C.c_void_p), 1, 1.0, 5, C.byref(out))
    assert st == b.LBM_ERR_ARG and not out.value


def test_null_arguments(L):
    b = L
    assert b.lib().lbm_step(None, 1) == b.LBM_ERR_ARG
    assert b.lib().lbm_destroy(None) == b.LBM_OK
    assert b.lib().lbm_macros(None, None, None) == b.LBM_ERR_ARG
    assert "NULL" in b.last_error()


def test_no_cpu_fallback_without_a_gpu(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    b = L
    specs, keep = make_specs(b, [1, 1, 0, 0, 1, 1])
    st, out = create(b, 8, 8, 8, 0.8, specs)
    assert st == b.LBM_ERR_CUDA
    import paper_0811_4593_gb300 as lbm
    with pytest.raises(RuntimeError):
        lbm.Lattice(8, 8, 8, 0.8, [None] * 6)


def test_header_compiles_as_plain_c(tmp_path):
    # the ABI is C: a C99 translation unit that includes the header and takes the address
    # of every declared function compiles without warnings
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = declared_functions()
    src = tmp_path / "use_lbm.c"
    src.write_text('#include "lbm.h"\n' + "void* table[] = {\n" + ",\n".join(f"  (void*){n}" for n in names) +
                   "\n};\nint main(void) { lbm_ctx* c = 0; lbm_status s = LBM_OK; (void)c; return (int)s; }\n")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-c", str(src), "-o", str(tmp_path / "use_lbm.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_a_c_program_links_and_calls_the_library(L, tmp_path):
    # a plain C program against liblbm.so: host-only calls work without a device, and
    # lbm_create either succeeds (a GPU is present) or reports LBM_ERR_CUDA
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "prog.c"
    src.write_text(r'''
#include <stdio.h>
#include "lbm.h"
int main(void) {
  uint32_t m = 0;
  if (lbm_rule_unknowns(1, &m) != LBM_OK) return 1;
  if (lbm_rule_unknowns(0, &m) != LBM_ERR_ARG) return 2;
  lbm_face_spec f[6] = {0};
  for (int i = 0; i < 6; ++i) f[i].kind = LBM_FACE_PERIODIC;
  f[4].kind = f[5].kind = LBM_FACE_VELOCITY;
  f[5].u[0] = 0.05;
  lbm_ctx* c = NULL;
  lbm_status s = lbm_create(8, 8, 17, 1.0, f, LBM_F64, 1.0, &c);
  if (s == LBM_OK) { if (lbm_step(c, 10) != LBM_OK) return 3; lbm_destroy(c); }
  else if (s != LBM_ERR_CUDA) return 4;
  if (lbm_create(2, 8, 17, 1.0, f, LBM_F64, 1.0, &c) != LBM_ERR_ARG) return 5;
  printf("%u %d %s\n", m, (int)s, lbm_last_error(NULL));
  return 0;
}
''')
    lib = L.library_path()
    exe = tmp_path / "prog"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), lib,
                        "-o", str(exe), f"-Wl,-rpath,{os.path.dirname(lib)}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, (run.returncode, run.stdout, run.stderr)
    mask = int(run.stdout.split()[0])
    assert mask == sum(1 << k for k in (0, 6, 7, 8, 9))   # c_1 = +x: the five populations with c_x > 0
