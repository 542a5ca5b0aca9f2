"""include/lcs_bound.h is a C header: a C11 program (and the same file as C++)
compiles against it with every warning an error, links with the library and
runs the calls that need no device (defaults, status strings, argument errors
raised before any CUDA call).  The structs the Python binding mirrors have the
C compiler's sizes and field offsets.
"""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT

PROGRAM = r"""
#include <stdio.h>
#include <string.h>

#include "lcs_bound.h"

int main(void) {
  lcs_bound_opts o;
  lcs_bound_t* h = NULL;
  uint64_t n_orbit = 0;
  if (lcs_bound_default_opts(&o) != LCS_OK) return 1;
  printf("defaults %d %d %d %d %d\n", o.check_every, o.r_mode, o.f_mode, o.frac_bits, o.symmetry);
  printf("errstr %s|%s\n", lcs_bound_errstr(LCS_OK), lcs_bound_errstr(LCS_EUNSUPPORTED));
  /* shapes the interface rejects before touching the device */
  printf("create %d %d %d\n", (int)lcs_bound_create(1, 2, 3, &o, &h), (int)lcs_bound_create(2, 17, 1, &o, &h),
         (int)lcs_bound_create(2, 2, 20, &o, &h));
  printf("handle %s\n", h == NULL ? "null" : "set");
  printf("last_error %d\n", (int)(strlen(lcs_bound_last_error()) > 0));
  printf("null %d %d\n", (int)lcs_bound_iterate(NULL, 1), (int)lcs_bound_orbit_size(NULL, &n_orbit));
  lcs_bound_destroy(NULL);
  return 0;
}
"""

WANT = """defaults 0 0 0 44 1
errstr ok|no kernel for this shape or mode
create 1 1 1
handle null
last_error 1
null 1 1
"""


@pytest.fixture(scope="module")
def lib_dir():
    from paper_2407_10925_gb300 import build

    return os.path.dirname(build.build())


@pytest.mark.parametrize("compiler,std", [("gcc", "-std=c11"), ("g++", "-std=c++17")])
def test_header_compiles_links_and_runs(tmp_path, lib_dir, compiler, std):
    cc = shutil.which(compiler)
    if cc is None:
        pytest.skip(f"{compiler} not installed")
    src = tmp_path / ("prog.c" if compiler == "gcc" else "prog.cpp")
    src.write_text(PROGRAM)
    exe = tmp_path / "prog"
    cmd = [cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", f"-I{os.path.join(ROOT, 'include')}", str(src),
           f"-L{lib_dir}", "-llcs_bound", f"-Wl,-rpath,{lib_dir}", "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout == WANT


def test_struct_layouts_match_the_binding(tmp_path):
    """Every struct the binding mirrors has the C compiler's size and field
    offsets, so no field is read from the wrong place."""
    import ctypes

    from paper_2407_10925_gb300 import binding

    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc not installed")
    structs = [binding.lcs_bound_opts, binding.lcs_bound_report, binding.lcs_bound_stats_t,
               binding.lcs_bound_check_record, binding.lcs_bound_batch_info_t]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "lcs_bound.h"', "int main(void) {"]
    want = []
    for st in structs:
        name = st.__name__
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        want.append(f"{name} {ctypes.sizeof(st)}")
        for field, _ in st._fields_:
            lines.append(f'  printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
            want.append(f"{name}.{field} {getattr(st, field).offset}")
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Werror", f"-I{os.path.join(ROOT, 'include')}", str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0
    assert r.stdout.split("\n")[:-1] == want
