"""The boundary from C: include/vfisv.h compiles as plain C11 and as C++17,
and a C program linked against libvfisv.so calls the entry points that need
no device (the default configuration, the error strings, argument checks that
return before any device work).  Runs without a GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "vfisv.h"

int main(void) {
  vfisv_config c;
  memset(&c, 0xff, sizeof c);
  vfisv_config_default(&c);
  if (c.max_iter != 50 || c.free_mask != 0x1FFu || c.conv_rtol != 1e-4 || c.conv_eps != 1.0 ||
      c.eps0 != 1.0 || c.restarts != 0 || c.seed != 0 || c.hess_reuse != 0.0 ||
      c.wfa_pol != 0.0 || c.fast_solve != 0)
    return 1;
  for (int e = VFISV_OK; e >= VFISV_E_CAPTURE; --e) {
    const char* s = vfisv_strerror(e);
    if (!s || !*s || !strcmp(s, vfisv_strerror(-1000))) return 2;
  }
  if (vfisv_create(NULL, 0) != VFISV_E_ARG) return 3;
  if (vfisv_check(NULL, NULL) != VFISV_E_ARG) return 4;
  const vfisv_line ln = {6173.34, 2.5, 1.0};
  float buf[24] = {0};
  int32_t ibuf[1] = {0};
  /* otherwise well-formed arguments with a null handle: rejected before any
   * device work */
  if (vfisv_invert(NULL, buf, buf, 0, buf, 6, buf, 1, &ln, NULL, &c, 1, buf, buf, ibuf, ibuf,
                   NULL, NULL) != VFISV_E_ARG)
    return 5;
  printf("%s\n", vfisv_strerror(VFISV_E_UNSUPPORTED));
  return 0;
}
"""


def _need(tool):
    if shutil.which(tool) is None:
        pytest.skip(f"{tool} not installed")


@pytest.mark.parametrize("lang,std,compiler", [("c", "c11", "gcc"), ("c++", "c++17", "g++")])
def test_header_compiles(tmp_path, lang, std, compiler):
    _need(compiler)
    src = tmp_path / ("h.c" if lang == "c" else "h.cpp")
    src.write_text('#include "vfisv.h"\nint vfisv_header_only_check;\n')
    r = subprocess.run([compiler, f"-std={std}", "-Wall", "-Wextra", "-Werror", "-pedantic",
                        "-fsyntax-only", f"-I{INC}", str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_program_links_and_calls_host_entry_points(tmp_path):
    _need("gcc")
    from paper_0901_2702_gb300 import build
    lib = build.build()
    src = tmp_path / "use.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "use"
    libdir = os.path.dirname(lib)
    name = os.path.basename(lib)
    assert name.startswith("lib") and name.endswith(".so")
    r = subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", f"-I{INC}", str(src), "-o", str(exe),
                        f"-L{libdir}", f"-l{name[3:-3]}", f"-Wl,-rpath,{libdir}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.strip() == "number of filters not compiled into this kernel"
