"""The C ABI used from a C program (no Python in between): the header compiles as C99 and C++,
the program links against the library, and the host-side checks answer through the ABI (no GPU:
every call below is rejected or answered before any device work)."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "pt.h"

int main(void) {
  pt_grid g;
  pt_coeff k;
  pt_options o;
  pt_problem* p = NULL;
  size_t bytes = 0;
  double steps[8] = {0.125, 0.125, 0.125, 0.125, 0.125, 0.125, 0.125, 0.5};
  pt_status s;
  memset(&g, 0, sizeof g);
  memset(&k, 0, sizeof k);
  memset(&o, 0, sizeof o);
  g.dim = 2;
  g.n[0] = g.n[1] = 6;              /* n + 1 = 7 is not a power of two */
  k.a0 = 1.0;
  s = pt_problem_create(&g, 8, 1.0, &k, NULL, 0, NULL, 0, &o, &p);
  printf("grid %s %d\n", pt_status_string(s), p == NULL);
  g.n[0] = g.n[1] = 7;
  o.tau_steps = steps;              /* sums to 1.375, not T = 1 */
  s = pt_problem_create(&g, 8, 1.0, &k, NULL, 0, NULL, 0, &o, &p);
  printf("steps %s %d\n", pt_status_string(s), strlen(pt_last_error()) > 0);
  o.tau_steps = NULL;
  s = pt_problem_estimate_bytes(&g, 8, &o, &bytes);
  printf("estimate %s %d\n", pt_status_string(s), bytes > 0);
  s = pt_solve(NULL, 1e-8, 10, NULL, 0, NULL, NULL);
  printf("solve %s\n", pt_status_string(s));
  pt_problem_destroy(NULL);
  return 0;
}
"""


@pytest.fixture(scope="module")
def library():
    from paper_1802_08126_gb300 import build
    build.build()
    return os.path.join(ROOT, "paper_1802_08126_gb300", "_lib")


@pytest.mark.parametrize("lang", ["c", "c++"])
def test_header_compiles(tmp_path, lang):
    src = tmp_path / ("h.c" if lang == "c" else "h.cpp")
    src.write_text('#include "pt.h"\nint main(void) { return (int)PT_OK; }\n')
    cc = ["gcc", "-std=c99"] if lang == "c" else ["g++", "-std=c++17"]
    r = subprocess.run(cc + ["-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                             "-fsyntax-only", str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_program_links_and_gets_host_side_answers(tmp_path, library):
    src = tmp_path / "consumer.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "consumer"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-L", library, "-lptuzawa", "-Wl,-rpath," + library, "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.split("\n")[:4] == ["grid PT_EINVAL 1", "steps PT_EINVAL 1", "estimate PT_OK 1",
                                        "solve PT_EINVAL"]
