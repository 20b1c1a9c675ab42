"""include/hgm.h is a plain C header: a C99 program compiles against it with every warning an error,
links libhgm.so and gets the paper's defaults and the host-side argument checks without a GPU; the
header also compiles as C++."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")

C_PROGRAM = r"""
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "hgm.h"

int main(void)
{
    hgm_params p;
    hgm_model *m = NULL;
    hgm_scene *s = NULL;
    float xy[4] = {0.0f, 0.0f, 1.0f, 1.0f};
    int32_t t[2] = {0, 1};
    float f[8] = {0.0f};
    int32_t n = 0, first = 0;

    hgm_default_params(&p);
    if (!(p.lambda1 == 0.6f && p.lambda2 == 0.2f && p.lambda3 == 5.0f && p.T == 10 && p.window == 3 &&
          p.K == 64))
        return 1;
    if (p.prune != NULL || p.keep != 8 || p.refine != 0 || !(p.dummy_cost < 0.0f) || p.precision != 0)
        return 2;
    if (hgm_create_model(xy, t, f, 2, 4, NULL, &m) != HGM_EINVAL || m != NULL)
        return 3;
    if (strstr(hgm_last_error(), "M >= 3") == NULL)
        return 4;
    if (hgm_create_scene(xy, t, f, -1, 4, 0, NULL, &s) != HGM_EINVAL || s != NULL)
        return 5;
    p.K = 0;
    if (hgm_offsets(NULL, NULL, &p, &n, &first) != HGM_EINVAL)
        return 6;
    hgm_default_params(&p);
    p.K = 100;
    if (hgm_offsets(NULL, NULL, &p, &n, &first) != HGM_EUNSUPPORTED)
        return 7;
    hgm_destroy(NULL);
    puts("ok");
    return 0;
}
"""


@pytest.fixture(scope="module")
def libdir():
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    from paper_1505_00581_gb300 import build
    return os.path.dirname(build.build())


def test_c99_program_links_and_checks_arguments(libdir, tmp_path):
    src = tmp_path / "use_hgm.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "use_hgm"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", INCLUDE, str(src),
                    "-L", libdir, "-lhgm", f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True,
                   capture_output=True, text=True)
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0 and run.stdout.strip() == "ok", (run.returncode, run.stdout, run.stderr)


def test_header_compiles_as_cxx(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("needs g++")
    src = tmp_path / "use_hgm.cpp"
    src.write_text('#include "hgm.h"\nint main() { hgm_params p; hgm_default_params(&p); return p.K == 64 ? 0 : 1; }\n')
    subprocess.run(["g++", "-std=c++17", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-I", INCLUDE,
                    str(src)], check=True, capture_output=True, text=True)
