"""The boundary is a plain C ABI (CPU only, nothing is launched): the header compiles as strict
C99, and a C program linked against libvqnnf.so, with no Python or torch involved, calls the
host-side entry points. It checks the version, the status names, the workspace sizes and the
host-side refusals."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "vqnnf.h"

int main(void)
{
    int bad = 0;
    float f[4];
    uint8_t lab[4];
    vqnnf_filter filt;
    vqnnf_rect r = {0, 0, 2, 2, 1};
    size_t ws;
    if (vqnnf_version() != 100) bad |= 1;
    if (strcmp(vqnnf_status_str(VQNNF_OK), "ok") != 0) bad |= 2;
    ws = vqnnf_workspace_bytes(VQNNF_OP_ASSIGN, 64, 64, 64, 16, 0, 0, 0, VQNNF_PREC_BF16);
    if (ws == 0 || ws % 256 != 0) bad |= 4;
    if (vqnnf_workspace_bytes(VQNNF_OP_ASSIGN, 64, 64, 64, 257, 0, 0, 0, VQNNF_PREC_BF16) != 0) bad |= 8;
    /* refused on the host before anything is enqueued: a null feature map, k = 0 */
    if (vqnnf_assign(NULL, 2, 2, 4, f, 1, VQNNF_PREC_FP32, lab, NULL, NULL, 0, NULL) != VQNNF_EINVAL) bad |= 16;
    if (vqnnf_assign(f, 2, 2, 4, f, 0, VQNNF_PREC_FP32, lab, NULL, NULL, 0, NULL) != VQNNF_EINVAL) bad |= 32;
    /* a rectangle outside a 1 x 1 window */
    filt.n_rects = 1;
    filt.rects = &r;
    filt.w_f = 1.0f;
    filt.area = 4.0f;
    if (vqnnf_filter_responses(lab, 1, 1, 2, &filt, 1, (int32_t *)f, NULL, 0, NULL) != VQNNF_EINVAL) bad |= 64;
    if (vqnnf_selftest_bounded_wait(0, NULL) != VQNNF_EINVAL) bad |= 128;
    printf("bad=%d ws=%zu\n", bad, ws);
    return bad;
}
"""


@pytest.fixture(scope="module")
def libdir():
    from paper_2306_15010_gb300 import build
    build.build()
    return os.path.join(ROOT, "paper_2306_15010_gb300")


def test_header_compiles_as_strict_c99(tmp_path):
    cc = shutil.which("gcc") or pytest.skip("no C compiler")
    src = tmp_path / "h.c"
    src.write_text('#include "vqnnf.h"\nint main(void) { return (int)sizeof(vqnnf_filter) == 0; }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                        os.path.join(ROOT, "include"), "-c", str(src), "-o", str(tmp_path / "h.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_program_calls_the_library(tmp_path, libdir):
    cc = shutil.which("gcc") or pytest.skip("no C compiler")
    src = tmp_path / "p.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "p"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-L", libdir, "-lvqnnf", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("bad=0")
