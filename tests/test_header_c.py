"""The public header is plain C: a C99 program compiles against
include/gbfft.h, links libgbfft.so and gets the documented argument checks
(no GPU needed for these calls), and its plan-info struct lays out as the
ctypes binding reads it."""
import ctypes
import os
import subprocess

import pytest

from paper_2203_09384_gb300 import _abi

C_SRC = r"""
#include <stdio.h>
#include <string.h>
#include "gbfft.h"

int main(void) {
    fft_plan_t plan = NULL;
    float w[2];
    int bad = 0;
    bad |= fft_validate(1024, 8, FFT_FORWARD, FFT_C64, 0u) != FFT_OK;
    bad |= fft_validate(1000, 8, FFT_FORWARD, FFT_C64, 0u) != FFT_ERR_INVALID_SIZE;
    bad |= fft_validate(1024, -1, FFT_FORWARD, FFT_C64, 0u) != FFT_ERR_INVALID_VALUE;
    bad |= fft_validate(64, 1, FFT_INVERSE, FFT_C64, FFT_FLAG_UNNORMALIZED | FFT_FLAG_VARIANT(0)) != FFT_OK;
    bad |= fft_plan_create(4096, 1, FFT_FORWARD, FFT_C64, &plan) != FFT_ERR_INVALID_SIZE;
    bad |= plan != NULL;
    bad |= fft_plan_destroy(NULL) != FFT_OK;
    bad |= fft_execute(NULL, NULL, NULL, NULL) != FFT_ERR_INVALID_VALUE;
    bad |= fft_variant_count(2048) < 1;
    bad |= fft_variant_count(3) != 0;
    fft_twiddle_fp32(16, 4, w);
    bad |= !(w[0] == 0.0f && w[1] == -1.0f);
    bad |= strlen(fft_status_string(FFT_ERR_MISALIGNED)) == 0;
    printf("%s %s\n", fft_version(), bad ? "FAIL" : "OK");
    return bad;
}
"""


def test_header_is_c99_and_links(tmp_path):
    lib = _abi.lib()  # builds must exist
    assert lib
    src = tmp_path / "abi_check.c"
    src.write_text(C_SRC)
    exe = tmp_path / "abi_check"
    inc = os.path.dirname(_abi.HEADER)
    libdir = os.path.dirname(_abi.LIB_PATH)
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", inc, str(src), "-o", str(exe),
           "-L", libdir, "-lgbfft", f"-Wl,-rpath,{libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "cannot find -lgbfft" in r.stderr:
        pytest.skip("libgbfft.so not linkable by name")
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and out.stdout.strip().endswith("OK"), out.stdout + out.stderr


def test_plan_info_layout_matches_ctypes(tmp_path):
    """The ctypes PlanInfo the binding reads must lay out exactly like the
    header's fft_plan_info_t (size and every field offset, as gcc sees it)."""
    fields = [name for name, _ in _abi.PlanInfo._fields_]
    body = "\n".join(f'    printf("{f} %zu\\n", offsetof(fft_plan_info_t, {f}));' for f in fields)
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "gbfft.h"\nint main(void) {\n'
                   '    printf("sizeof %zu\\n", sizeof(fft_plan_info_t));\n' + body + "\n    return 0;\n}\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(_abi.HEADER), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        timeout=60).stdout.splitlines())
    assert int(got["sizeof"]) == ctypes.sizeof(_abi.PlanInfo)
    for f in fields:
        assert int(got[f]) == getattr(_abi.PlanInfo, f).offset, f
