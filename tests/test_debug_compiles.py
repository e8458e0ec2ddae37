"""The GBFFT_DEBUG form of the kernels compiles (no GPU needed): one length's
translation unit with -DGBFFT_DEBUG, so the checked and poisoned exchange
code cannot rot between GPU runs (the GPU tests build and run the whole
debug library)."""
import os
import shutil
import subprocess

import pytest

from paper_2203_09384_gb300 import build as gbuild


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_debug_kernels_compile(tmp_path):
    src = os.path.join(gbuild.CSRC, "fft_kernels.cu")
    cmd = [gbuild.nvcc(), *gbuild.ARCH, *gbuild.CFLAGS, "-DGBFFT_DEBUG", "-DGBFFT_LOG2N=8", "-c", src,
           "-o", str(tmp_path / "k.o")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
