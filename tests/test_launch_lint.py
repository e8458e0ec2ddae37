"""Programmatic dependent launch protocol (no GPU).

Calls of 2^22 elements and more are launched with programmatic stream
serialization (gbfft::launch_kernel), so a kernel may start before the
previous kernel of its stream has finished.  Every kernel those calls can
launch must therefore begin with pdl_enter(), which waits for the
predecessor before any memory is touched.  This lint reads the CUDA sources
and checks that every __global__ function's body starts with that call, except
the kernels listed below, which are only ever launched plainly.
"""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2203_09384_gb300", "csrc")

# launched only with <<<>>> / cudaLaunchKernel (fft_execute_noalloc's setup)
PLAIN_ONLY = {"noalloc_prepare"}


def first_statements(text: str):
    """(kernel name, first statement of its body) for every __global__
    function of a CUDA source."""
    text = re.sub(r"//[^\n]*", "", text)
    out = []
    for m in re.finditer(r"__global__\b", text):
        head_end = text.index("{", m.end())
        head = text[m.end():head_end]
        names = [n for n in re.findall(r"(\w+)\s*\(", head) if not n.startswith("__")]
        assert names, head
        first = text[head_end + 1:head_end + 400].strip().split(";")[0].strip()
        out.append((names[0], first))
    return out


def _kernels():
    """(file, name, first statement of the body) for every __global__ function."""
    out = []
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cuh")):
            out += [(name, fn, first) for fn, first in first_statements(open(os.path.join(CSRC, name)).read())]
    return out


def test_every_kernel_waits_for_its_predecessor_first():
    ks = _kernels()
    assert len(ks) >= 10, ks  # the FFT kernel families are all found
    for name, fn, first in ks:
        if fn in PLAIN_ONLY:
            continue
        assert first == "pdl_enter()", (name, fn, first)


def test_the_plain_only_kernels_are_launched_plainly():
    """noalloc_prepare must not go through the programmatic launch helper."""
    text = open(os.path.join(CSRC, "fft_noalloc.cu")).read()
    assert "launch_kernel(" not in text
    assert "noalloc_prepare<<<" in text


def test_lint_catches_a_kernel_without_the_wait():
    planted = """
template <class C>
__global__ void __launch_bounds__(128) good_kernel(const float2* in) {
    pdl_enter();
    use(in);
}
__global__ void __launch_bounds__(128, 2) bad_kernel(const float2* in, float2* out) {
    out[threadIdx.x] = in[threadIdx.x];  // reads before waiting for the predecessor
}
"""
    got = dict(first_statements(planted))
    assert got["good_kernel"] == "pdl_enter()"
    assert got["bad_kernel"] != "pdl_enter()"
