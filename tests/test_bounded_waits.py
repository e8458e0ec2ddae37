"""Device-side waits stay bounded (CPU lint of the kernel sources).

Every spin on an mbarrier goes through ``mbar_wait_bounded``, which gives up
after the plan's wall-time limit and lets the caller record FFT_ERR_TIMEOUT;
the raw ``mbarrier.try_wait`` forms appear only inside the two helpers it
calls.  The kernels contain no trap or device assert, and every open-ended
loop is one of the reviewed ones below, whose exit does not depend on another
block or another kernel.  A new wait or loop has to be reviewed and listed
here before this test passes.
"""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2203_09384_gb300", "csrc")

# open-ended loops and why each ends
REVIEWED_LOOPS = {
    "mbar_wait_bounded": "returns on completion or once the wall-time limit has passed",
    "fft_ragged_kernel": "work loops: the item index only grows and the loop ends past n_items",
}


def sources():
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(CSRC, name)) as f:
                yield name, f.read()


KEYWORDS = {"if", "for", "while", "switch", "catch", "return", "sizeof", "constexpr", "__launch_bounds__"}


def blank(text: str, strings: bool = True) -> str:
    """Comments (and, with `strings`, the insides of string/char literals)
    replaced by spaces, positions kept, so braces in inline-PTX strings do not
    count as code."""
    out = list(text)
    i, n = 0, len(text)
    while i < n:
        if text.startswith("//", i):
            j = text.find("\n", i)
            j = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            j = n if j < 0 else j + 2
        elif text[i] in "\"'":
            j = i + 1
            while j < n and text[j] != text[i]:
                j += 2 if text[j] == "\\" else 1
            j += 1
            if strings:
                for k in range(i + 1, min(j - 1, n)):
                    out[k] = " " if text[k] != "\n" else "\n"
            i = j
            continue
        else:
            i += 1
            continue
        for k in range(i, j):
            out[k] = " " if text[k] != "\n" else "\n"
        i = j
    return "".join(out)


def function_spans(code: str):
    """(name, body start, body end) of every function body in blanked code."""
    spans = []
    head = re.compile(r"\b(\w+)\s*\([^;{}]*\)\s*(?:const\s*)?\{")
    pos = 0
    while True:
        m = head.search(code, pos)
        if not m:
            break
        pos = m.start(1) + len(m.group(1))  # overlapping: a header may follow __launch_bounds__(...)
        if m.group(1) in KEYWORDS:
            continue
        depth, k = 0, m.end() - 1
        while k < len(code):
            depth += {"{": 1, "}": -1}.get(code[k], 0)
            if depth == 0:
                break
            k += 1
        spans.append((m.group(1), m.end() - 1, k))
    return spans


def enclosing_function(code: str, pos: int) -> str:
    inside = [(e - b, name) for name, b, e in function_spans(code) if b < pos < e]
    return min(inside)[1] if inside else ""


def raw_wait_sites(text: str):
    """(function, position) of every mbarrier try_wait/test_wait in code or
    inline-PTX strings (comments ignored)."""
    code, with_strings = blank(text), blank(text, strings=False)
    return [(enclosing_function(code, m.start()), m.start())
            for m in re.finditer(r"mbarrier\.(try_wait|test_wait)", with_strings)]


def open_loops(text: str):
    code = blank(text)
    return [enclosing_function(code, m.start()) for m in re.finditer(r"for\s*\(\s*;\s*;\s*\)", code)]


def test_raw_mbarrier_waits_only_in_the_helpers():
    for name, text in sources():
        for fn, _ in raw_wait_sites(text):
            assert fn in {"mbar_try_wait", "mbar_try_wait_suspend"}, (name, fn)


def test_helpers_are_called_only_by_the_bounded_wait():
    for name, text in sources():
        code = blank(text)
        for m in re.finditer(r"\bmbar_try_wait(_suspend)?\s*\(", code):
            line_start = code.rfind("\n", 0, m.start()) + 1
            if "__device__" in code[line_start:m.start()]:
                continue  # the definition itself
            assert enclosing_function(code, m.start()) == "mbar_wait_bounded", (name, m.group(0))


def test_no_trap_or_device_assert():
    for name, text in sources():
        code = blank(text)
        assert "__trap" not in code and not re.search(r"\btrap\s*;", code), name
        assert not re.search(r"\bassert\s*\(", code), name


def test_open_ended_loops_are_reviewed():
    for name, text in sources():
        code = blank(text)
        assert not re.search(r"while\s*\(\s*(true|1)\s*\)", code), name
        for fn in open_loops(text):
            assert fn in REVIEWED_LOOPS, (name, fn)


PLANTED = r"""
// mbarrier.try_wait in a comment does not count
__device__ bool mbar_try_wait(uint64_t* b, uint32_t p) {
    asm volatile("{ .reg .pred q; mbarrier.try_wait.parity.shared::cta.b64 q, [%0], %1; }" :: "l"(b), "r"(p));
    return true;
}
template <int V>
__global__ void __launch_bounds__(128, 1) spin_kernel(int* flag) {
    if constexpr (V > 0) {
        for (;;) {
            asm volatile("mbarrier.try_wait.parity.shared::cta.b64 p, [%0], 0;" :: "r"(0));
        }
    }
}
"""


def test_the_checks_see_a_planted_unbounded_wait():
    assert [fn for fn, _ in raw_wait_sites(PLANTED)] == ["mbar_try_wait", "spin_kernel"]
    assert open_loops(PLANTED) == ["spin_kernel"]
