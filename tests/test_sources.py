"""Checks on the CUDA sources that need no GPU.

Every kernel launched with launch_pdl() or launch_strided() (programmatic
dependent launch) must call pdl_entry() before its first memory access:
without the grid-dependency wait at its start the kernel could read what the
kernel before it is still writing.  The check is textual: for each kernel name
passed to either, its __global__ definition's body must open with
`pdl_entry();`."""
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2110_06635_gb300", "csrc")


def _sources():
    out = {}
    for fn in sorted(os.listdir(CSRC)):
        if fn.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(CSRC, fn)) as f:
                out[fn] = f.read()
    return out


def _pdl_launched(srcs):
    names = set()
    for fn, s in srcs.items():
        if fn == "launch.h":
            continue
        for m in re.finditer(r"launch_(?:pdl|strided)\(\s*(k_\w+)", s):
            names.add(m.group(1))
    return names


def _body_start(srcs, name):
    """The first statement of kernel `name`'s body, or None if not found."""
    for s in srcs.values():
        m = re.search(r"__global__\s+void[^;{]*?\b" + name + r"\(", s)
        if m is None:
            continue
        # skip the parameter list to its closing parenthesis
        depth, k = 1, m.end()
        while depth:
            depth += {"(": 1, ")": -1}.get(s[k], 0)
            k += 1
        j = s.index("{", k)
        body = s[j + 1:].lstrip()
        return body.split("\n", 1)[0].strip()
    return None


def test_pdl_kernels_wait_first():
    srcs = _sources()
    names = _pdl_launched(srcs)
    assert len(names) >= 15, sorted(names)  # the render, backward, environment and photometric kernels
    for name in sorted(names):
        first = _body_start(srcs, name)
        assert first is not None, f"no __global__ definition of {name}"
        assert first == "pdl_entry();", f"{name} starts with {first!r}"


def test_kernels_with_plain_launches_are_not_pdl_launched():
    """The kernels still launched with <<<...>>> (nearest-neighbour radii, the
    atomic probe) are outside the programmatic chain, which is always safe;
    the check keeps the two lists disjoint so that a kernel is not launched
    both ways by mistake."""
    srcs = _sources()
    names = _pdl_launched(srcs)
    plain = set()
    for s in srcs.values():
        for m in re.finditer(r"\b(k_\w+)(?:<[^<>;]*>)?<<<", s):
            plain.add(m.group(1))
    assert plain, "expected some plain launches"
    assert not (plain & names), sorted(plain & names)
