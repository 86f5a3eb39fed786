"""Source invariant of the programmatic dependent launches (no GPU needed).

A kernel launched with launch_dep may start before the kernel ahead of it on
the stream has finished; it is correct only if its first statement is
griddep_wait(), which waits for that kernel and makes its writes visible.
This test reads the CUDA sources and checks every kernel passed to
launch_dep for that first statement.
"""
import re
from pathlib import Path

import pytest

CSRC = Path(__file__).resolve().parents[1] / "paper_1412_8502_b300" / "csrc"


def _sources():
    return {p.name: p.read_text() for p in sorted(CSRC.glob("*.cu*")) + sorted(CSRC.glob("*.h"))}


def _launched_with_dep(srcs):
    names = set()
    for text in srcs.values():
        for m in re.finditer(r"\blaunch_dep\(\s*([A-Za-z_][A-Za-z_0-9]*)", text):
            line = text[text.rfind("\n", 0, m.start()) + 1:m.start()]
            if "inline" not in line:             # not the helper's own definition
                names.add(m.group(1))
    return names


def _first_statement(text, name):
    """First statement of the body of __global__ kernel `name` (template
    parameters and launch bounds allowed), or None if it is not defined here."""
    pat = re.compile(r"__global__\s+void\s+(?:__launch_bounds__\([^)]*\)\s*)?" + re.escape(name) + r"\s*\(")
    m = pat.search(text)
    if not m:
        return None
    depth, i = 0, m.end() - 1
    while True:                      # skip the parameter list
        c = text[i]
        depth += c == "("
        depth -= c == ")"
        i += 1
        if depth == 0:
            break
    body = text.index("{", i) + 1
    rest = re.sub(r"//[^\n]*", "", text[body:])
    return rest.strip().split(";")[0].strip() + ";"


@pytest.mark.parametrize("name", sorted(_launched_with_dep(_sources())))
def test_dependent_launches_wait_first(name):
    srcs = _sources()
    found = [s for s in (_first_statement(t, name) for t in srcs.values()) if s is not None]
    assert found, f"{name} is launched with launch_dep but its definition was not found"
    for stmt in found:
        assert stmt == "griddep_wait();", f"{name} starts with {stmt!r}"


def test_some_kernels_use_dependent_launch():
    assert len(_launched_with_dep(_sources())) >= 10
