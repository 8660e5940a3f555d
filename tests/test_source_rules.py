"""Rules the CUDA sources keep, checked by reading them (CPU):

- every loop that waits on memory another block writes (an acquire load of
  the grid-barrier counter) reads the clock inside its body and gives up
  after a limit, so no wait can hang the GPU;
- device code ends a failure by recording a status and returning, never by
  trapping: no __trap, no device assert, no trap instruction."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SOURCES = sorted(glob.glob(os.path.join(ROOT, "paper_2001_01158_gb300", "csrc", "*.cu")) +
                 glob.glob(os.path.join(ROOT, "paper_2001_01158_gb300", "csrc", "*.cuh")))


def _code(path):
    """The source without comments (line structure kept)."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", lambda m: "\n" * m.group(0).count("\n"), text, flags=re.S)
    return re.sub(r"//[^\n]*", "", text)


def _loop_body(code, start):
    """The text of the braced body that follows position `start`."""
    i = code.index("{", start)
    depth = 0
    for j in range(i, len(code)):
        depth += {"{": 1, "}": -1}.get(code[j], 0)
        if depth == 0:
            return code[i:j + 1]
    raise AssertionError("unbalanced braces")


def test_sources_found():
    assert len(SOURCES) >= 10


def test_every_spin_wait_is_bounded():
    waits = 0
    for path in SOURCES:
        code = _code(path)
        for m in re.finditer(r"\bwhile\s*\(([^;{]*ld_acquire[^;{]*)\)", code):
            body = _loop_body(code, m.end())
            waits += 1
            assert "clock64()" in body and "break" in body, f"{os.path.basename(path)}: unbounded wait {m.group(0)}"
    assert waits >= 2   # the grid barrier and the pipelined solve's fused barrier


def test_no_trap_or_device_assert():
    for path in SOURCES:
        code = _code(path)
        name = os.path.basename(path)
        assert "__trap" not in code, name
        assert not re.search(r"\btrap\s*;", code), name
        assert not re.search(r"(?<![_a-z])assert\s*\(", code), name
