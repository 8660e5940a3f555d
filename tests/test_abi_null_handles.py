"""Every entry point of include/lc_api.h that takes a handle (context,
operator or batch) answers a null handle with an error code -- or, for the
destroy calls, as a no-op -- without touching a GPU (CPU only).  The calls
run in a child process, so a null dereference shows as a failed test naming
the entry point rather than ending the test run."""
import glob
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HANDLE = re.compile(r"^\s*(const\s+)?lc_(ctx|op|batch)\s*\*\s*\w+\s*$")


def prototypes():
    """(name, [parameter declarations]) of every LC_EXPORT int function."""
    out = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", " ", open(h).read(), flags=re.S)
        for m in re.finditer(r"LC_EXPORT\s+int\s+(lc_\w+)\s*\(([^)]*)\)\s*;", text):
            params = [p.strip() for p in m.group(2).replace("\n", " ").split(",")]
            out.append((m.group(1), params))
    return out


def handle_calls():
    return [(n, p) for n, p in prototypes() if p and HANDLE.match(p[0])]


CHILD = r"""
import ctypes as C, re, sys
sys.path.insert(0, {root!r})
import paper_2001_01158_gb300 as lcg
L = lcg.lib()
for name, params in {calls!r}:
    types, args = [], []
    for p in params:
        if "*" in p or "[" in p:
            types.append(C.c_void_p); args.append(None)
        elif re.match(r"^(const\s+)?double\b", p):
            types.append(C.c_double); args.append(0.0)
        elif re.match(r"^(const\s+)?int64_t\b", p):
            types.append(C.c_int64); args.append(0)
        else:
            types.append(C.c_int32); args.append(0)
    f = getattr(L, name)
    f.argtypes, f.restype = types, C.c_int
    print(name, f(*args), flush=True)
"""


def test_prototypes_parsed():
    names = [n for n, _ in handle_calls()]
    for required in ("lc_mark_residual", "lc_extract", "lc_pcg_solve", "lc_solve_local_then_global",
                     "lc_batch_solve", "lc_op_destroy", "lc_ctx_destroy"):
        assert required in names


def test_null_handles_are_refused():
    calls = handle_calls()
    code = CHILD.format(root=ROOT, calls=calls)
    p = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    lines = dict(ln.split() for ln in p.stdout.splitlines() if ln.startswith("lc_"))
    done = [n for n, _ in calls if n in lines]
    assert p.returncode == 0 and len(done) == len(calls), (
        f"stopped after {done[-1:] or 'nothing'}: {p.stderr[-500:]}")
    for name, rc in lines.items():
        if name.endswith("_destroy"):
            assert rc == "0", (name, rc)      # destroying a null handle is a no-op
        else:
            assert rc == "1", (name, rc)      # LC_ERR_INVALID_ARG
