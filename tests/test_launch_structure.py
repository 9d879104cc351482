"""Source-level check of the programmatic-dependent-launch rule in the CUDA sources: a kernel that
the library launches through `launch_dep` may start while the kernel before it in the stream is
still running, so its body must execute `pdl_wait()` (griddepcontrol.wait) before it touches
global memory that kernel writes.  This test finds every kernel passed to `launch_dep` and checks
that each of its definitions calls `pdl_wait()` (where in the body is left to review: the
order-7 kernels issue their first geometric-factor copy, which nothing in the solve writes,
before waiting)."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2210_03179_gb300", "csrc")


def _sources():
    out = {}
    for p in sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))):
        out[os.path.basename(p)] = open(p).read()
    return out


def _kernel_bodies(name, text):
    """Bodies of the __global__ functions called `name` in `text` (every overload/template)."""
    bodies = []
    for m in re.finditer(r"__global__[^;{]*?\b" + re.escape(name) + r"\s*\(", text):
        i = text.find("{", m.end())
        depth, j = 0, i
        while True:
            if text[j] == "{":
                depth += 1
            elif text[j] == "}":
                depth -= 1
                if depth == 0:
                    break
            j += 1
        bodies.append(text[i + 1:j])
    return bodies


def test_every_dependent_launch_waits_for_its_predecessor():
    src = _sources()
    launched = set()
    for text in src.values():
        launched.update(re.findall(r"launch_dep\(\s*(k_[A-Za-z0-9_]+)", text))
    assert len(launched) >= 25          # the solve path's kernels
    for name in sorted(launched):
        bodies = [b for text in src.values() for b in _kernel_bodies(name, text)]
        assert bodies, f"no __global__ definition found for {name}"
        for body in bodies:
            assert "pdl_wait();" in body, f"{name} is launched as a dependent but never waits"


def test_only_the_helper_sets_the_programmatic_attribute():
    # every programmatic launch goes through launch_dep, which honours g_pdl and stream capture
    src = _sources()
    hits = [f for f, t in src.items() if "cudaLaunchAttributeProgrammaticStreamSerialization" in t]
    assert hits == ["common.cuh"], hits
