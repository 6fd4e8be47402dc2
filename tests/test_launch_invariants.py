"""Source invariants of the programmatic dependent launches (host-only).

Kernels launched with the programmatic-serialization attribute may be
scheduled before the kernel ahead of them on the stream has finished; that
is only correct when the kernel waits (griddepcontrol.wait) before its first
memory access.  Every kernel of the step translation units therefore starts
with grid_dep_sync(), and no launch there bypasses the two launch helpers."""
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2509_10103_gb300", "csrc")
STEP_UNITS = ("kernels.cu", "transforms.cu")


def _kernels(src):
    for m in re.finditer(r"__global__[^{;]*?\b(k_\w+)\s*\(", src):
        body = src.index("{", m.end())
        yield m.group(1), src[body + 1:body + 200]


def test_every_kernel_waits_for_its_predecessor_first():
    n = 0
    for f in STEP_UNITS:
        src = open(os.path.join(CSRC, f)).read()
        for name, head in _kernels(src):
            first = head.strip().split(";")[0].strip()
            assert first == "grid_dep_sync()", f"{f}: {name} does not start with grid_dep_sync()"
            n += 1
    assert n >= 30


def test_no_launch_bypasses_the_helpers():
    for f in STEP_UNITS:
        src = open(os.path.join(CSRC, f)).read()
        assert "<<<" not in src, f"{f} launches a kernel with <<<>>>"
        assert len(re.findall(r"\blaunch_(?:pdl|serial)\(", src)) > 0


def test_the_wait_precedes_the_trigger():
    src = open(os.path.join(CSRC, "dev_common.cuh")).read()
    body = src[src.index("void grid_dep_sync()"):]
    body = body[:body.index("}")]
    assert body.index("griddepcontrol.wait") < body.index("griddepcontrol.launch_dependents")
