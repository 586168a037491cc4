"""Static checks on the CUDA sources (CPU only).

A kernel launched as a programmatic dependent (launch_pdl) may start while the
previous kernel of its stream is still running; it is race-free only if it waits
(pdl_wait) before its first memory access.  These tests find every such launch and
require pdl_wait() to be the first statement of the launched kernel."""
import glob
import os
import re

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2602_22625_gb300", "csrc")


def sources():
    out = {}
    for p in sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))):
        with open(p) as f:
            out[os.path.basename(p)] = f.read()
    return out


def kernel_body_start(src, name):
    """Text of kernel `name`'s body from its opening brace (None if not defined here)."""
    m = re.search(r"__global__\s+void\s+(?:__launch_bounds__\((?:[^()]|\([^()]*\))*\)\s+)?" + re.escape(name) + r"\s*\(",
                  src)
    if not m:
        return None
    depth, i = 0, m.end() - 1
    while i < len(src):   # skip the parameter list
        if src[i] == "(":
            depth += 1
        elif src[i] == ")":
            depth -= 1
            if depth == 0:
                break
        i += 1
    j = src.index("{", i)
    return src[j + 1:]


def first_statement(body):
    body = re.sub(r"//[^\n]*", "", body)
    return body.strip().split(";", 1)[0].strip()


def test_pdl_launches_found():
    names = set()
    for src in sources().values():
        names |= set(re.findall(r"launch_pdl\(\s*(\w+)\s*(?:<[^>]*>)?\s*,", src))
    names.discard("kernel")   # the helper's own parameter
    assert {"k_count", "k_colscan", "k_tilescan", "k_scatter", "k_finalize", "k_adam8", "k_adam",
            "k_step_inc", "k_item_order", "k_fwd", "k_bwd"} <= names


def violations(srcs):
    names = set()
    for src in srcs.values():
        names |= set(re.findall(r"launch_pdl\(\s*(\w+)\s*(?:<[^>]*>)?\s*,", src))
    names.discard("kernel")
    bad = []
    for name in sorted(names):
        bodies = [b for b in (kernel_body_start(s, name) for s in srcs.values()) if b is not None]
        if len(bodies) != 1:
            bad.append(f"{name}: {len(bodies)} definitions")
        elif first_statement(bodies[0]) != "pdl_wait()":
            bad.append(f"{name} starts with {first_statement(bodies[0])!r}")
    return bad


def test_every_dependent_kernel_waits_first():
    assert violations(sources()) == []


def test_the_check_catches_a_missing_wait():
    srcs = sources()
    bad = dict(srcs)
    bad["bin.cu"] = srcs["bin.cu"].replace("const DevStatus *status) {\n    pdl_wait();",
                                           "const DevStatus *status) {\n", 1)
    assert bad["bin.cu"] != srcs["bin.cu"]
    assert any(v.startswith("k_scatter") for v in violations(bad))


def test_pdl_helpers_are_the_documented_ptx():
    srcs = sources()
    assert 'asm volatile("griddepcontrol.wait;" ::: "memory")' in srcs["compositor.cuh"]
    assert "cudaLaunchAttributeProgrammaticStreamSerialization" in srcs["dbmp_internal.cuh"]
