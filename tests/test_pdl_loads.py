"""Source check of the kernels launched with programmatic stream serialisation.

Such a kernel starts while the previous kernel of the stream still runs and waits for it with
griddepcontrol.wait (griddep_wait()).  A load through a const __restrict__ pointer may be compiled
as invariant over the kernel and issued before that wait, i.e. before the previous kernel has
written the data.  So in every kernel that calls griddep_wait(), only the tables that stay fixed
while such kernels run (the coarse operator, its scales, the mass shifts, the rhs mask) may be
declared __restrict__; the vectors are read through plain pointers.
"""
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_0912_2186_b300", "csrc")

# parameters that may stay __restrict__: read-only tables, fixed while the waiting kernels run,
# and the error word (only ever written, by atomicExch)
FIXED_TABLES = {"A16", "sA", "shift", "active", "err"}


def _kernels(src):
    """(name, parameter text, body text) of every __global__ function definition."""
    out = []
    for m in re.finditer(r"__global__\s+void\s+(?:__launch_bounds__\([^)]*\)\s*)?(\w+)\s*\(", src):
        i = m.end()
        depth = 1
        while depth:
            depth += {"(": 1, ")": -1}.get(src[i], 0)
            i += 1
        params = src[m.end():i - 1]
        j = src.index("{", i)
        if src[i:j].strip():  # a declaration, not a definition
            continue
        k, depth = j + 1, 1
        while depth:
            depth += {"{": 1, "}": -1}.get(src[k], 0)
            k += 1
        out.append((m.group(1), params, src[j:k]))
    return out


def _waiting_kernels():
    found = []
    for f in sorted(os.listdir(CSRC)):
        if f.endswith(".cu"):
            with open(os.path.join(CSRC, f)) as fh:
                src = fh.read()
            found += [(f, *k) for k in _kernels(src) if "griddep_wait()" in k[2]]
    return found


def test_waiting_kernels_exist():
    names = {k[1] for k in _waiting_kernels()}
    assert {"k_cg_update", "k_cg_xpay", "k_coarse_apply_mma"} <= names


def test_no_restrict_vectors_in_waiting_kernels():
    for f, name, params, body in _waiting_kernels():
        for p in params.split(","):
            if "__restrict__" in p:
                pname = re.findall(r"(\w+)\s*$", p.strip())[0]
                assert pname in FIXED_TABLES, f"{f}: {name} takes its parameter {pname} as __restrict__"
        assert "__restrict__" not in body, f"{f}: {name} declares a __restrict__ pointer in its body"


def test_the_check_sees_a_restrict_vector():
    # the scan itself: a waiting kernel with a restrict vector parameter is reported
    src = """__global__ void k_demo(const float* __restrict__ v, int n) {
      griddep_wait();
      float t = v[threadIdx.x];
    }"""
    (name, params, body), = _kernels(src)
    assert name == "k_demo" and "griddep_wait()" in body
    assert any("__restrict__" in p and p.strip().endswith("v") for p in params.split(","))


def test_programmatic_launches_only_of_waiting_kernels():
    # a kernel launched with programmatic stream serialisation that never waits could run
    # entirely before its predecessor has finished: every such launch is of a waiting kernel
    waiting = {k[1] for k in _waiting_kernels()}
    launched = set()
    for f in sorted(os.listdir(CSRC)):
        if f.endswith(".cu"):
            with open(os.path.join(CSRC, f)) as fh:
                src = fh.read()
            if "programmaticStreamSerializationAllowed" in src:
                launched |= set(re.findall(r"cudaLaunchKernelEx\(\s*&\w+\s*,\s*(\w+)", src))
    assert launched, "no programmatic launches found"
    assert launched <= waiting, f"launched with programmatic serialisation without a wait: {launched - waiting}"
