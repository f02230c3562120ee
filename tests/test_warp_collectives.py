"""Static check of the CUDA sources: warp-collective intrinsics are never evaluated
conditionally within an expression.

A full-mask `__ballot_sync` / `__any_sync` / `__shfl_sync` / `__syncwarp` must be reached by
every lane of the mask.  Placed on the right of `&&`, `||` or `?`, C++ evaluation skips it in
the lanes whose left operand already decides the result, and the lanes that do reach it wait
for the others indefinitely.  The kernels take their warp votes on values every lane has
already computed; this test keeps it that way (per source line, comments excluded).
"""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2311_13081_gb300", "csrc")

SHORT_CIRCUIT = re.compile(r"(&&|\|\||\?)")
COLLECTIVE = re.compile(r"__(shfl\w*|ballot|any|all|match\w*|reduce\w*)_sync\s*\(|__syncwarp\s*\(")


def conditional_collectives(lines):
    """(line number, code) of every line where a warp-collective intrinsic follows a
    short-circuit or conditional operator."""
    hits = []
    for n, line in enumerate(lines, 1):
        code = line.split("//")[0]
        for m in SHORT_CIRCUIT.finditer(code):
            if COLLECTIVE.search(code[m.end():]):
                hits.append((n, code.strip()))
                break
    return hits


def test_checker_flags_a_vote_behind_a_short_circuit():
    bad = ["const bool fill = need && (tt == 0 || __popc(__ballot_sync(0xffffffffu, need)) >= 8);",
           "float v = lane < 4 ? __shfl_sync(0xffffffffu, x, 0) : 0.0f;",
           "if (ok || __any_sync(0xffffffffu, flag)) return;"]
    good = ["if (__any_sync(0xffffffffu, now || fill)) {",
            "if (__any_sync(0xffffffffu, bad) && lane == 0 && active) atomicCAS(p, 0, 3);",
            "const unsigned m = __ballot_sync(0xffffffffu, need);  // a || b ? c : d",
            "acc = gsum(acc) + b1[j];"]
    assert [n for n, _ in conditional_collectives(bad)] == [1, 2, 3]
    assert conditional_collectives(good) == []


def test_no_warp_collective_is_evaluated_conditionally():
    files = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh")))
    assert files, "no CUDA sources found"
    found = []
    for f in files:
        with open(f) as fh:
            for n, code in conditional_collectives(fh.read().splitlines()):
                found.append(f"{os.path.basename(f)}:{n}: {code}")
    assert not found, "warp-collective intrinsic behind a short-circuit:\n" + "\n".join(found)
