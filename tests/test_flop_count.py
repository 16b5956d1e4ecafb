"""The M2L flop count the benchmark's roofline uses (bench.m2l_flops), checked
against the arithmetic the generator writes into the FP32 M2L kernel
(csrc/gen_m2l.py): the swap steps and the z-translation of Sec. 2.4, with a
linear combination of t terms counted as t multiplies and t - 1 adds. The
count takes the swap blocks' non-zero entries by parity; the generator also
drops the few entries that vanish exactly, so the two may differ by a fraction
of a percent, never more. CPU only."""
import os
import re
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GEN = os.path.join(ROOT, "paper_2012_02207_gb300", "csrc", "gen_m2l.py")


def lin(t):
    return 2 * t - 1 if t > 0 else 0


def generated_flops(p):
    out = subprocess.run([sys.executable, GEN, str(p)], capture_output=True, text=True, check=True).stdout

    def body(name):
        i = out.index(f"void {name}<{p}>(")
        return out[i:out.index("\n}\n", i)]

    swaps = {}
    for name in ("swap_lit", "swap_lit_z"):
        swaps[name] = sum(lin(line.count(" * ")) for line in body(name).splitlines()
                          if re.match(r"\s*a\[\d+\] = ", line))
    trans = 0
    for line in body("ztrans_lit").splitlines():
        if re.match(r"\s*up\[[1-9]\d*\] = ", line):
            trans += 2  # u^k and v^k
        elif re.match(r"\s*const float [ri]\d+ = ", line):
            trans += 1  # u^k times an input
        elif re.match(r"\s*a\[\d+\] = vp", line):
            trans += lin(line[line.index("(") + 1:line.rindex(")")].count(" * ")) + 1  # the sum and its scale
    return swaps, trans


@pytest.mark.parametrize("p", [6, 10, 14])
def test_m2l_flop_count_matches_the_generated_arithmetic(p):
    swaps, trans = generated_flops(p)
    rot = sum(6 + 6 * (p - m + 1) for m in range(1, p + 1))
    rest = bench.m2l_flops(p) - 4 * rot - (p + 1) ** 2  # the swaps and the z-translation
    gen = 3 * swaps["swap_lit"] + swaps["swap_lit_z"] + trans
    assert abs(rest - gen) <= 0.01 * gen, (rest, gen)
    assert gen <= rest  # exact zeros only ever remove terms


def test_m2l_flop_count_at_the_benchmark_order():
    assert bench.m2l_flops(10) == 4923
