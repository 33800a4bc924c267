"""Host-side policies of the library, without a GPU (csrc/policy.h compiled
with the host C++ compiler): the segments a lane traces per queue visit, the
growth of an overflowing queue, and the halting radii of a finite speed of
light, which must equal the oracle's (reading R15: the light travel summed in
order since each package's emission)."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1012_2865_gb300 import build

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "policy.h"
using namespace rtg;
int main() {
  const double spp[] = {0.0, -1.0, 3.0, 10.0, 16.1, 49.0, 64.0, 100.0, 1e9};
  for (double v : spp) printf("spi %.17g %d %d\n", v, tuned_segs_per_iter(v), tuned_segs_per_iter(v, false));
  unsigned long long cap = 1ULL << 20; int passes = 1;
  for (int k = 0; k < 8; ++k) {
    const bool ok = grow_after_overflow(3000000ULL, 1ULL << 26, 5, &cap, &passes);
    printf("grow %d %llu %d\n", ok ? 1 : 0, cap, passes);
  }
  const unsigned long long counts[5] = {0, 48, 192, 768, 3072};  // level0 1: 48 roots, 3 levels of splits
  printf("worst %llu %llu\n", queue_worst_case(counts, 1, 5), queue_worst_case(counts, 3, 5));
  std::vector<double> r, n;
  const double cdt[] = {3.5, 3.5, 2.25, 4.0, 3.5, 3.5, 3.5, 3.5, 3.5, 3.5, 3.5, 3.5};
  for (double c : cdt) {
    flight_radii(r, !r.empty(), c, 30.0, n);
    r = n;
    printf("rlim");
    for (double v : r) printf(" %.17g", v);
    printf("\n");
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def output(tmp_path_factory):
    d = tmp_path_factory.mktemp("policy")
    src, exe = d / "policy.cpp", d / "policy"
    src.write_text(PROGRAM)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", os.path.join(build.ROOT, "paper_1012_2865_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True)
    return subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()


def test_segments_per_queue_visit(output):
    got = [int(l.split()[2]) for l in output if l.startswith("spi")]
    assert got == [16, 16, 32, 32, 32, 32, 32, 64, 64]  # with the in-warp hand-off of children
    got = [int(l.split()[3]) for l in output if l.startswith("spi")]
    assert got == [16, 16, 8, 8, 16, 32, 32, 64, 64]  # without (finite speed of light)


def test_queue_grows_then_passes_double(output):
    rows = [tuple(int(x) for x in l.split()[1:]) for l in output if l.startswith("grow")]
    caps = [c for _, c, _ in rows]
    assert rows[0] == (1, 4 << 20, 1)  # x4 while below the limit
    assert caps[:3] == [4 << 20, 16 << 20, 64 << 20] and all(c == 1 << 26 for c in caps[2:])
    passes = [p for _, _, p in rows]
    assert passes[:3] == [1, 1, 1] and passes[3] == 2 and passes[4] == 4 and max(passes) == 5
    assert rows[-1][0] == 0  # five sources cannot be split further


def test_worst_case_queue_counts_three_children_per_split(output):
    # the children at levels 2-4 (4 per split of 48 + 192 + 768 parents) -> 3 per split
    # through the queue at most; from level 3 on only the level-4 packages
    row = [l for l in output if l.startswith("worst")][0].split()
    assert int(row[1]) == (192 + 768 + 3072) // 4 * 3 and int(row[2]) == 3072 // 4 * 3


def test_halting_radii_equal_the_oracle(output):
    tables = [np.array([float(x) for x in l.split()[1:]]) for l in output if l.startswith("rlim")]
    cdt = [3.5, 3.5, 2.25, 4.0, 3.5, 3.5, 3.5, 3.5, 3.5, 3.5, 3.5, 3.5]
    fl = oracle.Flight()
    for k, (c, got) in enumerate(zip(cdt, tables)):
        ref = fl.advance(c)
        # the library drops ages that would lie beyond the box diagonal (30 + 1 cells here)
        n = got.size
        np.testing.assert_array_equal(got, ref[:n])
        assert np.all(ref[n:] > 31.0)  # what was dropped lies beyond the diagonal
    assert tables[-1].size < len(cdt)  # the table stops growing once light has crossed the box
