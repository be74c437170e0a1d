"""The resident-layout helpers of gol_internal.h (host-callable inline
functions used by the layout kernels), compiled for the host and checked
against the layout's definition: the low half of a resident word holds the
word's even columns (bit j = column 2j), the high half its odd columns."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1209_4408_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include "gol_internal.h"
int main(int argc, char **argv) {
    for (int i = 1; i < argc; ++i) {
        const uint64_t x = std::strtoull(argv[i], nullptr, 16);
        std::printf("%016llx %016llx\n", (unsigned long long)gol::to_resident(x),
                    (unsigned long long)gol::to_interchange(x));
    }
    for (int c = 0; c < 64; ++c) std::printf("%d ", gol::resident_bit(c));
    std::printf("\n");
    return 0;
}
"""


@pytest.fixture(scope="module")
def helper(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("layout")
    src = d / "layout.cpp"
    src.write_text(PROGRAM)
    exe = d / "layout"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CUDA_INC, "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def resident_by_definition(x):
    lo = sum(((x >> (2 * j)) & 1) << j for j in range(32))
    hi = sum(((x >> (2 * j + 1)) & 1) << j for j in range(32))
    return lo | (hi << 32)


def test_layout_conversions_match_their_definition(helper):
    rng = np.random.default_rng(7)
    words = [int(v) for v in rng.integers(0, 2 ** 63, size=48, dtype=np.uint64)]
    words += [0, 1, 2, 1 << 63, (1 << 64) - 1, 0x5555555555555555, 0xAAAAAAAAAAAAAAAA]
    out = subprocess.run([helper] + ["%x" % w for w in words], capture_output=True, text=True,
                         check=True).stdout.split("\n")
    for w, line in zip(words, out):
        assert int(line.split()[0], 16) == resident_by_definition(w), hex(w)
    bits = [int(t) for t in out[len(words)].split()]
    assert bits == [(32 + c // 2) if c & 1 else c // 2 for c in range(64)]


def test_interchange_inverts_resident(helper):
    rng = np.random.default_rng(8)
    words = [int(v) for v in rng.integers(0, 2 ** 63, size=32, dtype=np.uint64)]
    res = [resident_by_definition(w) for w in words]
    out = subprocess.run([helper] + ["%x" % r for r in res], capture_output=True, text=True,
                         check=True).stdout.split("\n")
    for w, line in zip(words, out):
        assert int(line.split()[1], 16) == w
