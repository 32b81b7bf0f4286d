"""Known-answer pin of the oracle's Philox4x32-10 against an implementation
this project did not write: ATen's ``philox_engine`` (the readable C++ header
``ATen/core/PhiloxRNGEngine.h`` that ships with PyTorch). CPU only.

Every sample point of the transfer (Sec. 4, step 3: independent uniforms per
sample) is a function of Philox words, and the CUDA path matches the oracle
bit for bit on the sample elements, so a misread round function, Weyl key
schedule or output word order would be shared by both sides; the
statistical pins in ``test_oracle_pins.py`` cannot see it. This test can.

Mapping of ATen's state onto the (counter, key) of Salmon et al.:
``philox_engine(seed, subsequence, offset)`` holds key = (seed low 32 bits,
seed high 32 bits) and the 128-bit counter (offset low, offset high,
subsequence low, subsequence high); its first four draws are output words
0..3 of one block. So the oracle's block for counter (c0, c1, c2, c3) and
key (k0, k1) is ATen's first four draws with seed = k0 | k1 << 32,
subsequence = c2 | c3 << 32 and offset = c0 | c1 << 32.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

_HARNESS = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
int main() {
  unsigned long long seed, sub, off;
  int nwords;
  while (std::scanf("%llu %llu %llu %d", &seed, &sub, &off, &nwords) == 4) {
    at::Philox4_32 eng(seed, sub, off);
    for (int i = 0; i < nwords; ++i) std::printf("%u ", eng());
    std::printf("\n");
  }
  return 0;
}
"""


def _aten_include():
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("ATen's PhiloxRNGEngine.h is not installed with this torch")
    return inc


@pytest.fixture(scope="module")
def aten_philox(tmp_path_factory):
    inc = _aten_include()
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("aten_philox")
    src = d / "harness.cpp"
    exe = d / "harness"
    src.write_text(_HARNESS)
    subprocess.run(["g++", "-std=c++17", "-O1", f"-I{inc}", str(src), "-o", str(exe)], check=True)

    def run(cases, nwords=4):
        lines = []
        for ctr, key in cases:
            seed = int(key[0]) | (int(key[1]) << 32)
            sub = int(ctr[2]) | (int(ctr[3]) << 32)
            off = int(ctr[0]) | (int(ctr[1]) << 32)
            lines.append(f"{seed} {sub} {off} {nwords}")
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True,
                             check=True).stdout.split()
        return np.array(out, dtype=np.uint64).astype(np.uint32).reshape(len(cases), nwords)

    return run


def _cases():
    M = 0xFFFFFFFF
    cases = [([0, 0, 0, 0], [0, 0]), ([M, M, M, M], [M, M]), ([0, 0, 0, 0], [M, M]), ([M, M, M, M], [0, 0]),
             ([1, 0, 0, 0], [0, 0]), ([0, 1, 0, 0], [0, 0]), ([0, 0, 1, 0], [0, 0]), ([0, 0, 0, 1], [0, 0]),
             ([0, 0, 0, 0], [1, 0]), ([0, 0, 0, 0], [0, 1]),
             ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0])]
    # the transfer's own counters: (unit j, target element t, stream, tag) under
    # seed 0 and a 64-bit seed, as the assembly, control, training-set and
    # workload generators form them
    for seed in (0, 12345, 0x0123456789ABCDEF):
        key = [seed & M, seed >> 32]
        for j in (0, 1, 7, 31, 63):
            for t in (0, 1, 999_999, 1_999_999, 2_958_233):
                for stream in (0, 3):
                    cases.append(([j, t, stream, 0], key))
        for tag in (1, 2, 3, 4, 5):
            cases.append(([5, 17, 0, tag], key))
    rng = np.random.default_rng(20260313)
    for _ in range(200):
        c = rng.integers(0, 1 << 32, size=4, dtype=np.uint64)
        k = rng.integers(0, 1 << 32, size=2, dtype=np.uint64)
        cases.append(([int(x) for x in c], [int(x) for x in k]))
    return cases


def test_oracle_philox_equals_aten_word_for_word(orc, aten_philox):
    cases = _cases()
    assert len(cases) >= 300
    want = aten_philox(cases)
    got = np.array([orc.philox4x32_10(c, k) for c, k in cases], dtype=np.uint32)
    bad = np.nonzero((got != want).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} blocks differ, first at case {cases[bad[0]]}: {got[bad[0]]} vs {want[bad[0]]}"


def test_aten_offset_addresses_blocks(orc, aten_philox):
    """The mapping addresses one block directly: offset n is the n-th block of
    a subsequence. One ATen engine drawing 12 words in a row from offset 0
    equals the oracle's blocks of counters (0, 0, 9, 0), (1, 0, 9, 0) and
    (2, 0, 9, 0); the same across a carry from the low counter word."""
    M = 0xFFFFFFFF
    for c0, c1 in ((0, 0), (M - 1, 0)):
        stream = aten_philox([([c0, c1, 9, 0], [3, 0])], nwords=12).ravel()
        blocks = []
        for i in range(3):
            lo = (c0 + i) & M
            hi = c1 + ((c0 + i) >> 32)
            blocks.append(orc.philox4x32_10([lo, hi, 9, 0], [3, 0]))
        assert np.array_equal(stream, np.concatenate(blocks).astype(np.uint32))
