"""Host checks of the conjugate-partner pairing of the register-staged row passes
(csrc/fft_pair.h), compiled with the host C++ compiler: the thread-to-butterfly map of a stage with
ns butterflies is a permutation, the butterfly of lane l ^ 16 is the conjugate partner of lane l's
(ns - jj) except for the two self-partnered butterflies 0 and ns / 2, and with the rule the
kernels apply (partner's output R - 1 - r by a shuffle; butterfly 0 its own output (R - r) mod R,
butterfly ns / 2 its own output R - 1 - r) every half-spectrum index k <= n / 2 of a forward row is
written once, next to z_{n-k}."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2210_01837_gb300", "csrc")

PROGRAM = r"""
#include <stdio.h>
#include "fft_pair.h"
int main() {
  const int cases[][2] = {{3072, 16}, {3072, 12}, {2048, 8}, {4096, 16}, {384, 4}, {384, 12}, {1024, 2}, {512, 16}};
  for (auto& c : cases) {
    const int n = c[0], R = c[1], ns = n / R;
    for (int t = 0; t < ns; ++t) printf("P %d %d %d %d %d\n", n, R, t, dps::pair_butterfly(t, ns),
                                        dps::pair_self(dps::pair_butterfly(t, ns), ns) ? 1 : 0);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def pairing(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("pair")
    src, exe = d / "pair.cpp", d / "pair"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", SRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        _, n, R, t, jj, self_ = line.split()
        table.setdefault((int(n), int(R)), []).append((int(t), int(jj), int(self_)))
    return table


def test_map_is_a_permutation_with_partners_in_lane_xor_16(pairing):
    for (n, R), rows in pairing.items():
        ns = n // R
        assert ns % 32 == 0
        jj = [b for _, b, _ in rows]
        assert sorted(jj) == list(range(ns)), (n, R)
        for t, b, self_ in rows:
            assert bool(self_) == (b == 0 or 2 * b == ns)
            p = jj[t ^ 16]
            if not self_:
                assert p == ns - b, (n, R, t)
        # the two self-partnered butterflies sit in lanes 0 and 16 of the first warp
        assert {t for t, _, s in rows if s} == {0, 16}


def test_forward_split_writes_every_half_spectrum_value_once_beside_its_partner(pairing):
    for (n, R), rows in pairing.items():
        ns = n // R
        jj = [b for _, b, _ in rows]
        written = []
        for t, b, self_ in rows:
            for r in range(R // 2):
                k = b + ns * r
                if b == 0:
                    src_b, src_r = b, (R - r) % R
                elif 2 * b == ns:
                    src_b, src_r = b, R - 1 - r
                else:
                    src_b, src_r = jj[t ^ 16], R - 1 - r
                assert (src_b + ns * src_r) % n == (n - k) % n, (n, R, t, r)
                written.append(k)
            if b == 0:
                written.append(n // 2)  # z_{n/2} is its own partner (output R / 2 of butterfly 0)
        assert sorted(written) == list(range(n // 2 + 1)), (n, R)


def test_inverse_first_stage_reads_each_value_once(pairing):
    """The inverse pass's first stage: a lane reads its inputs e = jj + ns r below n / 2 and hands
    z_{n-e} to the partner lane, whose input R - 1 - r it is; the two self-partnered butterflies
    read their upper inputs directly.  Every half-spectrum index is read, and only those."""
    for (n, R), rows in pairing.items():
        ns = n // R
        jj = [b for _, b, _ in rows]
        reads = []
        for t, b, self_ in rows:
            for r in range(R // 2):
                e = b + ns * r
                assert e < n // 2
                reads.append(e)
                if not self_:  # the partner's input R - 1 - r is n - e
                    assert jj[t ^ 16] + ns * (R - 1 - r) == n - e
            if self_:
                for r in range(R // 2, R):
                    e = b + ns * r
                    reads.append(e if e == n // 2 else n - e)
        # every value below n / 2 read once by its owner, plus the self-partnered lanes' re-reads
        assert set(reads) == set(range(n // 2 + 1)), (n, R)
