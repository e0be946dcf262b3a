"""Host checks of the tensor-core operand descriptor encoders (csrc/umma_desc.h), compiled with the
host C++ compiler: every field sits at the bit position of the PTX ISA's tcgen05 descriptor tables
(shared-memory matrix descriptor; instruction descriptor of .kind::tf32), and the K-major core-matrix
layout used for the operand tiles places every element once, in 128-byte core matrices at the
descriptor's strides, inside the tile."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2210_01837_gb300", "csrc", "umma_desc.h")

PROGRAM = r"""
#include <stdio.h>
#include <initializer_list>
#include "umma_desc.h"
int main() {
  using namespace dps::umma;
  const unsigned a[][3] = {{0x0, 16, 16}, {0x1230, 2048, 128}, {0x3FFF0, 1280, 128}, {0x4560, 0x3FFF0, 0x10}};
  for (auto& v : a) printf("S %u %u %u %llu\n", v[0], v[1], v[2], (unsigned long long)smem_desc(v[0], v[1], v[2]));
  const unsigned mn[][2] = {{128, 80}, {128, 112}, {128, 48}, {64, 16}, {128, 256}};
  for (auto& v : mn) printf("I %u %u %u\n", v[0], v[1], idesc_tf32(v[0], v[1]));
  for (unsigned rows : {128u, 80u}) {
    for (unsigned r = 0; r < rows; ++r)
      for (unsigned k = 0; k < 8; ++k) printf("O %u %u %u %u\n", rows, r, k, kmajor_offset(r, k));
  }
  printf("L %u %u\n", kLbo, kSbo);
  for (unsigned rows : {128u, 80u, 48u}) printf("T %u %u\n", rows, tile_bytes(rows));
  // descriptor arithmetic used by the issuing thread: desc(a) + (off >> 4) == desc(a + off) for
  // 16-byte aligned shared addresses below 256 KB
  unsigned bad = 0;
  for (unsigned a = 0; a < (1u << 18); a += 16 * 37)
    for (unsigned off = 0; a + off < (1u << 18); off += 16 * 1021)
      if (smem_desc(a, kLbo, kSbo) + (off >> 4) != smem_desc(a + off, kLbo, kSbo)) ++bad;
  printf("A %u\n", bad);
  // tf32 rounding of a spread of bit patterns (printed for the comparison in Python)
  unsigned long long seed = 12345;
  for (int i = 0; i < 20000; ++i) {
    seed = seed * 6364136223846793005ull + 1442695040888963407ull;
    unsigned x = (unsigned)(seed >> 32);
    if ((x & 0x7F800000u) == 0x7F800000u) continue;  // finite inputs only
    if (i % 7 == 0) x = (x & ~0x1FFFu) | 0x1000u;       // exact ties
    printf("R %u %u\n", x, tf32_rna_bits(x));
  }
  return 0;
}
"""


def _field(v, lo, width):
    return (v >> lo) & ((1 << width) - 1)


@pytest.fixture(scope="module")
def encodings(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("umma")
    src = d / "t.cpp"
    src.write_text(PROGRAM)
    exe = d / "t"
    subprocess.run([cxx, "-std=c++17", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    rows = [l.split() for l in out if l]
    return rows


def test_shared_memory_descriptor_fields(encodings):
    for r in (r for r in encodings if r[0] == "S"):
        addr, lbo, sbo, d = map(int, r[1:])
        assert _field(d, 0, 14) == (addr >> 4) & 0x3FFF
        assert _field(d, 14, 2) == 0
        assert _field(d, 16, 14) == (lbo >> 4) & 0x3FFF
        assert _field(d, 30, 2) == 0
        assert _field(d, 32, 14) == (sbo >> 4) & 0x3FFF
        assert _field(d, 46, 2) == 1          # tcgen05 descriptor version
        assert _field(d, 48, 1) == 0
        assert _field(d, 49, 3) == 0          # base offset
        assert _field(d, 52, 1) == 0          # relative leading-dimension offsets
        assert _field(d, 53, 8) == 0
        assert _field(d, 61, 3) == 0          # no swizzle


def test_instruction_descriptor_fields(encodings):
    for r in (r for r in encodings if r[0] == "I"):
        m, n, d = map(int, r[1:])
        assert _field(d, 0, 4) == 0           # dense, no saturation
        assert _field(d, 4, 2) == 1           # D: f32
        assert _field(d, 6, 1) == 0
        assert _field(d, 7, 3) == 2           # A: tf32
        assert _field(d, 10, 3) == 2          # B: tf32
        assert _field(d, 13, 4) == 0          # no negation, both K-major
        assert _field(d, 17, 6) == n >> 3
        assert _field(d, 23, 1) == 0
        assert _field(d, 24, 5) == m >> 4
        assert _field(d, 29, 3) == 0


def test_kmajor_layout_places_core_matrices_in_the_tile(encodings):
    lbo, sbo = next(tuple(map(int, r[1:])) for r in encodings if r[0] == "L")
    tiles = {int(r[1]): int(r[2]) for r in encodings if r[0] == "T"}
    assert lbo == 128 and sbo >= 256 and sbo % 16 == 0
    for rows in (128, 80):
        assert tiles[rows] == rows // 8 * sbo
        offs = {(int(r[2]), int(r[3])): int(r[4]) for r in encodings if r[0] == "O" and int(r[1]) == rows}
        assert len(offs) == rows * 8
        vals = sorted(offs.values())
        assert len(set(vals)) == len(vals)                 # every element once
        assert vals[-1] + 4 <= tiles[rows]                  # inside the tile
        for (row, k), o in offs.items():
            # core matrix (8 rows x 16 bytes, 128 contiguous bytes) at the descriptor's strides:
            # the leading-dimension offset along K, the stride-dimension offset along the rows
            base = (k // 4) * lbo + (row // 8) * sbo
            assert o == base + (row % 8) * 16 + (k % 4) * 4
        # the descriptor's addresses stay inside the tile even with the two offsets exchanged
        assert (rows // 8 - 1) * lbo + 1 * sbo + 127 < tiles[rows]


def test_descriptor_offsets_add(encodings):
    """The issuing thread forms an operand's descriptor as the stage's descriptor plus the byte
    offset in 16-byte units; that must equal encoding the operand's address (no carry out of the
    14-bit start-address field for shared addresses below 256 KB)."""
    assert next(int(r[1]) for r in encodings if r[0] == "A") == 0


def test_tf32_rounding_is_round_to_nearest_ties_away(encodings):
    """tf32_rna_bits against the definition: the nearest float with 10 mantissa bits, halfway cases
    away from zero, computed exactly with Python integers and fractions (finite inputs; a carry may
    reach infinity, as rounding up at the top of the range should)."""
    from fractions import Fraction

    def value(b):
        s, e, m = b >> 31, (b >> 23) & 0xFF, b & 0x7FFFFF
        v = Fraction(m, 1 << 23) * Fraction(2) ** (-126) if e == 0 else (1 + Fraction(m, 1 << 23)) * Fraction(2) ** (e - 127)
        return -v if s else v

    rows = [(int(r[1]), int(r[2])) for r in encodings if r[0] == "R"]
    assert len(rows) > 15000
    for x, y in rows:
        assert y & 0x1FFF == 0 and (y >> 31) == (x >> 31)
        if (y & 0x7F800000) == 0x7F800000:
            continue  # rounded past the largest tf32 value
        lo = x & ~0x1FFF                      # truncated (toward zero) tf32 neighbour
        hi = lo + 0x2000                      # the next one away from zero
        vx, vlo, vhi = abs(value(x)), abs(value(lo)), abs(value(hi))
        want = hi if (vx - vlo) >= (vhi - vx) else lo
        assert y == want, (hex(x), hex(y), hex(want))
