"""The host rounding of filter weights to the tensor cores' operand formats (TF32 hi/lo,
BF16, FP16), used at plan creation for the precision forms and the 3xTF32 split, against
independent definitions: FP16 against numpy's IEEE conversion (round to nearest even),
BF16 and TF32 against a brute-force choice of the nearest representable neighbour."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1802_05427_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "host_round.h"
int main(int argc, char** argv) {
  FILE* in = std::fopen(argv[1], "rb");
  FILE* out = std::fopen(argv[2], "wb");
  std::vector<float> x;
  float v;
  while (std::fread(&v, 4, 1, in) == 1) x.push_back(v);
  for (float f : x) {
    const float t = rapro::tf32_round_host(f);
    const uint16_t b = rapro::bf16_round_host(f), h = rapro::f16_round_host(f);
    std::fwrite(&t, 4, 1, out);
    std::fwrite(&b, 2, 1, out);
    std::fwrite(&h, 2, 1, out);
  }
  std::fclose(in);
  std::fclose(out);
  return 0;
}
"""


@pytest.fixture(scope="module")
def rounder(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("host_round")
    src, exe = d / "r.cpp", d / "r"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def run(x):
        x = np.ascontiguousarray(x, dtype=np.float32)
        fi, fo = d / "in.bin", d / "out.bin"
        x.tofile(fi)
        subprocess.run([str(exe), str(fi), str(fo)], check=True)
        raw = np.fromfile(fo, dtype=np.uint8).reshape(-1, 8)
        t = raw[:, 0:4].copy().view(np.float32).ravel()
        b = raw[:, 4:6].copy().view(np.uint16).ravel()
        h = raw[:, 6:8].copy().view(np.uint16).ravel()
        return t, b, h
    return run


def _values():
    rng = np.random.default_rng(7)
    x = np.concatenate([
        rng.standard_normal(20000).astype(np.float32),
        (rng.standard_normal(5000) * 1e-6).astype(np.float32),          # FP16 subnormal range
        (rng.standard_normal(2000) * 3e4).astype(np.float32),           # near FP16 overflow
        np.array([0.0, -0.0, 1.0, -1.0, 65504.0, 65519.0, 65520.0, 6.1035156e-05, 5.9604645e-08,
                  2.9802322e-08, 1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, 1.0 + 2.0 ** -8], np.float32),
    ])
    # exact ties of the BF16 and TF32 grids
    base = rng.standard_normal(2000).astype(np.float32).view(np.uint32)
    x = np.concatenate([x, ((base & 0xFFFF0000) | 0x8000).view(np.float32),
                        ((base & 0xFFFFE000) | 0x1000).view(np.float32)])
    return x


def _nearest(x, keep_bits, ties):
    """Brute force: the two neighbours of x on the grid that keeps `keep_bits` low bits zero,
    the nearer one (ties: 'even' low kept bit, or 'away' from zero)."""
    u = x.view(np.uint32).astype(np.uint64)
    step = np.uint64(1) << np.uint64(keep_bits)
    lo = (u // step) * step
    hi = lo + step
    xl, xh = lo.astype(np.uint32).view(np.float32), hi.astype(np.uint32).view(np.float32)
    dl = np.abs(x.astype(np.float64) - xl.astype(np.float64))
    dh = np.abs(xh.astype(np.float64) - x.astype(np.float64))
    pick_hi = dh < dl
    tie = dh == dl
    if ties == "even":
        pick_hi |= tie & (((lo // step) & np.uint64(1)) == 1)
    else:
        pick_hi |= tie                         # magnitudes: the larger one is away from zero
    return np.where(pick_hi, hi, lo).astype(np.uint32)


def test_fp16_rounding_matches_ieee(rounder):
    x = _values()
    _, _, h = rounder(x)
    with np.errstate(over="ignore"):         # values past 65520 round to infinity
        ref = x.astype(np.float16).view(np.uint16)
    np.testing.assert_array_equal(h, ref)


def test_bf16_rounding_is_nearest_even(rounder):
    x = _values()
    x = x[np.isfinite(x) & (np.abs(x) < 1e38)]
    _, b, _ = rounder(x)
    ref = (_nearest(x, 16, "even") >> np.uint32(16)).astype(np.uint16)
    np.testing.assert_array_equal(b, ref)


def test_tf32_rounding_is_nearest_ties_away(rounder):
    x = _values()
    x = x[np.isfinite(x) & (np.abs(x) < 1e38)]
    t, _, _ = rounder(x)
    ref = _nearest(x, 13, "away").view(np.float32)
    np.testing.assert_array_equal(t.view(np.uint32), ref.view(np.uint32))
    # the split hi + lo of the 3xTF32 passes: lo = f - hi is exact and rounds to < 2^-11 |f|
    lo = x - t
    np.testing.assert_array_equal((t.astype(np.float64) + lo.astype(np.float64)), x.astype(np.float64))
    nz = x != 0
    assert np.all(np.abs(lo[nz]) <= 2.0 ** -11 * np.abs(x[nz]) * (1 + 1e-7))
