"""Host logic of the binning's unit schedule (CPU only).

The stable scatters of the binning cut every segment (the sorted visible
entries of a view, the row items of a (view, tile row) bucket) into units of
kUnitFirst, 2 kUnitFirst, ... items up to a cap, one warp per unit, and the
workspace reserves ceil(items / cap) + segments x (ramp + 1) unit slots.
These tests compile the library's own `unit_start` / `unit_count` /
`unit_ramp` (gs_device.cuh) into a host program and check, for every count up
to a bound, that the units tile the segment exactly, that their sizes follow
the schedule, and that the reservation covers any split of the items over
segments (the per-segment bound units(c) <= floor(c / cap) + ramp + 1).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROG = r"""
#include <cstdio>
#include "gs_device.cuh"
using namespace gsb;

static int check(int cap, long max_c) {
  const int r = unit_ramp(cap);
  // the schedule: unit j holds kUnitFirst 2^j items while j < r, then cap
  for (long j = 0; j < r + 8; ++j) {
    const long size = unit_start(j + 1, cap) - unit_start(j, cap);
    const long want = j < r ? (long)kUnitFirst << j : cap;
    if (size != want) { std::printf("cap %d: unit %ld holds %ld, not %ld\n", cap, j, size, want); return 1; }
  }
  if (((long)kUnitFirst << (r - 1)) > cap || ((long)kUnitFirst << r) < cap) {
    std::printf("cap %d: ramp %d does not end at the cap\n", cap, r); return 1;
  }
  for (long c = 0; c <= max_c; ++c) {
    const long k = unit_count((uint32_t)c, cap);
    if (c == 0) {
      if (k != 0) { std::printf("cap %d: %ld units for no items\n", cap, k); return 1; }
      continue;
    }
    // the k units cover the c items and the last one is not empty
    if (unit_start(k, cap) < c || unit_start(k - 1, cap) >= c) {
      std::printf("cap %d: %ld units do not tile %ld items\n", cap, k, c); return 1;
    }
    if (k > c / cap + r + 1) { std::printf("cap %d: %ld units for %ld items exceed the bound\n", cap, k, c); return 1; }
  }
  std::printf("cap %d ramp %d ok\n", cap, r);
  return 0;
}

int main() {
  return check(kEntryUnit, 300000) | check(kRowUnit, 300000) | check(2 * kUnitFirst, 5000);
}
"""


@pytest.fixture(scope="module")
def unit_prog(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("units")
    src, exe = d / "units.cu", d / "units"
    src.write_text(PROG)
    cmd = [nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2507_04004_b300", "csrc"),
           str(src), "-o", str(exe)]
    subprocess.run(cmd, check=True, capture_output=True, timeout=600)
    return str(exe)


def test_unit_schedule_tiles_segments_and_fits_the_reservation(unit_prog):
    out = subprocess.run([unit_prog], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.count(" ok") == 3, out.stdout
