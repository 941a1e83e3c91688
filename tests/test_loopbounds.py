"""The loop bounds of the warp-wide byte comparison (loopbounds.h), compiled
for the host with g++: every offset a 32-bit comparison step forms stays below
2^32 for every key it is used on, the step count is ceil((sa + len) / 1024),
and keys from kNarrowLen up to 2^32 - 1 bytes are sent to the 64-bit
comparison.  (Before the bound, a key of about 4 GiB made the 32-bit loop
counter wrap and the loop never end.)"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HDR = os.path.join(os.path.dirname(HERE), "paper_2411_18183_gb300", "csrc", "loopbounds.h")

PROG = r"""
#include <cstdio>
#include "%s"
using namespace algsig;
int main() {
  unsigned long long bad_end = 0, bad_steps = 0, checked = 0, wide = 0;
  const unsigned long long lens[] = {0ull, 1ull, 15ull, 16ull, 1008ull, 1009ull, 1023ull, 1024ull, 1025ull,
                                     0xFFFFEC00ull, 0xFFFFEFFFull};
  auto check = [&](unsigned long long len) {
    for (unsigned sa = 0; sa < 16; sa++)
      for (unsigned d = 0; d < 16; d++) {
        const unsigned long long steps = narrow_steps(sa, (uint32_t)len);
        if (steps != (sa + len + 1023ull) / 1024ull) bad_steps++;
        if (narrow_offset_end(sa, (uint32_t)len, d) > 0x100000000ull) bad_end++;
        checked++;
      }
  };
  for (unsigned long long len : lens) check(len);
  for (unsigned long long len = kNarrowLen - 70000ull; len < kNarrowLen; len++) check(len);
  for (unsigned long long len = 0xFFFFFC00ull - 5000ull; len <= 0xFFFFFFFFull; len++)
    if (!(len < kNarrowLen)) wide++;
  printf("%%llu %%llu %%llu %%llu %%u\n", checked, bad_steps, bad_end, wide, kNarrowLen);
  return 0;
}
"""


def test_narrow_comparison_bounds(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "lb.cpp"
    src.write_text(PROG % HDR)
    exe = tmp_path / "lb"
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-o", str(exe), str(src)])
    checked, bad_steps, bad_end, wide, narrow_len = map(int, subprocess.check_output([str(exe)]).split())
    assert checked == (11 + 70000) * 256
    assert bad_steps == 0, "step count differs from ceil((sa + len) / 1024)"
    assert bad_end == 0, "a 32-bit comparison step forms an offset of 2^32 or more"
    # every length from kNarrowLen to 2^32 - 1 goes to the 64-bit comparison, in particular the
    # lengths around 0xFFFFFC00 that made the old 32-bit loop wrap
    assert narrow_len <= 0xFFFFFC00 - 1024
    assert wide == 0xFFFFFFFF - narrow_len + 1
