"""The quantiser's block scale, amax / 480, is computed as a product with
1/480 (rounded) plus one correction by the fused-multiply-add residual.  This
checks, with the host's IEEE fmaf, that the two-step form equals the
correctly rounded quotient for every float whose exponent lies in
[-100, 127], the range in which the kernel uses it.  The reference quotient
is the double-precision quotient rounded to float: a / 480 = (a / 15) 2^-5,
and a / 15 either is exact or has a 4-bit periodic binary expansion with a
one in every period, so the double never lands on a float midpoint and the
second rounding is the correct one."""
import os
import platform
import shutil
import subprocess
import tempfile

import pytest

SRC = r"""
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>
int main(void) {
  const float c = 1.0f / 480.0f;
  long bad = 0, tot = 0;
  for (int e = -100; e <= 127; e++) {
    for (uint32_t m = 0; m < (1u << 23); m++) {
      const uint32_t u = ((uint32_t)(e + 127) << 23) | m;
      float a;
      memcpy(&a, &u, 4);
      const float q0 = a * c;
      const float q1 = fmaf(fmaf(-q0, 480.0f, a), c, q0);
      const float want = (float)((double)a / 480.0);
      tot++;
      if (memcmp(&q1, &want, 4) != 0) bad++;
    }
  }
  printf("%ld %ld\n", tot, bad);
  return 0;
}
"""


def test_fma_corrected_division_by_480_is_correctly_rounded():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    flags = ["-O2", "-ffp-contract=off"]
    if platform.machine() in ("x86_64", "AMD64"):
        flags.append("-mfma")  # fmaf as one instruction; without it the library's fmaf is exact but slow
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "t.c"), os.path.join(d, "t")
        open(src, "w").write(SRC)
        subprocess.run([cc, *flags, "-o", exe, src, "-lm"], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=600).stdout.split()
    tot, bad = int(out[0]), int(out[1])
    assert tot == 228 * (1 << 23)  # every bit pattern of 228 exponents
    assert bad == 0
