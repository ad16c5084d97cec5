"""Host arithmetic of the answer bitmaps' layout, compiled from the library's own header with
nvcc and run on the host (no GPU): a row holds w bitmap words (m users rounded up to 1,024
words), w / 32 summary words and w / 1024 top words, and the kernels recover w from the row
stride alone, so the inversion must be exact for every user count."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include "sah_internal.cuh"
int main() {
  long long m;
  int bad = 0;
  while (std::scanf("%lld", &m) == 1) {
    const long long s = sah::answer_stride(m), w = sah::answer_words(s);
    if (w % 1024 != 0 || w * 32 < m || w * 32 - m >= 1024 * 32 || s != w + w / 32 + w / 1024) {
      std::printf("bad %lld\n", m);
      ++bad;
    }
  }
  std::printf("checked, %d bad\n", bad);
  return bad != 0;
}
"""


def test_answer_stride_inverts_for_every_user_count():
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("no nvcc")
    rng = np.random.default_rng(3)
    ms = set(range(1, 3000)) | {2 ** e + o for e in range(5, 31) for o in (-1, 0, 1)} | {2 ** 31 - 1}
    ms |= set(int(x) for x in rng.integers(1, 2 ** 31 - 1, 20000))
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.cu"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write(PROGRAM)
        subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
                        "-I", os.path.join(ROOT, "paper_2211_12751_gb300", "csrc"), src, "-o", exe],
                       check=True, capture_output=True)
        r = subprocess.run([exe], input="\n".join(str(m) for m in sorted(ms)), capture_output=True, text=True)
    assert r.returncode == 0, r.stdout[-2000:]
    assert "checked, 0 bad" in r.stdout
