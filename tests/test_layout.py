"""Host-side scratch layout: the bulk copies of the reflector digits and the
cp.async staging need 16-byte aligned regions of the right size.  Builds a
small host program against the kernels' header (no GPU needed) and checks
the offsets make_layout hands out."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2108_05345_gb300", "csrc")

CASES = [(4096, 2048, 152), (4097, 3, 152), (100, 333, 152), (8192, 8192, 148), (512, 1024, 1), (1, 1, 152)]

PROGRAM = r"""
#include <cstdio>
#include "lhdm_kernels.cuh"
int main() {
  const int cases[][3] = {%s};
  for (const auto& c : cases) {
    const lhdm::ScratchLayout L = lhdm::make_layout(c[0], c[1], c[2]);
    std::printf("%%d %%d %%d %%d %%zu %%zu %%zu %%zu %%zu %%zu\n", c[0], c[1], c[2], (int)L.pipelined, L.Vd, L.dtotal,
                L.Ver, L.itotal, L.part, L.W);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def layouts(tmp_path_factory):
    nvcc = shutil.which(os.environ.get("NVCC", "nvcc"))
    if not nvcc:
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("layout")
    src = d / "layout.cu"
    src.write_text(PROGRAM % ", ".join("{%d, %d, %d}" % c for c in CASES))
    exe = d / "layout"
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC, "-I",
                    os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    rows = [list(map(int, line.split())) for line in out if line.strip()]
    assert len(rows) == len(CASES)
    return rows


def test_digit_region_aligned_and_large_enough(layouts):
    ND = 8
    for m, n, team, pipelined, vd, dtotal, ver, itotal, part, w in layouts:
        assert pipelined == (1 if team > 1 else 0)
        # offsets are in doubles / ints from 256-byte aligned bases: the
        # digit rows are bulk-copied (16-byte rule), the rest loaded per word
        assert (vd * 8) % 16 == 0 and (ver * 4) % 16 == 0 and (part * 8) % 16 == 0
        if pipelined:
            assert (dtotal - vd) * 8 >= ND * max(m, 1) * 64  # m rows x ND planes x 64 bytes
            assert (itotal - ver) >= max(m, 1)
