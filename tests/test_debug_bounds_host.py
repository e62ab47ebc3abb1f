"""Host side of the debug-bounds build's records (no GPU): the file code a
check derives from its __FILE__ at compile time, and the name the library
prints for a record (file code << 16 | line).  Compiled with the host C++
compiler against csrc/debug_bounds.cuh."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2411_09605_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

PROGRAM = r"""
#include <cstdio>
#include <cstring>
#include "debug_bounds.cuh"
using namespace pic;
// compile-time: the code of a path is the index of the listed file it ends with
static_assert(bounds_file_code("es1d_mixed.cu") == 2, "bare name");
static_assert(bounds_file_code("/a/b/csrc/em2d_mixed.cu") == 3, "path");
static_assert(bounds_file_code("x\\y\\em1d_spectral.cu") == 4, "backslash path");
static_assert(bounds_file_code("/a/mixed_common.cuh") == 1, "header");
static_assert(bounds_file_code("/a/pic_api.cu") == 5, "runtime unit");
static_assert(bounds_file_code("/a/xes1d_mixed.cu") == 0, "no partial-name match");
static_assert(bounds_file_code("/a/es1d_mixed.cu.bak") == 0, "suffix must end the path");
static_assert(bounds_file_code("") == 0, "empty");
static_assert(!bounds_ends_with("abc", ""), "an empty name matches nothing");
int main() {
  const unsigned site = (3u << 16) | 417u;
  std::printf("%s:%u|%s|%s\n", bounds_file_name(site), site & 0xFFFFu, bounds_file_name(0u),
              bounds_file_name(99u << 16));
  return 0;
}
"""


def test_record_file_codes_and_names(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("needs a host C++ compiler and the CUDA headers")
    src = tmp_path / "records.cpp"
    exe = tmp_path / "records"
    src.write_text(PROGRAM)
    r = subprocess.run([cxx, "-std=c++17", "-I", CSRC, "-I", CUDA_INC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.strip()
    assert out == "em2d_mixed.cu:417|?|?"
