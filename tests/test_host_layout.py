"""Host-side work layout (csrc/launch.h, choose_layout) compiled with nvcc as host
code and checked on the CPU: lanes per candidate a power of two up to 32, blocks
within the pass kernels' 128-thread limit, one lane per candidate for
populations that fill the GPU, and the caller's forced block size honoured."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2109_01928_gb300", "csrc")

HARNESS = r'''
#include <cstdio>
#include "launch.h"
int main() {
  const long long per[] = {1, 2, 3, 7, 8, 16, 31, 32, 33, 64, 100, 256, 4096};
  const long long tot[] = {1, 100, 8192, 32768, 262144, 1LL << 20, 1LL << 40};
  const debyefit::Layout forced[] = {{0, 0}, {32, 0}, {128, 0}, {32, 4}, {0, 2}, {8, 16}};
  const debyefit::Layout tuned[] = {{0, 0}, {64, 1}, {128, 1}, {64, 2}, {32, 4}};
  for (long long p : per)
    for (long long t : tot)
      for (const auto& f : forced)
        for (const auto& u : tuned) {
          if (t < p) continue;
          int cb = 0, ks = 0;
          debyefit::choose_layout(p, t, 152, f, u, &cb, &ks);
          std::printf("%lld %lld %d %d %d %d %d %d\n", p, t, f.cb, f.ks, u.cb, u.ks, cb, ks);
        }
  std::printf("MAX_BLOCK %d\n", debyefit::MAX_BLOCK);
  return 0;
}
'''


@pytest.fixture(scope="module")
def layouts(tmp_path_factory):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("layout")
    src, exe = d / "h.cu", d / "h"
    src.write_text(HARNESS)
    r = subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    max_block = int([l for l in out if l.startswith("MAX_BLOCK")][0].split()[1])
    rows = [tuple(int(v) for v in l.split()) for l in out if l and not l.startswith("MAX_BLOCK")]
    return rows, max_block


def test_layout_invariants(layouts):
    rows, max_block = layouts
    assert len(rows) > 1500
    target = 152 * 2048
    for p, t, fc, fk, uc, uk, cb, ks in rows:
        assert ks in (1, 2, 4, 8, 16, 32), (p, t, fc, fk, uc, uk, cb, ks)
        assert cb >= 1 and cb * ks <= max_block, (p, t, fc, fk, uc, uk, cb, ks)
        if p >= 32 and (fc > 0 or 2 * t >= target):       # full population
            want_ks = fk if fk else (1 if fc else (uk if uk else 1))
            want_cb = fc if fc else (uc if uc else 64)
            assert (cb, ks) == (min(want_cb, max_block // want_ks), want_ks), (p, t, fc, fk, uc, uk, cb, ks)
        else:
            assert cb * ks == 64 or (cb == 1 and ks == 32)   # a 64-thread block (or one 32-lane candidate)


def test_small_batches_get_more_lanes(layouts):
    rows, _ = layouts
    by = {}
    for p, t, fc, fk, uc, uk, cb, ks in rows:
        if fc == fk == uc == uk == 0:
            by.setdefault(p, []).append((t, ks))
    for p, seq in by.items():
        seq.sort()
        ks = [k for _, k in seq]
        assert all(a >= b for a, b in zip(ks, ks[1:])), (p, seq)   # fewer lanes as the batch grows
