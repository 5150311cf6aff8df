"""CPU test of the per-device set-up cache (csrc/per_device.h).

Kernel attributes (the shared-memory opt-in) and occupancy are per-device in
CUDA, so the library keeps one set-up value per device ordinal.  This test
compiles the header with the host compiler against a fake device query and
checks: one set-up per device, a second device gets its own set-up, a failed
set-up is not cached, and an ordinal outside the table is served uncached."""

import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1706_02145_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "per_device.h"

static int g_dev = 0;
static bool dev_of(int* d) { *d = g_dev; return true; }
static bool dev_fail(int* d) { return false; }

#define CHECK(c) do { if (!(c)) { std::printf("FAIL line %d: %s\n", __LINE__, #c); return 1; } } while (0)

int main() {
  celes::PerDevice cache;
  int calls = 0;
  int value = 7;
  auto init = [&] { ++calls; return value; };
  g_dev = 0;
  CHECK(cache.get(dev_of, init) == 7 && calls == 1);
  CHECK(cache.get(dev_of, init) == 7 && calls == 1);       // cached on device 0
  g_dev = 1; value = 9;
  CHECK(cache.get(dev_of, init) == 9 && calls == 2);       // device 1 is set up on its own
  CHECK(cache.get(dev_of, init) == 9 && calls == 2);
  g_dev = 0;
  CHECK(cache.get(dev_of, init) == 7 && calls == 2);       // device 0 keeps its value
  // a failed set-up returns 0 and is retried on the next call
  g_dev = 2; value = 0;
  CHECK(cache.get(dev_of, init) == 0 && calls == 3);
  value = 5;
  CHECK(cache.get(dev_of, init) == 5 && calls == 4);
  CHECK(cache.get(dev_of, init) == 5 && calls == 4);
  // no cache slot: ordinal out of range or device query failed -> set-up every call
  g_dev = celes::kMaxDevices; value = 3;
  CHECK(cache.get(dev_of, init) == 3 && calls == 5);
  CHECK(cache.get(dev_of, init) == 3 && calls == 6);
  CHECK(cache.get(dev_fail, init) == 3 && calls == 7);
  // independent caches (one per kernel) do not share slots
  celes::PerDevice other;
  g_dev = 0; value = 11;
  CHECK(other.get(dev_of, init) == 11 && calls == 8);
  CHECK(cache.get(dev_of, init) == 7 && calls == 8);
  std::printf("ok\n");
  return 0;
}
"""


def test_per_device_cache_logic():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.cpp")
        exe = os.path.join(d, "t")
        with open(src, "w") as fh:
            fh.write(PROGRAM)
        r = subprocess.run([cxx, "-std=c++17", "-O1", "-I", HDR, src, "-o", exe], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        r = subprocess.run([exe], capture_output=True, text=True)
        assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
