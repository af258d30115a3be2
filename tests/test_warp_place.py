"""Host logic of the warp engine's plan (`csrc/warp_place.h`), compiled with
g++ and checked on the CPU: every subsystem placed once, no slot shared, the
two warps of a split subsystem in slots 2k, 2k + 1 of one CTA (the named
barrier 1 + k of the pair), the slot count the smallest that fits, and without
pairs subsystem s in CTA s % P, slot s / P."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2310_09410_gb300", "csrc")

DRIVER = r"""
#include "warp_place.h"
#include <cstdio>
#include <cstdlib>
#include <random>

using namespace opf;

static int fail(const char *what, int seed) { std::printf("FAIL %s seed %d\n", what, seed); return 1; }

int main() {
    std::mt19937 rng(12345);
    int cases = 0;
    for (int seed = 0; seed < 4000; ++seed) {
        const int S = 1 + (int)(rng() % 200);
        const int P = 1 + (int)(rng() % 16);
        const int pair_pct = (int)(rng() % 3) == 0 ? 0 : (int)(rng() % 100);
        std::vector<int> np(S);
        int W = 0;
        for (int s = 0; s < S; ++s) { np[s] = ((int)(rng() % 100) < pair_pct) ? 2 : 1; W += np[s]; }
        std::vector<int> cta, slot;
        const int warps = place_warp_items_min(np, P, 12, &cta, &slot);
        if (warps == 0) {
            // nothing fits: then not even 12 slots per CTA hold the items
            std::vector<int> c2, s2;
            if (place_warp_items(np, P, 12, &c2, &s2)) return fail("missed a fit", seed);
            continue;
        }
        ++cases;
        if (warps < (W + P - 1) / P || warps > 12) return fail("slot count range", seed);
        if (warps > (W + P - 1) / P) {
            std::vector<int> c2, s2;
            if (place_warp_items(np, P, warps - 1, &c2, &s2)) return fail("not the smallest slot count", seed);
        }
        std::vector<int> owner((size_t)P * warps, -1);
        for (int s = 0; s < S; ++s) {
            if (cta[s] < 0 || cta[s] >= P || slot[s] < 0 || slot[s] + np[s] > warps) return fail("range", seed);
            if (np[s] == 2 && (slot[s] & 1)) return fail("pair not at an even slot", seed);
            for (int q = 0; q < np[s]; ++q) {
                int &o = owner[(size_t)cta[s] * warps + slot[s] + q];
                if (o != -1) return fail("slot shared", seed);
                o = s;
            }
        }
        int pairs = 0;
        for (int s = 0; s < S; ++s) pairs += np[s] == 2;
        if (pairs == 0)
            for (int s = 0; s < S; ++s)
                if (cta[s] != s % P || slot[s] != s / P) return fail("FP32 mapping", seed);
    }
    std::printf("ok %d\n", cases);
    return 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_warp_placement_invariants(tmp_path):
    src = tmp_path / "place.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "place"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok "), out.stdout
    assert int(out.stdout.split()[1]) > 1000
