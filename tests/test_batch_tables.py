"""Host logic of the batched engine's global-update tables
(`csrc/batch_tables.h`), compiled with g++ and checked on the CPU on random
copy structures: every global in the permutation once, the computed globals
(bounded, or with several copies) first and the bounded ones first of all,
each in index order; the one-copy unbounded globals last; a computed entry's
first two rows, copy count, later-copy rows (in copy order) and bounded index
as given; every position's first row and copy count; and the refusals (a
global without a copy or with 256, a row beyond 24 bits)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2310_09410_gb300", "csrc")

DRIVER = r"""
#include "batch_tables.h"
#include <cstdio>
#include <random>

using namespace opf;

static int fail(const char *what, int seed) { std::printf("FAIL %s seed %d\n", what, seed); return 1; }

int main() {
    std::mt19937 rng(2024);
    int cases = 0;
    for (int seed = 0; seed < 3000; ++seed) {
        const int G = 1 + (int)(rng() % 300);
        const int pb = (int)(rng() % 101), pmulti = (int)(rng() % 101);
        std::vector<int> gstart(G + 1, 0), bidx(G, -1), crow;
        int nb = 0;
        for (int i = 0; i < G; ++i) {
            int cnt = 1;
            if ((int)(rng() % 100) < pmulti) cnt = 2 + (int)(rng() % 9);
            gstart[i + 1] = gstart[i] + cnt;
            if ((int)(rng() % 100) < pb) bidx[i] = nb++;
        }
        for (int k = 0; k < gstart[G]; ++k) crow.push_back((int)(rng() % (1u << 24)));
        GlobalTables t;
        if (!build_global_tables(G, gstart, crow, bidx, &t)) return fail("refused a valid structure", seed);
        ++cases;
        std::vector<int> seen(G, 0);
        for (int j = 0; j < G; ++j) {
            const int i = t.gperm[j];
            if (i < 0 || i >= G || seen[i]++) return fail("not a permutation", seed);
            const int cnt = gstart[i + 1] - gstart[i];
            const bool computed = bidx[i] >= 0 || cnt > 1;
            if (computed != (j < t.Gs)) return fail("computed globals first", seed);
            if (t.gx[j] != (crow[gstart[i]] | (cnt << 24))) return fail("first row and copies", seed);
            if (j > 0) {
                const int ip = t.gperm[j - 1];
                const int cp = gstart[ip + 1] - gstart[ip];
                const int rank = bidx[i] >= 0 ? 0 : (cnt > 1 ? 1 : 2);
                const int rankp = bidx[ip] >= 0 ? 0 : (cp > 1 ? 1 : 2);
                if (rankp > rank || (rankp == rank && ip > i)) return fail("order", seed);
            }
            if (j >= t.Gs) continue;
            const int *e = &t.gtab[(size_t)4 * j];
            if (e[0] != crow[gstart[i]]) return fail("first row", seed);
            if (e[1] != (cnt > 1 ? crow[gstart[i] + 1] : 0)) return fail("second row", seed);
            if ((e[2] & 0xff) != cnt) return fail("copies", seed);
            if (e[3] != bidx[i]) return fail("bounded index", seed);
            const int x0 = e[2] >> 8;
            for (int q = 2; q < cnt; ++q)
                if (x0 + q - 2 >= (int)t.uxt.size() || t.uxt[x0 + q - 2] != crow[gstart[i] + q])
                    return fail("later copies", seed);
        }
        size_t later = 0;
        for (int i = 0; i < G; ++i) {
            const int cnt = gstart[i + 1] - gstart[i];
            if (bidx[i] >= 0 || cnt > 1) later += cnt > 2 ? cnt - 2 : 0;
        }
        if (later != t.uxt.size()) return fail("later-copy count", seed);
    }
    // refusals
    {
        GlobalTables t;
        std::vector<int> gstart = {0, 1, 1}, bidx = {-1, 0}, crow = {5};
        if (build_global_tables(2, gstart, crow, bidx, &t)) return fail("a global without a copy", -1);
        std::vector<int> g2 = {0, 256}, b2 = {-1}, c2(256, 1);
        if (build_global_tables(1, g2, c2, b2, &t)) return fail("256 copies", -1);
        std::vector<int> g3 = {0, 1}, b3 = {0}, c3 = {1 << 24};
        if (build_global_tables(1, g3, c3, b3, &t)) return fail("row beyond 24 bits", -1);
    }
    std::printf("ok %d\n", cases);
    return 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_global_update_tables(tmp_path):
    src = tmp_path / "tables.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "tables"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok "), out.stdout
    assert int(out.stdout.split()[1]) == 3000
