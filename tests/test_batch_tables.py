"""Host logic of the batched engine's plan (`csrc/batch_tables.h`), compiled
with g++ and checked on the CPU.

Global-update tables, on random copy structures: every global in the
permutation once, the computed globals (bounded, or with several copies)
first and the bounded ones first of all, each in index order; the one-copy
unbounded globals last; a computed entry's first two rows, copy count,
later-copy rows (in copy order) and bounded index as given; every position's
first row and copy count; and the refusals (a global without a copy or with
256, a row beyond 24 bits).

Warp tasks, on random subsystem shapes and engine shapes: every subsystem on
exactly one member place of one task, with the task's position count; a
task's chunks and rows cover its members', rows even, modes as given; tasks in
decreasing cost (per lane quadrant with tensor memory, whose columns stay
within 512 and follow each other); every local slot on its own position inside
its task's chunks, the chunk's global entry K times its global, padding -1;
the chunk and factor counts; a subsystem wider than a warp refused."""
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


TASKS_DRIVER = r"""
#include "batch_tables.h"
#include <cstdio>
#include <random>

using namespace opf;

static int fail(const char *what, int seed) { std::printf("FAIL %s seed %d\n", what, seed); return 1; }

int main() {
    std::mt19937 rng(77);
    int cases = 0;
    const int shapes[6][2] = {{8, 4}, {4, 4}, {2, 4}, {4, 2}, {2, 2}, {1, 2}};   // (K, NQ)
    for (int seed = 0; seed < 3000; ++seed) {
        const int K = shapes[seed % 6][0], nq = shapes[seed % 6][1], J = 32 / K;
        const int S = 1 + (int)(rng() % 250), G = 1 + (int)(rng() % 500);
        const int nmax = 1 + (int)(rng() % 64);
        std::vector<int> npad(S), sf(S), mode(S), soff(S), sn(S), gk;
        int L = 0;
        for (int d = 0; d < S; ++d) {
            sn[d] = 1 + (int)(rng() % nmax);
            npad[d] = (sn[d] + 3) & ~3;
            sf[d] = 1 + (int)(rng() % (sn[d] < 32 ? sn[d] : 32));
            mode[d] = (int)(rng() % 2);
            soff[d] = L;
            L += sn[d];
            for (int c = 0; c < sn[d]; ++c) gk.push_back((int)(rng() % G));
        }
        const bool want_tm = K > 1 && (rng() % 2) == 0;
        TaskPlan tp;
        const int rc = build_task_plan(S, L, npad, sf, mode, soff, sn, gk, K, nq, want_tm, &tp);
        int maxpad = 0;
        for (int d = 0; d < S; ++d) maxpad = npad[d] > maxpad ? npad[d] : maxpad;
        if (maxpad > J * 4 * nq) { if (rc != 1) return fail("wide subsystem accepted", seed); continue; }
        if (rc != 0) return fail("refused a valid plan", seed);
        ++cases;
        const int T = (int)tp.tasks.size();
        if ((int)tp.memb.size() != T * J) return fail("member table size", seed);
        std::vector<int> seen(S, 0);
        int ch = 0, fo = 0;
        for (int t = 0; t < T; ++t) {
            const BatchTask &tk = tp.tasks[t];
            if (tk.p < 1 || (1 << tk.lp) != tk.p || J % tk.p) return fail("positions", seed);
            if (tk.ch0 != ch || tk.foff != fo) return fail("offsets", seed);
            if (tk.f & 1) return fail("odd rows", seed);
            for (int mb = 0; mb < J; ++mb) {
                const int d = tp.memb[t * J + mb];
                if (mb >= J / tk.p) { if (d != -1) return fail("member beyond J / p", seed); continue; }
                if (d < 0) continue;
                if (d >= S || seen[d]++) return fail("subsystem placed twice", seed);
                int q = 1;
                while (q * 4 * nq < npad[d]) q <<= 1;
                if (q != tk.p) return fail("member position count", seed);
                if (tk.p * 4 * tk.nq < npad[d] || tk.f < sf[d]) return fail("task smaller than member", seed);
                if (((tk.modes >> mb) & 1) != mode[d]) return fail("mode", seed);
            }
            ch += tk.nq * J;
            fo += tk.f * tk.nq * J * 4;
        }
        for (int d = 0; d < S; ++d) if (!seen[d]) return fail("subsystem missing", seed);
        if (tp.NCH != ch || tp.nF != ((fo + 3) & ~3) || (int)tp.chg.size() != 4 * ch) return fail("counts", seed);
        // order: decreasing cost, per quadrant with tensor memory
        if (tp.tm) {
            if (!want_tm || tp.qstart[0] != 0 || tp.qstart[4] != T) return fail("quadrant ranges", seed);
            for (int q = 0; q < 4; ++q) {
                int col = 0;
                if (tp.qstart[q + 1] < tp.qstart[q]) return fail("quadrant order", seed);
                for (int t = tp.qstart[q]; t < tp.qstart[q + 1]; ++t) {
                    const BatchTask &tk = tp.tasks[t];
                    if ((tk.tm & 3) != q || (tk.tm >> 2) != col) return fail("tensor-memory columns", seed);
                    col += 8 * tk.nq;
                    if (t > tp.qstart[q] && batch_task_cost(tp.tasks[t - 1]) < batch_task_cost(tk))
                        return fail("quadrant cost order", seed);
                }
                if (col > 512 || col > tp.tm_cols || tp.tm_cols > 512) return fail("quadrant columns", seed);
            }
        } else {
            for (int t = 1; t < T; ++t)
                if (batch_task_cost(tp.tasks[t - 1]) < batch_task_cost(tp.tasks[t])) return fail("cost order", seed);
        }
        // slots
        std::vector<int> used((size_t)4 * ch, 0);
        for (int t = 0; t < T; ++t) {
            const BatchTask &tk = tp.tasks[t];
            for (int mb = 0; mb < J / tk.p; ++mb) {
                const int d = tp.memb[t * J + mb];
                if (d < 0) continue;
                for (int c = 0; c < sn[d]; ++c) {
                    const int pos = tp.sch[soff[d] + c];
                    if (pos < 4 * tk.ch0 || pos >= 4 * (tk.ch0 + tk.nq * J)) return fail("slot outside its task", seed);
                    if (used[pos]++) return fail("position shared", seed);
                    if (tp.chg[pos] != gk[soff[d] + c] * K) return fail("chunk global", seed);
                }
            }
        }
        for (size_t x = 0; x < used.size(); ++x)
            if (!used[x] && tp.chg[x] != -1) return fail("padding entry", seed);
    }
    std::printf("ok %d\n", cases);
    return 0;
}
"""


def _run(tmp_path, name, driver):
    src = tmp_path / (name + ".cpp")
    src.write_text(driver)
    exe = tmp_path / name
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)])
    return subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_warp_tasks(tmp_path):
    out = _run(tmp_path, "tasks", TASKS_DRIVER)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok "), out.stdout
    assert int(out.stdout.split()[1]) > 1500


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
