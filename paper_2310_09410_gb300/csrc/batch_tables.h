// Host-side plan tables of the batched engine (no CUDA): the warp tasks and
// the global-update tables.
//
// Global-update tables:
// The engine's global update (Eq. closed_1) computes, for every global i that
// is bounded or has several copies, x_i from the copies' u and stores rho x_i
// into every copy's slot; a global with one copy and no bounds needs no
// global update (with a zero shifted cost, rho x_i is the u of its slot).
// The tables, from the copies' slot-array rows:
//   gperm  every global once: the bounded ones (in index order), the other
//          computed ones (in index order), then the one-copy unbounded ones;
//          Gs = the number of computed globals.
//   gtab   per computed global j < Gs, four ints: the rows of its first two
//          copies (the second 0 with one copy), copies | (first later copy in
//          uxt) << 8, bounded index or -1.
//   uxt    the rows of the third and later copies, global by global.
//   gx     per table position j < G: row of the first copy | copies << 24.
#pragma once

#include <algorithm>
#include <numeric>
#include <vector>

namespace opf {

// One warp task of the batched engine: J / p member subsystems of similar
// shape, each on p lane positions of the warp (lane = position * K + column).
struct BatchTask {
    int ch0;     // first chunk
    int nq;      // chunks per position
    int f;       // factor rows (maximum over the members; absent rows are zero)
    int foff;    // factor element (r, q, jpos, e) at foff + ((r * nq + q) * J + jpos) * 4 + e
    int p, lp;   // positions per member and log2(p)
    int modes;   // bit mb: member mb uses M = F^T F (1) or M = I - F^T F (0)
    int tm;      // tensor-memory plans: (first column << 2) | lane quadrant of the task's lambda / bbar~
};

// The warp tasks of a plan with K instance columns (J = 32 / K positions per
// warp) and NQ chunks of 4 slots per lane:
//   tasks, memb  the tasks in the engine's order and, per task, the
//                subsystem on each of its J / p member places (-1: empty),
//                J entries per task;
//   chg          per chunk 4 ints: K times the global of each slot (-1: pad);
//   sch          per local slot: its position (chunk * 4 + slot in chunk);
//   NCH, nF      chunk count, packed factor floats (a multiple of 4);
//   tm, tm_cols, qstart  tensor-memory plans: lambda and bbar~ of each task in
//                the lane quadrant of the warps that run it (a warp w reaches
//                lanes 32 (w % 4) .. + 31 only), 8 nq columns per task, at
//                most 512 per quadrant; the tasks of quadrant q are
//                [qstart[q], qstart[q + 1]).
struct TaskPlan {
    std::vector<BatchTask> tasks;
    std::vector<int> memb, chg, sch;
    int NCH = 0, nF = 0;
    bool tm = false;
    int tm_cols = 0, qstart[5] = {0, 0, 0, 0, 0};
};

// Estimated cycles of a task per iteration: a least-squares fit to per-task
// clock counts of the FP32 engine (8 instances per CTA, 16 warps) on the
// 1024 x 123-bus batch, over its chunks per lane nq, row pairs f / 2 and
// log2 p (the shuffle levels of a member on p > 1 positions); within 18 % of
// every measured task.  (A cost of nq (f (28 + 2 lp) + 40) + 30 before gave
// 12.33 ms per launch of 2000 iterations, this one 12.28 ms.)
inline double batch_task_cost(const BatchTask &t) {
    return 11.0 + 179.0 * t.nq + 0.5 * t.f * (107.0 + 66.0 * t.nq + 76.0 * t.lp);
}

// Per subsystem d (S of them): npad[d] padded slots, sf[d] factor rows,
// mode[d], soff[d] first local slot, sn[d] slots; gk[k] the global of local
// slot k (L slots).  Tasks group J / p subsystems of one position count p
// (the smallest power of 2 whose p * 4 * nq slots hold the subsystem),
// sorted by chunks then rows; the engine hands them out in decreasing cost;
// tensor memory when want_tm and the quadrants' columns fit (longest first
// to the least loaded quadrant).  Returns 0, 1 when a subsystem needs more
// positions than a warp has, 2 when a slot got no chunk.
inline int build_task_plan(int S, int L, const std::vector<int> &npad, const std::vector<int> &sf,
                           const std::vector<int> &mode, const std::vector<int> &soff, const std::vector<int> &sn,
                           const std::vector<int> &gk, int K, int nq, bool want_tm, TaskPlan *tp) {
    const int J = 32 / K, NPL = 4 * nq;
    auto ilog2 = [](int x) { int l = 0; while ((1 << l) < x) ++l; return l; };
    // per subsystem: positions and chunks per position
    std::vector<int> pd(S), nqd(S);
    for (int d = 0; d < S; ++d) {
        int q = 1;
        while (q * NPL < npad[d]) q <<= 1;
        if (q > J) return 1;
        pd[d] = q;
        nqd[d] = std::max(1, (npad[d] + 4 * q - 1) / (4 * q));
    }
    // tasks: per class p, J / p members of similar shape
    std::vector<BatchTask> tasks;
    std::vector<int> memb;
    for (int q = 1; q <= J; q <<= 1) {
        std::vector<int> cls;
        for (int d = 0; d < S; ++d) if (pd[d] == q) cls.push_back(d);
        std::stable_sort(cls.begin(), cls.end(), [&](int x, int y) {
            if (nqd[x] != nqd[y]) return nqd[x] > nqd[y];
            return sf[x] > sf[y];
        });
        const int per = J / q;
        for (size_t i = 0; i < cls.size(); i += per) {
            BatchTask t = {0, 0, 0, 0, q, ilog2(q), 0, 0};
            for (int mb = 0; mb < per; ++mb) {
                const int d = i + mb < cls.size() ? cls[i + mb] : -1;
                memb.push_back(d);
                if (d < 0) continue;
                t.nq = std::max(t.nq, nqd[d]);
                t.f = std::max(t.f, sf[d]);
                if (mode[d]) t.modes |= 1 << mb;
            }
            for (int mb = per; mb < J; ++mb) memb.push_back(-1);
            t.f += t.f & 1;        // rows in pairs (the packed extra row is zero)
            tasks.push_back(t);
        }
    }
    // decreasing cost (the engine hands tasks out in this order)
    {
        std::vector<int> ord(tasks.size());
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(),
                         [&](int x, int y) { return batch_task_cost(tasks[x]) > batch_task_cost(tasks[y]); });
        std::vector<BatchTask> t2;
        std::vector<int> m2;
        for (int t : ord) {
            t2.push_back(tasks[t]);
            m2.insert(m2.end(), memb.begin() + (size_t)t * J, memb.begin() + (size_t)(t + 1) * J);
        }
        tasks.swap(t2);
        memb.swap(m2);
    }
    // tensor memory: longest-first list scheduling over the 4 quadrants
    tp->tm = false;
    tp->tm_cols = 0;
    for (int q = 0; q < 5; ++q) tp->qstart[q] = 0;
    if (want_tm) {
        std::vector<double> load(4, 0.0);
        std::vector<int> used(4, 0), quad(tasks.size(), -1);
        bool fits = true;
        for (size_t t = 0; t < tasks.size() && fits; ++t) {
            int best = -1;
            for (int q = 0; q < 4; ++q)
                if (used[q] + 8 * tasks[t].nq <= 512 && (best < 0 || load[q] < load[best])) best = q;
            if (best < 0) { fits = false; break; }
            quad[t] = best;
            load[best] += batch_task_cost(tasks[t]);
            used[best] += 8 * tasks[t].nq;
        }
        if (fits) {
            std::vector<BatchTask> t2;
            std::vector<int> m2;
            int cols[4] = {0, 0, 0, 0};
            for (int q = 0; q < 4; ++q) {
                tp->qstart[q] = (int)t2.size();
                for (size_t t = 0; t < tasks.size(); ++t) {
                    if (quad[t] != q) continue;
                    BatchTask tk = tasks[t];
                    tk.tm = (cols[q] << 2) | q;
                    cols[q] += 8 * tk.nq;
                    t2.push_back(tk);
                    m2.insert(m2.end(), memb.begin() + t * J, memb.begin() + (t + 1) * J);
                }
            }
            tp->qstart[4] = (int)t2.size();
            tasks.swap(t2);
            memb.swap(m2);
            const int mx = std::max(std::max(cols[0], cols[1]), std::max(cols[2], cols[3]));
            tp->tm_cols = 32;
            while (tp->tm_cols < mx) tp->tm_cols <<= 1;
            tp->tm = true;
        }
    }
    // chunk / factor offsets and slot tables
    int ch = 0, fo = 0;
    std::vector<int> chg;
    std::vector<int> sch(L, -1);
    for (size_t t = 0; t < tasks.size(); ++t) {
        BatchTask &tk = tasks[t];
        tk.ch0 = ch;
        tk.foff = fo;
        chg.resize(((size_t)ch + (size_t)tk.nq * J) * 4, -1);
        for (int jpos = 0; jpos < J; ++jpos) {
            const int mb = jpos >> tk.lp, part = jpos & (tk.p - 1);
            const int d = memb[t * J + mb];
            if (d < 0) continue;
            const int so = soff[d], n = sn[d];
            for (int q = 0; q < tk.nq; ++q) {
                for (int e = 0; e < 4; ++e) {
                    const int c = (part * tk.nq + q) * 4 + e;
                    if (c < n) {
                        chg[((size_t)ch + q * J + jpos) * 4 + e] = gk[so + c] * K;   // shared-memory row of the global
                        sch[so + c] = (ch + q * J + jpos) * 4 + e;
                    }
                }
            }
        }
        ch += tk.nq * J;
        fo += tk.f * tk.nq * J * 4;
    }
    for (int k = 0; k < L; ++k)
        if (sch[k] < 0) return 2;
    tp->tasks.swap(tasks);
    tp->memb.swap(memb);
    tp->chg.swap(chg);
    tp->sch.swap(sch);
    tp->NCH = ch;
    tp->nF = (fo + 3) & ~3;
    return 0;
}

struct GlobalTables {
    std::vector<int> gperm, gtab, uxt, gx;   // gtab: 4 ints per computed global
    int Gs = 0;
};

// gstart[0..G]: copies of global i are [gstart[i], gstart[i+1]) in copy order;
// crow[k]: slot-array row of copy k; bidx[i]: bounded index or -1.  Returns
// false (tables left partial) when a global has no copy or 256 or more, a row
// does not fit 24 bits, or the later-copy list does not fit 23 bits.
inline bool build_global_tables(int G, const std::vector<int> &gstart, const std::vector<int> &crow,
                                const std::vector<int> &bidx, GlobalTables *t) {
    t->gperm.clear();
    t->gperm.reserve(G);
    auto copies = [&](int i) { return gstart[i + 1] - gstart[i]; };
    auto by_slot = [&](int i) { return copies(i) == 1 && bidx[i] < 0; };
    for (int i = 0; i < G; ++i) if (bidx[i] >= 0) t->gperm.push_back(i);
    for (int i = 0; i < G; ++i) if (bidx[i] < 0 && !by_slot(i)) t->gperm.push_back(i);
    t->Gs = (int)t->gperm.size();
    for (int i = 0; i < G; ++i) if (by_slot(i)) t->gperm.push_back(i);
    t->gtab.assign((size_t)4 * t->Gs, 0);
    t->uxt.clear();
    t->gx.assign(G, 0);
    for (int j = 0; j < G; ++j) {
        const int i = t->gperm[j], s0 = gstart[i], cnt = copies(i);
        if (cnt < 1 || cnt >= 256 || crow[s0] < 0 || crow[s0] >= (1 << 24) || t->uxt.size() >= (1u << 22))
            return false;
        t->gx[j] = crow[s0] | (cnt << 24);
        if (j >= t->Gs) continue;
        int *e = &t->gtab[(size_t)4 * j];
        e[0] = crow[s0];
        e[1] = cnt > 1 ? crow[s0 + 1] : 0;
        e[2] = cnt | ((int)t->uxt.size() << 8);
        e[3] = bidx[i];
        for (int q = 2; q < cnt; ++q) t->uxt.push_back(crow[s0 + q]);
    }
    return true;
}

}  // namespace opf
