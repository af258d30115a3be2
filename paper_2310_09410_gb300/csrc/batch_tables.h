// Global-update tables of the batched engine (host code, no CUDA).
//
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

#include <vector>

namespace opf {

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
