// Plan of the lane engine (lane.cu): the subsystems split into the parts of
// a cluster, the per-part tables, and the engine-layout arrays of the tiles.
//
// Parts: the subsystems in depth-first order of the graph in which two
// subsystems are adjacent when they share a global (on a radial feeder a
// run of this order is a connected piece of the tree, so few globals have
// copies in two parts), cut into at most 16 contiguous runs that minimise
// the largest run's estimated cost, each run within the tensor-memory
// budget (lambda~ and bbar~ of its slots: 2 x 4-aligned slots <= 512
// columns).  Inside a part the subsystems go to the item groups (warps of a
// lane quadrant) by longest-first list scheduling, and so do the globals.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "batch_internal.h"

namespace opf {
namespace bx {

namespace {

constexpr int kLaneMaxC = 16;      // CTAs of a cluster (non-portable size above 8)
constexpr int kLaneMaxSlots = 256; // 4-aligned slots of a part (two tensor-memory columns each)

int round4(int x) { return (x + 3) & ~3; }

// Longest-first assignment of items with cost c[i] to n bins; bin of each item.
std::vector<int> lpt(const std::vector<double> &c, int n) {
    std::vector<int> ord(c.size()), bin(c.size(), 0);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return c[x] > c[y]; });
    std::vector<double> load(n, 0.0);
    for (int i : ord) {
        int best = 0;
        for (int g = 1; g < n; ++g)
            if (load[g] < load[best]) best = g;
        bin[i] = best;
        load[best] += c[i];
    }
    return bin;
}

}  // namespace

int build_lane_plan(opf_batch *b, BPlan *p, int WG, int maxC) {
    opf_handle *h = b->h;
    cudaStream_t st = h->stream;
    p->release();
    if (WG < 1 || WG > kLaneMaxGroups || WG * 4 * 32 > 512 || maxC < 1 || maxC > kLaneMaxC) {
        set_last_error("lane plan: 1 to 4 warps per lane quadrant, 1 to 16 CTAs per cluster");
        return OPF_E_INVALID;
    }
    const int S = h->S, L = h->L, G = h->G;
    p->dbl = false;
    p->fg = false;
    p->K = kLaneInst;
    p->ks = 7;
    p->J = 1;
    p->W = 4 * WG;
    p->nq = 0;
    p->threads = 128 * WG;
    // per subsystem: factor width in 4-column groups, cost estimate
    std::vector<int> sub_of(L), f4(S);
    std::vector<double> cost(S);
    for (int d = 0; d < S; ++d) {
        f4[d] = std::max(1, (h->h_sf[d] + 3) / 4);
        if (f4[d] > kLaneMaxF4) {
            set_last_error("lane plan: a subsystem has more factor vectors than the engine holds");
            return OPF_E_CAPACITY;
        }
        if (round4(h->h_sn[d]) > kLaneMaxSlots) {
            set_last_error("lane plan: a subsystem has more slots than a part holds");
            return OPF_E_CAPACITY;
        }
        for (int r = 0; r < h->h_sn[d]; ++r) sub_of[h->h_soff[d] + r] = d;
        cost[d] = h->h_sn[d] * (14.0 + 10.0 * f4[d]) + 16.0;
    }
    // subsystem graph through the globals, depth-first order from subsystem 0
    std::vector<std::vector<int>> adj(S);
    for (int i = 0; i < G; ++i)
        for (int a = h->h_gstart[i]; a < h->h_gstart[i + 1]; ++a)
            for (int c = a + 1; c < h->h_gstart[i + 1]; ++c) {
                const int x = sub_of[h->h_uslot[a]], y = sub_of[h->h_uslot[c]];
                if (x != y) { adj[x].push_back(y); adj[y].push_back(x); }
            }
    std::vector<int> order;
    {
        std::vector<char> seen(S, 0);
        std::vector<int> stack;
        for (int root = 0; root < S; ++root) {
            if (seen[root]) continue;
            stack.push_back(root);
            while (!stack.empty()) {
                const int v = stack.back();
                stack.pop_back();
                if (seen[v]) continue;
                seen[v] = 1;
                order.push_back(v);
                std::vector<int> nb = adj[v];
                std::sort(nb.begin(), nb.end());
                nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
                for (auto it = nb.rbegin(); it != nb.rend(); ++it)
                    if (!seen[*it]) stack.push_back(*it);
            }
        }
    }
    // contiguous runs: smallest bound on a run's cost that needs <= maxC runs
    auto cut = [&](double bound, std::vector<int> &start) -> bool {
        start.assign(1, 0);
        double c = 0.0;
        int slots = 0;
        for (int k = 0; k < S; ++k) {
            const int d = order[k];
            const int sl = round4(h->h_sn[d]);
            if (k > start.back() && (c + cost[d] > bound || slots + sl > kLaneMaxSlots)) {
                start.push_back(k);
                c = 0.0;
                slots = 0;
            }
            if (cost[d] > bound) return false;
            c += cost[d];
            slots += sl;
        }
        start.push_back(S);
        return (int)start.size() - 1 <= maxC;
    };
    std::vector<int> start;
    {
        double lo = 0.0, hi = 0.0;
        for (int d = 0; d < S; ++d) { lo = std::max(lo, cost[d]); hi += cost[d]; }
        if (!cut(hi, start)) {
            set_last_error("lane plan: the model needs more parts than a cluster has CTAs");
            return OPF_E_CAPACITY;
        }
        for (int step = 0; step < 40 && hi - lo > 1.0; ++step) {
            const double mid = 0.5 * (lo + hi);
            std::vector<int> s2;
            if (cut(mid, s2)) hi = mid;
            else lo = mid;
        }
        cut(hi, start);
    }
    const int C = (int)start.size() - 1;
    // per part: subsystems to item groups, local slot positions, factors
    std::vector<int> part_of_slot(L), pos_of_slot(L);        // part and local position of each slot
    std::vector<LanePart> parts(C);
    std::vector<int4> lsub, fdesc;
    std::vector<int> sch(L, -1);
    int cb = 0, fo = 0;
    for (int r = 0; r < C; ++r) {
        LanePart &P = parts[r];
        memset(&P, 0, sizeof(P));
        std::vector<int> subs(order.begin() + start[r], order.begin() + start[r + 1]);
        std::vector<double> sc(subs.size());
        for (size_t k = 0; k < subs.size(); ++k) sc[k] = cost[subs[k]];
        const std::vector<int> grp = lpt(sc, WG);
        P.sub0 = (int)lsub.size();
        P.cb = cb;
        P.F0 = fo;
        int p0 = 0, foff = 0;
        for (int g = 0; g < WG; ++g) {
            P.gsub[g] = (int)lsub.size() - P.sub0;
            // the group's subsystems, costliest first
            std::vector<int> mine;
            for (size_t k = 0; k < subs.size(); ++k)
                if (grp[k] == g) mine.push_back((int)k);
            std::stable_sort(mine.begin(), mine.end(), [&](int x, int y) { return sc[x] > sc[y]; });
            for (int k : mine) {
                const int d = subs[k], n = h->h_sn[d];
                lsub.push_back(make_int4(p0, n, foff, (h->h_mode[d] ? 1 : 0) | (f4[d] << 8)));
                fdesc.push_back(make_int4(d, fo + foff, f4[d], 0));
                for (int e = 0; e < n; ++e) {
                    const int k2 = h->h_soff[d] + e;
                    part_of_slot[k2] = r;
                    pos_of_slot[k2] = p0 + e;
                    sch[k2] = 4 * cb + p0 + e;
                }
                p0 += round4(n);
                foff += n * 4 * f4[d];
            }
        }
        P.gsub[WG] = (int)lsub.size() - P.sub0;
        for (int g = WG + 1; g <= kLaneMaxGroups; ++g) P.gsub[g] = P.gsub[WG];
        P.nsub = (int)lsub.size() - P.sub0;
        P.nslot = p0;
        P.nF = round4(foff);
        cb += p0 / 4;
        fo += P.nF;
    }
    const int NCH = cb;
    for (int k = 0; k < L; ++k)
        if (sch[k] < 0) { set_last_error("lane plan: slot without a part"); return OPF_E_INVALID; }
    // globals: copies in canonical order; exchange rows for the copies of
    // globals that span parts
    std::vector<int> lux((size_t)4 * NCH, -1), lgk((size_t)4 * NCH, -1);
    std::vector<int> nux(C, 0);
    std::vector<char> spans(G, 0);
    for (int i = 0; i < G; ++i) {
        const int a0 = h->h_gstart[i], a1 = h->h_gstart[i + 1];
        for (int a = a0; a < a1; ++a) {
            const int k = h->h_uslot[a];
            lgk[sch[k]] = i;
            if (part_of_slot[k] != part_of_slot[h->h_uslot[a0]]) spans[i] = 1;
        }
        if (!spans[i]) continue;
        for (int a = a0; a < a1; ++a) {
            const int k = h->h_uslot[a];
            lux[sch[k]] = nux[part_of_slot[k]]++;
        }
    }
    // subsystems with exchange rows
    for (int r = 0; r < C; ++r)
        for (int k = 0; k < parts[r].nsub; ++k) {
            int4 &sr = lsub[parts[r].sub0 + k];
            for (int e = 0; e < sr.y; ++e)
                if (lux[4 * parts[r].cb + sr.x + e] >= 0) { sr.w |= 2; break; }
        }
    // global items per part: the part's own globals (every copy in the part)
    // then the others, each list spread over the item groups by copies
    std::vector<int4> lgi;
    std::vector<int> lcp;
    for (int r = 0; r < C; ++r) {
        LanePart &P = parts[r];
        P.nux = nux[r];
        std::vector<int> gl;
        for (int k = 0; k < L; ++k)
            if (part_of_slot[k] == r) gl.push_back(h->h_gk[k]);
        std::sort(gl.begin(), gl.end());
        gl.erase(std::unique(gl.begin(), gl.end()), gl.end());
        P.g0 = (int)lgi.size();
        P.cp0 = (int)lcp.size();
        for (int pass = 0; pass < 2; ++pass) {
            std::vector<int> mine;
            for (int i : gl)
                if ((spans[i] != 0) == (pass == 1)) mine.push_back(i);
            std::vector<double> gc(mine.size());
            for (size_t k = 0; k < mine.size(); ++k) gc[k] = 4.0 + (h->h_gstart[mine[k] + 1] - h->h_gstart[mine[k]]);
            const std::vector<int> grp = lpt(gc, WG);
            int *rng = pass ? P.gcut : P.gint;
            for (int g = 0; g < WG; ++g) {
                rng[g] = (int)lgi.size() - P.g0;
                for (size_t k = 0; k < mine.size(); ++k) {
                    if (grp[k] != g) continue;
                    const int i = mine[k];
                    const int a0 = h->h_gstart[i], a1 = h->h_gstart[i + 1];
                    const int owner = part_of_slot[h->h_uslot[a0]] == r ? 1 : 0;
                    lgi.push_back(make_int4(i, b->h_bidx[i], (int)lcp.size() - P.cp0, (a1 - a0) | (owner << 16)));
                    for (int a = a0; a < a1; ++a) {
                        const int k2 = h->h_uslot[a], r2 = part_of_slot[k2];
                        const int row = r2 == r ? pos_of_slot[k2] : lux[sch[k2]];
                        lcp.push_back((r2 << 24) | row);
                    }
                }
            }
            rng[WG] = (int)lgi.size() - P.g0;
            for (int g = WG + 1; g <= kLaneMaxGroups; ++g) rng[g] = rng[WG];
        }
        P.ng = (int)lgi.size() - P.g0;
        P.ncp = (int)lcp.size() - P.cp0;
    }
    // every index the engine follows stays inside its part's arrays
    for (int r = 0; r < C; ++r) {
        const LanePart &P = parts[r];
        bool ok = P.nslot <= kLaneMaxSlots && P.nslot % 4 == 0 && P.nF % 4 == 0;
        for (int k = 0; k < P.nsub && ok; ++k) {
            const int4 sr = lsub[P.sub0 + k];
            const int F4 = (sr.w >> 8) & 15;
            ok = sr.x % 4 == 0 && sr.x + round4(sr.y) <= P.nslot && sr.z % 4 == 0 && F4 >= 1 &&
                 F4 <= kLaneMaxF4 && sr.z + sr.y * 4 * F4 <= P.nF;
        }
        for (int k = 0; k < P.ng && ok; ++k) {
            const int4 gr = lgi[P.g0 + k];
            const int N = gr.w & 0xffff;
            ok = gr.x >= 0 && gr.x < G && gr.y < b->NB && N >= 1 && N < kBatchRecip && gr.z >= 0 &&
                 gr.z + N <= P.ncp;
            for (int q = 0; q < N && ok; ++q) {
                const int cp = lcp[P.cp0 + gr.z + q], r2 = cp >> 24, row = cp & 0xffffff;
                ok = r2 >= 0 && r2 < C && row >= 0 && row < (r2 == r ? parts[r2].nslot : parts[r2].nux);
            }
        }
        for (int k = 0; k < P.nslot && ok; ++k) {
            const int ux = lux[4 * P.cb + k], gi = lgk[4 * P.cb + k];
            ok = ux < P.nux && gi < G;
        }
        for (int g = 0; g < WG && ok; ++g)
            ok = P.gsub[g] <= P.gsub[g + 1] && P.gint[g] <= P.gint[g + 1] && P.gcut[g] <= P.gcut[g + 1];
        ok = ok && P.gsub[WG] == P.nsub && P.gint[0] == 0 && P.gint[WG] == P.gcut[0] && P.gcut[WG] == P.ng;
        if (!ok) { set_last_error("lane plan: inconsistent part tables"); return OPF_E_INVALID; }
    }
    // shared memory (the largest part) and tensor-memory columns
    int mslot = 4, mux = 1, mF = 4, msub = 1, mg = 1, mcp = 1;
    for (const LanePart &P : parts) {
        mslot = std::max(mslot, P.nslot);
        mux = std::max(mux, P.nux);
        mF = std::max(mF, P.nF);
        msub = std::max(msub, P.nsub);
        mg = std::max(mg, P.ng);
        mcp = std::max(mcp, P.ncp);
    }
    const size_t I = kLaneInst;
    unsigned *o = p->loff;
    o[0] = 0;                                                   // U
    o[1] = o[0] + a16((size_t)mslot * I * 4);                   // X
    o[2] = o[1] + a16((size_t)2 * mux * I * 4);                 // F
    o[3] = o[2] + a16((size_t)mF * 4);                          // subsystems
    o[4] = o[3] + a16((size_t)msub * sizeof(int4));             // global items
    o[5] = o[4] + a16((size_t)mg * sizeof(int4));               // copies
    o[6] = o[5] + a16((size_t)mcp * 4);                         // exchange row per slot
    o[7] = o[6] + a16((size_t)mslot * 4);                       // global per slot
    o[8] = o[7] + a16((size_t)mslot * 4);                       // 1 / (rho N)
    o[9] = o[8] + a16((size_t)kBatchRecip * 4);                 // test sums per item group
    o[10] = o[9] + a16((size_t)WG * 6 * I * 8);                 // test sums of the CTA
    o[11] = o[10] + a16((size_t)6 * I * 8);                     // flags
    p->bytes = o[11] + a16((size_t)2 * I * 4);
    if (p->bytes > kMaxSmem) { set_last_error("lane plan: shared memory"); return OPF_E_CAPACITY; }
    // one CTA per SM: CTAs of one cluster sharing an SM could each wait in
    // the tensor-memory allocation for columns another one holds until the
    // cluster's first barrier, which that one cannot pass
    p->bytes = std::max(p->bytes, kMaxSmem / 2 + 1024u);
    p->lane_nslm = mslot;
    p->tm_cols = 32;
    while (p->tm_cols < 2 * mslot) p->tm_cols <<= 1;
    if (p->tm_cols > 512) { set_last_error("lane plan: tensor-memory columns"); return OPF_E_CAPACITY; }
    p->tm = true;
    p->lane_C = C;
    p->lane_maxux = mux;
    if (lane_engine_prepare(C, p->bytes)) { set_last_error("lane plan: engine attributes"); return OPF_E_CUDA; }
    if (lane_engine_ctas_per_sm(p->threads, p->bytes) != 1) {
        set_last_error("lane plan: the engine needs an SM to itself");
        return OPF_E_CAPACITY;
    }
    if (lane_engine_max_clusters(C, p->threads, p->bytes) < 1) {
        set_last_error("lane plan: a cluster of this shape does not fit the device");
        return OPF_E_CAPACITY;
    }
    p->NCH = NCH;
    p->nF = fo;
    p->n_tasks = 0;
    p->NB = b->NB;
    p->C = (b->n + kLaneInst - 1) / kLaneInst;
    std::vector<int> inst((size_t)p->C * kLaneInst, -1), ipos(b->n);
    for (int i = 0; i < b->n; ++i) { inst[i] = i; ipos[i] = i; }
    std::vector<void *> &A = p->allocs;
    BTRY(bupload(A, &p->d_lparts, parts, st));
    BTRY(bupload(A, &p->d_lsub, lsub, st));
    BTRY(bupload(A, &p->d_lgi, lgi, st));
    BTRY(bupload(A, &p->d_lcp, lcp, st));
    BTRY(bupload(A, &p->d_lux, lux, st));
    BTRY(bupload(A, &p->d_lgk, lgk, st));
    BTRY(bupload(A, &p->d_sch, sch, st));
    BTRY(bupload(A, &p->d_inst, inst, st));
    BTRY(bupload(A, &p->d_ipos, ipos, st));
    int4 *d_fdesc = nullptr;
    BTRY(bupload(A, &d_fdesc, fdesc, st));
    const size_t nslot = (size_t)p->C * NCH * kLaneInst * 4, nglob = (size_t)p->C * G * kLaneInst;
    const size_t nbnd = (size_t)p->C * std::max(p->NB, 1) * kLaneInst;
    auto arr = [&](void **q, size_t n) -> int {
        float *t;
        BTRY(balloc(A, &t, n));
        *q = t;
        BCUDA(cudaMemsetAsync(t, 0, n * sizeof(float), st));
        return OPF_OK;
    };
    BTRY(arr(&p->d_F, (size_t)std::max(fo, 4)));
    BTRY(arr(&p->d_recip, (size_t)kBatchRecip));
    BTRY(arr(&p->d_cost, (size_t)G));
    BTRY(arr(&p->mu, nslot)); BTRY(arr(&p->ds, nslot)); BTRY(arr(&p->bt, nslot)); BTRY(arr(&p->lref, nslot));
    BTRY(arr(&p->xo, nglob)); BTRY(arr(&p->ct, nglob)); BTRY(arr(&p->xrf, nglob));
    BTRY(arr(&p->lbt, nbnd)); BTRY(arr(&p->ubt, nbnd)); BTRY(arr(&p->cbt, nbnd));
    launch_lpack((int)fdesc.size(), d_fdesc, h->d_sub, h->d_sub2, h->d_F64, (float *)p->d_F, st);
    BCUDA(cudaGetLastError());
    {
        std::vector<float> c32(h->model.c.begin(), h->model.c.end());
        BCUDA(cudaMemcpyAsync(p->d_cost, c32.data(), G * sizeof(float), cudaMemcpyHostToDevice, st));
        BCUDA(cudaStreamSynchronize(st));
    }
    p->rho = -1.0;
    p->lane = true;
    p->ok = true;
    return OPF_OK;
}

LaneArgs lane_args(opf_batch *b, const BPlan &p, double rho) {
    LaneArgs a;
    memset(&a, 0, sizeof(a));
    a.C = p.lane_C;
    a.WG = p.W / 4;
    a.G = b->G;
    a.NB = p.NB;
    a.NCH = p.NCH;
    a.nslm = p.lane_nslm;
    a.tm_cols = p.tm_cols;
    a.maxux = p.lane_maxux;
    a.off_U = p.loff[0]; a.off_X = p.loff[1]; a.off_F = p.loff[2]; a.off_sub = p.loff[3];
    a.off_gi = p.loff[4]; a.off_cp = p.loff[5]; a.off_ux = p.loff[6]; a.off_gk = p.loff[7];
    a.off_rc = p.loff[8]; a.off_red = p.loff[9]; a.off_part = p.loff[10]; a.off_flag = p.loff[11];
    a.parts = p.d_lparts;
    a.sub = p.d_lsub;
    a.gi = p.d_lgi;
    a.cp = p.d_lcp;
    a.ux = p.d_lux;
    a.gk = p.d_lgk;
    a.F = (const float *)p.d_F;
    a.recip = (const float *)p.d_recip;
    a.cost = (const float *)p.d_cost;
    a.mu = (float *)p.mu; a.ds = (float *)p.ds; a.xo = (float *)p.xo;
    a.bt = (const float *)p.bt; a.lref = (const float *)p.lref; a.ct = (const float *)p.ct;
    a.xrf = (const float *)p.xrf; a.lbt = (const float *)p.lbt; a.ubt = (const float *)p.ubt;
    a.inst = p.d_inst;
    a.st = b->d_st;
    a.rho = (float)rho;
    a.inv_rho = (float)(1.0 / rho);
    a.rho_d = rho;
    return a;
}

}  // namespace bx
}  // namespace opf
