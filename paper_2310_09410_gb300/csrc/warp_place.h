// Placement of the warp engine's work items on the warp slots of a cluster
// (host code, no CUDA).  Subsystem s takes nparts[s] warps, 1 or 2.  The two
// warps of a split subsystem must share a CTA and sit in slots 2k, 2k + 1, so
// that they are on different SM sub-partitions and meet at named barrier
// 1 + k.  Pairs go first, round-robin over the P CTAs (pair k: CTA k % P,
// slots 2 (k / P) and 2 (k / P) + 1); single warps follow in subsystem order,
// round-robin from CTA i % P, each in the lowest free slot of the first CTA
// with one.  With no pairs, subsystem s lands in CTA s % P, slot s / P.
#pragma once

#include <cstddef>
#include <vector>

namespace opf {

// Places the items on P CTAs of `warps` slots; false if they do not fit.
// cta_of[s] / slot_of[s]: CTA and first slot of subsystem s.
inline bool place_warp_items(const std::vector<int> &nparts, int P, int warps, std::vector<int> *cta_of,
                             std::vector<int> *slot_of) {
    const int S = (int)nparts.size();
    if (P < 1 || warps < 1) return false;
    cta_of->assign(S, 0);
    slot_of->assign(S, 0);
    std::vector<char> used((size_t)P * warps, 0);
    int k = 0;
    for (int s = 0; s < S; ++s) {
        if (nparts[s] != 2) continue;
        const int p = k % P, sl = 2 * (k / P);
        if (sl + 1 >= warps) return false;
        used[(size_t)p * warps + sl] = used[(size_t)p * warps + sl + 1] = 1;
        (*cta_of)[s] = p;
        (*slot_of)[s] = sl;
        ++k;
    }
    int i = 0;
    for (int s = 0; s < S; ++s) {
        if (nparts[s] != 1) continue;
        bool done = false;
        for (int t = 0; t < P && !done; ++t) {
            const int p = (i + t) % P;
            for (int sl = 0; sl < warps; ++sl)
                if (!used[(size_t)p * warps + sl]) {
                    used[(size_t)p * warps + sl] = 1;
                    (*cta_of)[s] = p;
                    (*slot_of)[s] = sl;
                    done = true;
                    break;
                }
        }
        if (!done) return false;
        ++i;
    }
    return true;
}

// The smallest slot count from ceil(W / P) up to max_warps at which the items
// fit; 0 if none does.
inline int place_warp_items_min(const std::vector<int> &nparts, int P, int max_warps, std::vector<int> *cta_of,
                                std::vector<int> *slot_of) {
    int W = 0;
    for (int x : nparts) W += x;
    for (int warps = (W + P - 1) / P; warps <= max_warps; ++warps)
        if (warps >= 1 && place_warp_items(nparts, P, warps, cta_of, slot_of)) return warps;
    return 0;
}

}  // namespace opf
