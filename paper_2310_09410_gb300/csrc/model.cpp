// Host construction of the consensus LP (Eq. OurModel) from a radial feeder.
//
// Rows follow Sec. II-A: power balance per bus phase (Eq. balance_eqns), the
// voltage-dependent load model (VDLM-1..5 for wye loads; for delta loads the
// bus-side powers of each delta branch, which is what VDLM-6..10 encode), and
// the linearized line flow (Eq. power_flow_eqns).  The decomposition is the
// one of Sec. V-A: a subsystem per bus and per line, a leaf bus merged into
// the line that feeds it.
//
// The 3x3 matrices M^p and M^q and the delta-load coupling are evaluated here
// from phasors with balanced 120-degree angles (theta_a = 0, theta_b = -120,
// theta_c = +120 degrees):
//   M^p_{ph,ps} = -2 Re(conj(z_{ph,ps}) g),  M^q_{ph,ps} = -2 Re(j conj(z_{ph,ps}) g),
//   g = exp(j (theta_ph - theta_ps)),
// which reproduces the two matrices printed under Eq. power_flow_eqns; a delta
// branch (ph, ps) carrying s^d draws s^d V_ph / (V_ph - V_ps) at phase ph and
// -s^d V_ps / (V_ph - V_ps) at phase ps.
#include <algorithm>
#include <cmath>
#include <complex>
#include <map>
#include <set>

#include "opf_internal.h"

namespace opf {

namespace {

using cplx = std::complex<double>;
const double kTheta[3] = {0.0, -2.0 * M_PI / 3.0, 2.0 * M_PI / 3.0};

inline int popc(unsigned m) { return __builtin_popcount(m & 7u); }
// position of phase p inside mask m (number of lower phases present)
inline int pos(unsigned m, int p) { return popc(m & ((1u << p) - 1u)); }
inline bool has(unsigned m, int p) { return (m >> p) & 1u; }

struct Row {
    std::vector<std::pair<int, double>> a;
    double rhs = 0.0;
    int src = -1;          // rhs = coef * (load value src), see HostSub::rsrc
    double coef = 0.0;
    int avar = -1;         // variable whose coefficient is acoef * (load value src)
    double acoef = 0.0;
    void add(int v, double x) { a.emplace_back(v, x); }
};

struct Index {
    std::vector<int> gen, bus, load, line;   // first variable of each component
};

}  // namespace

static int fail(std::string *err, const std::string &msg, int code = OPF_E_INVALID) {
    if (err) *err = msg;
    return code;
}

int build_feeder_model(const opf_feeder *f, HostModel *out, std::string *err) {
    if (!f || !out) return fail(err, "null feeder");
    const int nb = f->n_bus, nl = f->n_line, nd = f->n_load, ng = f->n_gen;
    if (nb < 2 || nl != nb - 1 || nd < 0 || ng < 0)
        return fail(err, "need n_bus >= 2, n_line == n_bus - 1, n_load >= 0, n_gen >= 0");
    if (!f->bus_phases || !f->bus_wmin || !f->bus_wmax || !f->line_from || !f->line_to ||
        !f->line_phases || !f->line_r || !f->line_x || (nd && (!f->load_bus || !f->load_phases ||
        !f->load_a || !f->load_b)) || (ng && (!f->gen_bus || !f->gen_phases || !f->gen_pmin ||
        !f->gen_pmax || !f->gen_qmin || !f->gen_qmax || !f->gen_cost)))
        return fail(err, "missing required feeder array");

    // ---- topology checks: a tree rooted at bus 0
    std::vector<int> in_line(nb, -1), parent(nb, -1);
    std::vector<std::vector<int>> out_lines(nb), loads_at(nb), gens_at(nb);
    for (int e = 0; e < nl; ++e) {
        int i = f->line_from[e], j = f->line_to[e];
        if (i < 0 || i >= nb || j <= 0 || j >= nb || i == j) return fail(err, "line endpoint out of range");
        if (in_line[j] >= 0) return fail(err, "a bus has two incoming lines");
        in_line[j] = e;
        parent[j] = i;
        out_lines[i].push_back(e);
        unsigned lm = f->line_phases[e] & 7u;
        if (!lm || (lm & ~(unsigned)f->bus_phases[i])) return fail(err, "line phases not within its from-bus");
        if ((unsigned)(f->bus_phases[j] & 7u) != lm) return fail(err, "bus phases differ from its incoming line");
    }
    if ((f->bus_phases[0] & 7u) == 0) return fail(err, "substation has no phase");
    for (int j = 1; j < nb; ++j) {
        int steps = 0;
        for (int k = j; k != 0; k = parent[k]) {
            if (k < 0 || ++steps > nb) return fail(err, "lines do not form a tree rooted at bus 0");
        }
    }
    for (int l = 0; l < nd; ++l) {
        int i = f->load_bus[l];
        if (i < 0 || i >= nb) return fail(err, "load bus out of range");
        unsigned m = f->load_phases[l] & 7u;
        if (!m || (m & ~(unsigned)f->bus_phases[i])) return fail(err, "load phases not within its bus");
        if (f->load_delta && f->load_delta[l] && m != 7u) return fail(err, "delta load needs three phases");
        loads_at[i].push_back(l);
    }
    for (int k = 0; k < ng; ++k) {
        int i = f->gen_bus[k];
        if (i < 0 || i >= nb) return fail(err, "generator bus out of range");
        unsigned m = f->gen_phases[k] & 7u;
        if (!m || (m & ~(unsigned)f->bus_phases[i])) return fail(err, "generator phases not within its bus");
        gens_at[i].push_back(k);
    }
    auto arr3 = [](const double *p, int comp, int ph, double dflt) { return p ? p[3 * comp + ph] : dflt; };

    // ---- global variables, canonical order
    HostModel &M = *out;
    M = HostModel();
    Index ix;
    int nv = 0;
    auto push = [&](double lo, double hi, double cost, uint8_t v) {
        M.lb.push_back(lo); M.ub.push_back(hi); M.c.push_back(cost); M.volt.push_back(v);
        return nv++;
    };
    const double inf = INFINITY;
    ix.gen.resize(ng);
    for (int k = 0; k < ng; ++k) {
        ix.gen[k] = nv;
        unsigned m = f->gen_phases[k] & 7u;
        for (int p = 0; p < 3; ++p) if (has(m, p)) {
            push(f->gen_pmin[3 * k + p], f->gen_pmax[3 * k + p], f->gen_cost[k], 0);
            push(f->gen_qmin[3 * k + p], f->gen_qmax[3 * k + p], 0.0, 0);
        }
    }
    ix.bus.resize(nb);
    for (int i = 0; i < nb; ++i) {
        ix.bus[i] = nv;
        for (int p = 0; p < 3; ++p) if (has(f->bus_phases[i], p))
            push(f->bus_wmin[3 * i + p], f->bus_wmax[3 * i + p], 0.0, 1);
    }
    ix.load.resize(nd);
    for (int l = 0; l < nd; ++l) {
        ix.load[l] = nv;
        for (int p = 0; p < 3; ++p) if (has(f->load_phases[l], p))
            for (int q = 0; q < 4; ++q) push(-inf, inf, 0.0, 0);
    }
    ix.line.resize(nl);
    for (int e = 0; e < nl; ++e) {
        ix.line[e] = nv;
        for (int p = 0; p < 3; ++p) if (has(f->line_phases[e], p))
            for (int q = 0; q < 4; ++q) push(-inf, inf, 0.0, 0);
    }
    M.n = nv;
    M.n_load = nd;
    for (int v = 0; v < nv; ++v)
        if (!(M.lb[v] <= M.ub[v]) || std::isnan(M.c[v])) return fail(err, "empty or NaN bound / cost");

    auto vgen = [&](int k, int p, int q) { return ix.gen[k] + 2 * pos(f->gen_phases[k], p) + q; };
    auto vbus = [&](int i, int p) { return ix.bus[i] + pos(f->bus_phases[i], p); };
    auto vload = [&](int l, int p, int q) { return ix.load[l] + 4 * pos(f->load_phases[l], p) + q; };
    auto vline = [&](int e, int p, int q) { return ix.line[e] + 4 * pos(f->line_phases[e], p) + q; };
    enum { PB = 0, QB = 1, PD = 2, QD = 3 };
    enum { PIJ = 0, QIJ = 1, PJI = 2, QJI = 3 };

    // ---- row generators
    auto bus_rows = [&](int i, std::vector<Row> &rows, std::set<int> &vars) {
        unsigned bm = f->bus_phases[i] & 7u;
        for (int p = 0; p < 3; ++p) {
            if (!has(bm, p)) continue;
            Row rp, rq;
            int w = vbus(i, p);
            vars.insert(w);
            for (int e : out_lines[i]) if (has(f->line_phases[e], p)) {
                rp.add(vline(e, p, PIJ), 1.0); rq.add(vline(e, p, QIJ), 1.0);
            }
            if (i != 0) {
                int e = in_line[i];
                rp.add(vline(e, p, PJI), 1.0); rq.add(vline(e, p, QJI), 1.0);
            }
            for (int l : loads_at[i]) if (has(f->load_phases[l], p)) {
                rp.add(vload(l, p, PB), 1.0); rq.add(vload(l, p, QB), 1.0);
            }
            rp.add(w, arr3(f->bus_gsh, i, p, 0.0));
            rq.add(w, -arr3(f->bus_bsh, i, p, 0.0));
            for (int k : gens_at[i]) if (has(f->gen_phases[k], p)) {
                rp.add(vgen(k, p, 0), -1.0); rq.add(vgen(k, p, 1), -1.0);
            }
            for (auto &t : rp.a) vars.insert(t.first);
            for (auto &t : rq.a) vars.insert(t.first);
            rows.push_back(rp); rows.push_back(rq);
        }
        for (int l : loads_at[i]) {
            unsigned lm = f->load_phases[l] & 7u;
            bool delta = f->load_delta && f->load_delta[l];
            double wscale = delta ? 3.0 : 1.0;
            for (int p = 0; p < 3; ++p) {
                if (!has(lm, p)) continue;
                for (int q = 0; q < 4; ++q) vars.insert(vload(l, p, q));
                double a = f->load_a[3 * l + p], b = f->load_b[3 * l + p];
                double al = arr3(f->load_alpha, l, p, 0.0), be = arr3(f->load_beta, l, p, 0.0);
                // p^d linear in w_hat around w_hat = 1 with slope a*alpha/2
                Row r1; r1.add(vload(l, p, PD), 1.0); r1.add(vbus(i, p), -0.5 * a * al * wscale);
                r1.rhs = a * (1.0 - 0.5 * al);
                r1.src = 2 * (3 * l + p); r1.coef = 1.0 - 0.5 * al;
                if (al != 0.0) { r1.avar = vbus(i, p); r1.acoef = -0.5 * al * wscale; }
                Row r2; r2.add(vload(l, p, QD), 1.0); r2.add(vbus(i, p), -0.5 * b * be * wscale);
                r2.rhs = b * (1.0 - 0.5 * be);
                r2.src = 2 * (3 * l + p) + 1; r2.coef = 1.0 - 0.5 * be;
                if (be != 0.0) { r2.avar = vbus(i, p); r2.acoef = -0.5 * be * wscale; }
                if (al != 0.0 || be != 0.0) M.A_depends_on_loads = true;
                rows.push_back(r1); rows.push_back(r2);
            }
            if (!delta) {
                for (int p = 0; p < 3; ++p) if (has(lm, p)) {
                    Row r; r.add(vload(l, p, PB), 1.0); r.add(vload(l, p, PD), -1.0); rows.push_back(r);
                    Row s; s.add(vload(l, p, QB), 1.0); s.add(vload(l, p, QD), -1.0); rows.push_back(s);
                }
            } else {
                // bus-side power of phase ph = sum over branches d of T[ph][d] * s^d_d
                const int br[3][2] = {{0, 1}, {1, 2}, {2, 0}};   // ab, bc, ca
                cplx V[3];
                for (int p = 0; p < 3; ++p) V[p] = std::polar(1.0, kTheta[p]);
                cplx T[3][3] = {};
                for (int d = 0; d < 3; ++d) {
                    int a_ = br[d][0], b_ = br[d][1];
                    cplx vb = V[a_] - V[b_];
                    T[a_][d] += V[a_] / vb;
                    T[b_][d] -= V[b_] / vb;
                }
                for (int p = 0; p < 3; ++p) {
                    Row re, im;
                    re.add(vload(l, p, PB), 1.0); im.add(vload(l, p, QB), 1.0);
                    for (int d = 0; d < 3; ++d) {
                        re.add(vload(l, d, PD), -T[p][d].real()); re.add(vload(l, d, QD), T[p][d].imag());
                        im.add(vload(l, d, PD), -T[p][d].imag()); im.add(vload(l, d, QD), -T[p][d].real());
                    }
                    rows.push_back(re); rows.push_back(im);
                }
            }
        }
    };
    auto line_rows = [&](int e, std::vector<Row> &rows, std::set<int> &vars) {
        int i = f->line_from[e], j = f->line_to[e];
        unsigned lm = f->line_phases[e] & 7u;
        const double *r = f->line_r + 9 * e, *x = f->line_x + 9 * e;
        for (int p = 0; p < 3; ++p) {
            if (!has(lm, p)) continue;
            for (int q = 0; q < 4; ++q) vars.insert(vline(e, p, q));
            vars.insert(vbus(i, p)); vars.insert(vbus(j, p));
            double gi = arr3(f->line_gs_from, e, p, 0.0), gj = arr3(f->line_gs_to, e, p, 0.0);
            double bi = arr3(f->line_bs_from, e, p, 0.0), bj = arr3(f->line_bs_to, e, p, 0.0);
            Row a; a.add(vline(e, p, PIJ), 1.0); a.add(vline(e, p, PJI), 1.0);
            a.add(vbus(i, p), -gi); a.add(vbus(j, p), -gj); rows.push_back(a);
            Row b; b.add(vline(e, p, QIJ), 1.0); b.add(vline(e, p, QJI), 1.0);
            b.add(vbus(i, p), bi); b.add(vbus(j, p), bj); rows.push_back(b);
            Row v; v.add(vbus(i, p), 1.0); v.add(vbus(j, p), -arr3(f->line_tap, e, p, 1.0));
            for (int s = 0; s < 3; ++s) {
                if (!has(lm, s)) continue;
                cplx z(r[3 * p + s], x[3 * p + s]);
                cplx g = std::polar(1.0, kTheta[p] - kTheta[s]);
                cplx w = std::conj(z) * g;
                double mp = -2.0 * w.real();
                double mq = -2.0 * (cplx(0.0, 1.0) * w).real();
                double gs = arr3(f->line_gs_from, e, s, 0.0), bs = arr3(f->line_bs_from, e, s, 0.0);
                v.add(vline(e, s, PIJ), mp);
                v.add(vbus(i, s), -mp * gs);
                v.add(vline(e, s, QIJ), mq);
                v.add(vbus(i, s), mq * bs);
            }
            rows.push_back(v);
        }
    };
    auto make_sub = [&](std::vector<Row> &rows, std::set<int> &vars) {
        HostSub s;
        s.vars.assign(vars.begin(), vars.end());
        s.n = (int)s.vars.size();
        s.m = (int)rows.size();
        s.A.assign((size_t)s.m * s.n, 0.0);
        s.b.resize(s.m);
        s.rsrc.resize(s.m);
        s.rcoef.resize(s.m);
        s.acol.assign(s.m, -1);
        s.acoef.assign(s.m, 0.0);
        std::map<int, int> col;
        for (int k = 0; k < s.n; ++k) col[s.vars[k]] = k;
        for (int r = 0; r < s.m; ++r) {
            for (auto &t : rows[r].a) s.A[(size_t)r * s.n + col.at(t.first)] += t.second;
            s.b[r] = rows[r].rhs;
            s.rsrc[r] = rows[r].src;
            s.rcoef[r] = rows[r].coef;
            if (rows[r].avar >= 0) {
                s.acol[r] = col.at(rows[r].avar);
                s.acoef[r] = rows[r].acoef;
            }
        }
        M.subs.push_back(std::move(s));
    };
    auto is_leaf = [&](int i) { return i != 0 && out_lines[i].empty(); };
    for (int i = 0; i < nb; ++i) {
        if (is_leaf(i)) continue;
        std::vector<Row> rows; std::set<int> vars;
        bus_rows(i, rows, vars);
        make_sub(rows, vars);
    }
    for (int e = 0; e < nl; ++e) {
        std::vector<Row> rows; std::set<int> vars;
        line_rows(e, rows, vars);
        int j = f->line_to[e];
        if (is_leaf(j)) bus_rows(j, rows, vars);
        make_sub(rows, vars);
    }
    for (auto &s : M.subs)
        if (s.n > OPF_MAX_NS) return fail(err, "subsystem larger than OPF_MAX_NS", OPF_E_CAPACITY);
    return OPF_OK;
}

int build_generic_model(int n, const double *c, const double *lb, const double *ub,
                        const uint8_t *volt, int S, const int *m_s, const int *n_s,
                        const double *A, const double *b, const int *idx,
                        HostModel *out, std::string *err) {
    if (n <= 0 || S <= 0 || !c || !lb || !ub || !m_s || !n_s || !idx)
        return fail(err, "generic model: need n > 0, S > 0 and the arrays");
    HostModel &M = *out;
    M = HostModel();
    M.n = n;
    M.c.assign(c, c + n);
    M.lb.assign(lb, lb + n);
    M.ub.assign(ub, ub + n);
    M.volt.assign(n, 0);
    if (volt) for (int i = 0; i < n; ++i) M.volt[i] = volt[i] ? 1 : 0;
    for (int i = 0; i < n; ++i)
        if (!(M.lb[i] <= M.ub[i]) || std::isnan(M.c[i])) return fail(err, "empty or NaN bound / cost");
    std::vector<int> covered(n, 0);
    size_t ao = 0, bo = 0, io = 0;
    for (int s = 0; s < S; ++s) {
        HostSub h;
        h.m = m_s[s];
        h.n = n_s[s];
        if (h.n <= 0 || h.m < 0) return fail(err, "subsystem with n_s <= 0 or m_s < 0");
        if (h.n > OPF_MAX_NS) return fail(err, "subsystem larger than OPF_MAX_NS", OPF_E_CAPACITY);
        if (h.m > 0 && (!A || !b)) return fail(err, "missing A or b");
        h.vars.assign(idx + io, idx + io + h.n);
        std::set<int> seen;
        for (int v : h.vars) {
            if (v < 0 || v >= n) return fail(err, "slot index out of range");
            if (!seen.insert(v).second) return fail(err, "global repeated inside a subsystem");
            covered[v] = 1;
        }
        if (h.m > 0) {
            h.A.assign(A + ao, A + ao + (size_t)h.m * h.n);
            h.b.assign(b + bo, b + bo + h.m);
        }
        for (double v : h.A) if (!std::isfinite(v)) return fail(err, "non-finite A");
        for (double v : h.b) if (!std::isfinite(v)) return fail(err, "non-finite b");
        ao += (size_t)h.m * h.n;
        bo += h.m;
        io += h.n;
        M.subs.push_back(std::move(h));
    }
    for (int i = 0; i < n; ++i)
        if (!covered[i]) return fail(err, "a global variable belongs to no subsystem");
    return OPF_OK;
}

}  // namespace opf
