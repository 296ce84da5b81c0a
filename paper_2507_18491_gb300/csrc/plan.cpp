// lmfmm_plan_check: the setup structures that the matvec kernels index, built
// with the same host code as lmfmm_build (classify_and_sort,
// build_host_structures, the matvec's work-item builder) on a context that
// never touches a device, then checked: tree nesting and point containment,
// the exact-once split of every (component, source leaf, target leaf) triple
// into far and near interactions (Sections 3.3 and 3.4.1: the FMM's partition of
// the double sum), the geometry of every far pair against its table's key, and
// the bounds of every index and range a kernel reads.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "kernels.cuh"

namespace {
using namespace lmf;

struct Check {
    int64_t n = 0;
    char first[256] = {0};
    void fail(const char *s)
    {
        if (n++ == 0) std::snprintf(first, sizeof first, "%s", s);
    }
    template <typename A0, typename... A>
    void fail(const char *fmt, A0 a0, A... a)
    {
        if (n++ == 0) std::snprintf(first, sizeof first, fmt, a0, a...);
    }
};

using ll = long long;

bool close_to(double a, double b, double scale) { return std::fabs(a - b) <= 1e-11 * scale; }

// coordinate magnitude of the point set: rounding of centres and their
// differences is relative to it, whatever the cell size
double coord_scale(const lmfmm_ctx *ctx)
{
    return ctx->root_h + std::fabs(ctx->root_c[0]) + std::fabs(ctx->root_c[1]) + std::fabs(ctx->root_c[2]);
}

// tree: levels partition each layer's points, children partition their parent,
// centres follow the cell indices, radii bound the points, leaves contain theirs
void check_tree(const lmfmm_ctx *ctx, Check &ck)
{
    const int L = ctx->med.L, D = ctx->depth;
    const int64_t N = ctx->N, nb = (int64_t)ctx->boxes.size();
    const double h = ctx->root_h;
    const double sc = coord_scale(ctx);
    int64_t p = 0;
    for (int l = 0; l <= L; ++l) {
        int64_t q = p;
        while (q < N && ctx->layer[ctx->perm[q]] == l) ++q;
        for (int lev = 0; lev <= D; ++lev) {
            const int64_t b0 = ctx->lvl0[l][lev], b1 = ctx->lvl1[l][lev];
            if (q == p) {
                if (b1 != b0) ck.fail("layer %d holds no points but has boxes at level %d", l, lev);
                continue;
            }
            if (b0 < 0 || b1 > nb || b0 >= b1) {
                ck.fail("layer %d level %d: box range [%lld, %lld) outside [0, %lld)", l, lev, (ll)b0, (ll)b1,
                        (ll)nb);
                continue;
            }
            if (lev == 0 && b1 - b0 != 1) ck.fail("layer %d: %lld root boxes", l, (ll)(b1 - b0));
            const double Sl = 2.0 * h / (double)(1u << lev);
            int64_t expect = p;
            for (int64_t b = b0; b < b1; ++b) {
                const Box &B = ctx->boxes[b];
                if (B.level != lev || B.layer != l) ck.fail("box %lld: level/layer %d/%d, expected %d/%d", (ll)b,
                                                            B.level, B.layer, lev, l);
                if (B.p0 != expect || B.p1 <= B.p0 || B.p1 > q) {
                    ck.fail("box %lld: points [%lld, %lld) break the partition of layer %d at %lld", (ll)b,
                            (ll)B.p0, (ll)B.p1, l, (ll)expect);
                    break;
                }
                expect = B.p1;
                const int ic[3] = {B.ix, B.iy, B.iz};
                for (int a = 0; a < 3; ++a)
                    if (!close_to(B.c[a], ctx->root_c[a] - h + (ic[a] + 0.5) * Sl, sc))
                        ck.fail("box %lld: centre %d is not its cell's", (ll)b, a);
                if (lev > 0) {
                    const int64_t pb = B.parent;
                    if (pb < ctx->lvl0[l][lev - 1] || pb >= ctx->lvl1[l][lev - 1]) {
                        ck.fail("box %lld: parent %lld not on level %d of layer %d", (ll)b, (ll)pb, lev - 1, l);
                    } else {
                        const Box &Pb = ctx->boxes[pb];
                        if ((B.key >> 3) != Pb.key || b < Pb.child0 || b >= Pb.child0 + Pb.nchild ||
                            B.p0 < Pb.p0 || B.p1 > Pb.p1)
                            ck.fail("box %lld: not a child of its parent %lld", (ll)b, (ll)pb);
                    }
                } else if (B.parent != -1) {
                    ck.fail("root box %lld has a parent", (ll)b);
                }
                if (lev == D) {
                    if (B.nchild != 0 || B.child0 != -1) ck.fail("leaf %lld has children", (ll)b);
                } else if (B.nchild < 1 || B.child0 < ctx->lvl0[l][lev + 1] ||
                           B.child0 + B.nchild > ctx->lvl1[l][lev + 1] || ctx->boxes[B.child0].p0 != B.p0 ||
                           ctx->boxes[B.child0 + B.nchild - 1].p1 != B.p1) {
                    ck.fail("box %lld: children do not partition its points", (ll)b);
                }
                double r2 = 0;
                for (int64_t t = B.p0; t < B.p1; ++t) {
                    if (ctx->layer[ctx->perm[t]] != l) ck.fail("sorted point %lld is not in layer %d", (ll)t, l);
                    double dd = 0;
                    for (int a = 0; a < 3; ++a) {
                        const double v = ctx->sxyz[3 * t + a] - B.c[a];
                        dd += v * v;
                        if (lev == D && std::fabs(v) > 0.5 * Sl + 1e-12 * sc)
                            ck.fail("point %lld lies outside its leaf %lld", (ll)t, (ll)b);
                    }
                    r2 = std::max(r2, dd);
                }
                if (std::sqrt(r2) > B.r * (1 + 1e-12) + 1e-300) ck.fail("box %lld: radius below its points'", (ll)b);
            }
            if (expect != q && expect != -1)
                ck.fail("layer %d level %d: boxes end at point %lld, the layer at %lld", l, lev, (ll)expect, (ll)q);
        }
        p = q;
    }
    if (p != N) ck.fail("sorted points are not grouped by layer (%lld of %lld)", (ll)p, (ll)N);
}

// leaves under box b: [lo, hi) in the leaf order of its layer
bool leaf_range(const lmfmm_ctx *ctx, int64_t b, int64_t &lo, int64_t &hi)
{
    const int D = ctx->depth;
    const int64_t nb = (int64_t)ctx->boxes.size();
    if (b < 0 || b >= nb) return false;
    const int l = ctx->boxes[b].layer;
    int64_t x = b, y = b;
    for (int it = 0; it <= D && ctx->boxes[x].level < D; ++it) {
        x = ctx->boxes[x].child0;
        if (x < 0 || x >= nb) return false;
    }
    for (int it = 0; it <= D && ctx->boxes[y].level < D; ++it) {
        y = ctx->boxes[y].child0 + ctx->boxes[y].nchild - 1;
        if (y < 0 || y >= nb) return false;
    }
    if (ctx->boxes[x].level != D || ctx->boxes[y].level != D) return false;
    lo = x - ctx->lvl0[l][D];
    hi = y - ctx->lvl0[l][D] + 1;
    return lo >= 0 && hi > lo;
}

// every far pair against its geometry's key, admissibility and direction; the
// geometries' pair ranges tile the pair array
void check_geometries(const lmfmm_ctx *ctx, Check &ck)
{
    const int64_t nb = (int64_t)ctx->boxes.size(), npair = (int64_t)ctx->m2l.size();
    const double h = ctx->root_h, theta = ctx->prm.theta, eta = ctx->prm.eta;
    const int nrc = ctx->n_react_comps, ncomp = (int)ctx->comps.size();
    const double sc = coord_scale(ctx);
    int64_t expect = 0;
    for (size_t gi = 0; gi < ctx->geoms.size(); ++gi) {
        const Geom &G = ctx->geoms[gi];
        if (G.pair0 != expect || G.pair1 < G.pair0 || G.pair1 > npair) {
            ck.fail("geometry %lld: pairs [%lld, %lld) do not continue at %lld", (ll)gi, (ll)G.pair0, (ll)G.pair1,
                    (ll)expect);
            expect = std::max(expect, std::min<int64_t>(G.pair1, npair));
            if (G.pair0 < 0 || G.pair1 > npair || G.pair1 < G.pair0) continue;
        } else {
            expect = G.pair1;
        }
        const bool react = gi < ctx->n_react_geoms;
        if (G.comp < 0 || G.comp >= ncomp || react != (G.comp < nrc)) {
            ck.fail("geometry %lld: component %d out of range", (ll)gi, G.comp);
            continue;
        }
        const CompDev &c = ctx->comps[G.comp];
        const double Sl = 2.0 * h / (double)(1u << G.level) + sc;   // tolerance scale
        for (int64_t q = G.pair0; q < G.pair1; ++q) {
            const M2LPair &mp = ctx->m2l[q];
            if (mp.src < 0 || mp.src >= nb || mp.tgt < 0 || mp.tgt >= nb) {
                ck.fail("far pair %lld: box index out of range", (ll)q);
                continue;
            }
            const Box &B = ctx->boxes[mp.src], &C = ctx->boxes[mp.tgt];
            if (B.level != G.level || C.level != G.level || B.layer != c.l || C.layer != c.lp)
                ck.fail("far pair %lld: boxes not on level %d of layers %d -> %d", (ll)q, G.level, c.l, c.lp);
            const double dx = B.c[0] - C.c[0], dy = B.c[1] - C.c[1], rr = std::sqrt(dx * dx + dy * dy);
            if (!close_to(rr, G.rho, Sl)) ck.fail("far pair %lld: rho %.17g, its table's %.17g", (ll)q, rr, G.rho);
            const double ex = rr > 0 ? dx / rr : 1.0, ey = rr > 0 ? dy / rr : 0.0;
            if (!close_to(mp.cphi, ex, 1.0) || !close_to(mp.sphi, ey, 1.0))
                ck.fail("far pair %lld: direction is not that of c_s - c_t", (ll)q);
            double zs, zt;
            if (react) {
                zs = comp_src_z(c, B.c[2]);
                zt = comp_tgt_z(c, C.c[2]);
                const bool key_ok = c.l == c.lp ? close_to(zs - zt, G.zs - G.zt, Sl)
                                                : close_to(zs, G.zs, Sl) && close_to(zt, G.zt, Sl);
                if (!key_ok) ck.fail("far pair %lld: mapped heights differ from its table's", (ll)q);
            } else {
                zs = B.c[2];
                zt = C.c[2];
                if (!close_to(zs - zt, G.zs - G.zt, Sl)) ck.fail("free far pair %lld: height offset", (ll)q);
                if (mp.src == mp.tgt) ck.fail("free far pair %lld: a box with itself", (ll)q);
            }
            const double dz = zs - zt, R = std::sqrt(dx * dx + dy * dy + dz * dz), vz = c.s * dz;
            const bool adm = (B.r + C.r <= theta * R * (1 + 1e-12)) &&
                             (!react || ((vz >= eta * R * (1 - 1e-12)) && vz > 0));
            if (!adm) ck.fail("far pair %lld fails the admissibility test", (ll)q);
        }
    }
    if (expect != npair) ck.fail("geometries cover %lld of %lld far pairs", (ll)expect, (ll)npair);
}

// near pairs: leaves of the right layers, coefficient offsets as a running sum
void check_near(const lmfmm_ctx *ctx, Check &ck)
{
    const int64_t nb = (int64_t)ctx->boxes.size();
    const int D = ctx->depth;
    int64_t run = 0;
    for (size_t i = 0; i < ctx->near.size(); ++i) {
        const NearPair &np = ctx->near[i];
        if (np.comp < 0 || np.comp >= ctx->n_react_comps || np.src < 0 || np.src >= nb || np.tgt < 0 ||
            np.tgt >= nb) {
            ck.fail("near pair %lld: index out of range", (ll)i);
            continue;
        }
        const Box &B = ctx->boxes[np.src], &C = ctx->boxes[np.tgt];
        const CompDev &c = ctx->comps[np.comp];
        if (B.level != D || C.level != D || B.layer != c.l || C.layer != c.lp)
            ck.fail("near pair %lld: not a leaf pair of layers %d -> %d", (ll)i, c.l, c.lp);
        if (np.coef0 != run) ck.fail("near pair %lld: coefficients at %lld, expected %lld", (ll)i, (ll)np.coef0, (ll)run);
        run += (B.p1 - B.p0) * (C.p1 - C.p0);
        if (!(np.dzmin > 0) || !(np.rhomax >= 0) || !std::isfinite(np.rhomax))
            ck.fail("near pair %lld: vertical separation %.3g, horizontal extent %.3g", (ll)i, np.dzmin, np.rhomax);
    }
    if (run != ctx->n_near_pp) ck.fail("near point pairs %lld, counted %lld", (ll)ctx->n_near_pp, (ll)run);
    int64_t runf = 0;
    for (size_t i = 0; i < ctx->free_near.size(); ++i) {
        const int64_t s = ctx->free_near[i].first, t = ctx->free_near[i].second;
        if (s < 0 || s >= nb || t < 0 || t >= nb) {
            ck.fail("free near pair %lld: index out of range", (ll)i);
            continue;
        }
        const Box &B = ctx->boxes[s], &C = ctx->boxes[t];
        if (B.level != D || C.level != D || B.layer != C.layer) ck.fail("free near pair %lld: not a leaf pair of one layer", (ll)i);
        runf += (B.p1 - B.p0) * (C.p1 - C.p0);
    }
    if (runf != ctx->n_free_pp) ck.fail("free near point pairs %lld, counted %lld", (ll)ctx->n_free_pp, (ll)runf);
}

// every (component, source leaf, target leaf) triple reached exactly once: per
// target leaf, the source-leaf intervals of the far pairs of its ancestors and of
// its near pairs, sorted, must tile [0, source leaves) without gap or overlap
void check_coverage(const lmfmm_ctx *ctx, Check &ck, int64_t &checked, int &unchecked)
{
    const int D = ctx->depth;
    const int64_t nb = (int64_t)ctx->boxes.size();
    struct Iv {
        int64_t t, s0, s1;
    };
    std::vector<Iv> iv;
    for (int ci = 0; ci < (int)ctx->comps.size(); ++ci) {
        const CompDev &c = ctx->comps[ci];
        const bool react = ci < ctx->n_react_comps;
        const int64_t ns = ctx->lvl1[c.l][D] - ctx->lvl0[c.l][D], nt = ctx->lvl1[c.lp][D] - ctx->lvl0[c.lp][D];
        if (ns <= 0 || nt <= 0) {
            ck.fail("component %d: a layer without leaves", ci);
            continue;
        }
        // intervals: one per (far pair, target leaf under its target box) and per near pair
        int64_t m = 0;
        for (const Geom &G : ctx->geoms)
            if (G.comp == ci && G.pair0 >= 0 && G.pair1 <= (int64_t)ctx->m2l.size())
                for (int64_t q = G.pair0; q < G.pair1; ++q) {
                    int64_t t0, t1;
                    if (leaf_range(ctx, ctx->m2l[q].tgt, t0, t1)) m += t1 - t0;
                }
        m += react ? (int64_t)ctx->near.size() : (int64_t)ctx->free_near.size();
        if (m > ((int64_t)1 << 25)) {
            ++unchecked;
            continue;
        }
        iv.clear();
        iv.reserve((size_t)m);
        for (size_t gi = 0; gi < ctx->geoms.size(); ++gi) {
            const Geom &G = ctx->geoms[gi];
            if (G.comp != ci || G.pair0 < 0 || G.pair1 > (int64_t)ctx->m2l.size()) continue;
            for (int64_t q = G.pair0; q < G.pair1; ++q) {
                int64_t s0, s1, t0, t1;
                if (!leaf_range(ctx, ctx->m2l[q].src, s0, s1) || !leaf_range(ctx, ctx->m2l[q].tgt, t0, t1) ||
                    s1 > ns || t1 > nt || ctx->boxes[ctx->m2l[q].src].layer != c.l ||
                    ctx->boxes[ctx->m2l[q].tgt].layer != c.lp) {
                    ck.fail("far pair %lld: its leaves cannot be found", (ll)q);
                    continue;
                }
                for (int64_t t = t0; t < t1; ++t) iv.push_back({t, s0, s1});
            }
        }
        if (react) {
            for (const NearPair &np : ctx->near) {
                if (np.comp != ci || np.src < 0 || np.src >= nb || np.tgt < 0 || np.tgt >= nb) continue;
                const int64_t s = np.src - ctx->lvl0[c.l][D], t = np.tgt - ctx->lvl0[c.lp][D];
                if (s >= 0 && s < ns && t >= 0 && t < nt) iv.push_back({t, s, s + 1});
            }
        } else {
            for (const auto &pr : ctx->free_near) {
                if (pr.first < 0 || pr.first >= nb || ctx->boxes[pr.first].layer != c.l) continue;
                const int64_t s = pr.first - ctx->lvl0[c.l][D], t = pr.second - ctx->lvl0[c.lp][D];
                if (s >= 0 && s < ns && t >= 0 && t < nt) iv.push_back({t, s, s + 1});
            }
        }
        std::sort(iv.begin(), iv.end(), [](const Iv &a, const Iv &b) { return a.t != b.t ? a.t < b.t : a.s0 < b.s0; });
        // walk the targets in order; 'missed' and 'twice' count leaf pairs
        int64_t missed = 0, twice = 0, t_bad = -1, s_bad = -1;
        size_t e = 0;
        for (int64_t t = 0; t < nt; ++t) {
            int64_t reach = 0;   // sources [0, reach) reached so far for target t
            for (; e < iv.size() && iv[e].t == t; ++e) {
                const Iv &v = iv[e];
                if (v.s0 > reach) {
                    if (!missed && !twice) t_bad = t, s_bad = reach;
                    missed += v.s0 - reach;
                } else if (v.s0 < reach) {
                    if (!missed && !twice) t_bad = t, s_bad = v.s0;
                    twice += std::min(reach, v.s1) - v.s0;
                }
                reach = std::max(reach, v.s1);
            }
            if (reach < ns) {
                if (!missed && !twice) t_bad = t, s_bad = reach;
                missed += ns - reach;
            }
        }
        if (missed || twice) {
            ck.fail("component %d (layers %d -> %d): %lld leaf pairs reached 0 times, %lld more than once "
                    "(first: target leaf %lld, source leaf %lld)",
                    ci, c.l, c.lp, (ll)missed, (ll)twice, (ll)t_bad, (ll)s_bad);
            ck.n += missed + twice - 1;
        }
        checked += ns * nt;
    }
}

// M2M / L2L groups: (child, parent) pairs of one level, layer and octant whose
// centres differ by the group's vector; every non-root box is a child once
void check_translations(const lmfmm_ctx *ctx, Check &ck)
{
    const int64_t nb = (int64_t)ctx->boxes.size(), np = (int64_t)ctx->tpair_child.size();
    const double h = ctx->root_h;
    if ((int64_t)ctx->tpair_parent.size() != np) ck.fail("translation pair arrays differ in length");
    std::vector<uint8_t> seen((size_t)nb, 0);
    int64_t expect = 0;
    for (size_t gi = 0; gi < ctx->tgroups.size(); ++gi) {
        const TransGroup &g = ctx->tgroups[gi];
        if (g.pair0 != expect || g.pair1 < g.pair0 || g.pair1 > np || g.level < 1 || g.level > ctx->depth) {
            ck.fail("translation group %lld: pairs [%lld, %lld) or level %d out of place", (ll)gi, (ll)g.pair0,
                    (ll)g.pair1, g.level);
            break;
        }
        expect = g.pair1;
        const double Sc = 2.0 * h / (double)(1u << g.level) + coord_scale(ctx);   // tolerance scale
        for (int64_t q = g.pair0; q < g.pair1; ++q) {
            const int64_t cb = ctx->tpair_child[q], pb = q < (int64_t)ctx->tpair_parent.size() ? ctx->tpair_parent[q] : -1;
            if (cb < 0 || cb >= nb || pb < 0 || pb >= nb) {
                ck.fail("translation pair %lld: index out of range", (ll)q);
                continue;
            }
            const Box &C = ctx->boxes[cb], &Pb = ctx->boxes[pb];
            if (C.level != g.level || C.layer != g.layer || (int)(C.key & 7) != g.octant || C.parent != pb)
                ck.fail("translation pair %lld: child %lld does not belong to its group", (ll)q, (ll)cb);
            for (int a = 0; a < 3; ++a)
                if (!close_to(C.c[a] - Pb.c[a], g.t[a], Sc)) ck.fail("translation pair %lld: vector", (ll)q);
            if (seen[(size_t)cb] < 255) ++seen[(size_t)cb];
        }
    }
    if (expect != np) ck.fail("translation groups cover %lld of %lld pairs", (ll)expect, (ll)np);
    for (int64_t b = 0; b < nb; ++b)
        if ((ctx->boxes[b].level > 0) != (seen[(size_t)b] == 1)) {
            ck.fail("box %lld is translated %d times", (ll)b, (int)seen[(size_t)b]);
            break;
        }
}

// work items: per geometry and table, consecutive runs of its pairs of at most
// 64 helical columns (one per pair for the (sigma5, 0) table, two for the others)
void check_work(const lmfmm_ctx *ctx, Check &ck, int64_t &nitems, int64_t &ncols)
{
    std::vector<M2LWork> mw;
    const int bn = 64;
    ncols = plan_work_items(ctx, bn, mw);
    nitems = (int64_t)mw.size();
    size_t w = 0;
    int64_t cols = 0;
    for (size_t gi = 0; gi < ctx->geoms.size(); ++gi) {
        const Geom &G = ctx->geoms[gi];
        for (int t = 0; t < NTAB; ++t) {
            const int per = t == 1 ? bn : bn / 2;
            for (int64_t q = G.pair0; q < G.pair1;) {
                if (w >= mw.size()) {
                    ck.fail("work items end before geometry %lld", (ll)gi);
                    return;
                }
                const M2LWork &W = mw[w++];
                if (W.geom != (int)gi || W.t != t || W.pair0 != q || W.npair < 1 || W.npair > per ||
                    W.pair0 + W.npair > G.pair1) {
                    ck.fail("work item %lld does not continue geometry %lld, table %d at pair %lld", (ll)(w - 1),
                            (ll)gi, t, (ll)q);
                    return;
                }
                q += W.npair;
                cols += (int64_t)W.npair * (t == 1 ? 1 : 2);
            }
        }
    }
    if (w != mw.size()) ck.fail("%lld work items beyond the geometries", (ll)(mw.size() - w));
    if (cols != ncols) ck.fail("work items hold %lld columns, the builder counted %lld", (ll)cols, (ll)ncols);
}

}  // namespace

extern "C" lmfmm_status lmfmm_plan_check(const lmfmm_params *prm, int L, const double *d, const lmfmm_c128 *k,
                                         int64_t N, const double *xyz, int flags, lmfmm_plan_info *out)
{
    if (!out) return LMFMM_ERR_ARG;
    std::memset(out, 0, sizeof *out);
    auto msg = [&](const std::string &s) { std::snprintf(out->message, sizeof out->message, "%s", s.c_str()); };
    if (!prm) {
        msg("plan_check: NULL params");
        return LMFMM_ERR_ARG;
    }
    if (prm->p < 1 || prm->p > 16 || !(prm->theta > 0 && prm->theta < 1) || !(prm->eta >= 0) || prm->depth > 20 ||
        (prm->depth < 0 && prm->leaf_cap < 1) || prm->components < LMFMM_REACTION || prm->components > LMFMM_TOTAL ||
        (flags & ~(LMFMM_PLAN_DROP_FAR_PAIR | LMFMM_PLAN_DROP_NEAR_PAIR))) {
        msg("plan_check: parameter out of range (1 <= p <= 16, 0 < theta < 1, eta >= 0, depth <= 20, "
            "components, flags)");
        return LMFMM_ERR_ARG;
    }
    lmfmm_ctx *ctx = new lmfmm_ctx();
    ctx->prm = *prm;
    lmfmm_status rc = lmfmm_set_layers(ctx, L, d, k);
    if (rc == LMFMM_OK) rc = lmfmm_set_points(ctx, N, xyz);
    if (rc == LMFMM_OK) rc = build_host_structures(ctx);
    if (rc != LMFMM_OK) {
        msg(ctx->err);
        delete ctx;
        return rc;
    }
    // test hooks: lose one far pair (the last of the first geometry that has any)
    // or the first near pair, keeping every range and offset consistent, so that
    // only the interaction it carried goes missing
    if (flags & LMFMM_PLAN_DROP_FAR_PAIR)
        for (size_t gi = 0; gi < ctx->geoms.size(); ++gi)
            if (ctx->geoms[gi].pair1 > ctx->geoms[gi].pair0) {
                ctx->m2l.erase(ctx->m2l.begin() + (ctx->geoms[gi].pair1 - 1));
                --ctx->geoms[gi].pair1;
                for (size_t gj = gi + 1; gj < ctx->geoms.size(); ++gj) {
                    --ctx->geoms[gj].pair0;
                    --ctx->geoms[gj].pair1;
                }
                break;
            }
    if ((flags & LMFMM_PLAN_DROP_NEAR_PAIR) && !ctx->near.empty()) {
        const NearPair np0 = ctx->near.front();
        const int64_t n0 = (ctx->boxes[np0.src].p1 - ctx->boxes[np0.src].p0) *
                           (ctx->boxes[np0.tgt].p1 - ctx->boxes[np0.tgt].p0);
        ctx->near.erase(ctx->near.begin());
        for (NearPair &np : ctx->near) np.coef0 -= n0;
        ctx->n_near_pp -= n0;
    }

    const int D = ctx->depth;
    out->depth = D;
    out->n_components = ctx->n_react_comps;
    out->n_free_components = (int)ctx->comps.size() - ctx->n_react_comps;
    out->n_boxes = (int64_t)ctx->boxes.size();
    for (int l = 0; l <= ctx->med.L && l < 9; ++l) out->n_leaves[l] = ctx->lvl1[l][D] - ctx->lvl0[l][D];
    std::vector<int64_t> per_cl((size_t)ctx->n_react_comps * (D + 1), 0);
    for (size_t gi = 0; gi < ctx->geoms.size(); ++gi) {
        const int64_t n = ctx->geoms[gi].pair1 - ctx->geoms[gi].pair0;
        if (gi < ctx->n_react_geoms) {
            out->n_geometries++;
            out->n_far_pairs += n;
            const int lev = ctx->geoms[gi].level, c = ctx->geoms[gi].comp;
            if (lev >= 0 && lev <= D && lev < 21 && c >= 0 && c < ctx->n_react_comps) {
                out->n_geometries_level[lev]++;
                const int64_t v = ++per_cl[(size_t)c * (D + 1) + lev];
                out->max_geometries_component_level = std::max(out->max_geometries_component_level, v);
            }
        } else {
            out->n_free_geometries++;
            out->n_free_far_pairs += n;
        }
    }
    out->n_near_pairs = (int64_t)ctx->near.size();
    out->n_near_point_pairs = ctx->n_near_pp;
    out->n_free_near_pairs = (int64_t)ctx->free_near.size();
    out->n_free_near_point_pairs = ctx->n_free_pp;
    out->n_translation_pairs = (int64_t)ctx->tpair_child.size();
    for (int a = 0; a < 3; ++a) out->root_center[a] = ctx->root_c[a];
    out->root_half = ctx->root_h;

    Check ck;
    check_tree(ctx, ck);
    const bool tree_ok = ck.n == 0;
    check_geometries(ctx, ck);
    check_near(ctx, ck);
    check_translations(ctx, ck);
    // the coverage walk descends child links: only on a consistent tree
    if (tree_ok) check_coverage(ctx, ck, out->n_leaf_pairs_checked, out->n_components_unchecked);
    check_work(ctx, ck, out->n_work_items, out->n_columns);
    out->n_violations = ck.n;
    if (ck.n) std::snprintf(out->message, sizeof out->message, "%s", ck.first);
    delete ctx;
    return ck.n ? LMFMM_ERR_INTERNAL : LMFMM_OK;
}

// Depth tuner: predicted matvec time per candidate leaf level from the host
// structures' counts and per-unit device costs.  Default costs (ns) are the
// GB300 measurements of the mixed form with the tensor-core M2L, M2M and L2L at
// p = 12 (four-layer N = 2^20 workload, depth 6: 8.79 ms of M2L over 109831 work
// items; 0.754 ms of near field over 2782511 point pairs; 0.551 ms of M2M + L2L
// over 37447 (child, parent) pairs; 1.154 ms of P2M, L2P and permutation over
// 2^20 points), scaled to other p by (P / 169)^2 for the M2L and translations
// and by P / 169 for the point terms.
extern "C" lmfmm_status lmfmm_plan_depth(const lmfmm_params *prm, int L, const double *d, const lmfmm_c128 *k,
                                         int64_t N, const double *xyz, int dmin, int dmax, const double *unit_ns,
                                         int *best, double *predicted_ms)
{
    if (!prm || !best || !predicted_ms || dmin < 0 || dmax < dmin || dmax > 10) return LMFMM_ERR_ARG;
    const double P = (double)((prm->p + 1) * (prm->p + 1)), r = P / 169.0;
    const double dflt[4] = {8.79e6 / 109831 * r * r, 0.754e6 / 2782511, 0.551e6 / 37447 * r * r,
                            1.154e6 / 1048576 * r};
    const double *u = unit_ns ? unit_ns : dflt;
    *best = -1;
    double best_ms = 0;
    for (int D = dmin; D <= dmax; ++D) {
        lmfmm_params q = *prm;
        q.depth = D;
        lmfmm_ctx *ctx = new lmfmm_ctx();
        ctx->prm = q;
        lmfmm_status rc = lmfmm_set_layers(ctx, L, d, k);
        if (rc == LMFMM_OK) rc = lmfmm_set_points(ctx, N, xyz);
        if (rc == LMFMM_OK) rc = build_host_structures(ctx);
        if (rc != LMFMM_OK) {
            delete ctx;
            return rc;
        }
        std::vector<M2LWork> mw;
        plan_work_items(ctx, 64, mw);
        const double ns = u[0] * (double)mw.size() + u[1] * (double)(ctx->n_near_pp + ctx->n_free_pp) +
                          u[2] * (double)ctx->tpair_child.size() + u[3] * (double)N;
        predicted_ms[D - dmin] = ns * 1e-6;
        if (*best < 0 || ns * 1e-6 < best_ms) {
            *best = D;
            best_ms = ns * 1e-6;
        }
        delete ctx;
    }
    return LMFMM_OK;
}

// The Chebyshev machinery of Appendices A and B exactly as the M2L tabulation
// builds it (host routines bcoef_table and gtensor), for unit tests of those
// routines against independent Legendre functions.
extern "C" lmfmm_status lmfmm_legendre_chebyshev(int p, double *B)
{
    if (p < 1 || p > 16 || !B) return LMFMM_ERR_ARG;
    std::vector<double> b;
    bcoef_table(p, (p + 1) / 2, b);
    std::copy(b.begin(), b.end(), B);
    return LMFMM_OK;
}

extern "C" lmfmm_status lmfmm_legendre_product(int p, lmfmm_c128 k, lmfmm_c128 kp, lmfmm_c128 *G)
{
    if (p < 1 || p > 16 || !G || (k.re == 0 && k.im == 0) || (kp.re == 0 && kp.im == 0) ||
        !std::isfinite(k.re) || !std::isfinite(k.im) || !std::isfinite(kp.re) || !std::isfinite(kp.im))
        return LMFMM_ERR_ARG;
    std::vector<double> b;
    const int KM = (p + 1) / 2;
    bcoef_table(p, KM, b);
    static_assert(sizeof(cd) == sizeof(lmfmm_c128), "complex layouts agree");
    gtensor(p, b, KM, zc(k.re, k.im), zc(kp.re, kp.im), reinterpret_cast<cd *>(G));
    return LMFMM_OK;
}
