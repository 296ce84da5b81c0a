// Host-side setup: point classification and Morton sort, per-layer octrees
// on one global grid, enumeration of reaction components, dual-tree traversal
// of every component into far (M2L) and near box pairs, deduplication of M2L
// geometries, translation groups, and the Chebyshev coefficient tables of
// Section 3.4 / Appendices A-B.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <tuple>
#include <thread>
#include <unordered_map>

#include "internal.h"

namespace lmf {

static uint64_t spread3(uint64_t v)
{
    uint64_t r = 0;
    for (int b = 0; b < 21; ++b) r |= ((v >> b) & 1ull) << (3 * b);
    return r;
}
static uint32_t compact3(uint64_t v)
{
    uint32_t r = 0;
    for (int b = 0; b < 21; ++b) r |= (uint32_t)((v >> (3 * b)) & 1ull) << b;
    return r;
}
// key bit order: x in bit 2, y in bit 1, z in bit 0 of every triple
static uint64_t morton(uint32_t ix, uint32_t iy, uint32_t iz)
{
    return (spread3(ix) << 2) | (spread3(iy) << 1) | spread3(iz);
}

lmfmm_status classify_and_sort(lmfmm_ctx *ctx)
{
    const int64_t N = ctx->N;
    const int L = ctx->med.L;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a) {
            double v = ctx->xyz[3 * i + a];
            if (!std::isfinite(v)) {
                ctx->err = "point " + std::to_string(i) + " has a non-finite coordinate";
                return LMFMM_ERR_ARG;
            }
            lo[a] = std::min(lo[a], v);
            hi[a] = std::max(hi[a], v);
        }
    double ext = 0;
    for (int a = 0; a < 3; ++a) ext = std::max(ext, hi[a] - lo[a]);
    double scale = std::max(1.0, ext);
    ctx->layer.assign(N, 0);
    for (int64_t i = 0; i < N; ++i) {
        double z = ctx->xyz[3 * i + 2];
        int l = 0;
        for (int j = 0; j < L; ++j) {
            if (std::fabs(z - ctx->med.d[j]) < 1e-12 * scale) {
                ctx->err = "point " + std::to_string(i) + " lies on interface " + std::to_string(j);
                return LMFMM_ERR_ARG;
            }
            if (z < ctx->med.d[j]) l = j + 1;
        }
        ctx->layer[i] = l;
    }
    double h = 0.5 * ext * (1.0 + 1e-9) + 1e-9 * scale;
    if (h <= 0) h = 1e-3;
    for (int a = 0; a < 3; ++a) ctx->root_c[a] = 0.5 * (lo[a] + hi[a]);
    ctx->root_h = h;
    // depth
    int D = ctx->prm.depth;
    if (D < 0) {
        std::vector<int64_t> cnt(L + 1, 0);
        for (int64_t i = 0; i < N; ++i) cnt[ctx->layer[i]]++;
        int64_t nmax = *std::max_element(cnt.begin(), cnt.end());
        D = 0;
        int cap = std::max(1, ctx->prm.leaf_cap);
        while (D < 10 && (double)nmax / std::pow(8.0, D) > cap) ++D;
    }
    if (D > 20) D = 20;
    ctx->depth = D;
    // keys and sort
    const double S = 2.0 * h / (double)(1u << D);
    std::vector<uint64_t> key(N);
    auto cell = [&](double v, int a) {
        long c = (long)std::floor((v - (ctx->root_c[a] - h)) / S);
        long mx = (long)(1u << D) - 1;
        return (uint32_t)std::min(std::max(c, 0L), mx);
    };
    for (int64_t i = 0; i < N; ++i)
        key[i] = morton(cell(ctx->xyz[3 * i], 0), cell(ctx->xyz[3 * i + 1], 1),
                        cell(ctx->xyz[3 * i + 2], 2));
    ctx->perm.resize(N);
    std::iota(ctx->perm.begin(), ctx->perm.end(), 0);
    std::sort(ctx->perm.begin(), ctx->perm.end(), [&](int64_t a, int64_t b) {
        if (ctx->layer[a] != ctx->layer[b]) return ctx->layer[a] < ctx->layer[b];
        if (key[a] != key[b]) return key[a] < key[b];
        return a < b;
    });
    ctx->sxyz.resize(3 * N);
    for (int64_t i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a) ctx->sxyz[3 * i + a] = ctx->xyz[3 * ctx->perm[i] + a];
    // tree: per layer, per level
    ctx->boxes.clear();
    ctx->lvl0.assign(L + 1, std::vector<int64_t>(D + 1, 0));
    ctx->lvl1.assign(L + 1, std::vector<int64_t>(D + 1, 0));
    int64_t p = 0;
    for (int l = 0; l <= L; ++l) {
        int64_t q = p;
        while (q < N && ctx->layer[ctx->perm[q]] == l) ++q;
        // levels 0..D; boxes of level lev group points by key >> 3(D-lev)
        for (int lev = 0; lev <= D; ++lev) {
            ctx->lvl0[l][lev] = (int64_t)ctx->boxes.size();
            int sh = 3 * (D - lev);
            int64_t a = p;
            while (a < q) {
                uint64_t k = key[ctx->perm[a]] >> sh;
                int64_t b = a + 1;
                while (b < q && (key[ctx->perm[b]] >> sh) == k) ++b;
                Box bx{};
                bx.key = k;
                bx.level = lev;
                bx.layer = l;
                bx.p0 = a;
                bx.p1 = b;
                bx.parent = -1;
                bx.child0 = -1;
                bx.nchild = 0;
                bx.ix = (int)compact3(k >> 2);
                bx.iy = (int)compact3(k >> 1);
                bx.iz = (int)compact3(k);
                double Sl = 2.0 * h / (double)(1u << lev);
                bx.c[0] = ctx->root_c[0] - h + (bx.ix + 0.5) * Sl;
                bx.c[1] = ctx->root_c[1] - h + (bx.iy + 0.5) * Sl;
                bx.c[2] = ctx->root_c[2] - h + (bx.iz + 0.5) * Sl;
                double r2 = 0;
                for (int64_t t = a; t < b; ++t) {
                    double dd = 0;
                    for (int e = 0; e < 3; ++e) {
                        double v = ctx->sxyz[3 * t + e] - bx.c[e];
                        dd += v * v;
                    }
                    r2 = std::max(r2, dd);
                }
                bx.r = std::sqrt(r2);
                ctx->boxes.push_back(bx);
                a = b;
            }
            ctx->lvl1[l][lev] = (int64_t)ctx->boxes.size();
        }
        // parent/child links
        for (int lev = 1; lev <= D; ++lev) {
            int64_t pb = ctx->lvl0[l][lev - 1];
            for (int64_t b = ctx->lvl0[l][lev]; b < ctx->lvl1[l][lev]; ++b) {
                while ((ctx->boxes[b].key >> 3) != ctx->boxes[pb].key) ++pb;
                ctx->boxes[b].parent = pb;
                if (ctx->boxes[pb].child0 < 0) ctx->boxes[pb].child0 = b;
                ctx->boxes[pb].nchild++;
            }
        }
        p = q;
    }
    return LMFMM_OK;
}

static double box_min_mapped(const lmfmm_ctx *ctx, const Box &b, const CompDev &c, bool src,
                             double *mx)
{
    double lo = 1e300, hi = -1e300;
    for (int64_t t = b.p0; t < b.p1; ++t) {
        double z = ctx->sxyz[3 * t + 2];
        double zm = src ? comp_src_z(c, z) : comp_tgt_z(c, z);
        lo = std::min(lo, zm);
        hi = std::max(hi, zm);
    }
    *mx = hi;
    return lo;
}

static void box_xy_extent(const lmfmm_ctx *ctx, const Box &b, double lo[2], double hi[2])
{
    lo[0] = lo[1] = 1e300;
    hi[0] = hi[1] = -1e300;
    for (int64_t t = b.p0; t < b.p1; ++t)
        for (int e = 0; e < 2; ++e) {
            lo[e] = std::min(lo[e], ctx->sxyz[3 * t + e]);
            hi[e] = std::max(hi[e], ctx->sxyz[3 * t + e]);
        }
}

lmfmm_status build_host_structures(lmfmm_ctx *ctx)
{
    const int L = ctx->med.L;
    const int D = ctx->depth;
    const double h = ctx->root_h;
    std::vector<int64_t> cnt(L + 1, 0);
    for (int64_t i = 0; i < ctx->N; ++i) cnt[ctx->layer[i]]++;
    // components
    ctx->comps.clear();
    if (L >= 1 && ctx->prm.components != LMFMM_FREE) {
        for (int l = 0; l <= L; ++l)
            for (int lp = 0; lp <= L; ++lp) {
                if (!cnt[l] || !cnt[lp]) continue;
                for (int tu = 1; tu >= 0; --tu)
                    for (int su = 1; su >= 0; --su) {
                        if (tu && l > L - 1) continue;
                        if (!tu && l < 1) continue;
                        if (su && lp < 1) continue;
                        if (!su && lp > L - 1) continue;
                        CompDev c{};
                        c.l = l; c.lp = lp; c.tu = tu; c.su = su;
                        c.s = comp_sign(l, lp, su);
                        const double *d = ctx->med.d;
                        // image of the first slot (eq. equivalent_imag_for_target)
                        if (tu && su) { c.has_src_refl = !(l < lp); c.refl_src = d[l < L ? l : 0]; }
                        else if (tu && !su) { c.has_src_refl = !(l <= lp); c.refl_src = d[l < L ? l : 0]; }
                        else if (!tu && su) { c.has_src_refl = (l < lp); c.refl_src = d[l - 1]; }
                        else { c.has_src_refl = (l <= lp); c.refl_src = d[l - 1]; }
                        // effective location of the second slot (eq. equivalent_imag_for_source)
                        if (!su) { c.has_tgt_refl = (l <= lp); c.refl_tgt = d[lp < L ? lp : 0]; }
                        else { c.has_tgt_refl = !(l < lp); c.refl_tgt = d[lp >= 1 ? lp - 1 : 0]; }
                        if (!c.has_src_refl) c.refl_src = 0;
                        if (!c.has_tgt_refl) c.refl_tgt = 0;
                        ctx->comps.push_back(c);
                    }
            }
    }
    ctx->n_react_comps = (int)ctx->comps.size();
    // dual-tree traversal
    const double theta = ctx->prm.theta, eta = ctx->prm.eta;
    struct PairRec { int comp, level; int64_t src, tgt; };
    std::vector<PairRec> far;
    ctx->near.clear();
    ctx->n_near_pp = 0;
    std::vector<std::pair<int64_t, int64_t>> stack;
    for (int ci = 0; ci < (int)ctx->comps.size(); ++ci) {
        const CompDev &c = ctx->comps[ci];
        stack.clear();
        stack.push_back({ctx->lvl0[c.l][0], ctx->lvl0[c.lp][0]});
        while (!stack.empty()) {
            auto [bs, bt] = stack.back();
            stack.pop_back();
            const Box &B = ctx->boxes[bs], &C = ctx->boxes[bt];
            double zs = comp_src_z(c, B.c[2]), zt = comp_tgt_z(c, C.c[2]);
            double dx = B.c[0] - C.c[0], dy = B.c[1] - C.c[1], dz = zs - zt;
            double R = std::sqrt(dx * dx + dy * dy + dz * dz);
            double vz = c.s * dz;
            bool adm = (B.r + C.r <= theta * R) && (vz >= eta * R) && (vz > 0);
            if (adm) {
                far.push_back({ci, B.level, bs, bt});
            } else if (B.level == D) {
                NearPair np{};
                np.comp = ci;
                np.src = bs;
                np.tgt = bt;
                np.coef0 = ctx->n_near_pp;
                double smx, tmx;
                double smn = box_min_mapped(ctx, B, c, true, &smx);
                double tmn = box_min_mapped(ctx, C, c, false, &tmx);
                np.dzmin = c.s > 0 ? smn - tmx : tmn - smx;
                if (!(np.dzmin > 0)) {
                    ctx->err = "internal: image and effective points not separated";
                    return LMFMM_ERR_ARG;
                }
                double blo[2], bhi[2], clo[2], chi[2];
                box_xy_extent(ctx, B, blo, bhi);
                box_xy_extent(ctx, C, clo, chi);
                double mx = std::max(std::fabs(bhi[0] - clo[0]), std::fabs(chi[0] - blo[0]));
                double my = std::max(std::fabs(bhi[1] - clo[1]), std::fabs(chi[1] - blo[1]));
                np.rhomax = std::sqrt(mx * mx + my * my);
                ctx->n_near_pp += (B.p1 - B.p0) * (C.p1 - C.p0);
                ctx->near.push_back(np);
            } else {
                for (int i = 0; i < B.nchild; ++i)
                    for (int j = 0; j < C.nchild; ++j)
                        stack.push_back({B.child0 + i, C.child0 + j});
            }
        }
    }
    // geometry deduplication.  A table depends on the horizontal distance rho and
    // on the mapped heights through Z = e^{i s (k_z z_s - k'_z z_t)} (Section 3.4,
    // eq. onedimensionintegral): key (comp, level, dx^2 + dy^2 in cells, iz_s, iz_t).
    // Within a layer (l = l', k = k') Z depends on z_s - z_t alone, so every pair
    // of equal vertical offset shares one table: key (comp, level, rho^2, offset),
    // the offset in half cells of the mapped centres (a mirrored box's mapped
    // height runs against its cell index).
    std::map<std::tuple<int, int, int64_t, int, int>, int> gid;
    std::vector<int> pg(far.size());
    ctx->geoms.clear();
    for (size_t i = 0; i < far.size(); ++i) {
        const Box &B = ctx->boxes[far[i].src], &C = ctx->boxes[far[i].tgt];
        int64_t ddx = B.ix - C.ix, ddy = B.iy - C.iy;
        const CompDev &cc = ctx->comps[far[i].comp];
        int kz0 = B.iz, kz1 = C.iz;
        if (cc.l == cc.lp) {
            const int ss = cc.has_src_refl ? -1 : 1, st = cc.has_tgt_refl ? -1 : 1;
            kz0 = ss * (2 * B.iz + 1) - st * (2 * C.iz + 1);
            kz1 = 0;
        }
        auto key = std::make_tuple(far[i].comp, far[i].level, ddx * ddx + ddy * ddy, kz0, kz1);
        auto it = gid.find(key);
        if (it == gid.end()) {
            Geom g{};
            g.comp = far[i].comp;
            g.level = far[i].level;
            double Sl = 2.0 * h / (double)(1u << g.level);
            g.rho = Sl * std::sqrt((double)(ddx * ddx + ddy * ddy));
            const CompDev &c = ctx->comps[g.comp];
            g.zs = comp_src_z(c, B.c[2]);
            g.zt = comp_tgt_z(c, C.c[2]);
            it = gid.emplace(key, (int)ctx->geoms.size()).first;
            ctx->geoms.push_back(g);
        }
        pg[i] = it->second;
    }
    std::vector<int64_t> off(ctx->geoms.size() + 1, 0);
    for (size_t i = 0; i < far.size(); ++i) off[pg[i] + 1]++;
    for (size_t g = 0; g < ctx->geoms.size(); ++g) off[g + 1] += off[g];
    ctx->m2l.assign(far.size(), M2LPair{});
    std::vector<int64_t> pos(off.begin(), off.end() - 1);
    for (size_t i = 0; i < far.size(); ++i) {
        const Box &B = ctx->boxes[far[i].src], &C = ctx->boxes[far[i].tgt];
        double dx = B.c[0] - C.c[0], dy = B.c[1] - C.c[1];
        double rr = std::sqrt(dx * dx + dy * dy);
        M2LPair mp{far[i].src, far[i].tgt, rr > 0 ? dx / rr : 1.0, rr > 0 ? dy / rr : 0.0};
        ctx->m2l[pos[pg[i]]++] = mp;
    }
    for (size_t g = 0; g < ctx->geoms.size(); ++g) {
        ctx->geoms[g].pair0 = off[g];
        ctx->geoms[g].pair1 = off[g + 1];
    }
    ctx->n_react_geoms = ctx->geoms.size();
    ctx->free_tables.clear();
    ctx->free_near.clear();
    ctx->n_free_pp = 0;
    if (ctx->prm.components != LMFMM_REACTION) {
        lmfmm_status fs = build_free_structures(ctx);
        if (fs != LMFMM_OK) return fs;
    }
    // translation groups (child level lev, octant from the child's key)
    ctx->tgroups.clear();
    ctx->tpair_child.clear();
    ctx->tpair_parent.clear();
    for (int l = 0; l <= L; ++l) {
        if (!cnt[l]) continue;
        for (int lev = 1; lev <= D; ++lev) {
            std::vector<int64_t> byoct[8];
            for (int64_t b = ctx->lvl0[l][lev]; b < ctx->lvl1[l][lev]; ++b)
                byoct[ctx->boxes[b].key & 7].push_back(b);
            double Sc = 2.0 * h / (double)(1u << lev);
            for (int o = 0; o < 8; ++o) {
                if (byoct[o].empty()) continue;
                TransGroup g{};
                g.layer = l;
                g.level = lev;
                g.octant = o;
                g.t[0] = ((o >> 2) & 1 ? 0.5 : -0.5) * Sc;
                g.t[1] = ((o >> 1) & 1 ? 0.5 : -0.5) * Sc;
                g.t[2] = (o & 1 ? 0.5 : -0.5) * Sc;
                g.pair0 = (int64_t)ctx->tpair_child.size();
                for (int64_t b : byoct[o]) {
                    ctx->tpair_child.push_back(b);
                    ctx->tpair_parent.push_back(ctx->boxes[b].parent);
                }
                g.pair1 = (int64_t)ctx->tpair_child.size();
                ctx->tgroups.push_back(g);
            }
        }
    }
    return LMFMM_OK;
}

int64_t all_leaf_pairs(const lmfmm_ctx *ctx, NearPair *out, int64_t cap, int64_t *npp_out)
{
    int64_t np = 0, npp = 0;
    const int D = ctx->depth;
    for (int ci = 0; ci < ctx->n_react_comps; ++ci) {
        const CompDev &c = ctx->comps[ci];
        for (int64_t bs = ctx->lvl0[c.l][D]; bs < ctx->lvl1[c.l][D]; ++bs)
            for (int64_t bt = ctx->lvl0[c.lp][D]; bt < ctx->lvl1[c.lp][D]; ++bt) {
                if (np >= cap) return -1;
                const Box &B = ctx->boxes[bs], &C = ctx->boxes[bt];
                double smx, tmx;
                const double smn = box_min_mapped(ctx, B, c, true, &smx);
                const double tmn = box_min_mapped(ctx, C, c, false, &tmx);
                double blo[2], bhi[2], clo[2], chi[2];
                box_xy_extent(ctx, B, blo, bhi);
                box_xy_extent(ctx, C, clo, chi);
                NearPair q{};
                q.comp = ci;
                q.src = bs;
                q.tgt = bt;
                q.coef0 = npp;
                q.dzmin = c.s > 0 ? smn - tmx : tmn - smx;
                const double mx = std::max(std::fabs(bhi[0] - clo[0]), std::fabs(chi[0] - blo[0]));
                const double my = std::max(std::fabs(bhi[1] - clo[1]), std::fabs(chi[1] - blo[1]));
                q.rhomax = std::sqrt(mx * mx + my * my);
                out[np++] = q;
                npp += (B.p1 - B.p0) * (C.p1 - C.p0);
            }
    }
    *npp_out = npp;
    return np;
}

// ---------------------------------------------------------------- Chebyshev

typedef long double ld;
typedef std::complex<long double> lz;

// K_n of Appendix B for (n, m >= 0)
static int cheb_K(int n, int m)
{
    if (n % 2 == 0) return n / 2;
    return (m % 2 == 0) ? (n + 1) / 2 : (n - 1) / 2;
}

// normalised P^_n^m(cos t), 0 <= m <= n <= p, long double
void legendre_ld(int p, ld x, ld s, std::vector<ld> &P)
{
    P.assign((p + 1) * (p + 2) / 2, 0);
    ld pmm = 1.0L / std::sqrt(4.0L * 3.14159265358979323846264338327950288L);
    for (int m = 0; m <= p; ++m) {
        if (m > 0) pmm = -pmm * s * std::sqrt((ld)(2 * m + 1) / (ld)(2 * m));
        P[tidx(m, m)] = pmm;
        if (m == p) break;
        ld p1 = std::sqrt((ld)(2 * m + 3)) * x * pmm;
        P[tidx(m + 1, m)] = p1;
        ld p0 = pmm;
        for (int n = m + 2; n <= p; ++n) {
            ld a = std::sqrt((ld)(4 * n * n - 1) / (ld)(n * n - m * m));
            ld b = std::sqrt((ld)((n - 1) * (n - 1) - m * m) / (ld)(4 * (n - 1) * (n - 1) - 1));
            ld p2 = a * (x * p1 - b * p0);
            P[tidx(n, m)] = p2;
            p0 = p1;
            p1 = p2;
        }
    }
}

// B^k_{n,m} (Appendix B): Chebyshev coefficients in T_k(cos 2 theta) of the
// polynomial P^_n^m(cos theta) / tau_{nm}(theta), obtained exactly by
// interpolation at K_n + 1 Chebyshev points (the printed backward recursion
// has an inconsistent n = 0 case; interpolation reproduces it elsewhere).
void bcoef_table(int p, int KMAX, std::vector<double> &B)
{
    const ld PI = 3.14159265358979323846264338327950288L;
    int T = (p + 1) * (p + 2) / 2;
    B.assign((size_t)T * (KMAX + 1), 0.0);
    std::vector<ld> P;
    for (int n = 0; n <= p; ++n)
        for (int m = 0; m <= n; ++m) {
            int K = cheb_K(n, m);
            std::vector<ld> f(K + 1), xs(K + 1);
            for (int j = 0; j <= K; ++j) {
                ld x = std::cos(PI * (j + 0.5L) / (K + 1));
                ld ct = std::sqrt((1 + x) / 2), st = std::sqrt((1 - x) / 2);
                legendre_ld(p, ct, st, P);
                ld tau = 1;
                if (n % 2 == 1 && m % 2 == 0) tau = 1 / ct;
                else if (n % 2 == 1 && m % 2 == 1) tau = st;
                else if (n % 2 == 0 && m % 2 == 1) tau = st / ct;
                f[j] = P[tidx(n, m)] / tau;
                xs[j] = x;
            }
            for (int k = 0; k <= K; ++k) {
                ld s = 0;
                for (int j = 0; j <= K; ++j) s += f[j] * std::cos(k * std::acos(xs[j]));
                s *= 2.0L / (K + 1);
                if (k == 0) s /= 2;
                B[(size_t)tidx(n, m) * (KMAX + 1) + k] = (double)s;
            }
        }
}

// C^{ab}_{js} (Appendix A): T_j(a x + b) = sum_s C_js T_s(x), by the
// three-term recurrence T_{j+1}(y) = 2 y T_j(y) - T_{j-1}(y) with
// x T_s = (T_{s+1} + T_{|s-1|}) / 2 in the Chebyshev basis.
static void ccoef(lz a, lz b, int J, std::vector<std::vector<lz>> &C)
{
    C.assign(J + 1, std::vector<lz>(J + 2, 0));
    C[0][0] = 1;
    if (J >= 1) { C[1][0] = b; C[1][1] = a; }
    for (int j = 1; j < J; ++j) {
        std::vector<lz> xT(J + 2, 0);
        for (int s = 0; s <= j; ++s) {
            if (C[j][s] == lz(0)) continue;
            xT[s + 1] += C[j][s] * 0.5L;
            xT[s == 0 ? 1 : s - 1] += C[j][s] * 0.5L;
        }
        for (int s = 0; s <= j + 1; ++s)
            C[j + 1][s] = 2.0L * (a * xT[s] + b * C[j][s]) - (s <= j - 1 ? C[j - 1][s] : lz(0));
    }
}

// G tensor of one (k, k') pair: G[(n',|m'|)][(nu,|mu|)][l], the coefficients of
// P^_{n'}^{m'}(cos b) P^_nu^mu(cos b') / (s_{m'mu} tau tau') in T_l(cos 2 b0),
// b0 the angle of the smaller |k| (eqs. legendre_Q_v, legendre_Q_w with the
// product T_i T_s = (T_{i+s} + T_{|i-s|})/2).
void gtensor(int p, const std::vector<double> &Bcoef, int KM, zc k_, zc kp_, cd *dst0)
{
    const int T = (p + 1) * (p + 2) / 2, LM = p + 2;
    lz k(k_.real(), k_.imag()), kp(kp_.real(), kp_.imag());
    bool src_primary = std::abs(k) <= std::abs(kp);
    lz a = src_primary ? (k / kp) * (k / kp) : (kp / k) * (kp / k);
    lz b = 1.0L - a;
    std::vector<std::vector<lz>> C;
    ccoef(a, b, KM, C);
    for (int n1 = 0; n1 <= p; ++n1)
        for (int m1 = 0; m1 <= n1; ++m1)
            for (int nu = 0; nu <= p; ++nu)
                for (int mu = 0; mu <= nu; ++mu) {
                    const double *Bs = &Bcoef[(size_t)tidx(n1, m1) * (KM + 1)];
                    const double *Bt = &Bcoef[(size_t)tidx(nu, mu) * (KM + 1)];
                    int Ks = cheb_K(n1, m1), Kt = cheb_K(nu, mu);
                    std::vector<lz> G(LM, 0);
                    int Kp = src_primary ? Ks : Kt, Kq = src_primary ? Kt : Ks;
                    const double *Bp = src_primary ? Bs : Bt, *Bq = src_primary ? Bt : Bs;
                    for (int i = 0; i <= Kp; ++i)
                        for (int j = 0; j <= Kq; ++j) {
                            lz w = (ld)Bp[i] * (ld)Bq[j] * 0.5L;
                            for (int s = 0; s <= j; ++s) {
                                lz v = w * C[j][s];
                                G[i + s] += v;
                                G[i > s ? i - s : s - i] += v;
                            }
                        }
                    cd *dst = dst0 + ((size_t)tidx(n1, m1) * T + tidx(nu, mu)) * LM;
                    for (int q = 0; q < LM; ++q) dst[q] = cd{(double)G[q].real(), (double)G[q].imag()};
                }
}

void chebyshev_tables(lmfmm_ctx *ctx)
{
    const int p = ctx->prm.p;
    ctx->KMAX = (p + 1) / 2;
    bcoef_table(p, ctx->KMAX, ctx->Bcoef);
    const int T = (p + 1) * (p + 2) / 2;
    ctx->LMAXC = p + 2;
    const int LM = ctx->LMAXC, KM = ctx->KMAX;
    std::map<std::pair<int, int>, int> seen;
    ctx->comp_gidx.assign(ctx->comps.size(), 0);
    ctx->Gten.clear();
    for (size_t ci = 0; ci < ctx->comps.size(); ++ci) {
        int l = ctx->comps[ci].l, lp = ctx->comps[ci].lp;
        auto key = std::make_pair(l, lp);
        auto it = seen.find(key);
        if (it != seen.end()) { ctx->comp_gidx[ci] = it->second; continue; }
        int gi = (int)seen.size();
        seen[key] = gi;
        ctx->comp_gidx[ci] = gi;
        size_t base = ctx->Gten.size();
        ctx->Gten.resize(base + (size_t)T * T * LM, cd{0, 0});
        gtensor(p, ctx->Bcoef, KM, zc(ctx->med.k[l].x, ctx->med.k[l].y),
                zc(ctx->med.k[lp].x, ctx->med.k[lp].y), &ctx->Gten[base]);
    }
}

}  // namespace lmf

namespace lmf {

// ------------------------------------------------- translation matrices
// M2M and L2L of Section 2 (eqs. maxwell_M2M_freespace, maxwell_L2L_freespace)
// act on the regular expansions of the reaction field.  Writing the ME as the
// spherical-harmonic coefficients of the far-field pattern
// F(K) = sum_j q_j e^{i k K.(r_j - c)} = sum M_nm i^n Y_nm(K), a shift of
// centre by t multiplies F by e^{i k K.t}; with the plane-wave expansion
// e^{i k K.t} = 4 pi sum_l i^l j_l(k|t|) sum_mu Y_l^mu(K) conj(Y_l^mu(t^)),
//   W_{nm,n'm'}(t) = int e^{ikK.t} Y_n'm' conj(Y_nm) dOmega
//                  = 4 pi sum_l i^l j_l(k|t|) conj(Y_l^{m-m'}(t^)) G(l, n', n),
// G = int Y_l^{m-m'} Y_n'^m' conj(Y_n^m) (Gaunt coefficients, exact by
// Gauss-Legendre quadrature of a polynomial).  Every entry is then accurate
// relative to its own size, which matters because M2L multiplies high orders
// by large factors.  M2M = i^(n'-n) W(t), L2L = i^(n-n') W(t), t = child - parent.

// P~_n^m(x) = (m<0 ? (-1)^m : 1) P^_n^|m|(x)
static ld ptilde(const std::vector<ld> &P, int n, int m)
{
    int am = m < 0 ? -m : m;
    ld v = P[tidx(n, am)];
    return (m < 0 && (am & 1)) ? -v : v;
}

void gaunt_table(int p, std::vector<int64_t> &off, std::vector<int> &lval, std::vector<double> &gval)
{
    const int P = (p + 1) * (p + 1);
    const int nq = 2 * p + 4;
    const int lmax = 2 * p;
    // Gauss-Legendre nodes (long double Newton)
    std::vector<ld> xq(nq), wq(nq);
    for (int i = 0; i < nq; ++i) {
        ld x = std::cos(3.14159265358979323846264338327950288L * (i + 0.75L) / (nq + 0.5L)), dp = 0;
        for (int it = 0; it < 100; ++it) {
            ld p0 = 1, p1 = x;
            for (int n = 2; n <= nq; ++n) {
                ld p2 = ((2 * n - 1) * x * p1 - (n - 1) * p0) / n;
                p0 = p1;
                p1 = p2;
            }
            dp = nq * (x * p1 - p0) / (x * x - 1);
            ld dx = p1 / dp;
            x -= dx;
            if (std::fabs((double)dx) < 1e-22) break;
        }
        xq[i] = x;
        wq[i] = 2.0L / ((1 - x * x) * dp * dp);
    }
    std::vector<std::vector<ld>> Pq(nq);
    for (int q = 0; q < nq; ++q) legendre_ld(lmax, xq[q], std::sqrt(1 - xq[q] * xq[q]), Pq[q]);
    const ld twopi = 2 * 3.14159265358979323846264338327950288L;
    off.assign((size_t)P * P + 1, 0);
    lval.clear();
    gval.clear();
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m)
            for (int n1 = 0; n1 <= p; ++n1)
                for (int m1 = -n1; m1 <= n1; ++m1) {
                    int mu = m - m1;
                    int amu = mu < 0 ? -mu : mu;
                    for (int l = std::abs(n - n1); l <= n + n1; ++l) {
                        if ((l + n + n1) & 1) continue;
                        if (l < amu) continue;
                        ld s = 0;
                        for (int q = 0; q < nq; ++q)
                            s += wq[q] * ptilde(Pq[q], l, mu) * ptilde(Pq[q], n1, m1) * ptilde(Pq[q], n, m);
                        s *= twopi;
                        if (std::fabs((double)s) < 1e-30) continue;
                        lval.push_back(l);
                        gval.push_back((double)s);
                    }
                    off[(size_t)nidx(n, m) * P + nidx(n1, m1) + 1] = (int64_t)lval.size();
                }
}

// spherical Bessel j_0..j_L at complex z (long double Miller recurrence,
// normalised against j_0 or j_1, whichever is larger)
static void sph_bessel_ld(lz z, int L, std::vector<lz> &j)
{
    j.assign(L + 1, 0);
    ld az = std::abs(z);
    if (az < 1e-18L) {
        j[0] = 1;
        return;
    }
    int N = L + 30 + (int)(1.5L * az);
    lz fnp1 = 0, fn = 1e-30L, f1 = 0;
    for (int k = N; k >= 1; --k) {
        if (k <= L) j[k] = fn;
        if (k == 1) f1 = fn;
        lz fkm1 = (ld)(2 * k + 1) / z * fn - fnp1;
        fnp1 = fn;
        fn = fkm1;
        if (std::abs(fn) > 1e300L) {
            fn *= 1e-300L;
            fnp1 *= 1e-300L;
            f1 *= 1e-300L;
            for (int q = k; q <= L; ++q) j[q] *= 1e-300L;
        }
    }
    j[0] = fn;
    lz j0 = std::sin(z) / z, j1 = std::sin(z) / (z * z) - std::cos(z) / z;
    lz sc = std::abs(j0) >= std::abs(j1) ? j0 / fn : j1 / f1;
    for (auto &v : j) v *= sc;
}

void translation_matrix(int p, zc kk, const double t[3], const std::vector<int64_t> &off,
                        const std::vector<int> &lval, const std::vector<double> &gval, cd *up,
                        cd *dn)
{
    const int P = (p + 1) * (p + 1);
    const int lmax = 2 * p;
    ld tn = std::sqrt((ld)t[0] * t[0] + (ld)t[1] * t[1] + (ld)t[2] * t[2]);
    std::vector<lz> jl;
    sph_bessel_ld(lz(kk.real(), kk.imag()) * tn, lmax, jl);
    std::vector<ld> Pt;
    ld ct = tn > 0 ? t[2] / tn : 1, st = tn > 0 ? std::sqrt((ld)t[0] * t[0] + (ld)t[1] * t[1]) / tn : 0;
    legendre_ld(lmax, ct, st, Pt);
    ld phi = std::atan2((ld)t[1], (ld)t[0]);
    const ld fourpi = 4 * 3.14159265358979323846264338327950288L;
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m)
            for (int n1 = 0; n1 <= p; ++n1)
                for (int m1 = -n1; m1 <= n1; ++m1) {
                    size_t e = (size_t)nidx(n, m) * P + nidx(n1, m1);
                    int mu = m - m1;
                    // conj(Y_l^mu(t^)) = P~_l^mu e^{-i mu phi}
                    lz eph = std::polar((ld)1, -(ld)mu * phi);
                    lz s = 0;
                    for (int64_t q = off[e]; q < off[e + 1]; ++q) {
                        int l = lval[q];
                        lz il = (l % 4 == 0) ? lz(1) : (l % 4 == 1) ? lz(0, 1) : (l % 4 == 2) ? lz(-1) : lz(0, -1);
                        s += il * jl[l] * ptilde(Pt, l, mu) * (ld)gval[q];
                    }
                    s *= fourpi * eph;
                    int d = n1 - n;
                    auto ip = [](int k) {
                        k = ((k % 4) + 4) % 4;
                        return k == 0 ? lz(1) : k == 1 ? lz(0, 1) : k == 2 ? lz(-1) : lz(0, -1);
                    };
                    lz u = ip(d) * s, v = ip(-d) * s;
                    up[e] = cd{(double)u.real(), (double)u.imag()};
                    dn[e] = cd{(double)v.real(), (double)v.imag()};
                }
}

}  // namespace lmf

namespace lmf {

// ------------------------------------------------------- free-space part
// Section 2 (eqs. freespace3dmulexpscaled, melecoeffreescaled,
// maxwell_M2L_freespace): the free-space part Phi^f = (I + grad grad / k^2) u,
// u = sum_j g(r, r_j) J_j, over the sources of the target's own layer.  The
// multipole expansion M_nm = 4 pi sum q j_n(k r) conj Y_nm is the one P2M
// already forms, and u = (ik / 4 pi) sum M_nm h_n(k r) Y_nm outside the box.
// The M2L re-expands the singular harmonics S_n^m = h_n Y_n^m about the
// target centre with the addition theorem,
//   S_n'^m'(rho + t) = sum SR_{nu mu, n' m'}(t) R_nu^mu(rho),  t = c_t - c_s,
//   SR = i^(nu - n') 4 pi sum_l i^l h_l(k |t|) conj(Y_l^(mu - m')(t^)) G(l; n', nu),
// G the Gaunt coefficient int Y_l^(mu-m') Y_n'^m' conj(Y_nu^mu), which is the
// L2L construction with h_l in place of j_l.  The Hessian acts on the singular
// coefficients exactly (d/dz and d/dx +- i d/dy map S_n^m to degrees n +- 1 with
// the coefficients of the regular harmonics), so the helical field is
//   A' = u_a + D+ w / k^2,  B' = u_b + D- w / k^2,  C' = u_c + d_z w / k^2,
//   w = (D- u_a + D+ u_b) / 2 + d_z u_c,
// whose nine blocks have the reaction M2L's structure (spin kappa = change of
// the order m): they are stored as its five tables with the same per-pair
// phase factors, so the M2L kernels apply them unchanged.

namespace {

// spherical Hankel functions h_0..h_L at complex z (upward recurrence, stable
// for this dominant solution)
void sph_hankel_ld(lz z, int L, std::vector<lz> &h)
{
    h.assign(L + 1, 0);
    const lz iz(0, 1);
    const lz e = std::exp(iz * z);
    h[0] = -iz * e / z;
    if (L >= 1) h[1] = -e * (z + iz) / (z * z);
    for (int n = 1; n < L; ++n) h[n + 1] = (ld)(2 * n + 1) / z * h[n] - h[n - 1];
}

// Gaunt coefficients G(l; n', nu) = int Y_l^(mu-m') Y_n'^m' conj(Y_nu^mu) for
// nu <= pout, n' <= pin, stored per (nu mu, n' m') as (l, value) runs
void gaunt_rect(int pout, int pin, std::vector<int64_t> &off, std::vector<int> &lval, std::vector<double> &gval)
{
    const int Po = (pout + 1) * (pout + 1), Pi = (pin + 1) * (pin + 1);
    const int lmax = pout + pin, nq = (pout + pin + lmax) / 2 + 2;
    std::vector<ld> xq(nq), wq(nq);
    for (int i = 0; i < nq; ++i) {
        ld x = std::cos(3.14159265358979323846264338327950288L * (i + 0.75L) / (nq + 0.5L)), dp = 0;
        for (int it = 0; it < 100; ++it) {
            ld p0 = 1, p1 = x;
            for (int n = 2; n <= nq; ++n) {
                ld p2 = ((2 * n - 1) * x * p1 - (n - 1) * p0) / n;
                p0 = p1;
                p1 = p2;
            }
            dp = nq * (x * p1 - p0) / (x * x - 1);
            ld dx = p1 / dp;
            x -= dx;
            if (std::fabs((double)dx) < 1e-22) break;
        }
        xq[i] = x;
        wq[i] = 2.0L / ((1 - x * x) * dp * dp);
    }
    std::vector<std::vector<ld>> Pq(nq);
    for (int q = 0; q < nq; ++q) legendre_ld(lmax, xq[q], std::sqrt(1 - xq[q] * xq[q]), Pq[q]);
    const ld twopi = 2 * 3.14159265358979323846264338327950288L;
    off.assign((size_t)Po * Pi + 1, 0);
    lval.clear();
    gval.clear();
    for (int n = 0; n <= pout; ++n)
        for (int m = -n; m <= n; ++m)
            for (int n1 = 0; n1 <= pin; ++n1)
                for (int m1 = -n1; m1 <= n1; ++m1) {
                    const int mu = m - m1, amu = mu < 0 ? -mu : mu;
                    for (int l = std::abs(n - n1); l <= n + n1; ++l) {
                        if (((l + n + n1) & 1) || l < amu) continue;
                        ld s = 0;
                        for (int q = 0; q < nq; ++q)
                            s += wq[q] * ptilde(Pq[q], l, mu) * ptilde(Pq[q], n1, m1) * ptilde(Pq[q], n, m);
                        s *= twopi;
                        if (std::fabs((double)s) < 1e-30) continue;
                        lval.push_back(l);
                        gval.push_back((double)s);
                    }
                    off[(size_t)nidx(n, m) * Pi + nidx(n1, m1) + 1] = (int64_t)lval.size();
                }
}

// derivative maps on coefficient vectors c[n^2 + n + m] (n <= N) of expansions
// in R_n^m or S_n^m: returns d/dz, D+ or D- (which = 0, 1, 2) of sum c R
void deriv_apply(int which, int N, lz k, const std::vector<lz> &c, std::vector<lz> &o)
{
    o.assign(c.size(), 0);
    auto sq = [](ld v) { return v > 0 ? std::sqrt(v) : (ld)0; };
    for (int n = 0; n <= N; ++n)
        for (int m = -n; m <= n; ++m) {
            const lz v = c[nidx(n, m)];
            if (v == lz(0)) continue;
            auto add = [&](int nn, int mm, lz w) {
                if (nn < 0 || nn > N || mm < -nn || mm > nn) return;
                o[nidx(nn, mm)] += w * v;
            };
            const ld n2 = (ld)n;
            if (which == 0) {
                add(n - 1, m, k * sq((n2 * n2 - (ld)m * m) / ((2 * n2 - 1) * (2 * n2 + 1))));
                add(n + 1, m, -k * sq(((n2 + 1) * (n2 + 1) - (ld)m * m) / ((2 * n2 + 1) * (2 * n2 + 3))));
            } else if (which == 1) {
                add(n + 1, m + 1, k * sq((n2 + m + 1) * (n2 + m + 2) / ((2 * n2 + 1) * (2 * n2 + 3))));
                add(n - 1, m + 1, k * sq((n2 - m) * (n2 - m - 1) / ((2 * n2 - 1) * (2 * n2 + 1))));
            } else {
                add(n + 1, m - 1, -k * sq((n2 - m + 1) * (n2 - m + 2) / ((2 * n2 + 1) * (2 * n2 + 3))));
                add(n - 1, m - 1, -k * sq((n2 + m) * (n2 + m - 1) / ((2 * n2 - 1) * (2 * n2 + 1))));
            }
        }
}

}  // namespace

void free_m2l_tables(int p, zc kk, double rho, double dz, cd *out5, cd *blocks9)
{
    const int P = (p + 1) * (p + 1), p2 = p + 2, P2 = (p2 + 1) * (p2 + 1);
    const lz k(kk.real(), kk.imag());
    // Hessian blocks H[o][v]: input unit vector (degree <= p, component v) ->
    // singular coefficients of the helical field component o (degree <= p + 2)
    std::vector<lz> Hb((size_t)9 * P2 * P, 0);
    auto H = [&](int o, int v, int r, int c) -> lz & { return Hb[((size_t)(3 * o + v) * P2 + r) * P + c]; };
    const lz ik2 = (ld)1 / (k * k);
    std::vector<lz> e(P2), d1, d2;
    for (int c = 0; c < P; ++c) {
        std::fill(e.begin(), e.end(), lz(0));
        e[c] = 1;
        // first derivatives of the unit input, then the second ones used below
        std::vector<lz> dzv, dpv, dmv;
        deriv_apply(0, p2, k, e, dzv);
        deriv_apply(1, p2, k, e, dpv);
        deriv_apply(2, p2, k, e, dmv);
        // w contributions: from a: D- a / 2, from b: D+ b / 2, from c: d_z c
        const std::vector<lz> *wv[3] = {&dmv, &dpv, &dzv};
        const ld wf[3] = {0.5L, 0.5L, 1.0L};
        for (int v = 0; v < 3; ++v) {
            std::vector<lz> w(P2);
            for (int r = 0; r < P2; ++r) w[r] = wf[v] * (*wv[v])[r];
            std::vector<lz> gp, gm, gz;
            deriv_apply(1, p2, k, w, gp);
            deriv_apply(2, p2, k, w, gm);
            deriv_apply(0, p2, k, w, gz);
            for (int r = 0; r < P2; ++r) {
                H(0, v, r, c) = ik2 * gp[r] + (v == 0 ? e[r] : lz(0));
                H(1, v, r, c) = ik2 * gm[r] + (v == 1 ? e[r] : lz(0));
                H(2, v, r, c) = ik2 * gz[r] + (v == 2 ? e[r] : lz(0));
            }
        }
    }
    // SR(t), t = c_t - c_s = (-rho, 0, -dz), rows nu <= p, columns n' <= p + 2
    std::vector<int64_t> goff;
    std::vector<int> gl;
    std::vector<double> gv;
    gaunt_rect(p, p2, goff, gl, gv);
    const ld tx = -rho, tz = -dz, tn = std::sqrt(tx * tx + tz * tz);
    std::vector<lz> hl;
    sph_hankel_ld(k * tn, p + p2, hl);
    std::vector<ld> Pt;
    legendre_ld(p + p2, tz / tn, std::fabs(tx) / tn, Pt);
    const ld phi = std::atan2((ld)0, tx);
    const ld fourpi = 4 * 3.14159265358979323846264338327950288L;
    std::vector<lz> SR((size_t)P * P2);
    auto ip = [](int q) {
        q = ((q % 4) + 4) % 4;
        return q == 0 ? lz(1) : q == 1 ? lz(0, 1) : q == 2 ? lz(-1) : lz(0, -1);
    };
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m)
            for (int n1 = 0; n1 <= p2; ++n1)
                for (int m1 = -n1; m1 <= n1; ++m1) {
                    const size_t ge = (size_t)nidx(n, m) * P2 + nidx(n1, m1);
                    const int mu = m - m1;
                    lz s = 0;
                    for (int64_t q = goff[ge]; q < goff[ge + 1]; ++q)
                        s += ip(gl[q]) * hl[gl[q]] * ptilde(Pt, gl[q], mu) * (ld)gv[q];
                    SR[ge] = ip(n - n1) * fourpi * std::polar((ld)1, -(ld)mu * phi) * s;
                }
    // T_ov = (ik / 4 pi) SR H_ov
    const lz pre = lz(0, 1) * k / fourpi;
    std::vector<lz> T((size_t)9 * P * P, 0);
    for (int ov = 0; ov < 9; ++ov)
        for (int r = 0; r < P; ++r)
            for (int c = 0; c < P; ++c) {
                lz acc = 0;
                for (int q = 0; q < P2; ++q) {
                    const lz h = Hb[((size_t)ov * P2 + q) * P + c];
                    if (h != lz(0)) acc += SR[(size_t)r * P2 + q] * h;
                }
                T[((size_t)ov * P + r) * P + c] = pre * acc;
            }
    if (blocks9)
        for (size_t i = 0; i < T.size(); ++i) blocks9[i] = cd{(double)T[i].real(), (double)T[i].imag()};
    // the five tables: block (out, in) of each table's kappa >= 0 column divided by
    // its factors coef i^(1+kappa) (-i)^(nu+mu) i^(n'+m') at phi = 0
    const int to_out[5] = {0, 2, 0, 2, 0}, to_in[5] = {0, 2, 2, 1, 1}, kap[5] = {0, 0, 1, 1, 2};
    const ld coef[5] = {0.5L, 1.0L, 1.0L, 0.5L, -0.5L};
    std::vector<int> deg(P), ord(P);
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) {
            deg[nidx(n, m)] = n;
            ord[nidx(n, m)] = m;
        }
    for (int t = 0; t < 5; ++t)
        for (int r = 0; r < P; ++r)
            for (int c = 0; c < P; ++c) {
                const lz f = coef[t] * ip(1 + kap[t]) * ip(-(deg[r] + ord[r])) * ip(deg[c] + ord[c]);
                const lz v = T[((size_t)(3 * to_out[t] + to_in[t]) * P + r) * P + c] / f;
                out5[((size_t)t * P + r) * P + c] = cd{(double)v.real(), (double)v.imag()};
            }
}

lmfmm_status build_free_structures(lmfmm_ctx *ctx)
{
    const int L = ctx->med.L, D = ctx->depth, p = ctx->prm.p, P = (p + 1) * (p + 1);
    const double h = ctx->root_h, theta = ctx->prm.theta;
    std::vector<int64_t> cnt(L + 1, 0);
    for (int64_t i = 0; i < ctx->N; ++i) cnt[ctx->layer[i]]++;
    struct PairRec { int comp, level; int64_t src, tgt; };
    std::vector<PairRec> far;
    std::vector<int> fcomp(L + 1, -1);
    for (int l = 0; l <= L; ++l) {
        if (!cnt[l]) continue;
        // pseudo-component: same layer, no images, s = +1
        CompDev c{};
        c.l = c.lp = l;
        c.s = 1.0;
        fcomp[l] = (int)ctx->comps.size();
        ctx->comps.push_back(c);
        std::vector<std::pair<int64_t, int64_t>> stack{{ctx->lvl0[l][0], ctx->lvl0[l][0]}};
        while (!stack.empty()) {
            auto [bs, bt] = stack.back();
            stack.pop_back();
            const Box &B = ctx->boxes[bs], &C = ctx->boxes[bt];
            const double dx = B.c[0] - C.c[0], dy = B.c[1] - C.c[1], dzz = B.c[2] - C.c[2];
            const double R = std::sqrt(dx * dx + dy * dy + dzz * dzz);
            if (bs != bt && B.r + C.r <= theta * R) {
                far.push_back({fcomp[l], B.level, bs, bt});
            } else if (B.level == D) {
                ctx->free_near.push_back({bs, bt});
                ctx->n_free_pp += (B.p1 - B.p0) * (C.p1 - C.p0);
            } else {
                for (int i = 0; i < B.nchild; ++i)
                    for (int j = 0; j < C.nchild; ++j) stack.push_back({B.child0 + i, C.child0 + j});
            }
        }
    }
    // free geometries: (layer, level, rho^2 in cells, dz in cells)
    std::map<std::tuple<int, int, int64_t, int>, int> gid;
    std::vector<int> pg(far.size());
    const size_t g0 = ctx->geoms.size();
    for (size_t i = 0; i < far.size(); ++i) {
        const Box &B = ctx->boxes[far[i].src], &C = ctx->boxes[far[i].tgt];
        const int64_t ddx = B.ix - C.ix, ddy = B.iy - C.iy;
        auto key = std::make_tuple(far[i].comp, far[i].level, ddx * ddx + ddy * ddy, B.iz - C.iz);
        auto it = gid.find(key);
        if (it == gid.end()) {
            Geom g{};
            g.comp = far[i].comp;
            g.level = far[i].level;
            const double Sl = 2.0 * h / (double)(1u << g.level);
            g.rho = Sl * std::sqrt((double)(ddx * ddx + ddy * ddy));
            g.zs = B.c[2];
            g.zt = B.c[2] - Sl * (double)(B.iz - C.iz);
            it = gid.emplace(key, (int)ctx->geoms.size()).first;
            ctx->geoms.push_back(g);
        }
        pg[i] = it->second;
    }
    const size_t nfg = ctx->geoms.size() - g0;
    std::vector<int64_t> off(nfg + 1, 0);
    for (size_t i = 0; i < far.size(); ++i) off[pg[i] - g0 + 1]++;
    for (size_t g = 0; g < nfg; ++g) off[g + 1] += off[g];
    const int64_t base = (int64_t)ctx->m2l.size();
    ctx->m2l.resize(base + far.size());
    std::vector<int64_t> pos(off.begin(), off.end() - 1);
    for (size_t i = 0; i < far.size(); ++i) {
        const Box &B = ctx->boxes[far[i].src], &C = ctx->boxes[far[i].tgt];
        const double dx = B.c[0] - C.c[0], dy = B.c[1] - C.c[1];
        const double rr = std::sqrt(dx * dx + dy * dy);
        ctx->m2l[base + pos[pg[i] - g0]++] = M2LPair{far[i].src, far[i].tgt, rr > 0 ? dx / rr : 1.0,
                                                    rr > 0 ? dy / rr : 0.0};
    }
    for (size_t g = 0; g < nfg; ++g) {
        ctx->geoms[g0 + g].pair0 = base + off[g];
        ctx->geoms[g0 + g].pair1 = base + off[g + 1];
    }
    // tables, in parallel over geometries
    ctx->free_tables.assign(nfg * NTAB * (size_t)P * P, cd{0, 0});
    const int nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (int w = 0; w < nth; ++w)
        pool.emplace_back([&, w]() {
            for (size_t g = w; g < nfg; g += nth) {
                const Geom &G = ctx->geoms[g0 + g];
                const CompDev &c = ctx->comps[G.comp];
                free_m2l_tables(p, zc(ctx->med.k[c.l].x, ctx->med.k[c.l].y), G.rho, G.zs - G.zt,
                                &ctx->free_tables[g * NTAB * (size_t)P * P], nullptr);
            }
        });
    for (auto &t : pool) t.join();
    return LMFMM_OK;
}

}  // namespace lmf
