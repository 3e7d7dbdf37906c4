// Host-side forest planning: leaf set, 2:1 balance, bricks, neighbour tables, cell classes.
//
// Sec. 3.2-3.3 of the paper: a uniform grid of root blocks, blocks split into 8 while the
// application marks them, extra splits so that neighbouring leaves (across faces, edges
// and corners) differ by at most one level, every leaf holding B^3 cells.  On top of the
// leaf set this file derives what the GPU kernels need per level:
//  - owned bricks (the level's leaves) and ghost bricks: block positions covered by the
//    next coarser level that touch an owned brick; they hold the fine ghost layers 1-2 of
//    Sec. 4 (layer 3 is a source only, whose value is the coarse parent's);
//  - a 27-entry neighbour table per brick (periodic axes wrap), parent links from ghost
//    bricks to the coarse brick under them (explosion, Eq. ctof) and child links from owned
//    bricks to the finer ghost bricks inside them (coalescence, Eq. ftoc);
//  - a cell class per cell, with ghost cells taking the obstacle flag of the coarse cell that
//    covers them, so fluid/obstacle marking agrees across the interface (Sec. 4.1);
//  - per owned cell the links that are not plain loads, in each sub-step, and per sub-step the
//    list of ghost values that some later pull reads (see ghost_work).
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr uint8_t ABSENT = 0, LEAF = 1, SPLIT = 2;
constexpr int64_t kMaxBlockGrid = int64_t(1) << 26;

struct Builder {
    Plan& p;
    lbm_refine_fn refine;
    lbm_flag_fn flag;
    void* user;

    int64_t lin(int L, int x, int y, int z) const {
        const int* n = p.lv[L].nb;
        return (int64_t(z) * n[1] + y) * n[0] + x;
    }
    // Wraps block coordinates on periodic axes; false if outside a walled face.
    bool wrap(int L, int b[3]) const {
        for (int a = 0; a < 3; a++) {
            int n = p.lv[L].nb[a];
            if (p.per[a]) b[a] = ((b[a] % n) + n) % n;
            else if (b[a] < 0 || b[a] >= n) return false;
        }
        return true;
    }
    uint8_t state(int L, int x, int y, int z) const { return p.st[L][lin(L, x, y, z)]; }

    bool region_marks(int L, int x, int y, int z) const {
        double e = double(p.B) / double(1 << L);
        double lo[3] = {x * e, y * e, z * e}, hi[3] = {(x + 1) * e, (y + 1) * e, (z + 1) * e};
        for (int r = 0; r < p.d.n_regions; r++) {
            const double* g = p.d.regions[r];
            if (L >= int(g[1])) continue;
            if (int(g[0]) == 0) {
                bool hit = true;
                for (int a = 0; a < 3; a++) hit = hit && g[2 + a] < hi[a] && lo[a] < g[5 + a];
                if (hit) return true;
            } else {
                double d2 = 0.0;
                for (int a = 0; a < 3; a++) {
                    double c = g[2 + a];
                    double t = c < lo[a] ? lo[a] - c : (c > hi[a] ? c - hi[a] : 0.0);
                    d2 += t * t;
                }
                if (d2 < g[5] * g[5]) return true;
            }
        }
        return false;
    }

    void split(int L, int x, int y, int z) {
        p.st[L][lin(L, x, y, z)] = SPLIT;
        for (int c = 0; c < 8; c++)
            p.st[L + 1][lin(L + 1, 2 * x + (c & 1), 2 * y + ((c >> 1) & 1), 2 * z + (c >> 2))] = LEAF;
    }

    // A leaf of level L is unbalanced when a split block of level L+1 touches it.
    bool unbalanced(int L, int x, int y, int z) const {
        for (int k = 2 * z - 1; k <= 2 * z + 2; k++)
            for (int j = 2 * y - 1; j <= 2 * y + 2; j++)
                for (int i = 2 * x - 1; i <= 2 * x + 2; i++) {
                    int b[3] = {i, j, k};
                    if (!wrap(L + 1, b)) continue;
                    if (state(L + 1, b[0], b[1], b[2]) == SPLIT) return true;
                }
        return false;
    }

    bool leaves(std::string& err) {
        int lmax = p.d.max_level;
        p.st.assign(lmax + 1, {});
        p.lv.assign(lmax + 1, HostLevel{});
        for (int L = 0; L <= lmax; L++) {
            int64_t n = 1;
            for (int a = 0; a < 3; a++) {
                p.lv[L].nb[a] = p.d.root_blocks[a] << L;
                p.lv[L].N[a] = p.lv[L].nb[a] * p.B;
                n *= p.lv[L].nb[a];
            }
            if (n > kMaxBlockGrid) {
                err = "block grid of a level exceeds 2^26 positions";
                return false;
            }
            p.st[L].assign(size_t(n), ABSENT);
        }
        std::fill(p.st[0].begin(), p.st[0].end(), LEAF);
        for (bool changed = true; changed;) {
            changed = false;
            for (int L = 0; L < lmax; L++)
                for (int z = 0; z < p.lv[L].nb[2]; z++)
                    for (int y = 0; y < p.lv[L].nb[1]; y++)
                        for (int x = 0; x < p.lv[L].nb[0]; x++) {
                            if (state(L, x, y, z) != LEAF) continue;
                            bool want = region_marks(L, x, y, z);
                            if (!want && refine) want = refine(L, x, y, z, user) != 0;
                            if (want) {
                                split(L, x, y, z);
                                changed = true;
                            }
                        }
            for (int L = 0; L < lmax; L++)
                for (int z = 0; z < p.lv[L].nb[2]; z++)
                    for (int y = 0; y < p.lv[L].nb[1]; y++)
                        for (int x = 0; x < p.lv[L].nb[0]; x++) {
                            if (state(L, x, y, z) != LEAF) continue;
                            if (unbalanced(L, x, y, z)) {
                                split(L, x, y, z);
                                changed = true;
                            }
                        }
        }
        p.nlev = 1;
        for (int L = 0; L <= lmax; L++)
            if (std::find(p.st[L].begin(), p.st[L].end(), LEAF) != p.st[L].end()) p.nlev = L + 1;
        p.st.resize(p.nlev);
        p.lv.resize(p.nlev);
        return true;
    }

    bool obstacle(int L, int gx, int gy, int gz) const {
        double s = 1.0 / double(1 << L);
        double c[3] = {(gx + 0.5) * s, (gy + 0.5) * s, (gz + 0.5) * s};
        for (int i = 0; i < p.d.n_spheres; i++) {
            const double* q = p.d.spheres[i];
            double d2 = (c[0] - q[0]) * (c[0] - q[0]) + (c[1] - q[1]) * (c[1] - q[1]) + (c[2] - q[2]) * (c[2] - q[2]);
            if (d2 < q[3] * q[3]) return true;
        }
        return flag && flag(L, c[0], c[1], c[2], user) != 0;
    }

    // Position of level-L block (x, y, z) in the traversal of the forest of octrees: its root block
    // in x-fastest order, then the Morton (z-order) key of its place within that root's octree, the
    // bits of the three coordinates interleaved, x lowest.  The paper linearises its blocks this way,
    // along a space-filling curve (Morton or Hilbert order), for load balancing (Sec. 3.3, 4.5);
    // here it is the order of every per-level block list (level 0: the roots, x fastest).
    uint64_t forest_key(int L, int x, int y, int z) const {
        const int* n0 = p.lv[0].nb;
        const uint64_t root = (uint64_t(z >> L) * n0[1] + uint64_t(y >> L)) * n0[0] + uint64_t(x >> L);
        uint64_t k = 0;
        for (int b = 0; b < L; b++)
            k |= (uint64_t((x >> b) & 1) << (3 * b)) | (uint64_t((y >> b) & 1) << (3 * b + 1)) |
                 (uint64_t((z >> b) & 1) << (3 * b + 2));
        return (root << (3 * L)) | k;
    }

    bool bricks(int L, std::string& err) {
        HostLevel& V = p.lv[L];
        const int B = p.B, B3 = B * B * B;
        const int64_t ngrid = int64_t(V.nb[0]) * V.nb[1] * V.nb[2];
        std::vector<int32_t> index(size_t(ngrid), -1);
        // the positions of a scan in the order of the forest's traversal
        std::vector<std::pair<uint64_t, int64_t>> order;
        order.reserve(size_t(ngrid));
        for (int z = 0; z < V.nb[2]; z++)
            for (int y = 0; y < V.nb[1]; y++)
                for (int x = 0; x < V.nb[0]; x++) order.push_back({forest_key(L, x, y, z), lin(L, x, y, z)});
        std::sort(order.begin(), order.end());
        auto xyz = [&](int64_t i, int& x, int& y, int& z) {
            x = int(i % V.nb[0]);
            y = int((i / V.nb[0]) % V.nb[1]);
            z = int(i / (int64_t(V.nb[0]) * V.nb[1]));
        };
        // owned bricks: the leaves of this level, in traversal order
        for (const auto& o : order) {
            int x, y, z;
            xyz(o.second, x, y, z);
            if (state(L, x, y, z) == LEAF) {
                index[o.second] = int32_t(V.pos.size() / 3);
                V.pos.insert(V.pos.end(), {x, y, z});
            }
        }
        V.nown = int(V.pos.size() / 3);
        // ghost bricks: coarser-covered positions touching an owned brick, in traversal order
        if (L > 0) {
            for (const auto& oo : order) {
                int x, y, z;
                xyz(oo.second, x, y, z);
                if (state(L, x, y, z) != ABSENT) continue;
                bool touch = false;
                for (int o = 0; o < 27 && !touch; o++) {
                    int b[3] = {x + o % 3 - 1, y + (o / 3) % 3 - 1, z + o / 9 - 1};
                    if (o == 13 || !wrap(L, b)) continue;
                    int32_t k = index[lin(L, b[0], b[1], b[2])];
                    touch = k >= 0 && k < V.nown;
                }
                if (!touch) continue;
                if (state(L - 1, x >> 1, y >> 1, z >> 1) != LEAF) {
                    err = "a block next to a leaf is covered by a leaf two levels coarser";
                    return false;
                }
                index[lin(L, x, y, z)] = int32_t(V.pos.size() / 3);
                V.pos.insert(V.pos.end(), {x, y, z});
            }
        }
        const int nbk = int(V.pos.size() / 3);
        V.nghost = nbk - V.nown;
        V.nbr.assign(size_t(nbk) * 27, NB_COARSE);
        V.kind.assign(size_t(nbk), 0);
        V.parent.assign(size_t(nbk), -1);
        for (int k = 0; k < nbk; k++) {
            const int* P = &V.pos[3 * k];
            for (int o = 0; o < 27; o++) {
                int b[3] = {P[0] + o % 3 - 1, P[1] + (o / 3) % 3 - 1, P[2] + o / 9 - 1};
                int32_t v;
                if (!wrap(L, b)) v = NB_WALL;
                else {
                    int32_t idx = index[lin(L, b[0], b[1], b[2])];
                    if (idx >= 0) v = idx;
                    else if (state(L, b[0], b[1], b[2]) == SPLIT) v = NB_FINER;
                    else v = NB_COARSE;
                }
                V.nbr[size_t(k) * 27 + o] = v;
                if (v == NB_FINER) V.kind[k] |= BK_TOUCH_FINER;
            }
            if (k >= V.nown) {
                V.kind[k] |= BK_GHOST;
                const HostLevel& C = p.lv[L - 1];
                int32_t pb = -1;
                // the coarse brick under this ghost brick is an owned brick of level L-1
                for (int c = 0; c < C.nown; c++)
                    if (C.pos[3 * c] == P[0] >> 1 && C.pos[3 * c + 1] == P[1] >> 1 && C.pos[3 * c + 2] == P[2] >> 1) {
                        pb = c;
                        break;
                    }
                if (pb < 0) {
                    err = "ghost brick without a coarse parent brick";
                    return false;
                }
                V.parent[k] = pb * 8 + ((P[0] & 1) | ((P[1] & 1) << 1) | ((P[2] & 1) << 2));
            }
        }
        // cell classes
        V.cell.assign(size_t(nbk) * B3, CK_FLUID);
        for (int k = 0; k < nbk; k++) {
            const int* P = &V.pos[3 * k];
            uint8_t* cells = &V.cell[size_t(k) * B3];
            if (k < V.nown) {
                bool pure = true;
                for (int z = 0; z < B; z++)
                    for (int y = 0; y < B; y++)
                        for (int x = 0; x < B; x++)
                            if (obstacle(L, P[0] * B + x, P[1] * B + y, P[2] * B + z)) {
                                cells[(z * B + y) * B + x] = CK_SOLID;
                                pure = false;
                            } else {
                                V.nfluid++;
                            }
                if (pure) V.kind[k] |= BK_PURE;
                continue;
            }
            for (int z = 0; z < B; z++)
                for (int y = 0; y < B; y++)
                    for (int x = 0; x < B; x++) {
                        int l[3] = {x, y, z};
                        int dmin = 1 << 20;
                        for (int o = 0; o < 27; o++) {
                            int32_t nk = V.nbr[size_t(k) * 27 + o];
                            if (o == 13 || nk < 0 || nk >= V.nown) continue;
                            int off[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
                            int d = 0;
                            for (int a = 0; a < 3; a++) {
                                int da = off[a] == 0 ? 0 : (off[a] > 0 ? B - l[a] : l[a] + 1);
                                d = std::max(d, da);
                            }
                            dmin = std::min(dmin, d);
                        }
                        int g[3] = {P[0] * B + x, P[1] * B + y, P[2] * B + z};
                        uint8_t ck;
                        if (obstacle(L - 1, g[0] >> 1, g[1] >> 1, g[2] >> 1)) ck = CK_SOLID;
                        else ck = dmin <= 2 ? CK_GHOST : (dmin == 3 ? CK_G3 : CK_FAR);
                        int c = (z * B + y) * B + x;
                        cells[c] = ck;
                        if (ck == CK_GHOST) V.nghost12++;
                    }
            // a ghost brick without obstacle cells: every source in it is a stored value
            bool pure = true;
            for (int c = 0; c < B3 && pure; c++) pure = cells[c] != CK_SOLID;
            if (pure) V.kind[k] |= BK_PURE;
        }
        return true;
    }

    // Source of pull q into cell (x, y, z) of brick k: its brick (or an NB_* code) and, for a
    // brick, the cell index in the level's grid.
    void source(const HostLevel& V, int k, int x, int y, int z, int q, int32_t& nb, int64_t& cell) const {
        const int B = p.B, B3 = B * B * B, M = B - 1;
        const int s[3] = {x - EX[q], y - EY[q], z - EZ[q]};
        int o[3];
        for (int a = 0; a < 3; a++) o[a] = s[a] < 0 ? -1 : (s[a] > M ? 1 : 0);
        nb = (o[0] | o[1] | o[2]) ? V.nbr[size_t(k) * 27 + 13 + o[0] + 3 * o[1] + 9 * o[2]] : k;
        cell = nb >= 0 ? int64_t(nb) * B3 + (int64_t(s[2] & M) * B + (s[1] & M)) * B + (s[0] & M) : -1;
    }

    // Coalescence links of owned fluid cell (x, y, z) of brick k (Eq. ftoc): bit q is set when
    // the upwind cell along e_q, or along one axis component of e_q, lies in the finer level.
    uint32_t coal_bits(const HostLevel& V, int k, int x, int y, int z) const {
        if (!(V.kind[k] & BK_TOUCH_FINER)) return 0;
        const int M = p.B - 1;
        const int32_t* nbr = &V.nbr[size_t(k) * 27];
        uint32_t m = 0;
        for (int q = 1; q < Q; q++) {
            int s[3] = {x - EX[q], y - EY[q], z - EZ[q]}, o[3];
            for (int a = 0; a < 3; a++) o[a] = s[a] < 0 ? -1 : (s[a] > M ? 1 : 0);
            bool coal = (o[0] | o[1] | o[2]) && nbr[13 + o[0] + 3 * o[1] + 9 * o[2]] == NB_FINER;
            if (EX[q] && o[0] && nbr[13 + o[0]] == NB_FINER) coal = true;
            if (EY[q] && o[1] && nbr[13 + 3 * o[1]] == NB_FINER) coal = true;
            if (EZ[q] && o[2] && nbr[13 + 9 * o[2]] == NB_FINER) coal = true;
            if (coal) m |= 1u << q;
        }
        return m;
    }

    // Link bits of cell (x, y, z) of brick k: bit q is set when pull q is not a plain load of a
    // stored value of this level (the source is an obstacle or lies beyond a wall, or, for owned
    // cells, coalescence replaces the PDF).  Sources in ghost layers 1-3 count as plain here.
    uint32_t link_bits(const HostLevel& V, int k, int x, int y, int z, bool owned) const {
        uint32_t m = owned ? coal_bits(V, k, x, y, z) : 0u;
        for (int q = 1; q < Q; q++) {
            int32_t nb;
            int64_t c;
            source(V, k, x, y, z, q, nb, c);
            const bool plain = nb >= 0 && (V.cell[c] == CK_FLUID || V.cell[c] == CK_GHOST || V.cell[c] == CK_G3);
            if (!plain) m |= 1u << q;
        }
        return m;
    }

    // Plain links of an owned cell (not in m) whose source lies in a ghost brick.
    uint32_t ghost_src_bits(const HostLevel& V, int k, int x, int y, int z, uint32_t m) const {
        uint32_t g = 0;
        for (int q = 1; q < Q; q++) {
            if ((m >> q) & 1u) continue;
            int32_t nb;
            int64_t c;
            source(V, k, x, y, z, q, nb, c);
            if (nb >= V.nown) g |= 1u << q;
        }
        return g;
    }

    // Wall face whose boundary condition a source beyond the domain takes: the first non-free-
    // slip face it lies beyond in the order z+, z-, y+, y-, x+, x-; -1 when every face it lies
    // beyond is free-slip (the source is then mirrored).
    int wall_face(const HostLevel& V, int k, int sx, int sy, int sz) const {
        const int B = p.B;
        const int g[3] = {V.pos[3 * k] * B + sx, V.pos[3 * k + 1] * B + sy, V.pos[3 * k + 2] * B + sz};
        for (int f = 5; f >= 0; f--) {
            const int a = f >> 1;
            const bool beyond = !p.per[a] && ((f & 1) ? g[a] >= V.N[a] : g[a] < 0);
            if (beyond && p.d.bc[f] != LBM_BC_FREESLIP) return f;
        }
        return -1;
    }

    // Free-slip mirror of pull q into cell (x, y, z) of brick k whose source lies beyond free-slip
    // faces only (wall_face < 0): the source moved back inside along those faces' normals, i.e. the
    // tangential neighbour, read in direction qm (q with the mirrored components reversed).  mb is
    // its brick (or an NB_* code) and mc its cell index in the level's grid (-1 for a code).
    void mirror(const HostLevel& V, int k, int x, int y, int z, int q, int32_t& mb, int64_t& mc, int& qm) const {
        const int B = p.B, B3 = B * B * B, M = B - 1;
        const int t[3] = {x, y, z}, e[3] = {EX[q], EY[q], EZ[q]};
        int m[3], r[3], o[3];
        for (int a = 0; a < 3; a++) {
            const int s = t[a] - e[a];
            const int g = V.pos[3 * k + a] * B + s;
            const bool beyond = !p.per[a] && (g < 0 || g >= V.N[a]);
            m[a] = beyond ? t[a] : s;
            r[a] = beyond ? -e[a] : e[a];
            o[a] = m[a] < 0 ? -1 : (m[a] > M ? 1 : 0);
        }
        qm = q;
        for (int j = 1; j < Q; j++)
            if (EX[j] == r[0] && EY[j] == r[1] && EZ[j] == r[2]) qm = j;
        mb = (o[0] | o[1] | o[2]) ? V.nbr[size_t(k) * 27 + 13 + o[0] + 3 * o[1] + 9 * o[2]] : k;
        mc = mb >= 0 ? int64_t(mb) * B3 + (int64_t(m[2] & M) * B + (m[1] & M)) * B + (m[0] & M) : -1;
    }

    // Fast-path bits of an owned cell's link mask m (Sec. 2.2, Eq. ftoc):
    //  bit 29 + face in bits 25-27 when every marked link is a bounce-back of the cell's own
    //  opposite value, from obstacle cells or from beyond one single wall face (7 = no wall);
    //  an obstacle link next to a velocity wall is left to the general pull;
    //  bit 28 when every marked link is a coalescence link.
    uint32_t fast_bits(const HostLevel& V, int k, int x, int y, int z, uint32_t m) const {
        const int B = p.B, B3 = B * B * B, M = B - 1;
        const int32_t* nbr = &V.nbr[size_t(k) * 27];
        const bool finer = V.kind[k] & BK_TOUCH_FINER;
        bool bounce = true, coal_all = finer;
        int face = 7;
        bool solid_seen = false;
        for (int q = 1; q < Q; q++) {
            if (!((m >> q) & 1u)) continue;
            int s[3] = {x - EX[q], y - EY[q], z - EZ[q]}, o[3];
            for (int a = 0; a < 3; a++) o[a] = s[a] < 0 ? -1 : (s[a] > M ? 1 : 0);
            int32_t nb = (o[0] | o[1] | o[2]) ? nbr[13 + o[0] + 3 * o[1] + 9 * o[2]] : k;
            bool coal = false;
            if (finer) {
                coal = nb == NB_FINER;
                if (EX[q] && o[0] && nbr[13 + o[0]] == NB_FINER) coal = true;
                if (EY[q] && o[1] && nbr[13 + 3 * o[1]] == NB_FINER) coal = true;
                if (EZ[q] && o[2] && nbr[13 + 9 * o[2]] == NB_FINER) coal = true;
            }
            coal_all = coal_all && coal;
            if (coal) {
                bounce = false;
            } else if (nb == NB_WALL) {
                const int f = wall_face(V, k, s[0], s[1], s[2]);
                if (f < 0) bounce = false;           // free-slip reflection: general pull
                else if (face == 7) face = f;
                else if (face != f) bounce = false;
            } else if (nb >= 0 && V.cell[size_t(nb) * B3 + ((size_t(s[2] & M) * B + (s[1] & M)) * B) + (s[0] & M)] == CK_SOLID) {
                solid_seen = true;
            } else {
                bounce = false;
            }
        }
        if (bounce && solid_seen && face != 7 && p.d.bc[face] == LBM_BC_VELOCITY) bounce = false;   // two terms
        uint32_t r = 0;
        if (bounce) r |= (1u << 29) | (uint32_t(face) << 25);
        if (coal_all) r |= 1u << 28;
        return r;
    }

    // Owned cells: link bits and bit 31 for non-fluid cells; per owned column the bitmap of its
    // non-fluid cells and whether any of its cells has a nonzero link mask.
    void links(int L) {
        HostLevel& V = p.lv[L];
        const int B = p.B, B3 = B * B * B;
        for (int k = 0; k < V.nown; k++) {
            bool plain = (V.kind[k] & BK_PURE) && !(V.kind[k] & BK_TOUCH_FINER);
            for (int o = 0; o < 27 && plain; o++) {
                const int32_t nb = V.nbr[size_t(k) * 27 + o];
                plain = nb >= 0 && (V.kind[nb] & BK_PURE);
            }
            if (plain) V.kind[k] |= BK_PLAIN;
        }
        // the FP32 / FP16 column walk handles plain and bounce-back links only
        const bool paired = p.d.precision != LBM_FP64;
        V.link.assign(size_t(V.nown) * B3, 0u);
        V.colsolid.assign(size_t(V.nown) * B * B, 0u);
        V.colspec.assign(size_t(V.nown) * B * B, 0);
        V.cwork.clear();
        for (int k = 0; k < V.nown; k++)
            for (int z = 0; z < B; z++)
                for (int y = 0; y < B; y++)
                    for (int x = 0; x < B; x++) {
                        const size_t c = size_t(k) * B3 + (size_t(z) * B + y) * B + x;
                        uint32_t m = link_bits(V, k, x, y, z, true);
                        if (m) m |= fast_bits(V, k, x, y, z, m);
                        if (V.cell[c] != CK_FLUID) {
                            m |= 1u << 31;
                            V.colsolid[size_t(k) * B * B + size_t(y) * B + x] |= 1u << z;
                        } else if (coal_bits(V, k, x, y, z) || (paired && (m & 0x7FFFEu) && !(m & (1u << 29)))) {
                            // coupled: its own thread (coalescence links; with the paired FP32 walk of
                            // the shifted layouts also every other link that is not a plain bounce-back)
                            V.colsolid[size_t(k) * B * B + size_t(y) * B + x] |= 1u << z;
                            V.cwork.push_back(uint32_t(c));
                        }
                        V.link[c] = m;
                        if (m) V.colspec[size_t(k) * B * B + size_t(y) * B + x] = 1;
                    }
    }

    // Explosion and ghost stream work of level L (Sec. 4.3-4.4).  The fine level reads ghost
    // values in four places: the owned pulls of sub-step 1 read layer 1 as exploded (Eq. ctof);
    // the owned pulls of sub-step 2 read layer 1 after its sub-step-1 stream; the coalescence of
    // the coarser level reads the children of each coalescing coarse cell after the sub-step-2
    // stream, in the coalescing directions only (Eq. ftoc); and each streamed value depends on the
    // value of its source one sub-step earlier (or, for a bounce-back, on the cell's own opposite
    // value).  Every other ghost value is never read, so the explosion writes and the stream
    // computes exactly this set.  A stream source in the ghost layers before sub-step 1, or in
    // layer 3 at any time, holds the exploded value, which the stream reads from the coarse parent.
    bool ghost_work(int L, std::string& err) {
        HostLevel& V = p.lv[L];
        if (L == 0 || V.nghost == 0) return true;
        const HostLevel& C = p.lv[L - 1];
        const int B = p.B, B3 = B * B * B, M = B - 1, LB = p.LB;
        const int64_t g0 = int64_t(V.nown) * B3, ng = int64_t(V.nghost) * B3;
        std::vector<uint32_t> need[2], coarse[2], special[2];
        for (int s = 0; s < 2; s++) {
            need[s].assign(size_t(ng), 0u);
            coarse[s].assign(size_t(ng), 0u);
            special[s].assign(size_t(ng), 0u);
        }
        // after sub-step 2: the children of coalescing coarse cells (Eq. ftoc)
        for (int kc = 0; kc < C.nown; kc++) {
            if (!(C.kind[kc] & BK_TOUCH_FINER)) continue;
            for (int z = 0; z < B; z++)
                for (int y = 0; y < B; y++)
                    for (int x = 0; x < B; x++) {
                        if (C.cell[size_t(kc) * B3 + (size_t(z) * B + y) * B + x] != CK_FLUID) continue;
                        const uint32_t cm = coal_bits(C, kc, x, y, z);
                        if (!cm) continue;
                        const int oct = ((2 * x) >> LB) | (((2 * y) >> LB) << 1) | (((2 * z) >> LB) << 2);
                        const int cb = C.child[size_t(kc) * 8 + oct];
                        if (cb < V.nown) {
                            err = "coalescing cell without a finer ghost brick";
                            return false;
                        }
                        for (int d = 0; d < 8; d++) {
                            const int cx = (2 * x & M) + (d & 1), cy = (2 * y & M) + ((d >> 1) & 1), cz = (2 * z & M) + (d >> 2);
                            const int64_t c = int64_t(cb) * B3 + (int64_t(cz) * B + cy) * B + cx;
                            if (V.cell[c] != CK_GHOST) {
                                err = "a coalescence child lies outside ghost layers 1-2";
                                return false;
                            }
                            need[1][c - g0] |= cm;
                        }
                    }
        }
        // after sub-step 1: the layer-1 values that owned cells pull in sub-step 2, directly or as
        // the mirror of a free-slip link (Sec. 4.1: the boundary treatment reaches into the ghost
        // layers where a level interface meets a free-slip face)
        for (int k = 0; k < V.nown; k++)
            for (int z = 0; z < B; z++)
                for (int y = 0; y < B; y++)
                    for (int x = 0; x < B; x++) {
                        const size_t c = size_t(k) * B3 + (size_t(z) * B + y) * B + x;
                        if (V.cell[c] != CK_FLUID) continue;
                        const uint32_t cb = coal_bits(V, k, x, y, z);
                        for (int q = 1; q < Q; q++) {
                            if (!((V.link[c] >> q) & 1u) || ((cb >> q) & 1u)) continue;
                            int32_t nb, mb;
                            int64_t sc, mc;
                            int qm;
                            source(V, k, x, y, z, q, nb, sc);
                            if (nb != NB_WALL || wall_face(V, k, x - EX[q], y - EY[q], z - EZ[q]) >= 0) continue;
                            mirror(V, k, x, y, z, q, mb, mc, qm);
                            if (mb < 0) {
                                err = "a free-slip mirror of an owned cell lies outside the level";
                                return false;
                            }
                            if (mb >= V.nown && V.cell[mc] == CK_GHOST) need[0][mc - g0] |= 1u << qm;
                        }
                        const uint32_t gq = ghost_src_bits(V, k, x, y, z, V.link[c] & 0x7FFFEu);
                        for (int q = 1; q < Q; q++) {
                            if (!((gq >> q) & 1u)) continue;
                            int32_t nb;
                            int64_t sc;
                            source(V, k, x, y, z, q, nb, sc);
                            if (V.cell[sc] != CK_GHOST) {
                                err = "an owned cell pulls from beyond ghost layer 1";
                                return false;
                            }
                            need[0][sc - g0] |= 1u << q;
                        }
                    }
        // the explosion writes these same layer-1 values before sub-step 1
        for (int64_t i = 0; i < ng; i++) {
            if (!need[0][i]) continue;
            const int k = int((g0 + i) / B3), l = int((g0 + i) % B3);
            const int x = l & M, y = (l >> LB) & M, z = l >> (2 * LB);
            const int pk = V.parent[k], pb = pk >> 3, oct = pk & 7;
            const int px = ((oct & 1) * B + x) >> 1, py = (((oct >> 1) & 1) * B + y) >> 1, pz = ((oct >> 2) * B + z) >> 1;
            const int64_t pc = int64_t(pb) * B3 + (int64_t(pz) * B + py) * B + px;
            V.ework.insert(V.ework.end(), {uint32_t(g0 + i), need[0][i], uint32_t(pc), 0u});
        }
        // sources of every needed value, sub-step 2 first (it adds sub-step-1 needs)
        for (int s = 1; s >= 0; s--)
            for (int64_t i = 0; i < ng; i++) {
                if (!need[s][i]) continue;
                const int k = int((g0 + i) / B3), l = int((g0 + i) % B3);
                const int x = l & M, y = (l >> LB) & M, z = l >> (2 * LB);
                const uint32_t gl = link_bits(V, k, x, y, z, false);
                for (int q = 1; q < Q; q++) {
                    if (!((need[s][i] >> q) & 1u)) continue;
                    int32_t nb;
                    int64_t sc;
                    source(V, k, x, y, z, q, nb, sc);
                    if ((gl >> q) & 1u) {
                        bool bounce = nb == NB_WALL || (nb >= 0 && V.cell[sc] == CK_SOLID);
                        if (nb == NB_WALL && wall_face(V, k, x - EX[q], y - EY[q], z - EZ[q]) < 0) {
                            // free-slip: the mirror's value, exploded (sub-step 1, layer 3), stored
                            // after its sub-step-1 stream (layers 1-2) or owned; an obstacle there
                            // bounces the cell's own value back
                            int32_t mb;
                            int64_t mc;
                            int qm;
                            mirror(V, k, x, y, z, q, mb, mc, qm);
                            if (mb < 0 || V.cell[mc] == CK_FAR) {
                                err = "a free-slip mirror of a ghost cell has no value within ghost layer 3";
                                return false;
                            }
                            if (V.cell[mc] != CK_SOLID) {
                                bounce = false;
                                special[s][i] |= 1u << q;
                                if (s == 1 && mb >= V.nown && V.cell[mc] == CK_GHOST) need[0][mc - g0] |= 1u << qm;
                                continue;
                            }
                        }
                        if (!bounce) {
                            err = "a needed ghost value has no source within ghost layer 3";
                            return false;
                        }
                        special[s][i] |= 1u << q;
                        if (s == 1) need[0][i] |= 1u << OPP[q];
                    } else if (nb >= V.nown) {
                        if (s == 0 || V.cell[sc] == CK_G3) coarse[s][i] |= 1u << q;
                        else need[0][sc - g0] |= 1u << q;
                    }
                }
            }
        for (int s = 0; s < 2; s++)
            for (int64_t i = 0; i < ng; i++)
                if (need[s][i]) V.gwork[s].insert(V.gwork[s].end(), {uint32_t(g0 + i), need[s][i], coarse[s][i], special[s][i]});
        return true;
    }

    void children(int L) {
        HostLevel& V = p.lv[L];
        V.child.assign(size_t(V.nown) * 8, -1);
        if (L + 1 >= p.nlev) return;
        const HostLevel& F = p.lv[L + 1];
        for (int g = F.nown; g < F.nbricks(); g++) {
            const int* P = &F.pos[3 * g];
            int pb = F.parent[g] >> 3, oct = F.parent[g] & 7;
            (void)P;
            V.child[size_t(pb) * 8 + oct] = g;
        }
    }
};

}  // namespace

double scale_rate(double w0, int L) {
    double p2 = std::ldexp(1.0, L);
    return 2.0 * w0 / (2.0 * p2 + (1.0 - p2) * w0);
}

double lambda_odd(double le, double magic) { return (4.0 - 2.0 * le) / (2.0 + (4.0 * magic - 1.0) * le); }

bool build_plan(const lbm_forest_desc* d, lbm_refine_fn refine, lbm_flag_fn flag, void* user, Plan& p,
                std::string& err) {
    if (!d) {
        err = "description is NULL";
        return false;
    }
    p.d = *d;
    int B = d->block_cells;
    if (B != 8 && B != 16 && B != 32) {
        err = "block_cells must be 8, 16 or 32";
        return false;
    }
    p.B = B;
    p.LB = B == 8 ? 3 : (B == 16 ? 4 : 5);
    if (d->max_level < 0 || d->max_level >= LBM_MAX_LEVELS) {
        err = "max_level out of range";
        return false;
    }
    if (d->n_spheres < 0 || d->n_spheres > LBM_MAX_SPHERES || d->n_regions < 0 || d->n_regions > LBM_MAX_REGIONS) {
        err = "too many spheres or regions";
        return false;
    }
    if (d->precision < LBM_FP64 || d->precision > LBM_FP16S || d->collision < LBM_SRT || d->collision > LBM_TRT) {
        err = "unknown precision or collision model";
        return false;
    }
    if (!(d->rho0 > 0.0)) {
        err = "rho0 must be positive";
        return false;
    }
    if (!(d->u_shift[0] * d->u_shift[0] + d->u_shift[1] * d->u_shift[1] + d->u_shift[2] * d->u_shift[2] < 0.09)) {
        err = "u_shift must be finite with |u_shift| < 0.3";
        return false;
    }
    for (int a = 0; a < 3; a++) {
        if (d->root_blocks[a] < 1 || d->root_blocks[a] > 4096) {
            err = "root_blocks out of range";
            return false;
        }
        for (int s = 0; s < 2; s++)
            if (d->bc[2 * a + s] < LBM_BC_PERIODIC || d->bc[2 * a + s] > LBM_BC_FREESLIP) {
                err = "unknown boundary condition";
                return false;
            }
        bool p0 = d->bc[2 * a] == LBM_BC_PERIODIC, p1 = d->bc[2 * a + 1] == LBM_BC_PERIODIC;
        if (p0 != p1) {
            err = "periodic faces must come in pairs";
            return false;
        }
        p.per[a] = p0;
        if ((int64_t(d->root_blocks[a]) * B) << d->max_level >= (int64_t(1) << 30)) {
            err = "domain too large";
            return false;
        }
    }
    Builder b{p, refine, flag, user};
    if (!b.leaves(err)) return false;
    for (int L = 0; L < p.nlev; L++)
        if (!b.bricks(L, err)) return false;
    for (int L = 0; L < p.nlev; L++) b.children(L);
    for (int L = 0; L < p.nlev; L++) {
        if (int64_t(p.lv[L].nbricks()) * p.B * p.B * p.B >= (int64_t(1) << 31)) {
            err = "a level holds more than 2^31 cells";
            return false;
        }
        b.links(L);
    }
    for (int L = 1; L < p.nlev; L++)
        if (!b.ghost_work(L, err)) return false;
    return true;
}

}  // namespace lbm
