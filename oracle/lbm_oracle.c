/*
 * Plain CPU oracle for the refined-grid D3Q19 lattice Boltzmann method of
 * Schornbaum & Ruede, "Massively parallel algorithms for the lattice Boltzmann
 * method on non-uniform grids" (arXiv:1508.07982).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or helper with the CUDA
 * library: it builds its own forest, its own lattice tables and its own cell
 * classification from the same user-level description.
 *
 * Storage: one dense array per level, at that level's resolution, over a
 * window that covers every level-L leaf block plus a pad of 5 cells (4 ghost
 * layers and one boundary layer).  There are no blocks in the arithmetic: the
 * equal-level "communication" of Alg. 1 is implicit in the dense array, so the
 * result does not depend on the block size.  All arithmetic is FP64.
 *
 * One coarse step follows Alg. 1 (NonUniformTimeStep, Sec. 4.1) literally:
 *   collide(L); [step(L+1)]; [explode(L) if L>0]; boundary(L); stream(L);
 *   [coalesce(L) if L<finest]; return if L==0;
 *   collide(L); [step(L+1)]; boundary(L); stream(L); [coalesce(L) if L<finest]
 *
 * Readings of passages the paper leaves open:
 *  - moments (Eq. fvelocity) are taken of f, not f^eq (the printed f^eq is a typo);
 *  - D3Q19 weights 1/3, 1/18, 1/36 (standard; not printed);
 *  - velocity bounce-back adds 6 w_a rho0 (e_a . u_w) (named only, Sec. 5.2);
 *  - ghost layers 3-4 keep their exploded value through both fine sub-steps;
 *  - coalescence writes (x, a) for owned coarse x whose upwind cell x - e_a is
 *    covered by the finer level; the mean of the 8 children of x is summed
 *    pairwise ((c0+c1)+(c2+c3))+((c4+c5)+(c6+c7)), children in z-y-x bit order;
 *  - a cell outside the domain takes the boundary condition of the first face
 *    it lies beyond in the order z+, z-, y+, y-, x+, x-, skipping free-slip faces;
 *    a cell beyond free-slip faces only is their mirror: for a direction a whose
 *    target streams it holds the value of the mirror cell (one step back inside
 *    along each of those faces' normals) in direction a with those normal
 *    components negated (specular reflection; free-slip is named only, Sec. 4.1),
 *    or the bounced value when the mirror cell is an obstacle; like every boundary
 *    treatment it serves each cell that streams, owned or in ghost layers 1-2, so level
 *    interfaces may meet free-slip faces (Sec. 4.1 extends the boundary handling to the
 *    innermost ghost layers);
 *  - cells covered by a coarser leaf take the flag of the covering coarse cell,
 *    which makes fluid/obstacle marking consistent across interfaces (Sec. 4.1).
 * Every cell that is not an owned fluid cell starts as NaN, so any read of a
 * value the scheme never wrote shows up in the result.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19
#define ORC_MAXLEV 8
#define ORC_MAXSPH 64
#define ORC_MAXREG 64
#define PAD 5
/* Loops over fewer items run on one thread: for the small pinned cases the cost of waking the
 * OpenMP team exceeds the work.  Every loop is element-wise, so the result does not depend on it. */
#define ORC_PAR_MIN 16384

enum { BC_PERIODIC = 0, BC_NOSLIP = 1, BC_VELOCITY = 2, BC_FREESLIP = 3 };
enum { COLL_SRT = 0, COLL_TRT = 1 };
enum { CLS_OUT = 0, CLS_OWNED = 1, CLS_G1 = 2, CLS_G2 = 3, CLS_G3 = 4, CLS_G4 = 5,
       CLS_FINER = 6, CLS_FAR = 7 };
enum { FL_FLUID = 0, FL_NOSLIP = 1, FL_VEL = 2, FL_FREE = 3 };
enum { ST_ABSENT = 0, ST_LEAF = 1, ST_SPLIT = 2 };

typedef int (*orc_refine_fn)(int level, int bx, int by, int bz, void *user);
typedef int (*orc_flag_fn)(int level, double x, double y, double z, void *user);

typedef struct {
    int nroot[3];
    int B;
    int lmax;
    int collision;
    double rho0;
    int bc[6];              /* faces x-, x+, y-, y+, z-, z+ */
    double bcu[6][3];       /* wall velocity of velocity faces */
    int nsph;
    double sph[ORC_MAXSPH][4];  /* obstacle spheres: centre, radius (level-0 cell units) */
    int nreg;
    double reg[ORC_MAXREG][8];  /* refinement regions: kind (0 box, 1 ball), target level,
                                   box lo[3] hi[3] | ball centre[3] radius */
} orc_desc;

typedef struct {
    int N[3];          /* domain extent in cells at this level */
    int s[3], n[3];    /* window start and length per axis */
    long ncell;
    double *f, *tmp;   /* [ncell][Q] */
    unsigned char *cls, *flag, *inS;
    signed char *vface;            /* wall face of velocity cells; mirrored axes (bits) of
                                      free-slip cells; else -1 */
    long *C; long nC;              /* owned fluid cells: collide set */
    long *S; long nS;              /* owned, G1, G2 fluid cells: stream set */
    long *G; long *Gp; long nG;    /* G1..G4 cells and their parent index on L-1 */
    long *Bd; long nBd;            /* boundary cells */
    long *Kc; int *Ka; long *Kch; long nK;  /* coalescence entries: cell, direction, 8 children */
} olevel;

typedef struct orc {
    orc_desc d;
    orc_refine_fn refine;
    orc_flag_fn flagfn;
    void *user;
    int per[3];
    int nlev;                          /* deepest leaf level + 1 */
    int nbk[ORC_MAXLEV][3];
    unsigned char *st[ORC_MAXLEV];
    olevel lv[ORC_MAXLEV];
    double le[ORC_MAXLEV], lo[ORC_MAXLEV], acc[ORC_MAXLEV][3];
} orc;

static char g_err[512];
const char *orc_error(void) { return g_err; }

/* ---------------- D3Q19 lattice (Sec. 2, Fig. 1) ---------------- */
static const int EV[Q][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static double W[Q];
static int OPP[Q];
static int lattice_ready = 0;

static void lattice_init(void) {
    if (lattice_ready) return;
    for (int a = 0; a < Q; a++) {
        int n2 = EV[a][0] * EV[a][0] + EV[a][1] * EV[a][1] + EV[a][2] * EV[a][2];
        W[a] = n2 == 0 ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        for (int b = 0; b < Q; b++)
            if (EV[b][0] == -EV[a][0] && EV[b][1] == -EV[a][1] && EV[b][2] == -EV[a][2]) OPP[a] = b;
    }
    lattice_ready = 1;
}

void orc_lattice(int *e, double *w, int *opp) {
    lattice_init();
    for (int a = 0; a < Q; a++) {
        for (int k = 0; k < 3; k++) e[3 * a + k] = EV[a][k];
        w[a] = W[a];
        opp[a] = OPP[a];
    }
}

/* ---------------- collision (Sec. 2 and 2.1) ---------------- */

/* Incompressible equilibrium, Eq. (fequ), with c = 1. */
static void feq_cell(double rho, const double u[3], double rho0, double *feq) {
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int a = 0; a < Q; a++) {
        double eu = EV[a][0] * u[0] + EV[a][1] * u[1] + EV[a][2] * u[2];
        feq[a] = W[a] * (rho + rho0 * (3.0 * eu + 4.5 * eu * eu - 1.5 * uu));
    }
}

void orc_feq(double rho, const double u[3], double rho0, double *feq) {
    lattice_init();
    feq_cell(rho, u, rho0, feq);
}

/* One collision of one cell: SRT or TRT operator of Sec. 2, with the body
 * force term F_a = w_a rho0 (e_a . a) / c_s^2 of Sec. 2.1 added afterwards.
 * Moments are taken of f (Eq. fvelocity, read with f in place of f^eq); the
 * velocity inside f^eq is left unmodified by the force, as Sec. 2.1 states. */
static void collide_cell(double *f, int coll, double le, double lo, const double acc[3], double rho0) {
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < Q; a++) {
        rho += f[a];
        for (int k = 0; k < 3; k++) j[k] += EV[a][k] * f[a];
    }
    double u[3] = {j[0] / rho0, j[1] / rho0, j[2] / rho0};
    double feq[Q], fo[Q];
    feq_cell(rho, u, rho0, feq);
    for (int a = 0; a < Q; a++) {
        double C;
        if (coll == COLL_SRT) {
            C = -le * (f[a] - feq[a]);
        } else {
            int b = OPP[a];
            double fp = 0.5 * (f[a] + f[b]), fm = 0.5 * (f[a] - f[b]);
            double ep = 0.5 * (feq[a] + feq[b]), em = 0.5 * (feq[a] - feq[b]);
            C = -le * (fp - ep) - lo * (fm - em);
        }
        double ea = EV[a][0] * acc[0] + EV[a][1] * acc[1] + EV[a][2] * acc[2];
        double F = W[a] * rho0 * ea * 3.0;   /* 1/c_s^2 = 3 */
        fo[a] = f[a] + C + F;
    }
    memcpy(f, fo, sizeof(fo));
}

void orc_collide(double *f, int coll, double le, double lo, const double acc[3], double rho0) {
    lattice_init();
    collide_cell(f, coll, le, lo, acc, rho0);
}

/* ---------------- relaxation and force scaling (Sec. 2.3) ---------------- */

/* Eq. (omega_scaling_0): the rate on level L that keeps nu fixed, Delta t_L = Delta t_0 / 2^L. */
double orc_scale_rate(double w0, int L) {
    double p = ldexp(1.0, L);
    return 2.0 * w0 / (2.0 * p + (1.0 - p) * w0);
}

/* Eq. (lambda_oL): lambda_o from lambda_e at fixed magic parameter Lambda_eo. */
double orc_lambda_odd(double le, double magic) {
    return (4.0 - 2.0 * le) / (2.0 + (4.0 * magic - 1.0) * le);
}

/* ---------------- forest: refinement and 2:1 balance (Sec. 3.2-3.3) ---------------- */

static long bidx(const orc *o, int L, const int b[3]) {
    return ((long)b[2] * o->nbk[L][1] + b[1]) * o->nbk[L][0] + b[0];
}

/* Wraps a block coordinate on periodic axes; returns 0 if outside a walled domain. */
static int bwrap(const orc *o, int L, int b[3]) {
    for (int a = 0; a < 3; a++) {
        int n = o->nbk[L][a];
        if (o->per[a]) b[a] = ((b[a] % n) + n) % n;
        else if (b[a] < 0 || b[a] >= n) return 0;
    }
    return 1;
}

static int region_wants(const orc *o, int L, const int b[3]) {
    double sz = (double)o->d.B / ldexp(1.0, L);     /* block edge in level-0 cells */
    double lo[3], hi[3];
    for (int a = 0; a < 3; a++) { lo[a] = b[a] * sz; hi[a] = (b[a] + 1) * sz; }
    for (int r = 0; r < o->d.nreg; r++) {
        const double *g = o->d.reg[r];
        if (L >= (int)g[1]) continue;
        if ((int)g[0] == 0) {
            int hit = 1;
            for (int a = 0; a < 3; a++) if (!(g[2 + a] < hi[a] && lo[a] < g[5 + a])) hit = 0;
            if (hit) return 1;
        } else {
            double d2 = 0.0;
            for (int a = 0; a < 3; a++) {
                double c = g[2 + a], t = 0.0;
                if (c < lo[a]) t = lo[a] - c; else if (c > hi[a]) t = c - hi[a];
                d2 += t * t;
            }
            if (d2 < g[5] * g[5]) return 1;
        }
    }
    return 0;
}

static void split_block(orc *o, int L, const int b[3]) {
    o->st[L][bidx(o, L, b)] = ST_SPLIT;
    for (int c = 0; c < 8; c++) {
        int cb[3] = {2 * b[0] + (c & 1), 2 * b[1] + ((c >> 1) & 1), 2 * b[2] + ((c >> 2) & 1)};
        o->st[L + 1][bidx(o, L + 1, cb)] = ST_LEAF;
    }
}

/* Leaf b on level L violates 2:1 balance iff a split block of level L+1 touches it
 * (across a face, an edge or a corner). */
static int unbalanced(const orc *o, int L, const int b[3]) {
    if (L + 1 >= ORC_MAXLEV || o->st[L + 1] == NULL) return 0;
    for (int z = 2 * b[2] - 1; z <= 2 * b[2] + 2; z++)
        for (int y = 2 * b[1] - 1; y <= 2 * b[1] + 2; y++)
            for (int x = 2 * b[0] - 1; x <= 2 * b[0] + 2; x++) {
                int p[3] = {x, y, z};
                if (!bwrap(o, L + 1, p)) continue;
                if (o->st[L + 1][bidx(o, L + 1, p)] == ST_SPLIT) return 1;
            }
    return 0;
}

static int build_forest(orc *o) {
    for (int L = 0; L <= o->d.lmax; L++) {
        for (int a = 0; a < 3; a++) o->nbk[L][a] = o->d.nroot[a] << L;
        long nb = (long)o->nbk[L][0] * o->nbk[L][1] * o->nbk[L][2];
        o->st[L] = (unsigned char *)calloc(nb, 1);
        if (!o->st[L]) { snprintf(g_err, sizeof g_err, "out of memory (block grid)"); return 0; }
    }
    long n0 = (long)o->nbk[0][0] * o->nbk[0][1] * o->nbk[0][2];
    memset(o->st[0], ST_LEAF, n0);
    int changed = 1;
    while (changed) {
        changed = 0;
        /* user refinement: any leaf below lmax that the regions or the callback mark is split */
        for (int L = 0; L < o->d.lmax; L++)
            for (int z = 0; z < o->nbk[L][2]; z++)
                for (int y = 0; y < o->nbk[L][1]; y++)
                    for (int x = 0; x < o->nbk[L][0]; x++) {
                        int b[3] = {x, y, z};
                        if (o->st[L][bidx(o, L, b)] != ST_LEAF) continue;
                        int want = region_wants(o, L, b);
                        if (!want && o->refine) want = o->refine(L, x, y, z, o->user) != 0;
                        if (want) { split_block(o, L, b); changed = 1; }
                    }
        /* 2:1 balance across faces, edges and corners */
        for (int L = 0; L < o->d.lmax; L++)
            for (int z = 0; z < o->nbk[L][2]; z++)
                for (int y = 0; y < o->nbk[L][1]; y++)
                    for (int x = 0; x < o->nbk[L][0]; x++) {
                        int b[3] = {x, y, z};
                        if (o->st[L][bidx(o, L, b)] != ST_LEAF) continue;
                        if (unbalanced(o, L, b)) { split_block(o, L, b); changed = 1; }
                    }
    }
    o->nlev = 1;
    for (int L = 0; L <= o->d.lmax; L++) {
        long nb = (long)o->nbk[L][0] * o->nbk[L][1] * o->nbk[L][2];
        for (long i = 0; i < nb; i++) if (o->st[L][i] == ST_LEAF) { o->nlev = L + 1; break; }
    }
    return 1;
}

int orc_num_levels(const orc *o) { return o->nlev; }

/* Leaf blocks of one level as (bx, by, bz) triples in x-fastest order; returns the count. */
long orc_leaves(const orc *o, int L, int *out) {
    long cnt = 0;
    if (L < 0 || L > o->d.lmax) return 0;
    for (int z = 0; z < o->nbk[L][2]; z++)
        for (int y = 0; y < o->nbk[L][1]; y++)
            for (int x = 0; x < o->nbk[L][0]; x++) {
                int b[3] = {x, y, z};
                if (o->st[L][bidx(o, L, b)] != ST_LEAF) continue;
                if (out) { out[3 * cnt] = x; out[3 * cnt + 1] = y; out[3 * cnt + 2] = z; }
                cnt++;
            }
    return cnt;
}

/* ---------------- per-level windows and cell classes ---------------- */

static long cidx(const olevel *V, int x, int y, int z) {
    return ((long)z * V->n[1] + y) * V->n[0] + x;
}

/* Global level-L coordinate -> window-local coordinate; 0 if outside the window. */
static int g2l(const orc *o, const olevel *V, const int g[3], int l[3]) {
    for (int a = 0; a < 3; a++) {
        int d = g[a] - V->s[a];
        if (o->per[a]) d = ((d % V->N[a]) + V->N[a]) % V->N[a];
        if (d < 0 || d >= V->n[a]) return 0;
        l[a] = d;
    }
    return 1;
}

static void l2g(const orc *o, const olevel *V, const int l[3], int g[3]) {
    for (int a = 0; a < 3; a++) {
        g[a] = V->s[a] + l[a];
        if (o->per[a]) g[a] = ((g[a] % V->N[a]) + V->N[a]) % V->N[a];
    }
}

/* Window index of the neighbour of window cell (x,y,z) at offset d, or -1. */
static long nbr(const orc *o, const olevel *V, int x, int y, int z, int dx, int dy, int dz) {
    int l[3] = {x, y, z}, g[3], m[3];
    l2g(o, V, l, g);
    g[0] += dx; g[1] += dy; g[2] += dz;
    if (!g2l(o, V, g, m)) return -1;
    return cidx(V, m[0], m[1], m[2]);
}

static void cell_xyz(const olevel *V, long c, int *x, int *y, int *z) {
    *x = (int)(c % V->n[0]);
    *y = (int)((c / V->n[0]) % V->n[1]);
    *z = (int)(c / ((long)V->n[0] * V->n[1]));
}

static void set_window(orc *o, int L) {
    olevel *V = &o->lv[L];
    int B = o->d.B;
    for (int a = 0; a < 3; a++) V->N[a] = (o->d.nroot[a] * B) << L;
    for (int a = 0; a < 3; a++) {
        int N = V->N[a];
        if (o->per[a]) {
            unsigned char *cov = (unsigned char *)calloc(N, 1);
            int any = 0;
            for (int z = 0; z < o->nbk[L][2]; z++)
                for (int y = 0; y < o->nbk[L][1]; y++)
                    for (int x = 0; x < o->nbk[L][0]; x++) {
                        int b[3] = {x, y, z};
                        if (o->st[L][bidx(o, L, b)] != ST_LEAF) continue;
                        any = 1;
                        for (int i = b[a] * B - PAD; i < (b[a] + 1) * B + PAD; i++) cov[((i % N) + N) % N] = 1;
                    }
            if (!any) { V->s[a] = 0; V->n[a] = 0; free(cov); continue; }
            /* smallest cyclic interval covering all marked cells: the complement of the longest gap */
            int best = 0, bestend = 0;
            for (int i = 0; i < N; i++) {
                if (cov[i]) continue;
                int len = 0;
                while (len < N && !cov[(i + len) % N]) len++;
                if (len > best) { best = len; bestend = (i + len) % N; }
            }
            if (best == 0) { V->s[a] = 0; V->n[a] = N; }
            else { V->s[a] = bestend; V->n[a] = N - best; }
            free(cov);
        } else {
            int lo = 1 << 30, hi = -(1 << 30);
            for (int z = 0; z < o->nbk[L][2]; z++)
                for (int y = 0; y < o->nbk[L][1]; y++)
                    for (int x = 0; x < o->nbk[L][0]; x++) {
                        int b[3] = {x, y, z};
                        if (o->st[L][bidx(o, L, b)] != ST_LEAF) continue;
                        if (b[a] * B - PAD < lo) lo = b[a] * B - PAD;
                        if ((b[a] + 1) * B + PAD > hi) hi = (b[a] + 1) * B + PAD;
                    }
            if (hi < lo) { V->s[a] = 0; V->n[a] = 0; }
            else { V->s[a] = lo; V->n[a] = hi - lo; }
        }
    }
    V->ncell = (long)V->n[0] * V->n[1] * V->n[2];
}

/* Level-m ancestor state of the level-L cell with global coordinate g. */
static int covering_leaf_level(const orc *o, int L, const int g[3]) {
    int b[3] = {g[0] / o->d.B, g[1] / o->d.B, g[2] / o->d.B};
    for (int m = L; m >= 0; m--) {
        unsigned char s = o->st[m][bidx(o, m, b)];
        if (s == ST_LEAF) return m;
        if (s == ST_SPLIT) return L + 1;   /* only reachable for m == L: covered by finer leaves */
        for (int a = 0; a < 3; a++) b[a] >>= 1;
    }
    return -1;
}

static int obstacle_at(const orc *o, int L, const int g[3]) {
    double sc = ldexp(1.0, -L);
    double p[3] = {(g[0] + 0.5) * sc, (g[1] + 0.5) * sc, (g[2] + 0.5) * sc};
    for (int i = 0; i < o->d.nsph; i++) {
        double d2 = 0.0;
        for (int a = 0; a < 3; a++) d2 += (p[a] - o->d.sph[i][a]) * (p[a] - o->d.sph[i][a]);
        if (d2 < o->d.sph[i][3] * o->d.sph[i][3]) return 1;
    }
    if (o->flagfn && o->flagfn(L, p[0], p[1], p[2], o->user) != 0) return 1;
    return 0;
}

static int classify(orc *o, int L) {
    olevel *V = &o->lv[L];
    long n = V->ncell;
    V->cls = (unsigned char *)malloc(n ? n : 1);
    V->flag = (unsigned char *)malloc(n ? n : 1);
    V->inS = (unsigned char *)calloc(n ? n : 1, 1);
    V->vface = (signed char *)malloc(n ? n : 1);
    unsigned char *dist = (unsigned char *)malloc(n ? n : 1);
    if (!V->cls || !V->flag || !V->inS || !V->vface || !dist) { snprintf(g_err, sizeof g_err, "out of memory (classes)"); return 0; }
    static const int face_order[6] = {5, 4, 3, 2, 1, 0};   /* z+, z-, y+, y-, x+, x- */
    for (long c = 0; c < n; c++) {
        int l[3], g[3];
        cell_xyz(V, c, &l[0], &l[1], &l[2]);
        l2g(o, V, l, g);
        V->vface[c] = -1;
        int out = 0;
        for (int a = 0; a < 3; a++) if (g[a] < 0 || g[a] >= V->N[a]) out = 1;
        if (out) {
            V->cls[c] = CLS_OUT;
            V->flag[c] = FL_FREE;
            int axes = 0;
            for (int k = 0; k < 6; k++) {
                int fce = face_order[k], a = fce / 2;
                int beyond = (fce & 1) ? (g[a] >= V->N[a]) : (g[a] < 0);
                if (!beyond) continue;
                if (o->d.bc[fce] == BC_FREESLIP) { axes |= 1 << a; continue; }
                if (o->d.bc[fce] == BC_VELOCITY) { V->flag[c] = FL_VEL; V->vface[c] = (signed char)fce; }
                else V->flag[c] = FL_NOSLIP;
                break;
            }
            if (V->flag[c] == FL_FREE) V->vface[c] = (signed char)axes;
            dist[c] = 255;
            continue;
        }
        int m = covering_leaf_level(o, L, g);
        if (m == L) {
            V->cls[c] = CLS_OWNED;
            V->flag[c] = obstacle_at(o, L, g) ? FL_NOSLIP : FL_FLUID;
            dist[c] = 0;
        } else if (m > L) {
            V->cls[c] = CLS_FINER;
            V->flag[c] = FL_FLUID;
            dist[c] = 255;
        } else {
            V->cls[c] = CLS_FAR;
            int pg[3];
            for (int a = 0; a < 3; a++) pg[a] = g[a] >> (L - m);
            V->flag[c] = obstacle_at(o, m, pg) ? FL_NOSLIP : FL_FLUID;
            dist[c] = 255;
        }
    }
    /* Chebyshev distance to the owned region by four 26-neighbour dilations */
    for (int k = 1; k <= 4; k++) {
        for (long c = 0; c < n; c++) {
            if (dist[c] != 255) continue;
            int x, y, z;
            cell_xyz(V, c, &x, &y, &z);
            int hit = 0;
            for (int dz = -1; dz <= 1 && !hit; dz++)
                for (int dy = -1; dy <= 1 && !hit; dy++)
                    for (int dx = -1; dx <= 1 && !hit; dx++) {
                        long m2 = nbr(o, V, x, y, z, dx, dy, dz);
                        if (m2 >= 0 && dist[m2] == k - 1) hit = 1;
                    }
            if (hit) dist[c] = (unsigned char)k;
        }
    }
    for (long c = 0; c < n; c++)
        if (V->cls[c] == CLS_FAR && dist[c] >= 1 && dist[c] <= 4) V->cls[c] = (unsigned char)(CLS_G1 + dist[c] - 1);
    free(dist);
    return 1;
}

static long *push(long *arr, long *cnt, long *cap, long v) {
    if (*cnt == *cap) {
        *cap = *cap ? 2 * *cap : 1024;
        arr = (long *)realloc(arr, *cap * sizeof(long));
    }
    arr[(*cnt)++] = v;
    return arr;
}

static int build_lists(orc *o, int L) {
    olevel *V = &o->lv[L];
    long capC = 0, capS = 0, capG = 0, capB = 0;
    for (long c = 0; c < V->ncell; c++) {
        unsigned char k = V->cls[c], fl = V->flag[c];
        if (fl == FL_FLUID && k == CLS_OWNED) V->C = push(V->C, &V->nC, &capC, c);
        if (fl == FL_FLUID && (k == CLS_OWNED || k == CLS_G1 || k == CLS_G2)) {
            V->S = push(V->S, &V->nS, &capS, c);
            V->inS[c] = 1;
        }
        if (k >= CLS_G1 && k <= CLS_G4) V->G = push(V->G, &V->nG, &capG, c);
        if (fl != FL_FLUID && k != CLS_FINER) V->Bd = push(V->Bd, &V->nBd, &capB, c);
    }
    /* explosion sources: the parent cell on level L-1 (Eq. ctof) */
    if (V->nG) {
        V->Gp = (long *)malloc(V->nG * sizeof(long));
        olevel *P = &o->lv[L - 1];
        for (long i = 0; i < V->nG; i++) {
            int l[3], g[3], pg[3], pl[3];
            cell_xyz(V, V->G[i], &l[0], &l[1], &l[2]);
            l2g(o, V, l, g);
            for (int a = 0; a < 3; a++) pg[a] = g[a] >> 1;
            if (!g2l(o, P, pg, pl)) { snprintf(g_err, sizeof g_err, "explosion parent outside window (level %d)", L); return 0; }
            V->Gp[i] = cidx(P, pl[0], pl[1], pl[2]);
        }
    }
    /* coalescence targets: owned fluid x and a with x - e_a covered by level L+1 (Eq. ftoc) */
    if (L + 1 < o->nlev) {
        olevel *Fv = &o->lv[L + 1];
        long cap = 0, capk = 0;
        for (long i = 0; i < V->nC; i++) {
            long c = V->C[i];
            int x, y, z;
            cell_xyz(V, c, &x, &y, &z);
            for (int a = 1; a < Q; a++) {
                /* the PDF enters x from the finer level if the upwind cell along e_a, or along
                   any one axis component of e_a, is covered by the finer level */
                int hit = 0;
                long sidx = nbr(o, V, x, y, z, -EV[a][0], -EV[a][1], -EV[a][2]);
                if (sidx >= 0 && V->cls[sidx] == CLS_FINER) hit = 1;
                for (int k = 0; k < 3 && !hit; k++) {
                    if (EV[a][k] == 0) continue;
                    int d[3] = {0, 0, 0};
                    d[k] = -EV[a][k];
                    long s2 = nbr(o, V, x, y, z, d[0], d[1], d[2]);
                    if (s2 >= 0 && V->cls[s2] == CLS_FINER) hit = 1;
                }
                if (!hit) continue;
                long k = V->nK;
                V->Kc = push(V->Kc, &V->nK, &cap, c);
                if (V->nK > capk) {
                    capk = cap;
                    V->Ka = (int *)realloc(V->Ka, capk * sizeof(int));
                    V->Kch = (long *)realloc(V->Kch, capk * 8 * sizeof(long));
                }
                V->Ka[k] = a;
                int l[3] = {x, y, z}, g[3];
                l2g(o, V, l, g);
                for (int j = 0; j < 8; j++) {
                    int cg[3] = {2 * g[0] + (j & 1), 2 * g[1] + ((j >> 1) & 1), 2 * g[2] + ((j >> 2) & 1)}, cl[3];
                    if (!g2l(o, Fv, cg, cl)) { snprintf(g_err, sizeof g_err, "coalescence child outside window (level %d)", L); return 0; }
                    V->Kch[8 * k + j] = cidx(Fv, cl[0], cl[1], cl[2]);
                }
            }
        }
    }
    return 1;
}

/* ---------------- the operations of Alg. 1 ---------------- */

static void op_collide(orc *o, int L) {
    olevel *V = &o->lv[L];
    #pragma omp parallel for schedule(static) if (V->nC > ORC_PAR_MIN)
    for (long i = 0; i < V->nC; i++)
        collide_cell(V->f + V->C[i] * Q, o->d.collision, o->le[L], o->lo[L], o->acc[L], o->d.rho0);
}

/* Eq. (ctof): every fine ghost cell of layers 1-4 receives all 19 PDFs of its coarse parent. */
static void op_explode(orc *o, int L) {
    olevel *V = &o->lv[L], *P = &o->lv[L - 1];
    #pragma omp parallel for schedule(static) if (V->nG > ORC_PAR_MIN)
    for (long i = 0; i < V->nG; i++)
        memcpy(V->f + V->G[i] * Q, P->f + V->Gp[i] * Q, Q * sizeof(double));
}

/* Boundary treatment as a pre-streaming step (Sec. 2.2): boundary cell b stores,
 * for every direction a whose target b + e_a streams, the bounced PDF of that target. */
static void op_boundary(orc *o, int L) {
    olevel *V = &o->lv[L];
    #pragma omp parallel for schedule(static) if (V->nBd > ORC_PAR_MIN)
    for (long i = 0; i < V->nBd; i++) {
        long b = V->Bd[i];
        int x, y, z;
        cell_xyz(V, b, &x, &y, &z);
        for (int a = 1; a < Q; a++) {
            long nn = nbr(o, V, x, y, z, EV[a][0], EV[a][1], EV[a][2]);
            if (nn < 0 || !V->inS[nn]) continue;
            double v = V->f[nn * Q + OPP[a]];
            if (V->flag[b] == FL_FREE) {
                /* specular reflection: the mirror cell one step back inside along each mirrored
                 * normal, direction a with those components negated */
                int axes = V->vface[b], d[3] = {0, 0, 0}, e[3];
                for (int k = 0; k < 3; k++) {
                    e[k] = EV[a][k];
                    if (axes >> k & 1) { d[k] = EV[a][k]; e[k] = -EV[a][k]; }
                }
                long m = nbr(o, V, x, y, z, d[0], d[1], d[2]);
                int am = 0;
                for (int k = 1; k < Q; k++)
                    if (EV[k][0] == e[0] && EV[k][1] == e[1] && EV[k][2] == e[2]) am = k;
                if (m >= 0 && V->flag[m] == FL_FLUID) v = V->f[m * Q + am];
            }
            if (V->flag[b] == FL_VEL) {
                const double *uw = o->d.bcu[(int)V->vface[b]];
                v += 6.0 * W[a] * o->d.rho0 * (EV[a][0] * uw[0] + EV[a][1] * uw[1] + EV[a][2] * uw[2]);
            }
            V->f[b * Q + a] = v;
        }
    }
}

/* Eq. (stream), pull form, two grids (Sec. 4.1): cells of the stream set pull; every other
 * cell keeps its value, so ghost layers 3-4 hold the exploded value for both fine sub-steps. */
static void op_stream(orc *o, int L) {
    olevel *V = &o->lv[L];
    memcpy(V->tmp, V->f, V->ncell * Q * sizeof(double));
    #pragma omp parallel for schedule(static) if (V->nS > ORC_PAR_MIN)
    for (long i = 0; i < V->nS; i++) {
        long c = V->S[i];
        int x, y, z;
        cell_xyz(V, c, &x, &y, &z);
        for (int a = 0; a < Q; a++) {
            long s = nbr(o, V, x, y, z, -EV[a][0], -EV[a][1], -EV[a][2]);
            V->tmp[c * Q + a] = s >= 0 ? V->f[s * Q + a] : NAN;
        }
    }
    double *t = V->f; V->f = V->tmp; V->tmp = t;
}

/* Eq. (ftoc) with n = 8, applied after the coarse stream to the PDFs that enter the coarse
 * block from the finer level; the fine values are those after both fine sub-steps. */
static void op_coalesce(orc *o, int L) {
    olevel *V = &o->lv[L], *Fv = &o->lv[L + 1];
    #pragma omp parallel for schedule(static) if (V->nK > ORC_PAR_MIN)
    for (long k = 0; k < V->nK; k++) {
        int a = V->Ka[k];
        const long *ch = V->Kch + 8 * k;
        double c0 = Fv->f[ch[0] * Q + a], c1 = Fv->f[ch[1] * Q + a], c2 = Fv->f[ch[2] * Q + a], c3 = Fv->f[ch[3] * Q + a];
        double c4 = Fv->f[ch[4] * Q + a], c5 = Fv->f[ch[5] * Q + a], c6 = Fv->f[ch[6] * Q + a], c7 = Fv->f[ch[7] * Q + a];
        double s = ((c0 + c1) + (c2 + c3)) + ((c4 + c5) + (c6 + c7));
        V->f[V->Kc[k] * Q + a] = s / 8.0;
    }
}

/* Alg. 1, NonUniformTimeStep(L). */
static void nonuniform_time_step(orc *o, int L) {
    int finest = o->nlev - 1;
    op_collide(o, L);
    if (L != finest) nonuniform_time_step(o, L + 1);
    if (L != 0) op_explode(o, L);
    op_boundary(o, L);
    op_stream(o, L);
    if (L != finest) op_coalesce(o, L);
    if (L == 0) return;
    op_collide(o, L);
    if (L != finest) nonuniform_time_step(o, L + 1);
    op_boundary(o, L);
    op_stream(o, L);
    if (L != finest) op_coalesce(o, L);
}

void orc_step(orc *o, int n) {
    for (int i = 0; i < n; i++) nonuniform_time_step(o, 0);
}

/* ---------------- construction and access ---------------- */

void orc_destroy(orc *o) {
    if (!o) return;
    for (int L = 0; L < ORC_MAXLEV; L++) {
        olevel *V = &o->lv[L];
        free(V->f); free(V->tmp); free(V->cls); free(V->flag); free(V->inS); free(V->vface);
        free(V->C); free(V->S); free(V->G); free(V->Gp); free(V->Bd); free(V->Kc); free(V->Ka); free(V->Kch);
        free(o->st[L]);
    }
    free(o);
}

orc *orc_create(const orc_desc *d, orc_refine_fn refine, orc_flag_fn flagfn, void *user) {
    lattice_init();
    g_err[0] = 0;
    if (d->B < 4 || (d->B & 1) || d->lmax < 0 || d->lmax >= ORC_MAXLEV || d->nsph > ORC_MAXSPH ||
        d->nreg > ORC_MAXREG || d->nroot[0] < 1 || d->nroot[1] < 1 || d->nroot[2] < 1) {
        snprintf(g_err, sizeof g_err, "invalid description");
        return NULL;
    }
    orc *o = (orc *)calloc(1, sizeof(orc));
    o->d = *d;
    o->refine = refine; o->flagfn = flagfn; o->user = user;
    for (int a = 0; a < 3; a++) {
        o->per[a] = d->bc[2 * a] == BC_PERIODIC;
        if ((d->bc[2 * a] == BC_PERIODIC) != (d->bc[2 * a + 1] == BC_PERIODIC)) {
            snprintf(g_err, sizeof g_err, "periodic faces must come in pairs");
            free(o);
            return NULL;
        }
    }
    if (!build_forest(o)) { orc_destroy(o); return NULL; }
    for (int L = 0; L < o->nlev; L++) set_window(o, L);
    for (int L = 0; L < o->nlev; L++) if (!classify(o, L)) { orc_destroy(o); return NULL; }
    for (int L = 0; L < o->nlev; L++) if (!build_lists(o, L)) { orc_destroy(o); return NULL; }
    for (int L = 0; L < o->nlev; L++) {
        olevel *V = &o->lv[L];
        V->f = (double *)malloc((V->ncell ? V->ncell : 1) * Q * sizeof(double));
        V->tmp = (double *)malloc((V->ncell ? V->ncell : 1) * Q * sizeof(double));
        if (!V->f || !V->tmp) { snprintf(g_err, sizeof g_err, "out of memory (PDFs)"); orc_destroy(o); return NULL; }
        for (long i = 0; i < V->ncell * Q; i++) V->f[i] = NAN;
        memcpy(V->tmp, V->f, V->ncell * Q * sizeof(double));
    }
    for (int L = 0; L < ORC_MAXLEV; L++) { o->le[L] = o->lo[L] = 1.0; o->acc[L][0] = o->acc[L][1] = o->acc[L][2] = 0.0; }
    return o;
}

/* Per-level parameters from the coarse ones: Eq. (omega_scaling_0) for lambda_e (or omega),
 * Eq. (lambda_oL) for lambda_o at fixed Lambda_eo, Eq. (force_scaling) a_L = a_0 / 2^L.
 * For SRT lambda_o equals lambda_e (the TRT operator then coincides with SRT). */
void orc_set_params(orc *o, double le0, double magic, const double a0[3]) {
    for (int L = 0; L < ORC_MAXLEV; L++) {
        o->le[L] = orc_scale_rate(le0, L);
        o->lo[L] = o->d.collision == COLL_TRT ? orc_lambda_odd(o->le[L], magic) : o->le[L];
        for (int a = 0; a < 3; a++) o->acc[L][a] = ldexp(a0 ? a0[a] : 0.0, -L);
    }
}

void orc_set_params_explicit(orc *o, const double *le, const double *lo, const double *acc) {
    for (int L = 0; L < o->nlev; L++) {
        o->le[L] = le[L]; o->lo[L] = lo[L];
        for (int a = 0; a < 3; a++) o->acc[L][a] = acc[3 * L + a];
    }
}

void orc_get_params(const orc *o, double *le, double *lo, double *acc) {
    for (int L = 0; L < o->nlev; L++) {
        le[L] = o->le[L]; lo[L] = o->lo[L];
        for (int a = 0; a < 3; a++) acc[3 * L + a] = o->acc[L][a];
    }
}

void orc_window(const orc *o, int L, int *s, int *n, int *N) {
    for (int a = 0; a < 3; a++) { s[a] = o->lv[L].s[a]; n[a] = o->lv[L].n[a]; N[a] = o->lv[L].N[a]; }
}

void orc_get_class(const orc *o, int L, unsigned char *cls, unsigned char *flag) {
    const olevel *V = &o->lv[L];
    if (cls) memcpy(cls, V->cls, V->ncell);
    if (flag) memcpy(flag, V->flag, V->ncell);
}

/* Initial post-streaming state: f = f^eq(rho, u) on owned fluid cells, NaN elsewhere.
 * rho and u are dense window arrays ([ncell] and [3][ncell]); NULL means rho0 and rest. */
void orc_init_eq(orc *o, int L, const double *rho, const double *u) {
    olevel *V = &o->lv[L];
    for (long i = 0; i < V->ncell * Q; i++) V->f[i] = NAN;
    for (long i = 0; i < V->nC; i++) {
        long c = V->C[i];
        double r = rho ? rho[c] : o->d.rho0;
        double uu[3] = {0.0, 0.0, 0.0};
        if (u) { uu[0] = u[c]; uu[1] = u[V->ncell + c]; uu[2] = u[2 * V->ncell + c]; }
        feq_cell(r, uu, o->d.rho0, V->f + c * Q);
    }
    memcpy(V->tmp, V->f, V->ncell * Q * sizeof(double));
}

/* Dense window copy of the PDFs ([ncell][19]); with post_collision, owned fluid cells
 * hold the state after one more collision of the current (post-streaming) state. */
void orc_get_f(const orc *o, int L, double *out, int post_collision) {
    const olevel *V = &o->lv[L];
    memcpy(out, V->f, V->ncell * Q * sizeof(double));
    if (post_collision)
        for (long i = 0; i < V->nC; i++)
            collide_cell(out + V->C[i] * Q, o->d.collision, o->le[L], o->lo[L], o->acc[L], o->d.rho0);
}

void orc_set_f(orc *o, int L, const double *in) {
    olevel *V = &o->lv[L];
    memcpy(V->f, in, V->ncell * Q * sizeof(double));
}

/* Macroscopic fields of owned fluid cells (Eq. fvelocity; velocity output adds a_L / 2 as in
 * Sec. 2.1); NaN elsewhere. */
void orc_macro(const orc *o, int L, double *rho, double *u) {
    const olevel *V = &o->lv[L];
    for (long c = 0; c < V->ncell; c++) { rho[c] = NAN; u[c] = u[V->ncell + c] = u[2 * V->ncell + c] = NAN; }
    for (long i = 0; i < V->nC; i++) {
        long c = V->C[i];
        const double *f = V->f + c * Q;
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < Q; a++) { r += f[a]; for (int k = 0; k < 3; k++) j[k] += EV[a][k] * f[a]; }
        rho[c] = r;
        for (int k = 0; k < 3; k++) u[k * V->ncell + c] = j[k] / o->d.rho0 + 0.5 * o->acc[L][k];
    }
}

/* Volume-weighted totals over owned fluid cells of all levels: out = {sum w rho, sum w j}
 * with w = 8^-L and j = sum_a e_a f_a of the current (post-streaming) state.  The totals use
 * Neumaier's compensated summation so that the measurement itself does not drift. */
static void neumaier_add(double *sum, double *comp, double v) {
    double t = *sum + v;
    if (fabs(*sum) >= fabs(v)) *comp += (*sum - t) + v;
    else *comp += (v - t) + *sum;
    *sum = t;
}

void orc_mass_momentum(const orc *o, double *out) {
    double s[4] = {0.0, 0.0, 0.0, 0.0}, cmp[4] = {0.0, 0.0, 0.0, 0.0};
    for (int L = 0; L < o->nlev; L++) {
        const olevel *V = &o->lv[L];
        double w = ldexp(1.0, -3 * L);
        for (long i = 0; i < V->nC; i++) {
            const double *f = V->f + V->C[i] * Q;
            for (int a = 0; a < Q; a++) {
                neumaier_add(&s[0], &cmp[0], w * f[a]);
                for (int k = 0; k < 3; k++)
                    if (EV[a][k]) neumaier_add(&s[1 + k], &cmp[1 + k], w * EV[a][k] * f[a]);
            }
        }
    }
    for (int k = 0; k < 4; k++) out[k] = s[k] + cmp[k];
}

/* Owned fluid cell count per level; the cell updates of one coarse step are sum_L N_L 2^L. */
long orc_num_fluid(const orc *o, int L) { return o->lv[L].nC; }
long orc_num_stream(const orc *o, int L) { return o->lv[L].nS; }
long orc_num_ghost(const orc *o, int L) { return o->lv[L].nG; }
long orc_num_coalesce(const orc *o, int L) { return o->lv[L].nK; }

/* Threads the OpenMP loops use (1 without OpenMP). */
int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
