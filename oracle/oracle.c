/*
 * oracle.c -- plain, slow, FP64 CPU oracle of the N-body/SPH interaction path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header or constant table with the
 * CUDA library; both sides only share the seeded input generators.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC.  Contraction is
 * disabled so that every a*b+c is two rounded operations, which makes the
 * discrete decisions below (Morton cells, neighbour ordering) reproducible on
 * any host.
 *
 * Each function follows one step of the method of Hirashima et al. (SC'25,
 * arXiv 2510.23330); the citation is in the comment above it.  Where the paper
 * is silent the reading taken is stated there as well.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXLEV 21

/* ------------------------------------------------------------------------ */
/* Softened pairwise gravity, Sec. 3.5 Eq. 1:                                */
/*   F_ij = -G m_i m_j r_ij / (r_ij^2 + eps_i^2 + eps_j^2)^{3/2},            */
/* reported as the acceleration a_i = F_i / m_i and the potential            */
/*   phi_i = -G sum_{j != i} m_j / (r_ij^2 + eps_i^2 + eps_j^2)^{1/2}.       */
/* asum_i = sum_j |a_ij| (the summation's condition number, for errors).     */
/* ------------------------------------------------------------------------ */
void orc_direct_gravity(int64_t n, const double *x, const double *y, const double *z,
                        const double *m, const double *eps, double G,
                        double *ax, double *ay, double *az, double *phi, double *asum)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
        double sx = 0, sy = 0, sz = 0, sp = 0, sa = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
            double r2 = dx * dx + dy * dy + dz * dz + eps[i] * eps[i] + eps[j] * eps[j];
            double rinv = 1.0 / sqrt(r2);
            double f = G * m[j] * rinv * rinv * rinv;
            sx -= f * dx;
            sy -= f * dy;
            sz -= f * dz;
            sp -= G * m[j] * rinv;
            sa += f * sqrt(dx * dx + dy * dy + dz * dz);
        }
        ax[i] = sx; ay[i] = sy; az[i] = sz; phi[i] = sp; asum[i] = sa;
    }
}

/* ------------------------------------------------------------------------ */
/* Root box of the tree (Sec. 3.4 treecode; the box rule is a reading):      */
/* lo_k = min x_k, ext = max_k (max x_k - lo_k), L = 2^ceil(log2 ext)        */
/* (L = 1 when ext = 0).                                                     */
/* ------------------------------------------------------------------------ */
void orc_root_box(int64_t n, const double *x, const double *y, const double *z,
                  double *lo, double *L)
{
    const double *p[3] = {x, y, z};
    double ext = 0.0;
    for (int k = 0; k < 3; k++) {
        double mn = p[k][0], mx = p[k][0];
        for (int64_t i = 1; i < n; i++) {
            if (p[k][i] < mn) mn = p[k][i];
            if (p[k][i] > mx) mx = p[k][i];
        }
        lo[k] = mn;
        double e = mx - mn;
        if (e > ext) ext = e;
    }
    if (ext <= 0.0) { *L = 1.0; return; }
    double l = 1.0;
    while (l < ext) l *= 2.0;
    while (l / 2.0 >= ext) l /= 2.0;
    *L = l;
}

/* Morton cell of each particle: c_k = min(floor((x_k - lo_k) * 2^21 / L),   */
/* 2^21 - 1); key interleaves bit b of c_x, c_y, c_z at 3b+2, 3b+1, 3b.       */
void orc_morton(int64_t n, const double *x, const double *y, const double *z,
                const double *lo, double L, uint64_t *key,
                int32_t *cx, int32_t *cy, int32_t *cz)
{
    const double scale = 2097152.0 / L; /* 2^21 / L: both powers of two */
    const double *p[3] = {x, y, z};
    int32_t *c[3] = {cx, cy, cz};
    for (int64_t i = 0; i < n; i++) {
        uint64_t k = 0;
        int32_t cc[3];
        for (int a = 0; a < 3; a++) {
            double d = p[a][i] - lo[a];
            double f = floor(d * scale);
            int64_t v = (int64_t)f;
            if (v < 0) v = 0;
            if (v > 2097151) v = 2097151;
            cc[a] = (int32_t)v;
            c[a][i] = (int32_t)v;
        }
        for (int b = 0; b < MAXLEV; b++) {
            k |= (uint64_t)((cc[0] >> b) & 1) << (3 * b + 2);
            k |= (uint64_t)((cc[1] >> b) & 1) << (3 * b + 1);
            k |= (uint64_t)((cc[2] >> b) & 1) << (3 * b);
        }
        key[i] = k;
    }
}

typedef struct { uint64_t key; int64_t idx; } keyidx_t;

static int cmp_keyidx(const void *a, const void *b)
{
    const keyidx_t *p = a, *q = b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return (p->idx > q->idx) - (p->idx < q->idx);
}

/* Particle order along the space-filling curve: by (key, input index). */
void orc_sort_order(int64_t n, const uint64_t *key, int64_t *order)
{
    keyidx_t *t = malloc(sizeof(keyidx_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) { t[i].key = key[i]; t[i].idx = i; }
    qsort(t, (size_t)n, sizeof(keyidx_t), cmp_keyidx);
    for (int64_t i = 0; i < n; i++) order[i] = t[i].idx;
    free(t);
}

/* ------------------------------------------------------------------------ */
/* Octree from sorted keys (Barnes-Hut, Sec. 1 and 3.4).  A cell at level l  */
/* holds the particles sharing the top 3l key bits.  A cell is split when    */
/* it holds more than n_leaf particles and l < 21; its non-empty children    */
/* are appended in Morton order, so the node array is the breadth-first     */
/* list.  Returns the node count, or -1 if cap is too small.                 */
/* ------------------------------------------------------------------------ */
int64_t orc_octree(int64_t n, const uint64_t *skey, int n_leaf, int64_t cap,
                   int32_t *level, uint64_t *prefix, int64_t *first, int64_t *count,
                   int64_t *child, int32_t *nchild)
{
    if (cap < 1) return -1;
    int64_t nn = 1;
    level[0] = 0; prefix[0] = 0; first[0] = 0; count[0] = n; child[0] = -1; nchild[0] = 0;
    for (int64_t k = 0; k < nn; k++) {
        child[k] = -1; nchild[k] = 0;
        int l = level[k];
        if (count[k] <= n_leaf || l >= MAXLEV) continue;
        int sh = 3 * (MAXLEV - (l + 1));
        int64_t b = first[k], e = first[k] + count[k];
        int64_t s = b;
        while (s < e) {
            uint64_t d = (skey[s] >> sh) & 7u;
            int64_t t = s;
            while (t < e && ((skey[t] >> sh) & 7u) == d) t++;
            if (nn >= cap) return -1;
            if (nchild[k] == 0) child[k] = nn;
            nchild[k]++;
            level[nn] = l + 1;
            prefix[nn] = (prefix[k] << 3) | d;
            first[nn] = s;
            count[nn] = t - s;
            child[nn] = -1; nchild[nn] = 0;
            nn++;
            s = t;
        }
    }
    return nn;
}

/* ------------------------------------------------------------------------ */
/* Cell moments (monopole per Sec. 5.4, quadrupole per the disk model):      */
/* M = sum m, com = sum m x / M, traceless Q_kl = sum m (3 d_k d_l - d^2     */
/* delta_kl) with d = x - com, and eps2 = sum m eps^2 / M.  Q is stored as   */
/* (xx, yy, zz, xy, xz, yz).  Inputs are in sorted order.                   */
/* ------------------------------------------------------------------------ */
void orc_moments(int64_t nn, const int64_t *first, const int64_t *count,
                 const double *x, const double *y, const double *z,
                 const double *m, const double *eps,
                 double *M, double *com, double *Q, double *eps2)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < nn; k++) {
        double mt = 0, sx = 0, sy = 0, sz = 0, se = 0;
        for (int64_t j = first[k]; j < first[k] + count[k]; j++) {
            mt += m[j];
            sx += m[j] * x[j]; sy += m[j] * y[j]; sz += m[j] * z[j];
            se += m[j] * eps[j] * eps[j];
        }
        double c0 = sx / mt, c1 = sy / mt, c2 = sz / mt;
        double q[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t j = first[k]; j < first[k] + count[k]; j++) {
            double d0 = x[j] - c0, d1 = y[j] - c1, d2 = z[j] - c2;
            double dd = d0 * d0 + d1 * d1 + d2 * d2;
            q[0] += m[j] * (3 * d0 * d0 - dd);
            q[1] += m[j] * (3 * d1 * d1 - dd);
            q[2] += m[j] * (3 * d2 * d2 - dd);
            q[3] += m[j] * 3 * d0 * d1;
            q[4] += m[j] * 3 * d0 * d2;
            q[5] += m[j] * 3 * d1 * d2;
        }
        M[k] = mt;
        com[3 * k] = c0; com[3 * k + 1] = c1; com[3 * k + 2] = c2;
        for (int a = 0; a < 6; a++) Q[6 * k + a] = q[a];
        eps2[k] = se / mt;
    }
}

/* ------------------------------------------------------------------------ */
/* Groups sharing one interaction list (n_g, Sec. 5.2.2 and 5.2.4): a depth- */
/* first pass from the root; a cell with count <= n_g, or a leaf, becomes a  */
/* group.  Writes group node ids in depth-first order; returns the count.    */
/* ------------------------------------------------------------------------ */
int64_t orc_groups(int64_t nn, const int64_t *count, const int64_t *child,
                   const int32_t *nchild, int64_t n_g, int64_t *groups)
{
    int64_t *stack = malloc(sizeof(int64_t) * (size_t)(nn + 8));
    int64_t sp = 0, ng = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        int64_t k = stack[--sp];
        if (count[k] <= n_g || nchild[k] == 0) { groups[ng++] = k; continue; }
        for (int c = nchild[k] - 1; c >= 0; c--) stack[sp++] = child[k] + c;
    }
    free(stack);
    return ng;
}

/* Integer geometry of cell k: corner C (Morton grid units) and side s. */
static void cell_box(int32_t lev, uint64_t pre, int64_t C[3], int64_t *s)
{
    int64_t c[3] = {0, 0, 0};
    for (int b = 0; b < lev; b++) {
        c[0] |= (int64_t)((pre >> (3 * b + 2)) & 1) << b;
        c[1] |= (int64_t)((pre >> (3 * b + 1)) & 1) << b;
        c[2] |= (int64_t)((pre >> (3 * b)) & 1) << b;
    }
    int sh = MAXLEV - lev;
    for (int a = 0; a < 3; a++) C[a] = c[a] << sh;
    *s = (int64_t)1 << sh;
}

/* ------------------------------------------------------------------------ */
/* Opening test (Barnes-Hut criterion, Sec. 1/3.4; the exact integer form is */
/* a reading).  With the group's bounding box [bmin, bmax] of particle cells */
/* and the cell's centre 2C+s in doubled grid units, d^2 is the squared      */
/* distance from the box to the centre; the cell is opened iff               */
/*   (2s)^2 > theta^2 d^2,                                                  */
/* or the cell's box overlaps the group box (never accept a cell holding     */
/* part of the group).                                                       */
/* ------------------------------------------------------------------------ */
static int must_open(const int64_t bmin[3], const int64_t bmax[3], int32_t lev,
                     uint64_t pre, double theta2)
{
    int64_t C[3], s;
    cell_box(lev, pre, C, &s);
    int overlap = 1;
    int64_t d2 = 0;
    for (int a = 0; a < 3; a++) {
        if (bmin[a] > C[a] + s - 1 || bmax[a] < C[a]) overlap = 0;
        int64_t cen = 2 * C[a] + s;
        int64_t d = 0;
        if (2 * bmin[a] > cen) d = 2 * bmin[a] - cen;
        else if (cen > 2 * bmax[a]) d = cen - 2 * bmax[a];
        d2 += d * d;
    }
    if (overlap) return 1;
    double lhs = (double)(2 * s) * (double)(2 * s);
    return lhs > theta2 * (double)d2;
}

/* Walk for one group: particles of opened leaves go to the particle list    */
/* (EPJ), accepted cells to the cell list (SPJ); depth-first, Morton order.  */
/* The root is always opened.  Returns 0, or -1 if a list overflows.         */
int orc_walk(int64_t g, const int32_t *level, const uint64_t *prefix,
             const int64_t *first, const int64_t *count, const int64_t *child,
             const int32_t *nchild, const int32_t *scx, const int32_t *scy,
             const int32_t *scz, double theta, int64_t nn,
             int64_t epj_cap, int64_t *epj, int64_t *n_epj,
             int64_t spj_cap, int64_t *spj, int64_t *n_spj)
{
    int64_t bmin[3] = {INT64_MAX, INT64_MAX, INT64_MAX};
    int64_t bmax[3] = {INT64_MIN, INT64_MIN, INT64_MIN};
    for (int64_t j = first[g]; j < first[g] + count[g]; j++) {
        int64_t c[3] = {scx[j], scy[j], scz[j]};
        for (int a = 0; a < 3; a++) {
            if (c[a] < bmin[a]) bmin[a] = c[a];
            if (c[a] > bmax[a]) bmax[a] = c[a];
        }
    }
    double th2 = theta * theta;
    int64_t *stack = malloc(sizeof(int64_t) * (size_t)(nn + 8));
    int64_t sp = 0, ne = 0, ns = 0;
    int rc = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        int64_t k = stack[--sp];
        int open = (k == 0) || must_open(bmin, bmax, level[k], prefix[k], th2);
        if (!open) {
            if (ns >= spj_cap) { rc = -1; break; }
            spj[ns++] = k;
        } else if (nchild[k] == 0) {
            for (int64_t j = first[k]; j < first[k] + count[k]; j++) {
                if (ne >= epj_cap) { rc = -1; break; }
                epj[ne++] = j;
            }
            if (rc) break;
        } else {
            for (int c = nchild[k] - 1; c >= 0; c--) stack[sp++] = child[k] + c;
        }
    }
    free(stack);
    *n_epj = ne; *n_spj = ns;
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Particle-cell interaction with a monopole + traceless quadrupole about    */
/* the cell's centre of mass, softened like Eq. 1 with R^2 = r^2 + eps_i^2 + */
/* eps2_cell:                                                                */
/*   a   = G [ -M r/R^3 + Q r/R^5 - (5/2)(r.Q.r) r/R^7 ]                     */
/*   phi = -G [ M/R + (1/2) r.Q.r / R^5 ]                                    */
/* r = x_i - com.  With quad = 0 only the monopole terms are kept.           */
/* ------------------------------------------------------------------------ */
static void pc_term(double rx, double ry, double rz, double e2i, double M,
                    const double *q, double e2c, int quad, double G,
                    double *a, double *ph, double *amag)
{
    double R2 = rx * rx + ry * ry + rz * rz + e2i + e2c;
    double Ri = 1.0 / sqrt(R2);
    double Ri2 = Ri * Ri, Ri3 = Ri2 * Ri;
    double tx = -M * Ri3 * rx, ty = -M * Ri3 * ry, tz = -M * Ri3 * rz;
    double p = -M * Ri;
    if (quad) {
        double Ri5 = Ri3 * Ri2, Ri7 = Ri5 * Ri2;
        double qx = q[0] * rx + q[3] * ry + q[4] * rz;
        double qy = q[3] * rx + q[1] * ry + q[5] * rz;
        double qz = q[4] * rx + q[5] * ry + q[2] * rz;
        double rqr = rx * qx + ry * qy + rz * qz;
        tx += qx * Ri5 - 2.5 * rqr * Ri7 * rx;
        ty += qy * Ri5 - 2.5 * rqr * Ri7 * ry;
        tz += qz * Ri5 - 2.5 * rqr * Ri7 * rz;
        p -= 0.5 * rqr * Ri5;
    }
    a[0] += G * tx; a[1] += G * ty; a[2] += G * tz;
    *ph += G * p;
    *amag += G * sqrt(tx * tx + ty * ty + tz * tz);
}

/* ------------------------------------------------------------------------ */
/* Barnes-Hut group walk gravity, step by step: root box, Morton keys, sort, */
/* octree, moments, groups, one walk per group, then for each i of the group */
/* the particle-particle sum over EPJ (Eq. 1, the j == i potential term      */
/* excluded) plus the particle-cell sum over SPJ.  Inputs and outputs are in */
/* input order.  stats = {nodes, groups, n_pp, n_pc}.  Returns 0 or -1.      */
/* ------------------------------------------------------------------------ */
static double wall_seconds(void)
{
#ifdef _OPENMP
    return omp_get_wtime();
#else
    return 0.0;
#endif
}

int orc_tree_gravity_ex(int64_t n, const double *x, const double *y, const double *z,
                        const double *m, const double *eps, double G, double theta,
                        int n_leaf, int64_t n_g, int quad,
                        double *ax, double *ay, double *az, double *phi, double *asum,
                        int64_t *stats, int64_t gstride, double *times);

int orc_tree_gravity(int64_t n, const double *x, const double *y, const double *z,
                     const double *m, const double *eps, double G, double theta,
                     int n_leaf, int64_t n_g, int quad,
                     double *ax, double *ay, double *az, double *phi, double *asum,
                     int64_t *stats)
{
    return orc_tree_gravity_ex(n, x, y, z, m, eps, G, theta, n_leaf, n_g, quad, ax, ay, az, phi,
                               asum, stats, 1, NULL);
}

/* As orc_tree_gravity; only every gstride-th group is walked and summed (the
 * others are left untouched), and times = {build seconds, walk seconds}.   */
int orc_tree_gravity_ex(int64_t n, const double *x, const double *y, const double *z,
                        const double *m, const double *eps, double G, double theta,
                        int n_leaf, int64_t n_g, int quad,
                        double *ax, double *ay, double *az, double *phi, double *asum,
                        int64_t *stats, int64_t gstride, double *times)
{
    double t0 = wall_seconds(), t1 = t0;
    if (gstride < 1) gstride = 1;
    double lo[3], L;
    orc_root_box(n, x, y, z, lo, &L);
    uint64_t *key = malloc(8 * (size_t)n);
    int32_t *cx = malloc(4 * (size_t)n), *cy = malloc(4 * (size_t)n), *cz = malloc(4 * (size_t)n);
    orc_morton(n, x, y, z, lo, L, key, cx, cy, cz);
    int64_t *ord = malloc(8 * (size_t)n);
    orc_sort_order(n, key, ord);
    uint64_t *sk = malloc(8 * (size_t)n);
    int32_t *scx = malloc(4 * (size_t)n), *scy = malloc(4 * (size_t)n), *scz = malloc(4 * (size_t)n);
    double *sx = malloc(8 * (size_t)n), *sy = malloc(8 * (size_t)n), *sz = malloc(8 * (size_t)n);
    double *sm = malloc(8 * (size_t)n), *se = malloc(8 * (size_t)n);
    for (int64_t i = 0; i < n; i++) {
        int64_t o = ord[i];
        sk[i] = key[o]; scx[i] = cx[o]; scy[i] = cy[o]; scz[i] = cz[o];
        sx[i] = x[o]; sy[i] = y[o]; sz[i] = z[o]; sm[i] = m[o]; se[i] = eps[o];
    }
    int64_t cap = 4 * n + 64;
    int32_t *lev = malloc(4 * (size_t)cap), *nch = malloc(4 * (size_t)cap);
    uint64_t *pre = malloc(8 * (size_t)cap);
    int64_t *fi = malloc(8 * (size_t)cap), *co = malloc(8 * (size_t)cap), *ch = malloc(8 * (size_t)cap);
    int64_t nn = orc_octree(n, sk, n_leaf, cap, lev, pre, fi, co, ch, nch);
    int rc = 0;
    int64_t ng = 0, npp = 0, npc = 0;
    double *M = NULL, *com = NULL, *Q = NULL, *e2 = NULL;
    int64_t *groups = NULL;
    if (nn < 0) { rc = -1; goto done; }
    M = malloc(8 * (size_t)nn); com = malloc(24 * (size_t)nn);
    Q = malloc(48 * (size_t)nn); e2 = malloc(8 * (size_t)nn);
    orc_moments(nn, fi, co, sx, sy, sz, sm, se, M, com, Q, e2);
    groups = malloc(8 * (size_t)nn);
    ng = orc_groups(nn, co, ch, nch, n_g, groups);
    t1 = wall_seconds();
#pragma omp parallel reduction(+ : npp, npc)
    {
        int64_t *epj = malloc(8 * (size_t)(n + 1));
        int64_t *spj = malloc(8 * (size_t)(nn + 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t gi = 0; gi < ng; gi += gstride) {
            int64_t g = groups[gi], ne, ns;
            if (orc_walk(g, lev, pre, fi, co, ch, nch, scx, scy, scz, theta, nn,
                         n + 1, epj, &ne, nn + 1, spj, &ns) != 0) {
#pragma omp atomic write
                rc = -1;
                continue;
            }
            for (int64_t i = fi[g]; i < fi[g] + co[g]; i++) {
                double a[3] = {0, 0, 0}, p = 0, am = 0;
                double e2i = se[i] * se[i];
                for (int64_t t = 0; t < ne; t++) {
                    int64_t j = epj[t];
                    if (j == i) continue;
                    double dx = sx[i] - sx[j], dy = sy[i] - sy[j], dz = sz[i] - sz[j];
                    double r2 = dx * dx + dy * dy + dz * dz + e2i + se[j] * se[j];
                    double ri = 1.0 / sqrt(r2);
                    double f = G * sm[j] * ri * ri * ri;
                    a[0] -= f * dx; a[1] -= f * dy; a[2] -= f * dz;
                    p -= G * sm[j] * ri;
                    am += f * sqrt(dx * dx + dy * dy + dz * dz);
                }
                for (int64_t t = 0; t < ns; t++) {
                    int64_t c = spj[t];
                    pc_term(sx[i] - com[3 * c], sy[i] - com[3 * c + 1], sz[i] - com[3 * c + 2],
                            e2i, M[c], Q + 6 * c, e2[c], quad, G, a, &p, &am);
                }
                int64_t o = ord[i];
                ax[o] = a[0]; ay[o] = a[1]; az[o] = a[2]; phi[o] = p; asum[o] = am;
            }
            npp += ne * co[g];
            npc += ns * co[g];
        }
        free(epj); free(spj);
    }
done:
    if (times) { times[0] = t1 - t0; times[1] = wall_seconds() - t1; }
    if (stats) { stats[0] = nn; stats[1] = ng; stats[2] = npp; stats[3] = npc; }
    free(key); free(cx); free(cy); free(cz); free(ord); free(sk);
    free(scx); free(scy); free(scz); free(sx); free(sy); free(sz); free(sm); free(se);
    free(lev); free(nch); free(pre); free(fi); free(co); free(ch);
    free(M); free(com); free(Q); free(e2); free(groups);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* SPH kernel size (Sec. 5.2.5 iterates to convergence; the definition taken */
/* is exact k-nearest neighbours, self included): for gas particle i the     */
/* neighbour set N_i is the first k entries of all gas particles ordered by  */
/* (d^2, index), with d^2 = (dx*dx + dy*dy) + dz*dz in FP64, and h_i^2 is    */
/* the d^2 of the k-th entry.  Computed for the ns particles in `sample`.    */
/* ------------------------------------------------------------------------ */
typedef struct { double d2; int64_t j; } d2idx_t;

static int cmp_d2idx(const void *a, const void *b)
{
    const d2idx_t *p = a, *q = b;
    if (p->d2 != q->d2) return p->d2 < q->d2 ? -1 : 1;
    return (p->j > q->j) - (p->j < q->j);
}

int orc_knn(int64_t n, const double *x, const double *y, const double *z, int k,
            int64_t ns, const int64_t *sample, int64_t *nbr, double *h2)
{
    if (k > n) return -1;
#pragma omp parallel
    {
        d2idx_t *t = malloc(sizeof(d2idx_t) * (size_t)n);
#pragma omp for schedule(dynamic, 4)
        for (int64_t s = 0; s < ns; s++) {
            int64_t i = sample[s];
            for (int64_t j = 0; j < n; j++) {
                double dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
                double dxx = dx * dx, dyy = dy * dy, dzz = dz * dz;
                double a = dxx + dyy;
                t[j].d2 = a + dzz;
                t[j].j = j;
            }
            qsort(t, (size_t)n, sizeof(d2idx_t), cmp_d2idx);
            for (int c = 0; c < k; c++) nbr[s * k + c] = t[c].j;
            h2[s] = t[k - 1].d2;
        }
        free(t);
    }
    return 0;
}

/* Cubic spline (M4) kernel with compact support h, normalised in 3D:        */
/* W = 8/(pi h^3) {1 - 6q^2 + 6q^3, q <= 1/2; 2(1-q)^3, 1/2 < q <= 1; 0}.    */
/* The paper does not name its kernel; this one is a reading.  dW is dW/dr.  */
static double kern_w(double r, double h)
{
    double q = r / h, s = 8.0 / (M_PI * h * h * h);
    if (q <= 0.5) return s * (1.0 - 6.0 * q * q + 6.0 * q * q * q);
    if (q <= 1.0) { double t = 1.0 - q; return s * 2.0 * t * t * t; }
    return 0.0;
}

static double kern_dw(double r, double h)
{
    double q = r / h, s = 8.0 / (M_PI * h * h * h * h);
    if (q <= 0.5) return s * (-12.0 * q + 18.0 * q * q);
    if (q <= 1.0) { double t = 1.0 - q; return s * (-6.0 * t * t); }
    return 0.0;
}

void orc_kernel_eval(int64_t n, const double *r, double h, double *w, double *dw)
{
    for (int64_t i = 0; i < n; i++) { w[i] = kern_w(r[i], h); dw[i] = kern_dw(r[i], h); }
}

/* ------------------------------------------------------------------------ */
/* SPH density and equation of state ("density and pressure" phase,          */
/* Table 3/4): rho_i = sum_{j in N_i} m_j W(r_ij, h_i) (self included),      */
/* P_i = (gamma-1) rho_i u_i, c_i = sqrt(gamma P_i / rho_i).                 */
/* nbr holds k indices per sampled particle; h2 the squared support radius.  */
/* ------------------------------------------------------------------------ */
/* pressure: 0 = P_i = (gamma - 1) rho_i u_i (density-energy SPH);
 * 1 = the smoothed pressure P_i = (gamma - 1) sum_j m_j u_j W_ij(h_i) of
 * pressure-energy SPH (Table 3 names a "density and pressure" interaction).
 * c_i = sqrt(gamma P_i / rho_i) in both. */
void orc_density(int64_t ns, const int64_t *sample, const double *x, const double *y,
                 const double *z, const double *m, const double *u, int k,
                 const int64_t *nbr, const double *h2, double gamma,
                 double *rho, double *P, double *c, int pressure)
{
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < ns; s++) {
        int64_t i = sample[s];
        double h = sqrt(h2[s]), r = 0.0, q = 0.0;
        for (int t = 0; t < k; t++) {
            int64_t j = nbr[s * k + t];
            double dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
            double w = kern_w(sqrt(dx * dx + dy * dy + dz * dz), h);
            r += m[j] * w;
            q += m[j] * u[j] * w;
        }
        rho[s] = r;
        P[s] = pressure ? (gamma - 1.0) * q : (gamma - 1.0) * r * u[i];
        c[s] = sqrt(gamma * P[s] / r);
    }
}

/* ------------------------------------------------------------------------ */
/* SPH pressure force and energy equation ("hydro force" phase, Table 3/4;   */
/* the formulation is a reading: standard symmetric SPH with the signal-     */
/* velocity artificial viscosity of Monaghan 1997 as written for Gadget-2).  */
/* Over S_i = {j != i : j in N_i or i in N_j}:                              */
/*   a_i  = -sum m_j [P_i/rho_i^2 gW_ij(h_i) + P_j/rho_j^2 gW_ij(h_j)        */
/*                    + Pi_ij gWbar_ij]                                      */
/*   du_i = sum m_j [P_i/rho_i^2 v_ij.gW_ij(h_i) + 1/2 Pi_ij v_ij.gWbar_ij] */
/* gW_ij(h) = W'(r_ij, h) x_ij / r_ij, Wbar = (W(h_i)+W(h_j))/2,            */
/* w = v_ij.x_ij/r_ij, Pi_ij = -(alpha/2)(c_i + c_j - 3w) w / rhobar if      */
/* w < 0 else 0, rhobar = (rho_i + rho_j)/2.  All arrays are full (n gas);   */
/* nbr is n*k.  asum_i = sum |acc term| (condition number).                  */
/* pressure = 1: pressure-energy SPH with the smoothed pressure P (see       */
/* orc_density) in place of the two pressure terms:                         */
/*   a_i  = -sum m_j [(g-1)^2 u_i u_j (gW_ij(h_i)/P_i + gW_ij(h_j)/P_j)      */
/*                    + Pi_ij gWbar_ij]                                      */
/*   du_i = sum m_j [(g-1)^2 u_i u_j / P_i v_ij.gW_ij(h_i)                   */
/*                   + 1/2 Pi_ij v_ij.gWbar_ij],  g = gamma.                 */
/* ------------------------------------------------------------------------ */
int orc_sph_force(int64_t n, const double *x, const double *y, const double *z,
                  const double *vx, const double *vy, const double *vz,
                  const double *m, const double *rho, const double *P, const double *c,
                  const double *h2, int k, const int64_t *nbr, double alpha,
                  double *ax, double *ay, double *az, double *dudt, double *asum,
                  const double *u, double gamma, int pressure, double *dusum)
{
    /* reverse lists: R_j = {i : j in N_i} */
    int64_t *cnt = calloc((size_t)n + 1, 8);
    for (int64_t i = 0; i < n; i++)
        for (int t = 0; t < k; t++) cnt[nbr[i * k + t] + 1]++;
    for (int64_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
    int64_t *rev = malloc(8 * (size_t)(n * k + 1));
    int64_t *fill = malloc(8 * (size_t)(n + 1));
    memcpy(fill, cnt, 8 * (size_t)(n + 1));
    for (int64_t i = 0; i < n; i++)
        for (int t = 0; t < k; t++) rev[fill[nbr[i * k + t]]++] = i;
    free(fill);
#pragma omp parallel
    {
        unsigned char *mark = calloc((size_t)n, 1);
        int64_t *lst = malloc(8 * (size_t)(2 * k + (n > 0 ? n : 1)));
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < n; i++) {
            int64_t nl = 0;
            for (int t = 0; t < k; t++) {
                int64_t j = nbr[i * k + t];
                if (j != i && !mark[j]) { mark[j] = 1; lst[nl++] = j; }
            }
            for (int64_t t = cnt[i]; t < cnt[i + 1]; t++) {
                int64_t j = rev[t];
                if (j != i && !mark[j]) { mark[j] = 1; lst[nl++] = j; }
            }
            double hi = sqrt(h2[i]);
            double a0 = 0, a1 = 0, a2 = 0, du = 0, am = 0, dm = 0;
            double pi_ = P[i] / (rho[i] * rho[i]);
            for (int64_t t = 0; t < nl; t++) {
                int64_t j = lst[t];
                mark[j] = 0;
                double hj = sqrt(h2[j]);
                double dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
                double r = sqrt(dx * dx + dy * dy + dz * dz);
                double dvx = vx[i] - vx[j], dvy = vy[i] - vy[j], dvz = vz[i] - vz[j];
                double dwi = kern_dw(r, hi), dwj = kern_dw(r, hj);
                double pj_ = P[j] / (rho[j] * rho[j]);
                double ex = 0, ey = 0, ez = 0, w = 0;
                if (r > 0) { ex = dx / r; ey = dy / r; ez = dz / r; w = dvx * ex + dvy * ey + dvz * ez; }
                double visc = 0.0;
                if (w < 0) {
                    double vsig = c[i] + c[j] - 3.0 * w;
                    visc = -0.5 * alpha * vsig * w / (0.5 * (rho[i] + rho[j]));
                }
                double dwbar = 0.5 * (dwi + dwj);
                double ci = pi_, cj = pj_;  /* coefficients of gW(h_i) and gW(h_j) */
                if (pressure) {
                    double uu = (gamma - 1.0) * (gamma - 1.0) * u[i] * u[j];
                    ci = uu / P[i];
                    cj = uu / P[j];
                }
                double f = ci * dwi + cj * dwj + visc * dwbar;
                double tx = m[j] * f * ex, ty = m[j] * f * ey, tz = m[j] * f * ez;
                a0 -= tx; a1 -= ty; a2 -= tz;
                am += sqrt(tx * tx + ty * ty + tz * tz);
                double vdotg = dvx * ex + dvy * ey + dvz * ez;
                du += m[j] * (ci * dwi * vdotg + 0.5 * visc * dwbar * vdotg);
                /* the scale of the du/dt sum: its pressure and viscosity terms in magnitude */
                dm += fabs(m[j] * ci * dwi * vdotg) + fabs(m[j] * 0.5 * visc * dwbar * vdotg);
            }
            ax[i] = a0; ay[i] = a1; az[i] = a2; dudt[i] = du; asum[i] = am;
            if (dusum) dusum[i] = dm;
        }
        free(mark); free(lst);
    }
    free(cnt); free(rev);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Voxelisation of one supernova region (Sec. 3.3: particles mapped to a     */
/* 64^3 grid by SPH kernel convolution and the Shepard method).  Voxel       */
/* centres x_v = lo + (i + 1/2) side/grid.  Accumulators per voxel:          */
/*   acc[0] = sum m_j W(|x_v - x_j|, h_j)             (density)              */
/*   acc[1] = sum (m_j/rho_j) W                       (Shepard denominator)   */
/*   acc[2..5] = sum f_j (m_j/rho_j) W, f = T, vx, vy, vz                    */
/* h_j is the kernel support.  acc has 6 * grid^3 doubles, voxel-major.    */
/* ------------------------------------------------------------------------ */
void orc_voxelise(int64_t n, const double *x, const double *y, const double *z, const double *m,
                  const double *h, const double *rho, const double *T, const double *vx,
                  const double *vy, const double *vz, const double *lo, double side, int grid,
                  double *acc)
{
    double d = side / grid;
    memset(acc, 0, sizeof(double) * 6 * (size_t)grid * grid * grid);
    for (int64_t j = 0; j < n; j++) {
        double p[3] = {x[j], y[j], z[j]};
        int i0[3], i1[3];
        for (int a = 0; a < 3; a++) {
            i0[a] = (int)floor((p[a] - h[j] - lo[a]) / d - 0.5);
            i1[a] = (int)ceil((p[a] + h[j] - lo[a]) / d - 0.5);
            if (i0[a] < 0) i0[a] = 0;
            if (i1[a] > grid - 1) i1[a] = grid - 1;
        }
        double wr = m[j] / rho[j];
        for (int iz = i0[2]; iz <= i1[2]; iz++)
            for (int iy = i0[1]; iy <= i1[1]; iy++)
                for (int ix = i0[0]; ix <= i1[0]; ix++) {
                    double dx = lo[0] + (ix + 0.5) * d - p[0];
                    double dy = lo[1] + (iy + 0.5) * d - p[1];
                    double dz = lo[2] + (iz + 0.5) * d - p[2];
                    double r = sqrt(dx * dx + dy * dy + dz * dz);
                    double w = kern_w(r, h[j]);
                    if (w <= 0.0) continue;
                    double *a = acc + 6 * (((size_t)iz * grid + iy) * grid + ix);
                    a[0] += m[j] * w;
                    a[1] += wr * w;
                    a[2] += T[j] * wr * w;
                    a[3] += vx[j] * wr * w;
                    a[4] += vy[j] * wr * w;
                    a[5] += vz[j] * wr * w;
                }
    }
}

/* SplitMix64 (Steele, Lea & Flood 2014; the constants of Vigna's public    */
/* reference version) and the counter-based uniform draw used by the remap: */
/*   U(seed, id, k) = (splitmix64(splitmix64(seed + id) + k) >> 11) 2^-53.   */
static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64(uint64_t x) { return splitmix64(x); }

double orc_uniform(uint64_t seed, uint64_t id, uint64_t k)
{
    return (double)(splitmix64(splitmix64(seed + id) + k) >> 11) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------ */
/* Grid -> particles by Gibbs sampling (Sec. 3.3: the predicted grid is      */
/* turned back into as many particles as went in, by a Markov chain Monte    */
/* Carlo method).  Reading: each particle starts in the voxel that holds its */
/* old position and makes `sweeps` Gibbs sweeps over x, y, z; each draw picks */
/* a voxel along the current line with probability proportional to the      */
/* voxel weight w (the predicted density).  Draw k of particle `id` uses    */
/* U(seed, id, k), k = 3 s + axis; the final offsets inside the voxel use    */
/* k = 3 sweeps + axis.  The CDF is FP64, summed from index 0 upwards, and   */
/* the voxel is the first index whose inclusive CDF exceeds U * total.      */
/* out: 3 voxel indices and 3 positions per particle.                        */
/* ------------------------------------------------------------------------ */
void orc_gibbs_remap(int64_t n, const int64_t *id, const int32_t *start, const double *w, int grid,
                     const double *lo, double side, uint64_t seed, int sweeps, int32_t *vox,
                     double *pos)
{
    double d = side / grid;
    for (int64_t j = 0; j < n; j++) {
        int c[3] = {start[3 * j], start[3 * j + 1], start[3 * j + 2]};
        uint64_t k = 0;
        for (int s = 0; s < sweeps; s++)
            for (int a = 0; a < 3; a++, k++) {
                double tot = 0.0;
                for (int i = 0; i < grid; i++) {
                    int cc[3] = {c[0], c[1], c[2]};
                    cc[a] = i;
                    tot += w[((size_t)cc[2] * grid + cc[1]) * grid + cc[0]];
                }
                double target = orc_uniform(seed, (uint64_t)id[j], k) * tot;
                double cum = 0.0;
                int pick = grid - 1;
                for (int i = 0; i < grid; i++) {
                    int cc[3] = {c[0], c[1], c[2]};
                    cc[a] = i;
                    cum += w[((size_t)cc[2] * grid + cc[1]) * grid + cc[0]];
                    if (cum > target) { pick = i; break; }
                }
                c[a] = pick;
            }
        for (int a = 0; a < 3; a++) {
            vox[3 * j + a] = c[a];
            pos[3 * j + a] = lo[a] + (c[a] + orc_uniform(seed, (uint64_t)id[j], (uint64_t)(3 * sweeps + a))) * d;
        }
    }
}

/* Eq. 1 direct sum for the ns particles listed in `sample` only (used to
 * check full-size runs on a subsample).  Outputs have length ns. */
void orc_direct_gravity_sample(int64_t n, const double *x, const double *y, const double *z,
                               const double *m, const double *eps, double G, int64_t ns,
                               const int64_t *sample, double *ax, double *ay, double *az,
                               double *phi, double *asum)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t s = 0; s < ns; s++) {
        int64_t i = sample[s];
        double sx = 0, sy = 0, sz = 0, sp = 0, sa = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
            double r2 = dx * dx + dy * dy + dz * dz + eps[i] * eps[i] + eps[j] * eps[j];
            double rinv = 1.0 / sqrt(r2);
            double f = G * m[j] * rinv * rinv * rinv;
            sx -= f * dx;
            sy -= f * dy;
            sz -= f * dz;
            sp -= G * m[j] * rinv;
            sa += f * sqrt(dx * dx + dy * dy + dz * dz);
        }
        ax[s] = sx; ay[s] = sy; az[s] = sz; phi[s] = sp; asum[s] = sa;
    }
}

/* ------------------------------------------------------------------------ */
/* Largest signal velocity of each gas particle over its symmetric pairs    */
/* S_i (the CFL condition of Sec. 1; the signal velocity is a reading):      */
/*   vsig_i = max(2 c_i, max_j c_i + c_j - 3 min(w_ij, 0)).                  */
/* ------------------------------------------------------------------------ */
void orc_sph_vsig(int64_t n, const double *x, const double *y, const double *z,
                  const double *vx, const double *vy, const double *vz, const double *c,
                  int k, const int64_t *nbr, double *vsig)
{
    for (int64_t i = 0; i < n; i++) vsig[i] = 2.0 * c[i];
    for (int64_t i = 0; i < n; i++) {
        for (int t = 0; t < k; t++) {
            int64_t j = nbr[i * k + t];
            if (j == i) continue;
            double dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            double w = 0.0;
            if (r > 0) w = ((vx[i] - vx[j]) * dx + (vy[i] - vy[j]) * dy + (vz[i] - vz[j]) * dz) / r;
            double v = c[i] + c[j] - 3.0 * (w < 0.0 ? w : 0.0);
            /* the pair belongs to S_i and to S_j */
            if (v > vsig[i]) vsig[i] = v;
            if (v > vsig[j]) vsig[j] = v;
        }
    }
}
