/*
 * bh_oracle.c -- plain CPU FP64 oracle for the group-shared Barnes-Hut force
 * evaluation of Iwasawa et al., "Implementation and performance of Barnes-Hut
 * N-body algorithm on extreme-scale heterogeneous many-core architectures"
 * (arXiv:1907.02289).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition that the CUDA library is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * library never calls it and shares no code, header or table with it.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off [-fopenmp] -shared -fPIC.
 * -ffp-contract=off is required: every floating-point expression below is
 * evaluated exactly as written (left to right, one rounding per operation),
 * so keys, boxes, moments and opening decisions are reproducible bit for bit.
 *
 * Readings of the paper that this file fixes (the paper leaves them open):
 *  - keys: 21 levels, 63-bit Morton key, bit 3b+2 = bit b of q_x, 3b+1 of
 *    q_y, 3b of q_z, q = min(floor((x-lo)*S), 2^21-1), S = 2^21/L, L = largest
 *    extent of the root box (1 if that is 0);
 *  - octree: a node at level l splits on the digit of level l+1 when it holds
 *    more than n_leaf particles and l < 21; nodes are numbered breadth-first,
 *    key order within a level;
 *  - groups (Sec. 4.2, groups built "using the tree structure itself"): the
 *    maximal nodes holding at most n_g particles (a level-21 leaf with more is
 *    a group anyway), ordered by first particle;
 *  - opening test on integer boxes: see orc_mac_open();
 *  - lists: depth-first walk in octant order, so both lists come out ordered
 *    by first particle;
 *  - Eq. (1) read as an acceleration, with Plummer softening eps added to the
 *    gravity part and gravity held at its r_coll value inside r_coll;
 *  - cell term: monopole about the centre of mass (Sec. 5.1) plus the
 *    textbook traceless quadrupole (order 2);
 *  - cylindrical frame (Sec. 4.3): keys, tree and opening test on
 *    (phi, r, z), phi from a fixed-operation atan (see orc_phi()), periodic
 *    in phi, contact clause from r_coll / r_min (see orc_cyl_geometry()).
 * Parity pins for every function live in tests/test_oracle_*.py.
 * Parity unpinned: the values of kappa and eta (the paper prints only the
 * radial restitution coefficient 0.5) and the accuracy of the tree force at
 * theta > 0 (the paper prints no force error).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_LEVELS 21
#define ORC_QMAX 2097151u /* 2^21 - 1 */

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Root box (Sec. 4.2 step 3a: the local tree is built from the particles).
 * Returns 0, or -1 when a coordinate is not finite.
 * ---------------------------------------------------------------------- */
int orc_root_box(int64_t n, const double* x, const double* y, const double* z,
                 double* lo, double* L)
{
    const double* c[3] = {x, y, z};
    double mn[3], mx[3];
    for (int a = 0; a < 3; ++a) {
        mn[a] = INFINITY;
        mx[a] = -INFINITY;
    }
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            double v = c[a][i];
            if (!isfinite(v)) return -1;
            if (v < mn[a]) mn[a] = v;
            if (v > mx[a]) mx[a] = v;
        }
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (n == 0) mn[a] = mx[a] = 0.0;
        lo[a] = mn[a];
        if (mx[a] - mn[a] > ext) ext = mx[a] - mn[a];
    }
    *L = (ext > 0.0) ? ext : 1.0;
    return 0;
}

/* Grid coordinate of one axis: min(floor((v - lo) * S), 2^21 - 1). */
static uint32_t orc_quantise(double v, double lo, double S)
{
    double t = floor((v - lo) * S);
    if (t < 0.0) t = 0.0;
    if (t > (double)ORC_QMAX) t = (double)ORC_QMAX;
    return (uint32_t)t;
}

/* Bit b of q goes to bit 3b of the result (written bit by bit on purpose). */
static uint64_t orc_spread(uint32_t q)
{
    uint64_t r = 0;
    for (int b = 0; b < ORC_LEVELS; ++b) r |= (uint64_t)((q >> b) & 1u) << (3 * b);
    return r;
}

/* Inverse of orc_spread for the bits at positions 3b + shift. */
static uint32_t orc_gather(uint64_t k, int shift)
{
    uint32_t q = 0;
    for (int b = 0; b < ORC_LEVELS; ++b) q |= (uint32_t)((k >> (3 * b + shift)) & 1u) << b;
    return q;
}

/* Morton keys (the spatial sort key of Sec. 4.2, "sorting" in tree build). */
void orc_keys(int64_t n, const double* x, const double* y, const double* z,
              const double* lo, double L, uint64_t* key)
{
    double S = 2097152.0 / L;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        uint32_t qx = orc_quantise(x[i], lo[0], S);
        uint32_t qy = orc_quantise(y[i], lo[1], S);
        uint32_t qz = orc_quantise(z[i], lo[2], S);
        key[i] = (orc_spread(qx) << 2) | (orc_spread(qy) << 1) | orc_spread(qz);
    }
}

/* ------------------------------------------------------------------------
 * Sec. 4.3: keys, tree and opening test in cylindrical coordinates
 * (phi, r, z), which for a narrow ring at r ~ 1 measure distance like
 * (x, y, z) (the paper's Eq. for ds^2); forces stay Cartesian.
 *
 * phi and r are FP32 numbers (a tree coordinate only has to place a
 * particle within its key cell, 2^-21 of the box, and the contact clause's
 * margin covers their error): x and y are rounded to FP32; phi comes from
 * atan reduced to [0, tan(pi/12)] by
 * atan(t) = pi/6 + atan((sqrt(3) t - 1) / (t + sqrt(3))) and the Taylor
 * series u - u^3/3 + ... - u^11/11 (truncation below 3e-9 rad), then placed
 * in its octant; r = sqrt(x^2 + y^2).  Only IEEE-rounded FP32 +, -, *, / and
 * sqrt are used, in a fixed order, so the angle (and the key) is a
 * deterministic function of (x, y); its error is below 1e-6 rad.
 * ---------------------------------------------------------------------- */
static float orc_atan01(float t)
{
    const float sqrt3 = 1.7320508075688772f, tan15 = 0.2679491924311227f, pi6 = 0.5235987755982988f;
    float base = 0.0f, u = t;
    if (t > tan15) {
        u = (t * sqrt3 - 1.0f) / (t + sqrt3);
        base = pi6;
    }
    float u2 = u * u;
    float p = -1.0f / 11.0f;
    p = p * u2 + 1.0f / 9.0f;
    p = p * u2 + -1.0f / 7.0f;
    p = p * u2 + 1.0f / 5.0f;
    p = p * u2 + -1.0f / 3.0f;
    p = p * u2 + 1.0f;
    return base + u * p;
}

static float orc_phi(float x, float y)
{
    const float pi2 = 1.5707963267948966f, pi = 3.141592653589793f, twopi = 6.283185307179586f;
    float ax = fabsf(x), ay = fabsf(y);
    float mx = ax > ay ? ax : ay, mn = ax > ay ? ay : ax;
    if (mx == 0.0f) return 0.0f;
    float a = orc_atan01(mn / mx);
    if (ay > ax) a = pi2 - a;
    if (x < 0.0f) a = pi - a;
    if (y < 0.0f) a = twopi - a;
    return a;
}

void orc_cyl(int64_t n, const double* x, const double* y, double* phi, double* r)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const float xf = (float)x[i], yf = (float)y[i];
        phi[i] = (double)orc_phi(xf, yf);
        r[i] = (double)sqrtf(xf * xf + yf * yf);
    }
}

/* Grid coordinates recovered from keys: q[3*i + axis]. */
void orc_key_coords(int64_t n, const uint64_t* key, uint32_t* q)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        q[3 * i + 0] = orc_gather(key[i], 2);
        q[3 * i + 1] = orc_gather(key[i], 1);
        q[3 * i + 2] = orc_gather(key[i], 0);
    }
}

/* ------------------------------------------------------------------------
 * Sort (Sec. 4.2: "the most time-consuming part of the tree construction").
 * perm[r] = original index of the particle of rank r; ties keep the original
 * order, i.e. this is a stable sort by key.
 * ---------------------------------------------------------------------- */
static const uint64_t* orc_sort_keys;
static int orc_cmp(const void* a, const void* b)
{
    uint32_t i = *(const uint32_t*)a, j = *(const uint32_t*)b;
    uint64_t ki = orc_sort_keys[i], kj = orc_sort_keys[j];
    if (ki != kj) return ki < kj ? -1 : 1;
    return i < j ? -1 : (i > j ? 1 : 0);
}
void orc_sort(int64_t n, const uint64_t* key, uint32_t* perm)
{
    for (int64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
    orc_sort_keys = key;
    qsort(perm, (size_t)n, sizeof(uint32_t), orc_cmp);
    orc_sort_keys = NULL;
}

/* ------------------------------------------------------------------------
 * Octree over sorted keys (Sec. 4.2 step 3a).
 * ---------------------------------------------------------------------- */
static int orc_digit(uint64_t k, int level) /* octant of level `level` (1..21) */
{
    return (int)((k >> (3 * (ORC_LEVELS - level))) & 7u);
}

static int64_t orc_count_rec(const uint64_t* sk, int64_t b, int64_t e, int level, int n_leaf)
{
    int64_t total = 1;
    if (e - b > n_leaf && level < ORC_LEVELS) {
        int64_t i = b;
        for (int o = 0; o < 8; ++o) {
            int64_t j = i;
            while (j < e && orc_digit(sk[j], level + 1) == o) ++j;
            if (j > i) total += orc_count_rec(sk, i, j, level + 1, n_leaf);
            i = j;
        }
    }
    return total;
}

/* Number of nodes the tree over sorted keys will have. */
int64_t orc_tree_count(int64_t n, const uint64_t* skey, int n_leaf)
{
    if (n <= 0) return 0;
    return orc_count_rec(skey, 0, n, 0, n_leaf);
}

/* Breadth-first build: the node array doubles as the queue, so every level
 * is contiguous and children of a node are contiguous and in octant order.
 * Returns the node count, or -1 if cap is too small. */
int64_t orc_tree(int64_t n, const uint64_t* skey, int n_leaf, int64_t cap,
                 uint8_t* level, uint32_t* begin, uint32_t* end, int32_t* parent,
                 int32_t* first_child, uint8_t* nchild)
{
    if (n <= 0) return 0;
    if (cap < 1) return -1;
    int64_t count = 1;
    level[0] = 0;
    begin[0] = 0;
    end[0] = (uint32_t)n;
    parent[0] = -1;
    for (int64_t h = 0; h < count; ++h) {
        first_child[h] = -1;
        nchild[h] = 0;
        if ((int64_t)(end[h] - begin[h]) > n_leaf && level[h] < ORC_LEVELS) {
            int64_t i = begin[h];
            for (int o = 0; o < 8; ++o) {
                int64_t j = i;
                while (j < (int64_t)end[h] && orc_digit(skey[j], level[h] + 1) == o) ++j;
                if (j > i) {
                    if (count >= cap) return -1;
                    if (nchild[h] == 0) first_child[h] = (int32_t)count;
                    level[count] = (uint8_t)(level[h] + 1);
                    begin[count] = (uint32_t)i;
                    end[count] = (uint32_t)j;
                    parent[count] = (int32_t)h;
                    nchild[h]++;
                    count++;
                }
                i = j;
            }
        }
    }
    return count;
}

/* Integer tight boxes: qlo/qhi[3*node + axis] = min/max grid coordinate of
 * the node's particles (q from orc_key_coords in sorted order). */
void orc_qboxes(int64_t n_nodes, const uint32_t* begin, const uint32_t* end,
                const int32_t* first_child, const uint8_t* nchild, const uint32_t* q,
                uint32_t* qlo, uint32_t* qhi)
{
    for (int64_t k = n_nodes - 1; k >= 0; --k) {
        for (int a = 0; a < 3; ++a) {
            uint32_t lo = ORC_QMAX, hi = 0;
            if (nchild[k] == 0) {
                for (uint32_t i = begin[k]; i < end[k]; ++i) {
                    if (q[3 * (int64_t)i + a] < lo) lo = q[3 * (int64_t)i + a];
                    if (q[3 * (int64_t)i + a] > hi) hi = q[3 * (int64_t)i + a];
                }
            } else {
                for (int c = 0; c < nchild[k]; ++c) {
                    int64_t ch = first_child[k] + c;
                    if (qlo[3 * ch + a] < lo) lo = qlo[3 * ch + a];
                    if (qhi[3 * ch + a] > hi) hi = qhi[3 * ch + a];
                }
            }
            qlo[3 * k + a] = lo;
            qhi[3 * k + a] = hi;
        }
    }
}

/* ------------------------------------------------------------------------
 * Moments (Sec. 4.2: node quantities are refreshed every step; Sec. 5.1:
 * centre-of-mass approximation).  Children have larger ids than parents, so
 * one pass in decreasing id is bottom-up.  Leaves sum their particles in
 * particle order; internal nodes sum their children in octant order.
 * Q[6*k + 0..5] = Qxx, Qyy, Qzz, Qxy, Qxz, Qyz, with
 * Q_ab = sum m (3 d_a d_b - d^2 delta_ab), d = x - c.  order 1 leaves Q = 0.
 * A node of zero total mass takes its first particle's position as centre.
 * ---------------------------------------------------------------------- */
void orc_moments(int64_t n_nodes, const uint32_t* begin, const uint32_t* end,
                 const int32_t* first_child, const uint8_t* nchild, const double* x,
                 const double* y, const double* z, const double* m, int order, double* M,
                 double* cx, double* cy, double* cz, double* Q)
{
    for (int64_t k = n_nodes - 1; k >= 0; --k) {
        double Mk = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        double q[6] = {0, 0, 0, 0, 0, 0};
        if (nchild[k] == 0) {
            for (uint32_t i = begin[k]; i < end[k]; ++i) {
                Mk = Mk + m[i];
                sx = sx + m[i] * x[i];
                sy = sy + m[i] * y[i];
                sz = sz + m[i] * z[i];
            }
            if (Mk > 0.0) {
                cx[k] = sx / Mk;
                cy[k] = sy / Mk;
                cz[k] = sz / Mk;
            } else {
                cx[k] = x[begin[k]];
                cy[k] = y[begin[k]];
                cz[k] = z[begin[k]];
            }
            if (order >= 2)
                for (uint32_t i = begin[k]; i < end[k]; ++i) {
                    double dx = x[i] - cx[k], dy = y[i] - cy[k], dz = z[i] - cz[k];
                    double d2 = dx * dx + dy * dy + dz * dz;
                    q[0] = q[0] + m[i] * (3.0 * dx * dx - d2);
                    q[1] = q[1] + m[i] * (3.0 * dy * dy - d2);
                    q[2] = q[2] + m[i] * (3.0 * dz * dz - d2);
                    q[3] = q[3] + m[i] * (3.0 * dx * dy);
                    q[4] = q[4] + m[i] * (3.0 * dx * dz);
                    q[5] = q[5] + m[i] * (3.0 * dy * dz);
                }
        } else {
            int64_t f = first_child[k];
            for (int c = 0; c < nchild[k]; ++c) {
                Mk = Mk + M[f + c];
                sx = sx + M[f + c] * cx[f + c];
                sy = sy + M[f + c] * cy[f + c];
                sz = sz + M[f + c] * cz[f + c];
            }
            if (Mk > 0.0) {
                cx[k] = sx / Mk;
                cy[k] = sy / Mk;
                cz[k] = sz / Mk;
            } else {
                cx[k] = cx[f];
                cy[k] = cy[f];
                cz[k] = cz[f];
            }
            if (order >= 2)
                for (int c = 0; c < nchild[k]; ++c) {
                    /* parallel-axis shift of the child's quadrupole */
                    double Mc = M[f + c];
                    double dx = cx[f + c] - cx[k], dy = cy[f + c] - cy[k], dz = cz[f + c] - cz[k];
                    double d2 = dx * dx + dy * dy + dz * dz;
                    const double* qc = Q + 6 * (f + c);
                    q[0] = q[0] + qc[0] + Mc * (3.0 * dx * dx - d2);
                    q[1] = q[1] + qc[1] + Mc * (3.0 * dy * dy - d2);
                    q[2] = q[2] + qc[2] + Mc * (3.0 * dz * dz - d2);
                    q[3] = q[3] + qc[3] + Mc * (3.0 * dx * dy);
                    q[4] = q[4] + qc[4] + Mc * (3.0 * dx * dz);
                    q[5] = q[5] + qc[5] + Mc * (3.0 * dy * dz);
                }
        }
        M[k] = Mk;
        for (int a = 0; a < 6; ++a) Q[6 * k + a] = q[a];
    }
}

/* ------------------------------------------------------------------------
 * Groups (Sec. 4.2: groups of neighbouring particles made from the tree).
 * A node is a group when it holds at most n_g particles (or is a leaf) and
 * it is the root or its parent holds more than n_g.  Output: group node ids
 * ordered by first particle.  Returns the number of groups.
 * ---------------------------------------------------------------------- */
static const uint32_t* orc_grp_begin;
static int orc_grp_cmp(const void* a, const void* b)
{
    uint32_t ba = orc_grp_begin[*(const int32_t*)a], bb = orc_grp_begin[*(const int32_t*)b];
    return ba < bb ? -1 : (ba > bb ? 1 : 0);
}
int64_t orc_groups(int64_t n_nodes, const uint32_t* begin, const uint32_t* end,
                   const int32_t* parent, const uint8_t* nchild, int n_g, int32_t* groups)
{
    int64_t ng = 0;
    for (int64_t k = 0; k < n_nodes; ++k) {
        int64_t cnt = (int64_t)end[k] - begin[k];
        int small = (cnt <= n_g) || (nchild[k] == 0);
        int top = (parent[k] < 0) || ((int64_t)end[parent[k]] - begin[parent[k]] > n_g);  /* a root */
        if (small && top) groups[ng++] = (int32_t)k;
    }
    orc_grp_begin = begin;
    qsort(groups, (size_t)ng, sizeof(int32_t), orc_grp_cmp);
    orc_grp_begin = NULL;
    return ng;
}

/* ------------------------------------------------------------------------
 * Opening test (the paper names theta but prints no criterion).
 * Boxes are the integer tight boxes in grid cells of side h = L / 2^21.
 * Per axis the gap in whole cells is
 *     delta = max(0, clo - ghi - 1, glo - chi - 1),
 * a lower bound of the true gap / h.  d2 = dx^2 + dy^2 + dz^2 (exact integer).
 * The node side at level l is s = 2^(21-l) cells.  The node is opened iff
 *     th2 * d2 < s^2        (one IEEE double multiply, th2 = theta*theta)
 *  or d2 <= rcq2            (rcq = r_coll * S, rcq2 = rcq*rcq),
 * the second clause keeping every possible contact partner a particle.
 * ---------------------------------------------------------------------- */
static int orc_mac_open(const uint32_t* glo, const uint32_t* ghi, const uint32_t* clo,
                        const uint32_t* chi, int level, double th2, double rcq2, int64_t period)
{
    int64_t d2 = 0;
    for (int a = 0; a < 3; ++a) {
        int64_t delta = 0;
        int64_t t1 = (int64_t)clo[a] - (int64_t)ghi[a] - 1;
        int64_t t2 = (int64_t)glo[a] - (int64_t)chi[a] - 1;
        if (t1 > delta) delta = t1;
        if (t2 > delta) delta = t2;
        if (a == 0 && period > 0 && delta > 0) {
            /* periodic phi axis: the shorter way round */
            int64_t w = (t1 > 0) ? (int64_t)glo[a] + period - (int64_t)chi[a] - 1
                                 : (int64_t)clo[a] + period - (int64_t)ghi[a] - 1;
            if (w < 0) w = 0;
            if (w < delta) delta = w;
        }
        d2 += delta * delta;
    }
    double s = ldexp(1.0, ORC_LEVELS - level);
    double s2 = s * s;
    return (th2 * (double)d2 < s2) || ((double)d2 <= rcq2);
}

typedef struct {
    const uint8_t* level;
    const int32_t* first_child;
    const uint8_t* nchild;
    const uint32_t* qlo;
    const uint32_t* qhi;
    double th2, rcq2;
    int64_t period;
} orc_walk_tree;

/* Depth-first walk in octant order for group node g (Sec. 4.2 step 3d:
 * one traversal per group builds its particle and node lists).  Opened
 * leaves go to P, accepted nodes to C.  With P/C NULL it only counts. */
static void orc_walk_rec(const orc_walk_tree* t, int32_t g, int32_t node, int32_t* P,
                         int64_t* np, int32_t* C, int64_t* nc)
{
    const uint32_t* glo = t->qlo + 3 * (int64_t)g;
    const uint32_t* ghi = t->qhi + 3 * (int64_t)g;
    if (orc_mac_open(glo, ghi, t->qlo + 3 * (int64_t)node, t->qhi + 3 * (int64_t)node,
                     t->level[node], t->th2, t->rcq2, t->period)) {
        if (t->nchild[node] == 0) {
            if (P) P[*np] = node;
            (*np)++;
        } else {
            for (int c = 0; c < t->nchild[node]; ++c)
                orc_walk_rec(t, g, t->first_child[node] + c, P, np, C, nc);
        }
    } else {
        if (C) C[*nc] = node;
        (*nc)++;
    }
}

/* Interaction lists of every group, in CSR form.  Call once with P and C NULL
 * to get pp_off / pc_off (sizes ng+1), then again with the arrays. */
void orc_lists_ex(int64_t ng, const int32_t* groups, const uint8_t* level,
                  const int32_t* first_child, const uint8_t* nchild, const uint32_t* qlo,
                  const uint32_t* qhi, double theta, double rcq2, int64_t period, int64_t* pp_off,
                  int32_t* P, int64_t* pc_off, int32_t* C)
{
    orc_walk_tree t;
    t.level = level;
    t.first_child = first_child;
    t.nchild = nchild;
    t.qlo = qlo;
    t.qhi = qhi;
    t.th2 = theta * theta;
    t.rcq2 = rcq2;
    t.period = period;
    if (P == NULL) {
        pp_off[0] = 0;
        pc_off[0] = 0;
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t k = 0; k < ng; ++k) {
            int64_t np = 0, nc = 0;
            orc_walk_rec(&t, groups[k], 0, NULL, &np, NULL, &nc);
            pp_off[k + 1] = np;
            pc_off[k + 1] = nc;
        }
        for (int64_t k = 0; k < ng; ++k) {
            pp_off[k + 1] += pp_off[k];
            pc_off[k + 1] += pc_off[k];
        }
        return;
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < ng; ++k) {
        int64_t np = 0, nc = 0;
        orc_walk_rec(&t, groups[k], 0, P + pp_off[k], &np, C + pc_off[k], &nc);
    }
}

/* Cartesian frame: contact threshold (r_coll S)^2 in grid units, no period. */
void orc_lists(int64_t ng, const int32_t* groups, const uint8_t* level,
               const int32_t* first_child, const uint8_t* nchild, const uint32_t* qlo,
               const uint32_t* qhi, double theta, double r_coll, double L, int64_t* pp_off,
               int32_t* P, int64_t* pc_off, int32_t* C)
{
    double S = 2097152.0 / L;
    double rcq = r_coll * S;
    orc_lists_ex(ng, groups, level, first_child, nchild, qlo, qhi, theta, rcq * rcq, 0, pp_off, P, pc_off,
                 C);
}

/* Cylindrical frame (phi, r, z grid with scale S = 2^21 / L): two particles
 * within r_coll have |dr|, |dz| <= r_coll and a phi difference of at most
 * ~r_coll / r_min, so (r_coll / r_min + 4e-6) S, squared, bounds their grid
 * distance (4e-6 covers twice the FP32 tree coordinates' error, and r_min's);
 * the phi axis has period floor(2 pi S) cells. */
void orc_cyl_geometry(double r_coll, double r_min, double L, double* rcq2, int64_t* period)
{
    double S = 2097152.0 / L;
    double a = r_coll / r_min;
    a = a + 4e-6;
    a = a * S;
    *rcq2 = a * a;
    *period = (int64_t)floor(6.283185307179586 * S);
}

/* ------------------------------------------------------------------------
 * Eq. (1), read as the acceleration of particle i due to particle j
 * (the paper calls F_ij "the acceleration of particle i"; gravity is
 * therefore G m_j).  r = x_j - x_i, v = v_j - v_i.
 *   r >  r_coll: a = G m_j r / (r^2 + eps^2)^(3/2)
 *   r <= r_coll: a = [G m_j / (r_coll^2 + eps^2)^(3/2)
 *                     + m_j/(m_i+m_j) (kappa (r - r_coll)/r + eta (r.v)/r^2)] r
 * A coincident pair (r = 0) contributes nothing.  "r > r_coll" is evaluated
 * as r2 > r_coll*r_coll with r2 = (dx*dx + dy*dy) + dz*dz.
 * ---------------------------------------------------------------------- */
typedef struct {
    double G, eps2, r_coll, kappa, eta;
} orc_pp_par;

static void orc_pair(const orc_pp_par* p, double xi, double yi, double zi, double vxi,
                     double vyi, double vzi, double mi, double xj, double yj, double zj,
                     double vxj, double vyj, double vzj, double mj, double* a)
{
    double dx = xj - xi, dy = yj - yi, dz = zj - zi;
    double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0.0) return;
    double rc2 = p->r_coll * p->r_coll;
    double f;
    if (r2 > rc2) {
        double s2 = r2 + p->eps2;
        f = p->G * mj / (s2 * sqrt(s2));
    } else {
        double s2 = rc2 + p->eps2;
        double r = sqrt(r2);
        double dvx = vxj - vxi, dvy = vyj - vyi, dvz = vzj - vzi;
        double rv = dx * dvx + dy * dvy + dz * dvz;
        f = p->G * mj / (s2 * sqrt(s2)) +
            (mj / (mi + mj)) * (p->kappa * (r - p->r_coll) / r + p->eta * rv / r2);
    }
    a[0] += f * dx;
    a[1] += f * dy;
    a[2] += f * dz;
}

/* Cell term for an accepted node with mass M, centre c and quadrupole Q:
 * R = x_i - c, R2 = R.R + eps^2,
 *   a = -G M R / R2^(3/2)                                   (monopole)
 *     + G [Q R / R2^(5/2) - 5/2 (R.Q.R) R / R2^(7/2)]       (order 2)
 * from the gradient of Phi = -G M/R - G/2 R.Q.R / R^5. */
static void orc_cell(double G, double eps2, int order, double xi, double yi, double zi,
                     double M, double cx, double cy, double cz, const double* Q, double* a)
{
    double Rx = xi - cx, Ry = yi - cy, Rz = zi - cz;
    double R2 = Rx * Rx + Ry * Ry + Rz * Rz + eps2;
    double R = sqrt(R2);
    double R3 = R2 * R;
    double mono = -G * M / R3;
    a[0] += mono * Rx;
    a[1] += mono * Ry;
    a[2] += mono * Rz;
    if (order >= 2) {
        double QRx = Q[0] * Rx + Q[3] * Ry + Q[4] * Rz;
        double QRy = Q[3] * Rx + Q[1] * Ry + Q[5] * Rz;
        double QRz = Q[4] * Rx + Q[5] * Ry + Q[2] * Rz;
        double RQR = Rx * QRx + Ry * QRy + Rz * QRz;
        double R5 = R3 * R2;
        double R7 = R5 * R2;
        a[0] += G * (QRx / R5 - 2.5 * RQR * Rx / R7);
        a[1] += G * (QRy / R5 - 2.5 * RQR * Ry / R7);
        a[2] += G * (QRz / R5 - 2.5 * RQR * Rz / R7);
    }
}

/* Single pair, exported for closed-form tests. */
void orc_pair_accel(double G, double eps, double r_coll, double kappa, double eta,
                    const double* xi, const double* vi, double mi, const double* xj,
                    const double* vj, double mj, double* a)
{
    orc_pp_par p = {G, eps * eps, r_coll, kappa, eta};
    a[0] = a[1] = a[2] = 0.0;
    orc_pair(&p, xi[0], xi[1], xi[2], vi[0], vi[1], vi[2], mi, xj[0], xj[1], xj[2], vj[0],
             vj[1], vj[2], mj, a);
}

/* Single cell, exported for multipole-convergence tests. */
void orc_cell_accel(double G, double eps, int order, const double* xi, double M,
                    const double* c, const double* Q, double* a)
{
    a[0] = a[1] = a[2] = 0.0;
    orc_cell(G, eps * eps, order, xi[0], xi[1], xi[2], M, c[0], c[1], c[2], Q, a);
}

/* Direct summation: a_i = sum over j != i, ascending j, of Eq. (1). */
void orc_direct(int64_t n, const double* x, const double* y, const double* z,
                const double* vx, const double* vy, const double* vz, const double* m,
                double G, double eps, double r_coll, double kappa, double eta, double* ax,
                double* ay, double* az)
{
    orc_pp_par p = {G, eps * eps, r_coll, kappa, eta};
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        double a[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            orc_pair(&p, x[i], y[i], z[i], vx[i], vy[i], vz[i], m[i], x[j], y[j], z[j], vx[j],
                     vy[j], vz[j], m[j], a);
        }
        ax[i] = a[0];
        ay[i] = a[1];
        az[i] = a[2];
    }
}

/* Tree force (Sec. 4.2 step 3d: double loop over the group's particles and
 * its list): for i in group k, sum Eq. (1) over the particles of the P
 * leaves (in list order, j != i), then the cell term over C (in list order).
 * Only groups [k0, k1) are evaluated; other outputs are left untouched. */
void orc_tree_forces(int64_t k0, int64_t k1, const int32_t* groups, const uint32_t* begin,
                     const uint32_t* end, const int64_t* pp_off, const int32_t* P,
                     const int64_t* pc_off, const int32_t* C, const double* M,
                     const double* cx, const double* cy, const double* cz, const double* Q,
                     int order, const double* x, const double* y, const double* z,
                     const double* vx, const double* vy, const double* vz, const double* m,
                     double G, double eps, double r_coll, double kappa, double eta,
                     double* ax, double* ay, double* az)
{
    orc_pp_par p = {G, eps * eps, r_coll, kappa, eta};
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = k0; k < k1; ++k) {
        int32_t g = groups[k];
        for (uint32_t i = begin[g]; i < end[g]; ++i) {
            double a[3] = {0.0, 0.0, 0.0};
            for (int64_t e = pp_off[k]; e < pp_off[k + 1]; ++e) {
                int32_t leaf = P[e];
                for (uint32_t j = begin[leaf]; j < end[leaf]; ++j) {
                    if (j == i) continue;
                    orc_pair(&p, x[i], y[i], z[i], vx[i], vy[i], vz[i], m[i], x[j], y[j], z[j],
                             vx[j], vy[j], vz[j], m[j], a);
                }
            }
            for (int64_t e = pc_off[k]; e < pc_off[k + 1]; ++e) {
                int32_t c = C[e];
                orc_cell(G, p.eps2, order, x[i], y[i], z[i], M[c], cx[c], cy[c], cz[c],
                         Q + 6 * (int64_t)c, a);
            }
            ax[i] = a[0];
            ay[i] = a[1];
            az[i] = a[2];
        }
    }
}

/* Central mass at the origin (the planet of Table 1): a = -G Mc x / |x|^3. */
void orc_central(int64_t n, const double* x, const double* y, const double* z, double G,
                 double Mc, double* ax, double* ay, double* az)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double r2 = x[i] * x[i] + y[i] * y[i] + z[i] * z[i];
        double f = -G * Mc / (r2 * sqrt(r2));
        ax[i] = f * x[i];
        ay[i] = f * y[i];
        az[i] = f * z[i];
    }
}

/* ---- Self-gravity potential (the energy diagnostic of a ring simulation,
 * Sec. 5.1 times steps with their diagnostics) ------------------------------
 * The potential of the gravity Eq. (1) applies (the contact spring and
 * dashpot are not gravity and have none here):
 *   r > r_coll:   phi_ij = -G m_j / sqrt(r^2 + eps^2)
 *   r <= r_coll:  gravity is held at its r_coll value, a = G m_j r / s^3 with
 *                 s^2 = r_coll^2 + eps^2, whose potential (continuous at r_coll)
 *                 is phi_ij = -G m_j / s - G m_j (r_coll^2 - r^2) / (2 s^3);
 *   coincident (r = 0) pairs contribute nothing, like their force.
 * A list cell (R = x_i - c, R2 = R.R + eps^2) contributes
 *   phi = -G M / sqrt(R2) - G/2 R.Q.R / R2^(5/2)
 * whose negative gradient is the cell term of orc_cell. */
static double orc_pair_pot(double G, double eps2, double r_coll, double xi, double yi, double zi, double xj,
                           double yj, double zj, double mj)
{
    double dx = xj - xi, dy = yj - yi, dz = zj - zi;
    double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0.0) return 0.0;
    double rc2 = r_coll * r_coll;
    if (r2 > rc2) {
        double s2 = r2 + eps2;
        return -G * mj / sqrt(s2);
    }
    double s2 = rc2 + eps2;
    double s = sqrt(s2);
    return -G * mj / s - G * mj * (rc2 - r2) / (2.0 * s2 * s);
}

static double orc_cell_pot(double G, double eps2, int order, double xi, double yi, double zi, double M, double cx,
                           double cy, double cz, const double* Q)
{
    double Rx = xi - cx, Ry = yi - cy, Rz = zi - cz;
    double R2 = Rx * Rx + Ry * Ry + Rz * Rz + eps2;
    double R = sqrt(R2);
    double phi = -G * M / R;
    if (order >= 2) {
        double QRx = Q[0] * Rx + Q[3] * Ry + Q[4] * Rz;
        double QRy = Q[3] * Rx + Q[1] * Ry + Q[5] * Rz;
        double QRz = Q[4] * Rx + Q[5] * Ry + Q[2] * Rz;
        double RQR = Rx * QRx + Ry * QRy + Rz * QRz;
        phi -= 0.5 * G * RQR / (R2 * R2 * R);
    }
    return phi;
}

/* Single pair and single cell, exported for closed-form tests. */
double orc_pair_potential(double G, double eps, double r_coll, const double* xi, const double* xj, double mj)
{
    return orc_pair_pot(G, eps * eps, r_coll, xi[0], xi[1], xi[2], xj[0], xj[1], xj[2], mj);
}

double orc_cell_potential(double G, double eps, int order, const double* xi, double M, const double* c,
                          const double* Q)
{
    return orc_cell_pot(G, eps * eps, order, xi[0], xi[1], xi[2], M, c[0], c[1], c[2], Q);
}

/* Direct summation: phi_i = sum over j != i, ascending j, of phi_ij. */
void orc_direct_potential(int64_t n, const double* x, const double* y, const double* z, const double* m, double G,
                          double eps, double r_coll, double* phi)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            s += orc_pair_pot(G, eps * eps, r_coll, x[i], y[i], z[i], x[j], y[j], z[j], m[j]);
        }
        phi[i] = s;
    }
}

/* Tree potential over the same lists and in the same order as
 * orc_tree_forces: the particles of the P leaves (j != i), then the cells. */
void orc_tree_potential(int64_t k0, int64_t k1, const int32_t* groups, const uint32_t* begin, const uint32_t* end,
                        const int64_t* pp_off, const int32_t* P, const int64_t* pc_off, const int32_t* C,
                        const double* M, const double* cx, const double* cy, const double* cz, const double* Q,
                        int order, const double* x, const double* y, const double* z, const double* m, double G,
                        double eps, double r_coll, double* phi)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = k0; k < k1; ++k) {
        int32_t g = groups[k];
        for (uint32_t i = begin[g]; i < end[g]; ++i) {
            double s = 0.0;
            for (int64_t e = pp_off[k]; e < pp_off[k + 1]; ++e) {
                int32_t leaf = P[e];
                for (uint32_t j = begin[leaf]; j < end[leaf]; ++j) {
                    if (j == i) continue;
                    s += orc_pair_pot(G, eps * eps, r_coll, x[i], y[i], z[i], x[j], y[j], z[j], m[j]);
                }
            }
            for (int64_t e = pc_off[k]; e < pc_off[k + 1]; ++e) {
                int32_t c = C[e];
                s += orc_cell_pot(G, eps * eps, order, x[i], y[i], z[i], M[c], cx[c], cy[c], cz[c],
                                  Q + 6 * (int64_t)c);
            }
            phi[i] = s;
        }
    }
}
