/*
 * wob_oracle.c -- slow, plain, FP64 CPU oracle for the walk-on-boundary (WoB)
 * estimator of Sugimoto, Chen, Jiang, Batty, Hachisuka, "A Practical
 * Walk-on-Boundary Method for Boundary Value Problems" (SIGGRAPH 2023).
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  The product path (the
 * CUDA library) never calls it, shares no code, header or table with it, and
 * must fail loudly when its own extension is missing.
 *
 * Everything here is brute force: every line is tested against every
 * triangle in double precision, no acceleration structure, no blocking.
 * Each function names the passage of the paper it follows.
 *
 * Readings of the paper used here (the paper is silent on these points):
 *  - Ray sampling (Sec. 4.4.1) is done with a LINE through the current point:
 *    the axis is uniform on the sphere, all intersections on both sides are
 *    collected, one of the m hits is picked uniformly.  With omega the unit
 *    direction from x to the hit y, r = |y - x|, the area density of the
 *    pick is |omega . n_y| / (2 pi m r^2).
 *  - "Pick one at random" is realised as: every hit gets a 64-bit key drawn
 *    from the counter-based generator with the hit's triangle id in the
 *    counter; the smallest key wins (ties: lower triangle id).  This is a
 *    uniform pick that does not depend on the order hits are found in.
 *  - The triangle the current boundary point lies on is excluded from its
 *    own line query.  A line with no hit (m = 0) ends the walk; what has
 *    been accumulated stays (the integral sample is zero).
 *  - The last vertex of a walk of M vertices gets half the source term
 *    (phi * g instead of 2 phi g), Sec. 4.1.2, for every estimator.
 *  - A line is "near-degenerate" (flagged) if, for a triangle whose
 *    bounding box padded by tau*L the line meets and whose tau*L-expanded
 *    projection contains the line, the line passes within tau*L of one of
 *    its edges or meets its plane at a grazing angle (|d . n| < graze), or
 *    if a non-self hit lies within |t| < tau*L.  L is the diagonal of the
 *    mesh bounding box.  (The box condition keeps the flag local: the
 *    expanded projection of a triangle seen nearly edge-on reaches far
 *    beyond the triangle along its thin direction.)
 *  - Random numbers: Philox4x32-10 (Salmon et al., SC'11), key =
 *    (seed_lo ^ problem, seed_hi), counter = (query, walk,
 *    step<<16 | purpose<<12 | attempt, extra).  Line axes by Marsaglia's
 *    (1972) method with an exact integer acceptance test.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

/* Test infrastructure: a nonzero ORACLE_PLANT compiles one known mistake
 * into the oracle so that a test can show its pins catch it (1: no half on
 * the last double-layer term; 2: first double-layer weight negated; 3:
 * double-layer recursion sign flipped; 4: hit sign s negated; 5: Robin term
 * of the single layer with the wrong sign; 6: direct-Neumann first line
 * without the 1/2; 7: direct-Neumann last source not halved; 8: forward
 * start weight without the 2 of f = 2 phi q; 9: forward step weight with the
 * wrong sign; 10: forward last vertex not halved; 11: weighted start density
 * not divided by the triangle's area).  0 (the default) is the oracle. */
#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif

enum { PURPOSE_DIR = 0, PURPOSE_HIT = 1, PURPOSE_AREA = 2, PURPOSE_BRANCH = 4, PURPOSE_RIS = 5 };
/* walk index of the forward paths' streams (path p uses query index p) */
#define FORWARD_WALK 0xFFFFFFFFu
enum { KIND_DIRICHLET_DL = 0, KIND_NEUMANN_SL = 1, KIND_ROBIN_SL = 2, KIND_MIXED_SL = 4 };
enum { BC_DIRICHLET = 0, BC_NEUMANN = 1, BC_ROBIN = 2 };
enum { DATA_VERTEX_P1 = 0, DATA_POLY = 1, DATA_POINT = 2 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 and Philox4x64-10, from the definition in Salmon, Moraes,  */
/* Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11).        */
/* One round: two widening multiplies of counter words 0 and 2; the high    */
/* halves are xored with the other two counter words and the round key; the */
/* round key is bumped by the Weyl constants between rounds.                */
/* ------------------------------------------------------------------------ */
static void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B97F4A7C15ull;
            k1 += 0xBB67AE8584CAA73Bull;
        }
        unsigned __int128 p0 = (unsigned __int128)0xD2E7470EE14C6C93ull * c0;
        unsigned __int128 p1 = (unsigned __int128)0xCA5A826395121157ull * c2;
        uint64_t n0 = (uint64_t)(p1 >> 64) ^ c1 ^ k0;
        uint64_t n1 = (uint64_t)p1;
        uint64_t n2 = (uint64_t)(p0 >> 64) ^ c3 ^ k1;
        uint64_t n3 = (uint64_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* One block of four 32-bit words of the stream addressed by
 * (seed, problem; query, walk, step, purpose, attempt, extra). */
static void stream_block(uint64_t seed, uint32_t problem, uint32_t q, uint32_t walk,
                         uint32_t step, uint32_t purpose, uint32_t attempt,
                         uint32_t extra, uint32_t out[4])
{
    uint32_t key[2] = { (uint32_t)seed ^ problem, (uint32_t)(seed >> 32) };
    uint32_t ctr[4] = { q, walk, (step << 16) | (purpose << 12) | attempt, extra };
    philox4x32_10(ctr, key, out);
}

static double u24(uint32_t x) { return ldexp((double)(x >> 8), -24); }

static double u53(uint32_t hi, uint32_t lo)
{
    uint64_t m = ((uint64_t)hi << 21) | (uint64_t)(lo >> 11);
    return ldexp((double)m, -53);
}

/* Line axis uniform on the unit sphere: Marsaglia (1972).  Draw (a, b)
 * uniform in the square until a^2 + b^2 < 1; then
 * (2a sqrt(1-s), 2b sqrt(1-s), 1 - 2s) is uniform on the sphere.  The
 * coordinates are odd multiples of 2^-24, so the acceptance test is an exact
 * integer test.  Returns the number of generator calls used. */
static int line_axis(uint64_t seed, uint32_t problem, uint32_t q, uint32_t walk,
                     uint32_t step, double d[3])
{
    for (uint32_t call = 0; call < 256; ++call) {
        uint32_t x[4];
        stream_block(seed, problem, q, walk, step, PURPOSE_DIR, call, 0, x);
        for (int a = 0; a < 2; ++a) {
            int64_t A = 2 * (int64_t)(x[2 * a] >> 8) - ((int64_t)1 << 24) + 1;
            int64_t B = 2 * (int64_t)(x[2 * a + 1] >> 8) - ((int64_t)1 << 24) + 1;
            int64_t S = A * A + B * B;
            if (S < ((int64_t)1 << 48)) {
                double av = ldexp((double)A, -24);
                double bv = ldexp((double)B, -24);
                double s = ldexp((double)S, -48);
                double root = sqrt(1.0 - s);
                d[0] = 2.0 * av * root;
                d[1] = 2.0 * bv * root;
                d[2] = 1.0 - 2.0 * s;
                return (int)call + 1;
            }
        }
    }
    d[0] = 0.0; d[1] = 0.0; d[2] = 1.0;
    return 256;
}

/* ------------------------------------------------------------------------ */
/* Mesh: plain arrays; derived quantities in double.                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    const float *verts;    /* V x 3 */
    const int32_t *tris;   /* T x 3, counter-clockwise seen from outside */
    int64_t V, T;
    double L;              /* bounding-box diagonal */
    double area;           /* total area |Gamma| */
    double *cdf;           /* inclusive prefix sums of triangle areas (SL only) */
} mesh_t;

static void vtx(const mesh_t *M, int64_t j, int c, double v[3])
{
    int32_t i = M->tris[3 * j + c];
    v[0] = (double)M->verts[3 * (int64_t)i + 0];
    v[1] = (double)M->verts[3 * (int64_t)i + 1];
    v[2] = (double)M->verts[3 * (int64_t)i + 2];
}

static void sub3(const double a[3], const double b[3], double r[3])
{
    r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2];
}
static void cross3(const double a[3], const double b[3], double r[3])
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }

/* N = (v1 - v0) x (v2 - v0): twice the area times the outward unit normal. */
static void tri_normal(const mesh_t *M, int64_t j, double N[3])
{
    double v0[3], v1[3], v2[3], e1[3], e2[3];
    vtx(M, j, 0, v0); vtx(M, j, 1, v1); vtx(M, j, 2, v2);
    sub3(v1, v0, e1); sub3(v2, v0, e2);
    cross3(e1, e2, N);
}

static int mesh_init(mesh_t *M, const float *verts, int64_t V, const int32_t *tris,
                     int64_t T, int want_cdf)
{
    M->verts = verts; M->tris = tris; M->V = V; M->T = T; M->cdf = NULL;
    double lo[3] = { INFINITY, INFINITY, INFINITY }, hi[3] = { -INFINITY, -INFINITY, -INFINITY };
    for (int64_t i = 0; i < V; ++i)
        for (int c = 0; c < 3; ++c) {
            double x = (double)verts[3 * i + c];
            if (x < lo[c]) lo[c] = x;
            if (x > hi[c]) hi[c] = x;
        }
    double diag[3];
    sub3(hi, lo, diag);
    M->L = norm3(diag);
    if (want_cdf) {
        M->cdf = (double *)malloc((size_t)(T > 0 ? T : 1) * sizeof(double));
        if (!M->cdf) return -1;
    }
    double acc = 0.0;
    for (int64_t j = 0; j < T; ++j) {
        double N[3];
        tri_normal(M, j, N);
        acc += 0.5 * norm3(N);
        if (M->cdf) M->cdf[j] = acc;
    }
    M->area = acc;
    return 0;
}

static void mesh_free(mesh_t *M) { free(M->cdf); M->cdf = NULL; }

/* ------------------------------------------------------------------------ */
/* Boundary data.  Three ways to give a function on Gamma:                  */
/*  P1     per-vertex values, interpolated linearly over each triangle;     */
/*  POLY   c0 + c.x + quadratic (x^2, y^2, z^2, xy, yz, zx coefficients);   */
/*  POINT  scale / |y - x0|.                                                 */
/* For the single-layer problems the data is the Neumann flux dh/dn         */
/* (Table 1, Neumann boundary) or the Robin data dh/dn + alpha h (Table 1,  */
/* Robin boundary) of the harmonic field h given by POLY or POINT; in P1    */
/* mode the vertex values are that data directly.                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t mode;
    int32_t pad;
    const float *vertex_data;
    double poly[10];
    double x0[3];
    double scale;
} oracle_data;

static double poly_value(const double c[10], const double y[3])
{
    double x = y[0], yy = y[1], z = y[2];
    return c[0] + c[1] * x + c[2] * yy + c[3] * z + c[4] * x * x + c[5] * yy * yy +
           c[6] * z * z + c[7] * x * yy + c[8] * yy * z + c[9] * z * x;
}

static void poly_grad(const double c[10], const double y[3], double g[3])
{
    double x = y[0], yy = y[1], z = y[2];
    g[0] = c[1] + 2.0 * c[4] * x + c[7] * yy + c[9] * z;
    g[1] = c[2] + 2.0 * c[5] * yy + c[7] * x + c[8] * z;
    g[2] = c[3] + 2.0 * c[6] * z + c[8] * yy + c[9] * x;
}

/* Harmonic field value h(y) and gradient for the analytic modes. */
static void field(const oracle_data *D, const double y[3], double *h, double g[3])
{
    if (D->mode == DATA_POLY) {
        *h = poly_value(D->poly, y);
        poly_grad(D->poly, y, g);
    } else {
        double r[3];
        sub3(y, D->x0, r);
        double rl = norm3(r);
        *h = D->scale / rl;
        double f = -D->scale / (rl * rl * rl);
        g[0] = f * r[0]; g[1] = f * r[1]; g[2] = f * r[2];
    }
}

/* Boundary data at y on triangle j with barycentrics b and unit normal n. */
static double boundary_data(const oracle_data *D, const mesh_t *M, int64_t j,
                            const double y[3], const double b[3], const double n[3],
                            int kind, double alpha)
{
    if (D->mode == DATA_VERTEX_P1) {
        double s = 0.0;
        for (int c = 0; c < 3; ++c)
            s += b[c] * (double)D->vertex_data[M->tris[3 * j + c]];
        return s;
    }
    double h, g[3];
    field(D, y, &h, g);
    if (kind == KIND_DIRICHLET_DL) return h;
    double dhdn = dot3(n, g);
    if (kind == KIND_NEUMANN_SL) return dhdn;
    return dhdn + alpha * h;
}

/* Barycentrics of a point y of the plane of triangle j, from 3D areas. */
static void barycentric(const mesh_t *M, int64_t j, const double y[3], double b[3])
{
    double v0[3], v1[3], v2[3], e1[3], e2[3], p[3], N[3], c[3];
    vtx(M, j, 0, v0); vtx(M, j, 1, v1); vtx(M, j, 2, v2);
    sub3(v1, v0, e1); sub3(v2, v0, e2); sub3(y, v0, p);
    cross3(e1, e2, N);
    double nn = dot3(N, N);
    cross3(p, e2, c);
    b[1] = dot3(c, N) / nn;
    cross3(e1, p, c);
    b[2] = dot3(c, N) / nn;
    b[0] = 1.0 - b[1] - b[2];
}

/* ------------------------------------------------------------------------ */
/* All-hits line query, brute force over every triangle (Sec. 4.4.1).     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t m;       /* number of hits */
    int32_t sum_s;   /* sum over all hits of s = sign(omega . n) */
    int32_t prim;    /* chosen triangle, -1 if m == 0 */
    int32_t s;       /* sign of the chosen hit */
    int32_t flag;    /* near-degenerate line */
    double t;        /* line parameter of the chosen hit */
    double y[3];     /* chosen hit point */
    double b[3];     /* its barycentrics */
} line_result;

/* Does the line {o + t d, t real} meet the bounding box of the triangle v,
 * padded by pad on every side?  Slab test over all t. */
static int line_meets_box(const double o[3], const double d[3], const double v[3][3], double pad)
{
    double tn = -INFINITY, tf = INFINITY;
    for (int c = 0; c < 3; ++c) {
        double lo = v[0][c], hi = v[0][c];
        for (int k = 1; k < 3; ++k) {
            if (v[k][c] < lo) lo = v[k][c];
            if (v[k][c] > hi) hi = v[k][c];
        }
        lo -= pad;
        hi += pad;
        if (d[c] == 0.0) {
            if (o[c] < lo || o[c] > hi) return 0;
            continue;
        }
        double t0 = (lo - o[c]) / d[c], t1 = (hi - o[c]) / d[c];
        if (t0 > t1) { double x = t0; t0 = t1; t1 = x; }
        if (t0 > tn) tn = t0;
        if (t1 < tf) tf = t1;
    }
    return tn <= tf;
}

static void trace_line(const mesh_t *M, const double o[3], const double d[3], int64_t exclude,
                       uint64_t seed, uint32_t problem, uint32_t q, uint32_t walk,
                       uint32_t step, double tauL, double graze, line_result *r)
{
    uint64_t best = UINT64_MAX;
    r->m = 0; r->sum_s = 0; r->prim = -1; r->s = 0; r->flag = 0; r->t = 0.0;
    for (int64_t j = 0; j < M->T; ++j) {
        if (j == exclude) continue;
        double v[3][3], A[3], B[3], C[3], cr[3], e[3], ed[3], l[3], delta[3];
        vtx(M, j, 0, v[0]); vtx(M, j, 1, v[1]); vtx(M, j, 2, v[2]);
        sub3(v[0], o, A); sub3(v[1], o, B); sub3(v[2], o, C);
        /* e[i] = d . ((v_i - o) x (v_{i+1} - o)): signed volume of the line
         * against edge (v_i, v_{i+1}) -- a Pluecker side test. */
        cross3(A, B, cr); e[0] = dot3(d, cr);
        cross3(B, C, cr); e[1] = dot3(d, cr);
        cross3(C, A, cr); e[2] = dot3(d, cr);
        /* Distance from the line to each edge's supporting line. */
        for (int i = 0; i < 3; ++i) {
            sub3(v[(i + 1) % 3], v[i], ed);
            cross3(d, ed, cr);
            l[i] = norm3(cr);
            delta[i] = l[i] > 0.0 ? e[i] / l[i] : 0.0;
        }
        double N[3], e1[3], e2[3];
        sub3(v[1], v[0], e1); sub3(v[2], v[0], e2);
        cross3(e1, e2, N);
        double dn = dot3(d, N);
        double nlen = norm3(N);
        int inside_pos = delta[0] > -tauL && delta[1] > -tauL && delta[2] > -tauL;
        int inside_neg = delta[0] < tauL && delta[1] < tauL && delta[2] < tauL;
        if ((inside_pos || inside_neg) && line_meets_box(o, d, v, tauL)) {
            double mind = fabs(delta[0]);
            if (fabs(delta[1]) < mind) mind = fabs(delta[1]);
            if (fabs(delta[2]) < mind) mind = fabs(delta[2]);
            if (mind < tauL || fabs(dn) < graze * nlen) r->flag = 1;
        }
        int hit = (e[0] > 0.0 && e[1] > 0.0 && e[2] > 0.0) ||
                  (e[0] < 0.0 && e[1] < 0.0 && e[2] < 0.0);
        if (!hit) continue;
        /* plane of the triangle: N . (o + t d - v0) = 0 */
        double t = dot3(N, A) / dn;
        if (fabs(t) < tauL) r->flag = 1;
        int s = ((t > 0.0) == (dn > 0.0)) ? 1 : -1;
#if ORACLE_PLANT == 4
        s = -s;
#endif
        r->m += 1;
        r->sum_s += s;
        uint32_t x[4];
        stream_block(seed, problem, q, walk, step, PURPOSE_HIT, 0, (uint32_t)j, x);
        uint64_t key = ((uint64_t)x[0] << 32) | (uint64_t)x[1];
        if (key < best || (key == best && j < r->prim)) {
            best = key;
            r->prim = (int32_t)j;
            r->s = s;
            r->t = t;
        }
    }
    if (r->m > 0) {
        for (int c = 0; c < 3; ++c) r->y[c] = o[c] + r->t * d[c];
        barycentric(M, r->prim, r->y, r->b);
    }
}

/* ------------------------------------------------------------------------ */
/* Dirichlet problem, double-layer formulation (Sec. 4.1; Table 1, row      */
/* "Dirichlet / source density"):                                           */
/*   nu(x_i)^ = 2 phi dG/dn_y(x_i, x_{i+1}) / p * nu(x_{i+1})^ + 2 phi g(x_i) */
/*   u(x_0)^  = -dG/dn_y(x_0, x_1) / p * nu(x_1)^                           */
/* truncated after M boundary vertices with nu(x_M)^ = phi g(x_M)          */
/* (Sec. 4.1.2).  dG/dn_y = -(r . n_y) / (4 pi r^3), r = y - x (App. A).    */
/* With the line pick density |omega.n_y| / (2 pi m r^2):                   */
/*   first weight  -dG/dn_y / p        = (m/2) s                            */
/*   later weights 2 phi dG/dn_y / p   = -phi m s                           */
/* ------------------------------------------------------------------------ */
/* start_prim >= 0: the walk starts ON the boundary, at x0 on that triangle,
 * and estimates the density nu(x0) (Eq. indirect_double_boundary_reordered2):
 * x0 is vertex 1 (first weight 1), and M - 1 lines follow. */
/* Per-line records of one walk (each pointer may be NULL): hit count (-1:
 * line not traced), picked triangle (-1: none) and near-degenerate flag of
 * line k. */
typedef struct {
    int32_t *m;
    int32_t *prim;
    uint8_t *flag;
} line_rec;

static void put_line(const line_rec *L, int32_t k, int32_t m, int32_t prim, int32_t flag)
{
    if (L->m) L->m[k] = m;
    if (L->prim) L->prim[k] = prim;
    if (L->flag) L->flag[k] = (uint8_t)flag;
}

/* Gradient weight of the first step (Sec. 4.1.3): the first line's weight
 * -dG/dn_y / p = (m/2) s becomes -grad_x dG/dn_y / p, with
 * grad_x dG/dn_y(x, y) = (n - 3 (w . n) w) / (4 pi r^3), w = (y - x) / r
 * (App. A), i.e. (m/2) s times -(n - 3 (w . n) w) / (r (w . n)).  Returns
 * that last factor. */
static void grad_factor(const mesh_t *M, int64_t prim, const double x[3], const double y[3],
                        double out[3])
{
    double N[3], n[3], w[3];
    tri_normal(M, prim, N);
    double nl = norm3(N);
    n[0] = N[0] / nl; n[1] = N[1] / nl; n[2] = N[2] / nl;
    sub3(y, x, w);
    double r = norm3(w);
    w[0] /= r; w[1] /= r; w[2] /= r;
    double wn = dot3(w, n);
    for (int c = 0; c < 3; ++c) out[c] = -(n[c] - 3.0 * wn * w[c]) / (r * wn);
}

static double dl_walk(const mesh_t *M, const oracle_data *D, int32_t phi, const double x0[3],
                      int64_t start_prim, uint32_t q, uint32_t walk, int32_t Mlen,
                      uint64_t seed, uint32_t problem, double tauL, double graze,
                      uint8_t *flag, const line_rec *lines, double *abs_terms, double grad[3])
{
    double gf[3] = { 0.0, 0.0, 0.0 };
    double x[3] = { x0[0], x0[1], x0[2] };
    int64_t exclude = -1;
    double S = 0.0, P = 1.0, W0 = 0.0, A = 0.0;
    int32_t k0 = 0;
    *flag = 0;
    if (start_prim >= 0) {
        double b[3], n[3] = { 0.0, 0.0, 0.0 };
        barycentric(M, start_prim, x, b);
        double g = boundary_data(D, M, start_prim, x, b, n, KIND_DIRICHLET_DL, 0.0);
        double c = (Mlen == 1) ? (double)phi : 2.0 * (double)phi;
        W0 = 1.0;
        S = c * g;
        A = fabs(c * g);
        exclude = start_prim;
        k0 = 1;
        put_line(lines, 0, -1, -1, 0);
    }
    for (int32_t k = k0; k < Mlen; ++k) {
        double d[3];
        line_axis(seed, problem, q, walk, (uint32_t)k, d);
        line_result r;
        trace_line(M, x, d, exclude, seed, problem, q, walk, (uint32_t)k, tauL, graze, &r);
        put_line(lines, k, r.m, r.prim, r.flag);
        if (r.flag) *flag = 1;
        if (r.m == 0) break;
        if (k == 0) {
            W0 = 0.5 * (double)r.m * (double)r.s;
            if (grad) grad_factor(M, r.prim, x, r.y, gf);
        } else {
            P *= -(double)phi * (double)r.m * (double)r.s;
        }
#if ORACLE_PLANT == 2
        if (k == 0) W0 = -W0;
#elif ORACLE_PLANT == 3
        if (k > 0) P = -P;
#endif
        /* line k reaches vertex k + 1 of the walk (density walks: vertex 1 is x0) */
        double n[3] = { 0.0, 0.0, 0.0 };
        double g = boundary_data(D, M, r.prim, r.y, r.b, n, KIND_DIRICHLET_DL, 0.0);
        double c = (k == Mlen - 1) ? (double)phi : 2.0 * (double)phi;
#if ORACLE_PLANT == 1
        c = 2.0 * (double)phi;
#endif
        S += P * c * g;
        A += fabs(P * c * g);
        x[0] = r.y[0]; x[1] = r.y[1]; x[2] = r.y[2];
        exclude = r.prim;
    }
    *abs_terms = fabs(W0) * A;
    if (grad)
        for (int c = 0; c < 3; ++c) grad[c] = gf[c] * W0 * S;
    return W0 * S;
}

/* ------------------------------------------------------------------------ */
/* Neumann / Robin problems, single-layer formulation (Sec. 4.3; Table 1,   */
/* rows "Neumann boundary" and "Robin boundary"):                           */
/*   u(x)   = int G mu dA                                                    */
/*   mu(x)  = -2 phi int (dG/dn_x + alpha G) mu dA + 2 phi f(x)              */
/* with dG/dn_x = (r . n_x) / (4 pi r^3), G = 1 / (4 pi r) (App. A), the    */
/* next point drawn uniformly by area (p = 1/|Gamma|), and the last vertex  */
/* weighted phi f instead of 2 phi f (Sec. 4.1.2).                          */
/* ------------------------------------------------------------------------ */
static void area_sample_at(const mesh_t *M, uint64_t seed, uint32_t problem, uint32_t q,
                           uint32_t walk, uint32_t step, uint32_t attempt, int64_t *tri,
                           double y[3], double b[3])
{
    uint32_t x[4];
    stream_block(seed, problem, q, walk, step, PURPOSE_AREA, attempt, 0, x);
    double target = u53(x[0], x[1]) * M->area;
    /* first triangle whose inclusive prefix area exceeds the target */
    int64_t lo = 0, hi = M->T - 1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (M->cdf[mid] > target) hi = mid; else lo = mid + 1;
    }
    *tri = lo;
    /* uniform point on the triangle: sqrt warp of the first coordinate */
    double su = sqrt(u24(x[2])), u2 = u24(x[3]);
    b[0] = 1.0 - su;
    b[1] = su * (1.0 - u2);
    b[2] = su * u2;
    double v0[3], v1[3], v2[3];
    vtx(M, lo, 0, v0); vtx(M, lo, 1, v1); vtx(M, lo, 2, v2);
    for (int c = 0; c < 3; ++c) y[c] = b[0] * v0[c] + b[1] * v1[c] + b[2] * v2[c];
}

static void area_sample(const mesh_t *M, uint64_t seed, uint32_t problem, uint32_t q,
                        uint32_t walk, uint32_t step, int64_t *tri, double y[3], double b[3])
{
    area_sample_at(M, seed, problem, q, walk, step, 0, tri, y, b);
}

/* Unit normal of triangle j. */
static void unit_normal(const mesh_t *M, int64_t j, double n[3])
{
    double N[3];
    tri_normal(M, j, N);
    double nl = norm3(N);
    n[0] = N[0] / nl; n[1] = N[1] / nl; n[2] = N[2] / nl;
}

/* Transition kernel of the single-layer recursion from x (boundary
 * condition bx, normal nx; bx < 0: the query, off the boundary) to y,
 * without the 1/p of the sampling (Table 1; Sec. 4.3 for Dirichlet parts):
 *   query:    G(x, y)                      (u = int G mu)
 *   Neumann:  -2 phi dG/dn_x(x, y)
 *   Robin:    -2 phi (dG/dn_x(x, y) + alpha G(x, y))
 *   Dirichlet (moving branch): -(k / p_k) G(x, y)
 * dG/dn_x(x, y) = (y - x) . n_x / (4 pi r^3).  Returns 0 for r < rmin. */
static double sl_kernel(int bx, const double x[3], const double nx[3], const double y[3],
                        int32_t phi, double alpha, double kmix, double pk, double rmin)
{
    double r[3];
    sub3(y, x, r);
    double rl = norm3(r);
    if (rl < rmin) return 0.0;
    const double four_pi = 4.0 * ORACLE_PI;
    double G = 1.0 / (four_pi * rl);
    if (bx < 0) return G;
    if (bx == BC_DIRICHLET) return -(kmix / pk) * G;
    double dgdn = dot3(r, nx) / (four_pi * rl * rl * rl);
    if (bx == BC_NEUMANN) return -2.0 * (double)phi * dgdn;
    double w = dgdn + alpha * G;
#if ORACLE_PLANT == 5
    w -= 2.0 * alpha * G;
#endif
    return -2.0 * (double)phi * w;
}

/* Single-layer walks (Table 1, Sec. 4.3): u(x0) = int G mu dA and, at a
 * boundary point x with condition bx, mu(x) = int K(x, y) mu(y) dA + src(x):
 *   Neumann   src = 2 phi q,            Robin src = 2 phi (q + alpha h),
 *   Dirichlet src = k u_D, and mu(x) = mu(x) - k int G mu + k u_D sampled by
 *   a branch: with probability p_k move (kernel -(k/p_k) G), otherwise stay
 *   at x with weight 1 / (1 - p_k) (mixed problems, Sec. 4.3).
 * The source of the last vertex is halved (Sec. 4.1.2).  bc (mixed problems
 * only, else NULL) gives each triangle's condition; kind NEUMANN_SL /
 * ROBIN_SL use that condition everywhere.  Next points: area-uniform
 * (ris <= 1) or resampled importance sampling (Talbot et al. 2005): ris
 * uniform candidates, one picked with probability proportional to |K|, the
 * weight sign(K) (sum of |Gamma| |K| over the candidates) / ris. */
static double sl_walk(const mesh_t *M, const oracle_data *D, int kind, double alpha, int32_t phi,
                      const double x0[3], uint32_t q, uint32_t walk, int32_t Mlen,
                      uint64_t seed, uint32_t problem, double *abs_terms, const uint8_t *bc,
                      double kmix, double pk, int32_t ris)
{
    double x[3] = { x0[0], x0[1], x0[2] };
    double nx[3] = { 0.0, 0.0, 0.0 };
    int bx = -1;
    int64_t jx = -1;
    double S = 0.0, P = 1.0, W0 = 0.0, Aabs = 0.0;
    const double rmin = 1e-12 * M->L;
    const int uniform_bc = kind == KIND_ROBIN_SL ? BC_ROBIN : BC_NEUMANN;
    for (int32_t k = 0; k < Mlen; ++k) {
        int64_t j;
        double y[3], b[3], ny[3];
        double wfac;
        int stay = 0;
        if (bx == BC_DIRICHLET) {
            uint32_t u[4];
            stream_block(seed, problem, q, walk, (uint32_t)k, PURPOSE_BRANCH, 0, 0, u);
            stay = u24(u[0]) >= pk;
        }
        if (stay) {
            j = jx;
            y[0] = x[0]; y[1] = x[1]; y[2] = x[2];
            barycentric(M, j, y, b);
            wfac = 1.0 / (1.0 - pk);
        } else if (ris <= 1) {
            area_sample(M, seed, problem, q, walk, (uint32_t)k, &j, y, b);
            double r[3];
            sub3(y, x, r);
            if (norm3(r) < rmin) break; /* a zero-measure coincidence: empty sample */
            wfac = M->area * sl_kernel(bx, x, nx, y, phi, alpha, kmix, pk, rmin);
        } else {
            double sumw = 0.0, wc[64];
            for (int32_t c = 0; c < ris; ++c) {
                int64_t jc;
                double yc[3], bc3[3];
                area_sample_at(M, seed, problem, q, walk, (uint32_t)k, (uint32_t)c, &jc, yc, bc3);
                wc[c] = fabs(sl_kernel(bx, x, nx, yc, phi, alpha, kmix, pk, rmin));
                sumw += wc[c];
            }
            if (!(sumw > 0.0)) break; /* every candidate has a zero kernel */
            uint32_t u[4];
            stream_block(seed, problem, q, walk, (uint32_t)k, PURPOSE_RIS, 0, 0, u);
            double target = u53(u[0], u[1]) * sumw, acc = 0.0;
            int32_t pick = ris - 1;
            for (int32_t c = 0; c < ris; ++c) {
                acc += wc[c];
                if (acc > target) { pick = c; break; }
            }
            area_sample_at(M, seed, problem, q, walk, (uint32_t)k, (uint32_t)pick, &j, y, b);
            double K = sl_kernel(bx, x, nx, y, phi, alpha, kmix, pk, rmin);
            wfac = (K > 0.0 ? 1.0 : -1.0) * M->area * sumw / (double)ris;
        }
        if (k == 0) W0 = wfac; else P *= wfac;
        unit_normal(M, j, ny);
        int by = bc ? (int)bc[j] : uniform_bc;
        double src;
        if (by == BC_DIRICHLET) {
            src = kmix * boundary_data(D, M, j, y, b, ny, KIND_DIRICHLET_DL, 0.0);
        } else {
            double f = boundary_data(D, M, j, y, b, ny,
                                     by == BC_ROBIN ? KIND_ROBIN_SL : KIND_NEUMANN_SL, alpha);
            src = 2.0 * (double)phi * f;
        }
        if (k == Mlen - 1) src *= 0.5;
        S += P * src;
        Aabs += fabs(P * src);
        x[0] = y[0]; x[1] = y[1]; x[2] = y[2];
        nx[0] = ny[0]; nx[1] = ny[1]; nx[2] = ny[2];
        bx = by;
        jx = j;
    }
    *abs_terms = fabs(W0) * Aabs;
    return W0 * S;
}

/* Neumann problem through the direct boundary integral equation (Sec. 4.2):
 * on the boundary u = -2 phi int dG/dn_y u dA + 2 phi int G q dA, at a point
 * off it u = -phi int dG/dn_y u dA + phi int G q dA (the Green representation
 * with the normal pointing out of Omega; phi = +1 interior, -1 exterior).
 * The dG/dn_y term is sampled with lines as in the double-layer walks: weight
 * -phi dG/dn_y / p = phi (m/2) s from the query, -2 phi dG/dn_y / p = phi m s
 * from a boundary vertex.  The G q term takes one area-uniform point x' per
 * vertex: phi |Gamma| G(x, x') q(x') at the query, twice that on the
 * boundary, and half of it at the last vertex x_M (the truncation rule of
 * Sec. 4.1.2).  q = dh/dn (or the P1 vertex data).  start_prim >= 0: the
 * query lies on that triangle and is boundary vertex 1 (weight 1). */
static double nd_walk(const mesh_t *M, const oracle_data *D, int32_t phi, const double x0[3],
                      int64_t start_prim, uint32_t q, uint32_t walk, int32_t Mlen,
                      uint64_t seed, uint32_t problem, double tauL, double graze,
                      uint8_t *flag, const line_rec *lines, double *abs_terms)
{
    double x[3] = { x0[0], x0[1], x0[2] };
    int64_t exclude = -1;
    double S = 0.0, P = 1.0, A = 0.0;
    const double four_pi = 4.0 * ORACLE_PI;
    int32_t k0 = 0;
    *flag = 0;
    if (start_prim >= 0) {
        exclude = start_prim;
        k0 = 1;
        put_line(lines, 0, -1, -1, 0);
    }
    for (int32_t k = k0; k <= Mlen; ++k) {
        /* source at vertex k */
        int64_t j;
        double y[3], b[3], r[3];
        area_sample(M, seed, problem, q, walk, (uint32_t)k, &j, y, b);
        sub3(y, x, r);
        double rl = norm3(r);
        if (rl >= 1e-12 * M->L) {
            double N[3], n[3];
            tri_normal(M, j, N);
            double nl = norm3(N);
            n[0] = N[0] / nl; n[1] = N[1] / nl; n[2] = N[2] / nl;
            double f = boundary_data(D, M, j, y, b, n, KIND_NEUMANN_SL, 0.0);
            double c = (k == 0) ? (double)phi : 2.0 * (double)phi;
#if ORACLE_PLANT != 7
            if (k == Mlen) c *= 0.5;
#endif
            double term = P * c * M->area * f / (four_pi * rl);
            S += term;
            A += fabs(term);
        }
        if (k == Mlen) break;
        /* line from vertex k to vertex k + 1 */
        double d[3];
        line_axis(seed, problem, q, walk, (uint32_t)k, d);
        line_result lr;
        trace_line(M, x, d, exclude, seed, problem, q, walk, (uint32_t)k, tauL, graze, &lr);
        put_line(lines, k, lr.m, lr.prim, lr.flag);
        if (lr.flag) *flag = 1;
        if (lr.m == 0) break;
        const double ms = (double)lr.m * (double)lr.s;
#if ORACLE_PLANT == 6
        P *= (double)phi * ms;
#else
        P *= (k == 0) ? 0.5 * (double)phi * ms : (double)phi * ms;
#endif
        x[0] = lr.y[0]; x[1] = lr.y[1]; x[2] = lr.y[2];
        exclude = lr.prim;
    }
    *abs_terms = A;
    return S;
}

/* ======================================================================== */
/* Exported entry points (called from Python through ctypes).               */
/* ======================================================================== */
static int set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) return nthreads;
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int oracle_num_threads(int nthreads) { return set_threads(nthreads); }

void oracle_philox4x32_10(const uint32_t *ctr, const uint32_t *key, int64_t n, uint32_t *out)
{
    for (int64_t i = 0; i < n; ++i) philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

void oracle_philox4x64_10(const uint64_t *ctr, const uint64_t *key, int64_t n, uint64_t *out)
{
    for (int64_t i = 0; i < n; ++i) philox4x64_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

/* qws: n x 3 (query, walk, step). */
void oracle_line_axes(uint64_t seed, uint32_t problem, const uint32_t *qws, int64_t n,
                      double *d, int32_t *calls)
{
    for (int64_t i = 0; i < n; ++i) {
        int c = line_axis(seed, problem, qws[3 * i], qws[3 * i + 1], qws[3 * i + 2], d + 3 * i);
        if (calls) calls[i] = c;
    }
}

void oracle_uniforms(uint64_t seed, uint32_t problem, const uint32_t *qws, int64_t n,
                     double *u53_out, double *u24_out /* n x 2 */)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t x[4];
        stream_block(seed, problem, qws[3 * i], qws[3 * i + 1], qws[3 * i + 2], PURPOSE_AREA, 0, 0, x);
        u53_out[i] = u53(x[0], x[1]);
        u24_out[2 * i] = u24(x[2]);
        u24_out[2 * i + 1] = u24(x[3]);
    }
}

/* out: L, total area, signed volume (divergence theorem), min area, max edge */
int oracle_mesh_stats(const float *verts, int64_t V, const int32_t *tris, int64_t T, double *out)
{
    mesh_t M;
    if (mesh_init(&M, verts, V, tris, T, 0)) return -1;
    double vol = 0.0, amin = INFINITY, emax = 0.0;
    for (int64_t j = 0; j < T; ++j) {
        double v0[3], v1[3], v2[3], N[3], c[3];
        vtx(&M, j, 0, v0); vtx(&M, j, 1, v1); vtx(&M, j, 2, v2);
        cross3(v1, v2, c);
        vol += dot3(v0, c) / 6.0;
        tri_normal(&M, j, N);
        double a = 0.5 * norm3(N);
        if (a < amin) amin = a;
        double e[3];
        sub3(v1, v0, e); if (norm3(e) > emax) emax = norm3(e);
        sub3(v2, v1, e); if (norm3(e) > emax) emax = norm3(e);
        sub3(v0, v2, e); if (norm3(e) > emax) emax = norm3(e);
    }
    out[0] = M.L; out[1] = M.area; out[2] = vol; out[3] = amin; out[4] = emax;
    mesh_free(&M);
    return 0;
}

/* n area-uniform boundary points: point i is the area sample of the stream
 * (query i, walk 0, step 0), as drawn at the vertices of the single-layer
 * walks (Sec. 4.3 with uniform area sampling). */
int oracle_area_points(const float *verts, int64_t V, const int32_t *tris, int64_t T, int64_t n,
                       uint64_t seed, uint32_t problem, double *points, int32_t *prims)
{
    mesh_t M;
    if (mesh_init(&M, verts, V, tris, T, 1)) return -1;
    for (int64_t i = 0; i < n; ++i) {
        int64_t j;
        double b[3];
        area_sample(&M, seed, problem, (uint32_t)i, 0u, 0u, &j, points + 3 * i, b);
        prims[i] = (int32_t)j;
    }
    mesh_free(&M);
    return 0;
}

/* Trace n explicit lines (origin o, axis d).  keys: n x 3 (query, walk,
 * step) address the hit-selection keys.  hits_prim / hits_s (n x max_hits,
 * optional) list every hit. */
int oracle_trace_lines(const float *verts, int64_t V, const int32_t *tris, int64_t T,
                       const double *o, const double *d, const int32_t *exclude,
                       const uint32_t *keys, int64_t n, uint64_t seed, uint32_t problem,
                       double tau, double graze, int32_t *m, int32_t *sum_s, int32_t *prim,
                       int32_t *s, double *t, double *y, uint8_t *flag, int nthreads)
{
    mesh_t M;
    if (mesh_init(&M, verts, V, tris, T, 0)) return -1;
    double tauL = tau * M.L;
    int nt = set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
    for (int64_t i = 0; i < n; ++i) {
        line_result r;
        trace_line(&M, o + 3 * i, d + 3 * i, exclude ? exclude[i] : -1, seed, problem,
                   keys[3 * i], keys[3 * i + 1], keys[3 * i + 2], tauL, graze, &r);
        m[i] = r.m;
        if (sum_s) sum_s[i] = r.sum_s;
        if (prim) prim[i] = r.prim;
        if (s) s[i] = r.s;
        if (t) t[i] = r.t;
        if (y) { y[3 * i] = r.y[0]; y[3 * i + 1] = r.y[1]; y[3 * i + 2] = r.y[2]; }
        if (flag) flag[i] = (uint8_t)r.flag;
    }
    mesh_free(&M);
    return 0;
}

/* Double-layer Dirichlet walks: per_walk[q*N + w] for walks
 * walk_begin .. walk_begin+N-1 of queries q_offset .. q_offset+Q-1.
 * walk_flag[q*N + w] = 1 if any line of the walk is near-degenerate;
 * line_m[(q*N + w)*M + k] = hit count of line k (-1: not traced),
 * line_prim[...] its picked triangle (-1: none), line_flag[...] its
 * near-degenerate flag (each of the three may be NULL). */
int oracle_dl_walks(const float *verts, int64_t V, const int32_t *tris, int64_t T,
                    const oracle_data *D, int32_t phi, const float *queries,
                    const int32_t *query_prim, int64_t Q,
                    int64_t q_offset, int64_t walk_begin, int32_t N, int32_t Mlen,
                    uint64_t seed, uint32_t problem, double tau, double graze,
                    double *per_walk, uint8_t *walk_flag, int32_t *line_m, int32_t *line_prim,
                    uint8_t *line_flag, double *abs_terms, double *per_walk_grad, int nthreads)
{
    mesh_t M;
    if (mesh_init(&M, verts, V, tris, T, 0)) return -1;
    double tauL = tau * M.L;
    int nt = set_threads(nthreads);
    int64_t total = Q * (int64_t)N;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
    for (int64_t i = 0; i < total; ++i) {
        int64_t qi = i / N, w = i % N;
        double x0[3] = { queries[3 * qi], queries[3 * qi + 1], queries[3 * qi + 2] };
        line_rec lr = { line_m ? line_m + i * Mlen : NULL, line_prim ? line_prim + i * Mlen : NULL,
                        line_flag ? line_flag + i * Mlen : NULL };
        for (int32_t k = 0; k < Mlen; ++k) put_line(&lr, k, -1, -1, 0);
        uint8_t f;
        double at;
        double g3[3];
        per_walk[i] = dl_walk(&M, D, phi, x0, query_prim ? query_prim[qi] : -1,
                              (uint32_t)(q_offset + qi),
                              (uint32_t)(walk_begin + w), Mlen, seed, problem, tauL, graze, &f, &lr,
                              &at, per_walk_grad ? g3 : NULL);
        if (per_walk_grad)
            for (int c = 0; c < 3; ++c) per_walk_grad[c * total + i] = g3[c];
        if (walk_flag) walk_flag[i] = f;
        if (abs_terms) abs_terms[i] = at;
    }
    mesh_free(&M);
    return 0;
}

/* Single-layer Neumann (kind 1) or Robin (kind 2) walks; query_prim is
 * accepted for symmetry with the library but the first step does not
 * depend on it (area sampling, u = int G mu dA holds on Gamma too). */
/* Direct-BIE Neumann walks (nd_walk), laid out as oracle_dl_walks. */
int oracle_nd_walks(const float *verts, int64_t V, const int32_t *tris, int64_t T,
                    const oracle_data *D, int32_t phi, const float *queries,
                    const int32_t *query_prim, int64_t Q,
                    int64_t q_offset, int64_t walk_begin, int32_t N, int32_t Mlen,
                    uint64_t seed, uint32_t problem, double tau, double graze,
                    double *per_walk, uint8_t *walk_flag, int32_t *line_m, int32_t *line_prim,
                    uint8_t *line_flag, double *abs_terms, int nthreads)
{
    mesh_t M;
    if (mesh_init(&M, verts, V, tris, T, 1)) return -1;
    double tauL = tau * M.L;
    int nt = set_threads(nthreads);
    int64_t total = Q * (int64_t)N;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
    for (int64_t i = 0; i < total; ++i) {
        int64_t qi = i / N, w = i % N;
        double x0[3] = { queries[3 * qi], queries[3 * qi + 1], queries[3 * qi + 2] };
        line_rec lr = { line_m ? line_m + i * Mlen : NULL, line_prim ? line_prim + i * Mlen : NULL,
                        line_flag ? line_flag + i * Mlen : NULL };
        for (int32_t k = 0; k < Mlen; ++k) put_line(&lr, k, -1, -1, 0);
        uint8_t f;
        double at;
        per_walk[i] = nd_walk(&M, D, phi, x0, query_prim ? query_prim[qi] : -1,
                              (uint32_t)(q_offset + qi), (uint32_t)(walk_begin + w), Mlen, seed,
                              problem, tauL, graze, &f, &lr, &at);
        if (walk_flag) walk_flag[i] = f;
        if (abs_terms) abs_terms[i] = at;
    }
    mesh_free(&M);
    return 0;
}

/* Forward (adjoint) single-layer Neumann paths (Sec. 4.4.3; the estimator
 * of Sabelfeld and Simonov that starts on the boundary).  With
 * u(x) = int G(x, y) mu(y) dA and mu = T mu + f, T's kernel
 * K(y, z) = -2 phi dG/dn_x(y, z) and f = 2 phi q, the truncated solution is
 * sum_j c_j <G(x, .), T^j f> (c_j = 1, 1/2 for j = M - 1, Sec. 4.1.2).  A
 * path reads that product from the source end: z_0 ~ p on the boundary,
 * weight a_0 = f(z_0) / p(z_0); from z_j a line (as the double-layer walks)
 * picks z_{j+1}, and K(z_{j+1}, z_j) / p = phi m s (s = sign(w . n at
 * z_{j+1})), so a_{j+1} = a_j phi m s.  Vertex j contributes
 * c_j a_j G(x, z_j) to every evaluation point x (the explicit connection).
 * Start density p: start_mode 0 area-uniform, 1 proportional per triangle to
 * area (|q(centroid)| + beta mean|q|) and uniform on the triangle (the
 * boundary-value-weighted start; beta > 0 keeps it positive everywhere).
 * Outputs per path: vertex positions zpos (M x 3) and weights zw (M, the
 * c_j a_j; 0 after a miss), flag (near-degenerate line). */
static void fwd_path(const mesh_t *M, const oracle_data *D, int32_t phi, const double *wcdf,
                     double wtot, int32_t start_mode, double beta, double qbar, uint32_t path,
                     int32_t Mlen, uint64_t seed, uint32_t problem, double tauL, double graze,
                     double *zpos, double *zw, uint8_t *flag)
{
    for (int32_t j = 0; j < Mlen; ++j) {
        zpos[3 * j] = zpos[3 * j + 1] = zpos[3 * j + 2] = 0.0;
        zw[j] = 0.0;
    }
    *flag = 0;
    /* start point */
    uint32_t u[4];
    stream_block(seed, problem, path, FORWARD_WALK, 0, PURPOSE_AREA, 0, 0, u);
    const double *cdf = start_mode == 1 ? wcdf : M->cdf;
    double tot = start_mode == 1 ? wtot : M->area;
    double target = u53(u[0], u[1]) * tot;
    int64_t lo = 0, hi = M->T - 1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (cdf[mid] > target) hi = mid; else lo = mid + 1;
    }
    double su = sqrt(u24(u[2])), u2 = u24(u[3]);
    double b[3] = { 1.0 - su, su * (1.0 - u2), su * u2 };
    double v0[3], v1[3], v2[3], z[3], n[3];
    vtx(M, lo, 0, v0); vtx(M, lo, 1, v1); vtx(M, lo, 2, v2);
    for (int c = 0; c < 3; ++c) z[c] = b[0] * v0[c] + b[1] * v1[c] + b[2] * v2[c];
    unit_normal(M, lo, n);
    double pdf;
    if (start_mode == 1) {
        double N[3];
        tri_normal(M, lo, N);
        double A = 0.5 * norm3(N);
        double w = cdf[lo] - (lo > 0 ? cdf[lo - 1] : 0.0);
#if ORACLE_PLANT == 11
        pdf = w / tot;
#else
        pdf = (w / A) / tot;
#endif
    } else {
        pdf = 1.0 / M->area;
    }
#if ORACLE_PLANT == 8
    double a = (double)phi * boundary_data(D, M, lo, z, b, n, KIND_NEUMANN_SL, 0.0) / pdf;
#else
    double a = 2.0 * (double)phi * boundary_data(D, M, lo, z, b, n, KIND_NEUMANN_SL, 0.0) / pdf;
#endif
    int64_t prim = lo;
    for (int32_t j = 0; j < Mlen; ++j) {
#if ORACLE_PLANT == 10
        double c = 1.0;
#else
        double c = (j == Mlen - 1) ? 0.5 : 1.0;
#endif
        zpos[3 * j] = z[0]; zpos[3 * j + 1] = z[1]; zpos[3 * j + 2] = z[2];
        zw[j] = c * a;
        if (j == Mlen - 1) break;
        double d[3];
        line_axis(seed, problem, path, FORWARD_WALK, (uint32_t)j, d);
        line_result r;
        trace_line(M, z, d, prim, seed, problem, path, FORWARD_WALK, (uint32_t)j, tauL, graze, &r);
        if (r.flag) *flag = 1;
        if (r.m == 0) break;
#if ORACLE_PLANT == 9
        a *= -(double)phi * (double)r.m * (double)r.s;
#else
        a *= (double)phi * (double)r.m * (double)r.s;
#endif
        z[0] = r.y[0]; z[1] = r.y[1]; z[2] = r.y[2];
        prim = r.prim;
    }
}

/* N forward paths (fwd_path); zpos: N x M x 3, zw: N x M, flag: N. */
int oracle_fwd_paths(const float *verts, int64_t V, const int32_t *tris, int64_t T,
                     const oracle_data *D, int32_t phi, int64_t N, int32_t Mlen, uint64_t seed,
                     uint32_t problem, int32_t start_mode, double beta, double tau, double graze,
                     double *zpos, double *zw, uint8_t *flag, int nthreads)
{
    mesh_t M;
    if (mesh_init(&M, verts, V, tris, T, 1)) return -1;
    double *wcdf = (double *)malloc((size_t)T * sizeof(double));
    if (!wcdf) { mesh_free(&M); return -1; }
    /* boundary-value-weighted start: per-triangle weight area (|q(c)| + beta qbar) */
    double qsum = 0.0;
    for (int64_t j = 0; j < T; ++j) {
        double v0[3], v1[3], v2[3], c[3], n[3], N3[3];
        double b[3] = { 1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0 };
        vtx(&M, j, 0, v0); vtx(&M, j, 1, v1); vtx(&M, j, 2, v2);
        for (int k = 0; k < 3; ++k) c[k] = (v0[k] + v1[k] + v2[k]) / 3.0;
        unit_normal(&M, j, n);
        tri_normal(&M, j, N3);
        double A = 0.5 * norm3(N3);
        wcdf[j] = A * fabs(boundary_data(D, &M, j, c, b, n, KIND_NEUMANN_SL, 0.0));
        qsum += wcdf[j];
    }
    double qbar = qsum / M.area, acc = 0.0;
    for (int64_t j = 0; j < T; ++j) {
        double N3[3];
        tri_normal(&M, j, N3);
        double A = 0.5 * norm3(N3);
        acc += wcdf[j] + beta * qbar * A;
        wcdf[j] = acc;
    }
    double tauL = tau * M.L;
    int nt = set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
    for (int64_t p = 0; p < N; ++p)
        fwd_path(&M, D, phi, wcdf, acc, start_mode, beta, qbar, (uint32_t)p, Mlen, seed, problem,
                 tauL, graze, zpos + p * Mlen * 3, zw + p * Mlen, flag + p);
    free(wcdf);
    mesh_free(&M);
    return 0;
}

/* Explicit connection of N forward paths to Q points: per_path[q][p] =
 * sum_j zw[p][j] G(x_q, z_pj), G = 1 / (4 pi r); est = mean over paths. */
void oracle_fwd_connect(const float *queries, int64_t Q, const double *zpos, const double *zw,
                        int64_t N, int32_t Mlen, double *per_path, int nthreads)
{
    int nt = set_threads(nthreads);
    const double four_pi = 4.0 * ORACLE_PI;
#pragma omp parallel for schedule(static) num_threads(nt)
    for (int64_t q = 0; q < Q; ++q) {
        double x[3] = { queries[3 * q], queries[3 * q + 1], queries[3 * q + 2] };
        for (int64_t p = 0; p < N; ++p) {
            double v = 0.0;
            for (int32_t j = 0; j < Mlen; ++j) {
                double w = zw[p * Mlen + j];
                if (w == 0.0) continue;
                const double *z = zpos + (p * Mlen + j) * 3;
                double r[3] = { z[0] - x[0], z[1] - x[1], z[2] - x[2] };
                v += w / (four_pi * norm3(r));
            }
            per_path[q * N + p] = v;
        }
    }
}

int oracle_sl_walks(const float *verts, int64_t V, const int32_t *tris, int64_t T,
                    const oracle_data *D, int32_t kind, double alpha, int32_t phi,
                    const float *queries, int64_t Q, int64_t q_offset, int64_t walk_begin,
                    int32_t N, int32_t Mlen, uint64_t seed, uint32_t problem,
                    double *per_walk, double *abs_terms, const uint8_t *bc, double kmix,
                    double pk, int32_t ris, int nthreads)
{
    if (ris > 64 || (kind == KIND_MIXED_SL && (!bc || !(kmix > 0.0) || !(pk > 0.0 && pk < 1.0))))
        return -1;
    mesh_t M;
    if (mesh_init(&M, verts, V, tris, T, 1)) return -1;
    int nt = set_threads(nthreads);
    int64_t total = Q * (int64_t)N;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
    for (int64_t i = 0; i < total; ++i) {
        int64_t qi = i / N, w = i % N;
        double x0[3] = { queries[3 * qi], queries[3 * qi + 1], queries[3 * qi + 2] };
        double at;
        per_walk[i] = sl_walk(&M, D, kind, alpha, phi, x0, (uint32_t)(q_offset + qi),
                              (uint32_t)(walk_begin + w), Mlen, seed, problem, &at,
                              kind == KIND_MIXED_SL ? bc : NULL, kmix, pk, ris);
        if (abs_terms) abs_terms[i] = at;
    }
    mesh_free(&M);
    return 0;
}

/* Per-query reduction (Sec. 4.1.1: the estimate is the mean of the N
 * samples): est = mean, var = unbiased sample variance of one walk. */
void oracle_reduce(const double *per_walk, int64_t Q, int32_t N, double *est, double *var)
{
    for (int64_t q = 0; q < Q; ++q) {
        const double *v = per_walk + q * (int64_t)N;
        double s = 0.0;
        for (int32_t w = 0; w < N; ++w) s += v[w];
        double mean = s / (double)N;
        double ss = 0.0;
        for (int32_t w = 0; w < N; ++w) ss += (v[w] - mean) * (v[w] - mean);
        est[q] = mean;
        var[q] = N > 1 ? ss / (double)(N - 1) : 0.0;
    }
}
