/*
 * rcb_oracle.c -- plain, slow, FP64 CPU oracle of the recursive coordinate bisection (RCB)
 * tree of Gafton & Rosswog (2011), "A fast recursive coordinate bisection tree for neighbour
 * search and gravity".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load this file.  The CUDA library never links or calls it and shares no
 * code, header, table or constant with it.
 *
 * Every step follows the paper in its own order and notation:
 *   Sec. 2.1.1  depth rule: split until the mean ll-cell occupancy drops below N_ll
 *   Sec. 2.1.3  split the longest side through the centre of mass (CMS); variant: through the
 *               median position (MPS)
 *   Sec. 2.1.4  quick-sort-like in-place partition of each cell's index range
 *   Sec. 2.1.5  heap labels: root 1, children 2n and 2n+1, level k spans 2^k .. 2^(k+1)-1
 *   Sec. 2.1.6  Eq. 1 (ll-cell quadrupoles) and Eq. 2 (shift-up to parents)
 *   Sec. 2.2    depth-first walk starting at node 2; Sec. 2.3.1 reachability test;
 *   Sec. 2.4.1  geometric MAC (Eq. 4) overruled by reachability
 *   Sec. 2.4.2  Eq. 5 far-field potential and the cell-cell Taylor expansion (Eq. 6)
 *   Sec. 2.4.3  Eq. 9-10 kernel-softened near field
 * Points on which the paper is silent are resolved as follows (one reading each):
 *   - centre of mass: exact integer sums of 62-bit fixed-point values of RN(m*x) and m,
 *     one binary scale per axis over the whole input, then one FP64 division;
 *   - cell size and geometric centre: the tight bounding box of the cell's particles;
 *     r_g = 0.5 * RN(min + max); ties in the longest side go to the lowest axis;
 *   - particles with x_axis < split go to the left (2n) child, all others to the right;
 *   - h_node_int(leaf) = max |r_b - r_g|; h_node_int(parent) = max over non-empty
 *     children C of (|r_gP - r_gC| + h_node_int(C)); h_node(ll-cell) = max(|r_a - r_g| + 2 h_a);
 *   - a reachable internal node is opened; a reachable ll-cell joins the near list and
 *     the neighbour-candidate list;
 *   - all walk and neighbour comparisons are made in squared form, in FP64 rounded after
 *     every operation (this file must be compiled with -ffp-contract=off);
 *   - neighbours of a are the b != a with |r_a - r_b| < 2 h_a (gather, self excluded),
 *     each row sorted by original index;
 *   - near-field potential: the integral of S with phi = -1/r beyond q = 2;
 *   - the far field keeps monopole and quadrupole and the sink expansion is the exact
 *     third-order Taylor polynomial of that truncated potential, whose negative gradient
 *     is the paper's f + J dr + 1/2 dr^T H dr.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_ALLOC = -2, ORC_ERR_CAPACITY = -3, ORC_ERR_STATE = -4 };
enum { ORC_SPLIT_CMS = 0, ORC_SPLIT_MPS = 1 };

/* ------------------------------------------------------------------------------------------ */
/* Tree storage.  Node labels follow Sec. 2.1.5: nodes 1 .. 2^(L+1)-1; arrays are sized 2^(L+1)
 * and entry 0 is unused.  Particles are held in the order the partition leaves them. */
typedef struct {
    int64_t N;
    int L;
    int64_t nn;      /* 2^(L+1) */
    int32_t n_ll;
    int32_t *perm;   /* sorted position -> original index */
    double *x[3], *m, *h;
    int64_t *P[3], *Pm; /* per-particle fixed-point values (see fixed_point) */
    int E[3], Em;
    int64_t *first, *count;
    int32_t *axis;
    double *split;
    i128 *S[3], *Msum;
    double *mass, *com[3], *bmin[3], *bmax[3], *rg[3], *H, *hint, *hnode, *Q[6];
    /* for comparing readings of Eq. 4 only: the longest side of each cell's bisection box, and
     * whether the walk reads it in place of H (see orc_walk_bisection_box) */
    double *Hbis;
    int mac_box;
    /* interaction lists, indexed by leaf number j = node - 2^L */
    int walked;
    double theta;
    uint8_t *walked_leaf;
    int64_t *near_n, *far_n;
    int32_t **near_ids;
    uint8_t **near_reach;
    int32_t **far_ids;
} orc_tree;

static void *xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }

int orc_depth(int64_t N, int32_t n_ll) {
    /* Sec. 2.1.1 / Table 1: L is the smallest level index (L >= 1) whose 2^L cells hold on
     * average fewer than N_ll particles: N / 2^L < N_ll  <=>  N < N_ll * 2^L. */
    if (N < 0 || n_ll < 1) return -1;
    int L = 1;
    while (!((double)N < (double)n_ll * ldexp(1.0, L))) ++L;
    return L;
}

/* ------------------------------------------------------------------------------------------ */
/* Exact centre of mass.  p = RN(m * x) per axis; E = binary exponent with max|p| < 2^E; each
 * p becomes the integer RN(p * 2^(62 - E)) (so |P| < 2^62); a cell's sum of those integers is
 * exact in 128 bits.  Masses are scaled the same way with their own exponent Em. */
static int frexp_exponent(double a) {
    int e = 0;
    if (a == 0.0) return 0;
    (void)frexp(a, &e);
    return e;
}

static int64_t to_fixed(double v, int E) {
    double s = ldexp(v, 62 - E); /* exact: a power-of-two scaling */
    return (int64_t)llrint(s);   /* round half to even (default rounding mode) */
}

static double com_of(i128 S, int E, i128 M, int Em) {
    double num = ldexp((double)S, E - 62);
    double den = ldexp((double)M, Em - 62);
    return num / den;
}

static double mass_of(i128 M, int Em) { return ldexp((double)M, Em - 62); }

/* |v| with FP64 rounding after each operation. */
static double norm3(double dx, double dy, double dz) {
    double s = dx * dx;
    s = s + dy * dy;
    s = s + dz * dz;
    return sqrt(s);
}

static double dist2(double ax, double ay, double az, double bx, double by, double bz) {
    double dx = ax - bx, dy = ay - by, dz = az - bz;
    double s = dx * dx;
    s = s + dy * dy;
    s = s + dz * dz;
    return s;
}

/* Tight bounding box, sums and the derived node quantities of one node from its particles. */
static void node_from_particles(orc_tree *t, int64_t n) {
    int64_t f = t->first[n], c = t->count[n];
    for (int d = 0; d < 3; ++d) { t->S[d][n] = 0; t->bmin[d][n] = INFINITY; t->bmax[d][n] = -INFINITY; }
    t->Msum[n] = 0;
    for (int64_t i = f; i < f + c; ++i) {
        for (int d = 0; d < 3; ++d) {
            t->S[d][n] += (i128)t->P[d][i];
            if (t->x[d][i] < t->bmin[d][n]) t->bmin[d][n] = t->x[d][i];
            if (t->x[d][i] > t->bmax[d][n]) t->bmax[d][n] = t->x[d][i];
        }
        t->Msum[n] += (i128)t->Pm[i];
    }
    if (c == 0) {
        t->mass[n] = 0.0;
        for (int d = 0; d < 3; ++d) { t->com[d][n] = 0.0; t->bmin[d][n] = 0.0; t->bmax[d][n] = 0.0; t->rg[d][n] = 0.0; }
        t->H[n] = 0.0;
        return;
    }
    t->mass[n] = mass_of(t->Msum[n], t->Em);
    double H = 0.0;
    for (int d = 0; d < 3; ++d) {
        t->com[d][n] = com_of(t->S[d][n], t->E[d], t->Msum[n], t->Em);
        t->rg[d][n] = 0.5 * (t->bmin[d][n] + t->bmax[d][n]);
        double ext = t->bmax[d][n] - t->bmin[d][n];
        if (ext > H) H = ext;
    }
    t->H[n] = H; /* Eq. 4: H_B = MAX(S_i,B) */
}

static void swap_particles(orc_tree *t, int64_t i, int64_t j) {
    for (int d = 0; d < 3; ++d) {
        double tx = t->x[d][i]; t->x[d][i] = t->x[d][j]; t->x[d][j] = tx;
        int64_t tp = t->P[d][i]; t->P[d][i] = t->P[d][j]; t->P[d][j] = tp;
    }
    double tm = t->m[i]; t->m[i] = t->m[j]; t->m[j] = tm;
    double th = t->h[i]; t->h[i] = t->h[j]; t->h[j] = th;
    int64_t tq = t->Pm[i]; t->Pm[i] = t->Pm[j]; t->Pm[j] = tq;
    int32_t tr = t->perm[i]; t->perm[i] = t->perm[j]; t->perm[j] = tr;
}

/* Eq. 1: Q_ij = sum_a [3 m_a dx_i dx_j - m_a dr^2 delta_ij], dx about the cell centre of mass. */
static void leaf_quadrupole(orc_tree *t, int64_t n) {
    double Q[3][3] = {{0}};
    for (int64_t a = t->first[n]; a < t->first[n] + t->count[n]; ++a) {
        double dx[3];
        for (int d = 0; d < 3; ++d) dx[d] = t->x[d][a] - t->com[d][n];
        double dr2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                Q[i][j] += 3.0 * t->m[a] * dx[i] * dx[j] - (i == j ? t->m[a] * dr2 : 0.0);
    }
    t->Q[0][n] = Q[0][0]; t->Q[1][n] = Q[0][1]; t->Q[2][n] = Q[0][2];
    t->Q[3][n] = Q[1][1]; t->Q[4][n] = Q[1][2]; t->Q[5][n] = Q[2][2];
}

/* Sec. 2.3.1 radii of an ll-cell about its geometric centre. */
static void leaf_radii(orc_tree *t, int64_t n) {
    double hint = 0.0, hnode = 0.0;
    for (int64_t a = t->first[n]; a < t->first[n] + t->count[n]; ++a) {
        double d = norm3(t->x[0][a] - t->rg[0][n], t->x[1][a] - t->rg[1][n], t->x[2][a] - t->rg[2][n]);
        if (d > hint) hint = d;
        double reach = d + 2.0 * t->h[a];
        if (reach > hnode) hnode = reach;
    }
    t->hint[n] = hint;
    t->hnode[n] = hnode;
}

/* Eq. 2 shift-up of the quadrupole and the enclosing radius of a parent from its children. */
static void parent_from_children(orc_tree *t, int64_t P) {
    double Q[3][3] = {{0}};
    double hint = 0.0;
    for (int64_t C = 2 * P; C <= 2 * P + 1; ++C) {
        if (t->count[C] == 0) continue;
        double dx[3];
        for (int d = 0; d < 3; ++d) dx[d] = t->com[d][C] - t->com[d][P];
        double dr2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
        double QC[3][3] = {{t->Q[0][C], t->Q[1][C], t->Q[2][C]},
                           {t->Q[1][C], t->Q[3][C], t->Q[4][C]},
                           {t->Q[2][C], t->Q[4][C], t->Q[5][C]}};
        double MC = t->mass[C];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                Q[i][j] += QC[i][j] + 3.0 * MC * dx[i] * dx[j] - (i == j ? MC * dr2 : 0.0);
        double r = norm3(t->rg[0][P] - t->rg[0][C], t->rg[1][P] - t->rg[1][C], t->rg[2][P] - t->rg[2][C]) + t->hint[C];
        if (r > hint) hint = r;
    }
    t->Q[0][P] = Q[0][0]; t->Q[1][P] = Q[0][1]; t->Q[2][P] = Q[0][2];
    t->Q[3][P] = Q[1][1]; t->Q[4][P] = Q[1][2]; t->Q[5][P] = Q[2][2];
    t->hint[P] = hint;
    t->hnode[P] = 0.0;
}

static void moments(orc_tree *t) {
    const int64_t leaf0 = (int64_t)1 << t->L;
    for (int64_t n = leaf0; n < 2 * leaf0; ++n) {
        if (t->count[n] == 0) {
            for (int k = 0; k < 6; ++k) t->Q[k][n] = 0.0;
            t->hint[n] = 0.0; t->hnode[n] = 0.0;
            continue;
        }
        leaf_quadrupole(t, n);
        leaf_radii(t, n);
    }
    for (int k = t->L - 1; k >= 0; --k)
        for (int64_t P = (int64_t)1 << k; P < ((int64_t)2 << k); ++P) {
            if (t->count[P] == 0) {
                for (int q = 0; q < 6; ++q) t->Q[q][P] = 0.0;
                t->hint[P] = 0.0; t->hnode[P] = 0.0;
                continue;
            }
            parent_from_children(t, P);
        }
}

void orc_free(orc_tree *t);

static int alloc_tree(orc_tree *t) {
    int64_t N = t->N, nn = t->nn;
    t->perm = xcalloc(N, sizeof(int32_t));
    t->m = xcalloc(N, sizeof(double));
    t->h = xcalloc(N, sizeof(double));
    t->Pm = xcalloc(N, sizeof(int64_t));
    t->first = xcalloc(nn, sizeof(int64_t));
    t->count = xcalloc(nn, sizeof(int64_t));
    t->axis = xcalloc(nn, sizeof(int32_t));
    t->split = xcalloc(nn, sizeof(double));
    t->Msum = xcalloc(nn, sizeof(i128));
    t->mass = xcalloc(nn, sizeof(double));
    t->H = xcalloc(nn, sizeof(double));
    t->hint = xcalloc(nn, sizeof(double));
    t->hnode = xcalloc(nn, sizeof(double));
    int ok = t->perm && t->m && t->h && t->Pm && t->first && t->count && t->axis && t->split &&
             t->Msum && t->mass && t->H && t->hint && t->hnode;
    for (int d = 0; d < 3; ++d) {
        t->x[d] = xcalloc(N, sizeof(double));
        t->P[d] = xcalloc(N, sizeof(int64_t));
        t->S[d] = xcalloc(nn, sizeof(i128));
        t->com[d] = xcalloc(nn, sizeof(double));
        t->bmin[d] = xcalloc(nn, sizeof(double));
        t->bmax[d] = xcalloc(nn, sizeof(double));
        t->rg[d] = xcalloc(nn, sizeof(double));
        ok = ok && t->x[d] && t->P[d] && t->S[d] && t->com[d] && t->bmin[d] && t->bmax[d] && t->rg[d];
    }
    for (int k = 0; k < 6; ++k) { t->Q[k] = xcalloc(nn, sizeof(double)); ok = ok && t->Q[k]; }
    return ok ? ORC_OK : ORC_ERR_ALLOC;
}

/* Fixed-point scales and per-particle integers from the particles' current values. */
static int fixed_point(orc_tree *t) {
    double A[3] = {0, 0, 0}, Am = 0.0;
    for (int64_t i = 0; i < t->N; ++i) {
        for (int d = 0; d < 3; ++d) {
            double p = fabs(t->m[i] * t->x[d][i]);
            if (p > A[d]) A[d] = p;
        }
        if (t->m[i] > Am) Am = t->m[i];
    }
    for (int d = 0; d < 3; ++d) t->E[d] = frexp_exponent(A[d]);
    t->Em = frexp_exponent(Am);
    for (int64_t i = 0; i < t->N; ++i) {
        for (int d = 0; d < 3; ++d) t->P[d][i] = to_fixed(t->m[i] * t->x[d][i], t->E[d]);
        t->Pm[i] = to_fixed(t->m[i], t->Em);
        if (t->Pm[i] < 1) return ORC_ERR_ARG; /* mass ratio beyond the fixed-point range */
    }
    return ORC_OK;
}

static int cmp_double(const void *a, const void *b) {
    double u = *(const double *)a, v = *(const double *)b;
    return (u > v) - (u < v);
}

/* Sec. 2.1.3, the median position split (MPS): the coordinate of rank floor(cnt/2), counted from
 * 0 in ascending order, of the cell's particles along the axis.  With distinct coordinates the
 * cut x < s leaves floor(cnt/2) particles on the left and the rest on the right; particles tied
 * with the median coordinate all go right. */
static double median_position(const orc_tree *t, int64_t f, int64_t cnt, int ax) {
    double *v = malloc(sizeof(double) * (size_t)cnt);
    if (!v) return NAN;
    for (int64_t i = 0; i < cnt; ++i) v[i] = t->x[ax][f + i];
    qsort(v, (size_t)cnt, sizeof(double), cmp_double);
    double s = v[cnt / 2];
    free(v);
    return s;
}

orc_tree *orc_build_split(const double *x, const double *m, const double *h, int64_t N, int32_t n_ll,
                          int split_mode, int *status);

orc_tree *orc_build(const double *x, const double *m, const double *h, int64_t N, int32_t n_ll, int *status) {
    return orc_build_split(x, m, h, N, n_ll, ORC_SPLIT_CMS, status);
}

orc_tree *orc_build_split(const double *x, const double *m, const double *h, int64_t N, int32_t n_ll,
                          int split_mode, int *status) {
    *status = ORC_ERR_ARG;
    if (N < 1 || N >= ((int64_t)1 << 31) || n_ll < 1) return NULL;
    if (split_mode != ORC_SPLIT_CMS && split_mode != ORC_SPLIT_MPS) return NULL;
    for (int64_t i = 0; i < N; ++i) {
        if (!isfinite(x[3 * i]) || !isfinite(x[3 * i + 1]) || !isfinite(x[3 * i + 2])) return NULL;
        if (!isfinite(m[i]) || !(m[i] > 0.0) || !isfinite(h[i]) || !(h[i] > 0.0)) return NULL;
    }
    int L = orc_depth(N, n_ll);
    if (L < 1 || L > 28) return NULL;
    orc_tree *t = xcalloc(1, sizeof(orc_tree));
    if (!t) { *status = ORC_ERR_ALLOC; return NULL; }
    t->N = N; t->L = L; t->nn = (int64_t)2 << L; t->n_ll = n_ll;
    if (alloc_tree(t) != ORC_OK) { orc_free(t); *status = ORC_ERR_ALLOC; return NULL; }
    for (int64_t i = 0; i < N; ++i) {
        t->perm[i] = (int32_t)i;
        for (int d = 0; d < 3; ++d) t->x[d][i] = x[3 * i + d] + 0.0; /* +0.0 turns -0 into +0 */
        t->m[i] = m[i];
        t->h[i] = h[i];
    }
    if (fixed_point(t) != ORC_OK) { orc_free(t); *status = ORC_ERR_ARG; return NULL; }

    /* Sec. 2.1: the root holds all particles; level by level, every cell is split. */
    t->first[1] = 0;
    t->count[1] = N;
    node_from_particles(t, 1);
    for (int k = 0; k < L; ++k) {
        for (int64_t c = (int64_t)1 << k; c < ((int64_t)2 << k); ++c) {
            int64_t f = t->first[c], cnt = t->count[c];
            int ax = 0;
            double s = 0.0;
            int64_t nleft = 0;
            if (cnt > 0) {
                /* Sec. 2.1.3: the longest side (ties -> lowest axis), cut through the CMS, or
                 * through the median position for the MPS variant. */
                double best = -1.0;
                for (int d = 0; d < 3; ++d) {
                    double ext = t->bmax[d][c] - t->bmin[d][c];
                    if (ext > best) { best = ext; ax = d; }
                }
                if (split_mode == ORC_SPLIT_MPS) {
                    s = median_position(t, f, cnt, ax);
                    if (isnan(s)) { orc_free(t); *status = ORC_ERR_ALLOC; return NULL; }
                } else {
                    s = t->com[ax][c];
                }
                /* Sec. 2.1.4: one pass; smaller coordinates to the front, the rest to the back. */
                int64_t i = f, j = f + cnt - 1;
                while (i <= j) {
                    if (t->x[ax][i] < s) ++i;
                    else { swap_particles(t, i, j); --j; }
                }
                nleft = i - f;
            }
            t->axis[c] = ax;
            t->split[c] = s;
            t->first[2 * c] = f;
            t->count[2 * c] = nleft;
            t->first[2 * c + 1] = f + nleft;
            t->count[2 * c + 1] = cnt - nleft;
            node_from_particles(t, 2 * c);
            node_from_particles(t, 2 * c + 1);
        }
    }
    moments(t);
    *status = ORC_OK;
    return t;
}

static void free_lists(orc_tree *t) {
    int64_t nl = (int64_t)1 << t->L;
    if (t->near_ids) for (int64_t j = 0; j < nl; ++j) free(t->near_ids[j]);
    if (t->near_reach) for (int64_t j = 0; j < nl; ++j) free(t->near_reach[j]);
    if (t->far_ids) for (int64_t j = 0; j < nl; ++j) free(t->far_ids[j]);
    free(t->near_ids); free(t->near_reach); free(t->far_ids);
    free(t->near_n); free(t->far_n); free(t->walked_leaf);
    t->near_ids = NULL; t->near_reach = NULL; t->far_ids = NULL;
    t->near_n = NULL; t->far_n = NULL; t->walked_leaf = NULL;
    t->walked = 0;
}

void orc_free(orc_tree *t) {
    if (!t) return;
    if (t->L > 0) free_lists(t);
    free(t->perm); free(t->m); free(t->h); free(t->Pm);
    free(t->first); free(t->count); free(t->axis); free(t->split); free(t->Msum);
    free(t->mass); free(t->H); free(t->hint); free(t->hnode); free(t->Hbis);
    for (int d = 0; d < 3; ++d) {
        free(t->x[d]); free(t->P[d]); free(t->S[d]); free(t->com[d]);
        free(t->bmin[d]); free(t->bmax[d]); free(t->rg[d]);
    }
    for (int k = 0; k < 6; ++k) free(t->Q[k]);
    free(t);
}

/* ------------------------------------------------------------------------------------------ */
/* Export helpers for the tests. */
void orc_info(const orc_tree *t, int64_t *out) {
    out[0] = t->N; out[1] = t->L; out[2] = t->nn;
    out[3] = t->E[0]; out[4] = t->E[1]; out[5] = t->E[2]; out[6] = t->Em; out[7] = t->n_ll;
}

void orc_export_nodes(const orc_tree *t, int64_t *first, int64_t *count, int32_t *axis, double *split,
                      int64_t *sums, double *mass, double *com, double *bmin, double *bmax, double *rg,
                      double *H, double *hint, double *hnode, double *Q) {
    for (int64_t n = 0; n < t->nn; ++n) {
        if (first) first[n] = t->first[n];
        if (count) count[n] = t->count[n];
        if (axis) axis[n] = t->axis[n];
        if (split) split[n] = t->split[n];
        if (sums) {
            i128 v[4] = {t->Msum[n], t->S[0][n], t->S[1][n], t->S[2][n]};
            for (int k = 0; k < 4; ++k) {
                sums[8 * n + 2 * k] = (int64_t)(uint64_t)(unsigned __int128)v[k];
                sums[8 * n + 2 * k + 1] = (int64_t)(v[k] >> 64);
            }
        }
        if (mass) mass[n] = t->mass[n];
        for (int d = 0; d < 3; ++d) {
            if (com) com[3 * n + d] = t->com[d][n];
            if (bmin) bmin[3 * n + d] = t->bmin[d][n];
            if (bmax) bmax[3 * n + d] = t->bmax[d][n];
            if (rg) rg[3 * n + d] = t->rg[d][n];
        }
        if (H) H[n] = t->H[n];
        if (hint) hint[n] = t->hint[n];
        if (hnode) hnode[n] = t->hnode[n];
        if (Q) for (int k = 0; k < 6; ++k) Q[6 * n + k] = t->Q[k][n];
    }
}

void orc_export_perm(const orc_tree *t, int32_t *perm) { memcpy(perm, t->perm, sizeof(int32_t) * t->N); }

void orc_export_fixed(const orc_tree *t, int64_t *P /* [N][4] in original order: m, x, y, z */) {
    for (int64_t i = 0; i < t->N; ++i) {
        int64_t o = t->perm[i];
        P[4 * o] = t->Pm[i];
        for (int d = 0; d < 3; ++d) P[4 * o + 1 + d] = t->P[d][i];
    }
}

double orc_i128_to_double(int64_t lo, int64_t hi) {
    i128 v = ((i128)hi << 64) | (i128)(uint64_t)lo;
    return (double)v;
}

/* ------------------------------------------------------------------------------------------ */
/* Sec. 2.2-2.4.1: per-sink depth-first walk from node 2 (the root is never accepted). */
typedef struct { int32_t *a; uint8_t *r; int64_t n, cap; } vec_t;

static int vpush(vec_t *v, int32_t id, uint8_t flag) {
    if (v->n == v->cap) {
        int64_t nc = v->cap ? 2 * v->cap : 64;
        int32_t *na = realloc(v->a, nc * sizeof(int32_t));
        if (!na) return ORC_ERR_ALLOC;
        v->a = na;
        uint8_t *nr = realloc(v->r, nc);
        if (!nr) return ORC_ERR_ALLOC;
        v->r = nr;
        v->cap = nc;
    }
    v->a[v->n] = id; v->r[v->n] = flag; v->n++;
    return ORC_OK;
}

/* mac_only: the variant of Sec. 2.5 without the reachability override (near lists from the MAC
 * alone); its near lists carry no neighbour candidates. */
static int walk_sink(const orc_tree *t, int64_t A, double theta2, int mac_only, vec_t *near, vec_t *far) {
    int64_t leaf0 = (int64_t)1 << t->L;
    int64_t n = 2;
    while (n != 1) {
        int descend = 0;
        if (t->count[n] > 0) {
            int is_leaf = n >= leaf0;
            double d2 = dist2(t->rg[0][A], t->rg[1][A], t->rg[2][A], t->rg[0][n], t->rg[1][n], t->rg[2][n]);
            double rr = t->hnode[A] + t->hint[n];
            if (!mac_only && d2 < rr * rr) {
                /* Sec. 2.3.1 reachable: never accepted by the MAC (Sec. 2.4.1). */
                if (is_leaf) { if (vpush(near, (int32_t)n, 1)) return ORC_ERR_ALLOC; }
                else descend = 1;
            } else {
                double R2 = dist2(t->com[0][A], t->com[1][A], t->com[2][A], t->com[0][n], t->com[1][n], t->com[2][n]);
                const double Hn = t->mac_box ? t->Hbis[n] : t->H[n];
                if (Hn * Hn < theta2 * R2) { if (vpush(far, (int32_t)n, 0)) return ORC_ERR_ALLOC; }
                else if (is_leaf) { if (vpush(near, (int32_t)n, 0)) return ORC_ERR_ALLOC; }
                else descend = 1;
            }
        }
        if (descend) n = 2 * n;
        else {
            while (n & 1) n >>= 1;
            n += 1;
        }
    }
    return ORC_OK;
}

static int walk_mode(orc_tree *t, double theta, const int32_t *sinks, int64_t nsinks, int mac_only);

int orc_walk(orc_tree *t, double theta, const int32_t *sinks, int64_t nsinks) {
    return walk_mode(t, theta, sinks, nsinks, 0);
}

/* The MAC-only walk (Sec. 2.5): every sink, near lists without the reachability override. */
/* The other reading of Eq. 4's cell size, for comparison (the library and the default walk read
 * H_B from the tight box of the cell's particles): Sec. 2.1.5 keeps each node's lowest-left
 * corner and size, which can also be read as the cell's bisection box, i.e. the root's tight box
 * cut by the split planes of all its ancestors.  The walk below takes H_B as that box's longest
 * side; everything else is the default walk. */
int orc_walk_bisection_box(orc_tree *t, double theta) {
    if (!t) return ORC_ERR_ARG;
    int64_t nn = t->nn;
    double *lo = xcalloc((size_t)(3 * nn), sizeof(double)), *hi = xcalloc((size_t)(3 * nn), sizeof(double));
    free(t->Hbis);
    t->Hbis = xcalloc((size_t)nn, sizeof(double));
    if (!lo || !hi || !t->Hbis) { free(lo); free(hi); return ORC_ERR_ALLOC; }
    for (int d = 0; d < 3; ++d) { lo[3 + d] = t->bmin[d][1]; hi[3 + d] = t->bmax[d][1]; }
    for (int64_t n = 1; n < nn; ++n) {
        double H = 0.0;
        for (int d = 0; d < 3; ++d) {
            double e = hi[3 * n + d] - lo[3 * n + d];
            if (e > H) H = e;
        }
        t->Hbis[n] = H;
        if (2 * n + 1 < nn) { /* the daughters: the box cut at the split plane of the cell's axis */
            for (int c = 0; c < 2; ++c)
                for (int d = 0; d < 3; ++d) { lo[3 * (2 * n + c) + d] = lo[3 * n + d]; hi[3 * (2 * n + c) + d] = hi[3 * n + d]; }
            hi[3 * (2 * n) + t->axis[n]] = t->split[n];
            lo[3 * (2 * n + 1) + t->axis[n]] = t->split[n];
        }
    }
    free(lo); free(hi);
    t->mac_box = 1;
    int r = walk_mode(t, theta, NULL, -1, 0);
    t->mac_box = 0;
    return r;
}

int orc_walk_mac_only(orc_tree *t, double theta) {
    return walk_mode(t, theta, NULL, -1, 1);
}

static int walk_mode(orc_tree *t, double theta, const int32_t *sinks, int64_t nsinks, int mac_only) {
    if (!(theta >= 0.0) || !isfinite(theta)) return ORC_ERR_ARG;
    free_lists(t);
    int64_t nl = (int64_t)1 << t->L, leaf0 = nl;
    t->theta = theta;
    t->walked_leaf = xcalloc(nl, 1);
    t->near_n = xcalloc(nl, sizeof(int64_t));
    t->far_n = xcalloc(nl, sizeof(int64_t));
    t->near_ids = xcalloc(nl, sizeof(int32_t *));
    t->near_reach = xcalloc(nl, sizeof(uint8_t *));
    t->far_ids = xcalloc(nl, sizeof(int32_t *));
    if (!t->walked_leaf || !t->near_n || !t->far_n || !t->near_ids || !t->near_reach || !t->far_ids) return ORC_ERR_ALLOC;
    if (nsinks < 0) {
        for (int64_t j = 0; j < nl; ++j) t->walked_leaf[j] = t->count[leaf0 + j] > 0;
    } else {
        for (int64_t s = 0; s < nsinks; ++s) {
            if (sinks[s] < 0 || sinks[s] >= nl) return ORC_ERR_ARG;
            t->walked_leaf[sinks[s]] = t->count[leaf0 + sinks[s]] > 0;
        }
    }
    double theta2 = theta * theta;
    int err = ORC_OK;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < nl; ++j) {
        if (!t->walked_leaf[j]) continue;
        vec_t near = {0}, far = {0};
        int e = walk_sink(t, leaf0 + j, theta2, mac_only, &near, &far);
        if (e) {
#pragma omp atomic write
            err = e;
        }
        t->near_ids[j] = near.a; t->near_reach[j] = near.r; t->near_n[j] = near.n;
        t->far_ids[j] = far.a; t->far_n[j] = far.n;
        free(far.r);
    }
    if (err) return err;
    t->walked = 1;
    return ORC_OK;
}

void orc_list_sizes(const orc_tree *t, int64_t *out) {
    int64_t nl = (int64_t)1 << t->L, a = 0, b = 0, c = 0;
    for (int64_t j = 0; t->walked && j < nl; ++j) {
        a += t->near_n[j];
        b += t->far_n[j];
        for (int64_t k = 0; k < t->near_n[j]; ++k) c += t->near_reach[j][k];
    }
    out[0] = a; out[1] = b; out[2] = c;
}

/* CSR over leaves j = 0 .. 2^L - 1 (node 2^L + j); lists in walk order. */
void orc_export_lists(const orc_tree *t, int64_t *near_off, int32_t *near_ids, uint8_t *near_reach,
                      int64_t *far_off, int32_t *far_ids) {
    int64_t nl = (int64_t)1 << t->L, pn = 0, pf = 0;
    near_off[0] = 0; far_off[0] = 0;
    for (int64_t j = 0; j < nl; ++j) {
        int64_t a = t->walked ? t->near_n[j] : 0, b = t->walked ? t->far_n[j] : 0;
        for (int64_t k = 0; k < a; ++k) { near_ids[pn + k] = t->near_ids[j][k]; near_reach[pn + k] = t->near_reach[j][k]; }
        for (int64_t k = 0; k < b; ++k) far_ids[pf + k] = t->far_ids[j][k];
        pn += a; pf += b;
        near_off[j + 1] = pn; far_off[j + 1] = pf;
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Sec. 2.3: neighbours of every particle of the walked sinks, culled from the candidate
 * (reachable) ll-cells: b != a with |r_a - r_b| < 2 h_a.  Rows in original order, each row
 * sorted by original index. */
static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int64_t orc_neighbours(const orc_tree *t, int64_t *offsets, int32_t *idx, int64_t cap) {
    if (!t->walked) return ORC_ERR_STATE;
    int64_t N = t->N, nl = (int64_t)1 << t->L, leaf0 = nl;
    int64_t *cnt = xcalloc(N, sizeof(int64_t));
    if (!cnt) return ORC_ERR_ALLOC;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < nl; ++j) {
        if (!t->walked_leaf[j]) continue;
        int64_t A = leaf0 + j;
        for (int64_t a = t->first[A]; a < t->first[A] + t->count[A]; ++a) {
            double s = 2.0 * t->h[a], s2 = s * s;
            int64_t c = 0;
            for (int64_t k = 0; k < t->near_n[j]; ++k) {
                if (!t->near_reach[j][k]) continue;
                int64_t B = t->near_ids[j][k];
                for (int64_t b = t->first[B]; b < t->first[B] + t->count[B]; ++b)
                    if (b != a && dist2(t->x[0][a], t->x[1][a], t->x[2][a], t->x[0][b], t->x[1][b], t->x[2][b]) < s2) ++c;
            }
            cnt[t->perm[a]] = c;
        }
    }
    offsets[0] = 0;
    for (int64_t i = 0; i < N; ++i) offsets[i + 1] = offsets[i] + cnt[i];
    int64_t total = offsets[N];
    free(cnt);
    if (!idx) return total;
    if (cap < total) return ORC_ERR_CAPACITY;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < nl; ++j) {
        if (!t->walked_leaf[j]) continue;
        int64_t A = leaf0 + j;
        for (int64_t a = t->first[A]; a < t->first[A] + t->count[A]; ++a) {
            double s = 2.0 * t->h[a], s2 = s * s;
            int64_t o = offsets[t->perm[a]], c = 0;
            for (int64_t k = 0; k < t->near_n[j]; ++k) {
                if (!t->near_reach[j][k]) continue;
                int64_t B = t->near_ids[j][k];
                for (int64_t b = t->first[B]; b < t->first[B] + t->count[B]; ++b)
                    if (b != a && dist2(t->x[0][a], t->x[1][a], t->x[2][a], t->x[0][b], t->x[1][b], t->x[2][b]) < s2)
                        idx[o + c++] = t->perm[b];
            }
            qsort(idx + o, (size_t)c, sizeof(int32_t), cmp_i32);
        }
    }
    return total;
}

/* Brute force O(N^2) reference for the neighbour test (the definition itself). */
int64_t orc_brute_neighbours(const double *x, const double *h, int64_t N, int64_t *offsets, int32_t *idx, int64_t cap) {
    offsets[0] = 0;
    for (int64_t a = 0; a < N; ++a) {
        double s = 2.0 * h[a], s2 = s * s;
        int64_t c = 0;
        for (int64_t b = 0; b < N; ++b) {
            if (b == a) continue;
            if (dist2(x[3 * a], x[3 * a + 1], x[3 * a + 2], x[3 * b], x[3 * b + 1], x[3 * b + 2]) < s2) {
                if (idx) {
                    if (offsets[a] + c >= cap) return ORC_ERR_CAPACITY;
                    idx[offsets[a] + c] = (int32_t)b;
                }
                ++c;
            }
        }
        offsets[a + 1] = offsets[a] + c;
    }
    return offsets[N];
}

/* ------------------------------------------------------------------------------------------ */
/* Sec. 2.4.3, Eq. 10: the softened force law S(q), q = r / h, h = (h_a + h_b) / 2. */
double orc_kernel_S(double r, double h) {
    double q = r / h;
    if (q < 1.0) return (4.0 / 3.0 * q - 6.0 / 5.0 * q * q * q + 0.5 * q * q * q * q) / (h * h);
    if (q < 2.0) return (8.0 / 3.0 * q - 3.0 * q * q + 6.0 / 5.0 * q * q * q - 1.0 / 6.0 * q * q * q * q - 1.0 / (15.0 * q * q)) / (h * h);
    return 1.0 / (r * r);
}

/* S(r) / r, written so that it stays finite at r = 0. */
double orc_kernel_S_over_r(double r, double h) {
    double q = r / h, h3 = h * h * h;
    if (q < 1.0) return (4.0 / 3.0 - 6.0 / 5.0 * q * q + 0.5 * q * q * q) / h3;
    if (q < 2.0) return (8.0 / 3.0 - 3.0 * q + 6.0 / 5.0 * q * q - 1.0 / 6.0 * q * q * q) / h3 - 1.0 / (15.0 * r * r * r);
    return 1.0 / (r * r * r);
}

/* (d/dr)(S/r) / r, finite at r = 0 (used by the backward pass). */
double orc_kernel_dSr_over_r(double r, double h) {
    double q = r / h, h5 = h * h * h * h * h;
    if (q < 1.0) return (-12.0 / 5.0 + 1.5 * q) / h5;
    if (q < 2.0) return (-3.0 / q + 12.0 / 5.0 - 0.5 * q) / h5 + 1.0 / (5.0 * r * r * r * r * r);
    return -3.0 / (r * r * r * r * r);
}

/* Softened potential per unit source mass: phi' = S and phi = -1/r for q >= 2. */
double orc_kernel_phi(double r, double h) {
    double q = r / h;
    if (q < 1.0) return (2.0 / 3.0 * q * q - 0.3 * q * q * q * q + 0.1 * q * q * q * q * q - 7.0 / 5.0) / h;
    if (q < 2.0) return (4.0 / 3.0 * q * q - q * q * q + 0.3 * q * q * q * q - 1.0 / 30.0 * q * q * q * q * q - 8.0 / 5.0) / h + 1.0 / (15.0 * r);
    return -1.0 / r;
}

/* ------------------------------------------------------------------------------------------ */
/* Derivatives of 1/r.  For a multi-index (i_1 .. i_n):
 *   d^n (1/r) = sum_k (-1)^(n-k) (2n-2k-1)!! r^-(2n-2k+1) * T_k,
 * where T_k sums, over every choice of k disjoint index pairs, the product of a Kronecker
 * delta per pair and x_i for every unpaired index. */
static double pairings(const int *idx, int n, unsigned mask, int k, const double *x) {
    if (mask == 0) return k == 0 ? 1.0 : 0.0;
    int p = __builtin_ctz(mask);
    unsigned rest = mask & ~(1u << p);
    double s = x[idx[p]] * pairings(idx, n, rest, k, x);
    if (k > 0)
        for (int q = p + 1; q < n; ++q)
            if ((rest >> q) & 1u)
                if (idx[p] == idx[q]) s += pairings(idx, n, rest & ~(1u << q), k - 1, x);
    return s;
}

double orc_dinv_r(int n, const int *idx, const double *x) {
    double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
    double r = sqrt(r2);
    double s = 0.0;
    for (int k = 0; 2 * k <= n; ++k) {
        double df = 1.0;
        for (int v = 2 * n - 2 * k - 1; v > 1; v -= 2) df *= v;
        double sign = ((n - k) & 1) ? -1.0 : 1.0;
        double T = pairings(idx, n, (n ? (1u << n) - 1u : 0u), k, x);
        s += sign * df * T / pow(r, 2 * n - 2 * k + 1);
    }
    return s;
}

/* Storage of symmetric tensors of order 0..3 in 1 + 3 + 6 + 10 = 20 coefficients: order n
 * keeps the sorted index tuples in lexicographic order. */
static const int ORD_OFF[4] = {0, 1, 4, 10};
static int sym_slot(int n, const int *idx) {
    int s[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i) s[i] = idx[i];
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (s[j] < s[i]) { int t = s[i]; s[i] = s[j]; s[j] = t; }
    int slot = 0;
    if (n == 1) slot = s[0];
    else if (n == 2) { static const int T2[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}}; slot = T2[s[0]][s[1]]; }
    else if (n == 3) {
        static const int T3[3][3][3] = {{{0, 1, 2}, {1, 3, 4}, {2, 4, 5}},
                                        {{1, 3, 4}, {3, 6, 7}, {4, 7, 8}},
                                        {{2, 4, 5}, {4, 7, 8}, {5, 8, 9}}};
        slot = T3[s[0]][s[1]][s[2]];
    }
    return ORD_OFF[n] + slot;
}

static void sym_tuple(int n, int slot, int *idx) {
    /* inverse of sym_slot: enumerate sorted tuples in lexicographic order */
    int c = 0;
    if (n == 0) return;
    if (n == 1) { idx[0] = slot; return; }
    if (n == 2) { for (int a = 0; a < 3; ++a) for (int b = a; b < 3; ++b) { if (c++ == slot) { idx[0] = a; idx[1] = b; return; } } }
    for (int a = 0; a < 3; ++a) for (int b = a; b < 3; ++b) for (int d = b; d < 3; ++d)
        if (c++ == slot) { idx[0] = a; idx[1] = b; idx[2] = d; return; }
}

static void q_full(const double *q6, double Q[3][3]) {
    Q[0][0] = q6[0]; Q[0][1] = Q[1][0] = q6[1]; Q[0][2] = Q[2][0] = q6[2];
    Q[1][1] = q6[3]; Q[1][2] = Q[2][1] = q6[4]; Q[2][2] = q6[5];
}

/* Eq. 5 about the source centre of mass: Phi_B(r) = -M/r - (1/2) x Q x / r^5, which for a
 * traceless Q equals -M D0 - (1/6) Q_lm D_lm.  Its derivatives of order 0..3 at R = r_A - r_B
 * are the sink's Taylor coefficients (Sec. 2.4.2, Eq. 6). */
void orc_far_coeffs(const double *R, double M, const double *q6, double *C) {
    double Q[3][3];
    q_full(q6, Q);
    for (int n = 0; n <= 3; ++n) {
        int cnt = n == 0 ? 1 : n == 1 ? 3 : n == 2 ? 6 : 10;
        for (int s = 0; s < cnt; ++s) {
            int idx[8];
            sym_tuple(n, s, idx);
            double v = -M * orc_dinv_r(n, idx, R);
            double qt = 0.0;
            for (int l = 0; l < 3; ++l)
                for (int mm = 0; mm < 3; ++mm) {
                    idx[n] = l; idx[n + 1] = mm;
                    qt += Q[l][mm] * orc_dinv_r(n + 2, idx, R);
                }
            C[ORD_OFF[n] + s] += v - qt / 6.0;
        }
    }
}

/* Phi(d) = C0 + C1 d + 1/2 d C2 d + 1/6 C3 d d d and a = -grad Phi, d = r_a - r_A. */
void orc_taylor_eval(const double *C, const double *d, double *phi, double *acc) {
    double p = C[0];
    double g[3] = {0, 0, 0};
    for (int i = 0; i < 3; ++i) {
        int ii[3] = {i, 0, 0};
        p += C[sym_slot(1, ii)] * d[i];
        g[i] += C[sym_slot(1, ii)];
        for (int j = 0; j < 3; ++j) {
            int ij[3] = {i, j, 0};
            p += 0.5 * C[sym_slot(2, ij)] * d[i] * d[j];
            g[i] += C[sym_slot(2, ij)] * d[j];
            for (int k = 0; k < 3; ++k) {
                int ijk[3] = {i, j, k};
                p += C[sym_slot(3, ijk)] * d[i] * d[j] * d[k] / 6.0;
                g[i] += 0.5 * C[sym_slot(3, ijk)] * d[j] * d[k];
            }
        }
    }
    *phi = p;
    for (int i = 0; i < 3; ++i) acc[i] = -g[i];
}

/* Sec. 2.4: gravity on every particle of the walked sinks (original order); other entries of
 * acc/pot are left as they are. */
int orc_gravity(const orc_tree *t, double *acc, double *pot) {
    if (!t->walked) return ORC_ERR_STATE;
    int64_t nl = (int64_t)1 << t->L, leaf0 = nl;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < nl; ++j) {
        if (!t->walked_leaf[j]) continue;
        int64_t A = leaf0 + j;
        double C[20] = {0};
        for (int64_t k = 0; k < t->far_n[j]; ++k) {
            int64_t B = t->far_ids[j][k];
            double R[3], q6[6];
            for (int d = 0; d < 3; ++d) R[d] = t->com[d][A] - t->com[d][B];
            for (int q = 0; q < 6; ++q) q6[q] = t->Q[q][B];
            orc_far_coeffs(R, t->mass[B], q6, C);
        }
        for (int64_t a = t->first[A]; a < t->first[A] + t->count[A]; ++a) {
            double d[3], phi, af[3];
            for (int q = 0; q < 3; ++q) d[q] = t->x[q][a] - t->com[q][A];
            orc_taylor_eval(C, d, &phi, af);
            /* near field, Eq. 9: a_a = -sum_{b != a} m_b S(r_ab, h) e_ab */
            double an[3] = {0, 0, 0}, pn = 0.0;
            for (int64_t k = 0; k < t->near_n[j]; ++k) {
                int64_t B = t->near_ids[j][k];
                for (int64_t b = t->first[B]; b < t->first[B] + t->count[B]; ++b) {
                    if (b == a) continue;
                    double rv[3] = {t->x[0][a] - t->x[0][b], t->x[1][a] - t->x[1][b], t->x[2][a] - t->x[2][b]};
                    double r = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
                    double hab = 0.5 * (t->h[a] + t->h[b]);
                    double sr = orc_kernel_S_over_r(r, hab);
                    for (int q = 0; q < 3; ++q) an[q] -= t->m[b] * sr * rv[q];
                    pn += t->m[b] * orc_kernel_phi(r, hab);
                }
            }
            int64_t o = t->perm[a];
            for (int q = 0; q < 3; ++q) acc[3 * o + q] = af[q] + an[q];
            if (pot) pot[o] = phi + pn;
        }
    }
    return ORC_OK;
}

/* The truth of Sec. 3.1: direct kernel-softened summation over all b != a, for a set of
 * target particles (original indices). */
void orc_direct(const double *x, const double *m, const double *h, int64_t N, const int64_t *targets, int64_t nt,
                double *acc, double *pot) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t s = 0; s < nt; ++s) {
        int64_t a = targets ? targets[s] : s;
        double an[3] = {0, 0, 0}, pn = 0.0;
        for (int64_t b = 0; b < N; ++b) {
            if (b == a) continue;
            double rv[3] = {x[3 * a] - x[3 * b], x[3 * a + 1] - x[3 * b + 1], x[3 * a + 2] - x[3 * b + 2]};
            double r = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
            double hab = 0.5 * (h[a] + h[b]);
            double sr = orc_kernel_S_over_r(r, hab);
            for (int q = 0; q < 3; ++q) an[q] -= m[b] * sr * rv[q];
            pn += m[b] * orc_kernel_phi(r, hab);
        }
        for (int q = 0; q < 3; ++q) acc[3 * s + q] = an[q];
        if (pot) pot[s] = pn;
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Gradients.  The pair term F(r) = (S/r)(r) r_vec has Jacobian (S/r) I + ((S/r)'/r) r r^T, and
 * d phi / d r_vec = S r_vec / r = (S/r) r_vec.  Given gA = dL/da_a and gP = dL/dPhi_a, one pair
 * (a, b) adds
 *   dL/dx_a += g,  dL/dx_b -= g,  g = -m_b [(S/r) gA + ((S/r)'/r) (r.gA) r] + gP m_b (S/r) r
 *   dL/dm_b += -(S/r) (r.gA) + gP phi. */
static void pair_grad(const double *rv, double ma_b, double hab, const double *gA, double gP, double *g, double *gm) {
    double r = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
    double sr = orc_kernel_S_over_r(r, hab);
    double dsr = orc_kernel_dSr_over_r(r, hab);
    double rg = rv[0] * gA[0] + rv[1] * gA[1] + rv[2] * gA[2];
    for (int q = 0; q < 3; ++q) g[q] = -ma_b * (sr * gA[q] + dsr * rg * rv[q]) + gP * ma_b * sr * rv[q];
    *gm = -sr * rg + gP * orc_kernel_phi(r, hab);
}

/* Analytic vector-Jacobian product of the direct sum (all particles are targets). */
void orc_direct_grad(const double *x, const double *m, const double *h, int64_t N, const double *gacc,
                     const double *gpot, double *gx, double *gm) {
    for (int64_t i = 0; i < 3 * N; ++i) gx[i] = 0.0;
    for (int64_t i = 0; i < N; ++i) gm[i] = 0.0;
    for (int64_t a = 0; a < N; ++a)
        for (int64_t b = 0; b < N; ++b) {
            if (b == a) continue;
            double rv[3] = {x[3 * a] - x[3 * b], x[3 * a + 1] - x[3 * b + 1], x[3 * a + 2] - x[3 * b + 2]};
            double g[3], gmb;
            pair_grad(rv, m[b], 0.5 * (h[a] + h[b]), gacc + 3 * a, gpot ? gpot[a] : 0.0, g, &gmb);
            for (int q = 0; q < 3; ++q) { gx[3 * a + q] += g[q]; gx[3 * b + q] -= g[q]; }
            gm[b] += gmb;
        }
}

/* Refit with a frozen structure (Sec. 2.1.8): new positions and masses (original order) keep
 * every particle in its ll-cell; sums, centres of mass, boxes, quadrupoles and radii are
 * recomputed bottom-up.  The interaction lists stay as they are. */
int orc_refit(orc_tree *t, const double *x, const double *m) {
    for (int64_t i = 0; i < t->N; ++i) {
        int64_t o = t->perm[i];
        for (int d = 0; d < 3; ++d) t->x[d][i] = x[3 * o + d] + 0.0;
        t->m[i] = m[o];
        if (!isfinite(t->x[0][i]) || !isfinite(t->x[1][i]) || !isfinite(t->x[2][i]) || !(m[o] > 0.0)) return ORC_ERR_ARG;
    }
    if (fixed_point(t) != ORC_OK) return ORC_ERR_ARG;
    for (int64_t n = 1; n < t->nn; ++n) node_from_particles(t, n);
    moments(t);
    return ORC_OK;
}

/* SPH density by summation over the neighbour lists (Sec. 2.3: smoothed quantities are sums of
 * kernel-weighted particle properties over the neighbours):
 *   rho_a = m_a W(0, h_a) + sum_{b in nb(a)} m_b W(r_ab, h_a),
 * with the cubic spline kernel W the paper uses (Monaghan & Lattanzio 1985, support 2h),
 *   W(r, h) = (1 - 3/2 q^2 + 3/4 q^3) / (pi h^3)   0 <= q < 1
 *             (2 - q)^3 / (4 pi h^3)                1 <= q < 2,   q = r / h,
 * and nb(a) the neighbour rows of orc_neighbours (b != a, r_ab < 2 h_a), original order. */
double orc_kernel_W(double r, double h) {
    double q = r / h, w;
    if (q < 1.0) w = 1.0 - 1.5 * q * q + 0.75 * q * q * q;
    else if (q < 2.0) w = 0.25 * (2.0 - q) * (2.0 - q) * (2.0 - q);
    else w = 0.0;
    return w / (3.14159265358979323846 * h * h * h);
}

int orc_density_csr(int64_t N, const double *x, const double *m, const double *h, const int64_t *off,
                    const int32_t *idx, double *rho) {
    for (int64_t a = 0; a < N; ++a) {
        double s = m[a] * orc_kernel_W(0.0, h[a]);
        for (int64_t k = off[a]; k < off[a + 1]; ++k) {
            int64_t b = idx[k];
            double dx = x[3 * a] - x[3 * b], dy = x[3 * a + 1] - x[3 * b + 1], dz = x[3 * a + 2] - x[3 * b + 2];
            s += m[b] * orc_kernel_W(sqrt(dx * dx + dy * dy + dz * dz), h[a]);
        }
        rho[a] = s;
    }
    return ORC_OK;
}

/* Tree update with its integrity check (Sec. 2.1.8).  A particle is still in its ll-cell when,
 * at its new position (original order), it lies on the side of every ancestor's split plane that
 * it was sorted to: x_axis < split for a left child, not less for a right child.  Only planes
 * with particles on both sides count: a cell whose other child is empty separates nothing (a
 * one-particle cell is split through that particle).  A non-finite coordinate counts as
 * outside.  *outside receives the number of particles that left their
 * ll-cells.  When it is zero, the smoothing lengths are replaced, the moments, boxes and radii
 * are refitted (orc_refit) and the interaction lists are dropped, for the caller to walk again;
 * otherwise the tree is left unchanged and the caller rebuilds. */
int orc_update(orc_tree *t, const double *x, const double *m, const double *h, int64_t *outside) {
    int64_t out = 0, leaf0 = (int64_t)1 << t->L;
    for (int64_t j = 0; j < leaf0; ++j) {
        int64_t n0 = leaf0 + j;
        for (int64_t a = t->first[n0]; a < t->first[n0] + t->count[n0]; ++a) {
            int64_t o = t->perm[a];
            int ok = isfinite(x[3 * o]) && isfinite(x[3 * o + 1]) && isfinite(x[3 * o + 2]);
            for (int64_t n = n0; n > 1 && ok; n >>= 1) {
                int64_t par = n >> 1;
                if (t->count[n ^ 1] == 0) continue;
                double v = x[3 * o + t->axis[par]];
                ok = (n & 1) == 0 ? (v < t->split[par]) : !(v < t->split[par]);
            }
            if (!ok) ++out;
        }
    }
    *outside = out;
    if (out > 0) return ORC_OK;
    for (int64_t i = 0; i < t->N; ++i)
        if (!isfinite(h[t->perm[i]]) || !(h[t->perm[i]] > 0.0)) return ORC_ERR_ARG;
    for (int64_t i = 0; i < t->N; ++i) t->h[i] = h[t->perm[i]];
    int r = orc_refit(t, x, m);
    free_lists(t);
    return r;
}

/* Vector-Jacobian product of orc_gravity with frozen lists, with respect to positions and
 * masses.  Node moments are the exact functions M = sum m_b, COM = sum m_b x_b / M,
 * Q = sum m_b (3 d d - d^2 I), d = x_b - COM (Eq. 2 reproduces Eq. 1 exactly); because
 * sum m_b d_b = 0, Q has no derivative through COM.  Requires every leaf walked. */
int orc_gravity_backward(const orc_tree *t, const double *gacc, const double *gpot, double *gx, double *gm) {
    if (!t->walked) return ORC_ERR_STATE;
    int64_t N = t->N, nl = (int64_t)1 << t->L, leaf0 = nl, nn = t->nn;
    for (int64_t j = 0; j < nl; ++j)
        if (t->count[leaf0 + j] > 0 && !t->walked_leaf[j]) return ORC_ERR_STATE;
    /* gradients in sorted order, then scattered */
    double *sx = xcalloc(3 * N, sizeof(double)), *sm = xcalloc(N, sizeof(double));
    double *Mbar = xcalloc(nn, sizeof(double)), *Cbar = xcalloc(3 * nn, sizeof(double)), *Qbar = xcalloc(9 * nn, sizeof(double));
    if (!sx || !sm || !Mbar || !Cbar || !Qbar) { free(sx); free(sm); free(Mbar); free(Cbar); free(Qbar); return ORC_ERR_ALLOC; }

    for (int64_t j = 0; j < nl; ++j) {
        if (!t->walked_leaf[j]) continue;
        int64_t A = leaf0 + j;
        /* far field: coefficients, then the adjoint of the Taylor evaluation */
        double C[20] = {0};
        for (int64_t k = 0; k < t->far_n[j]; ++k) {
            int64_t B = t->far_ids[j][k];
            double R[3], q6[6];
            for (int d = 0; d < 3; ++d) R[d] = t->com[d][A] - t->com[d][B];
            for (int q = 0; q < 6; ++q) q6[q] = t->Q[q][B];
            orc_far_coeffs(R, t->mass[B], q6, C);
        }
        double Cb[20] = {0};   /* dL/dC, one entry per stored (symmetric) slot */
        double comA_bar[3] = {0, 0, 0};
        for (int64_t a = t->first[A]; a < t->first[A] + t->count[A]; ++a) {
            int64_t o = t->perm[a];
            const double *v = gacc + 3 * o;
            double w = gpot ? gpot[o] : 0.0;
            double d[3];
            for (int q = 0; q < 3; ++q) d[q] = t->x[q][a] - t->com[q][A];
            /* Phi = sum over full index tuples; a_i = -(grad Phi)_i */
            double gd[3] = {0, 0, 0};
            Cb[0] += w;
            for (int i = 0; i < 3; ++i) {
                int ii[3] = {i, 0, 0};
                int s1 = sym_slot(1, ii);
                Cb[s1] += w * d[i] - v[i];
                gd[i] += w * C[s1];
                for (int jx = 0; jx < 3; ++jx) {
                    int ij[3] = {i, jx, 0};
                    int s2 = sym_slot(2, ij);
                    Cb[s2] += 0.5 * w * d[i] * d[jx] - v[i] * d[jx];
                    gd[jx] += w * C[s2] * d[i];           /* d/dd_j of 1/2 C2 d d (both slots) */
                    gd[jx] += -v[i] * C[s2];              /* a_i = -(C2_ij d_j + ...) */
                    for (int k = 0; k < 3; ++k) {
                        int ijk[3] = {i, jx, k};
                        int s3 = sym_slot(3, ijk);
                        Cb[s3] += w * d[i] * d[jx] * d[k] / 6.0 - 0.5 * v[i] * d[jx] * d[k];
                        gd[k] += w * C[s3] * d[i] * d[jx] / 2.0;
                        gd[k] += -v[i] * C[s3] * d[jx];
                    }
                }
            }
            for (int q = 0; q < 3; ++q) { sx[3 * a + q] += gd[q]; comA_bar[q] -= gd[q]; }

            /* near field pairs */
            for (int64_t k = 0; k < t->near_n[j]; ++k) {
                int64_t B = t->near_ids[j][k];
                for (int64_t b = t->first[B]; b < t->first[B] + t->count[B]; ++b) {
                    if (b == a) continue;
                    double rv[3] = {t->x[0][a] - t->x[0][b], t->x[1][a] - t->x[1][b], t->x[2][a] - t->x[2][b]};
                    double g[3], gmb;
                    pair_grad(rv, t->m[b], 0.5 * (t->h[a] + t->h[b]), v, w, g, &gmb);
                    for (int q = 0; q < 3; ++q) { sx[3 * a + q] += g[q]; sx[3 * b + q] -= g[q]; }
                    sm[b] += gmb;
                }
            }
        }
        /* adjoint of each far interaction C += T(R; M_B, Q_B), R = COM_A - COM_B */
        for (int64_t k = 0; k < t->far_n[j]; ++k) {
            int64_t B = t->far_ids[j][k];
            double R[3], Q[3][3], q6[6];
            for (int d = 0; d < 3; ++d) R[d] = t->com[d][A] - t->com[d][B];
            for (int q = 0; q < 6; ++q) q6[q] = t->Q[q][B];
            q_full(q6, Q);
            double M = t->mass[B], Rbar[3] = {0, 0, 0};
            for (int n = 0; n <= 3; ++n) {
                int cnt = n == 0 ? 1 : n == 1 ? 3 : n == 2 ? 6 : 10;
                for (int s = 0; s < cnt; ++s) {
                    double cb = Cb[ORD_OFF[n] + s];
                    if (cb == 0.0) continue;
                    int idx[10];
                    sym_tuple(n, s, idx);
                    Mbar[B] += -cb * orc_dinv_r(n, idx, R);
                    for (int p = 0; p < 3; ++p) {
                        idx[n] = p;
                        Rbar[p] += -M * cb * orc_dinv_r(n + 1, idx, R);
                    }
                    for (int l = 0; l < 3; ++l)
                        for (int mm = 0; mm < 3; ++mm) {
                            idx[n] = l; idx[n + 1] = mm;
                            Qbar[9 * B + 3 * l + mm] += -cb * orc_dinv_r(n + 2, idx, R) / 6.0;
                            for (int p = 0; p < 3; ++p) {
                                idx[n + 2] = p;
                                Rbar[p] += -Q[l][mm] * cb * orc_dinv_r(n + 3, idx, R) / 6.0;
                            }
                        }
                }
            }
            for (int q = 0; q < 3; ++q) { comA_bar[q] += Rbar[q]; Cbar[3 * B + q] -= Rbar[q]; }
        }
        for (int q = 0; q < 3; ++q) Cbar[3 * A + q] += comA_bar[q];
    }
    /* node moments -> particles: every node with a non-zero adjoint, over its particles */
    for (int64_t n = 1; n < nn; ++n) {
        if (t->count[n] == 0) continue;
        int nz = Mbar[n] != 0.0 || Cbar[3 * n] != 0.0 || Cbar[3 * n + 1] != 0.0 || Cbar[3 * n + 2] != 0.0;
        for (int k = 0; k < 9 && !nz; ++k) nz = Qbar[9 * n + k] != 0.0;
        if (!nz) continue;
        double M = t->mass[n];
        for (int64_t b = t->first[n]; b < t->first[n] + t->count[n]; ++b) {
            double d[3], d2 = 0.0;
            for (int q = 0; q < 3; ++q) { d[q] = t->x[q][b] - t->com[q][n]; d2 += d[q] * d[q]; }
            double gmb = Mbar[n];
            for (int q = 0; q < 3; ++q) gmb += Cbar[3 * n + q] * d[q] / M;
            for (int l = 0; l < 3; ++l)
                for (int mm = 0; mm < 3; ++mm)
                    gmb += Qbar[9 * n + 3 * l + mm] * (3.0 * d[l] * d[mm] - (l == mm ? d2 : 0.0));
            sm[b] += gmb;
            for (int k = 0; k < 3; ++k) {
                double g = Cbar[3 * n + k] * t->m[b] / M;
                for (int l = 0; l < 3; ++l)
                    for (int mm = 0; mm < 3; ++mm) {
                        double dq = 3.0 * ((l == k ? d[mm] : 0.0) + (mm == k ? d[l] : 0.0)) - (l == mm ? 2.0 * d[k] : 0.0);
                        g += Qbar[9 * n + 3 * l + mm] * t->m[b] * dq;
                    }
                sx[3 * b + k] += g;
            }
        }
    }
    for (int64_t i = 0; i < N; ++i) {
        int64_t o = t->perm[i];
        for (int q = 0; q < 3; ++q) gx[3 * o + q] = sx[3 * i + q];
        gm[o] = sm[i];
    }
    free(sx); free(sm); free(Mbar); free(Cbar); free(Qbar);
    return ORC_OK;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
