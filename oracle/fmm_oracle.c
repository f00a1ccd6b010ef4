/*
 * fmm_oracle.c -- plain, slow, FP64 CPU oracle for the 3-D Laplace FMM hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this code; the library's product path never does.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * What it computes (Yokota & Barba, "Hierarchical N-body simulations with
 * auto-tuning for heterogeneous systems"):
 *   * the Laplace potential and its gradient for N charges (Results section:
 *     "Laplace kernel potential and force"):
 *       phi_i  = sum_{j != i, r_ij > 0} q_j / r_ij
 *       grad_i = -sum_{j != i, r_ij > 0} q_j (x_i - x_j) / r_ij^3
 *     computed either exactly (direct all-pairs sum, Introduction / Gordon
 *     Bell section: the O(N^2) "all-pairs" summation) or by the FMM below;
 *   * the adaptive octree of cells holding at most N_crit particles
 *     (Results section, definition of N_crit);
 *   * the stack-based dual tree traversal (section "Dual tree traversal",
 *     Fig. "treewalk") with the MAC theta = (r_t + r_s)/R (Results section);
 *   * spherical-harmonic multipole/local expansions of order p (section
 *     "Hybrid treecode/FMM algorithm": "Our kernels are based on spherical
 *     harmonic expansions") -- P2M, M2M, M2L, L2L, L2P, M2P and P2P.
 *
 * Readings taken where the paper is silent:
 *   R1 quantisation: box = [lo, lo+side)^3 with lo = per-axis minimum,
 *      side = largest extent (1 if zero); k_d = min(2^21-1, floor((x_d-lo_d)*s)),
 *      s = 2^21/side, each a single IEEE FP64 operation; key bit 3b+a = bit b of k_a
 *      (a = 0,1,2 for x,y,z); sort by (key, original index).
 *   R2 tree: a cell at level l splits iff count > ncrit and l < max_depth; the
 *      children are the non-empty octants (x + 2y + 4z) in octant order.
 *   R3 MAC: r = half the cell side; accept iff R > 0 and (r_t + r_s)^2 <= theta^2 R^2,
 *      evaluated exactly in integer units of the finest grid.  With this reading
 *      theta = 0.5 reproduces the paper's statement that it is equivalent to a
 *      3x3x3 neighbour list.
 *   R4 traversal: interact(T,S) = MAC -> cell-cell (M2L); else both leaves ->
 *      particle-particle (P2P); else push.  Pop -> split the larger cell (target
 *      on a tie; the other one if the chosen cell is a leaf).  Flags select the
 *      literal "leaf pair first" order of the prose for comparison and, for
 *      the tests that show the split rule is pinned, two wrong split rules
 *      (split the smaller cell; split the source on a tie).
 *   R5 expansion centres are the geometric cell centres; truncation is n <= p
 *      for both multipole and local expansions.
 *   R6 coincident pairs (r = 0) contribute nothing.
 *   R9 hybrid selection (section "A new hybrid treecode-FMM with auto-tuning":
 *      the interaction type of a far pair is chosen during the traversal to
 *      minimise the cost, and particle-particle interactions may be taken above
 *      the leaf level): a pair accepted by the MAC becomes cell-cell or
 *      particle-particle by a table sel[b(n_t) * 128 + b(n_s)] (0 = M2L,
 *      1 = P2P) over the particle counts of the two cells, with the count
 *      bucket b(n) = n - 1 for n < 4, else 3 + 4(e - 2) + bits e-1..e-2 of n
 *      below its leading bit (e = floor(log2 n)).  The table is an input: how it
 *      was obtained (pre-timed kernels, a learned cost model) does not enter the
 *      traversal.  A P2P pair may have non-leaf cells; it acts on all particles
 *      of both.  Table value 2 selects the cell-particle interaction (M2P, the
 *      treecode kernel: the source multipole evaluated at every particle of
 *      the target cell); a table of all 2 is the paper's treecode.  Value 3
 *      selects the particle-cell interaction (P2L: the source particles added
 *      straight into the target cell's local expansion, before L2L).
 *
 * Harmonics (signed m, Condon-Shortley P_n^m):
 *   R_n^m(x) = r^n P_n^m(cos t) e^{i m f} / (n+m)!      (regular)
 *   I_n^m(x) = (n-m)! P_n^m(cos t) e^{i m f} / r^{n+1}  (irregular)
 * so that 1/|x-y| = sum_{n,m} conj(R_n^m(y)) I_n^m(x) for |y| < |x|
 * (Greengard & Rokhlin 1987, the paper's FMM reference).  Both are generated by
 * the Legendre three-term recurrence written in Cartesian form (u = x + iy):
 *   R_0^0 = 1, R_m^m = -u/(2m) R_{m-1}^{m-1},
 *   (n+m)(n-m) R_n^m = (2n-1) z R_{n-1}^m - r^2 R_{n-2}^m
 *   I_0^0 = 1/r, I_m^m = -(2m-1) u/r^2 I_{m-1}^{m-1},
 *   r^2 I_n^m = (2n-1) z I_{n-1}^m - (n+m-1)(n-m-1) I_{n-2}^m
 * and R_n^{-m} = (-1)^m conj(R_n^m), likewise for I.
 * Operators (c = expansion centre):
 *   P2M  M_n^m = sum_j q_j conj(R_n^m(y_j - c))
 *   M2M  M'_n^m = sum_{k,l} conj(R_k^l(c - c')) M_{n-k}^{m-l}
 *   M2L  L_j^l = (-1)^{j+l} sum_{n<=p,m} M_n^m I_{n+j}^{m-l}(c_t - c_s)
 *   L2L  L'_j^l = sum_{n>=j,m} L_n^m R_{n-j}^{m-l}(c' - c)
 *   L2P  phi = sum L_n^m R_n^m(x - c);  d/dz phi = sum L_n^m R_{n-1}^m;
 *        (d/dx + i d/dy) phi = sum L_n^m R_{n-1}^{m+1}
 *   P2L  L_n^m = sum_j q_j conj(I_n^m(y_j - c))   (expansion of 1/|x - y_j| about c)
 *   M2P  phi = sum M_n^m I_n^m(x - c);  d/dz I_n^m = -I_{n+1}^m;
 *        (d/dx + i d/dy) I_n^m = I_{n+1}^{m+1}
 * Coefficients are stored for all signed m at index n*n + n + m.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -fPIC -shared.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_KBITS 21
#define ORC_KMAX ((1LL << ORC_KBITS) - 1)
#define ORC_SEL_NB 128

/* flags of orc_fmm_create: the literal leaf-first order of the prose, and two
 * wrong split rules that exist only so that tests can show they are caught */
#define ORC_LEAF_FIRST 1
#define ORC_SPLIT_SMALLER 2
#define ORC_SPLIT_SOURCE_ON_TIE 4

static inline int hidx(int n, int m) { return n * n + n + m; }
static inline int nterms(int p) { return (p + 1) * (p + 1); }

/* ------------------------------------------------------------------ */
/* Harmonics                                                           */
/* ------------------------------------------------------------------ */

/* Regular solid harmonics R_n^m(x) for n <= p, all signed m. */
void orc_regular(const double x[3], int p, cplx *R)
{
    const double X = x[0], Y = x[1], Z = x[2];
    const double r2 = X * X + Y * Y + Z * Z;
    const cplx u = X + I * Y;
    for (int m = 0; m <= p; ++m) {
        if (m == 0)
            R[hidx(0, 0)] = 1.0;
        else
            R[hidx(m, m)] = -u / (2.0 * m) * R[hidx(m - 1, m - 1)];
        for (int n = m + 1; n <= p; ++n) {
            cplx prev2 = (n - 2 >= m) ? R[hidx(n - 2, m)] : 0.0;
            R[hidx(n, m)] = ((2.0 * n - 1.0) * Z * R[hidx(n - 1, m)] - r2 * prev2) /
                            ((double)(n + m) * (double)(n - m));
        }
    }
    for (int n = 1; n <= p; ++n)
        for (int m = 1; m <= n; ++m)
            R[hidx(n, -m)] = ((m & 1) ? -1.0 : 1.0) * conj(R[hidx(n, m)]);
}

/* Irregular solid harmonics I_n^m(x) for n <= p, all signed m (x != 0). */
void orc_irregular(const double x[3], int p, cplx *Ih)
{
    const double X = x[0], Y = x[1], Z = x[2];
    const double r2 = X * X + Y * Y + Z * Z;
    const double r = sqrt(r2);
    const cplx u = X + I * Y;
    for (int m = 0; m <= p; ++m) {
        if (m == 0)
            Ih[hidx(0, 0)] = 1.0 / r;
        else
            Ih[hidx(m, m)] = -(2.0 * m - 1.0) * u / r2 * Ih[hidx(m - 1, m - 1)];
        for (int n = m + 1; n <= p; ++n) {
            cplx prev2 = (n - 2 >= m) ? Ih[hidx(n - 2, m)] : 0.0;
            Ih[hidx(n, m)] = ((2.0 * n - 1.0) * Z * Ih[hidx(n - 1, m)] -
                              (double)(n + m - 1) * (double)(n - m - 1) * prev2) / r2;
        }
    }
    for (int n = 1; n <= p; ++n)
        for (int m = 1; m <= n; ++m)
            Ih[hidx(n, -m)] = ((m & 1) ? -1.0 : 1.0) * conj(Ih[hidx(n, m)]);
}

/* ------------------------------------------------------------------ */
/* Operators on single expansions                                      */
/* ------------------------------------------------------------------ */

/* P2M: M += sum_j q_j conj(R(y_j - c)). y is [n][3]. */
void orc_p2m(const double c[3], const double *y, const double *q, int64_t n, int p, cplx *M)
{
    cplx *R = malloc(sizeof(cplx) * nterms(p));
    for (int64_t j = 0; j < n; ++j) {
        double d[3] = {y[3 * j] - c[0], y[3 * j + 1] - c[1], y[3 * j + 2] - c[2]};
        orc_regular(d, p, R);
        for (int k = 0; k < nterms(p); ++k)
            M[k] += q[j] * conj(R[k]);
    }
    free(R);
}

/* M2M: shift the multipole M about c to M' about c' (accumulates into Mp). */
void orc_m2m(const double c[3], const double cp[3], int p, const cplx *M, cplx *Mp)
{
    cplx *R = malloc(sizeof(cplx) * nterms(p));
    double d[3] = {c[0] - cp[0], c[1] - cp[1], c[2] - cp[2]};
    orc_regular(d, p, R);
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) {
            cplx acc = 0.0;
            for (int k = 0; k <= n; ++k)
                for (int l = -k; l <= k; ++l) {
                    if (abs(m - l) > n - k)
                        continue;
                    acc += conj(R[hidx(k, l)]) * M[hidx(n - k, m - l)];
                }
            Mp[hidx(n, m)] += acc;
        }
    free(R);
}

/* M2L: multipole M about cs -> local expansion about ct (accumulates into L). */
void orc_m2l(const double cs[3], const double ct[3], int p, const cplx *M, cplx *L)
{
    cplx *Ih = malloc(sizeof(cplx) * nterms(2 * p));
    double d[3] = {ct[0] - cs[0], ct[1] - cs[1], ct[2] - cs[2]};
    orc_irregular(d, 2 * p, Ih);
    for (int j = 0; j <= p; ++j)
        for (int l = -j; l <= j; ++l) {
            cplx acc = 0.0;
            for (int n = 0; n <= p; ++n)
                for (int m = -n; m <= n; ++m)
                    acc += M[hidx(n, m)] * Ih[hidx(n + j, m - l)];
            L[hidx(j, l)] += (((j + l) & 1) ? -1.0 : 1.0) * acc;
        }
    free(Ih);
}

/* L2L: local expansion L about c -> L' about c' (accumulates into Lp). */
void orc_l2l(const double c[3], const double cp[3], int p, const cplx *L, cplx *Lp)
{
    cplx *R = malloc(sizeof(cplx) * nterms(p));
    double d[3] = {cp[0] - c[0], cp[1] - c[1], cp[2] - c[2]};
    orc_regular(d, p, R);
    for (int j = 0; j <= p; ++j)
        for (int l = -j; l <= j; ++l) {
            cplx acc = 0.0;
            for (int n = j; n <= p; ++n)
                for (int m = -n; m <= n; ++m) {
                    if (abs(m - l) > n - j)
                        continue;
                    acc += L[hidx(n, m)] * R[hidx(n - j, m - l)];
                }
            Lp[hidx(j, l)] += acc;
        }
    free(R);
}

/* L2P: potential and gradient at x from the local expansion L about c. */
void orc_l2p(const double c[3], int p, const cplx *L, const double x[3], double *phi, double g[3])
{
    cplx *R = malloc(sizeof(cplx) * nterms(p));
    double d[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
    orc_regular(d, p, R);
    cplx ph = 0.0, dz = 0.0, dplus = 0.0;
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) {
            ph += L[hidx(n, m)] * R[hidx(n, m)];
            if (n >= 1 && abs(m) <= n - 1)
                dz += L[hidx(n, m)] * R[hidx(n - 1, m)];
            if (n >= 1 && abs(m + 1) <= n - 1)
                dplus += L[hidx(n, m)] * R[hidx(n - 1, m + 1)];
        }
    *phi = creal(ph);
    g[0] = creal(dplus);
    g[1] = cimag(dplus);
    g[2] = creal(dz);
    free(R);
}

/* M2P: potential at x from the multipole M about c. */
double orc_m2p(const double c[3], int p, const cplx *M, const double x[3])
{
    cplx *Ih = malloc(sizeof(cplx) * nterms(p));
    double d[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
    orc_irregular(d, p, Ih);
    cplx acc = 0.0;
    for (int k = 0; k < nterms(p); ++k)
        acc += M[k] * Ih[k];
    free(Ih);
    return creal(acc);
}

/* P2L: local expansion about c of the n charges q at y (all |y - c| larger
 * than the evaluation radius), added to L. */
void orc_p2l(const double c[3], const double *y, const double *q, int64_t n, int p, cplx *L)
{
    cplx *Ih = malloc(sizeof(cplx) * nterms(p));
    for (int64_t j = 0; j < n; ++j) {
        double d[3] = {y[3 * j] - c[0], y[3 * j + 1] - c[1], y[3 * j + 2] - c[2]};
        orc_irregular(d, p, Ih);
        for (int k = 0; k < nterms(p); ++k)
            L[k] += q[j] * conj(Ih[k]);
    }
    free(Ih);
}

/* M2P with the gradient: phi and grad at x from the multipole M about c.
 * The derivatives of the irregular harmonics raise the degree by one. */
void orc_m2p_grad(const double c[3], int p, const cplx *M, const double x[3], double *phi,
                  double g[3])
{
    cplx *Ih = malloc(sizeof(cplx) * nterms(p + 1));
    double d[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
    orc_irregular(d, p + 1, Ih);
    cplx ph = 0.0, dz = 0.0, dplus = 0.0;
    for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) {
            ph += M[hidx(n, m)] * Ih[hidx(n, m)];
            dz -= M[hidx(n, m)] * Ih[hidx(n + 1, m)];
            dplus += M[hidx(n, m)] * Ih[hidx(n + 1, m + 1)];
        }
    *phi = creal(ph);
    g[0] = creal(dplus);
    g[1] = cimag(dplus);
    g[2] = creal(dz);
    free(Ih);
}

/* ------------------------------------------------------------------ */
/* Direct summation                                                    */
/* ------------------------------------------------------------------ */

/* Exact potential and gradient at the targets tidx[0..nt) (all N if tidx is NULL)
 * from all N sources; pairs at zero distance are skipped. */
void orc_direct(int64_t N, const double *x, const double *q, int64_t nt, const int64_t *tidx,
                double *phi, double *grad)
{
    if (!tidx)
        nt = N;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t a = 0; a < nt; ++a) {
        int64_t i = tidx ? tidx[a] : a;
        double ph = 0, gx = 0, gy = 0, gz = 0;
        for (int64_t j = 0; j < N; ++j) {
            double dx = x[3 * i] - x[3 * j], dy = x[3 * i + 1] - x[3 * j + 1],
                   dz = x[3 * i + 2] - x[3 * j + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0)
                continue;
            double r = sqrt(r2);
            double qr3 = q[j] / (r2 * r);
            ph += q[j] / r;
            gx -= qr3 * dx;
            gy -= qr3 * dy;
            gz -= qr3 * dz;
        }
        phi[a] = ph;
        grad[3 * a] = gx;
        grad[3 * a + 1] = gy;
        grad[3 * a + 2] = gz;
    }
}

/* ------------------------------------------------------------------ */
/* Morton keys (reading R1)                                            */
/* ------------------------------------------------------------------ */

static uint64_t spread3(uint64_t k)
{
    uint64_t out = 0;
    for (int b = 0; b < ORC_KBITS; ++b)
        out |= ((k >> b) & 1ULL) << (3 * b);
    return out;
}

static uint64_t compact3(uint64_t key)
{
    uint64_t out = 0;
    for (int b = 0; b < ORC_KBITS; ++b)
        out |= ((key >> (3 * b)) & 1ULL) << b;
    return out;
}

/* Box and keys for N points; returns 0, or 1 if a coordinate is not finite. */
int orc_morton_keys(int64_t N, const double *x, double lo[3], double *side_out, uint64_t *key)
{
    double hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = INFINITY;
        hi[a] = -INFINITY;
    }
    for (int64_t i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a) {
            double v = x[3 * i + a];
            if (!isfinite(v))
                return 1;
            if (v < lo[a])
                lo[a] = v;
            if (v > hi[a])
                hi[a] = v;
        }
    double side = 0.0;
    for (int a = 0; a < 3; ++a) {
        double ext = hi[a] - lo[a];
        if (ext > side)
            side = ext;
    }
    if (side == 0.0)
        side = 1.0;
    *side_out = side;
    const double s = 2097152.0 / side;
    for (int64_t i = 0; i < N; ++i) {
        uint64_t k[3];
        for (int a = 0; a < 3; ++a) {
            double t = x[3 * i + a] - lo[a];
            double f = floor(t * s);
            int64_t ki = (int64_t)f;
            if (ki > ORC_KMAX)
                ki = ORC_KMAX;
            k[a] = (uint64_t)ki;
        }
        key[i] = spread3(k[0]) | (spread3(k[1]) << 1) | (spread3(k[2]) << 2);
    }
    return 0;
}

typedef struct {
    uint64_t key;
    int64_t idx;
} keyidx;

static int cmp_keyidx(const void *a, const void *b)
{
    const keyidx *A = a, *B = b;
    if (A->key != B->key)
        return A->key < B->key ? -1 : 1;
    return A->idx < B->idx ? -1 : (A->idx > B->idx);
}

/* ------------------------------------------------------------------ */
/* The FMM solver state                                                */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t N;
    int p, ncrit, max_depth, leaf_first, split_variant;
    double theta;
    const unsigned char *sel; /* hybrid selection table (R9), NULL = plain FMM */
    double lo[3], side;
    double *x, *q;       /* sorted order */
    uint64_t *key;       /* sorted keys */
    int64_t *order;      /* order[i] = original index of sorted position i */
    /* cells (depth-first order) */
    int64_t ncells, cap;
    int *level;
    uint64_t *prefix; /* top 3*level bits of the key, right-aligned */
    int64_t *begin, *end, *child0, *parent;
    int *nchild;
    int depth;
    /* interaction lists */
    int64_t nm2l, np2p, cap_m2l, cap_p2p, nm2p, cap_m2p, np2l, cap_p2l;
    int64_t *m2l_t, *m2l_s, *p2p_t, *p2p_s, *m2p_t, *m2p_s, *p2l_t, *p2l_s;
    /* expansions */
    cplx *M, *L;
    int upward_done;
    /* results, sorted order */
    double *phi, *grad;
} orc_fmm;

static int64_t new_cell(orc_fmm *f)
{
    if (f->ncells == f->cap) {
        f->cap = f->cap ? 2 * f->cap : 1024;
        f->level = realloc(f->level, sizeof(int) * f->cap);
        f->prefix = realloc(f->prefix, sizeof(uint64_t) * f->cap);
        f->begin = realloc(f->begin, sizeof(int64_t) * f->cap);
        f->end = realloc(f->end, sizeof(int64_t) * f->cap);
        f->child0 = realloc(f->child0, sizeof(int64_t) * f->cap);
        f->parent = realloc(f->parent, sizeof(int64_t) * f->cap);
        f->nchild = realloc(f->nchild, sizeof(int) * f->cap);
    }
    return f->ncells++;
}

/* Recursive cell construction (reading R2).  Children are created
 * contiguously right after the parent's sibling block is known. */
static void build_cell(orc_fmm *f, int64_t c)
{
    int l = f->level[c];
    if (l > f->depth)
        f->depth = l;
    int64_t b = f->begin[c], e = f->end[c];
    f->child0[c] = -1;
    f->nchild[c] = 0;
    if (!(e - b > f->ncrit && l < f->max_depth))
        return;
    int shift = 3 * (ORC_KBITS - l - 1);
    int64_t start[8], stop[8];
    int64_t i = b;
    for (int o = 0; o < 8; ++o) {
        start[o] = i;
        while (i < e && (int)((f->key[i] >> shift) & 7ULL) == o)
            ++i;
        stop[o] = i;
    }
    int64_t first = -1;
    int cnt = 0;
    for (int o = 0; o < 8; ++o) {
        if (stop[o] == start[o])
            continue;
        int64_t ch = new_cell(f);
        if (first < 0)
            first = ch;
        ++cnt;
        f->level[ch] = l + 1;
        f->prefix[ch] = (f->prefix[c] << 3) | (uint64_t)o;
        f->begin[ch] = start[o];
        f->end[ch] = stop[o];
        f->parent[ch] = c;
    }
    f->child0[c] = first;
    f->nchild[c] = cnt;
    for (int k = 0; k < cnt; ++k)
        build_cell(f, first + k);
}

/* Integer geometry: centre in units of side/2^22 and half-side (= radius). */
static void cell_geom_int(const orc_fmm *f, int64_t c, int64_t C[3], int64_t *r)
{
    int l = f->level[c];
    uint64_t pre = f->prefix[c];
    int64_t h = 1LL << (ORC_KBITS - l);
    for (int a = 0; a < 3; ++a) {
        int64_t k = (int64_t)compact3(pre >> a);
        C[a] = (2 * k + 1) * h;
    }
    *r = h;
}

/* Real centre of a cell. */
static void cell_centre(const orc_fmm *f, int64_t c, double cen[3])
{
    int l = f->level[c];
    uint64_t pre = f->prefix[c];
    double half = f->side / (double)(1LL << (l + 1));
    for (int a = 0; a < 3; ++a) {
        int64_t k = (int64_t)compact3(pre >> a);
        cen[a] = f->lo[a] + (double)(2 * k + 1) * half;
    }
}

/* MAC (reading R3). */
static int mac_accept(const orc_fmm *f, int64_t T, int64_t S)
{
    int64_t Ct[3], Cs[3], rt, rs;
    cell_geom_int(f, T, Ct, &rt);
    cell_geom_int(f, S, Cs, &rs);
    int64_t R2 = 0;
    for (int a = 0; a < 3; ++a)
        R2 += (Ct[a] - Cs[a]) * (Ct[a] - Cs[a]);
    if (R2 == 0)
        return 0;
    int64_t rsum = rt + rs;
    return (double)(rsum * rsum) <= (f->theta * f->theta) * (double)R2;
}

static void push_pair(int64_t **t, int64_t **s, int64_t *n, int64_t *cap, int64_t a, int64_t b)
{
    if (*n == *cap) {
        *cap = *cap ? 2 * *cap : 4096;
        *t = realloc(*t, sizeof(int64_t) * *cap);
        *s = realloc(*s, sizeof(int64_t) * *cap);
    }
    (*t)[*n] = a;
    (*s)[*n] = b;
    ++*n;
}

typedef struct {
    int64_t *t, *s;
    int64_t n, cap;
} pairstack;

static int is_leaf(const orc_fmm *f, int64_t c) { return f->nchild[c] == 0; }

/* Count bucket of reading R9. */
int orc_count_bucket(int64_t n)
{
    int e = 0;
    while ((n >> (e + 1)) > 0)
        ++e;
    if (e < 2)
        return (int)(n - 1);
    return 3 + 4 * (e - 2) + (int)((n >> (e - 2)) & 3);
}

/* Interaction type of an accepted pair (R9): 0 = cell-cell, 1 = particle-particle,
 * 2 = cell-particle. */
static int choose_kind(const orc_fmm *f, int64_t T, int64_t S)
{
    if (!f->sel)
        return 0;
    int bt = orc_count_bucket(f->end[T] - f->begin[T]);
    int bs = orc_count_bucket(f->end[S] - f->begin[S]);
    return f->sel[bt * ORC_SEL_NB + bs];
}

/* interact(T,S) of reading R4. */
static void interact(orc_fmm *f, pairstack *st, int64_t T, int64_t S)
{
    if (f->leaf_first) {
        if (is_leaf(f, T) && is_leaf(f, S))
            push_pair(&f->p2p_t, &f->p2p_s, &f->np2p, &f->cap_p2p, T, S);
        else if (mac_accept(f, T, S))
            push_pair(&f->m2l_t, &f->m2l_s, &f->nm2l, &f->cap_m2l, T, S);
        else
            push_pair(&st->t, &st->s, &st->n, &st->cap, T, S);
        return;
    }
    if (mac_accept(f, T, S)) {
        int kind = choose_kind(f, T, S);
        if (kind == 1)
            push_pair(&f->p2p_t, &f->p2p_s, &f->np2p, &f->cap_p2p, T, S);
        else if (kind == 2)
            push_pair(&f->m2p_t, &f->m2p_s, &f->nm2p, &f->cap_m2p, T, S);
        else if (kind == 3)
            push_pair(&f->p2l_t, &f->p2l_s, &f->np2l, &f->cap_p2l, T, S);
        else
            push_pair(&f->m2l_t, &f->m2l_s, &f->nm2l, &f->cap_m2l, T, S);
    } else if (is_leaf(f, T) && is_leaf(f, S))
        push_pair(&f->p2p_t, &f->p2p_s, &f->np2p, &f->cap_p2p, T, S);
    else
        push_pair(&st->t, &st->s, &st->n, &st->cap, T, S);
}

/* Dual tree traversal with a LIFO stack of (target, source) pairs, seeded with
 * the pair of roots (section "Dual tree traversal"). */
static void traverse(orc_fmm *f)
{
    pairstack st = {0};
    interact(f, &st, 0, 0);
    while (st.n > 0) {
        --st.n;
        int64_t T = st.t[st.n], S = st.s[st.n];
        int split_source;
        if (f->split_variant == ORC_SPLIT_SMALLER) {
            /* planted mistake (tests only): split the smaller cell */
            if (is_leaf(f, T))
                split_source = 1;
            else if (f->level[S] > f->level[T] && !is_leaf(f, S))
                split_source = 1;
            else
                split_source = 0;
        } else if (f->split_variant == ORC_SPLIT_SOURCE_ON_TIE) {
            /* planted mistake (tests only): the source on a tie */
            if (is_leaf(f, T))
                split_source = 1;
            else if (f->level[S] <= f->level[T] && !is_leaf(f, S))
                split_source = 1;
            else
                split_source = 0;
        } else if (is_leaf(f, T))
            split_source = 1;
        else if (f->level[S] < f->level[T] && !is_leaf(f, S))
            split_source = 1;
        else
            split_source = 0;
        if (split_source) {
            for (int k = 0; k < f->nchild[S]; ++k)
                interact(f, &st, T, f->child0[S] + k);
        } else {
            for (int k = 0; k < f->nchild[T]; ++k)
                interact(f, &st, f->child0[T] + k, S);
        }
    }
    free(st.t);
    free(st.s);
}

/* Build keys, sorted order, tree and interaction lists.  Returns 0 on success,
 * 1 for a non-finite coordinate. */
orc_fmm *orc_fmm_create(int64_t N, const double *xyz, const double *q, int p, double theta,
                        int ncrit, int max_depth, int flags, const unsigned char *sel,
                        int *status)
{
    orc_fmm *f = calloc(1, sizeof(orc_fmm));
    f->sel = sel; /* only read during the traversal below */
    f->N = N;
    f->p = p;
    f->theta = theta;
    f->ncrit = ncrit;
    f->max_depth = max_depth;
    f->leaf_first = flags & ORC_LEAF_FIRST;
    f->split_variant = flags & (ORC_SPLIT_SMALLER | ORC_SPLIT_SOURCE_ON_TIE);
    uint64_t *key = malloc(sizeof(uint64_t) * N);
    if (orc_morton_keys(N, xyz, f->lo, &f->side, key)) {
        free(key);
        free(f);
        *status = 1;
        return NULL;
    }
    keyidx *ki = malloc(sizeof(keyidx) * N);
    for (int64_t i = 0; i < N; ++i) {
        ki[i].key = key[i];
        ki[i].idx = i;
    }
    qsort(ki, N, sizeof(keyidx), cmp_keyidx);
    f->key = malloc(sizeof(uint64_t) * N);
    f->order = malloc(sizeof(int64_t) * N);
    f->x = malloc(sizeof(double) * 3 * N);
    f->q = malloc(sizeof(double) * N);
    for (int64_t i = 0; i < N; ++i) {
        f->key[i] = ki[i].key;
        f->order[i] = ki[i].idx;
        for (int a = 0; a < 3; ++a)
            f->x[3 * i + a] = xyz[3 * ki[i].idx + a];
        f->q[i] = q[ki[i].idx];
    }
    free(ki);
    free(key);
    int64_t root = new_cell(f);
    f->level[root] = 0;
    f->prefix[root] = 0;
    f->begin[root] = 0;
    f->end[root] = N;
    f->parent[root] = -1;
    build_cell(f, root);
    traverse(f);
    f->sel = NULL;
    *status = 0;
    return f;
}

/* P2M at leaves, then M2M children -> parent.  Cells are in depth-first order,
 * so every child has a larger index than its parent: a reverse sweep visits
 * children before parents. */
void orc_fmm_upward(orc_fmm *f)
{
    if (f->upward_done)
        return;
    const int P2 = nterms(f->p);
    f->M = calloc((size_t)f->ncells * P2, sizeof(cplx));
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t c = 0; c < f->ncells; ++c) {
        if (!is_leaf(f, c))
            continue;
        double cen[3];
        cell_centre(f, c, cen);
        orc_p2m(cen, f->x + 3 * f->begin[c], f->q + f->begin[c], f->end[c] - f->begin[c], f->p,
                f->M + (size_t)c * P2);
    }
    for (int64_t c = f->ncells - 1; c >= 0; --c) {
        if (is_leaf(f, c))
            continue;
        double cp[3];
        cell_centre(f, c, cp);
        for (int k = 0; k < f->nchild[c]; ++k) {
            int64_t ch = f->child0[c] + k;
            double cc[3];
            cell_centre(f, ch, cc);
            orc_m2m(cc, cp, f->p, f->M + (size_t)ch * P2, f->M + (size_t)c * P2);
        }
    }
    f->upward_done = 1;
}

/* CSR of a pair list by target cell (stable: keeps list order per target). */
static void csr_by_target(int64_t ncells, int64_t npairs, const int64_t *t, int64_t **off_out,
                          int64_t **idx_out)
{
    int64_t *off = calloc(ncells + 1, sizeof(int64_t));
    int64_t *idx = malloc(sizeof(int64_t) * (npairs ? npairs : 1));
    for (int64_t k = 0; k < npairs; ++k)
        off[t[k] + 1]++;
    for (int64_t c = 0; c < ncells; ++c)
        off[c + 1] += off[c];
    int64_t *pos = malloc(sizeof(int64_t) * (ncells + 1));
    memcpy(pos, off, sizeof(int64_t) * (ncells + 1));
    for (int64_t k = 0; k < npairs; ++k)
        idx[pos[t[k]]++] = k;
    free(pos);
    *off_out = off;
    *idx_out = idx;
}

/* Near field for the particles of target leaf T: direct sum over the P2P lists
 * of T and of its ancestors (a P2P pair of reading R9 may have a non-leaf target,
 * and then acts on every particle below it). */
static void p2p_leaf(const orc_fmm *f, int64_t T, const int64_t *off, const int64_t *idx,
                     double *phi, double *grad, int64_t obase)
{
    for (int64_t i = f->begin[T]; i < f->end[T]; ++i) {
        double ph = 0, gx = 0, gy = 0, gz = 0;
        for (int64_t A = T; A >= 0; A = f->parent[A]) {
            for (int64_t k = off[A]; k < off[A + 1]; ++k) {
                int64_t S = f->p2p_s[idx[k]];
                for (int64_t j = f->begin[S]; j < f->end[S]; ++j) {
                    double dx = f->x[3 * i] - f->x[3 * j], dy = f->x[3 * i + 1] - f->x[3 * j + 1],
                           dz = f->x[3 * i + 2] - f->x[3 * j + 2];
                    double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 == 0.0)
                        continue;
                    double r = sqrt(r2);
                    double qr3 = f->q[j] / (r2 * r);
                    ph += f->q[j] / r;
                    gx -= qr3 * dx;
                    gy -= qr3 * dy;
                    gz -= qr3 * dz;
                }
            }
        }
        phi[i - obase] += ph;
        grad[3 * (i - obase)] += gx;
        grad[3 * (i - obase) + 1] += gy;
        grad[3 * (i - obase) + 2] += gz;
    }
}

/* Cell-particle far field for the particles of leaf T: the multipoles of the
 * M2P sources of T and of its ancestors (reading R9). */
static void m2p_leaf(const orc_fmm *f, int64_t T, const int64_t *off, const int64_t *idx,
                     double *phi, double *grad, int64_t obase)
{
    const int P2 = nterms(f->p);
    for (int64_t A = T; A >= 0; A = f->parent[A]) {
        for (int64_t k = off[A]; k < off[A + 1]; ++k) {
            int64_t S = f->m2p_s[idx[k]];
            double cs[3];
            cell_centre(f, S, cs);
            for (int64_t i = f->begin[T]; i < f->end[T]; ++i) {
                double ph, g[3];
                orc_m2p_grad(cs, f->p, f->M + (size_t)S * P2, f->x + 3 * i, &ph, g);
                phi[i - obase] += ph;
                grad[3 * (i - obase)] += g[0];
                grad[3 * (i - obase) + 1] += g[1];
                grad[3 * (i - obase) + 2] += g[2];
            }
        }
    }
}

/* Far field for the particles of leaf T from its local expansion. */
static void l2p_leaf(const orc_fmm *f, int64_t T, const cplx *L, double *phi, double *grad,
                     int64_t obase)
{
    double cen[3];
    cell_centre(f, T, cen);
    for (int64_t i = f->begin[T]; i < f->end[T]; ++i) {
        double ph, g[3];
        orc_l2p(cen, f->p, L, f->x + 3 * i, &ph, g);
        phi[i - obase] += ph;
        grad[3 * (i - obase)] += g[0];
        grad[3 * (i - obase) + 1] += g[1];
        grad[3 * (i - obase) + 2] += g[2];
    }
}

/* Full evaluation: M2L over the cell-cell list, L2L parent -> child (forward
 * sweep: parents precede children), L2P at leaves, P2P over the leaf list.
 * Results are stored in sorted order in f->phi / f->grad. */
void orc_fmm_evaluate(orc_fmm *f)
{
    orc_fmm_upward(f);
    const int P2 = nterms(f->p);
    free(f->L);
    f->L = calloc((size_t)f->ncells * P2, sizeof(cplx));
    int64_t *off, *idx;
    csr_by_target(f->ncells, f->nm2l, f->m2l_t, &off, &idx);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t T = 0; T < f->ncells; ++T) {
        double ct[3];
        cell_centre(f, T, ct);
        for (int64_t k = off[T]; k < off[T + 1]; ++k) {
            int64_t S = f->m2l_s[idx[k]];
            double cs[3];
            cell_centre(f, S, cs);
            orc_m2l(cs, ct, f->p, f->M + (size_t)S * P2, f->L + (size_t)T * P2);
        }
    }
    free(off);
    free(idx);
    /* particle-cell pairs of the selection table (R9), before L2L */
    for (int64_t k = 0; k < f->np2l; ++k) {
        int64_t T = f->p2l_t[k], S = f->p2l_s[k];
        double ct[3];
        cell_centre(f, T, ct);
        orc_p2l(ct, f->x + 3 * f->begin[S], f->q + f->begin[S], f->end[S] - f->begin[S], f->p,
                f->L + (size_t)T * P2);
    }
    for (int64_t c = 0; c < f->ncells; ++c) {
        if (f->parent[c] < 0)
            continue;
        double cp[3], cc[3];
        cell_centre(f, f->parent[c], cp);
        cell_centre(f, c, cc);
        orc_l2l(cp, cc, f->p, f->L + (size_t)f->parent[c] * P2, f->L + (size_t)c * P2);
    }
    free(f->phi);
    free(f->grad);
    f->phi = calloc(f->N, sizeof(double));
    f->grad = calloc(3 * f->N, sizeof(double));
    csr_by_target(f->ncells, f->np2p, f->p2p_t, &off, &idx);
    int64_t *qoff, *qidx;
    csr_by_target(f->ncells, f->nm2p, f->m2p_t, &qoff, &qidx);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t T = 0; T < f->ncells; ++T) {
        if (!is_leaf(f, T))
            continue;
        l2p_leaf(f, T, f->L + (size_t)T * P2, f->phi, f->grad, 0);
        m2p_leaf(f, T, qoff, qidx, f->phi, f->grad, 0);
        p2p_leaf(f, T, off, idx, f->phi, f->grad, 0);
    }
    free(off);
    free(idx);
    free(qoff);
    free(qidx);
}

/* Evaluation restricted to the particles of the given leaves: the local
 * expansion of each leaf is accumulated along its ancestor chain (M2L into each
 * ancestor, L2L down the chain), then L2P + P2P.  Outputs are written for the
 * particles of leaves[0..nl) in that order (sorted positions within a leaf). */
void orc_fmm_evaluate_leaves(orc_fmm *f, int64_t nl, const int64_t *leaves, double *phi,
                             double *grad, int64_t *positions)
{
    orc_fmm_upward(f);
    const int P2 = nterms(f->p);
    int64_t *moff, *midx, *poff, *pidx, *qoff, *qidx, *loff, *lidx;
    csr_by_target(f->ncells, f->np2l, f->p2l_t, &loff, &lidx);
    csr_by_target(f->ncells, f->nm2l, f->m2l_t, &moff, &midx);
    csr_by_target(f->ncells, f->np2p, f->p2p_t, &poff, &pidx);
    csr_by_target(f->ncells, f->nm2p, f->m2p_t, &qoff, &qidx);
    int64_t *base = malloc(sizeof(int64_t) * (nl + 1));
    base[0] = 0;
    for (int64_t a = 0; a < nl; ++a)
        base[a + 1] = base[a] + (f->end[leaves[a]] - f->begin[leaves[a]]);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t a = 0; a < nl; ++a) {
        int64_t T = leaves[a];
        int64_t chain[64];
        int depth = 0;
        for (int64_t c = T; c >= 0; c = f->parent[c])
            chain[depth++] = c;
        cplx *Lc = calloc(P2, sizeof(cplx));
        cplx *Ln = calloc(P2, sizeof(cplx));
        for (int d = depth - 1; d >= 0; --d) {
            int64_t c = chain[d];
            double cc[3];
            cell_centre(f, c, cc);
            memset(Ln, 0, sizeof(cplx) * P2);
            if (d < depth - 1) {
                double cp[3];
                cell_centre(f, chain[d + 1], cp);
                orc_l2l(cp, cc, f->p, Lc, Ln);
            }
            for (int64_t k = moff[c]; k < moff[c + 1]; ++k) {
                int64_t S = f->m2l_s[midx[k]];
                double cs[3];
                cell_centre(f, S, cs);
                orc_m2l(cs, cc, f->p, f->M + (size_t)S * P2, Ln);
            }
            for (int64_t k = loff[c]; k < loff[c + 1]; ++k) {
                int64_t S = f->p2l_s[lidx[k]];
                orc_p2l(cc, f->x + 3 * f->begin[S], f->q + f->begin[S], f->end[S] - f->begin[S], f->p, Ln);
            }
            memcpy(Lc, Ln, sizeof(cplx) * P2);
        }
        int64_t n = f->end[T] - f->begin[T];
        double *ph = phi + base[a], *gr = grad + 3 * base[a];
        for (int64_t i = 0; i < n; ++i) {
            ph[i] = 0.0;
            gr[3 * i] = gr[3 * i + 1] = gr[3 * i + 2] = 0.0;
            positions[base[a] + i] = f->begin[T] + i;
        }
        l2p_leaf(f, T, Lc, ph, gr, f->begin[T]);
        m2p_leaf(f, T, qoff, qidx, ph, gr, f->begin[T]);
        p2p_leaf(f, T, poff, pidx, ph, gr, f->begin[T]);
        free(Lc);
        free(Ln);
    }
    free(base);
    free(moff);
    free(midx);
    free(poff);
    free(pidx);
    free(qoff);
    free(qidx);
    free(loff);
    free(lidx);
}

void orc_fmm_destroy(orc_fmm *f)
{
    if (!f)
        return;
    free(f->x);
    free(f->q);
    free(f->key);
    free(f->order);
    free(f->level);
    free(f->prefix);
    free(f->begin);
    free(f->end);
    free(f->child0);
    free(f->parent);
    free(f->nchild);
    free(f->m2l_t);
    free(f->m2l_s);
    free(f->p2p_t);
    free(f->p2p_s);
    free(f->m2p_t);
    free(f->m2p_s);
    free(f->p2l_t);
    free(f->p2l_s);
    free(f->M);
    free(f->L);
    free(f->phi);
    free(f->grad);
    free(f);
}

/* ------------------------------------------------------------------ */
/* Accessors for the Python wrapper                                    */
/* ------------------------------------------------------------------ */

void orc_fmm_p2l_list(const orc_fmm *f, int64_t *n, int64_t *t, int64_t *s)
{
    *n = f->np2l;
    if (t)
        memcpy(t, f->p2l_t, sizeof(int64_t) * f->np2l);
    if (s)
        memcpy(s, f->p2l_s, sizeof(int64_t) * f->np2l);
}

void orc_fmm_m2p_list(const orc_fmm *f, int64_t *n, int64_t *t, int64_t *s)
{
    *n = f->nm2p;
    if (t)
        memcpy(t, f->m2p_t, sizeof(int64_t) * f->nm2p);
    if (s)
        memcpy(s, f->m2p_s, sizeof(int64_t) * f->nm2p);
}

void orc_fmm_sizes(const orc_fmm *f, int64_t out[6])
{
    out[0] = f->N;
    out[1] = f->ncells;
    out[2] = f->nm2l;
    out[3] = f->np2p;
    out[4] = f->depth;
    int64_t nleaves = 0;
    for (int64_t c = 0; c < f->ncells; ++c)
        nleaves += is_leaf(f, c);
    out[5] = nleaves;
}

void orc_fmm_box(const orc_fmm *f, double out[4])
{
    out[0] = f->lo[0];
    out[1] = f->lo[1];
    out[2] = f->lo[2];
    out[3] = f->side;
}

void orc_fmm_sorted(const orc_fmm *f, uint64_t *key, int64_t *order)
{
    memcpy(key, f->key, sizeof(uint64_t) * f->N);
    memcpy(order, f->order, sizeof(int64_t) * f->N);
}

void orc_fmm_cells(const orc_fmm *f, int64_t *level, uint64_t *prefix, int64_t *begin,
                   int64_t *end, int64_t *parent, int64_t *nchild)
{
    for (int64_t c = 0; c < f->ncells; ++c) {
        level[c] = f->level[c];
        prefix[c] = f->prefix[c];
        begin[c] = f->begin[c];
        end[c] = f->end[c];
        parent[c] = f->parent[c];
        nchild[c] = f->nchild[c];
    }
}

void orc_fmm_lists(const orc_fmm *f, int64_t *m2l_t, int64_t *m2l_s, int64_t *p2p_t,
                   int64_t *p2p_s)
{
    memcpy(m2l_t, f->m2l_t, sizeof(int64_t) * f->nm2l);
    memcpy(m2l_s, f->m2l_s, sizeof(int64_t) * f->nm2l);
    memcpy(p2p_t, f->p2p_t, sizeof(int64_t) * f->np2p);
    memcpy(p2p_s, f->p2p_s, sizeof(int64_t) * f->np2p);
}

/* Results in ORIGINAL particle order. */
void orc_fmm_results(const orc_fmm *f, double *phi, double *grad)
{
    for (int64_t i = 0; i < f->N; ++i) {
        int64_t o = f->order[i];
        phi[o] = f->phi[i];
        for (int a = 0; a < 3; ++a)
            grad[3 * o + a] = f->grad[3 * i + a];
    }
}

/* Multipole / local coefficients of one cell (all signed m, complex). */
void orc_fmm_expansion(const orc_fmm *f, int which, int64_t c, double *re, double *im)
{
    const int P2 = nterms(f->p);
    const cplx *E = which == 0 ? f->M : f->L;
    for (int k = 0; k < P2; ++k) {
        re[k] = E ? creal(E[(size_t)c * P2 + k]) : 0.0;
        im[k] = E ? cimag(E[(size_t)c * P2 + k]) : 0.0;
    }
}

void orc_fmm_centre(const orc_fmm *f, int64_t c, double cen[3]) { cell_centre(f, c, cen); }

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the parallel loops from now on (n >= 1); for the timed baselines. */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Thin complex-array wrappers for the operator pins (arrays of re/im pairs). */
void orc_regular_ri(const double x[3], int p, double *ri)
{
    orc_regular(x, p, (cplx *)ri);
}
void orc_irregular_ri(const double x[3], int p, double *ri)
{
    orc_irregular(x, p, (cplx *)ri);
}
void orc_p2m_ri(const double c[3], const double *y, const double *q, int64_t n, int p, double *M)
{
    orc_p2m(c, y, q, n, p, (cplx *)M);
}
void orc_m2m_ri(const double c[3], const double cp[3], int p, const double *M, double *Mp)
{
    orc_m2m(c, cp, p, (const cplx *)M, (cplx *)Mp);
}
void orc_m2l_ri(const double cs[3], const double ct[3], int p, const double *M, double *L)
{
    orc_m2l(cs, ct, p, (const cplx *)M, (cplx *)L);
}
void orc_l2l_ri(const double c[3], const double cp[3], int p, const double *L, double *Lp)
{
    orc_l2l(c, cp, p, (const cplx *)L, (cplx *)Lp);
}
void orc_l2p_ri(const double c[3], int p, const double *L, const double x[3], double *out4)
{
    orc_l2p(c, p, (const cplx *)L, x, &out4[0], &out4[1]);
}
void orc_p2l_ri(const double c[3], const double *y, const double *q, int64_t n, int p, double *L)
{
    orc_p2l(c, y, q, n, p, (cplx *)L);
}

void orc_m2p_grad_ri(const double c[3], int p, const double *M, const double x[3], double *out4)
{
    orc_m2p_grad(c, p, (const cplx *)M, x, out4, out4 + 1);
}

double orc_m2p_ri(const double c[3], int p, const double *M, const double x[3])
{
    return orc_m2p(c, p, (const cplx *)M, x);
}
