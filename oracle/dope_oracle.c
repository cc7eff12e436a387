/*
 * DOPE oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, CPU implementation of what the DOPE ADMM hot path computes
 * (Dolz, Ben Ayed, Desrosiers, "DOPE: Distributed Optimization for Pairwise
 * Energies", arXiv 1704.03116).  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load it.  The CUDA library
 * never links, includes or calls anything here, and nothing here comes from
 * the CUDA library.
 *
 * Floating point: every double operation is a single IEEE round-to-nearest
 * operation in the order written (the build passes -ffp-contract=off and no
 * fast-math), because several of these doubles decide integers (Eq. 8's
 * capacities are rounded to int64).
 *
 * Contents
 *   orc_quantise        instance canonicalisation of Eq. 1 (fixed point x1024)
 *   orc_energy          Eq. 1 / Eq. 3 on the quantised instance, int64
 *   orc_bk_mincut       Boykov-Kolmogorov max-flow (the serial solver the paper
 *                       uses for Eq. 8 and for sGC), written from the published
 *                       algorithm: two search trees, growth / augmentation /
 *                       adoption, with the distance + timestamp heuristic; the
 *                       canonical (pointwise-minimal) sink side is taken by a
 *                       backward residual BFS from t
 *   orc_bruteforce      enumeration of all 2^n labelings (n <= 24), any sign
 *   orc_shifted_caps    Eq. 8 unary of every block (Q = I), x1024, rounded
 *   orc_block_cuts      Eq. 8 solved exactly per block ("in parallel", Alg. 1)
 *   orc_update          Eq. 10 (y) and Eq. 11 (a) for Q = I, per-block ||yhat_k - S_k y||^2
 *   orc_admm            Algorithm 1 end to end
 *   orc_global_mincut   the whole-image serial graph cut (sGC) of Section 3
 *
 * Notation follows the paper: u (unary), w (pairwise), lambda, y (relaxed
 * global labels), yhat (block labels), a (scaled multipliers), mu.
 * For the non-overlapping partition (Q = I) Theorem 1 gives, for pixel i in
 * block b(i) with cross-block neighbours X(i) = { j in N(i) : b(j) != b(i) }:
 *   (C_k + R_k S_k) y  at i  =  sum_{j in X(i)} w_ij (y_i - y_j)
 * which is what orc_shifted_caps and orc_update evaluate (the literal matrix
 * form of Theorem 1 lives in oracle/theorem1.py and pins this).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Grid geometry                                                            */
/* ------------------------------------------------------------------------ */

/* Forward neighbour offsets (dz, dy, dx) in weight-layout order.
 * 2-D grids are stored with D = 1.  Direction k < d/2 is forward offset k,
 * direction k >= d/2 is the backward offset k - d/2. */
static const int OFF4[2][3] = {{0, 0, 1}, {0, 1, 0}};
static const int OFF8[4][3] = {{0, 0, 1}, {0, 1, 0}, {0, 1, 1}, {0, 1, -1}};
static const int OFF6[3][3] = {{0, 0, 1}, {0, 1, 0}, {1, 0, 0}};

/* Larger kernels (Section 3: kernel sizes 5, 7, 9; square in 2-D, spherical in
 * 3-D).  Forward offsets of radius r, in this order: dz = 0..r, dy = -r..r,
 * dx = -r..r, keeping the offsets that are lexicographically positive
 * (dz > 0, or dz = 0 and dy > 0, or dz = dy = 0 and dx > 0) and inside the
 * kernel (2-D: |dy|, |dx| <= r with dz = 0; 3-D: dz^2 + dy^2 + dx^2 <= r^2).
 * conn = number of neighbours: 2-D 24 / 48 / 80 (r = 2, 3, 4), 3-D 32 (r = 2). */
static int OFFK[128][3];
static int offk_conn = 0;

static int big_kernel(int conn, int *r, int *is3d)
{
    switch (conn) {
        case 24: *r = 2; *is3d = 0; return 1;
        case 48: *r = 3; *is3d = 0; return 1;
        case 80: *r = 4; *is3d = 0; return 1;
        case 32: *r = 2; *is3d = 1; return 1;
        default: return 0;
    }
}

static const int (*big_offsets(int conn))[3]
{
    int r, is3d, n = 0;
    if (!big_kernel(conn, &r, &is3d)) return NULL;
    if (offk_conn == conn) return (const int (*)[3])OFFK;
    for (int dz = 0; dz <= (is3d ? r : 0); dz++)
        for (int dy = -r; dy <= r; dy++)
            for (int dx = -r; dx <= r; dx++) {
                int pos = dz > 0 || (dz == 0 && dy > 0) || (dz == 0 && dy == 0 && dx > 0);
                int in = is3d ? (dz * dz + dy * dy + dx * dx <= r * r) : 1;
                if (!pos || !in) continue;
                OFFK[n][0] = dz; OFFK[n][1] = dy; OFFK[n][2] = dx;
                n++;
            }
    offk_conn = conn;
    return (const int (*)[3])OFFK;
}

typedef struct {
    int64_t D, H, W;      /* grid extent, D = 1 for 2-D */
    int conn;             /* 4, 8 (2-D) or 6 (3-D) */
    int bd, bh, bw;       /* block shape, bd = 1 for 2-D */
    int nh;               /* number of forward offsets = conn / 2 */
    const int (*off)[3];
} grid_t;

static int grid_init(grid_t *g, const int64_t *dims, int conn, const int *block)
{
    g->D = dims[0]; g->H = dims[1]; g->W = dims[2];
    g->conn = conn;
    g->bd = block[0]; g->bh = block[1]; g->bw = block[2];
    if (conn == 4) { g->off = OFF4; g->nh = 2; }
    else if (conn == 8) { g->off = OFF8; g->nh = 4; }
    else if (conn == 6) { g->off = OFF6; g->nh = 3; }
    else if (big_offsets(conn)) { g->off = big_offsets(conn); g->nh = conn / 2; }
    else return -1;
    if (g->D <= 0 || g->H <= 0 || g->W <= 0) return -1;
    if (g->bd <= 0 || g->bh <= 0 || g->bw <= 0) return -1;
    if (g->D % g->bd || g->H % g->bh || g->W % g->bw) return -1;
    return 0;
}

static inline int64_t g_n(const grid_t *g) { return g->D * g->H * g->W; }

/* Neighbour of pixel (z,y,x) along direction k, or -1 outside the grid. */
static inline int64_t g_nbr(const grid_t *g, int64_t z, int64_t y, int64_t x, int k,
                            int64_t *nz, int64_t *ny, int64_t *nx)
{
    int s = (k < g->nh) ? 1 : -1;
    int o = (k < g->nh) ? k : k - g->nh;
    int64_t zz = z + s * g->off[o][0], yy = y + s * g->off[o][1], xx = x + s * g->off[o][2];
    if (zz < 0 || zz >= g->D || yy < 0 || yy >= g->H || xx < 0 || xx >= g->W) return -1;
    *nz = zz; *ny = yy; *nx = xx;
    return (zz * g->H + yy) * g->W + xx;
}

/* Weight of the undirected edge between pixel i and its neighbour j along
 * direction k: forward edges are stored at i, backward ones at j. */
static inline int64_t g_wt(const grid_t *g, const int64_t *Wl, int64_t i, int64_t j, int k)
{
    int64_t n = g_n(g);
    if (k < g->nh) return Wl[(int64_t)k * n + i];
    return Wl[(int64_t)(k - g->nh) * n + j];
}

static inline int64_t g_block_of(const grid_t *g, int64_t z, int64_t y, int64_t x)
{
    int64_t nby = g->H / g->bh, nbx = g->W / g->bw;
    return ((z / g->bd) * nby + (y / g->bh)) * nbx + (x / g->bw);
}

static inline int64_t g_nblocks(const grid_t *g)
{
    return (g->D / g->bd) * (g->H / g->bh) * (g->W / g->bw);
}

/* Global pixel index of local node l of block k (block-local order is
 * row-major over (z, y, x) inside the block). */
static inline int64_t g_block_pixel(const grid_t *g, int64_t k, int l,
                                    int64_t *pz, int64_t *py, int64_t *px)
{
    int64_t nby = g->H / g->bh, nbx = g->W / g->bw;
    int64_t kz = k / (nby * nbx), ky = (k / nbx) % nby, kx = k % nbx;
    int lz = l / (g->bh * g->bw), ly = (l / g->bw) % g->bh, lx = l % g->bw;
    int64_t z = kz * g->bd + lz, y = ky * g->bh + ly, x = kx * g->bw + lx;
    *pz = z; *py = y; *px = x;
    return (z * g->H + y) * g->W + x;
}

/* ------------------------------------------------------------------------ */
/* Instance canonicalisation (Eq. 1, Eq. 2)                                 */
/* ------------------------------------------------------------------------ */

/* U_i = rne(1024 u_i), Wl_ij = rne(lambda * wq_ij); wq is already x1024.
 * Returns 0, or -2 if a weight is negative (not submodular, footnote on
 * submodularity in Section 1), -3 if a weight toward a pixel outside the
 * grid is non-zero. */
static int quantise_impl(const int64_t *dims, int conn, const int *block, const float *u,
                         const int32_t *wq, double lambda, int64_t *U, int64_t *Wl, int allow_negative);

int orc_quantise(const int64_t *dims, int conn, const int *block,
                 const float *u, const int32_t *wq, double lambda,
                 int64_t *U, int64_t *Wl)
{
    return quantise_impl(dims, conn, block, u, wq, lambda, U, Wl, 0);
}

/* The same with weights of any sign (non-submodular instances, Section 3.4). */
int orc_quantise_signed(const int64_t *dims, int conn, const int *block,
                        const float *u, const int32_t *wq, double lambda,
                        int64_t *U, int64_t *Wl)
{
    return quantise_impl(dims, conn, block, u, wq, lambda, U, Wl, 1);
}

static int quantise_impl(const int64_t *dims, int conn, const int *block, const float *u,
                         const int32_t *wq, double lambda, int64_t *U, int64_t *Wl, int allow_negative)
{
    grid_t g;
    if (grid_init(&g, dims, conn, block)) return -1;
    int64_t n = g_n(&g);
    for (int64_t i = 0; i < n; i++) U[i] = llrint(1024.0 * (double)u[i]);
    for (int k = 0; k < g.nh; k++) {
        for (int64_t z = 0; z < g.D; z++)
            for (int64_t y = 0; y < g.H; y++)
                for (int64_t x = 0; x < g.W; x++) {
                    int64_t i = (z * g.H + y) * g.W + x, nz, ny, nx;
                    int32_t w = wq[(int64_t)k * n + i];
                    if (w < 0 && !allow_negative) return -2;
                    if (g_nbr(&g, z, y, x, k, &nz, &ny, &nx) < 0 && w != 0) return -3;
                    Wl[(int64_t)k * n + i] = llrint(lambda * (double)w);
                }
    }
    return 0;
}

/* E_int(y) = sum_i U_i y_i + sum_{undirected edges} Wl_ij |y_i - y_j|  (Eq. 1,
 * each undirected edge counted once, as in y^T L y of Eq. 3).  E = E_int/1024. */
int64_t orc_energy(const int64_t *dims, int conn, const int *block,
                   const int64_t *U, const int64_t *Wl, const uint8_t *lab)
{
    grid_t g;
    if (grid_init(&g, dims, conn, block)) return INT64_MIN;
    int64_t n = g_n(&g), e = 0;
    for (int64_t i = 0; i < n; i++) e += U[i] * (int64_t)lab[i];
    for (int k = 0; k < g.nh; k++)
        for (int64_t z = 0; z < g.D; z++)
            for (int64_t y = 0; y < g.H; y++)
                for (int64_t x = 0; x < g.W; x++) {
                    int64_t i = (z * g.H + y) * g.W + x, nz, ny, nx;
                    int64_t j = g_nbr(&g, z, y, x, k, &nz, &ny, &nx);
                    if (j < 0) continue;
                    if (lab[i] != lab[j]) e += Wl[(int64_t)k * n + i];
                }
    return e;
}

/* ------------------------------------------------------------------------ */
/* Boykov-Kolmogorov max-flow                                               */
/* ------------------------------------------------------------------------ */

#define BK_TERMINAL (-1)
#define BK_ORPHAN (-2)
#define BK_FREE (-3)
#define TREE_NONE 0
#define TREE_S 1
#define TREE_T 2

typedef struct {
    int n, m;           /* nodes, arcs (arcs come in sister pairs a, a^1) */
    int *first, *next, *head;
    int64_t *rcap;      /* residual capacity of each arc */
    int64_t *tr;        /* >0: residual s->i, <0: residual i->t */
    int *parent;        /* arc from node to its tree parent, or BK_* */
    unsigned char *tree;
    int *ts, *dist;
    int *q; unsigned char *inq; int qh, qt;   /* FIFO of active nodes, size n+1 */
    int *orph; int norph;                       /* orphan stack */
    long time;
} bk_t;

static int bk_alloc(bk_t *b, int n, int medges)
{
    memset(b, 0, sizeof(*b));
    b->n = n; b->m = 0;
    b->first = malloc(sizeof(int) * (size_t)n);
    b->next = malloc(sizeof(int) * (size_t)(2 * medges + 2));
    b->head = malloc(sizeof(int) * (size_t)(2 * medges + 2));
    b->rcap = malloc(sizeof(int64_t) * (size_t)(2 * medges + 2));
    b->tr = calloc((size_t)n, sizeof(int64_t));
    b->parent = malloc(sizeof(int) * (size_t)n);
    b->tree = calloc((size_t)n, 1);
    b->ts = calloc((size_t)n, sizeof(int));
    b->dist = calloc((size_t)n, sizeof(int));
    b->q = malloc(sizeof(int) * (size_t)(n + 1));
    b->inq = calloc((size_t)n, 1);
    b->orph = malloc(sizeof(int) * (size_t)(n + 1));
    if (!b->first || !b->next || !b->head || !b->rcap || !b->tr || !b->parent ||
        !b->tree || !b->ts || !b->dist || !b->q || !b->inq || !b->orph) return -1;
    for (int i = 0; i < n; i++) b->first[i] = -1;
    return 0;
}

static void bk_free(bk_t *b)
{
    free(b->first); free(b->next); free(b->head); free(b->rcap); free(b->tr);
    free(b->parent); free(b->tree); free(b->ts); free(b->dist); free(b->q);
    free(b->inq); free(b->orph);
}

/* Undirected-with-two-capacities edge: cap(i->j) = cij, cap(j->i) = cji. */
static void bk_edge(bk_t *b, int i, int j, int64_t cij, int64_t cji)
{
    int a = b->m, s = b->m + 1;
    b->head[a] = j; b->rcap[a] = cij; b->next[a] = b->first[i]; b->first[i] = a;
    b->head[s] = i; b->rcap[s] = cji; b->next[s] = b->first[j]; b->first[j] = s;
    b->m += 2;
}

static void bk_activate(bk_t *b, int i)
{
    if (b->inq[i]) return;
    b->inq[i] = 1;
    b->q[b->qt] = i;
    b->qt = (b->qt + 1) % (b->n + 1);
}

static int bk_pop(bk_t *b)
{
    while (b->qh != b->qt) {
        int i = b->q[b->qh];
        b->qh = (b->qh + 1) % (b->n + 1);
        b->inq[i] = 0;
        if (b->tree[i] != TREE_NONE) return i;
    }
    return -1;
}

static void bk_orphan(bk_t *b, int i)
{
    b->parent[i] = BK_ORPHAN;
    b->orph[b->norph++] = i;
}

/* Augment along s ~> tail(a) -a-> head(a) ~> t. */
static void bk_augment(bk_t *b, int a)
{
    int x, pa;
    int64_t bn = b->rcap[a];
    /* bottleneck on the source side */
    for (x = b->head[a ^ 1];; x = b->head[pa]) {
        pa = b->parent[x];
        if (pa == BK_TERMINAL) { if (b->tr[x] < bn) bn = b->tr[x]; break; }
        if (b->rcap[pa ^ 1] < bn) bn = b->rcap[pa ^ 1];
    }
    /* bottleneck on the sink side */
    for (x = b->head[a];; x = b->head[pa]) {
        pa = b->parent[x];
        if (pa == BK_TERMINAL) { if (-b->tr[x] < bn) bn = -b->tr[x]; break; }
        if (b->rcap[pa] < bn) bn = b->rcap[pa];
    }
    b->rcap[a] -= bn; b->rcap[a ^ 1] += bn;
    for (x = b->head[a ^ 1];;) {
        pa = b->parent[x];
        if (pa == BK_TERMINAL) {
            b->tr[x] -= bn;
            if (b->tr[x] == 0) bk_orphan(b, x);
            break;
        }
        int nx = b->head[pa];
        b->rcap[pa] += bn; b->rcap[pa ^ 1] -= bn;
        if (b->rcap[pa ^ 1] == 0) bk_orphan(b, x);
        x = nx;
    }
    for (x = b->head[a];;) {
        pa = b->parent[x];
        if (pa == BK_TERMINAL) {
            b->tr[x] += bn;
            if (b->tr[x] == 0) bk_orphan(b, x);
            break;
        }
        int nx = b->head[pa];
        b->rcap[pa ^ 1] += bn; b->rcap[pa] -= bn;
        if (b->rcap[pa] == 0) bk_orphan(b, x);
        x = nx;
    }
}

/* Adoption stage: find each orphan a new parent in its own tree whose path
 * reaches the terminal, preferring the shortest; otherwise free it. */
static void bk_adopt(bk_t *b)
{
    while (b->norph > 0) {
        int p = b->orph[--b->norph];
        int tp = b->tree[p];
        int best = -1, dmin = 1 << 30;
        b->time++;
        for (int a = b->first[p]; a >= 0; a = b->next[a]) {
            int q = b->head[a];
            if (b->tree[q] != tp) continue;
            int64_t r = (tp == TREE_S) ? b->rcap[a ^ 1] : b->rcap[a];
            if (r <= 0) continue;
            /* walk to the root of q */
            int d = 0, j = q, ok = 0;
            for (;;) {
                if (b->ts[j] == b->time) { d += b->dist[j]; ok = 1; break; }
                int pj = b->parent[j];
                d++;
                if (pj == BK_TERMINAL) { b->ts[j] = (int)b->time; b->dist[j] = 1; ok = 1; break; }
                if (pj == BK_ORPHAN || pj == BK_FREE) break;
                j = b->head[pj];
            }
            if (!ok) continue;
            if (d < dmin) { dmin = d; best = a; }
            for (j = q; b->ts[j] != b->time; j = b->head[b->parent[j]]) {
                b->ts[j] = (int)b->time; b->dist[j] = d; d--;
            }
        }
        if (best >= 0) {
            b->parent[p] = best;
            b->ts[p] = (int)b->time;
            b->dist[p] = dmin + 1;
            continue;
        }
        /* no parent: p becomes free */
        for (int a = b->first[p]; a >= 0; a = b->next[a]) {
            int q = b->head[a];
            if (b->tree[q] != tp) continue;
            int64_t r = (tp == TREE_S) ? b->rcap[a ^ 1] : b->rcap[a];
            if (r > 0) bk_activate(b, q);
            int pq = b->parent[q];
            if (pq >= 0 && b->head[pq] == p) bk_orphan(b, q);
        }
        b->tree[p] = TREE_NONE;
        b->parent[p] = BK_FREE;
    }
}

/* Max-flow; afterwards lab[i] = 1 iff i reaches t in the residual graph,
 * which is the minimal sink side of all minimum cuts (the pointwise-minimal
 * minimiser of the energy, with y_i = 1 <=> sink side). */
static void bk_run(bk_t *b, uint8_t *lab)
{
    b->qh = b->qt = 0; b->norph = 0; b->time = 0;
    for (int i = 0; i < b->n; i++) {
        if (b->tr[i] > 0) { b->tree[i] = TREE_S; b->parent[i] = BK_TERMINAL; b->dist[i] = 1; bk_activate(b, i); }
        else if (b->tr[i] < 0) { b->tree[i] = TREE_T; b->parent[i] = BK_TERMINAL; b->dist[i] = 1; bk_activate(b, i); }
        else { b->tree[i] = TREE_NONE; b->parent[i] = BK_FREE; }
        b->ts[i] = 0;
    }
    for (;;) {
        int p = bk_pop(b);
        if (p < 0) break;
        int found = -1;
        if (b->tree[p] == TREE_S) {
            for (int a = b->first[p]; a >= 0; a = b->next[a]) {
                if (b->rcap[a] <= 0) continue;
                int q = b->head[a];
                if (b->tree[q] == TREE_NONE) {
                    b->tree[q] = TREE_S; b->parent[q] = a ^ 1;
                    b->ts[q] = b->ts[p]; b->dist[q] = b->dist[p] + 1;
                    bk_activate(b, q);
                } else if (b->tree[q] == TREE_T) { found = a; break; }
                else if (b->ts[q] <= b->ts[p] && b->dist[q] > b->dist[p]) {
                    b->parent[q] = a ^ 1; b->ts[q] = b->ts[p]; b->dist[q] = b->dist[p] + 1;
                }
            }
        } else {
            for (int a = b->first[p]; a >= 0; a = b->next[a]) {
                if (b->rcap[a ^ 1] <= 0) continue;
                int q = b->head[a];
                if (b->tree[q] == TREE_NONE) {
                    b->tree[q] = TREE_T; b->parent[q] = a ^ 1;
                    b->ts[q] = b->ts[p]; b->dist[q] = b->dist[p] + 1;
                    bk_activate(b, q);
                } else if (b->tree[q] == TREE_S) { found = a ^ 1; break; }
                else if (b->ts[q] <= b->ts[p] && b->dist[q] > b->dist[p]) {
                    b->parent[q] = a ^ 1; b->ts[q] = b->ts[p]; b->dist[q] = b->dist[p] + 1;
                }
            }
        }
        b->time++;
        if (found >= 0) {
            bk_activate(b, p);   /* p may have unexplored neighbours left */
            bk_augment(b, found);
            bk_adopt(b);
        }
    }
    /* canonical cut: backward BFS from t over residual arcs */
    int *queue = malloc(sizeof(int) * (size_t)(b->n + 1));
    int qh = 0, qt = 0;
    for (int i = 0; i < b->n; i++) {
        lab[i] = 0;
        if (b->tr[i] < 0) { lab[i] = 1; queue[qt++] = i; }
    }
    while (qh < qt) {
        int x = queue[qh++];
        for (int a = b->first[x]; a >= 0; a = b->next[a]) {
            int j = b->head[a];
            if (!lab[j] && b->rcap[a ^ 1] > 0) { lab[j] = 1; queue[qt++] = j; }
        }
    }
    free(queue);
}

/* Generic min-cut of  sum_i c_i y_i + sum_e [ cuv_e * (1-y_u) y_v + cvu_e * y_u (1-y_v) ]
 * with y_i = 1 <=> sink side: terminal capacity c_i > 0 is s->i, c_i < 0 is
 * i->t; cap(u->v) = cuv_e, cap(v->u) = cvu_e (both >= 0).
 * Writes the canonical (pointwise-minimal) minimiser to lab; returns 0. */
int orc_bk_mincut(int n, const int64_t *c, int m, const int32_t *eu, const int32_t *ev,
                  const int64_t *cuv, const int64_t *cvu, uint8_t *lab)
{
    bk_t b;
    if (bk_alloc(&b, n, m)) { bk_free(&b); return -1; }
    for (int i = 0; i < n; i++) b.tr[i] = c[i];
    for (int e = 0; e < m; e++) {
        if (cuv[e] < 0 || cvu[e] < 0) { bk_free(&b); return -2; }
        bk_edge(&b, eu[e], ev[e], cuv[e], cvu[e]);
    }
    bk_run(&b, lab);
    bk_free(&b);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Brute force (any sign of w): pins the cut on tiny instances              */
/* ------------------------------------------------------------------------ */

/* E(y) = sum_i c_i y_i + sum_e w_e |y_u - y_v| over all 2^n labelings.
 * Outputs the minimum, the AND and OR of all minimisers and their count. */
int orc_bruteforce(int n, const int64_t *c, int m, const int32_t *eu, const int32_t *ev,
                   const int64_t *w, int64_t *emin, uint8_t *and_lab, uint8_t *or_lab,
                   int64_t *count)
{
    if (n > 24 || n < 0) return -1;
    int64_t best = INT64_MAX, cnt = 0;
    uint32_t andm = 0, orm = 0;
    for (uint32_t s = 0; s < (1u << n); s++) {
        int64_t e = 0;
        for (int i = 0; i < n; i++) if (s >> i & 1u) e += c[i];
        for (int k = 0; k < m; k++)
            if (((s >> eu[k]) ^ (s >> ev[k])) & 1u) e += w[k];
        if (e < best) { best = e; cnt = 1; andm = s; orm = s; }
        else if (e == best) { cnt++; andm &= s; orm |= s; }
    }
    *emin = best; *count = cnt;
    for (int i = 0; i < n; i++) { and_lab[i] = (andm >> i) & 1u; or_lab[i] = (orm >> i) & 1u; }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* DOPE, Q = I (non-overlapping blocks)                                     */
/* ------------------------------------------------------------------------ */

/* Eq. 8 unary of every pixel, scaled by 1024 and rounded half-to-even:
 *   1024 c_i = U_i + sum_{j in X(i)} Wl_ij (y_i - y_j) + (1024 mu) ((a_i - y_i) + 1/2)
 * i.e. 1024 * ( u_i + lambda [(C_k + R_k S_k) y]_i + mu (a_i - y_i + 1/2) ).
 * Order of operations: start from U_i, add the cross terms in direction
 * order k = 0..d-1, then add the multiplier term.  s_out (may be NULL)
 * receives the unrounded double, C_out the rounded int64. */
int orc_shifted_caps(const int64_t *dims, int conn, const int *block,
                     const int64_t *U, const int64_t *Wl,
                     const double *y, const double *a, double mu,
                     double *s_out, int64_t *C_out)
{
    grid_t g;
    if (grid_init(&g, dims, conn, block)) return -1;
    double m1024 = 1024.0 * mu;
    for (int64_t z = 0; z < g.D; z++)
        for (int64_t yy = 0; yy < g.H; yy++)
            for (int64_t x = 0; x < g.W; x++) {
                int64_t i = (z * g.H + yy) * g.W + x, nz, ny, nx;
                int64_t bi = g_block_of(&g, z, yy, x);
                double s = (double)U[i];
                for (int k = 0; k < g.conn; k++) {
                    int64_t j = g_nbr(&g, z, yy, x, k, &nz, &ny, &nx);
                    if (j < 0 || g_block_of(&g, nz, ny, nx) == bi) continue;
                    double w = (double)g_wt(&g, Wl, i, j, k);
                    double dy = y[i] - y[j];
                    double t = w * dy;
                    s = s + t;
                }
                double v = a[i] - y[i];
                v = v + 0.5;
                double t = m1024 * v;
                s = s + t;
                if (s_out) s_out[i] = s;
                /* |1024 c_i| is clamped to 2^62 before rounding: n-link
                 * capacities are below 2^28 per node, so a node whose unary
                 * is that large takes the same label in every minimiser and
                 * the clamp changes no minimiser (it only keeps llrint in
                 * range when mu has grown for many iterations). */
                if (s > 4611686018427387904.0) s = 4611686018427387904.0;
                if (s < -4611686018427387904.0) s = -4611686018427387904.0;
                C_out[i] = llrint(s);
            }
    return 0;
}

/* Eq. 8 for every block, solved exactly by BK on the block graph: terminal
 * capacity C_i, n-links Wl_ij for edges with both ends in the block (edges
 * leaving the block are represented by the C_k, R_k terms already inside C).
 * Blocks are independent ("in parallel", Algorithm 1). */
int orc_block_cuts(const int64_t *dims, int conn, const int *block,
                   const int64_t *Wl, const int64_t *C, uint8_t *yhat)
{
    grid_t g;
    if (grid_init(&g, dims, conn, block)) return -1;
    int64_t K = g_nblocks(&g);
    int B = g.bd * g.bh * g.bw;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (int64_t k = 0; k < K; k++) {
        bk_t b;
        uint8_t *lab = malloc((size_t)B);
        int64_t *gidx = malloc(sizeof(int64_t) * (size_t)B);
        if (!lab || !gidx || bk_alloc(&b, B, B * g.nh)) { err |= 1; free(lab); free(gidx); continue; }
        for (int l = 0; l < B; l++) {
            int64_t z, y, x;
            gidx[l] = g_block_pixel(&g, k, l, &z, &y, &x);
            b.tr[l] = C[gidx[l]];
        }
        for (int l = 0; l < B; l++) {
            int64_t z, y, x, nz, ny, nx;
            int64_t i = g_block_pixel(&g, k, l, &z, &y, &x);
            for (int o = 0; o < g.nh; o++) {
                int64_t j = g_nbr(&g, z, y, x, o, &nz, &ny, &nx);
                if (j < 0 || g_block_of(&g, nz, ny, nx) != k) continue;
                int lj = (int)(((nz % g.bd) * g.bh + (ny % g.bh)) * g.bw + (nx % g.bw));
                int64_t w = Wl[(int64_t)o * g_n(&g) + i];
                if (w > 0) bk_edge(&b, l, lj, w, w);
            }
        }
        bk_run(&b, lab);
        for (int l = 0; l < B; l++) yhat[gidx[l]] = lab[l];
        bk_free(&b);
        free(lab); free(gidx);
    }
    return err ? -1 : 0;
}

/* Eq. 10 and Eq. 11 for Q = I, then the per-block quantity of the stop test:
 *   g_i   = sum_{j in X(i)} Wl_ij (yhat_i - yhat_j) / 1024   (= lambda [(C+RS)^T yhat]_i)
 *   y_i   = (yhat_i + a_i) - g_i / mu                        (Eq. 10)
 *   a_i   = a_i + (yhat_i - y_i)                             (Eq. 11)
 *   r2_k  = sum_{i in block k} (yhat_i - y_i)^2  (block-local order)
 * y and a are updated in place. */
int orc_update(const int64_t *dims, int conn, const int *block,
               const int64_t *Wl, const uint8_t *yhat, double mu,
               double *y, double *a, double *r2)
{
    grid_t g;
    if (grid_init(&g, dims, conn, block)) return -1;
    int64_t n = g_n(&g);
    for (int64_t z = 0; z < g.D; z++)
        for (int64_t yy = 0; yy < g.H; yy++)
            for (int64_t x = 0; x < g.W; x++) {
                int64_t i = (z * g.H + yy) * g.W + x, nz, ny, nx;
                int64_t bi = g_block_of(&g, z, yy, x);
                int64_t G = 0;
                for (int k = 0; k < g.conn; k++) {
                    int64_t j = g_nbr(&g, z, yy, x, k, &nz, &ny, &nx);
                    if (j < 0 || g_block_of(&g, nz, ny, nx) == bi) continue;
                    G += g_wt(&g, Wl, i, j, k) * ((int64_t)yhat[i] - (int64_t)yhat[j]);
                }
                double gi = (double)G / 1024.0;
                double yi = ((double)yhat[i] + a[i]) - gi / mu;
                y[i] = yi;
                a[i] = a[i] + ((double)yhat[i] - yi);
            }
    int64_t K = g_nblocks(&g);
    int B = g.bd * g.bh * g.bw;
    for (int64_t k = 0; k < K; k++) {
        double s = 0.0;
        for (int l = 0; l < B; l++) {
            int64_t z, yy, x;
            int64_t i = g_block_pixel(&g, k, l, &z, &yy, &x);
            double d = (double)yhat[i] - y[i];
            s = s + d * d;
        }
        r2[k] = s;
    }
    (void)n;
    return 0;
}

/* Algorithm 1.  y := 1/2, a := 0, mu := mu0; then repeat
 *   yhat_k <- argmin Eq. 8 (all blocks), y <- Eq. 10, a <- Eq. 11, mu <- mu * mu_fact
 * while some block has ||yhat_k - S_k y||_2 > eps (tested after the updates,
 * so at least one iteration runs), for at most max_iter iterations.
 * Outputs: labels = yhat of the last iteration, *iters, and per iteration t
 * (0-based, if the arrays are non-NULL): rmax[t] = max_k ||yhat_k - S_k y||,
 * flips[t] = number of labels that changed vs the previous iteration.
 * Returns 0 converged, 1 max_iter reached, <0 error. */
int orc_admm(const int64_t *dims, int conn, const int *block,
             const int64_t *U, const int64_t *Wl,
             double mu0, double mu_fact, double eps, int max_iter,
             uint8_t *labels, int *iters, double *rmax_trace, int64_t *flips_trace,
             double *y_out, double *a_out, double *mu_out)
{
    grid_t g;
    if (grid_init(&g, dims, conn, block)) return -1;
    int64_t n = g_n(&g), K = g_nblocks(&g);
    double *y = malloc(sizeof(double) * (size_t)n);
    double *a = malloc(sizeof(double) * (size_t)n);
    double *r2 = malloc(sizeof(double) * (size_t)K);
    int64_t *C = malloc(sizeof(int64_t) * (size_t)n);
    uint8_t *prev = malloc((size_t)n);
    if (!y || !a || !r2 || !C || !prev) { free(y); free(a); free(r2); free(C); free(prev); return -4; }
    for (int64_t i = 0; i < n; i++) { y[i] = 0.5; a[i] = 0.0; prev[i] = 0; }
    double mu = mu0;
    int t = 0, rc = 1;
    while (t < max_iter) {
        orc_shifted_caps(dims, conn, block, U, Wl, y, a, mu, NULL, C);
        orc_block_cuts(dims, conn, block, Wl, C, labels);
        orc_update(dims, conn, block, Wl, labels, mu, y, a, r2);
        double m2 = 0.0;
        for (int64_t k = 0; k < K; k++) if (r2[k] > m2) m2 = r2[k];
        double rmax = sqrt(m2);
        if (rmax_trace) rmax_trace[t] = rmax;
        if (flips_trace) {
            int64_t f = 0;
            for (int64_t i = 0; i < n; i++) f += (labels[i] != prev[i]);
            flips_trace[t] = f;
        }
        memcpy(prev, labels, (size_t)n);
        mu = mu * mu_fact;
        t++;
        if (!(rmax > eps)) { rc = 0; break; }
    }
    *iters = t;
    if (y_out) memcpy(y_out, y, sizeof(double) * (size_t)n);
    if (a_out) memcpy(a_out, a, sizeof(double) * (size_t)n);
    if (mu_out) *mu_out = mu;
    free(y); free(a); free(r2); free(C); free(prev);
    return rc;
}

/* One ADMM iteration from a given state (the same step orc_admm takes):
 * solve Eq. 8 with (y, a, mu), then Eq. 10 / Eq. 11 in place.  r2 per block. */
int orc_admm_step(const int64_t *dims, int conn, const int *block,
                  const int64_t *U, const int64_t *Wl, double mu,
                  double *y, double *a, uint8_t *yhat, double *r2)
{
    grid_t g;
    if (grid_init(&g, dims, conn, block)) return -1;
    int64_t n = g_n(&g);
    int64_t *C = malloc(sizeof(int64_t) * (size_t)n);
    if (!C) return -4;
    orc_shifted_caps(dims, conn, block, U, Wl, y, a, mu, NULL, C);
    orc_block_cuts(dims, conn, block, Wl, C, yhat);
    orc_update(dims, conn, block, Wl, yhat, mu, y, a, r2);
    free(C);
    return 0;
}

/* The serial graph cut (sGC) on the whole grid: exact global minimiser of
 * Eq. 1 (canonical, pointwise minimal).  Returns E_int of it. */
int64_t orc_global_mincut(const int64_t *dims, int conn, const int *block,
                          const int64_t *U, const int64_t *Wl, uint8_t *labels)
{
    grid_t g;
    if (grid_init(&g, dims, conn, block)) return INT64_MIN;
    int64_t n = g_n(&g);
    if (n > 0x7fffffff / (g.nh + 1)) return INT64_MIN;
    bk_t b;
    if (bk_alloc(&b, (int)n, (int)(n * g.nh))) { bk_free(&b); return INT64_MIN; }
    for (int64_t i = 0; i < n; i++) b.tr[i] = U[i];
    for (int64_t z = 0; z < g.D; z++)
        for (int64_t y = 0; y < g.H; y++)
            for (int64_t x = 0; x < g.W; x++) {
                int64_t i = (z * g.H + y) * g.W + x, nz, ny, nx;
                for (int o = 0; o < g.nh; o++) {
                    int64_t j = g_nbr(&g, z, y, x, o, &nz, &ny, &nx);
                    if (j < 0) continue;
                    int64_t w = Wl[(int64_t)o * n + i];
                    if (w > 0) bk_edge(&b, (int)i, (int)j, w, w);
                }
            }
    bk_run(&b, labels);
    bk_free(&b);
    return orc_energy(dims, conn, block, U, Wl, labels);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* DOPE, overlapping blocks (Q != I; the paper's Size10 / Size25 partitions) */
/* ------------------------------------------------------------------------ */
/*
 * Partition: the regular tiling by `block` (the Q = I partition) with every
 * tile grown by grow[a] pixels on both sides along axis a, clipped to the
 * grid (Section 3: blocks "increased" in size).  2 grow[a] <= block[a], so a
 * pixel lies in at most two tiles per axis and q_i (Proposition 1: the number
 * of blocks holding i) is a power of two, at most qmax = 2^(axes with grow > 0).
 * Block k is stored as the full box of (block + 2 grow) pixels per axis around
 * tile k; box nodes outside the grid do not belong to Omega_k ("phantoms":
 * label 0, multiplier 0, no terms).
 *
 * Theorem 1 in stencil form (derived from the matrix definitions; the literal
 * matrices of oracle/theorem1.py pin it), for i in Omega_k, with
 * phi_kj = 1 - [j in Omega_k] / q_j:
 *   u_hat_k[i]                 = u_i / q_i
 *   W_hat_k[i,j]               = w_ij / (q_i q_j)           (i, j in Omega_k)
 *   [(C_k + R_k S_k) y]_i      = (1/q_i) sum_{j in N(i)} w_ij phi_kj (y_i - y_j)
 *   [(C_k + R_k S_k)^T yh_k]_j = [j in Omega_k] (1/q_j) sum_{i in N(j)} w_ij phi_ki yh_k[j]
 *                                - phi_kj sum_{i in N(j), i in Omega_k} (w_ij / q_i) yh_k[i]
 * Integers: every block objective of Eq. 8 is multiplied by M = qmax^2 (a
 * positive constant: same minimisers), so the n-links M Wl_ij / (q_i q_j) are
 * integers, and the unary is rne(M * 1024 c_i).  Eq. 10's cross term is an
 * integer in units of 1 / (1024 M): the "G" below.  With grow = 0 every
 * formula here reduces, operation for operation, to the Q = I functions above.
 */

typedef struct {
    grid_t g;
    int gd, gh, gw;           /* grow per side */
    int ed, eh, ew, eb;       /* box extent, box volume */
    int64_t nbz, nby, nbx, K; /* tiles */
    int qmax, M;
    uint8_t *q;               /* q per pixel, computed once by ov_init (ov_free releases it) */
} ov_t;

static int ov_init(ov_t *o, const int64_t *dims, int conn, const int *block, const int *grow)
{
    if (grid_init(&o->g, dims, conn, block)) return -1;
    o->gd = grow[0]; o->gh = grow[1]; o->gw = grow[2];
    if (o->gd < 0 || o->gh < 0 || o->gw < 0) return -1;
    if (2 * o->gd > o->g.bd || 2 * o->gh > o->g.bh || 2 * o->gw > o->g.bw) return -1;
    o->ed = o->g.bd + 2 * o->gd; o->eh = o->g.bh + 2 * o->gh; o->ew = o->g.bw + 2 * o->gw;
    o->eb = o->ed * o->eh * o->ew;
    o->nbz = o->g.D / o->g.bd; o->nby = o->g.H / o->g.bh; o->nbx = o->g.W / o->g.bw;
    o->K = o->nbz * o->nby * o->nbx;
    o->qmax = (o->gd > 0 ? 2 : 1) * (o->gh > 0 ? 2 : 1) * (o->gw > 0 ? 2 : 1);
    o->M = o->qmax * o->qmax;
    o->q = NULL;
    return 0;
}

static void ov_free(ov_t *o) { free(o->q); o->q = NULL; }

/* Largest coordinate offset of the neighbourhood. */
static int64_t ov_radius(const grid_t *g)
{
    int r = 0;
    for (int o = 0; o < g->nh; o++)
        for (int a = 0; a < 3; a++) {
            int v = g->off[o][a] < 0 ? -g->off[o][a] : g->off[o][a];
            if (v > r) r = v;
        }
    return r;
}

/* Tiles along one axis whose grown range holds coordinate c. */
static int ov_axis_count(int64_t c, int64_t nb, int b, int gr)
{
    int n = 0;
    int64_t lo = (c - gr) / b - 1, hi = (c + gr) / b + 1;
    for (int64_t t = lo; t <= hi; t++) {
        if (t < 0 || t >= nb) continue;
        if (c >= t * b - gr && c < (t + 1) * b + gr) n++;
    }
    return n;
}

static int ov_q_count(const ov_t *o, int64_t z, int64_t y, int64_t x)
{
    return ov_axis_count(z, o->nbz, o->g.bd, o->gd) * ov_axis_count(y, o->nby, o->g.bh, o->gh) *
           ov_axis_count(x, o->nbx, o->g.bw, o->gw);
}

/* Fill the per-pixel table; -4 if out of memory. */
static int ov_make_q(ov_t *o)
{
    o->q = malloc((size_t)g_n(&o->g));
    if (!o->q) return -4;
    for (int64_t z = 0; z < o->g.D; z++)
        for (int64_t y = 0; y < o->g.H; y++)
            for (int64_t x = 0; x < o->g.W; x++)
                o->q[(z * o->g.H + y) * o->g.W + x] = (uint8_t)ov_q_count(o, z, y, x);
    return 0;
}

static inline int ov_q(const ov_t *o, int64_t z, int64_t y, int64_t x)
{
    return o->q[(z * o->g.H + y) * o->g.W + x];
}

/* Tile coordinates of block k. */
static void ov_tile(const ov_t *o, int64_t k, int64_t *kz, int64_t *ky, int64_t *kx)
{
    *kz = k / (o->nby * o->nbx); *ky = (k / o->nbx) % o->nby; *kx = k % o->nbx;
}

/* Box node l of block k -> grid coordinates; returns the pixel index or -1 for
 * a phantom (outside the grid). */
static int64_t ov_node(const ov_t *o, int64_t k, int l, int64_t *pz, int64_t *py, int64_t *px)
{
    int64_t kz, ky, kx;
    ov_tile(o, k, &kz, &ky, &kx);
    int lz = l / (o->eh * o->ew), ly = (l / o->ew) % o->eh, lx = l % o->ew;
    int64_t z = kz * o->g.bd - o->gd + lz, y = ky * o->g.bh - o->gh + ly, x = kx * o->g.bw - o->gw + lx;
    *pz = z; *py = y; *px = x;
    if (z < 0 || z >= o->g.D || y < 0 || y >= o->g.H || x < 0 || x >= o->g.W) return -1;
    return (z * o->g.H + y) * o->g.W + x;
}

/* Box-local index of grid pixel (z, y, x) in block k, or -1 if not in Omega_k. */
static int ov_local(const ov_t *o, int64_t k, int64_t z, int64_t y, int64_t x)
{
    int64_t kz, ky, kx;
    ov_tile(o, k, &kz, &ky, &kx);
    int64_t lz = z - (kz * o->g.bd - o->gd), ly = y - (ky * o->g.bh - o->gh), lx = x - (kx * o->g.bw - o->gw);
    if (lz < 0 || lz >= o->ed || ly < 0 || ly >= o->eh || lx < 0 || lx >= o->ew) return -1;
    return (int)((lz * o->eh + ly) * o->ew + lx);
}

/* Geometry query: q per pixel (image order), box extent, M. */
int orc_ov_geometry(const int64_t *dims, int conn, const int *block, const int *grow,
                    int32_t *q, int *box, int *M, int64_t *K)
{
    ov_t o;
    if (ov_init(&o, dims, conn, block, grow) || ov_make_q(&o)) return -1;
    if (q)
        for (int64_t z = 0; z < o.g.D; z++)
            for (int64_t y = 0; y < o.g.H; y++)
                for (int64_t x = 0; x < o.g.W; x++) q[(z * o.g.H + y) * o.g.W + x] = ov_q(&o, z, y, x);
    if (box) { box[0] = o.ed; box[1] = o.eh; box[2] = o.ew; }
    if (M) *M = o.M;
    if (K) *K = o.K;
    ov_free(&o);
    return 0;
}

/* Eq. 8 unary of every box node (K x eb, box-major), general Q:
 *   s  = U_i + sum_d (Wl_ij phi_kj)(y_i - y_j)     directions d = 0..conn-1, phi = 0 skipped
 *   s  = s / q_i + (1024 mu)((a_ki - y_i) + 1/2)
 *   C  = rne(M s), |M s| clamped to 2^62.
 * s_out (may be NULL) gets s, C_out gets C; phantoms get 0. */
int orc_ov_caps(const int64_t *dims, int conn, const int *block, const int *grow,
                const int64_t *U, const int64_t *Wl, const double *y, const double *a,
                double mu, double *s_out, int64_t *C_out)
{
    ov_t o;
    if (ov_init(&o, dims, conn, block, grow) || ov_make_q(&o)) return -1;
    const grid_t *g = &o.g;
    double m1024 = 1024.0 * mu;
    for (int64_t k = 0; k < o.K; k++)
        for (int l = 0; l < o.eb; l++) {
            int64_t z, yy, x, nz, ny, nx;
            int64_t i = ov_node(&o, k, l, &z, &yy, &x);
            int64_t kl = k * o.eb + l;
            if (i < 0) { if (s_out) s_out[kl] = 0.0; C_out[kl] = 0; continue; }
            double s = (double)U[i];
            for (int d = 0; d < g->conn; d++) {
                int64_t j = g_nbr(g, z, yy, x, d, &nz, &ny, &nx);
                if (j < 0) continue;
                double phi = 1.0;
                if (ov_local(&o, k, nz, ny, nx) >= 0) {
                    int qj = ov_q(&o, nz, ny, nx);
                    if (qj == 1) continue;
                    phi = 1.0 - 1.0 / (double)qj;
                }
                double w = (double)g_wt(g, Wl, i, j, d);
                double wf = w * phi;
                double dy = y[i] - y[j];
                double t = wf * dy;
                s = s + t;
            }
            s = s / (double)ov_q(&o, z, yy, x);
            double v = a[kl] - y[i];
            v = v + 0.5;
            double t = m1024 * v;
            s = s + t;
            if (s_out) s_out[kl] = s;
            double ms = (double)o.M * s;
            if (ms > 4611686018427387904.0) ms = 4611686018427387904.0;
            if (ms < -4611686018427387904.0) ms = -4611686018427387904.0;
            C_out[kl] = llrint(ms);
        }
    ov_free(&o);
    return 0;
}

/* Eq. 8 of every block by BK on its box graph: terminal C (box-major), n-link
 * M Wl_ij / (q_i q_j) between box nodes in the grid; phantoms get label 0. */
int orc_ov_block_cuts(const int64_t *dims, int conn, const int *block, const int *grow,
                      const int64_t *Wl, const int64_t *C, uint8_t *yhat)
{
    ov_t o;
    if (ov_init(&o, dims, conn, block, grow) || ov_make_q(&o)) return -1;
    const grid_t *g = &o.g;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (int64_t k = 0; k < o.K; k++) {
        bk_t b;
        uint8_t *lab = malloc((size_t)o.eb);
        if (!lab || bk_alloc(&b, o.eb, o.eb * g->nh)) { err |= 1; free(lab); continue; }
        for (int l = 0; l < o.eb; l++) b.tr[l] = C[k * o.eb + l];
        for (int l = 0; l < o.eb; l++) {
            int64_t z, y, x, nz, ny, nx;
            int64_t i = ov_node(&o, k, l, &z, &y, &x);
            if (i < 0) continue;
            int qi = ov_q(&o, z, y, x);
            for (int d = 0; d < g->nh; d++) {
                int64_t j = g_nbr(g, z, y, x, d, &nz, &ny, &nx);
                if (j < 0) continue;
                int lj = ov_local(&o, k, nz, ny, nx);
                if (lj < 0) continue;
                int qj = ov_q(&o, nz, ny, nx);
                int64_t w = Wl[(int64_t)d * g_n(g) + i] * (int64_t)(o.M / (qi * qj));
                if (w > 0) bk_edge(&b, l, lj, w, w);
            }
        }
        bk_run(&b, lab);
        for (int l = 0; l < o.eb; l++) {
            int64_t z, y, x;
            yhat[k * o.eb + l] = ov_node(&o, k, l, &z, &y, &x) < 0 ? 0 : lab[l];
        }
        bk_free(&b);
        free(lab);
    }
    ov_free(&o);
    return err ? -1 : 0;
}

/* Eq. 10 (y, image order) and Eq. 11 (a, box-major), general Q, then the
 * per-block stop quantity r2_k = sum_{l in Omega_k} (yhat_kl - y_i)^2 (box order):
 *   A_j  = sum_{k holding j, increasing k} (yhat_kj + a_kj)
 *   G_j  = 1024 M sum_k [(C_k + R_k S_k)^T yh_k]_j / lambda   (exact integer)
 *   y_j  = A_j / q_j - ((G_j / (1024 M)) / mu) / q_j
 *   a_kl = a_kl + (yhat_kl - y_i). */
int orc_ov_update(const int64_t *dims, int conn, const int *block, const int *grow,
                  const int64_t *Wl, const uint8_t *yhat, double mu, double *y, double *a, double *r2)
{
    ov_t o;
    if (ov_init(&o, dims, conn, block, grow) || ov_make_q(&o)) return -1;
    const grid_t *g = &o.g;
    for (int64_t z = 0; z < g->D; z++)
        for (int64_t yy = 0; yy < g->H; yy++)
            for (int64_t x = 0; x < g->W; x++) {
                int64_t j = (z * g->H + yy) * g->W + x, iz, iy, ix;
                int qj = ov_q(&o, z, yy, x);
                /* tiles whose box can hold j or a neighbour of j (up to R away) */
                int64_t R = ov_radius(g);
                int64_t k0z = (z - R - o.gd) / g->bd - 1, k1z = (z + R + o.gd) / g->bd + 1;
                int64_t k0y = (yy - R - o.gh) / g->bh - 1, k1y = (yy + R + o.gh) / g->bh + 1;
                int64_t k0x = (x - R - o.gw) / g->bw - 1, k1x = (x + R + o.gw) / g->bw + 1;
                double A = 0.0;
                int64_t G = 0;
                for (int64_t kz = k0z; kz <= k1z; kz++)
                    for (int64_t ky = k0y; ky <= k1y; ky++)
                        for (int64_t kx = k0x; kx <= k1x; kx++) {
                            if (kz < 0 || kz >= o.nbz || ky < 0 || ky >= o.nby || kx < 0 || kx >= o.nbx) continue;
                            int64_t k = (kz * o.nby + ky) * o.nbx + kx;
                            int lj = ov_local(&o, k, z, yy, x);
                            int64_t yj = lj >= 0 ? yhat[k * o.eb + lj] : 0;
                            if (lj >= 0) {
                                double t = (double)yhat[k * o.eb + lj] + a[k * o.eb + lj];
                                A = A + t;
                            }
                            for (int d = 0; d < g->conn; d++) {
                                int64_t i = g_nbr(g, z, yy, x, d, &iz, &iy, &ix);
                                if (i < 0) continue;
                                int li = ov_local(&o, k, iz, iy, ix);
                                int qi = ov_q(&o, iz, iy, ix);
                                int64_t w = g_wt(g, Wl, j, i, d);
                                if (lj >= 0 && yj) {   /* M (q_i - [i in Omega_k]) / (q_i q_j) */
                                    G += w * ((int64_t)o.M * (qi - (li >= 0)) / (qi * qj));
                                }
                                if (li >= 0 && yhat[k * o.eb + li]) {   /* M (q_j - [j in Omega_k]) / (q_j q_i) */
                                    G -= w * ((int64_t)o.M * (qj - (lj >= 0)) / (qj * qi));
                                }
                            }
                        }
                double yv = A / (double)qj;
                double gq = (double)G / (1024.0 * (double)o.M);
                double t = gq / mu;
                t = t / (double)qj;
                y[j] = yv - t;
            }
    for (int64_t k = 0; k < o.K; k++) {
        double s = 0.0;
        for (int l = 0; l < o.eb; l++) {
            int64_t z, yy, x;
            int64_t i = ov_node(&o, k, l, &z, &yy, &x);
            if (i < 0) continue;
            double yh = (double)yhat[k * o.eb + l];
            a[k * o.eb + l] = a[k * o.eb + l] + (yh - y[i]);
            double d = yh - y[i];
            s = s + d * d;
        }
        r2[k] = s;
    }
    ov_free(&o);
    return 0;
}

/* Proposition 1 for the output: label_i = 1 iff the block copies vote 1 by a
 * strict majority (2 sum_k yhat_ki > q_i); with consistent blocks this is the
 * common label, Q^-1 sum_k S_k^T yhat_k. */
int orc_ov_labels(const int64_t *dims, int conn, const int *block, const int *grow,
                  const uint8_t *yhat, uint8_t *labels)
{
    ov_t o;
    if (ov_init(&o, dims, conn, block, grow) || ov_make_q(&o)) return -1;
    const grid_t *g = &o.g;
    for (int64_t z = 0; z < g->D; z++)
        for (int64_t yy = 0; yy < g->H; yy++)
            for (int64_t x = 0; x < g->W; x++) {
                int votes = 0;
                for (int64_t kz = (z - o.gd) / g->bd - 1; kz <= (z + o.gd) / g->bd + 1; kz++)
                    for (int64_t ky = (yy - o.gh) / g->bh - 1; ky <= (yy + o.gh) / g->bh + 1; ky++)
                        for (int64_t kx = (x - o.gw) / g->bw - 1; kx <= (x + o.gw) / g->bw + 1; kx++) {
                            if (kz < 0 || kz >= o.nbz || ky < 0 || ky >= o.nby || kx < 0 || kx >= o.nbx) continue;
                            int64_t k = (kz * o.nby + ky) * o.nbx + kx;
                            int l = ov_local(&o, k, z, yy, x);
                            if (l >= 0) votes += yhat[k * o.eb + l];
                        }
                labels[(z * g->H + yy) * g->W + x] = (uint8_t)(2 * votes > ov_q(&o, z, yy, x));
            }
    ov_free(&o);
    return 0;
}

/* Algorithm 1 with overlapping blocks; same loop as orc_admm.  Outputs the
 * Proposition 1 labels, iterations, rmax trace, final y (image order), a and
 * yhat (box-major) and mu. */
int orc_ov_admm(const int64_t *dims, int conn, const int *block, const int *grow,
                const int64_t *U, const int64_t *Wl, double mu0, double mu_fact, double eps,
                int max_iter, uint8_t *labels, int *iters, double *rmax_trace,
                double *y_out, double *a_out, uint8_t *yhat_out, double *mu_out)
{
    ov_t o;
    if (ov_init(&o, dims, conn, block, grow)) return -1;
    int64_t n = g_n(&o.g), KB = o.K * o.eb;
    double *y = malloc(sizeof(double) * (size_t)n);
    double *a = calloc((size_t)KB, sizeof(double));
    double *r2 = malloc(sizeof(double) * (size_t)o.K);
    int64_t *C = malloc(sizeof(int64_t) * (size_t)KB);
    uint8_t *yh = calloc((size_t)KB, 1);
    if (!y || !a || !r2 || !C || !yh) { free(y); free(a); free(r2); free(C); free(yh); return -4; }
    for (int64_t i = 0; i < n; i++) y[i] = 0.5;
    double mu = mu0;
    int t = 0, rc = 1;
    while (t < max_iter) {
        orc_ov_caps(dims, conn, block, grow, U, Wl, y, a, mu, NULL, C);
        orc_ov_block_cuts(dims, conn, block, grow, Wl, C, yh);
        orc_ov_update(dims, conn, block, grow, Wl, yh, mu, y, a, r2);
        double m2 = 0.0;
        for (int64_t k = 0; k < o.K; k++) if (r2[k] > m2) m2 = r2[k];
        double rmax = sqrt(m2);
        if (rmax_trace) rmax_trace[t] = rmax;
        mu = mu * mu_fact;
        t++;
        if (!(rmax > eps)) { rc = 0; break; }
    }
    orc_ov_labels(dims, conn, block, grow, yh, labels);
    *iters = t;
    if (y_out) memcpy(y_out, y, sizeof(double) * (size_t)n);
    if (a_out) memcpy(a_out, a, sizeof(double) * (size_t)KB);
    if (yhat_out) memcpy(yhat_out, yh, (size_t)KB);
    if (mu_out) *mu_out = mu;
    free(y); free(a); free(r2); free(C); free(yh);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Non-submodular blocks: LSA-TR per block (Section 3.4 of the paper uses     */
/* the trust-region local submodular approximation of Gorelick et al. 2014)  */
/* ------------------------------------------------------------------------ */
/*
 * Block objective (Eq. 8, Q = I) with weights of any sign:
 *   E(x) = sum_i C_i x_i + sum_{edges ij in the block} Wl_ij |x_i - x_j|.
 * An edge with Wl_ij = -w < 0 equals -w x_i - w x_j + 2 w x_i x_j; its product
 * is replaced by the tangent of x_i x_j at the current labelling x^s,
 * x_i^s x_j + x_j^s x_i - x_i^s x_j^s, which makes the approximation
 * submodular and exact at x^s.  One trust-region step minimises
 *   approx(x) + lam * sum_i |x_i - x_i^s|
 * exactly (canonical minimal cut) and keeps the minimiser x* if E(x*) < E(x^s).
 * Trust region (integers): lam starts at LSA_LAM0; if x* = x^s the region
 * grows (lam /= 4; stop once lam = 0); an accepted step with actual decrease
 * R >= 3/4 of the predicted decrease P grows it too; a rejected step shrinks
 * it (lam = max(4 lam, 1)).  At most `steps` steps.  Everything is int64, so
 * the result is a deterministic function of (C, Wl, x^0).
 */
#define LSA_LAM0 1024

/* Exact block energy of labels x over the block's own edges. */
static int64_t lsa_energy(const grid_t *g, int64_t k, int B, const int64_t *Cb, const int64_t *Wl,
                          const uint8_t *x)
{
    int64_t e = 0;
    for (int l = 0; l < B; l++) {
        int64_t z, y, xx, nz, ny, nx;
        int64_t i = g_block_pixel(g, k, l, &z, &y, &xx);
        if (x[l]) e += Cb[l];
        for (int o = 0; o < g->nh; o++) {
            int64_t j = g_nbr(g, z, y, xx, o, &nz, &ny, &nx);
            if (j < 0 || g_block_of(g, nz, ny, nx) != k) continue;
            int lj = (int)(((nz % g->bd) * g->bh + (ny % g->bh)) * g->bw + (nx % g->bw));
            if (x[l] != x[lj]) e += Wl[(int64_t)o * g_n(g) + i];
        }
    }
    return e;
}

/* Per-step record of one LSA-TR run (test infrastructure: the CPU tests pin
 * every step against its definition).  Arrays have room for `cap` steps of B
 * nodes each; step s fills: xin[s*B..] the expansion point x^s, un[s*B..] the
 * approximation's unaries, cst[s] its constant, lam[s] the trust-region
 * weight, xout[s*B..] the step's minimiser, ecur[s] = E(x^s), ap[s] = the
 * approximation at the minimiser, enew[s] = E(minimiser) (ap, enew = 0 when
 * the minimiser is x^s), acc[s] = 1 if the minimiser was kept. */
typedef struct {
    int cap;
    uint8_t *xin, *xout;
    int64_t *un, *cst, *lam, *ecur, *ap, *enew;
    int *acc;
} lsa_trace_t;

/* LSA-TR on block k from x (in place); Cb = block unaries (local order). */
static int lsa_tr_block_traced(const grid_t *g, int64_t k, const int64_t *Cb, const int64_t *Wl, uint8_t *x,
                               int steps, int *steps_done, lsa_trace_t *tr);

static int lsa_tr_block(const grid_t *g, int64_t k, const int64_t *Cb, const int64_t *Wl, uint8_t *x,
                        int steps, int *steps_done)
{
    return lsa_tr_block_traced(g, k, Cb, Wl, x, steps, steps_done, NULL);
}

static int lsa_tr_block_traced(const grid_t *g, int64_t k, const int64_t *Cb, const int64_t *Wl, uint8_t *x,
                               int steps, int *steps_done, lsa_trace_t *tr)
{
    int B = g->bd * g->bh * g->bw;
    int64_t *un = malloc(sizeof(int64_t) * (size_t)B);
    uint8_t *xs = malloc((size_t)B);
    bk_t b;
    int rc = 0, s = 0;
    if (!un || !xs) { free(un); free(xs); return -4; }
    int64_t lam = LSA_LAM0;
    int64_t e_cur = lsa_energy(g, k, B, Cb, Wl, x);
    for (s = 0; s < steps; s++) {
        /* approximation around x: unaries, submodular n-links, constant */
        int64_t cst = 0;
        for (int l = 0; l < B; l++) un[l] = Cb[l];
        if (bk_alloc(&b, B, B * g->nh)) { rc = -4; break; }
        for (int l = 0; l < B; l++) {
            int64_t z, y, xx, nz, ny, nx;
            int64_t i = g_block_pixel(g, k, l, &z, &y, &xx);
            for (int o = 0; o < g->nh; o++) {
                int64_t j = g_nbr(g, z, y, xx, o, &nz, &ny, &nx);
                if (j < 0 || g_block_of(g, nz, ny, nx) != k) continue;
                int lj = (int)(((nz % g->bd) * g->bh + (ny % g->bh)) * g->bw + (nx % g->bw));
                int64_t w = Wl[(int64_t)o * g_n(g) + i];
                if (w > 0) {
                    bk_edge(&b, l, lj, w, w);
                } else if (w < 0) {
                    int64_t m = -w;
                    un[l] += -m + 2 * m * x[lj];
                    un[lj] += -m + 2 * m * x[l];
                    cst -= 2 * m * x[l] * x[lj];
                }
            }
        }
        for (int l = 0; l < B; l++) b.tr[l] = un[l] + lam * (1 - 2 * (int64_t)x[l]);
        bk_run(&b, xs);
        bk_free(&b);
        int same = 1;
        for (int l = 0; l < B; l++) same &= (xs[l] == x[l]);
        int rec = tr && s < tr->cap;
        if (rec) {
            memcpy(tr->xin + (size_t)s * B, x, (size_t)B);
            memcpy(tr->xout + (size_t)s * B, xs, (size_t)B);
            memcpy(tr->un + (size_t)s * B, un, sizeof(int64_t) * (size_t)B);
            tr->cst[s] = cst;
            tr->lam[s] = lam;
            tr->ecur[s] = e_cur;
            tr->ap[s] = 0;
            tr->enew[s] = 0;
            tr->acc[s] = 0;
        }
        if (same) {
            if (lam == 0) { s++; break; }
            lam /= 4;
            continue;
        }
        /* predicted value of the approximation at x* (at x it equals e_cur) */
        int64_t ap = cst;
        for (int l = 0; l < B; l++) if (xs[l]) ap += un[l];
        for (int l = 0; l < B; l++) {
            int64_t z, y, xx, nz, ny, nx;
            int64_t i = g_block_pixel(g, k, l, &z, &y, &xx);
            for (int o = 0; o < g->nh; o++) {
                int64_t j = g_nbr(g, z, y, xx, o, &nz, &ny, &nx);
                if (j < 0 || g_block_of(g, nz, ny, nx) != k) continue;
                int lj = (int)(((nz % g->bd) * g->bh + (ny % g->bh)) * g->bw + (nx % g->bw));
                int64_t w = Wl[(int64_t)o * g_n(g) + i];
                if (w > 0 && xs[l] != xs[lj]) ap += w;
            }
        }
        int64_t e_new = lsa_energy(g, k, B, Cb, Wl, xs);
        int64_t R = e_cur - e_new, P = e_cur - ap;
        if (rec) {
            tr->ap[s] = ap;
            tr->enew[s] = e_new;
            tr->acc[s] = R > 0;
        }
        if (R > 0) {
            memcpy(x, xs, (size_t)B);
            e_cur = e_new;
            if (4 * R >= 3 * P) lam /= 4;
        } else {
            lam = lam * 4 > 0 ? lam * 4 : 1;
            if (lam > ((int64_t)1 << 50)) lam = (int64_t)1 << 50;
        }
    }
    if (steps_done) *steps_done = s;
    free(un); free(xs);
    return rc;
}

/* Eq. 8 for every block by LSA-TR from the block's labels in yhat (image
 * order, updated in place); C = Eq. 8 unaries (image order). */
int orc_nsm_block_solve(const int64_t *dims, int conn, const int *block, const int64_t *Wl,
                        const int64_t *C, uint8_t *yhat, int steps)
{
    grid_t g;
    if (grid_init(&g, dims, conn, block)) return -1;
    int64_t K = g_nblocks(&g);
    int B = g.bd * g.bh * g.bw;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (int64_t k = 0; k < K; k++) {
        int64_t *Cb = malloc(sizeof(int64_t) * (size_t)B);
        uint8_t *x = malloc((size_t)B);
        int64_t *gi = malloc(sizeof(int64_t) * (size_t)B);
        if (!Cb || !x || !gi) { err |= 1; free(Cb); free(x); free(gi); continue; }
        for (int l = 0; l < B; l++) {
            int64_t z, y, xx;
            gi[l] = g_block_pixel(&g, k, l, &z, &y, &xx);
            Cb[l] = C[gi[l]];
            x[l] = yhat[gi[l]];
        }
        if (lsa_tr_block(&g, k, Cb, Wl, x, steps, NULL)) err |= 1;
        for (int l = 0; l < B; l++) yhat[gi[l]] = x[l];
        free(Cb); free(x); free(gi);
    }
    return err ? -1 : 0;
}

/* Algorithm 1 with LSA-TR block solves (Q = I); yhat^0 = 0 and each
 * iteration's LSA-TR starts from the block's previous labels.  Same loop and
 * outputs as orc_admm. */
int orc_nsm_admm(const int64_t *dims, int conn, const int *block, const int64_t *U, const int64_t *Wl,
                 double mu0, double mu_fact, double eps, int max_iter, int steps, uint8_t *labels,
                 int *iters, double *rmax_trace, double *y_out, double *a_out, double *mu_out)
{
    grid_t g;
    if (grid_init(&g, dims, conn, block)) return -1;
    int64_t n = g_n(&g), K = g_nblocks(&g);
    double *y = malloc(sizeof(double) * (size_t)n);
    double *a = malloc(sizeof(double) * (size_t)n);
    double *r2 = malloc(sizeof(double) * (size_t)K);
    int64_t *C = malloc(sizeof(int64_t) * (size_t)n);
    if (!y || !a || !r2 || !C) { free(y); free(a); free(r2); free(C); return -4; }
    for (int64_t i = 0; i < n; i++) { y[i] = 0.5; a[i] = 0.0; labels[i] = 0; }
    double mu = mu0;
    int t = 0, rc = 1;
    while (t < max_iter) {
        orc_shifted_caps(dims, conn, block, U, Wl, y, a, mu, NULL, C);
        orc_nsm_block_solve(dims, conn, block, Wl, C, labels, steps);
        orc_update(dims, conn, block, Wl, labels, mu, y, a, r2);
        double m2 = 0.0;
        for (int64_t k = 0; k < K; k++) if (r2[k] > m2) m2 = r2[k];
        double rmax = sqrt(m2);
        if (rmax_trace) rmax_trace[t] = rmax;
        mu = mu * mu_fact;
        t++;
        if (!(rmax > eps)) { rc = 0; break; }
    }
    *iters = t;
    if (y_out) memcpy(y_out, y, sizeof(double) * (size_t)n);
    if (a_out) memcpy(a_out, a, sizeof(double) * (size_t)n);
    if (mu_out) *mu_out = mu;
    free(y); free(a); free(r2); free(C);
    return rc;
}

/* Test hook: LSA-TR on block k of the grid from labels x (block-local order,
 * updated in place) with the block unaries Cb (local order), recording every
 * step (lsa_trace_t).  Returns the number of steps run, or < 0 on error. */
int orc_lsa_tr_block_trace(const int64_t *dims, int conn, const int *block, const int64_t *Wl, int64_t k,
                           const int64_t *Cb, uint8_t *x, int steps, int cap, uint8_t *xin, uint8_t *xout,
                           int64_t *un, int64_t *cst, int64_t *lam, int64_t *ecur, int64_t *ap, int64_t *enew,
                           int *acc)
{
    grid_t g;
    if (grid_init(&g, dims, conn, block)) return -1;
    if (k < 0 || k >= g_nblocks(&g)) return -1;
    lsa_trace_t tr = {cap, xin, xout, un, cst, lam, ecur, ap, enew, acc};
    int done = 0;
    if (lsa_tr_block_traced(&g, k, Cb, Wl, x, steps, &done, &tr)) return -4;
    return done;
}

/* Serial LSA-TR on the whole grid (one block = the grid) from x = 0: the
 * non-submodular counterpart of sGC the paper compares against (Table 3).
 * Returns E_int of the result. */
int64_t orc_lsa_tr_global(const int64_t *dims, int conn, const int64_t *U, const int64_t *Wl,
                          int steps, uint8_t *labels)
{
    int whole[3] = {(int)dims[0], (int)dims[1], (int)dims[2]};
    grid_t g;
    if (grid_init(&g, dims, conn, whole)) return INT64_MIN;
    int64_t n = g_n(&g);
    if (n > 0x7fffffff / (g.nh + 1)) return INT64_MIN;
    memset(labels, 0, (size_t)n);
    if (lsa_tr_block(&g, 0, U, Wl, labels, steps, NULL)) return INT64_MIN;
    return orc_energy(dims, conn, whole, U, Wl, labels);
}
