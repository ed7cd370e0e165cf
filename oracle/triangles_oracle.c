/* CPU oracle for triangle counting by a masked sparse product (the
 * triangle-counting experiment of Section 4.1, after Wolf et al.): the
 * vertices of an undirected graph (a symmetric pattern without self loops)
 * are relabelled in order of non-decreasing degree, L is the strictly lower
 * triangle of the relabelled pattern, and the number of triangles is the sum
 * of (L*L) masked by L, i.e. the sum over stored L_ij of the number of
 * common entries of rows i and j of L.  Each triangle x > y > z (in the new
 * labels) is counted once, at the stored L_xy with common entry z.
 *
 * Written as that definition: rows of L sorted, common entries counted by
 * merging two sorted rows.  No bitmasks, no hashing, nothing shared with the
 * CUDA library.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU baseline, never by the product path. */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t deg;
    int64_t v;
} deg_key;

static int cmp_deg(const void *x, const void *y) {
    const deg_key *a = (const deg_key *)x, *b = (const deg_key *)y;
    if (a->deg != b->deg) return a->deg < b->deg ? -1 : 1;
    return (a->v > b->v) - (a->v < b->v);
}

static int cmp_i64(const void *x, const void *y) {
    int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
    return (a > b) - (a < b);
}

/* Degree order: perm[u] = position of (deg(u), u) in ascending order. */
int oracle_degree_order(int64_t n, const int64_t *rp, int64_t *perm) {
    deg_key *k = (deg_key *)malloc(sizeof(deg_key) * (size_t)(n > 0 ? n : 1));
    if (!k) return -1;
    for (int64_t u = 0; u < n; u++) {
        k[u].deg = rp[u + 1] - rp[u];
        k[u].v = u;
    }
    qsort(k, (size_t)n, sizeof(deg_key), cmp_deg);
    for (int64_t i = 0; i < n; i++) perm[k[i].v] = i;
    free(k);
    return 0;
}

/* Total number of triangles; perm_in: new label of every vertex (NULL: the
 * degree order above); row_counts (may be NULL): for every original vertex
 * u, the triangles counted in row perm[u] of L (those whose highest-labelled
 * vertex is u).  Returns the total, -1 on allocation failure, -2 if perm_in
 * is not a permutation of 0..n-1. */
int64_t oracle_triangles(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *perm_in,
                         int64_t *row_counts) {
    const size_t nn = (size_t)(n > 0 ? n : 1);
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * nn);
    int64_t *iperm = (int64_t *)malloc(sizeof(int64_t) * nn);
    int64_t *lrp = (int64_t *)calloc(nn + 1, sizeof(int64_t));
    if (!perm || !iperm || !lrp) { free(perm); free(iperm); free(lrp); return -1; }
    if (perm_in) {
        memcpy(perm, perm_in, sizeof(int64_t) * (size_t)n);
    } else if (oracle_degree_order(n, rp, perm) != 0) {
        free(perm); free(iperm); free(lrp);
        return -1;
    }
    for (int64_t i = 0; i < n; i++) iperm[i] = -1;
    for (int64_t u = 0; u < n; u++) {
        if (perm[u] < 0 || perm[u] >= n || iperm[perm[u]] != -1) {
            free(perm); free(iperm); free(lrp);
            return -2;
        }
        iperm[perm[u]] = u;
    }
    /* rows of L: row perm[u] holds perm[v] for the neighbours v of u with a
     * smaller label, sorted */
    for (int64_t u = 0; u < n; u++) {
        int64_t c = 0;
        for (int64_t p = rp[u]; p < rp[u + 1]; p++) c += perm[col[p]] < perm[u];
        lrp[perm[u] + 1] = c;
    }
    for (int64_t i = 0; i < n; i++) lrp[i + 1] += lrp[i];
    int64_t *lcol = (int64_t *)malloc(sizeof(int64_t) * (size_t)(lrp[n] > 0 ? lrp[n] : 1));
    if (!lcol) { free(perm); free(iperm); free(lrp); return -1; }
    for (int64_t u = 0; u < n; u++) {
        int64_t w = lrp[perm[u]];
        for (int64_t p = rp[u]; p < rp[u + 1]; p++)
            if (perm[col[p]] < perm[u]) lcol[w++] = perm[col[p]];
        qsort(lcol + lrp[perm[u]], (size_t)(w - lrp[perm[u]]), sizeof(int64_t), cmp_i64);
    }
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : total)
    for (int64_t i = 0; i < n; i++) {
        int64_t t = 0;
        for (int64_t p = lrp[i]; p < lrp[i + 1]; p++) {
            const int64_t j = lcol[p];
            int64_t x = lrp[i], y = lrp[j];
            while (x < lrp[i + 1] && y < lrp[j + 1]) {
                if (lcol[x] < lcol[y]) x++;
                else if (lcol[x] > lcol[y]) y++;
                else { t++; x++; y++; }
            }
        }
        if (row_counts) row_counts[iperm[i]] = t;
        total += t;
    }
    free(perm); free(iperm); free(lrp); free(lcol);
    return total;
}
