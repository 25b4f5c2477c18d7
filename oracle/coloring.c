/* Oracle: exhaustive search for the torus colouring of Sec. 3, Eq. 15
 *     c(x) = sum_j sigma_j x_j  mod n_c
 * TEST INFRASTRUCTURE ONLY -- never linked into the product library.
 *
 * Validity (Sec. 3): every two distinct sites whose wrap-around (torus) L1
 * distance is <= d get different colours.  Reading of the search the paper
 * leaves open ("an appropriate exhaustive search", Sec. 3): n_c ascending
 * from 2; for each n_c, sigma in [0, n_c)^{n_D} in lexicographic order
 * (sigma_1 most significant); the first valid pair is returned.
 *
 * The check: list every nonzero torus displacement D (D_j in [0, L_j))
 * within distance d; two sites with that displacement differ in integer
 * coordinates by e_j = D_j or D_j - L_j (both occur when D_j != 0), so sigma
 * is valid iff sum_j sigma_j e_j != 0 (mod n_c) for every such e.
 *
 * The enumeration of sigma is a depth-first walk in lexicographic order; the
 * condition of a difference vector e whose last nonzero component is k is
 * tested as soon as sigma_0..sigma_k are fixed, and a failing prefix skips
 * its whole subtree.  This only drops tuples that would fail anyway, so the
 * first valid tuple is the same as in a flat lexicographic scan.
 */
#include <stdlib.h>
#include <string.h>

#define MAXD 8

typedef struct {
    int nD, nc;
    int *e;          /* difference vectors grouped by last nonzero component */
    int start[MAXD + 1];
    int s[MAXD];
} search_t;

static int torus_dist1(int D, int L) { int a = D, b = L - D; return a < b ? a : b; }

/* every integer difference vector e of a torus displacement within distance d,
 * grouped by the index of its last nonzero component */
static void build_diffs(search_t *S, const int *L, int d)
{
    int nD = S->nD;
    long total = 1;
    for (int j = 0; j < nD; ++j) total *= L[j];
    int cap = 1024, n = 0;
    int *e = (int *)malloc(sizeof(int) * cap * nD);
    int *grp = (int *)malloc(sizeof(int) * cap);
    int D[MAXD];
    for (long code = 1; code < total; ++code) {           /* code 0 = zero displacement */
        long c = code; int dist = 0;
        for (int j = nD - 1; j >= 0; --j) { D[j] = (int)(c % L[j]); c /= L[j]; }
        for (int j = 0; j < nD; ++j) dist += torus_dist1(D[j], L[j]);
        if (dist > d) continue;
        int nz[MAXD], nnz = 0;
        for (int j = 0; j < nD; ++j) if (D[j] != 0) nz[nnz++] = j;
        for (int w = 0; w < (1 << nnz); ++w) {
            if (n == cap) {
                cap *= 2;
                e = (int *)realloc(e, sizeof(int) * cap * nD);
                grp = (int *)realloc(grp, sizeof(int) * cap);
            }
            for (int j = 0; j < nD; ++j) e[n * nD + j] = D[j];
            for (int k = 0; k < nnz; ++k) if (w >> k & 1) e[n * nD + nz[k]] -= L[nz[k]];
            grp[n] = nz[nnz - 1];
            ++n;
        }
    }
    /* stable bucket by group */
    S->e = (int *)malloc(sizeof(int) * (n > 0 ? n : 1) * nD);
    int m = 0;
    for (int k = 0; k < nD; ++k) {
        S->start[k] = m;
        for (int i = 0; i < n; ++i)
            if (grp[i] == k) { memcpy(S->e + m * nD, e + i * nD, sizeof(int) * nD); ++m; }
    }
    S->start[nD] = m;
    free(e); free(grp);
}

static int group_ok(const search_t *S, int k)
{
    for (int i = S->start[k]; i < S->start[k + 1]; ++i) {
        long v = 0;
        for (int j = 0; j <= k; ++j) v += (long)S->s[j] * S->e[i * S->nD + j];
        v %= S->nc; if (v < 0) v += S->nc;
        if (v == 0) return 0;
    }
    return 1;
}

static int dfs(search_t *S, int k)
{
    if (k == S->nD) return 1;
    for (int v = 0; v < S->nc; ++v) {
        S->s[k] = v;
        if (group_ok(S, k) && dfs(S, k + 1)) return 1;
    }
    return 0;
}

/* Returns n_c (>= 2) and writes sigma[nD]; returns 0 if no colouring with
 * n_c <= max_nc exists. */
int oracle_torus_coloring(int nD, const int *L, int d, int max_nc, int *sigma)
{
    search_t S; S.nD = nD;
    build_diffs(&S, L, d);
    for (int nc = 2; nc <= max_nc; ++nc) {
        S.nc = nc;
        if (dfs(&S, 0)) {
            memcpy(sigma, S.s, sizeof(int) * nD);
            free(S.e);
            return nc;
        }
    }
    free(S.e);
    return 0;
}

/* Is there any sigma giving a valid colouring with exactly nc colours?
 * (used to examine Table 1's entries); writes the lexicographically first. */
int oracle_coloring_exists(int nD, const int *L, int d, int nc, int *sigma)
{
    search_t S; S.nD = nD; S.nc = nc;
    build_diffs(&S, L, d);
    int ok = dfs(&S, 0);
    if (ok) memcpy(sigma, S.s, sizeof(int) * nD);
    free(S.e);
    return ok;
}
