/*
 * Oracle (TEST INFRASTRUCTURE ONLY): constraint-incompatibility graph and
 * DSatur colouring, in plain C so the 200k-point workload colours in seconds.
 *
 * Definition 4.1 (constraint incompatibility graph): one vertex per distinct
 * sampling-constraint set (eq. h1constraints: Omega(I_beta) = G_beta, zero on
 * S \ {beta}); two vertices are joined when no test matrix can satisfy both.
 * Two constraint sets u, v conflict exactly when one requires random rows on a
 * box that the other requires to be zero:
 *      beta_u != beta_v  and  (beta_u in S_v  or  beta_v in S_u).
 * (Same beta: both ask for the same G_beta there, so they are compatible.)
 *
 * DSatur (Algorithm 2.3): repeatedly colour the uncoloured vertex with the
 * largest saturation (number of distinct colours among its neighbours) with the
 * smallest colour none of its neighbours uses.  Ties (the paper keys only on
 * saturation) are broken by larger degree, then by smaller vertex id.
 *
 * This file is written for clarity: neighbour sets are built from the
 * definition with a marker array, and selection is a linear scan.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* S sets in CSR form: s_ptr[v]..s_ptr[v+1] (sorted box ids), beta[v] in [0, nbox). */
static int build_adjacency(int nv, int nbox, const int *beta, const int64_t *s_ptr,
                           const int *s_idx, int64_t **adj_ptr_out, int **adj_out)
{
    /* vertices grouped by beta, and by boxes contained in their S */
    int64_t *bptr = calloc((size_t)nbox + 1, sizeof(int64_t));
    int64_t *cptr = calloc((size_t)nbox + 1, sizeof(int64_t));
    if (!bptr || !cptr) return -1;
    for (int v = 0; v < nv; ++v) {
        bptr[beta[v] + 1]++;
        for (int64_t t = s_ptr[v]; t < s_ptr[v + 1]; ++t) cptr[s_idx[t] + 1]++;
    }
    for (int b = 0; b < nbox; ++b) { bptr[b + 1] += bptr[b]; cptr[b + 1] += cptr[b]; }
    int *bv = malloc(sizeof(int) * (size_t)(bptr[nbox] + 1));
    int *cv = malloc(sizeof(int) * (size_t)(cptr[nbox] + 1));
    int64_t *bfill = malloc(sizeof(int64_t) * (size_t)(nbox + 1));
    int64_t *cfill = malloc(sizeof(int64_t) * (size_t)(nbox + 1));
    if (!bv || !cv || !bfill || !cfill) return -1;
    memcpy(bfill, bptr, sizeof(int64_t) * (size_t)(nbox + 1));
    memcpy(cfill, cptr, sizeof(int64_t) * (size_t)(nbox + 1));
    for (int v = 0; v < nv; ++v) {
        bv[bfill[beta[v]]++] = v;
        for (int64_t t = s_ptr[v]; t < s_ptr[v + 1]; ++t) cv[cfill[s_idx[t]]++] = v;
    }

    int *mark = malloc(sizeof(int) * (size_t)(nv + 1));
    int64_t *aptr = malloc(sizeof(int64_t) * (size_t)(nv + 1));
    int64_t cap = 1024, len = 0;
    int *adj = malloc(sizeof(int) * (size_t)cap);
    if (!mark || !aptr || !adj) return -1;
    for (int v = 0; v < nv; ++v) mark[v] = -1;
    aptr[0] = 0;
    for (int u = 0; u < nv; ++u) {
        /* beta_v in S_u, beta_v != beta_u */
        for (int64_t t = s_ptr[u]; t < s_ptr[u + 1]; ++t) {
            int g = s_idx[t];
            if (g == beta[u]) continue;
            for (int64_t w = bptr[g]; w < bptr[g + 1]; ++w) {
                int v = bv[w];
                if (mark[v] == u) continue;
                mark[v] = u;
                if (len == cap) { cap *= 2; adj = realloc(adj, sizeof(int) * (size_t)cap); if (!adj) return -1; }
                adj[len++] = v;
            }
        }
        /* beta_u in S_v, beta_v != beta_u */
        for (int64_t w = cptr[beta[u]]; w < cptr[beta[u] + 1]; ++w) {
            int v = cv[w];
            if (beta[v] == beta[u] || mark[v] == u) continue;
            mark[v] = u;
            if (len == cap) { cap *= 2; adj = realloc(adj, sizeof(int) * (size_t)cap); if (!adj) return -1; }
            adj[len++] = v;
        }
        aptr[u + 1] = len;
    }
    free(bptr); free(cptr); free(bv); free(cv); free(bfill); free(cfill); free(mark);
    *adj_ptr_out = aptr;
    *adj_out = adj;
    return 0;
}

/* DSatur on an adjacency list (CSR, both directions). */
static int dsatur(int nv, const int64_t *aptr, const int *adj, int *color, int *degree_out)
{
    /* a greedy colouring never needs more than max degree + 1 colours */
    int maxc = 1;
    for (int v = 0; v < nv; ++v)
        if (aptr[v + 1] - aptr[v] + 1 > maxc) maxc = (int)(aptr[v + 1] - aptr[v] + 1);
    /* forbidden[v * maxc + c] != 0 when a neighbour of v has colour c */
    unsigned char *forb = calloc((size_t)nv * (size_t)maxc, 1);
    int *sat = calloc((size_t)nv, sizeof(int));
    if (!forb || !sat) return -1;
    int nc = 0;
    for (int v = 0; v < nv; ++v) {
        color[v] = -1;
        degree_out[v] = (int)(aptr[v + 1] - aptr[v]);
    }
    for (int step = 0; step < nv; ++step) {
        int best = -1;
        for (int v = 0; v < nv; ++v) {
            if (color[v] >= 0) continue;
            if (best < 0 || sat[v] > sat[best] ||
                (sat[v] == sat[best] && degree_out[v] > degree_out[best]))
                best = v;           /* scanning v upward keeps the smaller id on ties */
        }
        int c = 0;
        while (forb[(size_t)best * maxc + c]) ++c;
        color[best] = c;
        if (c + 1 > nc) nc = c + 1;
        for (int64_t t = aptr[best]; t < aptr[best + 1]; ++t) {
            int w = adj[t];
            unsigned char *f = &forb[(size_t)w * maxc + c];
            if (!*f) { *f = 1; sat[w]++; }
        }
    }
    free(forb); free(sat);
    return nc;
}

/*
 * Colour the graph.  Returns the number of colours (>= 0) or -1 on failure.
 * n_edges_out receives the number of undirected edges.
 */
int oracle_color(int nv, int nbox, const int *beta, const int64_t *s_ptr, const int *s_idx,
                 int *color, int64_t *n_edges_out, int *degree_out)
{
    int64_t *aptr = NULL;
    int *adj = NULL;
    if (nv <= 0 || nbox <= 0) { *n_edges_out = 0; return nv == 0 ? 0 : -1; }
    if (build_adjacency(nv, nbox, beta, s_ptr, s_idx, &aptr, &adj)) return -1;
    *n_edges_out = aptr[nv] / 2;
    int nc = dsatur(nv, aptr, adj, color, degree_out);
    free(aptr); free(adj);
    return nc;
}

/*
 * Constraint sets with several random boxes (Section 4.2, eq.
 * unifh1constraints: box alpha asks for G_beta on every beta of int(alpha) and
 * zeros on near(alpha)): vertex v asks for random rows on the boxes G_v and
 * zeros on the boxes Z_v.  Two vertices conflict exactly when one asks for
 * random rows on a box the other asks to be zero:
 *      (G_u and Z_v intersect)  or  (G_v and Z_u intersect).
 * Coloured with the same DSatur.  Returns the number of colours or -1.
 */
int oracle_color_sets(int nv, int nbox, const int64_t *g_ptr, const int *g_idx, const int64_t *z_ptr,
                      const int *z_idx, int *color, int64_t *n_edges_out, int *degree_out)
{
    if (nv <= 0 || nbox <= 0) { *n_edges_out = 0; return nv == 0 ? 0 : -1; }
    /* for every box: the vertices asking for random rows, and for zeros, on it */
    int64_t *gp = calloc((size_t)nbox + 1, sizeof(int64_t)), *zp = calloc((size_t)nbox + 1, sizeof(int64_t));
    if (!gp || !zp) return -1;
    for (int v = 0; v < nv; ++v) {
        for (int64_t t = g_ptr[v]; t < g_ptr[v + 1]; ++t) gp[g_idx[t] + 1]++;
        for (int64_t t = z_ptr[v]; t < z_ptr[v + 1]; ++t) zp[z_idx[t] + 1]++;
    }
    for (int b = 0; b < nbox; ++b) { gp[b + 1] += gp[b]; zp[b + 1] += zp[b]; }
    int *gv = malloc(sizeof(int) * (size_t)(gp[nbox] + 1)), *zv = malloc(sizeof(int) * (size_t)(zp[nbox] + 1));
    int64_t *gf = malloc(sizeof(int64_t) * (size_t)(nbox + 1)), *zf = malloc(sizeof(int64_t) * (size_t)(nbox + 1));
    int *mark = malloc(sizeof(int) * (size_t)(nv + 1));
    int64_t *aptr = malloc(sizeof(int64_t) * (size_t)(nv + 1));
    int64_t cap = 1024, len = 0;
    int *adj = malloc(sizeof(int) * (size_t)cap);
    if (!gv || !zv || !gf || !zf || !mark || !aptr || !adj) return -1;
    memcpy(gf, gp, sizeof(int64_t) * (size_t)(nbox + 1));
    memcpy(zf, zp, sizeof(int64_t) * (size_t)(nbox + 1));
    for (int v = 0; v < nv; ++v) {
        for (int64_t t = g_ptr[v]; t < g_ptr[v + 1]; ++t) gv[gf[g_idx[t]]++] = v;
        for (int64_t t = z_ptr[v]; t < z_ptr[v + 1]; ++t) zv[zf[z_idx[t]]++] = v;
        mark[v] = -1;
    }
    aptr[0] = 0;
    for (int u = 0; u < nv; ++u) {
        for (int pass = 0; pass < 2; ++pass) {
            /* pass 0: boxes of G_u asked zero by v; pass 1: boxes of Z_u asked random by v */
            const int64_t *sp = pass ? z_ptr : g_ptr;
            const int *si = pass ? z_idx : g_idx;
            const int64_t *op = pass ? gp : zp;
            const int *ov = pass ? gv : zv;
            for (int64_t t = sp[u]; t < sp[u + 1]; ++t) {
                int b = si[t];
                for (int64_t w = op[b]; w < op[b + 1]; ++w) {
                    int v = ov[w];
                    if (v == u || mark[v] == u) continue;
                    mark[v] = u;
                    if (len == cap) { cap *= 2; adj = realloc(adj, sizeof(int) * (size_t)cap); if (!adj) return -1; }
                    adj[len++] = v;
                }
            }
        }
        aptr[u + 1] = len;
    }
    free(gp); free(zp); free(gv); free(zv); free(gf); free(zf); free(mark);
    *n_edges_out = aptr[nv] / 2;
    int nc = dsatur(nv, aptr, adj, color, degree_out);
    free(aptr); free(adj);
    return nc;
}
