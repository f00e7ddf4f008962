// Constraint-incompatibility graph and DSatur colouring on the GPU
// (Definition 4.1, Algorithm 2.3, Sections 4.1.2-4.1.3).
//
//  K4  vertices: the sampling constraint of pair (alpha, beta) is fixed by the
//      key (beta, S_alpha), S_alpha = near(alpha) u int(alpha) (near(alpha) only
//      for the leaf neighbour pairs).  A pair is a new vertex unless an earlier
//      pair (alpha' < alpha, same beta) has the same S; such an alpha' must lie
//      in S_alpha, so the test only scans S_alpha.  Vertex ids are in order of
//      first occurrence.
//      Edges: u ~ v iff beta_u != beta_v and (beta_u in S_v or beta_v in S_u).
//      By the symmetry of the lists, beta_u in S_v <=> alpha_v in S(beta_u), so
//      the neighbours of u are the vertices whose beta lies in S_u and the
//      vertices of pairs whose row box lies in S(beta_u).  Each CTA marks them
//      in a shared-memory bitmap and reads the sorted list back out of it.
//  K5  DSatur in one CTA: the uncoloured vertex with the largest (saturation,
//      degree, -id) takes the smallest colour unused by its neighbours.
//      Vertices are spread over 1024 buckets whose maxima live in shared memory;
//      each step re-scans only the bucket of the coloured vertex.
#include "ctx.cuh"

#include <algorithm>

namespace hm {

constexpr int DS_BUCKETS = 1024;
constexpr int VID_BITS = 20;                 // vertex ids < 2^20
constexpr unsigned long long VID_MASK = (1ull << VID_BITS) - 1;
constexpr int DEG_SHIFT = 20, SAT_SHIFT = 40;
constexpr unsigned long long UNCOLORED = 1ull << 62;
constexpr int FORB_WORDS = MAX_COLORS / 32;

__device__ __forceinline__ int find_in(const int *a, int lo, int hi, int key) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_pair_alpha(const int *ptr, int nc, int *alpha) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nc) return;
    for (int p = ptr[a]; p < ptr[a + 1]; ++p) alpha[p] = a;
}

// transpose index and first-occurrence test of every pair
__global__ void k_pair_keys(const int *ptr, const int *col, const int *alpha, int64_t np, const int *sptr,
                            const int *sidx, int *pairT, int64_t *first, int *rep) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int a = alpha[p], b = col[p];
    pairT[p] = ptr[b] + find_in(col, ptr[b], ptr[b + 1], a) - ptr[b];
    const int s0 = sptr[a], s1 = sptr[a + 1];
    int r = -1;
    for (int t = s0; t < s1 && r < 0; ++t) {
        const int a2 = sidx[t];
        if (a2 >= a) break;
        const int q = find_in(col, ptr[a2], ptr[a2 + 1], b);
        if (q >= ptr[a2 + 1] || col[q] != b) continue;
        if (sptr[a2 + 1] - sptr[a2] != s1 - s0) continue;
        bool same = true;
        for (int u = 0; u < s1 - s0 && same; ++u) same = sidx[sptr[a2] + u] == sidx[s0 + u];
        if (same) r = q;
    }
    first[p] = (r < 0);
    rep[p] = (r < 0) ? (int)p : r;
}

__global__ void k_vertex_ids(const int64_t *first, const int64_t *scan, const int *rep, const int *col,
                             int64_t np, int *pair_vertex, int *vertex_pair, int *vertex_beta) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int v = (int)scan[rep[p]];
    pair_vertex[p] = v;
    if (first[p]) {
        vertex_pair[v] = (int)p;
        vertex_beta[v] = col[p];
    }
}

// vertices grouped by beta, in vertex order: box b's vertices are the first
// occurrences among the pairs (a, b), a in list(b), taken in order of a.
__global__ void k_vby_beta(const int *ptr, const int *pairT, const int64_t *first, const int *pair_vertex,
                           int nc, int pass, int *cnt, const int64_t *off, int *out) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nc) return;
    int k = 0;
    for (int t = ptr[b]; t < ptr[b + 1]; ++t) {
        const int p = pairT[t];  // pair (a, b)
        if (first[p]) {
            if (pass) out[off[b] + k] = pair_vertex[p];
            ++k;
        }
    }
    if (!pass) cnt[b] = k;
}

// neighbours of vertex u through a shared-memory bitmap over all vertices
__global__ void k_edges(int64_t nv, const int *vertex_pair, const int *vertex_beta, const int *alpha,
                        const int *ptr, const int *pair_vertex, const int *sptr, const int *sidx,
                        const int *vb_ptr, const int *vb_idx, int pass, int *deg, const int64_t *adj_ptr,
                        int *adj) {
    extern __shared__ unsigned int bm[];
    __shared__ int wsum[32];
    const int u = blockIdx.x;
    const int nw = (int)((nv + 31) >> 5);
    for (int i = threadIdx.x; i < nw; i += blockDim.x) bm[i] = 0u;
    __syncthreads();
    const int au = alpha[vertex_pair[u]], bu = vertex_beta[u];
    // beta_v in S_u, beta_v != beta_u
    for (int t = sptr[au]; t < sptr[au + 1]; ++t) {
        const int g = sidx[t];
        if (g == bu) continue;
        for (int q = vb_ptr[g] + threadIdx.x; q < vb_ptr[g + 1]; q += blockDim.x) {
            const int v = vb_idx[q];
            atomicOr(&bm[v >> 5], 1u << (v & 31));
        }
    }
    // alpha_v in S(beta_u), beta_v != beta_u
    for (int t = sptr[bu]; t < sptr[bu + 1]; ++t) {
        const int a2 = sidx[t];
        for (int p = ptr[a2] + threadIdx.x; p < ptr[a2 + 1]; p += blockDim.x) {
            const int v = pair_vertex[p];
            if (vertex_beta[v] == bu) continue;
            atomicOr(&bm[v >> 5], 1u << (v & 31));
        }
    }
    __syncthreads();
    // contiguous word ranges per thread -> sorted output
    const int per = (nw + blockDim.x - 1) / blockDim.x;
    const int w0 = threadIdx.x * per, w1 = min(nw, w0 + per);
    int c = 0;
    for (int w = w0; w < w1; ++w) c += __popc(bm[w]);
    if (!pass) {
        c = block_sum(c, wsum);
        if (threadIdx.x == 0) deg[u] = c;
        return;
    }
    // exclusive prefix of c across threads
    __shared__ int pre[1024];
    pre[threadIdx.x] = c;
    __syncthreads();
    for (int o = 1; o < blockDim.x; o <<= 1) {
        int v = (threadIdx.x >= o) ? pre[threadIdx.x - o] : 0;
        __syncthreads();
        pre[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t o = adj_ptr[u] + pre[threadIdx.x] - c;
    for (int w = w0; w < w1; ++w) {
        unsigned int x = bm[w];
        while (x) {
            const int bit = __ffs(x) - 1;
            x &= x - 1;
            adj[o++] = w * 32 + bit;
        }
    }
}

// Uniform H^1 (Section 4.2, eq. unifh1constraints): box alpha asks for random
// rows on int(alpha) and zeros on near(alpha); u ~ v iff int(a_u) meets
// near(a_v) or near(a_u) meets int(a_v).  By the symmetry of both lists the
// neighbours of u are the vertex boxes in near(d) for d in int(a_u) and in
// int(d) for d in near(a_u).  vid: box -> vertex id (-1: no interaction list).
__global__ void k_box_edges(int64_t nv, const int *vbox, const int *vid, const int *near_ptr, const int *near_idx,
                            const int *int_ptr, const int *int_idx, int pass, int *deg, const int64_t *adj_ptr,
                            int *adj) {
    extern __shared__ unsigned int bm[];
    __shared__ int wsum[32];
    __shared__ int pre[1024];
    const int u = blockIdx.x;
    const int nw = (int)((nv + 31) >> 5);
    for (int i = threadIdx.x; i < nw; i += blockDim.x) bm[i] = 0u;
    __syncthreads();
    const int a = vbox[u];
    for (int h = 0; h < 2; ++h) {
        const int *p1 = h ? near_ptr : int_ptr, *i1 = h ? near_idx : int_idx;   // d in int(a), then near(a)
        const int *p2 = h ? int_ptr : near_ptr, *i2 = h ? int_idx : near_idx;   // b in near(d), then int(d)
        for (int t = p1[a]; t < p1[a + 1]; ++t) {
            const int d = i1[t];
            for (int q = p2[d] + threadIdx.x; q < p2[d + 1]; q += blockDim.x) {
                const int v = vid[i2[q]];
                if (v >= 0 && v != u) atomicOr(&bm[v >> 5], 1u << (v & 31));
            }
        }
    }
    __syncthreads();
    const int per = (nw + blockDim.x - 1) / blockDim.x;
    const int w0 = threadIdx.x * per, w1 = min(nw, w0 + per);
    int c = 0;
    for (int w = w0; w < w1; ++w) c += __popc(bm[w]);
    if (!pass) {
        c = block_sum(c, wsum);
        if (threadIdx.x == 0) deg[u] = c;
        return;
    }
    pre[threadIdx.x] = c;
    __syncthreads();
    for (int o = 1; o < blockDim.x; o <<= 1) {
        int v = (threadIdx.x >= o) ? pre[threadIdx.x - o] : 0;
        __syncthreads();
        pre[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t o = adj_ptr[u] + pre[threadIdx.x] - c;
    for (int w = w0; w < w1; ++w) {
        unsigned int x = bm[w];
        while (x) {
            const int bit = __ffs(x) - 1;
            x &= x - 1;
            adj[o++] = w * 32 + bit;
        }
    }
}

__global__ void k_box_vertices(const int *int_ptr, int nc, const int64_t *vscan, int *vbox, int *vid) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nc) return;
    const bool has = int_ptr[b + 1] > int_ptr[b];
    vid[b] = has ? (int)vscan[b] : -1;
    if (has) vbox[vscan[b]] = b;
}

__global__ void k_box_has_int(const int *int_ptr, int nc, int64_t *flag) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nc) flag[b] = int_ptr[b + 1] > int_ptr[b] ? 1 : 0;
}

// active (colour, box): every box of int(alpha) for the vertex boxes alpha of the colour
__global__ void k_act_mark_box(const int *vbox, const int *vertex_color, int64_t nv, const int *int_ptr,
                               const int *int_idx, int nc, unsigned char *act) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const int a = vbox[v];
    for (int t = int_ptr[a]; t < int_ptr[a + 1]; ++t) act[(int64_t)vertex_color[v] * nc + int_idx[t]] = 1;
}

__global__ void k_iota(int *x, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = (int)i;
}

__global__ void k_dsatur_init(int64_t nv, const int *deg, unsigned long long *key, unsigned int *forb) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= nv) return;
    key[v] = UNCOLORED | ((unsigned long long)deg[v] << DEG_SHIFT) | (VID_MASK - (unsigned long long)v);
    for (int w = 0; w < FORB_WORDS; ++w) forb[v * FORB_WORDS + w] = 0u;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
        v = t > v ? t : v;
    }
    return v;
}

// One CTA of 1024 threads; exactly nv steps, no waits on other blocks.
// Per step: (1) every warp reduces the 1024 bucket maxima, so the chosen
// vertex v is known after one barrier; (2) in parallel, warp 0 finds v's
// smallest free colour, every thread fetches its share of v's neighbours
// together with their keys and first four forbidden-colour words (colours
// < 128), and warp 1 re-scans v's bucket without v; (3) neighbours take the
// colour into their forbidden sets and raise their saturation.
constexpr int DS_PREFETCH = 2;  // neighbours fetched ahead per thread

__global__ void __launch_bounds__(1024) k_dsatur(int64_t nv, const int64_t *adj_ptr, const int *adj,
                                                 unsigned long long *key, unsigned int *forb, int *color,
                                                 int *status /* [0] = colours, [1] = error */) {
    __shared__ unsigned long long bmax[DS_BUCKETS];
    __shared__ unsigned long long red[32];
    __shared__ int sel_c, ncol;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    unsigned long long m0 = 0;
    for (int64_t v = t; v < nv; v += DS_BUCKETS) m0 = key[v] > m0 ? key[v] : m0;
    bmax[t] = m0;
    if (t == 0) ncol = 0;
    __syncthreads();
    for (int64_t step = 0; step < nv; ++step) {
        unsigned long long k = warp_max_u64(bmax[t]);
        if (lane == 0) red[w] = k;
        __syncthreads();
        k = warp_max_u64(red[lane]);
        const int v = (int)(VID_MASK - (k & VID_MASK));
        const int b = v & (DS_BUCKETS - 1);
        const int64_t e0 = adj_ptr[v], e1 = adj_ptr[v + 1];
        // neighbours, their keys and forbidden words 0..3, fetched before the colour is known
        int nu[DS_PREFETCH];
        unsigned long long nk[DS_PREFETCH];
        uint4 nf[DS_PREFETCH];
#pragma unroll
        for (int h = 0; h < DS_PREFETCH; ++h) {
            const int64_t e = e0 + t + (int64_t)h * blockDim.x;
            nu[h] = -1;
            if (e < e1) {
                nu[h] = adj[e];
                nk[h] = key[nu[h]];
                nf[h] = *reinterpret_cast<const uint4 *>(&forb[(int64_t)nu[h] * FORB_WORDS]);
            }
        }
        if (w == 0) {
            const unsigned int freebits = ~forb[(int64_t)v * FORB_WORDS + lane];
            const unsigned int has = __ballot_sync(0xffffffffu, freebits != 0u);
            if (lane == 0) sel_c = -1;
            __syncwarp();
            if (has) {
                const int l0 = __ffs(has) - 1;
                if (lane == l0) sel_c = l0 * 32 + __ffs(freebits) - 1;
            }
        } else if (w == 1) {
            unsigned long long mm = 0;
            for (int64_t x = b + (int64_t)lane * DS_BUCKETS; x < nv; x += 32ll * DS_BUCKETS)
                if (x != v) mm = key[x] > mm ? key[x] : mm;
            mm = warp_max_u64(mm);
            if (lane == 0) bmax[b] = mm;  // v leaves its bucket; raises follow by atomicMax
        }
        __syncthreads();
        const int c = sel_c;
        if (c < 0) {
            if (t == 0) status[1] = 1;
            return;  // uniform: every thread reads the same sel_c
        }
        const int cw = c >> 5;
        const unsigned int bit = 1u << (c & 31);
#pragma unroll
        for (int h = 0; h < DS_PREFETCH; ++h) {
            const int u = nu[h];
            if (u < 0 || !(nk[h] & UNCOLORED)) continue;
            unsigned int fw;
            if (cw < 4) fw = cw == 0 ? nf[h].x : (cw == 1 ? nf[h].y : (cw == 2 ? nf[h].z : nf[h].w));
            else fw = forb[(int64_t)u * FORB_WORDS + cw];
            if (!(fw & bit)) {
                forb[(int64_t)u * FORB_WORDS + cw] = fw | bit;
                const unsigned long long ku = nk[h] + (1ull << SAT_SHIFT);
                key[u] = ku;
                atomicMax(&bmax[u & (DS_BUCKETS - 1)], ku);
            }
        }
        // vertices of very large degree: the rest without prefetch
        for (int64_t e = e0 + t + (int64_t)DS_PREFETCH * blockDim.x; e < e1; e += blockDim.x) {
            const int u = adj[e];
            const unsigned long long ku = key[u];
            if (!(ku & UNCOLORED)) continue;
            unsigned int *f = &forb[(int64_t)u * FORB_WORDS + cw];
            const unsigned int fw = *f;
            if (!(fw & bit)) {
                *f = fw | bit;
                key[u] = ku + (1ull << SAT_SHIFT);
                atomicMax(&bmax[u & (DS_BUCKETS - 1)], ku + (1ull << SAT_SHIFT));
            }
        }
        if (t == 0) {
            key[v] = 0ull;
            color[v] = c;
            if (c + 1 > ncol) ncol = c + 1;
        }
        __syncthreads();
    }
    if (t == 0) status[0] = ncol;
}

__global__ void k_pair_color(const int *pair_vertex, const int *vertex_color, int64_t np, int *pair_color) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < np) pair_color[p] = vertex_color[pair_vertex[p]];
}

__global__ void k_act_mark(const int *vertex_beta, const int *vertex_color, int64_t nv, int nc,
                           unsigned char *act) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v < nv) act[(int64_t)vertex_color[v] * nc + vertex_beta[v]] = 1;
}

// colour c -> sorted active entries; one CTA per colour
__global__ void k_act_by_color(const unsigned char *act, int nc, int pass, int *cnt, const int64_t *off,
                               int *out) {
    __shared__ int wsum[32];
    __shared__ int pre[1024];
    const int c = blockIdx.x;
    const unsigned char *row = act + (int64_t)c * nc;
    const int per = (nc + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per, b1 = min(nc, b0 + per);
    int k = 0;
    for (int b = b0; b < b1; ++b) k += row[b];
    if (!pass) {
        k = block_sum(k, wsum);
        if (threadIdx.x == 0) cnt[c] = k;
        return;
    }
    pre[threadIdx.x] = k;
    __syncthreads();
    for (int o = 1; o < blockDim.x; o <<= 1) {
        int v = (threadIdx.x >= o) ? pre[threadIdx.x - o] : 0;
        __syncthreads();
        pre[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t o = off[c] + pre[threadIdx.x] - k;
    for (int b = b0; b < b1; ++b)
        if (row[b]) out[o++] = b;
}

// entry -> sorted colours it is active in
__global__ void k_act_by_entry(const unsigned char *act, int nc, int chi, int pass, int *cnt,
                               const int64_t *off, int *out) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nc) return;
    int k = 0;
    for (int c = 0; c < chi; ++c)
        if (act[(int64_t)c * nc + b]) {
            if (pass) out[off[b] + k] = c;
            ++k;
        }
    if (!pass) cnt[b] = k;
}

// Pairs of colour blockIdx.x in pair order (one CTA per colour): pass 0
// counts them, pass 1 writes their alpha boxes from off[c] on.
__global__ void __launch_bounds__(1024) k_pairs_by_color(const int *pair_color, const int *pair_alpha, int64_t np,
                                                         int pass, int *cnt, const int64_t *off, int *tile_box) {
    __shared__ int wsum[32];
    __shared__ int run;
    const int c = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) run = 0;
    __syncthreads();
    for (int64_t p0 = 0; p0 < np; p0 += 1024) {
        const int64_t p = p0 + t;
        const bool f = p < np && pair_color[p] == c;
        const unsigned int b = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wsum[w] = __popc(b);
        __syncthreads();
        int before = 0, tot = 0;
        for (int k = 0; k < 32; ++k) {
            const int v = wsum[k];
            if (k < w) before += v;
            tot += v;
        }
        if (pass == 1 && f) tile_box[off[c] + run + before + __popc(b & ((1u << lane) - 1u))] = pair_alpha[p];
        __syncthreads();
        if (t == 0) run += tot;
        __syncthreads();
    }
    if (pass == 0 && t == 0) cnt[c] = run;
}

__global__ void k_gather_ptr(const int64_t *rowoff, const int64_t *tptr, int chi, int64_t *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= chi) out[k] = rowoff[tptr[k]];
}

__global__ void k_act_sizes(const int *act_box, int64_t na, const int *ent, int *sz) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= na) return;
    const int *e = ent + (int64_t)act_box[i] * ENT_FIELDS;
    sz[i] = e[4] - e[3];
}

// rows of every (colour, active entry): one warp per entry
__global__ void k_act_rows(const int *act_box, int64_t na, const int *ent, const int64_t *rowoff, int *rows) {
    int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= na) return;
    const int *e = ent + (int64_t)act_box[i] * ENT_FIELDS;
    for (int r = e[3] + lane; r < e[4]; r += 32) rows[rowoff[i] + (r - e[3])] = r;
}

// DSatur over the adjacency (adj_ptr, adj), then the tables the sampler and
// the peel read: pair colours, active boxes per colour (the beta of every
// vertex, or int(alpha) of every vertex box for the uniform box graph),
// colours per box, active rows and output rows per colour.
static Err color_tail(Coloring &g, const Cut &cu, DBuf &adj_ptr, DBuf &adj, bool boxes, cudaStream_t st,
                      DBuf &scan_tmp) {
    const int nc = cu.nc;
    const int64_t np = g.n_pairs, nv = g.n_vertices;
    // DSatur
    DBuf key, forb, status;
    HM_TRY(alloc(key, nv * sizeof(unsigned long long)));
    HM_TRY(alloc(forb, nv * FORB_WORDS * sizeof(unsigned int)));
    HM_TRY(alloc(status, 2 * sizeof(int)));
    HM_CUDA(cudaMemsetAsync(status.p, 0, 2 * sizeof(int), st));
    k_dsatur_init<<<ceil_div(nv, 256), 256, 0, st>>>(nv, g.vertex_degree.as<int>(), key.as<unsigned long long>(),
                                                      forb.as<unsigned int>()); ::hm::count_launch();
    k_dsatur<<<1, 1024, 0, st>>>(nv, adj_ptr.as<int64_t>(), adj.as<int>(), key.as<unsigned long long>(),
                                 forb.as<unsigned int>(), g.vertex_color.as<int>(), status.as<int>()); ::hm::count_launch();
    HM_LAUNCH("dsatur");
    int hs[2];
    HM_CUDA(cudaStreamSynchronize(st));  // DSatur first, then the pageable copy (see to_host)
    HM_CUDA(cudaMemcpyAsync(hs, status.p, sizeof(hs), cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
    if (hs[1]) return fail(HM_ENOTSUP, "colour: more than 1024 colours");
    g.n_colors = hs[0];
    const int chi = g.n_colors;
    k_pair_color<<<ceil_div(np, 256), 256, 0, st>>>(g.pair_vertex.as<int>(), g.vertex_color.as<int>(), np,
                                                    g.pair_color.as<int>()); ::hm::count_launch();
    HM_LAUNCH("pair_color");

    // active tables
    DBuf act, cnt, off64;
    HM_TRY(alloc(act, (size_t)chi * nc));
    HM_CUDA(cudaMemsetAsync(act.p, 0, (size_t)chi * nc, st));
    if (boxes)
        k_act_mark_box<<<ceil_div(nv, 256), 256, 0, st>>>(g.pair_alpha.as<int>(), g.vertex_color.as<int>(), nv,
                                                           cu.int_ptr.as<int>(), cu.int_idx.as<int>(), nc,
                                                           act.as<unsigned char>());
    else
        k_act_mark<<<ceil_div(nv, 256), 256, 0, st>>>(g.vertex_beta.as<int>(), g.vertex_color.as<int>(), nv, nc,
                                                       act.as<unsigned char>());
    ::hm::count_launch();
    HM_TRY(alloc(cnt, std::max(chi, nc) * sizeof(int)));
    HM_TRY(alloc(off64, (std::max(chi, nc) + 1) * sizeof(int64_t)));
    k_act_by_color<<<chi, 1024, 0, st>>>(act.as<unsigned char>(), nc, 0, cnt.as<int>(), nullptr, nullptr); ::hm::count_launch();
    HM_TRY(scan_counts_i32(cnt.as<int>(), off64.as<int64_t>(), chi, st, scan_tmp));
    std::vector<int64_t> hoff;
    HM_TRY(to_host(hoff, off64.p, chi + 1, st));
    const int64_t na = hoff[chi];
    HM_TRY(alloc(g.act_box, na * sizeof(int)));
    k_act_by_color<<<chi, 1024, 0, st>>>(act.as<unsigned char>(), nc, 1, nullptr, off64.as<int64_t>(),
                                         g.act_box.as<int>()); ::hm::count_launch();
    HM_LAUNCH("act_by_color");
    {
        std::vector<int> h32(hoff.begin(), hoff.end());
        HM_TRY(to_dev(g.act_ptr, h32, st));
    }
    k_act_by_entry<<<ceil_div(nc, 128), 128, 0, st>>>(act.as<unsigned char>(), nc, chi, 0, cnt.as<int>(), nullptr,
                                                      nullptr); ::hm::count_launch();
    HM_TRY(scan_counts_i32(cnt.as<int>(), off64.as<int64_t>(), nc, st, scan_tmp));
    {
        std::vector<int64_t> h;
        HM_TRY(to_host(h, off64.p, nc + 1, st));
        HM_TRY(alloc(g.ent_col, std::max<int64_t>(h[nc], 1) * sizeof(int)));
        k_act_by_entry<<<ceil_div(nc, 128), 128, 0, st>>>(act.as<unsigned char>(), nc, chi, 1, nullptr,
                                                          off64.as<int64_t>(), g.ent_col.as<int>()); ::hm::count_launch();
        HM_LAUNCH("act_by_entry");
        std::vector<int> h32(h.begin(), h.end());
        HM_TRY(to_dev(g.ent_cptr, h32, st));
    }
    // rows of each colour
    {
        DBuf sz, rowoff;
        HM_TRY(alloc(sz, std::max<int64_t>(na, 1) * sizeof(int)));
        HM_TRY(alloc(rowoff, (na + 1) * sizeof(int64_t)));
        k_act_sizes<<<ceil_div(na, 256), 256, 0, st>>>(g.act_box.as<int>(), na, cu.ent.as<int>(), sz.as<int>()); ::hm::count_launch();
        HM_TRY(scan_counts_i32(sz.as<int>(), rowoff.as<int64_t>(), na, st, scan_tmp));
        std::vector<int64_t> hro;
        HM_TRY(to_host(hro, rowoff.p, na + 1, st));
        g.n_act_rows = hro[na];
        HM_TRY(alloc(g.act_rows, std::max<int64_t>(g.n_act_rows, 1) * sizeof(int)));
        k_act_rows<<<ceil_div(na * 32, 256), 256, 0, st>>>(g.act_box.as<int>(), na, cu.ent.as<int>(),
                                                           rowoff.as<int64_t>(), g.act_rows.as<int>()); ::hm::count_launch();
        HM_LAUNCH("act_rows");
        std::vector<int64_t> crp(chi + 1);
        for (int k = 0; k <= chi; ++k) crp[k] = hro[hoff[k]];
        HM_TRY(to_dev(g.act_rows_ptr, crp, st));
    }
    // output rows of each colour (rows of the alpha boxes of its pairs)
    {
        DBuf tcnt, tptr, tile_box, sz, rowoff;
        HM_TRY(alloc(tcnt, chi * sizeof(int)));
        HM_TRY(alloc(tptr, (chi + 1) * sizeof(int64_t)));
        HM_TRY(alloc(tile_box, np * sizeof(int)));
        k_pairs_by_color<<<chi, 1024, 0, st>>>(g.pair_color.as<int>(), g.pair_alpha.as<int>(), np, 0,
                                               tcnt.as<int>(), nullptr, nullptr); ::hm::count_launch();
        HM_TRY(scan_counts_i32(tcnt.as<int>(), tptr.as<int64_t>(), chi, st, scan_tmp));
        k_pairs_by_color<<<chi, 1024, 0, st>>>(g.pair_color.as<int>(), g.pair_alpha.as<int>(), np, 1, nullptr,
                                               tptr.as<int64_t>(), tile_box.as<int>()); ::hm::count_launch();
        HM_LAUNCH("pairs_by_color");
        HM_TRY(alloc(sz, np * sizeof(int)));
        HM_TRY(alloc(rowoff, (np + 1) * sizeof(int64_t)));
        k_act_sizes<<<ceil_div(np, 256), 256, 0, st>>>(tile_box.as<int>(), np, cu.ent.as<int>(), sz.as<int>()); ::hm::count_launch();
        HM_TRY(scan_counts_i32(sz.as<int>(), rowoff.as<int64_t>(), np, st, scan_tmp));
        HM_TRY(alloc(g.out_rows_ptr, (chi + 1) * sizeof(int64_t)));
        k_gather_ptr<<<ceil_div(chi + 1, 128), 128, 0, st>>>(rowoff.as<int64_t>(), tptr.as<int64_t>(), chi,
                                                             g.out_rows_ptr.as<int64_t>()); ::hm::count_launch();
        HM_TRY(to_host(g.h_out_rows_ptr, g.out_rows_ptr.p, chi + 1, st));
        HM_TRY(alloc(g.out_rows, std::max<int64_t>(g.h_out_rows_ptr[chi], 1) * sizeof(int)));
        k_act_rows<<<ceil_div(np * 32, 256), 256, 0, st>>>(tile_box.as<int>(), np, cu.ent.as<int>(),
                                                           rowoff.as<int64_t>(), g.out_rows.as<int>()); ::hm::count_launch();
        HM_LAUNCH("out_rows");
    }
    return ok();
}

Err color_cut(hm_ctx *c, int level, bool leaf) { return color_cut(c, level, leaf, c->st, c->scan_tmp); }

// Everything runs on `st`, with `scan_tmp` as the scan scratch, and the call
// returns after `st` has drained: a colouring reads and writes only its own
// cut's entry of c->colorings, so colourings of different levels may run on
// different host threads and streams.
Err color_cut(hm_ctx *c, int level, bool leaf, cudaStream_t st, DBuf &scan_tmp) {
    const int l = leaf ? c->L : level;
    if (l < 0 || l > c->L) return fail(HM_EINVAL, "colour: level out of range");
    Cut &cu = c->cuts[l];
    const int idx = leaf ? c->L + 1 : level;
    if ((int)c->colorings.size() < c->L + 2) return fail(HM_ESTATE, "colour: build the tree first");
    Coloring &g = c->colorings[idx];
    g = Coloring();
    g.leaf = leaf;
    g.level = l;
    g.pair_ptr = leaf ? cu.near_ptr.as<int>() : cu.int_ptr.as<int>();
    g.pair_col = leaf ? cu.near_idx.as<int>() : cu.int_idx.as<int>();
    g.n_pairs = leaf ? cu.n_near : cu.n_int;
    const int *sptr = leaf ? cu.near_ptr.as<int>() : cu.s_ptr.as<int>();
    const int *sidx = leaf ? cu.near_idx.as<int>() : cu.s_idx.as<int>();
    const int nc = cu.nc;
    const int64_t np = g.n_pairs;
    g.m_cols = c->cfg.r;
    if (leaf) g.m_cols = cu.max_rows;
    if (np == 0) {
        g.done = true;
        g.n_colors = 0;
        std::vector<int> z(1, 0);
        HM_TRY(to_dev(g.act_ptr, z, st));
        std::vector<int> zc(nc + 1, 0);
        HM_TRY(to_dev(g.ent_cptr, zc, st));
        std::vector<int64_t> z64(1, 0);
        HM_TRY(to_dev(g.act_rows_ptr, z64, st));
        return ok();
    }

    HM_TRY(alloc(g.pair_alpha, np * sizeof(int)));
    HM_TRY(alloc(g.pair_T, np * sizeof(int)));
    HM_TRY(alloc(g.pair_vertex, np * sizeof(int)));
    HM_TRY(alloc(g.pair_color, np * sizeof(int)));
    DBuf first, fscan, rep;
    HM_TRY(alloc(first, (np + 1) * sizeof(int64_t)));
    HM_TRY(alloc(fscan, (np + 1) * sizeof(int64_t)));
    HM_TRY(alloc(rep, np * sizeof(int)));
    k_pair_alpha<<<ceil_div(nc, 128), 128, 0, st>>>(g.pair_ptr, nc, g.pair_alpha.as<int>()); ::hm::count_launch();
    k_pair_keys<<<ceil_div(np, 128), 128, 0, st>>>(g.pair_ptr, g.pair_col, g.pair_alpha.as<int>(), np, sptr, sidx,
                                                   g.pair_T.as<int>(), first.as<int64_t>(), rep.as<int>()); ::hm::count_launch();
    HM_LAUNCH("pair_keys");
    HM_TRY(scan_exclusive(first.as<int64_t>(), fscan.as<int64_t>(), np, st));
    HM_TRY(read_scalar(g.n_vertices, fscan.as<int64_t>() + np, st));
    const int64_t nv = g.n_vertices;
    if (nv > (int64_t)VID_MASK) return fail(HM_ENOTSUP, "colour: more than 2^20 constraint sets");
    HM_TRY(alloc(g.vertex_pair, nv * sizeof(int)));
    HM_TRY(alloc(g.vertex_beta, nv * sizeof(int)));
    HM_TRY(alloc(g.vertex_color, nv * sizeof(int)));
    HM_TRY(alloc(g.vertex_degree, nv * sizeof(int)));
    k_vertex_ids<<<ceil_div(np, 256), 256, 0, st>>>(first.as<int64_t>(), fscan.as<int64_t>(), rep.as<int>(),
                                                    g.pair_col, np, g.pair_vertex.as<int>(),
                                                    g.vertex_pair.as<int>(), g.vertex_beta.as<int>()); ::hm::count_launch();
    HM_LAUNCH("vertex_ids");

    // vertices by beta
    DBuf vcnt, vptr64, vptr, vidx;
    HM_TRY(alloc(vcnt, nc * sizeof(int)));
    HM_TRY(alloc(vptr64, (nc + 1) * sizeof(int64_t)));
    HM_TRY(alloc(vidx, nv * sizeof(int)));
    k_vby_beta<<<ceil_div(nc, 128), 128, 0, st>>>(g.pair_ptr, g.pair_T.as<int>(), first.as<int64_t>(),
                                                  g.pair_vertex.as<int>(), nc, 0, vcnt.as<int>(), nullptr, nullptr); ::hm::count_launch();
    HM_TRY(scan_counts_i32(vcnt.as<int>(), vptr64.as<int64_t>(), nc, st, scan_tmp));
    k_vby_beta<<<ceil_div(nc, 128), 128, 0, st>>>(g.pair_ptr, g.pair_T.as<int>(), first.as<int64_t>(),
                                                  g.pair_vertex.as<int>(), nc, 1, nullptr, vptr64.as<int64_t>(),
                                                  vidx.as<int>()); ::hm::count_launch();
    HM_LAUNCH("vby_beta");
    {
        std::vector<int64_t> h;
        HM_TRY(to_host(h, vptr64.p, nc + 1, st));
        std::vector<int> h32(h.begin(), h.end());
        HM_TRY(to_dev(vptr, h32, st));
    }

    // edges
    const size_t bm_bytes = (size_t)((nv + 31) / 32) * 4;
    if (bm_bytes > 200 * 1024) return fail(HM_ENOTSUP, "colour: vertex bitmap exceeds shared memory");
    HM_TRY(allow_smem(k_edges, (size_t)(200 * 1024)));
    DBuf adj_ptr, adj;
    HM_TRY(alloc(adj_ptr, (nv + 1) * sizeof(int64_t)));
    k_edges<<<(int)nv, 256, bm_bytes, st>>>(nv, g.vertex_pair.as<int>(), g.vertex_beta.as<int>(),
                                            g.pair_alpha.as<int>(), g.pair_ptr, g.pair_vertex.as<int>(), sptr, sidx,
                                            vptr.as<int>(), vidx.as<int>(), 0, g.vertex_degree.as<int>(), nullptr,
                                            nullptr); ::hm::count_launch();
    HM_LAUNCH("edges count");
    HM_TRY(scan_counts_i32(g.vertex_degree.as<int>(), adj_ptr.as<int64_t>(), nv, st, scan_tmp));
    int64_t n_adj = 0;
    HM_TRY(read_scalar(n_adj, adj_ptr.as<int64_t>() + nv, st));
    g.n_edges = n_adj / 2;
    HM_TRY(alloc(adj, n_adj * sizeof(int)));
    k_edges<<<(int)nv, 256, bm_bytes, st>>>(nv, g.vertex_pair.as<int>(), g.vertex_beta.as<int>(),
                                            g.pair_alpha.as<int>(), g.pair_ptr, g.pair_vertex.as<int>(), sptr, sidx,
                                            vptr.as<int>(), vidx.as<int>(), 1, nullptr, adj_ptr.as<int64_t>(),
                                            adj.as<int>()); ::hm::count_launch();
    HM_LAUNCH("edges fill");

    HM_TRY(color_tail(g, cu, adj_ptr, adj, false, st, scan_tmp));
    HM_CUDA(cudaStreamSynchronize(st));
    g.done = true;
    return ok();
}

// Uniform H^1, first sampling stage of cut `level` (Section 4.2): one vertex
// per box with a non-empty interaction list (cut order); its "pair" is the box
// itself (pair_alpha = the box), so the sampler, the peel and the QR see the
// tiles Y(I_alpha, colour of alpha).  Written to c->box_colorings[level].
Err color_boxes(hm_ctx *c, int level, cudaStream_t st, DBuf &scan_tmp) {
    if (level < 2 || level > c->L) return fail(HM_EINVAL, "colour boxes: level out of range");
    const Cut &cu = c->cuts[level];
    if ((int)c->box_colorings.size() < c->L + 1) return fail(HM_ESTATE, "colour boxes: build the tree first");
    Coloring &g = c->box_colorings[level];
    g = Coloring();
    g.level = level;
    g.m_cols = c->cfg.r;
    const int nc = cu.nc;
    DBuf flag, vscan, vid;
    HM_TRY(alloc(flag, ((size_t)nc + 1) * sizeof(int64_t)));
    HM_TRY(alloc(vscan, ((size_t)nc + 1) * sizeof(int64_t)));
    HM_TRY(alloc(vid, (size_t)std::max(nc, 1) * sizeof(int)));
    k_box_has_int<<<ceil_div(nc, 128), 128, 0, st>>>(cu.int_ptr.as<int>(), nc, flag.as<int64_t>()); ::hm::count_launch();
    HM_TRY(scan_exclusive(flag.as<int64_t>(), vscan.as<int64_t>(), nc, st));
    int64_t nv = 0;
    HM_TRY(read_scalar(nv, vscan.as<int64_t>() + nc, st));
    g.n_pairs = g.n_vertices = nv;
    if (nv == 0) {
        g.done = true;
        std::vector<int> z(1, 0);
        HM_TRY(to_dev(g.act_ptr, z, st));
        std::vector<int> zc(nc + 1, 0);
        HM_TRY(to_dev(g.ent_cptr, zc, st));
        std::vector<int64_t> z64(1, 0);
        HM_TRY(to_dev(g.act_rows_ptr, z64, st));
        return ok();
    }
    if (nv > (int64_t)VID_MASK) return fail(HM_ENOTSUP, "colour boxes: more than 2^20 boxes");
    HM_TRY(alloc(g.pair_alpha, nv * sizeof(int)));
    HM_TRY(alloc(g.pair_vertex, nv * sizeof(int)));
    HM_TRY(alloc(g.pair_color, nv * sizeof(int)));
    HM_TRY(alloc(g.vertex_pair, nv * sizeof(int)));
    HM_TRY(alloc(g.vertex_color, nv * sizeof(int)));
    HM_TRY(alloc(g.vertex_degree, nv * sizeof(int)));
    k_box_vertices<<<ceil_div(nc, 128), 128, 0, st>>>(cu.int_ptr.as<int>(), nc, vscan.as<int64_t>(),
                                                      g.pair_alpha.as<int>(), vid.as<int>()); ::hm::count_launch();
    k_iota<<<ceil_div(nv, 256), 256, 0, st>>>(g.pair_vertex.as<int>(), nv); ::hm::count_launch();
    k_iota<<<ceil_div(nv, 256), 256, 0, st>>>(g.vertex_pair.as<int>(), nv); ::hm::count_launch();
    HM_LAUNCH("box vertices");
    const size_t bm_bytes = (size_t)((nv + 31) / 32) * 4;
    if (bm_bytes > 200 * 1024) return fail(HM_ENOTSUP, "colour boxes: vertex bitmap exceeds shared memory");
    HM_TRY(allow_smem(k_box_edges, (size_t)(200 * 1024)));
    DBuf adj_ptr, adj;
    HM_TRY(alloc(adj_ptr, (nv + 1) * sizeof(int64_t)));
    k_box_edges<<<(int)nv, 256, bm_bytes, st>>>(nv, g.pair_alpha.as<int>(), vid.as<int>(), cu.near_ptr.as<int>(),
                                                cu.near_idx.as<int>(), cu.int_ptr.as<int>(), cu.int_idx.as<int>(), 0,
                                                g.vertex_degree.as<int>(), nullptr, nullptr); ::hm::count_launch();
    HM_LAUNCH("box edges count");
    HM_TRY(scan_counts_i32(g.vertex_degree.as<int>(), adj_ptr.as<int64_t>(), nv, st, scan_tmp));
    int64_t n_adj = 0;
    HM_TRY(read_scalar(n_adj, adj_ptr.as<int64_t>() + nv, st));
    g.n_edges = n_adj / 2;
    HM_TRY(alloc(adj, std::max<int64_t>(n_adj, 1) * sizeof(int)));
    k_box_edges<<<(int)nv, 256, bm_bytes, st>>>(nv, g.pair_alpha.as<int>(), vid.as<int>(), cu.near_ptr.as<int>(),
                                                cu.near_idx.as<int>(), cu.int_ptr.as<int>(), cu.int_idx.as<int>(), 1,
                                                nullptr, adj_ptr.as<int64_t>(), adj.as<int>()); ::hm::count_launch();
    HM_LAUNCH("box edges fill");
    HM_TRY(color_tail(g, cu, adj_ptr, adj, true, st, scan_tmp));
    HM_CUDA(cudaStreamSynchronize(st));
    g.done = true;
    return ok();
}

}  // namespace hm
