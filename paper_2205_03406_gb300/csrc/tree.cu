// Cluster tree, cuts, neighbour and interaction lists (Section 3) on the GPU.
//
//  K1  quantize to a 2^21 grid per dimension, 63-bit Morton keys, bitonic sort
//      of (key, index) pairs -- the index breaks ties, so the order is the
//      unique stable Morton order;
//  K2  levels: a box is split while it holds more than m points (or above a
//      forced depth); boxes are the runs of equal Morton prefix among the
//      points of split parents;
//  K3  cuts (level-l boxes plus carried coarser leaves), parents/children,
//      neighbour lists (closed boxes touch) and interaction lists (children of
//      the parent's neighbours that are not neighbours).
//
// Everything after the FP64 quantisation is integer arithmetic, so the result
// is bit-identical to any other implementation of the same rules.
#include "ctx.cuh"

#include <algorithm>
#include <cmath>

namespace hm {

// ---------------------------------------------------------------------------
// scans (used by every module)
// ---------------------------------------------------------------------------

__global__ void k_scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n) {
    __shared__ int64_t sh[1024];
    const int t = threadIdx.x;
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t b = t * per, e = min(n, b + per);
    int64_t s = 0;
    for (int64_t i = b; i < e; ++i) s += in[i];
    sh[t] = s;
    __syncthreads();
    for (int o = 1; o < blockDim.x; o <<= 1) {
        int64_t v = (t >= o) ? sh[t - o] : 0;
        __syncthreads();
        sh[t] += v;
        __syncthreads();
    }
    int64_t run = (t == 0) ? 0 : sh[t - 1];
    for (int64_t i = b; i < e; ++i) {
        int64_t v = in[i];
        out[i] = run;
        run += v;
    }
    if (t == blockDim.x - 1) out[n] = sh[t];
}

Err scan_exclusive(const int64_t *in_dev, int64_t *out_dev, int64_t n, cudaStream_t st) {
    k_scan_exclusive_i64<<<1, 1024, 0, st>>>(in_dev, out_dev, n); ::hm::count_launch();
    HM_LAUNCH("scan_exclusive");
    return ok();
}

__global__ void k_i32_to_i64(const int *in, int64_t *out, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}

Err scan_counts_i32(const int *counts_dev, int64_t *out_dev, int64_t n, cudaStream_t st, DBuf &tmp) {
    HM_TRY(ensure(tmp, (size_t)(n + 1) * sizeof(int64_t)));
    if (n > 0) {
        k_i32_to_i64<<<ceil_div(n, 256), 256, 0, st>>>(counts_dev, tmp.as<int64_t>(), n); ::hm::count_launch();
        HM_LAUNCH("i32_to_i64");
    }
    return scan_exclusive(tmp.as<int64_t>(), out_dev, n, st);
}

// ---------------------------------------------------------------------------
// K1: bounding box, quantisation, Morton keys, sort
// ---------------------------------------------------------------------------

__global__ void k_minmax(const double *x, int64_t n, int d, double *out /* [2][3] per block */) {
    __shared__ double smin[3][256], smax[3][256];
    const int t = threadIdx.x;
    for (int k = 0; k < 3; ++k) { smin[k][t] = INFINITY; smax[k][t] = -INFINITY; }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + t; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < d; ++k) {
            double v = x[i * d + k];
            smin[k][t] = fmin(smin[k][t], v);
            smax[k][t] = fmax(smax[k][t], v);
        }
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o)
            for (int k = 0; k < 3; ++k) {
                smin[k][t] = fmin(smin[k][t], smin[k][t + o]);
                smax[k][t] = fmax(smax[k][t], smax[k][t + o]);
            }
        __syncthreads();
    }
    if (t == 0)
        for (int k = 0; k < 3; ++k) {
            out[blockIdx.x * 6 + k] = smin[k][0];
            out[blockIdx.x * 6 + 3 + k] = smax[k][0];
        }
}

// q = min(floor((x - lo) / side * 2^21), 2^21 - 1): explicit round-to-nearest
// intrinsics keep nvcc from contracting the subtraction and division.
__global__ void k_quantize(const double *x, int64_t n, int d, double lo0, double lo1, double lo2,
                           double side, int *q, ulonglong2 *keys, int64_t npad) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= npad) return;
    if (i >= n) {
        keys[i] = make_ulonglong2(~0ull, ~0ull);
        return;
    }
    const double lo[3] = {lo0, lo1, lo2};
    unsigned long long key = 0;
    for (int k = 0; k < 3; ++k) {
        int qi = 0;
        if (k < d) {
            double t = __ddiv_rn(__dsub_rn(x[i * d + k], lo[k]), side);
            double f = floor(__dmul_rn(t, (double)(1 << QBITS)));
            f = fmin(fmax(f, 0.0), (double)((1 << QBITS) - 1));
            qi = (int)f;
        }
        q[i * 3 + k] = qi;
    }
    for (int b = 0; b < QBITS; ++b)
        for (int k = 0; k < d; ++k)
            key |= (unsigned long long)((q[i * 3 + k] >> b) & 1) << (b * d + k);
    keys[i] = make_ulonglong2(key, (unsigned long long)i);
}

__device__ __forceinline__ bool key_less(ulonglong2 a, ulonglong2 b) {
    return a.x < b.x || (a.x == b.x && a.y < b.y);
}

__global__ void k_bitonic_step(ulonglong2 *a, int64_t npad, int64_t j, int64_t k) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= npad) return;
    int64_t l = i ^ j;
    if (l <= i) return;
    ulonglong2 ai = a[i], al = a[l];
    bool asc = (i & k) == 0;
    if (asc ? key_less(al, ai) : key_less(ai, al)) {
        a[i] = al;
        a[l] = ai;
    }
}

// Inner stages j < 2048 of one k in shared memory.
__global__ void k_bitonic_shared(ulonglong2 *a, int64_t npad, int64_t k, int64_t jstart) {
    __shared__ ulonglong2 s[2048];
    const int64_t base = blockIdx.x * 2048ll;
    for (int t = threadIdx.x; t < 2048; t += blockDim.x) s[t] = a[base + t];
    __syncthreads();
    for (int64_t j = jstart; j > 0; j >>= 1) {
        for (int t = threadIdx.x; t < 2048; t += blockDim.x) {
            int64_t i = base + t, l = i ^ j;
            if (l > i) {
                ulonglong2 ai = s[t], al = s[l - base];
                bool asc = (i & k) == 0;
                if (asc ? key_less(al, ai) : key_less(ai, al)) {
                    s[t] = al;
                    s[l - base] = ai;
                }
            }
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < 2048; t += blockDim.x) a[base + t] = s[t];
}

static Err bitonic_sort(ulonglong2 *a, int64_t npad, cudaStream_t st) {
    const int nb = ceil_div(npad, 256);
    for (int64_t k = 2; k <= npad; k <<= 1) {
        int64_t j = k >> 1;
        for (; j >= 2048; j >>= 1) {
            k_bitonic_step<<<nb, 256, 0, st>>>(a, npad, j, k); ::hm::count_launch();
        }
        if (npad >= 2048) {
            k_bitonic_shared<<<(int)(npad / 2048), 1024, 0, st>>>(a, npad, k, j); ::hm::count_launch();
        } else {
            for (; j > 0; j >>= 1) k_bitonic_step<<<nb, 256, 0, st>>>(a, npad, j, k); ::hm::count_launch();
        }
    }
    HM_LAUNCH("bitonic");
    return ok();
}

__global__ void k_gather_sorted(const ulonglong2 *keys, const double *x, const int *q, int64_t n, int d,
                                int *perm, double *xs, int *qs, unsigned long long *ksorted) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = (int64_t)keys[i].y;
    perm[i] = (int)o;
    ksorted[i] = keys[i].x;
    for (int k = 0; k < 3; ++k) {
        xs[i * 3 + k] = (k < d) ? x[o * d + k] : 0.0;
        qs[i * 3 + k] = q[o * 3 + k];
    }
}

// ---------------------------------------------------------------------------
// K2: levels
// ---------------------------------------------------------------------------

// Point i starts a level-(l+1) box when it is active at l+1 and its predecessor
// is inactive or has another Morton prefix.
__global__ void k_level_heads(const unsigned long long *ks, const int *box_of_l, const int *box_l,
                              int64_t n, int shift_next, int64_t *head, int *active_next) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int b = box_of_l[i];
    int act = (b >= 0) && (box_l[b * BOX_FIELDS + 6] == 0);  // parent box is split
    active_next[i] = act;
    int h = 0;
    if (act) {
        if (i == 0) h = 1;
        else {
            int bp = box_of_l[i - 1];
            int actp = (bp >= 0) && (box_l[bp * BOX_FIELDS + 6] == 0);
            h = !actp || ((ks[i] >> shift_next) != (ks[i - 1] >> shift_next));
        }
    }
    head[i] = h;
}

__global__ void k_level_fill(const int64_t *head_scan, const int64_t *head, const int *active_next,
                             const int *box_of_l, const int *qs, int64_t n, int lnext, int gid0,
                             int *box_next, int *box_of_next) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (!active_next[i]) {
        box_of_next[i] = -1;
        return;
    }
    const int b = (int)(head_scan[i] + head[i] - 1);
    box_of_next[i] = b;
    int *bx = box_next + (int64_t)b * BOX_FIELDS;
    if (head[i]) {
        bx[0] = (int)i;
        for (int k = 0; k < 3; ++k) bx[2 + k] = qs[i * 3 + k] >> (QBITS - lnext);
        bx[5] = box_of_l[i];
        bx[7] = gid0 + b;
    }
    const bool last = (i == n - 1) || !active_next[i + 1] || head[i + 1];
    if (last) bx[1] = (int)(i + 1);
}

// leaf flag: not split (count <= m, or forced depth reached, or grid resolution)
__global__ void k_level_leaf(int *box, int nb, int l, int m, int uniform_depth) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int *bx = box + (int64_t)b * BOX_FIELDS;
    int count = bx[1] - bx[0];
    bool split = uniform_depth > 0 ? (l < uniform_depth) : (count > m);
    split = split && l < QBITS && count > 0;
    bx[6] = split ? 0 : 1;
}

__global__ void k_leafgid_update(const int *box_of_l, const int *box_l, int64_t n, int *leafgid) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int b = box_of_l[i];
    if (b >= 0 && box_l[b * BOX_FIELDS + 6]) leafgid[i] = box_l[b * BOX_FIELDS + 7];
}

// ---------------------------------------------------------------------------
// K3: cuts, parents, lists
// ---------------------------------------------------------------------------

// Entry of cut l holding point i: its level-l box, else its (coarser) leaf.
__global__ void k_cut_heads(const int *box_of_l, const int *leafgid, int gid0, int64_t n, int *entgid,
                            int64_t *head) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int b = box_of_l[i];
    int g = (b >= 0) ? gid0 + b : leafgid[i];
    entgid[i] = g;
    int gp = (i > 0) ? ((box_of_l[i - 1] >= 0) ? gid0 + box_of_l[i - 1] : leafgid[i - 1]) : -1;
    head[i] = (i == 0) || (g != gp);
}

__global__ void k_cut_fill(const int64_t *head_scan, const int64_t *head, const int *entgid, int64_t n,
                           const int *gid_level, const int *gid_index, const int *qs, int *ent, int *pt2ent) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int e = (int)(head_scan[i] + head[i] - 1);
    pt2ent[i] = e;
    int *en = ent + (int64_t)e * ENT_FIELDS;
    if (head[i]) {
        const int g = entgid[i];
        const int lev = gid_level[g];
        en[0] = lev;
        en[1] = gid_index[g];
        en[2] = g;
        en[3] = (int)i;
        for (int k = 0; k < 3; ++k) en[5 + k] = qs[i * 3 + k] >> (QBITS - lev);
    }
    if (i == n - 1 || head[i + 1]) en[4] = (int)(i + 1);
}

__global__ void k_cut_links(const int *ent, int nc, const int *pt2ent_prev, int *parent) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nc) return;
    parent[e] = pt2ent_prev[ent[e * ENT_FIELDS + 3]];
}

__global__ void k_cut_kids(const int *ent_prev, int ncp, const int *pt2ent, int *kb, int *ke) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ncp) return;
    kb[e] = pt2ent[ent_prev[e * ENT_FIELDS + 3]];
    ke[e] = pt2ent[ent_prev[e * ENT_FIELDS + 4] - 1] + 1;
}

// Closed boxes of two entries of cut l overlap in every dimension.
__device__ __forceinline__ bool touch(const int *a, const int *b, int l, int d) {
    const int sa = l - a[0], sb = l - b[0];
    for (int k = 0; k < d; ++k) {
        const long long loa = (long long)a[5 + k] << sa, hia = (((long long)a[5 + k] + 1) << sa) - 1;
        const long long lob = (long long)b[5 + k] << sb, hib = (((long long)b[5 + k] + 1) << sb) - 1;
        if (loa > hib + 1 || lob > hia + 1) return false;
    }
    return true;
}

// pass 0: count near and int per entry; pass 1: fill both lists and their merge S.
__global__ void k_lists(const int *ent, int nc, int l, int d, const int *parent, const int *near_prev_ptr,
                        const int *near_prev_idx, const int *kb_prev, const int *ke_prev, int pass,
                        int *cnt_near, int *cnt_int, const int64_t *near_ptr, const int64_t *int_ptr,
                        int *near_idx, int *int_idx, int *s_idx) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nc) return;
    const int *me = ent + (int64_t)e * ENT_FIELDS;
    const int p = parent[e];
    int nn = 0, ni = 0;
    int64_t on = 0, oi = 0, os = 0;
    if (pass) {
        on = near_ptr[e];
        oi = int_ptr[e];
        os = on + oi;
    }
    for (int t = near_prev_ptr[p]; t < near_prev_ptr[p + 1]; ++t) {
        const int s = near_prev_idx[t];
        for (int c = kb_prev[s]; c < ke_prev[s]; ++c) {
            const bool nb = touch(me, ent + (int64_t)c * ENT_FIELDS, l, d);
            if (pass) {
                if (nb) near_idx[on + nn] = c;
                else int_idx[oi + ni] = c;
                s_idx[os + nn + ni] = c;  // candidates arrive in cut order
            }
            if (nb) ++nn;
            else ++ni;
        }
    }
    if (!pass) {
        cnt_near[e] = nn;
        cnt_int[e] = ni;
    }
}

__global__ void k_i64_to_i32(const int64_t *in, int *out, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int)in[i];
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------

Err build_tree(hm_ctx *c, const double *points_dev, int64_t n) {
    cudaStream_t st = c->st;
    const int d = c->cfg.d;
    c->n = n;
    c->d = d;

    // root cube (same rule as Section 3's unit cube when the points fit in it)
    {
        const int nb = 64;
        DBuf mm;
        HM_TRY(alloc(mm, nb * 6 * sizeof(double)));
        k_minmax<<<nb, 256, 0, st>>>(points_dev, n, d, mm.as<double>()); ::hm::count_launch();
        HM_LAUNCH("minmax");
        std::vector<double> h;
        HM_TRY(to_host(h, mm.p, nb * 6, st));
        mm.release();
        double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int b = 0; b < nb; ++b)
            for (int k = 0; k < 3; ++k) {
                mn[k] = std::min(mn[k], h[b * 6 + k]);
                mx[k] = std::max(mx[k], h[b * 6 + 3 + k]);
            }
        bool unit = true;
        for (int k = 0; k < d; ++k) unit = unit && mn[k] >= 0.0 && mx[k] <= 1.0;
        for (int k = 0; k < 3; ++k) c->lo[k] = 0.0;
        c->side = 1.0;
        if (!unit) {
            double side = 0.0;
            for (int k = 0; k < d; ++k) {
                c->lo[k] = mn[k];
                side = std::max(side, mx[k] - mn[k]);
            }
            c->side = side > 0.0 ? side : 1.0;
        }
    }

    int64_t npad = 1;
    while (npad < n) npad <<= 1;
    DBuf keys, q, ksorted;
    HM_TRY(alloc(keys, npad * sizeof(ulonglong2)));
    HM_TRY(alloc(q, n * 3 * sizeof(int)));
    HM_TRY(alloc(ksorted, n * sizeof(unsigned long long)));
    k_quantize<<<ceil_div(npad, 256), 256, 0, st>>>(points_dev, n, d, c->lo[0], c->lo[1], c->lo[2], c->side,
                                                    q.as<int>(), keys.as<ulonglong2>(), npad); ::hm::count_launch();
    HM_LAUNCH("quantize");
    HM_TRY(bitonic_sort(keys.as<ulonglong2>(), npad, st));
    HM_TRY(alloc(c->perm, n * sizeof(int)));
    HM_TRY(alloc(c->xs, n * 3 * sizeof(double)));
    HM_TRY(alloc(c->qs, n * 3 * sizeof(int)));
    k_gather_sorted<<<ceil_div(n, 256), 256, 0, st>>>(keys.as<ulonglong2>(), points_dev, q.as<int>(), n, d,
                                                      c->perm.as<int>(), c->xs.as<double>(), c->qs.as<int>(),
                                                      ksorted.as<unsigned long long>()); ::hm::count_launch();
    HM_LAUNCH("gather_sorted");
    keys.release();
    q.release();

    // levels
    c->levels.clear();
    c->level_off.clear();
    std::vector<DBuf> box_of;  // per level: int32 [n]
    DBuf head, head_scan, active, leafgid;
    HM_TRY(alloc(head, (n + 1) * sizeof(int64_t)));
    HM_TRY(alloc(head_scan, (n + 1) * sizeof(int64_t)));
    HM_TRY(alloc(active, n * sizeof(int)));
    HM_TRY(alloc(leafgid, n * sizeof(int)));
    {
        Level l0;
        l0.nb = 1;
        std::vector<int> b0 = {0, (int)n, 0, 0, 0, -1, 0, 0};
        HM_TRY(to_dev(l0.box, b0, st));
        c->levels.push_back(std::move(l0));
        c->level_off.push_back(0);
        DBuf bo;
        HM_TRY(alloc(bo, n * sizeof(int)));
        HM_CUDA(cudaMemsetAsync(bo.p, 0, n * sizeof(int), st));
        box_of.push_back(std::move(bo));
        k_level_leaf<<<1, 32, 0, st>>>(c->levels[0].box.as<int>(), 1, 0, c->leaf_size, c->cfg.uniform_depth); ::hm::count_launch();
        HM_LAUNCH("level_leaf");
    }
    int gid = 1;
    const int nbk = ceil_div(n, 256);
    for (int l = 0; l < QBITS; ++l) {
        k_leafgid_update<<<nbk, 256, 0, st>>>(box_of[l].as<int>(), c->levels[l].box.as<int>(), n,
                                              leafgid.as<int>()); ::hm::count_launch();
        const int shift = d * (QBITS - l - 1);
        k_level_heads<<<nbk, 256, 0, st>>>(ksorted.as<unsigned long long>(), box_of[l].as<int>(),
                                           c->levels[l].box.as<int>(), n, shift, head.as<int64_t>(),
                                           active.as<int>()); ::hm::count_launch();
        HM_LAUNCH("level_heads");
        HM_TRY(scan_exclusive(head.as<int64_t>(), head_scan.as<int64_t>(), n, st));
        int64_t nb_next = 0;
        HM_TRY(read_scalar(nb_next, head_scan.as<int64_t>() + n, st));
        if (nb_next == 0) break;
        Level nx;
        nx.nb = (int)nb_next;
        HM_TRY(alloc(nx.box, nb_next * BOX_FIELDS * sizeof(int)));
        DBuf bo;
        HM_TRY(alloc(bo, n * sizeof(int)));
        k_level_fill<<<nbk, 256, 0, st>>>(head_scan.as<int64_t>(), head.as<int64_t>(), active.as<int>(),
                                          box_of[l].as<int>(), c->qs.as<int>(), n, l + 1, gid, nx.box.as<int>(),
                                          bo.as<int>()); ::hm::count_launch();
        HM_LAUNCH("level_fill");
        k_level_leaf<<<ceil_div(nb_next, 256), 256, 0, st>>>(nx.box.as<int>(), (int)nb_next, l + 1,
                                                              c->leaf_size, c->cfg.uniform_depth); ::hm::count_launch();
        HM_LAUNCH("level_leaf");
        c->level_off.push_back(gid);
        gid += (int)nb_next;
        c->levels.push_back(std::move(nx));
        box_of.push_back(std::move(bo));
    }
    k_leafgid_update<<<nbk, 256, 0, st>>>(box_of.back().as<int>(), c->levels.back().box.as<int>(), n,
                                          leafgid.as<int>()); ::hm::count_launch();
    c->L = (int)c->levels.size() - 1;
    const int L = c->L;

    // gid -> (level, index) tables
    DBuf gid_level, gid_index;
    {
        std::vector<int> gl(gid), gi(gid);
        for (int l = 0; l <= L; ++l)
            for (int b = 0; b < c->levels[l].nb; ++b) {
                gl[c->level_off[l] + b] = l;
                gi[c->level_off[l] + b] = b;
            }
        HM_TRY(to_dev(gid_level, gl, st));
        HM_TRY(to_dev(gid_index, gi, st));
    }

    // cuts
    c->cuts.clear();
    c->cuts.resize(L + 1);
    DBuf entgid;
    HM_TRY(alloc(entgid, n * sizeof(int)));
    for (int l = 0; l <= L; ++l) {
        Cut &cu = c->cuts[l];
        k_cut_heads<<<nbk, 256, 0, st>>>(box_of[l].as<int>(), leafgid.as<int>(), c->level_off[l], n,
                                         entgid.as<int>(), head.as<int64_t>()); ::hm::count_launch();
        HM_LAUNCH("cut_heads");
        HM_TRY(scan_exclusive(head.as<int64_t>(), head_scan.as<int64_t>(), n, st));
        int64_t nc = 0;
        HM_TRY(read_scalar(nc, head_scan.as<int64_t>() + n, st));
        cu.nc = (int)nc;
        HM_TRY(alloc(cu.ent, nc * ENT_FIELDS * sizeof(int)));
        HM_CUDA(cudaMemsetAsync(cu.ent.p, 0, nc * ENT_FIELDS * sizeof(int), st));
        HM_TRY(alloc(cu.pt2ent, n * sizeof(int)));
        k_cut_fill<<<nbk, 256, 0, st>>>(head_scan.as<int64_t>(), head.as<int64_t>(), entgid.as<int>(), n,
                                        gid_level.as<int>(), gid_index.as<int>(), c->qs.as<int>(),
                                        cu.ent.as<int>(), cu.pt2ent.as<int>()); ::hm::count_launch();
        HM_LAUNCH("cut_fill");
        HM_TRY(alloc(cu.parent, nc * sizeof(int)));
        if (l == 0) {
            HM_CUDA(cudaMemsetAsync(cu.parent.p, 0, nc * sizeof(int), st));
        } else {
            k_cut_links<<<ceil_div(nc, 256), 256, 0, st>>>(cu.ent.as<int>(), cu.nc, c->cuts[l - 1].pt2ent.as<int>(),
                                                           cu.parent.as<int>()); ::hm::count_launch();
            HM_LAUNCH("cut_links");
            Cut &pv = c->cuts[l - 1];
            HM_TRY(alloc(pv.kid_begin, pv.nc * sizeof(int)));
            HM_TRY(alloc(pv.kid_end, pv.nc * sizeof(int)));
            k_cut_kids<<<ceil_div(pv.nc, 256), 256, 0, st>>>(pv.ent.as<int>(), pv.nc, cu.pt2ent.as<int>(),
                                                             pv.kid_begin.as<int>(), pv.kid_end.as<int>()); ::hm::count_launch();
            HM_LAUNCH("cut_kids");
        }
    }
    for (auto &b : box_of) b.release();
    head.release();
    head_scan.release();
    active.release();
    leafgid.release();
    entgid.release();
    ksorted.release();

    // lists
    for (int l = 0; l <= L; ++l) {
        Cut &cu = c->cuts[l];
        std::vector<int> ent;
        HM_TRY(to_host(ent, cu.ent.p, (size_t)cu.nc * ENT_FIELDS, st));
        cu.max_rows = 0;
        for (int e = 0; e < cu.nc; ++e) cu.max_rows = std::max(cu.max_rows, ent[e * ENT_FIELDS + 4] - ent[e * ENT_FIELDS + 3]);
        if (l == 0) {
            std::vector<int> np = {0, 1}, ni = {0}, ip = {0, 0}, ii;
            HM_TRY(to_dev(cu.near_ptr, np, st));
            HM_TRY(to_dev(cu.near_idx, ni, st));
            HM_TRY(to_dev(cu.int_ptr, ip, st));
            HM_TRY(to_dev(cu.int_idx, ii, st));
            HM_TRY(to_dev(cu.s_ptr, np, st));
            HM_TRY(to_dev(cu.s_idx, ni, st));
            cu.n_near = 1;
            cu.n_int = 0;
            continue;
        }
        Cut &pv = c->cuts[l - 1];
        DBuf cn, ci, pn64, pi64;
        HM_TRY(alloc(cn, cu.nc * sizeof(int)));
        HM_TRY(alloc(ci, cu.nc * sizeof(int)));
        HM_TRY(alloc(pn64, (cu.nc + 1) * sizeof(int64_t)));
        HM_TRY(alloc(pi64, (cu.nc + 1) * sizeof(int64_t)));
        const int g = ceil_div(cu.nc, 128);
        k_lists<<<g, 128, 0, st>>>(cu.ent.as<int>(), cu.nc, l, d, cu.parent.as<int>(), pv.near_ptr.as<int>(),
                                   pv.near_idx.as<int>(), pv.kid_begin.as<int>(), pv.kid_end.as<int>(), 0,
                                   cn.as<int>(), ci.as<int>(), nullptr, nullptr, nullptr, nullptr, nullptr); ::hm::count_launch();
        HM_LAUNCH("lists count");
        HM_TRY(scan_counts_i32(cn.as<int>(), pn64.as<int64_t>(), cu.nc, st, c->scan_tmp));
        HM_TRY(scan_counts_i32(ci.as<int>(), pi64.as<int64_t>(), cu.nc, st, c->scan_tmp));
        HM_TRY(read_scalar(cu.n_near, pn64.as<int64_t>() + cu.nc, st));
        HM_TRY(read_scalar(cu.n_int, pi64.as<int64_t>() + cu.nc, st));
        HM_TRY(alloc(cu.near_idx, cu.n_near * sizeof(int)));
        HM_TRY(alloc(cu.int_idx, cu.n_int * sizeof(int)));
        HM_TRY(alloc(cu.s_idx, (cu.n_near + cu.n_int) * sizeof(int)));
        k_lists<<<g, 128, 0, st>>>(cu.ent.as<int>(), cu.nc, l, d, cu.parent.as<int>(), pv.near_ptr.as<int>(),
                                   pv.near_idx.as<int>(), pv.kid_begin.as<int>(), pv.kid_end.as<int>(), 1,
                                   nullptr, nullptr, pn64.as<int64_t>(), pi64.as<int64_t>(), cu.near_idx.as<int>(),
                                   cu.int_idx.as<int>(), cu.s_idx.as<int>()); ::hm::count_launch();
        HM_LAUNCH("lists fill");
        HM_TRY(alloc(cu.near_ptr, (cu.nc + 1) * sizeof(int)));
        HM_TRY(alloc(cu.int_ptr, (cu.nc + 1) * sizeof(int)));
        HM_TRY(alloc(cu.s_ptr, (cu.nc + 1) * sizeof(int)));
        k_i64_to_i32<<<ceil_div(cu.nc + 1, 256), 256, 0, st>>>(pn64.as<int64_t>(), cu.near_ptr.as<int>(), cu.nc + 1); ::hm::count_launch();
        k_i64_to_i32<<<ceil_div(cu.nc + 1, 256), 256, 0, st>>>(pi64.as<int64_t>(), cu.int_ptr.as<int>(), cu.nc + 1); ::hm::count_launch();
        HM_LAUNCH("ptr convert");
        // S pointers: near_ptr + int_ptr
        std::vector<int64_t> hn, hi;
        HM_TRY(to_host(hn, pn64.p, cu.nc + 1, st));
        HM_TRY(to_host(hi, pi64.p, cu.nc + 1, st));
        std::vector<int> hs(cu.nc + 1);
        for (int e = 0; e <= cu.nc; ++e) hs[e] = (int)(hn[e] + hi[e]);
        HM_CUDA(cudaMemcpyAsync(cu.s_ptr.p, hs.data(), hs.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        HM_CUDA(cudaStreamSynchronize(st));
    }
    return ok();
}

}  // namespace hm
