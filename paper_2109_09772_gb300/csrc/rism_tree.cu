// rism_tree.cu -- barycentric-Lagrange particle-cluster treecode with a
// cell-list near field, fused with the output epilogue.
//
// The long-range sums Phi1 = sum q/d and Phik = sum q e^{-kappa d}/d are
// split as in the near/far decomposition of Sec. 2.3.1, eq. (exppot): for a
// target batch (a grid sub-box) the atoms of a source cluster that passes
// the acceptance test (r_batch + r_cluster) / R < theta (the MAC of
// Sec. 2.3.1, applied between a target box and a source box) are replaced by
// the cluster's (n+1)^3 Chebyshev proxy points carrying modified charges
//   Qhat_k = sum_j q_j L_k1(y_j1) L_k2(y_j2) L_k3(y_j3)
// (barycentric Lagrange interpolation, Berrut & Trefethen 2004; the
// kernel-independent particle-cluster form of Wang, Krasny & Tlupova 2020).
// Because the proxies are kernel independent, one set serves both 1/d and
// e^{-kappa d}/d.  This differs from the paper's Taylor cluster-particle
// treecode (tree on the targets, recurrences eqs. (coulombrecurrence) ...
// (screenedcoulombauxiliaryrecurrence)); see the design notes.
//
// The short-range parts -- LJ within the per-pair cut-off (Sec. 2.6) and the
// erfc remainders of eq. (dcf-r)/(tcf-r) within r_short -- are summed over
// the atoms of the cells that intersect the batch box grown by the largest
// cut-off.  The cells are Morton-code prefixes of the same sorted order the
// tree is built from, so one device radix sort serves both.
//
// Pipeline (all on the context's stream, no host synchronisation):
//   k_bbox_codes -> k_sort_build (one CTA: radix sort, octree, proxy plan)
//   -> k_node_boxes -> k_gather -> k_cells -> k_upward -> k_proxy_reduce
//   -> k_lists(count) -> k_scan -> k_lists(fill) -> k_eval32.
// List and node capacities are checked on the device; an overflow is
// reported through the state's flag and the host grows the buffers and
// re-runs the pipeline once.
#include <cmath>
#include <cstring>
#include <vector>

#include "rism_tree.h"

namespace rism {

namespace {

constexpr int kSortThreads = 1024;
constexpr int kMortonBits = 10;          // per axis
constexpr int kMaxLevel = kMortonBits;   // octree depth limit
constexpr int kChunk = 64;               // atoms per upward-pass work item
constexpr int kBX = 2, kBY = 8, kBZ = 8, kP = 4;  // eval CTA: 128 threads x 4 points = 8x8x8 batch
constexpr int kT = 64;                   // sources per shared-memory tile
constexpr int kStack = 8 * kMaxLevel + 8;

struct Node {
    int begin, end;        // range in the sorted atom order
    int first_child;       // index of the first child, -1 for a leaf
    int nchild;
    int level;
    int prox;              // proxy set index, -1 if none
    int pad0, pad1;
    double lo[3], hi[3];   // tight bounding box (grid units)
};

struct TreeMeta {
    int nnodes, nprox, nitems, nleaves;
    int overflow;          // capacity exceeded (nodes / items / far list)
    int far_total;         // entries the list fill needs
    int lc;                // cell level of the near field
    int pad;
    double cube_lo[3];     // Morton cube (grid units)
    double cube_side;
    double cell_side;      // cube_side / 2^lc
    double rnear;          // near-field radius (grid units): max(largest LJ cut-off, r_short)
    unsigned long long direct_pairs, proxy_pairs, near_pairs;
};

__device__ __forceinline__ uint32_t spread3(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__device__ __forceinline__ uint32_t morton3(uint32_t x, uint32_t y, uint32_t z) {
    return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

// ------------------------------------------------- bounding cube + codes
// One CTA: min/max of the atoms (grid units), the Morton cube, the codes,
// and the near-field plan (radius = max(largest LJ cut-off, r_short); cells
// at least half that radius wide, at most 8^7 of them).
__global__ void k_bbox_codes(const Geo* __restrict__ geoU, const LJd* __restrict__ ljd, int n, int S, int smax,
                             double rs, double h, TreeMeta* meta, uint32_t* code, uint32_t* idx) {
    __shared__ double red[7][kSortThreads / 32];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double rc2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        Geo g = geoU[i];
        double v[3] = {g.x, g.y, g.z};
        for (int d = 0; d < 3; ++d) {
            lo[d] = fmin(lo[d], v[d]);
            hi[d] = fmax(hi[d], v[d]);
        }
        for (int s = 0; s < S; ++s) rc2 = fmax(rc2, ljd[(int64_t)i * smax + s].rc2);
    }
    for (int d = 0; d < 3; ++d)
        for (int o = 16; o > 0; o >>= 1) {
            lo[d] = fmin(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = fmax(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
    for (int o = 16; o > 0; o >>= 1) rc2 = fmax(rc2, __shfl_xor_sync(0xffffffffu, rc2, o));
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        for (int d = 0; d < 3; ++d) {
            red[d][w] = lo[d];
            red[3 + d][w] = hi[d];
        }
        red[6][w] = rc2;
    }
    __syncthreads();
    __shared__ double cube[4];
    if (threadIdx.x == 0) {
        double L = 0.0, l0[3], r2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            double a = INFINITY, b = -INFINITY;
            for (int k = 0; k < nw; ++k) {
                a = fmin(a, red[d][k]);
                b = fmax(b, red[3 + d][k]);
            }
            if (n == 0) a = b = 0.0;
            l0[d] = a;
            L = fmax(L, b - a);
        }
        for (int k = 0; k < nw; ++k) r2 = fmax(r2, red[6][k]);
        L = L * (1.0 + 1e-9) + 1e-6;
        for (int d = 0; d < 3; ++d) {
            meta->cube_lo[d] = l0[d];
            cube[d] = l0[d];
        }
        meta->cube_side = L;
        cube[3] = L;
        const double rnear = fmax(sqrt(r2), rs) / h;  // infinite without an LJ cut-off
        int lc = 0;
        if (isfinite(rnear))
            while (lc < 7 && L / (double)(1 << (lc + 1)) >= 0.5 * rnear) ++lc;
        meta->lc = lc;
        meta->cell_side = L / (double)(1 << lc);
        meta->rnear = rnear;
    }
    __syncthreads();
    const double sc = (double)(1 << kMortonBits) / cube[3];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        Geo g = geoU[i];
        uint32_t c[3];
        double v[3] = {g.x, g.y, g.z};
        for (int d = 0; d < 3; ++d) {
            double t = floor((v[d] - cube[d]) * sc);
            c[d] = (uint32_t)fmin(fmax(t, 0.0), (double)((1 << kMortonBits) - 1));
        }
        code[i] = morton3(c[0], c[1], c[2]);
        idx[i] = (uint32_t)i;
    }
}

// --------------------------------------------- radix sort + tree (1 CTA)
// Stable LSD radix sort, 8-bit digits, 4 passes; each warp owns a
// contiguous segment, ranks inside a warp come from __match_any_sync.
// Then the octree is built level by level from the sorted codes, and the
// proxy work plan (items of kChunk atoms per proxied node) is laid out.
struct BuildArgs {
    int n, leaf, P3, max_nodes, max_prox, max_items;
};

__device__ int block_exclusive_scan(int v, int* tmp /* >= 32 ints */, int& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < nw ? tmp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) tmp[lane] = t;
    }
    __syncthreads();
    int base = w > 0 ? tmp[w - 1] : 0;
    total = tmp[nw - 1];
    __syncthreads();
    return base + x - v;
}

__global__ void __launch_bounds__(kSortThreads) k_sort_build(BuildArgs a, uint32_t* code, uint32_t* idx,
                                                             uint32_t* code2, uint32_t* idx2, Node* nodes,
                                                             int* items, int* prox_nodes, TreeMeta* meta) {
    extern __shared__ int sh[];
    int* hist = sh;                     // [256][32]
    int* tmp = sh + 256 * 32;           // [64]
    const int n = a.n;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int NW = kSortThreads / 32;
    const int seg = ((n + NW - 1) / NW + 31) / 32 * 32;
    const int s0 = min(n, w * seg), s1 = min(n, s0 + seg);
    uint32_t *kin = code, *vin = idx, *kout = code2, *vout = idx2;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 8 * pass;
        for (int k = threadIdx.x; k < 256 * NW; k += blockDim.x) hist[k] = 0;
        __syncthreads();
        for (int b = s0; b < s1; b += 32) {
            int i = b + lane;
            if (i < s1) atomicAdd(&hist[((kin[i] >> shift) & 255u) * NW + w], 1);
        }
        __syncthreads();
        // exclusive scan of hist in (digit, warp) order: 8192 entries, 8 per thread
        {
            int loc[8], sum = 0;
            for (int k = 0; k < 8; ++k) {
                loc[k] = hist[threadIdx.x * 8 + k];
                sum += loc[k];
            }
            int total;
            int base = block_exclusive_scan(sum, tmp, total);
            for (int k = 0; k < 8; ++k) {
                hist[threadIdx.x * 8 + k] = base;
                base += loc[k];
            }
        }
        __syncthreads();
        for (int b = s0; b < s1; b += 32) {
            int i = b + lane;
            bool act = i < s1;
            uint32_t key = act ? kin[i] : 0u, val = act ? vin[i] : 0u;
            uint32_t d = act ? ((key >> shift) & 255u) : 256u + lane;  // inactive lanes never match
            unsigned peers = __match_any_sync(0xffffffffu, d);
            int rank = __popc(peers & ((1u << lane) - 1u));
            int base = act ? hist[d * NW + w] : 0;
            if (act) {
                kout[base + rank] = key;
                vout[base + rank] = val;
            }
            __syncwarp();
            if (act && rank == 0) hist[d * NW + w] = base + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        uint32_t* t1 = kin; kin = kout; kout = t1;
        uint32_t* t2 = vin; vin = vout; vout = t2;
    }
    // after 4 passes the sorted data is back in code/idx

    // ---- octree, level by level: nodes [lvl_begin, lvl_end) at the current level
    __shared__ int s_nnodes, s_lvl_begin, s_lvl_end, s_overflow;
    if (threadIdx.x == 0) {
        nodes[0] = Node{0, n, -1, 0, 0, -1, 0, 0, {0, 0, 0}, {0, 0, 0}};
        s_nnodes = 1;
        s_lvl_begin = 0;
        s_lvl_end = 1;
        s_overflow = 0;
    }
    __syncthreads();
    for (int lvl = 0; lvl < kMaxLevel; ++lvl) {
        const int lb = s_lvl_begin, le = s_lvl_end;
        if (lb >= le) break;
        for (int base = lb; base < le; base += blockDim.x) {
            const int nid = base + threadIdx.x;
            int cb[9];
            int nch = 0;
            bool split = false;
            if (nid < le) {
                Node nd = nodes[nid];
                split = (nd.end - nd.begin) > a.leaf;
                if (split) {
                    const int sh3 = 3 * (kMortonBits - 1 - lvl);
                    cb[0] = nd.begin;
                    for (int ch = 1; ch < 8; ++ch) {
                        // first position in [begin, end) whose child digit >= ch
                        int lo = cb[ch - 1], hi = nd.end;
                        while (lo < hi) {
                            int mid = (lo + hi) >> 1;
                            if ((int)((code[mid] >> sh3) & 7u) < ch) lo = mid + 1; else hi = mid;
                        }
                        cb[ch] = lo;
                    }
                    cb[8] = nd.end;
                    for (int ch = 0; ch < 8; ++ch) nch += cb[ch + 1] > cb[ch];
                }
            }
            int total;
            int off = block_exclusive_scan(nch, tmp, total);
            const int start = s_nnodes;
            if (nid < le && split) {
                if (start + off + nch > a.max_nodes) {
                    s_overflow = 1;
                } else {
                    nodes[nid].first_child = start + off;
                    nodes[nid].nchild = nch;
                    int k = start + off;
                    for (int ch = 0; ch < 8; ++ch)
                        if (cb[ch + 1] > cb[ch])
                            nodes[k++] = Node{cb[ch], cb[ch + 1], -1, 0, lvl + 1, -1, 0, 0, {0, 0, 0}, {0, 0, 0}};
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) s_nnodes = min(start + total, a.max_nodes);
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            s_lvl_begin = le;
            s_lvl_end = s_nnodes;
        }
        __syncthreads();
    }
    // ---- proxy plan: nodes with more than P3 atoms get proxies; items of kChunk atoms
    const int nn = s_nnodes;
    __shared__ int s_prox, s_items, s_leaves;
    if (threadIdx.x == 0) {
        s_prox = 0;
        s_items = 0;
        s_leaves = 0;
    }
    __syncthreads();
    for (int base = 0; base < nn; base += blockDim.x) {
        const int nid = base + threadIdx.x;
        int isp = 0, nit = 0, leaf = 0;
        if (nid < nn) {
            Node nd = nodes[nid];
            int cnt = nd.end - nd.begin;
            isp = cnt > a.P3;
            nit = isp ? (cnt + kChunk - 1) / kChunk : 0;
            leaf = nd.first_child < 0;
        }
        int tp, ti, tl;
        int op = block_exclusive_scan(isp, tmp, tp);
        int oi = block_exclusive_scan(nit, tmp, ti);
        block_exclusive_scan(leaf, tmp, tl);
        const int p0 = s_prox, i0 = s_items;
        if (nid < nn && isp) {
            int k = p0 + op;
            if (k >= a.max_prox || i0 + oi + nit > a.max_items) {
                s_overflow = 1;
                nodes[nid].prox = -1;
            } else {
                nodes[nid].prox = k;
                prox_nodes[k] = nid;
                // item = (proxy set k, atom chunk start)
                for (int c = 0; c < nit; ++c) {
                    items[2 * (i0 + oi + c) + 0] = k;
                    items[2 * (i0 + oi + c) + 1] = nodes[nid].begin + c * kChunk;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_prox = min(p0 + tp, a.max_prox);
            s_items = min(i0 + ti, a.max_items);
            s_leaves += tl;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        meta->nnodes = nn;
        meta->nprox = s_prox;
        meta->nitems = s_items;
        meta->nleaves = s_leaves;
        meta->overflow = s_overflow;
    }
}

// --------------------------------- node boxes, gathered sources, cells
__global__ void k_node_boxes(Node* nodes, const TreeMeta* meta, const uint32_t* idx, const Geo* __restrict__ geoU) {
    if (meta->overflow) return;  // the tree is incomplete; the host reports it
    const int nn = meta->nnodes;
    const int lane = threadIdx.x & 31;
    for (int nid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; nid < nn; nid += (gridDim.x * blockDim.x) >> 5) {
        Node nd = nodes[nid];
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int i = nd.begin + lane; i < nd.end; i += 32) {
            Geo g = geoU[idx[i]];
            double v[3] = {g.x, g.y, g.z};
            for (int d = 0; d < 3; ++d) {
                lo[d] = fmin(lo[d], v[d]);
                hi[d] = fmax(hi[d], v[d]);
            }
        }
        for (int d = 0; d < 3; ++d)
            for (int o = 16; o > 0; o >>= 1) {
                lo[d] = fmin(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
                hi[d] = fmax(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
            }
        if (lane == 0)
            for (int d = 0; d < 3; ++d) {
                nodes[nid].lo[d] = lo[d];
                nodes[nid].hi[d] = hi[d];
            }
    }
}

// Sorted copies of the atom geometry and LJ tables (sources of the eval kernel).
__global__ void k_gather(int n, int smax, const uint32_t* idx, const Geo* __restrict__ geoU,
                         const LJf* __restrict__ ljf, Geo* src, LJf* ljs) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int j = (int)idx[i];
        src[i] = geoU[j];
        for (int s = 0; s < smax; ++s) ljs[(int64_t)i * smax + s] = ljf[(int64_t)j * smax + s];
    }
}

// cell_start[m] = first sorted position whose level-lc Morton prefix is >= m.
__global__ void k_cells(int n, const TreeMeta* meta, const uint32_t* code, int* cell_start) {
    const int lc = meta->lc;
    const int ncell = 1 << (3 * lc);
    const int sh = 3 * (kMortonBits - lc);
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m <= ncell; m += gridDim.x * blockDim.x) {
        int lo = 0, hi = n;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if ((int)(code[mid] >> sh) < m) lo = mid + 1; else hi = mid;
        }
        cell_start[m] = lo;
    }
}

// ------------------------------------------------------------ upward
// Chebyshev points of the second kind on a node box, widened where the box
// is thin so that the interpolation stays well conditioned.
__device__ __forceinline__ void cheb_box(const Node& nd, int d, double& c, double& r) {
    double w = 0.0;
    for (int e = 0; e < 3; ++e) w = fmax(w, nd.hi[e] - nd.lo[e]);
    c = 0.5 * (nd.lo[d] + nd.hi[d]);
    r = fmax(0.5 * (nd.hi[d] - nd.lo[d]), fmax(0.05 * w, 0.25));
}

// Work item = (proxy set, chunk of kChunk atoms): partial modified charges.
__global__ void k_upward(int deg, const TreeMeta* meta, const Node* nodes, const int* prox_nodes, const int* items,
                         const Geo* __restrict__ src, double* part) {
    extern __shared__ double Ls[];  // [kChunk][3][deg+1], then q[kChunk]
    const int np = deg + 1, P3 = np * np * np;
    double* qs = Ls + kChunk * 3 * np;
    if (meta->overflow) return;
    const int nitems = meta->nitems;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int k = items[2 * it], b = items[2 * it + 1];
        const Node nd = nodes[prox_nodes[k]];
        const int cnt = min(kChunk, nd.end - b);
        __syncthreads();
        for (int t = threadIdx.x; t < kChunk * 3; t += blockDim.x) {
            const int j = t / 3, d = t % 3;
            double* L = Ls + (j * 3 + d) * np;
            if (j >= cnt) {
                for (int m = 0; m < np; ++m) L[m] = 0.0;
                if (d == 0) qs[j] = 0.0;
                continue;
            }
            const Geo g = src[b + j];
            if (d == 0) qs[j] = g.q;
            const double y = d == 0 ? g.x : (d == 1 ? g.y : g.z);
            double c, r;
            cheb_box(nd, d, c, r);
            // barycentric Lagrange basis at Chebyshev-2 points t_m = c + r cos(m pi / deg),
            // weights (-1)^m, halved at both ends
            int exact = -1;
            double den = 0.0;
            for (int m = 0; m < np; ++m) {
                const double tm = c + r * cospi((double)m / deg);
                const double diff = y - tm;
                if (diff == 0.0) exact = m;
                double wm = (m & 1) ? -1.0 : 1.0;
                if (m == 0 || m == deg) wm *= 0.5;
                const double v = (diff == 0.0) ? 0.0 : wm / diff;
                L[m] = v;
                den += v;
            }
            if (exact >= 0) {
                for (int m = 0; m < np; ++m) L[m] = (m == exact) ? 1.0 : 0.0;
            } else {
                const double id = 1.0 / den;
                for (int m = 0; m < np; ++m) L[m] *= id;
            }
        }
        __syncthreads();
        for (int p = threadIdx.x; p < P3; p += blockDim.x) {
            const int m1 = p % np, m2 = (p / np) % np, m3 = p / (np * np);
            double acc = 0.0;
            for (int j = 0; j < cnt; ++j)
                acc += qs[j] * Ls[(j * 3 + 0) * np + m1] * Ls[(j * 3 + 1) * np + m2] * Ls[(j * 3 + 2) * np + m3];
            part[(int64_t)it * P3 + p] = acc;
        }
    }
}

// Sum the partials of each proxy set in item order (deterministic) and write
// the proxy points (grid units) with their modified charges after the atoms.
__global__ void k_proxy_reduce(int deg, int n, const TreeMeta* meta, const Node* nodes, const int* prox_nodes,
                               const int* items, const double* part, Geo* src) {
    const int np = deg + 1, P3 = np * np * np;
    if (meta->overflow) return;
    const int nprox = meta->nprox, nitems = meta->nitems;
    for (int k = blockIdx.x; k < nprox; k += gridDim.x) {
        // items of set k are contiguous: find them by scanning (few sets, few items)
        int i0 = 0;
        while (i0 < nitems && items[2 * i0] != k) ++i0;
        int i1 = i0;
        while (i1 < nitems && items[2 * i1] == k) ++i1;
        const Node nd = nodes[prox_nodes[k]];
        double c[3], r[3];
        for (int d = 0; d < 3; ++d) cheb_box(nd, d, c[d], r[d]);
        for (int p = threadIdx.x; p < P3; p += blockDim.x) {
            const int m1 = p % np, m2 = (p / np) % np, m3 = p / (np * np);
            double q = 0.0;
            for (int it = i0; it < i1; ++it) q += part[(int64_t)it * P3 + p];
            src[n + (int64_t)k * P3 + p] = Geo{c[0] + r[0] * cospi((double)m1 / deg), c[1] + r[1] * cospi((double)m2 / deg),
                                               c[2] + r[2] * cospi((double)m3 / deg), q};
        }
    }
}

// -------------------------------------------------------------- lists
struct ListArgs {
    int nbx, nby, nbz;        // batches per axis
    int bx, by, bz;           // batch dims (points)
    double theta;
    int n, P3;
    int cap;                  // capacity of the far-list entry buffer
};

// One thread per target batch: depth-first traversal.  Far list entries are
// (start, count) ranges of the source array: sorted atoms (direct) or a proxy
// set (n + k P3, P3).  Adjacent direct ranges are merged.
template <bool FILL>
__global__ void k_lists(ListArgs a, const Node* __restrict__ nodes, const int* off, int2* ent, int* cnt,
                        TreeMeta* meta) {
    const int nb = a.nbx * a.nby * a.nbz;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    if (meta->overflow && !FILL) {
        cnt[b] = 0;  // tree incomplete: empty lists, the host reports the overflow
        return;
    }
    if (meta->overflow) return;
    const int ib = b % a.nbx, jb = (b / a.nbx) % a.nby, kb = b / (a.nbx * a.nby);
    const double cb[3] = {ib * a.bx + 0.5 * (a.bx - 1), jb * a.by + 0.5 * (a.by - 1), kb * a.bz + 0.5 * (a.bz - 1)};
    const double rb = 0.5 * sqrt((double)((a.bx - 1) * (a.bx - 1) + (a.by - 1) * (a.by - 1) + (a.bz - 1) * (a.bz - 1)));
    int stack[kStack];
    int sp = 0;
    if (a.n > 0) stack[sp++] = 0;
    int m = 0;
    int base = FILL ? off[b] : 0;
    int last_s = -1, last_e = -1;
    long long dpairs = 0, ppairs = 0;
    const int cap = a.cap;
    while (sp > 0) {
        const Node nd = nodes[stack[--sp]];
        double R2 = 0.0, rn2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            const double cn = 0.5 * (nd.lo[d] + nd.hi[d]);
            R2 += (cb[d] - cn) * (cb[d] - cn);
            rn2 += 0.25 * (nd.hi[d] - nd.lo[d]) * (nd.hi[d] - nd.lo[d]);
        }
        const double rs = rb + sqrt(rn2);
        const bool sep = rs * rs < a.theta * a.theta * R2;
        const int cntn = nd.end - nd.begin;
        int s = -1, e = -1;
        if (sep && nd.prox >= 0) {
            // proxy set: never merged with atom ranges
            if (FILL && m < cap - base) ent[base + m] = make_int2(a.n + nd.prox * a.P3, a.P3);
            ++m;
            ppairs += a.P3;
            last_s = last_e = -1;
            continue;
        }
        if (nd.first_child < 0 || (sep && cntn <= a.P3)) {
            s = nd.begin;
            e = nd.end;
        } else {
            for (int ch = nd.nchild - 1; ch >= 0; --ch)
                if (sp < kStack) stack[sp++] = nd.first_child + ch;
            continue;
        }
        dpairs += e - s;
        if (s == last_e) {
            last_e = e;
            if (FILL && m - 1 < cap - base) ent[base + m - 1].y = last_e - last_s;
        } else {
            if (FILL && m < cap - base) ent[base + m] = make_int2(s, e - s);
            ++m;
            last_s = s;
            last_e = e;
        }
    }
    if (!FILL) {
        cnt[b] = m;
        const long long pts = (long long)a.bx * a.by * a.bz;
        atomicAdd(&meta->direct_pairs, (unsigned long long)(dpairs * pts));
        atomicAdd(&meta->proxy_pairs, (unsigned long long)(ppairs * pts));
    }
}

__global__ void k_scan(int nb, const int* cnt, int* off, int cap, TreeMeta* meta) {
    __shared__ int tmp[64];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? cnt[i] : 0;
        int total;
        const int ex = block_exclusive_scan(v, tmp, total);
        if (i < nb) off[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        off[nb] = carry;
        meta->far_total = carry;
        if (carry > cap) meta->overflow = 1;
    }
}

__global__ void k_reset_meta(TreeMeta* meta) {
    meta->direct_pairs = meta->proxy_pairs = meta->near_pairs = 0ull;
    meta->far_total = 0;
    meta->overflow = 0;
    meta->nnodes = meta->nprox = meta->nitems = meta->nleaves = 0;
    meta->lc = 0;
    meta->cube_lo[0] = meta->cube_lo[1] = meta->cube_lo[2] = 0.0;
    meta->cube_side = meta->cell_side = 1.0;
    meta->rnear = 0.0;
}

// ---------------------------------------------------------------- eval
struct EvalArgs {
    GridD g;
    Phys ph;
    int nbx, nby, nbz;
    int n;
    const Geo* src;        // [sorted atoms | proxies], grid units
    const LJf* ljs;        // sorted LJ tables
    const int* off;        // far-list offsets [nb+1]
    const int2* ent;       // far-list entries
    const int* cell_start; // [8^lc + 1]
    Outputs o;
    DevErr* err;
    TreeMeta* meta;
    long long wlim;
};

// Producer state (thread 0 only): walks the far list, then the cells.
struct Producer {
    int phase;            // 0 far, 1 near, 2 done
    int near_ok;          // the near phase has at least one candidate cell
    int lc;
    double cell_lo[3], cell_side, rnear, rnear2;
    int e, e_end, e_off;  // far entry cursor
    int cx, cy, cz;       // cell cursor
    int c0[3], c1[3];     // cell range
    int cell_pos, cell_end;
    double box_lo[3], box_hi[3];
    unsigned long long near_cand;
};

__device__ __forceinline__ void mbar_expect_tx_only(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int SM>
__device__ int produce_tile(Producer& P, const EvalArgs& a, Geo* sgeo, LJf* slj, uint64_t* bar, int& kind) {
    int filled = 0;
    kind = P.phase;
    while (P.phase == 0 && filled < kT) {
        if (P.e >= P.e_end) {
            P.phase = P.near_ok ? 1 : 2;
            break;
        }
        const int2 en = a.ent[P.e];
        const int take = min(kT - filled, en.y - P.e_off);
        const uint32_t bytes = take * sizeof(Geo);
        mbar_expect_tx_only(bar, bytes);
        bulk_g2s(sgeo + filled, a.src + en.x + P.e_off, bytes, bar);
        filled += take;
        P.e_off += take;
        if (P.e_off >= en.y) {
            ++P.e;
            P.e_off = 0;
        }
    }
    if (filled > 0) {
        mbar_arrive(bar);
        return filled;
    }
    kind = 1;
    while (P.phase == 1 && filled < kT) {
        if (P.cell_pos >= P.cell_end) {
            // advance to the next non-empty cell that can hold a pair within rnear
            bool found = false;
            while (!found) {
                if (++P.cx > P.c1[0]) {
                    P.cx = P.c0[0];
                    if (++P.cy > P.c1[1]) {
                        P.cy = P.c0[1];
                        if (++P.cz > P.c1[2]) {
                            P.phase = 2;
                            break;
                        }
                    }
                }
                // distance between the cell box and the batch box
                const int cc[3] = {P.cx, P.cy, P.cz};
                double d2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                    const double lo = P.cell_lo[d] + cc[d] * P.cell_side, hi = lo + P.cell_side;
                    const double gap = fmax(0.0, fmax(lo - P.box_hi[d], P.box_lo[d] - hi));
                    d2 += gap * gap;
                }
                if (d2 >= P.rnear2) continue;
                const uint32_t m = morton3((uint32_t)P.cx, (uint32_t)P.cy, (uint32_t)P.cz);
                P.cell_pos = a.cell_start[m];
                P.cell_end = a.cell_start[m + 1];
                found = P.cell_pos < P.cell_end;
            }
            if (P.phase == 2) break;
        }
        const int take = min(kT - filled, P.cell_end - P.cell_pos);
        const uint32_t b1 = take * sizeof(Geo), b2 = take * SM * sizeof(LJf);
        mbar_expect_tx_only(bar, b1 + b2);
        bulk_g2s(sgeo + filled, a.src + P.cell_pos, b1, bar);
        bulk_g2s(slj + filled * SM, a.ljs + (int64_t)P.cell_pos * SM, b2, bar);
        filled += take;
        P.cell_pos += take;
    }
    if (filled > 0) {
        mbar_arrive(bar);
        P.near_cand += filled;
    }
    return filled;
}

template <int SM, bool DU, bool DH>
__global__ void __launch_bounds__(kBX* kBY* kBZ) k_eval32(EvalArgs a) {
    constexpr int NT = kBX * kBY * kBZ, P = kP;
    extern __shared__ __align__(16) unsigned char smem[];
    Geo* sgeo = reinterpret_cast<Geo*>(smem);                                        // [2][kT]
    LJf* slj = reinterpret_cast<LJf*>(smem + 2 * kT * sizeof(Geo));                  // [2][kT*SM]
    GeoF* conv = reinterpret_cast<GeoF*>(smem + 2 * kT * sizeof(Geo) + 2 * kT * SM * sizeof(LJf));
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * kT * sizeof(Geo) + 2 * kT * SM * sizeof(LJf) +
                                                kT * sizeof(GeoF));
    __shared__ int s_cnt[2], s_kind[2];
    // lists that overflowed their buffer are incomplete: the host grows them and runs again
    if (a.meta->overflow) return;

    const int tid = threadIdx.x;
    const int tx = tid % kBX, ty = (tid / kBX) % kBY, tz = tid / (kBX * kBY);
    const int b = blockIdx.x;
    const int ib = b % a.nbx, jb = (b / a.nbx) % a.nby, kb = b / (a.nbx * a.nby);
    const int ti0 = ib * (kBX * P), tj0 = jb * kBY, tk0 = kb * kBZ;
    const int i0 = ti0 + tx * P, j = tj0 + ty, k = tk0 + tz;
    const float fx0 = (float)(tx * P), fy = (float)ty, fz = (float)tz;
    const float rs2 = (float)((a.ph.rs / a.g.h) * (a.ph.rs / a.g.h));
    const float xs = (float)(a.g.h / a.ph.eta);
    const float kap2 = (float)(-a.ph.kappa * a.g.h * 1.4426950408889634);
    const float aa_ = (float)a.ph.a;
    const float c0h = (float)(a.ph.phi_c0 * a.g.h), h0h = (float)(a.ph.phi_h0 * a.g.h);
    const bool DC = a.o.c != nullptr;

    float f1h[P], f1l[P], fkh[P], fkl[P], sch[P], scl[P], shh[P], shl[P], ljh[P][SM], ljl[P][SM];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        f1h[p] = f1l[p] = fkh[p] = fkl[p] = sch[p] = scl[p] = shh[p] = shl[p] = 0.f;
#pragma unroll
        for (int s = 0; s < SM; ++s) ljh[p][s] = ljl[p][s] = 0.f;
    }
    unsigned hit = 0u;
    __shared__ float s_rn2;
    if (tid == 0) s_rn2 = isfinite(a.meta->rnear) ? (float)(a.meta->rnear * a.meta->rnear) : INFINITY;

    Producer pr;
    if (tid == 0) {
        const TreeMeta* m = a.meta;
        pr.phase = 0;
        pr.e = a.off[b];
        pr.e_end = a.off[b + 1];
        pr.e_off = 0;
        pr.near_cand = 0;
        pr.lc = m->lc;
        pr.cell_side = m->cell_side;
        pr.rnear = m->rnear;
        pr.rnear2 = isfinite(m->rnear) ? m->rnear * m->rnear : INFINITY;
        for (int d = 0; d < 3; ++d) pr.cell_lo[d] = m->cube_lo[d];
        const double blo[3] = {(double)ti0, (double)tj0, (double)tk0};
        const double bhi[3] = {(double)(ti0 + kBX * P - 1), (double)(tj0 + kBY - 1), (double)(tk0 + kBZ - 1)};
        const int ncell = 1 << pr.lc;
        bool ok = a.n > 0;
        for (int d = 0; d < 3; ++d) {
            pr.box_lo[d] = blo[d];
            pr.box_hi[d] = bhi[d];
            double lo = floor((blo[d] - pr.rnear - pr.cell_lo[d]) / pr.cell_side);
            double hi = floor((bhi[d] + pr.rnear - pr.cell_lo[d]) / pr.cell_side);
            pr.c0[d] = (int)fmax(lo, 0.0);
            pr.c1[d] = (int)fmin(hi, (double)(ncell - 1));
            ok = ok && pr.c0[d] <= pr.c1[d];
        }
        pr.near_ok = ok;
        pr.cx = pr.c0[0] - 1;
        pr.cy = pr.c0[1];
        pr.cz = pr.c0[2];
        pr.cell_pos = pr.cell_end = 0;
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (int st = 0; st < 2; ++st) {
            int kind;
            int c = (pr.phase < 2) ? produce_tile<SM>(pr, a, sgeo + st * kT, slj + st * kT * SM, &bar[st], kind) : 0;
            s_cnt[st] = c;
            s_kind[st] = kind;
        }
    }
    __syncthreads();
    for (int t = 0;; ++t) {
        const int st = t & 1;
        const int cnt = s_cnt[st];
        if (cnt == 0) break;
        const bool near = s_kind[st] == 1;
        bool ok = mbar_wait_bounded(&bar[st], (t >> 1) & 1, a.wlim);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                report_error(a.err, DEV_TIMEOUT, WHERE_TREE_EVAL);
                for (int u2 = t; u2 < t + 2; ++u2)
                    if (s_cnt[u2 & 1] > 0) mbar_wait_bounded(&bar[u2 & 1], (u2 >> 1) & 1, a.wlim);
            }
            return;
        }
        if (tid < cnt) {
            const Geo A = sgeo[st * kT + tid];
            GeoF c;
            split_ff(A.x - (double)ti0, c.xh, c.xl);
            split_ff(A.y - (double)tj0, c.yh, c.yl);
            split_ff(A.z - (double)tk0, c.zh, c.zl);
            c.q = (float)A.q;
            c.pad = 0.f;
            conv[tid] = c;
        }
        __syncthreads();
        if (!near) {
            float p1[P], pk[P];
#pragma unroll
            for (int p = 0; p < P; ++p) p1[p] = pk[p] = 0.f;
            for (int s0 = 0; s0 < cnt; ++s0) {
                const float4 g0 = *reinterpret_cast<const float4*>(&conv[s0].xh);
                const float4 g1 = *reinterpret_cast<const float4*>(&conv[s0].xl);
                const float dy = (fy - g0.y) - g1.y;
                const float dz = (fz - g0.z) - g1.z;
                const float dyz2 = fmaf(dy, dy, dz * dz);
                const float bx = fx0 - g0.x;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const float dx = (bx + (float)p) - g1.x;
                    const float d2 = fmaf(dx, dx, dyz2);
                    const float rr = rsqrt_approx(d2);
                    const float ri = d2 > 0.f ? rr : 0.f;
                    const float qr = g0.w * ri;
                    p1[p] += qr;
                    if (DH) pk[p] = fmaf(qr, ex2_approx(kap2 * (d2 * ri)), pk[p]);
                }
            }
#pragma unroll
            for (int p = 0; p < P; ++p) {
                ff_add(f1h[p], f1l[p], p1[p]);
                if (DH) ff_add(fkh[p], fkl[p], pk[p]);
            }
        } else {
            const LJf* L = slj + st * kT * SM;
            const float rn2 = s_rn2;
            float psc[P], psh[P], plj[P][SM];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                psc[p] = psh[p] = 0.f;
#pragma unroll
                for (int s = 0; s < SM; ++s) plj[p][s] = 0.f;
            }
            for (int s0 = 0; s0 < cnt; ++s0) {
                const float4 g0 = *reinterpret_cast<const float4*>(&conv[s0].xh);
                const float4 g1 = *reinterpret_cast<const float4*>(&conv[s0].xl);
                const float dy = (fy - g0.y) - g1.y;
                const float dz = (fz - g0.z) - g1.z;
                const float dyz2 = fmaf(dy, dy, dz * dz);
                const float bx = fx0 - g0.x;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const float dx = (bx + (float)p) - g1.x;
                    const float d2 = fmaf(dx, dx, dyz2);
                    if (d2 >= rn2) continue;
                    if (d2 < rs2) {
                        if (d2 > 0.f) {
                            const float ri = rsqrt_approx(d2);
                            const float qr = g0.w * ri;
                            const float x = d2 * ri * xs;
                            if (DC) psc[p] = fmaf(qr, erfcf(x), psc[p]);
                            if (DH) psh[p] = fmaf(qr, __expf(-x * x) * (erfcxf(x - aa_) + erfcxf(x + aa_)), psh[p]);
                        } else {
                            hit |= 1u << p;
                            if (DC) psc[p] -= g0.w * c0h;
                            if (DH) psh[p] -= g0.w * h0h;
                        }
                    }
                    if (DU) {
                        const float r2i = rcp_approx(d2);
                        const float r6 = r2i * r2i * r2i;
#pragma unroll
                        for (int s = 0; s < SM; ++s) {
                            const float4 l = *reinterpret_cast<const float4*>(&L[s0 * SM + s]);
                            if (d2 < l.z) plj[p][s] = fmaf(r6, fmaf(l.x, r6, -l.y), plj[p][s]);
                        }
                    }
                }
            }
#pragma unroll
            for (int p = 0; p < P; ++p) {
                if (DC) ff_add(sch[p], scl[p], psc[p]);
                if (DH) ff_add(shh[p], shl[p], psh[p]);
                if (DU) {
#pragma unroll
                    for (int s = 0; s < SM; ++s) ff_add(ljh[p][s], ljl[p][s], plj[p][s]);
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            int kind = 2;
            int c = (pr.phase < 2) ? produce_tile<SM>(pr, a, sgeo + st * kT, slj + st * kT * SM, &bar[st], kind) : 0;
            s_cnt[st] = c;
            s_kind[st] = kind;
        }
        __syncthreads();
    }
    if (tid == 0) atomicAdd(&a.meta->near_pairs, pr.near_cand * (unsigned long long)(NT * P));

    const GridD& g = a.g;
    if (j >= g.ny || k >= g.nz || i0 >= g.nx) return;
    const int64_t plane = (int64_t)g.nx * g.ny * g.nz;
    const int64_t row = ((int64_t)k * g.ny + j) * g.nx;
    const bool vec_ok = (g.nx & 1) == 0;
    const double ih = 1.0 / g.h;
    const Phys& ph = a.ph;
    const double cu0 = ph.k_e * ih, cc0 = -ph.beta * ph.k_e * ih, ch0 = -ph.beta * ph.k_e / (2.0 * ph.eps_r) * ih;
    double F1[P], FK[P], SC[P], SH[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        F1[p] = (double)f1h[p] + (double)f1l[p];
        FK[p] = (double)fkh[p] + (double)fkl[p];
        SC[p] = (double)sch[p] + (double)scl[p];
        SH[p] = (double)shh[p] + (double)shl[p];
    }
    auto store = [&](double* base, const double (&v)[P]) {
        if (vec_ok && i0 + P <= g.nx) {
#pragma unroll
            for (int p = 0; p < P; p += 2)
                __stcs(reinterpret_cast<double2*>(base + i0 + p), make_double2(v[p], v[p + 1]));
        } else {
#pragma unroll
            for (int p = 0; p < P; ++p)
                if (i0 + p < g.nx) __stcs(base + i0 + p, v[p]);
        }
    };
#pragma unroll
    for (int s = 0; s < SM; ++s) {
        if (s >= ph.S) break;
        const double qs = ph.qs[s];
        double v[P];
        if (DU) {
#pragma unroll
            for (int p = 0; p < P; ++p)
                v[p] = (hit >> p & 1u) ? INFINITY : cu0 * qs * F1[p] + ((double)ljh[p][s] + (double)ljl[p][s]);
            store(a.o.u + s * plane + row, v);
        }
        if (DC) {
#pragma unroll
            for (int p = 0; p < P; ++p) v[p] = cc0 * qs * (F1[p] - SC[p]);
            store(a.o.c + s * plane + row, v);
        }
        if (DH) {
#pragma unroll
            for (int p = 0; p < P; ++p) v[p] = ch0 * qs * (2.0 * ph.ea2 * FK[p] - SH[p]);
            store(a.o.h + s * plane + row, v);
        }
    }
}

template <int SM>
cudaError_t launch_eval(const EvalArgs& a, int nb, cudaStream_t st) {
    const size_t sm = 2 * kT * sizeof(Geo) + 2 * kT * SM * sizeof(LJf) + kT * sizeof(GeoF) + 2 * sizeof(uint64_t);
    const bool du = a.o.u != nullptr, dh = a.o.h != nullptr;
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        kern<<<nb, kBX * kBY * kBZ, sm, st>>>(a);
    };
    if (du && dh) go(k_eval32<SM, true, true>);
    else if (du) go(k_eval32<SM, true, false>);
    else if (dh) go(k_eval32<SM, false, true>);
    else go(k_eval32<SM, false, false>);
    return cudaGetLastError();
}

}  // namespace

// ------------------------------------------------------------- state
struct TreeState {
    int64_t cap_n = 0;
    int cap_nodes = 0, cap_prox = 0, cap_items = 0, cap_far = 0, cap_nb = 0;
    int deg = 0, smax = 0;
    uint32_t *code = nullptr, *idx = nullptr, *code2 = nullptr, *idx2 = nullptr;
    Node* nodes = nullptr;
    int* items = nullptr;
    int* prox_nodes = nullptr;
    double* part = nullptr;
    Geo* src = nullptr;
    LJf* ljs = nullptr;
    int* cnt = nullptr;
    int* off = nullptr;
    int2* ent = nullptr;
    int* cell_start = nullptr;
    TreeMeta* meta = nullptr;
    TreeMeta* h_meta = nullptr;  // pinned copy, filled at the end of tree_eval
    int nb = 0, nbx = 0, nby = 0, nbz = 0;
    int launches = 0;
    bool prepared = false;
};

namespace {
constexpr int kMaxCells = (1 << 21) + 1;  // 8^7 + 1

void free_state(TreeState* s) {
    cudaFree(s->code);
    cudaFree(s->idx);
    cudaFree(s->code2);
    cudaFree(s->idx2);
    cudaFree(s->nodes);
    cudaFree(s->items);
    cudaFree(s->prox_nodes);
    cudaFree(s->part);
    cudaFree(s->src);
    cudaFree(s->ljs);
    cudaFree(s->cnt);
    cudaFree(s->off);
    cudaFree(s->ent);
    cudaFree(s->cell_start);
    cudaFree(s->meta);
    cudaFreeHost(s->h_meta);
}

rism_status cuda_err(std::string& err, cudaError_t e, const char* what) {
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? RISM_E_NOMEM : RISM_E_CUDA;
}

template <typename T>
cudaError_t regrow(T*& p, size_t count) {
    cudaFree(p);
    p = nullptr;
    return cudaMalloc(&p, (count > 0 ? count : 1) * sizeof(T));
}
}  // namespace

TreeState* tree_create() { return new TreeState(); }

void tree_destroy(TreeState* ts) {
    if (!ts) return;
    free_state(ts);
    delete ts;
}

// Enqueue a7..a9: codes, sort, octree, boxes, sorted sources, cells, upward
// pass and interaction lists.  Sizes that depend on the atoms are read by the
// kernels from the device meta block; nothing here waits for the GPU.
rism_status tree_prepare(TreeState* s, const DevTables& t, const GridD& g, const Phys& ph, const rism_options& o,
                         cudaStream_t st, std::string& err) {
    cudaError_t e = cudaSuccess;
    const int n = (int)t.n;
    const int deg = o.degree, np = deg + 1, P3 = np * np * np;
    s->nbx = (g.nx + kBX * kP - 1) / (kBX * kP);
    s->nby = (g.ny + kBY - 1) / kBY;
    s->nbz = (g.nz + kBZ - 1) / kBZ;
    s->nb = s->nbx * s->nby * s->nbz;
    // Capacity bounds.  Internal nodes hold > leaf atoms and are disjoint per level, so there are at most
    // n/(leaf+1) per level and 10 levels; each has at most 8 children.  Proxy sets hold > P3 atoms, so at most
    // n/(P3+1) per level.  Upward items are chunks of kChunk atoms of proxied nodes.
    const int max_nodes = (int)(90LL * n / (o.leaf + 1)) + 16;
    const int max_prox = 10 * n / (P3 + 1) + 2;
    const int max_items = 10 * (n / kChunk + 1) + 2;
    if (!s->meta) {
        if ((e = cudaMalloc(&s->meta, sizeof(TreeMeta))) != cudaSuccess) return cuda_err(err, e, "tree meta");
        if ((e = cudaMallocHost(&s->h_meta, sizeof(TreeMeta))) != cudaSuccess) return cuda_err(err, e, "tree meta");
        if ((e = regrow(s->cell_start, (size_t)kMaxCells)) != cudaSuccess) return cuda_err(err, e, "cell table");
    }
    if (n > s->cap_n || t.smax != s->smax || max_nodes > s->cap_nodes || deg != s->deg) {
        const size_t nn = n > 0 ? (size_t)n : 1;
        if ((e = regrow(s->code, nn)) || (e = regrow(s->idx, nn)) || (e = regrow(s->code2, nn)) ||
            (e = regrow(s->idx2, nn)) || (e = regrow(s->nodes, (size_t)max_nodes)) ||
            (e = regrow(s->items, 2 * (size_t)max_items)) || (e = regrow(s->prox_nodes, (size_t)max_prox)) ||
            (e = regrow(s->part, (size_t)max_items * P3)) || (e = regrow(s->src, nn + (size_t)max_prox * P3)) ||
            (e = regrow(s->ljs, nn * t.smax)))
            return cuda_err(err, e, "tree buffers");
        s->cap_n = (int64_t)nn;
        s->cap_nodes = max_nodes;
        s->cap_prox = max_prox;
        s->cap_items = max_items;
        s->smax = t.smax;
        s->deg = deg;
    }
    if (s->nb + 1 > s->cap_nb) {
        if ((e = regrow(s->cnt, (size_t)s->nb + 1)) || (e = regrow(s->off, (size_t)s->nb + 1)))
            return cuda_err(err, e, "list offsets");
        s->cap_nb = s->nb + 1;
    }
    if (s->cap_far < s->nb * 16 + 1024) {
        const int want = s->nb * 16 + 1024;
        if ((e = regrow(s->ent, (size_t)want))) return cuda_err(err, e, "far list");
        s->cap_far = want;
    }
    s->launches = 0;
    k_reset_meta<<<1, 1, 0, st>>>(s->meta);
    ++s->launches;
    if (n > 0) {
        k_bbox_codes<<<1, kSortThreads, 0, st>>>(t.geoU, t.ljd, n, ph.S, t.smax, ph.rs, g.h, s->meta, s->code, s->idx);
        BuildArgs ba{n, o.leaf, P3, max_nodes, max_prox, max_items};
        const size_t shb = (256 * 32 + 64) * sizeof(int);
        cudaFuncSetAttribute(k_sort_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shb);
        k_sort_build<<<1, kSortThreads, shb, st>>>(ba, s->code, s->idx, s->code2, s->idx2, s->nodes, s->items,
                                                   s->prox_nodes, s->meta);
        k_node_boxes<<<152, 256, 0, st>>>(s->nodes, s->meta, s->idx, t.geoU);
        k_gather<<<(n + 255) / 256, 256, 0, st>>>(n, t.smax, s->idx, t.geoU, t.ljf, s->src, s->ljs);
        k_cells<<<1024, 256, 0, st>>>(n, s->meta, s->code, s->cell_start);
        const size_t shu = (kChunk * 3 * np + kChunk) * sizeof(double);
        cudaFuncSetAttribute(k_upward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shu);
        k_upward<<<4 * 152, 256, shu, st>>>(deg, s->meta, s->nodes, s->prox_nodes, s->items, s->src, s->part);
        k_proxy_reduce<<<152, 256, 0, st>>>(deg, n, s->meta, s->nodes, s->prox_nodes, s->items, s->part, s->src);
        s->launches += 7;
    }
    ListArgs la{s->nbx, s->nby, s->nbz, kBX * kP, kBY, kBZ, o.theta, n, P3, s->cap_far};
    k_lists<false><<<(s->nb + 127) / 128, 128, 0, st>>>(la, s->nodes, s->off, s->ent, s->cnt, s->meta);
    k_scan<<<1, 1024, 0, st>>>(s->nb, s->cnt, s->off, s->cap_far, s->meta);
    k_lists<true><<<(s->nb + 127) / 128, 128, 0, st>>>(la, s->nodes, s->off, s->ent, s->cnt, s->meta);
    s->launches += 3;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(err, e, "tree build");
    s->prepared = true;
    return RISM_OK;
}

// Enqueue a10 + a11: the fused far/near evaluation and epilogue, then a copy
// of the meta block (counts, overflow flag) to pinned memory for tree_post.
rism_status tree_eval(TreeState* s, const DevTables& t, const GridD& g, const Phys& ph, const rism_options& o,
                      Outputs out, cudaStream_t st, std::string& err, rism_info& info) {
    if (!s->prepared) {
        err = "tree not prepared";
        return RISM_E_STATE;
    }
    EvalArgs a;
    a.g = g;
    a.ph = ph;
    a.nbx = s->nbx;
    a.nby = s->nby;
    a.nbz = s->nbz;
    a.n = (int)t.n;
    a.src = s->src;
    a.ljs = s->ljs;
    a.off = s->off;
    a.ent = s->ent;
    a.cell_start = s->cell_start;
    a.o = out;
    a.err = t.err;
    a.meta = s->meta;
    a.wlim = o.wait_limit;
    cudaError_t e;
    switch (t.smax) {
        case 2: e = launch_eval<2>(a, s->nb, st); break;
        case 4: e = launch_eval<4>(a, s->nb, st); break;
        default: e = launch_eval<8>(a, s->nb, st); break;
    }
    if (e != cudaSuccess) return cuda_err(err, e, "tree eval");
    if ((e = cudaMemcpyAsync(s->h_meta, s->meta, sizeof(TreeMeta), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_err(err, e, "tree meta copy");
    info.launches += s->launches + 1;
    info.batch[0] = kBX * kP;
    info.batch[1] = kBY;
    info.batch[2] = kBZ;
    return RISM_OK;
}

// After the stream has been synchronised: counters into info; a far-list
// overflow grows the buffer and asks the caller to run prepare + eval again.
rism_status tree_post(TreeState* s, rism_info& info, bool& retry, std::string& err) {
    const TreeMeta& m = *s->h_meta;
    retry = false;
    if (m.overflow) {
        if (m.far_total + 1024 > s->cap_far) {
            const int want = m.far_total + m.far_total / 4 + 1024;
            cudaError_t e = regrow(s->ent, (size_t)want);
            if (e != cudaSuccess) return cuda_err(err, e, "far list");
            s->cap_far = want;
            retry = true;
            return RISM_OK;
        }
        err = "tree node or proxy capacity exceeded";
        return RISM_E_NOMEM;
    }
    info.tree_nodes = m.nnodes;
    info.tree_proxied = m.nprox;
    info.tree_leaves = m.nleaves;
    info.direct_pairs = (int64_t)m.direct_pairs;
    info.proxy_pairs = (int64_t)m.proxy_pairs;
    info.near_pairs = (int64_t)m.near_pairs;
    return RISM_OK;
}

rism_status batch_eval(std::vector<BatchItem>&, const rism_options&, cudaStream_t, DevErr*, std::string& msg) {
    msg = "batched launch not built";
    return RISM_E_UNSUPPORTED;
}

}  // namespace rism
