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
// tree is built from, so one device sort serves both.
//
// Pipeline (all on the context's stream, no host synchronisation, so that it
// can be captured in a CUDA graph):
//   k_bounds -> k_codes (Morton cube, codes, near-field plan) -> k_sort_build
//   (one CTA: sort, octree, proxy plan, node boxes) -> k_gather_cells (sorted
//   tables, cell table) -> k_upward -> k_proxy_reduce (source proxies only)
//   -> k_tbox_lists per level (target boxes) -> k_far_lists / k_near_lists
//   (one warp per batch, per-batch slots) -> k_order -> k_cp_eval ->
//   k_cp_reduce -> k_l2l per level -> k_tdown (box-level far field)
//   -> k_far32 (far field) -> k_near32 (near field + epilogue).
// Many solutes: the same per-solute preparation, then one persistent far
// and one persistent near kernel draining all (solute, batch) work items.
// List capacities are checked on the device; an overflow is reported through
// the meta block and the host grows the buffers and runs again.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "rism_tree.h"

namespace rism {

namespace {

constexpr int kSortThreads = 1024;
// The radix histograms hold one count per (digit, warp), stored digit-major with a pitch of 33 so that the 32
// lanes of a warp, which update the entries of one warp column under different digits, fall in different banks
// (a pitch of 32 would put a whole warp's updates in one bank).
constexpr int kHistPitch = kSortThreads / 32 + 1;
constexpr int kHistInts = 256 * kHistPitch;
static_assert(kHistInts % 2 == 0, "the 64-bit sort keys after the histograms stay 8-byte aligned");
constexpr int kSortSmem = 4096;  // atoms sorted in shared memory (64-bit keys, sorted codes, positions: 96 KB)
constexpr int kNodeSmem = 1024;  // octree nodes kept in shared memory during the build (56 KB)
// Above kSortSmem atoms the keys are radix-sorted: up to kCodeSmem atoms in shared memory, where the sorted codes
// (64 KB) then stay for the octree's searches beside up to kNodeSmemL nodes (112 KB); beyond that through global
// memory.
constexpr int kCodeSmem = 16384;
constexpr int kNodeSmemL = 2048;
constexpr int kMortonBits = 10;          // per axis
constexpr int kMaxLevel = kMortonBits;   // octree depth limit
constexpr int kChunk = 16;               // atoms per upward-pass work item
constexpr int kT = 64;                   // sources per shared-memory tile (<= 64: the near culling uses two ballots)
constexpr double kCellFrac = 0.25;        // near-field cells are at least this fraction of the near radius wide

struct Node {
    int begin, end;        // range in the sorted atom order
    int first_child;       // index of the first child, -1 for a leaf
    int nchild;
    int level;
    int prox;              // proxy set index, -1 if none
    int pad0, pad1;
    float lo[3], hi[3];    // bounding box of the atoms' positions (grid units, FP32 high parts)
};

struct TreeMeta {
    int nnodes, nprox, nitems, nleaves;
    int overflow;          // any capacity exceeded (nodes, proxies, items, list slots, frontier)
    int build_overflow;    // the tree itself is incomplete (nodes, proxies, items)
    int far_need;          // largest far list of a batch (entries)
    int near_need;         // largest near list of a batch (entries)
    int wide;              // a traversal frontier exceeded kQCap
    int lc;                // cell level of the near field
    int bmin[3], bmax[3];  // atom bounds, order-preserving int encoding of the FP32 grid-unit positions
    int rc2max;            // largest per-pair LJ cut-off squared (grid units, FP32 bits; +inf without cut-off)
    int pad;
    double cube_lo[3];     // Morton cube (grid units)
    double cube_side;
    double cell_side;      // cube_side / 2^lc
    double rnear;          // near-field radius (grid units): max(largest LJ cut-off, r_short)
    unsigned long long direct_pairs, proxy_pairs, near_pairs;
    unsigned long long cp_pairs;  // (target proxy, atom) pairs of the box-level far field
    unsigned long long near_tested, lj_pairs, sr_pairs;  // near kernel: pairs tested, inside the LJ cut-off,
                                                          // inside r_short (d > 0)
    int cp_need, dn_need;  // largest accepted-range list / pass-down list of a target box
    int tboxes;            // target boxes that took proxies and have a non-empty list
    int pad2;
};

// ------------------------------------------------ target boxes (cluster-particle far field)
// Aligned cubes of the grid with edge 16 << l points (level l = 0 .. L-1), clipped to the grid.  A box with at
// least n+1 points along each axis and more than (n+1)^3 points takes (n+1)^3 Chebyshev proxy targets; its
// accepted source clusters are summed at the proxies and reach the grid points by interpolation.
constexpr int kMaxTL = 16;
constexpr int kTB0 = 16;   // edge of a level-0 box (points)

struct TBoxes {
    int L, nbox;
    int nbx[kMaxTL], nby[kMaxTL], nbz[kMaxTL], off[kMaxTL];
    int nx, ny, nz;
    int deg, P3;
    int enabled;
    int approx;                // RISM_APPROX_BARYCENTRIC: Chebyshev proxies; RISM_APPROX_TAYLOR: Taylor moments
    float kapg;                // kappa in 1/grid units (Taylor moments of e^{-kappa d}/d)
    float ck[kMaxDegree + 1];  // cos(k pi / n), exact 1, 0, -1 where they occur
};

// Centre and radius in FP32: the centre lo + (ext - 1) / 2 is a half-integer and r^2 a quarter-integer, both
// exact; r is the correctly rounded square root (no FP64 instruction in the kernels that place boxes).
struct TBox {
    int l, ib, jb, kb;
    int lo[3], ext[3];
    float c[3], r;
    bool proxied;
};

__host__ __device__ inline TBox tbox_at(const TBoxes& tb, int l, int ib, int jb, int kb) {
    TBox b;
    b.l = l;
    b.ib = ib;
    b.jb = jb;
    b.kb = kb;
    const int E = kTB0 << l;
    const int n[3] = {tb.nx, tb.ny, tb.nz}, ix[3] = {ib, jb, kb};
    float r2 = 0.f;
    long long pts = 1;
    bool big = true;
    for (int d = 0; d < 3; ++d) {
        b.lo[d] = ix[d] * E;
        b.ext[d] = n[d] - b.lo[d] < E ? n[d] - b.lo[d] : E;
        b.c[d] = (float)b.lo[d] + 0.5f * (float)(b.ext[d] - 1);
        r2 += 0.25f * (float)((b.ext[d] - 1) * (b.ext[d] - 1));
        pts *= b.ext[d];
        big = big && b.ext[d] >= tb.deg + 1;
    }
    b.r = sqrtf(r2);
    b.proxied = tb.enabled && big && pts > tb.P3;
    return b;
}

__host__ __device__ inline int tbox_index(const TBoxes& tb, int l, int ib, int jb, int kb) {
    return tb.off[l] + (kb * tb.nby[l] + jb) * tb.nbx[l] + ib;
}

__host__ __device__ inline TBox tbox_flat(const TBoxes& tb, int box) {
    int l = 0;
    while (l + 1 < tb.L && tb.off[l + 1] <= box) ++l;
    const int bi = box - tb.off[l];
    return tbox_at(tb, l, bi % tb.nbx[l], (bi / tb.nbx[l]) % tb.nby[l], bi / (tb.nbx[l] * tb.nby[l]));
}

// Lagrange basis of the (n+1) Chebyshev points of the second kind of an interval with half-width hw, in
// barycentric form with weights (-1)^k (halved at both ends), evaluated at offset t from the interval's
// centre.  Node k sits at hw ck[k] -- the same FP32 product the proxy kernel places its targets at.
__device__ inline void cheb_basis(int n, const float* ck, float hw, float t, float* L) {
    float den = 0.f;
    int hit = -1;
    for (int k = 0; k <= n; ++k) {
        const float dx = t - hw * ck[k];
        if (dx == 0.f) hit = k;
        float w = (k & 1) ? -1.f : 1.f;
        if (k == 0 || k == n) w *= 0.5f;
        L[k] = dx != 0.f ? w / dx : 0.f;
        den += L[k];
    }
    if (hit >= 0) {
        for (int k = 0; k <= n; ++k) L[k] = k == hit ? 1.f : 0.f;
        return;
    }
    const float inv = 1.f / den;
    for (int k = 0; k <= n; ++k) L[k] *= inv;
}

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
__device__ __forceinline__ Geo to_grid(const Geo& p, const GridD& g, double ih) {
    return Geo{(p.x - g.ox) * ih, (p.y - g.oy) * ih, (p.z - g.oz) * ih, p.q};
}

// Order-preserving int encoding of a float (for atomicMin / atomicMax).
__device__ __forceinline__ int f2ord(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

// Atom bounds (grid units, from the float-float source table) and the
// largest LJ cut-off, reduced with atomics into the meta block.
__global__ void k_bounds(const SrcF* __restrict__ srcf, const LJf* __restrict__ ljf, int n, int S, int smax,
                         TreeMeta* meta) {
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    int rc = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const SrcF s = srcf[i];
        const int v[3] = {f2ord(s.xh), f2ord(s.yh), f2ord(s.zh)};
        for (int d = 0; d < 3; ++d) {
            lo[d] = min(lo[d], v[d]);
            hi[d] = max(hi[d], v[d]);
        }
        for (int k = 0; k < S; ++k) rc = max(rc, __float_as_int(ljf[(int64_t)i * smax + k].rc2));
    }
    for (int o = 16; o > 0; o >>= 1) {
        for (int d = 0; d < 3; ++d) {
            lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
        rc = max(rc, __shfl_xor_sync(0xffffffffu, rc, o));
    }
    if ((threadIdx.x & 31) == 0) {
        for (int d = 0; d < 3; ++d) {
            atomicMin(&meta->bmin[d], lo[d]);
            atomicMax(&meta->bmax[d], hi[d]);
        }
        atomicMax(&meta->rc2max, rc);  // non-negative floats order as ints
    }
}

// Morton cube (a cube containing the atom bounds with a one-grid-unit
// margin), Morton codes of the atoms, and the near-field plan: radius =
// max(largest LJ cut-off, r_short); cells at least half that radius wide,
// at most 8^7 of them.  Every thread derives the same cube from the bounds.
__global__ void k_codes(const SrcF* __restrict__ srcf, int n, double rs_grid, TreeMeta* meta, uint32_t* code,
                        uint32_t* idx) {
    float lo[3];
    float L = 0.f;
    for (int d = 0; d < 3; ++d) {
        lo[d] = ord2f(meta->bmin[d]) - 1.0f;
        L = fmaxf(L, ord2f(meta->bmax[d]) + 1.0f - lo[d]);
    }
    const float sc = (float)(1 << kMortonBits) / L;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int d = 0; d < 3; ++d) meta->cube_lo[d] = lo[d];
        meta->cube_side = L;
        const float rc2 = __int_as_float(meta->rc2max);
        const double rnear = fmax(sqrt((double)rc2), rs_grid);  // infinite without an LJ cut-off
        int lc = 0;
        if (isfinite(rnear))
            while (lc < 7 && (double)L / (double)(1 << (lc + 1)) >= kCellFrac * rnear) ++lc;
        meta->lc = lc;
        meta->cell_side = (double)L / (double)(1 << lc);
        meta->rnear = rnear;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const SrcF s = srcf[i];
        const float v[3] = {s.xh, s.yh, s.zh};
        uint32_t c[3];
        for (int d = 0; d < 3; ++d) {
            const float tt = floorf((v[d] - lo[d]) * sc);
            c[d] = (uint32_t)fminf(fmaxf(tt, 0.f), (float)((1 << kMortonBits) - 1));
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
    const Geo* geo;        // physical positions (unsorted)
    const SrcF* srcf;      // float-float grid-unit positions (unsorted)
    const LJf* ljf;        // LJ tables (unsorted)
    int smax;
    GridD gd;
    double ih;             // 1 / h
    Geo* src;              // out: sorted FP64 grid units (null: not needed)
    SrcF* ssrcf;           // out: sorted float-float
    LJf* ljs;              // out: sorted LJ tables
    LJf* ljs2;             // out: the same as {A, A, -B, -B} (two-wide operands of the near field)
};

// Lanes of the warp whose 8-bit digit equals this lane's, among the lanes with act set: eight ballots, one per
// bit (a match instruction costs far more when a warp holds many distinct digits).  Every lane of the warp calls
// it; the result of a lane with act unset is unused.
__device__ __forceinline__ unsigned warp_digit_peers(uint32_t d, bool act) {
    unsigned m = __ballot_sync(0xffffffffu, act);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1u;
        const unsigned bb = __ballot_sync(0xffffffffu, bit);
        m &= bit ? bb : ~bb;
    }
    return m;
}

// Shared-memory slot of the radix histogram entry at (digit, warp)-order position L.
__device__ __forceinline__ int hist_at(int L) { return (L >> 5) * kHistPitch + (L & 31); }

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
                                                             int* items, int* prox_nodes, int* prox_items,
                                                             TreeMeta* meta) {
    extern __shared__ int sh[];
    int* hist = sh;                     // [256][kHistPitch]: radix histograms, (digit, warp) order
    int* tmp = sh + kHistInts;          // [64]
    const int n = a.n;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int NW = kSortThreads / 32;
    const int seg = ((n + NW - 1) / NW + 31) / 32 * 32;
    const int s0 = min(n, w * seg), s1 = min(n, s0 + seg);
    // up to kSortSmem atoms: a bitonic sort in shared memory of the 64-bit keys (code << 32 | index), unique,
    // so the order is that of the stable radix sort; the sorted codes stay there for the octree's searches.
    // Above that: the stable LSD radix sort, in shared memory up to kCodeSmem atoms, else through global memory.
    const bool in_smem = n <= kSortSmem;
    unsigned long long* sk = reinterpret_cast<unsigned long long*>(sh + kHistInts + 64);  // [kSortSmem]
    uint32_t* sc = reinterpret_cast<uint32_t*>(sk + kSortSmem);                          // [kSortSmem]
    if (in_smem) {
        // Bucket sort on the top 10 bits of the code, one bucket per thread: count, scan, scatter, then each
        // thread sorts its bucket by insertion on the unique 64-bit keys (the result does not depend on the
        // order of the scatter).  A bucket of more than kBucketMax keys (clustered atoms) hands over to the
        // bitonic sort below.
        static_assert(kSortThreads == 1024 && kSortSmem % kSortThreads == 0, "one bucket per thread");
        constexpr int KPT = kSortSmem / kSortThreads, kBucketShift = 3 * kMortonBits - 10, kBucketMax = 32;
        int* bcnt = hist;  // [1024] keys per bucket (the radix histogram is unused on this path)
        __shared__ int s_bmax;
        if (threadIdx.x == 0) s_bmax = 0;
        bcnt[threadIdx.x] = 0;
        __syncthreads();
        unsigned long long key[KPT];
        int slot[KPT];
#pragma unroll
        for (int u = 0; u < KPT; ++u) {
            const int i = threadIdx.x + u * kSortThreads;
            const uint32_t cd = i < n ? code[i] : 0u;
            key[u] = ((unsigned long long)cd << 32) | (i < n ? idx[i] : 0u);
            slot[u] = i < n ? atomicAdd(&bcnt[cd >> kBucketShift], 1) : 0;
        }
        __syncthreads();
        const int mycnt = bcnt[threadIdx.x];
        atomicMax(&s_bmax, mycnt);
        int total;
        const int start = block_exclusive_scan(mycnt, tmp, total);
        bcnt[kSortThreads + threadIdx.x] = start;  // bucket starts
        __syncthreads();
        const bool buckets = s_bmax <= kBucketMax;
        if (buckets) {
#pragma unroll
            for (int u = 0; u < KPT; ++u) {
                const int i = threadIdx.x + u * kSortThreads;
                if (i < n) sk[bcnt[kSortThreads + ((uint32_t)(key[u] >> 32) >> kBucketShift)] + slot[u]] = key[u];
            }
            __syncthreads();
            for (int x = start + 1; x < start + mycnt; ++x) {
                const unsigned long long v = sk[x];
                int y = x - 1;
                while (y >= start && sk[y] > v) {
                    sk[y + 1] = sk[y];
                    --y;
                }
                sk[y + 1] = v;
            }
            __syncthreads();
        }
        int N = 1;
        while (N < n) N <<= 1;
        if (!buckets) {
            for (int i = threadIdx.x; i < N; i += blockDim.x)
                sk[i] = i < n ? ((unsigned long long)code[i] << 32) | idx[i] : ~0ull;
            __syncthreads();
        }
        // a stage with j <= 32 pairs elements within the 64 of one warp (per 32 consecutive t), so between two
        // such stages the warp synchronises alone
        for (int k = 2; k <= (buckets ? 1 : N); k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int t = threadIdx.x; t < N / 2; t += blockDim.x) {
                    const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1)), l = i + j;
                    const unsigned long long x = sk[i], y = sk[l];
                    if ((x > y) == ((i & k) == 0)) {
                        sk[i] = y;
                        sk[l] = x;
                    }
                }
                const int jn = j > 1 ? j >> 1 : k;  // j of the next stage
                if (j >= 64 || jn >= 64)
                    __syncthreads();
                else
                    __syncwarp();
            }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const unsigned long long v = sk[i];
            sc[i] = code[i] = (uint32_t)(v >> 32);
            idx[i] = (uint32_t)v;
        }
        __syncthreads();
    } else if (n <= kCodeSmem) {
        // mid-sized solutes: the same stable LSD radix sort with the keys and values in shared memory.  Each
        // warp holds its segment (<= 16 keys per lane) in registers through a pass, so the scatter of a pass
        // writes in place (every key of the pass has been read before the first barrier); the scatter of
        // single words to global memory would cost a memory transaction each.
        constexpr int KPL = kCodeSmem / kSortThreads;  // 16
        uint32_t* skm = reinterpret_cast<uint32_t*>(sh + kHistInts + 64);  // [kCodeSmem] keys
        uint32_t* svm = skm + kCodeSmem;                                     // [kCodeSmem] values
        for (int pass = 0; pass < 4; ++pass) {
            const int shift = 8 * pass;
            const uint32_t* kin = pass == 0 ? code : skm;
            const uint32_t* vin = pass == 0 ? idx : svm;
            uint32_t kr[KPL], vr[KPL];
#pragma unroll
            for (int j = 0; j < KPL; ++j) {
                const int i = s0 + 32 * j + lane;
                const bool act = i < s1;
                kr[j] = act ? kin[i] : 0u;
                vr[j] = act ? vin[i] : 0u;
            }
            for (int k = threadIdx.x; k < kHistInts; k += blockDim.x) hist[k] = 0;
            __syncthreads();
#pragma unroll
            for (int j = 0; j < KPL; ++j)
                if (s0 + 32 * j + lane < s1) atomicAdd(&hist[((kr[j] >> shift) & 255u) * kHistPitch + w], 1);
            __syncthreads();
            {
                int loc[8], sum = 0;
                for (int k = 0; k < 8; ++k) {
                    loc[k] = hist[hist_at(threadIdx.x * 8 + k)];
                    sum += loc[k];
                }
                int total;
                int base = block_exclusive_scan(sum, tmp, total);
                for (int k = 0; k < 8; ++k) {
                    hist[hist_at(threadIdx.x * 8 + k)] = base;
                    base += loc[k];
                }
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < KPL; ++j) {
                const bool act = s0 + 32 * j + lane < s1;
                const uint32_t d = (kr[j] >> shift) & 255u;
                const unsigned peers = warp_digit_peers(d, act);
                const int rank = __popc(peers & ((1u << lane) - 1u));
                const int base = act ? hist[d * kHistPitch + w] : 0;
                if (act) {
                    skm[base + rank] = kr[j];
                    svm[base + rank] = vr[j];
                }
                __syncwarp();
                if (act && rank == 0) hist[d * kHistPitch + w] = base + __popc(peers);
                __syncwarp();
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            code[i] = skm[i];
            idx[i] = svm[i];
        }
        __syncthreads();
    } else {
        uint32_t *kin = code, *vin = idx, *kout = code2, *vout = idx2;
        for (int pass = 0; pass < 4; ++pass) {
            const int shift = 8 * pass;
            for (int k = threadIdx.x; k < kHistInts; k += blockDim.x) hist[k] = 0;
            __syncthreads();
            for (int b = s0; b < s1; b += 32) {
                int i = b + lane;
                if (i < s1) atomicAdd(&hist[((kin[i] >> shift) & 255u) * kHistPitch + w], 1);
            }
            __syncthreads();
            // exclusive scan of hist in (digit, warp) order: 8192 entries, 8 per thread
            {
                int loc[8], sum = 0;
                for (int k = 0; k < 8; ++k) {
                    loc[k] = hist[hist_at(threadIdx.x * 8 + k)];
                    sum += loc[k];
                }
                int total;
                int base = block_exclusive_scan(sum, tmp, total);
                for (int k = 0; k < 8; ++k) {
                    hist[hist_at(threadIdx.x * 8 + k)] = base;
                    base += loc[k];
                }
            }
            __syncthreads();
            for (int b = s0; b < s1; b += 32) {
                int i = b + lane;
                bool act = i < s1;
                uint32_t key = act ? kin[i] : 0u, val = act ? vin[i] : 0u;
                const uint32_t d = (key >> shift) & 255u;
                const unsigned peers = warp_digit_peers(d, act);
                int rank = __popc(peers & ((1u << lane) - 1u));
                int base = act ? hist[d * kHistPitch + w] : 0;
                if (act) {
                    kout[base + rank] = key;
                    vout[base + rank] = val;
                }
                __syncwarp();
                if (act && rank == 0) hist[d * kHistPitch + w] = base + __popc(peers);
                __syncwarp();
            }
            __syncthreads();
            uint32_t* t1 = kin; kin = kout; kout = t1;
            uint32_t* t2 = vin; vin = vout; vout = t2;
        }
        // after 4 passes the sorted data is back in code/idx
    }
    // a mid-sized solute keeps its sorted codes in shared memory for the searches of the octree build
    const bool mid = !in_smem && n <= kCodeSmem;
    uint32_t* scm = reinterpret_cast<uint32_t*>(sh + kHistInts + 64);  // [kCodeSmem] (mid-sized solutes)
    const uint32_t* scode = in_smem ? sc : (mid ? scm : code);  // sorted codes for the searches below
    // small solutes keep the sorted high-part positions and (while they fit) the nodes in shared memory, so
    // the level-by-level phases below do not wait on global memory between levels
    float* spos = reinterpret_cast<float*>(sc + kSortSmem);  // [kSortSmem][3]
    Node* snodes = reinterpret_cast<Node*>(spos + 3 * kSortSmem);  // [kNodeSmem]
    // sorted high-part positions for the bounding boxes (the sorted tables themselves: k_gather_cells)
    if (in_smem)
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const float4 f = *reinterpret_cast<const float4*>(&a.srcf[(uint32_t)sk[i]].xh);
            spos[3 * i] = f.x;
            spos[3 * i + 1] = f.y;
            spos[3 * i + 2] = f.z;
        }

    // ---- octree, level by level: nodes [lvl_begin, lvl_end) at the current level, built in shared memory
    // while they fit in kNodeSmem, else (built again) in global memory
    __shared__ int s_nnodes, s_lvl_begin, s_lvl_end, s_overflow, s_lvl[kMaxLevel + 2], s_nlvl;
    Node* snodes_mid = reinterpret_cast<Node*>(scm + kCodeSmem);  // [kNodeSmemL] (mid-sized solutes)
    Node* store = in_smem ? snodes : (mid ? snodes_mid : nodes);
    int cap = in_smem ? min(kNodeSmem, a.max_nodes) : (mid ? min(kNodeSmemL, a.max_nodes) : a.max_nodes);
    for (;;) {
        if (threadIdx.x == 0) {
            store[0] = Node{0, n, -1, 0, 0, -1, 0, 0, {0, 0, 0}, {0, 0, 0}};
            s_nnodes = 1;
            s_lvl_begin = 0;
            s_lvl_end = 1;
            s_overflow = 0;
            s_lvl[0] = 0;
            s_lvl[1] = 1;
            s_nlvl = 1;
        }
        __syncthreads();
        for (int lvl = 0; lvl < kMaxLevel; ++lvl) {
            const int lb = s_lvl_begin, le = s_lvl_end;
            // after an overflow the slots past the last written node hold no nodes: stop (uniform: shared flag
            // read after a barrier)
            if (lb >= le || s_overflow) break;
            // eight lanes per node: lane ch finds where child ch starts (a binary search over the node's range,
            // the eight searches run side by side); children are numbered in digit order as before
            for (int base = lb; base < le; base += blockDim.x / 8) {
                const int nid = base + (threadIdx.x >> 3), ch = threadIdx.x & 7, g0 = lane & ~7;
                Node nd{0, 0, -1, 0, 0, -1, 0, 0, {0, 0, 0}, {0, 0, 0}};
                bool split = false;
                int pos = 0;
                if (nid < le) {
                    nd = store[nid];
                    // a range outside [0, n) would index past the codes: never split it (cannot happen for a node
                    // this loop wrote; the check keeps the searches in bounds regardless)
                    split = nd.begin >= 0 && nd.end <= n && (nd.end - nd.begin) > a.leaf;
                    if (split) {
                        const int sh3 = 3 * (kMortonBits - 1 - lvl);
                        int lo = nd.begin, hi = nd.end;  // first position whose child digit >= ch
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if ((int)((scode[mid] >> sh3) & 7u) < ch) lo = mid + 1; else hi = mid;
                        }
                        pos = lo;
                    }
                }
                const int nxt = __shfl_sync(0xffffffffu, pos, (lane & 7) == 7 ? lane : lane + 1);
                const int cend = ch == 7 ? nd.end : nxt;
                const bool ne = split && cend > pos;  // child ch is not empty
                const unsigned grp = (__ballot_sync(0xffffffffu, ne) >> g0) & 0xffu;
                const int nch = __popc(grp), before = __popc(grp & ((1u << ch) - 1u));
                int total;
                const int off = __shfl_sync(0xffffffffu, block_exclusive_scan(ch == 0 ? nch : 0, tmp, total), g0);
                const int start = s_nnodes;
                if (split) {
                    if (start + off + nch > cap) {
                        s_overflow = 1;
                    } else {
                        if (ch == 0) {
                            store[nid].first_child = start + off;
                            store[nid].nchild = nch;
                        }
                        if (ne) store[start + off + before] = Node{pos, cend, -1, 0, lvl + 1, -1, 0, 0, {0, 0, 0}, {0, 0, 0}};
                    }
                }
                __syncthreads();
                if (threadIdx.x == 0) s_nnodes = min(start + total, cap);
                __syncthreads();
                if (s_overflow) break;
            }
            if (threadIdx.x == 0) {
                s_lvl_begin = le;
                s_lvl_end = s_nnodes;
                if (s_nnodes > le) {
                    s_lvl[s_nlvl + 1] = s_nnodes;
                    ++s_nlvl;
                }
            }
            __syncthreads();
        }
        if (!(s_overflow && store != nodes)) break;
        __syncthreads();  // every thread has read s_overflow before it is reset
        store = nodes;
        cap = a.max_nodes;
    }
    // ---- proxy plan: nodes with more than P3 atoms get proxies; items of kChunk atoms
    const int nn = s_nnodes;
    if (s_overflow) {  // the tree is incomplete: the host grows the node capacity and builds again
        if (threadIdx.x == 0) {
            meta->nnodes = nn;
            meta->nprox = meta->nitems = meta->nleaves = 0;
            meta->overflow = meta->build_overflow = 1;
            prox_items[0] = 0;
        }
        return;
    }
    __shared__ int s_prox, s_items, s_leaves;
    if (threadIdx.x == 0) {
        s_prox = 0;
        s_items = 0;
        s_leaves = 0;
    }
    __syncthreads();
    const bool plan = a.src != nullptr;  // the source proxies are wanted (no target boxes): lay out their work
    for (int base = 0; base < nn; base += blockDim.x) {
        const int nid = base + threadIdx.x;
        int isp = 0, nit = 0, leaf = 0;
        if (nid < nn) {
            const Node nd = store[nid];
            int cnt = nd.end - nd.begin;
            isp = plan && cnt > a.P3;
            nit = isp ? (cnt + kChunk - 1) / kChunk : 0;
            leaf = nd.first_child < 0;
        }
        int tp = 0, ti = 0, tl, op = 0, oi = 0;
        if (plan) {
            op = block_exclusive_scan(isp, tmp, tp);
            oi = block_exclusive_scan(nit, tmp, ti);
        }
        block_exclusive_scan(leaf, tmp, tl);
        const int p0 = s_prox, i0 = s_items;
        if (nid < nn && isp) {
            int k = p0 + op;
            if (k >= a.max_prox || i0 + oi + nit > a.max_items) {
                s_overflow = 1;
                store[nid].prox = -1;
            } else {
                store[nid].prox = k;
                prox_nodes[k] = nid;
                prox_items[k] = i0 + oi;
                // item = (proxy set k, atom chunk start)
                for (int c = 0; c < nit; ++c) {
                    items[2 * (i0 + oi + c) + 0] = k;
                    items[2 * (i0 + oi + c) + 1] = store[nid].begin + c * kChunk;
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
        meta->build_overflow = s_overflow;
        prox_items[s_prox] = s_items;
    }
    __syncthreads();
    if (s_overflow) return;
    // ---- tight bounding boxes (grid units) of a small solute, reduced in FP32 over the high parts of the
    // float-float positions (within 1e-5 grid units of the exact box; the box only steers the acceptance test
    // and the proxy placement): every leaf from its atoms' positions in shared memory, one thread per leaf, then
    // bottom-up, level by level, each internal node as the union of its children, one warp per node.  Larger
    // solutes take their boxes from k_node_boxes, over the sorted positions that k_gather_cells lays out (a
    // gather of every atom's position through this one SM would wait on memory for longer than the whole build).
    if (in_smem) {
        for (int nid = threadIdx.x; nid < nn; nid += blockDim.x) {
            const Node nd = store[nid];
            if (nd.first_child >= 0) continue;
            float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (int i = nd.begin; i < nd.end; ++i)
                for (int d = 0; d < 3; ++d) {
                    lo[d] = fminf(lo[d], spos[3 * i + d]);
                    hi[d] = fmaxf(hi[d], spos[3 * i + d]);
                }
            for (int d = 0; d < 3; ++d) {
                store[nid].lo[d] = lo[d];
                store[nid].hi[d] = hi[d];
            }
        }
        __syncthreads();
        for (int lv = s_nlvl - 1; lv >= 0; --lv) {
            for (int nid = s_lvl[lv] + w; nid < s_lvl[lv + 1]; nid += NW) {
                const Node nd = store[nid];
                if (nd.first_child < 0) continue;
                float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
                if (lane < nd.nchild) {
                    const Node ch = store[nd.first_child + lane];
                    for (int d = 0; d < 3; ++d) {
                        lo[d] = ch.lo[d];
                        hi[d] = ch.hi[d];
                    }
                }
                for (int d = 0; d < 3; ++d)
                    for (int o = 16; o > 0; o >>= 1) {
                        lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
                        hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
                    }
                if (lane == 0)
                    for (int d = 0; d < 3; ++d) {
                        store[nid].lo[d] = lo[d];
                        store[nid].hi[d] = hi[d];
                    }
            }
            __syncthreads();
        }
    }
    // the nodes kept in shared memory go out word by word (consecutive threads, consecutive words)
    if (store != nodes) {
        static_assert(sizeof(Node) % sizeof(int) == 0, "nodes copy as words");
        constexpr int kW = sizeof(Node) / sizeof(int);
        const int* sw = reinterpret_cast<const int*>(store);
        int* gw = reinterpret_cast<int*>(nodes);
        for (int k = threadIdx.x; k < nn * kW; k += blockDim.x) gw[k] = sw[k];
    }
}

// Tight bounding boxes (grid units) of the nodes of a solute above kSortSmem atoms: one CTA per node over its
// atoms' sorted float-float positions (high parts, within 1e-5 grid units of the exact box), reduced in FP32;
// min and max are exact, so the boxes do not depend on the order of the reduction.  The root's CTA reads every
// atom once; the other nodes run beside it on the other SMs.
constexpr int kBoxThreads = 512;
__global__ void __launch_bounds__(kBoxThreads) k_node_boxes(const TreeMeta* __restrict__ meta, Node* nodes,
                                                            const SrcF* __restrict__ ssrcf) {
    __shared__ float red[kBoxThreads / 32][6];
    if (meta->build_overflow) return;
    const int nn = meta->nnodes;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int nid = blockIdx.x; nid < nn; nid += gridDim.x) {
        const int b = nodes[nid].begin, e = nodes[nid].end;
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll 4
        for (int i = b + threadIdx.x; i < e; i += kBoxThreads) {
            const float4 f = __ldg(reinterpret_cast<const float4*>(&ssrcf[i].xh));
            lo[0] = fminf(lo[0], f.x);
            lo[1] = fminf(lo[1], f.y);
            lo[2] = fminf(lo[2], f.z);
            hi[0] = fmaxf(hi[0], f.x);
            hi[1] = fmaxf(hi[1], f.y);
            hi[2] = fmaxf(hi[2], f.z);
        }
        for (int d = 0; d < 3; ++d)
            for (int o = 16; o > 0; o >>= 1) {
                lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
                hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
            }
        if (lane == 0)
            for (int d = 0; d < 3; ++d) {
                red[w][d] = lo[d];
                red[w][3 + d] = hi[d];
            }
        __syncthreads();
        if (threadIdx.x < 6) {
            const int d = threadIdx.x;
            float v = red[0][d];
            for (int k = 1; k < kBoxThreads / 32; ++k) v = d < 3 ? fminf(v, red[k][d]) : fmaxf(v, red[k][d]);
            if (d < 3)
                nodes[nid].lo[d] = v;
            else
                nodes[nid].hi[d - 3] = v;
        }
        __syncthreads();
    }
}

// After the sort, in one launch: the sorted copies of the sources (FP64 grid units when the source proxies need
// them, float-float) and of the LJ tables, one thread per atom; and the near-field cell table, cell_start[m] =
// first sorted position whose level-lc Morton prefix is >= m, one thread per cell.
__global__ void k_gather_cells(BuildArgs a, const uint32_t* __restrict__ idx, const TreeMeta* meta,
                               const uint32_t* __restrict__ code, int* cell_start) {
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (int i = t0; i < a.n; i += stride) {
        const int j = (int)idx[i];
        if (a.src) a.src[i] = to_grid(a.geo[j], a.gd, a.ih);
        a.ssrcf[i] = a.srcf[j];
        for (int s = 0; s < a.smax; ++s) {
            const LJf l = a.ljf[(int64_t)j * a.smax + s];
            a.ljs[(int64_t)i * a.smax + s] = l;
            a.ljs2[(int64_t)i * a.smax + s] = LJf{l.A, l.A, -l.B, -l.B};
        }
    }
    const int lc = meta->lc;
    const int ncell = 1 << (3 * lc);
    const int sh = 3 * (kMortonBits - lc);
    for (int m = t0; m <= ncell; m += stride) {
        int lo = 0, hi = a.n;
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

// Chebyshev points of the second kind on node nd's box, all three axes, into
// tn[3][np] (threads of the CTA cooperate; caller synchronises).
__device__ __forceinline__ void cheb_table(const Node& nd, int deg, double* tn) {
    const int np = deg + 1;
    for (int k = threadIdx.x; k < 3 * np; k += blockDim.x) {
        const int d = k / np, m = k % np;
        double c, r;
        cheb_box(nd, d, c, r);
        tn[k] = c + r * cospi((double)m / deg);
    }
}

// Work item = (proxy set, chunk of kChunk atoms): partial modified charges
//   Qhat_k = sum_j q_j L_k1(y_j1) L_k2(y_j2) L_k3(y_j3)  (FP64)
// with the barycentric Lagrange basis at Chebyshev-2 points, weights (-1)^m
// halved at both ends (exact-node case handled).
__global__ void k_upward(int deg, const TreeMeta* meta, const Node* nodes, const int* prox_nodes, const int* items,
                         const Geo* __restrict__ src, double* part) {
    extern __shared__ double Ls[];  // [kChunk][3][deg+1], q[kChunk], tn[3][deg+1]
    const int np = deg + 1, P3 = np * np * np;
    double* qs = Ls + kChunk * 3 * np;
    double* tn = qs + kChunk;
    if (meta->build_overflow) return;
    const int nitems = meta->nitems;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int k = items[2 * it], b = items[2 * it + 1];
        const Node nd = nodes[prox_nodes[k]];
        const int cnt = min(kChunk, nd.end - b);
        __syncthreads();
        cheb_table(nd, deg, tn);
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
            int exact = -1;
            double den = 0.0;
            for (int m = 0; m < np; ++m) {
                const double diff = y - tn[d * np + m];
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
// Work = (proxy set, block of blockDim proxies), grid-stride.
__global__ void k_proxy_reduce(int deg, int n, const TreeMeta* meta, const Node* nodes, const int* prox_nodes,
                               const int* prox_items, const double* part, Geo* src, SrcF* srcf) {
    __shared__ double tn[3 * (kMaxDegree + 1)];
    const int np = deg + 1, P3 = np * np * np;
    if (meta->build_overflow) return;
    const int nprox = meta->nprox;
    const int nblk = (P3 + blockDim.x - 1) / blockDim.x;
    for (int wi = blockIdx.x; wi < nprox * nblk; wi += gridDim.x) {
        const int k = wi / nblk, pb = wi % nblk;
        const Node nd = nodes[prox_nodes[k]];
        __syncthreads();
        cheb_table(nd, deg, tn);
        __syncthreads();
        const int p = pb * blockDim.x + threadIdx.x;
        if (p >= P3) continue;
        const int i0 = prox_items[k], i1 = prox_items[k + 1];
        const int m1 = p % np, m2 = (p / np) % np, m3 = p / (np * np);
        double q = 0.0;
        for (int it = i0; it < i1; ++it) q += part[(int64_t)it * P3 + p];
        const Geo pp{tn[m1], tn[np + m2], tn[2 * np + m3], q};
        src[n + (int64_t)k * P3 + p] = pp;
        srcf[n + (int64_t)k * P3 + p] = make_srcf(pp.x, pp.y, pp.z, pp.q);
    }
}

// ------------------------------------------------------- target batches
// A target batch is NXB x NYB x NZB grid points.  The far kernel gives each
// thread PF consecutive x points and runs one CTA per batch; the near kernel
// works on sub-batches 8 points wide, a 4x4x4 block per warp and two points
// per lane, in persistent CTAs (the batched kernels: per work item).  The
// variants are the launch shapes the autotuner chooses from.
struct ShapeDesc {
    int nx, ny, nz, pf;
};
constexpr int kNumShapes = 3;
__host__ __device__ constexpr ShapeDesc shape_of(int v) {
    return v == 1 ? ShapeDesc{16, 8, 8, 8} : (v == 2 ? ShapeDesc{8, 8, 8, 8} : ShapeDesc{8, 8, 8, 4});
}

// Far-field buffer layout: blocks of 8x8x8 grid points (x fastest inside a block, the blocks x-fastest), the
// grid padded to whole blocks, so the points of an 8x8x8 target (sub-)batch are one contiguous 8 KB run.
__host__ __device__ inline int64_t far_index(int nx, int ny, int i, int j, int k) {
    const int bx = (nx + 7) >> 3, by = (ny + 7) >> 3;
    return ((((int64_t)(k >> 3) * by + (j >> 3)) * bx + (i >> 3)) << 9) + (((k & 7) << 6) | ((j & 7) << 3) | (i & 7));
}
__host__ __device__ inline int64_t far_points(int nx, int ny, int nz) {
    return (int64_t)((nx + 7) >> 3) * ((ny + 7) >> 3) * ((nz + 7) >> 3) * 512;
}

constexpr int kQCap = 2048;        // frontier capacity of the warp-cooperative traversal (nodes of one level)
constexpr int kListWarps = 2;      // warps (batches) per list-building CTA

struct ListArgs {
    int nbx, nby, nbz;        // batches per axis
    int bx, by, bz;           // batch dims (points)
    double theta;
    int n, P3;
    int cap;                  // capacity of the entry buffer
    // with target boxes: the traversal of a batch starts from the pass-down list of its level-0 box
    const int* dn_cnt;        // null: start from the root
    const int* dn_ent;
    int dn_cap;
    TBoxes tb;
    int use_pc;               // accept source proxies (off when the box level does the far field)
};

// Node index -> (is a node opened for this target?) helpers shared by the traversals.
__device__ __forceinline__ void node_sphere(const Node& nd, const float c[3], float& R2, float& rn) {
    float rn2 = 0.f;
    R2 = 0.f;
    for (int d = 0; d < 3; ++d) {
        const float cn = 0.5f * (nd.lo[d] + nd.hi[d]);
        R2 += (c[d] - cn) * (c[d] - cn);
        rn2 += 0.25f * (nd.hi[d] - nd.lo[d]) * (nd.hi[d] - nd.lo[d]);
    }
    rn = sqrtf(rn2);
}

// Loads a traversal's initial frontier: the root, or the pass-down list of the target's enclosing box.
// Returns its length (0 when the tree is unusable); sets ovf when it exceeds the frontier.
__device__ __forceinline__ int load_frontier(int* cur, const int* lst, int cnt, bool use_root, bool ok, int lane,
                                             bool& ovf) {
    if (!ok) return 0;
    if (use_root) {
        if (lane == 0) cur[0] = 0;
        __syncwarp();
        return 1;
    }
    if (cnt > kQCap) {
        ovf = true;
        cnt = kQCap;
    }
    for (int k = lane; k < cnt; k += 32) cur[k] = lst[k];
    __syncwarp();
    return cnt;
}

// Batch b: its point range, centre (half-integers, exact in FP32) and radius (the correctly rounded root of an
// exact integer); FP32 only, as in every list kernel.
__device__ __forceinline__ void batch_geom(const ListArgs& a, int b, float cb[3], float& rb, int lo[3], int hi[3]) {
    const int ib = b % a.nbx, jb = (b / a.nbx) % a.nby, kb = b / (a.nbx * a.nby);
    lo[0] = ib * a.bx;
    lo[1] = jb * a.by;
    lo[2] = kb * a.bz;
    hi[0] = lo[0] + a.bx - 1;
    hi[1] = lo[1] + a.by - 1;
    hi[2] = lo[2] + a.bz - 1;
    for (int d = 0; d < 3; ++d) cb[d] = 0.5f * (float)(lo[d] + hi[d]);
    rb = 0.5f * sqrtf((float)((a.bx - 1) * (a.bx - 1) + (a.by - 1) * (a.by - 1) + (a.bz - 1) * (a.bz - 1)));
}

// Far lists: one warp per target batch, level-synchronous traversal of the
// octree with the frontier in shared memory.  Entries are (start, count)
// ranges of the source array: atoms of a node evaluated directly, or a proxy
// set (n + k P3, P3) of an accepted node.  Order: by level, then by lane --
// deterministic.  Batch b owns entries [b cap, (b+1) cap); a longer list sets
// the overflow flag and records its length for the host to grow cap.
__global__ void __launch_bounds__(32 * kListWarps) k_far_lists(ListArgs a, const Node* __restrict__ nodes, int2* ent,
                                                              int* cnt, int* work, TreeMeta* meta) {
    __shared__ int qa[kListWarps][kQCap], qb[kListWarps][kQCap];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nb = a.nbx * a.nby * a.nbz;
    const bool tree_ok = !meta->build_overflow;
    const long long pts = (long long)a.bx * a.by * a.bz;
    const float th2 = (float)(a.theta * a.theta);
    for (int b = blockIdx.x * kListWarps + w; b < nb; b += gridDim.x * kListWarps) {
        float cbf[3], rbf;
        int lo[3], hi[3];
        batch_geom(a, b, cbf, rbf, lo, hi);
        int* cur = qa[w];
        int* nxt = qb[w];
        bool ovf = false;
        const int* dl = nullptr;
        int dc = 0;
        if (a.dn_cnt) {
            const int bx0 = lo[0] / kTB0, by0 = lo[1] / kTB0, bz0 = lo[2] / kTB0;
            const int box = tbox_index(a.tb, 0, bx0, by0, bz0);
            dl = a.dn_ent + (int64_t)box * a.dn_cap;
            dc = a.dn_cnt[box];
        }
        int ncur = load_frontier(cur, dl, dc, a.dn_cnt == nullptr, a.n > 0 && tree_ok, lane, ovf);
        int m = 0;
        int2* out = ent + (int64_t)b * a.cap;
        long long dp = 0, pp = 0;
        while (ncur > 0) {
            int nnext = 0;
            for (int c0 = 0; c0 < ncur; c0 += 32) {
                const int k = c0 + lane;
                int kind = 0;  // 0 none, 1 entry, 2 open
                int2 e = make_int2(0, 0);
                int nch = 0, fch = 0;
                if (k < ncur) {
                    const Node nd = nodes[cur[k]];
                    float R2, rn;
                    node_sphere(nd, cbf, R2, rn);
                    const float rs = rbf + rn;
                    const bool sep = rs * rs < th2 * R2;
                    const int cntn = nd.end - nd.begin;
                    if (sep && a.use_pc && nd.prox >= 0) {
                        kind = 1;
                        e = make_int2(a.n + nd.prox * a.P3, a.P3);
                        pp += a.P3;
                    } else if (nd.first_child < 0 || (sep && cntn <= a.P3)) {
                        kind = 1;
                        e = make_int2(nd.begin, cntn);
                        dp += cntn;
                    } else {
                        kind = 2;
                        nch = nd.nchild;
                        fch = nd.first_child;
                    }
                }
                const unsigned em = __ballot_sync(0xffffffffu, kind == 1);
                if (kind == 1) {
                    const int pos = m + __popc(em & ((1u << lane) - 1u));
                    if (pos < a.cap) out[pos] = e;
                }
                m += __popc(em);
                int x = nch;
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                const int tot = __shfl_sync(0xffffffffu, x, 31);
                const int at = nnext + x - nch;
                if (kind == 2) {
                    for (int ch = 0; ch < nch; ++ch) {
                        if (at + ch < kQCap) nxt[at + ch] = fch + ch;
                        else ovf = true;
                    }
                }
                nnext += tot;
            }
            __syncwarp();
            if (__any_sync(0xffffffffu, ovf) || nnext > kQCap) {
                // the frontier of this batch does not fit: a node or leaf-size setting beyond this build
                if (lane == 0) {
                    meta->overflow = 1;
                    meta->wide = 1;
                }
                break;
            }
            int* tq = cur;
            cur = nxt;
            nxt = tq;
            ncur = nnext;
            __syncwarp();
        }
        if (__any_sync(0xffffffffu, ovf) && lane == 0) {
            meta->overflow = 1;
            meta->wide = 1;
        }
        for (int o = 16; o > 0; o >>= 1) {
            dp += __shfl_xor_sync(0xffffffffu, dp, o);
            pp += __shfl_xor_sync(0xffffffffu, pp, o);
        }
        if (lane == 0) {
            work[b] = (int)min(dp + pp, (long long)INT_MAX);
            cnt[b] = min(m, a.cap);
            if (m > a.cap) {
                meta->overflow = 1;
                atomicMax(&meta->far_need, m);
            }
            atomicAdd(&meta->direct_pairs, (unsigned long long)(dp * pts));
            atomicAdd(&meta->proxy_pairs, (unsigned long long)(pp * pts));
        }
    }
}

// Target-box lists of level l: one warp per box, traversal from the parent's pass-down list (the root at the
// top level).  A node that meets the acceptance criterion (r_box + r_node)/R < theta of a box with proxies is
// summed at the box's proxies (its atom range goes to the box's accepted list); a node larger than the box
// is opened; anything else is passed down to the box's children (the pass-down list).  Entry order: by
// frontier round, then lane -- deterministic.  Lists longer than their slots set the overflow flag and
// record their length for the host to grow the slots.
struct TListArgs {
    TBoxes tb;
    int l;
    int n, P3;
    double theta;
    int cp_cap, dn_cap;
    int* cp_cnt;
    int2* cp_ent;   // [nbox][cp_cap] atom ranges (start, count)
    int* dn_cnt;
    int* dn_ent;    // [nbox][dn_cap] node indices
};

__global__ void __launch_bounds__(32 * kListWarps) k_tbox_lists(TListArgs a, const Node* __restrict__ nodes,
                                                               TreeMeta* meta) {
    __shared__ int qa[kListWarps][kQCap], qb[kListWarps][kQCap];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const TBoxes& tb = a.tb;
    const int l = a.l;
    const int nbl = tb.nbx[l] * tb.nby[l] * tb.nbz[l];
    const bool tree_ok = !meta->build_overflow;
    const float th2 = (float)(a.theta * a.theta);
    for (int bi = blockIdx.x * kListWarps + w; bi < nbl; bi += gridDim.x * kListWarps) {
        const int ib = bi % tb.nbx[l], jb = (bi / tb.nbx[l]) % tb.nby[l], kb = bi / (tb.nbx[l] * tb.nby[l]);
        const TBox T = tbox_at(tb, l, ib, jb, kb);
        const float tc[3] = {T.c[0], T.c[1], T.c[2]}, tr = T.r;
        const int box = tb.off[l] + bi;
        int* cur = qa[w];
        int* nxt = qb[w];
        bool ovf = false;
        const bool top = l == tb.L - 1;
        int pc = 0;
        const int* pl = nullptr;
        if (!top) {
            const int pbox = tbox_index(tb, l + 1, ib >> 1, jb >> 1, kb >> 1);
            pl = a.dn_ent + (int64_t)pbox * a.dn_cap;
            pc = a.dn_cnt[pbox];
        }
        int ncur = load_frontier(cur, pl, pc, top, a.n > 0 && tree_ok, lane, ovf);
        int mc = 0, md = 0;
        int2* cpo = a.cp_ent + (int64_t)box * a.cp_cap;
        int* dno = a.dn_ent + (int64_t)box * a.dn_cap;
        long long cpp = 0;
        while (ncur > 0 && !__any_sync(0xffffffffu, ovf)) {
            int nnext = 0;
            for (int c0 = 0; c0 < ncur; c0 += 32) {
                const int k = c0 + lane;
                int kind = 0;  // 0 none, 1 accepted, 2 open, 3 pass down
                int nch = 0, fch = 0, node = 0;
                int2 e = make_int2(0, 0);
                if (k < ncur) {
                    node = cur[k];
                    const Node nd = nodes[node];
                    float R2, rn;
                    node_sphere(nd, tc, R2, rn);
                    const float rs = tr + rn;
                    if (T.proxied && rs * rs < th2 * R2) {
                        kind = 1;
                        e = make_int2(nd.begin, nd.end - nd.begin);
                        cpp += (long long)a.P3 * (nd.end - nd.begin);
                    } else if (nd.first_child >= 0 && rn > tr) {
                        kind = 2;
                        nch = nd.nchild;
                        fch = nd.first_child;
                    } else {
                        kind = 3;
                    }
                }
                const unsigned ea = __ballot_sync(0xffffffffu, kind == 1);
                const unsigned ed = __ballot_sync(0xffffffffu, kind == 3);
                const unsigned below = (1u << lane) - 1u;
                if (kind == 1) {
                    const int pos = mc + __popc(ea & below);
                    if (pos < a.cp_cap) cpo[pos] = e;
                }
                if (kind == 3) {
                    const int pos = md + __popc(ed & below);
                    if (pos < a.dn_cap) dno[pos] = node;
                }
                mc += __popc(ea);
                md += __popc(ed);
                int x = nch;
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                const int tot = __shfl_sync(0xffffffffu, x, 31);
                const int at = nnext + x - nch;
                if (kind == 2) {
                    for (int ch = 0; ch < nch; ++ch) {
                        if (at + ch < kQCap) nxt[at + ch] = fch + ch;
                        else ovf = true;
                    }
                }
                nnext += tot;
            }
            __syncwarp();
            int* tq = cur;
            cur = nxt;
            nxt = tq;
            ncur = nnext;
            __syncwarp();
        }
        for (int o = 16; o > 0; o >>= 1) cpp += __shfl_xor_sync(0xffffffffu, cpp, o);
        const bool wide = __any_sync(0xffffffffu, ovf);
        if (lane == 0) {
            a.cp_cnt[box] = min(mc, a.cp_cap);
            a.dn_cnt[box] = min(md, a.dn_cap);
            if (wide) {
                meta->overflow = 1;
                meta->wide = 1;
            }
            if (mc > a.cp_cap) {
                meta->overflow = 1;
                atomicMax(&meta->cp_need, mc);
            }
            if (md > a.dn_cap) {
                meta->overflow = 1;
                atomicMax(&meta->dn_need, md);
            }
            if (mc > 0) {
                atomicAdd(&meta->cp_pairs, (unsigned long long)cpp);
                atomicAdd(&meta->tboxes, 1);
            }
        }
    }
}

// Near lists: one warp per target batch; lanes test the cells of the box
// grown by rnear (x fastest), keep those whose box lies within rnear of the
// batch box, and emit their atom ranges in cell order.
// Up to kNearSort entries of a near list are sorted by their first atom in shared memory and contiguous ranges
// merged: the cells of a batch's neighbourhood hold an atom or two each, and a tile built from one range per cell
// takes a bulk copy per atom, which starves the near kernel's consumers; neighbouring cells are mostly
// neighbours in the Morton order of the sorted atoms too, so merged ranges hold many cells.
constexpr int kNearSort = 512;

__global__ void __launch_bounds__(32 * kListWarps) k_near_lists(ListArgs a, const int* __restrict__ cell_start,
                                                               int2* ent, int* cnt, int* work, TreeMeta* meta) {
    __shared__ int2 sbuf[kListWarps][kNearSort];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nb = a.nbx * a.nby * a.nbz;
    const int lc = meta->lc, ncell = 1 << lc;
    const float side = (float)meta->cell_side, rnear = (float)meta->rnear;
    const float clo0[3] = {(float)meta->cube_lo[0], (float)meta->cube_lo[1], (float)meta->cube_lo[2]};
    // 0.01 grid units of slack: Morton codes are computed in FP32, so an atom may sit ~1e-5 outside its cell box
    const float rn = isfinite(rnear) ? rnear + 0.01f : 1e30f;
    const float rn2 = rn * rn;
    const bool tree_ok = !meta->build_overflow;
    const long long pts = (long long)a.bx * a.by * a.bz;
    for (int b = blockIdx.x * kListWarps + w; b < nb; b += gridDim.x * kListWarps) {
        float cb[3], rb;
        int lo[3], hi[3];
        batch_geom(a, b, cb, rb, lo, hi);
        int c0[3], c1[3];
        bool ok = a.n > 0 && tree_ok;
        for (int d = 0; d < 3; ++d) {
            c0[d] = (int)fmaxf(floorf((lo[d] - rn - clo0[d]) / side), 0.f);
            c1[d] = (int)fminf(floorf((hi[d] + rn - clo0[d]) / side), (float)(ncell - 1));
            ok = ok && c0[d] <= c1[d];
        }
        const int ex = ok ? c1[0] - c0[0] + 1 : 0, ey = ok ? c1[1] - c0[1] + 1 : 0, ez = ok ? c1[2] - c0[2] + 1 : 0;
        const int total = ex * ey * ez;
        int m = 0;
        long long cand = 0;
        int2* out = ent + (int64_t)b * a.cap;
        for (int k0 = 0; k0 < total; k0 += 32) {
            const int k = k0 + lane;
            int2 e = make_int2(0, 0);
            bool take = false;
            if (k < total) {
                const int cc[3] = {c0[0] + k % ex, c0[1] + (k / ex) % ey, c0[2] + k / (ex * ey)};
                float d2 = 0.f;
                for (int d = 0; d < 3; ++d) {
                    const float clo = clo0[d] + cc[d] * side, chi = clo + side;
                    const float gap = fmaxf(0.f, fmaxf(clo - hi[d], lo[d] - chi));
                    d2 += gap * gap;
                }
                if (d2 < rn2) {
                    const uint32_t mc = morton3((uint32_t)cc[0], (uint32_t)cc[1], (uint32_t)cc[2]);
                    const int s0 = cell_start[mc], s1 = cell_start[mc + 1];
                    if (s1 > s0) {
                        take = true;
                        e = make_int2(s0, s1 - s0);
                        cand += s1 - s0;
                    }
                }
            }
            const unsigned em = __ballot_sync(0xffffffffu, take);
            if (take) {
                const int pos = m + __popc(em & ((1u << lane) - 1u));
                if (pos < a.cap) out[pos] = e;
            }
            m += __popc(em);
        }
        for (int o = 16; o > 0; o >>= 1) cand += __shfl_xor_sync(0xffffffffu, cand, o);
        int mout = m;  // entries written
        if (m > 1 && m <= a.cap && m <= kNearSort) {
            // bitonic sort of the entries by first atom (padded to a power of two with empty ranges at the end)
            int P = 1;
            while (P < m) P <<= 1;
            int2* sb = sbuf[w];
            __syncwarp();
            for (int i = lane; i < P; i += 32) sb[i] = i < m ? out[i] : make_int2(INT_MAX, 0);
            __syncwarp();
            for (int k = 2; k <= P; k <<= 1)
                for (int j = k >> 1; j > 0; j >>= 1) {
                    for (int t = lane; t < P / 2; t += 32) {
                        const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1)), l = i + j;
                        const int2 x = sb[i], y = sb[l];
                        if ((x.x > y.x) == ((i & k) == 0)) {
                            sb[i] = y;
                            sb[l] = x;
                        }
                    }
                    __syncwarp();
                }
            // merge: an entry that starts where the previous one ends continues its range; each run's first entry
            // writes the start, its last entry the length
            int runs = 0;
            for (int i0 = 0; i0 < m; i0 += 32) {
                const int i = i0 + lane;
                const bool in = i < m;
                const int2 e = in ? sb[i] : make_int2(0, 0);
                const bool head = in && (i == 0 || sb[i - 1].x + sb[i - 1].y != e.x);
                const unsigned hm = __ballot_sync(0xffffffffu, head);
                const int r = runs + __popc(hm & ((2u << lane) - 1u)) - 1;  // run of entry i
                if (head) out[r].x = e.x;
                runs += __popc(hm);
                __syncwarp();
                const bool tail = in && (i == m - 1 || sb[i + 1].x != e.x + e.y);
                if (tail) out[r].y = e.x + e.y - out[r].x;
                __syncwarp();
            }
            mout = runs;
        }
        if (lane == 0) {
            work[b] = (int)min(cand, (long long)INT_MAX);
            cnt[b] = min(mout, a.cap);
            if (m > a.cap) {
                meta->overflow = 1;
                atomicMax(&meta->near_need, m);
            }
            atomicAdd(&meta->near_pairs, (unsigned long long)(cand * pts));
        }
    }
}

// Launch order of the batches (or target boxes), heaviest first: a counting sort of the items by the binary
// order of magnitude of their work (one CTA per list: CTA 0 orders work0 into order0, CTA 1 work1 into order1).
// The order changes nothing but which CTAs start first (each item is computed independently), so long items do
// not trail at the end of the launch.  The items may first be grouped by z slab for launches of their own
// (OrderGroups): the items of level l are [off[l], off[l+1]), item b of level l lies in layer (b - off[l]) /
// nbxy[l], and slab k holds the layers [bnd[l][k], bnd[l][k+1]) of every level; slab 0's items come first, and
// each slab's items fill one contiguous range of positions (the sizes of the groups are known on the host).
constexpr int kOrderBuckets = 33;
constexpr int kMaxSlabs = 16;
struct OrderGroups {
    int ns, nlev;
    int off[kMaxTL + 1], nbxy[kMaxTL];
    int bnd[kMaxTL][kMaxSlabs];  // first layer of each slab, per level, ascending
};
__host__ inline OrderGroups order_plain(int nb) {
    OrderGroups g{};
    g.ns = 1;
    g.nlev = 1;
    g.off[1] = nb;
    g.nbxy[0] = 1;
    return g;
}
// Batch layers in nslab slabs: slab k starts at layer ceil(k nbz / nslab).
__host__ inline int slab_start(int k, int nslab, int nbz) { return (int)(((int64_t)k * nbz + nslab - 1) / nslab); }
__global__ void __launch_bounds__(1024) k_order(int nb, const int* __restrict__ work0, int* order0,
                                                const int* __restrict__ work1, int* order1, OrderGroups og) {
    __shared__ int hist[kOrderBuckets * kMaxSlabs], start[kOrderBuckets * kMaxSlabs];
    const int* __restrict__ work = blockIdx.x == 0 ? work0 : work1;
    int* order = blockIdx.x == 0 ? order0 : order1;
    const int nkey = kOrderBuckets * og.ns;
    const int tid = threadIdx.x;
    for (int k = tid; k < nkey; k += blockDim.x) hist[k] = 0;
    __syncthreads();
    // key: group-major, then the work's order of magnitude from the largest (32) down to none (0)
    auto key = [&](int b) {
        const int w = work[b];
        const int mag = w <= 0 ? 0 : 32 - __clz(w);
        int l = 0;
        while (l + 1 < og.nlev && og.off[l + 1] <= b) ++l;
        const int layer = (b - og.off[l]) / og.nbxy[l];
        int sl = 0;
        for (int k = 1; k < og.ns; ++k)
            if (og.bnd[l][k] <= layer) sl = k;
        return sl * kOrderBuckets + (kOrderBuckets - 1 - mag);
    };
    for (int b = tid; b < nb; b += blockDim.x) atomicAdd(&hist[key(b)], 1);
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int k = 0; k < nkey; ++k) {
            start[k] = acc;
            acc += hist[k];
        }
    }
    __syncthreads();
    for (int b = tid; b < nb; b += blockDim.x) order[atomicAdd(&start[key(b)], 1)] = b;
}

__global__ void k_reset_meta(TreeMeta* meta) {
    meta->direct_pairs = meta->proxy_pairs = meta->near_pairs = meta->cp_pairs = 0ull;
    meta->near_tested = meta->lj_pairs = meta->sr_pairs = 0ull;
    meta->far_need = meta->near_need = meta->cp_need = meta->dn_need = 0;
    meta->tboxes = 0;
    meta->wide = 0;
    meta->build_overflow = 0;
    meta->overflow = 0;
    meta->nnodes = meta->nprox = meta->nitems = meta->nleaves = 0;
    meta->lc = 0;
    for (int d = 0; d < 3; ++d) {
        meta->bmin[d] = INT_MAX;
        meta->bmax[d] = INT_MIN;
    }
    meta->rc2max = 0;
    meta->cube_lo[0] = meta->cube_lo[1] = meta->cube_lo[2] = 0.0;
    meta->cube_side = meta->cell_side = 1.0;
    meta->rnear = 0.0;
}

// ---------------------------------------------------------------- eval
// Sources reach shared memory through bulk TMA copies issued by one producer
// lane into a kStages-deep ring of tiles guarded by full (copy landed) and empty
// (all warps done) mbarriers; every wait is bounded.
constexpr int kStages = 4;
constexpr int kNTab = 128;  // segments of the short-range kernel tables over [0, r_short]

struct EvalArgs {
    GridD g;
    Phys ph;
    int nbx, nby, nbz;
    int n;
    const SrcF* srcf;      // [sorted atoms | proxies], grid units, float-float
    const LJf* ljs;        // sorted LJ tables
    const LJf* ljs2;       // sorted LJ tables as {A, A, -B, -B}
    const int* far_cnt;    // far-list length per batch
    const int2* far_ent;   // [nb][far_cap]
    const int* near_cnt;
    const int2* near_ent;  // [nb][near_cap]
    int far_cap, near_cap;
    float4* far;           // per grid point (far_index layout): Phi1 (hi, lo), Phik (hi, lo), grid units
    int far_init;          // the far kernel starts from the box-level (interpolated) field already in `far`
    const float4* ntab;    // [2 kNTab] cubic pieces of erfc(x) and e^{-x^2}[erfcx(x-a) + erfcx(x+a)] in d
    float ntab_inv;        // kNTab / r_short (grid units)
    int uni_rc;            // every (atom, site) pair has the same LJ cut-off (global cut-off or none)
    const int* near_order; // work item -> batch of the per-solute near kernel (heaviest first)
    int* wq;               // [2] work queue of the persistent near kernel: items taken, CTAs done (0 between launches)
    int q0, q1;            // positions [q0, q1) of the near order (in sub-batches) that this near launch takes
    int f0;                // first position of the far order that this far launch takes (one CTA per batch)
    const int* far_order;  // the same for the far kernel
    const int* near_work;  // per batch: candidate atoms of the near list
    const int* far_work;   // per batch: atoms and proxies of the far list
    // epilogue constants per site (grid-unit sums -> physical fields), split into float pairs on the host:
    // u = cu Phi1 + LJ, c = cc (Phi1 - S_c), h = ch (2 e^{a^2} Phik - S_h)
    float cu_h[kMaxSites], cu_l[kMaxSites], cc[kMaxSites], ch[kMaxSites];
    float e2a_h, e2a_l;
    // FP32 constants of the kernels, rounded once on the host (no FP64 instruction in the kernels):
    float kap2;           // -kappa h log2(e): e^{-kappa d} = 2^(kap2 d_grid)
    float rs2, c0h, h0h;  // (r_short / h)^2; the d -> 0 limits of the two short-range kernels times h
    Outputs o;
    DevErr* err;
    TreeMeta* meta;
    long long wlim;
};

__device__ __forceinline__ void mbar_expect_tx_only(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int SM, bool WITH_LJ>
struct Ring {
    SrcF src[kStages][kT];
    LJf lj[WITH_LJ ? kStages : 1][WITH_LJ ? kT * SM : 1];
    uint64_t full[kStages], empty[kStages];
    int cnt[kStages];
    int abort;
    int inited;
    unsigned long long stat[3];  // per-CTA diagnostic pair counts (near kernel)
    int stat_warps;              // consumer warps that have added theirs
    int item[kStages];           // item stream: the work item of the tile in each slot (-1: end of stream)
    int last[kStages];           // item stream: nonzero on the last tile of its item
};

// Range-list producer state (the producer lane).
struct Cursor {
    int e, e_end, off;
    int left;              // sources still to deliver (a chunk of the list), INT_MAX: the whole list
    int produced;
    bool done;
    int last_phase[kStages];
};

template <int SM, bool LJ>
__device__ int fill_ranges(Cursor& c, const int2* __restrict__ ent, const SrcF* __restrict__ src,
                           const LJf* __restrict__ ljs, SrcF* dst, LJf* ldst, uint64_t* bar) {
    int filled = 0;
    while (filled < kT && c.e < c.e_end && c.left > 0) {
        const int2 en = ent[c.e];
        const int take = min(min(kT - filled, en.y - c.off), c.left);
        c.left -= take;
        const uint32_t b1 = take * sizeof(SrcF), b2 = LJ ? take * SM * sizeof(LJf) : 0;
        mbar_expect_tx_only(bar, b1 + b2);
        bulk_g2s(dst + filled, src + en.x + c.off, b1, bar);
        if (LJ) bulk_g2s(ldst + filled * SM, ljs + (int64_t)(en.x + c.off) * SM, b2, bar);
        filled += take;
        c.off += take;
        if (c.off >= en.y) {
            ++c.e;
            c.off = 0;
        }
    }
    return filled;
}

template <int SM, bool LJ, typename R>
__device__ __forceinline__ void produce(Cursor& c, R& r, int slot, const int2* ent, const SrcF* src, const LJf* ljs) {
    const int n = c.done ? 0 : fill_ranges<SM, LJ>(c, ent, src, ljs, r.src[slot], r.lj[LJ ? slot : 0], &r.full[slot]);
    if (n == 0) c.done = true;
    r.cnt[slot] = n;
    c.last_phase[slot] = c.produced / kStages;
    ++c.produced;
    mbar_arrive(&r.full[slot]);
}

// Ring setup for one work item (one thread), with the barriers of a previous
// item invalidated first.  Callers put a __syncthreads() on both sides.
template <typename R>
__device__ void ring_init(R& r, int nwarps) {
    for (int s = 0; s < kStages; ++s) {
        if (r.inited) {
            mbar_inval(&r.full[s]);
            mbar_inval(&r.empty[s]);
        }
        mbar_init(&r.full[s], 1);
        mbar_init(&r.empty[s], nwarps);
    }
    r.inited = 1;
    r.abort = 0;
    mbar_fence_init();
}

template <typename R>
__device__ void drain(R& r, const Cursor& c, long long wlim) {
    for (int s = 0; s < kStages; ++s)
        if (c.last_phase[s] >= 0) mbar_wait_bounded(&r.full[s], (uint32_t)(c.last_phase[s] & 1), wlim);
}

// Ring driver shared by the far, near and proxy-target bodies, warp-specialised: the warp after the NWARPS
// consumer warps produces (its lane 0 refills each slot as soon as every consumer warp has released it, so
// it runs up to kStages tiles ahead); each consumer warp, per landed tile, runs `stage(slot, cnt)` (reads the
// tile out of the ring), releases the slot and runs `consume(cnt)` on what it staged.  Every wait is bounded:
// a wait that runs out sets the abort flag and the device error word, and the producer waits (bounded) for
// its copies in flight before it leaves.
enum : int { kRingAbort = 0, kRingDone = 1, kRingProducer = 2 };

template <int SM, bool LJ, int NWARPS, typename R, typename FS, typename FC>
__device__ int run_ring(R& r, Cursor& cur, const int2* ent, const SrcF* src, const LJf* ljs, const EvalArgs& a,
                        FS&& stage, FC&& consume) {
    const int tid = threadIdx.x, lane = tid & 31;
    volatile int* abort_flag = &r.abort;
    if (tid >= NWARPS * 32) {
        if (tid == NWARPS * 32) {
            bool ok = true;
            for (int t = 0;; ++t) {
                const int slot = t % kStages;
                if (t >= kStages && !mbar_wait_bounded(&r.empty[slot], (uint32_t)((t / kStages - 1) & 1), a.wlim)) {
                    ok = false;
                    break;
                }
                if (*abort_flag) {
                    ok = false;
                    break;
                }
                produce<SM, LJ>(cur, r, slot, ent, src, ljs);
                if (cur.done) break;
            }
            if (!ok) {
                *abort_flag = 1;
                report_error(a.err, DEV_TIMEOUT, WHERE_TREE_EVAL);
                drain(r, cur, a.wlim);
            }
        }
        return kRingProducer;
    }
    for (int t = 0;; ++t) {
        const int slot = t % kStages;
        const uint32_t ph = (t / kStages) & 1;
        if (!mbar_wait_bounded(&r.full[slot], ph, a.wlim) || *abort_flag) {
            *abort_flag = 1;
            report_error(a.err, DEV_TIMEOUT, WHERE_TREE_EVAL);
            return kRingAbort;
        }
        const int cnt = r.cnt[slot];
        if (cnt == 0) return kRingDone;
        stage(slot, cnt);
        __syncwarp();
        if (lane == 0) mbar_arrive(&r.empty[slot]);
        consume(cnt);
    }
}

// Source list of one work item of an item stream.
struct ItemSrc {
    const int2* ent;  // range entries (first source, count)
    int e, e_end;     // the item's entries
    const SrcF* src;
    const LJf* ljs;
};

// Ring driver of a persistent CTA that works through a sequence of items (target batches): the producer lane
// fills the ring with the tiles of item after item without a pause (every item takes at least one tile, the
// last one flagged; an item without sources gets one empty tile), so the next item's sources load while the
// consumer warps finish the previous one.  next(n, item, src) gives the CTA's n-th item (false: none left);
// extra(n, item, bar) may add copies of its own to the barrier of the item's first tile (they land with it);
// each consumer warp calls begin(item) before the item's first tile, stage(slot, cnt) per tile (before the slot
// is released) and consume(cnt) after the release, and finish(item) after the item's last tile.  The ring
// barriers are initialised once per launch.  Waits are bounded as in run_ring.
template <int SM, bool LJ, int NWARPS, typename R, typename FN, typename FX, typename FB, typename FS, typename FC,
          typename FF>
__device__ int run_stream(R& r, long long wlim, DevErr* err, FN&& next, FX&& extra, FB&& begin, FS&& stage,
                          FC&& consume, FF&& finish) {
    const int tid = threadIdx.x, lane = tid & 31;
    volatile int* abort_flag = &r.abort;
    if (tid >= NWARPS * 32) {
        if (tid == NWARPS * 32) {
            Cursor c;
            c.produced = 0;
            for (int s = 0; s < kStages; ++s) c.last_phase[s] = -1;
            bool ok = true;
            for (int n = 0; ok; ++n) {
                int item = -1;
                ItemSrc is{nullptr, 0, 0, nullptr, nullptr};
                const bool have = next(n, item, is);
                c.e = have ? is.e : 0;
                c.e_end = have ? is.e_end : 0;
                c.off = 0;
                c.left = INT_MAX;
                for (bool more = true, first = true; more; first = false) {
                    const int t = c.produced, slot = t % kStages;
                    if (t >= kStages && !mbar_wait_bounded(&r.empty[slot], (uint32_t)((t / kStages - 1) & 1), wlim)) {
                        ok = false;
                        break;
                    }
                    if (*abort_flag) {
                        ok = false;
                        break;
                    }
                    if (have && first) extra(n, item, &r.full[slot]);
                    const int cnt = have ? fill_ranges<SM, LJ>(c, is.ent, is.src, is.ljs, r.src[slot],
                                                               r.lj[LJ ? slot : 0], &r.full[slot])
                                         : 0;
                    more = have && c.e < c.e_end;
                    r.cnt[slot] = cnt;
                    r.item[slot] = have ? item : -1;
                    r.last[slot] = more ? 0 : 1;
                    c.last_phase[slot] = t / kStages;
                    c.produced = t + 1;
                    mbar_arrive(&r.full[slot]);
                }
                if (!have) break;
            }
            if (!ok) {
                *abort_flag = 1;
                report_error(err, DEV_TIMEOUT, WHERE_TREE_EVAL);
                drain(r, c, wlim);
            }
        }
        return kRingProducer;
    }
    bool open = false;
    for (int t = 0;; ++t) {
        const int slot = t % kStages;
        const uint32_t ph = (t / kStages) & 1;
        if (!mbar_wait_bounded(&r.full[slot], ph, wlim) || *abort_flag) {
            *abort_flag = 1;
            report_error(err, DEV_TIMEOUT, WHERE_TREE_EVAL);
            return kRingAbort;
        }
        const int item = r.item[slot], cnt = r.cnt[slot], last = r.last[slot];
        if (item < 0) return kRingDone;
        if (!open) {
            begin(item);
            open = true;
        }
        if (cnt > 0) stage(slot, cnt);
        __syncwarp();
        if (lane == 0) mbar_arrive(&r.empty[slot]);
        if (cnt > 0) consume(cnt);
        if (last) {
            finish(item);
            open = false;
        }
    }
}

// ---- far field: Phi1 = sum q/d and Phik = sum q e^{-kappa d}/d over the batch's far list
template <int NXB, int NYB, int NZB, int PF>
struct FarShape {
    static constexpr int TX = NXB / PF, NT = TX * NYB * NZB, NW = NT / 32, NTP = NT + 32;  // + producer warp
};

// One tile re-staged per warp as source pairs: record l holds sources 2l and 2l+1, field by field, so that a
// 16-byte shared load yields two-wide operands (x_hi of both, x_lo of both, ...).  An odd count is padded with
// a zero charge 10^6 grid units away, whose terms are exactly zero.
struct PairRec {
    float4 x;  // xh0, xh1, xl0, xl1
    float4 y;  // yh0, yh1, yl0, yl1
    float4 z;  // zh0, zh1, zl0, zl1
    float4 q;  // q0, q1, 0, 0
};
constexpr int kPairs = kT / 2;
constexpr float kPadPos = 1.0e6f;

// Writes the pair records of one tile (lane l: sources 2l, 2l+1); returns whether any source of the tile sits
// on a lattice point (warp-uniform).
__device__ __forceinline__ bool stage_pairs(const SrcF* __restrict__ Sx, int cnt, PairRec* wp, int lane) {
    bool on = false;
    if (2 * lane < cnt) {
        const float4 a0 = *reinterpret_cast<const float4*>(&Sx[2 * lane].xh);
        const float4 a1 = *reinterpret_cast<const float4*>(&Sx[2 * lane].xl);
        float4 b0 = make_float4(kPadPos, kPadPos, kPadPos, 0.f), b1 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (2 * lane + 1 < cnt) {
            b0 = *reinterpret_cast<const float4*>(&Sx[2 * lane + 1].xh);
            b1 = *reinterpret_cast<const float4*>(&Sx[2 * lane + 1].xl);
        }
        PairRec& o = wp[lane];
        o.x = make_float4(a0.x, b0.x, a1.x, b1.x);
        o.y = make_float4(a0.y, b0.y, a1.y, b1.y);
        o.z = make_float4(a0.z, b0.z, a1.z, b1.z);
        o.q = make_float4(a0.w, b0.w, 0.f, 0.f);
        on = a1.w != 0.f || b1.w != 0.f;
    }
    return __any_sync(0xffffffffu, on);
}

// The pair loop of the far field: two sources per two-wide instruction, P points per thread along x.  Per pair
// and point the arithmetic is the scalar sequence dx = (x - x_hi) - x_lo, d2 = fma(dx, dx, dy^2 + dz^2),
// r = rsqrt(d2), qr = q r, Phi1 += qr, Phik = fma(qr, 2^(k (d2 r)), Phik).  ON: some source of the tile is on
// a lattice point, so the coincident pair (d2 = 0) is dropped here and left to the near field (d = 0 limit).
template <int P, bool DH, bool ON>
__device__ __forceinline__ void far_pairs(const PairRec* wp, int np, const f32x2 (&GX)[P], f32x2 FY, f32x2 FZ,
                                          f32x2 K2, f32x2 (&P1)[P], f32x2 (&PK)[P]) {
#pragma unroll 2
    for (int l = 0; l < np; ++l) {
        const ulonglong2 X = *reinterpret_cast<const ulonglong2*>(&wp[l].x);
        const ulonglong2 Y = *reinterpret_cast<const ulonglong2*>(&wp[l].y);
        const ulonglong2 Z = *reinterpret_cast<const ulonglong2*>(&wp[l].z);
        const f32x2 Q = *reinterpret_cast<const f32x2*>(&wp[l].q);
        const f32x2 DY = sub2(sub2(FY, Y.x), Y.y);
        const f32x2 DZ = sub2(sub2(FZ, Z.x), Z.y);
        const f32x2 DYZ = fma2(DY, DY, mul2(DZ, DZ));
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const f32x2 DX = sub2(sub2(GX[p], X.x), X.y);
            const f32x2 D2 = fma2(DX, DX, DYZ);
            const float2 d2 = up2(D2);
            float r0 = rsqrt_approx(d2.x), r1 = rsqrt_approx(d2.y);
            if (ON) {
                r0 = d2.x > 0.f ? r0 : 0.f;
                r1 = d2.y > 0.f ? r1 : 0.f;
            }
            const f32x2 RI = pk2(r0, r1);
            const f32x2 QR = mul2(Q, RI);
            P1[p] = add2(P1[p], QR);
            if (DH) {
                const float2 e = up2(mul2(K2, mul2(D2, RI)));
                PK[p] = fma2(QR, pk2(ex2_approx(e.x), ex2_approx(e.y)), PK[p]);
            }
        }
    }
}

// Points of a far-field thread in one target batch (PF consecutive points along x) and their float-pair sums.
template <int PF>
struct FarPts {
    int i0, j, k;
    f32x2 GX[PF], FY, FZ;
    float f1h[PF], f1l[PF], fkh[PF], fkl[PF];
    bool on;  // some source of the current tile sits on a lattice point
};

// Points of batch b; the sums start from the box-level field already in `far` when a.far_init.
template <int NXB, int NYB, int NZB, int PF>
__device__ __forceinline__ void far_begin(FarPts<PF>& q, const EvalArgs& a, int b) {
    using Sh = FarShape<NXB, NYB, NZB, PF>;
    const int tid = threadIdx.x;
    const int tx = tid % Sh::TX, ty = (tid / Sh::TX) % NYB, tz = tid / (Sh::TX * NYB);
    const int ib = b % a.nbx, jb = (b / a.nbx) % a.nby, kb = b / (a.nbx * a.nby);
    q.i0 = ib * NXB + tx * PF;
    q.j = jb * NYB + ty;
    q.k = kb * NZB + tz;
#pragma unroll
    for (int p = 0; p < PF; ++p)
        q.GX[p] = pk2((float)(q.i0 + p), (float)(q.i0 + p));
    q.FY = pk2((float)q.j, (float)q.j);
    q.FZ = pk2((float)q.k, (float)q.k);
#pragma unroll
    for (int p = 0; p < PF; ++p) q.f1h[p] = q.f1l[p] = q.fkh[p] = q.fkl[p] = 0.f;
    q.on = false;
    if (a.far_init && q.j < a.g.ny && q.k < a.g.nz) {
        const float4* src0 = a.far + far_index(a.g.nx, a.g.ny, q.i0, q.j, q.k) - q.i0;  // PF points in a block row
#pragma unroll
        for (int p = 0; p < PF; ++p)
            if (q.i0 + p < a.g.nx) {
                const float4 v = src0[q.i0 + p];
                q.f1h[p] = v.x;
                q.f1l[p] = v.y;
                q.fkh[p] = v.z;
                q.fkl[p] = v.w;
            }
    }
}

// The pair records of one tile (before the slot is released) ...
__device__ __forceinline__ void far_stage(bool& on, const SrcF* Sx, int cnt, PairRec* wp) {
    __syncwarp();  // the previous tile's records are no longer read
    on = stage_pairs(Sx, cnt, wp, threadIdx.x & 31);
}

// ... and their pairs with the thread's points, folded into its sums.
template <int PF, bool DH>
__device__ __forceinline__ void far_consume(FarPts<PF>& q, const PairRec* wp, int cnt, f32x2 K2) {
    f32x2 P1[PF], PK[PF];
#pragma unroll
    for (int p = 0; p < PF; ++p) P1[p] = PK[p] = 0ull;  // +0.0f in both halves
    const int np = (cnt + 1) >> 1;
    if (!q.on)
        far_pairs<PF, DH, false>(wp, np, q.GX, q.FY, q.FZ, K2, P1, PK);
    else
        far_pairs<PF, DH, true>(wp, np, q.GX, q.FY, q.FZ, K2, P1, PK);
#pragma unroll
    for (int p = 0; p < PF; ++p) {
        const float2 s1 = up2(P1[p]);
        ff_add(q.f1h[p], q.f1l[p], s1.x + s1.y);
        if (DH) {
            const float2 sk = up2(PK[p]);
            ff_add(q.fkh[p], q.fkl[p], sk.x + sk.y);
        }
    }
}

template <int PF>
__device__ __forceinline__ void far_finish(const FarPts<PF>& q, const EvalArgs& a) {
    const GridD& g = a.g;
    if (q.j >= g.ny || q.k >= g.nz || q.i0 >= g.nx) return;
    float4* dst = a.far + far_index(g.nx, g.ny, q.i0, q.j, q.k) - q.i0;  // PF points in a block row
#pragma unroll
    for (int p = 0; p < PF; ++p)
        if (q.i0 + p < g.nx) dst[q.i0 + p] = make_float4(q.f1h[p], q.f1l[p], q.fkh[p], q.fkl[p]);
}

__device__ __forceinline__ f32x2 far_k2(const EvalArgs& a) { return pk2(a.kap2, a.kap2); }

// One batch with its own ring setup: the body of the persistent batched kernel.
template <int NXB, int NYB, int NZB, int PF, bool DH>
__device__ void far_body(const EvalArgs& a, int b, Ring<1, false>& r, PairRec (*pairs)[kPairs]) {
    using Sh = FarShape<NXB, NYB, NZB, PF>;
    const int tid = threadIdx.x;
    const f32x2 K2 = far_k2(a);
    PairRec* wp = pairs[tid >> 5];
    FarPts<PF> q;
    if (tid < Sh::NT) far_begin<NXB, NYB, NZB, PF>(q, a, b);
    Cursor cur;
    __syncthreads();
    if (tid == Sh::NT) {
        cur.e = b * a.far_cap;
        cur.e_end = cur.e + a.far_cnt[b];
        cur.off = 0;
        cur.left = INT_MAX;
        cur.produced = 0;
        cur.done = false;
        for (int s = 0; s < kStages; ++s) cur.last_phase[s] = -1;
        ring_init(r, Sh::NW);
    }
    __syncthreads();
    const int rr = run_ring<1, false, Sh::NW>(
        r, cur, a.far_ent, a.srcf, nullptr, a, [&](int slot, int cnt) { far_stage(q.on, r.src[slot], cnt, wp); },
        [&](int cnt) { far_consume<PF, DH>(q, wp, cnt, K2); });
    if (rr != kRingDone) return;
    far_finish<PF>(q, a);
}

// ---- box-level far field: accepted clusters summed at the Chebyshev proxy targets of each target box,
// pushed down the box hierarchy and interpolated onto the grid points (cluster-particle form).
struct CPArgs {
    TBoxes tb;
    const int* cp_cnt;
    const int2* cp_ent;  // [nbox][cp_cap] accepted atom ranges
    int cp_cap;
    float2* tpot;        // [nbox][P3] (Phi1, Phik) at the proxies, index (kz (n+1) + ky)(n+1) + kx
    float2* tpart;       // [nbox][kCPChunks - 1][P3] sums of the list chunks after the first
    int* tnch;           // [nbox] chunks the box's list was split into
    int* tflag;          // [nbox] nonzero: the box's proxies hold a field (own or inherited)
    const int* order;    // launch order of the boxes, most accepted atoms first (null: index order from box0)
    int box0;            // first box of an index-order launch
};

// Source pairs relative to the box centre: x_s - c = (x_hi - c) + x_lo, one rounding; the proxies are
// well separated from every accepted source, so no exact-difference form is needed here.
struct RelRec {
    float4 xy;  // x0, x1, y0, y1
    float4 zq;  // z0, z1, q0, q1
};

__device__ __forceinline__ void stage_rel(const SrcF* __restrict__ Sx, int cnt, RelRec* wp, int lane, float cx,
                                          float cy, float cz, float sc) {
    if (2 * lane < cnt) {
        const float4 a0 = *reinterpret_cast<const float4*>(&Sx[2 * lane].xh);
        const float4 a1 = *reinterpret_cast<const float4*>(&Sx[2 * lane].xl);
        float4 b0 = make_float4(0.f, 0.f, 0.f, 0.f), b1 = make_float4(0.f, 0.f, 0.f, 0.f);
        float bx = kPadPos, by = kPadPos, bz = kPadPos;
        if (2 * lane + 1 < cnt) {
            b0 = *reinterpret_cast<const float4*>(&Sx[2 * lane + 1].xh);
            b1 = *reinterpret_cast<const float4*>(&Sx[2 * lane + 1].xl);
            bx = ((b0.x - cx) + b1.x) * sc;
            by = ((b0.y - cy) + b1.y) * sc;
            bz = ((b0.z - cz) + b1.z) * sc;
        }
        RelRec& o = wp[lane];
        o.xy = make_float4(((a0.x - cx) + a1.x) * sc, bx, ((a0.y - cy) + a1.y) * sc, by);
        o.zq = make_float4(((a0.z - cz) + a1.z) * sc, bz, a0.w, b0.w);
    }
}

template <int P, bool DH>
__device__ __forceinline__ void cp_pairs(const RelRec* wp, int l0, int np, int stride, const f32x2 (&GX)[P], f32x2 FY,
                                         f32x2 FZ, f32x2 (&P1)[P], f32x2 (&PK)[P]) {
    for (int l = l0; l < np; l += stride) {
        const ulonglong2 A = *reinterpret_cast<const ulonglong2*>(&wp[l].xy);
        const ulonglong2 B = *reinterpret_cast<const ulonglong2*>(&wp[l].zq);
        const f32x2 DY = sub2(FY, A.y);
        const f32x2 DZ = sub2(FZ, B.x);
        const f32x2 DYZ = fma2(DY, DY, mul2(DZ, DZ));
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const f32x2 DX = sub2(GX[p], A.x);
            const f32x2 D2 = fma2(DX, DX, DYZ);
            const float2 d2 = up2(D2);
            const f32x2 RI = pk2(rsqrt_approx(d2.x), rsqrt_approx(d2.y));
            const f32x2 QR = mul2(B.y, RI);
            P1[p] = add2(P1[p], QR);
            if (DH) {  // coordinates scaled by -kappa h log2(e): the exponent is -d' = -(d'^2 / d')
                const float2 e = up2(mul2(D2, RI));
                PK[p] = fma2(QR, pk2(ex2_approx(-e.x), ex2_approx(-e.y)), PK[p]);
            }
        }
    }
}

constexpr int kCPThreads = 256;
constexpr int kCPP = 3;          // proxies per thread (along x)
constexpr int kCPChunks = 8;     // CTAs a box's accepted list is split over at most
constexpr int kCPChunkMin = 256; // atoms per chunk at least
constexpr int kCPOrderBoxes = 1024;  // boxes from which the box-level launch runs heaviest first

// One CTA per (target box, list chunk, pass): the box's accepted atoms split into up to kCPChunks chunks of
// at least kCPChunkMin atoms; the (n+1)^2 proxy lines of the box split into chunks of kCPP nodes along x,
// kCPThreads chunks per pass.  Sources stream through the TMA ring.  Chunk 0 writes the box's proxy values,
// later chunks their partial sums (added in chunk order by k_cp_reduce).  At low degree a box has few proxy
// chunks (50 at degree 4): then G = kCPThreads / chunks groups of threads share them, group g taking the source
// pairs g, g + G, ..., and the groups' float-pair sums are added in group order at the end.
template <bool DH>
__global__ void __launch_bounds__(kCPThreads + 32) k_cp_eval(EvalArgs a, CPArgs c) {
    __shared__ Ring<1, false> r;
    __shared__ RelRec pairs[kCPThreads / 32][kPairs];
    __shared__ float4 gsum[kCPThreads][kCPP];  // the groups' sums (G > 1): f1h, f1l, fkh, fkl
    __shared__ int s_e, s_off, s_len, s_nch;
    constexpr int NW = kCPThreads / 32;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) r.inited = 0;
    if (a.meta->overflow) return;
    const int box = c.order ? c.order[blockIdx.x] : c.box0 + (int)blockIdx.x, chunk = blockIdx.y, pass = blockIdx.z;
    const TBox T = tbox_flat(c.tb, box);
    if (!T.proxied) return;
    const int deg = c.tb.deg, n1 = deg + 1, P3 = c.tb.P3;
    const int nxc = (n1 + kCPP - 1) / kCPP;
    const int ntask = n1 * n1 * nxc;
    const int cnt = c.cp_cnt[box];
    if (cnt == 0) {
        if (chunk == 0 && pass == 0) {
            float2* out = c.tpot + (int64_t)box * P3;
            for (int k = tid; k < P3; k += blockDim.x) out[k] = make_float2(0.f, 0.f);
            if (tid == 0) {
                c.tflag[box] = 0;
                c.tnch[box] = 1;
            }
        }
        return;
    }
    const int2* ent = c.cp_ent + (int64_t)box * c.cp_cap;
    if (tid == 0) {
        int tot = 0;
        for (int e = 0; e < cnt; ++e) tot += ent[e].y;
        const int nch = min(kCPChunks, max(1, tot / kCPChunkMin));
        s_nch = nch;
        if (chunk < nch) {
            const int a0 = (int)((long long)tot * chunk / nch), a1 = (int)((long long)tot * (chunk + 1) / nch);
            int e = 0, acc = 0;
            while (e < cnt && acc + ent[e].y <= a0) acc += ent[e++].y;
            s_e = e;
            s_off = a0 - acc;
            s_len = a1 - a0;
        }
    }
    __syncthreads();
    const int nch = s_nch;
    if (chunk >= nch || pass * kCPThreads >= ntask) return;
    if (chunk == 0 && pass == 0 && tid == 0) {
        c.tflag[box] = 1;
        c.tnch[box] = nch;
    }
    float2* out = chunk == 0 ? c.tpot + (int64_t)box * P3
                             : c.tpart + ((int64_t)box * (kCPChunks - 1) + chunk - 1) * P3;
    const int G = 2 * ntask <= kCPThreads ? kCPThreads / ntask : 1;  // thread groups sharing the proxy chunks
    const int grp = G > 1 && tid < G * ntask ? tid / ntask : 0;
    const int task = G > 1 ? tid % ntask : pass * kCPThreads + tid;
    const bool act = tid < kCPThreads && (G > 1 ? tid < G * ntask : task < ntask);
    const int tk = act ? task : 0;
    const int line = tk / nxc, xc = tk % nxc, ky = line % n1, kz = line / n1;
    const float hx = 0.5f * (T.ext[0] - 1), hy = 0.5f * (T.ext[1] - 1), hz = 0.5f * (T.ext[2] - 1);
    // With screening every coordinate is scaled by s = kappa h log2(e), so the screening exponent is the scaled
    // distance itself and both sums are multiplied by s at the end.  Below 1e-18 the exponent rounds to 0 either
    // way, so the floor changes no value; it keeps the scaled squared distances normal numbers.
    const float csc = DH ? fmaxf(-a.kap2, 1e-18f) : 1.f;
    f32x2 GX[kCPP];
#pragma unroll
    for (int p = 0; p < kCPP; ++p) {
        const int kx = min(xc * kCPP + p, deg);
        const float u = hx * c.tb.ck[kx] * csc;
        GX[p] = pk2(u, u);
    }
    const float uy = hy * c.tb.ck[ky] * csc, uz = hz * c.tb.ck[kz] * csc;
    const f32x2 FY = pk2(uy, uy), FZ = pk2(uz, uz);
    // box centre lo + (ext - 1) / 2: exact in FP32 (the same value as the FP64 centre)
    const float cx = (float)T.lo[0] + 0.5f * (float)(T.ext[0] - 1), cy = (float)T.lo[1] + 0.5f * (float)(T.ext[1] - 1),
                cz = (float)T.lo[2] + 0.5f * (float)(T.ext[2] - 1);
    RelRec* wp = pairs[tid >> 5];
    float f1h[kCPP], f1l[kCPP], fkh[kCPP], fkl[kCPP];
#pragma unroll
    for (int p = 0; p < kCPP; ++p) f1h[p] = f1l[p] = fkh[p] = fkl[p] = 0.f;
    Cursor cur;
    __syncthreads();
    if (tid == kCPThreads) {
        cur.e = box * c.cp_cap + s_e;
        cur.e_end = box * c.cp_cap + cnt;
        cur.off = s_off;
        cur.left = s_len;
        cur.produced = 0;
        cur.done = false;
        for (int st = 0; st < kStages; ++st) cur.last_phase[st] = -1;
        ring_init(r, NW);
    }
    __syncthreads();
    const int rr = run_ring<1, false, NW>(
        r, cur, c.cp_ent, a.srcf, nullptr, a,
        [&](int slot, int n) {
            __syncwarp();
            stage_rel(r.src[slot], n, wp, lane, cx, cy, cz, csc);
            __syncwarp();
        },
        [&](int n) {
            f32x2 P1[kCPP], PK[kCPP];
#pragma unroll
            for (int p = 0; p < kCPP; ++p) P1[p] = PK[p] = 0ull;
            // the unit-stride call is its own loop (a runtime stride costs the degree-8 loop 9%)
            if (G == 1) cp_pairs<kCPP, DH>(wp, 0, (n + 1) >> 1, 1, GX, FY, FZ, P1, PK);
            else cp_pairs<kCPP, DH>(wp, grp, (n + 1) >> 1, G, GX, FY, FZ, P1, PK);
#pragma unroll
            for (int p = 0; p < kCPP; ++p) {
                const float2 s1 = up2(P1[p]);
                ff_add(f1h[p], f1l[p], s1.x + s1.y);
                if (DH) {
                    const float2 sk = up2(PK[p]);
                    ff_add(fkh[p], fkl[p], sk.x + sk.y);
                }
            }
        });
    if (G > 1) {
        // every consumer warp leaves the ring (done or aborted, its waits are bounded) and meets the others here
        if (rr == kRingProducer) return;
        if (act && grp > 0)
#pragma unroll
            for (int p = 0; p < kCPP; ++p) gsum[tid][p] = make_float4(f1h[p], f1l[p], fkh[p], fkl[p]);
        asm volatile("bar.sync 1, %0;" ::"r"(kCPThreads) : "memory");
        if (rr != kRingDone || !act || grp > 0) return;
        for (int g = 1; g < G; ++g)
#pragma unroll
            for (int p = 0; p < kCPP; ++p) {
                const float4 o = gsum[g * ntask + tid][p];
                ff_add(f1h[p], f1l[p], o.x);
                f1l[p] += o.y;
                ff_add(fkh[p], fkl[p], o.z);
                fkl[p] += o.w;
            }
    } else if (rr != kRingDone || !act) {
        return;
    }
#pragma unroll
    for (int p = 0; p < kCPP; ++p) {
        const int kx = xc * kCPP + p;
        if (kx < n1) out[(kz * n1 + ky) * n1 + kx] = make_float2((f1h[p] + f1l[p]) * csc, (fkh[p] + fkl[p]) * csc);
    }
}

// Accepted atoms per box (0 for a box without proxies), one warp per box: the work that orders the box-level
// launch heaviest first, so the boxes with the longest chunks do not trail at the end of the launch.
__global__ void __launch_bounds__(256) k_cp_work(CPArgs c, const TreeMeta* meta, int* work) {
    const int box = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (box >= c.tb.nbox) return;
    int tot = 0;
    if (!meta->overflow && tbox_flat(c.tb, box).proxied) {
        const int cnt = c.cp_cnt[box];
        const int2* ent = c.cp_ent + (int64_t)box * c.cp_cap;
        for (int e = lane; e < cnt; e += 32) tot += ent[e].y;
        tot = __reduce_add_sync(0xffffffffu, tot);
    }
    if (lane == 0) work[box] = tot;
}

// Chunk partials added to the box's proxy values in chunk order (deterministic).
__global__ void __launch_bounds__(256) k_cp_reduce(CPArgs c, const TreeMeta* meta) {
    if (meta->overflow) return;
    const int box = c.order ? c.order[blockIdx.x] : c.box0 + (int)blockIdx.x;
    const TBox T = tbox_flat(c.tb, box);
    if (!T.proxied || c.cp_cnt[box] == 0) return;
    const int nch = c.tnch[box], P3 = c.tb.P3;
    if (nch <= 1) return;
    float2* dst = c.tpot + (int64_t)box * P3;
    const float2* part = c.tpart + (int64_t)box * (kCPChunks - 1) * P3;
    for (int k = threadIdx.x; k < P3; k += blockDim.x) {
        float2 v = dst[k];
        for (int ch = 1; ch < nch; ++ch) {
            const float2 w = part[(int64_t)(ch - 1) * P3 + k];
            v.x += w.x;
            v.y += w.y;
        }
        dst[k] = v;
    }
}

// Separable tensor-product interpolation: V holds N1^3 values on the source box's Chebyshev points (x
// fastest); W0/W1/W2 the 1D Lagrange weights [M][N1] of the target coordinates of each axis.  Each pass
// contracts one axis with a thread per output line: the thread loads the N1 inputs of its line once into
// registers and forms all M outputs of the line (the weights are the same for every thread of the pass, so
// their loads are broadcasts).  S1 = x-contracted [N1][N1][M] and S2 = y-contracted [N1][M][M] live in shared
// memory; the z pass hands each output value to emit(iz, iy, ix, v).  Every sum runs over k = 0 .. N1-1 in
// order.  Rows beyond a clipped box's extent are computed from zero weights; the caller skips them.
template <int N1, int M, typename FE>
__device__ void interp3(const float2* V, const float* W0, const float* W1, const float* W2, float2* S1, float2* S2,
                        FE&& emit) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int line = tid; line < N1 * N1; line += nt) {  // line = kz N1 + ky
        float2 v[N1];
#pragma unroll
        for (int k = 0; k < N1; ++k) v[k] = V[line * N1 + k];
#pragma unroll 4
        for (int ix = 0; ix < M; ++ix) {
            float ax = 0.f, ay = 0.f;
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                const float wv = W0[ix * N1 + k];
                ax = fmaf(wv, v[k].x, ax);
                ay = fmaf(wv, v[k].y, ay);
            }
            S1[line * M + ix] = make_float2(ax, ay);
        }
    }
    __syncthreads();
    for (int t = tid; t < N1 * M; t += nt) {  // t = kz M + ix
        const int ix = t % M, kz = t / M;
        float2 v[N1];
#pragma unroll
        for (int k = 0; k < N1; ++k) v[k] = S1[(kz * N1 + k) * M + ix];
#pragma unroll 4
        for (int iy = 0; iy < M; ++iy) {
            float ax = 0.f, ay = 0.f;
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                const float wv = W1[iy * N1 + k];
                ax = fmaf(wv, v[k].x, ax);
                ay = fmaf(wv, v[k].y, ay);
            }
            S2[(kz * M + iy) * M + ix] = make_float2(ax, ay);
        }
    }
    __syncthreads();
    for (int t = tid; t < M * M; t += nt) {  // t = iy M + ix
        const int ix = t % M, iy = t / M;
        float2 v[N1];
#pragma unroll
        for (int k = 0; k < N1; ++k) v[k] = S2[(k * M + iy) * M + ix];
#pragma unroll 4
        for (int iz = 0; iz < M; ++iz) {
            float ax = 0.f, ay = 0.f;
#pragma unroll
            for (int k = 0; k < N1; ++k) {
                const float wv = W2[iz * N1 + k];
                ax = fmaf(wv, v[k].x, ax);
                ay = fmaf(wv, v[k].y, ay);
            }
            emit(iz, iy, ix, make_float2(ax, ay));
        }
    }
    __syncthreads();
}

// Weight rows for axis d: row i is the Lagrange basis of box B's Chebyshev points along d evaluated at the
// offset t(i) from B's centre (grid units).
template <int N1, typename X>
__device__ void basis_rows(const TBoxes& tb, const TBox& B, int d, int m, int mpad, X t, float* W) {
    const float hw = 0.5f * (B.ext[d] - 1);
    for (int i = threadIdx.x; i < mpad; i += blockDim.x) {
        float L[N1];
        if (i < m) cheb_basis(N1 - 1, tb.ck, hw, t(i), L);
#pragma unroll
        for (int k = 0; k < N1; ++k) W[i * N1 + k] = i < m ? L[k] : 0.f;
    }
}

// Dynamic shared memory of k_l2l / k_tdown for degree n: V, S1, S2 and the weights.
__host__ __device__ constexpr size_t interp_smem(int n1, int m) {
    return sizeof(float2) * ((size_t)n1 * n1 * n1 + (size_t)n1 * n1 * m + (size_t)n1 * m * m) +
           sizeof(float) * 3 * (size_t)m * n1;
}

// Downward pass, level l + 1 -> l: a box with proxies adds its parent's field interpolated at its own proxies.
template <int N1>
__global__ void __launch_bounds__(256) k_l2l(CPArgs c, int l, int bi0, const TreeMeta* meta) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    constexpr int P3 = N1 * N1 * N1;
    if (meta->overflow) return;
    const TBoxes& tb = c.tb;
    const int bi = bi0 + (int)blockIdx.x;
    const int ib = bi % tb.nbx[l], jb = (bi / tb.nbx[l]) % tb.nby[l], kb = bi / (tb.nbx[l] * tb.nby[l]);
    const TBox T = tbox_at(tb, l, ib, jb, kb);
    if (!T.proxied) return;
    const TBox Pb = tbox_at(tb, l + 1, ib >> 1, jb >> 1, kb >> 1);
    const int box = tb.off[l] + bi, pbox = tbox_index(tb, l + 1, ib >> 1, jb >> 1, kb >> 1);
    if (!Pb.proxied || !c.tflag[pbox]) return;
    float2* V = reinterpret_cast<float2*>(sm_raw);
    float2* S1 = V + P3;
    float2* S2 = S1 + P3;
    float* W = reinterpret_cast<float*>(S2 + P3);
    const float2* src = c.tpot + (int64_t)pbox * P3;
    for (int k = threadIdx.x; k < P3; k += blockDim.x) V[k] = src[k];
    for (int d = 0; d < 3; ++d) {
        // child node i relative to the parent's centre: (c_child - c_parent) (exact: half-integers) + hw ck[i]
        const float off = T.c[d] - Pb.c[d], hd = 0.5f * (T.ext[d] - 1);
        basis_rows<N1>(tb, Pb, d, N1, N1, [&](int i) { return off + hd * tb.ck[i]; }, W + d * N1 * N1);
    }
    __syncthreads();
    float2* dst = c.tpot + (int64_t)box * P3;
    interp3<N1, N1>(V, W, W + N1 * N1, W + 2 * N1 * N1, S1, S2, [&](int iz, int iy, int ix, float2 o) {
        const int k = (iz * N1 + iy) * N1 + ix;
        const float2 v = dst[k];
        dst[k] = make_float2(v.x + o.x, v.y + o.y);
    });
    if (threadIdx.x == 0) c.tflag[box] = 1;
}

// Box field onto the grid: one CTA per level-0 box region; the lowest box with proxies that contains it
// (its field includes every ancestor's) is interpolated at the region's points and written to the far-field
// buffer as the starting value of the far kernel (zero where no box holds a field).
template <int N1>
__global__ void __launch_bounds__(256) k_tdown(CPArgs c, float4* far, int bi0, const TreeMeta* meta) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    constexpr int P3 = N1 * N1 * N1, M = kTB0;
    if (meta->overflow) return;
    const TBoxes& tb = c.tb;
    const int bi = bi0 + (int)blockIdx.x;
    const int ib = bi % tb.nbx[0], jb = (bi / tb.nbx[0]) % tb.nby[0], kb = bi / (tb.nbx[0] * tb.nby[0]);
    const TBox R = tbox_at(tb, 0, ib, jb, kb);
    int la = -1;
    TBox A = R;
    for (int l = 0; l < tb.L; ++l) {
        A = tbox_at(tb, l, ib >> l, jb >> l, kb >> l);
        if (A.proxied) {
            la = l;
            break;
        }
    }
    const int m0 = R.ext[0], m1 = R.ext[1], m2 = R.ext[2];
    const bool field = la >= 0 && c.tflag[tbox_index(tb, la, A.ib, A.jb, A.kb)];
    if (!field) {
        for (int t = threadIdx.x; t < M * M * M; t += blockDim.x) {
            const int ix = t % M, iy = (t / M) % M, iz = t / (M * M);
            if (ix < m0 && iy < m1 && iz < m2)
                far[far_index(tb.nx, tb.ny, R.lo[0] + ix, R.lo[1] + iy, R.lo[2] + iz)] =
                    make_float4(0.f, 0.f, 0.f, 0.f);
        }
        return;
    }
    float2* V = reinterpret_cast<float2*>(sm_raw);
    float2* S1 = V + P3;
    float2* S2 = S1 + N1 * N1 * M;
    float* W = reinterpret_cast<float*>(S2 + N1 * M * M);
    const float2* src = c.tpot + (int64_t)tbox_index(tb, la, A.ib, A.jb, A.kb) * P3;
    for (int k = threadIdx.x; k < P3; k += blockDim.x) V[k] = src[k];
    const int ms[3] = {m0, m1, m2};
    for (int d = 0; d < 3; ++d) {
        const float off = (float)R.lo[d] - A.c[d];  // grid point i of the region relative to A's centre (exact)
        basis_rows<N1>(tb, A, d, ms[d], M, [&](int i) { return off + (float)i; }, W + d * M * N1);
    }
    __syncthreads();
    interp3<N1, M>(V, W, W + M * N1, W + 2 * M * N1, S1, S2, [&](int iz, int iy, int ix, float2 o) {
        if (ix < m0 && iy < m1 && iz < m2)
            far[far_index(tb.nx, tb.ny, R.lo[0] + ix, R.lo[1] + iy, R.lo[2] + iz)] = make_float4(o.x, 0.f, o.y, 0.f);
    });
}

// The downward pass and the interpolation onto the grid, over the box layers [zr[l][0], zr[l][1]) of each level
// l (null: every layer): the levels from the second highest down, then the level-0 boxes' grid points.  Returns
// the number of launches.
template <int N1>
int launch_down(const TBoxes& tb, const CPArgs& c, float4* far, const TreeMeta* meta, cudaStream_t st,
                const int (*zr)[2]) {
    const size_t sl = interp_smem(N1, N1), sd = interp_smem(N1, kTB0);
    raise_dyn_smem(k_l2l<N1>, sl);
    raise_dyn_smem(k_tdown<N1>, sd);
    int n = 0;
    for (int l = tb.L - 1; l >= 0; --l) {
        const int nbxy = tb.nbx[l] * tb.nby[l], z0 = zr ? zr[l][0] : 0, z1 = zr ? zr[l][1] : tb.nbz[l];
        if (z1 <= z0) continue;
        if (l < tb.L - 1) {
            k_l2l<N1><<<(z1 - z0) * nbxy, 256, sl, st>>>(c, l, z0 * nbxy, meta);
            ++n;
        }
        if (l == 0) {
            k_tdown<N1><<<(z1 - z0) * nbxy, 256, sd, st>>>(c, far, z0 * nbxy, meta);
            ++n;
        }
    }
    return n;
}

int launch_down_deg(const TBoxes& tb, const CPArgs& c, float4* far, const TreeMeta* meta, cudaStream_t st,
                    const int (*zr)[2] = nullptr) {
    switch (tb.deg) {
        case 1: return launch_down<2>(tb, c, far, meta, st, zr);
        case 2: return launch_down<3>(tb, c, far, meta, st, zr);
        case 3: return launch_down<4>(tb, c, far, meta, st, zr);
        case 4: return launch_down<5>(tb, c, far, meta, st, zr);
        case 5: return launch_down<6>(tb, c, far, meta, st, zr);
        case 6: return launch_down<7>(tb, c, far, meta, st, zr);
        case 7: return launch_down<8>(tb, c, far, meta, st, zr);
        case 8: return launch_down<9>(tb, c, far, meta, st, zr);
        case 9: return launch_down<10>(tb, c, far, meta, st, zr);
        case 10: return launch_down<11>(tb, c, far, meta, st, zr);
        case 11: return launch_down<12>(tb, c, far, meta, st, zr);
        default: return launch_down<13>(tb, c, far, meta, st, zr);
    }
}

// ---- near field (LJ within cut-offs, erfc remainders within r_short) + epilogue
// A near CTA covers SX = min(NXB, 8) points along x of its batch (a batch wider than that takes NSUB CTAs, which
// read the same near list): 256 consumer threads keep the accumulators of a thread in registers at two CTAs
// per SM.
template <int NXB, int NYB, int NZB>
struct NearShape {
    static constexpr int P = 2, SX = NXB < 8 ? NXB : 8, NSUB = NXB / SX, TX = SX / P, NT = TX * NYB * NZB,
                         NW = NT / 32, NTP = NT + 32;  // + producer
    static_assert(NXB % SX == 0, "near sub-batches tile the batch along x");
    static_assert(NW <= 16, "the per-warp source lists of the near tile hold 16 warps");
};

// Segment index and offset of u in [0, kNTab] (up to rounding) for the cubic pieces, without conversion
// instructions: adding 1.5 2^23 leaves round(u - 1/2) (ties to even) in the low bits of the sum, and the sum
// minus 1.5 2^23 is that integer as a float.  A tie gives the lower segment at offset 1, its end point.
__device__ __forceinline__ float seg_split(float u, int& it) {
    const float sh = (u - 0.5f) + 12582912.0f;
    it = min(__float_as_int(sh) - 0x4B400000, kNTab - 1);
    return u - fminf(sh - 12582912.0f, (float)(kNTab - 1));
}

// One tile of near-field sources against the P points of a thread: LJ within the pair cut-offs (UNI: one
// cut-off for every pair, tested once per pair instead of once per site) and the short-range remainders of
// eq. (dcf-r) / eq. (tcf-r) within r_short from the cubic pieces in d.
// wlo/whi: bounding box of the warp's points; a source farther than the near radius from it (plus slack for
// the rounded source position) is skipped by the whole warp at once.
template <int P, int SM, bool DU, bool DH, bool UNI>
__device__ __forceinline__ void near_tile(const SrcF* __restrict__ Sx, const LJf* __restrict__ L, int cnt,
                                          const float (&gx)[P], float fy, float fz, float rn2, float rs2, float rcu2,
                                          float tinv, const float4* tab, bool DC, float c0h, float h0h,
                                          const float (&wlo)[3], const float (&whi)[3], float rcull2,
                                          float (&sch)[P], float (&scl)[P], float (&shh)[P], float (&shl)[P],
                                          float (&plj)[P][SM], unsigned& hit,
                                          unsigned (&cnt3)[3]) {
    // Warp-parallel culling of the tile: lane l tests sources l and l + 32 against the warp's point box; the
    // ballots list the survivors, which every lane then visits in tile order.  A culled source has no point
    // of the warp within the near radius, so skipping it changes no sum.
    const int lane = threadIdx.x & 31;
    auto keep = [&](int i) {
        if (i >= cnt) return false;
        const float4 g = *reinterpret_cast<const float4*>(&Sx[i].xh);
        const float qx = fmaxf(0.f, fmaxf(wlo[0] - g.x, g.x - whi[0]));
        const float qy = fmaxf(0.f, fmaxf(wlo[1] - g.y, g.y - whi[1]));
        const float qz = fmaxf(0.f, fmaxf(wlo[2] - g.z, g.z - whi[2]));
        return fmaf(qx, qx, fmaf(qy, qy, qz * qz)) < rcull2;
    };
    const unsigned long long live =
        (unsigned long long)__ballot_sync(0xffffffffu, keep(lane)) |
        ((unsigned long long)__ballot_sync(0xffffffffu, keep(lane + 32)) << 32);
    for (unsigned long long mk = live; mk != 0ull; mk &= mk - 1ull) {
        const int s0 = __ffsll((long long)mk) - 1;
        const float4 g0 = *reinterpret_cast<const float4*>(&Sx[s0].xh);
        const float4 g1 = *reinterpret_cast<const float4*>(&Sx[s0].xl);
        cnt3[0] += P;
        const float dy = (fy - g0.y) - g1.y;
        const float dz = (fz - g0.z) - g1.z;
        const float dyz2 = fmaf(dy, dy, dz * dz);
        const LJf* Ls = L + s0 * SM;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const float dx = (gx[p] - g0.x) - g1.x;
            const float d2 = fmaf(dx, dx, dyz2);
            if (d2 >= rn2) continue;
            if (d2 < rs2) {
                if (d2 > 0.f) {
                    // erfc(x)/d and e^{-x^2}[erfcx(x-a) + erfcx(x+a)]/d from the cubic pieces in d
                    ++cnt3[2];
                    const float ri = rsqrt_approx(d2);
                    const float qr = g0.w * ri;
                    const float uu = d2 * ri * tinv;
                    int it;
                    const float tt = seg_split(uu, it);
                    if (DC) {
                        const float4 cc = tab[2 * it];
                        ff_add(sch[p], scl[p], qr * fmaf(fmaf(fmaf(cc.w, tt, cc.z), tt, cc.y), tt, cc.x));
                    }
                    if (DH) {
                        const float4 ch = tab[2 * it + 1];
                        ff_add(shh[p], shl[p], qr * fmaf(fmaf(fmaf(ch.w, tt, ch.z), tt, ch.y), tt, ch.x));
                    }
                } else {
                    hit |= 1u << p;
                    if (DC) ff_add(sch[p], scl[p], -(g0.w * c0h));
                    if (DH) ff_add(shh[p], shl[p], -(g0.w * h0h));
                }
            }
            if (DU) {
                if (UNI) {
                    if (d2 < rcu2) {
                        ++cnt3[1];
                        const float r2i = rcp_approx(d2);
                        const float r6 = r2i * r2i * r2i;
#pragma unroll
                        for (int s = 0; s < SM; ++s) {
                            const float2 ab = *reinterpret_cast<const float2*>(&Ls[s]);
                            plj[p][s] = fmaf(r6, fmaf(ab.x, r6, -ab.y), plj[p][s]);
                        }
                    }
                } else {
                    ++cnt3[1];
                    const float r2i = rcp_approx(d2);
                    const float r6 = r2i * r2i * r2i;
#pragma unroll
                    for (int s = 0; s < SM; ++s) {
                        const float4 l = *reinterpret_cast<const float4*>(&Ls[s]);
                        if (d2 < l.z) plj[p][s] = fmaf(r6, fmaf(l.x, r6, -l.y), plj[p][s]);
                    }
                }
            }
        }
    }
}

// The same tile for two points per thread and one cut-off for every pair, with the distances and the LJ terms
// of both points in two-wide instructions: L2 holds {A, A, -B, -B} per (atom, site), so one shared load gives
// both operands of a site.  Per pair the arithmetic is that of near_tile; a point outside the near radius
// gets zero terms from both cut-off tests, so no separate radius test is needed.
template <int SM, bool DU, bool DH>
__device__ __forceinline__ void near_tile_uni2(const SrcF* __restrict__ Sx, const LJf* __restrict__ L2, int cnt,
                                               const float (&gx)[2], float fy, float fz, float rn2, float rs2,
                                               float rcu2, float tinv, const float4* tab, bool DC, float c0h,
                                               float h0h, const float (&wlo)[3], const float (&whi)[3], float rcull2,
                                               float (&sch)[2], float (&scl)[2], float (&shh)[2], float (&shl)[2],
                                               float (&plj)[2][SM], unsigned& hit,
                                               unsigned (&cnt3)[3]) {
    // the tile's sources that survive the culling, listed per warp in tile order (kernels of up to 16 warps)
    __shared__ int wl_all[16][kT];
    const int lane = threadIdx.x & 31;
    int* wl = wl_all[threadIdx.x >> 5];
    auto keep = [&](int i) {
        if (i >= cnt) return false;
        const float4 g = *reinterpret_cast<const float4*>(&Sx[i].xh);
        const float qx = fmaxf(0.f, fmaxf(wlo[0] - g.x, g.x - whi[0]));
        const float qy = fmaxf(0.f, fmaxf(wlo[1] - g.y, g.y - whi[1]));
        const float qz = fmaxf(0.f, fmaxf(wlo[2] - g.z, g.z - whi[2]));
        return fmaf(qx, qx, fmaf(qy, qy, qz * qz)) < rcull2;
    };
    const bool k0 = keep(lane), k1 = keep(lane + 32);
    const unsigned b0 = __ballot_sync(0xffffffffu, k0), b1 = __ballot_sync(0xffffffffu, k1);
    const unsigned lt = (1u << lane) - 1u;
    const int n0 = __popc(b0), n = n0 + __popc(b1);
    __syncwarp();  // the previous tile's list is no longer read
    if (k0) wl[__popc(b0 & lt)] = lane;
    if (k1) wl[n0 + __popc(b1 & lt)] = lane + 32;
    __syncwarp();
    cnt3[0] += 2u * (unsigned)n;
    const f32x2 GX2 = pk2(gx[0], gx[1]);
    f32x2 ACC[SM];
#pragma unroll
    for (int s = 0; s < SM; ++s) ACC[s] = 0ull;
    auto dist = [&](int s0, float& q, float2& d2) {
        const float4 g0 = *reinterpret_cast<const float4*>(&Sx[s0].xh);
        const float4 g1 = *reinterpret_cast<const float4*>(&Sx[s0].xl);
        const float dy = (fy - g0.y) - g1.y;
        const float dz = (fz - g0.z) - g1.z;
        const float dyz2 = fmaf(dy, dy, dz * dz);
        const f32x2 DX = sub2(sub2(GX2, pk2(g0.x, g0.x)), pk2(g1.x, g1.x));
        d2 = up2(fma2(DX, DX, pk2(dyz2, dyz2)));
        q = g0.w;
    };
    auto lj = [&](int s0, float2 d2) {
        const bool in0 = d2.x < rcu2, in1 = d2.y < rcu2;
        cnt3[1] += (unsigned)in0 + (unsigned)in1;
        const float r0 = rcp_approx(d2.x), r1 = rcp_approx(d2.y);
        const f32x2 R2 = pk2(in0 ? r0 : 0.f, in1 ? r1 : 0.f);  // a point outside the cut-off adds +0
        const f32x2 R6 = mul2(mul2(R2, R2), R2);
        const LJf* Ls = L2 + s0 * SM;
#pragma unroll
        for (int s = 0; s < SM; ++s) {
            const ulonglong2 ab = *reinterpret_cast<const ulonglong2*>(&Ls[s]);  // (A, A), (-B, -B)
            ACC[s] = fma2(R6, fma2(ab.x, R6, ab.y), ACC[s]);
        }
    };
    auto sr = [&](float q, float2 d2) {
        if (fminf(d2.x, d2.y) < rs2) {
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const float dd = p ? d2.y : d2.x;
                if (dd >= rs2) continue;
                if (dd > 0.f) {
                    ++cnt3[2];
                    const float ri = rsqrt_approx(dd);
                    const float qr = q * ri;
                    const float uu = dd * ri * tinv;
                    int it;
                    const float tt = seg_split(uu, it);
                    if (DC) {
                        const float4 cc = tab[2 * it];
                        ff_add(sch[p], scl[p], qr * fmaf(fmaf(fmaf(cc.w, tt, cc.z), tt, cc.y), tt, cc.x));
                    }
                    if (DH) {
                        const float4 ch = tab[2 * it + 1];
                        ff_add(shh[p], shl[p], qr * fmaf(fmaf(fmaf(ch.w, tt, ch.z), tt, ch.y), tt, ch.x));
                    }
                } else {
                    hit |= 1u << p;
                    if (DC) ff_add(sch[p], scl[p], -(q * c0h));
                    if (DH) ff_add(shh[p], shl[p], -(q * h0h));
                }
            }
        }
    };
    // two sources per step: their loads, distances and LJ terms are independent (more in flight per warp);
    // the sums still take the sources in tile order
    int i = 0;
    for (; i + 2 <= n; i += 2) {
        const int sa = wl[i], sb = wl[i + 1];
        float qa, qb;
        float2 da, db;
        dist(sa, qa, da);
        dist(sb, qb, db);
        if (DU) {
            lj(sa, da);
            lj(sb, db);
        }
        sr(qa, da);
        sr(qb, db);
    }
    if (i < n) {
        const int sa = wl[i];
        float qa;
        float2 da;
        dist(sa, qa, da);
        if (DU) lj(sa, da);
        sr(qa, da);
    }
#pragma unroll
    for (int s = 0; s < SM; ++s) {
        const float2 v = up2(ACC[s]);
        plj[0][s] += v.x;
        plj[1][s] += v.y;
    }
}

// Constants of the near field of one solute (grid units).
struct NearConst {
    float rs2, c0h, h0h, rn2, rcu2, rcull2, tinv;
    bool DC, uni;
};

__device__ __forceinline__ NearConst near_const(const EvalArgs& a) {
    NearConst c;
    c.rs2 = a.rs2;
    c.c0h = a.c0h;
    c.h0h = a.h0h;
    c.DC = a.o.c != nullptr;
    const double rnear = a.meta->rnear;
    c.rn2 = isfinite(rnear) ? (float)(rnear * rnear) : INFINITY;
    c.rcu2 = __int_as_float(a.meta->rc2max);  // the cut-off of every pair when a.uni_rc
    // culling radius: near radius + 0.01 grid units of slack for the source position rounded to its high part
    const float rcull = isfinite(rnear) ? (float)rnear + 0.01f : INFINITY;
    c.rcull2 = rcull * rcull;
    c.tinv = a.ntab_inv;
    c.uni = a.uni_rc != 0;
    return c;
}

// The two points of a near-field thread in one target batch, its warp's point box and its accumulators
// (float pairs: the sums of the tiles are folded in error-free).
template <int SM>
struct NearPts {
    int i0, j, k;
    float gx[2], fy, fz, wlo[3], whi[3];
    float sch[2], scl[2], shh[2], shl[2], ljh[2][SM], ljl[2][SM];
    unsigned hit;
};

// Points of sub-batch `sub` of batch b: each warp owns a 4x4x4 block of the sub-batch (compact: small culling
// box, coherent distances), a lane two consecutive points along x of it.  Called by whole warps.
template <int NXB, int NYB, int NZB, int SM>
__device__ __forceinline__ void near_begin(NearPts<SM>& q, const EvalArgs& a, int b, int sub) {
    using Sh = NearShape<NXB, NYB, NZB>;
    static_assert(Sh::P == 2 && Sh::SX % 4 == 0 && NYB % 4 == 0 && NZB % 4 == 0,
                  "near warps tile the batch in 4x4x4");
    constexpr int WX = Sh::SX / 4, WY = NYB / 4;
    const int tid = threadIdx.x, wq = tid >> 5, ln = tid & 31;
    const int wx = wq % WX, wy = (wq / WX) % WY, wz = wq / (WX * WY);
    const int ib = b % a.nbx, jb = (b / a.nbx) % a.nby, kb = b / (a.nbx * a.nby);
    q.i0 = ib * NXB + sub * Sh::SX + 4 * wx + 2 * (ln & 1);
    q.j = jb * NYB + 4 * wy + ((ln >> 1) & 3);
    q.k = kb * NZB + 4 * wz + (ln >> 3);
    q.gx[0] = (float)q.i0;
    q.gx[1] = (float)(q.i0 + 1);
    q.fy = (float)q.j;
    q.fz = (float)q.k;
    const int lo3[3] = {q.i0, q.j, q.k}, hi3[3] = {q.i0 + 1, q.j, q.k};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        q.wlo[d] = (float)__reduce_min_sync(0xffffffffu, lo3[d]);
        q.whi[d] = (float)__reduce_max_sync(0xffffffffu, hi3[d]);
    }
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        q.sch[p] = q.scl[p] = q.shh[p] = q.shl[p] = 0.f;
#pragma unroll
        for (int s = 0; s < SM; ++s) q.ljh[p][s] = q.ljl[p][s] = 0.f;
    }
    q.hit = 0u;
}

// One tile of the near list against the thread's points, folded into its accumulators.
template <int SM, bool DU, bool DH>
__device__ __forceinline__ void near_stage(NearPts<SM>& q, const NearConst& c, const SrcF* Sx, const LJf* L, int cnt,
                                           const float4* tab, unsigned (&cnt3)[3]) {
    float plj[2][SM];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
#pragma unroll
        for (int s = 0; s < SM; ++s) plj[p][s] = 0.f;
    }
    // the short-range remainders go straight into the float-pair sums (they nearly cancel the far field next
    // to an atom, so an FP32 partial sum of a tile's terms would lose the digits that survive the cancellation)
    if (c.uni)
        near_tile_uni2<SM, DU, DH>(Sx, L, cnt, q.gx, q.fy, q.fz, c.rn2, c.rs2, c.rcu2, c.tinv, tab, c.DC, c.c0h,
                                   c.h0h, q.wlo, q.whi, c.rcull2, q.sch, q.scl, q.shh, q.shl, plj, q.hit, cnt3);
    else
        near_tile<2, SM, DU, DH, false>(Sx, L, cnt, q.gx, q.fy, q.fz, c.rn2, c.rs2, c.rcu2, c.tinv, tab, c.DC, c.c0h,
                                        c.h0h, q.wlo, q.whi, c.rcull2, q.sch, q.scl, q.shh, q.shl, plj, q.hit,
                                        cnt3);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        if (DU) {
#pragma unroll
            for (int s = 0; s < SM; ++s) ff_add(q.ljh[p][s], q.ljl[p][s], plj[p][s]);
        }
    }
}

// Epilogue of one batch: the far-field sums of the point plus the near sums, assembled into u, c and h.
// fr: the far-field records of the thread's two points (global memory or a shared-memory copy).
template <int SM, bool DU, bool DH>
__device__ __forceinline__ void near_finish(const NearPts<SM>& q, const NearConst& c, const EvalArgs& a,
                                            const float4* fr) {
    constexpr int P = 2;
    const GridD& g = a.g;
    const int i0 = q.i0;
    if (q.j >= g.ny || q.k >= g.nz || i0 >= g.nx) return;
    const int64_t plane = (int64_t)g.nx * g.ny * g.nz;
    const int64_t row = ((int64_t)q.k * g.ny + q.j) * g.nx;
    const bool vec_ok = (g.nx & 1) == 0;
    // Assembly in float pairs (error-free sums and products), one rounding to float per output, then the
    // float -> double conversion on the integer pipe: no FP64 arithmetic per grid point.
    float F1h[P], F1l[P], DC_[P], DH_[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const float4 f = (i0 + p < g.nx) ? fr[p] : make_float4(0.f, 0.f, 0.f, 0.f);
        F1h[p] = f.x;
        F1l[p] = f.y;
        float s, e;
        two_sum(f.x, -q.sch[p], s, e);  // Phi1 - S_c
        DC_[p] = s + (e + (f.y - q.scl[p]));
        const float ph_ = a.e2a_h * f.z;  // 2 e^{a^2} Phik - S_h
        const float pe = fmaf(a.e2a_h, f.z, -ph_) + (a.e2a_h * f.w + a.e2a_l * f.z);
        two_sum(ph_, -q.shh[p], s, e);
        DH_[p] = s + (e + (pe - q.shl[p]));
    }
    auto store = [&](double* base, const float (&v)[P]) {
        if (vec_ok && i0 + P <= g.nx) {
            __stcs(reinterpret_cast<double2*>(base + i0), make_double2(f2d_alu(v[0]), f2d_alu(v[1])));
        } else {
#pragma unroll
            for (int p = 0; p < P; ++p)
                if (i0 + p < g.nx) __stcs(base + i0 + p, f2d_alu(v[p]));
        }
    };
#pragma unroll
    for (int s = 0; s < SM; ++s) {
        if (s >= a.ph.S) break;
        float v[P];
        if (DU) {
            const float cuh = a.cu_h[s], cul = a.cu_l[s];
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float pc = cuh * F1h[p];
                const float pce = fmaf(cuh, F1h[p], -pc) + (cuh * F1l[p] + cul * F1h[p]);
                float t, e;
                two_sum(pc, q.ljh[p][s], t, e);
                v[p] = (q.hit >> p & 1u) ? INFINITY : t + (e + (pce + q.ljl[p][s]));
            }
            store(a.o.u + s * plane + row, v);
        }
        if (c.DC) {
#pragma unroll
            for (int p = 0; p < P; ++p) v[p] = a.cc[s] * DC_[p];
            store(a.o.c + s * plane + row, v);
        }
        if (DH) {
#pragma unroll
            for (int p = 0; p < P; ++p) v[p] = a.ch[s] * DH_[p];
            store(a.o.h + s * plane + row, v);
        }
    }
}

// Diagnostic pair counts, one global update per CTA: each consumer warp adds its counts in shared memory, the
// last warp to arrive publishes the CTA's totals (when nonzero).  r.stat / r.stat_warps start at zero.
template <int NW, typename R>
__device__ __forceinline__ void near_publish(R& r, TreeMeta* meta, const unsigned (&cnt3)[3]) {
    unsigned long long c0 = cnt3[0], c1 = cnt3[1], c2 = cnt3[2];
    for (int o = 16; o > 0; o >>= 1) {
        c0 += __shfl_xor_sync(0xffffffffu, c0, o);
        c1 += __shfl_xor_sync(0xffffffffu, c1, o);
        c2 += __shfl_xor_sync(0xffffffffu, c2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (c0) {
            atomicAdd(&r.stat[0], c0);
            atomicAdd(&r.stat[1], c1);
            atomicAdd(&r.stat[2], c2);
        }
        __threadfence_block();
        if (atomicAdd(&r.stat_warps, 1) == NW - 1) {
            __threadfence_block();
            const unsigned long long t0 = atomicAdd(&r.stat[0], 0ull), t1 = atomicAdd(&r.stat[1], 0ull),
                                     t2 = atomicAdd(&r.stat[2], 0ull);
            if (t0) {
                atomicAdd(&meta->near_tested, t0);
                atomicAdd(&meta->lj_pairs, t1);
                atomicAdd(&meta->sr_pairs, t2);
            }
        }
    }
}

// ---- per-solute kernels
// Work queue of a persistent kernel: wq[0] counts the items taken, wq[1] the CTAs whose producer takes no more.
// The last CTA to leave resets both, so every launch (and every replay of a captured one) starts from zero.
__device__ __forceinline__ void queue_leave(int* wq) {
    __threadfence();
    if (atomicAdd(&wq[1], 1) == (int)gridDim.x - 1) {
        atomicExch(&wq[0], 0);
        atomicExch(&wq[1], 0);
    }
}

// Far field of one solute, one CTA per target batch (heaviest first).  A persistent form like k_near32's measured
// slower here: the far items carry no epilogue to hide, and the queue adds latency before each batch's first tile.
template <int NXB, int NYB, int NZB, int PF, bool DH>
__global__ void __launch_bounds__(FarShape<NXB, NYB, NZB, PF>::NTP) k_far32(EvalArgs a) {
    __shared__ Ring<1, false> r;
    __shared__ PairRec pairs[FarShape<NXB, NYB, NZB, PF>::NW][kPairs];
    if (threadIdx.x == 0) r.inited = 0;
    if (a.meta->overflow) return;  // incomplete lists: the host grows them and runs again
    far_body<NXB, NYB, NZB, PF, DH>(a, a.far_order[a.f0 + blockIdx.x], r, pairs);
}

// Register cap (resident CTAs of consumer warps + producer warp) for up to 4 sites: 3 when only u or only the
// asymptotics are wanted, 2 for u, c and h together (more accumulators; a tighter cap spills).
template <int NXB, int NYB, int NZB, int SM, bool DU, bool DH>
struct NearOcc {
    static constexpr int v = SM <= 4 ? ((DU && DH) ? 2 : 3) : 1;
};

constexpr int kFarBuf = 5;  // far-field record buffers of the persistent near kernel (sub-batches in flight)

// Persistent near-field kernel of one solute: the producer of each CTA takes the next item (sub-batch) of the
// heaviest-first order from the work queue and streams the near lists of its items through one ring
// (run_stream), so the per-batch setup and epilogue overlap the loading of the next batch's sources.
template <int NXB, int NYB, int NZB, int SM, bool DU, bool DH>
__global__ void __launch_bounds__(NearShape<NXB, NYB, NZB>::NTP, (NearOcc<NXB, NYB, NZB, SM, DU, DH>::v))
    k_near32(const __grid_constant__ EvalArgs a) {
    using Sh = NearShape<NXB, NYB, NZB>;
    constexpr int NS = Sh::NSUB;
    __shared__ Ring<SM, true> r;
    __shared__ float4 tab[2 * kNTab];
    // far-field records of the last kFarBuf sub-batches (one 8x8x8 block of the far buffer each), copied by the
    // producer with each sub-batch's first tile.  It runs at most kStages tiles, so kStages sub-batches, ahead
    // of the slowest warp, whose epilogue reads sub-batch n - kFarBuf's buffer before it releases the tile that
    // lets the producer start sub-batch n.
    static_assert(Sh::SX == 8 && NYB == 8 && NZB == 8, "a sub-batch is one 8x8x8 block of the far buffer");
    static_assert(kStages <= kFarBuf - 1, "the far-field buffers cover the sub-batches the producer runs ahead");
    extern __shared__ __align__(16) float4 farbuf[];  // [kFarBuf][512], dynamic
    const int tid = threadIdx.x;
    if (a.meta->overflow) {  // incomplete lists: the host grows them and runs again
        if (tid == Sh::NT) queue_leave(a.wq);
        return;
    }
    for (int k = tid; k < 2 * kNTab; k += blockDim.x) tab[k] = a.ntab[k];
    if (tid == Sh::NT) {
        r.inited = 0;
        ring_init(r, Sh::NW);
        r.stat[0] = r.stat[1] = r.stat[2] = 0ull;
        r.stat_warps = 0;
    }
    __syncthreads();
    const NearConst c = near_const(a);
    const LJf* ljt = c.uni ? a.ljs2 : a.ljs;  // the two-wide tile reads {A, A, -B, -B}
    NearPts<SM> q;
    unsigned cnt3[3] = {0u, 0u, 0u};  // pairs tested / inside the LJ cut-off / inside r_short
    int seq = 0;                      // sub-batches finished by this warp (the producer counts them alike)
    const int rr = run_stream<SM, true, Sh::NW>(
        r, a.wlim, a.err,
        [&](int, int& item, ItemSrc& is) {
            const int qi = a.q0 + atomicAdd(&a.wq[0], 1);  // next position of the heaviest-first order
            if (qi >= a.q1) return false;
            const int b = a.near_order[qi / NS];
            item = b * NS + qi % NS;
            is = ItemSrc{a.near_ent, b * a.near_cap, b * a.near_cap + a.near_cnt[b], a.srcf, ljt};
            return true;
        },
        [&](int n, int item, uint64_t* bar) {
            const int b = item / NS, ib = b % a.nbx, jb = (b / a.nbx) % a.nby, kb = b / (a.nbx * a.nby);
            const int64_t blk = far_index(a.g.nx, a.g.ny, ib * NXB + (item % NS) * 8, jb * NYB, kb * NZB);
            mbar_expect_tx_only(bar, 512 * sizeof(float4));
            bulk_g2s(farbuf + (n % kFarBuf) * 512, a.far + blk, 512 * sizeof(float4), bar);
        },
        [&](int item) { near_begin<NXB, NYB, NZB, SM>(q, a, item / NS, item % NS); },
        [&](int slot, int cnt) { near_stage<SM, DU, DH>(q, c, r.src[slot], r.lj[slot], cnt, tab, cnt3); },
        [](int) {},
        [&](int) {
            near_finish<SM, DU, DH>(q, c, a, farbuf + (seq % kFarBuf) * 512 + ((q.k & 7) << 6 | (q.j & 7) << 3 | (q.i0 & 7)));
            ++seq;
        });
    if (rr == kRingDone) near_publish<Sh::NW>(r, a.meta, cnt3);
    if (tid == Sh::NT) queue_leave(a.wq);
}

// ---- persistent kernels over the (solute, batch) items of many solutes
struct BatchEval {
    const EvalArgs* args;   // [count]
    const int* item_off;    // [count + 1] prefix of batch counts
    int count, total;
    int* queue;             // work counter, zeroed before the launch
    const int* order;       // queue position -> global item (heaviest first over all solutes)
};

// Work of every (solute, batch) item in one array (far: near = 0, near: near = 1), for the global order.
__global__ void k_gather_work(const EvalArgs* args, const int* item_off, int count, int near, int* work) {
    const int sid = blockIdx.x;
    if (sid >= count) return;
    const int* w = near ? args[sid].near_work : args[sid].far_work;
    const int b0 = item_off[sid], nb = item_off[sid + 1] - b0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) work[b0 + b] = w[b];
}

__device__ __forceinline__ int find_solute(const BatchEval& be, int it) {
    int lo = 0, hi = be.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (be.item_off[mid] <= it) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int NXB, int NYB, int NZB, int PF, bool DH>
__global__ void __launch_bounds__(FarShape<NXB, NYB, NZB, PF>::NTP) k_far32_batched(BatchEval be) {
    __shared__ Ring<1, false> r;
    __shared__ PairRec pairs[FarShape<NXB, NYB, NZB, PF>::NW][kPairs];
    __shared__ int s_item;
    __shared__ EvalArgs sa;
    if (threadIdx.x == 0) r.inited = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int q = atomicAdd(be.queue, 1);
            s_item = q < be.total ? be.order[q] : be.total;
            if (s_item < be.total) sa = be.args[find_solute(be, s_item)];
        }
        __syncthreads();
        const int it = s_item;
        if (it >= be.total) break;
        if (sa.meta->overflow) continue;
        const int sid = find_solute(be, it);
        far_body<NXB, NYB, NZB, PF, DH>(sa, it - be.item_off[sid], r, pairs);
    }
}

// Pair counters of one finished item, added to its solute's totals (one lane per warp).
__device__ __forceinline__ void near_count(TreeMeta* meta, const unsigned (&cnt3)[3]) {
    unsigned long long c0 = cnt3[0], c1 = cnt3[1], c2 = cnt3[2];
    for (int o = 16; o > 0; o >>= 1) {
        c0 += __shfl_xor_sync(0xffffffffu, c0, o);
        c1 += __shfl_xor_sync(0xffffffffu, c1, o);
        c2 += __shfl_xor_sync(0xffffffffu, c2, o);
    }
    if ((threadIdx.x & 31) == 0 && c0) {
        atomicAdd(&meta->near_tested, c0);
        atomicAdd(&meta->lj_pairs, c1);
        atomicAdd(&meta->sr_pairs, c2);
    }
}

// Persistent near-field kernel over the (solute, batch) items of many solutes, in the global heaviest-first
// order: the same item stream as k_near32 (the producer streams item after item through one ring, with each
// sub-batch's far-field records), every item resolved to its solute's arguments.  The short-range tables are
// read through the L1 cache from the item's own solute (solutes may differ in them); items of a solute whose
// lists overflowed are skipped (the host grows the lists and runs again).
template <int NXB, int NYB, int NZB, int SM, bool DU, bool DH>
__global__ void __launch_bounds__(NearShape<NXB, NYB, NZB>::NTP, (NearOcc<NXB, NYB, NZB, SM, DU, DH>::v))
    k_near32_batched(BatchEval be) {
    using Sh = NearShape<NXB, NYB, NZB>;
    constexpr int NS = Sh::NSUB;
    __shared__ Ring<SM, true> r;
    static_assert(Sh::SX == 8 && NYB == 8 && NZB == 8, "a sub-batch is one 8x8x8 block of the far buffer");
    static_assert(kStages <= kFarBuf - 1, "the far-field buffers cover the sub-batches the producer runs ahead");
    extern __shared__ __align__(16) float4 farbuf[];  // [kFarBuf][512], dynamic
    const int tid = threadIdx.x;
    if (tid == Sh::NT) {
        r.inited = 0;
        ring_init(r, Sh::NW);
    }
    __syncthreads();
    const int total = be.total * NS;
    NearPts<SM> q;
    NearConst c{};
    const EvalArgs* ap = be.args;
    unsigned cnt3[3] = {0u, 0u, 0u};
    int seq = 0;
    run_stream<SM, true, Sh::NW>(
        r, be.args[0].wlim, be.args[0].err,
        [&](int, int& item, ItemSrc& is) {
            for (;;) {
                const int qi = atomicAdd(be.queue, 1);
                if (qi >= total) return false;
                const int gi = be.order[qi / NS], sid = find_solute(be, gi);
                const EvalArgs& A = be.args[sid];
                if (A.meta->overflow) continue;
                const int b = gi - be.item_off[sid];
                item = gi * NS + qi % NS;
                is = ItemSrc{A.near_ent, b * A.near_cap, b * A.near_cap + A.near_cnt[b], A.srcf,
                             A.uni_rc ? A.ljs2 : A.ljs};
                return true;
            }
        },
        [&](int n, int item, uint64_t* bar) {
            const int gi = item / NS, sid = find_solute(be, gi);
            const EvalArgs& A = be.args[sid];
            const int b = gi - be.item_off[sid], ib = b % A.nbx, jb = (b / A.nbx) % A.nby, kb = b / (A.nbx * A.nby);
            const int64_t blk = far_index(A.g.nx, A.g.ny, ib * NXB + (item % NS) * 8, jb * NYB, kb * NZB);
            mbar_expect_tx_only(bar, 512 * sizeof(float4));
            bulk_g2s(farbuf + (n % kFarBuf) * 512, A.far + blk, 512 * sizeof(float4), bar);
        },
        [&](int item) {
            const int gi = item / NS, sid = find_solute(be, gi);
            ap = be.args + sid;
            c = near_const(*ap);
            cnt3[0] = cnt3[1] = cnt3[2] = 0u;
            near_begin<NXB, NYB, NZB, SM>(q, *ap, gi - be.item_off[sid], item % NS);
        },
        [&](int slot, int cnt) { near_stage<SM, DU, DH>(q, c, r.src[slot], r.lj[slot], cnt, ap->ntab, cnt3); },
        [](int) {},
        [&](int) {
            near_finish<SM, DU, DH>(q, c, *ap,
                                    farbuf + (seq % kFarBuf) * 512 + ((q.k & 7) << 6 | (q.j & 7) << 3 | (q.i0 & 7)));
            near_count(ap->meta, cnt3);
            ++seq;
        });
}

// ---- dispatch over (shape, sites, outputs)
template <int V>
struct VShape {
    static constexpr ShapeDesc d = shape_of(V);
    static constexpr int NX = d.nx, NY = d.ny, NZ = d.nz, PF = d.pf;
    static constexpr int FT = FarShape<NX, NY, NZ, PF>::NTP, NTN = NearShape<NX, NY, NZ>::NTP;
};

int sm_count();

template <int V, int SM, bool DU, bool DH>
struct Kern {
    using S = VShape<V>;
    static void far(const EvalArgs& a, int nb, cudaStream_t st) {
        k_far32<S::NX, S::NY, S::NZ, S::PF, DH><<<nb, S::FT, 0, st>>>(a);
    }
    static void near(const EvalArgs& a, int nb, cudaStream_t st) {
        // persistent: at most the CTAs that are resident at once
        constexpr size_t dyn = sizeof(float4) * 512 * kFarBuf;  // far-field record buffers
        static const int resident = [] {
            raise_dyn_smem(k_near32<S::NX, S::NY, S::NZ, SM, DU, DH>, dyn);
            int b = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_near32<S::NX, S::NY, S::NZ, SM, DU, DH>, S::NTN, dyn);
            return std::max(1, b) * sm_count();
        }();
        const int items = nb * NearShape<S::NX, S::NY, S::NZ>::NSUB;
        k_near32<S::NX, S::NY, S::NZ, SM, DU, DH><<<std::max(1, std::min(items, resident)), S::NTN, dyn, st>>>(a);
    }
    static void far_b(const BatchEval& be, int grid, cudaStream_t st) {
        k_far32_batched<S::NX, S::NY, S::NZ, S::PF, DH><<<grid, S::FT, 0, st>>>(be);
    }
    static constexpr size_t kNearDyn = sizeof(float4) * 512 * kFarBuf;  // far-field record buffers
    static void near_b(const BatchEval& be, int grid, cudaStream_t st) {
        raise_dyn_smem(k_near32_batched<S::NX, S::NY, S::NZ, SM, DU, DH>, kNearDyn);
        k_near32_batched<S::NX, S::NY, S::NZ, SM, DU, DH><<<grid, S::NTN, kNearDyn, st>>>(be);
    }
    static int occ_far() {
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_far32_batched<S::NX, S::NY, S::NZ, S::PF, DH>, S::FT, 0);
        return b;
    }
    static int occ_near() {
        int b = 0;
        raise_dyn_smem(k_near32_batched<S::NX, S::NY, S::NZ, SM, DU, DH>, kNearDyn);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_near32_batched<S::NX, S::NY, S::NZ, SM, DU, DH>, S::NTN,
                                                      kNearDyn);
        return b;
    }
};

// op: 0 per-solute far+near, 1 batched far+near (grid from occupancy)
template <int V, int SM>
cudaError_t dispatch_v(int op, bool du, bool dh, const EvalArgs* a, int nb, const BatchEval* be, int sms,
                       cudaStream_t st) {
    auto go = [&](auto k) {
        using K = decltype(k);
        if (op == 0 || op == 2) K::far(*a, nb, st);
        if (op == 0 || op == 3) K::near(*a, nb, st);
        if (op == 1) {
            K::far_b(*be, sms * std::max(1, K::occ_far()), st);
            BatchEval b2 = *be;
            b2.queue = be->queue + 1;
            b2.order = be->order + be->total;  // the near order follows the far order
            K::near_b(b2, sms * std::max(1, K::occ_near()), st);
        }
    };
    if (du && dh) go(Kern<V, SM, true, true>{});
    else if (du) go(Kern<V, SM, true, false>{});
    else if (dh) go(Kern<V, SM, false, true>{});
    else go(Kern<V, SM, false, false>{});
    return cudaGetLastError();
}

template <int SM>
cudaError_t dispatch_sm(int v, int op, bool du, bool dh, const EvalArgs* a, int nb, const BatchEval* be, int sms,
                        cudaStream_t st) {
    switch (v) {
        case 1: return dispatch_v<1, SM>(op, du, dh, a, nb, be, sms, st);
        case 2: return dispatch_v<2, SM>(op, du, dh, a, nb, be, sms, st);
        default: return dispatch_v<0, SM>(op, du, dh, a, nb, be, sms, st);
    }
}

cudaError_t dispatch(int smax, int v, int op, bool du, bool dh, const EvalArgs* a, int nb, const BatchEval* be,
                     int sms, cudaStream_t st) {
    switch (smax) {
        case 2: return dispatch_sm<2>(v, op, du, dh, a, nb, be, sms, st);
        case 4: return dispatch_sm<4>(v, op, du, dh, a, nb, be, sms, st);
        default: return dispatch_sm<8>(v, op, du, dh, a, nb, be, sms, st);
    }
}

}  // namespace

// ------------------------------------------------------------- state
struct BatchCache;
struct SoluteGraph;
struct AdjTree;

struct TreeState {
    int64_t cap_n = 0;
    int cap_nodes = 0, cap_prox = 0, cap_items = 0, cap_nb = 0;
    int cap_far = 0, cap_near = 0;          // entries per batch
    int64_t cap_far_ent = 0, cap_near_ent = 0;  // entries allocated
    int deg = 0, smax = 0;
    uint32_t *code = nullptr, *idx = nullptr, *code2 = nullptr, *idx2 = nullptr;
    Node* nodes = nullptr;
    int* items = nullptr;
    int* prox_nodes = nullptr;
    double* part = nullptr;
    Geo* src = nullptr;    // sorted atoms + proxies, FP64 grid units (upward pass)
    SrcF* srcf = nullptr;  // the same as float-float (evaluation kernels)
    LJf* ljs = nullptr;
    LJf* ljs2 = nullptr;   // sorted LJ tables as {A, A, -B, -B}
    float4* far = nullptr; // far-field sums per grid point
    int64_t cap_far_pts = 0;
    int *far_cnt = nullptr, *near_cnt = nullptr, *prox_items = nullptr, *near_work = nullptr, *near_order = nullptr;
    int *far_work = nullptr, *far_order = nullptr;
    int* wq = nullptr;  // work-queue counters of the persistent near kernel
    int2 *far_ent = nullptr, *near_ent = nullptr;
    int* cell_start = nullptr;
    TreeMeta* meta = nullptr;
    TreeMeta* h_meta = nullptr;  // pinned copy, filled at the end of tree_eval
    int nb = 0, nbx = 0, nby = 0, nbz = 0;
    int variant = 0, leaf = 64;  // launch shape and leaf size in use
    int max_nodes = 0, max_prox = 0, max_items = 0;
    int launches = 0;
    bool prepared = false;
    std::string tuned_key;       // problem class the current (variant, leaf) was tuned for
    BatchCache* bc = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // box / far / near timing (debug_flags bit 1)
    bool timed = false;
    // z slabs of the near launch: with nslab > 1 the near kernel runs as one launch per slab, each followed by a
    // record of slab_ev[k], so copies of a finished slab's outputs can overlap the next slabs' evaluation
    int nslab = 1;
    cudaEvent_t slab_ev[kMaxSlabs] = {};
    bool slabs_live = false;  // the last enqueued evaluation recorded the slab events
    // the box level of the last cp_enqueue stopped after the coarser levels: each slab's launches start with
    // its level-0 boxes (box_slab_launches: the launches those added)
    bool box_split = false;
    int box_slab_launches = 0;
    int box_pos = 0;  // box order positions taken by the slabs so far
    // side branch of the preparation: the near lists beside the box-level lists, the far lists and the launch
    // orders beside the box-level evaluation; joined back before anything reads them (side_pending until then)
    cudaStream_t side = nullptr;
    cudaEvent_t side_fork[2] = {nullptr, nullptr}, side_join = nullptr;
    bool side_pending = false;
    // target boxes (cluster-particle far field)
    TBoxes tb{};
    int cap_cp = 0, cap_dn = 0, cap_tbox = 0;
    int64_t cap_cp_ent = 0, cap_dn_ent = 0, cap_tpot = 0;
    int *cp_cnt = nullptr, *dn_cnt = nullptr, *dn_ent = nullptr, *tflag = nullptr, *tnch = nullptr;
    int *cp_work = nullptr, *cp_order = nullptr;  // box-level launch order (accepted atoms per box, heaviest first)
    int2* cp_ent = nullptr;
    float2 *tpot = nullptr, *tpart = nullptr;
    SoluteGraph* sg = nullptr;  // captured solute step (tree_graph_step)
    AdjTree* adj = nullptr;     // reverse-mode far field over grid boxes (tree_adjoint_far)
    // short-range kernel tables
    float4* ntab = nullptr;
    double ntab_key[4] = {0.0, 0.0, 0.0, -1.0};
    float ntab_inv = 0.f;
};

namespace {
constexpr int kMaxCells = (1 << 21) + 1;  // 8^7 + 1

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

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// Host allocations for one solute (never inside a stream capture).
rism_status tree_reserve(TreeState* s, const DevTables& t, const GridD& g, const Phys& ph, const rism_options& o,
                         std::string& err) {
    cudaError_t e = cudaSuccess;
    const int n = (int)t.n;
    const int deg = o.degree, np = deg + 1, P3 = np * np * np;
    const ShapeDesc sd = shape_of(s->variant);
    s->nbx = (g.nx + sd.nx - 1) / sd.nx;
    s->nby = (g.ny + sd.ny - 1) / sd.ny;
    s->nbz = (g.nz + sd.nz - 1) / sd.nz;
    s->nb = s->nbx * s->nby * s->nbz;
    // Capacity bounds.  Internal nodes hold > leaf atoms and are disjoint per level, so there are at most
    // n/(leaf+1) per level over 10 levels, each with at most 8 children.  Proxy sets hold > P3 atoms, so at
    // most n/(P3+1) per level.  Upward items are chunks of kChunk atoms of proxied nodes.
    s->max_nodes = (int)(90LL * n / (s->leaf + 1)) + 16;
    s->max_prox = 10 * n / (P3 + 1) + 2;
    s->max_items = 10 * (n / kChunk + 1) + 2;
    if (!s->meta) {
        if ((e = cudaMalloc(&s->meta, sizeof(TreeMeta))) != cudaSuccess) return cuda_err(err, e, "tree meta");
        if ((e = cudaMallocHost(&s->h_meta, sizeof(TreeMeta))) != cudaSuccess) return cuda_err(err, e, "tree meta");
        if ((e = regrow(s->cell_start, (size_t)kMaxCells)) != cudaSuccess) return cuda_err(err, e, "cell table");
        std::memset(s->h_meta, 0, sizeof(TreeMeta));
    }
    if (n > s->cap_n || t.smax != s->smax || s->max_nodes > s->cap_nodes || deg != s->deg) {
        const size_t nn = n > 0 ? (size_t)n : 1;
        if ((e = regrow(s->code, nn)) || (e = regrow(s->idx, nn)) || (e = regrow(s->code2, nn)) ||
            (e = regrow(s->idx2, nn)) || (e = regrow(s->nodes, (size_t)s->max_nodes)) ||
            (e = regrow(s->items, 2 * (size_t)s->max_items)) || (e = regrow(s->prox_nodes, (size_t)s->max_prox)) ||
            (e = regrow(s->prox_items, (size_t)s->max_prox + 1)) ||
            (e = regrow(s->part, (size_t)s->max_items * P3)) || (e = regrow(s->src, nn + (size_t)s->max_prox * P3)) ||
            (e = regrow(s->srcf, nn + (size_t)s->max_prox * P3)) || (e = regrow(s->ljs, nn * t.smax)) ||
            (e = regrow(s->ljs2, nn * t.smax)))
            return cuda_err(err, e, "tree buffers");
        s->cap_n = (int64_t)nn;
        s->cap_nodes = s->max_nodes;
        s->cap_prox = s->max_prox;
        s->cap_items = s->max_items;
        s->smax = t.smax;
        s->deg = deg;
    }
    const int64_t M = far_points(g.nx, g.ny, g.nz);
    if (M > s->cap_far_pts) {
        if ((e = regrow(s->far, (size_t)M))) return cuda_err(err, e, "far-field buffer");
        s->cap_far_pts = M;
    }
    if (!s->wq) {
        if ((e = cudaMalloc(&s->wq, 2 * sizeof(int))) || (e = cudaMemset(s->wq, 0, 2 * sizeof(int))))
            return cuda_err(err, e, "work queue");
    }
    if (!s->side) {
        if ((e = cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking)) ||
            (e = cudaEventCreateWithFlags(&s->side_fork[0], cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&s->side_fork[1], cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&s->side_join, cudaEventDisableTiming)))
            return cuda_err(err, e, "side stream");
    }
    if (s->nb + 1 > s->cap_nb) {
        if ((e = regrow(s->far_cnt, (size_t)s->nb + 1)) || (e = regrow(s->near_cnt, (size_t)s->nb + 1)) ||
            (e = regrow(s->near_work, (size_t)s->nb + 1)) || (e = regrow(s->near_order, (size_t)s->nb + 1)) ||
            (e = regrow(s->far_work, (size_t)s->nb + 1)) || (e = regrow(s->far_order, (size_t)s->nb + 1)))
            return cuda_err(err, e, "list counts");
        s->cap_nb = s->nb + 1;
    }
    if (s->cap_far == 0) s->cap_far = 128;
    if (s->cap_near == 0) s->cap_near = 512;
    if ((int64_t)s->nb * s->cap_far > s->cap_far_ent) {
        if ((e = regrow(s->far_ent, (size_t)s->nb * s->cap_far))) return cuda_err(err, e, "far list");
        s->cap_far_ent = (int64_t)s->nb * s->cap_far;
    }
    if ((int64_t)s->nb * s->cap_near > s->cap_near_ent) {
        if ((e = regrow(s->near_ent, (size_t)s->nb * s->cap_near))) return cuda_err(err, e, "near list");
        s->cap_near_ent = (int64_t)s->nb * s->cap_near;
    }
    // target boxes: levels of aligned 16 << l cubes up to one that covers the grid
    TBoxes& tb = s->tb;
    tb = TBoxes{};
    tb.nx = g.nx;
    tb.ny = g.ny;
    tb.nz = g.nz;
    tb.deg = deg;
    tb.P3 = P3;
    tb.enabled = o.target_proxies != 0 && n > 0;
    tb.approx = o.approx;
    tb.kapg = (float)(ph.kappa * g.h);
    for (int k = 0; k <= kMaxDegree; ++k)  // cos(k pi / n) as sin(pi (n - 2k) / (2n)): exact 0 at k = n/2
        tb.ck[k] = k <= deg ? (float)std::sin(3.14159265358979323846 * (deg - 2 * k) / (2.0 * deg)) : 0.f;
    const int nmax = std::max(g.nx, std::max(g.ny, g.nz));
    tb.L = 1;
    while ((kTB0 << (tb.L - 1)) < nmax && tb.L < kMaxTL) ++tb.L;
    tb.nbox = 0;
    for (int l = 0; l < tb.L; ++l) {
        const int E = kTB0 << l;
        tb.nbx[l] = (g.nx + E - 1) / E;
        tb.nby[l] = (g.ny + E - 1) / E;
        tb.nbz[l] = (g.nz + E - 1) / E;
        tb.off[l] = tb.nbox;
        tb.nbox += tb.nbx[l] * tb.nby[l] * tb.nbz[l];
    }
    if (tb.enabled) {
        if (s->cap_cp == 0) s->cap_cp = 64;
        if (s->cap_dn == 0) s->cap_dn = 128;
        if (tb.nbox + 1 > s->cap_tbox) {
            if ((e = regrow(s->cp_cnt, (size_t)tb.nbox + 1)) || (e = regrow(s->dn_cnt, (size_t)tb.nbox + 1)) ||
                (e = regrow(s->tflag, (size_t)tb.nbox + 1)) || (e = regrow(s->tnch, (size_t)tb.nbox + 1)) ||
                (e = regrow(s->cp_work, (size_t)tb.nbox + 1)) || (e = regrow(s->cp_order, (size_t)tb.nbox + 1)))
                return cuda_err(err, e, "target boxes");
            s->cap_tbox = tb.nbox + 1;
        }
        if ((int64_t)tb.nbox * s->cap_cp > s->cap_cp_ent) {
            if ((e = regrow(s->cp_ent, (size_t)tb.nbox * s->cap_cp))) return cuda_err(err, e, "box lists");
            s->cap_cp_ent = (int64_t)tb.nbox * s->cap_cp;
        }
        if ((int64_t)tb.nbox * s->cap_dn > s->cap_dn_ent) {
            if ((e = regrow(s->dn_ent, (size_t)tb.nbox * s->cap_dn))) return cuda_err(err, e, "pass-down lists");
            s->cap_dn_ent = (int64_t)tb.nbox * s->cap_dn;
        }
        if ((int64_t)tb.nbox * P3 > s->cap_tpot) {
            if ((e = regrow(s->tpot, (size_t)tb.nbox * P3)) ||
                (e = regrow(s->tpart, (size_t)tb.nbox * (kCPChunks - 1) * P3)))
                return cuda_err(err, e, "proxy targets");
            s->cap_tpot = (int64_t)tb.nbox * P3;
        }
    }
    // Short-range kernels of the near field as cubic Hermite pieces in d (grid units) over [0, r_short]:
    // F_c(d) = erfc(x) and F_h(d) = e^{-x^2}[erfcx(x-a) + erfcx(x+a)] = e^{a^2-2ax} erfc(x-a) + e^{a^2+2ax} erfc(x+a),
    // x = d h / eta, a = kappa eta / 2, with their derivatives dF_c/dx = -2/sqrt(pi) e^{-x^2} and
    // dF_h/dx = -2a e^{a^2-2ax} erfc(x-a) + 2a e^{a^2+2ax} erfc(x+a) - 4/sqrt(pi) e^{-x^2}; built in FP64.
    const double key[4] = {ph.eta, g.h, ph.a, ph.rs};
    if (!s->ntab || std::memcmp(key, s->ntab_key, sizeof key) != 0) {
        if (!s->ntab && (e = cudaMalloc(&s->ntab, sizeof(float4) * 2 * kNTab)) != cudaSuccess)
            return cuda_err(err, e, "kernel table");
        const double sx = g.h / ph.eta, a = ph.a, rsg = ph.rs / g.h, D = rsg / kNTab;
        const double tsp = 2.0 / std::sqrt(3.14159265358979323846);
        std::vector<double> fc(kNTab + 1), gc(kNTab + 1), fh(kNTab + 1), gh(kNTab + 1);
        for (int k = 0; k <= kNTab; ++k) {
            const double x = k * D * sx, ex = std::exp(-x * x);
            const double em = std::exp(a * a - 2.0 * a * x), ep = std::exp(a * a + 2.0 * a * x);
            const double cm = std::erfc(x - a), cp = std::erfc(x + a);
            fc[k] = std::erfc(x);
            gc[k] = -tsp * ex * sx * D;  // derivative per segment length
            fh[k] = em * cm + ep * cp;
            gh[k] = (-2.0 * a * em * cm + 2.0 * a * ep * cp - 2.0 * tsp * ex) * sx * D;
        }
        std::vector<float4> tab(2 * kNTab);
        auto herm = [](double f0, double f1, double g0, double g1) {
            return make_float4((float)f0, (float)g0, (float)(3.0 * (f1 - f0) - 2.0 * g0 - g1),
                               (float)(2.0 * (f0 - f1) + g0 + g1));
        };
        for (int k = 0; k < kNTab; ++k) {
            tab[2 * k] = herm(fc[k], fc[k + 1], gc[k], gc[k + 1]);
            tab[2 * k + 1] = herm(fh[k], fh[k + 1], gh[k], gh[k + 1]);
        }
        if ((e = cudaMemcpy(s->ntab, tab.data(), sizeof(float4) * 2 * kNTab, cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_err(err, e, "kernel table");
        std::memcpy(s->ntab_key, key, sizeof key);
        s->ntab_inv = (float)(kNTab / rsg);
    }
    return RISM_OK;
}

// Grow list slots after an overflow (powers of two); false when nothing can grow.
bool grow_lists(TreeState* s, const TreeMeta& m) {
    if (m.wide || m.build_overflow) return false;
    auto pow2 = [](int v) {
        int p = 1;
        while (p < v) p <<= 1;
        return p;
    };
    bool grew = false;
    auto grow = [&](int need, int& cap) {
        if (need > cap && need < (1 << 20)) {
            cap = pow2(need);
            grew = true;
        }
    };
    grow(m.far_need, s->cap_far);
    grow(m.near_need, s->cap_near);
    grow(m.cp_need, s->cap_cp);
    grow(m.dn_need, s->cap_dn);
    return grew;
}

CPArgs make_cp(TreeState* s) {
    CPArgs c;
    c.tb = s->tb;
    c.cp_cnt = s->cp_cnt;
    c.cp_ent = s->cp_ent;
    c.cp_cap = s->cap_cp;
    c.tpot = s->tpot;
    c.tpart = s->tpart;
    c.tnch = s->tnch;
    c.tflag = s->tflag;
    // heaviest-first box order from kCPOrderBoxes boxes on: below that the two launches that make it cost more
    // than the shorter tail saves (measured: +11 us of 0.22 ms at 585 boxes, -23 us of 1.47 ms at 1,935)
    c.order = s->tb.nbox >= kCPOrderBoxes ? s->cp_order : nullptr;
    c.box0 = 0;
    return c;
}

// ---- Taylor moments of the target boxes (the paper's cluster-particle approximation, Sec. 2.3)
// A box with accepted atoms y_j takes the moments M_k = sum_j q_j (-1)^{|k|} a_k(c, y_j), |k| <= p, of the
// order-p Taylor expansion about its centre c (eq. (taylor_approximation)), with the coefficients a_k of
// Sec. 2.3.2 / Sec. 2.4 from their recurrences: 1/d (eq. (coulombrecurrence)) for Phi1 and e^{-kappa d}/d (eq.
// (screenedcoulombrecurrence) with its auxiliary e^{-kappa d}, eq. (screenedcoulombauxiliaryrecurrence), the
// auxiliary term taken with kappa/|k|) for Phik.  Coordinates are scaled by the box radius s: with r = (c - y)/s
// and t = (x - c)/s the field is (1/s) sum_k M_k t^k and kappa becomes kappa s, so every coefficient is O(1).
// The recurrence runs one warp per atom, the lanes over the coefficients of one order |k| at a time (graded
// order: |k|, then k1 descending, then k2 descending); the moments are stored in lexicographic order (k1, k2,
// k3 ascending) for the nested Horner evaluation of k_tay_down.
constexpr int kTayWarps = 8;

__host__ __device__ constexpr int tay_nc(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }
__device__ __forceinline__ int tay_graded(int k1, int k2, int k3) {
    const int n = k1 + k2 + k3, i = n - k1;
    return n * (n + 1) * (n + 2) / 6 + i * (i + 1) / 2 + (i - k2);
}
// position of (k1, k2, 0) in the lexicographic order of the multi-indices with |k| <= p
__device__ __forceinline__ int tay_lexoff(int p, int k1, int k2) {
    int o = 0;
    for (int a = 0; a < k1; ++a) o += (p - a + 1) * (p - a + 2) / 2;
    for (int b = 0; b < k2; ++b) o += p - k1 - b + 1;
    return o;
}

template <int P, bool DH>
__global__ void __launch_bounds__(kTayWarps * 32 + 32) k_tay_eval(EvalArgs a, CPArgs c) {
    constexpr int NC = tay_nc(P), J = (NC + 31) / 32;
    __shared__ Ring<1, false> r;
    __shared__ int s_e, s_off, s_len, s_nch;
    __shared__ char4 kk[NC];                        // multi-index of each graded position
    __shared__ short2 lk[NC][3];                    // graded positions of k - e_d and k - 2 e_d (-1: none)
    // dynamic: per warp the 1/d, e^{-kappa d}/d and e^{-kappa d} (auxiliary) coefficients of its current atom,
    // then per warp its moments for the fixed-order CTA sum (tay_eval_smem bytes)
    extern __shared__ __align__(16) unsigned char tay_raw[];
    float2* red = reinterpret_cast<float2*>(tay_raw);                         // [kTayWarps][NC]
    float* sa = reinterpret_cast<float*>(red + kTayWarps * NC);              // [kTayWarps][NC]
    float* sA = sa + kTayWarps * NC;                                          // [kTayWarps][NC]
    float* sB = sA + kTayWarps * NC;                                          // [kTayWarps][NC]
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) r.inited = 0;
    if (a.meta->overflow) return;
    const int box = blockIdx.x, chunk = blockIdx.y;
    const TBox T = tbox_flat(c.tb, box);
    if (!T.proxied) return;
    const int cnt = c.cp_cnt[box];
    if (cnt == 0) {
        if (chunk == 0) {
            float2* out = c.tpot + (int64_t)box * c.tb.P3;
            for (int k = tid; k < NC; k += blockDim.x) out[k] = make_float2(0.f, 0.f);
            if (tid == 0) {
                c.tflag[box] = 0;
                c.tnch[box] = 1;
            }
        }
        return;
    }
    const int2* ent = c.cp_ent + (int64_t)box * c.cp_cap;
    if (tid == 0) {
        int tot = 0;
        for (int e = 0; e < cnt; ++e) tot += ent[e].y;
        const int nch = min(kCPChunks, max(1, tot / kCPChunkMin));
        s_nch = nch;
        if (chunk < nch) {
            const int a0 = (int)((long long)tot * chunk / nch), a1 = (int)((long long)tot * (chunk + 1) / nch);
            int e = 0, acc = 0;
            while (e < cnt && acc + ent[e].y <= a0) acc += ent[e++].y;
            s_e = e;
            s_off = a0 - acc;
            s_len = a1 - a0;
        }
    }
    for (int q = tid; q < NC; q += blockDim.x) {
        int n = 0;
        while (tay_nc(n) <= q) ++n;                  // graded level of position q
        const int t = q - (n > 0 ? tay_nc(n - 1) : 0);
        int i = 0;
        while ((i + 1) * (i + 2) / 2 <= t) ++i;
        const int k2 = i - (t - i * (i + 1) / 2);
        const int ks[3] = {n - i, k2, i - k2};
        kk[q] = make_char4((char)ks[0], (char)k2, (char)ks[2], (char)n);
        for (int d = 0; d < 3; ++d) {
            int m1[3] = {ks[0], ks[1], ks[2]}, m2[3] = {ks[0], ks[1], ks[2]};
            m1[d] -= 1;
            m2[d] -= 2;
            lk[q][d] = make_short2(m1[d] >= 0 ? (short)tay_graded(m1[0], m1[1], m1[2]) : (short)-1,
                                   m2[d] >= 0 ? (short)tay_graded(m2[0], m2[1], m2[2]) : (short)-1);
        }
    }
    __syncthreads();
    const int nch = s_nch;
    if (chunk >= nch) return;
    if (chunk == 0 && tid == 0) {
        c.tflag[box] = 1;
        c.tnch[box] = nch;
    }
    float2* out = chunk == 0 ? c.tpot + (int64_t)box * c.tb.P3
                             : c.tpart + ((int64_t)box * (kCPChunks - 1) + chunk - 1) * c.tb.P3;
    // box centre (exact half-integers) and radius; the scaled screening constant
    const float cx = (float)T.lo[0] + 0.5f * (float)(T.ext[0] - 1), cy = (float)T.lo[1] + 0.5f * (float)(T.ext[1] - 1),
                cz = (float)T.lo[2] + 0.5f * (float)(T.ext[2] - 1);
    const float sc = T.r, isc = 1.f / sc, kh = c.tb.kapg * sc;
    float m1h[J], m1l[J], mkh[J], mkl[J];
#pragma unroll
    for (int j = 0; j < J; ++j) m1h[j] = m1l[j] = mkh[j] = mkl[j] = 0.f;
    Cursor cur;
    __syncthreads();
    if (tid == kTayWarps * 32) {
        cur.e = box * c.cp_cap + s_e;
        cur.e_end = box * c.cp_cap + cnt;
        cur.off = s_off;
        cur.left = s_len;
        cur.produced = 0;
        cur.done = false;
        for (int st = 0; st < kStages; ++st) cur.last_phase[st] = -1;
        ring_init(r, kTayWarps);
    }
    __syncthreads();
    float* A1 = sa + w * NC;
    float* Ak = sA + w * NC;
    float* Bk = sB + w * NC;
    const int rr = run_ring<1, false, kTayWarps>(
        r, cur, c.cp_ent, a.srcf, nullptr, a, [&](int slot, int n) {
            float p1[J], pk[J];
#pragma unroll
            for (int j = 0; j < J; ++j) p1[j] = pk[j] = 0.f;
            for (int at = w; at < n; at += kTayWarps) {
                const SrcF y = r.src[slot][at];
                // r = (c - y) / s from the float-float source position (one rounding per component)
                const float rx = ((cx - y.xh) - y.xl) * isc, ry = ((cy - y.yh) - y.yl) * isc,
                            rz = ((cz - y.zh) - y.zl) * isc;
                const float rho2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                const float irho2 = 1.f / rho2, irho = rsqrtf(rho2), rho = rho2 * irho;
                if (lane == 0) {
                    A1[0] = irho;
                    if (DH) {
                        const float e = __expf(-kh * rho);
                        Bk[0] = e;
                        Ak[0] = e * irho;
                    }
                }
                __syncwarp();
                const float rv[3] = {rx, ry, rz};
                for (int lv = 1; lv <= P; ++lv) {
                    const int q0 = tay_nc(lv - 1), q1 = tay_nc(lv);
                    const float inv = 1.f / (float)lv, f1 = 2.f - inv, f2 = 1.f - inv, kn = kh * inv;
                    for (int q = q0 + lane; q < q1; q += 32) {
                        float s1 = 0.f, s2 = 0.f, t1 = 0.f, t2 = 0.f, u1 = 0.f, u2 = 0.f;
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            const short2 l = lk[q][d];
                            if (l.x >= 0) {
                                s1 = fmaf(rv[d], A1[l.x], s1);
                                if (DH) {
                                    t1 = fmaf(rv[d], Ak[l.x], t1);
                                    u1 = fmaf(rv[d], Bk[l.x], u1);
                                }
                            }
                            if (l.y >= 0) {
                                s2 += A1[l.y];
                                if (DH) {
                                    t2 += Ak[l.y];
                                    u2 += Bk[l.y];
                                }
                            }
                        }
                        A1[q] = (f1 * s1 - f2 * s2) * irho2;
                        if (DH) {
                            Ak[q] = (f1 * t1 - f2 * t2 + kn * (u1 - u2)) * irho2;
                            Bk[q] = kn * (t1 - t2);
                        }
                    }
                    __syncwarp();
                }
                // moments: q (-1)^{|k|} a_k, each lane its positions lane + 32 j
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const int q = lane + 32 * j;
                    if (q < NC) {
                        const float sq = (kk[q].w & 1) ? -y.q : y.q;
                        p1[j] = fmaf(sq, A1[q], p1[j]);
                        if (DH) pk[j] = fmaf(sq, Ak[q], pk[j]);
                    }
                }
                __syncwarp();
            }
#pragma unroll
            for (int j = 0; j < J; ++j) {
                ff_add(m1h[j], m1l[j], p1[j]);
                if (DH) ff_add(mkh[j], mkl[j], pk[j]);
            }
        },
        [](int) {});
    // every thread reaches this barrier (an aborted ring leaves uniformly, after it)
    if (__syncthreads_or(rr == kRingAbort)) return;
    if (w < kTayWarps) {
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int q = lane + 32 * j;
            if (q < NC) red[w * NC + q] = make_float2(m1h[j] + m1l[j], mkh[j] + mkl[j]);
        }
    }
    __syncthreads();
    for (int q = tid; q < NC; q += blockDim.x) {
        float2 v = make_float2(0.f, 0.f);
        for (int ww = 0; ww < kTayWarps; ++ww) {
            v.x += red[ww * NC + q].x;
            v.y += red[ww * NC + q].y;
        }
        const char4 k = kk[q];
        out[tay_lexoff(P, k.x, k.y) + k.z] = v;
    }
}

// Taylor field onto the grid: one CTA per level-0 box region; every box that contains it and holds moments
// adds (1/s) sum_k M_k t^k at the region's points, evaluated by nested Horner (z innermost: a thread takes 8
// points of one (x, y) column per pass).  Written to the far-field buffer as the far kernel's starting value.
template <int P>
__global__ void __launch_bounds__(256) k_tay_down(CPArgs c, float4* far, const TreeMeta* meta) {
    constexpr int NC = tay_nc(P), M = kTB0, NZP = 8;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    float2* mom = reinterpret_cast<float2*>(sm_raw);  // [L][NC]
    __shared__ int lexoff[(P + 1) * (P + 1)];
    __shared__ int lev[kMaxTL];
    __shared__ float cen[kMaxTL][4];
    __shared__ int nlev;
    if (meta->overflow) return;
    const TBoxes& tb = c.tb;
    const int bi = blockIdx.x;
    const int ib = bi % tb.nbx[0], jb = (bi / tb.nbx[0]) % tb.nby[0], kb = bi / (tb.nbx[0] * tb.nby[0]);
    const TBox R = tbox_at(tb, 0, ib, jb, kb);
    const int tid = threadIdx.x;
    if (tid == 0) {
        int k = 0;
        for (int l = 0; l < tb.L; ++l) {
            const TBox A = tbox_at(tb, l, ib >> l, jb >> l, kb >> l);
            if (A.proxied && c.tflag[tbox_index(tb, l, A.ib, A.jb, A.kb)]) {
                lev[k] = tbox_index(tb, l, A.ib, A.jb, A.kb);
                cen[k][0] = A.c[0];
                cen[k][1] = A.c[1];
                cen[k][2] = A.c[2];
                cen[k][3] = A.r;
                ++k;
            }
        }
        nlev = k;
    }
    for (int q = tid; q < (P + 1) * (P + 1); q += blockDim.x) {
        const int k1 = q / (P + 1), k2 = q % (P + 1);
        lexoff[q] = k1 + k2 <= P ? tay_lexoff(P, k1, k2) : 0;
    }
    __syncthreads();
    const int nl = nlev;
    for (int q = tid; q < nl * NC; q += blockDim.x) {
        const int k = q / NC;
        mom[q] = c.tpot[(int64_t)lev[k] * tb.P3 + (q - k * NC)];
    }
    __syncthreads();
    const int m0 = R.ext[0], m1 = R.ext[1], m2 = R.ext[2];
    const int ix = tid % M, iy = tid / M;  // the thread's (x, y) column
    for (int z0 = 0; z0 < M; z0 += NZP) {
        float2 v[NZP];
#pragma unroll
        for (int pz = 0; pz < NZP; ++pz) v[pz] = make_float2(0.f, 0.f);
        for (int k = 0; k < nl; ++k) {
            const float is = 1.f / cen[k][3];
            const float tx = ((float)(R.lo[0] + ix) - cen[k][0]) * is, ty = ((float)(R.lo[1] + iy) - cen[k][1]) * is;
            float tz[NZP];
#pragma unroll
            for (int pz = 0; pz < NZP; ++pz) tz[pz] = ((float)(R.lo[2] + z0 + pz) - cen[k][2]) * is;
            const float2* Mk = mom + k * NC;
            float2 V[NZP];
#pragma unroll
            for (int pz = 0; pz < NZP; ++pz) V[pz] = make_float2(0.f, 0.f);
            for (int k1 = P; k1 >= 0; --k1) {
                float2 W[NZP];
#pragma unroll
                for (int pz = 0; pz < NZP; ++pz) W[pz] = make_float2(0.f, 0.f);
                for (int k2 = P - k1; k2 >= 0; --k2) {
                    const float2* base = Mk + lexoff[k1 * (P + 1) + k2];
                    float2 Q[NZP];
#pragma unroll
                    for (int pz = 0; pz < NZP; ++pz) Q[pz] = make_float2(0.f, 0.f);
                    for (int k3 = P - k1 - k2; k3 >= 0; --k3) {
                        const float2 m = base[k3];
#pragma unroll
                        for (int pz = 0; pz < NZP; ++pz) {
                            Q[pz].x = fmaf(Q[pz].x, tz[pz], m.x);
                            Q[pz].y = fmaf(Q[pz].y, tz[pz], m.y);
                        }
                    }
#pragma unroll
                    for (int pz = 0; pz < NZP; ++pz) {
                        W[pz].x = fmaf(W[pz].x, ty, Q[pz].x);
                        W[pz].y = fmaf(W[pz].y, ty, Q[pz].y);
                    }
                }
#pragma unroll
                for (int pz = 0; pz < NZP; ++pz) {
                    V[pz].x = fmaf(V[pz].x, tx, W[pz].x);
                    V[pz].y = fmaf(V[pz].y, tx, W[pz].y);
                }
            }
#pragma unroll
            for (int pz = 0; pz < NZP; ++pz) {
                v[pz].x = fmaf(V[pz].x, is, v[pz].x);
                v[pz].y = fmaf(V[pz].y, is, v[pz].y);
            }
        }
#pragma unroll
        for (int pz = 0; pz < NZP; ++pz) {
            const int iz = z0 + pz;
            if (ix < m0 && iy < m1 && iz < m2)
                far[far_index(tb.nx, tb.ny, R.lo[0] + ix, R.lo[1] + iy, R.lo[2] + iz)] =
                    make_float4(v[pz].x, 0.f, v[pz].y, 0.f);
        }
    }
}

template <int P>
void launch_taylor(const TBoxes& tb, const EvalArgs& a, const CPArgs& c, float4* far, const TreeMeta* meta, bool dh,
                   cudaStream_t st) {
    const dim3 grid(tb.nbox, kCPChunks);
    const size_t se = (size_t)kTayWarps * tay_nc(P) * (sizeof(float2) + 3 * sizeof(float));
    if (dh) {
        raise_dyn_smem(k_tay_eval<P, true>, se);
        k_tay_eval<P, true><<<grid, kTayWarps * 32 + 32, se, st>>>(a, c);
    } else {
        raise_dyn_smem(k_tay_eval<P, false>, se);
        k_tay_eval<P, false><<<grid, kTayWarps * 32 + 32, se, st>>>(a, c);
    }
    k_cp_reduce<<<tb.nbox, 256, 0, st>>>(c, meta);
    const size_t sm = sizeof(float2) * (size_t)tb.L * tay_nc(P);
    raise_dyn_smem(k_tay_down<P>, sm);
    k_tay_down<P><<<tb.nbx[0] * tb.nby[0] * tb.nbz[0], 256, sm, st>>>(c, far, meta);
}

void launch_taylor_deg(const TBoxes& tb, const EvalArgs& a, const CPArgs& c, float4* far, const TreeMeta* meta,
                       bool dh, cudaStream_t st) {
    switch (tb.deg) {
        case 1: return launch_taylor<1>(tb, a, c, far, meta, dh, st);
        case 2: return launch_taylor<2>(tb, a, c, far, meta, dh, st);
        case 3: return launch_taylor<3>(tb, a, c, far, meta, dh, st);
        case 4: return launch_taylor<4>(tb, a, c, far, meta, dh, st);
        case 5: return launch_taylor<5>(tb, a, c, far, meta, dh, st);
        case 6: return launch_taylor<6>(tb, a, c, far, meta, dh, st);
        case 7: return launch_taylor<7>(tb, a, c, far, meta, dh, st);
        case 8: return launch_taylor<8>(tb, a, c, far, meta, dh, st);
        case 9: return launch_taylor<9>(tb, a, c, far, meta, dh, st);
        case 10: return launch_taylor<10>(tb, a, c, far, meta, dh, st);
        case 11: return launch_taylor<11>(tb, a, c, far, meta, dh, st);
        default: return launch_taylor<12>(tb, a, c, far, meta, dh, st);
    }
}

// Box-level far field (no allocation, no host wait): proxies of every target box, the downward pass and the
// interpolation onto the far-field buffer.  Returns the number of launches.
// The preparation's side branch joined back into st (its lists and orders are read after this point).
void side_join(TreeState* s, cudaStream_t st) {
    if (!s->side_pending) return;
    cudaStreamWaitEvent(st, s->side_join, 0);
    s->side_pending = false;
}

// Box layers [z0, z1) of level l that z slab k of the far and near launches needs first: every layer of the
// level that meets the slab's grid planes and no earlier slab's (a level-l box is 16 2^l points high, a batch
// layer 8 or 16).  The layers a slab needs at level l hold the parents of those it needs at level l - 1.
void box_layers(const TreeState* s, int l, int k, int& z0, int& z1) {
    const int nzb = shape_of(s->variant).nz, nbzl = s->tb.nbz[l], E = kTB0 << l;
    auto end = [&](int kk) {
        const int kb1 = slab_start(kk + 1, s->nslab, s->nbz);
        return std::min(nbzl, (int)(((int64_t)kb1 * nzb + E - 1) / E));
    };
    z0 = k == 0 ? 0 : end(k - 1);
    z1 = end(k);
}

void cp_launch(const EvalArgs& a, const CPArgs& c, int nbox, bool dh, cudaStream_t st, const TreeMeta* meta) {
    const int n1 = c.tb.deg + 1;
    const int npass = (n1 * n1 * ((n1 + kCPP - 1) / kCPP) + kCPThreads - 1) / kCPThreads;
    const dim3 grid(nbox, kCPChunks, npass);
    if (dh) k_cp_eval<true><<<grid, kCPThreads + 32, 0, st>>>(a, c);
    else k_cp_eval<false><<<grid, kCPThreads + 32, 0, st>>>(a, c);
    k_cp_reduce<<<nbox, 256, 0, st>>>(c, meta);
}

// Box-level far field (a10, cluster-particle form), then the join of the preparation's side branch.
// split (with z slabs): only the box order here, grouped by slab; each slab's launches start with the boxes of
// every level that the slab needs first (cp_slab), so the first slab's outputs are final after its share of the
// box level, and the side branch joins after the first slab's boxes.
int cp_enqueue(TreeState* s, const EvalArgs& a, bool dh, cudaStream_t st, bool split = false) {
    const TBoxes& tb = s->tb;
    s->box_split = false;
    if (!tb.enabled) {
        side_join(s, st);
        return 0;
    }
    CPArgs c = make_cp(s);
    if (tb.approx == RISM_APPROX_TAYLOR) {
        c.order = nullptr;  // the moment kernels run in index order (no box order is made for them)
        launch_taylor_deg(tb, a, c, s->far, s->meta, dh, st);
        side_join(s, st);
        return 3;
    }
    split = split && s->nslab > 1;
    if (split) c.order = s->cp_order;  // a slab's boxes of several levels are one launch: always by the order
    if (c.order) {
        OrderGroups og = order_plain(tb.nbox);
        if (split) {
            og.ns = s->nslab;
            og.nlev = tb.L;
            for (int l = 0; l < tb.L; ++l) {
                og.off[l] = tb.off[l];
                og.nbxy[l] = tb.nbx[l] * tb.nby[l];
                for (int k = 0; k < s->nslab; ++k) {
                    int z1;
                    box_layers(s, l, k, og.bnd[l][k], z1);
                }
            }
            og.off[tb.L] = tb.nbox;
        }
        k_cp_work<<<(tb.nbox + 7) / 8, 256, 0, st>>>(c, s->meta, s->cp_work);
        k_order<<<1, 1024, 0, st>>>(tb.nbox, s->cp_work, s->cp_order, nullptr, nullptr, og);
    }
    const int nord = c.order ? 2 : 0;
    if (split) {
        s->box_split = true;
        s->box_pos = 0;
        return nord;
    }
    cp_launch(a, c, tb.nbox, dh, st, s->meta);
    const int nd = launch_down_deg(tb, c, s->far, s->meta, st);
    side_join(s, st);
    return nord + 2 + nd;
}

// The boxes z slab k needs first after a split cp_enqueue (the next range of the box order): their proxies and
// chunk sums, the downward pass into their layers level by level, and the level-0 boxes' grid points.  Returns
// the number of launches.
int cp_slab(TreeState* s, const EvalArgs& a, bool dh, int k, cudaStream_t st) {
    const TBoxes& tb = s->tb;
    int zr[kMaxTL][2];
    int count = 0;
    for (int l = 0; l < tb.L; ++l) {
        box_layers(s, l, k, zr[l][0], zr[l][1]);
        count += (zr[l][1] - zr[l][0]) * tb.nbx[l] * tb.nby[l];
    }
    if (count == 0) return 0;
    CPArgs c = make_cp(s);
    c.order = s->cp_order + s->box_pos;
    s->box_pos += count;
    cp_launch(a, c, count, dh, st, s->meta);
    return 2 + launch_down_deg(tb, c, s->far, s->meta, st, zr);
}

// Kernel launches of a7..a9 for one solute (no allocation, no host wait:
// safe inside a stream capture).
rism_status tree_enqueue(TreeState* s, const DevTables& t, const GridD& g, const Phys& ph, const rism_options& o,
                         cudaStream_t st, std::string& err) {
    const int n = (int)t.n;
    const int deg = o.degree, np = deg + 1, P3 = np * np * np;
    const ShapeDesc sd = shape_of(s->variant);
    s->launches = 0;
    k_reset_meta<<<1, 1, 0, st>>>(s->meta);
    ++s->launches;
    if (n > 0) {
        const int gb = std::min((n + 255) / 256, 4 * sm_count());
        k_bounds<<<gb, 256, 0, st>>>(t.srcf, t.ljf, n, ph.S, t.smax, s->meta);
        k_codes<<<gb, 256, 0, st>>>(t.srcf, n, ph.rs / g.h, s->meta, s->code, s->idx);
        // the FP64 sorted positions feed only the source proxies' upward pass (off with target boxes)
        BuildArgs ba{n, s->leaf, P3, s->max_nodes, s->max_prox, s->max_items, t.geo, t.srcf, t.ljf, t.smax, g,
                     1.0 / g.h, s->tb.enabled ? nullptr : s->src, s->srcf, s->ljs, s->ljs2};
        const size_t shb = t.n <= kSortSmem ? (kHistInts + 64) * sizeof(int) +
                                                  kSortSmem * (sizeof(unsigned long long) + 4 * sizeof(uint32_t)) +
                                                  kNodeSmem * sizeof(Node)
                           : t.n <= kCodeSmem ? (kHistInts + 64) * sizeof(int) + kCodeSmem * sizeof(uint32_t) +
                                                    std::max(kCodeSmem * sizeof(uint32_t), kNodeSmemL * sizeof(Node))
                                              : (kHistInts + 64) * sizeof(int);
        raise_dyn_smem(k_sort_build, shb);
        k_sort_build<<<1, kSortThreads, shb, st>>>(ba, s->code, s->idx, s->code2, s->idx2, s->nodes, s->items,
                                                   s->prox_nodes, s->prox_items, s->meta);
        k_gather_cells<<<1024, 256, 0, st>>>(ba, s->idx, s->meta, s->code, s->cell_start);
        s->launches += 4;
        if (t.n > kSortSmem) {
            k_node_boxes<<<std::min(s->max_nodes, 4 * sm_count()), kBoxThreads, 0, st>>>(s->meta, s->nodes, s->srcf);
            ++s->launches;
        }
        if (!s->tb.enabled) {
            // source proxies: only the batch-level traversal uses them (with target boxes on, the box level
            // accepts every cluster a batch would)
            const size_t shu = (kChunk * 3 * np + kChunk + 3 * np) * sizeof(double);
            raise_dyn_smem(k_upward, shu);
            k_upward<<<4 * sm_count(), 256, shu, st>>>(deg, s->meta, s->nodes, s->prox_nodes, s->items, s->src,
                                                       s->part);
            k_proxy_reduce<<<2 * sm_count(), 256, 0, st>>>(deg, n, s->meta, s->nodes, s->prox_nodes,
                                                           s->prox_items, s->part, s->src, s->srcf);
            s->launches += 2;
        }
    }
    // side branch: the near lists need only the cell table, so they run beside the box-level lists; the far
    // lists (which start from the box level's pass-down lists) and the launch orders run beside the box-level
    // evaluation that the caller enqueues next (cp_enqueue joins the branch back)
    const TBoxes& tb = s->tb;
    ListArgs fa{s->nbx, s->nby, s->nbz, sd.nx, sd.ny, sd.nz, o.theta, n, P3, s->cap_far,
                tb.enabled ? s->dn_cnt : nullptr, s->dn_ent, s->cap_dn, tb, tb.enabled ? 0 : 1};
    ListArgs na = fa;
    na.cap = s->cap_near;
    const int lgrid = (s->nb + kListWarps - 1) / kListWarps;
    cudaEventRecord(s->side_fork[0], st);
    cudaStreamWaitEvent(s->side, s->side_fork[0], 0);
    k_near_lists<<<lgrid, 32 * kListWarps, 0, s->side>>>(na, s->cell_start, s->near_ent, s->near_cnt, s->near_work,
                                                          s->meta);
    if (tb.enabled) {
        TListArgs ta{tb, 0, n, P3, o.theta, s->cap_cp, s->cap_dn, s->cp_cnt, s->cp_ent, s->dn_cnt, s->dn_ent};
        for (int l = tb.L - 1; l >= 0; --l) {
            ta.l = l;
            const int nbl = tb.nbx[l] * tb.nby[l] * tb.nbz[l];
            k_tbox_lists<<<(nbl + kListWarps - 1) / kListWarps, 32 * kListWarps, 0, st>>>(ta, s->nodes, s->meta);
            ++s->launches;
        }
    }
    cudaEventRecord(s->side_fork[1], st);
    cudaStreamWaitEvent(s->side, s->side_fork[1], 0);
    k_far_lists<<<lgrid, 32 * kListWarps, 0, s->side>>>(fa, s->nodes, s->far_ent, s->far_cnt, s->far_work, s->meta);
    OrderGroups og = order_plain(s->nb);
    og.ns = std::max(1, s->nslab);
    og.nbxy[0] = s->nbx * s->nby;
    for (int k = 0; k < og.ns; ++k) og.bnd[0][k] = slab_start(k, og.ns, s->nbz);
    k_order<<<2, 1024, 0, s->side>>>(s->nb, s->near_work, s->near_order, s->far_work, s->far_order, og);
    cudaEventRecord(s->side_join, s->side);
    s->side_pending = true;
    s->launches += 3;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(err, e, "tree build");
    s->prepared = true;
    return RISM_OK;
}

EvalArgs make_args(TreeState* s, const DevTables& t, const GridD& g, const Phys& ph, const rism_options& o,
                   Outputs out) {
    EvalArgs a;
    a.g = g;
    a.ph = ph;
    a.nbx = s->nbx;
    a.nby = s->nby;
    a.nbz = s->nbz;
    a.n = (int)t.n;
    a.srcf = s->srcf;
    a.ljs = s->ljs;
    a.ljs2 = s->ljs2;
    a.far_cnt = s->far_cnt;
    a.far_ent = s->far_ent;
    a.near_cnt = s->near_cnt;
    a.near_ent = s->near_ent;
    a.far_cap = s->cap_far;
    a.near_cap = s->cap_near;
    a.far = s->far;
    a.far_init = s->tb.enabled ? 1 : 0;
    a.ntab = s->ntab;
    a.ntab_inv = s->ntab_inv;
    a.uni_rc = o.lj_mode != RISM_LJ_TOL ? 1 : 0;
    a.near_order = s->near_order;
    a.wq = s->wq;
    a.q0 = 0;
    a.q1 = s->nb * (shape_of(s->variant).nx / 8);  // sub-batches of 8 points along x
    a.f0 = 0;
    a.far_order = s->far_order;
    a.near_work = s->near_work;
    a.far_work = s->far_work;
    {
        const double ih = 1.0 / g.h;
        for (int k = 0; k < kMaxSites; ++k) {
            const double qs = k < ph.S ? ph.qs[k] : 0.0;
            const double cu = ph.k_e * ih * qs;
            a.cu_h[k] = (float)cu;
            a.cu_l[k] = (float)(cu - (double)a.cu_h[k]);
            a.cc[k] = (float)(-ph.beta * ph.k_e * ih * qs);
            a.ch[k] = (float)(-ph.beta * ph.k_e / (2.0 * ph.eps_r) * ih * qs);
        }
        const double e2 = 2.0 * ph.ea2;
        a.e2a_h = (float)e2;
        a.e2a_l = (float)(e2 - (double)a.e2a_h);
        a.kap2 = (float)(-ph.kappa * g.h * 1.4426950408889634);
        a.rs2 = (float)((ph.rs / g.h) * (ph.rs / g.h));
        a.c0h = (float)(ph.phi_c0 * g.h);
        a.h0h = (float)(ph.phi_h0 * g.h);
    }
    a.o = out;
    a.err = t.err;
    a.meta = s->meta;
    a.wlim = o.wait_limit;
    return a;
}

// ---- autotuner: problem class -> (shape variant, leaf size)
std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune;
bool g_tune_loaded = false;

std::string tune_path() {
    const char* p = std::getenv("RISM_AUTOTUNE_CACHE");
    return p ? std::string(p) : std::string();
}

void tune_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const std::string path = tune_path();
    if (path.empty()) return;
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return;
    char key[512];
    int v, l;
    // one entry per line: "<key>" variant leaf
    while (std::fscanf(f, " \"%511[^\"]\" %d %d", key, &v, &l) == 3) g_tune[key] = {v, l};
    std::fclose(f);
}

void tune_save() {
    const std::string path = tune_path();
    if (path.empty()) return;
    FILE* f = std::fopen(path.c_str(), "w");
    if (!f) return;
    for (auto& kv : g_tune) std::fprintf(f, "\"%s\" %d %d\n", kv.first.c_str(), kv.second.first, kv.second.second);
    std::fclose(f);
}

std::string problem_class(const DevTables& t, const GridD& g, const Phys& ph, const rism_options& o) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, dev);
    auto lg = [](double v) { return (int)std::lround(std::log2(v > 1 ? v : 1)); };
    char buf[400];
    std::snprintf(buf, sizeof buf, "%s|sm%d|S%d|n2^%d|m2^%d|p%d|th%d|lj%d|k%d|ap%d", p.name, p.multiProcessorCount,
                  t.smax, lg((double)t.n), lg((double)g.nx * g.ny * g.nz), o.degree, (int)std::lround(o.theta * 100),
                  o.lj_mode, ph.kappa > 0.0, o.approx);
    for (char* c = buf; *c; ++c)
        if (*c == '"') *c = '\'';
    return buf;
}

}  // namespace

TreeState* tree_create() { return new TreeState(); }

struct BatchCache {
    std::vector<unsigned char> sig;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr;  // private stream the sequence is captured on (the caller's may be the legacy one)
    EvalArgs* d_args = nullptr;
    int* d_off = nullptr;
    int* d_queue = nullptr;
    int* d_work = nullptr;   // [total] item work (far, then near)
    int* d_order = nullptr;  // [2 total] global orders: far, then near
    static constexpr int kBranches = 8;  // per-solute preparations captured on this many forked streams
    cudaStream_t side[kBranches] = {};
    cudaEvent_t fork = nullptr, join[kBranches] = {};
    int cap = 0;
    ~BatchCache() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
        cudaFree(d_args);
        cudaFree(d_off);
        cudaFree(d_queue);
        cudaFree(d_work);
        cudaFree(d_order);
        for (int k = 0; k < kBranches; ++k) {
            if (side[k]) cudaStreamDestroy(side[k]);
            if (join[k]) cudaEventDestroy(join[k]);
        }
        if (fork) cudaEventDestroy(fork);
    }
};

struct SoluteGraph {
    std::vector<unsigned char> sig;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr, side = nullptr;  // side: the LJ tail, a parallel branch of the graph
    cudaEvent_t fork = nullptr, join = nullptr;
    int launches = 0;
    ~SoluteGraph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
        if (side) cudaStreamDestroy(side);
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
    }
};

void tree_graph_reset(TreeState* s) {
    if (!s) return;
    delete s->sg;
    s->sg = nullptr;
}

void adjtree_delete(AdjTree* a);

void tree_destroy(TreeState* s) {
    if (!s) return;
    adjtree_delete(s->adj);
    delete s->sg;
    delete s->bc;
    for (int k = 0; k < 4; ++k)
        if (s->ev[k]) cudaEventDestroy(s->ev[k]);
    for (int k = 0; k < kMaxSlabs; ++k)
        if (s->slab_ev[k]) cudaEventDestroy(s->slab_ev[k]);
    for (int k = 0; k < 2; ++k)
        if (s->side_fork[k]) cudaEventDestroy(s->side_fork[k]);
    if (s->side_join) cudaEventDestroy(s->side_join);
    if (s->side) cudaStreamDestroy(s->side);
    cudaFree(s->cp_cnt);
    cudaFree(s->dn_cnt);
    cudaFree(s->dn_ent);
    cudaFree(s->tflag);
    cudaFree(s->cp_ent);
    cudaFree(s->tpot);
    cudaFree(s->tpart);
    cudaFree(s->tnch);
    cudaFree(s->cp_work);
    cudaFree(s->cp_order);
    cudaFree(s->ntab);
    cudaFree(s->code);
    cudaFree(s->idx);
    cudaFree(s->code2);
    cudaFree(s->idx2);
    cudaFree(s->nodes);
    cudaFree(s->items);
    cudaFree(s->prox_nodes);
    cudaFree(s->part);
    cudaFree(s->src);
    cudaFree(s->srcf);
    cudaFree(s->far);
    cudaFree(s->ljs);
    cudaFree(s->ljs2);
    cudaFree(s->far_cnt);
    cudaFree(s->near_cnt);
    cudaFree(s->near_work);
    cudaFree(s->near_order);
    cudaFree(s->wq);
    cudaFree(s->far_work);
    cudaFree(s->far_order);
    cudaFree(s->prox_items);
    cudaFree(s->far_ent);
    cudaFree(s->near_ent);
    cudaFree(s->cell_start);
    cudaFree(s->meta);
    cudaFreeHost(s->h_meta);
    delete s;
}

// Without the autotuner: the leaf size of the options and launch shape 0, or the shape that debug_flags bits 4-5
// name (value v + 1 forces shape v; a test hook).
static void fixed_shape(TreeState* s, const rism_options& o) {
    s->leaf = o.leaf;
    const int v = (o.debug_flags >> 4) & 3;
    s->variant = v >= 1 && v <= kNumShapes ? v - 1 : 0;
}

rism_status tree_prepare(TreeState* s, const DevTables& t, const GridD& g, const Phys& ph, const rism_options& o,
                         cudaStream_t st, std::string& err) {
    if (!o.autotune) fixed_shape(s, o);
    rism_status r = tree_reserve(s, t, g, ph, o, err);
    if (r != RISM_OK) return r;
    r = tree_enqueue(s, t, g, ph, o, st, err);
    side_join(s, st);  // callers of the prepared tree may read every list next
    return r;
}

// Time each (shape, leaf) candidate once (prepare + evaluation, CUDA events)
// and keep the fastest for this problem class.
static rism_status tree_autotune(TreeState* s, const DevTables& t, const GridD& g, const Phys& ph,
                                 const rism_options& o, Outputs out, cudaStream_t st, std::string& err) {
    const std::string key = problem_class(t, g, ph, o);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        tune_load();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            s->variant = it->second.first;
            s->leaf = it->second.second;
            s->tuned_key = key;
            rism_status r = tree_reserve(s, t, g, ph, o, err);
            return r != RISM_OK ? r : tree_enqueue(s, t, g, ph, o, st, err);
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bv = 0, bl = o.leaf;
    const int leaves[2] = {o.leaf, o.leaf >= 64 ? o.leaf / 2 : o.leaf * 2};
    for (int v = 0; v < kNumShapes; ++v)
        for (int li = 0; li < 2; ++li)
            for (int attempt = 0; attempt < 2; ++attempt) {
                s->variant = v;
                s->leaf = leaves[li];
                rism_status r = tree_reserve(s, t, g, ph, o, err);
                if (r != RISM_OK) return r;
                cudaEventRecord(e0, st);
                r = tree_enqueue(s, t, g, ph, o, st, err);
                if (r != RISM_OK) return r;
                EvalArgs a = make_args(s, t, g, ph, o, out);
                cp_enqueue(s, a, out.h != nullptr, st);
                dispatch(t.smax, v, 0, out.u != nullptr, out.h != nullptr, &a, s->nb, nullptr, 0, st);
                cudaEventRecord(e1, st);
                cudaMemcpyAsync(s->h_meta, s->meta, sizeof(TreeMeta), cudaMemcpyDeviceToHost, st);
                cudaError_t ce = cudaStreamSynchronize(st);
                if (ce != cudaSuccess) return cuda_err(err, ce, "autotune");
                const TreeMeta& m = *s->h_meta;
                if (m.overflow) {
                    // grow the list slots and time this candidate again
                    if (grow_lists(s, m)) continue;
                    break;  // too wide or too deep for this leaf size: skip the candidate
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                // two more timings of the same candidate (lists are now large enough); keep the fastest of three
                for (int rep = 0; rep < 2; ++rep) {
                    cudaEventRecord(e0, st);
                    if ((r = tree_enqueue(s, t, g, ph, o, st, err)) != RISM_OK) return r;
                    cp_enqueue(s, a, out.h != nullptr, st);
                    dispatch(t.smax, v, 0, out.u != nullptr, out.h != nullptr, &a, s->nb, nullptr, 0, st);
                    cudaEventRecord(e1, st);
                    if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_err(err, ce, "autotune");
                    float m2 = 0.f;
                    cudaEventElapsedTime(&m2, e0, e1);
                    ms = fminf(ms, m2);
                }
                if (ms < best) {
                    best = ms;
                    bv = v;
                    bl = leaves[li];
                }
                break;
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->variant = bv;
    s->leaf = bl;
    s->tuned_key = key;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[key] = {bv, bl};
        tune_save();
    }
    rism_status r = tree_reserve(s, t, g, ph, o, err);
    return r != RISM_OK ? r : tree_enqueue(s, t, g, ph, o, st, err);
}

// The far and near kernels (+ epilogue) as one launch each, or per z slab of batch layers (s->nslab > 1): the
// far and then the near launch of each slab, followed by a record of the slab's event (external records when the
// launches are being captured into a graph, so that streams outside the graph can wait on a slab).  After a split
// cp_enqueue each slab's launches start with its level-0 boxes.  The first slab's outputs are then complete after
// the coarser box levels and a slab's share of the rest, not after the whole box level and far field.
namespace {
cudaError_t farnear_enqueue(TreeState* s, int smax, const EvalArgs& a, bool du, bool dh, cudaStream_t st,
                            bool captured, cudaEvent_t mid = nullptr) {
    s->box_slab_launches = 0;
    if (s->nslab <= 1) {
        s->slabs_live = false;
        cudaError_t e = dispatch(smax, s->variant, 2, du, dh, &a, s->nb, nullptr, 0, st);
        if (e == cudaSuccess && mid)
            e = captured ? cudaEventRecordWithFlags(mid, st, cudaEventRecordExternal) : cudaEventRecord(mid, st);
        return e == cudaSuccess ? dispatch(smax, s->variant, 3, du, dh, &a, s->nb, nullptr, 0, st) : e;
    }
    const int NS = shape_of(s->variant).nx / 8, nbxy = s->nbx * s->nby;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < s->nslab && e == cudaSuccess; ++k) {
        const int kb0 = slab_start(k, s->nslab, s->nbz), kb1 = slab_start(k + 1, s->nslab, s->nbz);
        if (s->box_split) {
            s->box_slab_launches += cp_slab(s, a, dh, k, st);
            if (k == 0) side_join(s, st);
        }
        if (kb1 > kb0) {
            EvalArgs b = a;
            b.f0 = kb0 * nbxy;
            b.q0 = kb0 * nbxy * NS;
            b.q1 = kb1 * nbxy * NS;
            e = dispatch(smax, s->variant, 2, du, dh, &b, (kb1 - kb0) * nbxy, nullptr, 0, st);
            if (e == cudaSuccess) e = dispatch(smax, s->variant, 3, du, dh, &b, (kb1 - kb0) * nbxy, nullptr, 0, st);
        }
        if (e == cudaSuccess)
            e = captured ? cudaEventRecordWithFlags(s->slab_ev[k], st, cudaEventRecordExternal)
                         : cudaEventRecord(s->slab_ev[k], st);
    }
    if (e == cudaSuccess && mid)  // no separate far time: the interleaved launches count as far + near
        e = captured ? cudaEventRecordWithFlags(mid, st, cudaEventRecordExternal) : cudaEventRecord(mid, st);
    s->box_split = false;
    s->slabs_live = e == cudaSuccess;
    return e;
}
}  // namespace

rism_status tree_set_slabs(TreeState* s, int nslab, std::string& err) {
    nslab = std::max(1, std::min(nslab, kMaxSlabs));
    for (int k = 0; k < nslab; ++k)
        if (!s->slab_ev[k]) {
            const cudaError_t e = cudaEventCreateWithFlags(&s->slab_ev[k], cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_err(err, e, "slab events");
        }
    s->nslab = nslab;
    return RISM_OK;
}

int tree_slabs(const TreeState* s, const GridD& g, int (*z)[2], cudaEvent_t* ev) {
    if (!s->slabs_live || s->nslab <= 1) return 0;
    const int nzb = shape_of(s->variant).nz;
    for (int k = 0; k < s->nslab; ++k) {
        const int kb0 = slab_start(k, s->nslab, s->nbz), kb1 = slab_start(k + 1, s->nslab, s->nbz);
        z[k][0] = std::min(kb0 * nzb, g.nz);
        z[k][1] = std::min(kb1 * nzb, g.nz);
        ev[k] = s->slab_ev[k];
    }
    return s->nslab;
}

// Enqueue a10 + a11: far kernel, near kernel + epilogue, then a copy of the
// meta block (counts, overflow flag) to pinned memory for tree_post.
rism_status tree_eval(TreeState* s, const DevTables& t, const GridD& g, const Phys& ph, const rism_options& o,
                      Outputs out, cudaStream_t st, std::string& err, rism_info& info) {
    s->slabs_live = false;
    if (!s->prepared) {
        err = "tree not prepared";
        return RISM_E_STATE;
    }
    if (o.autotune && s->tuned_key != problem_class(t, g, ph, o)) {
        rism_status r = tree_autotune(s, t, g, ph, o, out, st, err);
        if (r != RISM_OK) return r;
    }
    EvalArgs a = make_args(s, t, g, ph, o, out);
    const bool du = out.u != nullptr, dh = out.h != nullptr;
    cudaError_t e;
    s->timed = (o.debug_flags & 2) != 0;
    int cpl = 0;
    if (s->timed) {
        for (int k = 0; k < 4; ++k)
            if (!s->ev[k]) cudaEventCreate(&s->ev[k]);
        cudaEventRecord(s->ev[0], st);
        cpl = cp_enqueue(s, a, dh, st, true);
        cudaEventRecord(s->ev[1], st);
        e = farnear_enqueue(s, t.smax, a, du, dh, st, false, s->ev[2]);
        cudaEventRecord(s->ev[3], st);
    } else {
        cpl = cp_enqueue(s, a, dh, st, true);
        e = farnear_enqueue(s, t.smax, a, du, dh, st, false);
    }
    if (e != cudaSuccess) return cuda_err(err, e, "tree eval");
    if ((e = cudaMemcpyAsync(s->h_meta, s->meta, sizeof(TreeMeta), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_err(err, e, "tree meta copy");
    info.launches += s->launches + 2 * std::max(1, s->nslab) + cpl + s->box_slab_launches;
    const ShapeDesc sd = shape_of(s->variant);
    info.batch[0] = sd.nx;
    info.batch[1] = sd.ny;
    info.batch[2] = sd.nz;
    info.kernel_variant = s->variant;
    return RISM_OK;
}

// After the stream has been synchronised: counters into info; a list
// overflow grows the buffer and asks the caller to run prepare + eval again.
rism_status tree_post(TreeState* s, rism_info& info, bool& retry, std::string& err) {
    const TreeMeta& m = *s->h_meta;
    retry = false;
    if (m.overflow && m.wide) {
        err = "an octree level is wider than the list builder's frontier (2048 nodes); use a larger leaf size";
        return RISM_E_NOMEM;
    }
    if (m.build_overflow) {
        err = "tree node, proxy or upward-item capacity exceeded";
        return RISM_E_NOMEM;
    }
    if (m.overflow) {
        if (grow_lists(s, m)) {
            delete s->bc;  // buffers moved: the captured graphs are stale
            s->bc = nullptr;
            tree_graph_reset(s);
            retry = true;
            char buf[256];
            std::snprintf(buf, sizeof buf,
                          "list slots grown: far need %d -> cap %d, near need %d -> cap %d, box need %d -> cap %d, "
                          "pass-down need %d -> cap %d",
                          m.far_need, s->cap_far, m.near_need, s->cap_near, m.cp_need, s->cap_cp, m.dn_need,
                          s->cap_dn);
            err = buf;
            return RISM_OK;
        }
        err = "list capacity exceeded";
        return RISM_E_NOMEM;
    }
    info.far_ms = info.near_ms = info.box_ms = 0.f;
    if (s->timed && s->ev[0]) {
        cudaEventElapsedTime(&info.box_ms, s->ev[0], s->ev[1]);
        cudaEventElapsedTime(&info.far_ms, s->ev[1], s->ev[2]);
        cudaEventElapsedTime(&info.near_ms, s->ev[2], s->ev[3]);
    }
    info.cp_pairs = (int64_t)m.cp_pairs;
    info.tree_boxes = m.tboxes;
    info.near_tested = (int64_t)m.near_tested;
    info.lj_pairs = (int64_t)m.lj_pairs;
    info.sr_pairs = (int64_t)m.sr_pairs;
    info.tree_nodes = m.nnodes;
    info.tree_proxied = m.nprox;
    info.tree_leaves = m.nleaves;
    info.direct_pairs = (int64_t)m.direct_pairs;
    info.proxy_pairs = (int64_t)m.proxy_pairs;
    info.near_pairs = (int64_t)m.near_pairs;
    return RISM_OK;
}

rism_status tree_graph_step(TreeState* s, const DevTables& t, const GridD& g, const Phys& ph, const rism_options& o,
                            Outputs out, const SoluteStep& step, cudaStream_t st, std::string& err, rism_info& info,
                            bool& used) {
    used = false;
    s->slabs_live = false;
    if (o.autotune && s->tuned_key != problem_class(t, g, ph, o)) return RISM_OK;  // time the candidates first
    if (!o.autotune) fixed_shape(s, o);
    rism_status r = tree_reserve(s, t, g, ph, o, err);
    if (r != RISM_OK) return r;
    const EvalArgs a = make_args(s, t, g, ph, o, out);
    const CPArgs cpa = make_cp(s);
    std::vector<unsigned char> sig;
    auto put = [&](const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        sig.insert(sig.end(), c, c + n);
    };
    put(&a, sizeof a);
    put(&cpa, sizeof cpa);
    put(&t, sizeof t);
    put(&step, sizeof step);
    put(step.sig_s, sizeof(double) * kMaxSites);
    put(step.eps_s, sizeof(double) * kMaxSites);
    put(&o, sizeof o);
    const void* ptrs[] = {s->code, s->idx, s->code2, s->idx2, s->nodes, s->items, s->prox_nodes, s->part,
                          s->src, s->srcf, s->ljs, s->far_cnt, s->near_cnt, s->prox_items, s->near_work,
                          s->near_order, s->far_work, s->far_order, s->far_ent, s->near_ent, s->cell_start,
                          s->meta, s->h_meta, s->dn_cnt, s->dn_ent, s->tflag, s->tnch, s->ntab, s->cp_work,
                          s->cp_order};
    put(ptrs, sizeof ptrs);
    const int ints[] = {s->variant, s->leaf, s->max_nodes, s->max_prox, s->max_items, s->cap_far, s->cap_near,
                        s->cap_cp, s->cap_dn, s->nb, s->nslab};
    put(ints, sizeof ints);
    cudaError_t e = cudaSuccess;
    if (!s->sg || s->sg->sig != sig) {
        tree_graph_reset(s);
        if (o.debug_flags & 2)
            for (int k = 0; k < 4; ++k)
                if (!s->ev[k] && (e = cudaEventCreate(&s->ev[k])) != cudaSuccess) return cuda_err(err, e, "events");
        SoluteGraph* G = new SoluteGraph();
        s->sg = G;
        if ((e = cudaStreamCreateWithFlags(&G->cs, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&G->side, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&G->fork, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&G->join, cudaEventDisableTiming)) != cudaSuccess) {
            tree_graph_reset(s);
            return cuda_err(err, e, "capture stream");
        }
        cudaStream_t cs = G->cs;
        if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
            tree_graph_reset(s);
            return cuda_err(err, e, "graph capture");
        }
        const bool dh = out.h != nullptr, du = out.u != nullptr;
        int launches = 0;
        cudaMemcpyAsync(step.d_raw, step.h_raw, sizeof(double) * 6 * step.n, cudaMemcpyHostToDevice, cs);
        DevTables tt = t;
        e = launch_setup(step.d_raw, step.n, ph.S, t.smax, step.sig_s, step.eps_s, step.lj_mode, step.lj_rcut,
                         step.lj_tol, g, tt, cs);
        ++launches;
        // the LJ tail needs only the per-pair tables: a branch parallel to the tree and the evaluation
        const bool tail = e == cudaSuccess && step.d_tail != nullptr;
        if (tail) {
            cudaEventRecord(G->fork, cs);
            cudaStreamWaitEvent(G->side, G->fork, 0);
            e = launch_lj_tail(t, ph.S, step.d_tail, G->side);
            ++launches;
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(step.h_tail, step.d_tail, sizeof(double) * ph.S, cudaMemcpyDeviceToHost, G->side);
            cudaEventRecord(G->join, G->side);
        }
        if (e == cudaSuccess) {
            r = tree_enqueue(s, t, g, ph, o, cs, err);
            launches += s->launches;
        }
        const bool timed = (o.debug_flags & 2) != 0;
        // timing events become event-record nodes of the graph (external records)
        auto rec = [&](int k) {
            if (timed && e == cudaSuccess) e = cudaEventRecordWithFlags(s->ev[k], cs, cudaEventRecordExternal);
        };
        if (e == cudaSuccess && r == RISM_OK) {
            rec(0);
            launches += cp_enqueue(s, a, dh, cs, true);
            rec(1);
            if (e == cudaSuccess) e = farnear_enqueue(s, t.smax, a, du, dh, cs, true, timed ? s->ev[2] : nullptr);
            rec(3);
            launches += 2 * std::max(1, s->nslab) + s->box_slab_launches;
        }
        if (tail) cudaStreamWaitEvent(cs, G->join, 0);
        if (e == cudaSuccess && r == RISM_OK)
            e = cudaMemcpyAsync(s->h_meta, s->meta, sizeof(TreeMeta), cudaMemcpyDeviceToHost, cs);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
        if (r != RISM_OK || e != cudaSuccess || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            tree_graph_reset(s);
            if (r != RISM_OK) return r;
            return cuda_err(err, e != cudaSuccess ? e : ce, "solute graph capture");
        }
        G->graph = graph;
        if ((e = cudaGraphInstantiate(&G->exec, graph, 0)) != cudaSuccess) {
            tree_graph_reset(s);
            return cuda_err(err, e, "graph instantiate");
        }
        G->sig = sig;
        G->launches = launches;
    }
    if ((e = cudaGraphLaunch(s->sg->exec, st)) != cudaSuccess) {
        tree_graph_reset(s);
        return cuda_err(err, e, "graph launch");
    }
    used = true;
    s->slabs_live = s->nslab > 1;  // the graph records the slab events (the slab count is in its signature)
    s->prepared = true;
    s->timed = (o.debug_flags & 2) != 0;
    info.launches = s->sg->launches;
    const ShapeDesc sd = shape_of(s->variant);
    info.batch[0] = sd.nx;
    info.batch[1] = sd.ny;
    info.batch[2] = sd.nz;
    info.kernel_variant = s->variant;
    return RISM_OK;
}

// Many solutes: tables, trees, lists and one persistent far + one persistent
// near kernel draining all (solute, batch) items, captured in a CUDA graph
// on the first context's stream and replayed while nothing that the captured
// launches depend on (pointers, sizes, constants) has changed.
rism_status batch_eval(std::vector<BatchItem>& items, const rism_options& o, cudaStream_t st, DevErr* err,
                       std::string& msg, bool& retry) {
    retry = false;
    const int count = (int)items.size();
    TreeState* s0 = items[0].tree;
    const int variant = s0->variant;
    std::vector<EvalArgs> args((size_t)count);
    std::vector<int> off((size_t)count + 1, 0);
    for (int b = 0; b < count; ++b) {
        BatchItem& it = items[b];
        it.tree->variant = variant;
        if (!o.autotune) it.tree->leaf = o.leaf;
        else it.tree->leaf = s0->leaf;
        rism_status r = tree_reserve(it.tree, *it.t, it.g, it.ph, o, msg);
        if (r != RISM_OK) return r;
        args[b] = make_args(it.tree, *it.t, it.g, it.ph, o, it.o);
        off[b + 1] = off[b] + it.tree->nb;
    }
    // signature of everything the captured launches depend on
    std::vector<unsigned char> sig;
    auto put = [&](const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        sig.insert(sig.end(), c, c + n);
    };
    put(args.data(), sizeof(EvalArgs) * args.size());
    for (int b = 0; b < count; ++b) {
        const BatchItem& it = items[b];
        TreeState* s = it.tree;
        const void* ptrs[] = {it.t->geo, it.t->srcf, it.t->ljd, it.t->ljf, it.raw, s->code, s->nodes, s->part,
                              s->cell_start, s->far_ent, s->near_ent, s->cp_cnt, s->cp_ent, s->dn_cnt, s->dn_ent,
                              s->tpot, s->tpart, s->tnch, s->tflag, s->cp_work, s->cp_order};
        put(ptrs, sizeof ptrs);
        put(&s->tb, sizeof(TBoxes));
        const int ints[] = {(int)it.t->n, it.t->smax, s->leaf, s->max_nodes, s->max_prox, s->max_items, s->cap_far,
                            s->cap_near, it.lj_mode, s->cap_cp, s->cap_dn};
        put(ints, sizeof ints);
        const double dbl[] = {it.lj_rcut, it.lj_tol};
        put(dbl, sizeof dbl);
        put(it.sig_s, sizeof(double) * kMaxSites);
        put(it.eps_s, sizeof(double) * kMaxSites);
    }
    put(&o, sizeof o);
    BatchCache*& bc = s0->bc;
    cudaError_t e = cudaSuccess;
    if (!bc || bc->sig != sig) {
        delete bc;
        bc = new BatchCache();
        if ((e = cudaMalloc(&bc->d_args, sizeof(EvalArgs) * count)) != cudaSuccess ||
            (e = cudaMalloc(&bc->d_off, sizeof(int) * (count + 1))) != cudaSuccess ||
            (e = cudaMalloc(&bc->d_queue, sizeof(int) * 2)) != cudaSuccess ||
            (e = cudaMalloc(&bc->d_work, sizeof(int) * ((size_t)off[count] + 1))) != cudaSuccess ||
            (e = cudaMalloc(&bc->d_order, sizeof(int) * (2 * (size_t)off[count] + 1))) != cudaSuccess)
            return cuda_err(msg, e, "batch buffers");
        if ((e = cudaMemcpy(bc->d_args, args.data(), sizeof(EvalArgs) * count, cudaMemcpyHostToDevice)) !=
                cudaSuccess ||
            (e = cudaMemcpy(bc->d_off, off.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_err(msg, e, "batch upload");
        if ((e = cudaStreamCreateWithFlags(&bc->cs, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_err(msg, e, "capture stream");
        if ((e = cudaEventCreateWithFlags(&bc->fork, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_err(msg, e, "capture events");
        for (int k = 0; k < BatchCache::kBranches; ++k)
            if ((e = cudaStreamCreateWithFlags(&bc->side[k], cudaStreamNonBlocking)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&bc->join[k], cudaEventDisableTiming)) != cudaSuccess)
                return cuda_err(msg, e, "capture streams");
        cudaStream_t cs = bc->cs;
        if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cuda_err(msg, e, "graph capture");
        rism_status r = RISM_OK;
        // the solutes' preparations are independent: fork them over side streams (parallel graph branches)
        const int nbr = std::min(count, (int)BatchCache::kBranches);
        cudaEventRecord(bc->fork, cs);
        for (int k = 0; k < nbr; ++k) cudaStreamWaitEvent(bc->side[k], bc->fork, 0);
        for (int b = 0; b < count && r == RISM_OK; ++b) {
            BatchItem& it = items[b];
            cudaStream_t bs = bc->side[b % nbr];
            DevTables tt = *it.t;
            if (tt.n > 0) {
                e = launch_setup(it.raw, tt.n, it.ph.S, tt.smax, it.sig_s, it.eps_s, it.lj_mode, it.lj_rcut, it.lj_tol,
                                 it.g, tt, bs);
                if (e != cudaSuccess) r = cuda_err(msg, e, "setup");
            }
            if (r == RISM_OK) r = tree_enqueue(it.tree, tt, it.g, it.ph, o, bs, msg);
            if (r == RISM_OK) cp_enqueue(it.tree, args[b], it.o.h != nullptr, bs);
        }
        for (int k = 0; k < nbr; ++k) {
            cudaEventRecord(bc->join[k], bc->side[k]);
            cudaStreamWaitEvent(cs, bc->join[k], 0);
        }
        if (r == RISM_OK) {
            cudaMemsetAsync(bc->d_queue, 0, sizeof(int) * 2, cs);
            for (int nr = 0; nr < 2; ++nr) {  // global heaviest-first orders over all (solute, batch) items
                k_gather_work<<<count, 256, 0, cs>>>(bc->d_args, bc->d_off, count, nr, bc->d_work);
                k_order<<<1, 1024, 0, cs>>>(off[count], bc->d_work, bc->d_order + (size_t)nr * off[count], nullptr,
                                            nullptr, order_plain(off[count]));
            }
            BatchEval be{bc->d_args, bc->d_off, count, off[count], bc->d_queue, bc->d_order};
            const bool du = items[0].o.u != nullptr, dh = items[0].o.h != nullptr;
            e = dispatch(s0->smax ? s0->smax : items[0].t->smax, variant, 1, du, dh, nullptr, 0, &be, sm_count(), cs);
            if (e != cudaSuccess) r = cuda_err(msg, e, "batched eval");
            for (int b = 0; b < count; ++b)
                cudaMemcpyAsync(items[b].tree->h_meta, items[b].tree->meta, sizeof(TreeMeta), cudaMemcpyDeviceToHost, cs);
        }
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamEndCapture(cs, &graph);
        if (r != RISM_OK) {
            if (graph) cudaGraphDestroy(graph);
            delete bc;
            bc = nullptr;
            return r;
        }
        if (ce != cudaSuccess) {
            delete bc;
            bc = nullptr;
            return cuda_err(msg, ce, "graph capture");
        }
        bc->graph = graph;
        if ((e = cudaGraphInstantiate(&bc->exec, graph, 0)) != cudaSuccess) {
            delete bc;
            bc = nullptr;
            return cuda_err(msg, e, "graph instantiate");
        }
        bc->sig = sig;
        bc->cap = count;
    }
    if ((e = cudaGraphLaunch(bc->exec, st)) != cudaSuccess) return cuda_err(msg, e, "graph launch");
    (void)err;
    return RISM_OK;
}


// ---------------------------------------------------------------- reverse mode: far field over grid boxes
// The far part of dL/dR_i and dL/dq_i is a field of the grid weights W(r) (A1 for 1/d, Ak for e^{-kappa d}/d)
// evaluated, with its gradient, at the atoms: sum_r W(r) K(|r - R_i|).  Transposed to the forward pass, the grid
// boxes become source clusters: a box's (n+1)^3 proxies carry the weights aggregated through its Lagrange basis,
// Q_k = sum_r W(r) L_k(r) (exact level to level, a child's basis reproduces the parent's polynomials), and an
// atom leaf sums Q_k K(|t_k - R_i|) for each box that meets the acceptance criterion, the grid points
// themselves for the level-0 regions that do not.
namespace {

constexpr int kAL = 32;             // atoms per target group (part of one octree leaf) in the reverse far field
constexpr int kADirect = 0x40000000; // entry flag: a level-0 region summed point by point

struct AdjTreeMeta {
    int overflow, need;
};

// Level-0 region -> the proxies of its lowest box with proxies: transposed separable interpolation.
template <int N1>
__global__ void __launch_bounds__(256) k_adj_qregion(TBoxes tb, const float4* __restrict__ w, float2* qpart,
                                                     int* rlow) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    constexpr int M = kTB0, P3 = N1 * N1 * N1;
    const int bi = blockIdx.x;
    const int ib = bi % tb.nbx[0], jb = (bi / tb.nbx[0]) % tb.nby[0], kb = bi / (tb.nbx[0] * tb.nby[0]);
    const TBox R = tbox_at(tb, 0, ib, jb, kb);
    int la = -1;
    TBox A = R;
    for (int l = 0; l < tb.L; ++l) {
        A = tbox_at(tb, l, ib >> l, jb >> l, kb >> l);
        if (A.proxied) {
            la = l;
            break;
        }
    }
    if (threadIdx.x == 0) rlow[bi] = la;
    if (la < 0) return;
    float2* V = reinterpret_cast<float2*>(sm_raw);  // [z][y][x]
    float2* S1 = V + M * M * M;                     // [z][y][kx]
    float2* S2 = S1 + M * M * N1;                   // [z][ky][kx]
    float* W = reinterpret_cast<float*>(S2 + M * N1 * N1);
    const int m0 = R.ext[0], m1 = R.ext[1], m2 = R.ext[2];
    const int64_t plane = (int64_t)tb.ny * tb.nx;
    for (int t = threadIdx.x; t < M * M * M; t += blockDim.x) {
        const int ix = t % M, iy = (t / M) % M, iz = t / (M * M);
        float2 v = make_float2(0.f, 0.f);
        if (ix < m0 && iy < m1 && iz < m2) {
            const float4 q = w[(R.lo[2] + iz) * plane + (int64_t)(R.lo[1] + iy) * tb.nx + R.lo[0] + ix];
            v = make_float2(q.x, q.y);
        }
        V[t] = v;
    }
    const int ms[3] = {m0, m1, m2};
    for (int d = 0; d < 3; ++d) {
        const float off = (float)R.lo[d] - A.c[d];
        basis_rows<N1>(tb, A, d, ms[d], M, [&](int i) { return off + (float)i; }, W + d * M * N1);
    }
    __syncthreads();
    const float *Wx = W, *Wy = W + M * N1, *Wz = W + 2 * M * N1;
    for (int t = threadIdx.x; t < M * M * N1; t += blockDim.x) {
        const int kx = t % N1, yz = t / N1;  // yz = z M + y
        float ax = 0.f, ay = 0.f;
#pragma unroll 4
        for (int x = 0; x < M; ++x) {
            const float wv = Wx[x * N1 + kx];
            const float2 v = V[yz * M + x];
            ax = fmaf(wv, v.x, ax);
            ay = fmaf(wv, v.y, ay);
        }
        S1[t] = make_float2(ax, ay);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < M * N1 * N1; t += blockDim.x) {
        const int kx = t % N1, ky = (t / N1) % N1, z = t / (N1 * N1);
        float ax = 0.f, ay = 0.f;
#pragma unroll 4
        for (int y = 0; y < M; ++y) {
            const float wv = Wy[y * N1 + ky];
            const float2 v = S1[(z * M + y) * N1 + kx];
            ax = fmaf(wv, v.x, ax);
            ay = fmaf(wv, v.y, ay);
        }
        S2[t] = make_float2(ax, ay);
    }
    __syncthreads();
    float2* out = qpart + (int64_t)bi * P3;
    for (int t = threadIdx.x; t < P3; t += blockDim.x) {
        const int kx = t % N1, ky = (t / N1) % N1, kz = t / (N1 * N1);
        float ax = 0.f, ay = 0.f;
#pragma unroll 4
        for (int z = 0; z < M; ++z) {
            const float wv = Wz[z * N1 + kz];
            const float2 v = S2[(z * N1 + ky) * N1 + kx];
            ax = fmaf(wv, v.x, ax);
            ay = fmaf(wv, v.y, ay);
        }
        out[t] = make_float2(ax, ay);
    }
}

// Proxies of the boxes of level l: the regions whose lowest box with proxies this is, plus the transposed
// level-to-level interpolation of every child with proxies (computed by the previous launch).  Fixed order.
template <int N1>
__global__ void __launch_bounds__(256) k_adj_qagg(TBoxes tb, int l, const float2* __restrict__ qpart,
                                                  const int* __restrict__ rlow, float2* qtot) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    constexpr int P3 = N1 * N1 * N1;
    const int bi = blockIdx.x;
    const int ib = bi % tb.nbx[l], jb = (bi / tb.nbx[l]) % tb.nby[l], kb = bi / (tb.nbx[l] * tb.nby[l]);
    const TBox A = tbox_at(tb, l, ib, jb, kb);
    if (!A.proxied) return;
    float2* acc = reinterpret_cast<float2*>(sm_raw);  // [P3]
    float2* V = acc + P3;                             // child proxies
    float2* S1 = V + P3;
    float2* S2 = S1 + P3;
    float* W = reinterpret_cast<float*>(S2 + P3);      // [3][N1][N1]
    for (int k = threadIdx.x; k < P3; k += blockDim.x) acc[k] = make_float2(0.f, 0.f);
    const int sp = 1 << l;
    const int r0x = ib * sp, r0y = jb * sp, r0z = kb * sp;
    const int r1x = min(r0x + sp, tb.nbx[0]), r1y = min(r0y + sp, tb.nby[0]), r1z = min(r0z + sp, tb.nbz[0]);
    for (int rz = r0z; rz < r1z; ++rz)
        for (int ry = r0y; ry < r1y; ++ry)
            for (int rx = r0x; rx < r1x; ++rx) {
                const int rb = (rz * tb.nby[0] + ry) * tb.nbx[0] + rx;
                if (rlow[rb] != l) continue;
                const float2* src = qpart + (int64_t)rb * P3;
                for (int k = threadIdx.x; k < P3; k += blockDim.x) {
                    const float2 v = src[k];
                    acc[k].x += v.x;
                    acc[k].y += v.y;
                }
            }
    __syncthreads();
    if (l > 0) {
        for (int c = 0; c < 8; ++c) {
            const int cx = 2 * ib + (c & 1), cy = 2 * jb + ((c >> 1) & 1), cz = 2 * kb + (c >> 2);
            if (cx >= tb.nbx[l - 1] || cy >= tb.nby[l - 1] || cz >= tb.nbz[l - 1]) continue;
            const TBox C = tbox_at(tb, l - 1, cx, cy, cz);
            if (!C.proxied) continue;
            const float2* src = qtot + (int64_t)tbox_index(tb, l - 1, cx, cy, cz) * P3;
            for (int k = threadIdx.x; k < P3; k += blockDim.x) V[k] = src[k];
            for (int d = 0; d < 3; ++d) {
                const float off = C.c[d] - A.c[d], hd = 0.5f * (C.ext[d] - 1);
                basis_rows<N1>(tb, A, d, N1, N1, [&](int i) { return off + hd * tb.ck[i]; }, W + d * N1 * N1);
            }
            __syncthreads();
            const float *Wx = W, *Wy = W + N1 * N1, *Wz = W + 2 * N1 * N1;
            for (int t = threadIdx.x; t < P3; t += blockDim.x) {  // contract the child's x index
                const int kx = t % N1, yz = t / N1;
                float ax = 0.f, ay = 0.f;
#pragma unroll
                for (int j = 0; j < N1; ++j) {
                    const float wv = Wx[j * N1 + kx];
                    const float2 v = V[yz * N1 + j];
                    ax = fmaf(wv, v.x, ax);
                    ay = fmaf(wv, v.y, ay);
                }
                S1[t] = make_float2(ax, ay);
            }
            __syncthreads();
            for (int t = threadIdx.x; t < P3; t += blockDim.x) {  // the child's y index
                const int kx = t % N1, ky = (t / N1) % N1, z = t / (N1 * N1);
                float ax = 0.f, ay = 0.f;
#pragma unroll
                for (int j = 0; j < N1; ++j) {
                    const float wv = Wy[j * N1 + ky];
                    const float2 v = S1[(z * N1 + j) * N1 + kx];
                    ax = fmaf(wv, v.x, ax);
                    ay = fmaf(wv, v.y, ay);
                }
                S2[t] = make_float2(ax, ay);
            }
            __syncthreads();
            for (int t = threadIdx.x; t < P3; t += blockDim.x) {  // the child's z index
                const int kx = t % N1, ky = (t / N1) % N1, kz = t / (N1 * N1);
                float ax = 0.f, ay = 0.f;
#pragma unroll
                for (int j = 0; j < N1; ++j) {
                    const float wv = Wz[j * N1 + kz];
                    const float2 v = S2[(j * N1 + ky) * N1 + kx];
                    ax = fmaf(wv, v.x, ax);
                    ay = fmaf(wv, v.y, ay);
                }
                acc[t].x += ax;
                acc[t].y += ay;
            }
            __syncthreads();
        }
    }
    float2* dst = qtot + (int64_t)(tb.off[l] + bi) * P3;
    for (int k = threadIdx.x; k < P3; k += blockDim.x) dst[k] = acc[k];
}

// Reverse-mode targets (one CTA): every octree leaf split into groups of at most kAL consecutive atoms, in node
// order; grp[g] = (first atom, count), *count = the number of groups.
__global__ void __launch_bounds__(1024) k_leaf_list(const TreeMeta* meta, const Node* __restrict__ nodes, int2* grp,
                                                    int* count) {
    __shared__ int tmp[64];
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const int nn = meta->nnodes;
    for (int b0 = 0; b0 < nn; b0 += blockDim.x) {
        const int nid = b0 + threadIdx.x;
        int ng = 0, nb = 0, ne = 0;
        if (nid < nn) {
            const Node nd = nodes[nid];
            if (nd.first_child < 0) {
                nb = nd.begin;
                ne = nd.end;
                ng = (ne - nb + kAL - 1) / kAL;
            }
        }
        int tot;
        const int off = block_exclusive_scan(ng, tmp, tot);
        for (int q = 0; q < ng; ++q) grp[base + off + q] = make_int2(nb + q * kAL, min(kAL, ne - nb - q * kAL));
        __syncthreads();
        if (threadIdx.x == 0) base += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base;
}

// Interaction lists of the atom leaves (one warp per leaf): the grid-box hierarchy from the top; a box with
// proxies that meets (r_leaf + r_box)/R < theta is accepted, another box is opened, a level-0 region that is
// not accepted is summed point by point.  Order: frontier round, then lane -- deterministic.
__global__ void __launch_bounds__(32 * kListWarps) k_adj_lists(TBoxes tb, const SrcF* __restrict__ ssrcf,
                                                              const int2* __restrict__ grp,
                                                              const int* __restrict__ nleaf_p, float theta, int cap,
                                                              int* cnt, int* ent, AdjTreeMeta* meta) {
    __shared__ int qa[kListWarps][kQCap], qb[kListWarps][kQCap];
    const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5;
    const int nleaf = *nleaf_p;
    const float th2 = theta * theta;
    for (int leaf = blockIdx.x * kListWarps + wv; leaf < nleaf; leaf += gridDim.x * kListWarps) {
        const int2 gr = grp[leaf];  // a group of consecutive atoms of one octree leaf: a compact box
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        if (lane < gr.y) {
            const SrcF sf = ssrcf[gr.x + lane];
            lo[0] = hi[0] = sf.xh;
            lo[1] = hi[1] = sf.yh;
            lo[2] = hi[2] = sf.zh;
        }
        float c[3], r2 = 0.f;
        for (int d = 0; d < 3; ++d) {
            for (int o = 16; o > 0; o >>= 1) {
                lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
                hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
            }
            c[d] = 0.5f * (lo[d] + hi[d]);
            r2 += 0.25f * (hi[d] - lo[d]) * (hi[d] - lo[d]);
        }
        const float rl = sqrtf(r2) + 0.01f;  // slack for the low parts of the positions
        int* cur = qa[wv];
        int* nxt = qb[wv];
        const int Lt = tb.L - 1;
        const int ntop = tb.nbx[Lt] * tb.nby[Lt] * tb.nbz[Lt];
        bool ovf = ntop > kQCap;
        for (int k = lane; k < min(ntop, kQCap); k += 32) cur[k] = tb.off[Lt] + k;
        __syncwarp();
        int ncur = min(ntop, kQCap), m = 0;
        int* out = ent + (int64_t)leaf * cap;
        while (ncur > 0 && !__any_sync(0xffffffffu, ovf)) {
            int nnext = 0;
            for (int c0 = 0; c0 < ncur; c0 += 32) {
                const int k = c0 + lane;
                int kind = 0, e = 0, nch = 0;
                int chl = 0, cx0 = 0, cy0 = 0, cz0 = 0;
                if (k < ncur) {
                    const TBox T = tbox_flat(tb, cur[k]);
                    float R2 = 0.f;
                    for (int d = 0; d < 3; ++d) R2 += (c[d] - (float)T.c[d]) * (c[d] - (float)T.c[d]);
                    const float rs = rl + (float)T.r;
                    if (T.proxied && rs * rs < th2 * R2) {
                        kind = 1;
                        e = cur[k];
                    } else if (T.l > 0) {
                        kind = 2;
                        chl = T.l - 1;
                        cx0 = 2 * T.ib;
                        cy0 = 2 * T.jb;
                        cz0 = 2 * T.kb;
                        nch = 0;
                        for (int q = 0; q < 8; ++q)
                            nch += (cx0 + (q & 1) < tb.nbx[chl] && cy0 + ((q >> 1) & 1) < tb.nby[chl] &&
                                    cz0 + (q >> 2) < tb.nbz[chl]);
                    } else {
                        kind = 1;
                        e = cur[k] | kADirect;
                    }
                }
                const unsigned em = __ballot_sync(0xffffffffu, kind == 1);
                if (kind == 1) {
                    const int pos = m + __popc(em & ((1u << lane) - 1u));
                    if (pos < cap) out[pos] = e;
                }
                m += __popc(em);
                int x = nch;
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                const int tot = __shfl_sync(0xffffffffu, x, 31);
                int at = nnext + x - nch;
                if (kind == 2) {
                    for (int q = 0; q < 8; ++q) {
                        const int cx = cx0 + (q & 1), cy = cy0 + ((q >> 1) & 1), cz = cz0 + (q >> 2);
                        if (cx >= tb.nbx[chl] || cy >= tb.nby[chl] || cz >= tb.nbz[chl]) continue;
                        if (at < kQCap) nxt[at] = tbox_index(tb, chl, cx, cy, cz);
                        else ovf = true;
                        ++at;
                    }
                }
                nnext += tot;
            }
            __syncwarp();
            int* tq = cur;
            cur = nxt;
            nxt = tq;
            ncur = min(nnext, kQCap);
            if (nnext > kQCap) ovf = true;
            __syncwarp();
        }
        const bool wide = __any_sync(0xffffffffu, ovf);
        if (lane == 0) {
            cnt[leaf] = min(m, cap);
            if (wide || m > cap) {
                meta->overflow = 1;
                atomicMax(&meta->need, wide ? (1 << 30) : m);
            }
        }
    }
}

constexpr int kADThreads = 128;  // 4 threads per atom of a leaf
constexpr int kADSub = kADThreads / kAL;

// One pair of the reverse far field: potential and radial factor of W1/d + Wk e^{-kappa d}/d.
template <bool DH>
__device__ __forceinline__ void adj_pair(float dx, float dy, float dz, float w1, float wk, float kap2, float kapg,
                                         float& pq, float& px, float& py, float& pz) {
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float rr = rsqrt_approx(d2);
    const float ri = d2 > 0.f ? rr : 0.f;  // a grid point on the atom: no term (d = 0 has no gradient)
    float t1 = w1 * ri, tg = t1;
    if (DH) {
        const float d = d2 * ri;
        const float tk = wk * ri * ex2_approx(kap2 * d);
        t1 += tk;
        tg = fmaf(tk, kapg * d, t1);
    }
    pq += t1;
    const float rad = tg * ri * ri;
    px = fmaf(dx, rad, px);
    py = fmaf(dy, rad, py);
    pz = fmaf(dz, rad, pz);
}

// One group of up to kAL atoms of a leaf (kADSub threads per atom, consecutive lanes) against the leaf's list.
template <bool DH>
__device__ void adj_leaf_group(const TBoxes& tb, const SrcF* __restrict__ ssrcf, const uint32_t* __restrict__ idx,
                               const float4* __restrict__ w, const float2* __restrict__ qtot,
                               const int* __restrict__ cnt, const int* __restrict__ ent, int cap, float kap2,
                               float kapg, double* part, float2* Q, int leaf, int j, bool act, int tid, int sub) {
    const SrcF sf = act ? ssrcf[j] : SrcF{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const int n1 = tb.deg + 1, P3 = tb.P3;
    float h[4] = {0.f, 0.f, 0.f, 0.f}, lo4[4] = {0.f, 0.f, 0.f, 0.f};
    const int ne = cnt[leaf];
    const int64_t plane = (int64_t)tb.ny * tb.nx;
    // proxy offsets from the box centre and the A1 weight (16-byte aligned after the even-sized Q array)
    float4* Pc = reinterpret_cast<float4*>(Q + ((P3 + 1) & ~1));
    for (int e = 0; e < ne; ++e) {
        const int code = ent[(int64_t)leaf * cap + e];
        float pq = 0.f, px = 0.f, py = 0.f, pz = 0.f;
        if (!(code & kADirect)) {
            const TBox T = tbox_flat(tb, code);
            const float hx = 0.5f * (T.ext[0] - 1), hy = 0.5f * (T.ext[1] - 1), hz = 0.5f * (T.ext[2] - 1);
            __syncthreads();
            const float2* src = qtot + (int64_t)code * P3;
            for (int k = tid; k < P3; k += kADThreads) {
                const int kx = k % n1, ky = (k / n1) % n1, kz = k / (n1 * n1);
                const float2 q = src[k];
                Q[k] = q;
                Pc[k] = make_float4(hx * tb.ck[kx], hy * tb.ck[ky], hz * tb.ck[kz], q.x);
            }
            __syncthreads();
            // atom relative to the box centre
            const float ax = (sf.xh - (float)T.c[0]) + sf.xl, ay = (sf.yh - (float)T.c[1]) + sf.yl,
                        az = (sf.zh - (float)T.c[2]) + sf.zl;
            for (int k = sub; k < P3; k += kADSub) {
                const float4 pc = Pc[k];
                adj_pair<DH>(pc.x - ax, pc.y - ay, pc.z - az, pc.w, DH ? Q[k].y : 0.f, kap2, kapg, pq, px, py, pz);
            }
        } else {
            const TBox R = tbox_flat(tb, code & ~kADirect);
            const int m0 = R.ext[0], m1 = R.ext[1], m2 = R.ext[2];
            // lattice point minus the atom: exact first subtraction for nearby atoms
            for (int iz = 0; iz < m2; ++iz) {
                const int gz = R.lo[2] + iz;
                const float dz = ((float)gz - sf.zh) - sf.zl;
                for (int iy = 0; iy < m1; ++iy) {
                    const int gy = R.lo[1] + iy;
                    const float dy = ((float)gy - sf.yh) - sf.yl;
                    const float4* row = w + gz * plane + (int64_t)gy * tb.nx + R.lo[0];
                    for (int ix = sub; ix < m0; ix += kADSub) {
                        const float4 wv = row[ix];
                        adj_pair<DH>(((float)(R.lo[0] + ix) - sf.xh) - sf.xl, dy, dz, wv.x, wv.y, kap2, kapg, pq,
                                     px, py, pz);
                    }
                }
            }
        }
        ff_add(h[0], lo4[0], pq);
        ff_add(h[1], lo4[1], px);
        ff_add(h[2], lo4[2], py);
        ff_add(h[3], lo4[3], pz);
    }
    // the kADSub threads of an atom are consecutive lanes: combine them in a fixed order
    double v[4];
    for (int q = 0; q < 4; ++q) {
        v[q] = (double)h[q] + (double)lo4[q];
        for (int o = 1; o < kADSub; o <<= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    }
    if (act && sub == 0) {
        double* o = part + (int64_t)idx[j] * 4;
        for (int q = 0; q < 4; ++q) o[q] = v[q];
    }
}

template <bool DH>
__global__ void __launch_bounds__(kADThreads) k_adj_treefar(TBoxes tb, const SrcF* __restrict__ ssrcf,
                                                           const uint32_t* __restrict__ idx,
                                                           const int2* __restrict__ grp,
                                                           const int* __restrict__ nleaf_p,
                                                           const float4* __restrict__ w,
                                                           const float2* __restrict__ qtot, const int* __restrict__ cnt,
                                                           const int* __restrict__ ent, int cap, float kap2,
                                                           float kapg, const AdjTreeMeta* meta, double* part) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    float2* Q = reinterpret_cast<float2*>(sm_raw);  // one box's proxies
    if (meta->overflow || blockIdx.x >= *nleaf_p) return;
    const int leaf = blockIdx.x, tid = threadIdx.x, a = tid / kADSub, sub = tid % kADSub;
    const int2 gr = grp[leaf];
    adj_leaf_group<DH>(tb, ssrcf, idx, w, qtot, cnt, ent, cap, kap2, kapg, part, Q, leaf, gr.x + a, a < gr.y, tid,
                       sub);
}

template <int N1>
void launch_adj_q(const TBoxes& tb, const float4* w, float2* qpart, int* rlow, float2* qtot, cudaStream_t st) {
    constexpr int M = kTB0, P3 = N1 * N1 * N1;
    const size_t sr = sizeof(float2) * (M * M * M + M * M * N1 + M * N1 * N1) + sizeof(float) * 3 * M * N1;
    const size_t sa = sizeof(float2) * 4 * P3 + sizeof(float) * 3 * N1 * N1;
    raise_dyn_smem(k_adj_qregion<N1>, sr);
    raise_dyn_smem(k_adj_qagg<N1>, sa);
    k_adj_qregion<N1><<<tb.nbx[0] * tb.nby[0] * tb.nbz[0], 256, sr, st>>>(tb, w, qpart, rlow);
    for (int l = 0; l < tb.L; ++l)
        k_adj_qagg<N1><<<tb.nbx[l] * tb.nby[l] * tb.nbz[l], 256, sa, st>>>(tb, l, qpart, rlow, qtot);
}

void launch_adj_q_deg(const TBoxes& tb, const float4* w, float2* qpart, int* rlow, float2* qtot, cudaStream_t st) {
    switch (tb.deg) {
        case 1: return launch_adj_q<2>(tb, w, qpart, rlow, qtot, st);
        case 2: return launch_adj_q<3>(tb, w, qpart, rlow, qtot, st);
        case 3: return launch_adj_q<4>(tb, w, qpart, rlow, qtot, st);
        case 4: return launch_adj_q<5>(tb, w, qpart, rlow, qtot, st);
        case 5: return launch_adj_q<6>(tb, w, qpart, rlow, qtot, st);
        case 6: return launch_adj_q<7>(tb, w, qpart, rlow, qtot, st);
        case 7: return launch_adj_q<8>(tb, w, qpart, rlow, qtot, st);
        case 8: return launch_adj_q<9>(tb, w, qpart, rlow, qtot, st);
        case 9: return launch_adj_q<10>(tb, w, qpart, rlow, qtot, st);
        case 10: return launch_adj_q<11>(tb, w, qpart, rlow, qtot, st);
        case 11: return launch_adj_q<12>(tb, w, qpart, rlow, qtot, st);
        default: return launch_adj_q<13>(tb, w, qpart, rlow, qtot, st);
    }
}

}  // namespace

struct AdjTree {
    float2 *qpart = nullptr, *qtot = nullptr;
    int* rlow = nullptr;
    int2* grp = nullptr;  // reverse-mode targets: (first atom, count) of each group of an octree leaf
    int* nleaf = nullptr;
    int64_t cap_grp = 0;
    int64_t cap_qpart = 0, cap_qtot = 0, cap_rlow = 0;
    int *cnt = nullptr, *ent = nullptr;
    int cap = 256, cap_leaf = 0;
    int64_t cap_ent = 0;
    AdjTreeMeta *meta = nullptr, *h_meta = nullptr;
    ~AdjTree() {
        cudaFree(qpart);
        cudaFree(qtot);
        cudaFree(rlow);
        cudaFree(grp);
        cudaFree(nleaf);
        cudaFree(cnt);
        cudaFree(ent);
        cudaFree(meta);
        cudaFreeHost(h_meta);
    }
};

void adjtree_delete(AdjTree* a) { delete a; }

const uint32_t* tree_atom_order(TreeState* s) { return (s && s->prepared) ? s->idx : nullptr; }

rism_status tree_adjoint_far(TreeState* s, const DevTables& t, const GridD& g, const Phys& ph, const rism_options& o,
                             const float4* w, bool dh, double* part, cudaStream_t st, std::string& err, bool& used) {
    used = false;
    const TBoxes& tb = s->tb;
    const int n = (int)t.n;
    // the transposed far field uses the Chebyshev proxies; with Taylor moments the caller's direct reverse
    // far part runs instead
    if (!tb.enabled || tb.approx != RISM_APPROX_BARYCENTRIC || !s->prepared || n == 0) return RISM_OK;
    if (!s->adj) s->adj = new AdjTree();
    AdjTree& A = *s->adj;
    cudaError_t e;
    const int nb0 = tb.nbx[0] * tb.nby[0] * tb.nbz[0];
    // upper bound of the target groups: every leaf adds at most one partial group (the count stays on the device)
    const int nleaf = n / kAL + s->max_nodes + 1;
    auto grow = [&](auto*& p, int64_t& cap, int64_t need) -> cudaError_t {
        if (need <= cap) return cudaSuccess;
        cudaFree(p);
        p = nullptr;
        cap = 0;
        cudaError_t r = cudaMalloc(&p, sizeof(*p) * (size_t)need);
        if (r == cudaSuccess) cap = need;
        return r;
    };
    if ((e = grow(A.qpart, A.cap_qpart, (int64_t)nb0 * tb.P3)) != cudaSuccess ||
        (e = grow(A.qtot, A.cap_qtot, (int64_t)tb.nbox * tb.P3)) != cudaSuccess ||
        (e = grow(A.rlow, A.cap_rlow, (int64_t)nb0)) != cudaSuccess)
        return cuda_err(err, e, "reverse-mode box buffers");
    if (!A.meta) {
        if ((e = cudaMalloc(&A.meta, sizeof(AdjTreeMeta))) != cudaSuccess ||
            (e = cudaMallocHost(&A.h_meta, sizeof(AdjTreeMeta))) != cudaSuccess ||
            (e = cudaMalloc(&A.nleaf, sizeof(int))) != cudaSuccess)
            return cuda_err(err, e, "reverse-mode meta");
    }
    if ((e = grow(A.grp, A.cap_grp, (int64_t)nleaf + 1)) != cudaSuccess)
        return cuda_err(err, e, "reverse-mode leaves");
    k_leaf_list<<<1, 1024, 0, st>>>(s->meta, s->nodes, A.grp, A.nleaf);
    launch_adj_q_deg(tb, w, A.qpart, A.rlow, A.qtot, st);
    const size_t sq = sizeof(float2) * ((tb.P3 + 1) & ~1) + sizeof(float4) * tb.P3;
    for (int attempt = 0; attempt < 4; ++attempt) {
        if (nleaf + 1 > A.cap_leaf) {
            cudaFree(A.cnt);
            A.cnt = nullptr;
            if ((e = cudaMalloc(&A.cnt, sizeof(int) * (nleaf + 1))) != cudaSuccess) return cuda_err(err, e, "lists");
            A.cap_leaf = nleaf + 1;
        }
        if ((e = grow(A.ent, A.cap_ent, (int64_t)nleaf * A.cap)) != cudaSuccess) return cuda_err(err, e, "lists");
        cudaMemsetAsync(A.meta, 0, sizeof(AdjTreeMeta), st);
        k_adj_lists<<<(nleaf + kListWarps - 1) / kListWarps, 32 * kListWarps, 0, st>>>(
            tb, s->srcf, A.grp, A.nleaf, (float)o.theta, A.cap, A.cnt, A.ent, A.meta);
        const float kap2 = (float)(-ph.kappa * g.h * 1.4426950408889634), kapg = (float)(ph.kappa * g.h);
        if (dh)
            k_adj_treefar<true><<<nleaf, kADThreads, sq, st>>>(tb, s->srcf, s->idx, A.grp, A.nleaf, w, A.qtot, A.cnt,
                                                               A.ent, A.cap, kap2, kapg, A.meta, part);
        else
            k_adj_treefar<false><<<nleaf, kADThreads, sq, st>>>(tb, s->srcf, s->idx, A.grp, A.nleaf, w, A.qtot,
                                                                A.cnt, A.ent, A.cap, kap2, kapg, A.meta, part);
        if ((e = cudaMemcpyAsync(A.h_meta, A.meta, sizeof(AdjTreeMeta), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_err(err, e, "reverse-mode lists");
        if (!A.h_meta->overflow) {
            used = true;
            return RISM_OK;
        }
        if (A.h_meta->need >= (1 << 30)) {
            err = "a reverse-mode traversal frontier exceeded 2048 boxes";
            return RISM_E_NOMEM;
        }
        int p2 = 1;
        while (p2 < A.h_meta->need) p2 <<= 1;
        A.cap = p2;
    }
    err = "reverse-mode list slots kept growing";
    return RISM_E_NOMEM;
}

}  // namespace rism
