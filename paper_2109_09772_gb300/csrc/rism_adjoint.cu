// rism_adjoint.cu -- reverse mode of the initialization grids.
//
// L = sum_s sum_r [G_u,s(r) u_s(r) + G_c,s(r) c_s(r) + G_h,s(r) h_s(r)] with u,
// c, h as defined in rism3d.h (Coulomb + truncated LJ, eq. (dcf-r),
// eq. (tcf-r)).  The paper has no gradient; these are the derivatives of
// those definitions.  Pair terms are recomputed, never stored.
//
// Site contraction first (per grid point, FP64 inputs):
//   W1 = k_e sum_s q_s G_u,s          (Coulomb part of u)
//   Wc = -beta k_e sum_s q_s G_c,s    (c)
//   Wh = -(beta k_e/(2 eps_r)) sum_s q_s G_h,s   (h)
// The long-range kernels split exactly as in the forward pass:
//   erf(x)/d = 1/d - erfc(x)/d,
//   phi_h(d) = 2 e^{a^2} e^{-kappa d}/d - Sh(d),
//   Sh(d) = e^{a^2}[e^{-kappa d} erfc(x-a) + e^{kappa d} erfc(x+a)]/d,
// so the far adjoint needs A1 = W1 + Wc (coefficient of 1/d) and
// Ak = 2 e^{a^2} Wh (coefficient of e^{-kappa d}/d) for every (point, atom)
// pair, and the near adjoint adds the erfc corrections within r_short and
// the LJ terms within the cut-offs.
//
//   k_adj_weights: W fields (float4 per point: A1, Ak, Wc, Wh; FP32)
//   k_adj_far:     atoms as targets (2 per thread), grid rows streamed through
//                  shared memory by bulk TMA copies; partials per row chunk
//   k_adj_near:    one CTA per atom over the grid points of its cut-off box
//   k_adj_final:   fixed-order sum of the partials, output in FP64
#include <cmath>

#include "rism_adjoint.h"
#include "rism_tree.h"

namespace rism {
namespace {

constexpr int kAT = 128;     // threads per far-adjoint CTA
constexpr int kAPT = 2;      // atoms per thread
constexpr int kRowT = 64;    // grid points per shared-memory tile (a row segment)
constexpr int kNearT = 256;  // threads per near-adjoint CTA

__global__ void k_adj_weights(int64_t M, int S, const double* __restrict__ gu, const double* __restrict__ gc,
                              const double* __restrict__ gh, Phys ph, float4* w, float4* gu4) {
    const double c1 = ph.k_e, cc = -ph.beta * ph.k_e, chh = -ph.beta * ph.k_e / (2.0 * ph.eps_r);
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < M; f += (int64_t)gridDim.x * blockDim.x) {
        double a = 0.0, b = 0.0, h = 0.0;
        float g8[kMaxSites] = {};
        for (int s = 0; s < S; ++s) {
            const double qs = ph.qs[s];
            if (gu) {
                const double v = gu[s * M + f];
                a += qs * v;
                g8[s] = (float)v;
            }
            if (gc) b += qs * gc[s * M + f];
            if (gh) h += qs * gh[s * M + f];
        }
        if (gu) {
            gu4[f] = make_float4(g8[0], g8[1], g8[2], g8[3]);
            if (S > 4) gu4[M + f] = make_float4(g8[4], g8[5], g8[6], g8[7]);
        }
        const double W1 = c1 * a, Wc = cc * b, Wh = chh * h;
        w[f] = make_float4((float)(W1 + Wc), (float)(2.0 * ph.ea2 * Wh), (float)Wc, (float)Wh);
    }
}

struct FarAdjArgs {
    int nx, ny, nz;
    int n;
    int seg_per_row, nseg;   // row segments of kRowT points
    int chunks;              // grid chunks (partials per atom)
    float kap_g;             // kappa in 1/grid units
    float kap2;              // -kappa h log2(e): e^{-kappa d} = 2^(kap2 d_grid)
    const SrcF* srcf;
    const float4* w;
    double* part;            // [chunks][n][4]: dq, Gx, Gy, Gz (grid units)
    DevErr* err;
    long long wlim;
};

// Atoms as targets, grid points as sources.  Row segments of kRowT points are
// contiguous in the W array, so one bulk copy brings a tile; y and z are
// constant along it and x advances by one grid unit per point.
template <bool DH>
__global__ void __launch_bounds__(kAT) k_adj_far(FarAdjArgs a) {
    __shared__ __align__(16) float4 tile[2][kRowT];
    __shared__ __align__(8) uint64_t bar[2];
    const int tid = threadIdx.x;
    const int chunk = blockIdx.y;
    const int s0 = (int)((int64_t)a.nseg * chunk / a.chunks), s1 = (int)((int64_t)a.nseg * (chunk + 1) / a.chunks);
    float xh[kAPT], yh[kAPT], zh[kAPT], xl[kAPT], yl[kAPT], zl[kAPT];
    float dqh[kAPT], dql[kAPT], gxh[kAPT], gxl[kAPT], gyh[kAPT], gyl[kAPT], gzh[kAPT], gzl[kAPT];
    int atom[kAPT];
#pragma unroll
    for (int u = 0; u < kAPT; ++u) {
        atom[u] = (blockIdx.x * kAPT + u) * kAT + tid;
        const SrcF s = atom[u] < a.n ? a.srcf[atom[u]] : SrcF{1e30f, 1e30f, 1e30f, 0.f, 0.f, 0.f, 0.f, 0.f};
        xh[u] = s.xh; yh[u] = s.yh; zh[u] = s.zh;
        xl[u] = s.xl; yl[u] = s.yl; zl[u] = s.zl;
        dqh[u] = dql[u] = gxh[u] = gxl[u] = gyh[u] = gyl[u] = gzh[u] = gzl[u] = 0.f;
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const int nt = s1 - s0;
    auto seg_len = [&](int sg) {
        const int within = sg % a.seg_per_row;
        return min(kRowT, a.nx - within * kRowT);
    };
    auto issue = [&](int t) {
        const int sg = s0 + t;
        const int row = sg / a.seg_per_row, within = sg % a.seg_per_row;
        const int len = seg_len(sg);
        const uint32_t bytes = len * sizeof(float4);
        mbar_expect_tx(&bar[t & 1], bytes);
        bulk_g2s(tile[t & 1], a.w + (int64_t)row * a.nx + within * kRowT, bytes, &bar[t & 1]);
    };
    if (tid == 0) {
        if (nt > 0) issue(0);
        if (nt > 1) issue(1);
    }
    for (int t = 0; t < nt; ++t) {
        const bool ok = mbar_wait_bounded(&bar[t & 1], (t >> 1) & 1, a.wlim);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                report_error(a.err, DEV_TIMEOUT, WHERE_ADJOINT);
                for (int u2 = t; u2 < min(t + 2, nt); ++u2) mbar_wait_bounded(&bar[u2 & 1], (u2 >> 1) & 1, a.wlim);
            }
            return;
        }
        const int sg = s0 + t;
        const int row = sg / a.seg_per_row, within = sg % a.seg_per_row;
        const int len = seg_len(sg);
        const float fy = (float)(row % a.ny), fz = (float)(row / a.ny);
        const float fx0 = (float)(within * kRowT);
        const float4* W = tile[t & 1];
        float dy[kAPT], dz[kAPT], dyz2[kAPT], pq[kAPT], px[kAPT], pyz[kAPT];
#pragma unroll
        for (int u = 0; u < kAPT; ++u) {
            dy[u] = (fy - yh[u]) - yl[u];
            dz[u] = (fz - zh[u]) - zl[u];
            dyz2[u] = fmaf(dy[u], dy[u], dz[u] * dz[u]);
            pq[u] = px[u] = pyz[u] = 0.f;
        }
        float fx = fx0;
        for (int p = 0; p < len; ++p, fx += 1.0f) {
            const float4 wv = W[p];
#pragma unroll
            for (int u = 0; u < kAPT; ++u) {
                const float dx = (fx - xh[u]) - xl[u];
                const float d2 = fmaf(dx, dx, dyz2[u]);
                const float rr = rsqrt_approx(d2);
                const float ri = d2 > 0.f ? rr : 0.f;
                const float ri2 = ri * ri;
                float t1 = wv.x * ri, tg = t1;
                if (DH) {
                    const float d = d2 * ri;
                    const float tk = wv.y * ri * ex2_approx(a.kap2 * d);
                    t1 += tk;
                    tg = fmaf(tk, a.kap_g * d, t1);
                }
                pq[u] += t1;
                const float rad = tg * ri2;
                px[u] = fmaf(dx, rad, px[u]);
                pyz[u] += rad;  // (dy, dz) are constant along the row
            }
        }
#pragma unroll
        for (int u = 0; u < kAPT; ++u) {
            ff_add(dqh[u], dql[u], pq[u]);
            ff_add(gxh[u], gxl[u], px[u]);
            ff_add(gyh[u], gyl[u], dy[u] * pyz[u]);
            ff_add(gzh[u], gzl[u], dz[u] * pyz[u]);
        }
        __syncthreads();
        if (tid == 0 && t + 2 < nt) issue(t + 2);
    }
#pragma unroll
    for (int u = 0; u < kAPT; ++u) {
        if (atom[u] >= a.n) continue;
        double* o = a.part + ((int64_t)chunk * a.n + atom[u]) * 4;
        o[0] = (double)dqh[u] + (double)dql[u];
        o[1] = (double)gxh[u] + (double)gxl[u];
        o[2] = (double)gyh[u] + (double)gyl[u];
        o[3] = (double)gzh[u] + (double)gzl[u];
    }
}

struct NearAdjArgs {
    GridD g;
    Phys ph;
    int n, S, smax;
    const double* raw;       // [n][6] x, y, z, q, sigma, eps (physical)
    const SrcF* srcf;
    const LJf* ljf;          // [n][smax] grid units
    const float4* w;
    const float4* gu4;       // [ceil(S/4)][M]: G_u of the sites in FP32, four per record (nullable)
    const uint32_t* order;   // CTA -> atom (Morton order from the tree, for cache reuse); null: identity
    double sig_s[kMaxSites], eps_s[kMaxSites];
    double rnear;            // max cut-off / r_short (A); infinite = whole grid
    double* out;             // [n][6]: dq, Gx, Gy, Gz (grid units as in the far part), dLJ/dR (3), ...
};

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    return s;
}

// One CTA per atom: grid points within rnear of the atom.  Accumulates, in
// grid units, the erfc corrections (dq, G) and the LJ terms: the radial
// factor sum G_u,s dLJ/dd / d (-> dR), dLJ/dsigma_i and dLJ/deps_i.
__global__ void __launch_bounds__(kNearT) k_adj_near(NearAdjArgs a) {
    __shared__ double red[kNearT / 32];
    if ((int)blockIdx.x >= a.n) return;
    const int i = a.order ? (int)a.order[blockIdx.x] : (int)blockIdx.x;
    const GridD& g = a.g;
    const int64_t M = (int64_t)g.nx * g.ny * g.nz;
    const SrcF sf = a.srcf[i];
    const double ux = (double)sf.xh + sf.xl, uy = (double)sf.yh + sf.yl, uz = (double)sf.zh + sf.zl;
    const double rn = a.rnear / g.h;  // grid units
    int lo[3], hi[3];
    const double uc[3] = {ux, uy, uz};
    const int nn[3] = {g.nx, g.ny, g.nz};
    for (int d = 0; d < 3; ++d) {
        lo[d] = isfinite(rn) ? max(0, (int)ceil(uc[d] - rn)) : 0;
        hi[d] = isfinite(rn) ? min(nn[d] - 1, (int)floor(uc[d] + rn)) : nn[d] - 1;
    }
    const double sg_i = a.raw[6 * i + 4], ep_i = a.raw[6 * i + 5];
    const float rs2 = (float)((a.ph.rs / g.h) * (a.ph.rs / g.h));
    const float xs = (float)(g.h / a.ph.eta);
    const float aa = (float)a.ph.a, kap_g = (float)(a.ph.kappa * g.h);
    const float c2 = (float)(4.0 / (a.ph.eta * sqrt(M_PI)) * g.h);  // 2 * (2/(eta sqrt pi)) in grid units
    const float c1 = 0.5f * c2;
    const float rn2 = isfinite(rn) ? (float)(rn * rn) : INFINITY;
    float Ls[kMaxSites], Bs[kMaxSites], Rc[kMaxSites], isg[kMaxSites], kep[kMaxSites];
    for (int s = 0; s < kMaxSites; ++s) {
        if (s < a.S) {
            const LJf l = a.ljf[(int64_t)i * a.smax + s];
            Ls[s] = l.A;
            Bs[s] = l.B;
            Rc[s] = l.rc2;
            const double sig = 0.5 * (sg_i + a.sig_s[s]);
            const double eps = sqrt(ep_i * a.eps_s[s]);
            isg[s] = sig > 0.0 ? (float)(0.5 / sig) : 0.f;                        // dsigma_is/dsigma_i / sigma_is
            kep[s] = eps > 0.0 ? (float)(a.eps_s[s] / (2.0 * eps * eps)) : 0.f;   // (deps_is/deps_i) / eps_is
        } else {
            Ls[s] = Bs[s] = Rc[s] = isg[s] = kep[s] = 0.f;
        }
    }
    const int bx = hi[0] - lo[0] + 1, by = hi[1] - lo[1] + 1, bz = hi[2] - lo[2] + 1;
    const int nplane = (bx > 0 && by > 0 && bz > 0) ? bx * by : 0;
    float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // dq, Gx, Gy, Gz, LJx, LJy, LJz, dsig, deps
    float hi9[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, lo9[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int cntp = 0;
    // threads over the (x, y) columns of the box (one 32-bit division each); z runs over the column's chord of
    // the near sphere (one grid unit of margin; the exact test below decides)
    for (int b = threadIdx.x; b < nplane; b += blockDim.x) {
    const int ii = lo[0] + b % bx, jj = lo[1] + b / bx;
    const float dx = ((float)ii - sf.xh) - sf.xl, dy = ((float)jj - sf.yh) - sf.yl;
    int k0 = lo[2], k1 = hi[2];
    if (isfinite(rn2)) {
        const float rem = rn2 - fmaf(dx, dx, dy * dy);
        if (rem < 0.f) continue;
        const float hz = sqrtf(rem) + 1.0f;
        k0 = max(k0, (int)floorf(sf.zh - hz));
        k1 = min(k1, (int)ceilf(sf.zh + hz));
    }
    for (int kk = k0; kk <= k1; ++kk) {
        const float dz = ((float)kk - sf.zh) - sf.zl;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (d2 >= rn2 || d2 == 0.f) continue;
        const int64_t f = ((int64_t)kk * g.ny + jj) * g.nx + ii;
        const float ri = rsqrt_approx(d2);
        float rad = 0.f, dq = 0.f;
        if (d2 < rs2) {
            const float4 wv = a.w[f];
            const float x = d2 * ri * xs, d = d2 * ri;
            const float ex2m = __expf(-x * x);
            // c: -Wc Sc(d), Sc = erfc(x)/d, Sc' = -(2/(eta sqrt pi)) e^{-x^2}/d - Sc/d
            const float Sc = erfcf(x) * ri;
            const float Scp = -(c1 * ex2m) * ri - Sc * ri;
            dq -= wv.z * Sc;
            rad -= wv.z * Scp * ri;
            if (wv.w != 0.f) {
                // h: -Wh Sh(d), Sh = e^{-x^2}[erfcx(x-a) + erfcx(x+a)]/d,
                // Sh' = [kappa e^{-x^2}(erfcx(x+a) - erfcx(x-a)) - (4/(eta sqrt pi)) e^{-x^2}]/d - Sh/d
                const float em = erfcxf(x - aa), ep = erfcxf(x + aa);
                const float Sh = ex2m * (em + ep) * ri;
                const float Shp = (kap_g * ex2m * (ep - em) - c2 * ex2m) * ri - Sh * ri;
                dq -= wv.w * Sh;
                rad -= wv.w * Shp * ri;
            }
            (void)d;
        }
        acc[0] += dq;
        acc[1] = fmaf(dx, rad, acc[1]);
        acc[2] = fmaf(dy, rad, acc[2]);
        acc[3] = fmaf(dz, rad, acc[3]);
        if (a.gu4) {
            const float r2i = rcp_approx(d2);
            const float r6 = r2i * r2i * r2i, r12 = r6 * r6;
            float lrad = 0.f, ds = 0.f, de = 0.f;
            float4 g4 = a.gu4[f];
            for (int s = 0; s < a.S; ++s) {
                if (s == 4) g4 = a.gu4[M + f];
                const int c4 = s & 3;
                const float G = c4 == 0 ? g4.x : (c4 == 1 ? g4.y : (c4 == 2 ? g4.z : g4.w));
                if (!(d2 < Rc[s])) continue;
                const float A12 = Ls[s] * r12, B6 = Bs[s] * r6;
                lrad = fmaf(G, (-12.f * A12 + 6.f * B6) * r2i, lrad);  // dLJ/dd / d, grid units
                ds = fmaf(G * isg[s], 12.f * A12 - 6.f * B6, ds);
                de = fmaf(G * kep[s], A12 - B6, de);
            }
            acc[4] = fmaf(dx, lrad, acc[4]);
            acc[5] = fmaf(dy, lrad, acc[5]);
            acc[6] = fmaf(dz, lrad, acc[6]);
            acc[7] += ds;
            acc[8] += de;
        }
        if (++cntp == 64) {
            for (int q = 0; q < 9; ++q) {
                ff_add(hi9[q], lo9[q], acc[q]);
                acc[q] = 0.f;
            }
            cntp = 0;
        }
    }
    }
    for (int q = 0; q < 9; ++q) ff_add(hi9[q], lo9[q], acc[q]);
    double tot[9];
    for (int q = 0; q < 9; ++q) tot[q] = block_sum((double)hi9[q] + (double)lo9[q], red);
    if (threadIdx.x == 0)
        for (int q = 0; q < 9; ++q) a.out[(int64_t)i * 9 + q] = tot[q];
}

struct FinalArgs {
    int n, chunks;
    double h;
    const double* raw;       // [n][6]
    const double* part;      // [chunks][n][4]
    const double* near;      // [n][9]
    double *d_xyz, *d_q, *d_sigma, *d_eps;
};

// dL/dq = (dq_far + dq_near)/h; dL/dR = -q (G_far + G_near)/h^2 - dLJ/dR;
// signs: d(1/d)/dR_i = (r - R_i)/d^3 and (r - R_i) = h (grid index - U).
__global__ void k_adj_final(FinalArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = 0; c < a.chunks; ++c)
        for (int k = 0; k < 4; ++k) s[k] += a.part[((int64_t)c * a.n + i) * 4 + k];
    const double* nr = a.near + (int64_t)i * 9;
    const double q = a.raw[6 * i + 3];
    const double ih = 1.0 / a.h, ih2 = ih * ih;
    if (a.d_q) a.d_q[i] = (s[0] + nr[0]) * ih;
    if (a.d_xyz) {
        // far: sum (r-R) * (A1/d + ...)/d^2 -> q * that / h^2 (grid units: r-R = h dvec, 1/d^3 = 1/(h^3 d_g^3));
        // near erfc terms carry their own radial factor (dphi/dd / d, grid units) with dL/dR = -q (r-R) * rad
        for (int k = 0; k < 3; ++k)
            a.d_xyz[3 * i + k] = q * s[1 + k] * ih2 - q * nr[1 + k] * ih2 - nr[4 + k] * ih;
    }
    if (a.d_sigma) a.d_sigma[i] = nr[7];
    if (a.d_eps) a.d_eps[i] = nr[8];
}

}  // namespace

struct AdjointState {
    float4* w = nullptr;
    int64_t cap_w = 0;
    float4* gu4 = nullptr;
    int64_t cap_gu4 = 0;
    double* part = nullptr;
    int64_t cap_part = 0;
    double* near = nullptr;
    int64_t cap_near = 0;
};

AdjointState* adjoint_create() { return new AdjointState(); }

void adjoint_destroy(AdjointState* s) {
    if (!s) return;
    cudaFree(s->w);
    cudaFree(s->gu4);
    cudaFree(s->part);
    cudaFree(s->near);
    delete s;
}

static rism_status aerr(std::string& err, cudaError_t e, const char* what) {
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? RISM_E_NOMEM : RISM_E_CUDA;
}

rism_status adjoint_run(AdjointState* s, TreeState* tree, const DevTables& t, const GridD& g, const Phys& ph,
                        const rism_options& o, const double* raw_dev, const double* sig_s, const double* eps_s,
                        const double* g_u, const double* g_c, const double* g_h, double* d_xyz, double* d_q,
                        double* d_sigma, double* d_eps, cudaStream_t st, std::string& err) {
    if (o.precision != RISM_PREC_FP32) {
        err = "the adjoint is implemented with FP32 pair terms (precision RISM_PREC_FP32)";
        return RISM_E_UNSUPPORTED;
    }
    const int n = (int)t.n;
    if (n == 0) return RISM_OK;
    const int64_t M = (int64_t)g.nx * g.ny * g.nz;
    cudaError_t e;
    if (M > s->cap_w) {
        cudaFree(s->w);
        s->w = nullptr;
        if ((e = cudaMalloc(&s->w, sizeof(float4) * M)) != cudaSuccess) return aerr(err, e, "adjoint weights");
        s->cap_w = M;
    }
    const int seg_per_row = (g.nx + kRowT - 1) / kRowT;
    const int nseg = seg_per_row * g.ny * g.nz;
    const int ablocks = (n + kAT * kAPT - 1) / (kAT * kAPT);
    // enough CTAs to fill the GPU several times; at most one per row segment
    int chunks = (4 * 152 + ablocks - 1) / ablocks;
    chunks = max(1, min(chunks, min(nseg, 256)));
    const int64_t need_part = (int64_t)chunks * n * 4;
    if (need_part > s->cap_part) {
        cudaFree(s->part);
        s->part = nullptr;
        if ((e = cudaMalloc(&s->part, sizeof(double) * need_part)) != cudaSuccess) return aerr(err, e, "adjoint partials");
        s->cap_part = need_part;
    }
    if ((int64_t)n * 9 > s->cap_near) {
        cudaFree(s->near);
        s->near = nullptr;
        if ((e = cudaMalloc(&s->near, sizeof(double) * 9 * n)) != cudaSuccess) return aerr(err, e, "adjoint near");
        s->cap_near = (int64_t)n * 9;
    }
    const int64_t need_gu4 = g_u ? M * ((ph.S + 3) / 4) : 0;
    if (need_gu4 > s->cap_gu4) {
        cudaFree(s->gu4);
        s->gu4 = nullptr;
        if ((e = cudaMalloc(&s->gu4, sizeof(float4) * need_gu4)) != cudaSuccess) return aerr(err, e, "adjoint G_u");
        s->cap_gu4 = need_gu4;
    }
    k_adj_weights<<<4 * 152, 256, 0, st>>>(M, ph.S, g_u, g_c, g_h, ph, s->w, s->gu4);
    FarAdjArgs fa;
    fa.nx = g.nx;
    fa.ny = g.ny;
    fa.nz = g.nz;
    fa.n = n;
    fa.seg_per_row = seg_per_row;
    fa.nseg = nseg;
    fa.chunks = chunks;
    fa.kap_g = (float)(ph.kappa * g.h);
    fa.kap2 = (float)(-ph.kappa * g.h * 1.4426950408889634);
    fa.srcf = t.srcf;
    fa.w = s->w;
    fa.part = s->part;
    fa.err = t.err;
    fa.wlim = o.wait_limit;
    const bool dh = g_h && ph.kappa > 0.0;
    bool tree_far = false;
    if (tree && o.method == RISM_METHOD_TREECODE) {
        rism_status r = tree_adjoint_far(tree, t, g, ph, o, s->w, dh, s->part, st, err, tree_far);
        if (r != RISM_OK) return r;
    }
    if (tree_far) {
        chunks = 1;  // one partial per atom, written in original atom order
    } else {
        dim3 grid(ablocks, chunks);
        if (dh) k_adj_far<true><<<grid, kAT, 0, st>>>(fa);
        else k_adj_far<false><<<grid, kAT, 0, st>>>(fa);
    }
    NearAdjArgs na;
    na.g = g;
    na.ph = ph;
    na.n = n;
    na.S = ph.S;
    na.smax = t.smax;
    na.raw = raw_dev;
    na.srcf = t.srcf;
    na.ljf = t.ljf;
    na.w = s->w;
    na.gu4 = g_u ? s->gu4 : nullptr;
    na.order = (tree && o.method == RISM_METHOD_TREECODE) ? tree_atom_order(tree) : nullptr;
    double rc_max = 0.0;
    if (o.lj_mode == RISM_LJ_RCUT) rc_max = o.lj_rcut;
    else rc_max = INFINITY;  // no cut-off, or per-pair cut-offs: scan the whole grid, the kernel tests each pair
    if (!g_u) rc_max = 0.0;
    na.rnear = fmax(rc_max, ph.rs);
    for (int k = 0; k < kMaxSites; ++k) {
        na.sig_s[k] = k < ph.S ? sig_s[k] : 0.0;
        na.eps_s[k] = k < ph.S ? eps_s[k] : 0.0;
    }
    na.out = s->near;
    k_adj_near<<<n, kNearT, 0, st>>>(na);
    FinalArgs fin{n, chunks, g.h, raw_dev, s->part, s->near, d_xyz, d_q, d_sigma, d_eps};
    k_adj_final<<<(n + 255) / 256, 256, 0, st>>>(fin);
    if ((e = cudaGetLastError()) != cudaSuccess) return aerr(err, e, "adjoint kernels");
    return RISM_OK;
}

}  // namespace rism
