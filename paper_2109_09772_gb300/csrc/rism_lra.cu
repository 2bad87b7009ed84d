// rism_lra.cu -- the all-space long-range integral of the excess chemical potential.
//
// The last integral of eq. (excess-chemical-potential-LRA) (Sec. 2.2), per solvent site s,
//   T_s = int over all space [ 1/2 (h_s^lr)^2 Theta(Q q_s) - 1/2 h_s^lr c_s^lr ] dr,
// with h^lr of eq. (tcf-r), c^lr of eq. (dcf-r) and Q the total solute charge.  Both asymptotic functions are
// sums over atoms of one radial kernel, so T_s is a double sum over atom pairs of two overlap integrals,
//   I_hh(R) = int phi_h(|r|) phi_h(|r - R|) dr,   I_hc(R) = int phi_h(|r|) phi_c(|r - R|) dr,
// and the paper counts its cost as O(N_atom^2) (Sec. 4.7).  Their wave-number integrals (products of the
// transforms of eq. (tcf-k) and eq. (dcf-k)) have closed forms; with sigma^2 = eta^2/2, b = kappa sigma,
// s = R/(2 sigma), E = e^{b^2}, g = e^{-s^2}, X1 = erfcx(s - b), X2 = erfcx(s + b):
//   I_hc(R) = (4 pi/kappa^2) [2/R - 2E e^{-kappa R}/R - (2 erfc(s) - g (X1 + X2))/R]
//   I_hh(R) = (8 pi E/kappa) e^{-kappa R} - 16 pi sigma^2 E e^{-kappa R}/R
//             + (4 pi/kappa) [g (X2 - X1) + (2 kappa sigma^2/R) g (X1 + X2)]
// -- the same exact long/short split as the grid kernels (eta -> eta sqrt 2): three smooth long-range pair
// sums, sum q/R, sum q e^{-kappa R}/R and sum q e^{-kappa R} (one rsqrt and one ex2 per pair), and short-range
// remainders that fall below 1e-15 relative beyond R = 6 sqrt(2) eta.  Within that radius the pair also takes
// 2(1 - E e^{-kappa R})/R in one piece (-expm1), which the two long-range terms would give only after a
// cancellation of several bits.  At R = 0 (an atom with itself) the
// limits I_hc(0) = 8 pi erfcx(b)/kappa and I_hh(0) = (8 pi/kappa) erfcx(b) + 16 pi sigma b erfcx(b)
// - 16 sigma sqrt(pi) apply.
//
//   k_lra_gather: the source table in the spatial order chosen on the host (cells of about 32 atoms in Morton
//                 order), so that a warp's targets and a tile's sources are each close together and the
//                 short-range branch of the pair term is taken by whole warps or by none
//   k_lra_pairs:  atoms as targets (two per thread) against one chunk of all atoms as sources, streamed through
//                 shared memory by bulk TMA copies; FP32 pair terms in grid units from the float-float source
//                 records, per-tile FP32 partials folded into float-float sums; partials per chunk in FP64.  A
//                 tile whose box lies beyond r_s from every target of a warp (most tiles, in the spatial
//                 order) takes a two-wide form of the far terms: two sources per instruction
//   k_lra_atoms:  fixed-order sum of the chunks, per-atom sums P_hc, P_hh (FP64), back in the original order
//   k_lra_total:  one CTA: S_hh = sum_a Q_a P_hh, S_hc = sum_a Q_a P_hc, Q, fixed-order tree reduction
#include <algorithm>
#include <cmath>

#include "rism_lra.h"

namespace rism {
namespace {

constexpr int kLT = 128;    // threads per pair CTA
constexpr int kLPT = 2;     // target atoms per thread
constexpr int kLTile = 64;  // source atoms per shared-memory tile
constexpr int kLParts = 10; // partial values per (chunk, atom)
constexpr int kLCtasPerSM = 4;  // pair CTAs resident per SM (registers: about 124 per thread)

struct LraPairArgs {
    const SrcF* srcf;   // [n] grid-unit float-float positions + charge (the pair sum's spatial order)
    int n;
    int chunk;          // source atoms per chunk
    float kap2;         // -kappa h log2(e): e^{-kappa R} = 2^(kap2 R_grid)
    float kapg;         // kappa h
    float bb;           // b^2 = (kappa sigma)^2
    float rs2;          // (short-range radius / h)^2
    float rsm2;         // (short-range radius / h + 0.01)^2: the far test of a whole tile
    float sgrid;        // h / (2 sigma): s = R_grid * sgrid
    float b;            // kappa sigma
    double* part;       // [chunks][n][kLParts]
    DevErr* err;
    long long wlim;
};

struct Acc {
    float h, l;
};

__device__ __forceinline__ void fold(Acc& a, float v) { ff_add(a.h, a.l, v); }

__global__ void __launch_bounds__(kLT) k_lra_pairs(LraPairArgs a) {
    __shared__ __align__(16) SrcF tile[2][kLTile];
    __shared__ __align__(8) uint64_t bar[2];
    // the current tile as pair records (x_hi, x_hi', x_lo, x_lo' | y.. | z.. | q, q', 0, 0: sources 2l, 2l + 1)
    // and the box of its sources' high parts, for the two-wide far form
    __shared__ __align__(16) float4 prec[kLTile / 2][4];
    __shared__ float tbox[6];
    const int tid = threadIdx.x;
    const int c = blockIdx.y;
    const int64_t s0 = (int64_t)c * a.chunk;
    const int scnt = (int)min((int64_t)a.chunk, (int64_t)a.n - s0);
    const int ntiles = scnt > 0 ? (scnt + kLTile - 1) / kLTile : 0;

    // two targets per thread: blockIdx.x * (kLT * kLPT) + tid + k * kLT
    float tx[kLPT], ty[kLPT], tz[kLPT], txl[kLPT], tyl[kLPT], tzl[kLPT];
    bool live[kLPT];
#pragma unroll
    for (int k = 0; k < kLPT; ++k) {
        const int i = blockIdx.x * (kLT * kLPT) + tid + k * kLT;
        live[k] = i < a.n;
        const SrcF s = a.srcf[live[k] ? i : 0];
        tx[k] = s.xh, ty[k] = s.yh, tz[k] = s.zh, txl[k] = s.xl, tyl[k] = s.yl, tzl[k] = s.zl;
    }
    // far pairs (R >= r_s): p1 = sum q/R, pk = sum q e^{-kappa R}/R; near pairs (0 < R < r_s): pkn = sum q
    // e^{-kappa R}/R, pd = sum q (1 - e^{b^2 - kappa R})/R (the long-range part of I_hc without the
    // cancellation of its two terms at small R), the short-range remainders; every pair: pe = sum q e^{-kappa R}
    Acc p1[kLPT], pk[kLPT], pkn[kLPT], pd[kLPT], pe[kLPT], shc[kLPT], sh1[kLPT], sh2[kLPT], zz[kLPT];
#pragma unroll
    for (int k = 0; k < kLPT; ++k)
        p1[k] = pk[k] = pkn[k] = pd[k] = pe[k] = shc[k] = sh1[k] = sh2[k] = zz[k] = Acc{0.f, 0.f};

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    auto issue = [&](int t) {
        const int cnt = min(kLTile, scnt - t * kLTile);
        const uint32_t bytes = cnt * sizeof(SrcF);
        mbar_expect_tx(&bar[t & 1], bytes);
        bulk_g2s(&tile[t & 1][0], a.srcf + s0 + (int64_t)t * kLTile, bytes, &bar[t & 1]);
    };
    if (tid == 0) {
        if (ntiles > 0) issue(0);
        if (ntiles > 1) issue(1);
    }
    for (int t = 0; t < ntiles; ++t) {
        const bool ok = mbar_wait_bounded(&bar[t & 1], (t >> 1) & 1, a.wlim);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                report_error(a.err, DEV_TIMEOUT, WHERE_LRA);
                for (int u = t; u < min(t + 2, ntiles); ++u) mbar_wait_bounded(&bar[u & 1], (u >> 1) & 1, a.wlim);
            }
            return;
        }
        const int cnt = min(kLTile, scnt - t * kLTile);
        const SrcF* S = tile[t & 1];
        float q1[kLPT] = {}, qk[kLPT] = {}, qkn[kLPT] = {}, qd[kLPT] = {}, qe[kLPT] = {}, qhc[kLPT] = {},
              qh1[kLPT] = {}, qh2[kLPT] = {}, qz[kLPT] = {};
        // restage the tile as pair records (the first warp; an odd count is padded with a zero charge 10^6 grid
        // units away, whose terms are exactly zero) and reduce the box of its sources
        if (tid < 32) {
            const int l = tid;
            float bl[3] = {INFINITY, INFINITY, INFINITY}, bh[3] = {-INFINITY, -INFINITY, -INFINITY};
            if (2 * l < cnt) {
                const float4 a0 = *reinterpret_cast<const float4*>(&S[2 * l].xh);
                const float4 a1 = *reinterpret_cast<const float4*>(&S[2 * l].xl);
                float4 b0 = make_float4(1.0e6f, 1.0e6f, 1.0e6f, 0.f), b1 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (2 * l + 1 < cnt) {
                    b0 = *reinterpret_cast<const float4*>(&S[2 * l + 1].xh);
                    b1 = *reinterpret_cast<const float4*>(&S[2 * l + 1].xl);
                }
                prec[l][0] = make_float4(a0.x, b0.x, a1.x, b1.x);
                prec[l][1] = make_float4(a0.y, b0.y, a1.y, b1.y);
                prec[l][2] = make_float4(a0.z, b0.z, a1.z, b1.z);
                prec[l][3] = make_float4(a0.w, b0.w, 0.f, 0.f);
                const float ax[3] = {a0.x, a0.y, a0.z}, bx[3] = {b0.x, b0.y, b0.z};
                for (int d = 0; d < 3; ++d) {
                    bl[d] = ax[d];
                    bh[d] = ax[d];
                    if (2 * l + 1 < cnt) {
                        bl[d] = fminf(bl[d], bx[d]);
                        bh[d] = fmaxf(bh[d], bx[d]);
                    }
                }
            }
            for (int d = 0; d < 3; ++d)
                for (int o = 16; o > 0; o >>= 1) {
                    bl[d] = fminf(bl[d], __shfl_xor_sync(0xffffffffu, bl[d], o));
                    bh[d] = fmaxf(bh[d], __shfl_xor_sync(0xffffffffu, bh[d], o));
                }
            if (l == 0)
                for (int d = 0; d < 3; ++d) {
                    tbox[d] = bl[d];
                    tbox[3 + d] = bh[d];
                }
        }
        __syncthreads();
        // far form when every target of the warp lies beyond r_s (plus 0.01 grid units for the sources' low
        // parts) from the tile's box: no pair of the tile takes the short-range branch
        bool far = true;
#pragma unroll
        for (int k = 0; k < kLPT; ++k) {
            if (!live[k]) continue;
            const float gx = fmaxf(0.f, fmaxf(tbox[0] - tx[k], tx[k] - tbox[3]));
            const float gy = fmaxf(0.f, fmaxf(tbox[1] - ty[k], ty[k] - tbox[4]));
            const float gz = fmaxf(0.f, fmaxf(tbox[2] - tz[k], tz[k] - tbox[5]));
            far = far && fmaf(gx, gx, fmaf(gy, gy, gz * gz)) > a.rsm2;
        }
        if (__all_sync(0xffffffffu, far)) {
            // two sources per two-wide instruction: 1/R by rsqrt, e^{-kappa R} by ex2, the far sums only
            const f32x2 K2 = pk2(a.kap2, a.kap2);
            f32x2 P1[kLPT], PK[kLPT], PE[kLPT];
#pragma unroll
            for (int k = 0; k < kLPT; ++k) P1[k] = PK[k] = PE[k] = 0ull;
            const int np = (cnt + 1) >> 1;
            for (int l = 0; l < np; ++l) {
                const ulonglong2 X = *reinterpret_cast<const ulonglong2*>(&prec[l][0]);
                const ulonglong2 Y = *reinterpret_cast<const ulonglong2*>(&prec[l][1]);
                const ulonglong2 Z = *reinterpret_cast<const ulonglong2*>(&prec[l][2]);
                const f32x2 Q = *reinterpret_cast<const f32x2*>(&prec[l][3]);
#pragma unroll
                for (int k = 0; k < kLPT; ++k) {
                    const f32x2 DX = add2(sub2(pk2(tx[k], tx[k]), X.x), sub2(pk2(txl[k], txl[k]), X.y));
                    const f32x2 DY = add2(sub2(pk2(ty[k], ty[k]), Y.x), sub2(pk2(tyl[k], tyl[k]), Y.y));
                    const f32x2 DZ = add2(sub2(pk2(tz[k], tz[k]), Z.x), sub2(pk2(tzl[k], tzl[k]), Z.y));
                    const f32x2 D2 = fma2(DX, DX, fma2(DY, DY, mul2(DZ, DZ)));
                    const float2 d2 = up2(D2);
                    const f32x2 RI = pk2(rsqrt_approx(d2.x), rsqrt_approx(d2.y));
                    const float2 e = up2(mul2(K2, mul2(D2, RI)));
                    const f32x2 E = pk2(ex2_approx(e.x), ex2_approx(e.y));
                    const f32x2 QR = mul2(Q, RI);
                    P1[k] = add2(P1[k], QR);
                    PK[k] = fma2(QR, E, PK[k]);
                    PE[k] = fma2(Q, E, PE[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < kLPT; ++k) {
                const float2 v1 = up2(P1[k]), vk = up2(PK[k]), ve = up2(PE[k]);
                q1[k] = v1.x + v1.y;
                qk[k] = vk.x + vk.y;
                qe[k] = ve.x + ve.y;
            }
        } else {
            for (int j = 0; j < cnt; ++j) {
                const float4 g0 = *reinterpret_cast<const float4*>(&S[j].xh);
                const float4 g1 = *reinterpret_cast<const float4*>(&S[j].xl);
#pragma unroll
                for (int k = 0; k < kLPT; ++k) {
                    // relative position to one rounding of each component: (hi - hi) + (lo - lo)
                    const float dx = (tx[k] - g0.x) + (txl[k] - g1.x);
                    const float dy = (ty[k] - g0.y) + (tyl[k] - g1.y);
                    const float dz = (tz[k] - g0.z) + (tzl[k] - g1.z);
                    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    const float rr = rsqrt_approx(d2);
                    const float ri = d2 > 0.f ? rr : 0.f;
                    const float R = d2 * ri;
                    const float e = d2 > 0.f ? ex2_approx(a.kap2 * R) : 0.f;  // R = 0 takes the limits below
                    const float qr = g0.w * ri;
                    qe[k] = fmaf(g0.w, e, qe[k]);
                    if (d2 >= a.rs2) {
                        q1[k] += qr;
                        qk[k] = fmaf(qr, e, qk[k]);
                    } else {
                        if (d2 > 0.f) {
                            qkn[k] = fmaf(qr, e, qkn[k]);
                            qd[k] = fmaf(qr, -expm1f(a.bb - a.kapg * R), qd[k]);
                            const float s = R * a.sgrid;
                            const float gg = __expf(-s * s);
                            const float X1 = erfcxf(s - a.b), X2 = erfcxf(s + a.b);
                            qhc[k] = fmaf(qr, 2.f * erfcf(s) - gg * (X1 + X2), qhc[k]);
                            qh1[k] = fmaf(g0.w, gg * (X2 - X1), qh1[k]);
                            qh2[k] = fmaf(qr, gg * (X1 + X2), qh2[k]);
                        } else {
                            // an atom with itself (or two atoms at one position): the R = 0 limits
                            qz[k] += g0.w;
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kLPT; ++k) {
            fold(p1[k], q1[k]);
            fold(pk[k], qk[k]);
            fold(pkn[k], qkn[k]);
            fold(pd[k], qd[k]);
            fold(pe[k], qe[k]);
            fold(shc[k], qhc[k]);
            fold(sh1[k], qh1[k]);
            fold(sh2[k], qh2[k]);
            fold(zz[k], qz[k]);
        }
        __syncthreads();
        if (tid == 0 && t + 2 < ntiles) issue(t + 2);
    }
#pragma unroll
    for (int k = 0; k < kLPT; ++k) {
        const int i = blockIdx.x * (kLT * kLPT) + tid + k * kLT;
        if (!live[k]) continue;
        double* o = a.part + ((int64_t)c * a.n + i) * kLParts;
        const Acc v[9] = {p1[k], pk[k], pkn[k], pd[k], pe[k], shc[k], sh1[k], sh2[k], zz[k]};
#pragma unroll
        for (int m = 0; m < 9; ++m) o[m] = (double)v[m].h + (double)v[m].l;
        o[9] = 0.0;
    }
}

struct LraConst {
    double h, kappa, E, sig2, I0hc, I0hh;
};

// The source table in the pair sum's order: ssrc[k] = srcf[perm[k]].
__global__ void k_lra_gather(const SrcF* __restrict__ srcf, const int* __restrict__ perm, int n, SrcF* ssrc) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) ssrc[k] = srcf[perm[k]];
}

// Per atom: fixed-order sum of the chunk partials and the assembly of the two overlap sums (FP64).
__global__ void k_lra_atoms(const double* __restrict__ part, int n, int chunks, LraConst k,
                            const int* __restrict__ perm, double2* atom) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int c = 0; c < chunks; ++c) {
        const double* o = part + ((int64_t)c * n + i) * kLParts;
#pragma unroll
        for (int m = 0; m < 9; ++m) v[m] += o[m];
    }
    const double ih = 1.0 / k.h;
    const double P1 = v[0] * ih, Pkf = v[1] * ih, Pkn = v[2] * ih, Pd = v[3] * ih, Pe = v[4];
    const double SRhc = v[5] * ih, SRh1 = v[6], SRh2 = v[7] * ih, z = v[8];
    const double pi4 = 4.0 * M_PI;
    const double phc = pi4 / (k.kappa * k.kappa) * (2.0 * P1 - 2.0 * k.E * Pkf + 2.0 * Pd - SRhc) + z * k.I0hc;
    const double phh = 2.0 * pi4 * k.E / k.kappa * Pe - 4.0 * pi4 * k.sig2 * k.E * (Pkf + Pkn) +
                       pi4 / k.kappa * (SRh1 + 2.0 * k.kappa * k.sig2 * SRh2) + z * k.I0hh;
    atom[perm[i]] = make_double2(phc, phh);
}

// S_hh, S_hc and Q in one CTA (fixed order: strided per-thread sums, then a tree).
constexpr int kTotT = 1024;
__global__ void __launch_bounds__(kTotT) k_lra_total(const double2* __restrict__ atom, const Geo* __restrict__ geo,
                                                    int n, double* tot) {
    __shared__ double red[3][kTotT];
    double a = 0.0, b = 0.0, q = 0.0;
    for (int i = threadIdx.x; i < n; i += kTotT) {
        const double qi = geo[i].q;
        const double2 p = atom[i];
        a += qi * p.y;
        b += qi * p.x;
        q += qi;
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    red[2][threadIdx.x] = q;
    __syncthreads();
    for (int w = kTotT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int m = 0; m < 3; ++m) red[m][threadIdx.x] += red[m][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) tot[threadIdx.x] = red[threadIdx.x][0];
}

}  // namespace

size_t lra_scratch_doubles(int64_t n, int sms) {
    const int chunks = lra_chunks(n, sms);
    return (size_t)chunks * (size_t)n * kLParts;
}

int lra_chunks(int64_t n, int sms) {
    if (n <= 0) return 1;
    const int64_t tblocks = (n + kLT * kLPT - 1) / (kLT * kLPT);
    int64_t c = (kLCtasPerSM * (int64_t)sms + tblocks - 1) / tblocks;  // every SM's CTA slots filled
    c = std::min<int64_t>(c, (n + kLTile - 1) / kLTile);        // at least one tile of sources per chunk
    return (int)std::max<int64_t>(c, 1);
}

cudaError_t launch_lra(const DevTables& t, const GridD& g, const Phys& ph, int sms, const int* perm, SrcF* ssrc,
                       double* part, double2* atom, double* tot, long long wait_limit, cudaStream_t st) {
    const int n = (int)t.n;
    if (n <= 0) return cudaSuccess;
    const int chunks = lra_chunks(n, sms);
    k_lra_gather<<<std::min((n + 255) / 256, 4 * sms), 256, 0, st>>>(t.srcf, perm, n, ssrc);
    LraPairArgs a;
    a.srcf = ssrc;
    a.n = n;
    a.chunk = (int)((n + chunks - 1) / chunks);
    // 16-byte aligned bulk copies: every chunk starts at a multiple of 2 records (SrcF is 32 bytes)
    a.kap2 = (float)(-ph.kappa * g.h * 1.4426950408889634);
    a.kapg = (float)(ph.kappa * g.h);
    const double sigma = ph.eta / std::sqrt(2.0);
    a.bb = (float)((ph.kappa * sigma) * (ph.kappa * sigma));
    const double rs = 6.0 * std::sqrt(2.0) * ph.eta;
    a.rs2 = (float)((rs / g.h) * (rs / g.h));
    a.rsm2 = (float)((rs / g.h + 0.01) * (rs / g.h + 0.01));
    a.sgrid = (float)(g.h / (2.0 * sigma));
    a.b = (float)(ph.kappa * sigma);
    a.part = part;
    a.err = t.err;
    a.wlim = wait_limit;
    dim3 grid((unsigned)((n + kLT * kLPT - 1) / (kLT * kLPT)), (unsigned)chunks);
    k_lra_pairs<<<grid, kLT, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    LraConst k;
    k.h = g.h;
    k.kappa = ph.kappa;
    const double b = ph.kappa * sigma;
    k.E = std::exp(b * b);
    k.sig2 = sigma * sigma;
    const double ex = std::exp(b * b) * std::erfc(b);  // erfcx(b), b small and positive
    k.I0hc = 8.0 * M_PI * ex / ph.kappa;
    k.I0hh = 8.0 * M_PI * ex / ph.kappa + 16.0 * M_PI * sigma * b * ex - 16.0 * sigma * std::sqrt(M_PI);
    k_lra_atoms<<<(n + 255) / 256, 256, 0, st>>>(part, n, chunks, k, perm, atom);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_lra_total<<<1, kTotT, 0, st>>>(atom, t.geo, n, tot);
    return cudaGetLastError();
}

}  // namespace rism
