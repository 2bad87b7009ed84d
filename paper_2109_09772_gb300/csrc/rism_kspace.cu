// rism_kspace.cu -- reciprocal-space long-range asymptotics on the grid's reciprocal lattice.
//
// Eq. (dcf-k) and eq. (tcf-k) (Sec. 2.2), times the Coulomb constant of the unit reading:
//   c_s(k) = -(4 pi beta k_e q_s / k^2) e^{-k^2 eta^2/4} S(k)
//   h_s(k) = -(4 pi beta k_e q_s / (eps_r (k^2 + kappa^2))) e^{-k^2 eta^2/4} S(k),
//   S(k)   = sum_a Q_a e^{i k.(R_a - o)},
// o the grid origin, k = 2 pi (m_x/(n_x h), m_y/(n_y h), m_z/(n_z h)) on the half spectrum of a real-to-complex
// transform ([n_z][n_y][n_x/2 + 1], m_x = j_x, m = j or j - n along y and z), c(0) = 0.  With the frequency
// cut-off of Sec. 2.5 only k^2 <= k_cut^2 is summed (the rest is 0).
//
// The structure factor is separable: e^{i k.R} = E_x(m_x) E_y(m_y) E_z(m_z), each a phase of one coordinate, so
//   k_kphase: per atom and axis the table of e^{i 2 pi m x / n} (x in grid units from the float-float source
//             record; the phase m x / n is reduced modulo one cycle exactly -- integer part of x modulo n in
//             integer arithmetic, the rest as an error-free product and float-float sum -- before sincospif),
//             the charge folded into the z table;
//   k_ksum:   CTAs of (one m_z, 32 m_y, 128 m_x); per tile of 32 atoms the x, y and z tables arrive as three
//             bulk TMA copies (the tables are blocked so that a tile is contiguous), the CTA forms T = E_y E_z Q
//             in shared memory, and each thread accumulates 4 m_x x 4 m_y complex sums S += E_x T (4 FP32 FMAs
//             per (k, atom) pair), partials of 32 atoms folded into float-float sums; rows beyond the cut-off
//             sphere are skipped warp by warp, CTAs wholly beyond it only write zeros.  The epilogue applies the k-dependent factors and writes c and h of every site
//             as FP64 complex values (each rounded once to FP32, widened on the integer pipe).
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "rism_kspace.h"

namespace rism {
namespace {

constexpr int kKT = 32;        // atoms per tile (the FP32 partials are folded after every tile)
constexpr int kKW = 8;         // warps per CTA
constexpr int kKMY = 4;        // m_y rows per warp
constexpr int kKMX = 4;        // m_x per lane (stride 32)
constexpr int kKBX = 32 * kKMX;    // m_x per CTA (128)
constexpr int kKBY = kKW * kKMY;   // m_y per CTA (32)
constexpr int kKThreads = 32 * kKW;

// Blocked so that one tile of a CTA (its m_x or m_y block, 32 atoms) is one contiguous bulk copy.
struct KTables {
    float2* ex;  // [mxp / 128][npad][128]
    float2* ey;  // [nyp / 32][npad][32]
    float2* ez;  // [nz][npad], charge folded in
    int npad, mxp, nyp;
};

// e^{i 2 pi m x / na} for x = xh + xl grid units (float-float), m a signed integer frequency.
__device__ __forceinline__ float2 lattice_phase(float xh, float xl, int m, int na) {
    const float fi = floorf(xh);
    const float ff = xh - fi;                       // exact: [0, 1)
    int ir = (int)fmodf(fi, (float)na);             // integer part modulo na (fmodf is exact)
    if (ir < 0) ir += na;
    long long prod = (long long)m * ir;             // |m| < 2^16, ir < 2^16
    int r0 = (int)(prod % na);
    if (r0 < 0) r0 += na;
    const float fm = (float)m;
    const float p2 = fm * ff;                       // m * frac(xh), with its rounding error e2
    const float e2 = fmaf(fm, ff, -p2);
    const float p3 = fm * xl;                       // the low part: a tiny correction
    float s, e1;
    two_sum((float)r0, p2, s, e1);                  // s + e1 = r0 + p2 exactly
    const float lo = e1 + e2 + p3;
    const float nf = (float)na;
    const float qn = rintf(s / nf);
    const float r = fmaf(-qn, nf, s);               // exact: |r| <= na/2 and a multiple of ulp(s)
    const float t = r + lo;                         // the phase in grid units, |t| <~ na/2
    float sn, cs;
    sincospif(__fdiv_rn(2.0f * t, nf), &sn, &cs);   // one rounding of the half-cycle count
    return make_float2(cs, sn);
}

__global__ void k_kphase(const SrcF* __restrict__ srcf, int n, int nx, int ny, int nz, KTables tb) {
    const int mxh = nx / 2 + 1;
    const int64_t per = (int64_t)tb.mxp + tb.nyp + nz;
    const int64_t total = (int64_t)tb.npad * per;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(t / per);
        const int j = (int)(t - (int64_t)a * per);
        const bool live = a < n;
        const SrcF s = srcf[live ? a : 0];
        if (j < tb.mxp) {
            const float2 v = (live && j < mxh) ? lattice_phase(s.xh, s.xl, j, nx) : make_float2(0.f, 0.f);
            tb.ex[((int64_t)(j / kKBX) * tb.npad + a) * kKBX + j % kKBX] = v;
        } else if (j < tb.mxp + tb.nyp) {
            const int jy = j - tb.mxp;
            const int m = jy <= (ny - 1) / 2 ? jy : jy - ny;
            const float2 v = (live && jy < ny) ? lattice_phase(s.yh, s.yl, m, ny) : make_float2(0.f, 0.f);
            tb.ey[((int64_t)(jy / kKBY) * tb.npad + a) * kKBY + jy % kKBY] = v;
        } else {
            const int jz = j - tb.mxp - tb.nyp;
            const int m = jz <= (nz - 1) / 2 ? jz : jz - nz;
            float2 v = make_float2(0.f, 0.f);
            if (live) {
                v = lattice_phase(s.zh, s.zl, m, nz);
                v.x *= s.q;
                v.y *= s.q;
            }
            tb.ez[(int64_t)jz * tb.npad + a] = v;
        }
    }
}

struct KSumArgs {
    KTables tb;
    int nx, ny, nz, S;
    double h, kc2;           // kc2 <= 0: no cut-off
    float fc0, fh0;          // -4 pi beta k_e and -4 pi beta k_e / eps_r
    float eta2q;             // eta^2 / 4
    float kap2;              // kappa^2 (0: h not requested / undefined)
    float qs[kMaxSites];
    double* c;               // [S][nz][ny][nxh] complex (re, im), or null
    double* hk;              // same, or null
    DevErr* err;
    long long wlim;
};

// k^2 of lattice point (jx, jy, jz) exactly as the FP64 definition orders it (no contraction).
__device__ __forceinline__ double lattice_k2(int jx, int jy, int jz, int nx, int ny, int nz, double h) {
    const int my = jy <= (ny - 1) / 2 ? jy : jy - ny;
    const int mz = jz <= (nz - 1) / 2 ? jz : jz - nz;
    const double tp = __dmul_rn(2.0, M_PI);
    const double kx = __ddiv_rn(__dmul_rn(tp, (double)jx), __dmul_rn((double)nx, h));
    const double ky = __ddiv_rn(__dmul_rn(tp, (double)my), __dmul_rn((double)ny, h));
    const double kz = __ddiv_rn(__dmul_rn(tp, (double)mz), __dmul_rn((double)nz, h));
    return __dadd_rn(__dadd_rn(__dmul_rn(kx, kx), __dmul_rn(ky, ky)), __dmul_rn(kz, kz));
}

__global__ void __launch_bounds__(kKThreads, 2) k_ksum(KSumArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2* sx = reinterpret_cast<float2*>(smem);                       // [2][kKT][kKBX]
    float2* sy = sx + 2 * kKT * kKBX;                                   // [2][kKT][kKBY]
    float2* sz = sy + 2 * kKT * kKBY;                                   // [2][kKT]
    float2* st = sz + 2 * kKT;                                          // [kKT][kKBY] (atom-major)
    uint64_t* bar = reinterpret_cast<uint64_t*>(st + kKT * kKBY);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int mxb = blockIdx.x * kKBX, my0 = blockIdx.y * kKBY, jz = blockIdx.z;
    const int nxh = a.nx / 2 + 1;
    const KTables tb = a.tb;

    // m_x groups of 32 this warp needs: rows beyond the cut-off sphere (or the grid) need none
    int ngrp = 0;
    {
        int jmax = -1;
        for (int j = 0; j < kKMY; ++j) {
            const int jy = my0 + w * kKMY + j;
            if (jy >= a.ny) continue;
            if (a.kc2 <= 0.0) {
                jmax = nxh - 1;
                continue;
            }
            const double r0 = lattice_k2(0, jy, jz, a.nx, a.ny, a.nz, a.h);
            if (r0 > a.kc2) continue;
            // largest m_x with kx^2 <= kc2 - (ky^2 + kz^2), one beyond for rounding (decided exactly below)
            const double kxm = sqrt(a.kc2 - r0) * (a.nx * a.h) / (2.0 * M_PI);
            jmax = max(jmax, min(nxh - 1, (int)kxm + 1));
        }
        if (jmax >= mxb) ngrp = min(kKMX, (jmax - mxb) / 32 + 1);
    }
    const int any = __syncthreads_or(ngrp > 0);

    float2 acc[kKMX][kKMY], hi[kKMX][kKMY], lo[kKMX][kKMY];
#pragma unroll
    for (int i = 0; i < kKMX; ++i)
#pragma unroll
        for (int j = 0; j < kKMY; ++j) hi[i][j] = lo[i][j] = make_float2(0.f, 0.f);

    if (any) {
        const int ntiles = tb.npad / kKT;
        if (tid == 0) {
            mbar_init(&bar[0], 1);
            mbar_init(&bar[1], 1);
            mbar_fence_init();
        }
        __syncthreads();
        auto issue = [&](int t) {
            const int b = t & 1, a0 = t * kKT;
            const uint32_t bx = kKT * kKBX * sizeof(float2), by = kKT * kKBY * sizeof(float2);
            const uint32_t bz = kKT * sizeof(float2);
            mbar_expect_tx(&bar[b], bx + by + bz);
            bulk_g2s(sx + b * kKT * kKBX, tb.ex + ((int64_t)blockIdx.x * tb.npad + a0) * kKBX, bx, &bar[b]);
            bulk_g2s(sy + b * kKT * kKBY, tb.ey + ((int64_t)blockIdx.y * tb.npad + a0) * kKBY, by, &bar[b]);
            bulk_g2s(sz + b * kKT, tb.ez + (int64_t)jz * tb.npad + a0, bz, &bar[b]);
        };
        if (tid == 0) {
            issue(0);
            if (ntiles > 1) issue(1);
        }
        for (int t = 0; t < ntiles; ++t) {
            const int b = t & 1;
            const bool ok = mbar_wait_bounded(&bar[b], (t >> 1) & 1, a.wlim);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    report_error(a.err, DEV_TIMEOUT, WHERE_KSPACE);
                    for (int u = t; u < min(t + 2, ntiles); ++u) mbar_wait_bounded(&bar[u & 1], (u >> 1) & 1, a.wlim);
                }
                return;
            }
            // T[a][my] = E_y(a, my) * (Q_a E_z(a, mz)): 32 atoms x 32 rows, four per thread
            for (int e = tid; e < kKT * kKBY; e += kKThreads) {
                const int aa = e / kKBY, yy = e - aa * kKBY;
                const float2 y = sy[(b * kKT + aa) * kKBY + yy], z = sz[b * kKT + aa];
                st[e] = make_float2(y.x * z.x - y.y * z.y, y.x * z.y + y.y * z.x);
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < kKMX; ++i)
#pragma unroll
                for (int j = 0; j < kKMY; ++j) acc[i][j] = make_float2(0.f, 0.f);
            const float2* X = sx + b * kKT * kKBX;
            auto body = [&](auto NG) {
                constexpr int G = decltype(NG)::value;
                for (int aa = 0; aa < kKT; ++aa) {
                    const float4 t01 = *reinterpret_cast<const float4*>(&st[aa * kKBY + w * kKMY]);
                    const float4 t23 = *reinterpret_cast<const float4*>(&st[aa * kKBY + w * kKMY + 2]);
                    const float2 T[kKMY] = {make_float2(t01.x, t01.y), make_float2(t01.z, t01.w),
                                            make_float2(t23.x, t23.y), make_float2(t23.z, t23.w)};
#pragma unroll
                    for (int i = 0; i < G; ++i) {
                        const float2 x = X[aa * kKBX + lane + 32 * i];
#pragma unroll
                        for (int j = 0; j < kKMY; ++j) {
                            acc[i][j].x = fmaf(x.x, T[j].x, fmaf(-x.y, T[j].y, acc[i][j].x));
                            acc[i][j].y = fmaf(x.x, T[j].y, fmaf(x.y, T[j].x, acc[i][j].y));
                        }
                    }
                }
            };
            switch (ngrp) {
                case 1: body(std::integral_constant<int, 1>{}); break;
                case 2: body(std::integral_constant<int, 2>{}); break;
                case 3: body(std::integral_constant<int, 3>{}); break;
                case 4: body(std::integral_constant<int, 4>{}); break;
                default: break;
            }
#pragma unroll
            for (int i = 0; i < kKMX; ++i)
#pragma unroll
                for (int j = 0; j < kKMY; ++j) {
                    ff_add(hi[i][j].x, lo[i][j].x, acc[i][j].x);
                    ff_add(hi[i][j].y, lo[i][j].y, acc[i][j].y);
                }
            __syncthreads();
            if (tid == 0 && t + 2 < ntiles) issue(t + 2);
        }
    }

    // epilogue: the k-dependent factors, every site, c and h; entries beyond the cut-off are zero
    const int64_t plane = (int64_t)a.ny * nxh;
    const int64_t site = plane * a.nz;
#pragma unroll
    for (int j = 0; j < kKMY; ++j) {
        const int jy = my0 + w * kKMY + j;
        if (jy >= a.ny) continue;
#pragma unroll
        for (int i = 0; i < kKMX; ++i) {
            const int jx = mxb + lane + 32 * i;
            if (jx >= nxh) continue;
            const double k2d = lattice_k2(jx, jy, jz, a.nx, a.ny, a.nz, a.h);
            const bool keep = (a.kc2 <= 0.0 || k2d <= a.kc2) && i < ngrp;
            float sre = 0.f, sim = 0.f, fc = 0.f, fh = 0.f;
            if (keep) {
                sre = hi[i][j].x + lo[i][j].x;
                sim = hi[i][j].y + lo[i][j].y;
                const float k2 = (float)k2d;
                const float g = expf(-k2 * a.eta2q);
                fc = k2 > 0.f ? a.fc0 * g / k2 : 0.f;
                fh = a.kap2 > 0.f ? a.fh0 * g / (k2 + a.kap2) : 0.f;
            }
            const int64_t o = (int64_t)jz * plane + (int64_t)jy * nxh + jx;
            for (int s = 0; s < a.S; ++s) {
                if (a.c) {
                    const float f = a.qs[s] * fc;
                    __stcs(reinterpret_cast<double2*>(a.c) + s * site + o, make_double2(f2d_alu(f * sre), f2d_alu(f * sim)));
                }
                if (a.hk) {
                    const float f = a.qs[s] * fh;
                    __stcs(reinterpret_cast<double2*>(a.hk) + s * site + o, make_double2(f2d_alu(f * sre), f2d_alu(f * sim)));
                }
            }
        }
    }
}

int round_up(int v, int m) { return (v + m - 1) / m * m; }

}  // namespace

size_t kspace_table_bytes(int64_t n, int nx, int ny, int nz) {
    const int64_t npad = round_up((int)std::max<int64_t>(n, 1), kKT);
    const int64_t mxp = round_up(nx / 2 + 1, kKBX), nyp = round_up(ny, kKBY);
    return sizeof(float2) * (size_t)(npad * (mxp + nyp) + (int64_t)nz * npad);
}

double kspace_bound(double k, const KspaceSetup& s) {
    return 4.0 * std::sqrt(2.0) * M_PI * s.beta * s.k_e * s.qmax * std::exp(-k * k * s.eta * s.eta / 4.0) * s.qabs /
           (k * k);
}

// k where the bound equals tol: Newton on log(bound) - log(tol) (decreasing and convex in k), from a start
// below the root, safeguarded by bisection on a bracket.
double kspace_kcut(const KspaceSetup& s, double tol) {
    if (!(tol > 0.0) || !(s.qabs > 0.0) || !(s.qmax > 0.0)) return 0.0;
    double lo = 1e-6, hi = 1.0;
    while (kspace_bound(hi, s) > tol && hi < 1e6) hi *= 2.0;
    if (kspace_bound(lo, s) <= tol) return lo;
    double k = lo;
    for (int it = 0; it < 200; ++it) {
        const double g = std::log(kspace_bound(k, s)) - std::log(tol);
        if (g > 0.0) lo = k; else hi = k;
        const double dg = -k * s.eta * s.eta / 2.0 - 2.0 / k;
        double kn = k - g / dg;
        if (!(kn > lo && kn < hi)) kn = 0.5 * (lo + hi);
        if (std::fabs(kn - k) <= 1e-15 * k) {
            k = kn;
            break;
        }
        k = kn;
    }
    return k;
}

cudaError_t launch_kspace(const DevTables& t, const GridD& g, const KspaceSetup& s, void* tables, double* c_k,
                          double* h_k, long long wait_limit, cudaStream_t st) {
    const int n = (int)t.n;
    KTables tb;
    tb.npad = round_up(std::max(n, 1), kKT);
    tb.mxp = round_up(g.nx / 2 + 1, kKBX);
    tb.nyp = round_up(g.ny, kKBY);
    tb.ex = static_cast<float2*>(tables);
    tb.ey = tb.ex + (int64_t)tb.npad * tb.mxp;
    tb.ez = tb.ey + (int64_t)tb.npad * tb.nyp;
    const int64_t total = (int64_t)tb.npad * (tb.mxp + tb.nyp + g.nz);
    const int nb = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    k_kphase<<<nb, 256, 0, st>>>(t.srcf, n, g.nx, g.ny, g.nz, tb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    KSumArgs a;
    a.tb = tb;
    a.nx = g.nx;
    a.ny = g.ny;
    a.nz = g.nz;
    a.S = s.S;
    a.h = g.h;
    a.kc2 = s.kcut > 0.0 ? s.kcut * s.kcut : 0.0;
    a.fc0 = (float)(-4.0 * M_PI * s.beta * s.k_e);
    a.fh0 = (float)(-4.0 * M_PI * s.beta * s.k_e / s.eps_r);
    a.eta2q = (float)(s.eta * s.eta / 4.0);
    a.kap2 = (float)(s.kappa * s.kappa);
    for (int k = 0; k < kMaxSites; ++k) a.qs[k] = (float)s.qs[k];
    a.c = c_k;
    a.hk = h_k;
    a.err = t.err;
    a.wlim = wait_limit;
    const size_t sm = sizeof(float2) * (2 * kKT * kKBX + 2 * kKT * kKBY + 2 * kKT + kKT * kKBY) + 2 * sizeof(uint64_t);
    raise_dyn_smem(k_ksum, sm);
    dim3 grid((unsigned)(tb.mxp / kKBX), (unsigned)(tb.nyp / kKBY), (unsigned)g.nz);
    k_ksum<<<grid, kKThreads, sm, st>>>(a);
    return cudaGetLastError();
}

}  // namespace rism
