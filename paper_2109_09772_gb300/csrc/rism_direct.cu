// rism_direct.cu -- solute/solvent setup and the direct-sum evaluation kernels.
//
// The direct kernels evaluate, for every grid point of a CTA tile and every
// atom, the pair terms of the generic pair sum of Sec. 2.3, eq. (pot):
//   Phi1  = sum q/d                 (Coulomb, and the long-range part of eq. (dcf-r))
//   Phik  = sum q e^{-kappa d}/d    (long-range part of eq. (tcf-r))
//   Sc    = sum_{d<rs} q erfc(d/eta)/d
//   Sh    = sum_{d<rs} q e^{-x^2}[erfcx(x-a)+erfcx(x+a)]/d,  x = d/eta, a = kappa eta/2
//   LJ_s  = sum_{d<rc_is} A_is/d^12 - B_is/d^6                (Sec. 2.6)
// and assemble u = k_e q_s Phi1 + LJ_s, c = -beta k_e q_s (Phi1 - Sc),
// h = -(beta k_e q_s/(2 eps_r)) (2 e^{a^2} Phik - Sh).  The split
// erf = 1 - erfc and e^{a^2}[e^{-kd}erfc(a-x) - e^{kd}erfc(a+x)] =
// 2 e^{a^2} e^{-kd} - e^{-x^2}[erfcx(x-a) + erfcx(x+a)] is exact; the
// remainders Sc, Sh fall below 1e-16 relative beyond rs ~ 6 eta, which is the
// exact form of the far-field simplification eq. (tcfexp) of Sec. 2.4.2.
//
// Data movement: atoms are streamed through shared memory in tiles of T by
// bulk TMA copies (cp.async.bulk + mbarrier, double-buffered, bounded waits);
// every thread owns a strip of P consecutive x points at one (y, z) and reads
// each atom as a shared-memory broadcast.
#include <cmath>

#include "rism_kernels.h"

namespace rism {

// ------------------------------------------------------------------ setup
__device__ double lj_u(double A, double B, double r) {
    double r2 = 1.0 / (r * r);
    double r6 = r2 * r2 * r2;
    return r6 * (A * r6 - B);
}

// Largest r with |A/r^12 - B/r^6| = tol (Sec. 2.6 per-pair cut-off), bisection.
__device__ double rcut_from_tol(double A, double B, double tol) {
    if (A <= 0.0 || B <= 0.0) return 0.0;
    double sig6 = A / B;                     // sigma^6
    double rmin = cbrt(sqrt(2.0 * sig6));    // 2^(1/6) sigma
    double eps = B * B / (4.0 * A);          // well depth
    double lo, hi;
    if (tol < eps) {
        lo = rmin;
        hi = rmin;
        for (int k = 0; k < 64 && fabs(lj_u(A, B, hi)) > tol; ++k) hi *= 2.0;
        for (int it = 0; it < 200; ++it) {
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (fabs(lj_u(A, B, mid)) > tol) lo = mid; else hi = mid;
        }
        return hi;
    }
    double sig = cbrt(sqrt(sig6));
    lo = 0.5 * sig;
    for (int k = 0; k < 64 && lj_u(A, B, lo) < tol; ++k) lo *= 0.5;
    hi = sig;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (lj_u(A, B, mid) > tol) lo = mid; else hi = mid;
    }
    return hi;
}

struct SetupArgs {
    const double* raw;
    int64_t n;
    int S, smax;
    double sig_s[kMaxSites], eps_s[kMaxSites];
    int lj_mode;
    double lj_rcut, lj_tol;
    GridD g;
};

// One thread per (atom, site slot): the pair's Lorentz-Berthelot LJ terms (FP64 and FP32 grid units); the
// thread of slot 0 also writes the atom's position records.
__global__ void k_setup(SetupArgs a, Geo* geo, SrcF* srcf, LJd* ljd, LJf* ljf) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= a.n * a.smax) return;
    const int64_t i = t / a.smax;
    const int s = (int)(t - i * a.smax);
    const double* r = a.raw + 6 * i;
    if (s == 0) {
        const double x = r[0], y = r[1], z = r[2], q = r[3];
        geo[i] = Geo{x, y, z, q};
        const double ih = 1.0 / a.g.h;
        srcf[i] = make_srcf((x - a.g.ox) * ih, (y - a.g.oy) * ih, (z - a.g.oz) * ih, q);
    }
    LJd d{0.0, 0.0, 0.0, 0.0};
    LJf f{0.f, 0.f, 0.f, 0.f};
    if (s < a.S) {
        const double sg = r[4], ep = r[5];
        const double h2 = a.g.h * a.g.h, h6 = h2 * h2 * h2;
        double sig = 0.5 * (sg + a.sig_s[s]);      // Lorentz
        double eps = sqrt(ep * a.eps_s[s]);        // Berthelot
        double s2 = sig * sig, s6 = s2 * s2 * s2;
        double A = 4.0 * eps * s6 * s6, B = 4.0 * eps * s6;
        double rc2;
        if (a.lj_mode == RISM_LJ_RCUT) rc2 = a.lj_rcut * a.lj_rcut;
        else if (a.lj_mode == RISM_LJ_TOL) { double rc = rcut_from_tol(A, B, a.lj_tol); rc2 = rc * rc; }
        else rc2 = INFINITY;
        d = LJd{A, B, rc2, 0.0};
        f = LJf{(float)(A / (h6 * h6)), (float)(B / h6), (float)(rc2 / h2), 0.f};
    }
    ljd[t] = d;
    ljf[t] = f;
}

cudaError_t launch_setup(const double* raw, int64_t n, int S, int smax, const double* sig_s, const double* eps_s,
                         int lj_mode, double lj_rcut, double lj_tol, const GridD& g, DevTables& t,
                         cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    SetupArgs a;
    a.raw = raw;
    a.n = n;
    a.S = S;
    a.smax = smax;
    for (int s = 0; s < kMaxSites; ++s) {
        a.sig_s[s] = s < S ? sig_s[s] : 0.0;
        a.eps_s[s] = s < S ? eps_s[s] : 0.0;
    }
    a.lj_mode = lj_mode;
    a.lj_rcut = lj_rcut;
    a.lj_tol = lj_tol;
    a.g = g;
    const int nb = (int)((n * smax + 127) / 128);
    k_setup<<<nb, 128, 0, st>>>(a, t.geo, t.srcf, t.ljd, t.ljf);
    return cudaGetLastError();
}

// I_s = sum_i 4 pi (A/(9 rc^9) - B/(3 rc^3)); one CTA per site, fixed-order reduction.
constexpr int kTailThreads = 1024;
__global__ void __launch_bounds__(kTailThreads) k_lj_tail(const LJd* lj, int64_t n, int smax, double* out) {
    constexpr int NT = kTailThreads;
    __shared__ double red[NT];
    int s = blockIdx.x;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += NT) {
        LJd p = lj[i * smax + s];
        if (isfinite(p.rc2) && p.rc2 > 0.0) {
            // 4 pi (A / (9 rc^9) - B / (3 rc^3)) with r3 = rc^-3 from one reciprocal square root
            const double ri = rsqrt(p.rc2), r3 = ri * ri * ri;
            acc += 4.0 * M_PI * r3 * (p.A * (1.0 / 9.0) * r3 * r3 - p.B * (1.0 / 3.0));
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = NT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[s] = red[0];
}

cudaError_t launch_lj_tail(const DevTables& t, int S, double* dev_out, cudaStream_t st) {
    k_lj_tail<<<S, kTailThreads, 0, st>>>(t.ljd, t.n, t.smax, dev_out);
    return cudaGetLastError();
}

// ------------------------------------------------------- common epilogue
template <int P>
__device__ __forceinline__ void store_strip(double* base, int i0, int nx, const double (&v)[P], bool vec_ok) {
    if (vec_ok && i0 + P <= nx) {
#pragma unroll
        for (int p = 0; p < P; p += 2)
            __stcs(reinterpret_cast<double2*>(base + i0 + p), make_double2(v[p], v[p + 1]));
    } else {
#pragma unroll
        for (int p = 0; p < P; ++p)
            if (i0 + p < nx) __stcs(base + i0 + p, v[p]);
    }
}

// ------------------------------------------------------------ FP64 direct
// Launch shape: BX x BY x BZ threads, P x-points per thread, T atoms per tile.
template <int SM, int P, int BX, int BY, int BZ, int T, bool DU, bool DH>
__global__ void __launch_bounds__(BX* BY* BZ) k_direct64(GridD g, Phys ph, const Geo* __restrict__ geo,
                                                          const LJd* __restrict__ lj, int64_t n, Outputs o,
                                                          DevErr* err, long long wlim, int dbg) {
    constexpr int NT = BX * BY * BZ;
    extern __shared__ __align__(16) unsigned char smem[];
    Geo* sgeo = reinterpret_cast<Geo*>(smem);
    LJd* slj = reinterpret_cast<LJd*>(smem + 2 * T * sizeof(Geo));
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * T * sizeof(Geo) + 2 * T * SM * sizeof(LJd));

    const int tid = threadIdx.x;
    const int tx = tid % BX, ty = (tid / BX) % BY, tz = tid / (BX * BY);
    const int i0 = (blockIdx.x * BX + tx) * P, j = blockIdx.y * BY + ty, k = blockIdx.z * BZ + tz;
    double gx[P];
#pragma unroll
    for (int p = 0; p < P; ++p) gx[p] = g.ox + g.h * (double)(i0 + p);
    const double gy = g.oy + g.h * (double)j, gz = g.oz + g.h * (double)k;
    const double rs2 = ph.rs * ph.rs, ieta = 1.0 / ph.eta, a = ph.a, kap = ph.kappa;
    const bool DC = o.c != nullptr;

    double f1[P], fk[P], sc[P], sh[P], lj_[P][SM];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        f1[p] = fk[p] = sc[p] = sh[p] = 0.0;
#pragma unroll
        for (int s = 0; s < SM; ++s) lj_[p][s] = 0.0;
    }
    unsigned hit = 0u;

    const int ntiles = (int)((n + T - 1) / T);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    auto issue = [&](int t) {
        int st = t & 1;
        int cnt = (int)min((int64_t)T, n - (int64_t)t * T);
        uint32_t b1 = cnt * sizeof(Geo), b2 = cnt * SM * sizeof(LJd);
        mbar_expect_tx(&bar[st], b1 + b2);
        bulk_g2s(sgeo + st * T, geo + (int64_t)t * T, b1, &bar[st]);
        bulk_g2s(slj + st * T * SM, lj + (int64_t)t * T * SM, b2, &bar[st]);
    };
    if (tid == 0) {
        // debug hook: without the first copy its wait can only run out
        if (ntiles > 0 && !(dbg & 1)) issue(0);
        if (ntiles > 1) issue(1);
    }
    for (int t = 0; t < ntiles; ++t) {
        const int st = t & 1;
        bool ok = mbar_wait_bounded(&bar[st], (t >> 1) & 1, wlim);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                report_error(err, DEV_TIMEOUT, WHERE_DIRECT);
                // drain the copies still in flight (bounded) before the CTA exits
                for (int u2 = t; u2 < min(t + 2, ntiles); ++u2) mbar_wait_bounded(&bar[u2 & 1], (u2 >> 1) & 1, wlim);
            }
            return;
        }
        const int cnt = (int)min((int64_t)T, n - (int64_t)t * T);
        const Geo* G = sgeo + st * T;
        const LJd* L = slj + st * T * SM;
        for (int aa = 0; aa < cnt; ++aa) {
            const Geo A = G[aa];
            const double dy = gy - A.y, dz = gz - A.z;
            const double dyz2 = dy * dy + dz * dz;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const double dx = gx[p] - A.x;
                const double d2 = fma(dx, dx, dyz2);
                const double ri = d2 > 0.0 ? rsqrt(d2) : 0.0;
                const double qr = A.q * ri;
                f1[p] += qr;
                if (DH) fk[p] += qr * exp(-kap * (d2 * ri));
                if (d2 < rs2) {
                    if (d2 > 0.0) {
                        const double x = d2 * ri * ieta;
                        if (DC) sc[p] += qr * erfc(x);
                        if (DH) sh[p] += qr * exp(-x * x) * (erfcx(x - a) + erfcx(x + a));
                    } else {
                        hit |= 1u << p;
                        if (DC) sc[p] -= A.q * ph.phi_c0;
                        if (DH) sh[p] -= A.q * ph.phi_h0;
                    }
                }
                if (DU) {
                    const double r2i = 1.0 / d2;
                    const double r6 = r2i * r2i * r2i;
#pragma unroll
                    for (int s = 0; s < SM; ++s) {
                        const LJd l = L[aa * SM + s];
                        if (d2 < l.rc2) lj_[p][s] += r6 * (l.A * r6 - l.B);
                    }
                }
            }
        }
        __syncthreads();
        if (tid == 0 && t + 2 < ntiles) issue(t + 2);
    }
    if (j >= g.ny || k >= g.nz || i0 >= g.nx) return;
    const int64_t plane = (int64_t)g.nx * g.ny * g.nz;
    const int64_t row = ((int64_t)k * g.ny + j) * g.nx;
    const bool vec_ok = (g.nx & 1) == 0;
    const double cu0 = ph.k_e, cc0 = -ph.beta * ph.k_e, ch0 = -ph.beta * ph.k_e / (2.0 * ph.eps_r);
#pragma unroll
    for (int s = 0; s < SM; ++s) {
        if (s >= ph.S) break;
        const double qs = ph.qs[s];
        double v[P];
        if (DU) {
#pragma unroll
            for (int p = 0; p < P; ++p) v[p] = (hit >> p & 1u) ? INFINITY : cu0 * qs * f1[p] + lj_[p][s];
            store_strip<P>(o.u + s * plane + row, i0, g.nx, v, vec_ok);
        }
        if (DC) {
#pragma unroll
            for (int p = 0; p < P; ++p) v[p] = cc0 * qs * (f1[p] - sc[p]);
            store_strip<P>(o.c + s * plane + row, i0, g.nx, v, vec_ok);
        }
        if (DH) {
#pragma unroll
            for (int p = 0; p < P; ++p) v[p] = ch0 * qs * (2.0 * ph.ea2 * fk[p] - sh[p]);
            store_strip<P>(o.h + s * plane + row, i0, g.nx, v, vec_ok);
        }
    }
}

// ------------------------------------------------------------ FP32 direct
// Pair terms in FP32 from float-float grid-unit source positions (SrcF): the
// grid coordinates are exact integers, so dx = (i - xh) - xl is exact to half
// an ulp of dx for every nearby atom.  Per-tile FP32 partial sums are folded
// into float-float totals (TwoSum), which carry ~48 bits.
template <int SM, int P, int BX, int BY, int BZ, int T, bool DU, bool DH>
__global__ void __launch_bounds__(BX* BY* BZ) k_direct32(GridD g, Phys ph, const SrcF* __restrict__ srcf,
                                                          const LJf* __restrict__ lj, int64_t n, Outputs o,
                                                          DevErr* err, long long wlim, int dbg) {
    extern __shared__ __align__(16) unsigned char smem[];
    SrcF* ssrc = reinterpret_cast<SrcF*>(smem);
    LJf* slj = reinterpret_cast<LJf*>(smem + 2 * T * sizeof(SrcF));
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * T * sizeof(SrcF) + 2 * T * SM * sizeof(LJf));

    const int tid = threadIdx.x;
    const int tx = tid % BX, ty = (tid / BX) % BY, tz = tid / (BX * BY);
    const int i0 = (blockIdx.x * BX + tx) * P, j = blockIdx.y * BY + ty, k = blockIdx.z * BZ + tz;
    float gx[P];
#pragma unroll
    for (int p = 0; p < P; ++p) gx[p] = (float)(i0 + p);
    const float fy = (float)j, fz = (float)k;
    const float rs2 = (float)((ph.rs / g.h) * (ph.rs / g.h));
    const float xs = (float)(g.h / ph.eta);                            // x = d_grid * xs
    const float kap2 = (float)(-ph.kappa * g.h * 1.4426950408889634);  // e^{-kappa d} = 2^(kap2 d_grid)
    const float a = (float)ph.a;
    const float c0h = (float)(ph.phi_c0 * g.h), h0h = (float)(ph.phi_h0 * g.h);
    const bool DC = o.c != nullptr;

    float f1h[P], f1l[P], fkh[P], fkl[P], sch[P], scl[P], shh[P], shl[P], ljh[P][SM], ljl[P][SM];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        f1h[p] = f1l[p] = fkh[p] = fkl[p] = sch[p] = scl[p] = shh[p] = shl[p] = 0.f;
#pragma unroll
        for (int s = 0; s < SM; ++s) ljh[p][s] = ljl[p][s] = 0.f;
    }
    unsigned hit = 0u;

    const int ntiles = (int)((n + T - 1) / T);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    auto issue = [&](int t) {
        int st = t & 1;
        int cnt = (int)min((int64_t)T, n - (int64_t)t * T);
        uint32_t b1 = cnt * sizeof(SrcF), b2 = cnt * SM * sizeof(LJf);
        mbar_expect_tx(&bar[st], b1 + b2);
        bulk_g2s(ssrc + st * T, srcf + (int64_t)t * T, b1, &bar[st]);
        bulk_g2s(slj + st * T * SM, lj + (int64_t)t * T * SM, b2, &bar[st]);
    };
    if (tid == 0) {
        // debug hook: without the first copy its wait can only run out
        if (ntiles > 0 && !(dbg & 1)) issue(0);
        if (ntiles > 1) issue(1);
    }
    for (int t = 0; t < ntiles; ++t) {
        const int st = t & 1;
        bool ok = mbar_wait_bounded(&bar[st], (t >> 1) & 1, wlim);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                report_error(err, DEV_TIMEOUT, WHERE_DIRECT);
                for (int u2 = t; u2 < min(t + 2, ntiles); ++u2) mbar_wait_bounded(&bar[u2 & 1], (u2 >> 1) & 1, wlim);
            }
            return;
        }
        const int cnt = (int)min((int64_t)T, n - (int64_t)t * T);
        const SrcF* Sx = ssrc + st * T;
        const LJf* L = slj + st * T * SM;
        float p1[P], pk[P], psc[P], psh[P], plj[P][SM];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            p1[p] = pk[p] = psc[p] = psh[p] = 0.f;
#pragma unroll
            for (int s = 0; s < SM; ++s) plj[p][s] = 0.f;
        }
        for (int aa = 0; aa < cnt; ++aa) {
            const float4 g0 = *reinterpret_cast<const float4*>(&Sx[aa].xh);
            const float4 g1 = *reinterpret_cast<const float4*>(&Sx[aa].xl);
            const float dy = (fy - g0.y) - g1.y;
            const float dz = (fz - g0.z) - g1.z;
            const float dyz2 = fmaf(dy, dy, dz * dz);
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float dx = (gx[p] - g0.x) - g1.x;
                const float d2 = fmaf(dx, dx, dyz2);
                const float rr = rsqrt_approx(d2);
                const float ri = d2 > 0.f ? rr : 0.f;
                const float qr = g0.w * ri;
                p1[p] += qr;
                if (DH) pk[p] = fmaf(qr, ex2_approx(kap2 * (d2 * ri)), pk[p]);
                if (d2 < rs2) {
                    if (d2 > 0.f) {
                        const float x = d2 * ri * xs;
                        if (DC) psc[p] = fmaf(qr, erfcf(x), psc[p]);
                        if (DH) psh[p] = fmaf(qr, __expf(-x * x) * (erfcxf(x - a) + erfcxf(x + a)), psh[p]);
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
                        const float4 l = *reinterpret_cast<const float4*>(&L[aa * SM + s]);
                        if (d2 < l.z) plj[p][s] = fmaf(r6, fmaf(l.x, r6, -l.y), plj[p][s]);
                    }
                }
            }
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
            ff_add(f1h[p], f1l[p], p1[p]);
            if (DH) ff_add(fkh[p], fkl[p], pk[p]);
            if (DC) ff_add(sch[p], scl[p], psc[p]);
            if (DH) ff_add(shh[p], shl[p], psh[p]);
            if (DU) {
#pragma unroll
                for (int s = 0; s < SM; ++s) ff_add(ljh[p][s], ljl[p][s], plj[p][s]);
            }
        }
        __syncthreads();
        if (tid == 0 && t + 2 < ntiles) issue(t + 2);
    }
    if (j >= g.ny || k >= g.nz || i0 >= g.nx) return;
    const int64_t plane = (int64_t)g.nx * g.ny * g.nz;
    const int64_t row = ((int64_t)k * g.ny + j) * g.nx;
    const bool vec_ok = (g.nx & 1) == 0;
    const double ih = 1.0 / g.h;
    const double cu0 = ph.k_e * ih, cc0 = -ph.beta * ph.k_e * ih, ch0 = -ph.beta * ph.k_e / (2.0 * ph.eps_r) * ih;
    double F1[P], FK[P], SC[P], SH[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        F1[p] = (double)f1h[p] + (double)f1l[p];
        FK[p] = (double)fkh[p] + (double)fkl[p];
        SC[p] = (double)sch[p] + (double)scl[p];
        SH[p] = (double)shh[p] + (double)shl[p];
    }
#pragma unroll
    for (int s = 0; s < SM; ++s) {
        if (s >= ph.S) break;
        const double qs = ph.qs[s];
        double v[P];
        if (DU) {
#pragma unroll
            for (int p = 0; p < P; ++p)
                v[p] = (hit >> p & 1u) ? INFINITY : cu0 * qs * F1[p] + ((double)ljh[p][s] + (double)ljl[p][s]);
            store_strip<P>(o.u + s * plane + row, i0, g.nx, v, vec_ok);
        }
        if (DC) {
#pragma unroll
            for (int p = 0; p < P; ++p) v[p] = cc0 * qs * (F1[p] - SC[p]);
            store_strip<P>(o.c + s * plane + row, i0, g.nx, v, vec_ok);
        }
        if (DH) {
#pragma unroll
            for (int p = 0; p < P; ++p) v[p] = ch0 * qs * (2.0 * ph.ea2 * FK[p] - SH[p]);
            store_strip<P>(o.h + s * plane + row, i0, g.nx, v, vec_ok);
        }
    }
}

// ---------------------------------------------------------------- launch
namespace {
constexpr int kP = 4, kBX = 8, kBY = 4, kBZ = 4, kT = 64;

template <int SM, bool DU, bool DH>
cudaError_t run_direct(const GridD& g, const Phys& ph, const DevTables& t, int prec, Outputs o, long long wl,
                       int dbg, cudaStream_t st) {
    dim3 grid((g.nx + kBX * kP - 1) / (kBX * kP), (g.ny + kBY - 1) / kBY, (g.nz + kBZ - 1) / kBZ);
    dim3 block(kBX * kBY * kBZ);
    if (prec == RISM_PREC_FP64) {
        size_t sm = 2 * kT * sizeof(Geo) + 2 * kT * SM * sizeof(LJd) + 2 * sizeof(uint64_t);
        auto kern = k_direct64<SM, kP, kBX, kBY, kBZ, kT, DU, DH>;
        raise_dyn_smem(kern, sm);
        kern<<<grid, block, sm, st>>>(g, ph, t.geo, t.ljd, t.n, o, t.err, wl, dbg);
    } else {
        size_t sm = 2 * kT * sizeof(SrcF) + 2 * kT * SM * sizeof(LJf) + 2 * sizeof(uint64_t);
        auto kern = k_direct32<SM, kP, kBX, kBY, kBZ, kT, DU, DH>;
        raise_dyn_smem(kern, sm);
        kern<<<grid, block, sm, st>>>(g, ph, t.srcf, t.ljf, t.n, o, t.err, wl, dbg);
    }
    return cudaGetLastError();
}

template <int SM>
cudaError_t run_direct_sm(const GridD& g, const Phys& ph, const DevTables& t, int prec, Outputs o, long long wl,
                          int dbg, cudaStream_t st) {
    const bool du = o.u != nullptr, dh = o.h != nullptr;
    if (du && dh) return run_direct<SM, true, true>(g, ph, t, prec, o, wl, dbg, st);
    if (du) return run_direct<SM, true, false>(g, ph, t, prec, o, wl, dbg, st);
    if (dh) return run_direct<SM, false, true>(g, ph, t, prec, o, wl, dbg, st);
    return run_direct<SM, false, false>(g, ph, t, prec, o, wl, dbg, st);
}
}  // namespace

int direct_variant_count() { return 1; }

cudaError_t launch_direct(const GridD& g, const Phys& ph, const DevTables& t, int precision, Outputs o,
                          long long wait_limit, int variant, int dbg, cudaStream_t st) {
    (void)variant;
    switch (t.smax) {
        case 2: return run_direct_sm<2>(g, ph, t, precision, o, wait_limit, dbg, st);
        case 4: return run_direct_sm<4>(g, ph, t, precision, o, wait_limit, dbg, st);
        case 8: return run_direct_sm<8>(g, ph, t, precision, o, wait_limit, dbg, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rism
