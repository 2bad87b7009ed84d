// rism_capi.cu -- the extern "C" boundary of librism3d (include/rism3d.h).
//
// Host-side logic only: argument validation, the per-context device tables,
// the physical constants (beta, Debye kappa of eq. (tcf-r), the d -> 0 limits
// of the two asymptotic kernels), dispatch to the kernels and status
// reporting.  Every grid value is computed by the CUDA kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rism_kernels.h"
#include "rism_tree.h"
#include "rism_adjoint.h"
#include "rism_validate.h"
#include "rism_lra.h"
#include "rism_kspace.h"

using namespace rism;

struct rism_ctx {
    rism_grid_desc g{};
    rism_options o{};
    cudaStream_t st = nullptr;
    int device = 0;
    std::string err;

    // host copies of the inputs
    int64_t n = 0;
    int S = 0;
    double qs[kMaxSites] = {}, sigs[kMaxSites] = {}, epss[kMaxSites] = {}, rho[kMaxSites] = {};
    int is_ion[kMaxSites] = {};
    bool have_solute = false, have_solvent = false, dirty = true;
    int64_t tree_calls = 0;  // treecode initializations of this context (the graph path starts at the second)

    // device state
    double* d_raw = nullptr;
    int64_t cap_n = 0;
    int cap_smax = 0;
    DevTables t;
    DevErr* d_err = nullptr;
    DevErr* h_err = nullptr;  // pinned
    double* d_tail = nullptr;
    // the solute, [n][6] x, y, z, q, sigma, eps, in page-locked host memory: uploaded as it stands (by the
    // replayed graph's copy node or an asynchronous copy); every entry point that uploads it synchronises its
    // stream before it returns, so rism_set_solute never overwrites it under a copy of a completed call
    double* h_raw = nullptr;
    int64_t cap_h_raw = 0;
    double* h_tail = nullptr;  // pinned [RISM_MAX_SITES]
    double* d_stage[3] = {nullptr, nullptr, nullptr};
    size_t stage_bytes[3] = {0, 0, 0};
    TreeState* tree = nullptr;
    AdjointState* adj = nullptr;

    rism_info info{};
    Phys ph{};
    GridD gd{};
    int setup_launches = 0;  // kernels launched by the last table rebuild
    cudaEvent_t ev[2] = {nullptr, nullptr};
    // host outputs: one copy stream per output grid, so the device-to-host copies run on several copy engines
    cudaStream_t cp_st[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t cp_fork = nullptr, cp_join[3] = {nullptr, nullptr, nullptr};
    // all-space long-range integral: chunk partials, per-atom sums, totals (device) and the totals' host copy
    double* d_lra_part = nullptr;
    size_t lra_part_cap = 0;
    double2* d_lra_atom = nullptr;
    int64_t lra_atom_cap = 0;
    double* d_lra_tot = nullptr;
    double* h_lra_tot = nullptr;  // pinned [3]
    // the atoms in a spatial order for the pair sum (position -> original index), recomputed for a new solute
    int* h_lra_perm = nullptr;    // pinned [lra_perm_cap]
    int* d_lra_perm = nullptr;
    void* d_lra_src = nullptr;    // the sorted source table
    int64_t lra_perm_cap = 0;
    int64_t lra_perm_version = -1;
    int64_t solute_version = 0;   // incremented by every rism_set_solute
    // reciprocal-space asymptotics: per-atom phase tables and device staging for host outputs
    void* d_ktab = nullptr;
    size_t ktab_bytes = 0;
    double* d_kstage[2] = {nullptr, nullptr};
    size_t kstage_bytes = 0;
};

namespace {

rism_status fail(rism_ctx* c, rism_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

rism_status cuda_fail(rism_ctx* c, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(c, RISM_E_NOMEM, m);
    return fail(c, RISM_E_CUDA, m);
}

int padded_sites(int S) { return S <= 2 ? 2 : (S <= 4 ? 4 : 8); }

rism_status check_options(rism_ctx* c, const rism_options& o) {
    bool unsupported = false;
    const char* m = rism::check_options(o, &unsupported);
    if (m) return fail(c, unsupported ? RISM_E_UNSUPPORTED : RISM_E_INVALID, m);
    return RISM_OK;
}

// Physical constants of the current solvent + options.
void make_phys(rism_ctx* c) {
    Phys& p = c->ph;
    const rism_options& o = c->o;
    p.S = c->S;
    p.beta = 1.0 / (o.k_B * o.T);
    p.k_e = o.k_e;
    p.eps_r = o.eps_r;
    p.eta = o.eta;
    if (o.kappa >= 0.0) {
        p.kappa = o.kappa;
    } else {
        double acc = 0.0;
        for (int s = 0; s < c->S; ++s)
            if (c->is_ion[s]) acc += c->rho[s] * c->qs[s] * c->qs[s];
        p.kappa = std::sqrt(4.0 * M_PI * p.beta * p.k_e * acc / p.eps_r);
    }
    p.a = 0.5 * p.kappa * p.eta;
    p.ea2 = std::exp(p.a * p.a);
    p.rs = o.r_short > 0.0 ? o.r_short : (o.precision == RISM_PREC_FP64 ? 6.0 : 5.0) * p.eta;
    p.phi_c0 = 2.0 / (p.eta * std::sqrt(M_PI));
    p.phi_h0 = 2.0 * (p.phi_c0 - p.kappa * p.ea2 * std::erfc(p.a));
    for (int s = 0; s < kMaxSites; ++s) p.qs[s] = s < c->S ? c->qs[s] : 0.0;
}

// Allocations of the per-solute tables and the physical constants; no kernel
// is launched (also used before a graph capture).
rism_status reserve_tables(rism_ctx* c) {
    cudaError_t e;
    const int smax = padded_sites(c->S);
    if (c->n > c->cap_n || smax != c->cap_smax) {
        cudaFree(c->d_raw);
        cudaFree(c->t.geo);
        cudaFree(c->t.srcf);
        cudaFree(c->t.ljd);
        cudaFree(c->t.ljf);
        c->d_raw = nullptr;
        c->t.geo = nullptr;
        c->t.srcf = nullptr;
        c->t.ljd = nullptr;
        c->t.ljf = nullptr;
        c->cap_n = 0;
        int64_t n = c->n > 0 ? c->n : 1;
        if ((e = cudaMalloc(&c->d_raw, sizeof(double) * 6 * n)) != cudaSuccess ||
            (e = cudaMalloc(&c->t.geo, sizeof(Geo) * n)) != cudaSuccess ||
            (e = cudaMalloc(&c->t.srcf, sizeof(SrcF) * n)) != cudaSuccess ||
            (e = cudaMalloc(&c->t.ljd, sizeof(LJd) * n * smax)) != cudaSuccess ||
            (e = cudaMalloc(&c->t.ljf, sizeof(LJf) * n * smax)) != cudaSuccess)
            return cuda_fail(c, e, "allocating solute tables");
        c->cap_n = n;
        c->cap_smax = smax;
    }
    c->t.n = c->n;
    c->t.smax = smax;
    c->t.err = c->d_err;
    c->gd = GridD{c->g.nx, c->g.ny, c->g.nz, c->g.h, c->g.origin[0], c->g.origin[1], c->g.origin[2]};
    make_phys(c);
    return RISM_OK;
}

rism_status ensure_tables(rism_ctx* c) {
    if (!c->dirty) return RISM_OK;
    cudaError_t e;
    rism_status rs = reserve_tables(c);
    if (rs != RISM_OK) return rs;
    const int smax = c->t.smax;
    if (c->n > 0) {
        if ((e = cudaMemcpyAsync(c->d_raw, c->h_raw, sizeof(double) * 6 * c->n, cudaMemcpyHostToDevice,
                                 c->st)) != cudaSuccess)
            return cuda_fail(c, e, "uploading solute");
        if ((e = launch_setup(c->d_raw, c->n, c->S, smax, c->sigs, c->epss, c->o.lj_mode, c->o.lj_rcut,
                              c->o.lj_tol, c->gd, c->t, c->st)) != cudaSuccess)
            return cuda_fail(c, e, "setup kernel");
        c->setup_launches += 1;
    }
    if (c->o.method == RISM_METHOD_TREECODE) {
        rism_status s = tree_prepare(c->tree, c->t, c->gd, c->ph, c->o, c->st, c->err);
        if (s != RISM_OK) return s;
    }
    c->dirty = false;
    return RISM_OK;
}

rism_status check_device_error(rism_ctx* c) {
    cudaError_t e = cudaMemcpyAsync(c->h_err, c->d_err, sizeof(DevErr), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "synchronising");
    if (c->h_err->code != DEV_OK) {
        int code = c->h_err->code, where = c->h_err->where;
        DevErr zero{0, 0};
        cudaMemcpyAsync(c->d_err, &zero, sizeof(DevErr), cudaMemcpyHostToDevice, c->st);
        cudaStreamSynchronize(c->st);
        char buf[128];
        snprintf(buf, sizeof buf, "device wait gave up (code %d, kernel %d)", code, where);
        return fail(c, code == DEV_TIMEOUT ? RISM_E_TIMEOUT : RISM_E_CUDA, buf);
    }
    return RISM_OK;
}

}  // namespace

extern "C" {

void rism_default_options(rism_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->method = RISM_METHOD_TREECODE;
    o->precision = RISM_PREC_FP32;
    o->degree = 8;
    o->theta = 0.7;
    o->leaf = 64;
    o->lj_mode = RISM_LJ_RCUT;
    o->lj_rcut = 9.0;
    o->lj_tol = 1e-6;
    o->eta = 1.0;
    o->T = 298.0;
    o->eps_r = 78.44;
    o->kappa = -1.0;
    o->k_e = 332.0522173;
    o->k_B = 0.0019872041;
    o->r_short = 0.0;
    o->autotune = 0;
    o->wait_limit = 1LL << 24;
    o->target_proxies = 1;
    o->approx = RISM_APPROX_BARYCENTRIC;
}

rism_status rism_grid_create(const rism_grid_desc* grid, const rism_options* opts, void* stream, rism_ctx** out) {
    if (!grid || !out) return RISM_E_INVALID;
    *out = nullptr;
    if (check_grid_desc(*grid)) return RISM_E_INVALID;
    rism_ctx* c = new (std::nothrow) rism_ctx;
    if (!c) return RISM_E_NOMEM;
    c->g = *grid;
    if (opts) c->o = *opts;
    else rism_default_options(&c->o);
    const rism_status cs = check_options(c, c->o);
    if (cs != RISM_OK) {
        delete c;
        return cs;
    }
    c->st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(DevErr));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_err, sizeof(DevErr));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tail, sizeof(double) * kMaxSites);
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_tail, sizeof(double) * kMaxSites);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(DevErr), c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        rism_status s = (e == cudaErrorMemoryAllocation) ? RISM_E_NOMEM : RISM_E_CUDA;
        rism_destroy(c);
        return s;
    }
    c->tree = tree_create();
    c->adj = adjoint_create();
    c->info.batch[0] = c->info.batch[1] = c->info.batch[2] = 0;
    *out = c;
    return RISM_OK;
}

rism_status rism_set_solute(rism_ctx* c, int64_t n, const double* xyz, const double* q, const double* sigma,
                            const double* eps) {
    if (!c) return RISM_E_INVALID;
    if (const char* m = check_host_solute(n, xyz, q, sigma, eps)) return fail(c, RISM_E_INVALID, m);
    if (n > c->cap_h_raw) {
        cudaFreeHost(c->h_raw);
        c->h_raw = nullptr;
        c->cap_h_raw = 0;
        c->n = 0;
        c->have_solute = false;
        const cudaError_t e = cudaMallocHost(&c->h_raw, sizeof(double) * 6 * n);
        if (e != cudaSuccess) return cuda_fail(c, e, "page-locked solute buffer");
        c->cap_h_raw = n;
    }
    double* raw = c->h_raw;
    for (int64_t i = 0; i < n; ++i) {
        raw[6 * i + 0] = xyz[3 * i + 0];
        raw[6 * i + 1] = xyz[3 * i + 1];
        raw[6 * i + 2] = xyz[3 * i + 2];
        raw[6 * i + 3] = q[i];
        raw[6 * i + 4] = sigma[i];
        raw[6 * i + 5] = eps[i];
    }
    c->n = n;
    c->have_solute = true;
    c->dirty = true;
    ++c->solute_version;
    c->err.clear();
    return RISM_OK;
}

rism_status rism_set_solvent(rism_ctx* c, int32_t nsite, const double* q, const double* sigma, const double* eps,
                             const double* rho, const int32_t* is_ion) {
    if (!c) return RISM_E_INVALID;
    if (const char* m = check_solvent(nsite, q, sigma, eps, rho)) return fail(c, RISM_E_INVALID, m);
    c->S = nsite;
    for (int s = 0; s < kMaxSites; ++s) {
        c->qs[s] = s < nsite ? q[s] : 0.0;
        c->sigs[s] = s < nsite ? sigma[s] : 0.0;
        c->epss[s] = s < nsite ? eps[s] : 0.0;
        c->rho[s] = (s < nsite && rho) ? rho[s] : 0.0;
        c->is_ion[s] = (s < nsite && is_ion) ? (is_ion[s] != 0) : 0;
    }
    c->have_solvent = true;
    c->dirty = true;
    c->err.clear();
    make_phys(c);  // beta, kappa, r_short are reported by rism_get_info from here on
    return RISM_OK;
}

namespace {

// z slabs of the treecode's far and near fields when the outputs go to host memory: the copy of a slab's planes
// (at the host link's rate) overlaps the evaluation of the slabs after it.
constexpr int kOutSlabs = 4;
static_assert(kOutSlabs <= kOutSlabsMax, "slab events of the tree state");

// Device staging -> caller's host buffers for the outputs staged in device memory: each grid on its own stream
// (forked from and joined back to the context's stream), so the copies overlap on several copy engines.  When
// the treecode's far and near fields ran in z slabs, each slab's planes of every site are copied as soon as the
// slab's event has fired, while the later slabs are still being evaluated; otherwise the whole grids after the
// step.
rism_status copy_outputs(rism_ctx* c, double* const (&user)[3], double* const (&dev)[3], const bool (&staged)[3],
                         size_t bytes) {
    cudaError_t e = cudaSuccess;
    int nhost = 0;
    for (int k = 0; k < 3; ++k) nhost += staged[k];
    if (nhost == 0) return RISM_OK;
    if (!c->cp_fork) {
        for (int k = 0; k < 3 && e == cudaSuccess; ++k)
            if ((e = cudaStreamCreateWithFlags(&c->cp_st[k], cudaStreamNonBlocking)) == cudaSuccess)
                e = cudaEventCreateWithFlags(&c->cp_join[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->cp_fork, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(c, e, "copy streams");
    }
    int z[kOutSlabsMax][2];
    cudaEvent_t sev[kOutSlabsMax];
    const int ns = (c->o.method == RISM_METHOD_TREECODE && c->tree) ? tree_slabs(c->tree, c->gd, z, sev) : 0;
    const size_t plane = (size_t)c->g.nx * c->g.ny, M = plane * c->g.nz;
    if (ns == 0 && (e = cudaEventRecord(c->cp_fork, c->st)) != cudaSuccess)
        return cuda_fail(c, e, "copying result to host");
    for (int k = 0; k < 3; ++k) {
        if (!staged[k]) continue;
        cudaStream_t cs = c->cp_st[k];
        if (ns == 0) {
            if ((e = cudaStreamWaitEvent(cs, c->cp_fork, 0)) != cudaSuccess ||
                (e = cudaMemcpyAsync(user[k], dev[k], bytes, cudaMemcpyDeviceToHost, cs)) != cudaSuccess)
                return cuda_fail(c, e, "copying result to host");
        } else {
            for (int j = 0; j < ns; ++j) {
                if ((e = cudaStreamWaitEvent(cs, sev[j], 0)) != cudaSuccess) return cuda_fail(c, e, "slab copy");
                if (z[j][1] <= z[j][0]) continue;
                const size_t off = (size_t)z[j][0] * plane, cnt = (size_t)(z[j][1] - z[j][0]) * plane;
                for (int s = 0; s < c->S; ++s)
                    if ((e = cudaMemcpyAsync(user[k] + s * M + off, dev[k] + s * M + off, cnt * sizeof(double),
                                             cudaMemcpyDeviceToHost, cs)) != cudaSuccess)
                        return cuda_fail(c, e, "slab copy");
            }
        }
        if ((e = cudaEventRecord(c->cp_join[k], cs)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(c->st, c->cp_join[k], 0)) != cudaSuccess)
            return cuda_fail(c, e, "copying result to host");
    }
    return RISM_OK;
}

}  // namespace

rism_status rism_init(rism_ctx* c, double* u, double* c_lr, double* h_lr, double* lj_tail) {
    if (!c) return RISM_E_INVALID;
    if (!c->have_solute || !c->have_solvent) return fail(c, RISM_E_STATE, "set_solute and set_solvent first");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    rism_status s = RISM_OK;
    if (h_lr && !(c->ph.kappa > 0.0)) return fail(c, RISM_E_INVALID, "h_lr needs kappa > 0 (ionic solvent)");
    const int64_t M = (int64_t)c->g.nx * c->g.ny * c->g.nz;
    const size_t bytes = sizeof(double) * (size_t)c->S * (size_t)M;
    double* user[3] = {u, c_lr, h_lr};
    double* dev[3] = {nullptr, nullptr, nullptr};
    bool staged[3] = {false, false, false};  // computed into a device buffer and copied to the host buffer
    bool host_out = false;
    for (int k = 0; k < 3; ++k) {
        if (!user[k]) continue;
        if (is_device_ptr(user[k])) {
            dev[k] = user[k];
        } else {
            // host memory (page-locked or not): computed into a device buffer, copied back.  Kernel stores
            // straight into page-locked host memory measured slower here than the copy engines.
            host_out = true;
            staged[k] = true;
            if (c->stage_bytes[k] < bytes) {
                cudaFree(c->d_stage[k]);
                c->d_stage[k] = nullptr;
                c->stage_bytes[k] = 0;
                if ((e = cudaMalloc(&c->d_stage[k], bytes)) != cudaSuccess) return cuda_fail(c, e, "staging buffer");
                c->stage_bytes[k] = bytes;
            }
            dev[k] = c->d_stage[k];
        }
    }
    Outputs o{dev[0], dev[1], dev[2]};
    // host outputs: the treecode's far and near fields run in z slabs whose copies overlap the rest of the
    // evaluation
    if (c->o.method == RISM_METHOD_TREECODE && c->tree &&
        (s = tree_set_slabs(c->tree, host_out ? kOutSlabs : 1, c->err)) != RISM_OK)
        return fail(c, s, c->err);
    // Graph-replayed step (treecode, new solute coordinates, from the context's second treecode call on; host
    // outputs use the staging buffers): solute upload from pinned memory, tables, tree, lists and evaluation in
    // one launch.
    const bool any_out = o.u || o.c || o.h;
    if (c->o.method == RISM_METHOD_TREECODE && any_out) ++c->tree_calls;
    if (c->o.method == RISM_METHOD_TREECODE && c->dirty && c->n > 0 && any_out && c->tree_calls > 1) {
        if ((s = reserve_tables(c)) != RISM_OK) return s;
        const bool tail = lj_tail && c->o.lj_mode != RISM_LJ_NONE;
        SoluteStep step{c->h_raw, c->d_raw, c->n, c->sigs, c->epss, c->o.lj_mode, c->o.lj_rcut, c->o.lj_tol,
                        tail ? c->d_tail : nullptr, c->h_tail};
        c->info.eval_ms = 0.f;
        bool used = false;
        s = tree_graph_step(c->tree, c->t, c->gd, c->ph, c->o, o, step, c->st, c->err, c->info, used);
        if (s != RISM_OK) return s;
        if (used) {
            // host outputs: the copies go out now, slab by slab as the replay completes them (a retry below
            // evaluates and copies again)
            rism_status st = host_out ? copy_outputs(c, user, dev, staged, bytes) : RISM_OK;
            if (st == RISM_OK) st = check_device_error(c);  // synchronises the stream, the copies included
            bool retry = false;
            if (st == RISM_OK) st = tree_post(c->tree, c->info, retry, c->err);
            if (st != RISM_OK) return st;
            if (!retry) {
                if (lj_tail)
                    for (int k = 0; k < c->S; ++k) lj_tail[k] = tail ? c->h_tail[k] : 0.0;
                c->dirty = false;
                c->setup_launches = 0;
                if (c->o.debug_flags & 2) c->info.eval_ms = c->info.box_ms + c->info.far_ms + c->info.near_ms;
                return RISM_OK;
            }
            // a list outgrew its slots (now enlarged): rebuild through the regular path below
        }
    }
    s = ensure_tables(c);
    if (s != RISM_OK) return s;
    c->info.launches = c->setup_launches;
    c->setup_launches = 0;
    c->info.eval_ms = 0.f;
    if (o.u || o.c || o.h) {
        const bool timed = (c->o.debug_flags & 2) != 0;
        if (timed) {
            if (!c->ev[0]) {
                cudaEventCreate(&c->ev[0]);
                cudaEventCreate(&c->ev[1]);
            }
            cudaEventRecord(c->ev[0], c->st);
        }
        if (c->o.method == RISM_METHOD_DIRECT) {
            e = launch_direct(c->gd, c->ph, c->t, c->o.precision, o, c->o.wait_limit, c->info.kernel_variant,
                              c->o.debug_flags, c->st);
            if (e != cudaSuccess) return cuda_fail(c, e, "direct kernel");
            c->info.direct_pairs = M * c->n;
            c->info.proxy_pairs = 0;
            c->info.near_pairs = 0;
            c->info.cp_pairs = 0;
            c->info.tree_boxes = 0;
            c->info.near_tested = c->info.lj_pairs = c->info.sr_pairs = 0;
            c->info.box_ms = 0.f;
            c->info.launches += 1;
        } else {
            s = tree_eval(c->tree, c->t, c->gd, c->ph, c->o, o, c->st, c->err, c->info);
            if (s != RISM_OK) return s;
        }
        if (timed) cudaEventRecord(c->ev[1], c->st);
    }
    if (lj_tail) {
        if (c->o.lj_mode == RISM_LJ_NONE || c->n == 0) {
            for (int k = 0; k < c->S; ++k) lj_tail[k] = 0.0;
        } else {
            if ((e = launch_lj_tail(c->t, c->S, c->d_tail, c->st)) != cudaSuccess) return cuda_fail(c, e, "lj tail");
            if ((e = cudaMemcpyAsync(lj_tail, c->d_tail, sizeof(double) * c->S, cudaMemcpyDeviceToHost, c->st)) !=
                cudaSuccess)
                return cuda_fail(c, e, "lj tail copy");
        }
    }
    if ((s = copy_outputs(c, user, dev, staged, bytes)) != RISM_OK) return s;
    (void)host_out;
    if (lj_tail && c->o.lj_mode != RISM_LJ_NONE && c->n > 0) c->info.launches += 1;
    // Status of the device-side bounded waits: synchronise and read the error word.
    rism_status st = check_device_error(c);
    if (st == RISM_OK && c->o.method == RISM_METHOD_TREECODE && (o.u || o.c || o.h)) {
        bool retry = false;
        st = tree_post(c->tree, c->info, retry, c->err);
        // a list outgrew its slots (now enlarged): rebuild the lists and evaluate again.  A truncated pass-down
        // list hides the length of the lists below it, so growth can take more than one round.
        for (int attempt = 0; attempt < 4 && st == RISM_OK && retry; ++attempt) {
            st = tree_prepare(c->tree, c->t, c->gd, c->ph, c->o, c->st, c->err);
            if (st == RISM_OK) st = tree_eval(c->tree, c->t, c->gd, c->ph, c->o, o, c->st, c->err, c->info);
            if (st == RISM_OK) st = copy_outputs(c, user, dev, staged, bytes);
            if (st == RISM_OK) st = check_device_error(c);
            if (st == RISM_OK) st = tree_post(c->tree, c->info, retry, c->err);
        }
        if (st == RISM_OK && retry) st = fail(c, RISM_E_NOMEM, "list slots kept growing (" + c->err + ")");
    }
    if (st == RISM_OK && (c->o.debug_flags & 2) && c->ev[0] && (o.u || o.c || o.h))
        cudaEventElapsedTime(&c->info.eval_ms, c->ev[0], c->ev[1]);
    return st;
}

rism_status rism_potential(rism_ctx* c, double* u, double* lj_tail) {
    return rism_init(c, u, nullptr, nullptr, lj_tail);
}

rism_status rism_asymptotics(rism_ctx* c, double* c_lr, double* h_lr) {
    return rism_init(c, nullptr, c_lr, h_lr, nullptr);
}

rism_status rism_potential_backward(rism_ctx* c, const double* g_u, const double* g_c, const double* g_h,
                                    double* d_xyz, double* d_q, double* d_sigma, double* d_eps) {
    if (!c) return RISM_E_INVALID;
    if (!c->have_solute || !c->have_solvent) return fail(c, RISM_E_STATE, "set_solute and set_solvent first");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    const void* ins[3] = {g_u, g_c, g_h};
    for (const void* p : ins)
        if (p && !is_device_ptr(p)) return fail(c, RISM_E_INVALID, "cotangents must be device memory");
    void* outs[4] = {d_xyz, d_q, d_sigma, d_eps};
    for (void* p : outs)
        if (p && !is_device_ptr(p)) return fail(c, RISM_E_INVALID, "gradient outputs must be device memory");
    rism_status s = ensure_tables(c);
    if (s != RISM_OK) return s;
    if (g_h && !(c->ph.kappa > 0.0)) g_h = nullptr;  // h is identically zero without ions
    s = adjoint_run(c->adj, c->tree, c->t, c->gd, c->ph, c->o, c->d_raw, c->sigs, c->epss, g_u, g_c, g_h, d_xyz,
                    d_q, d_sigma, d_eps, c->st, c->err);
    if (s != RISM_OK) return s;
    return check_device_error(c);
}

rism_status rism_potential_batched(rism_ctx* const* ctxs, int32_t count, double* const* u, double* const* c_lr,
                                   double* const* h_lr) {
    if (!ctxs || count < 1) return RISM_E_INVALID;
    rism_ctx* c0 = ctxs[0];
    if (!c0) return RISM_E_INVALID;
    if (c0->o.method != RISM_METHOD_TREECODE || c0->o.precision != RISM_PREC_FP32)
        return fail(c0, RISM_E_UNSUPPORTED, "the batched launch runs the FP32 treecode");
    cudaError_t e = cudaSetDevice(c0->device);
    if (e != cudaSuccess) return cuda_fail(c0, e, "cudaSetDevice");
    std::vector<BatchItem> items((size_t)count);
    for (int b = 0; b < count; ++b) {
        rism_ctx* c = ctxs[b];
        if (!c) return fail(c0, RISM_E_INVALID, "NULL context in batch");
        for (int k = 0; k < b; ++k)
            if (ctxs[k] == c) return fail(c0, RISM_E_INVALID, "a context appears twice in the batch");
        if (!c->have_solute || !c->have_solvent) return fail(c0, RISM_E_STATE, "set_solute and set_solvent first");
        if (c->o.method != c0->o.method || c->o.precision != c0->o.precision ||
            padded_sites(c->S) != padded_sites(c0->S) || c->device != c0->device || c->o.degree != c0->o.degree)
            return fail(c0, RISM_E_INVALID, "batched contexts must share device, method, precision, degree and sites");
        double* uu = u ? u[b] : nullptr;
        double* cc = c_lr ? c_lr[b] : nullptr;
        double* hh = h_lr ? h_lr[b] : nullptr;
        if ((uu != nullptr) != (u && u[0]) || (cc != nullptr) != (c_lr && c_lr[0]) ||
            (hh != nullptr) != (h_lr && h_lr[0]))
            return fail(c0, RISM_E_INVALID, "every solute of a batch must request the same outputs");
        if (!uu && !cc && !hh) return fail(c0, RISM_E_INVALID, "no output requested");
        if (hh && !(c->ph.kappa > 0.0)) return fail(c0, RISM_E_INVALID, "h_lr needs kappa > 0");
        const double* ptrs[3] = {uu, cc, hh};
        for (const double* p : ptrs)
            if (p && !is_device_ptr(p)) return fail(c0, RISM_E_INVALID, "batched outputs must be device memory");
        // allocations and the solute upload happen here, outside the captured graph
        rism_status s = reserve_tables(c);
        if (s != RISM_OK) return fail(c0, s, c->err);
        if (c->n > 0 && (e = cudaMemcpyAsync(c->d_raw, c->h_raw, sizeof(double) * 6 * c->n,
                                             cudaMemcpyHostToDevice, c0->st)) != cudaSuccess)
            return cuda_fail(c0, e, "uploading solute");
        BatchItem it;
        it.tree = c->tree;
        it.t = &c->t;
        it.g = c->gd;
        it.ph = c->ph;
        it.o = Outputs{uu, cc, hh};
        it.raw = c->d_raw;
        for (int k = 0; k < kMaxSites; ++k) {
            it.sig_s[k] = c->sigs[k];
            it.eps_s[k] = c->epss[k];
        }
        it.lj_mode = c->o.lj_mode;
        it.lj_rcut = c->o.lj_rcut;
        it.lj_tol = c->o.lj_tol;
        items[b] = it;
    }
    rism_status s = RISM_OK;
    for (int attempt = 0; attempt < 3; ++attempt) {
        bool retry = false;
        s = batch_eval(items, c0->o, c0->st, c0->d_err, c0->err, retry);
        if (s != RISM_OK) return s;
        s = check_device_error(c0);
        if (s != RISM_OK) return s;
        bool again = false;
        for (int b = 0; b < count; ++b) {
            s = tree_post(ctxs[b]->tree, ctxs[b]->info, retry, c0->err);
            if (s != RISM_OK) return s;
            again = again || retry;
        }
        if (!again) {
            // the tables now match the uploaded solutes; the tree state is not reusable by rism_init
            // without a rebuild (its batch shape is the batch's), so mark every context dirty
            for (int b = 0; b < count; ++b) ctxs[b]->dirty = true;
            return RISM_OK;
        }
    }
    return fail(c0, RISM_E_NOMEM, "list buffers kept growing");
}

namespace {

uint32_t spread10(uint32_t v) {  // the 10 low bits of v to every third bit
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Spatial order of the atoms for the all-space pair sum: cells of about 32 atoms over the atoms' bounding box,
// the cells in Morton order, the atoms of a cell in index order (a stable counting sort, O(n)).  A warp then
// takes nearby targets and a tile nearby sources, so the costly short-range branch of the pair term is taken by
// whole warps or by none.  perm[k] = original index of the atom at position k.
void lra_order(const double* raw, int64_t n, int* perm) {
    double lo[3] = {raw[0], raw[1], raw[2]}, hi[3] = {raw[0], raw[1], raw[2]};
    for (int64_t i = 1; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], raw[6 * i + d]);
            hi[d] = std::max(hi[d], raw[6 * i + d]);
        }
    double ext[3], vol = 1.0;
    for (int d = 0; d < 3; ++d) {
        ext[d] = std::max(hi[d] - lo[d], 1e-6);
        vol *= ext[d];
    }
    const double side = std::cbrt(vol / (double)std::max<int64_t>(1, n / 32));
    int nc[3];
    for (int d = 0; d < 3; ++d) nc[d] = std::max(1, std::min(1024, (int)std::ceil(ext[d] / side)));
    const int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    std::vector<uint64_t> key((size_t)ncell);
    for (int z = 0; z < nc[2]; ++z)
        for (int y = 0; y < nc[1]; ++y)
            for (int x = 0; x < nc[0]; ++x) {
                const uint64_t m = spread10((uint32_t)x) | (spread10((uint32_t)y) << 1) | (spread10((uint32_t)z) << 2);
                const int64_t lin = ((int64_t)z * nc[1] + y) * nc[0] + x;
                key[(size_t)lin] = (m << 32) | (uint64_t)lin;
            }
    std::sort(key.begin(), key.end());
    std::vector<int> rank((size_t)ncell), start((size_t)ncell + 1, 0);
    for (int64_t r = 0; r < ncell; ++r) rank[(size_t)(key[(size_t)r] & 0xffffffffu)] = (int)r;
    std::vector<int> cell((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        int cc[3];
        for (int d = 0; d < 3; ++d)
            cc[d] = std::min(nc[d] - 1, std::max(0, (int)((raw[6 * i + d] - lo[d]) / side)));
        cell[(size_t)i] = rank[(size_t)(((int64_t)cc[2] * nc[1] + cc[1]) * nc[0] + cc[0])];
        ++start[(size_t)cell[(size_t)i] + 1];
    }
    for (int64_t r = 0; r < ncell; ++r) start[(size_t)r + 1] += start[(size_t)r];
    for (int64_t i = 0; i < n; ++i) perm[start[(size_t)cell[(size_t)i]]++] = (int)i;
}

}  // namespace

rism_status rism_lra_integral(rism_ctx* c, double* T, double* atom_sums) {
    if (!c) return RISM_E_INVALID;
    if (!T) return fail(c, RISM_E_INVALID, "T (host [S]) is required");
    if (!c->have_solute || !c->have_solvent) return fail(c, RISM_E_STATE, "set_solute and set_solvent first");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    const int64_t n = c->n;
    if (!(c->ph.kappa > 0.0) || n == 0) {
        // no ionic screening: h^lr vanishes and so does the integral
        for (int s = 0; s < c->S; ++s) T[s] = 0.0;
        if (atom_sums && n > 0) {
            if (is_device_ptr(atom_sums)) {
                if ((e = cudaMemsetAsync(atom_sums, 0, sizeof(double) * 2 * n, c->st)) != cudaSuccess)
                    return cuda_fail(c, e, "clearing atom sums");
            } else {
                std::memset(atom_sums, 0, sizeof(double) * 2 * n);
            }
        }
        return RISM_OK;
    }
    rism_status s = ensure_tables(c);
    if (s != RISM_OK) return s;
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device)) != cudaSuccess)
        return cuda_fail(c, e, "device attribute");
    const size_t need = lra_scratch_doubles(n, sms);
    if (need > c->lra_part_cap) {
        cudaFree(c->d_lra_part);
        c->d_lra_part = nullptr;
        c->lra_part_cap = 0;
        if ((e = cudaMalloc(&c->d_lra_part, sizeof(double) * need)) != cudaSuccess)
            return cuda_fail(c, e, "LRA scratch");
        c->lra_part_cap = need;
    }
    if (n > c->lra_atom_cap) {
        cudaFree(c->d_lra_atom);
        c->d_lra_atom = nullptr;
        c->lra_atom_cap = 0;
        if ((e = cudaMalloc(&c->d_lra_atom, sizeof(double2) * n)) != cudaSuccess)
            return cuda_fail(c, e, "LRA atom sums");
        c->lra_atom_cap = n;
    }
    if (!c->d_lra_tot) {
        if ((e = cudaMalloc(&c->d_lra_tot, sizeof(double) * 3)) != cudaSuccess ||
            (e = cudaMallocHost(&c->h_lra_tot, sizeof(double) * 3)) != cudaSuccess)
            return cuda_fail(c, e, "LRA totals");
    }
    if (n > c->lra_perm_cap) {
        cudaFree(c->d_lra_perm);
        cudaFree(c->d_lra_src);
        cudaFreeHost(c->h_lra_perm);
        c->d_lra_perm = nullptr;
        c->d_lra_src = nullptr;
        c->h_lra_perm = nullptr;
        c->lra_perm_cap = 0;
        c->lra_perm_version = -1;
        if ((e = cudaMalloc(&c->d_lra_perm, sizeof(int) * n)) != cudaSuccess ||
            (e = cudaMalloc(&c->d_lra_src, sizeof(SrcF) * n)) != cudaSuccess ||
            (e = cudaMallocHost(&c->h_lra_perm, sizeof(int) * n)) != cudaSuccess)
            return cuda_fail(c, e, "LRA atom order");
        c->lra_perm_cap = n;
    }
    if (c->lra_perm_version != c->solute_version) {  // a new solute: its spatial order
        lra_order(c->h_raw, n, c->h_lra_perm);
        if ((e = cudaMemcpyAsync(c->d_lra_perm, c->h_lra_perm, sizeof(int) * n, cudaMemcpyHostToDevice, c->st)) !=
            cudaSuccess)
            return cuda_fail(c, e, "LRA atom order upload");
        c->lra_perm_version = c->solute_version;
    }
    if ((e = launch_lra(c->t, c->gd, c->ph, sms, c->d_lra_perm, static_cast<SrcF*>(c->d_lra_src), c->d_lra_part,
                        c->d_lra_atom, c->d_lra_tot, c->o.wait_limit, c->st)) != cudaSuccess)
        return cuda_fail(c, e, "LRA kernels");
    if ((e = cudaMemcpyAsync(c->h_lra_tot, c->d_lra_tot, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->st)) !=
        cudaSuccess)
        return cuda_fail(c, e, "LRA totals copy");
    if (atom_sums &&
        (e = cudaMemcpyAsync(atom_sums, c->d_lra_atom, sizeof(double2) * n, cudaMemcpyDefault, c->st)) != cudaSuccess)
        return cuda_fail(c, e, "LRA atom sums copy");
    if ((s = check_device_error(c)) != RISM_OK) return s;  // synchronises the stream
    const double Shh = c->h_lra_tot[0], Shc = c->h_lra_tot[1], Q = c->h_lra_tot[2];
    for (int k = 0; k < c->S; ++k) {
        const double A = -c->ph.beta * c->ph.k_e * c->qs[k] / (2.0 * c->ph.eps_r);
        const double B = -c->ph.beta * c->ph.k_e * c->qs[k];
        const double theta = (Q * c->qs[k] > 0.0) ? 1.0 : 0.0;
        T[k] = 0.5 * theta * A * A * Shh - 0.5 * A * B * Shc;
    }
    c->info.launches = 4;
    return RISM_OK;
}

rism_status rism_asymptotics_k(rism_ctx* c, double k_tol, double* c_k, double* h_k, double* k_cut) {
    if (!c) return RISM_E_INVALID;
    if (!c->have_solute || !c->have_solvent) return fail(c, RISM_E_STATE, "set_solute and set_solvent first");
    if (!std::isfinite(k_tol)) return fail(c, RISM_E_INVALID, "k_tol must be finite");
    if (h_k && !(c->ph.kappa > 0.0)) return fail(c, RISM_E_INVALID, "h_k needs kappa > 0 (ionic solvent)");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    KspaceSetup ks;
    ks.S = c->S;
    ks.beta = c->ph.beta;
    ks.k_e = c->ph.k_e;
    ks.eps_r = c->ph.eps_r;
    ks.eta = c->ph.eta;
    ks.kappa = c->ph.kappa;
    ks.qmax = 0.0;
    for (int k = 0; k < kMaxSites; ++k) {
        ks.qs[k] = k < c->S ? c->qs[k] : 0.0;
        if (k < c->S) ks.qmax = std::max(ks.qmax, std::fabs(c->qs[k]));
    }
    ks.qabs = 0.0;
    for (int64_t i = 0; i < c->n; ++i) ks.qabs += std::fabs(c->h_raw[6 * i + 3]);
    ks.kcut = k_tol > 0.0 ? kspace_kcut(ks, k_tol) : 0.0;
    if (k_cut) *k_cut = ks.kcut;
    if (!c_k && !h_k) return RISM_OK;
    rism_status s = ensure_tables(c);
    if (s != RISM_OK) return s;
    const size_t bytes = sizeof(double) * 2 * (size_t)c->S * (size_t)c->g.nz * c->g.ny * (c->g.nx / 2 + 1);
    double* user[2] = {c_k, h_k};
    double* dev[2] = {nullptr, nullptr};
    bool host = false;
    for (int k = 0; k < 2; ++k) {
        if (!user[k]) continue;
        if (is_device_ptr(user[k])) {
            dev[k] = user[k];
            continue;
        }
        host = true;
        if (c->kstage_bytes < bytes) {
            cudaFree(c->d_kstage[0]);
            cudaFree(c->d_kstage[1]);
            c->d_kstage[0] = c->d_kstage[1] = nullptr;
            c->kstage_bytes = 0;
            if ((e = cudaMalloc(&c->d_kstage[0], bytes)) != cudaSuccess ||
                (e = cudaMalloc(&c->d_kstage[1], bytes)) != cudaSuccess)
                return cuda_fail(c, e, "k-space staging buffer");
            c->kstage_bytes = bytes;
        }
        dev[k] = c->d_kstage[k];
    }
    const size_t tb = kspace_table_bytes(c->n, c->g.nx, c->g.ny, c->g.nz);
    if (tb > c->ktab_bytes) {
        cudaFree(c->d_ktab);
        c->d_ktab = nullptr;
        c->ktab_bytes = 0;
        if ((e = cudaMalloc(&c->d_ktab, tb)) != cudaSuccess) return cuda_fail(c, e, "k-space phase tables");
        c->ktab_bytes = tb;
    }
    const bool timed = (c->o.debug_flags & 2) != 0;
    if (timed) {
        if (!c->ev[0]) {
            cudaEventCreate(&c->ev[0]);
            cudaEventCreate(&c->ev[1]);
        }
        cudaEventRecord(c->ev[0], c->st);
    }
    if ((e = launch_kspace(c->t, c->gd, ks, c->d_ktab, dev[0], dev[1], c->o.wait_limit, c->st)) != cudaSuccess)
        return cuda_fail(c, e, "k-space kernels");
    if (timed) cudaEventRecord(c->ev[1], c->st);
    for (int k = 0; k < 2 && host; ++k)
        if (user[k] && dev[k] != user[k] &&
            (e = cudaMemcpyAsync(user[k], dev[k], bytes, cudaMemcpyDeviceToHost, c->st)) != cudaSuccess)
            return cuda_fail(c, e, "k-space result copy");
    c->info.launches = 2;
    s = check_device_error(c);  // synchronises the stream
    if (s == RISM_OK && timed) cudaEventElapsedTime(&c->info.eval_ms, c->ev[0], c->ev[1]);
    return s;
}

rism_status rism_get_info(const rism_ctx* c, rism_info* info) {
    if (!c || !info) return RISM_E_INVALID;
    *info = c->info;
    info->beta = 1.0 / (c->o.k_B * c->o.T);
    info->kappa = c->ph.kappa;
    info->r_short = c->ph.rs;
    info->natoms = c->n;
    info->nsite = c->S;
    return RISM_OK;
}

void rism_destroy(rism_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->st);
    tree_destroy(c->tree);
    adjoint_destroy(c->adj);
    cudaFree(c->d_raw);
    cudaFree(c->t.geo);
    cudaFree(c->t.srcf);
    cudaFree(c->t.ljd);
    cudaFree(c->t.ljf);
    cudaFree(c->d_err);
    cudaFreeHost(c->h_err);
    cudaFreeHost(c->h_tail);
    cudaFreeHost(c->h_raw);
    cudaFree(c->d_tail);
    for (int k = 0; k < 3; ++k) cudaFree(c->d_stage[k]);
    if (c->ev[0]) cudaEventDestroy(c->ev[0]);
    if (c->ev[1]) cudaEventDestroy(c->ev[1]);
    for (int k = 0; k < 3; ++k) {
        if (c->cp_st[k]) cudaStreamDestroy(c->cp_st[k]);
        if (c->cp_join[k]) cudaEventDestroy(c->cp_join[k]);
    }
    if (c->cp_fork) cudaEventDestroy(c->cp_fork);
    cudaFree(c->d_lra_part);
    cudaFree(c->d_lra_atom);
    cudaFree(c->d_lra_perm);
    cudaFree(c->d_lra_src);
    cudaFreeHost(c->h_lra_perm);
    cudaFree(c->d_lra_tot);
    cudaFreeHost(c->h_lra_tot);
    cudaFree(c->d_ktab);
    cudaFree(c->d_kstage[0]);
    cudaFree(c->d_kstage[1]);
    delete c;
}

const char* rism_last_error(const rism_ctx* c) {
    if (!c) return "invalid context (NULL)";
    return c->err.c_str();
}

// Table 3: p = max(2, (log10 tol + a) / -s) per kernel, rounded up; MAC 0.3, N0 500 (the 1e-9 keeps an order
// that the expression hits exactly, up to the rounding of log10, from rising by one).  Sec. 4.3.1: the
// reciprocal-space cut-off tolerance 0.04 tol^0.9; Sec. 4.4.1: the LJ cut-off tolerance tol / 10.
rism_status rism_parameter_guide(double tolerance, rism_guide* g) {
    if (!g || !std::isfinite(tolerance) || !(tolerance > 0.0) || !(tolerance < 1.0)) return RISM_E_INVALID;
    const double lt = std::log10(tolerance);
    auto order = [&](double a, double s) { return (int32_t)std::max(2.0, std::ceil((lt + a) / -s - 1e-9)); };
    g->p_tcf = order(5.7, 0.7);
    g->p_dcf = order(1.9, 0.8);
    g->p_coulomb = order(1.4, 0.8);
    g->mac = 0.3;
    g->n0 = 500;
    g->k_tol = 0.04 * std::pow(tolerance, 0.9);
    g->lj_tol = tolerance / 10.0;
    return RISM_OK;
}

}  // extern "C"
