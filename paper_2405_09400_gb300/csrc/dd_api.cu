// Host side of the C ABI (include/ddflow.h): context set-up, device memory,
// the half-iteration / flow-update drivers and the getters.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "dd_internal.h"

#define CK(x)                                                       \
    do {                                                            \
        cudaError_t e_ = (x);                                       \
        if (e_ != cudaSuccess) return dd_record_cuda_error(e_, #x); \
    } while (0)
#define RET(x)                         \
    do {                               \
        int r_ = (x);                  \
        if (r_ != DD_OK) return r_;    \
    } while (0)

static char g_last_error[256] = "";

int dd_record_cuda_error(cudaError_t e, const char* where) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
    return DD_ERR_CUDA;
}

namespace {

constexpr double kLn2 = 0.69314718055994530942;

template <typename T>
int dmalloc(T** p, size_t n) {
    if (n == 0) n = 1;
    return cudaMalloc((void**)p, sizeof(T) * n) == cudaSuccess ? DD_OK : DD_ERR_OOM;
}
template <typename T>
void dfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}
template <typename T>
int h2d(T* d, const T* h, size_t n, cudaStream_t s) {
    if (n == 0) return DD_OK;
    cudaError_t e = cudaMemcpyAsync(d, h, sizeof(T) * n, cudaMemcpyHostToDevice, s);
    return e == cudaSuccess ? DD_OK : dd_record_cuda_error(e, "host to device copy");
}
template <typename T>
int d2h(T* h, const T* d, size_t n, cudaStream_t s) {
    if (n == 0) return DD_OK;
    cudaError_t e = cudaMemcpyAsync(h, d, sizeof(T) * n, cudaMemcpyDeviceToHost, s);
    return e == cudaSuccess ? DD_OK : dd_record_cuda_error(e, "device to host copy");
}

// grow a float buffer (contents not kept); bumps the context's buffer generation
// so that captured graphs are rebuilt
int ensure_floats(dd_ctx* c, float** p, size_t* cap, size_t need) {
    if (*cap >= need && *p) return DD_OK;
    dfree(*p);
    size_t n = need + need / 4 + 4096;
    RET(dmalloc(p, n));
    *cap = n;
    c->gen += 1;
    return DD_OK;
}

// grow a float buffer keeping its first `keep` entries
int ensure_floats_keep(dd_ctx* c, float** p, size_t* cap, size_t need, size_t keep) {
    if (*cap >= need && *p) return DD_OK;
    float* q = nullptr;
    size_t n = need + need / 4 + 4096;
    RET(dmalloc(&q, n));
    if (*p && keep) CK(cudaMemcpyAsync(q, *p, sizeof(float) * std::min(keep, *cap), cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    dfree(*p);
    *p = q;
    *cap = n;
    c->gen += 1;
    return DD_OK;
}

// build partitions (Def. 2.2 / Fig. 3): A cells 2x2, B cells shifted by one and truncated
void build_part(dd_ctx* c, int part, std::vector<int32_t>& members, std::vector<int32_t>& xblk,
                std::vector<double>& mJ) {
    const int n1 = c->n1, n2 = c->n2, s = c->s;
    const int na = part == 0 ? n1 / 2 : n1 / 2 + 1;
    const int nbb = part == 0 ? n2 / 2 : n2 / 2 + 1;
    for (int a = 0; a < na; ++a)
        for (int b = 0; b < nbb; ++b) {
            int rows[2], cols[2], nr = 0, nc = 0;
            for (int t = 0; t < 2; ++t) {
                int r = part == 0 ? 2 * a + t : 2 * a - 1 + t;
                int q = part == 0 ? 2 * b + t : 2 * b - 1 + t;
                if (r >= 0 && r < n1) rows[nr++] = r;
                if (q >= 0 && q < n2) cols[nc++] = q;
            }
            int32_t mem[4] = {-1, -1, -1, -1};
            int k = 0;
            double mass = 0.0;
            for (int ri = 0; ri < nr; ++ri)
                for (int ci = 0; ci < nc; ++ci) {
                    int i = rows[ri] * n2 + cols[ci];
                    mem[k++] = i;
                    mass += c->h_m[i];
                }
            for (int t = 0; t < 4; ++t) members.push_back(mem[t]);
            int32_t xb[XB_N] = {rows[0] * s, cols[0] * s, nr * s, nc * s, k, 0, 0, 0};
            for (int t = 0; t < XB_N; ++t) xblk.push_back(xb[t]);
            mJ.push_back(mass);
        }
}

// box headers of the pool layout (rows of stride ceil(w/4)*4) and each box's
// offset in the packed array; bounds and sizes checked (host, O(#cells))
int plan_layout(dd_ctx* c, const int32_t* hdr, size_t n, std::vector<int32_t>& bh, std::vector<long long>& soff,
                size_t* total) {
    const int nb = c->nb;
    bh.assign((size_t)BH_N * nb, 0);
    soff.assign((size_t)nb + 1, 0);
    size_t tot = 0, src = 0;
    for (int i = 0; i < nb; ++i) {
        const int o1 = hdr[4 * i], o2 = hdr[4 * i + 1], h = hdr[4 * i + 2], w = hdr[4 * i + 3];
        if (h < 0 || w < 0 || (h == 0) != (w == 0)) return DD_ERR_ARG;
        if (h && (o1 < 0 || o2 < 0 || o1 + h > c->N1 || o2 + w > c->N2)) return DD_ERR_ARG;
        const int st = (w + 3) & ~3;
        bh[BH_N * i + BH_O1] = h ? o1 : 0;
        bh[BH_N * i + BH_O2] = h ? o2 : 0;
        bh[BH_N * i + BH_H] = h;
        bh[BH_N * i + BH_W] = w;
        bh[BH_N * i + BH_STRIDE] = st;
        bh[BH_N * i + BH_START] = (int32_t)tot;
        soff[i] = (long long)src;
        tot += (size_t)h * st;
        src += (size_t)h * w;
        if (tot > (size_t)INT32_MAX) return DD_ERR_POOL;
    }
    soff[nb] = (long long)src;
    if (src != n) return DD_ERR_ARG;
    *total = tot;
    return DD_OK;
}

int ensure_plan64(dd_ctx* c, size_t n) {
    if (c->plan64_cap >= n && c->d_plan64) return DD_OK;
    dfree(c->d_plan64);
    c->plan64_cap = 0;
    const size_t m = n + n / 4 + 1024;
    RET(dmalloc(&c->d_plan64, m));
    c->plan64_cap = m;
    return DD_OK;
}

// The caller's FP64 boxes go to the device as they are (one copy) and are packed
// there into the pool that is not current; with `validate` the device checks
// the plan in FP64 (entries finite and >= 0, |nu_i| = m_i and sum_i nu_i = nu
// within plan_tol, L1). The packed plan becomes the state only if it passes.
int upload_plan(dd_ctx* c, const int32_t* hdr, const double* data, size_t n, bool validate,
                bool data_on_device = false) {
    std::vector<int32_t> bh;
    std::vector<long long> soff;
    size_t total = 0;
    RET(plan_layout(c, hdr, n, bh, soff, &total));
    const int dst = 1 - c->cur;
    RET(ensure_plan64(c, n));
    RET(ensure_floats(c, &c->pool[dst], &c->pool_cap[dst], total));
    if (data_on_device) {
        if (n) CK(cudaMemcpyAsync(c->d_plan64, data, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        RET(h2d(c->d_plan64, data, n, c->stream));
    }
    RET(h2d(c->d_soff, soff.data(), soff.size(), c->stream));
    RET(h2d(c->bhdr[dst], bh.data(), bh.size(), c->stream));
    CK(cudaMemsetAsync(c->d_red, 0, sizeof(double) * 3, c->stream));
    if (validate) CK(cudaMemsetAsync(c->d_yacc, 0, sizeof(double) * c->N1 * c->N2, c->stream));
    RET(launch_pack_plan(c, dst, validate));
    c->n_launch += validate ? 2 : 1;
    double res[3] = {0.0, 0.0, 0.0};
    RET(d2h(res, c->d_red, 3, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->n_h2d += (long long)(sizeof(double) * n + sizeof(int32_t) * bh.size() + sizeof(long long) * soff.size());
    int bad = 0;
    std::memcpy(&bad, &res[2], sizeof(int));  // the kernels' flag word
    if (bad || (validate && (!(res[0] <= c->opt.plan_tol) || !(res[1] <= c->opt.plan_tol)))) return DD_ERR_ARG;
    c->cur = dst;
    c->part[0].solved = c->part[1].solved = false;
    c->flow_ready = false;
    c->last_part = -1;
    return DD_OK;
}

int choose_threads(dd_ctx* c, long long maxarea) {
    if (c->opt.threads > 0) return std::min(512, std::max(32, (c->opt.threads / 32) * 32));
    return maxarea <= 1024 ? 128 : 256;
}

int ensure_comp(dd_ctx* c, int part, size_t comp) {
    DevPart& P = c->part[part];
    if (P.comp_cap >= comp && P.comp_b) return DD_OK;
    dfree(P.comp_b);
    dfree(P.comp_nu);
    size_t n = comp + comp / 4 + 4096;
    RET(dmalloc(&P.comp_b, n));
    RET(dmalloc(&P.comp_nu, n));
    P.comp_cap = n;
    c->gen += 1;
    return DD_OK;
}

// per-cell buffers of the learned warm start, and the list of cells with a full
// 8 x 8 X block per partition (the rows dd_collect_cells returns)
int ensure_learned_buffers(dd_ctx* c) {
    if (c->d_feat) return DD_OK;
    const size_t mc = (size_t)std::max(c->part[0].ncell, c->part[1].ncell);
    RET(dmalloc(&c->d_feat, mc * DD_MLP_NIN));
    RET(dmalloc(&c->d_pred, mc * DD_MLP_NOUT));
    for (int p = 0; p < 2; ++p) RET(dmalloc(&c->d_pred_old[p], mc * DD_MLP_NOUT));
    RET(dmalloc(&c->d_targ, mc * DD_MLP_NOUT));
    CK(cudaMemsetAsync(c->d_feat, 0, mc * DD_MLP_NIN * sizeof(uint16_t), c->stream));
    CK(cudaMemsetAsync(c->d_pred, 0, mc * DD_MLP_NOUT * sizeof(float), c->stream));
    CK(cudaMemsetAsync(c->d_targ, 0, mc * DD_MLP_NOUT * sizeof(float), c->stream));
    for (int p = 0; p < 2; ++p) {
        const DevPart& P = c->part[p];
        std::vector<int32_t> full;
        for (int J = 0; J < P.ncell; ++J)
            if (P.h_xblk[XB_N * J + XB_HX] * P.h_xblk[XB_N * J + XB_WX] == 64) full.push_back(J);
        c->n_full[p] = (int)full.size();
        RET(dmalloc(&c->d_full[p], std::max<size_t>(1, full.size())));
        if (!full.empty()) RET(h2d(c->d_full[p], full.data(), full.size(), c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return DD_OK;
}

}  // namespace

extern "C" {

void dd_default_options(dd_options* o) {
    if (!o) return;
    o->tol = 1e-5;
    o->max_iter = 100000;
    o->fixed_iters = 0;
    o->trunc = 1e-15;
    o->init_kind = DD_INIT_PRODUCT;
    o->warm = DD_WARM_PREV;
    o->threads = 0;
    o->flags = 0;
    o->plan_tol = 1e-12;
    o->omega = 1.0;
    o->graph_margin = 0.5;
    o->eps_levels = 0;
    o->eps_factor = 4.0;
    o->eps_tol = 1e-3;
    o->tol_share = 0.0;
    o->tol_gamma = 0.0;
    o->anderson = 0;
    o->eps_gamma = 0.0;
}

const char* dd_last_error(void) { return g_last_error; }

const char* dd_strerror(int s) {
    switch (s) {
        case DD_OK: return "ok";
        case DD_ERR_ARG: return "invalid argument";
        case DD_ERR_OOM: return "out of memory";
        case DD_ERR_CUDA: return "CUDA error";
        case DD_ERR_MAXITER: return "Sinkhorn iteration cap reached in some cell";
        case DD_ERR_STALL: return "FP32 stall";
        case DD_ERR_FLOW: return "min-cost flow failed; stationary flow kept";
        case DD_ERR_POOL: return "bounding box too large for the cell kernel";
        case DD_ERR_STATE: return "call order violated";
        default: return "unknown status";
    }
}

void dd_destroy(dd_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (auto& g : c->graph)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (c->mcf) mcf_destroy(c->mcf);
    dfree(c->d_mu); dfree(c->d_nu); dfree(c->d_lgmu); dfree(c->d_m); dfree(c->d_xmom);
    dfree(c->d_lnmu); dfree(c->d_lnnu); dfree(c->d_lnnuf);
    dfree(c->d_nbr); dfree(c->d_rev);
    for (int p = 0; p < 2; ++p) {
        DevPart& P = c->part[p];
        dfree(P.members); dfree(P.xblk); dfree(P.mJ); dfree(P.chdr); dfree(P.alpha); dfree(P.gauge);
        dfree(P.budget);
        dfree(P.iters); dfree(P.err); dfree(P.Ecell); dfree(P.order); dfree(P.c2b_order); dfree(P.comp_b); dfree(P.comp_nu);
        dfree(c->pool[p]); dfree(c->bhdr[p]);
    }
    dfree(c->d_bmom); dfree(c->d_tot); dfree(c->d_queue); dfree(c->d_status); dfree(c->d_pre);
    dfree(c->d_gscr); dfree(c->d_goff); dfree(c->d_guard); dfree(c->d_fused);
    for (int p = 0; p < 2; ++p) { dfree(c->d_corder[p]); dfree(c->d_ccount[p]); }
    if (c->h_guard) cudaFreeHost(c->h_guard);
    for (auto& e : c->gev)
        if (e) cudaEventDestroy(e);
    if (c->gstream) cudaStreamDestroy(c->gstream);
    dfree(c->d_feat); dfree(c->d_pred); dfree(c->d_targ); dfree(c->d_full[0]); dfree(c->d_full[1]);
    dfree(c->d_pred_old[0]); dfree(c->d_pred_old[1]);
    dfree(c->d_trace[0]); dfree(c->d_trace[1]);
    if (c->mlp) dd_mlp_destroy(c->mlp);
    dfree(c->d_cbar); dfree(c->d_w); dfree(c->d_xhdr); dfree(c->d_yacc); dfree(c->d_red);
    dfree(c->d_plan64); dfree(c->d_soff); dfree(c->d_cellmass);
    dfree(c->d_gAB); dfree(c->d_pmom);
    if (c->h_tot) cudaFreeHost(c->h_tot);
    if (c->h_cbar) cudaFreeHost(c->h_cbar);
    if (c->h_w) cudaFreeHost(c->h_w);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_join2) cudaEventDestroy(c->ev_join2);
    if (c->ev_join3) cudaEventDestroy(c->ev_join3);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->side2) cudaStreamDestroy(c->side2);
    if (c->side3) cudaStreamDestroy(c->side3);
    delete c;
}

int dd_init(const double* mu, const double* nu, const dd_grid* grid, double eps, int cell_size,
            const dd_options* opt, void* stream, dd_ctx** out) {
    if (!mu || !nu || !grid || !out) return DD_ERR_ARG;
    *out = nullptr;
    const int N1 = grid->N1, N2 = grid->N2, s = cell_size;
    if (N1 <= 0 || N2 <= 0 || !(grid->h > 0) || !(eps > 0) || s <= 0 || N1 % s || N2 % s) return DD_ERR_ARG;
    if ((N1 / s) % 2 || (N2 / s) % 2 || 2 * s > 16) return DD_ERR_ARG;
    const size_t np = (size_t)N1 * N2;
    // DD_FLAG_DEVICE_PTRS: mu and nu are device arrays; the library keeps host
    // copies of both (checks, basic masses, statistics), so copy them in first
    std::vector<double> mu_h, nu_h;
    if (opt && (opt->flags & DD_FLAG_DEVICE_PTRS)) {
        cudaStream_t st = (cudaStream_t)stream;
        mu_h.resize(np);
        nu_h.resize(np);
        cudaError_t e = cudaMemcpyAsync(mu_h.data(), mu, sizeof(double) * np, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(nu_h.data(), nu, sizeof(double) * np, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return dd_record_cuda_error(e, "dd_init: device inputs");
        mu = mu_h.data();
        nu = nu_h.data();
    }
    // compensated (Neumaier) sums: a plain running sum over a megapixel grid is
    // off by ~1e-11 and would reject correctly normalised measures
    double smu = 0, snu = 0, cmu = 0, cnu = 0;
    for (size_t k = 0; k < np; ++k) {
        if (!(mu[k] >= 0) || !(nu[k] >= 0) || !std::isfinite(mu[k]) || !std::isfinite(nu[k])) return DD_ERR_ARG;
        double t = smu + mu[k];
        cmu += std::fabs(smu) >= mu[k] ? (smu - t) + mu[k] : (mu[k] - t) + smu;
        smu = t;
        t = snu + nu[k];
        cnu += std::fabs(snu) >= nu[k] ? (snu - t) + nu[k] : (nu[k] - t) + snu;
        snu = t;
    }
    if (std::fabs(smu + cmu - 1.0) > 1e-12 || std::fabs(snu + cnu - 1.0) > 1e-12) return DD_ERR_ARG;
    dd_ctx* c = new (std::nothrow) dd_ctx();
    if (!c) return DD_ERR_OOM;
    if (opt) c->opt = *opt; else dd_default_options(&c->opt);
    c->tune.threads[0] = 256; c->tune.threads[1] = 128; c->tune.threads[2] = 256;
    c->tune.small_area = 1536; c->tune.small_side = 64;
    c->tune.cl_size = 1; c->tune.cl_cells = 0; c->tune.sm_reserve = 0;
    const bool learned = c->opt.warm == DD_WARM_MLP || (c->opt.flags & DD_FLAG_COLLECT);
    if (!(c->opt.tol >= 0) || c->opt.max_iter <= 0 || !(c->opt.trunc >= 0) || !(c->opt.omega < 2.0) ||
        (c->opt.omega >= 0.0 && c->opt.omega < 1.0) || c->opt.warm < DD_WARM_PREV || c->opt.warm > DD_WARM_MLP ||
        c->opt.eps_levels < 0 || c->opt.eps_levels > 8 ||
        (c->opt.eps_levels > 0 && !(c->opt.eps_factor > 1.0 && c->opt.eps_tol > 0.0)) || (learned && s != 4) ||
        !(c->opt.tol_share >= 0.0 && c->opt.tol_share <= 1.0) || !(c->opt.tol_gamma >= 0.0 && c->opt.tol_gamma <= 4.0) ||
        c->opt.anderson < 0 || c->opt.anderson > 4 || !(c->opt.eps_gamma >= 0.0) || !std::isfinite(c->opt.eps_gamma) ||
        (c->opt.eps_gamma > 0.0 && s > 8)) {
        delete c;
        return DD_ERR_ARG;
    }
    c->N1 = N1; c->N2 = N2; c->s = s; c->n1 = N1 / s; c->n2 = N2 / s; c->nb = c->n1 * c->n2;
    c->amax = 4 * s * s;
    c->h = grid->h; c->eps = eps;
    c->k2d = grid->h * grid->h / eps / kLn2;
    c->k2 = (float)c->k2d;
    c->stream = (cudaStream_t)stream;
    c->h_mu.assign(mu, mu + np);
    c->h_nu.assign(nu, nu + np);
    // basic masses and X moments (pixel units)
    c->h_m.assign(c->nb, 0.0);
    std::vector<double> xmom(3 * (size_t)c->nb, 0.0);
    for (int i = 0; i < c->nb; ++i) {
        int bi = i / c->n2, bj = i % c->n2;
        double m = 0, m1 = 0, m2 = 0, q = 0;
        for (int p = bi * s; p < bi * s + s; ++p)
            for (int r = bj * s; r < bj * s + s; ++r) {
                double v = mu[(size_t)p * N2 + r];
                m += v; m1 += v * p; m2 += v * r;
            }
        if (!(m > 0)) { delete c; return DD_ERR_ARG; }
        m1 /= m; m2 /= m;
        for (int p = bi * s; p < bi * s + s; ++p)
            for (int r = bj * s; r < bj * s + s; ++r) {
                double v = mu[(size_t)p * N2 + r];
                q += v * ((p - m1) * (p - m1) + (r - m2) * (r - m2));
            }
        c->h_m[i] = m;
        xmom[3 * i] = m1; xmom[3 * i + 1] = m2; xmom[3 * i + 2] = q / m;
    }
    // neighbours (Def. 3.1): self, -axis1, +axis1, -axis2, +axis2
    c->h_nbr.assign(5 * (size_t)c->nb, -1);
    std::vector<int32_t> rev(5 * (size_t)c->nb, -1);
    for (int i = 0; i < c->nb; ++i) {
        int bi = i / c->n2, bj = i % c->n2;
        c->h_nbr[5 * i] = i;
        if (bi > 0) c->h_nbr[5 * i + 1] = i - c->n2;
        if (bi < c->n1 - 1) c->h_nbr[5 * i + 2] = i + c->n2;
        if (bj > 0) c->h_nbr[5 * i + 3] = i - 1;
        if (bj < c->n2 - 1) c->h_nbr[5 * i + 4] = i + 1;
    }
    for (int j = 0; j < c->nb; ++j)
        for (int k = 0; k < 5; ++k) {
            int i = c->h_nbr[5 * j + k];
            if (i < 0) continue;
            for (int t = 0; t < 5; ++t)
                if (c->h_nbr[5 * i + t] == j) rev[5 * j + k] = t;
        }
    int rc = DD_OK;
#define TRY(x)                          \
    do {                                \
        rc = (x);                       \
        if (rc != DD_OK) goto fail;     \
    } while (0)
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) { rc = DD_ERR_CUDA; goto fail; }
        c->dev = dev;
        if (cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            rc = DD_ERR_CUDA;
            goto fail;
        }
        std::vector<float> lgmu(np);
        for (size_t k = 0; k < np; ++k) lgmu[k] = mu[k] > 0 ? (float)std::log2(mu[k]) : DD_NEG;
        TRY(dmalloc(&c->d_mu, np)); TRY(h2d(c->d_mu, mu, np, c->stream));
        TRY(dmalloc(&c->d_nu, np)); TRY(h2d(c->d_nu, nu, np, c->stream));
        TRY(dmalloc(&c->d_lgmu, np)); TRY(h2d(c->d_lgmu, lgmu.data(), np, c->stream));
        {
            std::vector<double> lnm(np), lnn(np);
            for (size_t k = 0; k < np; ++k) {
                lnm[k] = mu[k] > 0 ? std::log(mu[k]) : -INFINITY;
                lnn[k] = nu[k] > 0 ? std::log(nu[k]) : -INFINITY;
            }
            TRY(dmalloc(&c->d_lnmu, np)); TRY(h2d(c->d_lnmu, lnm.data(), np, c->stream));
            TRY(dmalloc(&c->d_lnnu, np)); TRY(h2d(c->d_lnnu, lnn.data(), np, c->stream));
            std::vector<float> lnnf(np);
            for (size_t k = 0; k < np; ++k) lnnf[k] = nu[k] > 0 ? (float)lnn[k] : DD_NEG;
            TRY(dmalloc(&c->d_lnnuf, np)); TRY(h2d(c->d_lnnuf, lnnf.data(), np, c->stream));
            if (cudaStreamSynchronize(c->stream) != cudaSuccess) { rc = DD_ERR_CUDA; goto fail; }
        }
        TRY(dmalloc(&c->d_m, c->nb)); TRY(h2d(c->d_m, c->h_m.data(), c->nb, c->stream));
        TRY(dmalloc(&c->d_xmom, 3 * (size_t)c->nb)); TRY(h2d(c->d_xmom, xmom.data(), xmom.size(), c->stream));
        TRY(dmalloc(&c->d_nbr, 5 * (size_t)c->nb)); TRY(h2d(c->d_nbr, c->h_nbr.data(), c->h_nbr.size(), c->stream));
        TRY(dmalloc(&c->d_rev, 5 * (size_t)c->nb)); TRY(h2d(c->d_rev, rev.data(), rev.size(), c->stream));
        for (int p = 0; p < 2; ++p) {
            DevPart& P = c->part[p];
            std::vector<int32_t> members, xblk;
            std::vector<double> mJ;
            build_part(c, p, members, xblk, mJ);
            P.ncell = (int)mJ.size();
            double msum = 0.0;
            for (double x : mJ) msum += x;
            P.mbar = P.ncell > 0 ? msum / P.ncell : 0.0;
            P.h_members = members;
            P.h_xblk = xblk;
            std::vector<int32_t> order(P.ncell);
            for (int k = 0; k < P.ncell; ++k) order[k] = k;
            TRY(dmalloc(&P.members, members.size())); TRY(h2d(P.members, members.data(), members.size(), c->stream));
            TRY(dmalloc(&P.xblk, xblk.size())); TRY(h2d(P.xblk, xblk.data(), xblk.size(), c->stream));
            TRY(dmalloc(&P.mJ, mJ.size())); TRY(h2d(P.mJ, mJ.data(), mJ.size(), c->stream));
            TRY(dmalloc(&P.order, order.size())); TRY(h2d(P.order, order.data(), order.size(), c->stream));
            TRY(dmalloc(&P.c2b_order, order.size())); TRY(h2d(P.c2b_order, order.data(), order.size(), c->stream));
            TRY(dmalloc(&P.chdr, (size_t)CH_N * P.ncell));
            TRY(dmalloc(&P.alpha, (size_t)c->amax * P.ncell));
            TRY(dmalloc(&P.gauge, 8 * (size_t)P.ncell));
            TRY(dmalloc(&P.iters, P.ncell));
            TRY(dmalloc(&P.err, P.ncell));
            TRY(dmalloc(&P.Ecell, P.ncell));
            TRY(dmalloc(&P.budget, P.ncell));
            TRY(dmalloc(&c->bhdr[p], (size_t)BH_N * c->nb));
        }
        if (learned) TRY(ensure_learned_buffers(c));
        TRY(dmalloc(&c->d_bmom, (size_t)BM_N * c->nb));
        TRY(dmalloc(&c->d_tot, PT_N));
        if (cudaMallocHost((void**)&c->h_tot, sizeof(long long) * PT_N) != cudaSuccess) { rc = DD_ERR_OOM; goto fail; }
        TRY(dmalloc(&c->d_queue, 4));
        TRY(dmalloc(&c->d_status, kStatusInts));
        if (cudaMemsetAsync(c->d_status, 0, kStatusInts * sizeof(int), c->stream) != cudaSuccess) { rc = DD_ERR_CUDA; goto fail; }
        TRY(dmalloc(&c->d_guard, 4));
        if (cudaMemsetAsync(c->d_guard, 0, 4 * sizeof(int), c->stream) != cudaSuccess) { rc = DD_ERR_CUDA; goto fail; }
        if (cudaMallocHost((void**)&c->h_guard, 4 * sizeof(int)) != cudaSuccess) { rc = DD_ERR_OOM; goto fail; }
        TRY(dmalloc(&c->d_goff, (size_t)std::max(c->part[0].ncell, c->part[1].ncell)));
        TRY(dmalloc(&c->d_fused, (size_t)std::max(c->part[0].ncell, c->part[1].ncell)));
        if (cudaMemsetAsync(c->d_fused, 0, sizeof(int) * std::max(c->part[0].ncell, c->part[1].ncell), c->stream) !=
            cudaSuccess) {
            rc = DD_ERR_CUDA;
            goto fail;
        }
        if (c->opt.flags & DD_FLAG_TRACE)
            for (int p = 0; p < 2; ++p) {
                TRY(dmalloc(&c->d_trace[p], 8 * (size_t)c->part[p].ncell));
                if (cudaMemsetAsync(c->d_trace[p], 0, 8 * sizeof(long long) * c->part[p].ncell, c->stream) != cudaSuccess) {
                    rc = DD_ERR_CUDA;
                    goto fail;
                }
            }
        for (int p = 0; p < 2; ++p) {
            TRY(dmalloc(&c->d_corder[p], 3 * (size_t)c->part[p].ncell));
            TRY(dmalloc(&c->d_ccount[p], 4));
        }
        TRY(dmalloc(&c->d_cbar, 5 * (size_t)c->nb));
        TRY(dmalloc(&c->d_w, 5 * (size_t)c->nb));
        if (cudaMallocHost((void**)&c->h_cbar, sizeof(double) * 5 * c->nb) != cudaSuccess) { rc = DD_ERR_OOM; goto fail; }
        if (cudaMallocHost((void**)&c->h_w, sizeof(double) * 5 * c->nb) != cudaSuccess) { rc = DD_ERR_OOM; goto fail; }
        TRY(dmalloc(&c->d_xhdr, (size_t)CH_N * c->nb));
        TRY(dmalloc(&c->d_yacc, np));
        TRY(dmalloc(&c->d_red, 8));
        TRY(dmalloc(&c->d_soff, (size_t)c->nb + 1));
        TRY(dmalloc(&c->d_cellmass, (size_t)c->nb));
        for (auto& e : c->ev)
            if (cudaEventCreate(&e) != cudaSuccess) { rc = DD_ERR_CUDA; goto fail; }
        for (auto& e : c->gev)
            if (cudaEventCreate(&e) != cudaSuccess) { rc = DD_ERR_CUDA; goto fail; }
        // the large-box and cluster cells run on high-priority streams: released
        // together with the small-box class (all three wait on one fork event, or
        // in graphs on one node), their CTAs are placed before the small-box
        // kernel's persistent grid fills the SMs, so the longest solves start
        // first (in graphs: node priorities)
        int prio_lo = 0, prio_hi = 0;
        cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
        if (cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
            cudaStreamCreateWithPriority(&c->side2, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
            cudaStreamCreateWithPriority(&c->side3, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&c->ev_join3, cudaEventDisableTiming) != cudaSuccess) {
            rc = DD_ERR_CUDA;
            goto fail;
        }
        if (c->opt.eps_gamma > 0.0) {
            // gluing candidates: gamma_ij of every directed edge, once (mu is fixed)
            const size_t n = (size_t)c->s * c->s;
            TRY(dmalloc(&c->d_gAB, (size_t)c->nb * 4 * n * 3));
            TRY(dmalloc(&c->d_pmom, (size_t)c->nb * n * 3));
            if (cudaMemsetAsync(c->d_pmom, 0, sizeof(double) * c->nb * n * 3, c->stream) != cudaSuccess ||
                cudaMemsetAsync(c->d_status + 6, 0, sizeof(int), c->stream) != cudaSuccess) {
                rc = DD_ERR_CUDA;
                goto fail;
            }
            TRY(launch_gamma(c, c->d_status + 6));
            c->n_launch += 1;
        }
        if (c->opt.init_kind == DD_INIT_PRODUCT) {
            // nu_i = m_i nu on the whole grid, truncated like every other state
            std::vector<int32_t> hdr(4 * (size_t)c->nb);
            std::vector<double> data;
            data.reserve(np * c->nb);
            for (int i = 0; i < c->nb; ++i) {
                int lo1 = N1, hi1 = -1, lo2 = N2, hi2 = -1;
                for (int p = 0; p < N1; ++p)
                    for (int q = 0; q < N2; ++q)
                        if (c->h_m[i] * nu[(size_t)p * N2 + q] >= c->opt.trunc && nu[(size_t)p * N2 + q] > 0) {
                            lo1 = std::min(lo1, p); hi1 = std::max(hi1, p);
                            lo2 = std::min(lo2, q); hi2 = std::max(hi2, q);
                        }
                if (hi1 < 0) { rc = DD_ERR_ARG; goto fail; }
                hdr[4 * i] = lo1; hdr[4 * i + 1] = lo2; hdr[4 * i + 2] = hi1 - lo1 + 1; hdr[4 * i + 3] = hi2 - lo2 + 1;
                for (int p = lo1; p <= hi1; ++p)
                    for (int q = lo2; q <= hi2; ++q) {
                        double v = c->h_m[i] * nu[(size_t)p * N2 + q];
                        data.push_back(v >= c->opt.trunc ? v : 0.0);
                    }
            }
            TRY(upload_plan(c, hdr.data(), data.data(), data.size(), false));
        } else {
            if (cudaStreamSynchronize(c->stream) != cudaSuccess) { rc = DD_ERR_CUDA; goto fail; }
        }
    }
#undef TRY
    *out = c;
    return DD_OK;
fail:
    dd_destroy(c);
    return rc;
}

int dd_set_plan(dd_ctx* c, const int32_t* hdr, const double* data, size_t n) {
    if (!c || !hdr || (!data && n)) return DD_ERR_ARG;
    c->stats_pending = c->last_stats_valid = false;
    if (c->opt.flags & DD_FLAG_DEVICE_PTRS) {  // headers are laid out on the host
        std::vector<int32_t> hh(4 * (size_t)c->nb);
        CK(cudaMemcpyAsync(hh.data(), hdr, sizeof(int32_t) * hh.size(), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        return upload_plan(c, hh.data(), data, n, true, true);
    }
    return upload_plan(c, hdr, data, n, true);
}

// elapsed milliseconds between two recorded events (0 if they cannot be timed)
static float event_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        ms = 0.f;
    }
    return ms;
}

static int fill_stats(dd_ctx* c, int part, dd_stats* st, int slot = 0, cudaEvent_t e0 = nullptr,
                      cudaEvent_t e1 = nullptr, cudaEvent_t e2 = nullptr, cudaEvent_t ec = nullptr) {
    if (!e0) { e0 = c->ev[0]; e1 = c->ev[1]; e2 = c->ev[2]; ec = c->ev[7]; }
    DevPart& P = c->part[part];
    std::vector<int32_t> it(P.ncell), ch((size_t)CH_N * P.ncell), xb;
    std::vector<double> er(P.ncell), E(P.ncell);
    RET(d2h(it.data(), P.iters, P.ncell, c->stream));
    RET(d2h(er.data(), P.err, P.ncell, c->stream));
    RET(d2h(E.data(), P.Ecell, P.ncell, c->stream));
    RET(d2h(ch.data(), P.chdr, ch.size(), c->stream));
    int status[8];
    RET(d2h(status, c->d_status + 8 * slot, 8, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    double Es = 0, es = 0, im = 0, terms = 0;
    int imax = 0;
    for (int J = 0; J < P.ncell; ++J) {
        Es += E[J];
        es += er[J];
        im += it[J];
        imax = std::max(imax, it[J]);
        // Sinkhorn terms per iteration: hx*wx*w + h*w*hx + h*wx*w + hx*wx*h
        const int h = ch[CH_N * J + CH_H], w = ch[CH_N * J + CH_W];
        const double hx = P.h_xblk[XB_N * J + XB_HX], wx = P.h_xblk[XB_N * J + XB_WX];
        terms += (double)it[J] * (hx * wx * w + (double)h * w * hx + (double)h * wx * w + hx * wx * h);
    }
    c->last_E = Es;
    c->last_l1x = es;
    if (st) {
        st->part = part;
        st->ncell = P.ncell;
        st->iters_max = imax;
        st->iters_mean = P.ncell ? im / P.ncell : 0;
        st->n_maxiter = status[0];
        st->n_stalled = status[3];
        st->objective = Es;
        st->l1_x = es;
        st->lse_terms = terms;
        st->ms_total = event_ms(e0, e2);
        st->ms_cells = event_ms(e1, e2);
        std::vector<int32_t> bh((size_t)BH_N * c->nb);
        RET(d2h(bh.data(), c->bhdr[c->cur], bh.size(), c->stream));
        CK(cudaStreamSynchronize(c->stream));
        int64_t ent = 0;
        for (int i = 0; i < c->nb; ++i) ent += (int64_t)bh[BH_N * i + BH_H] * bh[BH_N * i + BH_W];
        st->stored_entries = ent;
        // CompositeToBasic, balancing, truncation: reads nu_J, writes the basic boxes
        double comp_entries = 0.0;
        for (int J = 0; J < P.ncell; ++J) comp_entries += (double)ch[CH_N * J + CH_H] * ch[CH_N * J + CH_W];
        st->ms_c2b = ec ? event_ms(ec, e2) : 0.0;
        st->bytes_c2b = 4.0 * (comp_entries + (double)ent);
    }
    // a kernel found its shared memory too small, or a pool slot beyond its buffer, and skipped
    if (status[2] > 0 || status[4] > 0) return DD_ERR_POOL;
    return status[0] > 0 ? DD_ERR_MAXITER : DD_OK;
}

}  // extern "C"

// most cells per half-iteration solved by clusters (0: clusters off)
static int cluster_cap(dd_ctx* c) {
    if (c->tune.cl_size < 2 || (c->opt.flags & DD_FLAG_COLLECT)) return 0;
    return std::max(0, std::min(c->tune.cl_cells, c->nsm / half_cluster_size(c->tune.cl_size)));
}

// the network's GEMM flag as read back from d_status[kStatusMlp]: DD_ERR_CUDA
// (and the flag cleared) if one of its waits timed out
static int mlp_status(dd_ctx* c, int flag) {
    if (!flag) return DD_OK;
    CK(cudaMemsetAsync(c->d_status + kStatusMlp, 0, sizeof(int), c->stream));
    return dd_record_cuda_error(cudaErrorLaunchTimeout, "warm-start network (tensor-memory GEMM): a wait timed out");
}

int half_iteration_eager(dd_ctx* c, int part, bool with_c2b) {
    DevPart& P = c->part[part];
    c->fuse_c2b = with_c2b;  // without k_c2b after them the solves must not mark cells done
    CK(cudaEventRecord(c->ev[0], c->stream));
    RET(launch_plan_half(c, part));
    c->n_launch += 1;
    if (mlp_active(c, part) || (c->opt.flags & DD_FLAG_COLLECT)) {
        // network inputs from the union boxes; the prediction initialises the solves
        RET(launch_feat(c, part));
        c->n_launch += 1;
        if (mlp_active(c, part)) {
            RET(mlp_forward_dev(c->mlp, c->d_feat, P.ncell, c->d_pred, c->stream, c->d_status + kStatusMlp));
            c->n_launch += 4;
        }
    }
    int mlp_flag = 0;
    if (mlp_active(c, part)) RET(d2h(&mlp_flag, c->d_status + kStatusMlp, 1, c->stream));
    RET(d2h(c->h_tot, c->d_tot, PT_N, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    RET(mlp_status(c, mlp_flag));
    const long long comp = c->h_tot[PT_COMP], outn = c->h_tot[PT_OUT];
    if (outn > (long long)INT32_MAX || comp > (long long)INT32_MAX * 4LL) return DD_ERR_POOL;
    if (P.comp_cap < (size_t)comp || !P.comp_b) RET(ensure_comp(c, part, (size_t)comp));
    c->status_slot = 0;
    c->seen.out = std::max(c->seen.out, outn);
    c->seen.comp[part] = std::max(c->seen.comp[part], comp);
    RET(ensure_floats(c, &c->pool[1 - c->cur], &c->pool_cap[1 - c->cur], (size_t)outn));
    if (c->opt.flags & DD_FLAG_KEEP_PREBALANCE) RET(ensure_floats(c, &c->d_pre, &c->pre_cap, (size_t)outn));
    // Work queue order: longest expected solve first (box area x the cell's
    // previous Sinkhorn iteration count). Cells are split in two size classes,
    // each launched with shared memory sized for its own largest box: the small
    // class (most cells) fits many CTAs per SM, the large class runs concurrently
    // on a second stream.
    std::vector<int32_t> ch((size_t)CH_N * P.ncell), itp(P.ncell, 1);
    RET(d2h(ch.data(), P.chdr, ch.size(), c->stream));
    if (P.warm_valid) RET(d2h(itp.data(), P.iters, P.ncell, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::vector<double> key(P.ncell);
    // classes: 0 large boxes (second stream), 1 small boxes, 2 boxes beyond shared
    // memory (their two box arrays in global scratch, also on the second stream)
    std::vector<int32_t> cls_cells[4];
    long long dims[4][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // [class][area, h, w]
    std::vector<long long> goff(P.ncell, -1);
    long long gtot = 0;
    // largest box area a shared-memory launch can hold next to the tables of the
    // tallest and widest boxes of this half-iteration
    long long hmax = 1, wmax = 1;
    for (int J = 0; J < P.ncell; ++J) {
        hmax = std::max(hmax, (long long)ch[CH_N * J + CH_H]);
        wmax = std::max(wmax, (long long)ch[CH_N * J + CH_W]);
    }
    const long long base = (long long)half_smem_bytes(c, 0, hmax, wmax);
    const long long a_cap = std::max(0LL, ((long long)half_kernel_max_smem() - base) / 8);
    for (int J = 0; J < P.ncell; ++J) {
        const int h = ch[CH_N * J + CH_H], w = ch[CH_N * J + CH_W];
        const long long a = (long long)h * half_padw(w);
        key[J] = (double)h * w * std::max(1, itp[J]);
        int cls = a <= c->tune.small_area && w <= c->tune.small_side && h <= c->tune.small_side ? 1 : 0;
        if (cls == 0 && a > a_cap) {
            cls = 2;
            goff[J] = gtot;
            gtot += 2 * a;
        }
        cls_cells[cls].push_back(J);
        dims[cls][0] = std::max(dims[cls][0], a);
        dims[cls][1] = std::max(dims[cls][1], (long long)h);
        dims[cls][2] = std::max(dims[cls][2], (long long)w);
    }
    if (!cls_cells[0].empty()) {
        c->seen.a0 = std::max(c->seen.a0, dims[0][0]);
        c->seen.h0 = std::max(c->seen.h0, dims[0][1]);
        c->seen.w0 = std::max(c->seen.w0, dims[0][2]);
    }
    c->seen.hmax = std::max(c->seen.hmax, hmax);
    c->seen.wmax = std::max(c->seen.wmax, wmax);
    c->seen.gscr = std::max(c->seen.gscr, gtot);
    c->seen.n0 = std::max(c->seen.n0, (long long)cls_cells[0].size());
    c->seen.n2 = std::max(c->seen.n2, (long long)cls_cells[2].size());
    // class 3: the largest-work cells of classes 0 and 2 on thread-block clusters,
    // by the rule k_classify applies in captured graphs (whole quarter-octave key
    // buckets from the top, then the first cells of the next bucket in index
    // order, cluster_cap cells in all)
    const int ccap = cluster_cap(c);
    if (ccap > 0) {
        std::vector<int> fbk(P.ncell, -1);
        int cntf[192] = {0};
        for (int k : {0, 2})
            for (int32_t J : cls_cells[k]) {
                const long long h = ch[CH_N * J + CH_H], w = ch[CH_N * J + CH_W];
                if (h * w < kClusterMinArea) continue;
                int bk = 0, fb = 0;
                cluster_key_bucket(h * w * std::max(1, itp[J]), bk, fb);
                fbk[J] = fb;
                ++cntf[fb];
            }
        int cum = 0, bstar = 192, fpart = -1, npart = 0;
        for (int f = 191; f >= 0; --f) {
            if (cntf[f] == 0) continue;
            if (cum + cntf[f] > ccap) {
                fpart = f;
                npart = ccap - cum;
                break;
            }
            cum += cntf[f];
            bstar = f;
        }
        // the partial bucket: its first cells in index order
        std::vector<char> sel(P.ncell, 0);
        for (int J = 0, taken = 0; J < P.ncell; ++J) {
            if (fbk[J] < 0) continue;
            if (fbk[J] >= bstar) sel[J] = 1;
            else if (fbk[J] == fpart && taken < npart) { sel[J] = 1; ++taken; }
        }
        if (cum + npart > 0) {
            for (int k : {0, 2}) {
                std::vector<int32_t> keep;
                for (int32_t J : cls_cells[k]) (sel[J] ? cls_cells[3] : keep).push_back(J);
                cls_cells[k].swap(keep);
            }
            for (int32_t J : cls_cells[3]) {
                const int h = ch[CH_N * J + CH_H], w = ch[CH_N * J + CH_W];
                if (goff[J] < 0) dims[3][0] = std::max(dims[3][0], (long long)h * half_padw(w));
                dims[3][1] = std::max(dims[3][1], (long long)h);
                dims[3][2] = std::max(dims[3][2], (long long)w);
            }
        }
    }
    auto by_key = [&](int32_t x, int32_t y) { return key[x] > key[y]; };
    std::vector<int32_t> order;
    size_t cls_off[4];
    for (int k = 0; k < 4; ++k) {
        std::stable_sort(cls_cells[k].begin(), cls_cells[k].end(), by_key);
        cls_off[k] = order.size();
        order.insert(order.end(), cls_cells[k].begin(), cls_cells[k].end());
    }
    RET(h2d(P.order, order.data(), order.size(), c->stream));
    // k_c2b: the cluster class, then the large, global-scratch and small classes
    // (each by descending work key), so the longest CompositeToBasic cells start first
    {
        std::vector<int32_t> c2b;
        c2b.reserve(order.size());
        for (int k : {3, 0, 2, 1}) c2b.insert(c2b.end(), cls_cells[k].begin(), cls_cells[k].end());
        RET(h2d(P.c2b_order, c2b.data(), c2b.size(), c->stream));
    }
    if (gtot > 0) RET(ensure_floats(c, &c->d_gscr, &c->gscr_cap, (size_t)gtot));
    if (!cls_cells[2].empty() || !cls_cells[3].empty()) RET(h2d(c->d_goff, goff.data(), goff.size(), c->stream));
    size_t smem_c[4] = {0, 0, 0, 0};
    for (int k = 0; k < 4; ++k) {
        if (cls_cells[k].empty()) continue;
        smem_c[k] = half_smem_bytes(c, k == 2 ? 0 : dims[k][0], dims[k][1], dims[k][2]);
        if (smem_c[k] > (size_t)half_kernel_max_smem()) return DD_ERR_POOL;
    }
    const int thr_c[3] = {c->opt.threads > 0 ? choose_threads(c, 0) : c->tune.threads[0],
                          c->opt.threads > 0 ? choose_threads(c, 0) : c->tune.threads[1],
                          c->opt.threads > 0 ? choose_threads(c, 0) : c->tune.threads[2]};
    CK(cudaMemsetAsync(c->d_queue, 0, sizeof(int) * 4, c->stream));
    CK(cudaMemsetAsync(c->d_status, 0, sizeof(int) * 8, c->stream));
    RET(launch_budget(c, part));
    c->n_launch += 1;
    CK(cudaEventRecord(c->ev[1], c->stream));
    // with both size classes, each waits on the same fork event (the small class
    // on its own stream): released together, the high-priority large class is
    // placed first, as in a captured graph. Stream-ordered after the budget
    // kernel, the small class would be released first and its persistent grid
    // would take every SM before the large cells could start.
    const bool side_used = !cls_cells[1].empty() && (!cls_cells[0].empty() || !cls_cells[2].empty());
    if (side_used) {
        CK(cudaEventRecord(c->ev_fork, c->stream));
        CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
        CK(cudaStreamWaitEvent(c->side3, c->ev_fork, 0));
    }
    if (!cls_cells[3].empty()) {  // clusters first, on their own high-priority stream
        CK(cudaEventRecord(c->ev_fork, c->stream));
        CK(cudaStreamWaitEvent(c->side2, c->ev_fork, 0));
        const int n = (int)cls_cells[3].size();
        const int ncl = std::max(1, std::min(n, c->nsm / half_cluster_size(c->tune.cl_size)));
        RET(launch_half_cluster(c, part, P.order + cls_off[3], n, c->d_queue + 3, dims[3], thr_c[0],
                                c->tune.cl_size, smem_c[3], ncl, c->side2));
        c->n_launch += 1;
        CK(cudaEventRecord(c->ev_join2, c->side2));
    }
    for (int k : {2, 0, 1}) {
        if (cls_cells[k].empty()) continue;
        const int n = (int)cls_cells[k].size();
        int occ = std::max(1, half_occupancy(thr_c[k], smem_c[k]));
        // the large-box classes leave sm_reserve SMs, and the SMs of the cluster
        // class, to a concurrent small-box class
        const int ncl_sm = cls_cells[3].empty() ? 0
                           : std::max(1, std::min((int)cls_cells[3].size(), c->nsm / half_cluster_size(c->tune.cl_size))) *
                                 half_cluster_size(c->tune.cl_size);
        const int sms = (k != 1 && side_used && c->tune.sm_reserve > 0)
                            ? std::max(1, c->nsm - c->tune.sm_reserve - ncl_sm) : c->nsm;
        int grid = std::max(1, std::min(n, sms * occ));
        cudaStream_t st = !side_used ? c->stream : (k != 1 ? c->side : c->side3);
        // the global-scratch class keeps no box array in shared memory: its carve
        // must see area 0, as its shared-memory size was computed with area 0
        const long long kd[3] = {k == 2 ? 0 : dims[k][0], dims[k][1], dims[k][2]};
        RET(launch_half(c, part, P.order + cls_off[k], n, c->d_queue + k, kd, thr_c[k], smem_c[k], grid, st,
                        k == 2));
        c->n_launch += 1;
    }
    if (side_used) {
        CK(cudaEventRecord(c->ev_join, c->side));
        CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
        CK(cudaEventRecord(c->ev_join3, c->side3));
        CK(cudaStreamWaitEvent(c->stream, c->ev_join3, 0));
    }
    if (!cls_cells[3].empty()) CK(cudaStreamWaitEvent(c->stream, c->ev_join2, 0));
    if (mlp_keeps_old(c) && with_c2b)
        CK(cudaMemcpyAsync(c->d_pred_old[part], c->d_pred, sizeof(float) * DD_MLP_NOUT * P.ncell,
                           cudaMemcpyDeviceToDevice, c->stream));
    if (with_c2b) {
        const long long dall[3] = {std::max({dims[0][0], dims[1][0], dims[2][0], dims[3][0]}),
                                   std::max({dims[0][1], dims[1][1], dims[2][1], dims[3][1]}),
                                   std::max({dims[0][2], dims[1][2], dims[2][2], dims[3][2]})};
        const size_t sm = c2b_smem_bytes(c, dall[1], dall[2]);
        if (sm > (size_t)half_kernel_max_smem()) return DD_ERR_POOL;
        CK(cudaEventRecord(c->ev[7], c->stream));
        RET(launch_c2b(c, part, dall, sm, P.c2b_order, nullptr));
        c->n_launch += 1;
    }
    CK(cudaEventRecord(c->ev[2], c->stream));
    return DD_OK;
}

extern "C" {

int dd_set_eps(dd_ctx* c, double eps) {
    if (!c || !(eps > 0.0) || !std::isfinite(eps)) return DD_ERR_ARG;
    c->stats_pending = c->last_stats_valid = false;
    const double f = c->eps / eps;
    for (int p = 0; p < 2; ++p) {
        DevPart& P = c->part[p];
        if (P.warm_valid) RET(launch_rescale_alpha(c, p, f));
        c->n_launch += P.warm_valid ? 1 : 0;
        P.pred_old_valid = false;
    }
    c->eps = eps;
    c->k2d = c->h * c->h / eps / kLn2;
    c->k2 = (float)c->k2d;
    c->gen += 1;  // captured graphs hold the old cost scale
    CK(cudaStreamSynchronize(c->stream));
    return DD_OK;
}

int dd_iterate(dd_ctx* c, int part, dd_stats* st) {
    if (!c) return DD_ERR_ARG;
    c->stats_pending = c->last_stats_valid = false;
    if (part < -1 || part > 1) return DD_ERR_ARG;
    if (c->pool[c->cur] == nullptr) return DD_ERR_STATE;
    if (part == -1) part = c->last_part == 0 ? 1 : 0;
    DevPart& P = c->part[part];
    if (c->opt.warm == DD_WARM_MLP && !c->mlp_ready) return DD_ERR_STATE;
    RET(half_iteration_eager(c, part, true));
    c->cur = 1 - c->cur;
    P.warm_valid = true;
    P.solved = true;
    P.pred_old_valid = mlp_keeps_old(c);
    c->last_part = part;
    c->flow_ready = true;
    return fill_stats(c, part, st);
}

// flow statistics from the host copy of w and the events (costs: ev[0..1],
// exchange: ev[2..3])
static void flow_stats(dd_ctx* c, double value, int32_t piv, double ms_solve, cudaEvent_t* ev, dd_flow_stats* st) {
    dd_flow_stats fs{};
    // entries read (source boxes with w_ij > 0) and written by the exchange,
    // totalled by its planning kernel
    long long xt[2] = {0, 0};
    if (d2h(xt, c->d_tot + PT_PAD0, 2, c->stream) == DD_OK && cudaStreamSynchronize(c->stream) == cudaSuccess)
        fs.bytes_exchange = 4.0 * (double)(xt[0] + xt[1]);
    else
        cudaGetLastError();
    fs.value = value;
    fs.pivots = piv;
    int nz = 0;
    double moved = 0;
    for (int i = 0; i < c->nb; ++i)
        for (int k = 1; k < 5; ++k)
            if (c->h_w[5 * i + k] > 0) { ++nz; moved += c->h_w[5 * i + k]; }
    fs.nonzero = nz;
    fs.moved = moved;
    fs.ms_costs = event_ms(ev[0], ev[1]);
    fs.ms_solve = ms_solve;
    fs.ms_exchange = event_ms(ev[2], ev[3]);
    fs.ms_host_step = event_ms(ev[1], ev[2]);
    c->last_flow = fs;
    if (st) *st = fs;
}

int dd_flow_update(dd_ctx* c, dd_flow_stats* st) {
    if (!c) return DD_ERR_ARG;
    c->stats_pending = c->last_stats_valid = false;
    if (!c->flow_ready) return DD_ERR_STATE;
    CK(cudaEventRecord(c->ev[3], c->stream));
    RET(launch_cbar(c));
    c->n_launch += 1;
    CK(cudaEventRecord(c->ev[4], c->stream));
    RET(d2h(c->h_cbar, c->d_cbar, 5 * (size_t)c->nb, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    auto t0 = std::chrono::steady_clock::now();
    double value = 0.0;
    int32_t piv = 0;
    int frc = DD_OK;
    if (!c->mcf) frc = mcf_create(c->nb, c->h_nbr.data(), c->h_m.data(), &c->mcf);
    if (frc == DD_OK) frc = mcf_solve(c->mcf, c->h_cbar, c->h_w, &value, &piv);
    if (frc != DD_OK) {  // keep the stationary flow (Lemma 3.6: always feasible)
        for (int i = 0; i < c->nb; ++i)
            for (int k = 0; k < 5; ++k) c->h_w[5 * i + k] = k == 0 ? c->h_m[i] : 0.0;
        value = 0.0;
    }
    auto t1 = std::chrono::steady_clock::now();
    RET(h2d(c->d_w, c->h_w, 5 * (size_t)c->nb, c->stream));
    CK(cudaEventRecord(c->ev[5], c->stream));
    RET(launch_plan_exchange(c));
    c->n_launch += 2;
    RET(d2h(c->h_tot, c->d_tot, PT_N, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (c->h_tot[PT_OUT] > (long long)INT32_MAX) return DD_ERR_POOL;
    RET(ensure_floats(c, &c->pool[1 - c->cur], &c->pool_cap[1 - c->cur], (size_t)c->h_tot[PT_OUT]));
    c->seen.out = std::max(c->seen.out, c->h_tot[PT_OUT]);
    CK(cudaMemsetAsync(c->d_status + 5, 0, sizeof(int), c->stream));
    RET(launch_exchange(c));
    c->n_launch += 1;
    CK(cudaEventRecord(c->ev[6], c->stream));
    c->cur = 1 - c->cur;
    c->flow_ready = false;
    int xs = 0;
    RET(d2h(&xs, c->d_status + 5, 1, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (xs > 0) return DD_ERR_POOL;
    flow_stats(c, value, piv, std::chrono::duration<double, std::milli>(t1 - t0).count(), c->ev + 3, st);
    return frc == DD_OK ? DD_OK : DD_ERR_FLOW;
}

// ---- dd_step: the hybrid iteration as one CUDA graph -------------------------

namespace {

// one eager hybrid iteration (A, B, flow) through the public steps
int step_eager(dd_ctx* c, dd_stats* sa, dd_stats* sb, dd_flow_stats* sf, int from = 0) {
    int rc = DD_OK;
    if (from <= 0) {
        int r = dd_iterate(c, 0, sa);
        if (r != DD_OK && r != DD_ERR_MAXITER) return r;
        if (r != DD_OK) rc = r;
    }
    if (from <= 1) {
        int r = dd_iterate(c, 1, sb);
        if (r != DD_OK && r != DD_ERR_MAXITER) return r;
        if (r != DD_OK) rc = r;
    }
    int r = dd_flow_update(c, sf);
    if (r != DD_OK && r != DD_ERR_FLOW) return r;
    return r != DD_OK ? r : rc;
}

// Capacities for a captured iteration, from the sizes eager steps have seen,
// with margins; grows the buffers to them. Returns DD_ERR_POOL if the boxes
// seen so far do not fit the launches a graph can hold.
int graph_prepare(dd_ctx* c) {
    dd_ctx::Caps g;
    const auto& sn = c->seen;
    const long long smax = half_kernel_max_smem();
    const double mg = std::max(0.0, c->opt.graph_margin);
    const long long slack = mg > 0.0 ? 1 : 0;
    auto grow = [&](long long x, double f, long long add) { return x + (long long)(f * mg * (double)x) + slack * add; };
    g.pool = grow(sn.out, 1.0, 65536);
    for (int p = 0; p < 2; ++p) g.comp[p] = grow(sn.comp[p], 1.0, 65536);
    const long long sa = c->tune.small_area, ss = c->tune.small_side;
    g.h0 = std::max(ss, grow(sn.h0, 0.5, 4));
    g.w0 = std::max(ss, grow(sn.w0, 0.5, 4));
    g.a0 = std::max(sa, grow(sn.a0, 0.5, 64));
    while (g.a0 > sa && (long long)half_smem_bytes(c, g.a0, g.h0, g.w0) > smax) g.a0 -= g.a0 / 16 + 1;
    if ((long long)half_smem_bytes(c, g.a0, g.h0, g.w0) > smax) return DD_ERR_POOL;
    g.h2 = std::max(g.h0, grow(sn.hmax, 1.0, 8));
    g.w2 = std::max(g.w0, grow(sn.wmax, 1.0, 8));
    auto fits2 = [&](long long h, long long w) {
        return (long long)half_smem_bytes(c, 0, h, w) <= smax && (long long)c2b_smem_bytes(c, h, w) <= smax;
    };
    while (!fits2(g.h2, g.w2) && (g.h2 > sn.hmax || g.w2 > sn.wmax)) {
        if (g.h2 > sn.hmax) g.h2 -= (g.h2 - sn.hmax + 7) / 8;
        if (g.w2 > sn.wmax) g.w2 -= (g.w2 - sn.wmax + 7) / 8;
    }
    if (!fits2(g.h2, g.w2)) return DD_ERR_POOL;
    // one launch for every large box: the tables sized for (h2, w2), box arrays
    // of up to a0 in shared memory, larger ones in global scratch
    while (g.a0 > 0 && (long long)half_smem_bytes(c, g.a0, g.h2, g.w2) > smax) g.a0 -= g.a0 / 16 + 4;
    g.a0 = std::max(0LL, g.a0);
    g.gscr = std::max(grow(sn.gscr, 1.0, 0), slack << 20);
    g.smem[1] = half_smem_bytes(c, sa, ss, ss);
    g.smem[0] = half_smem_bytes(c, g.a0, g.h2, g.w2);
    g.smem[2] = 0;
    g.smem_c2b = c2b_smem_bytes(c, g.h2, g.w2);
    g.cl_cap = cluster_cap(c);
    const int* thr = c->tune.threads;
    for (int k = 0; k < 2; ++k) {
        const int occ = std::max(1, half_occupancy(thr[k], g.smem[k]));
        // the large-box class leaves sm_reserve SMs, and the SMs of the cluster
        // class, to the small-box class
        const int used = c->tune.sm_reserve > 0 ? c->tune.sm_reserve + g.cl_cap * half_cluster_size(c->tune.cl_size) : 0;
        g.grid[k] = (k == 0 ? std::max(1, c->nsm - used) : c->nsm) * occ;
    }

    // full persistent grids: the class sizes vary between iterations, CTAs that
    // find the queue empty exit at once
    RET(ensure_floats_keep(c, &c->pool[c->cur], &c->pool_cap[c->cur], (size_t)g.pool, c->pool_cap[c->cur]));
    RET(ensure_floats_keep(c, &c->pool[1 - c->cur], &c->pool_cap[1 - c->cur], (size_t)g.pool, 0));
    for (int p = 0; p < 2; ++p) RET(ensure_comp(c, p, (size_t)g.comp[p]));
    RET(ensure_floats(c, &c->d_gscr, &c->gscr_cap, (size_t)g.gscr));
    if (c->opt.flags & DD_FLAG_KEEP_PREBALANCE) RET(ensure_floats(c, &c->d_pre, &c->pre_cap, (size_t)g.pool));
    // what the kernels were captured with must be what the buffers hold
    g.pool = (long long)std::min(c->pool_cap[0], c->pool_cap[1]);
    for (int p = 0; p < 2; ++p) g.comp[p] = (long long)c->part[p].comp_cap;
    g.gscr = (long long)c->gscr_cap;
    c->gcap = g;
    return DD_OK;
}

int enqueue_half_graph(dd_ctx* c, int part, int stage) {
    DevPart& P = c->part[part];
    c->fuse_c2b = true;
    const auto& g = c->gcap;
    c->status_slot = stage;
    cudaEvent_t* ev = c->gev + 3 * (stage - 1);
    // timing events inside a captured graph must be event-record nodes
    CK(cudaEventRecordWithFlags(ev[0], c->stream, cudaEventRecordExternal));
    // the stop budgets depend only on the previous solves' iteration counts: they
    // are computed on a side stream while the boxes are planned and classified
    CK(cudaEventRecord(c->ev_fork, c->stream));
    CK(cudaStreamWaitEvent(c->side3, c->ev_fork, 0));
    RET(launch_budget(c, part, c->side3));
    CK(cudaEventRecord(c->ev_join3, c->side3));
    RET(launch_plan_half(c, part));
    c->n_launch += 1;
    if (mlp_active(c, part) || (c->opt.flags & DD_FLAG_COLLECT)) {
        RET(launch_feat(c, part));
        c->n_launch += 1;
        if (mlp_active(c, part)) {
            RET(mlp_forward_dev(c->mlp, c->d_feat, P.ncell, c->d_pred, c->stream, c->d_status + kStatusMlp));
            c->n_launch += 4;
        }
    }
    CK(cudaMemsetAsync(c->d_queue, 0, sizeof(int) * 4, c->stream));
    CK(cudaMemsetAsync(c->d_status + 8 * stage, 0, sizeof(int) * 8, c->stream));
    RET(launch_classify(c, part, stage));
    CK(cudaStreamWaitEvent(c->stream, c->ev_join3, 0));
    c->n_launch += 2;
    CK(cudaEventRecordWithFlags(ev[1], c->stream, cudaEventRecordExternal));
    CK(cudaEventRecord(c->ev_fork, c->stream));
    CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    // large boxes (high-priority stream, pending from the start) and small boxes
    const long long d0[3] = {g.a0, g.h2, g.w2};
    const long long d1[3] = {c->tune.small_area, c->tune.small_side, c->tune.small_side};
    const int* thr = c->tune.threads;
    if (g.cl_cap > 0) {  // the cluster class, pending first on its own high-priority stream
        CK(cudaStreamWaitEvent(c->side2, c->ev_fork, 0));
        RET(launch_half_cluster(c, part, c->d_corder[part] + 2LL * P.ncell, P.ncell, c->d_queue + 2, d0, thr[0],
                                c->tune.cl_size, g.smem[0], g.cl_cap, c->side2, c->d_ccount[part] + 2));
        c->n_launch += 1;
        CK(cudaEventRecord(c->ev_join2, c->side2));
    }
    RET(launch_half(c, part, c->d_corder[part], P.ncell, c->d_queue + 0, d0, thr[0], g.smem[0], g.grid[0], c->side,
                    true, c->d_ccount[part] + 0));
    RET(launch_half(c, part, c->d_corder[part] + P.ncell, P.ncell, c->d_queue + 1, d1, thr[1], g.smem[1], g.grid[1],
                    c->stream, false, c->d_ccount[part] + 1));
    c->n_launch += 2;
    CK(cudaEventRecord(c->ev_join, c->side));
    CK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    if (g.cl_cap > 0) CK(cudaStreamWaitEvent(c->stream, c->ev_join2, 0));
    if (mlp_keeps_old(c))
        CK(cudaMemcpyAsync(c->d_pred_old[part], c->d_pred, sizeof(float) * DD_MLP_NOUT * P.ncell,
                           cudaMemcpyDeviceToDevice, c->stream));
    const long long dc[3] = {0, g.h2, g.w2};
    CK(cudaEventRecordWithFlags(c->gev[10 + (stage - 1)], c->stream, cudaEventRecordExternal));
    RET(launch_c2b(c, part, dc, g.smem_c2b, c->d_corder[part], c->d_ccount[part]));
    c->n_launch += 1;
    CK(cudaEventRecordWithFlags(ev[2], c->stream, cudaEventRecordExternal));
    c->cur = 1 - c->cur;
    return DD_OK;
}

// the min-cost flow of a captured iteration, as a host node (no CUDA calls)
void CUDART_CB flow_host_node(void* p) {
    dd_ctx* c = static_cast<dd_ctx*>(p);
    if (*c->h_guard) {
        c->g_skipped = true;
        return;
    }
    c->g_skipped = false;
    auto t0 = std::chrono::steady_clock::now();
    double value = 0.0;
    int32_t piv = 0;
    int frc = mcf_solve(c->mcf, c->h_cbar, c->h_w, &value, &piv);
    if (frc != DD_OK) {
        for (int i = 0; i < c->nb; ++i)
            for (int k = 0; k < 5; ++k) c->h_w[5 * i + k] = k == 0 ? c->h_m[i] : 0.0;
        value = 0.0;
    }
    c->g_value = value;
    c->g_piv = piv;
    c->g_frc = frc;
    c->g_ms_solve = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

int enqueue_flow_graph(dd_ctx* c) {
    CK(cudaEventRecordWithFlags(c->gev[6], c->stream, cudaEventRecordExternal));
    RET(launch_cbar(c));
    CK(cudaEventRecordWithFlags(c->gev[7], c->stream, cudaEventRecordExternal));
    RET(d2h(c->h_cbar, c->d_cbar, 5 * (size_t)c->nb, c->stream));
    RET(d2h(c->h_guard, c->d_guard, 1, c->stream));
    CK(cudaLaunchHostFunc(c->stream, flow_host_node, c));
    RET(h2d(c->d_w, c->h_w, 5 * (size_t)c->nb, c->stream));
    CK(cudaEventRecordWithFlags(c->gev[8], c->stream, cudaEventRecordExternal));
    CK(cudaMemsetAsync(c->d_status + 5, 0, sizeof(int), c->stream));
    RET(launch_plan_exchange(c, 3));
    RET(launch_exchange(c));
    c->n_launch += 4;  // k_cbar, k_xbox, k_plan_exchange, k_exchange
    CK(cudaEventRecordWithFlags(c->gev[9], c->stream, cudaEventRecordExternal));
    c->cur = 1 - c->cur;
    return DD_OK;
}

int graph_capture(dd_ctx* c, int parity) {
    cudaStream_t user = c->stream;
    const long long l0 = c->n_launch;
    c->stream = c->gstream;
    c->capturing = true;
    cudaError_t e = cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal);
    int rc = e == cudaSuccess ? DD_OK : dd_record_cuda_error(e, "cudaStreamBeginCapture");
    if (rc == DD_OK) rc = enqueue_half_graph(c, 0, 1);
    if (rc == DD_OK) rc = enqueue_half_graph(c, 1, 2);
    if (rc == DD_OK) rc = enqueue_flow_graph(c);
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess) {
        cudaError_t e2 = cudaStreamEndCapture(c->gstream, &graph);
        if (rc == DD_OK && e2 != cudaSuccess) rc = dd_record_cuda_error(e2, "cudaStreamEndCapture");
    }
    c->stream = user;
    c->capturing = false;
    c->status_slot = 0;
    c->cur = parity;
    const long long launches = c->n_launch - l0;
    c->n_launch = l0;
    if (rc == DD_OK) {
        auto& G = c->graph[parity];
        if (G.exec) cudaGraphExecDestroy(G.exec);
        G.exec = nullptr;
        cudaError_t e3 = cudaGraphInstantiate(&G.exec, graph, cudaGraphInstantiateFlagUseNodePriority);
        if (e3 != cudaSuccess) {
            G.exec = nullptr;
            rc = dd_record_cuda_error(e3, "cudaGraphInstantiate");
        } else {
            G.gen = c->gen;
            G.launches = launches;
        }
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc;
}

// one hybrid iteration from the captured graph; falls back to the eager steps
// from the stage whose buffers would have overflowed
int step_graph(dd_ctx* c, dd_stats* sa, dd_stats* sb, dd_flow_stats* sf, bool* used_graph) {
    const int parity = c->cur;
    auto& G = c->graph[parity];
    *used_graph = false;
    if (!G.exec || G.gen != c->gen) {
        int r = graph_prepare(c);
        if (r == DD_OK) r = graph_capture(c, parity);
        if (r != DD_OK) return step_eager(c, sa, sb, sf);  // boxes beyond what a graph holds
        c->n_capture += 1;
    }
    CK(cudaMemsetAsync(c->d_guard, 0, sizeof(int), c->stream));
    CK(cudaGraphLaunch(G.exec, c->stream));
    c->n_launch += G.launches;
    c->n_replay += 1;
    CK(cudaStreamSynchronize(c->stream));
    int status[kStatusInts];
    RET(d2h(c->h_guard, c->d_guard, 1, c->stream));
    RET(d2h(status, c->d_status, kStatusInts, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    RET(mlp_status(c, status[kStatusMlp]));
    const int guard = *c->h_guard;
    if (guard == 0) {
        c->cur = 1 - parity;
        for (auto& P : c->part) { P.warm_valid = true; P.solved = true; P.pred_old_valid = mlp_keeps_old(c); }
        c->last_part = 1;
        c->flow_ready = false;
        *used_graph = true;
        int rc = DD_OK;
        if (status[8 + 2] > 0 || status[16 + 2] > 0 || status[8 + 4] > 0 || status[16 + 4] > 0 || status[5] > 0)
            return DD_ERR_POOL;
        if (status[8 + 0] > 0 || status[16 + 0] > 0) rc = DD_ERR_MAXITER;
        if (c->g_frc != DD_OK) rc = DD_ERR_FLOW;
        return rc;
    }
    // a buffer would have overflowed at stage `guard`: nothing from that stage on
    // ran; continue eagerly from there (the eager steps grow the buffers and the
    // next iteration captures again with the sizes seen)
    CK(cudaMemsetAsync(c->d_guard, 0, sizeof(int), c->stream));
    c->gen += 1;
    c->n_fallback += 1;
    if (guard == 1) {
        c->cur = parity;
        return step_eager(c, sa, sb, sf, 0);
    }
    c->part[0].warm_valid = c->part[0].solved = true;
    c->part[0].pred_old_valid = mlp_keeps_old(c);
    // capped cells of the stages that ran in the graph stay in the returned status
    auto merge = [](int r_graph, int r_eager) {
        if (r_eager != DD_OK && r_eager != DD_ERR_MAXITER && r_eager != DD_ERR_FLOW) return r_eager;
        return r_eager == DD_ERR_FLOW ? r_eager : (r_graph != DD_OK ? r_graph : r_eager);
    };
    int rg = fill_stats(c, 0, sa, 1, c->gev[0], c->gev[1], c->gev[2], c->gev[10]);  // A ran in the graph
    if (rg != DD_OK && rg != DD_ERR_MAXITER) return rg;
    if (guard == 2) {
        c->cur = 1 - parity;
        c->last_part = 0;
        c->flow_ready = true;
        return merge(rg, step_eager(c, sa, sb, sf, 1));
    }
    c->part[1].warm_valid = c->part[1].solved = true;
    c->part[1].pred_old_valid = mlp_keeps_old(c);
    {
        int r = fill_stats(c, 1, sb, 2, c->gev[3], c->gev[4], c->gev[5], c->gev[11]);  // B ran in the graph
        if (r != DD_OK && r != DD_ERR_MAXITER) return r;
        if (r != DD_OK) rg = r;
    }
    c->cur = parity;
    c->last_part = 1;
    c->flow_ready = true;
    return merge(rg, step_eager(c, sa, sb, sf, 2));
}

}  // namespace

// statistics of the last replayed graph iteration into the context's copies
static int resolve_graph_stats(dd_ctx* c) {
    int r1 = fill_stats(c, 0, &c->last_sa, 1, c->gev[0], c->gev[1], c->gev[2], c->gev[10]);
    if (r1 != DD_OK && r1 != DD_ERR_MAXITER) return r1;
    int r2 = fill_stats(c, 1, &c->last_sb, 2, c->gev[3], c->gev[4], c->gev[5], c->gev[11]);
    if (r2 != DD_OK && r2 != DD_ERR_MAXITER) return r2;
    flow_stats(c, c->g_value, c->g_piv, c->g_ms_solve, c->gev + 6, &c->last_sf);
    c->stats_pending = false;
    c->last_stats_valid = true;
    return DD_OK;
}

int dd_step(dd_ctx* c, int n, dd_stats* sa, dd_stats* sb, dd_flow_stats* sf) {
    if (!c || n < 0) return DD_ERR_ARG;
    if (c->pool[c->cur] == nullptr) return DD_ERR_STATE;
    // statistics go to the context's copies; the caller's structures get the last
    // iteration's. Without any structure, a replayed iteration reads nothing back
    // (dd_step_stats and dd_get_objective do it when asked).
    const bool want = sa || sb || sf;
    int rc = DD_OK;
    for (int k = 0; k < n; ++k) {
        // the graph needs the sizes, flow solver and warm starts of one eager iteration
        const bool can_graph = !(c->opt.flags & DD_FLAG_NO_GRAPH) && c->mcf && c->seen.out > 0 &&
                               c->part[0].warm_valid && c->part[1].warm_valid;
        bool used_graph = false;
        int r = can_graph ? step_graph(c, &c->last_sa, &c->last_sb, &c->last_sf, &used_graph)
                          : step_eager(c, &c->last_sa, &c->last_sb, &c->last_sf);
        if (r != DD_OK && r != DD_ERR_MAXITER && r != DD_ERR_FLOW) return r;
        if (r == DD_ERR_FLOW || (r == DD_ERR_MAXITER && rc == DD_OK)) rc = r;  // a failed flow solve first
        c->stats_pending = used_graph;
        c->last_stats_valid = !used_graph;
        // capped cells (DD_ERR_MAXITER, already in r) neither end the statistics
        // nor the remaining iterations
        if (used_graph && want) RET(resolve_graph_stats(c));
    }
    if (n > 0 && want && c->last_stats_valid) {
        if (sa) *sa = c->last_sa;
        if (sb) *sb = c->last_sb;
        if (sf) *sf = c->last_sf;
    }
    return rc;
}

int dd_step_stats(dd_ctx* c, dd_stats* sa, dd_stats* sb, dd_flow_stats* sf) {
    if (!c) return DD_ERR_ARG;
    if (c->stats_pending) RET(resolve_graph_stats(c));
    if (!c->last_stats_valid) return DD_ERR_STATE;
    if (sa) *sa = c->last_sa;
    if (sb) *sb = c->last_sb;
    if (sf) *sf = c->last_sf;
    return DD_OK;
}

int dd_get_plan(dd_ctx* c, int32_t* hdr, double* data, size_t* count) {
    if (!c || !count) return DD_ERR_ARG;
    const int nb = c->nb;
    std::vector<int32_t> bh((size_t)BH_N * nb);
    RET(d2h(bh.data(), c->bhdr[c->cur], bh.size(), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::vector<long long> soff((size_t)nb + 1, 0);
    size_t n = 0;
    for (int i = 0; i < nb; ++i) {
        soff[i] = (long long)n;
        n += (size_t)bh[BH_N * i + BH_H] * bh[BH_N * i + BH_W];
    }
    soff[nb] = (long long)n;
    const bool devp = (c->opt.flags & DD_FLAG_DEVICE_PTRS) != 0;
    if (hdr) {
        std::vector<int32_t> hh(4 * (size_t)nb);
        for (int i = 0; i < nb; ++i)
            for (int k = 0; k < 4; ++k) hh[4 * i + k] = bh[BH_N * i + k];
        if (devp) {
            RET(h2d(hdr, hh.data(), hh.size(), c->stream));
            CK(cudaStreamSynchronize(c->stream));
        } else {
            std::memcpy(hdr, hh.data(), sizeof(int32_t) * hh.size());
        }
    }
    if (!data) { *count = n; return DD_OK; }
    if (*count < n) return DD_ERR_ARG;
    // unpack on the device (FP32 pool rows -> packed FP64) and copy out once
    RET(ensure_plan64(c, n));
    RET(h2d(c->d_soff, soff.data(), soff.size(), c->stream));
    RET(launch_unpack_plan(c));
    c->n_launch += 1;
    if (devp) {
        if (n) CK(cudaMemcpyAsync(data, c->d_plan64, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        RET(d2h(data, c->d_plan64, n, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    c->n_d2h += (long long)(sizeof(double) * n + sizeof(int32_t) * bh.size());
    *count = n;
    return DD_OK;
}

static int get_comp(dd_ctx* c, int part, std::vector<int32_t>& ch, std::vector<float>& b, std::vector<float>& nuJ,
                    bool want_b) {
    DevPart& P = c->part[part];
    ch.resize((size_t)CH_N * P.ncell);
    RET(d2h(ch.data(), P.chdr, ch.size(), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    size_t used = 0;
    for (int J = 0; J < P.ncell; ++J) {
        const int32_t* x = &ch[CH_N * J];
        long long comp = ((long long)x[CH_COMP_HI] << 32) | (unsigned int)x[CH_COMP_LO];
        used = std::max(used, (size_t)comp + (size_t)x[CH_H] * x[CH_STRIDE]);
    }
    nuJ.resize(used);
    RET(d2h(nuJ.data(), P.comp_nu, used, c->stream));
    if (want_b) {
        b.resize(used);
        RET(d2h(b.data(), P.comp_b, used, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return DD_OK;
}

int dd_get_composite(dd_ctx* c, int part, int32_t* hdr, double* data, size_t* count) {
    if (!c || !count || part < 0 || part > 1) return DD_ERR_ARG;
    DevPart& P = c->part[part];
    if (!P.solved) return DD_ERR_STATE;
    std::vector<int32_t> ch;
    std::vector<float> b, nuJ;
    RET(get_comp(c, part, ch, b, nuJ, false));
    size_t n = 0;
    for (int J = 0; J < P.ncell; ++J) n += (size_t)ch[CH_N * J + CH_H] * ch[CH_N * J + CH_W];
    if (hdr)
        for (int J = 0; J < P.ncell; ++J)
            for (int k = 0; k < 4; ++k) hdr[4 * J + k] = ch[CH_N * J + k];
    if (!data) { *count = n; return DD_OK; }
    if (*count < n) return DD_ERR_ARG;
    size_t k = 0;
    for (int J = 0; J < P.ncell; ++J) {
        const int32_t* x = &ch[CH_N * J];
        long long comp = ((long long)x[CH_COMP_HI] << 32) | (unsigned int)x[CH_COMP_LO];
        for (int r = 0; r < x[CH_H]; ++r)
            for (int q = 0; q < x[CH_W]; ++q) data[k++] = nuJ[(size_t)comp + (size_t)r * x[CH_STRIDE] + q];
    }
    *count = n;
    return DD_OK;
}

static int get_duals_host(dd_ctx* c, int part, double* alpha, int32_t* hdr, double* beta, size_t* count);

int dd_get_duals(dd_ctx* c, int part, double* alpha, int32_t* hdr, double* beta, size_t* count) {
    if (!c || !count || part < 0 || part > 1) return DD_ERR_ARG;
    if (!(c->opt.flags & DD_FLAG_DEVICE_PTRS)) return get_duals_host(c, part, alpha, hdr, beta, count);
    // device outputs: the gauge conversion runs on the host, the results are copied in once
    const size_t np = (size_t)c->N1 * c->N2;
    std::vector<int32_t> hh(4 * (size_t)c->part[part].ncell);
    size_t n = 0;
    RET(get_duals_host(c, part, nullptr, hh.data(), nullptr, &n));
    if (hdr) RET(h2d(hdr, hh.data(), hh.size(), c->stream));
    if (!alpha && !beta) {
        CK(cudaStreamSynchronize(c->stream));
        *count = n;
        return DD_OK;
    }
    if (beta && *count < n) return DD_ERR_ARG;
    std::vector<double> ah(alpha ? np : 0), bh(beta ? n : 0);
    size_t n2 = n;
    RET(get_duals_host(c, part, alpha ? ah.data() : nullptr, nullptr, beta ? bh.data() : nullptr, &n2));
    if (alpha) RET(h2d(alpha, ah.data(), np, c->stream));
    if (beta) RET(h2d(beta, bh.data(), n, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *count = n;
    return DD_OK;
}

static int get_duals_host(dd_ctx* c, int part, double* alpha, int32_t* hdr, double* beta, size_t* count) {
    DevPart& P = c->part[part];
    if (!P.solved) return DD_ERR_STATE;
    std::vector<int32_t> ch, xb((size_t)XB_N * P.ncell);
    std::vector<float> b, nuJ, al((size_t)c->amax * P.ncell), g(8 * (size_t)P.ncell);
    RET(get_comp(c, part, ch, b, nuJ, true));
    RET(d2h(xb.data(), P.xblk, xb.size(), c->stream));
    RET(d2h(al.data(), P.alpha, al.size(), c->stream));
    RET(d2h(g.data(), P.gauge, g.size(), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    size_t n = 0;
    for (int J = 0; J < P.ncell; ++J) n += (size_t)ch[CH_N * J + CH_H] * ch[CH_N * J + CH_W];
    if (hdr)
        for (int J = 0; J < P.ncell; ++J)
            for (int k = 0; k < 4; ++k) hdr[4 * J + k] = ch[CH_N * J + k];
    if (!beta && !alpha) { *count = n; return DD_OK; }
    if (beta && *count < n) return DD_ERR_ARG;
    const double k2 = c->k2d, eps = c->eps;
    size_t k = 0;
    for (int J = 0; J < P.ncell; ++J) {
        const int32_t* x = &ch[CH_N * J];
        const int32_t* X = &xb[XB_N * J];
        const int hx = X[XB_HX], wx = X[XB_WX], h = x[CH_H], w = x[CH_W];
        // undo the kernel's reparametrisation (shift d, stretch l, origins uc / vc)
        const float* gg = &g[8 * J];
        const double l1 = gg[2], l2 = gg[3];
        const double uc1 = gg[4], uc2 = gg[5], vc1 = gg[6], vc2 = gg[7];
        const double d1 = (double)(X[XB_R0] - x[CH_O1]) + uc1 - vc1, d2 = (double)(X[XB_C0] - x[CH_O2]) + uc2 - vc2;
        const double hd = 0.5 * k2 * (d1 * d1 + d2 * d2);
        // per-row / per-column kernel minima the kernel subtracted from b:
        // B(v) = k2 l (ubar* - t)^2 at the grid point nearest to t = vbar / l
        std::vector<double> B1(h), B2(w);
        for (int r = 0; r < h; ++r) {
            const double tt = (r - vc1) / l1;
            const int us = std::min(hx - 1, std::max(0, (int)std::nearbyint(tt + uc1)));
            const double w0 = 2.0 * ((us - uc1) - tt);
            B1[r] = 0.25 * k2 * l1 * w0 * w0;
        }
        for (int q = 0; q < w; ++q) {
            const double tt = (q - vc2) / l2;
            const int us = std::min(wx - 1, std::max(0, (int)std::nearbyint(tt + uc2)));
            const double w0 = 2.0 * ((us - uc2) - tt);
            B2[q] = 0.25 * k2 * l2 * w0 * w0;
        }
        if (alpha)
            for (int u1 = 0; u1 < hx; ++u1)
                for (int u2 = 0; u2 < wx; ++u2) {
                    size_t px = (size_t)(X[XB_R0] + u1) * c->N2 + X[XB_C0] + u2;
                    double a = al[(size_t)c->amax * J + u1 * wx + u2];
                    double mu = c->h_mu[px];
                    const double ub1 = u1 - uc1, ub2 = u2 - uc2;
                    alpha[px] = mu > 0 ? eps * (kLn2 * (a - k2 * ((l1 - 1) * ub1 * ub1 + (l2 - 1) * ub2 * ub2) +
                                                        2 * k2 * (d1 * ub1 + d2 * ub2) + hd) -
                                                std::log(mu))
                                       : -INFINITY;
                }
        long long comp = ((long long)x[CH_COMP_HI] << 32) | (unsigned int)x[CH_COMP_LO];
        for (int r = 0; r < h; ++r)
            for (int q = 0; q < w; ++q) {
                double nj = nuJ[(size_t)comp + (size_t)r * x[CH_STRIDE] + q];
                double bb = b[(size_t)comp + (size_t)r * x[CH_STRIDE] + q];
                size_t py = (size_t)(x[CH_O1] + r) * c->N2 + x[CH_O2] + q;
                double val = -INFINITY;
                const double vb1 = r - vc1, vb2 = q - vc2;
                if (nj > 0)
                    val = eps * (kLn2 * (bb + B1[r] + B2[q] - k2 * ((1 / l1 - 1) * vb1 * vb1 + (1 / l2 - 1) * vb2 * vb2) -
                                         2 * k2 * (d1 * vb1 + d2 * vb2) + hd) -
                                 std::log(c->h_nu[py]));
                if (beta) beta[k] = val;
                ++k;
            }
    }
    *count = n;
    return DD_OK;
}

int dd_get_cell_stats(dd_ctx* c, int part, int32_t* iters, double* err) {
    if (!c || part < 0 || part > 1) return DD_ERR_ARG;
    DevPart& P = c->part[part];
    if (!P.solved) return DD_ERR_STATE;
    if (iters) RET(d2h(iters, P.iters, P.ncell, c->stream));
    if (err) RET(d2h(err, P.err, P.ncell, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return DD_OK;
}

int dd_get_objective(dd_ctx* c, double* E, double* l1_x, double* l1_y) {
    if (!c) return DD_ERR_ARG;
    if (c->stats_pending) RET(resolve_graph_stats(c));  // sets the objective of the last half-iteration
    if (E) *E = c->last_E;
    if (l1_x) *l1_x = c->last_l1x;
    if (l1_y) {
        RET(launch_l1y(c, c->d_red));
        RET(d2h(l1_y, c->d_red, 1, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return DD_OK;
}

int dd_debug_cell(dd_ctx* c, int part, int J, float* a, float* b, float* gauge, int32_t* geom) {
    if (!c || part < 0 || part > 1 || !geom) return DD_ERR_ARG;
    DevPart& P = c->part[part];
    if (!P.solved || J < 0 || J >= P.ncell) return DD_ERR_STATE;
    int32_t ch[CH_N];
    RET(d2h(ch, P.chdr + (size_t)CH_N * J, CH_N, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const int32_t* X = &P.h_xblk[XB_N * J];
    int32_t gm[8] = {X[XB_R0], X[XB_C0], X[XB_HX], X[XB_WX], ch[CH_O1], ch[CH_O2], ch[CH_H], ch[CH_W]};
    std::memcpy(geom, gm, sizeof(gm));
    if (a) RET(d2h(a, P.alpha + (size_t)c->amax * J, (size_t)X[XB_HX] * X[XB_WX], c->stream));
    if (gauge) RET(d2h(gauge, P.gauge + 8 * (size_t)J, 8, c->stream));
    if (b) {
        long long comp = ((long long)ch[CH_COMP_HI] << 32) | (unsigned int)ch[CH_COMP_LO];
        for (int r = 0; r < ch[CH_H]; ++r)
            RET(d2h(b + (size_t)r * ch[CH_W], P.comp_b + comp + (size_t)r * ch[CH_STRIDE], ch[CH_W], c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return DD_OK;
}

int dd_get_trace(dd_ctx* c, int part, int64_t* trace) {
    if (!c || !trace || part < 0 || part > 1) return DD_ERR_ARG;
    if (!(c->opt.flags & DD_FLAG_TRACE)) return DD_ERR_STATE;
    RET(d2h(reinterpret_cast<long long*>(trace), c->d_trace[part], 8 * (size_t)c->part[part].ncell, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return DD_OK;
}

int dd_get_graph_counters(dd_ctx* c, int64_t* captures, int64_t* replays, int64_t* fallbacks) {
    if (!c) return DD_ERR_ARG;
    if (captures) *captures = c->n_capture;
    if (replays) *replays = c->n_replay;
    if (fallbacks) *fallbacks = c->n_fallback;
    return DD_OK;
}

int dd_get_counters(dd_ctx* c, int64_t* launches, int64_t* h2d_bytes, int64_t* d2h_bytes) {
    if (!c) return DD_ERR_ARG;
    if (launches) *launches = c->n_launch;
    if (h2d_bytes) *h2d_bytes = c->n_h2d;
    if (d2h_bytes) *d2h_bytes = c->n_d2h;
    return DD_OK;
}

int dd_get_partition(dd_ctx* c, int part, int32_t* members, int32_t* ncell) {
    if (!c || part < 0 || part > 1 || !ncell) return DD_ERR_ARG;
    DevPart& P = c->part[part];
    *ncell = P.ncell;
    if (members) std::memcpy(members, P.h_members.data(), sizeof(int32_t) * P.h_members.size());
    return DD_OK;
}

int dd_get_neighbours(dd_ctx* c, int32_t* nbr) {
    if (!c || !nbr) return DD_ERR_ARG;
    std::memcpy(nbr, c->h_nbr.data(), sizeof(int32_t) * c->h_nbr.size());
    return DD_OK;
}

int dd_get_basic_moments(dd_ctx* c, double* D, double* mass, double* ybar, double* var) {
    if (!c) return DD_ERR_ARG;
    std::vector<double> bm((size_t)BM_N * c->nb);
    RET(d2h(bm.data(), c->d_bmom, bm.size(), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < c->nb; ++i) {
        if (D) D[i] = bm[BM_N * i + BM_D];
        if (mass) mass[i] = bm[BM_N * i + BM_MASS];
        if (ybar) { ybar[2 * i] = bm[BM_N * i + BM_Y1]; ybar[2 * i + 1] = bm[BM_N * i + BM_Y2]; }
        if (var) var[i] = bm[BM_N * i + BM_VAR];
    }
    return DD_OK;
}

int dd_get_flow(dd_ctx* c, double* cbar, double* w) {
    if (!c) return DD_ERR_ARG;
    if (cbar) std::memcpy(cbar, c->h_cbar, sizeof(double) * 5 * c->nb);
    if (w) std::memcpy(w, c->h_w, sizeof(double) * 5 * c->nb);
    return DD_OK;
}

int dd_get_prebalance(dd_ctx* c, int32_t* hdr, double* data, size_t* count) {
    if (!c || !count) return DD_ERR_ARG;
    if (!(c->opt.flags & DD_FLAG_KEEP_PREBALANCE) || c->last_part < 0) return DD_ERR_STATE;
    DevPart& P = c->part[c->last_part];
    std::vector<int32_t> ch((size_t)CH_N * P.ncell);
    RET(d2h(ch.data(), P.chdr, ch.size(), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    // basic cell i -> (cell J, member k)
    std::vector<int> cellof(c->nb, -1), memk(c->nb, -1);
    for (int J = 0; J < P.ncell; ++J)
        for (int k = 0; k < 4; ++k) {
            int i = P.h_members[4 * J + k];
            if (i >= 0) { cellof[i] = J; memk[i] = k; }
        }
    size_t n = 0, used = 0;
    for (int i = 0; i < c->nb; ++i) {
        const int32_t* x = &ch[CH_N * cellof[i]];
        n += (size_t)x[CH_H] * x[CH_W];
        size_t area = (size_t)x[CH_H] * x[CH_STRIDE];
        used = std::max(used, (size_t)x[CH_OUT_SLOT] + (memk[i] + 1) * area);
    }
    if (hdr)
        for (int i = 0; i < c->nb; ++i)
            for (int k = 0; k < 4; ++k) hdr[4 * i + k] = ch[CH_N * cellof[i] + k];
    if (!data) { *count = n; return DD_OK; }
    if (*count < n) return DD_ERR_ARG;
    std::vector<float> buf(used);
    RET(d2h(buf.data(), c->d_pre, used, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    size_t k = 0;
    for (int i = 0; i < c->nb; ++i) {
        const int32_t* x = &ch[CH_N * cellof[i]];
        size_t area = (size_t)x[CH_H] * x[CH_STRIDE];
        size_t base = (size_t)x[CH_OUT_SLOT] + memk[i] * area;
        for (int r = 0; r < x[CH_H]; ++r)
            for (int q = 0; q < x[CH_W]; ++q) data[k++] = buf[base + (size_t)r * x[CH_STRIDE] + q];
    }
    *count = n;
    return DD_OK;
}

int dd_set_warmstart_weights(dd_ctx* c, const float* params, int64_t n) {
    if (!c || !params || n != DD_MLP_NPARAMS || c->s != 4) return DD_ERR_ARG;
    RET(ensure_learned_buffers(c));
    if (!c->mlp) RET(dd_mlp_create(std::max(c->part[0].ncell, c->part[1].ncell), c->stream, &c->mlp));
    RET(dd_mlp_set_params(c->mlp, params, n));
    c->mlp_ready = true;
    return DD_OK;
}

int dd_collect_cells(dd_ctx* c, int part, uint16_t* feat_dev, float* targ_dev, int32_t max_rows, int32_t* rows) {
    if (!c || !rows || part < 0 || part > 1) return DD_ERR_ARG;
    if (!(c->opt.flags & DD_FLAG_COLLECT) || c->last_part != part || !c->part[part].solved) return DD_ERR_STATE;
    const int n = c->n_full[part];
    *rows = n;
    if (!feat_dev) return DD_OK;
    if (!targ_dev || max_rows < n) return DD_ERR_ARG;
    RET(launch_collect(c, n, c->d_full[part], feat_dev, targ_dev));
    c->n_launch += 1;
    CK(cudaStreamSynchronize(c->stream));
    return DD_OK;
}

}  // extern "C"
