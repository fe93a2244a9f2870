// Gluing edge candidates with entropic gamma_ij (Def. 3.7, Remark 3.8; the
// paper's small-eps_gamma choice), in the basic-cell box representation.
//
// The flow update only needs the edge costs c_bar_ij of the candidates (the new
// basic marginals, Eq. (flow-update-cell-marginals), do not depend on the
// candidate). For the glued candidate pi_hat_ij(x, y) = sum_{x'} gamma(x', x)
// pi_i(x', y) / mu(x') and D_i = <c, pi_i> from the same plan,
//     c_bar_ij = (h^2 / m_i) sum_{x' in X_i} r(x') [A_ij(x') - 2 B_ij(x') . d(x')],
// with, for every pixel x' of basic cell i,
//     A_ij(x') = E_gamma[|x - x'|^2 | x'],  B_ij(x') = E_gamma[x - x' | x']
// (moments of the disintegration of gamma_ij at x', pixels), and
//     r(x') = sum_y pi_i(x', y),  d(x') = E_pi[y | x'] - x'
// (mass and mean displacement of the cell plan at x'). (The variance terms of
// <c, pi_hat_ij> and D_i / m_i cancel because every disintegration of gamma_ij
// is a probability measure.)
//
//  k_gamma       gamma_ij between mu_i / m_i and mu_j / m_j for the squared
//                distance on X and eps_gamma: log-domain Sinkhorn in FP64 with
//                Anderson acceleration of the X-side potential, one warp per
//                directed edge, to an L1 marginal error <= 1e-13; writes A, B.
//                mu never changes, so this runs once per context.
//  k_cbar_glued  the edge costs above, one thread per basic cell, FP64.
// r and d come from k_c2b (per-pixel moments of the Gibbs cell plan).
#include <cuda_runtime.h>

#include <cstdint>

#include "dd_internal.h"

namespace {

constexpr int kGamMaxPix = 64;  // basic cells up to 8 x 8 pixels
constexpr int kGamAA = 5;       // Anderson memory of the gamma solve
constexpr int kGamWarps = 4;    // warps (edges) per CTA

__device__ __forceinline__ double warp_sum_d(double x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
__device__ __forceinline__ double warp_max_d(double x) {
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

struct GamSmem {
    double a[kGamMaxPix], b[kGamMaxPix], la[kGamMaxPix], lb[kGamMaxPix];
    double u[kGamMaxPix], v[kGamMaxPix], un[kGamMaxPix];
    int p1[kGamMaxPix], p2[kGamMaxPix], q1[kGamMaxPix], q2[kGamMaxPix];  // pixel coordinates (X_i, X_j)
    double dG[kGamAA][kGamMaxPix], dX[kGamAA][kGamMaxPix], gp[kGamMaxPix], xp[kGamMaxPix];
    double M[kGamAA][kGamAA];
};

// v(x) = -e log sum_{x'} exp((u(x') - c(x', x)) / e) a(x')   (lane owns columns x = lane, lane + 32)
__device__ void gam_v_update(GamSmem& S, int n, double k2) {
    const int lane = threadIdx.x & 31;
    for (int x = lane; x < n; x += 32) {
        double mx = -1e300;
        for (int q = 0; q < n; ++q) {
            const double d1 = S.p1[q] - S.q1[x], d2 = S.p2[q] - S.q2[x];
            mx = fmax(mx, S.u[q] - k2 * (d1 * d1 + d2 * d2) + S.la[q]);
        }
        double s = 0.0;
        for (int q = 0; q < n; ++q) {
            const double d1 = S.p1[q] - S.q1[x], d2 = S.p2[q] - S.q2[x];
            s += exp(S.u[q] - k2 * (d1 * d1 + d2 * d2) + S.la[q] - mx);
        }
        S.v[x] = -(mx + log(s));
    }
    __syncwarp();
}

// un(x') = -log sum_x exp(v(x) - c(x', x)) b(x)   (potentials in units of e)
__device__ void gam_u_update(GamSmem& S, int n, double k2) {
    const int lane = threadIdx.x & 31;
    for (int q = lane; q < n; q += 32) {
        double mx = -1e300;
        for (int x = 0; x < n; ++x) {
            const double d1 = S.p1[q] - S.q1[x], d2 = S.p2[q] - S.q2[x];
            mx = fmax(mx, S.v[x] - k2 * (d1 * d1 + d2 * d2) + S.lb[x]);
        }
        double s = 0.0;
        for (int x = 0; x < n; ++x) {
            const double d1 = S.p1[q] - S.q1[x], d2 = S.p2[q] - S.q2[x];
            s += exp(S.v[x] - k2 * (d1 * d1 + d2 * d2) + S.lb[x] - mx);
        }
        S.un[q] = -(mx + log(s));
    }
    __syncwarp();
}

// One warp per directed edge (i, k), k = 1..4. Potentials are kept divided by
// eps_gamma; k2 = h^2 / eps_gamma per squared pixel.
__global__ void __launch_bounds__(32 * kGamWarps) k_gamma(int nb, int s, int n2, const int32_t* __restrict__ nbr,
                                                         const double* __restrict__ mu, double k2, int max_iter,
                                                         double* __restrict__ gAB, int* __restrict__ status) {
    __shared__ GamSmem sm[kGamWarps];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long e = (long long)blockIdx.x * kGamWarps + w;  // edge index i * 4 + (k - 1)
    if (e >= 4LL * nb) return;
    const int i = (int)(e >> 2), k = (int)(e & 3) + 1;
    const int j = nbr[5 * i + k];
    GamSmem& S = sm[w];
    const int n = s * s;
    double* out = gAB + e * 3 * n;
    if (j < 0) {
        for (int q = lane; q < 3 * n; q += 32) out[q] = 0.0;
        return;
    }
    const int nc = n2 / s;
    const int ri = (i / nc) * s, ci = (i % nc) * s, rj = (j / nc) * s, cj = (j % nc) * s;
    double sa = 0.0, sb = 0.0;
    for (int q = lane; q < n; q += 32) {
        S.p1[q] = ri + q / s; S.p2[q] = ci + q % s;
        S.q1[q] = rj + q / s; S.q2[q] = cj + q % s;
        S.a[q] = mu[(long long)S.p1[q] * n2 + S.p2[q]];
        S.b[q] = mu[(long long)S.q1[q] * n2 + S.q2[q]];
        sa += S.a[q];
        sb += S.b[q];
    }
    sa = warp_sum_d(sa);
    sb = warp_sum_d(sb);
    for (int q = lane; q < n; q += 32) {
        S.a[q] /= sa;
        S.b[q] /= sb;
        S.la[q] = S.a[q] > 0.0 ? log(S.a[q]) : -1e300;
        S.lb[q] = S.b[q] > 0.0 ? log(S.b[q]) : -1e300;
        S.u[q] = 0.0;
    }
    __syncwarp();
    int cnt = 0, head = 0;
    bool prev = false, done = false;
    double err_last = 1e300;
    for (int it = 0; it < max_iter && !done; ++it) {
        gam_v_update(S, n, k2);
        gam_u_update(S, n, k2);
        // L1 X-marginal error of the pair (u, v): sum a |exp(u - un) - 1|
        double el = 0.0;
        for (int q = lane; q < n; q += 32)
            if (S.a[q] > 0.0) el += S.a[q] * fabs(expm1(S.u[q] - S.un[q]));
        const double err = warp_sum_d(el);
        if (err <= 1e-13) {
            done = true;
            break;
        }
        // Anderson step on u (restart when the error more than doubled)
        if (prev && err > 2.0 * err_last) {
            cnt = head = 0;
            prev = false;
        }
        err_last = err;
        for (int q = lane; q < n; q += 32) {
            const double g = S.a[q] > 0.0 ? S.un[q] - S.u[q] : 0.0;
            if (prev) {
                S.dG[head][q] = g - S.gp[q];
                S.dX[head][q] = S.u[q] - S.xp[q];
            }
            S.gp[q] = g;
            S.xp[q] = S.u[q];
        }
        __syncwarp();
        const int qn = prev ? min(cnt + 1, kGamAA) : cnt;
        if (prev) {
            for (int jj = 0; jj < qn; ++jj) {
                double pm = 0.0;
                for (int q = lane; q < n; q += 32) pm += S.a[q] * S.dG[head][q] * S.dG[jj][q];
                pm = warp_sum_d(pm);
                if (lane == 0) { S.M[head][jj] = pm; S.M[jj][head] = pm; }
            }
            cnt = qn;
            head = head + 1 == kGamAA ? 0 : head + 1;
        }
        prev = true;
        __syncwarp();
        double gam[kGamAA] = {0.0, 0.0, 0.0, 0.0, 0.0};
        bool ok = qn > 0;
        if (ok) {
            double r[kGamAA];
            for (int jj = 0; jj < qn; ++jj) {
                double pr = 0.0;
                for (int q = lane; q < n; q += 32) pr += S.a[q] * S.dG[jj][q] * S.gp[q];
                r[jj] = warp_sum_d(pr);
            }
            // Cholesky of M + lam I, every lane alike
            double L[kGamAA][kGamAA];
            double tr = 0.0;
            for (int a = 0; a < qn; ++a) tr += S.M[a][a];
            const double lam = 1e-12 * tr / qn + 1e-300;
            for (int a = 0; a < qn && ok; ++a) {
                for (int b = 0; b <= a; ++b) {
                    double v = S.M[a][b] + (a == b ? lam : 0.0);
                    for (int c = 0; c < b; ++c) v -= L[a][c] * L[b][c];
                    if (a == b) {
                        if (!(v > 0.0)) { ok = false; break; }
                        L[a][a] = sqrt(v);
                    } else {
                        L[a][b] = v / L[b][b];
                    }
                }
            }
            if (ok) {
                double y[kGamAA];
                for (int a = 0; a < qn; ++a) {
                    double v = r[a];
                    for (int c = 0; c < a; ++c) v -= L[a][c] * y[c];
                    y[a] = v / L[a][a];
                }
                for (int a = qn - 1; a >= 0; --a) {
                    double v = y[a];
                    for (int c = a + 1; c < qn; ++c) v -= L[c][a] * gam[c];
                    gam[a] = v / L[a][a];
                }
                double gs = 0.0;
                for (int a = 0; a < qn; ++a) gs += fabs(gam[a]);
                ok = gs <= 1e6 && isfinite(gs);
            }
            if (!ok) {
                cnt = head = 0;
                prev = false;
            }
        }
        for (int q = lane; q < n; q += 32) {
            if (!(S.a[q] > 0.0)) { S.u[q] = S.un[q]; continue; }
            double x = S.un[q];
            if (ok) {
                x = S.xp[q] + S.gp[q];
                for (int a = 0; a < qn; ++a) x -= gam[a] * (S.dX[a][q] + S.dG[a][q]);
            }
            S.u[q] = x;
        }
        __syncwarp();
    }
    if (!done && lane == 0) atomicAdd(status, 1);
    // the plan of the last pair: gamma(x', x) = a b exp(u + v - c) with v = V(u):
    // recompute v from the final u, then the conditional moments at each x'
    gam_v_update(S, n, k2);
    for (int q = lane; q < n; q += 32) {
        double mass = 0.0, A = 0.0, B1 = 0.0, B2 = 0.0;
        for (int x = 0; x < n; ++x) {
            const double d1 = S.q1[x] - S.p1[q], d2 = S.q2[x] - S.p2[q];
            const double g = (S.a[q] > 0.0 && S.b[x] > 0.0)
                                 ? exp(S.u[q] + S.v[x] - k2 * (d1 * d1 + d2 * d2) + S.la[q] + S.lb[x])
                                 : 0.0;
            mass += g;
            A += g * (d1 * d1 + d2 * d2);
            B1 += g * d1;
            B2 += g * d2;
        }
        const double inv = mass > 0.0 ? 1.0 / mass : 0.0;
        out[3 * q + 0] = A * inv;
        out[3 * q + 1] = B1 * inv;
        out[3 * q + 2] = B2 * inv;
    }
}

// c_bar_ij = (h^2 / m_i) sum_{x'} r(x') [A_ij(x') - 2 B_ij(x') . d(x')], c_bar_ii = 0
__global__ void k_cbar_glued(int nb, int n, const int32_t* __restrict__ nbr, const double* __restrict__ gAB,
                             const double* __restrict__ pmom, const double* __restrict__ m, double h2,
                             double* __restrict__ cbar, const int* __restrict__ guard) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 5 * nb || (guard && *guard)) return;
    const int i = t / 5, k = t - 5 * i;
    const int j = nbr[5 * i + k];
    double c = 0.0;
    if (j >= 0 && j != i) {
        const double* ab = gAB + ((long long)i * 4 + (k - 1)) * 3 * n;
        const double* pm = pmom + (long long)i * 3 * n;
        for (int q = 0; q < n; ++q)
            c += pm[3 * q] * (ab[3 * q] - 2.0 * (ab[3 * q + 1] * pm[3 * q + 1] + ab[3 * q + 2] * pm[3 * q + 2]));
        c *= h2 / m[i];
    }
    cbar[t] = c;
}

}  // namespace

size_t glue_smem_probe() { return sizeof(GamSmem) * kGamWarps; }

int launch_gamma(dd_ctx* c, int* status_dev) {
    const int n = c->s * c->s;
    if (n > kGamMaxPix) return DD_ERR_ARG;
    const double k2 = c->h * c->h / c->opt.eps_gamma;
    const long long edges = 4LL * c->nb;
    const int grid = (int)((edges + kGamWarps - 1) / kGamWarps);
    k_gamma<<<grid, 32 * kGamWarps, 0, c->stream>>>(c->nb, c->s, c->N2, c->d_nbr, c->d_mu, k2, 20000, c->d_gAB,
                                                   status_dev);
    return launch_status(__func__);
}

int launch_cbar_glued(dd_ctx* c) {
    const int n = c->s * c->s;
    k_cbar_glued<<<(5 * c->nb + 255) / 256, 256, 0, c->stream>>>(c->nb, n, c->d_nbr, c->d_gAB, c->d_pmom, c->d_m,
                                                                 c->h * c->h, c->d_cbar,
                                                                 c->capturing ? c->d_guard : nullptr);
    return launch_status(__func__);
}
