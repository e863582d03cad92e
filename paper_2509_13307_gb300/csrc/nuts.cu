// No-U-Turn sampler driver (Hoffman & Gelman 2014: the efficient NUTS with the
// slice variable and dual averaging) on the library's likelihood gradients,
// for the HMC comparison runs the paper sets against nested sampling (Sec. 3.2).
//
// The chains advance in lockstep: every trajectory doubling of every active
// chain builds its new subtree of the same height, so each leapfrog round is
// one batched gradient evaluation (loglike_grad_batch on the device) over the
// chains still building.  The per-chain control (slice, U-turn checks of every
// completed sub-subtree, reservoir choice of the subtree candidate, merge,
// dual averaging, diagonal mass adaptation) runs on the host in FP64; the
// target is the posterior in unconstrained coordinates z with unit-cube
// coordinate c = 1 / (1 + e^-z) and theta = prior transform(c) (device),
// log p(z) = log L(theta) + sum ln(c (1 - c)).  Random numbers: Philox4x32-10
// counters (purpose | j << 8, iteration, chain, extra) shared with the oracle.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "likelihood.cuh"

namespace gpuns {
namespace {

enum NutsPurpose : uint32_t { P_NUTS_MOM = 7, P_NUTS_SLICE = 8, P_NUTS_DIR = 9, P_NUTS_MERGE = 10, P_NUTS_LEAF = 11 };
constexpr double kDeltaMax = 1000.0;

double u01(unsigned long long seed, uint32_t purpose, uint32_t j, uint32_t it, uint32_t chain, uint32_t extra = 0) {
    return philox_uniforms(seed, purpose, j, it, chain, extra).a;
}

// d standard normals by Box-Muller on the pairs (dims 2j, 2j + 1)
void momentum_normals(unsigned long long seed, uint32_t it, uint32_t chain, int d, double* out) {
    for (int j = 0; 2 * j < d; ++j) {
        const Draw2 q = philox_uniforms(seed, P_NUTS_MOM, (uint32_t)j, it, chain, 0);
        const double r = std::sqrt(-2.0 * std::log(q.a));
        const double ang = 6.283185307179586 * q.b;
        out[2 * j] = r * std::cos(ang);
        if (2 * j + 1 < d) out[2 * j + 1] = r * std::sin(ang);
    }
}

double dot(const double* a, const double* b, int d) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) s += a[i] * b[i];
    return s;
}

struct Chain {
    std::vector<double> z, g;       // current sample and gradient of log p
    double lp = 0.0;
    std::vector<double> zm, rm, gm, zp, rp, gp;     // trajectory ends
    std::vector<double> zc, rc, gc;                 // subtree front
    std::vector<double> cz, cg;                     // subtree candidate
    double clp = 0.0;
    std::vector<std::vector<double>> lz, lr;        // left states per level
    std::vector<double> minv;
    double H0 = 0.0, log_u = 0.0, eps = 0.1, a_sum = 0.0;
    long long n = 1, n1 = 0, n_a = 0;
    int j = 0, v = 1;
    bool s = true, s1 = true, cand = false, divergent = false;
    // dual averaging and mass adaptation
    double mu = 0.0, hbar = 0.0, log_eps_bar = 0.0;
    int m_da = 0;
    std::vector<double> wsum, wsq;
    int wn = 0;
};

struct Evaluator {
    const ns_problem* p;
    int d, cap;
    cudaStream_t st;
    std::vector<int> kind;
    std::vector<double> pa, pb;
    double *d_cube = nullptr, *d_theta = nullptr, *d_logL = nullptr, *d_grad = nullptr;
    std::vector<double> h_cube, h_theta, h_logL, h_grad;
    long long calls = 0, evals = 0;

    int init() {
        const size_t n = (size_t)cap * d;
        if (cudaMalloc(&d_cube, n * 8) != cudaSuccess || cudaMalloc(&d_theta, n * 8) != cudaSuccess ||
            cudaMalloc(&d_grad, n * 8) != cudaSuccess || cudaMalloc(&d_logL, (size_t)cap * 8) != cudaSuccess)
            return NS_ENOMEM;
        h_cube.resize(n); h_theta.resize(n); h_grad.resize(n); h_logL.resize(cap);
        for (const ns_prior& q : p->priors) {
            if (q.kind == NS_PRIOR_FIXED) continue;
            kind.push_back(q.kind); pa.push_back(q.a); pb.push_back(q.b);
        }
        return NS_OK;
    }
    ~Evaluator() { cudaFree(d_cube); cudaFree(d_theta); cudaFree(d_logL); cudaFree(d_grad); }

    // rows of z (B x d) -> log p and grad_z log p
    int eval(const std::vector<const double*>& zs, std::vector<double>& lp, std::vector<double*>& grads) {
        const int B = (int)zs.size();
        if (B == 0) return NS_OK;
        for (int b = 0; b < B; ++b)
            for (int i = 0; i < d; ++i) h_cube[(size_t)b * d + i] = 1.0 / (1.0 + std::exp(-zs[b][i]));
        NS_CUDA_TRY(cudaMemcpyAsync(d_cube, h_cube.data(), sizeof(double) * B * d, cudaMemcpyHostToDevice, st));
        NS_TRY(ns_prior_transform(p, d_cube, B, d_theta, st));
        NS_TRY(loglike_grad_batch(p, d_theta, B, d_logL, d_grad, st));
        NS_CUDA_TRY(cudaMemcpyAsync(h_theta.data(), d_theta, sizeof(double) * B * d, cudaMemcpyDeviceToHost, st));
        NS_CUDA_TRY(cudaMemcpyAsync(h_grad.data(), d_grad, sizeof(double) * B * d, cudaMemcpyDeviceToHost, st));
        NS_CUDA_TRY(cudaMemcpyAsync(h_logL.data(), d_logL, sizeof(double) * B, cudaMemcpyDeviceToHost, st));
        NS_CUDA_TRY(cudaStreamSynchronize(st));
        ++calls;
        evals += B;
        for (int b = 0; b < B; ++b) {
            double jac = 0.0;
            for (int i = 0; i < d; ++i) {
                const double c = h_cube[(size_t)b * d + i];
                double dth;
                if (kind[i] == NS_PRIOR_UNIFORM) {
                    dth = pb[i] - pa[i];
                } else {
                    const double x = (h_theta[(size_t)b * d + i] - pa[i]) / pb[i];
                    dth = pb[i] * std::sqrt(2.0 * M_PI) * std::exp(0.5 * x * x);
                }
                grads[b][i] = h_grad[(size_t)b * d + i] * dth * c * (1.0 - c) + (1.0 - 2.0 * c);
                jac += std::log(c) + std::log1p(-c);
            }
            lp[b] = h_logL[b] + jac;
        }
        return NS_OK;
    }
};

}  // namespace
}  // namespace gpuns

using namespace gpuns;

extern "C" int ns_nuts_run(const ns_problem* p, const ns_nuts_config* cfg, const double* z0, double* samples,
                           double* logp_out, double* step_size, ns_nuts_stats* stats, void* stream) {
    if (!p || !cfg || !z0 || !samples || !p->has_lik) return NS_EINVAL;
    const int C = cfg->n_chains, d = p->d, W = cfg->n_warmup, S = cfg->n_samples, maxd = cfg->max_depth;
    if (C < 1 || C > p->max_batch || W < 0 || S < 1 || maxd < 1 || maxd > 20 || !(cfg->init_step > 0) ||
        !(cfg->target_accept > 0 && cfg->target_accept < 1))
        return NS_EINVAL;
    if (p->kind != NS_KIND_SHEAR && p->kind != NS_KIND_GAUSS) return NS_ENOTSUP;
    const unsigned long long seed = cfg->seed;
    Evaluator ev{p, d, C, (cudaStream_t)stream};
    NS_TRY(ev.init());
    std::vector<Chain> ch(C);
    for (int c = 0; c < C; ++c) {
        Chain& k = ch[c];
        k.z.assign(z0 + (size_t)c * d, z0 + (size_t)(c + 1) * d);
        k.g.assign(d, 0.0);
        k.minv.assign(d, 1.0);
        k.eps = cfg->init_step;
        k.mu = std::log(10.0 * cfg->init_step);
        k.lz.assign(maxd + 1, std::vector<double>(d));
        k.lr.assign(maxd + 1, std::vector<double>(d));
        k.wsum.assign(d, 0.0);
        k.wsq.assign(d, 0.0);
    }
    {
        std::vector<const double*> zs(C);
        std::vector<double> lp(C);
        std::vector<double*> gs(C);
        for (int c = 0; c < C; ++c) { zs[c] = ch[c].z.data(); gs[c] = ch[c].g.data(); }
        NS_TRY(ev.eval(zs, lp, gs));
        for (int c = 0; c < C; ++c) ch[c].lp = lp[c];
    }
    const int w_lo = W / 4, w_hi = (3 * W) / 4;
    long long div_after = 0, depth_sum = 0;
    double acc_sum = 0.0;
    std::vector<double> nrm(d);
    std::vector<const double*> zs;
    std::vector<double> lp;
    std::vector<double*> gs;
    std::vector<int> who;
    for (int it = 0; it < W + S; ++it) {
        // momentum, slice and trajectory start
        for (int c = 0; c < C; ++c) {
            Chain& k = ch[c];
            momentum_normals(seed, (uint32_t)it, (uint32_t)c, d, nrm.data());
            k.rm.resize(d);
            double kin = 0.0;
            for (int i = 0; i < d; ++i) {
                k.rm[i] = nrm[i] / std::sqrt(k.minv[i]);
                kin += k.minv[i] * k.rm[i] * k.rm[i];
            }
            k.H0 = k.lp - 0.5 * kin;
            k.log_u = k.H0 + std::log(u01(seed, P_NUTS_SLICE, 0, (uint32_t)it, (uint32_t)c));
            k.zm = k.z; k.gm = k.g;
            k.zp = k.z; k.rp = k.rm; k.gp = k.g;
            k.n = 1; k.s = true; k.j = 0; k.a_sum = 0.0; k.n_a = 0; k.divergent = false;
        }
        std::vector<double> new_lp(C);
        std::vector<std::vector<double>> new_z(C), new_g(C);
        for (int c = 0; c < C; ++c) { new_z[c] = ch[c].z; new_g[c] = ch[c].g; new_lp[c] = ch[c].lp; }
        for (int depth = 0; depth < maxd; ++depth) {
            bool any = false;
            for (int c = 0; c < C; ++c) {
                Chain& k = ch[c];
                if (!k.s) continue;
                any = true;
                k.v = u01(seed, P_NUTS_DIR, (uint32_t)depth, (uint32_t)it, (uint32_t)c) < 0.5 ? -1 : 1;
                if (k.v < 0) { k.zc = k.zm; k.rc = k.rm; k.gc = k.gm; }
                else { k.zc = k.zp; k.rc = k.rp; k.gc = k.gp; }
                k.n1 = 0; k.s1 = true; k.cand = false;
            }
            if (!any) break;
            const long long len = 1LL << depth;
            for (long long i = 0; i < len; ++i) {
                zs.clear(); gs.clear(); who.clear();
                for (int c = 0; c < C; ++c) {
                    Chain& k = ch[c];
                    if (!k.s || !k.s1) continue;
                    const double he = 0.5 * k.v * k.eps;
                    for (int q = 0; q < d; ++q) k.rc[q] += he * k.gc[q];
                    for (int q = 0; q < d; ++q) k.zc[q] += k.v * k.eps * k.minv[q] * k.rc[q];
                    zs.push_back(k.zc.data());
                    gs.push_back(k.gc.data());
                    who.push_back(c);
                }
                if (who.empty()) break;
                lp.assign(who.size(), 0.0);
                NS_TRY(ev.eval(zs, lp, gs));
                for (size_t b = 0; b < who.size(); ++b) {
                    const int c = who[b];
                    Chain& k = ch[c];
                    const double he = 0.5 * k.v * k.eps;
                    for (int q = 0; q < d; ++q) k.rc[q] += he * k.gc[q];
                    double kin = 0.0;
                    for (int q = 0; q < d; ++q) kin += k.minv[q] * k.rc[q] * k.rc[q];
                    double H = lp[b] - 0.5 * kin;
                    if (!std::isfinite(H)) H = -INFINITY;
                    k.a_sum += (H > -INFINITY) ? std::min(1.0, std::exp(std::min(0.0, H - k.H0))) : 0.0;
                    k.n_a += 1;
                    if (k.log_u - H > kDeltaMax) { k.s1 = false; k.divergent = true; continue; }
                    if (k.log_u <= H) {
                        k.n1 += 1;
                        if (u01(seed, P_NUTS_LEAF, (uint32_t)depth, (uint32_t)it, (uint32_t)c, (uint32_t)i) *
                                (double)k.n1 < 1.0) {
                            k.cz = k.zc; k.cg = k.gc; k.clp = lp[b]; k.cand = true;
                        }
                    }
                    for (int lev = 1; lev <= depth; ++lev)
                        if (i % (1LL << lev) == 0) { k.lz[lev] = k.zc; k.lr[lev] = k.rc; }
                    for (int lev = 1; lev <= depth; ++lev) {
                        if ((i + 1) % (1LL << lev) != 0) continue;
                        double a = 0.0, e = 0.0;
                        for (int q = 0; q < d; ++q) {
                            const double dz = k.v * (k.zc[q] - k.lz[lev][q]);
                            a += dz * k.lr[lev][q];
                            e += dz * k.rc[q];
                        }
                        if (a < 0.0 || e < 0.0) { k.s1 = false; break; }
                    }
                }
            }
            for (int c = 0; c < C; ++c) {
                Chain& k = ch[c];
                if (!k.s) continue;
                if (k.v < 0) { k.zm = k.zc; k.rm = k.rc; k.gm = k.gc; }
                else { k.zp = k.zc; k.rp = k.rc; k.gp = k.gc; }
                if (k.s1 && k.n1 > 0 && k.cand &&
                    u01(seed, P_NUTS_MERGE, (uint32_t)depth, (uint32_t)it, (uint32_t)c) * (double)k.n < (double)k.n1) {
                    new_z[c] = k.cz; new_g[c] = k.cg; new_lp[c] = k.clp;
                }
                k.n += k.n1;
                std::vector<double> dz(d);
                for (int q = 0; q < d; ++q) dz[q] = k.zp[q] - k.zm[q];
                k.s = k.s1 && dot(dz.data(), k.rm.data(), d) >= 0.0 && dot(dz.data(), k.rp.data(), d) >= 0.0;
                k.j = depth + 1;
            }
        }
        for (int c = 0; c < C; ++c) {
            Chain& k = ch[c];
            k.z = new_z[c]; k.g = new_g[c]; k.lp = new_lp[c];
            const double acc = k.a_sum / (double)std::max<long long>(k.n_a, 1);
            if (it < W) {
                k.m_da += 1;
                const double eta = 1.0 / (k.m_da + 10.0);
                k.hbar = (1.0 - eta) * k.hbar + eta * (cfg->target_accept - acc);
                const double log_eps = k.mu - std::sqrt((double)k.m_da) / 0.05 * k.hbar;
                const double wgt = std::pow((double)k.m_da, -0.75);
                k.log_eps_bar = wgt * log_eps + (1.0 - wgt) * k.log_eps_bar;
                k.eps = std::exp(log_eps);
                if (cfg->adapt_mass && it >= w_lo && it < w_hi) {
                    // running mean / M2 (Welford) of z over the window
                    k.wn += 1;
                    for (int q = 0; q < d; ++q) {
                        const double dlt = k.z[q] - k.wsum[q];
                        k.wsum[q] += dlt / k.wn;
                        k.wsq[q] += dlt * (k.z[q] - k.wsum[q]);
                    }
                }
                if (cfg->adapt_mass && it == w_hi - 1 && k.wn > 1) {
                    const double nw = (double)k.wn;
                    for (int q = 0; q < d; ++q) {
                        const double var = k.wsq[q] / (nw - 1.0);
                        k.minv[q] = (nw / (nw + 5.0)) * var + 1e-3 * (5.0 / (nw + 5.0));
                    }
                    k.mu = std::log(10.0 * k.eps);
                    k.hbar = 0.0; k.log_eps_bar = 0.0; k.m_da = 0;
                }
                if (it == W - 1) k.eps = std::exp(k.log_eps_bar);
            } else {
                const long long row = (long long)c * S + (it - W);
                std::memcpy(samples + row * d, k.z.data(), sizeof(double) * d);
                if (logp_out) logp_out[row] = k.lp;
                div_after += k.divergent ? 1 : 0;
                depth_sum += k.j;
                acc_sum += acc;
            }
        }
    }
    if (step_size)
        for (int c = 0; c < C; ++c) step_size[c] = ch[c].eps;
    if (stats) {
        stats->gradient_evals = ev.evals;
        stats->batched_calls = ev.calls;
        stats->divergences = (int)div_after;
        stats->mean_depth = (double)depth_sum / ((double)C * S);
        stats->mean_accept = acc_sum / ((double)C * S);
    }
    return NS_OK;
}
