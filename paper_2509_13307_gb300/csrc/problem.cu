// Problem construction and the batched-likelihood entry points of the C ABI.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "likelihood.cuh"

static thread_local char g_last_err[512] = {0};

void ns_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    snprintf(g_last_err, sizeof(g_last_err), "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
}

extern "C" const char* ns_strerror(int code) {
    switch (code) {
        case NS_OK: return "ok";
        case NS_EINVAL: return "invalid argument";
        case NS_ECUDA: return g_last_err[0] ? g_last_err : "CUDA error";
        case NS_ENOMEM: return "out of memory";
        case NS_ETIMEOUT: return "device wait timed out";
        case NS_ESLICE: return "slice step cap reached";
        case NS_ENONFINITE: return "non-finite log-likelihood";
        case NS_ENOTSUP: return "not supported";
        default: return "unknown status";
    }
}

namespace gpuns {

template <typename T>
static int upload(const T* host, size_t n, T** dev, std::vector<void*>& owned) {
    *dev = nullptr;
    if (n == 0) return NS_OK;
    if (cudaMalloc((void**)dev, n * sizeof(T)) != cudaSuccess) return NS_ENOMEM;
    owned.push_back(*dev);
    NS_CUDA_TRY(cudaMemcpy(*dev, host, n * sizeof(T), cudaMemcpyHostToDevice));
    return NS_OK;
}

static int dalloc(size_t bytes, void** dev, std::vector<void*>& owned) {
    *dev = nullptr;
    if (bytes == 0) return NS_OK;
    if (cudaMalloc(dev, bytes) != cudaSuccess) return NS_ENOMEM;
    owned.push_back(*dev);
    return NS_OK;
}

static uint16_t f32_to_bf16_rne(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);   // inf / nan
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

// Catmull-Rom taps of coordinate s on a uniform grid [lo, lo + (n-1) step], ghosts folded.
static void cr_taps(double s, double lo, double step, int n, int idx[4], double w[4]) {
    const double u = (s - lo) / step;
    int i = (int)std::floor(u);
    if (i < 0) i = 0;
    if (i > n - 2) i = n - 2;
    double wi[4];
    catmull_rom<double>(u - i, wi);
    fold_taps<double>(i, n, wi, idx, w);
}

// Host FP64 Cholesky C = L L^T (lower, row-major) and L^-1; false if not SPD.
static bool cholesky_inverse(const double* C, int D, std::vector<double>& L, std::vector<double>& Linv) {
    L.assign((size_t)D * D, 0.0);
    for (int j = 0; j < D; ++j) {
        double s = C[(size_t)j * D + j];
        for (int k = 0; k < j; ++k) s -= L[(size_t)j * D + k] * L[(size_t)j * D + k];
        if (!(s > 0.0)) return false;
        const double ljj = std::sqrt(s);
        L[(size_t)j * D + j] = ljj;
        for (int i = j + 1; i < D; ++i) {
            double t = C[(size_t)i * D + j];
            for (int k = 0; k < j; ++k) t -= L[(size_t)i * D + k] * L[(size_t)j * D + k];
            L[(size_t)i * D + j] = t / ljj;
        }
    }
    Linv.assign((size_t)D * D, 0.0);
    for (int c = 0; c < D; ++c) {          // solve L x = e_c
        for (int i = c; i < D; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = c; k < i; ++k) s -= L[(size_t)i * D + k] * Linv[(size_t)k * D + c];
            Linv[(size_t)i * D + c] = s / L[(size_t)i * D + i];
        }
    }
    return true;
}

int workspace_create(const ns_problem* p, int cap, Workspace* ws) {
    ws->cap = cap;
    void* v;
    NS_TRY(dalloc(sizeof(int), &v, ws->owned));
    ws->d_nrows = (int*)v;
    NS_TRY(dalloc(sizeof(int), &v, ws->owned));
    ws->d_err = (int*)v;
    NS_CUDA_TRY(cudaMemset(ws->d_err, 0, sizeof(int)));
    if (cudaMallocHost(&ws->h_err, sizeof(int)) != cudaSuccess) return NS_ENOMEM;
    *ws->h_err = 0;
    NS_TRY(dalloc(sizeof(double) * (size_t)cap * p->P, &v, ws->owned));
    ws->theta_full = (double*)v;
    NS_TRY(dalloc(sizeof(double) * (size_t)cap, &v, ws->owned));
    ws->logL = (double*)v;
    if (p->kind == NS_KIND_GAUSS) return NS_OK;
    const int elt = (p->precision == NS_PREC_FP64) ? 8 : (p->precision == NS_PREC_FP32 ? 4 : 2);
    if (p->kind == NS_KIND_CMB) {
        const int tab_elt = (p->precision == NS_PREC_FP64) ? 8 : 4;
        const int rows_pad = ((cap + 127) / 128) * 128;
        for (int i = 0; i < 2; ++i) {
            NS_TRY(dalloc((size_t)elt * rows_pad * p->hidden_max, &v, ws->owned));
            ws->act[i] = v;
            NS_CUDA_TRY(cudaMemset(v, 0, (size_t)elt * rows_pad * p->hidden_max));
        }
        NS_TRY(dalloc((size_t)tab_elt * cap * std::max(p->D, p->dims.back()), &v, ws->owned));
        ws->table = v;
        if (p->cmb_solve == NS_SOLVE_LITERAL && p->cmb_form == NS_CMB_GAUSS) {
            NS_TRY(dalloc(sizeof(double) * (size_t)cap * p->D, &v, ws->owned));
            ws->resid = v;
        }
        if (p->precision == NS_PREC_BF16) {
            ws->tmA.resize(p->n_layers);
            int cur = 0;
            for (int l = 1; l + 1 < p->n_layers; ++l) {
                NS_TRY(make_tensor_map_bf16(&ws->tmA[l], ws->act[cur], rows_pad, p->dims[l], 128,
                                            gemm_tc_kps(p->dims[l])));
                cur ^= 1;
            }
        }
        return NS_OK;
    }
    const int tab_elt = (p->precision == NS_PREC_FP64) ? 8 : 4;
    const int rows_pad = ((cap + 127) / 128) * 128;
    for (int i = 0; i < 2; ++i) {
        NS_TRY(dalloc((size_t)elt * rows_pad * p->hidden_max, &v, ws->owned));
        ws->act[i] = v;
        NS_CUDA_TRY(cudaMemset(v, 0, (size_t)elt * rows_pad * p->hidden_max));
    }
    const int n_out = p->dims.back();
    NS_TRY(dalloc((size_t)tab_elt * cap * n_out, &v, ws->owned));
    ws->table = v;
    if (p->n_z_emu != p->sp.n_z) {
        NS_TRY(dalloc((size_t)tab_elt * cap * p->sp.n_z * p->sp.n_k, &v, ws->owned));
        ws->table_fine = v;
    }
    NS_TRY(dalloc((size_t)tab_elt * cap * p->sp.D, &v, ws->owned));
    ws->resid = v;
    NS_TRY(dalloc((size_t)tab_elt * cap * (p->sp.nb + 1) * ((p->sp.N + 3) & ~3), &v, ws->owned));
    ws->win = v;
    NS_CUDA_TRY(cudaStreamCreateWithFlags(&ws->side, cudaStreamNonBlocking));
    NS_CUDA_TRY(cudaEventCreateWithFlags(&ws->ev_fork, cudaEventDisableTiming));
    NS_CUDA_TRY(cudaEventCreateWithFlags(&ws->ev_join, cudaEventDisableTiming));

    if (p->precision == NS_PREC_BF16 || p->precision == NS_PREC_BF16_F64CHI2) {
        ws->tmA.resize(p->n_layers);
        int cur = 0;
        for (int l = 1; l < p->n_layers; ++l) {
            NS_TRY(make_tensor_map_bf16(&ws->tmA[l], ws->act[cur], rows_pad, p->dims[l], 128,
                                        gemm_tc_kps(p->dims[l])));
            if (l == p->n_layers - 1)
                NS_TRY(make_tensor_map_bf16(&ws->tmX_out, ws->act[cur], rows_pad, p->dims[l], kSwapRows));
            if (p->fused_cs && l == p->n_layers - 2)
                NS_TRY(make_tensor_map_bf16(&ws->tmF_out, ws->act[cur ^ 1], rows_pad, p->dims[l + 1], 64, 2));
            cur ^= 1;
        }
    }
    return NS_OK;
}

int workspace_err_fetch(Workspace* ws, cudaStream_t st) {
    NS_CUDA_TRY(cudaMemcpyAsync(ws->h_err, ws->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    return NS_OK;
}

void workspace_free(Workspace* ws) {
    for (void* q : ws->owned) cudaFree(q);
    ws->owned.clear();
    if (ws->h_err) cudaFreeHost(ws->h_err);
    ws->h_err = nullptr;
    if (ws->ev_fork) cudaEventDestroy(ws->ev_fork);
    if (ws->ev_join) cudaEventDestroy(ws->ev_join);
    if (ws->side) cudaStreamDestroy(ws->side);
    ws->ev_fork = ws->ev_join = nullptr;
    ws->side = nullptr;
}

// Upload a host FP64 vector in the problem's compute dtype (FP64, else FP32).
static int upload_compute(const ns_problem* p, const double* h, size_t n, void** out, std::vector<void*>& owned) {
    if (p->precision == NS_PREC_FP64) {
        double* v;
        NS_TRY(upload(h, n, &v, owned));
        *out = v;
    } else {
        std::vector<float> f(h, h + n);
        float* v;
        NS_TRY(upload(f.data(), n, &v, owned));
        *out = v;
    }
    return NS_OK;
}

// CMB set-up: FP64 factorisation of the covariance (host for D <= 256, else
// blocked kernels on the device), the constant c0, and either L^-T for the
// literal per-evaluation whitening or the fold of the linear head:
// W' = L^-1 diag(sigma) W_out, c' = L^-1 (d - mu - sigma b_out).
static int cmb_setup(ns_problem* p, const ns_problem_desc* desc) {
    p->cmb_solve = desc->cmb.solve;
    p->cmb_form = desc->cmb.form;
    if (!p->has_lik) return NS_OK;
    if (p->cmb_form == NS_CMB_TT_CV) {
        // log L = c0 - sum_ell (k/2) g(C / d),  g(r) = ln r + 1/r - 1, with
        // c0 = sum_ell [(k/2 - 1) ln(k d) - (k/2) ln 2 - ln Gamma(k/2) + ln k - (k/2)(ln d + 1)]
        const int n = desc->cmb.n_tt;
        p->n_tt = n;
        std::vector<double> hk(n);
        double c0 = 0.0;
        for (int i = 0; i < n; ++i) {
            const double k = 2.0 * desc->cmb.ell[i] + 1.0, d = desc->data[i];
            hk[i] = 0.5 * k;
            c0 += (0.5 * k - 1.0) * std::log(k * d) - 0.5 * k * std::log(2.0) - std::lgamma(0.5 * k) + std::log(k) -
                  0.5 * k * (std::log(d) + 1.0);
        }
        p->c0 = c0;
        NS_TRY(upload_compute(p, desc->data, n, &p->d_tt_obs, p->owned));
        NS_TRY(upload_compute(p, hk.data(), n, &p->d_tt_halfk, p->owned));
        return NS_OK;
    }
    const ns_emulator_desc& e = desc->emu;
    const int L = e.n_layers, D = p->D, H = e.dims[L - 1];
    const double* Wout = e.W[L - 1];
    const double* bout = e.b[L - 1];
    std::vector<double> sig(D), v(D);
    for (int a = 0; a < D; ++a) {
        sig[a] = e.out_sigma_vec ? e.out_sigma_vec[a] : e.out_sigma;
        v[a] = desc->data[a] - e.out_mu[a] - sig[a] * bout[a];
    }
    const bool literal = p->cmb_solve == NS_SOLVE_LITERAL;
    if (literal) {
        std::vector<double> lm(D), ls(D);
        for (int a = 0; a < D; ++a) { lm[a] = desc->data[a] - e.out_mu[a]; ls[a] = -sig[a]; }
        NS_TRY(upload(lm.data(), D, &p->d_lit_mu, p->owned));
        NS_TRY(upload(ls.data(), D, &p->d_lit_sig, p->owned));
    }
    std::vector<double> zeros(std::max(D, H), 0.0);
    NS_TRY(upload_compute(p, zeros.data(), D, &p->d_zeroD, p->owned));
    std::vector<double> Wf((size_t)D * H), cf(D);
    if (D <= 256) {
        std::vector<double> Lh, Linv;
        if (!cholesky_inverse(desc->cov, D, Lh, Linv)) return NS_EINVAL;
        double c0 = -0.5 * D * std::log(2.0 * M_PI);
        for (int a = 0; a < D; ++a) c0 -= std::log(Lh[(size_t)a * D + a]);
        p->c0 = c0;
        if (literal) {
            std::vector<double> LT((size_t)D * D);
            for (int a = 0; a < D; ++a)
                for (int b = 0; b < D; ++b) LT[(size_t)b * D + a] = Linv[(size_t)a * D + b];
            return upload(LT.data(), LT.size(), &p->d_LinvT64, p->owned);
        }
        for (int a = 0; a < D; ++a) {
            double c = 0.0;
            for (int b = 0; b <= a; ++b) c += Linv[(size_t)a * D + b] * v[b];
            cf[a] = c;
            for (int h = 0; h < H; ++h) {
                double w = 0.0;
                for (int b = 0; b <= a; ++b) w += Linv[(size_t)a * D + b] * sig[b] * Wout[(size_t)b * H + h];
                Wf[(size_t)a * H + h] = w;
            }
        }
    } else {
        cudaStream_t st = nullptr;
        double* dC = nullptr;
        double* X = nullptr;
        std::vector<void*> tmp;
        auto done = [&](int code) {
            for (void* q : tmp) cudaFree(q);
            cudaFree(dC);
            cudaFree(X);
            return code;
        };
        if (upload(desc->cov, (size_t)D * D, &dC, tmp)) return done(NS_ENOMEM);
        tmp.clear();
        double sum_log = 0.0;
        int s = device_cholesky_inverse(dC, D, &X, &sum_log, st);
        if (s) return done(s);
        p->c0 = -0.5 * D * std::log(2.0 * M_PI) - sum_log;
        if (literal) {
            double* LT = nullptr;
            if (cudaMalloc(&LT, sizeof(double) * (size_t)D * D) != cudaSuccess) return done(NS_ENOMEM);
            p->owned.push_back(LT);
            if ((s = device_transpose(X, LT, D, st))) return done(s);
            if (cudaStreamSynchronize(st) != cudaSuccess) return done(NS_ECUDA);
            p->d_LinvT64 = LT;
            return done(NS_OK);
        }
        // W' = X (sigma W_out) and c' = X v as FP64 GEMMs on the device
        std::vector<double> Wt((size_t)H * D);
        for (int b = 0; b < D; ++b)
            for (int h = 0; h < H; ++h) Wt[(size_t)h * D + b] = sig[b] * Wout[(size_t)b * H + h];
        double *dWt, *dv, *dz, *dWf, *dcf;
        int* dn;
        if (upload(Wt.data(), Wt.size(), &dWt, tmp) || upload(v.data(), D, &dv, tmp) ||
            upload(zeros.data(), zeros.size(), &dz, tmp) || upload(&D, 1, &dn, tmp))
            return done(NS_ENOMEM);
        if (cudaMalloc(&dWf, sizeof(double) * (size_t)D * H) != cudaSuccess) return done(NS_ENOMEM);
        tmp.push_back(dWf);
        if (cudaMalloc(&dcf, sizeof(double) * (size_t)D) != cudaSuccess) return done(NS_ENOMEM);
        tmp.push_back(dcf);
        if ((s = gemm_f64_plain(X, dWt, dWf, dn, D, H, D, dz, st))) return done(s);
        if ((s = gemm_f64_plain(X, dv, dcf, dn, D, 1, D, dz, st))) return done(s);
        if (cudaMemcpyAsync(Wf.data(), dWf, sizeof(double) * Wf.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(cf.data(), dcf, sizeof(double) * D, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return done(NS_ECUDA);
        done(NS_OK);
    }
    NS_TRY(upload_compute(p, Wf.data(), Wf.size(), &p->d_Wfold, p->owned));
    NS_TRY(upload_compute(p, cf.data(), cf.size(), &p->d_cfold, p->owned));
    return NS_OK;
}

// Tile autotuner for the tensor-core hidden layers: each candidate N-tile
// width (16, 32, 64, 128) runs the layer on max_batch rows (at most 384, about the
// average batch of a nested-sampling likelihood round with k = 500) of the
// workspace-sized activations, timed with CUDA events over 5 launches after a
// warm-up; a wider tile replaces a narrower one only when it is at least 3%
// faster, since in the nested-sampling rounds narrow tiles leave shared
// memory for the other chain group's kernels.  Every width gives bit-identical
// results (the accumulation order per element does not depend on it).
static int autotune_hidden_tiles(ns_problem* p, int last_hidden) {
    if (last_hidden < 1) return NS_OK;
    const int rows = std::min(p->max_batch, 384);
    const int rows_pad = ((rows + 127) / 128) * 128;
    int kmax = 0, nmax = 0;
    for (int l = 1; l <= last_hidden; ++l) { kmax = std::max(kmax, p->dims[l]); nmax = std::max(nmax, p->dims[l + 1]); }
    void *a = nullptr, *o = nullptr;
    int* dn = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto done = [&](int code) {
        cudaFree(a); cudaFree(o); cudaFree(dn);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
        return code;
    };
    if (cudaMalloc(&a, (size_t)2 * rows_pad * kmax) != cudaSuccess ||
        cudaMalloc(&o, (size_t)2 * rows_pad * nmax) != cudaSuccess || cudaMalloc(&dn, sizeof(int)) != cudaSuccess)
        return done(NS_ENOMEM);
    if (cudaMemset(a, 0, (size_t)2 * rows_pad * kmax) != cudaSuccess ||
        cudaMemcpy(dn, &rows, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return done(NS_ECUDA);
    p->tile_ms.assign(p->n_layers, 0.0f);
    for (int l = 1; l <= last_hidden; ++l) {
        const int K = p->dims[l], N = p->dims[l + 1];
        CUtensorMap tmA, tmB;
        int s = make_tensor_map_bf16(&tmA, a, rows_pad, K, 128, gemm_tc_kps(K));
        if (s) return done(s);
        int best = p->tile_n[l];
        float best_ms = 1e30f;
        for (int tn : {16, 32, 64, 128}) {
            if (tn > N) continue;
            if ((s = make_tensor_map_bf16(&tmB, p->d_W[l], N, K, tn, gemm_tc_kps(K)))) return done(s);
            auto run = [&]() {
                return launch_gemm_tc(&tmA, &tmB, tn, (const float*)p->d_b[l], nullptr, 0.f, o, dn, rows, N, K,
                                      TC_EPI_TANH, nullptr, nullptr, st);
            };
            if ((s = run())) return done(s);
            if (cudaEventRecord(e0, st) != cudaSuccess) return done(NS_ECUDA);
            for (int i = 0; i < 5; ++i)
                if ((s = run())) return done(s);
            float ms = 0.f;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                return done(NS_ECUDA);
            if (ms < 0.97f * best_ms) { best = tn; best_ms = ms; }
        }
        p->tile_n[l] = best;
        p->tile_ms[l] = best_ms / 5.f;
        if ((s = make_tensor_map_bf16(&p->tmB[l], p->d_W[l], N, K, best, gemm_tc_kps(K)))) return done(s);
    }
    return done(NS_OK);
}

static int validate_desc(const ns_problem_desc* d) {
    if (!d || !d->priors || d->n_params < 1 || d->n_params > 256 || d->max_batch < 1) return NS_EINVAL;
    if (d->precision < 0 || d->precision > NS_PREC_BF16_F64CHI2) return NS_EINVAL;
    if (d->hidden_tile != 0 && d->hidden_tile != -1 && d->hidden_tile != 16 && d->hidden_tile != 32 &&
        d->hidden_tile != 64 && d->hidden_tile != 128)
        return NS_EINVAL;
    int nfree = 0;
    for (int i = 0; i < d->n_params; ++i) {
        const ns_prior& q = d->priors[i];
        if (q.kind == NS_PRIOR_FIXED) continue;
        if (q.kind == NS_PRIOR_UNIFORM && !(q.b > q.a)) return NS_EINVAL;
        if (q.kind == NS_PRIOR_GAUSS && !(q.b > 0)) return NS_EINVAL;
        if (q.kind != NS_PRIOR_UNIFORM && q.kind != NS_PRIOR_GAUSS) return NS_EINVAL;
        ++nfree;
    }
    if (nfree < 1 || nfree > 64) return NS_EINVAL;
    if (d->kind == NS_KIND_GAUSS) return (d->gauss.sigma > 0) ? NS_OK : NS_EINVAL;
    if (d->kind != NS_KIND_SHEAR && d->kind != NS_KIND_CMB) return NS_EINVAL;
    const ns_emulator_desc& e = d->emu;
    if (e.n_layers < 2 || !e.dims || !e.W || !e.b || !e.inputs || !e.in_center || !e.in_scale || !e.out_mu)
        return NS_EINVAL;
    if (e.activation != NS_ACT_TANH && e.activation != NS_ACT_SIGMOID_LINEAR) return NS_EINVAL;
    if (e.activation == NS_ACT_SIGMOID_LINEAR && (!e.act_g || !e.act_beta)) return NS_EINVAL;
    const bool tt = d->kind == NS_KIND_CMB && d->cmb.form == NS_CMB_TT_CV;
    if (!tt && (d->data == nullptr) != (d->cov == nullptr)) return NS_EINVAL;
    if (d->kind == NS_KIND_CMB) {
        if (e.dims[0] < 1 || e.dims[0] > 32) return NS_EINVAL;
        if (d->cmb.form != NS_CMB_GAUSS && d->cmb.form != NS_CMB_TT_CV) return NS_EINVAL;
        if (tt) {
            if (d->cmb.n_tt < 1 || d->cmb.n_tt > e.dims[e.n_layers] || !d->cmb.ell || d->cov) return NS_EINVAL;
            if (d->data && d->n_data != d->cmb.n_tt) return NS_EINVAL;
            for (int i = 0; i < d->cmb.n_tt; ++i)
                if (!(d->cmb.ell[i] >= 0) || (d->data && !(d->data[i] > 0))) return NS_EINVAL;
        } else if (d->n_data != e.dims[e.n_layers] || d->n_data < 1) {
            return NS_EINVAL;
        }
        for (int j = 0; j < e.dims[0]; ++j)
            if (e.inputs[j] < 0 || e.inputs[j] >= d->n_params || !(e.in_scale[j] != 0)) return NS_EINVAL;
        if (d->cmb.solve != NS_SOLVE_FOLD && d->cmb.solve != NS_SOLVE_LITERAL) return NS_EINVAL;
        if (d->cmb.solve == NS_SOLVE_LITERAL && d->precision != NS_PREC_FP64) return NS_ENOTSUP;
        if (d->precision == NS_PREC_BF16_F64CHI2) return NS_ENOTSUP;
        return NS_OK;
    }
    const ns_shear_desc& s = d->shear;
    if (s.n_bins < 1 || s.n_bins > 5 || s.n_ell < 1 || s.n_k < 4 || s.n_z < 4 || s.n_chi < 3 || !(s.a_min > 0 && s.a_min < 1))
        return NS_EINVAL;
    if (s.n_z_emu < 4 || s.n_z_emu > s.n_z) return NS_EINVAL;
    if (s.z_interp != 0 && s.z_interp != 1) return NS_EINVAL;
    if (d->n_params != 11 + 2 * s.n_bins + s.n_tmpl) return NS_EINVAL;
    const int D = s.n_bins * (s.n_bins + 1) / 2 * s.n_ell;
    if (d->n_data != D) return NS_EINVAL;
    if (s.n_tmpl > 0 && !s.tmpl) return NS_EINVAL;
    if (e.dims[0] < 1 || e.dims[0] > 32) return NS_EINVAL;
    if (e.dims[e.n_layers] != s.n_k * s.n_z_emu) return NS_EINVAL;
    for (int j = 0; j < e.dims[0]; ++j)
        if (e.inputs[j] < 0 || e.inputs[j] >= d->n_params || !(e.in_scale[j] != 0)) return NS_EINVAL;
    return NS_OK;
}

}  // namespace gpuns

using namespace gpuns;

void gpuns_release_grad_state(const ns_problem* p);

static void problem_release(ns_problem* p) {
    if (!p) return;
    gpuns_release_grad_state(p);
    workspace_free(&p->ws);
    for (void* q : p->owned) cudaFree(q);
    delete p;
}

extern "C" int ns_problem_create(const ns_problem_desc* desc, ns_problem** out) {
    if (!out) return NS_EINVAL;
    *out = nullptr;
    NS_TRY(validate_desc(desc));
    ns_problem* p = new (std::nothrow) ns_problem();
    if (!p) return NS_ENOMEM;
    auto fail = [&](int code) { problem_release(p); return code; };
    p->kind = desc->kind;
    p->precision = desc->precision;
    p->P = desc->n_params;
    p->max_batch = desc->max_batch;
    p->priors.assign(desc->priors, desc->priors + desc->n_params);
    {
        std::vector<int> kind(p->P), fof(p->P);
        std::vector<double> pa(p->P), pb(p->P);
        int f = 0;
        for (int i = 0; i < p->P; ++i) {
            kind[i] = p->priors[i].kind;
            pa[i] = p->priors[i].a;
            pb[i] = p->priors[i].b;
            fof[i] = (kind[i] == NS_PRIOR_FIXED) ? -1 : f++;
        }
        p->d = f;
        int s;
        if ((s = upload(kind.data(), kind.size(), &p->d_pkind, p->owned))) return fail(s);
        if ((s = upload(pa.data(), pa.size(), &p->d_pa, p->owned))) return fail(s);
        if ((s = upload(pb.data(), pb.size(), &p->d_pb, p->owned))) return fail(s);
        if ((s = upload(fof.data(), fof.size(), &p->d_free_of_full, p->owned))) return fail(s);
    }
    if (p->kind == NS_KIND_GAUSS) {
        p->g_mu = desc->gauss.mu;
        p->g_sigma = desc->gauss.sigma;
        int s = workspace_create(p, p->max_batch, &p->ws);
        if (s) return fail(s);
        *out = p;
        return NS_OK;
    }

    // ---------------- emulator
    const ns_emulator_desc& e = desc->emu;
    const bool bf16 = (p->precision == NS_PREC_BF16 || p->precision == NS_PREC_BF16_F64CHI2);
    const bool f64 = (p->precision == NS_PREC_FP64);
    p->n_layers = e.n_layers;
    p->dims.assign(e.dims, e.dims + e.n_layers + 1);
    p->hidden_max = 0;
    for (int l = 1; l < e.n_layers; ++l) p->hidden_max = std::max(p->hidden_max, p->dims[l]);
    const bool cmb = p->kind == NS_KIND_CMB;
    // BF16 layers on tensor cores: every layer >= 1 for shear; the hidden
    // layers only for CMB (its head runs on CUDA cores in FP32)
    auto tc_layer = [&](int l) { return bf16 && l >= 1 && !(cmb && l == e.n_layers - 1); };
    if (bf16) {
        for (int l = 1; l < e.n_layers; ++l)
            if (tc_layer(l) && !gemm_tc_supported(p->dims[l + 1], p->dims[l]) &&
                !(l == e.n_layers - 1 && p->dims[l + 1] % 4 == 0 && p->dims[l] % 8 == 0))
                return fail(NS_ENOTSUP);
    }
    p->d_W.assign(e.n_layers, nullptr);
    p->d_b.assign(e.n_layers, nullptr);
    for (int l = 0; l < e.n_layers; ++l) {
        const size_t nw = (size_t)p->dims[l + 1] * p->dims[l];
        const size_t nb = p->dims[l + 1];
        int s;
        if (f64) {
            double* w; double* b;
            if ((s = upload(e.W[l], nw, &w, p->owned))) return fail(s);
            if ((s = upload(e.b[l], nb, &b, p->owned))) return fail(s);
            p->d_W[l] = w; p->d_b[l] = b;
        } else {
            std::vector<float> bf(nb);
            for (size_t i = 0; i < nb; ++i) bf[i] = (float)e.b[l][i];
            float* b;
            if ((s = upload(bf.data(), nb, &b, p->owned))) return fail(s);
            p->d_b[l] = b;
            if (tc_layer(l)) {
                std::vector<uint16_t> wb(nw);
                for (size_t i = 0; i < nw; ++i) wb[i] = f32_to_bf16_rne((float)e.W[l][i]);
                uint16_t* w;
                if ((s = upload(wb.data(), nw, &w, p->owned))) return fail(s);
                p->d_W[l] = w;
            } else {
                std::vector<float> wf(nw);
                for (size_t i = 0; i < nw; ++i) wf[i] = (float)e.W[l][i];
                float* w;
                if ((s = upload(wf.data(), nw, &w, p->owned))) return fail(s);
                p->d_W[l] = w;
            }
        }
    }
    {
        int s;
        if ((s = upload(e.inputs, (size_t)p->dims[0], &p->d_inputs, p->owned))) return fail(s);
        if ((s = upload(e.in_center, (size_t)p->dims[0], &p->d_in_center, p->owned))) return fail(s);
        if ((s = upload(e.in_scale, (size_t)p->dims[0], &p->d_in_scale, p->owned))) return fail(s);
        std::vector<double> inv(p->dims[0]);
        for (int j = 0; j < p->dims[0]; ++j) inv[j] = 1.0 / e.in_scale[j];
        if ((s = upload(inv.data(), inv.size(), &p->d_in_inv_scale, p->owned))) return fail(s);
        const size_t no = p->dims.back();
        if (f64) {
            double* m;
            if ((s = upload(e.out_mu, no, &m, p->owned))) return fail(s);
            p->d_out_mu = m;
        } else {
            std::vector<float> mf(no);
            for (size_t i = 0; i < no; ++i) mf[i] = (float)e.out_mu[i];
            float* m;
            if ((s = upload(mf.data(), no, &m, p->owned))) return fail(s);
            p->d_out_mu = m;
        }
        p->out_sigma = e.out_sigma;
        if (e.out_sigma_vec) {
            if (f64) {
                double* v;
                if ((s = upload(e.out_sigma_vec, no, &v, p->owned))) return fail(s);
                p->d_out_sig = v;
            } else {
                std::vector<float> vf(no);
                for (size_t i = 0; i < no; ++i) vf[i] = (float)e.out_sigma_vec[i];
                float* v;
                if ((s = upload(vf.data(), no, &v, p->owned))) return fail(s);
                p->d_out_sig = v;
            }
        }
        p->act = e.activation;
        if (p->act == NS_ACT_SIGMOID_LINEAR) {
            p->d_act_g.assign(e.n_layers - 1, nullptr);
            p->d_act_beta.assign(e.n_layers - 1, nullptr);
            for (int l = 0; l + 1 < e.n_layers; ++l) {
                const size_t n = p->dims[l + 1];
                for (int w = 0; w < 2; ++w) {
                    const double* src = w ? e.act_beta[l] : e.act_g[l];
                    void* dst = nullptr;
                    if (f64) {
                        double* v;
                        if ((s = upload(src, n, &v, p->owned))) return fail(s);
                        dst = v;
                    } else {
                        std::vector<float> vf(src, src + n);
                        float* v;
                        if ((s = upload(vf.data(), n, &v, p->owned))) return fail(s);
                        dst = v;
                    }
                    (w ? p->d_act_beta[l] : p->d_act_g[l]) = dst;
                }
            }
        }
    }
    if (bf16) {
        p->tmB.resize(e.n_layers);
        p->tile_n.assign(e.n_layers, 128);
        for (int l = 1; l < e.n_layers; ++l) {
            if (!tc_layer(l)) continue;
            const int N = p->dims[l + 1];
            const bool last = (l == e.n_layers - 1);
            // hidden layers have few M tiles (rows = active chains): narrow N
            // tiles give more CTAs; the output layer is wide enough for 128
            int tn = last ? 128 : 32;
            if (N < tn) tn = (N >= 64) ? 64 : 32;
            p->tile_n[l] = tn;
            // the swapped output layer (tile 128) reads W through 2-D boxes
            const int kps = (last && tn == 128) ? 1 : gemm_tc_kps(p->dims[l]);
            int s = make_tensor_map_bf16(&p->tmB[l], p->d_W[l], N, p->dims[l], tn, kps);
            if (s) return fail(s);
        }
        int s = NS_OK;
        // the fused input + hidden stack (on request, hidden_tile = -1): tanh
        // shear emulators whose hidden widths all equal 128 CS (CS = 4 or 8),
        // at most kFusedMaxHidden hidden layers, at most 32 inputs
        const int n_h = e.n_layers - 2;
        bool fuse = !cmb && desc->hidden_tile == -1 && e.activation == NS_ACT_TANH && n_h >= 1 &&
                    n_h <= kFusedMaxHidden && p->dims[0] <= 32 && p->dims[1] % 128 == 0 &&
                    (p->dims[1] == 512 || p->dims[1] == 1024);
        for (int l = 1; fuse && l <= n_h; ++l) fuse = p->dims[l] == p->dims[1] && p->dims[l + 1] == p->dims[1];
        if (fuse) {
            p->fused_cs = p->dims[1] / 128;
            p->tmF.resize(e.n_layers);
            p->tile_ms.assign(e.n_layers, 0.0f);
            for (int l = 1; l <= n_h && !s; ++l) {
                p->tile_n[l] = 128;
                s = make_tensor_map_bf16(&p->tmF[l], p->d_W[l], p->dims[l + 1], p->dims[l], 128, 2);
            }
        } else if (desc->hidden_tile == -1) {
            return fail(NS_ENOTSUP);   // the fused stack was requested for an emulator it cannot take
        } else if (desc->hidden_tile > 0) {
            // a caller-chosen N-tile for every tensor-core hidden layer (no autotuning)
            p->tile_ms.assign(e.n_layers, 0.0f);
            for (int l = 1; l <= e.n_layers - 2 && !s; ++l) {
                if (!tc_layer(l)) continue;
                if (desc->hidden_tile > p->dims[l + 1]) return fail(NS_EINVAL);
                p->tile_n[l] = desc->hidden_tile;
                s = make_tensor_map_bf16(&p->tmB[l], p->d_W[l], p->dims[l + 1], p->dims[l], desc->hidden_tile,
                                         gemm_tc_kps(p->dims[l]));
            }
        } else {
            s = autotune_hidden_tiles(p, e.n_layers - 2);   // hidden layers 1 .. L-2
        }
        if (s) return fail(s);
    }

    p->D = desc->n_data;
    p->has_lik = desc->cov != nullptr;
    if (cmb && desc->cmb.form == NS_CMB_TT_CV) p->has_lik = desc->data != nullptr;
    if (cmb) {
        int s = cmb_setup(p, desc);
        if (!s) s = workspace_create(p, p->max_batch, &p->ws);
        if (s) return fail(s);
        *out = p;
        return NS_OK;
    }

    // ---------------- shear grids and constants
    const ns_shear_desc& sd = desc->shear;
    ShearParams& sp = p->sp;
    sp.n_params = p->P;
    sp.nb = sd.n_bins;
    sp.n_pairs = sd.n_bins * (sd.n_bins + 1) / 2;
    sp.n_ell = sd.n_ell;
    sp.n_k = sd.n_k;
    sp.n_z = sd.n_z;
    sp.N = sd.n_chi;
    sp.D = desc->n_data;
    sp.n_tmpl = sd.n_tmpl;
    if (!projection_fits(sp, p->precision == NS_PREC_FP64 ? 8 : 4)) return fail(NS_ENOTSUP);
    sp.lnk_min = sd.lnk_min;
    sp.lnk_max = sd.lnk_max;
    sp.dlnk = (sd.lnk_max - sd.lnk_min) / (sd.n_k - 1);
    sp.ia_pivot = sd.ia_pivot;
    sp.c1rho = sd.c1rho;
    p->D = sp.D;
    p->n_z_emu = sd.n_z_emu;
    {
        const int N = sp.N;
        const double da = (1.0 - sd.a_min) / (N - 1);
        std::vector<double> a(N), lna(N), z(N), wa(N, da), zw(4 * N);
        std::vector<int> zrow(4 * N);
        const double dz = sd.z_max / (sd.n_z - 1);
        for (int n = 0; n < N; ++n) {
            a[n] = 1.0 - da * n;
            lna[n] = std::log(a[n]);
            z[n] = 1.0 / a[n] - 1.0;
            cr_taps(z[n], 0.0, dz, sd.n_z, &zrow[4 * n], &zw[4 * n]);
        }
        wa[0] *= 0.5;
        wa[N - 1] *= 0.5;
        std::vector<double> lnell(sd.n_ell);
        for (int l = 0; l < sd.n_ell; ++l) lnell[l] = std::log(sd.ell[l] + 0.5);
        std::vector<int> pi, pj;
        for (int i = 0; i < sd.n_bins; ++i)
            for (int j = i; j < sd.n_bins; ++j) { pi.push_back(i); pj.push_back(j); }
        double *da_, *dlna, *dz_, *dwa, *dzw, *dlnell, *dmu, *dsg, *ddata, *dtm = nullptr;
        int *dzrow, *dpi, *dpj;
        int s;
        if ((s = upload(a.data(), N, &da_, p->owned)) || (s = upload(lna.data(), N, &dlna, p->owned)) ||
            (s = upload(z.data(), N, &dz_, p->owned)) || (s = upload(wa.data(), N, &dwa, p->owned)) ||
            (s = upload(zw.data(), 4 * N, &dzw, p->owned)) || (s = upload(zrow.data(), 4 * N, &dzrow, p->owned)) ||
            (s = upload(lnell.data(), sd.n_ell, &dlnell, p->owned)) ||
            (s = upload(sd.nz_mean, sd.n_bins, &dmu, p->owned)) || (s = upload(sd.nz_sigma, sd.n_bins, &dsg, p->owned)) ||
            (s = upload(pi.data(), pi.size(), &dpi, p->owned)) || (s = upload(pj.data(), pj.size(), &dpj, p->owned)) ||
            (s = upload(desc->data ? desc->data : std::vector<double>(sp.D, 0.0).data(), sp.D, &ddata, p->owned)))
            return fail(s);
        if (sd.n_tmpl > 0 && (s = upload(sd.tmpl, (size_t)sp.D * sd.n_tmpl, &dtm, p->owned))) return fail(s);
        sp.a = da_; sp.lna = dlna; sp.z = dz_; sp.wa = dwa; sp.zw = dzw; sp.zrow = dzrow; sp.lnell = dlnell;
        sp.dz = dz;
        {
            std::vector<float> af(a.begin(), a.end()), lf(lna.begin(), lna.end()), zf(z.begin(), z.end()),
                wf(wa.begin(), wa.end());
            float *daf, *dlf, *dzf, *dwf;
            if ((s = upload(af.data(), N, &daf, p->owned)) || (s = upload(lf.data(), N, &dlf, p->owned)) ||
                (s = upload(zf.data(), N, &dzf, p->owned)) || (s = upload(wf.data(), N, &dwf, p->owned)))
                return fail(s);
            sp.a_f = daf; sp.lna_f = dlf; sp.z_f = dzf; sp.wa_f = dwf;
            // padded-table z-taps: the cell bracket, unfolded (ghost rows exist) and doubled
            std::vector<int> zrp(N);
            std::vector<double> z4(4 * N);
            std::vector<float> z4f(4 * N);
            for (int n = 0; n < N; ++n) {
                const double u = z[n] / dz;
                int j = (int)std::floor(u);
                j = std::max(0, std::min(j, sd.n_z - 2));
                double w[4];
                catmull_rom<double>(u - j, w);
                zrp[n] = j;
                for (int q = 0; q < 4; ++q) { z4[4 * n + q] = 2.0 * w[q]; z4f[4 * n + q] = (float)(2.0 * w[q]); }
            }
            int* dzr;
            double* dz4;
            float* dz4f;
            if ((s = upload(zrp.data(), N, &dzr, p->owned)) || (s = upload(z4.data(), 4 * N, &dz4, p->owned)) ||
                (s = upload(z4f.data(), 4 * N, &dz4f, p->owned)))
                return fail(s);
            sp.zrp = dzr; sp.zw4d = dz4; sp.zw4f = dz4f;
        }
        sp.nz_mean = dmu; sp.nz_sigma = dsg; sp.pi = dpi; sp.pj = dpj; sp.data = ddata; sp.tmpl = dtm;
        {
            // FP32 copies for the float kernels
            sp.lnk_min_f = (float)sd.lnk_min;
            sp.lnk_max_f = (float)sd.lnk_max;
            sp.inv_dlnk_f = 1.0f / (float)sp.dlnk;
            sp.ia_pivot_f = (float)sd.ia_pivot;
            sp.c1rho_f = (float)sd.c1rho;
            std::vector<float> lef(lnell.begin(), lnell.end()), muf(sd.nz_mean, sd.nz_mean + sd.n_bins),
                sgf(sd.nz_sigma, sd.nz_sigma + sd.n_bins), daf(sp.D, 0.f), tmf((size_t)sp.D * sd.n_tmpl);
            if (desc->data)
                for (int a = 0; a < sp.D; ++a) daf[a] = (float)desc->data[a];
            for (size_t i = 0; i < tmf.size(); ++i) tmf[i] = (float)sd.tmpl[i];
            float *dlef, *dmuf, *dsgf, *ddaf, *dtmf = nullptr;
            if ((s = upload(lef.data(), sd.n_ell, &dlef, p->owned)) ||
                (s = upload(muf.data(), sd.n_bins, &dmuf, p->owned)) ||
                (s = upload(sgf.data(), sd.n_bins, &dsgf, p->owned)) || (s = upload(daf.data(), sp.D, &ddaf, p->owned)))
                return fail(s);
            if (sd.n_tmpl > 0 && (s = upload(tmf.data(), tmf.size(), &dtmf, p->owned))) return fail(s);
            sp.lnell_f = dlef; sp.nz_mean_f = dmuf; sp.nz_sigma_f = dsgf; sp.data_f = ddaf; sp.tmpl_f = dtmf;
        }
        if (p->n_z_emu != sd.n_z) {
            std::vector<int> zr(4 * sd.n_z);
            std::vector<double> zwt(4 * sd.n_z);
            const double dzc = sd.z_max / (p->n_z_emu - 1);
            for (int j = 0; j < sd.n_z; ++j) {
                if (sd.z_interp == 1) {
                    // linear: taps (i, i + 1) with weights (1 - t, t); unused taps weight 0
                    const double u = j * dz / dzc;
                    int i = (int)std::floor(u);
                    i = std::max(0, std::min(i, p->n_z_emu - 2));
                    const double t = u - i;
                    zr[4 * j] = i; zr[4 * j + 1] = i + 1; zr[4 * j + 2] = i + 1; zr[4 * j + 3] = i + 1;
                    zwt[4 * j] = 1.0 - t; zwt[4 * j + 1] = t; zwt[4 * j + 2] = 0.0; zwt[4 * j + 3] = 0.0;
                } else {
                    cr_taps(j * dz, 0.0, dzc, p->n_z_emu, &zr[4 * j], &zwt[4 * j]);
                }
            }
            if ((s = upload(zr.data(), zr.size(), &p->d_zi_row, p->owned)) ||
                (s = upload(zwt.data(), zwt.size(), &p->d_zi_w, p->owned)))
                return fail(s);
        }
    }
    // ---------------- Gaussian likelihood: FP64 Cholesky, L^-1, constant
    if (p->has_lik) {
        const int D = sp.D;
        std::vector<double> L, Linv;
        if (!cholesky_inverse(desc->cov, D, L, Linv)) return fail(NS_EINVAL);
        double c0 = -0.5 * D * std::log(2.0 * M_PI);
        for (int a = 0; a < D; ++a) c0 -= std::log(L[(size_t)a * D + a]);
        p->c0 = c0;
        std::vector<double> LT((size_t)D * D);
        std::vector<float> LT32((size_t)D * D);
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) {
                LT[(size_t)b * D + a] = Linv[(size_t)a * D + b];
                LT32[(size_t)b * D + a] = (float)Linv[(size_t)a * D + b];
            }
        int s;
        if ((s = upload(LT.data(), LT.size(), &p->d_LinvT64, p->owned))) return fail(s);
        if ((s = upload(LT32.data(), LT32.size(), &p->d_LinvT32, p->owned))) return fail(s);
    }
    int s = workspace_create(p, p->max_batch, &p->ws);
    if (s) return fail(s);
    *out = p;
    return NS_OK;
}

extern "C" int ns_problem_free(ns_problem* p) {
    if (!p) return NS_EINVAL;
    cudaDeviceSynchronize();
    problem_release(p);
    return NS_OK;
}

extern "C" int ns_problem_dim(const ns_problem* p, int* d) {
    if (!p || !d) return NS_EINVAL;
    *d = p->d;
    return NS_OK;
}

namespace gpuns {
int launch_cube_to_free(const ns_problem* p, const double* cube, int B, double* theta, cudaStream_t st);
int launch_free_to_full(const ns_problem* p, const double* theta, int B, double* theta_full, cudaStream_t st);
}

extern "C" int ns_prior_transform(const ns_problem* p, const double* cube_dev, int B, double* theta_dev,
                                  void* stream) {
    if (!p || B < 0 || B > p->max_batch || (B > 0 && (!cube_dev || !theta_dev))) return NS_EINVAL;
    if (B == 0) return NS_OK;
    return launch_cube_to_free(p, cube_dev, B, theta_dev, (cudaStream_t)stream);
}

static int batch_common(const ns_problem* p, const double* theta_dev, int B, cudaStream_t st) {
    ns_problem* mp = const_cast<ns_problem*>(p);
    NS_TRY(launch_free_to_full(p, theta_dev, B, mp->ws.theta_full, st));
    k_set_int<<<1, 1, 0, st>>>(mp->ws.d_nrows, B);
    NS_CUDA_TRY(cudaGetLastError());
    return NS_OK;
}

extern "C" int loglike_batch(const ns_problem* p, const double* theta_dev, int B, double* logL_dev, void* stream) {
    if (!p || !p->has_lik || B < 0 || B > p->max_batch || (B > 0 && (!theta_dev || !logL_dev))) return NS_EINVAL;
    if (B == 0) return NS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    NS_TRY(batch_common(p, theta_dev, B, st));
    return run_likelihood(p, const_cast<Workspace*>(&p->ws), B, logL_dev, nullptr, st);
}

extern "C" int ns_model_batch(const ns_problem* p, const double* theta_dev, int B, double* model_dev, void* stream) {
    if (!p || p->kind == NS_KIND_GAUSS || B < 0 || B > p->max_batch || (B > 0 && (!theta_dev || !model_dev)))
        return NS_EINVAL;
    if (B == 0) return NS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    NS_TRY(batch_common(p, theta_dev, B, st));
    return run_likelihood(p, const_cast<Workspace*>(&p->ws), B, nullptr, model_dev, st);
}

extern "C" int ns_problem_fused(const ns_problem* p, int* cluster_size) {
    if (!p || !cluster_size) return NS_EINVAL;
    *cluster_size = p->fused_cs;
    return NS_OK;
}

extern "C" int ns_problem_tiles(const ns_problem* p, int* tile_n, float* ms, int n) {
    if (!p || !tile_n || n < p->n_layers) return NS_EINVAL;
    for (int l = 0; l < p->n_layers; ++l) {
        tile_n[l] = ((int)p->tile_n.size() > l && l >= 1) ? p->tile_n[l] : 0;
        if (ms) ms[l] = ((int)p->tile_ms.size() > l) ? p->tile_ms[l] : 0.f;
    }
    return NS_OK;
}

extern "C" int ns_problem_status(ns_problem* p, int* bits, int clear) {
    if (!p || !bits) return NS_EINVAL;
    NS_CUDA_TRY(cudaDeviceSynchronize());
    NS_CUDA_TRY(cudaMemcpy(bits, p->ws.d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (clear) NS_CUDA_TRY(cudaMemset(p->ws.d_err, 0, sizeof(int)));
    return NS_OK;
}

extern "C" int ns_emulator_batch(const ns_problem* p, const double* theta_dev, int B, double* out_dev,
                                 void* stream) {
    if (!p || p->kind == NS_KIND_GAUSS || B < 0 || B > p->max_batch || (B > 0 && (!theta_dev || !out_dev)))
        return NS_EINVAL;
    if (B == 0) return NS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    NS_TRY(batch_common(p, theta_dev, B, st));
    return run_emulator_only(p, const_cast<Workspace*>(&p->ws), B, out_dev, st);
}
