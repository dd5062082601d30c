// Multi-geometry audit (Sec. 6.2-6.3): for each operator (geometry)
// and each observation arm, the age probes, anchor-connected reach, direct
// age boundary and old-age innovation, and the restricted Gram spectrum with
// its operational rank.  Host orchestration of the library's kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "rtt_internal.cuh"

using namespace rtt;

extern "C" rtt_status rtt_gram(rtt_op op, int arm_mask, const double* Q, int d, double* G,
                               void* stream);
extern "C" rtt_status rtt_gram_normal(rtt_op op, int arm_mask, const double* Q, int d, double* G,
                                      void* stream);
extern "C" rtt_status rtt_eig_sym(int n, double* A, double* evals_host, double* V, int max_sweeps,
                                  int* sweeps_host, void* stream);
extern "C" rtt_status rtt_probe_info(rtt_op op, int arm_mask, int n_ages, const double* ages,
                                     double h, double* info, void* stream);
extern "C" rtt_status rtt_direct_age_quantile(rtt_op op, double q, double* out, void* stream);
extern "C" rtt_status rtt_reach(rtt_op op, int arm_mask, int n_ages, const double* ages,
                                const double* info, double h, double a0q, double age_step,
                                rtt_reach_result* out, uint8_t* pass);

extern "C" rtt_status rtt_gram_class(rtt_op op, int arm_mask, int kind, double* G, void* stream);

extern "C" rtt_status rtt_eigvals_sym_batched(int n, int batch, double* A, double* evals_host,
                                              void* stream);

extern "C" rtt_status rtt_eig_sym_batched(int n, int batch, double* A, double* evals_host,
                                          double* V, int max_sweeps, int* sweeps_host,
                                          void* stream);

extern "C" rtt_status rtt_operational_rank(int n, const double* evals, double rho, int* rank_out,
                                           double* margin_out, double* sigma_out) {
    if (n < 1 || !evals || !rank_out || !margin_out || !(rho > 0.0) || !std::isfinite(rho)) {
        set_error("invalid operational-rank arguments (n=%d, rho=%g)", n, rho);
        return RTT_EINVAL;
    }
    std::vector<double> sig(n);
    for (int i = 0; i < n; ++i) {
        if (!std::isfinite(evals[i])) {
            set_error("operational rank: eigenvalue %d is not finite", i);
            return RTT_EINVAL;
        }
        sig[i] = std::sqrt(evals[i] > 0.0 ? evals[i] : 0.0);
    }
    std::sort(sig.begin(), sig.end(), [](double a, double c) { return a > c; });
    int rank = 0;
    double margin = INFINITY;
    for (int i = 0; i < n; ++i) {
        if (sig[i] >= rho) ++rank;
        margin = std::fmin(margin, std::fabs(sig[i] - rho) / rho);
    }
    *rank_out = rank;
    *margin_out = margin;
    if (sigma_out) std::copy(sig.begin(), sig.end(), sigma_out);
    return RTT_OK;
}

extern "C" rtt_status rtt_rank_audit(const rtt_op* ops, int n_ops, const double* const* Q_dev,
                                     int d, const int* arm_masks, int n_arms, int n_ages,
                                     const double* ages_host, double h, double quantile,
                                     int gram_mode, rtt_audit_record* out, double* sigma_out,
                                     void* stream) {
    if (!ops || n_ops < 1 || !Q_dev || d < 1 || d > 4096 || !arm_masks || n_arms < 1 ||
        gram_mode < RTT_GRAM_DATA || gram_mode > RTT_GRAM_CLASS_L224 ||
        (gram_mode >= RTT_GRAM_CLASS_S224 && d != 224) ||
        n_ages < 1 || n_ages > 256 || !ages_host || !(h > 0.0) || !(quantile > 0.0) || !out) {
        set_error("invalid rank-audit arguments");
        return RTT_EINVAL;
    }
    for (int g = 0; g < n_ops; ++g) RTT_TRY(whole_only(ops[g], "the rank audit"));
    const int nb = n_ops * n_arms;
    double *G = nullptr, *V = nullptr;
    cudaError_t e = cudaMalloc(&G, (size_t)nb * d * d * 8);
    if (e == cudaSuccess) e = cudaMalloc(&V, (size_t)nb * d * d * 8);
    if (e != cudaSuccess) {
        cudaFree(G);
        cudaFree(V);
        set_error("rank audit: allocation failed");
        return RTT_ENOMEM;
    }
    std::vector<double> info(n_ages), ev((size_t)nb * d);
    std::vector<int> sweeps(nb);
    const double age_step = n_ages > 1 ? ages_host[1] - ages_host[0] : 1.0;
    rtt_status s = RTT_OK;
    // probes, reach and restricted Grams of every (geometry, arm)
    for (int g = 0; g < n_ops && s == RTT_OK; ++g) {
        rtt_op op = ops[g];
        if (!op || (!Q_dev[g] && gram_mode < RTT_GRAM_CLASS_S224)) {
            set_error("rank audit: operator or class %d missing", g);
            s = RTT_EINVAL;
            break;
        }
        double a0 = 0.0;
        s = rtt_direct_age_quantile(op, quantile, &a0, stream);
        for (int ai = 0; ai < n_arms && s == RTT_OK; ++ai) {
            const auto t0 = std::chrono::steady_clock::now();
            rtt_audit_record& r = out[(size_t)g * n_arms + ai];
            r.arm_mask = arm_masks[ai];
            s = rtt_probe_info(op, arm_masks[ai], n_ages, ages_host, h, info.data(), stream);
            if (s != RTT_OK) break;
            rtt_reach_result rr;
            s = rtt_reach(op, arm_masks[ai], n_ages, ages_host, info.data(), h, a0, age_step, &rr,
                          nullptr);
            if (s != RTT_OK) break;
            r.reach = rr;
            const auto t1 = std::chrono::steady_clock::now();
            double* Gi = G + ((size_t)g * n_arms + ai) * d * d;
            if (gram_mode >= RTT_GRAM_CLASS_S224) {
                s = rtt_gram_class(op, arm_masks[ai],
                                   gram_mode == RTT_GRAM_CLASS_S224 ? RTT_CLASS_S224 : RTT_CLASS_L224,
                                   Gi, stream);
                if (s == RTT_ESTATE) {  // rows the class path does not handle
                    s = Q_dev[g] ? rtt_gram_normal(op, arm_masks[ai], Q_dev[g], d, Gi, stream)
                                 : RTT_EINVAL;
                    if (s == RTT_EINVAL) set_error("rank audit: class Gram unavailable and no Q");
                }
            } else {
                s = gram_mode == RTT_GRAM_NORMAL
                        ? rtt_gram_normal(op, arm_masks[ai], Q_dev[g], d, Gi, stream)
                        : rtt_gram(op, arm_masks[ai], Q_dev[g], d, Gi, stream);
            }
            if (s == RTT_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
                set_error("rank audit: Gram failed: %s", cudaGetErrorString(cudaGetLastError()));
                s = RTT_ECUDA;
            }
            r.s_ref = op->s_ref;
            const auto t2 = std::chrono::steady_clock::now();
            r.seconds_probe = std::chrono::duration<double>(t1 - t0).count();
            r.seconds_gram = std::chrono::duration<double>(t2 - t1).count();
            r.seconds = std::chrono::duration<double>(t2 - t0).count();
        }
    }
    // all spectra: eigenvalues of every matrix by tridiagonal reduction and
    // bisection (on a copy), then cyclic Jacobi for any matrix with an
    // eigenvalue within the reduction's error bound of the threshold rho^2
    if (s == RTT_OK) {
        const auto t0 = std::chrono::steady_clock::now();
        cudaStream_t st = (cudaStream_t)stream;
        const size_t bytes = (size_t)nb * d * d * 8;
        if (cudaMemcpyAsync(V, G, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
            set_error("rank audit: copy failed");
            s = RTT_ECUDA;
        }
        if (s == RTT_OK) s = rtt_eigvals_sym_batched(d, nb, V, ev.data(), stream);
        for (int b = 0; s == RTT_OK && b < nb; ++b) {
            const double rho = ops[b / n_arms]->opt.rho;
            double amax = 0.0;
            for (int i = 0; i < d; ++i) amax = std::fmax(amax, std::fabs(ev[(size_t)b * d + i]));
            const double bound = 64.0 * d * 2.220446049250313e-16 * amax;
            bool near = false;
            for (int i = 0; i < d; ++i) near = near || std::fabs(ev[(size_t)b * d + i] - rho * rho) <= bound;
            sweeps[b] = 0;
            if (near) {  // decide this matrix with the Jacobi spectrum (relative accuracy)
                s = rtt_eig_sym(d, G + (size_t)b * d * d, ev.data() + (size_t)b * d, V, 80,
                                &sweeps[b], stream);
            }
        }
        const double te = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        for (int b = 0; s == RTT_OK && b < nb; ++b) {
            rtt_audit_record& r = out[b];
            std::vector<double> sig(d);
            const double rho = ops[b / n_arms]->opt.rho;
            int rank = 0;
            double margin = INFINITY, smin_pos = INFINITY;
            s = rtt_operational_rank(d, ev.data() + (size_t)b * d, rho, &rank, &margin, sig.data());
            if (s != RTT_OK) break;
            for (int i = 0; i < d; ++i)
                if (sig[i] > 0.0) smin_pos = std::fmin(smin_pos, sig[i]);
            r.rank = rank;
            r.margin = margin;
            r.sigma_max = sig[0];
            r.sigma_min_pos = smin_pos;
            r.jacobi_sweeps = sweeps[b];
            r.seconds += te / nb;
            r.seconds_eig = te / nb;
            if (sigma_out)
                for (int i = 0; i < d; ++i) sigma_out[(size_t)b * d + i] = sig[i];
        }
    }
    cudaFree(G);
    cudaFree(V);
    return s;
}
