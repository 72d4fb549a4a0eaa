// Gaussian-approximation (GA) mean recursion of Sec. III in FP64 on the GPU, for the flooding
// schedule: one warp per Eb/N0 point runs
//   mu_v,i = mu0 + (i - 1) mu_c,   mu_c <- sum_j rho_j Phi^-1(1 - (1 - sum_i lambda_i Phi(mu_v,i))^(j-1))
// (Eqs. (4), (15), (16) with every other CN of class a), mu0 = 2 / sigma^2, until mu_c passes a
// cap (error-free decoding, the end of Sec. III), stops moving (a fixed point) or max_iter.
//
// Phi is Eq. (14), Phi(mu) = 1 - E[tanh(T/2)], T ~ N(mu, 2 mu), written as E[2 / (1 + e^T)]
// and integrated by the trapezoidal rule in x (T = mu + 2 sqrt(mu) x, weight e^{-x^2} / sqrt(pi))
// over [-12, 12] with step 1/32, the 769 nodes split over the warp's lanes; the rule converges
// geometrically for this analytic integrand.  Alternatively the closed form of the GA analysis
// the paper cites.  Phi^-1 is bisection on [0, 200].
#include <cmath>
#include <vector>

#include "device_common.cuh"
#include "ndgsbp_internal.h"

namespace ndgsbp {

constexpr int kGaNodes = 769;            // x = -12 + k / 32, k = 0..768
constexpr double kGaStep = 1.0 / 32.0;
constexpr int kGaMaxDeg = 64;

struct GaArgs {
    double lam[kGaMaxDeg + 1];
    double rho[kGaMaxDeg + 1];
    int dv_max, dc_max;
    double rate;
    const double* ebn0;
    int n;
    int kind;
    int max_iter;
    double mu_cap;
    unsigned char* conv;
    int* iters;
    double* mu;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Eq. (14), the same value in every lane of the warp.
__device__ double ga_phi(double mu, int kind, int lane) {
    if (mu <= 0.0) return 1.0;
    if (kind == NDGSBP_GA_PHI_CLOSED) {
        if (mu < 10.0) return exp(-0.4527 * pow(mu, 0.86) + 0.0218);
        return sqrt(M_PI / mu) * exp(-mu / 4.0) * (1.0 - 10.0 / (7.0 * mu));
    }
    const double s = 2.0 * sqrt(mu);
    double acc = 0.0;
    for (int k = lane; k < kGaNodes; k += 32) {
        const double x = -12.0 + k * kGaStep;
        const double t = mu + s * x;
        // 2 / (1 + e^t), without overflow for large t
        const double f = t > 0.0 ? 2.0 * exp(-t) / (1.0 + exp(-t)) : 2.0 / (1.0 + exp(t));
        acc += f * exp(-x * x);
    }
    return warp_sum(acc) * kGaStep * 0.56418958354775628;   // 1 / sqrt(pi)
}

__device__ double ga_phi_inv(double p, int kind, int lane) {
    if (p >= 1.0 && kind != NDGSBP_GA_PHI_CLOSED) return 0.0;
    double lo = 0.0, hi = 200.0;
    if (ga_phi(hi, kind, lane) >= p) return hi;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (ga_phi(mid, kind, lane) > p)
            lo = mid;
        else
            hi = mid;
        if (hi - lo <= 1e-13 * fmax(1.0, hi)) break;
    }
    return 0.5 * (lo + hi);
}

__global__ void ga_flood_kernel(const GaArgs a) {
    const int lane = threadIdx.x & 31;
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (k >= a.n) return;   // whole warps leave together
    const double sigma2 = 1.0 / (2.0 * a.rate * pow(10.0, a.ebn0[k] / 10.0));
    const double mu0 = 2.0 / sigma2;
    double mu_c = 0.0;
    int it = 1;
    unsigned char conv = 0;
    for (; it <= a.max_iter; ++it) {
        double s = 0.0;
        for (int i = 2; i <= a.dv_max; ++i)
            if (a.lam[i] > 0.0) s += a.lam[i] * ga_phi(mu0 + (i - 1) * mu_c, a.kind, lane);
        double next = 0.0;
        for (int j = 2; j <= a.dc_max; ++j)
            if (a.rho[j] > 0.0) next += a.rho[j] * ga_phi_inv(1.0 - pow(1.0 - s, j - 1), a.kind, lane);
        if (next >= a.mu_cap) {
            conv = 1;
            mu_c = next;
            break;
        }
        const bool still = fabs(next - mu_c) <= 1e-12 * fmax(1.0, next);
        mu_c = next;
        if (still) break;
    }
    if (lane == 0) {
        a.conv[k] = conv;
        a.iters[k] = it > a.max_iter ? a.max_iter : it;
        a.mu[k] = mu_c;
    }
}

}  // namespace ndgsbp

using namespace ndgsbp;

#define GA_TRY(expr)                                                                               \
    do {                                                                                           \
        cudaError_t _e = (expr);                                                                   \
        if (_e != cudaSuccess) {                                                                   \
            st = fail(NDGSBP_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(_e));                 \
            goto done;                                                                             \
        }                                                                                          \
    } while (0)

extern "C" {

ndgsbp_status ndgsbp_ga_flood(const double* lambda, int32_t dv_max, const double* rho, int32_t dc_max, double rate,
                              const double* ebn0_db, int32_t n_points, int32_t phi_kind, int32_t max_iter,
                              double mu_cap, uint8_t* converged, int32_t* iters, double* mu_c) {
    clear_error();
    if (!lambda || !rho || !ebn0_db || !converged || !iters || !mu_c || n_points < 1 || max_iter < 1 ||
        dv_max < 2 || dv_max > kGaMaxDeg || dc_max < 2 || dc_max > kGaMaxDeg || !(rate > 0.0 && rate < 1.0) ||
        !(mu_cap > 0.0 && mu_cap < 200.0) ||
        (phi_kind != NDGSBP_GA_PHI_EXACT && phi_kind != NDGSBP_GA_PHI_CLOSED))
        return fail(NDGSBP_ERR_INVALID, "ga_flood: bad arguments");
    GaArgs a{};
    for (int i = 0; i <= dv_max; ++i) a.lam[i] = lambda[i];
    for (int j = 0; j <= dc_max; ++j) a.rho[j] = rho[j];
    a.dv_max = dv_max;
    a.dc_max = dc_max;
    a.rate = rate;
    a.n = n_points;
    a.kind = phi_kind;
    a.max_iter = max_iter;
    a.mu_cap = mu_cap;
    ndgsbp_status st = NDGSBP_OK;
    double* d_e = nullptr;
    double* d_mu = nullptr;
    int* d_it = nullptr;
    unsigned char* d_cv = nullptr;
    constexpr int warps = 4;
    GA_TRY(cudaMalloc(&d_e, sizeof(double) * n_points));
    GA_TRY(cudaMalloc(&d_mu, sizeof(double) * n_points));
    GA_TRY(cudaMalloc(&d_it, sizeof(int) * n_points));
    GA_TRY(cudaMalloc(&d_cv, n_points));
    GA_TRY(cudaMemcpy(d_e, ebn0_db, sizeof(double) * n_points, cudaMemcpyHostToDevice));
    a.ebn0 = d_e;
    a.conv = d_cv;
    a.iters = d_it;
    a.mu = d_mu;
    ga_flood_kernel<<<(n_points + warps - 1) / warps, 32 * warps>>>(a);
    GA_TRY(cudaGetLastError());
    GA_TRY(cudaMemcpy(converged, d_cv, n_points, cudaMemcpyDeviceToHost));
    GA_TRY(cudaMemcpy(iters, d_it, sizeof(int) * n_points, cudaMemcpyDeviceToHost));
    GA_TRY(cudaMemcpy(mu_c, d_mu, sizeof(double) * n_points, cudaMemcpyDeviceToHost));
done:
    cudaFree(d_e);
    cudaFree(d_mu);
    cudaFree(d_it);
    cudaFree(d_cv);
    return st;
}

ndgsbp_status ndgsbp_ga_flood_threshold(const double* lambda, int32_t dv_max, const double* rho, int32_t dc_max,
                                        double rate, int32_t phi_kind, int32_t max_iter, double mu_cap, double lo_db,
                                        double hi_db, double tol_db, double* threshold_db) {
    clear_error();
    if (!threshold_db || !(hi_db > lo_db) || !(tol_db > 0.0))
        return fail(NDGSBP_ERR_INVALID, "ga_flood_threshold: need lo < hi and tol > 0");
    constexpr int n = 64;
    std::vector<double> e(n), mu(n);
    std::vector<uint8_t> cv(n);
    std::vector<int32_t> it(n);
    // the recursion converges at every SNR above the threshold: refine the bracketing pair of a
    // grid of points until it is narrower than tol
    for (int round = 0; round < 16; ++round) {
        for (int k = 0; k < n; ++k) e[k] = lo_db + (hi_db - lo_db) * k / (n - 1);
        ndgsbp_status st = ndgsbp_ga_flood(lambda, dv_max, rho, dc_max, rate, e.data(), n, phi_kind, max_iter, mu_cap,
                                           cv.data(), it.data(), mu.data());
        if (st) return st;
        int first = -1;
        for (int k = 0; k < n; ++k)
            if (cv[k]) {
                first = k;
                break;
            }
        if (first < 0) return fail(NDGSBP_ERR_INFEASIBLE, "ga_flood_threshold: no convergence below %.4f dB", hi_db);
        if (first == 0) {
            *threshold_db = e[0];
            return NDGSBP_OK;
        }
        lo_db = e[first - 1];
        hi_db = e[first];
        if (hi_db - lo_db <= tol_db) break;
    }
    *threshold_db = hi_db;
    return NDGSBP_OK;
}

}  // extern "C"
