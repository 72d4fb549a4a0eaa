// Gaussian-approximation (GA) mean recursions of Sec. III in FP64 on the GPU, one warp per Eb/N0
// point, mu0 = 2 / sigma^2, each run until mu_c passes a cap (error-free decoding, the end of
// Sec. III), stops moving (a fixed point) or max_iter:
//   flooding (ga_flood_kernel):  mu_v,i = mu0 + (i - 1) mu_c,
//     mu_c <- sum_j rho_j Phi^-1(1 - (1 - sum_i lambda_i Phi(mu_v,i))^(j-1))
//     (Eqs. (4), (15), (16) with every other CN of class a);
//   G groups with overlap ratio r (ga_group_kernel; r = 0 is GSBP): per sub-iteration g the VN
//     means of Eqs. (4)-(9) over the classes a (not updated yet in this iteration), b (the overlap
//     with group g - 1, Eq. (12)) and d (already updated, Eqs. (10)-(11)), the class-c and class-b
//     CN outputs of Eqs. (13), (15), (16), and the iteration's mean of Eq. (17).  The readings of
//     the classes and of Eqs. (6)-(9) are those of the library's design notes: the current
//     group's own term in Eqs. (6)-(7) is its output of the previous iteration (what its fresh CNs
//     hold during the sub-iteration), Eq. (8) is linear in (p, q) and so reduces to
//     mu0 + (i - 1)(y mu_d + z mu_b + (1 - y - z) mu_a), and class-b outputs use the weights of
//     Eq. (9) restricted to p >= 1.
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
constexpr int kGaMaxGroups = 64;

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
    int G;        // groups (ga_group_kernel)
    double r;     // overlap ratio (ga_group_kernel)
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

// Eqs. (15)-(16): the CN mean from the VN means mu_v[i], i = 2 .. dv_max.
__device__ double ga_cn_mean(const GaArgs& a, const double* mu_v, int lane) {
    double s = 0.0;
    for (int i = 2; i <= a.dv_max; ++i)
        if (a.lam[i] > 0.0) s += a.lam[i] * ga_phi(mu_v[i], a.kind, lane);
    double next = 0.0;
    for (int j = 2; j <= a.dc_max; ++j)
        if (a.rho[j] > 0.0) next += a.rho[j] * ga_phi_inv(1.0 - pow(1.0 - s, j - 1), a.kind, lane);
    return next;
}

// Stop test shared by both recursions: returns true when the run ends after this iteration.
__device__ __forceinline__ bool ga_step(const GaArgs& a, double next, double& mu_c, unsigned char& conv) {
    if (next >= a.mu_cap) {
        conv = 1;
        mu_c = next;
        return true;
    }
    const bool still = fabs(next - mu_c) <= 1e-12 * fmax(1.0, next);
    mu_c = next;
    return still;
}

__device__ __forceinline__ double ga_mu0(const GaArgs& a, int k) {
    const double sigma2 = 1.0 / (2.0 * a.rate * pow(10.0, a.ebn0[k] / 10.0));
    return 2.0 / sigma2;
}

__global__ void ga_flood_kernel(const GaArgs a) {
    const int lane = threadIdx.x & 31;
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (k >= a.n) return;   // whole warps leave together
    const double mu0 = ga_mu0(a, k);
    double mu_c = 0.0, mu_v[kGaMaxDeg + 1];
    int it = 1;
    unsigned char conv = 0;
    for (; it <= a.max_iter; ++it) {
        for (int i = 2; i <= a.dv_max; ++i) mu_v[i] = mu0 + (i - 1) * mu_c;
        if (ga_step(a, ga_cn_mean(a, mu_v, lane), mu_c, conv)) break;
    }
    if (lane == 0) {
        a.conv[k] = conv;
        a.iters[k] = it > a.max_iter ? a.max_iter : it;
        a.mu[k] = mu_c;
    }
}

__global__ void ga_group_kernel(const GaArgs a) {
    const int lane = threadIdx.x & 31;
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (k >= a.n) return;   // whole warps leave together
    const double mu0 = ga_mu0(a, k);
    const int G = a.G;
    const double r = a.r;
    const double D = G - (G - 1) * r;   // N_G / M of the size relation G N_G - (G - 1) N_G r = M
    const double x = 1.0 / D, z = r / D;
    // cc[g] / cb[g]: class-c and class-b outputs of group g in this iteration; prev: last iteration's cc
    double cc[kGaMaxGroups + 1], cb[kGaMaxGroups + 1], prev[kGaMaxGroups + 1], mu_v[kGaMaxDeg + 1];
    for (int g = 0; g <= G; ++g) prev[g] = 0.0;
    double mu_c = 0.0;
    int it = 1;
    unsigned char conv = 0;
    for (; it <= a.max_iter; ++it) {
        for (int g = 1; g <= G; ++g) {
            double mu_d, fd, fb, mu_b;
            if (g == 1) {
                // Eq. (10): class d is group 1's own fresh CNs, holding their last update
                mu_d = prev[1];
                fd = x;
                fb = 0.0;
                mu_b = 0.0;
            } else {
                // Eqs. (6)-(7): mean of the updated CNs (groups 1 .. g, the current one from the
                // last iteration); Eq. (11) fraction y, Eq. (12) fraction z
                double acc = cc[1] + prev[g];
                for (int kk = 2; kk < g; ++kk)
                    acc += r < 0.5 ? (r / (1.0 - r)) * cb[kk] + ((1.0 - 2.0 * r) / (1.0 - r)) * cc[kk] : cb[kk];
                mu_d = acc / g;
                fd = g * (1.0 - r) / D;
                fb = z;
                mu_b = (g - 1 == 1 || r < 0.5) ? cc[g - 1] : cb[g - 1];
            }
            const double fa = fmax(0.0, 1.0 - fd - fb);
            // Eq. (8) with the weights of Eq. (9): linear in (p, q)
            const double other = fd * mu_d + fb * mu_b + fa * mu_c;
            for (int i = 2; i <= a.dv_max; ++i) mu_v[i] = mu0 + (i - 1) * other;
            cc[g] = ga_cn_mean(a, mu_v, lane);
            if (g > 1 && r > 0.0) {
                // class-b CN: at least one class-d neighbour among the other i - 1 (p >= 1)
                for (int i = 2; i <= a.dv_max; ++i) {
                    if (!(a.lam[i] > 0.0)) continue;
                    const int n = i - 1;
                    double tot = 0.0, acc = 0.0, cnp = 1.0;   // cnp = C(n, p)
                    for (int pp = 1; pp <= n; ++pp) {
                        cnp = cnp * (n - pp + 1) / pp;
                        double cq = 1.0;                        // C(n - p, q)
                        for (int q = 0; q <= n - pp; ++q) {
                            if (q > 0) cq = cq * (n - pp - q + 1) / q;
                            const double w = cnp * cq * pow(fd, pp) * pow(fb, q) * pow(fa, n - pp - q);
                            tot += w;
                            acc += w * (mu0 + pp * mu_d + q * mu_b + (n - pp - q) * mu_c);
                        }
                    }
                    if (tot > 0.0) mu_v[i] = acc / tot;
                }
                cb[g] = ga_cn_mean(a, mu_v, lane);
            } else {
                cb[g] = cc[g];
            }
        }
        // Eq. (17): the iteration's CN mean
        const double next = z * cb[G] + ((G - G * r) / D) * cc[G];
        if (ga_step(a, next, mu_c, conv)) break;
        for (int g = 1; g <= G; ++g) prev[g] = cc[g];
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

// Fill the common arguments; false when they are invalid.
static bool ga_args(GaArgs& a, const double* lambda, int32_t dv_max, const double* rho, int32_t dc_max, double rate,
                    int32_t phi_kind, int32_t max_iter, double mu_cap) {
    if (!lambda || !rho || max_iter < 1 || dv_max < 2 || dv_max > kGaMaxDeg || dc_max < 2 || dc_max > kGaMaxDeg ||
        !(rate > 0.0 && rate < 1.0) || !(mu_cap > 0.0 && mu_cap < 200.0) ||
        (phi_kind != NDGSBP_GA_PHI_EXACT && phi_kind != NDGSBP_GA_PHI_CLOSED))
        return false;
    a = GaArgs{};
    for (int i = 0; i <= dv_max; ++i) a.lam[i] = lambda[i];
    for (int j = 0; j <= dc_max; ++j) a.rho[j] = rho[j];
    a.dv_max = dv_max;
    a.dc_max = dc_max;
    a.rate = rate;
    a.kind = phi_kind;
    a.max_iter = max_iter;
    a.mu_cap = mu_cap;
    a.G = 1;
    a.r = 0.0;
    return true;
}

// Run a recursion (groups = false: flooding) for n points; synchronous.
static ndgsbp_status ga_run(GaArgs a, bool groups, const double* ebn0_db, int32_t n_points, uint8_t* converged,
                            int32_t* iters, double* mu_c) {
    a.n = n_points;
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
    if (groups)
        ga_group_kernel<<<(n_points + warps - 1) / warps, 32 * warps>>>(a);
    else
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

// The smallest Eb/N0 in [lo, hi] at which the recursion converges: the recursion converges at
// every Eb/N0 above the threshold, so the bracketing pair of a 64-point grid is refined until it
// is narrower than tol; the upper end of the final pair is returned.
static ndgsbp_status ga_threshold(const GaArgs& a, bool groups, double lo_db, double hi_db, double tol_db,
                                  double* threshold_db, const char* who) {
    constexpr int n = 64;
    std::vector<double> e(n), mu(n);
    std::vector<uint8_t> cv(n);
    std::vector<int32_t> it(n);
    for (int round = 0; round < 16; ++round) {
        for (int k = 0; k < n; ++k) e[k] = lo_db + (hi_db - lo_db) * k / (n - 1);
        ndgsbp_status st = ga_run(a, groups, e.data(), n, cv.data(), it.data(), mu.data());
        if (st) return st;
        int first = -1;
        for (int k = 0; k < n; ++k)
            if (cv[k]) {
                first = k;
                break;
            }
        if (first < 0) return fail(NDGSBP_ERR_INFEASIBLE, "%s: no convergence below %.4f dB", who, hi_db);
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

static bool ga_groups_ok(int32_t G, double r) { return G >= 1 && G <= kGaMaxGroups && r >= 0.0 && r < 1.0; }

extern "C" {

ndgsbp_status ndgsbp_ga_flood(const double* lambda, int32_t dv_max, const double* rho, int32_t dc_max, double rate,
                              const double* ebn0_db, int32_t n_points, int32_t phi_kind, int32_t max_iter,
                              double mu_cap, uint8_t* converged, int32_t* iters, double* mu_c) {
    clear_error();
    GaArgs a;
    if (!ebn0_db || !converged || !iters || !mu_c || n_points < 1 ||
        !ga_args(a, lambda, dv_max, rho, dc_max, rate, phi_kind, max_iter, mu_cap))
        return fail(NDGSBP_ERR_INVALID, "ga_flood: bad arguments");
    return ga_run(a, false, ebn0_db, n_points, converged, iters, mu_c);
}

ndgsbp_status ndgsbp_ga_flood_threshold(const double* lambda, int32_t dv_max, const double* rho, int32_t dc_max,
                                        double rate, int32_t phi_kind, int32_t max_iter, double mu_cap, double lo_db,
                                        double hi_db, double tol_db, double* threshold_db) {
    clear_error();
    GaArgs a;
    if (!threshold_db || !(hi_db > lo_db) || !(tol_db > 0.0) ||
        !ga_args(a, lambda, dv_max, rho, dc_max, rate, phi_kind, max_iter, mu_cap))
        return fail(NDGSBP_ERR_INVALID, "ga_flood_threshold: bad arguments (need lo < hi and tol > 0)");
    return ga_threshold(a, false, lo_db, hi_db, tol_db, threshold_db, "ga_flood_threshold");
}

ndgsbp_status ndgsbp_ga_groups(const double* lambda, int32_t dv_max, const double* rho, int32_t dc_max, double rate,
                               int32_t G, double r, const double* ebn0_db, int32_t n_points, int32_t phi_kind,
                               int32_t max_iter, double mu_cap, uint8_t* converged, int32_t* iters, double* mu_c) {
    clear_error();
    GaArgs a;
    if (!ebn0_db || !converged || !iters || !mu_c || n_points < 1 || !ga_groups_ok(G, r) ||
        !ga_args(a, lambda, dv_max, rho, dc_max, rate, phi_kind, max_iter, mu_cap))
        return fail(NDGSBP_ERR_INVALID, "ga_groups: bad arguments");
    a.G = G;
    a.r = r;
    return ga_run(a, true, ebn0_db, n_points, converged, iters, mu_c);
}

ndgsbp_status ndgsbp_ga_groups_threshold(const double* lambda, int32_t dv_max, const double* rho, int32_t dc_max,
                                         double rate, int32_t G, double r, int32_t phi_kind, int32_t max_iter,
                                         double mu_cap, double lo_db, double hi_db, double tol_db,
                                         double* threshold_db) {
    clear_error();
    GaArgs a;
    if (!threshold_db || !(hi_db > lo_db) || !(tol_db > 0.0) || !ga_groups_ok(G, r) ||
        !ga_args(a, lambda, dv_max, rho, dc_max, rate, phi_kind, max_iter, mu_cap))
        return fail(NDGSBP_ERR_INVALID, "ga_groups_threshold: bad arguments (need lo < hi and tol > 0)");
    a.G = G;
    a.r = r;
    return ga_threshold(a, true, lo_db, hi_db, tol_db, threshold_db, "ga_groups_threshold");
}

}  // extern "C"
