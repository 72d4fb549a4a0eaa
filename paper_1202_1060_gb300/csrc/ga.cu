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
// the paper cites.  Phi^-1 is bisection on [0, 200]; for the closed form, whose one evaluation
// needs no warp, the lanes evaluate the next five levels' midpoints at once.
#include <cmath>
#include <vector>

#include "device_common.cuh"
#include "ndgsbp_internal.h"

namespace ndgsbp {

constexpr int kGaNodes = 769;            // x = -12 + k / 32, k = 0..768
constexpr double kGaStep = 1.0 / 32.0;
constexpr int kGaMaxDeg = 64;
constexpr int kGaMaxGroups = 64;
constexpr int kGaWarps = 1;              // one point per block: a point's serial FP64 chain gets an SM's FP64 pipe
constexpr int kGaWTab = 512;             // class-b weights of Eq. (9) cached per warp (shared memory)

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
    // closed form: Phi(10-), Phi(10) and Phi(0+), which only sort p into the cases of
    // ga_phi_inv_closed (with a 1e-9 relative margin; computed on the host)
    double p_left, p_right, p_zero;
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

// Bisection for the closed form, five levels per step, from the bracket (lo, hi) reached after
// `steps` halvings of [0, 200]: lane j - 1 evaluates node j (1..31, heap order: children 2j below
// the midpoint, 2j + 1 above) of the next five levels' tree, its bracket rebuilt from (lo, hi) by
// the same halvings; the ballot then replays the five decisions one by one with the stop test
// after each, so every midpoint, decision and the result are those of the one-level loop of
// ga_phi_inv.
__device__ double ga_bisect_closed(double p, double lo, double hi, int steps, int lane) {
    const int j = lane + 1;
    const int depth = 31 - __clz(j);
    while (steps < 200) {
        double l = lo, h = hi;
        for (int b = depth - 1; b >= 0; --b) {
            const double m = 0.5 * (l + h);
            if ((j >> b) & 1)
                l = m;
            else
                h = m;
        }
        const bool above = lane < 31 && ga_phi(0.5 * (l + h), NDGSBP_GA_PHI_CLOSED, lane) > p;
        const unsigned ball = __ballot_sync(0xffffffffu, above);
        int node = 1;
        for (int lev = 0; lev < 5 && steps < 200; ++lev, ++steps) {
            const double m = 0.5 * (lo + hi);
            if ((ball >> (node - 1)) & 1u) {
                lo = m;
                node = 2 * node + 1;
            } else {
                hi = m;
                node = 2 * node;
            }
            if (hi - lo <= 1e-13 * fmax(1.0, hi)) return 0.5 * (lo + hi);
        }
    }
    return 0.5 * (lo + hi);
}

// Phi^-1 of the closed form, with the result of the one-level bisection.  Each piece of the closed
// form decreases, and the jump at mu = 10 goes up (from Phi(10-) = 0.03847 to Phi(10) = 0.03944):
// outside that band of p and below Phi(0+) = e^0.0218 there is one root r, in closed form on
// (0, 10) and by Newton's method on the logarithm above.  Every bisection midpoint farther than
// delta = 4e-14 max(1, r) from r is decided by its side of r (there Phi moves by over ten times
// its rounding error), and the midpoints of the levels above a bracket are that bracket's ends;
// so the bisection starts from the bracket five levels above the last one (the level at which
// the width first meets the stop test), when both its ends are that far from r, and runs from
// [0, 200] otherwise (the band, p near Phi(0+), or an end within delta).
__device__ double ga_phi_inv_closed(const GaArgs& a, double p, double phi_top, int lane) {
    if (phi_top >= p) return 200.0;
    const bool left = p > a.p_right * (1.0 + 1e-9) && p < a.p_zero * (1.0 - 1e-9);
    if (!left && !(p < a.p_left * (1.0 - 1e-9))) return ga_bisect_closed(p, 0.0, 200.0, 0, lane);
    const double lp = log(p);
    double r;
    if (left) {
        r = pow((0.0218 - lp) / 0.4527, 1.0 / 0.86);
    } else {
        r = fmin(200.0, fmax(10.0, -4.0 * lp));
        for (int it = 0; it < 6; ++it) {
            const double g = log(sqrt(M_PI / r) * (1.0 - 10.0 / (7.0 * r))) - r / 4.0 - lp;
            const double dg = -0.5 / r - 0.25 + (10.0 / (7.0 * r * r)) / (1.0 - 10.0 / (7.0 * r));
            r = fmin(200.0, fmax(10.0, r - g / dg));
        }
    }
    // the first level whose bracket around r meets the stop test (two to four levels below k)
    int k = (int)ceil(log2(200.0 / (1e-13 * fmax(1.0, r)))) - 2;
    bool found = false;
    for (int t = 0; t < 8 && !found; ++t, ++k) {
        const double w = ldexp(200.0, -k);
        const double lo = w * floor(r / w);
        found = w <= 1e-13 * fmax(1.0, lo + w);
    }
    if (!found) return ga_bisect_closed(p, 0.0, 200.0, 0, lane);
    k -= 6;   // the loop stepped once past the level found
    const double w = ldexp(200.0, -k);
    const double lo = w * floor(r / w), hi = lo + w;
    const double delta = 4e-14 * fmax(1.0, r);
    if (lo <= r && r < hi && (lo == 0.0 || r - lo > delta) && (hi == 200.0 || hi - r > delta))
        return ga_bisect_closed(p, lo, hi, k, lane);
    return ga_bisect_closed(p, 0.0, 200.0, 0, lane);
}

// phi_top = Phi(200), the upper end of the search (the same in every call of a kernel).
__device__ double ga_phi_inv(const GaArgs& a, double p, double phi_top, int kind, int lane) {
    if (kind == NDGSBP_GA_PHI_CLOSED) return ga_phi_inv_closed(a, p, phi_top, lane);
    if (p >= 1.0) return 0.0;
    double lo = 0.0, hi = 200.0;
    if (phi_top >= p) return hi;
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
__device__ double ga_cn_mean(const GaArgs& a, const double* mu_v, double phi_top, int lane) {
    double s = 0.0;
    for (int i = 2; i <= a.dv_max; ++i)
        if (a.lam[i] > 0.0) s += a.lam[i] * ga_phi(mu_v[i], a.kind, lane);
    double next = 0.0;
    for (int j = 2; j <= a.dc_max; ++j)
        if (a.rho[j] > 0.0) next += a.rho[j] * ga_phi_inv(a, 1.0 - pow(1.0 - s, j - 1), phi_top, a.kind, lane);
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
    const double phi_top = ga_phi(200.0, a.kind, lane);
    double mu_c = 0.0, mu_v[kGaMaxDeg + 1];
    int it = 1;
    unsigned char conv = 0;
    for (; it <= a.max_iter; ++it) {
        for (int i = 2; i <= a.dv_max; ++i) mu_v[i] = mu0 + (i - 1) * mu_c;
        if (ga_step(a, ga_cn_mean(a, mu_v, phi_top, lane), mu_c, conv)) break;
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
    const double phi_top = ga_phi(200.0, a.kind, lane);
    const int G = a.G;
    const double r = a.r;
    const double D = G - (G - 1) * r;   // N_G / M of the size relation G N_G - (G - 1) N_G r = M
    const double x = 1.0 / D, z = r / D;
    // The weights of Eq. (9) restricted to p >= 1 depend on g, i, p and q only: when they fit,
    // the lanes compute them once (term t by lane t mod 32) into a table read by every iteration.
    __shared__ double wtab[kGaWarps][kGaWTab];
    double* wt = wtab[threadIdx.x >> 5];
    int terms = 0;   // terms per group: sum over the VN degrees i of (i - 1) i / 2
    for (int i = 2; i <= a.dv_max; ++i)
        if (a.lam[i] > 0.0) terms += (i - 1) * i / 2;
    const bool tab = r > 0.0 && G > 1 && (G - 1) * terms <= kGaWTab;
    if (tab) {
        int t = 0;
        for (int g = 2; g <= G; ++g) {
            const double fd = g * (1.0 - r) / D, fb = z, fa = fmax(0.0, 1.0 - fd - fb);
            for (int i = 2; i <= a.dv_max; ++i) {
                if (!(a.lam[i] > 0.0)) continue;
                const int n = i - 1;
                double cnp = 1.0;
                for (int pp = 1; pp <= n; ++pp) {
                    cnp = cnp * (n - pp + 1) / pp;
                    double cq = 1.0;
                    for (int q = 0; q <= n - pp; ++q, ++t) {
                        if (q > 0) cq = cq * (n - pp - q + 1) / q;
                        if ((t & 31) == lane) wt[t] = cnp * cq * pow(fd, pp) * pow(fb, q) * pow(fa, n - pp - q);
                    }
                }
            }
        }
        __syncwarp();
    }
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
            cc[g] = ga_cn_mean(a, mu_v, phi_top, lane);
            if (g > 1 && r > 0.0) {
                // class-b CN: at least one class-d neighbour among the other i - 1 (p >= 1)
                int t = (g - 2) * terms;
                for (int i = 2; i <= a.dv_max; ++i) {
                    if (!(a.lam[i] > 0.0)) continue;
                    const int n = i - 1;
                    double tot = 0.0, acc = 0.0, cnp = 1.0;   // cnp = C(n, p)
                    for (int pp = 1; pp <= n; ++pp) {
                        cnp = cnp * (n - pp + 1) / pp;
                        double cq = 1.0;                        // C(n - p, q)
                        for (int q = 0; q <= n - pp; ++q) {
                            if (q > 0) cq = cq * (n - pp - q + 1) / q;
                            const double w =
                                tab ? wt[t++] : cnp * cq * pow(fd, pp) * pow(fb, q) * pow(fa, n - pp - q);
                            tot += w;
                            acc += w * (mu0 + pp * mu_d + q * mu_b + (n - pp - q) * mu_c);
                        }
                    }
                    if (tot > 0.0) mu_v[i] = acc / tot;
                }
                cb[g] = ga_cn_mean(a, mu_v, phi_top, lane);
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
    a.p_left = std::exp(-0.4527 * std::pow(10.0, 0.86) + 0.0218);
    a.p_right = std::sqrt(M_PI / 10.0) * std::exp(-10.0 / 4.0) * (1.0 - 10.0 / 70.0);
    a.p_zero = std::exp(0.0218);
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
        ga_group_kernel<<<(n_points + kGaWarps - 1) / kGaWarps, 32 * kGaWarps>>>(a);
    else
        ga_flood_kernel<<<(n_points + kGaWarps - 1) / kGaWarps, 32 * kGaWarps>>>(a);
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
// every Eb/N0 above the threshold, so the bracketing pair of a grid of at most 64 points is
// refined until it is narrower than tol; the upper end of the final pair is returned.  A grid no
// finer than tol is used where one suffices: points closer to the threshold than that only cost
// iterations (the recursion slows down on both sides of it), and a launch lasts as long as its
// slowest point.
static ndgsbp_status ga_threshold(const GaArgs& a, bool groups, double lo_db, double hi_db, double tol_db,
                                  double* threshold_db, const char* who) {
    constexpr int n_max = 64;
    std::vector<double> e(n_max), mu(n_max);
    std::vector<uint8_t> cv(n_max);
    std::vector<int32_t> it(n_max);
    for (int round = 0; round < 16; ++round) {
        const double need = std::ceil((hi_db - lo_db) / tol_db) + 1.0;
        const int n = need < n_max ? std::max(3, (int)need) : n_max;
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
