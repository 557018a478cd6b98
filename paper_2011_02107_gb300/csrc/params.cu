// Parameter heuristic on the GPU (Sec. III): Lanczos upper bound on |E|
// (the "upper-bound-estimator" the paper cites: largest |Ritz value| plus the
// residual norm), and the window a from a kernel-polynomial estimate of the
// density of states built from Chebyshev moments of the same start vector.
// The H.v steps reuse the fused stencil kernel; these kernels do the vector
// updates, the small tridiagonal eigenproblem and the window search.

#include <float.h>
#include <math.h>

#include "../../include/dacp.h"
#include "common.cuh"
#include "ops.h"

namespace dacp {

__device__ __forceinline__ double warp_sum_p(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// w -= alpha_r v (alpha_r = moment row 2j+1 of realization r), then ||w||^2 per
// realization into beta2[r * steps + j] (deterministic last-CTA reduction).
template <typename T>
__global__ void __launch_bounds__(kThreads) lanczos_orth_kernel(const Item* __restrict__ items,
                                                                const RealInfo* __restrict__ real, const T* v,
                                                                T* w, const double* __restrict__ lmom,
                                                                int rows, int j, double* part,
                                                                unsigned* real_done, double* beta2, int steps) {
    __shared__ double red_s[kThreads / 32];
    __shared__ int last_s;
    const int tid = threadIdx.x;
    const Item it = items[blockIdx.x];
    const RealInfo R = real[it.r];
    const double alpha = lmom[static_cast<int64_t>(it.r) * rows + 2 * j + 1];
    const T al = static_cast<T>(alpha);
    const int tstates = 1 << R.tbits;
    const int64_t base = R.off + (static_cast<int64_t>(it.tile) << R.tbits);
    double acc = 0.0;
    for (int sl = tid; sl < tstates; sl += kThreads) {
        const T nv = w[base + sl] - al * v[base + sl];
        w[base + sl] = nv;
        acc = fma(static_cast<double>(nv), static_cast<double>(nv), acc);
    }
    acc = warp_sum_p(acc);
    if ((tid & 31) == 0) red_s[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) s += red_s[i];
        part[blockIdx.x] = s;
        __threadfence();
        last_s = (atomicAdd(&real_done[it.r], 1u) == static_cast<unsigned>(R.item_count - 1));
    }
    __syncthreads();
    if (last_s && tid == 0) {
        __threadfence();
        double s = 0.0;
        for (int i = 0; i < R.item_count; ++i) s += __ldcg(part + R.item_begin + i);
        beta2[it.r * steps + j] = s;
        real_done[it.r] = 0u;
    }
}

// w /= beta_{j+1}; a zero residual (invariant subspace) leaves w = 0.
template <typename T>
__global__ void __launch_bounds__(kThreads) lanczos_scale_kernel(const Item* __restrict__ items,
                                                                 const RealInfo* __restrict__ real, T* w,
                                                                 const double* __restrict__ beta2, int j,
                                                                 int steps) {
    const Item it = items[blockIdx.x];
    const RealInfo R = real[it.r];
    const double b2 = beta2[it.r * steps + j];
    const T sc = b2 > 0.0 ? static_cast<T>(1.0 / sqrt(b2)) : T(0);
    const int tstates = 1 << R.tbits;
    const int64_t base = R.off + (static_cast<int64_t>(it.tile) << R.tbits);
    for (int sl = threadIdx.x; sl < tstates; sl += kThreads) w[base + sl] *= sc;
}

// coef[r] = {1, -beta_{j+1}, 0} for the next Lanczos apply.
__global__ void lanczos_coef_kernel(int R, const double* __restrict__ beta2, int j, int steps, double* coef) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    coef[8 * r + 0] = 1.0;
    coef[8 * r + 1] = -sqrt(beta2[r * steps + j]);
    coef[8 * r + 2] = 0.0;
}

// Number of eigenvalues of the k x k tridiagonal (alpha, beta) below x (Sturm count).
__host__ __device__ int sturm_count(const double* al, const double* b2, int k, double x) {
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < k; ++i) {
        const double off = i > 0 ? b2[i - 1] : 0.0;          // beta_{i}^2
        d = (al[i] - x) - (i > 0 ? off / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

// The idx-th smallest eigenvalue (0-based) of the k x k tridiagonal, by bisection
// on the Sturm count inside the Gershgorin interval [-gmax, gmax], until the interval
// is a few units of rounding of the matrix scale wide (about 52 halvings): the bounds
// below need the eigenvalues to the matrix's absolute accuracy only.
__host__ __device__ double tridiag_eig(const double* al, const double* b2, int k, int idx, double gmax) {
    double lo = -gmax - 1.0, hi = gmax + 1.0;
    const double tol = 4.0 * DBL_EPSILON * (gmax + 1.0);
    for (int it = 0; it < 200; ++it) {
        if (!(hi - lo > tol)) break;
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(al, b2, k, mid) >= idx + 1) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Gershgorin radius of the tridiagonal: max_i |alpha_i| + beta_i + beta_{i+1}.
__host__ __device__ double tridiag_gmax_row(const double* al, const double* b2, int k, int i) {
    const double bl = i > 0 ? sqrt(b2[i - 1]) : 0.0;
    const double br = i < k - 1 ? sqrt(b2[i]) : 0.0;
    return fabs(al[i]) + bl + br;
}

// z_{k,i}^2, the squared last component of the tridiagonal's i-th eigenvector, from its
// eigenvalues th[0..k) and those of the leading (k-1) x (k-1) block mu[0..k-1):
// prod_j (theta_i - mu_j) / prod_{j != i} (theta_i - theta_j). Cauchy interlacing pairs each
// factor into a ratio of magnitude at most one; a zero denominator counts as one, which can
// only enlarge the bound.
__host__ __device__ double ritz_last_comp2(const double* th, const double* mu, int k, int i) {
    double v = 1.0;
    for (int j = 0; j < k; ++j) {
        if (j == i) continue;
        const double num = th[i] - mu[j < i ? j : j - 1];
        const double den = th[i] - th[j];
        if (den != 0.0) v *= fmin(1.0, fabs(num / den));
    }
    return v;
}

// Ritz-residual rule (rule 1): max |theta| + beta_{k+1} max_i |e_k^T z_i|, before the
// safety factor. The last components come without the vectors (ritz_last_comp2).
// b2[0..k-2] are the squared off-diagonals, b2[k-1] the squared residual norm. k <= 64.
// Host form (test hook); the kernel below spreads the same steps over a warp.
__host__ __device__ double ritz_rule_bound(const double* al, const double* b2, int k) {
    double gmax = 0.0;
    for (int i = 0; i < k; ++i) gmax = fmax(gmax, tridiag_gmax_row(al, b2, k, i));
    double th[64], mu[64];
    for (int i = 0; i < k; ++i) th[i] = tridiag_eig(al, b2, k, i, gmax);
    for (int i = 0; i < k - 1; ++i) mu[i] = tridiag_eig(al, b2, k - 1, i, gmax);
    double zmax = k == 1 ? 1.0 : 0.0;
    for (int i = 0; k > 1 && i < k; ++i) zmax = fmax(zmax, sqrt(ritz_last_comp2(th, mu, k, i)));
    return fmax(fabs(th[0]), fabs(th[k - 1])) + sqrt(b2[k - 1]) * zmax;
}

__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

constexpr int kBoundWarps = 4;

// Extreme Ritz values by bisection; bound = max(|theta_min|, |theta_max|) + beta_{k+1}
// (rule 0) or the Ritz-residual rule (rule 1), times (1 + safety), clamped to the
// Pauli 1-norm pnorm[r]. One warp per realization: the lanes bisect different
// eigenvalues (rule 1 needs all k of them and the k - 1 of the leading block). The first
// `steps` of a run of `stride` Lanczos steps (beta2's row length) enter the bound.
__global__ void __launch_bounds__(32 * kBoundWarps) lanczos_bound_kernel(int R, const double* __restrict__ lmom,
                                                                         int rows, const double* __restrict__ beta2,
                                                                         int steps, int stride,
                                                                         const double* __restrict__ pnorm,
                                                                         double safety, double* emax, int rule) {
    __shared__ double s_al[kBoundWarps][64], s_b2[kBoundWarps][64], s_th[kBoundWarps][64], s_mu[kBoundWarps][64];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * kBoundWarps + wid;
    if (r >= R) return;                          // uniform per warp; no block-wide barrier follows
    double* al = s_al[wid];
    double* b2 = s_b2[wid];
    double* th = s_th[wid];
    double* mu = s_mu[wid];
    const int k = steps;
    for (int i = lane; i < k; i += 32) {
        al[i] = lmom[static_cast<int64_t>(r) * rows + 2 * i + 1];
        b2[i] = beta2[static_cast<int64_t>(r) * stride + i];
    }
    __syncwarp();
    double gmax = 0.0;
    for (int i = lane; i < k; i += 32) gmax = fmax(gmax, tridiag_gmax_row(al, b2, k, i));
    gmax = warp_max_d(gmax);
    double bound;
    if (rule == 1) {
        for (int i = lane; i < k; i += 32) th[i] = tridiag_eig(al, b2, k, i, gmax);
        for (int i = lane; i < k - 1; i += 32) mu[i] = tridiag_eig(al, b2, k - 1, i, gmax);
        __syncwarp();
        double zmax = k == 1 ? 1.0 : 0.0;
        for (int i = lane; k > 1 && i < k; i += 32) zmax = fmax(zmax, sqrt(ritz_last_comp2(th, mu, k, i)));
        zmax = warp_max_d(zmax);
        bound = (fmax(fabs(th[0]), fabs(th[k - 1])) + sqrt(b2[k - 1]) * zmax) * (1.0 + safety);
    } else {
        double t = 0.0;
        if (lane < 2) t = tridiag_eig(al, b2, k, lane == 0 ? 0 : k - 1, gmax);
        const double tmin = __shfl_sync(0xffffffffu, t, 0), tmax = __shfl_sync(0xffffffffu, t, 1);
        bound = (fmax(fabs(tmin), fabs(tmax)) + sqrt(b2[k - 1])) * (1.0 + safety);
    }
    if (lane == 0) emax[r] = fmin(bound, pnorm[r]);
}

// Kernel-polynomial window: mu_j = 2 P_j - P_{j mod 2} (j < M) of the
// normalised start vector under G = H/E_max; Jackson damping; expected count
// in [-a_r, a_r] = D [g_0 mu_0 (pi - 2 phi)/pi + 2 sum g_j mu_j (sin(j(pi-phi)) - sin(j phi))/(pi j)],
// phi = acos(a_r); bisection for count = d_target. Then K = ceil(c E_max / a)
// and n = ceil((basis_ratio d / b - 1) / 2).
__global__ void kpm_window_kernel(int R, const RealInfo* __restrict__ real, const double* __restrict__ P,
                                  int M, const double* __restrict__ emax, double d_target, double c_order,
                                  double basis_ratio, int b, const float* __restrict__ knobs, int n_eigs,
                                  double* a_out, int* K_out, int* n_out) {
    // one warp per realization: the lanes share the moment sum of each count evaluation
    const int r = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (r >= R) return;
    if (knobs) {
        // learned knobs per realization: log(window ratio), filter constant, basis ratio;
        // clamped to the range the network was trained on
        d_target = n_eigs * exp(fmin(fmax(static_cast<double>(knobs[3 * r + 0]), 0.0), log(4.0)));
        c_order = fmin(fmax(static_cast<double>(knobs[3 * r + 1]), 3.0), 24.0);
        basis_ratio = fmin(fmax(static_cast<double>(knobs[3 * r + 2]), 0.6), 3.0);
    }
    const double D = ldexp(1.0, real[r].N);
    const double* Pr = P + static_cast<int64_t>(r) * M;
    const double q = M_PI / (M + 1);
    const double cq = 1.0 / tan(q);
    auto count = [&](double ar) {
        const double phi = acos(ar);
        double tot = lane == 0 ? Pr[0] * (M_PI - 2.0 * phi) / M_PI : 0.0;   // g_0 = 1, mu_0 = P_0
        for (int j = 1 + lane; j < M; j += 32) {
            const double g = ((M - j + 1) * cos(q * j) + sin(q * j) * cq) / (M + 1);
            const double mu = 2.0 * Pr[j] - Pr[j & 1];
            tot += 2.0 * g * mu * (sin(j * (M_PI - phi)) - sin(j * phi)) / (M_PI * j);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
        return D * tot;
    };
    const double em = emax[r];
    double a;
    if (count(0.999) <= d_target) {           // a < E_max keeps E_0 > 0
        a = 0.999 * em;
    } else {
        double lo = 0.0, hi = 0.999;
        for (int it = 0; it < 100; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (count(mid) < d_target) lo = mid; else hi = mid;
        }
        a = 0.5 * (lo + hi) * em;
    }
    if (lane == 0) {
        a_out[r] = a;
        K_out[r] = static_cast<int>(ceil(c_order * em / a));
        const double n = ceil((basis_ratio * d_target / b - 1.0) / 2.0);
        n_out[r] = n < 1.0 ? 1 : static_cast<int>(n);
    }
}

cudaError_t launch_lanczos_orth(int prec, const Item* items, const RealInfo* real, int n_items, const void* v,
                                void* w, const double* lmom, int rows, int j, double* part, unsigned* real_done,
                                double* beta2, int steps, cudaStream_t st) {
    DACP_FOR_PREC(prec, lanczos_orth_kernel<T><<<n_items, kThreads, 0, st>>>(items, real, static_cast<const T*>(v),
                                                                             static_cast<T*>(w), lmom, rows, j, part,
                                                                             real_done, beta2, steps);
                        return cudaGetLastError());
    return cudaErrorInvalidValue;
}

cudaError_t launch_lanczos_scale(int prec, const Item* items, const RealInfo* real, int n_items, void* w,
                                 const double* beta2, int j, int steps, double* coef, int R, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    switch (prec) {
        case kPrecF32:
            lanczos_scale_kernel<float><<<n_items, kThreads, 0, st>>>(items, real, static_cast<float*>(w), beta2, j, steps);
            break;
        case kPrecDF32:
            lanczos_scale_kernel<df32><<<n_items, kThreads, 0, st>>>(items, real, static_cast<df32*>(w), beta2, j, steps);
            break;
        default:
            lanczos_scale_kernel<double><<<n_items, kThreads, 0, st>>>(items, real, static_cast<double*>(w), beta2, j, steps);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    lanczos_coef_kernel<<<(R + 127) / 128, 128, 0, st>>>(R, beta2, j, steps, coef);
    return cudaGetLastError();
}

cudaError_t launch_lanczos_bound(int R, const double* lmom, int rows, const double* beta2, int steps, int stride,
                                 const double* pnorm, double safety, double* emax, int rule, cudaStream_t st) {
    if (steps < 1 || steps > stride || steps > 64) return cudaErrorInvalidValue;
    lanczos_bound_kernel<<<(R + kBoundWarps - 1) / kBoundWarps, 32 * kBoundWarps, 0, st>>>(
        R, lmom, rows, beta2, steps, stride, pnorm, safety, emax, rule);
    return cudaGetLastError();
}

cudaError_t launch_kpm_window(int R, const RealInfo* real, const double* P, int M, const double* emax,
                              double d_target, double c_order, double basis_ratio, int b, const float* knobs,
                              int n_eigs, double* a_out, int* K_out, int* n_out, cudaStream_t st) {
    kpm_window_kernel<<<(R + 3) / 4, 128, 0, st>>>(R, real, P, M, emax, d_target, c_order, basis_ratio, b, knobs,
                                                   n_eigs, a_out, K_out, n_out);
    return cudaGetLastError();
}

// Features of each realization for the parameter network (kFeatures floats):
// N, log(n_eigs / 2^N), mean/std of the x-fields, mean/std of the nonzero zz
// couplings, mean/std of the z-fields, and mu_1..mu_32 of the normalised
// start vector under G = H / E_max (from the KPM rows P).
__global__ void features_kernel(int R, const RealInfo* __restrict__ real, const double* __restrict__ J,
                                const double* __restrict__ h, const double* __restrict__ g, const double* __restrict__ P,
                                int M, int n_eigs, float* __restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int N = real[r].N;
    float* o = out + static_cast<int64_t>(r) * kFeatures;
    auto stats = [](const double* v, int stride, int n, float* dst) {
        double s = 0.0, s2 = 0.0;
        for (int i = 0; i < n; ++i) { s += v[i * stride]; s2 += v[i * stride] * v[i * stride]; }
        const double mean = n > 0 ? s / n : 0.0;
        dst[0] = static_cast<float>(mean);
        dst[1] = static_cast<float>(n > 0 ? sqrt(fmax(s2 / n - mean * mean, 0.0)) : 0.0);
    };
    o[0] = static_cast<float>(N);
    o[1] = static_cast<float>(log(static_cast<double>(n_eigs)) - N * log(2.0));
    stats(g + static_cast<int64_t>(r) * kMaxSpins, 1, N, o + 2);
    const double* Jr = J + static_cast<int64_t>(r) * kMaxSpins * kMaxSpins;
    double s = 0.0, s2 = 0.0;
    int cnt = 0;
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
            const double v = Jr[i * kMaxSpins + j];
            if (v != 0.0) { s += v; s2 += v * v; ++cnt; }
        }
    const double jm = cnt ? s / cnt : 0.0;
    o[4] = static_cast<float>(jm);
    o[5] = static_cast<float>(cnt ? sqrt(fmax(s2 / cnt - jm * jm, 0.0)) : 0.0);
    stats(h + static_cast<int64_t>(r) * kMaxSpins, 1, N, o + 6);
    const double* Pr = P + static_cast<int64_t>(r) * M;
    for (int j = 1; j <= kFeatureMoments; ++j)
        o[7 + j] = j < M ? static_cast<float>(2.0 * Pr[j] - Pr[j & 1]) : 0.f;
}

cudaError_t launch_features(int R, const RealInfo* real, const double* J, const double* h, const double* g,
                            const double* P, int M, int n_eigs, float* out, cudaStream_t st) {
    features_kernel<<<(R + 63) / 64, 64, 0, st>>>(R, real, J, h, g, P, M, n_eigs, out);
    return cudaGetLastError();
}

}  // namespace dacp

// Host entry to the bound arithmetic the Lanczos kernel runs (test hook).
extern "C" dacp_status dacp_test_emax_rule(int k, const double* alpha, const double* beta2, int rule,
                                           double* bound) {
    if (k < 1 || k > 64 || !alpha || !beta2 || !bound || (rule != 0 && rule != 1)) return DACP_ERR_ARG;
    if (rule == 1) {
        *bound = dacp::ritz_rule_bound(alpha, beta2, k);
        return DACP_OK;
    }
    double gmax = 0.0;
    for (int i = 0; i < k; ++i) gmax = fmax(gmax, dacp::tridiag_gmax_row(alpha, beta2, k, i));
    const double tmin = dacp::tridiag_eig(alpha, beta2, k, 0, gmax);
    const double tmax = dacp::tridiag_eig(alpha, beta2, k, k - 1, gmax);
    *bound = fmax(fabs(tmin), fabs(tmax)) + sqrt(beta2[k - 1]);
    return DACP_OK;
}
