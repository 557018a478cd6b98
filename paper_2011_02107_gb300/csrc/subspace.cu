// Moment -> (S, H) assembly, rank cut-off and central selection kernels
// (Appendix C). The dense symmetric eigensolves and the two products
// U^T H U are cuSOLVER / cuBLAS calls issued by the host driver.

#include <math.h>

#include "common.cuh"
#include "ops.h"

namespace dacp {

// Basis orders x = [0, k_1-1, k_1, ..., k_n-1, k_n], k_m = floor(m pi / a_r) (Eq. set2).
__global__ void orders_kernel(int L, double a_r, int* __restrict__ orders) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L) return;
    if (i == 0) { orders[0] = 0; return; }
    const int m = (i + 1) / 2;
    const int km = static_cast<int>(floor(static_cast<double>(m) * M_PI / a_r));
    orders[i] = (i & 1) ? km - 1 : km;
}

// mu_j = 2 P_j - P_{j mod 2} (doubling identities), symmetrised over (p, q);
// nu_j = E_max (mu_{j+1} + mu_{|j-1|}) / 2 since H = E_max G and
// G T_j = (T_{j+1} + T_{|j-1|}) / 2. rows = 2 k_n + 2 moment rows of b x b.
// bad[0] is set when |mu_j^{pp}| exceeds mu_0^{pp} (E_max not a bound) or a
// value is not finite.
__global__ void moments_kernel(const double* __restrict__ P, int rows, int b, double emax,
                               double* __restrict__ mus, double* __restrict__ nus, int* bad) {
    const int bb = b * b;
    const int64_t n = static_cast<int64_t>(rows - 1) * bb;   // nu needs j+1 <= rows-1
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < static_cast<int64_t>(rows) * bb;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int j = static_cast<int>(e / bb);
        const int pq = static_cast<int>(e % bb);
        const int p = pq / b, q = pq % b;
        auto mu = [&](int jj, int pp, int qq) {
            return 2.0 * P[static_cast<int64_t>(jj) * bb + pp * b + qq] - P[static_cast<int64_t>(jj & 1) * bb + pp * b + qq];
        };
        const double m = 0.5 * (mu(j, p, q) + mu(j, q, p));
        mus[e] = m;
        if (!isfinite(m)) atomicOr(bad, 1);
        if (p == q) {
            const double m0 = P[p * b + p];
            // |T_j(G)| <= 1 when E_max bounds the spectrum; a violation grows
            // exponentially with j, so a loose tolerance catches it.
            if (fabs(m) > m0 * (1.0 + 1e-3) + 1e-300) atomicOr(bad, 2);
        }
        if (e < n) {
            const int jm = j >= 1 ? j - 1 : 1;
            const double a1 = 0.5 * (mu(j + 1, p, q) + mu(j + 1, q, p));
            const double a2 = 0.5 * (mu(jm, p, q) + mu(jm, q, p));
            nus[e] = emax * 0.5 * (a1 + a2);
        }
    }
}

// S_{(i,p),(j,q)} = (mu_{x_i+x_j} + mu_{|x_i-x_j|}) / 2, H likewise with nu.
// Row index i*b + p; column-major M x M (symmetric).
__global__ void assemble_kernel(int L, int b, const int* __restrict__ orders, const double* __restrict__ mus,
                                const double* __restrict__ nus, double* __restrict__ S, double* __restrict__ H,
                                int ld) {
    const int M = L * b;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int col = blockIdx.y;
    if (row >= M || col >= M) return;
    const int i = row / b, p = row % b;
    const int j = col / b, q = col % b;
    const int xi = orders[i], xj = orders[j];
    const int ks = xi + xj;
    const int kd = xi > xj ? xi - xj : xj - xi;
    const int bb = b * b;
    const int64_t e1 = static_cast<int64_t>(ks) * bb + p * b + q;
    const int64_t e2 = static_cast<int64_t>(kd) * bb + p * b + q;
    const int64_t o = static_cast<int64_t>(col) * ld + row;
    S[o] = 0.5 * (mus[e1] + mus[e2]);
    H[o] = 0.5 * (nus[e1] + nus[e2]);
}

// Rank cut-off on the ascending eigenvalues lam of S: keep lam > eps * lam_max
// (relative) -- m columns, the last m of V -- and scale them by lam^{-1/2}
// (U = V~ Lam~^{-1/2}, Appendix C). Single CTA.
__global__ void cutoff_kernel(const double* __restrict__ lam, int M, double eps, int absolute,
                              double* __restrict__ V, int* m_out) {
    __shared__ int first_s;
    const double lmax = lam[M - 1];
    const double thr = absolute ? eps : eps * lmax;
    if (threadIdx.x == 0) {
        int lo = 0, hi = M;          // first index with lam > thr
        while (lo < hi) {
            const int mid = (lo + hi) / 2;
            if (lam[mid] > thr) hi = mid; else lo = mid + 1;
        }
        first_s = lo;
        *m_out = M - lo;
    }
    __syncthreads();
    const int f = first_s;
    for (int c = f + blockIdx.y; c < M; c += gridDim.y) {
        const double sc = 1.0 / sqrt(lam[c]);
        for (int rr = threadIdx.x; rr < M; rr += blockDim.x) V[static_cast<int64_t>(c) * M + rr] *= sc;
    }
}

// n_eigs eigenvalues of smallest |E| inside [-w, w] from ascending lam[0..m),
// written ascending; ties in |E| go to the lower index (the negative value).
__global__ void select_kernel(const double* __restrict__ lam, int m, int n_eigs, double w,
                              double* __restrict__ out, int* n_found) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int lo = 0, hi = m;
    while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (lam[mid] >= 0.0) hi = mid; else lo = mid + 1;
    }
    int l = lo - 1, h = lo, cnt = 0;
    while (cnt < n_eigs) {
        const bool okl = l >= 0 && fabs(lam[l]) <= w;
        const bool okh = h < m && fabs(lam[h]) <= w;
        if (!okl && !okh) break;
        if (okl && (!okh || fabs(lam[l]) <= fabs(lam[h]))) --l; else ++h;
        ++cnt;
    }
    for (int t = 0; t < cnt; ++t) out[t] = lam[l + 1 + t];
    *n_found = cnt;
}

// Batched variant helpers. For realization i of a group: zero the columns
// [M - m_max, M - m_i) of V_i (dropped directions inside the common width),
// and put `big` on the first m_max - m_i diagonal entries of H~_i (their rows
// and columns are zero, so those eigenvalues are exactly `big`, outside every
// window).
__global__ void pad_columns_kernel(double* __restrict__ V, int M, int64_t strideV, const int* __restrict__ m, int m_max) {
    const int i = blockIdx.y;
    double* Vi = V + strideV * i;
    const int c0 = M - m_max, c1 = M - m[i];
    for (int c = c0 + blockIdx.x; c < c1; c += gridDim.x)
        for (int rr = threadIdx.x; rr < M; rr += blockDim.x) Vi[static_cast<int64_t>(c) * M + rr] = 0.0;
}

__global__ void pad_diagonal_kernel(double* __restrict__ Ht, int m_max, int64_t strideH, const int* __restrict__ m,
                                    const double* __restrict__ big) {
    const int i = blockIdx.x;
    double* Hi = Ht + strideH * i;
    for (int t = threadIdx.x; t < m_max - m[i]; t += blockDim.x) Hi[static_cast<int64_t>(t) * m_max + t] = big[i];
}

cudaError_t launch_pad_columns(double* V, int M, int64_t strideV, const int* m, int m_max, int count, cudaStream_t st) {
    dim3 grid(64, count);
    pad_columns_kernel<<<grid, 256, 0, st>>>(V, M, strideV, m, m_max);
    return cudaGetLastError();
}

cudaError_t launch_pad_diagonal(double* Ht, int m_max, int64_t strideH, const int* m, const double* big, int count,
                                cudaStream_t st) {
    pad_diagonal_kernel<<<count, 256, 0, st>>>(Ht, m_max, strideH, m, big);
    return cudaGetLastError();
}

// <psi| H^2 T_k |psi> = E_max^2 <psi| G^2 T_k |psi>, with
// G^2 T_k = (T_{k+2} + T_k + T_{|k-1|+1} + T_{||k-1|-1|}) / 4 (two uses of
// G T_j = (T_{j+1} + T_{|j-1|}) / 2); mus holds the symmetrised mu rows.
__global__ void omega_kernel(const double* __restrict__ mus, int rows_out, int b, double emax,
                             double* __restrict__ om) {
    const int bb = b * b;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < static_cast<int64_t>(rows_out) * bb;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int k = static_cast<int>(e / bb);
        const int pq = static_cast<int>(e % bb);
        const int k1 = k >= 1 ? k - 1 : 1;               // |k-1|
        const int k2 = k1 >= 1 ? k1 - 1 : 1;             // ||k-1|-1|
        const double v = mus[static_cast<int64_t>(k + 2) * bb + pq] + mus[static_cast<int64_t>(k) * bb + pq] +
                         mus[static_cast<int64_t>(k1 + 1) * bb + pq] + mus[static_cast<int64_t>(k2) * bb + pq];
        om[e] = emax * emax * 0.25 * v;
    }
}

// Index range [first, first + count) of the selected levels in ascending lam.
__global__ void select_range_kernel(const double* __restrict__ lam, int m, int n_eigs, double w, int* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int lo = 0, hi = m;
    while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (lam[mid] >= 0.0) hi = mid; else lo = mid + 1;
    }
    int l = lo - 1, h = lo, cnt = 0;
    while (cnt < n_eigs) {
        const bool okl = l >= 0 && fabs(lam[l]) <= w;
        const bool okh = h < m && fabs(lam[h]) <= w;
        if (!okl && !okh) break;
        if (okl && (!okh || fabs(lam[l]) <= fabs(lam[h]))) --l; else ++h;
        ++cnt;
    }
    out[0] = l + 1;
    out[1] = cnt;
}

// resid_j = sqrt(max(0, b_j^T (H^2 b_j) - lam_j^2)); one CTA per column j.
__global__ void residual_kernel(const double* __restrict__ Bsel, const double* __restrict__ W2, int M,
                                const double* __restrict__ lam, double* __restrict__ resid) {
    __shared__ double red[256];
    const int j = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < M; i += blockDim.x)
        s += Bsel[static_cast<int64_t>(j) * M + i] * W2[static_cast<int64_t>(j) * M + i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) resid[j] = sqrt(fmax(0.0, red[0] - lam[j] * lam[j]));
}

cudaError_t launch_omega(const double* mus, int rows_out, int b, double emax, double* om, cudaStream_t st) {
    const int64_t n = static_cast<int64_t>(rows_out) * b * b;
    const int grid = static_cast<int>((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    omega_kernel<<<grid, 256, 0, st>>>(mus, rows_out, b, emax, om);
    return cudaGetLastError();
}

cudaError_t launch_select_range(const double* lam, int m, int n_eigs, double w, int* out, cudaStream_t st) {
    select_range_kernel<<<1, 32, 0, st>>>(lam, m, n_eigs, w, out);
    return cudaGetLastError();
}

cudaError_t launch_residual(const double* Bsel, const double* W2, int M, int count, const double* lam, double* resid,
                            cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    residual_kernel<<<count, 256, 0, st>>>(Bsel, W2, M, lam, resid);
    return cudaGetLastError();
}

cudaError_t launch_orders(int L, double a_r, int* orders, cudaStream_t st) {
    orders_kernel<<<(L + 255) / 256, 256, 0, st>>>(L, a_r, orders);
    return cudaGetLastError();
}

cudaError_t launch_moments(const double* P, int rows, int b, double emax, double* mus, double* nus, int* bad,
                           cudaStream_t st) {
    const int64_t n = static_cast<int64_t>(rows) * b * b;
    const int grid = static_cast<int>((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    moments_kernel<<<grid, 256, 0, st>>>(P, rows, b, emax, mus, nus, bad);
    return cudaGetLastError();
}

cudaError_t launch_assemble(int L, int b, const int* orders, const double* mus, const double* nus, double* S,
                            double* H, cudaStream_t st, int ld) {
    const int M = L * b;
    dim3 grid((M + 127) / 128, M);
    assemble_kernel<<<grid, 128, 0, st>>>(L, b, orders, mus, nus, S, H, ld > 0 ? ld : M);
    return cudaGetLastError();
}

cudaError_t launch_cutoff(const double* lam, int M, double eps, int absolute, double* V, int* m_out,
                          cudaStream_t st) {
    dim3 grid(1, M < 1024 ? M : 1024);
    // one CTA column-group; every CTA repeats the tiny binary search
    cutoff_kernel<<<grid, 256, 0, st>>>(lam, M, eps, absolute, V, m_out);
    return cudaGetLastError();
}

cudaError_t launch_select(const double* lam, int m, int n_eigs, double w, double* out, int* n_found,
                          cudaStream_t st) {
    select_kernel<<<1, 32, 0, st>>>(lam, m, n_eigs, w, out, n_found);
    return cudaGetLastError();
}

// Residual norms |H y_j - theta_j y_j| of Ritz pairs, from HY = H V Z and Y = V Z (column-major,
// columns of length D): one block per column, float64 sums reduced over the block.
__global__ void ritz_residual_kernel(const double* __restrict__ HY, const double* __restrict__ Y,
                                     const double* __restrict__ th, int64_t D, double* __restrict__ res) {
    __shared__ double red[256 / 32];
    const int j = blockIdx.x;
    const double t = th[j];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < D; i += blockDim.x) {
        const double d = HY[j * D + i] - t * Y[j * D + i];
        s = fma(d, d, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < 256 / 32; ++w) tot += red[w];
        res[j] = sqrt(tot);
    }
}

// The Ritz values whose residual is at most tol, in their (ascending) order.
__global__ void compact_converged_kernel(const double* __restrict__ th, const double* __restrict__ res, int m,
                                         double tol, double* __restrict__ out, int* __restrict__ count) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int c = 0;
    for (int j = 0; j < m; ++j)
        if (res[j] <= tol) out[c++] = th[j];
    *count = c;
}

cudaError_t launch_ritz_residual(const double* HY, const double* Y, const double* th, int64_t D, int m, double* res,
                                 cudaStream_t st) {
    if (m < 1) return cudaSuccess;
    ritz_residual_kernel<<<m, 256, 0, st>>>(HY, Y, th, D, res);
    return cudaGetLastError();
}

cudaError_t launch_compact_converged(const double* th, const double* res, int m, double tol, double* out, int* count,
                                     cudaStream_t st) {
    compact_converged_kernel<<<1, 32, 0, st>>>(th, res, m, tol, out, count);
    return cudaGetLastError();
}

}  // namespace dacp
