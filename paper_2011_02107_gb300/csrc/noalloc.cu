// Allocation-free Chebyshev moments: dacp_moments_noalloc.
//
// Some callers cannot call cudaMalloc: engines whose device memory all
// belongs to their own pool or arena, and latency-critical loops that forbid
// allocator calls. For them this entry point runs the float64 evolution
// stencil (H.v fused with the Chebyshev recurrence and the moment sums) for
// one realization without allocating anything: its working vectors,
// diagonal, couplings, partial sums and counters live in one file-scope
// device array, and the caller passes only the input vector and the output
// moments. The call copies its small host inputs into the array on the
// caller's stream and waits for that stream before it returns.
//
// The array holds at most kMaxSpins states' worth of scratch, so N <= 16. It
// is loaded with the library and every GPU that loads it keeps it until the
// process exits. Its address is looked up once per device, on that device's
// first call, and cached.

#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "../../include/dacp.h"
#include "common.cuh"
#include "ops.h"

namespace dacp {
namespace {

constexpr int kNaMaxSpins = 16;                           // N limit of this entry point
constexpr int64_t kNaStates = int64_t(1) << kNaMaxSpins;
constexpr int kNaTileStates = 8192;                       // 64 KB float64 tiles
constexpr int kNaMaxItems = int(kNaStates / kNaTileStates);

// Layout of the scratch array, in doubles (every region 256-byte aligned).
constexpr int64_t kRegA = 0;                              // w_k / w_{k+1}
constexpr int64_t kRegB = kRegA + kNaStates;              // w_{k-1}
constexpr int64_t kRegDiag = kRegB + kNaStates;           // diagonal of H
constexpr int64_t kRegGam = kRegDiag + kNaStates;         // x-fields [kMaxSpins]
constexpr int64_t kRegJ = kRegGam + 32;                   // zz couplings [kMaxSpins][kMaxSpins]
constexpr int64_t kRegH = kRegJ + 704;                    // z-fields [kMaxSpins]
constexpr int64_t kRegCoef = kRegH + 32;                  // recurrence coefficients [8]
constexpr int64_t kRegPart = kRegCoef + 32;               // per-tile moment partials [items][2]
constexpr int64_t kRegInfo = kRegPart + 2 * kNaMaxItems + 32;   // RealInfo
constexpr int64_t kRegItems = kRegInfo + 32;              // Item[kNaMaxItems]
constexpr int64_t kRegCount = kRegItems + kNaMaxItems + 32;     // counters (unsigned / int)
constexpr int64_t kNaTotal = kRegCount + 32;

static_assert(sizeof(RealInfo) <= 32 * sizeof(double), "RealInfo region too small");
static_assert(sizeof(Item) * kNaMaxItems <= (kNaMaxItems + 32) * sizeof(double), "Item region too small");

// The scratch. In host code this name is only a stand-in for the device
// array: host code must use the address from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[kNaTotal];

std::mutex g_na_mu;
double* g_na_ptr[128] = {};   // device address of the scratch, per device

// mu_j = 2 P_j - P_{j mod 2} in place (j >= 2 reads only P_0 and P_1, which stay).
__global__ void noalloc_moments_from_products(double* mu, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= 2 && j < n) mu[j] = 2.0 * mu[j] - mu[j & 1];
}

}  // namespace
}  // namespace dacp

using namespace dacp;

extern "C" dacp_status dacp_moments_noalloc(int n_spins, const double* J, const double* h, const double* gamma,
                                            double emax, const double* psi_dev, int n_orders, double* mu_dev,
                                            void* stream) {
    if (n_spins < 1 || n_spins > kNaMaxSpins) return DACP_ERR_ARG;      // beyond the scratch array
    if (!J || !h || !gamma || !psi_dev || !mu_dev || !(emax > 0.0) || !isfinite(emax) || n_orders < 1 ||
        n_orders > (1 << 28))
        return DACP_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return DACP_ERR_CUDA;

    // Set-up, once per device, with that device current: the scratch address
    // and the shared-memory attribute of the stencil kernel.
    double* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DACP_ERR_CUDA;
            if (prepare_step(kPrecF64, 1, kNaTileStates * static_cast<int>(sizeof(double))) != cudaSuccess)
                return DACP_ERR_CUDA;
            g_na_ptr[dev] = static_cast<double*>(p);
        }
        base = g_na_ptr[dev];
    }

    const int N = n_spins;
    const int64_t D = int64_t(1) << N;
    RealInfo R;
    memset(&R, 0, sizeof(R));
    R.N = N;
    R.tbits = N < 13 ? N : 13;
    R.off = 0;
    R.item_begin = 0;
    R.item_count = 1 << (N - R.tbits);
    R.nf = 0;
    R.ne = n_orders;
    R.mom_off = 0;
    Item items[kNaMaxItems];
    for (int t = 0; t < R.item_count; ++t) items[t] = Item{0, t};
    double Jp[kMaxSpins * kMaxSpins];
    double hp[kMaxSpins], gp[kMaxSpins];
    memset(Jp, 0, sizeof(Jp));
    memset(hp, 0, sizeof(hp));
    memset(gp, 0, sizeof(gp));
    for (int i = 0; i < N; ++i) {
        hp[i] = h[i];
        gp[i] = gamma[i];
        for (int j = i + 1; j < N; ++j) Jp[i * kMaxSpins + j] = J[i * N + j];
    }
    // order 0: w_1 = G psi; then w_{k+1} = 2 G w_k - w_{k-1}, G = H / E_max
    const double coef[8] = {1.0 / emax, 0.0, 0.0, 2.0 / emax, -1.0, 0.0, 0.0, 0.0};

    unsigned* counters = reinterpret_cast<unsigned*>(base + kRegCount);   // real_done, launch_done, step, err, bar[2]
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    // Calls share the array and it keeps the last call's contents: everything
    // read before it is written is set again here, counters cleared to zero.
    bool good = ok(cudaMemcpyAsync(base + kRegInfo, &R, sizeof(R), cudaMemcpyHostToDevice, st)) &&
                ok(cudaMemcpyAsync(base + kRegItems, items, sizeof(Item) * R.item_count, cudaMemcpyHostToDevice, st)) &&
                ok(cudaMemcpyAsync(base + kRegJ, Jp, sizeof(Jp), cudaMemcpyHostToDevice, st)) &&
                ok(cudaMemcpyAsync(base + kRegH, hp, sizeof(hp), cudaMemcpyHostToDevice, st)) &&
                ok(cudaMemcpyAsync(base + kRegGam, gp, sizeof(gp), cudaMemcpyHostToDevice, st)) &&
                ok(cudaMemcpyAsync(base + kRegCoef, coef, sizeof(coef), cudaMemcpyHostToDevice, st)) &&
                ok(cudaMemsetAsync(counters, 0, 8 * sizeof(unsigned), st)) &&
                ok(cudaMemcpyAsync(base + kRegA, psi_dev, sizeof(double) * D, cudaMemcpyDeviceToDevice, st));
    if (!good) return DACP_ERR_CUDA;
    const RealInfo* info_d = reinterpret_cast<const RealInfo*>(base + kRegInfo);
    if (launch_diag(kPrecF64, info_d, 0, N, base + kRegJ, base + kRegH, base + kRegDiag, st) != cudaSuccess)
        return DACP_ERR_CUDA;

    StepArgs a;
    memset(&a, 0, sizeof(a));
    a.items = reinterpret_cast<const Item*>(base + kRegItems);
    a.real = info_d;
    a.diag = base + kRegDiag;
    a.gam = base + kRegGam;
    a.coef = base + kRegCoef;
    a.bufA = base + kRegA;
    a.bufB = base + kRegB;
    a.bufU = base + kRegB;
    a.real_done = counters + 0;
    a.launch_done = counters + 1;
    a.step_ctr = reinterpret_cast<int*>(counters + 2);
    a.err_flag = reinterpret_cast<int*>(counters + 3);
    a.bar_count = counters + 4;
    a.bar_gen = counters + 5;
    a.part = base + kRegPart;
    a.mom = mu_dev;                      // product rows P_0 .. P_{2 n_orders - 1}
    const int smem = (1 << R.tbits) * static_cast<int>(sizeof(double));
    for (int k = 0; k < n_orders; ++k)
        if (launch_step(kPrecF64, 1, kEvolve, a, 0, R.item_count, smem, st) != cudaSuccess) return DACP_ERR_CUDA;
    const int n = 2 * n_orders;
    noalloc_moments_from_products<<<(n + 255) / 256, 256, 0, st>>>(mu_dev, n);
    if (cudaGetLastError() != cudaSuccess) return DACP_ERR_CUDA;
    int err = 0;
    if (!ok(cudaMemcpyAsync(&err, counters + 3, sizeof(int), cudaMemcpyDeviceToHost, st)) ||
        !ok(cudaStreamSynchronize(st)))
        return DACP_ERR_CUDA;
    return err ? DACP_ERR_TIMEOUT : DACP_OK;
}
