// C ABI of the DACP library: handle, parameter set-up, the two Chebyshev
// recurrences (graph-replayed fused stencil launches) and the float64
// subspace solve. Declarations and documentation: include/dacp.h.

#include <cublas_v2.h>
#include <cusolverDn.h>
#include <math.h>
#include <nvtx3/nvToolsExt.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <functional>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "../../include/dacp.h"
#include "common.cuh"
#include "ops.h"

using namespace dacp;

namespace {

constexpr int kGraphOrders = 32;   // orders per captured graph
constexpr int kMinTileBytes = 8192; // smallest tile the autotuner tries
constexpr int kMaxLanes = 16;      // concurrent subspace solves
constexpr double kLaneBytes = 24e9;  // device memory budget of the lanes
// Float32 vectors: round-off in the recurrence leaves a noise floor near
// 1e-5 of the largest moment, so the rank cut-off rises to 1e-6 (relative)
// and the filter order constant drops from 18 to 6: e^{2c} then matches the
// dynamic range float32 moments resolve, and the requested levels keep
// weights above the noise (measured on N=10..14 shards against dense eigh).
constexpr double kEpsFp32 = 1e-6;
constexpr double kCOrderFp32 = 6.0;
constexpr double kCOrderFp64 = 18.0;
// Double-float vectors carry about 2^-44 relative round-off per operation:
// the float64 filter constant holds, the cut-off sits a decade above 1e-12.
constexpr double kEpsDf32 = 1e-11;

struct Graph {
    cudaGraphExec_t exec = nullptr;
    int mode = -1;
};

}  // namespace

// One concurrent subspace-solve lane: its own stream, library handles and
// workspace, so that independent realizations' eigensolves overlap.
struct Lane {
    cudaStream_t st = nullptr;
    cusolverDnHandle_t sol = nullptr;
    cublasHandle_t blas = nullptr;
    cusolverDnParams_t sp = nullptr;
    cudaEvent_t done = nullptr;
    double *S = nullptr, *H = nullptr, *W = nullptr, *Ht = nullptr, *lam = nullptr, *lamt = nullptr;
    double *mus = nullptr, *nus = nullptr, *sel = nullptr;
    int *orders = nullptr, *mi = nullptr, *bad = nullptr, *info = nullptr, *nf = nullptr;
    void* work = nullptr;
    size_t dbytes = 0, hbytes = 0;
    std::vector<char> work_h;
    std::vector<double> out_h;
    int hv[3] = {0, 0, 0};
    int cnt = -1;
    int r = -1;
};

struct dacp_ctx {
    int R = 0, b = 1;
    int prec = kPrecF64;                // vector precision (kPrecF64 / kPrecF32 / kPrecDF32)
    bool fp32 = false;
    size_t esz = 8;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int device = 0;
    std::vector<int> N;
    std::vector<RealInfo> info;
    std::vector<Item> items;
    int64_t Dtot = 0;
    int smem = 0;
    int tile_bytes = 0;
    int tb_uniform = 0;                 // tile bits shared by every realization, else 0
    std::vector<double> J_h, h_h, g_h;   // [R][kMaxSpins(^2)]
    std::vector<double> pnorm;          // Pauli 1-norm of each H: clamp of the E_max bound
    std::vector<double> pnorm0;         // the same without the pair couplings
    bool has_pairs = false;             // dacp_set_pair_couplings gave nonzero XX / YY terms
    std::vector<double> jxx_h, jyy_h;   // the caller's pair couplings (packed as given), for re-runs
    std::vector<double> pnorm_pairs;    // sum |Jxx| + |Jyy| of each realization
    std::vector<double> gflip_h;        // coefficient of the global flip X_0 ... X_{N-1} per realization
    bool has_gflip = false;
    bool sector_pairs = false;          // dacp_create_parity_sectors: realizations 2m, 2m+1 are model m's sectors
    double* gflip_d = nullptr;          // [R]
    std::vector<double> psi0_h;         // the caller's start vectors (packed float64), for re-runs
    int* n_pairs_d = nullptr;           // [R]
    int* pair_ij_d = nullptr;           // [R][kMaxPairs]
    double* pair_c_d = nullptr;         // [R][kMaxPairs][2]

    // device
    std::vector<void*> allocs;
    RealInfo* info_d = nullptr;
    Item* items_d = nullptr;
    double *J_d = nullptr, *h_d = nullptr, *g64_d = nullptr, *pnorm_d = nullptr;
    float* feats_d = nullptr;
    void *gam_d = nullptr, *diag_d = nullptr;
    void *psi0_d = nullptr, *A_d = nullptr, *B_d = nullptr, *U_d = nullptr, *psiE_d = nullptr;
    double *coef_d = nullptr, *apply_coef_d = nullptr, *part_d = nullptr, *norms_d = nullptr;
    unsigned *real_done_d = nullptr, *launch_done_d = nullptr;
    int* step_ctr_d = nullptr;
    int* err_d = nullptr;               // set by a stencil CTA whose bounded wait gave up
    unsigned* bar_d = nullptr;          // grid barrier (count, generation) of the persistent launch
    int launch_mode = 0;                // 0: per-order launches replayed from a CUDA graph, 1: persistent,
                                        // 2: as 0 with every HBM read of a tile staged (float32 only)
    bool poison_barrier = false;        // test hook: the next persistent launch's barrier never opens
    bool batched_solve = true;          // equal basis sizes: batched cuSOLVER instead of lanes
    int emax_rule = 0;                  // E_max bound: 0 Ritz value + residual norm, 1 Ritz-residual rule
    double* mom_d = nullptr;
    int64_t mom_cap = 0;

    // parameters
    std::vector<double> emax, a;
    std::vector<int> K, n, kn;
    int state = 0;                      // 0 created, 1 params, 2 filtered, 3 moments
    std::vector<int> bad;               // per realization numeric failure after moments

    // subspace workspace
    cusolverDnHandle_t sol = nullptr;
    cublasHandle_t blas = nullptr;
    cusolverDnParams_t sp = nullptr;

    // second solver (stream + handles) that overlaps subspace solves with the evolution
    cudaStream_t st2 = nullptr;
    cusolverDnHandle_t sol2 = nullptr;
    cublasHandle_t blas2 = nullptr;
    cusolverDnParams_t sp2 = nullptr;

    std::vector<Lane> lanes;
    int lane_M = 0, lane_neigs = 0;
    int64_t lane_rows = 0;

    Graph gf, ge;
    cudaEvent_t ev[6] = {};
    double t_ms[3] = {0, 0, 0};
    std::atomic<int64_t> launches{0};   // kernels of this library launched so far
    std::string err;
};

namespace {

std::mutex g_err_mu;   // lanes may report failures from several host threads

dacp_status fail(dacp_ctx* c, dacp_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) {
        std::lock_guard<std::mutex> lk(g_err_mu);
        c->err = buf;
    }
    return s;
}

#define CK(call)                                                                                        \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return fail(c, e_ == cudaErrorMemoryAllocation ? DACP_ERR_NOMEM : DACP_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                             \
    } while (0)

#define CKS(call)                                                                                       \
    do {                                                                                                \
        cusolverStatus_t e_ = (call);                                                                   \
        if (e_ != CUSOLVER_STATUS_SUCCESS)                                                              \
            return fail(c, DACP_ERR_LIBRARY, "%s: cusolver status %d (%s:%d)", #call, (int)e_, __FILE__, __LINE__); \
    } while (0)

#define CKB(call)                                                                                       \
    do {                                                                                                \
        cublasStatus_t e_ = (call);                                                                     \
        if (e_ != CUBLAS_STATUS_SUCCESS)                                                                \
            return fail(c, DACP_ERR_LIBRARY, "%s: cublas status %d (%s:%d)", #call, (int)e_, __FILE__, __LINE__); \
    } while (0)

#define TRY(expr)                                 \
    do {                                          \
        dacp_status s_ = (expr);                  \
        if (s_ != DACP_OK) return s_;             \
    } while (0)

// NVTX range over one library call (T_F / T_E / T_D and the rest show by name on an
// Nsight timeline; without a tool attached a push / pop costs a few nanoseconds).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Allocation-failure injection (dacp_test_fail_alloc): the number of device allocations still to
// succeed before one fails; negative = off. Process-wide, so that dacp_create can be reached too.
static std::atomic<int64_t> g_alloc_countdown{-1};

dacp_status dalloc(dacp_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    for (int64_t left = g_alloc_countdown.load(); left >= 0;) {
        if (g_alloc_countdown.compare_exchange_weak(left, left - 1)) {
            if (left == 0) return fail(c, DACP_ERR_NOMEM, "injected allocation failure (%zu bytes)", bytes);
            break;
        }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, DACP_ERR_NOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    c->allocs.push_back(*p);
    return DACP_OK;
}

template <typename T>
dacp_status dalloc_t(dacp_ctx* c, T** p, size_t count) {
    void* v = nullptr;
    dacp_status s = dalloc(c, &v, count * sizeof(T));
    *p = static_cast<T*>(v);
    return s;
}

void dfree(dacp_ctx* c, void* p) {
    if (!p) return;
    auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
    if (it != c->allocs.end()) c->allocs.erase(it);
    cudaFree(p);
}

void free_lanes(dacp_ctx* c) {
    for (auto& L : c->lanes) {
        if (L.st) cudaStreamSynchronize(L.st);
        for (void* p : {static_cast<void*>(L.S), static_cast<void*>(L.H), static_cast<void*>(L.W),
                        static_cast<void*>(L.Ht), static_cast<void*>(L.lam), static_cast<void*>(L.lamt),
                        static_cast<void*>(L.mus), static_cast<void*>(L.nus), static_cast<void*>(L.sel),
                        static_cast<void*>(L.orders), static_cast<void*>(L.mi), static_cast<void*>(L.bad),
                        static_cast<void*>(L.info), static_cast<void*>(L.nf), L.work})
            dfree(c, p);
        if (L.sp) cusolverDnDestroyParams(L.sp);
        if (L.sol) cusolverDnDestroy(L.sol);
        if (L.blas) cublasDestroy(L.blas);
        if (L.done) cudaEventDestroy(L.done);
        if (L.st) cudaStreamDestroy(L.st);
    }
    c->lanes.clear();
    c->lane_M = 0;
    c->lane_rows = 0;
    c->lane_neigs = 0;
}

// Lanes able to solve problems of order <= M with <= rows moment rows.
dacp_status ensure_lanes(dacp_ctx* c, int M, int64_t rows, int n_eigs) {
    if (!c->lanes.empty() && M <= c->lane_M && rows <= c->lane_rows && n_eigs <= c->lane_neigs) return DACP_OK;
    free_lanes(c);
    const double per_lane = 4.0 * 8.0 * M * static_cast<double>(M) + 2.0 * 8.0 * rows * c->b * c->b;
    int nl = std::min(c->R, kMaxLanes);
    nl = std::max(1, std::min(nl, static_cast<int>(kLaneBytes / std::max(per_lane, 1.0))));
    c->lanes.resize(nl);
    const size_t MM = static_cast<size_t>(M) * M;
    for (auto& L : c->lanes) {
        CK(cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming));
        CKS(cusolverDnCreate(&L.sol));
        CKS(cusolverDnSetStream(L.sol, L.st));
        CKS(cusolverDnCreateParams(&L.sp));
        CKB(cublasCreate(&L.blas));
        CKB(cublasSetStream(L.blas, L.st));
        TRY(dalloc_t(c, &L.S, MM));
        TRY(dalloc_t(c, &L.H, MM));
        TRY(dalloc_t(c, &L.W, MM));
        TRY(dalloc_t(c, &L.Ht, MM));
        TRY(dalloc_t(c, &L.lam, M));
        TRY(dalloc_t(c, &L.lamt, M));
        TRY(dalloc_t(c, &L.mus, static_cast<size_t>(rows) * c->b * c->b));
        TRY(dalloc_t(c, &L.nus, static_cast<size_t>(rows) * c->b * c->b));
        TRY(dalloc_t(c, &L.sel, static_cast<size_t>(std::max(n_eigs, 1))));
        TRY(dalloc_t(c, &L.orders, M));
        TRY(dalloc_t(c, &L.mi, 4));
        TRY(dalloc_t(c, &L.bad, 1));
        TRY(dalloc_t(c, &L.info, 1));
        TRY(dalloc_t(c, &L.nf, 1));
        CKS(cusolverDnXsyevd_bufferSize(L.sol, L.sp, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, M, CUDA_R_64F,
                                        L.S, M, CUDA_R_64F, L.lam, CUDA_R_64F, &L.dbytes, &L.hbytes));
        TRY(dalloc(c, &L.work, L.dbytes));
        L.work_h.resize(std::max<size_t>(L.hbytes, 1));
        L.out_h.resize(std::max(n_eigs, 1));
    }
    c->lane_M = M;
    c->lane_rows = rows;
    c->lane_neigs = n_eigs;
    return DACP_OK;
}

StepArgs base_args(dacp_ctx* c) {
    StepArgs a;
    memset(&a, 0, sizeof(a));
    a.items = c->items_d;
    a.real = c->info_d;
    a.diag = c->diag_d;
    a.gam = c->gam_d;
    a.coef = c->coef_d;
    a.bufA = c->A_d;
    a.bufB = c->B_d;
    a.bufU = c->U_d;
    a.step_ctr = c->step_ctr_d;
    a.launch_done = c->launch_done_d;
    a.real_done = c->real_done_d;
    a.part = c->part_d;
    a.mom = c->mom_d;
    a.err_flag = c->err_d;
    a.bar_count = c->bar_d;
    a.bar_gen = c->bar_d + 1;
    // the kernels specialised on a uniform tile size carry no pair terms
    a.tbits_uniform = c->has_pairs ? 0 : c->tb_uniform;
    if (c->has_pairs) {
        a.n_pairs = c->n_pairs_d;
        a.pair_ij = c->pair_ij_d;
        a.pair_c = c->pair_c_d;
    }
    if (c->has_gflip) a.gflip = c->gflip_d;
    return a;
}

// Launch `orders` Chebyshev orders of the filter (two stencil passes each) or of
// the evolution (one pass each) on the handle stream. A graph of kGraphOrders
// orders is captured once and replayed; realizations whose run is shorter
// skip the surplus orders inside the kernel.
dacp_status run_orders(dacp_ctx* c, bool filter, int orders,
                       const std::function<dacp_status(int)>& after = std::function<dacp_status(int)>()) {
    if (orders <= 0) return DACP_OK;
    CK(cudaMemsetAsync(c->step_ctr_d, 0, sizeof(int), c->st));
    const StepArgs a = base_args(c);
    const int ni = static_cast<int>(c->items.size());
    if (c->launch_mode == 1) {
        // every order in one cooperative launch with a bounded grid barrier
        // a poisoned arrival count can never reach gridDim - 1: every CTA's bounded wait runs out
        CK(cudaMemsetAsync(c->bar_d, c->poison_barrier ? 0x40 : 0, sizeof(unsigned), c->st));
        CK(cudaMemsetAsync(c->bar_d + 1, 0, sizeof(unsigned), c->st));
        c->poison_barrier = false;
        int grid = 0;
        CK(launch_persistent(c->prec, c->b, filter ? 0 : 1, a, ni, orders, c->smem, c->st, &grid));
        c->launches += 1;
        if (after) TRY(after(orders));
        return DACP_OK;
    }
    auto pass = [&](int mode) -> cudaError_t {
        return c->launch_mode == 2 ? launch_step_staged(c->b, mode, a, 0, ni, c->smem, c->st)
                                   : launch_step(c->prec, c->b, mode, a, 0, ni, c->smem, c->st);
    };
    auto launch_order = [&]() -> cudaError_t {
        cudaError_t e;
        if (filter) {
            if ((e = pass(kFilter1)) != cudaSuccess) return e;
            return pass(kFilter2);
        }
        return pass(kEvolve);
    };
    Graph& g = filter ? c->gf : c->ge;
    if (!g.exec && orders >= kGraphOrders) {
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
        cudaError_t le = cudaSuccess;
        for (int i = 0; i < kGraphOrders && le == cudaSuccess; ++i) le = launch_order();
        cudaError_t ee = cudaStreamEndCapture(c->st, &graph);
        if (le != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(c, DACP_ERR_CUDA, "stencil launch during capture: %s", cudaGetErrorString(le));
        }
        CK(ee);
        cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(ie);
    }
    int done = 0;
    if (g.exec) {
        for (; done + kGraphOrders <= orders; done += kGraphOrders) {
            CK(cudaGraphLaunch(g.exec, c->st));
            c->launches += kGraphOrders * (filter ? 2 : 1);
            if (after) TRY(after(done + kGraphOrders));
        }
    }
    for (; done < orders; ++done) {
        CK(launch_order());
        c->launches += filter ? 2 : 1;
        if (after) TRY(after(done + 1));
    }
    return DACP_OK;
}

// Work decomposition: tiles of at most tile_bytes of the vector per CTA.
void tile_geometry(dacp_ctx* c, int tile_bytes) {
    int tb_cap = 0;
    while ((static_cast<int64_t>(2) << tb_cap) * c->b * static_cast<int64_t>(c->esz) <= tile_bytes) ++tb_cap;
    c->items.clear();
    int max_tstates = 1;
    for (int r = 0; r < c->R; ++r) {
        RealInfo& R = c->info[r];
        R.tbits = std::min(R.N, tb_cap);
        R.item_begin = static_cast<int>(c->items.size());
        R.item_count = 1 << (R.N - R.tbits);
        for (int t = 0; t < R.item_count; ++t) c->items.push_back(Item{r, t});
        max_tstates = std::max(max_tstates, 1 << R.tbits);
    }
    c->smem = static_cast<int>(max_tstates * c->b * c->esz);
    c->tile_bytes = tile_bytes;
    c->tb_uniform = c->R > 0 ? c->info[0].tbits : 0;
    for (int r = 1; r < c->R; ++r)
        if (c->info[r].tbits != c->tb_uniform) c->tb_uniform = 0;
}

// Partial-sum slots for the smallest tile the autotuner may pick.
size_t part_capacity(const dacp_ctx* c) {
    int64_t worst = 0;
    for (int r = 0; r < c->R; ++r) {
        int tb = 0;
        while ((static_cast<int64_t>(2) << tb) * c->b * static_cast<int64_t>(c->esz) <= kMinTileBytes) ++tb;
        worst += static_cast<int64_t>(1) << (c->info[r].N - std::min(c->info[r].N, tb));
    }
    return static_cast<size_t>(std::max<int64_t>(worst, 1)) * 2 * c->b * c->b + 64;
}

// Switch the handle to a new tile size: items, smem attribute, graphs.
dacp_status retile(dacp_ctx* c, int tile_bytes) {
    tile_geometry(c, tile_bytes);
    if (prepare_step(c->prec, c->b, c->smem) != cudaSuccess || prepare_step(c->prec, 1, c->smem) != cudaSuccess)
        return fail(c, DACP_ERR_CUDA, "shared-memory attribute for %d bytes", c->smem);
    if (c->launch_mode == 2 && prepare_step_staged(c->b, c->smem) != cudaSuccess)
        return fail(c, DACP_ERR_CUDA, "staged shared-memory attribute for a %d-byte tile", c->smem);
    dfree(c, c->items_d);
    c->items_d = nullptr;
    TRY(dalloc_t(c, &c->items_d, c->items.size()));
    CK(cudaMemcpyAsync(c->items_d, c->items.data(), sizeof(Item) * c->items.size(), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->info_d, c->info.data(), sizeof(RealInfo) * c->R, cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    for (Graph* g : {&c->gf, &c->ge}) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
    }
    return DACP_OK;
}

// A stencil CTA whose bounded wait on its tile copy gave up sets err_d.
dacp_status check_device_flag(dacp_ctx* c) {
    int e = 0;
    CK(cudaMemcpyAsync(&e, c->err_d, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (e) {
        CK(cudaMemsetAsync(c->err_d, 0, sizeof(int), c->st));
        return fail(c, DACP_ERR_TIMEOUT, "a tile copy did not complete within the wait limit");
    }
    return DACP_OK;
}

dacp_status check_handle(dacp_ctx* c) {
    if (!c) return DACP_ERR_ARG;
    c->err.clear();
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(c, DACP_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return DACP_OK;
}

// Apply explicit parameters: run lengths, moment storage.
dacp_status apply_params(dacp_ctx* c) {
    int64_t rows_total = 0;
    for (int r = 0; r < c->R; ++r) {
        const double ar = c->a[r] / c->emax[r];
        c->kn[r] = static_cast<int>(floor(static_cast<double>(c->n[r]) * M_PI / ar));
        c->info[r].nf = c->K[r];
        c->info[r].ne = c->kn[r] + 2;   // one order beyond mu_{2k_n+1}: mu_{2k_n+3} for the H^2 elements
        c->info[r].mom_off = rows_total;
        rows_total += 2 * static_cast<int64_t>(c->kn[r]) + 4;
    }
    const int64_t need = rows_total * c->b * c->b;
    if (need > c->mom_cap) {
        dfree(c, c->mom_d);
        c->mom_d = nullptr;
        c->mom_cap = 0;
        TRY(dalloc_t(c, &c->mom_d, static_cast<size_t>(need)));
        c->mom_cap = need;
    }
    CK(cudaMemcpyAsync(c->info_d, c->info.data(), sizeof(RealInfo) * c->R, cudaMemcpyHostToDevice, c->st));
    std::vector<double> coef(8 * static_cast<size_t>(c->R), 0.0);
    for (int r = 0; r < c->R; ++r) {
        const double em = c->emax[r], aa = c->a[r];
        const double ec = (em * em + aa * aa) / 2.0, e0 = (em * em - aa * aa) / 2.0;
        // filter: order 0 -> T_1(F) = F, then 2F w_k - w_{k-1}
        coef[8 * r + 0] = 1.0 / e0;
        coef[8 * r + 1] = -ec / e0;
        coef[8 * r + 2] = 0.0;
        coef[8 * r + 3] = 2.0 / e0;
        coef[8 * r + 4] = -2.0 * ec / e0;
        coef[8 * r + 5] = -1.0;
    }
    CK(cudaMemcpyAsync(c->coef_d, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->bad.assign(c->R, 0);
    c->state = 1;
    return DACP_OK;
}

dacp_status set_evolution_coef(dacp_ctx* c, const std::vector<double>& emax) {
    std::vector<double> coef(8 * static_cast<size_t>(c->R), 0.0);
    for (int r = 0; r < c->R; ++r) {
        coef[8 * r + 0] = 1.0 / emax[r];
        coef[8 * r + 1] = 0.0;
        coef[8 * r + 3] = 2.0 / emax[r];
        coef[8 * r + 4] = -1.0;
    }
    CK(cudaMemcpyAsync(c->coef_d, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
    return DACP_OK;
}

}  // namespace

extern "C" {

const char* dacp_status_string(int s) {
    switch (s) {
        case DACP_OK: return "DACP_OK";
        case DACP_ERR_ARG: return "DACP_ERR_ARG";
        case DACP_ERR_CUDA: return "DACP_ERR_CUDA";
        case DACP_ERR_NOMEM: return "DACP_ERR_NOMEM";
        case DACP_ERR_NUMERIC: return "DACP_ERR_NUMERIC";
        case DACP_ERR_TIMEOUT: return "DACP_ERR_TIMEOUT";
        case DACP_ERR_STATE: return "DACP_ERR_STATE";
        case DACP_ERR_NOT_CONVERGED: return "DACP_ERR_NOT_CONVERGED";
        case DACP_ERR_LIBRARY: return "DACP_ERR_LIBRARY";
    }
    return "DACP_ERR_UNKNOWN";
}

const char* dacp_last_error(dacp_handle c) { return c ? c->err.c_str() : "NULL handle"; }

void dacp_destroy(dacp_handle c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->st) cudaStreamSynchronize(c->st);
    if (c->st2) cudaStreamSynchronize(c->st2);
    free_lanes(c);
    if (c->gf.exec) cudaGraphExecDestroy(c->gf.exec);
    if (c->ge.exec) cudaGraphExecDestroy(c->ge.exec);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->sp2) cusolverDnDestroyParams(c->sp2);
    if (c->sol2) cusolverDnDestroy(c->sol2);
    if (c->blas2) cublasDestroy(c->blas2);
    if (c->st2) cudaStreamDestroy(c->st2);
    if (c->sp) cusolverDnDestroyParams(c->sp);
    if (c->sol) cusolverDnDestroy(c->sol);
    if (c->blas) cublasDestroy(c->blas);
    for (void* p : c->allocs) cudaFree(p);
    if (c->own_stream && c->st) cudaStreamDestroy(c->st);
    delete c;
}

dacp_status dacp_create(dacp_handle* out, int n_real, const int* n_spins, const double* J, const double* h,
                        const double* gamma, int block_b, int precision, const double* psi0, void* stream) {
    NvtxRange nvtx_("dacp_create");
    if (!out) return DACP_ERR_ARG;
    *out = nullptr;
    if (n_real <= 0 || !n_spins || !J || !h || !gamma || !psi0) return DACP_ERR_ARG;
    if (!(block_b == 1 || block_b == 2 || block_b == 4)) return DACP_ERR_ARG;
    if (precision != DACP_FP64 && precision != DACP_FP32 && precision != DACP_DF32) return DACP_ERR_ARG;
    for (int r = 0; r < n_real; ++r)
        if (n_spins[r] < 1 || n_spins[r] > kMaxSpins) return DACP_ERR_ARG;
    // every coupling and field finite, checked before any device use
    {
        int64_t jo = 0, ho = 0;
        for (int r = 0; r < n_real; ++r) {
            const int Nr = n_spins[r];
            for (int i = 0; i < Nr; ++i) {
                if (!isfinite(h[ho + i]) || !isfinite(gamma[ho + i])) return DACP_ERR_ARG;
                for (int j = i + 1; j < Nr; ++j)
                    if (!isfinite(J[jo + static_cast<int64_t>(i) * Nr + j])) return DACP_ERR_ARG;
            }
            jo += static_cast<int64_t>(Nr) * Nr;
            ho += Nr;
        }
    }

    dacp_ctx* c = new dacp_ctx();
    auto bail = [&](dacp_status s) {
        dacp_destroy(c);
        return s;
    };
    cudaGetDevice(&c->device);
    c->R = n_real;
    c->b = block_b;
    c->prec = precision == DACP_FP32 ? kPrecF32 : (precision == DACP_DF32 ? kPrecDF32 : kPrecF64);
    c->fp32 = c->prec == kPrecF32;
    c->esz = c->fp32 ? 4 : 8;             // double-float pairs are 8 bytes like float64
    if (stream) {
        c->st = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) return bail(DACP_ERR_CUDA);
        c->own_stream = true;
    }
    c->N.assign(n_spins, n_spins + n_real);
    c->info.resize(n_real);
    c->J_h.assign(static_cast<size_t>(n_real) * kMaxSpins * kMaxSpins, 0.0);
    c->h_h.assign(static_cast<size_t>(n_real) * kMaxSpins, 0.0);
    c->g_h.assign(static_cast<size_t>(n_real) * kMaxSpins, 0.0);
    c->pnorm.assign(n_real, 0.0);
    int64_t jo = 0, ho = 0, off = 0;
    for (int r = 0; r < n_real; ++r) {
        const int Nr = n_spins[r];
        RealInfo& R = c->info[r];
        R.N = Nr;
        R.off = off;
        R.nf = 0;
        R.ne = 0;
        R.mom_off = 0;
        double pn = 0.0;
        for (int i = 0; i < Nr; ++i) {
            for (int j = 0; j < Nr; ++j) {
                const double v = J[jo + static_cast<int64_t>(i) * Nr + j];
                if (j > i) {
                    c->J_h[static_cast<size_t>(r) * kMaxSpins * kMaxSpins + i * kMaxSpins + j] = v;
                    pn += fabs(v);
                }
            }
            const double hv = h[ho + i], gv = gamma[ho + i];
            if (!isfinite(hv) || !isfinite(gv)) return bail(fail(c, DACP_ERR_ARG, "non-finite field"));
            c->h_h[static_cast<size_t>(r) * kMaxSpins + i] = hv;
            c->g_h[static_cast<size_t>(r) * kMaxSpins + i] = gv;
            pn += fabs(hv) + fabs(gv);
        }
        if (!isfinite(pn)) {
            dacp_destroy(c);
            return DACP_ERR_ARG;
        }
        c->pnorm[r] = pn;
        jo += static_cast<int64_t>(Nr) * Nr;
        ho += Nr;
        off += ((static_cast<int64_t>(1) << Nr) + 3) & ~static_cast<int64_t>(3);   // 16-byte aligned units
    }
    c->Dtot = off;
    c->pnorm0 = c->pnorm;
    tile_geometry(c, kTileBytes);
    c->emax.assign(n_real, 0.0);
    c->a.assign(n_real, 0.0);
    c->K.assign(n_real, 0);
    c->n.assign(n_real, 0);
    c->kn.assign(n_real, 0);
    c->bad.assign(n_real, 0);

    const size_t vec_bytes = static_cast<size_t>(c->Dtot) * block_b * c->esz;
    const int ni = static_cast<int>(c->items.size());
    dacp_status s;
#define ALLOC(expr) if ((s = (expr)) != DACP_OK) return bail(s)
    ALLOC(dalloc_t(c, &c->info_d, n_real));
    ALLOC(dalloc_t(c, &c->items_d, ni));
    ALLOC(dalloc_t(c, &c->J_d, c->J_h.size()));
    ALLOC(dalloc_t(c, &c->h_d, c->h_h.size()));
    ALLOC(dalloc_t(c, &c->pnorm_d, n_real));
    ALLOC(dalloc(c, &c->gam_d, c->g_h.size() * c->esz));
    ALLOC(dalloc(c, &c->diag_d, static_cast<size_t>(c->Dtot) * c->esz));
    ALLOC(dalloc(c, &c->psi0_d, vec_bytes));
    ALLOC(dalloc(c, &c->A_d, vec_bytes));
    ALLOC(dalloc(c, &c->B_d, vec_bytes));
    ALLOC(dalloc(c, &c->U_d, vec_bytes));
    ALLOC(dalloc(c, &c->psiE_d, vec_bytes));
    ALLOC(dalloc_t(c, &c->coef_d, 8 * static_cast<size_t>(n_real)));
    ALLOC(dalloc_t(c, &c->apply_coef_d, 8 * static_cast<size_t>(n_real)));
    ALLOC(dalloc_t(c, &c->part_d, part_capacity(c)));
    ALLOC(dalloc_t(c, &c->norms_d, static_cast<size_t>(n_real) * block_b));
    ALLOC(dalloc_t(c, &c->real_done_d, n_real));
    ALLOC(dalloc_t(c, &c->launch_done_d, 1));
    ALLOC(dalloc_t(c, &c->step_ctr_d, 1));
    ALLOC(dalloc_t(c, &c->err_d, 1));
    ALLOC(dalloc_t(c, &c->bar_d, 2));
#undef ALLOC

    auto ck = [&](cudaError_t e) { return e == cudaSuccess; };
    bool ok = ck(cudaMemcpyAsync(c->info_d, c->info.data(), sizeof(RealInfo) * n_real, cudaMemcpyHostToDevice, c->st)) &&
              ck(cudaMemcpyAsync(c->items_d, c->items.data(), sizeof(Item) * ni, cudaMemcpyHostToDevice, c->st)) &&
              ck(cudaMemcpyAsync(c->J_d, c->J_h.data(), c->J_h.size() * 8, cudaMemcpyHostToDevice, c->st)) &&
              ck(cudaMemcpyAsync(c->h_d, c->h_h.data(), c->h_h.size() * 8, cudaMemcpyHostToDevice, c->st)) &&
              ck(cudaMemcpyAsync(c->pnorm_d, c->pnorm.data(), n_real * 8, cudaMemcpyHostToDevice, c->st)) &&
              ck(cudaMemsetAsync(c->real_done_d, 0, sizeof(unsigned) * n_real, c->st)) &&
              ck(cudaMemsetAsync(c->launch_done_d, 0, sizeof(unsigned), c->st)) &&
              ck(cudaMemsetAsync(c->err_d, 0, sizeof(int), c->st)) &&
              ck(cudaMemsetAsync(c->bar_d, 0, 2 * sizeof(unsigned), c->st));
    if (!ok) return bail(fail(c, DACP_ERR_CUDA, "upload failed"));
    // x-fields in the vector precision
    {
        if ((s = dalloc_t(c, &c->g64_d, c->g_h.size())) != DACP_OK) return bail(s);
        double* tmp = c->g64_d;
        ok = ck(cudaMemcpyAsync(tmp, c->g_h.data(), c->g_h.size() * 8, cudaMemcpyHostToDevice, c->st)) &&
             ck(launch_convert(c->prec, tmp, c->gam_d, static_cast<int64_t>(c->g_h.size()), c->st));
        // start vectors: host float64 -> device, converted in place of psi0
        double* tmp2 = nullptr;
        const int64_t nv = c->Dtot * block_b;
        if (ok && (s = dalloc_t(c, &tmp2, static_cast<size_t>(nv))) != DACP_OK) return bail(s);
        // the caller's layout is packed; the device layout pads each realization to 4 states
        int64_t packed_total = 0;
        for (int r = 0; r < n_real; ++r) packed_total += (static_cast<int64_t>(1) << c->N[r]) * block_b;
        c->psi0_h.assign(psi0, psi0 + packed_total);
        ok = ok && ck(cudaMemsetAsync(c->psi0_d, 0, static_cast<size_t>(nv) * c->esz, c->st)) &&
             ck(cudaMemcpyAsync(tmp2, psi0, static_cast<size_t>(packed_total) * 8, cudaMemcpyHostToDevice, c->st));
        std::vector<int64_t> src_off(n_real);
        int64_t so = 0;
        for (int r = 0; r < n_real; ++r) {
            src_off[r] = so;
            so += (static_cast<int64_t>(1) << c->N[r]) * block_b;
        }
        int64_t* src_off_d = nullptr;
        int max_N0 = 1;
        for (int r = 0; r < n_real; ++r) max_N0 = std::max(max_N0, c->N[r]);
        if (ok && (s = dalloc_t(c, &src_off_d, n_real)) != DACP_OK) return bail(s);
        ok = ok && ck(cudaMemcpyAsync(src_off_d, src_off.data(), sizeof(int64_t) * n_real, cudaMemcpyHostToDevice, c->st)) &&
             ck(launch_scatter_convert(c->prec, tmp2, src_off_d, c->info_d, n_real, max_N0, block_b, c->psi0_d, c->st)) &&
             ck(cudaStreamSynchronize(c->st));
        dfree(c, src_off_d);
        int max_N = 1;
        for (int r = 0; r < n_real; ++r) max_N = std::max(max_N, c->N[r]);
        ok = ok && ck(launch_diag_all(c->prec, c->info_d, n_real, max_N, c->J_d, c->h_d, c->diag_d, c->st));
        c->launches += 3;
        std::vector<double> ac(8 * static_cast<size_t>(n_real), 0.0);
        for (int r = 0; r < n_real; ++r) ac[8 * r] = 1.0;
        ok = ok && ck(cudaMemcpyAsync(c->apply_coef_d, ac.data(), ac.size() * 8, cudaMemcpyHostToDevice, c->st)) &&
             ck(cudaStreamSynchronize(c->st));
        dfree(c, tmp2);
        if (!ok) return bail(fail(c, DACP_ERR_CUDA, "set-up kernels failed: %s", cudaGetErrorString(cudaGetLastError())));
    }
    // b-column stencil for the recurrences, 1-column stencil for the Lanczos / KPM pre-pass
    if (prepare_step(c->prec, block_b, c->smem) != cudaSuccess || prepare_step(c->prec, 1, c->smem) != cudaSuccess)
        return bail(DACP_ERR_CUDA);
    for (auto& e : c->ev)
        if (cudaEventCreate(&e) != cudaSuccess) return bail(DACP_ERR_CUDA);
    if (cusolverDnCreate(&c->sol) != CUSOLVER_STATUS_SUCCESS || cusolverDnSetStream(c->sol, c->st) != CUSOLVER_STATUS_SUCCESS ||
        cusolverDnCreateParams(&c->sp) != CUSOLVER_STATUS_SUCCESS)
        return bail(DACP_ERR_LIBRARY);
    if (cublasCreate(&c->blas) != CUBLAS_STATUS_SUCCESS || cublasSetStream(c->blas, c->st) != CUBLAS_STATUS_SUCCESS)
        return bail(DACP_ERR_LIBRARY);
    *out = c;
    return DACP_OK;
}

dacp_status dacp_set_params(dacp_handle c, const double* emax, const double* a, const int* K, const int* n) {
    TRY(check_handle(c));
    if (!emax || !a || !K || !n) return fail(c, DACP_ERR_ARG, "NULL parameter array");
    for (int r = 0; r < c->R; ++r) {
        if (!(emax[r] > 0.0) || !(a[r] > 0.0) || !(a[r] < emax[r]) || K[r] < 0 || n[r] < 1 || !isfinite(emax[r]))
            return fail(c, DACP_ERR_ARG, "bad parameters for realization %d", r);
        const double kn = floor(static_cast<double>(n[r]) * M_PI / (a[r] / emax[r]));
        if (kn > 2.0e8) return fail(c, DACP_ERR_ARG, "k_n too large for realization %d", r);
    }
    c->emax.assign(emax, emax + c->R);
    c->a.assign(a, a + c->R);
    c->K.assign(K, K + c->R);
    c->n.assign(n, n + c->R);
    return apply_params(c);
}

}  // extern "C"

namespace {

constexpr int kRule1LanczosSteps = 64;

// Lanczos bound + KPM moments of column 0 of psi0, then the window, order and
// basis size: from (d_ratio, basis_ratio, c_order) or from the network.
dacp_status choose_impl(dacp_ctx* c, int n_eigs, double d_ratio, double basis_ratio, double c_order,
                        int lanczos_steps, int kpm_moments, dacp_mlp net) {
    if (!(c_order > 0)) c_order = c->fp32 ? kCOrderFp32 : kCOrderFp64;
    if (n_eigs < 1 || !(d_ratio > 0) || !(basis_ratio > 0) || !(c_order > 0) || lanczos_steps < 2 ||
        lanczos_steps > 64 || kpm_moments < 2 * (kFeatureMoments + 1) || (kpm_moments & 1))
        return fail(c, DACP_ERR_ARG, "bad heuristic arguments");
    if (net && (mlp_n_in(net) != kFeatures || mlp_n_out(net) != 3))
        return fail(c, DACP_ERR_ARG, "the parameter network needs %d inputs and 3 outputs", kFeatures);
    int minN = kMaxSpins;
    for (int r = 0; r < c->R; ++r) minN = std::min(minN, c->N[r]);
    // Rule 0 takes the first lanczos_steps steps. Rule 1 runs the same recurrence on to
    // kRule1LanczosSteps: its bound falls from about 1.14 to 1.08 times the spectral radius
    // (N = 11, 12 shards), and rule 0's bound, hence the window and the network's features, is
    // unchanged because the first steps are the same.
    const int64_t dim_min = static_cast<int64_t>(1) << minN;
    const int steps0 = static_cast<int>(std::min<int64_t>(lanczos_steps, dim_min));
    const int steps = c->emax_rule == 1
                          ? static_cast<int>(std::min<int64_t>(std::max(lanczos_steps, kRule1LanczosSteps), dim_min))
                          : steps0;
    const int R = c->R;
    const int ni = static_cast<int>(c->items.size());
    const size_t sv = static_cast<size_t>(c->Dtot) * c->esz;   // one column
    void *v0 = nullptr, *v1 = nullptr, *v2 = nullptr, *kA = nullptr, *kB = nullptr;
    double *lmom = nullptr, *beta2 = nullptr, *emax_d = nullptr, *emax1_d = nullptr, *a_d = nullptr, *kp = nullptr;
    int *K_d = nullptr, *n_d = nullptr;
    float* knobs = nullptr;
    auto cleanup = [&]() {
        for (void* p : {v0, v1, v2, kA, kB, static_cast<void*>(lmom), static_cast<void*>(beta2),
                        static_cast<void*>(emax_d), static_cast<void*>(emax1_d), static_cast<void*>(a_d),
                        static_cast<void*>(kp),
                        static_cast<void*>(K_d), static_cast<void*>(n_d), static_cast<void*>(knobs)})
            dfree(c, p);
    };
    auto run = [&]() -> dacp_status {
        TRY(dalloc(c, &v0, sv));
        TRY(dalloc(c, &v1, sv));
        TRY(dalloc(c, &v2, sv));
        TRY(dalloc(c, &kA, sv));
        TRY(dalloc(c, &kB, sv));
        const int rows = 2 * steps;
        TRY(dalloc_t(c, &lmom, static_cast<size_t>(R) * rows));
        TRY(dalloc_t(c, &beta2, static_cast<size_t>(R) * steps));
        TRY(dalloc_t(c, &emax_d, R));
        TRY(dalloc_t(c, &emax1_d, R));
        TRY(dalloc_t(c, &a_d, R));
        TRY(dalloc_t(c, &kp, static_cast<size_t>(R) * kpm_moments));
        TRY(dalloc_t(c, &K_d, R));
        TRY(dalloc_t(c, &n_d, R));
        TRY(dalloc_t(c, &knobs, static_cast<size_t>(R) * 3));
        if (!c->feats_d) TRY(dalloc_t(c, &c->feats_d, static_cast<size_t>(R) * kFeatures));
        // v = column 0 of psi0, normalised; kept in kA for the KPM run
        CK(launch_extract_col(c->prec, c->b, c->psi0_d, v2, c->Dtot, c->st));
        c->launches += 3 + 4 * static_cast<int64_t>(steps) + 1 + kpm_moments / 2 + 2;
        CK(launch_normalize(c->prec, 1, c->items_d, c->info_d, ni, v2, v2, 0, c->part_d, c->real_done_d,
                            c->norms_d, v1, kA, c->st));
        // Lanczos: w = H v - beta v_prev; alpha = <w, v>; w -= alpha v; beta = |w|
        std::vector<double> lc(8 * static_cast<size_t>(R), 0.0);
        for (int r = 0; r < R; ++r) lc[8 * r] = 1.0;
        CK(cudaMemcpyAsync(c->apply_coef_d, lc.data(), lc.size() * 8, cudaMemcpyHostToDevice, c->st));
        void* vp = v0;   // v_{j-1}
        void* vc = v1;   // v_j
        void* w = v2;
        CK(cudaMemsetAsync(vp, 0, sv, c->st));
        for (int j = 0; j < steps; ++j) {
            StepArgs a = base_args(c);
            a.coef = c->apply_coef_d;
            a.x = vc;
            a.y1 = vp;
            a.out = w;
            a.apply_moments = 1;
            a.apply_row = j;
            a.mom = lmom;
            a.mom_rows_fixed = rows;
            CK(launch_step(c->prec, 1, kApply, a, 0, ni, c->smem, c->st));
            CK(launch_lanczos_orth(c->prec, c->items_d, c->info_d, ni, vc, w, lmom, rows, j, c->part_d,
                                   c->real_done_d, beta2, steps, c->st));
            CK(launch_lanczos_scale(c->prec, c->items_d, c->info_d, ni, w, beta2, j, steps, c->apply_coef_d, R, c->st));
            void* t = vp;
            vp = vc;
            vc = w;
            w = t;
        }
        // the residual rule's bound normalises the KPM moments, the network's features and the window
        // whatever the rule; rule 1's tighter bound only shortens the two recurrences (below)
        CK(launch_lanczos_bound(R, lmom, rows, beta2, steps0, steps, c->pnorm_d, 1e-3, emax_d, 0, c->st));
        if (c->emax_rule == 1)
            CK(launch_lanczos_bound(R, lmom, rows, beta2, steps, steps, c->pnorm_d, 1e-3, emax1_d, 1, c->st));
        // reset the apply coefficients of the test hook
        for (int r = 0; r < R; ++r) lc[8 * r + 1] = 0.0;
        CK(cudaMemcpyAsync(c->apply_coef_d, lc.data(), lc.size() * 8, cudaMemcpyHostToDevice, c->st));
        std::vector<double> em(R), em1(R);
        CK(cudaMemcpyAsync(em.data(), emax_d, R * 8, cudaMemcpyDeviceToHost, c->st));
        if (c->emax_rule == 1) CK(cudaMemcpyAsync(em1.data(), emax1_d, R * 8, cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        // KPM moments of the normalised start vector under G = H / E_max
        TRY(set_evolution_coef(c, em));
        StepArgs a = base_args(c);
        a.bufA = kA;
        a.bufB = kB;
        a.mom = kp;
        a.mom_rows_fixed = kpm_moments;
        a.nsteps_override = kpm_moments / 2;
        CK(cudaMemsetAsync(c->step_ctr_d, 0, sizeof(int), c->st));
        for (int k = 0; k < kpm_moments / 2; ++k) CK(launch_step(c->prec, 1, kEvolve, a, 0, ni, c->smem, c->st));
        CK(launch_features(R, c->info_d, c->J_d, c->h_d, c->g64_d, kp, kpm_moments, n_eigs, c->feats_d, c->st));
        if (net) {
            int64_t nl = 0;
            CK(mlp_forward_device(net, c->feats_d, R, knobs, c->st, &nl));
            c->launches += nl;
        }
        CK(launch_kpm_window(R, c->info_d, kp, kpm_moments, emax_d, d_ratio * n_eigs, c_order, basis_ratio, c->b,
                             net ? knobs : nullptr, n_eigs, a_d, K_d, n_d, c->st));
        std::vector<double> av(R);
        std::vector<int> Kv(R), nv(R);
        CK(cudaMemcpyAsync(av.data(), a_d, R * 8, cudaMemcpyDeviceToHost, c->st));
        CK(cudaMemcpyAsync(Kv.data(), K_d, R * 4, cudaMemcpyDeviceToHost, c->st));
        CK(cudaMemcpyAsync(nv.data(), n_d, R * 4, cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        if (c->emax_rule == 1) {
            // K = c E_max / a: the filter's growth inside the window, exp(2c sqrt(a^2 - E^2) / a), and the
            // basis orders' energy resolution pi E_max / (k_m a_r) do not depend on E_max, so the
            // tighter bound keeps both and removes orders
            for (int r = 0; r < R; ++r) {
                if (!(em1[r] > 0.0) || !(em1[r] <= em[r]))
                    return fail(c, DACP_ERR_NUMERIC, "E_max rule 1 failed for realization %d", r);
                Kv[r] = static_cast<int>(ceil(static_cast<double>(Kv[r]) * em1[r] / em[r] - 1e-9));
                em[r] = em1[r];
            }
        }
        for (int r = 0; r < R; ++r) {
            const double kn = floor(static_cast<double>(nv[r]) * M_PI / (av[r] / em[r]));
            if (!(av[r] > 0.0) || !(av[r] < em[r]) || kn > 2.0e8)
                return fail(c, DACP_ERR_NUMERIC, "parameter choice failed for realization %d (a = %g)", r, av[r]);
        }
        TRY(check_device_flag(c));
        c->emax = em;
        c->a = av;
        c->K = Kv;
        c->n = nv;
        return apply_params(c);
    };
    dacp_status s = run();
    cleanup();
    return s;
}

}  // namespace

extern "C" {

dacp_status dacp_choose_params(dacp_handle c, int n_eigs, double d_ratio, double basis_ratio, double c_order,
                               int lanczos_steps, int kpm_moments) {
    NvtxRange nvtx_("dacp_choose_params");
    TRY(check_handle(c));
    return choose_impl(c, n_eigs, d_ratio, basis_ratio, c_order, lanczos_steps, kpm_moments, nullptr);
}

dacp_status dacp_choose_params_mlp(dacp_handle c, dacp_mlp net, int n_eigs, int lanczos_steps, int kpm_moments) {
    NvtxRange nvtx_("dacp_choose_params_mlp");
    TRY(check_handle(c));
    if (!net) return fail(c, DACP_ERR_ARG, "NULL network");
    return choose_impl(c, n_eigs, 2.0, 1.5, 0.0, lanczos_steps, kpm_moments, net);
}

dacp_status dacp_get_features(dacp_handle c, float* feats, int64_t cap) {
    TRY(check_handle(c));
    if (!c->feats_d) return fail(c, DACP_ERR_STATE, "no parameter choice yet");
    if (!feats || cap < static_cast<int64_t>(c->R) * kFeatures) return fail(c, DACP_ERR_ARG, "capacity too small");
    CK(cudaMemcpyAsync(feats, c->feats_d, sizeof(float) * c->R * kFeatures, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return DACP_OK;
}

dacp_status dacp_get_params(dacp_handle c, double* emax, double* a, int* K, int* n, int* kn) {
    TRY(check_handle(c));
    if (c->state < 1) return fail(c, DACP_ERR_STATE, "no parameters set");
    for (int r = 0; r < c->R; ++r) {
        if (emax) emax[r] = c->emax[r];
        if (a) a[r] = c->a[r];
        if (K) K[r] = c->K[r];
        if (n) n[r] = c->n[r];
        if (kn) kn[r] = c->kn[r];
    }
    return DACP_OK;
}

dacp_status dacp_filter(dacp_handle c) {
    NvtxRange nvtx_("dacp_filter (T_F)");
    TRY(check_handle(c));
    if (c->state < 1) return fail(c, DACP_ERR_STATE, "dacp_filter before parameters");
    const size_t vec_bytes = static_cast<size_t>(c->Dtot) * c->b * c->esz;
    int maxK = 0;
    for (int r = 0; r < c->R; ++r) maxK = std::max(maxK, c->K[r]);
    CK(cudaEventRecord(c->ev[0], c->st));
    CK(cudaMemcpyAsync(c->A_d, c->psi0_d, vec_bytes, cudaMemcpyDeviceToDevice, c->st));
    TRY(run_orders(c, true, maxK));
    // psi_E = w_K / |w_K| per column; w_K sits in A (K even) or B (K odd); also w_0 of the evolution
    c->launches += 2;
    CK(launch_normalize(c->prec, c->b, c->items_d, c->info_d, static_cast<int>(c->items.size()), c->A_d, c->B_d, 1,
                        c->part_d, c->real_done_d, c->norms_d, c->psiE_d, nullptr, c->st));
    CK(cudaEventRecord(c->ev[1], c->st));
    CK(cudaStreamSynchronize(c->st));
    TRY(check_device_flag(c));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
    c->t_ms[0] = ms;
    c->state = 2;
    return DACP_OK;
}

dacp_status dacp_basis_moments(dacp_handle c) {
    NvtxRange nvtx_("dacp_basis_moments (T_E)");
    TRY(check_handle(c));
    if (c->state < 2) return fail(c, DACP_ERR_STATE, "dacp_basis_moments before dacp_filter");
    const size_t vec_bytes = static_cast<size_t>(c->Dtot) * c->b * c->esz;
    int maxE = 0;
    for (int r = 0; r < c->R; ++r) maxE = std::max(maxE, c->info[r].ne);
    TRY(set_evolution_coef(c, c->emax));
    CK(cudaEventRecord(c->ev[2], c->st));
    CK(cudaMemcpyAsync(c->A_d, c->psiE_d, vec_bytes, cudaMemcpyDeviceToDevice, c->st));
    TRY(run_orders(c, false, maxE));
    CK(cudaEventRecord(c->ev[3], c->st));
    CK(cudaStreamSynchronize(c->st));
    TRY(check_device_flag(c));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]);
    c->t_ms[1] = ms;
    // restore the filter coefficients for a later dacp_filter
    TRY(apply_params(c));
    c->state = 3;
    return DACP_OK;
}

}  // extern "C"

namespace {

constexpr double kBatchBytes = 24e9;   // device memory budget of one batched subspace group
// Up to 256 realizations per batched eigensolver call: at M = 748 the per-matrix time of the
// batched syev (with vectors) falls from 5.05 ms at 64 to 4.43 ms at 256, that of the values-only
// syev from 2.72 to 2.20 ms. kBatchBytes still caps the group for large bases.
constexpr int kMaxBatch = 256;

// Streams and library handles one batched subspace solve runs on.
struct SolveRes {
    cudaStream_t st = nullptr;
    cusolverDnHandle_t sol = nullptr;
    cublasHandle_t blas = nullptr;
    cusolverDnParams_t sp = nullptr;
};

// Device workspace of batched subspace solves: G slots of basis size <= M.
struct BatchWs {
    int G = 0, M = 0, L = 0, n_eigs = 0;
    int64_t mstride = 0;
    double *S = nullptr, *H = nullptr, *W = nullptr, *Ht = nullptr, *lam = nullptr, *lamt = nullptr,
           *mus = nullptr, *nus = nullptr, *sel = nullptr, *big = nullptr;
    int *orders = nullptr, *mi = nullptr, *bad = nullptr, *info = nullptr, *nf = nullptr;
    void* work = nullptr;
    size_t dbytes = 0, hbytes = 0;
    std::vector<char> work_h;
};

void ws_free(dacp_ctx* c, BatchWs& w) {
    for (void* p : {static_cast<void*>(w.S), static_cast<void*>(w.H), static_cast<void*>(w.W), static_cast<void*>(w.Ht),
                    static_cast<void*>(w.lam), static_cast<void*>(w.lamt), static_cast<void*>(w.mus),
                    static_cast<void*>(w.nus), static_cast<void*>(w.sel), static_cast<void*>(w.big),
                    static_cast<void*>(w.orders), static_cast<void*>(w.mi), static_cast<void*>(w.bad),
                    static_cast<void*>(w.info), static_cast<void*>(w.nf), w.work})
        dfree(c, p);
    w = BatchWs();
}

// Number of slots that fit the batch budget for basis size M.
int ws_slots(int R, int M, int64_t rows_max, int b) {
    const double per = 4.0 * 8.0 * M * static_cast<double>(M) + 2.0 * 8.0 * rows_max * b * b;
    return std::max(1, std::min(std::min(R, kMaxBatch), static_cast<int>(kBatchBytes / per)));
}

dacp_status ws_alloc(dacp_ctx* c, BatchWs& w, const SolveRes& s, int G, int M, int64_t rows_max, int n_eigs) {
    const int b = c->b;
    w.G = G;
    w.M = M;
    w.L = M / b;
    w.n_eigs = n_eigs;
    w.mstride = rows_max * b * b;
    const size_t MM = static_cast<size_t>(M) * M;
    TRY(dalloc_t(c, &w.S, G * MM));
    TRY(dalloc_t(c, &w.H, G * MM));
    TRY(dalloc_t(c, &w.W, G * MM));
    TRY(dalloc_t(c, &w.Ht, G * MM));
    TRY(dalloc_t(c, &w.lam, static_cast<size_t>(G) * M));
    TRY(dalloc_t(c, &w.lamt, static_cast<size_t>(G) * M));
    TRY(dalloc_t(c, &w.mus, static_cast<size_t>(G) * w.mstride));
    TRY(dalloc_t(c, &w.nus, static_cast<size_t>(G) * w.mstride));
    TRY(dalloc_t(c, &w.sel, static_cast<size_t>(G) * n_eigs));
    TRY(dalloc_t(c, &w.big, G));
    TRY(dalloc_t(c, &w.orders, static_cast<size_t>(G) * w.L));
    TRY(dalloc_t(c, &w.mi, G));
    TRY(dalloc_t(c, &w.bad, G));
    TRY(dalloc_t(c, &w.info, G));
    TRY(dalloc_t(c, &w.nf, G));
    size_t d1 = 0, h1 = 0, d2 = 0, h2 = 0;
    CKS(cusolverDnXsyevBatched_bufferSize(s.sol, s.sp, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, M, CUDA_R_64F,
                                          w.S, M, CUDA_R_64F, w.lam, CUDA_R_64F, &d1, &h1, G));
    CKS(cusolverDnXsyevBatched_bufferSize(s.sol, s.sp, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, M,
                                          CUDA_R_64F, w.Ht, M, CUDA_R_64F, w.lamt, CUDA_R_64F, &d2, &h2, G));
    w.dbytes = std::max(d1, d2);
    w.hbytes = std::max(h1, h2);
    TRY(dalloc(c, &w.work, w.dbytes));
    w.work_h.resize(std::max<size_t>(w.hbytes, 1));
    return DACP_OK;
}

// Batched subspace solve of the g <= G realizations idx[0..g) on stream s.st.
// Every realization's S and H sit in the top-left corner of an Mg x Mg slot
// (Mg = the group's largest basis size), zero elsewhere: the zero rows and
// columns give S eigenvalues 0, which the cut-off removes, so the padding
// changes nothing. One batched syev of S (with vectors), the cut-off, two
// strided-batched dgemm for H~ = U^T H U (U padded to the group's largest rank
// with zero columns), one batched syev of H~ (values; the padded directions
// sit on a decoupled diagonal at 3 E_max, outside every window) and the
// central selection.
dacp_status solve_batch(dacp_ctx* c, BatchWs& w, const SolveRes& s, const int* idx, int g, int n_eigs, double window,
                        double eps, double* eigs, int* n_found, int* rank) {
    NvtxRange nvtx_("solve_batch");
    const int b = c->b;
    int Mg = 0;
    for (int i = 0; i < g; ++i) Mg = std::max(Mg, b * (2 * c->n[idx[i]] + 1));
    if (g > w.G || Mg > w.M || n_eigs > w.n_eigs) return fail(c, DACP_ERR_ARG, "batched solve beyond its workspace");
    const int L = Mg / b;
    const int64_t MM = static_cast<int64_t>(Mg) * Mg;
    const int64_t mstride = w.mstride;
    size_t d1 = 0, h1 = 0, d2 = 0, h2 = 0;
    CKS(cusolverDnXsyevBatched_bufferSize(s.sol, s.sp, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, Mg, CUDA_R_64F,
                                          w.S, Mg, CUDA_R_64F, w.lam, CUDA_R_64F, &d1, &h1, g));
    if (d1 > w.dbytes || h1 > w.work_h.size()) return fail(c, DACP_ERR_CUDA, "batched eigensolver workspace grew");
    std::vector<int> hm(g), hbad(g), hinfo(g), hnf(g);
    std::vector<double> hbig(g), hsel(static_cast<size_t>(g) * n_eigs);
    const double one = 1.0, zero = 0.0;
    CK(cudaMemsetAsync(w.bad, 0, sizeof(int) * g, s.st));
    bool padded = false;
    for (int i = 0; i < g; ++i) padded = padded || b * (2 * c->n[idx[i]] + 1) != Mg;
    if (padded) {
        CK(cudaMemsetAsync(w.S, 0, sizeof(double) * g * MM, s.st));
        CK(cudaMemsetAsync(w.H, 0, sizeof(double) * g * MM, s.st));
    }
    for (int i = 0; i < g; ++i) {
        const int r = idx[i];
        const int rows = 2 * c->kn[r] + 2;
        const int Lr = 2 * c->n[r] + 1;
        CK(launch_orders(Lr, c->a[r] / c->emax[r], w.orders + static_cast<int64_t>(i) * L, s.st));
        CK(launch_moments(c->mom_d + c->info[r].mom_off * b * b, rows, b, c->emax[r], w.mus + i * mstride,
                          w.nus + i * mstride, w.bad + i, s.st));
        CK(launch_assemble(Lr, b, w.orders + static_cast<int64_t>(i) * L, w.mus + i * mstride, w.nus + i * mstride,
                           w.S + i * MM, w.H + i * MM, s.st, Mg));
    }
    CKS(cusolverDnXsyevBatched(s.sol, s.sp, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, Mg, CUDA_R_64F, w.S, Mg,
                               CUDA_R_64F, w.lam, CUDA_R_64F, w.work, w.dbytes, w.work_h.data(), w.hbytes, w.info, g));
    for (int i = 0; i < g; ++i)
        CK(launch_cutoff(w.lam + static_cast<int64_t>(i) * Mg, Mg, eps, 0, w.S + i * MM, w.mi + i, s.st));
    c->launches += 4 * g;
    CK(cudaMemcpyAsync(hm.data(), w.mi, sizeof(int) * g, cudaMemcpyDeviceToHost, s.st));
    CK(cudaMemcpyAsync(hbad.data(), w.bad, sizeof(int) * g, cudaMemcpyDeviceToHost, s.st));
    CK(cudaMemcpyAsync(hinfo.data(), w.info, sizeof(int) * g, cudaMemcpyDeviceToHost, s.st));
    CK(cudaStreamSynchronize(s.st));
    int m_max = 0;
    for (int i = 0; i < g; ++i)
        if (!hbad[i] && hinfo[i] == 0) m_max = std::max(m_max, hm[i]);
    if (m_max < 1) {
        for (int i = 0; i < g; ++i) n_found[idx[i]] = hbad[i] ? -DACP_ERR_NUMERIC : -DACP_ERR_NOT_CONVERGED;
        return DACP_OK;
    }
    for (int i = 0; i < g; ++i) {
        if (rank) rank[idx[i]] = hm[i];
        if (hbad[i] || hinfo[i] != 0) hm[i] = m_max;     // excluded below; keep the padding a no-op
        hbig[i] = 3.0 * c->emax[idx[i]];
    }
    CK(cudaMemcpyAsync(w.mi, hm.data(), sizeof(int) * g, cudaMemcpyHostToDevice, s.st));
    CK(cudaMemcpyAsync(w.big, hbig.data(), sizeof(double) * g, cudaMemcpyHostToDevice, s.st));
    CK(launch_pad_columns(w.S, Mg, MM, w.mi, m_max, g, s.st));
    const double* U = w.S + static_cast<int64_t>(Mg - m_max) * Mg;
    CKB(cublasDgemmStridedBatched(s.blas, CUBLAS_OP_N, CUBLAS_OP_N, Mg, m_max, Mg, &one, w.H, Mg, MM, U, Mg, MM, &zero,
                                  w.W, Mg, static_cast<int64_t>(Mg) * m_max, g));
    // H~ = U^T W, one strided-batched dgemm over the group. A per-realization syrkx (the lower
    // triangle only, half the flops) ran at 0.40 TF/s against the batched dgemm's 1.03 at M = 748.
    CKB(cublasDgemmStridedBatched(s.blas, CUBLAS_OP_T, CUBLAS_OP_N, m_max, m_max, Mg, &one, U, Mg, MM, w.W, Mg,
                                  static_cast<int64_t>(Mg) * m_max, &zero, w.Ht, m_max,
                                  static_cast<int64_t>(m_max) * m_max, g));
    CK(launch_pad_diagonal(w.Ht, m_max, static_cast<int64_t>(m_max) * m_max, w.mi, w.big, g, s.st));
    CKS(cusolverDnXsyevBatched_bufferSize(s.sol, s.sp, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, m_max,
                                          CUDA_R_64F, w.Ht, m_max, CUDA_R_64F, w.lamt, CUDA_R_64F, &d2, &h2, g));
    if (d2 > w.dbytes || h2 > w.work_h.size()) return fail(c, DACP_ERR_CUDA, "batched eigensolver workspace grew");
    CKS(cusolverDnXsyevBatched(s.sol, s.sp, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, m_max, CUDA_R_64F,
                               w.Ht, m_max, CUDA_R_64F, w.lamt, CUDA_R_64F, w.work, w.dbytes, w.work_h.data(),
                               w.hbytes, w.info, g));
    for (int i = 0; i < g; ++i) {
        const double wd = window > 0.0 ? window : c->a[idx[i]];
        CK(launch_select(w.lamt + static_cast<int64_t>(i) * m_max, m_max, n_eigs, wd,
                         w.sel + static_cast<int64_t>(i) * n_eigs, w.nf + i, s.st));
    }
    c->launches += 2 + g;
    CK(cudaMemcpyAsync(hsel.data(), w.sel, sizeof(double) * g * n_eigs, cudaMemcpyDeviceToHost, s.st));
    CK(cudaMemcpyAsync(hnf.data(), w.nf, sizeof(int) * g, cudaMemcpyDeviceToHost, s.st));
    CK(cudaMemcpyAsync(hinfo.data(), w.info, sizeof(int) * g, cudaMemcpyDeviceToHost, s.st));
    CK(cudaStreamSynchronize(s.st));
    for (int i = 0; i < g; ++i) {
        const int r = idx[i];
        if (hbad[i]) { n_found[r] = -DACP_ERR_NUMERIC; continue; }
        if (hinfo[i] != 0) { n_found[r] = -DACP_ERR_NOT_CONVERGED; continue; }
        memcpy(eigs + static_cast<size_t>(r) * n_eigs, hsel.data() + static_cast<size_t>(i) * n_eigs,
               sizeof(double) * hnf[i]);
        n_found[r] = hnf[i];
    }
    return DACP_OK;
}

// All realizations through batched solves on the handle's stream.
dacp_status central_eigs_batched(dacp_ctx* c, int n_eigs, double window, double eps, double* eigs, int* n_found,
                                 int* rank, int M, int64_t rows_max) {
    const SolveRes s{c->st, c->sol, c->blas, c->sp};
    const int G = ws_slots(c->R, M, rows_max, c->b);
    BatchWs w;
    dacp_status st = ws_alloc(c, w, s, G, M, rows_max, n_eigs);
    std::vector<int> idx(G);
    for (int r0 = 0; r0 < c->R && st == DACP_OK; r0 += G) {
        const int g = std::min(G, c->R - r0);
        for (int i = 0; i < g; ++i) idx[i] = r0 + i;
        st = solve_batch(c, w, s, idx.data(), g, n_eigs, window, eps, eigs, n_found, rank);
    }
    cudaStreamSynchronize(c->st);
    ws_free(c, w);
    return st;
}

}  // namespace

extern "C" {

dacp_status dacp_central_eigs(dacp_handle c, int n_eigs, double window, double eps, double* eigs, int* n_found,
                              int* rank) {
    NvtxRange nvtx_("dacp_central_eigs (T_D)");
    TRY(check_handle(c));
    if (c->state < 3) return fail(c, DACP_ERR_STATE, "dacp_central_eigs before dacp_basis_moments");
    if (n_eigs < 1 || !eigs || !n_found) return fail(c, DACP_ERR_ARG, "bad output arguments");
    if (!(eps > 0.0)) eps = c->fp32 ? kEpsFp32 : (c->prec == kPrecDF32 ? kEpsDf32 : 1e-12);
    const int b = c->b;
    int Mmax = 0;
    int64_t rows_max = 0;
    for (int r = 0; r < c->R; ++r) {
        Mmax = std::max(Mmax, b * (2 * c->n[r] + 1));
        rows_max = std::max<int64_t>(rows_max, 2 * static_cast<int64_t>(c->kn[r]) + 2);
    }
    // batched whenever there are several realizations and their sizes are within
    // 25 % of the largest (padding beyond that would cost more than lanes)
    bool batch = c->R >= 2 && c->batched_solve;
    for (int r = 0; r < c->R && batch; ++r) batch = 4 * b * (2 * c->n[r] + 1) >= 3 * Mmax;
    if (batch) {
        // one batched cuSOLVER call per group of equal-size problems
        CK(cudaEventRecord(c->ev[4], c->st));
        TRY(central_eigs_batched(c, n_eigs, window, eps, eigs, n_found, rank, Mmax, rows_max));
        CK(cudaEventRecord(c->ev[5], c->st));
        CK(cudaStreamSynchronize(c->st));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev[4], c->ev[5]);
        c->t_ms[2] = ms;
        return DACP_OK;
    }
    TRY(ensure_lanes(c, Mmax, rows_max, n_eigs));
    const int nl = static_cast<int>(c->lanes.size());
    CK(cudaEventRecord(c->ev[4], c->st));
    for (auto& L : c->lanes) CK(cudaStreamWaitEvent(L.st, c->ev[4], 0));

    // Phase A on lane r % nl: moments -> S, H; S = V Lam V^T; cut-off -> m (device).
    auto phase_a = [&](int r, Lane& L) -> dacp_status {
        const int Ln = 2 * c->n[r] + 1;
        const int M = b * Ln;
        const int rows = 2 * c->kn[r] + 2;
        CK(cudaMemsetAsync(L.bad, 0, sizeof(int), L.st));
        c->launches += 4;
        CK(launch_orders(Ln, c->a[r] / c->emax[r], L.orders, L.st));
        CK(launch_moments(c->mom_d + c->info[r].mom_off * b * b, rows, b, c->emax[r], L.mus, L.nus, L.bad, L.st));
        CK(launch_assemble(Ln, b, L.orders, L.mus, L.nus, L.S, L.H, L.st));
        CKS(cusolverDnXsyevd(L.sol, L.sp, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, M, CUDA_R_64F, L.S, M,
                             CUDA_R_64F, L.lam, CUDA_R_64F, L.work, L.dbytes, L.work_h.data(), L.hbytes, L.info));
        CK(launch_cutoff(L.lam, M, eps, 0, L.S, L.mi, L.st));
        CK(cudaMemcpyAsync(&L.hv[0], L.mi, sizeof(int), cudaMemcpyDeviceToHost, L.st));
        CK(cudaMemcpyAsync(&L.hv[1], L.bad, sizeof(int), cudaMemcpyDeviceToHost, L.st));
        CK(cudaMemcpyAsync(&L.hv[2], L.info, sizeof(int), cudaMemcpyDeviceToHost, L.st));
        return DACP_OK;
    };
    // Phase B: W = H U, Ht = U^T W, eigenvalues of Ht, central selection.
    auto phase_b = [&](int r, Lane& L) -> dacp_status {
        CK(cudaStreamSynchronize(L.st));
        const int M = b * (2 * c->n[r] + 1);
        const int m = L.hv[0];
        if (rank) rank[r] = m;
        L.cnt = -1;
        if (L.hv[1]) { n_found[r] = -DACP_ERR_NUMERIC; return DACP_OK; }
        if (L.hv[2] != 0 || m < 1) { n_found[r] = -DACP_ERR_NOT_CONVERGED; return DACP_OK; }
        const double* U = L.S + static_cast<size_t>(M - m) * M;
        const double one = 1.0, zero = 0.0;
        CKB(cublasDgemm(L.blas, CUBLAS_OP_N, CUBLAS_OP_N, M, m, M, &one, L.H, M, U, M, &zero, L.W, M));
        CKB(cublasDgemm(L.blas, CUBLAS_OP_T, CUBLAS_OP_N, m, m, M, &one, U, M, L.W, M, &zero, L.Ht, m));
        CKS(cusolverDnXsyevd(L.sol, L.sp, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, m, CUDA_R_64F, L.Ht, m,
                             CUDA_R_64F, L.lamt, CUDA_R_64F, L.work, L.dbytes, L.work_h.data(), L.hbytes, L.info));
        const double w = window > 0.0 ? window : c->a[r];
        CK(launch_select(L.lamt, m, n_eigs, w, L.sel, L.nf, L.st));
        c->launches += 1;
        CK(cudaMemcpyAsync(&L.cnt, L.nf, sizeof(int), cudaMemcpyDeviceToHost, L.st));
        CK(cudaMemcpyAsync(&L.hv[2], L.info, sizeof(int), cudaMemcpyDeviceToHost, L.st));
        CK(cudaMemcpyAsync(L.out_h.data(), L.sel, sizeof(double) * n_eigs, cudaMemcpyDeviceToHost, L.st));
        L.r = r;
        return DACP_OK;
    };
    auto collect = [&](Lane& L) -> dacp_status {
        if (L.r < 0) return DACP_OK;
        CK(cudaStreamSynchronize(L.st));
        if (L.cnt >= 0) {
            if (L.hv[2] != 0) {
                n_found[L.r] = -DACP_ERR_NOT_CONVERGED;
            } else {
                memcpy(eigs + static_cast<size_t>(L.r) * n_eigs, L.out_h.data(), sizeof(double) * L.cnt);
                n_found[L.r] = L.cnt;
            }
        }
        L.r = -1;
        return DACP_OK;
    };
    // One host thread per lane: cuSOLVER's syevd keeps part of its work on the
    // host, so lanes driven from a single thread would serialise on it.
    for (auto& L : c->lanes) L.r = -1;
    std::vector<dacp_status> lane_status(nl, DACP_OK);
    auto worker = [&](int li) {
        cudaSetDevice(c->device);
        Lane& L = c->lanes[li];
        for (int r = li; r < c->R; r += nl) {
            dacp_status st = phase_a(r, L);
            if (st == DACP_OK) st = phase_b(r, L);
            if (st == DACP_OK) st = collect(L);
            if (st != DACP_OK) {
                lane_status[li] = st;
                return;
            }
        }
    };
    {
        std::vector<std::thread> pool;
        for (int li = 0; li < nl; ++li) pool.emplace_back(worker, li);
        for (auto& t : pool) t.join();
    }
    for (dacp_status st : lane_status) TRY(st);
    for (auto& L : c->lanes) {
        CK(cudaEventRecord(L.done, L.st));
        CK(cudaStreamWaitEvent(c->st, L.done, 0));
    }
    CK(cudaEventRecord(c->ev[5], c->st));
    CK(cudaStreamSynchronize(c->st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev[4], c->ev[5]);
    c->t_ms[2] = ms;
    return DACP_OK;
}

}  // extern "C"

namespace {

dacp_status ensure_solver2(dacp_ctx* c) {
    if (c->st2) return DACP_OK;
    // highest priority: the solves' kernels take SM slots as the stencil's CTAs retire
    int least = 0, greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CK(cudaStreamCreateWithPriority(&c->st2, cudaStreamNonBlocking, greatest));
    CKS(cusolverDnCreate(&c->sol2));
    CKS(cusolverDnSetStream(c->sol2, c->st2));
    CKS(cusolverDnCreateParams(&c->sp2));
    CKB(cublasCreate(&c->blas2));
    CKB(cublasSetStream(c->blas2, c->st2));
    return DACP_OK;
}

// Realizations in rising completion order, cut into sub-batches whose basis
// sizes stay within 25 % of the sub-batch's largest (padding beyond that
// would cost more than it saves).
void size_batches(const dacp_ctx* c, std::vector<int>& idx, int G, std::vector<std::pair<int, int>>& out) {
    const int b = c->b;
    auto M = [&](int r) { return b * (2 * c->n[r] + 1); };
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return M(x) > M(y); });
    out.clear();
    for (size_t p = 0; p < idx.size();) {
        size_t q = p + 1;
        while (q < idx.size() && static_cast<int>(q - p) < G && 4 * M(idx[q]) >= 3 * M(idx[p])) ++q;
        out.emplace_back(static_cast<int>(p), static_cast<int>(q));
        p = q;
    }
}

}  // namespace

extern "C" {

dacp_status dacp_solve(dacp_handle c, int n_eigs, double window, double eps, double* eigs, int* n_found, int* rank) {
    NvtxRange nvtx_("dacp_solve");
    TRY(check_handle(c));
    if (c->state < 1) return fail(c, DACP_ERR_STATE, "dacp_solve before parameters");
    if (n_eigs < 1 || !eigs || !n_found) return fail(c, DACP_ERR_ARG, "bad output arguments");
    if (!(eps > 0.0)) eps = c->fp32 ? kEpsFp32 : (c->prec == kPrecDF32 ? kEpsDf32 : 1e-12);
    const int R = c->R, b = c->b;
    int Mmax = 0, maxE = 0;
    int64_t rows_max = 0;
    for (int r = 0; r < R; ++r) {
        Mmax = std::max(Mmax, b * (2 * c->n[r] + 1));
        rows_max = std::max<int64_t>(rows_max, 2 * static_cast<int64_t>(c->kn[r]) + 2);
        maxE = std::max(maxE, c->info[r].ne);
        n_found[r] = 0;
        if (rank) rank[r] = 0;
    }
    TRY(dacp_filter(c));
    TRY(ensure_solver2(c));
    const SolveRes s2{c->st2, c->sol2, c->blas2, c->sp2};
    const int G = ws_slots(R, Mmax, rows_max, b);
    // a job is handed to the solver once this many realizations have finished: quarters of the
    // batch, since the batched eigensolvers run faster per matrix in larger groups
    const int chunk = std::max(1, std::min(G, std::max(8, R / 4)));

    struct Job {
        std::vector<int> idx;
        cudaEvent_t ev = nullptr;
    };
    BatchWs w;
    std::vector<cudaEvent_t> events;
    std::deque<Job> queue;
    std::mutex mu;
    std::condition_variable cv;
    bool closed = false;
    dacp_status wst = DACP_OK;
    cudaEvent_t evD = nullptr;

    // Worker: one batched solve per job (split by basis size), on the second
    // stream, after the evolution orders that finished the job's realizations.
    auto worker = [&]() {
        cudaSetDevice(c->device);
        std::vector<std::pair<int, int>> parts;
        for (;;) {
            Job j;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return !queue.empty() || closed; });
                if (queue.empty()) return;
                j = std::move(queue.front());
                queue.pop_front();
            }
            if (wst != DACP_OK) continue;
            if (cudaStreamWaitEvent(s2.st, j.ev, 0) != cudaSuccess) {
                wst = fail(c, DACP_ERR_CUDA, "cudaStreamWaitEvent on the solver stream");
                continue;
            }
            size_batches(c, j.idx, G, parts);
            for (auto& pq : parts) {
                if (wst != DACP_OK) break;
                wst = solve_batch(c, w, s2, j.idx.data() + pq.first, pq.second - pq.first, n_eigs, window, eps, eigs,
                                  n_found, rank);
            }
        }
    };

    std::thread th;
    auto push = [&](const std::vector<int>& order, int from, int to) -> dacp_status {
        cudaEvent_t ev = nullptr;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        events.push_back(ev);
        CK(cudaEventRecord(ev, c->st));
        Job j;
        j.idx.assign(order.begin() + from, order.begin() + to);
        j.ev = ev;
        {
            std::lock_guard<std::mutex> lk(mu);
            queue.push_back(std::move(j));
        }
        cv.notify_one();
        return DACP_OK;
    };
    auto run = [&]() -> dacp_status {
        TRY(ws_alloc(c, w, s2, G, Mmax, rows_max, n_eigs));
        CK(cudaEventCreate(&evD));
        std::vector<int> order(R);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return c->info[x].ne < c->info[y].ne; });
        th = std::thread(worker);
        int dispatched = 0, complete = 0;
        auto after = [&](int done) -> dacp_status {
            while (complete < R && c->info[order[complete]].ne <= done) ++complete;
            if (complete - dispatched >= chunk) {
                TRY(push(order, dispatched, complete));
                dispatched = complete;
            }
            return DACP_OK;
        };
        const size_t vec_bytes = static_cast<size_t>(c->Dtot) * c->b * c->esz;
        TRY(set_evolution_coef(c, c->emax));
        CK(cudaEventRecord(c->ev[2], c->st));
        CK(cudaMemcpyAsync(c->A_d, c->psiE_d, vec_bytes, cudaMemcpyDeviceToDevice, c->st));
        TRY(run_orders(c, false, maxE, after));
        CK(cudaEventRecord(c->ev[3], c->st));
        if (dispatched < R) TRY(push(order, dispatched, R));
        return DACP_OK;
    };
    dacp_status st = run();
    {
        std::lock_guard<std::mutex> lk(mu);
        closed = true;
    }
    cv.notify_one();
    if (th.joinable()) th.join();
    if (st == DACP_OK) st = wst;
    if (st == DACP_OK && evD) {
        if (cudaEventRecord(evD, s2.st) != cudaSuccess) st = fail(c, DACP_ERR_CUDA, "cudaEventRecord");
    }
    cudaStreamSynchronize(s2.st);
    cudaStreamSynchronize(c->st);
    if (st == DACP_OK) st = check_device_flag(c);
    if (st == DACP_OK) {
        float te = 0.f, td = 0.f;
        cudaEventElapsedTime(&te, c->ev[2], c->ev[3]);
        cudaEventElapsedTime(&td, c->ev[3], evD);
        c->t_ms[1] = te;
        c->t_ms[2] = td > 0.f ? td : 0.0;   // the part of the solves not hidden under the evolution
    }
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    if (evD) cudaEventDestroy(evD);
    ws_free(c, w);
    if (st != DACP_OK) return st;
    // restore the filter coefficients for a later dacp_filter
    TRY(apply_params(c));
    c->state = 3;
    return DACP_OK;
}

// A handle over realizations rs of c, built from c's host copies of their couplings, fields, pair
// couplings, global flips and start vectors (the re-runs of dacp_solve_learned and dacp_solve_sectors).
static dacp_status sub_handle(dacp_ctx* c, const std::vector<int>& rs, dacp_handle* out) {
    const int nr = static_cast<int>(rs.size()), b = c->b;
    std::vector<int64_t> psi_off(c->R + 1, 0), j_off(c->R + 1, 0);
    for (int r = 0; r < c->R; ++r) {
        psi_off[r + 1] = psi_off[r] + (static_cast<int64_t>(1) << c->N[r]) * b;
        j_off[r + 1] = j_off[r] + static_cast<int64_t>(c->N[r]) * c->N[r];
    }
    std::vector<int> ns;
    std::vector<double> J, h, g, psi, jxx, jyy;
    for (int r : rs) {
        const int Nr = c->N[r];
        ns.push_back(Nr);
        for (int i = 0; i < Nr; ++i) {
            h.push_back(c->h_h[static_cast<size_t>(r) * kMaxSpins + i]);
            g.push_back(c->g_h[static_cast<size_t>(r) * kMaxSpins + i]);
            for (int j = 0; j < Nr; ++j)
                J.push_back(c->J_h[static_cast<size_t>(r) * kMaxSpins * kMaxSpins + i * kMaxSpins + j]);
        }
        psi.insert(psi.end(), c->psi0_h.begin() + psi_off[r], c->psi0_h.begin() + psi_off[r + 1]);
        if (c->has_pairs) {
            jxx.insert(jxx.end(), c->jxx_h.begin() + j_off[r], c->jxx_h.begin() + j_off[r + 1]);
            jyy.insert(jyy.end(), c->jyy_h.begin() + j_off[r], c->jyy_h.begin() + j_off[r + 1]);
        }
    }
    dacp_handle sub = nullptr;
    dacp_status st = dacp_create(&sub, nr, ns.data(), J.data(), h.data(), g.data(), b, c->prec, psi.data(), c->st);
    if (st != DACP_OK) return st;
    if (c->has_pairs) st = dacp_set_pair_couplings(sub, jxx.data(), jyy.data());
    if (st == DACP_OK && c->has_gflip) {
        std::vector<double> gsub;
        for (int r : rs) gsub.push_back(c->gflip_h[r]);
        st = dacp_set_global_flips(sub, gsub.data());
    }
    if (st != DACP_OK) {
        dacp_destroy(sub);
        return st;
    }
    *out = sub;
    return DACP_OK;
}

// Realizations whose learned parameters returned fewer than n_eigs levels go
// through the heuristic on a handle of their own, built from this handle's host
// copies of their couplings, fields and start vectors.
dacp_status dacp_solve_learned(dacp_handle c, dacp_mlp net, int n_eigs, double window, double eps, double* eigs,
                               int* n_found, int* rank, int* n_fallback) {
    NvtxRange nvtx_("dacp_solve_learned");
    TRY(check_handle(c));
    if (!net) return fail(c, DACP_ERR_ARG, "NULL network");
    if (n_eigs < 1 || !eigs || !n_found) return fail(c, DACP_ERR_ARG, "bad output arguments");
    if (n_fallback) *n_fallback = 0;
    TRY(choose_impl(c, n_eigs, 2.0, 1.5, 0.0, 20, 256, net));
    TRY(dacp_solve(c, n_eigs, window, eps, eigs, n_found, rank));
    std::vector<int> redo;
    for (int r = 0; r < c->R; ++r)
        if (n_found[r] < n_eigs) redo.push_back(r);
    if (n_fallback) *n_fallback = static_cast<int>(redo.size());
    if (redo.empty()) return DACP_OK;
    const int nr = static_cast<int>(redo.size());
    dacp_handle sub = nullptr;
    dacp_status st = sub_handle(c, redo, &sub);
    if (st != DACP_OK) return fail(c, st, "heuristic re-run: set-up failed");
    std::vector<double> e2(static_cast<size_t>(nr) * n_eigs, 0.0);
    std::vector<int> nf2(nr, 0), rk2(nr, 0);
    if (st == DACP_OK) st = dacp_set_emax_rule(sub, 0);      // the true bound: also recovers a rule-1 failure
    if (st == DACP_OK) st = dacp_choose_params(sub, n_eigs, 2.0, 1.5, 0.0, 20, 256);
    if (st == DACP_OK) st = dacp_solve(sub, n_eigs, window, eps, e2.data(), nf2.data(), rk2.data());
    if (st != DACP_OK) {
        const std::string msg = dacp_last_error(sub);
        dacp_destroy(sub);
        return fail(c, st, "heuristic re-run: %s", msg.c_str());
    }
    c->launches += sub->launches.load();
    dacp_destroy(sub);
    for (int j = 0; j < nr; ++j) {
        const int r = redo[j];
        memcpy(eigs + static_cast<size_t>(r) * n_eigs, e2.data() + static_cast<size_t>(j) * n_eigs,
               sizeof(double) * n_eigs);
        n_found[r] = nf2[j];
        if (rank) rank[r] = rk2[j];
    }
    return DACP_OK;
}

dacp_status dacp_get_moments(dacp_handle c, int r, double* mu, int64_t cap, int64_t* count) {
    TRY(check_handle(c));
    if (c->state < 3) return fail(c, DACP_ERR_STATE, "no moments yet");
    if (r < 0 || r >= c->R || !mu) return fail(c, DACP_ERR_ARG, "bad realization or buffer");
    const int b = c->b;
    const int rows = 2 * c->kn[r] + 2;
    const int64_t nvals = static_cast<int64_t>(rows) * b * b;
    if (count) *count = nvals;
    if (cap < nvals) return fail(c, DACP_ERR_ARG, "capacity %lld < %lld", (long long)cap, (long long)nvals);
    double *mus = nullptr, *nus = nullptr;
    int* bad = nullptr;
    auto run = [&]() -> dacp_status {
        TRY(dalloc_t(c, &mus, static_cast<size_t>(nvals)));
        TRY(dalloc_t(c, &nus, static_cast<size_t>(nvals)));
        TRY(dalloc_t(c, &bad, 1));
        CK(cudaMemsetAsync(bad, 0, sizeof(int), c->st));
        CK(launch_moments(c->mom_d + c->info[r].mom_off * b * b, rows, b, c->emax[r], mus, nus, bad, c->st));
        c->launches += 1;
        CK(cudaMemcpyAsync(mu, mus, sizeof(double) * nvals, cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        return DACP_OK;
    };
    dacp_status s = run();
    dfree(c, mus);
    dfree(c, nus);
    dfree(c, bad);
    return s;
}

dacp_status dacp_get_filtered(dacp_handle c, int r, double* psi, int64_t cap) {
    TRY(check_handle(c));
    if (c->state < 2) return fail(c, DACP_ERR_STATE, "no filtered vectors yet");
    if (r < 0 || r >= c->R || !psi) return fail(c, DACP_ERR_ARG, "bad realization or buffer");
    const int64_t n = (static_cast<int64_t>(1) << c->N[r]) * c->b;
    if (cap < n) return fail(c, DACP_ERR_ARG, "capacity too small");
    double* tmp = nullptr;
    auto run = [&]() -> dacp_status {
        TRY(dalloc_t(c, &tmp, static_cast<size_t>(n)));
        const char* src = static_cast<const char*>(c->psiE_d) + static_cast<size_t>(c->info[r].off) * c->b * c->esz;
        CK(launch_to_double(c->prec, src, tmp, n, c->b, c->st));
        c->launches += 1;
        CK(cudaMemcpyAsync(psi, tmp, sizeof(double) * n, cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        return DACP_OK;
    };
    dacp_status s = run();
    dfree(c, tmp);
    return s;
}

}  // extern "C"

namespace {

// Selected Ritz pairs of realization r (device): the coefficients
// Bsel = U Y[:, first:first+cnt] (M x cnt, column-major) of the Ritz vectors
// phi_j = sum_(i,p) Bsel[i*b+p, j] T_{x_i}(G) psi_p, their eigenvalues lam
// (cnt, ascending) and, when want_h2, the H^2 matrix H2 (M x M) assembled
// from omega_k = <psi|H^2 T_k|psi>. cnt < 0 is -dacp_status of a failed
// realization. The buffers are the caller's to free (ritz_free).
struct Ritz {
    int M = 0, cnt = 0;
    double *Bsel = nullptr, *lam = nullptr, *H2 = nullptr;
    std::vector<void*> tmp;
};

void ritz_free(dacp_ctx* c, Ritz& z) {
    cudaStreamSynchronize(c->st);
    for (void* p : z.tmp) dfree(c, p);
    z = Ritz();
}

dacp_status ritz_select(dacp_ctx* c, int r, int n_eigs, double window, double eps, bool want_h2, Ritz& z) {
    const int b = c->b, Ln = 2 * c->n[r] + 1, M = b * Ln;
    const int rows = 2 * c->kn[r] + 4;          // mu_0 .. mu_{2 k_n + 3}
    const int64_t bb = static_cast<int64_t>(b) * b, MM = static_cast<int64_t>(M) * M;
    z.M = M;
    auto get = [&](auto** p, size_t count) -> dacp_status {
        TRY(dalloc_t(c, p, count));
        z.tmp.push_back(*p);
        return DACP_OK;
    };
    double *mus, *nus, *om, *S, *H, *W, *Ht, *lam, *lamt;
    int *orders, *ints;
    TRY(get(&mus, static_cast<size_t>(rows * bb)));
    TRY(get(&nus, static_cast<size_t>(rows * bb)));
    TRY(get(&S, static_cast<size_t>(MM)));
    TRY(get(&H, static_cast<size_t>(MM)));
    TRY(get(&W, static_cast<size_t>(MM)));
    TRY(get(&Ht, static_cast<size_t>(MM)));
    TRY(get(&lam, M));
    TRY(get(&lamt, M));
    TRY(get(&orders, Ln));
    TRY(get(&ints, 8));                          // bad, m, info, first, count
    if (want_h2) {
        TRY(get(&om, static_cast<size_t>(rows * bb)));
        TRY(get(&z.H2, static_cast<size_t>(MM)));
    }
    size_t d1 = 0, h1 = 0;
    CKS(cusolverDnXsyevd_bufferSize(c->sol, c->sp, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, M, CUDA_R_64F, S,
                                    M, CUDA_R_64F, lam, CUDA_R_64F, &d1, &h1));
    void* work = nullptr;
    TRY(dalloc(c, &work, std::max<size_t>(d1, 8)));
    z.tmp.push_back(work);
    std::vector<char> work_h(std::max<size_t>(h1, 1));
    CK(cudaMemsetAsync(ints, 0, 8 * sizeof(int), c->st));
    CK(launch_orders(Ln, c->a[r] / c->emax[r], orders, c->st));
    CK(launch_moments(c->mom_d + c->info[r].mom_off * bb, rows, b, c->emax[r], mus, nus, ints + 0, c->st));
    CK(launch_assemble(Ln, b, orders, mus, nus, S, H, c->st));
    if (want_h2) {
        // H2 from omega (S is written again with the same values)
        CK(launch_omega(mus, rows - 2, b, c->emax[r], om, c->st));
        CK(launch_assemble(Ln, b, orders, mus, om, S, z.H2, c->st));
    }
    CKS(cusolverDnXsyevd(c->sol, c->sp, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, M, CUDA_R_64F, S, M,
                         CUDA_R_64F, lam, CUDA_R_64F, work, d1, work_h.data(), h1, ints + 2));
    CK(launch_cutoff(lam, M, eps, 0, S, ints + 1, c->st));
    c->launches += want_h2 ? 6 : 4;
    int hv[3] = {0, 0, 0};
    CK(cudaMemcpyAsync(hv, ints, 3 * sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (hv[0]) { z.cnt = -DACP_ERR_NUMERIC; return DACP_OK; }
    if (hv[2] != 0 || hv[1] < 1) { z.cnt = -DACP_ERR_NOT_CONVERGED; return DACP_OK; }
    const int m = hv[1];
    const double* U = S + static_cast<int64_t>(M - m) * M;
    const double one = 1.0, zero = 0.0;
    CKB(cublasDgemm(c->blas, CUBLAS_OP_N, CUBLAS_OP_N, M, m, M, &one, H, M, U, M, &zero, W, M));
    CKB(cublasDgemm(c->blas, CUBLAS_OP_T, CUBLAS_OP_N, m, m, M, &one, U, M, W, M, &zero, Ht, m));
    size_t d2 = 0, h2 = 0;
    CKS(cusolverDnXsyevd_bufferSize(c->sol, c->sp, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, m, CUDA_R_64F, Ht,
                                    m, CUDA_R_64F, lamt, CUDA_R_64F, &d2, &h2));
    if (d2 > d1) {
        CK(cudaStreamSynchronize(c->st));
        TRY(dalloc(c, &work, d2));
        z.tmp.push_back(work);
        d1 = d2;
    }
    if (h2 > work_h.size()) work_h.resize(h2);
    // H~ = Y diag(lamt) Y^T; Y overwrites Ht
    CKS(cusolverDnXsyevd(c->sol, c->sp, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, m, CUDA_R_64F, Ht, m,
                         CUDA_R_64F, lamt, CUDA_R_64F, work, d1, work_h.data(), h2, ints + 2));
    const double w = window > 0.0 ? window : c->a[r];
    CK(launch_select_range(lamt, m, n_eigs, w, ints + 3, c->st));
    c->launches += 1;
    CK(cudaMemcpyAsync(hv, ints + 2, 3 * sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (hv[0] != 0) { z.cnt = -DACP_ERR_NOT_CONVERGED; return DACP_OK; }
    const int first = hv[1], cnt = hv[2];
    z.cnt = cnt;
    if (cnt < 1) return DACP_OK;
    TRY(get(&z.Bsel, static_cast<size_t>(M) * cnt));
    // b_j = U y_j for the selected columns of Y
    CKB(cublasDgemm(c->blas, CUBLAS_OP_N, CUBLAS_OP_N, M, cnt, m, &one, U, M, Ht + static_cast<int64_t>(first) * m, m,
                    &zero, z.Bsel, M));
    z.lam = lamt + first;
    return DACP_OK;
}

}  // namespace

extern "C" {

dacp_status dacp_residuals(dacp_handle c, int r, int n_eigs, double window, double eps, double* eigs, double* resid,
                           int* n_found) {
    NvtxRange nvtx_("dacp_residuals");
    TRY(check_handle(c));
    if (c->state < 3) return fail(c, DACP_ERR_STATE, "dacp_residuals before dacp_basis_moments");
    if (r < 0 || r >= c->R || n_eigs < 1 || !eigs || !resid || !n_found)
        return fail(c, DACP_ERR_ARG, "bad realization or output arguments");
    if (!(eps > 0.0)) eps = c->fp32 ? kEpsFp32 : (c->prec == kPrecDF32 ? kEpsDf32 : 1e-12);
    Ritz z;
    auto run = [&]() -> dacp_status {
        TRY(ritz_select(c, r, n_eigs, window, eps, true, z));
        *n_found = z.cnt;
        if (z.cnt < 1) return DACP_OK;
        const int M = z.M, cnt = z.cnt;
        double *W2 = nullptr, *rs = nullptr;
        TRY(dalloc_t(c, &W2, static_cast<size_t>(M) * cnt));
        z.tmp.push_back(W2);
        TRY(dalloc_t(c, &rs, cnt));
        z.tmp.push_back(rs);
        const double one = 1.0, zero = 0.0;
        CKB(cublasDgemm(c->blas, CUBLAS_OP_N, CUBLAS_OP_N, M, cnt, M, &one, z.H2, M, z.Bsel, M, &zero, W2, M));
        CK(launch_residual(z.Bsel, W2, M, cnt, z.lam, rs, c->st));
        c->launches += 1;
        CK(cudaMemcpyAsync(eigs, z.lam, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->st));
        CK(cudaMemcpyAsync(resid, rs, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        return DACP_OK;
    };
    dacp_status s = run();
    ritz_free(c, z);
    return s;
}

dacp_status dacp_eigenvectors(dacp_handle c, int r, int n_eigs, double window, double eps, double* eigs,
                              double* phi_dev, int64_t ld, int* n_found) {
    NvtxRange nvtx_("dacp_eigenvectors");
    TRY(check_handle(c));
    if (c->state < 3) return fail(c, DACP_ERR_STATE, "dacp_eigenvectors before dacp_basis_moments");
    if (r < 0 || r >= c->R || n_eigs < 1 || !eigs || !phi_dev || !n_found)
        return fail(c, DACP_ERR_ARG, "bad realization or output arguments");
    const int64_t D = static_cast<int64_t>(1) << c->N[r];
    if (ld < D) return fail(c, DACP_ERR_ARG, "ld %lld < 2^N = %lld", (long long)ld, (long long)D);
    if (reinterpret_cast<uintptr_t>(phi_dev) & 7) return fail(c, DACP_ERR_ARG, "phi_dev must be 8-byte aligned");
    if (!(eps > 0.0)) eps = c->fp32 ? kEpsFp32 : (c->prec == kPrecDF32 ? kEpsDf32 : 1e-12);
    const int b = c->b, Ln = 2 * c->n[r] + 1;
    Ritz z;
    double* V = nullptr;
    auto run = [&]() -> dacp_status {
        TRY(ritz_select(c, r, n_eigs, window, eps, false, z));
        *n_found = z.cnt;
        if (z.cnt < 1) return DACP_OK;
        const int M = z.M, cnt = z.cnt;
        // basis orders x_i on the host (the same list the device kernel builds)
        std::vector<int> x(Ln);
        {
            int* od = nullptr;
            TRY(dalloc_t(c, &od, Ln));
            z.tmp.push_back(od);
            CK(launch_orders(Ln, c->a[r] / c->emax[r], od, c->st));
            CK(cudaMemcpyAsync(x.data(), od, sizeof(int) * Ln, cudaMemcpyDeviceToHost, c->st));
            CK(cudaStreamSynchronize(c->st));
        }
        // V = [T_{x_0} psi_E, T_{x_1} psi_E, ...], float64, column (i*b + p) of length 2^N
        TRY(dalloc_t(c, &V, static_cast<size_t>(D) * M));
        z.tmp.push_back(V);
        const size_t shift = static_cast<size_t>(c->info[r].off) * b * c->esz;
        char* A = static_cast<char*>(c->A_d) + shift;
        char* Bv = static_cast<char*>(c->B_d) + shift;
        const size_t bytes = static_cast<size_t>(D) * b * c->esz;
        // replay the evolution of realization r alone, w_0 = psi_E
        TRY(set_evolution_coef(c, c->emax));
        CK(cudaMemcpyAsync(A, static_cast<const char*>(c->psiE_d) + shift, bytes, cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemsetAsync(c->step_ctr_d, 0, sizeof(int), c->st));
        int next = 0;
        if (x[0] == 0) {
            CK(launch_gather_basis(c->prec, b, A, D, V, D, 0, c->st));
            next = 1;
        }
        StepArgs a = base_args(c);
        const int i0 = c->info[r].item_begin, ni = c->info[r].item_count;
        for (int k = 0; next < Ln; ++k) {
            CK(launch_step(c->prec, b, kEvolve, a, i0, ni, c->smem, c->st));   // w_{k+1}
            c->launches += 1;
            while (next < Ln && x[next] == k + 1) {
                CK(launch_gather_basis(c->prec, b, (k & 1) ? A : Bv, D, V, D, next * b, c->st));
                c->launches += 1;
                ++next;
            }
        }
        const double one = 1.0, zero = 0.0;
        CKB(cublasDgemm(c->blas, CUBLAS_OP_N, CUBLAS_OP_N, static_cast<int>(D), cnt, M, &one, V, static_cast<int>(D),
                        z.Bsel, M, &zero, phi_dev, static_cast<int>(ld)));
        CK(cudaMemcpyAsync(eigs, z.lam, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        TRY(check_device_flag(c));
        return DACP_OK;
    };
    dacp_status s = run();
    ritz_free(c, z);
    if (s != DACP_OK) return s;
    // restore the filter coefficients; the moments of r were rewritten with the same values
    TRY(apply_params(c));
    c->state = 3;
    return DACP_OK;
}


// The comparison method of Appendix D on this library's kernels: a Krylov
// space of the filtered operator T_K(F) (each new direction one dacp_filter of
// a single-column handle of realization r, then classical Gram-Schmidt twice
// against all earlier directions with cuBLAS), Rayleigh-Ritz of H in it, and
// the converged Ritz values.
dacp_status dacp_lanczos_filtered(dacp_handle c, int r, int steps, int n_eigs, double res_tol, double* eigs,
                                  int* n_found, int* dim_out, double* ms_out, int64_t* hv_out) {
    NvtxRange nvtx_("dacp_lanczos_filtered");
    TRY(check_handle(c));
    if (c->state < 1) return fail(c, DACP_ERR_STATE, "dacp_lanczos_filtered before parameters");
    if (r < 0 || r >= c->R || n_eigs < 1 || !eigs || !n_found) return fail(c, DACP_ERR_ARG, "bad arguments");
    const int N = c->N[r];
    const int64_t D = static_cast<int64_t>(1) << N;
    if (steps < 1 || steps > 4096 || steps > D) return fail(c, DACP_ERR_ARG, "steps must be in [1, min(4096, 2^N)]");
    if (!(res_tol > 0.0)) res_tol = 1e-8;
    // directions below this part of |A v_j| are the filter's own rounding, not Krylov directions
    const double thr = c->fp32 ? 1e-4 : 1e-8;
    const int b = c->b;
    // the single-column handle: realization r's couplings, fields, pair terms and start column 0
    std::vector<double> J(static_cast<size_t>(N) * N), hz(N), gx(N), v0(static_cast<size_t>(D));
    for (int i = 0; i < N; ++i) {
        hz[i] = c->h_h[static_cast<size_t>(r) * kMaxSpins + i];
        gx[i] = c->g_h[static_cast<size_t>(r) * kMaxSpins + i];
        for (int j = 0; j < N; ++j)
            J[static_cast<size_t>(i) * N + j] = c->J_h[static_cast<size_t>(r) * kMaxSpins * kMaxSpins + i * kMaxSpins + j];
    }
    int64_t off = 0, joff = 0;
    for (int q = 0; q < r; ++q) {
        off += (static_cast<int64_t>(1) << c->N[q]) * b;
        joff += static_cast<int64_t>(c->N[q]) * c->N[q];
    }
    double nrm0 = 0.0;
    for (int64_t s2 = 0; s2 < D; ++s2) {
        v0[s2] = c->psi0_h[off + s2 * b];
        nrm0 += v0[s2] * v0[s2];
    }
    if (!(nrm0 > 0.0)) return fail(c, DACP_ERR_ARG, "start column 0 of realization %d is zero", r);
    for (auto& x : v0) x /= sqrt(nrm0);
    dacp_handle S = nullptr;
    dacp_status st = dacp_create(&S, 1, &N, J.data(), hz.data(), gx.data(), 1, c->prec, v0.data(), c->st);
    if (st != DACP_OK) return fail(c, st, "single-column handle: set-up failed");
    double* V = nullptr;
    double* HV = nullptr;
    double* Y = nullptr;
    double* HY = nullptr;
    double* w = nullptr;
    double* hbuf = nullptr;
    double* Hm = nullptr;
    double* Hs = nullptr;
    double* lam = nullptr;
    double* res = nullptr;
    double* conv = nullptr;
    double* sel = nullptr;
    int* ints = nullptr;
    void* xbuf = nullptr;
    void* ybuf = nullptr;
    void* work = nullptr;
    auto run = [&]() -> dacp_status {
        if (c->has_pairs) {
            std::vector<double> jx(c->jxx_h.begin() + joff, c->jxx_h.begin() + joff + static_cast<int64_t>(N) * N);
            std::vector<double> jy(c->jyy_h.begin() + joff, c->jyy_h.begin() + joff + static_cast<int64_t>(N) * N);
            TRY(dacp_set_pair_couplings(S, jx.data(), jy.data()));
        }
        if (c->has_gflip) TRY(dacp_set_global_flips(S, &c->gflip_h[r]));
        const int one = 1, K = c->K[r];
        TRY(dacp_set_params(S, &c->emax[r], &c->a[r], &K, &one));
        const int m = steps;
        TRY(dalloc_t(c, &V, static_cast<size_t>(D) * m));
        TRY(dalloc_t(c, &HV, static_cast<size_t>(D) * m));
        TRY(dalloc_t(c, &w, static_cast<size_t>(D)));
        TRY(dalloc_t(c, &hbuf, static_cast<size_t>(m)));
        TRY(dalloc_t(c, &lam, static_cast<size_t>(m)));
        TRY(dalloc_t(c, &res, static_cast<size_t>(m)));
        TRY(dalloc_t(c, &conv, static_cast<size_t>(m)));
        TRY(dalloc_t(c, &sel, static_cast<size_t>(n_eigs)));
        TRY(dalloc_t(c, &ints, 2));
        TRY(dalloc(c, &xbuf, static_cast<size_t>(D) * c->esz + 64));
        TRY(dalloc(c, &ybuf, static_cast<size_t>(D) * c->esz + 64));
        CK(cudaMemcpyAsync(V, v0.data(), sizeof(double) * D, cudaMemcpyHostToDevice, c->st));
        const double one_d = 1.0, zero_d = 0.0, mone_d = -1.0;
        double t_filter = 0.0, t_orth = 0.0;
        int dim = 1;
        for (int j = 0; j + 1 < m; ++j) {
            // w = T_K(F) v_j / |T_K(F) v_j|
            CK(launch_convert(c->prec, V + static_cast<int64_t>(j) * D, S->psi0_d, D, c->st));
            TRY(dacp_filter(S));
            t_filter += S->t_ms[0];
            CK(cudaEventRecord(c->ev[2], c->st));
            CK(launch_to_double(c->prec, S->psiE_d, w, D, 1, c->st));
            c->launches += 2;
            // classical Gram-Schmidt against v_0 .. v_j, twice
            for (int pass = 0; pass < 2; ++pass) {
                CKB(cublasDgemv(c->blas, CUBLAS_OP_T, static_cast<int>(D), j + 1, &one_d, V, static_cast<int>(D), w, 1,
                                &zero_d, hbuf, 1));
                CKB(cublasDgemv(c->blas, CUBLAS_OP_N, static_cast<int>(D), j + 1, &mone_d, V, static_cast<int>(D), hbuf, 1,
                                &one_d, w, 1));
            }
            double nrm = 0.0;
            CKB(cublasDnrm2(c->blas, static_cast<int>(D), w, 1, &nrm));
            CK(cudaEventRecord(c->ev[3], c->st));
            CK(cudaStreamSynchronize(c->st));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]));
            t_orth += ms;
            if (!(nrm >= thr)) break;                 // the space is exhausted (or the filter broke)
            const double inv = 1.0 / nrm;
            CKB(cublasDscal(c->blas, static_cast<int>(D), &inv, w, 1));
            CK(cudaMemcpyAsync(V + static_cast<int64_t>(j + 1) * D, w, sizeof(double) * D, cudaMemcpyDeviceToDevice,
                               c->st));
            ++dim;
        }
        // Rayleigh-Ritz of H in the space
        CK(cudaEventRecord(c->ev[4], c->st));
        for (int j = 0; j < dim; ++j) {
            CK(launch_convert(c->prec, V + static_cast<int64_t>(j) * D, xbuf, D, c->st));
            TRY(dacp_apply_h(S, 0, xbuf, ybuf));
            CK(launch_to_double(c->prec, ybuf, HV + static_cast<int64_t>(j) * D, D, 1, c->st));
            c->launches += 2;
        }
        TRY(dalloc_t(c, &Hm, static_cast<size_t>(dim) * dim));
        TRY(dalloc_t(c, &Hs, static_cast<size_t>(dim) * dim));
        TRY(dalloc_t(c, &Y, static_cast<size_t>(D) * dim));
        TRY(dalloc_t(c, &HY, static_cast<size_t>(D) * dim));
        CKB(cublasDgemm(c->blas, CUBLAS_OP_T, CUBLAS_OP_N, dim, dim, static_cast<int>(D), &one_d, V, static_cast<int>(D),
                        HV, static_cast<int>(D), &zero_d, Hm, dim));
        const double half = 0.5;
        CKB(cublasDgeam(c->blas, CUBLAS_OP_N, CUBLAS_OP_T, dim, dim, &half, Hm, dim, &half, Hm, dim, Hs, dim));
        size_t dbytes = 0, hbytes = 0;
        CKS(cusolverDnXsyevd_bufferSize(c->sol, c->sp, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, dim, CUDA_R_64F,
                                        Hs, dim, CUDA_R_64F, lam, CUDA_R_64F, &dbytes, &hbytes));
        TRY(dalloc(c, &work, dbytes + 64));
        std::vector<char> work_h(hbytes + 64);
        CKS(cusolverDnXsyevd(c->sol, c->sp, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, dim, CUDA_R_64F, Hs, dim,
                             CUDA_R_64F, lam, CUDA_R_64F, work, dbytes, work_h.data(), hbytes, ints + 1));
        // residuals of the Ritz pairs: |H V z - theta V z|
        CKB(cublasDgemm(c->blas, CUBLAS_OP_N, CUBLAS_OP_N, static_cast<int>(D), dim, dim, &one_d, V, static_cast<int>(D),
                        Hs, dim, &zero_d, Y, static_cast<int>(D)));
        CKB(cublasDgemm(c->blas, CUBLAS_OP_N, CUBLAS_OP_N, static_cast<int>(D), dim, dim, &one_d, HV,
                        static_cast<int>(D), Hs, dim, &zero_d, HY, static_cast<int>(D)));
        CK(launch_ritz_residual(HY, Y, lam, D, dim, res, c->st));
        CK(launch_compact_converged(lam, res, dim, res_tol * c->emax[r], conv, ints, c->st));
        int host_ints[2] = {0, 0};
        CK(cudaMemcpyAsync(host_ints, ints, sizeof(int) * 2, cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        if (host_ints[1] != 0) return fail(c, DACP_ERR_NOT_CONVERGED, "Rayleigh-Ritz eigensolve: info %d", host_ints[1]);
        CK(launch_select(conv, host_ints[0], n_eigs, c->a[r], sel, ints + 1, c->st));
        c->launches += 3;
        int nf = 0;
        CK(cudaMemcpyAsync(&nf, ints + 1, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        if (nf > 0) {
            CK(cudaMemcpyAsync(eigs, sel, sizeof(double) * nf, cudaMemcpyDeviceToHost, c->st));
        }
        CK(cudaEventRecord(c->ev[5], c->st));
        CK(cudaStreamSynchronize(c->st));
        float ms_rr = 0.f;
        CK(cudaEventElapsedTime(&ms_rr, c->ev[4], c->ev[5]));
        *n_found = nf;
        if (dim_out) *dim_out = dim;
        if (ms_out) {
            ms_out[0] = t_filter;
            ms_out[1] = t_orth;
            ms_out[2] = ms_rr;
        }
        if (hv_out) *hv_out = static_cast<int64_t>(dim - 1) * 2 * K + dim;
        c->launches += S->launches.load();
        return DACP_OK;
    };
    dacp_status s2 = run();
    for (void* p : {static_cast<void*>(V), static_cast<void*>(HV), static_cast<void*>(Y), static_cast<void*>(HY),
                    static_cast<void*>(w), static_cast<void*>(hbuf), static_cast<void*>(Hm), static_cast<void*>(Hs),
                    static_cast<void*>(lam), static_cast<void*>(res), static_cast<void*>(conv), static_cast<void*>(sel),
                    static_cast<void*>(ints), xbuf, ybuf, work})
        if (p) dfree(c, p);
    if (s2 != DACP_OK && S) {
        const std::string msg = dacp_last_error(S);
        if (!msg.empty() && c->err.empty()) fail(c, s2, "single-column handle: %s", msg.c_str());
    }
    dacp_destroy(S);
    return s2;
}

dacp_status dacp_apply_h(dacp_handle c, int r, const void* x_dev, void* y_dev) {
    TRY(check_handle(c));
    if (r < 0 || r >= c->R || !x_dev || !y_dev || x_dev == y_dev) return fail(c, DACP_ERR_ARG, "bad arguments");
    if ((reinterpret_cast<uintptr_t>(x_dev) & 15) || (reinterpret_cast<uintptr_t>(y_dev) & 15))
        return fail(c, DACP_ERR_ARG, "x and y must be 16-byte aligned");
    StepArgs a = base_args(c);
    a.coef = c->apply_coef_d;
    // the kernel indexes x and y by the batch offset of realization r
    const size_t shift = static_cast<size_t>(c->info[r].off) * c->b * c->esz;
    a.x = static_cast<const char*>(x_dev) - shift;
    a.y1 = nullptr;
    a.out = static_cast<char*>(y_dev) - shift;
    CK(launch_step(c->prec, c->b, kApply, a, c->info[r].item_begin, c->info[r].item_count, c->smem, c->st));
    c->launches += 1;
    CK(cudaStreamSynchronize(c->st));
    return check_device_flag(c);
}

// Bytes of the largest vector tile at tile_bytes (as tile_geometry sets c->smem).
static int tile_smem_for(const dacp_ctx* c, int tile_bytes) {
    int tb_cap = 0;
    while ((static_cast<int64_t>(2) << tb_cap) * c->b * static_cast<int64_t>(c->esz) <= tile_bytes) ++tb_cap;
    int max_tstates = 1;
    for (int r = 0; r < c->R; ++r) max_tstates = std::max(max_tstates, 1 << std::min(c->info[r].N, tb_cap));
    return static_cast<int>(max_tstates * c->b * c->esz);
}

// Launch mode 2 (staged tiles) runs float32 vectors whose staged tiles fit shared memory.
static bool staged_possible(const dacp_ctx* c, int tile_bytes) {
    return c->prec == kPrecF32 && staged_fits(c->b, tile_smem_for(c, tile_bytes));
}

// Tile sizes the autotuner tries, and its cache keyed by (sizes, b, precision).
static const int kTileCandidates[] = {8192, 16384, 32768, 65536, 131072};
static const int kNumTiles = 5;
static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune_cache;

dacp_status dacp_autotune(dacp_handle c, int orders, int* tile_bytes_out) {
    NvtxRange nvtx_("dacp_autotune");
    TRY(check_handle(c));
    if (c->state < 1) return fail(c, DACP_ERR_STATE, "dacp_autotune before parameters");
    if (orders < 4 || orders > 100000) return fail(c, DACP_ERR_ARG, "orders out of range");
    std::vector<int> ns = c->N;
    std::sort(ns.begin(), ns.end());
    std::string key = std::to_string(c->b) + "p" + std::to_string(c->prec);
    for (int v : ns) key += "," + std::to_string(v);
    int best = -1;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) best = it->second;
    }
    if (best < 0) {
        const size_t vec_bytes = static_cast<size_t>(c->Dtot) * c->b * c->esz;
        double best_ms = 1e300;
        for (int cand = 0; cand < 3 * kNumTiles; ++cand) {
            const int tb = kTileCandidates[cand % kNumTiles];
            if (cand / kNumTiles == 2 && !staged_possible(c, tb)) continue;
            c->launch_mode = cand / kNumTiles;
            TRY(retile(c, tb));
            TRY(set_evolution_coef(c, c->emax));
            CK(cudaMemcpyAsync(c->A_d, c->psi0_d, vec_bytes, cudaMemcpyDeviceToDevice, c->st));
            TRY(run_orders(c, false, kGraphOrders));         // warm-up; captures the graph
            CK(cudaMemcpyAsync(c->A_d, c->psi0_d, vec_bytes, cudaMemcpyDeviceToDevice, c->st));
            CK(cudaEventRecord(c->ev[0], c->st));
            TRY(run_orders(c, false, orders));
            CK(cudaEventRecord(c->ev[1], c->st));
            CK(cudaStreamSynchronize(c->st));
            TRY(check_device_flag(c));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
            if (ms < best_ms) {
                best_ms = ms;
                best = cand;
            }
        }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    c->launch_mode = best / kNumTiles;
    TRY(retile(c, kTileCandidates[best % kNumTiles]));
    TRY(apply_params(c));          // filter coefficients back; results must be recomputed
    if (tile_bytes_out) *tile_bytes_out = kTileCandidates[best % kNumTiles];
    return DACP_OK;
}

dacp_status dacp_set_launch(dacp_handle c, int mode, int tile_bytes) {
    TRY(check_handle(c));
    if (mode < 0 || mode > 2) return fail(c, DACP_ERR_ARG, "launch mode must be 0, 1 or 2");
    if (tile_bytes < 1024 || tile_bytes > 131072 || (tile_bytes & (tile_bytes - 1)))
        return fail(c, DACP_ERR_ARG, "tile_bytes must be a power of two in [1 KB, 128 KB]");
    if (mode == 2 && c->prec != kPrecF32) return fail(c, DACP_ERR_ARG, "launch mode 2 runs float32 vectors only");
    if (mode == 2 && !staged_possible(c, tile_bytes))
        return fail(c, DACP_ERR_ARG, "staged tiles of %d bytes exceed shared memory", tile_bytes);
    c->launch_mode = mode;
    TRY(retile(c, tile_bytes));
    if (c->state > 1) c->state = 1;
    return DACP_OK;
}

dacp_status dacp_set_pair_couplings(dacp_handle c, const double* Jxx, const double* Jyy) {
    TRY(check_handle(c));
    std::vector<int> np(c->R, 0), ij(static_cast<size_t>(c->R) * kMaxPairs, 0);
    std::vector<double> cf(static_cast<size_t>(c->R) * kMaxPairs * 2, 0.0);
    std::vector<double> pn(c->R, 0.0);
    int64_t jo = 0;
    for (int r = 0; r < c->R; ++r) {
        const int Nr = c->N[r];
        for (int i = 0; i < Nr; ++i)
            for (int j = i + 1; j < Nr; ++j) {
                const double x = Jxx ? Jxx[jo + static_cast<int64_t>(i) * Nr + j] : 0.0;
                const double y = Jyy ? Jyy[jo + static_cast<int64_t>(i) * Nr + j] : 0.0;
                if (!isfinite(x) || !isfinite(y)) return fail(c, DACP_ERR_ARG, "non-finite pair coupling");
                if (x == 0.0 && y == 0.0) continue;
                const size_t t = static_cast<size_t>(r) * kMaxPairs + np[r]++;
                ij[t] = i | (j << 8);
                cf[2 * t] = x - y;          // bits i and j equal: z_i z_j = +1
                cf[2 * t + 1] = x + y;      // bits differ: z_i z_j = -1
                pn[r] += fabs(x) + fabs(y);
            }
        jo += static_cast<int64_t>(Nr) * Nr;
    }
    c->pnorm_pairs = pn;
    for (int r = 0; r < c->R; ++r)
        pn[r] += c->pnorm0[r] + (c->has_gflip ? fabs(c->gflip_h[r]) : 0.0);
    bool any = false;
    for (int r = 0; r < c->R; ++r) any = any || np[r] > 0;
    if (any && !c->n_pairs_d) {
        TRY(dalloc_t(c, &c->n_pairs_d, static_cast<size_t>(c->R)));
        TRY(dalloc_t(c, &c->pair_ij_d, ij.size()));
        TRY(dalloc_t(c, &c->pair_c_d, cf.size()));
    }
    if (any) {
        CK(cudaMemcpyAsync(c->n_pairs_d, np.data(), sizeof(int) * np.size(), cudaMemcpyHostToDevice, c->st));
        CK(cudaMemcpyAsync(c->pair_ij_d, ij.data(), sizeof(int) * ij.size(), cudaMemcpyHostToDevice, c->st));
        CK(cudaMemcpyAsync(c->pair_c_d, cf.data(), sizeof(double) * cf.size(), cudaMemcpyHostToDevice, c->st));
    }
    c->pnorm = pn;
    CK(cudaMemcpyAsync(c->pnorm_d, c->pnorm.data(), sizeof(double) * c->R, cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->has_pairs = any;
    c->jxx_h.clear();
    c->jyy_h.clear();
    if (any) {
        c->jxx_h.assign(static_cast<size_t>(jo), 0.0);
        c->jyy_h.assign(static_cast<size_t>(jo), 0.0);
        if (Jxx) c->jxx_h.assign(Jxx, Jxx + jo);
        if (Jyy) c->jyy_h.assign(Jyy, Jyy + jo);
    }
    for (Graph* g : {&c->gf, &c->ge}) {          // captured launches hold the old arguments
        if (g->exec) cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
    }
    c->state = 0;                                 // H changed: parameters and results are stale
    return DACP_OK;
}

dacp_status dacp_set_global_flips(dacp_handle c, const double* coef) {
    TRY(check_handle(c));
    std::vector<double> g(c->R, 0.0);
    bool any = false;
    for (int r = 0; r < c->R && coef; ++r) {
        if (!isfinite(coef[r])) return fail(c, DACP_ERR_ARG, "non-finite global-flip coefficient");
        g[r] = coef[r];
        any = any || coef[r] != 0.0;
    }
    if (any && !c->gflip_d) TRY(dalloc_t(c, &c->gflip_d, static_cast<size_t>(c->R)));
    if (any) CK(cudaMemcpyAsync(c->gflip_d, g.data(), sizeof(double) * c->R, cudaMemcpyHostToDevice, c->st));
    c->gflip_h = g;
    c->has_gflip = any;
    for (int r = 0; r < c->R; ++r)
        c->pnorm[r] = c->pnorm0[r] + (c->pnorm_pairs.empty() ? 0.0 : c->pnorm_pairs[r]) + fabs(g[r]);
    CK(cudaMemcpyAsync(c->pnorm_d, c->pnorm.data(), sizeof(double) * c->R, cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    for (Graph* gr : {&c->gf, &c->ge}) {         // captured launches hold the old arguments
        if (gr->exec) cudaGraphExecDestroy(gr->exec);
        gr->exec = nullptr;
    }
    c->state = 0;                                 // H changed: parameters and results are stale
    return DACP_OK;
}

dacp_status dacp_create_parity_sectors(dacp_handle* out, int n_real, const int* n_spins, const double* J,
                                       const double* h, const double* gamma, int block_b, int precision,
                                       const double* psi0, void* stream) {
    if (!out) return DACP_ERR_ARG;
    *out = nullptr;
    if (n_real <= 0 || !n_spins || !J || !h || !gamma || !psi0) return DACP_ERR_ARG;
    int64_t jo = 0, ho = 0;
    std::vector<int> ns;
    std::vector<double> Js, hs, gs, gf;
    for (int r = 0; r < n_real; ++r) {
        const int N = n_spins[r];
        if (N < 2 || N > kMaxSpins) return DACP_ERR_ARG;
        for (int i = 0; i < N; ++i)
            if (h[ho + i] != 0.0) return DACP_ERR_ARG;           // a z-field breaks the parity symmetry
        for (int sigma = 1; sigma >= -1; sigma -= 2) {
            const int M = N - 1;
            ns.push_back(M);
            for (int i = 0; i < M; ++i)
                for (int j = 0; j < M; ++j) Js.push_back(j > i ? J[jo + static_cast<int64_t>(i) * N + j] : 0.0);
            for (int i = 0; i < M; ++i) {
                hs.push_back(J[jo + static_cast<int64_t>(i) * N + (N - 1)]);    // z_{N-1} = +1 on the representatives
                gs.push_back(gamma[ho + i]);
            }
            gf.push_back(sigma * gamma[ho + N - 1]);
        }
        jo += static_cast<int64_t>(N) * N;
        ho += N;
    }
    dacp_handle c = nullptr;
    dacp_status st = dacp_create(&c, 2 * n_real, ns.data(), Js.data(), hs.data(), gs.data(), block_b, precision, psi0,
                                 stream);
    if (st != DACP_OK) return st;
    st = dacp_set_global_flips(c, gf.data());
    if (st != DACP_OK) {
        dacp_destroy(c);
        return st;
    }
    c->sector_pairs = true;
    *out = c;
    return DACP_OK;
}

dacp_status dacp_merge_sectors(int n_real, int n_in, const double* eigs_in, const int* n_found_in, int n_eigs,
                               double* eigs, int* n_found) {
    if (n_real <= 0 || n_in < 1 || n_eigs < 1 || !eigs_in || !n_found_in || !eigs || !n_found) return DACP_ERR_ARG;
    for (int r = 0; r < n_real; ++r) {
        const int a = 2 * r, b = 2 * r + 1;
        if (n_found_in[a] < 0 || n_found_in[b] < 0) {          // a failed sector fails the realization
            n_found[r] = n_found_in[a] < 0 ? n_found_in[a] : n_found_in[b];
            continue;
        }
        // every level of a sector inside the largest |E| it returned came back: the union is complete
        // up to the smaller of the two radii
        double cover = 1e300;
        std::vector<double> all;
        for (int s2 : {a, b}) {
            const int nf = std::min(n_found_in[s2], n_in);
            double m = 0.0;
            for (int i = 0; i < nf; ++i) {
                const double v = eigs_in[static_cast<int64_t>(s2) * n_in + i];
                all.push_back(v);
                m = std::max(m, fabs(v));
            }
            cover = std::min(cover, m);
        }
        std::stable_sort(all.begin(), all.end(), [](double x, double y) {
            return fabs(x) < fabs(y) || (fabs(x) == fabs(y) && x < y);
        });
        int cnt = 0;
        for (double v : all) {
            if (cnt == n_eigs || fabs(v) > cover) break;
            eigs[static_cast<int64_t>(r) * n_eigs + cnt++] = v;
        }
        std::sort(eigs + static_cast<int64_t>(r) * n_eigs, eigs + static_cast<int64_t>(r) * n_eigs + cnt);
        n_found[r] = cnt;
    }
    return DACP_OK;
}

dacp_status dacp_solve_sectors(dacp_handle c, dacp_mlp net, int n_eigs, int n_sector, double* eigs, int* n_found,
                               int* n_redone) {
    NvtxRange nvtx_("dacp_solve_sectors");
    TRY(check_handle(c));
    if (!c->sector_pairs) return fail(c, DACP_ERR_ARG, "not a parity-sector handle (dacp_create_parity_sectors)");
    if (n_eigs < 1 || n_sector < 1 || n_sector > n_eigs || !eigs || !n_found)
        return fail(c, DACP_ERR_ARG, "need 1 <= n_sector <= n_eigs and output buffers");
    const int nm = c->R / 2;
    if (n_redone) *n_redone = 0;
    std::vector<double> es(static_cast<size_t>(c->R) * n_sector, 0.0);
    std::vector<int> nfs(c->R, 0);
    if (net) {
        TRY(dacp_solve_learned(c, net, n_sector, 0.0, 0.0, es.data(), nfs.data(), nullptr, nullptr));
    } else {
        TRY(dacp_choose_params(c, n_sector, 2.0, 1.5, 0.0, 20, 256));
        TRY(dacp_solve(c, n_sector, 0.0, 0.0, es.data(), nfs.data(), nullptr));
    }
    TRY(dacp_merge_sectors(nm, n_sector, es.data(), nfs.data(), n_eigs, eigs, n_found));
    // models whose merge came up short (or whose sectors failed): both sectors again, each asked for
    // all n_eigs levels, so the union's n_eigs central levels lie inside both returned radii
    std::vector<int> redo_m, redo_r;
    for (int m = 0; m < nm; ++m)
        if (n_found[m] < n_eigs) {
            redo_m.push_back(m);
            redo_r.push_back(2 * m);
            redo_r.push_back(2 * m + 1);
        }
    if (n_redone) *n_redone = static_cast<int>(redo_m.size());
    if (redo_m.empty()) return DACP_OK;
    const int nr = static_cast<int>(redo_r.size());
    dacp_handle sub = nullptr;
    dacp_status st = sub_handle(c, redo_r, &sub);
    if (st != DACP_OK) return fail(c, st, "sector re-run: set-up failed");
    std::vector<double> e2(static_cast<size_t>(nr) * n_eigs, 0.0), em(static_cast<size_t>(nr / 2) * n_eigs, 0.0);
    std::vector<int> nf2(nr, 0), nfm(nr / 2, 0);
    st = dacp_set_emax_rule(sub, 0);                 // the true bound: also recovers a rule-1 failure
    if (st == DACP_OK) st = dacp_choose_params(sub, n_eigs, 2.0, 1.5, 0.0, 20, 256);
    if (st == DACP_OK) st = dacp_solve(sub, n_eigs, 0.0, 0.0, e2.data(), nf2.data(), nullptr);
    if (st != DACP_OK) {
        const std::string msg = dacp_last_error(sub);
        dacp_destroy(sub);
        return fail(c, st, "sector re-run: %s", msg.c_str());
    }
    c->launches += sub->launches.load();
    dacp_destroy(sub);
    TRY(dacp_merge_sectors(nr / 2, n_eigs, e2.data(), nf2.data(), n_eigs, em.data(), nfm.data()));
    for (size_t j = 0; j < redo_m.size(); ++j) {
        const int m = redo_m[j];
        memcpy(eigs + static_cast<size_t>(m) * n_eigs, em.data() + j * n_eigs, sizeof(double) * n_eigs);
        n_found[m] = nfm[j];
    }
    return DACP_OK;
}

dacp_status dacp_set_emax_rule(dacp_handle c, int rule) {
    TRY(check_handle(c));
    if (rule != 0 && rule != 1) return fail(c, DACP_ERR_ARG, "E_max rule must be 0 or 1");
    c->emax_rule = rule;
    return DACP_OK;
}

dacp_status dacp_set_solver(dacp_handle c, int mode) {
    TRY(check_handle(c));
    if (mode != 0 && mode != 1) return fail(c, DACP_ERR_ARG, "solver mode must be 0 or 1");
    c->batched_solve = mode == 1;
    return DACP_OK;
}

dacp_status dacp_test_fail_alloc(int64_t after) {
    g_alloc_countdown.store(after < 0 ? -1 : after);
    return DACP_OK;
}

dacp_status dacp_test_poison_barrier(dacp_handle c) {
    TRY(check_handle(c));
    c->poison_barrier = true;
    return DACP_OK;
}

dacp_status dacp_get_launch(dacp_handle c, int* mode, int* tile_bytes) {
    TRY(check_handle(c));
    if (mode) *mode = c->launch_mode;
    if (tile_bytes) *tile_bytes = c->tile_bytes;
    return DACP_OK;
}

dacp_status dacp_get_launch_count(dacp_handle c, int64_t* count) {
    TRY(check_handle(c));
    if (!count) return DACP_ERR_ARG;
    *count = c->launches;
    return DACP_OK;
}

dacp_status dacp_get_timings(dacp_handle c, double* ms) {
    TRY(check_handle(c));
    if (!ms) return DACP_ERR_ARG;
    for (int i = 0; i < 3; ++i) ms[i] = c->t_ms[i];
    return DACP_OK;
}

}  // extern "C"
