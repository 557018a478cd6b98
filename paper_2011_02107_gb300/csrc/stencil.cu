// Fused matrix-free H.v stencil + Chebyshev three-term recurrence + moments.
//
// One CTA owns one tile of 2^tbits consecutive basis states of one
// realization. The tile of the vector H acts on is staged in shared memory;
// a bit flip s -> s ^ 2^i with i < tbits reads the partner from the tile,
// with i >= tbits from the partner tile in global memory (L2 resident when the
// vector is). The diagonal (sum J_ij z_i z_j + sum h_i z_i) is read per state.
//
//   kApply   out = c_h H x + c_1 y1                       (test hook, Lanczos)
//   kFilter1 u = H w_k                                     (Sec. II A, F = (H^2-E_c)/E_0)
//   kFilter2 w_{k+1} = c_h H u + c_1 w_k + c_2 w_{k-1}     c_h = 2/E_0, c_1 = -2E_c/E_0, c_2 = -1
//   kEvolve  w_{k+1} = c_h H w_k + c_1 w_{k-1}             c_h = 2/E_max, c_1 = -1 (Sec. II B)
// Order 0 uses its own coefficients (T_1 = x): 1/E_0, -E_c/E_0, 0 and 1/E_max, 0.
//
// kEvolve also emits the moment rows P_2k = <w_k, w_k> and P_{2k+1} =
// <w_{k+1}, w_k> (b x b blocks, float64). With T_2k = 2T_k^2 - 1 and
// T_{2k+1} = 2T_{k+1}T_k - T_1, mu_j = 2 P_j - P_{j mod 2} (Appendix C moments
// without a second pass). Per-tile partials are reduced by the last CTA of
// each realization in tile order, so the result does not depend on scheduling.
//
// The order k is read from a device counter that the last CTA of a launch
// advances, so the same launch can be captured once and replayed in a CUDA
// graph; the two vector buffers swap roles by the parity of k and the write of
// w_{k+1} goes in place over w_{k-1} (each element is read and written by the
// same thread; partners are only read from w_k).

#include <string.h>

#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "common.cuh"
#include "ops.h"

namespace dacp {

// Per-thread moment accumulation: float32 over the thread's short run (then
// float64 across threads), float64 as is, and the Dot2 compensated sum for
// double-float values.
template <typename T> struct MomOps {
    using acc = T;
    __device__ static acc zero() { return T(0); }
    __device__ static void mad(acc& s, T a, T b) { s = fma(a, b, s); }
    __device__ static double to_double(acc s) { return static_cast<double>(s); }
    __device__ static df32 to_df(acc s) { return df32(static_cast<float>(s), 0.f); }   // float32 only
};
template <> struct MomOps<df32> {
    using acc = Dot2;
    __device__ static acc zero() { return dot2_zero(); }
    __device__ static void mad(acc& s, df32 a, df32 b) { dot2_mad(s, a, b); }
    __device__ static double to_double(acc s) { return static_cast<double>(s.hi) + static_cast<double>(s.err); }
    __device__ static df32 to_df(acc s) { return dot2_final(s); }
};

// L2-coherent scalar load, and read-only scalar load.
template <typename T>
__device__ __forceinline__ T ld_cg(const T* p) { return __ldcg(p); }
template <>
__device__ __forceinline__ df32 ld_cg<df32>(const df32* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return df32(v.x, v.y);
}
template <typename T>
__device__ __forceinline__ T ld_ro(const T* p) { return __ldg(p); }
template <>
__device__ __forceinline__ df32 ld_ro<df32>(const df32* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return df32(v.x, v.y);
}

template <typename T, int B>
__device__ __forceinline__ void load_vals(const T* __restrict__ p, T (&v)[B]) {
#pragma unroll
    for (int q = 0; q < B; ++q) v[q] = p[q];
}

template <typename T, int B>
__device__ __forceinline__ void load_vals_ro(const T* __restrict__ p, T (&v)[B]) {
#pragma unroll
    for (int q = 0; q < B; ++q) v[q] = __ldg(p + q);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ df32 shfl_xor_df(df32 v, int o) {
    return df32(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

// Sums V = 2^v double-float values per lane over the lanes of a warp and
// scatters the totals (a reduce-scatter butterfly): at each of the first v
// levels (lane offsets 16, 8, ...) a lane keeps the half of its values that its
// lane bit selects and adds the partner's copy of that half; the offsets left,
// down to OMIN, sum the one value kept. On return (OMIN = 1) lane L holds the
// total of value L / (32 / V), every lane of a group of 32 / V the same; with
// OMIN > 1 lanes that differ below OMIN keep separate sums. For V = 32 this is
// 31 double-float additions per lane on the float32 pipes, where a float64
// butterfly per value takes 5 V float64 additions: GB300 issues float64 at
// 1/64 of the float32 rate, and that once-per-tile reduction used to bound the
// float32 evolution kernel.
template <int V, int OMIN = 1>
__device__ __forceinline__ df32 warp_reduce_scatter(df32 (&x)[V], const int lane) {
    static_assert((V & (V - 1)) == 0 && V <= 32 / OMIN, "V a power of two, at most the lanes summed over");
#pragma unroll
    for (int half = V / 2, o = 16; half >= 1; half >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const df32 send = up ? x[i] : x[i + half];
            const df32 keep = up ? x[i + half] : x[i];
            x[i] = keep + shfl_xor_df(send, o);
        }
    }
    df32 v = x[0];
#pragma unroll
    for (int o = 16 / V; o >= OMIN; o >>= 1) v = v + shfl_xor_df(v, o);
    return v;
}

// 16-byte vector units: a unit holds kStates consecutive states x B columns
// (float32: 4 states at b = 1, 2 at b = 2, 1 at b = 4; float64: 2 states at
// b = 1, 1 at b = 2, one 32-byte state at b = 4). Bit flips inside a unit are
// register permutations; flips inside the tile read shared memory; flips
// beyond the tile read the partner unit from global memory (L2).
template <typename T, int B>
struct Unit {
    static constexpr int kBytes = (B * static_cast<int>(sizeof(T)) >= 16) ? B * static_cast<int>(sizeof(T)) : 16;
    static constexpr int kVals = kBytes / static_cast<int>(sizeof(T));
    static constexpr int kStates = kVals / B;
    static constexpr int kLog = kStates == 4 ? 2 : (kStates == 2 ? 1 : 0);
    static constexpr int kVec = kBytes / 16;          // float4 per unit
};

template <typename T, int B>
__device__ __forceinline__ void ld_unit(const T* p, T (&v)[Unit<T, B>::kVals]) {
#pragma unroll
    for (int q = 0; q < Unit<T, B>::kVec; ++q) {
        const float4 f = reinterpret_cast<const float4*>(p)[q];
        memcpy(reinterpret_cast<char*>(v) + 16 * q, &f, 16);
    }
}

template <typename T, int B>
__device__ __forceinline__ void ld_unit_nc(const T* p, T (&v)[Unit<T, B>::kVals]) {
#pragma unroll
    for (int q = 0; q < Unit<T, B>::kVec; ++q) {
        const float4 f = __ldg(reinterpret_cast<const float4*>(p) + q);
        memcpy(reinterpret_cast<char*>(v) + 16 * q, &f, 16);
    }
}

// L2-coherent load (bypasses L1): for vectors rewritten inside one persistent launch.
template <typename T, int B>
__device__ __forceinline__ void ld_unit_cg(const T* p, T (&v)[Unit<T, B>::kVals]) {
#pragma unroll
    for (int q = 0; q < Unit<T, B>::kVec; ++q) {
        const float4 f = __ldcg(reinterpret_cast<const float4*>(p) + q);
        memcpy(reinterpret_cast<char*>(v) + 16 * q, &f, 16);
    }
}

template <typename T, int B, bool COHERENT>
__device__ __forceinline__ void ld_unit_g(const T* p, T (&v)[Unit<T, B>::kVals]) {
    if (COHERENT) ld_unit_cg<T, B>(p, v); else ld_unit_nc<T, B>(p, v);
}

template <typename T, int B, bool COHERENT>
__device__ __forceinline__ void ld_unit_rw(const T* p, T (&v)[Unit<T, B>::kVals]) {
    if (COHERENT) ld_unit_cg<T, B>(p, v); else ld_unit<T, B>(p, v);
}

template <typename T, int B>
__device__ __forceinline__ void st_unit(T* p, const T (&v)[Unit<T, B>::kVals]) {
#pragma unroll
    for (int q = 0; q < Unit<T, B>::kVec; ++q) {
        float4 f;
        memcpy(&f, reinterpret_cast<const char*>(v) + 16 * q, 16);
        reinterpret_cast<float4*>(p)[q] = f;
    }
}

// ---- TMA bulk copy of the tile into shared memory, with a bounded wait -----

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Several bulk copies completing on one barrier phase: one arrive that announces
// the bytes of all of them, then the copies themselves.
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bulk prefetch of [src, src + bytes) into L2 (no shared memory, no barrier):
// src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

constexpr uint64_t kWaitNs = 1000000000ull;   // bounded waits give up after one second

// Wait for the barrier phase `parity`; false when kWaitNs pass first.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int /*unused*/) {
    const uint64_t t0 = global_ns();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
}

constexpr int kWaitLimit = 0;         // (time-based: kWaitNs)
// Units per thread in flight: two for float32; one for the 8-byte types,
// whose units and accumulators already use twice the registers.
template <typename T> struct UnitsPerPass { static constexpr int value = sizeof(T) == 4 ? 2 : 1; };
// Minimum resident CTAs per SM the compiler must allow: three for float32
// (80 registers, no spills), two for the 8-byte types (128 registers; three
// would spill their double-float / float64 accumulators at one thread per
// state).
template <typename T, int B> struct MinBlocks { static constexpr int value = sizeof(T) == 4 ? 3 : 2; };
// double-float at b = 4 runs two threads per state (tile_step_df4): three CTAs per SM
template <> struct MinBlocks<df32, 4> { static constexpr int value = 3; };
// Beyond-tile partner units whose loads are issued before the in-tile flips,
// so that their L2 latency overlaps the shared-memory work: three for
// double-float, whose long in-tile flip phase hides them; none otherwise.
template <typename T> struct EarlyGlobal { static constexpr int value = 0; };
template <> struct EarlyGlobal<df32> { static constexpr int value = 3; };
constexpr int kMaxTileUnitBits = 14;   // unit bits of the largest tile (128 KB of float32 b = 1)
constexpr int kMaxGlobalBitsUnrolled = 10;

// One tile of one realization at order `step`. COHERENT = the vectors may have
// been rewritten earlier in the same (persistent) launch: global reads then
// bypass L1. STAGED = every HBM read of the tile (x, the recurrence's y1 / y2
// and the diagonal) lands in shared memory through bulk copies on one barrier
// phase at the start, so a CTA has its whole input in flight at once instead
// of a few 16-byte loads per thread; dynamic shared memory then holds
// [x | y1 | y2 (kFilter2) | diagonal] (see staged_smem_bytes).
template <typename T, int B, int MODE, bool COHERENT, bool STAGED = false>
__device__ __forceinline__ void tile_step(const StepArgs& a, const int item, const int step) {
    using U = Unit<T, B>;
    constexpr int VU = U::kVals, SU = U::kStates, LS = U::kLog, UP = UnitsPerPass<T>::value;
    constexpr bool kEarlyY = sizeof(T) == 4;     // prefetch y1 / y2 before the flips (float32 only)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* tile = reinterpret_cast<T*>(smem_raw);
    __shared__ T gam_s[kMaxSpins + 1];             // x-fields, then the global-flip coefficient
    __shared__ double red_s[kThreads / 32][2 * B * B];
    __shared__ int last_s;
    __shared__ __align__(8) uint64_t bar_s;

    const int tid = threadIdx.x;
    const Item it = a.items[item];
    const RealInfo R = a.real[it.r];
    int nsteps = (MODE == kEvolve) ? R.ne : (MODE == kApply ? 1 : R.nf);
    if (MODE != kApply && a.nsteps_override > 0) nsteps = a.nsteps_override;
    const bool active = step < nsteps;
    const bool want_mom = (MODE == kEvolve) || (MODE == kApply && a.apply_moments);
    // <w_{k+1}, w_k> is symmetric in the columns; float32 storage rounding makes
    // the computed block asymmetric at 1e-7, and averaging both triangles (the
    // moments kernel symmetrises) halves that noise, so float32 keeps both.
    constexpr bool kSymOX = MODE == kEvolve && sizeof(T) != 4;

    using MO = MomOps<T>;
    using AC = Accum<T>;
    typename MO::acc xx[B][B], ox[B][B];
#pragma unroll
    for (int p = 0; p < B; ++p)
#pragma unroll
        for (int q = 0; q < B; ++q) { xx[p][q] = MO::zero(); ox[p][q] = MO::zero(); }

    if (active) {
        T* wA = static_cast<T*>(a.bufA);
        T* wB = static_cast<T*>(a.bufB);
        T* wk = (step & 1) ? wB : wA;      // w_k
        T* wo = (step & 1) ? wA : wB;      // w_{k-1}, overwritten by w_{k+1}
        const T* x;
        const T* y1 = nullptr;
        const T* y2 = nullptr;
        T* out;
        double c_h, c_1 = 0.0, c_2 = 0.0;
        const double* cf = a.coef + 8 * it.r + (step == 0 ? 0 : 3);
        if (MODE == kApply) {
            x = static_cast<const T*>(a.x); y1 = static_cast<const T*>(a.y1); out = static_cast<T*>(a.out);
            c_h = cf[0]; c_1 = cf[1];
        } else if (MODE == kFilter1) {
            x = wk; out = static_cast<T*>(a.bufU); c_h = 1.0;
        } else if (MODE == kFilter2) {
            x = static_cast<const T*>(a.bufU); y1 = wk; y2 = wo; out = wo;
            c_h = cf[0]; c_1 = cf[1]; c_2 = cf[2];
        } else {
            x = wk; y1 = wo; out = wo;
            c_h = cf[0]; c_1 = cf[1];
        }
        const bool use1 = (c_1 != 0.0) && (y1 != nullptr);
        const bool use2 = (c_2 != 0.0) && (y2 != nullptr);
        const T ch = static_cast<T>(c_h), c1 = static_cast<T>(c_1), c2 = static_cast<T>(c_2);

        const int tstates = 1 << R.tbits;
        const int64_t tile0 = static_cast<int64_t>(it.tile) << R.tbits;   // first local state
        const int64_t gbase = R.off * B;                                  // first value of the realization
        const T* xg = x + gbase;
        const T* dg = static_cast<const T*>(a.diag) + R.off;
        // float64 / double-float: c_h folds into the x-fields and the diagonal,
        // acc = c_h H x directly. float32 scales the sum once at the end instead:
        // folding moves its rounding enough to tip the float32 moment floor.
        constexpr bool kFold = sizeof(T) != 4;
        if (tid < R.N) {
            const T g = static_cast<const T*>(a.gam)[it.r * kMaxSpins + tid];
            gam_s[tid] = kFold ? ch * g : g;
        }
        if (tid == kMaxSpins && a.gflip) {
            const T g = static_cast<T>(__ldg(a.gflip + it.r));
            gam_s[kMaxSpins] = kFold ? ch * g : g;
        }

        if (tstates >= SU) {
            // ---- unit path: stage the tile with one bulk copy -------------------
            const uint32_t nbytes = static_cast<uint32_t>(tstates) * B * sizeof(T);
            // staged reads need a diagonal tile of whole 16-byte lines (4 float32 states)
            const bool stg = STAGED && (static_cast<uint32_t>(tstates) * sizeof(T)) % 16u == 0u;
            const T* ys1 = tile + static_cast<int64_t>(tstates) * B;        // staged y1
            const T* ys2 = tile + 2 * static_cast<int64_t>(tstates) * B;    // staged y2 (kFilter2)
            constexpr int kNY = MODE == kFilter2 ? 2 : (MODE == kFilter1 ? 0 : 1);
            const T* dsg = tile + (1 + kNY) * static_cast<int64_t>(tstates) * B;   // staged diagonal
            if (tid == 0) {
                mbar_init(&bar_s, 1);
                if (stg) {
                    const uint32_t dbytes = static_cast<uint32_t>(tstates) * sizeof(T);
                    mbar_expect(&bar_s, nbytes * (1u + (use1 ? 1u : 0u) + (use2 ? 1u : 0u)) + dbytes);
                    bulk_copy(tile, xg + tile0 * B, nbytes, &bar_s);
                    if (use1) bulk_copy(const_cast<T*>(ys1), y1 + gbase + tile0 * B, nbytes, &bar_s);
                    if (use2) bulk_copy(const_cast<T*>(ys2), y2 + gbase + tile0 * B, nbytes, &bar_s);
                    bulk_copy(const_cast<T*>(dsg), dg + tile0, dbytes, &bar_s);
                } else {
                    bulk_load(tile, xg + tile0 * B, nbytes, &bar_s);
                }
            }
            __syncthreads();
            const bool landed = mbar_wait(&bar_s, 0, kWaitLimit);
            if (!landed) {
                atomicExch(a.err_flag, 1);
                mbar_wait(&bar_s, 0, kWaitLimit);        // let the copy land before the CTA exits
            }
            __syncthreads();
            if (tid == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar_s)) : "memory");
            if (!landed) goto reduce;
            const int nunits = tstates / SU;
            const int tub = R.tbits - LS;                // unit bits inside the tile
            for (int ub = 0; ub < nunits; ub += kThreads * UP) {
                int uu[UP];
                bool val[UP];
                T xv[UP][VU], yv[UP][VU], zv[UP][VU], dv[UP][SU];
                typename AC::type acc[UP][VU];
#pragma unroll
                for (int k = 0; k < UP; ++k) {
                    uu[k] = ub + k * kThreads + tid;
                    val[k] = uu[k] < nunits;
                    const int64_t s0 = tile0 + static_cast<int64_t>(uu[k]) * SU;
                    if (val[k]) {
                        ld_unit<T, B>(tile + uu[k] * VU, xv[k]);
                        if (STAGED && stg) {
                            if (use1) ld_unit<T, B>(ys1 + uu[k] * VU, yv[k]);
                            if (use2) ld_unit<T, B>(ys2 + uu[k] * VU, zv[k]);
#pragma unroll
                            for (int j = 0; j < SU; ++j)
                                dv[k][j] = kFold ? ch * dsg[uu[k] * SU + j] : dsg[uu[k] * SU + j];
                        } else {
                            if (kEarlyY && use1) ld_unit_rw<T, B, COHERENT>(y1 + gbase + s0 * B, yv[k]);
                            if (kEarlyY && use2) ld_unit_rw<T, B, COHERENT>(y2 + gbase + s0 * B, zv[k]);
#pragma unroll
                            for (int j = 0; j < SU; ++j)
                                dv[k][j] = kFold ? ch * ld_ro(dg + s0 + j) : ld_ro(dg + s0 + j);
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < UP; ++k)
#pragma unroll
                    for (int j = 0; j < SU; ++j)
#pragma unroll
                        for (int p = 0; p < B; ++p) acc[k][j * B + p] = AC::prod(dv[k][j], xv[k][j * B + p]);
                // flips inside the unit
#pragma unroll
                for (int i = 0; i < LS; ++i) {
                    const T g = gam_s[i];
#pragma unroll
                    for (int k = 0; k < UP; ++k)
#pragma unroll
                        for (int j = 0; j < SU; ++j)
#pragma unroll
                            for (int p = 0; p < B; ++p)
                                AC::mad(acc[k][j * B + p], g, xv[k][(j ^ (1 << i)) * B + p]);
                }
                // the first EG beyond-tile partners: loads issued now, summed after the tile flips
                constexpr int EG = EarlyGlobal<T>::value;
                const int ngb = R.N - R.tbits;
                int64_t sbase[UP];
                if (EG > 0) {   // (without early loads, set after the in-tile flips: fewer live registers)
#pragma unroll
                    for (int k = 0; k < UP; ++k) sbase[k] = val[k] ? tile0 + static_cast<int64_t>(uu[k]) * SU : tile0;
                }
                T pe[EG > 0 ? EG : 1][UP][VU];
#pragma unroll
                for (int j = 0; j < EG; ++j)
                    if (j < ngb)
#pragma unroll
                        for (int k = 0; k < UP; ++k)
                            ld_unit_g<T, B, COHERENT>(xg + (sbase[k] ^ (static_cast<int64_t>(1) << (R.tbits + j))) * B,
                                                      pe[j][k]);
                // flips inside the tile (shared memory). Unrolled at compile time and
                // predicated on the tile's bit count so that every partner load of a
                // unit is independent; idle slots read a masked, in-range address.
                const int umask = nunits - 1;
#pragma unroll
                for (int i = 0; i < kMaxTileUnitBits; ++i) {
                    if (i < tub) {
                        const T g = gam_s[LS + i];
#pragma unroll
                        for (int k = 0; k < UP; ++k) {
                            T pv[VU];
                            ld_unit<T, B>(tile + ((uu[k] ^ (1 << i)) & umask) * VU, pv);
#pragma unroll
                            for (int v = 0; v < VU; ++v) AC::mad(acc[k][v], g, pv[v]);
                        }
                    }
                }
                // flips beyond the tile (global memory, L2-resident partner tiles)
                if (EG == 0) {
#pragma unroll
                    for (int k = 0; k < UP; ++k) sbase[k] = val[k] ? tile0 + static_cast<int64_t>(uu[k]) * SU : tile0;
                }
#pragma unroll
                for (int j = 0; j < EG; ++j) {
                    if (j < ngb) {
                        const T g = gam_s[R.tbits + j];
#pragma unroll
                        for (int k = 0; k < UP; ++k)
#pragma unroll
                            for (int v = 0; v < VU; ++v) AC::mad(acc[k][v], g, pe[j][k][v]);
                    }
                }
#pragma unroll
                for (int j = EG; j < kMaxGlobalBitsUnrolled; ++j) {
                    if (j < ngb) {
                        const T g = gam_s[R.tbits + j];
                        T pv[UP][VU];
#pragma unroll
                        for (int k = 0; k < UP; ++k)
                            ld_unit_g<T, B, COHERENT>(xg + (sbase[k] ^ (static_cast<int64_t>(1) << (R.tbits + j))) * B, pv[k]);
#pragma unroll
                        for (int k = 0; k < UP; ++k)
#pragma unroll
                            for (int v = 0; v < VU; ++v) AC::mad(acc[k][v], g, pv[k][v]);
                    }
                }
                for (int j = kMaxGlobalBitsUnrolled; j < ngb; ++j) {
                    const T g = gam_s[R.tbits + j];
#pragma unroll
                    for (int k = 0; k < UP; ++k) {
                        T pv[VU];
                        ld_unit_g<T, B, COHERENT>(xg + (sbase[k] ^ (static_cast<int64_t>(1) << (R.tbits + j))) * B, pv);
#pragma unroll
                        for (int v = 0; v < VU; ++v) AC::mad(acc[k][v], g, pv[v]);
                    }
                }
                // two-body flips X_i X_j, Y_i Y_j: partner s XOR (2^i + 2^j) with coefficient
                // Jxx - Jyy z_i(s) z_j(s); element by element, from the tile when both bits lie
                // inside it, else from global memory
                const int npair = a.n_pairs ? a.n_pairs[it.r] : 0;
                for (int t = 0; t < npair; ++t) {
                    const int ij = __ldg(a.pair_ij + it.r * kMaxPairs + t);
                    const int pi = ij & 255, pj = ij >> 8;
                    const double* pc = a.pair_c + (static_cast<int64_t>(it.r) * kMaxPairs + t) * 2;
                    const T ceq = kFold ? ch * static_cast<T>(__ldg(pc)) : static_cast<T>(__ldg(pc));
                    const T cne = kFold ? ch * static_cast<T>(__ldg(pc + 1)) : static_cast<T>(__ldg(pc + 1));
                    const int64_t msk = (static_cast<int64_t>(1) << pi) | (static_cast<int64_t>(1) << pj);
                    const bool inside = pj < R.tbits;
#pragma unroll
                    for (int k = 0; k < UP; ++k) {
                        if (!val[k]) continue;
#pragma unroll
                        for (int js = 0; js < SU; ++js) {
                            const int64_t sl = static_cast<int64_t>(uu[k]) * SU + js;   // state within the tile
                            const int64_t sx = tile0 + sl;
                            const T cf2 = (((sx >> pi) ^ (sx >> pj)) & 1) ? cne : ceq;
#pragma unroll
                            for (int col = 0; col < B; ++col) {
                                const T xp = inside ? tile[(sl ^ msk) * B + col]
                                                    : (COHERENT ? ld_cg(xg + (sx ^ msk) * B + col)
                                                                : ld_ro(xg + (sx ^ msk) * B + col));
                                AC::mad(acc[k][js * B + col], cf2, xp);
                            }
                        }
                    }
                }
                // global flip X_0 ... X_{N-1}: partner s XOR (2^N - 1); within a unit of SU
                // states the partners run backwards, so one unit's worth is read element by element
                if (a.gflip) {
                    const T gf = gam_s[kMaxSpins];
                    const int64_t fm = (static_cast<int64_t>(1) << R.N) - 1;
#pragma unroll
                    for (int k = 0; k < UP; ++k) {
                        if (!val[k]) continue;
                        const int64_t s0 = tile0 + static_cast<int64_t>(uu[k]) * SU;
                        if constexpr (SU == 1) {
                            T pv[VU];
                            ld_unit_g<T, B, COHERENT>(xg + (s0 ^ fm) * B, pv);
#pragma unroll
                            for (int v = 0; v < VU; ++v) AC::mad(acc[k][v], gf, pv[v]);
                        } else {
#pragma unroll
                            for (int js = 0; js < SU; ++js) {
#pragma unroll
                                for (int col = 0; col < B; ++col) {
                                    const int64_t e = ((s0 + js) ^ fm) * B + col;
                                    const T xp = COHERENT ? ld_cg(xg + e) : ld_ro(xg + e);
                                    AC::mad(acc[k][js * B + col], gf, xp);
                                }
                            }
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < UP; ++k) {
                    if (!val[k]) continue;
                    if (!kEarlyY && !(STAGED && stg)) {
                        const int64_t sy = tile0 + static_cast<int64_t>(uu[k]) * SU;
                        if (use1) ld_unit_rw<T, B, COHERENT>(y1 + gbase + sy * B, yv[k]);
                        if (use2) ld_unit_rw<T, B, COHERENT>(y2 + gbase + sy * B, zv[k]);
                    }
                    T o[VU];
#pragma unroll
                    for (int v = 0; v < VU; ++v) {
                        typename AC::type t = acc[k][v];
                        if (!kFold) t = AC::prod(ch, AC::final(acc[k][v]));
                        if (use1) AC::mad(t, c1, yv[k][v]);
                        if (use2) AC::mad(t, c2, zv[k][v]);
                        o[v] = AC::final(t);
                    }
                    const int64_t s0 = tile0 + static_cast<int64_t>(uu[k]) * SU;
                    st_unit<T, B>(out + gbase + s0 * B, o);
                    if (want_mom) {
#pragma unroll
                        for (int j = 0; j < SU; ++j)
#pragma unroll
                            for (int p = 0; p < B; ++p)
#pragma unroll
                                for (int q = 0; q < B; ++q) {
                                    const T xq = xv[k][j * B + q];
                                    // <x_p, x_q> is symmetric, and so is <T_{k+1} psi_p, T_k psi_q>
                                    // (T_{k+1} T_k is a symmetric polynomial in H): only q >= p
                                    if (q >= p) MO::mad(xx[p][q], xv[k][j * B + p], xq);
                                    if (q >= p || !kSymOX) MO::mad(ox[p][q], o[j * B + p], xq);
                                }
                    }
                }
            }
        } else {
            // ---- scalar path for vectors smaller than one unit (N = 1) ----------
            for (int i = tid; i < tstates * B; i += kThreads) tile[i] = COHERENT ? ld_cg(xg + tile0 * B + i) : xg[tile0 * B + i];
            __syncthreads();
            for (int sl = tid; sl < tstates; sl += kThreads) {
                const int64_t s = tile0 + sl;
                T xv[B], acc[B];
                load_vals<T, B>(tile + sl * B, xv);
                const T d = kFold ? ch * dg[s] : dg[s];
#pragma unroll
                for (int p = 0; p < B; ++p) acc[p] = d * xv[p];
                for (int i = 0; i < R.tbits; ++i) {
                    const T g = gam_s[i];
                    const T* q = tile + (sl ^ (1 << i)) * B;
#pragma unroll
                    for (int p = 0; p < B; ++p) acc[p] = fma(g, q[p], acc[p]);
                }
                if (a.gflip) {                       // global flip: the whole realization is this tile
                    const T gf = gam_s[kMaxSpins];
                    const T* q = tile + (sl ^ ((1 << R.N) - 1)) * B;
#pragma unroll
                    for (int p = 0; p < B; ++p) acc[p] = fma(gf, q[p], acc[p]);
                }
                T o[B];
#pragma unroll
                for (int p = 0; p < B; ++p) {
                    T t = kFold ? acc[p] : ch * acc[p];
                    if (use1) t = fma(c1, COHERENT ? ld_cg(y1 + gbase + s * B + p) : y1[gbase + s * B + p], t);
                    if (use2) t = fma(c2, COHERENT ? ld_cg(y2 + gbase + s * B + p) : y2[gbase + s * B + p], t);
                    o[p] = t;
                }
#pragma unroll
                for (int p = 0; p < B; ++p) out[gbase + s * B + p] = o[p];
                if (want_mom) {
#pragma unroll
                    for (int p = 0; p < B; ++p)
#pragma unroll
                        for (int q = 0; q < B; ++q) {
                            if (q >= p) MO::mad(xx[p][q], xv[p], xv[q]);
                            if (q >= p || !kSymOX) MO::mad(ox[p][q], o[p], xv[q]);
                        }
                }
            }
        }
    }

reduce:
    if (want_mom && active) {
        const int lane = tid & 31, warp = tid >> 5;
        if constexpr (std::is_same<T, double>::value) {
#pragma unroll
            for (int p = 0; p < B; ++p)
#pragma unroll
                for (int q = 0; q < B; ++q) {
                    const double v1 = warp_sum(MO::to_double(xx[p < q ? p : q][p < q ? q : p]));
                    const double v2 = warp_sum(MO::to_double(kSymOX ? ox[p < q ? p : q][p < q ? q : p] : ox[p][q]));
                    if (lane == 0) { red_s[warp][p * B + q] = v1; red_s[warp][B * B + p * B + q] = v2; }
                }
        } else {
            // float32 / double-float partials: the warp sum runs in double-float arithmetic
            constexpr int V = 2 * B * B, G = 32 / V;
            df32 xv[V];
#pragma unroll
            for (int p = 0; p < B; ++p)
#pragma unroll
                for (int q = 0; q < B; ++q) {
                    xv[p * B + q] = MO::to_df(xx[p < q ? p : q][p < q ? q : p]);
                    xv[B * B + p * B + q] = MO::to_df(kSymOX ? ox[p < q ? p : q][p < q ? q : p] : ox[p][q]);
                }
            const df32 t = warp_reduce_scatter<V>(xv, lane);
            if (lane % G == 0) red_s[warp][lane / G] = static_cast<double>(t);
        }
        __syncthreads();
        if (tid < 2 * B * B) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < kThreads / 32; ++w) s += red_s[w][tid];
            a.part[static_cast<int64_t>(item) * 2 * B * B + tid] = s;
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const unsigned prev = atomicAdd(&a.real_done[it.r], 1u);
            last_s = (prev == static_cast<unsigned>(R.item_count - 1));
        }
        __syncthreads();
        if (last_s) {
            __threadfence();
            if (tid < 2 * B * B) {
                double s = 0.0;
                for (int j = 0; j < R.item_count; ++j)
                    s += __ldcg(a.part + static_cast<int64_t>(R.item_begin + j) * 2 * B * B + tid);
                const int row = (MODE == kEvolve) ? 2 * step : 2 * a.apply_row;
                const int64_t row0 = a.mom_rows_fixed > 0
                                         ? static_cast<int64_t>(it.r) * a.mom_rows_fixed : R.mom_off;
                a.mom[(row0 + row) * B * B + tid] = s;
            }
            if (tid == 0) a.real_done[it.r] = 0u;
        }
    }

    __syncthreads();   // the tile buffer is reused by the next tile of a persistent CTA
}

// ---- double-float at b = 4: two threads per state ----------------------------
//
// The one-thread-per-state unit path holds a 32-byte unit and the b x b
// moment sums per thread, which caps it at two CTAs per SM (128 registers)
// and leaves shared-memory latency exposed. Here thread h of each pair holds
// columns 2h, 2h+1 of one state (16 bytes): half the registers, three CTAs
// per SM. Moment sums: thread h has its own x (a), its outputs o and, after
// one shuffle with the neighbouring lane, the other pair's x (c). It keeps
// ten sums: <a,a> and <o,a> within its pair (three each) and four cross sums,
// h = 0: <o_p, x_q> and h = 1: <x_p, x_q> for p in {0,1}, q in {2,3}. Only the
// evolution emits moments on this path (its <o, x> block is symmetric).

// A column pair of one state: 16 bytes (hi_p, hi_{p+1}, lo_p, lo_{p+1}) (VecAt<df32>).
__device__ __forceinline__ void ld2_s(const df32* p, df32& v0, df32& v1) {
    const float4 f = *reinterpret_cast<const float4*>(p);
    v0 = df32(f.x, f.z);
    v1 = df32(f.y, f.w);
}

template <bool COHERENT>
__device__ __forceinline__ void ld2_g(const df32* p, df32& v0, df32& v1) {
    const float4 f = COHERENT ? __ldcg(reinterpret_cast<const float4*>(p)) : __ldg(reinterpret_cast<const float4*>(p));
    v0 = df32(f.x, f.z);
    v1 = df32(f.y, f.w);
}

template <bool COHERENT>
__device__ __forceinline__ void ld2_rw(const df32* p, df32& v0, df32& v1) {
    const float4 f = COHERENT ? __ldcg(reinterpret_cast<const float4*>(p)) : *reinterpret_cast<const float4*>(p);
    v0 = df32(f.x, f.z);
    v1 = df32(f.y, f.w);
}

__device__ __forceinline__ void st2(df32* p, df32 v0, df32 v1) {
    *reinterpret_cast<float4*>(p) = make_float4(v0.hi, v1.hi, v0.lo, v1.lo);
}

static_assert((static_cast<int64_t>(1) << kMaxSpins) * 4 < (static_cast<int64_t>(1) << 31),
              "per-state offsets of the double-float b = 4 pass are 32-bit");
constexpr int kDf4TileBits = 12;   // in-tile flips unrolled: tiles up to 4096 states (128 KB)

// TB > 0: the tile has TB bits in every realization of the launch (compile-time
// flip loop); TB = 0: read from RealInfo.
template <int MODE, bool COHERENT, int TB = 0>
__device__ __forceinline__ void tile_step_df4(const StepArgs& a, const int item, const int step) {
    using T = df32;
    constexpr int B = 4, EG = EarlyGlobal<T>::value;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* tile = reinterpret_cast<T*>(smem_raw);
    __shared__ T gam_s[kMaxSpins];
    __shared__ double red_s[kThreads / 32][2 * B * B];
    __shared__ int last_s;
    __shared__ __align__(8) uint64_t bar_s;

    const int tid = threadIdx.x;
    const int h = tid & 1;
    const Item it = a.items[item];
    const RealInfo R = a.real[it.r];
    int nsteps = (MODE == kEvolve) ? R.ne : (MODE == kApply ? 1 : R.nf);
    if (MODE != kApply && a.nsteps_override > 0) nsteps = a.nsteps_override;
    const bool active = step < nsteps;
    constexpr bool want_mom = MODE == kEvolve;
    Dot2 ms[10];
#pragma unroll
    for (int e = 0; e < 10; ++e) ms[e] = dot2_zero();

    if (active) {
        T* wA = static_cast<T*>(a.bufA);
        T* wB = static_cast<T*>(a.bufB);
        T* wk = (step & 1) ? wB : wA;
        T* wo = (step & 1) ? wA : wB;
        const T* x;
        const T* y1 = nullptr;
        const T* y2 = nullptr;
        T* out;
        double c_h, c_1 = 0.0, c_2 = 0.0;
        const double* cf = a.coef + 8 * it.r + (step == 0 ? 0 : 3);
        if (MODE == kApply) {
            x = static_cast<const T*>(a.x); y1 = static_cast<const T*>(a.y1); out = static_cast<T*>(a.out);
            c_h = cf[0]; c_1 = cf[1];
        } else if (MODE == kFilter1) {
            x = wk; out = static_cast<T*>(a.bufU); c_h = 1.0;
        } else if (MODE == kFilter2) {
            x = static_cast<const T*>(a.bufU); y1 = wk; y2 = wo; out = wo;
            c_h = cf[0]; c_1 = cf[1]; c_2 = cf[2];
        } else {
            x = wk; y1 = wo; out = wo;
            c_h = cf[0]; c_1 = cf[1];
        }
        const bool use1 = (c_1 != 0.0) && (y1 != nullptr);
        const bool use2 = (c_2 != 0.0) && (y2 != nullptr);
        const T ch = static_cast<T>(c_h), c1 = static_cast<T>(c_1), c2 = static_cast<T>(c_2);

        const int tbits = TB > 0 ? TB : R.tbits;           // compile-time when specialised
        const int tstates = 1 << tbits;
        const int64_t tile0 = static_cast<int64_t>(it.tile) << tbits;
        const int64_t gbase = R.off * B;
        const T* xg = x + gbase;
        const T* y1g = (MODE != kFilter1 && y1) ? y1 + gbase : nullptr;   // kFilter1 has no y
        const T* y2g = (MODE == kFilter2 && y2) ? y2 + gbase : nullptr;   // only kFilter2 has a z
        T* outg = out + gbase;
        const T* dg = static_cast<const T*>(a.diag) + R.off;
        if (tid < R.N) gam_s[tid] = ch * static_cast<const T*>(a.gam)[it.r * kMaxSpins + tid];

        const uint32_t nbytes = static_cast<uint32_t>(tstates) * B * sizeof(T);
        if (tid == 0) {
            mbar_init(&bar_s, 1);
            bulk_load(tile, xg + tile0 * B, nbytes, &bar_s);
        }
        __syncthreads();
        const bool landed = mbar_wait(&bar_s, 0, kWaitLimit);
        if (!landed) {
            atomicExch(a.err_flag, 1);
            mbar_wait(&bar_s, 0, kWaitLimit);        // let the copy land before the CTA exits
        }
        __syncthreads();
        if (tid == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar_s)) : "memory");
        if (!landed) goto reduce_df4;

        const int ngb = R.N - tbits;
        const int nhalf = 2 * tstates;                   // (state, column pair) slots of the tile
        for (int hb = 0; hb < nhalf; hb += kThreads) {
            const int hs = hb + tid;
            // both lanes of a pair agree (nhalf is even); a specialised tile of >= 128 states fills every pass
            const bool val = (TB >= 7) || hs < nhalf;
            const int sl = val ? (hs >> 1) : 0;          // idle lanes work on state 0 and store nothing
            // state within the realization: N <= kMaxSpins keeps sg * B below 2^31, so the
            // per-state offsets are 32-bit and only the realization's base pointers are 64-bit
            const uint32_t sg = static_cast<uint32_t>(tile0) + static_cast<uint32_t>(sl);
            const int col = 2 * h;
            T a0, a1;
            ld2_s(tile + sl * B + col, a0, a1);
            T pe[EG > 0 ? EG : 1][2];
#pragma unroll
            for (int j = 0; j < EG; ++j)
                if (j < ngb) ld2_g<COHERENT>(xg + ((sg ^ (1u << (tbits + j))) * B + col), pe[j][0],
                                             pe[j][1]);
            // the diagonal and w_{k-1} are loaded now and used last, so their
            // latency hides under the in-tile flips
            const T dr = ld_ro(dg + sg);
            T y0 = T(0), y1v = T(0), z0 = T(0), z1 = T(0);
            if (MODE != kFilter1 && use1) ld2_rw<COHERENT>(y1g + (sg * B + col), y0, y1v);
            if (MODE == kFilter2 && use2) ld2_rw<COHERENT>(y2g + (sg * B + col), z0, z1);
            // flips inside the tile (shared memory); bit 0 starts the sums (tbits >= 1)
            Dot2 acc0, acc1;
            {
                const T g = gam_s[0];
                T p0, p1;
                ld2_s(tile + (sl ^ 1) * B + col, p0, p1);
                acc0 = Accum<T>::prod(g, p0);
                acc1 = Accum<T>::prod(g, p1);
            }
#pragma unroll
            for (int i = 1; i < (TB > 0 ? TB : kDf4TileBits); ++i) {
                if (TB > 0 || i < R.tbits) {
                    const T g = gam_s[i];
                    T p0, p1;
                    ld2_s(tile + (sl ^ (1 << i)) * B + col, p0, p1);
                    dot2_mad(acc0, g, p0);
                    dot2_mad(acc1, g, p1);
                }
            }
            for (int i = kDf4TileBits; TB == 0 && i < R.tbits; ++i) {
                const T g = gam_s[i];
                T p0, p1;
                ld2_s(tile + (sl ^ (1 << i)) * B + col, p0, p1);
                dot2_mad(acc0, g, p0);
                dot2_mad(acc1, g, p1);
            }
            // flips beyond the tile (global memory, L2-resident partner tiles)
#pragma unroll
            for (int j = 0; j < EG; ++j) {
                if (j < ngb) {
                    const T g = gam_s[tbits + j];
                    dot2_mad(acc0, g, pe[j][0]);
                    dot2_mad(acc1, g, pe[j][1]);
                }
            }
            for (int j = EG; j < ngb; ++j) {
                const T g = gam_s[tbits + j];
                T p0, p1;
                ld2_g<COHERENT>(xg + ((sg ^ (1u << (tbits + j))) * B + col), p0, p1);
                dot2_mad(acc0, g, p0);
                dot2_mad(acc1, g, p1);
            }
            if constexpr (TB == 0) {
                // two-body flips (the launch picks TB = 0 when the handle has them)
                const int npair = a.n_pairs ? a.n_pairs[it.r] : 0;
                for (int t = 0; t < npair; ++t) {
                    const int ij = __ldg(a.pair_ij + it.r * kMaxPairs + t);
                    const int pi = ij & 255, pj = ij >> 8;
                    const double* pc = a.pair_c + (static_cast<int64_t>(it.r) * kMaxPairs + t) * 2;
                    const uint32_t msk = (1u << pi) | (1u << pj);
                    const T cf2 = ch * T(__ldg(pc + (((sg >> pi) ^ (sg >> pj)) & 1u)));
                    T p0, p1;
                    if (pj < tbits) ld2_s(tile + (static_cast<uint32_t>(sl) ^ msk) * B + col, p0, p1);
                    else ld2_g<COHERENT>(xg + ((sg ^ msk) * B + col), p0, p1);
                    dot2_mad(acc0, cf2, p0);
                    dot2_mad(acc1, cf2, p1);
                }
            }
            if (a.gflip) {                                  // global flip X_0 ... X_{N-1}
                const double gfv = __ldg(a.gflip + it.r);
                if (gfv != 0.0) {
                    const T gf = ch * T(gfv);
                    const uint32_t fm = (R.N >= 32) ? 0xffffffffu : ((1u << R.N) - 1u);
                    T p0, p1;
                    ld2_g<COHERENT>(xg + ((sg ^ fm) * B + col), p0, p1);
                    dot2_mad(acc0, gf, p0);
                    dot2_mad(acc1, gf, p1);
                }
            }
            // diagonal term, then w_{k+1} = c_h H x + c_1 y + c_2 z
            const T d = ch * dr;
            dot2_mad(acc0, d, a0);
            dot2_mad(acc1, d, a1);
            if (MODE != kFilter1 && use1) {
                dot2_mad(acc0, c1, y0);
                dot2_mad(acc1, c1, y1v);
            }
            if (MODE == kFilter2 && use2) {
                dot2_mad(acc0, c2, z0);
                dot2_mad(acc1, c2, z1);
            }
            const T o0 = dot2_final(acc0), o1 = dot2_final(acc1);
            if (val) st2(outg + (sg * B + col), o0, o1);
            if (want_mom) {
                const T cx0 = shfl_xor_df(a0, 1), cx1 = shfl_xor_df(a1, 1);   // the other pair's x
                if (val) {
                    dot2_mad(ms[0], a0, a0);
                    dot2_mad(ms[1], a0, a1);
                    dot2_mad(ms[2], a1, a1);
                    dot2_mad(ms[3], o0, a0);
                    dot2_mad(ms[4], o0, a1);
                    dot2_mad(ms[5], o1, a1);
                    // p in {0,1}, q in {2,3}: h = 0 sums <o_p, x_q>, h = 1 sums <x_p, x_q>
                    const T u0 = h ? cx0 : o0, u1 = h ? cx1 : o1;
                    const T v0 = h ? a0 : cx0, v1 = h ? a1 : cx1;
                    dot2_mad(ms[6], u0, v0);
                    dot2_mad(ms[7], u0, v1);
                    dot2_mad(ms[8], u1, v0);
                    dot2_mad(ms[9], u1, v1);
                }
            }
        }
    }

reduce_df4:
    if (want_mom && active) {
        const int lane = tid & 31, warp = tid >> 5;
        // the ten sums of each pair half, over the 16 lanes of one parity, in
        // double-float arithmetic (reduce-scatter: lane L keeps sum (L >> 1) & 15)
        df32 xs[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) xs[e] = e < 10 ? dot2_final(ms[e]) : df32(0.f, 0.f);
        const df32 t = warp_reduce_scatter<16, 2>(xs, lane);
        const int e = (lane >> 1) & 15;          // h = lane & 1 is the thread's pair half
        if (e < 10) {
            // h = 0 holds columns 0, 1 and <o_p, x_q> across the pairs; h = 1 columns 2, 3 and <x_p, x_q>
            int blk, p, q;
            if (e < 6) {
                blk = e / 3;
                const int k = e % 3;
                p = 2 * h + (k == 2 ? 1 : 0);
                q = 2 * h + (k >= 1 ? 1 : 0);
            } else {
                blk = h == 0 ? 1 : 0;
                p = (e - 6) >> 1;
                q = 2 + ((e - 6) & 1);
            }
            const double v = static_cast<double>(t);
            double* rw = red_s[warp];
            rw[blk * B * B + p * B + q] = v;
            rw[blk * B * B + q * B + p] = v;
        }
        __syncthreads();
        if (tid < 2 * B * B) {
            double sm = 0.0;
#pragma unroll
            for (int w = 0; w < kThreads / 32; ++w) sm += red_s[w][tid];
            a.part[static_cast<int64_t>(item) * 2 * B * B + tid] = sm;
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const unsigned prev = atomicAdd(&a.real_done[it.r], 1u);
            last_s = (prev == static_cast<unsigned>(R.item_count - 1));
        }
        __syncthreads();
        if (last_s) {
            __threadfence();
            if (tid < 2 * B * B) {
                double sm = 0.0;
                for (int j = 0; j < R.item_count; ++j)
                    sm += __ldcg(a.part + static_cast<int64_t>(R.item_begin + j) * 2 * B * B + tid);
                const int row = 2 * step;
                const int64_t row0 = a.mom_rows_fixed > 0 ? static_cast<int64_t>(it.r) * a.mom_rows_fixed : R.mom_off;
                a.mom[(row0 + row) * B * B + tid] = sm;
            }
            if (tid == 0) a.real_done[it.r] = 0u;
        }
    }
    __syncthreads();   // the tile buffer is reused by the next tile of a persistent CTA
}

// ---- the same pass on paired float32 instructions ---------------------------
//
// Each thread's two columns are the two lanes of every .f32x2 instruction
// (DF2: one register pair holds both columns' hi parts, one their lo parts).
// Every arithmetic step is the scalar Dot2 step of tile_step_df4, in the same
// order, so the vectors and moments are bit-identical; the paired form halves
// the issue slots of the float32 work, which bounds this kernel. The factor
// -1 of w_{k-1} (evolution) and of w_{k-1} in the filter's second pass is a
// subtraction without a product. Tiles of TB bits in every realization, no
// two-body flips (those handles launch tile_step_df4 with TB = 0).

// The 16 bytes of a column pair are (hi_p, hi_{p+1} | lo_p, lo_{p+1}): the two
// register pairs of a DF2 as they are.
__device__ __forceinline__ DF2 ld_df2_s(const df32* p) {
    const ulonglong2 f = *reinterpret_cast<const ulonglong2*>(p);
    return DF2{f.x, f.y};
}

template <bool COHERENT>
__device__ __forceinline__ DF2 ld_df2_g(const df32* p) {
    const ulonglong2 f = COHERENT ? __ldcg(reinterpret_cast<const ulonglong2*>(p))
                                  : __ldg(reinterpret_cast<const ulonglong2*>(p));
    return DF2{f.x, f.y};
}

template <bool COHERENT>
__device__ __forceinline__ DF2 ld_df2_rw(const df32* p) {
    const ulonglong2 f = COHERENT ? __ldcg(reinterpret_cast<const ulonglong2*>(p))
                                  : *reinterpret_cast<const ulonglong2*>(p);
    return DF2{f.x, f.y};
}

__device__ __forceinline__ void st_df2(df32* p, DF2 v) {
    *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2(v.hi, v.lo);
}

// lanes swapped: (x1 | x0)
__device__ __forceinline__ DF2 df2_swap(DF2 v) {
    float h0, h1, l0, l1;
    upk2(v.hi, h0, h1);
    upk2(v.lo, l0, l1);
    return DF2{pk2(h1, h0), pk2(l1, l0)};
}

__device__ __forceinline__ DF2 df2_shfl_xor(DF2 v, int o) {
    float h0, h1, l0, l1;
    upk2(v.hi, h0, h1);
    upk2(v.lo, l0, l1);
    return DF2{pk2(__shfl_xor_sync(0xffffffffu, h0, o), __shfl_xor_sync(0xffffffffu, h1, o)),
               pk2(__shfl_xor_sync(0xffffffffu, l0, o), __shfl_xor_sync(0xffffffffu, l1, o))};
}

template <int MODE, bool COHERENT, int TB>
__device__ __forceinline__ void tile_step_df4x2(const StepArgs& a, const int item, const int step) {
    static_assert(TB > 0, "the paired pass is specialised on the tile's bit count");
    using T = df32;
    constexpr int B = 4, EG = EarlyGlobal<T>::value;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* tile = reinterpret_cast<T*>(smem_raw);
    // per spin: (g.hi, g.hi, g.lo, g.lo) and (-g.hi, -g.hi), the register pairs of a DF2m
    __shared__ __align__(16) float4 gam_s[kMaxSpins + 1];        // slot kMaxSpins: the global flip
    __shared__ __align__(8) float2 ngam_s[kMaxSpins + 1];
    __shared__ double red_s[kThreads / 32][2 * B * B];
    __shared__ int last_s;
    __shared__ __align__(8) uint64_t bar_s;

    const int tid = threadIdx.x;
    const int h = tid & 1;
    const Item it = a.items[item];
    const RealInfo R = a.real[it.r];
    int nsteps = (MODE == kEvolve) ? R.ne : (MODE == kApply ? 1 : R.nf);
    if (MODE != kApply && a.nsteps_override > 0) nsteps = a.nsteps_override;
    const bool active = step < nsteps;
    constexpr bool want_mom = MODE == kEvolve;
    Dot2x2 mp[5];
#pragma unroll
    for (int e = 0; e < 5; ++e) mp[e] = Dot2x2{0ull, 0ull};

    if (active) {
        T* wA = static_cast<T*>(a.bufA);
        T* wB = static_cast<T*>(a.bufB);
        T* wk = (step & 1) ? wB : wA;
        T* wo = (step & 1) ? wA : wB;
        const T* x;
        const T* y1 = nullptr;
        const T* y2 = nullptr;
        T* out;
        double c_h, c_1 = 0.0, c_2 = 0.0;
        const double* cf = a.coef + 8 * it.r + (step == 0 ? 0 : 3);
        if (MODE == kApply) {
            x = static_cast<const T*>(a.x); y1 = static_cast<const T*>(a.y1); out = static_cast<T*>(a.out);
            c_h = cf[0]; c_1 = cf[1];
        } else if (MODE == kFilter1) {
            x = wk; out = static_cast<T*>(a.bufU); c_h = 1.0;
        } else if (MODE == kFilter2) {
            x = static_cast<const T*>(a.bufU); y1 = wk; y2 = wo; out = wo;
            c_h = cf[0]; c_1 = cf[1]; c_2 = cf[2];
        } else {
            x = wk; y1 = wo; out = wo;
            c_h = cf[0]; c_1 = cf[1];
        }
        const bool use1 = (c_1 != 0.0) && (y1 != nullptr);
        const bool use2 = (c_2 != 0.0) && (y2 != nullptr);
        const bool sub1 = c_1 == -1.0, sub2v = c_2 == -1.0;    // uniform over the CTA
        const T ch = static_cast<T>(c_h);
        const DF2m C1 = df2m_bcast(static_cast<T>(c_1)), C2 = df2m_bcast(static_cast<T>(c_2));

        constexpr int tstates = 1 << TB;
        const int64_t tile0 = static_cast<int64_t>(it.tile) << TB;
        const int64_t gbase = R.off * B;
        const T* xg = x + gbase;
        const T* y1g = (MODE != kFilter1 && y1) ? y1 + gbase : nullptr;
        const T* y2g = (MODE == kFilter2 && y2) ? y2 + gbase : nullptr;
        T* outg = out + gbase;
        const T* dg = static_cast<const T*>(a.diag) + R.off;
        if (tid < R.N) {
            const T g = ch * static_cast<const T*>(a.gam)[it.r * kMaxSpins + tid];
            gam_s[tid] = make_float4(g.hi, g.hi, g.lo, g.lo);
            ngam_s[tid] = make_float2(-g.hi, -g.hi);
        }
        if (tid == kMaxSpins && a.gflip) {
            const T g = ch * T(__ldg(a.gflip + it.r));
            gam_s[kMaxSpins] = make_float4(g.hi, g.hi, g.lo, g.lo);
            ngam_s[kMaxSpins] = make_float2(-g.hi, -g.hi);
        }

        constexpr uint32_t nbytes = static_cast<uint32_t>(tstates) * B * sizeof(T);
        if (tid == 0) {
            mbar_init(&bar_s, 1);
            bulk_load(tile, xg + tile0 * B, nbytes, &bar_s);
            // evolution: the tile's rows of w_{k-1} and of the diagonal, which the threads
            // read once each, into L2 while the tile lands (offsets are multiples of 4
            // states, so every start is 16-byte aligned). 176 against 184 us per order on
            // the 256-shard batch; in the filter's second pass, prefetching w_k and w_{k-1}
            // pushed u out of L2 (292 against 275 us), so the filter does without.
            if (MODE == kEvolve && use1) bulk_prefetch_l2(y1g + tile0 * B, nbytes);
            if (MODE == kEvolve) bulk_prefetch_l2(dg + tile0, static_cast<uint32_t>(tstates) * sizeof(T));
        }
        __syncthreads();
        const bool landed = mbar_wait(&bar_s, 0, kWaitLimit);
        if (!landed) {
            atomicExch(a.err_flag, 1);
            mbar_wait(&bar_s, 0, kWaitLimit);        // let the copy land before the CTA exits
        }
        __syncthreads();
        if (tid == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar_s)) : "memory");
        if (!landed) goto reduce_df4x2;

        {
        const int ngb = R.N - TB;
        constexpr int nhalf = 2 * tstates;               // (state, column pair) slots of the tile
        const ulonglong2* g2 = reinterpret_cast<const ulonglong2*>(gam_s);
        const uint64_t* ng2 = reinterpret_cast<const uint64_t*>(ngam_s);

        for (int hb = 0; hb < nhalf; hb += kThreads) {
            const int hs = hb + tid;
            const bool val = (TB >= 7) || hs < nhalf;
            const int sl = val ? (hs >> 1) : 0;
            const uint32_t sg = static_cast<uint32_t>(tile0) + static_cast<uint32_t>(sl);
            const int col = 2 * h;
            const DF2 A = ld_df2_s(tile + sl * B + col);
            // the global flip's partner takes the first free early slot (parity sectors: ngb = 2)
            const bool gflip = a.gflip != nullptr;
            const uint32_t gfm = (1u << R.N) - 1u;
            DF2 pe[EG > 0 ? EG : 1];
#pragma unroll
            for (int j = 0; j < EG; ++j) {
                if (j < ngb) pe[j] = ld_df2_g<COHERENT>(xg + ((sg ^ (1u << (TB + j))) * B + col));
                else if (j == ngb && gflip) pe[j] = ld_df2_g<COHERENT>(xg + ((sg ^ gfm) * B + col));
            }
            const T dr = ld_ro(dg + sg);
            DF2 Y = DF2{0ull, 0ull}, Z = DF2{0ull, 0ull};
            if (MODE != kFilter1 && use1) Y = ld_df2_rw<COHERENT>(y1g + (sg * B + col));
            if (MODE == kFilter2 && use2) Z = ld_df2_rw<COHERENT>(y2g + (sg * B + col));
            // flips inside the tile; bit 0 starts the sums
            Dot2x2 acc;
            {
                const ulonglong2 gv = g2[0];
                acc = dot2x2_prod(DF2m{gv.x, ng2[0], gv.y}, ld_df2_s(tile + (sl ^ 1) * B + col));
            }
#pragma unroll
            for (int i = 1; i < TB; ++i) {
                const ulonglong2 gv = g2[i];
                dot2x2_mad(acc, DF2m{gv.x, ng2[i], gv.y}, ld_df2_s(tile + (sl ^ (1 << i)) * B + col));
            }
            // flips beyond the tile
#pragma unroll
            for (int j = 0; j < EG; ++j) {
                if (j < ngb) {
                    const ulonglong2 gv = g2[TB + j];
                    dot2x2_mad(acc, DF2m{gv.x, ng2[TB + j], gv.y}, pe[j]);
                } else if (j == ngb && gflip) {           // global flip X_0 ... X_{N-1}, loaded early
                    const ulonglong2 gv = g2[kMaxSpins];
                    dot2x2_mad(acc, DF2m{gv.x, ng2[kMaxSpins], gv.y}, pe[j]);
                }
            }
            for (int j = EG; j < ngb; ++j) {
                const ulonglong2 gv = g2[TB + j];
                dot2x2_mad(acc, DF2m{gv.x, ng2[TB + j], gv.y},
                           ld_df2_g<COHERENT>(xg + ((sg ^ (1u << (TB + j))) * B + col)));
            }
            if (gflip && ngb >= EG) {                       // global flip, no early slot left
                const ulonglong2 gv = g2[kMaxSpins];
                dot2x2_mad(acc, DF2m{gv.x, ng2[kMaxSpins], gv.y},
                           ld_df2_g<COHERENT>(xg + ((sg ^ gfm) * B + col)));
            }
            // diagonal term, then w_{k+1} = c_h H x + c_1 y + c_2 z
            dot2x2_mad(acc, df2m_bcast(ch * dr), A);
            if (MODE != kFilter1 && use1) {
                if (sub1) dot2x2_sub(acc, Y);
                else dot2x2_mad(acc, C1, Y);
            }
            if (MODE == kFilter2 && use2) {
                if (sub2v) dot2x2_sub(acc, Z);
                else dot2x2_mad(acc, C2, Z);
            }
            const DF2 O = dot2x2_final(acc);
            if (val) st_df2(outg + (sg * B + col), O);
            if (want_mom) {
                const DF2 Cx = df2_shfl_xor(A, 1);        // the other pair's x
                if (val) {
                    // h = 0: (x0 x0 | x1 x1), (o0 x0 | o1 x1), (x0 x1 | o0 x1), (o0 x2 | o1 x3), (o0 x3 | o1 x2)
                    // h = 1: the same with columns 2, 3 for 0, 1, and <x_p, x_q> across the pairs
                    const DF2m Am = df2m(A);
                    dot2x2_mad(mp[0], Am, A);
                    dot2x2_mad(mp[1], Am, O);
                    {
                        float ah0, ah1, al0, al1, oh0, oh1, ol0, ol1;
                        upk2(A.hi, ah0, ah1);
                        upk2(A.lo, al0, al1);
                        upk2(O.hi, oh0, oh1);
                        upk2(O.lo, ol0, ol1);
                        const DF2 X01 = DF2{pk2(ah0, oh0), pk2(al0, ol0)};
                        dot2x2_mad(mp[2], df2m(X01), DF2{pk2(ah1, ah1), pk2(al1, al1)});
                    }
                    const DF2 U = h ? Cx : O, V = h ? A : Cx;
                    const DF2m Um = df2m(U);
                    dot2x2_mad(mp[3], Um, V);
                    dot2x2_mad(mp[4], Um, df2_swap(V));
                }
            }
        }
        }
    }

reduce_df4x2:
    if (want_mom && active) {
        const int lane = tid & 31, warp = tid >> 5;
        // the ten sums in the order of tile_step_df4: (x0x0, x0x1, x1x1, o0x0, o0x1, o1x1,
        // u0v0, u0v1, u1v0, u1v1) for h = 0; columns shifted by two for h = 1
        Dot2 ms[10];
        dot2x2_split(mp[0], ms[0], ms[2]);
        dot2x2_split(mp[1], ms[3], ms[5]);
        dot2x2_split(mp[2], ms[1], ms[4]);
        dot2x2_split(mp[3], ms[6], ms[9]);
        dot2x2_split(mp[4], ms[7], ms[8]);
        df32 xs[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) xs[e] = e < 10 ? dot2_final(ms[e]) : df32(0.f, 0.f);
        const df32 t = warp_reduce_scatter<16, 2>(xs, lane);
        const int e = (lane >> 1) & 15;
        if (e < 10) {
            int blk, p, q;
            if (e < 6) {
                blk = e / 3;
                const int k = e % 3;
                p = 2 * h + (k == 2 ? 1 : 0);
                q = 2 * h + (k >= 1 ? 1 : 0);
            } else {
                blk = h == 0 ? 1 : 0;
                p = (e - 6) >> 1;
                q = 2 + ((e - 6) & 1);
            }
            const double v = static_cast<double>(t);
            double* rw = red_s[warp];
            rw[blk * B * B + p * B + q] = v;
            rw[blk * B * B + q * B + p] = v;
        }
        __syncthreads();
        if (tid < 2 * B * B) {
            double sm = 0.0;
#pragma unroll
            for (int w = 0; w < kThreads / 32; ++w) sm += red_s[w][tid];
            a.part[static_cast<int64_t>(item) * 2 * B * B + tid] = sm;
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const unsigned prev = atomicAdd(&a.real_done[it.r], 1u);
            last_s = (prev == static_cast<unsigned>(R.item_count - 1));
        }
        __syncthreads();
        if (last_s) {
            __threadfence();
            if (tid < 2 * B * B) {
                double sm = 0.0;
                for (int j = 0; j < R.item_count; ++j)
                    sm += __ldcg(a.part + static_cast<int64_t>(R.item_begin + j) * 2 * B * B + tid);
                const int row = 2 * step;
                const int64_t row0 = a.mom_rows_fixed > 0 ? static_cast<int64_t>(it.r) * a.mom_rows_fixed : R.mom_off;
                a.mom[(row0 + row) * B * B + tid] = sm;
            }
            if (tid == 0) a.real_done[it.r] = 0u;
        }
    }
    __syncthreads();
}

template <typename T, int B, int MODE, bool COHERENT>
__device__ __forceinline__ void tile_step_any(const StepArgs& a, const int item, const int step) {
    if constexpr (std::is_same<T, df32>::value && B == 4) tile_step_df4<MODE, COHERENT>(a, item, step);
    else tile_step<T, B, MODE, COHERENT>(a, item, step);
}

// Double-float b = 4 with a tile of TB bits in every realization.
template <int MODE, int TB>
__global__ void __launch_bounds__(kThreads, MinBlocks<df32, 4>::value) step_kernel_df4tb(const StepArgs a,
                                                                                         int item_base) {
    int step = 0;
    if (MODE != kApply) step = *a.step_ctr;
    tile_step_df4x2<MODE, false, TB>(a, item_base + blockIdx.x, step);
    if (MODE == kFilter2 || MODE == kEvolve) {
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned prev = atomicAdd(a.launch_done, 1u);
            if (prev == gridDim.x - 1) {
                *a.launch_done = 0u;
                __threadfence();
                atomicAdd(a.step_ctr, 1);
            }
        }
    }
}

template <typename T, int B, int MODE>
__global__ void __launch_bounds__(kThreads, MinBlocks<T, B>::value) step_kernel(const StepArgs a, int item_base) {
    int step = 0;
    if (MODE != kApply) step = *a.step_ctr;
    tile_step_any<T, B, MODE, false>(a, item_base + blockIdx.x, step);
    if (MODE == kFilter2 || MODE == kEvolve) {
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned prev = atomicAdd(a.launch_done, 1u);
            if (prev == gridDim.x - 1) {
                *a.launch_done = 0u;
                __threadfence();
                atomicAdd(a.step_ctr, 1);
            }
        }
    }
}

// float32 recurrences with every HBM read of a tile staged in shared memory by
// bulk copies (tile_step STAGED); per-order launches, replayed from a graph.
template <int B, int MODE>
__global__ void __launch_bounds__(kThreads, MinBlocks<float, B>::value) step_kernel_staged(const StepArgs a,
                                                                                          int item_base) {
    const int step = *a.step_ctr;
    tile_step<float, B, MODE, false, true>(a, item_base + blockIdx.x, step);
    if (MODE == kFilter2 || MODE == kEvolve) {
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned prev = atomicAdd(a.launch_done, 1u);
            if (prev == gridDim.x - 1) {
                *a.launch_done = 0u;
                __threadfence();
                atomicAdd(a.step_ctr, 1);
            }
        }
    }
}

// Device-wide barrier of a cooperative launch. The wait is bounded (kWaitNs):
// on expiry it raises err_flag (2) and every CTA leaves the order loop at its
// next barrier, so no CTA spins forever.

__device__ __forceinline__ bool grid_sync(const StepArgs& a) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = a.bar_gen;
        const unsigned g = *gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(a.bar_count, 1u) == gridDim.x - 1) {
            atomicExch(a.bar_count, 0u);
            __threadfence();
            atomicAdd(a.bar_gen, 1u);
        } else {
            const uint64_t t0 = global_ns();
            while (*gen == g) {
                if (global_ns() - t0 > kWaitNs) {
                    ok = 0;
                    atomicExch(a.err_flag, 2);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_s = ok && (*reinterpret_cast<volatile int*>(a.err_flag) == 0);
    }
    __syncthreads();
    return ok_s;
}

// All orders of the filter (SEQ = 0: two passes per order) or the evolution
// (SEQ = 1) in one cooperative launch; CTAs take tiles round-robin.
template <typename T, int B, int SEQ>
__global__ void __launch_bounds__(kThreads, MinBlocks<T, B>::value) persistent_kernel(const StepArgs a, int n_items,
                                                                                 int orders) {
    for (int k = 0; k < orders; ++k) {
        if (SEQ == 0) {
            for (int item = blockIdx.x; item < n_items; item += gridDim.x) tile_step_any<T, B, kFilter1, true>(a, item, k);
            if (!grid_sync(a)) return;
            for (int item = blockIdx.x; item < n_items; item += gridDim.x) tile_step_any<T, B, kFilter2, true>(a, item, k);
            if (!grid_sync(a)) return;
        } else {
            for (int item = blockIdx.x; item < n_items; item += gridDim.x) tile_step_any<T, B, kEvolve, true>(a, item, k);
            if (!grid_sync(a)) return;
        }
    }
}

template <typename T, int B, int MODE>
static cudaError_t launch_one(const StepArgs& a, int item_base, int n_items, int smem, cudaStream_t st) {
    if constexpr (std::is_same<T, df32>::value && B == 4) {
        switch (a.tbits_uniform) {
            case 10: step_kernel_df4tb<MODE, 10><<<n_items, kThreads, smem, st>>>(a, item_base); return cudaGetLastError();
            case 11: step_kernel_df4tb<MODE, 11><<<n_items, kThreads, smem, st>>>(a, item_base); return cudaGetLastError();
            case 12: step_kernel_df4tb<MODE, 12><<<n_items, kThreads, smem, st>>>(a, item_base); return cudaGetLastError();
            default: break;
        }
    }
    step_kernel<T, B, MODE><<<n_items, kThreads, smem, st>>>(a, item_base);
    return cudaGetLastError();
}

// cudaFuncAttributeMaxDynamicSharedMemorySize is process-wide per kernel and
// device, while handles with different tile sizes share the kernels: a later
// handle with a smaller tile must not lower the limit an earlier handle (or
// an already instantiated graph) launches with. So the attribute only grows:
// the largest value set so far is kept per (kernel, device) under a mutex,
// and the runtime is called only when a launch needs more.
static std::mutex g_smem_mu;
static std::map<std::pair<const void*, int>, int> g_smem_max;

static cudaError_t grow_smem_attr(const void* func, int smem) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_smem_mu);
    int& have = g_smem_max[std::make_pair(func, dev)];
    if (smem <= have) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) have = smem;
    return e;
}

template <typename K>
static cudaError_t grow_smem(K* kernel, int smem) {
    return grow_smem_attr(reinterpret_cast<const void*>(kernel), smem);
}

template <int MODE>
static cudaError_t prepare_df4tb(int smem) {
    cudaError_t e;
    if ((e = grow_smem(step_kernel_df4tb<MODE, 10>, smem)) != cudaSuccess) return e;
    if ((e = grow_smem(step_kernel_df4tb<MODE, 11>, smem)) != cudaSuccess) return e;
    return grow_smem(step_kernel_df4tb<MODE, 12>, smem);
}

template <typename T, int B>
static cudaError_t prepare_tb(int smem) {
    cudaError_t e;
    if ((e = grow_smem(step_kernel<T, B, kApply>, smem)) != cudaSuccess) return e;
    if ((e = grow_smem(step_kernel<T, B, kFilter1>, smem)) != cudaSuccess) return e;
    if ((e = grow_smem(step_kernel<T, B, kFilter2>, smem)) != cudaSuccess) return e;
    if constexpr (std::is_same<T, df32>::value && B == 4) {
        if ((e = prepare_df4tb<kApply>(smem)) != cudaSuccess) return e;
        if ((e = prepare_df4tb<kFilter1>(smem)) != cudaSuccess) return e;
        if ((e = prepare_df4tb<kFilter2>(smem)) != cudaSuccess) return e;
        if ((e = prepare_df4tb<kEvolve>(smem)) != cudaSuccess) return e;
    }
    return grow_smem(step_kernel<T, B, kEvolve>, smem);
}

// Allow the dynamic shared-memory tile for every mode of (precision, b);
// called once per handle, outside any stream capture.
cudaError_t prepare_step(int prec, int b, int smem) {
    DACP_FOR_PREC(prec, DACP_FOR_B(b, return prepare_tb<T, BB>(smem)));
    return cudaErrorInvalidValue;
}

template <typename T, int B>
static cudaError_t launch_mode(int mode, const StepArgs& a, int item_base, int n_items, int smem,
                               cudaStream_t st) {
    switch (mode) {
        case kApply: return launch_one<T, B, kApply>(a, item_base, n_items, smem, st);
        case kFilter1: return launch_one<T, B, kFilter1>(a, item_base, n_items, smem, st);
        case kFilter2: return launch_one<T, B, kFilter2>(a, item_base, n_items, smem, st);
        case kEvolve: return launch_one<T, B, kEvolve>(a, item_base, n_items, smem, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t launch_b(int b, int mode, const StepArgs& a, int item_base, int n_items, int smem,
                            cudaStream_t st) {
    switch (b) {
        case 1: return launch_mode<T, 1>(mode, a, item_base, n_items, smem, st);
        case 2: return launch_mode<T, 2>(mode, a, item_base, n_items, smem, st);
        case 4: return launch_mode<T, 4>(mode, a, item_base, n_items, smem, st);
    }
    return cudaErrorInvalidValue;
}

// ---- staged float32 launches ------------------------------------------------

// Dynamic shared memory of a staged launch whose largest tile takes tile_smem
// bytes: the x tile, one y tile per recurrence term (kEvolve 1, kFilter2 2) and
// the tile's float32 diagonal (tile_smem / b bytes).
int staged_smem_bytes(int mode, int b, int tile_smem) {
    const int ny = mode == kFilter2 ? 2 : (mode == kFilter1 ? 0 : 1);
    return tile_smem * (1 + ny) + tile_smem / b;
}

template <int B, int MODE>
static bool staged_mode_fits(int tile_smem, int optin) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, step_kernel_staged<B, MODE>) != cudaSuccess) return false;
    return staged_smem_bytes(MODE, B, tile_smem) + static_cast<int>(fa.sharedSizeBytes) <= optin;
}

template <int B>
static bool staged_fits_b(int tile_smem) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
    return staged_mode_fits<B, kFilter1>(tile_smem, optin) && staged_mode_fits<B, kFilter2>(tile_smem, optin) &&
           staged_mode_fits<B, kEvolve>(tile_smem, optin);
}

// Whether the staged kernels' shared memory fits the device for this tile.
bool staged_fits(int b, int tile_smem) {
    switch (b) {
        case 1: return staged_fits_b<1>(tile_smem);
        case 2: return staged_fits_b<2>(tile_smem);
        case 4: return staged_fits_b<4>(tile_smem);
    }
    return false;
}

template <int B>
static cudaError_t prepare_staged_b(int tile_smem) {
    cudaError_t e;
    if ((e = grow_smem(step_kernel_staged<B, kFilter1>, staged_smem_bytes(kFilter1, B, tile_smem))) != cudaSuccess)
        return e;
    if ((e = grow_smem(step_kernel_staged<B, kFilter2>, staged_smem_bytes(kFilter2, B, tile_smem))) != cudaSuccess)
        return e;
    return grow_smem(step_kernel_staged<B, kEvolve>, staged_smem_bytes(kEvolve, B, tile_smem));
}

// Allow the staged kernels' dynamic shared memory (call staged_fits first);
// once per handle and tile size, outside any stream capture.
cudaError_t prepare_step_staged(int b, int tile_smem) {
    if (!staged_fits(b, tile_smem)) return cudaErrorInvalidValue;
    switch (b) {
        case 1: return prepare_staged_b<1>(tile_smem);
        case 2: return prepare_staged_b<2>(tile_smem);
        case 4: return prepare_staged_b<4>(tile_smem);
    }
    return cudaErrorInvalidValue;
}

template <int B>
static cudaError_t launch_staged_b(int mode, const StepArgs& a, int item_base, int n_items, int tile_smem,
                                   cudaStream_t st) {
    switch (mode) {
        case kFilter1:
            step_kernel_staged<B, kFilter1><<<n_items, kThreads, staged_smem_bytes(kFilter1, B, tile_smem), st>>>(
                a, item_base);
            return cudaGetLastError();
        case kFilter2:
            step_kernel_staged<B, kFilter2><<<n_items, kThreads, staged_smem_bytes(kFilter2, B, tile_smem), st>>>(
                a, item_base);
            return cudaGetLastError();
        case kEvolve:
            step_kernel_staged<B, kEvolve><<<n_items, kThreads, staged_smem_bytes(kEvolve, B, tile_smem), st>>>(
                a, item_base);
            return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
}

// One staged float32 recurrence pass (kFilter1, kFilter2 or kEvolve) over items
// [item_base, item_base + n_items); tile_smem = bytes of the largest vector tile.
cudaError_t launch_step_staged(int b, int mode, const StepArgs& a, int item_base, int n_items, int tile_smem,
                               cudaStream_t st) {
    switch (b) {
        case 1: return launch_staged_b<1>(mode, a, item_base, n_items, tile_smem, st);
        case 2: return launch_staged_b<2>(mode, a, item_base, n_items, tile_smem, st);
        case 4: return launch_staged_b<4>(mode, a, item_base, n_items, tile_smem, st);
    }
    return cudaErrorInvalidValue;
}

template <typename T, int B, int SEQ>
static cudaError_t launch_persistent_tb(const StepArgs& a, int n_items, int orders, int smem, cudaStream_t st,
                                       int* grid_out) {
    auto k = persistent_kernel<T, B, SEQ>;
    cudaError_t e = grow_smem(k, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int grid = sms * per_sm;
    if (grid > n_items) grid = n_items;
    if (grid_out) *grid_out = grid;
    StepArgs args = a;
    int ni = n_items, no = orders;
    void* params[] = {&args, &ni, &no};
    return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k), dim3(grid), dim3(kThreads), params, smem, st);
}

// Every filter (seq 0) or evolution (seq 1) order in one cooperative launch.
cudaError_t launch_persistent(int prec, int b, int seq, const StepArgs& a, int n_items, int orders, int smem,
                              cudaStream_t st, int* grid_out) {
    DACP_FOR_PREC(prec, DACP_FOR_B(b, return seq == 0
                                                   ? launch_persistent_tb<T, BB, 0>(a, n_items, orders, smem, st, grid_out)
                                                   : launch_persistent_tb<T, BB, 1>(a, n_items, orders, smem, st, grid_out)));
    return cudaErrorInvalidValue;
}

cudaError_t launch_step(int prec, int b, int mode, const StepArgs& a, int item_base, int n_items,
                        int smem, cudaStream_t st) {
    DACP_FOR_PREC(prec, return launch_b<T>(b, mode, a, item_base, n_items, smem, st));
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Set-up kernels: diagonal, precision conversion, column norms, normalisation.

// diag(s) = sum_{i<j} J_ij z_i z_j + sum_i h_i z_i, z_i = 1 - 2 bit_i(s), in float64.
template <typename T>
__global__ void diag_kernel(const RealInfo* __restrict__ real, int r, const double* __restrict__ J,
                            const double* __restrict__ h, T* __restrict__ diag) {
    const RealInfo R = real[r];
    const int64_t D = static_cast<int64_t>(1) << R.N;
    const double* Jr = J + static_cast<int64_t>(r) * kMaxSpins * kMaxSpins;
    const double* hr = h + static_cast<int64_t>(r) * kMaxSpins;
    for (int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; s < D;
         s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double d = 0.0;
        for (int i = 0; i < R.N; ++i) {
            const double zi = ((s >> i) & 1) ? -1.0 : 1.0;
            d += hr[i] * zi;
            for (int j = i + 1; j < R.N; ++j) {
                const double zj = ((s >> j) & 1) ? -1.0 : 1.0;
                d += Jr[i * kMaxSpins + j] * zi * zj;
            }
        }
        diag[R.off + s] = static_cast<T>(d);
    }
}

// All realizations in one launch: blockIdx.y is the realization.
template <typename T>
__global__ void diag_all_kernel(const RealInfo* __restrict__ real, const double* __restrict__ J,
                                const double* __restrict__ h, T* __restrict__ diag) {
    const int r = blockIdx.y;
    const RealInfo R = real[r];
    const int64_t D = static_cast<int64_t>(1) << R.N;
    const double* Jr = J + static_cast<int64_t>(r) * kMaxSpins * kMaxSpins;
    const double* hr = h + static_cast<int64_t>(r) * kMaxSpins;
    for (int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; s < D;
         s += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double d = 0.0;
        for (int i = 0; i < R.N; ++i) {
            const double zi = ((s >> i) & 1) ? -1.0 : 1.0;
            d += hr[i] * zi;
            for (int j = i + 1; j < R.N; ++j) {
                const double zj = ((s >> j) & 1) ? -1.0 : 1.0;
                d += Jr[i * kMaxSpins + j] * zi * zj;
            }
        }
        diag[R.off + s] = static_cast<T>(d);
    }
}

// Start vectors: realization r's packed float64 block (at src_off[r]) into its
// padded slot of the device layout, converted to T. blockIdx.y is r.
template <typename T>
__global__ void scatter_convert_kernel(const double* __restrict__ src, const int64_t* __restrict__ src_off,
                                       const RealInfo* __restrict__ real, int b, T* __restrict__ dst) {
    const int r = blockIdx.y;
    const RealInfo R = real[r];
    const int64_t n = (static_cast<int64_t>(1) << R.N) * b;
    const double* s = src + src_off[r];
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        VecAt<T>::set(dst, R.off + i / b, static_cast<int>(i % b), b, static_cast<T>(s[i]));
}

template <typename T>
__global__ void convert_kernel(const double* __restrict__ src, T* __restrict__ dst, int64_t n) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        dst[i] = static_cast<T>(src[i]);
}

template <typename T>
__global__ void extract_col_kernel(const T* __restrict__ src, T* __restrict__ dst, int b, int64_t states) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < states;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        dst[i] = VecAt<T>::get(src, i, 0, b);
}

// n / b states of a [state][b] vector to float64, element (s, p) at s * b + p.
template <typename T>
__global__ void to_double_kernel(const T* __restrict__ src, double* __restrict__ dst, int64_t n, int b) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        dst[i] = static_cast<double>(VecAt<T>::get(src, i / b, static_cast<int>(i % b), b));
}

// Squared column norms of each realization's vector; src is chosen per
// realization by the parity of its filter order (w_K lives in A when K is even).
template <typename T, int B>
__global__ void __launch_bounds__(kThreads) colnorm_kernel(const Item* __restrict__ items,
                                                           const RealInfo* __restrict__ real,
                                                           const T* A, const T* Bv, int by_parity,
                                                           double* part, unsigned* real_done,
                                                           double* norms) {
    __shared__ double red_s[kThreads / 32][B];
    __shared__ int last_s;
    const int tid = threadIdx.x;
    const Item it = items[blockIdx.x];
    const RealInfo R = real[it.r];
    const T* src = (by_parity && (R.nf & 1)) ? Bv : A;
    const int tstates = 1 << R.tbits;
    const int64_t tile0 = static_cast<int64_t>(it.tile) << R.tbits;
    double acc[B];
#pragma unroll
    for (int p = 0; p < B; ++p) acc[p] = 0.0;
    for (int sl = tid; sl < tstates; sl += kThreads) {
        const int64_t sg = R.off + tile0 + sl;
#pragma unroll
        for (int p = 0; p < B; ++p) {
            const double v = static_cast<double>(VecAt<T>::get(src, sg, p, B));
            acc[p] = fma(v, v, acc[p]);
        }
    }
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int p = 0; p < B; ++p) {
        const double v = warp_sum(acc[p]);
        if (lane == 0) red_s[warp][p] = v;
    }
    __syncthreads();
    if (tid < B) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red_s[w][tid];
        part[static_cast<int64_t>(blockIdx.x) * B + tid] = s;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last_s = (atomicAdd(&real_done[it.r], 1u) == static_cast<unsigned>(R.item_count - 1));
    __syncthreads();
    if (last_s) {
        __threadfence();
        if (tid < B) {
            double s = 0.0;
            for (int j = 0; j < R.item_count; ++j) s += __ldcg(part + static_cast<int64_t>(R.item_begin + j) * B + tid);
            norms[it.r * B + tid] = s;
        }
        if (tid == 0) real_done[it.r] = 0u;
    }
}

// psi_E = w_K / ||w_K|| per column (Eq. target), written to dst and dst2.
template <typename T, int B>
__global__ void __launch_bounds__(kThreads) normalize_kernel(const Item* __restrict__ items,
                                                             const RealInfo* __restrict__ real,
                                                             const T* A, const T* Bv, int by_parity,
                                                             const double* __restrict__ norms,
                                                             T* dst, T* dst2) {
    const int tid = threadIdx.x;
    const Item it = items[blockIdx.x];
    const RealInfo R = real[it.r];
    const T* src = (by_parity && (R.nf & 1)) ? Bv : A;
    const int tstates = 1 << R.tbits;
    const int64_t tile0 = static_cast<int64_t>(it.tile) << R.tbits;
    T sc[B];
#pragma unroll
    for (int p = 0; p < B; ++p) sc[p] = static_cast<T>(1.0 / sqrt(norms[it.r * B + p]));
    for (int sl = tid; sl < tstates; sl += kThreads) {
        const int64_t sg = R.off + tile0 + sl;
#pragma unroll
        for (int p = 0; p < B; ++p) {
            const T v = VecAt<T>::get(src, sg, p, B) * sc[p];
            VecAt<T>::set(dst, sg, p, B, v);
            if (dst2) VecAt<T>::set(dst2, sg, p, B, v);
        }
    }
}

cudaError_t launch_diag(int prec, const RealInfo* real, int r, int N, const double* J, const double* h,
                        void* diag, cudaStream_t st) {
    const int64_t D = static_cast<int64_t>(1) << N;
    const int grid = static_cast<int>((D + 255) / 256 < 4096 ? (D + 255) / 256 : 4096);
    DACP_FOR_PREC(prec, diag_kernel<T><<<grid, 256, 0, st>>>(real, r, J, h, static_cast<T*>(diag));
                        return cudaGetLastError());
    return cudaErrorInvalidValue;
}

cudaError_t launch_diag_all(int prec, const RealInfo* real, int R, int max_N, const double* J, const double* h,
                            void* diag, cudaStream_t st) {
    const int64_t D = static_cast<int64_t>(1) << max_N;
    dim3 grid(static_cast<unsigned>((D + 255) / 256 < 1024 ? (D + 255) / 256 : 1024), static_cast<unsigned>(R));
    DACP_FOR_PREC(prec, diag_all_kernel<T><<<grid, 256, 0, st>>>(real, J, h, static_cast<T*>(diag));
                        return cudaGetLastError());
    return cudaErrorInvalidValue;
}

cudaError_t launch_scatter_convert(int prec, const double* src, const int64_t* src_off, const RealInfo* real, int R,
                                   int max_N, int b, void* dst, cudaStream_t st) {
    const int64_t n = (static_cast<int64_t>(1) << max_N) * b;
    dim3 grid(static_cast<unsigned>((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), static_cast<unsigned>(R));
    DACP_FOR_PREC(prec, scatter_convert_kernel<T><<<grid, 256, 0, st>>>(src, src_off, real, b, static_cast<T*>(dst));
                        return cudaGetLastError());
    return cudaErrorInvalidValue;
}

cudaError_t launch_convert(int prec, const double* src, void* dst, int64_t n, cudaStream_t st) {
    const int grid = static_cast<int>((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192);
    if (n == 0) return cudaSuccess;
    DACP_FOR_PREC(prec, convert_kernel<T><<<grid, 256, 0, st>>>(src, static_cast<T*>(dst), n);
                        return cudaGetLastError());
    return cudaErrorInvalidValue;
}

// dst[s] = src[s][0]: column 0 of a [state][b] vector.
cudaError_t launch_extract_col(int prec, int b, const void* src, void* dst, int64_t states, cudaStream_t st) {
    const int grid = static_cast<int>((states + 255) / 256 < 8192 ? (states + 255) / 256 : 8192);
    DACP_FOR_PREC(prec, extract_col_kernel<T><<<grid, 256, 0, st>>>(static_cast<const T*>(src), static_cast<T*>(dst), b, states);
                        return cudaGetLastError());
    return cudaErrorInvalidValue;
}

// Columns col0 .. col0 + b - 1 of the column-major float64 basis matrix V
// (leading dimension ldv) from one [state][b] vector of D states.
template <typename T>
__global__ void gather_basis_kernel(const T* __restrict__ src, int b, int64_t D, double* __restrict__ V, int64_t ldv,
                                    int col0) {
    const int64_t n = D * b;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int p = static_cast<int>(i / D);
        const int64_t s = i % D;
        V[(col0 + p) * ldv + s] = static_cast<double>(VecAt<T>::get(src, s, p, b));
    }
}

cudaError_t launch_gather_basis(int prec, int b, const void* src, int64_t D, double* V, int64_t ldv, int col0,
                                cudaStream_t st) {
    const int64_t n = D * b;
    const int grid = static_cast<int>((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192);
    DACP_FOR_PREC(prec, gather_basis_kernel<T><<<grid, 256, 0, st>>>(static_cast<const T*>(src), b, D, V, ldv, col0);
                        return cudaGetLastError());
    return cudaErrorInvalidValue;
}

cudaError_t launch_to_double(int prec, const void* src, double* dst, int64_t n, int b, cudaStream_t st) {
    const int grid = static_cast<int>((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192);
    if (n == 0) return cudaSuccess;
    DACP_FOR_PREC(prec, to_double_kernel<T><<<grid, 256, 0, st>>>(static_cast<const T*>(src), dst, n, b);
                        return cudaGetLastError());
    return cudaErrorInvalidValue;
}

template <typename T, int B>
static cudaError_t norm_and_scale(const Item* items, const RealInfo* real, int n_items, const void* A,
                                  const void* Bv, int by_parity, double* part, unsigned* real_done,
                                  double* norms, void* dst, void* dst2, cudaStream_t st) {
    colnorm_kernel<T, B><<<n_items, kThreads, 0, st>>>(items, real, static_cast<const T*>(A),
                                                        static_cast<const T*>(Bv), by_parity, part,
                                                        real_done, norms);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    normalize_kernel<T, B><<<n_items, kThreads, 0, st>>>(items, real, static_cast<const T*>(A),
                                                          static_cast<const T*>(Bv), by_parity, norms,
                                                          static_cast<T*>(dst), static_cast<T*>(dst2));
    return cudaGetLastError();
}

cudaError_t launch_normalize(int prec, int b, const Item* items, const RealInfo* real, int n_items,
                             const void* A, const void* Bv, int by_parity, double* part,
                             unsigned* real_done, double* norms, void* dst, void* dst2, cudaStream_t st) {
    DACP_FOR_PREC(prec, DACP_FOR_B(b, return norm_and_scale<T, BB>(items, real, n_items, A, Bv, by_parity, part,
                                                                   real_done, norms, dst, dst2, st)));
    return cudaErrorInvalidValue;
}

}  // namespace dacp
