// Shared definitions of the DACP CUDA library (device kernels and host driver).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "df32.cuh"

namespace dacp {

constexpr int kThreads = 256;       // threads per CTA of the stencil kernels
constexpr int kMaxSpins = 26;       // N limit (2^26 states per realization)
constexpr int kMaxPairs = kMaxSpins * (kMaxSpins - 1) / 2;   // two-body flip terms per realization
constexpr int kTileBytes = 65536;   // shared-memory tile of one stencil CTA
constexpr int kFeatureMoments = 32; // Chebyshev moments fed to the parameter network
constexpr int kFeatures = 8 + kFeatureMoments;

// Element (s, p) of a [state][b] vector in precision T. Double-float vectors
// with b = 4 keep each state's two column pairs as (hi_0, hi_1, lo_0, lo_1 |
// hi_2, hi_3, lo_2, lo_3): one 16-byte load then gives the hi parts and the lo
// parts of two columns in two 64-bit registers, the operands of the paired
// float32 instructions of the stencil. Every other precision and block size
// stores element (s, p) at s * b + p.
template <typename T>
struct VecAt {
    __device__ static T get(const T* v, int64_t s, int p, int b) { return v[s * b + p]; }
    __device__ static void set(T* v, int64_t s, int p, int b, T x) { v[s * b + p] = x; }
};
template <>
struct VecAt<df32> {
    __device__ static int64_t hi_index(int64_t s, int p) { return s * 8 + (p >> 1) * 4 + (p & 1); }
    __device__ static df32 get(const df32* v, int64_t s, int p, int b) {
        if (b != 4) return v[s * b + p];
        const float* f = reinterpret_cast<const float*>(v);
        const int64_t i = hi_index(s, p);
        return df32(f[i], f[i + 2]);
    }
    __device__ static void set(df32* v, int64_t s, int p, int b, df32 x) {
        if (b != 4) {
            v[s * b + p] = x;
            return;
        }
        float* f = reinterpret_cast<float*>(v);
        const int64_t i = hi_index(s, p);
        f[i] = x.hi;
        f[i + 2] = x.lo;
    }
};

// Per-realization geometry and run lengths, read by every stencil CTA.
struct RealInfo {
    int N;            // spins
    int tbits;        // log2(states per tile), tbits <= N
    int64_t off;      // first state of this realization in the batch vectors
    int item_begin;   // first work item (tile) of this realization
    int item_count;   // tiles of this realization = 2^(N - tbits)
    int nf;           // filter orders K to run
    int ne;           // evolution launches = k_n + 1
    int64_t mom_off;  // first moment row (of b*b doubles) of this realization
};

// One work item = one tile of one realization.
struct Item {
    int r;
    int tile;
};

enum StepMode { kApply = 0, kFilter1 = 1, kFilter2 = 2, kEvolve = 3 };

// Vector precision: float64, float32, or double-float (float32 pairs).
enum Precision { kPrecF64 = 0, kPrecF32 = 1, kPrecDF32 = 2 };

// Run the body (the variadic argument) with T bound to the vector element type of `prec` (the body returns).
#define DACP_FOR_PREC(prec, ...)                   \
    switch (prec) {                                 \
        case ::dacp::kPrecF32: {                    \
            using T = float;                        \
            __VA_ARGS__;                            \
        }                                           \
        case ::dacp::kPrecDF32: {                   \
            using T = ::dacp::df32;                 \
            __VA_ARGS__;                            \
        }                                           \
        default: {                                  \
            using T = double;                       \
            __VA_ARGS__;                            \
        }                                           \
    }

// Run the body with BB bound to the block size b in {1, 2, 4} (the body returns).
#define DACP_FOR_B(b, ...)                                  \
    switch (b) {                                             \
        case 1: { constexpr int BB = 1; __VA_ARGS__; }              \
        case 2: { constexpr int BB = 2; __VA_ARGS__; }              \
        case 4: { constexpr int BB = 4; __VA_ARGS__; }              \
        default: return cudaErrorInvalidValue;               \
    }

// Arguments of one stencil launch. Vectors are [state][b] in precision T.
struct StepArgs {
    const Item* items;
    const RealInfo* real;
    const void* diag;        // T per state: diagonal of H
    const void* gam;         // T [R][kMaxSpins]: x-fields
    const double* coef;      // [R][8]: {c_h, c_1, c_2} at order 0, then steady
    void* bufA;              // rotating vectors (filter / evolution)
    void* bufB;
    void* bufU;              // u = H w_k between the two filter passes
    // kApply: explicit vectors
    const void* x;
    const void* y1;
    void* out;
    int apply_row;           // kApply with moments: moment row pair 2*row, 2*row+1
    int apply_moments;       // kApply: accumulate moments
    int* step_ctr;           // device step counter (order k) for graph replay
    unsigned* launch_done;   // CTAs finished in this launch
    unsigned* real_done;     // [R] CTAs of each realization finished
    double* part;            // [items][2 b^2] per-tile moment partials
    double* mom;             // moment rows
    int nsteps_override;     // > 0: run this many orders instead of RealInfo.nf / ne
    int mom_rows_fixed;      // > 0: realization r's rows start at r * mom_rows_fixed
    int* err_flag;           // set to 1 when a bounded device wait gives up
    unsigned* bar_count;     // grid barrier of the persistent launch: arrivals
    unsigned* bar_gen;       // and generation
    int tbits_uniform;       // > 0: every realization's tile has this many bits (lets a launch pick a
                             // kernel specialised on it); 0: mixed
    // two-body flip couplings sum_{i<j} (Jxx_ij X_i X_j + Jyy_ij Y_i Y_j); n_pairs == nullptr: none
    const int* n_pairs;      // [R] terms of each realization
    const int* pair_ij;      // [R][kMaxPairs] bit i | (bit j << 8), i < j
    const double* pair_c;    // [R][kMaxPairs][2] coefficient when bits i, j are equal (Jxx - Jyy)
                             // and when they differ (Jxx + Jyy)
    const double* gflip;     // [R] coefficient of the global flip X_0 X_1 ... X_{N-1}; nullptr: none
};

}  // namespace dacp
