// Double-float numbers: a value is the unevaluated sum hi + lo of two float32,
// with |lo| <= ulp(hi) / 2, carrying about 48 significant bits. Arithmetic is
// built from error-free transformations (Knuth's TwoSum, Dekker's
// Fast2Sum, and the FMA form of TwoProduct; see Muller et al., "Handbook of
// Floating-Point Arithmetic", chs. 4-5), so it runs on the float32 pipes.
// On GB300 the float64 pipes deliver 1/64 of the float32 rate, which makes
// this the fast route to near-float64 accuracy for the recurrences.
//
// Every primitive uses the _rn intrinsics so that the compiler cannot fuse
// or reassociate the steps the error terms depend on.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dacp {

using ::fma;   // keep the float / double overloads visible next to the df32 one

struct __align__(8) df32 {
    float hi, lo;
    df32() = default;
    __host__ __device__ constexpr df32(float h, float l) : hi(h), lo(l) {}
    // from float64: hi = rn(x), lo = rn(x - hi)
    __host__ __device__ explicit df32(double x) : hi(static_cast<float>(x)), lo(static_cast<float>(x - static_cast<double>(static_cast<float>(x)))) {}
    __host__ __device__ explicit df32(int x) : hi(static_cast<float>(x)), lo(0.f) {}
    __host__ __device__ explicit operator double() const { return static_cast<double>(hi) + static_cast<double>(lo); }
};

// s + e = a + b exactly (Knuth, no ordering needed)
__device__ __forceinline__ df32 df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df32(s, e);
}

// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ df32 df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df32(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// p + e = a * b exactly (FMA form)
__device__ __forceinline__ df32 df_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return df32(p, __fmaf_rn(a, b, -p));
}

__device__ __forceinline__ df32 operator+(df32 a, df32 b) {
    df32 s = df_two_sum(a.hi, b.hi);
    const float t = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return df_fast_two_sum(s.hi, t);
}

__device__ __forceinline__ df32 operator-(df32 a) { return df32(-a.hi, -a.lo); }
__device__ __forceinline__ df32 operator-(df32 a, df32 b) { return a + (-b); }

__device__ __forceinline__ df32 operator*(df32 a, df32 b) {
    df32 p = df_two_prod(a.hi, b.hi);
    const float t = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return df_fast_two_sum(p.hi, t);
}

__device__ __forceinline__ df32& operator*=(df32& a, df32 b) {
    a = a * b;
    return a;
}

// a * b + c
__device__ __forceinline__ df32 fma(df32 a, df32 b, df32 c) {
    df32 p = df_two_prod(a.hi, b.hi);
    const float cross = __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi));
    df32 s = df_two_sum(p.hi, c.hi);
    const float t = __fadd_rn(s.lo, __fadd_rn(__fadd_rn(p.lo, cross), c.lo));
    return df_fast_two_sum(s.hi, t);
}

// Compensated dot-product accumulator (Ogita, Rump & Oishi, "Accurate sum and
// dot product", SIAM J. Sci. Comput. 26, 2005, algorithm Dot2): the running
// sum is a float32 `hi` plus one float32 `err` that collects the exact
// TwoProduct / TwoSum error terms; it is folded into a double-float only at
// the end. Each term costs TwoProduct (2) + TwoSum (6) + four error-term updates (4).
struct Dot2 {
    float hi, err;
};

__device__ __forceinline__ Dot2 dot2_init(df32 x) { return Dot2{x.hi, x.lo}; }
__device__ __forceinline__ Dot2 dot2_zero() { return Dot2{0.f, 0.f}; }

// acc += a * b. The cross terms a.hi b.lo and a.lo b.hi go straight into the
// error term by two FMAs: 12 float32 instructions per term.
__device__ __forceinline__ void dot2_mad(Dot2& acc, df32 a, df32 b) {
    const df32 p = df_two_prod(a.hi, b.hi);
    const df32 s = df_two_sum(acc.hi, p.hi);
    acc.hi = s.hi;
    acc.err = __fadd_rn(__fadd_rn(__fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.lo, acc.err)), p.lo), s.lo);
}

__device__ __forceinline__ df32 dot2_final(Dot2 acc) { return df_fast_two_sum(acc.hi, acc.err); }

// ---- two double-floats per instruction (paired float32 arithmetic) ----------
//
// sm_100-family GPUs execute add / sub / mul / fma on pairs of float32
// (.f32x2) as one instruction. On GB300 a paired instruction takes the
// float32 pipe for two cycles, so it does not raise the float32 rate, but it
// halves the issue slots of float32 work: in an issue-bound kernel the loads,
// shuffles and address arithmetic then issue in the slots freed. A register
// pair lane 0 | lane 1 holds one component (hi or lo) of two double-floats.
// Every step below is the same error-free operation as its scalar form above,
// in the same order, so results are bit-identical to the scalar path.

__device__ __forceinline__ uint64_t pk2(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(uint64_t r, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// -x on both lanes: flips the two sign bits (integer pipe, exact)
__device__ __forceinline__ uint64_t neg2(uint64_t a) { return a ^ 0x8000000080000000ull; }

// Two double-floats: hi = (x0.hi | x1.hi), lo = (x0.lo | x1.lo).
struct DF2 {
    uint64_t hi, lo;
};
// A multiplier with its negated hi part, for the TwoProduct below.
struct DF2m {
    uint64_t hi, nhi, lo;
};
__device__ __forceinline__ DF2m df2m(DF2 a) { return DF2m{a.hi, neg2(a.hi), a.lo}; }
__device__ __forceinline__ DF2m df2m_bcast(df32 a) {
    const uint64_t h = pk2(a.hi, a.hi);
    return DF2m{h, neg2(h), pk2(a.lo, a.lo)};
}

// Two Dot2 accumulators (running float32 sum and error term per lane).
struct Dot2x2 {
    uint64_t hi, err;
};

// acc = a * b: TwoProduct (q = -p with p = fl(a.hi b.hi), a.hi b.hi - p exact)
// and the cross terms in the error term.
__device__ __forceinline__ Dot2x2 dot2x2_prod(const DF2m& a, DF2 b) {
    const uint64_t q = mul2(a.nhi, b.hi);
    const uint64_t pe = fma2(a.hi, b.hi, q);
    return Dot2x2{neg2(q), add2(pe, fma2(a.hi, b.lo, mul2(a.lo, b.hi)))};
}

// acc += a * b (the Dot2 step): TwoProduct, Knuth's TwoSum of acc.hi + p written
// with q = -p, and four updates of the error term. 12 paired instructions.
__device__ __forceinline__ void dot2x2_mad(Dot2x2& acc, const DF2m& a, DF2 b) {
    const uint64_t q = mul2(a.nhi, b.hi);                  // -p
    const uint64_t pe = fma2(a.hi, b.hi, q);               // a.hi b.hi - p, exact
    const uint64_t s = sub2(acc.hi, q);                    // fl(acc.hi + p)
    const uint64_t bb = sub2(s, acc.hi);
    const uint64_t e = sub2(sub2(acc.hi, sub2(s, bb)), add2(q, bb));   // acc.hi + p - s, exact
    acc.hi = s;
    acc.err = add2(add2(fma2(a.lo, b.hi, fma2(a.hi, b.lo, acc.err)), pe), e);
}

// acc -= y: the Dot2 step with the factor -1, whose TwoProduct is exact (8 paired
// instructions).
__device__ __forceinline__ void dot2x2_sub(Dot2x2& acc, DF2 y) {
    const uint64_t s = sub2(acc.hi, y.hi);
    const uint64_t bb = sub2(s, acc.hi);
    const uint64_t e = sub2(sub2(acc.hi, sub2(s, bb)), add2(y.hi, bb));
    acc.hi = s;
    acc.err = add2(sub2(acc.err, y.lo), e);
}

// Dekker's Fast2Sum of the two parts: the double-float results.
__device__ __forceinline__ DF2 dot2x2_final(Dot2x2 acc) {
    const uint64_t s = add2(acc.hi, acc.err);
    return DF2{s, sub2(acc.err, sub2(s, acc.hi))};
}

// Lane k of a pair of double-floats, and the scalar Dot2 of lane k.
__device__ __forceinline__ df32 df2_lane0(DF2 v) {
    float h0, h1, l0, l1;
    upk2(v.hi, h0, h1);
    upk2(v.lo, l0, l1);
    return df32(h0, l0);
}
__device__ __forceinline__ df32 df2_lane1(DF2 v) {
    float h0, h1, l0, l1;
    upk2(v.hi, h0, h1);
    upk2(v.lo, l0, l1);
    return df32(h1, l1);
}
__device__ __forceinline__ void dot2x2_split(Dot2x2 a, Dot2& l0, Dot2& l1) {
    upk2(a.hi, l0.hi, l1.hi);
    upk2(a.err, l0.err, l1.err);
}

// Generic accumulation used by the stencil: plain FMA for float / double,
// Dot2 for double-float.
template <typename T> struct Accum {
    using type = T;
    __device__ static T zero() { return T(0); }
    __device__ static T prod(T a, T b) { return a * b; }
    __device__ static void mad(T& acc, T a, T b) { acc = fma(a, b, acc); }
    __device__ static T final(T acc) { return acc; }
};
template <> struct Accum<df32> {
    using type = Dot2;
    __device__ static Dot2 zero() { return dot2_zero(); }
    // an accumulator started at a * b: the exact TwoProduct and the cross terms
    __device__ static Dot2 prod(df32 a, df32 b) {
        const df32 p = df_two_prod(a.hi, b.hi);
        return Dot2{p.hi, __fadd_rn(p.lo, __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi)))};
    }
    __device__ static void mad(Dot2& acc, df32 a, df32 b) { dot2_mad(acc, a, b); }
    __device__ static df32 final(Dot2 acc) { return dot2_final(acc); }
};

}  // namespace dacp
