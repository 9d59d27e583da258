// Arithmetic policies of the three value types (device code).
//
//  I64   int64 values, wrapping adds: exact.
//  F64   fp64 values, plain fp64 adds.
//  F32C  fp32 double-word values (hi, lo), value = hi + lo.
//          - chain prefix scan: double-word + double-word addition,
//            "AccurateDWPlusDW" of Joldes, Muller, Popescu, "Tight and
//            rigorous error bounds for basic building blocks of double-word
//            arithmetic", ACM TOMS 44(2), 2017 (Alg. 6 there), relative error
//            below 3u^2 + 13u^3 per addition (u = 2^-24);
//          - gather: cascaded summation "Sum2" of Ogita, Rump, Oishi,
//            "Accurate sum and dot product", SIAM J. Sci. Comput. 26(6), 2005
//            (Alg. 4.4 there): the hi parts go through an error-free TwoSum
//            chain, the rounding errors and the lo parts are summed in fp32,
//            and the pair is normalised once at the end;
//          - Moebius: fp64 prefixes (the forward substitution cancels).
//        The error-free transformations are Knuth's TwoSum and Dekker's
//        Fast2Sum, written with __fadd_rn / __fsub_rn so that nvcc cannot
//        contract or reorder them.
#pragma once

#include <cstdint>

namespace mz {

// ---------------------------------------------------------------- error-free transformations
struct DW {
    float hi, lo;
};

__device__ __forceinline__ DW two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float ap = __fsub_rn(s, b);
    float bp = __fsub_rn(s, ap);
    float da = __fsub_rn(a, ap);
    float db = __fsub_rn(b, bp);
    return {s, __fadd_rn(da, db)};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ DW fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float z = __fsub_rn(s, a);
    return {s, __fsub_rn(b, z)};
}

__device__ __forceinline__ DW dw_add(DW x, DW y) {
    DW s = two_sum(x.hi, y.hi);
    DW t = two_sum(x.lo, y.lo);
    float c = __fadd_rn(s.lo, t.hi);
    DW v = fast_two_sum(s.hi, c);
    float w = __fadd_rn(t.lo, v.lo);
    return fast_two_sum(v.hi, w);
}

// ---------------------------------------------------------------- packed fp32 pairs
// Two fp32 values in one 64-bit register pair (the first in the low half), operated on
// by the paired fp32 instructions of sm_100 and later: one instruction, two IEEE
// round-to-nearest operations, each with the result __fadd_rn / __fsub_rn gives, so a
// pair runs the same error-free transformations as two scalar lanes, bit for bit.
using f32x2 = unsigned long long;

__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Knuth's TwoSum on both halves: s + e = a + b exactly.
__device__ __forceinline__ void two_sum2(f32x2 a, f32x2 b, f32x2 &s, f32x2 &e) {
    s = f2_add(a, b);
    const f32x2 ap = f2_sub(s, b);
    const f32x2 bp = f2_sub(s, ap);
    e = f2_add(f2_sub(a, ap), f2_sub(b, bp));
}

// Dekker's Fast2Sum on both halves (|a| >= |b| or a == 0 in each).
__device__ __forceinline__ void fast_two_sum2(f32x2 a, f32x2 b, f32x2 &s, f32x2 &e) {
    s = f2_add(a, b);
    e = f2_sub(b, f2_sub(s, a));
}

__device__ __forceinline__ f32x2 f2_neg(f32x2 a) { return a ^ 0x8000000080000000ull; }

// dw_add on both halves: (xh, xl) + (yh, yl) -> (rh, rl).
__device__ __forceinline__ void dw_add2(f32x2 xh, f32x2 xl, f32x2 yh, f32x2 yl, f32x2 &rh, f32x2 &rl) {
    f32x2 sh, sl, th, tl, vh, vl;
    two_sum2(xh, yh, sh, sl);
    two_sum2(xl, yl, th, tl);
    fast_two_sum2(sh, f2_add(sl, th), vh, vl);
    fast_two_sum2(vh, f2_add(tl, vl), rh, rl);
}

// Sum2 accumulator of two columns (the fp32 pair form of PolF32C::Acc).
struct Acc2 {
    f32x2 s, e;
};
__device__ __forceinline__ void acc2_add(Acc2 &a, f32x2 hi, f32x2 lo) {
    f32x2 t, err;
    two_sum2(a.s, hi, t, err);
    a.s = t;
    a.e = f2_add(a.e, f2_add(err, lo));
}

// ---------------------------------------------------------------- value policies
// Each policy gives:
//   P_t            the element type of the zeta prefix array (8 bytes)
//   load_in(p, i)  input element i of a [n][B] array (F32C: hi plane, lo plane at +nB)
//   scan_add       the operator of the chain prefix scan
//   Acc / acc_*    the gather accumulator
//   store_out      output element i
struct PolI64 {
    using P_t = long long;
    using Acc = long long;
    static __device__ __forceinline__ P_t zero() { return 0; }
    static __device__ __forceinline__ P_t load_in(const void *p, int64_t i, int64_t) {
        return reinterpret_cast<const long long *>(p)[i];
    }
    static __device__ __forceinline__ P_t scan_add(P_t a, P_t b) {
        return (long long)((unsigned long long)a + (unsigned long long)b);
    }
    static __device__ __forceinline__ Acc acc_zero() { return 0; }
    static __device__ __forceinline__ void acc_add(Acc &a, P_t v) {
        a = (long long)((unsigned long long)a + (unsigned long long)v);
    }
    static __device__ __forceinline__ void store_out(void *p, int64_t i, int64_t, Acc a) {
        reinterpret_cast<long long *>(p)[i] = a;
    }
};

struct PolF64 {
    using P_t = double;
    using Acc = double;
    static __device__ __forceinline__ P_t zero() { return 0.0; }
    static __device__ __forceinline__ P_t load_in(const void *p, int64_t i, int64_t) {
        return reinterpret_cast<const double *>(p)[i];
    }
    static __device__ __forceinline__ P_t scan_add(P_t a, P_t b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ Acc acc_zero() { return 0.0; }
    static __device__ __forceinline__ void acc_add(Acc &a, P_t v) { a = __dadd_rn(a, v); }
    static __device__ __forceinline__ void store_out(void *p, int64_t i, int64_t, Acc a) {
        reinterpret_cast<double *>(p)[i] = a;
    }
};

struct PolF32C {
    using P_t = float2;  // (hi, lo)
    struct Acc {
        float s, e;      // running TwoSum sum of the hi parts, fp32 sum of errors and lo parts
    };
    static __device__ __forceinline__ P_t zero() { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ P_t load_in(const void *p, int64_t i, int64_t nB) {
        const float *q = reinterpret_cast<const float *>(p);
        return make_float2(q[i], q[nB + i]);
    }
    static __device__ __forceinline__ P_t scan_add(P_t a, P_t b) {
        DW r = dw_add({a.x, a.y}, {b.x, b.y});
        return make_float2(r.hi, r.lo);
    }
    static __device__ __forceinline__ Acc acc_zero() { return {0.f, 0.f}; }
    static __device__ __forceinline__ void acc_add(Acc &a, P_t v) {
        DW t = two_sum(a.s, v.x);
        a.s = t.hi;
        a.e = __fadd_rn(a.e, __fadd_rn(t.lo, v.y));
    }
    static __device__ __forceinline__ void store_out(void *p, int64_t i, int64_t nB, Acc a) {
        DW r = two_sum(a.s, a.e);   // normalise once; |e| may exceed |s| after cancellation
        float *q = reinterpret_cast<float *>(p);
        q[i] = r.hi;
        q[nB + i] = r.lo;
    }
};

// ---------------------------------------------------------------- Moebius value policies
// The forward substitution keeps y' in a 64-bit word per (slot, column) that
// doubles as the readiness flag: the workspace is filled with a sentinel
// first and a consumer polls until the word differs from it.
//
// int64: every 64-bit pattern is a possible value, INT64_MIN included, so a value
// equal to the sentinel is published as kSentinel + 1 with an escape flag set for
// its word first (kEscapes); a reader that sees kSentinel + 1 checks the flag.
// This keeps the int64 transform exact modulo 2^64 for every input.
struct MobI64 {
    using T = long long;
    static constexpr bool kEscapes = true;
    static constexpr bool kDW = false;
    static constexpr unsigned long long kSentinel = 0x8000000000000000ull;  // INT64_MIN
    static __device__ __forceinline__ T from_bits(unsigned long long b) { return (long long)b; }
    static __device__ __forceinline__ unsigned long long to_bits(T v) { return (unsigned long long)v; }
    static __device__ __forceinline__ T add(T a, T b) {
        return (long long)((unsigned long long)a + (unsigned long long)b);
    }
    static __device__ __forceinline__ T sub(T a, T b) {
        return (long long)((unsigned long long)a - (unsigned long long)b);
    }
    static __device__ __forceinline__ T load_in(const void *p, int64_t i, int64_t) {
        return reinterpret_cast<const long long *>(p)[i];
    }
    static __device__ __forceinline__ void store_out(void *p, int64_t i, int64_t, T v) {
        reinterpret_cast<long long *>(p)[i] = v;
    }
};

struct MobF64 {
    using T = double;
    static constexpr bool kEscapes = false;
    static constexpr bool kDW = false;
    // a signalling-NaN pattern: fp64 arithmetic never produces it (results are quiet)
    static constexpr unsigned long long kSentinel = 0xFFF4000DEADBEEFull;
    static __device__ __forceinline__ T from_bits(unsigned long long b) { return __longlong_as_double((long long)b); }
    static __device__ __forceinline__ unsigned long long to_bits(T v) {
        unsigned long long b = (unsigned long long)__double_as_longlong(v);
        return b == kSentinel ? 0x7FF8000000000000ull : b;   // that NaN input copied through: another NaN
    }
    static __device__ __forceinline__ T add(T a, T b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ T sub(T a, T b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ T load_in(const void *p, int64_t i, int64_t) {
        return reinterpret_cast<const double *>(p)[i];
    }
    static __device__ __forceinline__ void store_out(void *p, int64_t i, int64_t, T v) {
        reinterpret_cast<double *>(p)[i] = v;
    }
};

// F32C Moebius: pair planes in and out, fp64 prefixes in the forward substitution.
struct MobF32C : MobF64 {
    static constexpr bool kDW = true;
    static __device__ __forceinline__ T load_in(const void *p, int64_t i, int64_t nB) {
        const float *q = reinterpret_cast<const float *>(p);
        return __dadd_rn((double)q[i], (double)q[nB + i]);
    }
    static __device__ __forceinline__ void store_out(void *p, int64_t i, int64_t nB, T v) {
        float hi = __double2float_rn(v);
        float lo = __double2float_rn(__dsub_rn(v, (double)hi));
        float *q = reinterpret_cast<float *>(p);
        q[i] = hi;
        q[nB + i] = lo;
    }
    // the double-word copy of a prefix the forward substitution publishes for the
    // later stages (leaf gather, V^-1), which run in compensated fp32
    static __device__ __forceinline__ float2 to_dw(T v) {
        float hi = __double2float_rn(v);
        return make_float2(hi, __double2float_rn(__dsub_rn(v, (double)hi)));
    }
};

// ---------------------------------------------------------------- leaf gather policies
// After the forward substitution has produced y' at every slot some other row reads,
// the remaining rows (read by no other row) are a plain gather:
// y'(x) = g(x) - sum_j y'(niv_j(x)) over the gather's tiled map, whose entry on x's own
// chain is x's own slot, zeroed beforehand so that it adds nothing. Each policy gives
// the word type W of the prefix array it reads and writes, the accumulator, and the
// final subtraction from g(x).
struct LeafI64 {
    using W = long long;
    using Acc = long long;
    static __device__ __forceinline__ Acc acc_zero() { return 0; }
    static __device__ __forceinline__ void acc_add(Acc &a, W v) {
        a = (long long)((unsigned long long)a + (unsigned long long)v);
    }
    static __device__ __forceinline__ W result(const void *g, int64_t i, int64_t, const Acc &a) {
        return (long long)((unsigned long long)reinterpret_cast<const long long *>(g)[i] - (unsigned long long)a);
    }
};

struct LeafF64 {
    using W = double;
    using Acc = double;
    static __device__ __forceinline__ Acc acc_zero() { return 0.0; }
    static __device__ __forceinline__ void acc_add(Acc &a, W v) { a = __dadd_rn(a, v); }
    static __device__ __forceinline__ W result(const void *g, int64_t i, int64_t, const Acc &a) {
        return __dsub_rn(reinterpret_cast<const double *>(g)[i], a);
    }
};

// Compensated fp32: Sum2 (as the zeta gather) over the double-word prefixes, then
// g(x) minus the sum in double-word arithmetic.
struct LeafF32C {
    using W = float2;
    using Acc = PolF32C::Acc;
    static __device__ __forceinline__ Acc acc_zero() { return {0.f, 0.f}; }
    static __device__ __forceinline__ void acc_add(Acc &a, W v) { PolF32C::acc_add(a, v); }
    static __device__ __forceinline__ W result(const void *g, int64_t i, int64_t nB, const Acc &a) {
        const float *q = reinterpret_cast<const float *>(g);
        const DW s = two_sum(a.s, a.e);
        const DW r = dw_add({q[i], q[nB + i]}, {-s.hi, -s.lo});
        return make_float2(r.hi, r.lo);
    }
};

}  // namespace mz
