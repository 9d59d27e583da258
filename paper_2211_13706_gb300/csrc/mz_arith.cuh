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
struct MobI64 {
    using T = long long;
    static constexpr unsigned long long kSentinel = 0x8000000000000000ull;  // INT64_MIN
    static __device__ __forceinline__ T from_bits(unsigned long long b) { return (long long)b; }
    static __device__ __forceinline__ unsigned long long to_bits(T v) {
        // INT64_MIN itself is outside the documented value range; never publish the sentinel
        unsigned long long b = (unsigned long long)v;
        return b == kSentinel ? kSentinel + 1 : b;
    }
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
    // a signalling-NaN pattern: fp64 arithmetic never produces it (results are quiet)
    static constexpr unsigned long long kSentinel = 0xFFF4000DEADBEEFull;
    static __device__ __forceinline__ T from_bits(unsigned long long b) { return __longlong_as_double((long long)b); }
    static __device__ __forceinline__ unsigned long long to_bits(T v) {
        unsigned long long b = (unsigned long long)__double_as_longlong(v);
        return b == kSentinel ? 0x7FF8000000000000ull : b;   // an input copied through unchanged
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

// F32C Moebius: pair planes in and out, fp64 prefixes in between.
struct MobF32C : MobF64 {
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
};

}  // namespace mz
