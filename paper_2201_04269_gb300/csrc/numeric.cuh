// numeric.cuh - complex arithmetic for the two precisions of libmbc.
//
// FP64:  complex double; products and sums in native double (fused multiply-add).
// MIXED: complex "double-float" (each real part a pair hi + lo of floats, about 48
//        significant bits) built from error-free transformations on FP32:
//          TwoSum (Knuth), FastTwoSum (Dekker), TwoProd via fmaf (exact product error),
//        and Dekker's double-length division.  Products use __fmul_rn/__fadd_rn where the
//        rounded value itself is part of an error-free transformation, so the compiler
//        never fuses those operations.
// Accumulators keep an unnormalised (hi, lo) pair and are renormalised once at the end.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mbc {

struct cd { double re, im; };
struct __align__(32) d4 { double x, y, z, w; };
__host__ __device__ __forceinline__ d4 make_d4(double x, double y, double z, double w) { d4 r; r.x = x; r.y = y; r.z = z; r.w = w; return r; }
struct df { float hi, lo; };
struct cdf { df re, im; };

__host__ __device__ __forceinline__ cd cd_make(double r, double i) { cd z; z.re = r; z.im = i; return z; }

// ------------------------------------------------------------------ error-free pieces
__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    df r; r.hi = s; r.lo = e; return r;
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {   // needs |a| >= |b| or a == 0
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    df r; r.hi = s; r.lo = e; return r;
}
__device__ __forceinline__ df df_from_double(double x) {
    df r; r.hi = __double2float_rn(x); r.lo = __double2float_rn(x - (double)r.hi); return r;
}
__device__ __forceinline__ double df_to_double(df x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ df df_neg(df x) { df r; r.hi = -x.hi; r.lo = -x.lo; return r; }
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df df_mul(df x, df y) {
    float p = __fmul_rn(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}
// Dekker's double-length division x / y.
__device__ __forceinline__ df df_div(df x, df y) {
    float q1 = __fdiv_rn(x.hi, y.hi);
    float p = __fmul_rn(q1, y.hi);
    float pe = fmaf(q1, y.hi, -p);
    float r = __fsub_rn(__fsub_rn(x.hi, p), pe);
    r = __fadd_rn(r, __fsub_rn(x.lo, __fmul_rn(q1, y.lo)));
    float q2 = __fdiv_rn(r, y.hi);
    return fast_two_sum(q1, q2);
}

// unnormalised accumulator
struct dacc { float hi, lo; };
__device__ __forceinline__ void dacc_zero(dacc& a) { a.hi = 0.f; a.lo = 0.f; }
// a += x * y
__device__ __forceinline__ void dacc_fma(dacc& a, df x, df y) {
    float p = __fmul_rn(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    float s = __fadd_rn(a.hi, p);
    float bp = __fsub_rn(s, a.hi);
    float t = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, __fadd_rn(t, e));
}
// a += w * x with a float w (exact: w has no low part)
__device__ __forceinline__ void dacc_fma_f(dacc& a, float w, df x) {
    float p = __fmul_rn(x.hi, w);
    float e = fmaf(x.hi, w, -p);
    e = fmaf(x.lo, w, e);
    float s = __fadd_rn(a.hi, p);
    float bp = __fsub_rn(s, a.hi);
    float t = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, __fadd_rn(t, e));
}
// a += x
__device__ __forceinline__ void dacc_add(dacc& a, df x) {
    float s = __fadd_rn(a.hi, x.hi);
    float bp = __fsub_rn(s, a.hi);
    float t = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(x.hi, bp));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, __fadd_rn(t, x.lo));
}
__device__ __forceinline__ df dacc_get(const dacc& a) { return fast_two_sum(a.hi, a.lo); }

// ------------------------------------------------------------------ precision traits
// Each trait provides: value type V (complex), accumulator A, and
//   zero(), acc_zero(A&), fma(A&, V a, V b) [A += a*b], fms(A&, V a, V b) [A -= a*b],
//   get(A) -> V, mul(V, V), add(V, V), neg(V), div(V, V), mag(V) (pivot size),
//   from_cd(cd, scale) [value * 2^scale], to_cd(V) -> cd, is_zero(V).
struct FP64 {
    typedef cd V;
    typedef cd A;
    static constexpr int kind = 0;
    __device__ __forceinline__ static V zero() { return cd_make(0.0, 0.0); }
    __device__ __forceinline__ static V one() { return cd_make(1.0, 0.0); }
    __device__ __forceinline__ static void acc_zero(A& a) { a.re = 0.0; a.im = 0.0; }
    __device__ __forceinline__ static void fma(A& a, V x, V y) {
        a.re = __fma_rn(x.re, y.re, a.re); a.re = __fma_rn(-x.im, y.im, a.re);
        a.im = __fma_rn(x.re, y.im, a.im); a.im = __fma_rn(x.im, y.re, a.im);
    }
    __device__ __forceinline__ static void fms(A& a, V x, V y) {
        a.re = __fma_rn(-x.re, y.re, a.re); a.re = __fma_rn(x.im, y.im, a.re);
        a.im = __fma_rn(-x.re, y.im, a.im); a.im = __fma_rn(-x.im, y.re, a.im);
    }
    __device__ __forceinline__ static void add(A& a, V x) { a.re += x.re; a.im += x.im; }
    // a += w * x for a real w (the real part of a precision-P value)
    __device__ __forceinline__ static void fma_real(A& a, V w, V x) {
        a.re = __fma_rn(w.re, x.re, a.re); a.im = __fma_rn(w.re, x.im, a.im);
    }
    // a += w * x for a real scalar weight
    typedef double S;
    __device__ __forceinline__ static void fma_s(A& a, S w, V x) {
        a.re = __fma_rn(w, x.re, a.re); a.im = __fma_rn(w, x.im, a.im);
    }
    __device__ __forceinline__ static V vadd(V a, V b) { return cd_make(a.re + b.re, a.im + b.im); }
    __device__ __forceinline__ static V get(const A& a) { return a; }
    // accumulator that starts from a value; get_s reads an accumulator fed only by
    // acc_set and fma_s
    __device__ __forceinline__ static void acc_set(A& a, V x) { a = x; }
    __device__ __forceinline__ static V get_s(const A& a) { return a; }
    __device__ __forceinline__ static V mul(V x, V y) {
        return cd_make(__fma_rn(x.re, y.re, -x.im * y.im), __fma_rn(x.re, y.im, x.im * y.re));
    }
    __device__ __forceinline__ static V neg(V x) { return cd_make(-x.re, -x.im); }
    // x for s > 0, -x otherwise, by the sign bits (integer operations only)
    __device__ __forceinline__ static V flip(V x, int s) {
        const long long m = s > 0 ? 0ll : (long long)0x8000000000000000ull;
        return cd_make(__longlong_as_double(__double_as_longlong(x.re) ^ m),
                       __longlong_as_double(__double_as_longlong(x.im) ^ m));
    }
    // Smith's complex division (R. L. Smith, 1962)
    __device__ __forceinline__ static V div(V a, V b) {
        if (fabs(b.re) >= fabs(b.im)) {
            double q = b.im / b.re, d = b.re + b.im * q;
            return cd_make((a.re + a.im * q) / d, (a.im - a.re * q) / d);
        }
        double q = b.re / b.im, d = b.re * q + b.im;
        return cd_make((a.re * q + a.im) / d, (a.im * q - a.re) / d);
    }
    __device__ __forceinline__ static double mag(V x) { return fabs(x.re) + fabs(x.im); }
    __device__ __forceinline__ static bool is_zero(V x) { return x.re == 0.0 && x.im == 0.0; }
    __device__ __forceinline__ static V from_cd(cd x, int) { return x; }
    __device__ __forceinline__ static cd to_cd(V x) { return x; }
    __device__ __forceinline__ static bool scaled() { return false; }
    // smallest pivot magnitude taken as nonzero by the LU
    __device__ __forceinline__ static double tiny() { return 0.0; }
};

struct MIXED {
    typedef cdf V;
    // four independent chains (re: +x.re y.re and -x.im y.im; im: x.re y.im and x.im y.re)
    // so that consecutive multiply-adds do not wait on each other
    struct A { dacc r0, r1, i0, i1; };
    static constexpr int kind = 1;
    __device__ __forceinline__ static V zero() { V z; z.re.hi = z.re.lo = z.im.hi = z.im.lo = 0.f; return z; }
    __device__ __forceinline__ static V one() { V z = zero(); z.re.hi = 1.f; return z; }
    __device__ __forceinline__ static void acc_zero(A& a) { dacc_zero(a.r0); dacc_zero(a.r1); dacc_zero(a.i0); dacc_zero(a.i1); }
    __device__ __forceinline__ static void fma(A& a, V x, V y) {
        dacc_fma(a.r0, x.re, y.re); dacc_fma(a.r1, df_neg(x.im), y.im);
        dacc_fma(a.i0, x.re, y.im); dacc_fma(a.i1, x.im, y.re);
    }
    __device__ __forceinline__ static void fms(A& a, V x, V y) {
        dacc_fma(a.r0, df_neg(x.re), y.re); dacc_fma(a.r1, x.im, y.im);
        dacc_fma(a.i0, df_neg(x.re), y.im); dacc_fma(a.i1, df_neg(x.im), y.re);
    }
    __device__ __forceinline__ static void add(A& a, V x) { dacc_add(a.r0, x.re); dacc_add(a.i0, x.im); }
    // a += w * x for a real w (the real part of a precision-P value)
    __device__ __forceinline__ static void fma_real(A& a, V w, V x) { dacc_fma(a.r0, w.re, x.re); dacc_fma(a.i0, w.re, x.im); }
    // a += w * x for a real scalar weight held exactly in a float
    typedef float S;
    __device__ __forceinline__ static void fma_s(A& a, S w, V x) { dacc_fma_f(a.r0, w, x.re); dacc_fma_f(a.i0, w, x.im); }
    __device__ __forceinline__ static V vadd(V a, V b) { V r; r.re = df_add(a.re, b.re); r.im = df_add(a.im, b.im); return r; }
    // accumulator that starts from a value (chains r0, i0); get_s reads an accumulator fed
    // only by acc_set and fma_s, which leave r1, i1 at zero, as an unnormalised pair
    // (hi + lo with |lo| small: every double-float operation here accepts that form)
    __device__ __forceinline__ static void acc_set(A& a, V x) {
        a.r0.hi = x.re.hi; a.r0.lo = x.re.lo; a.i0.hi = x.im.hi; a.i0.lo = x.im.lo;
        dacc_zero(a.r1); dacc_zero(a.i1);
    }
    __device__ __forceinline__ static V get_s(const A& a) {
        V v; v.re.hi = a.r0.hi; v.re.lo = a.r0.lo; v.im.hi = a.i0.hi; v.im.lo = a.i0.lo; return v;
    }
    __device__ __forceinline__ static V get(const A& a) {
        V v;
        v.re = df_add(dacc_get(a.r0), dacc_get(a.r1));
        v.im = df_add(dacc_get(a.i0), dacc_get(a.i1));
        return v;
    }
    __device__ __forceinline__ static V mul(V x, V y) {
        A a; acc_zero(a); fma(a, x, y); return get(a);
    }
    __device__ __forceinline__ static V neg(V x) { V r; r.re = df_neg(x.re); r.im = df_neg(x.im); return r; }
    // x for s > 0, -x otherwise, by the sign bits (integer operations only)
    __device__ __forceinline__ static V flip(V x, int s) {
        const unsigned m = s > 0 ? 0u : 0x80000000u;
        V r;
        r.re.hi = __uint_as_float(__float_as_uint(x.re.hi) ^ m); r.re.lo = __uint_as_float(__float_as_uint(x.re.lo) ^ m);
        r.im.hi = __uint_as_float(__float_as_uint(x.im.hi) ^ m); r.im.lo = __uint_as_float(__float_as_uint(x.im.lo) ^ m);
        return r;
    }
    // Smith's complex division in double-float arithmetic
    __device__ __forceinline__ static V div(V a, V b) {
        V r;
        if (fabsf(b.re.hi) >= fabsf(b.im.hi)) {
            df q = df_div(b.im, b.re);
            df d = df_add(b.re, df_mul(b.im, q));
            r.re = df_div(df_add(a.re, df_mul(a.im, q)), d);
            r.im = df_div(df_add(a.im, df_neg(df_mul(a.re, q))), d);
        } else {
            df q = df_div(b.re, b.im);
            df d = df_add(df_mul(b.re, q), b.im);
            r.re = df_div(df_add(df_mul(a.re, q), a.im), d);
            r.im = df_div(df_add(df_mul(a.im, q), df_neg(a.re)), d);
        }
        return r;
    }
    __device__ __forceinline__ static float mag(V x) { return fabsf(x.re.hi) + fabsf(x.im.hi); }
    __device__ __forceinline__ static bool is_zero(V x) { return x.re.hi == 0.f && x.im.hi == 0.f; }
    __device__ __forceinline__ static V from_cd(cd x, int e) {
        V r; r.re = df_from_double(ldexp(x.re, e)); r.im = df_from_double(ldexp(x.im, e)); return r;
    }
    __device__ __forceinline__ static cd to_cd(V x) { return cd_make(df_to_double(x.re), df_to_double(x.im)); }
    __device__ __forceinline__ static bool scaled() { return true; }
    // Blocks are scaled to entries of order one; a pivot below 2^-64 is rounding residue
    // of repeated rows or columns (a zero-determinant tuple), and inverting it could
    // leave the FP32 exponent range, so the LU treats it as an exact zero.
    __device__ __forceinline__ static float tiny() { return 0x1p-64f; }
};

// 16-byte read-only load of a precision-P value from global memory
template <class V>
__device__ __forceinline__ V ldv(const void* base, int64_t i) {
    union { int4 raw; V v; } u;
    u.raw = __ldg(reinterpret_cast<const int4*>(base) + i);
    return u.v;
}

// conjugate
__device__ __forceinline__ cd conj(cd x) { return cd_make(x.re, -x.im); }
__device__ __forceinline__ cdf conj(cdf x) { cdf r = x; r.im = df_neg(x.im); return r; }

// ------------------------------------------------------------------ double reductions
// Compensated double accumulator (TwoSum of each addend, errors summed separately).
struct kacc { double hi, lo; };
__device__ __forceinline__ void kacc_add(kacc& s, double x) {
    double t = __dadd_rn(s.hi, x);
    double bp = __dsub_rn(t, s.hi);
    s.lo = __dadd_rn(s.lo, __dadd_rn(__dsub_rn(s.hi, __dsub_rn(t, bp)), __dsub_rn(x, bp)));
    s.hi = t;
}
__device__ __forceinline__ void kacc_merge(kacc& s, kacc o) { kacc_add(s, o.hi); s.lo = __dadd_rn(s.lo, o.lo); }

// Exponent e with max |re|, |im| of a 12x12 block in [0.5, 1) after scaling by 2^-e
// (0 for an all-zero block).
__device__ __forceinline__ int block_exponent(double m) {
    if (m == 0.0 || !isfinite(m)) return 0;
    int e; frexp(m, &e); return e;
}

}  // namespace mbc
