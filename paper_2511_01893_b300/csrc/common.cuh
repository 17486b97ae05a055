// common.cuh - types and helpers shared by the laminography kernels.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace lam {

// Complex element of precision T, interleaved (re, im): float2 / double2 layout.
template <typename T> struct C;
template <> struct __align__(8) C<float> {
    float x, y;
};
template <> struct __align__(16) C<double> {
    double x, y;
};

template <typename T> __host__ __device__ __forceinline__ C<T> cmake(T re, T im) {
    C<T> r;
    r.x = re;
    r.y = im;
    return r;
}
template <typename T> __host__ __device__ __forceinline__ C<T> cadd(C<T> a, C<T> b) {
    return cmake<T>(a.x + b.x, a.y + b.y);
}
template <typename T> __host__ __device__ __forceinline__ C<T> csub(C<T> a, C<T> b) {
    return cmake<T>(a.x - b.x, a.y - b.y);
}
// Products of complex numbers are written with explicit fused multiply-adds:
// an expression a b - c d could otherwise be fused either way by the compiler,
// depending on the surrounding code, so the same butterfly inlined into two
// kernels could round differently.  With the fusion spelled out every kernel
// variant (runtime or compile-time FFT length, pipelined or not, single-plan
// or batched) computes bitwise the same values.
template <typename T> __host__ __device__ __forceinline__ C<T> cmul(C<T> a, C<T> b) {
    return cmake<T>(fma(a.x, b.x, -(a.y * b.y)), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
template <typename T> __host__ __device__ __forceinline__ C<T> cmulc(C<T> a, C<T> b) {
    return cmake<T>(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -(a.x * b.y)));
}
template <typename T> __host__ __device__ __forceinline__ C<T> cscale(C<T> a, T s) {
    return cmake<T>(a.x * s, a.y * s);
}
template <typename T> __host__ __device__ __forceinline__ C<T> cconj(C<T> a) {
    return cmake<T>(a.x, -a.y);
}
// multiply by i^dir, dir = +1 (i) or -1 (-i)
template <int DIR, typename T> __host__ __device__ __forceinline__ C<T> cmul_i(C<T> a) {
    return DIR > 0 ? cmake<T>(-a.y, a.x) : cmake<T>(a.y, -a.x);
}

// Fast exponential for Gaussian weights: exp(x) for x <= 0.
#ifdef LAM_ACCURATE_EXP
__device__ __forceinline__ float gexp(float x) { return expf(x); }
#else
__device__ __forceinline__ float gexp(float x) { return __expf(x); }
#endif
__device__ __forceinline__ double gexp(double x) { return exp(x); }

// Per-angle slice-coordinate constants.  Grid position of the point (ku, kv)
// along padded axis a is ku * A_a + kv * S_a (a = x: M1 cos th / w,
// M1 sin phi sin th / h; a = y: M2 sin th / w, -M2 sin phi cos th / h).
// FP32 kernels carry each constant as an unevaluated sum hi + lo so that the
// position keeps ~1e-7 absolute accuracy at |position| ~ 2000.
// high parts first: the line tests read only them (one 16-byte load)
struct __align__(16) AngleF {
    float ax_hi, sx_hi, ay_hi, sy_hi, ax_lo, sx_lo, ay_lo, sy_lo;
};
struct AngleD {
    double ax, sx, ay, sy;
};

// Tap window: j0 = floor(t + kTapShift) for a grid position t, fr = t - j0 in
// [-kTapShift, 1 - kTapShift).  The shift keeps the window switch away from
// grid nodes, where whole lines of slice points sit up to ~1e-16 at angles
// that are multiples of pi/2; there FP32 and FP64 arithmetic would otherwise
// pick different windows from rounding noise alone.
constexpr double kTapShift = 1.0 / 131072.0;  // 2^-17

// floor and fractional part of ku*a + kv*s, a = a_hi + a_lo, s = s_hi + s_lo.
// ku and kv are small integers, so ku*a_hi and kv*s_hi are split exactly with
// fma; the sum is carried as (hi, lo) and the floor taken on the pair.
__device__ __forceinline__ void grid_pos(int ku, int kv, float a_hi, float a_lo, float s_hi,
                                         float s_lo, int& j0, float& fr) {
    // __f*_rn intrinsics are never contracted into fma, which the exact
    // splits below rely on.
    const float fku = (float)ku, fkv = (float)kv;
    const float p1 = __fmul_rn(fku, a_hi);
    const float e1 = fmaf(fku, a_hi, -p1);
    const float p2 = __fmul_rn(fkv, s_hi);
    const float e2 = fmaf(fkv, s_hi, -p2);
    // two-sum p1 + p2 = s + t exactly
    const float s = __fadd_rn(p1, p2);
    const float bb = __fsub_rn(s, p1);
    const float t = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bb)), __fsub_rn(p2, bb));
    const float lo = t + e1 + e2 + fku * a_lo + fkv * s_lo;
    float fl = floorf(s);
    float f = __fsub_rn(s, fl) + (lo + (float)kTapShift);  // s - fl is exact
    if (f >= 1.0f) {
        f -= 1.0f;
        fl += 1.0f;
    } else if (f < 0.0f) {
        f += 1.0f;
        fl -= 1.0f;
    }
    j0 = (int)fl;
    fr = f - (float)kTapShift;
}
__device__ __forceinline__ void grid_pos(int ku, int kv, double a, double s, int& j0, double& fr) {
    const double p = fma((double)ku, a, (double)kv * s);
    const double fl = floor(p + kTapShift);
    j0 = (int)fl;
    fr = p - fl;
}

// Index checks (LAM_BOUNDS_CHECK builds).  LAM_INB(i, n, err, site) is true
// when 0 <= i < n; otherwise it records `site` in the plan's error word *err
// (the first failing site wins) and is false, and the caller skips the access:
// no trap, no out-of-range access.  In other builds it is the constant true.
enum { kSiteZWeights = 1, kSiteGatherWindow = 2, kSiteGatherOut = 3, kSiteSpreadIn = 4, kSiteSelftest = 99 };
#ifdef LAM_BOUNDS_CHECK
__device__ __forceinline__ bool lam_in_bounds(long long i, long long n, int* err, int site) {
    if (i >= 0 && i < n) return true;
    if (err) atomicCAS(err, 0, site);
    return false;
}
#define LAM_INB(i, n, err, site) ::lam::lam_in_bounds((long long)(i), (long long)(n), (err), (site))
#else
#define LAM_INB(i, n, err, site) true
#endif

// j mod M in [0, M) for any M >= 1 (a mask when M is a power of two)
__host__ __device__ __forceinline__ int wrap(int j, int M) {
    if ((M & (M - 1)) == 0) return j & (M - 1);
    const int r = j % M;
    return r < 0 ? r + M : r;
}

// Asynchronous global -> shared copy of one complex element (cp.async: no
// register staging, so every copy a thread issues is in flight at once).
// After cp_async_wait_all() a thread sees its own copies; other threads'
// copies need a barrier as well.
template <typename T> __device__ __forceinline__ void cp_async_elem(C<T>* dst, const C<T>* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(C<T>) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

}  // namespace lam
