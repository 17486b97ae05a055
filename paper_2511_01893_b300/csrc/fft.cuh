// fft.cuh - batched mixed-radix FFTs in shared memory (Stockham autosort).
//
// Each call transforms `nlines` lines of length N = 2^a 3^b 5^c stored at
// stride `lstride` in shared memory.  The power-of-two part runs as radix-8
// stages (then one radix-4 or radix-2 stage), followed by radix-3 and radix-5
// stages; every thread of the block takes butterflies q = tid, tid + nthr, ...
// of a stage, reads R inputs N/R apart, applies twiddles, does an in-register
// radix-R DFT and writes the R outputs Ns apart (self-sorting, so the result
// is in natural order).  The stage sequence is a code from fft_code(N).
//
// Sign convention: DIR = -1 computes sum_x a[x] exp(-2 pi i j x / N),
// DIR = +1 computes sum_x a[x] exp(+2 pi i j x / N) (no normalisation).
// Twiddles come from a table tw[q] = exp(-2 pi i q / Nmax), q < Nmax, where
// Nmax is a multiple of N (twstride = Nmax / N).
#pragma once

#include "common.cuh"

namespace lam {

template <int DIR, typename T> __device__ __forceinline__ void dft2(C<T>* v) {
    const C<T> a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <int DIR, typename T> __device__ __forceinline__ void dft4(C<T>* v) {
    const C<T> a0 = cadd(v[0], v[2]);
    const C<T> a1 = csub(v[0], v[2]);
    const C<T> a2 = cadd(v[1], v[3]);
    const C<T> a3 = cmul_i<DIR>(csub(v[1], v[3]));
    v[0] = cadd(a0, a2);
    v[2] = csub(a0, a2);
    v[1] = cadd(a1, a3);
    v[3] = csub(a1, a3);
}

template <int DIR, typename T> __device__ __forceinline__ void dft8(C<T>* v) {
    C<T> e[4] = {v[0], v[2], v[4], v[6]};
    C<T> o[4] = {v[1], v[3], v[5], v[7]};
    dft4<DIR>(e);
    dft4<DIR>(o);
    const T r = (T)0.70710678118654752440;
    // W8^k = exp(DIR 2 pi i k / 8)
    const C<T> o1 = cmake<T>(r * (o[1].x - DIR * o[1].y), r * (o[1].y + DIR * o[1].x));
    const C<T> o2 = cmul_i<DIR>(o[2]);
    const C<T> o3 = cmake<T>(r * (-o[3].x - DIR * o[3].y), r * (-o[3].y + DIR * o[3].x));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
}

// radix-16 DFT as 4 x 4, in place: with x[4 n1 + n2], DFT-4 over n1 for each
// n2, twiddle by W16^(n2 k1) (W16 = e^{DIR 2 pi i / 16}), then DFT-4 over n2
// for each k1.  Output k1 + 4 k2 is left in v[4 k1 + k2] (transposed order;
// dft16_out maps an output index to its register).
__host__ __device__ constexpr int dft16_out(int r) { return 4 * (r & 3) + (r >> 2); }

template <int DIR, typename T> __device__ __forceinline__ void dft16(C<T>* v) {
    const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;  // cos, sin (pi / 8)
    const T r2 = (T)0.70710678118654752440;
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        C<T> t[4] = {v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]};
        dft4<DIR>(t);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) v[n2 + 4 * k1] = t[k1];  // a[n2][k1] at v[n2 + 4 k1]
    }
    // W16^e, e = n2 k1 in {1, 2, 3, 4, 6, 9}: multiply by cos + DIR i sin of 2 pi e / 16
    auto tw = [&](C<T> x, T c, T sn) {
        return cmake<T>(fma(x.x, c, (T)(-DIR) * (x.y * sn)), fma(x.y, c, (T)DIR * (x.x * sn)));
    };
    v[1 + 4] = tw(v[1 + 4], c1, s1);      // n2 1, k1 1
    v[1 + 8] = tw(v[1 + 8], r2, r2);      // n2 1, k1 2
    v[2 + 4] = tw(v[2 + 4], r2, r2);      // n2 2, k1 1
    v[1 + 12] = tw(v[1 + 12], s1, c1);    // n2 1, k1 3
    v[3 + 4] = tw(v[3 + 4], s1, c1);      // n2 3, k1 1
    v[2 + 8] = cmul_i<DIR>(v[2 + 8]);     // n2 2, k1 2
    v[2 + 12] = tw(v[2 + 12], -r2, r2);   // n2 2, k1 3
    v[3 + 8] = tw(v[3 + 8], -r2, r2);     // n2 3, k1 2
    v[3 + 12] = tw(v[3 + 12], -c1, -s1);  // n2 3, k1 3
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<DIR>(v + 4 * k1);  // over n2; result k2 at v[4 k1 + k2]
}

// radix-3 DFT: with c = -1/2 and s = DIR sqrt(3)/2 (the primitive cube root
// of unity e^{DIR 2 pi i / 3} = c + i s)
template <int DIR, typename T> __device__ __forceinline__ void dft3(C<T>* v) {
    const T hs = (T)0.86602540378443864676;
    const C<T> b = cadd(v[1], v[2]);
    const C<T> d = csub(v[1], v[2]);
    const C<T> t = cmake<T>(fma((T)-0.5, b.x, v[0].x), fma((T)-0.5, b.y, v[0].y));
    const C<T> e = cmul_i<DIR>(cmake<T>(hs * d.x, hs * d.y));
    v[0] = cadd(v[0], b);
    v[1] = cadd(t, e);
    v[2] = csub(t, e);
}

// radix-5 DFT from the pairs b_k = a_k + a_{5-k}, d_k = a_k - a_{5-k}:
// y_1,4 = a_0 + c1 b_1 + c2 b_2 +- DIR i (s1 d_1 + s2 d_2),
// y_2,3 = a_0 + c2 b_1 + c1 b_2 +- DIR i (s2 d_1 - s1 d_2),
// c_k = cos(2 pi k / 5), s_k = sin(2 pi k / 5)
template <int DIR, typename T> __device__ __forceinline__ void dft5(C<T>* v) {
    const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;
    const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;
    const C<T> b1 = cadd(v[1], v[4]), d1 = csub(v[1], v[4]);
    const C<T> b2 = cadd(v[2], v[3]), d2 = csub(v[2], v[3]);
    const C<T> t1 = cmake<T>(fma(c2, b2.x, fma(c1, b1.x, v[0].x)), fma(c2, b2.y, fma(c1, b1.y, v[0].y)));
    const C<T> t2 = cmake<T>(fma(c1, b2.x, fma(c2, b1.x, v[0].x)), fma(c1, b2.y, fma(c2, b1.y, v[0].y)));
    const C<T> e1 = cmul_i<DIR>(cmake<T>(fma(s1, d1.x, s2 * d2.x), fma(s1, d1.y, s2 * d2.y)));
    const C<T> e2 = cmul_i<DIR>(cmake<T>(fma(s2, d1.x, -(s1 * d2.x)), fma(s2, d1.y, -(s1 * d2.y))));
    v[0] = cadd(v[0], cadd(b1, b2));
    v[1] = cadd(t1, e1);
    v[4] = csub(t1, e1);
    v[2] = cadd(t2, e2);
    v[3] = csub(t2, e2);
}

// ---------------------------------------------------------------------------
// Stage codes: 3 bits per stage, first stage in the low bits; 1 -> radix 2,
// 2 -> radix 4, 3 -> radix 8, 4 -> radix 3, 5 -> radix 5, 0 ends.  The
// power-of-two stages come first, so Ns is a power of two in them.
// ---------------------------------------------------------------------------

__host__ __device__ constexpr int fft_stage_radix(int c) {
    return c == 1 ? 2 : c == 2 ? 4 : c == 3 ? 8 : c == 4 ? 3 : c == 5 ? 5 : c == 6 ? 16 : 1;
}

// code for length N, or -1 if N is not 2^a 3^b 5^c (N >= 2) or needs more
// than 10 stages.  The power-of-two part uses the fewest stages of radix at
// most maxr (16 or 8), its bits spread evenly (2048 = 16 16 8 with maxr 16).
inline int fft_code(int N, int maxr = 8) {
    if (N < 2) return -1;
    int a = 0, m = N;
    while (m % 2 == 0) { m /= 2; ++a; }
    int codes[16], ns = 0;
    const int maxbits = maxr >= 16 ? 4 : 3;
    const int nst = (a + maxbits - 1) / maxbits;
    for (int k = 0; k < nst; ++k) {
        const int bits = (a + (nst - k) - 1) / (nst - k);  // ceil of the remaining share
        codes[ns++] = bits == 4 ? 6 : bits == 3 ? 3 : bits == 2 ? 2 : 1;
        a -= bits;
    }
    while (m % 3 == 0) { m /= 3; codes[ns++] = 4; if (ns > 10) return -1; }
    while (m % 5 == 0) { m /= 5; codes[ns++] = 5; if (ns > 10) return -1; }
    if (m != 1) return -1;
    int code = 0;
    for (int i = ns - 1; i >= 0; --i) code = (code << 3) | codes[i];
    return code;
}

// Butterflies per thread of a radix-R stage for a register budget MAXB (in
// radix-8 butterflies): the power-of-two stages hold 8 MAXB values; the
// radix-3 and radix-5 stages, whose butterflies need more temporaries, hold
// fewer (4 MAXB / 2 MAXB butterflies -> 12 / 10 values at MAXB = 2).
__host__ __device__ constexpr int fft_stage_maxb(int R, int maxb) {
    return R == 3 ? 2 * maxb : R == 5 ? maxb : (8 * maxb) / R;
}
// largest power-of-two radix a precision's register budget holds (one
// radix-16 butterfly per thread needs MAXB = 2)
template <typename T> constexpr int fft_max_radix() { return sizeof(T) == 4 ? 16 : 8; }

// true when the code has a radix-3 or radix-5 stage (those kernels are built
// separately: the extra stage kinds cost registers in the power-of-two ones)
inline bool fft_mixed(int code) {
    for (int c = code; c; c >>= 3)
        if ((c & 7) == 4 || (c & 7) == 5) return true;
    return false;
}

// Most elements per thread the stages of `code` cover: the minimum of
// R * fft_stage_maxb(R) over its radices; a call needs
// nlines * N <= fft_capacity(code, MAXB) * blockDim.x.
inline int fft_capacity(int code, int maxb) {
    int cap = 8 * maxb;
    for (int c = code; c; c >>= 3) {
        const int R = fft_stage_radix(c & 7);
        const int v = R * fft_stage_maxb(R, maxb);
        if (v < cap) cap = v;
    }
    return cap;
}

// ---------------------------------------------------------------------------
// In-place variant: one shared buffer.  Each stage first loads every
// butterfly input the thread owns into registers (at most MAXB butterflies of
// radix <= 8 per thread: nlines * N <= 8 * MAXB * blockDim.x), synchronises,
// then writes the outputs.  Half the shared memory of the ping-pong form, so
// blocks can hold twice the lines.
//
// Element e of a line lives at fpad(e) = e + e / 16: one pad slot per 16
// complex values keeps the stride-R stores of the early stages free of bank
// conflicts.  A line of length N occupies fpad_len(N) slots.
// Twiddles: per butterfly w^1, w^2, w^4 come from the table, the rest are
// products (w^3 = w w^2, w^5 = w w^4, w^6 = w^2 w^4, w^7 = w^3 w^4).
// ---------------------------------------------------------------------------

__host__ __device__ __forceinline__ int fpad(int e) { return e + (e >> 4); }
__host__ __device__ __forceinline__ int fpad_len(int n) { return n + (n >> 4) + 1; }

// idx1 = k * twstep with k < Ns and twstep = (N / (Ns R)) twstride, so
// r * idx1 < Nmax for every r < R: the table needs no index reduction.
template <int R, int DIR, typename T>
__device__ __forceinline__ void twiddles(C<T>* wv, const C<T>* __restrict__ tw, int idx1) {
#ifndef LAM_TW_TABLE
    if constexpr (R == 2 || R == 4 || R == 8 || R == 16) {
        C<T> w1 = tw[idx1];
        if (DIR > 0) w1.y = -w1.y;
        wv[1] = w1;
        if constexpr (R >= 4) {
            C<T> w2 = tw[2 * idx1];
            if (DIR > 0) w2.y = -w2.y;
            wv[2] = w2;
            wv[3] = cmul(w1, w2);
        }
        if constexpr (R >= 8) {
            C<T> w4 = tw[4 * idx1];
            if (DIR > 0) w4.y = -w4.y;
            wv[4] = w4;
            wv[5] = cmul(w1, w4);
            wv[6] = cmul(wv[2], w4);
            wv[7] = cmul(wv[3], w4);
        }
        if constexpr (R == 16) {
            C<T> w8 = tw[8 * idx1];
            if (DIR > 0) w8.y = -w8.y;
            wv[8] = w8;
#pragma unroll
            for (int r = 9; r < 16; ++r) wv[r] = cmul(wv[r - 8], w8);
        }
    } else
#endif
    {
#pragma unroll
        for (int r = 1; r < R; ++r) {
            C<T> w = tw[r * idx1];
            if (DIR > 0) w.y = -w.y;
            wv[r] = w;
        }
    }
}

// q / d for a block-uniform divisor: a shift when d is a power of two (P2 says
// it always is; otherwise it is tested), a division otherwise
template <bool P2> __device__ __forceinline__ int udiv(int q, int d, int ld) {
    if (P2 || (d & (d - 1)) == 0) return q >> ld;
    return q / d;
}
__device__ __forceinline__ int ilog2_pow2(int d) { return __ffs(d) - 1; }

template <int R, int DIR, int MAXB, typename T, bool P2>
__device__ __forceinline__ void fft_stage_ip(C<T>* buf, int nlines, int lstride, int N, int Ns,
                                             const C<T>* __restrict__ tw, int twstride, int tid, int nthr) {
    const int nb = N / R;
    const int lnb = ilog2_pow2(nb);
    const int total = nlines * nb;
    const int twstep = (N / (Ns * R)) * twstride;
    C<T> v[MAXB][R];
#pragma unroll
    for (int bb = 0; bb < MAXB; ++bb) {
        const int q = tid + bb * nthr;
        if (q < total) {
            const int line = q / nb;  // (a shift here raises the register count past the budget)
            const int j = q - line * nb;
            const C<T>* s = buf + line * lstride;
#pragma unroll
            for (int r = 0; r < R; ++r) v[bb][r] = s[fpad(j + r * nb)];
        }
    }
    __syncthreads();
#pragma unroll
    for (int bb = 0; bb < MAXB; ++bb) {
        const int q = tid + bb * nthr;
        if (q < total) {
            const int line = udiv<P2>(q, nb, lnb);
            const int j = q - line * nb;
            // Ns is a power of two in the radix-2/4/8 stages (they come first)
            const int k = (R == 3 || R == 5) ? j % Ns : (j & (Ns - 1));
            if (Ns > 1) {
                if constexpr (R == 16) {
                    // powers w^r built from w, w^2, w^4, w^8 and applied as they are made
                    const int i1 = k * twstep;
                    C<T> w1 = tw[i1], w2 = tw[2 * i1], w4 = tw[4 * i1], w8 = tw[8 * i1];
                    if (DIR > 0) {
                        w1.y = -w1.y;
                        w2.y = -w2.y;
                        w4.y = -w4.y;
                        w8.y = -w8.y;
                    }
                    C<T> w = w1;
#pragma unroll
                    for (int r = 1; r < 8; ++r) {
                        if (r == 2) w = w2;
                        else if (r == 4) w = w4;
                        else if (r > 1) w = cmul(w, w1);  // w^3 = w^2 w, w^5 = w^4 w, w^6, w^7
                        v[bb][r] = cmul(v[bb][r], w);
                        v[bb][r + 8] = cmul(v[bb][r + 8], cmul(w, w8));
                    }
                    v[bb][8] = cmul(v[bb][8], w8);
                } else {
                    C<T> wv[R];
                    twiddles<R, DIR, T>(wv, tw, k * twstep);
#pragma unroll
                    for (int r = 1; r < R; ++r) v[bb][r] = cmul(v[bb][r], wv[r]);
                }
            }
            if (R == 16) dft16<DIR>(v[bb]);
            else if (R == 8) dft8<DIR>(v[bb]);
            else if (R == 5) dft5<DIR>(v[bb]);
            else if (R == 4) dft4<DIR>(v[bb]);
            else if (R == 3) dft3<DIR>(v[bb]);
            else dft2<DIR>(v[bb]);
            C<T>* d = buf + line * lstride;
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) d[fpad(base + r * Ns)] = v[bb][R == 16 ? dft16_out(r) : r];
        }
    }
    __syncthreads();
}

// Butterflies per thread per radix-8 stage the in-place kernels are built for
// (register budget at 512 threads: 2 x 8 complex floats, 1 x 8 complex doubles).
template <typename T> struct FftMaxB;
template <> struct FftMaxB<float> { static constexpr int value = 2; };
template <> struct FftMaxB<double> { static constexpr int value = 1; };
constexpr int kFftThreads = 512;

// In-place FFT of nlines lines in buf, line l starting at buf + l * lstride,
// element e at fpad(e) (lstride >= fpad_len(N)).  The caller must
// __syncthreads() before; the call ends with a __syncthreads().  Requires
// nlines * N <= fft_capacity(code, MAXB) * blockDim.x; code = fft_code(N); tw
// has Nmax = N * twstride entries.  MIXED must be true when the code has
// radix-3 or radix-5 stages (fft_mixed).
template <int DIR, int MAXB, typename T, bool MIXED>
__device__ __forceinline__ void fft_lines_ip(C<T>* buf, int nlines, int lstride, int N, int code,
                                             const C<T>* __restrict__ tw, int twstride) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    int Ns = 1;
    for (int c = code; c; c >>= 3) {
        switch (c & 7) {
            case 6:
                if constexpr (fft_stage_maxb(16, MAXB) >= 1) {
                    fft_stage_ip<16, DIR, fft_stage_maxb(16, MAXB), T, !MIXED>(buf, nlines, lstride, N, Ns, tw,
                                                                              twstride, tid, nthr);
                    Ns *= 16;
                }
                break;
            case 3:
                fft_stage_ip<8, DIR, fft_stage_maxb(8, MAXB), T, !MIXED>(buf, nlines, lstride, N, Ns, tw, twstride, tid, nthr);
                Ns *= 8;
                break;
            case 2:
                fft_stage_ip<4, DIR, fft_stage_maxb(4, MAXB), T, !MIXED>(buf, nlines, lstride, N, Ns, tw, twstride, tid, nthr);
                Ns *= 4;
                break;
            case 1:
                fft_stage_ip<2, DIR, fft_stage_maxb(2, MAXB), T, !MIXED>(buf, nlines, lstride, N, Ns, tw, twstride, tid, nthr);
                Ns *= 2;
                break;
            default:
                if constexpr (MIXED) {
                    if ((c & 7) == 4) {
                        fft_stage_ip<3, DIR, fft_stage_maxb(3, MAXB), T, !MIXED>(buf, nlines, lstride, N, Ns, tw, twstride,
                                                                         tid, nthr);
                        Ns *= 3;
                    } else {
                        fft_stage_ip<5, DIR, fft_stage_maxb(5, MAXB), T, !MIXED>(buf, nlines, lstride, N, Ns, tw, twstride,
                                                                         tid, nthr);
                        Ns *= 5;
                    }
                }
                break;
        }
    }
}

// ---------------------------------------------------------------------------
// Compile-time length.  The same stages and arithmetic as fft_lines_ip (the
// same stage sequence, butterflies, twiddles and operation order, so the
// result is bitwise the same), with N, the stage radices, Ns and the line
// stride fpad_len(N) known to the compiler: divisions become shifts and the
// padded shared-memory offsets of a butterfly's R inputs and outputs become
// constants from one base address.  For power-of-two N only.
// ---------------------------------------------------------------------------

__host__ __device__ constexpr int fft_code_pow2(int N, int maxr) {
    int a = 0;
    for (int m = N; m > 1; m >>= 1) ++a;
    const int maxbits = maxr >= 16 ? 4 : 3;
    const int nst = (a + maxbits - 1) / maxbits;
    int code = 0, shift = 0;
    for (int k = 0; k < nst; ++k) {
        const int bits = (a + (nst - k) - 1) / (nst - k);
        code |= (bits == 4 ? 6 : bits == 3 ? 3 : bits == 2 ? 2 : 1) << shift;
        shift += 3;
        a -= bits;
    }
    return code;
}

// padded offset of element e + r * step relative to fpad(e), when step is a
// multiple of 16 (the pad count then grows by step / 16 per r)
template <int STEP> __device__ __forceinline__ constexpr int fpad_step(int r) { return r * (STEP + STEP / 16); }

template <int R, int DIR, int MAXB, typename T, int N, int NS>
__device__ __forceinline__ void fft_stage_ct(C<T>* buf, int nlines, const C<T>* __restrict__ tw, int twstride, int tid,
                                             int nthr) {
    constexpr int nb = N / R;
    constexpr int LS = N + N / 16 + 1;  // fpad_len(N)
    const int total = nlines * nb;
    const int twstep = (N / (NS * R)) * twstride;
    C<T> v[MAXB][R];
#pragma unroll
    for (int bb = 0; bb < MAXB; ++bb) {
        const int q = tid + bb * nthr;
        if (q < total) {
            const int line = q / nb, j = q % nb;
            const C<T>* s = buf + line * LS;
            if constexpr (nb % 16 == 0) {
                const C<T>* s0 = s + fpad(j);
#pragma unroll
                for (int r = 0; r < R; ++r) v[bb][r] = s0[fpad_step<nb>(r)];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) v[bb][r] = s[fpad(j + r * nb)];
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int bb = 0; bb < MAXB; ++bb) {
        const int q = tid + bb * nthr;
        if (q < total) {
            const int line = q / nb, j = q % nb;
            const int k = j & (NS - 1);
            if constexpr (NS > 1) {
                if constexpr (R == 16) {
                    const int i1 = k * twstep;
                    C<T> w1 = tw[i1], w2 = tw[2 * i1], w4 = tw[4 * i1], w8 = tw[8 * i1];
                    if (DIR > 0) {
                        w1.y = -w1.y;
                        w2.y = -w2.y;
                        w4.y = -w4.y;
                        w8.y = -w8.y;
                    }
                    C<T> w = w1;
#pragma unroll
                    for (int r = 1; r < 8; ++r) {
                        if (r == 2) w = w2;
                        else if (r == 4) w = w4;
                        else if (r > 1) w = cmul(w, w1);
                        v[bb][r] = cmul(v[bb][r], w);
                        v[bb][r + 8] = cmul(v[bb][r + 8], cmul(w, w8));
                    }
                    v[bb][8] = cmul(v[bb][8], w8);
                } else {
                    C<T> wv[R];
                    twiddles<R, DIR, T>(wv, tw, k * twstep);
#pragma unroll
                    for (int r = 1; r < R; ++r) v[bb][r] = cmul(v[bb][r], wv[r]);
                }
            }
            if constexpr (R == 16) dft16<DIR>(v[bb]);
            else if constexpr (R == 8) dft8<DIR>(v[bb]);
            else if constexpr (R == 4) dft4<DIR>(v[bb]);
            else dft2<DIR>(v[bb]);
            C<T>* d = buf + line * LS;
            const int base = (j - k) * R + k;
            if constexpr (NS % 16 == 0) {
                C<T>* d0 = d + fpad(base);
#pragma unroll
                for (int r = 0; r < R; ++r) d0[fpad_step<NS>(r)] = v[bb][R == 16 ? dft16_out(r) : r];
            } else if constexpr (NS == 1 && R == 16) {
                C<T>* d0 = d + 17 * j;  // fpad(16 j + r) = 17 j + r
#pragma unroll
                for (int r = 0; r < R; ++r) d0[r] = v[bb][dft16_out(r)];
            } else if constexpr (NS == 1 && R == 8) {
                C<T>* d0 = d + 8 * j + (j >> 1);  // fpad(8 j + r) = 8 j + j / 2 + r for r < 8
#pragma unroll
                for (int r = 0; r < R; ++r) d0[r] = v[bb][r];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) d[fpad(base + r * NS)] = v[bb][R == 16 ? dft16_out(r) : r];
            }
        }
    }
    __syncthreads();
}

template <int DIR, int MAXB, typename T, int N, int CODE, int NS>
__device__ __forceinline__ void fft_stages_ct(C<T>* buf, int nlines, const C<T>* __restrict__ tw, int twstride,
                                              int tid, int nthr) {
    if constexpr (CODE != 0) {
        constexpr int R = fft_stage_radix(CODE & 7);
        fft_stage_ct<R, DIR, fft_stage_maxb(R, MAXB), T, N, NS>(buf, nlines, tw, twstride, tid, nthr);
        fft_stages_ct<DIR, MAXB, T, N, (CODE >> 3), NS * R>(buf, nlines, tw, twstride, tid, nthr);
    }
}

// fft_lines_ip for a compile-time power-of-two length N (the stage code is
// fft_code(N, fft_max_radix<T>())), lines at stride fpad_len(N).
template <int DIR, int MAXB, typename T, int N>
__device__ __forceinline__ void fft_lines_ct(C<T>* buf, int nlines, const C<T>* __restrict__ tw, int twstride) {
    static_assert(N >= 16 && (N & (N - 1)) == 0, "power-of-two length");
    constexpr int code = fft_code_pow2(N, fft_max_radix<T>());
    fft_stages_ct<DIR, MAXB, T, N, code, 1>(buf, nlines, tw, twstride, threadIdx.x, blockDim.x);
}

// fft_lines_ct for NC > 0 (then N == NC and lstride == fpad_len(NC)), else
// the runtime-length fft_lines_ip
template <int DIR, typename T, bool MIXED, int NC>
__device__ __forceinline__ void fft_lines(C<T>* buf, int nlines, int lstride, int N, int code,
                                          const C<T>* __restrict__ tw, int twstride) {
    if constexpr (NC > 0) fft_lines_ct<DIR, FftMaxB<T>::value, T, NC>(buf, nlines, tw, twstride);
    else fft_lines_ip<DIR, FftMaxB<T>::value, T, MIXED>(buf, nlines, lstride, N, code, tw, twstride);
}

}  // namespace lam
