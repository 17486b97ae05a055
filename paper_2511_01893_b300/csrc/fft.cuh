// fft.cuh - batched power-of-two FFTs in shared memory (Stockham autosort).
//
// Each call transforms `nlines` lines of length N stored at stride `lstride`
// in shared memory.  Stages are radix 8 (then one radix 4 or 2 stage); every
// thread of the block takes butterflies q = tid, tid + nthr, ... of a stage,
// reads R inputs N/R apart, applies twiddles, does an in-register radix-R
// DFT and writes the R outputs Ns apart (self-sorting, so the result is in
// natural order).
//
// Sign convention: DIR = -1 computes sum_x a[x] exp(-2 pi i j x / N),
// DIR = +1 computes sum_x a[x] exp(+2 pi i j x / N) (no normalisation).
// Twiddles come from a table tw[q] = exp(-2 pi i q / Nmax), q < Nmax, where
// Nmax is a power-of-two multiple of N (twstride = Nmax / N).
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

template <int R, int DIR, typename T>
__device__ __forceinline__ void twiddles(C<T>* wv, const C<T>* __restrict__ tw, int idx1, int tmask) {
#ifdef LAM_TW_TABLE
#pragma unroll
    for (int r = 1; r < R; ++r) {
        C<T> w = tw[(r * idx1) & tmask];
        if (DIR > 0) w.y = -w.y;
        wv[r] = w;
    }
    return;
#endif
    // idx1 = k * twstep; table index r * idx1 reduced mod table length (tmask = len - 1)
    C<T> w1 = tw[idx1 & tmask];
    if (DIR > 0) w1.y = -w1.y;
    wv[1] = w1;
    if (R >= 4) {
        C<T> w2 = tw[(2 * idx1) & tmask];
        if (DIR > 0) w2.y = -w2.y;
        wv[2] = w2;
        wv[3] = cmul(w1, w2);
    }
    if (R == 8) {
        C<T> w4 = tw[(4 * idx1) & tmask];
        if (DIR > 0) w4.y = -w4.y;
        wv[4] = w4;
        wv[5] = cmul(w1, w4);
        wv[6] = cmul(wv[2], w4);
        wv[7] = cmul(wv[3], w4);
    }
}

template <int R, int DIR, int MAXB, typename T>
__device__ __forceinline__ void fft_stage_ip(C<T>* buf, int nlines, int lstride, int N, int Ns,
                                             const C<T>* __restrict__ tw, int twstride, int tmask, int tid,
                                             int nthr) {
    const int nb = N / R;
    const int total = nlines * nb;
    const int twstep = (N / (Ns * R)) * twstride;
    C<T> v[MAXB][R];
#pragma unroll
    for (int bb = 0; bb < MAXB; ++bb) {
        const int q = tid + bb * nthr;
        if (q < total) {
            const int line = q / nb;
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
            const int line = q / nb;
            const int j = q - line * nb;
            const int k = j & (Ns - 1);
            if (Ns > 1) {
                C<T> wv[R];
                twiddles<R, DIR, T>(wv, tw, k * twstep, tmask);
#pragma unroll
                for (int r = 1; r < R; ++r) v[bb][r] = cmul(v[bb][r], wv[r]);
            }
            if (R == 8) dft8<DIR>(v[bb]);
            else if (R == 4) dft4<DIR>(v[bb]);
            else dft2<DIR>(v[bb]);
            C<T>* d = buf + line * lstride;
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) d[fpad(base + r * Ns)] = v[bb][r];
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
// element e at fpad(e) (lstride >= fpad_len(N)).  The caller must __syncthreads() before; the call ends with a
// __syncthreads().  Requires nlines * N <= 8 * MAXB * blockDim.x.  tlen is the
// twiddle table length (a power of two).
template <int DIR, int MAXB, typename T>
__device__ __forceinline__ void fft_lines_ip(C<T>* buf, int nlines, int lstride, int N, int logN,
                                             const C<T>* __restrict__ tw, int twstride) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int tmask = N * twstride - 1;
    int Ns = 1;
    int bits = logN;
    while (bits > 0) {
        if (bits >= 3 && bits != 4) {
            fft_stage_ip<8, DIR, MAXB, T>(buf, nlines, lstride, N, Ns, tw, twstride, tmask, tid, nthr);
            Ns *= 8;
            bits -= 3;
        } else if (bits >= 2) {
            fft_stage_ip<4, DIR, 2 * MAXB, T>(buf, nlines, lstride, N, Ns, tw, twstride, tmask, tid, nthr);
            Ns *= 4;
            bits -= 2;
        } else {
            fft_stage_ip<2, DIR, 4 * MAXB, T>(buf, nlines, lstride, N, Ns, tw, twstride, tmask, tid, nthr);
            Ns *= 2;
            bits -= 1;
        }
    }
}

}  // namespace lam
