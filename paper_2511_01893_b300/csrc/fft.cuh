// fft.cuh - batched power-of-two FFTs in shared memory (Stockham autosort).
//
// Each call transforms `nlines` lines of length N stored at stride `lstride`
// in shared memory.  Stages are radix 8 (then one radix 4 or 2 stage); every
// thread of the block takes butterflies q = tid, tid + nthr, ... of a stage,
// reads R inputs N/R apart, applies twiddles, does an in-register radix-R
// DFT and writes the R outputs Ns apart (self-sorting, so the result is in
// natural order).  Stages ping-pong between two buffers.
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

template <int R, int DIR, typename T>
__device__ __forceinline__ void fft_stage(const C<T>* __restrict__ src, C<T>* __restrict__ dst,
                                          int nlines, int lstride, int N, int Ns,
                                          const C<T>* __restrict__ tw, int twstride, int tid,
                                          int nthr) {
    const int nb = N / R;  // butterflies per line
    const int total = nlines * nb;
    const int twstep = (N / (Ns * R)) * twstride;  // table step per unit of r*k
    for (int q = tid; q < total; q += nthr) {
        const int line = q / nb;
        const int j = q - line * nb;
        const C<T>* s = src + line * lstride;
        C<T>* d = dst + line * lstride;
        C<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[j + r * nb];
        const int k = j & (Ns - 1);
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C<T> wv = tw[r * k * twstep];
                if (DIR > 0) wv.y = -wv.y;
                v[r] = cmul(v[r], wv);
            }
        }
        if (R == 8) dft8<DIR>(v);
        else if (R == 4) dft4<DIR>(v);
        else dft2<DIR>(v);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) d[base + r * Ns] = v[r];
    }
}

// Transforms the lines in `a`; returns the buffer (a or b) holding the result.
// Callers must __syncthreads() before the call (input complete); the call
// ends with a __syncthreads().
template <int DIR, typename T>
__device__ C<T>* fft_lines(C<T>* a, C<T>* b, int nlines, int lstride, int N, int logN,
                           const C<T>* __restrict__ tw, int twstride) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    C<T>* src = a;
    C<T>* dst = b;
    int Ns = 1;
    int bits = logN;
    while (bits > 0) {
        if (bits >= 3 && bits != 4) {
            fft_stage<8, DIR, T>(src, dst, nlines, lstride, N, Ns, tw, twstride, tid, nthr);
            Ns *= 8;
            bits -= 3;
        } else if (bits >= 2) {
            fft_stage<4, DIR, T>(src, dst, nlines, lstride, N, Ns, tw, twstride, tid, nthr);
            Ns *= 4;
            bits -= 2;
        } else {
            fft_stage<2, DIR, T>(src, dst, nlines, lstride, N, Ns, tw, twstride, tid, nthr);
            Ns *= 2;
            bits -= 1;
        }
        __syncthreads();
        C<T>* t = src;
        src = dst;
        dst = t;
    }
    return src;
}

// ---------------------------------------------------------------------------
// In-place variant: one shared buffer.  Each stage first loads every
// butterfly input the thread owns into registers (at most MAXB butterflies of
// radix <= 8 per thread: nlines * N <= 8 * MAXB * blockDim.x), synchronises,
// then writes the outputs.  Half the shared memory of the ping-pong form, so
// blocks can hold twice the lines.
// ---------------------------------------------------------------------------

template <int R, int DIR, int MAXB, typename T>
__device__ __forceinline__ void fft_stage_ip(C<T>* buf, int nlines, int lstride, int N, int Ns,
                                             const C<T>* __restrict__ tw, int twstride, int tid, int nthr) {
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
            for (int r = 0; r < R; ++r) v[bb][r] = s[j + r * nb];
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
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    C<T> wv = tw[r * k * twstep];
                    if (DIR > 0) wv.y = -wv.y;
                    v[bb][r] = cmul(v[bb][r], wv);
                }
            }
            if (R == 8) dft8<DIR>(v[bb]);
            else if (R == 4) dft4<DIR>(v[bb]);
            else dft2<DIR>(v[bb]);
            C<T>* d = buf + line * lstride;
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) d[base + r * Ns] = v[bb][r];
        }
    }
    __syncthreads();
}

// In-place FFT of nlines lines in buf (same conventions as fft_lines).  The
// caller must __syncthreads() before; the call ends with a __syncthreads().
// Requires nlines * N <= 8 * MAXB * blockDim.x (radix-8 stages); radix-4 and
// radix-2 stages need at most 2x / 4x that many butterflies, which the
// register arrays hold as well because they are sized for radix 8.
// Butterflies per thread per radix-8 stage the in-place kernels are built for
// (register budget at 512 threads: 2 x 8 complex floats, 1 x 8 complex doubles).
template <typename T> struct FftMaxB;
template <> struct FftMaxB<float> { static constexpr int value = 2; };
template <> struct FftMaxB<double> { static constexpr int value = 1; };
constexpr int kFftThreads = 512;

template <int DIR, int MAXB, typename T>
__device__ __forceinline__ void fft_lines_ip(C<T>* buf, int nlines, int lstride, int N, int logN, const C<T>* __restrict__ tw,
                             int twstride) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    int Ns = 1;
    int bits = logN;
    while (bits > 0) {
        if (bits >= 3 && bits != 4) {
            fft_stage_ip<8, DIR, MAXB, T>(buf, nlines, lstride, N, Ns, tw, twstride, tid, nthr);
            Ns *= 8;
            bits -= 3;
        } else if (bits >= 2) {
            fft_stage_ip<4, DIR, 2 * MAXB, T>(buf, nlines, lstride, N, Ns, tw, twstride, tid, nthr);
            Ns *= 4;
            bits -= 2;
        } else {
            fft_stage_ip<2, DIR, 4 * MAXB, T>(buf, nlines, lstride, N, Ns, tw, twstride, tid, nthr);
            Ns *= 2;
            bits -= 1;
        }
    }
}

}  // namespace lam
