// fft2d.cu - F_2D and F*_2D: centred 2D DFT of every angle's h x w grid.
//
// F*_2D (Section 2, the last step of L) is the per-angle inverse 2D FFT on the
// equispaced detector-frequency grid; F_2D (Algorithm 2, d_hat = F_2D d) is its
// inverse.  With centred indices (ku - w/2, iu - w/2, ...) the centred DFT of
// even-length axes equals a plain DFT with the input and output multiplied by
// (-1)^index and the whole result by (-1)^(h/2 + w/2):
//   exp(s 2 pi i (k - n/2)(i - n/2) / n) = (-1)^(k + i + n/2) exp(s 2 pi i k i / n).
// Row pass: load * (-1)^(kv + ku), FFT along w, store * (-1)^iu.
// Column pass (in place): FFT along h, store * (-1)^(iv + h/2 + w/2) * scale.
#include "fft.cuh"
#include "kernels.h"

namespace lam {

template <int DIR, typename T, bool MIXED>
__global__ void __launch_bounds__(kFftThreads) k_fft2d_rows(const C<T>* in, C<T>* out,
                                                    int RB, Fft2dArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T>* bufa = reinterpret_cast<C<T>*>(smem_raw);
    const int th = blockIdx.y, r0 = blockIdx.x * RB;
    const size_t base = ((size_t)th * a.h + r0) * a.w;
    const int LS = fpad_len(a.w);
    for (int i = threadIdx.x; i < RB * a.w; i += blockDim.x) {
        const int r = udiv<!MIXED>(i, a.w, ilog2_pow2(a.w)), k = i - r * a.w;
        const C<T> v = in[base + i];
        bufa[r * LS + fpad(k)] = ((r0 + r + k) & 1) ? cmake<T>(-v.x, -v.y) : v;
    }
    __syncthreads();
    fft_lines_ip<DIR, FftMaxB<T>::value, T, MIXED>(bufa, RB, LS, a.w, a.fcw, a.tw, a.tww);
    for (int i = threadIdx.x; i < RB * a.w; i += blockDim.x) {
        const int r = udiv<!MIXED>(i, a.w, ilog2_pow2(a.w)), k = i - r * a.w;
        const C<T> v = bufa[r * LS + fpad(k)];
        out[base + i] = (k & 1) ? cmake<T>(-v.x, -v.y) : v;
    }
}

template <int DIR, typename T, bool MIXED>
__global__ void __launch_bounds__(kFftThreads) k_fft2d_cols(C<T>* __restrict__ io, int CB, T scale, Fft2dArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T>* bufa = reinterpret_cast<C<T>*>(smem_raw);
    const int th = blockIdx.y, c0 = blockIdx.x * CB;
    C<T>* pl = io + (size_t)th * a.h * a.w + c0;
    const int LS = fpad_len(a.h);
    for (int i = threadIdx.x; i < a.h * CB; i += blockDim.x) {
        const int r = i >> ilog2_pow2(CB), c = i - r * CB;  // CB is a power of two
        bufa[c * LS + fpad(r)] = pl[(size_t)r * a.w + c];
    }
    __syncthreads();
    fft_lines_ip<DIR, FftMaxB<T>::value, T, MIXED>(bufa, CB, LS, a.h, a.fch, a.tw, a.twh);
    const int gsign = ((a.h / 2 + a.w / 2) & 1);
    for (int i = threadIdx.x; i < a.h * CB; i += blockDim.x) {
        const int r = i >> ilog2_pow2(CB), c = i - r * CB;  // CB is a power of two
        const C<T> v = bufa[c * LS + fpad(r)];
        const T s = ((r + gsign) & 1) ? -scale : scale;
        pl[(size_t)r * a.w + c] = cscale(v, s);
    }
}

// lines per block: at most 128 KB of shared memory, within the in-place FFT's
// register capacity (lines * len <= capacity * threads), at most 32 lines,
// dividing the number of lines
template <typename T> static int lines_per_block(int len, int code, int nlines) {
    const size_t elem = sizeof(C<T>);
    const int capacity = fft_capacity(code, FftMaxB<T>::value) * kFftThreads;
    int l = 32;
    while (l > 1 && ((size_t)l * fpad_len(len) * elem > 128 * 1024 || l * len > capacity || nlines % l != 0))
        l >>= 1;
    return l;
}

template <typename T>
cudaError_t launch_fft2d_angles(const C<T>* in, C<T>* out, int dir, T scale, const Fft2dArgs<T>& a,
                                cudaStream_t s) {
    const int RB = lines_per_block<T>(a.w, a.fcw, a.h);
    const int CB = lines_per_block<T>(a.h, a.fch, a.w);
    const size_t sr = (size_t)RB * fpad_len(a.w) * sizeof(C<T>);
    const size_t sc = (size_t)CB * fpad_len(a.h) * sizeof(C<T>);
    const bool mixed = fft_mixed(a.fch) || fft_mixed(a.fcw);
#define LAM_F2(D, MX)                                                                              \
    k_fft2d_rows<D, T, MX><<<dim3(a.h / RB, a.T_), kFftThreads, sr, s>>>(in, out, RB, a);          \
    k_fft2d_cols<D, T, MX><<<dim3(a.w / CB, a.T_), kFftThreads, sc, s>>>(out, CB, scale, a);
    if (dir > 0) {
        if (mixed) { LAM_F2(1, true) } else { LAM_F2(1, false) }
    } else {
        if (mixed) { LAM_F2(-1, true) } else { LAM_F2(-1, false) }
    }
#undef LAM_F2
    return cudaGetLastError();
}

// FBP ramp: io[th][kv][iu] *= c0 * |iu - w/2| (c0 / 4 at iu = w/2), in place
// on the centred spectrum F_2D d; n_rows = T h rows of w values
template <typename T>
__global__ void __launch_bounds__(256) k_ramp(C<T>* __restrict__ io, long long n_rows, int w, T c0) {
    const long long n = n_rows * w;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int iu = (int)(i % w);
        const int k = iu - w / 2;
        const T r = k == 0 ? (T)0.25 : (T)(k < 0 ? -k : k);
        io[i] = cscale(io[i], c0 * r);
    }
}

template <typename T> cudaError_t launch_ramp(C<T>* io, long long n_rows, int w, T c0, cudaStream_t s) {
    const long long n = n_rows * w;
    const long long b = (n + 255) / 256;
    k_ramp<T><<<(int)(b < 148 * 8 ? b : 148 * 8), 256, 0, s>>>(io, n_rows, w, c0);
    return cudaGetLastError();
}
template cudaError_t launch_ramp<float>(C<float>*, long long, int, float, cudaStream_t);
template cudaError_t launch_ramp<double>(C<double>*, long long, int, double, cudaStream_t);

template <typename T> cudaError_t configure_fft2d() {
    const int mx = kMaxDynSmem;
    cudaError_t e = cudaSuccess;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (!e) e = cudaFuncSetAttribute(k_fft2d_rows<1, T, false>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_fft2d_rows<-1, T, false>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_fft2d_cols<1, T, false>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_fft2d_cols<-1, T, false>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_fft2d_rows<1, T, true>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_fft2d_rows<-1, T, true>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_fft2d_cols<1, T, true>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_fft2d_cols<-1, T, true>, at, mx);
    return e;
}

template cudaError_t launch_fft2d_angles<float>(const C<float>*, C<float>*, int, float, const Fft2dArgs<float>&,
                                                cudaStream_t);
template cudaError_t launch_fft2d_angles<double>(const C<double>*, C<double>*, int, double,
                                                 const Fft2dArgs<double>&, cudaStream_t);
template cudaError_t configure_fft2d<float>();
template cudaError_t configure_fft2d<double>();

}  // namespace lam
