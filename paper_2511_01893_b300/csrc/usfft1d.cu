// usfft1d.cu - F_u1D and its transpose: the unequally-spaced FFT along z.
//
// F_u1D (Section 2) maps u[n1, n0, n2] to u1[n1, h, n2]: for every (x, y)
// column it evaluates sum_z u[x, z, y] exp(-2 pi i xi_z z) at the h
// frequencies xi_z = (kv / h) cos(phi).  Gaussian USFFT (Dutt-Rokhlin):
// deapodise, zero-pad to M0 = 2 nz, FFT, then 2m-tap Gaussian interpolation
// with per-kv taps and weights from the plan's FP64-built tables.
//
// One block owns TY adjacent y-columns of one x-slab: it reads u[x][:][y0:y0+TY]
// (TY contiguous values per z row), holds the TY padded lines in shared
// memory, transforms them and writes u1[kv][x][y0:y0+TY] for every kv.  u1 is
// stored plane-major ([h][n1][n2]) so the per-plane 2D stage reads contiguous
// planes.
//
// The transpose spreads the h values of each column onto the padded line in
// gather form: each padded cell sums, over the contiguous kv range whose taps
// reach it (a plan table), weight * value.  This keeps the spread atomic-free
// and deterministic and makes it the exact transpose of the gather.
#include "fft.cuh"
#include "kernels.h"

namespace lam {

template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_usfft1d_fwd(const T* __restrict__ u, C<T>* __restrict__ u1,
                                                     Usfft1dArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T>* bufa = reinterpret_cast<C<T>*>(smem_raw);
    const int tiles = a.n2 / a.TY;
    const int x = blockIdx.x / tiles;
    const int y0 = (blockIdx.x - x * tiles) * a.TY;
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int i = tid; i < a.TY * a.M0; i += nthr) bufa[i] = cmake<T>(0, 0);
    __syncthreads();
    const T* src = u + (size_t)x * a.nz * a.n2 + y0;
    for (int i = tid; i < a.nz * a.TY; i += nthr) {
        const int z = i / a.TY, c = i - z * a.TY;
        const T v = src[(size_t)z * a.n2 + c] * a.dz[z];
        bufa[c * a.M0 + wrap(z - a.nz / 2, a.M0)] = cmake<T>(v, 0);
    }
    __syncthreads();
    fft_lines_ip<-1, FftMaxB<T>::value, T>(bufa, a.TY, a.M0, a.M0, a.logM0, a.tw, a.twstride);
    const C<T>* P = bufa;
    const int nt = 2 * a.m;
    C<T>* dst = u1 + (size_t)x * a.n2 + y0;
    const size_t plane = (size_t)a.n1 * a.n2;
    for (int i = tid; i < a.h * a.TY; i += nthr) {
        const int kv = i / a.TY, c = i - kv * a.TY;
        const int jb = a.j0z[kv] - a.m + 1;
        const T* wz = a.wz + kv * nt;
        const C<T>* line = P + c * a.M0;
        T sr = 0, si = 0;
        for (int t = 0; t < nt; ++t) {
            const C<T> p = line[wrap(jb + t, a.M0)];
            sr += wz[t] * p.x;
            si += wz[t] * p.y;
        }
        dst[kv * plane + c] = cmake<T>(sr, si);
    }
}

template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_usfft1d_adj(const C<T>* __restrict__ u1, T* __restrict__ u,
                                                     Usfft1dArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T>* bufa = reinterpret_cast<C<T>*>(smem_raw);
    C<T>* vals = bufa + a.TY * a.M0;  // [TY][h]
    const int tiles = a.n2 / a.TY;
    const int x = blockIdx.x / tiles;
    const int y0 = (blockIdx.x - x * tiles) * a.TY;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const C<T>* src = u1 + (size_t)x * a.n2 + y0;
    const size_t plane = (size_t)a.n1 * a.n2;
    for (int i = tid; i < a.h * a.TY; i += nthr) {
        const int kv = i / a.TY, c = i - kv * a.TY;
        vals[c * a.h + kv] = src[kv * plane + c];
    }
    __syncthreads();
    const int nt = 2 * a.m;
    // spread in gather form: cell j collects every unwrapped cell e == j (mod M0)
    for (int i = tid; i < a.TY * a.M0; i += nthr) {
        const int c = i / a.M0, j = i - c * a.M0;
        T sr = 0, si = 0;
        // smallest e >= jmin with e == j (mod M0)
        int e = j + ((a.jmin - j + a.M0 - 1 + 64 * a.M0) / a.M0 - 64) * a.M0;
        for (; e <= a.jmax; e += a.M0) {
            const int lo = a.kvlo[e - a.jmin], hi = a.kvhi[e - a.jmin];
            for (int kv = lo; kv < hi; ++kv) {
                const T wt = a.wz[kv * nt + (e - (a.j0z[kv] - a.m + 1))];
                const C<T> v = vals[c * a.h + kv];
                sr += wt * v.x;
                si += wt * v.y;
            }
        }
        bufa[i] = cmake<T>(sr, si);
    }
    __syncthreads();
    fft_lines_ip<+1, FftMaxB<T>::value, T>(bufa, a.TY, a.M0, a.M0, a.logM0, a.tw, a.twstride);
    const C<T>* q = bufa;
    T* dst = u + (size_t)x * a.nz * a.n2 + y0;
    for (int i = tid; i < a.nz * a.TY; i += nthr) {
        const int z = i / a.TY, c = i - z * a.TY;
        dst[(size_t)z * a.n2 + c] = q[c * a.M0 + wrap(z - a.nz / 2, a.M0)].x * a.dz[z];
    }
}

template <typename T>
cudaError_t launch_usfft1d_fwd(const T* u, C<T>* u1, const Usfft1dArgs<T>& a, cudaStream_t s) {
    const size_t smem = (size_t)a.TY * a.M0 * sizeof(C<T>);
    k_usfft1d_fwd<T><<<a.n1 * (a.n2 / a.TY), kFftThreads, smem, s>>>(u, u1, a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_usfft1d_adj(const C<T>* u1, T* u, const Usfft1dArgs<T>& a, cudaStream_t s) {
    const size_t smem = (size_t)(a.M0 + a.h) * a.TY * sizeof(C<T>);
    k_usfft1d_adj<T><<<a.n1 * (a.n2 / a.TY), kFftThreads, smem, s>>>(u1, u, a);
    return cudaGetLastError();
}

template <typename T> cudaError_t configure_usfft1d() {
    const int mx = kMaxDynSmem;
    cudaError_t e = cudaFuncSetAttribute(k_usfft1d_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (!e) e = cudaFuncSetAttribute(k_usfft1d_adj<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    return e;
}

template cudaError_t launch_usfft1d_fwd<float>(const float*, C<float>*, const Usfft1dArgs<float>&, cudaStream_t);
template cudaError_t launch_usfft1d_fwd<double>(const double*, C<double>*, const Usfft1dArgs<double>&, cudaStream_t);
template cudaError_t launch_usfft1d_adj<float>(const C<float>*, float*, const Usfft1dArgs<float>&, cudaStream_t);
template cudaError_t launch_usfft1d_adj<double>(const C<double>*, double*, const Usfft1dArgs<double>&, cudaStream_t);
template cudaError_t configure_usfft1d<float>();
template cudaError_t configure_usfft1d<double>();

}  // namespace lam
