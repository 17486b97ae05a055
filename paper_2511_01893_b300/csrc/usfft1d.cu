// usfft1d.cu - F_u1D and its transpose: the unequally-spaced FFT along z.
//
// F_u1D (Section 2) maps u[n1, n0, n2] to u1[n1, h, n2]: for every (x, y)
// column it evaluates sum_z u[x, z, y] exp(-2 pi i xi_z z) at the h
// frequencies xi_z = (kv / h) cos(phi).  Gaussian USFFT (Dutt-Rokhlin):
// deapodise, zero-pad to M0 = 2 nz, FFT, then 2m-tap Gaussian interpolation
// with per-kv taps and weights from the plan's FP64-built tables.
//
// One block owns TY adjacent y-columns of one x-slab: it reads u[x][:][y0:y0+TY]
// (TY contiguous values per z row), transforms them in shared memory and
// writes u1[kv][x][y0:y0+TY] for every kv the operator needs (in the paired
// operators of a real volume the conjugate-mirror planes are skipped).  u1 is
// stored plane-major ([h][n1][n2]) so the per-plane 2D stage reads contiguous
// planes.
//
// The transpose spreads the h values of each column onto the padded line in
// gather form: each padded cell sums, over the contiguous kv range whose taps
// reach it (plan tables; without the mirror planes when paired), weight *
// value.  This keeps the spread atomic-free and deterministic and makes it the
// exact transpose of the gather.
#include "fft.cuh"
#include "kernels.h"

namespace lam {

// Two real columns a, b travel as one complex line z = a + i b.  The padded
// transform of length M0 = 2 nz splits into even and odd outputs:
//   P[2k]   = sum_x f[x] e^{-2 pi i k x / nz}                 (E = DFT_nz f)
//   P[2k+1] = sum_x f[x] w^x e^{-2 pi i k x / nz}, w = e^{-2 pi i / M0}   (O)
// with f placed at x mod nz, and the two real spectra separate as
//   P_a[j] = (P_z[j] + conj P_z[-j]) / 2,  P_b[j] = (P_z[j] - conj P_z[-j]) / (2i).
// So TY columns need TY FFTs of length nz instead of TY of length 2 nz.

template <typename T> __device__ __forceinline__ C<T> pz_at(const C<T>* E, const C<T>* O, int j, int M0) {
    const int jj = wrap(j, M0);
    return (jj & 1) ? O[fpad(jj >> 1)] : E[fpad(jj >> 1)];
}

template <typename T, bool MIXED, int NC = 0>
__device__ __forceinline__ void k_usfft1d_fwd_body(const T* __restrict__ u, C<T>* __restrict__ u1, const Usfft1dArgs<T>& a, int bx) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);  // lines 2p (E) and 2p+1 (O), length nz
    const int nz = NC ? NC : a.nz, npair = a.TY / 2, M0 = 2 * nz;  // NC: compile-time nz
    const int LS = fpad_len(nz);
    const int tiles = a.n2 / a.TY;
    const int x = bx / tiles;
    const int y0 = (bx - x * tiles) * a.TY;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int twM0 = a.twstride;  // Nmax / M0
    const T* src = u + (size_t)x * nz * a.n2 + y0;
    // the column pair (2p, 2p + 1) is one aligned complex element (n2, y0 even);
    // it is copied raw into the even line, then scaled and twiddled in place by
    // the thread that copied it
    for (int i = tid; i < nz * npair; i += nthr) {
        const int z = i >> ilog2_pow2(npair), p = i - z * npair;  // npair = TY / 2, a power of two
        const int q = wrap(z - nz / 2, nz);
        cp_async_elem<T>(buf + (2 * p) * LS + fpad(q), reinterpret_cast<const C<T>*>(src + (size_t)z * a.n2 + 2 * p));
    }
    cp_async_commit();
    cp_async_wait_all();
    for (int i = tid; i < nz * npair; i += nthr) {
        const int z = i >> ilog2_pow2(npair), p = i - z * npair;
        const int xc = z - nz / 2;
        const int q = wrap(xc, nz);
        const T d = a.dz[z];
        const C<T> raw = buf[(2 * p) * LS + fpad(q)];
        const T va = raw.x * d, vb = raw.y * d;
        const C<T> w = a.tw[wrap(xc, M0) * twM0];  // e^{-2 pi i xc / M0}
        buf[(2 * p) * LS + fpad(q)] = cmake<T>(va, vb);
        buf[(2 * p + 1) * LS + fpad(q)] = cmul(cmake<T>(va, vb), w);
    }
    __syncthreads();
    fft_lines<-1, T, MIXED, NC>(buf, a.TY, LS, nz, a.fcz, a.tw, 2 * twM0);
    const int nt = 2 * a.m;
    C<T>* dst = u1 + (size_t)x * a.n2 + y0;
    const size_t plane = (size_t)a.n1 * a.n2;
    for (int i = tid; i < a.h * npair; i += nthr) {
        const int kv = i >> ilog2_pow2(npair), p = i - kv * npair;
        if (a.skip && a.skip[kv]) continue;  // a conjugate-mirror plane: not stored, not computed
        const C<T>* E = buf + (2 * p) * LS;
        const C<T>* O = E + LS;
        const int jb = a.j0z[kv] - a.m + 1;
        const T* wz = a.wz + kv * nt;
        T sar = 0, sai = 0, sbr = 0, sbi = 0;
        for (int t = 0; t < nt; ++t) {
            const C<T> pp = pz_at(E, O, jb + t, M0);
            const C<T> pm = pz_at(E, O, -(jb + t), M0);
            const T wt = wz[t];
            sar = fma(wt, pp.x + pm.x, sar);
            sai = fma(wt, pp.y - pm.y, sai);
            sbr = fma(wt, pp.x - pm.x, sbr);
            sbi = fma(wt, pp.y + pm.y, sbi);
        }
        // a = (sa) / 2, b = (sb) / (2i) = (sb.im, -sb.re) / 2
        C<T>* o = dst + kv * plane + 2 * p;
        o[0] = cmake<T>((T)0.5 * sar, (T)0.5 * sai);
        o[1] = cmake<T>((T)0.5 * sbi, (T)-0.5 * sbr);
    }
}

template <typename T, bool MIXED, int NC = 0>
__global__ void __launch_bounds__(kFftThreads) k_usfft1d_fwd(const T* __restrict__ u, C<T>* __restrict__ u1,
                                                             Usfft1dArgs<T> a) {
    k_usfft1d_fwd_body<T, MIXED, NC>(u, u1, a, (int)blockIdx.x);
}

// Transpose.  For real outputs only the Hermitian part of each spread column
// matters, Re IDFT(Q) = IDFT((Q[j] + conj Q[-j]) / 2), so two columns pack as
//   Q_c[j] = (Q_a[j] + conj Q_a[-j]) / 2 + i (Q_b[j] + conj Q_b[-j]) / 2,
// whose inverse transform is Re f_a + i Re f_b.  One thread builds Q_c at the
// mirror pair j, M0 - j from the gather-form spreads of both columns at j and
// at -j (one pass over each cell's kv range and weights serves both
// columns), then the even / odd halves go through two inverse FFTs of length
// nz and recombine as
//   f[x] = E'[x mod nz] + e^{+2 pi i x / M0} O'[x mod nz].
template <typename T>
__device__ __forceinline__ void spread_pair_at(const C<T>* va, const C<T>* vb, int j, int M0, const Usfft1dArgs<T>& a,
                                               C<T>& sa, C<T>& sb) {
    // columns a and b of a pair share each cell's kv range and weights
    T ar = 0, ai = 0, br = 0, bi = 0;
    int e = j + ((a.jmin - j + M0 - 1 + 64 * M0) / M0 - 64) * M0;  // smallest e >= jmin, e == j
    for (; e <= a.jmax; e += M0) {
        const int c = e - a.jmin;
        const int lo = a.kvslo[c], hi = a.kvshi[c];
        // a non-empty kv range must lie in the cell's row of cw weights
        if (hi > lo && !(LAM_INB(lo - a.kvlo[c], a.cw, a.err, kSiteZWeights) &&
                         LAM_INB(hi - 1 - a.kvlo[c], a.cw, a.err, kSiteZWeights) &&
                         LAM_INB(hi - 1, a.h, a.err, kSiteZWeights)))
            continue;
        const T* wt = a.wzc + (size_t)c * a.cw - a.kvlo[c];  // indexed by kv
        for (int kv = lo; kv < hi; ++kv) {
            const T wk = wt[kv];
            const C<T> x = va[kv], y = vb[kv];
            ar = fma(wk, x.x, ar);
            ai = fma(wk, x.y, ai);
            br = fma(wk, y.x, br);
            bi = fma(wk, y.y, bi);
        }
    }
    sa = cmake<T>(ar, ai);
    sb = cmake<T>(br, bi);
}

template <typename T, bool MIXED, int NC = 0>
__device__ __forceinline__ void k_usfft1d_adj_body(const C<T>* __restrict__ u1, T* __restrict__ u, const Usfft1dArgs<T>& a, int bx) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nz = NC ? NC : a.nz, npair = a.TY / 2, M0 = 2 * nz;  // NC: compile-time nz
    const int LS = fpad_len(nz);
    C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);  // TY lines of length nz (E, O per pair)
    C<T>* vals = buf + a.TY * LS;                  // [TY][h]
    const int tiles = a.n2 / a.TY;
    const int x = bx / tiles;
    const int y0 = (bx - x * tiles) * a.TY;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const C<T>* src = u1 + (size_t)x * a.n2 + y0;
    const size_t plane = (size_t)a.n1 * a.n2;
    for (int i = tid; i < a.h * a.TY; i += nthr) {
        const int kv = i >> ilog2_pow2(a.TY), c = i - kv * a.TY;  // TY is a power of two
        if (a.skip && a.skip[kv]) vals[c * a.h + kv] = cmake<T>(0, 0);
        else cp_async_elem<T>(vals + c * a.h + kv, src + kv * plane + c);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    const int half = M0 / 2;
    // i / (half + 1) through FP32: i < 2^24 and (i + 1/2) / (half + 1) stays at
    // least 1 / (2 half + 2) away from an integer, far above the rounding error
    const float rcp = 1.0f / (float)(half + 1);
    for (int i = tid; i < npair * (half + 1); i += nthr) {
        const int p = (int)(((float)i + 0.5f) * rcp), j = i - p * (half + 1);
        const int jm = wrap(-j, M0);
        const C<T>* va = vals + (2 * p) * a.h;
        const C<T>* vb = va + a.h;
        C<T> ap, am, bp, bm;
        spread_pair_at(va, vb, j, M0, a, ap, bp);
        spread_pair_at(va, vb, jm, M0, a, am, bm);
        // Q_c[j] = (ap + conj am)/2 + i (bp + conj bm)/2
        const C<T> qj = cmake<T>((T)0.5 * ((ap.x + am.x) - (bp.y - bm.y)), (T)0.5 * ((ap.y - am.y) + (bp.x + bm.x)));
        // Q_c[-j] = (am + conj ap)/2 + i (bm + conj bp)/2
        const C<T> qm = cmake<T>((T)0.5 * ((am.x + ap.x) - (bm.y - bp.y)), (T)0.5 * ((am.y - ap.y) + (bm.x + bp.x)));
        C<T>* E = buf + (2 * p) * LS;
        C<T>* O = E + LS;
        ((j & 1) ? O : E)[fpad(j >> 1)] = qj;
        if (jm != j) ((jm & 1) ? O : E)[fpad(jm >> 1)] = qm;
    }
    __syncthreads();
    fft_lines<+1, T, MIXED, NC>(buf, a.TY, LS, nz, a.fcz, a.tw, 2 * a.twstride);
    T* dst = u + (size_t)x * nz * a.n2 + y0;
    for (int i = tid; i < nz * npair; i += nthr) {
        const int z = i >> ilog2_pow2(npair), p = i - z * npair;  // npair = TY / 2, a power of two
        const int xc = z - nz / 2;
        const int q = wrap(xc, nz);
        const C<T> e = buf[(2 * p) * LS + fpad(q)], o = buf[(2 * p + 1) * LS + fpad(q)];
        C<T> w = a.tw[wrap(xc, M0) * a.twstride];  // e^{-2 pi i xc / M0}; use its conjugate
        const C<T> ow = cmulc(o, w);  // o e^{+2 pi i xc / M0}
        const T fr = e.x + ow.x;
        const T fi = e.y + ow.y;
        const T d = a.dz[z];
        dst[(size_t)z * a.n2 + 2 * p] = fr * d;
        dst[(size_t)z * a.n2 + 2 * p + 1] = fi * d;
    }
}

template <typename T, bool MIXED, int NC = 0>
__global__ void __launch_bounds__(kFftThreads) k_usfft1d_adj(const C<T>* __restrict__ u1, T* __restrict__ u,
                                                             Usfft1dArgs<T> a) {
    k_usfft1d_adj_body<T, MIXED, NC>(u1, u, a, (int)blockIdx.x);
}

// The FP32 z-stage kernels are also built for the power-of-two nz of the
// large workloads, with nz a compile-time constant (bitwise the same
// results); other lengths and FP64 take the runtime-length kernels.
#define LAM_Z_NC(len, CALL)                  \
    do {                                     \
        if constexpr (sizeof(T) == 4) {      \
            switch (len) {                   \
                case 256: CALL(256); break;   \
                case 512: CALL(512); break;   \
                case 1024: CALL(1024); break; \
                case 2048: CALL(2048); break; \
                default: CALL(0); break;      \
            }                                \
        } else {                             \
            CALL(0);                         \
        }                                    \
    } while (0)

template <typename T>
cudaError_t launch_usfft1d_fwd(const T* u, C<T>* u1, const Usfft1dArgs<T>& a, cudaStream_t s) {
    const size_t smem = (size_t)a.TY * fpad_len(a.nz) * sizeof(C<T>);
#define LAM_ZF(NC) k_usfft1d_fwd<T, false, NC><<<a.n1 * (a.n2 / a.TY), a.nthr, smem, s>>>(u, u1, a)
    if (fft_mixed(a.fcz)) k_usfft1d_fwd<T, true><<<a.n1 * (a.n2 / a.TY), a.nthr, smem, s>>>(u, u1, a);
    else LAM_Z_NC(a.nz, LAM_ZF);
#undef LAM_ZF
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_usfft1d_adj(const C<T>* u1, T* u, const Usfft1dArgs<T>& a, cudaStream_t s) {
    const size_t smem = (size_t)(fpad_len(a.nz) + a.h) * a.TY * sizeof(C<T>);
#define LAM_ZA(NC) k_usfft1d_adj<T, false, NC><<<a.n1 * (a.n2 / a.TY), a.nthr, smem, s>>>(u1, u, a)
    if (fft_mixed(a.fcz)) k_usfft1d_adj<T, true><<<a.n1 * (a.n2 / a.TY), a.nthr, smem, s>>>(u1, u, a);
    else LAM_Z_NC(a.nz, LAM_ZA);
#undef LAM_ZA
    return cudaGetLastError();
}

template <typename T> cudaError_t configure_usfft1d() {
    const int mx = kMaxDynSmem;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(k_usfft1d_fwd<T, false>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_usfft1d_adj<T, false>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_usfft1d_fwd<T, true>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_usfft1d_adj<T, true>, at, mx);
    if constexpr (sizeof(T) == 4) {
#define LAM_NCA(NC)                                                            \
    if (!e) e = cudaFuncSetAttribute(k_usfft1d_fwd<T, false, NC>, at, mx); \
    if (!e) e = cudaFuncSetAttribute(k_usfft1d_adj<T, false, NC>, at, mx);
        LAM_NCA(256) LAM_NCA(512) LAM_NCA(1024) LAM_NCA(2048)
#undef LAM_NCA
    }
    return e;
}

// batched z stage: one persistent launch over every problem's column tiles
template <typename A> __device__ __forceinline__ void copy_block_args_z(A& dst, const A& src) {
    static_assert(sizeof(A) % 4 == 0, "argument block size");
    const int* s = reinterpret_cast<const int*>(&src);
    int* d = reinterpret_cast<int*>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(A) / 4); i += blockDim.x) d[i] = s[i];
}

template <typename T, bool MIXED, bool FWD>
__global__ void __launch_bounds__(kFftThreads) kb_z(const BatchTable<T>* __restrict__ bt) {
    __shared__ Usfft1dArgs<T> sa;
    constexpr int STAGE = FWD ? kBZFwd : kBZAdj;
    const int* st = bt->start[STAGE];
    const int total = st[bt->count];
    int cur = -1;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        int p = 0;
        while (p + 1 < bt->count && w >= st[p + 1]) ++p;
        if (p != cur) {  // block-uniform; the previous item ended with a barrier
            copy_block_args_z(sa, FWD ? bt->zf[p] : bt->za[p]);
            __syncthreads();
            cur = p;
        }
        const int l = w - st[p];
        if (FWD) k_usfft1d_fwd_body<T, MIXED>((const T*)bt->in[p], bt->u1[p], sa, l);
        else k_usfft1d_adj_body<T, MIXED>(bt->u1[p], (T*)bt->out[p], sa, l);
        __syncthreads();
    }
}

template <typename T> static const void* batch_z_kernel(bool fwd, bool mixed) {
    if (fwd) return mixed ? (const void*)kb_z<T, true, true> : (const void*)kb_z<T, false, true>;
    return mixed ? (const void*)kb_z<T, true, false> : (const void*)kb_z<T, false, false>;
}

template <typename T>
cudaError_t launch_batch_z(const BatchTable<T>* dev, bool fwd, bool mixed, const BatchLaunch& L, cudaStream_t s) {
    void* args[] = {(void*)&dev};
    return cudaLaunchKernel(batch_z_kernel<T>(fwd, mixed), dim3(L.grid), dim3(kFftThreads), args, L.smem, s);
}

template <typename T> int batch_occupancy_z(bool fwd, bool mixed, size_t smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_z_kernel<T>(fwd, mixed), kFftThreads, smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

template <typename T> cudaError_t configure_batch_z() {
    cudaError_t e = cudaSuccess;
    for (bool fwd : {false, true})
        for (bool mixed : {false, true})
            if (!e)
                e = cudaFuncSetAttribute(batch_z_kernel<T>(fwd, mixed), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kMaxDynSmem - 2048);
    return e;
}

template cudaError_t launch_batch_z<float>(const BatchTable<float>*, bool, bool, const BatchLaunch&, cudaStream_t);
template cudaError_t launch_batch_z<double>(const BatchTable<double>*, bool, bool, const BatchLaunch&, cudaStream_t);
template int batch_occupancy_z<float>(bool, bool, size_t);
template int batch_occupancy_z<double>(bool, bool, size_t);
template cudaError_t configure_batch_z<float>();
template cudaError_t configure_batch_z<double>();

template cudaError_t launch_usfft1d_fwd<float>(const float*, C<float>*, const Usfft1dArgs<float>&, cudaStream_t);
template cudaError_t launch_usfft1d_fwd<double>(const double*, C<double>*, const Usfft1dArgs<double>&, cudaStream_t);
template cudaError_t launch_usfft1d_adj<float>(const C<float>*, float*, const Usfft1dArgs<float>&, cudaStream_t);
template cudaError_t launch_usfft1d_adj<double>(const C<double>*, double*, const Usfft1dArgs<double>&, cudaStream_t);
template cudaError_t configure_usfft1d<float>();
template cudaError_t configure_usfft1d<double>();

}  // namespace lam
