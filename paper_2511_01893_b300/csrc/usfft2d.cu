// usfft2d.cu - F_u2D and its transpose: one 2D unequally-spaced FFT per kv plane.
//
// F_u2D (Section 2) maps u1[n1, h, n2] to u2[n_theta, h, w]: for each kv plane
// it evaluates sum_{x,y} u1[x, kv, y] exp(-2 pi i (xi_x x + xi_y y)) at the
// n_theta * w slice points (xi_x, xi_y)(theta, kv, ku).  Gaussian USFFT in 2D:
// deapodise, zero-pad to M1 x M2 = 2 n1 x 2 n2, row FFTs (only the n1 non-zero
// rows), column FFTs, then a separable 2m x 2m Gaussian gather.  For a real
// volume a plane job pairs plane kv with its conjugate mirror h - kv: one
// padded FFT serves both.
//
// Forward (type 2) kernels, per batch of nb plane jobs held in P[nb][M1][M2]:
//   k_rowfft_fwd       u1 rows -> deapodised, padded, FFT along y -> P rows
//   k_colfft_fwd_pipe  P columns (n1 non-zero entries) -> FFT along x, in
//                      place; persistent, the next column strip loading while
//                      the current one is transformed
//   k_gather2d_tiled   a 64 x 64 tile of P (+ halo) staged in shared memory,
//                      one lane per slice point: 64 taps, optional fused
//                      subtraction (out = value - sub, Section 4.2); a paired
//                      job's mirror-plane point is the conjugate of its
//                      partner's sum, so each pair is summed once
// Transpose (type 1):
//   k_spread2d_tiles   (default) a block owns a 32 x 32 tile of the padded
//                      plane; each of its warps sums the slice points whose
//                      windows meet the tile into a private tile, and the
//                      warp tiles are added in a fixed order: no atomics,
//                      bitwise reproducible; a paired job's two planes share
//                      one record per pair of mirror points
//   k_spread2d_halo, k_scatter2d_atomic   options (owner tiles with a halo
//                      pass; shared-memory atomics, plain or exact fixed point)
//   k_colfft_adj_pipe  inverse FFT along x, keep the n1 rows the crop needs
//   k_rowfft_adj       inverse FFT along y, crop, deapodise -> u1 rows
// The FP32 row / column kernels are also built for the large power-of-two
// lengths with the length a compile-time constant (LAM_PLANE_NC).
#include <algorithm>

#include "fft.cuh"
#include "kernels.h"

namespace lam {

__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

// --------------------------------------------------------------------------
// row / column passes
// --------------------------------------------------------------------------

template <typename T, bool MIXED, int NC = 0>
__device__ __forceinline__ void k_rowfft_fwd_body(const C<T>* __restrict__ u1, C<T>* __restrict__ P, int j0, const Usfft2dArgs<T>& a, int bx, int by) {
    const int n2 = NC ? NC / 2 : a.n2, M2 = NC ? NC : a.M2;  // the FFT axis (y)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T>* bufa = reinterpret_cast<C<T>*>(smem_raw);
    const int b = by, kv = a.jobs[j0 + b].x;
    const int x0 = bx * a.RB;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int LS = fpad_len(M2);
    for (int i = tid; i < a.RB * LS; i += nthr) bufa[i] = cmake<T>(0, 0);
    __syncthreads();
    const C<T>* src = u1 + ((size_t)kv * a.n1 + x0) * n2;
    for (int i = tid; i < a.RB * n2; i += nthr) {
        const int r = udiv<!MIXED>(i, n2, ilog2_pow2(n2)), y = i - r * n2;
        cp_async_elem<T>(bufa + r * LS + fpad(wrap(y - n2 / 2, M2)), src + i);
    }
    cp_async_commit();
    cp_async_wait_all();
    // each thread deapodises the elements it copied
    for (int i = tid; i < a.RB * n2; i += nthr) {
        const int r = udiv<!MIXED>(i, n2, ilog2_pow2(n2)), y = i - r * n2;
        C<T>* e = bufa + r * LS + fpad(wrap(y - n2 / 2, M2));
        *e = cscale(*e, a.d1[x0 + r] * a.d2[y]);
    }
    __syncthreads();
    fft_lines<-1, T, MIXED, NC>(bufa, a.RB, LS, M2, a.fcM2, a.tw, a.tw2);
    C<T>* dst = P + (size_t)b * a.M1 * M2;
    for (int i = tid; i < a.RB * M2; i += nthr) {
        const int r = udiv<!MIXED>(i, M2, ilog2_pow2(M2)), j = i - r * M2;
        dst[(size_t)wrap(x0 + r - a.n1 / 2, a.M1) * M2 + j] = bufa[r * LS + fpad(j)];
    }
}

template <typename T, bool MIXED, int NC = 0>
__global__ void __launch_bounds__(kFftThreads) k_rowfft_fwd(const C<T>* __restrict__ u1, C<T>* __restrict__ P,
                                                    int j0, Usfft2dArgs<T> a) {
    k_rowfft_fwd_body<T, MIXED, NC>(u1, P, j0, a, (int)blockIdx.x, (int)blockIdx.y);
}

template <typename T, bool MIXED>
__device__ __forceinline__ void k_colfft_fwd_body(C<T>* __restrict__ P, const Usfft2dArgs<T>& a, int bx, int by) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T>* bufa = reinterpret_cast<C<T>*>(smem_raw);
    const int b = by;
    const int c0 = bx * a.CB;
    const int tid = threadIdx.x, nthr = blockDim.x;
    C<T>* pl = P + (size_t)b * a.M1 * a.M2 + c0;
    const int LS = fpad_len(a.M1);
    for (int i = tid; i < a.CB * LS; i += nthr) bufa[i] = cmake<T>(0, 0);
    __syncthreads();
    for (int i = tid; i < a.n1 * a.CB; i += nthr) {
        const int x = i >> ilog2_pow2(a.CB), c = i - x * a.CB;  // CB is a power of two
        const int row = wrap(x - a.n1 / 2, a.M1);
        bufa[c * LS + fpad(row)] = pl[(size_t)row * a.M2 + c];
    }
    __syncthreads();
    fft_lines_ip<-1, FftMaxB<T>::value, T, MIXED>(bufa, a.CB, LS, a.M1, a.fcM1, a.tw, a.tw1);
    for (int i = tid; i < a.M1 * a.CB; i += nthr) {
        const int j = i >> ilog2_pow2(a.CB), c = i - j * a.CB;
        pl[(size_t)j * a.M2 + c] = bufa[c * LS + fpad(j)];
    }
}

template <typename T, bool MIXED>
__device__ __forceinline__ void k_colfft_adj_body(C<T>* __restrict__ P, const Usfft2dArgs<T>& a, int bx, int by) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T>* bufa = reinterpret_cast<C<T>*>(smem_raw);
    const int b = by;
    const int c0 = bx * a.CB;
    const int tid = threadIdx.x, nthr = blockDim.x;
    C<T>* pl = P + (size_t)b * a.M1 * a.M2 + c0;
    const int LS = fpad_len(a.M1);
    for (int i = tid; i < a.M1 * a.CB; i += nthr) {
        const int j = i >> ilog2_pow2(a.CB), c = i - j * a.CB;
        bufa[c * LS + fpad(j)] = pl[(size_t)j * a.M2 + c];
    }
    __syncthreads();
    fft_lines_ip<+1, FftMaxB<T>::value, T, MIXED>(bufa, a.CB, LS, a.M1, a.fcM1, a.tw, a.tw1);
    for (int i = tid; i < a.n1 * a.CB; i += nthr) {
        const int x = i >> ilog2_pow2(a.CB), c = i - x * a.CB;  // CB is a power of two
        const int row = wrap(x - a.n1 / 2, a.M1);
        pl[(size_t)row * a.M2 + c] = bufa[c * LS + fpad(row)];
    }
}

// ---------------------------------------------------------------------------
// Pipelined column passes: persistent blocks walk the (plane, column strip)
// items with two shared-memory buffers; the next strip's loads (cp.async)
// are in flight while the current strip is transformed and stored.
// ---------------------------------------------------------------------------


// forward: rows wrap(x - n1/2) (x < n1) hold data, the others are zero padding;
// the FFT overwrites every row, so after the stores the padding rows are
// zeroed again for the buffer's next strip
template <typename T, bool MIXED, int NC = 0>
__global__ void __launch_bounds__(kFftThreads) k_colfft_fwd_pipe(C<T>* __restrict__ P, Usfft2dArgs<T> a, int nb) {
    const int n1 = NC ? NC / 2 : a.n1, M1 = NC ? NC : a.M1;  // the FFT axis (x)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int LS = fpad_len(M1);
    C<T>* buf[2] = {reinterpret_cast<C<T>*>(smem_raw), reinterpret_cast<C<T>*>(smem_raw) + a.CB * LS};
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lcb = ilog2_pow2(a.CB);
    const int ncg = a.M2 / a.CB, total = ncg * nb;
    const int half = n1 / 2, hi0 = M1 - half;  // data rows: [0, half) and [hi0, M1)
    for (int i = tid; i < 2 * a.CB * LS; i += nthr) buf[0][i] = cmake<T>(0, 0);
    __syncthreads();
    auto issue = [&](int w, C<T>* bb) {
        const int b = w / ncg, c0 = (w - b * ncg) * a.CB;
        const C<T>* pl = P + (size_t)b * M1 * a.M2 + c0;
        for (int i = tid; i < n1 * a.CB; i += nthr) {
            const int x = i >> lcb, c = i - (x << lcb);
            const int row = wrap(x - half, M1);
            cp_async_elem<T>(bb + c * LS + fpad(row), pl + (size_t)row * a.M2 + c);
        }
        cp_async_commit();
    };
    int k = 0;
    if ((int)blockIdx.x < total) issue(blockIdx.x, buf[0]);
    for (int w = blockIdx.x; w < total; w += gridDim.x, ++k) {
        C<T>* cur = buf[k & 1];
        const int wn = w + gridDim.x;
        if (wn < total) issue(wn, buf[(k + 1) & 1]);
        else cp_async_commit();  // an empty group keeps the wait count uniform
        cp_async_wait_prev();
        __syncthreads();
        fft_lines<-1, T, MIXED, NC>(cur, a.CB, LS, M1, a.fcM1, a.tw, a.tw1);
        const int b = w / ncg, c0 = (w - b * ncg) * a.CB;
        C<T>* pl = P + (size_t)b * M1 * a.M2 + c0;
        for (int i = tid; i < M1 * a.CB; i += nthr) {
            const int j = i >> lcb, c = i - (j << lcb);
            C<T>* e = cur + c * LS + fpad(j);
            pl[(size_t)j * a.M2 + c] = *e;
            if (j >= half && j < hi0) *e = cmake<T>(0, 0);
        }
        __syncthreads();  // cur is free before it is refilled two items later
    }
    cp_async_wait_all();
}

// transpose: every row is loaded; the n1 rows the crop keeps are stored
template <typename T, bool MIXED, int NC = 0>
__global__ void __launch_bounds__(kFftThreads) k_colfft_adj_pipe(C<T>* __restrict__ P, Usfft2dArgs<T> a, int nb,
                                                                int j0) {
    const int n1 = NC ? NC / 2 : a.n1, M1 = NC ? NC : a.M1;  // the FFT axis (x)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int LS = fpad_len(M1);
    C<T>* buf[2] = {reinterpret_cast<C<T>*>(smem_raw), reinterpret_cast<C<T>*>(smem_raw) + a.CB * LS};
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lcb = ilog2_pow2(a.CB);
    const int ncg = a.M2 / a.CB, total = ncg * nb;
    // plane jobs served from the memoization cache are not loaded or transformed
    auto skipped = [&](int w) { return a.memo_hit && a.memo_hit[j0 + w / ncg]; };
    auto issue = [&](int w, C<T>* bb) {
        const int b = w / ncg, c0 = (w - b * ncg) * a.CB;
        const C<T>* pl = P + (size_t)b * M1 * a.M2 + c0;
        if (!skipped(w))
            for (int i = tid; i < M1 * a.CB; i += nthr) {
                const int j = i >> lcb, c = i - (j << lcb);
                cp_async_elem<T>(bb + c * LS + fpad(j), pl + (size_t)j * a.M2 + c);
            }
        cp_async_commit();
    };
    int k = 0;
    if ((int)blockIdx.x < total) issue(blockIdx.x, buf[0]);
    for (int w = blockIdx.x; w < total; w += gridDim.x, ++k) {
        C<T>* cur = buf[k & 1];
        const int wn = w + gridDim.x;
        if (wn < total) issue(wn, buf[(k + 1) & 1]);
        else cp_async_commit();
        cp_async_wait_prev();
        __syncthreads();
        if (!skipped(w)) {  // block-uniform
            fft_lines<+1, T, MIXED, NC>(cur, a.CB, LS, M1, a.fcM1, a.tw, a.tw1);
            const int b = w / ncg, c0 = (w - b * ncg) * a.CB;
            C<T>* pl = P + (size_t)b * M1 * a.M2 + c0;
            for (int i = tid; i < n1 * a.CB; i += nthr) {
                const int x = i >> lcb, c = i - (x << lcb);
                const int row = wrap(x - n1 / 2, M1);
                pl[(size_t)row * a.M2 + c] = cur[c * LS + fpad(row)];
            }
        }
        __syncthreads();
    }
    cp_async_wait_all();
}

// persistent grid of a pipelined column pass: as many blocks as fit on the
// SMs by registers (the FFT blocks run at up to 128 registers a thread: one
// 512-thread or two 256-thread blocks per SM), at most one per item
static int pipe_grid(int items, int threads, size_t smem) {
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            nsm = 148;
    }
    int per_sm = threads <= 256 ? 2 : 1;
    // 228 KB of shared memory per SM, 1 KB of it reserved per block
    while (per_sm > 1 && (size_t)per_sm * (smem + 1024) > 228 * 1024) --per_sm;
    const int g = nsm * per_sm;
    return items < g ? items : g;
}

template <typename T, bool MIXED, int NC = 0>
__device__ __forceinline__ void k_rowfft_adj_body(const C<T>* __restrict__ P, C<T>* __restrict__ u1, int j0, const Usfft2dArgs<T>& a, int bx, int by) {
    const int n2 = NC ? NC / 2 : a.n2, M2 = NC ? NC : a.M2;  // the FFT axis (y)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T>* bufa = reinterpret_cast<C<T>*>(smem_raw);
    if (a.memo_hit && a.memo_hit[j0 + by]) return;  // the cached plane is copied into u1 instead
    const int b = by, kv = a.jobs[j0 + b].x;
    const int x0 = bx * a.RB;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const C<T>* pl = P + (size_t)b * a.M1 * M2;
    const int LS = fpad_len(M2);
    for (int i = tid; i < a.RB * M2; i += nthr) {
        const int r = udiv<!MIXED>(i, M2, ilog2_pow2(M2)), j = i - r * M2;
        cp_async_elem<T>(bufa + r * LS + fpad(j), pl + (size_t)wrap(x0 + r - a.n1 / 2, a.M1) * M2 + j);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    fft_lines<+1, T, MIXED, NC>(bufa, a.RB, LS, M2, a.fcM2, a.tw, a.tw2);
    C<T>* dst = u1 + ((size_t)kv * a.n1 + x0) * n2;
    for (int i = tid; i < a.RB * n2; i += nthr) {
        const int r = udiv<!MIXED>(i, n2, ilog2_pow2(n2)), y = i - r * n2;
        const T s = a.d1[x0 + r] * a.d2[y];
        dst[i] = cscale(bufa[r * LS + fpad(wrap(y - n2 / 2, M2))], s);
    }
}

template <typename T, bool MIXED, int NC = 0>
__global__ void __launch_bounds__(kFftThreads) k_rowfft_adj(const C<T>* __restrict__ P, C<T>* __restrict__ u1,
                                                    int j0, Usfft2dArgs<T> a) {
    k_rowfft_adj_body<T, MIXED, NC>(P, u1, j0, a, (int)blockIdx.x, (int)blockIdx.y);
}

// --------------------------------------------------------------------------
// slice-point positions
// --------------------------------------------------------------------------

__device__ __forceinline__ void point_pos(const AngleF& g, int kuc, int kvc, int& jx, float& fx, int& jy,
                                          float& fy) {
    grid_pos(kuc, kvc, g.ax_hi, g.ax_lo, g.sx_hi, g.sx_lo, jx, fx);
    grid_pos(kuc, kvc, g.ay_hi, g.ay_lo, g.sy_hi, g.sy_lo, jy, fy);
}
__device__ __forceinline__ void point_pos(const AngleD& g, int kuc, int kvc, int& jx, double& fx, int& jy,
                                          double& fy) {
    grid_pos(kuc, kvc, g.ax, g.sx, jx, fx);
    grid_pos(kuc, kvc, g.ay, g.sy, jy, fy);
}
__device__ __forceinline__ void line_coef(const AngleF& g, int kvc, float& Ax, float& Cx, float& Ay, float& Cy) {
    Ax = g.ax_hi;
    Cx = (float)kvc * g.sx_hi;
    Ay = g.ay_hi;
    Cy = (float)kvc * g.sy_hi;
}
__device__ __forceinline__ void line_coef(const AngleD& g, int kvc, double& Ax, double& Cx, double& Ay,
                                          double& Cy) {
    Ax = g.ax;
    Cx = (double)kvc * g.sx;
    Ay = g.ay;
    Cy = (double)kvc * g.sy;
}

// ku interval [lo, hi] (centred) of points on the line p = A ku + Cc whose
// position lies in [bmin, bmax); conservative by one point at each end.
template <typename T>
__device__ __forceinline__ void clip_line(T A, T Cc, T bmin, T bmax, int& lo, int& hi) {
    if (fabs(A) < (T)1e-6) {
        if (!(Cc >= bmin - (T)1 && Cc < bmax + (T)1)) {
            lo = 1;
            hi = 0;
        }
        return;
    }
    T t0 = (bmin - Cc) / A, t1 = (bmax - Cc) / A;
    if (t0 > t1) {
        const T tmp = t0;
        t0 = t1;
        t1 = tmp;
    }
    // clamp before the conversion so that huge quotients stay in int range
    t0 = fmax(t0, (T)-1e8);
    t1 = fmin(t1, (T)1e8);
    const int l = (int)floor(t0) - 1, h = (int)ceil(t1) + 1;
    lo = max(lo, l);
    hi = min(hi, h);
}

// Hands out the points of the warp's up to 32 lines (lane i: line th_i with
// the centred ku interval [lo_i, hi_i]; th_i = -1 or lo_i > hi_i for none)
// 32 at a time, one per lane, in lane order and ku order within a line:
// fn(th, kuc) is called by all lanes together, with th = -1 for idle lanes.
template <typename F>
__device__ __forceinline__ void walk_line_points(int th, int lo, int hi, F&& fn) {
    const int lane = threadIdx.x & 31;
    const int cnt = th >= 0 && hi >= lo ? hi - lo + 1 : 0;
    // inclusive scan of cnt over the warp
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int excl = incl - cnt;
    for (int p0 = 0; p0 < total; p0 += 32) {
        const int p = p0 + lane;
        // owner lane: the last lane whose exclusive prefix is <= p (with cnt > 0)
        int owner = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int cand = owner + step;
            const int ex = __shfl_sync(0xffffffffu, excl, cand);
            if (ex <= p) owner = cand;
        }
        const int ocnt = __shfl_sync(0xffffffffu, cnt, owner);
        const int oex = __shfl_sync(0xffffffffu, excl, owner);
        const int olo = __shfl_sync(0xffffffffu, lo, owner);
        const int oth = __shfl_sync(0xffffffffu, th, owner);
        const bool valid = p < total && ocnt > 0 && p - oex < ocnt;
        const int kuc = olo + (p - oex);
        fn(valid ? oth : -1, kuc);
    }
}

// ---------------------------------------------------------------------------
// Warp-level enumeration of the slice points that may touch one tile image.
// The warp tests 32 lines at a time against the tile's position box (lane
// parallel, a distance test only) and appends the crossing lines to a per-warp
// list in shared memory.  Each time 32 lines are listed (and once at the end)
// it computes their ku intervals (clipping to the box), scans the interval
// lengths and hands the flattened point list out 32 points at a time, one per
// lane, across line boundaries.  Lines keep their order and points their ku
// order, so the sequence of points a warp sees does not depend on how they
// are batched.  fn(th, kuc) is called for each lane's point (active lanes
// first in each batch; inactive lanes get th = -1), by all lanes together.
// ---------------------------------------------------------------------------
template <typename T, int NW, typename F>
__device__ __forceinline__ void for_tile_points(const Usfft2dArgs<T>& a, int kvc, T cx, T cy, T hbox,
                                                T bxmin, T bxmax, T bymin, T bymax, int w, int kext, F&& fn) {
    __shared__ int s_lines[NW][64];
    int* list = s_lines[w];
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    // kext = 1 adds the point ku = w/2 past each line's end (the partner of
    // the mirror plane's ku = -w/2 point in the paired operators)
    const int kmin = -a.w / 2, kmax = a.w / 2 - 1 + kext;
    // clip up to 32 listed lines (lane i takes list[i]) and enumerate their points
    auto flush = [&](int count) {
        const int th = lane < count ? list[lane] : -1;
        int lo = 1, hi = 0;
        if (th >= 0) {
            const typename AngleT<T>::type g = a.ang[th];
            T Ax, Cx, Ay, Cy;
            line_coef(g, kvc, Ax, Cx, Ay, Cy);
            lo = kmin;
            hi = kmax;
            clip_line<T>(Ax, Cx, bxmin, bxmax, lo, hi);
            clip_line<T>(Ay, Cy, bymin, bymax, lo, hi);
        }
        walk_line_points(th, lo, hi, fn);
    };
    int nlist = 0;  // warp-uniform
    for (int base = 0; base * NW < a.T_; base += 32) {
        const int th = (base + lane) * NW + w;
        bool pass = false;
        if (th < a.T_) {
            const typename AngleT<T>::type g = a.ang[th];
            T Ax, Cx, Ay, Cy;
            line_coef(g, kvc, Ax, Cx, Ay, Cy);
            const T nrm = sqrt(Ax * Ax + Ay * Ay);
            const T nx = -Ay / nrm, ny = Ax / nrm;
            const T dist = fabs((cx - Cx) * nx + (cy - Cy) * ny);
            pass = dist <= hbox * (fabs(nx) + fabs(ny)) + (T)1;
        }
        const unsigned m = __ballot_sync(0xffffffffu, pass);
        if (pass) list[nlist + __popc(m & lt)] = th;
        nlist += __popc(m);
        __syncwarp();
        if (nlist >= 32) {
            flush(32);
            // keep the overflow (fewer than 32 lines) at the front of the list
            const int rest = nlist - 32;
            const int v = lane < rest ? list[32 + lane] : 0;
            __syncwarp();
            if (lane < rest) list[lane] = v;
            __syncwarp();
            nlist = rest;
        }
    }
    if (nlist > 0) flush(nlist);
    __syncwarp();
}

// Tiled gather: one block per TS x TS tile of tap-window origins.  The block
// stages its tile plus a (2m - 1) halo of the padded plane in shared memory
// (and one more row and column on the low side, below) and evaluates exactly
// the points whose window origin (j0 - m + 1 in both axes, unwrapped) falls in
// the tile or one of its periodic images, one point per lane, with the slice
// lines dealt to the warps and each warp's point list flattened across lines.
// Each point is owned by exactly one (tile, image), so every output is
// written once.
//
// Paired jobs (real volumes): the mirror plane -kv is the conjugate mirror of
// this plane's padded FFT, P_mirror[j] = conj P[-j], and its slice point
// (theta, -ku, -kv) sits at exactly the negated position of this plane's point
// (theta, ku, kv).  Where the two tap windows mirror (j0' = -j0 - 1 on both
// axes) the mirror point's value is conj of this point's sum, so each pair is
// summed once.  Where a position lies within the tap shift of a grid node the
// mirror point's window is this one shifted down by one cell; it is summed
// separately over the staged cells one row / column below, which is what the
// extra low row and column are for.  The mirror point ku = -w/2 has no partner
// among this plane's points: its partner is the point ku = w/2 one step past
// the line's end, which the enumeration adds for paired jobs (it has no output
// of its own).
template <typename T, int TPB, int MH>
__device__ __forceinline__ void k_gather2d_tiled_body(const C<T>* __restrict__ P, C<T>* __restrict__ out, const C<T>* __restrict__ sub, int j0, const Usfft2dArgs<T>& a, int bx, int by) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int nt = 2 * MH;
    const int TS = a.TG;
    const int SH = TS + nt;      // staged rows: window origins tx0 - 1 .. tx0 + TS - 1
    const int SW = TS + nt + 1;  // staged row stride (odd: lanes two rows apart hit different banks)
    const int warp = threadIdx.x >> 5;
    const int tiles_y = a.M2 / TS;
    const int tile = bx;
    C<T>* st = reinterpret_cast<C<T>*>(smem_raw);
    const int tx0 = (tile / tiles_y) * TS, ty0 = (tile % tiles_y) * TS;
    const int b = by;
    const int2 job = a.jobs[j0 + b];
    const bool paired = job.y >= 0;
    const int kv = job.x, kvc = kv - a.h / 2;
    const C<T>* pl = P + (size_t)b * a.M1 * a.M2;
    for (int i = threadIdx.x; i < SH * SH; i += blockDim.x) {
        const int r = i / SH, c = i - r * SH;
        cp_async_elem<T>(st + r * SW + c, pl + (size_t)wrap(tx0 - 1 + r, a.M1) * a.M2 + wrap(ty0 - 1 + c, a.M2));
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    // sum of the (2m)^2 taps whose window starts at staged row sx0, column sy0
    // (tile-relative origin + 1), at fractions fx, fy
    auto window_sum = [&](int sx0, int sy0, T fx, T fy) {
        T wy[nt];
#pragma unroll
        for (int t = 0; t < nt; ++t) {
            const T d = fy + (T)(MH - 1 - t);
            wy[t] = gexp(-d * d * a.inv4beta);
        }
        T sr = 0, si = 0;
#ifdef LAM_GATHER_KAHAN
        T csr = 0, csi = 0;
#endif
#pragma unroll
        for (int sx = 0; sx < nt; ++sx) {
            const T d = fx + (T)(MH - 1 - sx);
            const T wx = gexp(-d * d * a.inv4beta);
            const C<T>* rowp = st + (sx0 + sx) * SW + sy0;
            T rr = 0, ri = 0;
#pragma unroll
            for (int t = 0; t < nt; ++t) {
                const C<T> pv = rowp[t];
                rr = fma(wy[t], pv.x, rr);
                ri = fma(wy[t], pv.y, ri);
            }
#ifdef LAM_GATHER_KAHAN
            {
                const T yr = wx * rr - csr, yi = wx * ri - csi;
                const T tr = add_rn(sr, yr), ti = add_rn(si, yi);
                csr = sub_rn(sub_rn(tr, sr), yr);
                csi = sub_rn(sub_rn(ti, si), yi);
                sr = tr;
                si = ti;
            }
#else
            sr = fma(wx, rr, sr);
            si = fma(wx, ri, si);
#endif
        }
        return cmake<T>(sr, si);
    };
    const T hb = (T)TS * (T)0.5 + (T)1;
    for (int ix = -a.nimg; ix <= a.nimg; ++ix) {
        const int bx0 = tx0 + ix * a.M1;
        for (int iy = -a.nimg; iy <= a.nimg; ++iy) {
            const int by0 = ty0 + iy * a.M2;
            // positions whose window origin is in [b0, b0 + TS): p in [b0 + m - 1, b0 + TS + m - 1)
            const T cx = (T)(bx0 + a.m - 1) + (T)TS * (T)0.5, cy = (T)(by0 + a.m - 1) + (T)TS * (T)0.5;
            if (sqrt(cx * cx + cy * cy) > a.rmax + hb * (T)1.5) continue;
            for_tile_points<T, TPB>(a, kvc, cx, cy, hb, (T)(bx0 + a.m - 1), (T)(bx0 + TS + a.m - 1),
                               (T)(by0 + a.m - 1), (T)(by0 + TS + a.m - 1), warp, paired ? 1 : 0, [&](int th, int kuc) {
                if (th < 0) return;
                const typename AngleT<T>::type g = a.ang[th];
                int jx, jy;
                T fx, fy;
                point_pos(g, kuc, kvc, jx, fx, jy, fy);
                const int ox = jx - a.m + 1 - bx0, oy = jy - a.m + 1 - by0;
                if (ox < 0 || ox >= TS || oy < 0 || oy >= TS) return;
                // the window's last staged row and column
                if (!(LAM_INB(ox + nt, SH, a.err, kSiteGatherWindow) &&
                      LAM_INB(oy + nt, SH, a.err, kSiteGatherWindow)))
                    return;
                if (!(LAM_INB(th, a.T_, a.err, kSiteGatherOut))) return;
                const bool has_p = kuc < a.w / 2;              // a point of this plane (not the one past the end)
                const bool has_q = paired && kuc > -a.w / 2;   // its partner (theta, -ku) in the mirror plane
                int jxq = 0, jyq = 0;
                T fxq = 0, fyq = 0;
                bool mir = true;
                if (has_q) {
                    point_pos(g, -kuc, -kvc, jxq, fxq, jyq, fyq);
                    mir = jxq == -jx - 1 && jyq == -jy - 1;
                }
                C<T> vp = cmake<T>(0, 0);
                if (has_p || (has_q && mir)) vp = window_sum(ox + 1, oy + 1, fx, fy);
                if (has_p) {
                    const size_t o = ((size_t)th * a.h + kv) * a.w + (kuc + a.w / 2);
                    C<T> v = vp;
                    if (sub) v = csub(v, sub[o]);
                    out[o] = v;
                }
                if (has_q) {
                    if (!mir) {
                        // the mirror window in this plane's grid: origin -j0' - m,
                        // fraction 1 - fr' (one cell below this point's window)
                        const int sxq = (-jxq - 1) - a.m + 1 - bx0 + 1, syq = (-jyq - 1) - a.m + 1 - by0 + 1;
                        if (!(LAM_INB(sxq, TS + 1, a.err, kSiteGatherWindow) &&
                              LAM_INB(syq, TS + 1, a.err, kSiteGatherWindow)))
                            return;
                        if ((unsigned)sxq > (unsigned)TS || (unsigned)syq > (unsigned)TS) return;
                        vp = window_sum(sxq, syq, (T)1 - fxq, (T)1 - fyq);
                    }
                    const size_t o = ((size_t)th * a.h + job.y) * a.w + (a.w / 2 - kuc);
                    C<T> v = cconj(vp);
                    if (sub) v = csub(v, sub[o]);
                    out[o] = v;
                }
            });
        }
    }
}

template <typename T, int TPB, int MH>
__global__ void __launch_bounds__(TPB * 32) k_gather2d_tiled(const C<T>* __restrict__ P, C<T>* __restrict__ out,
                                                             const C<T>* __restrict__ sub, int j0, Usfft2dArgs<T> a) {
    k_gather2d_tiled_body<T, TPB, MH>(P, out, sub, j0, a, (int)blockIdx.x, (int)blockIdx.y);
}

// Cells are stored planar (real parts, then imaginary parts) with the column
// index XOR-swizzled by the row: lanes working on neighbouring points of one
// line (origins about two cells apart in any direction) then mostly hit
// different banks.  The swizzle only permutes the low five bits within each
// 32-cell row, so it is a bijection on [0, TS*TS) for power-of-two TS.
__device__ __forceinline__ int swz(int cell) { return cell ^ ((cell >> 5) & 31); }

// Scatter: one block per tile; the block's warps share one accumulator and
// split the crossing lines, and each lane spreads its own point's (2m)^2 taps
// independently with shared-memory atomic adds.  With exact fixed-point cells
// (ACC 3) the order of the adds does not matter; with plain floating-point
// cells (ACC 0) the rounding depends on scheduling.

// Accumulator cells for the scatter: ACC 0 plain atomic adds, ACC 3 exact
// fixed point (below).

template <typename T, int ACC> struct AtomAcc {  // ACC 0: plain FP32 / FP64 atomic adds
    T* base;
    int ncell;
    __device__ __forceinline__ void zero(int t, int nt_) {
        for (int i = t; i < 2 * ncell; i += nt_) base[i] = (T)0;
    }
    __device__ __forceinline__ void add(int cell, T vr, T vi) {
        const int c = swz(cell);
        atomicAdd(base + c, vr);
        atomicAdd(base + ncell + c, vi);
    }
    __device__ __forceinline__ C<T> get(int cell) const {
        const int c = swz(cell);
        return cmake<T>(base[c], base[ncell + c]);
    }
};

// Exact fixed-point cells: each product is scaled by a power of two (chosen
// from a bound on every cell's magnitude, so no cell can overflow) and rounded
// to a 64-bit integer, i.e. to a fixed grid of step ~ bound_count * maxabs *
// 2^-61.  Integer adds are exact and associative, so a cell is the exact sum
// of its rounded products, bitwise independent of the order the lanes and
// warps add in.  The per-product error is bounded in absolute terms (half a
// grid step), not relative to the cell: cells far smaller than maxabs lose
// relative precision, and in FP64 the grid step can exceed FP64 rounding.
template <typename T> struct AtomAcc<T, 3> {
    unsigned long long* base;
    int ncell;
    T scale, inv_scale;
    __device__ __forceinline__ void zero(int t, int nt_) {
        for (int i = t; i < 2 * ncell; i += nt_) base[i] = 0ull;
    }
    __device__ __forceinline__ void add(int cell, T vr, T vi) {
        const int c = swz(cell);
        atomicAdd(base + c, (unsigned long long)to_ll(vr * scale));
        atomicAdd(base + ncell + c, (unsigned long long)to_ll(vi * scale));
    }
    __device__ __forceinline__ C<T> get(int cell) const {
        const int c = swz(cell);
        return cmake<T>(from_ll((long long)base[c]) * inv_scale, from_ll((long long)base[ncell + c]) * inv_scale);
    }
    static __device__ __forceinline__ long long to_ll(float x) { return __float2ll_rn(x); }
    static __device__ __forceinline__ long long to_ll(double x) { return __double2ll_rn(x); }
    static __device__ __forceinline__ T from_ll(long long x) {
        if (sizeof(T) == 4) return (T)__ll2float_rn(x);
        return (T)__ll2double_rn(x);
    }
};

template <typename T, int ACC> __host__ __device__ constexpr int atom_acc_bytes() {
    return ACC == 3 ? 16 : 2 * (int)sizeof(T);
}

// Power-of-two scale for the fixed-point cells: every cell is a sum of at most
// bound_count products |w v| <= maxabs (w <= 1), so 2^61 / (bound_count *
// maxabs), rounded down to a power of two, keeps every partial sum below 2^61.
template <typename T> __device__ __forceinline__ void fixed_scale(T maxabs, float bound_count, T& s, T& inv) {
    if (!(maxabs > (T)0)) {
        s = inv = (T)1;
        return;
    }
    int e1, e2;
    frexp((double)maxabs, &e1);       // maxabs < 2^e1
    frexp((double)bound_count, &e2);  // bound_count < 2^e2
    int e = 61 - e1 - e2;
    const int lim = sizeof(T) == 4 ? 120 : 1000;
    if (e > lim) e = lim;
    if (e < -lim) e = -lim;
    s = (T)ldexp(1.0, e);
    inv = (T)ldexp(1.0, -e);
}

template <typename T, int TPB, int MH, int ACC>
__global__ void __launch_bounds__(TPB * 32, TPB >= 16 ? (sizeof(T) == 4 ? 2 : 1) : (sizeof(T) == 4 ? 6 : 2)) k_scatter2d_atomic(
    const C<T>* __restrict__ in, C<T>* __restrict__ P, int j0, Usfft2dArgs<T> a) {
    constexpr int nt = 2 * MH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (a.memo_hit && a.memo_hit[j0 + blockIdx.y]) return;  // served from the memoization cache
    const int TS = a.TS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_y = a.M2 / TS;
    const int tile = blockIdx.x;
    const int ncell = TS * TS;
    AtomAcc<T, ACC> acc;
    acc.base = reinterpret_cast<decltype(acc.base)>(smem_raw);
    acc.ncell = ncell;
    if constexpr (ACC == 3) fixed_scale<T>(*a.maxabs, a.bound_count, acc.scale, acc.inv_scale);
    acc.zero(threadIdx.x, blockDim.x);
    __syncthreads();
    const int tx0 = (tile / tiles_y) * TS, ty0 = (tile % tiles_y) * TS;
    const int b = blockIdx.y;
    const int2 job = a.jobs[j0 + b];
    const T hb = (T)(TS + 2 * a.m) * (T)0.5;
    // pass 0: the job's own plane; pass 1: its mirror plane, whose point at
    // position p spreads conj(value) around -p (window origin -j0' - m,
    // fraction 1 - fr'), which is where the mirror plane's padded grid lands
    // in this plane's grid
    for (int pass = 0; pass < 2; ++pass) {
        const int kv = pass ? job.y : job.x;
        if (kv < 0) break;
        const int kvc = kv - a.h / 2;
        const T sg = pass ? (T)-1 : (T)1;
        for (int ix = -a.nimg; ix <= a.nimg; ++ix) {
            const int bx0 = tx0 + ix * a.M1;
            for (int iy = -a.nimg; iy <= a.nimg; ++iy) {
                const int by0 = ty0 + iy * a.M2;
                const T cx = (T)bx0 + (T)(TS - 1) * (T)0.5, cy = (T)by0 + (T)(TS - 1) * (T)0.5;
                if (sqrt(cx * cx + cy * cy) > a.rmax + hb * (T)1.5) continue;
                // box of positions (own plane's coordinates) whose taps reach the tile image
                T bxl = (T)(bx0 - a.m), bxh = (T)(bx0 + TS + a.m - 1);
                T byl = (T)(by0 - a.m), byh = (T)(by0 + TS + a.m - 1);
                if (pass) {
                    const T t0 = -bxh, t1 = -bxl + (T)1, t2 = -byh, t3 = -byl + (T)1;
                    bxl = t0; bxh = t1; byl = t2; byh = t3;
                }
                for_tile_points<T, TPB>(a, kvc, sg * cx, sg * cy, hb, bxl, bxh, byl, byh, warp, 0, [&](int th, int kuc) {
                    if (th < 0) return;
                    const typename AngleT<T>::type g = a.ang[th];
                    int jx, jy;
                    T fx, fy;
                    point_pos(g, kuc, kvc, jx, fx, jy, fy);
                    C<T> v = in[((size_t)th * a.h + kv) * a.w + (kuc + a.w / 2)];
                    if (pass) {
                        jx = -jx - 1;
                        jy = -jy - 1;
                        fx = (T)1 - fx;
                        fy = (T)1 - fy;
                        v.y = -v.y;
                    }
                    const int ox = jx - MH + 1 - bx0, oy = jy - MH + 1 - by0;
                    if (ox <= -nt || ox >= TS || oy <= -nt || oy >= TS) return;
                    T wy[nt];
#pragma unroll
                    for (int t = 0; t < nt; ++t) {
                        const T dy = fy + (T)(MH - 1 - t);
                        wy[t] = gexp(-dy * dy * a.inv4beta);
                    }
#pragma unroll
                    for (int sx = 0; sx < nt; ++sx) {
                        const int cxx = ox + sx;
                        if (cxx < 0 || cxx >= TS) continue;
                        const T dx = fx + (T)(MH - 1 - sx);
                        const T wx = gexp(-dx * dx * a.inv4beta);
                        const T vr = wx * v.x, vi = wx * v.y;
#pragma unroll
                        for (int sy = 0; sy < nt; ++sy) {
                            const int cyy = oy + sy;
                            if (cyy >= 0 && cyy < TS) acc.add(cxx * TS + cyy, wy[sy] * vr, wy[sy] * vi);
                        }
                    }
                });
            }
        }
    }
    __syncthreads();
    C<T>* pl = P + (size_t)b * a.M1 * a.M2;
    for (int i = threadIdx.x; i < ncell; i += blockDim.x) {
        const int cxx = i / TS, cyy = i - cxx * TS;
        pl[(size_t)(tx0 + cxx) * a.M2 + ty0 + cyy] = acc.get(i);
    }
    (void)lane;
}

// Spread without atomics (default): every warp accumulates into its own
// kSpreadTS x kSpreadTS tile in shared memory; the block's warps split the
// crossing lines as in the atomic kernel.  Each lane first finds its own point;
// the warp compacts the points whose window meets the tile into a list of
// records (window origin, the 2m weights along x, the 2m weights along y
// times the value), then takes them one at a time, its 32 lanes covering the
// point's (2m) x (2m) window (RPP rows of 2m columns per pass), each lane a
// read-add-write of one cell per pass.  One point's cells are distinct, so
// there is no race within the warp, and a __syncwarp orders consecutive
// points.  The next record is read before the current point's cells are
// updated, to overlap the two.  At the end the warp tiles are summed in warp
// order: the result does not depend on scheduling.
// Records are stored transposed with a row pitch of 33 (lane-major writes and
// per-row reads both free of bank conflicts); a lane's x weights for all its
// passes sit next to the window origin, one load.  Tile cells are complex, row-major, with the column
// XOR-swizzled by the row's parity: the 4-row x 8-column block of one pass
// then covers 16 distinct pairs of banks (FP32), two lanes per pair, the
// minimum for 256 bytes.
constexpr int kSpreadTS = 32;
constexpr int kRecPitch = 33;
__device__ __forceinline__ int swz_row(int x, int y) { return y ^ ((x & 1) << 3); }

// a lane's view of a point record: its x weights for every pass and the
// window origin, read with one load (16 bytes for FP32 at m = 4)
template <typename T, int NPASS> struct alignas(sizeof(T) * NPASS + 8 == 16 ? 16 : 8) SpreadRec {
    T wx[NPASS];
    int ox, oy;
};
// split: points a warp spreads at once (1: all 32 lanes cover one point's
// window; 2: each half-warp covers its own point in its own tile)
__host__ __device__ constexpr int spread_rpp(int mh, int split = 1) { return 32 / split / (2 * mh); }
__host__ __device__ constexpr int spread_npass(int mh, int split = 1) {
    return (2 * mh + spread_rpp(mh, split) - 1) / spread_rpp(mh, split);
}
template <typename T> size_t spread_rec_bytes(int mh, int split = 1) {
    switch (spread_npass(mh, split)) {
        case 1: return sizeof(SpreadRec<T, 1>);
        case 2: return sizeof(SpreadRec<T, 2>);
        case 3: return sizeof(SpreadRec<T, 3>);
        case 4: return sizeof(SpreadRec<T, 4>);
        case 6: return sizeof(SpreadRec<T, 6>);
        case 7: return sizeof(SpreadRec<T, 7>);
        case 8: return sizeof(SpreadRec<T, 8>);
        default: return sizeof(SpreadRec<T, 16>);
    }
}
// exact: the tile cells are 64-bit fixed-point pairs (16 bytes) instead of complex T
template <typename T> size_t spread_tiles_smem(int nw, int mh, bool exact = false, int split = 1) {
    const size_t cell = exact ? 16 : sizeof(C<T>);
    return (size_t)nw * split * kSpreadTS * kSpreadTS * cell + (size_t)nw * (2 * mh) * kRecPitch * sizeof(C<T>) +
           (size_t)nw * spread_rpp(mh, split) * kRecPitch * spread_rec_bytes<T>(mh, split);
}

__device__ __forceinline__ void lds_ll2(unsigned ad, long long& a, long long& b) {
    asm volatile("ld.shared.v2.s64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(ad) : "memory");
}
__device__ __forceinline__ void sts_ll2(unsigned ad, long long a, long long b) {
    asm volatile("st.shared.v2.s64 [%0], {%1, %2};" ::"r"(ad), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ long long fixed_ll(float x) { return __float2ll_rn(x); }
__device__ __forceinline__ long long fixed_ll(double x) { return __double2ll_rn(x); }
template <typename T> __device__ __forceinline__ T fixed_back(long long x) {
    if constexpr (sizeof(T) == 4) return (T)__ll2float_rn(x);
    else return (T)__ll2double_rn(x);
}

__device__ __forceinline__ void lds_c(unsigned ad, C<float>& v) {
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(ad) : "memory");
}
__device__ __forceinline__ void lds_c(unsigned ad, C<double>& v) {
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(ad) : "memory");
}
__device__ __forceinline__ void sts_c(unsigned ad, const C<float>& v) {
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(ad), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void sts_c(unsigned ad, const C<double>& v) {
    asm volatile("st.shared.v2.f64 [%0], {%1, %2};" ::"r"(ad), "d"(v.x), "d"(v.y) : "memory");
}


// EXACT: the warp tiles hold 64-bit fixed-point cells (each product w v scaled
// by a power of two from a bound on the cell sums and rounded to an integer,
// as the atomic exact spread) and are added with integer read-add-writes: the
// exact sum of the rounded products, independent of order, without atomics.
// 16-byte cells need no swizzle: the 8 cells of a pass row span 128 bytes.
// SPLIT = 2: each half-warp takes every other record into a tile of its own
// (2 rows x 8 columns per pass for m = 4): the same shared-memory bytes per
// point with half the instructions; the two tiles per warp are summed at the end.
template <typename T, int NW, int MH, bool EXACT = false, int SPLIT = 1>
__device__ __forceinline__ void k_spread2d_tiles_body(const C<T>* __restrict__ in, C<T>* __restrict__ P, int j0, const Usfft2dArgs<T>& a, int bx, int by) {
    static_assert(SPLIT == 1 || !EXACT, "the exact tiles take one point per warp");
    constexpr int nt = 2 * MH;
    constexpr int LP = 32 / SPLIT;  // lanes per point
    constexpr int RPP = LP / nt;    // window rows per pass
    constexpr int NPASS = (nt + RPP - 1) / RPP;
    constexpr int TS = kSpreadTS;
    constexpr int ncell = TS * TS;
    constexpr unsigned kCell = EXACT ? 16u : (unsigned)sizeof(C<T>);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int hw = lane / LP, lp = lane - hw * LP;  // sub-warp and lane within it
    C<T>* tiles = reinterpret_cast<C<T>*>(smem_raw);  // [NW * SPLIT][ncell]
    C<T>* mine = tiles + (size_t)(warp * SPLIT + hw) * ncell;
    long long* xtiles = reinterpret_cast<long long*>(smem_raw);  // EXACT: [NW][ncell][2]
    long long* xmine = xtiles + (size_t)warp * ncell * 2;
    unsigned char* recb = smem_raw + (size_t)NW * SPLIT * ncell * kCell;
    T fscale = (T)1, finv = (T)1;
    if constexpr (EXACT) fixed_scale<T>(*a.maxabs, a.bound_count, fscale, finv);
    // records: wyv[sy][pitch] (complex), then rec[rr][pitch] (x weights of the
    // lane row's passes + window origin)
    typedef SpreadRec<T, NPASS> Rec;
    C<T>* r_wyv = reinterpret_cast<C<T>*>(recb) + (size_t)warp * nt * kRecPitch;
    Rec* r_rec = reinterpret_cast<Rec*>(recb + (size_t)NW * nt * kRecPitch * sizeof(C<T>)) +
                 (size_t)warp * RPP * kRecPitch;
    if (a.memo_hit && a.memo_hit[j0 + by]) return;  // served from the memoization cache (block-uniform)
    if constexpr (EXACT) {
        for (int i = lane; i < 2 * ncell; i += 32) xmine[i] = 0;
    } else {
        C<T>* wt = tiles + (size_t)warp * SPLIT * ncell;  // the warp's SPLIT tiles
        for (int i = lane; i < SPLIT * ncell; i += 32) wt[i] = cmake<T>(0, 0);
    }
    __syncwarp();
    const int tiles_y = a.M2 / TS;
    const int tile = bx;
    const int tx0 = (tile / tiles_y) * TS, ty0 = (tile % tiles_y) * TS;
    const int b = by;
    const int2 job = a.jobs[j0 + b];
    const T hb = (T)(TS + 2 * a.m) * (T)0.5;
    const int rr = lp / nt, sy = lp - rr * nt;
    const bool lane_on = rr < RPP;
    const int rrc = lane_on ? rr : 0;
    // lane-constant shared addresses of the record entries this lane reads
    const unsigned tile_ad = EXACT ? (unsigned)__cvta_generic_to_shared(xmine) : (unsigned)__cvta_generic_to_shared(mine);
    const unsigned wyv_ad = (unsigned)__cvta_generic_to_shared(r_wyv + sy * kRecPitch);
    const Rec* rec_lane = r_rec + (size_t)rrc * kRecPitch;
    const unsigned lt = (1u << lane) - 1u;
    // One pass over this plane's points.  For a paired job the mirror plane's
    // point (theta, -ku, -kv) sits at exactly the negated position of this
    // plane's point (theta, ku, kv), and the mirror plane lands in this grid
    // conjugated around -position: where the two tap windows mirror
    // (j0' = -j0 - 1 on both axes) its conj(value) joins this point's value in
    // one record.  Where a position lies within the tap shift of a grid node the
    // mirror window is this one shifted down by a cell; those mirror points get
    // records of their own (origin -j0' - m, fraction 1 - fr').  The point
    // ku = w/2 past each line's end (no value of its own) carries the mirror
    // plane's ku = -w/2 point.
    const bool paired = job.y >= 0;
    const int kv = job.x, kvc = kv - a.h / 2;
    // writes one record per lane with ok set (compacted in lane order) and adds
    // the records' windows into the warp's tile(s)
    auto emit = [&](bool ok, int ox, int oy, T fx, T fy, C<T> v) {
        const unsigned mask = __ballot_sync(0xffffffffu, ok);
        if (!mask) return;
        if (ok) {
            const int k = __popc(mask & lt);  // compacted record index
#pragma unroll
            for (int t = 0; t < nt; ++t) {
                const T dy = fy + (T)(MH - 1 - t);
                const T wy = gexp(-dy * dy * a.inv4beta);
                r_wyv[t * kRecPitch + k] = cmake<T>(wy * v.x, wy * v.y);
            }
#pragma unroll
            for (int r = 0; r < RPP; ++r) {
                Rec rc;
#pragma unroll
                for (int q = 0; q < NPASS; ++q) {
                    const int t = q * RPP + r;
                    const T dx = fx + (T)(MH - 1 - t);
                    rc.wx[q] = t < nt ? gexp(-dx * dx * a.inv4beta) : (T)0;
                }
                rc.ox = ox;
                rc.oy = oy;
                r_rec[r * kRecPitch + k] = rc;
            }
        }
        __syncwarp();
        const int cnt = __popc(mask);
        // sub-warp hw takes records hw, hw + SPLIT, ...; the value
        // records are complex T whatever the tile cells are
        constexpr unsigned kRecCell = sizeof(C<T>);
        const int k0 = hw < cnt ? hw : cnt - 1;
        Rec rc = rec_lane[k0];
        C<T> wv;
        lds_c(wyv_ad + k0 * kRecCell, wv);
        for (int kk = 0; kk < cnt; kk += SPLIT) {
            const int k = kk + hw;
            const bool kon = SPLIT == 1 || k < cnt;
            // read the next record first (its latency overlaps the update)
            const int kn = k + SPLIT < cnt ? k + SPLIT : (kon ? k : cnt - 1);
            const Rec nrc = rec_lane[kn];
            C<T> nwv;
            lds_c(wyv_ad + kn * kRecCell, nwv);
            const int2 o = make_int2(rc.ox, rc.oy);
            const int cx0 = o.x + rrc, ccy = o.y + sy;
            const int col = EXACT ? ccy : ccy ^ ((cx0 & 1) << 3);
            const unsigned ad0 = tile_ad + (unsigned)(cx0 * TS + col) * kCell;
            const bool yok = lane_on && (unsigned)ccy < (unsigned)TS;
#pragma unroll
            for (int q = 0; q < NPASS; ++q) {
                const int row = cx0 + q * RPP;
                // rows q * RPP apart: same swizzle when RPP is even
                const unsigned ad = (!EXACT && ((q * RPP) & 1))
                                        ? tile_ad + (unsigned)(row * TS + (col ^ 8)) * kCell
                                        : ad0 + (unsigned)(q * RPP * TS) * kCell;
                if (kon && yok && q * RPP + rr < nt && (unsigned)row < (unsigned)TS) {
                    if constexpr (EXACT) {
                        long long xr, xi;
                        lds_ll2(ad, xr, xi);
                        xr += fixed_ll(rc.wx[q] * wv.x * fscale);
                        xi += fixed_ll(rc.wx[q] * wv.y * fscale);
                        sts_ll2(ad, xr, xi);
                    } else {
                        C<T> acc;
                        lds_c(ad, acc);
                        acc.x = fma(rc.wx[q], wv.x, acc.x);
                        acc.y = fma(rc.wx[q], wv.y, acc.y);
                        sts_c(ad, acc);
                    }
                }
            }
            __syncwarp();
            rc = nrc;
            wv = nwv;
        }
    };
    for (int ix = -a.nimg; ix <= a.nimg; ++ix) {
        const int bx0 = tx0 + ix * a.M1;
        for (int iy = -a.nimg; iy <= a.nimg; ++iy) {
            const int by0 = ty0 + iy * a.M2;
            const T cx = (T)bx0 + (T)(TS - 1) * (T)0.5, cy = (T)by0 + (T)(TS - 1) * (T)0.5;
            if (sqrt(cx * cx + cy * cy) > a.rmax + hb * (T)1.5) continue;
            // positions whose window (or, paired, the mirror window one cell
            // below it) reaches the tile image
            const T bxl = (T)(bx0 - a.m), bxh = (T)(bx0 + TS + a.m - 1 + (paired ? 1 : 0));
            const T byl = (T)(by0 - a.m), byh = (T)(by0 + TS + a.m - 1 + (paired ? 1 : 0));
            for_tile_points<T, NW>(a, kvc, cx, cy, hb, bxl, bxh, byl, byh, warp, paired ? 1 : 0, [&](int th, int kuc) {
                bool ok = th >= 0;
                if (ok) ok = LAM_INB(th, a.T_, a.err, kSiteSpreadIn);
                const bool has_p = ok && kuc < a.w / 2;
                const bool has_q = ok && paired && kuc > -a.w / 2;
                int ox = 0, oy = 0, oxq = 0, oyq = 0;
                T fx = 0, fy = 0, fxq = 0, fyq = 0;
                C<T> v = cmake<T>(0, 0), vq = cmake<T>(0, 0);
                bool mir = true;
                if (ok) {
                    const typename AngleT<T>::type g = a.ang[th];
                    int jx, jy;
                    point_pos(g, kuc, kvc, jx, fx, jy, fy);
                    ox = jx - MH + 1 - bx0;
                    oy = jy - MH + 1 - by0;
                    if (has_p && LAM_INB(kuc + a.w / 2, a.w, a.err, kSiteSpreadIn))
                        v = in[((size_t)th * a.h + kv) * a.w + (kuc + a.w / 2)];
                    if (has_q && LAM_INB(a.w / 2 - kuc, a.w, a.err, kSiteSpreadIn)) {
                        int jxq, jyq;
                        point_pos(g, -kuc, -kvc, jxq, fxq, jyq, fyq);
                        mir = jxq == -jx - 1 && jyq == -jy - 1;
                        vq = in[((size_t)th * a.h + job.y) * a.w + (a.w / 2 - kuc)];
                        vq.y = -vq.y;
                        oxq = (-jxq - 1) - MH + 1 - bx0;
                        oyq = (-jyq - 1) - MH + 1 - by0;
                        fxq = (T)1 - fxq;
                        fyq = (T)1 - fyq;
                        if (mir) {
                            v.x += vq.x;
                            v.y += vq.y;
                        }
                    }
                }
                const bool ok_a = (has_p || (has_q && mir)) && !(ox <= -nt || ox >= TS || oy <= -nt || oy >= TS);
                emit(ok_a, ox, oy, fx, fy, v);
                const bool ok_b = has_q && !mir && !(oxq <= -nt || oxq >= TS || oyq <= -nt || oyq >= TS);
                if (__any_sync(0xffffffffu, ok_b)) emit(ok_b, oxq, oyq, fxq, fyq, vq);
            });
        }
    }
    __syncthreads();
    C<T>* pl = P + (size_t)b * a.M1 * a.M2;
    for (int i = threadIdx.x; i < ncell; i += blockDim.x) {
        const int ccx = i / TS, ccy = i - ccx * TS;
        C<T> sum;
        if constexpr (EXACT) {
            long long sr = xtiles[2 * i], si = xtiles[2 * i + 1];
#pragma unroll
            for (int w = 1; w < NW; ++w) {
                sr += xtiles[((size_t)w * ncell + i) * 2];
                si += xtiles[((size_t)w * ncell + i) * 2 + 1];
            }
            sum = cmake<T>(fixed_back<T>(sr) * finv, fixed_back<T>(si) * finv);
        } else {
            const int si = ccx * TS + swz_row(ccx, ccy);
            sum = tiles[si];
#pragma unroll
            for (int w = 1; w < NW * SPLIT; ++w) {
                const C<T> t = tiles[(size_t)w * ncell + si];
                sum.x += t.x;
                sum.y += t.y;
            }
        }
        pl[(size_t)(tx0 + ccx) * a.M2 + ty0 + ccy] = sum;
    }
}

// Owner-tile (halo) spread: every slice point is visited once, by the tile
// that holds its window origin.  Each warp sums into a private extended tile
// of (TS + 2m - 1)^2 cells (core + halo), so every window fits, all lanes are
// active and no bounds checks are needed; a row pitch of 8 (mod 16) cells
// keeps a 4-row x 8-column pass on 16 distinct bank pairs without a swizzle.
// The warp tiles are summed in a fixed order into H[b][tile]; k_halo_sum then
// adds the overlapping halos into the padded plane (fixed order as well).
__host__ __device__ constexpr int spread_halo_pitch(int mh) { return ((32 + 2 * mh - 1 + 7) / 16) * 16 + 8; }
template <typename T> size_t spread_halo_smem(int nw, int mh) {
    return (size_t)nw * (32 + 2 * mh - 1) * spread_halo_pitch(mh) * sizeof(C<T>) +
           (size_t)nw * (2 * mh) * kRecPitch * sizeof(C<T>) + (size_t)nw * spread_rpp(mh) * kRecPitch * spread_rec_bytes<T>(mh);
}

template <typename T, int NW, int MH>
__device__ __forceinline__ void k_spread2d_halo_body(const C<T>* __restrict__ in, C<T>* __restrict__ H, int j0, const Usfft2dArgs<T>& a, int bx, int by) {
    constexpr int nt = 2 * MH;
    constexpr int RPP = 32 / nt;  // window rows per pass
    constexpr int NPASS = (nt + RPP - 1) / RPP;
    constexpr int TS = kSpreadTS;
    constexpr int EXT = TS + nt - 1;        // core + halo rows / columns
    constexpr int PITCH = spread_halo_pitch(MH);
    constexpr int ncell = EXT * PITCH;
    constexpr unsigned kCell = sizeof(C<T>);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C<T>* tiles = reinterpret_cast<C<T>*>(smem_raw);  // [NW][ncell]
    C<T>* mine = tiles + (size_t)warp * ncell;
    unsigned char* recb = smem_raw + (size_t)NW * ncell * sizeof(C<T>);
    // records: wyv[sy][pitch] (complex), then rec[rr][pitch] (x weights of the
    // lane row's passes + window origin)
    typedef SpreadRec<T, NPASS> Rec;
    C<T>* r_wyv = reinterpret_cast<C<T>*>(recb) + (size_t)warp * nt * kRecPitch;
    Rec* r_rec = reinterpret_cast<Rec*>(recb + (size_t)NW * nt * kRecPitch * sizeof(C<T>)) +
                 (size_t)warp * RPP * kRecPitch;
    for (int i = lane; i < ncell; i += 32) mine[i] = cmake<T>(0, 0);
    __syncwarp();
    const int tiles_y = a.M2 / TS;
    const int tile = bx;
    const int tx0 = (tile / tiles_y) * TS, ty0 = (tile % tiles_y) * TS;
    const int b = by;
    const int2 job = a.jobs[j0 + b];
    const T hb = (T)TS * (T)0.5 + (T)1;
    const int rr = lane / nt, sy = lane - rr * nt;
    const bool lane_on = rr < RPP;
    const int rrc = lane_on ? rr : 0;
    // lane-constant shared addresses of the record entries this lane reads
    const unsigned tile_ad = (unsigned)__cvta_generic_to_shared(mine);
    const unsigned wyv_ad = (unsigned)__cvta_generic_to_shared(r_wyv + sy * kRecPitch);
    const Rec* rec_lane = r_rec + (size_t)rrc * kRecPitch;
    const unsigned lt = (1u << lane) - 1u;
    // pass 0: the job's own plane; pass 1: its mirror plane (conjugate values
    // spread around the negated positions, as in the atomic kernel)
    for (int pass = 0; pass < 2; ++pass) {
        const int kv = pass ? job.y : job.x;
        if (kv < 0) break;
        const int kvc = kv - a.h / 2;
        const T sg = pass ? (T)-1 : (T)1;
        for (int ix = -a.nimg; ix <= a.nimg; ++ix) {
            const int bx0 = tx0 + ix * a.M1;
            for (int iy = -a.nimg; iy <= a.nimg; ++iy) {
                const int by0 = ty0 + iy * a.M2;
                // positions whose window origin lies in the core [b0, b0 + TS)
                const T cx = (T)(bx0 + a.m - 1) + (T)TS * (T)0.5, cy = (T)(by0 + a.m - 1) + (T)TS * (T)0.5;
                if (sqrt(cx * cx + cy * cy) > a.rmax + hb * (T)1.5) continue;
                T bxl = (T)(bx0 + a.m - 1), bxh = (T)(bx0 + TS + a.m - 1);
                T byl = (T)(by0 + a.m - 1), byh = (T)(by0 + TS + a.m - 1);
                if (pass) {
                    const T t0 = -bxh, t1 = -bxl + (T)1, t2 = -byh, t3 = -byl + (T)1;
                    bxl = t0; bxh = t1; byl = t2; byh = t3;
                }
                for_tile_points<T, NW>(a, kvc, sg * cx, sg * cy, hb, bxl, bxh, byl, byh, warp, 0, [&](int th, int kuc) {
                    bool ok = th >= 0;
                    int ox = 0, oy = 0;
                    T fx = 0, fy = 0;
                    C<T> v = cmake<T>(0, 0);
                    if (ok)
                        ok = LAM_INB(kuc + a.w / 2, a.w, a.err, kSiteSpreadIn) && LAM_INB(th, a.T_, a.err, kSiteSpreadIn);
                    if (ok) {
                        const typename AngleT<T>::type g = a.ang[th];
                        int jx, jy;
                        point_pos(g, kuc, kvc, jx, fx, jy, fy);
                        v = in[((size_t)th * a.h + kv) * a.w + (kuc + a.w / 2)];
                        if (pass) {
                            jx = -jx - 1;
                            jy = -jy - 1;
                            fx = (T)1 - fx;
                            fy = (T)1 - fy;
                            v.y = -v.y;
                        }
                        ox = jx - MH + 1 - bx0;
                        oy = jy - MH + 1 - by0;
                        ok = ox >= 0 && ox < TS && oy >= 0 && oy < TS;
                    }
                    const unsigned mask = __ballot_sync(0xffffffffu, ok);
                    if (!mask) return;
                    if (ok) {
                        const int k = __popc(mask & lt);  // compacted record index
#pragma unroll
                        for (int t = 0; t < nt; ++t) {
                            const T dy = fy + (T)(MH - 1 - t);
                            const T wy = gexp(-dy * dy * a.inv4beta);
                            r_wyv[t * kRecPitch + k] = cmake<T>(wy * v.x, wy * v.y);
                        }
#pragma unroll
                        for (int r = 0; r < RPP; ++r) {
                            Rec rc;
#pragma unroll
                            for (int q = 0; q < NPASS; ++q) {
                                const int t = q * RPP + r;
                                const T dx = fx + (T)(MH - 1 - t);
                                rc.wx[q] = t < nt ? gexp(-dx * dx * a.inv4beta) : (T)0;
                            }
                            rc.ox = ox;
                            rc.oy = oy;
                            r_rec[r * kRecPitch + k] = rc;
                        }
                    }
                    __syncwarp();
                    const int cnt = __popc(mask);
                    Rec rc = rec_lane[0];
                    C<T> wv;
                    lds_c(wyv_ad, wv);
                    for (int k = 0; k < cnt; ++k) {
                        // read the next record first (its latency overlaps the update)
                        const int kn = k + 1 < cnt ? k + 1 : k;
                        const Rec nrc = rec_lane[kn];
                        C<T> nwv;
                        lds_c(wyv_ad + kn * kCell, nwv);
                        const int2 o = make_int2(rc.ox, rc.oy);
                        // the window lies inside the extended tile: no bounds checks
                        const unsigned ad0 = tile_ad + (unsigned)((o.x + rrc) * PITCH + o.y + sy) * kCell;
#pragma unroll
                        for (int q = 0; q < NPASS; ++q) {
                            const unsigned ad = ad0 + (unsigned)(q * RPP * PITCH) * kCell;
                            if (lane_on && q * RPP + rr < nt) {
                                C<T> acc;
                                lds_c(ad, acc);
                                acc.x = fma(rc.wx[q], wv.x, acc.x);
                                acc.y = fma(rc.wx[q], wv.y, acc.y);
                                sts_c(ad, acc);
                            }
                        }
                        __syncwarp();
                        rc = nrc;
                        wv = nwv;
                    }
                });
            }
        }
    }
    __syncthreads();
    // the extended tile (core + halo) of this job's plane: H[b][tile][EXT][EXT]
    const int ntiles = (a.M1 / TS) * tiles_y;
    C<T>* ht = H + ((size_t)b * ntiles + tile) * EXT * EXT;
    for (int i = threadIdx.x; i < EXT * EXT; i += blockDim.x) {
        const int r = i / EXT, c = i - r * EXT;
        const int si = r * PITCH + c;
        C<T> sum = tiles[si];
#pragma unroll
        for (int w = 1; w < NW; ++w) {
            const C<T> t = tiles[(size_t)w * ncell + si];
            sum.x += t.x;
            sum.y += t.y;
        }
        ht[i] = sum;
    }
}

template <typename T, int NW, int MH>
__global__ void __launch_bounds__(NW * 32, sizeof(T) == 4 ? 3 : 2) k_spread2d_halo(
    const C<T>* __restrict__ in, C<T>* __restrict__ H, int j0, Usfft2dArgs<T> a) {
    k_spread2d_halo_body<T, NW, MH>(in, H, j0, a, (int)blockIdx.x, (int)blockIdx.y);
}

// P[b][x][y] = the core cell of tile (x / TS, y / TS) plus the halo cells of the
// tiles before it in x, in y and in both (periodic), added in that order
template <typename T>
__global__ void __launch_bounds__(256) k_halo_sum(const C<T>* __restrict__ H, C<T>* __restrict__ P, int nb,
                                                 int ext, Usfft2dArgs<T> a) {
    constexpr int TS = kSpreadTS;
    const int tx_n = a.M1 / TS, ty_n = a.M2 / TS, ntiles = tx_n * ty_n;
    const int hw = ext - TS;
    const long long n = (long long)nb * a.M1 * a.M2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long bp = i / ((long long)a.M1 * a.M2);
        const int rem = (int)(i - bp * a.M1 * a.M2);
        const int x = rem / a.M2, y = rem - x * a.M2;
        const int tx = x / TS, dx = x - tx * TS, ty = y / TS, dy = y - ty * TS;
        const int txm = tx == 0 ? tx_n - 1 : tx - 1, tym = ty == 0 ? ty_n - 1 : ty - 1;
        const C<T>* hb = H + (size_t)bp * ntiles * ext * ext;
        C<T> s = hb[((size_t)(tx * ty_n + ty) * ext + dx) * ext + dy];
        if (dx < hw) {
            const C<T> t = hb[((size_t)(txm * ty_n + ty) * ext + dx + TS) * ext + dy];
            s.x += t.x;
            s.y += t.y;
        }
        if (dy < hw) {
            const C<T> t = hb[((size_t)(tx * ty_n + tym) * ext + dx) * ext + dy + TS];
            s.x += t.x;
            s.y += t.y;
        }
        if (dx < hw && dy < hw) {
            const C<T> t = hb[((size_t)(txm * ty_n + tym) * ext + dx + TS) * ext + dy + TS];
            s.x += t.x;
            s.y += t.y;
        }
        P[i] = s;
    }
}

template <typename T, int NW, int MH>
__global__ void __launch_bounds__(NW * 32, sizeof(T) == 4 ? 4 : 2) k_spread2d_tiles(
    const C<T>* __restrict__ in, C<T>* __restrict__ P, int j0, Usfft2dArgs<T> a) {
    k_spread2d_tiles_body<T, NW, MH, false>(in, P, j0, a, (int)blockIdx.x, (int)blockIdx.y);
}

// the tile spread with one point per half-warp
template <typename T, int NW, int MH>
__global__ void __launch_bounds__(NW * 32, sizeof(T) == 4 ? 4 : 2) k_spread2d_tiles2(
    const C<T>* __restrict__ in, C<T>* __restrict__ P, int j0, Usfft2dArgs<T> a) {
    k_spread2d_tiles_body<T, NW, MH, false, 2>(in, P, j0, a, (int)blockIdx.x, (int)blockIdx.y);
}

// the exact (64-bit fixed-point) tile spread
template <typename T, int NW, int MH>
__global__ void __launch_bounds__(NW * 32, sizeof(T) == 4 ? 4 : 2) k_spread2d_tiles_exact(
    const C<T>* __restrict__ in, C<T>* __restrict__ P, int j0, Usfft2dArgs<T> a) {
    k_spread2d_tiles_body<T, NW, MH, true>(in, P, j0, a, (int)blockIdx.x, (int)blockIdx.y);
}

// ---------------------------------------------------------------------------
// Row-sweep spread (LAM_SPREAD_SWEEP): the window sums stay in registers; no
// shared-memory read-add-write per tap.
//
// One block of kSweepWarps = 4 warps per kSweepX x kSweepY tile (x rows by y
// cells; y is the contiguous axis of the padded plane) of one plane job; warp
// w owns the band of y cells [8w, 8w + 8).  For every pass (plane, mirror
// plane) and periodic image the block lists the slice lines that cross the
// tile's box (warp w tests the angles th = w mod 4, in order); each warp then
// clips the listed lines against its band's box and walks their points,
// writing one record per point whose window meets the band: the value, the
// y fraction, the nt x weights and the window's origin.  A record's key is
// its window's x origin; its rank within the key (match-any groups, in
// walking order) makes the bucketing a stable counting sort.  When the
// warp's records fill its buffer (and at the end) it sorts them by key and
// sweeps the rows: lane 8q + l owns y cell 8w + l and holds the nt window
// rows of its current origin as nt complex registers; quarter q takes the
// q-th quarter of the sorted records, so the four quarters cover disjoint,
// increasing origin ranges.  Moving on to a larger origin, a quarter adds
// the rows it leaves into the shared tile (no other quarter touches those
// rows during the sweep); the rows each quarter holds at the end are added
// quarter by quarter.  The order of every sum follows from the input alone,
// so the result is bitwise reproducible.
// ---------------------------------------------------------------------------
#ifndef LAM_SWEEP_CAP
#define LAM_SWEEP_CAP 128  // FP32 records per warp buffer (FP64: half)
#endif
#ifndef LAM_SWEEP_MINB
#define LAM_SWEEP_MINB 4  // FP32 blocks per SM the registers are sized for
#endif
constexpr int kSweepX = 64, kSweepY = 32, kSweepWarps = kSweepY / 8, kSweepCap = LAM_SWEEP_CAP;
template <typename T> __host__ __device__ constexpr int sweep_cap() { return sizeof(T) == 4 ? kSweepCap : kSweepCap / 2; }
// bucket counters per warp: window x origins -(nt - 1) .. kSweepX - 1, padded to a multiple of 32
__host__ __device__ constexpr int sweep_keys(int mh) { return (kSweepX + 2 * mh - 1 + 31) / 32 * 32; }
__host__ __device__ constexpr int sweep_line_pitch(int nang) {
    return ((nang + kSweepWarps - 1) / kSweepWarps + 31) / 32 * 32;
}

// a point record: value, y fraction, pk = key | (y origin in the band + 16) << 8 | rank << 16, x weights
template <typename T, int NT> struct alignas(16) SweepRec {
    T vx, vy, fy;
    int pk;
    T wx[NT];
};
template <typename T> size_t sweep_rec_bytes(int mh) {
    switch (mh) {
        case 2: return sizeof(SweepRec<T, 4>);
        case 3: return sizeof(SweepRec<T, 6>);
        case 4: return sizeof(SweepRec<T, 8>);
        case 5: return sizeof(SweepRec<T, 10>);
        case 6: return sizeof(SweepRec<T, 12>);
        case 7: return sizeof(SweepRec<T, 14>);
        default: return sizeof(SweepRec<T, 16>);
    }
}
template <typename T> size_t spread_sweep_smem(int mh, int nang) {
    return (size_t)kSweepX * kSweepY * sizeof(C<T>) +
           (size_t)kSweepWarps * sweep_cap<T>() * (sweep_rec_bytes<T>(mh) + sizeof(unsigned short)) +
           (size_t)kSweepWarps * sweep_keys(mh) * sizeof(int) + (size_t)kSweepWarps * sweep_line_pitch(nang) * sizeof(int);
}

template <int NT>
__device__ __forceinline__ void sweep_load(const SweepRec<float, NT>* r, float& vx, float& vy, float& fy, int& pk,
                                           float (&w)[NT]) {
    const float4 h = *reinterpret_cast<const float4*>(r);
    vx = h.x;
    vy = h.y;
    fy = h.z;
    pk = __float_as_int(h.w);
    if constexpr (NT % 4 == 0) {
#pragma unroll
        for (int k = 0; k < NT / 4; ++k) {
            const float4 t = reinterpret_cast<const float4*>(r->wx)[k];
            w[4 * k] = t.x;
            w[4 * k + 1] = t.y;
            w[4 * k + 2] = t.z;
            w[4 * k + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int t = 0; t < NT; ++t) w[t] = r->wx[t];
    }
}
template <int NT>
__device__ __forceinline__ void sweep_load(const SweepRec<double, NT>* r, double& vx, double& vy, double& fy, int& pk,
                                           double (&w)[NT]) {
    const double2 h = *reinterpret_cast<const double2*>(r);
    vx = h.x;
    vy = h.y;
    fy = r->fy;
    pk = r->pk;
#pragma unroll
    for (int k = 0; k < NT / 2; ++k) {
        const double2 t = reinterpret_cast<const double2*>(r->wx)[k];
        w[2 * k] = t.x;
        w[2 * k + 1] = t.y;
    }
}

template <typename T, int MH>
__global__ void __launch_bounds__(kSweepWarps * 32, sizeof(T) == 4 ? LAM_SWEEP_MINB : 1) k_spread2d_sweep(
    const C<T>* __restrict__ in, C<T>* __restrict__ P, int j0, Usfft2dArgs<T> a) {
    constexpr int NT = 2 * MH, SX = kSweepX, SY = kSweepY, CAP = sweep_cap<T>(), NKP = sweep_keys(MH);
    static_assert(NT <= 16 && SX + NT - 1 < 256, "key and y origin fields of the record");
    typedef SweepRec<T, NT> Rec;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_nl[kSweepWarps];
    if (a.memo_hit && a.memo_hit[j0 + blockIdx.y]) return;  // served from the memoization cache (block-uniform)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = lane >> 3, l8 = lane & 7;
    const unsigned lt = (1u << lane) - 1u;
    const int lp = sweep_line_pitch(a.T_);
    C<T>* tile = reinterpret_cast<C<T>*>(smem_raw);  // [SX][SY]
    unsigned char* sp = smem_raw + (size_t)SX * SY * sizeof(C<T>);
    Rec* recs = reinterpret_cast<Rec*>(sp) + (size_t)warp * CAP;
    sp += (size_t)kSweepWarps * CAP * sizeof(Rec);
    unsigned short* ent = reinterpret_cast<unsigned short*>(sp) + (size_t)warp * CAP;
    sp += (size_t)kSweepWarps * CAP * sizeof(unsigned short);
    int* cnt = reinterpret_cast<int*>(sp) + (size_t)warp * NKP;
    sp += (size_t)kSweepWarps * NKP * sizeof(int);
    int* lines = reinterpret_cast<int*>(sp);  // [kSweepWarps][lp]
    for (int i = threadIdx.x; i < SX * SY; i += blockDim.x) tile[i] = cmake<T>(0, 0);
    for (int i = lane; i < NKP; i += 32) cnt[i] = 0;
    __syncthreads();
    // edge tiles may reach past the plane (sides not multiples of the tile):
    // their outside cells are summed like the others and not written
    const int tiles_y = (a.M2 + SY - 1) / SY;
    const int tx0 = ((int)blockIdx.x / tiles_y) * SX, ty0 = ((int)blockIdx.x % tiles_y) * SY;
    const int2 job = a.jobs[j0 + blockIdx.y];
    const int ycell = warp * 8 + l8;
    int nrec = 0;  // warp-uniform

    // adds a held window row (key row = x origin + nt - 1) into the tile if it lies inside
    auto put = [&](int row, T x, T y) {
        const int xr = row - (NT - 1);
        if ((unsigned)xr < (unsigned)SX) {
            C<T>& c = tile[xr * SY + ycell];
            c.x += x;
            c.y += y;
        }
    };
    // sort the warp's records by key and sweep them into the tile
    auto process = [&]() {
        constexpr int PER = NKP / 32;
        int cv[PER], s = 0;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            cv[k] = cnt[lane * PER + k];
            s += cv[k];
        }
        int incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        int run = incl - s;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            cnt[lane * PER + k] = run;
            run += cv[k];
        }
        __syncwarp();
        for (int i = lane; i < nrec; i += 32) {
            const int pk = recs[i].pk;
            ent[cnt[pk & 0xff] + (pk >> 16)] = (unsigned short)i;
        }
        __syncwarp();
        const int e0 = (nrec * q) >> 2, e1 = (nrec * (q + 1)) >> 2;
        const int iters = (nrec + 3) >> 2;
        T ax[NT], ay[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) ax[t] = ay[t] = (T)0;
        int cur = e0 < e1 ? (recs[ent[e0]].pk & 0xff) : 0;
        // the quarter's current record; the next one is read while it is applied
        T vx = 0, vy = 0, fy = 0, w[NT];
        int pk = 0;
        if (e0 < e1) sweep_load<NT>(recs + ent[e0], vx, vy, fy, pk, w);
        for (int it = 0; it < iters; ++it) {
            const int e = e0 + it;
            if (e < e1) {
                T nvx, nvy, nfy, nw[NT];
                int npk;
                sweep_load<NT>(recs + ent[e + 1 < e1 ? e + 1 : e], nvx, nvy, nfy, npk, nw);
                const int key = pk & 0xff;
                while (cur < key) {
                    if (key - cur >= NT) {
#pragma unroll
                        for (int t = 0; t < NT; ++t) {
                            put(cur + t, ax[t], ay[t]);
                            ax[t] = ay[t] = (T)0;
                        }
                        cur = key;
                    } else {
                        put(cur, ax[0], ay[0]);
#pragma unroll
                        for (int t = 0; t < NT - 1; ++t) {
                            ax[t] = ax[t + 1];
                            ay[t] = ay[t + 1];
                        }
                        ax[NT - 1] = ay[NT - 1] = (T)0;
                        ++cur;
                    }
                }
                const int dyl = l8 - (((pk >> 8) & 0xff) - 16);
                T wy = (T)0;
                if ((unsigned)dyl < (unsigned)NT) {
                    const T d = fy + (T)(MH - 1 - dyl);
                    wy = gexp(-d * d * a.inv4beta);
                }
                const T px = wy * vx, py = wy * vy;
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    ax[t] = fma(px, w[t], ax[t]);
                    ay[t] = fma(py, w[t], ay[t]);
                }
                vx = nvx;
                vy = nvy;
                fy = nfy;
                pk = npk;
#pragma unroll
                for (int t = 0; t < NT; ++t) w[t] = nw[t];
            }
        }
        __syncwarp();
        for (int qq = 0; qq < 4; ++qq) {
            if (q == qq && e0 < e1) {
#pragma unroll
                for (int t = 0; t < NT; ++t) put(cur + t, ax[t], ay[t]);
            }
            __syncwarp();
        }
        for (int i = lane; i < NKP; i += 32) cnt[i] = 0;
        __syncwarp();
        nrec = 0;
    };

    const int kmin = -a.w / 2, kmax = a.w / 2 - 1;
    const T hx = (T)(SX + 2 * a.m) * (T)0.5, hy = (T)(SY + 2 * a.m) * (T)0.5;
    // pass 0: the job's own plane; pass 1: its mirror plane (conjugate values
    // spread around the negated positions)
    for (int pass = 0; pass < 2; ++pass) {
        const int kv = pass ? job.y : job.x;
        if (kv < 0) break;
        const int kvc = kv - a.h / 2;
        const T sg = pass ? (T)-1 : (T)1;
        for (int ix = -a.nimg; ix <= a.nimg; ++ix) {
            const int bx0 = tx0 + ix * a.M1;
            for (int iy = -a.nimg; iy <= a.nimg; ++iy) {
                const int by0 = ty0 + iy * a.M2;
                const T cx = (T)bx0 + (T)(SX - 1) * (T)0.5, cy = (T)by0 + (T)(SY - 1) * (T)0.5;
                if (sqrt(cx * cx + cy * cy) > a.rmax + hx + hy) continue;  // block-uniform
                // list the lines crossing the tile's box (distance test against its support)
                int n = 0;  // warp-uniform
                for (int base = 0; base * kSweepWarps < a.T_; base += 32) {
                    const int th = (base + lane) * kSweepWarps + warp;
                    bool cross = false;
                    if (th < a.T_) {
                        const typename AngleT<T>::type g = a.ang[th];
                        T Ax, Cx, Ay, Cy;
                        line_coef(g, kvc, Ax, Cx, Ay, Cy);
                        const T nrm = sqrt(Ax * Ax + Ay * Ay);
                        const T nx = -Ay / nrm, ny = Ax / nrm;
                        const T dist = fabs((sg * cx - Cx) * nx + (sg * cy - Cy) * ny);
                        cross = dist <= hx * fabs(nx) + hy * fabs(ny) + (T)1;
                    }
                    const unsigned mk = __ballot_sync(0xffffffffu, cross);
                    if (cross) lines[warp * lp + n + __popc(mk & lt)] = th;
                    n += __popc(mk);
                }
                if (lane == 0) s_nl[warp] = n;
                __syncthreads();
                // the warp's band box in this pass's positions
                T bxl = (T)(bx0 - a.m), bxh = (T)(bx0 + SX + a.m - 1);
                T byl = (T)(by0 + 8 * warp - a.m), byh = (T)(by0 + 8 * warp + 8 + a.m - 1);
                if (pass) {
                    const T t0 = -bxh, t1 = -bxl + (T)1, t2 = -byh, t3 = -byl + (T)1;
                    bxl = t0; bxh = t1; byl = t2; byh = t3;
                }
                for (int lw = 0; lw < kSweepWarps; ++lw) {
                    const int nl = s_nl[lw];
                    for (int c0 = 0; c0 < nl; c0 += 32) {
                        const int th = c0 + lane < nl ? lines[lw * lp + c0 + lane] : -1;
                        int lo = 1, hi = 0;
                        if (th >= 0) {
                            const typename AngleT<T>::type g = a.ang[th];
                            T Ax, Cx, Ay, Cy;
                            line_coef(g, kvc, Ax, Cx, Ay, Cy);
                            lo = kmin;
                            hi = kmax;
                            clip_line<T>(Ax, Cx, bxl, bxh, lo, hi);
                            clip_line<T>(Ay, Cy, byl, byh, lo, hi);
                        }
                        walk_line_points(th, lo, hi, [&](int tp, int kuc) {
                            bool ok = tp >= 0;
                            int ox = 0, oyb = 0;
                            T fx = 0, fy = 0;
                            C<T> v = cmake<T>(0, 0);
                            if (ok)
                                ok = LAM_INB(kuc + a.w / 2, a.w, a.err, kSiteSpreadIn) && LAM_INB(tp, a.T_, a.err, kSiteSpreadIn);
                            if (ok) {
                                const typename AngleT<T>::type g = a.ang[tp];
                                int jx, jy;
                                point_pos(g, kuc, kvc, jx, fx, jy, fy);
                                v = in[((size_t)tp * a.h + kv) * a.w + (kuc + a.w / 2)];
                                if (pass) {
                                    jx = -jx - 1;
                                    jy = -jy - 1;
                                    fx = (T)1 - fx;
                                    fy = (T)1 - fy;
                                    v.y = -v.y;
                                }
                                ox = jx - MH + 1 - bx0;
                                oyb = jy - MH + 1 - by0 - 8 * warp;
                                ok = ox > -NT && ox < SX && oyb > -NT && oyb < 8;
                            }
                            const unsigned mk = __ballot_sync(0xffffffffu, ok);
                            if (!mk) return;
                            const int c = __popc(mk);
                            if (nrec + c > CAP) process();
                            const int key = ox + NT - 1;
                            const unsigned peers = __match_any_sync(0xffffffffu, ok ? key : -1);
                            int rank = 0;
                            if (ok) rank = cnt[key] + __popc(peers & lt);
                            __syncwarp();
                            // the group's lowest lane moves the key's count past the group
                            if (ok && !(peers & lt)) cnt[key] = rank + __popc(peers);
                            if (ok) {
                                Rec* r = recs + nrec + __popc(mk & lt);
                                r->vx = v.x;
                                r->vy = v.y;
                                r->fy = fy;
                                r->pk = key | ((oyb + 16) << 8) | (rank << 16);
#pragma unroll
                                for (int t = 0; t < NT; ++t) {
                                    const T d = fx + (T)(MH - 1 - t);
                                    r->wx[t] = gexp(-d * d * a.inv4beta);
                                }
                            }
                            nrec += c;
                            __syncwarp();
                        });
                    }
                }
                __syncthreads();  // the line lists are rewritten for the next image
            }
        }
    }
    if (nrec > 0) process();
    __syncthreads();
    C<T>* pl = P + (size_t)blockIdx.y * a.M1 * a.M2;
    for (int i = threadIdx.x; i < SX * SY; i += blockDim.x) {
        const int x = i / SY, y = i - x * SY;
        if (tx0 + x < a.M1 && ty0 + y < a.M2) pl[(size_t)(tx0 + x) * a.M2 + ty0 + y] = tile[i];
    }
}

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------

// warps per tile-block in the gather and the scatter (16 measured slower)
constexpr int kScatterWarps = 4;
// warps per block of the tiled gather (they share the block's staged tile)
constexpr int kGatherWarps = 4;
// warps per block of the tile spread (each with its private 32 x 32 tile):
// 2 measured fastest (1024^3 L-hat^H: 145 ms against 153 with 3, 154 with 4
// and 151 with 1); the warps of a tile split its slice lines, and fewer warps
// per tile leave less of them idle at the tile's end
constexpr int kSpreadWarps = 2;

// The FP32 row / column FFT kernels are also built for the power-of-two plane
// lengths 2n of the large workloads, with the length a compile-time constant
// (bitwise the same results); other lengths and FP64 take the runtime-length
// kernels.  CALL(NC) launches the NC instantiation.
#define LAM_PLANE_NC(len, CALL)             \
    do {                                    \
        if constexpr (sizeof(T) == 4) {     \
            switch (len) {                  \
                case 512: CALL(512); break;   \
                case 1024: CALL(1024); break; \
                case 2048: CALL(2048); break; \
                case 4096: CALL(4096); break; \
                default: CALL(0); break;      \
            }                               \
        } else {                            \
            CALL(0);                        \
        }                                   \
    } while (0)
#define LAM_RF(NC) k_rowfft_fwd<T, false, NC><<<dim3(a.n1 / a.RB, nb), a.fthr, sr, s>>>(u1, P, kv0, a)
#define LAM_CF(NC) k_colfft_fwd_pipe<T, false, NC><<<gp, a.fthr, 2 * sc, s>>>(P, a, nb)
#define LAM_CA(NC) k_colfft_adj_pipe<T, false, NC><<<gp, a.fthr, 2 * sc, s>>>(P, a, nb, kv0)
#define LAM_RA(NC) k_rowfft_adj<T, false, NC><<<dim3(a.n1 / a.RB, nb), a.fthr, sr, s>>>(P, u1, kv0, a)

template <typename T>
cudaError_t launch_usfft2d_fwd(const C<T>* u1, C<T>* P, C<T>* out, const C<T>* sub, int j0, int nb,
                               const Usfft2dArgs<T>& a, cudaStream_t s) {
    const int kv0 = j0;
    const size_t sr = (size_t)a.RB * fpad_len(a.M2) * sizeof(C<T>);
    const size_t sc = (size_t)a.CB * fpad_len(a.M1) * sizeof(C<T>);
    const int gp = pipe_grid((a.M2 / a.CB) * nb, a.fthr, 2 * sc);
    if (fft_mixed(a.fcM1) || fft_mixed(a.fcM2)) {
        k_rowfft_fwd<T, true><<<dim3(a.n1 / a.RB, nb), a.fthr, sr, s>>>(u1, P, kv0, a);
        k_colfft_fwd_pipe<T, true><<<gp, a.fthr, 2 * sc, s>>>(P, a, nb);
    } else {
        LAM_PLANE_NC(a.M2, LAM_RF);
        LAM_PLANE_NC(a.M1, LAM_CF);
    }
    constexpr int NW = kGatherWarps;
    const int ntiles = (a.M1 / a.TG) * (a.M2 / a.TG);
    const size_t sg = gather_smem_bytes<T>(a.TG, a.m);
    const dim3 grid(ntiles, nb);
    switch (a.m) {
#define LAM_G(MH) case MH: k_gather2d_tiled<T, NW, MH><<<grid, NW * 32, sg, s>>>(P, out, sub, kv0, a); break;
        LAM_G(2) LAM_G(3) LAM_G(4) LAM_G(5) LAM_G(6) LAM_G(7) LAM_G(8)
#undef LAM_G
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// the plane FFTs of the forward alone (deapodise, pad, row and column FFTs of
// planes j0 .. j0 + nb - 1 into P), for timing against library FFTs
template <typename T>
cudaError_t launch_usfft2d_planes(const C<T>* u1, C<T>* P, int j0, int nb, const Usfft2dArgs<T>& a, cudaStream_t s) {
    const size_t sr = (size_t)a.RB * fpad_len(a.M2) * sizeof(C<T>);
    const size_t sc = (size_t)a.CB * fpad_len(a.M1) * sizeof(C<T>);
    const int gp = pipe_grid((a.M2 / a.CB) * nb, a.fthr, 2 * sc);
    const int kv0 = j0;
    if (fft_mixed(a.fcM1) || fft_mixed(a.fcM2)) {
        k_rowfft_fwd<T, true><<<dim3(a.n1 / a.RB, nb), a.fthr, sr, s>>>(u1, P, kv0, a);
        k_colfft_fwd_pipe<T, true><<<gp, a.fthr, 2 * sc, s>>>(P, a, nb);
    } else {
        LAM_PLANE_NC(a.M2, LAM_RF);
        LAM_PLANE_NC(a.M1, LAM_CF);
    }
    return cudaGetLastError();
}

// FP32 FMA throughput probe: eight independent FMA chains per thread
__global__ void __launch_bounds__(256) k_fma_peak(float* sink, int iters, float a, float b) {
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
    }
    float t = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += x[k];
    if (t == 1.2345f) sink[blockIdx.x] = t;  // never true: keeps the chains live
}

cudaError_t launch_fma_peak(float* sink, int blocks, int iters, cudaStream_t s) {
    k_fma_peak<<<blocks, 256, 0, s>>>(sink, iters, 0.99999994f, 1e-7f);
    return cudaGetLastError();
}

// Self-test of the index checks: one checked write of 1 at scratch[index],
// scratch holding kSelftestCells ints.  An index outside the scratch is caught
// by the check (the site is recorded, the write skipped), never performed.
__global__ void k_bounds_selftest(int* scratch, int index, int* err) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (LAM_INB(index, kSelftestCells, err, kSiteSelftest)) scratch[index] = 1;
}

cudaError_t launch_bounds_selftest(int* scratch, int index, int* err, cudaStream_t s) {
    k_bounds_selftest<<<1, 32, 0, s>>>(scratch, index, err);
    return cudaGetLastError();
}

// the adjoint spread alone: slice values of plane jobs j0 .. j0 + nb - 1 onto
// their padded planes P[0 .. nb) (the spread variant a.spread selects)
template <typename T>
cudaError_t launch_spread2d(const C<T>* in, C<T>* P, int j0, int nb, const Usfft2dArgs<T>& a, cudaStream_t s) {
    const int kv0 = j0;
    constexpr int NW = kScatterWarps;
    const int ntiles = (a.M1 / a.TS) * (a.M2 / a.TS);
    // exact fixed-point accumulation (default) or plain atomic adds
    const size_t cells = (size_t)a.TS * a.TS;
    const dim3 grid1(ntiles, nb);
#define LAM_S(MH, ACC)                                                                                   \
    case MH:                                                                                             \
        k_scatter2d_atomic<T, NW, MH, ACC><<<grid1, NW * 32, cells * atom_acc_bytes<T, ACC>(), s>>>(in, P, \
                                                                                                kv0, a); \
        break;
#define LAM_SW(ACC)                                                                              \
    switch (a.m) {                                                                               \
        LAM_S(2, ACC) LAM_S(3, ACC) LAM_S(4, ACC) LAM_S(5, ACC) LAM_S(6, ACC) LAM_S(7, ACC) LAM_S(8, ACC) \
        default: return cudaErrorInvalidValue;                                                   \
    }
    // the tile and halo spreads are built for 32 x 32 tiles; planes smaller
    // than that (n < 16) take the exact atomic spread
    if (a.spread == kSpreadTilesExact && a.TS == kSpreadTS && a.maxabs) {
        const size_t sx = spread_tiles_smem<T>(kSpreadWarps, a.m, true);
        switch (a.m) {
#define LAM_X(MH) case MH: k_spread2d_tiles_exact<T, kSpreadWarps, MH><<<grid1, kSpreadWarps * 32, sx, s>>>(in, P, kv0, a); break;
            LAM_X(2) LAM_X(3) LAM_X(4) LAM_X(5) LAM_X(6) LAM_X(7) LAM_X(8)
#undef LAM_X
            default: return cudaErrorInvalidValue;
        }
    } else if (a.spread == kSpreadHalo && a.TS == kSpreadTS && a.halo) {
        const size_t st = spread_halo_smem<T>(NW, a.m);
        switch (a.m) {
#define LAM_H(MH) case MH: k_spread2d_halo<T, NW, MH><<<grid1, NW * 32, st, s>>>(in, a.halo, kv0, a); break;
            LAM_H(2) LAM_H(3) LAM_H(4) LAM_H(5) LAM_H(6) LAM_H(7) LAM_H(8)
#undef LAM_H
            default: return cudaErrorInvalidValue;
        }
        const long long ncells = (long long)nb * a.M1 * a.M2;
        const long long hb = (ncells + 255) / 256;
        k_halo_sum<T><<<(int)(hb < 148 * 8 ? hb : 148 * 8), 256, 0, s>>>(a.halo, P, nb, kSpreadTS + 2 * a.m - 1, a);
    } else if ((a.spread == kSpreadTiles || a.spread == kSpreadTiles2 || a.spread == kSpreadHalo ||
                a.spread == kSpreadSweep) && a.TS == kSpreadTS) {
        // the first a.nacc plane jobs (the centre planes: every slice line
        // passes close to the origin there, so the cells near it sum thousands
        // of nearly equal products, where FP32 running sums round
        // systematically) take the exact fixed-point accumulation; the others
        // the tile spread
        const int nx = a.maxabs ? std::max(0, std::min(nb, a.nacc - j0)) : 0;
        if (nx > 0) {
            const dim3 gx(ntiles, nx);
            const size_t sx = spread_tiles_smem<T>(kSpreadWarps, a.m, true);
            switch (a.m) {
#define LAM_X(MH) case MH: k_spread2d_tiles_exact<T, kSpreadWarps, MH><<<gx, kSpreadWarps * 32, sx, s>>>(in, P, kv0, a); break;
                LAM_X(2) LAM_X(3) LAM_X(4) LAM_X(5) LAM_X(6) LAM_X(7) LAM_X(8)
#undef LAM_X
                default: return cudaErrorInvalidValue;
            }
        }
        if (nb > nx) {
            const dim3 gt(ntiles, nb - nx);
            C<T>* Pt = P + (size_t)nx * a.M1 * a.M2;
            const size_t sw = spread_sweep_smem<T>(a.m, a.T_);
            if (a.spread == kSpreadSweep && sw <= (size_t)kMaxDynSmem - 1024) {
                const dim3 gw(((a.M1 + kSweepX - 1) / kSweepX) * ((a.M2 + kSweepY - 1) / kSweepY), nb - nx);
                switch (a.m) {
#define LAM_W(MH) case MH: k_spread2d_sweep<T, MH><<<gw, kSweepWarps * 32, sw, s>>>(in, Pt, kv0 + nx, a); break;
                    LAM_W(2) LAM_W(3) LAM_W(4) LAM_W(5) LAM_W(6) LAM_W(7) LAM_W(8)
#undef LAM_W
                    default: return cudaErrorInvalidValue;
                }
            } else if (a.spread == kSpreadTiles2) {
                const size_t st = spread_tiles_smem<T>(kSpreadWarps, a.m, false, 2);
                switch (a.m) {
#define LAM_T(MH) case MH: k_spread2d_tiles2<T, kSpreadWarps, MH><<<gt, kSpreadWarps * 32, st, s>>>(in, Pt, kv0 + nx, a); break;
                    LAM_T(2) LAM_T(3) LAM_T(4) LAM_T(5) LAM_T(6) LAM_T(7) LAM_T(8)
#undef LAM_T
                    default: return cudaErrorInvalidValue;
                }
            } else {
                const size_t st = spread_tiles_smem<T>(kSpreadWarps, a.m);
                switch (a.m) {
#define LAM_T(MH) case MH: k_spread2d_tiles<T, kSpreadWarps, MH><<<gt, kSpreadWarps * 32, st, s>>>(in, Pt, kv0 + nx, a); break;
                    LAM_T(2) LAM_T(3) LAM_T(4) LAM_T(5) LAM_T(6) LAM_T(7) LAM_T(8)
#undef LAM_T
                    default: return cudaErrorInvalidValue;
                }
            }
        }
    } else if (a.spread != kSpreadAtomic) { LAM_SW(3) }
    else { LAM_SW(0) }
#undef LAM_SW
#undef LAM_S
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_usfft2d_adj(const C<T>* in, C<T>* P, C<T>* u1, int j0, int nb, const Usfft2dArgs<T>& a,
                               cudaStream_t s) {
    const int kv0 = j0;
    const size_t sr = (size_t)a.RB * fpad_len(a.M2) * sizeof(C<T>);
    const size_t sc = (size_t)a.CB * fpad_len(a.M1) * sizeof(C<T>);
    cudaError_t e = launch_spread2d<T>(in, P, j0, nb, a, s);
    if (e != cudaSuccess) return e;
    const int gp = pipe_grid((a.M2 / a.CB) * nb, a.fthr, 2 * sc);
    if (fft_mixed(a.fcM1) || fft_mixed(a.fcM2)) {
        k_colfft_adj_pipe<T, true><<<gp, a.fthr, 2 * sc, s>>>(P, a, nb, kv0);
        k_rowfft_adj<T, true><<<dim3(a.n1 / a.RB, nb), a.fthr, sr, s>>>(P, u1, kv0, a);
    } else {
        LAM_PLANE_NC(a.M1, LAM_CA);
        LAM_PLANE_NC(a.M2, LAM_RA);
    }
    return cudaGetLastError();
}

// max over the array of max(|re|, |im|), as the bit pattern of a non-negative
// float / double (monotone in the value) combined with atomicMax; *out must
// be zero beforehand.  The result does not depend on the order.
template <typename T>
__global__ void __launch_bounds__(256) k_absmax(const C<T>* __restrict__ in, long long n, T* out) {
    T m = (T)0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const C<T> v = in[i];
        m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) {
        if (sizeof(T) == 4) atomicMax(reinterpret_cast<unsigned int*>(out), __float_as_uint((float)m));
        else atomicMax(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong((double)m));
    }
}

template <typename T> cudaError_t launch_absmax(const C<T>* in, long long n, T* out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(T), s);
    if (e != cudaSuccess) return e;
    long long b = (n + 255) / 256;
    k_absmax<T><<<(int)(b < 1184 ? b : 1184), 256, 0, s>>>(in, n, out);
    return cudaGetLastError();
}
template cudaError_t launch_absmax<float>(const C<float>*, long long, float*, cudaStream_t);
template cudaError_t launch_absmax<double>(const C<double>*, long long, double*, cudaStream_t);

template <typename T> cudaError_t configure_usfft2d() {
    const int mx = kMaxDynSmem;
    cudaError_t e = cudaSuccess;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (!e) e = cudaFuncSetAttribute(k_rowfft_fwd<T, false>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_rowfft_adj<T, false>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_rowfft_fwd<T, true>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_rowfft_adj<T, true>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_colfft_fwd_pipe<T, false>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_colfft_fwd_pipe<T, true>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_colfft_adj_pipe<T, false>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_colfft_adj_pipe<T, true>, at, mx);
    if constexpr (sizeof(T) == 4) {
#define LAM_NCA(NC)                                                                  \
    if (!e) e = cudaFuncSetAttribute(k_rowfft_fwd<T, false, NC>, at, mx);      \
    if (!e) e = cudaFuncSetAttribute(k_rowfft_adj<T, false, NC>, at, mx);      \
    if (!e) e = cudaFuncSetAttribute(k_colfft_fwd_pipe<T, false, NC>, at, mx); \
    if (!e) e = cudaFuncSetAttribute(k_colfft_adj_pipe<T, false, NC>, at, mx);
        LAM_NCA(512) LAM_NCA(1024) LAM_NCA(2048) LAM_NCA(4096)
#undef LAM_NCA
    }
    // the tile kernels also hold static shared memory (the per-warp line lists)
    const int mt = kMaxDynSmem - 4096;
#define LAM_A(MH)                                                                          \
    if (!e) e = cudaFuncSetAttribute(k_gather2d_tiled<T, kGatherWarps, MH>, at, mt);       \
    if (!e) e = cudaFuncSetAttribute(k_scatter2d_atomic<T, kScatterWarps, MH, 0>, at, mt);  \
    if (!e) e = cudaFuncSetAttribute(k_scatter2d_atomic<T, kScatterWarps, MH, 3>, at, mt);    \
    if (!e) e = cudaFuncSetAttribute(k_spread2d_tiles<T, kSpreadWarps, MH>, at, mt);    \
    if (!e) e = cudaFuncSetAttribute(k_spread2d_tiles_exact<T, kSpreadWarps, MH>, at, mt); \
    if (!e) e = cudaFuncSetAttribute(k_spread2d_tiles2<T, kSpreadWarps, MH>, at, mt); \
    if (!e) e = cudaFuncSetAttribute(k_spread2d_halo<T, kScatterWarps, MH>, at, mt); \
    if (!e) e = cudaFuncSetAttribute(k_spread2d_sweep<T, MH>, at, kMaxDynSmem - 1024);
    LAM_A(2) LAM_A(3) LAM_A(4) LAM_A(5) LAM_A(6) LAM_A(7) LAM_A(8)
#undef LAM_A
    return e;
}

// ---------------------------------------------------------------------------
// batched stages (one persistent launch per stage over a work list)
// ---------------------------------------------------------------------------

// copies an argument block (a plain struct) with the whole thread block
template <typename A> __device__ __forceinline__ void copy_block_args(A& dst, const A& src) {
    static_assert(sizeof(A) % 4 == 0, "argument block size");
    const int* s = reinterpret_cast<const int*>(&src);
    int* d = reinterpret_cast<int*>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(A) / 4); i += blockDim.x) d[i] = s[i];
}

// problem owning work item w (start[p] <= w < start[p + 1])
__device__ __forceinline__ int batch_problem(const int* start, int count, int w) {
    int p = 0;
    while (p + 1 < count && w >= start[p + 1]) ++p;
    return p;
}

constexpr size_t kBatchDynSmem = kMaxDynSmem - 6144;  // room for the static argument copy and line lists

template <typename T>
__global__ void kb_set_ptrs(BatchTable<T>* __restrict__ bt, BatchPtrs ptrs, int count) {
    const int t = threadIdx.x;
    if (t < count) {
        bt->in[t] = ptrs.in[t];
        bt->out[t] = ptrs.out[t];
    }
}

template <typename T, bool MIXED, int STAGE>
__global__ void __launch_bounds__(kFftThreads) kb_plane_fft(const BatchTable<T>* __restrict__ bt) {
    __shared__ Usfft2dArgs<T> sa;
    const int* st = bt->start[STAGE];
    const int total = st[bt->count];
    int cur = -1;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int p = batch_problem(st, bt->count, w);
        if (p != cur) {  // block-uniform; the previous item ended with a barrier
            copy_block_args(sa, bt->a2[p]);
            __syncthreads();
            cur = p;
        }
        const int l = w - st[p], gx = bt->gx[STAGE][p];
        const int bx = l % gx, by = l / gx;
        if (STAGE == kBRowFwd) k_rowfft_fwd_body<T, MIXED>(bt->u1[p], bt->P[p], 0, sa, bx, by);
        else if (STAGE == kBColFwd) k_colfft_fwd_body<T, MIXED>(bt->P[p], sa, bx, by);
        else if (STAGE == kBColAdj) k_colfft_adj_body<T, MIXED>(bt->P[p], sa, bx, by);
        else k_rowfft_adj_body<T, MIXED>(bt->P[p], bt->u1[p], 0, sa, bx, by);
        __syncthreads();
    }
}

template <typename T, int NW, int MH>
__global__ void __launch_bounds__(NW * 32) kb_gather(const BatchTable<T>* __restrict__ bt) {
    __shared__ Usfft2dArgs<T> sa;
    const int* st = bt->start[kBGather];
    const int total = st[bt->count];
    int cur = -1;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int p = batch_problem(st, bt->count, w);
        if (p != cur) {  // block-uniform; the previous item ended with a barrier
            copy_block_args(sa, bt->a2[p]);
            __syncthreads();
            cur = p;
        }
        const int l = w - st[p], gx = bt->gx[kBGather][p];
        const int t = l / gx;
        k_gather2d_tiled_body<T, NW, MH>(bt->P[p], (C<T>*)bt->out[p], nullptr, 0, sa, l - t * gx, t);
        __syncthreads();
    }
}

template <typename T, int NW, int MH>
__global__ void __launch_bounds__(NW * 32, sizeof(T) == 4 ? 4 : 2) kb_spread(const BatchTable<T>* __restrict__ bt) {
    __shared__ Usfft2dArgs<T> sa;
    const int* st = bt->start[kBSpread];
    const int total = st[bt->count];
    int cur = -1;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int p = batch_problem(st, bt->count, w);
        if (p != cur) {  // block-uniform; the previous item ended with a barrier
            copy_block_args(sa, bt->a2[p]);
            __syncthreads();
            cur = p;
        }
        const int l = w - st[p], gx = bt->gx[kBSpread][p];
        // the problem's first sa.nacc plane jobs were spread exactly by their own launches
        k_spread2d_tiles_body<T, NW, MH>((const C<T>*)bt->in[p], bt->P[p] + (size_t)sa.nacc * sa.M1 * sa.M2, sa.nacc,
                                         sa, l % gx, l / gx);
        __syncthreads();
    }
}

template <typename T> cudaError_t launch_batch_ptrs(BatchTable<T>* dev, const BatchPtrs& ptrs, int count, cudaStream_t s) {
    kb_set_ptrs<T><<<1, kMaxBatch, 0, s>>>(dev, ptrs, count);
    return cudaGetLastError();
}

// the kernel of a batched plane stage, as a void pointer for occupancy queries
template <typename T> const void* batch_plane_kernel(int stage, bool mixed, int m) {
#define LAM_FFTK(ST) return mixed ? (const void*)kb_plane_fft<T, true, ST> : (const void*)kb_plane_fft<T, false, ST>;
    switch (stage) {
        case kBRowFwd: LAM_FFTK(kBRowFwd)
        case kBColFwd: LAM_FFTK(kBColFwd)
        case kBColAdj: LAM_FFTK(kBColAdj)
        case kBRowAdj: LAM_FFTK(kBRowAdj)
        default: break;
    }
#undef LAM_FFTK
#define LAM_MH(MH) case MH: return stage == kBGather ? (const void*)kb_gather<T, kGatherWarps, MH> : (const void*)kb_spread<T, kSpreadWarps, MH>;
    switch (m) {
        LAM_MH(2) LAM_MH(3) LAM_MH(4) LAM_MH(5) LAM_MH(6) LAM_MH(7) LAM_MH(8)
        default: return nullptr;
    }
#undef LAM_MH
}

// threads per block of a batched plane stage: the same block shapes as the
// single-plan kernels, so both give bitwise the same results
static int batch_plane_threads(int stage) {
    return stage == kBGather ? kGatherWarps * 32 : stage == kBSpread ? kSpreadWarps * 32 : kFftThreads;
}

template <typename T>
cudaError_t launch_batch_plane(const BatchTable<T>* dev, int stage, bool mixed, int m, const BatchLaunch& L,
                               cudaStream_t s) {
    const void* k = batch_plane_kernel<T>(stage, mixed, m);
    if (!k) return cudaErrorInvalidValue;
    const int threads = batch_plane_threads(stage);
    void* args[] = {(void*)&dev};
    return cudaLaunchKernel(k, dim3(L.grid), dim3(threads), args, L.smem, s);
}

template <typename T> int batch_occupancy(int stage, bool mixed, int m, size_t smem) {
    const void* k = batch_plane_kernel<T>(stage, mixed, m);
    const int threads = batch_plane_threads(stage);
    int nb = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, smem) != cudaSuccess) return 0;
    return nb;
}

template <typename T> cudaError_t configure_batch_plane() {
    cudaError_t e = cudaSuccess;
    for (int stage : {kBRowFwd, kBColFwd, kBColAdj, kBRowAdj, kBGather, kBSpread})
        for (bool mixed : {false, true})
            for (int m = 2; m <= 8; ++m) {
                const void* k = batch_plane_kernel<T>(stage, mixed, m);
                if (!e && k) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchDynSmem);
                if (stage != kBGather && stage != kBSpread) break;  // the FFT stages do not depend on m
            }
    return e;
}

template <typename T> size_t spread_tiles_bytes(int m) { return spread_tiles_smem<T>(kSpreadWarps, m); }
template size_t spread_tiles_bytes<float>(int);
template size_t spread_tiles_bytes<double>(int);

template cudaError_t launch_batch_ptrs<float>(BatchTable<float>*, const BatchPtrs&, int, cudaStream_t);
template cudaError_t launch_batch_ptrs<double>(BatchTable<double>*, const BatchPtrs&, int, cudaStream_t);
template cudaError_t launch_batch_plane<float>(const BatchTable<float>*, int, bool, int, const BatchLaunch&, cudaStream_t);
template cudaError_t launch_batch_plane<double>(const BatchTable<double>*, int, bool, int, const BatchLaunch&,
                                                cudaStream_t);
template int batch_occupancy<float>(int, bool, int, size_t);
template int batch_occupancy<double>(int, bool, int, size_t);
template cudaError_t configure_batch_plane<float>();
template cudaError_t configure_batch_plane<double>();

template cudaError_t launch_usfft2d_fwd<float>(const C<float>*, C<float>*, C<float>*, const C<float>*, int, int,
                                               const Usfft2dArgs<float>&, cudaStream_t);
template cudaError_t launch_usfft2d_fwd<double>(const C<double>*, C<double>*, C<double>*, const C<double>*, int,
                                                int, const Usfft2dArgs<double>&, cudaStream_t);
template cudaError_t launch_spread2d<float>(const C<float>*, C<float>*, int, int, const Usfft2dArgs<float>&, cudaStream_t);
template cudaError_t launch_spread2d<double>(const C<double>*, C<double>*, int, int, const Usfft2dArgs<double>&,
                                             cudaStream_t);
template cudaError_t launch_usfft2d_planes<float>(const C<float>*, C<float>*, int, int, const Usfft2dArgs<float>&,
                                                  cudaStream_t);
template cudaError_t launch_usfft2d_planes<double>(const C<double>*, C<double>*, int, int, const Usfft2dArgs<double>&,
                                                   cudaStream_t);
template cudaError_t launch_usfft2d_adj<float>(const C<float>*, C<float>*, C<float>*, int, int,
                                               const Usfft2dArgs<float>&, cudaStream_t);
template cudaError_t launch_usfft2d_adj<double>(const C<double>*, C<double>*, C<double>*, int, int,
                                                const Usfft2dArgs<double>&, cudaStream_t);
template cudaError_t configure_usfft2d<float>();
template cudaError_t configure_usfft2d<double>();

}  // namespace lam
