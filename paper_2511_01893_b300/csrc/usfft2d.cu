// usfft2d.cu - F_u2D and its transpose: one 2D unequally-spaced FFT per kv plane.
//
// F_u2D (Section 2) maps u1[n1, h, n2] to u2[n_theta, h, w]: for each kv plane
// it evaluates sum_{x,y} u1[x, kv, y] exp(-2 pi i (xi_x x + xi_y y)) at the
// n_theta * w slice points (xi_x, xi_y)(theta, kv, ku).  Gaussian USFFT in 2D:
// deapodise, zero-pad to M1 x M2 = 2 n1 x 2 n2, row FFTs (only the n1 non-zero
// rows), column FFTs, then a separable 2m x 2m Gaussian gather.
//
// Forward (type 2) kernels, per batch of nb planes held in P[nb][M1][M2]:
//   k_rowfft_fwd   u1 rows -> deapodised, padded, FFT along y -> P rows
//   k_colfft_fwd   P columns (n1 non-zero entries) -> FFT along x, in place
//   k_gather2d     one thread per slice point: 64 taps from P, optional fused
//                  subtraction (out = value - sub, Section 4.2)
// Transpose (type 1):
//   k_scatter2d    tile-owned accumulation: a warp owns a TS x TS tile of the
//                  padded plane, finds the slice lines that cross it and, per
//                  line, the (contiguous) ku range of points whose taps reach
//                  the tile, and accumulates weight * value in a shared-memory
//                  copy of the tile (compensated summation in FP32); the tile
//                  is written once.  No atomics; the result does not depend on
//                  scheduling.
//   k_colfft_adj   inverse FFT along x, keep the n1 rows the crop needs
//   k_rowfft_adj   inverse FFT along y, crop, deapodise -> u1 rows
#include "fft.cuh"
#include "kernels.h"

namespace lam {

// --------------------------------------------------------------------------
// row / column passes
// --------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_rowfft_fwd(const C<T>* __restrict__ u1, C<T>* __restrict__ P,
                                                    int kv0, Usfft2dArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T>* bufa = reinterpret_cast<C<T>*>(smem_raw);
    const int b = blockIdx.y, kv = kv0 + b;
    const int x0 = blockIdx.x * a.RB;
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int i = tid; i < a.RB * a.M2; i += nthr) bufa[i] = cmake<T>(0, 0);
    __syncthreads();
    const C<T>* src = u1 + ((size_t)kv * a.n1 + x0) * a.n2;
    for (int i = tid; i < a.RB * a.n2; i += nthr) {
        const int r = i / a.n2, y = i - r * a.n2;
        const T s = a.d1[x0 + r] * a.d2[y];
        bufa[r * a.M2 + wrap(y - a.n2 / 2, a.M2)] = cscale(src[i], s);
    }
    __syncthreads();
    fft_lines_ip<-1, FftMaxB<T>::value, T>(bufa, a.RB, a.M2, a.M2, a.logM2, a.tw, a.tw2);
    const C<T>* res = bufa;
    C<T>* dst = P + (size_t)b * a.M1 * a.M2;
    for (int i = tid; i < a.RB * a.M2; i += nthr) {
        const int r = i / a.M2, j = i - r * a.M2;
        dst[(size_t)wrap(x0 + r - a.n1 / 2, a.M1) * a.M2 + j] = res[i];
    }
}

template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_colfft_fwd(C<T>* __restrict__ P, Usfft2dArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T>* bufa = reinterpret_cast<C<T>*>(smem_raw);
    const int b = blockIdx.y;
    const int c0 = blockIdx.x * a.CB;
    const int tid = threadIdx.x, nthr = blockDim.x;
    C<T>* pl = P + (size_t)b * a.M1 * a.M2 + c0;
    for (int i = tid; i < a.CB * a.M1; i += nthr) bufa[i] = cmake<T>(0, 0);
    __syncthreads();
    for (int i = tid; i < a.n1 * a.CB; i += nthr) {
        const int x = i / a.CB, c = i - x * a.CB;
        const int row = wrap(x - a.n1 / 2, a.M1);
        bufa[c * a.M1 + row] = pl[(size_t)row * a.M2 + c];
    }
    __syncthreads();
    fft_lines_ip<-1, FftMaxB<T>::value, T>(bufa, a.CB, a.M1, a.M1, a.logM1, a.tw, a.tw1);
    const C<T>* res = bufa;
    for (int i = tid; i < a.M1 * a.CB; i += nthr) {
        const int j = i / a.CB, c = i - j * a.CB;
        pl[(size_t)j * a.M2 + c] = res[c * a.M1 + j];
    }
}

template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_colfft_adj(C<T>* __restrict__ P, Usfft2dArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T>* bufa = reinterpret_cast<C<T>*>(smem_raw);
    const int b = blockIdx.y;
    const int c0 = blockIdx.x * a.CB;
    const int tid = threadIdx.x, nthr = blockDim.x;
    C<T>* pl = P + (size_t)b * a.M1 * a.M2 + c0;
    for (int i = tid; i < a.M1 * a.CB; i += nthr) {
        const int j = i / a.CB, c = i - j * a.CB;
        bufa[c * a.M1 + j] = pl[(size_t)j * a.M2 + c];
    }
    __syncthreads();
    fft_lines_ip<+1, FftMaxB<T>::value, T>(bufa, a.CB, a.M1, a.M1, a.logM1, a.tw, a.tw1);
    const C<T>* res = bufa;
    for (int i = tid; i < a.n1 * a.CB; i += nthr) {
        const int x = i / a.CB, c = i - x * a.CB;
        const int row = wrap(x - a.n1 / 2, a.M1);
        pl[(size_t)row * a.M2 + c] = res[c * a.M1 + row];
    }
}

template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_rowfft_adj(const C<T>* __restrict__ P, C<T>* __restrict__ u1,
                                                    int kv0, Usfft2dArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C<T>* bufa = reinterpret_cast<C<T>*>(smem_raw);
    const int b = blockIdx.y, kv = kv0 + b;
    const int x0 = blockIdx.x * a.RB;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const C<T>* pl = P + (size_t)b * a.M1 * a.M2;
    for (int i = tid; i < a.RB * a.M2; i += nthr) {
        const int r = i / a.M2, j = i - r * a.M2;
        bufa[i] = pl[(size_t)wrap(x0 + r - a.n1 / 2, a.M1) * a.M2 + j];
    }
    __syncthreads();
    fft_lines_ip<+1, FftMaxB<T>::value, T>(bufa, a.RB, a.M2, a.M2, a.logM2, a.tw, a.tw2);
    const C<T>* res = bufa;
    C<T>* dst = u1 + ((size_t)kv * a.n1 + x0) * a.n2;
    for (int i = tid; i < a.RB * a.n2; i += nthr) {
        const int r = i / a.n2, y = i - r * a.n2;
        const T s = a.d1[x0 + r] * a.d2[y];
        dst[i] = cscale(res[r * a.M2 + wrap(y - a.n2 / 2, a.M2)], s);
    }
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

// --------------------------------------------------------------------------
// gather (type 2 interpolation) with optional fused subtraction
// --------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(256) k_gather2d(const C<T>* __restrict__ P, C<T>* __restrict__ out,
                                                  const C<T>* __restrict__ sub, int kv0, Usfft2dArgs<T> a) {
    const int th = blockIdx.x, b = blockIdx.y, kv = kv0 + b;
    const int kvc = kv - a.h / 2;
    const typename AngleT<T>::type g = a.ang[th];
    const C<T>* pl = P + (size_t)b * a.M1 * a.M2;
    const int nt = 2 * a.m;
    for (int ku = threadIdx.x; ku < a.w; ku += blockDim.x) {
        int jx, jy;
        T fx, fy;
        point_pos(g, ku - a.w / 2, kvc, jx, fx, jy, fy);
        T wy[16];
        for (int t = 0; t < nt; ++t) {
            const T d = fy + (T)(a.m - 1 - t);
            wy[t] = gexp(-d * d * a.inv4beta);
        }
        T sr = 0, si = 0;
        for (int s = 0; s < nt; ++s) {
            const T dx = fx + (T)(a.m - 1 - s);
            const T wx = gexp(-dx * dx * a.inv4beta);
            const C<T>* row = pl + (size_t)wrap(jx - a.m + 1 + s, a.M1) * a.M2;
            T rr = 0, ri = 0;
            for (int t = 0; t < nt; ++t) {
                const C<T> p = row[wrap(jy - a.m + 1 + t, a.M2)];
                rr += wy[t] * p.x;
                ri += wy[t] * p.y;
            }
            sr += wx * rr;
            si += wx * ri;
        }
        const size_t o = ((size_t)th * a.h + kv) * a.w + ku;
        C<T> v = cmake<T>(sr, si);
        if (sub) v = csub(v, sub[o]);
        out[o] = v;
    }
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

// Tiled gather: one warp per TS x TS tile of tap-window origins.  The warp
// stages its tile plus a (2m - 1) halo of the padded plane in shared memory,
// culls the slice lines against the tile, and evaluates exactly the points
// whose window origin (j0 - m + 1 in both axes, unwrapped) falls in the tile
// (or one of its periodic images), one point per lane.  Each point is owned
// by exactly one (tile, image), so every output is written once.
template <typename T, int TPB>
__global__ void __launch_bounds__(TPB * 32) k_gather2d_tiled(const C<T>* __restrict__ P, C<T>* __restrict__ out,
                                                             const C<T>* __restrict__ sub, int kv0, Usfft2dArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TS = a.TS, nt = 2 * a.m;
    const int SH = TS + nt - 1;  // staged rows
    const int SW = TS + nt;      // staged row stride
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_x = a.M1 / TS, tiles_y = a.M2 / TS;
    const int tile = blockIdx.x * TPB + warp;
    if (tile >= tiles_x * tiles_y) return;
    C<T>* st = reinterpret_cast<C<T>*>(smem_raw) + (size_t)warp * SH * SW;
    const int tx0 = (tile / tiles_y) * TS, ty0 = (tile % tiles_y) * TS;
    const int b = blockIdx.y, kv = kv0 + b, kvc = kv - a.h / 2;
    const C<T>* pl = P + (size_t)b * a.M1 * a.M2;
    for (int i = lane; i < SH * SH; i += 32) {
        const int r = i / SH, c = i - r * SH;
        st[r * SW + c] = pl[(size_t)wrap(tx0 + r, a.M1) * a.M2 + wrap(ty0 + c, a.M2)];
    }
    __syncwarp();
    const int kmin = -a.w / 2, kmax = a.w / 2 - 1;
    const T hx = (T)TS * (T)0.5 + (T)1;
    for (int ix = -a.nimg; ix <= a.nimg; ++ix) {
        const int bx0 = tx0 + ix * a.M1;
        for (int iy = -a.nimg; iy <= a.nimg; ++iy) {
            const int by0 = ty0 + iy * a.M2;
            // positions whose window origin is in [b0, b0 + TS): p in [b0 + m - 1, b0 + TS + m - 1)
            const T cx = (T)(bx0 + a.m - 1) + (T)TS * (T)0.5, cy = (T)(by0 + a.m - 1) + (T)TS * (T)0.5;
            if (sqrt(cx * cx + cy * cy) > a.rmax + hx * (T)1.5) continue;
            for (int base = 0; base < a.T_; base += 32) {
                const int th = base + lane;
                bool hit = false;
                if (th < a.T_) {
                    const typename AngleT<T>::type g = a.ang[th];
                    T Ax, Cx, Ay, Cy;
                    line_coef(g, kvc, Ax, Cx, Ay, Cy);
                    const T nrm = sqrt(Ax * Ax + Ay * Ay);
                    const T nx = -Ay / nrm, ny = Ax / nrm;
                    const T dist = fabs((cx - Cx) * nx + (cy - Cy) * ny);
                    hit = dist <= hx * (fabs(nx) + fabs(ny)) + (T)1;
                }
                unsigned mask = __ballot_sync(0xffffffffu, hit);
                while (mask) {
                    const int th2 = base + __ffs(mask) - 1;
                    mask &= mask - 1;
                    const typename AngleT<T>::type g = a.ang[th2];
                    T Ax, Cx, Ay, Cy;
                    line_coef(g, kvc, Ax, Cx, Ay, Cy);
                    int lo = kmin, hi = kmax;
                    clip_line<T>(Ax, Cx, (T)(bx0 + a.m - 1), (T)(bx0 + TS + a.m - 1), lo, hi);
                    clip_line<T>(Ay, Cy, (T)(by0 + a.m - 1), (T)(by0 + TS + a.m - 1), lo, hi);
                    const size_t orow = ((size_t)th2 * a.h + kv) * a.w + a.w / 2;
                    for (int k0 = lo; k0 <= hi; k0 += 32) {
                        const int kuc = k0 + lane;
                        if (kuc > hi) continue;
                        int jx, jy;
                        T fx, fy;
                        point_pos(g, kuc, kvc, jx, fx, jy, fy);
                        const int ox = jx - a.m + 1 - bx0, oy = jy - a.m + 1 - by0;
                        if (ox < 0 || ox >= TS || oy < 0 || oy >= TS) continue;
                        T wy[16];
#pragma unroll
                        for (int t = 0; t < 16; ++t)
                            if (t < nt) {
                                const T d = fy + (T)(a.m - 1 - t);
                                wy[t] = gexp(-d * d * a.inv4beta);
                            }
                        T sr = 0, si = 0;
#pragma unroll
                        for (int sx = 0; sx < 16; ++sx) {
                            if (sx >= nt) break;
                            const T d = fx + (T)(a.m - 1 - sx);
                            const T wx = gexp(-d * d * a.inv4beta);
                            const C<T>* rowp = st + (ox + sx) * SW + oy;
                            T rr = 0, ri = 0;
#pragma unroll
                            for (int t = 0; t < 16; ++t)
                                if (t < nt) {
                                    const C<T> pv = rowp[t];
                                    rr += wy[t] * pv.x;
                                    ri += wy[t] * pv.y;
                                }
                            sr += wx * rr;
                            si += wx * ri;
                        }
                        const size_t o = orow + kuc;
                        C<T> v = cmake<T>(sr, si);
                        if (sub) v = csub(v, sub[o]);
                        out[o] = v;
                    }
                }
            }
        }
    }
}

// --------------------------------------------------------------------------
// scatter (type 1 spreading), tile-owned, per-warp accumulators
// --------------------------------------------------------------------------

template <typename T> struct Acc;  // accumulator cell
template <> struct Acc<float> {
    float sr, si, cr, ci;  // sum and Kahan compensation
    __device__ __forceinline__ void zero() { sr = si = cr = ci = 0.f; }
    __device__ __forceinline__ void add(float vr, float vi) {
        const float yr = vr - cr, yi = vi - ci;
        const float tr = sr + yr, ti = si + yi;
        cr = (tr - sr) - yr;
        ci = (ti - si) - yi;
        sr = tr;
        si = ti;
    }
};
template <> struct Acc<double> {
    double sr, si;
    __device__ __forceinline__ void zero() { sr = si = 0.0; }
    __device__ __forceinline__ void add(double vr, double vi) {
        sr += vr;
        si += vi;
    }
};

// One warp owns one TS x TS tile of the padded plane and a private
// accumulator for it (compensated in FP32); a block holds TPB tiles.  The warp
// culls the n_theta slice lines against its tile with a lane-parallel distance
// test, then walks each crossing line 32 points at a time, one point per lane:
// the lane computes the point's tap window and 2 x 2m Gaussian weights in
// registers, and the warp steps through the (2m)^2 taps in lock-step.  Window
// origins of points 2 cells apart on one line are distinct, so the 32 lanes
// of one tap step never touch the same cell.
template <typename T, int TPB>
__global__ void __launch_bounds__(TPB * 32) k_scatter2d(const C<T>* __restrict__ in, C<T>* __restrict__ P,
                                                        int kv0, Usfft2dArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TS = a.TS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_x = a.M1 / TS, tiles_y = a.M2 / TS;
    const int tile = blockIdx.x * TPB + warp;
    if (tile >= tiles_x * tiles_y) return;  // whole warp exits; no block-wide sync below
    Acc<T>* my = reinterpret_cast<Acc<T>*>(smem_raw) + (size_t)warp * TS * TS;
    for (int i = lane; i < TS * TS; i += 32) my[i].zero();
    __syncwarp();
    const int tx0 = (tile / tiles_y) * TS, ty0 = (tile % tiles_y) * TS;
    const int b = blockIdx.y, kv = kv0 + b, kvc = kv - a.h / 2;
    const int nt = 2 * a.m;
    const int kmin = -a.w / 2, kmax = a.w / 2 - 1;
    const T hx = (T)(TS + 2 * a.m) * (T)0.5;
    for (int ix = -a.nimg; ix <= a.nimg; ++ix) {
        const int bx0 = tx0 + ix * a.M1;
        for (int iy = -a.nimg; iy <= a.nimg; ++iy) {
            const int by0 = ty0 + iy * a.M2;
            const T cx = (T)bx0 + (T)(TS - 1) * (T)0.5, cy = (T)by0 + (T)(TS - 1) * (T)0.5;
            if (sqrt(cx * cx + cy * cy) > a.rmax + hx * (T)1.5) continue;
            for (int base = 0; base < a.T_; base += 32) {
                const int th = base + lane;
                bool hit = false;
                if (th < a.T_) {
                    const typename AngleT<T>::type g = a.ang[th];
                    T Ax, Cx, Ay, Cy;
                    line_coef(g, kvc, Ax, Cx, Ay, Cy);
                    const T nrm = sqrt(Ax * Ax + Ay * Ay);
                    const T nx = -Ay / nrm, ny = Ax / nrm;
                    const T dist = fabs((cx - Cx) * nx + (cy - Cy) * ny);
                    hit = dist <= hx * (fabs(nx) + fabs(ny)) + (T)1;
                }
                unsigned mask = __ballot_sync(0xffffffffu, hit);
                while (mask) {
                    const int th2 = base + __ffs(mask) - 1;
                    mask &= mask - 1;
                    const typename AngleT<T>::type g = a.ang[th2];
                    T Ax, Cx, Ay, Cy;
                    line_coef(g, kvc, Ax, Cx, Ay, Cy);
                    int lo = kmin, hi = kmax;
                    clip_line<T>(Ax, Cx, (T)(bx0 - a.m), (T)(bx0 + TS + a.m - 1), lo, hi);
                    clip_line<T>(Ay, Cy, (T)(by0 - a.m), (T)(by0 + TS + a.m - 1), lo, hi);
                    const C<T>* row = in + ((size_t)th2 * a.h + kv) * a.w + a.w / 2;
                    // lanes take points pstride apart (>= sqrt 2 cells), so their
                    // window origins differ; pstride passes cover every point
                    const int ps = a.pstride;
                    for (int kq = 0; lo + (kq / ps) * 32 * ps <= hi; ++kq) {
                        const int kuc = lo + (kq / ps) * 32 * ps + (kq % ps) + lane * ps;
                        const bool act = kuc <= hi;
                        int ox = -1 << 20, oy = -1 << 20;
                        T wx[16], wy[16];
                        C<T> v = cmake<T>(0, 0);
                        if (act) {
                            int jx, jy;
                            T fx, fy;
                            point_pos(g, kuc, kvc, jx, fx, jy, fy);
                            ox = jx - a.m + 1 - bx0;
                            oy = jy - a.m + 1 - by0;
#pragma unroll
                            for (int t = 0; t < 16; ++t) {
                                if (t < nt) {
                                    const T dx = fx + (T)(a.m - 1 - t), dy = fy + (T)(a.m - 1 - t);
                                    wx[t] = gexp(-dx * dx * a.inv4beta);
                                    wy[t] = gexp(-dy * dy * a.inv4beta);
                                }
                            }
                            v = row[kuc];
                        }
#pragma unroll
                        for (int sx = 0; sx < 16; ++sx) {
                            if (sx >= nt) break;
                            const int cxx = ox + sx;
                            const bool rowin = act && cxx >= 0 && cxx < TS;
                            const T wxs = wx[sx];
#pragma unroll
                            for (int sy = 0; sy < 16; ++sy) {
                                if (sy >= nt) break;
                                const int cyy = oy + sy;
                                if (rowin && cyy >= 0 && cyy < TS) {
                                    const T wgt = wxs * wy[sy];
                                    my[cxx * TS + cyy].add(wgt * v.x, wgt * v.y);
                                }
                                __syncwarp();
                            }
                        }
                    }
                }
            }
        }
    }
    __syncwarp();
    C<T>* pl = P + (size_t)b * a.M1 * a.M2;
    for (int i = lane; i < TS * TS; i += 32) {
        const int cxx = i / TS, cyy = i - cxx * TS;
        pl[(size_t)(tx0 + cxx) * a.M2 + ty0 + cyy] = cmake<T>(my[i].sr, my[i].si);
    }
}

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------

constexpr int kScatterWarps = 4;  // tiles (warps) per block

template <typename T>
cudaError_t launch_usfft2d_fwd(const C<T>* u1, C<T>* P, C<T>* out, const C<T>* sub, int kv0, int nb,
                               const Usfft2dArgs<T>& a, cudaStream_t s) {
    const size_t sr = (size_t)a.RB * a.M2 * sizeof(C<T>);
    const size_t sc = (size_t)a.CB * a.M1 * sizeof(C<T>);
    k_rowfft_fwd<T><<<dim3(a.n1 / a.RB, nb), kFftThreads, sr, s>>>(u1, P, kv0, a);
    k_colfft_fwd<T><<<dim3(a.M2 / a.CB, nb), kFftThreads, sc, s>>>(P, a);
    constexpr int NW = kScatterWarps;
    const int ntiles = (a.M1 / a.TS) * (a.M2 / a.TS);
    const size_t sg = (size_t)NW * (a.TS + 2 * a.m - 1) * (a.TS + 2 * a.m) * sizeof(C<T>);
    k_gather2d_tiled<T, NW><<<dim3((ntiles + NW - 1) / NW, nb), NW * 32, sg, s>>>(P, out, sub, kv0, a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_usfft2d_adj(const C<T>* in, C<T>* P, C<T>* u1, int kv0, int nb, const Usfft2dArgs<T>& a,
                               cudaStream_t s) {
    constexpr int NW = kScatterWarps;
    const size_t sa = (size_t)NW * a.TS * a.TS * sizeof(Acc<T>);
    const int ntiles = (a.M1 / a.TS) * (a.M2 / a.TS);
    const size_t sr = (size_t)a.RB * a.M2 * sizeof(C<T>);
    const size_t sc = (size_t)a.CB * a.M1 * sizeof(C<T>);
    k_scatter2d<T, NW><<<dim3((ntiles + NW - 1) / NW, nb), NW * 32, sa, s>>>(in, P, kv0, a);
    k_colfft_adj<T><<<dim3(a.M2 / a.CB, nb), kFftThreads, sc, s>>>(P, a);
    k_rowfft_adj<T><<<dim3(a.n1 / a.RB, nb), kFftThreads, sr, s>>>(P, u1, kv0, a);
    return cudaGetLastError();
}

template <typename T> size_t scatter_acc_bytes() { return sizeof(Acc<T>) * kScatterWarps; }

template <typename T> cudaError_t configure_usfft2d() {
    const int mx = kMaxDynSmem;
    cudaError_t e = cudaSuccess;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (!e) e = cudaFuncSetAttribute(k_rowfft_fwd<T>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_colfft_fwd<T>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_rowfft_adj<T>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_colfft_adj<T>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_scatter2d<T, kScatterWarps>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_gather2d_tiled<T, kScatterWarps>, at, mx);
    return e;
}

template cudaError_t launch_usfft2d_fwd<float>(const C<float>*, C<float>*, C<float>*, const C<float>*, int, int,
                                               const Usfft2dArgs<float>&, cudaStream_t);
template cudaError_t launch_usfft2d_fwd<double>(const C<double>*, C<double>*, C<double>*, const C<double>*, int,
                                                int, const Usfft2dArgs<double>&, cudaStream_t);
template cudaError_t launch_usfft2d_adj<float>(const C<float>*, C<float>*, C<float>*, int, int,
                                               const Usfft2dArgs<float>&, cudaStream_t);
template cudaError_t launch_usfft2d_adj<double>(const C<double>*, C<double>*, C<double>*, int, int,
                                                const Usfft2dArgs<double>&, cudaStream_t);
template size_t scatter_acc_bytes<float>();
template size_t scatter_acc_bytes<double>();
template cudaError_t configure_usfft2d<float>();
template cudaError_t configure_usfft2d<double>();

}  // namespace lam
