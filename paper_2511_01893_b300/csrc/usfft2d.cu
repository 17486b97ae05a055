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

// ---------------------------------------------------------------------------
// Warp-level enumeration of the slice points that may touch one tile image.
// The warp tests 32 lines at a time against the tile's position box (lane
// parallel), computes each crossing line's ku interval, scans the interval
// lengths, and hands the flattened point list out 32 points at a time, one per
// lane, across line boundaries.  fn(th, kuc, g) is called for each lane's
// point (with active lanes first in each batch; inactive lanes get th = -1).
// ---------------------------------------------------------------------------
template <typename T, typename F>
__device__ __forceinline__ void for_tile_points(const Usfft2dArgs<T>& a, int kvc, T cx, T cy, T hbox,
                                                T bxmin, T bxmax, T bymin, T bymax, F&& fn) {
    const int lane = threadIdx.x & 31;
    const int kmin = -a.w / 2, kmax = a.w / 2 - 1;
    for (int base = 0; base < a.T_; base += 32) {
        const int th = base + lane;
        int lo = 1, hi = 0;
        if (th < a.T_) {
            const typename AngleT<T>::type g = a.ang[th];
            T Ax, Cx, Ay, Cy;
            line_coef(g, kvc, Ax, Cx, Ay, Cy);
            const T nrm = sqrt(Ax * Ax + Ay * Ay);
            const T nx = -Ay / nrm, ny = Ax / nrm;
            const T dist = fabs((cx - Cx) * nx + (cy - Cy) * ny);
            if (dist <= hbox * (fabs(nx) + fabs(ny)) + (T)1) {
                lo = kmin;
                hi = kmax;
                clip_line<T>(Ax, Cx, bxmin, bxmax, lo, hi);
                clip_line<T>(Ay, Cy, bymin, bymax, lo, hi);
            }
        }
        const int cnt = hi >= lo ? hi - lo + 1 : 0;
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
            // skip empty intervals that share the prefix: move to the owner with cnt > 0
            const int ocnt = __shfl_sync(0xffffffffu, cnt, owner);
            const int oex = __shfl_sync(0xffffffffu, excl, owner);
            const int olo = __shfl_sync(0xffffffffu, lo, owner);
            const bool valid = p < total && ocnt > 0 && p - oex < ocnt;
            const int kuc = olo + (p - oex);
            fn(valid ? base + owner : -1, kuc);
        }
    }
}

// Tiled gather: one warp per TS x TS tile of tap-window origins.  The warp
// stages its tile plus a (2m - 1) halo of the padded plane in shared memory
// and evaluates exactly the points whose window origin (j0 - m + 1 in both
// axes, unwrapped) falls in the tile or one of its periodic images, one point
// per lane with the point list flattened across slice lines.  Each point is
// owned by exactly one (tile, image), so every output is written once.
template <typename T, int TPB, int MH>
__global__ void __launch_bounds__(TPB * 32) k_gather2d_tiled(const C<T>* __restrict__ P, C<T>* __restrict__ out,
                                                             const C<T>* __restrict__ sub, int kv0, Usfft2dArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int nt = 2 * MH;
    const int TS = a.TS;
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
    const T hb = (T)TS * (T)0.5 + (T)1;
    for (int ix = -a.nimg; ix <= a.nimg; ++ix) {
        const int bx0 = tx0 + ix * a.M1;
        for (int iy = -a.nimg; iy <= a.nimg; ++iy) {
            const int by0 = ty0 + iy * a.M2;
            // positions whose window origin is in [b0, b0 + TS): p in [b0 + m - 1, b0 + TS + m - 1)
            const T cx = (T)(bx0 + a.m - 1) + (T)TS * (T)0.5, cy = (T)(by0 + a.m - 1) + (T)TS * (T)0.5;
            if (sqrt(cx * cx + cy * cy) > a.rmax + hb * (T)1.5) continue;
            for_tile_points<T>(a, kvc, cx, cy, hb, (T)(bx0 + a.m - 1), (T)(bx0 + TS + a.m - 1),
                               (T)(by0 + a.m - 1), (T)(by0 + TS + a.m - 1), [&](int th, int kuc) {
                if (th < 0) return;
                const typename AngleT<T>::type g = a.ang[th];
                int jx, jy;
                T fx, fy;
                point_pos(g, kuc, kvc, jx, fx, jy, fy);
                const int ox = jx - a.m + 1 - bx0, oy = jy - a.m + 1 - by0;
                if (ox < 0 || ox >= TS || oy < 0 || oy >= TS) return;
                T wy[nt];
#pragma unroll
                for (int t = 0; t < nt; ++t) {
                    const T d = fy + (T)(MH - 1 - t);
                    wy[t] = gexp(-d * d * a.inv4beta);
                }
                T sr = 0, si = 0;
#pragma unroll
                for (int sx = 0; sx < nt; ++sx) {
                    const T d = fx + (T)(MH - 1 - sx);
                    const T wx = gexp(-d * d * a.inv4beta);
                    const C<T>* rowp = st + (ox + sx) * SW + oy;
                    T rr = 0, ri = 0;
#pragma unroll
                    for (int t = 0; t < nt; ++t) {
                        const C<T> pv = rowp[t];
                        rr += wy[t] * pv.x;
                        ri += wy[t] * pv.y;
                    }
                    sr += wx * rr;
                    si += wx * ri;
                }
                const size_t o = ((size_t)th * a.h + kv) * a.w + (kuc + a.w / 2);
                C<T> v = cmake<T>(sr, si);
                if (sub) v = csub(v, sub[o]);
                out[o] = v;
            });
        }
    }
}

// One warp owns one TS x TS tile of the padded plane and an accumulator for
// it (sum and compensation in separate arrays; compensated in FP32); a block
// holds TPB tiles.  The points that may reach the tile come from
// for_tile_points, 32 per round, one per lane; each lane computes its point's
// tap window and 2 x 2m Gaussian weights in registers, and the warp steps
// through the (2m)^2 taps in lock-step.  Lanes whose window origins coincide
// (points of different lines can share one) are ranked with __match_any_sync
// and take successive passes, so within a pass no two lanes touch one cell.
template <typename T> struct AccArr;
template <> struct AccArr<float> {
    C<float>* s;
    C<float>* c;
    __device__ __forceinline__ void add(int i, float vr, float vi) {
        C<float> sum = s[i], cmp = c[i];
        const float yr = vr - cmp.x, yi = vi - cmp.y;
        const float tr = sum.x + yr, ti = sum.y + yi;
        cmp.x = (tr - sum.x) - yr;
        cmp.y = (ti - sum.y) - yi;
        s[i] = cmake<float>(tr, ti);
        c[i] = cmp;
    }
};
template <> struct AccArr<double> {
    C<double>* s;
    C<double>* c;
    __device__ __forceinline__ void add(int i, double vr, double vi) {
        C<double> sum = s[i];
        s[i] = cmake<double>(sum.x + vr, sum.y + vi);
    }
};

template <typename T, int TPB, int MH>
__global__ void __launch_bounds__(TPB * 32, sizeof(T) == 4 ? 4 : 1) k_scatter2d(const C<T>* __restrict__ in, C<T>* __restrict__ P,
                                                        int kv0, Usfft2dArgs<T> a) {
    constexpr int nt = 2 * MH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TS = a.TS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_x = a.M1 / TS, tiles_y = a.M2 / TS;
    const int tile = blockIdx.x * TPB + warp;
    if (tile >= tiles_x * tiles_y) return;  // whole warp exits; no block-wide sync below
    const int ncell = TS * TS;
    AccArr<T> acc;
    acc.s = reinterpret_cast<C<T>*>(smem_raw) + (size_t)warp * 2 * ncell;
    acc.c = acc.s + ncell;
    for (int i = lane; i < 2 * ncell; i += 32) acc.s[i] = cmake<T>(0, 0);
    __syncwarp();
    const int tx0 = (tile / tiles_y) * TS, ty0 = (tile % tiles_y) * TS;
    const int b = blockIdx.y, kv = kv0 + b, kvc = kv - a.h / 2;
    const T hb = (T)(TS + 2 * a.m) * (T)0.5;
    for (int ix = -a.nimg; ix <= a.nimg; ++ix) {
        const int bx0 = tx0 + ix * a.M1;
        for (int iy = -a.nimg; iy <= a.nimg; ++iy) {
            const int by0 = ty0 + iy * a.M2;
            const T cx = (T)bx0 + (T)(TS - 1) * (T)0.5, cy = (T)by0 + (T)(TS - 1) * (T)0.5;
            if (sqrt(cx * cx + cy * cy) > a.rmax + hb * (T)1.5) continue;
            for_tile_points<T>(a, kvc, cx, cy, hb, (T)(bx0 - a.m), (T)(bx0 + TS + a.m - 1), (T)(by0 - a.m),
                               (T)(by0 + TS + a.m - 1), [&](int th, int kuc) {
                bool act = th >= 0;
                int ox = 0, oy = 0;
                T wx[nt], wy[nt];
                C<T> v = cmake<T>(0, 0);
                if (act) {
                    const typename AngleT<T>::type g = a.ang[th];
                    int jx, jy;
                    T fx, fy;
                    point_pos(g, kuc, kvc, jx, fx, jy, fy);
                    ox = jx - a.m + 1 - bx0;
                    oy = jy - a.m + 1 - by0;
                    // no tap inside the tile: drop the point
                    act = ox > -nt && ox < TS && oy > -nt && oy < TS;
                    if (act) {
#pragma unroll
                        for (int t = 0; t < nt; ++t) {
                            const T dx = fx + (T)(MH - 1 - t), dy = fy + (T)(MH - 1 - t);
                            wx[t] = gexp(-dx * dx * a.inv4beta);
                            wy[t] = gexp(-dy * dy * a.inv4beta);
                        }
                        v = in[((size_t)th * a.h + kv) * a.w + (kuc + a.w / 2)];
                    }
                }
                const unsigned amask = __ballot_sync(0xffffffffu, act);
                if (amask == 0) return;
                // rank lanes that share a window origin
                const int key = act ? ((ox + 64) << 10) | (oy + 64) : -1 - lane;
                const unsigned peers = __match_any_sync(0xffffffffu, key);
                const int rank = act ? __popc(peers & ((1u << lane) - 1)) : 0;
                int maxrank = rank;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) maxrank = max(maxrank, __shfl_xor_sync(0xffffffffu, maxrank, o));
                for (int r = 0; r <= maxrank; ++r) {
                    const bool go = act && rank == r;
#pragma unroll
                    for (int sx = 0; sx < nt; ++sx) {
                        const int cxx = ox + sx;
                        const bool rowin = go && cxx >= 0 && cxx < TS;
                        const T wxs = wx[sx];
#pragma unroll
                        for (int sy = 0; sy < nt; ++sy) {
                            const int cyy = oy + sy;
                            if (rowin && cyy >= 0 && cyy < TS) {
                                const T wgt = wxs * wy[sy];
                                acc.add(cxx * TS + cyy, wgt * v.x, wgt * v.y);
                            }
                            __syncwarp();
                        }
                    }
                }
            });
        }
    }
    __syncwarp();
    C<T>* pl = P + (size_t)b * a.M1 * a.M2;
    for (int i = lane; i < ncell; i += 32) {
        const int cxx = i / TS, cyy = i - cxx * TS;
        pl[(size_t)(tx0 + cxx) * a.M2 + ty0 + cyy] = acc.s[i];
    }
}

// Fast scatter: the same tile ownership and point enumeration, but each lane
// spreads its own point's (2m)^2 taps independently with shared-memory atomic
// adds into one FP32 (or FP64) accumulator per tile.  No lock-step, no rank
// passes; the summation order inside a cell depends on scheduling, so results
// agree with the deterministic kernel to rounding, not bit for bit.
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

// Accumulator cells for the atomic scatter (ACC: 0 plain, 1 compensated, 2 FP64).
template <typename T, int ACC> struct AtomAcc {
    T* base;
    int ncell;
    __device__ __forceinline__ void zero(int lane) {
        for (int i = lane; i < 2 * ncell * (ACC == 1 ? 2 : 1); i += 32) base[i] = (T)0;
    }
    __device__ __forceinline__ void add(int cell, T vr, T vi) {
        if (ACC == 1) {
            // the atomic returns the value it added to; two-sum recovers the
            // exact rounding error of the stored sum, which goes to the second half
            const T ar = atomicAdd(base + 2 * cell, vr), ai = atomicAdd(base + 2 * cell + 1, vi);
            // (_rn intrinsics: no fma contraction with the product that formed v)
            const T sr = add_rn(ar, vr), si = add_rn(ai, vi);
            const T br = sub_rn(sr, ar), bi = sub_rn(si, ai);
            const T er = add_rn(sub_rn(ar, sub_rn(sr, br)), sub_rn(vr, br));
            const T ei = add_rn(sub_rn(ai, sub_rn(si, bi)), sub_rn(vi, bi));
            atomicAdd(base + 2 * ncell + 2 * cell, er);
            atomicAdd(base + 2 * ncell + 2 * cell + 1, ei);
        } else {
            atomicAdd(base + 2 * cell, vr);
            atomicAdd(base + 2 * cell + 1, vi);
        }
    }
    __device__ __forceinline__ C<T> get(int cell) const {
        if (ACC == 1) return cmake<T>(base[2 * cell] + base[2 * ncell + 2 * cell], base[2 * cell + 1] + base[2 * ncell + 2 * cell + 1]);
        return cmake<T>(base[2 * cell], base[2 * cell + 1]);
    }
};
template <typename T> struct AtomAcc<T, 2> {  // FP64 cells
    double* base;
    int ncell;
    __device__ __forceinline__ void zero(int lane) {
        for (int i = lane; i < 2 * ncell; i += 32) base[i] = 0.0;
    }
    __device__ __forceinline__ void add(int cell, T vr, T vi) {
        atomicAdd(base + 2 * cell, (double)vr);
        atomicAdd(base + 2 * cell + 1, (double)vi);
    }
    __device__ __forceinline__ C<T> get(int cell) const { return cmake<T>((T)base[2 * cell], (T)base[2 * cell + 1]); }
};
template <typename T, int ACC> __host__ __device__ constexpr int atom_acc_bytes() {
    return ACC == 2 ? 16 : (ACC == 1 ? 4 * (int)sizeof(T) : 2 * (int)sizeof(T));
}

template <typename T, int TPB, int MH, int ACC>
__global__ void __launch_bounds__(TPB * 32, sizeof(T) == 4 ? 6 : 2) k_scatter2d_atomic(
    const C<T>* __restrict__ in, C<T>* __restrict__ P, int kv0, Usfft2dArgs<T> a) {
    constexpr int nt = 2 * MH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TS = a.TS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_x = a.M1 / TS, tiles_y = a.M2 / TS;
    const int tile = blockIdx.x * TPB + warp;
    if (tile >= tiles_x * tiles_y) return;
    const int ncell = TS * TS;
    AtomAcc<T, ACC> acc;
    acc.base = reinterpret_cast<decltype(acc.base)>(smem_raw + (size_t)warp * ncell * atom_acc_bytes<T, ACC>());
    acc.ncell = ncell;
    acc.zero(lane);
    __syncwarp();
    const int tx0 = (tile / tiles_y) * TS, ty0 = (tile % tiles_y) * TS;
    const int b = blockIdx.y, kv = kv0 + b, kvc = kv - a.h / 2;
    const T hb = (T)(TS + 2 * a.m) * (T)0.5;
    for (int ix = -a.nimg; ix <= a.nimg; ++ix) {
        const int bx0 = tx0 + ix * a.M1;
        for (int iy = -a.nimg; iy <= a.nimg; ++iy) {
            const int by0 = ty0 + iy * a.M2;
            const T cx = (T)bx0 + (T)(TS - 1) * (T)0.5, cy = (T)by0 + (T)(TS - 1) * (T)0.5;
            if (sqrt(cx * cx + cy * cy) > a.rmax + hb * (T)1.5) continue;
            for_tile_points<T>(a, kvc, cx, cy, hb, (T)(bx0 - a.m), (T)(bx0 + TS + a.m - 1), (T)(by0 - a.m),
                               (T)(by0 + TS + a.m - 1), [&](int th, int kuc) {
                if (th < 0) return;
                const typename AngleT<T>::type g = a.ang[th];
                int jx, jy;
                T fx, fy;
                point_pos(g, kuc, kvc, jx, fx, jy, fy);
                const int ox = jx - MH + 1 - bx0, oy = jy - MH + 1 - by0;
                if (ox <= -nt || ox >= TS || oy <= -nt || oy >= TS) return;
                const C<T> v = in[((size_t)th * a.h + kv) * a.w + (kuc + a.w / 2)];
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
    __syncwarp();
    C<T>* pl = P + (size_t)b * a.M1 * a.M2;
    for (int i = lane; i < ncell; i += 32) {
        const int cxx = i / TS, cyy = i - cxx * TS;
        pl[(size_t)(tx0 + cxx) * a.M2 + ty0 + cyy] = acc.get(i);
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
    const dim3 grid((ntiles + NW - 1) / NW, nb);
    switch (a.m) {
#define LAM_G(MH) case MH: k_gather2d_tiled<T, NW, MH><<<grid, NW * 32, sg, s>>>(P, out, sub, kv0, a); break;
        LAM_G(2) LAM_G(3) LAM_G(4) LAM_G(5) LAM_G(6) LAM_G(7) LAM_G(8)
#undef LAM_G
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_usfft2d_adj(const C<T>* in, C<T>* P, C<T>* u1, int kv0, int nb, const Usfft2dArgs<T>& a,
                               cudaStream_t s) {
    constexpr int NW = kScatterWarps;
    const size_t sa = (size_t)NW * 2 * a.TS * a.TS * sizeof(C<T>);
    const int ntiles = (a.M1 / a.TS) * (a.M2 / a.TS);
    const size_t sr = (size_t)a.RB * a.M2 * sizeof(C<T>);
    const size_t sc = (size_t)a.CB * a.M1 * sizeof(C<T>);
    const dim3 grid((ntiles + NW - 1) / NW, nb);
    if (a.deterministic) {
        switch (a.m) {
#define LAM_S(MH) case MH: k_scatter2d<T, NW, MH><<<grid, NW * 32, sa, s>>>(in, P, kv0, a); break;
            LAM_S(2) LAM_S(3) LAM_S(4) LAM_S(5) LAM_S(6) LAM_S(7) LAM_S(8)
#undef LAM_S
            default: return cudaErrorInvalidValue;
        }
    } else {
        const int accm = a.scatter_acc;
        const size_t cells = (size_t)NW * a.TS * a.TS;
#define LAM_S(MH, ACC)                                                                                   \
    case MH:                                                                                             \
        k_scatter2d_atomic<T, NW, MH, ACC><<<grid, NW * 32, cells * atom_acc_bytes<T, ACC>(), s>>>(in, P, \
                                                                                                kv0, a); \
        break;
#define LAM_SW(ACC)                                                                              \
    switch (a.m) {                                                                               \
        LAM_S(2, ACC) LAM_S(3, ACC) LAM_S(4, ACC) LAM_S(5, ACC) LAM_S(6, ACC) LAM_S(7, ACC) LAM_S(8, ACC) \
        default: return cudaErrorInvalidValue;                                                   \
    }
        if (accm == 0) { LAM_SW(0) }
        else if (accm == 2) { LAM_SW(2) }
        else { LAM_SW(1) }
#undef LAM_SW
#undef LAM_S
    }
    k_colfft_adj<T><<<dim3(a.M2 / a.CB, nb), kFftThreads, sc, s>>>(P, a);
    k_rowfft_adj<T><<<dim3(a.n1 / a.RB, nb), kFftThreads, sr, s>>>(P, u1, kv0, a);
    return cudaGetLastError();
}

template <typename T> cudaError_t configure_usfft2d() {
    const int mx = kMaxDynSmem;
    cudaError_t e = cudaSuccess;
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (!e) e = cudaFuncSetAttribute(k_rowfft_fwd<T>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_colfft_fwd<T>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_rowfft_adj<T>, at, mx);
    if (!e) e = cudaFuncSetAttribute(k_colfft_adj<T>, at, mx);
#define LAM_A(MH)                                                                          \
    if (!e) e = cudaFuncSetAttribute(k_scatter2d<T, kScatterWarps, MH>, at, mx);          \
    if (!e) e = cudaFuncSetAttribute(k_gather2d_tiled<T, kScatterWarps, MH>, at, mx);       \
    if (!e) e = cudaFuncSetAttribute(k_scatter2d_atomic<T, kScatterWarps, MH, 0>, at, mx);  \
    if (!e) e = cudaFuncSetAttribute(k_scatter2d_atomic<T, kScatterWarps, MH, 1>, at, mx);  \
    if (!e) e = cudaFuncSetAttribute(k_scatter2d_atomic<T, kScatterWarps, MH, 2>, at, mx);
    LAM_A(2) LAM_A(3) LAM_A(4) LAM_A(5) LAM_A(6) LAM_A(7) LAM_A(8)
#undef LAM_A
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
template cudaError_t configure_usfft2d<float>();
template cudaError_t configure_usfft2d<double>();

}  // namespace lam
