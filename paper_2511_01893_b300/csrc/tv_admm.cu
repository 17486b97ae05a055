// tv_admm.cu - TV gradient / divergence and the fused ADMM-TV elementwise steps.
//
// Readings of the paper (which names the steps but not their discretisation):
//   grad  forward differences along x, z, y of u[x][z][y] with a zero
//         difference at the last index; div = -grad^T (Section 2, the nabla of
//         Algorithms 1 and 2).
//   LSP   G = Re L_hat^H r / (h w) - rho div(grad u - psi + lambda / rho),
//         Dai-Yuan direction p = -G + beta p, beta = ||G||^2 / <p, G - G_prev>,
//         exact line search gamma = -<G, p> / (||L_hat p||^2 / (h w) + rho ||grad p||^2),
//         u += gamma p and r += gamma L_hat p (r = L_hat u - d_hat kept by linearity).
//   RSP   psi = shrink_iso(grad u + lambda / rho, alpha / rho);
//         lambda += rho (grad u - psi); residuals r = ||grad u - psi||,
//         s = rho ||div(psi - psi_old)||; rho doubles if r > 10 s, halves if s > 10 r.
//
// Conditioning.  psi is close to grad u wherever the shrinkage is active, so
// grad u - psi (which enters both the LSP gradient and the multiplier update)
// is a small difference of two large numbers: formed from FP32 arrays it
// carries an absolute error of ~1e-7 |grad u|, i.e. ~1e-4 relative.  The state
// therefore stores the shrinkage residual e = grad u - psi itself, computed
// from its closed form (e = kappa z/|z| - lambda/rho where the shrinkage is
// active, e = grad u elsewhere, z = grad u + lambda/rho, kappa = alpha/rho),
// and each LSP accumulates its increment du = u - u_start separately, so that
// grad u - psi = grad du + e and psi - psi_old = grad du - (e - e_old) are
// formed without cancellation.  psi itself is never stored.
//
// Reductions are deterministic: each block folds its elements (FP32 partial
// sums of at most 8 terms per thread in the FP32 path, then FP64; threads take
// four consecutive voxels per pass, so their loads overlap), writes one
// FP64 partial per quantity, and the last block to finish sums the partials in
// a fixed order.  Scalars (rho, beta, gamma, norms) stay in device memory so a
// whole outer iteration can be replayed as a CUDA graph.
#include "admm.h"

namespace lam {

// ---------------------------------------------------------------------------
// indexing helpers
// ---------------------------------------------------------------------------

// forward difference of f at (x,z,y) along axis a (0: x, 1: z, 2: y)
template <typename T>
__device__ __forceinline__ T fdiff(const T* __restrict__ f, long long i, int x, int z, int y, int a, const Vol& v) {
    if (a == 0) return x + 1 < v.n1 ? f[i + (long long)v.nz * v.n2] - f[i] : (T)0;
    if (a == 1) return z + 1 < v.nz ? f[i + v.n2] - f[i] : (T)0;
    return y + 1 < v.n2 ? f[i + 1] - f[i] : (T)0;
}

__device__ __forceinline__ long long astride(int a, const Vol& v) {
    return a == 0 ? (long long)v.nz * v.n2 : (a == 1 ? (long long)v.n2 : 1LL);
}
__device__ __forceinline__ int acoord(int a, int x, int z, int y) { return a == 0 ? x : (a == 1 ? z : y); }
__device__ __forceinline__ int alen(int a, const Vol& v) { return a == 0 ? v.n1 : (a == 1 ? v.nz : v.n2); }

// Grid-stride walk over the volume four voxels at a time: a thread takes four
// consecutive y (n2 is a multiple of 4) and runs body(i, x, z, y) for each,
// fully unrolled, so the four voxels' loads are independent and in flight
// together.  after_quad() runs once per four voxels.
template <typename F, typename G>
__device__ __forceinline__ void for_voxel_quads(const Vol& v, F body, G after_quad) {
    const long long nq = v.N >> 2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nq; q += (long long)gridDim.x * blockDim.x) {
        const long long i0 = q << 2;
        int x, z, y;
        v.coords(i0, x, z, y);
#pragma unroll
        for (int k = 0; k < 4; ++k) body(i0 + k, x, z, y + k);
        after_quad();
    }
}

// ---------------------------------------------------------------------------
// quad access: four consecutive voxels (i0 a multiple of 4, so a 16-byte
// aligned FP32 vector; two 16-byte halves in FP64).  Volume arrays start on a
// 256-byte boundary and n2 is a multiple of 4, so the neighbouring quads at
// +-n2 and +-nz n2 are aligned too.
// ---------------------------------------------------------------------------

template <typename T> struct Q4 {
    T v[4];
};
__device__ __forceinline__ Q4<float> ld4(const float* __restrict__ p) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    return Q4<float>{{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Q4<double> ld4(const double* __restrict__ p) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    return Q4<double>{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(float* __restrict__ p, const Q4<float>& q) {
    *reinterpret_cast<float4*>(p) = make_float4(q.v[0], q.v[1], q.v[2], q.v[3]);
}
__device__ __forceinline__ void st4(double* __restrict__ p, const Q4<double>& q) {
    reinterpret_cast<double2*>(p)[0] = make_double2(q.v[0], q.v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(q.v[2], q.v[3]);
}
template <typename T> __device__ __forceinline__ Q4<T> zero4() { return Q4<T>{{(T)0, (T)0, (T)0, (T)0}}; }

// Grid-stride walk over the quads: body(i0, x, z, y0) once per quad, then
// after_quad().  The same traversal as for_voxel_quads.
template <typename F, typename G>
__device__ __forceinline__ void for_quads(const Vol& v, F body, G after_quad) {
    const long long nq = v.N >> 2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nq; q += (long long)gridDim.x * blockDim.x) {
        const long long i0 = q << 2;
        int x, z, y;
        v.coords(i0, x, z, y);
        body(i0, x, z, y);
        after_quad();
    }
}

// Forward differences of f for the four voxels of a quad along x, z, y, each
// zero at the last index (fdiff, with the quad's loads shared).
template <typename T> struct QuadDiff {
    Q4<T> c, d[3];
};
template <typename T>
__device__ __forceinline__ QuadDiff<T> quad_fdiff(const T* __restrict__ f, long long i0, int x, int z, int y0, const Vol& v) {
    QuadDiff<T> q;
    q.c = ld4(f + i0);
    const long long X = (long long)v.nz * v.n2, Z = v.n2;
    const Q4<T> fx = x + 1 < v.n1 ? ld4(f + i0 + X) : q.c;
    const Q4<T> fz = z + 1 < v.nz ? ld4(f + i0 + Z) : q.c;
    const T fy4 = y0 + 4 < v.n2 ? f[i0 + 4] : (T)0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        q.d[0].v[k] = x + 1 < v.n1 ? fx.v[k] - q.c.v[k] : (T)0;
        q.d[1].v[k] = z + 1 < v.nz ? fz.v[k] - q.c.v[k] : (T)0;
        const T nb = k < 3 ? q.c.v[k + 1] : fy4;
        q.d[2].v[k] = y0 + k + 1 < v.n2 ? nb - q.c.v[k] : (T)0;
    }
    return q;
}

// ---------------------------------------------------------------------------
// deterministic block + grid reduction of K doubles
// ---------------------------------------------------------------------------

template <int K>
__device__ void reduce_store(double (&val)[K], double* partials, unsigned int* counter, double* sc, int dst) {
    __shared__ double sh[K][32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double v = val[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < K; ++k) {
            double s = 0;
            for (int w = 0; w < nw; ++w) s += sh[k][w];
            partials[blockIdx.x * K + k] = s;
        }
        __threadfence();
        const unsigned int t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = 0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += ((volatile double*)partials)[b * K + k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh[k][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < K; ++k) {
            double s = 0;
            for (int w = 0; w < nw; ++w) s += sh[k][w];
            sc[dst + k] = s;
        }
        *counter = 0;
    }
}

// ---------------------------------------------------------------------------
// grad / div
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_grad(const T* __restrict__ u, T* __restrict__ g, Vol v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < v.N; i += (long long)gridDim.x * blockDim.x) {
        int x, z, y;
        v.coords(i, x, z, y);
        for (int a = 0; a < 3; ++a) g[a * v.N + i] = fdiff(u, i, x, z, y, a, v);
    }
}

// div p at one voxel: sum_a p_a[i] [i_a <= N_a - 2] - p_a[i - e_a] [i_a >= 1]
template <typename F>
__device__ __forceinline__ auto div_at(F pa, long long i, int x, int z, int y, const Vol& v) -> decltype(pa(0, 0LL)) {
    decltype(pa(0, 0LL)) s = 0;
    for (int a = 0; a < 3; ++a) {
        const int c = acoord(a, x, z, y), n = alen(a, v);
        if (c + 1 < n) s += pa(a, i);
        if (c >= 1) s -= pa(a, i - astride(a, v));
    }
    return s;
}

template <typename T>
__global__ void k_div(const T* __restrict__ p, T* __restrict__ out, Vol v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < v.N; i += (long long)gridDim.x * blockDim.x) {
        int x, z, y;
        v.coords(i, x, z, y);
        out[i] = div_at([&](int a, long long j) { return p[a * v.N + j]; }, i, x, z, y, v);
    }
}

// ---------------------------------------------------------------------------
// LSP steps
// ---------------------------------------------------------------------------

// G = Gd * inv_hw - rho * div(q),  q_a(j) = d_a du(j) + e_a(j) + lambda_a(j) / rho
// (= d_a u - psi_a + lambda_a / rho; du = 0 on the first CG step).
// Reduces ||G||^2, <p, G>, <p, G_prev> into sc[SC_GG..SC_GG+2].
// three blocks per SM (<= 85 registers): the kernel is load-latency bound, and
// 24 resident warps measured faster than 16 (at 98 registers) or 32 (at 64,
// with spills)
template <typename T>
__global__ void __launch_bounds__(256, 3) k_lsp_G(const T* __restrict__ Gd, const T* __restrict__ du,
                                               const T* __restrict__ e, const T* __restrict__ lam,
                                               const T* __restrict__ p, const T* __restrict__ Gprev,
                                               T* __restrict__ G, int first, AdmmRed r, Vol v) {
    const double rho_d = r.sc[SC_RHO];
    const T rho = (T)rho_d, irho = (T)(1.0 / rho_d), ihw = (T)r.sc[SC_INVHW];
    const long long N = v.N, X = (long long)v.nz * v.n2, Z = v.n2;
    double acc[3] = {0, 0, 0};
    T loc[3] = {0, 0, 0};
    int cnt = 0;
    for_quads(v, [&](long long i0, int x, int z, int y0) {
        // du at the quad and its six neighbour quads / values (grad du at i and
        // at i - e_a); e, lambda at the quad and at i - e_a
        Q4<T> uc = zero4<T>(), uxp = zero4<T>(), uxm = zero4<T>(), uzp = zero4<T>(), uzm = zero4<T>();
        T uym = 0, uyp = 0;
        if (!first) {
            uc = ld4(du + i0);
            if (x + 1 < v.n1) uxp = ld4(du + i0 + X);
            if (x >= 1) uxm = ld4(du + i0 - X);
            if (z + 1 < v.nz) uzp = ld4(du + i0 + Z);
            if (z >= 1) uzm = ld4(du + i0 - Z);
            if (y0 >= 1) uym = du[i0 - 1];
            if (y0 + 4 < v.n2) uyp = du[i0 + 4];
        }
        const Q4<T> e0 = ld4(e + i0), e1 = ld4(e + N + i0), e2 = ld4(e + 2 * N + i0);
        const Q4<T> l0 = ld4(lam + i0), l1 = ld4(lam + N + i0), l2 = ld4(lam + 2 * N + i0);
        const Q4<T> e0m = x >= 1 ? ld4(e + i0 - X) : zero4<T>(), l0m = x >= 1 ? ld4(lam + i0 - X) : zero4<T>();
        const Q4<T> e1m = z >= 1 ? ld4(e + N + i0 - Z) : zero4<T>(), l1m = z >= 1 ? ld4(lam + N + i0 - Z) : zero4<T>();
        const T e2m = y0 >= 1 ? e[2 * N + i0 - 1] : (T)0, l2m = y0 >= 1 ? lam[2 * N + i0 - 1] : (T)0;
        const Q4<T> gd = ld4(Gd + i0);
        Q4<T> pq = zero4<T>(), gp = zero4<T>();
        if (!first) {
            pq = ld4(p + i0);
            gp = ld4(Gprev + i0);
        }
        Q4<T> gout;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int y = y0 + k;
            const T c = uc.v[k];
            // q_a(j) = d_a du(j) + e_a(j) + lambda_a(j) / rho, as in div_at's order
            T sdiv = 0;
            if (x + 1 < v.n1) sdiv += (first ? (T)0 : uxp.v[k] - c) + e0.v[k] + l0.v[k] * irho;
            if (x >= 1) sdiv -= (first ? (T)0 : c - uxm.v[k]) + e0m.v[k] + l0m.v[k] * irho;
            if (z + 1 < v.nz) sdiv += (first ? (T)0 : uzp.v[k] - c) + e1.v[k] + l1.v[k] * irho;
            if (z >= 1) sdiv -= (first ? (T)0 : c - uzm.v[k]) + e1m.v[k] + l1m.v[k] * irho;
            const T ynext = k < 3 ? uc.v[k + 1] : uyp;
            const T yprev = k > 0 ? uc.v[k - 1] : uym;
            const T e2p = k > 0 ? e2.v[k - 1] : e2m, l2p = k > 0 ? l2.v[k - 1] : l2m;
            if (y + 1 < v.n2) sdiv += (first ? (T)0 : ynext - c) + e2.v[k] + l2.v[k] * irho;
            if (y >= 1) sdiv -= (first ? (T)0 : c - yprev) + e2p + l2p * irho;
            const T g = gd.v[k] * ihw - rho * sdiv;
            gout.v[k] = g;
            loc[0] += g * g;
            if (!first) {
                loc[1] += pq.v[k] * g;
                loc[2] += pq.v[k] * gp.v[k];
            }
        }
        st4(G + i0, gout);
    }, [&]() {
        if (++cnt == 2) {  // FP32 partials of at most 8 terms
            for (int k = 0; k < 3; ++k) { acc[k] += (double)loc[k]; loc[k] = 0; }
            cnt = 0;
        }
    });
    for (int k = 0; k < 3; ++k) acc[k] += (double)loc[k];
    reduce_store<3>(acc, r.partials, r.counter, r.sc, SC_GG);
}

// beta (Dai-Yuan, 0 on the first step) and <G, p_new> = -||G||^2 + beta <p_old, G>
__global__ void k_beta(double* sc, int first) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double GG = sc[SC_GG], pG = sc[SC_PG], pGp = sc[SC_PGP];
    double beta = 0.0;
    if (!first) {
        const double den = pG - pGp;
        beta = den != 0.0 ? GG / den : 0.0;
    }
    if (!isfinite(beta) || !isfinite(GG)) {
        sc[SC_STATUS] = -5.0;
        beta = 0.0;
    }
    sc[SC_BETA] = beta;
    sc[SC_GP] = -GG + (first ? 0.0 : beta * pG);
}

template <typename T>
__global__ void __launch_bounds__(256) k_lsp_p(const T* __restrict__ G, T* __restrict__ p, const double* sc, Vol v) {
    const T beta = (T)sc[SC_BETA];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < v.N; i += (long long)gridDim.x * blockDim.x)
        p[i] = -G[i] + beta * p[i];
}

// ||grad f||^2 into sc[dst]
template <typename T>
__global__ void __launch_bounds__(256) k_gradnorm2(const T* __restrict__ f, AdmmRed r, int dst, Vol v) {
    double acc[1] = {0};
    T loc = 0;
    int cnt = 0;
    for_quads(v, [&](long long i0, int x, int z, int y0) {
        const QuadDiff<T> q = quad_fdiff(f, i0, x, z, y0, v);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            for (int a = 0; a < 3; ++a) loc += q.d[a].v[k] * q.d[a].v[k];
    }, [&]() {
        if (++cnt == 2) { acc[0] += (double)loc; loc = 0; cnt = 0; }
    });
    acc[0] += (double)loc;
    reduce_store<1>(acc, r.partials, r.counter, r.sc, dst);
}

// ||c||^2 of a complex array into sc[dst]
template <typename T>
__global__ void __launch_bounds__(256) k_cnorm2(const C<T>* __restrict__ c, long long n, AdmmRed r, int dst) {
    double acc[1] = {0};
    T loc = 0;
    int cnt = 0;
    // four consecutive values per thread and pass (n is a multiple of 4), so
    // four independent loads are in flight per thread
    const long long nq = n >> 2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nq; q += (long long)gridDim.x * blockDim.x) {
        C<T> z[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) z[k] = c[4 * q + k];
#pragma unroll
        for (int k = 0; k < 4; ++k) loc += z[k].x * z[k].x + z[k].y * z[k].y;
        if (++cnt == 2) { acc[0] += (double)loc; loc = 0; cnt = 0; }
    }
    for (long long i = 4 * nq + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const C<T> z = c[i];
        loc += z.x * z.x + z.y * z.y;
    }
    acc[0] += (double)loc;
    reduce_store<1>(acc, r.partials, r.counter, r.sc, dst);
}

__global__ void k_gamma(double* sc) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double den = sc[SC_LP2] * sc[SC_INVHW] + sc[SC_RHO] * sc[SC_GRADP2];
    double g = den > 0.0 ? -sc[SC_GP] / den : 0.0;
    if (!isfinite(g)) {
        sc[SC_STATUS] = -5.0;
        g = 0.0;
    }
    sc[SC_GAMMA] = g;
}

// du = gamma p (first CG step) or du += gamma p; on the last step also u += du
template <typename T>
__global__ void __launch_bounds__(256) k_axpy_u(T* __restrict__ du, T* __restrict__ u, const T* __restrict__ p,
                                                int first, int last, const double* sc, Vol v) {
    const T g = (T)sc[SC_GAMMA];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < v.N; i += (long long)gridDim.x * blockDim.x) {
        const T d = first ? g * p[i] : du[i] + g * p[i];
        du[i] = d;
        if (last) u[i] += d;
    }
}

// r += gamma Lp; ||r||^2 into sc[SC_R2]
template <typename T>
__global__ void __launch_bounds__(256) k_axpy_r(C<T>* __restrict__ rr, const C<T>* __restrict__ Lp, long long n,
                                                AdmmRed r) {
    const T g = (T)r.sc[SC_GAMMA];
    double acc[1] = {0};
    T loc = 0;
    int cnt = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        C<T> a = rr[i];
        const C<T> b = Lp[i];
        a.x += g * b.x;
        a.y += g * b.y;
        rr[i] = a;
        loc += a.x * a.x + a.y * a.y;
        if (++cnt == 8) { acc[0] += (double)loc; loc = 0; cnt = 0; }
    }
    acc[0] += (double)loc;
    reduce_store<1>(acc, r.partials, r.counter, r.sc, SC_R2);
}

// a + b as hi + lo exactly (Knuth's two-sum; no contraction, no reassociation)
template <typename T> __device__ __forceinline__ T add_exact(T a, T b, T& err);
template <> __device__ __forceinline__ float add_exact<float>(float a, float b, float& err) {
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}
template <> __device__ __forceinline__ double add_exact<double>(double a, double b, double& err) {
    const double s = __dadd_rn(a, b), bb = __dsub_rn(s, a);
    err = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
    return s;
}
template <typename T> __device__ __forceinline__ T mul_rn(T a, T b);
template <> __device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }
template <> __device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }

// one component of the compensated update (hi, lo) += g b: the product's
// rounding error (an FMA gives it exactly) and the sum's two-sum error go to
// lo, which is then folded back (fast two-sum), so hi is the nearest value to
// hi + lo and the pair carries the residual to about twice the working precision
template <typename T> __device__ __forceinline__ void comp_axpy(T& hi, T& lo, T g, T b) {
    const T y = mul_rn(g, b);
    const T ey = fma(g, b, -y);
    T es;
    const T s = add_exact(hi, y, es);
    const T l = lo + (ey + es);
    hi = s + l;
    lo = l - (hi - s);
}

// (r, rlo) += gamma Lp with the residual carried as r + rlo; ||r + rlo||^2 into sc[SC_R2]
template <typename T>
__global__ void __launch_bounds__(256) k_axpy_r_comp(C<T>* __restrict__ rr, C<T>* __restrict__ rlo,
                                                     const C<T>* __restrict__ Lp, long long n, AdmmRed r) {
    const T g = (T)r.sc[SC_GAMMA];
    double acc[1] = {0};
    T loc = 0;
    int cnt = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        C<T> a = rr[i], l = rlo[i];
        const C<T> b = Lp[i];
        comp_axpy(a.x, l.x, g, b.x);
        comp_axpy(a.y, l.y, g, b.y);
        rr[i] = a;
        rlo[i] = l;
        loc += a.x * a.x + a.y * a.y;
        if (++cnt == 8) { acc[0] += (double)loc; loc = 0; cnt = 0; }
    }
    acc[0] += (double)loc;
    reduce_store<1>(acc, r.partials, r.counter, r.sc, SC_R2);
}

// ---------------------------------------------------------------------------
// RSP, multiplier, residuals
// ---------------------------------------------------------------------------

// psi = shrink(z, kappa), z = grad u + lambda / rho, kappa = alpha / rho, held as
// e = grad u - psi; lambda += rho e; dpsi = psi - psi_old = grad du - (e - e_old).
// Reduces ||e||^2 (the primal residual r^2) and TV(u) into sc[SC_RP2], sc[SC_TVSUM].
template <typename T>
__global__ void __launch_bounds__(256) k_rsp(const T* __restrict__ u, const T* __restrict__ du, T* __restrict__ e,
                                             T* __restrict__ lam, T* __restrict__ dpsi, AdmmRed r, Vol v) {
    const double rho_d = r.sc[SC_RHO];
    const T rho = (T)rho_d, irho = (T)(1.0 / rho_d), kappa = (T)(r.sc[SC_ALPHA] / rho_d);
    const long long N = v.N;
    double acc[2] = {0, 0};
    T loc[2] = {0, 0};
    int cnt = 0;
    for_quads(v, [&](long long i0, int x, int z, int y0) {
        const QuadDiff<T> gq = quad_fdiff(u, i0, x, z, y0, v);
        const QuadDiff<T> dq = quad_fdiff(du, i0, x, z, y0, v);
        Q4<T> lq[3], eq[3], en4[3], ln4[3], dp4[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lq[a] = ld4(lam + a * N + i0);
            eq[a] = ld4(e + a * N + i0);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            T gu[3], zz[3], lm[3];
            T m2 = 0, g2 = 0;
            for (int a = 0; a < 3; ++a) {
                gu[a] = gq.d[a].v[k];
                lm[a] = lq[a].v[k];
                zz[a] = gu[a] + lm[a] * irho;
                m2 += zz[a] * zz[a];
                g2 += gu[a] * gu[a];
            }
            const T mag = sqrt(m2);
            const bool active = mag > kappa;
            const T kz = active ? kappa / mag : (T)0;
            T e2 = 0;
            for (int a = 0; a < 3; ++a) {
                const T en = active ? kz * zz[a] - lm[a] * irho : gu[a];
                const T ln = active ? rho * kz * zz[a] : lm[a] + rho * gu[a];
                dp4[a].v[k] = dq.d[a].v[k] - (en - eq[a].v[k]);
                en4[a].v[k] = en;
                ln4[a].v[k] = ln;
                e2 += en * en;
            }
            loc[0] += e2;
            loc[1] += sqrt(g2);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            st4(dpsi + a * N + i0, dp4[a]);
            st4(e + a * N + i0, en4[a]);
            st4(lam + a * N + i0, ln4[a]);
        }
    }, [&]() {
        if (++cnt == 2) {
            acc[0] += (double)loc[0];
            acc[1] += (double)loc[1];
            loc[0] = loc[1] = 0;
            cnt = 0;
        }
    });
    acc[0] += (double)loc[0];
    acc[1] += (double)loc[1];
    reduce_store<2>(acc, r.partials, r.counter, r.sc, SC_RP2);
}

// ||div dpsi||^2 into sc[SC_SD2]
template <typename T>
__global__ void __launch_bounds__(256) k_divnorm2(const T* __restrict__ p, AdmmRed r, Vol v) {
    double acc[1] = {0};
    T loc = 0;
    int cnt = 0;
    for_voxel_quads(v, [&](long long i, int x, int z, int y) {
        const T d = div_at([&](int a, long long j) { return p[a * v.N + j]; }, i, x, z, y, v);
        loc += d * d;
    }, [&]() {
        if (++cnt == 2) { acc[0] += (double)loc; loc = 0; cnt = 0; }
    });
    acc[0] += (double)loc;
    reduce_store<1>(acc, r.partials, r.counter, r.sc, SC_SD2);
}

// Smoothed isotropic TV: value sum_i sqrt(|grad u|_i^2 + eps^2) into sc[dst] and,
// if g != nullptr, its gradient g = -div(grad u / sqrt(|grad u|^2 + eps^2)).
template <typename T>
__device__ __forceinline__ T tv_unit(const T* __restrict__ u, long long j, int x, int z, int y, int a, T eps2,
                                     const Vol& v) {
    const T g0 = fdiff(u, j, x, z, y, 0, v), g1 = fdiff(u, j, x, z, y, 1, v), g2 = fdiff(u, j, x, z, y, 2, v);
    const T ga = a == 0 ? g0 : (a == 1 ? g1 : g2);
    return ga / sqrt(g0 * g0 + g1 * g1 + g2 * g2 + eps2);
}

template <typename T>
__global__ void __launch_bounds__(256) k_tv_smooth(const T* __restrict__ u, T* __restrict__ g, T eps, AdmmRed r,
                                                   int dst, Vol v) {
    const T eps2 = eps * eps;
    double acc[1] = {0};
    T loc = 0;
    int cnt = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < v.N; i += (long long)gridDim.x * blockDim.x) {
        int x, z, y;
        v.coords(i, x, z, y);
        const T g0 = fdiff(u, i, x, z, y, 0, v), g1 = fdiff(u, i, x, z, y, 1, v), g2 = fdiff(u, i, x, z, y, 2, v);
        loc += sqrt(g0 * g0 + g1 * g1 + g2 * g2 + eps2);
        if (g) {
            auto nrm = [&](int a, long long j) -> T {
                int xx = x, zz = z, yy = y;
                if (j != i) {
                    if (a == 0) --xx;
                    else if (a == 1) --zz;
                    else --yy;
                }
                return tv_unit(u, j, xx, zz, yy, a, eps2, v);
            };
            g[i] = -div_at(nrm, i, x, z, y, v);
        }
        if (++cnt == 8) { acc[0] += (double)loc; loc = 0; cnt = 0; }
    }
    acc[0] += (double)loc;
    reduce_store<1>(acc, r.partials, r.counter, r.sc, dst);
}

// residuals, objective, history, penalty update, iteration count
__global__ void k_outer_scalars(double* sc, double* hist, int hist_cap) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double rho = sc[SC_RHO];
    const double rr = sqrt(sc[SC_RP2]);
    const double ss = rho * sqrt(sc[SC_SD2]);
    const double data2 = sc[SC_R2] * sc[SC_INVHW];
    const double obj = 0.5 * data2 + sc[SC_ALPHA] * sc[SC_TVSUM];
    sc[SC_RESID_R] = rr;
    sc[SC_RESID_S] = ss;
    sc[SC_DATA2] = data2;
    sc[SC_TV] = sc[SC_TVSUM];
    sc[SC_OBJ] = obj;
    if (!isfinite(obj) || !isfinite(rr) || !isfinite(ss)) sc[SC_STATUS] = -5.0;
    const int it = (int)sc[SC_ITER];
    if (it < hist_cap) {
        hist[4 * it + 0] = obj;
        hist[4 * it + 1] = rho;
        hist[4 * it + 2] = rr;
        hist[4 * it + 3] = ss;
    }
    if (sc[SC_ADAPT] != 0.0) {
        if (rr > 10.0 * ss) sc[SC_RHO] = 2.0 * rho;
        else if (ss > 10.0 * rr) sc[SC_RHO] = 0.5 * rho;
    }
    sc[SC_ITER] = it + 1;
}

// r = -d_hat (u = 0 at start), data weight, scalars
template <typename T>
__global__ void k_neg_copy(const C<T>* __restrict__ src, C<T>* __restrict__ dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const C<T> a = src[i];
        dst[i] = cmake<T>(-a.x, -a.y);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

static inline int egrid(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < kRedBlocks ? b : kRedBlocks);
}

template <typename T>
cudaError_t Admm<T>::grad(const T* u, T* g, cudaStream_t s) const {
    k_grad<T><<<egrid(v.N), 256, 0, s>>>(u, g, v);
    return cudaGetLastError();
}
template <typename T>
cudaError_t Admm<T>::div(const T* g, T* u, cudaStream_t s) const {
    k_div<T><<<egrid(v.N), 256, 0, s>>>(g, u, v);
    return cudaGetLastError();
}
template <typename T>
cudaError_t Admm<T>::lsp_G(const T* Gd, const T* du, const T* e, const T* lam, const T* p, const T* Gprev, T* G,
                           int first, const AdmmRed& r, cudaStream_t s) const {
    k_lsp_G<T><<<egrid(v.N), 256, 0, s>>>(Gd, du, e, lam, p, Gprev, G, first, r, v);
    k_beta<<<1, 32, 0, s>>>(r.sc, first);
    return cudaGetLastError();
}
template <typename T>
cudaError_t Admm<T>::lsp_p(const T* G, T* p, const AdmmRed& r, cudaStream_t s) const {
    k_lsp_p<T><<<egrid(v.N), 256, 0, s>>>(G, p, r.sc, v);
    k_gradnorm2<T><<<egrid(v.N), 256, 0, s>>>(p, r, SC_GRADP2, v);
    return cudaGetLastError();
}
template <typename T>
cudaError_t Admm<T>::lsp_update(T* du, T* u, const T* p, int first, int last, C<T>* res, C<T>* rlo, const C<T>* Lp,
                                long long nd, const AdmmRed& r, cudaStream_t s) const {
    k_cnorm2<T><<<egrid(nd), 256, 0, s>>>(Lp, nd, r, SC_LP2);
    k_gamma<<<1, 32, 0, s>>>(r.sc);
    k_axpy_u<T><<<egrid(v.N), 256, 0, s>>>(du, u, p, first, last, r.sc, v);
    if (rlo) k_axpy_r_comp<T><<<egrid(nd), 256, 0, s>>>(res, rlo, Lp, nd, r);
    else k_axpy_r<T><<<egrid(nd), 256, 0, s>>>(res, Lp, nd, r);
    return cudaGetLastError();
}
template <typename T>
cudaError_t Admm<T>::rsp(const T* u, const T* du, T* e, T* lam, T* dpsi, const AdmmRed& r, double* hist,
                         int hist_cap, cudaStream_t s) const {
    k_rsp<T><<<egrid(v.N), 256, 0, s>>>(u, du, e, lam, dpsi, r, v);
    k_divnorm2<T><<<egrid(v.N), 256, 0, s>>>(dpsi, r, v);
    k_outer_scalars<<<1, 32, 0, s>>>(r.sc, hist, hist_cap);
    return cudaGetLastError();
}
// out = a + b (the current LSP iterate u + du of the Algorithm 1 form)
template <typename T>
__global__ void k_vadd(const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] + b[i];
}

template <typename T>
cudaError_t Admm<T>::vadd(const T* a, const T* b, T* out, cudaStream_t s) const {
    k_vadd<T><<<egrid(v.N), 256, 0, s>>>(a, b, out, v.N);
    return cudaGetLastError();
}

// dst -= src (the data-space residual of the Algorithm 1 form)
template <typename T>
__global__ void k_csub(const C<T>* __restrict__ src, C<T>* __restrict__ dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const C<T> a = dst[i], b = src[i];
        dst[i] = cmake<T>(a.x - b.x, a.y - b.y);
    }
}

template <typename T>
cudaError_t Admm<T>::csub(const C<T>* src, C<T>* dst, long long n, cudaStream_t s) const {
    k_csub<T><<<egrid(n), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Admm<T>::neg_copy(const C<T>* src, C<T>* dst, long long n, cudaStream_t s) const {
    k_neg_copy<T><<<egrid(n), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}
template <typename T>
cudaError_t Admm<T>::residual_norm(const C<T>* res, long long n, const AdmmRed& r, cudaStream_t s) const {
    k_cnorm2<T><<<egrid(n), 256, 0, s>>>(res, n, r, SC_R2);
    return cudaGetLastError();
}

template <typename T>
cudaError_t Admm<T>::tv_smooth(const T* u, T* g, double eps, const AdmmRed& r, int dst, cudaStream_t s) const {
    k_tv_smooth<T><<<egrid(v.N), 256, 0, s>>>(u, g, (T)eps, r, dst, v);
    return cudaGetLastError();
}

template struct Admm<float>;
template struct Admm<double>;

}  // namespace lam
