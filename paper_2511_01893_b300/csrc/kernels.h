// kernels.h - argument blocks and launchers of the laminography kernels
// (internal to liblamino; the public ABI is include/lamino.h).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace lam {

// dynamic shared memory opt-in granted to every kernel (227 KB, the sm_100+
// per-block maximum); set once per plan creation so launches need no
// attribute calls (and stay legal under stream capture).
constexpr int kMaxDynSmem = 227 * 1024;

// adjoint spread variants (F*_u2D): per-warp tiles without atomics
// (deterministic, default), plain shared-memory atomic adds, or exact
// fixed-point shared-memory atomics (deterministic and correctly rounded)
constexpr int kSpreadTiles = 0;
constexpr int kSpreadAtomic = 1;
constexpr int kSpreadExact = 3;

template <typename T> cudaError_t configure_usfft1d();
template <typename T> cudaError_t configure_usfft2d();
template <typename T> cudaError_t configure_fft2d();

// ---- F_u1D -----------------------------------------------------------------
template <typename T> struct Usfft1dArgs {
    int n1, nz, n2, h;
    int M0, fcz;       // fcz: FFT stage code of length nz (fft_code)
    int m;             // half-width; 2m taps
    int TY;            // columns per block (divides n2)
    const T* dz;       // [nz] deapodisation along z
    const int* j0z;    // [h] floor(M0 xi_z(kv))
    const T* wz;       // [h][2m] Gaussian weights of taps j0z - m + 1 + t
    const int* kvlo;   // [jmax - jmin + 1] first kv whose taps reach unwrapped cell e
    const int* kvhi;   // one past the last such kv
    int jmin, jmax;    // unwrapped cell range touched by any tap
    const C<T>* tw;    // twiddles exp(-2 pi i q / Nmax)
    int twstride;      // Nmax / M0
    const int* skip;   // [h] or nullptr: planes that are mirrors of a paired plane
                       // (forward: not written; transpose: read as zero)
};

template <typename T>
cudaError_t launch_usfft1d_fwd(const T* u, C<T>* u1, const Usfft1dArgs<T>& a, cudaStream_t s);
template <typename T>
cudaError_t launch_usfft1d_adj(const C<T>* u1, T* u, const Usfft1dArgs<T>& a, cudaStream_t s);

// ---- F_u2D -----------------------------------------------------------------
template <typename T> struct AngleT;
template <> struct AngleT<float> { typedef AngleF type; };
template <> struct AngleT<double> { typedef AngleD type; };

template <typename T> struct Usfft2dArgs {
    int n1, n2, h, w, T_;          // T_ = number of angles
    int M1, M2, fcM1, fcM2;         // fc*: FFT stage codes (fft_code)
    int m;
    T inv4beta;                     // 1 / (4 beta)
    const T* d1;                    // [n1] deapodisation along x
    const T* d2;                    // [n2] deapodisation along y
    const typename AngleT<T>::type* ang;   // [T_] slice-coordinate constants
    const C<T>* tw;
    int tw1, tw2;                   // Nmax / M1, Nmax / M2
    int RB;                         // rows per block (row passes)
    int CB;                         // columns per block (column passes)
    int TS;                         // scatter tile side
    int TG;                         // gather tile side
    int nimg;                       // tile images +-1..nimg checked per line (unwrapped positions)
    T rmax;                         // bound on |slice position| in grid units
    int pstride;                    // scatter: lanes take points this far apart along a line
    int spread;                     // adjoint spread: kSpreadTiles, kSpreadAtomic or kSpreadExact
    const int2* jobs;               // plane jobs: .x plane computed, .y its conjugate mirror plane or -1
    const T* maxabs;                // device scalar: max |re|, |im| of the scatter input (fixed point)
    float bound_count;              // bound on the products summed into one padded cell
};

// forward: plane jobs j0 .. j0 + nb - 1 of u1 ([h][n1][n2]) -> out ([T][h][w]),
// using the padded-plane buffer P ([nb][M1][M2]).  Job j computes plane
// jobs[j].x and, if jobs[j].y >= 0, its mirror plane from the same padded FFT
// (P_mirror[j] = conj P[-j]).  If sub != nullptr the output is the value minus
// sub (same layout as out).
template <typename T>
cudaError_t launch_usfft2d_fwd(const C<T>* u1, C<T>* P, C<T>* out, const C<T>* sub, int kv0, int nb,
                               const Usfft2dArgs<T>& a, cudaStream_t s);
// transpose: plane jobs j0 .. j0 + nb - 1 of in ([T][h][w]) -> u1 ([h][n1][n2]);
// a paired job spreads both planes (the mirror plane mirrored and conjugated)
// into one grid and writes u1[jobs[j].x] = u1'(kv) + conj u1'(-kv)
template <typename T>
cudaError_t launch_usfft2d_adj(const C<T>* in, C<T>* P, C<T>* u1, int kv0, int nb,
                               const Usfft2dArgs<T>& a, cudaStream_t s);

// max(|re|, |im|) over n complex values into the device scalar *out
template <typename T> cudaError_t launch_absmax(const C<T>* in, long long n, T* out, cudaStream_t s);

// ---- F_2D / F*_2D (centred, per angle) ----------------------------------------
template <typename T> struct Fft2dArgs {
    int T_, h, w, fch, fcw;         // fc*: FFT stage codes (fft_code)
    const C<T>* tw;
    int twh, tww;                   // Nmax / h, Nmax / w
};
// dir = -1: sum exp(-...), dir = +1: sum exp(+...); result scaled by `scale`
template <typename T>
cudaError_t launch_fft2d_angles(const C<T>* in, C<T>* out, int dir, T scale, const Fft2dArgs<T>& a,
                                cudaStream_t s);

}  // namespace lam
