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
constexpr int kSpreadHalo = 4;  // owner-tile spread with halos (one visit per point)
constexpr int kSpreadTilesExact = 5;  // per-warp tiles of 64-bit fixed-point cells (exact, no atomics)
constexpr int kSpreadTiles2 = 6;      // the tile spread with one point per half-warp (two tiles per warp)
constexpr int kSpreadSweep = 7;       // row sweep: window rows in registers, records sorted by window row

template <typename T> cudaError_t configure_usfft1d();
template <typename T> cudaError_t configure_usfft2d();
template <typename T> cudaError_t configure_fft2d();

// ---- F_u1D -----------------------------------------------------------------
template <typename T> struct Usfft1dArgs {
    int n1, nz, n2, h;
    int M0, fcz;       // fcz: FFT stage code of length nz (fft_code)
    int m;             // half-width; 2m taps
    int TY;            // columns per block (divides n2)
    int nthr;          // threads per block (256 or 512)
    const T* dz;       // [nz] deapodisation along z
    const int* j0z;    // [h] floor(M0 xi_z(kv))
    const T* wz;       // [h][2m] Gaussian weights of taps j0z - m + 1 + t
    const int* kvlo;   // [jmax - jmin + 1] first kv whose taps reach unwrapped cell e
    const int* kvhi;   // one past the last such kv
    const T* wzc;      // [jmax - jmin + 1][cw]: weight of kv kvlo[e] + i on cell e at i
    int cw;            // columns of wzc (most kv reaching one cell)
    const int* kvslo;  // kv range the transpose sums over per cell: kvlo / kvhi,
    const int* kvshi;  // or without the skipped (mirror) planes when paired
    int jmin, jmax;    // unwrapped cell range touched by any tap
    const C<T>* tw;    // twiddles exp(-2 pi i q / Nmax)
    int twstride;      // Nmax / M0
    const int* skip;   // [h] or nullptr: planes that are mirrors of a paired plane
                       // (forward: not written; transpose: read as zero)
    int* err;          // the plan's error word (index checks, LAM_BOUNDS_CHECK builds)
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
    int fthr;                       // threads per row / column FFT block (256 or 512)
    int TS;                         // scatter tile side
    int TG;                         // gather tile side
    int nimg;                       // tile images +-1..nimg checked per line (unwrapped positions)
    T rmax;                         // bound on |slice position| in grid units
    int pstride;                    // scatter: lanes take points this far apart along a line
    int spread;                     // adjoint spread: kSpreadTiles, kSpreadHalo, kSpreadAtomic or kSpreadExact
    C<T>* halo;                     // workspace of the halo spread: [nb][tiles][ext][ext] (ext = 32 + 2m - 1)
    const int2* jobs;               // plane jobs: .x plane computed, .y its conjugate mirror plane or -1
    const T* maxabs;                // device scalar: max |re|, |im| of the scatter input (fixed point)
    float bound_count;              // bound on the products summed into one padded cell
    int nacc;                       // tile spread: leading plane jobs (the centre planes, which
                                    // the paired job list puts first) spread with exact
                                    // fixed-point accumulation instead
    int* err;                       // the plan's error word (index checks, LAM_BOUNDS_CHECK builds)
    const int* memo_hit;            // adjoint with memoization: per plane job (absolute index), nonzero
                                    // = served from the cache, so the spread and inverse FFTs skip it
};

// forward: plane jobs j0 .. j0 + nb - 1 of u1 ([h][n1][n2]) -> out ([T][h][w]),
// using the padded-plane buffer P ([nb][M1][M2]).  Job j computes plane
// jobs[j].x and, if jobs[j].y >= 0, its mirror plane from the same padded FFT
// (P_mirror[j] = conj P[-j]).  If sub != nullptr the output is the value minus
// sub (same layout as out).
// shared memory of one tiled-gather block: the tile of window origins plus
// the (2m - 1) halo and one more row and column below (the shifted windows of
// mirror points next to grid nodes), rows padded to an odd stride
template <typename T> constexpr size_t gather_smem_bytes(int tg, int m) {
    return (size_t)(tg + 2 * m) * (size_t)(tg + 2 * m + 1) * sizeof(C<T>);
}
template <typename T>
cudaError_t launch_usfft2d_fwd(const C<T>* u1, C<T>* P, C<T>* out, const C<T>* sub, int kv0, int nb,
                               const Usfft2dArgs<T>& a, cudaStream_t s);
// transpose: plane jobs j0 .. j0 + nb - 1 of in ([T][h][w]) -> u1 ([h][n1][n2]);
// a paired job spreads both planes (the mirror plane mirrored and conjugated)
// into one grid and writes u1[jobs[j].x] = u1'(kv) + conj u1'(-kv)
template <typename T>
cudaError_t launch_spread2d(const C<T>* in, C<T>* P, int j0, int nb, const Usfft2dArgs<T>& a, cudaStream_t s);
template <typename T>
cudaError_t launch_usfft2d_adj(const C<T>* in, C<T>* P, C<T>* u1, int kv0, int nb,
                               const Usfft2dArgs<T>& a, cudaStream_t s);

// ---- memoization of F*_u2D per plane job ------------------------------------------
struct MemoArgs {
    int njobs, K;          // plane jobs; key samples per plane
    const int2* jobs;      // the paired job list
    const int* samples;    // [K] sample positions th * w + ku within a plane
    int h, w;
    long long plane;       // n1 * n2 (values per u1 plane)
    double tau;            // reuse when the cosine similarity of the keys exceeds tau
    int* hit;              // [njobs] this call: 1 = served from the cache
    int* valid;            // [njobs] the slot holds a value
    double* scale;         // [njobs] least-squares factor <now, cached> / |cached|^2 of a hit
    double* stats;         // [2]: hits, lookups (accumulated)
};
// keys of this call's input, gate against the cached keys: key[j] holds
// 2 planes x K complex samples (the mirror plane's half is zero when unpaired)
template <typename T>
cudaError_t launch_memo_lookup(const C<T>* in, T* key_cached, T* key_now, const MemoArgs& m, cudaStream_t s);
// after the plane stage: hits copy the cached plane (times the factor) into u1,
// misses store the computed plane and their key in the slot
template <typename T>
cudaError_t launch_memo_update(C<T>* u1, C<T>* val, T* key_cached, const T* key_now, const MemoArgs& m,
                               cudaStream_t s);

// max(|re|, |im|) over n complex values into the device scalar *out
template <typename T>
cudaError_t launch_usfft2d_planes(const C<T>* u1, C<T>* P, int j0, int nb, const Usfft2dArgs<T>& a, cudaStream_t s);
cudaError_t launch_fma_peak(float* sink, int blocks, int iters, cudaStream_t s);
// ints in the plan's self-test scratch (after its error word)
constexpr int kSelftestCells = 64;
cudaError_t launch_bounds_selftest(int* scratch, int index, int* err, cudaStream_t s);
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
// FBP ramp along the detector's u frequency, in place on [n_rows][w]:
// value *= c0 |ku| with |ku| read as 1/4 at ku = 0 (ku = iu - w/2)
template <typename T> cudaError_t launch_ramp(C<T>* io, long long n_rows, int w, T c0, cudaStream_t s);

// ---- batched operators -------------------------------------------------------
// A batch runs the plane-stage operators of up to kMaxBatch plans (of one
// precision and half-width, uneven sizes) in one persistent launch per stage:
// the grid strides over a work list that concatenates every problem's blocks;
// a block finds its problem from the prefix table, copies that problem's
// argument block into shared memory and runs the single-problem kernel body.
// All of a problem's plane jobs go in one launch (its workspace holds them).
constexpr int kMaxBatch = 32;
enum BatchStage { kBZFwd = 0, kBRowFwd, kBColFwd, kBGather, kBSpread, kBColAdj, kBRowAdj, kBZAdj, kBStages };

template <typename T> struct BatchTable {
    int count;
    int start[kBStages][kMaxBatch + 1];  // first work item of each problem (prefix of block counts)
    int gx[kBStages][kMaxBatch];         // block grid of each problem: x extent,
    int gy[kBStages][kMaxBatch];         // y extent (z follows)
    Usfft1dArgs<T> zf[kMaxBatch];        // z stage, forward and transpose shapes
    Usfft1dArgs<T> za[kMaxBatch];
    Usfft2dArgs<T> a2[kMaxBatch];
    C<T>* u1[kMaxBatch];                 // per-problem workspace pieces (bound at creation)
    C<T>* P[kMaxBatch];
    const void* in[kMaxBatch];           // per-call operands (set by launch_batch_ptrs)
    void* out[kMaxBatch];
};

struct BatchPtrs {
    const void* in[kMaxBatch];
    void* out[kMaxBatch];
};

// launch facts of one batched stage, fixed at batch creation
struct BatchLaunch {
    int grid;       // persistent grid (blocks)
    size_t smem;    // dynamic shared memory (maximum over the problems)
};

template <typename T> cudaError_t launch_batch_ptrs(BatchTable<T>* dev, const BatchPtrs& ptrs, int count, cudaStream_t s);
// stage launches; mixed: some problem has radix-3/5 FFT lengths; m: half-width
template <typename T>
cudaError_t launch_batch_z(const BatchTable<T>* dev, bool fwd, bool mixed, const BatchLaunch& L, cudaStream_t s);
template <typename T>
cudaError_t launch_batch_plane(const BatchTable<T>* dev, int stage, bool mixed, int m, const BatchLaunch& L,
                               cudaStream_t s);
// resident blocks per SM of a batched stage kernel with `smem` dynamic bytes
template <typename T> int batch_occupancy(int stage, bool mixed, int m, size_t smem);
template <typename T> int batch_occupancy_z(bool fwd, bool mixed, size_t smem);
template <typename T> cudaError_t configure_batch_plane();
// dynamic shared memory of the tile spread for half-width m
template <typename T> size_t spread_tiles_bytes(int m);
template <typename T> cudaError_t configure_batch_z();

}  // namespace lam
