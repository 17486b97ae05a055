// admm.h - TV and ADMM-TV elementwise launchers (internal).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace lam {

// Scalar slots in the state's FP64 array.  0..15 are public (lamino.h).
enum {
    SC_RHO = 0,
    SC_ALPHA = 1,
    SC_OBJ = 2,
    SC_RESID_R = 3,
    SC_RESID_S = 4,
    SC_ITER = 5,
    SC_DATA2 = 6,
    SC_TV = 7,
    SC_STATUS = 8,
    SC_MEMO_HITS = 9,     // plane jobs of the adjoint served from the memoization cache (accumulated)
    SC_MEMO_LOOKUPS = 10, // plane jobs looked up
    // internal
    SC_GG = 16,      // ||G||^2
    SC_PG = 17,      // <p_old, G>
    SC_PGP = 18,     // <p_old, G_prev>
    SC_BETA = 19,
    SC_GP = 20,      // <G, p_new>
    SC_GRADP2 = 21,  // ||grad p||^2
    SC_LP2 = 22,     // ||L_hat p||^2
    SC_GAMMA = 23,
    SC_R2 = 24,      // ||r||^2, r = L_hat u - d_hat
    SC_RP2 = 25,     // ||grad u - psi||^2
    SC_TVSUM = 26,   // TV(u)
    SC_SD2 = 27,     // ||div(psi - psi_old)||^2
    SC_INVHW = 28,   // 1 / (h w)
    SC_ADAPT = 29,   // penalty adaptation on/off
    SC_COUNT = 64
};

constexpr int kRedBlocks = 1184;  // 148 SMs x 8: grid of every reducing kernel
constexpr int kHistCap = 4096;

struct AdmmRed {
    double* sc;             // [SC_COUNT]
    double* partials;       // [kRedBlocks * 4]
    unsigned int* counter;  // zero between reductions
};

// volume [n1][nz][n2], N = n1 * nz * n2.  When nz and n2 are powers of two
// (ln2 = log2 n2, lnz = log2 nz) coordinates come from shifts and masks; else
// ln2 = lnz = -1 and they come from divisions (32-bit when N < 2^31).
struct Vol {
    int n1, nz, n2;
    int ln2, lnz;
    long long N;
    __device__ __forceinline__ void coords(long long i, int& x, int& z, int& y) const {
        if (ln2 >= 0) {
            y = (int)(i & (n2 - 1));
            const long long t = i >> ln2;
            z = (int)(t & (nz - 1));
            x = (int)(t >> lnz);
        } else if (N < (1LL << 31)) {
            const unsigned ii = (unsigned)i, t = ii / (unsigned)n2;
            y = (int)(ii - t * (unsigned)n2);
            const unsigned xx = t / (unsigned)nz;
            z = (int)(t - xx * (unsigned)nz);
            x = (int)xx;
        } else {
            const long long t = i / n2;
            y = (int)(i - t * n2);
            const long long xx = t / nz;
            z = (int)(t - xx * nz);
            x = (int)xx;
        }
    }
};

template <typename T> struct Admm {
    Vol v;
    cudaError_t grad(const T* u, T* g, cudaStream_t s) const;
    cudaError_t div(const T* g, T* u, cudaStream_t s) const;
    cudaError_t lsp_G(const T* Gd, const T* du, const T* e, const T* lam, const T* p, const T* Gprev, T* G,
                      int first, const AdmmRed& r, cudaStream_t s) const;
    cudaError_t lsp_p(const T* G, T* p, const AdmmRed& r, cudaStream_t s) const;
    // rlo != nullptr: the residual is carried as res + rlo (compensated)
    cudaError_t lsp_update(T* du, T* u, const T* p, int first, int last, C<T>* res, C<T>* rlo, const C<T>* Lp,
                           long long nd, const AdmmRed& r, cudaStream_t s) const;
    cudaError_t rsp(const T* u, const T* du, T* e, T* lam, T* dpsi, const AdmmRed& r, double* hist, int hist_cap,
                    cudaStream_t s) const;
    cudaError_t neg_copy(const C<T>* src, C<T>* dst, long long n, cudaStream_t s) const;
    cudaError_t csub(const C<T>* src, C<T>* dst, long long n, cudaStream_t s) const;
    cudaError_t vadd(const T* a, const T* b, T* out, cudaStream_t s) const;
    cudaError_t tv_smooth(const T* u, T* g, double eps, const AdmmRed& r, int dst, cudaStream_t s) const;
    cudaError_t residual_norm(const C<T>* res, long long n, const AdmmRed& r, cudaStream_t s) const;
};

}  // namespace lam
