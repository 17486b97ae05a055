// capi.cu - plans, geometry tables and the C ABI of liblamino (include/lamino.h).
//
// The plan computes every table in FP64 on the host (deapodisation factors,
// z-gather taps and weights, the kv ranges of the gather-form z spread,
// twiddles and per-angle slice-coordinate constants) and uploads them once.
// Operator calls only enqueue kernels on the caller's stream and use the
// caller's workspace; ADMM keeps all of its vectors and FP64 scalars in the
// caller's state buffer.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lamino.h"
#include "../../include/lamino_stages.h"
#include "admm.h"
#include "fft.cuh"
#include "kernels.h"

using namespace lam;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------

static thread_local std::string g_err;

static lam_status fail(lam_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(LAM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------

namespace {

struct AdmmHost {
    int n_inner = 4;
    int form = 2;  // LSP form: 2 (Algorithm 2, default) or 1 (Algorithm 1)
    int resid = 0;  // residual handling (LAM_OPT_RESIDUAL bits)
    double memo_tau = 0;  // memoization of F*_u2D (0: off)
    void* ws = nullptr;
    cudaGraphExec_t graph = nullptr;
    size_t graph_kernels = 0;  // kernel nodes in the captured outer iteration
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// NVTX range over a host scope: the stages show by name in a profiler's
// timeline (free when no profiler is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// plane jobs nearest the centre plane that an FP32 plan spreads exactly by
// default: kv = h/2 and the pairs h/2 +- 1, h/2 +- 2 (|kv - h/2| <= 2)
constexpr int kDefaultExactCentreJobs = 3;

static int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}
static bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

struct lam_plan {
    int n1, nz, n2, h, w, T, m, R, prec;
    int M0, M1, M2, Nmax;
    double phi, beta;
    int device;
    std::vector<void*> dev_allocs;
    // device tables
    void *dz, *d1, *d2, *wz, *tw, *ang;
    int *j0z, *kvlo, *kvhi;
    void* wzc;  // z weights cell by cell ([jmax - jmin + 1][zcw])
    int *kvplo, *kvphi;  // per cell: the kv range the paired transpose needs
    int zcw;
    int jmin, jmax;
    // plane jobs: paired (for real volumes) and one job per plane
    int2* jobs_pair;
    std::vector<int2> jobs_pair_h;  // host copy of jobs_pair
    int2* jobs_all;
    int* skip;  // [h] 1 for the mirror plane of a paired job
    int* err;   // error word of the index checks, then kSelftestCells ints of self-test scratch
    int njobs_pair;
    // launch shapes
    int TYf, TYa, RB, CB, TS, TG, nimg, nbatch;
    int zthr = kFftThreads, pthr = kFftThreads;  // threads per z-stage / plane-FFT block
    double rmax;
    int pstride;
    int spread = kSpreadTiles;
    int nacc = 0;  // leading plane jobs the tile spread accumulates exactly (LAM_OPT_EXACT_CENTRE_JOBS)
    int lsp_form = 2;  // LSP form new ADMM states take (LAM_OPT_LSP_FORM)
    int resid = 0;     // residual handling new ADMM states take (LAM_OPT_RESIDUAL)
    double memo_tau = 0;  // memoization threshold new ADMM states take (LAM_OPT_MEMO_TAU; 0: off)
    int* memo_samples = nullptr;  // [memo_K] key sample positions th * w + ku within a data plane
    int memo_K = 0;
    // workspace layout
    size_t ws_u1, ws_planes, ws_halo, ws_tmp, ws_red, ws_bytes;
    mutable std::mutex mu;
    mutable std::map<void*, AdmmHost> admm;

    size_t elem() const { return prec == LAM_F64 ? sizeof(double) : sizeof(float); }
    size_t celem() const { return 2 * elem(); }
    long long nvox() const { return (long long)n1 * nz * n2; }
    long long ndata() const { return (long long)T * h * w; }
};

// a batch of plans run together by the batched operators (lam_batch_create)
// side streams of a new batch's concurrent ADMM mode (8 and 16 measured alike
// on 16 problems of n = 96 .. 192)
constexpr int kDefaultBatchStreams = 8;

struct lam_batch {
    int count = 0;
    int prec = LAM_F32;
    int device = -1;
    int m = 4;
    bool mixed = false;  // some problem has radix-3/5 FFT lengths
    std::vector<const lam_plan*> plans;
    std::vector<void*> ws;
    void* dev = nullptr;  // BatchTable<T> in device memory
    BatchLaunch L[kBStages];
    int total[kBStages] = {};
    // ADMM graph of one outer iteration over the states it was captured for
    std::vector<void*> graph_states;
    cudaGraphExec_t graph = nullptr;
    size_t graph_kernels = 0;
    // concurrent mode (lam_batch_set_streams): side streams and fork / join events
    int nstreams = 0;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
};

namespace {

template <typename T> void* upload(lam_plan* p, const std::vector<T>& v, lam_status* st) {
    void* d = nullptr;
    if (cudaMalloc(&d, std::max<size_t>(v.size() * sizeof(T), 16)) != cudaSuccess) {
        *st = fail(LAM_ENOMEM, "cudaMalloc of %zu bytes for a plan table failed", v.size() * sizeof(T));
        return nullptr;
    }
    p->dev_allocs.push_back(d);
    if (!v.empty() && cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
        *st = fail(LAM_ECUDA, "upload of a plan table failed");
        return nullptr;
    }
    return d;
}

template <typename T> std::vector<T> cast_vec(const std::vector<double>& v) {
    return std::vector<T>(v.begin(), v.end());
}

// deapodisation 1/(M g^(x)) = exp(4 pi^2 beta x^2 / M^2) / sqrt(4 pi beta), x centred
std::vector<double> deapod(int N, int M, double beta) {
    std::vector<double> d(N);
    for (int i = 0; i < N; ++i) {
        const double x = i - N / 2;
        d[i] = std::exp(4.0 * M_PI * M_PI * beta * x * x / ((double)M * M)) / std::sqrt(4.0 * M_PI * beta);
    }
    return d;
}

template <typename T> lam_status build_tables(lam_plan* p, const double* theta) {
    lam_status st = LAM_OK;
    const double beta = p->beta;
    const int m = p->m, nt = 2 * m;
    p->dz = upload(p, cast_vec<T>(deapod(p->nz, p->M0, beta)), &st);
    if (st) return st;
    p->d1 = upload(p, cast_vec<T>(deapod(p->n1, p->M1, beta)), &st);
    if (st) return st;
    p->d2 = upload(p, cast_vec<T>(deapod(p->n2, p->M2, beta)), &st);
    if (st) return st;
    // z gather: xi_z = (kv - h/2)/h cos(phi), taps j0 - m + 1 + t with j0 = floor(M0 xi + kTapShift),
    // weights exp(-(M0 xi - j)^2/(4 beta))
    std::vector<int> j0(p->h);
    std::vector<double> wz((size_t)p->h * nt);
    const double cp = std::cos(p->phi);
    for (int kv = 0; kv < p->h; ++kv) {
        const double t = p->M0 * ((double)(kv - p->h / 2) / p->h * cp);
        const double f = std::floor(t + kTapShift);
        j0[kv] = (int)f;
        for (int q = 0; q < nt; ++q) {
            const double dd = t - (f - m + 1 + q);
            wz[(size_t)kv * nt + q] = std::exp(-dd * dd / (4.0 * beta));
        }
    }
    int jmin = j0[0] - m + 1, jmax = j0[0] + m;
    for (int kv = 0; kv < p->h; ++kv) {
        jmin = std::min(jmin, j0[kv] - m + 1);
        jmax = std::max(jmax, j0[kv] + m);
    }
    const int E = jmax - jmin + 1;
    std::vector<int> lo(E), hi(E);
    for (int e = 0; e < E; ++e) {
        const int cell = jmin + e;
        int l = p->h, r = 0;
        for (int kv = 0; kv < p->h; ++kv)
            if (j0[kv] - m + 1 <= cell && cell <= j0[kv] + m) {
                l = std::min(l, kv);
                r = std::max(r, kv + 1);
            }
        if (l >= r) l = r = 0;
        // j0 is non-decreasing in kv (cos phi >= 0), so the kv set is contiguous
        lo[e] = l;
        hi[e] = r;
    }
    p->jmin = jmin;
    p->jmax = jmax;
    p->j0z = (int*)upload(p, j0, &st);
    if (st) return st;
    p->wz = upload(p, cast_vec<T>(wz), &st);
    if (st) return st;
    p->kvlo = (int*)upload(p, lo, &st);
    if (st) return st;
    p->kvhi = (int*)upload(p, hi, &st);
    if (st) return st;
    // the same weights cell by cell: wzc[e][kv - lo[e]] for kv in [lo[e], hi[e])
    int cw = 1;
    for (int e = 0; e < E; ++e) cw = std::max(cw, hi[e] - lo[e]);
    std::vector<double> wzc((size_t)E * cw, 0.0);
    for (int e = 0; e < E; ++e)
        for (int kv = lo[e]; kv < hi[e]; ++kv)
            wzc[(size_t)e * cw + (kv - lo[e])] = wz[(size_t)kv * nt + (jmin + e - (j0[kv] - m + 1))];
    p->zcw = cw;
    p->wzc = upload(p, cast_vec<T>(wzc), &st);
    if (st) return st;
    // Hermitian pairs: for a real volume, u1 at -kv is the conjugate of u1 at kv
    // when the z windows of -kv mirror those of kv (j0(-t) = -j0(t) - 1; the
    // tap positions negate exactly); then one padded FFT serves both planes.
    {
        const int h = p->h;
        std::vector<int2> jp, ja;
        std::vector<int> skip(h, 0);
        auto generic = [&](int kv) {  // kv in [1, h/2 - 1], partner h - kv
            return j0[h - kv] == -j0[kv] - 1;
        };
        for (int kv = 0; kv <= h / 2; ++kv) {
            int2 j;
            j.x = kv;
            j.y = (kv >= 1 && kv <= h / 2 - 1 && generic(kv)) ? h - kv : -1;
            if (j.y >= 0) skip[j.y] = 1;
            jp.push_back(j);
        }
        for (int kv = h / 2 + 1; kv < h; ++kv)
            if (!generic(h - kv)) {
                int2 j;
                j.x = kv;
                j.y = -1;
                jp.push_back(j);
            }
        for (int kv = 0; kv < h; ++kv) {
            int2 j;
            j.x = kv;
            j.y = -1;
            ja.push_back(j);
        }
        // planes near kv = h/2 carry the densest tiles (every slice line passes
        // close to the origin there): run them first, so their heaviest blocks
        // start early instead of forming a tail
        std::stable_sort(jp.begin(), jp.end(),
                         [h](const int2& a, const int2& b) { return std::abs(a.x - h / 2) < std::abs(b.x - h / 2); });
        p->njobs_pair = (int)jp.size();
        p->jobs_pair_h = jp;
        p->jobs_pair = (int2*)upload(p, jp, &st);
        if (st) return st;
        p->jobs_all = (int2*)upload(p, ja, &st);
        if (st) return st;
        p->skip = (int*)upload(p, skip, &st);
        if (st) return st;
        p->err = (int*)upload(p, std::vector<int>(1 + kSelftestCells, 0), &st);
        if (st) return st;
        {
            // memoization key samples: K slice points per data plane at fixed
            // pseudo-random positions (a 64-bit LCG, seed fixed per plan shape)
            const long long nplane = (long long)p->T * p->w;
            p->memo_K = (int)std::min<long long>(1024, nplane);
            std::vector<int> pos(p->memo_K);
            unsigned long long x = 0x9E3779B97F4A7C15ull ^ (unsigned long long)nplane;
            for (int k = 0; k < p->memo_K; ++k) {
                x = x * 6364136223846793005ull + 1442695040888963407ull;
                pos[k] = (int)((x >> 17) % (unsigned long long)nplane);
            }
            p->memo_samples = (int*)upload(p, pos, &st);
            if (st) return st;
        }
        // the paired transpose's kv range per cell: the non-skipped kv of
        // [lo, hi) when they are contiguous (skipped planes carry zeros), else
        // the whole range
        std::vector<int> plo(E), phi(E);
        for (int e = 0; e < E; ++e) {
            int a = hi[e], b = lo[e];
            for (int kv = lo[e]; kv < hi[e]; ++kv)
                if (!skip[kv]) {
                    a = std::min(a, kv);
                    b = std::max(b, kv + 1);
                }
            bool contiguous = true;
            for (int kv = a; kv < b; ++kv)
                if (skip[kv]) contiguous = false;
            if (a >= b) a = b = lo[e];
            plo[e] = contiguous ? a : lo[e];
            phi[e] = contiguous ? b : hi[e];
        }
        p->kvplo = (int*)upload(p, plo, &st);
        if (st) return st;
        p->kvphi = (int*)upload(p, phi, &st);
        if (st) return st;
    }
    // twiddles exp(-2 pi i q / Nmax)
    std::vector<T> tw(2 * (size_t)p->Nmax);
    for (int q = 0; q < p->Nmax; ++q) {
        const double a = -2.0 * M_PI * q / p->Nmax;
        tw[2 * q] = (T)std::cos(a);
        tw[2 * q + 1] = (T)std::sin(a);
    }
    p->tw = upload(p, tw, &st);
    if (st) return st;
    // per-angle slice coordinates (grid units):
    //   x: ku * M1 cos th / w + kv * M1 sin phi sin th / h
    //   y: ku * M2 sin th / w - kv * M2 sin phi cos th / h
    const double sp = std::sin(p->phi);
    if (sizeof(T) == sizeof(float)) {
        std::vector<AngleF> ang(p->T);
        auto split = [](double v, float& hi, float& lo) {
            hi = (float)v;
            lo = (float)(v - (double)hi);
        };
        for (int k = 0; k < p->T; ++k) {
            const double c = std::cos(theta[k]), s = std::sin(theta[k]);
            split(p->M1 * c / p->w, ang[k].ax_hi, ang[k].ax_lo);
            split(p->M1 * sp * s / p->h, ang[k].sx_hi, ang[k].sx_lo);
            split(p->M2 * s / p->w, ang[k].ay_hi, ang[k].ay_lo);
            split(-p->M2 * sp * c / p->h, ang[k].sy_hi, ang[k].sy_lo);
        }
        p->ang = upload(p, ang, &st);
    } else {
        std::vector<AngleD> ang(p->T);
        for (int k = 0; k < p->T; ++k) {
            const double c = std::cos(theta[k]), s = std::sin(theta[k]);
            ang[k].ax = p->M1 * c / p->w;
            ang[k].sx = p->M1 * sp * s / p->h;
            ang[k].ay = p->M2 * s / p->w;
            ang[k].sy = -p->M2 * sp * c / p->h;
        }
        p->ang = upload(p, ang, &st);
    }
    return st;
}

// lines per block for the in-place FFT kernels: shared memory (extra + lines *
// len elements) within `budget`, lines * len within the register budget
// 8 * MAXB * threads, `divides` a multiple of lines, at most `cap`
// lines per block for an in-place FFT of length len: within the shared-memory
// budget, within the FFT's register capacity (lines * len <= capacity * 512
// threads), and dividing `divides` (the grid covers it exactly)
static int pick_lines(int len, size_t celem, size_t budget, int divides, int cap, int maxb, size_t extra_per_line = 0,
                      int threads = kFftThreads) {
    const long long capacity = (long long)fft_capacity(fft_code(len), maxb) * threads;
    int l = cap;
    while (l > 1 && ((size_t)l * ((len + len / 16 + 1) * celem + extra_per_line) > budget ||
                     (long long)l * len > capacity || divides % l != 0))
        l >>= 1;
    return l;
}

// z stage: TY columns per block (column pairs share one complex line; E and
// O halves are nz long each); plane FFTs: RB rows / CB columns per block.
// Each within the FFT's capacity for the stage's block size.
static void pick_fft_shapes(lam_plan* p) {
    const size_t ce_ = p->celem();
    // two blocks per SM: the compile-time-length z kernels run at ~60 registers
    const size_t budget = p->zthr <= 256 ? 56 * 1024 : 110 * 1024;
    const size_t pbudget = p->pthr <= 256 ? 64 * 1024 : 128 * 1024;
    const int maxb = p->prec == LAM_F32 ? 2 : 1;
    p->TYf = std::max(2, pick_lines(p->nz, ce_, budget, p->n2, 16, maxb, 0, p->zthr));
    p->TYa = std::max(2, pick_lines(p->nz, ce_, budget, p->n2, 16, maxb, (size_t)p->h * ce_, p->zthr));
    p->RB = pick_lines(p->M2, ce_, pbudget, p->n1, 16, maxb, 0, p->pthr);
    p->CB = pick_lines(p->M1, ce_, pbudget, p->M2, 16, maxb, 0, p->pthr);
}

template <typename T> Usfft1dArgs<T> args1d(const lam_plan* p, int TY, bool paired) {
    Usfft1dArgs<T> a;
    a.n1 = p->n1;
    a.nz = p->nz;
    a.n2 = p->n2;
    a.h = p->h;
    a.M0 = p->M0;
    a.fcz = fft_code(p->nz, fft_max_radix<T>());
    a.m = p->m;
    a.TY = TY;
    a.nthr = p->zthr;
    a.dz = (const T*)p->dz;
    a.j0z = p->j0z;
    a.wz = (const T*)p->wz;
    a.kvlo = p->kvlo;
    a.kvhi = p->kvhi;
    a.wzc = (const T*)p->wzc;
    a.cw = p->zcw;
    a.kvslo = paired ? p->kvplo : p->kvlo;
    a.kvshi = paired ? p->kvphi : p->kvhi;
    a.jmin = p->jmin;
    a.jmax = p->jmax;
    a.tw = (const C<T>*)p->tw;
    a.twstride = p->Nmax / p->M0;
    a.skip = paired ? p->skip : nullptr;
    a.err = p->err;
    return a;
}

template <typename T> Usfft2dArgs<T> args2d(const lam_plan* p, bool paired) {
    Usfft2dArgs<T> a;
    a.n1 = p->n1;
    a.n2 = p->n2;
    a.h = p->h;
    a.w = p->w;
    a.T_ = p->T;
    a.M1 = p->M1;
    a.M2 = p->M2;
    a.fcM1 = fft_code(p->M1, fft_max_radix<T>());
    a.fcM2 = fft_code(p->M2, fft_max_radix<T>());
    a.m = p->m;
    a.inv4beta = (T)(1.0 / (4.0 * p->beta));
    a.d1 = (const T*)p->d1;
    a.d2 = (const T*)p->d2;
    a.ang = (const typename AngleT<T>::type*)p->ang;
    a.tw = (const C<T>*)p->tw;
    a.tw1 = p->Nmax / p->M1;
    a.tw2 = p->Nmax / p->M2;
    a.RB = p->RB;
    a.CB = p->CB;
    a.fthr = p->pthr;
    a.TS = p->TS;
    a.TG = p->TG;
    a.nimg = p->nimg;
    a.rmax = (T)p->rmax;
    a.pstride = p->pstride;
    a.spread = p->spread;
    a.jobs = paired ? p->jobs_pair : p->jobs_all;
    a.maxabs = nullptr;
    a.halo = nullptr;
    a.err = p->err;
    a.nacc = paired ? p->nacc : 0;
    a.memo_hit = nullptr;
    // points whose 2m x 2m window covers one cell: at most (2m / spacing + 2)^2 per
    // line neighbourhood, over all T lines and all periodic images; doubled for safety
    {
        const double sp = std::max(1.0, (double)p->M1 / p->w);
        const double per_line = std::ceil(2.0 * p->m * std::sqrt(2.0) / sp) + 2.0;
        const double imgs = (2.0 * p->nimg + 1) * (2.0 * p->nimg + 1);
        a.bound_count = (float)(2.0 * per_line * p->T * imgs);
    }
    return a;
}

template <typename T> Fft2dArgs<T> argsfft(const lam_plan* p) {
    Fft2dArgs<T> a;
    a.T_ = p->T;
    a.h = p->h;
    a.w = p->w;
    a.fch = fft_code(p->h, fft_max_radix<T>());
    a.fcw = fft_code(p->w, fft_max_radix<T>());
    a.tw = (const C<T>*)p->tw;
    a.twh = p->Nmax / p->h;
    a.tww = p->Nmax / p->w;
    return a;
}

// ---- operator sequences ----------------------------------------------------

// planes per launch: the workspace holds p->nbatch planes; split njobs into
// equal launches (no small last batch)
int even_batch(const lam_plan* p, int njobs) {
    const int nlaunch = (njobs + p->nbatch - 1) / p->nbatch;
    return (njobs + nlaunch - 1) / nlaunch;
}

template <typename T>
lam_status fwd_hat(const lam_plan* p, const T* u, C<T>* out, const C<T>* sub, void* ws, cudaStream_t s) {
    NvtxRange range("lam: L_hat (F_u1D, F_u2D)");
    char* w = (char*)ws;
    C<T>* u1 = (C<T>*)(w + p->ws_u1);
    C<T>* P = (C<T>*)(w + p->ws_planes);
    CK(launch_usfft1d_fwd<T>(u, u1, args1d<T>(p, p->TYf, true), s));
    const Usfft2dArgs<T> a = args2d<T>(p, true);
    const int per = even_batch(p, p->njobs_pair);
    for (int j0 = 0; j0 < p->njobs_pair; j0 += per) {
        const int nb = std::min(per, p->njobs_pair - j0);
        CK(launch_usfft2d_fwd<T>(u1, P, out, sub, j0, nb, a, s));
    }
    return LAM_OK;
}

// the fixed-point scatter needs a bound on its input: max(|re|, |im|) into the
// workspace's scalar slot
// device scalar slot for max(|re|, |im|) of a spread input, in the workspace's
// reduction area
template <typename T> T* maxabs_slot(const lam_plan* p, void* ws) {
    return (T*)((char*)ws + p->ws_red + align256(SC_COUNT * sizeof(double)) +
                align256((size_t)kRedBlocks * 4 * sizeof(double)) + 256);
}

template <typename T> lam_status prep_scatter(const lam_plan* p, const C<T>* in, void* ws, cudaStream_t s,
                                              Usfft2dArgs<T>& a) {
    // the exact spread runs when chosen, and for the tile spread's small-plane
    // fallback (tiles narrower than 32)
    const bool exact = p->spread == kSpreadExact || p->spread == kSpreadTilesExact ||
                       ((p->spread == kSpreadTiles || p->spread == kSpreadTiles2 || p->spread == kSpreadHalo ||
                         p->spread == kSpreadSweep) &&
                        p->TS != 32) ||
                       ((p->spread == kSpreadTiles || p->spread == kSpreadTiles2 || p->spread == kSpreadSweep) &&
                        a.nacc > 0);
    if (!exact) return LAM_OK;
    T* mx = maxabs_slot<T>(p, ws);
    CK(launch_absmax<T>(in, p->ndata(), mx, s));
    a.maxabs = mx;
    return LAM_OK;
}

// memoization of the plane stage inside ADMM (memo.cu): the state's slots and
// the threshold
template <typename T> struct MemoState {
    T *key, *now;
    C<T>* val;
    MemoArgs m;
};

template <typename T>
lam_status adj_hat(const lam_plan* p, const C<T>* in, T* u, void* ws, cudaStream_t s, const MemoState<T>* memo = nullptr) {
    NvtxRange range("lam: L_hat^H (F*_u2D, F*_u1D)");
    char* w = (char*)ws;
    C<T>* u1 = (C<T>*)(w + p->ws_u1);
    C<T>* P = (C<T>*)(w + p->ws_planes);
    Usfft2dArgs<T> a = args2d<T>(p, true);
    a.halo = (C<T>*)(w + p->ws_halo);
    if (lam_status st = prep_scatter<T>(p, in, ws, s, a)) return st;
    if (memo) {
        // keys of this input; jobs whose key is close enough to their slot's are
        // skipped by the spread and the inverse plane FFTs
        CK(launch_memo_lookup<T>(in, memo->key, memo->now, memo->m, s));
        a.memo_hit = memo->m.hit;
    }
    const int per = even_batch(p, p->njobs_pair);
    for (int j0 = 0; j0 < p->njobs_pair; j0 += per) {
        const int nb = std::min(per, p->njobs_pair - j0);
        CK(launch_usfft2d_adj<T>(in, P, u1, j0, nb, a, s));
    }
    if (memo) CK(launch_memo_update<T>(u1, memo->val, memo->key, memo->now, memo->m, s));
    CK(launch_usfft1d_adj<T>(u1, u, args1d<T>(p, p->TYa, true), s));
    return LAM_OK;
}

// FBP-style single pass: u = Re L_hat^H (W . F_2D d), W(ku) = pi cos(phi) |ku| / (T w^2 h)
// (|ku| read as 1/4 at ku = 0): the density compensation of the slice points
template <typename T> lam_status fbp_t(const lam_plan* p, const C<T>* d, T* u, void* ws, cudaStream_t s);

template <typename T> lam_status fft2d(const lam_plan* p, const C<T>* in, C<T>* out, int dir, T scale, cudaStream_t s) {
    CK(launch_fft2d_angles<T>(in, out, dir, scale, argsfft<T>(p), s));
    return LAM_OK;
}

template <typename T> lam_status fbp_t(const lam_plan* p, const C<T>* d, T* u, void* ws, cudaStream_t s) {
    NvtxRange range("lam: FBP single pass");
    C<T>* tmp = (C<T>*)((char*)ws + p->ws_tmp);
    if (lam_status st = fft2d<T>(p, d, tmp, -1, (T)1, s)) return st;
    const double c0 = M_PI * std::cos(p->phi) / ((double)p->T * p->w * p->w * p->h);
    CK(launch_ramp<T>(tmp, (long long)p->T * p->h, p->w, (T)c0, s));
    return adj_hat<T>(p, tmp, u, ws, s);
}

// ---- ADMM state layout -------------------------------------------------------

struct StateLayout {
    size_t sc, hist, partials, counter, u, du, Gd, G0, G1, p, e, lam, dpsi, dhat, r, Lp, rlo;
    // memoization pieces (at the end; empty when the state has no memoization)
    size_t mkey, mnow, mval, mhit, mvalid, mscale, total;
};

// memo: the state memoizes F*_u2D (the pieces after rlo; nothing before them
// depends on it)
StateLayout layout(const lam_plan* p, bool memo = false) {
    StateLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    const size_t vb = (size_t)p->nvox() * p->elem();
    const size_t db = (size_t)p->ndata() * p->celem();
    L.sc = take(SC_COUNT * sizeof(double));
    L.hist = take((size_t)kHistCap * 4 * sizeof(double));
    L.partials = take((size_t)kRedBlocks * 4 * sizeof(double));
    L.counter = take(sizeof(unsigned int));
    L.u = take(vb);
    L.du = take(vb);
    L.Gd = take(vb);
    L.G0 = take(vb);
    L.G1 = take(vb);
    L.p = take(vb);
    L.e = take(3 * vb);
    L.lam = take(3 * vb);
    L.dpsi = take(3 * vb);
    L.dhat = take(db);
    L.r = take(db);
    L.Lp = take(db);
    L.rlo = take(p->prec == LAM_F32 ? db : 0);  // low part of the compensated residual (FP32 only)
    const size_t nj = memo ? (size_t)p->njobs_pair : 0;
    const size_t nk = (size_t)4 * p->memo_K;
    L.mkey = take(nj * nk * p->elem());
    L.mnow = take(nj * nk * p->elem());
    L.mval = take(nj * p->n1 * p->n2 * p->celem());
    L.mhit = take(nj * sizeof(int));
    L.mvalid = take(nj * sizeof(int));
    L.mscale = take(nj * sizeof(double));
    L.total = o;
    return L;
}

__global__ void k_init_scalars(double* sc, double rho, double alpha, double invhw, double adapt,
                               unsigned int* counter) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = 0; i < SC_COUNT; ++i) sc[i] = 0.0;
    sc[SC_RHO] = rho;
    sc[SC_ALPHA] = alpha;
    sc[SC_INVHW] = invhw;
    sc[SC_ADAPT] = adapt;
    *counter = 0;
}

template <typename T> struct StatePtrs {
    T *u, *du, *Gd, *G0, *G1, *p, *e, *lam, *dpsi;
    C<T>*dhat, *r, *Lp, *rlo;
    AdmmRed red;
    double* hist;
    // memoization (null without it)
    T *mkey, *mnow;
    C<T>* mval;
    int *mhit, *mvalid;
    double* mscale;
};

template <typename T> StatePtrs<T> ptrs(const lam_plan* p, void* state, bool memo = false) {
    const StateLayout L = layout(p, memo);
    char* b = (char*)state;
    StatePtrs<T> s;
    s.u = (T*)(b + L.u);
    s.du = (T*)(b + L.du);
    s.Gd = (T*)(b + L.Gd);
    s.G0 = (T*)(b + L.G0);
    s.G1 = (T*)(b + L.G1);
    s.p = (T*)(b + L.p);
    s.e = (T*)(b + L.e);
    s.lam = (T*)(b + L.lam);
    s.dpsi = (T*)(b + L.dpsi);
    s.dhat = (C<T>*)(b + L.dhat);
    s.r = (C<T>*)(b + L.r);
    s.Lp = (C<T>*)(b + L.Lp);
    s.rlo = (C<T>*)(b + L.rlo);
    s.red.sc = (double*)(b + L.sc);
    s.red.partials = (double*)(b + L.partials);
    s.red.counter = (unsigned int*)(b + L.counter);
    s.hist = (double*)(b + L.hist);
    s.mkey = memo ? (T*)(b + L.mkey) : nullptr;
    s.mnow = memo ? (T*)(b + L.mnow) : nullptr;
    s.mval = memo ? (C<T>*)(b + L.mval) : nullptr;
    s.mhit = memo ? (int*)(b + L.mhit) : nullptr;
    s.mvalid = memo ? (int*)(b + L.mvalid) : nullptr;
    s.mscale = memo ? (double*)(b + L.mscale) : nullptr;
    return s;
}

template <typename T> Admm<T> admm_ops(const lam_plan* p) {
    Admm<T> a;
    a.v.n1 = p->n1;
    a.v.nz = p->nz;
    a.v.n2 = p->n2;
    const bool shifts = pow2(p->n2) && pow2(p->nz);
    a.v.ln2 = shifts ? ilog2(p->n2) : -1;
    a.v.lnz = shifts ? ilog2(p->nz) : -1;
    a.v.N = p->nvox();
    return a;
}

template <typename T>
lam_status admm_init_t(const lam_plan* p, void* state, const void* d, double alpha, double rho, int adapt,
                       int form, bool memo, cudaStream_t s) {
    const StateLayout L = layout(p, memo);
    StatePtrs<T> S = ptrs<T>(p, state, memo);
    if (memo) {
        CK(cudaMemsetAsync(S.mkey, 0, (size_t)p->njobs_pair * 4 * p->memo_K * sizeof(T), s));
        CK(cudaMemsetAsync(S.mvalid, 0, (size_t)p->njobs_pair * sizeof(int), s));
    }
    const size_t vb = (size_t)p->nvox() * p->elem();
    CK(cudaMemsetAsync(S.u, 0, vb, s));
    CK(cudaMemsetAsync(S.p, 0, vb, s));
    CK(cudaMemsetAsync(S.e, 0, 3 * vb, s));
    CK(cudaMemsetAsync(S.lam, 0, 3 * vb, s));
    if (p->prec == LAM_F32) CK(cudaMemsetAsync(S.rlo, 0, (size_t)p->ndata() * p->celem(), s));
    (void)L;
    // Algorithm 2 works on d_hat = F_2D d with the Parseval weight 1/(hw);
    // Algorithm 1 keeps d in the data space (the slot holds d) with weight 1
    k_init_scalars<<<1, 32, 0, s>>>(S.red.sc, rho, alpha, form == 1 ? 1.0 : 1.0 / ((double)p->h * p->w),
                                    adapt ? 1.0 : 0.0, S.red.counter);
    CK(cudaGetLastError());
    if (form == 1) {
        CK(cudaMemcpyAsync(S.dhat, d, (size_t)p->ndata() * p->celem(), cudaMemcpyDeviceToDevice, s));
    } else {
        lam_status st = fft2d<T>(p, (const C<T>*)d, S.dhat, -1, (T)1, s);
        if (st) return st;
    }
    const Admm<T> ops = admm_ops<T>(p);
    CK(ops.neg_copy(S.dhat, S.r, p->ndata(), s));
    CK(ops.residual_norm(S.r, p->ndata(), S.red, s));
    return LAM_OK;
}

template <typename T>
lam_status admm_step_t(const lam_plan* p, void* state, void* ws, int n_inner, int form, int resid, double memo_tau,
                       cudaStream_t s) {
    NvtxRange range("lam: ADMM outer iteration");
    const bool memo = memo_tau > 0 && form == 2;
    StatePtrs<T> S = ptrs<T>(p, state, memo);
    MemoState<T> M{};
    if (memo) {
        M.key = S.mkey;
        M.now = S.mnow;
        M.val = S.mval;
        M.m.njobs = p->njobs_pair;
        M.m.K = p->memo_K;
        M.m.jobs = p->jobs_pair;
        M.m.samples = p->memo_samples;
        M.m.h = p->h;
        M.m.w = p->w;
        M.m.plane = (long long)p->n1 * p->n2;
        M.m.tau = memo_tau;
        M.m.hit = S.mhit;
        M.m.valid = S.mvalid;
        M.m.scale = S.mscale;
        M.m.stats = S.red.sc + SC_MEMO_HITS;
    }
    const Admm<T> ops = admm_ops<T>(p);
    const long long nd = p->ndata();
    const T sc = (T)(1.0 / ((double)p->h * p->w));
    C<T>* tmp = (C<T>*)((char*)ws + p->ws_tmp);
    lam_status st;
    for (int i = 0; i < n_inner; ++i) {
        T* Gc = (i & 1) ? S.G1 : S.G0;
        T* Gp = (i & 1) ? S.G0 : S.G1;
        if (form == 1) {
            // Algorithm 1: r = L u_k - d in the data space (F*_2D after L_hat) for
            // the current iterate u_k (u + du after the first step: u takes the
            // LSP increment du only at its end), then G = Re L^H r - rho div(...)
            // with L^H = L_hat^H F_2D / (hw).  Gd holds u + du until the adjoint
            // pass overwrites it.
            const T* uk = S.u;
            if (i > 0) {
                CK(ops.vadd(S.u, S.du, S.Gd, s));
                uk = S.Gd;
            }
            if ((st = fwd_hat<T>(p, uk, S.r, nullptr, ws, s))) return st;
            if ((st = fft2d<T>(p, S.r, S.r, +1, sc, s))) return st;
            CK(ops.csub(S.dhat, S.r, nd, s));
            if ((st = fft2d<T>(p, S.r, tmp, -1, sc, s))) return st;
            if ((st = adj_hat<T>(p, tmp, S.Gd, ws, s))) return st;
        } else {
            // residual refresh: r = L_hat u - d_hat evaluated afresh (the
            // subtraction fused into the gather) at the start of each LSP, so
            // the rounding of the carried updates r += gamma L_hat p does not
            // accumulate from one LSP to the next
            if (i == 0 && (resid & LAM_RESID_REFRESH)) {
                if ((st = fwd_hat<T>(p, S.u, S.r, S.dhat, ws, s))) return st;
                if (resid & LAM_RESID_COMPENSATED)
                    CK(cudaMemsetAsync(S.rlo, 0, (size_t)nd * sizeof(C<T>), s));
            }
            // adjoint pass: G = Re L_hat^H r / (hw) - rho div(grad u - g)
            if ((st = adj_hat<T>(p, S.r, S.Gd, ws, s, memo ? &M : nullptr))) return st;
        }
        CK(ops.lsp_G(S.Gd, S.du, S.e, S.lam, S.p, Gp, Gc, i == 0, S.red, s));
        // CG direction and its forward pass
        CK(ops.lsp_p(Gc, S.p, S.red, s));
        if ((st = fwd_hat<T>(p, S.p, S.Lp, nullptr, ws, s))) return st;
        if (form == 1 && (st = fft2d<T>(p, S.Lp, S.Lp, +1, sc, s))) return st;
        // exact line search, increment and residual update (u += du on the last step)
        CK(ops.lsp_update(S.du, S.u, S.p, i == 0, i == n_inner - 1, S.r,
                          form == 2 && (resid & LAM_RESID_COMPENSATED) ? S.rlo : nullptr, S.Lp, nd, S.red, s));
    }
    NvtxRange rsp("lam: RSP, multiplier, penalty");
    CK(ops.rsp(S.u, S.du, S.e, S.lam, S.dpsi, S.red, S.hist, kHistCap, s));
    return LAM_OK;
}

__global__ void k_real_to_complex(const float* __restrict__ src, C<float>* __restrict__ dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = cmake<float>(src[i], 0.f);
}

template <typename T> lam_status u2d_fwd_t(const lam_plan* p, const void* u1, void* out, const void* sub,
                                                  void* ws, cudaStream_t s) {
    C<T>* P = (C<T>*)((char*)ws + p->ws_planes);
    const Usfft2dArgs<T> a = args2d<T>(p, false);
    for (int j0 = 0; j0 < p->h; j0 += p->nbatch)
        CK(launch_usfft2d_fwd<T>((const C<T>*)u1, P, (C<T>*)out, (const C<T>*)sub, j0,
                                 std::min(p->nbatch, p->h - j0), a, s));
    return LAM_OK;
}
template <typename T>
lam_status spread_t(const lam_plan* p, const void* d_hat, void* ws, int j0, int nb, cudaStream_t s) {
    char* w = (char*)ws;
    Usfft2dArgs<T> a = args2d<T>(p, true);
    a.halo = (C<T>*)(w + p->ws_halo);
    if (lam_status st = prep_scatter<T>(p, (const C<T>*)d_hat, ws, s, a)) return st;
    CK(launch_spread2d<T>((const C<T>*)d_hat, (C<T>*)(w + p->ws_planes), j0, nb, a, s));
    return LAM_OK;
}

template <typename T> lam_status u2d_adj_t(const lam_plan* p, const void* in, void* u1, void* ws,
                                                  cudaStream_t s) {
    C<T>* P = (C<T>*)((char*)ws + p->ws_planes);
    Usfft2dArgs<T> a = args2d<T>(p, false);
    a.halo = (C<T>*)((char*)ws + p->ws_halo);
    if (lam_status st = prep_scatter<T>(p, (const C<T>*)in, ws, s, a)) return st;
    for (int j0 = 0; j0 < p->h; j0 += p->nbatch)
        CK(launch_usfft2d_adj<T>((const C<T>*)in, P, (C<T>*)u1, j0, std::min(p->nbatch, p->h - j0), a, s));
    return LAM_OK;
}

lam_status check_plan(const lam_plan* p) {
    if (!p) return fail(LAM_EINVAL, "plan is NULL");
    return LAM_OK;
}


// ---- batches -------------------------------------------------------------------

template <typename T> lam_status batch_build(lam_batch* b) {
    std::unique_ptr<BatchTable<T>> H(new BatchTable<T>());
    std::memset(H.get(), 0, sizeof(BatchTable<T>));
    H->count = b->count;
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device));
    size_t smem[kBStages] = {};
    const size_t ce = sizeof(C<T>);
    for (int i = 0; i < b->count; ++i) {
        const lam_plan* q = b->plans[i];
        char* w = (char*)b->ws[i];
        H->zf[i] = args1d<T>(q, q->TYf, true);
        H->za[i] = args1d<T>(q, q->TYa, true);
        H->a2[i] = args2d<T>(q, true);
        H->u1[i] = (C<T>*)(w + q->ws_u1);
        H->P[i] = (C<T>*)(w + q->ws_planes);
        const int nj = q->njobs_pair;
        const int gx[kBStages] = {q->n1 * (q->n2 / q->TYf),          q->n1 / q->RB, q->M2 / q->CB,
                                  (q->M1 / q->TG) * (q->M2 / q->TG), (q->M1 / q->TS) * (q->M2 / q->TS),
                                  q->M2 / q->CB,                     q->n1 / q->RB, q->n1 * (q->n2 / q->TYa)};
        const int nacc = std::min(q->nacc, nj);  // centre jobs the exact spread takes (own launches)
        H->a2[i].nacc = nacc;
        const int gy[kBStages] = {1, nj, nj, nj, nj - nacc, nj, nj, 1};
        const int gz[kBStages] = {1, 1, 1, 1, 1, 1, 1, 1};
        const size_t sm[kBStages] = {(size_t)q->TYf * fpad_len(q->nz) * ce,
                                     (size_t)q->RB * fpad_len(q->M2) * ce,
                                     (size_t)q->CB * fpad_len(q->M1) * ce,
                                     gather_smem_bytes<T>(q->TG, q->m),
                                     spread_tiles_bytes<T>(q->m),
                                     (size_t)q->CB * fpad_len(q->M1) * ce,
                                     (size_t)q->RB * fpad_len(q->M2) * ce,
                                     (size_t)(fpad_len(q->nz) + q->h) * q->TYa * ce};
        for (int st = 0; st < kBStages; ++st) {
            H->start[st][i] = b->total[st];
            H->gx[st][i] = gx[st];
            H->gy[st][i] = gy[st];
            const long long add = (long long)gx[st] * gy[st] * gz[st];
            if ((long long)b->total[st] + add > (1LL << 30)) return fail(LAM_EUNSUPPORTED, "batch too large");
            b->total[st] += (int)add;
            smem[st] = std::max(smem[st], sm[st]);
        }
    }
    for (int st = 0; st < kBStages; ++st) {
        H->start[st][b->count] = b->total[st];
        const int occ = st == kBZFwd   ? batch_occupancy_z<T>(true, b->mixed, smem[st])
                        : st == kBZAdj ? batch_occupancy_z<T>(false, b->mixed, smem[st])
                                       : batch_occupancy<T>(st, b->mixed, b->m, smem[st]);
        if (occ < 1) return fail(LAM_EUNSUPPORTED, "batched stage %d does not fit on an SM (%zu bytes)", st, smem[st]);
        b->L[st].grid = std::max(1, std::min(b->total[st], occ * nsm));
        b->L[st].smem = smem[st];
    }
    if (cudaMalloc(&b->dev, sizeof(BatchTable<T>)) != cudaSuccess)
        return fail(LAM_ENOMEM, "cudaMalloc of the batch table failed");
    CK(cudaMemcpy(b->dev, H.get(), sizeof(BatchTable<T>), cudaMemcpyHostToDevice));
    return LAM_OK;
}

template <typename T>
lam_status batch_fwd_hat(const lam_batch* b, const void* const* in, void* const* out, cudaStream_t s) {
    BatchPtrs ptrs{};
    for (int i = 0; i < b->count; ++i) {
        ptrs.in[i] = in[i];
        ptrs.out[i] = out[i];
    }
    BatchTable<T>* dev = (BatchTable<T>*)b->dev;
    CK(launch_batch_ptrs<T>(dev, ptrs, b->count, s));
    CK(launch_batch_z<T>(dev, true, b->mixed, b->L[kBZFwd], s));
    for (int st : {(int)kBRowFwd, (int)kBColFwd, (int)kBGather})
        CK(launch_batch_plane<T>(dev, st, b->mixed, b->m, b->L[st], s));
    return LAM_OK;
}

template <typename T>
lam_status batch_adj_hat(const lam_batch* b, const void* const* in, void* const* out, cudaStream_t s) {
    BatchPtrs ptrs{};
    for (int i = 0; i < b->count; ++i) {
        ptrs.in[i] = in[i];
        ptrs.out[i] = out[i];
    }
    BatchTable<T>* dev = (BatchTable<T>*)b->dev;
    CK(launch_batch_ptrs<T>(dev, ptrs, b->count, s));
    // centre plane jobs with exact accumulation (LAM_OPT_EXACT_CENTRE_JOBS), per
    // problem, as the single-plan adjoint does; the batched tile spread skips them
    for (int i = 0; i < b->count; ++i) {
        const lam_plan* q = b->plans[i];
        const int nacc = std::min(q->nacc, q->njobs_pair);
        if (nacc <= 0) continue;
        Usfft2dArgs<T> a = args2d<T>(q, true);
        a.spread = kSpreadTiles;  // the batch spreads with tiles whatever the plan's choice
        a.maxabs = maxabs_slot<T>(q, b->ws[i]);
        CK(launch_absmax<T>((const C<T>*)in[i], q->ndata(), (T*)a.maxabs, s));
        CK(launch_spread2d<T>((const C<T>*)in[i], (C<T>*)((char*)b->ws[i] + q->ws_planes), 0, nacc, a, s));
    }
    for (int st : {(int)kBSpread, (int)kBColAdj, (int)kBRowAdj})
        CK(launch_batch_plane<T>(dev, st, b->mixed, b->m, b->L[st], s));
    CK(launch_batch_z<T>(dev, false, b->mixed, b->L[kBZAdj], s));
    return LAM_OK;
}

// one ADMM outer iteration of every problem: the operators run batched, the
// elementwise steps per problem (Section 2: LSP in the Algorithm 2 form, RSP,
// multiplier and penalty updates), in the order admm_step uses
template <typename T>
lam_status batch_admm_step(const lam_batch* b, void* const* states, const int* resid, int n_inner, cudaStream_t s) {
    std::vector<StatePtrs<T>> S;
    std::vector<Admm<T>> ops;
    for (int i = 0; i < b->count; ++i) {
        S.push_back(ptrs<T>(b->plans[i], states[i]));
        ops.push_back(admm_ops<T>(b->plans[i]));
    }
    const void* in[kMaxBatch];
    void* out[kMaxBatch];
    for (int k = 0; k < n_inner; ++k) {
        for (int i = 0; i < b->count; ++i) {
            in[i] = S[i].r;
            out[i] = S[i].Gd;
        }
        if (lam_status st = batch_adj_hat<T>(b, in, out, s)) return st;
        for (int i = 0; i < b->count; ++i) {
            T* Gc = (k & 1) ? S[i].G1 : S[i].G0;
            T* Gp = (k & 1) ? S[i].G0 : S[i].G1;
            CK(ops[i].lsp_G(S[i].Gd, S[i].du, S[i].e, S[i].lam, S[i].p, Gp, Gc, k == 0, S[i].red, s));
            CK(ops[i].lsp_p(Gc, S[i].p, S[i].red, s));
            in[i] = S[i].p;
            out[i] = S[i].Lp;
        }
        if (lam_status st = batch_fwd_hat<T>(b, in, out, s)) return st;
        for (int i = 0; i < b->count; ++i)
            CK(ops[i].lsp_update(S[i].du, S[i].u, S[i].p, k == 0, k == n_inner - 1, S[i].r,
                                 (resid[i] & LAM_RESID_COMPENSATED) ? S[i].rlo : nullptr, S[i].Lp,
                                 b->plans[i]->ndata(), S[i].red, s));
    }
    for (int i = 0; i < b->count; ++i)
        CK(ops[i].rsp(S[i].u, S[i].du, S[i].e, S[i].lam, S[i].dpsi, S[i].red, S[i].hist, kHistCap, s));
    return LAM_OK;
}

// ---- allocation-free F_u2D (no counterpart in the paper) ----------------------
// Some callers cannot give the library a workspace: code that runs inside a
// device allocator's own hooks (it must not call back into the allocator), or
// a process whose device memory is owned by another pool once it has started.
// For them lamx_u2d_fwd_static takes its batch of padded planes from the
// fixed array below instead of ws, and allocates nothing.  The array holds
// kStaticPlaneBytes: one padded plane (2n)^2 of complex values fits up to
// n = 512 in FP32 and n = 256 in FP64; larger planes are rejected.  Every
// byte the kernels read from it is written earlier in the same call, so
// nothing needs to start at zero.  There is one array per device: calls that
// overlap in time (other streams, other threads, other plans) race on it.
}  // namespace

constexpr size_t kStaticPlaneBytes = (size_t)8 << 20;
static __device__ __align__(256) unsigned char g_static_planes[kStaticPlaneBytes];

namespace {

// device address of g_static_planes, looked up once per device (the first
// call on a device does the lookup)
constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kStaticMaxDevices] = {};

lam_status static_planes(int dev, void** out) {
    if (dev < 0 || dev >= kStaticMaxDevices) return fail(LAM_EUNSUPPORTED, "device %d: at most %d devices", dev,
                                                         kStaticMaxDevices);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_planes);
        if (e != cudaSuccess || !ptr)
            return fail(LAM_ECUDA, "cudaGetSymbolAddress of the static plane scratch failed: %s",
                        cudaGetErrorString(e));
        g_static_ptr[dev] = ptr;
    }
    *out = g_static_ptr[dev];
    return LAM_OK;
}

// an array argument must be device (or managed) memory of the plan's device:
// a pointer into another GPU's memory or into pageable host memory would
// otherwise reach the kernels
lam_status check_device_ptr(const void* ptr, int dev, const char* name) {
    if (!ptr) return LAM_OK;
    cudaPointerAttributes at;
    const cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();  // the failed query leaves a (non-sticky) error behind: clear it
        return fail(LAM_EINVAL, "%s: not a CUDA pointer (%s)", name, cudaGetErrorString(e));
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(LAM_EINVAL, "%s: not device memory", name);
    if (at.device != dev) return fail(LAM_EINVAL, "%s lives on device %d, the plan on device %d", name, at.device, dev);
    return LAM_OK;
}

template <typename T> lam_status u2d_fwd_static_t(const lam_plan* p, const void* u1, void* out, const void* sub,
                                                  cudaStream_t s) {
    const size_t plane = (size_t)p->M1 * p->M2 * sizeof(C<T>);
    if (plane > kStaticPlaneBytes)
        return fail(LAM_EUNSUPPORTED, "one padded %dx%d plane needs %zu bytes; the static scratch holds %zu", p->M1,
                    p->M2, plane, kStaticPlaneBytes);
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != p->device) return fail(LAM_EINVAL, "current device %d is not the plan's device %d", dev, p->device);
    if (lam_status st = check_device_ptr(u1, dev, "u1")) return st;
    if (lam_status st = check_device_ptr(out, dev, "d_hat")) return st;
    if (lam_status st = check_device_ptr(sub, dev, "sub")) return st;
    void* scratch = nullptr;
    if (lam_status st = static_planes(dev, &scratch)) return st;
    C<T>* P = (C<T>*)scratch;
    const int nb = (int)std::min<size_t>((size_t)p->h, kStaticPlaneBytes / plane);
    const Usfft2dArgs<T> a = args2d<T>(p, false);
    for (int j0 = 0; j0 < p->h; j0 += nb)
        CK(launch_usfft2d_fwd<T>((const C<T>*)u1, P, (C<T>*)out, (const C<T>*)sub, j0, std::min(nb, p->h - j0), a,
                                 s));
    return LAM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

const char* lam_last_error(void) { return g_err.c_str(); }

lam_status lam_plan_create(lam_plan** out, int n, int nz, int det_h, int det_w, int n_theta, const double* theta,
                           double phi, int oversample, int half_width, int prec) {
    if (!out) return fail(LAM_EINVAL, "out is NULL");
    *out = nullptr;
    const int dims[4] = {n, nz, det_h, det_w};
    const char* names[4] = {"n", "nz", "det_h", "det_w"};
    for (int i = 0; i < 4; ++i)
        if (dims[i] < 8 || dims[i] > 2048 || dims[i] % 2 != 0 || fft_code(dims[i]) < 0)
            return fail(LAM_EUNSUPPORTED, "%s = %d: must be even, 2^a 3^b 5^c, in [8, 2048]", names[i], dims[i]);
    if (n % 8 != 0) return fail(LAM_EUNSUPPORTED, "n = %d: must be a multiple of 8 (plane tiles)", n);
    if (n_theta < 1 || n_theta > 65536) return fail(LAM_EINVAL, "n_theta = %d out of range", n_theta);
    if (!theta) return fail(LAM_EINVAL, "theta is NULL");
    for (int k = 0; k < n_theta; ++k)
        if (!std::isfinite(theta[k])) return fail(LAM_EINVAL, "theta[%d] is not finite", k);
    if (!(phi >= 0.0 && phi < M_PI / 2)) return fail(LAM_EINVAL, "phi = %g must be in [0, pi/2)", phi);
    if (oversample != 2) return fail(LAM_EUNSUPPORTED, "oversample = %d: only 2 is supported", oversample);
    if (half_width < 2 || half_width > 8) return fail(LAM_EUNSUPPORTED, "half_width = %d not in [2, 8]", half_width);
    if (prec != LAM_F32 && prec != LAM_F64) return fail(LAM_EINVAL, "prec = %d", prec);

    lam_plan* p = new lam_plan();
    p->n1 = p->n2 = n;
    p->nz = nz;
    p->h = det_h;
    p->w = det_w;
    p->T = n_theta;
    p->m = half_width;
    p->R = oversample;
    p->prec = prec;
    // FP32 defaults (measured on the 512^3 workload, FP32 vs FP64 ADMM-TV):
    // the centre plane jobs spread exactly and the LSP residual carried in a
    // compensated pair.  FP64 sums need neither.
    p->nacc = prec == LAM_F32 ? kDefaultExactCentreJobs : 0;
    p->resid = prec == LAM_F32 ? LAM_RESID_COMPENSATED : 0;
    p->phi = phi;
    p->M0 = 2 * nz;
    p->M1 = 2 * n;
    p->M2 = 2 * n;
    // twiddle table length: a common multiple of every FFT length the plan runs
    {
        long long L = 1;
        for (int v : {p->nz, p->M0, p->M1, p->M2, p->h, p->w}) {
            long long a = L, b = v;
            while (b) { const long long t = a % b; a = b; b = t; }
            L = L / a * v;
        }
        if (L > (1LL << 22)) {
            delete p;
            return fail(LAM_EUNSUPPORTED, "sizes n = %d, nz = %d, det %d x %d need a twiddle table of %lld entries",
                        n, nz, det_h, det_w, L);
        }
        p->Nmax = (int)L;
    }
    p->beta = half_width * 2.0 / (4.0 * M_PI * 1.5);
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return fail(LAM_ECUDA, "no CUDA device");
    }
    lam_status st = prec == LAM_F32 ? build_tables<float>(p, theta) : build_tables<double>(p, theta);
    cudaError_t ce = prec == LAM_F32 ? configure_usfft1d<float>() : configure_usfft1d<double>();
    if (!ce) ce = prec == LAM_F32 ? configure_usfft2d<float>() : configure_usfft2d<double>();
    if (!ce) ce = prec == LAM_F32 ? configure_fft2d<float>() : configure_fft2d<double>();
    if (!st && ce) st = fail(LAM_ECUDA, "kernel configuration failed: %s", cudaGetErrorString(ce));
    if (st) {
        lam_plan_destroy(p);
        return st;
    }
    pick_fft_shapes(p);
    const size_t ce_ = p->celem();
    // plane tiles divide M1 = M2 = 2n (a multiple of 16): spread tiles 32 (the
    // tile spread's size) when possible; gather tiles up to 64, since larger
    // tiles amortise the per-block line tests over more points
    p->TS = p->M1 % 32 == 0 ? 32 : 16;
    p->TG = p->M1 % 64 == 0 ? 64 : p->TS;
    if (const char* env = std::getenv("LAMINO_GATHER_TILE")) {
        const int v = std::atoi(env);
        if (v >= 16 && v <= std::min(p->M1, p->M2) && (v & (v - 1)) == 0) p->TG = v;
    }
    // unwrapped slice positions reach |p| <= M (1 + sin phi) / 2 + m + 2
    const double reach = std::max(p->M1, p->M2) * (1.0 + std::sin(phi)) / 2.0 + p->m + 2;
    p->nimg = (int)std::ceil(reach / std::min(p->M1, p->M2));
    // |position| <= (w/2) M / w + (h/2) M sin(phi) / h (+ 1 for the grid offset)
    p->rmax = std::hypot(p->M1 * 0.5, p->M1 * 0.5 * std::sin(phi)) + 1.0;
    // consecutive slice points are M1 / w cells apart; points at least sqrt 2
    // cells apart have distinct tap-window origins
    p->pstride = (int)std::ceil(std::sqrt(2.0) * p->w / (double)p->M1 - 1e-9);
    if (p->pstride < 1) p->pstride = 1;
    const size_t plane = (size_t)p->M1 * p->M2 * ce_;
    // padded planes per batch: up to 8 GiB in FP32 (fewer, larger launches: at
    // 1024^3 three batches of <= 171 plane jobs ran the L-hat / L-hat^H pair
    // 2.4 % faster than 17 batches of <= 31 under 1 GiB); 1 GiB in FP64, whose
    // ADMM state at 1024^3 (~180 GB) leaves no room for more
    const size_t plane_budget = (size_t)(prec == LAM_F32 ? 8 : 1) << 30;
    p->nbatch = (int)std::max<size_t>(1, std::min<size_t>((size_t)p->h, plane_budget / plane));
    // LAMINO_PLANES_PER_BATCH overrides the number of padded planes processed per
    // batch (workspace size follows); for tuning
    if (const char* env = std::getenv("LAMINO_PLANES_PER_BATCH")) {
        const int v = std::atoi(env);
        if (v >= 1 && v <= p->h) p->nbatch = v;
    }
    p->ws_u1 = 0;
    p->ws_planes = align256((size_t)p->h * p->n1 * p->n2 * ce_);
    // halo spread: a batch of extended tiles (core + halo) per plane
    p->ws_halo = p->ws_planes + align256((size_t)p->nbatch * plane);
    {
        const size_t ext = 32 + 2 * (size_t)p->m - 1;
        const size_t ntiles = p->TS == 32 ? (size_t)(p->M1 / 32) * (p->M2 / 32) : 0;
        p->ws_red = p->ws_halo + align256((size_t)p->nbatch * ntiles * ext * ext * ce_);
    }
    // reduction scratch: scalars, per-block partials, completion counter
    // + one scalar slot for the scatter's input bound
    p->ws_tmp = p->ws_red + align256(SC_COUNT * sizeof(double)) + align256((size_t)kRedBlocks * 4 * sizeof(double)) +
                256 + 256;
    // last: the data-space buffer only L^H (lam_adjoint) and the Algorithm 1
    // form use; the L_hat / L_hat^H calls need only the workspace before it
    p->ws_bytes = p->ws_tmp + align256((size_t)p->ndata() * ce_);
    *out = p;
    return LAM_OK;
}

lam_status lam_plan_set_option(lam_plan* p, int option, int value) {
    if (lam_status st = check_plan(p)) return st;
    switch (option) {
        case LAM_OPT_FAST_ADJOINT:
        case LAM_OPT_ADJOINT_SPREAD:
            if (option == LAM_OPT_FAST_ADJOINT) p->spread = value ? kSpreadAtomic : kSpreadTiles;
            else if (value == LAM_SPREAD_TILES) p->spread = kSpreadTiles;
            else if (value == LAM_SPREAD_ATOMIC) p->spread = kSpreadAtomic;
            else if (value == LAM_SPREAD_EXACT) p->spread = kSpreadExact;
            else if (value == LAM_SPREAD_HALO) p->spread = kSpreadHalo;
            else if (value == LAM_SPREAD_TILES_EXACT) p->spread = kSpreadTilesExact;
            else if (value == LAM_SPREAD_TILES2) p->spread = kSpreadTiles2;
            else if (value == LAM_SPREAD_SWEEP) p->spread = kSpreadSweep;
            else return fail(LAM_EINVAL, "unknown adjoint spread %d", value);
            {
                // captured ADMM graphs hold the old kernel choice
                std::lock_guard<std::mutex> lk(p->mu);
                for (auto& kv : p->admm)
                    if (kv.second.graph) {
                        cudaGraphExecDestroy(kv.second.graph);
                        kv.second.graph = nullptr;
                    }
            }
            return LAM_OK;
        case LAM_OPT_LSP_FORM:
            if (value != 1 && value != 2) return fail(LAM_EINVAL, "LSP form %d: 1 or 2", value);
            p->lsp_form = value;
            return LAM_OK;
        case LAM_OPT_MEMO_TAU:
            if (value < 0 || value >= 10000) return fail(LAM_EINVAL, "memo threshold %d: 0 (off) or tau * 10000 in [1, 9999]", value);
            p->memo_tau = value / 10000.0;
            return LAM_OK;
        case LAM_OPT_EXACT_CENTRE_JOBS:
            if (value < 0) return fail(LAM_EINVAL, "exact centre jobs %d < 0", value);
            p->nacc = value;
            {
                // captured ADMM graphs hold the old launch sequence
                std::lock_guard<std::mutex> lk(p->mu);
                for (auto& kv : p->admm)
                    if (kv.second.graph) {
                        cudaGraphExecDestroy(kv.second.graph);
                        kv.second.graph = nullptr;
                    }
            }
            return LAM_OK;
        case LAM_OPT_RESIDUAL:
            if (value & ~(LAM_RESID_REFRESH | LAM_RESID_COMPENSATED))
                return fail(LAM_EINVAL, "residual mode %d: a combination of LAM_RESID_REFRESH and LAM_RESID_COMPENSATED", value);
            p->resid = value;
            return LAM_OK;
        case LAM_OPT_Z_THREADS:
        case LAM_OPT_PLANE_FFT_THREADS: {
            if (value != 256 && value != 512) return fail(LAM_EINVAL, "threads per block %d: 256 or 512", value);
            (option == LAM_OPT_Z_THREADS ? p->zthr : p->pthr) = value;
            pick_fft_shapes(p);  // batches built earlier keep their own shapes
            std::lock_guard<std::mutex> lk(p->mu);
            for (auto& kv : p->admm)
                if (kv.second.graph) {
                    cudaGraphExecDestroy(kv.second.graph);
                    kv.second.graph = nullptr;
                }
            return LAM_OK;
        }
        default:
            return fail(LAM_EINVAL, "unknown option %d", option);
    }
}

lam_status lam_plan_destroy(lam_plan* plan) {
    if (!plan) return LAM_OK;
    for (auto& kv : plan->admm)
        if (kv.second.graph) cudaGraphExecDestroy(kv.second.graph);
    for (void* d : plan->dev_allocs) cudaFree(d);
    delete plan;
    return LAM_OK;
}

size_t lam_workspace_bytes(const lam_plan* plan) { return plan ? plan->ws_bytes : 0; }
size_t lam_workspace_bytes_hat(const lam_plan* plan) { return plan ? plan->ws_tmp : 0; }

#define DISPATCH(p, F32CALL, F64CALL) ((p)->prec == LAM_F32 ? (F32CALL) : (F64CALL))

// the z stage copies volume columns in pairs (one complex element each), so
// a real volume must start on a two-element boundary
static lam_status check_vol_align(int prec, const void* u, int i = -1) {
    const size_t al = prec == LAM_F32 ? 8 : 16;
    if ((uintptr_t)u % al) {
        if (i >= 0) return fail(LAM_EINVAL, "volume %d is not %zu-byte aligned", i, al);
        return fail(LAM_EINVAL, "volume is not %zu-byte aligned", al);
    }
    return LAM_OK;
}

lam_status lam_forward_hat(const lam_plan* p, const void* u, void* d_hat, const void* sub, void* ws, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    if (!u || !d_hat || !ws) return fail(LAM_EINVAL, "NULL array argument");
    if (lam_status st = check_vol_align(p->prec, u)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    return DISPATCH(p, fwd_hat<float>(p, (const float*)u, (C<float>*)d_hat, (const C<float>*)sub, ws, s),
                    fwd_hat<double>(p, (const double*)u, (C<double>*)d_hat, (const C<double>*)sub, ws, s));
}

lam_status lam_adjoint_hat(const lam_plan* p, const void* d_hat, void* u, void* ws, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    if (!u || !d_hat || !ws) return fail(LAM_EINVAL, "NULL array argument");
    cudaStream_t s = (cudaStream_t)stream;
    return DISPATCH(p, adj_hat<float>(p, (const C<float>*)d_hat, (float*)u, ws, s),
                    adj_hat<double>(p, (const C<double>*)d_hat, (double*)u, ws, s));
}

lam_status lam_forward(const lam_plan* p, const void* u, void* d, void* ws, void* stream) {
    if (lam_status st = lam_forward_hat(p, u, d, nullptr, ws, stream)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const double sc = 1.0 / ((double)p->h * p->w);
    return DISPATCH(p, fft2d<float>(p, (const C<float>*)d, (C<float>*)d, +1, (float)sc, s),
                    fft2d<double>(p, (const C<double>*)d, (C<double>*)d, +1, sc, s));
}

lam_status lam_adjoint(const lam_plan* p, const void* d, void* u, void* ws, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    if (!u || !d || !ws) return fail(LAM_EINVAL, "NULL array argument");
    cudaStream_t s = (cudaStream_t)stream;
    void* tmp = (char*)ws + p->ws_tmp;
    const double sc = 1.0 / ((double)p->h * p->w);
    lam_status st = DISPATCH(p, fft2d<float>(p, (const C<float>*)d, (C<float>*)tmp, -1, (float)sc, s),
                             fft2d<double>(p, (const C<double>*)d, (C<double>*)tmp, -1, sc, s));
    if (st) return st;
    return lam_adjoint_hat(p, tmp, u, ws, stream);
}

lam_status lam_fbp(const lam_plan* p, const void* d, void* u, void* ws, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    if (!d || !u || !ws) return fail(LAM_EINVAL, "NULL array argument");
    cudaStream_t s = (cudaStream_t)stream;
    return DISPATCH(p, fbp_t<float>(p, (const C<float>*)d, (float*)u, ws, s),
                    fbp_t<double>(p, (const C<double>*)d, (double*)u, ws, s));
}

lam_status lam_fft2d(const lam_plan* p, const void* in, void* out, int inverse, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    if (!in || !out) return fail(LAM_EINVAL, "NULL array argument");
    cudaStream_t s = (cudaStream_t)stream;
    const double sc = inverse ? 1.0 / ((double)p->h * p->w) : 1.0;
    const int dir = inverse ? +1 : -1;
    return DISPATCH(p, fft2d<float>(p, (const C<float>*)in, (C<float>*)out, dir, (float)sc, s),
                    fft2d<double>(p, (const C<double>*)in, (C<double>*)out, dir, sc, s));
}

lam_status tv_grad(const lam_plan* p, const void* u, void* g, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    if (!u || !g) return fail(LAM_EINVAL, "NULL array argument");
    cudaStream_t s = (cudaStream_t)stream;
    CK(DISPATCH(p, admm_ops<float>(p).grad((const float*)u, (float*)g, s),
                admm_ops<double>(p).grad((const double*)u, (double*)g, s)));
    return LAM_OK;
}

lam_status tv_div(const lam_plan* p, const void* g, void* u, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    if (!u || !g) return fail(LAM_EINVAL, "NULL array argument");
    cudaStream_t s = (cudaStream_t)stream;
    CK(DISPATCH(p, admm_ops<float>(p).div((const float*)g, (float*)u, s),
                admm_ops<double>(p).div((const double*)g, (double*)u, s)));
    return LAM_OK;
}

lam_status tv_smooth(const lam_plan* p, const void* u, double eps, void* grad, double* value, void* ws,
                     void* stream) {
    if (lam_status st = check_plan(p)) return st;
    if (!u || !ws) return fail(LAM_EINVAL, "NULL array argument");
    if (!(eps > 0) || !std::isfinite(eps)) return fail(LAM_EINVAL, "eps = %g must be positive", eps);
    cudaStream_t s = (cudaStream_t)stream;
    char* base = (char*)ws + p->ws_red;
    AdmmRed r;
    r.sc = (double*)base;
    r.partials = (double*)(base + align256(SC_COUNT * sizeof(double)));
    r.counter = (unsigned int*)(base + align256(SC_COUNT * sizeof(double)) +
                                align256((size_t)kRedBlocks * 4 * sizeof(double)));
    CK(cudaMemsetAsync(r.counter, 0, sizeof(unsigned int), s));
    CK(DISPATCH(p, admm_ops<float>(p).tv_smooth((const float*)u, (float*)grad, eps, r, 0, s),
                admm_ops<double>(p).tv_smooth((const double*)u, (double*)grad, eps, r, 0, s)));
    if (value) {
        CK(cudaMemcpyAsync(value, r.sc, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return LAM_OK;
}

lam_status lam_plan_status(const lam_plan* p, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int word = 0;
    CK(cudaMemcpyAsync(&word, p->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (word == 0) return LAM_OK;
    CK(cudaMemsetAsync(p->err, 0, sizeof(int), s));
    CK(cudaStreamSynchronize(s));
    return fail(LAM_EBOUNDS, "index check failed at site %d (%s)", word,
                word == kSiteZWeights      ? "z transpose weights"
                : word == kSiteGatherWindow ? "2D gather window"
                : word == kSiteGatherOut    ? "2D gather output"
                : word == kSiteSpreadIn     ? "2D spread input"
                : word == kSiteSelftest     ? "self-test"
                                            : "unknown");
}

int lam_bounds_checked(void) {
#ifdef LAM_BOUNDS_CHECK
    return 1;
#else
    return 0;
#endif
}

lam_status lamx_bounds_selftest(const lam_plan* p, int index, void* stream) {
#ifdef LAM_BOUNDS_CHECK
    if (lam_status st = check_plan(p)) return st;
    CK(launch_bounds_selftest(p->err + 1, index, p->err, (cudaStream_t)stream));
    return LAM_OK;
#else
    (void)p;
    (void)index;
    (void)stream;
    return fail(LAM_EUNSUPPORTED, "the self-test needs a LAM_BOUNDS_CHECK build");
#endif
}

lam_status admm_state_bytes(const lam_plan* p, size_t* bytes) {
    if (lam_status st = check_plan(p)) return st;
    if (!bytes) return fail(LAM_EINVAL, "bytes is NULL");
    *bytes = layout(p, p->lsp_form == 2 && p->memo_tau > 0).total;
    return LAM_OK;
}

lam_status admm_init(const lam_plan* p, void* state, const void* d, double alpha, double rho, int n_inner,
                     int adapt_rho, void* ws, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    if (!state || !d || !ws) return fail(LAM_EINVAL, "NULL array argument");
    if (n_inner < 1 || n_inner > 64) return fail(LAM_EINVAL, "n_inner = %d not in [1, 64]", n_inner);
    if (!(rho > 0) || !std::isfinite(rho)) return fail(LAM_EINVAL, "rho = %g must be positive", rho);
    if (!(alpha >= 0) || !std::isfinite(alpha)) return fail(LAM_EINVAL, "alpha = %g must be >= 0", alpha);
    cudaStream_t s = (cudaStream_t)stream;
    {
        std::lock_guard<std::mutex> lk(p->mu);
        AdmmHost& h = p->admm[state];
        if (h.graph) cudaGraphExecDestroy(h.graph);
        h.graph = nullptr;
        h.n_inner = n_inner;
        h.ws = ws;
        h.form = p->lsp_form;
        h.resid = p->prec == LAM_F32 ? p->resid : (p->resid & LAM_RESID_REFRESH);  // no lo part in FP64
        h.memo_tau = p->lsp_form == 2 ? p->memo_tau : 0.0;
    }
    const bool memo = p->lsp_form == 2 && p->memo_tau > 0;
    return DISPATCH(p, admm_init_t<float>(p, state, d, alpha, rho, adapt_rho, p->lsp_form, memo, s),
                    admm_init_t<double>(p, state, d, alpha, rho, adapt_rho, p->lsp_form, memo, s));
}

static lam_status lookup(const lam_plan* p, void* state, AdmmHost** h) {
    std::lock_guard<std::mutex> lk(p->mu);
    auto it = p->admm.find(state);
    if (it == p->admm.end()) return fail(LAM_EINVAL, "state was not initialised with admm_init on this plan");
    *h = &it->second;
    return LAM_OK;
}

lam_status admm_step(const lam_plan* p, void* state, void* ws, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    if (!state || !ws) return fail(LAM_EINVAL, "NULL array argument");
    AdmmHost* h;
    if (lam_status st = lookup(p, state, &h)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    return DISPATCH(p, admm_step_t<float>(p, state, ws, h->n_inner, h->form, h->resid, h->memo_tau, s),
                    admm_step_t<double>(p, state, ws, h->n_inner, h->form, h->resid, h->memo_tau, s));
}

lam_status admm_run(const lam_plan* p, void* state, void* ws, int iters, int use_graph, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    if (!state || !ws) return fail(LAM_EINVAL, "NULL array argument");
    if (iters < 0) return fail(LAM_EINVAL, "iters = %d", iters);
    AdmmHost* h;
    if (lam_status st = lookup(p, state, &h)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (!use_graph) {
        for (int k = 0; k < iters; ++k)
            if (lam_status st = admm_step(p, state, ws, stream)) return st;
        return LAM_OK;
    }
    if (s == nullptr) return fail(LAM_EINVAL, "graph replay needs a non-default stream");
    if (!h->graph || h->ws != ws) {
        if (h->graph) cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
        h->ws = ws;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        lam_status st = admm_step(p, state, ws, stream);
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(s, &g);
        if (st) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (ce != cudaSuccess) return fail(LAM_ECUDA, "stream capture failed: %s", cudaGetErrorString(ce));
        size_t nn = 0;
        h->graph_kernels = 0;
        if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
            std::vector<cudaGraphNode_t> nodes(nn);
            if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
                for (size_t i = 0; i < nn; ++i) {
                    cudaGraphNodeType ty;
                    if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel)
                        ++h->graph_kernels;
                }
        }
        ce = cudaGraphInstantiate(&h->graph, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) return fail(LAM_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
    }
    for (int k = 0; k < iters; ++k) CK(cudaGraphLaunch(h->graph, s));
    return LAM_OK;
}

void* admm_u(const lam_plan* p, void* state) {
    if (!p || !state) return nullptr;
    return (char*)state + layout(p).u;
}

lam_status admm_read_scalars(const lam_plan* p, const void* state, double* out, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    if (!state || !out) return fail(LAM_EINVAL, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(out, (const char*)state + layout(p).sc, LAM_NSCALARS * sizeof(double),
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return LAM_OK;
}

lam_status admm_read_history(const lam_plan* p, const void* state, int count, double* out, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    if (!state || !out) return fail(LAM_EINVAL, "NULL argument");
    if (count < 0 || count > kHistCap) return fail(LAM_EINVAL, "count = %d not in [0, %d]", count, kHistCap);
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(out, (const char*)state + layout(p).hist, (size_t)count * 4 * sizeof(double),
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return LAM_OK;
}

lam_status admm_status(const lam_plan* p, const void* state, void* stream) {
    double sc[LAM_NSCALARS];
    if (lam_status st = admm_read_scalars(p, state, sc, stream)) return st;
    if (sc[LAM_SC_STATUS] != 0.0) return fail(LAM_ENAN, "a non-finite value appeared in an ADMM reduction");
    return LAM_OK;
}

static bool on_device(const void* ptr) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

lam_status reconstruct(const float* data, const double* theta, double phi, int n, int nz, int det_h, int det_w,
                       int n_theta, int iters, double alpha, double rho, float* u_out) {
    if (!data || !theta || !u_out) return fail(LAM_EINVAL, "NULL argument");
    if (iters < 0) return fail(LAM_EINVAL, "iters = %d", iters);
    lam_plan* p = nullptr;
    if (lam_status st = lam_plan_create(&p, n, nz, det_h, det_w, n_theta, theta, phi, 2, 4, LAM_F32)) return st;
    size_t sb = 0;
    admm_state_bytes(p, &sb);
    const size_t nd = (size_t)p->ndata();
    void *ws = nullptr, *state = nullptr, *dreal = nullptr, *dc = nullptr;
    cudaStream_t s = nullptr;
    lam_status st = LAM_OK;
    auto cleanup = [&]() {
        if (s) cudaStreamSynchronize(s);
        cudaFree(ws);
        cudaFree(state);
        cudaFree(dreal);
        cudaFree(dc);
        if (s) cudaStreamDestroy(s);
        lam_plan_destroy(p);
    };
    if (cudaMalloc(&ws, p->ws_bytes) || cudaMalloc(&state, sb) || cudaMalloc(&dreal, nd * sizeof(float)) ||
        cudaMalloc(&dc, nd * sizeof(C<float>)) || cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) {
        cleanup();
        return fail(LAM_ENOMEM, "reconstruct: device allocation failed");
    }
    const bool in_dev = on_device(data), out_dev = on_device(u_out);
    if (cudaMemcpyAsync(dreal, data, nd * sizeof(float), in_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        s) != cudaSuccess) {
        cleanup();
        return fail(LAM_ECUDA, "reconstruct: data copy failed");
    }
    k_real_to_complex<<<1184, 256, 0, s>>>((const float*)dreal, (C<float>*)dc, (long long)nd);
    if ((st = admm_init(p, state, dc, alpha, rho, 4, 1, ws, s)) == LAM_OK)
        st = admm_run(p, state, ws, iters, 1, s);
    if (st == LAM_OK) {
        const size_t vb = (size_t)p->nvox() * sizeof(float);
        if (cudaMemcpyAsync(u_out, admm_u(p, state), vb, out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = fail(LAM_ECUDA, "reconstruct: %s", cudaGetErrorString(cudaGetLastError()));
    }
    if (st == LAM_OK) {
        double sc[LAM_NSCALARS];
        if (admm_read_scalars(p, state, sc, s) == LAM_OK && sc[LAM_SC_STATUS] != 0.0)
            st = fail(LAM_ENAN, "reconstruct: non-finite ADMM scalar");
    }
    cleanup();
    return st;
}

// ---- stage entry points (lamino_stages.h) ------------------------------------

lam_status lamx_u1d_fwd(const lam_plan* p, const void* u, void* u1, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    if (lam_status st = check_vol_align(p->prec, u)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    CK(DISPATCH(p, launch_usfft1d_fwd<float>((const float*)u, (C<float>*)u1, args1d<float>(p, p->TYf, false), s),
                launch_usfft1d_fwd<double>((const double*)u, (C<double>*)u1, args1d<double>(p, p->TYf, false), s)));
    return LAM_OK;
}

lam_status lamx_u1d_adj(const lam_plan* p, const void* u1, void* u, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    CK(DISPATCH(p, launch_usfft1d_adj<float>((const C<float>*)u1, (float*)u, args1d<float>(p, p->TYa, false), s),
                launch_usfft1d_adj<double>((const C<double>*)u1, (double*)u, args1d<double>(p, p->TYa, false), s)));
    return LAM_OK;
}

lam_status lamx_u2d_fwd(const lam_plan* p, const void* u1, void* d_hat, const void* sub, void* ws, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    return DISPATCH(p, u2d_fwd_t<float>(p, u1, d_hat, sub, ws, s), u2d_fwd_t<double>(p, u1, d_hat, sub, ws, s));
}

lam_status lamx_u2d_adj(const lam_plan* p, const void* d_hat, void* u1, void* ws, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    return DISPATCH(p, u2d_adj_t<float>(p, d_hat, u1, ws, s), u2d_adj_t<double>(p, d_hat, u1, ws, s));
}

lam_status lamx_spread(const lam_plan* p, const void* d_hat, void* ws, int j0, int nb, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    if (!d_hat || !ws) return fail(LAM_EINVAL, "NULL array argument");
    if (j0 < 0 || nb < 1 || j0 + nb > p->njobs_pair)
        return fail(LAM_EINVAL, "plane jobs [%d, %d) outside [0, %d)", j0, j0 + nb, p->njobs_pair);
    if (nb > p->nbatch) return fail(LAM_EINVAL, "nb = %d: the workspace holds %d planes", nb, p->nbatch);
    cudaStream_t s = (cudaStream_t)stream;
    return DISPATCH(p, spread_t<float>(p, d_hat, ws, j0, nb, s), spread_t<double>(p, d_hat, ws, j0, nb, s));
}

int lamx_jobs_per_batch(const lam_plan* p) { return p ? even_batch(p, p->njobs_pair) : 0; }

int lamx_job_planes(const lam_plan* p, int j0, int nb) {
    if (!p || j0 < 0 || nb < 0 || j0 + nb > p->njobs_pair) return -1;
    int planes = 0;
    for (int j = j0; j < j0 + nb; ++j) planes += p->jobs_pair_h[j].y >= 0 ? 2 : 1;
    return planes;
}

lam_status lamx_u2d_fwd_static(const lam_plan* p, const void* u1, void* d_hat, const void* sub, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    if (!u1 || !d_hat) return fail(LAM_EINVAL, "NULL array argument");
    cudaStream_t s = (cudaStream_t)stream;
    return DISPATCH(p, u2d_fwd_static_t<float>(p, u1, d_hat, sub, s), u2d_fwd_static_t<double>(p, u1, d_hat, sub, s));
}

// ---- autotuner ------------------------------------------------------------------

static void drop_admm_graphs(const lam_plan* p) {
    std::lock_guard<std::mutex> lk(p->mu);
    for (auto& kv : p->admm)
        if (kv.second.graph) {
            cudaGraphExecDestroy(kv.second.graph);
            kv.second.graph = nullptr;
        }
}

lam_status lam_plan_autotune(lam_plan* p, void* u, void* d_hat, void* ws, int reps, double* seconds, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    if (!u || !d_hat || !ws) return fail(LAM_EINVAL, "NULL array argument");
    if (reps < 1) reps = 1;
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cs;
    CK(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return fail(LAM_EINVAL, "autotuning cannot run under stream capture");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(LAM_ECUDA, "cudaEventCreate failed");
    }
    lam_status err = LAM_OK;
    // one L_hat + L_hat^H pair: warm once, then the mean of reps
    auto measure = [&](double* t) -> lam_status {
        for (int r = -1; r < reps; ++r) {
            if (r == 0 && cudaEventRecord(e0, s) != cudaSuccess) return fail(LAM_ECUDA, "cudaEventRecord failed");
            if (lam_status st = lam_forward_hat(p, u, d_hat, nullptr, ws, stream)) return st;
            if (lam_status st = lam_adjoint_hat(p, d_hat, u, ws, stream)) return st;
        }
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        *t = ms * 1e-3 / reps;
        return LAM_OK;
    };
    // coordinate descent over the launch shapes; candidates keep every
    // divisibility and shared-memory rule the plan's own choice obeys
    double best = 0;
    err = measure(&best);
    // threads per block first: each choice re-picks the lines per block
    for (int which = 0; which < 2 && !err; ++which) {
        int& thr = which ? p->pthr : p->zthr;
        const int keep = thr;
        thr = keep == 512 ? 256 : 512;
        pick_fft_shapes(p);
        double t = 0;
        if ((err = measure(&t))) break;
        if (t < best) {
            best = t;
        } else {
            thr = keep;
            pick_fft_shapes(p);
        }
    }
    struct Knob {
        int* v;
        std::vector<int> cand;
    };
    std::vector<Knob> knobs;
    {
        std::vector<int> tg;
        for (int c : {16, 32, 64})
            if (p->M1 % c == 0 && p->M2 % c == 0) tg.push_back(c);
        knobs.push_back({&p->TG, tg});
        auto halves = [](int v, int lo) {
            std::vector<int> c;
            for (int x = v; x >= lo; x /= 2) c.push_back(x);
            return c;
        };
        knobs.push_back({&p->RB, halves(p->RB, 1)});
        knobs.push_back({&p->CB, halves(p->CB, 1)});
        knobs.push_back({&p->TYf, halves(p->TYf, 2)});
        knobs.push_back({&p->TYa, halves(p->TYa, 2)});
    }
    for (size_t k = 0; k < knobs.size() && !err; ++k) {
        const int keep = *knobs[k].v;
        int chosen = keep;
        for (int c : knobs[k].cand) {
            if (c == keep) continue;
            *knobs[k].v = c;
            double t = 0;
            if ((err = measure(&t))) break;
            if (t < best) {
                best = t;
                chosen = c;
            }
        }
        *knobs[k].v = chosen;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    drop_admm_graphs(p);
    if (seconds) *seconds = best;
    return err;
}

// ---- batched operators and ADMM ------------------------------------------------

lam_status lam_batch_create(lam_batch** out, const lam_plan* const* plans, void* const* ws, int count) {
    if (!out) return fail(LAM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!plans || !ws) return fail(LAM_EINVAL, "NULL array argument");
    if (count < 1 || count > kMaxBatch) return fail(LAM_EINVAL, "count = %d not in [1, %d]", count, kMaxBatch);
    int dev = -1;
    CK(cudaGetDevice(&dev));
    for (int i = 0; i < count; ++i) {
        const lam_plan* q = plans[i];
        if (!q || !ws[i]) return fail(LAM_EINVAL, "plan or workspace %d is NULL", i);
        if (q->prec != plans[0]->prec || q->m != plans[0]->m)
            return fail(LAM_EINVAL, "plan %d: every plan of a batch needs the same precision and half-width", i);
        if (q->device != dev) return fail(LAM_EINVAL, "plan %d lives on device %d, not the current %d", i, q->device, dev);
        if (q->TS != 32)
            return fail(LAM_EUNSUPPORTED, "plan %d: batched adjoints use 32 x 32 spread tiles (n a multiple of 16)", i);
        if (q->nbatch < q->njobs_pair)
            return fail(LAM_EUNSUPPORTED, "plan %d: its workspace holds %d planes; a batch runs all %d plane jobs at once",
                        i, q->nbatch, q->njobs_pair);
    }
    lam_batch* b = new lam_batch();
    b->count = count;
    b->prec = plans[0]->prec;
    b->device = dev;
    b->m = plans[0]->m;
    for (int i = 0; i < count; ++i) {
        const lam_plan* q = plans[i];
        b->plans.push_back(q);
        b->ws.push_back(ws[i]);
        if (fft_mixed(fft_code(q->nz)) || fft_mixed(fft_code(q->M1))) b->mixed = true;
    }
    cudaError_t ce = b->prec == LAM_F32 ? configure_batch_plane<float>() : configure_batch_plane<double>();
    if (!ce) ce = b->prec == LAM_F32 ? configure_batch_z<float>() : configure_batch_z<double>();
    lam_status st = ce ? fail(LAM_ECUDA, "batched kernel configuration failed: %s", cudaGetErrorString(ce)) : LAM_OK;
    if (!st) st = b->prec == LAM_F32 ? batch_build<float>(b) : batch_build<double>(b);
    // ADMM runs concurrently by default (lam_batch_set_streams), unless two
    // problems share a workspace
    bool shared = false;
    for (int i = 0; i < count; ++i)
        for (int j = 0; j < i; ++j) shared = shared || ws[i] == ws[j];
    if (!st && !shared) st = lam_batch_set_streams(b, std::min(count, kDefaultBatchStreams));
    if (st) {
        lam_batch_destroy(b);
        return st;
    }
    *out = b;
    return LAM_OK;
}

static void release_streams(lam_batch* b) {
    for (cudaStream_t x : b->side) cudaStreamDestroy(x);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    b->side.clear();
    b->join.clear();
    b->fork = nullptr;
}

lam_status lam_batch_destroy(lam_batch* b) {
    if (!b) return LAM_OK;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    release_streams(b);
    if (b->dev) cudaFree(b->dev);
    delete b;
    return LAM_OK;
}

lam_status lam_batch_set_streams(lam_batch* b, int streams) {
    if (!b) return fail(LAM_EINVAL, "batch is NULL");
    if (streams < 0 || streams > kMaxBatch) return fail(LAM_EINVAL, "streams = %d (0 .. %d)", streams, kMaxBatch);
    if (streams > 0) {
        // problems on different streams must not share a workspace
        for (int i = 0; i < b->count; ++i)
            for (int j = 0; j < i; ++j)
                if (b->ws[i] == b->ws[j])
                    return fail(LAM_EINVAL, "problems %d and %d share a workspace: they cannot run concurrently", j, i);
    }
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != b->device) return fail(LAM_EINVAL, "current device %d is not the batch's device %d", dev, b->device);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_states.clear();
    release_streams(b);
    b->nstreams = streams;
    for (int k = 0; k < streams; ++k) {
        cudaStream_t x = nullptr;
        cudaEvent_t e = nullptr;
        CK(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
        b->side.push_back(x);
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        b->join.push_back(e);
    }
    if (streams > 0) CK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    return LAM_OK;
}

static lam_status check_batch_arrays(const lam_batch* b, const void* const* a, const void* const* c) {
    if (!b) return fail(LAM_EINVAL, "batch is NULL");
    if (!a || !c) return fail(LAM_EINVAL, "NULL array argument");
    for (int i = 0; i < b->count; ++i)
        if (!a[i] || !c[i]) return fail(LAM_EINVAL, "array %d is NULL", i);
    return LAM_OK;
}

lam_status lam_forward_hat_batched(const lam_batch* b, const void* const* u, void* const* d_hat, void* stream) {
    if (lam_status st = check_batch_arrays(b, u, (const void* const*)d_hat)) return st;
    for (int i = 0; i < b->count; ++i)
        if (lam_status st = check_vol_align(b->prec, u[i], i)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    return b->prec == LAM_F32 ? batch_fwd_hat<float>(b, u, d_hat, s) : batch_fwd_hat<double>(b, u, d_hat, s);
}

lam_status lam_adjoint_hat_batched(const lam_batch* b, const void* const* d_hat, void* const* u, void* stream) {
    if (lam_status st = check_batch_arrays(b, d_hat, (const void* const*)u)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    return b->prec == LAM_F32 ? batch_adj_hat<float>(b, d_hat, u, s) : batch_adj_hat<double>(b, d_hat, u, s);
}

lam_status lam_forward_batched(const lam_batch* b, const void* const* u, void* const* d, void* stream) {
    if (lam_status st = lam_forward_hat_batched(b, u, d, stream)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < b->count; ++i) {
        const lam_plan* p = b->plans[i];
        const double sc = 1.0 / ((double)p->h * p->w);
        if (lam_status st = DISPATCH(p, fft2d<float>(p, (const C<float>*)d[i], (C<float>*)d[i], +1, (float)sc, s),
                                     fft2d<double>(p, (const C<double>*)d[i], (C<double>*)d[i], +1, sc, s)))
            return st;
    }
    return LAM_OK;
}

lam_status lam_adjoint_batched(const lam_batch* b, const void* const* d, void* const* u, void* stream) {
    if (lam_status st = check_batch_arrays(b, d, (const void* const*)u)) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const void* tmp[kMaxBatch];
    for (int i = 0; i < b->count; ++i) {
        const lam_plan* p = b->plans[i];
        void* t = (char*)b->ws[i] + p->ws_tmp;
        const double sc = 1.0 / ((double)p->h * p->w);
        if (lam_status st = DISPATCH(p, fft2d<float>(p, (const C<float>*)d[i], (C<float>*)t, -1, (float)sc, s),
                                     fft2d<double>(p, (const C<double>*)d[i], (C<double>*)t, -1, sc, s)))
            return st;
        tmp[i] = t;
    }
    return lam_adjoint_hat_batched(b, tmp, u, stream);
}

lam_status admm_run_batched(lam_batch* b, void* const* states, int iters, int use_graph, void* stream) {
    if (!b) return fail(LAM_EINVAL, "batch is NULL");
    if (!states) return fail(LAM_EINVAL, "states is NULL");
    if (iters < 0) return fail(LAM_EINVAL, "iters = %d", iters);
    int n_inner = -1;
    int resid[kMaxBatch] = {};
    AdmmHost* hosts[kMaxBatch] = {};
    const bool conc = b->nstreams > 0;
    for (int i = 0; i < b->count; ++i) {
        if (!states[i]) return fail(LAM_EINVAL, "state %d is NULL", i);
        AdmmHost* h;
        if (lam_status st = lookup(b->plans[i], states[i], &h)) return st;
        hosts[i] = h;
        for (int j = 0; j < i; ++j)
            if (states[j] == states[i]) return fail(LAM_EINVAL, "states %d and %d are the same state", j, i);
        if (conc) continue;  // each problem runs its own admm_step: any form and options
        if (n_inner >= 0 && h->n_inner != n_inner)
            return fail(LAM_EINVAL, "state %d: every state of a batch needs the same number of CG steps", i);
        if (h->form != 2) return fail(LAM_EUNSUPPORTED, "state %d: batched ADMM runs the Algorithm 2 form", i);
        if (h->memo_tau > 0) return fail(LAM_EUNSUPPORTED, "state %d: batched ADMM does not memoize", i);
        if (h->resid & LAM_RESID_REFRESH)
            return fail(LAM_EUNSUPPORTED, "state %d: batched ADMM carries the residual (no per-LSP refresh)", i);
        resid[i] = h->resid;
        n_inner = h->n_inner;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // concurrent mode: problem i's own outer iteration (the single-plan
    // kernels, as admm_step) on side stream i mod nstreams, forked from and
    // joined to s; problems on different streams overlap on the GPU
    auto conc_step = [&]() -> lam_status {
        CK(cudaEventRecord(b->fork, s));
        for (int j = 0; j < b->nstreams; ++j) CK(cudaStreamWaitEvent(b->side[j], b->fork, 0));
        for (int i = 0; i < b->count; ++i) {
            const lam_plan* p = b->plans[i];
            const AdmmHost* h = hosts[i];
            cudaStream_t x = b->side[i % b->nstreams];
            if (lam_status st = DISPATCH(
                    p, admm_step_t<float>(p, states[i], b->ws[i], h->n_inner, h->form, h->resid, h->memo_tau, x),
                    admm_step_t<double>(p, states[i], b->ws[i], h->n_inner, h->form, h->resid, h->memo_tau, x)))
                return st;
        }
        for (int j = 0; j < b->nstreams; ++j) {
            CK(cudaEventRecord(b->join[j], b->side[j]));
            CK(cudaStreamWaitEvent(s, b->join[j], 0));
        }
        return LAM_OK;
    };
    auto step = [&]() -> lam_status {
        if (conc) return conc_step();
        return b->prec == LAM_F32 ? batch_admm_step<float>(b, states, resid, n_inner, s)
                                  : batch_admm_step<double>(b, states, resid, n_inner, s);
    };
    if (!use_graph) {
        for (int k = 0; k < iters; ++k)
            if (lam_status st = step()) return st;
        return LAM_OK;
    }
    if (s == nullptr) return fail(LAM_EINVAL, "graph replay needs a non-default stream");
    std::vector<void*> sv(states, states + b->count);
    if (!b->graph || b->graph_states != sv) {
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_states = sv;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        lam_status st = step();
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(s, &g);
        if (st) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (ce != cudaSuccess) return fail(LAM_ECUDA, "stream capture failed: %s", cudaGetErrorString(ce));
        size_t nn = 0;
        b->graph_kernels = 0;
        if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
            std::vector<cudaGraphNode_t> nodes(nn);
            if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
                for (size_t i = 0; i < nn; ++i) {
                    cudaGraphNodeType ty;
                    if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel)
                        ++b->graph_kernels;
                }
        }
        ce = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) return fail(LAM_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
    }
    for (int k = 0; k < iters; ++k) CK(cudaGraphLaunch(b->graph, s));
    return LAM_OK;
}

lam_status lamx_batch_info(const lam_batch* b, int* out, int count) {
    if (!b || !out) return fail(LAM_EINVAL, "NULL argument");
    // per stage: total work items and persistent grid; then graph kernel nodes
    int v[2 * kBStages + 1];
    for (int st = 0; st < kBStages; ++st) {
        v[2 * st] = b->total[st];
        v[2 * st + 1] = b->L[st].grid;
    }
    v[2 * kBStages] = (int)b->graph_kernels;
    for (int i = 0; i < count && i < 2 * kBStages + 1; ++i) out[i] = v[i];
    return LAM_OK;
}

lam_status lamx_plane_ffts(const lam_plan* p, const void* u1, void* P, int j0, int nb, void* stream) {
    if (lam_status st = check_plan(p)) return st;
    if (!u1 || !P) return fail(LAM_EINVAL, "NULL array argument");
    if (j0 < 0 || nb < 1 || j0 + nb > p->h) return fail(LAM_EINVAL, "planes %d + %d out of [0, %d)", j0, nb, p->h);
    cudaStream_t s = (cudaStream_t)stream;
    CK(DISPATCH(p, launch_usfft2d_planes<float>((const C<float>*)u1, (C<float>*)P, j0, nb, args2d<float>(p, false), s),
                launch_usfft2d_planes<double>((const C<double>*)u1, (C<double>*)P, j0, nb, args2d<double>(p, false),
                                              s)));
    return LAM_OK;
}

lam_status lamx_fma_peak(void* sink, int sink_floats, double* flops_per_s, void* stream) {
    if (!sink || !flops_per_s) return fail(LAM_EINVAL, "NULL argument");
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = nsm * 8, iters = 1 << 16;
    if (sink_floats < blocks) return fail(LAM_EINVAL, "sink holds %d floats; %d needed", sink_floats, blocks);
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(LAM_ECUDA, "cudaEventCreate failed");
    }
    cudaError_t e = launch_fma_peak((float*)sink, blocks, iters, s);
    if (!e) e = cudaEventRecord(e0, s);
    if (!e) e = launch_fma_peak((float*)sink, blocks, iters, s);
    if (!e) e = cudaEventRecord(e1, s);
    if (!e) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e) return fail(LAM_ECUDA, "FMA probe failed: %s", cudaGetErrorString(e));
    *flops_per_s = 2.0 * 8.0 * iters * (double)blocks * 256 / (ms * 1e-3);
    return LAM_OK;
}

lam_status lamx_admm_graph_kernels(const lam_plan* p, void* state, size_t* count) {
    if (lam_status st = check_plan(p)) return st;
    if (!count) return fail(LAM_EINVAL, "count is NULL");
    AdmmHost* h;
    if (lam_status st = lookup(p, state, &h)) return st;
    *count = h->graph ? h->graph_kernels : 0;
    return LAM_OK;
}

lam_status lamx_admm_layout(const lam_plan* p, size_t* out, int count) {
    if (lam_status st = check_plan(p)) return st;
    if (!out || count < 1) return fail(LAM_EINVAL, "out is NULL or count < 1");
    const StateLayout L = layout(p);
    const size_t v[18] = {L.sc, L.hist, L.partials, L.counter, L.u, L.du, L.Gd, L.G0, L.G1,
                          L.p, L.e, L.lam, L.dpsi, L.dhat, L.r, L.Lp, L.rlo, L.total};
    for (int i = 0; i < count && i < 18; ++i) out[i] = v[i];
    return LAM_OK;
}

lam_status lamx_plan_info(const lam_plan* p, int* out, int count) {
    if (lam_status st = check_plan(p)) return st;
    // the adjoint spread as its LAM_SPREAD_* value
    int spread = LAM_SPREAD_TILES;
    switch (p->spread) {
        case kSpreadAtomic: spread = LAM_SPREAD_ATOMIC; break;
        case kSpreadExact: spread = LAM_SPREAD_EXACT; break;
        case kSpreadHalo: spread = LAM_SPREAD_HALO; break;
        case kSpreadTilesExact: spread = LAM_SPREAD_TILES_EXACT; break;
        case kSpreadTiles2: spread = LAM_SPREAD_TILES2; break;
        case kSpreadSweep: spread = LAM_SPREAD_SWEEP; break;
        default: break;
    }
    const int v[] = {p->TYf,  p->TYa,  p->RB,   p->CB,         p->TS, p->nimg, p->nbatch,
                     p->jmin, p->jmax, p->njobs_pair, p->TG, p->zthr, p->pthr, spread};
    const int nv = (int)(sizeof(v) / sizeof(v[0]));
    for (int i = 0; i < count && i < nv; ++i) out[i] = v[i];
    return LAM_OK;
}

}  // extern "C"
