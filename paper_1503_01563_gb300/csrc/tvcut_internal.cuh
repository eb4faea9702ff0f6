// Internal declarations shared by the tvcut CUDA translation units.
// Not part of the public ABI (see include/tvcut.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "tvcut.h"

namespace tvcut {

// Chains of one grid axis k: chain c = (o, q) with o < outer = prod(dims[:k])
// and q < inner = prod(dims[k+1:]); element j of chain c sits at
// o*m*inner + q + j*inner, the weight of its edge (j, j+1) at
// o*(m-1)*inner + q + j*inner (compact layout).
struct ChainGeom {
    int64_t outer;
    int64_t inner;
    int64_t nchains;
    int m;
};

// One block of the scan launch (scan.cu): every chain of one axis.  Element j
// of chain c sits at o*m*inner + q + j*inner (c = o*inner + q), or, when
// `transposed`, at j*nchains + c; the weights follow the same rule with m-1
// elements per chain.
template <typename T>
struct ScanAxis {
    int64_t nchains;
    int64_t inner;
    int64_t block_begin;   // first CTA of this axis (set by the launcher)
    int m;
    int transposed;
    const T* v;
    const T* a;
    T* x;
};

template <typename T>
struct ScanArgs {
    int naxes;
    int force;             // 0 automatic, 1 thread per chain, 2/3/4/5: 32/16/8/4 lanes per chain
    int shadow;            // 1: write v - prox(v) (the projection onto K_k) instead of prox(v)
    ScanAxis<T> ax[3];
};

enum UpdateMode : int { UPD_AAR = 0, UPD_AP = 1, UPD_EVAL = 2 };

// Elementwise update over the grid viewed as rows x cols (cols = last dim);
// block r-1 (s and x) is stored transposed.
template <typename T>
struct UpdateArgs {
    int64_t rows;
    int64_t cols;
    int r;
    int check;
    T* s[3];
    const T* x[3];
    const T* w;
    T* xout;
};

// Per-element epilogues of one chain sweep (what is done with y = v - prox(v)).
enum SweepMode : int {
    MODE_PROJ = 0,      // out = y
    MODE_PROX = 1,      // out = x = prox(v)
    MODE_AAR_FIRST = 2, // P = w + v - 2y; block state <- y
    MODE_AAR_MID = 3,   // P += v - 2y;   block state <- y
    MODE_AAR_LAST = 4,  // c = (P + v - 2y)/r; z_k <- y_k + c for all k; x = w - sum y
    MODE_AP_FIRST = 5,  // P = w - y;      block state <- y
    MODE_AP_MID = 6,    // P -= y;         block state <- y
    MODE_AP_LAST = 7,   // c = (P - y)/r;  lambda_k <- y_k + c; x = P - y
    MODE_EVAL_FIRST = 8,// P = w - y       (state untouched)
    MODE_EVAL_MID = 9,  // P -= y
    MODE_EVAL_LAST = 10,// x = P - y
};

template <typename T>
struct SweepArgs {
    ChainGeom g;
    const T* v;        // chain input (block state or standalone input)
    const T* a;        // compact weights of the chain axis
    T* out;            // PROJ/PROX output, or the block state written with y
    T* P;              // running per-vertex sum across the blocks of one iteration
    const T* w;        // unary
    T* Z[3];           // block states (LAST modes update all of them)
    T* x;              // primal output (LAST modes when check != 0)
    int r;             // number of blocks
    int check;         // LAST modes: also write x
    int mapping;       // -1 auto, 0 thread per chain from global memory,
                       // 1/2/3 shared-memory tiles of 8/16/32 chains
};

// FP64/int64 partial sums of one check (energy, bounds, gaps).
struct CheckPartial {
    double energy;
    double lb;
    double tv;
    double ytx;
    double xabs;
    long long energy_i;
    long long n1;
    long long pad;
};

constexpr int kMaxLevels = 17;     // threshold, plus up to 8 levels on each side

struct LevelPartial {
    double energy[kMaxLevels];
    long long energy_i[kMaxLevels];
    long long n1[kMaxLevels];
};

struct DevStatus {
    CheckPartial sum;
    LevelPartial levels;
    int flags;          // validation flags of the last conversion
    unsigned absmax_bits; // max |v| of the last conversion (float bits)
    int pad[14];
};

template <typename T>
struct CheckArgs {
    int ndim;
    int64_t dims[3];
    int64_t inner[3];
    int64_t n;
    const T* x;
    const T* w;
    const T* a[3];
    uint8_t* labels;
    T threshold;
    int last_transposed;           // weights of axis ndim-1 stored transposed
    CheckPartial* partials;
    int nlevels;                   // level-set ladder size (0: none)
    T levels[kMaxLevels];
    LevelPartial* level_partials;
};

// Validation flags raised by the conversion kernels.
enum : int {
    FLAG_NONFINITE = 1,
    FLAG_NEGATIVE = 2,
    FLAG_INEXACT = 4,   // integer too large to be exact in the iterate type
};

// Launchers (sweep.cu)
template <typename T>
cudaError_t launch_sweep(int mode, const SweepArgs<T>& args, cudaStream_t s);

// Launchers (aux.cu)
constexpr int kCheckBlocks = 608;     // 4 x 152 SMs
constexpr int kCheckThreads = 256;
template <typename T>
cudaError_t launch_check(const CheckArgs<T>& args, bool exact, DevStatus* status, cudaStream_t s);
template <typename T>
cudaError_t launch_convert(const void* src, int src_dtype, T* dst, int64_t n, bool nonneg,
                           int* flags, unsigned* absmax_bits, cudaStream_t s);
template <typename T>
cudaError_t launch_labels(const T* x, T threshold, uint8_t* labels, int64_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_convert_out(const T* src, void* dst, int dst_dtype, int64_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_cold_ap(const T* w, T* state, int r, int64_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_warmstart(const T* w, const float* xhat, float tau, T* state, int r,
                             int64_t n, cudaStream_t s);

// Launchers (scan.cu)
template <typename T>
cudaError_t launch_scan(ScanArgs<T> args, cudaStream_t s);
template <typename T>
cudaError_t launch_update(int mode, const UpdateArgs<T>& args, cudaStream_t s);
template <typename T>
cudaError_t launch_transpose(const T* in, T* out, int64_t rows, int64_t cols, cudaStream_t s);
template <typename T>
cudaError_t launch_bcd_prepare(const UpdateArgs<T>& args, int skip, cudaStream_t s);

// FISTA step inputs (scan-schedule layout: the last block transposed).
template <typename T>
struct FistaArgs {
    int64_t rows;
    int64_t cols;
    int r;
    T beta;                // extrapolation weight (t_{k-1} - 1) / t_k
    const T* y[3];         // current iterate y_k
    const T* p[3];         // previous iterate y_{k-1}
    T* v[3];               // out: Pi_L(y + beta (y - p)), the point the scan projects
    const T* w;
};
template <typename T>
cudaError_t launch_fista_prepare(const FistaArgs<T>& args, cudaStream_t s);

ChainGeom chain_geom(int ndim, const int64_t* dims, int axis);

}  // namespace tvcut
