// Internal declarations shared by the tvcut CUDA translation units.
// Not part of the public ABI (see include/tvcut.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

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
    const T* a;            // compact weights (m - 1 per chain)
    const T* ap;           // the same weights in the state's layout, 0 at each chain's end; may be null
    T* x;
};

template <typename T>
struct CertifyArgs {
    ScanAxis<T> X;
    int layout;
    int first;
    int64_t H, W;
    double* Y;
};

template <typename T>
struct ScanArgs {
    int naxes;
    int force;             // 0 automatic, 1 thread per chain, 2/3/4/5: 32/16/8/4 lanes per chain
    int shadow;            // 1: write v - prox(v) (the projection onto K_k) instead of prox(v)
    ScanAxis<T> ax[4];
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
    const T* adiag;                // 8-connected 2D grid: diagonal (r, c)-(r+1, c+1) and
    const T* aanti;                // anti-diagonal (r, c+1)-(r+1, c) weights, (H-1) x (W-1); else null
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

// Rigorous discrete lower bound: block k's dual y_k (X.v, in the block's
// layout X describes, X.a its compact weights) made exactly feasible chain by
// chain and added into the FP64 vertex array Y (grid layout; written when
// `first`).  layout: 0 natural, 1 the transposed last axis (grid rows of
// length X.m), 2 / 3 the zig-zag paths of an H x W 8-connected grid.
template <typename T>
cudaError_t launch_certify_block(const CertifyArgs<T>& A, cudaStream_t s);
// part[2b] = sum of min(Y_i - w_i, 0), part[2b+1] = sum of |min(Y_i - w_i, 0)| + |Y_i|
// over CTA b's share (kCheckBlocks CTAs)
template <typename T>
cudaError_t launch_certify_lb(const double* Y, const T* w, int64_t n, double* part, cudaStream_t s);

// Launchers (scan.cu)
template <typename T>
cudaError_t launch_scan(ScanArgs<T> args, cudaStream_t s);
// ap[idx] = the weight after element idx of its chain, 0 at a chain's last
// element, for every idx of a block stored as X describes (X.a compact).
template <typename T>
cudaError_t launch_pad_weights(const ScanAxis<T>& X, T* ap, cudaStream_t s);
// Chain prox by parametric min-cuts with message passing (mpprox.cu): one CTA
// per chain, chains of at most kMpMaxLen elements.
constexpr int kMpMaxLen = 2048;

// Lane-group chain prox (lanescan.cu): G lanes per chain for launches with
// few, long chains; the local form, or the funnel form for mapping 11.
template <typename T>
bool lane_scan_fits(int m);
template <typename T>
cudaError_t launch_lane_scan(ScanArgs<T> wrp, cudaStream_t s);
template <typename T>
bool funnel_scan_fits(int m);
template <typename T>
cudaError_t launch_funnel_scan(ScanArgs<T> fun, cudaStream_t s);
template <typename T>
cudaError_t launch_mp_prox(const ScanArgs<T>& A, cudaStream_t s);
template <typename T>
cudaError_t launch_update(int mode, const UpdateArgs<T>& args, cudaStream_t s);
template <typename T>
cudaError_t launch_transpose(const T* in, T* out, int64_t rows, int64_t cols, cudaStream_t s);
template <typename T>
cudaError_t launch_bcd_prepare(const UpdateArgs<T>& args, int skip, cudaStream_t s);

// 8-connected 2D grids (Sec. 3.1, Fig. 2 middle): blocks 2 and 3 are the
// zig-zag paths between rows (2p, 2p+1) and (2p+1, 2p+2).  Path q starts at
// (q, 0); in column c it sits at row zz_row(q, c) (its partner row in odd
// columns when row q is paired in that block).  Element c of path q is
// stored at c * H + q, like the transposed row block, so every path scan is
// coalesced.  zz_row is an involution in each column, so it also maps a
// vertex (r, c) to its position: path zz_row(r, c).
__host__ __device__ __forceinline__ int zz_row(int q, int c, int H, int block)
{
    if (!(c & 1)) return q;
    if (block == 2) return (q ^ 1) < H ? (q ^ 1) : q;
    if (q == 0) return 0;
    const int p = 1 + ((q - 1) ^ 1);
    return p < H ? p : q;
}

template <typename T>
struct Update8Args {
    int64_t rows;          // H
    int64_t cols;          // W
    int check;
    T* s[4];               // block states: natural, transposed, zig-zag (even), zig-zag (odd)
    const T* x[4];         // block prox outputs, same layouts
    const T* w;
    T* xout;
};
template <typename T>
cudaError_t launch_update8(int mode, const Update8Args<T>& args, cudaStream_t s);

// Dual-iterate passes of an 8-connected grid (states hold y_k):
//   PREP8_BCD:    v = w - sum_{j != k} y_j into out[k], in block k's layout;
//   PREP8_PRIMAL: x = w - sum_j y_j into xout (grid layout);
//   PREP8_FISTA:  out[j] = Pi_L(y + beta (y - p))_j for all four blocks.
enum Prep8Kind : int { PREP8_BCD = 0, PREP8_PRIMAL = 1, PREP8_FISTA = 2 };
template <typename T>
struct Prep8Args {
    int64_t rows;
    int64_t cols;
    int k;                 // PREP8_BCD: the block being updated
    T beta;                // PREP8_FISTA
    const T* y[4];
    const T* p[4];         // PREP8_FISTA: previous iterate
    T* out[4];
    const T* w;
    T* xout;
};
template <typename T>
cudaError_t launch_prep8(int kind, const Prep8Args<T>& args, cudaStream_t s);
// path weights of block 2 or 3 ((W-1) x H, element c of path q at c * H + q)
// from the diagonal and anti-diagonal weights ((H-1) x (W-1), natural)
template <typename T>
cudaError_t launch_zz_weights(const T* ad, const T* aa, T* wz, int H, int W, int block, cudaStream_t s);
// natural (H x W) <-> path layout of block 2 or 3
template <typename T>
cudaError_t launch_zz_relayout(const T* in, T* out, int H, int W, int block, bool to_paths, cudaStream_t s);

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

// A 2D 4-connected handle's problem as the learned warm start reads it
// (unet.cu): device unary and weights in the handle's layouts, its state
// blocks, the scale of the network's features and the handle's stream.
struct ProblemView {
    int esize;               // 4 (FP32 iterates) or 8 (FP64)
    int64_t H, W;
    const void* w;           // H x W
    const void* a0;          // (H-1) x W vertical weights (r, c)-(r+1, c) at r*W + c
    const void* a1;          // horizontal weights (r, c)-(r, c+1): at r*(W-1) + c, or c*H + r when a1_transposed
    int a1_transposed;
    void* s0;                // state block 0 (columns), H x W
    void* s1;                // state block 1 (rows): r*W + c, or c*H + r when s1_transposed
    int s1_transposed;
    double scale;            // max(max|w|, max a) of the inputs as set
    cudaStream_t stream;
};
// OK, or INVALID / STATE with `why` set (not a 2D 4-connected grid, inputs missing).
tvcut_status problem_view(tvcut_t h, ProblemView* v, std::string* why);
// After the state was written from outside tvcut.cu: restart FISTA's momentum
// and drop the cached primal and labels (stream-ordered on the handle's stream).
tvcut_status state_written(tvcut_t h);

}  // namespace tvcut
