/*
 * tvcut -- exact minimum cuts of submodular pairwise grid energies on one
 * GB300 GPU, by total-variation denoising and product-space projection
 * methods, after "Convex Optimization for Parallel Energy Minimization"
 * (Kumar, Barbero, Jegelka, Sra, Bach).
 *
 * Problem (Sec. 2, Eq. 1-2 and problem (D)): on a 2D 4-connected or 3D
 * 6-connected grid with n vertices, find labels l in {0,1}^n minimising
 *     E(l) = sum_e a_e [l_i != l_j] - sum_i w_i l_i ,    a_e >= 0,
 * where every undirected grid edge e = (i, j) is counted once.  Label 1 is
 * favoured where w_i > 0 (the paper's sign: E = f(x) - w^T x).
 *
 * Method (Sec. 2.3-4): solve the TV-denoising problem
 *     min_x f(x) + 1/2 ||x - w||^2 ,   f(x) = sum_e a_e |x_i - x_j| ,
 * by splitting f into one block of chains per grid axis (Sec. 3.1) and running
 * averaged alternating reflections (Eq. 3) or alternating projections
 * (Sec. 4.2) in the product space; every projection onto a block is an exact
 * weighted 1D-TV prox on each of its chains (Sec. 3.2).  The labels are the
 * thresholded primal, l_i = [x_i > threshold] with threshold 0 by default
 * (Sec. 2.3).
 *
 * Layout.  Grids are row-major with the LAST axis fastest (numpy order):
 * dims = {H, W} or {D, H, W}, vertex (i_0, .., i_{ndim-1}) at flat index
 * sum_k i_k * prod(dims[k+1:]).  Edge weights along axis k are one array in
 * "compact" layout: the grid's shape with dims[k]-1 along axis k, entry
 * (.., i_k, ..) being the weight of the edge between (.., i_k, ..) and
 * (.., i_k + 1, ..).  Product-space states hold ndim arrays of n values, the
 * block of axis k at offset k*n.
 *
 * Memory and streams.  Every handle owns its device buffers.  Input pointers
 * are read during the call and never retained; output buffers belong to the
 * caller.  `space` says whether a pointer is host (TVCUT_HOST) or device
 * (TVCUT_DEVICE) memory.  All work is ordered on the stream given at
 * creation (NULL = the legacy default stream); calls that return results to
 * the host synchronise that stream.
 *
 * Errors.  Every call returns a tvcut_status; no exception or abort crosses
 * the ABI.  tvcut_last_error(h) describes the last failure on h (or, with
 * h == NULL, the last failure of a call without a valid handle on this
 * thread).  A handle is not thread-safe.
 */
#ifndef TVCUT_H
#define TVCUT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tvcut_ctx* tvcut_t;

typedef enum {
    TVCUT_OK = 0,
    TVCUT_NOT_CONVERGED = 1,   /* max_iters reached without a stop criterion */
    TVCUT_ERR_INVALID = -1,    /* bad argument or input value */
    TVCUT_ERR_CUDA = -2,       /* a CUDA call failed (message has details) */
    TVCUT_ERR_OOM = -3,        /* device allocation failed */
    TVCUT_ERR_STATE = -4,      /* call out of order (e.g. iterate before inputs) */
    TVCUT_ERR_TIMEOUT = -5     /* a bounded device-side wait gave up */
} tvcut_status;

enum { TVCUT_I32 = 0, TVCUT_F32 = 1, TVCUT_F64 = 2 };    /* element types */
enum { TVCUT_HOST = 0, TVCUT_DEVICE = 1 };                /* pointer space */
enum { TVCUT_AAR = 0, TVCUT_AP = 1, TVCUT_BCD = 2, TVCUT_FISTA = 3 };  /* algorithms */

typedef struct {
    int algo;            /* TVCUT_AAR (Eq. 3, default), TVCUT_AP (Sec. 4.2) or
                            TVCUT_BCD (Sec. 4.1, cyclic projections: blocks in
                            turn, y_k <- Pi_{K_k}(w - sum_{j != k} y_j); state y,
                            cold start 0) or TVCUT_FISTA (Sec. 4.1, accelerated
                            projected gradient on the smooth dual
                            1/2 ||sum_k y_k - w||^2 with step 1/r:
                            y <- Pi_K(Pi_L(u)), u = y + ((t_{k-1} - 1)/t_k)(y - y_prev);
                            state y, cold start 0; one extra ndim*n buffer).
                            BCD and FISTA need mapping -1, 0 or 5..9. */
    int iterate_dtype;   /* TVCUT_F32 (default) or TVCUT_F64: precision of the
                            state and of the chain prox; gaps and energies are
                            always accumulated in FP64 (and int64 for exact
                            integer energies) */
    int check_every;     /* evaluate labels, energy and gaps every k
                            iterations (default 10; the last iteration of each
                            tvcut_iterate call is always evaluated) */
    int mapping;         /* iteration schedule: -1 automatic (default) or 0:
                            one scan launch computes the chain prox of every
                            block (the last axis' block stored transposed so
                            that all loads coalesce), then one elementwise
                            update launch; the scan gives each chain a thread,
                            or, when there are too few chains to fill the GPU,
                            a group of lanes (speculative pieces, see
                            csrc/lanescan.cu: the lane count and the kernel
                            form are chosen per launch shape by timing trial
                            launches on the caller's stream, which never
                            changes a result);
                            5: that schedule with thread-per-chain scans
                            forced; 6, 7, 8, 9: with 32, 16, 8 or 4 lanes per
                            chain (speculative pieces) forced; 10: the chain
                            prox by parametric min-cuts with message passing
                            (Sec. 3.2, "Message passing"), one CTA per chain
                            of up to 2048 elements (longer chains as 5); 11:
                            the speculative pieces of 6..9 with the funnel
                            form of the taut string (no restarts behind a
                            bend, linear in the chain length), lanes per
                            chain chosen as in the automatic rule; 1, 2,
                            3: one fused
                            sweep per block (prox and update in the same pass)
                            on shared-memory tiles of 8, 16, 32 chains; 4: the
                            fused sweeps with one thread per chain reading
                            global memory */
    double gap_tol;      /* stop when the TV duality gap f(x) - y^T x
                            (Sec. 2.3) is <= gap_tol; 0 disables (default) */
    double threshold;    /* labels are [x_i > threshold] (default 0) */
    int level_sets;      /* L >= 0: each check also evaluates the level sets
                            [x_i > threshold +- S 10^-j], j = 2..L+1, S = max|w|,
                            and keeps the lowest-energy one.  Sec. 2.1: every
                            level set of a solution of the relaxation solves
                            (D); near convergence this removes the arbitrary
                            signs of iterates on regions where x* is exactly 0.
                            Default 8 (at most 8); 0 thresholds at `threshold`
                            only */
    int connectivity;    /* 0 (default) or 4 / 6: edges along the axes (2D
                            4-connected, 3D 6-connected); 8: a 2D grid that
                            also has diagonal and anti-diagonal edges, split
                            (Sec. 3.1, Fig. 2 middle) into columns, rows and
                            two blocks of zig-zag paths between rows (2p, 2p+1)
                            and (2p+1, 2p+2); weights axis 2 = diagonal edges
                            (r, c)-(r+1, c+1), axis 3 = anti-diagonal edges
                            (r, c+1)-(r+1, c), both (H-1) x (W-1) row-major.
                            8 needs ndim 2 and the scan schedule (mapping -1, 0
                            or 5..9); states then have 4*n values */
    int certify;         /* when to evaluate the rigorous lower bound
                            (stats.certified_lb) on integer data: 0 (default)
                            for FP64 iterates when the approximate bound is
                            within 1 + 1e-7 |energy| of the energy, never for
                            FP32 iterates; 2: when close, for both (FP32
                            iterates then get their block duals recomputed in
                            FP64 from the FP32 state, about the cost of one
                            FP64 iteration, and certify grids of 10^7
                            vertices); 1: at every check */
    int stop_on_approx;  /* 1: tvcut_iterate also stops when energy -
                            discrete_lb < 1 on integer data, the certificate
                            evaluated with the iterate's own (approximate)
                            dual.  Not a proof, and no FP64 work: the cheap
                            stop rule for FP32 iterates (certify 2 turns the
                            same moment into a proof).  Default 0 */
    int reserved[4];     /* must be zero */
} tvcut_params;

typedef struct {
    int64_t iters;         /* iterations run since the last cold start */
    double energy;         /* E(l) of the current labels (FP64 sum) */
    int64_t energy_i64;    /* E(l) in exact integer arithmetic; valid when
                              energy_exact != 0 */
    int energy_exact;      /* unary and all weights were set as TVCUT_I32 */
    int certified;         /* energy_exact and energy - certified_lb < 1:
                              with integer data the labels are then a minimum
                              cut (Sec. 2.2 certificate), whatever the iterate
                              precision */
    double discrete_lb;    /* sum_i min(y_i - w_i, 0) = -sum_i max(x_i, 0) with
                              y = w - x, the dual bound of problem (C) (Sec. 2.2)
                              at the iterate; only approximately a lower bound
                              on E*, since y lies in K up to the rounding of the
                              iterates (with drifting FP32 AAR states it can
                              exceed E* by far) */
    double tv_value;       /* f(x) */
    double tv_gap;         /* f(x) - y^T x, the TV duality gap (Sec. 2.3) */
    double x_absmax;       /* max_i |x_i| */
    int64_t n_label1;      /* number of vertices labelled 1 */
    double threshold;      /* level at which the labels were cut */
    double certified_lb;   /* a rigorous lower bound on E*: the block duals of
                              the current state (BCD, FISTA: the state; AAR,
                              AP: its chain projections) made exactly feasible
                              chain by chain (running sums of each chain's dual
                              clamped to [-a, a]) and evaluated as
                              sum_i min(y_i - w_i, 0) in FP64, minus a bound on
                              that sum's rounding.  With FP32 iterates the
                              block duals are recomputed in FP64 from the FP32
                              state first (AAR, AP: FP64 chain projections;
                              BCD, FISTA: one FP64 block-coordinate sweep), as
                              duals computed in FP32 leave the bound ~1e-5 |E|
                              low on large grids.  When it is evaluated: see
                              params.certify; -infinity when not evaluated */
    int64_t reserved[2];
} tvcut_stats;

/* Fill *p with the defaults listed above. */
void tvcut_default_params(tvcut_params* p);

/* Create a solver for one grid.  ndim is 2 or 3; dims[k] >= 1.  p may be
 * NULL (defaults).  cuda_stream is a cudaStream_t or NULL.  Allocates the
 * device state (about (2 ndim + 4) n values of the iterate type plus n
 * bytes).  Errors: INVALID (bad ndim/dims/params), OOM, CUDA. */
tvcut_status tvcut_create(int ndim, const int64_t* dims, const tvcut_params* p,
                          void* cuda_stream, tvcut_t* out);

/* Release every device buffer of h (h may be NULL). */
void tvcut_destroy(tvcut_t h);

/* Message of the last failure on h (h == NULL: this thread's last failure
 * without a handle).  The string stays valid until the next call on h. */
const char* tvcut_last_error(tvcut_t h);

/* Set the unary terms w (n values in grid layout).  dtype TVCUT_I32,
 * TVCUT_F32 or TVCUT_F64.  Values must be finite; with an FP32 iterate,
 * integers must satisfy |w_i| <= 2^24 so that they stay exact.
 * Resets the iteration state to a cold start. Errors: INVALID, CUDA. */
tvcut_status tvcut_set_unary(tvcut_t h, const void* w, int dtype, int space);

/* Set the edge weights along grid axis `axis` (0 <= axis < ndim) in compact
 * layout (see above).  Values must be finite and >= 0 (submodularity, Eq. 2);
 * the same 2^24 rule applies to integers with an FP32 iterate.  Resets the
 * iteration state to a cold start.  Errors: INVALID, CUDA. */
tvcut_status tvcut_set_weights(tvcut_t h, int axis, const void* a, int dtype,
                               int space);

/* Cold start: AAR z = 0, AP lambda_k = w / ndim (the projection of 0 onto the
 * consensus set L of Eq. dualdec), BCD y = 0.  Errors: STATE (no unary yet),
 * CUDA. */
tvcut_status tvcut_reset(tvcut_t h);

/* Run up to max_iters iterations (max_iters >= 1).  Every check_every
 * iterations and after the last one, the primal x = w - sum_k y_k of the
 * current shadow (Eq. dualA, Sec. 2.3) is thresholded and its energy and
 * gaps are evaluated; iteration stops early when `certified` holds, when the
 * TV gap reaches gap_tol, or (params.stop_on_approx) when energy -
 * discrete_lb < 1.  Returns OK when a criterion held, NOT_CONVERGED when
 * max_iters ran out, STATE if unary or weights are missing, CUDA on device
 * errors.  out (may be NULL) receives the statistics of the last check. */
tvcut_status tvcut_iterate(tvcut_t h, int64_t max_iters, tvcut_stats* out);

/* Labels of the latest primal (computed from the current state when no
 * check has run since the last change): labels[i] = [x_i > t] for the n
 * vertices, t the level chosen by the last check (stats.threshold), uint8, written to `labels` in `space` (labels may be NULL
 * to get statistics only).  out (may be NULL) receives energy and gaps.
 * Errors: STATE, INVALID, CUDA. */
tvcut_status tvcut_cut(tvcut_t h, uint8_t* labels, int space, tvcut_stats* out);

/* Copy the latest primal x (n values) out as TVCUT_F32 or TVCUT_F64. */
tvcut_status tvcut_get_primal(tvcut_t h, void* x, int dtype, int space);

/* Copy the product-space state (ndim*n values of the iterate type: z for AAR,
 * lambda for AP, the block duals y for BCD and FISTA) out of / into the
 * handle: checkpoint, resume, and the warm start of Sec. 4.4 (reuse the state
 * of a similar, earlier problem).  Setting a FISTA state restarts its
 * momentum (previous iterate = the state, t = 1). */
tvcut_status tvcut_get_state(tvcut_t h, void* s, int space);
tvcut_status tvcut_set_state(tvcut_t h, const void* s, int space);

/* Shadow dual variables of the current state: y_k = Pi_{K_k}(s_k), the
 * projection of each block's state onto its polytope (Sec. 4.2-4.3), ndim*n
 * values of the iterate type in grid layout.  These are the y_i that Sec. 4.4
 * reuses to warm-start a similar problem: tvcut_set_state(h2, y) starts h2
 * from them.  (Reusing the state itself also carries its divergent part,
 * which grows with the iteration count, Sec. 4.3.)  For TVCUT_BCD and
 * TVCUT_FISTA the state is already y and this copies it.  Errors: STATE, CUDA. */
tvcut_status tvcut_get_dual(tvcut_t h, void* y, int space);

/* Warm start from a predicted primal xhat (n FP32 values): every block gets
 * s_k = (w - xhat)/ndim + tau * xhat.  (With tau = 0 the blocks split w - xhat
 * evenly; tau > 0 adds the drift that the AAR iterates acquire, Sec. 4.3.)
 * Errors: STATE, INVALID, CUDA. */
tvcut_status tvcut_warmstart_primal(tvcut_t h, const float* xhat, float tau,
                                    int space);

/* Stateless chain operator on device arrays: for every chain along `axis` of
 * a grid with the given dims, computes the exact weighted 1D-TV prox
 * (Sec. 3.2) of v with the compact weights a (what = 1: out = prox(v)) or the
 * projection onto that block's polytope (what = 0: out = v - prox(v), Sec.
 * 2.3 and 3.3).  v, a, out are DEVICE pointers of dtype TVCUT_F32 or
 * TVCUT_F64 (all the same); out may equal v.  Allocates nothing; ordered on
 * `cuda_stream`; does not synchronise.  Errors: INVALID, CUDA (launch). */
tvcut_status tvcut_project_chains(int ndim, const int64_t* dims, int axis,
                                  const void* v, const void* a, void* out,
                                  int dtype, int what, void* cuda_stream);

/* Tracing.  Kernel kinds counted and timed per handle. */
enum {
    TVCUT_K_PROX = 0,     /* chain prox of the blocks: the scan launch (all blocks
                             at once), or the fused sweeps of blocks 0..ndim-2 */
    TVCUT_K_UPDATE = 1,   /* reflection/averaging update: the update launch, or
                             the fused sweep of the last block */
    TVCUT_K_CHECK = 2,    /* threshold + energy + gap evaluation and reductions */
    TVCUT_K_OTHER = 3,    /* conversions, layout changes, cold/warm starts */
    TVCUT_NKINDS = 4
};

/* enable != 0: bracket every later kernel launch of h with CUDA events on
 * h's stream and accumulate device time per kind; 0: stop.  Either way the
 * accumulated times and launch counts are reset.  Errors: INVALID, CUDA. */
tvcut_status tvcut_profile(tvcut_t h, int enable);

/* Read the accumulators: ms[TVCUT_NKINDS] (device milliseconds, only while
 * profiling) and launches[TVCUT_NKINDS] (kernel launches since the last
 * tvcut_profile call; counted always).  Synchronises h's stream. */
tvcut_status tvcut_profile_read(tvcut_t h, double* ms, int64_t* launches);

/* ---- Batched grids -------------------------------------------------------
 * Many independent 2D grids of different sizes solved together (the method
 * above on each grid; the grids share nothing).  One iteration of every grid
 * is one chain-prox launch over all chains of all grids (persistent CTAs
 * taking work items, longest chains first) and one update launch over all
 * vertices; each tvcut_batch_iterate call (its iterations and the closing
 * check) runs as one CUDA graph, captured on first use for that iteration
 * count and replayed afterwards.  Parameters as for tvcut_create (mapping is
 * ignored; tvcut_batch_autotune picks the launch shape); algo TVCUT_AAR,
 * TVCUT_AP or TVCUT_FISTA (one step launch, the projection-mode scan and a
 * one-thread momentum launch per iteration; the momentum sequence is kept on
 * the device, so replays continue it).  TVCUT_BCD is refused (INVALID). */
typedef struct tvcut_batch_ctx* tvcut_batch_t;

/* G grids; dims holds G pairs {H_g, W_g} (1 <= H_g, W_g <= 2^20).  Allocates
 * about 8 arrays of sum_g H_g W_g values (10 for FISTA).  Errors: INVALID,
 * OOM, CUDA. */
tvcut_status tvcut_batch_create(int G, const int64_t* dims, const tvcut_params* p,
                                void* cuda_stream, tvcut_batch_t* out);
void tvcut_batch_destroy(tvcut_batch_t b);
const char* tvcut_batch_last_error(tvcut_batch_t b);

/* Inputs of grid g, as tvcut_set_unary / tvcut_set_weights (axis 0: the
 * (H-1) x W vertical weights, axis 1: the H x (W-1) horizontal weights). */
tvcut_status tvcut_batch_set_unary(tvcut_batch_t b, int g, const void* w, int dtype,
                                   int space);
tvcut_status tvcut_batch_set_weights(tvcut_batch_t b, int g, int axis, const void* a,
                                     int dtype, int space);

/* Cold start of every grid (as tvcut_reset).  Errors: STATE, CUDA. */
tvcut_status tvcut_batch_reset(tvcut_batch_t b);

/* Exactly `iters` iterations of every grid, then a check of every grid
 * (labels, energy, bounds, level sets).  out: NULL or G tvcut_stats.  For
 * batched grids `certified` compares the energy with the approximate bound
 * discrete_lb (the rigorous certified_lb of single grids is not evaluated
 * here and reads -infinity): a screen, not a proof, with FP32 iterates.
 * Returns OK if every grid is so certified, NOT_CONVERGED otherwise. */
tvcut_status tvcut_batch_iterate(tvcut_batch_t b, int64_t iters, tvcut_stats* out);

/* Labels (H_g x W_g uint8) and statistics of grid g after the last check. */
tvcut_status tvcut_batch_cut(tvcut_batch_t b, int g, uint8_t* labels, int space,
                             tvcut_stats* out);

/* Product-space state of grid g (2 x H_g x W_g values of the iterate type). */
tvcut_status tvcut_batch_get_state(tvcut_batch_t b, int g, void* s, int space);

/* Time the chain-prox launch for CTA sizes {64, 128, 256}, {4, 8, 16} CTAs
 * per SM and three forms of the scan step (0: with branches; 1: predicated,
 * so that the lanes of a warp share one instruction stream; 2: with branches
 * on weights padded to the state layout, each element loaded one step ahead)
 * on the current inputs and keep the fastest; chosen (may be NULL, else 3
 * ints) receives {threads, ctas_per_sm, step}.  The three steps do the same
 * arithmetic, so results do not depend on the choice.  FISTA's projection
 * scan takes step 0 when 2 is chosen. */
tvcut_status tvcut_batch_autotune(tvcut_batch_t b, int* chosen);

/* Set the chain-prox launch without timing (e.g. a choice saved from an
 * earlier tvcut_batch_autotune): threads in {64, 128, 256}, ctas_per_sm in
 * 1..32, step in {0, 1, 2} as above; anything else is TVCUT_ERR_INVALID. */
tvcut_status tvcut_batch_set_launch(tvcut_batch_t b, int threads, int ctas_per_sm, int step);

/* ---- Learned warm start -------------------------------------------------
 * A U-Net (4 levels, `base` channels at full resolution, 3x3 convolutions
 * with ReLU, 2x2 average pooling, nearest 2x upsampling, skip
 * concatenations) with BF16 weights/activations and FP32 accumulation and
 * master weights, trained on the GPU by its own forward/backward kernels and
 * Adam.  It maps a 2D problem to the per-block dual variables y_0, y_1 of the
 * product-space iteration; a solver started from z = y_hat (tvcut_set_state)
 * begins from the predicted iterate instead of 0 (the warm start of Sec.
 * 4.4 reuses dual variables).  Input: batch x H x W x 3 FP32 (caller-
 * normalised w, vertical and horizontal weight of each vertex); output:
 * batch x H x W x 2 FP32.  H and W must be multiples of 8.  Parameters are
 * one FP32 vector: for each of the 18 convolutions in forward order, weights
 * [9][Cout][Cin] (tap 3*ky + kx reads pixel (y+ky-1, x+kx-1)) then bias
 * [Cout]. */
typedef struct tvcut_unet_ctx* tvcut_unet_t;

tvcut_status tvcut_unet_create(int base, int batch, int H, int W, uint64_t seed,
                               void* cuda_stream, tvcut_unet_t* out);
void tvcut_unet_destroy(tvcut_unet_t u);
const char* tvcut_unet_last_error(tvcut_unet_t u);
/* Reallocate activations for a new batch/size (parameters kept). */
tvcut_status tvcut_unet_resize(tvcut_unet_t u, int batch, int H, int W);
/* in, out: DEVICE pointers; out may be NULL (keeps the result internal). */
tvcut_status tvcut_unet_forward(tvcut_unet_t u, const float* in, float* out);
/* After a forward: MSE loss against target (DEVICE, batch x H x W x 2),
 * parameter gradients (overwritten), loss to *loss (host, may be NULL).
 * Deterministic: every reduction (weight and bias gradients, loss) sums its
 * per-block partials in a fixed order, so equal inputs give equal bits and
 * training from the same seed is reproducible.  The first call at a shape
 * allocates the partials' scratch (a few MB). */
tvcut_status tvcut_unet_backward(tvcut_unet_t u, const float* target, float* loss);
/* One Adam step on the FP32 master weights. */
tvcut_status tvcut_unet_adam(tvcut_unet_t u, float lr, float beta1, float beta2, float eps);
tvcut_status tvcut_unet_num_params(tvcut_unet_t u, int64_t* count);
/* which = 0: parameters, 1: last gradients; dst is HOST memory. */
tvcut_status tvcut_unet_get_params(tvcut_unet_t u, float* dst, int which);
tvcut_status tvcut_unet_set_params(tvcut_unet_t u, const float* src);
/* Single-layer kernels (DEVICE, BF16 as raw 16-bit words, NHWC, channels
 * multiples of 16): out = relu?(bias + conv3x3(in, wt)) with wt
 * [9][Cout][Cin]; dw[9][Cout][Cin] += sum_p dout[p][co] in[p + tap][ci]
 * (the single-layer weight gradient adds with atomics: its summation order,
 * and so its last bits, may vary between calls). */
tvcut_status tvcut_conv3x3_bf16(const void* in, const void* wt, const float* bias, void* out,
                                int N, int H, int W, int Cin, int Cout, int relu,
                                void* cuda_stream);
tvcut_status tvcut_conv3x3_wgrad_bf16(const void* in, const void* dout, float* dw, int N,
                                      int H, int W, int Cin, int Cout, void* cuda_stream);

/* tvcut_conv3x3_bf16 with the engine chosen: 0 automatic (what
 * tvcut_conv3x3_bf16 does), 1 the mma.sync kernel, 2 the tcgen05 kernel
 * (tensor memory accumulators, TMA-loaded operands; persistent CTAs with
 * the TMA producer, the MMA issuer and the epilogue in separate warps and
 * two accumulator buffers, so that one tile's epilogue overlaps the next
 * tile's loads and MMAs; for 16-64 input channels the tile's three input
 * rows are loaded once and all nine taps read from them), 3 the tcgen05
 * kernel with one 128-pixel tile per CTA, 4 the persistent tcgen05 kernel
 * without the three-row form.  All tcgen05 forms issue the same MMAs in the
 * same order, so their outputs are identical.  2-4 are INVALID for shapes
 * the tcgen05 kernel does not take: it
 * needs Cin 16, 32 or a multiple of 64, Cout <= 256, W a multiple of 128 or
 * a divisor of 128, H*W a multiple of 128, 16-byte aligned tensors.
 * Stream-ordered; a tcgen05 launch that gives up waiting (2 s per wait) is
 * reported by tvcut_conv_tc_error. */
tvcut_status tvcut_conv3x3_bf16_ex(const void* in, const void* wt, const float* bias, void* out,
                                   int N, int H, int W, int Cin, int Cout, int relu, int engine,
                                   void* cuda_stream);

/* Synchronises the device; returns 1 if a tcgen05 convolution gave up
 * waiting since the last call (and clears that), 0 if not, -1 on a CUDA
 * error. */
int tvcut_conv_tc_error(void);

/* Test hook for the bounded waits: while on (nonzero), CTA 0 of every
 * tcgen05 convolution launched skips its first operand load, so that its
 * MMA issuer's wait gives up after 2 s; the launch then ends (every role of
 * every CTA stops at its next tile and frees its tensor memory), its output
 * is incomplete, and tvcut_conv_tc_error reports 1.  Off by default; the
 * convolutions are unaffected while it is off. */
tvcut_status tvcut_conv_tc_stall(int on);

/* Learned warm start of a solver handle (row a8; the warm start of Sec. 4.4
 * reuses dual variables, here they are predicted): the network's input is
 * built on the device from h's unary and edge weights as set -- pixel (r, c)
 * gets [w, a_vertical (r,c)-(r+1,c), a_horizontal (r,c)-(r,c+1)] / s with
 * s = max(max|w|, max a), 0 on the last row / column -- the forward pass runs,
 * and output channel k times s becomes block k's state (z = y_hat for AAR and
 * AP, y = y_hat for BCD and FISTA, whose momentum restarts).  h must be a 2D
 * 4-connected grid with H and W multiples of 8; the network is resized to
 * (1, H, W) when its shape differs (that reallocates its activations).  The
 * work is ordered after h's stream and h's stream after it; nothing
 * synchronises.  Errors (tvcut_unet_last_error(u)): INVALID, STATE (h's
 * inputs missing), OOM, CUDA. */
tvcut_status tvcut_unet_predict_state(tvcut_unet_t u, tvcut_t h);

/* The U-Net's convolutions (forward and input gradient): engine 0 (default)
 * uses the persistent tcgen05 kernel for every layer whose shape it takes
 * and the mma.sync kernel for the others; 1 uses the mma.sync kernel
 * throughout; 3 is 0 with the one-tile-per-CTA tcgen05 kernel, 4 is 0
 * without the three-row form (the engines of tvcut_conv3x3_bf16_ex). */
tvcut_status tvcut_unet_set_engine(tvcut_unet_t u, int engine);

/* Diagnostic of mapping 10 (the message-passing chain prox): the number of
 * chains, since the library was loaded or last reset, whose result failed
 * the FP64 check of the chain prox's optimality conditions and was
 * recomputed by the taut string.  *count receives it; reset != 0 sets it to
 * 0.  Synchronises the device.  Errors: INVALID (NULL count), CUDA. */
tvcut_status tvcut_mp_fallbacks(unsigned long long* count, int reset);

/* Iterations without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot let a library allocate
 * device memory -- code whose framework allocator owns all of the GPU's
 * memory, or latency-critical loops where a cudaMalloc (which can
 * synchronise the device) is not acceptable.  It runs `iters` iterations of
 * `algo` (TVCUT_AAR or TVCUT_AP), the same iteration as tvcut_iterate, on
 * caller-owned DEVICE buffers of element type `dtype` (TVCUT_F32 or
 * TVCUT_F64).  It always takes the fused per-block sweep kernels (one launch
 * per block and iteration), not the all-blocks scan plus separate update that
 * tvcut_iterate uses on large grids, so the two agree within rounding (FP64
 * 1e-9, FP32 1e-4 of max|x| in the tests), not bit for bit, and this path is
 * the slower of the two.  Buffers:
 *   w      n unary values;
 *   a      a[k] = axis k's compact edge weights (k < ndim);
 *   state  ndim*n product-space state (z for AAR, lambda for AP), updated in
 *          place -- start from zeros (AAR) or w/ndim in every block (AP);
 *   x      NULL, or n values that receive the primal of the last iteration
 *          (left unwritten when iters == 0).
 * The one scratch array an iteration needs (a per-vertex running sum) is a
 * fixed 8 MiB array inside the library image, so grids are limited to
 * 2^21 vertices with TVCUT_F32 and 2^20 with TVCUT_F64; larger grids return
 * TVCUT_ERR_INVALID with a message.  Every GPU that loads the library holds
 * those 8 MiB until the process exits.  The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress, with that device
 * current) and caches it; make that first call before any stream capture.
 * All calls share the array: calls that overlap on the GPU race on it.
 * Work is ordered on cuda_stream; the call does not synchronise.  Errors
 * (read with tvcut_last_error(NULL)): INVALID, CUDA. */
tvcut_status tvcut_iterate_noalloc(int ndim, const int64_t* dims, int algo, int dtype,
                                   const void* w, const void* const* a, void* state,
                                   void* x, int64_t iters, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* TVCUT_H */
